"""The no-allocation entry point, bsde_solve_noalloc, through the C ABI.

Callers that may not allocate device memory while solving (an application
that owns the GPU through its own allocator, a latency-critical loop where
an allocation would stall the device) use this entry point; it runs the same
kernels as bsde_solve on a fixed workspace that the library reserves once.
This test checks its output against the planned entry point (bsde_plan +
bsde_solve) within the tolerances of the parity tests, on two calls in a row
(the second reuses the array the first one left behind), and that a problem
too large for the fixed workspace is refused.  The file sorts last so that a
run stopping at the first failure has already run every other test; it also
passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_1909_13560_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32c": 2e-7}


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_13560_gb300 import bsde
    bsde.load()
    return bsde


def _noalloc(B, p, prec, init=None):
    import torch
    prob = B.make_problem(p, prec)
    nx = int(p["Nx"])
    oy, oz = np.zeros(nx), np.zeros(nx)
    iy = iz = 0
    keep = []
    if init is not None:
        a = np.ascontiguousarray(init[0], dtype=np.float64)
        b = np.ascontiguousarray(init[1], dtype=np.float64)
        keep += [a, b]
        iy, iz = a.ctypes.data, b.ctypes.data
    stream = torch.cuda.current_stream().cuda_stream
    r = B.bsde_solve_noalloc(prob, stream, iy, iz, init is not None,
                             oy.ctypes.data, oz.ctypes.data, True)
    return {"y0": r.y0, "z0": r.z0, "y": oy, "z": oz, "status": r.status,
            "picard_iters_max": r.picard_iters_max}


def _check(got, ref, tol, what):
    scale = max(1.0, float(np.max(np.abs(ref["y"]))))
    zscale = max(1.0, float(np.max(np.abs(ref["z"]))))
    ey = float(np.max(np.abs(got["y"] - ref["y"])))
    ez = float(np.max(np.abs(got["z"] - ref["z"])))
    print(f"{what}: max|dy|={ey:.3e} max|dz|={ez:.3e}")
    assert ey <= tol * scale and ez <= tol * zscale, what
    assert abs(got["y0"] - ref["y0"]) <= tol * scale, what
    assert abs(got["z0"] - ref["z0"]) <= tol * zscale, what
    assert got["status"] == ref["status"]


def test_noalloc_matches_planned_solve_on_consecutive_calls(B):
    calls = [
        (W.call_problem(Nx=4096, N=48, k=4), "fp64", None),
        (W.sin_problem(Nx=1537, N=24, k=3, L=12), "fp32c", None),
    ]
    # a third call with caller-supplied initial levels, smaller than the
    # previous ones, over the array the earlier calls filled
    p3 = W.sin_problem(Nx=700, N=10, k=2, L=8)
    calls.append((p3, "fp64", W.initial_levels(p3)))
    # the one-step start-up (Section 3.1 step 2): its own node tables and the
    # sub-run regions of the array
    p4 = dict(W.call_problem(Nx=1000, N=16, k=3), init_mode="ONESTEP", init_substeps=2)
    calls.append((p4, "fp32c", None))
    for i, (p, prec, init) in enumerate(calls):
        got = _noalloc(B, p, prec, init)
        ref = B.solve(p, prec, init=init, want_level=True)
        _check(got, ref, TOL[prec], f"call {i + 1} {prec} Nx={p['Nx']}")


def test_noalloc_refuses_problems_beyond_the_fixed_workspace(B):
    import torch
    p = W.config3()  # Nx = 2^20: ~170 MB of workspace
    prob = B.make_problem(p, "fp64")
    assert B.bsde_workspace_bytes(prob) > (32 << 20)
    with pytest.raises(B.BsdeError) as ei:
        B.bsde_solve_noalloc(prob, torch.cuda.current_stream().cuda_stream)
    assert ei.value.code == B.BSDE_ENOSPC
    assert "no-allocation workspace" in str(ei.value)
