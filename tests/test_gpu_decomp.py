"""The domain decomposition of one problem on the real kernels: the problem
solved as 2..5 slabs with halo exchange after every step (LocalTransport, all
slabs on one GPU) against the same problem as one plan, level 0 compared
point by point, both precisions, closed-form and caller start."""
import numpy as np
import pytest

from paper_1909_13560_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_13560_gb300 import bsde
    bsde.load()
    return bsde


CASES = {
    "call_k3": (W.call_problem(Nx=8192, N=32, k=3), [2, 3, 5]),
    "sin_k2": (W.sin_problem(Nx=6001, N=24, k=2, L=8), [2, 4]),
    "lb_k2": (W.config3(Nx=1 << 15, N=64, k=2), [2, 4]),
}


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32c", 1e-7)])
@pytest.mark.parametrize("name", list(CASES))
def test_sharded_equals_unsharded(B, name, prec, tol):
    from paper_1909_13560_gb300 import decomp
    p, parts_list = CASES[name]
    ref = B.solve(p, prec, want_level=True)
    for parts in parts_list:
        got = decomp.solve_sharded(p, parts, prec, want_level=True)
        scale = max(1.0, float(np.max(np.abs(ref["y"]))))
        zs = max(1.0, float(np.max(np.abs(ref["z"]))))
        ey = float(np.max(np.abs(got["y"] - ref["y"])))
        ez = float(np.max(np.abs(got["z"] - ref["z"])))
        print(f"{name} {prec} parts={parts} halo={decomp.halo_width(p)}: "
              f"max|dy|={ey:.2e} max|dz|={ez:.2e} dy0={abs(got['y0'] - ref['y0']):.2e}")
        assert ey <= tol * scale and ez <= tol * zs
        assert abs(got["y0"] - ref["y0"]) <= tol * scale
        assert abs(got["z0"] - ref["z0"]) <= tol * zs
        assert got["levels_done"] == ref["levels_done"]


def test_sharded_with_caller_levels(B):
    from paper_1909_13560_gb300 import decomp
    p = W.call_problem(Nx=8192, N=32, k=3)
    iy, iz = W.initial_levels(p)
    iy = iy * (1.0 + 1e-3 * np.sin(np.arange(p["Nx"]) / 50.0))
    ref = B.solve(p, "fp64", init=(iy, iz), want_level=True)
    got = decomp.solve_sharded(p, 3, "fp64", want_level=True, init=(iy, iz))
    assert float(np.max(np.abs(got["y"] - ref["y"]))) <= 1e-12 * float(np.max(np.abs(ref["y"])))


def test_sharded_graph_replay_equals_direct(B):
    """The level loop captured into a CUDA graph and replayed gives the
    directly launched result."""
    import torch
    from paper_1909_13560_gb300 import decomp
    p = W.call_problem(Nx=8192, N=32, k=3)
    ss = decomp.ShardedSolver(p, 3, "fp32c")
    stream = torch.cuda.current_stream()
    ss.enqueue(stream)
    a = ss.result(stream)
    ss.replay(stream)
    ss.replay(stream)
    b = ss.result(stream)
    ss.close()
    assert a["y0"] == b["y0"] and a["z0"] == b["z0"]
