"""Host-side checks of the CUDA library: it builds, loads without a GPU,
exports every entry point include/bsde.h declares, and its host-computed plan
constants are right.  No kernel is launched here."""
import ctypes
import math
import os
import re
from fractions import Fraction

import numpy as np
import pytest

from paper_1909_13560_gb300 import bsde as B
from paper_1909_13560_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"BSDE_API\s+[\w\s\*]+?\b(\w+)\s*\(", text)
    return names


def test_header_declares_the_abi():
    names = _declared()
    for n in ("bsde_plan", "bsde_solve", "bsde_free", "bsde_workspace_bytes"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = B.load()
    for name in _declared():
        assert hasattr(lib, name), name
        assert getattr(lib, name) is not None


def test_binding_structs_match_header_layout(tmp_path):
    """Compile a probe against include/bsde.h with the host C compiler and
    compare sizes and offsets with the ctypes mirror."""
    import subprocess
    src = tmp_path / "probe.c"
    fields_p = [f for f, _ in B.bsde_problem._fields_]
    fields_r = [f for f, _ in B.bsde_result._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bsde.h"', 'int main(void){',
             'printf("%zu %zu\\n", sizeof(bsde_problem), sizeof(bsde_result));']
    lines += [f'printf("%zu\\n", offsetof(bsde_problem, {f}));' for f in fields_p]
    lines += [f'printf("%zu\\n", offsetof(bsde_result, {f}));' for f in fields_r]
    lines += ['return 0;}']
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    vals = [int(v) for v in out]
    assert vals[0] == ctypes.sizeof(B.bsde_problem)
    assert vals[1] == ctypes.sizeof(B.bsde_result)
    offs = vals[2:]
    for f, o in zip(fields_p, offs[:len(fields_p)]):
        assert getattr(B.bsde_problem, f).offset == o, f
    for f, o in zip(fields_r, offs[len(fields_p):]):
        assert getattr(B.bsde_result, f).offset == o, f


@pytest.mark.parametrize("L", [1, 2, 5, 8, 16, 32, 64])
def test_device_plan_gauss_hermite(L):
    a, w = B.bsde_gauss_hermite(L)
    ra, rw = np.polynomial.hermite.hermgauss(L)
    assert np.max(np.abs(a - ra)) <= 1e-13 * max(1.0, np.abs(ra).max())
    assert np.max(np.abs(w - rw) / rw) <= 2e-12
    for p in range(0, 2 * L, 2):
        assert float(np.sum(w * a ** p)) == pytest.approx(math.gamma((p + 1) / 2), rel=1e-12)


@pytest.mark.parametrize("k", range(1, 7))
def test_device_plan_gamma_tables(k):
    gy, gz = B.bsde_gamma(k)
    # exact sums and the closed forms of the small cases (trapezoid, Simpson,
    # Simpson 3/8, Adams-Moulton in Table 2)
    assert sum(Fraction(x).limit_denominator(2000) for x in gy) == 1
    assert sum(Fraction(x).limit_denominator(2000) for x in gz) == 1
    known_y = {1: [1 / 2, 1 / 2], 2: [1 / 6, 2 / 3, 1 / 6], 3: [1 / 8, 3 / 8, 3 / 8, 1 / 8]}
    known_z = {1: [1 / 2, 1 / 2], 2: [5 / 12, 8 / 12, -1 / 12],
               3: [9 / 24, 19 / 24, -5 / 24, 1 / 24]}
    if k in known_y:
        assert np.allclose(gy, known_y[k], rtol=0, atol=1e-16)
        assert np.allclose(gz, known_z[k], rtol=0, atol=1e-16)


def test_gamma_rejects_k_beyond_tables():
    with pytest.raises(B.BsdeError):
        B.bsde_gamma(7)


@pytest.mark.parametrize("bad", [dict(k=7), dict(k=5, N=4), dict(Nx=3), dict(L=0),
                                 dict(L=65), dict(x0=9.0), dict(T=0.0),
                                 dict(picard_max=0)])
def test_invalid_problems_rejected(bad):
    p = W.sin_problem()
    p.update(bad)
    with pytest.raises(B.BsdeError) as ei:
        B.bsde_workspace_bytes(B.make_problem(p))
    assert ei.value.code == B.BSDE_EINVAL


def test_workspace_bytes_scale_with_ring():
    p = W.config2(k=6)
    b64 = B.bsde_workspace_bytes(B.make_problem(p, "fp64"))
    b32 = B.bsde_workspace_bytes(B.make_problem(p, "fp32c"))
    nx, ns = p["Nx"], p["k"] + 1
    # FP64: (y, M_y, z, M_z) per node; FP32C: (y_hi, z_hi, y_lo, z_lo) per node
    # plus the second derivatives (M_y, M_z)
    assert ns * nx * 32 <= b64 < ns * nx * 32 + (8 << 20)
    assert ns * nx * 24 <= b32 < ns * nx * 24 + (8 << 20)


@pytest.mark.parametrize("bad", [dict(kz=7), dict(kz=-1), dict(kz=6, N=5), dict(zform=2),
                                 dict(init_mode=2), dict(init_mode=1, init_substeps=0),
                                 dict(init_mode=1, init_substeps=1 << 25),
                                 dict(step_kernel=3), dict(step_kernel=-1)])
def test_invalid_variants_rejected(bad):
    p = W.sin_problem()
    p.update(bad)
    with pytest.raises(B.BsdeError) as ei:
        B.bsde_workspace_bytes(B.make_problem(p))
    assert ei.value.code == B.BSDE_EINVAL


def test_workspace_bytes_of_the_variants():
    """K_z widens the ring to max(k, kz) + 1 slots; the one-step start-up adds
    a ring of two slots (and its small node tables), the z form nothing."""
    p = W.call_problem(Nx=1 << 16, N=64, k=2)
    for prec, per_node in (("fp64", 32), ("fp32c", 24)):
        base = B.bsde_workspace_bytes(B.make_problem(p, prec))
        wide = B.bsde_workspace_bytes(B.make_problem(dict(p, kz=5), prec))
        zf = B.bsde_workspace_bytes(B.make_problem(dict(p, zform=1), prec))
        one = B.bsde_workspace_bytes(B.make_problem(dict(p, init_mode="ONESTEP",
                                                         init_substeps=4), prec))
        nx = p["Nx"]
        assert zf == base
        # 3 more ring slots and 3 more rows of the staging area (2 x 8 B per node)
        assert wide - base >= 3 * nx * (per_node + 16)
        assert 2 * nx * per_node <= one - base < 2 * nx * per_node + (1 << 16)
        # K = 1 has nothing to start up
        k1 = dict(p, k=1)
        assert (B.bsde_workspace_bytes(B.make_problem(dict(k1, init_mode="ONESTEP",
                                                           init_substeps=4), prec))
                == B.bsde_workspace_bytes(B.make_problem(k1, prec)))


def test_batch_and_server_reject_the_startup():
    p = dict(W.call_problem(Nx=1024, N=32, k=3), init_mode="ONESTEP", init_substeps=2)
    with pytest.raises(B.BsdeError):
        B.bsde_batch_workspace_bytes([p])
    n = ctypes.c_size_t()
    assert B.load().bsde_request_bytes(ctypes.byref(B.make_problem(p, "fp32c")),
                                       ctypes.byref(n)) == B.BSDE_EINVAL
    # the variants without a start-up are accepted
    B.bsde_batch_workspace_bytes([dict(p, init_mode="EXACT", kz=4, zform=1)])


def test_binding_2d_structs_match_header_layout(tmp_path):
    import subprocess
    src = tmp_path / "probe2.c"
    fp = [f for f, _ in B.bsde2_problem._fields_]
    fr = [f for f, _ in B.bsde2_result._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bsde2d.h"', 'int main(void){',
             'printf("%zu %zu\\n", sizeof(bsde2_problem), sizeof(bsde2_result));']
    lines += [f'printf("%zu\\n", offsetof(bsde2_problem, {f}));' for f in fp]
    lines += [f'printf("%zu\\n", offsetof(bsde2_result, {f}));' for f in fr]
    lines += ['return 0;}']
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe2"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                            text=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(B.bsde2_problem)
    assert vals[1] == ctypes.sizeof(B.bsde2_result)
    for f, o in zip(fp + fr, vals[2:]):
        cls = B.bsde2_problem if f in fp else B.bsde2_result
        assert getattr(cls, f).offset == o, f


@pytest.mark.parametrize("bad", [dict(k=7), dict(k=9, N=8), dict(Nx1=5), dict(L=0), dict(L=17),
                                 dict(x01=9.0), dict(T=0.0), dict(picard_max=0)])
def test_invalid_2d_problems_rejected(bad):
    p = W.ex4_problem()
    p.update(bad)
    with pytest.raises(B.BsdeError) as ei:
        B.bsde2_workspace_bytes(B.make_problem2(p))
    assert ei.value.code == B.BSDE_EINVAL


def test_invalid_2d_step_forms_rejected():
    # the tensor-product passes need an uncorrelated forward process
    p = dict(W.ex5_problem(rho=0.5), step_form="TENSOR")
    with pytest.raises(B.BsdeError) as ei:
        B.bsde2_workspace_bytes(B.make_problem2(p))
    assert ei.value.code == B.BSDE_EINVAL
    for bad in (-1, 3):
        s = B.make_problem2(W.ex4_problem())
        s.step_form = bad
        with pytest.raises(B.BsdeError) as ei:
            B.bsde2_workspace_bytes(s)
        assert ei.value.code == B.BSDE_EINVAL


def test_2d_workspace_bytes():
    p = W.ex4_problem(M=1024, N=64, k=6)
    np_ = 1025 * 1025
    # ring 7 x 3 x 32 B, new values 24 B, staging 6 x 24 B per point
    base = 7 * 96 * np_ + 24 * np_ + 6 * 24 * np_
    b = B.bsde2_workspace_bytes(B.make_problem2(dict(p, step_form="NODEWISE")))
    assert base <= b < base + (1 << 20)
    # the tensor form (the default for b21 = 0) adds the x2 pass's buffer of
    # k records per point: 96 B in FP64, 64 B in FP32C
    for form in ("AUTO", "TENSOR"):
        b = B.bsde2_workspace_bytes(B.make_problem2(dict(p, step_form=form)))
        assert base + 6 * 96 * np_ <= b < base + 6 * 96 * np_ + (1 << 20)
    b32 = B.bsde2_workspace_bytes(B.make_problem2(p, precision="fp32c"))
    base32 = 7 * 64 * np_ + 24 * np_ + 6 * 24 * np_
    assert base32 + 6 * 64 * np_ <= b32 < base32 + 6 * 64 * np_ + (1 << 20)
    # a correlated process keeps the node-wise form under AUTO
    b5 = B.bsde2_workspace_bytes(B.make_problem2(W.ex5_problem(M=1024, N=64, k=6, rho=0.5)))
    assert base <= b5 < base + (1 << 20)


@pytest.mark.parametrize("bad", [
    dict(W.vasicek_problem(), a_1=0.1),
    dict(W.vasicek_problem(), b_1=0.01),
    dict(W.vasicek_problem(), forward="CONST"),
    dict(W.gbm_call_problem(), x_min=-1.0),
    dict(W.gbm_call_problem(), b_x=0.1),
    dict(W.sin_problem(), forward=2),
])
def test_invalid_general_forward_problems_rejected(bad):
    p = dict(bad)
    prec = "fp32c" if p.pop("precision_fp32c", False) else "fp64"
    with pytest.raises(B.BsdeError) as ei:
        B.bsde_workspace_bytes(B.make_problem(p, prec))
    assert ei.value.code == B.BSDE_EINVAL


def test_general_forward_problems_accepted():
    for p in (W.vasicek_problem(), W.gbm_call_problem(),
              dict(W.sin_problem(), driver="SHORT_RATE")):
        for prec in ("fp64", "fp32c"):
            assert B.bsde_workspace_bytes(B.make_problem(p, prec)) > 0
    # batches and the server run the constant-shift kernels only
    with pytest.raises(B.BsdeError):
        B.bsde_batch_workspace_bytes([W.vasicek_problem()])
