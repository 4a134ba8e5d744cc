"""ctypes front end of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the slow, plain definition of the multistep BSDE
scheme (Kapllani & Teng, arXiv:1909.13560, Eq. 20-21, Tables 1-2) that the
CUDA path is checked against.  Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark import this module.  It shares no code with
the product package and never imports it.

Problems are plain dicts (see ``paper_1909_13560_gb300.workloads``); this
module marshals them into its own C struct.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRC2 = os.path.join(_HERE, "oracle2d.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# A prebuilt library used in place of liboracle.so (the mutation tests load
# copies of the oracle with planted mistakes this way).
_LIB_OVERRIDE = os.environ.get("BSDE_ORACLE_LIB")
_lock = threading.Lock()
_lib = None

DRIVERS = {"LIN_SIN": 0, "BS": 1, "LB": 2, "EX1": 3, "EX2": 4, "SHORT_RATE": 5}
TERMINALS = {"SIN": 0, "CALL_LOG": 1, "LOGISTIC": 2, "LNSIN": 3, "ONE": 4, "CALL_PRICE": 5}
FORWARDS = {"CONST": 0, "AFFINE": 1}
INIT_MODES = {"EXACT": 0, "ONESTEP": 1}


class _Problem(ctypes.Structure):
    _fields_ = [
        ("driver", ctypes.c_int), ("terminal", ctypes.c_int),
        ("smoothing", ctypes.c_int), ("picard_max", ctypes.c_int),
        ("T", ctypes.c_double), ("x_min", ctypes.c_double),
        ("x_max", ctypes.c_double), ("x0", ctypes.c_double),
        ("a_x", ctypes.c_double), ("b_x", ctypes.c_double),
        ("r", ctypes.c_double), ("mu", ctypes.c_double),
        ("sigma", ctypes.c_double), ("R", ctypes.c_double),
        ("delta", ctypes.c_double), ("lb_sign", ctypes.c_double),
        ("strike", ctypes.c_double), ("picard_tol", ctypes.c_double),
        ("Nx", ctypes.c_longlong), ("N", ctypes.c_int), ("k", ctypes.c_int),
        ("L", ctypes.c_int), ("kz", ctypes.c_int), ("zform", ctypes.c_int),
        ("init_mode", ctypes.c_int), ("init_substeps", ctypes.c_int),
        ("forward", ctypes.c_int), ("pad_f", ctypes.c_int),
        ("a_1", ctypes.c_double), ("b_1", ctypes.c_double),
    ]


class _Problem2(ctypes.Structure):
    _fields_ = [
        ("driver", ctypes.c_int), ("terminal", ctypes.c_int),
        ("picard_max", ctypes.c_int), ("pad", ctypes.c_int),
        ("T", ctypes.c_double), ("x1_min", ctypes.c_double), ("x1_max", ctypes.c_double),
        ("x2_min", ctypes.c_double), ("x2_max", ctypes.c_double),
        ("x01", ctypes.c_double), ("x02", ctypes.c_double),
        ("a1", ctypes.c_double), ("a2", ctypes.c_double), ("b11", ctypes.c_double),
        ("b21", ctypes.c_double), ("b22", ctypes.c_double),
        ("alpha", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
        ("picard_tol", ctypes.c_double),
        ("Nx1", ctypes.c_longlong), ("Nx2", ctypes.c_longlong),
        ("N", ctypes.c_int), ("k", ctypes.c_int), ("L", ctypes.c_int), ("pad2", ctypes.c_int),
    ]


class _Result2(ctypes.Structure):
    _fields_ = [
        ("y0", ctypes.c_double), ("z0", ctypes.c_double * 2),
        ("picard_resid_max", ctypes.c_double), ("levels_done", ctypes.c_longlong),
        ("status", ctypes.c_int), ("picard_iters_max", ctypes.c_int),
    ]


DRIVERS2 = {"LINEAR": 0}
TERMINALS2 = {"SIN_SUM": 0, "SPREAD_LOG": 1}


class _Result(ctypes.Structure):
    _fields_ = [
        ("y0", ctypes.c_double), ("z0", ctypes.c_double),
        ("picard_resid_max", ctypes.c_double), ("levels_done", ctypes.c_longlong),
        ("status", ctypes.c_int), ("picard_iters_max", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (plain C, FP64, no FMA
    contraction, OpenMP over grid points)."""
    if _LIB_OVERRIDE:
        return _LIB_OVERRIDE
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                                  os.path.getmtime(_SRC2))):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        compile_library(_SRC, _SRC2, tmp)
        os.replace(tmp, _LIB)
        return _LIB


def compile_library(src: str, src2: str, out: str) -> None:
    """Compile the oracle's two C sources into the shared library `out`."""
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", src, src2, "-o", out, "-lm"]
    subprocess.run(cmd, check=True)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d = ctypes.c_double
        lib.orc_gauss_hermite.argtypes = [ctypes.c_int, P(d), P(d)]
        lib.orc_gamma.argtypes = [ctypes.c_int, P(d), P(d)]
        lib.orc_spline.argtypes = [ctypes.c_longlong, d, P(d), P(d)]
        lib.orc_interp.argtypes = [ctypes.c_longlong, d, d, P(d), P(d), d]
        lib.orc_interp.restype = d
        lib.orc_driver.argtypes = [P(_Problem), d, d, d, d]
        lib.orc_driver.restype = d
        lib.orc_exact.argtypes = [P(_Problem), d, d, P(d), P(d)]
        lib.orc_init_levels.argtypes = [P(_Problem), P(d), P(d)]
        lib.orc_expectations.argtypes = [P(_Problem), ctypes.c_int, P(d), P(d),
                                         P(ctypes.c_longlong), ctypes.c_longlong, P(d)]
        lib.orc_solve.argtypes = [P(_Problem), P(d), P(d), ctypes.c_longlong,
                                  P(d), P(d), P(_Result), ctypes.c_int]
        lib.orc_onestep_levels.argtypes = [P(_Problem), P(d), P(d), P(_Result),
                                           ctypes.c_int]
        lib.orc_max_threads.restype = ctypes.c_int
        lib.orc2_derivatives.argtypes = [ctypes.c_longlong, ctypes.c_longlong, P(d), P(d),
                                         P(d), P(d)]
        lib.orc2_interp.argtypes = [P(_Problem2), P(d), P(d), P(d), P(d), d, d]
        lib.orc2_interp.restype = d
        lib.orc2_exact.argtypes = [P(_Problem2), d, d, d, P(d), P(d)]
        lib.orc2_init_levels.argtypes = [P(_Problem2), P(d), P(d), P(d)]
        lib.orc2_solve.argtypes = [P(_Problem2), P(d), P(d), P(d), ctypes.c_longlong,
                                   P(d), P(d), P(d), P(_Result2), ctypes.c_int]
        _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _problem(p: dict) -> _Problem:
    s = _Problem()
    s.driver = DRIVERS[p["driver"]]
    s.terminal = TERMINALS[p["terminal"]]
    s.smoothing = int(p.get("smoothing", 0))
    s.picard_max = int(p.get("picard_max", 30))
    for f in ("T", "x_min", "x_max", "x0", "a_x", "b_x"):
        setattr(s, f, float(p[f]))
    for f in ("r", "mu", "sigma", "R", "delta", "strike"):
        setattr(s, f, float(p.get(f, 0.0)))
    s.lb_sign = float(p.get("lb_sign", 1.0))
    if s.sigma == 0.0:
        s.sigma = 1.0
    s.picard_tol = float(p.get("picard_tol", 1e-12))
    s.Nx = int(p["Nx"])
    s.N = int(p["N"])
    s.k = int(p["k"])
    s.L = int(p["L"])
    s.kz = int(p.get("kz", 0))
    s.zform = int(p.get("zform", 0))
    mode = p.get("init_mode", 0)
    s.init_mode = INIT_MODES[mode] if isinstance(mode, str) else int(mode)
    s.init_substeps = int(p.get("init_substeps", 0))
    fwd = p.get("forward", "CONST")
    s.forward = FORWARDS[fwd] if isinstance(fwd, str) else int(fwd)
    s.a_1 = float(p.get("a_1", 0.0))
    s.b_1 = float(p.get("b_1", 0.0))
    return s


def levels_K(p: dict) -> int:
    """K = max(K_y, K_z): the levels one backward step reads (Eq. 16)."""
    kz = int(p.get("kz", 0)) or int(p["k"])
    return max(int(p["k"]), kz)


def gauss_hermite(L: int):
    lib = _load()
    a = np.zeros(L)
    w = np.zeros(L)
    if lib.orc_gauss_hermite(L, _dptr(a), _dptr(w)) != 0:
        raise ValueError("bad L")
    return a, w


def gamma(K: int):
    lib = _load()
    gy = np.zeros(K + 1)
    gz = np.zeros(K + 1)
    if lib.orc_gamma(K, _dptr(gy), _dptr(gz)) != 0:
        raise ValueError("K out of the tables' range 1..6")
    return gy, gz


def spline(v: np.ndarray, dx: float) -> np.ndarray:
    lib = _load()
    v = np.ascontiguousarray(v, dtype=np.float64)
    M = np.zeros_like(v)
    if lib.orc_spline(len(v), dx, _dptr(v), _dptr(M)) != 0:
        raise ValueError("spline needs at least 2 points")
    return M


def interp(v: np.ndarray, M: np.ndarray, x_min: float, dx: float, X: float) -> float:
    lib = _load()
    v = np.ascontiguousarray(v, dtype=np.float64)
    M = np.ascontiguousarray(M, dtype=np.float64)
    return lib.orc_interp(len(v), x_min, dx, _dptr(v), _dptr(M), float(X))


def driver(p: dict, t: float, y: float, z: float, x: float = 0.0) -> float:
    lib = _load()
    s = _problem(p)
    return lib.orc_driver(ctypes.byref(s), t, x, y, z)


def exact(p: dict, t: float, x: float):
    lib = _load()
    s = _problem(p)
    u = ctypes.c_double()
    z = ctypes.c_double()
    if lib.orc_exact(ctypes.byref(s), t, x, ctypes.byref(u), ctypes.byref(z)) != 0:
        raise ValueError("no closed form for this terminal id")
    return u.value, z.value


def init_levels(p: dict):
    """Closed-form levels N..N-K+1 (rows 0..K-1), level N smoothed when the
    problem asks for it."""
    lib = _load()
    s = _problem(p)
    K = levels_K(p)
    iy = np.zeros((K, s.Nx))
    iz = np.zeros((K, s.Nx))
    if lib.orc_init_levels(ctypes.byref(s), _dptr(iy), _dptr(iz)) != 0:
        raise ValueError("no closed form for this problem")
    return iy, iz


def onestep_levels(p: dict, threads: int = 1):
    """Levels N..N-K+1 by the one-step start-up (Section 3.1 step 2) with
    p["init_substeps"] steps of the 1-step scheme per dt."""
    lib = _load()
    s = _problem(p)
    K = levels_K(p)
    iy = np.zeros((K, s.Nx))
    iz = np.zeros((K, s.Nx))
    res = _Result()
    if lib.orc_onestep_levels(ctypes.byref(s), _dptr(iy), _dptr(iz), ctypes.byref(res),
                              int(threads)) != 0:
        raise ValueError("bad problem or init_substeps < 1")
    return iy, iz


def expectations(p: dict, n: int, levels_y: np.ndarray, levels_z: np.ndarray,
                 idx) -> np.ndarray:
    """E_j[z^], E_j[f], E_j[f dW], E_j[y^], E_j[y^ dW] (j = 1..K) at grid
    points idx for level n; row j-1 of levels_* is level n+j.
    Returns an array of shape (len(idx), K, 5)."""
    lib = _load()
    s = _problem(p)
    ly = np.ascontiguousarray(levels_y, dtype=np.float64)
    lz = np.ascontiguousarray(levels_z, dtype=np.float64)
    ix = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    out = np.zeros((len(ix), levels_K(p), 5))
    rc = lib.orc_expectations(ctypes.byref(s), int(n), _dptr(ly), _dptr(lz),
                              ix.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                              len(ix), _dptr(out))
    if rc != 0:
        raise ValueError("bad problem")
    return out


def solve(p: dict, init_y=None, init_z=None, levels: int = 0, threads: int = 1,
          want_level: bool = False) -> dict:
    """Run the backward loop.  Returns y0, z0 (readout at x0 of the last
    computed level), Picard statistics and, if asked, that level's arrays."""
    lib = _load()
    s = _problem(p)
    res = _Result()
    iy = iz = None
    if init_y is not None:
        iy = np.ascontiguousarray(init_y, dtype=np.float64)
        iz = np.ascontiguousarray(init_z, dtype=np.float64)
        K = levels_K(p)
        if iy.shape != (K, s.Nx) or iz.shape != (K, s.Nx):
            raise ValueError("initial levels must have shape (K, Nx), K = max(k, kz)")
    oy = np.zeros(s.Nx) if want_level else None
    oz = np.zeros(s.Nx) if want_level else None
    rc = lib.orc_solve(ctypes.byref(s),
                       _dptr(iy) if iy is not None else None,
                       _dptr(iz) if iz is not None else None,
                       int(levels),
                       _dptr(oy) if oy is not None else None,
                       _dptr(oz) if oz is not None else None,
                       ctypes.byref(res), int(threads))
    if rc != 0:
        raise ValueError(f"oracle rejected the problem (rc={rc})")
    out = {"y0": res.y0, "z0": res.z0, "status": res.status,
           "picard_iters_max": res.picard_iters_max,
           "picard_resid_max": res.picard_resid_max,
           "levels_done": res.levels_done}
    if want_level:
        out["y"] = oy
        out["z"] = oz
    return out


def max_threads() -> int:
    return int(_load().orc_max_threads())


# --- two space dimensions (oracle2d.c) --------------------------------------

def _problem2(p: dict) -> _Problem2:
    s = _Problem2()
    s.driver = DRIVERS2[p["driver"]]
    s.terminal = TERMINALS2[p["terminal"]]
    s.picard_max = int(p.get("picard_max", 30))
    for f in ("T", "x1_min", "x1_max", "x2_min", "x2_max", "x01", "x02", "a1", "a2",
              "b11", "b21", "b22", "alpha", "beta1", "beta2"):
        setattr(s, f, float(p[f]))
    s.picard_tol = float(p.get("picard_tol", 1e-12))
    s.Nx1, s.Nx2 = int(p["Nx1"]), int(p["Nx2"])
    s.N, s.k, s.L = int(p["N"]), int(p["k"]), int(p["L"])
    return s


def derivatives2(v: np.ndarray):
    """Scaled fourth-order finite-difference derivatives (fx, fy, fxy) of a
    field v of shape (Nx2, Nx1) (x1 fastest)."""
    lib = _load()
    v = np.ascontiguousarray(v, dtype=np.float64)
    fx, fy, fxy = np.zeros_like(v), np.zeros_like(v), np.zeros_like(v)
    if lib.orc2_derivatives(v.shape[1], v.shape[0], _dptr(v), _dptr(fx), _dptr(fy),
                            _dptr(fxy)) != 0:
        raise ValueError("a line needs at least 6 points")
    return fx, fy, fxy


def interp2(p: dict, v, fx, fy, fxy, X1: float, X2: float) -> float:
    lib = _load()
    s = _problem2(p)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (v, fx, fy, fxy)]
    return lib.orc2_interp(ctypes.byref(s), *[_dptr(a) for a in arrs], float(X1), float(X2))


def exact2(p: dict, t: float, x1: float, x2: float):
    lib = _load()
    s = _problem2(p)
    u = ctypes.c_double()
    z = (ctypes.c_double * 2)()
    if lib.orc2_exact(ctypes.byref(s), t, x1, x2, ctypes.byref(u), z) != 0:
        raise ValueError("no closed form")
    return u.value, (z[0], z[1])


def init_levels2(p: dict):
    lib = _load()
    s = _problem2(p)
    shape = (s.k, s.Nx2, s.Nx1)
    iy, iz1, iz2 = np.zeros(shape), np.zeros(shape), np.zeros(shape)
    if lib.orc2_init_levels(ctypes.byref(s), _dptr(iy), _dptr(iz1), _dptr(iz2)) != 0:
        raise ValueError("no closed form")
    return iy, iz1, iz2


def solve2(p: dict, init=None, levels: int = 0, threads: int = 1,
           want_level: bool = False) -> dict:
    """The two-dimensional backward loop.  init: None (closed form) or
    (y, z1, z2), each (k, Nx2, Nx1).  Returns y0, z0 = (z1, z2) at (x01, x02)
    and, if asked, the last level's fields of shape (Nx2, Nx1)."""
    lib = _load()
    s = _problem2(p)
    res = _Result2()
    ptrs = [None, None, None]
    keep = []
    if init is not None:
        for q, a in enumerate(init):
            a = np.ascontiguousarray(a, dtype=np.float64)
            if a.shape != (s.k, s.Nx2, s.Nx1):
                raise ValueError("initial levels must have shape (k, Nx2, Nx1)")
            keep.append(a)
            ptrs[q] = _dptr(a)
    outs = [np.zeros((s.Nx2, s.Nx1)) for _ in range(3)] if want_level else [None] * 3
    rc = lib.orc2_solve(ctypes.byref(s), ptrs[0], ptrs[1], ptrs[2], int(levels),
                        *[(_dptr(o) if o is not None else None) for o in outs],
                        ctypes.byref(res), int(threads))
    if rc != 0:
        raise ValueError(f"oracle rejected the problem (rc={rc})")
    out = {"y0": res.y0, "z0": (res.z0[0], res.z0[1]), "status": res.status,
           "picard_iters_max": res.picard_iters_max,
           "picard_resid_max": res.picard_resid_max, "levels_done": res.levels_done}
    if want_level:
        out["y"], out["z1"], out["z2"] = outs
    return out
