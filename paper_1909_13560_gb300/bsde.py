"""Python binding of the C ABI in include/bsde.h (argument marshalling only).

Every step of the solve runs in the CUDA kernels of libbsde.so; PyTorch is
used for device memory (the workspace) and streams.  Importing this module
does not touch the GPU; the first call loads the library and raises if it is
missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbsde.so")

BSDE_DRIVER = {"LIN_SIN": 0, "BS": 1, "LB": 2, "EX1": 3, "EX2": 4, "SHORT_RATE": 5}
BSDE_TERMINAL = {"SIN": 0, "CALL_LOG": 1, "LOGISTIC": 2, "LNSIN": 3, "ONE": 4, "CALL_PRICE": 5}
BSDE_FORWARD = {"CONST": 0, "AFFINE": 1}
BSDE_PRECISION = {"fp64": 0, "fp32c": 1}
BSDE_INIT = {"EXACT": 0, "ONESTEP": 1}
BSDE_STEP = {"AUTO": 0, "GROUPED": 1, "FLAT": 2}
BSDE_ZFORM = {"EZ": 0, "EYDW": 1}
BSDE2_STEP = {"AUTO": 0, "NODEWISE": 1, "TENSOR": 2}

BSDE_OK = 0
BSDE_WARN_NOCONV = 1
BSDE_BUSY = 2
BSDE_EINVAL = -1
BSDE_ENOSPC = -2
BSDE_ECUDA = -3
BSDE_ENOMEM = -4
BSDE_ETIMEOUT = -5


class bsde_problem(ctypes.Structure):
    _fields_ = [
        ("driver", ctypes.c_int32), ("terminal", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("smoothing", ctypes.c_int32),
        ("picard_max", ctypes.c_int32), ("N", ctypes.c_int32),
        ("k", ctypes.c_int32), ("L", ctypes.c_int32),
        ("Nx", ctypes.c_int64),
        ("T", ctypes.c_double), ("x_min", ctypes.c_double),
        ("x_max", ctypes.c_double), ("x0", ctypes.c_double),
        ("a_x", ctypes.c_double), ("b_x", ctypes.c_double),
        ("r", ctypes.c_double), ("mu", ctypes.c_double),
        ("sigma", ctypes.c_double), ("R", ctypes.c_double),
        ("delta", ctypes.c_double), ("lb_sign", ctypes.c_double),
        ("strike", ctypes.c_double), ("picard_tol", ctypes.c_double),
        ("k_z", ctypes.c_int32), ("z_form", ctypes.c_int32),
        ("init_mode", ctypes.c_int32), ("init_substeps", ctypes.c_int32),
        ("forward", ctypes.c_int32), ("step_kernel", ctypes.c_int32),
        ("a_1", ctypes.c_double), ("b_1", ctypes.c_double),
    ]


class bsde2_problem(ctypes.Structure):
    _fields_ = [
        ("driver", ctypes.c_int32), ("terminal", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("picard_max", ctypes.c_int32),
        ("N", ctypes.c_int32), ("k", ctypes.c_int32), ("L", ctypes.c_int32),
        ("step_form", ctypes.c_int32),
        ("Nx1", ctypes.c_int64), ("Nx2", ctypes.c_int64),
        ("T", ctypes.c_double), ("x1_min", ctypes.c_double), ("x1_max", ctypes.c_double),
        ("x2_min", ctypes.c_double), ("x2_max", ctypes.c_double),
        ("x01", ctypes.c_double), ("x02", ctypes.c_double),
        ("a1", ctypes.c_double), ("a2", ctypes.c_double), ("b11", ctypes.c_double),
        ("b21", ctypes.c_double), ("b22", ctypes.c_double),
        ("alpha", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
        ("picard_tol", ctypes.c_double),
    ]


class bsde2_result(ctypes.Structure):
    _fields_ = [
        ("y0", ctypes.c_double), ("z0", ctypes.c_double * 2),
        ("picard_resid_max", ctypes.c_double), ("status", ctypes.c_int32),
        ("picard_iters_max", ctypes.c_int32), ("levels_done", ctypes.c_int64),
    ]


BSDE2_DRIVER = {"LINEAR": 0}
BSDE2_TERMINAL = {"SIN_SUM": 0, "SPREAD_LOG": 1}


class bsde_batch_config(ctypes.Structure):
    _fields_ = [("cluster", ctypes.c_int32), ("target_groups", ctypes.c_int32),
                ("flat_tiles", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]


class bsde_result(ctypes.Structure):
    _fields_ = [
        ("y0", ctypes.c_double), ("z0", ctypes.c_double),
        ("picard_resid_max", ctypes.c_double),
        ("status", ctypes.c_int32), ("picard_iters_max", ctypes.c_int32),
        ("levels_done", ctypes.c_int64),
    ]


_lib = None
_SYMBOLS = ("bsde_workspace_bytes", "bsde_plan", "bsde_solve", "bsde_result_fetch",
            "bsde_enqueue_level", "bsde_free", "bsde_plan_launches", "bsde_strerror",
            "bsde_last_error", "bsde_gauss_hermite", "bsde_gamma", "bsde_solve_noalloc",
            "bsde_batch_workspace_bytes", "bsde_plan_batch", "bsde_batch_set_config",
            "bsde_batch_get_config", "bsde_batch_autotune", "bsde_solve_batch", "bsde_batch_free",
            "bsde_request_bytes", "bsde_server_workspace_bytes", "bsde_server_create",
            "bsde_server_start", "bsde_server_submit", "bsde_server_poll", "bsde_server_stop",
            "bsde_server_free", "bsde_l2_read_probe", "bsde_fma_probe",
            "bsde2_workspace_bytes", "bsde2_plan", "bsde2_solve", "bsde2_result_fetch",
            "bsde2_enqueue_level", "bsde2_plan_launches", "bsde2_free",
            "bsde_enqueue_start", "bsde_enqueue_finish", "bsde_level_records")


def load(path: str = LIB_PATH):
    """Load libbsde.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    if _build._stale():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing and could not be built")
    lib = ctypes.CDLL(path)
    P, vp = ctypes.POINTER, ctypes.c_void_p
    d = ctypes.c_double
    lib.bsde_workspace_bytes.argtypes = [P(bsde_problem), P(ctypes.c_size_t)]
    lib.bsde_plan.argtypes = [P(bsde_problem), vp, ctypes.c_size_t, P(vp)]
    lib.bsde_solve.argtypes = [vp, vp, vp, vp, ctypes.c_int, vp, vp, ctypes.c_int,
                               P(bsde_result)]
    lib.bsde_result_fetch.argtypes = [vp, vp, P(bsde_result)]
    lib.bsde_enqueue_level.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int]
    lib.bsde_free.argtypes = [vp]
    lib.bsde_free.restype = None
    lib.bsde_plan_launches.argtypes = [vp]
    lib.bsde_plan_launches.restype = ctypes.c_int64
    lib.bsde_strerror.argtypes = [ctypes.c_int]
    lib.bsde_strerror.restype = ctypes.c_char_p
    lib.bsde_last_error.restype = ctypes.c_char_p
    lib.bsde_gauss_hermite.argtypes = [ctypes.c_int, P(d), P(d)]
    lib.bsde_gamma.argtypes = [ctypes.c_int, P(d), P(d)]
    lib.bsde_solve_noalloc.argtypes = [P(bsde_problem), vp, vp, vp, ctypes.c_int, vp, vp,
                                       ctypes.c_int, P(bsde_result)]
    lib.bsde_batch_workspace_bytes.argtypes = [ctypes.c_int, P(bsde_problem), P(ctypes.c_size_t)]
    lib.bsde_plan_batch.argtypes = [ctypes.c_int, P(bsde_problem), vp, ctypes.c_size_t, P(vp)]
    lib.bsde_batch_set_config.argtypes = [vp, P(bsde_batch_config)]
    lib.bsde_batch_get_config.argtypes = [vp, P(bsde_batch_config)]
    lib.bsde_batch_autotune.argtypes = [vp, vp, P(bsde_batch_config)]
    lib.bsde_solve_batch.argtypes = [vp, vp, P(bsde_result)]
    lib.bsde_batch_free.argtypes = [vp]
    lib.bsde_batch_free.restype = None
    lib.bsde_request_bytes.argtypes = [P(bsde_problem), P(ctypes.c_size_t)]
    lib.bsde_server_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_size_t, P(ctypes.c_size_t)]
    lib.bsde_server_create.argtypes = [vp, ctypes.c_size_t, ctypes.c_int, ctypes.c_size_t, P(vp)]
    lib.bsde_server_start.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int]
    lib.bsde_server_submit.argtypes = [vp, P(bsde_problem), P(ctypes.c_int)]
    lib.bsde_server_poll.argtypes = [vp, ctypes.c_int, P(ctypes.c_int), P(bsde_result)]
    lib.bsde_server_stop.argtypes = [vp]
    lib.bsde_server_free.argtypes = [vp]
    lib.bsde_server_free.restype = None
    lib.bsde_l2_read_probe.argtypes = [vp, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, vp, vp]
    lib.bsde_fma_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp,
                                   P(ctypes.c_int64)]
    lib.bsde2_workspace_bytes.argtypes = [P(bsde2_problem), P(ctypes.c_size_t)]
    lib.bsde2_plan.argtypes = [P(bsde2_problem), vp, ctypes.c_size_t, P(vp)]
    lib.bsde2_solve.argtypes = [vp, vp, vp, vp, vp, ctypes.c_int, vp, vp, vp, ctypes.c_int,
                                P(bsde2_result)]
    lib.bsde2_result_fetch.argtypes = [vp, vp, P(bsde2_result)]
    lib.bsde2_enqueue_level.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int]
    lib.bsde2_plan_launches.argtypes = [vp]
    lib.bsde2_plan_launches.restype = ctypes.c_int64
    lib.bsde2_free.argtypes = [vp]
    lib.bsde2_free.restype = None
    lib.bsde_enqueue_start.argtypes = [vp, vp, vp, vp, ctypes.c_int]
    lib.bsde_enqueue_finish.argtypes = [vp, vp, vp, vp, ctypes.c_int]
    lib.bsde_level_records.argtypes = [vp, ctypes.c_int, P(vp), P(ctypes.c_size_t)]
    _lib = lib
    return lib


class BsdeError(RuntimeError):
    def __init__(self, code: int, what: str):
        lib = load()
        msg = f"{what}: {lib.bsde_strerror(code).decode()} ({code})"
        detail = lib.bsde_last_error().decode()
        if detail:
            msg += f": {detail}"
        super().__init__(msg)
        self.code = code


def _check(code: int, what: str) -> int:
    if code < 0:
        raise BsdeError(code, what)
    return code


def make_problem(p: dict, precision: str = "fp64") -> bsde_problem:
    s = bsde_problem()
    s.driver = BSDE_DRIVER[p["driver"]]
    s.terminal = BSDE_TERMINAL[p["terminal"]]
    s.precision = BSDE_PRECISION[precision]
    s.smoothing = int(p.get("smoothing", 0))
    s.picard_max = int(p.get("picard_max", 30))
    s.N, s.k, s.L, s.Nx = int(p["N"]), int(p["k"]), int(p["L"]), int(p["Nx"])
    for f in ("T", "x_min", "x_max", "x0", "a_x", "b_x"):
        setattr(s, f, float(p[f]))
    for f in ("r", "mu", "sigma", "R", "delta", "strike"):
        setattr(s, f, float(p.get(f, 0.0)))
    s.lb_sign = float(p.get("lb_sign", 1.0))
    if s.sigma == 0.0:
        s.sigma = 1.0
    s.picard_tol = float(p.get("picard_tol", 1e-12))
    s.k_z = int(p.get("kz", 0))
    s.z_form = int(p.get("zform", 0))
    mode = p.get("init_mode", 0)
    s.init_mode = BSDE_INIT[mode] if isinstance(mode, str) else int(mode)
    s.init_substeps = int(p.get("init_substeps", 0))
    fwd = p.get("forward", "CONST")
    s.forward = BSDE_FORWARD[fwd] if isinstance(fwd, str) else int(fwd)
    s.a_1 = float(p.get("a_1", 0.0))
    s.b_1 = float(p.get("b_1", 0.0))
    sk = p.get("step_kernel", 0)
    s.step_kernel = BSDE_STEP[sk] if isinstance(sk, str) else int(sk)
    return s


def levels_K(p: dict) -> int:
    """K = max(K_y, K_z): initial levels and levels read per step (Eq. 16)."""
    return max(int(p["k"]), int(p.get("kz", 0)) or int(p["k"]))


# --- thin wrappers with the C names ----------------------------------------

def bsde_workspace_bytes(prob: bsde_problem) -> int:
    n = ctypes.c_size_t()
    _check(load().bsde_workspace_bytes(ctypes.byref(prob), ctypes.byref(n)),
           "bsde_workspace_bytes")
    return int(n.value)


def bsde_plan(prob: bsde_problem, dev_ptr: int, nbytes: int) -> int:
    h = ctypes.c_void_p()
    _check(load().bsde_plan(ctypes.byref(prob), ctypes.c_void_p(dev_ptr), nbytes,
                            ctypes.byref(h)), "bsde_plan")
    return h.value


def bsde_solve(plan: int, stream: int, init_y: int = 0, init_z: int = 0,
               init_on_host: bool = False, out_y: int = 0, out_z: int = 0,
               out_on_host: bool = False, want_result: bool = True):
    res = bsde_result()
    rc = load().bsde_solve(ctypes.c_void_p(plan), ctypes.c_void_p(stream),
                           ctypes.c_void_p(init_y or None), ctypes.c_void_p(init_z or None),
                           int(init_on_host), ctypes.c_void_p(out_y or None),
                           ctypes.c_void_p(out_z or None), int(out_on_host),
                           ctypes.byref(res) if want_result else None)
    _check(rc, "bsde_solve")
    return res if want_result else None


class ConcurrentSolves:
    """Independent solves (each its own plan and workspace) run concurrently:
    every call forks from the caller's stream onto one stream per solver,
    enqueues each solver's graph there, and joins back, so the dependent
    launch chains of the solves overlap on the GPU.  Results are read with
    bsde_result_fetch on the caller's stream afterwards."""

    def __init__(self, solvers, device=None):
        import torch
        self.solvers = list(solvers)
        dev = device if device is not None else self.solvers[0].device
        self.streams = [torch.cuda.Stream(dev) for _ in self.solvers]
        self.fork = torch.cuda.Event()
        self.joins = [torch.cuda.Event() for _ in self.solvers]

    def enqueue(self, stream) -> None:
        """Enqueue one solve of every solver, ordered after `stream`'s prior
        work, with `stream` waiting for all of them."""
        self.fork.record(stream)
        for s, st, ev in zip(self.solvers, self.streams, self.joins):
            st.wait_event(self.fork)
            bsde_solve(s.plan, st.cuda_stream, want_result=False)
            ev.record(st)
        for ev in self.joins:
            stream.wait_event(ev)


def bsde_result_fetch(plan: int, stream: int) -> bsde_result:
    res = bsde_result()
    _check(load().bsde_result_fetch(ctypes.c_void_p(plan), ctypes.c_void_p(stream),
                                    ctypes.byref(res)), "bsde_result_fetch")
    return res


def bsde_enqueue_level(plan: int, stream: int, n: int, parts: int = 1) -> None:
    _check(load().bsde_enqueue_level(ctypes.c_void_p(plan), ctypes.c_void_p(stream),
                                     int(n), int(parts)), "bsde_enqueue_level")


def bsde_solve_noalloc(prob: bsde_problem, stream: int, init_y: int = 0, init_z: int = 0,
                       init_on_host: bool = False, out_y: int = 0, out_z: int = 0,
                       out_on_host: bool = False) -> bsde_result:
    """Solve with the library's fixed device workspace: for callers that may
    not allocate memory at solve time (see include/bsde.h)."""
    res = bsde_result()
    rc = load().bsde_solve_noalloc(ctypes.byref(prob), ctypes.c_void_p(stream),
                                   ctypes.c_void_p(init_y or None), ctypes.c_void_p(init_z or None),
                                   int(init_on_host), ctypes.c_void_p(out_y or None),
                                   ctypes.c_void_p(out_z or None), int(out_on_host),
                                   ctypes.byref(res))
    _check(rc, "bsde_solve_noalloc")
    return res


def bsde_free(plan: int) -> None:
    if plan:
        load().bsde_free(ctypes.c_void_p(plan))


def bsde_plan_launches(plan: int) -> int:
    return int(load().bsde_plan_launches(ctypes.c_void_p(plan)))


def bsde_gauss_hermite(L: int):
    a = np.zeros(L)
    w = np.zeros(L)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(load().bsde_gauss_hermite(L, a.ctypes.data_as(dp), w.ctypes.data_as(dp)),
           "bsde_gauss_hermite")
    return a, w


def bsde_gamma(k: int):
    gy = np.zeros(k + 1)
    gz = np.zeros(k + 1)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(load().bsde_gamma(k, gy.ctypes.data_as(dp), gz.ctypes.data_as(dp)), "bsde_gamma")
    return gy, gz


# --- convenience: a plan bound to a torch-allocated workspace ---------------

def _result_dict(r: bsde_result) -> dict:
    return {"y0": r.y0, "z0": r.z0, "status": r.status,
            "picard_iters_max": r.picard_iters_max,
            "picard_resid_max": r.picard_resid_max, "levels_done": r.levels_done}


class Solver:
    """One problem, one device workspace (a torch uint8 tensor), one plan."""

    def __init__(self, problem: dict, precision: str = "fp64", device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the BSDE solver needs a CUDA device (no CPU fallback)")
        self.problem = dict(problem)
        self.precision = precision
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self._prob = make_problem(problem, precision)
        self.ws_bytes = bsde_workspace_bytes(self._prob)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
            base = self.workspace.data_ptr()
            self._base = (base + 255) // 256 * 256
            self.plan = bsde_plan(self._prob, self._base, self.ws_bytes)

    @property
    def launches(self) -> int:
        return bsde_plan_launches(self.plan)

    def solve(self, init=None, want_level: bool = False, stream=None) -> dict:
        """init: None (the problem's start: closed form or one-step start-up)
        or (init_y, init_z), each (K, Nx), K = max(k, kz), float64 host
        arrays or device tensors (row m = level N - m)."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        sp = stream.cuda_stream
        iy = iz = 0
        on_host = False
        keep = []
        if init is not None:
            y, z = init
            if isinstance(y, torch.Tensor) and y.is_cuda:
                y = y.contiguous().to(torch.float64)
                z = z.contiguous().to(torch.float64)
                keep += [y, z]
                iy, iz = y.data_ptr(), z.data_ptr()
            else:
                y = np.ascontiguousarray(y, dtype=np.float64)
                z = np.ascontiguousarray(z, dtype=np.float64)
                keep += [y, z]
                iy, iz = y.ctypes.data, z.ctypes.data
                on_host = True
        oy = oz = None
        if want_level:
            oy = np.zeros(int(self.problem["Nx"]))
            oz = np.zeros(int(self.problem["Nx"]))
        res = bsde_solve(self.plan, sp, iy, iz, on_host,
                         oy.ctypes.data if want_level else 0,
                         oz.ctypes.data if want_level else 0, True, True)
        out = _result_dict(res)
        if want_level:
            out["y"] = oy
            out["z"] = oz
        return out

    def solve_levels(self, levels: int, stream=None) -> dict:
        """The first `levels` backward levels only (n = N-K down to
        N-K-levels+1), driven level by level through bsde_enqueue_start and
        bsde_enqueue_level from the problem's own start; returns the last
        computed level's y and z (float64 host arrays, read from the plan's
        ring through bsde_level_records) and its index n."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        sp = stream.cuda_stream
        p = self.problem
        K = levels_K(p)
        n_last = int(p["N"]) - K - int(levels) + 1
        if levels < 1 or n_last < 0:
            raise ValueError("levels outside 1..N-K+1")
        lib = load()
        _check(lib.bsde_enqueue_start(ctypes.c_void_p(self.plan), ctypes.c_void_p(sp), None, None,
                                      0), "bsde_enqueue_start")
        for n in range(int(p["N"]) - K, n_last - 1, -1):
            bsde_enqueue_level(self.plan, sp, n, 3)
        rec = ctypes.c_void_p()
        rb = ctypes.c_size_t()
        _check(lib.bsde_level_records(ctypes.c_void_p(self.plan), n_last, ctypes.byref(rec),
                                      ctypes.byref(rb)), "bsde_level_records")
        torch.cuda.synchronize(self.device)
        nx = int(p["Nx"])
        off = int(rec.value) - self.workspace.data_ptr()
        raw = self.workspace[off:off + nx * int(rb.value)]
        if int(rb.value) == 32:  # FP64 record (y, M_y, z, M_z)
            v = raw.view(torch.float64).view(nx, 4).cpu().numpy()
            y, z = v[:, 0].copy(), v[:, 2].copy()
        else:  # FP32C record (y_hi, z_hi, y_lo, z_lo)
            v = raw.view(torch.float32).view(nx, 4).cpu().numpy().astype(np.float64)
            y, z = v[:, 0] + v[:, 2], v[:, 1] + v[:, 3]
        return {"n": n_last, "y": y, "z": z}

    def close(self) -> None:
        if getattr(self, "plan", None):
            bsde_free(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(problem: dict, precision: str = "fp64", init=None, want_level: bool = False) -> dict:
    s = Solver(problem, precision)
    try:
        return s.solve(init=init, want_level=want_level)
    finally:
        s.close()


# --- batched solves ---------------------------------------------------------

def _problem_array(problems, precision):
    arr = (bsde_problem * len(problems))()
    for i, p in enumerate(problems):
        arr[i] = make_problem(p, precision)
    return arr


def bsde_batch_workspace_bytes(problems, precision: str = "fp32c") -> int:
    arr = _problem_array(problems, precision)
    n = ctypes.c_size_t()
    _check(load().bsde_batch_workspace_bytes(len(problems), arr, ctypes.byref(n)),
           "bsde_batch_workspace_bytes")
    return int(n.value)


class BatchSolver:
    """Many problems, one workspace, one persistent launch per solve."""

    def __init__(self, problems, precision: str = "fp32c", device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the BSDE solver needs a CUDA device (no CPU fallback)")
        self.problems = [dict(p) for p in problems]
        self.n = len(problems)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self._arr = _problem_array(problems, precision)
        need = ctypes.c_size_t()
        _check(load().bsde_batch_workspace_bytes(self.n, self._arr, ctypes.byref(need)),
               "bsde_batch_workspace_bytes")
        self.ws_bytes = int(need.value)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
            base = (self.workspace.data_ptr() + 255) // 256 * 256
            h = ctypes.c_void_p()
            _check(load().bsde_plan_batch(self.n, self._arr, ctypes.c_void_p(base), self.ws_bytes,
                                          ctypes.byref(h)), "bsde_plan_batch")
            self.batch = h.value

    def config(self) -> dict:
        c = bsde_batch_config()
        _check(load().bsde_batch_get_config(ctypes.c_void_p(self.batch), ctypes.byref(c)),
               "bsde_batch_get_config")
        return {"cluster": c.cluster, "target_groups": c.target_groups,
                "flat_tiles": c.flat_tiles}

    def set_config(self, cluster: int, target_groups: int, flat_tiles: int = 0) -> None:
        c = bsde_batch_config()
        c.cluster, c.target_groups, c.flat_tiles = cluster, target_groups, flat_tiles
        _check(load().bsde_batch_set_config(ctypes.c_void_p(self.batch), ctypes.byref(c)),
               "bsde_batch_set_config")

    def autotune(self, stream=None) -> dict:
        import torch
        s = stream or torch.cuda.current_stream(self.device)
        c = bsde_batch_config()
        _check(load().bsde_batch_autotune(ctypes.c_void_p(self.batch), ctypes.c_void_p(s.cuda_stream),
                                          ctypes.byref(c)), "bsde_batch_autotune")
        return {"cluster": c.cluster, "target_groups": c.target_groups,
                "flat_tiles": c.flat_tiles}

    def solve(self, stream=None, want_results: bool = True):
        import torch
        s = stream or torch.cuda.current_stream(self.device)
        if not want_results:
            _check(load().bsde_solve_batch(ctypes.c_void_p(self.batch), ctypes.c_void_p(s.cuda_stream),
                                           None), "bsde_solve_batch")
            return None
        res = (bsde_result * self.n)()
        _check(load().bsde_solve_batch(ctypes.c_void_p(self.batch), ctypes.c_void_p(s.cuda_stream),
                                       res), "bsde_solve_batch")
        return [_result_dict(r) for r in res]

    def close(self) -> None:
        if getattr(self, "batch", None):
            load().bsde_batch_free(ctypes.c_void_p(self.batch))
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- continuous-batching server ---------------------------------------------

def bsde_request_bytes(problem: dict) -> int:
    n = ctypes.c_size_t()
    _check(load().bsde_request_bytes(ctypes.byref(make_problem(problem, "fp32c")), ctypes.byref(n)),
           "bsde_request_bytes")
    return int(n.value)


class Server:
    """A persistent device kernel solving requests as they are submitted.
    Device memory: one torch tensor (slot statistics + the request pool)."""

    def __init__(self, slots: int = 512, pool_bytes: int = 4 << 30, device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the BSDE server needs a CUDA device (no CPU fallback)")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.slots = slots
        need = ctypes.c_size_t()
        _check(load().bsde_server_workspace_bytes(slots, pool_bytes, ctypes.byref(need)),
               "bsde_server_workspace_bytes")
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(int(need.value) + 256, dtype=torch.uint8, device=self.device)
            base = (self.workspace.data_ptr() + 255) // 256 * 256
            h = ctypes.c_void_p()
            _check(load().bsde_server_create(ctypes.c_void_p(base), int(need.value), slots, pool_bytes,
                                             ctypes.byref(h)), "bsde_server_create")
        self.handle = h.value
        self.stream = None
        self._slot_buf = (ctypes.c_int * slots)()
        self._res_buf = (bsde_result * slots)()

    def start(self, cluster: int = 1, idle_ms: int = 30000):
        import torch
        # a stream of its own: the persistent kernel occupies it until stop()
        self.stream = torch.cuda.Stream(self.device)
        _check(load().bsde_server_start(ctypes.c_void_p(self.handle),
                                        ctypes.c_void_p(self.stream.cuda_stream), cluster, idle_ms),
               "bsde_server_start")

    def submit(self, problem: dict):
        """Slot index, or None when no slot or pool memory is free now."""
        sl = ctypes.c_int(-1)
        rc = load().bsde_server_submit(ctypes.c_void_p(self.handle),
                                       ctypes.byref(make_problem(problem, "fp32c")), ctypes.byref(sl))
        if rc == BSDE_BUSY:
            return None
        _check(rc, "bsde_server_submit")
        return sl.value

    def poll(self):
        n = _check(load().bsde_server_poll(ctypes.c_void_p(self.handle), self.slots,
                                           self._slot_buf, self._res_buf), "bsde_server_poll")
        return [(self._slot_buf[i], _result_dict(self._res_buf[i])) for i in range(n)]

    def stop(self):
        _check(load().bsde_server_stop(ctypes.c_void_p(self.handle)), "bsde_server_stop")

    def close(self):
        if getattr(self, "handle", None):
            load().bsde_server_free(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def l2_read_bandwidth(mib: int = 48, reps: int = 40, device=None) -> float:
    """L2 -> SM read bandwidth in GB/s: a buffer that fits in L2, read `reps`
    times by one launch of 16-byte loads (after one warm-up launch), timed
    with CUDA events on the launching stream; the best of five launches (a
    peak probe: slower launches were disturbed)."""
    import torch
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    props = torch.cuda.get_device_properties(dev)
    grid = 8 * props.multi_processor_count
    buf = torch.ones((mib << 20) // 4, dtype=torch.float32, device=dev)
    sink = torch.zeros(grid, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    lib = load()
    args = (ctypes.c_void_p(buf.data_ptr()), buf.numel() * 4, 1, grid,
            ctypes.c_void_p(sink.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    _check(lib.bsde_l2_read_probe(*args), "bsde_l2_read_probe")
    best = 0.0
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _check(lib.bsde_l2_read_probe(args[0], args[1], reps, grid, args[4], args[5]),
               "bsde_l2_read_probe")
        e1.record(stream)
        torch.cuda.synchronize(dev)
        best = max(best, buf.numel() * 4 * reps / (e0.elapsed_time(e1) / 1e3) / 1e9)
    return best


FMA_KINDS = {"fp64": 0, "fp32": 1, "fp32x2": 2}


def fma_peak_tflops(kind: str, iters: int = 4096, device=None) -> float:
    """The FMA pipe's rate in TFLOP/s (2 flop per FMA): one launch of
    independent FMA chains on 8 CTAs of 256 threads per SM (after one warm-up
    launch), timed with CUDA events on the launching stream; the best of
    five launches.  kind: "fp64", "fp32" or "fp32x2" (packed)."""
    import torch
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    props = torch.cuda.get_device_properties(dev)
    grid = 8 * props.multi_processor_count
    if kind == "fp64":
        iters = max(1, iters // 32)  # the FP64 pipe is far slower: a launch of similar length
    sink = torch.zeros(grid * 256, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    lib = load()
    flops = ctypes.c_int64()
    args = (FMA_KINDS[kind], iters, grid, ctypes.c_void_p(sink.data_ptr()),
            ctypes.c_void_p(stream.cuda_stream), ctypes.byref(flops))
    _check(lib.bsde_fma_probe(*args), "bsde_fma_probe")
    best = 0.0
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _check(lib.bsde_fma_probe(*args), "bsde_fma_probe")
        e1.record(stream)
        torch.cuda.synchronize(dev)
        best = max(best, flops.value / (e0.elapsed_time(e1) / 1e3) / 1e12)
    return best


# --- two space dimensions (include/bsde2d.h) ---------------------------------

def make_problem2(p: dict, precision: str = "fp64") -> bsde2_problem:
    s = bsde2_problem()
    s.driver = BSDE2_DRIVER[p["driver"]]
    s.terminal = BSDE2_TERMINAL[p["terminal"]]
    s.precision = BSDE_PRECISION[precision]
    s.picard_max = int(p.get("picard_max", 30))
    s.N, s.k, s.L = int(p["N"]), int(p["k"]), int(p["L"])
    s.Nx1, s.Nx2 = int(p["Nx1"]), int(p["Nx2"])
    for f in ("T", "x1_min", "x1_max", "x2_min", "x2_max", "x01", "x02", "a1", "a2",
              "b11", "b21", "b22", "alpha", "beta1", "beta2"):
        setattr(s, f, float(p[f]))
    s.picard_tol = float(p.get("picard_tol", 1e-12))
    s.step_form = BSDE2_STEP[p.get("step_form", "AUTO")]
    return s


def bsde2_workspace_bytes(prob: bsde2_problem) -> int:
    n = ctypes.c_size_t()
    _check(load().bsde2_workspace_bytes(ctypes.byref(prob), ctypes.byref(n)),
           "bsde2_workspace_bytes")
    return int(n.value)


class Solver2:
    """One two-dimensional problem, one device workspace, one plan."""

    def __init__(self, problem: dict, device=None, precision: str = "fp64"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the BSDE solver needs a CUDA device (no CPU fallback)")
        self.problem = dict(problem)
        self.precision = precision
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self._prob = make_problem2(problem, precision)
        self.ws_bytes = bsde2_workspace_bytes(self._prob)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
            self._base = (self.workspace.data_ptr() + 255) // 256 * 256
            h = ctypes.c_void_p()
            _check(load().bsde2_plan(ctypes.byref(self._prob), ctypes.c_void_p(self._base),
                                     self.ws_bytes, ctypes.byref(h)), "bsde2_plan")
            self.plan = h.value

    @property
    def launches(self) -> int:
        return int(load().bsde2_plan_launches(ctypes.c_void_p(self.plan)))

    def enqueue(self, stream: int) -> None:
        """Enqueue one solve from the closed-form start; no wait, no result."""
        _check(load().bsde2_solve(ctypes.c_void_p(self.plan), ctypes.c_void_p(stream),
                                  None, None, None, 0, None, None, None, 0, None),
               "bsde2_solve")

    def fetch(self, stream: int) -> dict:
        r = bsde2_result()
        rc = load().bsde2_result_fetch(ctypes.c_void_p(self.plan), ctypes.c_void_p(stream),
                                       ctypes.byref(r))
        if rc < 0:
            _check(rc, "bsde2_result_fetch")
        return self._dict(r)

    @staticmethod
    def _dict(r) -> dict:
        return {"y0": r.y0, "z0": (r.z0[0], r.z0[1]), "status": r.status,
                "picard_iters_max": r.picard_iters_max,
                "picard_resid_max": r.picard_resid_max, "levels_done": r.levels_done}

    def enqueue_level(self, stream: int, n: int, parts: int = 1) -> None:
        _check(load().bsde2_enqueue_level(ctypes.c_void_p(self.plan), ctypes.c_void_p(stream),
                                          int(n), int(parts)), "bsde2_enqueue_level")

    def solve(self, init=None, want_level: bool = False, stream=None) -> dict:
        """init: None (closed-form start) or (y, z1, z2), each (k, Nx2, Nx1)
        float64 host arrays (row m = level N - m, x1 fastest)."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        p = self.problem
        shape = (int(p["Nx2"]), int(p["Nx1"]))
        ins = [None, None, None]
        keep = []
        if init is not None:
            for q, a in enumerate(init):
                a = np.ascontiguousarray(a, dtype=np.float64)
                keep.append(a)
                ins[q] = ctypes.c_void_p(a.ctypes.data)
        outs = [np.zeros(shape) for _ in range(3)] if want_level else None
        r = bsde2_result()
        rc = load().bsde2_solve(ctypes.c_void_p(self.plan), ctypes.c_void_p(stream.cuda_stream),
                                *ins, 1 if init is not None else 0,
                                *([ctypes.c_void_p(o.ctypes.data) for o in outs] if outs
                                  else [None, None, None]),
                                1, ctypes.byref(r))
        if rc < 0:
            _check(rc, "bsde2_solve")
        out = self._dict(r)
        if want_level:
            out["y"], out["z1"], out["z2"] = outs
        return out

    def close(self) -> None:
        if getattr(self, "plan", None):
            load().bsde2_free(ctypes.c_void_p(self.plan))
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve2(problem: dict, init=None, want_level: bool = False, precision: str = "fp64") -> dict:
    s = Solver2(problem, precision=precision)
    try:
        return s.solve(init=init, want_level=want_level)
    finally:
        s.close()
