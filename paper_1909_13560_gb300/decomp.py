"""Domain decomposition of one 1-D problem over several plans: each plan owns
a slab of the grid and keeps a halo wide enough that its owned points never
see the slab's ends.

Per backward level every slab runs its step kernel, the halo part of the new
level's value records is replaced by the neighbours' owned values, and every
slab runs its spline kernel.  The halo is the reach of the Gauss-Hermite
nodes (the largest cell shift of any (j, l), plus the right cell of a node)
plus a margin over which the spline's end condition at the slab's end decays
below double precision (the LU recurrences of tridiag(1, 4, 1) contract by
2 - sqrt 3 per node: 40 nodes give 1e-23).  The initial levels come from the
closed form (or the caller's levels) on every slab's whole local grid, so they
need no exchange.

Two transports move the halo records:
  * LocalTransport: all slabs on one device, copies between their
    workspaces on one stream (the exchange the multi-GPU run does, with the
    wire replaced by device copies);
  * DistTransport: one slab per rank of torch.distributed, point-to-point
    send/recv of the edge records to the neighbouring ranks between launches
    (NCCL on GPUs; gloo carries the same protocol on CPU tensors in the
    tests).
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import bsde as B

MARGIN = 40  # spline margin in grid nodes


def node_reach(problem: dict) -> int:
    """Largest |cell index offset| a node of any (j, l) reaches from its grid
    point, counting the right cell node: max over j <= K, l of
    max(|floor(o)|, |floor(o) + 1|), o = (a_x j dt + b_x sqrt(2 j dt) a_l) / dx."""
    if problem.get("forward", "CONST") not in ("CONST", 0):
        raise ValueError("the decomposition needs a constant-coefficient forward process")
    K = B.levels_K(problem)
    L = int(problem["L"])
    a = (ctypes.c_double * L)()
    w = (ctypes.c_double * L)()
    B._check(B.load().bsde_gauss_hermite(L, a, w), "bsde_gauss_hermite")
    dt = float(problem["T"]) / int(problem["N"])
    dx = (float(problem["x_max"]) - float(problem["x_min"])) / (int(problem["Nx"]) - 1)
    reach = 0
    for j in range(1, K + 1):
        for l in range(L):
            o = (float(problem["a_x"]) * j * dt + float(problem["b_x"]) * math.sqrt(2.0 * j * dt) * a[l]) / dx
            f = math.floor(o)
            reach = max(reach, abs(f), abs(f + 1))
    return int(reach)


def halo_width(problem: dict) -> int:
    return node_reach(problem) + MARGIN


def slabs(Nx: int, parts: int, halo: int):
    """Owned ranges [own_lo, own_hi) split evenly, local ranges [lo, hi) with
    the halo clipped to the grid.  Every owned range must be at least `halo`
    wide, so that a halo comes from the immediate neighbours only."""
    if parts < 1:
        raise ValueError("parts >= 1")
    out = []
    for r in range(parts):
        own_lo = r * Nx // parts
        own_hi = (r + 1) * Nx // parts
        if parts > 1 and own_hi - own_lo < halo:
            raise ValueError(f"slab {r} owns {own_hi - own_lo} points, fewer than the halo {halo}")
        out.append({"own": (own_lo, own_hi), "local": (max(0, own_lo - halo), min(Nx, own_hi + halo))})
    return out


def slab_problem(problem: dict, lo: int, hi: int) -> dict:
    """The problem restricted to grid points [lo, hi) (same spacing; the
    readout point clamped into the slab)."""
    Nx = int(problem["Nx"])
    dx = (float(problem["x_max"]) - float(problem["x_min"])) / (Nx - 1)
    q = dict(problem)
    q["x_min"] = float(problem["x_min"]) + lo * dx
    q["x_max"] = float(problem["x_min"]) + (hi - 1) * dx
    q["Nx"] = hi - lo
    q["x0"] = min(max(float(problem["x0"]), q["x_min"]), q["x_max"])
    return q


def _records(solver, n: int):
    """(uint8 tensor view of level n's value records, record size) of a
    Solver: a slice of its workspace tensor."""
    vp = ctypes.c_void_p()
    rb = ctypes.c_size_t()
    B._check(B.load().bsde_level_records(ctypes.c_void_p(solver.plan), int(n), ctypes.byref(vp),
                                         ctypes.byref(rb)), "bsde_level_records")
    off = int(vp.value) - solver.workspace.data_ptr()
    nb = int(solver.problem["Nx"]) * int(rb.value)
    return solver.workspace[off:off + nb], int(rb.value)


class LocalTransport:
    """All slabs in this process on one device: halo records copied between
    the slabs' workspaces on the solve's stream."""

    def exchange(self, solvers, layout, n: int) -> None:
        views = [_records(s, n) for s in solvers]
        for r, sl in enumerate(layout):
            lo, hi = sl["local"]
            own_lo, own_hi = sl["own"]
            dst, rb = views[r]
            if r > 0 and lo < own_lo:  # left halo from slab r - 1
                src, _ = views[r - 1]
                slo = layout[r - 1]["local"][0]
                dst[(0) * rb:(own_lo - lo) * rb].copy_(src[(lo - slo) * rb:(own_lo - slo) * rb])
            if r < len(layout) - 1 and own_hi < hi:  # right halo from slab r + 1
                src, _ = views[r + 1]
                slo = layout[r + 1]["local"][0]
                dst[(own_hi - lo) * rb:(hi - lo) * rb].copy_(src[(own_hi - slo) * rb:(hi - slo) * rb])


class DistTransport:
    """One slab per rank: the edge records go to the neighbouring ranks by
    point-to-point send/recv between launches.  stage_on_host moves device
    records through host memory for backends without device tensors (gloo)."""

    def __init__(self, dist, stage_on_host: bool = False):
        self.dist = dist
        self.stage_on_host = stage_on_host

    def exchange_views(self, rank: int, layout, view, rb: int) -> None:
        """Exchange halos of this rank's records `view` (uint8, local grid)."""
        d = self.dist
        lo, hi = layout[rank]["local"]
        own_lo, own_hi = layout[rank]["own"]
        world = len(layout)
        ops, recvs = [], []

        def buf(t):
            return t.cpu() if self.stage_on_host else t

        if rank > 0:
            # my first owned records -> left neighbour's right halo; its last
            # owned records -> my left halo
            nl = layout[rank - 1]["local"][1] - own_lo
            send = buf(view[(own_lo - lo) * rb:(own_lo - lo + nl) * rb].contiguous())
            recv = buf(view[0:(own_lo - lo) * rb].clone())
            ops += [d.P2POp(d.isend, send, rank - 1), d.P2POp(d.irecv, recv, rank - 1)]
            recvs.append((recv, 0, (own_lo - lo) * rb))
        if rank < world - 1:
            nr = own_hi - layout[rank + 1]["local"][0]
            send = buf(view[(own_hi - lo - nr) * rb:(own_hi - lo) * rb].contiguous())
            recv = buf(view[(own_hi - lo) * rb:(hi - lo) * rb].clone())
            ops += [d.P2POp(d.isend, send, rank + 1), d.P2POp(d.irecv, recv, rank + 1)]
            recvs.append((recv, (own_hi - lo) * rb, (hi - lo) * rb))
        if ops:
            for req in d.batch_isend_irecv(ops):
                req.wait()
        for recv, a, b in recvs:
            view[a:b].copy_(recv.to(view.device) if self.stage_on_host else recv)


class ShardedSolver:
    """One problem as `parts` slabs on one device (LocalTransport): the slabs'
    plans are made once; each enqueue() runs the level-by-level loop with a
    halo exchange after every step, and result() reads the owner's result."""

    def __init__(self, problem: dict, parts: int, precision: str = "fp64", device=None):
        if problem.get("init_mode", 0) not in (0, "EXACT") and B.levels_K(problem) > 1:
            raise ValueError("the decomposition starts from the closed form or caller levels")
        self.problem = dict(problem)
        self.Nx = int(problem["Nx"])
        self.layout = slabs(self.Nx, parts, halo_width(problem))
        self.subs = [slab_problem(problem, *sl["local"]) for sl in self.layout]
        self.solvers = [B.Solver(q, precision, device=device) for q in self.subs]
        self.device = self.solvers[0].device
        self.transport = LocalTransport()
        x0 = float(problem["x0"])
        dx = (float(problem["x_max"]) - float(problem["x_min"])) / (self.Nx - 1)
        g0 = min(int(math.floor((x0 - float(problem["x_min"])) / dx)), self.Nx - 1)
        self.owner = next(r for r, sl in enumerate(self.layout)
                          if sl["own"][0] <= g0 < sl["own"][1])

    def enqueue(self, stream, init=None, outs=None, keep=None) -> None:
        """Enqueue one solve on `stream` (torch stream).  init: None or host
        arrays (K, Nx) of the caller's levels; outs: None or per slab a pair of
        host arrays for its local level 0 (the call then waits for them)."""
        sp = stream.cuda_stream
        lib = B.load()
        keep = [] if keep is None else keep
        for s, sl in zip(self.solvers, self.layout):
            iy = iz = None
            if init is not None:
                lo, hi = sl["local"]
                iy = np.ascontiguousarray(init[0][:, lo:hi], dtype=np.float64)
                iz = np.ascontiguousarray(init[1][:, lo:hi], dtype=np.float64)
                keep += [iy, iz]
            B._check(lib.bsde_enqueue_start(ctypes.c_void_p(s.plan), ctypes.c_void_p(sp),
                                            iy.ctypes.data if iy is not None else None,
                                            iz.ctypes.data if iz is not None else None,
                                            1 if iy is not None else 0), "bsde_enqueue_start")
        K = B.levels_K(self.problem)
        for n in range(int(self.problem["N"]) - K, -1, -1):
            for s in self.solvers:
                B.bsde_enqueue_level(s.plan, sp, n, 1)
            self.transport.exchange(self.solvers, self.layout, n)
            for s in self.solvers:
                B.bsde_enqueue_level(s.plan, sp, n, 2)
        for r, s in enumerate(self.solvers):
            oy = oz = None
            if outs is not None:
                oy, oz = outs[r]
            B._check(lib.bsde_enqueue_finish(ctypes.c_void_p(s.plan), ctypes.c_void_p(sp),
                                             oy.ctypes.data if oy is not None else None,
                                             oz.ctypes.data if oz is not None else None,
                                             1 if oy is not None else 0), "bsde_enqueue_finish")

    def replay(self, stream) -> None:
        """One solve from the closed-form start as a CUDA graph: the
        level-by-level loop (a few launches and copies per slab and level,
        which the host would otherwise issue one by one) is captured at the
        first call and replayed on `stream` after that."""
        import torch
        if getattr(self, "_graph", None) is None:
            self._graph = torch.cuda.CUDAGraph()
            cap = torch.cuda.Stream(self.device)
            cap.wait_stream(stream)
            with torch.cuda.graph(self._graph, stream=cap):
                self.enqueue(cap)
            stream.wait_stream(cap)
        self._graph.replay()

    def result(self, stream) -> dict:
        res = [B.bsde_result_fetch(s.plan, stream.cuda_stream) for s in self.solvers]
        r0 = res[self.owner]
        return {"y0": r0.y0, "z0": r0.z0,
                "picard_iters_max": max(r.picard_iters_max for r in res),
                "picard_resid_max": max(r.picard_resid_max for r in res),
                "levels_done": r0.levels_done, "slabs": self.layout}

    def close(self) -> None:
        self._graph = None
        for s in self.solvers:
            s.close()


def solve_sharded(problem: dict, parts: int, precision: str = "fp64", device=None,
                  want_level: bool = False, init=None) -> dict:
    """Solve one problem as `parts` slabs on one device (LocalTransport).
    Returns y0, z0 (from the slab that owns x0), the merged Picard statistics
    and, if asked, the assembled level 0."""
    import torch
    ss = ShardedSolver(problem, parts, precision, device)
    stream = torch.cuda.current_stream(ss.device)
    outs = [(np.zeros(int(q["Nx"])), np.zeros(int(q["Nx"]))) for q in ss.subs] if want_level else None
    ss.enqueue(stream, init=init, outs=outs)
    out = ss.result(stream)
    if want_level:
        y = np.zeros(ss.Nx)
        z = np.zeros(ss.Nx)
        for (oy, oz), sl in zip(outs, ss.layout):
            lo = sl["local"][0]
            a, b = sl["own"]
            y[a:b] = oy[a - lo:b - lo]
            z[a:b] = oz[a - lo:b - lo]
        out["y"], out["z"] = y, z
    ss.close()
    return out
