"""Host logic of the domain decomposition of one problem (package module
decomp): the node reach against a direct scan of the node offsets, the slab
layout, and the halo exchange protocol of DistTransport between gloo ranks
on CPU (world sizes 2 and 3): after one exchange every halo record holds the
neighbour's owned record for the same grid point."""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1909_13560_gb300 import decomp
from paper_1909_13560_gb300 import workloads as W


def test_node_reach_matches_the_offsets():
    p = W.call_problem(Nx=65536, N=256, k=6, L=16)
    r = decomp.node_reach(p)
    dt, dx = p["T"] / p["N"], (p["x_max"] - p["x_min"]) / (p["Nx"] - 1)
    a = np.polynomial.hermite.hermgauss(16)[0]
    o = np.array([(p["a_x"] * j * dt + p["b_x"] * math.sqrt(2 * j * dt) * al) / dx
                  for j in range(1, 7) for al in a])
    assert r == int(max(np.max(np.abs(np.floor(o))), np.max(np.abs(np.floor(o) + 1))))
    assert decomp.halo_width(p) == r + decomp.MARGIN


def test_slab_layout_covers_the_grid():
    lay = decomp.slabs(1000, 4, 100)
    owned = [i for sl in lay for i in range(*sl["own"])]
    assert owned == list(range(1000))
    for r, sl in enumerate(lay):
        lo, hi = sl["local"]
        a, b = sl["own"]
        assert lo == max(0, a - 100) and hi == min(1000, b + 100)
    with pytest.raises(ValueError):
        decomp.slabs(1000, 8, 200)  # owned ranges narrower than the halo


def test_slab_problem_keeps_the_spacing():
    p = W.call_problem(Nx=4097, N=16, k=2)
    q = decomp.slab_problem(p, 1000, 2001)
    dx = (p["x_max"] - p["x_min"]) / (p["Nx"] - 1)
    assert q["Nx"] == 1001
    assert (q["x_max"] - q["x_min"]) / (q["Nx"] - 1) == pytest.approx(dx, rel=1e-13)
    assert q["x_min"] <= q["x0"] <= q["x_max"]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, Nx, halo, rb, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lay = decomp.slabs(Nx, world, halo)
    lo, hi = lay[rank]["local"]
    a, b = lay[rank]["own"]
    # records: rb bytes per grid point; owned records carry their global index
    recs = np.full((hi - lo, rb // 8), -1.0)
    recs[a - lo:b - lo, :] = np.arange(a, b)[:, None]
    view = torch.from_numpy(recs.view(np.uint8).reshape(-1).copy())
    decomp.DistTransport(dist).exchange_views(rank, lay, view, rb)
    got = view.numpy().view(np.float64).reshape(hi - lo, rb // 8)
    ok = bool(np.all(got[:, 0] == np.arange(lo, hi)) and np.all(got == got[:, :1]))
    out = [None] * world
    dist.all_gather_object(out, ok)
    if rank == 0:
        q.put(out)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_halo_exchange_between_ranks(world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, 600, 37, 32, q))
             for r in range(world)]
    for p in procs:
        p.start()
    out = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [True] * world
