"""The multi-process sharded step on CPU: two (and three) gloo ranks each hold one slab of a
linear-advection mesh with its two-layer upstream halo, exchange the halo by point-to-point
messages every step and advance their slab with the oracle; the gathered interiors equal the
oracle's steps on the whole mesh (the slab partition and halo logic of Sec. 5's domain
decomposition, without a GPU)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(case):
    if case == "2d+":
        w = dict(flux="advection", dim=2, n=(7, 10), M=2, vel=(0.6, 1.0), lo=(0.0, 0.0),
                 hi=(1.0, 1.0), cfl=0.3)
    else:  # 3D with a negative velocity along the slab axis
        w = dict(flux="advection", dim=3, n=(4, 3, 9), M=1, vel=(0.5, 0.3, -1.0),
                 lo=(0.0,) * 3, hi=(1.0,) * 3, cfl=0.3)
    q = np.random.default_rng(5).standard_normal((int(np.prod(w["n"])), (w["M"] + 1) ** w["dim"]))
    return w, q


def _worker(rank, ws, port, case, nsteps, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from oracle import linear as OL
    from paper_2101_01231_gb300 import shard as S
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    w, q = _problem(case)
    ax = w["dim"] - 1
    n = w["n"][ax]
    a = w["vel"][ax]
    dt, _ = OL.advection_time_step(w)
    first, nloc = S.partition(n, ws)[rank]
    layers = S.local_layers(first, nloc, n, a)
    per_layer = q.shape[0] // n
    Q = q.reshape(n, per_layer, -1)
    loc = torch.from_numpy(np.ascontiguousarray(Q[layers]).reshape(len(layers), -1))
    # the slab as a locally periodic mesh with the global cell size
    h = (w["hi"][ax] - w["lo"][ax]) / n
    wl = dict(w, n=tuple(w["n"][:ax]) + (len(layers),))
    wl["hi"] = tuple(w["hi"][:ax]) + (w["lo"][ax] + len(layers) * h,)
    ex = S.SlabExchange(rank, ws, a, nloc)
    for _ in range(nsteps):
        ex.exchange(loc)
        ql = loc.numpy().reshape(-1, q.shape[1])
        loc = torch.from_numpy(OL.step(ql, wl, dt).reshape(len(layers), -1))
    h0 = S.halo_layers(a) if a > 0 else 0
    mine = loc[h0:h0 + nloc].numpy()
    got = [None] * ws
    dist.all_gather_object(got, (first, mine))
    dist.barrier()
    dist.destroy_process_group()
    if rank == 0:
        full = np.empty((n, per_layer * q.shape[1]))
        for f, m in got:
            full[f:f + m.shape[0]] = m
        ref = OL.run(q, w, dt, nsteps)
        out.put(float(np.abs(full.reshape(q.shape) - ref).max() / np.abs(ref).max()))


@pytest.mark.parametrize("case,ws", [("2d+", 2), ("3d-", 3)])
def test_sharded_oracle_steps_over_gloo_ranks(case, ws):
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, case, 3, q)) for r in range(ws)]
    for p in procs:
        p.start()
    err = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert err < 1e-12, err


def test_partition_and_halo_layers():
    from paper_2101_01231_gb300 import shard as S
    assert S.partition(10, 3) == [(0, 4), (4, 3), (7, 3)]
    with pytest.raises(ValueError):
        S.partition(5, 3)
    assert S.local_layers(0, 4, 10, 1.0) == [8, 9, 0, 1, 2, 3]
    assert S.local_layers(7, 3, 10, -1.0) == [7, 8, 9, 0, 1]
    assert S.local_layers(4, 3, 10, 0.0) == [4, 5, 6]
    assert S.neighbours(0, 3, 1.0) == (2, 1) and S.neighbours(0, 3, -1.0) == (1, 2)
