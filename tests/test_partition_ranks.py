"""The z-partitioned multi-GPU design, checked on CPU ranks with the oracle.

Each rank owns a contiguous z range [z0, z1) of the grid (a group of slabs)
and, per pass of k steps, receives the h = k r boundary planes of each
z-neighbour (one exchange per pass over a gloo process group, standing in for
NCCL send/recv), advances its window [z0 - h, z1 + h) by k steps and keeps
[z0, z1): the temporal blocking of Sec. 3.1 applied across ranks.  The
gathered result must equal the unpartitioned oracle run bit for bit (FP64,
same operations per point).  Heat over three ranks (a middle rank with two
neighbours), wave (two levels and the read-only model) over two.  The
library itself runs one sweep per GPU (replicas); this pins the exchange
that a sweep sharded over GPUs would need.
"""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _bounds(nz, world, rank):
    per = nz // world
    return rank * per, (nz if rank == world - 1 else (rank + 1) * per)


def _exchange(dist, torch, mine, h, rank, world):
    """(planes below, planes above) of this rank's range from its neighbours."""
    lo = hi = None
    reqs = []
    if rank > 0:
        reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(mine[:h])), rank - 1))
        lo = torch.empty((h,) + mine.shape[1:], dtype=torch.float64)
        reqs.append(dist.irecv(lo, rank - 1))
    if rank < world - 1:
        reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(mine[-h:])), rank + 1))
        hi = torch.empty((h,) + mine.shape[1:], dtype=torch.float64)
        reqs.append(dist.irecv(hi, rank + 1))
    for r in reqs:
        r.wait()
    return (lo.numpy() if lo is not None else None), (hi.numpy() if hi is not None else None)


def _window(lo, mine, hi):
    parts = [p for p in (lo, mine, hi) if p is not None]
    return np.concatenate(parts, axis=0), (0 if lo is None else lo.shape[0])


def _rank(rank, world, port, scheme, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import oracle
    import synthetic
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        if scheme == "heat":
            u0 = synthetic.heat_initial(48).astype(np.float64)
            coef, r, k, passes = synthetic.heat_star_coef(0.1), 1, 3, 4
        else:
            shape = (64, 32, 32)
            u0 = (1e-3 * synthetic.uniform_field(shape, 3)).astype(np.float64)
            u0[:4] = u0[-4:] = 0.0
            u0[:, :4] = u0[:, -4:] = u0[:, :, :4] = u0[:, :, -4:] = 0.0
            m = synthetic.wave_model(shape).astype(np.float64)
            coef, r, k, passes = synthetic.wave_star_coef(), 4, 2, 3
        h = k * r
        z0, z1 = _bounds(u0.shape[0], world, rank)
        u = u0[z0:z1].copy()
        up = u.copy()
        for _ in range(passes):
            lo, hi = _exchange(dist, torch, u, h, rank, world)
            wu, off = _window(lo, u, hi)
            if scheme == "heat":
                wu = oracle.heat_run(wu, coef, k)
            else:
                plo, phi = _exchange(dist, torch, up, h, rank, world)
                wup, _ = _window(plo, up, phi)
                wm = m[max(z0 - h, 0):min(z1 + h, u0.shape[0])]
                wu, wup = oracle.wave_run(wu, wup, wm, coef, k)
                up = wup[off:off + (z1 - z0)].copy()
            u = wu[off:off + (z1 - z0)].copy()
        q.put((rank, z0, z1, u))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("scheme,world", [("heat", 3), ("wave", 2)])
def test_partitioned_sweep_equals_global(scheme, world):
    mp = pytest.importorskip("torch.multiprocessing")
    import oracle
    import synthetic
    oracle.build()  # compile once, before the ranks load it
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, scheme, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = sorted((q.get(timeout=240) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = np.concatenate([u for _, _, _, u in parts], axis=0)
    if scheme == "heat":
        u0 = synthetic.heat_initial(48).astype(np.float64)
        ref = oracle.heat_run(u0, synthetic.heat_star_coef(0.1), 3 * 4)
    else:
        shape = (64, 32, 32)
        u0 = (1e-3 * synthetic.uniform_field(shape, 3)).astype(np.float64)
        u0[:4] = u0[-4:] = 0.0
        u0[:, :4] = u0[:, -4:] = u0[:, :, :4] = u0[:, :, -4:] = 0.0
        m = synthetic.wave_model(shape).astype(np.float64)
        ref, _ = oracle.wave_run(u0, u0.copy(), m, synthetic.wave_star_coef(), 2 * 3)
    assert np.array_equal(got, ref)
    assert not np.array_equal(got, u0)
