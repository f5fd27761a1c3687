"""The multi-GPU path of bench.py on the CPU: replicas combined over a gloo
process group of two ranks (the slowest replica's time, whole-job throughput,
the line's replica fields)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        ms = bench.max_over_ranks(torch, 100.0 + 50.0 * rank, "cpu")
        value = bench.replica_throughput(1e9, w, ms)

        class A:
            steps, warmup = 5, 3
        line = bench.base_line(A, w, bench.OOC_SHAPE[0])
        q.put((r, w, local, ms, value, line["n_gpus"], line["config"]["parallelism"], line["scaling"]))
    finally:
        dist.destroy_process_group()


def test_two_replicas_over_gloo():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, local, ms, value, n, par, scaling) in enumerate(out):
        assert (rank, world, local) == (r, 2, r)
        assert ms == 150.0  # the slower replica sets the time on every rank
        assert value == pytest.approx(2 * 1e9 / 0.150 / 1e9)
        assert (n, par, scaling) == (2, "replicas2", "weak")


def test_one_process_needs_no_group():
    import torch

    import bench
    assert bench.max_over_ranks(torch, 12.5, "cpu") == 12.5
    assert bench.replica_throughput(2e9, 1, 1000.0) == pytest.approx(2.0)


def test_headline_planes_follow_host_memory():
    """Each replica holds one raw FP32 array of its grid in pinned host memory:
    the headline keeps nz = 5120 when the host holds it, else shrinks nz (a
    multiple of 64) to what fits, per rank."""
    import bench

    class A:
        planes = 0
    plane = bench.OOC_SHAPE[1] * bench.OOC_SHAPE[2] * 4
    real = bench.host_mem_available
    try:
        bench.host_mem_available = lambda: 199 * 10 ** 9
        assert bench.ooc_planes(A, 1) == 5120
        nz2 = bench.ooc_planes(A, 2)
        assert nz2 % 64 == 0 and nz2 * plane <= 0.9 * 199e9 / 2 and nz2 < 5120
        bench.host_mem_available = lambda: None
        assert bench.ooc_planes(A, 8) == 5120
    finally:
        bench.host_mem_available = real
    A.planes = 512
    assert bench.ooc_planes(A, 1) == 512


def test_cube_origins_are_block_aligned_and_inside():
    import bench
    shape = bench.OOC_SHAPE
    side = bench.CUBE_IN + 2 * bench.CUBE_HALO
    for o in bench.cube_origins(shape, 64):
        for a in range(3):
            assert o[a] % 4 == 0
            assert o[a] - bench.CUBE_HALO >= 1 and o[a] - bench.CUBE_HALO + side <= shape[a] - 1
