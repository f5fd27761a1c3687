"""The profiler (oocs_set_profiling) and the per-visit timeline
(oocs_get_timeline): every profiled copy and kernel of a sweep is counted
once, with its bytes or points, and placed on the stream its role gives it
(one working buffer: host->device copies on stream 0, kernels on stream 1,
device->host copies on stream 2); the order of a visit's items follows the
dependencies of Algorithm 1; profiling changes no result."""
import numpy as np
import pytest

import synthetic
from gpu_util import heat_desc, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2204_11315_gb300 as P
    P.lib()
    return P


def _run(P, desc, u0, nsteps, prof):
    st = P.OutOfCoreStencil(desc)
    try:
        st.compress(P.OOCS_FIELD_U, u0)
        st.synchronize(60.0)
        st.set_profiling(prof)
        b = st.stats()
        st.step(nsteps)
        st.synchronize(120.0)
        a = st.stats()
        tl = P.oocs_get_timeline(st.ctx)
        out = st.decompress(P.OOCS_FIELD_U)
        st.synchronize(60.0)
        return out.numpy().copy(), b, a, tl, st.plan
    finally:
        st.close()


def test_timeline_of_a_sweep(P):
    torch_cuda()
    shape = (96, 72, 136)
    u0 = synthetic.uniform_field(shape, 31)
    desc = heat_desc(P, shape, rate=16, k=2, T=32)
    ref, _, _, _, _ = _run(P, desc, u0, 6, 0)
    got, b, a, tl, plan = _run(P, desc, u0, 6, 31)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))  # profiling changes nothing
    visits = a["slabs_done"] - b["slabs_done"]
    assert visits == 3 * plan.num_slabs
    by = {}
    for e in tl:
        assert e["end_ms"] >= e["start_ms"]
        by.setdefault(e["cls"], []).append(e)
    # one load, one step group, one store, one host->device and one
    # device->host item per visit, each on the stream of its role
    for cls, stream in (("h2d", 0), ("load", 1), ("step", 1), ("store", 1), ("d2h", 2)):
        assert len(by[cls]) == visits, cls
        assert {e["stream"] for e in by[cls]} == {stream}, cls
        assert sorted(e["visit"] for e in by[cls]) == list(range(b["slabs_done"], a["slabs_done"]))
    # the stats of the profiled classes: copies in bytes, kernels in points
    assert a["h2d"]["units"] - b["h2d"]["units"] == a["h2d_bytes"] - b["h2d_bytes"]
    assert a["d2h"]["units"] - b["d2h"]["units"] == a["d2h_bytes"] - b["d2h_bytes"]
    for cls in ("load", "step", "store", "h2d", "d2h"):
        assert a[cls]["device_ms"] > b[cls]["device_ms"]
    # within a visit: its copy in ends before its decode starts, the decode
    # before the steps, the steps before the encode, the encode before its
    # copy out
    first = {(e["cls"], e["visit"]): e for e in tl}
    eps = 1e-3
    for v in range(b["slabs_done"], a["slabs_done"]):
        h, ld, sp = first[("h2d", v)], first[("load", v)], first[("step", v)]
        sto, d = first[("store", v)], first[("d2h", v)]
        assert h["end_ms"] <= ld["start_ms"] + eps
        assert ld["end_ms"] <= sp["start_ms"] + eps
        assert sp["end_ms"] <= sto["start_ms"] + eps
        assert sto["end_ms"] <= d["start_ms"] + eps
    # kernels of consecutive visits never overlap (one working buffer)
    kern = sorted((e for e in tl if e["stream"] == 1), key=lambda e: e["start_ms"])
    for x, y in zip(kern, kern[1:]):
        assert x["end_ms"] <= y["start_ms"] + eps


def test_profiling_off_records_nothing(P):
    torch_cuda()
    shape = (64, 36, 68)
    u0 = synthetic.uniform_field(shape, 32)
    _, b, a, tl, _ = _run(P, heat_desc(P, shape, rate=16, k=2, T=32), u0, 4, 0)
    assert tl == []
    for cls in ("load", "step", "store", "h2d", "d2h"):
        assert a[cls]["device_ms"] == b[cls]["device_ms"]
    assert a["load"]["launches"] > b["load"]["launches"]  # counted even when not timed
