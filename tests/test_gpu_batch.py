"""Batches of independent problems through one pipeline (oocs_batch_*), on the GPU.

Every problem of a batch must end with the host stores it gets when it runs
alone with the same desc (same kernels, same arithmetic, byte for byte), for
mixed heat / wave problems with different grids, slab thicknesses, temporal
depths, rates, sources and resident models; split calls continue each
problem's time; a captured CUDA graph replayed twice equals two direct batch
steps; a problem with a time-dependent source cannot be captured.
"""
import numpy as np
import pytest

import synthetic
from gpu_util import heat_desc, torch_cuda, wave_desc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2204_11315_gb300 as P
    P.lib()
    return P


def _problems(P, with_source=True):
    """(desc, inputs) pairs; inputs: dict field -> FP32 array, optional source."""
    out = []
    u = synthetic.heat_initial(64)
    out.append((heat_desc(P, u.shape, rate=16, k=2, T=32), {0: u}, None))
    u = synthetic.uniform_field((96, 40, 128), 7)
    out.append((heat_desc(P, u.shape, rate=0, k=3, T=32, alpha=0.12), {0: u}, None))
    for shape, rate, k, T, ro, seed in (((128, 72, 40), 16, 4, 32, 0, 11), ((96, 48, 64), 12, 3, 24, 1, 12),
                                        ((80, 40, 40), 0, 1, 16, 1, 13)):
        m = synthetic.wave_model(shape)
        if with_source:
            z = np.zeros(shape, np.float32)
            src = (synthetic.centre(shape)[::-1], synthetic.ricker(40))
            fields = {0: z, 1: z, 2: m}
        else:
            u0 = (1e-3 * synthetic.uniform_field(shape, seed)).astype(np.float32)
            fields = {0: u0, 1: u0, 2: m}
            src = None
        out.append((wave_desc(P, shape, rate=rate, k=k, T=T, ro=ro), fields, src))
    return out


def _load(prob, fields, src):
    for f, a in fields.items():
        prob.compress(f, a)
    if src is not None:
        (x, y, z), w = src
        prob.set_source(x, y, z, w)


def _alone(P, desc, fields, src, calls):
    st = P.OutOfCoreStencil(desc)
    try:
        _load(st, fields, src)
        for n in calls:
            st.step(n)
        st.synchronize(120.0)
        return [s.numpy().copy() for s in st.stores], st.stats()
    finally:
        st.close()


def _batch(P, probs):
    b = P.OutOfCoreBatch([d for d, _, _ in probs])
    for bp, (d, fields, src) in zip(b.problems, probs):
        _load(bp, fields, src)
    b.synchronize(120.0)
    return b


@pytest.mark.parametrize("calls", [[10], [4, 6]])
def test_batch_matches_problems_run_alone(P, calls):
    torch_cuda()
    probs = _problems(P)
    b = _batch(P, probs)
    try:
        for n in calls:
            b.step(n)
        b.synchronize(120.0)
        got = [[s.numpy().copy() for s in bp.stores] for bp in b.problems]
        stats = [bp.stats() for bp in b.problems]
    finally:
        b.close()
    for i, (d, fields, src) in enumerate(probs):
        # the same calls: with a lossy rate the sweep boundaries (where the
        # codec rounds) depend on how the steps are split into calls
        ref, rstats = _alone(P, d, fields, src, calls)
        nout = 2 if d.scheme == P.OOCS_WAVE else 1
        for f in range(nout):
            assert np.array_equal(got[i][f], ref[f]), (i, f)
        assert stats[i]["steps_done"] == sum(calls)
        assert stats[i]["h2d_bytes"] == rstats["h2d_bytes"] and stats[i]["d2h_bytes"] == rstats["d2h_bytes"]


def test_one_problem_of_a_batch_steps_alone(P):
    """oocs_step on a batch member advances that problem only, through the batch's pipeline."""
    torch_cuda()
    probs = _problems(P)
    b = _batch(P, probs)
    try:
        b.problems[2].step(8)
        b.synchronize(120.0)
        got = [s.numpy().copy() for s in b.problems[2].stores]
        assert b.problems[0].stats()["steps_done"] == 0
        with pytest.raises(P.OOCSError):
            P.oocs_destroy(b.problems[0].ctx)
    finally:
        b.close()
    d, fields, src = probs[2]
    ref, _ = _alone(P, d, fields, src, [8])
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


@pytest.mark.parametrize("with_source", [False, True])
def test_graph_replay_equals_direct_steps(P, with_source):
    """Two replays of a captured 6-step batch equal two direct batch steps; with
    sources, each replay reads the wavelet at its own time index (steps 0-5,
    then 6-11), byte for byte."""
    torch_cuda()
    probs = _problems(P, with_source=with_source)
    outs = []
    for mode in ("direct", "graph"):
        b = _batch(P, probs)
        try:
            if mode == "direct":
                b.step(6)
                b.step(6)
            else:
                b.capture(6)
                assert all(bp.stats()["steps_done"] == 0 for bp in b.problems)
                b.launch()
                b.launch()
            b.synchronize(120.0)
            outs.append(([[s.numpy().copy() for s in bp.stores] for bp in b.problems],
                         [bp.stats() for bp in b.problems]))
        finally:
            b.close()
    (sd, std), (sg, stg) = outs
    for i in range(len(probs)):
        for a, c in zip(sd[i], sg[i]):
            assert np.array_equal(a, c), i
        for key in ("steps_done", "h2d_bytes", "d2h_bytes", "kernel_launches", "slabs_done"):
            assert std[i][key] == stg[i][key], (i, key)
    assert std[0]["steps_done"] == 12


def test_capture_refuses_a_wavelet_the_device_cannot_hold(P):
    torch_cuda()
    probs = _problems(P, with_source=True)
    d, fields, ((x, y, z), w) = probs[2]
    probs[2] = (d, fields, ((x, y, z), np.zeros(70000, np.float32)))
    b = _batch(P, probs)
    try:
        with pytest.raises(P.OOCSError) as e:
            b.capture(4)
        assert e.value.status == 7
        b.step(2)  # the batch stays usable
        b.synchronize(60.0)
    finally:
        b.close()


def test_replays_and_direct_steps_interleave(P):
    """Direct steps between replays move every problem's time index; the next
    replay continues from it (source included)."""
    torch_cuda()
    probs = _problems(P, with_source=True)
    outs = []
    for mode in ("direct", "mixed"):
        b = _batch(P, probs)
        try:
            if mode == "direct":
                for n in (4, 3, 4):
                    b.step(n)
            else:
                b.capture(4)
                b.launch()
                b.step(3)
                b.launch()
            b.synchronize(120.0)
            outs.append([[s.numpy().copy() for s in bp.stores] for bp in b.problems])
        finally:
            b.close()
    for i in range(len(probs)):
        for a, c in zip(outs[0][i], outs[1][i]):
            assert np.array_equal(a, c), i


def test_tuned_problems_run_as_a_batch(P, tmp_path):
    """The autotuner times real candidates and returns plans that run as a batch
    (and give the stores of each problem run alone)."""
    torch_cuda()
    from paper_2204_11315_gb300 import autotune
    probs = _problems(P, with_source=False)[1:3]
    descs, rep = autotune.tune([d for d, _, _ in probs], 2e-3, 2 << 30, str(tmp_path / "t.json"), steps=2)
    assert rep["candidates_timed"] > 0
    assert all(r["rate"] in (12, 16) for r in rep["problems"])
    tuned = [(d, f, s) for d, (_, f, s) in zip(descs, probs)]
    b = _batch(P, tuned)
    try:
        b.step(6)
        b.synchronize(120.0)
        got = [[s.numpy().copy() for s in bp.stores] for bp in b.problems]
    finally:
        b.close()
    for i, (d, fields, src) in enumerate(tuned):
        ref, _ = _alone(P, d, fields, src, [6])
        assert np.array_equal(got[i][0], ref[0])


def test_batch_mixing_codecs_matches_problems_run_alone(P):
    """Members of one batch keep their own codec (transform or block quantiser):
    each ends with the stores it gets when it runs alone."""
    torch_cuda()
    probs = []
    u = synthetic.heat_initial(64)
    probs.append((heat_desc(P, u.shape, rate=16, k=2, T=32, codec=1), {0: u}, None))
    probs.append((heat_desc(P, u.shape, rate=16, k=2, T=32, codec=0), {0: u}, None))
    shape = (96, 48, 64)
    m = synthetic.wave_model(shape)
    z = np.zeros(shape, np.float32)
    src = (synthetic.centre(shape)[::-1], synthetic.ricker(40))
    probs.append((wave_desc(P, shape, rate=20, k=3, T=24, ro=1, codec=1), {0: z, 1: z, 2: m}, src))
    b = _batch(P, probs)
    try:
        b.step(8)
        b.synchronize(120.0)
        got = [[s.numpy().copy() for s in bp.stores] for bp in b.problems]
    finally:
        b.close()
    for i, (d, fields, s) in enumerate(probs):
        ref, _ = _alone(P, d, fields, s, [8])
        for f in range(2 if d.scheme == P.OOCS_WAVE else 1):
            assert np.array_equal(got[i][f], ref[f]), (i, f)


def test_batch_members_match_the_oracle(P, orc):
    """One batch step of a mixed batch (heat at rate 16 and uncompressed, wave
    at rate 16 and uncompressed with a resident model, each with a source),
    every member checked against the FP64 oracle run of its own problem,
    point by point and in rel-L2, within the bars of its rate."""
    from gpu_util import assert_compressed, assert_uncompressed
    torch_cuda()
    steps = 12
    probs = []
    u = synthetic.uniform_field((64, 36, 44), 21)
    probs.append((heat_desc(P, u.shape, rate=16, k=4, T=16), {0: u}, None, ("heat", u)))
    u = synthetic.uniform_field((48, 40, 52), 22)
    probs.append((heat_desc(P, u.shape, rate=0, k=3, T=12, alpha=0.12), {0: u}, None, ("heat12", u)))
    for shape, rate, ro in (((96, 40, 48), 16, 0), ((64, 44, 36), 0, 1)):
        m = synthetic.wave_model(shape)
        z = np.zeros(shape, np.float32)
        w = synthetic.ricker(steps)
        probs.append((wave_desc(P, shape, rate=rate, k=2, T=32, ro=ro), {0: z, 1: z, 2: m},
                      (synthetic.centre(shape)[::-1], w), ("wave", z, m, w, shape)))
    b = _batch(P, [(d, f, s) for d, f, s, _ in probs])
    try:
        b.step(steps)
        b.synchronize(300.0)
        got = []
        for bp in b.problems:
            out = bp.decompress(P.OOCS_FIELD_U)
            bp.synchronize(120.0)
            got.append(out.numpy().copy())
    finally:
        b.close()
    for g, (d, _, _, ref_in) in zip(got, probs):
        if ref_in[0].startswith("heat"):
            alpha = 0.12 if ref_in[0] == "heat12" else 0.1
            ref = orc.heat_run(ref_in[1], synthetic.heat_star_coef(alpha), steps)
            scheme = "heat"
        else:
            _, z, m, w, shape = ref_in
            ref, _ = orc.wave_run(z, z, m, synthetic.wave_star_coef(), steps, src=synthetic.centre(shape), w=w)
            scheme = "wave"
        if int(d.rate_bits):
            assert_compressed(g, ref, int(d.rate_bits), f"{scheme} rate {int(d.rate_bits)}")
        else:
            assert_uncompressed(g, ref, scheme, f"{scheme} uncompressed")
