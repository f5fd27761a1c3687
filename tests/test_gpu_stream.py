"""Out-of-core slab streaming (oocs_step) on the GPU.

Uncompressed: the slab-streamed run (z-slabs, temporal blocking with halo
h = 4 ceil(k r / 4), region sharing, single working buffer; Sec. 3.1, Sec. 5,
Algorithm 1) must be bit-exact against the in-core GPU run of the same FP32
arithmetic.  Compressed (Sec. 4): within the per-rate bar of the FP64 oracle.
"""
import numpy as np
import pytest

import synthetic
from gpu_util import assert_compressed, heat_desc, incore, streamed, wave_desc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2204_11315_gb300 as P
    P.lib()
    return P


# ------------------------------------------------------------- heat ------

@pytest.mark.parametrize("k", [1, 2, 5])
@pytest.mark.parametrize("wb", [1, 3])
def test_heat_streamed_bitexact_vs_incore(P, k, wb):
    u0 = synthetic.heat_initial(128)
    desc = heat_desc(P, u0.shape, rate=0, k=k, T=32, wb=wb)
    ref = incore(P, desc, u0, 10)
    got, _, _, stats, plan = streamed(P, desc, u0, 10)
    assert plan.num_slabs == 4
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    # region sharing: every layer crosses the link once per sweep in each direction
    passes = -(-10 // k)
    assert stats["passes_done"] == passes
    assert stats["h2d_bytes"] == passes * plan.host_store_bytes
    assert stats["d2h_bytes"] == passes * plan.host_store_bytes


@pytest.mark.parametrize("shape,T,k", [((120, 52, 44), 32, 3), ((64, 36, 100), 8, 2),
                                       ((40, 16, 24), 64, 4)])
def test_heat_ragged_slabs_bitexact(P, shape, T, k):
    """Last slab thinner than T, x-y sizes off the tile grid, one-slab case."""
    u0 = synthetic.uniform_field(shape, 5)
    desc = heat_desc(P, shape, rate=0, k=k, T=T, alpha=0.12)
    ref = incore(P, desc, u0, 7)
    got, _, _, _, _ = streamed(P, desc, u0, 7, chunks=[3, 4])
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("rate", [16, 12, 8])
def test_heat_compressed_within_tolerance(P, orc, rate):
    u0 = synthetic.heat_initial(128)
    desc = heat_desc(P, u0.shape, rate=rate, k=1, T=32)
    got, _, stores, stats, plan = streamed(P, desc, u0, 10)
    ref = orc.heat_run(u0, synthetic.heat_star_coef(0.1), 10)
    assert_compressed(got, ref, rate, f"heat rate {rate}")
    # fixed rate: exactly rate bits per value in the store and over the link
    assert plan.host_store_bytes == u0.size * rate // 8
    assert stats["h2d_bytes"] == 10 * plan.host_store_bytes


def test_compress_matches_reference_codec(P, orc):
    """oocs_compress writes exactly the reference codec's bytes into the host store."""
    u0 = synthetic.heat_initial(128)
    desc = heat_desc(P, u0.shape, rate=16, k=1, T=32)
    st = P.OutOfCoreStencil(desc)
    try:
        st.compress(P.OOCS_FIELD_U, u0)
        st.synchronize(60.0)
        got = st.stores[0].numpy().view(np.uint32).copy()
        back = st.decompress(P.OOCS_FIELD_U)
        st.synchronize(60.0)
        back = back.numpy().copy()
    finally:
        st.close()
    ref = orc.encode_field(u0, 16)
    assert np.array_equal(got, ref)
    assert np.array_equal(back.view(np.uint32), orc.decode_field(ref, u0.shape, 16).view(np.uint32))


# ------------------------------------------------------------- wave ------

def _wave_inputs(shape, steps):
    m = synthetic.wave_model(shape)
    w = synthetic.ricker(steps)
    cz, cy, cx = synthetic.centre(shape)
    z = np.zeros(shape, np.float32)
    return m, w, (cx, cy, cz), z


@pytest.mark.parametrize("shape,T,k,wb", [((128, 72, 40), 32, 4, 1), ((128, 72, 40), 32, 4, 3),
                                          ((96, 48, 64), 24, 3, 1), ((80, 40, 40), 16, 1, 1)])
def test_wave_streamed_bitexact_vs_incore(P, shape, T, k, wb):
    steps = 10
    m, w, src, z = _wave_inputs(shape, steps)
    desc = wave_desc(P, shape, rate=0, k=k, T=T, wb=wb)
    ru, rup = incore(P, desc, z, steps, up0=z, m=m, src=src, w=w)
    gu, gup, _, stats, plan = streamed(P, desc, z, steps, up0=z, m=m, src=src, w=w)
    assert np.array_equal(gu.view(np.uint32), ru.view(np.uint32))
    assert np.array_equal(gup.view(np.uint32), rup.view(np.uint32))
    passes = -(-steps // k)
    assert stats["h2d_bytes"] == 3 * passes * plan.host_store_bytes
    assert stats["d2h_bytes"] == 2 * passes * plan.host_store_bytes


def test_wave_split_calls_bitexact(P):
    """Several oocs_step calls continue the source time index and the state."""
    shape = (96, 40, 48)
    steps = 11
    m, w, src, z = _wave_inputs(shape, steps)
    desc = wave_desc(P, shape, rate=0, k=4, T=32)
    ru, rup = incore(P, desc, z, steps, up0=z, m=m, src=src, w=w)
    gu, gup, _, _, _ = streamed(P, desc, z, steps, up0=z, m=m, src=src, w=w, chunks=[5, 2, 4])
    assert np.array_equal(gu.view(np.uint32), ru.view(np.uint32))
    assert np.array_equal(gup.view(np.uint32), rup.view(np.uint32))


@pytest.mark.parametrize("rate", [16, 12, 8])
def test_wave_compressed_within_tolerance(P, orc, rate):
    shape = (128, 128, 128)
    steps = 100
    m, w, src, z = _wave_inputs(shape, steps)
    desc = wave_desc(P, shape, rate=rate, k=4, T=32)
    gu, gup, _, _, _ = streamed(P, desc, z, steps, up0=z, m=m, src=src, w=w)
    ru, rup = orc.wave_run(z, z, m, synthetic.wave_star_coef(), steps,
                           src=synthetic.centre(shape), w=w)
    assert_compressed(gu, ru, rate, f"wave u rate {rate}")
    assert_compressed(gup, rup, rate, f"wave u_prev rate {rate}")


@pytest.mark.parametrize("rate,wb", [(0, 1), (16, 1), (12, 3)])
def test_wave_resident_model_bitexact(P, rate, wb):
    """readonly_resident keeps m on the device (decoded once): the stores after
    the run are byte-identical to streaming m with every visit, and m crosses
    the link once instead of once per sweep (compressed, oocs_compress already
    decodes it into the device copy; raw, the first step copies it)."""
    shape = (128, 72, 40)
    steps = 10
    m, w, src, z = _wave_inputs(shape, steps)
    runs = [streamed(P, wave_desc(P, shape, rate=rate, k=4, T=32, wb=wb, ro=ro), z, steps, up0=z, m=m,
                     src=src, w=w) for ro in (0, 1)]
    (_, _, st0, _, p0), (_, _, st1, stats1, p1) = runs
    assert np.array_equal(st0[0], st1[0]) and np.array_equal(st0[1], st1[1])
    assert (p0.fields_in, p0.readonly_resident) == (3, 0)
    assert (p1.fields_in, p1.readonly_resident) == (2, 1)
    passes = -(-steps // 4)
    assert stats1["h2d_bytes"] == (2 * passes + (1 if rate == 0 else 0)) * p1.host_store_bytes


@pytest.mark.parametrize("ro", [0, 1])
def test_wave_full_size_uncompressed_bitexact(P, ro):
    """The benchmark workload's grid and plan (512^3, 8 slabs of 64, k = 4), uncompressed,
    with m streamed or resident."""
    shape = (512, 512, 512)
    steps = 12
    m, w, src, z = _wave_inputs(shape, steps)
    desc = wave_desc(P, shape, rate=0, k=4, T=64, budget=4 << 30, ro=ro)
    ru, rup = incore(P, desc, z, steps, up0=z, m=m, src=src, w=w)
    gu, gup, _, _, plan = streamed(P, desc, z, steps, up0=z, m=m, src=src, w=w)
    assert plan.num_slabs == 8 and plan.workspace_bytes <= 4 << 30
    assert np.array_equal(gu.view(np.uint32), ru.view(np.uint32))
    assert np.array_equal(gup.view(np.uint32), rup.view(np.uint32))


def test_budget_too_small(P):
    desc = wave_desc(P, (128, 128, 128), rate=16, k=4, T=0, budget=1 << 20)
    with pytest.raises(P.OOCSError) as e:
        P.oocs_query(desc)
    assert e.value.status == 2


def test_restore_and_set_time_repeat_the_run(P):
    """Resetting the host stores and the time index repeats the same run bit for bit."""
    shape = (64, 40, 48)
    steps = 9
    m, w, src, z = _wave_inputs(shape, steps)
    desc = wave_desc(P, shape, rate=12, k=4, T=32)
    st = P.OutOfCoreStencil(desc)
    try:
        st.compress(P.OOCS_FIELD_U, z)
        st.compress(P.OOCS_FIELD_U_PREV, z)
        st.compress(P.OOCS_FIELD_M, m)
        st.set_source(src[0], src[1], src[2], w)
        st.synchronize(60.0)
        snap = st.snapshot_stores()
        outs = []
        for _ in range(2):
            st.restore_stores(snap, 0)
            st.step(steps)
            st.synchronize(60.0)
            outs.append([s.numpy().copy() for s in st.stores])
        assert st.stats()["steps_done"] == steps
    finally:
        st.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)
    assert not np.array_equal(outs[0][0], snap[0].numpy())


@pytest.mark.slow
def test_wave_benchmark_plan_within_tolerance_of_oracle(P, orc):
    """The benchmark's exact configuration and plan (512^3, 100 steps, rate 16,
    m on the device, 8 slabs of 64, k = 4, one working buffer) against the
    FP64 oracle over the whole grid."""
    shape = (512, 512, 512)
    steps = 100
    m, w, src, z = _wave_inputs(shape, steps)
    desc = wave_desc(P, shape, rate=16, k=4, T=64, budget=4 << 30, ro=1)
    gu, gup, _, stats, plan = streamed(P, desc, z, steps, up0=z, m=m, src=src, w=w)
    assert plan.num_slabs == 8 and plan.readonly_resident == 1 and plan.workspace_bytes <= 4 << 30
    ru, rup = orc.wave_run(z, z, m, synthetic.wave_star_coef(), steps, src=synthetic.centre(shape), w=w)
    assert_compressed(gu, ru, 16, "512^3 wave u")
    assert_compressed(gup, rup, 16, "512^3 wave u_prev")


@pytest.mark.parametrize("rate", [16, 8, 32])
def test_compress_and_decompress_in_place(P, orc, rate):
    """The store living in the first bytes of the raw FP32 array itself (a field
    that fills host memory needs no second array): oocs_compress writes the
    oracle codec's bytes, the sweep runs on them, and oocs_decompress returns
    the same values as with separate arrays, over eight chunks on two streams."""
    import torch
    u0 = synthetic.heat_initial(128)
    desc = heat_desc(P, u0.shape, rate=rate, k=2, T=16)
    ref, _, ref_stores, _, _ = streamed(P, desc, u0, 6)
    buf = torch.empty(u0.size * 4, dtype=torch.uint8, pin_memory=True)
    raw = buf.view(torch.float32).reshape(u0.shape)
    raw.numpy()[...] = u0
    st = P.OutOfCoreStencil(desc, stores=[buf])
    try:
        assert st.stores[0].data_ptr() == raw.data_ptr()
        st.compress(P.OOCS_FIELD_U, raw)
        st.synchronize(60.0)
        assert np.array_equal(buf[:st.plan.host_store_bytes].numpy().view(np.uint32), orc.encode_field(u0, rate))
        st.step(6)
        st.synchronize(60.0)
        assert np.array_equal(buf[:st.plan.host_store_bytes].numpy(), ref_stores[0])
        st.decompress(P.OOCS_FIELD_U, raw)
        st.synchronize(60.0)
        assert np.array_equal(raw.numpy().view(np.uint32), ref.view(np.uint32))
    finally:
        st.close()
    if rate == 32:  # the store is the whole array: no room for an offset store
        return
    # an overlap that does not start at the array's address is refused
    st = P.OutOfCoreStencil(desc, stores=[buf[4096:]])
    try:
        with pytest.raises(P.OOCSError) as e:
            st.compress(P.OOCS_FIELD_U, raw)
        assert e.value.status == 1 and "in place" in str(e.value)
    finally:
        st.close()


@pytest.mark.parametrize("shape,T,k,rate", [((64, 200, 264), 24, 4, 0), ((64, 200, 264), 24, 4, 16),
                                            ((96, 72, 136), 32, 3, 0), ((40, 36, 52), 64, 2, 16),
                                            ((128, 128, 128), 32, 4, 12)])
def test_heat_fused_step_pairs_bitexact(P, shape, T, k, rate):
    """Heat steps fused in pairs (the middle step of each pair kept in shared
    memory, temporal blocking on chip) give the same stores and field, bit for
    bit, as one kernel per step: ragged tiles in x and y, windows clipped at
    both faces, an odd depth (a pair and a single step), several slabs."""
    u0 = synthetic.uniform_field(shape, 21)
    ref = None
    for fusion in (0, 1):
        nz, ny, nx = shape
        desc = P.make_desc(nx, ny, nz, P.OOCS_HEAT, synthetic.heat_star_coef(0.1), 8 << 30, rate_bits=rate,
                           temporal_depth=k, slab_planes=T, step_fusion=fusion)
        got, _, stores, stats, _ = streamed(P, desc, u0, 2 * k + 1)
        if ref is None:
            ref = (got, stores, stats)
        else:
            assert np.array_equal(got.view(np.uint32), ref[0].view(np.uint32))
            assert np.array_equal(stores[0], ref[1][0])
            assert stats["step"]["units"] == ref[2]["step"]["units"]
            assert stats["kernel_launches"] < ref[2]["kernel_launches"]
    if rate == 0:
        inc = incore(P, heat_desc(P, shape, rate=0, k=k, T=T), u0, 2 * k + 1)
        assert np.array_equal(ref[0].view(np.uint32), inc.view(np.uint32))


@pytest.mark.parametrize("shape,T,k,rate,wb,tile", [((64, 200, 264), 24, 4, 16, 1, 0),
                                                    ((96, 72, 136), 32, 3, 8, 1, 0),
                                                    ((40, 36, 52), 64, 1, 16, 1, 0),
                                                    ((128, 128, 128), 32, 4, 32, 1, 0),
                                                    ((64, 52, 68), 16, 2, 12, 3, 0),
                                                    ((64, 52, 68), 16, 3, 16, 1, 1)])
def test_heat_fused_codec_bitexact(P, shape, T, k, rate, wb, tile):
    """The codec fused into the steps (codec_fusion: step 1 decodes the window
    in shared memory, the last step encodes its layers in its epilogue)
    writes the same store bytes, and decodes to the same field, bit for bit,
    as the separate decode and encode kernels: tiles ragged in x and y, one
    or several layers per chunk, depths 1 to 4 (a visit of one step keeps its
    encode kernel), rates 8 to 32, several slabs, one or three working
    buffers."""
    u0 = synthetic.uniform_field(shape, 23)
    ref = None
    for fusion in (0, 1):
        nz, ny, nx = shape
        desc = P.make_desc(nx, ny, nz, P.OOCS_HEAT, synthetic.heat_star_coef(0.1), 8 << 30, rate_bits=rate,
                           temporal_depth=k, slab_planes=T, working_buffers=wb, codec_fusion=fusion,
                           step_tile=tile)
        got, _, stores, stats, plan = streamed(P, desc, u0, 2 * k + 1)
        if ref is None:
            ref = (got, stores, stats)
        else:
            assert np.array_equal(stores[0], ref[1][0])
            assert np.array_equal(got.view(np.uint32), ref[0].view(np.uint32))
            assert stats["store"]["units"] == ref[2]["store"]["units"]
            assert stats["load"]["units"] == ref[2]["load"]["units"]
            visits = stats["slabs_done"]
            one_step = plan.num_slabs * (3 if k == 1 else 1)  # 2k + 1 steps: visits of a single step
            assert stats["kernel_launches"] == ref[2]["kernel_launches"] - (2 * visits - one_step)


def test_fused_encode_flags_nonfinite_results(P):
    """A field whose step produces an infinity (the neighbour sum of a point
    inside a cube of 3e38 values overflows FP32) is reported by the fused
    epilogue like the separate encoder: OOCS_ERR_NONFINITE at oocs_synchronize."""
    shape = (32, 32, 32)
    u0 = synthetic.uniform_field(shape, 3)
    u0[15:18, 15:18, 15:18] = 3.0e38
    nz, ny, nx = shape
    desc = P.make_desc(nx, ny, nz, P.OOCS_HEAT, synthetic.heat_star_coef(0.1), 8 << 30, rate_bits=16,
                       temporal_depth=2, slab_planes=16, codec_fusion=1)
    st = P.OutOfCoreStencil(desc)
    try:
        st.compress(P.OOCS_FIELD_U, u0)
        st.synchronize(60.0)
        st.step(2)
        with pytest.raises(P.OOCSError) as e:
            st.synchronize(60.0)
        assert e.value.status == P.OOCS_ERR_NONFINITE
    finally:
        st.close()
