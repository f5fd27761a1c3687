"""The block quantiser (OOCS_CODEC_QUANT) on the GPU against the oracle.

The simpler fixed-rate codec that the comparison of compression libraries
(Sec. 7, future work (1)) sets against the transform codec.  Device encode
must give the oracle's bytes and device decode its values, bit for bit, over
rates 2..32 and extreme blocks; oocs_compress / oocs_decompress go through
the same kernels; sweeps with the quantised store stay within an error bound
that follows from the codec's half-quantum bound.
"""
import numpy as np
import pytest

import synthetic
from gpu_util import heat_desc, rel_l2, streamed, torch_cuda, wave_desc

pytestmark = pytest.mark.gpu

QUANT = 1
KINDS = ["noise", "smooth", "mixed", "tiny", "huge", "const", "zero", "subnormal"]


@pytest.fixture(scope="module")
def P():
    import paper_2204_11315_gb300 as P
    P.lib()
    return P


def _field(shape, kind):
    if kind == "subnormal":
        f = synthetic.blocks_field(shape, 5, "noise").astype(np.float64) * 1e-39
        f[::3] = 0.0
        return f.astype(np.float32)
    return synthetic.blocks_field(shape, 5, kind)


def _encode(P, f, rate):
    torch = torch_cuda()
    nz, ny, nx = f.shape
    d = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    out = torch.full(((nx // 4) * (ny // 4) * (nz // 4) * 2 * rate,), -1, dtype=torch.int32, device="cuda")
    P.oocs_encode_device(d.data_ptr(), nx, ny, nz, rate, out.data_ptr(), torch.cuda.current_stream().cuda_stream,
                         codec=QUANT)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


def _decode(P, words, shape, rate):
    torch = torch_cuda()
    nz, ny, nx = shape
    w = torch.from_numpy(np.ascontiguousarray(words).view(np.int32)).cuda()
    out = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
    P.oocs_decode_device(w.data_ptr(), nx, ny, nz, rate, out.data_ptr(), torch.cuda.current_stream().cuda_stream,
                         codec=QUANT)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("rate", [2, 5, 8, 12, 16, 23, 25, 32])
def test_encode_decode_match_oracle(P, orc, kind, rate):
    shape = (12, 20, 36)  # 135 blocks: a ragged tail on the 128-thread CTA
    f = _field(shape, kind)
    ref = orc.bq_encode_field(f, rate)
    assert np.array_equal(_encode(P, f, rate), ref)
    assert np.array_equal(_decode(P, ref, shape, rate).view(np.uint32),
                          orc.bq_decode_field(ref, shape, rate).view(np.uint32))


def test_decode_arbitrary_words(P, orc):
    """Any word pattern (headers 1..255, negative fields the encoder never
    writes, overflow to infinity) decodes as the oracle decodes it."""
    rng = np.random.default_rng(11)
    shape = (8, 8, 16)
    for rate in [2, 9, 16, 26, 32]:
        w = rng.integers(0, 2 ** 32, 16 * 2 * rate, dtype=np.uint64).astype(np.uint32)
        got = _decode(P, w, shape, rate)
        ref = orc.bq_decode_field(w, shape, rate)
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_argument_errors(P):
    torch = torch_cuda()
    buf = torch.empty(4096, dtype=torch.float32, device="cuda")
    with pytest.raises(P.OOCSError):
        P.oocs_encode_device(buf.data_ptr(), 4, 4, 4, 1, buf.data_ptr(), codec=QUANT)  # rate >= 2
    with pytest.raises(P.OOCSError):
        P.oocs_encode_device(buf.data_ptr(), 4, 4, 4, 8, buf.data_ptr(), codec=2)
    with pytest.raises(P.OOCSError):
        P.oocs_query(heat_desc(P, (16, 16, 16), rate=1, k=1, T=16, codec=QUANT))


def test_store_holds_the_oracle_bytes(P, orc):
    """oocs_compress writes exactly the oracle quantiser's bytes into the host
    store, and oocs_decompress returns the oracle's decoded values."""
    u0 = synthetic.heat_initial(64)
    desc = heat_desc(P, u0.shape, rate=12, k=1, T=16, codec=QUANT)
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
    ref = orc.bq_encode_field(u0, 12)
    assert np.array_equal(got, ref)
    assert np.array_equal(back.view(np.uint32), orc.bq_decode_field(ref, u0.shape, 12).view(np.uint32))


def _block_max_norm(u):
    """|| B(u) ||_2, B(u) = every value replaced by its 4x4x4 block's max |u|."""
    nz, ny, nx = u.shape
    b = np.abs(u.astype(np.float64)).reshape(nz // 4, 4, ny // 4, 4, nx // 4, 4).max(axis=(1, 3, 5))
    return float(np.sqrt(64.0 * np.sum(b * b)))


@pytest.mark.parametrize("rate", [16, 12])
def test_heat_sweep_within_the_quantisation_bound(P, orc, rate):
    """A quantisation moves a value by at most half its block's quantum,
    2^(emax-q) <= 2^(1-q) max|block|, so one pass adds at most 2^(1-q)||B(u)||
    in L2; the explicit heat step (alpha = 0.1) does not amplify L2 errors, so
    after P passes (one per step at k = 1, one initial encode) the error is at
    most (P + 1) 2^(1-q) max ||B(u)|| plus the FP32 bar."""
    u0 = synthetic.heat_initial(128)
    steps = 10
    desc = heat_desc(P, u0.shape, rate=rate, k=1, T=32, codec=QUANT)
    got, _, _, _, plan = streamed(P, desc, u0, steps)
    ref = orc.heat_run(u0, synthetic.heat_star_coef(0.1), steps)
    q = rate - 1
    bound = (steps + 1) * 2.0 ** (1 - q) * _block_max_norm(u0) / np.linalg.norm(ref) + synthetic.TOL_UNCOMPRESSED["heat"]
    err = rel_l2(got, ref)
    assert err <= bound, (err, bound)
    assert err > 0.0  # the store is lossy at this rate
    assert plan.host_store_bytes == u0.size * rate // 8


def test_wave_sweep_within_the_quantisation_bound(P, orc):
    """Wave, 100 steps in 25 passes of k = 4, both u and u_prev quantised each
    pass: (2 x 26) 2^(1-q) max_t ||B(u^t)|| / ||u||, doubled because the
    leapfrog scheme conserves rather than dissipates energy."""
    shape = (128, 128, 128)
    steps, rate = 100, 16
    m = synthetic.wave_model(shape)
    w = synthetic.ricker(steps)
    cz, cy, cx = synthetic.centre(shape)
    z = np.zeros(shape, np.float32)
    desc = wave_desc(P, shape, rate=rate, k=4, T=32, ro=1, codec=QUANT)
    gu, gup, _, _, _ = streamed(P, desc, z, steps, up0=z, m=m, src=(cx, cy, cz), w=w)
    ru, rup = orc.wave_run(z, z, m, synthetic.wave_star_coef(), steps, src=(cz, cy, cx), w=w)
    q = rate - 1
    bmax = max(_block_max_norm(ru.astype(np.float32)), _block_max_norm(rup.astype(np.float32)))
    bound = 2 * 2 * 26 * 2.0 ** (1 - q) * bmax / np.linalg.norm(ru) + synthetic.TOL_UNCOMPRESSED["wave"]
    assert rel_l2(gu, ru) <= bound, (rel_l2(gu, ru), bound)
    assert rel_l2(gup, rup) <= bound
