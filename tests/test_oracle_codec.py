"""Pins of the reference block codec (oracle/oracle.c, part 2).

The paper integrates a fixed-rate transform codec (Sec. 4.2, Sec. 5: rate 32
bits per double) without describing it; the oracle follows the published ZFP
method.  These tests tie every stage to something other than itself:
exact sizes from the rate, the published 4-point transform matrix, base -2
digit expansions, lossless and embedded (prefix) bit-plane coding, and a
per-block error bound derived from the stages.
"""
import math
import os

import numpy as np
import pytest

import synthetic

RATES = [1, 2, 4, 8, 12, 16, 20, 24, 32]
INV_GAIN = 3.75          # L-inf norm of the inverse 4-point transform (published matrix)


def test_exact_compressed_size(orc):
    """Fixed rate: a field of N values at rate R takes exactly N*R/8 bytes."""
    for shape in [(4, 4, 4), (8, 12, 16), (12, 8, 4)]:
        f = synthetic.blocks_field(shape, 1, "noise")
        for rate in RATES:
            words = orc.encode_field(f, rate)
            assert words.nbytes == f.size * rate // 8


def test_negabinary_is_base_minus_two(orc):
    rng = np.random.default_rng(0)
    vals = [0, 1, -1, 2, -2, 3, 2 ** 29 - 1, -(2 ** 29) + 1, 2 ** 30, -(2 ** 30), 123456789, -987654321]
    vals += [int(x) for x in rng.integers(-(2 ** 31), 2 ** 31, 2000)]
    for x in vals:
        u = orc.to_negabinary(x)
        digits = sum(((u >> i) & 1) * (-2) ** i for i in range(32))
        # the 32-digit base -2 expansion equals x modulo 2^32
        assert (digits - x) % (1 << 32) == 0
        assert orc.from_negabinary(u) == x
    # injective on a random sample
    us = {orc.to_negabinary(int(x)) for x in rng.integers(-(2 ** 31), 2 ** 31, 5000)}
    assert len(us) > 4990
    # small magnitudes have few significant digits (what makes bit planes compressible)
    for x in range(-10, 11):
        assert orc.to_negabinary(x) < 64


def test_lift_matches_published_matrix(orc):
    """Forward 4-point transform = (1/16) [[4,4,4,4],[5,1,-1,-5],[-4,4,4,-4],[-2,6,-6,2]]."""
    F = np.array([[4, 4, 4, 4], [5, 1, -1, -5], [-4, 4, 4, -4], [-2, 6, -6, 2]]) / 16.0
    s = 1 << 24
    for j in range(4):
        e = np.zeros(4, np.int64)
        e[j] = s
        assert np.allclose(orc.fwd_lift4(e) / s, F[:, j], atol=1e-6)
    Finv = np.linalg.inv(F)
    for j in range(4):
        e = np.zeros(4, np.int64)
        e[j] = s
        assert np.allclose(orc.inv_lift4(e) / s, Finv[:, j], atol=1e-6)
    assert abs(np.max(np.sum(np.abs(Finv), axis=1)) - INV_GAIN) < 1e-12
    # linear data: only the first two coefficients survive (decorrelation)
    c = orc.fwd_lift4([1000, 2000, 3000, 4000])
    assert abs(c[2]) <= 1 and abs(c[3]) <= 1


def test_xform_range_and_roundtrip(orc):
    rng = np.random.default_rng(1)
    worst = 0
    lim = (1 << 29) - 1
    for t in range(4000):
        kind = t % 4
        if kind == 0:
            q = rng.integers(-lim, lim + 1, 64)
        elif kind == 1:
            q = rng.choice([-lim, lim], 64)
        elif kind == 2:
            q = rng.integers(-40, 41, 64)
        else:
            q = np.cumsum(rng.integers(-5000, 5000, 64)).clip(-lim, lim)
        c = orc.fwd_xform(q)
        assert np.max(np.abs(c.astype(np.int64))) < (1 << 30)
        r = orc.inv_xform(c)
        worst = max(worst, int(np.max(np.abs(r.astype(np.int64) - q))))
    assert not orc.xform_overflowed()
    assert worst <= 32
    # the DC of a constant block is the constant, and nothing else survives
    c = orc.fwd_xform(np.full(64, 777))
    assert c[0] == 777 and np.all(c[1:] == 0)


def test_sequency_order(orc):
    perm = orc.sequency_order()
    assert sorted(perm.tolist()) == list(range(64))
    seq = [(p & 3) + ((p >> 2) & 3) + (p >> 4) for p in perm]
    assert seq == sorted(seq)
    assert perm[0] == 0 and perm[-1] == 63
    assert set(perm[1:4].tolist()) == {1, 4, 16}


def test_bitplane_coder_lossless_and_embedded(orc):
    rng = np.random.default_rng(2)
    full = 64 * 32 + 64 + 32  # enough for every plane of every coefficient
    for t in range(300):
        kind = t % 3
        if kind == 0:
            u = rng.integers(0, 2 ** 32, 64, dtype=np.uint64).astype(np.uint32)
        elif kind == 1:   # decaying magnitudes, as after a decorrelating transform
            u = (rng.integers(0, 2 ** 20, 64) >> np.minimum(np.arange(64) // 3, 19)).astype(np.uint32)
        else:
            u = np.zeros(64, np.uint32)
            u[rng.integers(0, 64, 3)] = rng.integers(1, 2 ** 31, 3)
        w = orc.encode_planes(u, full)
        dec, low = orc.decode_planes(w, full)
        assert np.array_equal(dec, u)
        assert low == 0
        # embedded: a shorter budget codes a prefix of the same bit string
        b = int(rng.integers(1, 1500))
        ws = orc.encode_planes(u, b)
        bits_full = np.unpackbits(w.view(np.uint8), bitorder="little")[:b]
        bits_short = np.unpackbits(ws.view(np.uint8), bitorder="little")
        assert np.array_equal(bits_short[:b], bits_full)
        assert not bits_short[b:].any()
        # and the truncated decode agrees with the coefficients on every complete plane
        dec_s, low_s = orc.decode_planes(ws, b)
        mask = np.uint32(0xFFFFFFFF) << np.uint32(low_s) if low_s < 32 else np.uint32(0)
        assert np.array_equal(dec_s & mask, u & mask)


def test_zero_and_constant_blocks(orc):
    z = np.zeros(64, np.float32)
    z[5] = -0.0
    for rate in RATES:
        w = orc.encode_block(z, rate)
        assert not w.any()
        v, _ = orc.decode_block(w, rate)
        assert np.all(v == 0.0)
    for rate in [2, 4, 8, 16]:
        c = np.full(64, -3.140625, np.float32)
        v, _ = orc.decode_block(orc.encode_block(c, rate), rate)
        assert np.array_equal(v, c)


def test_block_floating_point(orc):
    rng = np.random.default_rng(3)
    for t in range(500):
        scale = 2.0 ** rng.integers(-90, 100)
        v = (rng.standard_normal(64) * scale).astype(np.float32)
        h = orc.block_header(v)
        emax = h - 127
        m = np.max(np.abs(v.astype(np.float64)))
        assert 2.0 ** (emax - 1) <= m < 2.0 ** emax or emax == -95
        q = orc.quantize(v, emax)
        assert np.max(np.abs(q.astype(np.int64))) < 2 ** 29
        back = orc.dequantize(q, emax).astype(np.float64)
        # truncation toward zero: never larger in magnitude, error below one step
        assert np.all(np.abs(back) <= np.abs(v.astype(np.float64)))
        assert np.max(np.abs(back - v)) < 2.0 ** (emax - 29)
    # values on the quantisation grid are kept exactly
    v = (np.arange(64) - 31.0).astype(np.float32) * np.float32(2.0 ** -3)
    emax = orc.block_header(v) - 127
    assert np.array_equal(orc.dequantize(orc.quantize(v, emax), emax), v)
    # the exponent clamp: a block below 2^-124 quantises to zero
    tiny = np.full(64, 2.0 ** -126, np.float32)
    assert orc.block_header(tiny) - 127 == -95
    assert not orc.quantize(tiny, -95).any()


@pytest.mark.parametrize("kind", ["noise", "smooth", "mixed", "tiny", "huge", "const"])
def test_error_bound_every_block(orc, kind):
    """|v' - v| <= (G^3 2^p + 33) 2^(emax-29) + ulp(v')/2 for every value, where p is the
    lowest completely decoded plane and G = 3.75 the inverse transform gain.

    Coefficient planes >= p are exact, so each coefficient is off by < 2^p; the
    inverse transform multiplies that by at most G per dimension; lifting
    round-off adds at most 32 units (round trip, test above) and quantisation
    truncation one more; the final FP32 rounding adds half an ulp.
    """
    shape = (8, 8, 12)
    f = synthetic.blocks_field(shape, 11, kind)
    for rate in RATES:
        words = orc.encode_field(f, rate)
        g, low = orc.decode_field(words, shape, rate, with_planes=True)
        fb = f.reshape(2, 4, 2, 4, 3, 4).transpose(0, 2, 4, 1, 3, 5).reshape(-1, 64).astype(np.float64)
        gb = g.reshape(2, 4, 2, 4, 3, 4).transpose(0, 2, 4, 1, 3, 5).reshape(-1, 64).astype(np.float64)
        for b in range(fb.shape[0]):
            h = orc.block_header(fb[b].astype(np.float32))
            if h == 0:
                assert np.all(gb[b] == 0)
                continue
            unit = 2.0 ** (h - 127 - 29)
            p = int(low[b])
            fin = np.isfinite(gb[b])
            ulp_half = np.where(fin, np.spacing(np.where(fin, np.abs(gb[b]), 0).astype(np.float32)), 0).astype(np.float64) / 2
            bound = (INV_GAIN ** 3 * 2.0 ** p + 33.0) * unit + ulp_half
            assert np.all(np.abs(gb[b] - fb[b])[fin] <= bound[fin]), (kind, rate, b)
            # a value may round past FLT_MAX only where the bound reaches beyond it
            big = np.float64(np.finfo(np.float32).max)
            assert np.all(np.abs(fb[b])[~fin] + bound[~fin] >= big), (kind, rate, b)


def test_error_falls_with_rate(orc):
    for kind in ["noise", "smooth"]:
        f = synthetic.blocks_field((16, 16, 16), 4, kind)
        errs = []
        for rate in [4, 8, 12, 16, 24]:
            g = orc.decode_field(orc.encode_field(f, rate), f.shape, rate)
            errs.append(np.linalg.norm((g - f).ravel()) / np.linalg.norm(f.ravel()))
        # strictly better with rate until the FP32 rounding floor is reached
        assert all(errs[i + 1] < errs[i] or errs[i] < 2e-8 for i in range(len(errs) - 1)), errs
        assert all(errs[i + 1] <= errs[i] for i in range(len(errs) - 1)), errs
    # about one more bit of precision per extra bit of rate on noise
    f = synthetic.blocks_field((16, 16, 16), 4, "noise")
    e8 = np.linalg.norm(orc.decode_field(orc.encode_field(f, 8), f.shape, 8) - f)
    e16 = np.linalg.norm(orc.decode_field(orc.encode_field(f, 16), f.shape, 16) - f)
    assert 2 ** 6 < e8 / e16 < 2 ** 10


def test_block_layout_in_field(orc):
    """Block (bx, by, bz) is at word offset ((bz*(ny/4)+by)*(nx/4)+bx)*2*rate."""
    shape = (8, 12, 16)
    f = synthetic.blocks_field(shape, 2, "noise")
    rate = 8
    words = orc.encode_field(f, rate)
    for (bz, by, bx) in [(0, 0, 0), (1, 2, 3), (1, 0, 2), (0, 2, 1)]:
        blk = f[4 * bz:4 * bz + 4, 4 * by:4 * by + 4, 4 * bx:4 * bx + 4].reshape(64)
        off = ((bz * 3 + by) * 4 + bx) * 2 * rate
        assert np.array_equal(words[off:off + 2 * rate], orc.encode_block(blk, rate))


@pytest.mark.parametrize("bad", [np.inf, -np.inf, np.nan])
def test_nonfinite_block_is_stored_as_zeros_and_reported(orc, bad):
    """The codec is defined for finite values; a block holding an Inf or a NaN
    is written as an all-zero block and reported, by both codecs, and the other
    blocks of a field are coded as if it were not there."""
    rng = np.random.default_rng(11)
    v = rng.standard_normal(64).astype(np.float32)
    clean = orc.encode_block(v, 16)
    v[37] = bad
    for enc in (orc.encode_block, orc.bq_encode_block):
        words, flagged = enc(v, 16, with_flag=True)
        assert flagged and not words.any()
    assert not orc.encode_block(np.ones(64, np.float32), 16, with_flag=True)[1]
    f = rng.standard_normal((8, 8, 8)).astype(np.float32)
    ref = orc.encode_field(f, 12).reshape(8, 24)
    f[5, 1, 6] = bad  # block (bx, by, bz) = (1, 0, 1): index 5
    for enc in (orc.encode_field, orc.bq_encode_field):
        got, n = enc(f, 12, with_nonfinite=True)
        assert n == 1
        got = got.reshape(8, 24)
        assert not got[5].any()
    got = orc.encode_field(f, 12).reshape(8, 24)
    keep = [b for b in range(8) if b != 5]
    assert np.array_equal(got[keep], ref[keep])
    assert clean.any()


# ---------------------------------------------------------------------------
# A block worked by hand (tests/golden/xform_block_rate16.txt): pins every
# stage, the sequency tie-break and the group-test rule of the bitstream
# ---------------------------------------------------------------------------

XGOLDEN = os.path.join(os.path.dirname(__file__), "golden", "xform_block_rate16.txt")


def _xgolden():
    rows = {}
    for line in open(XGOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        key, *vals = line.split()
        rows[key] = vals
    return rows


def _xgolden_block(g):
    f, gg, h = ([int(x) for x in g[k]] for k in ("f", "g", "h"))
    v = np.zeros(64, np.float32)
    for k in range(4):
        for j in range(4):
            for i in range(4):
                v[i + 4 * j + 16 * k] = f[i] * gg[j] * h[k] / 64.0
    return v, f, gg, h


def test_worked_transform_block_stages(orc):
    g = _xgolden()
    v, f, gg, h = _xgolden_block(g)
    assert orc.block_header(v) == int(g["header"][0])
    emax = int(g["header"][0]) - 127
    q = orc.quantize(v, emax)
    assert [int(x) for x in q] == [f[i % 4] * gg[(i // 4) % 4] * h[i // 16] * 2 ** 22 for i in range(64)]
    c = orc.fwd_xform(q)
    want = np.zeros(64, np.int64)
    for item in g["coef"]:
        idx, val = item.split(":")
        want[int(idx)] = int(val)
    assert np.array_equal(np.asarray(c, np.int64), want)
    order = [int(x) for x in g["order"]]
    assert sorted(order) == list(range(64))
    assert list(orc.sequency_order()) == order
    nb = np.zeros(64, np.uint32)
    for item in g["negabinary"]:
        pos, val = item.split(":")
        nb[int(pos)] = int(val, 16)
    assert np.array_equal(np.array([orc.to_negabinary(int(c[order[n]])) for n in range(64)], np.uint32), nb)


def _pack_bits(bitstring, nwords):
    bits = bitstring.ljust(32 * nwords, "0")[:32 * nwords]
    return np.array([int(bits[32 * i:32 * i + 32][::-1], 2) for i in range(nwords)], np.uint32)


@pytest.mark.parametrize("rate", [16, 8, 1])
def test_worked_transform_block_bitstream(orc, rate):
    """The header bits (LSB first), the five empty planes, planes 26 and 25
    with their group tests, the verbatim planes 24 and 23, then zeros; cut at
    exactly 64 rate bits."""
    g = _xgolden()
    v, _, _, _ = _xgolden_block(g)
    bitstring = "".join(g["bits"])
    assert bitstring[:8] == format(int(g["header"][0]), "08b")[::-1]
    assert len(bitstring) == 8 + 5 + 7 + 24 + 22 + 22
    want = _pack_bits(bitstring, 2 * rate)
    assert np.array_equal(want[:3], np.array([int(w, 16) for w in g["words"]], np.uint32)[:2 * rate])
    assert np.array_equal(orc.encode_block(v, rate), want)
    if rate >= 8:  # everything significant fits: lossless
        back, low = orc.decode_block(want, rate)
        assert np.array_equal(back, v)
