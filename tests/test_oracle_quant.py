"""Pins of the oracle's block quantiser (the simpler fixed-rate codec that the
comparison of compression libraries, Sec. 7 future work (1), sets against the
transform codec), against facts that do not come from the oracle itself: a
block worked by hand, numpy's frexp, a big-integer unpacking of the bit
layout, the half-quantum error bound, exactness on the quantisation grid,
idempotence and sign symmetry."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bq_block_rate16.txt")
RATES = (2, 5, 8, 12, 16, 23, 25, 32)


def _golden():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        key, *vals = line.split()
        rows[key] = vals
    return rows


def _unpack(words, rate):
    """Header and the 64 signed q-bit integers, read from the words as one
    little-endian big integer."""
    big = 0
    for i, w in enumerate(words):
        big |= int(w) << (32 * i)
    q = rate - 1
    hdr = big & 0xFF
    ns = []
    for j in range(64):
        u = (big >> (8 + j * q)) & ((1 << q) - 1)
        ns.append(u - (1 << q) if u >> (q - 1) else u)
    tail = big >> (8 + 64 * q)
    return hdr, ns, tail


def _blocks(seed, n=200):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        scale = 2.0 ** rng.integers(-60, 60)
        v = (rng.standard_normal(64) * scale).astype(np.float32)
        if i % 7 == 0:
            v[rng.integers(0, 64, 20)] = 0.0
        out.append(v)
    return out


def test_worked_block():
    g = _golden()
    rate = int(g["rate"][0])
    v = np.zeros(64, np.float32)
    v[:3] = [float(x) for x in g["input"]]
    w = oracle.bq_encode_block(v, rate)
    want = np.zeros(2 * rate, np.uint32)
    want[:2] = [int(x, 16) for x in g["words"]]
    assert np.array_equal(w, want)
    d = oracle.bq_decode_block(w, rate)
    assert list(d[:3]) == [float(x) for x in g["decoded"]] and not d[3:].any()


@pytest.mark.parametrize("rate", RATES)
def test_layout_header_and_error_bound(rate):
    q = rate - 1
    for v in _blocks(rate):
        w = oracle.bq_encode_block(v, rate)
        hdr, ns, tail = _unpack(w, rate)
        assert tail == 0  # the last 56 bits are zero
        mx = float(np.max(np.abs(v)))
        if mx == 0.0:
            assert hdr == 0 and not any(ns)
            continue
        emax = max(int(np.frexp(np.float32(mx))[1]), -126)
        assert hdr == emax + 127
        lim = 2 ** (q - 1) - 1
        assert all(-lim <= n <= lim for n in ns)
        d = oracle.bq_decode_block(w, rate).astype(np.float64)
        quantum = 2.0 ** (emax - q + 1)
        # decode = the stored integers times the quantum (exact when q <= 25)
        if q <= 24:
            assert np.array_equal(d, np.array(ns, np.float64) * quantum)
        err = np.abs(d - v.astype(np.float64))
        # half a quantum, plus half an FP32 ulp of the value when the integer
        # (q > 24) or the product (subnormal) is rounded; a clamped value
        # (v 2^(q-1-emax) >= lim + 1/2) is off by less than one quantum
        ulp = np.spacing(np.abs(v).astype(np.float32)).astype(np.float64)
        clamped = np.abs(v.astype(np.float64)) / quantum >= lim + 0.5
        bound = np.where(clamped, quantum, 0.5 * quantum) + 0.5 * ulp + 2.0 ** -149
        assert np.all(err <= bound), (rate, float(np.max(err / bound)))


@pytest.mark.parametrize("rate", [3, 8, 16, 25])
def test_grid_values_exact_and_idempotent(rate):
    q = rate - 1
    rng = np.random.default_rng(100 + rate)
    lim = 2 ** (q - 1) - 1
    for emax in (-120, -3, 0, 7, 100):
        n = rng.integers(-lim, lim + 1, 64)
        n[0] = lim  # a value whose frexp exponent is emax (or the grid's top)
        v = (n.astype(np.float64) * 2.0 ** (emax - q + 1)).astype(np.float32)
        d = oracle.bq_decode_block(oracle.bq_encode_block(v, rate), rate)
        assert np.array_equal(d, v)
    for v in _blocks(7 + rate, 50):
        w = oracle.bq_encode_block(v, rate)
        d = oracle.bq_decode_block(w, rate)
        if np.all((np.abs(d) >= 2.0 ** -126) | (d == 0)):
            assert np.array_equal(oracle.bq_encode_block(d, rate), w)


@pytest.mark.parametrize("rate", [4, 16])
def test_sign_symmetry_and_special_blocks(rate):
    for v in _blocks(50 + rate, 40):
        a = oracle.bq_decode_block(oracle.bq_encode_block(v, rate), rate)
        b = oracle.bq_decode_block(oracle.bq_encode_block(-v, rate), rate)
        assert np.array_equal(a, -b)
    z = np.zeros(64, np.float32)
    z[3] = -0.0
    assert not oracle.bq_encode_block(z, rate).any()
    sub = np.full(64, 1e-40, np.float32)  # subnormal: emax clamps to -126
    hdr, _, _ = _unpack(oracle.bq_encode_block(sub, rate), rate)
    assert hdr == 1
    big = np.full(64, np.float32(3.0e38))
    d = oracle.bq_decode_block(oracle.bq_encode_block(big, rate), rate)
    # one quantum 2^(emax - q + 1), emax = 128: the top value is clamped
    assert np.all(np.isfinite(d)) and np.all(np.abs(d.astype(np.float64) - 3.0e38) <= 2.0 ** (128 - rate + 2))


def test_field_layout():
    rng = np.random.default_rng(9)
    nz, ny, nx = 8, 12, 16
    f = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    rate = 11
    words = oracle.bq_encode_field(f, rate).reshape(nz // 4, ny // 4, nx // 4, 2 * rate)
    blocks = f.reshape(nz // 4, 4, ny // 4, 4, nx // 4, 4).transpose(0, 2, 4, 1, 3, 5)
    for bz in range(nz // 4):
        for by in range(ny // 4):
            for bx in range(nx // 4):
                v = blocks[bz, by, bx].reshape(64)  # index i + 4j + 16k
                assert np.array_equal(words[bz, by, bx], oracle.bq_encode_block(v, rate))
    g = oracle.bq_decode_field(words.reshape(-1), f.shape, rate)
    assert float(np.abs(g - f).max()) <= 2.0 ** (int(np.frexp(np.abs(f).max())[1]) - rate + 1)
