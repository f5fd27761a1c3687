"""GPU codec kernels against the CPU reference codec: byte-identical bytes, bit-identical values.

Fixed-rate block codec of Sec. 4.2 (rate in bits/value); the CUDA side is
reached through the C ABI (oocs_encode_device / oocs_decode_device).
"""
import numpy as np
import pytest

import synthetic
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu

KINDS = ["noise", "smooth", "mixed", "tiny", "huge", "const", "zero"]


@pytest.fixture(scope="module")
def P():
    import paper_2204_11315_gb300 as P
    P.lib()
    return P


def gpu_encode(P, f, rate):
    torch = torch_cuda()
    nz, ny, nx = f.shape
    d = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    nb = (nx // 4) * (ny // 4) * (nz // 4)
    out = torch.full((nb * 2 * rate,), -1, dtype=torch.int32, device="cuda")
    P.oocs_encode_device(d.data_ptr(), nx, ny, nz, rate, out.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


def gpu_decode(P, words, shape, rate):
    torch = torch_cuda()
    nz, ny, nx = shape
    w = torch.from_numpy(np.ascontiguousarray(words).view(np.int32)).cuda()
    out = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
    P.oocs_decode_device(w.data_ptr(), nx, ny, nz, rate, out.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("rate", [1, 3, 8, 12, 16, 24, 32])
def test_encode_decode_match_reference(P, orc, kind, rate):
    # 9 x 5 x 3 blocks: not a multiple of the 128-thread CTA, ragged tail
    shape = (12, 20, 36)
    f = synthetic.blocks_field(shape, 3, kind)
    ref_words = orc.encode_field(f, rate)
    got_words = gpu_encode(P, f, rate)
    assert np.array_equal(got_words, ref_words)
    ref_vals = orc.decode_field(ref_words, shape, rate)
    got_vals = gpu_decode(P, ref_words, shape, rate)
    assert np.array_equal(got_vals.view(np.uint32), ref_vals.view(np.uint32))


def test_decode_arbitrary_words(P, orc):
    """Any word pattern decodes identically (two's-complement wrap is part of the definition)."""
    rng = np.random.default_rng(9)
    shape = (8, 8, 16)
    nb = 2 * 2 * 4
    for rate in [2, 7, 16, 31]:
        w = rng.integers(0, 2 ** 32, nb * 2 * rate, dtype=np.uint64).astype(np.uint32)
        ref = orc.decode_field(w, shape, rate)
        got = gpu_decode(P, w, shape, rate)
        assert np.array_equal(np.nan_to_num(got).view(np.uint32), np.nan_to_num(ref).view(np.uint32))


def test_full_size_sampled_blocks(P, orc):
    """512 x 512 x 64 layered-model slab at rate 16: sampled blocks against the reference."""
    shape = (64, 512, 512)
    f = synthetic.wave_model(shape)
    rate = 16
    words = gpu_encode(P, f, rate).reshape(-1, 2 * rate)
    rng = np.random.default_rng(4)
    bnz, bny, bnx = 16, 128, 128
    for b in rng.integers(0, bnz * bny * bnx, 400):
        bz, by, bx = b // (bny * bnx), (b // bnx) % bny, b % bnx
        blk = f[4 * bz:4 * bz + 4, 4 * by:4 * by + 4, 4 * bx:4 * bx + 4].reshape(64)
        assert np.array_equal(words[b], orc.encode_block(blk, rate))
    back = gpu_decode(P, words.reshape(-1), shape, rate)
    for b in rng.integers(0, bnz * bny * bnx, 400):
        bz, by, bx = b // (bny * bnx), (b // bnx) % bny, b % bnx
        v, _ = orc.decode_block(words[b], rate)
        got = back[4 * bz:4 * bz + 4, 4 * by:4 * by + 4, 4 * bx:4 * bx + 4].reshape(64)
        assert np.array_equal(got.view(np.uint32), v.view(np.uint32))


def test_argument_errors(P):
    torch = torch_cuda()
    buf = torch.empty(1024, dtype=torch.float32, device="cuda")
    with pytest.raises(P.OOCSError):
        P.oocs_encode_device(buf.data_ptr(), 6, 4, 4, 8, buf.data_ptr())
    with pytest.raises(P.OOCSError):
        P.oocs_encode_device(buf.data_ptr(), 4, 4, 4, 33, buf.data_ptr())
    with pytest.raises(P.OOCSError):
        P.oocs_decode_device(buf.data_ptr() + 4, 4, 4, 4, 8, buf.data_ptr())


@pytest.mark.parametrize("rate", [16, 8, 1])
def test_worked_block_on_the_gpu(P, rate):
    """The block worked by hand in tests/golden/xform_block_rate16.txt, encoded
    by the GPU kernel: exactly the hand-derived words (and decoded back exactly
    where the whole stream fits)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "xform_block_rate16.txt")
    rows = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            key, *vals = line.split()
            rows[key] = vals
    f, g, h = ([int(x) for x in rows[k]] for k in ("f", "g", "h"))
    blk = np.array([[[f[i] * g[j] * h[k] / 64.0 for i in range(4)] for j in range(4)] for k in range(4)],
                   np.float32)
    bits = "".join(rows["bits"]).ljust(64 * rate, "0")[:64 * rate]
    want = np.array([int(bits[32 * i:32 * i + 32][::-1], 2) for i in range(2 * rate)], np.uint32)
    got = gpu_encode(P, blk, rate)
    assert np.array_equal(got, want)
    if rate >= 8:
        assert np.array_equal(gpu_decode(P, want, blk.shape, rate), blk)
