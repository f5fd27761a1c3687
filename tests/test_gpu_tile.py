"""The step kernel's two x-y tiles (oocs_desc.step_tile: 64 x 16 and 64 x 8
points per CTA) compute the same arithmetic per point in the same order, so
every result is bit-identical between them: in core, streamed out of core
(compressed and not), and in the adjoint and gradient entry points.  Shapes
with ny not a multiple of 8 or 16 cover ragged last tile rows."""
import numpy as np
import pytest

import synthetic
from gpu_util import heat_desc, incore, streamed, torch_cuda, wave_desc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2204_11315_gb300 as P
    P.lib()
    return P


def _tiled(desc, tile):
    desc.step_tile = tile
    return desc


def _same(a, b):
    return np.array_equal(np.asarray(a).view(np.uint32), np.asarray(b).view(np.uint32))


@pytest.mark.parametrize("shape", [(40, 52, 68), (36, 100, 132)])
def test_heat_incore_tiles_bitexact(P, shape):
    u0 = synthetic.uniform_field(shape, 5)
    ref = incore(P, _tiled(heat_desc(P, shape), 0), u0, 5)
    got = incore(P, _tiled(heat_desc(P, shape), 1), u0, 5)
    assert _same(got, ref)


def test_wave_incore_tiles_bitexact(P):
    shape = (48, 44, 72)
    m = synthetic.wave_model(shape)
    w = synthetic.ricker(7)
    cz, cy, cx = synthetic.centre(shape)
    z = np.zeros(shape, np.float32)
    ref = incore(P, _tiled(wave_desc(P, shape), 0), z, 7, up0=z, m=m, src=(cx, cy, cz), w=w)
    got = incore(P, _tiled(wave_desc(P, shape), 1), z, 7, up0=z, m=m, src=(cx, cy, cz), w=w)
    assert _same(got[0], ref[0]) and _same(got[1], ref[1])


@pytest.mark.parametrize("rate", [0, 16])
def test_heat_streamed_tiles_bitexact(P, rate):
    shape = (64, 36, 68)
    u0 = synthetic.uniform_field(shape, 6)
    ref = streamed(P, _tiled(heat_desc(P, shape, rate=rate, k=4, T=16), 0), u0, 9)
    got = streamed(P, _tiled(heat_desc(P, shape, rate=rate, k=4, T=16), 1), u0, 9)
    assert _same(got[0], ref[0])
    assert all(np.array_equal(a, b) for a, b in zip(got[2], ref[2]))


def test_wave_streamed_tiles_bitexact(P):
    shape = (96, 44, 64)
    m = synthetic.wave_model(shape)
    w = synthetic.ricker(10)
    cz, cy, cx = synthetic.centre(shape)
    z = np.zeros(shape, np.float32)
    ref = streamed(P, _tiled(wave_desc(P, shape, rate=16, k=2, T=32), 0), z, 10, up0=z, m=m,
                   src=(cx, cy, cz), w=w)
    got = streamed(P, _tiled(wave_desc(P, shape, rate=16, k=2, T=32), 1), z, 10, up0=z, m=m,
                   src=(cx, cy, cz), w=w)
    assert _same(got[0], ref[0]) and _same(got[1], ref[1])
    assert all(np.array_equal(a, b) for a, b in zip(got[2], ref[2]))


def test_adjoint_and_gradient_tiles_bitexact(P):
    torch = torch_cuda()
    shape = (40, 36, 44)
    rng = np.random.default_rng(2)
    m = synthetic.wave_model(shape)

    def interior():
        a = np.zeros(shape, np.float32)
        a[4:-4, 4:-4, 4:-4] = rng.standard_normal((shape[0] - 8, shape[1] - 8, shape[2] - 8))
        return a

    lam, lp, u = interior(), interior(), interior()
    g0 = rng.standard_normal(shape).astype(np.float32)
    res = rng.standard_normal(shape[1:]).astype(np.float32)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    s = torch.cuda.current_stream().cuda_stream
    outs = []
    for tile in (0, 1):
        nz, ny, nx = shape
        d = P.make_desc(nx, ny, nz, P.OOCS_WAVE, synthetic.wave_star_coef(), 1 << 40, temporal_depth=1,
                        slab_planes=nz, step_tile=tile)
        L, LP, M, MU, R = T(lam), T(lp), T(m), T(m * lam), T(res)
        MO = torch.empty_like(L)
        P.oocs_adjoint_step(d, L.data_ptr(), LP.data_ptr(), MU.data_ptr(), MO.data_ptr(), M.data_ptr(),
                            R.data_ptr(), 7, s)
        G, U = T(g0), T(u)
        P.oocs_gradient_accumulate(d, G.data_ptr(), L.data_ptr(), U.data_ptr(), 0.75, (20, 18, 16), s)
        torch.cuda.synchronize()
        outs.append((LP.cpu().numpy(), MO.cpu().numpy(), G.cpu().numpy()))
    for a, b in zip(outs[0], outs[1]):
        assert _same(a, b)


def test_invalid_tile_is_rejected(P):
    d = heat_desc(P, (32, 32, 32))
    d.step_tile = 2
    with pytest.raises(P.OOCSError):
        P.oocs_query(d)
