"""Degenerate and extreme cases of the slab sweep, on the GPU.

Zero steps change nothing; the smallest grids (one codec block layer per
slab side, Dirichlet shell everywhere but a few planes), a single slab
(T = nz), and slab windows clipped at both faces of the grid stay bit-exact
against the in-core run; the transform codec at its extreme rates (1 and 32
bits/value) runs, and at 32 bits it is within the uncompressed bar of the
FP64 oracle.
"""
import numpy as np
import pytest

import synthetic
from gpu_util import assert_uncompressed, heat_desc, incore, streamed, torch_cuda, wave_desc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2204_11315_gb300 as P
    P.lib()
    return P


def test_zero_steps_change_nothing(P):
    torch_cuda()
    u0 = synthetic.heat_initial(32)
    desc = heat_desc(P, u0.shape, rate=16, k=2, T=16)
    st = P.OutOfCoreStencil(desc)
    try:
        st.compress(P.OOCS_FIELD_U, u0)
        st.synchronize(60.0)
        before = st.stores[0].numpy().copy()
        st.step(0)
        st.synchronize(60.0)
        stats = st.stats()
        assert np.array_equal(st.stores[0].numpy(), before)
        assert stats["steps_done"] == 0 and stats["slabs_done"] == 0 and stats["h2d_bytes"] == 0
        with pytest.raises(P.OOCSError):
            st.step(-1)
    finally:
        st.close()


@pytest.mark.parametrize("shape,T,k", [((8, 8, 8), 8, 1),       # one slab, 2 interior planes per axis
                                       ((16, 8, 12), 8, 1),     # two slabs of the smallest T = 2 h
                                       ((24, 12, 8), 8, 1),     # three slabs
                                       ((12, 8, 8), 12, 3)])    # one slab, k = 3
def test_smallest_heat_grids_bitexact(P, shape, T, k):
    torch_cuda()
    u0 = synthetic.uniform_field(shape, 21)
    desc = heat_desc(P, shape, rate=0, k=k, T=T)
    got, _, _, _, _ = streamed(P, desc, u0, 6)
    assert np.array_equal(got, incore(P, desc, u0, 6))


@pytest.mark.parametrize("shape,T,k", [((32, 24, 24), 32, 4),   # one slab: the window is the grid
                                       ((24, 32, 32), 16, 2),   # h = 8: both windows clipped by the grid
                                       ((48, 16, 64), 16, 2)])  # middle window unclipped, outer ones clipped
def test_single_slab_and_clipped_windows_bitexact(P, shape, T, k):
    torch_cuda()
    steps = 9
    m = synthetic.wave_model(shape)
    w = synthetic.ricker(steps)
    cz, cy, cx = synthetic.centre(shape)
    z = np.zeros(shape, np.float32)
    for ro in (0, 1):
        desc = wave_desc(P, shape, rate=0, k=k, T=T, ro=ro)
        gu, gup, _, _, plan = streamed(P, desc, z, steps, up0=z, m=m, src=(cx, cy, cz), w=w)
        ru, rup = incore(P, desc, z, steps, up0=z, m=m, src=(cx, cy, cz), w=w)
        assert np.array_equal(gu, ru) and np.array_equal(gup, rup), (ro, plan.num_slabs)
        assert float(np.abs(gu).max()) > 0.0


def test_extreme_rates(P, orc):
    torch_cuda()
    u0 = synthetic.heat_initial(64)
    ref = orc.heat_run(u0, synthetic.heat_star_coef(0.1), 6)
    got32, _, _, _, p32 = streamed(P, heat_desc(P, u0.shape, rate=32, k=2, T=16), u0, 6)
    assert_uncompressed(got32, ref, "heat", "rate 32")
    assert p32.host_store_bytes == u0.size * 4
    got1, _, _, _, p1 = streamed(P, heat_desc(P, u0.shape, rate=1, k=2, T=16), u0, 6)
    assert np.all(np.isfinite(got1)) and p1.host_store_bytes == u0.size // 8
