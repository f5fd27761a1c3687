"""A grid far larger than the device budget: 7-point heat on 2560 x 2560 x 5120
(one FP32 field of 134 GB), seeded U[0,1), 20 steps in 5 sweeps of k = 4 over
42 slabs, a 16 GiB device budget, rate 16, the host store in exact-size
pinned memory (67 GB) filled from planes drawn on the GPU.

Full-size parity on sampled outputs: after n steps a point depends only on the
initial values within distance n, so the FP64 oracle run on the (2n+1)^3 cube
around a sample (its faces held, which the centre cannot see within n steps)
gives that point's exact value; 8 seeded samples are compared with the
decompressed GPU values: each within the rate-16 max-abs bar, and all eight
within the rate-16 rel-L2 bar.
"""
import numpy as np
import pytest

import synthetic
from gpu_util import rel_l2, torch_cuda

SHAPE, STEPS, SEED, BUDGET = (5120, 2560, 2560), 20, 31, 16 << 30


def _cube(shape, seed, z, y, x, r):
    """The (2r+1)^3 cube of uniform_field(shape, seed) centred at (z, y, x), row by row."""
    nz, ny, nx = shape
    c = np.empty((2 * r + 1,) * 3, np.float32)
    for i, zz in enumerate(range(z - r, z + r + 1)):
        for j, yy in enumerate(range(y - r, y + r + 1)):
            c[i, j] = synthetic.uniform01(seed, 2 * r + 1, offset=(zz * ny + yy) * nx + x - r)
    return c


@pytest.mark.gpu
@pytest.mark.slow
def test_true_out_of_core_heat_sampled_against_oracle(orc):
    torch = torch_cuda()
    import paper_2204_11315_gb300 as P
    nz, ny, nx = SHAPE
    coef = synthetic.heat_star_coef(0.1)
    desc = P.make_desc(nx, ny, nz, P.OOCS_HEAT, coef, BUDGET, rate_bits=16, temporal_depth=4)
    plan = P.oocs_query(desc)
    assert plan.num_slabs > 8 and plan.workspace_bytes <= BUDGET
    host = P.HostBuffer(plan.host_store_bytes)
    st = P.OutOfCoreStencil(desc, stores=[host.tensor()])
    try:
        for z0 in range(0, nz, 64):
            f = synthetic.uniform_field_planes_torch(SHAPE, SEED, z0, z0 + 64, device="cuda")
            torch.cuda.synchronize()  # drawn on torch's stream; the context reads on its own
            P.oocs_compress_device(st.ctx, P.OOCS_FIELD_U, f.data_ptr(), z0, 64)
            st.synchronize(600.0)
            del f
        st.step(STEPS)
        st.synchronize(3600.0)
        assert st.stats()["passes_done"] == STEPS // 4
        rng = np.random.default_rng(3)
        samples = [(int(rng.integers(24, nz - 24)), int(rng.integers(24, ny - 24)), int(rng.integers(24, nx - 24)))
                   for _ in range(8)]
        buf = torch.empty((4, ny, nx), dtype=torch.float32, device="cuda")
        got, ref = [], []
        for (z, y, x) in samples:
            P.oocs_decompress_device(st.ctx, P.OOCS_FIELD_U, buf.data_ptr(), z // 4 * 4, 4)
            st.synchronize(600.0)
            got.append(float(buf[z % 4, y, x]))
            cube = _cube(SHAPE, SEED, z, y, x, STEPS)
            ref.append(orc.heat_run(cube, coef, STEPS)[STEPS, STEPS, STEPS])
    finally:
        st.close()
        host.close()
        torch.cuda.empty_cache()
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    assert rel_l2(got, ref) <= synthetic.TOL_COMPRESSED[16]
    # each sample on its own: |got - ref| within the rate-16 max-abs bar of the
    # largest sampled value (at most the field's peak, so no looser than the
    # bar against the peak)
    bound = synthetic.TOL_MAXABS_COMPRESSED[16] * float(np.max(np.abs(ref)))
    for i, (g, r) in enumerate(zip(got, ref)):
        assert abs(g - r) <= bound, (i, samples[i], g, r, bound)


def test_cube_reading_is_exact(orc):
    """The cone argument on a small grid: the cube oracle equals the whole-grid oracle."""
    shape = (60, 52, 56)
    u = synthetic.uniform_field(shape, 5)
    coef = synthetic.heat_star_coef(0.1)
    full = orc.heat_run(u, coef, 9)
    for (z, y, x) in ((20, 20, 20), (30, 25, 40), (11, 12, 13)):
        cube = _cube(shape, 5, z, y, x, 9)
        assert np.array_equal(cube, u[z - 9:z + 10, y - 9:y + 10, x - 9:x + 10])
        assert orc.heat_run(cube, coef, 9)[9, 9, 9] == full[z, y, x]
