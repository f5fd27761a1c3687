"""In-core GPU stencil kernels against the FP64 oracle (Sec. 3.1 stencil, Sec. 6 wave code).

FP32 GPU arithmetic against FP64: relative L2 within 1e-6 (heat) and 1e-5
(wave), the uncompressed bars, and every point within ten times that of the
field's peak.  Grids with x-y sizes that are not multiples of
the 64 x 16 CTA tile exercise the ragged tail.
"""
import math

import numpy as np
import pytest

import synthetic
from gpu_util import assert_parity, assert_uncompressed, heat_desc, incore, wave_desc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2204_11315_gb300 as P
    P.lib()
    return P


def test_heat_eigenmode_decay(P):
    n, alpha = 128, 0.1
    lam = 1.0 - 12.0 * alpha * math.sin(math.pi / 254.0) ** 2
    mode = synthetic.sine_mode(n)
    u = incore(P, heat_desc(P, (n, n, n)), mode.astype(np.float32), 10)
    assert_parity(u, lam ** 10 * mode, 1e-6, 1e-5, "eigenmode")


def test_heat_workload_vs_oracle(P, orc):
    u0 = synthetic.heat_initial(128)
    ref = orc.heat_run(u0, synthetic.heat_star_coef(0.1), 10)
    got = incore(P, heat_desc(P, u0.shape), u0, 10)
    assert_uncompressed(got, ref, "heat", "heat 128^3")
    assert np.all(got[0] == 0) and np.all(got[:, :, -1] == 0)


@pytest.mark.parametrize("shape", [(36, 44, 52), (20, 100, 68)])
def test_heat_ragged_vs_oracle(P, orc, shape):
    u0 = synthetic.uniform_field(shape, 7)
    ref = orc.heat_run(u0, synthetic.heat_star_coef(0.15), 6)
    got = incore(P, heat_desc(P, shape, alpha=0.15), u0, 6)
    assert_uncompressed(got, ref, "heat", f"heat {shape}")


@pytest.mark.parametrize("shape,steps", [((64, 64, 64), 40), ((72, 40, 104), 30)])
def test_wave_vs_oracle(P, orc, shape, steps):
    m = synthetic.wave_model(shape)
    w = synthetic.ricker(steps)
    src = synthetic.centre(shape)
    z = np.zeros(shape, np.float32)
    ru, rup = orc.wave_run(z, z, m, synthetic.wave_star_coef(), steps, src=src, w=w)
    gu, gup = incore(P, wave_desc(P, shape), z, steps, up0=z, m=m, src=(src[2], src[1], src[0]), w=w)
    assert_uncompressed(gu, ru, "wave", "u")
    assert_uncompressed(gup, rup, "wave", "u_prev")


def test_wave_random_state_vs_oracle(P, orc):
    """Non-zero (u, u_prev) everywhere in the interior, no source."""
    shape = (48, 56, 40)
    rng = np.random.default_rng(1)
    u = np.zeros(shape, np.float32)
    up = np.zeros(shape, np.float32)
    u[4:-4, 4:-4, 4:-4] = rng.standard_normal((40, 48, 32))
    up[4:-4, 4:-4, 4:-4] = rng.standard_normal((40, 48, 32))
    m = synthetic.wave_model(shape)
    ru, rup = orc.wave_run(u, up, m, synthetic.wave_star_coef(), 7)
    gu, gup = incore(P, wave_desc(P, shape), u, 7, up0=up, m=m)
    assert_uncompressed(gu, ru, "wave", "u")
    assert_uncompressed(gup, rup, "wave", "u_prev")
