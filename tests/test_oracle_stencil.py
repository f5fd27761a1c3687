"""Pins of the FP64 stencil oracle against closed forms, brute force and invariants.

Each test checks the oracle against something other than itself: the exact
eigenvalue of the discrete Dirichlet Laplacian, a dense operator built by
enumerating stencil offsets, exactness of the 8th-order weights on
polynomials, the leapfrog stability limit, and time reversibility.
"""
import math

import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _dense_star(n, r, coef):
    """Dense operator of the star stencil on an n^3 grid, built by enumerating
    the 6r neighbour offsets of each interior point.  Shell rows are zero."""
    N = n ** 3
    A = np.zeros((N, N))
    interior = np.zeros(N, bool)
    for z in range(n):
        for y in range(n):
            for x in range(n):
                p = (z * n + y) * n + x
                if min(x, y, z) < r or max(x, y, z) >= n - r:
                    continue
                interior[p] = True
                A[p, p] += coef[0]
                for d in range(1, r + 1):
                    for (dx, dy, dz) in ((d, 0, 0), (-d, 0, 0), (0, d, 0), (0, -d, 0), (0, 0, d), (0, 0, -d)):
                        q = ((z + dz) * n + (y + dy)) * n + (x + dx)
                        A[p, q] += coef[d]
    return A, interior


# ---------------------------------------------------------------- heat -----

def test_heat_eigenmode_closed_form(orc):
    """sin(pi i/127) sin(pi j/127) sin(pi k/127) decays by 1 - 12 alpha sin^2(pi/254) per step."""
    n, alpha, steps = 128, 0.1, 10
    lam = 1.0 - 12.0 * alpha * math.sin(math.pi / 254.0) ** 2
    # the values stated for this workload's mode, to 14 digits
    assert abs(lam - 0.99981643435185) < 5e-15
    assert abs(lam ** 10 - 0.99816585911210) < 5e-15
    u0 = synthetic.sine_mode(n)
    u1 = orc.heat_run(u0, synthetic.heat_star_coef(alpha), 1)
    assert np.max(np.abs(u1 - lam * u0)) <= 1e-13 * np.max(np.abs(u0))
    u10 = orc.heat_run(u0, synthetic.heat_star_coef(alpha), steps)
    assert np.max(np.abs(u10 - lam ** steps * u0)) <= 1e-13 * np.max(np.abs(u0))


def test_heat_constant_field_domain_of_dependence(orc):
    """Interior constant c with a zero shell: points farther than n*r from the
    shell are still c after n steps, and the point next to the shell is not."""
    n, steps, c = 24, 5, 0.625
    u0 = np.full((n, n, n), c)
    u0[0] = u0[-1] = 0
    u0[:, 0] = u0[:, -1] = 0
    u0[:, :, 0] = u0[:, :, -1] = 0
    u = orc.heat_run(u0, synthetic.heat_star_coef(0.1), steps)
    inner = u[1 + steps:n - 1 - steps, 1 + steps:n - 1 - steps, 1 + steps:n - 1 - steps]
    assert np.max(np.abs(inner - c)) <= 1e-14
    assert abs(u[1, n // 2, n // 2] - c) > 1e-3
    assert np.all(u[0] == 0) and np.all(u[:, :, -1] == 0)


def test_heat_bruteforce_8cubed(orc):
    n, steps = 8, 6
    coef = synthetic.heat_star_coef(0.13)
    A, interior = _dense_star(n, 1, coef)
    M = A + np.diag(~interior * 1.0)      # shell rows keep their value
    rng = np.random.default_rng(5)
    u0 = rng.standard_normal((n, n, n))
    ref = np.linalg.matrix_power(M, steps) @ u0.reshape(-1)
    got = orc.heat_run(u0, coef, steps).reshape(-1)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_heat_linearity_and_max_principle(orc):
    n = 16
    coef = synthetic.heat_star_coef(0.1)
    rng = np.random.default_rng(1)
    a, b = rng.random((n, n, n)), rng.random((n, n, n))
    ua = orc.heat_run(a, coef, 3)
    ub = orc.heat_run(b, coef, 3)
    uab = orc.heat_run(a + 2.0 * b, coef, 3)
    assert np.max(np.abs(uab - (ua + 2.0 * ub))) <= 1e-13
    # alpha <= 1/6: all weights non-negative and sum to 1
    assert ua.min() >= a.min() - 1e-15 and ua.max() <= a.max() + 1e-15


# ---------------------------------------------------------------- wave -----

def test_wave_weights_exact_on_polynomials():
    """The 8th-order weights give the exact second derivative of x^p, p <= 9."""
    c = np.array(synthetic.WAVE_COEF_1D)
    for p in range(10):
        val = (c[0] if p == 0 else 0.0) + sum(c[d] * (d ** p + (-d) ** p) for d in range(1, 5))
        exact = 2.0 if p == 2 else 0.0
        assert abs(val - exact) < 1e-9, (p, val)
    # and not for x^10 (order exactly 8)
    val = sum(c[d] * 2 * d ** 10 for d in range(1, 5))
    assert abs(val) > 1.0
    assert synthetic.wave_star_coef()[0] == 3.0 * c[0]


def test_wave_constant_state_invariant(orc):
    n = 16
    u = np.full((n, n, n), 1.75)
    m = np.full((n, n, n), 0.12)
    u1, u0 = orc.wave_run(u, u, m, synthetic.wave_star_coef(), 7)
    assert np.max(np.abs(u1 - 1.75)) <= 1e-12
    assert np.max(np.abs(u0 - 1.75)) <= 1e-12


def test_wave_bruteforce_12cubed_with_source(orc):
    n, steps = 12, 5
    coef = synthetic.wave_star_coef()
    A, interior = _dense_star(n, 4, coef)
    rng = np.random.default_rng(2)
    m = 0.05 + 0.1 * rng.random(n ** 3)
    u = rng.standard_normal(n ** 3)
    up = rng.standard_normal(n ** 3)
    src = (6, 6, 6)
    s = (6 * n + 6) * n + 6
    w = rng.standard_normal(steps)
    a, b = u.copy(), up.copy()
    for k in range(steps):
        Lu = A @ a
        Lu[s] += w[k]
        nxt = np.where(interior, 2.0 * a - b + m * Lu, a)
        a, b = nxt, a
    g1, g0 = orc.wave_run(u.reshape(n, n, n), up.reshape(n, n, n), m.reshape(n, n, n), coef, steps,
                          src=src, w=w)
    scale = np.max(np.abs(a))
    assert np.max(np.abs(g1.reshape(-1) - a)) <= 1e-12 * scale
    assert np.max(np.abs(g0.reshape(-1) - b)) <= 1e-12 * scale


def test_wave_time_reversible(orc):
    """Leapfrog is time symmetric: swapping (u^n, u^(n-1)) and stepping back returns the start."""
    n, steps = 20, 12
    rng = np.random.default_rng(3)
    m = 0.1 * (0.5 + rng.random((n, n, n)))
    u0 = np.zeros((n, n, n))
    u0[4:-4, 4:-4, 4:-4] = rng.standard_normal((n - 8, n - 8, n - 8))
    up0 = u0.copy()
    u1, up1 = orc.wave_run(u0, up0, m, synthetic.wave_star_coef(), steps)
    b0, b1 = orc.wave_run(up1, u1, m, synthetic.wave_star_coef(), steps)
    assert np.max(np.abs(b0 - up0)) <= 1e-9 * np.max(np.abs(u0))
    assert np.max(np.abs(b1 - u0)) <= 1e-9 * np.max(np.abs(u0))


def test_wave_cfl_limit(orc):
    """Leapfrog with the 3D 25-point star is stable for Courant <= 2/sqrt(3*6.50159)."""
    c = np.array(synthetic.WAVE_COEF_1D)
    symbol_max = -(c[0] + 2 * sum(c[d] * (-1) ** d for d in range(1, 5)))
    assert abs(symbol_max - 6.50159) < 1e-5
    limit = 2.0 / math.sqrt(3.0 * symbol_max)
    assert abs(limit - 0.45286) < 1e-5
    n = 24
    rng = np.random.default_rng(4)
    u0 = np.zeros((n, n, n))
    u0[4:-4, 4:-4, 4:-4] = rng.standard_normal((n - 8, n - 8, n - 8))
    grow = {}
    for courant in (0.95 * limit, 1.04 * limit):
        m = np.full((n, n, n), courant ** 2)
        u, _ = orc.wave_run(u0, u0, m, synthetic.wave_star_coef(), 300)
        grow[courant] = np.max(np.abs(u)) / np.max(np.abs(u0))
    lo, hi = sorted(grow)
    assert grow[lo] < 20.0
    assert grow[hi] > 1e6


def test_wave_workload_courant_below_limit():
    v = synthetic.layered_velocity((64, 8, 8))
    courant = v.max() * synthetic.WAVE_DT / synthetic.WAVE_DX
    assert courant <= 4725.0 * synthetic.WAVE_DT / synthetic.WAVE_DX + 1e-12
    assert courant < 0.45286
    assert v.min() >= 1500.0 * 0.95 - 1e-9 and v.max() <= 4500.0 * 1.05 + 1e-9
