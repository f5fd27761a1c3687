"""Pins of the FP64 adjoint oracle (gradient of the receiver misfit of the wave workload).

The adjoint step must be the exact transpose of the linearised leapfrog step
(dot-product test to FP64 rounding), and the gradient it accumulates must
match central finite differences of the misfit.  Putting m on the wrong side
of the stencil (m L lam instead of L(m lam)) or a sign error fails both.
"""
import numpy as np
import pytest

import synthetic


def _interior(shape, rng, r=4):
    a = np.zeros(shape)
    nz, ny, nx = shape
    a[r:nz - r, r:ny - r, r:nx - r] = rng.standard_normal((nz - 2 * r, ny - 2 * r, nx - 2 * r))
    return a


def _forward_linear(orc, u, up, m, coef):
    """F(u, up) = (2u - up + m L u, u) (no source)."""
    return orc.star_step(u, coef, "wave", m=m, up=up), u.copy()


def test_adjoint_step_is_the_transpose(orc):
    shape = (16, 14, 18)
    rng = np.random.default_rng(0)
    coef = synthetic.wave_star_coef()
    m = 0.05 + 0.1 * rng.random(shape)
    u, up = _interior(shape, rng), _interior(shape, rng)
    y1, y2 = _interior(shape, rng), _interior(shape, rng)
    f1, f2 = _forward_linear(orc, u, up, m, coef)
    lhs = np.vdot(f1, y1) + np.vdot(f2, y2)
    # F^T (y1, y2) = (G(y1, -y2)[0], -y1) with G(a, b) = 2a - b + L(m a)
    g = orc.wave_adjoint_step(y1, -y2, m, coef)
    rhs = np.vdot(u, g) + np.vdot(up, -y1)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)
    # the transpose of m L is L m, not m L: the other placement fails
    wrong = 2 * y1 + y2 + m * orc.star_apply(y1, coef)
    assert abs(lhs - (np.vdot(u, wrong) - np.vdot(up, y1))) > 1e-6 * abs(lhs)


def test_whole_run_dot_product(orc):
    """<F^N x, y> = <x, (F^T)^N y> for the linear part of N leapfrog steps."""
    shape = (14, 12, 16)
    rng = np.random.default_rng(1)
    coef = synthetic.wave_star_coef()
    m = 0.05 + 0.1 * rng.random(shape)
    u, up = _interior(shape, rng), _interior(shape, rng)
    y1, y2 = _interior(shape, rng), _interior(shape, rng)
    a, b = u, up
    for _ in range(9):
        a, b = _forward_linear(orc, a, b, m, coef)
    lhs = np.vdot(a, y1) + np.vdot(b, y2)
    # transpose steps in the (lam, -lam_prev) form
    p, q = y1, -y2
    for _ in range(9):
        p, q = orc.wave_adjoint_step(p, q, m, coef), p
    rhs = np.vdot(u, p) + np.vdot(up, -q)
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), 1.0)


def _problem(shape=(20, 18, 22), nsteps=24, seed=3):
    rng = np.random.default_rng(seed)
    coef = synthetic.wave_star_coef()
    z, y, x = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    m = 0.08 + 0.02 * np.sin(0.3 * x) * np.cos(0.25 * y) + 0.01 * rng.random(shape)
    src = (shape[0] // 2, shape[1] // 2, shape[2] // 2)
    w = synthetic.ricker(nsteps, dt=0.004, f0=25.0).astype(np.float64)
    zr = 5
    m_true = m * (1.0 + 0.05 * np.exp(-((x - 11) ** 2 + (y - 9) ** 2 + (z - 10) ** 2) / 8.0))
    return coef, m, m_true, src, w, zr, nsteps, rng


def test_gradient_matches_central_differences(orc):
    coef, m, m_true, src, w, zr, nsteps, rng = _problem()
    d = orc.wave_receiver_data(m_true, coef, nsteps, src, w, zr)
    J, g = orc.wave_misfit_gradient(m, coef, nsteps, src, w, zr, d)
    assert J > 0
    shape = m.shape
    pts = [(rng.integers(4, shape[0] - 4), rng.integers(4, shape[1] - 4), rng.integers(4, shape[2] - 4))
           for _ in range(6)]
    pts.append(src)
    for p in pts:
        h = 1e-5 * m[p]
        mp, mm = m.copy(), m.copy()
        mp[p] += h
        mm[p] -= h
        Jp, _ = orc.wave_misfit_gradient(mp, coef, nsteps, src, w, zr, d)
        Jm, _ = orc.wave_misfit_gradient(mm, coef, nsteps, src, w, zr, d)
        fd = (Jp - Jm) / (2 * h)
        assert abs(fd - g[p]) <= 1e-5 * max(abs(fd), 1e-3 * np.max(np.abs(g))), (p, fd, g[p])
    # the shell carries no gradient
    assert np.all(g[:4] == 0) and np.all(g[:, :, -4:] == 0)


def test_gradient_directional_derivative(orc):
    coef, m, m_true, src, w, zr, nsteps, rng = _problem(seed=4)
    d = orc.wave_receiver_data(m_true, coef, nsteps, src, w, zr)
    J, g = orc.wave_misfit_gradient(m, coef, nsteps, src, w, zr, d)
    dm = _interior(m.shape, rng) * 1e-3
    eps = 1e-2
    Jp, _ = orc.wave_misfit_gradient(m + eps * dm, coef, nsteps, src, w, zr, d)
    Jm, _ = orc.wave_misfit_gradient(m - eps * dm, coef, nsteps, src, w, zr, d)
    fd = (Jp - Jm) / (2 * eps)
    assert abs(fd - np.vdot(g, dm)) <= 1e-6 * abs(fd)
    # zero misfit at the true model: zero gradient
    J0, g0 = orc.wave_misfit_gradient(m_true, coef, nsteps, src, w, zr, d)
    assert J0 < 1e-24 and np.max(np.abs(g0)) < 1e-12
