"""GPU adjoint of the leapfrog wave scheme and the autograd gradient of the receiver misfit.

Checked against the FP64 oracle (tests/test_oracle_adjoint.py pins it): the
adjoint step and gradient kernels elementwise, the dot-product test
<F x, y> = <x, F^T y> in FP32 for one and for ten steps, the autograd gradient
against the oracle's gradient and against oracle central differences of the
misfit in the velocity (h = 1e-3 relative) at 16 random voxels, and the
workload size (256^3, 400 steps, checkpoints every 10 steps at 16 bits/value).
"""
import numpy as np
import pytest

import synthetic
from gpu_util import assert_parity, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2204_11315_gb300 as P
    P.lib()
    return P


def _desc(P, shape):
    nz, ny, nx = shape
    return P.make_desc(nx, ny, nz, P.OOCS_WAVE, synthetic.wave_star_coef(), 1 << 40, temporal_depth=1,
                       slab_planes=nz)


def _interior(shape, rng, r=4):
    a = np.zeros(shape, np.float32)
    nz, ny, nx = shape
    a[r:nz - r, r:ny - r, r:nx - r] = rng.standard_normal((nz - 2 * r, ny - 2 * r, nx - 2 * r))
    return a


def _gpu_adjoint(P, torch, desc, lam, lam_prev, m, res=None, zr=-1):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    L, LP, M = t(lam), t(lam_prev), t(m)
    MU = t(m * lam)
    MO = torch.empty_like(L)
    R = t(res) if res is not None else None
    P.oocs_adjoint_step(desc, L.data_ptr(), LP.data_ptr(), MU.data_ptr(), MO.data_ptr(), M.data_ptr(),
                        R.data_ptr() if R is not None else 0, zr, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return LP.cpu().numpy(), MO.cpu().numpy()


def test_adjoint_step_vs_oracle(P, orc):
    torch = torch_cuda()
    shape = (40, 36, 44)
    rng = np.random.default_rng(0)
    m = synthetic.wave_model(shape)
    lam, lp = _interior(shape, rng), _interior(shape, rng)
    res = rng.standard_normal((36, 44)).astype(np.float32)
    got, mu = _gpu_adjoint(P, torch, _desc(P, shape), lam, lp, m, res, 7)
    ref = orc.wave_adjoint_step(lam, lp, m, synthetic.wave_star_coef(), res, 7)
    assert_parity(got, ref, synthetic.TOL_KERNEL, synthetic.TOL_MAXABS_KERNEL, "lam^n")
    assert_parity(mu, m.astype(np.float64) * ref, synthetic.TOL_KERNEL, synthetic.TOL_MAXABS_KERNEL, "m lam^n")
    assert np.all(got[:4] == 0) and np.all(mu[:, :, -4:] == 0)


def test_gradient_accumulate_vs_oracle(P, orc):
    torch = torch_cuda()
    shape = (32, 28, 36)
    rng = np.random.default_rng(1)
    u, lam = _interior(shape, rng), _interior(shape, rng)
    g0 = rng.standard_normal(shape).astype(np.float32)
    src = (18, 14, 16)  # x, y, z
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    G, L, U = T(g0), T(lam), T(u)
    P.oocs_gradient_accumulate(_desc(P, shape), G.data_ptr(), L.data_ptr(), U.data_ptr(), 0.75, src,
                               torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    t = orc.star_apply(u, synthetic.wave_star_coef())
    t[src[2], src[1], src[0]] += 0.75
    ref = g0.astype(np.float64) + lam.astype(np.float64) * t
    ref[:4] = g0[:4]
    assert_parity(G.cpu().numpy(), ref, synthetic.TOL_KERNEL, synthetic.TOL_MAXABS_KERNEL, "dJ/dm")


@pytest.mark.parametrize("nsteps", [1, 10])
def test_dot_product_fp32(P, orc, nsteps):
    """<F^N x, y> = <x, (F^T)^N y> with the GPU forward step and the GPU adjoint step."""
    torch = torch_cuda()
    shape = (40, 40, 40)
    rng = np.random.default_rng(2)
    desc = _desc(P, shape)
    m = synthetic.wave_model(shape)
    u0, up0 = _interior(shape, rng), _interior(shape, rng)
    y1, y2 = _interior(shape, rng), _interior(shape, rng)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    s = torch.cuda.current_stream().cuda_stream
    U, UP, M, SC = T(u0), T(up0), T(m), torch.empty(shape, device="cuda")
    P.oocs_incore_run(desc, U.data_ptr(), UP.data_ptr(), M.data_ptr(), SC.data_ptr(), nsteps, 0, None,
                      None, s)
    # transpose steps in the (lam, -lam_prev) form: lam_new = 2 lam - lam_prev + L(m lam)
    LAM, LP = T(y1), T(-y2)
    MU, MO = T(m * y1), torch.empty(shape, device="cuda")
    for _ in range(nsteps):
        P.oocs_adjoint_step(desc, LAM.data_ptr(), LP.data_ptr(), MU.data_ptr(), MO.data_ptr(),
                            M.data_ptr(), 0, -1, s)
        LAM, LP = LP, LAM
        MU, MO = MO, MU
    torch.cuda.synchronize()
    f1, f2 = U.cpu().numpy().astype(np.float64), UP.cpu().numpy().astype(np.float64)
    a1, a2 = LAM.cpu().numpy().astype(np.float64), LP.cpu().numpy().astype(np.float64)
    lhs = np.vdot(f1, y1) + np.vdot(f2, y2)
    rhs = np.vdot(u0, a1) + np.vdot(up0, -a2)
    assert abs(lhs - rhs) <= 1e-5 * (np.linalg.norm(f1) * np.linalg.norm(y1) + np.linalg.norm(f2) * np.linalg.norm(y2))


def _small_problem(P, rate, shape=(40, 36, 44), nsteps=80):
    """Layered model at dx = 10 m, dt = 0.8 ms (stable), 40 Hz Ricker 8 planes
    below the receiver plane z = 6, so the recorded wave is well inside the run."""
    import paper_2204_11315_gb300.adjoint as A
    dt, dx = synthetic.WAVE_DT, synthetic.WAVE_DX
    w = synthetic.ricker(nsteps, dt=dt, f0=40.0)
    v = synthetic.layered_velocity(shape).astype(np.float32)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    bump = np.exp(-((x - 24) ** 2 + (y - 18) ** 2 + (z - 10) ** 2) / 20.0)
    v_true = (v * (1.0 + 0.05 * bump)).astype(np.float32)
    prob = A.WaveProblem(shape=shape, dt=dt, dx=dx, coef=synthetic.wave_star_coef(),
                         src_xyz=(nx // 2, ny // 2, 14), wavelet=w, zr=6, nsteps=nsteps,
                         checkpoint_every=10, rate=rate)
    return A, prob, v, v_true, w


@pytest.mark.parametrize("rate,tol", [(0, 1e-4), (16, 1e-3)])
def test_autograd_gradient_vs_oracle(P, orc, rate, tol):
    torch = torch_cuda()
    A, prob, v, v_true, w = _small_problem(P, rate)
    s = prob.dt / prob.dx
    m64 = (v.astype(np.float64) * s) ** 2
    mt64 = (v_true.astype(np.float64) * s) ** 2
    src_zyx = prob.src_xyz[::-1]
    d = orc.wave_receiver_data(mt64, prob.coef, prob.nsteps, src_zyx, w, prob.zr)
    J_ref, gm_ref = orc.wave_misfit_gradient(m64, prob.coef, prob.nsteps, src_zyx, w, prob.zr, d)
    gv_ref = gm_ref * 2.0 * v.astype(np.float64) * s * s
    vt = torch.from_numpy(v).cuda().requires_grad_(True)
    J = A.wave_misfit(vt, torch.from_numpy(d.astype(np.float32)).cuda(), prob)
    J.backward()
    assert J_ref > 0 and np.abs(gv_ref).max() > 0
    assert abs(float(J.detach()) - J_ref) <= 1e-4 * J_ref
    assert rel_l2(vt.grad.cpu().numpy(), gv_ref) <= tol


def test_autograd_gradient_vs_oracle_finite_differences(P, orc):
    """Central differences of the FP64 oracle misfit in v (h = 1e-3 relative) at 16 voxels."""
    torch = torch_cuda()
    A, prob, v, v_true, w = _small_problem(P, 16, shape=(32, 32, 36), nsteps=70)
    s = prob.dt / prob.dx
    src_zyx = prob.src_xyz[::-1]
    mt64 = (v_true.astype(np.float64) * s) ** 2
    d = orc.wave_receiver_data(mt64, prob.coef, prob.nsteps, src_zyx, w, prob.zr)
    vt = torch.from_numpy(v).cuda().requires_grad_(True)
    A.wave_misfit(vt, torch.from_numpy(d.astype(np.float32)).cuda(), prob).backward()
    g = vt.grad.cpu().numpy().astype(np.float64)
    assert np.abs(g).max() > 0
    rng = np.random.default_rng(5)
    nz, ny, nx = v.shape
    # voxels where the gradient is not negligible (inside the illuminated region)
    cand = np.argwhere(np.abs(g) > 0.05 * np.abs(g).max())
    pick = cand[rng.choice(len(cand), 16, replace=False)]
    for (z, y, x) in pick:
        h = 1e-3 * float(v[z, y, x])
        vals = []
        for sgn in (1, -1):
            vv = v.astype(np.float64).copy()
            vv[z, y, x] += sgn * h
            J, _ = orc.wave_misfit_gradient((vv * s) ** 2, prob.coef, prob.nsteps, src_zyx, w, prob.zr, d)
            vals.append(J)
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g[z, y, x]) <= 2e-2 * abs(fd) + 1e-3 * np.abs(g).max(), (z, y, x, fd, g[z, y, x])


def test_workload_gradient_256cubed(P):
    """256^3, 400 steps, checkpoints every 10 steps at rate 16 (the adjoint workload).

    The 15 Hz source sits at depth z = 32 under the receiver plane z = 8 (a
    source at the centre, z = 128, would not reach the receivers within 400
    steps at these velocities, leaving a zero misfit)."""
    torch = torch_cuda()
    import paper_2204_11315_gb300.adjoint as A
    shape = (256, 256, 256)
    nsteps = 400
    w = synthetic.ricker(nsteps)
    v = synthetic.layered_velocity(shape, seed=4).astype(np.float32)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    v_true = (v * (1.0 + 0.05 * np.exp(-((x - 140) ** 2 + (y - 120) ** 2 + (z - 40) ** 2) / 400.0))).astype(np.float32)
    del x, y, z
    kw = dict(shape=shape, dt=synthetic.WAVE_DT, dx=synthetic.WAVE_DX, coef=synthetic.wave_star_coef(),
              src_xyz=(128, 128, 32), wavelet=w, zr=8, nsteps=nsteps, checkpoint_every=10)
    prob16 = A.WaveProblem(rate=16, **kw)
    d = A.receiver_data(torch.from_numpy(v_true).cuda(), prob16)
    grads = {}
    for rate in (16, 0):
        prob = A.WaveProblem(rate=rate, **kw)
        vt = torch.from_numpy(v).cuda().requires_grad_(True)
        J = A.wave_misfit(vt, d, prob)
        J.backward()
        assert float(J.detach()) > 0
        grads[rate] = vt.grad.cpu().numpy()
        assert np.all(np.isfinite(grads[rate]))
    assert np.abs(grads[0]).max() > 0
    # compressing the checkpoints at rate 16 changes the gradient very little
    assert rel_l2(grads[16], grads[0]) <= 1e-3


def _granular_gradient(P, torch, prob, v, d):
    """The backward pass written out with the per-step entry points (no driver):
    raw states of every step, adjoint step, gradient accumulation."""
    nz, ny, nx = prob.shape
    n = nz * ny * nx
    desc = prob.desc()
    s = torch.cuda.current_stream().cuda_stream
    m = torch.empty_like(v)
    P.oocs_model_from_velocity(v.data_ptr(), m.data_ptr(), n, prob.dt / prob.dx, s)
    w = np.asarray(prob.wavelet, np.float32)
    N = prob.nsteps
    states = torch.zeros((N + 1,) + tuple(prob.shape), device="cuda")  # states[k] = u^k
    up = torch.zeros_like(v)
    sc = torch.empty_like(v)
    for k in range(N):
        u = states[k].clone()
        P.oocs_incore_run(desc, u.data_ptr(), up.data_ptr(), m.data_ptr(), sc.data_ptr(), 1, k,
                          prob.src_xyz, w, s)
        states[k + 1].copy_(u)
        up.copy_(states[k])
    res = torch.empty((N, ny, nx), device="cuda")
    mis = torch.zeros(1, dtype=torch.float64, device="cuda")
    plane = ny * nx
    for k in range(N):
        P.oocs_receiver_residual(states[k + 1].data_ptr() + 4 * prob.zr * plane, d[k].data_ptr(), plane,
                                 res[k].data_ptr(), mis.data_ptr(), s)
    lam, lp, mu, mo, g = (torch.zeros_like(v) for _ in range(5))
    for k in range(N, 0, -1):
        P.oocs_adjoint_step(desc, lam.data_ptr(), lp.data_ptr(), mu.data_ptr(), mo.data_ptr(), m.data_ptr(),
                            res[k - 1].data_ptr(), prob.zr, s)
        lam, lp = lp, lam
        mu, mo = mo, mu
        P.oocs_gradient_accumulate(desc, g.data_ptr(), lam.data_ptr(), states[k - 1].data_ptr(),
                                   float(w[k - 1]), prob.src_xyz, s)
    torch.cuda.synchronize()
    return float(mis.item()), g


@pytest.mark.parametrize("K", [10, 7, 1])
def test_driver_matches_per_step_entry_points(P, K):
    """oocs_misfit_forward / _backward with raw checkpoints give bit for bit the
    misfit and dJ/dm of the per-step loop, for segment lengths that divide the
    run, leave a short last segment, and hold a single state."""
    torch = torch_cuda()
    A, prob, v, v_true, w = _small_problem(P, 0, shape=(32, 28, 36), nsteps=40)
    prob.checkpoint_every = K
    vv = torch.from_numpy(v).cuda()
    d = A.receiver_data(torch.from_numpy(v_true).cuda(), prob)
    J_ref, g_ref = _granular_gradient(P, torch, prob, vv, d)
    nbytes = prob.workspace_bytes()
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    m = torch.empty_like(vv)
    s = torch.cuda.current_stream().cuda_stream
    P.oocs_model_from_velocity(vv.data_ptr(), m.data_ptr(), vv.numel(), prob.dt / prob.dx, s)
    res = torch.empty((prob.nsteps,) + tuple(prob.shape[1:]), device="cuda")
    mis = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty_like(vv)
    P.oocs_misfit_forward(prob.desc(), m.data_ptr(), prob.src_xyz, prob.wavelet32(), prob.zr, d.data_ptr(),
                          prob.nsteps, K, 0, ws.data_ptr(), nbytes, res.data_ptr(), mis.data_ptr(), s)
    P.oocs_misfit_backward(prob.desc(), m.data_ptr(), prob.src_xyz, prob.wavelet32(), prob.zr, res.data_ptr(),
                           prob.nsteps, K, 0, ws.data_ptr(), nbytes, g.data_ptr(), s)
    torch.cuda.synchronize()
    assert J_ref > 0
    assert abs(float(mis.item()) - J_ref) <= 1e-12 * J_ref  # double accumulation order may differ
    assert torch.equal(g, g_ref)


@pytest.mark.slow
def test_dot_product_at_workload_size(P):
    """<F^N x, y> = <x, (F^T)^N y> on the adjoint workload's grid and length
    (256^3, N = 400 GPU steps, FP32; x, y seeded interior fields)."""
    torch = torch_cuda()
    shape = (256, 256, 256)
    N = 400
    rng = np.random.default_rng(11)
    desc = _desc(P, shape)
    m = synthetic.wave_model(shape)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    s = torch.cuda.current_stream().cuda_stream
    u0, up0, y1, y2 = (_interior(shape, rng) for _ in range(4))
    U, UP, M, SC = T(u0), T(up0), T(m), torch.empty(shape, device="cuda")
    P.oocs_incore_run(desc, U.data_ptr(), UP.data_ptr(), M.data_ptr(), SC.data_ptr(), N, 0, None, None, s)
    LAM, LP = T(y1), T(-y2)
    MU, MO = T(m * y1), torch.empty(shape, device="cuda")
    for _ in range(N):
        P.oocs_adjoint_step(desc, LAM.data_ptr(), LP.data_ptr(), MU.data_ptr(), MO.data_ptr(), M.data_ptr(),
                            0, -1, s)
        LAM, LP = LP, LAM
        MU, MO = MO, MU
    torch.cuda.synchronize()
    d = lambda a, b: float(torch.dot(a.double().ravel(), b.double().ravel()))
    lhs = d(U, T(y1)) + d(UP, T(y2))
    rhs = d(T(u0), LAM) - d(T(up0), LP)
    scale = (float(U.double().norm()) * np.linalg.norm(y1) + float(UP.double().norm()) * np.linalg.norm(y2))
    assert abs(lhs - rhs) <= 1e-4 * scale, (lhs, rhs, scale)


def _ooc_problem(P, rate, K, nsteps=60, budget=None, slab=32):
    import paper_2204_11315_gb300.adjoint as A
    shape = (96, 40, 48)
    dt, dx = synthetic.WAVE_DT, synthetic.WAVE_DX
    w = synthetic.ricker(nsteps, dt=dt, f0=40.0)
    v = synthetic.layered_velocity(shape).astype(np.float32)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    v_true = (v * (1.0 + 0.05 * np.exp(-((x - 24) ** 2 + (y - 20) ** 2 + (z - 28) ** 2) / 30.0))).astype(np.float32)
    # source 8 planes below the receiver plane; the slabs are [0, 32), [32, 64), [64, 96)
    prob = A.WaveProblem(shape=shape, dt=dt, dx=dx, coef=synthetic.wave_star_coef(), src_xyz=(24, 20, 32),
                         wavelet=w, zr=24, nsteps=nsteps, checkpoint_every=K, rate=rate, device_budget=budget,
                         slab_planes=slab if budget else 0)
    return A, prob, v, v_true


@pytest.mark.parametrize("K,nsteps", [(10, 60), (7, 55), (10, 51)])
def test_out_of_core_gradient_equals_in_core_uncompressed(P, K, nsteps):
    """Uncompressed, the slab-swept forward, the recomputation of each segment
    (sweeps of depth 1 and 2, states kept by the state record) and the adjoint
    sweeps (3 slabs, reverse z order) perform the in-core driver's operations
    on the same values: J to double rounding, dJ/dv bit for bit.  Segments of
    7 steps end on a depth-1 sweep; 51 = 5 x 10 + 1 ends on a one-step segment."""
    torch = torch_cuda()
    A, prob_in, v, v_true = _ooc_problem(P, 0, K, nsteps)
    _, prob_oc, _, _ = _ooc_problem(P, 0, K, nsteps, budget=8 << 30)
    d = A.receiver_data(torch.from_numpy(v_true).cuda(), prob_in)
    out = []
    for prob in (prob_in, prob_oc):
        vt = torch.from_numpy(v).cuda().requires_grad_(True)
        J = A.wave_misfit(vt, d, prob)
        J.backward()
        out.append((float(J.detach()), vt.grad.clone()))
    (J0, g0), (J1, g1) = out
    assert J0 > 0 and abs(J1 - J0) <= 1e-12 * J0
    assert float(g0.abs().max()) > 0
    assert torch.equal(g0, g1)


def test_out_of_core_gradient_rate16_vs_oracle(P, orc):
    torch = torch_cuda()
    A, prob, v, v_true = _ooc_problem(P, 16, 10, 60, budget=8 << 30)
    s = prob.dt / prob.dx
    src_zyx = prob.src_xyz[::-1]
    mt64 = (v_true.astype(np.float64) * s) ** 2
    d = orc.wave_receiver_data(mt64, prob.coef, prob.nsteps, src_zyx, prob.wavelet, prob.zr)
    J_ref, gm_ref = orc.wave_misfit_gradient((v.astype(np.float64) * s) ** 2, prob.coef, prob.nsteps, src_zyx,
                                             prob.wavelet, prob.zr, d)
    gv_ref = gm_ref * 2.0 * v.astype(np.float64) * s * s
    vt = torch.from_numpy(v).cuda().requires_grad_(True)
    J = A.wave_misfit(vt, torch.from_numpy(d.astype(np.float32)).cuda(), prob)
    J.backward()
    assert J_ref > 0 and abs(float(J.detach()) - J_ref) <= 1e-3 * J_ref
    assert rel_l2(vt.grad.cpu().numpy(), gv_ref) <= 2e-3


def test_adjoint_multi_step_needs_the_forward_states(P):
    """More than one adjoint step per call reads u^(k-1) from a state record:
    without one the call is refused, and a record that lacks a needed state is
    refused before anything is enqueued (the context stays usable)."""
    torch = torch_cuda()
    A, prob, v, _ = _ooc_problem(P, 16, 10, 20, budget=8 << 30)
    adj = P.OutOfCoreStencil(A._ooc_desc(prob, P.OOCS_WAVE_ADJOINT, 1))
    try:
        adj.synchronize(60.0)
        adj.set_time(6)
        with pytest.raises(P.OOCSError) as e:
            adj.step(2)
        assert e.value.status == 1
        nb = adj.plan.host_store_bytes
        ring = torch.zeros((3, nb), dtype=torch.uint8, pin_memory=True)
        P.oocs_set_state_record(adj.ctx, [ring[i].data_ptr() for i in range(3)], 4)  # u^4 .. u^6
        with pytest.raises(P.OOCSError) as e:
            adj.step(3)  # k = 6, 5, 4 needs u^5, u^4, u^3
        assert e.value.status == 6
        adj.step(2)  # u^5, u^4: allowed
        adj.synchronize(60.0)
        assert adj.stats()["steps_done"] == 4
    finally:
        adj.close()
