"""Gradient of the receiver misfit of the wave scheme as a torch.autograd.Function.

Forward: u^(n+1) = 2u^n - u^(n-1) + m (L u^n + w_n e_src) from rest, m = (v dt/dx)^2,
J = 1/2 sum_{n=1..N} |u^n(z_r) - d^n|^2.  Backward: the discrete adjoint run
backwards in time with gradient accumulation.  The forward states are not kept:
every `checkpoint_every` steps the pair (u^n, u^(n-1)) is compressed with the
fixed-rate block codec (the same codec the out-of-core sweep streams, Sec. 4.2)
and the backward pass recomputes each segment from its checkpoint, so device
memory holds the compressed checkpoints plus one segment of states.

Both passes are single calls of the library's native driver
(oocs_misfit_forward / oocs_misfit_backward, include/oocs.h); this module only
allocates the workspace with PyTorch and marshals arguments.

With `device_budget` set, the same gradient is computed out of core, for grids
that do not fit the device: the forward run is the slab sweep (Sec. 3.1, k
steps per visit) recording the receiver plane, its checkpoints are snapshots
of the compressed host stores every `checkpoint_every` steps; the backward
pass recomputes each segment's states one step per sweep (snapshotting the
compressed u store after each), then runs one adjoint sweep per time step
(scheme OOCS_WAVE_ADJOINT: slabs in reverse z order, lam streamed through the
codec, m and dJ/dm on the device).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import oocs as O


@dataclass
class WaveProblem:
    """A receiver-misfit problem of the 25-point wave scheme on one GPU."""
    shape: tuple                 # (nz, ny, nx), multiples of 4
    dt: float                    # s
    dx: float                    # m
    coef: np.ndarray             # [centre, c1..c4] of the 3D star
    src_xyz: tuple               # source voxel (x, y, z)
    wavelet: np.ndarray          # w[n] added at the source on step n
    zr: int                      # receiver plane (interior z)
    nsteps: int
    checkpoint_every: int = 10
    rate: int = 16               # codec rate of the checkpoints; 0 = raw copies
    device_budget: int | None = None  # set: out-of-core sweeps within this many bytes
    slab_planes: int = 0         # out of core: T (0 = from the budget)
    forward_depth: int = 0       # out of core: temporal depth of the forward sweep (0 = auto)
    _desc: object = field(default=None, repr=False)

    def desc(self):
        if self._desc is None:
            nz, ny, nx = self.shape
            self._desc = O.make_desc(nx, ny, nz, O.OOCS_WAVE, self.coef, 1 << 40, rate_bits=0,
                                     temporal_depth=1, slab_planes=nz)
        return self._desc

    def wavelet32(self):
        return np.ascontiguousarray(self.wavelet, dtype=np.float32)

    def workspace_bytes(self):
        return O.oocs_misfit_workspace_bytes(self.desc(), self.nsteps, self.checkpoint_every, self.rate)


def _ptr(t):
    return t.data_ptr()


# ------------------------------------------------------------ out of core --

def _ooc_desc(prob: WaveProblem, scheme: int, depth: int):
    nz, ny, nx = prob.shape
    return O.make_desc(nx, ny, nz, scheme, prob.coef, prob.device_budget, rate_bits=prob.rate,
                       temporal_depth=depth, slab_planes=prob.slab_planes, readonly_resident=1)


def _forward_depth(prob: WaveProblem) -> int:
    """The forward sweep's temporal depth: prob.forward_depth when set, else
    the largest divisor of the checkpoint interval K (at most 8) that gives a
    valid plan, so that every segment is a whole number of sweeps (K = 10:
    depth 5, two sweeps per segment instead of 4 + 4 + 2; measured 91 against
    111 ms for the 256^3 x 400-step forward pass in four slabs)."""
    if prob.forward_depth:
        return prob.forward_depth
    K = prob.checkpoint_every
    for d in sorted((d for d in range(1, min(K, 8) + 1) if K % d == 0), reverse=True):
        try:
            O.oocs_query(_ooc_desc(prob, O.OOCS_WAVE, d))
            return d
        except O.OOCSError:
            continue
    return 1


def _ooc_forward(torch, m, d_obs, prob: WaveProblem):
    """Slab-swept forward run from rest: the receiver record, the residuals, J
    and the checkpoints, the compressed (u^s, u^(s-1)) stores at every segment
    start s, which the sweep ending at s writes into the state record."""
    nz, ny, nx = prob.shape
    plane = ny * nx
    N, K = prob.nsteps, prob.checkpoint_every
    dev = m.device
    st = O.OutOfCoreStencil(_ooc_desc(prob, O.OOCS_WAVE, _forward_depth(prob)), device=dev.index or 0)
    try:
        zero = torch.zeros(prob.shape, dtype=torch.float32, device=dev)
        torch.cuda.synchronize(dev)  # m and zero are written on torch's stream
        for f, src in ((O.OOCS_FIELD_U, zero), (O.OOCS_FIELD_U_PREV, zero), (O.OOCS_FIELD_M, m)):
            O.oocs_compress_device(st.ctx, f, _ptr(src), 0, nz)
        st.set_source(*prob.src_xyz, prob.wavelet32())
        rec = torch.empty((N, ny, nx), dtype=torch.float32, device=dev)
        O.oocs_set_receiver(st.ctx, prob.zr, _ptr(rec), N)
        starts = list(range(0, N, K))
        pool = torch.empty((len(starts), 2, st.plan.host_store_bytes), dtype=torch.uint8, pin_memory=True)
        st.synchronize(600.0)
        pool[0, 0].copy_(st.stores[O.OOCS_FIELD_U])
        pool[0, 1].copy_(st.stores[O.OOCS_FIELD_U_PREV])
        ptrs = [0] * (N + 1)  # entry t + 1: state u^t, t = -1 .. N - 1
        for i, s0 in enumerate(starts[1:], 1):
            ptrs[s0 + 1], ptrs[s0] = pool[i, 0].data_ptr(), pool[i, 1].data_ptr()
        O.oocs_set_state_record(st.ctx, ptrs, -1)
        for s0 in starts:  # each call ends its last sweep at the next segment start
            st.step(min(K, N - s0))
        st.synchronize(3600.0)
        res = torch.empty_like(rec)
        misfit = torch.zeros(1, dtype=torch.float64, device=dev)
        O.oocs_receiver_residual(_ptr(rec), _ptr(d_obs), N * plane, _ptr(res), _ptr(misfit),
                                 torch.cuda.current_stream(dev).cuda_stream)
        torch.cuda.synchronize(dev)
    finally:
        st.close()
    return misfit, res, {s0: (pool[i, 0], pool[i, 1]) for i, s0 in enumerate(starts)}


def _ooc_backward(torch, m, res, ckpt, prob: WaveProblem):
    """dJ/dm by adjoint sweeps over the segments in reverse.  Each segment's
    states u^s .. u^(e-1) are recomputed from its checkpoint by sweeps of
    depth 2 (the first of depth 1), whose two outputs the state record keeps;
    the recomputation of one segment overlaps the adjoint sweeps of the
    segment after it (two record rings, ordered by events on stream 0)."""
    nz, ny, nx = prob.shape
    N, K = prob.nsteps, prob.checkpoint_every
    dev = m.device
    fwd = O.OutOfCoreStencil(_ooc_desc(prob, O.OOCS_WAVE, 2), device=dev.index or 0)
    adj = O.OutOfCoreStencil(_ooc_desc(prob, O.OOCS_WAVE_ADJOINT, 1), device=dev.index or 0)
    try:
        torch.cuda.synchronize(dev)
        O.oocs_compress_device(fwd.ctx, O.OOCS_FIELD_M, _ptr(m), 0, nz)
        O.oocs_compress_device(adj.ctx, O.OOCS_FIELD_M, _ptr(m), 0, nz)
        fwd.set_source(*prob.src_xyz, prob.wavelet32())
        adj.set_source(*prob.src_xyz, prob.wavelet32())
        O.oocs_set_receiver(adj.ctx, prob.zr, _ptr(res), N)
        # lam^N = r^(N-1) on the receiver plane's interior, lam^(N+1) = 0
        lam = torch.zeros(prob.shape, dtype=torch.float32, device=dev)
        lam[prob.zr, 4:ny - 4, 4:nx - 4] = res[N - 1, 4:ny - 4, 4:nx - 4]
        zero = torch.zeros_like(lam)
        torch.cuda.synchronize(dev)
        O.oocs_compress_device(adj.ctx, O.OOCS_FIELD_LAM, _ptr(lam), 0, nz)
        O.oocs_compress_device(adj.ctx, O.OOCS_FIELD_LAM_PREV, _ptr(zero), 0, nz)
        adj.synchronize(600.0)
        del lam, zero
        nb = fwd.plan.host_store_bytes
        rings = [torch.empty((K, nb), dtype=torch.uint8, pin_memory=True) for _ in range(2)]
        ring_free = [None, None]  # event after the adjoint sweeps that last read each ring
        for j, s0 in enumerate(reversed(range(0, N, K))):
            e0 = min(s0 + K, N)
            ring = rings[j % 2]
            ck_u, ck_p = ckpt[s0]
            if e0 - s0 == 1:
                states = [ck_u]
            else:
                if ring_free[j % 2] is not None:
                    fwd.streams[0].wait_event(ring_free[j % 2])
                # the checkpoint stores are consumed: the sweeps overwrite them
                fwd.bind(O.OOCS_FIELD_U, ck_u)
                fwd.bind(O.OOCS_FIELD_U_PREV, ck_p)
                fwd.set_time(s0)
                O.oocs_set_state_record(fwd.ctx, [ring[i].data_ptr() for i in range(K)], s0)
                fwd.step(1)                # u^(s0+1) and u^s0
                if e0 - s0 > 2:
                    fwd.step(e0 - s0 - 2)  # u^(s0+2) .. u^(e0-1), two per sweep
                done = torch.cuda.Event()
                done.record(fwd.streams[0])
                adj.streams[0].wait_event(done)
                states = [ring[i] for i in range(e0 - s0)]
            # the segment's adjoint steps k = e0 .. s0+1 in one call: lam^k and
            # u^(k-1) -> the dJ/dm term k-1 and lam^(k-1)
            O.oocs_set_state_record(adj.ctx, [st.data_ptr() for st in states], s0)
            adj.set_time(e0)
            adj.step(e0 - s0)
            ev = torch.cuda.Event()
            ev.record(adj.streams[0])
            ring_free[j % 2] = ev
        adj.synchronize(3600.0)
        fwd.synchronize(600.0)
        grad_m = torch.empty_like(m)
        O.oocs_decompress_device(adj.ctx, O.OOCS_FIELD_GRAD, _ptr(grad_m), 0, nz)
        adj.synchronize(600.0)
    finally:
        fwd.close()
        adj.close()
    return grad_m


def _make_function():
    import torch

    class WaveMisfit(torch.autograd.Function):
        @staticmethod
        def forward(ctx, v, d_obs, prob: WaveProblem):
            assert v.is_cuda and v.dtype == torch.float32 and v.is_contiguous()
            assert d_obs.is_cuda and d_obs.dtype == torch.float32 and d_obs.is_contiguous()
            nz, ny, nx = prob.shape
            n = nz * ny * nx
            stream = torch.cuda.current_stream(v.device).cuda_stream
            m = torch.empty_like(v)
            O.oocs_model_from_velocity(_ptr(v), _ptr(m), n, prob.dt / prob.dx, stream)
            if prob.device_budget is not None:
                misfit, res, ckpt = _ooc_forward(torch, m, d_obs, prob)
                ctx.prob, ctx.ckpt, ctx.ws = prob, ckpt, None
                ctx.save_for_backward(v, m, res)
                return misfit[0]
            nbytes = prob.workspace_bytes()
            ws = torch.empty(nbytes, dtype=torch.uint8, device=v.device)
            res = torch.empty((prob.nsteps, ny, nx), dtype=torch.float32, device=v.device)
            misfit = torch.empty(1, dtype=torch.float64, device=v.device)
            O.oocs_misfit_forward(prob.desc(), _ptr(m), prob.src_xyz, prob.wavelet32(), prob.zr,
                                  _ptr(d_obs), prob.nsteps, prob.checkpoint_every, prob.rate, _ptr(ws),
                                  nbytes, _ptr(res), _ptr(misfit), stream)
            ctx.prob = prob
            ctx.ws = ws
            ctx.save_for_backward(v, m, res)
            return misfit[0]

        @staticmethod
        def backward(ctx, gJ):
            v, m, res = ctx.saved_tensors
            prob, ws = ctx.prob, ctx.ws
            n = v.numel()
            stream = torch.cuda.current_stream(v.device).cuda_stream
            if prob.device_budget is not None:
                grad_m = _ooc_backward(torch, m, res, ctx.ckpt, prob)
                ctx.ckpt = None
            else:
                grad_m = torch.empty_like(v)
                O.oocs_misfit_backward(prob.desc(), _ptr(m), prob.src_xyz, prob.wavelet32(), prob.zr, _ptr(res),
                                       prob.nsteps, prob.checkpoint_every, prob.rate, _ptr(ws), ws.numel(),
                                       _ptr(grad_m), stream)
            ctx.ws = None
            grad_v = torch.empty_like(v)
            O.oocs_velocity_gradient(_ptr(grad_m), _ptr(v), _ptr(grad_v), n, prob.dt / prob.dx, stream)
            if not (gJ.numel() == 1 and float(gJ) == 1.0):
                grad_v = grad_v * gJ.to(grad_v.dtype)
            return grad_v, None, None

    return WaveMisfit


_WaveMisfit = None


def wave_misfit(v, d_obs, prob: WaveProblem):
    """J(v) as a differentiable scalar (float64 CUDA tensor); .backward() gives dJ/dv."""
    global _WaveMisfit
    if _WaveMisfit is None:
        _WaveMisfit = _make_function()
    return _WaveMisfit.apply(v, d_obs, prob)


def receiver_data(v, prob: WaveProblem):
    """Plane z_r of u^1 .. u^N of the forward run from rest, [N][ny][nx] on the device
    (the residuals of a forward run against zero data)."""
    import torch
    nz, ny, nx = prob.shape
    n = nz * ny * nx
    stream = torch.cuda.current_stream(v.device).cuda_stream
    m = torch.empty_like(v)
    O.oocs_model_from_velocity(_ptr(v), _ptr(m), n, prob.dt / prob.dx, stream)
    zero = torch.zeros((prob.nsteps, ny, nx), dtype=torch.float32, device=v.device)
    out = torch.empty_like(zero)
    misfit = torch.empty(1, dtype=torch.float64, device=v.device)
    nbytes = prob.workspace_bytes()
    ws = torch.empty(nbytes, dtype=torch.uint8, device=v.device)
    O.oocs_misfit_forward(prob.desc(), _ptr(m), prob.src_xyz, prob.wavelet32(), prob.zr, _ptr(zero),
                          prob.nsteps, prob.checkpoint_every, prob.rate, _ptr(ws), nbytes, _ptr(out),
                          _ptr(misfit), stream)
    return out
