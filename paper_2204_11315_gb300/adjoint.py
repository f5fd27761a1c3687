"""Gradient of the receiver misfit of the wave scheme as a torch.autograd.Function.

Forward: u^(n+1) = 2u^n - u^(n-1) + m (L u^n + w_n e_src) from rest, m = (v dt/dx)^2,
J = 1/2 sum_{n=1..N} |u^n(z_r) - d^n|^2.  Backward: the discrete adjoint run
backwards in time (oocs_adjoint_step) with gradient accumulation
(oocs_gradient_accumulate).  The forward states are not kept: every
`checkpoint_every` steps the pair (u^n, u^(n-1)) is compressed with the
fixed-rate block codec (the same codec the out-of-core sweep streams, Sec. 4.2)
and the backward pass recomputes each segment from its checkpoint, so device
memory holds the compressed checkpoints plus one segment of states.

This module only orchestrates calls to the C ABI (include/oocs.h); every
arithmetic step runs in the library's CUDA kernels.  PyTorch provides the
device buffers and the stream.
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
    wavelet: np.ndarray          # w[n] added at the source on step n (>= nsteps values)
    zr: int                      # receiver plane (interior z)
    nsteps: int
    checkpoint_every: int = 10
    rate: int = 16               # codec rate of the checkpoints; 0 = raw copies
    _desc: object = field(default=None, repr=False)

    def desc(self):
        if self._desc is None:
            nz, ny, nx = self.shape
            self._desc = O.make_desc(nx, ny, nz, O.OOCS_WAVE, self.coef, 1 << 40, rate_bits=0,
                                     temporal_depth=1, slab_planes=nz)
        return self._desc


def _ptr(t):
    return t.data_ptr()


class _Checkpoints:
    """Compressed (or raw) copies of (u^s, u^(s-1)) at segment starts, on the device."""

    def __init__(self, torch, prob: WaveProblem, device):
        self.torch = torch
        self.prob = prob
        nz, ny, nx = prob.shape
        self.n = nz * ny * nx
        self.words = self.n * prob.rate // 32 if prob.rate else 0
        self.device = device
        self.store = {}

    def put(self, s, u, up, stream):
        torch, p = self.torch, self.prob
        nz, ny, nx = p.shape
        if p.rate:
            a = torch.empty(self.words, dtype=torch.int32, device=self.device)
            b = torch.empty(self.words, dtype=torch.int32, device=self.device)
            O.oocs_encode_device(_ptr(u), nx, ny, nz, p.rate, _ptr(a), stream)
            O.oocs_encode_device(_ptr(up), nx, ny, nz, p.rate, _ptr(b), stream)
        else:
            a, b = u.clone(), up.clone()
        self.store[s] = (a, b)

    def get(self, s, u, up, stream):
        p = self.prob
        nz, ny, nx = p.shape
        a, b = self.store[s]
        if p.rate:
            O.oocs_decode_device(_ptr(a), nx, ny, nz, p.rate, _ptr(u), stream)
            O.oocs_decode_device(_ptr(b), nx, ny, nz, p.rate, _ptr(up), stream)
        else:
            u.copy_(a)
            up.copy_(b)

    def nbytes(self):
        return sum(a.numel() * a.element_size() + b.numel() * b.element_size()
                   for a, b in self.store.values())


def _forward_step(prob, m, u, up, scratch, n, stream):
    """One leapfrog step in place: (u, up) <- (u^(n+1), u^n)."""
    w = np.ascontiguousarray(prob.wavelet, dtype=np.float32)
    O.oocs_incore_run(prob.desc(), _ptr(u), _ptr(up), _ptr(m), _ptr(scratch), 1, n,
                      prob.src_xyz, w, stream)


def _make_function():
    import torch

    class WaveMisfit(torch.autograd.Function):
        @staticmethod
        def forward(ctx, v, d_obs, prob: WaveProblem):
            assert v.is_cuda and v.dtype == torch.float32 and v.is_contiguous()
            nz, ny, nx = prob.shape
            n = nz * ny * nx
            plane = ny * nx
            N = prob.nsteps
            stream = torch.cuda.current_stream(v.device).cuda_stream
            m = torch.empty_like(v)
            O.oocs_model_from_velocity(_ptr(v), _ptr(m), n, prob.dt / prob.dx, stream)
            u = torch.zeros_like(v)
            up = torch.zeros_like(v)
            scratch = torch.empty_like(v)
            res = torch.empty((N, ny, nx), dtype=torch.float32, device=v.device)
            misfit = torch.zeros(1, dtype=torch.float64, device=v.device)
            ck = _Checkpoints(torch, prob, v.device)
            for step in range(N):
                if step % prob.checkpoint_every == 0:
                    ck.put(step, u, up, stream)
                _forward_step(prob, m, u, up, scratch, step, stream)
                O.oocs_receiver_residual(_ptr(u) + 4 * prob.zr * plane, _ptr(d_obs[step]), plane,
                                         _ptr(res[step]), _ptr(misfit), stream)
            ctx.prob = prob
            ctx.ck = ck
            ctx.save_for_backward(v, m, res)
            return misfit[0]

        @staticmethod
        def backward(ctx, gJ):
            v, m, res = ctx.saved_tensors
            prob, ck = ctx.prob, ctx.ck
            desc = prob.desc()
            nz, ny, nx = prob.shape
            n = nz * ny * nx
            N, K = prob.nsteps, prob.checkpoint_every
            stream = torch.cuda.current_stream(v.device).cuda_stream
            w = np.asarray(prob.wavelet, dtype=np.float64)
            lam = torch.zeros_like(v)       # lam^(n+1)
            lam_prev = torch.zeros_like(v)  # lam^(n+2)
            mu = torch.zeros_like(v)        # m lam^(n+1)
            mu_out = torch.zeros_like(v)
            grad_m = torch.zeros_like(v)
            states = torch.empty((K + 1,) + tuple(prob.shape), dtype=torch.float32, device=v.device)
            u = torch.empty_like(v)
            up = torch.empty_like(v)
            scratch = torch.empty_like(v)
            for s in reversed(range(0, N, K)):
                e = min(s + K, N)
                ck.get(s, u, up, stream)          # (u^s, u^(s-1))
                states[0].copy_(u)
                for step in range(s, e):          # states[i] = u^(s+i)
                    _forward_step(prob, m, u, up, scratch, step, stream)
                    states[step + 1 - s].copy_(u)
                for k in range(e, s, -1):         # lam^k, then the term n = k-1
                    O.oocs_adjoint_step(desc, _ptr(lam), _ptr(lam_prev), _ptr(mu), _ptr(mu_out), _ptr(m),
                                        _ptr(res[k - 1]), prob.zr, stream)
                    lam, lam_prev = lam_prev, lam  # lam = lam^k, lam_prev = lam^(k+1)
                    mu, mu_out = mu_out, mu
                    O.oocs_gradient_accumulate(desc, _ptr(grad_m), _ptr(lam), _ptr(states[k - 1 - s]),
                                               float(w[k - 1]), prob.src_xyz, stream)
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
    """Plane z_r of u^1 .. u^N of the forward run from rest, [N][ny][nx] on the device."""
    import torch
    nz, ny, nx = prob.shape
    n = nz * ny * nx
    stream = torch.cuda.current_stream(v.device).cuda_stream
    m = torch.empty_like(v)
    O.oocs_model_from_velocity(_ptr(v), _ptr(m), n, prob.dt / prob.dx, stream)
    u = torch.zeros_like(v)
    up = torch.zeros_like(v)
    scratch = torch.empty_like(v)
    out = torch.empty((prob.nsteps, ny, nx), dtype=torch.float32, device=v.device)
    for step in range(prob.nsteps):
        _forward_step(prob, m, u, up, scratch, step, stream)
        out[step].copy_(u[prob.zr])
    return out
