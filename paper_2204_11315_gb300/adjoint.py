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
