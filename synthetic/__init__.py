"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module only draws numbers and lays out input fields.  It holds none of the
stencil or codec arithmetic, so the CPU oracle and the CUDA path can both take
their inputs from here without sharing any of the method.

Random numbers come from a counter-based generator: SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), applied
to ``key(seed) + index``.  Uniform floats keep the top 24 bits of the 64-bit
output, so every value is exactly representable in FP32 and the same field is
obtained on any machine.

Workloads stand in for the paper's acoustic dataset (Table 1: four datasets of
(1152+2*4)^3 doubles), which is not available: a layered velocity model with
noise and a Ricker point source for the 25-point wave stencil, and a noisy
field with a discrete sine mode for the 7-point heat stencil.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function of a uint64 counter array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (x.astype(np.uint64) + _GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        k = splitmix64(np.array([np.uint64(seed) * np.uint64(1_000_003) + np.uint64(stream)],
                                dtype=np.uint64))[0]
    return k


def uniform01(seed: int, n: int, stream: int = 0, offset: int = 0) -> np.ndarray:
    """n floats in [0, 1), each the top 24 bits of SplitMix64(key + offset + i) over 2^24.

    Counter-based: ``uniform01(s, n, offset=o)[i] == uniform01(s, o + n)[o + i]``.
    """
    key = _key(seed, stream)
    with np.errstate(over="ignore"):
        ctr = key + np.arange(offset, offset + n, dtype=np.uint64)
    bits = splitmix64(ctr) >> np.uint64(40)
    return (bits.astype(np.float64) * (1.0 / 16777216.0)).astype(np.float32)


# ----------------------------------------------------------------------------
# 7-point heat workload (128^3, alpha = 0.1)
# ----------------------------------------------------------------------------

def sine_mode(n: int) -> np.ndarray:
    """sin(pi i/(n-1)) sin(pi j/(n-1)) sin(pi k/(n-1)) on nodes 0..n-1, FP64, [z][y][x]."""
    s = np.sin(np.pi * np.arange(n) / (n - 1))
    s[0] = 0.0
    s[-1] = 0.0
    return s[:, None, None] * s[None, :, None] * s[None, None, :]


def heat_initial(n: int = 128, seed: int = 1, noise: bool = True, mode: bool = True) -> np.ndarray:
    """Initial FP32 field of the heat workload: seeded U[0,1) noise plus the sine mode.

    The Dirichlet shell (any index 0 or n-1) is exactly zero; noise is added to
    interior nodes only.  Layout [z][y][x], x fastest.
    """
    f = np.zeros((n, n, n), dtype=np.float64)
    if mode:
        f += sine_mode(n)
    if noise:
        f += uniform01(seed, n * n * n).astype(np.float64).reshape(n, n, n)
    f[0, :, :] = f[-1, :, :] = 0.0
    f[:, 0, :] = f[:, -1, :] = 0.0
    f[:, :, 0] = f[:, :, -1] = 0.0
    return f.astype(np.float32)


def uniform_field(shape, seed: int) -> np.ndarray:
    """FP32 U[0,1) field of the given (nz, ny, nx) shape, shell of width 1 zeroed."""
    nz, ny, nx = shape
    f = uniform01(seed, nz * ny * nx).reshape(nz, ny, nx)
    f[0] = f[-1] = 0.0
    f[:, 0] = f[:, -1] = 0.0
    f[:, :, 0] = f[:, :, -1] = 0.0
    return f


# ----------------------------------------------------------------------------
# 25-point acoustic wave workload (512^3, dx = 10 m, dt = 0.8 ms)
# ----------------------------------------------------------------------------

WAVE_DX = 10.0          # m
WAVE_DT = 0.8e-3        # s; Courant 4725*0.8e-3/10 = 0.378
WAVE_F0 = 15.0          # Hz, Ricker peak frequency
WAVE_VMIN = 1500.0      # m/s
WAVE_VMAX = 4500.0      # m/s
WAVE_NOISE = 0.05       # +-5 % uniform multiplicative noise
WAVE_LAYERS = 8


def layered_velocity(shape, seed: int = 2, layers: int = WAVE_LAYERS,
                     vmin: float = WAVE_VMIN, vmax: float = WAVE_VMAX,
                     noise: float = WAVE_NOISE) -> np.ndarray:
    """Layered velocity model v[z][y][x] in m/s (FP64).

    ``layers`` layers stacked along z whose inner boundaries are seeded sorted
    depths; layer velocities rise linearly from vmin to vmax; every voxel is then
    scaled by (1 + U(-noise, noise)).
    """
    nz, ny, nx = shape
    cuts = np.sort((uniform01(seed, layers - 1, stream=1).astype(np.float64) * nz).astype(np.int64))
    layer_of_z = np.searchsorted(cuts, np.arange(nz), side="right")
    vel_layer = vmin + (vmax - vmin) * np.arange(layers) / max(layers - 1, 1)
    v = np.broadcast_to(vel_layer[layer_of_z][:, None, None], (nz, ny, nx)).astype(np.float64)
    u = uniform01(seed, nz * ny * nx, stream=2).astype(np.float64).reshape(nz, ny, nx)
    return v * (1.0 + noise * (2.0 * u - 1.0))


def wave_model(shape, seed: int = 2, dt: float = WAVE_DT, dx: float = WAVE_DX) -> np.ndarray:
    """FP32 model field m = (v dt / dx)^2 of the layered velocity model."""
    v = layered_velocity(shape, seed)
    return ((v * dt / dx) ** 2).astype(np.float32)


def ricker(nsteps: int, dt: float = WAVE_DT, f0: float = WAVE_F0, t0: float | None = None) -> np.ndarray:
    """Ricker wavelet samples w[n] = (1 - 2 (pi f0 (t-t0))^2) exp(-(pi f0 (t-t0))^2), t = n dt, FP32."""
    if t0 is None:
        t0 = 1.0 / f0
    t = np.arange(nsteps, dtype=np.float64) * dt
    a = (math.pi * f0 * (t - t0)) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(np.float32)


def centre(shape):
    """Grid centre (z, y, x) = (nz/2, ny/2, nx/2) used as the source voxel."""
    nz, ny, nx = shape
    return nz // 2, ny // 2, nx // 2


# 8th-order central second-derivative weights (Fornberg), for offsets 0..4.
WAVE_COEF_1D = (-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0)


def wave_star_coef() -> np.ndarray:
    """Coefficients [centre, c1..c4] of the 3D 25-point star: centre = 3 c0 (FP64)."""
    c = np.array(WAVE_COEF_1D, dtype=np.float64)
    c[0] *= 3.0
    return c


def heat_star_coef(alpha: float = 0.1) -> np.ndarray:
    """Coefficients [centre, c1] of u' = u + alpha (sum6 - 6u): [1 - 6 alpha, alpha] (FP64)."""
    return np.array([1.0 - 6.0 * alpha, alpha], dtype=np.float64)


def blocks_field(shape, seed: int, kind: str) -> np.ndarray:
    """FP32 test fields for the codec: 'noise', 'smooth', 'zero', 'const', 'mixed', 'tiny', 'huge'."""
    nz, ny, nx = shape
    n = nz * ny * nx
    if kind == "zero":
        return np.zeros(shape, np.float32)
    if kind == "const":
        return np.full(shape, 0.7314, np.float32)
    u = uniform01(seed, n, stream=7).astype(np.float64).reshape(shape)
    if kind == "noise":
        return (2.0 * u - 1.0).astype(np.float32)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    smooth = np.sin(0.11 * x + 0.3) * np.cos(0.07 * y - 0.2) * np.sin(0.05 * z + 1.1) * 3.0
    if kind == "smooth":
        return smooth.astype(np.float32)
    if kind == "mixed":
        # magnitudes spanning many binades plus signs, noise and structure
        e = np.floor(u * 40.0) - 20.0
        s = np.where(uniform01(seed, n, stream=8).reshape(shape) < 0.5, -1.0, 1.0)
        return (s * np.exp2(e) * (1.0 + 0.5 * smooth)).astype(np.float32)
    if kind == "tiny":
        return ((2.0 * u - 1.0) * 1e-30).astype(np.float32)
    if kind == "huge":
        return ((2.0 * u - 1.0) * 3e38).astype(np.float32)
    raise ValueError(kind)


# ----------------------------------------------------------------------------
# Accuracy bars of each workload against the FP64 oracle, fixed before any
# timed run.
#
# Relative L2 error ||got - ref|| / ||ref||: uncompressed FP32 runs 1e-6
# (heat), 1e-5 (wave); compressed, per codec rate in bits/value.
#
# Max-abs error, point by point, against the field's peak:
# max |got - ref| <= bar * max |ref|, with each bar ten times the rel-L2 bar of
# the same run.  An error confined to a few points (a wrong halo plane at a
# slab seam, a source or receiver in the wrong slab) is of the order of the
# field itself there and fails it, while it can pass a global L2 norm; spread
# codec or rounding error stays well inside it.  Single kernels (one adjoint or
# gradient step in FP32): 1e-6 and 1e-5.
# ----------------------------------------------------------------------------

TOL_UNCOMPRESSED = {"heat": 1e-6, "wave": 1e-5}
TOL_COMPRESSED = {16: 1e-4, 12: 2e-3, 8: 3e-2}
TOL_MAXABS_UNCOMPRESSED = {"heat": 1e-5, "wave": 1e-4}
TOL_MAXABS_COMPRESSED = {16: 1e-3, 12: 2e-2, 8: 3e-1}
TOL_KERNEL, TOL_MAXABS_KERNEL = 1e-6, 1e-5


# ----------------------------------------------------------------------------
# Batched workload: many independent problems of uneven size
# ----------------------------------------------------------------------------

def batch_shapes(n: int, seed: int = 9, lo: int = 64, hi: int = 384, step: int = 16):
    """n (scheme, (nz, ny, nx)) pairs: every side drawn independently from
    {lo, lo + step, ..., hi}, heat and wave alternating."""
    k = (hi - lo) // step + 1
    u = uniform01(seed, 3 * n)
    sides = (lo + step * np.minimum((u * k).astype(np.int64), k - 1)).reshape(n, 3)
    return [("heat" if i % 2 == 0 else "wave", tuple(int(v) for v in sides[i])) for i in range(n)]


def wave_initial(shape, seed: int, amplitude: float = 1e-3) -> np.ndarray:
    """FP32 amplitude * U[0,1) field with the 4-wide shell of the 25-point star zeroed."""
    nz, ny, nx = shape
    f = (amplitude * uniform01(seed, nz * ny * nx)).astype(np.float32).reshape(nz, ny, nx)
    f[:4] = f[-4:] = 0.0
    f[:, :4] = f[:, -4:] = 0.0
    f[:, :, :4] = f[:, :, -4:] = 0.0
    return f


# ----------------------------------------------------------------------------
# The same generator in PyTorch (for fields too large to draw on the host)
# ----------------------------------------------------------------------------

def _signed(u: int) -> int:
    return u - (1 << 64) if u >= (1 << 63) else u


def _srl(torch, x, k: int):
    """Logical right shift of int64 lanes holding uint64 bit patterns."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def uniform01_torch(seed: int, n: int, offset: int = 0, stream: int = 0, device="cpu"):
    """uniform01(seed, n, stream, offset) as an FP32 torch tensor on `device`,
    bit for bit (int64 lanes wrap like uint64 for +, *, ^ and masked shifts)."""
    import torch
    key = _signed(int(_key(seed, stream)))
    z = torch.arange(offset, offset + n, dtype=torch.int64, device=device) + key
    z = z + _signed(int(_GOLDEN))
    z = (z ^ _srl(torch, z, 30)) * _signed(int(_M1))
    z = (z ^ _srl(torch, z, 27)) * _signed(int(_M2))
    z = z ^ _srl(torch, z, 31)
    bits = _srl(torch, z, 40)
    return bits.to(torch.float32) * (1.0 / 16777216.0)


def uniform_field_planes_torch(shape, seed: int, z0: int, z1: int, device="cpu"):
    """Planes [z0, z1) of uniform_field(shape, seed) as a torch tensor on `device`."""
    nz, ny, nx = shape
    plane = ny * nx
    f = uniform01_torch(seed, (z1 - z0) * plane, offset=z0 * plane, device=device).reshape(z1 - z0, ny, nx)
    if z0 == 0:
        f[0] = 0.0
    if z1 == nz:
        f[-1] = 0.0
    f[:, 0] = 0.0
    f[:, -1] = 0.0
    f[:, :, 0] = 0.0
    f[:, :, -1] = 0.0
    return f


def uniform_field_box(shape, seed: int, z0: int, y0: int, x0: int, n: int) -> np.ndarray:
    """The n^3 box of uniform_field(shape, seed) starting at (z0, y0, x0), drawn
    directly from the counter (no need to hold the field); the box must lie
    inside the grid, and the field's zero shell (any index 0 or n-1) is kept."""
    nz, ny, nx = shape
    assert 0 <= z0 and z0 + n <= nz and 0 <= y0 and y0 + n <= ny and 0 <= x0 and x0 + n <= nx
    z = np.arange(z0, z0 + n, dtype=np.uint64)[:, None, None]
    y = np.arange(y0, y0 + n, dtype=np.uint64)[None, :, None]
    x = np.arange(x0, x0 + n, dtype=np.uint64)[None, None, :]
    key = _key(seed, 0)
    with np.errstate(over="ignore"):
        idx = (z * np.uint64(ny) + y) * np.uint64(nx) + x + key
    bits = splitmix64(idx) >> np.uint64(40)
    f = (bits.astype(np.float64) * (1.0 / 16777216.0)).astype(np.float32)
    shell = ((z == 0) | (z == nz - 1)) | ((y == 0) | (y == ny - 1)) | ((x == 0) | (x == nx - 1))
    f[np.broadcast_to(shell, f.shape)] = 0.0
    return f
