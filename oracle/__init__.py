"""CPU oracle for the compressed out-of-core stencil method (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares no
code with the CUDA path (``paper_2204_11315_gb300``), which never imports it.

The arithmetic lives in ``oracle.c`` (plain C, FP64 stencils, reference block
codec); this module compiles it with gcc on first use and wraps it with ctypes
and numpy.  See ``oracle.c`` for what each function computes and which part of
the paper it follows (Sec. 3.1 and Sec. 6 for the stencils, Sec. 4.2 and Sec. 5
for the fixed-rate codec).

Parity status: the stencil functions are pinned by closed forms and brute
force; the codec by exact sizes, bijective stages, lossless coding at full
budget and its error bound.  Bit compatibility with cuZFP itself is "parity
unpinned": neither zfp nor its bitstream definition is available.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
          "-std=c11", "-Wall"]


def build(force: bool = False) -> str:
    """Compile oracle.c into _liboracle.so (gcc, no CUDA).  Returns the path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


_i64 = ctypes.c_int64
_i32 = ctypes.c_int
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i32p = ctypes.POINTER(ctypes.c_int32)
_ip = ctypes.POINTER(ctypes.c_int)
_i8p = ctypes.POINTER(ctypes.c_int8)


def _declare(L):
    L.oracle_threads.restype = _i32
    L.oracle_star_step.argtypes = [_i64, _i64, _i64, _i32, _dp, _i32, _dp, _dp, _dp, _dp, _i64,
                                   ctypes.c_double]
    L.oracle_heat_run.argtypes = [_i64, _i64, _i64, _i32, _dp, _i32, _dp, _dp]
    L.oracle_wave_run.argtypes = [_i64, _i64, _i64, _dp, _dp, _i32, _dp, _dp, _dp, _i64, _dp]
    L.oracle_star_apply.argtypes = [_i64, _i64, _i64, _i32, _dp, _dp, _dp]
    L.oracle_wave_adjoint_step.argtypes = [_i64, _i64, _i64, _dp, _dp, _dp, _dp, _dp, _dp, _i64, _dp]
    L.oracle_wave_misfit_gradient.argtypes = [_i64, _i64, _i64, _dp, _dp, _i32, _i64, _dp, _i64,
                                              _dp, _dp]
    L.oracle_wave_misfit_gradient.restype = ctypes.c_double
    L.oracle_block_header.argtypes = [_fp]
    L.oracle_block_header.restype = _i32
    L.oracle_quantize.argtypes = [_fp, _i32, _i32p]
    L.oracle_dequantize.argtypes = [_i32p, _i32, _fp]
    L.oracle_fwd_lift4.argtypes = [_i32p]
    L.oracle_inv_lift4.argtypes = [_i32p]
    L.oracle_fwd_xform.argtypes = [_i32p]
    L.oracle_inv_xform.argtypes = [_i32p]
    L.oracle_sequency_order.argtypes = [_ip]
    L.oracle_to_negabinary.argtypes = [ctypes.c_int32]
    L.oracle_to_negabinary.restype = ctypes.c_uint32
    L.oracle_from_negabinary.argtypes = [ctypes.c_uint32]
    L.oracle_from_negabinary.restype = ctypes.c_int32
    L.oracle_encode_planes.argtypes = [_u32p, _i32, _u32p, _i32]
    L.oracle_decode_planes.argtypes = [_u32p, _i32, _i32, _u32p]
    L.oracle_decode_planes.restype = _i32
    L.oracle_encode_block.argtypes = [_fp, _i32, _u32p]
    L.oracle_encode_block.restype = _i32
    L.oracle_decode_block.argtypes = [_u32p, _i32, _fp]
    L.oracle_decode_block.restype = _i32
    L.oracle_encode_field.argtypes = [_fp, _i64, _i64, _i64, _i32, _u32p]
    L.oracle_encode_field.restype = _i64
    L.oracle_decode_field.argtypes = [_u32p, _i64, _i64, _i64, _i32, _fp, _i8p]
    L.oracle_bq_header.argtypes = [_fp]
    L.oracle_bq_header.restype = _i32
    L.oracle_bq_encode_block.argtypes = [_fp, _i32, _u32p]
    L.oracle_bq_encode_block.restype = _i32
    L.oracle_bq_decode_block.argtypes = [_u32p, _i32, _fp]
    L.oracle_bq_encode_field.argtypes = [_fp, _i64, _i64, _i64, _i32, _u32p]
    L.oracle_bq_encode_field.restype = _i64
    L.oracle_bq_decode_field.argtypes = [_u32p, _i64, _i64, _i64, _i32, _fp]


def _p(a, t):
    return a.ctypes.data_as(t)


def threads() -> int:
    """OpenMP threads the oracle loops use on this host."""
    return int(lib().oracle_threads())


# ---------------------------------------------------------------------------
# stencils (FP64)
# ---------------------------------------------------------------------------

def star_step(u, coef, scheme="heat", m=None, up=None, src=None, w=0.0):
    """One FP64 step of the star stencil on the whole grid; returns the new field.

    coef = [centre, c1..cr]; radius r = len(coef) - 1.  scheme 'heat':
    out = L(u); scheme 'wave': out = 2u - up + m (L(u) + w at src).
    """
    u = np.ascontiguousarray(u, dtype=np.float64)
    nz, ny, nx = u.shape
    c = np.ascontiguousarray(coef, dtype=np.float64)
    r = len(c) - 1
    out = np.empty_like(u)
    wave = scheme == "wave"
    mm = np.ascontiguousarray(m, dtype=np.float64) if wave else u
    uu = np.ascontiguousarray(up, dtype=np.float64) if wave else u
    s = -1 if src is None else int((src[0] * ny + src[1]) * nx + src[2])
    lib().oracle_star_step(nx, ny, nz, r, _p(c, _dp), 1 if wave else 0, _p(mm, _dp), _p(u, _dp),
                           _p(uu, _dp), _p(out, _dp), s, float(w))
    return out


def heat_run(u0, coef, nsteps):
    """nsteps FP64 steps of the heat stencil from u0 (any float dtype)."""
    u = np.array(u0, dtype=np.float64, order="C", copy=True)
    nz, ny, nx = u.shape
    c = np.ascontiguousarray(coef, dtype=np.float64)
    scratch = np.empty_like(u)
    lib().oracle_heat_run(nx, ny, nz, len(c) - 1, _p(c, _dp), int(nsteps), _p(u, _dp),
                          _p(scratch, _dp))
    return u


def wave_run(u0, up0, m, coef, nsteps, src=None, w=None):
    """nsteps FP64 leapfrog steps; returns (u^(t+n), u^(t+n-1)).  Step n adds w[n] at src."""
    u = np.array(u0, dtype=np.float64, order="C", copy=True)
    up = np.array(up0, dtype=np.float64, order="C", copy=True)
    mm = np.ascontiguousarray(m, dtype=np.float64)
    nz, ny, nx = u.shape
    c = np.ascontiguousarray(coef, dtype=np.float64)
    assert len(c) == 5
    scratch = np.empty_like(u)
    s = -1 if src is None else int((src[0] * ny + src[1]) * nx + src[2])
    ww = None
    if w is not None:
        ww = np.ascontiguousarray(np.asarray(w, dtype=np.float64)[:nsteps])
        assert len(ww) >= nsteps
    lib().oracle_wave_run(nx, ny, nz, _p(c, _dp), _p(mm, _dp), int(nsteps), _p(u, _dp),
                          _p(up, _dp), _p(scratch, _dp), s,
                          _p(ww, _dp) if ww is not None else None)
    return u, up


def star_apply(u, coef):
    """L u on the interior (0 on the shell of width r = len(coef) - 1), FP64."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    nz, ny, nx = u.shape
    c = np.ascontiguousarray(coef, dtype=np.float64)
    out = np.empty_like(u)
    lib().oracle_star_apply(nx, ny, nz, len(c) - 1, _p(c, _dp), _p(u, _dp), _p(out, _dp))
    return out


def wave_adjoint_step(lam, lam_prev, m, coef, res=None, zr=-1):
    """lam_new = 2 lam - lam_prev + L(m lam) + res at plane zr (shell 0), FP64."""
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    lp = np.ascontiguousarray(lam_prev, dtype=np.float64)
    mm = np.ascontiguousarray(m, dtype=np.float64)
    nz, ny, nx = lam.shape
    c = np.ascontiguousarray(coef, dtype=np.float64)
    out = np.empty_like(lam)
    scratch = np.empty(2 * lam.size)
    rr = np.ascontiguousarray(res, dtype=np.float64) if res is not None else None
    lib().oracle_wave_adjoint_step(nx, ny, nz, _p(c, _dp), _p(mm, _dp), _p(lam, _dp), _p(lp, _dp),
                                   _p(out, _dp), _p(rr, _dp) if rr is not None else None, int(zr),
                                   _p(scratch, _dp))
    return out


def wave_misfit_gradient(m, coef, nsteps, src, w, zr, d):
    """(J, dJ/dm) of the wave workload: forward + discrete adjoint, FP64.

    d[n-1] (ny x nx) is the observed plane zr at time n, n = 1..nsteps."""
    mm = np.ascontiguousarray(m, dtype=np.float64)
    nz, ny, nx = mm.shape
    c = np.ascontiguousarray(coef, dtype=np.float64)
    ww = np.ascontiguousarray(np.asarray(w, dtype=np.float64)[:nsteps])
    dd = np.ascontiguousarray(d, dtype=np.float64)
    assert dd.shape == (nsteps, ny, nx)
    g = np.empty_like(mm)
    s = -1 if src is None else int((src[0] * ny + src[1]) * nx + src[2])
    J = lib().oracle_wave_misfit_gradient(nx, ny, nz, _p(c, _dp), _p(mm, _dp), int(nsteps), s,
                                          _p(ww, _dp), int(zr), _p(dd, _dp), _p(g, _dp))
    return float(J), g


def wave_receiver_data(m, coef, nsteps, src, w, zr):
    """Plane zr of u^1 .. u^nsteps of the forward run from rest, FP64, [n][ny][nx]."""
    mm = np.ascontiguousarray(m, dtype=np.float64)
    u = np.zeros_like(mm)
    up = np.zeros_like(mm)
    out = []
    for k in range(nsteps):
        u, up = wave_run(u, up, mm, coef, 1, src=src, w=np.asarray(w)[k:k + 1])
        out.append(u[zr].copy())
    return np.array(out)


# ---------------------------------------------------------------------------
# codec
# ---------------------------------------------------------------------------

def block_header(v64) -> int:
    v = np.ascontiguousarray(v64, dtype=np.float32).reshape(64)
    return int(lib().oracle_block_header(_p(v, _fp)))


def quantize(v64, emax):
    v = np.ascontiguousarray(v64, dtype=np.float32).reshape(64)
    q = np.empty(64, np.int32)
    lib().oracle_quantize(_p(v, _fp), int(emax), _p(q, _i32p))
    return q


def dequantize(q64, emax):
    q = np.ascontiguousarray(q64, dtype=np.int32).reshape(64)
    v = np.empty(64, np.float32)
    lib().oracle_dequantize(_p(q, _i32p), int(emax), _p(v, _fp))
    return v


def xform_overflowed(reset: bool = True) -> bool:
    """True if any lifting result left int32 since the last reset."""
    flag = ctypes.c_int.in_dll(lib(), "oracle_xform_overflow")
    val = bool(flag.value)
    if reset:
        flag.value = 0
    return val


def fwd_lift4(v4):
    a = np.array(v4, dtype=np.int32).reshape(4).copy()
    lib().oracle_fwd_lift4(_p(a, _i32p))
    return a


def inv_lift4(v4):
    a = np.array(v4, dtype=np.int32).reshape(4).copy()
    lib().oracle_inv_lift4(_p(a, _i32p))
    return a


def fwd_xform(q64):
    a = np.array(q64, dtype=np.int32).reshape(64).copy()
    lib().oracle_fwd_xform(_p(a, _i32p))
    return a


def inv_xform(q64):
    a = np.array(q64, dtype=np.int32).reshape(64).copy()
    lib().oracle_inv_xform(_p(a, _i32p))
    return a


def sequency_order():
    perm = np.empty(64, np.intc)
    lib().oracle_sequency_order(_p(perm, _ip))
    return perm.astype(np.int64)


def to_negabinary(x: int) -> int:
    return int(lib().oracle_to_negabinary(int(np.int32(x))))


def from_negabinary(u: int) -> int:
    return int(lib().oracle_from_negabinary(int(u) & 0xFFFFFFFF))


def encode_planes(u64, budget):
    """Embedded coding of 64 uint32 coefficients into `budget` bits (from bit 0)."""
    u = np.ascontiguousarray(u64, dtype=np.uint32).reshape(64)
    words = np.zeros((budget + 31) // 32 + 1, np.uint32)
    lib().oracle_encode_planes(_p(u, _u32p), int(budget), _p(words, _u32p), 0)
    return words


def decode_planes(words, budget):
    w = np.ascontiguousarray(words, dtype=np.uint32)
    u = np.empty(64, np.uint32)
    low = lib().oracle_decode_planes(_p(w, _u32p), 0, int(budget), _p(u, _u32p))
    return u, int(low)


def encode_block(v64, rate, with_flag=False):
    """Words of one block; with_flag: also whether it held an Inf or NaN
    (such a block is coded as all zeros)."""
    v = np.ascontiguousarray(v64, dtype=np.float32).reshape(64)
    words = np.zeros(2 * rate, np.uint32)
    bad = lib().oracle_encode_block(_p(v, _fp), int(rate), _p(words, _u32p))
    return (words, bool(bad)) if with_flag else words


def decode_block(words, rate):
    w = np.ascontiguousarray(words, dtype=np.uint32).reshape(2 * rate)
    v = np.empty(64, np.float32)
    low = lib().oracle_decode_block(_p(w, _u32p), int(rate), _p(v, _fp))
    return v, int(low)


def encode_field(f, rate, with_nonfinite=False):
    """Compress an [nz][ny][nx] FP32 field (multiples of 4) into uint32 words.

    Block (bx, by, bz) occupies words [(((bz*(ny/4)+by)*(nx/4)+bx)*2*rate, +2*rate).
    with_nonfinite: also return how many blocks held an Inf or NaN.
    """
    f = np.ascontiguousarray(f, dtype=np.float32)
    nz, ny, nx = f.shape
    assert nx % 4 == 0 and ny % 4 == 0 and nz % 4 == 0
    nb = (nx // 4) * (ny // 4) * (nz // 4)
    out = np.zeros(nb * 2 * rate, np.uint32)
    bad = lib().oracle_encode_field(_p(f, _fp), nx, ny, nz, int(rate), _p(out, _u32p))
    return (out, int(bad)) if with_nonfinite else out


def decode_field(words, shape, rate, with_planes=False):
    nz, ny, nx = shape
    w = np.ascontiguousarray(words, dtype=np.uint32)
    nb = (nx // 4) * (ny // 4) * (nz // 4)
    assert w.size == nb * 2 * rate
    f = np.empty((nz, ny, nx), np.float32)
    low = np.empty(nb, np.int8)
    lib().oracle_decode_field(_p(w, _u32p), nx, ny, nz, int(rate), _p(f, _fp), _p(low, _i8p))
    return (f, low) if with_planes else f


# ---------------------------------------------------------------------------
# block quantiser (oracle.c item 3; Sec. 7 future work (1))
# ---------------------------------------------------------------------------

def bq_header(v64) -> int:
    v = np.ascontiguousarray(v64, dtype=np.float32).reshape(64)
    return int(lib().oracle_bq_header(_p(v, _fp)))


def bq_encode_block(v64, rate, with_flag=False):
    v = np.ascontiguousarray(v64, dtype=np.float32).reshape(64)
    words = np.zeros(2 * rate, np.uint32)
    bad = lib().oracle_bq_encode_block(_p(v, _fp), int(rate), _p(words, _u32p))
    return (words, bool(bad)) if with_flag else words


def bq_decode_block(words, rate):
    w = np.ascontiguousarray(words, dtype=np.uint32).reshape(2 * rate)
    v = np.empty(64, np.float32)
    lib().oracle_bq_decode_block(_p(w, _u32p), int(rate), _p(v, _fp))
    return v


def bq_encode_field(f, rate, with_nonfinite=False):
    """Block-quantise an [nz][ny][nx] FP32 field; same block layout as encode_field."""
    f = np.ascontiguousarray(f, dtype=np.float32)
    nz, ny, nx = f.shape
    assert nx % 4 == 0 and ny % 4 == 0 and nz % 4 == 0 and 2 <= rate <= 32
    nb = (nx // 4) * (ny // 4) * (nz // 4)
    out = np.zeros(nb * 2 * rate, np.uint32)
    bad = lib().oracle_bq_encode_field(_p(f, _fp), nx, ny, nz, int(rate), _p(out, _u32p))
    return (out, int(bad)) if with_nonfinite else out


def bq_decode_field(words, shape, rate):
    nz, ny, nx = shape
    w = np.ascontiguousarray(words, dtype=np.uint32)
    assert w.size == (nx // 4) * (ny // 4) * (nz // 4) * 2 * rate
    f = np.empty((nz, ny, nx), np.float32)
    lib().oracle_bq_decode_field(_p(w, _u32p), nx, ny, nz, int(rate), _p(f, _fp))
    return f
