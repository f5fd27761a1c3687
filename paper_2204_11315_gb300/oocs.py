"""ctypes binding of include/oocs.h (argument marshalling only).

Every function here has the name of the C entry point it wraps and does no
arithmetic of its own: all work runs in liboocs.so's CUDA kernels.  There is no
CPU fallback: if the library is missing, ``lib()`` raises.

PyTorch is used only as plumbing by the ``OutOfCoreStencil`` helper: device
workspace (``torch.empty(..., device='cuda')``), page-locked host stores
(``pin_memory=True``, or views of oocs_host_alloc memory for large stores) and
the three CUDA streams the pipeline runs on.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

OOCS_OK = 0
STATUS_NAMES = {0: "OOCS_OK", 1: "OOCS_ERR_INVALID_ARG", 2: "OOCS_ERR_BUDGET",
                3: "OOCS_ERR_HOST_ALLOC", 4: "OOCS_ERR_CUDA", 5: "OOCS_ERR_TIMEOUT",
                6: "OOCS_ERR_STATE", 7: "OOCS_ERR_UNSUPPORTED", 8: "OOCS_ERR_NONFINITE"}
OOCS_ERR_INVALID_ARG, OOCS_ERR_TIMEOUT, OOCS_ERR_NONFINITE = 1, 5, 8
OOCS_DEVERR_WAIT_TIMEOUT, OOCS_DEVERR_NONFINITE = 1, 2
OOCS_HEAT, OOCS_WAVE, OOCS_WAVE_ADJOINT = 0, 1, 2
OOCS_CODEC_TRANSFORM, OOCS_CODEC_QUANT = 0, 1
OOCS_FIELD_U, OOCS_FIELD_U_PREV, OOCS_FIELD_M = 0, 1, 2
OOCS_FIELD_LAM, OOCS_FIELD_LAM_PREV, OOCS_FIELD_FWD, OOCS_FIELD_GRAD = 0, 1, 3, 4
BOUND_FIELDS = {OOCS_HEAT: 1, OOCS_WAVE: 3, OOCS_WAVE_ADJOINT: 4}
OOCS_SWB, OOCS_CLASSIC = 1, 3
MAX_RADIUS = 4


class OOCSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class oocs_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
                ("scheme", ctypes.c_int32), ("radius", ctypes.c_int32),
                ("coef", ctypes.c_float * (MAX_RADIUS + 1)),
                ("device_budget", ctypes.c_uint64), ("rate_bits", ctypes.c_int32),
                ("temporal_depth", ctypes.c_int32), ("slab_planes", ctypes.c_int32),
                ("working_buffers", ctypes.c_int32), ("readonly_resident", ctypes.c_int32),
                ("codec", ctypes.c_int32), ("step_fusion", ctypes.c_int32), ("step_tile", ctypes.c_int32),
                ("codec_fusion", ctypes.c_int32)]


class oocs_plan(ctypes.Structure):
    _fields_ = [("slab_planes", ctypes.c_int32), ("temporal_depth", ctypes.c_int32),
                ("halo_planes", ctypes.c_int32), ("num_slabs", ctypes.c_int32),
                ("window_planes", ctypes.c_int32), ("fields_in", ctypes.c_int32),
                ("fields_out", ctypes.c_int32), ("readonly_resident", ctypes.c_int32),
                ("layer_bytes", ctypes.c_uint64), ("host_store_bytes", ctypes.c_uint64),
                ("workspace_bytes", ctypes.c_uint64), ("workspace_swb_bytes", ctypes.c_uint64),
                ("workspace_classic_bytes", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class oocs_kernel_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("units", ctypes.c_uint64),
                ("device_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class oocs_stats(ctypes.Structure):
    _fields_ = [("h2d_bytes", ctypes.c_uint64), ("d2h_bytes", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64), ("steps_done", ctypes.c_uint64),
                ("passes_done", ctypes.c_uint64), ("slabs_done", ctypes.c_uint64),
                ("workspace_bytes", ctypes.c_uint64), ("last_step_ms", ctypes.c_double),
                ("load", oocs_kernel_stats), ("step", oocs_kernel_stats),
                ("store", oocs_kernel_stats), ("h2d", oocs_kernel_stats), ("d2h", oocs_kernel_stats)]

    def as_dict(self):
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            d[k] = v.as_dict() if isinstance(v, oocs_kernel_stats) else v
        return d


class oocs_timeline_entry(ctypes.Structure):
    _fields_ = [("cls", ctypes.c_int32), ("stream", ctypes.c_int32), ("visit", ctypes.c_int64),
                ("start_ms", ctypes.c_double), ("end_ms", ctypes.c_double)]


class oocs_trace_access(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("index", ctypes.c_int32), ("lo", ctypes.c_int64),
                ("hi", ctypes.c_int64), ("write", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class oocs_trace_op(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("stream", ctypes.c_int32), ("event", ctypes.c_int32),
                ("naccess", ctypes.c_int32), ("visit", ctypes.c_int64),
                ("access", oocs_trace_access * 4)]


OOCS_OP_NAMES = {1: "WAIT", 2: "RECORD", 3: "H2D", 4: "D2H", 5: "LOAD", 6: "STEP", 7: "STORE"}
OOCS_RES_NAMES = {1: "WORK", 2: "IN_SLOT", 3: "OUT_SLOT", 4: "HOST"}


_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64

# name -> (restype, argtypes); the C-ABI of include/oocs.h
SIGNATURES = {
    "oocs_version": (ctypes.c_char_p, []),
    "oocs_query": (_i32, [ctypes.POINTER(oocs_desc), ctypes.POINTER(oocs_plan)]),
    "oocs_create": (_i32, [ctypes.POINTER(oocs_desc), _vp, _u64, ctypes.POINTER(_vp),
                           ctypes.POINTER(_vp)]),
    "oocs_bind_field": (_i32, [_vp, _i32, _vp, _u64]),
    "oocs_set_source": (_i32, [_vp, _i64, _i64, _i64, _vp, _i32]),
    "oocs_compress": (_i32, [_vp, _i32, _vp]),
    "oocs_decompress": (_i32, [_vp, _i32, _vp]),
    "oocs_set_time": (_i32, [_vp, _i64]),
    "oocs_step": (_i32, [_vp, _i32]),
    "oocs_synchronize": (_i32, [_vp, _u64]),
    "oocs_get_stats": (_i32, [_vp, ctypes.POINTER(oocs_stats)]),
    "oocs_set_profiling": (_i32, [_vp, _i32]),
    "oocs_last_error": (ctypes.c_char_p, [_vp]),
    "oocs_destroy": (_i32, [_vp]),
    "oocs_incore_run": (_i32, [ctypes.POINTER(oocs_desc), _vp, _vp, _vp, _vp, _i32, _i64, _vp, _vp,
                               _i32, _vp]),
    "oocs_incore_run_noalloc": (_i32, [ctypes.POINTER(oocs_desc), _vp, _vp, _vp, _i32, _i64, _vp,
                                       _vp, _i32, _vp]),
    "oocs_trace_schedule": (_i32, [ctypes.POINTER(oocs_desc), ctypes.POINTER(_i32), _i32,
                                   ctypes.POINTER(oocs_trace_op), _i64, ctypes.POINTER(_i64)]),
    "oocs_adjoint_step": (_i32, [ctypes.POINTER(oocs_desc), _vp, _vp, _vp, _vp, _vp, _vp, _i64, _vp]),
    "oocs_gradient_accumulate": (_i32, [ctypes.POINTER(oocs_desc), _vp, _vp, _vp, ctypes.c_float, _vp,
                                        _vp]),
    "oocs_receiver_residual": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp]),
    "oocs_model_from_velocity": (_i32, [_vp, _vp, _i64, ctypes.c_float, _vp]),
    "oocs_velocity_gradient": (_i32, [_vp, _vp, _vp, _i64, ctypes.c_float, _vp]),
    "oocs_misfit_workspace_bytes": (_i64, [ctypes.POINTER(oocs_desc), _i32, _i32, _i32]),
    "oocs_misfit_forward": (_i32, [ctypes.POINTER(oocs_desc), _vp, _vp, _vp, _i32, _i64, _vp, _i32, _i32,
                                   _i32, _vp, _i64, _vp, _vp, _vp]),
    "oocs_misfit_backward": (_i32, [ctypes.POINTER(oocs_desc), _vp, _vp, _vp, _i32, _i64, _vp, _i32, _i32,
                                    _i32, _vp, _i64, _vp, _vp]),
    "oocs_batch_query": (_i32, [ctypes.POINTER(oocs_desc), _i32, ctypes.POINTER(_u64)]),
    "oocs_batch_create": (_i32, [ctypes.POINTER(oocs_desc), _i32, _vp, _u64, ctypes.POINTER(_vp),
                                 ctypes.POINTER(_vp)]),
    "oocs_batch_context": (_i32, [_vp, _i32, ctypes.POINTER(_vp)]),
    "oocs_batch_step": (_i32, [_vp, _i32]),
    "oocs_batch_capture": (_i32, [_vp, _i32]),
    "oocs_batch_launch": (_i32, [_vp]),
    "oocs_batch_synchronize": (_i32, [_vp, _u64]),
    "oocs_batch_destroy": (_i32, [_vp]),
    "oocs_batch_trace_schedule": (_i32, [ctypes.POINTER(oocs_desc), _i32, ctypes.POINTER(_i32), _i32,
                                         ctypes.POINTER(oocs_trace_op), _i64, ctypes.POINTER(_i64)]),
    "oocs_set_receiver": (_i32, [_vp, _i64, _vp, _i64]),
    "oocs_set_state_record": (_i32, [_vp, ctypes.POINTER(_vp), _i64, _i64]),
    "oocs_selftest_stuck_wait": (_i32, [_vp]),
    "oocs_device_errors": (_i32, [ctypes.POINTER(ctypes.c_uint32), _i32]),
    "oocs_set_fault_injection": (_i32, [_vp, _i64]),
    "oocs_get_timeline": (_i32, [_vp, ctypes.POINTER(oocs_timeline_entry), _i64, ctypes.POINTER(_i64)]),
    "oocs_compress_device": (_i32, [_vp, _i32, _vp, _i64, _i64]),
    "oocs_decompress_device": (_i32, [_vp, _i32, _vp, _i64, _i64]),
    "oocs_host_alloc": (_i32, [_u64, ctypes.POINTER(_vp)]),
    "oocs_host_free": (_i32, [_vp]),
    "oocs_encode_device": (_i32, [_vp, _i64, _i64, _i64, _i32, _i32, _vp, _vp]),
    "oocs_decode_device": (_i32, [_vp, _i64, _i64, _i64, _i32, _i32, _vp, _vp]),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load liboocs.so (building it in-tree with nvcc if absent).  Raises if unavailable."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path) or not _build.up_to_date():
                if not build_if_missing:
                    raise RuntimeError(f"CUDA library {path} is not built")
                _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int, ctx=None):
    if status != OOCS_OK:
        msg = lib().oocs_last_error(ctx)
        raise OOCSError(status, msg.decode() if msg else "")


def make_desc(nx, ny, nz, scheme, coef, device_budget, rate_bits=0, temporal_depth=0,
              slab_planes=0, working_buffers=OOCS_SWB, radius=None, readonly_resident=0,
              codec=0, step_fusion=0, step_tile=0, codec_fusion=0) -> oocs_desc:
    coef = [float(c) for c in coef]
    d = oocs_desc()
    d.nx, d.ny, d.nz = int(nx), int(ny), int(nz)
    d.scheme = int(scheme)
    d.radius = int(radius if radius is not None else len(coef) - 1)
    for i, c in enumerate(coef):
        d.coef[i] = c
    d.device_budget = int(device_budget)
    d.rate_bits = int(rate_bits)
    d.temporal_depth = int(temporal_depth)
    d.slab_planes = int(slab_planes)
    d.working_buffers = int(working_buffers)
    d.readonly_resident = int(readonly_resident)
    d.codec = int(codec)
    d.step_fusion = int(step_fusion)
    d.step_tile = int(step_tile)
    d.codec_fusion = int(codec_fusion)
    return d


# ---------------------------------------------------------------- C ABI --

def oocs_version() -> str:
    return lib().oocs_version().decode()


def oocs_query(desc: oocs_desc) -> oocs_plan:
    p = oocs_plan()
    _check(lib().oocs_query(ctypes.byref(desc), ctypes.byref(p)))
    return p


def oocs_create(desc: oocs_desc, workspace_ptr: int, workspace_bytes: int, streams) -> int:
    arr = (_vp * 3)(*[int(s) for s in streams])
    out = _vp()
    _check(lib().oocs_create(ctypes.byref(desc), _vp(workspace_ptr), workspace_bytes, arr,
                             ctypes.byref(out)))
    return out.value


def oocs_bind_field(ctx: int, field: int, host_ptr: int, nbytes: int):
    _check(lib().oocs_bind_field(ctx, field, _vp(host_ptr), nbytes), ctx)


def oocs_set_source(ctx: int, x: int, y: int, z: int, w: np.ndarray):
    w = np.ascontiguousarray(w, dtype=np.float32)
    _check(lib().oocs_set_source(ctx, x, y, z, w.ctypes.data_as(_vp), int(w.size)), ctx)


def oocs_compress(ctx: int, field: int, src_ptr: int):
    _check(lib().oocs_compress(ctx, field, _vp(src_ptr)), ctx)


def oocs_decompress(ctx: int, field: int, dst_ptr: int):
    _check(lib().oocs_decompress(ctx, field, _vp(dst_ptr)), ctx)


def oocs_set_time(ctx: int, t: int):
    _check(lib().oocs_set_time(ctx, int(t)), ctx)


def oocs_step(ctx: int, nsteps: int):
    _check(lib().oocs_step(ctx, int(nsteps)), ctx)


def oocs_synchronize(ctx: int, timeout_ns: int = 0):
    _check(lib().oocs_synchronize(ctx, int(timeout_ns)), ctx)


def oocs_get_stats(ctx: int) -> oocs_stats:
    s = oocs_stats()
    _check(lib().oocs_get_stats(ctx, ctypes.byref(s)), ctx)
    return s


OOCS_PROF_LOAD, OOCS_PROF_STEP, OOCS_PROF_STORE, OOCS_PROF_H2D, OOCS_PROF_D2H = 1, 2, 4, 8, 16


def oocs_set_profiling(ctx: int, classes: int):
    """classes: bit mask of OOCS_PROF_LOAD / _STEP / _STORE / _H2D / _D2H (0 = off)."""
    _check(lib().oocs_set_profiling(ctx, int(classes)), ctx)


def oocs_last_error(ctx=None) -> str:
    return lib().oocs_last_error(ctx).decode()


def oocs_destroy(ctx: int):
    _check(lib().oocs_destroy(ctx))


def oocs_incore_run(desc, u_ptr, up_ptr, m_ptr, scratch_ptr, nsteps, t0=0, src=None, w=None,
                    stream=0):
    srcarr = (_i64 * 3)(*src) if src is not None else None
    wv = np.ascontiguousarray(w if w is not None else np.zeros(0), dtype=np.float32)
    _check(lib().oocs_incore_run(ctypes.byref(desc), _vp(u_ptr), _vp(up_ptr), _vp(m_ptr),
                                 _vp(scratch_ptr), int(nsteps), int(t0),
                                 ctypes.cast(srcarr, _vp) if srcarr is not None else None,
                                 wv.ctypes.data_as(_vp), int(wv.size), _vp(stream)))


def oocs_incore_run_noalloc(desc, u_ptr, up_ptr, m_ptr, nsteps, t0=0, src=None, w=None, stream=0):
    """oocs_incore_run without a scratch argument (library-owned device scratch)."""
    srcarr = (_i64 * 3)(*src) if src is not None else None
    wv = np.ascontiguousarray(w if w is not None else np.zeros(0), dtype=np.float32)
    _check(lib().oocs_incore_run_noalloc(ctypes.byref(desc), _vp(u_ptr), _vp(up_ptr), _vp(m_ptr),
                                         int(nsteps), int(t0),
                                         ctypes.cast(srcarr, _vp) if srcarr is not None else None,
                                         wv.ctypes.data_as(_vp), int(wv.size), _vp(stream)))


def oocs_trace_schedule(desc, nsteps_calls):
    """Operations oocs_step(n) would enqueue for each n in nsteps_calls, as dicts:
    {op, stream, event, visit, access: [(kind, index, lo, hi, write), ...]}."""
    calls = (_i32 * len(nsteps_calls))(*[int(n) for n in nsteps_calls])
    count = _i64(0)
    lib().oocs_trace_schedule(ctypes.byref(desc), calls, len(nsteps_calls), None, 0, ctypes.byref(count))
    buf = (oocs_trace_op * max(count.value, 1))()
    _check(lib().oocs_trace_schedule(ctypes.byref(desc), calls, len(nsteps_calls), buf, count.value,
                                     ctypes.byref(count)))
    out = []
    for i in range(count.value):
        o = buf[i]
        out.append({"op": OOCS_OP_NAMES[o.op], "stream": o.stream, "event": o.event,
                    "visit": o.visit,
                    "access": [(OOCS_RES_NAMES[a.kind], a.index, a.lo, a.hi, bool(a.write))
                               for a in o.access[:o.naccess]]})
    return out


def _trace_ops(buf, n):
    out = []
    for i in range(n):
        o = buf[i]
        out.append({"op": OOCS_OP_NAMES[o.op], "stream": o.stream, "event": o.event,
                    "visit": o.visit,
                    "access": [(OOCS_RES_NAMES[a.kind], a.index, a.lo, a.hi, bool(a.write))
                               for a in o.access[:o.naccess]]})
    return out


def _desc_array(descs):
    arr = (oocs_desc * len(descs))()
    for i, d in enumerate(descs):
        arr[i] = d
    return arr


def oocs_batch_trace_schedule(descs, nsteps_calls):
    """oocs_trace_schedule for successive oocs_batch_step calls of a batch."""
    arr = _desc_array(descs)
    calls = (_i32 * len(nsteps_calls))(*[int(n) for n in nsteps_calls])
    count = _i64(0)
    lib().oocs_batch_trace_schedule(arr, len(descs), calls, len(nsteps_calls), None, 0, ctypes.byref(count))
    buf = (oocs_trace_op * max(count.value, 1))()
    _check(lib().oocs_batch_trace_schedule(arr, len(descs), calls, len(nsteps_calls), buf, count.value,
                                           ctypes.byref(count)))
    return _trace_ops(buf, count.value)


def oocs_batch_query(descs) -> int:
    n = _u64(0)
    _check(lib().oocs_batch_query(_desc_array(descs), len(descs), ctypes.byref(n)))
    return n.value


def oocs_adjoint_step(desc, lam_ptr, lam_prev_ptr, mu_ptr, mu_out_ptr, m_ptr, res_ptr=0, zr=-1,
                      stream=0):
    _check(lib().oocs_adjoint_step(ctypes.byref(desc), _vp(lam_ptr), _vp(lam_prev_ptr), _vp(mu_ptr),
                                   _vp(mu_out_ptr), _vp(m_ptr), _vp(res_ptr) if res_ptr else None,
                                   int(zr), _vp(stream)))


def oocs_gradient_accumulate(desc, grad_ptr, lam_ptr, u_ptr, w=0.0, src=None, stream=0):
    srcarr = (_i64 * 3)(*src) if src is not None else None
    _check(lib().oocs_gradient_accumulate(ctypes.byref(desc), _vp(grad_ptr), _vp(lam_ptr), _vp(u_ptr),
                                          float(w),
                                          ctypes.cast(srcarr, _vp) if srcarr is not None else None,
                                          _vp(stream)))


def oocs_receiver_residual(u_plane_ptr, d_plane_ptr, n, res_ptr, misfit_ptr=0, stream=0):
    _check(lib().oocs_receiver_residual(_vp(u_plane_ptr), _vp(d_plane_ptr), int(n), _vp(res_ptr),
                                        _vp(misfit_ptr) if misfit_ptr else None, _vp(stream)))


def oocs_model_from_velocity(v_ptr, m_ptr, n, dt_over_dx, stream=0):
    _check(lib().oocs_model_from_velocity(_vp(v_ptr), _vp(m_ptr), int(n), float(dt_over_dx), _vp(stream)))


def oocs_velocity_gradient(gm_ptr, v_ptr, gv_ptr, n, dt_over_dx, stream=0):
    _check(lib().oocs_velocity_gradient(_vp(gm_ptr), _vp(v_ptr), _vp(gv_ptr), int(n), float(dt_over_dx),
                                        _vp(stream)))


def oocs_misfit_workspace_bytes(desc, nsteps, checkpoint_every, rate_bits):
    n = lib().oocs_misfit_workspace_bytes(ctypes.byref(desc), int(nsteps), int(checkpoint_every),
                                          int(rate_bits))
    if n < 0:
        raise OOCSError(1, "bad misfit workspace arguments")
    return n


def _src_w(src, w):
    srcarr = (_i64 * 3)(*[int(v) for v in src])
    wv = np.ascontiguousarray(w if w is not None else np.zeros(0), dtype=np.float32)
    return srcarr, wv


def oocs_misfit_forward(desc, m_ptr, src, w, zr, d_obs_ptr, nsteps, checkpoint_every, rate_bits, ws_ptr,
                        ws_bytes, res_ptr, misfit_ptr, stream=0):
    srcarr, wv = _src_w(src, w)
    _check(lib().oocs_misfit_forward(ctypes.byref(desc), _vp(m_ptr), ctypes.cast(srcarr, _vp),
                                     wv.ctypes.data_as(_vp), int(wv.size), int(zr), _vp(d_obs_ptr),
                                     int(nsteps), int(checkpoint_every), int(rate_bits), _vp(ws_ptr),
                                     int(ws_bytes), _vp(res_ptr), _vp(misfit_ptr), _vp(stream)))


def oocs_misfit_backward(desc, m_ptr, src, w, zr, res_ptr, nsteps, checkpoint_every, rate_bits, ws_ptr,
                         ws_bytes, grad_ptr, stream=0):
    srcarr, wv = _src_w(src, w)
    _check(lib().oocs_misfit_backward(ctypes.byref(desc), _vp(m_ptr), ctypes.cast(srcarr, _vp),
                                      wv.ctypes.data_as(_vp), int(wv.size), int(zr), _vp(res_ptr),
                                      int(nsteps), int(checkpoint_every), int(rate_bits), _vp(ws_ptr),
                                      int(ws_bytes), _vp(grad_ptr), _vp(stream)))


def oocs_set_receiver(ctx, zr, planes_ptr, nplanes):
    _check(lib().oocs_set_receiver(_vp(ctx), int(zr), _vp(planes_ptr) if planes_ptr else None, int(nplanes)), ctx)


def oocs_selftest_stuck_wait(ctx):
    _check(lib().oocs_selftest_stuck_wait(_vp(ctx)), ctx)


TIMELINE_CLASSES = ("load", "step", "store", "h2d", "d2h")


def oocs_get_timeline(ctx):
    """Profiled items of the last collection as dicts {cls, stream, visit, start_ms, end_ms}."""
    n = _i64()
    _check(lib().oocs_get_timeline(_vp(ctx), None, 0, ctypes.byref(n)), ctx)
    arr = (oocs_timeline_entry * max(n.value, 1))()
    _check(lib().oocs_get_timeline(_vp(ctx), arr, n.value, ctypes.byref(n)), ctx)
    return [{"cls": TIMELINE_CLASSES[e.cls], "stream": e.stream, "visit": e.visit, "start_ms": e.start_ms,
             "end_ms": e.end_ms} for e in arr[:n.value]]


def oocs_set_fault_injection(ctx, nth_call):
    _check(lib().oocs_set_fault_injection(_vp(ctx), int(nth_call)), ctx)


def oocs_device_errors(clear=True) -> int:
    """OOCS_DEVERR_* flags of the current device's error word (synchronises the device)."""
    f = ctypes.c_uint32()
    _check(lib().oocs_device_errors(ctypes.byref(f), 1 if clear else 0))
    return int(f.value)


def oocs_set_state_record(ctx, store_ptrs, t0=0):
    """store_ptrs[i]: host address receiving the compressed state u^(t0 + i), or 0 to skip it."""
    n = len(store_ptrs)
    arr = (_vp * max(n, 1))(*[p or None for p in store_ptrs])
    _check(lib().oocs_set_state_record(_vp(ctx), arr if n else None, int(t0), n), ctx)


def oocs_compress_device(ctx, field, src_ptr, z0, nplanes):
    _check(lib().oocs_compress_device(_vp(ctx), int(field), _vp(src_ptr), int(z0), int(nplanes)), ctx)


def oocs_decompress_device(ctx, field, dst_ptr, z0, nplanes):
    _check(lib().oocs_decompress_device(_vp(ctx), int(field), _vp(dst_ptr), int(z0), int(nplanes)), ctx)


class HostBuffer:
    """Page-locked host memory of an exact size (oocs_host_alloc), viewable as
    a uint8 torch tensor; freed by close() or garbage collection."""

    def __init__(self, nbytes: int):
        p = _vp()
        _check(lib().oocs_host_alloc(int(nbytes), ctypes.byref(p)))
        self.ptr, self.nbytes = p.value, int(nbytes)

    def tensor(self):
        """A uint8 tensor over the buffer; the tensor (and its views) keep the
        buffer alive until close() is called explicitly."""
        import torch
        carr = (ctypes.c_uint8 * self.nbytes).from_address(self.ptr)
        carr._owner = self
        return torch.from_numpy(np.ctypeslib.as_array(carr))

    def close(self):
        if self.ptr:
            lib().oocs_host_free(_vp(self.ptr))
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pinned_bytes(nbytes: int):
    """A zero-filled uint8 tensor of nbytes in page-locked host memory from
    oocs_host_alloc, freed when the tensor and all of its views are gone.
    Each call maps and registers new memory (milliseconds per gigabyte), so it
    suits long-lived buffers such as large host stores."""
    return HostBuffer(int(nbytes)).tensor()


def oocs_encode_device(field_ptr, nx, ny, nz, rate, blocks_ptr, stream=0, codec=0):
    _check(lib().oocs_encode_device(_vp(field_ptr), nx, ny, nz, rate, codec, _vp(blocks_ptr), _vp(stream)))


def oocs_decode_device(blocks_ptr, nx, ny, nz, rate, field_ptr, stream=0, codec=0):
    _check(lib().oocs_decode_device(_vp(blocks_ptr), nx, ny, nz, rate, codec, _vp(field_ptr), _vp(stream)))


# ------------------------------------------------- torch-plumbed helper --

class OutOfCoreStencil:
    """A context plus the memory it needs, allocated through PyTorch.

    Device workspace: one ``torch.uint8`` CUDA tensor of plan.workspace_bytes.
    Host stores: one pinned ``torch.uint8`` tensor per streamed field (PyTorch's
    caching host allocator), or the caller's (``stores=``): for stores of tens
    of gigabytes, tensors over oocs_host_alloc memory (``pinned_bytes``,
    ``HostBuffer``), which keeps its copy speed under sustained traffic.
    Streams: three ``torch.cuda.Stream`` objects.
    """

    def __init__(self, desc: oocs_desc, device: int = 0, stores=None):
        """stores: optional pinned uint8 tensors (one per field, each at least
        plan.host_store_bytes) to bind instead of allocating new ones."""
        import torch
        self.torch = torch
        self.desc = desc
        self.plan = oocs_query(desc)
        self.device = torch.device("cuda", device)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(self.plan.workspace_bytes + 256, dtype=torch.uint8,
                                         device=self.device)
            base = self.workspace.data_ptr()
            self._ws_ptr = (base + 255) // 256 * 256
            self.streams = [torch.cuda.Stream(device=self.device) for _ in range(3)]
            self.ctx = oocs_create(desc, self._ws_ptr, self.plan.workspace_bytes,
                                   [s.cuda_stream for s in self.streams])
        nfields = BOUND_FIELDS[desc.scheme]
        self.stores = []
        for f in range(nfields):
            if stores is not None:
                st = stores[f][:self.plan.host_store_bytes]
            else:
                st = torch.zeros(self.plan.host_store_bytes, dtype=torch.uint8, pin_memory=True)
            oocs_bind_field(self.ctx, f, st.data_ptr(), st.numel())
            self.stores.append(st)
        self._keep = []

    @property
    def shape(self):
        return (self.desc.nz, self.desc.ny, self.desc.nx)

    def pinned_field(self):
        return self.torch.empty(self.shape, dtype=self.torch.float32, pin_memory=True)

    def set_source(self, x, y, z, w):
        oocs_set_source(self.ctx, x, y, z, w)

    def compress(self, field: int, src):
        """src: pinned FP32 torch tensor (or numpy array, copied into pinned memory)."""
        t = src
        if not hasattr(t, "data_ptr"):
            t = self.pinned_field()
            t.numpy()[...] = np.asarray(src, dtype=np.float32)
        assert t.dtype == self.torch.float32 and t.is_contiguous() and t.numel() == np.prod(self.shape)
        self._keep.append(t)
        oocs_compress(self.ctx, field, t.data_ptr())

    def decompress(self, field: int, dst=None):
        if dst is None:
            dst = self.pinned_field()
        oocs_decompress(self.ctx, field, dst.data_ptr())
        self._keep.append(dst)
        return dst

    def step(self, nsteps: int):
        oocs_step(self.ctx, nsteps)
        if self.desc.scheme == OOCS_WAVE_ADJOINT and nsteps % 2:  # the library swapped the two stores
            self.stores[OOCS_FIELD_LAM], self.stores[OOCS_FIELD_LAM_PREV] = \
                self.stores[OOCS_FIELD_LAM_PREV], self.stores[OOCS_FIELD_LAM]

    def set_time(self, t: int):
        oocs_set_time(self.ctx, t)

    def bind(self, field: int, store):
        """Bind a pinned uint8 tensor (at least plan.host_store_bytes) as the store of `field`."""
        oocs_bind_field(self.ctx, field, store.data_ptr(), store.numel())
        self.stores[field] = store

    def snapshot_stores(self):
        """Pinned host copies of the current stores (call after synchronize)."""
        return [s.clone().pin_memory() for s in self.stores]

    def restore_stores(self, snap, t: int = 0):
        """Put the stores back to a snapshot and the time index to t (after synchronize)."""
        for s, c in zip(self.stores, snap):
            s.copy_(c)
        self.set_time(t)

    def synchronize(self, timeout_s: float = 0.0):
        oocs_synchronize(self.ctx, int(timeout_s * 1e9))
        self._keep.clear()

    def set_profiling(self, classes: int = 7):
        oocs_set_profiling(self.ctx, classes)

    def stats(self) -> dict:
        return oocs_get_stats(self.ctx).as_dict()

    def close(self):
        if getattr(self, "ctx", None):
            oocs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchProblem(OutOfCoreStencil):
    """One problem of an OutOfCoreBatch: a context owned by the batch, with its
    own pinned host stores (the OutOfCoreStencil methods apply to it)."""

    def __init__(self, batch, i: int, desc: oocs_desc):
        import torch
        self.torch = torch
        self.desc = desc
        self.plan = oocs_query(desc)
        self.device = batch.device
        self.streams = batch.streams
        c = _vp()
        _check(lib().oocs_batch_context(_vp(batch.handle), int(i), ctypes.byref(c)))
        self.ctx = c.value
        nfields = BOUND_FIELDS[desc.scheme]
        self.stores = []
        for f in range(nfields):
            st = torch.zeros(self.plan.host_store_bytes, dtype=torch.uint8, pin_memory=True)
            oocs_bind_field(self.ctx, f, st.data_ptr(), st.numel())
            self.stores.append(st)
        self._keep = []

    def close(self):
        self.ctx = None  # owned by the batch


class OutOfCoreBatch:
    """A batch (oocs_batch_*) plus its workspace and streams, allocated through
    PyTorch; problems[i] are BatchProblem objects."""

    def __init__(self, descs, device: int = 0):
        import torch
        self.torch = torch
        self.descs = list(descs)
        self.device = torch.device("cuda", device)
        self.workspace_bytes = oocs_batch_query(self.descs)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device=self.device)
            ws = (self.workspace.data_ptr() + 255) // 256 * 256
            self.streams = [torch.cuda.Stream(device=self.device) for _ in range(3)]
            arr = (_vp * 3)(*[s.cuda_stream for s in self.streams])
            out = _vp()
            _check(lib().oocs_batch_create(_desc_array(self.descs), len(self.descs), _vp(ws),
                                           self.workspace_bytes, arr, ctypes.byref(out)))
            self.handle = out.value
        self.problems = [BatchProblem(self, i, d) for i, d in enumerate(self.descs)]

    def step(self, nsteps: int):
        _check(lib().oocs_batch_step(_vp(self.handle), int(nsteps)))

    def capture(self, nsteps: int):
        _check(lib().oocs_batch_capture(_vp(self.handle), int(nsteps)))

    def launch(self):
        _check(lib().oocs_batch_launch(_vp(self.handle)))

    def synchronize(self, timeout_s: float = 0.0):
        _check(lib().oocs_batch_synchronize(_vp(self.handle), int(timeout_s * 1e9)))
        for p in self.problems:
            p._keep.clear()

    def close(self):
        if getattr(self, "handle", None):
            lib().oocs_batch_destroy(_vp(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
