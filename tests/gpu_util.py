"""Helpers for the GPU tests: run the C-ABI path through the ctypes binding."""
import numpy as np

import synthetic


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def heat_desc(P, shape, rate=0, k=1, T=32, wb=1, alpha=0.1, budget=8 << 30, codec=0):
    nz, ny, nx = shape
    return P.make_desc(nx, ny, nz, P.OOCS_HEAT, synthetic.heat_star_coef(alpha), budget,
                       rate_bits=rate, temporal_depth=k, slab_planes=T, working_buffers=wb, codec=codec)


def wave_desc(P, shape, rate=0, k=4, T=64, wb=1, budget=8 << 30, ro=0, codec=0):
    nz, ny, nx = shape
    return P.make_desc(nx, ny, nz, P.OOCS_WAVE, synthetic.wave_star_coef(), budget,
                       rate_bits=rate, temporal_depth=k, slab_planes=T, working_buffers=wb,
                       readonly_resident=ro, codec=codec)


def incore(P, desc, u0, nsteps, up0=None, m=None, src=None, w=None, t0=0):
    """In-core GPU run (oocs_incore_run) on device copies; returns numpy arrays."""
    torch = torch_cuda()
    u = torch.from_numpy(np.ascontiguousarray(u0, np.float32)).cuda()
    scratch = torch.empty_like(u)
    wave = desc.scheme == P.OOCS_WAVE
    up = torch.from_numpy(np.ascontiguousarray(up0, np.float32)).cuda() if wave else None
    mm = torch.from_numpy(np.ascontiguousarray(m, np.float32)).cuda() if wave else None
    s = torch.cuda.current_stream().cuda_stream
    P.oocs_incore_run(desc, u.data_ptr(), up.data_ptr() if wave else 0,
                      mm.data_ptr() if wave else 0, scratch.data_ptr(), nsteps, t0,
                      src, w, s)
    torch.cuda.synchronize()
    if wave:
        return u.cpu().numpy(), up.cpu().numpy()
    return u.cpu().numpy()


def streamed(P, desc, u0, nsteps, up0=None, m=None, src=None, w=None, chunks=None):
    """Out-of-core run through oocs_compress / oocs_step / oocs_decompress.

    chunks: optional list of step counts for several oocs_step calls."""
    st = P.OutOfCoreStencil(desc)
    try:
        wave = desc.scheme == P.OOCS_WAVE
        st.compress(P.OOCS_FIELD_U, u0)
        if wave:
            st.compress(P.OOCS_FIELD_U_PREV, up0)
            st.compress(P.OOCS_FIELD_M, m)
            if src is not None:
                st.set_source(src[0], src[1], src[2], w)
        for n in (chunks or [nsteps]):
            st.step(n)
        st.synchronize(120.0)
        out = st.decompress(P.OOCS_FIELD_U)
        outp = st.decompress(P.OOCS_FIELD_U_PREV) if wave else None
        st.synchronize(120.0)
        stores = [s.numpy().copy() for s in st.stores]
        stats = st.stats()
        res = (out.numpy().copy(), outp.numpy().copy() if wave else None, stores, stats, st.plan)
    finally:
        st.close()
    return res


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def max_abs_rel(a, b):
    """max |a - b| over max |b|: the largest pointwise error against the field's peak."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def assert_parity(got, ref, l2_bar, maxabs_bar, what=""):
    """Relative L2 error within l2_bar and, element by element,
    |got - ref| <= maxabs_bar * max |ref| (the worst point is named on failure)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    e2 = rel_l2(got, ref)
    peak = float(np.max(np.abs(ref)))
    err = np.abs(got - ref)
    worst = np.unravel_index(int(np.argmax(err)), err.shape)
    ok = err <= maxabs_bar * peak
    assert e2 <= l2_bar and bool(np.all(ok)), (
        f"{what}: rel-L2 {e2:.3e} (bar {l2_bar:.1e}); max-abs {err[worst]:.3e} = "
        f"{err[worst] / peak:.3e} of the peak {peak:.3e} at {tuple(int(i) for i in worst)} "
        f"(bar {maxabs_bar:.1e}); {int(np.size(ok) - np.count_nonzero(ok))} points over")


def assert_uncompressed(got, ref, scheme, what=""):
    assert_parity(got, ref, synthetic.TOL_UNCOMPRESSED[scheme], synthetic.TOL_MAXABS_UNCOMPRESSED[scheme], what)


def assert_compressed(got, ref, rate, what=""):
    assert_parity(got, ref, synthetic.TOL_COMPRESSED[rate], synthetic.TOL_MAXABS_COMPRESSED[rate], what)
