"""Failure detection on the GPU without a fault.

- A kernel's bounded wait runs out (an mbarrier no thread arrives on): the
  device error word records it, the context reports it at oocs_synchronize and
  keeps reporting it, and a new context on the same GPU sweeps normally.
- A CUDA call of the scheduler is reported as failed by the host-side
  injection hook: sticky OOCS_ERR_CUDA, and a new context sweeps bit-exactly.
- oocs_synchronize runs out of time on a running sweep: sticky
  OOCS_ERR_TIMEOUT, and the enqueued work still completes.
- The codec meets an Inf and a NaN: OOCS_ERR_NONFINITE, the two blocks stored
  as zeros and every other byte equal to the oracle codec's.
None of these traps, faults or hangs a kernel."""
import numpy as np
import pytest

import synthetic
from gpu_util import heat_desc, incore, streamed, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2204_11315_gb300 as P
    P.lib()
    return P


def test_bounded_wait_reports_and_the_gpu_stays_usable(P):
    torch_cuda()
    u0 = synthetic.heat_initial(64)
    desc = heat_desc(P, u0.shape, rate=0, k=2, T=16)
    st = P.OutOfCoreStencil(desc)
    try:
        st.compress(P.OOCS_FIELD_U, u0)
        st.synchronize(60.0)
        P.oocs_selftest_stuck_wait(st.ctx)
        with pytest.raises(P.OOCSError) as e:
            st.synchronize(30.0)
        assert e.value.status == 4 and "bounded wait ran out" in str(e.value)
        with pytest.raises(P.OOCSError):  # sticky on this context
            st.step(2)
    finally:
        st.close()
    got, _, _, _, _ = streamed(P, desc, u0, 4)
    assert np.array_equal(got, incore(P, desc, u0, 4))


# ---------------------------------------------------------------------------
# Host-side fault injection: a CUDA call of the scheduler reported as failed
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nth", [1, 6, 23, 57])
def test_injected_cuda_failure_is_sticky_and_a_new_context_sweeps_bitexactly(P, nth):
    torch_cuda()
    u0 = synthetic.heat_initial(64)
    desc = heat_desc(P, u0.shape, rate=16, k=2, T=16)
    ref, _, ref_stores, _, _ = streamed(P, desc, u0, 6)
    st = P.OutOfCoreStencil(desc)
    try:
        st.compress(P.OOCS_FIELD_U, u0)
        st.synchronize(60.0)
        P.oocs_set_fault_injection(st.ctx, nth)
        with pytest.raises(P.OOCSError) as e:
            st.step(6)
        assert e.value.status == 4 and "injected failure" in str(e.value)
        for call in (lambda: st.synchronize(60.0), lambda: st.step(2)):  # sticky
            with pytest.raises(P.OOCSError) as e2:
                call()
            assert e2.value.status == 4
    finally:
        st.close()  # waits for whatever was enqueued before the failure
    got, _, stores, _, _ = streamed(P, desc, u0, 6)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    assert np.array_equal(stores[0], ref_stores[0])


# ---------------------------------------------------------------------------
# oocs_synchronize runs out of time while a sweep is still running
# ---------------------------------------------------------------------------

def test_synchronize_timeout_is_sticky_and_the_work_completes(P):
    torch = torch_cuda()
    shape = (512, 512, 512)
    desc = P.make_desc(512, 512, 512, P.OOCS_WAVE, synthetic.wave_star_coef(), 4 << 30, rate_bits=16,
                       temporal_depth=4, slab_planes=64, readonly_resident=1)
    st = P.OutOfCoreStencil(desc)
    try:
        m = synthetic.wave_model(shape)
        z = np.zeros(shape, np.float32)
        st.compress(P.OOCS_FIELD_U, z)
        st.compress(P.OOCS_FIELD_U_PREV, z)
        st.compress(P.OOCS_FIELD_M, m)
        st.synchronize(120.0)
        st.step(100)  # about 0.1 s of work
        with pytest.raises(P.OOCSError) as e:
            st.synchronize(1e-6)  # 1 microsecond
        assert e.value.status == P.OOCS_ERR_TIMEOUT
        with pytest.raises(P.OOCSError) as e2:  # sticky
            st.synchronize(120.0)
        assert e2.value.status == P.OOCS_ERR_TIMEOUT
        for s in st.streams:  # the work itself goes on and completes
            s.synchronize()
        assert st.stats()["passes_done"] == 25
    finally:
        st.close()
    torch.cuda.synchronize()


# ---------------------------------------------------------------------------
# Non-finite input to the codec: reported, the blocks stored as zeros
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("codec", [0, 1])
def test_nonfinite_field_is_reported_and_stored_as_zero_blocks(P, orc, codec):
    torch = torch_cuda()
    u0 = synthetic.heat_initial(64)
    u0[20, 21, 22] = np.inf
    u0[41, 9, 50] = np.nan
    desc = heat_desc(P, u0.shape, rate=16, k=1, T=16, codec=codec)
    st = P.OutOfCoreStencil(desc)
    try:
        st.compress(P.OOCS_FIELD_U, u0)
        with pytest.raises(P.OOCSError) as e:
            st.synchronize(60.0)
        assert e.value.status == P.OOCS_ERR_NONFINITE
        with pytest.raises(P.OOCSError):  # sticky
            st.step(1)
        got = st.stores[0].numpy().view(np.uint32).copy()
    finally:
        st.close()
    enc = orc.encode_field if codec == 0 else orc.bq_encode_field
    ref, bad = enc(u0, 16, with_nonfinite=True)
    assert bad == 2
    assert np.array_equal(got, ref)
    # the two blocks are all-zero words
    words = ref.reshape(-1, 32)
    for (z, y, x) in ((20, 21, 22), (41, 9, 50)):
        b = ((z // 4) * 16 + y // 4) * 16 + x // 4
        assert not words[b].any()
    # the device-level encoder raises the same flag in the device error word
    assert P.oocs_device_errors(clear=True) == 0  # cleared by the context's synchronize
    f = torch.from_numpy(u0).cuda()
    blocks = torch.empty(ref.size, dtype=torch.int32, device="cuda")
    P.oocs_encode_device(f.data_ptr(), 64, 64, 64, 16, blocks.data_ptr(), codec=codec)
    assert P.oocs_device_errors(clear=True) == P.OOCS_DEVERR_NONFINITE
    assert np.array_equal(blocks.cpu().numpy().view(np.uint32), ref)
    assert P.oocs_device_errors(clear=True) == 0
