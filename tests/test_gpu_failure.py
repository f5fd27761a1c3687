"""Failure detection on the GPU without a fault: a kernel's bounded wait runs
out (an mbarrier no thread arrives on), the device error word records it, the
context reports it at oocs_synchronize and keeps reporting it, and a new
context on the same GPU then runs a sweep normally."""
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
