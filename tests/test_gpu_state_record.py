"""The state record (oocs_set_state_record), on the GPU.

A recorded state must hold exactly the bytes the field's own store held when
that state was written: a run of several sweeps with the record on is compared
with the same sweeps made as separate calls, the stores snapshotted after
each.  Wave at temporal depth 2 records every state (the two outputs of each
visit); heat at depth 1 likewise.  Indices outside the record, null entries
and n = 0 are skipped; a batch member with a record cannot be captured.
"""
import numpy as np
import pytest

import synthetic
from gpu_util import heat_desc, torch_cuda, wave_desc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2204_11315_gb300 as P
    P.lib()
    return P


def _wave_inputs(shape):
    m = synthetic.wave_model(shape)
    z = np.zeros(shape, np.float32)
    src = (synthetic.centre(shape)[::-1], synthetic.ricker(40))
    return {0: z, 1: z, 2: m}, src


def _load(P, desc, fields, src):
    st = P.OutOfCoreStencil(desc)
    for f, a in fields.items():
        st.compress(f, a)
    if src is not None:
        (x, y, z), w = src
        st.set_source(x, y, z, w)
    st.synchronize(60.0)
    return st


@pytest.mark.parametrize("rate,T", [(16, 32), (0, 24), (12, 96)])
def test_wave_record_equals_store_snapshots(P, rate, T):
    torch = torch_cuda()
    shape = (96, 40, 48)
    fields, src = _wave_inputs(shape)
    desc = wave_desc(P, shape, rate=rate, k=2, T=T, ro=1)
    n = 11  # sweeps 0->2->...->10->11: states 1 .. 11 all written
    snaps = {}
    st = _load(P, desc, fields, src)
    try:
        t = 0
        while t < n:
            kk = min(2, n - t)
            st.step(kk)
            st.synchronize(60.0)
            t += kk
            snaps[t] = st.stores[P.OOCS_FIELD_U].clone()
            snaps[t - 1] = st.stores[P.OOCS_FIELD_U_PREV].clone()
    finally:
        st.close()
    nb = snaps[n].numel()
    rec = torch.zeros((n + 2, nb), dtype=torch.uint8, pin_memory=True)
    st = _load(P, desc, fields, src)
    try:
        ptrs = [rec[i].data_ptr() for i in range(n + 2)]
        ptrs[5] = 0  # a null entry is skipped
        P.oocs_set_state_record(st.ctx, ptrs, -1)  # entry i <- u^(i-1)
        before = st.stats()["d2h_bytes"]
        st.step(n)
        st.synchronize(60.0)
        extra = st.stats()["d2h_bytes"] - before
    finally:
        st.close()
    for t in range(1, n + 1):
        if t + 1 == 5:
            assert not rec[5].any()
        else:
            assert torch.equal(rec[t + 1], snaps[t]), t
    assert not rec[0].any() and not rec[1].any()  # u^-1 and u^0 are not written by a sweep
    # the copies count in d2h_bytes: beside the sweeps' own 6 x 2 stores, two
    # states per sweep (u^10 is written by two of them) less the null entry
    assert extra == 12 * nb + 11 * nb


def test_heat_record_and_stop(P):
    torch = torch_cuda()
    u0 = synthetic.uniform_field((64, 36, 40), 3)
    desc = heat_desc(P, u0.shape, rate=16, k=1, T=16)
    n = 6
    snaps = {}
    st = _load(P, desc, {0: u0}, None)
    try:
        for t in range(1, n + 1):
            st.step(1)
            st.synchronize(60.0)
            snaps[t] = st.stores[0].clone()
    finally:
        st.close()
    nb = snaps[n].numel()
    rec = torch.zeros((4, nb), dtype=torch.uint8, pin_memory=True)
    st = _load(P, desc, {0: u0}, None)
    try:
        P.oocs_set_state_record(st.ctx, [rec[i].data_ptr() for i in range(4)], 2)  # u^2 .. u^5
        st.step(4)
        P.oocs_set_state_record(st.ctx, [])  # u^5, u^6 not recorded
        st.step(2)
        st.synchronize(60.0)
    finally:
        st.close()
    for i in range(3):
        assert torch.equal(rec[i], snaps[2 + i]), i
    assert not rec[3].any()


def test_capture_refuses_a_member_with_a_record(P):
    torch = torch_cuda()
    shape = (64, 32, 32)
    u0 = (1e-3 * synthetic.uniform_field(shape, 5)).astype(np.float32)
    fields = {0: u0, 1: u0, 2: synthetic.wave_model(shape)}
    b = P.OutOfCoreBatch([wave_desc(P, shape, rate=16, k=2, T=32, ro=1)])
    try:
        for f, a in fields.items():
            b.problems[0].compress(f, a)
        rec = torch.zeros((2, b.problems[0].plan.host_store_bytes), dtype=torch.uint8, pin_memory=True)
        P.oocs_set_state_record(b.problems[0].ctx, [rec[0].data_ptr(), rec[1].data_ptr()], 1)
        with pytest.raises(P.OOCSError) as e:
            b.capture(2)
        assert e.value.status == 7
        b.step(2)  # a direct step records
        b.synchronize(60.0)
        assert rec[0].any() and rec[1].any()
        P.oocs_set_state_record(b.problems[0].ctx, [])
        b.capture(2)
        b.launch()
        b.synchronize(60.0)
    finally:
        b.close()
