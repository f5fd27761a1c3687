"""oocs_host_alloc / oocs_host_free: zero-filled page-locked host memory of an
exact size, usable by the copy engines, tied to the lifetime of its tensors,
and a free that rejects pointers it did not hand out."""
import gc

import numpy as np
import pytest

from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2204_11315_gb300 as P
    P.lib()
    return P


def test_alloc_is_zero_filled_and_copies_both_ways(P):
    torch = torch_cuda()
    n = (3 << 20) + 40  # not a multiple of any page size
    h = P.HostBuffer(n)
    t = h.tensor()
    assert t.numel() == n and int(t.sum()) == 0
    src = torch.arange(n, dtype=torch.int64).remainder(251).to(torch.uint8)
    d = src.cuda()
    t.copy_(d, non_blocking=True)
    torch.cuda.synchronize()
    assert torch.equal(t, src)
    d2 = torch.empty(n, dtype=torch.uint8, device="cuda")
    d2.copy_(t, non_blocking=True)
    torch.cuda.synchronize()
    assert torch.equal(d2.cpu(), src)
    h.close()


def test_tensor_keeps_its_buffer_alive(P):
    torch_cuda()
    t = P.pinned_bytes(1 << 20)
    v = t[1000:2000]
    del t
    gc.collect()
    v.fill_(7)  # still mapped through the view
    assert int(v.sum()) == 7 * 1000
    f = P.pinned_bytes(4 * 24).view(torch_cuda().float32).reshape(2, 3, 4)
    f[1, 2, 3] = 1.5
    assert float(f.sum()) == 1.5


def test_free_rejects_foreign_and_repeated_pointers(P):
    import ctypes
    torch_cuda()
    buf = (ctypes.c_uint8 * 64)()
    assert P.lib().oocs_host_free(ctypes.c_void_p(ctypes.addressof(buf))) == P.OOCS_ERR_INVALID_ARG
    h = P.HostBuffer(4096)
    p = h.ptr
    h.close()
    st = P.lib().oocs_host_free(ctypes.c_void_p(p))
    assert st == P.OOCS_ERR_INVALID_ARG  # already freed
    assert P.lib().oocs_host_free(None) == 0
