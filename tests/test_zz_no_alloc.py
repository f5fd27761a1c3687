"""oocs_incore_run_noalloc: the in-core run for callers that cannot allocate device memory.

Such callers (a plugin inside a host application whose allocator owns the
device memory pool, or a latency-critical loop that cannot afford cudaMalloc's
device synchronisation) pass only inputs and outputs; the scratch field comes
from a library-owned static device array.  Checked through the C ABI against
the existing oocs_incore_run (same FP32 arithmetic: bit-identical, the bar the
other same-arithmetic GPU tests use) on calls made back to back, so a call
that reuses the array's leftover contents would show.  Collected last, so a
failure here stops a -x run only after every other test has run.
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


def _run(P, desc, u0, nsteps, noalloc, up0=None, m=None, src=None, w=None):
    torch = torch_cuda()
    u = torch.from_numpy(np.ascontiguousarray(u0, np.float32)).cuda()
    wave = desc.scheme == P.OOCS_WAVE
    up = torch.from_numpy(np.ascontiguousarray(up0, np.float32)).cuda() if wave else None
    mm = torch.from_numpy(np.ascontiguousarray(m, np.float32)).cuda() if wave else None
    s = torch.cuda.current_stream().cuda_stream
    upp = up.data_ptr() if wave else 0
    mp = mm.data_ptr() if wave else 0
    if noalloc:
        P.oocs_incore_run_noalloc(desc, u.data_ptr(), upp, mp, nsteps, 0, src, w, s)
    else:
        scratch = torch.empty_like(u)
        P.oocs_incore_run(desc, u.data_ptr(), upp, mp, scratch.data_ptr(), nsteps, 0, src, w, s)
    torch.cuda.synchronize()
    return (u.cpu().numpy(), up.cpu().numpy()) if wave else (u.cpu().numpy(),)


def _same(a, b):
    return all(np.array_equal(x.view(np.uint32), y.view(np.uint32)) for x, y in zip(a, b))


def test_noalloc_matches_incore_on_calls_in_a_row(P):
    # call 1: 7-point heat, 128^3 (2 Mi values), 10 steps from the noisy sine field
    u0 = synthetic.heat_initial(128)
    d_heat = heat_desc(P, u0.shape)
    ref1 = _run(P, d_heat, u0, 10, noalloc=False)
    got1 = _run(P, d_heat, u0, 10, noalloc=True)
    assert _same(got1, ref1)

    # call 2, right after: 25-point wave, 96 x 80 x 112 with source, odd step count
    shape = (96, 80, 112)
    m = synthetic.wave_model(shape)
    w = synthetic.ricker(9)
    cz, cy, cx = synthetic.centre(shape)
    z = np.zeros(shape, np.float32)
    d_wave = wave_desc(P, shape)
    ref2 = _run(P, d_wave, z, 9, noalloc=False, up0=z, m=m, src=(cx, cy, cz), w=w)
    got2 = _run(P, d_wave, z, 9, noalloc=True, up0=z, m=m, src=(cx, cy, cz), w=w)
    assert _same(got2, ref2)

    # call 3: heat again on another field, after the array held wave data
    u1 = synthetic.uniform_field((64, 72, 88), 11)
    d_heat2 = heat_desc(P, u1.shape, alpha=0.12)
    ref3 = _run(P, d_heat2, u1, 7, noalloc=False)
    got3 = _run(P, d_heat2, u1, 7, noalloc=True)
    assert _same(got3, ref3)


def test_noalloc_rejects_grids_above_the_maximum(P):
    cap = 8 << 20
    ok = heat_desc(P, (128, 256, 256))           # exactly the maximum
    assert 128 * 256 * 256 == cap
    big = heat_desc(P, (132, 256, 256))
    torch = torch_cuda()
    u = torch.zeros(132 * 256 * 256, device="cuda")
    with pytest.raises(P.OOCSError) as e:
        P.oocs_incore_run_noalloc(big, u.data_ptr(), 0, 0, 1)
    assert e.value.status == 1
    assert "exceeds the no-allocation scratch" in str(e.value)
    # the largest allowed grid still runs
    P.oocs_incore_run_noalloc(ok, u.data_ptr(), 0, 0, 1,
                              stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()


def test_noalloc_and_incore_from_two_host_threads(P):
    """oocs_incore_run and oocs_incore_run_noalloc called at the same time from
    two host threads, each on its own stream: the per-device caches (the step
    kernel's shared-memory opt-in, the scratch address) are taken under their
    locks, only the no-allocation call uses the library's array, and both
    results equal the same runs made one after the other."""
    import threading
    torch = torch_cuda()
    u0 = synthetic.heat_initial(128)
    d_heat = heat_desc(P, u0.shape)
    ref = _run(P, d_heat, u0, 10, noalloc=False)
    shape = (96, 80, 112)
    m = synthetic.wave_model(shape)
    z = np.zeros(shape, np.float32)
    d_wave = wave_desc(P, shape)
    ref_w = _run(P, d_wave, z + 1e-3, 6, noalloc=False, up0=z, m=m)

    results, errors = {}, []

    def worker(name, desc, fields, nsteps, noalloc):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                dev = [torch.from_numpy(np.ascontiguousarray(f, np.float32)).cuda() for f in fields]
                wave = desc.scheme == P.OOCS_WAVE
                ptrs = [dev[0].data_ptr(), dev[1].data_ptr() if wave else 0, dev[2].data_ptr() if wave else 0]
                for _ in range(3):
                    for t, f in zip(dev, fields):
                        t.copy_(torch.from_numpy(np.ascontiguousarray(f, np.float32)))
                    if noalloc:
                        P.oocs_incore_run_noalloc(desc, *ptrs, nsteps, stream=s.cuda_stream)
                    else:
                        scratch = torch.empty_like(dev[0])
                        P.oocs_incore_run(desc, *ptrs, scratch.data_ptr(), nsteps, stream=s.cuda_stream)
                s.synchronize()
                results[name] = tuple(t.cpu().numpy() for t in dev[:2 if wave else 1])
        except Exception as e:  # reported by the main thread
            errors.append(e)

    th = [threading.Thread(target=worker, args=("heat_noalloc", d_heat, [u0], 10, True)),
          threading.Thread(target=worker, args=("wave_incore", d_wave, [z + 1e-3, z, m], 6, False))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    assert _same(results["heat_noalloc"], ref)
    assert _same(results["wave_incore"], ref_w)
