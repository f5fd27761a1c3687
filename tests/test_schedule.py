"""Hazard check of the slab scheduler on the host (no GPU).

oocs_trace_schedule returns, in enqueue order, the operations oocs_step would
issue on its three streams (Algorithm 1's copies, kernels and event
records/waits; Fig. 8).  From them this test builds the happens-before
relation of CUDA streams and events (stream order; a wait depends on the most
recent record of its event enqueued before it) and checks:

* no race: every pair of operations that touch the same physical buffer (the
  working buffer set, a staging slot) or the same host-store layer, one of them
  writing, is ordered;
* single working buffer (Sec. 5): all kernels of different slab visits are
  ordered, i.e. they never overlap;
* region sharing (Sec. 3.1): the overlap a visit borrows from the previous
  visit's staging slot is exactly what that slot last received;
* the in-place host store: in sweep p+1 every layer read was last written by
  sweep p.

Deleting any one kind of cross-stream wait from a trace must make the check
fail, which shows the check can see the hazards the waits prevent.
"""
import itertools

import pytest

import synthetic

SHARED = {"WORK", "IN_SLOT", "OUT_SLOT"}  # physical buffers: any two accesses overlap


@pytest.fixture(scope="module")
def P():
    import paper_2204_11315_gb300 as P
    P.lib()
    return P


def happens_before(trace):
    """preds[i] = bit set of ops that happen before op i."""
    n = len(trace)
    preds = [0] * n
    last_in_stream = {}
    last_record = {}
    for i, o in enumerate(trace):
        p = 0
        s = o["stream"]
        if s in last_in_stream:
            j = last_in_stream[s]
            p |= preds[j] | (1 << j)
        if o["op"] == "WAIT" and o["event"] in last_record:
            j = last_record[o["event"]]
            p |= preds[j] | (1 << j)
        preds[i] = p
        last_in_stream[s] = i
        if o["op"] == "RECORD":
            last_record[o["event"]] = i
    return preds


def conflicts(a, b):
    for (ka, ia, la, ha, wa) in a["access"]:
        for (kb, ib, lb, hb, wb) in b["access"]:
            if ka != kb or ia != ib or not (wa or wb):
                continue
            if ka in SHARED or (la < hb and lb < ha):
                return True
    return False


def check(trace, swb=True):
    preds = happens_before(trace)
    data_ops = [i for i, o in enumerate(trace) if o["access"]]
    for i, j in itertools.combinations(data_ops, 2):
        if conflicts(trace[i], trace[j]) and not (preds[j] >> i) & 1:
            return f"race between {trace[i]} and {trace[j]}"
    kernels = [i for i in data_ops if trace[i]["op"] in ("LOAD", "STEP", "STORE")]
    if swb:
        for i, j in itertools.combinations(kernels, 2):
            if trace[i]["visit"] != trace[j]["visit"] and not (preds[j] >> i) & 1:
                return f"kernels of visits {trace[i]['visit']} and {trace[j]['visit']} may overlap"
    # borrowed overlap: each staging-slot read lies inside the slot's last write
    last_slot_write = {}
    for o in trace:
        for (k, idx, lo, hi, w) in o["access"]:
            if k == "IN_SLOT" and not w:
                wl = last_slot_write.get(idx)
                if wl is None or not (wl[0] <= lo and hi <= wl[1]):
                    return f"visit {o['visit']} reads slot {idx} layers [{lo},{hi}) not staged there"
        for (k, idx, lo, hi, w) in o["access"]:
            if k == "IN_SLOT" and w:
                last_slot_write[idx] = (lo, hi)
    return None


def host_dataflow(trace, nlayers, nfields_out):
    """Sweep index of the last writer of each host layer read by each H2D."""
    writer = {}
    reads = []
    sweep_of_visit = {}
    for o in trace:
        if o["op"] == "H2D":
            for (k, f, lo, hi, w) in o["access"]:
                if k == "HOST" and f < nfields_out:
                    reads.append((o["visit"], [writer.get((f, l)) for l in range(lo, hi)]))
        if o["op"] == "D2H":
            for (k, f, lo, hi, w) in o["access"]:
                if k == "HOST" and w:
                    for l in range(lo, hi):
                        writer[(f, l)] = o["visit"]
    return reads


CASES = [
    # (scheme, shape, rate, k, T, wb, calls)
    ("heat", (128, 128, 128), 16, 1, 32, 1, [10]),
    ("heat", (128, 128, 128), 0, 2, 32, 3, [10]),
    ("heat", (120, 52, 44), 16, 3, 32, 1, [3, 4]),
    ("heat", (64, 36, 100), 8, 2, 8, 1, [7]),
    ("heat", (40, 16, 24), 16, 4, 64, 1, [9]),
    ("wave", (128, 72, 40), 16, 4, 32, 1, [10]),
    ("wave", (96, 48, 64), 12, 3, 24, 3, [10]),
    ("wave", (512, 512, 512), 16, 4, 64, 1, [12]),
    ("wave", (96, 40, 48), 0, 4, 32, 1, [5, 2, 4]),
    ("wave", (160, 40, 40), 16, 4, 32, 1, [16]),
]


def _desc(P, scheme, shape, rate, k, T, wb, ro=0):
    nz, ny, nx = shape
    if scheme == "heat":
        return P.make_desc(nx, ny, nz, P.OOCS_HEAT, synthetic.heat_star_coef(0.1), 8 << 30,
                           rate_bits=rate, temporal_depth=k, slab_planes=T, working_buffers=wb)
    return P.make_desc(nx, ny, nz, P.OOCS_WAVE, synthetic.wave_star_coef(), 8 << 30,
                       rate_bits=rate, temporal_depth=k, slab_planes=T, working_buffers=wb,
                       readonly_resident=ro)


@pytest.mark.parametrize("case", CASES)
def test_schedule_is_race_free(P, case):
    scheme, shape, rate, k, T, wb, calls = case
    desc = _desc(P, scheme, shape, rate, k, T, wb)
    trace = P.oocs_trace_schedule(desc, calls)
    assert check(trace, swb=(wb == 1)) is None
    plan = P.oocs_query(desc)
    visits = {o["visit"] for o in trace if o["visit"] >= 0}
    sweeps = sum(-(-c // k) for c in calls)
    assert len(visits) == sweeps * plan.num_slabs
    # every layer of every streamed field crosses the link once per sweep
    h2d_layers = sum(o["access"][0][3] - o["access"][0][2] for o in trace if o["op"] == "H2D")
    assert h2d_layers == sweeps * (shape[0] // 4)
    # in sweep p+1 every host layer read was written back in sweep p
    fout = 2 if scheme == "wave" else 1
    for visit, writers in host_dataflow(trace, shape[0] // 4, fout):
        sweep = visit // plan.num_slabs
        expect = None if sweep == 0 else sweep - 1
        got = {None if w is None else w // plan.num_slabs for w in writers}
        assert got == {expect}, (visit, got)


@pytest.mark.parametrize("wb", [1, 3])
def test_schedule_with_resident_model(P, wb):
    """m kept on the device: only U and U_PREV are copied per visit; the
    schedule stays race-free and every streamed layer still crosses once."""
    desc = _desc(P, "wave", (128, 72, 40), 16, 4, 32, wb, ro=1)
    trace = P.oocs_trace_schedule(desc, [10])
    assert check(trace, swb=(wb == 1)) is None
    fields = {f for o in trace if o["op"] == "H2D" for (k, f, lo, hi, w) in o["access"] if k == "HOST"}
    assert fields == {0, 1}
    h2d_layers = sum(o["access"][0][3] - o["access"][0][2] for o in trace if o["op"] == "H2D")
    assert h2d_layers == 3 * (128 // 4)


@pytest.mark.parametrize("drop", ["d2h", "decoded", "wrel", "h2d"])
def test_check_detects_missing_waits(P, drop):
    """Removing one kind of cross-stream wait leaves a hazard the check reports."""
    base = {"d2h": range(1000, 2000), "decoded": range(100, 103), "wrel": range(300, 303),
            "h2d": range(200, 203)}[drop]
    # with one working buffer the borrowed-overlap wait is implied by the
    # working-buffer chain; with three (classic) it is the only guard
    wb = 3 if drop == "h2d" else 1
    desc = _desc(P, "wave", (128, 72, 40), 16, 4, 32, wb)
    trace = P.oocs_trace_schedule(desc, [12])
    assert check(trace, swb=(wb == 1)) is None
    cut = [o for o in trace if not (o["op"] == "WAIT" and o["event"] in base)]
    assert len(cut) < len(trace)
    assert check(cut, swb=(wb == 1)) is not None


def test_classic_mode_lets_visits_overlap(P):
    """With three working buffers (Fig. 6a) kernels of consecutive visits are not ordered."""
    desc = _desc(P, "heat", (128, 128, 128), 0, 1, 32, 3)
    trace = P.oocs_trace_schedule(desc, [4])
    assert check(trace, swb=False) is None
    assert check(trace, swb=True) is not None


def test_trace_capacity_error(P):
    import ctypes
    desc = _desc(P, "heat", (128, 128, 128), 16, 1, 32, 1)
    calls = (ctypes.c_int32 * 1)(3)
    count = ctypes.c_int64(0)
    buf = (P.oocs.oocs_trace_op * 2)()
    st = P.lib().oocs_trace_schedule(ctypes.byref(desc), calls, 1, buf, 2, ctypes.byref(count))
    assert st == 1 and count.value > 2


# ----------------------------------------------------------------- batches

BATCH = [("heat", (128, 128, 128), 16, 2, 32, 0), ("wave", (128, 72, 40), 16, 4, 32, 0),
         ("heat", (64, 36, 100), 0, 3, 16, 0), ("wave", (96, 48, 64), 12, 3, 24, 1),
         ("wave", (40, 16, 24), 8, 4, 64, 0)]


def _batch_descs(P, spec=BATCH):
    return [_desc(P, sc, sh, rate, k, T, 1, ro) for sc, sh, rate, k, T, ro in spec]


@pytest.mark.parametrize("calls", [[10], [3, 4], [1, 7, 2]])
def test_batch_schedule_is_race_free(P, calls):
    """Several problems through one pipeline: no race on the shared working
    buffer and staging slots, kernels of all visits ordered (one working
    buffer), and per problem every host layer read in sweep p+1 was written
    back in sweep p."""
    descs = _batch_descs(P)
    trace = P.oocs_batch_trace_schedule(descs, calls)
    assert check(trace, swb=True) is None
    plans = [P.oocs_query(d) for d in descs]
    h2d = {}
    for o in trace:
        if o["op"] == "H2D":
            i = o["access"][1][1] // 3
            h2d[i] = h2d.get(i, 0) + o["access"][0][3] - o["access"][0][2]
    for i, (sc, sh, rate, k, T, ro) in enumerate(BATCH):
        sweeps = sum(-(-c // k) for c in calls)
        assert h2d[i] == sweeps * (sh[0] // 4)
    # host dataflow per problem: the last writer of every layer read is the previous sweep
    writer, sweep_of = {}, {}
    visits = sorted({o["visit"] for o in trace if o["visit"] >= 0})
    for o in trace:
        for (kd, idx, lo, hi, w) in o["access"]:
            if kd == "HOST":
                sweep_of.setdefault((idx // 3, o["visit"]), None)
    count = {}
    order = []
    for o in trace:
        if o["op"] == "H2D":
            order.append((o["access"][1][1] // 3, o["visit"]))
    seen = {}
    for i, v in order:
        seen.setdefault(i, []).append(v)
    for i, vs in seen.items():
        S = plans[i].num_slabs
        for n, v in enumerate(vs):
            sweep_of[(i, v)] = n // S
    for o in trace:
        if o["op"] == "H2D":
            i = o["access"][1][1] // 3
            sw = sweep_of[(i, o["visit"])]
            for (kd, idx, lo, hi, w) in o["access"][1:]:
                if idx % 3 >= (2 if BATCH[i][0] == "wave" else 1):
                    continue
                got = {writer.get((idx, l)) for l in range(lo, hi)}
                assert got == {None if sw == 0 else sw - 1}, (i, o["visit"], got)
        if o["op"] == "D2H":
            for (kd, idx, lo, hi, w) in o["access"]:
                if kd == "HOST" and w:
                    for l in range(lo, hi):
                        writer[(idx, l)] = sweep_of[(idx // 3, o["visit"])]
    assert len(visits) == sum(sum(-(-c // BATCH[i][3]) for c in calls) * plans[i].num_slabs
                              for i in range(len(BATCH)))


@pytest.mark.parametrize("drop", ["decoded", "wrel"])
def test_batch_check_detects_missing_waits(P, drop):
    base = {"decoded": range(100, 103), "wrel": range(300, 303)}[drop]
    trace = P.oocs_batch_trace_schedule(_batch_descs(P), [6])
    cut = [o for o in trace if not (o["op"] == "WAIT" and o["event"] in base)]
    assert len(cut) < len(trace)
    assert check(cut, swb=True) is not None


def test_batch_workspace_is_per_region_maximum(P):
    """One working buffer and one slot set, each region sized for the largest
    problem's, plus the resident models: the exact sum of the layout."""
    descs = _batch_descs(P)
    a256 = lambda b: -(-b // 256) * 256
    buf = slot_in = slot_out = 0
    nbuf = fin = fout = 0
    resident = 0
    for (sc, (nz, ny, nx), rate, k, T, ro), d in zip(BATCH, descs):
        p = P.oocs_query(d)
        wave = sc == "wave"
        buf = max(buf, a256(p.window_planes * nx * ny * 4))
        slot_in = max(slot_in, a256(min(-(-(T + p.halo_planes) // 4), nz // 4) * p.layer_bytes))
        slot_out = max(slot_out, a256(min(T // 4, nz // 4) * p.layer_bytes))
        nbuf = max(nbuf, 3 if wave and not ro else 2)
        fin = max(fin, p.fields_in)
        fout = max(fout, p.fields_out)
        resident += a256(nz * ny * nx * 4) if wave and ro else 0
        resident += (256 + 65536 * 4) if wave else 0  # device wavelet and time index
    want = nbuf * buf + 3 * fin * slot_in + 3 * fout * slot_out + resident
    assert P.oocs_batch_query(descs) == want
    # many copies of one problem cost one problem's pipeline (plus each wave
    # problem's own device wavelet)
    one = [descs[1]]
    assert P.oocs_batch_query(one * 16) == P.oocs_query(descs[1]).workspace_bytes + 15 * (256 + 65536 * 4)


@pytest.mark.parametrize("rate", [16, 0])
def test_adjoint_sweep_schedule(P, rate):
    """Adjoint sweeps (slabs in reverse z order, whole windows copied): race-free,
    kernels of different visits ordered, every layer of lam^(k+1) overwritten
    once per step with lam^(k-1), nothing written to lam^k or u^(k-1)."""
    nz, ny, nx = 96, 40, 48
    d = P.make_desc(nx, ny, nz, P.OOCS_WAVE_ADJOINT, synthetic.wave_star_coef(), 8 << 30, rate_bits=rate,
                    temporal_depth=1, slab_planes=32, readonly_resident=1)
    plan = P.oocs_query(d)
    assert (plan.num_slabs, plan.halo_planes, plan.temporal_depth) == (3, 4, 1)
    trace = P.oocs_trace_schedule(d, [1, 1, 1])
    assert check(trace, swb=True) is None
    order = [o["visit"] for o in trace if o["op"] == "H2D"]
    firsts = [lo for o in trace if o["op"] == "H2D" for (k, i, lo, hi, w) in o["access"] if k == "HOST" and i == 1]
    assert firsts[:3] == [64 // 4, 32 // 4, 0]  # slabs in reverse z order
    writes = [(i, lo, hi) for o in trace if o["op"] == "D2H" for (k, i, lo, hi, w) in o["access"] if w]
    # the two lam stores trade roles every step: steps alternate between them
    assert [i for i, _, _ in writes] == [1] * 3 + [0] * 3 + [1] * 3
    assert sum(hi - lo for _, lo, hi in writes) == 3 * (nz // 4)


@pytest.mark.parametrize("calls", [[3], [2, 2], [5]])
def test_adjoint_steps_in_one_call(P, calls):
    """Several adjoint steps per call are chained by the previous step's
    per-slab D2H events instead of a join: still race-free on the host stores
    (whose roles alternate) and the device buffers, kernels of different
    visits still ordered; without the chained waits the check finds a race."""
    nz, ny, nx = 96, 40, 48
    d = P.make_desc(nx, ny, nz, P.OOCS_WAVE_ADJOINT, synthetic.wave_star_coef(), 8 << 30, rate_bits=16,
                    temporal_depth=1, slab_planes=32, readonly_resident=1)
    trace = P.oocs_trace_schedule(d, calls)
    assert check(trace, swb=True) is None
    steps = sum(calls)
    writes = [(i, hi - lo) for o in trace if o["op"] == "D2H" for (k, i, lo, hi, w) in o["access"] if w]
    assert sum(n for _, n in writes) == steps * (nz // 4)  # every layer of lam once per step
    assert [i for i, _ in writes] == [(j + 1) % 2 for j in range(steps) for _ in range(3)]
    cut = [o for o in trace if not (o["op"] == "WAIT" and 1000 <= o["event"] < 2000)]
    if max(calls) > 1:
        assert len(cut) < len(trace)
        assert check(cut, swb=True) is not None


def test_streams_by_role_with_one_working_buffer(P):
    """One working buffer: host->device copies on stream 0, kernels on stream
    1, device->host copies on stream 2 (classic mode keeps the round robin),
    and dropping the wait that keeps an out slot until its copy-back has run
    leaves a race the check reports."""
    desc = _desc(P, "wave", (128, 72, 40), 16, 4, 32, 1)
    trace = P.oocs_trace_schedule(desc, [12])
    assert check(trace) is None
    streams = {op: {o["stream"] for o in trace if o["op"] == op} for op in ("H2D", "LOAD", "STEP", "STORE", "D2H")}
    assert streams == {"H2D": {0}, "LOAD": {1}, "STEP": {1}, "STORE": {1}, "D2H": {2}}
    cut = [o for o in trace if not (o["op"] == "WAIT" and o["event"] in range(600, 603))]
    assert len(cut) < len(trace)
    assert "race" in check(cut)
    classic = P.oocs_trace_schedule(_desc(P, "wave", (128, 72, 40), 16, 4, 32, 3), [12])
    assert {o["stream"] for o in classic if o["op"] == "H2D"} == {0, 1, 2}


@pytest.mark.parametrize("case", [c for c in CASES if c[0] == "heat" and c[2] > 0])
def test_schedule_with_fused_codec_is_race_free(P, case):
    """codec_fusion: step 1 of a visit reads the staging slots itself (the
    slots are released after it) and the last step writes the out slot
    itself (the slot's copy-back by visit g-3 is ordered before the steps);
    the traced schedule stays race-free, with no decode launch and, where a
    visit has two or more steps, no encode launch."""
    scheme, shape, rate, k, T, wb, calls = case
    desc = _desc(P, scheme, shape, rate, k, T, wb)
    desc.codec_fusion = 1
    trace = P.oocs_trace_schedule(desc, calls)
    assert check(trace, swb=(wb == 1)) is None
    assert not any(o["op"] == "LOAD" for o in trace)
    assert any(o["op"] == "STEP" and any(a[0] == "IN_SLOT" for a in o["access"]) for o in trace)
    if k > 1:
        assert any(o["op"] == "STEP" and any(a[0] == "OUT_SLOT" for a in o["access"]) for o in trace)
        if all(c % k == 0 for c in calls):
            assert not any(o["op"] == "STORE" for o in trace)
