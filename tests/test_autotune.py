"""Host logic of the autotuner (no GPU): candidate plans, classes, the cache,
and fitting a batch into its budget.  Timing is replaced by a cost model."""
import json

import pytest

import synthetic


@pytest.fixture(scope="module")
def P():
    import paper_2204_11315_gb300 as P
    P.lib()
    return P


@pytest.fixture
def A(monkeypatch):
    from paper_2204_11315_gb300 import autotune as A
    calls = []

    def fake_time(desc, steps, probe=None):
        # cheaper with fewer slabs, k = 4 and lower rates
        S = -(-int(desc.nz) // int(desc.slab_planes))
        calls.append((int(desc.nz), S, int(desc.temporal_depth), int(desc.rate_bits)))
        # the 64 x 8 tile costs A.tile8_cost more (negative: it is faster)
        return (1.0 * S + abs(int(desc.temporal_depth) - 4) * 0.1 + int(desc.rate_bits) * 0.01
                + A.tile8_cost * int(desc.step_tile))

    class NoProbe:
        def __init__(self, desc, seed=0, data=None):
            self.data = data

    errors = {8: 3e-3, 12: 2e-4, 16: 1e-5, 20: 6e-7, 24: 4e-8}

    def fake_errors(desc, steps, probe, rates=A.RATES):
        A.err_calls.append((int(desc.nz), steps, probe.data))
        return {r: errors[r] for r in rates}

    monkeypatch.setattr(A, "time_candidate", fake_time)
    monkeypatch.setattr(A, "measure_rate_errors", fake_errors)
    monkeypatch.setattr(A, "_Probe", NoProbe)
    A.calls = calls
    A.tile8_cost = 0.05
    A.err_calls = []
    A.errors = errors
    return A


def _wave(P, nz, ny, nx, budget=8 << 30):
    return P.make_desc(nx, ny, nz, P.OOCS_WAVE, synthetic.wave_star_coef(), budget)


def _heat(P, nz, ny, nx, budget=8 << 30):
    return P.make_desc(nx, ny, nz, P.OOCS_HEAT, synthetic.heat_star_coef(0.1), budget)


def test_rate_follows_the_measured_error(A):
    e = {8: 3e-3, 12: 2e-4, 16: 1e-5}
    assert A.rate_for(e, 1e-4) == 16        # 1e-5 <= 0.5e-4
    assert A.rate_for(e, 2e-3) == 12        # 2e-4 <= 1e-3 < 3e-3
    assert A.rate_for(e, 0.05) == 8
    assert A.rate_for(e, 1e-6) == 0         # nothing close enough: uncompressed
    assert A.rate_for({**e, 20: 6e-7, 24: 4e-8}, 2e-6) == 20  # the higher rates when 16 misses
    assert A.rate_for({**e, 20: 6e-7, 24: 4e-8}, 1e-6) == 24
    assert A.rate_for({8: 0.0, 16: 0.0}, 1e-9) == 8


def test_rate_error_is_measured_on_the_problem_data(P, A):
    descs = [_heat(P, 96, 96, 96), _wave(P, 64, 64, 64)]
    data = [{0: "heat field"}, {0: "u", 2: "m"}]
    out, rep = A.tune(descs, 1e-4, 8 << 30, data=data, err_steps=50)
    assert [c[2] for c in A.err_calls] == data and all(c[1] == 50 for c in A.err_calls)
    assert [r["rate"] for r in rep["problems"]] == [16, 16]
    assert rep["problems"][0]["errors"] == {"8": 3e-3, "12": 2e-4, "16": 1e-5, "20": 6e-7, "24": 4e-8}


def test_candidate_plans_respect_region_sharing(P, A):
    d = _wave(P, 64, 64, 64)
    # k = 4, r = 4: h = 16, so four slabs of 16 planes (< 2h) are not a plan
    assert A.with_plan(d, 4, 4, 16) is None
    two = A.with_plan(d, 2, 4, 16)
    assert (two.slab_planes, two.temporal_depth, two.rate_bits) == (32, 4, 16)
    assert P.oocs_query(two).num_slabs == 2
    one = A.with_plan(_heat(P, 100, 36, 44), 1, 8, 12)
    assert P.oocs_query(one).num_slabs == 1


def test_tune_picks_the_fastest_and_reuses_classes(P, A, tmp_path):
    cache = tmp_path / "tune.json"
    descs = [_wave(P, 128, 128, 128), _wave(P, 128, 128, 124), _heat(P, 96, 96, 96)]
    out, rep = A.tune(descs, 2e-3, 8 << 30, str(cache))
    assert rep["classes"] == 2  # the two wave grids share a class
    for d in out:
        assert P.oocs_query(d).num_slabs == 1
        assert int(d.temporal_depth) == 4 and int(d.rate_bits) == 12
    n_timed = len(A.calls)
    assert rep["candidates_timed"] == n_timed
    # cached: nothing is timed again
    out2, rep2 = A.tune(descs, 2e-3, 8 << 30, str(cache))
    assert rep2["candidates_timed"] == 0 and len(A.calls) == n_timed
    assert [(int(a.slab_planes), int(a.temporal_depth)) for a in out] == \
        [(int(a.slab_planes), int(a.temporal_depth)) for a in out2]
    assert set(json.loads(cache.read_text())) == {r["class"] for r in rep["problems"]}


def test_batch_is_fitted_into_the_budget(P, A):
    """One slab each is fastest, but the shared workspace must fit: the largest
    windows are split into more slabs until it does."""
    descs = [_wave(P, 384, 384, 384), _wave(P, 64, 64, 64), _heat(P, 256, 256, 256)]
    loose, _ = A.tune(descs, 1e-4, 8 << 30)
    budget = P.oocs_batch_query(loose) // 2
    tight, rep = A.tune(descs, 1e-4, budget)
    assert P.oocs_batch_query(tight) <= budget
    assert P.oocs_query(tight[0]).num_slabs > 1


def test_class_plan_adapts_to_a_thin_member(P, A, tmp_path):
    """A class groups grids by volume, so its measured plan (here 4 slabs at
    k = 4) can be invalid for a member with few planes: 64 x 192 x 192 has the
    class's cube root, but 4 slabs of 16 planes break region sharing for the
    25-point star (h = 16).  The member takes the nearest valid plan (fewer
    slabs) instead of failing the whole batch."""
    cache = tmp_path / "tune.json"
    member = _wave(P, 64, 192, 192)
    key = A.class_key(A.O.oocs_desc.from_buffer_copy(member), 8 << 30, 1e-4)
    assert key == A.class_key(_wave(P, 128, 128, 144), 8 << 30, 1e-4)
    cache.write_text(json.dumps({key: {"slabs": 4, "k": 4, "rate": 16, "ms_per_step": 1.0,
                                       "tried": [], "errors": {}}}))
    assert A.with_plan(member, 4, 4, 16) is None
    out, rep = A.tune([member], 1e-4, 8 << 30, str(cache))
    assert rep["candidates_timed"] == 0
    assert (rep["problems"][0]["slabs"], rep["problems"][0]["k"]) == (2, 4)
    assert P.oocs_query(out[0]).num_slabs == 2 and int(out[0].temporal_depth) == 4


def test_tile_is_searched_and_kept_per_class(P, A, tmp_path):
    """Both step tiles are timed for every (slabs, k); the faster one is the
    class's choice, cached and applied to every member, and a desc with it
    is a valid plan of the library."""
    cache = tmp_path / "tune.json"
    descs = [_heat(P, 96, 96, 96), _heat(P, 96, 100, 92)]
    out, rep = A.tune(descs, 2e-3, 8 << 30, str(cache))
    assert all(int(d.step_tile) == 0 for d in out)
    tried = json.loads(cache.read_text())[rep["problems"][0]["class"]]["tried"]
    assert {t["tile"] for t in tried} == {0, 1}
    assert len(tried) == 2 * len({(t["slabs"], t["k"]) for t in tried})
    A.tile8_cost = -0.05
    out8, rep8 = A.tune(descs, 2e-3, 8 << 30, str(tmp_path / "tune8.json"))
    assert all(int(d.step_tile) == 1 for d in out8)
    assert all(r["tile"] == 1 for r in rep8["problems"])
    assert P.oocs_query(out8[0]).num_slabs >= 1
    bad = A.with_plan(descs[0], 1, 4, 12, 1)
    bad.step_tile = 2
    with pytest.raises(P.OOCSError):
        P.oocs_query(bad)
