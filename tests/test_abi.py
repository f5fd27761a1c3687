"""The C ABI library builds for sm_103a, loads without a GPU, exports every
symbol include/oocs.h declares, and plans workloads (host logic only: no call
here touches a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

import synthetic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    import paper_2204_11315_gb300 as P
    P.lib()
    return P


def header_symbols():
    text = open(os.path.join(ROOT, "include", "oocs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(oocs_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_header_symbol(P):
    syms = header_symbols()
    assert len(syms) >= 15
    L = ctypes.CDLL(P.library_path())
    for s in syms:
        assert hasattr(L, s), s
    # the binding wraps exactly the header's entry points
    assert sorted(P.oocs.SIGNATURES) == syms
    out = subprocess.run(["nm", "-D", "--defined-only", P.library_path()], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (oocs_\w+)", out))
    assert exported == set(syms)


def test_version(P):
    assert "sm_103a" in P.oocs_version()


def _c1(P, **kw):
    args = dict(rate_bits=16, temporal_depth=1, slab_planes=32)
    args.update(kw)
    return P.make_desc(128, 128, 128, P.OOCS_HEAT, synthetic.heat_star_coef(0.1), 1 << 30, **args)


def test_plan_heat_workload(P):
    p = P.oocs_query(_c1(P))
    assert (p.slab_planes, p.num_slabs, p.temporal_depth, p.halo_planes) == (32, 4, 1, 4)
    assert p.window_planes == 40
    assert p.host_store_bytes == 128 ** 3 * 16 // 8
    assert p.layer_bytes == 32 * 32 * 8 * 16


def test_plan_wave_workload(P):
    d = P.make_desc(512, 512, 512, P.OOCS_WAVE, synthetic.wave_star_coef(), 4 << 30,
                    rate_bits=16, temporal_depth=4, slab_planes=64)
    p = P.oocs_query(d)
    assert (p.num_slabs, p.halo_planes, p.window_planes) == (8, 16, 96)
    assert (p.fields_in, p.fields_out) == (3, 2)
    assert p.workspace_bytes <= 4 << 30
    # single working buffer saves two working sets of three window buffers
    buf = 96 * 512 * 512 * 4
    assert p.workspace_classic_bytes - p.workspace_swb_bytes == 2 * 3 * buf
    # workspace = 3 window buffers + 3 staging slots per field in + 3 per field out
    slot_in = (64 + 16) // 4 * p.layer_bytes
    slot_out = 64 // 4 * p.layer_bytes
    # + the device wavelet and time index read by replayed graphs
    src = 256 + 65536 * 4
    assert p.workspace_swb_bytes == 3 * buf + 3 * 3 * slot_in + 3 * 2 * slot_out + src


def test_plan_wave_resident_model(P):
    """readonly_resident: m leaves the staging slots and the window buffers and
    takes one FP32 grid in the workspace; heat ignores the flag."""
    kw = dict(rate_bits=16, temporal_depth=4, slab_planes=64)
    coef = synthetic.wave_star_coef()
    p0 = P.oocs_query(P.make_desc(512, 512, 512, P.OOCS_WAVE, coef, 4 << 30, **kw))
    p1 = P.oocs_query(P.make_desc(512, 512, 512, P.OOCS_WAVE, coef, 4 << 30, readonly_resident=1, **kw))
    assert (p1.fields_in, p1.fields_out, p1.readonly_resident) == (2, 2, 1)
    buf = 96 * 512 * 512 * 4
    slot_in = (64 + 16) // 4 * p1.layer_bytes
    grid = 512 ** 3 * 4
    assert p1.workspace_swb_bytes == p0.workspace_swb_bytes - buf - 3 * slot_in + grid
    assert p1.workspace_classic_bytes == p0.workspace_classic_bytes - 3 * buf - 3 * slot_in + grid
    assert p1.workspace_bytes <= 4 << 30
    h = P.oocs_query(P.make_desc(128, 128, 128, P.OOCS_HEAT, synthetic.heat_star_coef(0.1), 1 << 30,
                                 rate_bits=16, readonly_resident=1))
    assert (h.fields_in, h.readonly_resident) == (1, 0)
    with pytest.raises(P.OOCSError):
        P.oocs_query(P.make_desc(128, 128, 128, P.OOCS_WAVE, coef, 1 << 30, readonly_resident=2))


def test_auto_slab_thickness_from_budget(P):
    # the budget of the T = 32 plan makes the planner pick T = 32 (4 slabs)
    need = P.oocs_query(_c1(P)).workspace_bytes
    d = P.make_desc(128, 128, 128, P.OOCS_HEAT, synthetic.heat_star_coef(0.1), need,
                    rate_bits=16, temporal_depth=1, slab_planes=0)
    p = P.oocs_query(d)
    assert p.slab_planes == 32 and p.num_slabs == 4
    d.device_budget = need - 1
    assert P.oocs_query(d).slab_planes < 32


@pytest.mark.parametrize("field,value", [("nx", 130), ("nz", 0), ("scheme", 5), ("radius", 2),
                                         ("rate_bits", 33), ("slab_planes", 6),
                                         ("working_buffers", 2), ("temporal_depth", -1),
                                         ("step_tile", 2), ("step_fusion", 3), ("codec_fusion", 2),
                                         ("codec", 2)])
def test_invalid_descriptions(P, field, value):
    d = _c1(P)
    setattr(d, field, value)
    with pytest.raises(P.OOCSError) as e:
        P.oocs_query(d)
    assert e.value.status == 1
    assert P.oocs_last_error()


def test_halo_rule_and_budget_errors(P):
    d = P.make_desc(256, 64, 64, P.OOCS_WAVE, synthetic.wave_star_coef(), 1 << 30,
                    rate_bits=8, temporal_depth=4, slab_planes=16)
    with pytest.raises(P.OOCSError) as e:  # T = 16 < 2h = 32
        P.oocs_query(d)
    assert e.value.status == 1
    d.slab_planes = 32
    d.device_budget = 1000
    with pytest.raises(P.OOCSError) as e:
        P.oocs_query(d)
    assert e.value.status == 2
    d.scheme = P.OOCS_WAVE
    d.radius = 1
    with pytest.raises(P.OOCSError):
        P.oocs_query(d)


def test_null_arguments(P):
    L = P.lib()
    assert L.oocs_query(None, None) == 1
    assert L.oocs_step(None, 1) == 1
    assert L.oocs_synchronize(None, 0) == 1
    assert L.oocs_destroy(None) == 0
    assert L.oocs_last_error(None)


def test_stats_binding_layout(P):
    """The stats record of the binding mirrors oocs_stats: nested per-class
    counters for the kernels and the copies, as dicts."""
    d = P.oocs.oocs_stats().as_dict()
    for k in ("load", "step", "store", "h2d", "d2h"):
        assert set(d[k]) == {"launches", "units", "device_ms"}
    assert d["h2d_bytes"] == 0 and d["last_step_ms"] == 0.0
    e = P.oocs.oocs_timeline_entry()
    assert [f for f, _ in e._fields_] == ["cls", "stream", "visit", "start_ms", "end_ms"]


def test_codec_fusion_excludes_step_pairs(P):
    """The codec fused into the steps and the fused step pairs are exclusive;
    each alone is a valid plan with the same workspace as the unfused one."""
    d = _c1(P)
    base = P.oocs_query(d).workspace_bytes
    d.codec_fusion = 1
    assert P.oocs_query(d).workspace_bytes == base
    d.step_fusion = 1
    with pytest.raises(P.OOCSError) as e:
        P.oocs_query(d)
    assert e.value.status == 1 and "codec_fusion" in str(e.value)
    d.codec_fusion = 0
    assert P.oocs_query(d).workspace_bytes == base
