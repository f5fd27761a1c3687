"""Autotuner of a problem's slab thickness T, temporal depth k and codec rate.

The knobs of the out-of-core sweep (Sec. 3.1 temporal blocking, Sec. 4.2
fixed rate) trade redundant halo work, pipeline depth and link bytes against
each other differently for every grid, so they are measured, not modelled:

* rate: measured on the problem's own seeded data.  The problem runs
  `err_steps` time steps uncompressed and at each rate in {8, 12, 16, 20, 24} with the
  shallowest temporal depth tried (the most codec round trips of any
  candidate); the lowest rate whose relative L2 error against the
  uncompressed run is within half the tolerance is taken (rate 0 when none
  is);
* slabs: S in {1, 2, 4} (T = nz / S rounded up to the 4-plane layer), kept
  only when T >= 2 h so region sharing holds and the plan fits the budget;
* temporal depth: k in {2, 4, 8} for the 7-point heat stencil, {2, 4} for the
  25-point wave stencil;
* the step kernel's x-y tile: 64 x 16 or 64 x 8 points per CTA
  (`oocs_desc.step_tile`; smaller tiles give more CTAs on small planes).

Each (S, k, tile) candidate at the chosen rate runs `steps` time steps of the
problem's grid through a fresh context: one warm-up call, then the median of
`reps` calls timed with CUDA events on stream 0 (every oocs_step joins its
three streams into stream 0 at its end, so the event follows the last copy).
Problems are grouped into classes (scheme and the rounded cube root of the
volume); one problem per class is measured and its (S, k, rate) is applied to
the class.  Choices are cached in a JSON file keyed by class, budget and
tolerance.  The launch geometry of each step (z chunks or balanced ranges)
is chosen per launch by the occupancy model in the library.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import oocs as O

RATES = (8, 12, 16, 20, 24)  # bits per value; 20 and 24 for fields whose rate-16 error is above the bar
ERROR_MARGIN = 0.5  # a rate is taken when its measured error is within this share of the tolerance
SLABS = (1, 2, 4)
DEPTHS = {O.OOCS_HEAT: (2, 4, 8), O.OOCS_WAVE: (2, 4)}
TILES = (0, 1)  # oocs_desc.step_tile: 64 x 16, 64 x 8


def rate_for(errors: dict, tol: float) -> int:
    """The lowest rate whose measured error is within ERROR_MARGIN * tol; 0 when none is."""
    ok = [r for r in sorted(errors) if r and errors[r] <= ERROR_MARGIN * tol]
    return ok[0] if ok else 0


def with_plan(desc, slabs: int, k: int, rate: int, tile: int = 0):
    """desc with S = slabs slabs (T rounded up to 4 planes), depth k, rate and
    step tile; None if invalid."""
    d = O.oocs_desc.from_buffer_copy(desc)
    T = -(-int(d.nz) // slabs)
    T = -(-T // 4) * 4
    h = 4 * -(-(k * d.radius) // 4)
    if slabs > 1 and T < 2 * h:
        return None
    d.slab_planes = min(T, int(d.nz))
    d.temporal_depth = k
    d.rate_bits = rate
    d.step_tile = tile
    try:
        O.oocs_query(d)
    except O.OOCSError:
        return None
    return d


def member_plan(desc, slabs: int, k: int, rate: int, tile: int = 0):
    """(desc, slabs, k) of the class's plan applied to one member of the class;
    members differ in shape, so when the class's plan is invalid for this one
    (too few planes per slab for region sharing, or a window over the budget)
    the nearest valid plan is taken: fewer slabs first, then more, then the
    next shallower depths.  (None, slabs, k) when none is valid."""
    depths = [k] + [j for j in sorted(DEPTHS[desc.scheme], reverse=True) if j < k]
    for kk in depths:
        for s in [slabs] + list(range(slabs - 1, 0, -1)) + [slabs << j for j in range(1, 7)]:
            t = with_plan(desc, s, kk, rate, tile)
            if t is not None:
                return t, s, kk
    return None, slabs, k


def class_key(desc, budget: int, tol: float) -> str:
    vol = int(desc.nx) * int(desc.ny) * int(desc.nz)
    side = int(round(vol ** (1.0 / 3.0) / 32.0)) * 32
    scheme = "heat" if desc.scheme == O.OOCS_HEAT else "wave"
    return f"{scheme}:{side}:{budget}:{tol:g}:ro{int(desc.readonly_resident)}"


class _Probe:
    """FP32 fields of one grid and host stores, pinned once and reused by
    every candidate of the grid: the problem's
    own initial fields when given (`data`: field id -> array), else seeded
    stand-ins of the same kind."""

    def __init__(self, desc, seed: int = 0, data=None):
        import torch
        shape = (int(desc.nz), int(desc.ny), int(desc.nx))
        rng = np.random.default_rng(seed)
        nf = 1 if desc.scheme == O.OOCS_HEAT else 3
        self.shape = shape
        self.fields = {}
        for f in range(nf):
            t = torch.empty(shape, dtype=torch.float32, pin_memory=True)
            a = t.numpy()
            if data is not None and f in data:
                a[...] = np.asarray(data[f], dtype=np.float32).reshape(shape)
            elif desc.scheme == O.OOCS_HEAT:
                a[...] = rng.random(shape, dtype=np.float32)
            elif f == O.OOCS_FIELD_M:
                a[...] = 0.02 + 0.1 * rng.random(shape, dtype=np.float32)
            else:
                a[...] = 1e-3 * rng.random(shape, dtype=np.float32)
            self.fields[f] = t
        raw = 4 * int(desc.nx) * int(desc.ny) * int(desc.nz)  # the largest store (rate 0)
        self.stores = [torch.empty(raw, dtype=torch.uint8, pin_memory=True) for _ in range(nf)]


def time_candidate(desc, steps: int, probe: _Probe | None = None, reps: int = 3) -> float:
    """Milliseconds per time step: the median of `reps` oocs_step(steps) calls
    after one warm-up call, on the probe's data."""
    import torch
    probe = probe or _Probe(desc)
    st = O.OutOfCoreStencil(desc, stores=probe.stores)
    try:
        for f, t in probe.fields.items():
            st.compress(f, t)
        st.synchronize(600.0)
        st.step(steps)
        st.synchronize(600.0)
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st.streams[0])
            st.step(steps)
            e1.record(st.streams[0])  # oocs_step ends with a join of its streams into stream 0
            st.synchronize(600.0)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / steps)
        return float(np.median(times))
    finally:
        st.close()


def measure_rate_errors(desc, steps: int, probe: _Probe, rates=RATES) -> dict:
    """Relative L2 error of u after `steps` time steps at each rate against the
    uncompressed run of the same plan (one slab, the shallowest depth tried:
    the most codec round trips of any candidate), on the probe's data."""
    k = min(DEPTHS[desc.scheme])

    def run(rate):
        d = with_plan(desc, 1, k, rate)
        if d is None:
            return None
        st = O.OutOfCoreStencil(d, stores=probe.stores)
        try:
            for f, t in probe.fields.items():
                st.compress(f, t)
            st.step(steps)
            out = st.decompress(O.OOCS_FIELD_U)
            st.synchronize(600.0)
            return out.numpy().astype(np.float64)
        finally:
            st.close()

    ref = run(0)
    errs = {}
    for r in rates:
        got = run(r)
        if ref is None or got is None:
            continue
        errs[r] = float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))
    return errs


def tune_one(desc, tol: float, steps: int = 4, data=None, err_steps: int | None = None):
    """(best desc, ms per step, every candidate timed, measured errors by rate)
    for one problem."""
    tried = []
    best, best_ms = None, math.inf
    probe = _Probe(desc, data=data)
    errors = measure_rate_errors(desc, err_steps or steps, probe)
    rate = rate_for(errors, tol)
    for slabs in SLABS:
        for k in DEPTHS[desc.scheme]:
            for tile in TILES:
                d = with_plan(desc, slabs, k, rate, tile)
                if d is None:
                    continue
                ms = time_candidate(d, max(steps, k), probe)
                tried.append({"slabs": slabs, "k": k, "rate": rate, "tile": tile, "ms_per_step": ms})
                if ms < best_ms:
                    best, best_ms = d, ms
    return best, best_ms, tried, errors


def tune(descs, tol: float, budget: int, cache_path: str | None = None, steps: int = 4, data=None,
         err_steps: int | None = None):
    """Tuned copies of descs (and a report).  data: optional per-problem dict
    (field id -> initial array) on which a class's rate error is measured;
    err_steps: time steps of that measurement (default `steps`).  The batch of
    the tuned descs is kept within `budget` bytes of shared workspace by adding
    slabs to the largest problems if needed."""
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    out, report, timed = [], [], 0
    for i, d in enumerate(descs):
        d = O.oocs_desc.from_buffer_copy(d)
        d.device_budget = budget
        key = class_key(d, budget, tol)
        if key not in cache:
            best, ms, tried, errors = tune_one(d, tol, steps, data[i] if data is not None else None, err_steps)
            timed += len(tried)
            if best is None:
                raise O.OOCSError(2, f"no plan of {key} fits the budget")
            cache[key] = {"slabs": -(-int(d.nz) // int(best.slab_planes)), "k": int(best.temporal_depth),
                          "rate": int(best.rate_bits), "tile": int(best.step_tile), "ms_per_step": ms,
                          "tried": tried,
                          "errors": {str(r): e for r, e in errors.items()}}
        c = cache[key]
        t, slabs, k = member_plan(d, c["slabs"], c["k"], c["rate"], c.get("tile", 0))
        if t is None:
            raise O.OOCSError(2, f"no plan of class {key} fits problem {i}")
        out.append(t)
        report.append({"class": key, "slabs": slabs, "k": k, "rate": c["rate"], "tile": c.get("tile", 0),
                       "errors": c.get("errors", {})})
    # shared workspace of the batch within the budget: split the largest windows
    while O.oocs_batch_query(out) > budget:
        i = max(range(len(out)), key=lambda j: int(out[j].nx) * int(out[j].ny) * int(out[j].slab_planes))
        slabs = 2 * -(-int(out[i].nz) // int(out[i].slab_planes))
        t = with_plan(out[i], slabs, int(out[i].temporal_depth), int(out[i].rate_bits), int(out[i].step_tile))
        if t is None:
            raise O.OOCSError(2, "the batch does not fit the budget")
        out[i] = t
        report[i]["slabs"] = slabs
    if cache_path:
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    return out, {"problems": report, "candidates_timed": timed, "classes": len({r["class"] for r in report})}
