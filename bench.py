#!/usr/bin/env python
"""Benchmark of the compressed out-of-core stencil sweep on one GB300 per rank.

Workload (the metric's configuration): 25-point 8th-order acoustic wave
(leapfrog), FP32, 512^3 grid, dx = 10 m, dt = 0.8 ms, seeded 8-layer velocity
model 1500-4500 m/s with +-5 % noise, 15 Hz Ricker source at the centre,
device budget 4 GiB, 8 z-slabs of 64 planes, temporal blocking depth k = 4,
fixed-rate codec at 16 bits/value, single working buffer (Sec. 5).  The
read-only model m is kept on the device (decoded once from its rate-16 store,
inside the budget), so u and u_prev stream; ``compare`` also times the
paper's dataflow, which streams m with every slab visit.

One bench step = one oocs_step(100) from rest (the host stores are reset to
the compressed initial state and the time index to 0 before each, untimed):
100 time steps = 25 sweeps over the 8 slabs, every slab's u and u_prev
streamed host->GPU, decoded, advanced 4 steps, encoded and streamed back.  ``value`` = interior point-updates / s (Gpoint-updates/s) with
the fields already in the compressed host store (pinned host memory: where
the method keeps them); ``e2e`` adds the conversion from and to raw FP32 host
arrays through oocs_compress / oocs_decompress.

--impl reference times the CPU oracle (FP64, OpenMP on the host cores) on a
bounded sample of the same workload.  Multi-GPU: independent replicas, one per
rank (the method is single-GPU; no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "out-of-core Gpoint-updates/s at stated max error; % of HBM/host-link roofline"
UNIT = "Gpoint-updates/s"
N = 512
STEPS_PER_CALL = 100
K_DEPTH = 4
SLAB = 64
BUDGET = 4 << 30
RATE = 16
RO_RESIDENT = 1  # keep m on the device (oocs_desc.readonly_resident)
WAVE_BYTES_PER_POINT = 16  # read u, u_prev, m; write u_next (FP32)
WORKLOAD = "wave25_512cubed_100steps_8slabs_k4_rate16_swb_m_resident"
# DRAM bytes (read + write) per updated point of the wave step kernel from one ncu
# capture of a 512x512x80 launch, the window size of the sweep's balanced step
# launches; scaled to a launch by its points.  Set to None whenever the kernel
# changes.
STEP_TRAFFIC_B_PER_POINT = 15.78


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rate", type=int, default=RATE)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-true-ooc", action="store_true")
    ap.add_argument("--profile-run", choices=["sweep", "kernels"], default=None,
                    help="run only the region to capture under ncu --profile-from-start off: "
                         "'sweep' = one oocs_step(100) of the workload; 'kernels' = one launch each "
                         "of the wave step, encode and decode kernels on a 512x512x192 grid, then "
                         "one wave step on a 512x512x80 grid")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def guarded(fn, *args):
    """Run one of the sections measured after the headline; a failure (say a
    host with too little free memory for a 134 GB pinned store) is reported
    in its place instead of losing the whole line."""
    try:
        return fn(*args)
    except Exception as e:  # noqa: BLE001 - any failure of an optional section
        import torch
        if torch.cuda.is_available():
            torch.cuda.empty_cache()
        return {"error": f"{type(e).__name__}: {e}"[:400]}


def max_over_ranks(torch, value: float, device) -> float:
    """The largest of every rank's value (the slowest replica's time)."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(points_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job Gpoint-updates/s of `world` replicas, each updating
    points_per_rank points, timed by the slowest one."""
    return points_per_rank * world / (ms_max / 1e3) / 1e9


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def interior_points(n=N, r=4):
    return (n - 2 * r) ** 3


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        self.file.close()
        os.unlink(self.file.name)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                power.append(float(r[3]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        srt = sorted(sm)
        return {"sm_mhz": srt[len(srt) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def link_bandwidth(torch, dev):
    """Pinned host <-> device copy bandwidth (GB/s, best of 5, 1 GiB), each way and both at once."""
    n = 1 << 30
    h1 = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    h2 = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    d1 = torch.empty(n, dtype=torch.uint8, device=dev)
    d2 = torch.empty(n, dtype=torch.uint8, device=dev)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def timed(fn):
        best = 1e30
        for _ in range(5):
            torch.cuda.synchronize(dev)
            t = time.perf_counter()
            fn()
            torch.cuda.synchronize(dev)
            best = min(best, time.perf_counter() - t)
        return best

    def h2d():
        with torch.cuda.stream(s1):
            d1.copy_(h1, non_blocking=True)

    def d2h():
        with torch.cuda.stream(s2):
            h2.copy_(d2, non_blocking=True)

    def both():
        h2d()
        d2h()

    t_h2d, t_d2h, t_both = timed(h2d), timed(d2h), timed(both)
    del h1, h2, d1, d2
    return {"h2d_GBs": n / t_h2d / 1e9, "d2h_GBs": n / t_d2h / 1e9,
            "bidir_GBs": 2 * n / t_both / 1e9}


def make_inputs(total_steps):
    import numpy as np

    import synthetic
    shape = (N, N, N)
    m = synthetic.wave_model(shape)
    w = synthetic.ricker(total_steps)
    cz, cy, cx = synthetic.centre(shape)
    z = np.zeros(shape, np.float32)
    return m, w, (cx, cy, cz), z


def wave_desc(P, rate, wb=1, ro=RO_RESIDENT, codec=0):
    import synthetic
    return P.make_desc(N, N, N, P.OOCS_WAVE, synthetic.wave_star_coef(), BUDGET, rate_bits=rate,
                       temporal_depth=K_DEPTH, slab_planes=SLAB, working_buffers=wb, readonly_resident=ro,
                       codec=codec)


def open_ctx(P, torch, rate, wb, inputs, ro=RO_RESIDENT, codec=0):
    m, w, src, z = inputs
    st = P.OutOfCoreStencil(wave_desc(P, rate, wb, ro, codec))
    pin = {}
    for name, arr in (("z", z), ("m", m)):
        t = torch.empty(arr.shape, dtype=torch.float32, pin_memory=True)
        t.numpy()[...] = arr
        pin[name] = t
    st.compress(P.OOCS_FIELD_U, pin["z"])
    st.compress(P.OOCS_FIELD_U_PREV, pin["z"])
    st.compress(P.OOCS_FIELD_M, pin["m"])
    st.set_source(src[0], src[1], src[2], w)
    st.synchronize(600.0)
    return st, pin


def timed_calls(torch, st, k, snap, calls=STEPS_PER_CALL):
    """k runs of the workload, each from rest: the host stores are restored to
    the initial compressed state and the time index to 0 (untimed), then one
    oocs_step(calls) is bracketed by CUDA events on stream 0 (the context joins
    its three streams into stream 0 at the start and end of every call).
    Returns the summed device milliseconds."""
    s0 = st.streams[0]
    total = 0.0
    for _ in range(k):
        st.restore_stores(snap, 0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s0)
        st.step(calls)
        e1.record(s0)
        st.synchronize(600.0)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    return total


SAMPLE_PLANES = 128


def cpu_oracle_sample(inputs, rate=RATE, planes=SAMPLE_PLANES):
    """One slab-sized sample of the workload on the CPU oracle: 4 FP64 leapfrog
    steps (one sweep's depth) on a 512 x 512 x `planes` sub-grid of the model
    (Dirichlet shell included) plus the reference codec round trip of u,
    u_prev and m at `rate`.  Returns (seconds, interior points updated, threads)."""
    import numpy as np

    import oracle
    import synthetic
    m, w, src, z = inputs
    z0 = (N - planes) // 2
    mm = np.ascontiguousarray(m[z0:z0 + planes])
    shape = mm.shape
    rng = np.random.default_rng(0)
    u = np.zeros(shape, np.float64)
    up = np.zeros(shape, np.float64)
    u[4:-4, 4:-4, 4:-4] = rng.standard_normal((planes - 8, N - 8, N - 8)) * 1e-3
    t = time.perf_counter()
    u, up = oracle.wave_run(u, up, mm, synthetic.wave_star_coef(), K_DEPTH,
                            src=(planes // 2, src[1], src[0]), w=w)
    for f in (u, up, mm):
        oracle.decode_field(oracle.encode_field(np.asarray(f, np.float32), rate), shape, rate)
    dt = time.perf_counter() - t
    return dt, (planes - 8) * (N - 8) ** 2 * K_DEPTH, oracle.threads()


def base_line(args, world):
    peaks, _ = measured_peaks()
    return {"metric": METRIC, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [N, N, N], "stencil": "25-point star, r=4",
                       "time_steps_per_step": STEPS_PER_CALL, "slabs": N // SLAB,
                       "slab_planes": SLAB, "temporal_depth": K_DEPTH, "rate_bits": args.rate,
                       "working_buffers": 1, "device_budget_bytes": BUDGET,
                       "model_m": "device-resident (decoded once from its store)" if RO_RESIDENT
                       else "streamed with every slab visit",
                       "l2": "inputs larger than L2 (one 512^3 FP32 field = 537 MB)",
                       "parallelism": f"replicas{world}"}}


# ----------------------------------------------------------------- ours --

def run_ours(args):
    import numpy as np
    import torch

    import paper_2204_11315_gb300 as P
    rank, world, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    P.lib()
    peaks, peak_src = measured_peaks()
    total_steps = (args.warmup + args.steps + 2) * STEPS_PER_CALL
    inputs = make_inputs(total_steps)
    link = link_bandwidth(torch, dev)

    # ---- main timed region: oocs_step from the compressed host store
    st, pin = open_ctx(P, torch, args.rate, 1, inputs)
    snap = st.snapshot_stores()
    # live timing of the dominant kernel class only (two event records per
    # step-kernel launch); the warm-up creates the event pool
    st.set_profiling(P.OOCS_PROF_STEP)
    timed_calls(torch, st, args.warmup, snap)
    before = st.stats()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    ms = timed_calls(torch, st, args.steps, snap)
    clk = clocks.stop()
    after = st.stats()
    ms = max_over_ranks(torch, ms, dev)
    value = replica_throughput(interior_points() * STEPS_PER_CALL * args.steps, world, ms)

    d = {k: after[k] - before[k] for k in ("h2d_bytes", "d2h_bytes", "kernel_launches",
                                            "slabs_done", "passes_done")}
    cls = {c: {k: after[c][k] - before[c][k] for k in ("launches", "units", "device_ms")}
           for c in ("load", "step", "store")}
    hbm_peak = float(peaks["hbm_gbs"])
    step_bytes = cls["step"]["units"] * WAVE_BYTES_PER_POINT
    step_gbs = step_bytes / (cls["step"]["device_ms"] / 1e3) / 1e9 if cls["step"]["device_ms"] else None
    roofline = {"bound": "hbm", "kernel": "k_star_step<4,wave>",
                "achieved": step_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": (step_gbs / hbm_peak) if step_gbs else None,
                "traffic": (STEP_TRAFFIC_B_PER_POINT * cls["step"]["units"] / max(cls["step"]["launches"], 1)
                            if STEP_TRAFFIC_B_PER_POINT else None),
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of a 512x512x80 "
                                  "launch, scaled by points per launch",
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_bytes_per_launch": step_bytes / max(cls["step"]["launches"], 1),
                "avg_launch_ms": cls["step"]["device_ms"] / max(cls["step"]["launches"], 1)}
    # binding roofline of the whole sweep: HBM algorithmic bytes vs host link.
    # Per sweep and grid value of a streamed field: in = H2D write (c) + decode
    # read (c) + write (4); out = encode read (4) + write (c) + D2H read (c);
    # c = 4 uncompressed (the decode / encode are copies).
    n_all = N ** 3
    c_bytes = args.rate / 8.0 if args.rate else 4.0
    passes = d["passes_done"]
    f_in = st.plan.fields_in
    hbm_alg = STEPS_PER_CALL * args.steps * interior_points() * WAVE_BYTES_PER_POINT \
        + passes * n_all * (f_in * (2 * c_bytes + 4) + 2 * (4 + 2 * c_bytes))
    t_hbm = hbm_alg / (hbm_peak * 1e9)
    t_h2d = d["h2d_bytes"] / (link["h2d_GBs"] * 1e9)
    t_d2h = d["d2h_bytes"] / (link["d2h_GBs"] * 1e9)
    t_bi = (d["h2d_bytes"] + d["d2h_bytes"]) / (link["bidir_GBs"] * 1e9)
    t_roof = max(t_hbm, t_h2d, t_d2h, t_bi)
    sweep_roofline = {"t_roof_ms": t_roof * 1e3, "t_measured_ms": ms / world if world else ms,
                      "frac": t_roof / (ms / 1e3),
                      "binding": ["hbm", "h2d", "d2h", "bidir"][[t_hbm, t_h2d, t_d2h, t_bi].index(t_roof)],
                      "t_hbm_ms": t_hbm * 1e3, "t_h2d_ms": t_h2d * 1e3, "t_d2h_ms": t_d2h * 1e3,
                      "t_bidir_ms": t_bi * 1e3, "hbm_algorithmic_bytes": hbm_alg,
                      "h2d_bytes": d["h2d_bytes"], "d2h_bytes": d["d2h_bytes"], "link": link}
    # per-class device time from one extra call with every class timed (not in `value`)
    st.set_profiling(P.OOCS_PROF_LOAD | P.OOCS_PROF_STEP | P.OOCS_PROF_STORE)
    b2 = st.stats()
    timed_calls(torch, st, 1, snap)
    a2 = st.stats()
    kernels = {}
    for c in ("load", "step", "store"):
        k = {q: a2[c][q] - b2[c][q] for q in ("launches", "units", "device_ms")}
        k["avg_ms"] = k["device_ms"] / max(k["launches"], 1)
        kernels[c] = k
    kernels["note"] = "one extra oocs_step(100) with all classes event-timed; ms per call"
    st.set_profiling(0)
    # what binds the call as measured: the serial chain of kernels (one working
    # buffer: the visits' kernels never overlap) or the host-link floor
    chain_ms = sum(kernels[c]["device_ms"] for c in ("load", "step", "store"))
    t_call = ms / world if world else ms
    sweep_roofline["kernel_chain_ms_per_call"] = chain_ms
    sweep_roofline["link_floor_ms_per_call"] = t_roof * 1e3 / args.steps
    sweep_roofline["measured_binding"] = ("kernel chain" if chain_ms > t_roof * 1e3 / args.steps
                                          else "host link")
    sweep_roofline["ms_per_call"] = t_call / args.steps

    # ---- e2e: raw FP32 host arrays in, result back in host memory
    e2e_ms = []
    res_host = st.pinned_field()
    for i in range(max(2, min(args.steps, 3)) + 1):
        s0 = st.streams[0]
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        st.set_time(0)
        e0.record(s0)
        st.compress(P.OOCS_FIELD_U, pin["z"])
        st.compress(P.OOCS_FIELD_U_PREV, pin["z"])
        st.compress(P.OOCS_FIELD_M, pin["m"])
        st.step(STEPS_PER_CALL)
        st.decompress(P.OOCS_FIELD_U, res_host)
        e1.record(s0)
        st.synchronize(600.0)
        e1.synchronize()
        if i > 0:  # first round is a warm-up
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_step_ms = float(np.median(e2e_ms))
    raw = n_all * 4
    comp = n_all * args.rate // 8 if args.rate else raw
    per_call_h2d = d["h2d_bytes"] / args.steps
    per_call_d2h = d["d2h_bytes"] / args.steps
    e2e = {"value": interior_points() * STEPS_PER_CALL * world / (e2e_step_ms / 1e3) / 1e9,
           "unit": UNIT, "ms_per_step": e2e_step_ms,
           "h2d_bytes_per_step": int(3 * raw + per_call_h2d + comp),
           "d2h_bytes_per_step": int(3 * comp + per_call_d2h + raw),
           "note": "oocs_compress(u, u_prev, m from pinned FP32) + oocs_step(100) + "
                   "oocs_decompress(u to pinned FP32), CUDA events on stream 0"}
    st.close()
    del st, pin
    torch.cuda.empty_cache()

    # The sections below characterise the method on one GPU; replicas under
    # torchrun (N > 1) report the headline only (the true out-of-core run
    # alone pins up to 134 GB of host memory per process).
    single = world == 1

    # ---- accuracy at the stated configuration: 100 steps from rest
    accuracy = guarded(check_accuracy, P, torch, dev, args.rate, inputs) if single else None

    # ---- the adjoint workload (gradient of a receiver misfit)
    adjoint = guarded(run_adjoint, P, torch, dev, float(peaks["hbm_gbs"])) \
        if single and not args.no_adjoint else None

    # ---- the batched workload (many independent problems, one pipeline)
    batched = guarded(run_batched, P, torch, dev) if single and not args.no_batch else None

    # ---- a grid larger than the device budget by far (two 134 GB arrays)
    true_ooc = guarded(run_true_out_of_core, P, torch, dev) if single and not args.no_true_ooc else None

    # ---- comparison: uncompressed streaming, SWB and classic (Fig. 9, Fig. 11 analogues)
    compare = guarded(run_compare, P, torch, dev, args, inputs, peaks, value, world) \
        if single and not args.no_compare else None

    line = base_line(args, world)
    line.update({"value": value, "ms_per_step": ms / args.steps, "dtype": "f32",
                 "gpu_launches": int(d["kernel_launches"]), "e2e": e2e, "roofline": roofline,
                 "clocks": clk, "sweep_roofline": sweep_roofline, "kernels": kernels,
                 "accuracy": accuracy, "compare": compare, "adjoint": adjoint, "batched": batched,
                 "true_out_of_core": true_ooc,
                 "workspace_bytes": P.oocs_query(wave_desc(P, args.rate)).workspace_bytes})
    if rank == 0 and not args.no_cpu_baseline:
        tot, pts_cpu = 0.0, 0
        for _ in range(3):
            dt, npts, cores = cpu_oracle_sample(inputs, args.rate)
            tot += dt
            pts_cpu += npts
        line["cpu_baseline"] = {"value": pts_cpu / tot / 1e9, "unit": UNIT, "cores": cores,
                                "kind": "oracle", "seconds": tot,
                                "sample": f"3 x (4 FP64 leapfrog steps on a 512x512x{SAMPLE_PLANES} "
                                          "sub-grid of the model + reference codec round trip of u, "
                                          f"u_prev, m at rate {args.rate})"}
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


BATCH_N, BATCH_STEPS, BATCH_BUDGET, BATCH_TOL = 64, 50, 8 << 30, 1e-4


def run_batched(P, torch, dev):
    """64 independent problems (heat and wave alternating, every side seeded
    in 64..384 by 16), 50 steps each, one shared 8 GiB workspace, (slabs, k,
    rate) autotuned per size class at the rate-16 tolerance.  Timed three ways
    on the same problems from the same compressed state: each problem alone
    (its own context, one after another), one batch step through the shared
    pipeline, and a replay of the batch step captured as a CUDA graph."""
    import numpy as np

    import synthetic
    from paper_2204_11315_gb300 import autotune
    t0 = time.time()
    descs = []
    for sc, (nz, ny, nx) in synthetic.batch_shapes(BATCH_N):
        if sc == "heat":
            descs.append(P.make_desc(nx, ny, nz, P.OOCS_HEAT, synthetic.heat_star_coef(0.1), BATCH_BUDGET))
        else:
            descs.append(P.make_desc(nx, ny, nz, P.OOCS_WAVE, synthetic.wave_star_coef(), BATCH_BUDGET))
    cache = os.path.join(tempfile.gettempdir(), f"oocs_autotune_{os.getpid()}.json")
    tuned, report = autotune.tune(descs, BATCH_TOL, BATCH_BUDGET, cache)
    t_tune = time.time() - t0
    b = P.OutOfCoreBatch(tuned)
    for i, (bp, d) in enumerate(zip(b.problems, tuned)):
        shape = (d.nz, d.ny, d.nx)
        if d.scheme == P.OOCS_HEAT:
            bp.compress(P.OOCS_FIELD_U, synthetic.uniform_field(shape, 100 + i))
        else:
            u0 = synthetic.wave_initial(shape, 200 + i)
            bp.compress(P.OOCS_FIELD_U, u0)
            bp.compress(P.OOCS_FIELD_U_PREV, u0)
            bp.compress(P.OOCS_FIELD_M, synthetic.wave_model(shape))
        bp.synchronize(600.0)
    snaps = [bp.snapshot_stores() for bp in b.problems]

    def restore():
        for bp, sn in zip(b.problems, snaps):
            bp.restore_stores(sn, 0)

    def timed(fn, stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        b.synchronize(600.0)
        e1.synchronize()
        return e0.elapsed_time(e1)

    s0 = b.streams[0]
    restore()
    b.step(BATCH_STEPS)  # warm-up
    b.synchronize(600.0)
    restore()
    l0 = sum(bp.stats()["kernel_launches"] for bp in b.problems)
    ms_batch = timed(lambda: b.step(BATCH_STEPS), s0)
    launches_per_step = sum(bp.stats()["kernel_launches"] for bp in b.problems) - l0
    after_batch = [[s.clone() for s in bp.stores] for bp in b.problems]
    restore()
    b.capture(BATCH_STEPS)
    b.launch()  # warm-up replay
    b.synchronize(600.0)
    restore()
    ms_graph = timed(b.launch, s0)
    # each problem alone: a context of its own over the same host stores
    restore()
    ms_alone, ws_alone = 0.0, []
    for bp, d in zip(b.problems, tuned):
        st = P.OutOfCoreStencil(d, stores=bp.stores)
        try:
            ws_alone.append(st.plan.workspace_bytes)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st.streams[0])
            st.step(BATCH_STEPS)
            e1.record(st.streams[0])
            st.synchronize(600.0)
            e1.synchronize()
            ms_alone += e0.elapsed_time(e1)
        finally:
            st.close()
    # every problem ends with the same host store bytes either way
    identical = all(torch.equal(a, s) for ab, bp in zip(after_batch, b.problems) for a, s in zip(ab, bp.stores))
    b.close()
    pts = sum((int(d.nx) - 2 * d.radius) * (int(d.ny) - 2 * d.radius) * (int(d.nz) - 2 * d.radius)
              for d in tuned) * BATCH_STEPS
    gpts = lambda ms: pts / (ms / 1e3) / 1e9
    rates, slabs, depths = {}, {}, {}
    for r in report["problems"]:
        rates[r["rate"]] = rates.get(r["rate"], 0) + 1
        slabs[r["slabs"]] = slabs.get(r["slabs"], 0) + 1
        depths[r["k"]] = depths.get(r["k"], 0) + 1
    return {"workload": f"{BATCH_N}_problems_heat_wave_sides64to384_{BATCH_STEPS}steps_budget8GiB_tol1e-4",
            "unit": UNIT, "value": gpts(ms_graph),
            "graph_replay": {"value": gpts(ms_graph), "ms": ms_graph},
            "batch_step": {"value": gpts(ms_batch), "ms": ms_batch},
            "each_alone": {"value": gpts(ms_alone), "ms": ms_alone},
            "speedup_graph_vs_alone": ms_alone / ms_graph,
            "stores_identical_batch_vs_alone": identical,
            "interior_point_updates": pts, "workspace_bytes": P.oocs_batch_query(tuned),
            "sum_of_alone_workspaces": int(sum(ws_alone)), "kernel_launches_per_batch_step": launches_per_step,
            "tuning": {"seconds": t_tune, "classes": report["classes"],
                       "candidates_timed": report["candidates_timed"], "rates": rates, "slabs": slabs,
                       "temporal_depths": depths}}


OOC_SHAPE, OOC_STEPS, OOC_K, OOC_BUDGET, OOC_SEED = (5120, 2560, 2560), 20, 4, 16 << 30, 31


def ooc_samples(shape, n=64, seed=32, margin=24):
    """n seeded interior points (z, y, x) at least `margin` from every face."""
    import synthetic
    u = synthetic.uniform01(seed, 3 * n).reshape(n, 3)
    return [tuple(int(margin + u[i, a] * (shape[a] - 2 * margin)) for a in range(3)) for i in range(n)]


def run_compare(P, torch, dev, args, inputs, peaks, value, world):
    """Comparison on the same GPU (Fig. 9, Fig. 11 analogues): uncompressed
    streaming, SWB and classic, other rates and the block quantiser with their
    accuracy, the codec kernels alone, and the call replayed as a CUDA graph."""
    compare = {}
    ref = incore_reference(P, torch, dev, inputs)
    for name, rate, wb, ro, codec in (("uncompressed_swb", 0, 1, RO_RESIDENT, 0),
                                      ("uncompressed_classic", 0, 3, RO_RESIDENT, 0),
                                      (f"rate{args.rate}_classic", args.rate, 3, RO_RESIDENT, 0),
                                      ("rate8_swb", 8, 1, RO_RESIDENT, 0), ("rate12_swb", 12, 1, RO_RESIDENT, 0),
                                      (f"rate{args.rate}_swb_m_streamed", args.rate, 1, 0, 0),
                                      ("uncompressed_swb_m_streamed", 0, 1, 0, 0),
                                      ("uncompressed_classic_m_streamed", 0, 3, 0, 0),
                                      # the simpler codec of the Sec. 7 (1) comparison
                                      ("quant12_swb", 12, 1, RO_RESIDENT, 1),
                                      ("quant16_swb", 16, 1, RO_RESIDENT, 1),
                                      ("quant20_swb", 20, 1, RO_RESIDENT, 1)):
        st, pin = open_ctx(P, torch, rate, wb, inputs, ro, codec)
        snap_u = st.snapshot_stores()
        timed_calls(torch, st, 1, snap_u)
        k = 2
        cms = timed_calls(torch, st, k, snap_u)
        compare[name] = {"value": interior_points() * STEPS_PER_CALL * k / (cms / 1e3) / 1e9,
                         "workspace_bytes": st.plan.workspace_bytes}
        st.close()
        del st, pin, snap_u
        torch.cuda.empty_cache()
        if rate and wb == 1 and ro == RO_RESIDENT:  # accuracy of each codec and rate
            compare[name]["rel_l2_vs_uncompressed_fp32"] = check_accuracy(
                P, torch, dev, rate, inputs, codec, ref)["rel_l2_vs_uncompressed_fp32"]
    del ref
    compare["codec_kernels"] = codec_kernel_rates(P, torch, dev, args.rate, float(peaks["hbm_gbs"]))
    # the same workload as a batch of one, its 100-step call replayed as one CUDA graph
    m, w, src, z = inputs
    b = P.OutOfCoreBatch([wave_desc(P, args.rate)])
    bp = b.problems[0]
    pin = {}
    for name, arr in (("z", z), ("m", m)):
        t = torch.empty(arr.shape, dtype=torch.float32, pin_memory=True)
        t.numpy()[...] = arr
        pin[name] = t
    bp.compress(P.OOCS_FIELD_U, pin["z"])
    bp.compress(P.OOCS_FIELD_U_PREV, pin["z"])
    bp.compress(P.OOCS_FIELD_M, pin["m"])
    bp.set_source(src[0], src[1], src[2], w)
    b.synchronize(600.0)
    snap_g = bp.snapshot_stores()
    b.capture(STEPS_PER_CALL)
    gms = []
    for i in range(3):
        bp.restore_stores(snap_g, 0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(b.streams[0])
        b.launch()
        e1.record(b.streams[0])
        b.synchronize(600.0)
        e1.synchronize()
        if i:
            gms.append(e0.elapsed_time(e1))
    compare[f"rate{args.rate}_swb_graph_replay"] = {
        "value": interior_points() * STEPS_PER_CALL * len(gms) / (sum(gms) / 1e3) / 1e9,
        "note": "the 100-step call captured once (oocs_batch_capture) and replayed"}
    b.close()
    del b, bp, pin, snap_g
    torch.cuda.empty_cache()
    compare["speedup_compressed_vs_uncompressed"] = value / world / compare["uncompressed_swb"]["value"]
    compare["speedup_compressed_vs_uncompressed_m_streamed"] = \
        compare[f"rate{args.rate}_swb_m_streamed"]["value"] / compare["uncompressed_swb_m_streamed"]["value"]
    # the paper's memory comparison (Sec. 6.2): compressed SWB against
    # uncompressed classic, both streaming m as the paper does
    compare["memory_reduction_vs_uncompressed_classic"] = \
        1.0 - compare[f"rate{args.rate}_swb_m_streamed"]["workspace_bytes"] \
        / compare["uncompressed_classic_m_streamed"]["workspace_bytes"]
    compare["paper_v100"] = {"speedup": 1.1, "memory_reduction": 0.330,
                             "source": "Sec. 6.1 and Sec. 6.2 (V100-PCIe, FP64, context only)"}
    return compare


def run_true_out_of_core(P, torch, dev):
    """7-point heat, FP32, 2560 x 2560 x 5120 (one field of 134 GB), seeded
    U[0,1), 20 steps, k = 4, a 16 GiB device budget, rate 16 and uncompressed.
    The host store is exact-size pinned memory (67 GB compressed, 134 GB raw),
    filled from planes drawn on the GPU (oocs_compress_device); one
    oocs_step(20) is timed per rate.  Accuracy: the rate-16 result against the
    uncompressed streamed result (bit-exact to an in-core run by the tests) at
    64 seeded points."""
    import numpy as np

    import synthetic
    nz, ny, nx = OOC_SHAPE
    plane = nx * ny
    samples = ooc_samples(OOC_SHAPE)
    out, values = {}, {}
    for rate in (16, 0):
        desc = P.make_desc(nx, ny, nz, P.OOCS_HEAT, synthetic.heat_star_coef(0.1), OOC_BUDGET, rate_bits=rate,
                           temporal_depth=OOC_K)
        plan = P.oocs_query(desc)
        t0 = time.time()
        host = P.HostBuffer(plan.host_store_bytes)
        t_pin = time.time() - t0
        st = P.OutOfCoreStencil(desc, stores=[host.tensor()])
        try:
            t0 = time.time()
            chunk = 64
            for z0 in range(0, nz, chunk):
                z1 = min(z0 + chunk, nz)
                f = synthetic.uniform_field_planes_torch(OOC_SHAPE, OOC_SEED, z0, z1, device=dev)
                torch.cuda.synchronize(dev)  # drawn on torch's stream; the context reads on its own
                P.oocs_compress_device(st.ctx, P.OOCS_FIELD_U, f.data_ptr(), z0, z1 - z0)
                st.synchronize(600.0)
                del f
            t_fill = time.time() - t0
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st.streams[0])
            st.step(OOC_STEPS)
            e1.record(st.streams[0])
            st.synchronize(3600.0)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            stats = st.stats()
            buf = torch.empty((4, ny, nx), dtype=torch.float32, device=dev)
            vals = []
            for (z, y, x) in samples:
                P.oocs_decompress_device(st.ctx, P.OOCS_FIELD_U, buf.data_ptr(), z // 4 * 4, 4)
                st.synchronize(600.0)
                vals.append(float(buf[z % 4, y, x]))
            values[rate] = np.array(vals, np.float64)
            pts = (nx - 2) * (ny - 2) * (nz - 2) * OOC_STEPS
            out[f"rate{rate}"] = {"value": pts / (ms / 1e3) / 1e9, "unit": UNIT, "ms": ms,
                                  "slabs": plan.num_slabs, "slab_planes": plan.slab_planes,
                                  "workspace_bytes": plan.workspace_bytes,
                                  "host_store_bytes": plan.host_store_bytes,
                                  "h2d_bytes": stats["h2d_bytes"], "d2h_bytes": stats["d2h_bytes"],
                                  "pin_seconds": t_pin, "fill_seconds": t_fill}
        finally:
            st.close()
            host.close()
            torch.cuda.empty_cache()
    err = values[16] - values[0]
    out["workload"] = "heat7_2560x2560x5120_20steps_k4_budget16GiB"
    out["grid_bytes_fp32"] = nx * ny * nz * 4
    out["note"] = ("out of core by the device budget (16 GiB); the field alone is 134 GB and the "
                   "GB300 has 284 GB of HBM")
    out["speedup_rate16_vs_uncompressed"] = out["rate0"]["ms"] / out["rate16"]["ms"]
    out["accuracy_rate16_vs_uncompressed"] = {
        "samples": len(samples), "rel_l2": float(np.linalg.norm(err) / np.linalg.norm(values[0])),
        "max_abs": float(np.abs(err).max()), "stated_max_rel_l2": 1e-4}
    return out


ADJ_N, ADJ_STEPS, ADJ_EVERY, ADJ_RATE = 256, 400, 10, 16


def run_adjoint(P, torch, dev, hbm_peak):
    """dJ/dv of J = 1/2 sum_n |u^n(z = 8) - d^n|^2 on a 256^3 wave grid, 400
    steps, (u^n, u^(n-1)) checkpointed every 10 steps at 16 bits/value, through
    the autograd Function (one forward + one backward call of the library's
    driver).  Target data d from a smooth +5 % velocity bump.  Also the live
    bandwidth of the adjoint-step kernel (24 B per point: read m lam^(n+1)
    (stencil), lam^(n+1), lam^(n+2), m; write lam^n, m lam^n)."""
    import numpy as np

    import paper_2204_11315_gb300.adjoint as A
    import synthetic
    n = ADJ_N
    shape = (n, n, n)
    w = synthetic.ricker(ADJ_STEPS)
    v = synthetic.layered_velocity(shape, seed=4).astype(np.float32)
    z, y, x = np.ogrid[:n, :n, :n]
    bump = np.exp(-((x - 140.0) ** 2 + (y - 120.0) ** 2 + (z - 40.0) ** 2) / 400.0)
    v_true = (v * (1.0 + 0.05 * bump)).astype(np.float32)
    prob = A.WaveProblem(shape=shape, dt=synthetic.WAVE_DT, dx=synthetic.WAVE_DX,
                         coef=synthetic.wave_star_coef(), src_xyz=(n // 2, n // 2, 32), wavelet=w, zr=8,
                         nsteps=ADJ_STEPS, checkpoint_every=ADJ_EVERY, rate=ADJ_RATE)
    d = A.receiver_data(torch.from_numpy(v_true).to(dev), prob)
    v_dev = torch.from_numpy(v).to(dev)
    times = []
    for rep_i in range(3):
        vt = v_dev.clone().requires_grad_(True)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize(dev)
        e[0].record()
        J = A.wave_misfit(vt, d, prob)
        e[1].record()
        J.backward()
        e[2].record()
        torch.cuda.synchronize(dev)
        if rep_i:  # the first is a warm-up
            times.append((e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])))
        grad_norm = float(vt.grad.norm())
    fwd = float(np.median([t[0] for t in times]))
    bwd = float(np.median([t[1] for t in times]))
    interior = (n - 8) ** 3
    # live bandwidth of the adjoint-step kernel on the same grid
    desc = prob.desc()
    f = [torch.zeros(shape, device=dev) for _ in range(4)]
    m = torch.full(shape, 0.1, device=dev)
    s = torch.cuda.current_stream(dev).cuda_stream
    reps = 40
    for _ in range(3):
        P.oocs_adjoint_step(desc, f[0].data_ptr(), f[1].data_ptr(), f[2].data_ptr(), f[3].data_ptr(),
                            m.data_ptr(), 0, -1, s)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(reps):
        a, b = (2, 3) if i % 2 == 0 else (3, 2)
        P.oocs_adjoint_step(desc, f[0].data_ptr(), f[1].data_ptr(), f[a].data_ptr(), f[b].data_ptr(),
                            m.data_ptr(), 0, -1, s)
    e1.record()
    torch.cuda.synchronize(dev)
    k_ms = e0.elapsed_time(e1) / reps
    k_gbs = 24 * n ** 3 / (k_ms / 1e3) / 1e9
    # the same gradient out of core: slab sweeps of 64 planes (4 slabs), m and
    # dJ/dm resident, lam, the checkpoints and the recomputed states in pinned
    # host memory through the codec; a warm-up call, then one timed call
    # (its pinned buffers come from PyTorch's host allocator cache, as in an
    # optimisation loop)
    g_in = vt.grad.detach().clone()
    del f, m
    oprob = A.WaveProblem(**{**prob.__dict__, "device_budget": 2 << 30, "slab_planes": 64, "_desc": None})
    for rep_i in range(2):
        vt = v_dev.clone().requires_grad_(True)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize(dev)
        e[0].record()
        J_oc = A.wave_misfit(vt, d, oprob)
        e[1].record()
        J_oc.backward()
        e[2].record()
        torch.cuda.synchronize(dev)
    oc_fwd, oc_bwd = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
    ooc = {"slabs": 4, "slab_planes": 64, "device_budget": 2 << 30,
           "ms_per_gradient": oc_fwd + oc_bwd, "forward_ms": oc_fwd, "backward_ms": oc_bwd,
           "value": interior * ADJ_STEPS / ((oc_fwd + oc_bwd) / 1e3) / 1e9,
           "misfit_rel_diff_vs_in_core": abs(float(J_oc.detach()) - float(J.detach())) / float(J.detach()),
           "grad_rel_l2_vs_in_core": float((vt.grad - g_in).norm() / g_in.norm())}
    return {"workload": f"wave25_{n}cubed_{ADJ_STEPS}steps_misfit_gradient_checkpoints{ADJ_EVERY}_rate{ADJ_RATE}",
            "value": interior * ADJ_STEPS / ((fwd + bwd) / 1e3) / 1e9,
            "unit": "Gpoint-steps/s of the whole gradient (forward + backward)",
            "ms_per_gradient": fwd + bwd, "forward_ms": fwd, "backward_ms": bwd,
            "grad_norm": grad_norm, "misfit": float(J.detach()),
            "workspace_bytes": prob.workspace_bytes(),
            "roofline": {"bound": "hbm", "kernel": "k_star_step<4,adjoint>", "achieved": k_gbs, "peak": hbm_peak,
                         "unit": "GB/s", "frac": k_gbs / hbm_peak, "bytes_per_point": 24,
                         "avg_launch_ms": k_ms, "grid": [n, n, n]},
            "out_of_core": ooc}


def codec_kernel_rates(P, torch, dev, rate, hbm_peak, reps=10):
    """Live rates of the codec kernels alone: encode and decode of a 512 x 512
    x 192 field (201 MB FP32, above the 129 MB L2) at `rate`, each codec,
    CUDA events over `reps` launches after a warm-up.  Algorithmic bytes per
    value: 4 (FP32) + rate/8 (compressed)."""
    nz = 192
    noise = torch.randn((nz, N, N), device=dev) * 1e-3
    zero = torch.zeros_like(noise)  # the sweep's fields are mostly all-zero blocks (a point source from rest)
    g = torch.empty_like(noise)
    blocks = torch.empty(N * N * nz * rate // 32, dtype=torch.int32, device=dev)
    s = torch.cuda.current_stream(dev).cuda_stream
    vals = N * N * nz
    out = {}
    for name, codec, f in (("transform", 0, noise), ("quant", 1, noise), ("transform_zero_field", 0, zero)):
        enc = lambda: P.oocs_encode_device(f.data_ptr(), N, N, nz, rate, blocks.data_ptr(), s, codec=codec)
        dec = lambda: P.oocs_decode_device(blocks.data_ptr(), N, N, nz, rate, g.data_ptr(), s, codec=codec)
        r = {}
        for kind, fn in (("encode", enc), ("decode", dec)):
            fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / reps
            gbs = vals * (4 + rate / 8) / (ms / 1e3) / 1e9
            r[kind] = {"avg_launch_ms": ms, "gvalues_per_s": vals / (ms / 1e3) / 1e9, "achieved_gbs": gbs,
                       "frac_of_hbm": gbs / hbm_peak}
        out[name] = r
    del noise, zero, g, blocks
    torch.cuda.empty_cache()
    return {"grid": [N, N, nz], "rate": rate, "bytes_per_value": 4 + rate / 8, **out}


def check_accuracy(P, torch, dev, rate, inputs, codec=0, ref=None):
    """Compressed run of the workload (100 steps from rest) against the
    uncompressed in-core GPU run of the same FP32 arithmetic (which the tests
    hold within 1e-5 of the FP64 oracle); `ref` reuses that run."""
    import numpy as np

    import synthetic
    st, pin = open_ctx(P, torch, rate, 1, inputs, codec=codec)
    st.step(STEPS_PER_CALL)
    st.synchronize(600.0)
    out = st.decompress(P.OOCS_FIELD_U)
    st.synchronize(600.0)
    got = out.numpy().astype(np.float64)
    st.close()
    del st, pin
    torch.cuda.empty_cache()
    if ref is None:
        ref = incore_reference(P, torch, dev, inputs)
    rel = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    tol = synthetic.TOL_COMPRESSED.get(rate) if rate else synthetic.TOL_UNCOMPRESSED["wave"]
    return {"rel_l2_vs_uncompressed_fp32": rel, "max_abs": float(np.max(np.abs(got - ref))),
            "max_ref": float(np.max(np.abs(ref))), "stated_max_rel_l2": tol,
            "within": bool(tol is not None and rel <= tol)}


def incore_reference(P, torch, dev, inputs):
    """The workload's 100 steps from rest, uncompressed and in core on the GPU (FP64 copy of u)."""
    import numpy as np
    m, w, src, z = inputs
    u = torch.zeros((N, N, N), device=dev)
    up = torch.zeros((N, N, N), device=dev)
    mm = torch.from_numpy(m).to(dev)
    sc = torch.empty_like(u)
    srcv = (src[0], src[1], src[2])
    P.oocs_incore_run(wave_desc(P, 0), u.data_ptr(), up.data_ptr(), mm.data_ptr(), sc.data_ptr(),
                      STEPS_PER_CALL, 0, srcv, w, torch.cuda.current_stream(dev).cuda_stream)
    ref = u.cpu().numpy().astype(np.float64)
    del u, up, mm, sc
    torch.cuda.empty_cache()
    return ref


# ------------------------------------------------------------ reference --

def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    inputs = make_inputs(K_DEPTH * (args.warmup + args.steps + 1))
    for _ in range(args.warmup):
        cpu_oracle_sample(inputs, args.rate)
    times = []
    for _ in range(args.steps):
        dt, npts, cores = cpu_oracle_sample(inputs, args.rate)
        times.append(dt)
    total = sum(times)
    value = npts * len(times) / total / 1e9
    line = base_line(args, world)
    sample = (f"per step: 4 FP64 leapfrog steps on a 512x512x{SAMPLE_PLANES} sub-grid of the "
              f"model + reference codec round trip of u, u_prev, m at rate {args.rate}")
    line.update({"impl": "reference", "value": value, "ms_per_step": total / len(times) * 1e3,
                 "dtype": "f64",
                 "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                                  "sample": sample},
                 "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                         "d2h_bytes_per_step": 0}})
    print(json.dumps(line), flush=True)


def run_profile(args):
    """Workloads for ncu: the captured region is bracketed by cudaProfilerStart/Stop."""
    import numpy as np
    import torch

    import paper_2204_11315_gb300 as P
    import synthetic
    dev = torch.device("cuda", 0)
    P.lib()
    if args.profile_run == "sweep":
        inputs = make_inputs(3 * STEPS_PER_CALL)
        st, pin = open_ctx(P, torch, args.rate, 1, inputs)
        snap = st.snapshot_stores()
        st.step(STEPS_PER_CALL)
        st.synchronize(600.0)
        st.restore_stores(snap, 0)
        torch.cuda.profiler.start()
        st.step(STEPS_PER_CALL)
        st.synchronize(600.0)
        torch.cuda.profiler.stop()
        print(json.dumps({"profile_run": "sweep", "stats": st.stats()}))
        st.close()
        return
    nz = 192
    shape = (nz, N, N)
    m = torch.from_numpy(synthetic.wave_model(shape)).to(dev)
    u = torch.randn(shape, device=dev) * 1e-3
    up = torch.randn(shape, device=dev) * 1e-3
    sc = torch.empty_like(u)
    blocks = torch.empty(N * N * nz * args.rate // 32, dtype=torch.int32, device=dev)
    s = torch.cuda.current_stream(dev).cuda_stream
    d = P.make_desc(N, N, nz, P.OOCS_WAVE, synthetic.wave_star_coef(), BUDGET, rate_bits=0,
                    temporal_depth=K_DEPTH, slab_planes=SLAB)
    # an 80-plane grid: the window size of the sweep's balanced step launches
    d80 = P.make_desc(N, N, 80, P.OOCS_WAVE, synthetic.wave_star_coef(), BUDGET, rate_bits=0,
                      temporal_depth=K_DEPTH, slab_planes=SLAB)
    u80, up80, sc80, m80 = (t[:80].clone() for t in (u, up, sc, m))
    torch.cuda.synchronize(dev)
    torch.cuda.profiler.start()
    P.oocs_incore_run(d, u.data_ptr(), up.data_ptr(), m.data_ptr(), sc.data_ptr(), 1, 0, None, None, s)
    P.oocs_encode_device(u.data_ptr(), N, N, nz, args.rate, blocks.data_ptr(), s)
    P.oocs_decode_device(blocks.data_ptr(), N, N, nz, args.rate, sc.data_ptr(), s)
    P.oocs_incore_run(d80, u80.data_ptr(), up80.data_ptr(), m80.data_ptr(), sc80.data_ptr(), 1, 0, None, None,
                      s)
    # the block quantiser's kernels on the same field and rate
    P.oocs_encode_device(u.data_ptr(), N, N, nz, args.rate, blocks.data_ptr(), s, codec=1)
    P.oocs_decode_device(blocks.data_ptr(), N, N, nz, args.rate, sc.data_ptr(), s, codec=1)
    torch.cuda.synchronize(dev)
    torch.cuda.profiler.stop()
    print(json.dumps({"profile_run": "kernels", "grid": [N, N, nz], "rate": args.rate,
                      "finite": bool(np.isfinite(sc.cpu().numpy()).all())}))


def main():
    args = parse()
    if args.profile_run:
        run_profile(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
