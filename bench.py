"""Benchmark of the 0th persistent homology barcode path on GB300.

One step = the whole path (distances, sort, de-duplication, boundary matrix,
column reduction, bar read-out) over one point cloud: 32,768 points in R^16
on 4 noisy unit circles, 536,854,528 edges.  The metric is edges sorted and
reduced per second (edges of the cloud / device time of one step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: one process per GPU (torchrun); each rank computes its own cloud
(replicas, no collective on the data path); value = edges of all ranks /
max-over-ranks time.  --impl reference times the CPU oracle on a bounded
sample of the same workload on the host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2203_02527_gb300 import inputs  # noqa: E402
from paper_2203_02527_gb300.replicas import job_throughput, max_over_ranks, replica_seed  # noqa: E402

WORKLOAD = "circles32768"
# DRAM bytes per edge (dram__bytes_read.sum + dram__bytes_write.sum over the
# launch, divided by its edges) of the kernels of the distance+sort phase,
# from one ncu capture per kernel on the 8192-point circles cloud
# (profiles/kernels_circles8192.md), scaled by edges to the benchmark cloud:
# the distance kernel, one radix pass (mean of the captured slots 4, 5 and
# the top pass), the fix-up.
PHASE_TRAFFIC_PER_EDGE = {"k_dist": 10.24, "k_onesweep": 25.31, "k_sort_fixup": 8.18}
ONESWEEP_TRAFFIC_PER_EDGE = PHASE_TRAFFIC_PER_EDGE["k_onesweep"]
# The packed sort (clouds up to 32768 points, the benchmark's form): DRAM
# bytes per edge of the distance kernel, its four passes and its fix-up with
# the fix-up's second kernel (whose key gathers grow with the share of edges
# in groups of equal key >> 22), from ncu on the benchmark cloud itself
# (profiles/launches_packed_circles32768.md); and the algorithmic bytes of
# each pass: pass 0 reads the key (8 B) and the value (4 B) and writes the
# word (8 B), the others read and write the word.
PACKED_TRAFFIC_PER_EDGE = {"k_dist": 11.95, "k_psweep": [22.98, 18.91, 17.94, 17.70], "k_pfixup": 42.29}
PACKED_PASS_BYTES = [20.0, 16.0, 16.0, 16.0]
# the algorithmic floor of the phase (steps 1-3): write the records (12 B),
# read and write them once to sort (24 B), read the keys and write a (12 B)
PHASE_FLOOR_PER_EDGE = 48.0
# binary64 additions per SM per clock: the nominal rate (1.25 TFLOP/s counting
# a fused multiply-add as 2, at 152 SMs and 2.07 GHz) and the rate a probe
# kernel of dependent-free additions measured on GB300
ADDS_PER_SM_CLK_NOMINAL = 2.0
ADDS_PER_SM_CLK_MEASURED = 1.6
METRIC = "edges sorted+reduced/s at N=32768"
PACKED_PASSES = 4
# bounded sample of the workload for the CPU oracle: every 5th point
SAMPLE_STRIDE = 5


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload_points(args, seed=inputs.DEFAULT_SEED) -> np.ndarray:
    """The benchmark cloud; --n smaller than 32768 gives the same construction
    (4 noisy circles in R^16) at n points, for profiling captures."""
    if args.n == 32768:
        return inputs.config_points(WORKLOAD, seed=seed)
    return inputs.noisy_circles(args.n // 4, 4, 16, noise=0.02, center_range=5.0, seed=seed)


def cpu_sample(x: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(x[::SAMPLE_STRIDE])


def time_oracle(x: np.ndarray):
    import oracle
    xs = cpu_sample(x)
    n = len(xs)
    m = n * (n - 1) // 2
    t0 = time.perf_counter()
    oracle.barcodes(xs)
    dt = time.perf_counter() - t0
    return m / dt, dt, n, m


def time_paper_cpu(x: np.ndarray, gpu_bars=None):
    """The paper-style CPU baseline (OpenMP, all host cores) on the whole
    cloud, once; its bars are compared with the GPU's."""
    import oracle
    n = len(x)
    m = n * (n - 1) // 2
    t0 = time.perf_counter()
    b, _, _ = oracle.barcodes_paper_cpu(x)
    dt = time.perf_counter() - t0
    out = {"value": m / dt, "unit": "edges/s", "cores": oracle.paper_cpu_threads(),
           "kind": "paper-style OpenMP CPU program (Sec. 3): parallel distance loop, parallel merge sort, "
                   "parallel de-duplication, sequential reduction stopping at n-1 pivots",
           "sample": f"the whole cloud: N={n}, {m} edges, {dt:.1f} s",
           "affinity_cores": len(os.sched_getaffinity(0))}
    if gpu_bars is not None:
        out["bars_identical_to_gpu"] = b.tobytes() == gpu_bars.cpu().numpy().tobytes()
    return out


def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores, on a bounded sample."""
    if rank != 0:
        return
    x = workload_points(args)
    for _ in range(args.warmup):
        time_oracle(x)
    rates, secs = [], []
    for _ in range(args.steps):
        r, dt, n, m = time_oracle(x)
        rates.append(r)
        secs.append(dt)
    value = float(statistics.mean(rates))
    workload = WORKLOAD if args.n == 32768 else f"circles{args.n}"
    sample = (f"every {SAMPLE_STRIDE}th point of the {workload} cloud: N={n}, d=16, "
              f"{m} edges per step, single-threaded oracle (steps 1-5, full reduction)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "edges/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload, "n": args.n, "d": 16, "sample": sample},
        "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2203_02527_gb300 import ph0

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    # each rank computes its own cloud (independent replicas)
    x = workload_points(args, seed=replica_seed(inputs.DEFAULT_SEED, rank))
    n, d = x.shape
    m = n * (n - 1) // 2
    pts = torch.from_numpy(x).to(dev)
    tuning = None
    if not args.no_tune:
        from paper_2203_02527_gb300 import autotune
        tuning = autotune.tune(d, n=n)  # cached for ph0.barcodes below
    # --sort: the whole path's sort form, else the tuned or built-in choice
    run_tuning = None
    if args.sort != "auto":
        run_tuning = dict(tuning or {}, packed_sort=1 if args.sort == "packed" else 0)
    ws = ph0.Workspace(n, d, dev)
    bars = torch.empty((n - 1, 40), dtype=torch.uint8, device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > L2 (129 MB)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        flush.zero_()
        ph0.barcodes_profiled(pts, ws, bars, tuning=run_tuning)
    stats = ph0.finish(ws)

    profs = []
    sampler = ClockSampler(local_rank)
    barrier()
    wall0 = time.perf_counter()
    with sampler:
        for _ in range(args.steps):
            flush.zero_()  # L2 flush, outside the timed events
            _, prof = ph0.barcodes_profiled(pts, ws, bars, tuning=run_tuning)
            profs.append(prof)
    barrier()
    wall = time.perf_counter() - wall0
    st = ph0.finish(ws)
    if st["status"] != 0:
        raise RuntimeError(f"device status {st['status']}")
    ms = max_over_ranks(float(np.mean([p["total_ms"] for p in profs])), dev)

    # end to end through the public API: pinned host points in, bars out to host
    host_pts = torch.from_numpy(x).pin_memory()
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        dpts = host_pts.to(dev, non_blocking=True)
        b = ph0.barcodes(dpts, ws, tuning=run_tuning)
        host_bars = b.raw.to("cpu")
        host_inf = b.inf_raw.to("cpu")  # the bar that never dies
        e1.record()
        e1.synchronize()
        if i >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e = max_over_ranks(float(np.mean(e2e_ms)), dev)

    # the early-terminating path (ph0_barcodes_early; it waits between its
    # rounds, so it is timed on the host clock): the same bars, sorting only
    # the prefix of the edge order that the reduction needs
    early_ms = []
    early_same = True
    for i in range(0 if args.no_early else args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eb = ph0.barcodes_early(pts, ws)
        t1 = time.perf_counter()
        early_same = early_same and bool(torch.equal(eb.raw, bars))
        if i >= args.warmup:
            early_ms.append((t1 - t0) * 1e3)
    early = None
    if early_ms:
        early_t = max_over_ranks(float(np.mean(early_ms)), dev)
        early = {"value": job_throughput(m, world, early_t), "unit": "edges/s", "ms_per_step": early_t,
                 "sorted_edges": int(eb.stats["sorted_edges"]), "identical_to_whole_path": early_same,
                 "timing": "host clock around the synchronous call, L2 flushed before each",
                 "choice": "built-in (sorts in rounds from 2^27 edges on)"}
        if rank == 0 and world == 1:
            early["configs"] = time_early_configs(args, dev, flush)

    if rank != 0:
        return
    # roofline of the dominant kernel
    mean = lambda k: float(np.mean([p[k] for p in profs]))  # noqa: E731
    passes = int(st["sort_passes"])
    packed = int(st.get("sort_form", 0)) == 1
    # the short sort runs the passes from slot 2 on (the slots below sort key
    # bits 0..15, which the fix-up completes), so slots 0 and 1 stay empty;
    # the packed sort's four passes take slots 0-3
    pass_ms = [float(np.mean([p["pass_ms"][i] for p in profs])) for i in range(passes)]
    ran = [t for t in pass_ms if t > 0.05]
    stages = {"dist_ms": mean("dist_ms"), "sort_ms": mean("sort_ms"), "pass_ms": pass_ms,
              "fixup_ms": mean("fixup_ms"), "dedupe_ms": mean("dedupe_ms"),
              "reduce_ms": mean("reduce_ms"), "emit_ms": mean("emit_ms"),
              "sort_form": "packed" if packed else "short"}
    hbm, hbm_src = peaks()
    per_pass_ms = float(np.mean(ran)) if ran else 0.0
    if packed:
        # the four passes together: their algorithmic bytes over their time
        alg = sum(PACKED_PASS_BYTES) * m
        t_all = sum(pass_ms[:PACKED_PASSES]) if len(pass_ms) >= PACKED_PASSES else 0.0
        achieved = alg / (t_all * 1e-3) / 1e9 if t_all > 0 else 0.0
        roof_sort = {"kernel": "k_psweep", "bound": "hbm", "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": sum(PACKED_TRAFFIC_PER_EDGE["k_psweep"]) * m / PACKED_PASSES,
                     "traffic_source": "ncu dram bytes of the four passes on the benchmark cloud, per launch",
                     "algorithmic_bytes": alg / PACKED_PASSES, "peak_source": hbm_src,
                     "launches": PACKED_PASSES, "ms_per_launch": t_all / PACKED_PASSES,
                     "per_pass": [{"ms": t, "algorithmic_bytes_per_edge": b,
                                   "achieved": b * m / (t * 1e-3) / 1e9 if t > 0 else 0.0,
                                   "frac": b * m / (t * 1e-3) / 1e9 / hbm if t > 0 else 0.0}
                                  for t, b in zip(pass_ms[:PACKED_PASSES], PACKED_PASS_BYTES)]}
    else:
        # the radix passes: 24 algorithmic bytes per edge per pass, against HBM
        achieved = 24.0 * m / (per_pass_ms * 1e-3) / 1e9 if per_pass_ms > 0 else 0.0
        roof_sort = {"kernel": "k_onesweep", "bound": "hbm", "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": ONESWEEP_TRAFFIC_PER_EDGE * m,
                     "traffic_source": "ncu on the 8192-point cloud (slots 4-6), scaled by edges",
                     "algorithmic_bytes": 24.0 * m, "peak_source": hbm_src,
                     "launches": len(ran), "ms_per_launch": per_pass_ms}
    # the distance kernel: its binding unit is the binary64 adder, which takes
    # the d-1 running-sum additions per edge (the exact squares are formed on
    # the integer ALU); peak = additions per SM per clock x the device's SMs x
    # the SM clock sampled during the timed region
    clocks = sampler.summary()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_hz = (clocks["sm_mhz"] or 2070.0) * 1e6
    adds = max(d - 1, 1) * m
    adder_peak = sms * ADDS_PER_SM_CLK_NOMINAL * clk_hz
    adder_meas = sms * ADDS_PER_SM_CLK_MEASURED * clk_hz
    achieved = adds / (stages["dist_ms"] * 1e-3) if stages["dist_ms"] > 0 else 0.0
    roof_dist = {"kernel": "k_dist", "bound": "alu", "achieved": achieved / 1e12, "peak": adder_peak / 1e12,
                 "unit": "T binary64 additions/s", "frac": achieved / adder_peak, "traffic": None,
                 "algorithmic_ops": adds,
                 "frac_of_probe_rate": achieved / adder_meas,
                 "peak_source": (f"derived: {ADDS_PER_SM_CLK_NOMINAL:g} binary64 additions per SM per clock "
                                 f"(nominal) x {sms} SMs x {clk_hz / 1e9:.3f} GHz (median sampled SM clock); "
                                 f"frac_of_probe_rate uses the {ADDS_PER_SM_CLK_MEASURED:g} per SM per clock "
                                 f"a probe measured")}
    # the dominant kernel by time: the radix passes together, or the distances
    if stages["dist_ms"] >= sum(ran):
        roof, roof_other = roof_dist, roof_sort
    else:
        roof, roof_other = roof_sort, roof_dist
    # the distance+sort phase (steps 1-2 and the counts of step 3): DRAM bytes
    # of its kernels (ncu, scaled by edges) over its device time, against the
    # copy peak; and the algorithmic floor's bytes over the same time
    phase_ms = stages["dist_ms"] + stages["sort_ms"]
    if packed:
        phase_bytes = m * (PACKED_TRAFFIC_PER_EDGE["k_dist"] + sum(PACKED_TRAFFIC_PER_EDGE["k_psweep"])
                           + PACKED_TRAFFIC_PER_EDGE["k_pfixup"])
        phase_kernels = "k_dist, k_psweep x4, k_pfixup"
    else:
        phase_bytes = m * (PHASE_TRAFFIC_PER_EDGE["k_dist"] + len(ran) * PHASE_TRAFFIC_PER_EDGE["k_onesweep"]
                           + PHASE_TRAFFIC_PER_EDGE["k_sort_fixup"])
        phase_kernels = "k_dist, k_onesweep x%d, k_sort_fixup" % len(ran)
    phase = {"kernels": phase_kernels, "ms": phase_ms,
             "traffic": phase_bytes, "traffic_per_edge": phase_bytes / m,
             "achieved": phase_bytes / (phase_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
             "frac": phase_bytes / (phase_ms * 1e-3) / 1e9 / hbm,
             "floor_per_edge": PHASE_FLOOR_PER_EDGE,
             "floor_frac": PHASE_FLOOR_PER_EDGE * m / (phase_ms * 1e-3) / 1e9 / hbm,
             "traffic_source": ("ncu dram bytes per edge of each kernel on the benchmark cloud"
                                if packed else
                                "ncu dram bytes per edge of each kernel on the 8192-point cloud, scaled by edges"),
             "peak_source": hbm_src}
    # sort init, distances, the short sort (passes from slot 2: 8 launches
    # with slot 6's compaction and its two instances) and its fix-up (and
    # the kernel for deferred groups), gated fallback (sort init, distances,
    # 8 pass slots in 10 launches, de-duplication recount: they return at
    # once unless needed), the de-duplication scan, reduction (init, kernel),
    # pivot-order sort (sort init, key stats, 10 launches), emission, the
    # infinite bar; the packed sort adds its check, 4 passes, 2 fix-up
    # kernels and the short sort's gated key statistics (the short sort's
    # launches then return at once)
    launches_per_step = 1 + 1 + (8 + 2) + (1 + 1 + 10 + 1) + 1 + 2 + (1 + 1 + 10) + 1 + 1
    if packed:
        launches_per_step += 1 + 4 + 2 + 1
    cpu = cpu_all = cpu_full = None
    if world == 1 and not args.no_cpu_baseline:
        r, dt, ns, ms_ = time_oracle(x)
        cpu = {"value": r, "unit": "edges/s", "cores": 1, "kind": "oracle",
               "sample": f"every {SAMPLE_STRIDE}th point of the cloud: N={ns}, {ms_} edges, "
                         f"{dt:.1f} s single-threaded"}
        # the paper-style multi-core CPU program (OpenMP loops, sequential
        # reduction) on the whole cloud, once; it computes the same bars
        cpu_all = time_paper_cpu(x, bars)
        if args.cpu_full_oracle:  # the single-threaded oracle on the whole cloud (minutes, ~40 GB)
            import oracle
            t0 = time.perf_counter()
            want, _, _ = oracle.barcodes(x)
            dt = time.perf_counter() - t0
            same = want.tobytes() == bars.cpu().numpy().tobytes()
            cpu_full = {"value": m / dt, "unit": "edges/s", "cores": 1, "kind": "oracle", "seconds": dt,
                        "sample": "the whole cloud", "bars_identical_to_gpu": same}
    serving = run_serving(args, dev) if (args.serve_clouds > 0 and world == 1) else None
    descent = run_descent(args, dev) if (world == 1 and not args.no_descent) else None
    h1 = None
    if world == 1 and not args.no_h1:
        try:
            h1 = run_h1(args, dev)
        except Exception as exc:  # reported in the line; the other measurements stand
            h1 = {"error": str(exc)}
    line = {
        "metric": METRIC, "value": job_throughput(m, world, ms), "unit": "edges/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if n == 32768 else f"circles{n}", "n": n, "d": d,
                   "edges_per_cloud": m,
                   "l2": "flushed between steps (512 MB write)",
                   "parallelism": f"replicas x{world}"},
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                   "reasons": clocks["reasons"]},
        "e2e": {"value": job_throughput(m, world, e2e), "unit": "edges/s",
                "h2d_bytes_per_step": int(x.nbytes), "d2h_bytes_per_step": int(host_bars.numel() + host_inf.numel())},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roof,
        "roofline_other": roof_other,
        "phase": phase,
        "cpu_baseline": cpu,
        "cpu_baseline_allcores": cpu_all,
        "cpu_baseline_full_oracle": cpu_full,
        "tuning": run_tuning if run_tuning is not None else tuning,
        "serving": serving,
        "descent": descent,
        "h1": h1,
        "early_exit": early,
        "stages_ms": stages,
        "stats": {k: int(v) for k, v in st.items()},
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)


def run_descent(args, dev):
    """The differentiation workload: 64 clouds of 2048 uniform points in
    [0,1)^3, loss = sum of squared finite deaths, SGD (lr 1e-2) on the
    coordinates.  Time per step (forward, backward, update) with one call
    per cloud, with the clouds spread over 8 streams (ph0.Batch), and with
    that batched step captured once into a CUDA graph and replayed (the
    statuses of all clouds read in one copy after each replay)."""
    import torch

    from paper_2203_02527_gb300 import ph0
    xs = [inputs.uniform(2048, 3, seed=1000 + c) for c in range(64)]
    m = 2048 * 2047 // 2
    out = {"clouds": 64, "n": 2048, "d": 3, "edges_per_step": 64 * m}
    for mode in ("one_at_a_time", "batched"):
        pts = [torch.from_numpy(x).to(dev).requires_grad_(True) for x in xs]
        opt = torch.optim.SGD(pts, lr=1e-2)
        batch = ph0.Batch([x.shape for x in xs], streams=8, device=dev)
        ws = batch.workspaces[0]
        losses, times = [], []
        for step in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            opt.zero_grad()
            if mode == "batched":
                deaths = batch.death_values(pts)
            else:
                deaths = [ph0.death_values(p, ws) for p in pts]
            total = sum((dv ** 2).sum() for dv in deaths)
            total.backward()
            opt.step()
            losses.append(float(total.detach()))  # reads the loss back: a sync
            if step >= args.warmup:
                times.append(time.perf_counter() - t0)
        ms = 1e3 * float(np.mean(times))
        out[mode] = {"ms_per_step": ms, "clouds_per_s": 64 / (ms * 1e-3), "edges_per_s": 64 * m / (ms * 1e-3),
                     "loss_first": losses[0], "loss_last": losses[-1]}
        del batch
        torch.cuda.empty_cache()
    out["graphed"] = descent_graphed(args, dev, xs, m)
    out["timing"] = "host clock around each step (the loss is read back every step)"
    return out


def descent_graphed(args, dev, xs, m):
    """The batched descent step captured into a CUDA graph after eager
    warm-up steps, then replayed: the same steps as 'batched', with no host
    launch per cloud."""
    import torch

    from paper_2203_02527_gb300 import ph0
    pts = [torch.from_numpy(x).to(dev).requires_grad_(True) for x in xs]
    opt = torch.optim.SGD(pts, lr=1e-2)
    batch = ph0.Batch([x.shape for x in xs], streams=8, device=dev)

    def step():
        deaths = batch.death_values(pts)
        total = sum((dv ** 2).sum() for dv in deaths)
        total.backward()
        opt.step()
        return total

    losses, times = [], []
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # eager warm-up steps before the capture
        for _ in range(max(args.warmup, 3)):
            opt.zero_grad(set_to_none=True)
            losses.append(float(step().detach()))
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    opt.zero_grad(set_to_none=True)
    with torch.cuda.graph(graph):
        static_total = step()
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        graph.replay()
        losses.append(float(static_total.detach()))
        batch.check()
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    return {"ms_per_step": ms, "clouds_per_s": 64 / (ms * 1e-3), "edges_per_s": 64 * m / (ms * 1e-3),
            "loss_first": losses[0], "loss_last": losses[-1], "warmup_steps_eager": max(args.warmup, 3)}


def run_h1(args, dev):
    """First homology (ph0_h1) on uniform points in the unit square, the
    paper's workload (256 points, its largest N of 700, and the largest cloud
    ph0_h1 takes, 4096): host clock around the synchronous call, stage times
    from CUDA events; the oracle's literal reduction timed beside it on one
    core where it finishes in seconds."""
    import torch

    from paper_2203_02527_gb300 import ph0
    out = {}
    for n in (256, 700, 4096):
        x = inputs.uniform(n, 2, seed=20260109 + n)
        pts = torch.from_numpy(x).to(dev)
        times = []
        for i in range(1 + min(args.steps, 3)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            bars, st = ph0.h1(pts)
            if i:
                times.append(time.perf_counter() - t0)
        ms = 1e3 * float(np.mean(times))
        out[f"uniform{n}_2d"] = {"ms": ms, "triangles": st["n_triangles"], "bars": st["n_bars"],
                                 "triangles_per_s": st["n_triangles"] / (ms * 1e-3), "apparent": st["apparent"],
                                 "reduced_columns": st["reduced"], "additions": st["additions"],
                                 "max_column": st["max_column"], "pool_entries": st["pool_entries"],
                                 "nonzero_bars": int((bars["death_sq"] > bars["birth_sq"]).sum()),
                                 "stage_ms": {k: round(st[k], 4) for k in
                                              ("edges_ms", "scan_ms", "reduce_ms", "emit_ms")}}
    if not args.no_cpu_baseline:
        import oracle
        x = inputs.uniform(256, 2, seed=20260109 + 256)
        t0 = time.perf_counter()
        oracle.h1(x)
        dt = time.perf_counter() - t0
        out["oracle_uniform256_2d"] = {"ms": 1e3 * dt, "cores": 1, "kind": "oracle"}
    out["timing"] = ("host clock around the synchronous call (workspace allocated inside); "
                     "stage_ms: CUDA events on the call's stream, last call")
    return out


def time_early_configs(args, dev, flush):
    """ph0_barcodes_early with its built-in choice against the plain whole
    path on the three single-cloud workloads, both on the host clock around
    the synchronous calls (L2 flushed before each); bars compared."""
    import torch

    from paper_2203_02527_gb300 import ph0
    out = {}
    for name in ("uniform256", "mixture4096", "circles32768"):
        x = inputs.config_points(name)
        pts = torch.from_numpy(x).to(dev)
        ws = ph0.Workspace(len(x), x.shape[1], dev)
        times = {"whole": [], "early": []}
        same = True
        for i in range(args.warmup + args.steps):
            for kind in ("whole", "early"):
                flush.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                b = ph0.barcodes(pts, ws) if kind == "whole" else ph0.barcodes_early(pts, ws)
                t1 = time.perf_counter()
                if i >= args.warmup:
                    times[kind].append((t1 - t0) * 1e3)
                if kind == "whole":
                    ref = b.raw.clone()
                else:
                    same = same and bool(torch.equal(b.raw, ref))
                    sorted_edges = int(b.stats["sorted_edges"])
        out[name] = {"whole_ms": float(np.mean(times["whole"])), "early_ms": float(np.mean(times["early"])),
                     "sorted_edges": sorted_edges, "edges": len(x) * (len(x) - 1) // 2, "identical": same}
        del ws
        torch.cuda.empty_cache()
    return out


def percentile(vals, q):
    return float(np.percentile(np.asarray(vals), q)) if len(vals) else None


def run_serving(args, dev):
    """Mixed stream (the serving workload): N log-uniform in [64, 8192], d in
    {2,3,8,32}, Gaussian mixtures.  One-at-a-time plain calls (points in from
    pinned host memory, bars out, synchronized) against the serving context
    (admission by memory budget, concurrent streams, fused small-cloud
    batches) under Poisson arrivals at 0.9x and 2x the plain rate and with
    every cloud queued at once.  Latency = result on the host - arrival."""
    import torch

    from paper_2203_02527_gb300 import ph0
    from paper_2203_02527_gb300.serve import Server, run_stream

    clouds = inputs.stream_clouds(args.serve_clouds)
    # plain, one at a time
    ws = ph0.Workspace(8192, 32, dev)
    for x in clouds[:20]:
        ph0.barcodes(torch.from_numpy(x).to(dev), ws)
    torch.cuda.synchronize()

    def plain_call(x):
        pts = torch.from_numpy(x).pin_memory().to(dev, non_blocking=True)
        return ph0.barcodes(pts, ws).raw.to("cpu")

    lat, plain_hash = [], {}
    t0 = time.perf_counter()
    for i, x in enumerate(clouds):
        a = time.perf_counter()
        b = plain_call(x)
        lat.append(time.perf_counter() - a)
        plain_hash[i] = hashlib.blake2b(b.numpy().tobytes(), digest_size=16).digest()
    plain_s = time.perf_counter() - t0
    plain_rate = len(clouds) / plain_s
    out = {"clouds": len(clouds),
           "plain": {"clouds_per_s": plain_rate, "p50_ms": 1e3 * percentile(lat, 50),
                     "p99_ms": 1e3 * percentile(lat, 99),
                     "note": "back-to-back calls: service time, no queueing"}}
    # the plain calls under the same Poisson arrivals as the served form: one
    # call at a time, each starting at its arrival or when the previous ends;
    # latency = result on the host - arrival
    for name, load in (("plain_load_0.9x", 0.9), ("plain_load_2x", 2.0)):
        arr = inputs.poisson_arrivals(len(clouds), load * plain_rate)
        lats, t0 = [], time.perf_counter()
        for i, x in enumerate(clouds):
            while time.perf_counter() - t0 < arr[i]:
                pass
            plain_call(x)
            lats.append(time.perf_counter() - t0 - arr[i])
        wall = time.perf_counter() - t0
        out[name] = {"clouds_per_s": len(clouds) / (wall - arr[0]), "p50_ms": 1e3 * percentile(lats, 50),
                     "p99_ms": 1e3 * percentile(lats, 99), "wall_s": wall}
    edges = sum(len(x) * (len(x) - 1) // 2 for x in clouds)
    out["edges"] = edges
    checked = 0
    with Server(mem_budget=args.serve_budget << 30, host_budget=2 << 30, streams=args.serve_streams,
                small_max_n=180, batch_max=512) as srv:
        run_stream(srv, clouds[:50], tag0=10_000_000)  # warm-up
        for name, load in (("load_0.9x", 0.9), ("load_2x", 2.0), ("saturated", None)):
            arr = None if load is None else inputs.poisson_arrivals(len(clouds), load * plain_rate)
            t0 = time.perf_counter()
            done = run_stream(srv, clouds, arr)
            wall = time.perf_counter() - t0
            first = min(f.submit_time for f in done.values())
            last = max(f.done_time for f in done.values())
            lats = [f.latency for f in done.values()]
            bad = sum(f.status != 0 for f in done.values())
            out[name] = {"clouds_per_s": len(clouds) / (last - first), "p50_ms": 1e3 * percentile(lats, 50),
                         "p99_ms": 1e3 * percentile(lats, 99), "wall_s": wall, "errors": bad}
            for i, want in plain_hash.items():  # every served result against its plain call
                got = hashlib.blake2b(done[i].bars.tobytes(), digest_size=16).digest()
                if got != want or done[i].inf_vertex != 0:
                    raise RuntimeError(f"served cloud {i} differs from the plain call")
                checked += 1
    out["bit_identical_to_plain_checked"] = checked
    out["compare"] = ("plain_load_* and load_* share the arrival stream of each load; "
                      "'saturated' queues every cloud at once")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-full-oracle", action="store_true",
                    help="also time the single-threaded oracle on the whole cloud (minutes, ~40 GB of host memory)")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (built-in tuning)")
    ap.add_argument("--sort", choices=["auto", "short", "packed"], default="auto",
                    help="the whole path's sort: the tuned or built-in choice (auto), the short sort of "
                         "(key, value) records, or the packed sort of 64-bit words")
    ap.add_argument("--no-early", action="store_true", help="skip timing the early-terminating path")
    ap.add_argument("--no-descent", action="store_true", help="skip the 64-cloud gradient-descent timing")
    ap.add_argument("--no-h1", action="store_true", help="skip the first-homology timing")
    ap.add_argument("--serve-clouds", type=int, default=10000,
                    help="clouds in the serving stream (0 = skip the serving measurement)")
    ap.add_argument("--serve-budget", type=int, default=64, help="serving device arena, GiB")
    ap.add_argument("--serve-streams", type=int, default=8)
    ap.add_argument("--n", type=int, default=32768,
                    help="points (multiple of 4); the benchmark workload is 32768")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
