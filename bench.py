#!/usr/bin/env python
"""Benchmark of the NOMAD SGD hot path on GB300.

One step = one NOMAD epoch over the whole training set (every rating updated
once, through the persistent kernel: token queues, routing, fused SGD step)
followed by the test-RMSE reduction, on the Netflix-shaped synthetic
workload (m=480,189, n=17,770, ~100.5M train + ~1.4M test ratings, k=100,
lambda=0.05, Table 1's alpha=0.012, beta=0.05).  The ratings and factors
(about 1.2 GB) are larger than the 129 MB L2, so no flush is needed between
steps.

value  = rating updates per second over the timed steps, whole job (sum of
         the ranks' updates / max over ranks of the timed span).
e2e    = the same metric through the C ABI with host buffers: every step
         loads the ratings from pinned host memory (H2D + device layout
         build), runs one epoch, and evaluates the test RMSE from pinned host
         arrays (H2D, result D2H).
roofline = algorithmic HBM bytes of the epoch kernel (per update: w_i read +
         write, 2*k*4 bytes, plus the 8-byte rating record; h_j stays
         on-chip) / its CUDA-event duration, against the measured copy
         bandwidth.
cpu_baseline = the serial CPU oracle (binary64 shuffled SGD, one thread) on
         a bounded sample of the same workload.

Several GPUs (torchrun): the path does not shard (one problem per GPU), so
every rank runs an independent replica.  --impl reference times the CPU
oracle instead (rank 0 only).

--sweep N: N independent seeded problems of random shape, k and lambda
(synth.sweep_specs), one epoch each per step, run as one persistent launch
(nomad_epoch_many) with per-problem knobs picked by an autotuner (workers,
the circulation of the tokens, tokens taken at once; from calibration
launches and each problem's measured device time span) and, as the
baseline, as N launches one after another (each problem alone on every
resident warp); the tuned launch is also timed with bfloat16 storage.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("SGD rating-updates/sec and time-to-target test RMSE, 1×GB300, "
          "% HBM roofline")
UNIT = "updates/s"

CONFIGS = {
    # name: (generator, k, lambda, alpha, beta)
    "netflix": ("netflix_shaped", 100, 0.05, 0.012, 0.05),
    "yahoo": ("yahoo_shaped", 100, 1.0, 0.00075, 0.01),
    "hugewiki": ("hugewiki_shaped", 100, 0.01, 0.001, 0.0),
    "tiny": ("tiny_planted", 10, 0.05, 0.012, 0.05),
}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.file is None or self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.file.seek(0)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- distributed
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max_sum(t_local: float, units_local: float, world: int, device=None):
    """(max over ranks of t_local, sum over ranks of units_local)."""
    if world == 1:
        return t_local, units_local
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- workloads
def make_workload(cfg: str, device, scale: float = 1.0):
    import synth
    gen, k, lam, alpha, beta = CONFIGS[cfg]
    fn = getattr(synth, gen)
    r = fn(device=device) if cfg == "tiny" else fn(scale, device=device)
    release_cache(device)
    return r, k, lam, alpha, beta


def release_cache(device):
    """Hand the generator's freed device memory back to the driver: the
    library allocates with the CUDA runtime, not through torch's cache."""
    import torch
    if torch.device(device).type == "cuda":
        torch.cuda.synchronize(device)
        torch.cuda.empty_cache()


def workload_name(r, k):
    return "%s m=%d n=%d train=%d test=%d k=%d" % (
        r.name, r.m, r.n, r.nnz, int(r.test_rows.numel()), k)


def host_cpu():
    """(logical CPUs, CPU model name) of the host running the oracle."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return os.cpu_count(), model or "unknown"


def cpu_sample_run(r, k, lam, alpha, beta, target_updates: int, seed: int = 5):
    """The CPU oracle (binary64 shuffled SGD, one thread) for one epoch over a
    sample of the workload: the ratings of every `stride`-th user.  Returns
    (updates, seconds, description)."""
    import numpy as np
    import oracle
    rows = r.train_rows.cpu().numpy()
    cols = r.train_cols.cpu().numpy()
    vals = r.train_vals.cpu().numpy()
    stride = max(1, int(round(rows.size / max(target_updates, 1))))
    sel = (rows % stride) == 0
    rs, cs, vs = rows[sel], cols[sel], vals[sel]
    W = oracle.init_factor(r.m, k, 1, 0)
    H = oracle.init_factor(r.n, k, 1, 1)
    t0 = time.perf_counter()
    oracle.shuffled_sgd(rs, cs, vs, W, H, lam, alpha, beta, 1, seed)
    dt = time.perf_counter() - t0
    desc = ("one epoch of binary64 shuffled SGD over the ratings of every %d-th user "
            "(%d of %d ratings), k=%d" % (stride, rs.size, rows.size, k))
    return int(rs.size), dt, desc


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch
    from paper_1312_0193_gb300 import Nomad

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    r, k, lam, alpha, beta = make_workload(args.config, dev, args.scale)
    nnz = r.nnz
    nm = Nomad(r.m, r.n, k, lam, alpha=alpha, beta=beta, device=local,
               n_workers=args.workers, warps_per_block=args.warps_per_block,
               precision=args.precision, mode=args.mode, routing=args.routing)
    stream = torch.cuda.current_stream(dev)
    t_load0 = time.perf_counter()
    nm.load_coo(r.train_rows, r.train_cols, r.train_vals)
    load_s = time.perf_counter() - t_load0
    info = nm.info()
    te_r, te_c, te_v = r.test_rows, r.test_cols, r.test_vals

    def step():
        nm.epoch(1)
        return nm.rmse(te_r, te_c, te_v)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    launches0 = nm.info()["kernel_launches"]
    barrier(world)
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    kernel_ms = []
    rmses = []
    with ClockSampler(local) as clocks:
        ev0.record(stream)
        for _ in range(args.steps):
            nm.epoch(1)
            rmses.append(nm.rmse(te_r, te_c, te_v))
            kernel_ms.append(nm.last_epoch_kernel_ms())
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    barrier(world)
    t_local = ev0.elapsed_time(ev1) / 1000.0
    launches = nm.info()["kernel_launches"] - launches0
    t_max, units = reduce_max_sum(t_local, float(nnz) * args.steps, world, dev)
    value = units / t_max

    # end to end through the C ABI with pinned host buffers
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    h_rows = r.train_rows.cpu().pin_memory()
    h_cols = r.train_cols.cpu().pin_memory()
    h_vals = r.train_vals.cpu().pin_memory()
    h_te = [t.cpu().pin_memory() for t in (te_r, te_c, te_v)]
    barrier(world)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        nm.load_coo(h_rows, h_cols, h_vals)
        nm.epoch(1)
        nm.rmse(*h_te)
    torch.cuda.synchronize(dev)
    e2e_local = time.perf_counter() - t0
    e2e_t, e2e_units = reduce_max_sum(e2e_local, float(nnz) * e2e_steps, world, dev)
    h2d = 12 * nnz + 12 * int(te_r.numel())

    # w_i read and written (FP8: codes and the row's scale) + the rating record
    bytes_per_update = (2 * k * 4 + 8 if args.precision == "fp32" else
                        2 * k * 2 + 8 if args.precision == "bf16" else 2 * k + 2 * 4 + 8)
    kern_avg_s = statistics.mean(kernel_ms) / 1000.0
    achieved_gbs = nnz * bytes_per_update / kern_avg_s / 1e9
    peak, peak_src = load_peaks()
    traffic = None
    l2_hit = None
    tr_path = os.path.join(ROOT, "profiles", "epoch_kernel_traffic.json")
    if os.path.exists(tr_path):
        try:
            with open(tr_path) as f:
                tj = json.load(f)
            if (tj.get("config") == args.config and tj.get("scale", 1.0) == args.scale
                    and tj.get("precision", "fp32") == args.precision
                    and tj.get("kernel_rev") == kernel_rev()):
                traffic = tj.get("dram_bytes_per_launch")
                if "l2_sector_hit_rate_pct" in tj:
                    l2_hit = {"pct": tj["l2_sector_hit_rate_pct"],
                              "case": tj.get("l2_hit_rate_case", "")}
        except Exception:
            traffic = l2_hit = None

    ttt = None
    if rank == 0 and world == 1 and not args.no_ttt:
        ttt = time_to_target(args, dev, local)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        upd, secs, desc = cpu_sample_run(r, k, lam, alpha, beta, args.cpu_sample)
        nproc, model = host_cpu()
        cpu = {"value": upd / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": desc, "seconds": round(secs, 2), "host_nproc": nproc,
               "host_cpu": model}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max * 1000.0 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16": "bf16-storage/f32",
                      "fp8": "e4m3-storage(W)/f32"}[args.precision],
            "data": "synthetic (seeded; stands in for the paper's dataset)",
            "config": {
                "workload": workload_name(r, k), "lambda": lam, "alpha": alpha,
                "beta": beta,
                "mode": "epoch (permutation circulation)" if args.mode == "epoch" else
                        "uniform (Alg. 1), %s routing" % args.routing,
                "workers": info["p"], "warps_per_block": info["warps_per_block"],
                "segments": info["n_segments"],
                "ratings_per_visit": round(nnz / max(info["n_segments"], 1), 3),
                "step": "one epoch (all ratings) + test RMSE",
                "l2": "inputs larger than L2 (ratings %.0f MB, W %.0f MB); no flush" % (
                    nnz * 8 / 1e6,
                    r.m * info["pitch"] * {"fp32": 4, "bf16": 2, "fp8": 1}[args.precision] / 1e6),
                "parallelism": "replicas x%d (one independent problem per GPU)" % world,
                "load_seconds_first": round(load_s, 3),
            },
            "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": peak,
                         "unit": "GB/s", "frac": achieved_gbs / peak, "traffic": traffic,
                         "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_src
                         if peak_src == "measured" else "fallback 6.8 TB/s",
                         "kernel": "nomad_batched_kernel" if args.mode == "epoch" else
                                   "nomad_uniform_kernel", "kernel_ms": kern_avg_s * 1e3,
                         "bytes_per_update": bytes_per_update,
                         "l2_hit_rate": l2_hit},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_units / e2e_t, "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 8,
                    "steps": e2e_steps,
                    "step": "load_ratings(pinned host COO) + epoch + rmse(pinned host)"},
            "time_to_target": ttt,
            "gpu_launches": launches,
            "clocks": clocks.summary(),
            "test_rmse_last": rmses[-1] if rmses else None,
        }
        print(json.dumps(out), flush=True)
    nm.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def sweep_blocks(nnz, total):
    """Blocks per problem: at least one each, the rest in proportion to the
    ratings (largest remainders)."""
    n = len(nnz)
    assert 0 < n <= total
    s = float(sum(nnz))
    want = [total * x / s for x in nnz]
    b = [max(1, int(w)) for w in want]
    while sum(b) > total:
        i = max((i for i in range(n) if b[i] > 1), key=lambda i: b[i] - want[i])
        b[i] -= 1
    while sum(b) < total:
        i = max(range(n), key=lambda i: want[i] - b[i])
        b[i] += 1
    return b


def run_sweep(args):
    import torch
    import synth
    from paper_1312_0193_gb300 import Nomad

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    if args.sweep > sms:
        raise SystemExit("--sweep %d: at most %d problems (one block each, every block "
                         "resident)" % (args.sweep, sms))
    specs = synth.sweep_specs(args.sweep, seed=5)
    t0 = time.perf_counter()
    probs = [synth.sweep_problem(sp, device=dev) for sp in specs]
    release_cache(dev)
    gen_s = time.perf_counter() - t0
    nnz = [r.nnz for r in probs]
    total = float(sum(nnz))
    wpb = 8
    alpha, beta = 0.012, 0.05

    def handles(knobs, precision="fp32"):
        out = []
        for sp, r, kn in zip(specs, probs, knobs):
            nm = Nomad(r.m, r.n, sp["k"], sp["lam"], alpha=alpha, beta=beta, device=local,
                       n_workers=kn["blocks"] * wpb, warps_per_block=wpb, precision=precision,
                       circulation=kn["circulation"], batch_tokens=kn["batch_tokens"])
            nm.load_coo(r.train_rows, r.train_cols, r.train_vals)
            out.append(nm)
        return out

    def calibrate(knobs):
        """One epoch of every problem in one launch: (kernel ms, span ns per
        problem)."""
        cal = handles(knobs)
        Nomad.epoch_many(cal, 1)
        ms = cal[0].last_epoch_kernel_ms()
        spans = [nm.last_epoch_span_ns() for nm in cal]
        for nm in cal:
            nm.close()
        return ms, spans

    # The autotuner.  Knobs per problem: its blocks (workers = 8 x blocks),
    # the circulation of its tokens (flat, or the hybrid of Sec. 3.4) and the
    # tokens a worker takes at once (16 or 8).  Start: blocks in proportion
    # to the ratings, flat, 16.  Each knob is chosen per problem from
    # calibration launches (every problem's device time span read back; the
    # launch waits for its slowest problem), then --sweep-tune rounds
    # re-allocate the blocks in proportion to each problem's block-seconds
    # (span x blocks); the allocation measured fastest is kept.  Queue
    # capacity and the chunks per lane are not knobs: a ring holds every
    # token a worker can be sent, and a lane holds ceil(k / 128) chunks.
    knobs = [{"blocks": b, "circulation": "flat", "batch_tokens": 0}
             for b in sweep_blocks(nnz, sms)]
    tuning = []

    best = None  # (launch ms, knobs) of the fastest trial so far

    def trial(kn, what):
        nonlocal best
        ms, spans = calibrate(kn)
        tuning.append({"trial": what, "kernel_ms": round(ms, 2),
                       "slowest_span_ms": round(max(spans) / 1e6, 2),
                       "mean_span_ms": round(statistics.mean(spans) / 1e6, 2)})
        if best is None or ms < best[0]:
            best = (ms, [dict(k) for k in kn])
        return ms, spans

    if args.sweep_tune > 0:
        ms_flat, sp_flat = trial(knobs, "flat circulation, 16 tokens")
        alt = [dict(k, circulation="block") for k in knobs]
        ms_blk, sp_blk = trial(alt, "hybrid circulation, 16 tokens")
        knobs = [dict(k, circulation="block" if b < f else "flat")
                 for k, f, b in zip(knobs, sp_flat, sp_blk)]
        ms16, sp16 = trial(knobs, "per-problem circulation, 16 tokens")
        alt = [dict(k, batch_tokens=8) for k in knobs]
        ms8, sp8 = trial(alt, "per-problem circulation, 8 tokens")
        knobs = [dict(k, batch_tokens=8 if e < s_ else 0)
                 for k, s_, e in zip(knobs, sp16, sp8)]
        ms, spans = trial(knobs, "per-problem circulation and tokens")
        for _ in range(args.sweep_tune):
            blocks = sweep_blocks([max(sp, 1) * k["blocks"] for sp, k in zip(spans, knobs)],
                                  sms)
            if blocks == [k["blocks"] for k in knobs]:
                break
            knobs = [dict(k, blocks=b) for k, b in zip(knobs, blocks)]
            ms, spans = trial(knobs, "blocks re-allocated")
        knobs = best[1]  # the fastest of all trials
    many = handles(knobs)
    alone = handles([{"blocks": 0, "circulation": "flat", "batch_tokens": 0}] * len(specs))
    stream = torch.cuda.current_stream(dev)

    def run_many():
        Nomad.epoch_many(many, 1)

    def run_alone():
        for nm in alone:
            nm.epoch(1)

    for _ in range(args.warmup):
        run_many()
        run_alone()
    torch.cuda.synchronize(dev)
    launches0 = sum(nm.info()["kernel_launches"] for nm in many)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    kern_many = []
    barrier(world)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clocks:
        ev[0].record(stream)
        for _ in range(args.steps):
            run_many()
            kern_many.append(many[0].last_epoch_kernel_ms())
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
    launches = sum(nm.info()["kernel_launches"] for nm in many) - launches0
    ev[2].record(stream)
    for _ in range(args.steps):
        run_alone()
    ev[3].record(stream)
    torch.cuda.synchronize(dev)
    # the same tuned launch with bfloat16 storage
    many_bf = handles(knobs, precision="bf16")
    for _ in range(args.warmup):
        Nomad.epoch_many(many_bf, 1)
    torch.cuda.synchronize(dev)
    ev[4].record(stream)
    for _ in range(args.steps):
        Nomad.epoch_many(many_bf, 1)
    ev[5].record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    t_many, units = reduce_max_sum(ev[0].elapsed_time(ev[1]) / 1e3, total * args.steps, world, dev)
    t_seq, _ = reduce_max_sum(ev[2].elapsed_time(ev[3]) / 1e3, total * args.steps, world, dev)
    t_bf, _ = reduce_max_sum(ev[4].elapsed_time(ev[5]) / 1e3, total * args.steps, world, dev)
    # the same problems after the same epochs: test RMSE of the arms (the
    # worker counts differ, so the visit orders and the iterates do too)
    rm_many, rm_alone, rm_bf = [], [], []
    for a, b, c, r in zip(many, alone, many_bf, probs):
        a.check()
        b.check()
        c.check()
        rm_many.append(a.rmse(r.test_rows, r.test_cols, r.test_vals))
        rm_alone.append(b.rmse(r.test_rows, r.test_cols, r.test_vals))
        rm_bf.append(c.rmse(r.test_rows, r.test_cols, r.test_vals))
    bytes_upd = sum(n * (2 * sp["k"] * 4 + 8) for n, sp in zip(nnz, specs))
    kern_s = statistics.mean(kern_many) / 1e3
    peak, peak_src = load_peaks()
    if rank == 0:
        out = {
            "metric": "SGD rating-updates/sec, %d independent problems per step, 1×GB300"
                      % len(specs),
            "value": units / t_many, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_many * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded planted problems)",
            "config": {
                "workload": "sweep of %d planted problems: m~U[2k,200k], n~U[1k,50k], "
                            "density~U[0.1%%,2%%], k in {16,32,64,128}, lambda in "
                            "{0.01,0.05,0.1,0.5}; %.3g train ratings" % (len(specs), total),
                "alpha": alpha, "beta": beta, "step": "one epoch of every problem",
                "warps_per_block": wpb, "tuning": tuning,
                "knobs": [dict(k, problem=i, workers=k["blocks"] * wpb, k=sp["k"], nnz=n)
                          for i, (k, sp, n) in enumerate(zip(knobs, specs, nnz))],
                "l2": "inputs larger than L2 (ratings %.1f GB); no flush" % (total * 8 / 1e9),
                "generate_seconds": round(gen_s, 1),
                "parallelism": "replicas x%d" % world,
            },
            "sequential": {"value": units / t_seq, "unit": UNIT,
                           "ms_per_step": t_seq * 1e3 / args.steps,
                           "step": "%d nomad_epoch calls, each problem on every resident warp"
                                   % len(specs)},
            "speedup_vs_sequential": t_seq / t_many,
            "bf16": {"value": units / t_bf, "unit": UNIT, "ms_per_step": t_bf * 1e3 / args.steps,
                     "step": "the tuned one-launch sweep with bfloat16 storage",
                     "test_rmse_mean": statistics.mean(rm_bf)},
            "test_rmse": {"epochs": args.warmup + args.steps,
                          "one_launch_mean": statistics.mean(rm_many),
                          "sequential_mean": statistics.mean(rm_alone),
                          "max_rel_diff": max(abs(a - b) / b for a, b in zip(rm_many, rm_alone)),
                          "note": "different worker counts per problem give different "
                                  "visit orders"},
            "roofline": {"bound": "hbm", "achieved": bytes_upd / kern_s / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": bytes_upd / kern_s / 1e9 / peak,
                         "traffic": None, "peak_source": peak_src,
                         "kernel": "nomad_batched_many_kernel", "kernel_ms": kern_s * 1e3},
            "gpu_launches": launches,
            "clocks": clocks.summary(),
        }
        print(json.dumps(out), flush=True)
    for nm in many + alone + many_bf:
        nm.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def time_to_target(args, dev, local):
    """Time to the oracle's test RMSE: the Netflix-shaped workload at
    `--ttt-scale`, generated on the CPU from its seed exactly as the oracle's
    target script did, from the same initial factors.  Target = 1.005 x the
    binary64 oracle's test RMSE after E epochs (tests/golden/rmse_targets.json).
    GPU time = sum of the epoch kernels' CUDA-event times until the test RMSE
    reaches the target (RMSE evaluation excluded), for binary32 and bfloat16
    storage."""
    import torch
    import synth
    from paper_1312_0193_gb300 import Nomad
    path = os.path.join(ROOT, "tests", "golden", "rmse_targets.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        t = json.load(f).get("%s@%g" % (args.config, args.ttt_scale))
    if not t:
        return None
    gen, k, lam, alpha, beta = CONFIGS[args.config]
    r = getattr(synth, gen)(args.ttt_scale, device="cpu").to(dev)
    E = int(t["epochs"])
    target = 1.005 * float(t["test_rmse"][-1])
    out = {"workload": r.name, "nnz_train": r.nnz, "oracle_epochs": E,
           "oracle_test_rmse": float(t["test_rmse"][-1]), "target": target,
           "max_epochs": 2 * E}
    for prec in ("fp32", "bf16"):
        nm = Nomad(r.m, r.n, k, lam, alpha=alpha, beta=beta, device=local, precision=prec,
                   seed=int(t.get("init_seed", 1)))
        nm.load_coo(r.train_rows, r.train_cols, r.train_vals)
        secs, ep, rm = 0.0, 0, float("inf")
        trace = []  # test RMSE against GPU seconds (Sec. 5.1's curves)
        while ep < 2 * E and not rm <= target:
            nm.epoch(1)
            secs += nm.last_epoch_kernel_ms() / 1e3
            rm = nm.rmse(r.test_rows, r.test_cols, r.test_vals)
            ep += 1
            trace.append([ep, round(secs, 5), round(rm, 6)])
        out[prec] = {"reached": bool(rm <= target), "epochs": ep, "seconds": secs,
                     "test_rmse": rm, "trace_epoch_seconds_rmse": trace}
        nm.close()
    return out


def run_gaps(args):
    """Test-RMSE gap to the binary64 oracle per workload and storage format:
    every workload of tests/golden/rmse_targets.json (data generated on the
    CPU from its seed, as the oracle's target script did), E epochs of the
    timed kernel with p workers from the library's initial factors, against
    the oracle's serial NOMAD with the same p after the same E epochs (and,
    for reference, its textbook shuffled SGD).  One JSON line per (workload,
    format), then a summary line."""
    import torch
    import synth
    from paper_1312_0193_gb300 import Nomad
    dev = torch.device("cuda", 0)
    with open(os.path.join(ROOT, "tests", "golden", "rmse_targets.json")) as f:
        targets = json.load(f)
    gens = {"netflix": "netflix_shaped", "yahoo": "yahoo_shaped",
            "hugewiki": "hugewiki_shaped", "hugewiki-flat": "hugewiki_flat"}
    rows = []
    for key in sorted(targets):
        t = targets[key]
        if t.get("config") not in gens or "nomad" not in t:
            continue
        r = getattr(synth, gens[t["config"]])(t["scale"], device="cpu").to(dev)
        for prec in ("fp32", "bf16", "fp8"):
            nm = Nomad(r.m, r.n, t["k"], t["lambda"], alpha=t["alpha"], beta=t["beta"],
                       seed=int(t["init_seed"]), precision=prec,
                       n_workers=int(t["nomad"]["p"]))
            nm.load_coo(r.train_rows, r.train_cols, r.train_vals)
            ms = 0.0
            for _ in range(int(t["epochs"])):
                nm.epoch(1)
                ms += nm.last_epoch_kernel_ms()
            nm.check()
            got = nm.rmse(r.test_rows, r.test_cols, r.test_vals)
            nm.close()
            want = float(t["nomad"]["test_rmse"])
            want_sd = float(t["nomad"].get("test_rmse_std", 0.0))
            shuf = float(t["test_rmse"][-1])
            row = {"workload": t["workload"], "nnz_train": t["nnz_train"], "precision": prec,
                   "epochs": int(t["epochs"]), "workers": int(t["nomad"]["p"]),
                   "gpu_test_rmse": got, "oracle_nomad_test_rmse": want,
                   "oracle_nomad_std": want_sd,
                   "oracle_nomad_draws": len(t["nomad"].get("runs", [1])),
                   "gap_pct": 100.0 * (got / want - 1.0),
                   "oracle_shuffled_sgd_test_rmse": shuf,
                   "gap_to_shuffled_pct": 100.0 * (got / shuf - 1.0), "gpu_seconds": ms / 1e3}
            rows.append(row)
            print(json.dumps(row), flush=True)
        del r
        release_cache(dev)
    print(json.dumps({"rmse_gaps": rows}), flush=True)


def kernel_rev():
    """Hash of the batched worker kernel's sources, to tie profile figures
    to the code they were taken from."""
    import hashlib
    hs = hashlib.sha256()
    for name in ("epoch_batched.cuh", "epoch_batched.cu", "epoch_batched_f32.cu",
                 "epoch_batched_bf16.cu", "epoch_batched_fp8.cu", "sgd_common.cuh",
                 "nomad_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1312_0193_gb300", "csrc", name), "rb") as f:
            hs.update(f.read())
    return hs.hexdigest()[:16]


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    """The CPU oracle as it stands, on the host cores, rank 0 only."""
    world, rank, local = dist_env()
    if rank != 0:
        return
    import torch
    dev = torch.device("cuda", local) if torch.cuda.is_available() else "cpu"
    r, k, lam, alpha, beta = make_workload(args.config, dev, args.scale)
    # the same sample as the cpu_baseline leg of our arm (--cpu-sample)
    per_step = max(1, args.ref_sample if args.ref_sample > 0 else args.cpu_sample)
    for _ in range(args.warmup):
        cpu_sample_run(r, k, lam, alpha, beta, per_step // 4)
    tot_u, tot_t, desc = 0, 0.0, ""
    for s in range(args.steps):
        u, t, desc = cpu_sample_run(r, k, lam, alpha, beta, per_step, seed=11 + s)
        tot_u += u
        tot_t += t
    v = tot_u / tot_t
    out = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot_t * 1000.0 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded; stands in for the paper's dataset)",
        "config": {"workload": workload_name(r, k), "lambda": lam, "alpha": alpha,
                   "beta": beta},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": desc, "host_nproc": host_cpu()[0],
                         "host_cpu": host_cpu()[1]},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=sorted(CONFIGS), default="netflix")
    ap.add_argument("--precision", choices=["fp32", "bf16", "fp8"], default="fp32")
    ap.add_argument("--mode", choices=["epoch", "uniform"], default="epoch",
                    help="routing of tokens: permutation circulation or Alg. 1")
    ap.add_argument("--routing", choices=["uniform", "shorter"], default="uniform",
                    help="uniform mode: next worker uniform or the shorter of two queues")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink the workload (same shape) for profiler captures")
    ap.add_argument("--workers", type=int, default=0)
    ap.add_argument("--warps-per-block", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-sample", type=int, default=25_000_000,
                    help="ratings in the CPU-oracle baseline sample")
    ap.add_argument("--ref-sample", type=int, default=0,
                    help="ratings per step of the reference arm (0: --cpu-sample, the "
                         "cpu_baseline leg's sample)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ttt", action="store_true", help="skip the time-to-target leg")
    ap.add_argument("--ttt-scale", type=float, default=0.1,
                    help="workload scale of the time-to-target leg")
    ap.add_argument("--sweep", type=int, default=0,
                    help="time N independent problems in one launch against N launches")
    ap.add_argument("--sweep-tune", type=int, default=2,
                    help="autotuner: 0 = no tuning; else per-problem circulation and batch "
                         "size from calibration launches, then this many rounds of block "
                         "re-allocation from measured per-problem spans")
    ap.add_argument("--gaps", action="store_true",
                    help="test-RMSE gap to the oracle for every golden workload and format")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.gaps:
        run_gaps(args)
    elif args.sweep > 0:
        run_sweep(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
