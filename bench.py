#!/usr/bin/env python
"""Benchmark of the GB300 MrDFT: input Gsamples/s and fraction of the HBM roofline.

Default workload (one GPU): one complex64 signal of N = 2^24 samples, i.i.d.
N(0,1) (seed 1), all 24 levels.  A step is one forward MrDFT of that signal;
the adjoint of the same size is timed the same way and reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload single_16m|batch_256x64k|ragged_1024|grad_64x256k|single_1k]

Under torchrun each rank runs its own replica of the workload on its own GPU
(the transform has no cross-signal exchange): weak scaling, barrier-bracketed
CUDA-event timing, max over ranks.  `--impl reference` times the FP64 CPU
oracle (the only reference this paper has) on a bounded sample of the same
workload on the host cores.  One JSON line is printed by rank 0.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MrDFT input Gsamples/s & % of HBM roofline (fwd, adjoint) on 1 GB300"
FALLBACK_HBM_GBS = 6800.0


def log2i(n: int) -> int:
    return int(n).bit_length() - 1


# ------------------------------------------------------------------ workloads

def workload_spec(name: str):
    """(lengths list, real_input, description) of a named workload."""
    from paper_1507_02525_gb300 import inputs
    if name == "single_16m":
        return [1 << 24], False, "1 complex64 signal, N=2^24, re/im i.i.d. N(0,1) seed 1, all 24 levels"
    if name == "single_1k":
        return [1 << 10], False, "1 complex64 signal, N=2^10, seed 0"
    if name == "single_4m":
        return [1 << 22], False, "1 complex64 signal, N=2^22, seed 1 (profiling size)"
    if name == "tiles_4096x4k":
        return [1 << 12] * 4096, False, "4096 complex64 signals of N=2^12, seed 6 (in-tile levels only)"
    if name == "batch_256x64k":
        return [1 << 16] * 256, False, "256 complex64 signals of N=2^16, seed 2, one launch set"
    if name == "grad_64x256k":
        return [1 << 18] * 64, False, "64 complex64 signals of N=2^18, seed 4"
    if name == "ragged_1024":
        lengths, _ = inputs.ragged_real()
        return [int(v) for v in lengths], True, "1024 real FP32 signals, N=2^k, k~U{8..18} seed 3"
    raise SystemExit(f"unknown workload {name}")


def make_input(name: str, rank: int = 0):
    """The workload's input; rank r > 0 of a multi-GPU job draws its own
    shard of the global batch (same shapes, seed + 1000 r)."""
    from paper_1507_02525_gb300 import inputs
    off = 1000 * rank
    if name == "single_16m":
        return inputs.complex_signals(1, 1 << 24, seed=1 + off).reshape(-1)
    if name == "single_1k":
        return inputs.complex_signals(1, 1 << 10, seed=0 + off).reshape(-1)
    if name == "single_4m":
        return inputs.complex_signals(1, 1 << 22, seed=1 + off).reshape(-1)
    if name == "tiles_4096x4k":
        return inputs.complex_signals(4096, 1 << 12, seed=6 + off).reshape(-1)
    if name == "batch_256x64k":
        return inputs.complex_signals(256, 1 << 16, seed=2 + off).reshape(-1)
    if name == "grad_64x256k":
        return inputs.complex_signals(64, 1 << 18, seed=4 + off).reshape(-1)
    if name == "ragged_1024":
        lengths, samples = inputs.ragged_real()
        if rank:  # same lengths, other samples
            import numpy as np
            samples = np.random.default_rng(3 + off).standard_normal(samples.size, dtype=np.float32)
        return samples
    raise SystemExit(name)


def algorithmic_bytes(lengths, real_input: bool) -> int:
    """Roofline bytes of one forward (or adjoint): x once + every level once."""
    in_b = 4 if real_input else 8
    return sum(n * in_b + 8 * log2i(n) * n for n in lengths)


# ----------------------------------------------------------------- utilities

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy read+write)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback (6.8 TB/s, no MEASURED_PEAKS.json)"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1507_02525_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def traffic_key(workload: str, opts: dict) -> str:
    """Key of a plan's DRAM-traffic record: the workload, segment size x
    streams, and a digest of every execution option."""
    dig = hashlib.sha1(json.dumps(opts, sort_keys=True).encode()).hexdigest()[:8]
    return f"{workload}:seg{opts.get('seg_log')}x{opts.get('streams')}:{dig}"


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` from profiles/ncu_traffic.txt, only if the
    recorded source hash matches the kernels built now (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    cur = kernel_source_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and not line.startswith("#"):
            h, k, w, b = parts[:4]
            if h == cur and k == kernel and w == workload:
                return int(float(b))
    return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", self.gpu_id],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        t0 = time.time()
        while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.05)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


# ------------------------------------------------------------- oracle timing

def oracle_sample(lengths, x_np, budget_s: float = 15.0):
    """Time the FP64 oracle (per-window FFT path) on a bounded sample and
    extrapolate to the whole workload.

    For each signal length present, level i is timed on a window-aligned slice
    of max(2^i, 2^22) samples (the oracle's per-level cost is proportional to
    the samples covered) and scaled to the full signal; levels are visited in
    order until the time budget is spent (later levels are then extrapolated
    as proportional to i), and the whole sweep is repeated while less than
    60 % of the budget is used, the estimates averaged.  Returns (samples/s,
    cores, description)."""
    import numpy as np
    from oracle import oracle as O
    O.build()
    cores = O.num_threads()
    uniq = {}
    off = 0
    for n in lengths:
        uniq.setdefault(n, (off, 0))
        uniq[n] = (uniq[n][0], uniq[n][1] + 1)
        off += n
    spent = 0.0
    estimates = []
    timed_levels = 0
    while not estimates or (spent < 0.6 * budget_s and len(estimates) < 20):
        total_est = 0.0
        for n, (first, count) in sorted(uniq.items()):
            m = log2i(n)
            x = np.asarray(x_np[first:first + n], dtype=np.complex128)
            last = None
            for i in range(1, m + 1):
                if spent < budget_s:
                    s = max(1 << i, min(n, 1 << 22))
                    t0 = time.perf_counter()
                    O.forward_level(x[:s], i) if s < n else O.forward_level(x, i)
                    dt = time.perf_counter() - t0
                    spent += dt
                    timed_levels += 1
                    per = dt * (n / s)
                    last = (i, per)
                else:
                    per = last[1] * i / last[0]
                total_est += per * count
        estimates.append(total_est)
    total = sum(lengths)
    desc = (f"oracle per-window FFT path (FP64, C, OpenMP); {timed_levels} (length, level) timings "
            f"on window-aligned slices of <= 2^22 samples (whole signal when a window is larger), "
            f"scaled by samples covered, {len(estimates)} sweep(s) averaged; {spent:.1f} s of oracle time")
    return total / (sum(estimates) / len(estimates)), cores, desc


# --------------------------------------------------------- other workloads

OTHER_WORKLOADS = ("single_1k", "batch_256x64k", "ragged_1024", "grad_64x256k")


def measure_other(name: str, dev, stream, timed_fn, tune: bool, peak: float):
    """Forward and adjoint of another named workload on this GPU, timed like the
    headline one (graph replay, CUDA events on the launch stream, warm-up
    first); the execution shape tuned per direction when `tune`."""
    import torch
    from paper_1507_02525_gb300 import _lib
    lengths, real_input, desc = workload_spec(name)
    x_np = make_input(name)
    nsamp = sum(lengths)
    alg = algorithmic_bytes(lengths, real_input)
    opts_f = opts_a = {}
    if tune:
        from paper_1507_02525_gb300 import autotune
        opts_f = autotune.tune_plan(lengths, len(lengths), real_input, objective="forward", reps=3)
        opts_a = autotune.tune_plan(lengths, len(lengths), real_input, objective="adjoint", reps=3)
    pf = _lib.Plan(lengths, len(lengths), real_input=real_input, graph=True, opts=opts_f)
    pa = pf if opts_a == opts_f else _lib.Plan(lengths, len(lengths), real_input=real_input, graph=True, opts=opts_a)
    xt = torch.from_numpy(x_np).to(dev)
    y = torch.empty(pf.out_elems, dtype=torch.complex64, device=dev)
    gx = torch.empty(pf.in_elems, dtype=torch.complex64, device=dev)
    sp = stream.cuda_stream
    small = nsamp < (1 << 20)
    steps = 200 if small else 20
    ms_f = timed_fn(lambda: pf.forward(xt.data_ptr(), y.data_ptr(), sp), steps, 5)
    ms_a = timed_fn(lambda: pa.adjoint(y.data_ptr(), gx.data_ptr(), sp), steps, 5)
    pf.status_poll()
    pa.status_poll()
    out = {"desc": desc, "signals": len(lengths), "samples": nsamp, "alg_bytes": alg,
           "exec_opts": {"forward": pf.opts(), "adjoint": pa.opts(), "tuned": bool(tune)},
           "forward": {"ms": round(ms_f, 5), "gsamples_per_s": round(nsamp / (ms_f * 1e-3) / 1e9, 4),
                       "hbm_frac_step": round(alg / (ms_f * 1e-3) / 1e9 / peak, 4)},
           "adjoint": {"ms": round(ms_a, 5), "gsamples_per_s": round(nsamp / (ms_a * 1e-3) / 1e9, 4),
                       "hbm_frac_step": round(alg / (ms_a * 1e-3) / 1e9 / peak, 4)},
           "fwd_launches": pf.info()["fwd_launches"], "adj_launches": pa.info()["adj_launches"]}
    if small:
        out["forward"]["us_per_call"] = round(ms_f * 1e3, 2)
        out["adjoint"]["us_per_call"] = round(ms_a * 1e3, 2)
        out["note"] = "latency-bound size: time per call through graph replay, back to back"
    if pa is not pf:
        pa.close()
    pf.close()
    del xt, y, gx
    torch.cuda.empty_cache()
    return out


def self_check(y, x_np, lengths, samples: int = 48, seed: int = 0):
    """Sampled output bins of the timed forward against the oracle's direct sum
    of Eq. 1 (part of the CPU-baseline leg, which runs the oracle anyway).
    Returns (ok, summary)."""
    import numpy as np
    from oracle import oracle as O
    rng = np.random.default_rng(seed)
    x128 = np.asarray(x_np).astype(np.complex128)
    worst = 0.0
    offs_in, offs_out = [0], [0]
    for n in lengths:
        offs_in.append(offs_in[-1] + n)
        offs_out.append(offs_out[-1] + log2i(n) * n)
    sig = rng.integers(0, len(lengths), size=samples)
    for k in range(samples):
        s_ = int(sig[k])
        n = lengths[s_]
        m = log2i(n)
        i = int(rng.integers(1, m + 1))
        pos = int(rng.integers(0, n))
        xs = x128[offs_in[s_]:offs_in[s_ + 1]]
        ref = O.bin_value(xs, i, pos)
        got = complex(y[offs_out[s_] + (i - 1) * n + pos].item())
        worst = max(worst, abs(got - ref) / float(np.linalg.norm(xs)))
    ok = worst <= 1e-5
    return ok, {"bins": samples, "max_abs_err_over_norm_x": worst, "bound": 1e-5, "ok": ok,
                "what": "random (signal, level, bin) of the timed forward output vs the oracle's direct sum of Eq. 1"}


# ---------------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="single_16m")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cufft", action="store_true")
    ap.add_argument("--no-train", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-others", action="store_true", help="skip the other workloads' extra keys")
    ap.add_argument("--profile-run", default=None, choices=["fwd", "adj"],
                    help="profiling mode: plan the workload with --opts (JSON execution options, else the "
                         "library defaults), run --warmup + --steps calls in that direction and exit; prints "
                         "the kernel launches of one call (for ncu -s / -c)")
    ap.add_argument("--opts", default=None, help="execution options (JSON) for --profile-run")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    lengths, real_input, desc = workload_spec(args.workload)
    nsamp = sum(lengths)
    alg_bytes = algorithmic_bytes(lengths, real_input)

    if args.impl == "reference":
        if rank != 0:
            return 0
        x_np = make_input(args.workload)
        vals = []
        # every step a bounded sample, so that the whole run stays within minutes
        per_step = max(0.5, min(4.0, 150.0 / (args.warmup + args.steps)))
        for k in range(args.warmup + args.steps):
            v, cores, sdesc = oracle_sample(lengths, x_np, budget_s=per_step)
            if k >= args.warmup:
                vals.append(v)
        value = statistics.median(vals) / 1e9
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gsamples/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": nsamp / (value * 1e9) * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "desc": desc, "signals": len(lengths),
                           "samples": nsamp},
                "cpu_baseline": {"value": value, "unit": "Gsamples/s", "cores": cores,
                                 "kind": "oracle", "sample": sdesc},
                "e2e": {"value": value, "unit": "Gsamples/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0

    import torch
    from paper_1507_02525_gb300 import _lib, replicas

    if args.profile_run:
        opts = json.loads(args.opts) if args.opts else {}
        plan = _lib.Plan(lengths, len(lengths), real_input=real_input, opts=opts)
        x_np = make_input(args.workload)
        xt = torch.from_numpy(x_np).cuda()
        y = torch.empty(plan.out_elems, dtype=torch.complex64, device="cuda")
        gx = torch.empty(plan.in_elems, dtype=torch.complex64, device="cuda")
        sp = torch.cuda.current_stream().cuda_stream
        if args.profile_run == "adj":
            plan.forward(xt.data_ptr(), y.data_ptr(), sp)
        for _ in range(args.warmup + args.steps):
            if args.profile_run == "fwd":
                plan.forward(xt.data_ptr(), y.data_ptr(), sp)
            else:
                plan.adjoint(y.data_ptr(), gx.data_ptr(), sp)
        torch.cuda.synchronize()
        plan.status_poll()
        info = plan.info()
        print(json.dumps({"profile_run": args.profile_run, "workload": args.workload, "opts": plan.opts(),
                          "launches_per_call": info["fwd_launches" if args.profile_run == "fwd" else "adj_launches"],
                          "launches_before_timed": (1 if args.profile_run == "adj" else 0) * info["fwd_launches"]}))
        return 0

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    barrier = replicas.barrier

    def max_over_ranks(v: float) -> float:
        return replicas.max_over_ranks(v, device=dev)

    x_np = make_input(args.workload, rank)
    # execution shapes tuned per direction: the forward plan on forward time,
    # the adjoint plan on adjoint time (one plan when both pick the same shape)
    opts_f = opts_a = {}
    if not args.no_autotune:
        from paper_1507_02525_gb300 import autotune
        opts_f = autotune.tune_plan(lengths, len(lengths), real_input, objective="forward")
        opts_a = autotune.tune_plan(lengths, len(lengths), real_input, objective="adjoint")
    plan = _lib.Plan(lengths, len(lengths), real_input=real_input, graph=True, opts=opts_f)
    plan_adj = plan if opts_a == opts_f else \
        _lib.Plan(lengths, len(lengths), real_input=real_input, graph=True, opts=opts_a)
    info = plan.info()
    info_adj = plan_adj.info()
    xt = torch.from_numpy(x_np).to(dev)
    y = torch.empty(plan.out_elems, dtype=torch.complex64, device=dev)
    gx = torch.empty(plan.in_elems, dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream

    def fwd():
        plan.forward(xt.data_ptr(), y.data_ptr(), sp)

    def adj():
        plan_adj.adjoint(y.data_ptr(), gx.data_ptr(), sp)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        return max_over_ranks(e0.elapsed_time(e1) / steps)

    def timed_trials(fn, steps, warmup, min_s=1.5, max_trials=50):
        """The K-step measurement above, repeated until about min_s seconds of
        device time have passed (so that the clock sampler sees the GPU under
        load for many samples); returns (median ms per step, trial count)."""
        first = timed(fn, steps, warmup)
        vals = [first]
        want = min(max_trials, max(1, int(min_s * 1e3 / max(first * steps, 1e-3))))
        while len(vals) < want:
            vals.append(timed(fn, steps, 0))
        return statistics.median(vals), len(vals)

    try:
        gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
        gpu_id = gpu_id if gpu_id.startswith("GPU-") else f"GPU-{gpu_id}"
    except Exception:
        gpu_id = str(local)
    clocks = ClockSampler(gpu_id)
    clocks.start()
    ms_fwd, trials_fwd = timed_trials(fwd, args.steps, args.warmup)
    ms_adj, trials_adj = timed_trials(adj, args.steps, args.warmup)
    clk = clocks.stop()
    plan.status_poll()
    plan_adj.status_poll()

    # per-kernel device time: events around each launch, launches serialised
    # on the bench stream so that each bracketed kernel has the GPU to itself,
    # on plans with the timed plans' own execution options (the same
    # segments, launches and work lists as the timed steps)
    def kernel_times(opts, direction):
        kp = _lib.Plan(lengths, len(lengths), real_input=real_input, graph=False, opts=opts)
        kp.timing_enable(True, serial=True)
        for _ in range(2):
            if direction == "fwd":
                kp.forward(xt.data_ptr(), y.data_ptr(), sp)
            else:
                kp.adjoint(y.data_ptr(), gx.data_ptr(), sp)
        kt = kp.timing_read()
        kp.timing_enable(False)
        kp.status_poll()
        kp.close()
        return kt

    kf = kernel_times(plan.opts(), "fwd")
    ka = kernel_times(plan_adj.opts(), "adj")

    peak, peak_src = measured_peaks()

    # a two-pass level is one unit: the cols launch writes only the plan's
    # intermediate (no algorithmic bytes), the rows launch writes the level
    partner = {"fwd_cols": "fwd_rows", "adj_cols": "adj_rows"}

    def dominant(kt, total_ms_per_step, opts):
        units = {}
        for k, (ms, n, b) in kt.items():
            if k in partner:
                continue
            units[k] = [ms, n, b, [k]]
        for k, p in partner.items():
            if k in kt and p in units:
                units[p][0] += kt[k][0]
                units[p][3].insert(0 if k.endswith("cols") and p.startswith("fwd") else 1, k)
        name, (ms, n, b, parts) = max(units.items(), key=lambda kv: kv[1][0])
        per_launch_ms = ms / n
        bytes_per_launch = b / n
        ach = bytes_per_launch / (per_launch_ms * 1e-3) / 1e9 if bytes_per_launch else 0.0
        # DRAM bytes per launch of each part (profiles/ncu_traffic.txt), summed
        # over the part's launches and spread over the unit's launches (a
        # dual-level cols launch serves two rows launches)
        traffic = None
        tr = [ncu_traffic(q, traffic_key(args.workload, opts)) for q in parts]
        if all(t is not None for t in tr):
            traffic = int(sum(t * kt[q][1] for t, q in zip(tr, parts)) / n)
        share = ms / sum(v[0] for v in kt.values())
        return {"bound": "hbm", "kernel": "+".join(f"k_{q}" for q in parts), "achieved": round(ach, 1),
                "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4), "traffic": traffic,
                "alg_bytes_per_launch": int(bytes_per_launch), "ms_per_launch": round(per_launch_ms, 4),
                "share_of_kernel_time": round(share, 3), "peak_source": peak_src,
                "timing": ("CUDA events around every launch on the bench stream, launches serialised, "
                           "2 steps of the timed plan's own execution options"),
                "traffic_key": traffic_key(args.workload, opts),
                "per_kernel_ms_per_step": {k: round(v[0] / 2, 4) for k, v in kt.items()},
                "per_kernel_gbs": {k: round(v[2] / (v[0] * 1e-3) / 1e9, 1) for k, v in kt.items() if v[2]}}

    roof_fwd = dominant(kf, ms_fwd, plan.opts())
    roof_adj = dominant(ka, ms_adj, plan_adj.opts())
    total_samples = replicas.sum_over_ranks(nsamp, device=dev)
    value = replicas.job_throughput(total_samples, ms_fwd) / 1e9
    value_adj = replicas.job_throughput(total_samples, ms_adj) / 1e9
    step_frac = alg_bytes / (ms_fwd * 1e-3) / 1e9 / peak
    step_frac_adj = alg_bytes / (ms_adj * 1e-3) / 1e9 / peak

    # comparison: the method of computing every level separately (one batched
    # cuFFT of all windows per level, through torch.fft) into the same output
    cufft = None
    if not args.no_cufft:
        def per_level_fft():
            xs = xt.to(torch.complex64) if real_input else xt
            if len(set(lengths)) == 1:
                n = lengths[0]
                m = log2i(n)
                xv = xs.view(len(lengths), n)
                yv = y.view(len(lengths), m, n)
                for i in range(1, m + 1):
                    torch.fft.fft(xv.view(len(lengths), n >> i, 1 << i),
                                  out=yv[:, i - 1, :].view(len(lengths), n >> i, 1 << i))
            else:
                yo = 0
                xo = 0
                for n in lengths:
                    m = log2i(n)
                    for i in range(1, m + 1):
                        torch.fft.fft(xs[xo:xo + n].view(-1, 1 << i), out=y[yo + (i - 1) * n:yo + i * n].view(-1, 1 << i))
                    xo += n
                    yo += m * n
        ksteps = max(3, min(args.steps, 20))
        ms_fft = timed(per_level_fft, ksteps, 3)
        cufft = {"ms_per_step": round(ms_fft, 4), "value": round(total_samples / (ms_fft * 1e-3) / 1e9, 4),
                 "unit": "Gsamples/s", "mrdft_speedup": round(ms_fft / ms_fwd, 3),
                 "what": "every level computed separately: one batched cuFFT (torch.fft.fft) of all windows per level, "
                         "written into the same output layout"}

    # training step for fitting the level spectra to targets T (uniform batches):
    # L = sum_i 2^-i ||Y_i - T_i||^2 and dL/dx*, fused (mrdft_loss_grad: the
    # adjoint reads Y and T) against forward + residual in torch + adjoint
    train = None
    if not args.no_train and len(set(lengths)) == 1:
        n = lengths[0]
        m = log2i(n)
        B = len(lengths)
        gen = torch.Generator(device=dev)
        gen.manual_seed(5 + 1000 * rank)
        tt = torch.randn((B, m, n), dtype=torch.complex64, device=dev, generator=gen)
        loss_t = torch.zeros((), dtype=torch.float64, device=dev)
        wlev = torch.tensor([2.0 ** -(i + 1) for i in range(m)], dtype=torch.float32, device=dev).view(1, m, 1)

        def fused():
            plan.loss_grad(xt.data_ptr(), tt.data_ptr(), y.data_ptr(), gx.data_ptr(), loss_t.data_ptr(), sp)

        def unfused():
            plan.forward(xt.data_ptr(), y.data_ptr(), sp)
            gy = (2.0 * wlev) * (y.view(B, m, n) - tt)
            plan.adjoint(gy.data_ptr(), gx.data_ptr(), sp)

        ksteps = max(3, min(args.steps, 20))
        ms_fused = timed(fused, ksteps, 3)
        ms_unfused = timed(unfused, ksteps, 3)
        train = {"fused_ms": round(ms_fused, 4), "unfused_ms": round(ms_unfused, 4),
                 "speedup": round(ms_unfused / ms_fused, 3),
                 "what": "L = sum_i 2^-i ||Y_i - T_i||^2 and dL/dx*: mrdft_loss_grad vs mrdft_forward + "
                         "torch residual + mrdft_adjoint; T ~ CN(0,1) seeded on the device"}
        del tt

    # end to end through the C ABI with host buffers (H2D + transform + D2H)
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(x_np).pin_memory()
        yh = torch.empty(plan.out_elems, dtype=torch.complex64).pin_memory()
        s2 = torch.cuda.Stream(dev)
        for _ in range(2):
            plan.forward_host(xh.data_ptr(), yh.data_ptr(), s2.cuda_stream)
        e2e_steps = max(3, min(args.steps, 10))
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            plan.forward_host(xh.data_ptr(), yh.data_ptr(), s2.cuda_stream)
        dt = (time.perf_counter() - t0) / e2e_steps
        dt = max_over_ranks(dt)
        e2e = {"value": total_samples / dt / 1e9, "unit": "Gsamples/s", "ms_per_step": dt * 1e3,
               "h2d_bytes_per_step": int(xh.numel() * xh.element_size()),
               "d2h_bytes_per_step": int(yh.numel() * yh.element_size()),
               "api": "mrdft_forward_host (pinned host buffers)"}
        del xh, yh

    others = None
    if not args.no_others and world == 1:
        others = {}
        for name in OTHER_WORKLOADS:
            if name != args.workload:
                others[name] = measure_other(name, dev, stream, timed, not args.no_autotune, peak)

    cpu = None
    check = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sdesc = oracle_sample(lengths, x_np, budget_s=15.0)
        cpu = {"value": v / 1e9, "unit": "Gsamples/s", "cores": cores, "kind": "oracle", "sample": sdesc}
        # the output of the last timed forward, checked on sampled bins
        plan.forward(xt.data_ptr(), y.data_ptr(), sp)
        torch.cuda.synchronize(dev)
        ok, check = self_check(y, x_np, lengths)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "Gsamples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_fwd, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "desc": desc, "signals": len(lengths),
                       "samples_per_gpu": nsamp, "alg_bytes_per_step_per_gpu": alg_bytes,
                       "l2": "inputs and outputs larger than L2 (no flush needed)" if alg_bytes > 2e8
                       else "working set smaller than L2",
                       "parallelism": f"signals sharded over {world} rank(s), no collective in the path",
                       "graph": True,
                       "exec_opts": {"forward": plan.opts(), "adjoint": plan_adj.opts(),
                                     "chosen_by": ("autotuner per direction: shape, then kernel variants"
                                                   if not args.no_autotune else "library defaults")},
                       "kernel_source": kernel_source_hash()},
            "hbm_frac_step": round(step_frac, 4),
            "timing_trials": {"forward": trials_fwd, "adjoint": trials_adj,
                              "what": "each trial times exactly `steps` steps between barriers and device "
                                      "synchronisations with CUDA events; ms_per_step is the median trial"},
            "roofline": roof_fwd,
            "adjoint": {"value": round(value_adj, 4), "unit": "Gsamples/s", "ms_per_step": round(ms_adj, 4),
                        "hbm_frac_step": round(step_frac_adj, 4), "roofline": roof_adj},
            "e2e": e2e,
            "per_level_cufft": cufft,
            "train_step": train,
            "cpu_baseline": cpu,
            "clocks": clk,
            "self_check": check,
            "other_workloads": others,
            "gpu_launches": int(args.steps * info["fwd_launches"]),
            "gpu_launches_adjoint": int(args.steps * info_adj["adj_launches"]),
        }
        print(json.dumps(line), flush=True)
        if check is not None and not check["ok"]:
            print("bench: the timed forward's output does not match the oracle on sampled bins", file=sys.stderr)
            return 1
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
