#!/usr/bin/env python
"""Benchmark of the GB300 CT-AUX walker (one JSON line on rank 0).

A step is one sweep per walker of the workload: proposals, candidate
extension, Metropolis decisions with the Gamma (B^-1) growth, the N update with
compaction, the measurement of G(tau) that ends the sweep and the periodic
recompute of N.  Under the lockstep schedule every walker runs one sweep;
under the pooled schedule the walkers together run n_walkers sweeps, each
taking part in every window (walkers of small order then run more sweeps).  The metric is walker vertex updates per second (decided
proposals per second, all walkers, all ranks) and the N-update TFLOP/s.

  python bench.py [--workload NAME] [--steps K] [--warmup W] [--gpus N]
  python bench.py --impl reference ...   # the oracle on the host cores

Multi-GPU: replicas only (independent Markov chains per rank, no collective
on the data path; the ranks only meet at the timing barriers).
"""
import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1901_01047_gb300 import inputs  # noqa: E402

# The configuration the throughput and roofline targets are stated on: 256
# independent walkers of uneven order in one batch, mixed precision,
# autotuned k_s.
DEFAULT_WORKLOAD = "batched256"
METRIC = "walker vertex updates/sec"
UNIT = "updates/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# Nominal GB300 FP64 rate (the recipe's figure); the FP64 path is bound by it.
FP64_TFLOPS = 1.25
# Dense TF32 / BF16 tensor rate ratio from the nominal figures (1.1 / 2.25),
# applied to the measured BF16 peak.
TF32_PER_BF16 = 1.1 / 2.25
# Mixed-path recompute, bound by FP32 issue: 152 SMs x 128 FP32 lanes x 2.07 GHz
# = 40.3e12 instructions/s.  The residual I - A N (2n^3 flop) takes 11 FP32
# instructions per double-float multiply-add (2 flop), the correction N R
# (2n^3 flop) one FMA per 2 flop, so the 4n^3 flop of a recompute run at most
# at 4 / (2 / 7.32 + 2 / 80.5) TFLOP/s.
FP32_INSTR_PER_S = 152 * 128 * 2.07e9
MIXED_RECOMPUTE_TFLOPS = 4.0 / (2.0 / (FP32_INSTR_PER_S * 2 / 11 / 1e12) + 2.0 / (FP32_INSTR_PER_S * 2 / 1e12))
# With the residual from digit planes on the tensor cores (the default), its
# 2n^3 flop take 17 FP16 plane products of 2n^3 flop each at the measured
# dense 16-bit tensor rate (the sustained BF16 figure: FP16 runs at the same
# rate), the correction 2n^3 flop at the FP32 issue rate.
OZ_PRODUCTS = 17


def sliced_recompute_tflops(peaks):
    p16 = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
    return 4.0 / (2.0 * OZ_PRODUCTS / p16 + 2.0 / (FP32_INSTR_PER_S * 2 / 1e12))

# DRAM bytes (read + write) per window of a kernel group from ncu captures of
# the named workload (one window of the pooled schedule carries all walkers;
# mean of two captured launches per kernel), quoted as `traffic` for that group
# on that workload only:
#   update  k_upd_tc 789.1 MB read + 457.0 MB written;
#   extend  k_cand_zero 56.0 + 86.7, k_ext_g_tc 664.6 + 44.2, k_ext_x_tc
#           654.2 + 23.2, k_cand_cc 101.1 + 1.5 (MB read + written).
NCU_TRAFFIC = {("batched256", "update"): 1.246e9, ("batched256", "extend"): 1.632e9}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def order_stats(stats):
    k = [s["order"] for s in stats]
    return {"min": min(k), "mean": sum(k) / len(k), "max": max(k)}


def workload_of(args):
    wl = inputs.WORKLOADS[args.workload]
    if getattr(args, "schedule", None):
        wl = dataclasses.replace(wl, schedule=args.schedule)
    if getattr(args, "duplicate_rule", None):
        wl = dataclasses.replace(wl, duplicate_rule=args.duplicate_rule)
    if getattr(args, "walkers", None):
        wl = dataclasses.replace(wl, walkers=args.walkers)
    return wl


def config_of(wl, world):
    return {"workload": wl.name, "nc": wl.nc, "t": wl.t, "tp": wl.tp, "U": wl.U, "beta": wl.beta, "mu": wl.mu,
            "K": wl.K, "walkers_per_gpu": wl.walkers, "k_sub": wl.k_sub, "n_tau": wl.n_tau,
            "n_tau_meas": wl.n_tau_meas, "recompute_every": wl.recompute_every, "recompute_sweeps": wl.recompute_sweeps,
            "recompute_at_measure": wl.recompute_at_measure, "n_omega_meas": wl.n_omega_meas,
            **({"freq_method": wl.freq_method} if wl.n_omega_meas else {}),
            **({"n_w4": wl.n_w4, "w4_transfer": wl.w4_transfer, "q4_transfer": wl.q4_transfer} if wl.n_w4 else {}),
            "precision": wl.precision, "schedule": wl.schedule, "duplicate_rule": wl.duplicate_rule,
            "recompute_method": wl.recompute_method,
            "parallelism": "replicas%d" % world, "l2": "flushed between steps (256 MB write)",
            **({"per_walker": {"nc": list(wl.nc_choices), "beta": list(wl.beta_range), "U": list(wl.U_range),
                               "mu": "U/2"}} if wl.nc_choices else {})}


def build_problem(pp, use_gpu_builder):
    c = inputs.cluster(pp["nc"])
    eps = inputs.square_dispersion(c.kpts, pp["t"], pp["tp"])
    kr = inputs.k_dot_r(c)
    if use_gpu_builder:
        from paper_1901_01047_gb300 import walker
        G0 = walker.g0_isolated_cluster(eps, kr, pp["mu"], pp["U"], pp["beta"], pp["n_tau"])
    else:
        from oracle import g0 as og0
        G0 = og0.g0_table(eps, kr, pp["mu"], pp["U"], pp["beta"], pp["n_tau"])
    return dict(nc=pp["nc"], site_sub=c.site_sub, U=pp["U"], beta=pp["beta"], K=pp["K"], G0=G0, k_dot_r=kr,
                k_sub=c.k_sub)


def workload_problems(wl, use_gpu_builder):
    params, walker_problem = wl.problem_params()
    return [build_problem(pp, use_gpu_builder) for pp in params], walker_problem


# --------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, on a bounded sample of the workload
# --------------------------------------------------------------------------
def _oracle_worker(stats, stop, ready, wl_name, walker_id, seed):
    """One oracle walker of the workload in its own process: warmed up once,
    then sweeping until told to stop, publishing after every sweep its decided
    proposals, the time (monotonic clock) and the sweep count."""
    sys.path.insert(0, ROOT)
    from oracle import ctaux
    wl = inputs.WORKLOADS[wl_name]
    params, walker_problem = wl.problem_params()
    pr = build_problem(params[walker_problem[walker_id % len(walker_problem)]], use_gpu_builder=False)
    w = ctaux.OracleWalker(pr["nc"], pr["site_sub"], pr["U"], pr["beta"], pr["K"], pr["G0"],
                           warmup_sweeps=wl.warmup_sweeps,
                           n_tau_meas=wl.n_tau_meas, seed=seed, walker_id=walker_id,
                           init_config_size=wl.init_config_size)
    w.sweep(wl.warmup_sweeps)
    sweeps = 0

    def publish():
        with stats.get_lock():
            stats[0] = float(w.counters()["proposals"])
            stats[1] = time.perf_counter()
            stats[2] = float(sweeps)

    publish()
    ready.set()
    while not stop.is_set():
        w.sweep(1)
        sweeps += 1
        publish()


class OraclePool:
    """The oracle on the host cores: one walker of the workload per core
    (spawned processes), each warmed up once and then sweeping continuously.
    The rate between two snapshots is the sum over walkers of decided
    proposals over time, each walker between its own sweep boundaries."""

    def __init__(self, wl_name):
        import multiprocessing as mp
        wl = inputs.WORKLOADS[wl_name]
        self.wl = wl
        self.cores = max(1, min(wl.walkers, os.cpu_count() or 1))
        ctx = mp.get_context("spawn")
        self.stop = ctx.Event()
        self.stats, self.ready, self.procs = [], [], []
        for i in range(self.cores):
            st = ctx.Array("d", 3)
            ev = ctx.Event()
            p = ctx.Process(target=_oracle_worker, args=(st, self.stop, ev, wl_name, i, wl.seed), daemon=True)
            p.start()
            self.stats.append(st)
            self.ready.append(ev)
            self.procs.append(p)
        for ev in self.ready:
            if not ev.wait(timeout=1800):
                raise RuntimeError("oracle warm-up did not finish")

    def snapshot(self):
        out = []
        for st in self.stats:
            with st.get_lock():
                out.append((st[0], st[1], st[2]))
        return out

    def advanced(self, s0, limit=600.0):
        """Wait until every walker has finished a sweep after snapshot s0."""
        t0 = time.perf_counter()
        while True:
            s1 = self.snapshot()
            if all(b[1] > a[1] for a, b in zip(s0, s1)) or time.perf_counter() - t0 > limit:
                return s1
            time.sleep(0.02)

    def measure(self, s0, s1, seconds):
        rate = sum((b[0] - a[0]) / (b[1] - a[1]) for a, b in zip(s0, s1) if b[1] > a[1])
        sample = "%d walkers, one per core, %d measured sweeps in %.1f s (after %d warm-up sweeps each)" % (
            self.cores, int(sum(b[2] - a[2] for a, b in zip(s0, s1))), seconds, self.wl.warmup_sweeps)
        return {"value": rate, "unit": UNIT, "cores": self.cores, "kind": "oracle", "sample": sample}

    def close(self):
        self.stop.set()
        for p in self.procs:
            p.join(timeout=120)
            if p.is_alive():
                p.terminate()


def g_error_sample(wl, k_sub, stream, warmup=17, measured=6):
    """G error of the workload's mixed-precision arithmetic against the oracle
    on identical trajectories: two of its walkers (the problems with beta
    nearest 10 and 15) are run by the oracle (warm-up with the batched
    recompute at sweeps 8 and 16, then measured sweeps) and replayed on the
    GPU with the oracle's decisions, under both recompute schedules of the
    mixed path; value = max over walkers of max|G - G_oracle| / max|G_oracle|
    of the accumulated sign * G."""
    import threading
    import numpy as np
    from oracle import ctaux
    from paper_1901_01047_gb300 import walker
    params, wp = wl.problem_params()
    betas = np.array([p["beta"] for p in params])
    picks = sorted({int(np.argmin(np.abs(betas - b))) for b in (10.0, 15.0)})
    probs = {i: build_problem(params[wp[i]], use_gpu_builder=False) for i in picks}
    sweeps = warmup + measured
    runs = {}

    def run_oracle(i):
        # walker index within the sample: the GPU handle of the sample keys its
        # Philox streams by that index
        pr = probs[i]
        ow = ctaux.OracleWalker(pr["nc"], pr["site_sub"], pr["U"], pr["beta"], pr["K"], pr["G0"],
                                warmup_sweeps=warmup, n_tau_meas=wl.n_tau_meas, seed=wl.seed,
                                walker_id=picks.index(i), init_config_size=wl.init_config_size)
        ow.enable_log(1 << 24)
        ow.sweep(sweeps)
        runs[i] = (ow.log(), ow.G(), ow.order)

    th = [threading.Thread(target=run_oracle, args=(i,)) for i in picks]
    for t in th:
        t.start()
    for t in th:
        t.join()
    out = {"norm": "max|G - G_oracle| / max|G_oracle| of the accumulated sign * G",
           "sample": "walkers %s of the workload (N_c %s, beta %s, order %s after %d sweeps), %d warm-up and %d "
                     "measured sweeps, the oracle's decisions replayed, k_s = %d" % (
                         picks, [params[wp[i]]["nc"] for i in picks], [round(params[wp[i]]["beta"], 2) for i in picks],
                         [runs[i][2] for i in picks], sweeps, warmup, measured, k_sub)}
    for fresh in (wl.recompute_at_measure, not wl.recompute_at_measure):
        gw = walker.Walkers([probs[i] for i in picks], n_walkers=len(picks), k_sub=k_sub, recompute_every=0,
                            recompute_sweeps=wl.recompute_sweeps, warmup_sweeps=warmup, n_tau_meas=wl.n_tau_meas,
                            precision="mixed", init_config_size=wl.init_config_size, seed=wl.seed,
                            recompute_at_measure=fresh, log_capacity=1 << 24, duplicate_rule=wl.duplicate_rule,
                            stream=stream.cuda_stream)
        errs = []
        for j, i in enumerate(picks):
            gw.set_forced_decisions(j, runs[i][0])
        gw.sweep(sweeps)
        G, ss, nm = gw.measure_G()
        for j, i in enumerate(picks):
            Go = runs[i][1][0]
            errs.append(float(np.abs(G[j] - Go).max() / np.abs(Go).max()))
        gw.close()
        key = "value" if fresh == wl.recompute_at_measure else "other_recompute"
        out[key] = max(errs)
        out[key + "_per_walker"] = errs
    out["recompute_at_measure"] = wl.recompute_at_measure
    return out


def cpu_baseline(wl_name, seconds=12.0):
    pool = OraclePool(wl_name)
    try:
        s0 = pool.snapshot()
        t0 = time.perf_counter()
        time.sleep(seconds)
        s1 = pool.advanced(s0)
        return pool.measure(s0, s1, time.perf_counter() - t0)
    finally:
        pool.close()


def run_reference(args, rank):
    if rank != 0:
        return
    wl = workload_of(args)
    # the walkers are warmed up once; the timed steps together sample about a minute
    per_step = max(0.2, min(10.0, 60.0 / max(1, args.steps + args.warmup)))
    pool = OraclePool(args.workload)
    try:
        for _ in range(args.warmup):
            time.sleep(per_step)
        s0 = pool.snapshot()
        t0 = time.perf_counter()
        for _ in range(args.steps):  # each step: per_step seconds of every walker's sweeps
            time.sleep(per_step)
        s1 = pool.advanced(s0)
        dt = time.perf_counter() - t0
        cb = pool.measure(s0, s1, dt)
    finally:
        pool.close()
    v = cb["value"]
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * dt / max(1, args.steps),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": config_of(wl, args.gpus),
           "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_1901_01047_gb300 import walker

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    wl = workload_of(args)
    stream = torch.cuda.current_stream()
    probs, walker_problem = workload_problems(wl, use_gpu_builder=True)
    seed = wl.seed + 1000003 * rank
    gw = walker.Walkers(probs, n_walkers=wl.walkers, walker_problem=walker_problem, k_sub=wl.k_sub,
                        recompute_every=wl.recompute_every, recompute_sweeps=wl.recompute_sweeps,
                        warmup_sweeps=wl.warmup_sweeps, n_tau_meas=wl.n_tau_meas, precision=wl.precision,
                        init_config_size=wl.init_config_size, seed=seed, schedule=wl.schedule,
                        recompute_at_measure=wl.recompute_at_measure, n_omega_meas=wl.n_omega_meas,
                        freq_method=wl.freq_method, n_w4=wl.n_w4, w4_transfer=wl.w4_transfer,
                        q4_transfer=wl.q4_transfer, duplicate_rule=wl.duplicate_rule,
                        recompute_method=wl.recompute_method, stream=stream.cuda_stream)
    gw.sweep(wl.warmup_sweeps)            # the chain's own warm-up (no measurements)
    tuned = None
    if wl.autotune and not args.no_autotune:  # untimed; the trial sweeps are ordinary sweeps of the chains
        from paper_1901_01047_gb300 import autotune
        tuned = autotune.tune(gw, wl.precision, sweeps=2, settle=1)
    for _ in range(args.warmup):          # bench warm-up steps (measured sweeps, untimed)
        gw.sweep(1)

    # Calibration (untimed): which kernel group dominates a step, over one
    # recompute period of the batched schedule.
    gw.set_timing(walker.GROUPS)
    gw.timing(reset=True)
    cal_sweeps = max(3, wl.recompute_sweeps)
    for _ in range(cal_sweeps):
        gw.sweep(1)
    times, _ = gw.timing(reset=True)
    dominant = max(times, key=lambda g: times[g][0])

    # L2 flush buffer (larger than the 129 MB L2), written between steps.
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # Timed region 1 (the value): device-side window loop, no kernel events.
    # Under --profile-region the same kernels are launched from the host
    # instead (ncu does not see kernels inside conditional graph bodies).
    gw.set_timing(["propose"] if args.profile_region else [])
    st0 = gw.stats()
    gw.timing(reset=True)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    phys = vis.split(",")[local_rank] if vis and len(vis.split(",")) > local_rank else str(local_rank)
    clocks = ClockSampler(phys)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if args.profile_region:
        torch.cuda.profiler.start()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        gw.sweep(1, sync=False)  # enqueues the step; the events bracket the device work only
        ends[k].record(stream)
    torch.cuda.synchronize()
    if args.profile_region:
        torch.cuda.profiler.stop()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    gw.sync()  # raises if a walker stopped with an error during the timed steps
    st1 = gw.stats()
    _, launches = gw.timing(reset=True)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    dev_ms = sum(step_ms)

    # The same batch under the other schedule, for comparison (shorter, untimed for `value`).
    other = None
    if wl.schedule == "pooled" and not args.profile_region:
        gw.set_schedule("lockstep")
        gw.sweep(1)
        k_other = max(3, args.steps // 5)
        so0 = gw.stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(k_other):
            gw.sweep(1, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        gw.sync()
        so1 = gw.stats()
        o_props = sum(b["proposals"] - a["proposals"] for a, b in zip(so0, so1))
        o_ms = e0.elapsed_time(e1)
        other = {"schedule": "lockstep", "value": o_props / (o_ms / 1000.0), "unit": UNIT, "steps": k_other,
                 "ms_per_step": o_ms / k_other, "note": "one sweep of every walker per step; L2 not flushed"}
        gw.set_schedule(wl.schedule)

    # The other recompute schedule of the mixed path (N recomputed at every
    # measurement, or only every recompute_sweeps sweeps), same batch, shorter.
    alt = None
    if wl.precision == "mixed" and wl.recompute_sweeps > 0 and not args.profile_region:
        alt_fresh = not wl.recompute_at_measure
        gw.set_recompute(wl.recompute_every, wl.recompute_sweeps, alt_fresh)
        gw.sweep(1)
        k_alt = max(3, args.steps // 4)
        sa0 = gw.stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(k_alt):
            flush.fill_(float(k))
            gw.sweep(1, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        gw.sync()
        sa1 = gw.stats()
        a_props = sum(b["proposals"] - a["proposals"] for a, b in zip(sa0, sa1))
        a_ms = e0.elapsed_time(e1)
        alt = {"recompute_at_measure": alt_fresh, "value": a_props / (a_ms / 1000.0), "unit": UNIT, "steps": k_alt,
               "ms_per_step": a_ms / k_alt, "note": "L2 flush inside the events"}
        gw.set_recompute(wl.recompute_every, wl.recompute_sweeps, wl.recompute_at_measure)

    # Timed region 2 (the roofline): the same steps driven from the host with
    # CUDA events on the walker's stream around the dominant kernel group and
    # around the N-update kernel.
    gw.set_timing(sorted({dominant, "update", "recompute"}))
    st_k0 = gw.stats()
    for k in range(args.steps):
        flush.fill_(float(k))
        gw.sweep(1)
    torch.cuda.synchronize()
    gtimes, _ = gw.timing(reset=True)
    st_k1 = gw.stats()
    gw.set_timing([])
    props = sum(b["proposals"] - a["proposals"] for a, b in zip(st0, st1))
    flops = sum(b["n_update_flops"] - a["n_update_flops"] for a, b in zip(st0, st1))
    kflops = sum(b["n_update_flops"] - a["n_update_flops"] for a, b in zip(st_k0, st_k1))
    ubytes = sum(b["n_update_bytes"] - a["n_update_bytes"] for a, b in zip(st_k0, st_k1))
    eflops = sum(b["extend_flops"] - a["extend_flops"] for a, b in zip(st_k0, st_k1))
    ebytes = sum(b["extend_bytes"] - a["extend_bytes"] for a, b in zip(st_k0, st_k1))
    rkflops = sum(b["recompute_flops"] - a["recompute_flops"] for a, b in zip(st_k0, st_k1))
    work = {"update": (ubytes, kflops), "extend": (ebytes, eflops), "recompute": (None, rkflops)}
    rflops = sum(b["recompute_flops"] - a["recompute_flops"] for a, b in zip(st0, st1))
    seconds, props_all, flops_all, rflops_all = combine_ranks(dist, dev_ms / 1000.0, [float(props), flops, rflops],
                                                              "cuda")
    value = props_all / seconds

    # End to end through the public API with host buffers: every problem's bare
    # propagator uploaded from pinned memory (the per-iteration input of an
    # outer DCA loop; validated on the device), one step, and every walker's
    # G read back, every step.  The upload of step k + 1's tables is issued
    # while step k's sweep runs (the library copies on its own stream and
    # commits the tables after that sweep), as a pipelined caller would.
    G0_host = torch.from_numpy(np.concatenate([np.ascontiguousarray(p["G0"], np.float64).reshape(-1)
                                               for p in probs])).pin_memory()
    G0_np = G0_host.numpy()
    h2d = int(G0_host.numel() * 8)
    g_bytes = sum(2 * nc * wl.n_tau_meas * 8 for nc in gw.nc) + 16 * wl.walkers
    st2 = gw.stats()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    gw.update_G0_all(G0_np)  # the first step's tables
    for k in range(args.steps):
        gw.sweep(1, sync=False)
        if k + 1 < args.steps:
            # the next step's tables: one copy of every problem's table (overlapping
            # this step's sweep), checked and committed on the device after it
            gw.update_G0_all(G0_np)
        gw.measure_G()  # synchronises
    gw.sync()
    torch.cuda.synchronize()
    te = time.perf_counter() - te0
    st3 = gw.stats()
    e_props = sum(b["proposals"] - a["proposals"] for a, b in zip(st2, st3))
    e_sec, e_props_all = combine_ranks(dist, te, [float(e_props)], "cuda")
    e_value = e_props_all / e_sec

    if rank == 0:
        peaks, kind = _peaks()
        windows = max(1, gtimes["propose"][1])  # one proposal kernel per window
        roof = roofline(dominant, gtimes[dominant][0], windows, work, peaks, kind, wl)
        roof_upd = roofline("update", gtimes["update"][0], windows, work, peaks, kind, wl)
        roof["traffic"] = NCU_TRAFFIC.get((wl.name, dominant))
        roof_upd["traffic"] = NCU_TRAFFIC.get((wl.name, "update"))
        roof_rec = roofline("recompute", gtimes["recompute"][0], windows, work, peaks, kind, wl)
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * seconds / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if wl.precision == "fp64" else wl.precision,
            "data": "synthetic",
            "config": {**config_of(wl, world), "k_sub": gw.k_sub,
                       **({"autotune": {"k_sub": tuned["k_sub"], "update_kernel": tuned["update_kernel"],
                                        "update_tile": tuned["update_tile"],
                                        "updates_per_s": {"%d/%s" % (r["k_sub"], r["update_kernel"]):
                                                          round(r["updates_per_s"]) for r in tuned["table"]},
                                        "tile_update_group_updates_per_s": {str(r["update_tile"]): round(r["updates_per_s"])
                                                               for r in tuned["tiles"]}}}
                          if tuned else {})},
            "final_order": st1[0]["order"],
            "n_update_tflops": flops_all / seconds / 1e12,
            "wall_s": wall,
            "clocks": clk,
            "gpu_launches": launches,
            "kernel_ms": {g: round(v[0], 4) for g, v in times.items()},
            "roofline": roof,
            "n_update_roofline": roof_upd,
            "recompute_roofline": roof_rec,
            "orders": order_stats(st1),
            "recompute_tflops_fp64": rflops_all / seconds / 1e12,
            "e2e": {"value": e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": int(g_bytes)},
            "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms),
                        "stdev": statistics.pstdev(step_ms)},
            **({"other_schedule": other} if other else {}),
            **({"other_recompute": alt} if alt else {}),
        }
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.workload)
            if wl.precision == "mixed":
                out["g_error"] = g_error_sample(wl, gw.k_sub, stream)
        print(json.dumps(out))
    gw.close()
    if dist:
        dist.destroy_process_group()


def combine_ranks(dist, seconds, sums, device):
    """Whole-job figures of a replicas run: the slowest rank's time and the sum
    over ranks of the counted work.  Returns (max seconds, *sums over ranks)."""
    import torch
    t = torch.tensor([seconds] + list(sums), dtype=torch.float64, device=device)
    if dist is not None:
        tmax = t[:1].clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        rest = t[1:].clone()
        dist.all_reduce(rest, op=dist.ReduceOp.SUM)
        t = torch.cat([tmax, rest])
    return tuple(t.tolist())


def roofline(group, g_ms, windows, work, peaks, kind, wl):
    """Roofline of one kernel group from its CUDA-event time over the timed
    steps.  `work` maps a group to its algorithmic (bytes, flop) over the same
    steps; the recompute counts flop only (FP64 arithmetic bound)."""
    sec = g_ms / 1000.0
    launch_ms = g_ms / max(1, windows)
    base = {"kernel": group, "launch_ms": launch_ms, "traffic": None}
    if group not in work or sec <= 0:
        return {**base, "bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
                "note": "latency-bound kernel group without an algorithmic byte or flop count"}
    work_b, work_f = work[group]
    tfs = work_f / sec / 1e12
    if work_b is None:
        if wl.precision == "mixed" and wl.recompute_method == "auto":
            pk = sliced_recompute_tflops(peaks)
            return {**base, "bound": "tensor", "achieved": tfs, "peak": pk, "unit": "TFLOP/s", "frac": tfs / pk,
                    "peak_kind": "derived (%s): the residual's 2n^3 flop as %d FP16 plane products at the sustained "
                                 "16-bit tensor rate, the correction's 2n^3 at the FP32 issue rate (152 SMs x 128 "
                                 "lanes x 2.07 GHz)" % (kind, OZ_PRODUCTS)}
        if wl.precision == "mixed":
            return {**base, "bound": "alu", "achieved": tfs, "peak": MIXED_RECOMPUTE_TFLOPS, "unit": "TFLOP/s",
                    "frac": tfs / MIXED_RECOMPUTE_TFLOPS,
                    "peak_kind": "derived: FP32 issue rate (152 SMs x 128 lanes x 2.07 GHz), 11 instructions per "
                                 "double-float multiply-add in the residual, one FMA in the correction"}
        return {**base, "bound": "alu", "achieved": tfs, "peak": FP64_TFLOPS, "unit": "TFLOP/s",
                "frac": tfs / FP64_TFLOPS, "peak_kind": "nominal FP64 (recipe table)"}
    gbs = work_b / sec / 1e9
    hbm = peaks["hbm_gbs"]
    ai = work_f / max(work_b, 1.0)
    out = {**base, "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
           "peak_kind": kind, "tflops": tfs, "flop_per_byte": ai}
    if wl.precision == "fp64" and ai > FP64_TFLOPS * 1e12 / (hbm * 1e9):
        out.update({"bound": "alu", "achieved": tfs, "peak": FP64_TFLOPS, "unit": "TFLOP/s",
                    "frac": tfs / FP64_TFLOPS, "peak_kind": "nominal FP64 (recipe table)", "hbm_gbs": gbs})
    elif wl.precision == "mixed":
        tf32 = peaks["bf16_tflops"] * TF32_PER_BF16
        out.update({"tf32_peak_tflops": tf32, "tf32_frac": tfs / tf32})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(inputs.WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the workload's stored k_s and update kernel")
    ap.add_argument("--schedule", choices=["lockstep", "pooled"], default=None,
                    help="walker schedule (default: the workload's)")
    ap.add_argument("--duplicate-rule", choices=["abort", "update"], default=None,
                    help="a spin changed twice in one window (default: the workload's)")
    ap.add_argument("--walkers", type=int, default=None,
                    help="run only the first K walkers of the workload (small profiling captures; "
                         "the line is then not the workload's)")
    ap.add_argument("--profile-region", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu --profile-from-start off) "
                         "and launch the window kernels from the host in that region")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
