"""Benchmark of the nested-MLMC level path on GB300.

One step = one launch of the whole level work list of the nested workload:
European and digital call on GBM (S0 = K = 100, r = 0.05, sigma = 0.2, T = 1),
Euler-Maruyama, levels 0..8, approximate estimator (Method-1 table, d = 10,
fixed point with the default per-level formats) with N~_l = max(10^4, 10^7
2^-1.5l) samples and correction estimator (FP32 exact minus fixed point on
shared uniforms) with 10^4 samples per level.  Inputs (the work list and
tables) are resident in device memory when the timed region starts; L2 is
flushed between steps (256 MiB write) outside the per-step events.

Prints one JSON line.  `--impl reference` times the CPU oracle instead (the
reference arm).  Under torchrun each rank simulates a disjoint sample range
(first_sample offset by rank), the step time is the max over ranks and the
value is the path-steps of all ranks per second (weak scaling).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2502_07123_gb300 import workloads as W  # noqa: E402

METRIC = "time-to-ε price & path-steps/s: nested approx-RV vs plain MLMC; p50/p99 latency"
UNIT = "path-steps/s"
WORKLOAD = ("nested MLMC step: euro+digital call GBM, EM, levels 0-8, N~ 1e7..1e4 fixed-point approx "
            "(packed draws) + 1e4 FP32-fixed corrections")

# Algorithmic 32-bit lane operations per fine path-step (approximate fixed-point
# estimator, Euler-Maruyama, terminal payoff):
#   Philox4x32-10: 10 rounds x (2 wide multiplies + 2 three-input XORs) / 4 words = 10
#   table index, lookup and sign: 5
#   fixed-point Algorithm-1 fine step (2 products, 2 sums, 4 roundings): 10
#   coarse step every other fine step: (1 + 10) / 2 = 5.5
OPS_APPROX_FIXED_EM = 30.5
# level 0 has no coarse path (P_-1 = 0): 30.5 - 5.5
OPS_APPROX_FIXED_EM_L0 = 25.0
# Correction estimator (FP32 exact minus fixed point on the same J), Euler-Maruyama:
#   Philox4x32-10, one word per path-step: 10
#   exact Normal: U = 2^-32 (J + 1/2) with the symmetric fold 3, Phi^-1 in single
#     precision as a published algorithm computes it (Giles 2012: one logarithm,
#     a degree-8 polynomial by Horner, 8 further operations) 17
#   exact fine step 2 (increment, S update); coarse every other step (3) / 2 = 1.5
#   approximate part: index, lookup and sign 5, fine Algorithm-1 step 10, coarse 5.5
OPS_CORR_FIXED_EM = 54.0
# level 0: no coarse path, exact or approximate: 54 - 1.5 - 5.5
OPS_CORR_FIXED_EM_L0 = 47.0
# SM issue peak: 152 SMs x 4 schedulers x 32 lanes x 2070 MHz (one warp instruction per scheduler per clock)
ALU_PEAK_TOPS = 152 * 4 * 32 * 2.070e9 / 1e12
# DRAM bytes (read + write) of the dominant launch, from one ncu capture of this
# bench command (dram__bytes_read.sum + dram__bytes_write.sum of the merged
# nested launch in its pre-scaled form, family 24, 80,148,728 path-steps):
#   ncu --set full --clock-control none -k regex:^nested_kernel -s 2 -c 1 -o prof \
#       python bench.py --steps 3 --warmup 3 --no-cpu-baseline --no-tte \
#       --no-serving-sample --no-optimiser --no-sweep-levels
# keyed by (family, path-steps per launch); another launch reports null
DOMINANT_TRAFFIC = {(24, 80148728): 175872}


def build_items(m, rank=0, formats=None):
    """The nested workload's work items (per-level formats: the default schedule,
    or `formats`, a list indexed by level)."""
    cfg = W.nested_config()
    items, meta = [], []
    cache = {}
    for it in cfg["items"]:
        p = it["params"]
        key = p["payoff"]
        if key not in cache:
            fm = formats[:9] if formats else [W.default_format(p, lev) for lev in range(9)]
            cache[key] = m.make_params(p, d=cfg["d"], method=cfg["method"], formats=fm,
                                       request=it["request"], rng_pack=cfg["rng_pack"])
        items.append(dict(params=cache[key], level=it["level"], variant=it["variant"],
                          first_sample=rank * it["N"], N=it["N"]))
        meta.append(it)
    return items, meta, cfg


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dominant_alone(m, torch, items, seed, tuning, plan, j, flush, stream, reps=10):
    """Launch j of the step's plan (the dominant one) on its own: a plan of the
    same work items, timed with CUDA events with the GPU to itself, outside the
    timed region.  None unless that plan is exactly one launch of the same
    family and path-steps."""
    fam, _, _, ps = plan.launch_info(j)
    sub_plan = m.Plan([items[i] for i in plan.launch_items(j)], seed, tuning)
    try:
        if sub_plan.info()["kernels"] != 1 or sub_plan.launch_info(0)[0] != fam or sub_plan.launch_info(0)[3] != ps:
            return None
        for _ in range(3):
            sub_plan.launch(stream)
        ms = []
        for _ in range(reps):
            flush.zero_()
            sub_plan.launch(stream)
            ms.append(sub_plan.kernel_time(0)[1])
        torch.cuda.synchronize()
        return statistics.median(ms)
    finally:
        sub_plan.close()


def _oracle_share(task):
    """One host process's share of the oracle sample: (item index, meta item,
    first sample, count) quadruples; returns the path-steps simulated and the
    oracle's sums of each share."""
    from oracle import core
    shares, cfg = task
    steps, sums = 0, []
    for k, it, first, n in shares:
        p = it["params"]
        fmt = W.default_format(p, it["level"]) if it["variant"] in (W.FIXED_APPROX, W.CORR_FIXED) else None
        o, _ = core.level(p, it["level"], first, n, it["variant"], cfg["seed"], request=it["request"],
                          d=cfg["d"], method=cfg["method"], fmt=fmt,
                          pack=cfg["rng_pack"] if it["variant"] == W.FIXED_APPROX else 0)
        steps += n << it["level"]
        sums.append((k, o["sum"], o["sum2"], o["isum"], o["isum2"]))
    return steps, sums


class OraclePool:
    """The CPU oracle on every host core: spawned worker processes (started
    after the GPU is in use, so never forked), each taking a contiguous share
    of every work item's samples."""

    def __init__(self):
        import multiprocessing as mp
        from oracle import build as ob
        ob.build()
        try:
            self.cores = len(os.sched_getaffinity(0))
        except AttributeError:
            self.cores = os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.pool.map(_oracle_share, [([], {})] * self.cores)   # start and import in every worker

    def step(self, meta, cfg, fraction, rank=0, sums=None):
        """Samples [rank N, rank N + fraction N) of every item; returns (path_steps,
        seconds); with a list `sums`, also each item's oracle sums (undiscounted:
        sum, sum2, exact integer isum, isum2) appended to it."""
        shares = [[] for _ in range(self.cores)]
        for k, it in enumerate(meta):
            n = max(1, int(it["N"] * fraction))
            base = rank * it["N"]
            for c in range(self.cores):
                lo, hi = n * c // self.cores, n * (c + 1) // self.cores
                if hi > lo:
                    shares[c].append((k, it, base + lo, hi - lo))
        t0 = time.perf_counter()
        out = self.pool.map(_oracle_share, [(sh, cfg) for sh in shares])
        dt = time.perf_counter() - t0
        if sums is not None:
            acc = [[0.0, 0.0, 0, 0] for _ in meta]
            for _, part in out:
                for k, s1, s2, i1, i2 in part:
                    acc[k][0] += s1
                    acc[k][1] += s2
                    acc[k][2] += i1
                    acc[k][3] += i2
            sums.extend(acc)
        return sum(x[0] for x in out), dt

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args):
    """Reference arm: the CPU oracle on all host cores, same workload, one step's
    first `--ref-fraction` of every work item per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg = W.nested_config()
    meta = cfg["items"]
    frac = args.ref_fraction
    pool = OraclePool()
    try:
        for _ in range(args.warmup):
            pool.step(meta, cfg, frac * 0.1)
        tot_steps, tot_s = 0, 0.0
        for _ in range(args.steps):
            s_, dt = pool.step(meta, cfg, frac)
            tot_steps += s_
            tot_s += dt
    finally:
        pool.close()
    v = tot_steps / tot_s
    sample = "first %.3g of every work item per step, split over %d processes" % (frac, pool.cores)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": pool.cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def workload_config():
    """The benchmark's workload (the same for both arms)."""
    cfg = W.nested_config()
    return {"workload": WORKLOAD, "path_steps_per_step": sum(it["N"] << it["level"] for it in cfg["items"]),
            "work_items": len(cfg["items"]), "l2": "flushed between steps (256 MiB write)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--steps-per-thread", type=int, default=0)
    ap.add_argument("--cpu-fraction", type=float, default=1.0)
    ap.add_argument("--ref-fraction", type=float, default=1.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tte", action="store_true")
    ap.add_argument("--no-serving-sample", action="store_true")
    ap.add_argument("--no-optimiser", action="store_true")
    ap.add_argument("--no-sweep-levels", action="store_true",
                    help="skip the brief level-kernel sweep (levels 0-10, every variant, 2^22 paths)")
    ap.add_argument("--sweep", action="store_true",
                    help="also run the level-kernel throughput sweep (Milstein; payoffs x variants x levels)")
    ap.add_argument("--autotune", action="store_true",
                    help="time launch shapes per kernel class first and use the fastest (the default is the "
                         "library's fixed shape table, so that a profile of the same command sees the same launches)")
    ap.add_argument("--serving", action="store_true",
                    help="also run the batched (256 options) and serving (Poisson arrivals) workloads")
    ap.add_argument("--serving-sample-n", type=int, default=200,
                    help="requests per arrival rate of the bounded serving sample (eps in [1e-3, 1e-2])")
    ap.add_argument("--serving-n", type=int, default=200,
                    help="requests per arrival rate of --serving (full accuracy range)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2502_07123_gb300 import mlmc as m

    items, meta, cfg = build_items(m, rank)
    tuning = None
    shape = "library default shape table"
    if args.threads or args.steps_per_thread:
        tuning = dict(threads=args.threads, steps_per_thread=args.steps_per_thread)
        shape = "fixed %d threads x %d path-steps per thread" % (args.threads, args.steps_per_thread)
    elif args.autotune:
        # launch shape per kernel class, timed on this GPU (outside the timed region)
        shapes = m.mlmc_autotune(items, cfg["seed"], reps=3)
        shape = "autotuned per kernel class: " + ", ".join("%dx%d" % t for t in sorted(set(shapes)))
    plan = m.Plan(items, cfg["seed"], tuning)
    info = plan.info()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    for _ in range(max(3, args.warmup)):
        plan.launch(stream)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # a step's device time: the plan's own CUDA events on the launch stream,
    # recorded right before its first kernel and after its last (the L2 flush
    # runs before them; mlmc_plan_elapsed waits for the step)
    step_ms = []
    kern_ms = {}
    launch_ms = {}
    with ClockSampler(local) as clocks:
        barrier()
        t_wall = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            plan.launch(stream)
            step_ms.append(plan.elapsed_ms())
            for j in range(info["kernels"]):
                fam, ms = plan.kernel_time(j)
                kern_ms.setdefault(fam, []).append(ms)
                launch_ms.setdefault(j, []).append(ms)
        barrier()
        t_wall = time.perf_counter() - t_wall
    local_ms = sum(step_ms) / len(step_ms)
    ms = local_ms
    if world > 1:
        t = torch.tensor([local_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    steps_per_launch = info["path_steps"] * world
    value = steps_per_launch / (ms * 1e-3)

    # results of the last launch, merged over ranks on the host (no data-path collective)
    res = plan.results()

    # end-to-end: the same work through the host-buffer C-ABI call (plan build,
    # H2D of the work descriptors through pinned staging, launch, the sums
    # written device-to-host into mapped pinned memory by each item's last CTA,
    # results as one structured array) on a work list marshalled once
    work = m.WorkList(items)
    e2e_ms = []
    for _ in range(max(3, min(10, args.steps))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m.mlmc_run(work, cfg["seed"], tuning, raw=True)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_value = info["path_steps"] / (statistics.median(e2e_ms) * 1e-3)

    # roofline of the dominant kernel: the launch with the most path-steps among
    # the fixed-point families (24 / 17: the merged nested launch of the approximate
    # and correction chunks, with / without the pre-scaled product; 15 / 8: approximate packed / one sample per thread,
    # 32-bit S; 12 / 2 general).  Its algorithmic ops are each estimator's ops
    # per path-step times that estimator's path-steps in the launch.
    fam_names = {24: "nested_kernel<FX32,EM,terminal,pre-scaled> (approximate packed + one sample per thread + "
                     "correction)",
                 17: "nested_kernel<FX32,EM,terminal> (approximate packed + one sample per thread + correction)",
                 15: "level_kernel<APPROX,F32,FX32,EM,terminal,packed x3>",
                 8: "level_kernel<APPROX,F32,FX32,EM,terminal>",
                 12: "level_kernel<APPROX,F32,FIXED,EM,terminal,packed x3>",
                 2: "level_kernel<APPROX,F32,FIXED,EM,terminal>"}
    launches = [plan.launch_info(j) for j in range(info["kernels"])]
    cand = [(ps, j, fam) for j, (fam, _, _, ps) in enumerate(launches) if fam in fam_names]
    roofline = None
    if cand:
        ps, j, dom = max(cand)
        idx = plan.launch_items(j)
        ps_a = sum(items[i]["N"] << items[i]["level"] for i in idx if items[i]["variant"] != W.CORR_FIXED)
        ps_c = sum(items[i]["N"] << items[i]["level"] for i in idx if items[i]["variant"] == W.CORR_FIXED)
        # level-0 path-steps have no coarse step
        ps_a0 = sum(items[i]["N"] for i in idx if items[i]["variant"] != W.CORR_FIXED and items[i]["level"] == 0)
        ps_c0 = sum(items[i]["N"] for i in idx if items[i]["variant"] == W.CORR_FIXED and items[i]["level"] == 0)
        ops = (OPS_APPROX_FIXED_EM * (ps_a - ps_a0) + OPS_APPROX_FIXED_EM_L0 * ps_a0
               + OPS_CORR_FIXED_EM * (ps_c - ps_c0) + OPS_CORR_FIXED_EM_L0 * ps_c0)
        dom_ms = sum(launch_ms[j]) / len(launch_ms[j])
        achieved = ops / (dom_ms * 1e-3) / 1e12
        fam_, _, ctas_, _ = launches[j]
        roofline = {"bound": "alu", "achieved": achieved, "peak": ALU_PEAK_TOPS, "unit": "Top/s",
                    "frac": achieved / ALU_PEAK_TOPS, "traffic": DOMINANT_TRAFFIC.get((dom, ps)),
                    "kernel": fam_names[dom], "ctas": ctas_,
                    "ms_per_launch": dom_ms,
                    "ops_per_path_step": {"approximate": OPS_APPROX_FIXED_EM, "correction": OPS_CORR_FIXED_EM,
                                          "approximate_level0": OPS_APPROX_FIXED_EM_L0,
                                          "correction_level0": OPS_CORR_FIXED_EM_L0},
                    "ops_per_launch": ops,
                    "path_steps_per_launch": ps, "approximate_path_steps": ps_a, "correction_path_steps": ps_c,
                    "level0_path_steps": {"approximate": ps_a0, "correction": ps_c0}}
        alone_ms = dominant_alone(m, torch, items, cfg["seed"], tuning, plan, j, flush, stream)
        if alone_ms:
            # the same launch with the GPU to itself (in the step it may share the
            # SMs with other level kernels)
            a = ops / (alone_ms * 1e-3) / 1e12
            roofline["alone"] = {"ms_per_launch": alone_ms, "achieved": a, "frac": a / ALU_PEAK_TOPS}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "i64+f32", "data": "synthetic",
        "config": workload_config(),
        "launch": {"kernels_per_step": info["kernels"], "ctas_per_step": info["ctas"], "launch_shape": shape,
                   "path_steps_per_step_all_ranks": steps_per_launch, "wall_s": t_wall},
        "gpu_launches": info["kernels"] * args.steps,
        "kernel_ms": {str(f): sum(v) / len(v) for f, v in kern_ms.items()},
        "clocks": clocks.summary(),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": info["h2d_bytes"],
                "d2h_bytes_per_step": info["d2h_bytes"], "ms": statistics.median(e2e_ms)},
        "roofline": roofline,
    }
    formats_opt = None
    if rank == 0 and world == 1 and not args.no_optimiser:
        out["bitwidth_optimiser"], formats_opt = optimiser_run(m, torch)
        out["nested_step_optimised_widths"] = nested_step_with_formats(m, torch, formats_opt, flush, stream)
    if rank == 0 and not args.no_tte:
        out["time_to_eps"] = time_to_eps(m, torch, formats_opt=formats_opt)
    if rank == 0 and world == 1 and args.sweep:
        out["sweep"] = sweep_run(m, torch)
    elif rank == 0 and world == 1 and not args.no_sweep_levels:
        # the level-kernel workload in brief: every level 0-10 and every variant
        # at 2^22 paths (Milstein, European call, sigma 0.2)
        out["sweep_levels"] = sweep_run(m, torch, levels=range(11), sizes=(1 << 22,), grid=False)
    if rank == 0 and world == 1 and not args.no_serving_sample:
        # bounded serving samples: 200 requests (--serving-sample-n) drawn as the
        # serving workload at 100, 1000 and 10000 req/s, accuracies in the coarser
        # half [1e-3, 1e-2] of its range (--serving runs the full range; its
        # eps ~ 1e-4 tail takes minutes)
        out["serving_sample"] = [serving_run(m, rate, n=args.serving_sample_n, eps_range=(1e-3, 1e-2))
                                 for rate in (100, 1000, 10000)]
    if rank == 0 and world == 1 and args.serving:
        out["batched"] = batched_run(m)
        out["serving"] = [serving_run(m, rate, n=args.serving_n) for rate in (100, 1000, 10000)]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = OraclePool()
        osums = []
        try:
            steps_c, secs = pool.step(meta, cfg, args.cpu_fraction, sums=osums)
        finally:
            pool.close()
        out["cpu_baseline"] = {"value": steps_c / secs, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                               "sample": "first %.3g of every work item of one step (%d path-steps, %.1f s), "
                                         "split over %d processes" % (args.cpu_fraction, steps_c, secs, pool.cores)}
        if args.cpu_fraction == 1.0:
            # the step's results against the FP64 oracle on the same samples: the
            # integer (approximate) items exactly, the real-valued (correction)
            # items by |sum difference| / sqrt(n sum2)
            int_equal, real_err = 0, []
            for it, r, o in zip(meta, res, osums):
                disc = math.exp(-it["params"]["r"] * it["params"]["T"])
                if r["exact_int"]:
                    int_equal += int(r["isum"] == o[2] and r["isum2"] == o[3])
                else:
                    scale = math.sqrt(r["n"] * disc * disc * o[1])    # >= sum |Y|; zero if every Y is
                    diff = abs(r["sum"] - disc * o[0])
                    real_err.append(diff / scale if scale > 0 else (0.0 if diff == 0 else float("inf")))
            out["cpu_baseline"]["step_vs_oracle"] = {
                "integer_items_bit_equal": "%d of %d" % (int_equal, sum(1 for r in res if r["exact_int"])),
                "real_items_max_rel_err_of_sum": max(real_err) if real_err else None}
    if rank == 0:
        print(json.dumps(out))
    plan.close()
    if world > 1:
        dist.destroy_process_group()


def _bs_price(o):
    """Black-Scholes value of a European or digital call (None for other payoffs)."""
    from scipy.stats import norm
    S0, K, r, sig, T = o["S0"], o["K"], o["r"], o["sigma"], o["T"]
    d1 = (math.log(S0 / K) + (r + 0.5 * sig * sig) * T) / (sig * math.sqrt(T))
    d2 = d1 - sig * math.sqrt(T)
    if o["payoff"] == W.EURO:
        return S0 * norm.cdf(d1) - K * math.exp(-r * T) * norm.cdf(d2)
    if o["payoff"] == W.DIGITAL:
        return math.exp(-r * T) * norm.cdf(d2)
    return None


def _engine_params(m, o, request, max_level=10):
    return m.make_params(o, d=10, method=1, formats=[W.default_format(o, lev) for lev in range(max_level + 1)],
                         request=request, rng_pack=1)


def _accuracy(done, opts, max_level):
    """RMS of (price - Black-Scholes) / eps over the European and digital requests;
    the requests that stopped at the maximum level, with their final bias
    estimate over the target eps / sqrt(2) (above 1: the bias test was not met,
    the result is flagged as not converged)."""
    errs = [(done[i]["price"] - _bs_price(o)) / o["eps"] for i, o in enumerate(opts) if _bs_price(o) is not None]
    at_max = [i for i in range(len(opts)) if done[i]["L"] >= max_level]
    ratio = {i: done[i].get("bias_estimate", float("nan")) / (opts[i]["eps"] / math.sqrt(2)) for i in at_max}
    return {"rms_err_over_eps_vs_black_scholes": math.sqrt(sum(e * e for e in errs) / len(errs)),
            "checked_against_black_scholes": len(errs), "stopped_at_max_level": len(at_max),
            "max_level": max_level,
            "not_converged": sum(1 for v in ratio.values() if v > 1.0),
            "bias_over_target_at_max_level": sorted(ratio.values())}


def batched_run(m, n=256, seed=7, mode=5, iters_per_launch=-4096, max_level=16):
    """The batched workload: all n options submitted at once to one engine; with a
    negative iters_per_launch the whole adaptive run of all of them is one graph
    launch iterating on the device (what mlmc_batch_estimate does, with the
    engine's counters kept).  The launch shapes (CTA threads, path-steps per
    thread) are autotuned first on a work list of the same kernel classes (eight
    of the options, approximate and correction items on levels 0-12) and
    installed for the engine's admissions; the default table is restored after."""
    opts = W.batched_options(n, seed)
    tune_items = []
    for i, o in enumerate(opts[:8]):
        P = _engine_params(m, o, 1000 + i, max_level)
        for lev in range(0, 13):
            tune_items.append(dict(params=P, level=lev, variant=W.FIXED_APPROX, N=max(2000, (1 << 22) >> lev)))
            tune_items.append(dict(params=P, level=lev, variant=W.CORR_FIXED, N=max(1000, (1 << 18) >> lev)))
    shapes = m.mlmc_autotune(tune_items, seed, reps=3)
    eng = m.Engine(max_slots=n, max_level=max_level, iters_per_launch=iters_per_launch)
    _engine_solve(eng, _engine_params(m, opts[0], 0, max_level), 1e-2, mode, 99)   # warm tables and kernels
    s0 = eng.stats()
    t0 = time.perf_counter()
    index = {eng.submit(_engine_params(m, o, i, max_level), o["eps"], mode, 1): i for i, o in enumerate(opts)}
    done = {}
    while len(done) < n:
        eng.step()
        for rid in eng.completed():
            if rid in index:
                res = eng.poll(rid)
                res.update(bias_estimate=eng.request_info(rid)["bias_estimate"])
                done[index[rid]] = res
    wall = time.perf_counter() - t0
    st = eng.stats()
    gi = eng.graph_info()
    eng.close()
    m.mlmc_tuning_reset()
    lat = sorted(done[i]["latency_s"] for i in range(n))
    out = {"requests": n, "mode": mode, "wall_s": wall, "requests_per_s": n / wall,
           "autotuned_shapes": sorted({"%dx%d" % t for t in shapes}),
           "graph_launches": st["launches"] - s0["launches"], "iters_per_launch": iters_per_launch,
           "graph_captures": gi["captures"], "launch_classes": gi["groups"],
           "path_steps": st["path_steps"] - s0["path_steps"],
           "path_steps_per_s": (st["path_steps"] - s0["path_steps"]) / wall,
           "p50_latency_s": lat[n // 2], "p99_latency_s": lat[min(n - 1, int(0.99 * n))]}
    out.update(_accuracy(done, opts, max_level))
    return out


def serving_run(m, rate, n=400, seed=11, mode=5, max_level=16, eps_range=(1e-4, 1e-2)):
    """Poisson arrivals at `rate` req/s, options drawn as the batched workload;
    requests are admitted while others run (continuous batching)."""
    arrivals = W.poisson_arrivals(rate, n, seed)
    opts = W.batched_options(n, seed, eps_range)
    eng = m.Engine(max_slots=256, max_level=max_level)
    _engine_solve(eng, _engine_params(m, opts[0], 0, max_level), 1e-2, mode, 99)   # warm tables and kernels
    s0 = eng.stats()
    index = {}      # request id -> option index
    done = {}
    nxt = 0
    t0 = time.perf_counter()
    while len(done) < n:
        t = time.perf_counter() - t0
        while nxt < n and arrivals[nxt] <= t:
            index[eng.submit(_engine_params(m, opts[nxt], nxt, max_level), opts[nxt]["eps"], mode, 1)] = nxt
            nxt += 1
        if nxt == len(done) and nxt < n:
            time.sleep(max(0.0, min(arrivals[nxt] - t, 0.01)))
            continue
        eng.step()
        # only the requests that completed in this step (mlmc_engine_completed)
        for rid in eng.completed():
            if rid in index:
                res = eng.poll(rid)
                res.update(bias_estimate=eng.request_info(rid)["bias_estimate"])
                done[index[rid]] = res
    wall = time.perf_counter() - t0
    st = eng.stats()
    gi = eng.graph_info()
    eng.close()
    lat = sorted(done[i]["latency_s"] for i in range(n))
    out = {"arrival_rate": rate, "requests": n, "eps_range": list(eps_range), "mode": mode, "wall_s": wall,
           "requests_per_s": n / wall,
           "p50_latency_s": lat[n // 2], "p99_latency_s": lat[min(n - 1, int(0.99 * n))],
           "engine_steps": st["steps"] - s0["steps"], "graph_launches": st["launches"] - s0["launches"],
           "graph_captures": gi["captures"], "path_steps": st["path_steps"] - s0["path_steps"],
           "path_steps_per_s": (st["path_steps"] - s0["path_steps"]) / wall}
    out.update(_accuracy(done, opts, max_level))
    return out


def sweep_run(m, torch, levels=(0, 2, 4, 6, 8, 10), sizes=(1 << 20, 1 << 24, 1 << 28), grid_n=1 << 22,
              sigmas=(0.1, 0.2, 0.4), grid=True):
    """Level-kernel throughput sweep (Milstein): path-steps/s of one level-kernel
    launch by CUDA events (median of 5 after 2 warm-up launches, L2 flushed).
    (a) sizes: European call, sigma = 0.2, every variant, N in `sizes` paths at
    each level; (b) grid: European / Asian / lookback x sigma x level x variant
    at `grid_n` paths.  A point holds at most 2^32 path-steps (2^28 for FP64,
    which runs at 1/64 of the FP32 rate on this part): N is reduced to fit."""
    variants = (("fp64_exact", W.FP64_EXACT), ("fp32_exact", W.FP32_EXACT), ("fp16_approx", W.FP16_APPROX),
                ("bf16_approx", W.BF16_APPROX), ("fixed_approx", W.FIXED_APPROX),
                ("nested_corr_fixed", W.CORR_FIXED))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def point(P, lev, v, n):
        plan = m.Plan([dict(params=P, level=lev, variant=v, N=n)], 7)
        for _ in range(2):
            plan.launch()
        ts = []
        for _ in range(5):
            flush.zero_()
            plan.launch()
            ts.append(plan.kernel_time(0)[1])
        plan.close()
        ms = statistics.median(ts)
        return ms, (n << lev) / (ms * 1e-3)

    def cap(n, lev, v):
        lim = 1 << (28 if v == W.FP64_EXACT else 32)
        return max(1, min(n, lim >> lev))

    rows = []
    params = {}

    def P_of(pay, sig):
        if (pay, sig) not in params:
            p = W.params(payoff=pay, scheme=W.MILSTEIN, sigma=sig)
            params[(pay, sig)] = m.make_params(p, d=10, method=1, formats=[W.default_format(p, k) for k in range(11)],
                                               rng_pack=1)
        return params[(pay, sig)]

    for n0 in sizes:
        for lev in levels:
            for vname, v in variants:
                n = cap(n0, lev, v)
                ms, rate = point(P_of(W.EURO, 0.2), lev, v, n)
                rows.append({"part": "sizes", "payoff": "euro", "sigma": 0.2, "level": lev, "variant": vname,
                             "paths": n, "ms": ms, "path_steps_per_s": rate})
    for pay_name, pay in ((("euro", W.EURO), ("asian", W.ASIAN), ("lookback", W.LOOKBACK)) if grid else ()):
        for sig in sigmas:
            for lev in levels:
                for vname, v in variants:
                    n = cap(grid_n, lev, v)
                    ms, rate = point(P_of(pay, sig), lev, v, n)
                    rows.append({"part": "grid", "payoff": pay_name, "sigma": sig, "level": lev, "variant": vname,
                                 "paths": n, "ms": ms, "path_steps_per_s": rate})
    return {"scheme": "milstein", "rows": rows}


def optimiser_run(m, torch, levels=range(11), n_sens=1_000_000, n_check=400_000):
    """Offline bit-width optimisation of the test case (Sec. 4-6): error-model
    statistics from 10^6 exact paths per level on the GPU, optimal widths and table
    size (paper's FPGA cost model, C_RNG = 1e4), then the GPU fixed-point correction
    estimator run with those widths to check the model (Var <= V'_corr).  Returns
    the report and the optimised formats of every level."""
    mse = [0.0, 0.0] + [m.icdf_mse(d) for d in range(2, 15)]
    p = W.params()
    rows, formats = [], []
    sens_ms = None
    for lev in levels:
        P = m.make_params(p)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = m.mlmc_sensitivities(lev, n_sens, P, 77)
        dt = time.perf_counter() - t0
        if lev == 8:
            sens_ms = dt * 1e3
        o = m.mlmc_optimise_level(lev, s, lut_mse=mse, lut_max_bits=14)
        formats.append(o["format"])
        # lut_bits 0: no table of at most 14 bits meets the model's bound; use 14
        lut = o["lut_bits"] or 14
        fmts = [W.default_format(p, k) for k in range(lev)] + [o["format"]]
        res = m.mlmc_level(lev, n_check, m.make_params(p, d=lut, method=1, formats=fmts), W.CORR_FIXED, 5)
        mean = res["sum"] / n_check
        var = res["sum2"] / n_check - mean * mean
        v_corr = (math.sqrt(o["v_corr"]) + s["B"][0] * math.sqrt(mse[lut])) ** 2
        v_ind = o["v_indep"] + s["A"][0] * mse[lut]
        rows.append({"level": lev, "d": o["d"], "e": o["e"], "lut_bits": o["lut_bits"], "lut_bits_run": lut,
                     "level_cost_ratio": o["level_cost_ratio"], "V": s["var"], "v_indep_ext": v_ind,
                     "v_corr_ext": v_corr, "var_corrections_measured": var, "bound_holds": var <= v_corr,
                     "saturations": res["saturations"]})
    return {"paths_per_level": n_sens, "cost_model": "FPGA eq. cost_sq, C_RNG = 1e4 per step",
            "variables": ["Z", "con1", "con2", "mul1", "sum1", "mul2", "S"],
            "sensitivity_ms_level_8": sens_ms,
            "sensitivity_path_steps_per_s": n_sens * (1 << 8) / (sens_ms * 1e-3) if sens_ms else None,
            "levels": rows}, formats


def nested_step_with_formats(m, torch, formats, flush, stream, reps=10):
    """The nested workload's step with other fixed-point formats (the optimiser's,
    table d = 10 kept): device time per step and the per-level variance of the
    corrections, beside the same figures with the default formats."""
    out = {}
    for name, fm in (("default_formats", None), ("optimised_formats", formats)):
        items, meta, cfg = build_items(m, formats=fm)
        plan = m.Plan(items, cfg["seed"])
        for _ in range(3):
            plan.launch(stream)
        step_ms = []
        for k in range(reps):
            flush.zero_()
            plan.launch(stream)
            step_ms.append(plan.elapsed_ms())   # the step's device time, as in the headline
        torch.cuda.synchronize()
        res = plan.results()
        plan.close()
        ms = statistics.median(step_ms)
        var_corr = {}
        sat = 0
        for it, r in zip(meta, res):
            sat += r["saturations"]
            if it["variant"] == W.CORR_FIXED and it["params"]["payoff"] == W.EURO:
                mean = r["sum"] / r["n"]
                var_corr[it["level"]] = r["sum2"] / r["n"] - mean * mean
        out[name] = {"ms_per_step": ms, "path_steps_per_s": plan_steps(items) / (ms * 1e-3),
                     "var_corrections_euro": [var_corr[k] for k in sorted(var_corr)], "saturations": sat}
    return out


def plan_steps(items):
    return sum(it["N"] << it["level"] for it in items)


def _engine_solve(eng, P, eps, mode, seed):
    rid = eng.submit(P, eps, mode, seed)
    while True:
        eng.step()
        r = eng.poll(rid)
        if r is not None:
            return r


def time_to_eps(m, torch, eps=1e-3, seeds=tuple(range(1, 12)), formats_opt=None):
    """Wall time of mlmc_estimate at RMS error eps (European call, median of the
    seeds): plain FP32 MLMC against the nested estimator (Sec. 2.2) with its
    approximate path in fixed point, binary16 and bfloat16 (all variables, or
    the increments with S in FP32: fp16s / bf16s), each with the Method-1
    and the Method-3 table (Sec. 3.1, 3.3); the paper's nested estimator samples
    every level, the exact-low modes compute the approximate terms of levels 0-1
    by enumeration instead.  With formats_opt, the fixed-point runs again with the
    bit-width optimiser's formats.  Accuracy: RMS over the seeds of
    (price - Black-Scholes) / eps."""
    p = W.params()
    bs = _bs_price(p)
    fm = [W.default_format(p, lev) for lev in range(11)]

    def P(method=1, formats=fm):
        return m.make_params(p, d=10, method=method, formats=formats, rng_pack=1)

    configs = [("plain_fp32", m.MODE_PLAIN_FP32, P())]
    for tag, method in (("m1", 1), ("m3", 3)):
        configs += [("nested_fixed_" + tag, m.MODE_NESTED_FIXED, P(method)),
                    ("nested_fp16_" + tag, m.MODE_NESTED_FP16, P(method)),
                    ("nested_bf16_" + tag, m.MODE_NESTED_BF16, P(method)),
                    ("nested_fp16s_" + tag, m.MODE_NESTED_FP16S, P(method)),
                    ("nested_bf16s_" + tag, m.MODE_NESTED_BF16S, P(method)),
                    ("nested_fixed_exact_low_" + tag, m.MODE_NESTED_FIXED_EXACT_LOW, P(method)),
                    ("nested_fp16_exact_low_" + tag, m.MODE_NESTED_FP16_EXACT_LOW, P(method)),
                    ("nested_fp16s_exact_low_" + tag, m.MODE_NESTED_FP16S_EXACT_LOW, P(method)),
                    ("nested_bf16s_exact_low_" + tag, m.MODE_NESTED_BF16S_EXACT_LOW, P(method))]
    if formats_opt:
        configs += [("nested_fixed_m1_optimised_widths", m.MODE_NESTED_FIXED, P(1, formats_opt)),
                    ("nested_fixed_exact_low_m1_optimised_widths", m.MODE_NESTED_FIXED_EXACT_LOW, P(1, formats_opt))]
    out = {"eps": eps, "payoff": "european call", "seeds": len(seeds)}
    for name, mode, PP in configs:
        m.mlmc_estimate(1e-2, PP, mode, 99, 10)   # warm tables and contexts
        ts, prices = [], []
        for s_ in seeds:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = m.mlmc_estimate(eps, PP, mode, s_, 10)
            ts.append(time.perf_counter() - t0)
            prices.append(r["price"])
        out[name] = {"s_median": statistics.median(ts), "prices": prices, "L": r["L"], "N": r["N"],
                     "rms_err_over_eps": math.sqrt(sum((x - bs) ** 2 for x in prices) / len(prices)) / eps}
    for name, _, _ in configs[1:]:
        out["speedup_%s_vs_plain_fp32" % name] = out["plain_fp32"]["s_median"] / out[name]["s_median"]
    # the same adaptive algorithm driven on the device: one request through a
    # (created and warmed) engine, four iterations per CUDA-graph launch,
    # instead of host-driven plans
    for name, mode in (("plain_fp32_graph", m.MODE_PLAIN_FP32),
                       ("nested_fixed_exact_low_m1_graph", m.MODE_NESTED_FIXED_EXACT_LOW)):
        PP = P()
        eng = m.Engine(max_slots=1, max_level=10, iters_per_launch=4)
        _engine_solve(eng, PP, 1e-2, mode, 99)
        ts, prices = [], []
        for s_ in seeds:
            torch.cuda.synchronize()
            l0 = eng.stats()["launches"]
            t0 = time.perf_counter()
            r = _engine_solve(eng, PP, eps, mode, s_)
            ts.append(time.perf_counter() - t0)
            prices.append(r["price"])
        out[name] = {"s_median": statistics.median(ts), "prices": prices, "L": r["L"],
                     "graph_launches": eng.stats()["launches"] - l0}
        eng.close()
    out["speedup_nested_fixed_exact_low_m1_graph_vs_plain_fp32_graph"] = (
        out["plain_fp32_graph"]["s_median"] / out["nested_fixed_exact_low_m1_graph"]["s_median"])
    return out


if __name__ == "__main__":
    main()
