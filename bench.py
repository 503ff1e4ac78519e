#!/usr/bin/env python
"""Benchmark of the GB300 destriper on a synthetic scan shaped like the paper's
12-month LATTE-like IQU radiometer (1.6e9 samples at 50 Hz; one I/Q/U output;
nside 512; 1 s baselines; 2% flagged samples): the largest workload that fits
one GPU.  --config 2 runs the 30-day B-Machine-like channel (1.3e8 samples;
I, q, u outputs; nside 256; 60 s baselines).

One step = the whole destriping job on inputs already resident in HBM: plan
(hits, pixel matrices, rcond cut), right-hand side, CG to ||r||/||b|| < 1e-10,
gauge, destriped map.  value = timestream samples x CG iterations / step time,
summed over ranks and divided by the slowest rank's time.  Beside it, outside
the timed region: the plain float64 path on the same workload (fp64_path), the
errors of the mixed result against it and against the float64 oracle on sampled
pixels and baselines (error_vs_oracle), the end-to-end job from host buffers
(e2e) and the oracle's own rate on the host cores (cpu_baseline).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--config 4|2|1|3|5] [--precision mixed|fp64]

N > 1 runs N independent replicas (one per GPU; the single-problem solve has
no data-path exchange), launched with torch.distributed.run.  --impl reference
times the float64 CPU oracle on a bounded prefix of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "timestream samples/s per CG iteration (% HBM roofline); full-solve time; p50/p99"
UNIT = "samples/s"
BYTES_PER_SAMPLE_PASS = 12  # int32 pixel + float32 cos 2psi + float32 sin 2psi, per pass
L2_BYTES = 129 * 10 ** 6
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=4, choices=[1, 2, 3, 4, 5])
    ap.add_argument("--serve-seconds", type=float, default=30.0,
                    help="length of the request trace (config 5)")
    ap.add_argument("--serve-master", type=int, default=100_000_000,
                    help="samples of the host-resident master scans (config 5)")
    ap.add_argument("--serve-comparator", type=int, default=0,
                    help="config 5: requests of the measured float64 FIFO (0 = all)")
    ap.add_argument("--serve-cap", type=float, default=0.0,
                    help="config 5: cap on the samples of the admitted requests (0 = none)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--n-samples", type=int, default=None, help="cut the workload (testing)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-path", action="store_true",
                    help="single-problem workloads: skip the plain float64 comparator")
    ap.add_argument("--oracle-procs", type=int, default=0,
                    help="processes of the all-core oracle timing (0 = every host core)")
    ap.add_argument("--oracle-samples", type=int, default=1_000_000)
    ap.add_argument("--oracle-iters", type=int, default=20)
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched workload: keep the default launch shape")
    ap.add_argument("--no-fp64-comparator", action="store_true",
                    help="batched workload: skip the sequential float64 comparator")
    ap.add_argument("--tune", default="",
                    help="plan tuning knobs for the single-problem workloads, key=value,...")
    return ap.parse_args()


def parse_tune(text):
    out = {}
    for item in filter(None, (t.strip() for t in text.split(","))):
        k, v = item.split("=")
        out[k.strip()] = float(v)
    return out


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_traffic(n_t, kernel, workload):
    """Per-launch DRAM bytes of `kernel` on `workload` from the committed ncu
    summary (bytes per sample times samples), or None if the summary is missing,
    has no line for the workload, or the kernel's source file has changed since."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.md")
    try:
        text = open(path).read()
        m_sha = re.search(r"(\w+\.cu) sha256\[:16\]:\s*([0-9a-f]+)", text)
        if not m_sha:
            return None
        src = os.path.join(ROOT, "paper_1309_5609_gb300", "csrc", m_sha.group(1))
        if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != m_sha.group(2):
            return None
        for key, bps in re.findall(r"dram bytes per sample \[([\w.-]+)\]:\s*([0-9.]+)", text):
            if workload.startswith(key):
                return float(bps) * n_t
        return None
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={CLOCK_FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() in ("active", "1", "yes"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_over_ranks(t_ms, units, dist, device):
    """Slowest rank's time and the units all ranks processed (replicas, weak scaling)."""
    import torch
    tt = torch.tensor([t_ms, units], dtype=torch.float64, device=device)
    tmax = tt.clone()
    dist.all_reduce(tmax[:1], op=dist.ReduceOp.MAX)
    dist.all_reduce(tt[1:], op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tt[1])


def workload(args, device):
    from synth import CONFIGS, WORKLOAD_NAMES, config_problem
    import torch
    kw = {}
    if args.n_samples:
        kw["n_t"] = args.n_samples
    ydt = torch.float32 if args.precision == "mixed" else torch.float64
    prob = config_problem(args.config, device=device, y_dtype=ydt, keep_f64_trig=False, **kw)
    name = WORKLOAD_NAMES[args.config]
    if args.n_samples:
        name += f"-prefix{args.n_samples}"
    return prob, name


def config_dict(args, name=None):
    """The workload as configured (the full size unless --n-samples cuts it)."""
    from synth import CONFIGS, WORKLOAD_NAMES
    c = dict(CONFIGS[args.config])
    n_t = args.n_samples or c["n_t"]
    if name is None:
        name = WORKLOAD_NAMES[args.config] + (f"-prefix{args.n_samples}" if args.n_samples else "")
    n_b = -(-n_t // c["baseline_len"])
    pointing = 12 * n_t
    l2 = ("inputs larger than L2: the pointing streams from HBM every pass "
          f"({pointing / 1e9:.2f} GB against a 129 MB L2)" if pointing > L2_BYTES else
          f"L2-resident: {pointing / 1e6:.1f} MB of pointing fit the 129 MB L2, so this "
          "workload measures parity and launch overheads, not HBM")
    return {"workload": name, "n_samples": n_t, "nside": c["nside"],
            "outputs": ",".join(c["kinds"]), "baseline_len": c["baseline_len"],
            "unknowns": len(c["kinds"]) * n_b, "precision": args.precision, "tol": args.tol,
            "flagged_fraction": c.get("flag_frac", 0.0), "l2": l2,
            "step": "plan + RHS + CG to tol + gauge + destriped map"}


def oracle_rate(prob_np, n_iters, tol=1e-10):
    """Oracle on a bounded sample: plan, RHS and n_iters CG iterations; returns
    (sample-iterations per second, iterations, seconds)."""
    import numpy as np
    import oracle
    try:
        from threadpoolctl import threadpool_limits
        lim = threadpool_limits(1)
    except Exception:
        lim = None
    t0 = time.perf_counter()
    plan = oracle.make_plan(prob_np["pix"], prob_np["c"], prob_np["s"], prob_np["valid"],
                            prob_np["nside"], prob_np["kinds"], prob_np["baseline_len"])
    b = oracle.rhs(plan, prob_np["y"])
    x, iters, _ = oracle.cg(plan, b, tol=tol, max_iter=n_iters)
    dt = time.perf_counter() - t0
    if lim is not None:
        lim.unregister() if hasattr(lim, "unregister") else None
    return plan.n_t * max(iters, 1) / dt, iters, dt


def host_cpu():
    """Core count and CPU model of the host the oracle runs on."""
    info = {"nproc": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            key, _, val = line.partition(":")
            if key.strip() == "Model name" and val.strip():
                info["model"] = val.strip()
            elif key.strip() == "Vendor ID" and val.strip():
                info["vendor"] = val.strip()
    except Exception:
        pass
    return info


def _oracle_worker_init():
    # one thread per process: the all-core figure is processes x single-thread oracles
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"


def _oracle_worker(job):
    d, n_iters = job
    t0 = time.perf_counter()
    rate, it, dt = oracle_rate(d, n_iters)
    return d["pix"].shape[0] * max(it, 1), t0, time.perf_counter()


def oracle_all_cores(d, n_iters, procs):
    """The oracle as it stands, one copy per host core on the same sample, run at
    the same time (a spawned pool: the parent already holds a CUDA context).
    Returns (sample-iterations per second over the wall time of the concurrent
    runs, processes)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs, initializer=_oracle_worker_init) as pool:
        res = pool.map(_oracle_worker, [(d, n_iters)] * procs, chunksize=1)
    units = sum(r[0] for r in res)
    wall = max(r[2] for r in res) - min(r[1] for r in res)
    return units / wall, procs


def prefix_numpy(prob, n):
    import numpy as np
    n = min(n, prob.n_t)
    return dict(pix=prob.pix[:n].cpu().numpy().astype(np.int64),
                c=prob.c32[:n].cpu().numpy().astype(np.float64),
                s=prob.s32[:n].cpu().numpy().astype(np.float64),
                y=prob.y[:, :n].cpu().numpy().astype(np.float64),
                valid=None if prob.valid is None else prob.valid[:n].cpu().numpy(),
                nside=prob.nside, kinds=prob.kinds, baseline_len=prob.baseline_len), n


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    from synth import WORKLOAD_NAMES, batch_configs, config_problem, make_problem
    import torch
    n = min(args.oracle_samples, args.n_samples or 10 ** 12)
    ydt = torch.float32 if args.precision == "mixed" else torch.float64
    if args.config == 3:  # the batch's first problem
        c = dict(batch_configs(64, seed=1003)[0], n_t=n)
        prob, name = make_problem(keep_f64_trig=False, y_dtype=ydt, **c), "batch64 problem 0"
    elif args.config == 5:  # a two-output request of the serving trace's kind
        prob = make_problem(n, 256, ("q", "u"), baseline_len=500, f_knee=0.1, alpha=1.7,
                            seed=5000, keep_f64_trig=False, y_dtype=ydt)
        name = "serving request (q,u, nside 256, L 500)"
    else:
        prob = config_problem(args.config, n_t=n, keep_f64_trig=False, y_dtype=ydt)
        name = WORKLOAD_NAMES[args.config]
    d, n = prefix_numpy(prob, n)
    iters_per_step = max(1, args.oracle_iters // 2)
    for _ in range(args.warmup):
        oracle_rate(d, 2)
    tot_si, tot_t, tot_it = 0.0, 0.0, 0
    for _ in range(args.steps):
        rate, it, dt = oracle_rate(d, iters_per_step)
        tot_si += n * max(it, 1)
        tot_t += dt
        tot_it += it
    value = tot_si / tot_t
    sample = (f"prefix of {n} samples of {name}: plan + RHS + {iters_per_step} CG iterations "
              f"per step, float64 numpy, 1 thread")
    if args.config in (1, 2, 4):
        cfg = config_dict(args)
        cfg.update(workload=f"{cfg['workload']}-prefix{n}", n_samples=n,
                   unknowns=len(prob.kinds) * (-(-n // prob.baseline_len)),
                   full_workload=config_dict(args)["workload"],
                   full_n_samples=config_dict(args)["n_samples"],
                   l2=f"host run: the oracle on a {n}-sample prefix ({12 * n / 1e6:.0f} MB "
                      "of pointing) on the host cores; the GPU's L2 does not apply")
    else:
        cfg = {"workload": name, "n_samples": n}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded scan, Gaussian sky, 1/f noise)", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample, "host": host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist
    import paper_1309_5609_gb300 as ds

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    ds.load_library()
    prob, name = workload(args, dev)
    n_o, n_b, npix = prob.n_o, prob.n_b, prob.npix
    from synth import components
    n_c = len(components(prob.kinds))
    stream = torch.cuda.current_stream(dev)
    a = torch.zeros(n_o * n_b, dtype=torch.float64, device=dev)
    m = torch.zeros(n_c * npix, dtype=torch.float64, device=dev)
    hits = torch.zeros(npix, dtype=torch.int32, device=dev)
    mask = torch.zeros(npix, dtype=torch.uint8, device=dev)

    tune = parse_tune(args.tune)
    layout = {}  # the float32 operator's form, as the plans report it

    def step(prof_acc):
        plan = ds.destripe_plan(prob.pix, prob.c32, prob.s32, prob.valid, nside=prob.nside,
                                kinds=prob.kinds, baseline_len=prob.baseline_len,
                                precision=args.precision)
        for k, v in tune.items():
            ds.destripe_tune(plan, k, v)
        if prof_acc is not None:
            ds.destripe_profile(plan, 1)
        st, iters, rel = ds.destripe_solve(plan, prob.y, a, tol=args.tol)
        info = ds.destripe_plan_info(plan)  # after the solve: records built by it count
        layout.update(layout=info["layout"], n_runs=info["n_runs"], bin_order=info["bin_order"])
        ds.destripe_map(plan, prob.y, a, m, hits, mask)
        if prof_acc is not None:
            p = ds.destripe_profile(plan, -1)
            for k, v in p.items():
                prof_acc[k] = prof_acc.get(k, 0) + v
            prof_acc["plan_launches"] = prof_acc.get("plan_launches", 0) + 3
        plan.close()
        if st != ds.DS_OK:
            raise RuntimeError(f"solve did not converge: status {st}, {iters} iterations, "
                               f"residual {rel:.3e}")
        return iters, rel

    for _ in range(args.warmup):
        step(None)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    prof = {}
    iters_tot = 0
    rels = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            it, rel = step(None)
            iters_tot += it
            rels.append(rel)
        ev1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    t_ms = ev0.elapsed_time(ev1)
    units = float(prob.n_t) * iters_tot
    # the per-kernel times of the roofline from one more job with the plan's CUDA-event
    # profile on, after the timed region (the events cost launch-bound jobs time)
    step(prof)
    if world > 1:
        t_ms_all, units_all = reduce_over_ranks(t_ms, units, dist, dev)
    else:
        t_ms_all, units_all = t_ms, units
    value = units_all / (t_ms_all / 1e3)

    # dominant kernel of the CG iteration and its roofline
    ti = max(1, int(prof.get("timed_iterations", 0)))
    per_launch = {"bin": prof.get("bin_ms", 0.0) / ti, "rescan": prof.get("rescan_ms", 0.0) / ti}
    dom = max(per_launch, key=per_launch.get)
    alg_bytes = BYTES_PER_SAMPLE_PASS * prob.n_t
    peak, peak_kind = peaks()
    dur_s = per_launch[dom] / 1e3
    achieved = alg_bytes / dur_s / 1e9 if dur_s > 0 else None
    mixed = args.precision == "mixed"
    form = layout.get("layout", 0) if mixed else 0
    kname = {0: {"bin": "k_bin", "rescan": "k_rescan"},
             1: {"bin": "k_ck_bin", "rescan": "k_ck_rescan"},
             2: {"bin": "k_pm_bin" if layout.get("bin_order") else "k_rl_bin",
                 "rescan": "k_rescan" if (tune.get("rescan_samples", 0) or
                                        layout.get("n_runs", 0) > 0.6 * prob.n_t)
                 else "k_rl_rescan"},
             3: {"bin": "k_tl_bin_lanes", "rescan": "k_tl_rescan"}}[form][dom]
    roof = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
            "traffic": kernel_traffic(prob.n_t, kname, name),
            "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)",
            "algorithmic_bytes_per_launch": alg_bytes,
            "launch_ms": per_launch[dom],
            "other_kernel_launch_ms": {k: v for k, v in per_launch.items() if k != dom},
            "iteration_ms": prof.get("iteration_ms", 0.0) / ti,
            "pixel_solve_ms": prof.get("solve_ms", 0.0) / ti}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "mixed" else "f64",
            "data": "synthetic (seeded scan, Gaussian sky, 1/f noise), resident in HBM",
            "config": dict(config_dict(args, name), tune=tune,
                           operator_layout={0: "time-ordered pixels", 1: "chunk-local pixel index",
                                            2: "run-length records",
                                            3: "time-tiled pixel-sorted run records"}[form]
                           + (", pixel-major binning" if form == 2 and layout.get("bin_order")
                              else ""),
                           runs_per_sample=layout.get("n_runs", 0) / prob.n_t), "roofline": roof,
            "iterations_per_step": iters_tot / args.steps,
            "full_solve_s": t_ms_all / args.steps / 1e3,
            "timeline_samples_per_s": float(prob.n_t) * world / (t_ms_all / args.steps / 1e3),
            "rel_resid_max": max(rels) if rels else None,
            # the profiled job's launches, times the timed jobs (all alike)
            "gpu_launches": int(prof.get("kernel_launches", 0)) * args.steps,
            "clocks": clk.summary()}

    # outside the timed region: the plain float64 path on the same workload, and the
    # errors of the last timed job's result against it
    sigma = float(prob.meta.get("sigma", 1.0))
    if rank == 0 and not args.no_fp64_path and args.precision == "mixed":
        line["fp64_path"], line["error_vs_fp64_path"] = fp64_path_leg(args, prob, ds, a, m,
                                                                      n_c, sigma)
    # sampled outputs of the mixed path for the oracle (taken on the GPU here; the
    # oracle runs in the CPU leg below)
    sampled = None
    if rank == 0 and not args.no_cpu_baseline:
        sampled = gpu_sampled_outputs(args, prob, ds, a, m, n_c)
    # end to end through the C ABI with host buffers (copies inside the timed region)
    if not args.no_e2e:
        line["e2e"] = e2e_leg(args, prob, ds, world, dist if world > 1 else None)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"], line["error_vs_oracle"] = cpu_baseline_leg(args, prob, sampled,
                                                                         sigma)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def rel_rms(a, b):
    import numpy as np
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    den = float(np.sqrt(np.mean(b ** 2))) if b.size else 0.0
    return float(np.sqrt(np.mean((a - b) ** 2)) / (den if den > 0 else 1.0)) if b.size else 0.0


def fp64_path_leg(args, prob, ds, a_mixed, m_mixed, n_c, sigma):
    """One job of the plain float64 single-problem path (float64 timelines, float64
    per-sample work) on the same workload, timed with CUDA events; and the mixed
    result's differences from it, plus the float64 residual of the mixed
    baselines recomputed by this float64 plan."""
    import torch
    dev = prob.pix.device
    y64 = prob.y.double().contiguous()  # promotion outside the timed region
    a64 = torch.zeros_like(a_mixed)
    m64 = torch.zeros_like(m_mixed)
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    plan = ds.destripe_plan(prob.pix, prob.c32, prob.s32, prob.valid, nside=prob.nside,
                            kinds=prob.kinds, baseline_len=prob.baseline_len, precision="fp64")
    st, iters, rel = ds.destripe_solve(plan, y64, a64, tol=args.tol)
    ds.destripe_map(plan, y64, a64, m64)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    # float64 residual of the mixed solution: ||b - A a|| / ||b|| with this plan
    b = torch.empty_like(a64)
    ds.destripe_rhs(plan, y64, b)
    Aa = torch.empty_like(a64)
    ds.destripe_apply_A(plan, a_mixed, Aa)
    res_mixed = float(torch.linalg.norm(b - Aa) / torch.linalg.norm(b))
    plan.close()
    del y64, b, Aa
    comp = {"value": prob.n_t * iters / (ms / 1e3), "unit": UNIT, "ms_per_job": ms,
            "iterations": iters, "rel_resid": rel, "status": int(st),
            "note": "float64 plan and timelines on the same workload, one job, outside the "
                    "timed region (timelines promoted to float64 beforehand)"}
    da = (a_mixed - a64).abs()
    err = {"baselines_max_abs_over_sigma": float(da.max()) / sigma,
           "baselines_rel_rms": rel_rms(a_mixed.cpu().numpy(), a64.cpu().numpy()),
           "map_rel_rms": rel_rms(m_mixed.cpu().numpy(), m64.cpu().numpy()),
           "mixed_solution_fp64_residual": res_mixed, "sigma_white": sigma}
    del a64, m64
    torch.cuda.empty_cache()
    return comp, err


def sampled_baselines(n_b, cfg, k):
    import numpy as np
    rng = np.random.default_rng(cfg)
    return sorted(set(rng.integers(0, n_b, k).tolist()) | {0, n_b - 1})


def gpu_sampled_outputs(args, prob, ds, a, m, n_c):
    """The mixed path's outputs at the pixels touched by a few sampled baselines:
    every sample on those pixels (renumbered) with the GPU's hits, mask, binned
    map, destriped map (given the timed job's baselines) and the float32
    operator's (A x) on the sampled baselines.  Host arrays for the oracle."""
    import numpy as np
    import torch
    dev = prob.pix.device
    L, n_t, n_b = prob.baseline_len, prob.n_t, prob.n_b
    baselines = sampled_baselines(n_b, args.config, 6 if L >= 1000 else 12)
    T = torch.cat([torch.arange(b * L, min((b + 1) * L, n_t), device=dev) for b in baselines])
    P = torch.unique(prob.pix[T])
    U = torch.nonzero(torch.isin(prob.pix, P)).squeeze(1)
    plan = ds.destripe_plan(prob.pix, prob.c32, prob.s32, prob.valid, nside=prob.nside,
                            kinds=prob.kinds, baseline_len=L, precision="mixed")
    mb = torch.zeros_like(m)
    hits = torch.zeros(prob.npix, dtype=torch.int32, device=dev)
    mask = torch.zeros(prob.npix, dtype=torch.uint8, device=dev)
    ds.destripe_bin(plan, prob.y, None, mb, hits, mask)
    x = torch.randn(prob.n_o * n_b, dtype=torch.float64, device=dev,
                    generator=torch.Generator(dev).manual_seed(3))
    Ax = torch.empty_like(x)
    ds.destripe_apply_A(plan, x, Ax)
    plan.close()
    cols = torch.tensor(baselines, device=dev)
    out = {"baselines": np.array(baselines), "L": L, "nside": prob.nside, "kinds": prob.kinds,
           "P": P.cpu().numpy(), "U": U.cpu().numpy(), "T": T.cpu().numpy(),
           "pix": prob.pix[U].cpu().numpy(), "c": prob.c32[U].double().cpu().numpy(),
           "s": prob.s32[U].double().cpu().numpy(),
           "valid": None if prob.valid is None else prob.valid[U].cpu().numpy(),
           "y": prob.y[:, U].double().cpu().numpy(),
           "a": a.view(prob.n_o, n_b).cpu().numpy(),
           "x": x.view(prob.n_o, n_b)[:, :].cpu().numpy(),
           "hits": hits[P].cpu().numpy(), "mask": mask[P].cpu().numpy().astype(bool),
           "bin_map": mb.view(n_c, prob.npix)[:, P].cpu().numpy(),
           "map": m.view(n_c, prob.npix)[:, P].cpu().numpy(),
           "Ax": Ax.view(prob.n_o, n_b)[:, cols].cpu().numpy()}
    del mb, hits, mask, x, Ax
    torch.cuda.empty_cache()
    return out


def oracle_sampled_errors(g):
    """The oracle on the sampled subset (every sample of the touched pixels, so
    that their cut, map and the sampled baselines' (A x) are exact) against the
    mixed path's outputs there."""
    import numpy as np
    import oracle
    t0 = time.perf_counter()
    L, U, T = g["L"], g["U"], g["T"]
    local = np.searchsorted(g["P"], g["pix"])
    sub = oracle.make_plan(local, g["c"], g["s"], g["valid"], g["nside"], g["kinds"], L,
                           npix=len(g["P"]))
    bin_ref = oracle.bin_map(sub, g["y"])
    map_ref = oracle.bin_map(sub, g["y"] - g["a"][:, U // L])
    Zz = oracle.apply_Z(sub, g["x"][:, U // L])
    pos = np.searchsorted(U, T)
    idx = {b: i for i, b in enumerate(g["baselines"].tolist())}
    col = np.array([idx[t // L] for t in T])
    Ax_ref = np.stack([np.bincount(col, weights=Zz[o, pos], minlength=len(idx))
                       for o in range(Zz.shape[0])])
    return {"method": "sampled: the oracle on every sample of the pixels touched by "
                      f"{len(idx)} sampled baselines (hits, mask, maps and (A x) there are "
                      "exact on that subset)",
            "sampled_baselines": len(idx), "sampled_pixels": int(len(g["P"])),
            "sampled_samples": int(len(U)),
            "hits_mask_bitexact": bool(np.array_equal(g["hits"], sub.hits)
                                       and np.array_equal(g["mask"], sub.mask)),
            "binned_map_rel_rms": rel_rms(g["bin_map"], bin_ref),
            "destriped_map_rel_rms": rel_rms(g["map"], map_ref),
            "operator_rel_rms": rel_rms(g["Ax"], Ax_ref),
            "oracle_s": time.perf_counter() - t0}


def cpu_baseline_leg(args, prob, sampled, sigma):
    """The oracle on the host cores: its rate on a bounded prefix of the same
    workload (one thread, then one copy per core at once), and the mixed path's
    errors against it on the sampled subset."""
    d, n = prefix_numpy(prob, args.oracle_samples)
    rate1, it, dt = oracle_rate(d, args.oracle_iters)
    host = host_cpu()
    procs = args.oracle_procs or host.get("nproc") or 1
    try:
        rate_all, procs = oracle_all_cores(d, args.oracle_iters, procs)
    except Exception as e:  # the one-thread figure still stands
        rate_all, procs = None, 0
        host["all_cores_error"] = str(e)[:200]
    base = {"value": rate_all if rate_all else rate1, "unit": UNIT,
            "cores": procs if rate_all else 1, "kind": "oracle",
            "sample": f"first {n} samples of the same workload: oracle plan + RHS + {it} CG "
                      f"iterations (float64 numpy; {dt:.1f} s on one thread); value = "
                      + (f"{procs} single-thread copies run at once" if rate_all else
                         "one thread"),
            "one_thread": rate1, "all_cores": rate_all, "host": host}
    err = oracle_sampled_errors(sampled) if sampled is not None else None
    return base, err


def e2e_leg(args, prob, ds, world, dist):
    import torch
    h = {"pix": prob.pix.cpu().pin_memory(), "c": prob.c32.cpu().pin_memory(),
         "s": prob.s32.cpu().pin_memory(), "y": prob.y.cpu().pin_memory(),
         "valid": None if prob.valid is None else prob.valid.cpu().pin_memory()}
    from synth import components
    n_c = len(components(prob.kinds))
    out_a = torch.zeros(prob.n_o * prob.n_b, dtype=torch.float64).pin_memory()
    out_m = torch.zeros(n_c * prob.npix, dtype=torch.float64).pin_memory()
    out_h = torch.zeros(prob.npix, dtype=torch.int32).pin_memory()
    out_k = torch.zeros(prob.npix, dtype=torch.uint8).pin_memory()

    def once():
        st, it, rel = ds.destripe_run_host(h["pix"], h["c"], h["s"], h["valid"], h["y"],
                                           nside=prob.nside, kinds=prob.kinds,
                                           baseline_len=prob.baseline_len,
                                           precision=args.precision, tol=args.tol,
                                           out_a=out_a, out_map=out_m, out_hits=out_h,
                                           out_mask=out_k)
        return it

    once()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    iters = 0
    steps = max(1, min(args.steps, 3))
    for _ in range(steps):
        iters += once()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    units = float(prob.n_t) * iters
    if dist is not None:
        dt, units = reduce_over_ranks(dt, units, dist, torch.device("cuda"))
    ysz = 4 if args.precision == "mixed" else 8
    h2d = prob.n_t * (4 + 4 + 4 + ysz * prob.n_o + (1 if prob.valid is not None else 0))
    d2h = 8 * prob.n_o * prob.n_b + 8 * n_c * prob.npix + 4 * prob.npix + prob.npix
    return {"value": units / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * dt / steps,
            "api": "destripe_run_host (pinned host buffers; copies, plan, solve, map, copies back)"}


def _dist_setup():
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    return rank, world, local, dev, (dist if world > 1 else None)


def run_batch(args):
    """Config 3: 64 independent problems of uneven size in one batch."""
    import numpy as np
    import torch
    import paper_1309_5609_gb300 as ds
    from synth import batch_configs, make_problem
    rank, world, local, dev, dist = _dist_setup()
    ds.load_library()
    cfgs = batch_configs(64, seed=1003)
    if args.n_samples:  # each problem cut to its first n_samples (small profiling runs)
        cfgs = [dict(c, n_t=min(c["n_t"], args.n_samples)) for c in cfgs]
    probs = [make_problem(device=dev, y_dtype=torch.float32, keep_f64_trig=False, **c) for c in cfgs]

    shape, tuning = {}, None

    def step(tune=False):
        nonlocal tuning
        plans = [ds.destripe_plan(p.pix, p.c32, p.s32, None, nside=p.nside, kinds=p.kinds,
                                  baseline_len=p.baseline_len, precision="mixed") for p in probs]
        b = ds.destripe_batch_create(len(probs))
        for k, v in shape.items():
            ds.destripe_batch_tune(b, k, v)
        slots = [ds.destripe_batch_add(b, pl, p.y, tol=args.tol) for pl, p in zip(plans, probs)]
        if tune:
            # the autotuner's trials are CG iterations of this job; its shape is
            # kept for the timed jobs
            tuning = ds.destripe_batch_autotune(b)
            shape.update({k: tuning[k] for k in ("tile_samples", "tile_pixels",
                                                 "tile_unknowns", "blocks_per_sm")})
        while ds.destripe_batch_step(b, 8) > 0:
            pass
        iters, stats = [], []
        for sl, pl in zip(slots, plans):
            a = torch.empty(pl.n_u, dtype=torch.float64, device=dev)
            st, it, rel = ds.destripe_batch_retire(b, sl, a)
            iters.append(it)
            stats.append(st)
        launches = ds.destripe_batch_info(b)["kernel_launches"] + 3 * len(plans)
        b.close()
        for pl in plans:
            pl.close()
        return iters, stats, launches

    for w in range(args.warmup):
        step(tune=(w == 0 and not args.no_autotune))
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    units, launches, iters_all, ok = 0.0, 0, [], True
    with Clocks(local) as clk:
        ev0.record()
        for _ in range(args.steps):
            iters, stats, l = step()
            units += sum(p.n_t * it for p, it in zip(probs, iters))
            launches += l
            iters_all += iters
            ok &= all(s == ds.DS_OK for s in stats)
        ev1.record()
        torch.cuda.synchronize()
    t_ms = ev0.elapsed_time(ev1)
    if dist is not None:
        t_ms, units = reduce_over_ranks(t_ms, units, dist, dev)
    # comparator: the same problems solved one after the other
    ev0.record()
    seq_units = 0.0
    for p in probs:
        pl = ds.destripe_plan(p.pix, p.c32, p.s32, None, nside=p.nside, kinds=p.kinds,
                              baseline_len=p.baseline_len, precision="mixed")
        a = torch.empty(pl.n_u, dtype=torch.float64, device=dev)
        st, it, rel = ds.destripe_solve(pl, p.y, a, tol=args.tol)
        seq_units += p.n_t * it
        pl.close()
    ev1.record()
    torch.cuda.synchronize()
    seq_ms = ev0.elapsed_time(ev1)
    # the plain float64 single-problem path on the same problems
    seq64 = None
    if not args.no_fp64_comparator:
        ev0.record()
        s64_units = 0.0
        for p in probs:
            pl = ds.destripe_plan(p.pix, p.c32, p.s32, None, nside=p.nside, kinds=p.kinds,
                                  baseline_len=p.baseline_len, precision="fp64")
            a = torch.empty(pl.n_u, dtype=torch.float64, device=dev)
            st, it, rel = ds.destripe_solve(pl, p.y.double().contiguous(), a, tol=args.tol)
            s64_units += p.n_t * it
            pl.close()
        ev1.record()
        torch.cuda.synchronize()
        s64_ms = ev0.elapsed_time(ev1)
        seq64 = {"value": s64_units / (s64_ms / 1e3), "unit": UNIT, "ms": s64_ms,
                 "note": "float64 plans, one solve after another (y promoted to float64 "
                         "inside the timed region)"}
    peak, peak_kind = peaks()
    value = units / (t_ms / 1e3)
    achieved = 2 * BYTES_PER_SAMPLE_PASS * value / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (64 seeded scans), resident in HBM",
            "config": {"workload": "batch64-qu-nside64-256-1e6-3e7-L50-3000"
                       + (f"-cap{args.n_samples}" if args.n_samples else ""),
                       "problems": len(probs), "n_samples_total": int(sum(p.n_t for p in probs)),
                       "precision": "mixed", "tol": args.tol,
                       "step": "64 plans + batched RHS/CG (one graph per 8 iterations) + retire"},
            "roofline": {"bound": "hbm", "kernel": "whole batched job (all kernels)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "note": "24 B per sample-iteration over the whole job time"},
            "iterations": {"mean": float(np.mean(iters_all)), "max": int(max(iters_all))},
            "all_converged": bool(ok), "gpu_launches": int(launches),
            "sequential_single_solves": {"value": seq_units / (seq_ms / 1e3), "unit": UNIT,
                                         "ms": seq_ms},
            "sequential_fp64_single_solves": seq64,
            "autotune": tuning, "launch_shape": shape or "defaults",
            "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def iteration_stats(reqs, ok_status):
    """Iterations of converged requests, and the share of the work spent on the rest."""
    import numpy as np
    it_ok = [r.iters for r in reqs if r.status == ok_status]
    work = [r.n_t * r.iters for r in reqs]
    bad = [r.n_t * r.iters for r in reqs if r.status != ok_status]
    tot = float(sum(work)) or 1.0
    share = lambda sel: float(sum(r.n_t * r.iters for r in reqs if sel(r)) / tot)
    return {"converged_p50": float(np.percentile(it_ok, 50)) if it_ok else None,
            "converged_p99": float(np.percentile(it_ok, 99)) if it_ok else None,
            "converged_max": int(max(it_ok)) if it_ok else None,
            "not_converged": len(bad),
            "not_converged_work_share": float(sum(bad) / tot),
            "work_share_lone_q": share(lambda r: len(r.kinds) == 1),
            "work_share_over_1000_iterations": share(lambda r: r.iters > 1000),
            "requests_over_1000_iterations": sum(1 for r in reqs if r.iters > 1000)}


def run_serve(args):
    """Config 5: Poisson request stream served with continuous batching."""
    import numpy as np
    import torch
    import paper_1309_5609_gb300 as ds
    from paper_1309_5609_gb300.serve import Request, Server, fifo_latencies, poisson_trace
    from synth import make_problem
    rank, world, local, dev, dist = _dist_setup()
    ds.load_library()
    n_master = args.serve_master
    nsides = (64, 128, 256, 512)
    master = {}
    for ns in nsides:  # one scan, pixelised at each nside; same trig and noise seed
        p = make_problem(n_master, ns, ("q", "u"), baseline_len=500, f_knee=0.1, alpha=1.7,
                         seed=5000, device=dev, y_dtype=torch.float32, keep_f64_trig=False)
        master[ns] = (p.pix.cpu().pin_memory(), p.c32.cpu().pin_memory(),
                      p.s32.cpu().pin_memory(), [p.y[0].cpu().pin_memory(), p.y[1].cpu().pin_memory()])
        del p
    torch.cuda.empty_cache()
    trace = poisson_trace(20.0, args.serve_seconds, seed=5000 + rank, n_min=1e5,
                          n_max=min(2e8, n_master), nsides=nsides)
    reqs = []
    for i, r in enumerate(trace):
        pix, c, s, y = master[r["nside"]]
        n = min(r["n_t"], n_master)
        s0 = r["start"] % (n_master - n + 1)
        rows = [y[o][s0:s0 + n] for o in range(len(r["kinds"]))]
        reqs.append(Request(i, r["arrival"], r["nside"], r["kinds"], r["baseline_len"],
                            pix[s0:s0 + n], c[s0:s0 + n], s[s0:s0 + n], rows, tol=args.tol))
    # warm-up on a few requests (kernels, graph capture)
    warm = Server(max_slots=64, hbm_budget=200 << 30)
    warm.run([Request(**{**r.__dict__, "arrival": 0.0}) for r in reqs[:3]])
    warm.close()
    cap = int(args.serve_cap) if args.serve_cap > 0 else None
    srv = Server(max_slots=64, hbm_budget=200 << 30, iters_per_step=8, max_resident_samples=cap)
    with Clocks(local) as clk:
        stats = srv.run(reqs)
    srv.close()
    summ = stats.summary()
    ok = sum(r.status == ds.DS_OK for r in reqs)
    # comparator: the same requests served one after the other by plain float64
    # solves (copies to the device, plan, solve, baselines back), each request's
    # service time measured, the FIFO latencies computed from the arrivals
    svc, seq_units = [], 0.0
    limit = args.serve_comparator if args.serve_comparator > 0 else len(reqs)
    for r in reqs[:limit]:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = [t.to(dev) for t in (r.pix, r.cos2psi, r.sin2psi)]
        y64 = torch.stack([row.to(dev) for row in r.y]).double().contiguous()
        pl = ds.destripe_plan(g[0], g[1], g[2], None, nside=r.nside, kinds=r.kinds,
                              baseline_len=r.baseline_len, precision="fp64")
        a = torch.empty(pl.n_u, dtype=torch.float64, device=dev)
        try:
            st, it, rel = ds.destripe_solve(pl, y64, a, tol=args.tol)
        except ds.DestripeError:
            it = 0
        a_h = a.cpu()
        svc.append(time.perf_counter() - t0)
        seq_units += r.n_t * it
        pl.close()
        del g, y64, a
    seq_lat = fifo_latencies([r.arrival for r in reqs[:limit]], svc)
    seq_wall = max(r.arrival + l for r, l in zip(reqs[:limit], seq_lat))
    units = float(stats.sample_iters)
    t_s = stats.wall
    if dist is not None:
        t_ms, units = reduce_over_ranks(1e3 * t_s, units, dist, dev)
        t_s = t_ms / 1e3
    peak, peak_kind = peaks()
    value = units / t_s
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": 1,
            "warmup": 1, "ms_per_step": 1e3 * t_s, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic requests: windows of host-resident master scans",
            "config": {"workload": f"serve-poisson20-{args.serve_seconds:g}s",
                       "requests": len(reqs), "rate_per_s": 20.0,
                       "lengths": f"log-uniform 1e5..{min(2e8, n_master):.0e}",
                       "nside": list(nsides), "baselines_s": [0.5, 60.0], "outputs": "q or q,u",
                       "precision": "mixed", "tol": args.tol, "max_slots": 64,
                       "max_resident_samples": cap},
            "p50_s": summ["p50_s"], "p99_s": summ["p99_s"], "mean_latency_s": summ["mean_s"],
            "iterations": iteration_stats(reqs, ds.DS_OK),
            "samples_per_s": summ["samples_per_s"], "converged": int(ok),
            "host_time_s": {k: summ[k] for k in ("host_admit_s", "host_step_s", "host_retire_s")},
            "max_resident": summ["max_resident"], "gpu_launches": summ["kernel_launches"],
            "sequential_fp64_fifo": {
                "p50_s": float(np.percentile(seq_lat, 50)), "p99_s": float(np.percentile(seq_lat, 99)),
                "value": seq_units / seq_wall, "unit": UNIT, "requests": limit,
                "note": "every request's float64 solve timed one after the other on the same "
                        "GPU (copies, plan, solve, copy back); FIFO latencies from the arrivals"},
            "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.config == 3:
        return run_batch(args)
    if args.config == 5:
        return run_serve(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
