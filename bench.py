#!/usr/bin/env python
"""Benchmark of the GB300 destriper on a synthetic scan shaped like the paper's
30-day B-Machine channel (1.3e8 samples at 50 Hz; I, q, u outputs; nside 256;
60 s baselines).

One step = the whole destriping job on inputs already resident in HBM: plan
(hits, pixel matrices, rcond cut), right-hand side, CG to ||r||/||b|| < 1e-10,
gauge, destriped map.  value = timestream samples x CG iterations / step time,
summed over ranks and divided by the slowest rank's time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--config 2|4|1] [--precision mixed|fp64]

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
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 4])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--n-samples", type=int, default=None, help="cut the workload (testing)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--oracle-samples", type=int, default=1_000_000)
    ap.add_argument("--oracle-iters", type=int, default=20)
    return ap.parse_args()


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


def kernel_traffic(n_t, kernel):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, scaled by
    samples, or None if the summary is missing or the kernel source has changed."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.md")
    src = os.path.join(ROOT, "paper_1309_5609_gb300", "csrc", "apply.cu")
    try:
        text = open(path).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        m_sha = re.search(r"apply\.cu sha256\[:16\]:\s*([0-9a-f]+)", text)
        m_bps = re.search(r"dram bytes per sample:\s*([0-9.]+)", text)
        if not m_sha or not m_bps or m_sha.group(1) != sha:
            return None
        return float(m_bps.group(1)) * n_t
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
    return {"workload": name, "n_samples": n_t, "nside": c["nside"],
            "outputs": ",".join(c["kinds"]), "baseline_len": c["baseline_len"],
            "unknowns": len(c["kinds"]) * n_b, "precision": args.precision, "tol": args.tol,
            "flagged_fraction": c.get("flag_frac", 0.0),
            "l2": "inputs larger than L2 (pointing and timelines stream from HBM every pass)",
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
    from synth import WORKLOAD_NAMES, config_problem
    import torch
    n = min(args.oracle_samples, args.n_samples or 10 ** 12)
    prob = config_problem(args.config, n_t=n, keep_f64_trig=False,
                          y_dtype=torch.float32 if args.precision == "mixed" else torch.float64)
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
    name = WORKLOAD_NAMES[args.config]
    sample = (f"prefix of {n} samples of {name}: plan + RHS + {iters_per_step} CG iterations "
              f"per step, float64 numpy, 1 thread")
    cfg = config_dict(args)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded scan, Gaussian sky, 1/f noise)", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
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

    def step(prof_acc):
        plan = ds.destripe_plan(prob.pix, prob.c32, prob.s32, prob.valid, nside=prob.nside,
                                kinds=prob.kinds, baseline_len=prob.baseline_len,
                                precision=args.precision)
        if prof_acc is not None:
            ds.destripe_profile(plan, 1)
        st, iters, rel = ds.destripe_solve(plan, prob.y, a, tol=args.tol)
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
            it, rel = step(prof)
            iters_tot += it
            rels.append(rel)
        ev1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    t_ms = ev0.elapsed_time(ev1)
    units = float(prob.n_t) * iters_tot
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
    kname = {"bin": "k_bin", "rescan": "k_rescan"}[dom]
    roof = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
            "traffic": kernel_traffic(prob.n_t, kname),
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
            "config": config_dict(args, name), "roofline": roof,
            "iterations_per_step": iters_tot / args.steps,
            "rel_resid_max": max(rels) if rels else None,
            "gpu_launches": int(prof.get("kernel_launches", 0)),
            "clocks": clk.summary()}

    # end to end through the C ABI with host buffers (copies inside the timed region)
    if not args.no_e2e:
        line["e2e"] = e2e_leg(args, prob, ds, world, dist if world > 1 else None)
    if rank == 0 and not args.no_cpu_baseline:
        d, n = prefix_numpy(prob, args.oracle_samples)
        rate, it, dt = oracle_rate(d, args.oracle_iters)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"first {n} samples of the same workload: oracle "
                                          f"plan + RHS + {it} CG iterations in {dt:.1f} s "
                                          f"(float64 numpy, 1 thread)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


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


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
