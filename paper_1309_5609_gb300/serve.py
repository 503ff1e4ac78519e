"""Serving loop: destriping requests answered with iteration-level continuous
batching on one GPU.

Requests arrive over time (e.g. a Poisson stream).  A request is a window of a
host-resident scan: pointing, rotation trig and the timelines of one or two
outputs.  The server

  * admits an arrived request when a batch slot is free and its device
    footprint fits the HBM budget: its arrays are copied to the device on a side
    stream, a plan is built and the problem joins the running batch;
  * advances every admitted problem by a few CG iterations per step (one graph
    replay covering all of them, so newly admitted work overlaps with work in
    progress);
  * retires problems as soon as they converge: baselines are gauge-fixed and
    copied back, device memory returns to the budget;
  * records per-request latency (arrival to result on the host) and iteration
    counts, and reports p50 / p99 and aggregate throughput.

Every computational step runs in libdestripe.so (plan, right-hand side, batched
CG, gauge).  This module only schedules and moves data.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

from . import (DS_OK, DestripeError, destripe_batch_add, destripe_batch_create, destripe_batch_info,
               destripe_batch_retire, destripe_batch_slot_status, destripe_batch_step,
               destripe_plan, destripe_tune)


@dataclass
class Request:
    rid: int
    arrival: float            # seconds after the server's start
    nside: int
    kinds: tuple              # ("q",) or ("q", "u")
    baseline_len: int
    pix: object               # host tensors (pinned) of this request's window
    cos2psi: object
    sin2psi: object
    y: object                 # float32 [n_o, n_t], or a list of n_o float32 [n_t] rows
    tol: float = 1e-10
    accurate_start: Optional[bool] = None  # None: the server's size rule
    # filled by the server
    admitted: float = -1.0
    finished: float = -1.0
    iters: int = 0
    rel_resid: float = float("nan")
    status: int = -1
    a: Optional[object] = None  # host float64 baselines

    @property
    def n_t(self) -> int:
        return int(self.pix.numel())

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def device_bytes(n_t: int, n_o: int, nside: int, baseline_len: int) -> int:
    """Upper bound of the device footprint of one admitted request: its arrays and
    its mixed-precision plan (the plan reports its exact figure once built)."""
    npix = 12 * nside * nside
    n_b = -(-n_t // baseline_len)
    n_u = n_o * n_b
    arrays = n_t * (4 + 4 + 4 + 4 * n_o)          # pix, cos, sin, y (float32)
    per_pixel = 4 + 1 + 8 * 6 + 8 * 4 * 2 + 4 * 4 * 3 + 4   # hits, mask, M^-1, sums, maps, runs
    runs = int(0.6 * (36 + 24) * n_t)              # run records, time- and pixel-major (<= 0.6/sample)
    plan = (n_t * 4 + npix * per_pixel + n_u * (8 * 7 + 8 + 4) + n_b * (4 + 48) + runs
            + (n_t // 512 + 1) * 8 + (1 << 16))  # per-baseline counts and packed baselines, scalars
    return int(arrays + plan)


@dataclass
class ServeStats:
    latencies: List[float] = field(default_factory=list)
    samples: int = 0
    sample_iters: int = 0
    wall: float = 0.0
    steps: int = 0
    max_resident: int = 0
    kernel_launches: int = 0
    t_admit: float = 0.0     # host seconds in admission (copies, plan, right-hand side)
    t_step: float = 0.0      # host seconds in batch steps (graph replays, waits)
    t_retire: float = 0.0    # host seconds in retirement (gauge, copy back)

    def summary(self) -> dict:
        lat = np.array(self.latencies) if self.latencies else np.array([np.nan])
        return {"requests": len(self.latencies), "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
                "samples_per_s": self.samples / self.wall if self.wall else None,
                "sample_iters_per_s": self.sample_iters / self.wall if self.wall else None,
                "wall_s": self.wall, "steps": self.steps, "max_resident": self.max_resident,
                "kernel_launches": self.kernel_launches, "host_admit_s": self.t_admit,
                "host_step_s": self.t_step, "host_retire_s": self.t_retire}


class Server:
    """Continuous-batching destriping server on the current CUDA device.

    Requests shorter than accurate_below samples iterate with the accurate
    operator from the start: on small, ill-conditioned problems the float32
    operator costs CG its conjugacy and several times the iterations, while their
    accurate iterations are cheap.

    max_resident_samples (optional) caps the samples of the admitted problems: the
    batch shares the GPU among everything admitted, so an unbounded resident set
    stretches every request; with a cap, arrivals wait in the queue (in arrival
    order) while the admitted ones finish sooner.  A request larger than the cap
    is admitted when nothing else is resident."""

    def __init__(self, max_slots: int = 64, hbm_budget: int = 64 << 30,
                 iters_per_step: int = 8, clock: Callable[[], float] = time.perf_counter,
                 accurate_below: int = 3_000_000, max_resident_samples: Optional[int] = None):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.stream = torch.cuda.current_stream(self.dev)
        self.copy_stream = torch.cuda.Stream(self.dev)
        self.batch = destripe_batch_create(max_slots, self.stream.cuda_stream)
        self.max_slots = max_slots
        self.budget = int(hbm_budget)
        self.iters_per_step = iters_per_step
        self.accurate_below = accurate_below
        self.clock = clock
        self.used = 0
        self.max_resident_samples = max_resident_samples
        self.resident_samples = 0
        self.queue: List[Request] = []       # arrived, not admitted
        self.resident = {}                   # slot -> (request, plan, device tensors, bytes)
        self.done: List[Request] = []
        self.stats = ServeStats()
        self.t0 = None

    def now(self) -> float:
        return self.clock() - self.t0

    def _admit(self, req: Request) -> bool:
        torch = self.torch
        need = device_bytes(req.n_t, len(req.kinds), req.nside, req.baseline_len)
        if need > self.budget:
            raise ValueError(f"request {req.rid} needs {need} bytes, above the HBM budget")
        if self.used + need > self.budget or len(self.resident) >= self.max_slots:
            return False
        if (self.max_resident_samples is not None and self.resident
                and self.resident_samples + req.n_t > self.max_resident_samples):
            return False
        rows = list(req.y) if isinstance(req.y, (list, tuple)) else [req.y[o] for o in range(len(req.kinds))]
        with torch.cuda.stream(self.copy_stream):
            pix = req.pix.to(self.dev, non_blocking=True)
            c = req.cos2psi.to(self.dev, non_blocking=True)
            s = req.sin2psi.to(self.dev, non_blocking=True)
            y = torch.empty((len(rows), req.n_t), dtype=torch.float32, device=self.dev)
            for o, row in enumerate(rows):
                y[o].copy_(row, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.copy_stream)
        self.stream.wait_event(ev)
        for t in (pix, c, s, y):
            t.record_stream(self.stream)
        plan = destripe_plan(pix, c, s, None, nside=req.nside, kinds=req.kinds,
                             baseline_len=req.baseline_len, precision="mixed",
                             stream=self.stream.cuda_stream)
        acc = req.accurate_start if req.accurate_start is not None else req.n_t < self.accurate_below
        if acc:
            destripe_tune(plan, "accurate_start", 1)
        try:
            slot = destripe_batch_add(self.batch, plan, y, tol=req.tol)
        except DestripeError as e:
            # refused at admission (non-finite data): answered at once, no slot held
            req.admitted = req.finished = self.now()
            req.status, req.iters = e.status, 0
            plan.close()
            self.done.append(req)
            self.stats.latencies.append(req.latency)
            return True
        req.admitted = self.now()
        self.resident[slot] = (req, plan, (pix, c, s, y), need)
        self.used += need
        self.resident_samples += req.n_t
        self.stats.max_resident = max(self.stats.max_resident, len(self.resident))
        return True

    def _retire_finished(self):
        torch = self.torch
        for slot in list(self.resident):
            done, it, rel = destripe_batch_slot_status(self.batch, slot)
            if not done:
                continue
            req, plan, arrays, need = self.resident.pop(slot)
            a = torch.empty(plan.n_u, dtype=torch.float64, device=self.dev)
            st, it, rel = destripe_batch_retire(self.batch, slot, a)
            req.a = a.cpu()
            req.finished = self.now()
            req.iters, req.rel_resid, req.status = it, rel, st
            plan.close()
            self.used -= need
            self.resident_samples -= req.n_t
            self.done.append(req)
            self.stats.latencies.append(req.latency)
            self.stats.samples += req.n_t
            self.stats.sample_iters += req.n_t * it

    def run(self, requests: List[Request], time_limit: Optional[float] = None) -> ServeStats:
        """Serve a trace (requests sorted by arrival time) until every request is answered."""
        pending = sorted(requests, key=lambda r: r.arrival)
        self.t0 = self.clock()
        while pending or self.queue or self.resident:
            t = self.now()
            while pending and pending[0].arrival <= t:
                self.queue.append(pending.pop(0))
            c0 = self.clock()
            while self.queue and self._admit(self.queue[0]):
                self.queue.pop(0)
            c1 = self.clock()
            self.stats.t_admit += c1 - c0
            if self.resident:
                destripe_batch_step(self.batch, self.iters_per_step)
                self.stats.steps += 1
                c2 = self.clock()
                self.stats.t_step += c2 - c1
                self._retire_finished()
                self.stats.t_retire += self.clock() - c2
            elif pending:
                time.sleep(max(0.0, min(0.01, pending[0].arrival - self.now())))
            if time_limit is not None and self.now() > time_limit:
                break
        self.stats.wall = self.now()
        self.stats.kernel_launches = destripe_batch_info(self.batch)["kernel_launches"]
        return self.stats

    def close(self):
        for slot, (req, plan, arrays, need) in list(self.resident.items()):
            plan.close()
        self.resident = {}
        self.batch.close()


def poisson_trace(rate: float, duration: float, seed: int, n_min: float, n_max: float,
                  nsides=(64, 128, 256, 512), baselines_s=(0.5, 60.0), f_samp: float = 50.0,
                  kinds=(("q",), ("q", "u"))):
    """Seeded request parameters: Poisson arrivals, log-uniform lengths, nside from
    the list, baseline length log-uniform in seconds, outputs drawn from `kinds`
    (by default a lone q output or a q, u pair, with equal odds)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        n_t = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        L = int(round(f_samp * np.exp(rng.uniform(np.log(baselines_s[0]), np.log(baselines_s[1])))))
        out.append(dict(arrival=t, n_t=n_t, nside=int(rng.choice(nsides)),
                        kinds=tuple(kinds[int(rng.integers(0, len(kinds)))]),
                        baseline_len=max(1, L), start=int(rng.integers(0, 1 << 30))))
    return out


def fifo_latencies(arrivals, service_times):
    """Latencies of a single FIFO server with the given service times."""
    free, lat = 0.0, []
    for a, s in zip(arrivals, service_times):
        start = max(a, free)
        free = start + s
        lat.append(free - a)
    return lat
