"""Continuous-batching request loop for EXACT reconstructions on one GPU.

A request carries a scan geometry, the energy attenuations and window weights,
the counts (on the host), the source intensity, a relative-residual tolerance
and an iteration cap.  The loop admits waiting requests, first come first
served, while their device footprint fits the HBM budget, a batch slot is free
and the resident jobs' work per iteration (nonzeros of A) stays below what
fills the GPU on its own (`sat_work`, about one 512^2 x 720-view fan scan:
past that, interleaving more jobs adds latency but no throughput, so larger
jobs run one after another): it builds the plan,
binds a workspace, uploads the counts, estimates ||A||^2 (FP32 power
iteration) for the step size 1/(4L), and keeps all of it resident.  Every
round runs `round_iters` extragradient iterations of all resident jobs in one
persistent launch (exact_batch_solve); a job resumes from its own iterate, so a
round boundary changes nothing in its arithmetic.  After a round the loop reads
each job's residual, retires the converged ones (their memory is freed) and
admits new arrivals, which therefore overlap on the device with the jobs
already running.  A round with a single resident job runs it with
exact_solve instead, with the adjoint split autotuned for its shape (the
persistent kernel runs one CTA per adjoint tile, which only pays when several
jobs share the GPU).

This is host orchestration only: all arithmetic runs in libexact.so.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass

import torch

from .exact import Batch, Geometry, Job, Plan


@dataclass
class Request:
    """One reconstruction request; y is a host tensor [W][V][B] (float32 or
    bfloat16), mu the K attenuations, S the [W][K] window weights."""
    geometry: Geometry
    mu: list
    S: list
    y: torch.Tensor
    I0: float
    tol: float = 1e-4
    max_iters: int = 2000
    check_every: int = 1
    lo: float = 0.0
    hi: float = math.inf
    arrival: float = 0.0          # seconds on the server clock
    tag: object = None


@dataclass
class Result:
    tag: object
    x: torch.Tensor               # host float32 image
    iters: int
    rel_res: float
    status: int
    arrival: float
    admitted: float
    finished: float

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Active:
    req: Request
    plan: Plan
    y: torch.Tensor
    x: torch.Tensor
    eta: float
    footprint: int
    iters: int = 0
    admitted: float = 0.0
    work: float = 0.0
    tuned: bool = False


def work_per_iter(geometry: Geometry) -> float:
    """Nonzeros of A, about rays x the driving-axis length (an estimate of
    the gather work of one forward or adjoint)."""
    return float(geometry.n_views) * geometry.n_bins * max(geometry.nx, geometry.ny)


def footprint_bytes(geometry: Geometry, W: int, y_itemsize: int) -> int:
    """Device bytes a resident job holds: plan tables (FP32 and FP64 ray
    records, bits, steps, views, forward units), the workspace (padded image
    copies, residual and collapsed counts, FP64 power-iteration buffers,
    partial sums), the counts and the iterate.  An upper estimate; the plan's
    own figure is used once it exists."""
    n = geometry.n_views * geometry.n_bins
    d = geometry.nx * geometry.ny
    ldr, ldc = geometry.nx + 8, geometry.ny + 8
    tables = n * (16 + 16 + 4 + 4 + 32) + geometry.n_views * 48 + (n // 16 + 1) * 32 * 8
    ws = 4 * 2 * (geometry.ny * ldr + geometry.nx * ldc) + 8 * n + 8 * (geometry.ny * ldr + geometry.nx * ldc) \
        + 8 * n + 8 * d + 4 * d + (1 << 20) + (13 + 1) * 4 * d + (64 << 10)  # + TV-ball projection buffers
    return tables + ws + W * n * y_itemsize + 4 * d


class Server:
    """Continuous-batching EXACT server on the current CUDA device."""

    def __init__(self, budget_bytes: float = 150e9, max_slots: int = 64, round_iters: int = 20,
                 norm_iters: int = 60, norm_rtol: float = 1e-5, sat_work: float = 4e8):
        self.budget = int(budget_bytes)
        self.sat_work = float(sat_work)
        self.work = 0.0
        self.max_slots = max_slots
        self.round_iters = round_iters
        self.norm_iters = norm_iters
        self.norm_rtol = norm_rtol
        self.batch = Batch(max_slots)
        self.waiting: deque[Request] = deque()
        self.active: list[_Active] = []
        self.used = 0
        self.t0 = time.perf_counter()
        self.rounds = 0
        self.peak_used = 0

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req: Request):
        self.waiting.append(req)

    def _admit(self):
        while self.waiting and len(self.active) < self.max_slots:
            req = self.waiting[0]
            need = footprint_bytes(req.geometry, len(req.S), req.y.element_size())
            if self.used + need > self.budget and self.active:
                break  # wait for memory to free up
            w = work_per_iter(req.geometry)
            if self.active and self.work + w > self.sat_work:
                break  # the GPU is full: wait for a job to finish
            self.waiting.popleft()
            plan = Plan(req.geometry, req.mu, req.S)
            y = req.y.to(plan.device, non_blocking=True).contiguous()
            x = torch.zeros(plan.shape_img, dtype=torch.float32, device=plan.device)
            lam, _ = plan.norm_estimate_f32(self.norm_iters, self.norm_rtol)
            eta = plan.recommended_eta(req.I0, lam)
            self.active.append(_Active(req, plan, y, x, eta, need, 0, self.now(), w))
            self.used += need
            self.work += w
            self.peak_used = max(self.peak_used, self.used)

    def step(self) -> list[Result]:
        """Admit, run one round over the resident jobs, retire finished ones."""
        self._admit()
        if not self.active:
            return []
        jobs = []
        for a in self.active:
            k = min(self.round_iters, a.req.max_iters - a.iters)
            jobs.append(Job(plan=a.plan, y=a.y, I0=a.req.I0, eta=a.eta, iters=k, x=a.x, lo=a.req.lo, hi=a.req.hi,
                            tol=a.req.tol, check_every=a.req.check_every))
        if len(self.active) == 1:
            a, jb = self.active[0], jobs[0]
            if not a.tuned:
                a.plan.autotune()
                a.tuned = True
            _, info = a.plan.solve(jb.y, jb.I0, jb.eta, jb.iters, x=jb.x, lo=jb.lo, hi=jb.hi, tol=jb.tol,
                                   check_every=jb.check_every, sync=True)
            infos = [info]
        else:
            _, infos = self.batch.solve(jobs, sync=True)
        self.rounds += 1
        done, keep = [], []
        for a, jb, info in zip(self.active, jobs, infos):
            a.iters += info.iters_done
            stopped = info.iters_done < jb.iters or (a.req.tol > 0 and info.rel_res <= a.req.tol
                                                     and a.iters % a.req.check_every == 0)
            if stopped or a.iters >= a.req.max_iters or info.status != 0:
                res = Result(a.req.tag, a.x.cpu(), a.iters, info.rel_res, info.status, a.req.arrival, a.admitted,
                             self.now())
                done.append(res)
                a.plan.close()
                self.used -= a.footprint
                self.work -= a.work
            else:
                keep.append(a)
        self.active = keep
        return done

    def run(self, requests: list[Request], realtime: bool = True) -> list[Result]:
        """Serve `requests` (sorted by arrival).  With realtime, a request is
        only visible once the server clock passes its arrival time."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        results = []
        self.t0 = time.perf_counter()
        while pending or self.waiting or self.active:
            now = self.now()
            while pending and (not realtime or pending[0].arrival <= now):
                self.submit(pending.popleft())
            if not self.waiting and not self.active:
                time.sleep(max(0.0, min(0.01, pending[0].arrival - now)))
                continue
            results.extend(self.step())
        return results

    def close(self):
        for a in self.active:
            a.plan.close()
        self.active = []
        self.batch.close()


def serve_sequential(requests: list[Request], realtime: bool = True, norm_iters: int = 60,
                     norm_rtol: float = 1e-5) -> list[Result]:
    """The plain baseline: first come, first served, each request solved alone
    with exact_solve (same tolerance test every check_every iterations), each
    plan with the autotuned adjoint split of its shape."""
    pending = deque(sorted(requests, key=lambda r: r.arrival))
    out = []
    t0 = time.perf_counter()
    while pending:
        now = time.perf_counter() - t0
        req = pending[0]
        if realtime and req.arrival > now:
            time.sleep(min(0.01, req.arrival - now))
            continue
        pending.popleft()
        admitted = time.perf_counter() - t0
        plan = Plan(req.geometry, req.mu, req.S)
        y = req.y.to(plan.device).contiguous()
        plan.autotune()
        lam, _ = plan.norm_estimate_f32(norm_iters, norm_rtol)
        eta = plan.recommended_eta(req.I0, lam)
        x, info = plan.solve(y, req.I0, eta, req.max_iters, lo=req.lo, hi=req.hi, tol=req.tol,
                             check_every=req.check_every)
        out.append(Result(req.tag, x.cpu(), info.iters_done, info.rel_res, info.status, req.arrival, admitted,
                          time.perf_counter() - t0))
        plan.close()
    return out
