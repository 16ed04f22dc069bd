"""Continuous-batching request loop for EXACT reconstructions on one GPU.

A request carries a scan geometry, the energy attenuations and window weights,
the counts (on the host), the source intensity, a relative-residual tolerance
and an iteration cap.  The loop admits waiting requests, first come first
served, while their device footprint fits the HBM budget, a batch slot is free
and the resident jobs' work per iteration (nonzeros of A) stays below what
fills the GPU on its own (`sat_work`, about one 512^2 x 720-view fan scan:
past that, interleaving more jobs adds latency but no throughput, so larger
jobs run one after another).

Admitting a request means building its plan (host FP64 tables), binding a
workspace, uploading the counts and estimating ||A||^2 (FP32 power iteration)
for the step size 1/(4L).  That work runs on a worker thread with a CUDA
stream of its own, so it overlaps the jobs already running on the device.
Everything a job needs stays resident until it retires; retiring frees the
plan on another worker thread (freeing device memory waits for the device).

Two ways to run the resident jobs (Server.mode):
 - "streams" (default): each job's whole solve is one exact_solve call on a
   CUDA stream of its own, its iterations looping on the device in a CUDA
   graph until the tolerance stop; jobs admitted while others run start at
   once and their kernels overlap with the others' on the GPU.  Each result
   is bitwise the job's plain solve.
 - "rounds": every round runs `round_iters` iterations of all resident jobs
   in one persistent launch (exact_batch_solve); a job resumes from its own
   iterate, so a round boundary changes nothing in its arithmetic.  After a
   round the loop retires the converged jobs and takes in prepared arrivals.
   A round with a single resident job runs exact_solve instead.

Both the server and the one-at-a-time baseline (serve_sequential) give every
request the same set-up: the plan's default adjoint split (no per-request
autotuning), the same power iteration and the same tolerance test.

This is host orchestration only: all arithmetic runs in libexact.so.
"""
from __future__ import annotations

import math
import time
from collections import deque
from concurrent.futures import Future, ThreadPoolExecutor
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
    stream: object = None         # streams mode: the job's CUDA stream
    info: object = None           # streams mode: the solve's info (filled at its end)
    done: object = None           # streams mode: event recorded after the solve


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
        + 8 * n + 8 * d + 4 * d + (1 << 20) + (13 + 1) * 4 * d + (64 << 10) \
        + 4 * W * n + 4 * d + 64 * d  # + TV-ball projection buffers, host-buffer staging, view-split partials
    return tables + ws + W * n * y_itemsize + 4 * d


def prepare(req: Request, norm_iters: int, norm_rtol: float):
    """Plan, resident counts, zero image and step size 1/(4L) of a request,
    on the current device and stream (synchronises that stream)."""
    plan = Plan(req.geometry, req.mu, req.S)
    y = req.y.to(plan.device, non_blocking=True).contiguous()
    x = torch.zeros(plan.shape_img, dtype=torch.float32, device=plan.device)
    lam, _ = plan.norm_estimate_f32(norm_iters, norm_rtol)
    return plan, y, x, plan.recommended_eta(req.I0, lam)


class Server:
    """Continuous-batching EXACT server on the current CUDA device.

    mode "streams" (default): every resident job runs its whole solve --
    iterations looping on the device in a CUDA graph until its tolerance stop
    or cap -- on a CUDA stream of its own, so the kernels of concurrent jobs
    overlap on the GPU wherever one job leaves SMs idle; the host only admits,
    launches and retires.  mode "rounds": all resident jobs advance
    `round_iters` iterations at a time in one persistent launch of
    exact_batch_solve (a lone job through exact_solve), with the host
    retiring converged jobs and admitting new ones between rounds."""

    def __init__(self, budget_bytes: float = 150e9, max_slots: int = 64, round_iters: int = 20,
                 norm_iters: int = 60, norm_rtol: float = 1e-5, sat_work: float = 4e8, prepare_workers: int = 1,
                 mode: str = "streams"):
        if mode not in ("streams", "rounds"):
            raise ValueError("mode must be 'streams' or 'rounds'")
        self.mode = mode
        self.budget = int(budget_bytes)
        self.sat_work = float(sat_work)
        self.work = 0.0
        self.max_slots = max_slots
        self.round_iters = round_iters
        self.norm_iters = norm_iters
        self.norm_rtol = norm_rtol
        self.batch = Batch(max_slots) if mode == "rounds" else None
        self.device = torch.device("cuda", torch.cuda.current_device()) if torch.cuda.is_available() else None
        self.waiting: deque[Request] = deque()
        self.preparing: deque[tuple[Future, Request, int, float]] = deque()
        self.active: list[_Active] = []
        self.used = 0
        self.t0 = time.perf_counter()
        self.rounds = 0
        self.launches = 0
        self.peak_used = 0
        self.peak_resident = 0
        self._pool = ThreadPoolExecutor(max_workers=prepare_workers) if prepare_workers > 0 else None
        self._prep_stream = torch.cuda.Stream(device=self.device) if self._pool and self.device else None
        # plan teardown frees device memory, which waits for the device: off the serving thread
        self._reaper = ThreadPoolExecutor(max_workers=1)
        self._streams: list = []

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req: Request):
        self.waiting.append(req)

    def _prepare_async(self, req: Request):
        if self._prep_stream is None:
            return prepare(req, self.norm_iters, self.norm_rtol)
        with torch.cuda.device(self.device), torch.cuda.stream(self._prep_stream):
            return prepare(req, self.norm_iters, self.norm_rtol)

    def _admit(self):
        """Start preparing waiting requests, first come first served, while
        slots, memory and the work limit allow."""
        while self.waiting and len(self.active) + len(self.preparing) < self.max_slots:
            req = self.waiting[0]
            need = footprint_bytes(req.geometry, len(req.S), req.y.element_size())
            busy = self.active or self.preparing
            if self.used + need > self.budget and busy:
                break  # wait for memory to free up
            w = work_per_iter(req.geometry)
            if busy and self.work + w > self.sat_work:
                break  # the GPU is full: wait for a job to finish
            self.waiting.popleft()
            self.used += need
            self.work += w
            self.peak_used = max(self.peak_used, self.used)
            if self._pool is None:
                fut: Future = Future()
                fut.set_result(prepare(req, self.norm_iters, self.norm_rtol))
            else:
                fut = self._pool.submit(self._prepare_async, req)
            self.preparing.append((fut, req, need, w))

    def _stream(self):
        """A CUDA stream for a new resident job (reused once free)."""
        busy = {id(a.stream) for a in self.active if a.stream is not None}
        for s in self._streams:
            if id(s) not in busy:
                return s
        s = torch.cuda.Stream(device=self.device) if self.device is not None else None
        self._streams.append(s)
        return s

    def _launch(self, a: _Active):
        """Streams mode: enqueue the job's whole solve on its own stream."""
        a.stream = self._stream()
        ctx = torch.cuda.stream(a.stream) if a.stream is not None else _nullcontext()
        with ctx:
            for t in (a.y, a.x, getattr(a.plan, "_ws", None)):
                if isinstance(t, torch.Tensor) and t.is_cuda:
                    t.record_stream(a.stream)
            _, a.info = a.plan.solve(a.y, a.req.I0, a.eta, a.req.max_iters, x=a.x, lo=a.req.lo, hi=a.req.hi,
                                     tol=a.req.tol, check_every=a.req.check_every, sync=False)
            a.done = torch.cuda.Event() if a.stream is not None else None
            if a.done is not None:
                a.done.record(a.stream)
        self.launches += 1

    def _take_prepared(self, block: bool):
        """Move finished preparations into the resident set (waiting for the
        oldest one when `block` and nothing is resident); in streams mode
        launch their solves."""
        keep = deque()
        main = torch.cuda.current_stream(self.device) if self._prep_stream is not None else None
        for k, (fut, req, need, w) in enumerate(self.preparing):
            if block and k == 0 and not self.active:
                fut.result()
            if not fut.done():
                keep.append((fut, req, need, w))
                continue
            plan, y, x, eta = fut.result()
            a = _Active(req, plan, y, x, eta, need, 0, self.now(), w)
            if self.mode == "rounds" and main is not None:
                for t in (y, x, plan._ws):  # allocated on the preparation stream, now used on this one
                    t.record_stream(main)
            self.active.append(a)
            if self.mode == "streams":
                self._launch(a)
        self.preparing = keep
        self.peak_resident = max(self.peak_resident, len(self.active))

    def _retire(self, a: _Active, iters: int, rel_res: float, status: int) -> Result:
        res = Result(a.req.tag, a.x.cpu(), iters, rel_res, status, a.req.arrival, a.admitted, self.now())
        self._reaper.submit(a.plan.close)
        self.used -= a.footprint
        self.work -= a.work
        return res

    def _step_streams(self) -> list[Result]:
        done, keep = [], []
        for a in self.active:
            if a.done is None or a.done.query():
                if a.done is not None:
                    a.done.synchronize()  # the solve's info callback has run
                done.append(self._retire(a, a.info.iters_done, a.info.rel_res, a.info.status))
            else:
                keep.append(a)
        self.active = keep
        if not done:
            time.sleep(1e-4)  # nothing finished: poll again shortly
        return done

    def _step_rounds(self) -> list[Result]:
        jobs = []
        for a in self.active:
            k = min(self.round_iters, a.req.max_iters - a.iters)
            jobs.append(Job(plan=a.plan, y=a.y, I0=a.req.I0, eta=a.eta, iters=k, x=a.x, lo=a.req.lo, hi=a.req.hi,
                            tol=a.req.tol, check_every=a.req.check_every))
        if len(self.active) == 1:
            jb = jobs[0]
            _, info = jb.plan.solve(jb.y, jb.I0, jb.eta, jb.iters, x=jb.x, lo=jb.lo, hi=jb.hi, tol=jb.tol,
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
                done.append(self._retire(a, a.iters, info.rel_res, info.status))
            else:
                keep.append(a)
        self.active = keep
        return done

    def step(self) -> list[Result]:
        """Admit and activate what is ready, then (rounds) run one round over
        the resident jobs or (streams) collect the finished ones; retire."""
        self._admit()
        self._take_prepared(block=True)
        if not self.active:
            return []
        return self._step_rounds() if self.mode == "rounds" else self._step_streams()

    def run(self, requests: list[Request], realtime: bool = True) -> list[Result]:
        """Serve `requests` (sorted by arrival).  With realtime, a request is
        only visible once the server clock passes its arrival time."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        results = []
        self.t0 = time.perf_counter()
        while pending or self.waiting or self.preparing or self.active:
            now = self.now()
            while pending and (not realtime or pending[0].arrival <= now):
                self.submit(pending.popleft())
            if not self.waiting and not self.active and not self.preparing:
                time.sleep(max(0.0, min(0.01, pending[0].arrival - now)))
                continue
            results.extend(self.step())
        self._reaper.submit(lambda: None).result()  # every retired plan is freed
        return results

    def close(self):
        for fut, _, _, _ in self.preparing:
            plan, _, _, _ = fut.result()
            plan.close()
        self.preparing = deque()
        for a in self.active:
            if a.done is not None:
                a.done.synchronize()
            a.plan.close()
        self.active = []
        if self._pool is not None:
            self._pool.shutdown(wait=True)
        self._reaper.shutdown(wait=True)
        if self.batch is not None:
            self.batch.close()


class _nullcontext:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


def serve_sequential(requests: list[Request], realtime: bool = True, norm_iters: int = 60,
                     norm_rtol: float = 1e-5) -> list[Result]:
    """The plain baseline: first come, first served, each request prepared
    like the server prepares it and solved alone with exact_solve (the same
    tolerance test every check_every iterations, the iterations looping on the
    device until the stop)."""
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
        plan, y, x, eta = prepare(req, norm_iters, norm_rtol)
        x, info = plan.solve(y, req.I0, eta, req.max_iters, x=x, lo=req.lo, hi=req.hi, tol=req.tol,
                             check_every=req.check_every)
        out.append(Result(req.tag, x.cpu(), info.iters_done, info.rel_res, info.status, req.arrival, admitted,
                          time.perf_counter() - t0))
        plan.close()
    return out
