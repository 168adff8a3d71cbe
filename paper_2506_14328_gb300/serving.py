"""Continuous-batching service for many IBM solves on one GPU.

Requests (a grid, a geometry, physics and a step count) arrive over time.
The server:
  * admits a request as soon as it has arrived, a slot is free and its
    device footprint (fields + workspace + weights) fits the HBM budget;
  * keeps every admitted solve's fields, pressure and weights resident on
    the device until it completes;
  * advances all resident solves together: one CUDA graph per tick forks
    onto each solve's own stream, runs min(steps_per_tick, remaining) full
    steps of every member, and joins (ibm_batch_set / ibm_batch_run), so
    solves of different sizes overlap on the device; the graph is
    re-captured only when the resident set or a step count changes;
  * advances the momentum predictors of the small solves (at most job_cells
    cells) in one persistent launch per substage that walks a work list of
    all their tiles (ibm_batch_jobs);
  * keeps two ticks in flight: the next tick is enqueued before the host
    waits for the previous one, and the solves that tick finished are read
    back while the next one runs;
  * sets up newly admitted solves on a host thread of their own (each on its
    own stream), so admission never stalls the tick loop;
  * records each request's latency (arrival to completion) and reports
    p50/p99 together with the aggregate cell-update throughput.
All numerical work is in libibm.so; this module only schedules.
"""
from __future__ import annotations

import json
import os
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import ibm_batch_create, ibm_batch_set, ibm_batch_run, ibm_batch_jobs, ibm_batch_destroy
from .solver import Solver

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune_cache.json")


class TuneCache:
    """z-chunk choices of the autotuner per grid shape and precision (a JSON file)."""

    def __init__(self, path: str = _CACHE):
        self.path = path
        self.lock = threading.Lock()      # solves are set up on several host threads
        try:
            self.table = json.load(open(path))
        except (OSError, ValueError):
            self.table = {}

    @staticmethod
    def key(n, precision) -> str:
        return f"{n[0]}x{n[1]}x{n[2]}:{precision}"

    def apply(self, solver: Solver, n, precision, tune: bool = True):
        k = self.key(n, precision)
        with self.lock:
            known = self.table.get(k)
        if known is not None:
            solver.set_tiles(*known)
        elif tune:
            choice = list(solver.autotune())
            with self.lock:
                self.table[k] = choice
                try:
                    with open(self.path, "w") as f:
                        json.dump(self.table, f, indent=1, sort_keys=True)
                except OSError:
                    pass


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of serve()
    case: object            # anything with the attributes Solver.from_case reads
    steps: int
    init: dict | None = None   # host arrays u, v, w, p sent with the request (else init_field(case))
    result: dict = field(default_factory=dict)


@dataclass
class _Resident:
    req: Request
    solver: Solver
    remaining: int
    bytes: int


def _percentile(a, q):
    return float(np.percentile(np.asarray(a), q)) if len(a) else None


class Server:
    def __init__(self, device="cuda", hbm_budget_bytes: int | None = None, max_resident: int = 64,
                 steps_per_tick: int = 25, autotune: bool = True, keep_state: bool = False,
                 init_field=None, autotune_min_cells: int = 1 << 21, job_cells: int = 1 << 18):
        self.device = torch.device(device)
        if self.device.index is None:                   # "cuda": the current device, by number
            self.device = torch.device("cuda", torch.cuda.current_device())
        free, total = torch.cuda.mem_get_info(self.device)
        self.budget = int(hbm_budget_bytes) if hbm_budget_bytes else int(0.8 * free)
        self.max_resident = max_resident
        self.steps_per_tick = steps_per_tick
        self.autotune = autotune
        self.keep_state = keep_state
        self.init_field = init_field      # callable(case) -> dict(u, v, w, p) of host arrays
        self.autotune_min_cells = autotune_min_cells
        self.stream = torch.cuda.Stream(self.device)
        self.batch = ibm_batch_create(self.stream.cuda_stream)
        # solves of at most job_cells cells advance their momentum predictors together, in one
        # persistent launch per substage (0: every solve steps on its own stream)
        self.job_cells = int(job_cells)
        ibm_batch_jobs(self.batch, self.job_cells)
        self.tunes = TuneCache()

    def close(self):
        if getattr(self, "batch", None):
            ibm_batch_destroy(self.batch)
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------------
    def _admit(self, req: Request) -> _Resident:
        s = Solver.from_case(req.case, device=str(self.device))
        f = req.init if req.init is not None else (self.init_field(req.case) if self.init_field else None)
        if f is not None:
            s.set_state(f["u"], f["v"], f["w"], f["p"])
            s.project()
        # tiling is tuned for large 3D grids; small ones keep the defaults
        big = req.case.ndim == 3 and s.N >= self.autotune_min_cells
        self.tunes.apply(s, req.case.n, req.case.precision, tune=self.autotune and big)
        s.sync()
        return _Resident(req, s, req.steps, s.footprint_bytes())

    def _finish(self, r: _Resident, t0: float):
        d = r.solver.diagnostics()
        res = {"latency_s": time.perf_counter() - t0 - r.req.arrival, "diag": d,
               "cells": r.solver.N, "steps": r.req.steps}
        if self.keep_state:
            u, p = r.solver.state()
            res["state"] = (u, p)
        r.req.result = res
        r.solver.close()

    def serve(self, requests: list) -> dict:
        """Serve requests (sorted by arrival); returns latency and throughput statistics.

        Ticks overlap with host work: tick n+1 is enqueued before the host waits for tick n
        (an event on the batch stream), the members that tick n finished are read back while
        tick n+1 runs, and new solves are set up on a separate host thread (each on its own
        stream) and join the resident set at the next tick boundary."""
        pending = sorted(requests, key=lambda q: q.arrival)
        resident: list[_Resident] = []
        done: list[Request] = []
        used = 0
        cur = None
        ticks = 0
        recaptures = 0
        busy_cells = 0
        ready: "queue.Queue" = queue.Queue()
        reserved = [0]              # bytes of admitted solves still being set up
        inflight = []               # (event, finished residents) of ticks not yet retired
        errors = []
        t0 = time.perf_counter()

        def setup(req):
            try:
                torch.cuda.set_device(self.device)
                ready.put((req.rid, self._admit(req)))
            except Exception as e:      # reported by the main loop
                errors.append(e)
                ready.put((req.rid, None))

        workers = {}                # rid -> (thread, estimated bytes) of solves being set up
        while pending or resident or inflight or workers:
            # admissions: requests that have arrived and fit go to the set-up thread
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now and len(resident) + len(workers) < self.max_resident:
                est = _estimate_bytes(pending[0].case)
                if used + reserved[0] + est > self.budget and (resident or workers):
                    break
                req = pending.pop(0)
                reserved[0] += est
                th = threading.Thread(target=setup, args=(req,), daemon=True)
                th.start()
                workers[req.rid] = (th, est)
            # solves whose set-up finished join at this tick boundary
            while True:
                try:
                    rid, r = ready.get_nowait()
                except queue.Empty:
                    break
                th, est = workers.pop(rid)
                th.join()
                reserved[0] -= est
                if r is None:
                    raise errors[0]
                used += r.bytes
                resident.append(r)
            # one tick of every resident solve, enqueued before waiting for the previous one
            if resident:
                steps = [min(self.steps_per_tick, r.remaining) for r in resident]
                key = ([id(r) for r in resident], steps)
                if key != cur:
                    ibm_batch_set(self.batch, [r.solver.h for r in resident], steps)
                    cur = key
                    recaptures += 1
                ibm_batch_run(self.batch)
                ev = torch.cuda.Event()
                ev.record(self.stream)
                ticks += 1
                finished = []
                for r, st in zip(resident, steps):
                    r.remaining -= st
                    busy_cells += r.solver.N * st
                    if r.remaining <= 0:
                        finished.append(r)
                if finished:
                    resident = [r for r in resident if r.remaining > 0]
                    cur = None
                inflight.append((ev, finished))
            # retire the oldest tick once a newer one is queued (or nothing else is left)
            while inflight and (len(inflight) > 1 or not resident):
                ev, finished = inflight.pop(0)
                ev.synchronize()
                for r in finished:
                    self._finish(r, t0)
                    used -= r.bytes
                    done.append(r.req)
            if not resident and not inflight:
                if workers:
                    time.sleep(0.0005)
                elif pending:
                    wait = pending[0].arrival - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
        wall = time.perf_counter() - t0
        lat = [q.result["latency_s"] for q in done]
        return {"requests": len(done), "wall_s": wall, "p50_s": _percentile(lat, 50),
                "p99_s": _percentile(lat, 99), "mean_s": float(np.mean(lat)) if lat else None,
                "gcell_updates_per_s": busy_cells / wall / 1e9, "ticks": ticks, "recaptures": recaptures}


def _estimate_bytes(case) -> int:
    """Admission estimate of a solve's device footprint: four fields, the
    workspace (about 13 fields' worth) and a weights allowance."""
    n = case.n[0] * case.n[1] * case.n[2]
    esz = 8 if case.precision == "fp64" else 4
    return int(n * esz * 4 + n * (esz * 10 + 32) + 0.1 * n * esz * 12)
