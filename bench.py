"""Throughput of the IBM time step on one GB300 (or N independent replicas).

Default workload: the tortuous airway-like duct, 512x384x256 cells (the largest
single-GPU configuration): a seeded union of tubes, inflow and convective
outflow in x, IBM weights built on the device, FP32 mode (see
inputs.configs.airway_c4).  A "step" is one full RK3 time step: three
substages, each a momentum predictor with the implicit IBM division followed
by the projection.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c4|c4s|c3|c3s|c3_fp64|c1|c2|c2_fp64|c2_periodic] [--impl reference]

One JSON line on stdout (rank 0).  `value` is cells x steps / time over all
ranks (replicas: every rank advances its own copy of the workload, no
collective on the data path).  The timed region is bracketed by a barrier and
a device synchronize; each rank's time is its CUDA-event duration on the
solver's stream, and the maximum over ranks is reported.
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

METRIC = "IBM-NS step Gcell-updates/s"
UNIT = "Gcell-updates/s"

# Algorithmic bytes per cell per launch of each kernel in FP32 mode (fields 4 B,
# pivots and the forward-sweep temporary FP64); the momentum figure is the
# average over the three RK3 stages (41, 53, 41 B) plus the mask byte and the
# IBM segment offsets.  IBM coefficient bytes are added per launch from the
# actual IBM-point counts.
ALG_BYTES_PER_CELL = {
    "momentum": (41.0 + 53.0 + 41.0) / 3.0 + 3 * 4.0 / 32.0,
    "flux_control": 9.0,
    "divergence": 16.0,
    "correct": 36.0,
}
# tridiag, per spectral point: one read of the right-hand side and of the pivot and one write of
# the solution (the forward sweep's temporary is not counted): FP32 storage 8 + 4 + 8 B for a
# system that sweeps in FP32 (FP32 pivot), 8 + 8 + 8 B for one that sweeps in FP64; FP64
# storage 16 + 8 + 16 B
TRIDIAG_BYTES_PER_SPECTRAL_POINT = {"fp32": 20.0, "fp32_fp64sweep": 24.0, "fp64": 40.0}

PRECISION_DETAIL = {
    "fp32": ("fp32 fields, momentum stencil, IBM division, per-cell divergence and FFTs; fp64 tridiagonal "
             "sweeps of the near-singular spectral systems (K dy^2 < 1) and fp64 Thomas pivots of every system; "
             "fp32 sweeps of the strongly dominant systems (K dy^2 >= 1, condition <= 5); fp64 sums in every "
             "reduction (flow rate, outflow balance, diagnostics); IBM weights computed in fp64"),
    "fp64": "fp64 throughout",
}

# DRAM traffic per launch measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum),
# keyed by kernel, with the hash of the source file it was taken on; a changed
# source makes the figure stale and it is reported as null.
NCU_TRAFFIC = {
    # (kernel, workload): (DRAM bytes per launch, mean of the three RK3 stages of one step, and
    # the sha256[:16] of the kernel's source file the capture ran on)
    # the momentum interval: k_momentum_tma and k_ibm_division, summed per stage
    # profiles/c3_wavy_384x256x256_momentum_tma_ncu.md
    ("momentum", "c3"): ((1060.3e6 + 1360.8e6 + 1079.7e6) / 3.0, "4c54badae3509d9c"),
    # profiles/c4_airway_512x384x256_momentum_tma_traffic.md
    ("momentum", "c4"): ((2186.2e6 + 2790.4e6 + 2203.9e6) / 3.0, "4c54badae3509d9c"),
}

KERNEL_FILE = {"momentum": "momentum.cu"}   # other kernels of this library live in step.cu


def src_hash(name="step.cu") -> str:
    p = os.path.join(ROOT, "paper_2506_14328_gb300", "csrc", name)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d.get("hbm_gbs", 6800.0)), "source": "measured (MEASURED_PEAKS.json)"}
    return {"hbm_gbs": 6800.0, "source": "fallback 6.8 TB/s"}


def workload(name: str):
    from inputs import wavy_c3, channel_c1, cylinder_c2, cylinder_c2_io, airway_c4
    if name == "c3":
        return wavy_c3(precision="fp32")
    if name == "c3_fp64":
        return wavy_c3(precision="fp64")
    if name == "c3s":   # profiling size: 6.3M cells, working set well above L2
        return wavy_c3(precision="fp32", n=(384, 256, 64))
    if name == "c1":
        return channel_c1(precision="fp64")
    if name == "c2":         # uniform inflow, convective outflow, free-slip lateral walls
        return cylinder_c2_io(re=100.0, precision="fp32")
    if name == "c2_fp64":
        return cylinder_c2_io(re=100.0, precision="fp64")
    if name == "c2_periodic":  # the periodic-x stand-in with a constant flow rate
        return cylinder_c2(re=100.0, precision="fp32")
    if name == "c4":         # tube-union airway, inflow / convective outflow, weights built on the device
        return airway_c4(precision="fp32")
    if name == "c4s":        # profiling size: the airway layout on 512x384x64 (dz = 4 dx), 12.6M cells
        return airway_c4(precision="fp32", n=(512, 384, 64))
    raise SystemExit(f"unknown workload {name}")


def tridiag_alg_bytes(case) -> float:
    """Algorithmic bytes of one tridiagonal launch: every spectral point once in and once out with
    its pivot.  In FP32 mode the near-singular systems (K dy^2 < 1) sweep in FP64 with FP64
    pivots, the others in FP32 with FP32 pivots (the same split the library makes)."""
    import numpy as np
    nx, ny, nz = case.n
    xper = case.bc_lo[0] == 0
    nxh = nx // 2 + 1 if xper else nx
    dx, dy = case.L[0] / nx, case.L[1] / ny
    kx = np.arange(nxh)
    sx = np.sin(np.pi * kx / nx) if xper else np.sin(np.pi * kx / (2.0 * nx))
    K = (4.0 * sx ** 2 / dx ** 2)[None, :]
    if case.ndim == 3 and nz > 1:
        dz = case.L[2] / nz
        nzs = nz if xper else nz // 2 + 1     # a real transform in z on a Neumann x
        K = K + (4.0 * np.sin(np.pi * np.arange(nzs) / nz) ** 2 / dz ** 2)[:, None]
    nsys = K.size
    if case.precision == "fp64":
        return TRIDIAG_BYTES_PER_SPECTRAL_POINT["fp64"] * nsys * ny
    n64 = int(np.count_nonzero(K * dy * dy < 1.0))
    return ny * (TRIDIAG_BYTES_PER_SPECTRAL_POINT["fp32_fp64sweep"] * n64 +
                 TRIDIAG_BYTES_PER_SPECTRAL_POINT["fp32"] * (nsys - n64))


def reduce_max(x: float, dist=None, device="cpu") -> float:
    """Maximum of x over the ranks of the process group (x itself without one)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(cells: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job Gcell-updates/s: every rank advances its own replica of `cells` cells."""
    return world * cells * steps / seconds / 1e9


def serving_sample(device, n_requests: int = 16, seed: int = 0, load: float = 0.8,
                   capacity: float = 3.0e9) -> dict:
    """A bounded sample of the serving mix (C5) at its stated distributions (2D n^2 with n in
    [128, 1024], 3D n^3 with n in [64, 192], 500-5000 steps), with Poisson arrivals at `load`
    of an assumed aggregate capacity of `capacity` cell-updates/s."""
    from inputs import serving_mix, initial_field
    from paper_2506_14328_gb300.serving import Server, Request
    probe = serving_mix(seed=seed, n_requests=n_requests, rate_hz=1.0)
    work = sum(c.ncells * s for _, c, s in probe) / len(probe)
    rate = load * capacity / work
    mix = serving_mix(seed=seed, n_requests=n_requests, rate_hz=rate)
    # each client sends its initial state with the request (prepared before arrival)
    reqs = [Request(q, t, c, s, init=initial_field(c)) for q, (t, c, s) in enumerate(mix)]
    # default tiles (no autotuning inside the timed run: a deployed server has its tile choices
    # cached per grid shape); small solves share the persistent momentum launches
    srv = Server(device=str(device), max_resident=32, steps_per_tick=25, autotune=False)
    stats = srv.serve(reqs)
    srv.close()
    # capacity: the same requests all arriving at once (the server saturated)
    sat = [Request(q, 0.0, c, s, init=r.init) for q, ((t, c, s), r) in enumerate(zip(mix, reqs))]
    srv = Server(device=str(device), max_resident=32, steps_per_tick=25, autotune=False)
    st2 = srv.serve(sat)
    srv.close()
    stats["saturated"] = {"gcell_updates_per_s": st2["gcell_updates_per_s"], "wall_s": st2["wall_s"],
                          "p50_s": st2["p50_s"], "p99_s": st2["p99_s"],
                          "what": "the same requests, all arriving at t = 0"}
    stats.update({"arrival_rate_hz": rate, "assumed_capacity_gcell_s": capacity / 1e9,
                  "mix": "C5 at its stated distributions: 2D n^2 n in [128,1024], 3D n^3 n in [64,192], "
                         "steps 500-5000, Re 10-2000, FP32 mode, Poisson arrivals", "seed": seed})
    return stats


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle arm
def oracle_slab(case, nz: int):
    """The same workload on a slab of nz cells in z (same spacing, physics and flux per area)."""
    if case.ndim != 3:
        return case.with_(precision="fp64")
    from inputs import GEOM_TUBES
    if case.geom_kind == GEOM_TUBES:
        nz = min(nz, 4)      # the tube level set costs every segment at every point: a thinner slab
    n = (case.n[0], case.n[1], min(nz, case.n[2]))
    frac = n[2] / case.n[2]
    # a slab through the middle of the box in z, where a body or a duct has fluid
    k0 = (case.n[2] - n[2]) // 2 if case.geom_kind == GEOM_TUBES else 0
    origin = (case.origin[0], case.origin[1], case.origin[2] + k0 * case.L[2] / case.n[2])
    return case.with_(n=n, L=(case.L[0], case.L[1], case.L[2] * frac), origin=origin, precision="fp64",
                      target_flux=case.target_flux * frac)


def _oracle_run(args):
    """One oracle process: `steps` full steps on the slab; returns (cells x steps, seconds)."""
    case, steps, nz = args
    from oracle import OracleSolver
    from inputs import initial_field
    sample = oracle_slab(case, nz)
    o = OracleSolver(sample)
    f = initial_field(sample)
    o.set_state(f["u"], f["v"], f["w"], f["p"])
    t = time.perf_counter()
    o.step(steps)
    return sample.ncells * steps, time.perf_counter() - t, sample.n


def oracle_sample(case, steps: int = 2, nz: int = 32, procs: int = 1):
    """Time the FP64 oracle, as it stands, on a bounded slab of the same workload: one process
    (procs = 1), or `procs` independent processes at once, each stepping its own copy of the
    slab (the host's cores used as replicas; throughput = all their cell updates / wall time)."""
    if procs <= 1:
        work, dt, n = _oracle_run((case, steps, nz))
        desc = (f"{steps} full steps of the FP64 numpy oracle on a {n[0]}x{n[1]}x{n[2]} slab of the "
                f"same workload (same spacing and physics), one process, {dt:.1f} s")
        return {"value": work / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}
    import multiprocessing as mp
    # numpy's own threads off in the workers, so that each process holds one core
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    ctx = mp.get_context("spawn")        # never fork a process that has used the GPU
    with ctx.Pool(procs) as pool:
        pool.map(_ping, range(procs))   # the workers are up (imports done) before the clock starts
        t = time.perf_counter()
        res = pool.map(_oracle_run, [(case, steps, nz)] * procs)
        wall = time.perf_counter() - t
    work = sum(r[0] for r in res)
    n = res[0][2]
    desc = (f"{procs} oracle processes at once (spawned, one per host core), each {steps} full FP64 steps on "
            f"its own {n[0]}x{n[1]}x{n[2]} slab of the same workload, {wall:.1f} s wall")
    return {"value": work / wall / 1e9, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": desc}


def _ping(_):
    import oracle  # noqa: F401
    return os.getpid()


def run_reference(args):
    """The oracle on the host cores: W untimed then K timed full steps on a slab of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import OracleSolver
    from inputs import initial_field
    case = workload(args.workload)
    sample = oracle_slab(case, nz=8)
    o = OracleSolver(sample)
    f = initial_field(sample)
    o.set_state(f["u"], f["v"], f["w"], f["p"])
    o.step(args.warmup)
    t = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t
    v = sample.ncells * args.steps / dt / 1e9
    n = sample.n
    desc = (f"{args.steps} timed full steps (after {args.warmup} untimed) of the FP64 numpy oracle on a "
            f"{n[0]}x{n[1]}x{n[2]} slab of the workload, {dt:.1f} s")
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / max(args.steps, 1) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": case.name, "cells": case.ncells, "sample_cells": sample.ncells,
                       "parallelism": "none"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import numpy as np
    import torch
    from inputs import initial_field
    from inputs.configs import describe

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)

    from paper_2506_14328_gb300.solver import Solver
    case = workload(args.workload)
    torch.cuda.synchronize(device)
    t_setup = time.perf_counter()
    s = Solver.from_case(case, device=str(device))     # classification, lists, weights, plans
    if args.projection == "masked":
        s.set_projection("masked", tol=1e-6, maxit=200)
    s.sync()
    setup_s = time.perf_counter() - t_setup
    f = initial_field(case)
    s.set_state(f["u"], f["v"], f["w"], f["p"])
    s.project()
    s.step(args.warmup)
    s.sync()

    def barrier():
        torch.cuda.synchronize(device)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(device)

    # ---- device-timed region -------------------------------------------------
    clocks = ClockSampler(local)
    clocks.start()
    s.timing(True)
    barrier()
    launches0 = s.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(s.stream)
    s.step(args.steps)
    ev1.record(s.stream)
    barrier()
    launches = s.launch_count() - launches0
    ms = ev0.elapsed_time(ev1)
    kt = s.get_timing()
    s.timing(False)
    clk = clocks.stop()
    diag = s.diagnostics()
    ms_max = reduce_max(ms, dist, device)
    value = aggregate_rate(case.ncells, args.steps, world, ms_max * 1e-3)

    # ---- end to end through the public API with host buffers -----------------
    # Two solvers take turns, as a server keeps two requests in flight: every step imports its
    # input state (u, v, w, p) from pinned host memory, steps once, and exports the stepped
    # state (u, v, w, p) back into pinned host memory.  While one solver steps, the other's
    # copies run.  Every step's H2D copy and D2H copy of the whole field lie inside the timed
    # region.
    nbytes = s.state_bytes()
    host_in = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    host_out = [torch.empty(nbytes, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
    s.export_state(host_in.numpy())
    s2 = Solver.from_case(case, device=str(device))
    if args.projection == "masked":
        s2.set_projection("masked", tol=1e-6, maxit=200)
    pair = (s, s2)
    for q, out in zip(pair, host_out):                # untimed: one step through each
        q.import_state_ptr(host_in.data_ptr(), nbytes)
        q.step(1)
        q.export_state(out.numpy())
    e2e_steps = max(2, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    for n in range(e2e_steps):
        cur = pair[n % 2]
        cur.import_state_ptr(host_in.data_ptr(), nbytes)     # H2D of step n's input state
        cur.step(1)
        if n > 0:
            pair[(n - 1) % 2].export_state(host_out[(n - 1) % 2].numpy())   # D2H of step n-1's state
    pair[(e2e_steps - 1) % 2].export_state(host_out[(e2e_steps - 1) % 2].numpy())
    barrier()
    e2e_s = time.perf_counter() - t0
    diag2 = s2.diagnostics()
    s2.close()
    e2e_value = aggregate_rate(case.ncells, e2e_steps, world, reduce_max(e2e_s, dist, device))

    if rank == 0:
        peaks = measured_peaks()
        mask, counts = s.classification()
        nibm = sum(len(c) for c in counts)
        ncomp = 3 if case.ndim == 3 else 2
        ninternal = sum(int(np.count_nonzero(mask & (1 << c))) for c in range(ncomp))
        per_kernel = {}
        for name, (n, tot) in kt.items():
            per_kernel[name] = {"launches": n, "ms_total": tot, "share": tot / ms if ms > 0 else None}
            if name == "ibm_division":   # timed inside the momentum interval
                per_kernel[name]["within"] = "momentum"
        # roofline of the dominant kernel of this library
        mine = {k: v for k, v in kt.items() if not k.startswith("fft")}   # cuFFT is library code
        dom = max(mine, key=lambda k: mine[k][1]) if mine else "momentum"
        n_l, tot_ms = mine.get(dom, (1, float("nan")))
        avg_s = tot_ms / n_l * 1e-3
        if dom == "tridiag":
            alg = tridiag_alg_bytes(case)
        else:
            alg = ALG_BYTES_PER_CELL.get(dom, 0.0) * case.ncells
            if dom == "momentum":
                alg += nibm * 16.0
        achieved = alg / avg_s / 1e9 if avg_s > 0 else None
        traffic = None
        rec = NCU_TRAFFIC.get((dom, args.workload))
        if rec and rec[1] == src_hash(KERNEL_FILE.get(dom, "step.cu")):
            traffic = rec[0]
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"] if achieved else None, "traffic": traffic, "kernel": dom,
                "alg_bytes_per_launch": alg, "avg_launch_ms": avg_s * 1e3,
                "launches_timed": ("k_momentum_tma and the IBM division after it (k_ibm_division), one interval"
                                   if dom == "momentum" else dom),
                "peak_source": peaks["source"] + ", copy bandwidth; kernel timed inside a long step"}
        cpu = None
        if world == 1:
            ncores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
            cpu = oracle_sample(case, procs=ncores)
            cpu["single_core"] = oracle_sample(case, procs=1)
            cpu["nproc"] = os.cpu_count()
        cfg = describe(case)
        cfg.update({"model": "IBM RK3 step + projection", "parallelism": "replicas" if world > 1 else "single",
                    "l2": "inputs larger than L2 (working set ~%.1f GB)" % (
                        (s.work.numel() + 4 * s.N * (4 if case.precision == 'fp32' else 8)) / 1e9),
                    "precision_detail": PRECISION_DETAIL[case.precision],
                    "ibm_points": nibm, "ibm_fraction_of_fluid_points": nibm / max(ninternal, 1),
                    "projection": args.projection,
                    "setup_s": setup_s, "final_div_linf": diag["div_linf"], "final_flux_u": diag["flux"][0]})
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if case.precision == "fp32" else "f64", "data": "synthetic", "config": cfg,
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                        "d2h_bytes_per_step": nbytes, "steps": e2e_steps,
                        "what": "two solvers in turn; per step: import u,v,w,p from pinned host memory, one "
                                "full step, export u,v,w,p to pinned host memory",
                        "final_div_linf": diag2["div_linf"]},
                "clocks": clk, "gpu_launches": launches, "kernels": per_kernel}
        if args.serving > 0:
            line["serving"] = serving_sample(device, n_requests=args.serving)
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="c4")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--serving", type=int, default=16, help="requests in the serving sample (0: skip)")
    ap.add_argument("--projection", default="fullbox", choices=["fullbox", "masked"],
                    help="masked: D M G over the internal cells by conjugate gradients (residual 1e-6)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
