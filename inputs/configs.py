"""Workload descriptions: the synthetic stand-ins for the paper's cases.

Each `Case` is plain data: grid, box boundary kinds, geometry kind and
parameters, physical constants, time step and step count.  The integer codes
below are the ones the C-ABI header declares (ibm_bc, ibm_geom_kind,
ibm_bmode, ibm_flow_mode); they are data-format constants, not arithmetic.

Cases (the paper's own runs need data that is not available, so these stand in):
  * channel_c1  - 2D laminar plane channel, 64x32, walls off-grid at
                  y=0.137 and y=0.861 imposed by the IBM (Sec. 2.2 / Eq. 3-6 style
                  steady Laplacian test generalised to Navier-Stokes).
  * cylinder_c2 - 2D cylinder, D=1, seeded sub-cell centre offset (Sec. 4.1 shape).
  * wavy_c3     - 3D channel over a sinusoidal lower wall, 384x256x256,
                  constant flow rate, Re_b=5600 (Sec. 4.2 shape).
  * small_case  - the same physics at sizes the oracle finishes in seconds,
                  with ragged tails against 32-wide warps.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
import math
import numpy as np

BC_PERIODIC, BC_NOSLIP, BC_FREESLIP, BC_INFLOW, BC_OUTFLOW = 0, 1, 2, 3, 4
GEOM_NONE, GEOM_PLANES, GEOM_CYLINDER, GEOM_SPHERE, GEOM_SINE_WALL, GEOM_TUBES, GEOM_SAMPLED = range(7)
B_EXACT, B_EULER, B_TAYLOR2, B_EXPLICIT = 0, 1, 2, 3
FLOW_FORCED, FLOW_CONST_FLUX = 0, 1


@dataclass
class Case:
    name: str
    ndim: int
    n: tuple            # (nx, ny, nz); nz == 1 in 2D
    L: tuple            # box lengths
    origin: tuple       # box lower corner
    bc_lo: tuple        # per direction, BC_* codes
    bc_hi: tuple
    geom_kind: int
    geom_params: tuple  # kind-specific, see include/ibm.h
    nu: float
    dt: float
    g: tuple = (0.0, 0.0, 0.0)
    bmode: int = B_EXACT
    flow_mode: int = FLOW_FORCED
    target_flux: float = 0.0   # volume integral of u over the fluid (FLOW_CONST_FLUX)
    wall_u: tuple = (0.0, 0.0, 0.0)
    inflow: tuple = (0.0, 0.0, 0.0)   # velocity entering through the -x face (x inflow / outflow boxes)
    projection: str = "fullbox"       # "fullbox" (the unmodified projection) or "masked" (internal faces only)
    g_amp: tuple = (0.0, 0.0, 0.0)    # time-periodic forcing g + g_amp sin(2 pi g_freq t)
    g_freq: float = 0.0
    y_faces: tuple = ()        # stretched wall-normal grid: the ny + 1 face heights (empty: uniform)
    body_velocity: tuple = ()  # a translating cylinder or sphere: its velocity (empty: at rest)
    body_omega: float = 0.0    # a cylinder rotating about its own axis: the rate
    precision: str = "fp64"    # "fp64" or "fp32" (FP32 momentum, FP64 tridiagonal/reductions)
    steps: int = 1
    init: dict = field(default_factory=lambda: {"kind": "zero"})
    seed: int = 0

    @property
    def ncells(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    def with_(self, **kw) -> "Case":
        return replace(self, **kw)


def channel_c1(precision: str = "fp64", steps: int = 2000) -> Case:
    """2D plane channel: 64x32 on [0,2]x[0,1], periodic x, IBM walls at y=0.137/0.861.

    Re = 10 on the centreline velocity U_c = 1 and the half height h = 0.362,
    so nu = 0.0362; the body force g_x = 2 nu / h^2 makes the exact profile
    u = 1 - ((y - y_c)/h)^2 with y_c = 0.499.
    """
    h = 0.362
    nu = 1.0 * h / 10.0
    return Case(name="c1_channel_64x32", ndim=2, n=(64, 32, 1), L=(2.0, 1.0, 1.0),
                origin=(0.0, 0.0, 0.0), bc_lo=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC),
                bc_hi=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC), geom_kind=GEOM_PLANES,
                geom_params=(0.137, 0.861), nu=nu, dt=0.008, g=(2.0 * nu / h ** 2, 0.0, 0.0),
                precision=precision, steps=steps, init={"kind": "zero"})


def tanh_faces(ny: int, y0: float, L: float, beta: float) -> tuple:
    """ny + 1 face heights on [y0, y0 + L] clustered toward both ends by a tanh map of
    strength beta (the usual wall-normal stretching of channel simulations)."""
    eta = np.arange(ny + 1) / ny
    y = y0 + 0.5 * L * (1.0 + np.tanh(beta * (2.0 * eta - 1.0)) / np.tanh(beta))
    y[0], y[-1] = y0, y0 + L
    return tuple(float(v) for v in y)


def couette_case(nx: int = 16, ny: int = 24, a: float = 0.113, b: float = 0.871,
                 U: float = 1.0, nu: float = 0.05) -> Case:
    """Plane Couette flow between an IBM wall at rest (y=a) and one moving at U (y=b)."""
    return Case(name=f"couette_{nx}x{ny}", ndim=2, n=(nx, ny, 1), L=(1.0, 1.0, 1.0),
                origin=(0.0, 0.0, 0.0), bc_lo=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC),
                bc_hi=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC), geom_kind=GEOM_PLANES,
                geom_params=(a, b), nu=nu, dt=0.2 * (1.0 / ny) ** 2 / nu,
                wall_u=(U, 0.0, 0.0), init={"kind": "couette", "a": a, "b": b, "U": U})


def cylinder_c2_io(re: float = 40.0, precision: str = "fp64", steps: int = 10, seed: int = 0,
                   n=(1536, 768)) -> Case:
    """2D cylinder D=1 at a seeded sub-cell offset from (0, 0) in the box
    x in [-10, 20], y in [-7.5, 7.5]: uniform inflow U = 1 at x = -10, convective
    outflow at x = 20, free-slip lateral walls; Re = U D / nu."""
    from .generators import cell_offset
    nx, ny = n
    Lx, Ly = 30.0, 15.0
    dx = Lx / nx
    ox, oy = cell_offset(seed, dx)
    return Case(name=f"c2_cylinder_io_{nx}x{ny}_re{int(re)}", ndim=2, n=(nx, ny, 1), L=(Lx, Ly, 1.0),
                origin=(-10.0, -7.5, 0.0), bc_lo=(BC_INFLOW, BC_FREESLIP, BC_PERIODIC),
                bc_hi=(BC_OUTFLOW, BC_FREESLIP, BC_PERIODIC), geom_kind=GEOM_CYLINDER,
                geom_params=(ox, oy, 0.5, -1.0), nu=1.0 / re, dt=0.004 if re <= 40 else 0.008,
                inflow=(1.0, 0.0, 0.0), precision=precision, steps=steps, init={"kind": "uniform", "U": 1.0},
                seed=seed)


def cylinder_paper(re: float = 30.0, precision: str = "fp32", h: float = 0.02, steps: int = 0) -> Case:
    """The cylinder flow of the paper's first example (Sec. 4.1): D = 1 at the origin, domain
    x in [-9, 40], y in [-17, 17], here on a uniform grid of step h (the paper's step near the
    body).  Uniform inflow U = 1, convective outflow; the lateral faces are free-slip walls
    (not stated in the paper).  dt is 80% of the explicit viscous limit of RK3 (2.51 / (8 nu / h^2))
    or 0.4 h / U, whichever is smaller."""
    nx, ny = int(round(49.0 / h)), int(round(34.0 / h))
    nu = 1.0 / re
    dt = min(0.8 * 2.51 / (8.0 * nu / (h * h)), 0.4 * h)
    return Case(name=f"cylinder_paper_re{int(re)}_{nx}x{ny}", ndim=2, n=(nx, ny, 1), L=(49.0, 34.0, 1.0),
                origin=(-9.0, -17.0, 0.0), bc_lo=(BC_INFLOW, BC_FREESLIP, BC_PERIODIC),
                bc_hi=(BC_OUTFLOW, BC_FREESLIP, BC_PERIODIC), geom_kind=GEOM_CYLINDER,
                geom_params=(0.0, 0.0, 0.5, -1.0), nu=nu, dt=dt, inflow=(1.0, 0.0, 0.0),
                precision=precision, steps=steps, init={"kind": "uniform", "U": 1.0})


def cylinder_c2(re: float = 40.0, precision: str = "fp64", steps: int = 10, seed: int = 0,
                n=(1536, 768)) -> Case:
    """2D cylinder D=1 in a 30D x 15D box; centre offset by a seeded fraction of a cell.

    Stand-in reading: x is periodic (the box is long enough for the wake to
    decay) and the lateral faces are free-slip walls; the stream is driven at
    a constant flow rate U = 1 by a uniform forcing adjusted every substage.
    This keeps the Poisson operator separable with the tridiagonal direction
    along y.  Uniform inflow with convective outflow is not built.
    """
    from .generators import cell_offset
    nx, ny = n
    Lx, Ly = 30.0, 15.0
    dx = Lx / nx
    ox, oy = cell_offset(seed, dx)
    return Case(name=f"c2_cylinder_{nx}x{ny}_re{int(re)}", ndim=2, n=(nx, ny, 1), L=(Lx, Ly, 1.0),
                origin=(-10.0, -7.5, 0.0), bc_lo=(BC_PERIODIC, BC_FREESLIP, BC_PERIODIC),
                bc_hi=(BC_PERIODIC, BC_FREESLIP, BC_PERIODIC), geom_kind=GEOM_CYLINDER,
                geom_params=(ox, oy, 0.5, -1.0), nu=1.0 / re, dt=0.004 if re <= 40 else 0.008,
                flow_mode=FLOW_CONST_FLUX, target_flux=1.0 * (Lx * Ly - math.pi * 0.25),
                precision=precision, steps=steps, init={"kind": "uniform", "U": 1.0}, seed=seed)


def wavy_c3(precision: str = "fp32", steps: int = 10, n=(384, 256, 256), seed: int = 0) -> Case:
    """3D channel over y_w(x) = 0.1 sin(2 pi x) (A = 0.1h, lambda = h, h = 1).

    Box x in [0,4], y in [-0.125, 1.875], z in [0,2]; periodic x and z; the top
    box face y = 1.875 is an on-grid no-slip wall.  Constant flow rate with
    bulk velocity U_b = 1 and Re_b = U_b 2h / nu = 5600.
    """
    nx, ny, nz = n
    nu = 2.0 / 5600.0
    ylo, ytop = 0.0, 1.875
    # target volume flux: U_b times the mean fluid cross-section times the box length
    target = 1.0 * (ytop - ylo) * 4.0 * 2.0
    return Case(name=f"c3_wavy_{nx}x{ny}x{nz}", ndim=3, n=(nx, ny, nz), L=(4.0, 2.0, 2.0),
                origin=(0.0, -0.125, 0.0), bc_lo=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC),
                bc_hi=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC), geom_kind=GEOM_SINE_WALL,
                geom_params=(0.0, 0.1, 1.0, 1.0e30), nu=nu, dt=0.002,
                flow_mode=FLOW_CONST_FLUX, target_flux=target, precision=precision, steps=steps,
                init={"kind": "channel_noise", "ylo": ylo, "yhi": ytop, "Ub": 1.0, "noise": 0.05},
                seed=seed)


def airway_c4(precision: str = "fp32", steps: int = 10, n=(512, 384, 256), seed: int = 0,
              re: float = 1000.0) -> Case:
    """3D airway-like duct: a seeded union of 6-12 tubes (radius 0.05-0.2, seeded
    Catmull-Rom centre lines, radius bumps of 10%) in the box [0,1]x[0,0.75]x[0,0.5].
    Uniform inflow U = 1 on the fluid part of x = 0, convective outflow at x = 1; the
    y and z faces lie in the solid (no-slip y walls, periodic z).  Re = U D / nu on the
    inlet diameter D; dt at a Courant number 0.5 for a peak speed 2U."""
    from .generators import tube_union
    nx, ny, nz = n
    L = (1.0, 0.75, 0.5)
    geo = tube_union(seed, L=L)
    d_in = 2.0 * geo[2 + 3]              # twice the trunk's radius at its first point
    dx = L[0] / nx
    return Case(name=f"c4_airway_{nx}x{ny}x{nz}", ndim=3, n=(nx, ny, nz), L=L, origin=(0.0, 0.0, 0.0),
                bc_lo=(BC_INFLOW, BC_NOSLIP, BC_PERIODIC), bc_hi=(BC_OUTFLOW, BC_NOSLIP, BC_PERIODIC),
                geom_kind=GEOM_TUBES, geom_params=geo, nu=1.0 * d_in / re, dt=0.25 * dx,
                inflow=(1.0, 0.0, 0.0), precision=precision, steps=steps,
                init={"kind": "uniform", "U": 1.0}, seed=seed)


def pipe_case(N: int = 40, R: float = 1.0, nu: float = 1.0, nz: int = 1) -> Case:
    """Straight circular pipe along z on a 2.5R square of N x N cells (Sec. 2.3 example)."""
    L = 2.5 * R
    return Case(name=f"pipe_{N}", ndim=3, n=(N, N, nz), L=(L, L, 1.0),
                origin=(-L / 2, -L / 2, 0.0), bc_lo=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC),
                bc_hi=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC), geom_kind=GEOM_CYLINDER,
                geom_params=(0.0, 0.0, R, 1.0), nu=nu, dt=0.1 * (L / N) ** 2 / nu)


def small_case(kind: str, precision: str = "fp64", seed: int = 0) -> Case:
    """Oracle-sized cases spanning several 32-wide tiles with ragged tails."""
    if kind == "channel2d":
        c = channel_c1(precision=precision, steps=3)
        return c.with_(name="channel2d_70x37", n=(70, 37, 1), dt=0.004, seed=seed,
                       init={"kind": "channel_noise", "ylo": 0.137, "yhi": 0.861, "Ub": 0.6667,
                             "noise": 0.05})
    if kind == "cylinder2d":
        c = cylinder_c2(re=100.0, precision=precision, steps=2, seed=seed, n=(96, 50))
        return c.with_(name="cylinder2d_96x50", dt=0.01)
    if kind == "wavy3d":
        c = wavy_c3(precision=precision, steps=2, n=(70, 36, 20), seed=seed)
        return c.with_(name="wavy3d_70x36x20", dt=0.002)
    if kind == "cylinder2d_io":
        c = cylinder_c2_io(re=100.0, precision=precision, steps=2, seed=seed, n=(96, 50))
        return c.with_(name="cylinder2d_io_96x50", dt=0.01,
                       init={"kind": "uniform_noise", "U": 1.0, "noise": 0.1})
    if kind == "sphere3d_io":
        return Case(name="sphere3d_io_48x30x26", ndim=3, n=(48, 30, 26), L=(1.6, 1.0, 1.0),
                    origin=(0.0, 0.0, 0.0), bc_lo=(BC_INFLOW, BC_NOSLIP, BC_PERIODIC),
                    bc_hi=(BC_OUTFLOW, BC_FREESLIP, BC_PERIODIC), geom_kind=GEOM_SPHERE,
                    geom_params=(0.61, 0.47, 0.52, 0.23, -1.0), nu=0.01, dt=0.004, inflow=(0.8, 0.0, 0.0),
                    precision=precision, steps=2, seed=seed,
                    init={"kind": "uniform_noise", "U": 0.8, "noise": 0.1})
    if kind == "tubes3d_io":
        c = airway_c4(precision=precision, steps=2, n=(64, 48, 32), seed=seed)
        return c.with_(name="tubes3d_io_64x48x32", nu=0.01, dt=0.002,
                       init={"kind": "uniform_noise", "U": 1.0, "noise": 0.1})
    if kind == "sphere3d":
        return Case(name="sphere3d_48x30x26", ndim=3, n=(48, 30, 26), L=(1.6, 1.0, 1.0),
                    origin=(0.0, 0.0, 0.0), bc_lo=(BC_PERIODIC, BC_FREESLIP, BC_PERIODIC),
                    bc_hi=(BC_PERIODIC, BC_FREESLIP, BC_PERIODIC), geom_kind=GEOM_SPHERE,
                    geom_params=(0.61, 0.47, 0.52, 0.23, -1.0), nu=0.01, dt=0.004,
                    g=(1.0, 0.0, 0.0), precision=precision, steps=2, seed=seed,
                    init={"kind": "uniform_noise", "U": 0.5, "noise": 0.1})
    raise ValueError(kind)


def describe(case: Case) -> dict:
    """A JSON-friendly summary used by the bench line's `config`."""
    return {"workload": case.name, "cells": case.ncells, "grid": list(case.n[:case.ndim]),
            "precision": case.precision, "geometry": case.geom_kind, "nu": case.nu,
            "dt": case.dt, "flow_mode": case.flow_mode}



def serving_mix(seed: int = 0, n_requests: int = 1000, rate_hz: float = 10.0, step_scale: float = 1.0,
                size_scale: float = 1.0, precision: str = "fp32") -> list:
    """C5: a Poisson-arrival stream of 2D and 3D IBM solves.

    Each request: 2D n x n with n log-uniform in [128, 1024] or 3D n^3 with n
    log-uniform in [64, 192] (half and half); a seeded cylinder (2D) or
    sphere (3D) in a channel periodic in x (and z) with no-slip box walls in
    y; Re log-uniform in [10, 2000] on the body diameter and a unit stream;
    steps uniform in [500, 5000].  `step_scale` and `size_scale` shrink the
    steps and the linear sizes for bounded runs (sizes rounded to multiples
    of 8).  Returns [(arrival_seconds, Case, steps)] sorted by arrival.
    """
    from .generators import request_draws
    out = []
    for q, d in enumerate(request_draws(seed, n_requests)):
        t = d["arrival"] / rate_hz
        three = d["three"]
        lo, hi = (64, 192) if three else (128, 1024)
        n = int(round(lo * (hi / lo) ** d["size"] * size_scale / 8.0)) * 8
        n = max(n, 16)
        Lx = Ly = 2.0
        D = 0.5
        re = 10.0 * 200.0 ** d["re"]
        nu = 1.0 * D / re
        dx = Lx / n
        dt = min(0.4 * dx / 1.5, 0.12 * dx * dx / nu)
        steps = max(1, int(round((500 + 4500 * d["steps"]) * step_scale)))
        cx = 0.5 + d["cx"] * (Lx - 1.0)
        cy = 0.5 + d["cy"] * (Ly - 1.0)
        g = (8.0 * nu / Ly ** 2, 0.0, 0.0)   # unit centreline Poiseuille drive
        init = {"kind": "uniform_noise", "U": 0.5, "noise": 0.05}
        if three:
            cz = 0.5 + d["cz"] * (Ly - 1.0)
            case = Case(name=f"req{q}_3d_{n}", ndim=3, n=(n, n, n), L=(Lx, Ly, Ly), origin=(0.0, 0.0, 0.0),
                        bc_lo=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC), bc_hi=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC),
                        geom_kind=GEOM_SPHERE, geom_params=(cx, cy, cz, D / 2, -1.0), nu=nu, dt=dt, g=g,
                        precision=precision, steps=steps, init=init, seed=seed * 100003 + q)
        else:
            case = Case(name=f"req{q}_2d_{n}", ndim=2, n=(n, n, 1), L=(Lx, Ly, 1.0), origin=(0.0, 0.0, 0.0),
                        bc_lo=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC), bc_hi=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC),
                        geom_kind=GEOM_CYLINDER, geom_params=(cx, cy, D / 2, -1.0), nu=nu, dt=dt, g=g,
                        precision=precision, steps=steps, init=init, seed=seed * 100003 + q)
        out.append((t, case, steps))
    return sorted(out, key=lambda r: r[0])
