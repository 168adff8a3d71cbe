"""Seeded draws and initial-condition recipes.

Random numbers come from numpy's PCG64 (`numpy.random.default_rng(seed)`),
one independent stream per (seed, purpose) pair.  Nothing here classifies,
weights or advances a field: an initial condition is an analytic profile
evaluated at the staggered point positions plus seeded noise, defined over
the whole box (solid included); the solver masks it.

Staggered positions (the array layout every consumer uses): arrays have shape
(nz, ny, nx) with x fastest; cell (i,j,k) has centre
origin + ((i+1/2)dx, (j+1/2)dy, (k+1/2)dz); the u value of index (i,j,k)
sits on the cell's +x face, v on its +y face, w on its +z face.
"""
from __future__ import annotations

import numpy as np

_PURPOSE = {"u": 1, "v": 2, "w": 3, "offset": 7, "requests": 11, "tubes": 13}


def _rng(seed: int, purpose: str) -> np.random.Generator:
    return np.random.default_rng([int(seed), _PURPOSE[purpose]])


def request_draws(seed: int, n: int) -> list:
    """Seeded draws of a request stream: unit-rate Poisson arrival times and
    uniform [0, 1) numbers for size, Re, steps and body position.  Request q
    draws from its own stream, so the first k requests do not depend on n."""
    out = []
    t = 0.0
    for q in range(n):
        rng = np.random.default_rng([int(seed), _PURPOSE["requests"], q])
        t += float(rng.exponential(1.0))
        u = rng.random(7)
        out.append({"arrival": t, "three": bool(u[0] < 0.5), "size": float(u[1]), "re": float(u[2]),
                    "steps": float(u[3]), "cx": float(u[4]), "cy": float(u[5]), "cz": float(u[6])})
    return out


def cell_offset(seed: int, dx: float) -> tuple:
    """A seeded sub-cell offset in [0, dx)^2 for a body centre."""
    r = _rng(seed, "offset").random(2)
    return float(r[0] * dx), float(r[1] * dx)


def _catmull_rom(ctrl: np.ndarray, npts: int) -> np.ndarray:
    """npts points of the uniform Catmull-Rom spline through the control points ctrl
    (m, 3), taken at equal steps of the spline parameter; the end points are
    repeated to give the end segments their tangents.  The first and last points
    are the first and last control points."""
    m = len(ctrl)
    ext = np.vstack([ctrl[:1], ctrl, ctrl[-1:]])
    out = np.zeros((npts, 3))
    for q, u in enumerate(np.linspace(0.0, m - 1.0, npts)):
        s = min(int(u), m - 2)
        t = u - s
        p0, p1, p2, p3 = ext[s], ext[s + 1], ext[s + 2], ext[s + 3]
        out[q] = 0.5 * (2.0 * p1 + (p2 - p0) * t + (2.0 * p0 - 5.0 * p1 + 4.0 * p2 - p3) * t * t
                        + (3.0 * p1 - p0 - 3.0 * p2 + p3) * t * t * t)
    return out


def tube_union(seed: int, L=(1.0, 0.75, 0.5), ntubes=(6, 12), radius=(0.05, 0.2), npts: int = 24,
               margin: float = 0.01) -> tuple:
    """A seeded airway-like union of tubes in the box [0, L]: the geometry data
    (ntubes, npts, then per tube npts points (x, y, z, r)).

    Tube 0 is the trunk: it enters through the x = 0 face and leaves through the
    x = L_x face along a Catmull-Rom spline through 5 seeded control points.  Every
    other tube branches off a seeded interior point of an earlier tube, no wider
    than its parent there (or than the smallest radius, where the parent is
    narrower), and ends inside the box after 3 seeded steps of
    0.15-0.3 box units.  Each radius is r0 (1 + 0.1 sin(k s + ph)) along the tube,
    s in [0, 1] the sample position and k, ph seeded (the wall bumps).  Every point
    keeps its tube clear of the y and z faces by `margin`, and branches keep clear of
    the x faces too, so the box faces other than the trunk's ends lie in the solid.
    """
    rng = _rng(seed, "tubes")
    Lx, Ly, Lz = L
    nt = int(rng.integers(ntubes[0], ntubes[1] + 1))
    tubes = []

    def clamp(P, rmax, xfree):
        lo = rmax + margin
        P[:, 1] = np.clip(P[:, 1], lo, Ly - lo)
        P[:, 2] = np.clip(P[:, 2], lo, Lz - lo)
        if not xfree:
            P[:, 0] = np.clip(P[:, 0], lo, Lx - lo)
        return P

    def radii(r0):
        k = 2.0 * np.pi * (1.0 + 2.0 * rng.random())
        ph = 2.0 * np.pi * rng.random()
        s = np.linspace(0.0, 1.0, npts)
        return r0 * (1.0 + 0.1 * np.sin(k * s + ph))

    # trunk
    r0 = radius[0] + (radius[1] - radius[0]) * rng.random()
    rmax = 1.1 * r0
    xs = np.array([-0.05, 0.25, 0.5, 0.75, 1.05]) * Lx
    ctrl = np.zeros((5, 3))
    ctrl[:, 0] = xs
    ctrl[:, 1] = rmax + margin + (Ly - 2.0 * (rmax + margin)) * rng.random(5)
    ctrl[:, 2] = rmax + margin + (Lz - 2.0 * (rmax + margin)) * rng.random(5)
    P = clamp(_catmull_rom(ctrl, npts), rmax, xfree=True)
    tubes.append(np.column_stack([P, radii(r0)]))
    # branches
    while len(tubes) < nt:
        parent = tubes[int(rng.integers(len(tubes)))]
        inner = [q for q in range(1, npts - 1) if 0.1 * Lx <= parent[q, 0] <= 0.9 * Lx]
        q = inner[int(rng.integers(len(inner)))]
        rcap = min(radius[1], parent[q, 3])
        r0 = radius[0] + (max(rcap, radius[0]) - radius[0]) * rng.random()
        rmax = 1.1 * r0
        ctrl = np.zeros((4, 3))
        ctrl[0] = parent[q, :3]
        for m in range(1, 4):
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            ctrl[m] = ctrl[m - 1] + (0.15 + 0.15 * rng.random()) * d
        ctrl[1:] = clamp(ctrl[1:], rmax, xfree=False)
        P = _catmull_rom(ctrl, npts)
        P[1:] = clamp(P[1:], rmax, xfree=False)
        tubes.append(np.column_stack([P, radii(r0)]))
    data = np.stack(tubes)
    return (float(nt), float(npts)) + tuple(float(v) for v in data.ravel())


def noise_field(seed: int, comp: str, shape: tuple, amplitude: float) -> np.ndarray:
    """Uniform noise in [-amplitude, amplitude) for velocity component `comp`."""
    return amplitude * (2.0 * _rng(seed, comp).random(shape) - 1.0)


def _axes(case):
    nx, ny, nz = case.n
    dx, dy, dz = (case.L[0] / nx, case.L[1] / ny, case.L[2] / nz)
    x0, y0, z0 = case.origin
    yc = y0 + (np.arange(ny) + 0.5) * dy        # y of u and w points
    return yc, (nz, ny, nx)


def initial_field(case) -> dict:
    """Initial (u, v, w, p) as float64 arrays of shape (nz, ny, nx)."""
    yc, shape = _axes(case)
    u = np.zeros(shape)
    v = np.zeros(shape)
    w = np.zeros(shape)
    p = np.zeros(shape)
    init = case.init
    kind = init.get("kind", "zero")
    if kind == "zero":
        pass
    elif kind == "uniform":
        u[...] = init["U"]
    elif kind == "uniform_noise":
        u[...] = init["U"]
        a = init["noise"] * init["U"]
        u += noise_field(case.seed, "u", shape, a)
        v += noise_field(case.seed, "v", shape, a)
        if case.ndim == 3:
            w += noise_field(case.seed, "w", shape, a)
    elif kind == "channel_noise":
        ylo, yhi, ub = init["ylo"], init["yhi"], init["Ub"]
        H = yhi - ylo
        prof = np.clip(6.0 * ub * (yc - ylo) * (yhi - yc) / H ** 2, 0.0, None)
        u[...] = prof[None, :, None]
        a = init["noise"] * ub
        u += noise_field(case.seed, "u", shape, a)
        v += noise_field(case.seed, "v", shape, a)
        if case.ndim == 3:
            w += noise_field(case.seed, "w", shape, a)
    elif kind == "couette":
        a, b, U = init["a"], init["b"], init["U"]
        prof = np.where((yc > a) & (yc < b), U * (yc - a) / (b - a), 0.0)
        u[...] = prof[None, :, None]
    else:
        raise ValueError(f"unknown initial condition {kind!r}")
    return {"u": u, "v": v, "w": w, "p": p}
