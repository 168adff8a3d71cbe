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

_PURPOSE = {"u": 1, "v": 2, "w": 3, "offset": 7, "requests": 11}


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
