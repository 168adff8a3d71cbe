"""Steady single-component problems solved by direct matrix inversion.

Paper Sec. 2.3 solves the steady Laplacian with the IBM "by direct matrix
inversion"; this module assembles the same discrete operator for one
velocity component with no convection and no pressure:
    nu L_masked q - lambda q + s + f = 0   at the internal points of component c,
where L_masked reads external points as zero and y walls through mirror
ghosts (the same box rule as momentum.nb).  It is used for:
  * the Hagen-Poiseuille pipe (Eq. lapl): f Re_b against the exact 64;
  * the discrete steady state of the plane channel that the time-stepped
    solution must reach;
  * staircase (lambda = 0) versus IBM convergence slopes.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .grid import AX


def laplacian_matrix(grid, cls, c: int):
    """Sparse Laplacian (without nu) of component c over its internal points.

    Arm (d, s) of internal point P contributes -1/Delta_d^2 to P's column and:
      * +1/Delta_d^2 to the neighbour's column if the neighbour is internal;
      * nothing if the neighbour is external or a wall face (value zero);
      * sign/Delta_d^2 to P's own column if the arm leaves the box through a
        y wall and c is tangential to it (mirror ghost, -1 no-slip, +1 free-slip).
    """
    N = grid.shape[0] * grid.shape[1] * grid.shape[2]
    ids = np.arange(N).reshape(grid.shape)
    internal = cls.internal[c]
    rows, cols, vals = [], [], []
    for d in range(grid.ndim):
        inv = 1.0 / grid.d[d] ** 2
        ax = AX[d]
        n = grid.n[d]
        pos = np.arange(n).reshape([n if a == ax else 1 for a in range(3)])
        for s in (+1, -1):
            if d == 1 and grid.stretched:
                # uneven three-point second difference: arm s weighs 2 / (Delta_s (Delta_- + Delta_+))
                hm, hp = grid.y_spacing(c)
                inv = np.broadcast_to(2.0 / ((hp if s > 0 else hm) * (hm + hp)), grid.shape)
            w = (lambda sel: inv[sel]) if isinstance(inv, np.ndarray) else (lambda sel: np.full(int(sel.sum()), inv))
            r = ids[internal]
            rows.append(r)
            cols.append(r)
            vals.append(-w(internal))
            q_ids = np.roll(ids, -s, axis=ax)
            q_int = np.roll(internal, -s, axis=ax)
            if grid.periodic(d):
                inbox = np.ones(grid.shape, dtype=bool)
            else:
                inbox = np.broadcast_to((pos + s >= 0) & (pos + s <= n - 1), grid.shape)
            take = internal & inbox & q_int
            rows.append(ids[take])
            cols.append(q_ids[take])
            vals.append(w(take))
            if not grid.periodic(d) and c != d:
                out = internal & ~inbox
                sign = grid.wall_sign("hi" if s > 0 else "lo")
                rows.append(ids[out])
                cols.append(ids[out])
                vals.append(sign * w(out))
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    sel = np.flatnonzero(internal.ravel())
    return A[sel][:, sel], sel


def solve_component(grid, cls, weights, c: int, nu: float, f: float, use_ibm: bool = True):
    """Internal values of component c solving nu L q - lambda q + s + f = 0; zeros elsewhere."""
    A, sel = laplacian_matrix(grid, cls, c)
    lam = weights.lam[c].ravel()[sel] if use_ibm else np.zeros(sel.size)
    src = weights.src[c].ravel()[sel] if use_ibm else np.zeros(sel.size)
    M = nu * A - sp.diags(lam)
    q = spla.spsolve(M.tocsc(), -(src + f))
    out = np.zeros(grid.shape)
    out.ravel()[sel] = q
    return out
