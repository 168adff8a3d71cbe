"""Staircase classification (paper Sec. 3.3, "The underlying staircase approximation").

* Each velocity grid is compared with the true boundary on its own: a point
  of component c is internal (fluid, its momentum equation is solved) when
  phi_c < 0 and external (solid, velocity set to zero) otherwise.  Prescribed
  box-face points (normal component on a wall) are neither: they keep their
  boundary value.
* A pressure cell is internal when at least one of the velocity points on its
  faces is internal.
* An IBM point of component c is an internal point with at least one
  external neighbour on the same component grid along a stencil arm
  (Sec. 2.2: the correction applies only to stencils that cross the boundary).
  Neighbours beyond a wall box face are box-boundary ghosts, not arms.

* With an inflow/outflow x direction, the inflow face (x = x_0, not stored)
  and the outflow face (u at i = n_x - 1, a boundary point) are fluid where
  phi_u < 0 there: the inflow velocity enters, and the outflow value is read by
  the stencils and advanced by the convective condition, only on fluid faces.

Packed mask byte per cell (the format the C-ABI returns):
  bit0..2  u, v, w internal;  bit3  p internal;  bit4..6  u, v, w IBM point;
  bit7  (inflow/outflow x only) at i = 0: the inflow face of the row is fluid,
        at i = n_x - 1: the outflow face of the row is fluid.
IBM-point lists are sorted by ascending linear index i + nx (j + ny k).
"""
from __future__ import annotations

from dataclasses import dataclass
import numpy as np

from .grid import AX


@dataclass
class Classification:
    internal: list          # per component: bool arrays
    external: list
    boundary: list
    p_internal: np.ndarray
    ibm: list               # per component: bool arrays
    phi: list               # per component: level-set samples (FP64)
    mask: np.ndarray        # packed uint8
    lists: list             # per component: int64 ascending linear indices of IBM points
    inflow_fluid: np.ndarray = None    # (nz, ny, 1) bool: inflow face fluid (inflow/outflow x)
    outflow_fluid: np.ndarray = None   # (nz, ny, 1) bool: outflow face fluid


def _neighbour_external(ext: np.ndarray, grid, d: int, s: int) -> np.ndarray:
    """ext evaluated at P + s e_d for every P; False where the neighbour is beyond a wall face."""
    if grid.periodic(d):
        return np.roll(ext, -s, axis=AX[d])
    out = np.zeros_like(ext)
    n = grid.n[d]
    src = [slice(None)] * 3
    dst = [slice(None)] * 3
    if s > 0:
        src[AX[d]] = slice(1, n)
        dst[AX[d]] = slice(0, n - 1)
    else:
        src[AX[d]] = slice(0, n - 1)
        dst[AX[d]] = slice(1, n)
    out[tuple(dst)] = ext[tuple(src)]
    return out


def _face_minus(internal: np.ndarray, grid, d: int) -> np.ndarray:
    """internal of component d at the -d face of each cell (index - 1 along d)."""
    if grid.periodic(d):
        return np.roll(internal, 1, axis=AX[d])
    out = np.zeros_like(internal)
    n = grid.n[d]
    src = [slice(None)] * 3
    dst = [slice(None)] * 3
    src[AX[d]] = slice(0, n - 1)
    dst[AX[d]] = slice(1, n)
    out[tuple(dst)] = internal[tuple(src)]
    return out


def classify(grid, levelset) -> Classification:
    nc = grid.ncomp
    internal, external, boundary, phis = [], [], [], []
    for c in range(3):
        if c >= nc:
            z = np.zeros(grid.shape, dtype=bool)
            internal.append(z)
            external.append(z.copy())
            boundary.append(z.copy())
            phis.append(np.zeros(grid.shape))
            continue
        phi = levelset.phi_points(grid, c)
        bnd = grid.boundary_points(c)
        regular = ~bnd
        internal.append(regular & (phi < 0.0))
        external.append(regular & ~(phi < 0.0))
        boundary.append(bnd)
        phis.append(phi)

    # internal-pressure rule: any of the 2*ndim face velocities internal
    p_int = np.zeros(grid.shape, dtype=bool)
    for d in range(nc):
        p_int |= internal[d]
        p_int |= _face_minus(internal[d], grid, d)

    ibm = []
    for c in range(3):
        if c >= nc:
            ibm.append(np.zeros(grid.shape, dtype=bool))
            continue
        has_ext = np.zeros(grid.shape, dtype=bool)
        for d in range(grid.ndim):
            for s in (+1, -1):
                has_ext |= _neighbour_external(external[c], grid, d, s)
        ibm.append(internal[c] & has_ext)

    mask = np.zeros(grid.shape, dtype=np.uint8)
    for c in range(3):
        mask |= (internal[c].astype(np.uint8) << c)
        mask |= (ibm[c].astype(np.uint8) << (4 + c))
    mask |= (p_int.astype(np.uint8) << 3)

    inflow_fluid = outflow_fluid = None
    if grid.xflow:
        x, y, z = grid.coords(0)
        x_in = np.full_like(x[..., :1], grid.origin[0])          # u point at i = -1: the inflow face
        inflow_fluid = np.broadcast_to(levelset.phi(x_in, y, z) < 0.0, grid.shape[:2] + (1,)).copy()
        outflow_fluid = (phis[0][..., -1:] < 0.0).copy()
        mask[..., 0] |= (inflow_fluid[..., 0].astype(np.uint8) << 7)
        mask[..., -1] |= (outflow_fluid[..., 0].astype(np.uint8) << 7)

    lists = [np.flatnonzero(ibm[c].ravel()) for c in range(3)]
    return Classification(internal, external, boundary, p_int, ibm, phis, mask, lists, inflow_fluid, outflow_fluid)
