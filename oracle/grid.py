"""Staggered Cartesian grid (paper Sec. 2.1, figure `staggered-grid`).

Pressure lives at cell centres and each velocity component on the cell face
normal to it.  Arrays have shape (nz, ny, nx), x fastest.  Direction d
(0=x, 1=y, 2=z) maps to numpy axis AX[d].  Cell (i,j,k) has centre
origin + ((i+1/2)dx, (j+1/2)dy, (k+1/2)dz); component c of index (i,j,k)
sits on the cell's +c face, i.e. its coordinate along c is origin_c+(idx_c+1)d_c.

Box boundaries: a periodic direction wraps.  In a non-periodic direction d
the +d box face carries the stored value of index n_d-1 of component d (a
prescribed "boundary" point, never solved by the momentum equation); the -d
box face value is implied by the boundary condition.
  * y: walls, no-slip or free-slip; both wall faces carry zero normal velocity.
  * x: either periodic, or an inflow at the -x face and a convective outflow at
    the +x face.  The inflow face is not stored: its normal velocity is the
    inflow velocity on fluid faces and zero on solid ones; tangential
    velocities are zero there.  The outflow face value u(n_x-1) is advanced by
    the convective condition (momentum.outflow_update); tangential velocities
    have zero normal gradient there.
"""
from __future__ import annotations

import numpy as np

AX = {0: 2, 1: 1, 2: 0}
BC_PERIODIC, BC_NOSLIP, BC_FREESLIP, BC_INFLOW, BC_OUTFLOW = 0, 1, 2, 3, 4


class Grid:
    def __init__(self, case):
        self.ndim = int(case.ndim)
        self.n = tuple(int(v) for v in case.n)
        self.L = tuple(float(v) for v in case.L)
        self.origin = tuple(float(v) for v in case.origin)
        self.bc_lo = tuple(int(v) for v in case.bc_lo)
        self.bc_hi = tuple(int(v) for v in case.bc_hi)
        # grid spacing: Delta_d = L_d / n_d
        self.d = tuple(self.L[i] / self.n[i] for i in range(3))
        self.shape = (self.n[2], self.n[1], self.n[0])
        self.ncomp = 3 if self.ndim == 3 else 2
        if self.ndim == 2 and self.n[2] != 1:
            raise ValueError("2D grids have nz == 1")
        if self.bc_lo[2] != BC_PERIODIC or self.bc_hi[2] != BC_PERIODIC:
            raise NotImplementedError("z must be periodic")
        xbc = (self.bc_lo[0], self.bc_hi[0])
        if xbc not in ((BC_PERIODIC, BC_PERIODIC), (BC_INFLOW, BC_OUTFLOW)):
            raise NotImplementedError("x is periodic or has an inflow at -x and an outflow at +x")
        if xbc[0] == BC_INFLOW and self.n[0] < 2:
            raise ValueError("an inflow/outflow x direction needs nx >= 2")
        self.inflow = tuple(float(v) for v in getattr(case, "inflow", (0.0, 0.0, 0.0)))
        if self.bc_lo[1] not in (BC_NOSLIP, BC_FREESLIP) or self.bc_hi[1] not in (BC_NOSLIP, BC_FREESLIP):
            raise NotImplementedError("y box faces must be no-slip or free-slip walls")
        if self.n[1] < 2:
            raise ValueError("ny >= 2")
        # stretched wall-normal grid (y): the ny + 1 face heights; cell centres midway
        # between faces, v on the faces (its index j on face j + 1)
        yf = tuple(getattr(case, "y_faces", ()))
        self.stretched = len(yf) > 0
        if self.stretched:
            yf = np.asarray(yf, dtype=np.float64)
            ny = self.n[1]
            if yf.shape != (ny + 1,) or np.any(np.diff(yf) <= 0.0):
                raise ValueError("y_faces: ny + 1 increasing heights")
            if abs(yf[0] - self.origin[1]) > 1e-12 * self.L[1] or \
                    abs(yf[-1] - self.origin[1] - self.L[1]) > 1e-12 * self.L[1]:
                raise ValueError("y_faces must span the box")
            self.yf = yf
            self.dyc = np.diff(yf)                       # cell heights
            self.yc = 0.5 * (yf[:-1] + yf[1:])           # cell centres
            # distance from centre j to centre j + 1; past the walls the mirror ghost of the
            # first / last centre, at its own height from the wall on the other side
            yc_ext = np.concatenate(([2 * yf[0] - self.yc[0]], self.yc, [2 * yf[-1] - self.yc[-1]]))
            self.hc = np.diff(yc_ext)                    # ny + 1 values: hc[j] spans centres j-1 .. j

    def periodic(self, d: int) -> bool:
        return self.bc_lo[d] == BC_PERIODIC

    def axis_coords(self, d: int, offset: float) -> np.ndarray:
        """origin_d + (index + offset) * Delta_d for every index along d (offset 0.5: cell
        centres, 1.0: the +d faces); on a stretched y the centres and faces given."""
        if d == 1 and self.stretched:
            return self.yc.copy() if offset == 0.5 else self.yf[1:].copy()
        return self.origin[d] + (np.arange(self.n[d]) + offset) * self.d[d]

    # ---- stretched y: spacings at every point, shaped (1, ny, 1) -------------------------
    def ycol(self, a) -> np.ndarray:
        return np.asarray(a, dtype=np.float64).reshape(1, self.n[1], 1)

    def y_spacing(self, c: int):
        """(h_minus, h_plus): distances from each point of component c to its y neighbours
        below and above (centres for u, w, p; faces for v).  Past a wall the mirror ghost of a
        centre; v's last index is the wall face itself (never solved, given its cell height)."""
        if c == 1:
            up = np.concatenate((self.dyc[1:], self.dyc[-1:]))
            return self.ycol(self.dyc), self.ycol(up)
        return self.ycol(self.hc[:-1]), self.ycol(self.hc[1:])

    def cell_heights(self) -> np.ndarray:
        return self.ycol(self.dyc)

    def face_heights(self) -> np.ndarray:
        """Distance between the centres on either side of each v face (the v control height);
        the last entry (the wall face) repeats the last cell height."""
        return self.ycol(np.concatenate((self.hc[1:-1], self.dyc[-1:])))

    def coords(self, c: int):
        """Broadcastable (x, y, z) coordinates of the points of component c.

        c = 0,1,2 for u,v,w; c = 3 for cell centres (pressure)."""
        out = []
        for d in range(3):
            off = 1.0 if d == c else 0.5
            a = self.axis_coords(d, off)
            shp = [1, 1, 1]
            shp[AX[d]] = self.n[d]
            out.append(a.reshape(shp))
        return out

    def boundary_points(self, c: int) -> np.ndarray:
        """Mask of prescribed box-face points of component c (normal component on a wall)."""
        m = np.zeros(self.shape, dtype=bool)
        if c < 3 and not self.periodic(c):
            idx = [slice(None)] * 3
            idx[AX[c]] = self.n[c] - 1
            m[tuple(idx)] = True
        return m

    def cell_volumes(self) -> np.ndarray:
        """Volume (area in 2D) of every cell, broadcastable to the field shape."""
        if not self.stretched:
            return np.full((1, 1, 1), self.cell_volume())
        v = self.d[0] * self.cell_heights()
        return v * self.d[2] if self.ndim == 3 else v

    def cell_volume(self) -> float:
        if self.stretched:
            raise ValueError("a stretched grid has no single cell volume (cell_volumes)")
        v = self.d[0] * self.d[1]
        if self.ndim == 3:
            v *= self.d[2]
        return v

    def wall_sign(self, side: str) -> float:
        """Ghost factor for tangential velocity beyond a y wall: -1 no-slip, +1 free-slip."""
        bc = self.bc_lo[1] if side == "lo" else self.bc_hi[1]
        return -1.0 if bc == BC_NOSLIP else 1.0

    def ghost_sign(self, d: int, side: str) -> float:
        """Ghost factor for a tangential velocity beyond the d box face: the y walls as
        above; -1 at an inflow face (tangential velocity zero on the face), +1 at an
        outflow face (zero normal gradient)."""
        if d == 1:
            return self.wall_sign(side)
        bc = self.bc_lo[d] if side == "lo" else self.bc_hi[d]
        return -1.0 if bc == BC_INFLOW else 1.0

    @property
    def xflow(self) -> bool:
        """x has an inflow (-x) and a convective outflow (+x) instead of wrapping."""
        return self.bc_lo[0] == BC_INFLOW
