"""Level-set description of the body and the distance delta to the true boundary.

The paper compares each velocity grid with "the true boundary" (Sec. 3.3) and
needs, for every stencil arm that crosses it, the distance delta from the
internal point to the boundary along the arm (Sec. 2.2, Eq. interp-lin).  The
paper does not say how delta is found.  Reading taken: delta is the root of
the level set phi on the segment [P, Q] along the grid line:
  * closed form where one exists (planes, circles/spheres on any axis line,
    the sine wall on vertical lines);
  * otherwise bisection on phi restricted to the segment, run until the
    bracket cannot shrink in FP64, returning the upper end of the bracket.
phi < 0 is fluid; phi >= 0 is solid (strict inequality: a point exactly on
the interface is external).  If phi(Q) == 0 the interface passes through Q
and delta = Delta exactly, which gives lambda = 0 and the standard stencil.
delta is clamped to [1e-12 Delta, Delta].

Level sets (parameters as in include/ibm.h):
  NONE      phi = -1
  PLANES    [a, b]:            phi = max(a - y, y - b)        fluid a < y < b
  CYLINDER  [xc, yc, R, s]:    phi = s((x-xc)^2 + (y-yc)^2 - R^2)   (axis along z)
  SPHERE    [xc, yc, zc, R, s]: phi = s((x-xc)^2 + (y-yc)^2 + (z-zc)^2 - R^2)
            s = +1: fluid inside (pipe);  s = -1: fluid outside (body)
  SINE_WALL [y0, A, lam, ytop]: y_w = y0 + A sin(2 pi (x/lam)); phi = max(y_w - y, y - ytop)
  SAMPLED   phi given at the points; delta by linear interpolation
            delta = Delta phi_P / (phi_P - phi_Q)
"""
from __future__ import annotations

import math
import numpy as np

NONE, PLANES, CYLINDER, SPHERE, SINE_WALL, TUBES, SAMPLED = range(7)
TWO_PI = 6.283185307179586


class LevelSet:
    def __init__(self, kind: int, params=(), samples=None):
        self.kind = int(kind)
        self.p = tuple(float(v) for v in params)
        self.samples = samples  # SAMPLED: list of 3 arrays of shape (nz, ny, nx)
        if self.kind == TUBES:
            raise NotImplementedError("tube-union geometry is not in this oracle")

    # phi at arbitrary broadcastable coordinates (FP64, evaluated in the written order)
    def phi(self, x, y, z):
        k, p = self.kind, self.p
        if k == NONE:
            return np.full(np.broadcast(x, y, z).shape, -1.0)
        if k == PLANES:
            a, b = p[0], p[1]
            return np.maximum(a - y, y - b) + 0.0 * (x + z)
        if k == CYLINDER:
            xc, yc, R, s = p[0], p[1], p[2], p[3]
            dx = x - xc
            dy = y - yc
            return s * ((dx * dx + dy * dy) - R * R) + 0.0 * z
        if k == SPHERE:
            xc, yc, zc, R, s = p[0], p[1], p[2], p[3], p[4]
            dx = x - xc
            dy = y - yc
            dz = z - zc
            return s * (((dx * dx + dy * dy) + dz * dz) - R * R)
        if k == SINE_WALL:
            y0, A, lam, ytop = p[0], p[1], p[2], p[3]
            yw = y0 + A * np.sin(TWO_PI * (x / lam))
            return np.maximum(yw - y, y - ytop) + 0.0 * z
        raise ValueError(f"phi not defined for kind {k}")

    def phi_points(self, grid, c: int) -> np.ndarray:
        if self.kind == SAMPLED:
            return np.asarray(self.samples[c], dtype=np.float64)
        x, y, z = grid.coords(c)
        return np.broadcast_to(self.phi(x, y, z), grid.shape).copy()

    # ---- distance to the boundary along one arm ---------------------------------
    def delta(self, P, d: int, s: int, Delta: float, phiP: float, phiQ: float) -> float:
        """Distance from P (phi<0) to the interface towards Q = P + s Delta e_d (phi>=0)."""
        if phiQ == 0.0:
            return Delta
        if self.kind == SAMPLED:
            dl = Delta * (phiP / (phiP - phiQ))
        else:
            dl = self._closed_form(P, d, s, Delta)
            if dl is None:
                dl = self._bisect(P, d, s, Delta)
        return min(max(dl, 1e-12 * Delta), Delta)

    def _closed_form(self, P, d, s, Delta):
        k, p = self.kind, self.p
        x, y, z = P
        if k == PLANES and d == 1:
            return (y - p[0]) if s < 0 else (p[1] - y)
        if k == SINE_WALL and d == 1:
            if s < 0:
                yw = p[0] + p[1] * math.sin(TWO_PI * (x / p[2]))
                return y - yw
            return p[3] - y
        if k in (CYLINDER, SPHERE):
            ctr = [p[0], p[1], p[2] if k == SPHERE else 0.0]
            R = p[3] if k == SPHERE else p[2]
            dims = (0, 1, 2) if k == SPHERE else (0, 1)
            if d not in dims:
                return None
            rho2 = 0.0
            for e in dims:
                if e != d:
                    t = P[e] - ctr[e]
                    rho2 = rho2 + t * t
            h2 = R * R - rho2
            if h2 < 0.0:
                return None
            h = math.sqrt(h2)
            xp = P[d]
            xq = xp + s * Delta
            lo, hi = min(xp, xq), max(xp, xq)
            roots = [r for r in (ctr[d] - h, ctr[d] + h) if lo <= r <= hi]
            if len(roots) != 1:
                return None
            return abs(roots[0] - xp)
        return None

    def _bisect(self, P, d, s, Delta):
        lo, hi = 0.0, Delta
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if mid <= lo or mid >= hi:
                break
            Q = list(P)
            Q[d] = P[d] + s * mid
            if float(self.phi(Q[0], Q[1], Q[2])) < 0.0:
                lo = mid
            else:
                hi = mid
        return hi

    def wall_velocity_factor(self, d: int, s: int) -> float:
        """1 if the arm crosses the moving surface, else 0.

        Reading taken for wall velocity (Sec. 3.1 moving bodies): for PLANES the
        upper plane y=b moves, for SINE_WALL the wavy lower wall moves, for
        bodies (cylinder, sphere, sampled) the whole body moves."""
        if self.kind == PLANES:
            return 1.0 if (d == 1 and s > 0) else 0.0
        if self.kind == SINE_WALL:
            return 0.0 if (d == 1 and s > 0) else 1.0
        return 1.0
