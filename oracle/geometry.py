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
  TUBES     [ntubes, npts, then per tube npts points (x, y, z, r)]: a union of tubes
            along polylines; phi = min over tubes and segments [A, B] of |X - C| - r(t),
            C = A + t (B - A) the projection of X clamped to t in [0, 1], r(t) linear
            between the end radii (fluid inside).  No closed form for delta: bisection.
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
            nt, npts = int(self.p[0]), int(self.p[1])
            self.tubes = np.asarray(self.p[2:2 + nt * npts * 4], dtype=np.float64).reshape(nt, npts, 4)

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
        if k == TUBES:
            x, y, z = np.broadcast_arrays(np.asarray(x, dtype=np.float64), np.asarray(y, dtype=np.float64),
                                          np.asarray(z, dtype=np.float64))
            if x.size == 1:
                return self._tubes_point(float(x.ravel()[0]), float(y.ravel()[0]), float(z.ravel()[0]))
            best = np.full(x.shape, 1e300)
            for tube in self.tubes:
                for a, b in zip(tube[:-1], tube[1:]):
                    ex, ey, ez = b[0] - a[0], b[1] - a[1], b[2] - a[2]
                    ee = (ex * ex + ey * ey) + ez * ez
                    wx, wy, wz = x - a[0], y - a[1], z - a[2]
                    we = (wx * ex + wy * ey) + wz * ez
                    t = np.minimum(np.maximum(we / ee, 0.0), 1.0)
                    dx = x - (a[0] + t * ex)
                    dy = y - (a[1] + t * ey)
                    dz = z - (a[2] + t * ez)
                    dist = np.sqrt((dx * dx + dy * dy) + dz * dz)
                    r = a[3] + t * (b[3] - a[3])
                    best = np.minimum(best, dist - r)
            return best
        raise ValueError(f"phi not defined for kind {k}")

    def _tubes_point(self, x: float, y: float, z: float) -> float:
        """phi of TUBES at one point: the same per-segment arithmetic as phi, with the
        segments of all tubes taken as one array."""
        if not hasattr(self, "_seg"):
            a = self.tubes[:, :-1, :].reshape(-1, 4)
            b = self.tubes[:, 1:, :].reshape(-1, 4)
            self._seg = (a, b)
        a, b = self._seg
        ex, ey, ez = b[:, 0] - a[:, 0], b[:, 1] - a[:, 1], b[:, 2] - a[:, 2]
        ee = (ex * ex + ey * ey) + ez * ez
        wx, wy, wz = x - a[:, 0], y - a[:, 1], z - a[:, 2]
        we = (wx * ex + wy * ey) + wz * ez
        t = np.minimum(np.maximum(we / ee, 0.0), 1.0)
        dx = x - (a[:, 0] + t * ex)
        dy = y - (a[:, 1] + t * ey)
        dz = z - (a[:, 2] + t * ez)
        dist = np.sqrt((dx * dx + dy * dy) + dz * dz)
        r = a[:, 3] + t * (b[:, 3] - a[:, 3])
        return float(np.min(dist - r))

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

    def delta_many(self, P, d, s, Delta, phiP, phiQ) -> np.ndarray:
        """delta for many arms at once (P: (m, 3)); each value equals delta(P[q], d[q], ...):
        the closed forms and the sampled interpolation arm by arm, the bisection for all
        remaining arms together (the same steps, stopped arm by arm)."""
        m = len(Delta)
        out = np.zeros(m)
        todo = []
        for q in range(m):
            if phiQ[q] == 0.0:
                out[q] = Delta[q]
            elif self.kind == SAMPLED:
                out[q] = Delta[q] * (phiP[q] / (phiP[q] - phiQ[q]))
            else:
                dl = self._closed_form(list(P[q]), int(d[q]), int(s[q]), float(Delta[q]))
                if dl is None:
                    todo.append(q)
                else:
                    out[q] = dl
        if todo:
            t = np.array(todo)
            out[t] = self._bisect_many(P[t], d[t], s[t], Delta[t])
        return np.minimum(np.maximum(out, 1e-12 * Delta), Delta)

    def _bisect_many(self, P, d, s, Delta):
        """_bisect for many arms: every arm takes the same midpoints and stops where its
        own bracket cannot shrink."""
        m = len(Delta)
        lo = np.zeros(m)
        hi = np.array(Delta, dtype=np.float64)
        active = np.ones(m, dtype=bool)
        rows = np.arange(m)
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            active &= ~((mid <= lo) | (mid >= hi))
            if not active.any():
                break
            a = rows[active]
            Q = P[a].copy()
            Q[np.arange(len(a)), d[a]] = P[a, d[a]] + s[a] * mid[a]
            inside = np.asarray(self.phi(Q[:, 0], Q[:, 1], Q[:, 2])) < 0.0
            lo[a[inside]] = mid[a[inside]]
            hi[a[~inside]] = mid[a[~inside]]
        return hi

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
