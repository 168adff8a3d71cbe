"""IBM weights: lambda per IBM point, wall-velocity source, per-stage coefficients.

Paper Sec. 2.2: the ghost value across an arm that crosses the boundary at
distance delta is the linear extrapolation (Eq. interp-lin-extr)
    w_{i-1} = ((delta - Delta)/delta) w_i,
which folds into the centre weight of the 3-point second derivative
(Eq. disclapl-extr) as  d~(0) = d(0) - d(-1)(Delta - delta)/delta,  and the
correction term (Eq. lambda) is lambda = d(-1)(Delta - delta)/delta with
d(-1) = 1/Delta^2 on a uniform grid.  Corrections from different arms are
additive (end of Sec. 2.2).

Readings taken:
  * lambda carries the viscosity: the Laplacian in Eq. (ns) is multiplied by
    nu = 1/Re, so lambda_P = nu * sum_arms (Delta_d - delta)/(delta Delta_d^2)
    and enters the momentum equation as -lambda w (Eq. semidisc-mom-comp).
  * A wall moving with velocity U_w (Sec. 3.1: apply the IBM in the frame of
    the body) extrapolates through (delta, U_w) instead of (delta, 0).  The
    ghost becomes w_P (delta-Delta)/delta + U_w Delta/delta, i.e. the same
    -lambda w plus an explicit source s_P = nu * sum_arms U_w/(delta Delta_d).

Time integration (Sec. 2.4): A w^{n+1} - B w^n = C F with C = Delta t,
B = x/(e^x - 1), A = x + B, x = lambda Delta t (Eq. Bexpr, expint); with the
Rai-Moin RK3 (Eq. rk3-rai) the stage-k value of x is lambda c_k Delta t.
B(0) is 0/0; reading taken: B := 1 when x == 0, so the plain scheme is
recovered exactly.  EULER mode is B = 1 (Eq. time-adv-impl); TAYLOR2 is the
reciprocal of the 2-term Taylor expansion of (e^x - 1)/x, B = 1/(1 + x/2)
(the option mentioned after Eq. Bexpr).  EXPLICIT is the classic explicit treatment
the paper compares against (end of Sec. 2.5): -lambda w joins the explicit right-hand
side and there is no division (B = 1, x = 0 in the stage update).
"""
from __future__ import annotations

from dataclasses import dataclass
import numpy as np

# Rai & Moin (1991) coefficients as printed after Eq. (rk3-rai)
RK3_A = (64.0 / 120.0, 50.0 / 120.0, 90.0 / 120.0)
RK3_B = (0.0, -34.0 / 120.0, -50.0 / 120.0)
RK3_C = tuple(a + b for a, b in zip(RK3_A, RK3_B))

B_EXACT, B_EULER, B_TAYLOR2, B_EXPLICIT = 0, 1, 2, 3

# stage times of the Rai-Moin RK3 as fractions of the step: stage k evaluates its explicit
# right-hand side at t_n + RK3_T[k] dt (RK3_T[k] = sum of the c of the earlier stages)
RK3_T = (0.0, RK3_C[0], RK3_C[0] + RK3_C[1])


def B_of_x(x, mode: int):
    x = np.asarray(x, dtype=np.float64)
    if mode in (B_EULER, B_EXPLICIT):
        return np.ones_like(x)
    if mode == B_TAYLOR2:
        return 1.0 / (1.0 + x / 2.0)
    out = np.ones_like(x)
    pos = x > 0.0
    with np.errstate(over="ignore"):
        out[pos] = x[pos] / np.expm1(x[pos])
    return out


@dataclass
class Weights:
    lam: list        # per component: dense FP64 array, 0 away from IBM points
    src: list        # per component: dense FP64 source s_P
    lam_list: list   # per component: lambda at the IBM points in list order
    src_list: list


def build_weights(grid, levelset, cls, nu: float, wall_u=(0.0, 0.0, 0.0), no_ibm: bool = False,
                  wall_field=None) -> Weights:
    """lambda and the wall source at every IBM point, arms taken in the order d = x, y, z
    and s = +1, -1 (the distance of every crossed arm comes from levelset.delta_many,
    which gives each arm the same value as levelset.delta).  wall_field(X, c): the wall's
    velocity component c at the crossing point X (a rotating body), in place of wall_u."""
    lam, src, lam_list, src_list = [], [], [], []
    nx, ny, nz = grid.n
    for c in range(3):
        L = np.zeros(grid.shape)
        S = np.zeros(grid.shape)
        lst = cls.lists[c]
        ll = np.zeros(len(lst))
        sl = np.zeros(len(lst))
        if c < grid.ncomp and not no_ibm and len(lst):
            ext = cls.external[c]
            phi = cls.phi[c]
            # pass 1: the crossed arms of every IBM point, in accumulation order
            arms = []          # (m, P, d, s, Delta, phiP, phiQ, Delta_- + Delta_+)
            if grid.stretched:
                ycs = grid.axis_coords(1, 1.0 if c == 1 else 0.5)
                hm_y, hp_y = (a.ravel() for a in grid.y_spacing(c))
            for m, lin in enumerate(lst):
                i = lin % nx
                j = (lin // nx) % ny
                k = lin // (nx * ny)
                idx = [i, j, k]
                P = [grid.origin[d] + (idx[d] + (1.0 if d == c else 0.5)) * grid.d[d] for d in range(3)]
                if grid.stretched:
                    P[1] = float(ycs[j])
                for d in range(grid.ndim):
                    for s in (+1, -1):
                        q = list(idx)
                        q[d] = q[d] + s
                        if grid.periodic(d):
                            q[d] %= grid.n[d]
                        elif not (0 <= q[d] < grid.n[d]):
                            continue
                        qk = (q[2], q[1], q[0])
                        if not ext[qk]:
                            continue
                        if d == 1 and grid.stretched:
                            Dd = float(hp_y[j] if s > 0 else hm_y[j])
                            Dsum = float(hm_y[j] + hp_y[j])
                        else:
                            Dd = grid.d[d]
                            Dsum = 2.0 * Dd
                        arms.append((m, P, d, s, Dd, float(phi[k, j, i]), float(phi[qk]), Dsum))
            deltas = levelset.delta_many(np.array([a[1] for a in arms]).reshape(-1, 3),
                                         np.array([a[2] for a in arms], dtype=int),
                                         np.array([a[3] for a in arms], dtype=int),
                                         np.array([a[4] for a in arms], dtype=np.float64),
                                         np.array([a[5] for a in arms], dtype=np.float64),
                                         np.array([a[6] for a in arms], dtype=np.float64))
            # pass 2: lambda and the source, summed arm by arm
            lam_p = np.zeros(len(lst))
            src_p = np.zeros(len(lst))
            for (m, P, d, s, Dd, _, _, Dsum), delta in zip(arms, deltas):
                if wall_field is not None:
                    X = list(P)
                    X[d] = X[d] + s * delta
                    uw = wall_field(X, c) * levelset.wall_velocity_factor(d, s)
                else:
                    uw = wall_u[c] * levelset.wall_velocity_factor(d, s)
                if d == 1 and grid.stretched:
                    # d(s) = 2 / (Delta_s (Delta_- + Delta_+)) of the uneven three-point second
                    # difference in place of 1 / Delta^2 (same extrapolation, same form)
                    lam_p[m] += nu * 2.0 * (Dd - delta) / (delta * Dd * Dsum)
                    src_p[m] += nu * uw * 2.0 / (delta * Dsum)
                else:
                    lam_p[m] += nu * (Dd - delta) / (delta * Dd * Dd)
                    src_p[m] += nu * uw / (delta * Dd)
            for m, lin in enumerate(lst):
                i = lin % nx
                j = (lin // nx) % ny
                k = lin // (nx * ny)
                ll[m] = lam_p[m]
                sl[m] = src_p[m]
                L[k, j, i] = lam_p[m]
                S[k, j, i] = src_p[m]
        lam.append(L)
        src.append(S)
        lam_list.append(ll)
        src_list.append(sl)
    return Weights(lam, src, lam_list, src_list)

