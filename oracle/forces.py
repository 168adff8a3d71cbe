"""Force of the fluid on the body, from the discrete momentum budget (test infrastructure).

The paper reports drag and lift (Sec. 4.1, Tables re30 and re185) without saying how
they are computed.  Reading taken: the momentum the body exchanges with the fluid in
one time step, read off the discrete equations themselves.

Summed over the internal points of component c, the momentum stage of the solver
(momentum.stage_update) and the projection change the fluid momentum by
    sum_P dV (u^k_P - u^{k-1}_P) = sum_P dV (R_P + I_P) - c_k dt sum_P dV (G phi)_P
with R_P the explicit part of the stage (momentum.stage_update) and I_P what the
implicit IBM division adds on top of it.  In the flux-form right-hand side the flux
through a face between two internal points enters the two points with opposite
signs, and so does the pressure difference across it; what is left are the terms on
faces toward the box boundary and on faces toward external (solid) points.  The
latter, together with I_P and the wall source, are the body's share:

    BN_k = sum over internal P, over arms (d, s) whose neighbour Q = P + s e_d is
           external:  -s F_{c,d,s}(P) / Delta_d + nu (u_Q - u_P) / Delta_d^2
           (+ the wall source at P)
    with F_{c,d,s} the convective flux of component c through that face, as the
    right-hand side forms it (u_Q reads 0):
        d == c:  ((u_P + u_Q) / 2)^2
        d != c:  (advecting u_d at the face) (u_P + u_Q) / 2,
                 advecting u_d = (u_d(P) + u_d(P + e_c)) / 2            for s = +1,
                                 (u_d(P - e_d) + u_d(P - e_d + e_c)) / 2 for s = -1;
    BP_k(q) = sum over internal P, over arms along d = c with an external neighbour:
           +q(cell P + e_c) / Delta_c for s = +1,  -q(cell P) / Delta_c for s = -1
           (the ends of the runs of internal points in the sum of G q);
    impulse on the fluid in stage k:
        J_k = dV ( sum_P I_P  +  dt (a_k BN_k + b_k BN_{k-1})  -  c_k dt BP_k(p^k) ),
    p^k = p^{k-1} + phi^k (the pressure of the stage and its correction together).

The force on the body over the step is F = -(J_0 + J_1 + J_2) / dt.  In a box whose
faces exchange no momentum along c (periodic, or a free-slip wall for a tangential c)
the budget closes: sum_P dV (u^{n+1} - u^n) = g_c V_c dt - F dt (the test pin).
"""
from __future__ import annotations

import numpy as np

from .classify import _neighbour_external
from .grid import AX
from .momentum import masked, nb


def _shift_cells(q, grid, d: int, s: int):
    """Cell field q at (cell) P + s e_d; zero beyond a non-periodic face (never used there)."""
    if grid.periodic(d):
        return np.roll(q, -s, axis=AX[d])
    out = np.zeros_like(q)
    n = grid.n[d]
    src = [slice(None)] * 3
    dst = [slice(None)] * 3
    if s > 0:
        src[AX[d]], dst[AX[d]] = slice(1, n), slice(0, n - 1)
    else:
        src[AX[d]], dst[AX[d]] = slice(0, n - 1), slice(1, n)
    out[tuple(dst)] = q[tuple(src)]
    return out


def body_terms(grid, cls, u_prev, src, nu: float, lam_explicit=None):
    """BN_k per component (the body's share of sum_P N_P over internal points), from the
    stage's starting velocity u_prev (the fields the right-hand side reads).  With the
    explicit IBM treatment the right-hand side also holds -lambda u (lam_explicit)."""
    U = masked(grid, cls, u_prev)
    uin = None
    if grid.xflow:
        from .momentum import inflow_face
        uin = inflow_face(grid, cls)
    out = np.zeros(3)
    for c in range(grid.ncomp):
        inside = cls.internal[c]
        total = float(np.sum(np.where(inside, src[c], 0.0)))
        if lam_explicit is not None:
            total -= float(np.sum(np.where(inside, lam_explicit[c] * U[c], 0.0)))
        for d in range(grid.ndim):
            Dd = grid.d[d]
            for s in (+1, -1):
                arm = inside & _neighbour_external(cls.external[c], grid, d, s)
                if not arm.any():
                    continue
                uQ = nb(U[c], grid, c, d, s)
                if d == c:
                    F = ((U[c] + uQ) / 2) ** 2
                else:
                    # at an arm both points of the average lie in the box (or wrap), so the
                    # order of the two shifts does not matter
                    ud = U[d]
                    if s > 0:
                        adv = (ud + nb(ud, grid, d, c, +1)) / 2
                    else:
                        a = nb(ud, grid, d, d, -1, uin if d == 0 else None)
                        adv = (a + nb(a, grid, d, c, +1)) / 2
                    F = adv * ((U[c] + uQ) / 2)
                term = -s * F / Dd + nu * (uQ - U[c]) / Dd ** 2
                total += float(np.sum(np.where(arm, term, 0.0)))
        out[c] = total
    return out


def pressure_terms(grid, cls, q):
    """BP(q) per component: the body's share of sum_P (G q)_P over internal points."""
    out = np.zeros(3)
    for c in range(grid.ncomp):
        inside = cls.internal[c]
        Dc = grid.d[c]
        up = inside & _neighbour_external(cls.external[c], grid, c, +1)
        dn = inside & _neighbour_external(cls.external[c], grid, c, -1)
        out[c] = (float(np.sum(np.where(up, _shift_cells(q, grid, c, +1), 0.0)))
                  - float(np.sum(np.where(dn, q, 0.0)))) / Dc
    return out


def stage_impulse(grid, cls, I, BN_k, BN_prev, p_new, k: int, dt: float, a, b, cc):
    """J_k: the momentum the body gives the fluid in stage k (a vector over components);
    I per component is the IBM division's share at every point (zero off internal points)."""
    dV = grid.cell_volume()
    BP = pressure_terms(grid, cls, p_new)
    out = np.zeros(3)
    for c in range(grid.ncomp):
        sI = float(np.sum(np.where(cls.internal[c], I[c], 0.0)))
        out[c] = dV * (sI + dt * (a[k] * BN_k[c] + b[k] * BN_prev[c]) - cc[k] * dt * BP[c])
    return out


# ---- wall-shear stress along a lower wall (Sec. 4.2: the Fourier components tau_1c, tau_1s) ----
#
# Reading taken (the paper defines tau_1c and tau_1s from the time-averaged wall shear tau(x) but
# not how tau is read off the grid): along each vertical line of u points the lowest internal
# point P whose -y arm crosses the wall (distance delta, from the level set as for the weights)
# and the point Q above it give the quadratic through u = 0 at the wall, u_P at delta and u_Q at
# delta + Delta_y; its slope at the wall is
#     u'(0) = (u_P (delta + Delta)^2 - u_Q delta^2) / (delta Delta (delta + Delta)),
# exact for a parabola (u_P / delta when Q is not internal).  tau = nu u'(0), averaged over z;
# tau_1c = (2 / n_x) sum_i tau(x_i) cos(2 pi x_i / lambda), tau_1s likewise with sin, x_i the
# u points' x and lambda the wall's wavelength (the box length for other walls).

def wall_shear(grid, cls, levelset, u, nu: float, wavelength: float):
    """(tau(x) per u column, tau_1c, tau_1s); columns without a lower-wall arm are NaN.  On a
    stretched y the arm below P and the step from P to Q are the row's own centre distances."""
    nx, ny, nz = grid.n
    Dy = grid.d[1]
    if grid.stretched:
        hm_y, hp_y = (a.ravel() for a in grid.y_spacing(0))
    x, y, z = [np.broadcast_to(a, grid.shape) for a in grid.coords(0)]
    phi = cls.phi[0]
    ext = cls.external[0]
    inside = cls.internal[0]
    tau_sum = np.zeros(nx)
    cnt = np.zeros(nx)
    for k in range(nz):
        for i in range(nx):
            for j in range(1, ny):
                if not (inside[k, j, i] and ext[k, j - 1, i]):
                    continue
                P = [float(x[k, j, i]), float(y[k, j, i]), float(z[k, j, i])]
                Dm, Dp = (float(hm_y[j]), float(hp_y[j])) if grid.stretched else (Dy, Dy)
                delta = levelset.delta(P, 1, -1, Dm, float(phi[k, j, i]), float(phi[k, j - 1, i]))
                uP = float(u[k, j, i])
                if j + 1 < ny and inside[k, j + 1, i]:
                    uQ = float(u[k, j + 1, i])
                    slope = (uP * (delta + Dp) ** 2 - uQ * delta ** 2) / (delta * Dp * (delta + Dp))
                else:
                    slope = uP / delta
                tau_sum[i] += nu * slope
                cnt[i] += 1.0
    with np.errstate(invalid="ignore"):
        tau = np.where(cnt > 0, tau_sum / np.where(cnt > 0, cnt, 1.0), np.nan)
    xi = grid.axis_coords(0, 1.0)
    ok = np.isfinite(tau)
    t1c = 2.0 / nx * float(np.sum(np.where(ok, tau * np.cos(2.0 * np.pi * xi / wavelength), 0.0)))
    t1s = 2.0 / nx * float(np.sum(np.where(ok, tau * np.sin(2.0 * np.pi * xi / wavelength), 0.0)))
    return tau, t1c, t1s
