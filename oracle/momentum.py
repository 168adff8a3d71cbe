"""Explicit right-hand side and the implicit-IBM RK3 stage (paper Sec. 2.1, 2.4).

Right-hand side at internal points (Eq. ns, Eq. semidisc-mom):
    N_c = -C_c(u) + nu L_c(u) + g_c + s_c
  * L is the 3-point-per-direction Laplacian (Eq. disclapl) with d(+-1) =
    1/Delta^2, d(0) = -2/Delta^2, read with every external velocity equal to
    zero.  With the explicit right-hand side the ghost term then vanishes on
    its own and the IBM reduces to -lambda w (Eq. semidisc-mom-comp).
  * C is not written out in the paper.  Reading taken: the divergence
    (flux) form on the staggered grid with two-point arithmetic averages
    (Harlow-Welch):  C_u = d(uu)/dx + d(vu)/dy + d(wu)/dz with uu at cell
    centres, vu / wu at cell edges; no IBM correction of convection (Sec. 2).
  * s_c is the wall-velocity source (zero for walls at rest).
Box walls in y: tangential velocity ghosts mirror the adjacent value (sign -1
no-slip, +1 free-slip); the wall-normal velocity on the wall face is zero.
Inflow/outflow in x (readings; the paper states only that inflow and outflow
faces exist, Sec. 4): the normal velocity at the inflow face is the inflow
velocity on fluid faces and zero on solid ones, tangential ghosts are the
negated adjacent value (zero tangential velocity on the face); at the outflow
face the stored u(n_x-1) is read, tangential ghosts repeat the adjacent value.
The outflow value follows the convective condition du/dt + U_c du/dx = 0
(outflow_update), U_c the inflow flux over the fluid outflow area.

Stage k (Eq. rk3-rai), with the pressure of the incremental projection
(Sec. 2.1) carried with weight c_k (reading taken):
    R   = Delta t (a_k N^{k-1} + b_k N^{k-2}) - c_k Delta t G p^{k-1}
    x   = lambda c_k Delta t
    u*  = (B(x) u^{k-1} + R) / (B(x) + x)     at internal points
    u*  = 0                                   at external points
"""
from __future__ import annotations

import numpy as np

from .grid import AX


def readable(grid, cls, c: int) -> np.ndarray:
    """Points whose stored value the operators read: internal points, and the fluid
    outflow face of u.  Everything else (external points, wall faces, solid outflow
    faces) reads zero."""
    r = cls.internal[c]
    if c == 0 and grid.xflow:
        r = r.copy()
        r[..., -1] = cls.outflow_fluid[..., 0]
    return r


def masked(grid, cls, fields):
    """Velocity with every unreadable point read as zero (external and wall faces)."""
    return [np.where(readable(grid, cls, c), fields[c], 0.0) if c < grid.ncomp else np.zeros(grid.shape)
            for c in range(3)]


def inflow_face(grid, cls) -> np.ndarray:
    """Normal velocity on the inflow face, shape (nz, ny, 1)."""
    return np.where(cls.inflow_fluid, grid.inflow[0], 0.0)


def nb(q, grid, c: int, d: int, s: int, lo_normal=None):
    """Values of component-c field q at P + s e_d, with the box rules: y walls, and
    for an inflow/outflow x the inflow face value lo_normal of the normal component."""
    if grid.periodic(d):
        return np.roll(q, -s, axis=AX[d])
    n = grid.n[d]
    ax = AX[d]
    out = np.empty_like(q)
    src = [slice(None)] * 3
    dst = [slice(None)] * 3
    edge_dst = [slice(None)] * 3
    edge_src = [slice(None)] * 3
    if s > 0:
        src[ax] = slice(1, n)
        dst[ax] = slice(0, n - 1)
        edge_dst[ax] = slice(n - 1, n)
        edge_src[ax] = slice(n - 1, n)
        sign = grid.ghost_sign(d, "hi")
    else:
        src[ax] = slice(0, n - 1)
        dst[ax] = slice(1, n)
        edge_dst[ax] = slice(0, 1)
        edge_src[ax] = slice(0, 1)
        sign = grid.ghost_sign(d, "lo")
    out[tuple(dst)] = q[tuple(src)]
    if c == d:
        # normal component: the value beyond is the face value (zero on walls and
        # beyond the outflow face, where it is never read; the inflow value at -x)
        out[tuple(edge_dst)] = 0.0
        if s < 0 and lo_normal is not None:
            out[tuple(edge_dst)] = lo_normal
    else:
        out[tuple(edge_dst)] = sign * q[tuple(edge_src)]
    return out


def rhs(grid, cls, fields, nu: float, g, src, body_u=None):
    """N_c at every point (meaningful at internal points), FP64.  body_u: the velocity of a
    translating body, which the convective terms read at its (external) points; the
    Laplacian still reads them as zero, its wall term being -lambda w + s (reading R24)."""
    if body_u is not None:
        return rhs_moving(grid, cls, fields, nu, g, src, body_u)
    if grid.stretched:
        return rhs_stretched(grid, cls, fields, nu, g, src)
    U, V, W = masked(grid, cls, fields)
    dx, dy, dz = grid.d
    three = grid.ndim == 3
    uin = inflow_face(grid, cls) if grid.xflow else None
    out = []

    # ---- u ----
    uE, uW = nb(U, grid, 0, 0, +1), nb(U, grid, 0, 0, -1, uin)
    uN, uS = nb(U, grid, 0, 1, +1), nb(U, grid, 0, 1, -1)
    cx = (((U + uE) / 2) ** 2 - ((uW + U) / 2) ** 2) / dx
    vN = (V + nb(V, grid, 1, 0, +1)) / 2                       # v(i,j) + v(i+1,j)
    vS = (nb(V, grid, 1, 1, -1) + nb(nb(V, grid, 1, 0, +1), grid, 1, 1, -1)) / 2
    cy = (vN * ((U + uN) / 2) - vS * ((uS + U) / 2)) / dy
    lap = (uE - 2 * U + uW) / dx ** 2 + (uN - 2 * U + uS) / dy ** 2
    cz = 0.0
    if three:
        uT, uB = nb(U, grid, 0, 2, +1), nb(U, grid, 0, 2, -1)
        wT = (W + nb(W, grid, 2, 0, +1)) / 2                   # w(i,j,k) + w(i+1,j,k)
        wB = (nb(W, grid, 2, 2, -1) + nb(nb(W, grid, 2, 0, +1), grid, 2, 2, -1)) / 2
        cz = (wT * ((U + uT) / 2) - wB * ((uB + U) / 2)) / dz
        lap = lap + (uT - 2 * U + uB) / dz ** 2
    out.append(-(cx + cy + cz) + nu * lap + g[0] + src[0])

    # ---- v ----
    vE, vW = nb(V, grid, 1, 0, +1), nb(V, grid, 1, 0, -1)
    vNn, vSs = nb(V, grid, 1, 1, +1), nb(V, grid, 1, 1, -1)
    uEe = (U + nb(U, grid, 0, 1, +1)) / 2                      # u(i,j) + u(i,j+1)
    uWe = (nb(U, grid, 0, 0, -1, uin) + nb(nb(U, grid, 0, 0, -1, uin), grid, 0, 1, +1)) / 2
    cx = (uEe * ((V + vE) / 2) - uWe * ((vW + V) / 2)) / dx
    cy = (((V + vNn) / 2) ** 2 - ((vSs + V) / 2) ** 2) / dy
    lap = (vE - 2 * V + vW) / dx ** 2 + (vNn - 2 * V + vSs) / dy ** 2
    cz = 0.0
    if three:
        vT, vB = nb(V, grid, 1, 2, +1), nb(V, grid, 1, 2, -1)
        wTe = (W + nb(W, grid, 2, 1, +1)) / 2                  # w(i,j,k) + w(i,j+1,k)
        wBe = (nb(W, grid, 2, 2, -1) + nb(nb(W, grid, 2, 2, -1), grid, 2, 1, +1)) / 2
        cz = (wTe * ((V + vT) / 2) - wBe * ((vB + V) / 2)) / dz
        lap = lap + (vT - 2 * V + vB) / dz ** 2
    out.append(-(cx + cy + cz) + nu * lap + g[1] + src[1])

    # ---- w ----
    if three:
        wE, wW = nb(W, grid, 2, 0, +1), nb(W, grid, 2, 0, -1)
        wN, wS = nb(W, grid, 2, 1, +1), nb(W, grid, 2, 1, -1)
        wT, wB = nb(W, grid, 2, 2, +1), nb(W, grid, 2, 2, -1)
        uEe = (U + nb(U, grid, 0, 2, +1)) / 2                  # u(i,j,k) + u(i,j,k+1)
        uWe = (nb(U, grid, 0, 0, -1, uin) + nb(nb(U, grid, 0, 0, -1, uin), grid, 0, 2, +1)) / 2
        cx = (uEe * ((W + wE) / 2) - uWe * ((wW + W) / 2)) / dx
        vNe = (V + nb(V, grid, 1, 2, +1)) / 2                  # v(i,j,k) + v(i,j,k+1)
        vSe = (nb(V, grid, 1, 1, -1) + nb(nb(V, grid, 1, 1, -1), grid, 1, 2, +1)) / 2
        cy = (vNe * ((W + wN) / 2) - vSe * ((wS + W) / 2)) / dy
        cz = (((W + wT) / 2) ** 2 - ((wB + W) / 2) ** 2) / dz
        lap = (wE - 2 * W + wW) / dx ** 2 + (wN - 2 * W + wS) / dy ** 2 + (wT - 2 * W + wB) / dz ** 2
        out.append(-(cx + cy + cz) + nu * lap + g[2] + src[2])
    else:
        out.append(np.zeros(grid.shape))
    return out


def rhs_moving(grid, cls, fields, nu: float, g, src, body_u):
    """rhs with a translating body (uniform grid): convection of the field whose external
    points hold the body velocity, plus nu times the Laplacian of the field whose external
    points hold zero; each is the uniform rhs of its own field, so the split is
    N = rhs(convection part, nu = 0) + (rhs(diffusion part) - its own convection)."""
    from dataclasses import replace
    conv_field = [np.where(cls.external[c], body_u[c], fields[c]) if c < grid.ncomp else fields[c]
                  for c in range(3)]
    # the body's points made readable for the convective call (they hold body_u now)
    cls_b = replace(cls, internal=[cls.internal[c] | cls.external[c] for c in range(3)])
    zero = [np.zeros(grid.shape)] * 3
    Nc = rhs(grid, cls_b, conv_field, 0.0, (0.0, 0.0, 0.0), zero)    # -C(u with the body's velocity)
    Nd = rhs(grid, cls, fields, nu, g, src)                          # -C(u masked) + nu L + g + s
    Nd0 = rhs(grid, cls, fields, 0.0, (0.0, 0.0, 0.0), zero)         # -C(u masked)
    return [Nc[c] + (Nd[c] - Nd0[c]) for c in range(3)]


def d2_y(q, qn, qs, hm, hp):
    """The three-point second difference along y on unevenly spaced points: with hm, hp the
    distances to the neighbours below and above, d(+1) = 2/(hp (hm + hp)),
    d(-1) = 2/(hm (hm + hp)), d(0) = -2/(hm hp) (exact on quadratics)."""
    return 2.0 * qn / (hp * (hm + hp)) + 2.0 * qs / (hm * (hm + hp)) - 2.0 * q / (hm * hp)


def y_face_value(q, qn, dyc, dyc_up):
    """A cell-centred quantity (q at this centre, qn at the centre above) linearly
    interpolated to the face between them, which lies dyc/2 above this centre and
    dyc_up/2 below the other."""
    return (dyc_up * q + dyc * qn) / (dyc + dyc_up)


def rhs_stretched(grid, cls, fields, nu: float, g, src):
    """N_c on a stretched y (readings of the paper's stretched wall-normal grids, Sec. 4.2,
    which it does not write out): x and z as on the uniform grid; along y
      * the Laplacian is the three-point second difference on the uneven points (d2_y);
      * the convective fluxes stay in flux form: a cell-centred quantity (u, w) is carried
        to a v face by linear interpolation (y_face_value) and the flux difference is
        divided by the height of the point's own control volume (the cell height for u and
        w, the distance between the centres on either side for v); v is carried to a
        centre by the plain average (the centre lies midway between its faces)."""
    U, V, W = masked(grid, cls, fields)
    dx, _, dz = grid.d
    three = grid.ndim == 3
    uin = inflow_face(grid, cls) if grid.xflow else None
    dyc = grid.cell_heights()
    dyc_up = grid.ycol(np.concatenate((grid.dyc[1:], grid.dyc[-1:])))    # the cell above (mirror)
    dyc_dn = grid.ycol(np.concatenate((grid.dyc[:1], grid.dyc[:-1])))    # the cell below (mirror)
    hv = grid.face_heights()
    hm_c, hp_c = grid.y_spacing(0)
    hm_v, hp_v = grid.y_spacing(1)
    out = []

    # ---- u ----
    uE, uW = nb(U, grid, 0, 0, +1), nb(U, grid, 0, 0, -1, uin)
    uN, uS = nb(U, grid, 0, 1, +1), nb(U, grid, 0, 1, -1)
    cx = (((U + uE) / 2) ** 2 - ((uW + U) / 2) ** 2) / dx
    vN = (V + nb(V, grid, 1, 0, +1)) / 2                       # v on the top face at the u point's x
    vS = (nb(V, grid, 1, 1, -1) + nb(nb(V, grid, 1, 0, +1), grid, 1, 1, -1)) / 2
    cy = (vN * y_face_value(U, uN, dyc, dyc_up) - vS * y_face_value(uS, U, dyc_dn, dyc)) / dyc
    lap = (uE - 2 * U + uW) / dx ** 2 + d2_y(U, uN, uS, hm_c, hp_c)
    cz = 0.0
    if three:
        uT, uB = nb(U, grid, 0, 2, +1), nb(U, grid, 0, 2, -1)
        wT = (W + nb(W, grid, 2, 0, +1)) / 2
        wB = (nb(W, grid, 2, 2, -1) + nb(nb(W, grid, 2, 0, +1), grid, 2, 2, -1)) / 2
        cz = (wT * ((U + uT) / 2) - wB * ((uB + U) / 2)) / dz
        lap = lap + (uT - 2 * U + uB) / dz ** 2
    out.append(-(cx + cy + cz) + nu * lap + g[0] + src[0])

    # ---- v (on the face above its cell: between centres j and j + 1) ----
    vE, vW = nb(V, grid, 1, 0, +1), nb(V, grid, 1, 0, -1)
    vNn, vSs = nb(V, grid, 1, 1, +1), nb(V, grid, 1, 1, -1)
    uEe = y_face_value(U, nb(U, grid, 0, 1, +1), dyc, dyc_up)            # u at this face, x = i + 1
    uWl = nb(U, grid, 0, 0, -1, uin)
    uWe = y_face_value(uWl, nb(uWl, grid, 0, 1, +1), dyc, dyc_up)
    cx = (uEe * ((V + vE) / 2) - uWe * ((vW + V) / 2)) / dx
    cy = (((V + vNn) / 2) ** 2 - ((vSs + V) / 2) ** 2) / hv
    lap = (vE - 2 * V + vW) / dx ** 2 + d2_y(V, vNn, vSs, hm_v, hp_v)
    cz = 0.0
    if three:
        vT, vB = nb(V, grid, 1, 2, +1), nb(V, grid, 1, 2, -1)
        wTe = y_face_value(W, nb(W, grid, 2, 1, +1), dyc, dyc_up)
        wBl = nb(W, grid, 2, 2, -1)
        wBe = y_face_value(wBl, nb(wBl, grid, 2, 1, +1), dyc, dyc_up)
        cz = (wTe * ((V + vT) / 2) - wBe * ((vB + V) / 2)) / dz
        lap = lap + (vT - 2 * V + vB) / dz ** 2
    out.append(-(cx + cy + cz) + nu * lap + g[1] + src[1])

    # ---- w ----
    if three:
        wE, wW = nb(W, grid, 2, 0, +1), nb(W, grid, 2, 0, -1)
        wN, wS = nb(W, grid, 2, 1, +1), nb(W, grid, 2, 1, -1)
        wT, wB = nb(W, grid, 2, 2, +1), nb(W, grid, 2, 2, -1)
        uEe = (U + nb(U, grid, 0, 2, +1)) / 2
        uWe = (nb(U, grid, 0, 0, -1, uin) + nb(nb(U, grid, 0, 0, -1, uin), grid, 0, 2, +1)) / 2
        cx = (uEe * ((W + wE) / 2) - uWe * ((wW + W) / 2)) / dx
        vNe = (V + nb(V, grid, 1, 2, +1)) / 2
        vSe = (nb(V, grid, 1, 1, -1) + nb(nb(V, grid, 1, 1, -1), grid, 1, 2, +1)) / 2
        cy = (vNe * y_face_value(W, wN, dyc, dyc_up) - vSe * y_face_value(wS, W, dyc_dn, dyc)) / dyc
        cz = (((W + wT) / 2) ** 2 - ((wB + W) / 2) ** 2) / dz
        lap = (wE - 2 * W + wW) / dx ** 2 + d2_y(W, wN, wS, hm_c, hp_c) + (wT - 2 * W + wB) / dz ** 2
        out.append(-(cx + cy + cz) + nu * lap + g[2] + src[2])
    else:
        out.append(np.zeros(grid.shape))
    return out


def pressure_gradient(grid, p):
    """(G p)_c on the faces; zero on wall faces (Gp is not used there)."""
    out = []
    for c in range(3):
        if c >= grid.ncomp:
            out.append(np.zeros(grid.shape))
            continue
        if grid.periodic(c):
            out.append((np.roll(p, -1, axis=AX[c]) - p) / grid.d[c])
        else:
            gph = np.zeros(grid.shape)
            n = grid.n[c]
            a = [slice(None)] * 3
            b = [slice(None)] * 3
            o = [slice(None)] * 3
            a[AX[c]] = slice(1, n)
            b[AX[c]] = slice(0, n - 1)
            o[AX[c]] = slice(0, n - 1)
            if c == 1 and grid.stretched:
                gph[tuple(o)] = (p[tuple(a)] - p[tuple(b)]) / grid.face_heights()[:, :-1, :]
            else:
                gph[tuple(o)] = (p[tuple(a)] - p[tuple(b)]) / grid.d[c]
            out.append(gph)
    return out


def stage_update(grid, cls, u_prev, N_cur, N_prev, gradp, lam, k: int, dt: float,
                 bmode: int, a, b, cc, B_of_x):
    """u* of Eq. (rk3-rai) at internal points, zero elsewhere (k = 0, 1, 2)."""
    out = []
    for c in range(3):
        if c >= grid.ncomp:
            out.append(np.zeros(grid.shape))
            continue
        R = dt * (a[k] * N_cur[c] + b[k] * N_prev[c]) - cc[k] * dt * gradp[c]
        x = lam[c] * cc[k] * dt
        B = B_of_x(x, bmode)
        ustar = (B * u_prev[c] + R) / (B + x)
        out.append(np.where(cls.internal[c], ustar, 0.0))
    return out


# ---- convective outflow (inflow/outflow x) ------------------------------------------
def outflow_speed(grid, cls) -> float:
    """U_c: the inflow flux divided by the fluid outflow area (reading: the mean speed
    through the outflow face, fixed by the geometry)."""
    if grid.stretched:                    # face areas differ from row to row: weigh by them
        A = grid.cell_heights()[..., :1]
        a_in = float(np.sum(np.where(cls.inflow_fluid, A, 0.0)))
        a_out = float(np.sum(np.where(cls.outflow_fluid, A, 0.0)))
        return grid.inflow[0] * a_in / a_out if a_out else 0.0
    n_in = int(np.count_nonzero(cls.inflow_fluid))
    n_out = int(np.count_nonzero(cls.outflow_fluid))
    return grid.inflow[0] * n_in / n_out if n_out else 0.0


def outflow_update(grid, cls, u_prev, N_prev_b, k: int, dt: float, a, b):
    """RK3 stage k of du/dt = -U_c (u_b - u_{b-1}) / dx on the fluid outflow faces
    (u_b = u(n_x-1), u_{b-1} = u(n_x-2) read as the operators read it); the same
    low-storage combination as the momentum stage, with no pressure and no IBM term.
    Returns u*_b and N_b, each of shape (nz, ny, 1); zero on solid outflow faces."""
    Uc = outflow_speed(grid, cls)
    ub = u_prev[0][..., -1:]
    um = np.where(cls.internal[0][..., -2:-1], u_prev[0][..., -2:-1], 0.0)
    Nb = -Uc * (ub - um) / grid.d[0]
    R = dt * a[k] * Nb + dt * b[k] * N_prev_b
    return np.where(cls.outflow_fluid, ub + R, 0.0), np.where(cls.outflow_fluid, Nb, 0.0)


def outflow_balance(grid, cls, ub):
    """Shift the fluid outflow face velocities by one constant so that the outflow flux
    equals the inflow flux (reading; the Poisson problem with prescribed normal velocity
    on every box face is solvable only then)."""
    if grid.stretched:                    # the fluxes through faces of unequal area
        A = grid.cell_heights()[..., :1]
        a_in = float(np.sum(np.where(cls.inflow_fluid, A, 0.0)))
        a_out = float(np.sum(np.where(cls.outflow_fluid, A, 0.0)))
        if a_out == 0.0:
            return ub
        shift = (grid.inflow[0] * a_in - np.sum(np.where(cls.outflow_fluid, ub * A, 0.0))) / a_out
        return np.where(cls.outflow_fluid, ub + shift, 0.0)
    n_in = int(np.count_nonzero(cls.inflow_fluid))
    n_out = int(np.count_nonzero(cls.outflow_fluid))
    if n_out == 0:
        return ub
    shift = (grid.inflow[0] * n_in - np.sum(np.where(cls.outflow_fluid, ub, 0.0))) / n_out
    return np.where(cls.outflow_fluid, ub + shift, 0.0)
