"""The full oracle time step: RK3 + implicit IBM predictor, projection after every substage.

Order per substage k (paper Sec. 2.1 and Eq. rk3-rai):
  1. N^{k-1} = RHS(u^{k-1})                               (momentum.rhs)
  2. u* from the implicit-IBM stage update                 (momentum.stage_update)
  3. constant flow rate only: uniform forcing Pi on u      (reading below)
  4. phi: D G phi = D u* / (c_k Delta t)                   (poisson.solve_*)
  5. u^k = u* - c_k Delta t G phi,  p^k = p^{k-1} + phi

Projection: "fullbox" (the default) solves D G phi on the whole box and corrects every face
whose velocity is not prescribed; "masked" (poisson.solve_masked) solves D M G phi over the
internal cells and corrects only the internal faces, so the external faces keep u* = 0.

Constant flow rate is not described in the paper (its nose case imposes a
pressure drop, its channel keeps the flow rate).  Reading taken: a uniform
forcing Pi enters R as + c_k Delta t Pi on every internal u point, so it
raises u* there by Pi c_k Delta t / (B + x).  Pi is chosen so that the volume
integral of u* over the internal u points equals the target:
  Pi = (Q_target - Q(u*_0)) / S_k,  S_k = sum_internal c_k Delta t / (B + x) Delta V.
The projection keeps the box integral of u in a periodic x direction.

A translating body (reading R24; the paper, Sec. 3.1 end: apply the IBM in the frame in which
the body is at rest, i.e. subtract its velocity): a cylinder or sphere whose centre moves with
the constant velocity U_b.  At the start of every step the level set is placed at the step's
time, the points are classified again and the weights rebuilt with the wall velocity U_b (the
source s of the moving-wall extrapolation); points that became fluid take U_b.  Within the step
the body stays there.  The convective terms read the body's points as U_b, the Laplacian reads
them as zero (its wall term is -lambda w + s), and u* on the body's points is U_b.
A cylinder rotating about its own axis with the rate omega (the same reading) keeps its place:
its points hold omega x r, and each crossed arm's wall velocity is omega x r at the crossing.
"""
from __future__ import annotations

import numpy as np

from .grid import Grid
from .geometry import LevelSet, CYLINDER, SPHERE
from .classify import classify
from .weights import build_weights, B_of_x, RK3_A, RK3_B, RK3_C, RK3_T, B_EXPLICIT
from .momentum import (rhs, stage_update, pressure_gradient, masked, inflow_face, outflow_update,
                       outflow_balance)
from .poisson import divergence, gradient, solve_spectral, solve_direct, solve_masked
from .forces import body_terms, stage_impulse

FLOW_FORCED, FLOW_CONST_FLUX = 0, 1


class OracleSolver:
    def __init__(self, case, samples=None, no_ibm: bool = False, poisson: str = "spectral", projection=None):
        self.case = case
        self.grid = Grid(case)
        self.levelset = LevelSet(case.geom_kind, case.geom_params, samples)
        self.cls = classify(self.grid, self.levelset)
        self.nu = float(case.nu)
        self.dt = float(case.dt)
        self.g = tuple(float(v) for v in case.g)
        # time-periodic forcing (Sec. 2.5): g(t) = g + g_amp sin(2 pi g_freq t), evaluated at the
        # time of the stage's explicit right-hand side
        self.g_amp = tuple(float(v) for v in getattr(case, "g_amp", (0.0, 0.0, 0.0)))
        self.g_freq = float(getattr(case, "g_freq", 0.0))
        self.bmode = int(case.bmode)
        self.flow_mode = int(case.flow_mode)
        self.target_flux = float(case.target_flux)
        self.body_u = tuple(float(v) for v in getattr(case, "body_velocity", ()))
        self.moving = any(v != 0.0 for v in self.body_u)
        self.omega = float(getattr(case, "body_omega", 0.0))
        self.rotating = self.omega != 0.0
        self.no_ibm = no_ibm
        if (self.moving or self.rotating) and (case.geom_kind not in (CYLINDER, SPHERE) or self.grid.stretched):
            raise NotImplementedError("a translating or rotating cylinder or sphere on a uniform grid")
        if self.moving and self.rotating:
            raise NotImplementedError("a body that translates and rotates")
        if self.rotating and case.geom_kind != CYLINDER:
            raise NotImplementedError("rotation: a cylinder about its own axis")
        # the body's velocity at every point of each component (what its points hold)
        self.body_field = None
        wall_field = None
        if self.moving:
            self._place_body(0.0)
            self.body_field = list(self.body_u)
        if self.rotating:
            xc, yc = float(case.geom_params[0]), float(case.geom_params[1])
            om = self.omega
            x0, y0, _ = self.grid.coords(0)
            x1, y1, _ = self.grid.coords(1)
            self.body_field = [np.broadcast_to(-om * (y0 - yc), self.grid.shape).copy(),
                               np.broadcast_to(om * (x1 - xc), self.grid.shape).copy(), 0.0]
            wall_field = lambda X, c: (-om * (X[1] - yc), om * (X[0] - xc), 0.0)[c]   # omega x r at X
        self.w = build_weights(self.grid, self.levelset, self.cls, self.nu,
                               self.body_u if self.moving else case.wall_u, no_ibm=no_ibm, wall_field=wall_field)
        if self.grid.xflow and self.flow_mode == FLOW_CONST_FLUX:
            raise ValueError("a constant flow rate needs a periodic x direction")
        self.poisson = solve_spectral if poisson == "spectral" else solve_direct
        # "fullbox": the unmodified projection (D G of the whole box, every non-prescribed face
        # corrected); "masked": D M G over the internal cells, only internal faces corrected
        self.projection = projection or getattr(case, "projection", "fullbox")
        if self.projection not in ("fullbox", "masked"):
            raise ValueError("projection is 'fullbox' or 'masked'")
        z = np.zeros(self.grid.shape)
        self.u = [z.copy(), z.copy(), z.copy()]
        self.p = z.copy()
        self.Nprev = [z.copy(), z.copy(), z.copy()]
        self.step_count = 0
        self.last_pi = 0.0
        # force of the fluid on the body (forces.py): per step, and summed since the last read
        self.BN_prev = np.zeros(3)
        self.step_impulse = np.zeros(3)
        self.last_force = np.zeros(3)
        self.force_sum = np.zeros(3)
        self.force_steps = 0

    # ---- state --------------------------------------------------------------
    def _place_body(self, t: float):
        """Level set and classification with the body's centre moved by U_b t."""
        p = list(self.case.geom_params)
        for d in range(2 if self.case.geom_kind == CYLINDER else 3):
            p[d] = p[d] + self.body_u[d] * t
        self.levelset = LevelSet(self.case.geom_kind, tuple(p))
        self.cls = classify(self.grid, self.levelset)

    def _move_body(self):
        """Start of a step: the body at t_n, weights again, fresh fluid points set to U_b."""
        was = [a.copy() for a in self.cls.internal]
        self._place_body(self.step_count * self.dt)
        self.w = build_weights(self.grid, self.levelset, self.cls, self.nu, self.body_u, no_ibm=self.no_ibm)
        for c in range(self.grid.ncomp):
            fresh = self.cls.internal[c] & ~was[c]
            self.u[c] = np.where(fresh, self.body_u[c], self.u[c])

    def set_state(self, u, v, w, p):
        self.u = [np.array(u, dtype=np.float64), np.array(v, dtype=np.float64),
                  np.array(w, dtype=np.float64)]
        self.p = np.array(p, dtype=np.float64)

    def state(self):
        return [a.copy() for a in self.u], self.p.copy()

    # ---- one substage -------------------------------------------------------
    def substage(self, k: int, predictor_only: bool = False):
        g, cls = self.grid, self.cls
        t = (self.step_count + RK3_T[k]) * self.dt
        gk = tuple(self.g[c] + self.g_amp[c] * np.sin(2.0 * np.pi * self.g_freq * t) for c in range(3))
        N = rhs(g, cls, self.u, self.nu, gk, self.w.src, self.body_field)
        gp = pressure_gradient(g, self.p)
        um = masked(g, cls, self.u)
        lam = self.w.lam
        if self.bmode == B_EXPLICIT:
            # the classic explicit treatment: -lambda w in the right-hand side, no division
            N = [N[c] - np.where(cls.internal[c], lam[c] * um[c], 0.0) for c in range(3)]
            lam = [np.zeros(g.shape) for _ in range(3)]
        ustar = stage_update(g, cls, um, N, self.Nprev, gp, lam, k, self.dt,
                             self.bmode, RK3_A, RK3_B, RK3_C, B_of_x)
        if self.body_field is not None:      # the body's points move with it
            ustar = [np.where(cls.external[c], self.body_field[c], ustar[c]) if c < g.ncomp else ustar[c]
                     for c in range(3)]
        # the body's share of the stage: the IBM division's part I of u* - u (what the
        # explicit R does not explain) and the right-hand side's faces toward the solid
        R = [self.dt * (RK3_A[k] * N[c] + RK3_B[k] * self.Nprev[c]) - RK3_C[k] * self.dt * gp[c] for c in range(3)]
        I = [np.where(cls.internal[c], ustar[c] - um[c] - R[c], 0.0) for c in range(3)]
        # (the force accounting is written for the uniform grid; a stretched one reports NaN)
        BN = None if (g.stretched or self.body_field is not None) else body_terms(g, cls, self.u, self.w.src, self.nu,
                                                 self.w.lam if self.bmode == B_EXPLICIT else None)
        if g.xflow:
            # the outflow face: convective condition, then the flux balance
            ub, Nb = outflow_update(g, cls, self.u, self.Nprev[0][..., -1:], k, self.dt, RK3_A, RK3_B)
            ustar[0][..., -1:] = outflow_balance(g, cls, ub)
            N[0] = N[0].copy()
            N[0][..., -1:] = Nb
        self.Nprev = N
        if self.flow_mode == FLOW_CONST_FLUX:
            ckdt = RK3_C[k] * self.dt
            x = self.w.lam[0] * ckdt if self.bmode != B_EXPLICIT else np.zeros(g.shape)
            beta = np.where(cls.internal[0], 1.0 / (B_of_x(x, self.bmode) + x), 0.0)
            if g.stretched:
                dV = g.cell_volumes()
                Q0 = np.sum(np.where(cls.internal[0], ustar[0], 0.0) * dV)
                S = np.sum(ckdt * beta * dV)
            else:
                dV = g.cell_volume()
                Q0 = np.sum(np.where(cls.internal[0], ustar[0], 0.0)) * dV
                S = np.sum(ckdt * beta) * dV
            Pi = (self.target_flux - Q0) / S
            ustar[0] = ustar[0] + Pi * ckdt * beta
            self.last_pi = Pi
        if predictor_only:
            self.u = ustar
            return
        self._project(ustar, RK3_C[k] * self.dt, update_p=True)
        if g.stretched or self.body_field is not None:
            self.step_impulse = np.full(3, np.nan)
            return
        self.step_impulse = self.step_impulse + stage_impulse(g, cls, I, BN, self.BN_prev, self.p, k, self.dt,
                                                              RK3_A, RK3_B, RK3_C)
        self.BN_prev = BN

    def _project(self, ustar, ckdt: float, update_p: bool):
        g = self.grid
        r = divergence(g, ustar, inflow_face(g, self.cls) if g.xflow else None) / ckdt
        if self.projection == "masked":
            phi = solve_masked(g, self.cls, r)
            G = gradient(g, phi)
            self.u = [np.where(self.cls.internal[c], ustar[c] - ckdt * G[c], ustar[c]) for c in range(3)]
        else:
            phi = self.poisson(g, r)
            G = gradient(g, phi)
            self.u = [ustar[c] - ckdt * G[c] for c in range(3)]
        if update_p:
            self.p = self.p + phi
        self.last_phi = phi

    # ---- public -------------------------------------------------------------
    def step(self, nsteps: int = 1):
        for _ in range(nsteps):
            if self.moving:
                self._move_body()
            self.step_impulse = np.zeros(3)
            for k in range(3):
                self.substage(k)
            self.step_count += 1
            self.last_force = -self.step_impulse / self.dt
            self.force_sum = self.force_sum + self.last_force
            self.force_steps += 1

    def mean_force(self, reset: bool = True):
        """Mean force of the fluid on the body over the steps since the last reset."""
        f = self.force_sum / self.force_steps if self.force_steps else np.full(3, np.nan)
        if reset:
            self.force_sum = np.zeros(3)
            self.force_steps = 0
        return f

    def project(self):
        """Initial-condition projection: zero the unreadable velocities, balance the outflow
        (inflow/outflow x), then project (p unchanged)."""
        um = masked(self.grid, self.cls, self.u)
        if self.body_field is not None:      # a moving body's points hold its velocity
            um = [np.where(self.cls.external[c], self.body_field[c], um[c]) if c < self.grid.ncomp else um[c]
                  for c in range(3)]
        if self.grid.xflow:
            um[0] = um[0].copy()
            um[0][..., -1:] = outflow_balance(self.grid, self.cls, um[0][..., -1:])
        self._project(um, 1.0, update_p=False)

    def diagnostics(self) -> dict:
        g, cls = self.grid, self.cls
        div = divergence(g, self.u, inflow_face(g, cls) if g.xflow else None)
        dV = g.cell_volumes() if g.stretched else g.cell_volume()
        out = {"div_l2": float(np.sqrt(np.mean(div ** 2))), "div_linf": float(np.max(np.abs(div)))}
        cfl = 0.0
        flux = [0.0, 0.0, 0.0]
        ke = 0.0
        for c in range(g.ncomp):
            ui = np.where(cls.internal[c], self.u[c], 0.0)
            if g.stretched:
                # v moves between the cells on either side of its face: the smaller of the two
                sp_c = np.minimum(g.cell_heights(), g.ycol(np.concatenate((g.dyc[1:], g.dyc[-1:])))) \
                    if c == 1 else g.d[c]
                cfl += float(np.max(np.abs(ui) / sp_c))
                flux[c] = float(np.sum(ui * dV))
                ke += 0.5 * float(np.sum(ui * ui * dV))
            else:
                cfl += float(np.max(np.abs(ui))) / g.d[c]
                flux[c] = float(np.sum(ui)) * dV
                ke += 0.5 * float(np.sum(ui * ui)) * dV
        out["cfl"] = cfl * self.dt
        out["flux"] = flux
        out["ke"] = ke
        out["finite"] = bool(all(np.all(np.isfinite(a)) for a in self.u) and np.all(np.isfinite(self.p)))
        return out
