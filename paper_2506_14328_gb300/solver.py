"""A solver object over the C ABI, with device memory from PyTorch.

PyTorch provides the device buffers (fields, workspace, weights) and the
stream; every computation is a call into libibm.so.  Host copies of the
fields are plain numpy arrays of shape (nz, ny, nx).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import (ibm_grid_desc, ibm_geom_desc, ibm_buffers, ibm_physics, IBM_FP64, IBM_FP32,
               ibm_workspace_bytes, ibm_setup_geometry, ibm_weights_bytes, ibm_weights_bytes_moving,
               ibm_build_weights, ibm_step,
               ibm_project, ibm_poisson, ibm_diagnostics, ibm_get_classification, ibm_get_weights,
               ibm_state_bytes, ibm_export_state, ibm_import_state, ibm_timing, ibm_get_timing,
               ibm_launch_count, ibm_autotune, ibm_set_tiles, ibm_get_tiles, ibm_set_momentum_tma, ibm_set_own_fft, ibm_set_tridiag_form,
               ibm_destroy, ibm_projection_bytes, ibm_set_projection, IBM_PROJ_FULLBOX, IBM_PROJ_MASKED,
               ibm_wall_shear)


class Solver:
    """One IBM solve resident on a CUDA device.

    Parameters mirror the C structs: ndim, n=(nx,ny,nz), L, origin, bc_lo,
    bc_hi, precision ('fp64'|'fp32'), geom_kind, geom_params, and physics
    nu, dt, g, bmode, flow_mode, target_flux, wall_u, no_ibm, body_force; inflow (x inflow/outflow);
    y_faces (a stretched wall-normal grid: the ny + 1 face heights)."""

    def __init__(self, *, ndim, n, L, origin, bc_lo, bc_hi, precision, geom_kind, geom_params, nu, dt,
                 g=(0.0, 0.0, 0.0), bmode=0, flow_mode=0, target_flux=0.0, wall_u=(0.0, 0.0, 0.0), no_ibm=False,
                 body_force=False, g_amp=(0.0, 0.0, 0.0), g_freq=0.0, inflow=(0.0, 0.0, 0.0), samples=None,
                 y_faces=(), body_u=(0.0, 0.0, 0.0), body_omega=0.0, device="cuda", stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("the IBM solver needs a CUDA device")
        self.device = torch.device(device)
        # a stream of its own: graph capture is not allowed on the legacy default stream
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self.ndim = int(ndim)
        self.n = tuple(int(v) for v in n)
        self.shape = (self.n[2], self.n[1], self.n[0])
        self.N = self.n[0] * self.n[1] * self.n[2]
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.np_dtype = np.float64 if precision == "fp64" else np.float32
        gd = ibm_grid_desc()
        gd.ndim = self.ndim
        for d in range(3):
            gd.n[d] = self.n[d]
            gd.L[d] = float(L[d])
            gd.origin[d] = float(origin[d])
            gd.bc_lo[d] = int(bc_lo[d])
            gd.bc_hi[d] = int(bc_hi[d])
        gd.precision = IBM_FP64 if precision == "fp64" else IBM_FP32
        for d in range(3):
            gd.inflow[d] = float(inflow[d])
        self.y_faces = np.ascontiguousarray(y_faces, dtype=np.float64) if len(y_faces) else None
        if self.y_faces is not None:
            if self.y_faces.shape != (self.n[1] + 1,):
                raise ValueError("y_faces: ny + 1 face heights")
            gd.y_faces = self.y_faces.ctypes.data_as(C.POINTER(C.c_double))
        self.grid = gd
        geo = ibm_geom_desc()
        geo.kind = int(geom_kind)
        if geo.kind == 5:      # IBM_GEOM_TUBES: the parameters are the tube data array
            self._geom_data = (C.c_double * len(geom_params))(*[float(v) for v in geom_params])
            geo.data = C.cast(self._geom_data, C.POINTER(C.c_double))
            geo.ndata = len(geom_params)
            geo.nparam = 0
        elif geo.kind == 6:    # IBM_GEOM_SAMPLED: phi of each component at its points, on the device
            if samples is None:
                raise ValueError("a sampled geometry needs samples: phi of u, v (and w) at their points")
            self._sdf = [torch.as_tensor(np.ascontiguousarray(samples[c], dtype=np.float64).reshape(self.shape),
                                         device=self.device) for c in range(3 if self.ndim == 3 else 2)]
            for c, t in enumerate(self._sdf):
                geo.sdf[c] = t.data_ptr()
            torch.cuda.synchronize(self.device)
        else:
            geo.nparam = len(geom_params)
            for q, v in enumerate(geom_params):
                geo.param[q] = float(v)
        self.geom = geo
        # every torch operation of this solver runs on its own stream, so setting up
        # one solve never waits for work that other solves have on the device
        with torch.cuda.device(self.device), torch.cuda.stream(self.stream):
            kw = dict(dtype=self.dtype, device=self.device)
            self.u = [torch.zeros(self.shape, **kw) for _ in range(3)]
            self.p = torch.zeros(self.shape, **kw)
            wb = ibm_workspace_bytes(gd)
            self.work = torch.empty(wb, dtype=torch.uint8, device=self.device)
            bufs = ibm_buffers()
            for c in range(3):
                bufs.u[c] = self.u[c].data_ptr()
            bufs.p = self.p.data_ptr()
            bufs.work = self.work.data_ptr()
            bufs.work_bytes = wb
            self.buffers = bufs
            self.stream.synchronize()
            self.h = ibm_setup_geometry(gd, geo, bufs, self.stream.cuda_stream)
            self.weights = None
            self.set_physics(nu=nu, dt=dt, g=g, bmode=bmode, flow_mode=flow_mode, target_flux=target_flux,
                             wall_u=wall_u, no_ibm=no_ibm, body_force=body_force, g_amp=g_amp, g_freq=g_freq,
                             body_u=body_u, body_omega=body_omega)

    @classmethod
    def from_case(cls, case, precision=None, no_ibm=False, **kw):
        """Build from any object with the attributes of a workload description.  A sampled
        geometry takes its samples through kw (samples=[phi_u, phi_v, phi_w]); a workload
        with projection 'masked' gets the masked projection."""
        s = cls(ndim=case.ndim, n=case.n, L=case.L, origin=case.origin, bc_lo=case.bc_lo, bc_hi=case.bc_hi,
                precision=precision or case.precision, geom_kind=case.geom_kind, geom_params=case.geom_params,
                nu=case.nu, dt=case.dt, g=case.g, bmode=case.bmode, flow_mode=case.flow_mode,
                target_flux=case.target_flux, wall_u=case.wall_u, no_ibm=no_ibm,
                inflow=getattr(case, "inflow", (0.0, 0.0, 0.0)), g_amp=getattr(case, "g_amp", (0.0, 0.0, 0.0)),
                g_freq=getattr(case, "g_freq", 0.0), y_faces=tuple(getattr(case, "y_faces", ())),
                body_u=tuple(getattr(case, "body_velocity", ())) or (0.0, 0.0, 0.0),
                body_omega=float(getattr(case, "body_omega", 0.0)), **kw)
        if getattr(case, "projection", "fullbox") == "masked":
            s.set_projection("masked")
        return s

    def set_physics(self, *, nu, dt, g=(0.0, 0.0, 0.0), bmode=0, flow_mode=0, target_flux=0.0,
                    wall_u=(0.0, 0.0, 0.0), no_ibm=False, body_force=False, g_amp=(0.0, 0.0, 0.0), g_freq=0.0,
                    body_u=(0.0, 0.0, 0.0), body_omega=0.0):
        ph = ibm_physics()
        ph.nu = float(nu)
        ph.dt = float(dt)
        for c in range(3):
            ph.g[c] = float(g[c])
            ph.wall_u[c] = float(wall_u[c])
        ph.bmode = int(bmode)
        ph.flow_mode = int(flow_mode)
        ph.target_flux = float(target_flux)
        ph.no_ibm = 1 if no_ibm else 0
        ph.body_force = 1 if body_force else 0
        for c in range(3):
            ph.g_amp[c] = float(g_amp[c])
        ph.g_freq = float(g_freq)
        bu = tuple(body_u) + (0.0,) * (3 - len(tuple(body_u)))
        for c in range(3):
            ph.body_u[c] = float(bu[c])
        ph.body_omega = float(body_omega)
        self.phys = ph
        # a translating body's IBM-point counts change as it crosses the grid: room to spare
        wb = ibm_weights_bytes_moving(self.h) if any(v != 0.0 for v in bu) else ibm_weights_bytes(self.h)
        if self.weights is None or self.weights.numel() < wb:
            with torch.cuda.stream(self.stream):
                self.weights = torch.empty(max(wb, 256), dtype=torch.uint8, device=self.device)
            self.stream.synchronize()
        ibm_build_weights(self.h, ph, self.weights.data_ptr(), self.weights.numel())

    def wall_shear(self, wavelength):
        """(tau(x) per u column, tau_1c, tau_1s) of the current velocity along the lower wall."""
        self.stream.synchronize()
        tau = np.empty(self.n[0])
        t1 = np.empty(2)
        ibm_wall_shear(self.h, wavelength, tau.ctypes.data, t1.ctypes.data)
        return tau, float(t1[0]), float(t1[1])

    def set_projection(self, mode="masked", tol=1e-10, maxit=500):
        """'fullbox' (the unmodified projection) or 'masked' (D M G over the internal cells,
        conjugate gradients in FP64 with a buffer of five fields held by this object)."""
        if mode == "fullbox":
            ibm_set_projection(self.h, IBM_PROJ_FULLBOX, 1.0, 1, 0, 0)
            self._proj_buf = None
            return
        if mode != "masked":
            raise ValueError("mode is 'fullbox' or 'masked'")
        nbytes = ibm_projection_bytes(self.h)
        with torch.cuda.stream(self.stream):
            self._proj_buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream.synchronize()
        ibm_set_projection(self.h, IBM_PROJ_MASKED, tol, maxit, self._proj_buf.data_ptr(), nbytes)

    # ---- calls -------------------------------------------------------------
    def step(self, nsteps=1, flags=0):
        ibm_step(self.h, nsteps, flags)

    def project(self):
        ibm_project(self.h)

    def poisson(self, rhs: torch.Tensor):
        assert rhs.dtype == self.dtype and rhs.is_contiguous() and rhs.numel() == self.N
        torch.cuda.synchronize(self.device)
        ibm_poisson(self.h, rhs.data_ptr())
        self.stream.synchronize()

    def diagnostics(self, raise_on_diverged=True) -> dict:
        d = ibm_diagnostics(self.h, raise_on_diverged)
        return {"div_l2": d.div_l2, "div_linf": d.div_linf, "cfl": d.cfl, "flux": list(d.flux), "ke": d.ke,
                "pi": d.pi, "step": d.step, "status": d.status, "force": list(d.force),
                "force_steps": d.force_steps, "proj_iters": d.proj_iters, "proj_resid": d.proj_resid}

    def classification(self):
        counts = ibm_get_classification(self.h, None, None)
        mask = np.empty(self.shape, dtype=np.uint8)
        lists = [np.empty(max(c, 1), dtype=np.int32) for c in counts]
        ibm_get_classification(self.h, mask.ctypes.data, [l.ctypes.data for l in lists])
        return mask, [lists[c][:counts[c]].astype(np.int64) for c in range(3)]

    def weights_lists(self):
        counts = ibm_get_classification(self.h, None, None)
        lam = [np.empty(max(c, 1)) for c in counts]
        src = [np.empty(max(c, 1)) for c in counts]
        ibm_get_weights(self.h, [a.ctypes.data for a in lam], [a.ctypes.data for a in src])
        return [lam[c][:counts[c]] for c in range(3)], [src[c][:counts[c]] for c in range(3)]

    def set_state(self, u, v, w, p):
        self.stream.synchronize()
        with torch.cuda.stream(self.stream):
            for t, a in zip(self.u + [self.p], (u, v, w, p)):
                t.copy_(torch.as_tensor(np.ascontiguousarray(a, dtype=self.np_dtype)).reshape(self.shape))
        self.stream.synchronize()

    def sync(self):
        self.stream.synchronize()

    def state(self):
        self.stream.synchronize()
        with torch.cuda.stream(self.stream):
            out = [t.detach().cpu().numpy().astype(np.float64) for t in self.u + [self.p]]
        return out[:3], out[3]

    def state_bytes(self) -> int:
        return ibm_state_bytes(self.h)

    def export_state(self, host: np.ndarray):
        ibm_export_state(self.h, host.ctypes.data, host.nbytes)

    def import_state(self, host: np.ndarray):
        ibm_import_state(self.h, host.ctypes.data, host.nbytes)

    def import_state_ptr(self, ptr: int, nbytes: int):
        ibm_import_state(self.h, ptr, nbytes)

    def autotune(self):
        """Pick the z-chunks of the momentum and march kernels by timing them (blocking)."""
        return ibm_autotune(self.h)

    def set_tiles(self, kz_momentum, kz_march):
        ibm_set_tiles(self.h, kz_momentum, kz_march)

    def tiles(self):
        """(kz_momentum, kz_march, momentum predictor runs its TMA form)"""
        return ibm_get_tiles(self.h)

    def use_tma(self, enable=True):
        ibm_set_momentum_tma(self.h, enable)

    def use_own_fft(self, enable=True) -> bool:
        """The own x-row FFT: True (wherever it can run), False (never) or "auto" (the
        default choice); returns whether it runs on this grid."""
        mode = 2 if enable == "auto" else (1 if enable else 0)
        return ibm_set_own_fft(self.h, mode)

    def tridiag_form(self, form="auto"):
        """FP64 tridiagonal sweeps: "auto", "warp" (one warp per system) or "thread"."""
        ibm_set_tridiag_form(self.h, {"auto": 0, "warp": 1, "thread": 2}[form])

    def footprint_bytes(self) -> int:
        return (sum(t.numel() * t.element_size() for t in self.u + [self.p]) + self.work.numel() +
                (self.weights.numel() if self.weights is not None else 0))

    def timing(self, enable=True):
        ibm_timing(self.h, enable)

    def get_timing(self) -> dict:
        return ibm_get_timing(self.h)

    def launch_count(self) -> int:
        return ibm_launch_count(self.h)

    def close(self):
        if getattr(self, "h", None):
            ibm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

