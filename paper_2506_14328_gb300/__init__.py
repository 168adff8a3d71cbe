"""Python binding of libibm.so (include/ibm.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method; all work runs in the CUDA library.  Importing this
package loads libibm.so and fails loudly when it has not been built (run
`__graft_entry__.build()`); there is no CPU fallback.

`solver.Solver` wraps the calls with device memory allocated by PyTorch.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libibm.so")

IBM_OK, IBM_E_INVALID, IBM_E_CUDA, IBM_E_NOMEM, IBM_E_UNSUPPORTED, IBM_E_DIVERGED, IBM_E_TIMEOUT, IBM_E_STATE = \
    0, -1, -2, -3, -4, -5, -6, -7
IBM_BC_PERIODIC, IBM_BC_NOSLIP, IBM_BC_FREESLIP, IBM_BC_INFLOW, IBM_BC_OUTFLOW = 0, 1, 2, 3, 4
IBM_FP64, IBM_FP32 = 0, 1
IBM_STEP_PREDICTOR_ONLY, IBM_STEP_GRAPH = 1, 2
IBM_PROJ_FULLBOX, IBM_PROJ_MASKED = 0, 1

STATUS_NAMES = {0: "IBM_OK", -1: "IBM_E_INVALID", -2: "IBM_E_CUDA", -3: "IBM_E_NOMEM", -4: "IBM_E_UNSUPPORTED",
                -5: "IBM_E_DIVERGED", -6: "IBM_E_TIMEOUT", -7: "IBM_E_STATE"}

# every symbol the header declares
EXPORTED = ("ibm_version", "ibm_last_error", "ibm_workspace_bytes", "ibm_setup_geometry", "ibm_weights_bytes", "ibm_weights_bytes_moving",
            "ibm_build_weights", "ibm_step", "ibm_project", "ibm_poisson", "ibm_projection_bytes",
            "ibm_set_projection", "ibm_wall_shear", "ibm_diagnostics",
            "ibm_get_classification", "ibm_get_weights", "ibm_state_bytes", "ibm_export_state",
            "ibm_import_state", "ibm_timing", "ibm_get_timing", "ibm_launch_count", "ibm_diagnostics_noalloc",
            "ibm_autotune", "ibm_set_tiles", "ibm_get_tiles", "ibm_set_momentum_tma", "ibm_set_own_fft", "ibm_set_tridiag_form", "ibm_selftest_conversions", "ibm_batch_create", "ibm_batch_set", "ibm_batch_run", "ibm_batch_jobs",
            "ibm_batch_destroy", "ibm_destroy")


class ibm_grid_desc(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 3), ("L", C.c_double * 3), ("origin", C.c_double * 3),
                ("bc_lo", C.c_int * 3), ("bc_hi", C.c_int * 3), ("precision", C.c_int),
                ("inflow", C.c_double * 3), ("y_faces", C.POINTER(C.c_double))]


class ibm_geom_desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("nparam", C.c_int), ("param", C.c_double * 32),
                ("data", C.POINTER(C.c_double)), ("ndata", C.c_int), ("sdf", C.c_void_p * 3)]


class ibm_buffers(C.Structure):
    _fields_ = [("u", C.c_void_p * 3), ("p", C.c_void_p), ("work", C.c_void_p), ("work_bytes", C.c_size_t)]


class ibm_physics(C.Structure):
    _fields_ = [("nu", C.c_double), ("dt", C.c_double), ("g", C.c_double * 3), ("bmode", C.c_int),
                ("flow_mode", C.c_int), ("target_flux", C.c_double), ("wall_u", C.c_double * 3),
                ("no_ibm", C.c_int), ("body_force", C.c_int), ("g_amp", C.c_double * 3), ("g_freq", C.c_double),
                ("body_u", C.c_double * 3), ("body_omega", C.c_double)]


class ibm_diag(C.Structure):
    _fields_ = [("div_l2", C.c_double), ("div_linf", C.c_double), ("cfl", C.c_double), ("flux", C.c_double * 3),
                ("ke", C.c_double), ("pi", C.c_double), ("step", C.c_longlong), ("status", C.c_int),
                ("force", C.c_double * 3), ("force_steps", C.c_longlong), ("proj_iters", C.c_int),
                ("proj_resid", C.c_double)]


class ibm_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char_p), ("launches", C.c_int), ("total_ms", C.c_double)]


class IbmError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(LIB_PATH)
    P = C.POINTER
    sig = {
        "ibm_version": ([], C.c_int),
        "ibm_last_error": ([], C.c_char_p),
        "ibm_workspace_bytes": ([P(ibm_grid_desc), P(C.c_size_t)], C.c_int),
        "ibm_setup_geometry": ([P(ibm_grid_desc), P(ibm_geom_desc), P(ibm_buffers), C.c_void_p, P(C.c_void_p)], C.c_int),
        "ibm_weights_bytes": ([C.c_void_p, P(C.c_size_t)], C.c_int),
        "ibm_weights_bytes_moving": ([C.c_void_p, P(C.c_size_t)], C.c_int),
        "ibm_build_weights": ([C.c_void_p, P(ibm_physics), C.c_void_p, C.c_size_t], C.c_int),
        "ibm_step": ([C.c_void_p, C.c_int, C.c_uint], C.c_int),
        "ibm_project": ([C.c_void_p], C.c_int),
        "ibm_poisson": ([C.c_void_p, C.c_void_p], C.c_int),
        "ibm_projection_bytes": ([C.c_void_p, P(C.c_size_t)], C.c_int),
        "ibm_wall_shear": ([C.c_void_p, C.c_double, C.c_void_p, C.c_void_p], C.c_int),
        "ibm_set_projection": ([C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_void_p, C.c_size_t], C.c_int),
        "ibm_diagnostics": ([C.c_void_p, P(ibm_diag)], C.c_int),
        "ibm_get_classification": ([C.c_void_p, C.c_void_p, P(C.c_void_p), P(C.c_int)], C.c_int),
        "ibm_get_weights": ([C.c_void_p, P(C.c_void_p), P(C.c_void_p)], C.c_int),
        "ibm_state_bytes": ([C.c_void_p, P(C.c_size_t)], C.c_int),
        "ibm_export_state": ([C.c_void_p, C.c_void_p, C.c_size_t], C.c_int),
        "ibm_import_state": ([C.c_void_p, C.c_void_p, C.c_size_t], C.c_int),
        "ibm_timing": ([C.c_void_p, C.c_int], C.c_int),
        "ibm_get_timing": ([C.c_void_p, P(ibm_kernel_time), C.c_int, P(C.c_int)], C.c_int),
        "ibm_launch_count": ([C.c_void_p, P(C.c_longlong)], C.c_int),
        "ibm_diagnostics_noalloc": ([P(ibm_grid_desc), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_double, C.c_void_p, P(ibm_diag)], C.c_int),
        "ibm_autotune": ([C.c_void_p, P(C.c_int), P(C.c_int)], C.c_int),
        "ibm_set_tiles": ([C.c_void_p, C.c_int, C.c_int], C.c_int),
        "ibm_get_tiles": ([C.c_void_p, P(C.c_int), P(C.c_int), P(C.c_int)], C.c_int),
        "ibm_set_momentum_tma": ([C.c_void_p, C.c_int], C.c_int),
        "ibm_set_own_fft": ([C.c_void_p, C.c_int, P(C.c_int)], C.c_int),
        "ibm_set_tridiag_form": ([C.c_void_p, C.c_int], C.c_int),
        "ibm_selftest_conversions": ([C.c_longlong, P(C.c_longlong)], C.c_int),
        "ibm_batch_create": ([C.c_void_p, P(C.c_void_p)], C.c_int),
        "ibm_batch_set": ([C.c_void_p, P(C.c_void_p), P(C.c_int), C.c_int], C.c_int),
        "ibm_batch_run": ([C.c_void_p], C.c_int),
        "ibm_batch_jobs": ([C.c_void_p, C.c_longlong], C.c_int),
        "ibm_batch_destroy": ([C.c_void_p], None),
        "ibm_destroy": ([C.c_void_p], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


lib = _load()


def _check(st: int, where: str):
    if st != IBM_OK:
        raise IbmError(st, where, lib.ibm_last_error().decode())


def ibm_version() -> int:
    return lib.ibm_version()


def ibm_last_error() -> str:
    return lib.ibm_last_error().decode()


def ibm_workspace_bytes(grid: ibm_grid_desc) -> int:
    b = C.c_size_t(0)
    _check(lib.ibm_workspace_bytes(C.byref(grid), C.byref(b)), "ibm_workspace_bytes")
    return b.value


def ibm_setup_geometry(grid: ibm_grid_desc, geom: ibm_geom_desc, buffers: ibm_buffers, stream: int) -> int:
    h = C.c_void_p(0)
    _check(lib.ibm_setup_geometry(C.byref(grid), C.byref(geom), C.byref(buffers), C.c_void_p(stream), C.byref(h)),
           "ibm_setup_geometry")
    return h.value


def ibm_weights_bytes(h: int) -> int:
    b = C.c_size_t(0)
    _check(lib.ibm_weights_bytes(C.c_void_p(h), C.byref(b)), "ibm_weights_bytes")
    return b.value


def ibm_weights_bytes_moving(h: int) -> int:
    b = C.c_size_t(0)
    _check(lib.ibm_weights_bytes_moving(C.c_void_p(h), C.byref(b)), "ibm_weights_bytes_moving")
    return b.value


def ibm_build_weights(h: int, phys: ibm_physics, weights_ptr: int, nbytes: int):
    _check(lib.ibm_build_weights(C.c_void_p(h), C.byref(phys), C.c_void_p(weights_ptr), nbytes), "ibm_build_weights")


def ibm_step(h: int, nsteps: int, flags: int = 0):
    _check(lib.ibm_step(C.c_void_p(h), nsteps, flags), "ibm_step")


def ibm_project(h: int):
    _check(lib.ibm_project(C.c_void_p(h)), "ibm_project")


def ibm_poisson(h: int, rhs_ptr: int):
    _check(lib.ibm_poisson(C.c_void_p(h), C.c_void_p(rhs_ptr)), "ibm_poisson")


def ibm_wall_shear(h: int, wavelength: float, tau_ptr: int, tau1_ptr: int):
    _check(lib.ibm_wall_shear(C.c_void_p(h), float(wavelength), C.c_void_p(tau_ptr), C.c_void_p(tau1_ptr)),
           "ibm_wall_shear")


def ibm_projection_bytes(h: int) -> int:
    b = C.c_size_t(0)
    _check(lib.ibm_projection_bytes(C.c_void_p(h), C.byref(b)), "ibm_projection_bytes")
    return b.value


def ibm_set_projection(h: int, mode: int, tol: float, maxit: int, buf_ptr: int, nbytes: int):
    _check(lib.ibm_set_projection(C.c_void_p(h), int(mode), float(tol), int(maxit), C.c_void_p(buf_ptr),
                                  C.c_size_t(nbytes)), "ibm_set_projection")


def ibm_diagnostics(h: int, raise_on_diverged: bool = True) -> ibm_diag:
    d = ibm_diag()
    st = lib.ibm_diagnostics(C.c_void_p(h), C.byref(d))
    if st != IBM_E_DIVERGED or raise_on_diverged:
        _check(st, "ibm_diagnostics")
    return d


def ibm_get_classification(h: int, mask_ptr: int | None, idx_ptrs) -> tuple:
    counts = (C.c_int * 3)()
    arr = None
    if idx_ptrs is not None:
        arr = (C.c_void_p * 3)(*[C.c_void_p(p) if p else None for p in idx_ptrs])
    _check(lib.ibm_get_classification(C.c_void_p(h), C.c_void_p(mask_ptr) if mask_ptr else None, arr, counts),
           "ibm_get_classification")
    return tuple(counts)


def ibm_get_weights(h: int, lam_ptrs, src_ptrs):
    la = (C.c_void_p * 3)(*[C.c_void_p(p) if p else None for p in lam_ptrs]) if lam_ptrs else None
    sa = (C.c_void_p * 3)(*[C.c_void_p(p) if p else None for p in src_ptrs]) if src_ptrs else None
    _check(lib.ibm_get_weights(C.c_void_p(h), la, sa), "ibm_get_weights")


def ibm_state_bytes(h: int) -> int:
    b = C.c_size_t(0)
    _check(lib.ibm_state_bytes(C.c_void_p(h), C.byref(b)), "ibm_state_bytes")
    return b.value


def ibm_export_state(h: int, host_ptr: int, nbytes: int):
    _check(lib.ibm_export_state(C.c_void_p(h), C.c_void_p(host_ptr), nbytes), "ibm_export_state")


def ibm_import_state(h: int, host_ptr: int, nbytes: int):
    _check(lib.ibm_import_state(C.c_void_p(h), C.c_void_p(host_ptr), nbytes), "ibm_import_state")


def ibm_timing(h: int, enable: bool):
    _check(lib.ibm_timing(C.c_void_p(h), 1 if enable else 0), "ibm_timing")


def ibm_get_timing(h: int) -> dict:
    out = (ibm_kernel_time * 32)()
    n = C.c_int(0)
    _check(lib.ibm_get_timing(C.c_void_p(h), out, 32, C.byref(n)), "ibm_get_timing")
    return {out[q].name.decode(): (out[q].launches, out[q].total_ms) for q in range(min(n.value, 32))}


def ibm_launch_count(h: int) -> int:
    n = C.c_longlong(0)
    _check(lib.ibm_launch_count(C.c_void_p(h), C.byref(n)), "ibm_launch_count")
    return n.value


def ibm_diagnostics_noalloc(grid: ibm_grid_desc, u: int, v: int, w: int, p: int, mask: int, dt: float,
                            stream: int, raise_on_diverged: bool = True) -> ibm_diag:
    """Diagnostics from device pointers alone, for callers that must not allocate device memory."""
    d = ibm_diag()
    st = lib.ibm_diagnostics_noalloc(C.byref(grid), C.c_void_p(u), C.c_void_p(v), C.c_void_p(w or None),
                                     C.c_void_p(p), C.c_void_p(mask), float(dt), C.c_void_p(stream), C.byref(d))
    if st != IBM_E_DIVERGED or raise_on_diverged:
        _check(st, "ibm_diagnostics_noalloc")
    return d


def ibm_autotune(h: int) -> tuple:
    a, b = C.c_int(0), C.c_int(0)
    _check(lib.ibm_autotune(C.c_void_p(h), C.byref(a), C.byref(b)), "ibm_autotune")
    return a.value, b.value


def ibm_set_tiles(h: int, kz_momentum: int, kz_march: int):
    _check(lib.ibm_set_tiles(C.c_void_p(h), kz_momentum, kz_march), "ibm_set_tiles")


def ibm_get_tiles(h: int) -> tuple:
    a, b, t = C.c_int(0), C.c_int(0), C.c_int(0)
    _check(lib.ibm_get_tiles(C.c_void_p(h), C.byref(a), C.byref(b), C.byref(t)), "ibm_get_tiles")
    return a.value, b.value, bool(t.value)


def ibm_set_momentum_tma(h: int, enable: bool):
    _check(lib.ibm_set_momentum_tma(C.c_void_p(h), 1 if enable else 0), "ibm_set_momentum_tma")


def ibm_set_own_fft(h: int, mode: int) -> bool:
    own = C.c_int(0)
    _check(lib.ibm_set_own_fft(C.c_void_p(h), int(mode), C.byref(own)), "ibm_set_own_fft")
    return bool(own.value)


def ibm_set_tridiag_form(h: int, form: int):
    _check(lib.ibm_set_tridiag_form(C.c_void_p(h), int(form)), "ibm_set_tridiag_form")


def ibm_selftest_conversions(n: int) -> int:
    bad = C.c_longlong(0)
    _check(lib.ibm_selftest_conversions(int(n), C.byref(bad)), "ibm_selftest_conversions")
    return bad.value


def ibm_batch_create(stream: int) -> int:
    b = C.c_void_p(0)
    _check(lib.ibm_batch_create(C.c_void_p(stream), C.byref(b)), "ibm_batch_create")
    return b.value


def ibm_batch_set(b: int, handles, steps):
    n = len(handles)
    hs = (C.c_void_p * max(n, 1))(*[C.c_void_p(h) for h in handles])
    st = (C.c_int * max(n, 1))(*[int(s) for s in steps])
    _check(lib.ibm_batch_set(C.c_void_p(b), hs, st, n), "ibm_batch_set")


def ibm_batch_run(b: int):
    _check(lib.ibm_batch_run(C.c_void_p(b)), "ibm_batch_run")


def ibm_batch_jobs(b: int, max_cells: int):
    _check(lib.ibm_batch_jobs(C.c_void_p(b), int(max_cells)), "ibm_batch_jobs")


def ibm_batch_destroy(b: int):
    lib.ibm_batch_destroy(C.c_void_p(b))


def ibm_destroy(h: int):
    lib.ibm_destroy(C.c_void_p(h))
