"""ibm_diagnostics_noalloc: diagnostics for callers that must not allocate device memory.

Such callers (code whose device memory is owned entirely by another
allocator, or latency-critical loops that cannot pay for cudaMalloc) hold
device pointers to the fields but no workspace.  The entry point keeps its
scratch in a fixed array of the library's own device memory.  This file is
collected last so that, if it fails, a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

TOL = 1e-12   # the FP64 tolerance of the parity tests


def _close(a, b, scale):
    return abs(a - b) <= TOL * max(abs(scale), 1e-300)


def test_rejects_grids_above_the_limit_before_any_gpu_work():
    import paper_2506_14328_gb300 as P
    g = P.ibm_grid_desc()
    g.ndim = 3
    for d, n in enumerate((1024, 1024, 129)):      # 135,266,304 > 134,217,728 cells
        g.n[d] = n
        g.L[d] = 1.0
    g.bc_lo[1] = g.bc_hi[1] = P.IBM_BC_NOSLIP
    g.precision = P.IBM_FP32
    d = P.ibm_diag()
    st = P.lib.ibm_diagnostics_noalloc(ctypes.byref(g), ctypes.c_void_p(16), ctypes.c_void_p(16),
                                       ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), 1.0, None,
                                       ctypes.byref(d))
    assert st == P.IBM_E_INVALID
    assert "134217728" in P.ibm_last_error()


def test_rejects_sizes_whose_product_would_overflow():
    """Three extents near 2^31 multiply past 2^63; the limit check must still refuse them
    (it compares factor by factor) instead of letting a wrapped product through."""
    import paper_2506_14328_gb300 as P
    g = P.ibm_grid_desc()
    g.ndim = 3
    for d in range(3):
        g.n[d] = 2 ** 31 - 1
        g.L[d] = 1.0
    g.bc_lo[1] = g.bc_hi[1] = P.IBM_BC_NOSLIP
    g.precision = P.IBM_FP64
    d = P.ibm_diag()
    st = P.lib.ibm_diagnostics_noalloc(ctypes.byref(g), ctypes.c_void_p(16), ctypes.c_void_p(16),
                                       ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), 1.0, None,
                                       ctypes.byref(d))
    assert st == P.IBM_E_INVALID
    assert "134217728" in P.ibm_last_error()


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["wavy3d", "channel2d", "cylinder2d_io", "sphere3d_io"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_diagnostics_match_ibm_diagnostics_on_two_calls(precision, name):
    """Periodic and inflow/outflow x, 2D (no w: a NULL pointer) and 3D, both precisions."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from inputs import small_case, initial_field
    from paper_2506_14328_gb300 import ibm_diagnostics_noalloc
    from paper_2506_14328_gb300.solver import Solver

    case = small_case(name, precision=precision)
    s = Solver.from_case(case)
    f = initial_field(case)
    s.set_state(f["u"], f["v"], f["w"], f["p"])
    s.project()
    mask_host, _ = s.classification()
    mask = torch.from_numpy(mask_host).to(s.device).contiguous()
    torch.cuda.synchronize()
    for call in range(2):
        s.step(1)
        ref = s.diagnostics()
        w = s.u[2].data_ptr() if case.ndim == 3 else 0
        got = ibm_diagnostics_noalloc(s.grid, s.u[0].data_ptr(), s.u[1].data_ptr(), w,
                                      s.p.data_ptr(), mask.data_ptr(), case.dt, s.stream.cuda_stream)
        assert got.status == 0
        assert _close(got.div_l2, ref["div_l2"], ref["div_l2"]), call
        assert _close(got.div_linf, ref["div_linf"], ref["div_linf"]), call
        assert _close(got.cfl, ref["cfl"], ref["cfl"]), call
        assert _close(got.ke, ref["ke"], ref["ke"]), call
        for c in range(case.ndim):
            assert _close(got.flux[c], ref["flux"][c], max(abs(v) for v in ref["flux"])), (call, c)
    assert np.isfinite(got.ke)
