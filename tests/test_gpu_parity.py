"""GPU path (libibm.so through the C ABI) against the FP64 oracle.

Tolerances:
  * integer/byte work (mask, IBM-point lists): bit-exact;
  * FP64 fields: 1e-12 relative per step (max abs difference over the
    component's internal points divided by the oracle's max magnitude);
  * FP32 fields: the error against FP64 is stated as a number in the test.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

from inputs import (small_case, channel_c1, couette_case, wavy_c3, pipe_case, initial_field,  # noqa: E402
                    B_EULER, B_TAYLOR2, GEOM_NONE)
from oracle import OracleSolver, solve_spectral  # noqa: E402

CASES = ["channel2d", "wavy3d", "sphere3d", "cylinder2d", "cylinder2d_io", "sphere3d_io", "tubes3d_io"]
TOL64 = 1e-12


def _gpu(case, **kw):
    from paper_2506_14328_gb300.solver import Solver
    return Solver.from_case(case, **kw)


def _pair(case, no_ibm=False, precision=None):
    f = initial_field(case)
    g = _gpu(case, no_ibm=no_ibm, precision=precision)
    g.set_state(f["u"], f["v"], f["w"], f["p"])
    o = OracleSolver(case, no_ibm=no_ibm)
    o.set_state(f["u"], f["v"], f["w"], f["p"])
    return g, o


def _rel(o, got, ref, c):
    m = o.cls.internal[c]
    if not m.any():
        return 0.0
    scale = max(np.abs(ref[m]).max(), 1e-300)
    return float(np.abs(got[m] - ref[m]).max() / scale)


def _rel_p(o, got, ref):
    m = o.cls.p_internal
    return float(np.abs(got[m] - ref[m]).max() / max(np.abs(ref[m]).max(), 1e-300))


@pytest.mark.parametrize("name", CASES)
def test_classification_bit_exact(name):
    case = small_case(name)
    g = _gpu(case)
    mask, lists = g.classification()
    o = OracleSolver(case)
    assert np.array_equal(mask, o.cls.mask)
    for c in range(3):
        assert np.array_equal(lists[c], o.cls.lists[c])


def test_classification_pipe_3d_single_layer():
    case = pipe_case(N=41, nz=1)
    g = _gpu(case)
    mask, lists = g.classification()
    o = OracleSolver(case)
    assert np.array_equal(mask, o.cls.mask)
    assert all(np.array_equal(lists[c], o.cls.lists[c]) for c in range(3))


@pytest.mark.parametrize("name", CASES + ["couette"])
def test_weights_match_oracle(name):
    case = couette_case() if name == "couette" else small_case(name)
    g = _gpu(case)
    lam, src = g.weights_lists()
    o = OracleSolver(case)
    for c in range(3):
        ref = o.w.lam_list[c]
        assert lam[c].shape == ref.shape
        if ref.size:
            assert np.abs(lam[c] - ref).max() <= TOL64 * max(np.abs(ref).max(), 1.0)
            rs = o.w.src_list[c]
            assert np.abs(src[c] - rs).max() <= TOL64 * max(np.abs(rs).max(), 1.0)


@pytest.mark.parametrize("name", CASES)
def test_predictor_matches_oracle(name):
    case = small_case(name)
    g, o = _pair(case)
    g.step(1, flags=1)           # IBM_STEP_PREDICTOR_ONLY
    o.substage(0, predictor_only=True)
    ug, _ = g.state()
    for c in range(o.grid.ncomp):
        assert _rel(o, ug[c], o.u[c], c) < TOL64, c


@pytest.mark.parametrize("name", CASES)
def test_poisson_matches_oracle(name):
    case = small_case(name)
    g = _gpu(case)
    rng = np.random.default_rng(11)
    r = rng.standard_normal(g.shape)
    r -= r.mean()
    t = torch.tensor(r, dtype=torch.float64, device="cuda").contiguous()
    g.poisson(t)
    torch.cuda.synchronize()
    ref = solve_spectral(OracleSolver(case).grid, r)
    assert np.abs(t.cpu().numpy() - ref).max() < TOL64 * np.abs(ref).max()


@pytest.mark.parametrize("form", ["warp", "thread"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["wavy3d", "cylinder2d_io", "sphere3d_io", "channel2d"])
def test_poisson_tridiag_forms_match_oracle(name, precision, form):
    """Both forms of the FP64 sweeps (a warp or a thread per system) against the oracle's
    Poisson solve: 1e-12 in FP64; in FP32 mode (FP32 transforms, FP64 sweeps of the
    near-singular systems, FP32 sweeps of the dominant ones) within 2e-6 of the largest value."""
    case = small_case(name)
    g = _gpu(case, precision=precision)
    g.tridiag_form(form)
    rng = np.random.default_rng(12)
    r = rng.standard_normal(g.shape)
    r -= r.mean()
    dt = torch.float64 if precision == "fp64" else torch.float32
    t = torch.tensor(r, dtype=dt, device="cuda").contiguous()
    g.poisson(t)
    torch.cuda.synchronize()
    ref = solve_spectral(OracleSolver(case).grid, r.astype(np.float32).astype(np.float64)
                         if precision == "fp32" else r)
    tol = TOL64 if precision == "fp64" else 2e-6
    assert np.abs(t.cpu().numpy().astype(np.float64) - ref).max() < tol * np.abs(ref).max()


def test_integer_pipe_conversions_match_the_hardware_bit_for_bit():
    """The FP64 sweeps of FP32 fields widen and narrow with integer instructions; 2^24 bit
    patterns (random doubles, exact ties, random floats, the FP32 range ends) must convert
    exactly as the hardware conversions do."""
    from paper_2506_14328_gb300 import ibm_selftest_conversions
    assert ibm_selftest_conversions(1 << 24) == 0


@pytest.mark.parametrize("name", CASES)
def test_full_steps_match_oracle(name):
    case = small_case(name)
    g, o = _pair(case)
    for s in range(case.steps):
        g.step(1)
        o.step(1)
        ug, pg = g.state()
        for c in range(o.grid.ncomp):
            assert _rel(o, ug[c], o.u[c], c) < TOL64, (s, c)
        assert _rel_p(o, pg, o.p) < 1e-11, s


@pytest.mark.parametrize("inflow", [False, True])
def test_tma_form_without_ibm_points_matches_oracle(inflow):
    """A box with no body in the TMA form of the predictor (48 x 30 x 26, nx a multiple of 16): no
    IBM points, so no IBM division follows the predictor; periodic and inflow/outflow x, full steps
    against the oracle to 1e-12."""
    from inputs import GEOM_NONE
    case = small_case("sphere3d_io" if inflow else "sphere3d").with_(geom_kind=GEOM_NONE, geom_params=())
    g, o = _pair(case)
    assert g.tiles()[2]                       # the TMA form
    assert all(len(x) == 0 for x in g.classification()[1])
    for s in range(case.steps):
        g.step(1)
        o.step(1)
        ug, pg = g.state()
        for c in range(3):
            assert _rel(o, ug[c], o.u[c], c) < TOL64, (s, c)
        assert _rel_p(o, pg, o.p) < 1e-11, s
    g.close()


def test_project_matches_oracle():
    case = small_case("sphere3d")
    g, o = _pair(case)
    g.project()
    o.project()
    ug, _ = g.state()
    for c in range(3):
        assert _rel(o, ug[c], o.u[c], c) < TOL64
    d = g.diagnostics()
    assert d["div_linf"] < 1e-12 * max(np.abs(u).max() for u in ug) / min(o.grid.d)


@pytest.mark.parametrize("mode", [B_EULER, B_TAYLOR2])
def test_other_B_modes_match_oracle(mode):
    case = small_case("channel2d").with_(bmode=mode)
    g, o = _pair(case)
    g.step(2)
    o.step(2)
    ug, _ = g.state()
    for c in range(2):
        assert _rel(o, ug[c], o.u[c], c) < TOL64


def test_staircase_flag_matches_oracle():
    case = small_case("sphere3d")
    g, o = _pair(case, no_ibm=True)
    g.step(1)
    o.step(1)
    ug, _ = g.state()
    for c in range(3):
        assert _rel(o, ug[c], o.u[c], c) < TOL64


def test_diagnostics_match_oracle():
    case = small_case("wavy3d")
    g, o = _pair(case)
    g.step(1)
    o.step(1)
    dg = g.diagnostics()
    do = o.diagnostics()
    for k in ("cfl", "ke"):
        assert abs(dg[k] - do[k]) <= 1e-12 * abs(do[k])
    for c in range(3):
        assert abs(dg["flux"][c] - do["flux"][c]) <= 1e-12 * max(abs(do["flux"][0]), 1.0)
    assert abs(dg["div_linf"]) < 1e-9 and abs(do["div_linf"]) < 1e-9
    assert abs(dg["pi"] - o.last_pi) <= 1e-10 * max(1.0, abs(o.last_pi))


def test_couette_fixed_point_on_gpu():
    case = couette_case()
    f = initial_field(case)
    g = _gpu(case)
    g.set_state(f["u"], f["v"], f["w"], f["p"])
    o = OracleSolver(case)
    u0 = np.where(o.cls.internal[0], f["u"], 0.0)
    g.step(5)
    ug, _ = g.state()
    u1 = np.where(o.cls.internal[0], ug[0], 0.0)
    assert np.abs(u1 - u0).max() < 1e-13


def test_channel_c1_2000_steps_matches_oracle_and_parabola():
    case = channel_c1(steps=2000)
    g, o = _pair(case)
    g.step(case.steps, flags=2)   # graph replay
    o.step(case.steps)
    ug, _ = g.state()
    assert _rel(o, ug[0], o.u[0], 0) < TOL64
    y = o.grid.coords(0)[1]
    exact = np.broadcast_to(1.0 - ((y - 0.499) / 0.362) ** 2, o.grid.shape)
    m = o.cls.internal[0]
    assert np.abs(ug[0] - exact)[m].max() < 5e-3


def test_graph_replay_equals_stream_launches():
    case = small_case("wavy3d")
    g1, _ = _pair(case)
    g2, _ = _pair(case)
    g1.step(3)
    g2.step(3, flags=2)
    a, pa = g1.state()
    b, pb = g2.state()
    for c in range(3):
        assert np.array_equal(a[c], b[c])
    assert np.array_equal(pa, pb)


def test_checkpoint_resume_is_bitwise():
    case = small_case("sphere3d")
    g1, _ = _pair(case)
    g1.step(2)
    snap = np.empty(g1.state_bytes(), dtype=np.uint8)
    g1.export_state(snap)
    g1.step(2)
    a, pa = g1.state()
    g2 = _gpu(case)
    g2.import_state(snap)
    g2.step(2)
    b, pb = g2.state()
    for c in range(3):
        assert np.array_equal(a[c], b[c])
    assert np.array_equal(pa, pb)
    assert g2.diagnostics()["step"] == 4


@pytest.mark.parametrize("name", ["channel2d", "wavy3d", "sphere3d", "cylinder2d_io", "sphere3d_io", "tubes3d_io"])
def test_fp32_error_against_fp64(name):
    """FP32 momentum / FP32 FFT / FP64 tridiagonal against the FP64 path after the case's steps."""
    case = small_case(name)
    g64, _ = _pair(case, precision="fp64")
    g32, o = _pair(case, precision="fp32")
    g64.step(case.steps)
    g32.step(case.steps)
    a, _ = g64.state()
    b, _ = g32.state()
    err = max(_rel(o, b[c], a[c], c) for c in range(o.grid.ncomp))
    assert err < 2e-5, err


def test_fp32_laminar_steady_state_within_1e5():
    """FP32 steady laminar channel against FP64: <= 1e-5 relative (C1 physics, 2000 steps)."""
    case = channel_c1(steps=2000)
    g64, o = _pair(case, precision="fp64")
    g32, _ = _pair(case, precision="fp32")
    g64.step(case.steps, flags=2)
    g32.step(case.steps, flags=2)
    a, _ = g64.state()
    b, _ = g32.state()
    assert _rel(o, b[0], a[0], 0) <= 1e-5


def test_diverged_status_on_nonfinite_field():
    from paper_2506_14328_gb300 import IBM_E_DIVERGED
    case = small_case("channel2d")
    g, _ = _pair(case)
    g.u[0][0, 5, 7] = float("nan")
    torch.cuda.synchronize()
    d = g.diagnostics(raise_on_diverged=False)
    assert d["status"] == IBM_E_DIVERGED
    g.u[0][0, 5, 7] = 0.0
    torch.cuda.synchronize()
    assert g.diagnostics()["status"] == 0


def test_no_body_box_projection_divergence_free():
    case = small_case("wavy3d").with_(geom_kind=GEOM_NONE, geom_params=(), flow_mode=0)
    g, o = _pair(case)
    g.project()
    assert g.diagnostics()["div_linf"] < 1e-12 * 2.0 / min(o.grid.d)


def test_full_size_wavy_channel_launch_configuration():
    """384x256x256 in the bench's launch configuration: bit-exact classification against the
    oracle at full size, and the properties every step must keep (flux at target, divergence
    at FP32 round-off, finite fields)."""
    case = wavy_c3(precision="fp32", steps=2)
    f = initial_field(case)
    g = _gpu(case)
    mask, lists = g.classification()
    from oracle import Grid, LevelSet, classify
    cls = classify(Grid(case), LevelSet(case.geom_kind, case.geom_params))
    mism = int((mask != cls.mask).sum())
    assert mism == 0, mism
    for c in range(3):
        assert np.array_equal(lists[c], cls.lists[c])
    g.set_state(f["u"], f["v"], f["w"], f["p"])
    g.project()
    g.step(2)
    d = g.diagnostics()
    assert d["status"] == 0
    umax = 3.0
    assert d["div_linf"] < 1e-4 * umax / (2.0 / 256)
    assert abs(g.diagnostics()["pi"]) < 1e3


@pytest.mark.parametrize("nx", [70, 64])
@pytest.mark.parametrize("flow", ["forced", "const_flux", "inflow"])
def test_predictor_every_z_chunk_matches_oracle(flow, nx):
    """The momentum predictor at every z-chunk the autotuner may pick and at lengths
    between them, on a grid whose z extent (23) leaves odd and short chunks, against the
    oracle to 1e-12.  nx = 64 runs
    the TMA form (x a multiple of 16), nx = 70 the register form.  With a forced flow or an
    inflow/outflow x, u* is also the same bit for bit at every chunk; under the constant
    flow rate the forcing sums per-block partials, whose grouping follows the chunking."""
    from inputs import FLOW_FORCED
    if flow == "inflow":
        case = small_case("sphere3d_io").with_(n=(nx, 36, 23), name=f"sphere3d_io_{nx}x36x23")
    else:
        case = small_case("wavy3d").with_(n=(nx, 36, 23), name=f"wavy3d_{nx}x36x23")
    if flow == "forced":
        case = case.with_(flow_mode=FLOW_FORCED, g=(0.3, 0.0, 0.0))
    o = OracleSolver(case)
    f = initial_field(case)
    o.set_state(f["u"], f["v"], f["w"], f["p"])
    o.substage(0, predictor_only=True)
    first = None
    for kz in (8, 9, 11, 12, 13, 14, 16, 24, 32, 48, 64, 86):
        g = _gpu(case)
        g.set_state(f["u"], f["v"], f["w"], f["p"])
        g.set_tiles(kz, 16)
        assert g.tiles() == (kz, 16, nx % 16 == 0)
        g.step(1, flags=1)
        ug, _ = g.state()
        for c in range(3):
            assert _rel(o, ug[c], o.u[c], c) < TOL64, (kz, c)
        if first is None:
            first = ug
        elif flow != "const_flux":
            for c in range(3):
                assert np.array_equal(first[c], ug[c]), (kz, c, int((first[c] != ug[c]).sum()))
        g.close()


@pytest.mark.parametrize("name", ["sphere3d", "sphere3d_io", "tubes3d_io"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tma_and_register_momentum_forms_agree(precision, name):
    """Both forms of the momentum predictor on grids with x a multiple of 16 (48 x 30 x 26:
    a half-empty x tile, a partial y tile, free-slip ghosts; with inflow / outflow x the
    ghost columns and the outflow face; the tube union), over full steps: FP64 to 1e-12
    of each other, FP32 to 1e-5."""
    case = small_case(name, precision=precision)
    f = initial_field(case)
    runs = []
    for tma in (True, False):
        g = _gpu(case)
        g.use_tma(tma)
        assert g.tiles()[2] == tma
        g.set_state(f["u"], f["v"], f["w"], f["p"])
        g.step(case.steps)
        runs.append(g.state())
        g.close()
    o = OracleSolver(case)
    tol = TOL64 if precision == "fp64" else 1e-5
    for c in range(3):
        assert _rel(o, runs[0][0][c], runs[1][0][c], c) < tol, c


@pytest.mark.parametrize("name", ["cylinder2d_io", "sphere3d_io", "tubes3d_io"])
def test_inflow_outflow_faces_and_balance_match_oracle(name):
    """Inflow / convective outflow: the outflow face values (boundary points the parity helper
    skips) match the oracle to 1e-12 after full steps, their flux equals the inflow flux, and
    the divergence with the inflow face is round-off."""
    case = small_case(name)
    g, o = _pair(case)
    g.project()
    o.project()
    for _ in range(case.steps):
        g.step(1)
        o.step(1)
    ug, _ = g.state()
    fl = o.cls.outflow_fluid[..., 0]
    ref = o.u[0][..., -1]
    got = ug[0][..., -1]
    assert np.abs(got[fl] - ref[fl]).max() <= TOL64 * np.abs(ref[fl]).max()
    assert np.all(got[~fl] == 0.0)
    q_in = case.inflow[0] * np.count_nonzero(o.cls.inflow_fluid)
    assert abs(got[fl].sum() - q_in) < 1e-12 * q_in
    d = g.diagnostics()
    assert d["div_linf"] < 1e-11 * case.inflow[0] / min(o.grid.d[:o.grid.ndim])


@pytest.mark.parametrize("name", CASES + ["couette"])
def test_body_force_matches_oracle(name):
    """The force of the fluid on the body (IBM division, faces toward solid points, pressure
    at run ends) per step and as the mean over several steps, FP64 against the oracle.  It is
    a sum of terms that cancel in part, so the tolerance is 1e-10 of the larger of the force
    and the wall shear scale."""
    case = couette_case() if name == "couette" else small_case(name)
    f = initial_field(case)
    g = _gpu(case, body_force=True)
    g.set_state(f["u"], f["v"], f["w"], f["p"])
    o = OracleSolver(case)
    o.set_state(f["u"], f["v"], f["w"], f["p"])
    nc = o.grid.ncomp
    for _ in range(2):
        g.step(1)
        o.step(1)
        d = g.diagnostics()
        assert d["force_steps"] == 1
        ref = o.last_force[:nc]
        scale = max(np.abs(ref).max(), case.nu * 1.0)
        assert np.abs(np.array(d["force"][:nc]) - ref).max() < 1e-10 * scale, (d["force"], ref)
    o.mean_force(reset=True)
    g.step(3)
    o.step(3)
    d = g.diagnostics()
    ref = o.mean_force()[:nc]
    assert d["force_steps"] == 3
    assert np.abs(np.array(d["force"][:nc]) - ref).max() < 1e-10 * max(np.abs(ref).max(), case.nu)
    assert g.diagnostics()["force_steps"] == 0     # the read resets the sums
    g.close()


def test_body_force_off_reports_nan_and_fp32_is_close():
    case = small_case("sphere3d_io")
    f = initial_field(case)
    g = _gpu(case)
    g.set_state(f["u"], f["v"], f["w"], f["p"])
    g.step(1)
    d = g.diagnostics()
    assert d["force_steps"] == 0 and all(math.isnan(v) for v in d["force"])
    g.close()
    g32 = _gpu(case, precision="fp32", body_force=True)
    g32.set_state(f["u"], f["v"], f["w"], f["p"])
    o = OracleSolver(case)
    o.set_state(f["u"], f["v"], f["w"], f["p"])
    g32.step(2)
    o.step(2)
    F32 = np.array(g32.diagnostics()["force"])
    F64 = o.mean_force()
    assert np.abs(F32 - F64).max() < 1e-3 * np.abs(F64).max()
    g32.close()


def _sphere_samples(case):
    """phi of the sphere (exact signed distance |X - C| - R) at the u, v, w points."""
    nx, ny, nz = case.n
    d = [case.L[a] / case.n[a] for a in range(3)]
    cx, cy, cz, R, sgn = case.geom_params
    out = []
    for c in range(3):
        ax = [case.origin[a] + (np.arange(case.n[a]) + (1.0 if a == c else 0.5)) * d[a] for a in range(3)]
        z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        out.append(-sgn * (np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) - R))
    return out


def test_sampled_geometry_matches_oracle():
    """A sampled level set (the sphere's distance at the velocity points) through the device
    path: classification bit-exact, weights (straight-line root of the samples) and two full
    steps to 1e-12."""
    from inputs import GEOM_SAMPLED
    base = small_case("sphere3d")
    samples = _sphere_samples(base)
    case = base.with_(geom_kind=GEOM_SAMPLED, geom_params=())
    f = initial_field(case)
    g = _gpu(case, samples=samples)
    o = OracleSolver(case, samples=samples)
    mask, lists = g.classification()
    assert np.array_equal(mask, o.cls.mask)
    for c in range(3):
        assert np.array_equal(lists[c], o.cls.lists[c])
    lam, _ = g.weights_lists()
    for c in range(3):
        ref = o.w.lam_list[c]
        assert np.abs(lam[c] - ref).max() <= TOL64 * np.abs(ref).max()
    g.set_state(f["u"], f["v"], f["w"], f["p"])
    o.set_state(f["u"], f["v"], f["w"], f["p"])
    for _ in range(2):
        g.step(1)
        o.step(1)
        ug, _ = g.state()
        for c in range(3):
            assert _rel(o, ug[c], o.u[c], c) < TOL64, c
    g.close()


@pytest.mark.parametrize("name", ["sphere3d", "cylinder2d", "cylinder2d_io", "wavy3d", "tubes3d_io"])
def test_masked_projection_matches_oracle(name):
    """The masked projection (D M G over the internal cells by preconditioned conjugate
    gradients, FP64, to a residual of 1e-11 of the right-hand side) against the oracle's sparse
    solve: the initial projection and full steps to 1e-9, external faces exactly zero."""
    case = small_case(name).with_(projection="masked")
    f = initial_field(case)
    g = _gpu(case)
    g.set_projection("masked", tol=1e-11, maxit=1000)
    o = OracleSolver(case)
    g.set_state(f["u"], f["v"], f["w"], f["p"])
    o.set_state(f["u"], f["v"], f["w"], f["p"])
    g.project()
    o.project()
    for s in range(case.steps + 1):
        if s:
            g.step(1)
            o.step(1)
        ug, _ = g.state()
        for c in range(o.grid.ncomp):
            assert _rel(o, ug[c], o.u[c], c) < 1e-9, (s, c)
            assert np.all(ug[c][o.cls.external[c]] == 0.0), (s, c)
    d = g.diagnostics()
    assert 0 < d["proj_iters"] < 1000 and d["proj_resid"] <= 1e-11
    g.close()


@pytest.mark.parametrize("variant", ["periodic_forcing", "explicit_ibm"])
def test_forcing_and_explicit_ibm_match_oracle(variant):
    """Time-periodic forcing at each stage's own time, and the explicit IBM treatment, over
    full steps against the oracle (1e-12)."""
    from inputs import B_EXPLICIT
    if variant == "periodic_forcing":
        case = small_case("sphere3d").with_(g_amp=(0.5, -0.2, 0.1), g_freq=3.0)
    else:
        case = small_case("channel2d").with_(bmode=B_EXPLICIT)
    g, o = _pair(case)
    for s in range(case.steps):
        g.step(1)
        o.step(1)
        assert all(np.all(np.isfinite(o.u[c])) for c in range(3))
        ug, _ = g.state()
        for c in range(o.grid.ncomp):
            assert _rel(o, ug[c], o.u[c], c) < TOL64, (s, c)


@pytest.mark.parametrize("name", ["wavy3d", "channel2d", "cylinder2d", "sphere3d"])
def test_wall_shear_matches_oracle(name):
    """tau(x) along the lower wall and its Fourier components after a full step, FP64, against
    the oracle (the same columns undefined, values to 1e-10 of the largest)."""
    from inputs import GEOM_SINE_WALL
    from oracle.forces import wall_shear
    case = small_case(name)
    g, o = _pair(case)
    g.step(1)
    o.step(1)
    lam = case.geom_params[2] if case.geom_kind == GEOM_SINE_WALL else case.L[0]
    tg, cg, sg = g.wall_shear(lam)
    to, co, so = wall_shear(o.grid, o.cls, o.levelset, o.u[0], case.nu, lam)
    assert np.array_equal(np.isnan(tg), np.isnan(to))
    ok = np.isfinite(to)
    assert ok.any()
    scale = np.abs(to[ok]).max()
    assert np.abs(tg[ok] - to[ok]).max() <= 1e-10 * scale
    assert abs(cg - co) <= 1e-10 * scale and abs(sg - so) <= 1e-10 * scale
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [(384, 24, 8), (512, 20, 6), (96, 50, 1), (1536, 12, 1)])
def test_own_row_fft_matches_cufft_and_oracle(n, precision):
    """The own x-row FFT (Stockham, radices 4, 2, 3) against cuFFT's R2C / C2R on the same grid,
    through the full Poisson solve, and against the oracle's spectral solve: FP64 to 1e-12, FP32
    to 2e-6 of the solution; inflow/outflow boxes (the DCT rows) with nz = 6 and nz = 1."""
    from inputs import GEOM_NONE, BC_INFLOW, BC_OUTFLOW
    nx, ny, nz = n
    base = small_case("sphere3d" if nz > 1 else "cylinder2d", precision=precision)
    case = base.with_(n=n, L=(nx / 64.0, ny / 64.0, max(nz, 1) / 64.0 if nz > 1 else 1.0), geom_kind=GEOM_NONE,
                      geom_params=())
    if nx == 512:
        case = case.with_(bc_lo=(BC_INFLOW,) + tuple(case.bc_lo[1:]), bc_hi=(BC_OUTFLOW,) + tuple(case.bc_hi[1:]),
                          inflow=(1.0, 0.0, 0.0), flow_mode=0, g=(0.0, 0.0, 0.0))
    g = _gpu(case, precision=precision)
    rng = np.random.default_rng(13)
    r = rng.standard_normal(g.shape)
    r -= r.mean()
    dt = torch.float64 if precision == "fp64" else torch.float32
    out = []
    for own in (True, False):
        assert g.use_own_fft(own) == own
        t = torch.tensor(r, dtype=dt, device="cuda").contiguous()
        g.poisson(t)
        torch.cuda.synchronize()
        out.append(t.cpu().numpy().astype(np.float64))
    ref = solve_spectral(OracleSolver(case).grid, r)
    tol = TOL64 if precision == "fp64" else 2e-6
    scale = np.abs(ref).max()
    assert np.abs(out[0] - ref).max() < tol * scale
    assert np.abs(out[1] - ref).max() < tol * scale
    assert np.abs(out[0] - out[1]).max() < tol * scale
    g.close()


@pytest.mark.parametrize("variant", ["wavy3d_flux", "sphere3d_forced", "cylinder2d_io", "tubes3d_io"])
def test_fused_divergence_fp32_rows_of_128_cells(variant):
    """FP32 fields with nx a multiple of 128 take the fused divergence's 16-byte row loads (four
    cells per lane, the flow-rate increment's IBM coefficients found by a prefix over the
    segment's lanes, pairs stored in the real or DCT order).  Over full steps against the FP64
    oracle within 2e-5 of the largest value (the FP32 mode's stated bound), and within 1e-5 of
    the unfused FP32 path (cuFFT rows, per-cell divergence)."""
    from inputs import FLOW_FORCED
    case = {
        "wavy3d_flux": small_case("wavy3d", precision="fp32").with_(n=(128, 36, 20), name="wavy3d_128x36x20"),
        "sphere3d_forced": small_case("sphere3d", precision="fp32").with_(n=(128, 30, 26), L=(4.2666, 1.0, 1.0)),
        "cylinder2d_io": small_case("cylinder2d_io", precision="fp32").with_(n=(256, 50, 1)),
        "tubes3d_io": small_case("tubes3d_io", precision="fp32").with_(n=(128, 48, 32)),
    }[variant]
    f = initial_field(case)
    o = OracleSolver(case.with_(precision="fp64"))
    o.set_state(f["u"], f["v"], f["w"], f["p"])
    runs = []
    for own in (True, False):
        g = _gpu(case)
        assert g.use_own_fft(own) == own
        g.set_state(f["u"], f["v"], f["w"], f["p"])
        g.step(case.steps)
        runs.append(g.state()[0])
        g.close()
    o.step(case.steps)
    for c in range(o.grid.ncomp):
        assert _rel(o, runs[0][c], o.u[c], c) < 2e-5, c
        assert _rel(o, runs[0][c], runs[1][c], c) < 1e-5, c


@pytest.mark.parametrize("variant", ["wavy3d_flux", "cylinder2d_flux", "sphere3d_forced", "channel2d_forced",
                                     "cylinder2d_io", "sphere3d_io", "tubes3d_io"])
def test_fused_divergence_and_row_transform_match_oracle(variant):
    """The divergence fused with the own transform of the x rows (periodic x, rows whose half
    length has a factor 3): 3D and 2D, with and without the constant-flow-rate increment, over
    full steps against the oracle (1e-12); the unfused path (cuFFT rows) agrees as well.  The
    inflow/outflow boxes fuse it with the DCT of the rows instead (inflow face as the left
    neighbour of the first cell)."""
    from inputs import FLOW_FORCED
    case = {
        "wavy3d_flux": small_case("wavy3d").with_(n=(96, 36, 20), name="wavy3d_96x36x20"),
        "cylinder2d_flux": small_case("cylinder2d"),
        "sphere3d_forced": small_case("sphere3d"),
        "channel2d_forced": small_case("channel2d").with_(n=(96, 32, 1), flow_mode=FLOW_FORCED, g=(0.5, 0.0, 0.0)),
        "cylinder2d_io": small_case("cylinder2d_io"),
        "sphere3d_io": small_case("sphere3d_io"),
        "tubes3d_io": small_case("tubes3d_io"),
    }[variant]
    f = initial_field(case)
    o = OracleSolver(case)
    o.set_state(f["u"], f["v"], f["w"], f["p"])
    runs = []
    for own in (True, False):
        g = _gpu(case)
        assert g.use_own_fft(own) == own
        g.set_state(f["u"], f["v"], f["w"], f["p"])
        g.step(case.steps)
        runs.append(g.state()[0])
        g.close()
    o.step(case.steps)
    for c in range(o.grid.ncomp):
        assert _rel(o, runs[0][c], o.u[c], c) < TOL64, c
        assert _rel(o, runs[1][c], o.u[c], c) < TOL64, c
