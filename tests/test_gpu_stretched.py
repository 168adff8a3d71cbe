"""The stretched wall-normal grid on the GPU (reading R23 of the paper's stretched channel
grids, Sec. 4.2 and Table wavy-parameters) against the FP64 oracle, through the C ABI.

Tolerances as in test_gpu_parity: classification and IBM lists bit-exact; FP64 fields 1e-12
relative per step (pressure 1e-11); FP32 mode's error against FP64 stated as a bound."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

from inputs import small_case, initial_field, tanh_faces, GEOM_SINE_WALL  # noqa: E402
from oracle import OracleSolver, solve_spectral  # noqa: E402

TOL64 = 1e-12
# (small case, tanh strength of the face map)
CASES = {"channel2d": 1.5, "wavy3d": 1.5, "cylinder2d_io": 1.4, "sphere3d": 1.2, "tubes3d_io": 1.3,
         "sphere3d_io": 1.6}


def _case(name, precision="fp64"):
    c = small_case(name, precision=precision)
    return c.with_(y_faces=tanh_faces(c.n[1], c.origin[1], c.L[1], CASES[name]), name=c.name + "_str")


def _gpu(case, **kw):
    from paper_2506_14328_gb300.solver import Solver
    return Solver.from_case(case, **kw)


def _pair(case, precision=None):
    f = initial_field(case)
    g = _gpu(case, precision=precision)
    g.set_state(f["u"], f["v"], f["w"], f["p"])
    o = OracleSolver(case)
    o.set_state(f["u"], f["v"], f["w"], f["p"])
    return g, o


def _rel(o, got, ref, c):
    m = o.cls.internal[c]
    if not m.any():
        return 0.0
    return float(np.abs(got[m] - ref[m]).max() / max(np.abs(ref[m]).max(), 1e-300))


@pytest.mark.parametrize("name", list(CASES))
def test_stretched_classification_bit_exact(name):
    case = _case(name)
    g = _gpu(case)
    mask, lists = g.classification()
    o = OracleSolver(case)
    assert np.array_equal(mask, o.cls.mask)
    for c in range(3):
        assert np.array_equal(lists[c], o.cls.lists[c])


@pytest.mark.parametrize("name", list(CASES))
def test_stretched_weights_match_oracle(name):
    case = _case(name)
    g = _gpu(case)
    lam, src = g.weights_lists()
    o = OracleSolver(case)
    for c in range(3):
        ref = o.w.lam_list[c]
        assert lam[c].shape == ref.shape
        if ref.size:
            assert np.abs(lam[c] - ref).max() <= TOL64 * max(np.abs(ref).max(), 1.0), c
            rs = o.w.src_list[c]
            assert np.abs(src[c] - rs).max() <= TOL64 * max(np.abs(rs).max(), 1.0), c


@pytest.mark.parametrize("name", list(CASES))
def test_stretched_predictor_matches_oracle(name):
    case = _case(name)
    g, o = _pair(case)
    g.step(1, flags=1)           # IBM_STEP_PREDICTOR_ONLY
    o.substage(0, predictor_only=True)
    ug, _ = g.state()
    for c in range(o.grid.ncomp):
        assert _rel(o, ug[c], o.u[c], c) < TOL64, c


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["channel2d", "wavy3d", "cylinder2d_io", "sphere3d_io"])
def test_stretched_poisson_matches_oracle(name, precision):
    """The symmetric unit off-diagonal form of the stretched rows, its per-row scalings and the
    zero-mode gauge against the oracle's direct Thomas solve of the same operator: 1e-12 in FP64,
    2e-6 of the largest value in FP32 mode."""
    case = _case(name)
    g = _gpu(case, precision=precision)
    rng = np.random.default_rng(13)
    r = rng.standard_normal(g.shape)
    r -= r.mean()
    dt = torch.float64 if precision == "fp64" else torch.float32
    t = torch.tensor(r, dtype=dt, device="cuda").contiguous()
    g.poisson(t)
    torch.cuda.synchronize()
    ref = solve_spectral(OracleSolver(case).grid,
                         r.astype(np.float32).astype(np.float64) if precision == "fp32" else r)
    tol = TOL64 if precision == "fp64" else 2e-6
    assert np.abs(t.cpu().numpy().astype(np.float64) - ref).max() < tol * np.abs(ref).max()


@pytest.mark.parametrize("name", list(CASES))
def test_stretched_full_steps_match_oracle(name):
    case = _case(name)
    g, o = _pair(case)
    for s in range(case.steps):
        g.step(1)
        o.step(1)
        ug, pg = g.state()
        for c in range(o.grid.ncomp):
            assert _rel(o, ug[c], o.u[c], c) < TOL64, (s, c)
        m = o.cls.p_internal
        assert np.abs(pg[m] - o.p[m]).max() < 1e-11 * max(np.abs(o.p[m]).max(), 1e-300), s


@pytest.mark.parametrize("name", ["wavy3d", "cylinder2d_io", "tubes3d_io"])
def test_stretched_diagnostics_match_oracle(name):
    case = _case(name)
    g, o = _pair(case)
    g.step(1)
    o.step(1)
    d, r = g.diagnostics(), o.diagnostics()
    for k in ("div_l2", "div_linf"):
        umax = max(np.abs(o.u[c]).max() for c in range(o.grid.ncomp))
        assert abs(d[k] - r[k]) <= 1e-12 * umax / o.grid.dyc.min(), k
    for k in ("cfl", "ke"):
        assert abs(d[k] - r[k]) <= TOL64 * abs(r[k]), k
    fs = max(abs(v) for v in r["flux"])
    for c in range(o.grid.ncomp):
        assert abs(d["flux"][c] - r["flux"][c]) <= TOL64 * fs, c


@pytest.mark.parametrize("name", ["channel2d", "wavy3d", "cylinder2d_io"])
def test_equal_faces_given_explicitly_match_the_uniform_path(name):
    """Equal face spacing passed as y_faces runs the stretched kernels; after the case's steps
    they agree with the uniform kernels to 1e-12 (the two paths round differently)."""
    base = small_case(name)
    ny = base.n[1]
    yf = tuple(base.origin[1] + np.arange(ny + 1) * base.L[1] / ny)
    f = initial_field(base)
    a = _gpu(base)
    b = _gpu(base.with_(y_faces=yf))
    for s in (a, b):
        s.set_state(f["u"], f["v"], f["w"], f["p"])
        s.step(base.steps)
    ua, _ = a.state()
    ub, _ = b.state()
    for c in range(base.ndim):
        scale = max(np.abs(ua[c]).max(), 1e-300)
        assert np.abs(ua[c] - ub[c]).max() <= 1e-12 * scale, c


@pytest.mark.parametrize("name", ["wavy3d", "channel2d"])
def test_stretched_wall_shear_matches_oracle(name):
    from oracle.forces import wall_shear
    case = _case(name)
    g, o = _pair(case)
    g.step(1)
    o.step(1)
    lam = case.geom_params[2] if case.geom_kind == GEOM_SINE_WALL else case.L[0]
    tg, cg, sg = g.wall_shear(lam)
    to, co, so = wall_shear(o.grid, o.cls, o.levelset, o.u[0], case.nu, lam)
    assert np.array_equal(np.isnan(tg), np.isnan(to))
    ok = np.isfinite(to)
    assert ok.any()
    sc = np.abs(to[ok]).max()
    assert np.abs(tg[ok] - to[ok]).max() <= 1e-10 * sc
    assert abs(cg - co) <= 1e-10 * sc and abs(sg - so) <= 1e-10 * sc


@pytest.mark.parametrize("name", ["channel2d", "wavy3d", "cylinder2d_io", "tubes3d_io"])
def test_stretched_fp32_error_against_fp64(name):
    """FP32 mode (FP32 momentum and transforms, FP64 sweeps of the near-singular systems) on
    the stretched grid against FP64 after the case's steps: below 2e-5 of the largest value."""
    case = _case(name)
    g64, _ = _pair(case, precision="fp64")
    g32, o = _pair(case, precision="fp32")
    g64.step(case.steps)
    g32.step(case.steps)
    a, _ = g64.state()
    b, _ = g32.state()
    err = max(_rel(o, b[c], a[c], c) for c in range(o.grid.ncomp))
    assert err < 2e-5, err


def test_stretched_grid_refuses_what_is_uniform_only():
    """The force accounting and the masked projection are written for a uniform y."""
    from paper_2506_14328_gb300 import IbmError
    case = _case("sphere3d")
    g = _gpu(case)
    with pytest.raises(IbmError, match="UNSUPPORTED"):
        g.set_projection("masked")
    with pytest.raises(IbmError, match="UNSUPPORTED"):
        g.set_physics(nu=case.nu, dt=case.dt, g=case.g, body_force=True)
