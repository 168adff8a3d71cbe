"""Moving bodies on the GPU (reading R24 of Sec. 3.1's remark that the IBM applies in the frame
in which the body is at rest) against the FP64 oracle, through the C ABI: a translating
cylinder or sphere (classified again every step, fresh fluid points set to the body velocity,
the wall term in its body-frame form -lambda (w - U_b)) and a cylinder rotating about its axis.

Tolerances: FP64 fields 1e-12 relative per step; the exact solutions of the oracle's pins
(tests/test_oracle_moving_body.py) hold to 1e-12 on the GPU as well."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

from inputs import Case, BC_PERIODIC, BC_FREESLIP, GEOM_CYLINDER, GEOM_SPHERE  # noqa: E402
from oracle import OracleSolver  # noqa: E402

TOL64 = 1e-12


def _moving(ndim, ub, precision="fp64"):
    if ndim == 2:
        return Case(name="mov2", ndim=2, n=(40, 24, 1), L=(2.0, 1.2, 1.0), origin=(0.0, 0.0, 0.0),
                    bc_lo=(BC_PERIODIC, BC_FREESLIP, BC_PERIODIC), bc_hi=(BC_PERIODIC, BC_FREESLIP, BC_PERIODIC),
                    geom_kind=GEOM_CYLINDER, geom_params=(0.71, 0.583, 0.27, -1.0), nu=0.02,
                    dt=0.37 * (2.0 / 40) / abs(ub[0]), body_velocity=ub, precision=precision)
    return Case(name="mov3", ndim=3, n=(24, 16, 20), L=(1.2, 0.8, 1.0), origin=(0.0, 0.0, 0.0),
                bc_lo=(BC_PERIODIC, BC_FREESLIP, BC_PERIODIC), bc_hi=(BC_PERIODIC, BC_FREESLIP, BC_PERIODIC),
                geom_kind=GEOM_SPHERE, geom_params=(0.43, 0.41, 0.37, 0.19, -1.0), nu=0.02,
                dt=0.41 * (1.2 / 24) / abs(ub[0]), body_velocity=ub, precision=precision)


def _pipe(ndim, omega, precision="fp64"):
    n = (36, 36, 1) if ndim == 2 else (28, 28, 6)
    nu = 0.05
    return Case(name="rot", ndim=ndim, n=n, L=(1.0, 1.0, 1.0 if ndim == 2 else 0.3), origin=(0.0, 0.0, 0.0),
                bc_lo=(BC_PERIODIC, BC_FREESLIP, BC_PERIODIC), bc_hi=(BC_PERIODIC, BC_FREESLIP, BC_PERIODIC),
                geom_kind=GEOM_CYLINDER, geom_params=(0.493, 0.512, 0.37, 1.0), nu=nu,
                dt=0.2 * (1.0 / n[0]) ** 2 / nu, body_omega=omega, projection="masked", precision=precision)


def _gpu(case, **kw):
    from paper_2506_14328_gb300.solver import Solver
    return Solver.from_case(case, **kw)


def _random_state(o, seed):
    g = o.grid
    rng = np.random.default_rng(seed)
    u = [np.where(o.cls.internal[c], 0.5 + 0.2 * rng.standard_normal(g.shape), 0.0) if c < g.ncomp
         else np.zeros(g.shape) for c in range(3)]
    return u, 0.1 * rng.standard_normal(g.shape)


@pytest.mark.parametrize("ndim,ub", [(2, (0.7, 0.0, 0.0)), (3, (0.5, 0.0, 0.3)), (2, (-0.6, 0.25, 0.0))])
def test_translating_body_matches_oracle_while_it_crosses_cells(ndim, ub):
    case = _moving(ndim, ub)
    o = OracleSolver(case)
    u, p = _random_state(o, 5)
    o.set_state(u[0], u[1], u[2], p)
    g = _gpu(case)
    g.set_state(u[0], u[1], u[2], p)
    lists0 = [o.cls.lists[c].copy() for c in range(o.grid.ncomp)]
    for s in range(6):
        g.step(1)
        o.step(1)
        ug, _ = g.state()
        for c in range(o.grid.ncomp):
            m = o.cls.internal[c]
            scale = np.abs(o.u[c][m]).max()
            assert np.abs(ug[c][m] - o.u[c][m]).max() < TOL64 * scale, (s, c)
        mask, lists = g.classification()
        assert np.array_equal(mask, o.cls.mask), s
        for c in range(o.grid.ncomp):
            assert np.array_equal(lists[c], o.cls.lists[c]), (s, c)
    assert any(len(lists0[c]) != len(o.cls.lists[c]) or np.any(lists0[c] != o.cls.lists[c])
               for c in range(o.grid.ncomp))


@pytest.mark.parametrize("ndim,ub", [(2, (0.7, 0.0, 0.0)), (3, (0.5, 0.0, 0.3))])
def test_uniform_stream_moving_with_the_body_stays_exact_on_the_gpu(ndim, ub):
    case = _moving(ndim, ub)
    g = _gpu(case)
    mask, _ = g.classification()
    nc = 3 if ndim == 3 else 2
    u = [np.where((mask >> c) & 1 == 1, ub[c], 0.0) if c < nc else np.zeros(g.shape) for c in range(3)]
    g.set_state(u[0], u[1], u[2], np.zeros(g.shape))
    g.step(6)
    ug, p = g.state()
    mask, _ = g.classification()
    for c in range(nc):
        inside = (mask >> c) & 1 == 1
        assert np.abs(ug[c][inside] - ub[c]).max() < TOL64 * max(abs(v) for v in ub), c
    assert np.abs(p - p.mean()).max() < 1e-10


@pytest.mark.parametrize("ndim", [2, 3])
def test_rotating_cylinder_matches_oracle_and_keeps_rigid_rotation(ndim):
    om = 1.3
    case = _pipe(ndim, om)
    o = OracleSolver(case)
    g = o.grid
    xc, yc = 0.493, 0.512
    x0, y0, _ = g.coords(0)
    x1, y1, _ = g.coords(1)
    xp, yp, _ = g.coords(3)
    u = np.where(o.cls.internal[0], -om * (y0 - yc), 0.0)
    v = np.where(o.cls.internal[1], om * (x1 - xc), 0.0)
    p = np.broadcast_to(0.5 * om ** 2 * ((xp - xc) ** 2 + (yp - yc) ** 2), g.shape).copy()
    gs = _gpu(case)
    gs.set_state(u, v, np.zeros(g.shape), p)
    gs.step(3)
    ug, _ = gs.state()
    scale = om * 0.37
    assert np.abs(np.where(o.cls.internal[0], ug[0] - u, 0.0)).max() < TOL64 * scale
    assert np.abs(np.where(o.cls.internal[1], ug[1] - v, 0.0)).max() < TOL64 * scale
    # a perturbed rotation against the oracle, step by step: 1e-9, the masked projection's
    # tolerance in the parity tests (conjugate gradients to 1e-10 here, 1e-14 in the oracle)
    rng = np.random.default_rng(9)
    du = [0.05 * scale * rng.standard_normal(g.shape) for _ in range(2)]
    u2 = np.where(o.cls.internal[0], u + du[0], 0.0)
    v2 = np.where(o.cls.internal[1], v + du[1], 0.0)
    o.set_state(u2, v2, np.zeros(g.shape), p)
    gs2 = _gpu(case)
    gs2.set_state(u2, v2, np.zeros(g.shape), p)
    for s in range(3):
        o.step(1)
        gs2.step(1)
        ug, _ = gs2.state()
        for c in range(2):
            m = o.cls.internal[c]
            assert np.abs(ug[c][m] - o.u[c][m]).max() < 1e-9 * np.abs(o.u[c][m]).max(), (s, c)


def test_translating_body_fp32_against_fp64():
    ub = (0.5, 0.0, 0.3)
    case = _moving(3, ub)
    o = OracleSolver(case)
    u, p = _random_state(o, 6)
    a = _gpu(case)
    b = _gpu(case, precision="fp32")
    for s in (a, b):
        s.set_state(u[0], u[1], u[2], p)
        s.step(4)
    ua, _ = a.state()
    ubb, _ = b.state()
    mask, _ = a.classification()
    for c in range(3):
        m = (mask >> c) & 1 == 1
        assert np.abs(ubb[c][m] - ua[c][m]).max() < 2e-5 * np.abs(ua[c][m]).max(), c


def test_moving_body_refusals():
    """Graph replay and batches need the same launches every step (a translating body is
    classified again), and the moving-body form needs a periodic x and the forced flow."""
    from paper_2506_14328_gb300 import IbmError
    case = _moving(2, (0.7, 0.0, 0.0))
    g = _gpu(case)
    with pytest.raises(IbmError, match="UNSUPPORTED"):
        g.step(1, flags=2)
    with pytest.raises(IbmError, match="UNSUPPORTED"):
        g.set_physics(nu=case.nu, dt=case.dt, body_u=(0.7, 0.0, 0.0), flow_mode=1, target_flux=1.0)
    with pytest.raises(IbmError, match="UNSUPPORTED"):
        g.set_physics(nu=case.nu, dt=case.dt, body_u=(0.7, 0.0, 0.0), body_omega=1.0)
