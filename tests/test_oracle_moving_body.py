"""Pins of the oracle's translating body (reading R24: the IBM applied in the frame in which the
body is at rest, Sec. 3.1 end).  No GPU.

A uniform stream moving with the body is an exact solution of the discrete equations: in the
body's frame nothing moves.  The convection of a uniform field is zero, the extrapolation through
the wall velocity returns the wall velocity, so -lambda w + s balances the missing neighbour, and
the implicit stage returns w.  It stays exact while the body crosses grid cells, which needs the
reclassification at every step, the fresh fluid points set to the body velocity, the source with
the body velocity, and the body's points read as the body velocity by the convective terms; a
mistake in any of them breaks it."""
import numpy as np
import pytest

from inputs import Case, BC_PERIODIC, BC_FREESLIP, GEOM_CYLINDER, GEOM_SPHERE
from oracle import OracleSolver


def _case(ndim, ub):
    if ndim == 2:
        return Case(name="mov2", ndim=2, n=(40, 24, 1), L=(2.0, 1.2, 1.0), origin=(0.0, 0.0, 0.0),
                    bc_lo=(BC_PERIODIC, BC_FREESLIP, BC_PERIODIC), bc_hi=(BC_PERIODIC, BC_FREESLIP, BC_PERIODIC),
                    geom_kind=GEOM_CYLINDER, geom_params=(0.71, 0.583, 0.27, -1.0), nu=0.02,
                    dt=0.37 * (2.0 / 40) / abs(ub[0]), body_velocity=ub)
    return Case(name="mov3", ndim=3, n=(24, 16, 20), L=(1.2, 0.8, 1.0), origin=(0.0, 0.0, 0.0),
                bc_lo=(BC_PERIODIC, BC_FREESLIP, BC_PERIODIC), bc_hi=(BC_PERIODIC, BC_FREESLIP, BC_PERIODIC),
                geom_kind=GEOM_SPHERE, geom_params=(0.43, 0.41, 0.37, 0.19, -1.0), nu=0.02,
                dt=0.41 * (1.2 / 24) / abs(ub[0]), body_velocity=ub)


@pytest.mark.parametrize("ndim,ub", [(2, (0.7, 0.0, 0.0)), (3, (0.5, 0.0, 0.3))])
def test_uniform_stream_moving_with_the_body_is_exact(ndim, ub):
    case = _case(ndim, ub)
    s = OracleSolver(case)
    g = s.grid
    u = [np.where(s.cls.internal[c], ub[c], 0.0) if c < g.ncomp else np.zeros(g.shape) for c in range(3)]
    s.set_state(u[0], u[1], u[2], np.zeros(g.shape))
    lists0 = [s.cls.lists[c].copy() for c in range(g.ncomp)]
    s.step(6)
    for c in range(g.ncomp):
        err = np.abs(np.where(s.cls.internal[c], s.u[c] - ub[c], 0.0)).max()
        assert err < 1e-12 * max(abs(v) for v in ub), (c, err)
    # the body crossed cells: the IBM points are not the same ones
    assert any(len(lists0[c]) != len(s.cls.lists[c]) or np.any(lists0[c] != s.cls.lists[c])
               for c in range(g.ncomp))
    assert np.abs(s.p - s.p.mean()).max() < 1e-10


def test_a_body_at_rest_is_not_a_fixed_point_of_the_moving_stream():
    """The same stream past the body held still is not steady (so the pin above has teeth)."""
    case = _case(2, (0.7, 0.0, 0.0))
    rest = case.with_(body_velocity=())
    s = OracleSolver(rest)
    g = s.grid
    u = np.where(s.cls.internal[0], 0.7, 0.0)
    s.set_state(u, np.zeros(g.shape), np.zeros(g.shape), np.zeros(g.shape))
    s.step(2)
    assert np.abs(np.where(s.cls.internal[0], s.u[0] - 0.7, 0.0)).max() > 1e-3


def _pipe(ndim, omega):
    n = (36, 36, 1) if ndim == 2 else (28, 28, 6)
    nu = 0.05
    return Case(name="rot", ndim=ndim, n=n, L=(1.0, 1.0, 1.0 if ndim == 2 else 0.3), origin=(0.0, 0.0, 0.0),
                bc_lo=(BC_PERIODIC, BC_FREESLIP, BC_PERIODIC), bc_hi=(BC_PERIODIC, BC_FREESLIP, BC_PERIODIC),
                geom_kind=GEOM_CYLINDER, geom_params=(0.493, 0.512, 0.37, 1.0), nu=nu,
                dt=0.2 * (1.0 / n[0]) ** 2 / nu, body_omega=omega, projection="masked")


def _rigid_rotation(s, omega):
    g = s.grid
    xc, yc = 0.493, 0.512
    x0, y0, _ = g.coords(0)
    x1, y1, _ = g.coords(1)
    xp, yp, _ = g.coords(3)
    u = np.where(s.cls.internal[0], -omega * (y0 - yc), 0.0)
    v = np.where(s.cls.internal[1], omega * (x1 - xc), 0.0)
    p = np.broadcast_to(0.5 * omega ** 2 * ((xp - xc) ** 2 + (yp - yc) ** 2), g.shape).copy()
    return u, v, p


@pytest.mark.parametrize("ndim", [2, 3])
def test_solid_body_rotation_in_a_rotating_pipe_is_exact(ndim):
    """Fluid turning with its pipe: the velocity is linear, so the flux form, the Laplacian and
    the extrapolation through the wall velocity omega x r (taken at each crossing point) are all
    exact, and the quadratic pressure balances the centripetal acceleration exactly: the
    rigid rotation is a fixed point of the whole step.  The masked projection (the internal
    cells only): the solid's rigid rotation reaches the box walls, where its normal velocity is
    not zero, so the full-box projection would see a divergence there."""
    om = 1.3
    s = OracleSolver(_pipe(ndim, om))
    g = s.grid
    u, v, p = _rigid_rotation(s, om)
    s.set_state(u, v, np.zeros(g.shape), p)
    s.step(3)
    scale = om * 0.37
    assert np.abs(np.where(s.cls.internal[0], s.u[0] - u, 0.0)).max() < 1e-12 * scale
    assert np.abs(np.where(s.cls.internal[1], s.u[1] - v, 0.0)).max() < 1e-12 * scale
    dp = np.where(s.cls.p_internal, s.p - p, 0.0)
    dp = dp - dp[s.cls.p_internal].mean()
    assert np.abs(np.where(s.cls.p_internal, dp, 0.0)).max() < 1e-11 * scale ** 2
    assert np.count_nonzero(s.w.src[0]) > 0 and np.count_nonzero(s.w.src[1]) > 0


def test_rigid_rotation_in_a_pipe_at_rest_is_not_steady():
    om = 1.3
    s = OracleSolver(_pipe(2, 0.0))
    u, v, p = _rigid_rotation(s, om)
    s.set_state(u, v, np.zeros(s.grid.shape), p)
    s.step(3)
    assert np.abs(np.where(s.cls.internal[0], s.u[0] - u, 0.0)).max() > 1e-4 * om * 0.37


def test_body_frame_form_of_the_wall_term_equals_the_moving_wall_source():
    """Reading the body's points as U_b in the Laplacian too adds nu d(s) U_b per crossed arm, so
    the source becomes lambda_arm U_b and the wall term -lambda (w - U_b): the same right-hand side
    at every internal point as the moving-wall extrapolation, for any field."""
    from dataclasses import replace
    from oracle.momentum import rhs
    ub = (0.7, 0.0, 0.3)
    case = _case(3, ub)
    s = OracleSolver(case)
    g, cls = s.grid, s.cls
    rng = np.random.default_rng(8)
    u = [np.where(cls.internal[c], rng.standard_normal(g.shape), 0.0) for c in range(3)]
    Na = rhs(g, cls, u, case.nu, (0.1, 0.0, 0.0), s.w.src, list(ub))
    readable = replace(cls, internal=[cls.internal[c] | cls.external[c] for c in range(3)])
    ub_field = [np.where(cls.external[c], ub[c], u[c]) for c in range(3)]
    Nb = rhs(g, readable, ub_field, case.nu, (0.1, 0.0, 0.0), [s.w.lam[c] * ub[c] for c in range(3)])
    for c in range(3):
        inside = cls.internal[c]
        scale = np.abs(Na[c][inside]).max()
        assert np.abs(Na[c] - Nb[c])[inside].max() < 1e-11 * scale, c
