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
