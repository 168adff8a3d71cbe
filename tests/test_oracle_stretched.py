"""Pins of the oracle on a stretched wall-normal (y) grid (the paper's channel runs stretch the
wall-normal spacing, Sec. 4.2, Table wavy-parameters).  Each pin is fixed by the mathematics,
not by the oracle itself:
  * equal face spacing given explicitly reproduces the uniform grid (classification bit for
    bit, lambda and a full step to round-off);
  * the uneven three-point second difference is exact on quadratics;
  * linear extrapolation and the uneven second difference are exact on a linear profile, so
    plane Couette flow between off-grid IBM walls is a fixed point at any stretching;
  * the projection leaves a divergence-free field, is idempotent, and its D and G are
    adjoint in the cell and face volumes (discrete integration by parts);
  * the flux form telescopes: with no body and walls that take no flux, the u- and w-momentum
    sums over the cell volumes do not change by convection;
  * the steady channel between off-grid walls converges at second order under refinement at
    fixed stretching (first order without the IBM correction).
No GPU."""
import numpy as np
import pytest

from inputs import (Case, BC_PERIODIC, BC_NOSLIP, GEOM_PLANES, GEOM_NONE, small_case, initial_field,
                    couette_case, tanh_faces)
from oracle import OracleSolver, Grid, divergence, gradient, solve_spectral, solve_direct
from oracle import steady
from oracle.momentum import d2_y, y_face_value, rhs


def _faces(case, beta):
    return tanh_faces(case.n[1], case.origin[1], case.L[1], beta)


@pytest.mark.parametrize("name", ["channel2d", "wavy3d", "cylinder2d_io", "sphere3d", "tubes3d_io"])
def test_equal_faces_reproduce_the_uniform_grid(name):
    case = small_case(name)
    ny = case.n[1]
    yf = tuple(case.origin[1] + np.arange(ny + 1) * case.L[1] / ny)
    f = initial_field(case)
    a, b = OracleSolver(case), OracleSolver(case.with_(y_faces=yf))
    for c in range(3):
        assert np.array_equal(a.cls.internal[c], b.cls.internal[c])
        assert np.array_equal(a.cls.lists[c], b.cls.lists[c])
        # pointwise: a point very near the wall has a large lambda = O(1/delta), whose relative
        # round-off grows like ulp(y)/delta (the centres are formed differently)
        assert np.all(np.abs(a.w.lam[c] - b.w.lam[c]) <= 1e-9 * np.abs(a.w.lam[c]))
    for s in (a, b):
        s.set_state(f["u"], f["v"], f["w"], f["p"])
        s.step(1)
    for c in range(3):
        scale = max(np.abs(a.u[c]).max(), 1e-300)
        assert np.abs(a.u[c] - b.u[c]).max() <= 1e-12 * scale, c


def test_uneven_second_difference_is_exact_on_quadratics():
    rng = np.random.default_rng(3)
    y = np.cumsum(rng.uniform(0.2, 2.0, 40))
    c0, c1, c2 = 0.7, -1.3, 2.9
    q = c0 + c1 * y + c2 * y ** 2
    hm, hp = y[1:-1] - y[:-2], y[2:] - y[1:-1]
    d2 = d2_y(q[1:-1], q[2:], q[:-2], hm, hp)
    assert np.abs(d2 - 2.0 * c2).max() < 1e-9
    # and swapped weights fail it
    assert np.abs(d2_y(q[1:-1], q[2:], q[:-2], hp, hm) - 2.0 * c2).max() > 1e-3


def test_face_interpolation_is_exact_on_linear_profiles():
    rng = np.random.default_rng(4)
    yf = np.cumsum(rng.uniform(0.2, 2.0, 30))
    yc = 0.5 * (yf[:-1] + yf[1:])
    dyc = np.diff(yf)
    q = 0.3 - 1.7 * yc
    got = y_face_value(q[:-1], q[1:], dyc[:-1], dyc[1:])
    assert np.abs(got - (0.3 - 1.7 * yf[1:-1])).max() < 1e-12
    assert np.abs(y_face_value(q[:-1], q[1:], dyc[1:], dyc[:-1]) - (0.3 - 1.7 * yf[1:-1])).max() > 1e-3


@pytest.mark.parametrize("beta", [1.2, 2.2])
def test_couette_linear_profile_is_a_fixed_point_on_a_stretched_grid(beta):
    case = couette_case(ny=24)
    case = case.with_(y_faces=_faces(case, beta))
    s = OracleSolver(case)
    g = s.grid
    a, b, U = case.init["a"], case.init["b"], case.init["U"]
    y = np.broadcast_to(g.coords(0)[1], g.shape)
    u = np.where(s.cls.internal[0], U * (y - a) / (b - a), 0.0)
    z = np.zeros(g.shape)
    s.set_state(u, z, z, z)
    s.step(3)
    u1 = np.where(s.cls.internal[0], s.u[0], 0.0)
    assert np.abs(u1 - u).max() < 1e-13 * U
    assert np.abs(s.u[1]).max() < 1e-13
    # the uneven grid really is uneven, and the walls cut it off the grid lines
    assert g.dyc.max() / g.dyc.min() > 1.5
    assert np.count_nonzero(s.w.lam[0]) > 0


def _box(ndim, beta, n=(12, 20, 8)):
    nx, ny, nz = n if ndim == 3 else (n[0], n[1], 1)
    case = Case(name="box", ndim=ndim, n=(nx, ny, nz), L=(1.3, 1.0, 0.9 if ndim == 3 else 1.0),
                origin=(0.0, -0.2, 0.0), bc_lo=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC),
                bc_hi=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC), geom_kind=GEOM_NONE, geom_params=(),
                nu=0.0, dt=1e-3)
    return case.with_(y_faces=_faces(case, beta))


def _random_velocity(g, seed):
    rng = np.random.default_rng(seed)
    vel = [rng.standard_normal(g.shape) if c < g.ncomp else np.zeros(g.shape) for c in range(3)]
    vel[1][:, -1, :] = 0.0                    # the upper wall face (v's last index)
    return vel


@pytest.mark.parametrize("ndim", [2, 3])
def test_stretched_projection_is_divergence_free_idempotent_and_adjoint(ndim):
    g = Grid(_box(ndim, 1.8))
    vel = _random_velocity(g, 11)
    r = divergence(g, vel)
    # the right-hand side of a field with no flux through the walls sums to zero over the volumes
    assert abs(np.sum(r * g.cell_volumes())) < 1e-12 * np.abs(r).max()
    phi = solve_spectral(g, r)
    phid = solve_direct(g, r)
    G = gradient(g, phi)
    assert np.abs((phi - phi.mean()) - (phid - phid.mean())).max() < 1e-10 * np.abs(phi).max()
    proj = [vel[c] - G[c] for c in range(3)]
    div = divergence(g, proj)
    assert np.abs(div).max() < 1e-11 * np.abs(r).max()
    again = [proj[c] - gradient(g, solve_spectral(g, divergence(g, proj)))[c] for c in range(3)]
    assert max(np.abs(again[c] - proj[c]).max() for c in range(3)) < 1e-11 * np.abs(vel[0]).max()
    # sum_cells V (D u) psi = - sum_faces V_face u (G psi): V_face = dx dy_face dz for v faces
    psi = np.random.default_rng(12).standard_normal(g.shape)
    Gp = gradient(g, psi)
    lhs = np.sum(g.cell_volumes() * divergence(g, vel) * psi)
    dz = g.d[2] if g.ndim == 3 else 1.0
    vol_face = [g.cell_volumes(), g.d[0] * g.face_heights() * dz, g.cell_volumes()]
    rhs_ = -sum(np.sum(vol_face[c] * vel[c] * Gp[c]) for c in range(g.ncomp))
    assert abs(lhs - rhs_) < 1e-11 * (abs(lhs) + abs(rhs_))
    # a wrong metric in G (the cell height instead of the centre distance) breaks it
    Gw = [Gp[0], Gp[1] * g.face_heights() / g.cell_heights(), Gp[2]]
    bad = -sum(np.sum(vol_face[c] * vel[c] * Gw[c]) for c in range(g.ncomp))
    assert abs(lhs - bad) > 1e-6 * abs(lhs)


@pytest.mark.parametrize("ndim", [2, 3])
def test_stretched_convection_conserves_u_and_w_momentum(ndim):
    """No body, nu = 0, g = 0: N_u and N_w are pure convection; the flux form telescopes in
    x and z (periodic) and in y (the wall faces carry v = 0), so their volume sums vanish."""
    case = _box(ndim, 2.0)
    s = OracleSolver(case)
    g = s.grid
    vel = _random_velocity(g, 21)
    N = rhs(g, s.cls, vel, 0.0, (0.0, 0.0, 0.0), [np.zeros(g.shape)] * 3)
    V = g.cell_volumes()
    scale = np.abs(N[0]).max() * np.sum(V * np.ones(g.shape))
    assert abs(np.sum(V * N[0])) < 1e-13 * scale
    if ndim == 3:
        assert abs(np.sum(V * N[2])) < 1e-13 * np.abs(N[2]).max() * np.sum(V * np.ones(g.shape))


def _ycon_errors(ny, beta=1.5):
    """y-convection of fields that depend on y only (nu = 0, no body): N_u = -(V U)' and
    N_v = -(V^2)' against the exact derivatives, at points two cells or more from the walls."""
    case = Case(name="ycon", ndim=2, n=(4, ny, 1), L=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0),
                bc_lo=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC), bc_hi=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC),
                geom_kind=GEOM_NONE, geom_params=(), nu=0.0, dt=1e-3)
    case = case.with_(y_faces=tanh_faces(ny, 0.0, 1.0, beta))
    s = OracleSolver(case)
    g = s.grid
    yc = np.broadcast_to(g.coords(0)[1], g.shape)
    yv = np.broadcast_to(g.coords(1)[1], g.shape)
    Uf = lambda y: 1.0 + 2.0 * y - 1.5 * y ** 2
    Vf = lambda y: np.sin(np.pi * y)                      # zero on both walls
    U, V = Uf(yc), Vf(yv)
    V[:, -1, :] = 0.0
    N = rhs(g, s.cls, [U, V, np.zeros(g.shape)], 0.0, (0.0, 0.0, 0.0), [np.zeros(g.shape)] * 3)
    dUV = lambda y: np.pi * np.cos(np.pi * y) * Uf(y) + Vf(y) * (2.0 - 3.0 * y)
    dVV = lambda y: 2.0 * np.pi * np.sin(np.pi * y) * np.cos(np.pi * y)
    inner = slice(2, ny - 2)
    eu = np.abs(N[0] + dUV(yc))[:, inner, :].max()
    ev = np.abs(N[1] + dVV(yv))[:, inner, :].max()
    return eu, ev


def test_stretched_y_convection_is_second_order():
    """The face interpolation and the control heights of the flux form: second order in y on
    a smoothly stretched grid (a wrong weight or metric leaves a first-order error)."""
    e = [_ycon_errors(n) for n in (32, 64, 128)]
    for c in range(2):
        slopes = [np.log2(e[i][c] / e[i + 1][c]) for i in range(2)]
        assert min(slopes) > 1.8, (c, e, slopes)


def _steady_error(ny, beta, use_ibm, c=0):
    a, b = 0.137, 0.861
    case = Case(name="ch", ndim=2, n=(4, ny, 1), L=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0),
                bc_lo=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC), bc_hi=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC),
                geom_kind=GEOM_PLANES, geom_params=(a, b), nu=1.0, dt=1e-3)
    case = case.with_(y_faces=tanh_faces(ny, 0.0, 1.0, beta))
    s = OracleSolver(case)
    g, cls = s.grid, s.cls
    q = steady.solve_component(g, cls, s.w, c, 1.0, 2.0, use_ibm=use_ibm)   # nu q'' = -2: q = (y-a)(b-y)
    y = np.broadcast_to(g.coords(c)[1], g.shape)
    exact = (y - a) * (b - y)
    return np.abs(q - exact)[cls.internal[c]].max()


def test_stretched_steady_channel_converges_at_second_order():
    ns = (16, 32, 64, 128)
    e = [_steady_error(n, 1.6, True) for n in ns]
    slopes = [np.log2(e[i] / e[i + 1]) for i in range(len(e) - 1)]
    assert min(slopes[1:]) > 1.85, (e, slopes)
    e0 = [_steady_error(n, 1.6, False) for n in ns]
    s0 = [np.log2(e0[i] / e0[i + 1]) for i in range(len(e0) - 1)]
    assert max(s0[1:]) < 1.5, (e0, s0)


def _tanh_map(eta, beta):
    return 0.5 * (1.0 + np.tanh(beta * (2.0 * eta - 1.0)) / np.tanh(beta))


def _fixed_fraction_error(ny, beta, c, use_ibm=True):
    """Steady error of component c with both walls at a fixed sub-cell fraction of the mapped
    coordinate (between faces ny/8 and ny/8 + 1 at 0.37, and symmetrically at 0.29 from the
    top), so that refinement changes the spacing and not where the wall cuts its cell."""
    m = ny // 8
    a = float(_tanh_map((m + 0.37) / ny, beta))
    b = float(_tanh_map(1.0 - (m + 0.29) / ny, beta))
    case = Case(name="ch", ndim=2, n=(4, ny, 1), L=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0),
                bc_lo=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC), bc_hi=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC),
                geom_kind=GEOM_PLANES, geom_params=(a, b), nu=1.0, dt=1e-3)
    case = case.with_(y_faces=tanh_faces(ny, 0.0, 1.0, beta))
    s = OracleSolver(case)
    g, cls = s.grid, s.cls
    q = steady.solve_component(g, cls, s.w, c, 1.0, 2.0, use_ibm=use_ibm)   # nu q'' = -2: q = (y-a)(b-y)
    y = np.broadcast_to(g.coords(c)[1], g.shape)
    return np.abs(q - (y - a) * (b - y))[cls.internal[c]].max()


@pytest.mark.parametrize("beta", [0.5, 1.5])
def test_both_components_converge_at_second_order_with_the_wall_at_a_fixed_sub_cell_fraction(beta):
    """Sec. 2.3 (second order of the implicit IBM) on the stretched grid, for the cell-centred
    u and for v on the faces (arms of face spacing): slopes of 2 between ny = 32, 64, 128
    once the wall keeps its place within its cell, 1 without the IBM correction."""
    ns = (32, 64, 128)
    for c in (0, 1):
        e = [_fixed_fraction_error(n, beta, c) for n in ns]
        slopes = [np.log2(e[i] / e[i + 1]) for i in range(len(e) - 1)]
        assert all(1.9 < p < 2.2 for p in slopes), (c, e, slopes)
    e0 = [_fixed_fraction_error(n, beta, 1, use_ibm=False) for n in ns]
    s0 = [np.log2(e0[i] / e0[i + 1]) for i in range(len(e0) - 1)]
    assert all(0.8 < p < 1.2 for p in s0), (e0, s0)


def test_stretched_three_dimensional_run_keeps_the_divergence_at_round_off():
    case = small_case("wavy3d").with_(n=(24, 36, 8), name="wavy3d_st")
    case = case.with_(y_faces=_faces(case, 1.5))
    s = OracleSolver(case)
    f = initial_field(case)
    s.set_state(f["u"], f["v"], f["w"], f["p"])
    s.project()
    s.step(2)
    d = s.diagnostics()
    assert d["finite"]
    umax = max(np.abs(s.u[c]).max() for c in range(3))
    assert d["div_linf"] < 1e-10 * umax / s.grid.dyc.min()
    assert np.isnan(s.last_force).all()      # force accounting is uniform-grid only


def test_wall_normal_laplacian_is_exact_for_a_quadratic_between_the_box_walls():
    """v between the two y walls (its wall values are the faces' zero): nu v'' = -2 has the
    solution v = y (1 - y), a quadratic, which the uneven second difference solves exactly."""
    case = _box(2, 1.7).with_(origin=(0.0, 0.0, 0.0), y_faces=tanh_faces(20, 0.0, 1.0, 1.7))
    s = OracleSolver(case, no_ibm=True)
    g = s.grid
    q = steady.solve_component(g, s.cls, s.w, 1, 1.0, 2.0, use_ibm=False)
    y = np.broadcast_to(g.coords(1)[1], g.shape)
    inside = s.cls.internal[1]
    assert np.abs(q - y * (1.0 - y))[inside].max() < 1e-12


def test_hydrostatic_pressure_balances_the_body_force_on_a_stretched_grid():
    """Fluid at rest under g = (0, g_y) with p = g_y y at the cell centres: the pressure
    gradient between the centres on either side of each face equals g_y, so the predictor
    leaves v* = 0 (the gradient's metric is the centre distance, not the cell height)."""
    gy = -3.0
    case = _box(2, 2.0).with_(g=(0.0, gy, 0.0), nu=0.1)
    s = OracleSolver(case)
    g = s.grid
    z = np.zeros(g.shape)
    p = np.broadcast_to(gy * g.coords(3)[1], g.shape).copy()
    s.set_state(z, z, z, p)
    s.substage(0, predictor_only=True)
    assert np.abs(s.u[1]).max() < 1e-13 * abs(gy) * case.dt
    assert np.abs(s.u[0]).max() < 1e-15


def test_wall_shear_of_a_parabola_is_exact_on_a_stretched_grid():
    """The quadratic through the wall, P and Q is exact for a parabola whatever the spacing: with
    the rows' own distances tau = 2 nu U / h in every column (1e-12)."""
    from oracle.forces import wall_shear
    case = couette_case(ny=28).with_(wall_u=(0.0, 0.0, 0.0))
    case = case.with_(y_faces=_faces(case, 1.9))
    s = OracleSolver(case)
    g = s.grid
    a, b = case.geom_params
    h, yc, U = (b - a) / 2, (a + b) / 2, 1.3
    y = np.broadcast_to(g.coords(0)[1], g.shape)
    u = U * (1.0 - ((y - yc) / h) ** 2)
    tau, t1c, t1s = wall_shear(g, s.cls, s.levelset, u, case.nu, g.L[0])
    exact = 2.0 * case.nu * U / h
    assert np.all(np.isfinite(tau)) and np.abs(tau - exact).max() < 1e-12 * exact


@pytest.mark.parametrize("name", ["cylinder2d_io", "tubes3d_io"])
def test_stretched_inflow_outflow_box_projects_to_round_off(name):
    """An inflow/outflow x (cosine transform in x) with a stretched y: after the initial projection
    and two steps the divergence over the cells is at round-off, and the outflow keeps the inflow's
    flux."""
    case = small_case(name)
    case = case.with_(y_faces=_faces(case, 1.4))
    s = OracleSolver(case)
    f = initial_field(case)
    s.set_state(f["u"], f["v"], f["w"], f["p"])
    s.project()
    s.step(2)
    d = s.diagnostics()
    g = s.grid
    umax = max(np.abs(s.u[c]).max() for c in range(g.ncomp))
    assert d["finite"] and d["div_linf"] < 1e-10 * umax / min(g.d[0], g.dyc.min())
    inflow = np.sum(np.where(s.cls.inflow_fluid, case.inflow[0], 0.0) * g.cell_heights()[..., :1])
    outflow = np.sum(np.where(s.cls.outflow_fluid, s.u[0][..., -1:], 0.0) * g.cell_heights()[..., :1])
    assert abs(outflow - inflow) < 1e-10 * abs(inflow)


def test_stretched_constant_flow_rate_holds_the_volume_integral():
    """The constant-flow-rate forcing on a stretched grid: after the predictor the volume integral
    of u over the internal u points, with each row's own cell height, equals the target."""
    case = small_case("wavy3d").with_(n=(24, 36, 8), name="wavy3d_st")
    case = case.with_(y_faces=_faces(case, 1.5))
    s = OracleSolver(case)
    f = initial_field(case)
    s.set_state(f["u"], f["v"], f["w"], f["p"])
    s.substage(0, predictor_only=True)
    yf = np.asarray(case.y_faces)
    dV = (case.L[0] / case.n[0]) * np.diff(yf)[None, :, None] * (case.L[2] / case.n[2])
    Q = float(np.sum(np.where(s.cls.internal[0], s.u[0], 0.0) * dV))
    assert abs(Q - case.target_flux) < 1e-12 * abs(case.target_flux)


def test_stretched_wall_normal_ibm_is_exact_on_a_line_through_the_wall():
    """v = y - a vanishes on the lower off-grid wall: the linear extrapolation through the wall
    returns the line itself, so with the stretched IBM weights of v (arms of face spacing) the
    discrete Laplacian nu L v - lambda v is zero at every v point of the lower half (1e-12)."""
    a, b = 0.137, 0.861
    case = Case(name="ch", ndim=2, n=(4, 30, 1), L=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0),
                bc_lo=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC), bc_hi=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC),
                geom_kind=GEOM_PLANES, geom_params=(a, b), nu=1.0, dt=1e-3)
    case = case.with_(y_faces=tanh_faces(30, 0.0, 1.0, 1.7))
    s = OracleSolver(case)
    g, cls = s.grid, s.cls
    A, sel = steady.laplacian_matrix(g, cls, 1)
    y = np.broadcast_to(g.coords(1)[1], g.shape).ravel()[sel]
    v = y - a
    res = A @ v - s.w.lam[1].ravel()[sel] * v
    lower = y < 0.5 * (a + b) - 0.1
    assert np.count_nonzero(s.w.lam[1].ravel()[sel][lower]) > 0
    assert np.abs(res[lower]).max() < 1e-12 * np.abs(A).max()
