"""The momentum predictor at the full 384 x 256 x 256 wavy-channel and 512 x 384 x 256
airway sizes, in the launch configuration the benchmark times (FP32, default z-chunk, the TMA form:
wrap boxes on the periodic channel, ghost columns on the inflow/outflow duct),
against the FP64 oracle on sampled points; on the airway also the classification byte
and lambda of the device-built weights at the sampled points.

The predictor at a point depends only on its 3 x 3 x 3 neighbourhood, its IBM weight
and the pressure next to it, so the oracle evaluates each sample on a 7-point window
cut out of the same input fields around it (the window keeps a box wall where it
touches one).  The flow is driven by a uniform body force here: under the constant
flow rate the predictor would add a scalar that only the whole field determines.

Tolerance: the GPU reads the fields in FP32 and the oracle the same FP32-rounded
values in FP64, so the difference is FP32 arithmetic in about 40 operations per
point on O(1) values: 2e-6 of the largest velocity.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

from inputs import wavy_c3, airway_c4, initial_field, FLOW_FORCED, BC_PERIODIC, BC_NOSLIP  # noqa: E402
from oracle import OracleSolver, Grid, LevelSet, classify  # noqa: E402

R = 3   # window half-width


def _window_case(case, i, j, k):
    nx, ny, nz = case.n
    d = [case.L[a] / case.n[a] for a in range(3)]
    jlo, jhi = max(0, j - R), min(ny, j + R + 1)
    bc_lo = (BC_PERIODIC, case.bc_lo[1] if jlo == 0 else BC_NOSLIP, BC_PERIODIC)
    bc_hi = (BC_PERIODIC, case.bc_hi[1] if jhi == ny else BC_NOSLIP, BC_PERIODIC)
    n = (2 * R + 1, jhi - jlo, 2 * R + 1)
    origin = (case.origin[0] + (i - R) * d[0], case.origin[1] + jlo * d[1], case.origin[2] + (k - R) * d[2])
    L = (n[0] * d[0], n[1] * d[1], n[2] * d[2])
    # samples keep R cells from the x faces, so the window is periodic in x and sees no inflow
    w = case.with_(n=n, origin=origin, L=L, bc_lo=bc_lo, bc_hi=bc_hi, inflow=(0.0, 0.0, 0.0), name="window")
    ii = (i - R + np.arange(n[0])) % nx
    jj = np.arange(jlo, jhi)
    kk = (k - R + np.arange(n[2])) % nz
    return w, (ii, jj, kk), (R, j - jlo, R)


def _samples(case, cls, kzm, rng):
    nx, ny, nz = case.n
    pts = set()
    for _ in range(60):
        pts.add((int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz))))
    # tile, chunk and box edges
    edges_i = [0, 1, 31, 32, 33, nx - 33, nx - 32, nx - 1]
    edges_j = [0, 1, 15, 16, 17, ny - 17, ny - 16, ny - 2, ny - 1]
    edges_k = [0, kzm - 1, kzm, 2 * kzm - 1, nz - 1]
    for _ in range(80):
        pts.add((int(rng.choice(edges_i)), int(rng.choice(edges_j)), int(rng.choice(edges_k))))
    # IBM points of each component (the oracle's own lists)
    for c in range(3):
        lst = cls.lists[c]
        for idx in rng.choice(lst, size=min(30, lst.size), replace=False):
            idx = int(idx)
            pts.add((idx % nx, (idx // nx) % ny, idx // (nx * ny)))
    return sorted(pts)


def test_predictor_full_size_sampled_against_oracle():
    from paper_2506_14328_gb300.solver import Solver
    case = wavy_c3(precision="fp32", steps=1).with_(flow_mode=FLOW_FORCED, g=(0.01, 0.0, 0.0))
    f = initial_field(case)
    # both sides read the same FP32-rounded inputs
    f32 = {q: np.asarray(f[q], dtype=np.float32).astype(np.float64) for q in ("u", "v", "w", "p")}
    g = Solver.from_case(case)
    kzm, _, tma = g.tiles()
    assert tma, "the full-size FP32 grid runs the TMA form"
    g.set_state(f32["u"], f32["v"], f32["w"], f32["p"])
    g.step(1, flags=1)                     # IBM_STEP_PREDICTOR_ONLY: u* of stage 1
    us, _ = g.state()
    g.close()
    cls = classify(Grid(case), LevelSet(case.geom_kind, case.geom_params))
    rng = np.random.default_rng(2024)
    pts = _samples(case, cls, kzm, rng)
    assert len(pts) >= 200
    umax = max(np.abs(f32[q]).max() for q in ("u", "v", "w"))
    worst = 0.0
    for (i, j, k) in pts:
        wc, (ii, jj, kk), (ci, cj, ck) = _window_case(case, i, j, k)
        o = OracleSolver(wc)
        sub = {q: f32[q][np.ix_(kk, jj, ii)] for q in ("u", "v", "w", "p")}
        o.set_state(sub["u"], sub["v"], sub["w"], sub["p"])
        o.substage(0, predictor_only=True)
        for c in range(3):
            if not o.cls.internal[c][ck, cj, ci]:
                continue   # non-internal points carry no equation
            err = abs(us[c][k, j, i] - o.u[c][ck, cj, ci]) / umax
            worst = max(worst, err)
            assert err < 2e-6, ((i, j, k), c, err)
    assert worst > 0.0     # FP32 arithmetic leaves a trace; an exact match would mean nothing ran


def _airway_samples(case, ls, kzm, rng):
    """Cells near the tube walls (|phi| < 2 cells at the centre), a few deep in the fluid,
    a few on the 32 x 16 tile and z-chunk edges, and a few anywhere (mostly solid).  Every
    sample keeps R cells from the x faces.  Chosen with the oracle's level set alone."""
    nx, ny, nz = case.n
    h = case.L[0] / nx
    cand = np.stack([rng.integers(R, nx - R, 40000), rng.integers(ny, size=40000), rng.integers(nz, size=40000)], 1)
    xc = (cand + 0.5) * h
    phi = np.asarray(ls.phi(xc[:, 0], xc[:, 1], xc[:, 2]))
    near = cand[np.abs(phi) < 2 * h]
    deep = cand[phi < -3 * h]
    edge = near[((near[:, 0] % 32 == 0) | (near[:, 0] % 32 == 31)) | ((near[:, 1] % 16 == 0) | (near[:, 1] % 16 == 15))
                | ((near[:, 2] % kzm == 0) | (near[:, 2] % kzm == kzm - 1))]
    pts = set()
    for arr, m in ((near, 200), (deep, 30), (edge, 40), (cand, 30)):
        for q in rng.permutation(len(arr))[:m]:
            pts.add(tuple(int(v) for v in arr[q]))
    return sorted(pts)


def test_airway_full_size_sampled_against_oracle():
    from paper_2506_14328_gb300.solver import Solver
    from oracle import LevelSet as LS
    case = airway_c4(precision="fp32", steps=1).with_(init={"kind": "uniform_noise", "U": 1.0, "noise": 0.1})
    nx, ny, nz = case.n
    f = initial_field(case)
    f32 = {q: np.asarray(f[q], dtype=np.float32).astype(np.float64) for q in ("u", "v", "w", "p")}
    del f
    g = Solver.from_case(case)
    kzm, _, tma = g.tiles()
    assert tma, "the full-size FP32 duct runs the TMA form (x a multiple of 16)"
    mask, lists = g.classification()
    lam, _ = g.weights_lists()
    g.set_state(f32["u"], f32["v"], f32["w"], f32["p"])
    g.step(1, flags=1)                     # IBM_STEP_PREDICTOR_ONLY: u* of stage 1
    us, _ = g.state()
    g.close()
    ls = LS(case.geom_kind, case.geom_params)
    pts = _airway_samples(case, ls, kzm, np.random.default_rng(7))
    assert len(pts) >= 200
    umax = max(np.abs(f32[q]).max() for q in ("u", "v", "w"))
    worst, nibm, nint = 0.0, 0, 0
    for (i, j, k) in pts:
        wc, (ii, jj, kk), (ci, cj, ck) = _window_case(case, i, j, k)
        o = OracleSolver(wc)
        # the grid spacing is a power of two, so the window's coordinates are the box's bit for bit
        assert mask[k, j, i] == o.cls.mask[ck, cj, ci], (i, j, k)
        sub = {q: f32[q][np.ix_(kk, jj, ii)] for q in ("u", "v", "w", "p")}
        o.set_state(sub["u"], sub["v"], sub["w"], sub["p"])
        o.substage(0, predictor_only=True)
        lin = (k * ny + j) * nx + i
        wlin = (ck * wc.n[1] + cj) * wc.n[0] + ci
        for c in range(3):
            if mask[k, j, i] & (16 << c):
                pos = int(np.searchsorted(lists[c], lin))
                wpos = int(np.searchsorted(o.cls.lists[c], wlin))
                ref = o.w.lam_list[c][wpos]
                assert abs(lam[c][pos] - ref) <= 1e-12 * abs(ref), ((i, j, k), c)
                nibm += 1
            if not o.cls.internal[c][ck, cj, ci]:
                continue
            nint += 1
            err = abs(us[c][k, j, i] - o.u[c][ck, cj, ci]) / umax
            worst = max(worst, err)
            assert err < 2e-6, ((i, j, k), c, err)
    assert nibm >= 80 and nint >= 300
    assert worst > 0.0


def test_wavy_channel_fp32_against_fp64_after_ten_steps():
    """The 384 x 256 x 256 wavy channel (constant flow rate at Re_b 5600, laminar profile plus 5%
    noise) in FP32 mode and in FP64 mode from the same initial field: after 10 steps, the largest
    difference of each velocity component over its internal points relative to the largest FP64
    velocity, and the difference of the mean streamwise profile u(y) (the average over x and z)
    relative to its largest value."""
    from paper_2506_14328_gb300.solver import Solver
    base = wavy_c3(precision="fp64", steps=10)
    f = initial_field(base)
    runs = {}
    for prec in ("fp64", "fp32"):
        g = Solver.from_case(base.with_(precision=prec))
        g.set_state(f["u"], f["v"], f["w"], f["p"])
        g.project()
        g.step(10)
        assert g.diagnostics()["status"] == 0
        u, _ = g.state()
        runs[prec] = [np.asarray(x, dtype=np.float64) for x in u]
        g.close()
    del f
    cls = classify(Grid(base), LevelSet(base.geom_kind, base.geom_params))
    a, b = runs["fp64"], runs["fp32"]
    scale = max(np.abs(a[c][cls.internal[c]]).max() for c in range(3))
    field = [float(np.abs(b[c] - a[c])[cls.internal[c]].max() / scale) for c in range(3)]
    pa, pb = a[0].mean(axis=(0, 2)), b[0].mean(axis=(0, 2))
    prof = float(np.abs(pb - pa).max() / np.abs(pa).max())
    print(f"FP32 against FP64 after 10 steps: largest difference per component {field}, "
          f"mean u(y) {prof:.3e}")
    # measured on a GB300: 6.4e-7, 2.1e-7, 2.1e-7 and 1.3e-7
    assert max(field) < 1e-5
    assert prof < 2e-6


def test_airway_fp32_against_fp64_after_ten_steps():
    """The 512 x 384 x 256 airway (inflow/outflow x, tube union, weights built on the device) in
    FP32 mode and in FP64 mode from the same initial field: after 10 steps, the largest difference
    of each velocity component over its internal points (the device classification's bits)
    relative to the largest FP64 velocity, and the difference of the flow rate through the
    outflow face."""
    from paper_2506_14328_gb300.solver import Solver
    base = airway_c4(precision="fp64", steps=10)
    f = initial_field(base)
    runs, mask = {}, None
    for prec in ("fp64", "fp32"):
        g = Solver.from_case(base.with_(precision=prec))
        g.set_state(f["u"], f["v"], f["w"], f["p"])
        g.project()
        g.step(10)
        assert g.diagnostics()["status"] == 0
        u, _ = g.state()
        runs[prec] = [np.asarray(x, dtype=np.float64) for x in u]
        if mask is None:
            mask, _ = g.classification()
        g.close()
    del f
    a, b = runs["fp64"], runs["fp32"]
    inside = [(mask >> c) & 1 == 1 for c in range(3)]
    scale = max(np.abs(a[c][inside[c]]).max() for c in range(3))
    field = [float(np.abs(b[c] - a[c])[inside[c]].max() / scale) for c in range(3)]
    qa, qb = a[0][..., -1].sum(), b[0][..., -1].sum()
    flow = float(abs(qb - qa) / abs(qa))
    print(f"airway FP32 against FP64 after 10 steps: largest difference per component {field}, "
          f"outflow flow rate {flow:.3e}")
    # measured on a GB300: 9.6e-7, 7.6e-7, 9.2e-7 and 7.7e-9
    assert max(field) < 1e-5
    assert flow < 1e-7
