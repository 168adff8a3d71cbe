"""The momentum predictor at the full 384 x 256 x 256 wavy-channel size, in the launch
configuration the benchmark times (FP32, TMA form, default z-chunk), against the FP64
oracle on sampled points.

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

from inputs import wavy_c3, initial_field, FLOW_FORCED, BC_PERIODIC, BC_NOSLIP  # noqa: E402
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
    w = case.with_(n=n, origin=origin, L=L, bc_lo=bc_lo, bc_hi=bc_hi, name="window")
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
