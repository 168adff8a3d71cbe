"""The seeded serving mix (C5) follows its stated recipe.

The recipe: 2D n x n with n log-uniform in [128, 1024] or 3D n^3 with n log-uniform in [64, 192],
half and half; Re log-uniform in [10, 2000] on the body diameter; 500-5000 steps; Poisson arrivals
at the given rate; the body inside the box; dt within the convective and viscous limits of the
explicit RK3 predictor.  Host-only: no solver is built.
"""
import math

import numpy as np

from inputs import serving_mix, GEOM_CYLINDER, GEOM_SPHERE


def test_serving_mix_sizes_steps_and_reynolds_numbers_stay_in_their_ranges():
    mix = serving_mix(seed=0, n_requests=400, rate_hz=10.0)
    assert len(mix) == 400
    three = [c for _, c, _ in mix if c.ndim == 3]
    two = [c for _, c, _ in mix if c.ndim == 2]
    assert 0.4 < len(three) / len(mix) < 0.6
    for c in three:
        n = c.n[0]
        assert c.n == (n, n, n) and 64 <= n <= 192 and n % 8 == 0
        assert c.geom_kind == GEOM_SPHERE
    for c in two:
        n = c.n[0]
        assert c.n == (n, n, 1) and 128 <= n <= 1024 and n % 8 == 0
        assert c.geom_kind == GEOM_CYLINDER
    steps = np.array([s for _, _, s in mix])
    assert steps.min() >= 500 and steps.max() <= 5000
    D = 0.5
    re = np.array([D / c.nu for _, c, _ in mix])
    assert re.min() >= 10.0 * (1 - 1e-12) and re.max() <= 2000.0 * (1 + 1e-12)
    # log-uniform: the median of log10(Re) sits near the middle of [1, log10 2000]
    mid = 0.5 * (1.0 + math.log10(2000.0))
    assert abs(np.median(np.log10(re)) - mid) < 0.25


def test_serving_mix_arrivals_are_a_poisson_stream_at_the_given_rate():
    rate = 10.0
    mix = serving_mix(seed=1, n_requests=1000, rate_hz=rate)
    t = np.array([a for a, _, _ in mix])
    assert np.all(np.diff(t) >= 0.0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    # exponential gaps: mean 1/rate, coefficient of variation 1
    assert abs(gaps.mean() * rate - 1.0) < 0.1
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.15


def test_serving_mix_bodies_lie_inside_the_box_and_dt_is_within_the_explicit_limits():
    for _, c, _ in serving_mix(seed=2, n_requests=200, rate_hz=5.0):
        dx = c.L[0] / c.n[0]
        r = c.geom_params[c.ndim]                      # (centre..., radius, sign)
        for d in range(c.ndim):
            x = c.geom_params[d]
            assert r < x < c.L[d] - r
        assert c.dt * 1.5 / dx <= 0.4 * (1 + 1e-12)     # convective: speeds up to 1.5
        assert c.nu * c.dt / dx ** 2 <= 0.12 * (1 + 1e-12)


def test_serving_mix_is_reproducible_from_its_seed():
    a = serving_mix(seed=7, n_requests=20, rate_hz=3.0)
    b = serving_mix(seed=7, n_requests=20, rate_hz=3.0)
    c = serving_mix(seed=8, n_requests=20, rate_hz=3.0)
    assert [(x[0], x[1].n, x[1].nu, x[2]) for x in a] == [(x[0], x[1].n, x[1].nu, x[2]) for x in b]
    assert [(x[1].n, x[2]) for x in a] != [(x[1].n, x[2]) for x in c]


def _tubes(seed, L=(1.0, 0.75, 0.5)):
    from inputs import tube_union
    g = tube_union(seed, L=L)
    nt, npts = int(g[0]), int(g[1])
    return nt, npts, np.array(g[2:]).reshape(nt, npts, 4)


def test_tube_union_counts_radii_and_face_clearances_follow_the_recipe():
    """6-12 tubes of 24 points; radii r0 (1 + 0.1 sin(ks + ph)) with r0 in [0.05, 0.2]; the points
    0.01 clear of the y and z faces (a branch's first point lies on its parent); branches clear of the
    x faces; the trunk crosses both x faces."""
    L = (1.0, 0.75, 0.5)
    counts = set()
    for seed in range(12):
        nt, npts, T = _tubes(seed, L)
        counts.add(nt)
        assert 6 <= nt <= 12 and npts == 24
        for q in range(nt):
            r = T[q, :, 3]
            assert r.min() >= 0.05 * 0.9 - 1e-12 and r.max() <= 0.2 * 1.1 + 1e-12
            assert r.max() / r.min() <= 1.1 / 0.9 + 1e-12
            rmax = r.max()                        # at most the 1.1 r0 the clamp keeps clear
            P = T[q] if q == 0 else T[q, 1:]
            for d, Ld in ((1, L[1]), (2, L[2])):
                x = P[:, d]
                assert np.all(x >= rmax + 0.01 - 1e-9) and np.all(x <= Ld - rmax - 0.01 + 1e-9)
            if q > 0:
                x = P[:, 0]
                assert np.all(x >= rmax + 0.01 - 1e-9) and np.all(x <= L[0] - rmax - 0.01 + 1e-9)
        assert T[0, 0, 0] < 0.0 and T[0, -1, 0] > L[0]      # the trunk enters and leaves through x
    assert len(counts) > 1                                  # the seed changes the tree


def test_tube_union_branches_start_on_an_earlier_tube_no_wider_than_it():
    """A branch starts at an interior sample of an earlier tube with x in [0.1, 0.9], and its r0 is at
    most the parent's radius there (or the smallest radius, 0.05, where the parent is narrower)."""
    for seed in range(8):
        nt, npts, T = _tubes(seed)
        for q in range(1, nt):
            start = T[q, 0, :3]
            found = False
            for p in range(q):
                dist = np.linalg.norm(T[p, 1:-1, :3] - start, axis=1)
                k = int(np.argmin(dist))
                if dist[k] < 1e-12:
                    found = True
                    x = T[p, 1 + k, 0]
                    assert 0.1 - 1e-12 <= x <= 0.9 + 1e-12
                    # r0 >= max / 1.1 (the bump is at most +10%), so this bounds r0 from below
                    r0_low = T[q, :, 3].max() / 1.1
                    assert r0_low <= max(min(0.2, T[p, 1 + k, 3]), 0.05) + 1e-12
                    break
            assert found, (seed, q)
