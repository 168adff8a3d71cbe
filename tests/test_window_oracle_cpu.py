"""The full-size GPU test evaluates the oracle's predictor on 7-point windows cut
out around sampled points.  Here, on a grid the oracle runs whole, the windowed
predictor equals the whole-grid predictor bit for bit, at wrapped x/z edges,
next to both walls and at IBM points, and the windows classify the same."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

from inputs import wavy_c3, initial_field, FLOW_FORCED  # noqa: E402
from oracle import OracleSolver  # noqa: E402
from test_gpu_fullsize import _window_case  # noqa: E402


def test_window_predictor_equals_whole_grid_predictor():
    case = wavy_c3(precision="fp64", steps=1, n=(64, 48, 20)).with_(flow_mode=FLOW_FORCED, g=(0.01, 0.0, 0.0))
    f = initial_field(case)
    o = OracleSolver(case)
    o.set_state(f["u"], f["v"], f["w"], f["p"])
    o.substage(0, predictor_only=True)
    rng = np.random.default_rng(1)
    pts = [(0, 0, 0), (63, 47, 19), (5, 1, 3), (40, 46, 10), (10, 3, 0)]
    pts += [(int(rng.integers(64)), int(rng.integers(48)), int(rng.integers(20))) for _ in range(20)]
    for c in range(3):
        for idx in o.cls.lists[c][:8]:
            pts.append((int(idx % 64), int((idx // 64) % 48), int(idx // (64 * 48))))
    compared = 0
    for (i, j, k) in pts:
        wc, (ii, jj, kk), (ci, cj, ck) = _window_case(case, i, j, k)
        w = OracleSolver(wc)
        sub = {q: f[q][np.ix_(kk, jj, ii)] for q in ("u", "v", "w", "p")}
        w.set_state(sub["u"], sub["v"], sub["w"], sub["p"])
        w.substage(0, predictor_only=True)
        for c in range(3):
            assert o.cls.internal[c][k, j, i] == w.cls.internal[c][ck, cj, ci], ((i, j, k), c)
            if o.cls.internal[c][k, j, i]:
                assert o.u[c][k, j, i] == w.u[c][ck, cj, ci], ((i, j, k), c)
                compared += 1
    assert compared > 60
