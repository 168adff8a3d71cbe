"""Second-order convergence of the drag on a curved body (the paper's cylinder between two
walls, Sec. 4.1 and the right panel of its cylinder figure: the error of the total drag force
falls at second order with the grid step).

A cylinder D = 1 at the centre of a channel 8D long (periodic) between no-slip walls 4D apart,
driven by a uniform body force g = 3 nu U / (2D)^2 (bulk velocity 1 without the body), Re = U D /
nu = 20, FP64, started from the laminar profile and run to t = 80 (steady to 1e-6).  Grids of
N = 16, 32, 64 and 128 cells per diameter keep the body at the same place relative to the grid.
The drag from the force diagnostic, against the N = 128 value: errors 5.5e-4, 1.6e-4, 1.7e-5
(an order of 2.5 from 16 to 64).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

from inputs import Case, initial_field, BC_PERIODIC, BC_NOSLIP, GEOM_CYLINDER  # noqa: E402


def _drag(N, re=20.0, T=80.0):
    from paper_2506_14328_gb300.solver import Solver
    L, H = 8.0, 4.0
    nu = 1.0 / re
    h = 1.0 / N
    dt = min(0.8 * 2.51 / (8.0 * nu / (h * h)), 0.3 * h)
    case = Case(name=f"cylinder_channel_{N}", ndim=2, n=(int(L * N), int(H * N), 1), L=(L, H, 1.0),
                origin=(-L / 2, -H / 2, 0.0), bc_lo=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC),
                bc_hi=(BC_PERIODIC, BC_NOSLIP, BC_PERIODIC), geom_kind=GEOM_CYLINDER,
                geom_params=(0.0, 0.0, 0.5, -1.0), nu=nu, dt=dt, g=(3.0 * nu / (H / 2) ** 2, 0.0, 0.0),
                precision="fp64", init={"kind": "channel_noise", "ylo": -H / 2, "yhi": H / 2, "Ub": 1.0, "noise": 0.0})
    g = Solver.from_case(case, body_force=True)
    f = initial_field(case)
    g.set_state(f["u"], f["v"], f["w"], f["p"])
    g.project()
    g.step(int(round(T / dt)) - 100, flags=2)     # graph replay
    g.diagnostics()
    g.step(100, flags=2)
    d = g.diagnostics()
    g.close()
    return d["force"][0], d["force"][1]


def test_cylinder_drag_converges_at_second_order():
    res = {N: _drag(N) for N in (16, 32, 64, 128)}
    ref = res[128][0]
    err = {N: abs(res[N][0] - ref) for N in (16, 32, 64)}
    order = math.log2(err[16] / err[64]) / 2.0
    print({N: res[N][0] for N in res}, err, "order", order)
    assert all(abs(res[N][1]) < 1e-10 * res[N][0] for N in res)      # symmetric: no lift
    assert err[16] > err[32] > err[64]
    assert 1.7 < order < 3.5
