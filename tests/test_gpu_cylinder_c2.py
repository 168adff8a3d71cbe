"""The 2D cylinder workload as configured (D = 1 at a seeded sub-cell offset, box 30D x 15D on
1536 x 768, uniform inflow U = 1, convective outflow, free-slip lateral walls; Re 40 steady and
Re 100 shedding), FP32 mode, on the GPU: drag and lift coefficients from the solver's force
diagnostic (reading R21), the divergence norms, and the FP32-vs-FP64 difference after 10 steps.

These Reynolds numbers are not in the paper (its tables give Re 30 and 185, pinned in
test_gpu_cylinder_paper.py), so the assertions here are physical bands, not paper values:
a steady symmetric wake with C_d between 1.4 and 1.8 at Re 40 (the free-stream value is about
1.5-1.6; the walls at 7.5D add blockage), and at Re 100 periodic shedding with a mean C_d between
1.25 and 1.6 and a Strouhal number between 0.15 and 0.20.  The printed numbers are the report."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

from inputs import cylinder_c2_io, initial_field  # noqa: E402


def _solver(case, **kw):
    from paper_2506_14328_gb300.solver import Solver
    g = Solver.from_case(case, **kw)
    f = initial_field(case)
    g.set_state(f["u"], f["v"], f["w"], f["p"])
    g.project()
    return g


def test_c2_re40_steady_drag_lift_and_divergence():
    case = cylinder_c2_io(re=40.0, precision="fp32")
    g = _solver(case, body_force=True)
    n10 = int(round(10.0 / case.dt))
    g.step(13 * n10)                   # t = 130
    g.diagnostics()                    # restart the force sums
    g.step(n10)
    cd_a = 2.0 * g.diagnostics()["force"][0]
    g.step(n10)                        # t = 150
    d = g.diagnostics()
    g.close()
    cd, cl = 2.0 * d["force"][0], 2.0 * d["force"][1]
    print(f"C2 Re 40: C_d(t 130-140) = {cd_a:.4f}, C_d(t 140-150) = {cd:.4f}, C_l = {cl:.2e}, "
          f"div_l2 = {d['div_l2']:.2e}, div_linf = {d['div_linf']:.2e}, cfl = {d['cfl']:.3f}")
    assert abs(cd - cd_a) < 0.005 * cd         # steady
    assert abs(cl) < 2e-3 * cd                 # symmetric wake
    assert 1.4 < cd < 1.8
    assert d["div_linf"] < 1e-3                # FP32 projection: round-off of O(U / dx) terms


def test_c2_re100_shedding():
    case = cylinder_c2_io(re=100.0, precision="fp32").with_(
        init={"kind": "uniform_noise", "U": 1.0, "noise": 0.01})
    g = _solver(case, body_force=True)
    g.step(int(round(150.0 / case.dt)))
    g.diagnostics()
    every = 10
    nsamp = int(round(50.0 / case.dt)) // every       # t in [150, 200]
    cd, cl = np.zeros(nsamp), np.zeros(nsamp)
    for q in range(nsamp):
        g.step(every)
        d = g.diagnostics()
        cd[q] = 2.0 * d["force"][0]
        cl[q] = 2.0 * d["force"][1]
    g.close()
    t = (np.arange(nsamp) + 0.5) * every * case.dt
    up = np.flatnonzero((cl[:-1] < 0.0) & (cl[1:] >= 0.0))
    tz = t[up] - cl[up] * (t[up + 1] - t[up]) / (cl[up + 1] - cl[up])
    st = (len(tz) - 1) / (tz[-1] - tz[0])
    cl_rms = np.sqrt(np.mean((cl - cl.mean()) ** 2))
    print(f"C2 Re 100: mean C_d = {cd.mean():.4f}, C_l' (r.m.s.) = {cl_rms:.4f}, St = {st:.4f}, "
          f"{len(tz)} crossings, div_linf = {d['div_linf']:.2e}")
    assert len(tz) >= 5
    assert 1.25 < cd.mean() < 1.6
    assert 0.15 < st < 0.20
    assert cl_rms > 0.1


def test_c2_fp32_against_fp64_after_ten_steps():
    """Both Reynolds numbers, from the same initial field: the largest FP32-FP64 difference of
    each velocity component over the internal points after 10 steps, relative to the largest
    FP64 value (the precision pattern's stated error), and the FP64 run's divergence norms."""
    for re in (40.0, 100.0):
        case = cylinder_c2_io(re=re, precision="fp64").with_(
            init={"kind": "uniform_noise", "U": 1.0, "noise": 0.05})
        a = _solver(case)
        b = _solver(case, precision="fp32")
        a.step(10)
        b.step(10)
        ua, _ = a.state()
        ub, _ = b.state()
        mask, _ = a.classification()
        d64 = a.diagnostics()
        errs = []
        for c in range(2):
            m = (mask >> c) & 1 == 1
            errs.append(float(np.abs(ub[c][m] - ua[c][m]).max() / np.abs(ua[c][m]).max()))
        a.close()
        b.close()
        print(f"C2 Re {re:g}: FP32 vs FP64 after 10 steps: u {errs[0]:.2e}, v {errs[1]:.2e}; "
              f"FP64 div_l2 {d64['div_l2']:.2e}, div_linf {d64['div_linf']:.2e}")
        assert max(errs) < 1e-5
        assert d64["div_linf"] < 1e-10
