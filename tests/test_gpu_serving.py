"""Batched stepping, tile autotuning and the continuous-batching server on the GPU.

The serving contract: a solve's result is the same alone and in the mix.
Every solve's kernels read and write only its own buffers, and every
reduction has a fixed order for a fixed tiling, so a batch of whole steps is
bitwise equal to stepping alone.  The momentum job kernel of small members
computes the register form of the predictor in another kernel, whose
instruction selection may round FP32 differently: there the comparison is
1e-12 of the largest value in FP64 and 2e-5 in FP32 (the FP32 mode's stated
bound against FP64), as for the two forms of the predictor.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

from inputs import small_case, serving_mix, initial_field  # noqa: E402


def _solver(case):
    from paper_2506_14328_gb300.solver import Solver
    s = Solver.from_case(case)
    f = initial_field(case)
    s.set_state(f["u"], f["v"], f["w"], f["p"])
    s.project()
    return s


def _same(a, b):
    ua, pa = a
    ub, pb = b
    return all(np.array_equal(x, y) for x, y in zip(ua, ub)) and np.array_equal(pa, pb)


def _close(a, b, precision):
    """Velocities within 1e-12 (FP64) or 2e-5 (FP32) of each component's largest value."""
    tol = 1e-12 if precision == "fp64" else 2e-5
    return all(np.abs(x - y).max() <= tol * max(np.abs(y).max(), 1e-300) for x, y in zip(a[0], b[0]))


def test_batch_graph_equals_separate_stepping():
    from paper_2506_14328_gb300 import ibm_batch_create, ibm_batch_set, ibm_batch_run, ibm_batch_destroy
    c1 = small_case("wavy3d", precision="fp32")
    c2 = small_case("channel2d", precision="fp64")
    a1, a2 = _solver(c1), _solver(c2)
    b1, b2 = _solver(c1), _solver(c2)
    st = torch.cuda.Stream()
    batch = ibm_batch_create(st.cuda_stream)
    ibm_batch_set(batch, [a1.h, a2.h], [3, 5])
    ibm_batch_run(batch)
    ibm_batch_run(batch)
    st.synchronize()
    b1.step(6)
    b2.step(10)
    assert _same(a1.state(), b1.state())
    assert _same(a2.state(), b2.state())
    assert a1.diagnostics()["step"] == 6 and a2.diagnostics()["step"] == 10
    ibm_batch_destroy(batch)


def test_batch_with_the_momentum_job_kernel_equals_separate_stepping():
    """Small members advance their momentum predictors in one persistent launch per substage
    (ibm_batch_jobs); each member's fields are bit for bit those of stepping it alone with the
    register form of the predictor, to the tolerances above, for uneven step counts (members
    drop out of the lockstep as their steps run out), both precisions, 2D and 3D, periodic and
    inflow/outflow x."""
    from paper_2506_14328_gb300 import (ibm_batch_create, ibm_batch_set, ibm_batch_run, ibm_batch_jobs,
                                        ibm_batch_destroy)
    cases = [small_case("wavy3d", precision="fp32"), small_case("channel2d", precision="fp64"),
             small_case("sphere3d", precision="fp32"), small_case("cylinder2d_io", precision="fp32"),
             small_case("sphere3d_io", precision="fp64")]
    steps = [3, 5, 2, 4, 1]
    a = [_solver(c) for c in cases]
    b = [_solver(c) for c in cases]
    for s in a + b:
        s.use_tma(False)
        s.sync()
    st = torch.cuda.Stream()
    batch = ibm_batch_create(st.cuda_stream)
    ibm_batch_jobs(batch, 1 << 22)
    ibm_batch_set(batch, [s.h for s in a], steps)
    ibm_batch_run(batch)
    ibm_batch_run(batch)
    st.synchronize()
    for s, n in zip(b, steps):
        s.step(2 * n)
    for x, y, n, c in zip(a, b, steps, cases):
        assert _close(x.state(), y.state(), c.precision), c.name
        assert x.diagnostics()["step"] == 2 * n
    ibm_batch_destroy(batch)


def test_autotune_choices_and_results():
    case = small_case("wavy3d", precision="fp64")
    a, b = _solver(case), _solver(case)
    kzm, kzd = a.autotune()
    assert kzm in (8, 12, 16, 24, 32, 48, 64, 86) and kzd in (4, 8, 16, 32)
    a.step(2)
    b.step(2)
    (ua, pa), (ub, pb) = a.state(), b.state()
    for c in range(3):
        assert np.abs(ua[c] - ub[c]).max() <= 1e-12 * np.abs(ub[c]).max()


def test_server_result_is_the_same_alone_and_in_the_mix():
    from paper_2506_14328_gb300.serving import Server, Request
    mix = serving_mix(seed=3, n_requests=6, rate_hz=40.0, step_scale=0.01, size_scale=0.35)
    reqs = [Request(q, t, c, s) for q, (t, c, s) in enumerate(mix)]
    srv = Server(max_resident=4, steps_per_tick=4, autotune=False, keep_state=True, init_field=initial_field)
    stats = srv.serve(reqs)
    assert stats["requests"] == len(reqs)
    assert stats["p50_s"] is not None and stats["p99_s"] >= stats["p50_s"]
    assert stats["recaptures"] >= 2
    for r in reqs:
        s = _solver(r.case)
        s.step(r.steps)
        assert _close(s.state(), r.result["state"], r.case.precision), r.case.name
        assert r.result["diag"]["status"] == 0
    srv.close()


def test_server_admits_by_hbm_footprint():
    from paper_2506_14328_gb300.serving import Server, Request
    mix = serving_mix(seed=5, n_requests=4, rate_hz=1000.0, step_scale=0.004, size_scale=0.3)
    reqs = [Request(q, 0.0, c, s) for q, (t, c, s) in enumerate(mix)]
    # a budget below two solves' footprint: the server must still finish all of them, one at a time
    srv = Server(hbm_budget_bytes=1, max_resident=4, steps_per_tick=2, autotune=False, init_field=initial_field)
    stats = srv.serve(reqs)
    assert stats["requests"] == 4
    srv.close()
