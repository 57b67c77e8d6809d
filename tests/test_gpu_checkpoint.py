"""Checkpoint and restart of the float64 PCG (Section 5: the solver state is
saved every 20 iterations by default, five map vectors and six scalars, and a
run can restart from any checkpoint).

The failure is made on the host: a checkpoint callback that writes the state
to disk and then stops the solve stands in for a job that dies; a fresh plan
(as in a restarted process) resumes from the file.  No GPU fault is involved.
"""

from __future__ import annotations

import numpy as np
import pytest

from tests.gpu_helpers import cuda, host, make_plan
from tests.helpers import rel_rms, system_for, tiny_IQU, tiny_T

pytestmark = pytest.mark.gpu

FP64_MAP_TOL = 1e-10
KW = dict(precision="fp64", rel_tol=1e-12, max_iter=400)


def _problem(kind):
    if kind == "IQU":
        return tiny_IQU(seed=61, n_per_det=2500, width=10, n_lags=16, n_ivl_lo=200, n_ivl_hi=1500)
    return tiny_T(seed=62, n=6000, width=12, ivls=(2500, 2300, 1200), n_lags=16)


@pytest.mark.parametrize("kind", ["IQU", "T"])
@pytest.mark.parametrize("graph", [2, 1, 0])
def test_checkpoints_leave_the_solve_unchanged(kind, graph):
    p = _problem(kind)
    plan = make_plan(p)
    d = cuda(p.d[0])
    m0, i0 = plan.solve(d, use_graph=graph, **KW)
    seen = []
    m1, i1 = plan.solve(d, use_graph=graph, checkpoint_every=5, on_checkpoint=lambda s: seen.append(s) and False,
                        **KW)
    assert i1["iters"] == i0["iters"] and i1["best_iter"] == i0["best_iter"] and i1["status"] == i0["status"]
    assert rel_rms(host(m1), host(m0)) < 1e-12
    assert [s["iters"] for s in seen] == list(range(5, i0["iters"], 5))
    for s in seen:
        assert s["n_obs"] == plan.n_obs and s["n_stokes"] == p.n_stokes and 0 <= s["best_iter"] <= s["iters"]
        assert s["x"].shape == (plan.n_obs, p.n_stokes) and np.all(np.isfinite(s["p"]))
        assert s["best_rel_res"] <= s["rel_res"] * (1 + 1e-12)


@pytest.mark.parametrize("kind", ["IQU", "T"])
def test_stop_write_restart_resume(kind, tmp_path):
    import paper_0906_1775_gb300 as mm
    p = _problem(kind)
    S = system_for(p)
    plan = make_plan(p)
    d = cuda(p.d[0])
    m0, i0 = plan.solve(d, **KW)
    assert i0["iters"] > 12
    path = tmp_path / "ckpt.npz"

    def crash_at_second(state):
        mm.save_checkpoint(path, state)
        return state["iters"] >= 8          # the job "dies" after writing its second checkpoint

    m_stop, i_stop = plan.solve(d, checkpoint_every=4, on_checkpoint=crash_at_second, **KW)
    assert i_stop["status"] == mm._lib.MADMAP_STOPPED and i_stop["iters"] == 8
    # the stopped solve returns its best iterate so far
    assert rel_rms(host(m_stop), mm.load_checkpoint(path)["x_best"]) == 0.0
    # restart: a new plan over the same pointing and filters, state read back from disk
    plan2 = make_plan(p)
    state = mm.load_checkpoint(path)
    assert state["iters"] == 8
    m2, i2 = plan2.solve_resume(state, rel_tol=KW["rel_tol"], max_iter=KW["max_iter"])
    assert i2["iters"] == i0["iters"] and i2["best_iter"] == i0["best_iter"] and i2["status"] == mm._lib.MADMAP_OK
    assert rel_rms(host(m2), host(m0)) < 1e-11
    x, oi = S.solve(p.d[0], rel_tol=KW["rel_tol"], max_iter=KW["max_iter"])
    assert rel_rms(host(m2), x) < FP64_MAP_TOL
    # resuming can itself checkpoint and be stopped again
    seen = []
    m3, i3 = plan2.solve_resume(state, rel_tol=KW["rel_tol"], max_iter=KW["max_iter"], checkpoint_every=3,
                                on_checkpoint=lambda s: seen.append(s["iters"]) and False)
    assert seen == list(range(11, i0["iters"], 3)) and i3["iters"] == i0["iters"]


def test_resume_at_max_iter_returns_the_saved_best():
    import paper_0906_1775_gb300 as mm
    p = _problem("IQU")
    plan = make_plan(p)
    d = cuda(p.d[0])
    states = []
    plan.solve(d, checkpoint_every=6, on_checkpoint=lambda s: states.append(s) or True, **KW)
    m, info = plan.solve_resume(states[0], rel_tol=KW["rel_tol"], max_iter=6)
    assert info["iters"] == 6 and info["status"] == mm._lib.MADMAP_WARN_MAXITER
    assert np.array_equal(host(m), states[0]["x_best"])


def test_checkpoint_arguments_are_validated():
    import paper_0906_1775_gb300 as mm
    p = _problem("IQU")
    plan = make_plan(p)
    d = cuda(p.d[0])
    states = []
    plan.solve(d, checkpoint_every=5, on_checkpoint=lambda s: states.append(s) or True, **KW)
    bad = dict(states[0])
    bad["n_obs"] = bad["n_obs"] + 1
    with pytest.raises(mm.MadmapError) as e:
        plan.solve_resume(bad)
    assert e.value.status == mm._lib.MADMAP_ERR_INVALID_ARG
    with pytest.raises(mm.MadmapError) as e:
        plan.solve(d, precision="mixed", checkpoint_every=5, on_checkpoint=lambda s: False)
    assert e.value.status == mm._lib.MADMAP_ERR_INVALID_ARG


def test_exception_in_checkpoint_callback_stops_and_propagates():
    p = _problem("T")
    plan = make_plan(p)
    d = cuda(p.d[0])

    def boom(state):
        raise RuntimeError("callback failed at %d" % state["iters"])

    with pytest.raises(RuntimeError, match="callback failed at 4"):
        plan.solve(d, checkpoint_every=4, on_checkpoint=boom, **KW)
    # the plan stays usable
    m, info = plan.solve(d, **KW)
    assert info["status"] == 0
