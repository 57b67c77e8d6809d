"""Deterministic plans: map-domain sums in a fixed order (bit-reproducible maps).

The paper fixes no summation order; with floating-point atomics the order of
the scatter A^T w varies from run to run, so repeated solves agree only to
rounding.  A deterministic plan sums each observed pixel's samples in
ascending sample order, so repeated operator applications and solves on the
plan give identical bits, while matching the FP64 oracle at the parity
tolerances.
"""

from __future__ import annotations

import numpy as np
import pytest

from tests.gpu_helpers import cuda, host, make_plan
from tests.helpers import rel_rms, system_for, tiny_IQU, tiny_T

pytestmark = pytest.mark.gpu

FP64_OP_TOL = 1e-11
FP32_OP_TOL = 2e-5


def _cases():
    from synth import make_config
    return {"T": lambda: tiny_T(seed=31, flag_frac=0.05),
            "IQU": lambda: tiny_IQU(seed=32, flag_frac=0.03),
            "cfg2_quarter": lambda: make_config(2, scale=2)}


@pytest.mark.parametrize("case", ["T", "IQU", "cfg2_quarter"])
def test_deterministic_operator_matches_oracle_and_repeats_bitwise(case):
    import torch
    p = _cases()[case]()
    S = system_for(p)
    plan = make_plan(p, deterministic=True)
    assert plan.stats["deterministic"] == 1 and plan.stats["n_map_replicas"] == 1
    x = np.random.default_rng(7).standard_normal((S.n_obs, p.n_stokes))
    x[S.excised] = 0.0
    ref = S.H(x)
    for prec, tol, dt in (("fp64", FP64_OP_TOL, torch.float64), ("df64", FP64_OP_TOL, torch.float64),
                          ("fp32", FP32_OP_TOL, torch.float32)):
        xd = cuda(x, dt)
        y1 = plan.apply_ATNA(xd, precision=prec)
        y2 = plan.apply_ATNA(xd, precision=prec)
        assert torch.equal(y1, y2), prec
        assert rel_rms(host(y1)[0], ref) < tol, (prec, rel_rms(host(y1)[0], ref))
    b1 = plan.rhs(cuda(p.d), precision="fp64")
    b2 = plan.rhs(cuda(p.d), precision="fp64")
    assert torch.equal(b1, b2)
    assert rel_rms(host(b1)[0], S.rhs(p.d[0])) < FP64_OP_TOL


@pytest.mark.parametrize("case", ["T", "IQU", "cfg2_quarter"])
def test_deterministic_solves_repeat_bitwise(case):
    import torch
    p = _cases()[case]()
    S = system_for(p)
    plan = make_plan(p, deterministic=True)
    d = cuda(p.d[0])
    x_ref, _ = S.solve(p.d[0], rel_tol=1e-12, max_iter=3000)
    for kw in (dict(precision="fp64", rel_tol=1e-12, max_iter=3000),
               dict(precision="mixed", rel_tol=1e-10, max_iter=3000, max_outer=20),
               dict(precision="fp64", rel_tol=1e-12, max_iter=3000, use_graph=0)):
        m1, i1 = plan.solve(d, **kw)
        m2, i2 = plan.solve(d, **kw)
        assert torch.equal(m1, m2), kw
        assert i1["iters"] == i2["iters"] and i1["best_rel_res"] == i2["best_rel_res"]
        tol = 1e-10 if kw["precision"] == "fp64" else 1e-6
        assert rel_rms(host(m1), x_ref) < tol, (kw, rel_rms(host(m1), x_ref))


def test_deterministic_batched_solve_repeats_bitwise():
    import torch
    p = tiny_IQU(seed=33)
    plan = make_plan(p, deterministic=True)
    d = torch.stack([cuda(p.d[0]), cuda(p.d[0][::-1].copy()), cuda(0.5 * p.d[0])])
    m1, i1 = plan.solve_batched(d, precision="mixed", rel_tol=1e-9, max_iter=500)
    m2, i2 = plan.solve_batched(d, precision="mixed", rel_tol=1e-9, max_iter=500)
    assert torch.equal(m1, m2)
    single, _ = plan.solve(d[2].contiguous(), precision="mixed", rel_tol=1e-9, max_iter=500)
    assert rel_rms(host(m1[2]), host(single)) < 1e-6


def test_deterministic_plan_rejects_unsupported_layouts():
    import torch
    import paper_0906_1775_gb300 as mm
    p = tiny_T(seed=34)
    extra = torch.zeros(p.n_samples, dtype=torch.int32, device="cuda")
    with pytest.raises(mm.MadmapError) as e:
        make_plan(p, deterministic=True, extra_index=extra, n_extra=1)
    assert e.value.status == mm._lib.MADMAP_ERR_INVALID_ARG
