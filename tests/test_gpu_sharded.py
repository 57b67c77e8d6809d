"""Sharded plans on the GPU: two ranks (processes) each plan their share of the
intervals (Section 5.1, concatenated distribution balanced by sample count) on
the one GPU of this machine, and sum every map-domain result across ranks through
the allreduce callback (Section 5.5, the role of MM_SomeReduce), here over
gloo with host copies.  No kernel of one rank waits on the other's: the
exchange runs on the host between launches.

The sharded plan must reproduce the single plan over all samples: the same
observed pixels and excisions, the operator H x and right-hand side b to
float64 rounding (1e-12), the float64 solve's map within the float64 map
tolerance (1e-10) and within one iteration, the mixed solve's map within 1e-6
of the float64 map, and the backward pass's lag gradients.
"""

from __future__ import annotations

import os
import socket
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _worker(rank, world, port, kind, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import paper_0906_1775_gb300 as mm
    from tests.gpu_helpers import cuda, host, lib_lags, make_plan
    from tests.helpers import tiny_IQU, tiny_T
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = {"rank": rank}
    try:
        if kind == "IQU":
            p = tiny_IQU(seed=21, n_per_det=2000, n_lags=48, n_ivl_lo=100, n_ivl_hi=900, flag_frac=0.02)
        else:
            p = tiny_T(seed=22, n=4000, width=8, n_lags=64, ivls=(700, 1300, 900, 1100))
        lags = lib_lags(p)
        i0, i1, lo, hi = mm.shard_range(p.interval_offsets, world, rank)
        off = np.asarray(p.interval_offsets[i0:i1 + 1], dtype=np.int64) - lo
        pix = cuda(np.ascontiguousarray(p.pix[lo:hi]))
        psi = cuda(np.ascontiguousarray(p.psi[lo:hi])) if p.psi is not None else None
        shard = mm.Plan(pix, psi, p.n_pix, off, p.interval_filter[i0:i1], lags, allreduce=mm.torch_allreduce())
        full = make_plan(p)
        ns = 3 if kind == "IQU" else 1
        o_s, e_s = shard.observed()
        o_f, e_f = full.observed()
        out["observed_equal"] = bool(np.array_equal(host(o_s), host(o_f)) and np.array_equal(host(e_s), host(e_f)))
        out["n_samples"] = hi - lo
        x = np.random.default_rng(3).standard_normal((full.n_obs, ns))
        for prec, dt in (("fp64", torch.float64), ("df64", torch.float64), ("fp32", torch.float32)):
            ys = host(shard.apply_ATNA(cuda(x, dt), precision=prec))[0]
            yf = host(full.apply_ATNA(cuda(x, dt), precision=prec))[0]
            out["op_" + prec] = _rel(ys, yf)
        d_s = cuda(np.ascontiguousarray(p.d[0][lo:hi]))
        d_f = cuda(p.d[0])
        out["rhs_fp64"] = _rel(host(shard.rhs(d_s, precision="fp64"))[0], host(full.rhs(d_f, precision="fp64"))[0])
        ms, i_s = shard.solve(d_s, precision="fp64", rel_tol=1e-12, max_iter=500)
        mf, i_f = full.solve(d_f, precision="fp64", rel_tol=1e-12, max_iter=500)
        out["map_fp64"] = _rel(host(ms), host(mf))
        out["iters"] = (i_s["iters"], i_f["iters"])
        mx, _ = shard.solve(d_s, precision="mixed", rel_tol=1e-9, max_iter=500, max_outer=20)
        out["map_mixed_vs_fp64"] = _rel(host(mx), host(mf))
        g = cuda(np.random.default_rng(4).standard_normal((full.n_obs, ns)))
        _, gl_s, _ = shard.solve_backward(d_s, ms, g, want_d=False, precision="fp64", rel_tol=1e-12)
        _, gl_f, _ = full.solve_backward(d_f, mf, g, want_d=False, precision="fp64", rel_tol=1e-12)
        out["grad_lags"] = _rel(host(gl_s), host(gl_f))
        shard.close()
        full.close()
    except Exception as e:  # reported to the test
        out["error"] = repr(e)
    finally:
        q.put(out)
        dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["IQU", "T"])
def test_sharded_plan_over_two_ranks_equals_single_plan(kind):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, kind, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=600) for _ in procs]
    for pr in procs:
        pr.join(timeout=120)
    for r in res:
        assert "error" not in r, r
        assert r["observed_equal"] and r["n_samples"] > 0, r
        assert r["op_fp64"] < 1e-12 and r["op_df64"] < 1e-12 and r["op_fp32"] < 2e-5, r
        assert r["rhs_fp64"] < 1e-12, r
        assert r["map_fp64"] < 1e-10 and abs(r["iters"][0] - r["iters"][1]) <= 1, r
        assert r["map_mixed_vs_fp64"] < 1e-6, r
        assert r["grad_lags"] < 1e-8, r
    for pr in procs:
        assert pr.exitcode == 0
