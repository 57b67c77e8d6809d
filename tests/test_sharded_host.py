"""Sharded solves, host side (no GPU): the concatenated data distribution of
Section 5.1 and the per-iteration map sum of Section 5.5 over two gloo ranks.

* madmap_partition_intervals (host C) against its definition written out with
  exact rational targets, on random and degenerate interval layouts.
* Two gloo ranks each apply the FP64 oracle's A^T N^-1 A to their share of a
  seeded problem (whole intervals, so each rank's N^-1 is exactly the blocks of
  its intervals); the sum across ranks equals the whole problem's operator.
  This is the exchange the library's sharded plans make once per operator
  application (tests/test_gpu_sharded.py runs the library's side on a GPU).
"""

from __future__ import annotations

import os
import socket
import sys
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _mm():
    import paper_0906_1775_gb300 as mm
    from paper_0906_1775_gb300 import build
    if not os.path.exists(mm.library_path()):
        build.build()
    return mm


def _partition_by_definition(off, n_ranks):
    off = [int(v) for v in off]
    n = len(off) - 1
    first = [0]
    prev = 0
    for r in range(n_ranks - 1):
        target = Fraction(off[-1] * (r + 1), n_ranks)
        best = min(range(prev, n + 1), key=lambda j: (abs(off[j] - target), j))
        first.append(best)
        prev = best
    first.append(n)
    return first


@pytest.mark.parametrize("seed", range(6))
def test_partition_matches_definition(seed):
    mm = _mm()
    rng = np.random.default_rng(seed)
    n_ivl = int(rng.integers(1, 40))
    lens = rng.integers(0, 1000, n_ivl)
    if seed % 2:
        lens[rng.integers(0, n_ivl, 3)] = 0        # empty intervals
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    for n_ranks in (1, 2, 3, 4, 7, 64):
        got = mm.partition_intervals(off, n_ranks)
        assert list(got) == _partition_by_definition(off, n_ranks), (n_ranks, off)
        assert np.all(np.diff(got) >= 0) and got[0] == 0 and got[-1] == n_ivl


def test_partition_balances_equal_intervals():
    mm = _mm()
    off = np.arange(0, 1001, 100, dtype=np.int64)      # 10 intervals of 100 samples
    assert list(mm.partition_intervals(off, 2)) == [0, 5, 10]
    assert list(mm.partition_intervals(off, 5)) == [0, 2, 4, 6, 8, 10]
    assert list(mm.partition_intervals(np.array([0, 0, 0]), 3)) == [0, 0, 0, 2]


def test_partition_rejects_bad_offsets():
    mm = _mm()
    with pytest.raises(mm.MadmapError):
        mm.partition_intervals(np.array([0, 5, 3]), 2)
    with pytest.raises(mm.MadmapError):
        mm.partition_intervals(np.array([1, 5]), 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _operator_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from oracle import noise as nz
    from oracle import pointing as pt
    from tests.helpers import lags_for, tiny_IQU
    import paper_0906_1775_gb300 as mm
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = tiny_IQU(seed=9, n_per_det=900, n_ivl_lo=40, n_ivl_hi=300, flag_frac=0.05)
        lags = lags_for(p)
        x = np.random.default_rng(1).standard_normal((p.n_pix, 3))

        def operator(lo, hi, i0, i1):
            pl = np.asarray(p.pix[lo:hi], dtype=np.int64)
            w = pt.weights(p.psi[lo:hi], 3)
            y = pt.unpoint(x, pl, w)
            off = np.asarray(p.interval_offsets[i0:i1 + 1]) - lo
            z = nz.apply_ninv_direct(y, off, np.asarray(p.interval_filter[i0:i1]), lags)
            return pt.point(z, pl, w, p.n_pix, 3)

        i0, i1, lo, hi = mm.shard_range(p.interval_offsets, world, rank)
        part = torch.from_numpy(operator(lo, hi, i0, i1))
        dist.all_reduce(part)
        full = operator(0, p.n_samples, 0, p.n_intervals)
        err = float(np.linalg.norm(part.numpy() - full) / np.linalg.norm(full))
        q.put((rank, err, hi - lo))
    finally:
        dist.destroy_process_group()


def test_sum_of_shard_operators_is_the_operator_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_operator_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    got = sorted(q.get(timeout=300) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert all(e < 1e-13 for _, e, _ in got), got
    assert all(n > 0 for _, _, n in got)                # both ranks hold samples
