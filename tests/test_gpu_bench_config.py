"""Parity of the configuration that bench.py times, against the CPU oracle.

The bench factors independent seeded matrices of the n = 8192, nmin = 256, rank-10,
column-scaled (condition ~1e14) workload at tol = 1e-12 as one batched CUDA graph, with the
bench's cluster size and several factorizations in flight: the QR and Jacobi kernels then take their
shared-memory-capped, blocked and one-CTA forms.  A batch of three matrices (different
seeds) puts the kernels in the same forms as the bench's larger batches.  Every matrix of the
batch is compared with the oracle's hQR (Alg. 2) of the same seeded input:

* e_orth = ||Q^T Q - I||_2 and e_acc / ||A||_2 = ||Q R - A||_2 / ||A||_2 at most 100 tol (the
  Frobenius norms, upper bounds of the 2-norms, are checked) and within 10x of the oracle's
  own 2-norm errors (plus a roundoff floor);
* the sign-normalised diagonal of R within 1e3 tol ||A||_2 of the oracle's;
* ||A||_2 estimated on the device equal to the oracle's power iteration.
"""
import numpy as np
import pytest

import oracle.core as O
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from tests import gpu_util as U  # noqa: E402
from paper_1809_10585_gb300 import binding as B  # noqa: E402

SEEDS = (0, 1, 2)
TOL = 1e-12
from bench import BATCH_CLUSTER as BENCH_CLUSTER  # noqa: E402  (the cluster size bench.py uses)


def test_batched_graph_of_bench_workload_matches_oracle():
    c = U.ctx()
    cmax = c.cluster
    c.cluster = min(cmax, BENCH_CLUSTER)
    try:
        inps = [W.config1(seed=s) for s in SEEDS]
        mats = [B.Matrix(c, inp, rank_cap=128) for inp in inps]
        for M in mats:
            M.snapshot()
        # twice, as the bench does (the first call records the graph, the second replays it)
        for _ in range(2):
            B.qr_batched(c, mats, TOL, 0.0, graph=True)
            c.sync()
        for inp, M in zip(inps, mats):
            st, anorm = M.status()
            assert st == 0
            res = O.hqr(O.from_input(inp), TOL)
            assert abs(anorm - res.anorm) <= 1e-10 * res.anorm
            A = torch.from_numpy(W.to_dense(inp)).cuda()
            an = U.norm2(A)
            Y, T, R = U.factors_dense(M)
            (eo, ea), (eoF, eaF) = U.errors_both(Y, T, R, A)
            dg = torch.diagonal(R).abs()
            del Y, T, R
            Yo, To, Ro = (torch.from_numpy(x).cuda() for x in (res.Y_dense(), res.T_dense(), res.R_dense()))
            (eoo, eao), _ = U.errors_both(Yo, To, Ro, A)
            dgo = torch.diagonal(Ro).abs()
            del Yo, To, Ro
            floor = 1e-14 * np.sqrt(inp.n)
            assert eoF <= 100 * TOL and eaF / an <= 100 * TOL, (eoF, eaF / an)
            assert eo <= 10 * eoo + floor and ea <= 10 * eao + floor * an, (eo, eoo, ea, eao)
            assert (dg - dgo).abs().max().item() <= 1e3 * TOL * an
    finally:
        c.cluster = cmax


def test_sample_of_batch_family_matches_oracle():
    """A sample of the 256-matrix batch family (n log-uniform, nmin 128 or 256, ranks 5-20,
    every second matrix column-scaled to condition ~1e10), factored together as the batch bench
    does (uploaded into device matrices, one batched call, merged schedules per partition, rank
    capacity 256), each against the oracle's hQR of the same input: 2-norm errors within 10x of
    the oracle's, the Frobenius errors at most 100 tol, and the diagonal of R."""
    import workloads as W
    fam = W.batched_family(count=64, seed0=0, n_lo=2048, n_hi=4096)
    inps = [x for x in fam if x.n <= 4096][:5]
    c = U.ctx()
    cmax = c.cluster
    c.cluster = min(cmax, BENCH_CLUSTER)
    c.set_batch_group(4)
    try:
        mats = [B.Matrix(c, x, rank_cap=256) for x in inps]
        B.qr_batched(c, mats, TOL, 0.0)
        c.sync()
        for inp, M in zip(inps, mats):
            st, anorm = M.status()
            assert st == 0
            res = O.hqr(O.from_input(inp), TOL)
            assert abs(anorm - res.anorm) <= 1e-10 * res.anorm
            A = torch.from_numpy(W.to_dense(inp)).cuda()
            an = U.norm2(A)
            (eo, ea), (eoF, eaF) = U.errors_both(*U.factors_dense(M), A)
            Yo, To, Ro = (torch.from_numpy(x).cuda() for x in (res.Y_dense(), res.T_dense(), res.R_dense()))
            (eoo, eao), _ = U.errors_both(Yo, To, Ro, A)
            floor = 1e-14 * np.sqrt(inp.n)
            assert eoF <= 100 * TOL and eaF / an <= 100 * TOL, (inp.name, eoF, eaF / an)
            assert eo <= 10 * eoo + floor and ea <= 10 * eao + floor * an, (inp.name, eo, eoo, ea, eao)
            R = U.dense_of(M, 2).T
            assert (torch.diagonal(R).abs() - torch.diagonal(Ro).abs()).abs().max().item() <= 1e3 * TOL * an
    finally:
        c.cluster = cmax
        c.set_batch_group(0)
