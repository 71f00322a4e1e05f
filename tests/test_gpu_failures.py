"""Failure detection without a GPU fault: every failure here is made on the host side.

* Memory: the device bytes a matrix holds after hodlr_build + hodlr_snapshot + hodlr_qr (+ a
  solve plan) equal hodlr_footprint's host-side count, the context's account returns to zero
  when the matrices are freed, and a memory limit on the context turns the allocation that
  would exceed it into HODLR_ENOMEM (build, and later the factorization's plan), after which
  the same handle factors normally once the limit is raised.
* Malformed input: a NaN or an infinity in a leaf or a factor is rejected with HODLR_EINVAL
  before anything is uploaded.
* A singular R: a leaf with a zero column gives a zero diagonal entry of R (Householder with
  tau = 0 handles the column itself, Alg. 1), and hodlr_solve reports HODLR_ESINGULAR.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from tests import gpu_util as U  # noqa: E402
from paper_1809_10585_gb300 import binding as B  # noqa: E402


def _fresh_ctx():
    U.ctx()                      # builds the library
    return B.Context(0)


@pytest.mark.parametrize("n,nmin,k,kc,est,nrhs", [(1024, 128, 5, 64, True, 0), (2048, 256, 10, 128, False, 16),
                                                  (777, 64, 4, 32, True, 3)])
def test_device_bytes_equal_host_footprint(n, nmin, k, kc, est, nrhs):
    ctx = _fresh_ctx()
    try:
        assert ctx.memory_used() == 0
        inp = W.random_hodlr(n, nmin, k, seed=1)
        M = B.Matrix(ctx, inp, rank_cap=kc)
        M.snapshot()
        M.qr(1e-10, 0.0 if est else 10.0)
        if nrhs:
            X = torch.randn(nrhs, n, dtype=torch.float64, device="cuda")
            M.solve_async(nrhs, X.data_ptr(), n)
        ctx.sync()
        assert M.status()[0] == 0
        want = B.footprint(n, inp.leaf_sizes, kc, estimate_norm=est, with_snapshot=True, nrhs=nrhs)
        assert M.device_bytes() == want
        assert ctx.memory_used() == want
        M.free()
        assert ctx.memory_used() == 0
    finally:
        ctx.close()


def test_memory_limit_gives_enomem_then_recovers():
    ctx = _fresh_ctx()
    try:
        inp = W.random_hodlr(2048, 256, 8, seed=2)
        kc = 64
        full = B.footprint(2048, inp.leaf_sizes, kc, estimate_norm=True)
        # 1) a limit below the storage: hodlr_build fails with HODLR_ENOMEM, nothing stays held
        ctx.set_memory_limit(1 << 20)
        with pytest.raises(B.HodlrError) as e:
            B.Matrix(ctx, inp, rank_cap=kc)
        assert e.value.code == B.HODLR_ENOMEM
        assert ctx.memory_used() == 0
        # 2) room for the matrix but not for the factorization's plan and scratch
        ctx.set_memory_limit(full // 2)
        M = B.Matrix(ctx, inp, rank_cap=kc)
        held = ctx.memory_used()
        assert 0 < held <= full // 2
        with pytest.raises(B.HodlrError) as e:
            M.qr(1e-10)
        assert e.value.code == B.HODLR_ENOMEM
        assert ctx.memory_used() <= full // 2
        # 3) limit raised: the same handle factors and the result is correct
        ctx.set_memory_limit(0)
        M.qr(1e-10)
        ctx.sync()
        assert M.status()[0] == 0
        assert ctx.memory_used() == full
        Y, T, R = U.factors_dense(M)
        A = torch.from_numpy(W.to_dense(inp)).cuda()
        eo, ea = U.errors_torch(Y, T, R, A, upper=True)
        assert eo <= 1e-8 and ea / U.norm2(A) <= 1e-8
        M.free()
        assert ctx.memory_used() == 0
    finally:
        ctx.close()


@pytest.mark.parametrize("where", ["leaf", "U12", "V21"])
@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_nonfinite_input_is_rejected(where, bad):
    ctx = U.ctx()
    inp = W.random_hodlr(512, 64, 4, seed=3)
    if where == "leaf":
        inp.leaves[2][5, 7] = bad
    elif where == "U12":
        inp.U12[1][3, 0] = bad
    else:
        inp.V21[0][10, 2] = bad
    with pytest.raises(B.HodlrError) as e:
        B.Matrix(ctx, inp, rank_cap=64)
    assert e.value.code == B.HODLR_EINVAL


def test_zero_column_gives_singular_solve():
    ctx = U.ctx()
    inp = W.random_hodlr(512, 64, 0, seed=4)      # zero off-diagonal ranks: per-leaf QRs
    inp.leaves[3][:, 5] = 0.0                      # a zero column of A
    M = B.Matrix(ctx, inp, rank_cap=32)
    M.qr(1e-12)
    ctx.sync()
    assert M.status()[0] == 0
    R = U.dense_of(M, 2).T.cpu().numpy()
    j = sum(inp.leaf_sizes[:3]) + 5
    assert R[j, j] == 0.0                         # tau = 0 for that column, r_jj = 0
    b = torch.randn(1, inp.n, dtype=torch.float64, device="cuda")
    rc = M.solve(1, b.data_ptr(), inp.n)
    assert rc == B.HODLR_ESINGULAR


def test_memory_pool_serves_allocations_and_rejects_overflow():
    """A context with a device memory pool takes every allocation of its matrices from the pool
    (no cudaMalloc/cudaFree while matrices come and go): results equal those of a context
    without a pool, the account returns to zero when the matrices are freed, a second context
    sharing the pool draws from the same account, and a matrix larger than the pool fails with
    HODLR_ENOMEM."""
    inp = W.random_hodlr(2048, 256, 8, seed=7)
    need = B.footprint(2048, inp.leaf_sizes, 64, estimate_norm=True)
    ref = U.gpu_qr(inp, 1e-10, anorm=0.0, rank_cap=64)
    Rref = U.dense_of(ref, 2).cpu().numpy()
    ctx = _fresh_ctx()
    ctx2 = B.Context(0)
    small = B.Context(0)
    try:
        ctx.set_memory_pool(2 << 30)                   # room for the dense copies below too
        ctx2.share_memory(ctx)
        with pytest.raises(B.HodlrError) as e:
            ctx.set_memory_pool(need)                  # already has one
        assert e.value.code == B.HODLR_ESTATE
        for rep in range(3):                           # memory is reused across matrices
            M = B.Matrix(ctx, inp, rank_cap=64)
            M2 = B.Matrix(ctx2, inp, rank_cap=64)
            M.qr(1e-10)
            M2.qr(1e-10)
            ctx.sync()
            ctx2.sync()
            assert ctx.memory_used() == 2 * need and ctx2.memory_used() == 2 * need
            for X in (M, M2):
                R = U.dense_of(X, 2).cpu().numpy()
                np.testing.assert_allclose(R, Rref, rtol=0, atol=1e-12 * np.abs(Rref).max())
            M.free()
            M2.free()
            assert ctx.memory_used() == 0
        small.set_memory_pool(need // 4)               # smaller than one factorization
        with pytest.raises(B.HodlrError) as e:
            X = B.Matrix(small, inp, rank_cap=64)
            X.qr(1e-10)
        assert e.value.code == B.HODLR_ENOMEM
    finally:
        small.close()
        ctx2.close()
        ctx.close()
