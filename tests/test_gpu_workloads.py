"""The other workload families at their sizes, through the C ABI:

* kernel-generated nonsymmetric matrix A_ij = 1/(x_i - y_j) + n delta_ij at n = 65536, nmin = 256,
  tol = 1e-12: too large for dense checks, so orthogonality and accuracy are measured with the
  operators themselves (Q and Q^T applied to seeded probe blocks, R and A applied by HODLR
  products) and the leading diagonal block of R is compared with a dense QR of the leading
  block column;
* a sample of the cross-matrix batch family (n log-uniform, nmin in {128, 256}, ranks 5-20,
  every second matrix column-scaled), factored in one batched CUDA graph: each matrix agrees
  with its factorization alone to rounding (with several factorizations in flight the cluster
  kernels may run in another form) and meets the error bounds against a dense reference;
* symmetric banded matrices (b = 8) as HODLR matrices with exact rank-b off-diagonal blocks."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from tests import gpu_util as U  # noqa: E402
from paper_1809_10585_gb300 import binding as B  # noqa: E402


def _probe_errors(M, A_op, n, nprobe=8, seed=0):
    """max over probe columns of ||Q^T Q x - x|| / ||x|| and ||Q R x - A x|| / (||A x||)."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, nprobe))
    tX, pX, ld = U.dev(X)
    # orthogonality: Q^T (Q x) - x
    tq = tX.clone()
    M.apply_q(nprobe, tq.data_ptr(), ld)
    M.apply_qt(nprobe, tq.data_ptr(), ld)
    U.ctx().sync()
    eo = ((tq - tX).norm(dim=1) / tX.norm(dim=1)).max().item()
    # accuracy: Q (R x) against A x
    tR, pR, _ = U.empty(n, nprobe)
    M.matvec(2, 0, nprobe, pX, ld, pR, ld)
    M.apply_q(nprobe, pR, ld)
    tA, pA, _ = U.empty(n, nprobe)
    A_op.matvec(0, 0, nprobe, pX, ld, pA, ld)
    U.ctx().sync()
    ea = ((tR - tA).norm(dim=1) / tA.norm(dim=1)).max().item()
    return eo, ea


def test_kernel_matrix_n65536():
    tol = 1e-12
    n, nmin = 65536, 256
    inp = W.kernel_hodlr(n, nmin, 1e-12, seed=0, device="cuda")
    ranks = [u.shape[1] for u in inp.U12] + [u.shape[1] for u in inp.U21]
    assert 10 <= max(ranks) <= 40
    A_op = B.Matrix(U.ctx(), inp, rank_cap=256)          # unfactored copy for A x
    M = U.gpu_qr(inp, tol, anorm=0.0, rank_cap=256, graph=True)
    st, anorm = M.status()
    assert st == 0 and anorm > 0
    eo, ea = _probe_errors(M, A_op, n)
    assert eo <= 100 * tol, eo
    assert ea <= 100 * tol * anorm / 1.0, ea
    # the leading leaf of R equals the R factor of a dense QR of the first block column of A,
    # up to row signs (the first block column is exact: leaf + stacked low-rank blocks)
    m = inp.leaf_sizes[0]
    tcol, pcol, ld = U.empty(n, m)
    E = np.zeros((n, m)); E[:m, :m] = np.eye(m)
    tE, pE, _ = U.dev(E)
    A_op.matvec(0, 0, m, pE, n, pcol, n)
    U.ctx().sync()
    col = tcol.T.contiguous()                             # n x m, row-major view of the column block
    Rd = torch.linalg.qr(col, mode="r")[1]
    tRE, pRE, _ = U.empty(n, m)
    M.matvec(2, 0, m, pE, n, pRE, n)                      # R E: the first m columns of R
    U.ctx().sync()
    Rg = tRE[:, :m].T                                     # R's leading leaf (row, col)
    s = torch.sign(torch.diagonal(Rd)) * torch.sign(torch.diagonal(Rg))
    diff = (Rg * s[:, None] - Rd).abs().max().item()
    assert diff <= 1e3 * tol * anorm, diff


def test_batched_family_sample():
    tol = 1e-12
    fam = W.batched_family(count=12, seed0=7, n_lo=1024, n_hi=8192)
    c = U.ctx()
    cmax = c.cluster
    c.cluster = min(cmax, 4)
    try:
        alone = []
        for inp in fam:
            M = U.gpu_qr(inp, tol, anorm=0.0, rank_cap=256)
            assert M.status()[0] == 0
            alone.append([U.dense_of(M, w).cpu().numpy() for w in (1, 2, 3)])
            M.free()
        mats = [B.Matrix(c, inp, rank_cap=256) for inp in fam]
        for M in mats:
            M.snapshot()
        B.qr_batched(c, mats, tol, 0.0, graph=True)
        c.sync()
        for M, ref, inp in zip(mats, alone, fam):
            assert M.status()[0] == 0
            got = [U.dense_of(M, w).cpu().numpy() for w in (1, 2, 3)]
            for a, b in zip(got, ref):
                assert np.max(np.abs(a - b)) <= 1e-9 * max(1.0, np.max(np.abs(b))), inp.name
            Y, R, T = (torch.from_numpy(np.ascontiguousarray(x.T)).cuda() for x in got)
            A = torch.from_numpy(W.to_dense(inp)).cuda()
            an = U.norm2(A)
            eo, ea = U.errors_torch(Y, T, R, A, upper=True)
            assert eo <= 100 * tol and ea / an <= 100 * tol, (inp.name, eo, ea / an)
            M.free()
    finally:
        c.cluster = cmax


@pytest.mark.parametrize("n,b,nmin", [(4096, 8, 256), (2000, 8, 125)])
def test_banded_matrices(n, b, nmin):
    tol = 1e-12
    inp = W.banded_hodlr(n, b, nmin, seed=3)
    M = U.gpu_qr(inp, tol, anorm=0.0, rank_cap=256)
    assert M.status()[0] == 0
    Y, T, R = U.factors_dense(M)
    A = torch.from_numpy(W.to_dense(inp)).cuda()
    an = U.norm2(A)
    eo, ea = U.errors_torch(Y, T, R, A, upper=True)
    assert eo <= 100 * tol and ea / an <= 100 * tol, (eo, ea / an)
    Rd = torch.linalg.qr(A, mode="r")[1]
    assert (torch.diagonal(R).abs() - torch.diagonal(Rd).abs()).abs().max().item() <= 1e3 * tol * an
