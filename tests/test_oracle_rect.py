"""Pins of the rectangular permuted-QR oracle (Sec. 6) against what the paper and the
mathematics fix, independent of the oracle itself:

* the Householder QR of the row-permuted matrix is LAPACK's dgeqrt of P A, permuted back
  (no truncation: the permuted QR is exact up to rounding);
* the structure Sec. 6 states: R is zero outside the first n_j rows of every row block and
  upper triangular there (the triangle of block column j on top of diagonal block j); Y is unit
  lower trapezoidal in the permuted row order; A = (I - Y T Y^T) R and Q is orthogonal;
* a planted mistake (the unpermuted QR) breaks that structure, so the structure check can fail;
* with square blocks (m_j = n_j) the permutation is the identity and the permuted QR is the
  hQR of Alg. 2 at tol = 0;
* compression: exact rank-k blocks are recovered with rank k, and thr = 0 reproduces the matrix;
* Example 6.2 / Table 5 at a reduced size: errors at the level of the truncation tolerance and
  factor ranks and memory of the same size as the paper's.
"""
import json
import pathlib

import numpy as np
import pytest
import scipy.linalg.lapack as lapack

import oracle.core as O
import oracle.rect as R
import workloads as W

GOLD = json.loads((pathlib.Path(__file__).parent / "golden" / "paper_values.json").read_text())


def _inp(m=600, n=300, nmin=40, k=3, seed=1):
    inp = W.random_rect_hodlr(m, n, nmin, k, seed=seed)
    return inp, W.rect_to_dense(inp)


def test_permutation_layout():
    p = R.row_permutation([5, 4, 6, 3], [2, 4, 1, 3])
    assert p.tolist() == [0, 1, 5, 6, 7, 8, 9, 15, 16, 17, 2, 3, 4, 10, 11, 12, 13, 14]
    assert R.row_permutation([4, 4], [4, 4]).tolist() == list(range(8))
    with pytest.raises(ValueError):
        R.row_permutation([3, 5], [4, 4])


def test_permuted_qr_equals_lapack_on_permuted_rows():
    inp, A = _inp()
    Y, T, Rm = R.permuted_qr(A, inp.m_sizes, inp.n_sizes)
    p = R.row_permutation(inp.m_sizes, inp.n_sizes)
    n = A.shape[1]
    v, t, info = lapack.dgeqrt(n, np.asfortranarray(A[p]))
    assert info == 0
    Yl = np.tril(v, -1)[:, :n]
    Yl[:n, :n] += np.eye(n)
    kappa = np.linalg.cond(A)
    np.testing.assert_allclose(Y[p], Yl, atol=1e-14 * kappa)
    np.testing.assert_allclose(T, np.triu(t[:n, :n]), atol=1e-14 * kappa)
    np.testing.assert_allclose(Rm[p[:n]], np.triu(v[:n, :n]), atol=1e-14 * kappa * np.abs(A).max())


def _structure_ok(Y, Rm, m_sizes, n_sizes):
    p = R.row_permutation(m_sizes, n_sizes)
    n = Rm.shape[1]
    rest = np.setdiff1d(np.arange(Rm.shape[0]), p[:n])
    return (np.all(Rm[rest] == 0.0) and np.all(np.tril(Rm[p[:n]], -1) == 0.0)
            and np.all(np.diag(Y[p]) == 1.0) and np.all(np.triu(Y[p][:n], 1) == 0.0))


def test_permuted_structure_and_factorization():
    inp, A = _inp(seed=2)
    Y, T, Rm = R.permuted_qr(A, inp.m_sizes, inp.n_sizes)
    assert _structure_ok(Y, Rm, inp.m_sizes, inp.n_sizes)
    Q = np.eye(A.shape[0]) - Y @ T @ Y.T
    an = np.linalg.norm(A, 2)
    assert np.linalg.norm(Q @ Rm - A, 2) <= 1e-13 * an
    assert np.linalg.norm(Q.T @ Q - np.eye(A.shape[0]), 2) <= 1e-13
    # the triangle of block column j lies in the first n_j rows of row block j
    ro, co = R.offsets(inp.m_sizes), R.offsets(inp.n_sizes)
    for j in range(len(inp.m_sizes)):
        blk = Rm[ro[j]:ro[j] + inp.n_sizes[j], co[j]:co[j + 1]]
        assert np.all(np.abs(np.diag(blk)) > 0)


def test_planted_mistake_unpermuted_qr_breaks_the_structure():
    inp, A = _inp(seed=3)
    Yu, Tu, Ru = O.block_qr(A)                 # the plain QR: triangle in the first n rows
    m, n = A.shape
    Rfull = np.zeros((m, n)); Rfull[:n] = Ru
    assert not _structure_ok(Yu, Rfull, inp.m_sizes, inp.n_sizes)


def test_square_blocks_reduce_to_hqr_at_tol_zero():
    sq = W.random_hodlr(256, 32, 3, seed=4)
    A = W.to_dense(sq)
    Y, T, Rm = R.permuted_qr(A, sq.leaf_sizes, sq.leaf_sizes)
    res = O.hqr(O.from_input(sq), 0.0)
    np.testing.assert_allclose(Y, res.Y_dense(), atol=1e-12)
    np.testing.assert_allclose(T, res.T_dense(), atol=1e-12)
    np.testing.assert_allclose(Rm, res.R_dense(), atol=1e-12 * np.abs(A).max())


def test_compression_recovers_exact_ranks_and_thr_zero_is_exact():
    inp, A = _inp(k=2, seed=5)
    H = R.compress(A, inp.m_sizes, inp.n_sizes, 1e-9 * np.linalg.norm(A, 2))
    assert H.ranks() == (2, 2)
    np.testing.assert_allclose(H.to_dense(), A, atol=1e-12 * np.abs(A).max())
    H0 = R.compress(A, inp.m_sizes, inp.n_sizes, 0.0)
    np.testing.assert_allclose(H0.to_dense(), A, atol=1e-12 * np.abs(A).max())


def test_example_6_2_reduced_size_matches_table5_in_magnitude():
    """Example 6.2 at m = 2000, n = 1000 (8 leaves instead of 16): rank-one random blocks,
    eps = 1e-10.  The paper reports, at 8000 x 4000, e_orth 2.8e-13, e_acc 1.4e-11, maximal ranks
    Y 8, T 12, Q 12, R 8, memory of Y and T 1.6x, of Q 2.2x and of R 1.1x that of A."""
    g = GOLD["table5_rectangular"]
    inp = W.random_rect_hodlr(2000, 1000, 125, g["k"], seed=0)
    A = W.rect_to_dense(inp)
    res = R.rect_qr(A, inp.m_sizes, inp.n_sizes, g["eps"])
    eo, ea = R.errors(res, A)
    assert eo <= 10 * g["e_orth"] and ea <= 10 * g["e_acc"], (eo, ea)
    assert max(res.Y.ranks()) <= g["max_rank"]["Y"] and max(res.T.ranks()) <= g["max_rank"]["T"]
    assert max(res.R.ranks()) <= g["max_rank"]["R"]
    A_h = R.compress(A, inp.m_sizes, inp.n_sizes, g["eps"] * res.anorm)
    mem_yt = (res.Y.storage() + res.T.storage()) / A_h.storage()
    mem_r = res.R.storage() / A_h.storage()
    assert abs(mem_yt - g["memory_vs_A"]["Y_and_T"]) <= 0.3 and abs(mem_r - g["memory_vs_A"]["R"]) <= 0.2
    # Q = I - Y T Y^T itself, compressed in the square format of the row partition (Table 5's
    # "Q" columns): larger ranks and memory than Y and T together, as the paper reports
    Qh = R.compress(res.Q_dense(), inp.m_sizes, inp.m_sizes, g["eps"])
    assert max(Qh.ranks()) <= g["max_rank"]["Q"]
    assert abs(Qh.storage() / A_h.storage() - g["memory_vs_A"]["Q"]) <= 0.3


def test_least_squares_from_the_permuted_qr():
    """min ||A X - B|| through the permuted QR: at tol = 0 it equals LAPACK's least-squares
    solution (scipy lstsq) to rounding times the condition number, with the same residual norm;
    at tol = 1e-10 the normal-equation residual A^T (A X - B) stays at the truncation level."""
    inp, A = _inp(m=500, n=200, nmin=30, k=2, seed=11)
    rng = np.random.default_rng(12)
    B = rng.standard_normal((A.shape[0], 3))
    import scipy.linalg as sla
    Xr, res_r, _, _ = sla.lstsq(A, B)
    kappa = np.linalg.cond(A)
    exact = R.rect_qr(A, inp.m_sizes, inp.n_sizes, 0.0)
    X0, r0 = R.lstsq(exact, B, inp.m_sizes, inp.n_sizes)
    np.testing.assert_allclose(X0, Xr, atol=1e-13 * kappa * np.abs(Xr).max())
    np.testing.assert_allclose(r0, np.linalg.norm(A @ Xr - B, axis=0), rtol=1e-10)
    tol = 1e-10
    approx = R.rect_qr(A, inp.m_sizes, inp.n_sizes, tol)
    X1, r1 = R.lstsq(approx, B, inp.m_sizes, inp.n_sizes)
    an = np.linalg.norm(A, 2)
    gram = np.linalg.norm(A.T @ (A @ X1 - B), axis=0)
    assert np.all(gram <= 100 * tol * an * an * np.linalg.norm(X1, axis=0) + 100 * tol * an * np.linalg.norm(B, axis=0))
    np.testing.assert_allclose(r1, np.linalg.norm(A @ X1 - B, axis=0), rtol=1e-6)
