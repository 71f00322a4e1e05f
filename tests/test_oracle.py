"""Pins for the CPU oracle: each test checks the oracle against something other than itself
(LAPACK through scipy, dense SVD, closed forms, invariants, brute force, the paper's printed
values).  No GPU needed."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.linalg.lapack as lapack

import oracle.core as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dgeqrt_full(A):
    """LAPACK's compact-WY QR with one block of width n: returns (V, T, R)."""
    m, n = A.shape
    v, t, info = lapack.dgeqrt(n, np.asfortranarray(A))
    assert info == 0
    V = np.tril(v[:, :n], -1)
    V[:n, :n] += np.eye(n)
    return V, np.triu(t[:n, :n]), np.triu(v[:n, :n])


# ---------------------------------------------------------------------------------- Alg. 1
@pytest.mark.parametrize("x", [np.array([3.0, 4.0]), np.array([-2.0, 1.0, 2.0]),
                               np.array([0.0, 1.0, -1.0]), np.array([-0.0, 2.0]),
                               np.array([5.0]), np.array([2.0, 0.0, 0.0]),
                               # magnitudes whose squares overflow / underflow: dlarfg scales
                               np.array([3e160, -4e160, 1e160]), np.array([-2e-170, 1e-170, 5e-171]),
                               np.array([1e-170, 3e160]), np.array([3e160, 1e-170])])
def test_householder_matches_dlarfg(x):
    y, gamma, rho = O.householder(x)
    beta, xs, tau = lapack.dlarfg(len(x), x[0], x[1:].copy() if len(x) > 1 else np.zeros(1))
    xs = xs[:len(x) - 1]
    assert math.isclose(rho, beta, rel_tol=1e-15, abs_tol=0)
    assert math.isclose(gamma, tau, rel_tol=1e-14, abs_tol=1e-300)
    np.testing.assert_allclose(y[1:], xs, rtol=1e-14, atol=0)
    Hx = x - gamma * y * (y @ x)
    np.testing.assert_allclose(Hx, np.r_[rho, np.zeros(len(x) - 1)], atol=1e-14 * len(x) * np.abs(x).max())


@pytest.mark.parametrize("m,n,seed", [(1, 1, 0), (7, 7, 1), (20, 5, 2), (33, 17, 3), (64, 64, 4), (70, 31, 5)])
def test_block_qr_equals_lapack_dgeqrt(m, n, seed):
    A = np.random.default_rng(seed).standard_normal((m, n))
    Y, T, R = O.block_qr(A)
    V, Tl, Rl = dgeqrt_full(A)
    sc = np.linalg.norm(A)
    np.testing.assert_allclose(R, Rl, atol=1e-13 * sc)
    np.testing.assert_allclose(Y, V, atol=1e-12)
    np.testing.assert_allclose(T, Tl, atol=1e-12)


def test_block_qr_equals_lapack_at_extreme_column_scales():
    # columns near 1e+-160: their squares overflow or underflow unless the norm is scaled
    A = np.random.default_rng(9).standard_normal((40, 17))
    A[:, 3] *= 1e160
    A[:, 5] *= 1e-160
    A[:, 11] *= 1e-160
    Y, T, R = O.block_qr(A)
    V, Tl, Rl = dgeqrt_full(A)
    assert np.isfinite(R).all() and np.isfinite(Y).all() and np.isfinite(T).all()
    # column j of R has the scale of column j of A
    assert (np.abs(R - Rl) / np.abs(Rl).max(axis=0)[None, :]).max() <= 1e-13
    np.testing.assert_allclose(Y, V, atol=1e-12)
    np.testing.assert_allclose(T, Tl, atol=1e-12)


def test_block_qr_zero_and_dependent_columns():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((12, 6))
    A[:, 2] = 0.0
    A[:, 4] = A[:, 1]
    Y, T, R = O.block_qr(A)
    Q = np.eye(12) - Y @ T @ Y.T
    np.testing.assert_allclose(Q @ np.vstack([R, np.zeros((6, 6))]), A, atol=1e-13)
    np.testing.assert_allclose(Q.T @ Q, np.eye(12), atol=1e-14)
    V, Tl, Rl = dgeqrt_full(A)
    # after the dependent column the factorization is not unique; compare the part before it
    np.testing.assert_allclose(np.abs(np.diag(R))[:4], np.abs(np.diag(Rl))[:4], atol=1e-13)


def test_block_qr_wy_identity():
    """T^{-1} + T^{-T} = Y^T Y holds for every compact-WY form of an orthogonal product."""
    A = np.random.default_rng(11).standard_normal((40, 24))
    Y, T, R = O.block_qr(A)
    Ti = np.linalg.inv(T)
    np.testing.assert_allclose(Ti + Ti.T, Y.T @ Y, atol=1e-12)
    assert np.allclose(np.triu(Y[:24, :24], 1), 0) and np.allclose(np.diag(Y), 1)
    assert np.allclose(np.tril(T, -1), 0) and np.allclose(np.tril(R, -1), 0)


# ------------------------------------------------------------------------ HODLR primitives
def _tree(n, nmin, k, seed, **kw):
    inp = W.random_hodlr(n, nmin, k, seed=seed, **kw)
    return inp, O.from_input(inp), W.to_dense(inp)


@pytest.mark.parametrize("part", ["full", "unit_lower", "upper"])
@pytest.mark.parametrize("trans", [False, True])
def test_matmat_matches_dense(part, trans):
    inp, H, _ = _tree(300, 40, 4, 3)
    Ad = O.to_dense(H, part)
    if part == "unit_lower":
        ref = np.tril(W.to_dense(inp), -1) + np.eye(300)
    elif part == "upper":
        ref = np.triu(W.to_dense(inp))
    else:
        ref = W.to_dense(inp)
    np.testing.assert_allclose(Ad, ref, atol=1e-14)
    X = np.random.default_rng(0).standard_normal((300, 5))
    Y = O.matmat(H, X, trans, part)
    np.testing.assert_allclose(Y, (ref.T if trans else ref) @ X, atol=1e-12)


@pytest.mark.parametrize("nL,nR,K,decay", [(50, 40, 12, 1.0), (30, 60, 30, 0.5), (10, 80, 25, 0.3), (64, 64, 0, 1.0)])
def test_truncate_matches_dense_svd(nL, nR, K, decay):
    rng = np.random.default_rng(nL + K)
    L = rng.standard_normal((nL, K)) * (decay ** np.arange(K))[None, :]
    Rt = rng.standard_normal((nR, K))
    eps = 1e-6
    Ln, Rn = O.truncate(L, Rt, eps)
    M = L @ Rt.T
    s = np.linalg.svd(M, compute_uv=False) if M.size else np.zeros(0)
    k_ref = int(np.sum(s > eps))
    assert Ln.shape[1] == k_ref
    err = np.linalg.norm(M - Ln @ Rn.T, 2) if M.size else 0.0
    sk1 = s[k_ref] if k_ref < len(s) else 0.0
    assert err <= sk1 * (1 + 1e-8) + 1e-13 * (s[0] if len(s) else 1)
    if k_ref:
        np.testing.assert_allclose(Ln.T @ Ln, np.eye(k_ref), atol=1e-13)


def test_truncate_rank_rule_ties_are_truncated():
    """k_eps is the smallest k with sigma_{k+1} <= eps: a singular value equal to eps goes."""
    U = np.eye(6)[:, :3]
    V = np.eye(5)[:, :3] * np.array([2.0, 0.5, 0.25])[None, :]
    Ln, Rn = O.truncate(U, V, 0.5)
    assert Ln.shape[1] == 1


def test_left_orthogonalize_preserves_product():
    rng = np.random.default_rng(2)
    L, Rt = rng.standard_normal((40, 6)), rng.standard_normal((30, 6))
    Q, Rn = O.left_orthogonalize(L, Rt)
    np.testing.assert_allclose(Q.T @ Q, np.eye(6), atol=1e-14)
    np.testing.assert_allclose(Q @ Rn.T, L @ Rt.T, atol=1e-13)


def test_lr_update_error_bound():
    inp, H, Ad = _tree(256, 32, 3, 9)
    rng = np.random.default_rng(1)
    U, V = rng.standard_normal((256, 4)), rng.standard_normal((256, 4))
    eps = 1e-9
    O.lr_update(H, U, V, eps)
    err = np.linalg.norm(O.to_dense(H) - (Ad - U @ V.T), 2)
    assert err <= 3 * eps * 1.01          # level-l HODLR: error <= l * eps (Sec. 2.1.1)
    O2 = O.from_input(inp)
    O.lr_update(O2, U, V, 0.0)
    np.testing.assert_allclose(O.to_dense(O2), Ad - U @ V.T, atol=1e-12)


def test_norm2_estimate():
    _, H, Ad = _tree(256, 32, 3, 4)
    est = O.norm2_estimate(H)
    assert abs(est - np.linalg.norm(Ad, 2)) <= 0.05 * np.linalg.norm(Ad, 2)
    assert est <= np.linalg.norm(Ad, 2) * (1 + 1e-12)


# ---------------------------------------------------------------------------------- Alg. 2
def test_level0_is_dense_householder():
    """A HODLR matrix of level 0 is one dense block: hQR reduces to Alg. 1 = dgeqrt."""
    inp, H, Ad = _tree(48, 64, 0, 5)
    assert H.leaf
    res = O.hqr(H, 1e-10)
    V, T, R = dgeqrt_full(Ad)
    np.testing.assert_allclose(res.R_dense(), R, atol=1e-12)
    np.testing.assert_allclose(res.Y_dense(), V, atol=1e-12)
    np.testing.assert_allclose(res.T_dense(), T, atol=1e-12)


def test_zero_rank_gives_per_leaf_qr():
    """All off-diagonal ranks zero: S = 0, T12 = 0 and every leaf is factored alone."""
    inp = W.zero_rank(200, 32, seed=2)
    res = O.hqr(O.from_input(inp), 1e-10)
    ranges = W.node_ranges(inp.leaf_sizes)
    nleaf = len(inp.leaf_sizes)
    Yd, Td, Rd = res.Y_dense(), res.T_dense(), res.R_dense()
    for j in range(nleaf):
        lo, hi = ranges[nleaf - 1 + j]
        V, T, R = dgeqrt_full(inp.leaves[j])
        np.testing.assert_allclose(Rd[lo:hi, lo:hi], R, atol=1e-12)
        np.testing.assert_allclose(Yd[lo:hi, lo:hi], V, atol=1e-12)
        np.testing.assert_allclose(Td[lo:hi, lo:hi], T, atol=1e-12)
    off = np.ones((200, 200), bool)
    for j in range(nleaf):
        lo, hi = ranges[nleaf - 1 + j]
        off[lo:hi, lo:hi] = False
    assert np.abs(Yd[off]).max() == 0 and np.abs(Td[off]).max() == 0 and np.abs(Rd[off]).max() == 0
    assert O.max_offdiag_rank(res.YR) == 0 and O.max_offdiag_rank(res.T) == 0


@pytest.mark.parametrize("n,nmin,k,seed", [(96, 16, 3, 1), (130, 20, 2, 2), (200, 24, 4, 3), (256, 32, 5, 4)])
def test_no_truncation_equals_dense_householder(n, nmin, k, seed):
    """With tol = 0 nothing is truncated, so the densified (Y, T, R) must equal LAPACK's
    compact-WY QR of the dense matrix: orthonormal B_L keeps every reflector's norm and pivot
    (Sec. 4, preprocessing), Y_B = B_L Y~_B restores the dense vectors (postprocessing), and T
    is fixed by Y."""
    inp, H, Ad = _tree(n, nmin, k, seed)
    res = O.hqr(H, 0.0)
    V, T, R = dgeqrt_full(Ad)
    kap = np.linalg.cond(Ad)
    tol = 1e-14 * kap
    np.testing.assert_allclose(res.R_dense(), R, atol=tol * np.linalg.norm(Ad, 2))
    np.testing.assert_allclose(res.Y_dense(), V, atol=tol)
    np.testing.assert_allclose(res.T_dense(), T, atol=tol)


def test_no_truncation_ragged_and_ill_conditioned():
    inp = W.random_hodlr(150, 20, 3, seed=8, col_scale_decades=6.0)
    Ad = W.to_dense(inp)
    res = O.hqr(O.from_input(inp), 0.0)
    V, T, R = dgeqrt_full(Ad)
    np.testing.assert_allclose(np.diag(res.R_dense()), np.diag(R), rtol=1e-6)
    np.testing.assert_allclose(res.Y_dense(), V, atol=1e-8)


@pytest.mark.parametrize("n,nmin,k,tol,dec", [(512, 64, 4, 1e-10, 0.0), (1000, 128, 5, 1e-10, 0.0),
                                              (1024, 128, 6, 1e-12, 10.0)])
def test_invariants_at_tolerance(n, nmin, k, tol, dec):
    inp, H, Ad = _tree(n, nmin, k, 0, col_scale_decades=dec)
    res = O.hqr(H, tol)
    e_orth, e_acc = O.errors_dense(res, Ad)
    an = np.linalg.norm(Ad, 2)
    assert e_orth <= 100 * tol and e_acc / an <= 100 * tol
    Yd, Rd, Td = res.Y_dense(), res.R_dense(), res.T_dense()
    assert np.all(np.tril(Rd, -1) == 0) and np.all(np.triu(Yd, 1) == 0) and np.all(np.diag(Yd) == 1)
    assert np.all(np.tril(Td, -1) == 0)
    # Q^T Q = I  <=>  T + T^T = T^T (Y^T Y) T  (T may be singular: the last reflector of a square
    # matrix is the identity, gamma = 0)
    G = Td.T @ (Yd.T @ Yd) @ Td
    assert np.linalg.norm(Td + Td.T - G, 2) <= 1e3 * tol * np.linalg.norm(G, 2)
    # the sign-normalised diagonal of R agrees with dense Householder QR
    Rr = np.linalg.qr(Ad, mode="r")
    assert np.max(np.abs(np.abs(np.diag(Rd)) - np.abs(np.diag(Rr)))) <= 1e3 * tol * an


def test_errors_decrease_with_tolerance():
    """Errors scale roughly with eps until roundoff dominates (Sec. 5, Example 5.3)."""
    inp = W.random_hodlr(512, 64, 8, seed=3, col_scale_decades=8.0)
    Ad = W.to_dense(inp)
    errs = []
    for tol in [1e-4, 1e-6, 1e-8, 1e-10]:
        e_orth, e_acc = O.errors_dense(O.hqr(O.from_input(inp), tol), Ad)
        errs.append(max(e_orth, e_acc / np.linalg.norm(Ad, 2)))
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1))
    assert errs[0] <= 100 * 1e-4 and errs[-1] <= 100 * 1e-10


def test_apply_and_solve():
    inp, H, Ad = _tree(300, 40, 4, 6)
    res = O.hqr(H, 1e-12)
    B = np.random.default_rng(3).standard_normal((300, 3))
    Q = res.Q_dense()
    np.testing.assert_allclose(O.apply_q(res, B), Q @ B, atol=1e-12)
    np.testing.assert_allclose(O.apply_qt(res, B), Q.T @ B, atol=1e-12)
    x = O.solve(res, B)
    np.testing.assert_allclose(Ad @ x, B, atol=1e-9 * np.linalg.norm(B))
    np.testing.assert_allclose(O.upper_solve(res.YR, B), scipy.linalg.solve_triangular(res.R_dense(), B), atol=1e-10)


def test_power_errors_match_dense():
    inp, H, Ad = _tree(400, 50, 4, 12, col_scale_decades=4.0)
    res = O.hqr(H, 1e-8)
    eo, ea = O.errors_dense(res, Ad)
    eop, eap = O.errors_power(res, H, iters=60)
    assert eop <= eo * 1.001 and eop >= 0.3 * eo
    assert eap <= ea * 1.001 and eap >= 0.3 * ea


# --------------------------------------------------------------------- the paper's numbers
def test_cauchy_condition_numbers_match_table4():
    g = json.load(open(os.path.join(GOLDEN, "paper_values.json")))["table4_cauchy"]
    for which, kap in zip((1, 2, 3), g["kappa"]):
        c = np.linalg.cond(W.cauchy_dense(which))
        assert kap / 10 <= c <= kap * 10, (which, c, kap)


@pytest.mark.slow
def test_table2_order_of_magnitude():
    """Example 5.1 at n = 1000: hQR errors are at the level the paper prints (Table 2; seeds
    and distributions unknown, so only the order of magnitude is checked)."""
    g = json.load(open(os.path.join(GOLDEN, "paper_values.json")))["table2_random_hodlr"]
    inp = W.rank1_example(1000, 250, seed=0)
    Ad = W.to_dense(inp)
    res = O.hqr(O.from_input(inp), 1e-10)
    e_orth, e_acc = O.errors_dense(res, Ad)
    assert e_orth <= 100 * g["e_orth_hqr"][0]
    assert e_acc <= 100 * g["e_acc_hqr"][0] * max(1.0, np.linalg.norm(Ad, 2) / 100)
    assert O.max_offdiag_rank(res.YR, "lower") <= 10 * json.load(open(os.path.join(GOLDEN, "paper_values.json")))["table3_ranks"]["Y"][0]


def test_cauchy_a1_accuracy_order_of_magnitude():
    """Example 5.2: hQR on the Cauchy matrix A_1 reaches the accuracy of Table 4."""
    g = json.load(open(os.path.join(GOLDEN, "paper_values.json")))["table4_cauchy"]
    A = W.cauchy_dense(1, n=2000)
    inp = W.dense_to_hodlr_input(A, 250, 1e-10)
    res = O.hqr(O.from_input(inp), 1e-10)
    e_orth, e_acc = O.errors_dense(res, A)
    assert e_orth <= 100 * g["e_orth_hqr"][0]
    assert e_acc <= 100 * g["e_acc_hqr"][0]
    assert O.max_offdiag_rank(res.YR, "lower") <= 3 * g["max_rank_YT"]


# ------------------------------------------------- planted mistakes must fail the pins above
def test_planted_sign_mistake_is_caught(monkeypatch):
    def flipped(x):
        x = np.asarray(x, dtype=np.float64)
        alpha = float(x[0]); xn = float(np.linalg.norm(x[1:])) if len(x) > 1 else 0.0
        y = np.zeros_like(x); y[0] = 1.0
        if xn == 0.0:
            return y, 0.0, alpha
        h = math.hypot(alpha, xn)
        beta = math.copysign(h, alpha)               # wrong sign convention
        y[1:] = x[1:] / (alpha - beta)
        return y, (beta - alpha) / beta, beta
    monkeypatch.setattr(O, "householder", flipped)
    A = np.random.default_rng(4).standard_normal((20, 8))
    Y, T, R = O.block_qr(A)
    V, Tl, Rl = dgeqrt_full(A)
    assert not np.allclose(R, Rl, atol=1e-10)


def test_planted_dropped_term_is_caught(monkeypatch):
    """Dropping the last column of every concatenated truncation input (a dropped term of S~ or
    T~12) breaks the tol = 0 pin."""
    orig = O.truncate

    def dropping(L, Rt, eps, step="a9_recompress"):
        if step in ("a5_S", "a8_T12") and L.shape[1] > 1:
            L, Rt = L[:, :-1], Rt[:, :-1]
        return orig(L, Rt, eps, step)
    monkeypatch.setattr(O, "truncate", dropping)
    inp, H, Ad = _tree(96, 16, 3, 1)
    res = O.hqr(H, 0.0)
    V, T, R = dgeqrt_full(Ad)
    assert not np.allclose(res.R_dense(), R, atol=1e-8)


def test_planted_missing_transpose_is_caught(monkeypatch):
    """Using T1 instead of T1^T in S = T1^T S~ breaks the tol = 0 pin."""
    orig = O.matmat

    def wrong(H, X, trans=False, part="full", step="matvec"):
        if step == "a6_TS":
            trans = not trans
        return orig(H, X, trans, part, step)
    monkeypatch.setattr(O, "matmat", wrong)
    inp, H, Ad = _tree(96, 16, 3, 1)
    res = O.hqr(H, 0.0)
    V, T, R = dgeqrt_full(Ad)
    assert not np.allclose(res.R_dense(), R, atol=1e-8)


def test_truncate_falls_back_to_dgesvd_when_dgesdd_fails(monkeypatch):
    """Sec. 2.1.1: the truncation is defined by the SVD, whichever LAPACK driver computes it."""
    rng = np.random.default_rng(11)
    L = rng.standard_normal((60, 14)) * (10.0 ** -np.arange(14))[None, :]
    Rt = rng.standard_normal((50, 14))
    ref_L, ref_R = O.truncate(L, Rt, 1e-9)

    def failing_svd(*a, **k):
        raise np.linalg.LinAlgError("SVD did not converge")
    monkeypatch.setattr(np.linalg, "svd", failing_svd)
    got_L, got_R = O.truncate(L, Rt, 1e-9)
    assert got_L.shape == ref_L.shape
    s = scipy.linalg.svd(L @ Rt.T, compute_uv=False, lapack_driver="gesvd")
    assert got_L.shape[1] == int(np.sum(s > 1e-9))
    np.testing.assert_allclose(got_L @ got_R.T, ref_L @ ref_R.T, atol=1e-12)


def test_compress_recovers_exact_hodlr_and_bounds_every_block():
    """Sec. 2.1.1 construction: an exactly rank-k HODLR matrix is recovered with rank k in every
    block; on a matrix of full-rank blocks each block keeps #{sigma > thr} terms and its error in
    the 2-norm is below thr."""
    inp = W.random_hodlr(300, 40, 5, seed=8)
    A = W.to_dense(inp)
    H = O.compress(A, inp.leaf_sizes, 1e-10 * np.linalg.norm(A, 2))
    assert O.max_offdiag_rank(H) == 5
    np.testing.assert_allclose(O.to_dense(H), A, atol=1e-12 * np.linalg.norm(A, 2))
    # graded full-rank blocks: entries decay away from the diagonal
    rng = np.random.default_rng(9)
    n = 256
    i = np.arange(n)
    B = rng.standard_normal((n, n)) * np.exp(-np.abs(i[:, None] - i[None, :]) / 6.0)
    sizes = W.balanced_leaf_sizes(n, 32)
    thr = 1e-6
    H = O.compress(B, sizes, thr)
    D = O.to_dense(H)
    ranges = W.node_ranges(sizes)
    for v in range(len(sizes) - 1):
        (lo1, hi1), (lo2, hi2) = ranges[2 * v + 1], ranges[2 * v + 2]
        for (r0, r1, c0, c1) in ((lo1, hi1, lo2, hi2), (lo2, hi2, lo1, hi1)):
            blk = B[r0:r1, c0:c1]
            err = np.linalg.norm(blk - D[r0:r1, c0:c1], 2)
            s = np.linalg.svd(blk, compute_uv=False)
            k = int(np.sum(s > thr))
            assert err <= thr * (1 + 1e-9) and (k == len(s) or abs(err - s[k]) <= 1e-9 * s[0])
    np.testing.assert_array_equal(np.diag(D), np.diag(B))
