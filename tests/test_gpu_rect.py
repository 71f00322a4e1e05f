"""Rectangular HODLR matrices and their permuted QR (Sec. 6) on the GPU, against the oracle
(oracle/rect.py) on the same seeded inputs:

* hodlr_permuted_qr against the oracle's Householder QR of the row-permuted matrix (LAPACK's
  dgeqrt of P A): R per entry relative to its column's scale, Y and T entrywise, on sizes with
  several 64-column panels and a ragged last panel;
* hodlr_rect_compress: exact-rank blocks come back with their rank, the dense reconstruction
  within the threshold;
* hodlr_rect_qr on Example 6.2 at reduced size: e_orth and e_acc within 10x of the oracle's (plus
  a roundoff floor), ranks of Y, T, R within one of the oracle's per block, the same memory
  ratios; and at the paper's size (8000 x 4000) against Table 5;
* argument checks (m_j < n_j, inconsistent partitions) give HODLR_EINVAL.
"""
import json
import pathlib

import numpy as np
import pytest

import oracle.rect as OR
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from tests import gpu_util as U  # noqa: E402
from paper_1809_10585_gb300 import binding as B  # noqa: E402

GOLD = json.loads((pathlib.Path(__file__).parent / "golden" / "paper_values.json").read_text())


def _norm2(op, n, iters=40, seed=0):
    """||op||_2 by power iteration on op^T op (op maps a torch (n, 1) vector both ways)."""
    g = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.randn((n, 1), dtype=torch.float64, device="cuda", generator=g)
    x /= torch.linalg.norm(x)
    s = 0.0
    for _ in range(iters):
        z = op(op(x, False), True)
        s = float(torch.linalg.norm(z))
        if s == 0.0:
            return 0.0
        x = z / s
    return float(np.sqrt(s))


@pytest.mark.parametrize("m,n,nmin,k", [(600, 300, 40, 3), (1000, 270, 70, 2), (400, 64, 16, 1)])
def test_permuted_qr_matches_oracle(m, n, nmin, k):
    inp = W.random_rect_hodlr(m, n, nmin, k, seed=m + n)
    A = W.rect_to_dense(inp)
    Y, T, R = OR.permuted_qr(A, inp.m_sizes, inp.n_sizes)
    ta, pa, lda = U.dev(A)
    tt, pt, ldt = U.empty(n, n)
    B.permuted_qr(U.ctx(), inp.m_sizes, inp.n_sizes, pa, lda, pt, ldt)
    Ag, Tg = U.host(ta, m, n), U.host(tt, n, n)
    p = OR.row_permutation(inp.m_sizes, inp.n_sizes)
    C = Ag[p]                                      # LAPACK layout of the QR of P A
    Yg = np.tril(C, -1)
    Yg[:n, :n] += np.eye(n)
    Rg = np.zeros((m, n))
    Rg[p[:n]] = np.triu(C[:n])
    Yo = Y[p]
    colscale = np.abs(R).max(axis=0)[None, :]
    assert (np.abs(Rg - R) / colscale).max() <= 1e-12 * np.sqrt(m)
    np.testing.assert_allclose(Yg, Yo, atol=1e-11)
    np.testing.assert_allclose(Tg, T, atol=1e-11)
    assert np.all(np.tril(Tg, -1) == 0.0)


def test_rect_compress_recovers_ranks_and_matrix():
    inp = W.random_rect_hodlr(900, 500, 70, 4, seed=9)
    A = W.rect_to_dense(inp)
    thr = 1e-9 * np.linalg.norm(A, 2)
    ta, pa, lda = U.dev(A)
    H, rc = B.RectMatrix.compress(U.ctx(), inp.m_sizes, inp.n_sizes, pa, lda, thr, rank_cap=32, seed=1)
    assert rc == 0
    r12, r21 = H.ranks()
    assert np.all(r12 == 4) and np.all(r21 == 4)
    to, po, ldo = U.empty(900, 500)
    H.to_dense(po, ldo)
    Ad = U.host(to, 900, 500)
    assert np.abs(Ad - A).max() <= 10 * thr
    Ho = OR.compress(A, inp.m_sizes, inp.n_sizes, thr)
    assert H.storage() == Ho.storage()
    H.free()


def _dense(Hm, rows, cols):
    t, p, ld = U.empty(rows, cols)
    Hm.to_dense(p, ld)
    torch.cuda.synchronize()
    return t.T                                       # natural (row, col) orientation


def _errors_gpu(Y, T, R, A):
    """e_orth = ||Q^T Q - I||_2, e_acc = ||A - Q R||_2 for Q = I - Y T Y^T (power iteration)."""
    m = Y.shape[0]

    def q(x, tr):
        return x - (Y @ (T.T @ (Y.T @ x)) if tr else Y @ (T @ (Y.T @ x)))

    def orth(x, tr):
        return q(q(x, False), True) - x

    def acc(x, tr):
        return (A.T @ x - R.T @ q(x, True)) if tr else (A @ x - q(R @ x, False))

    return _norm2(orth, m), _norm2(acc, A.shape[1])


def test_rect_qr_matches_oracle_example_6_2_reduced():
    g = GOLD["table5_rectangular"]
    inp = W.random_rect_hodlr(2000, 1000, 125, g["k"], seed=0)
    A = W.rect_to_dense(inp)
    res = OR.rect_qr(A, inp.m_sizes, inp.n_sizes, g["eps"])
    eo_o, ea_o = OR.errors(res, A)
    ta, pa, lda = U.dev(A)
    Yh, Th, Rh, an, rc = B.rect_qr(U.ctx(), inp.m_sizes, inp.n_sizes, pa, lda, g["eps"], anorm=res.anorm,
                                   rank_cap=64, seed=3)
    assert rc == 0 and an == res.anorm
    Y, T, R = _dense(Yh, 2000, 1000), _dense(Th, 1000, 1000), _dense(Rh, 2000, 1000)
    eo, ea = _errors_gpu(Y, T, R, torch.from_numpy(A).cuda())
    floor = 1e-14 * np.sqrt(2000)
    assert eo <= 10 * eo_o + floor and ea <= 10 * ea_o + floor * res.anorm, (eo, eo_o, ea, ea_o)
    for Hg, Ho in ((Yh, res.Y), (Th, res.T), (Rh, res.R)):
        r12, r21 = Hg.ranks()
        o12 = np.array([u.shape[1] for u in Ho.U12])
        o21 = np.array([u.shape[1] for u in Ho.U21])
        assert np.abs(r12 - o12).max() <= 1 and np.abs(r21 - o21).max() <= 1, (r12, o12, r21, o21)
    A_h = OR.compress(A, inp.m_sizes, inp.n_sizes, g["eps"] * res.anorm)
    mem_o = (res.Y.storage() + res.T.storage()) / A_h.storage()
    mem_g = (Yh.storage() + Th.storage()) / A_h.storage()
    assert abs(mem_g - mem_o) <= 0.02 * mem_o
    for h in (Yh, Th, Rh):
        h.free()


def test_rect_qr_example_6_2_full_size_against_table5():
    """Example 6.2 at the paper's size: random 8000 x 4000 rectangular HODLR matrix with rank-one
    blocks, n_min = 250, eps = 1e-10.  Table 5: e_orth 2.8e-13, e_acc 1.4e-11, maximal ranks
    Y 8, T 12, R 8, memory of Y and T 1.6x and of R 1.1x that of A (order of magnitude: the
    paper's random draw is not known)."""
    g = GOLD["table5_rectangular"]
    inp = W.random_rect_hodlr(g["m"], g["n"], g["nmin"], g["k"], seed=0)
    A = W.rect_to_dense(inp)
    ta, pa, lda = U.dev(A)
    Yh, Th, Rh, an, rc = B.rect_qr(U.ctx(), inp.m_sizes, inp.n_sizes, pa, lda, g["eps"], rank_cap=64, seed=3)
    assert rc == 0
    At = torch.from_numpy(A).cuda()
    assert abs(an - OR.norm2(A)) <= 1e-10 * an      # the same 30-step power iteration as the oracle
    Y, T, R = _dense(Yh, g["m"], g["n"]), _dense(Th, g["n"], g["n"]), _dense(Rh, g["m"], g["n"])
    eo, ea = _errors_gpu(Y, T, R, At)
    assert eo <= 10 * g["e_orth"] and ea <= 10 * g["e_acc"], (eo, ea)
    assert max(Yh.ranks()[0].max(), Yh.ranks()[1].max()) <= 2 * g["max_rank"]["Y"]
    assert Th.ranks()[0].max() <= 2 * g["max_rank"]["T"] and Rh.ranks()[0].max() <= 2 * g["max_rank"]["R"]
    for h in (Yh, Th, Rh):
        h.free()


def test_rect_argument_checks():
    c = U.ctx()
    ta, pa, lda = U.dev(np.ones((10, 10)))
    tt, pt, ldt = U.empty(10, 10)
    with pytest.raises(B.HodlrError) as e:
        B.permuted_qr(c, [4, 6], [5, 5], pa, lda, pt, ldt)        # m_1 < n_1
    assert e.value.code == B.HODLR_EINVAL
    with pytest.raises(B.HodlrError) as e:
        B.permuted_qr(c, [5, 5, 0], [5, 5, 0], pa, lda, pt, ldt)  # not a power of two, empty leaf
    assert e.value.code == B.HODLR_EINVAL
