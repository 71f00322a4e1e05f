"""hodlr_build_dense (Sec. 2.1.1 construction of a HODLR matrix from a dense one) against the
oracle's block-by-block truncated SVD, plus hodlr_stats."""
import numpy as np
import pytest

import oracle.core as O
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from tests import gpu_util as U  # noqa: E402
from paper_1809_10585_gb300 import binding as B  # noqa: E402


def _blocks(H, sizes):
    """{v: [(rows, cols, U, V) of A12, of A21]} for every internal node of an oracle tree."""
    ranges = W.node_ranges(sizes)
    out = {}

    def walk(node, v):
        if node.leaf:
            return
        (lo1, hi1), (lo2, hi2) = ranges[2 * v + 1], ranges[2 * v + 2]
        out[v] = [((lo1, hi1), (lo2, hi2), node.U12, node.V12), ((lo2, hi2), (lo1, hi1), node.U21, node.V21)]
        walk(node.c1, 2 * v + 1)
        walk(node.c2, 2 * v + 2)
    walk(H, 0)
    return out


def test_kernel_matrix_matches_oracle_compression():
    n, nmin, thr = 2048, 128, 1e-9
    x, y = W.kernel_points(n, seed=1)
    A = 1.0 / (x[:, None] - y[None, :])
    A[np.diag_indices(n)] += n
    sizes = W.balanced_leaf_sizes(n, nmin)
    tA, pA, ld = U.dev(A)
    M = B.Matrix.from_dense(U.ctx(), n, sizes, pA, ld, thr, rank_cap=96, seed=3)
    D = U.dense_of(M, 0).cpu().numpy().T
    H = O.compress(A, sizes, thr)
    blocks = _blocks(H, sizes)
    r12, r21, _ = M.ranks()
    k = 0
    for v in range(len(sizes) - 1):
        for which in (0, 1):
            (r0, r1), (c0, c1), Uo, Vo = blocks[v][which]
            blk = A[r0:r1, c0:c1]
            kg = (r12 if which == 0 else r21)[v]
            s = np.linalg.svd(blk, compute_uv=False)
            ko = Uo.shape[1]
            assert abs(kg - ko) <= 1 and (kg == ko or np.min(np.abs(s - thr)) < 0.05 * thr), (v, which, kg, ko)
            err = np.linalg.norm(blk - D[r0:r1, c0:c1], 2)
            assert err <= 2 * thr + 1e-14 * s[0], (v, which, err)
            k = max(k, kg)
    st = M.stats()
    assert st["max_rank_R"] == max(r12) and st["max_rank_Y"] == max(r21) and st["bytes"] > 0
    # leaves are copied exactly
    for j, (lo, hi) in enumerate(W.node_ranges(sizes)[len(sizes) - 1:]):
        assert np.array_equal(D[lo:hi, lo:hi], A[lo:hi, lo:hi])


def test_exact_low_rank_blocks_are_recovered_and_factor():
    inp = W.random_hodlr(1024, 128, 5, seed=12)
    A = W.to_dense(inp)
    an = np.linalg.norm(A, 2)
    tA, pA, ld = U.dev(A)
    M = B.Matrix.from_dense(U.ctx(), inp.n, inp.leaf_sizes, pA, ld, 1e-12 * an, rank_cap=32, seed=1)
    r12, r21, _ = M.ranks()
    assert r12.max() == 5 and r21.max() == 5 and r12.min() == 5
    D = U.dense_of(M, 0).cpu().numpy().T
    assert np.abs(D - A).max() <= 1e-12 * an
    M.qr(1e-12, 0.0)
    U.ctx().sync()
    assert M.status()[0] == 0
    Y, T, R = U.factors_dense(M)
    At = torch.from_numpy(A).cuda()
    eo, ea = U.errors_torch(Y, T, R, At, upper=True)
    assert eo <= 1e-10 and ea / an <= 1e-10


def test_rank_capacity_is_reported():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((512, 512))
    tA, pA, ld = U.dev(A)
    with pytest.raises(B.HodlrError) as e:
        B.Matrix.from_dense(U.ctx(), 512, W.balanced_leaf_sizes(512, 64), pA, ld, 1e-12, rank_cap=16)
    assert e.value.code == 3
