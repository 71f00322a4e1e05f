"""CPU FP64 oracle of the permuted QR of rectangular HODLR matrices (Sec. 6 of Kressner &
Susnjara, arXiv:1809.10585).

TEST INFRASTRUCTURE ONLY, like ``oracle.core``: only the test-suite, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  It shares no
code with the CUDA path.

What Sec. 6 specifies, and how it is read here:

* A rectangular HODLR matrix A (m x n) has two partitions m = m_1 + ... + m_L and
  n = n_1 + ... + n_L (L = 2^l leaves, m_j >= n_j); the recursive 2 x 2 splitting of Sec. 2.1
  applies to the row index by the m-partition and to the column index by the n-partition, so
  leaf j is the dense m_j x n_j block and every off-diagonal block of an internal node is low
  rank.
* The QR reduces every leaf block column to a *permuted* triangular form: the n_j x n_j
  triangle of block column j sits in the first n_j rows of row block j ("on top of the dense
  diagonal block"), and everything else of the unreduced rows becomes zero.  Block column j is
  reduced on the rows not yet holding a triangle (the first n_i rows of the earlier blocks i < j
  are final).  Reading: this is the Householder QR (Alg. 1, LAPACK sign convention) of P A,
  where the row permutation P lists the first n_j rows of every row block j (j = 1 .. L, in
  order) followed by all remaining rows (in order).  Column j of P A is then reduced on exactly
  the rows the paper names, with its pivot on the first row of the triangle's place, so
  Y = P^T Y~, R = P^T [R~; 0] and T = T~ for P A = (I - Y~ T~ Y~^T) [R~; 0], and
  A = (I - Y T Y^T) R with Y "permuted lower trapezoidal" and R "permuted upper triangular".
* The paper's experiments (Ex. 6.1, 6.2) apply "a dense version of the algorithm" and compress
  the factors afterwards into the formats of Fig. 6.3: Y and R in the rectangular format of A,
  T (n x n) in the square format of the n-partition.  The compression here is the truncated SVD
  of every off-diagonal block, keeping the singular values above the threshold (Sec. 2.1.1),
  with the thresholds of the square case: eps ||A||_2 for R (it carries A's scale) and plain eps
  for Y and T (scale-free).
"""
from __future__ import annotations

import numpy as np

from . import core as O


def offsets(sizes):
    return np.concatenate([[0], np.cumsum(np.asarray(sizes, dtype=int))]).astype(int)


def row_permutation(m_sizes, n_sizes) -> np.ndarray:
    """Indices p with (P A) = A[p]: the first n_j rows of every row block j, then the rest."""
    if len(m_sizes) != len(n_sizes) or any(mj < nj for mj, nj in zip(m_sizes, n_sizes)):
        raise ValueError("needs two partitions of equal length with m_j >= n_j")
    ro = offsets(m_sizes)
    top = [np.arange(ro[j], ro[j] + n_sizes[j]) for j in range(len(m_sizes))]
    rest = [np.arange(ro[j] + n_sizes[j], ro[j + 1]) for j in range(len(m_sizes))]
    return np.concatenate(top + rest).astype(int)


def permuted_qr(A, m_sizes, n_sizes):
    """Dense permuted QR of Sec. 6: returns Y (m x n), T (n x n, upper), R (m x n) with
    A = (I - Y T Y^T) R, the triangle of block column j in the first n_j rows of row block j."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    if sum(m_sizes) != m or sum(n_sizes) != n:
        raise ValueError("partitions do not match the matrix")
    p = row_permutation(m_sizes, n_sizes)
    Yt, T, Rt = O.block_qr(A[p])
    Y = np.zeros((m, n))
    Y[p] = Yt
    R = np.zeros((m, n))
    R[p[:n]] = Rt
    return Y, T, R


class RectHodlr:
    """Rectangular HODLR matrix: heap-ordered tree (node v has children 2v + 1, 2v + 2; leaf j is
    node L - 1 + j) with dense leaves and low-rank off-diagonal blocks A12 = U12 V12^T (rows of
    the first child by columns of the second) and A21 = U21 V21^T."""

    def __init__(self, m_sizes, n_sizes, leaves, U12, V12, U21, V21):
        self.m_sizes, self.n_sizes = list(m_sizes), list(n_sizes)
        self.leaves, self.U12, self.V12, self.U21, self.V21 = leaves, U12, V12, U21, V21
        L = len(self.m_sizes)
        ro, co = offsets(self.m_sizes), offsets(self.n_sizes)
        self.rlo, self.rhi, self.clo, self.chi = [0] * (2 * L - 1), [0] * (2 * L - 1), [0] * (2 * L - 1), [0] * (2 * L - 1)
        for j in range(L):
            v = L - 1 + j
            self.rlo[v], self.rhi[v], self.clo[v], self.chi[v] = ro[j], ro[j + 1], co[j], co[j + 1]
        for v in range(L - 2, -1, -1):
            self.rlo[v], self.rhi[v] = self.rlo[2 * v + 1], self.rhi[2 * v + 2]
            self.clo[v], self.chi[v] = self.clo[2 * v + 1], self.chi[2 * v + 2]

    @property
    def shape(self):
        return sum(self.m_sizes), sum(self.n_sizes)

    def to_dense(self):
        A = np.zeros(self.shape)
        L = len(self.m_sizes)
        for j in range(L):
            v = L - 1 + j
            A[self.rlo[v]:self.rhi[v], self.clo[v]:self.chi[v]] = self.leaves[j]
        for v in range(L - 1):
            a, b = 2 * v + 1, 2 * v + 2
            A[self.rlo[a]:self.rhi[a], self.clo[b]:self.chi[b]] = self.U12[v] @ self.V12[v].T
            A[self.rlo[b]:self.rhi[b], self.clo[a]:self.chi[a]] = self.U21[v] @ self.V21[v].T
        return A

    def ranks(self):
        """(max rank of the blocks A12, max rank of the blocks A21)."""
        r12 = max([u.shape[1] for u in self.U12] or [0])
        r21 = max([u.shape[1] for u in self.U21] or [0])
        return r12, r21

    def storage(self):
        """Doubles stored: the dense leaves and the low-rank factors."""
        s = sum(d.size for d in self.leaves)
        for lst in (self.U12, self.V12, self.U21, self.V21):
            s += sum(x.size for x in lst)
        return s


def compress(A, m_sizes, n_sizes, thr) -> RectHodlr:
    """Rectangular HODLR approximation of a dense matrix (Sec. 2.1.1 on both partitions): dense
    leaves, every off-diagonal block replaced by its truncated SVD (sigma > thr; U = left
    vectors, V = right vectors times sigma)."""
    A = np.asarray(A, dtype=np.float64)
    shell = RectHodlr(m_sizes, n_sizes, [], [], [], [], [])
    L = len(m_sizes)
    leaves = []
    for j in range(L):
        v = L - 1 + j
        leaves.append(np.array(A[shell.rlo[v]:shell.rhi[v], shell.clo[v]:shell.chi[v]]))

    def block_svd(B):
        if B.size == 0:
            return np.zeros((B.shape[0], 0)), np.zeros((B.shape[1], 0))
        u, sv, vt = np.linalg.svd(B, full_matrices=False)
        k = int(np.sum(sv > thr))
        return np.array(u[:, :k]), np.array(vt[:k].T * sv[:k][None, :])

    U12, V12, U21, V21 = [], [], [], []
    for v in range(L - 1):
        a, b = 2 * v + 1, 2 * v + 2
        u, w = block_svd(A[shell.rlo[a]:shell.rhi[a], shell.clo[b]:shell.chi[b]])
        U12.append(u); V12.append(w)
        u, w = block_svd(A[shell.rlo[b]:shell.rhi[b], shell.clo[a]:shell.chi[a]])
        U21.append(u); V21.append(w)
    return RectHodlr(m_sizes, n_sizes, leaves, U12, V12, U21, V21)


def norm2(A, iters=O.POWER_ITERS):
    """||A||_2 by the oracle's power iteration (same start and count as the square case)."""
    x = np.ones((A.shape[1], 1)) / np.sqrt(A.shape[1])
    for _ in range(iters):
        z = A.T @ (A @ x)
        s = np.linalg.norm(z)
        if s == 0:
            return 0.0
        x = z / s
    return float(np.linalg.norm(A @ x))


class RectQRResult:
    def __init__(self, Y, T, R, anorm, tol):
        self.Y, self.T, self.R, self.anorm, self.tol = Y, T, R, anorm, tol

    def Q_dense(self):
        Y, T = self.Y.to_dense(), self.T.to_dense()
        return np.eye(Y.shape[0]) - Y @ T @ Y.T


def rect_qr(A, m_sizes, n_sizes, tol, anorm=None) -> RectQRResult:
    """The Sec. 6 evaluation: dense permuted QR, then Y and R compressed in the rectangular
    format of A (R at tol ||A||_2, Y at tol) and T in the square format of the n-partition
    (at tol)."""
    A = np.asarray(A, dtype=np.float64)
    if anorm is None or anorm <= 0:
        anorm = norm2(A)
    Y, T, R = permuted_qr(A, m_sizes, n_sizes)
    return RectQRResult(compress(Y, m_sizes, n_sizes, tol), compress(T, n_sizes, n_sizes, tol),
                        compress(R, m_sizes, n_sizes, tol * anorm), anorm, tol)


def errors(res: RectQRResult, A):
    """e_orth = ||Q^T Q - I||_2 and e_acc = ||A - Q R||_2 (absolute, as the paper's Eq. (26))
    of the compressed factors."""
    Q = res.Q_dense()
    R = res.R.to_dense()
    e_orth = float(np.linalg.norm(Q.T @ Q - np.eye(Q.shape[0]), 2))
    e_acc = float(np.linalg.norm(A - Q @ R, 2))
    return e_orth, e_acc


def lstsq(res: RectQRResult, B, m_sizes, n_sizes):
    """Least-squares solution of min ||A X - B|| from the permuted QR (the use of a QR
    decomposition the paper's introduction names for rectangular A): with A = Q R and the
    triangle R~ = R[p[:n]], ||A X - B|| = ||R X - Q^T B||, minimized by R~ X = (Q^T B)[p[:n]];
    the rows p[n:] of Q^T B are the residual.  Returns (X, residual norms per column)."""
    import scipy.linalg as sla
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    Y, T, Rd = res.Y.to_dense(), res.T.to_dense(), res.R.to_dense()
    QtB = B - Y @ (T.T @ (Y.T @ B))
    p = row_permutation(m_sizes, n_sizes)
    n = Rd.shape[1]
    X = sla.solve_triangular(Rd[p[:n]], QtB[p[:n]], lower=False)
    return X, np.linalg.norm(QtB[p[n:]], axis=0)
