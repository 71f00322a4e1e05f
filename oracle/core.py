"""CPU FP64 oracle of hQR — Kressner & Susnjara, "Fast QR decomposition of HODLR matrices"
(arXiv:1809.10585).

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously-correct statement of
what the CUDA path computes.  Only the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it; the product path
never does.  It shares no code with the CUDA path.

Everything is float64 numpy.  Library primitives used as single steps: matrix products,
the economy QR and SVD of ``numpy.linalg`` (steps 1 and 2 of the recompression T_eps,
Sec. 2.1.1; the economy QR of the left-orthogonalization, Sec. 2.1), and the dense
triangular solve of ``scipy.linalg`` at the leaves of the back-substitution.  The Householder
reflector and the recursive block QR (Alg. 1) and hQR itself (Alg. 2) are written out here.

Readings of places where the paper is silent or ambiguous:

* Householder reflector (Alg. 1, n = 1): LAPACK dlarfg convention,
  beta = -sign(alpha) * ||x|| where sign takes the sign bit of alpha (so -0.0 counts as
  negative, as in LAPACK),
  gamma = (beta - alpha) / beta, y = [1; x_2 / (alpha - beta)], rho = beta; gamma = 0,
  y = e_1, rho = alpha when x_2 = 0.
* The update of Alg. 1 uses Q_1^T = I - Y_1 T_1^T Y_1^T (the transpose is what Sec. 3
  derives; the printed "(I - Y_1 T Y_1^T)^T" is the same thing).
* Alg. 2, second recursive call: its C argument is the *updated* [B^_{R,2}; C^_2].
* Truncation thresholds: eps * ||A||_2 for S~, A^12 and the HODLR update of A^22;
  plain eps for T~12 (Y and T are scale-free).  k_eps is the smallest k with
  sigma_{k+1} <= threshold (Sec. 2.1.1), i.e. the number of sigma > threshold.
* ||A||_2: ``POWER_ITERS`` power iterations on A^T A from the normalized all-ones vector,
  returning ||A x|| for the final unit vector x.
* S~ and T~12 are truncated once after concatenating all terms (as Alg. 2 writes these two
  steps), not in (l+1)k separate additions.
* Left-orthogonalization (Alg. 2, conditional on B_L lacking orthonormal columns) is always performed; on an
  already orthonormal B_L it only changes column signs up to rounding.
* The HODLR low-rank update  A -_H U V^T  (Table 1) subtracts U_i V_i^T from every dense
  leaf and replaces every off-diagonal block L R^T by T_eps([L, -U_rows][R, V_cols]^T).
"""
from __future__ import annotations

import collections
import math

import numpy as np
import scipy.linalg

POWER_ITERS = 30

# Algorithmic flop counts, keyed by the step of the hot path.  Standard counts per primitive:
#   Householder QR of h x w (R and Y):  2 h w^2 - 2 w^3 / 3
#   compact-WY T of h x w:              h w^2 - w^3 / 3
#   economy QR of h x K plus forming Q: 4 h K^2 - 4 K^3 / 3
#   SVD of a p x q core (p >= q):       4 p^2 q + 8 p q^2 + 9 q^3   (R-SVD, Golub & Van Loan)
#   dense product (m x k)(k x n):       2 m n k
FLOPS = collections.Counter()
# Every truncation's (rows, cols, K_in, k_out, step) is appended here when TRACE is on.
TRACE = []
TRACE_ON = False


def reset_counters():
    FLOPS.clear()
    TRACE.clear()


def _mm(A, B, step):
    FLOPS[step] += 2 * A.shape[0] * A.shape[1] * B.shape[1]
    return A @ B


# --------------------------------------------------------------------------------------
# HODLR container (Sec. 2.1): a node is a dense leaf or a 2x2 block with two children and
# factored off-diagonal blocks A12 = U12 V12^T, A21 = U21 V21^T  (Eq. (3) with A_L = U,
# A_R = V^T).
# --------------------------------------------------------------------------------------
class HNode:
    __slots__ = ("m", "D", "c1", "c2", "U12", "V12", "U21", "V21")

    def __init__(self, m):
        self.m = m
        self.D = None
        self.c1 = self.c2 = None
        self.U12 = self.V12 = self.U21 = self.V21 = None

    @property
    def leaf(self):
        return self.c1 is None

    @staticmethod
    def make_leaf(D):
        h = HNode(D.shape[0])
        h.D = np.array(D, dtype=np.float64)
        return h

    @staticmethod
    def make_internal(c1, c2, U12, V12, U21, V21):
        h = HNode(c1.m + c2.m)
        h.c1, h.c2 = c1, c2
        h.U12, h.V12 = np.array(U12, dtype=np.float64), np.array(V12, dtype=np.float64)
        h.U21, h.V21 = np.array(U21, dtype=np.float64), np.array(V21, dtype=np.float64)
        return h

    def copy(self):
        if self.leaf:
            return HNode.make_leaf(self.D)
        return HNode.make_internal(self.c1.copy(), self.c2.copy(), self.U12, self.V12,
                                   self.U21, self.V21)


def from_input(inp) -> HNode:
    """Build the oracle's tree from a workloads.HodlrInput (heap-ordered node lists)."""
    nleaf = len(inp.leaf_sizes)

    def build(v):
        if v >= nleaf - 1:
            return HNode.make_leaf(inp.leaves[v - (nleaf - 1)])
        return HNode.make_internal(build(2 * v + 1), build(2 * v + 2),
                                   inp.U12[v], inp.V12[v], inp.U21[v], inp.V21[v])

    return build(0)


def compress(A, leaf_sizes, thr) -> HNode:
    """HODLR approximation of a dense matrix by the construction of Sec. 2.1.1: on the cluster
    tree of the partition ``leaf_sizes`` (first half of every split to the first child), the
    diagonal blocks of the leaves are kept dense and every off-diagonal block A12 / A21 of an
    internal node is replaced by its truncated SVD, the singular triplets with sigma > thr
    (U = left vectors, V = right vectors times sigma)."""
    A = np.asarray(A, dtype=np.float64)
    offs = np.concatenate([[0], np.cumsum(leaf_sizes)]).astype(int)
    nleaf = len(leaf_sizes)

    def block_svd(B):
        u, sv, vt = _svd(B)
        k = int(np.sum(sv > thr))
        return np.asfortranarray(u[:, :k]), np.asfortranarray(vt[:k].T * sv[:k][None, :])

    def build(first, count):
        lo, hi = offs[first], offs[first + count]
        if count == 1:
            return HNode.make_leaf(np.asfortranarray(A[lo:hi, lo:hi]))
        h = count // 2
        mid = offs[first + h]
        U12, V12 = block_svd(A[lo:mid, mid:hi])
        U21, V21 = block_svd(A[mid:hi, lo:mid])
        return HNode.make_internal(build(first, h), build(first + h, count - h), U12, V12, U21, V21)

    return build(0, nleaf)

def to_dense(H: HNode, part="full") -> np.ndarray:
    """Dense matrix of a HODLR node.  part='full' | 'unit_lower' (strictly lower leaves, unit
    diagonal, lower blocks) | 'upper' (upper-triangular leaves and upper blocks)."""
    if H.leaf:
        if part == "unit_lower":
            return np.tril(H.D, -1) + np.eye(H.m)
        if part == "upper":
            return np.triu(H.D)
        return H.D.copy()
    m1 = H.c1.m
    A = np.zeros((H.m, H.m))
    A[:m1, :m1] = to_dense(H.c1, part)
    A[m1:, m1:] = to_dense(H.c2, part)
    if part in ("full", "upper"):
        A[:m1, m1:] = H.U12 @ H.V12.T
    if part in ("full", "unit_lower"):
        A[m1:, :m1] = H.U21 @ H.V21.T
    return A


def max_offdiag_rank(H: HNode, which="both"):
    if H.leaf:
        return 0
    r = max(max_offdiag_rank(H.c1, which), max_offdiag_rank(H.c2, which))
    if which in ("both", "upper"):
        r = max(r, H.U12.shape[1])
    if which in ("both", "lower"):
        r = max(r, H.U21.shape[1])
    return r


def matmat(H: HNode, X: np.ndarray, trans=False, part="full", step="matvec") -> np.ndarray:
    """op(H) @ X for a block of vectors X (Table 1, matrix-vector multiplication with
    several vectors at once).  op = transpose when trans; part selects the triangular parts
    as in to_dense."""
    X = np.asarray(X, dtype=np.float64)
    if H.leaf:
        if part == "unit_lower":
            D = np.tril(H.D, -1) + np.eye(H.m)
            FLOPS[step] += H.m * H.m * X.shape[1]
        elif part == "upper":
            D = np.triu(H.D)
            FLOPS[step] += H.m * H.m * X.shape[1]
        else:
            D = H.D
            FLOPS[step] += 2 * H.m * H.m * X.shape[1]
        return (D.T if trans else D) @ X
    m1 = H.c1.m
    X1, X2 = X[:m1], X[m1:]
    Y1 = matmat(H.c1, X1, trans, part, step)
    Y2 = matmat(H.c2, X2, trans, part, step)
    up = part in ("full", "upper")
    lo = part in ("full", "unit_lower")
    if not trans:
        if up:
            Y1 = Y1 + _mm(H.U12, _mm(H.V12.T, X2, step), step)
        if lo:
            Y2 = Y2 + _mm(H.U21, _mm(H.V21.T, X1, step), step)
    else:
        # H^T = [[A11^T, A21^T], [A12^T, A22^T]],  A21^T = V21 U21^T,  A12^T = V12 U12^T
        if lo:
            Y1 = Y1 + _mm(H.V21, _mm(H.U21.T, X2, step), step)
        if up:
            Y2 = Y2 + _mm(H.V12, _mm(H.U12.T, X1, step), step)
    return np.vstack([Y1, Y2])


# --------------------------------------------------------------------------------------
# Low-rank primitives (Sec. 2.1 and 2.1.1)
# --------------------------------------------------------------------------------------
def _econ_qr(A, step):
    h, K = A.shape
    q = min(h, K)
    FLOPS[step] += max(0, int(4 * h * K * q - 4 * q ** 3 / 3))
    return np.linalg.qr(A, mode="reduced")


def _svd(M):
    """Economy SVD (the SVD of Sec. 2.1.1).  LAPACK's divide-and-conquer driver (dgesdd) can
    fail to converge on rare, strongly graded cores; the QR-iteration driver (dgesvd) then
    computes the same decomposition."""
    try:
        return np.linalg.svd(M, full_matrices=False)
    except np.linalg.LinAlgError:
        return scipy.linalg.svd(M, full_matrices=False, lapack_driver="gesvd")


def left_orthogonalize(L, Rt, step="a3_left_orth"):
    """Left-orthogonal form of the block L Rt^T (Sec. 2.1): L = Q R, L <- Q, Rt <- Rt R^T."""
    Q, R = _econ_qr(L, step)
    return Q, _mm(Rt, R.T, step)


def truncate(L, Rt, eps, step="a9_recompress"):
    """Recompression T_eps of the block L Rt^T (Sec. 2.1.1):
    1. L = Q1 R1 and Rt = Q2 R2 (economy QR),
    2. SVD  R1 R2^T = U~ S V~^T,
    3. keep k_eps = #{sigma_i > eps}:  L <- Q1 U~_k,  Rt <- Q2 V~_k S_k.
    Returns (L_new, Rt_new); L_new has orthonormal columns."""
    L = np.asarray(L, dtype=np.float64)
    Rt = np.asarray(Rt, dtype=np.float64)
    nL, K = L.shape
    nR = Rt.shape[0]
    if K == 0 or nL == 0 or nR == 0:
        return np.zeros((nL, 0)), np.zeros((nR, 0))
    Q1, R1 = _econ_qr(L, step)
    Q2, R2 = _econ_qr(Rt, step)
    M = _mm(R1, R2.T, step)
    p, q = max(M.shape), min(M.shape)
    FLOPS[step] += 4 * p * p * q + 8 * p * q * q + 9 * q ** 3
    Ut, s, Vth = _svd(M)
    k = int(np.sum(s > eps))
    if TRACE_ON:
        TRACE.append((step, nL, nR, K, k))
    Ln = _mm(Q1, Ut[:, :k], step)
    Rn = _mm(Q2, Vth[:k].T * s[:k][None, :], step)
    return Ln, Rn


def lr_update(H: HNode, U, V, eps, step="a7_update"):
    """HODLR low-rank update  H <- H -_H U V^T  (Table 1): dense subtraction at the leaves,
    append-and-recompress T_eps in every off-diagonal block.  Modifies H in place."""
    if U.shape[1] == 0:
        return
    if H.leaf:
        H.D = H.D - _mm(U, V.T, step)
        return
    m1 = H.c1.m
    U1, U2 = U[:m1], U[m1:]
    V1, V2 = V[:m1], V[m1:]
    H.U12, H.V12 = truncate(np.hstack([H.U12, -U1]), np.hstack([H.V12, V2]), eps, step)
    H.U21, H.V21 = truncate(np.hstack([H.U21, -U2]), np.hstack([H.V21, V1]), eps, step)
    lr_update(H.c1, U1, V1, eps, step)
    lr_update(H.c2, U2, V2, eps, step)


# --------------------------------------------------------------------------------------
# Dense recursive block QR (Alg. 1)
# --------------------------------------------------------------------------------------
def _scaled_norm(v):
    """||v||_2 without overflow or underflow of the squares: v is divided by its largest
    magnitude first, as LAPACK's dnrm2 (the norm inside dlarfg) avoids the same."""
    if v.shape[0] == 0:
        return 0.0
    m = float(np.max(np.abs(v)))
    if m == 0.0:
        return 0.0
    w = v / m
    return m * math.sqrt(float(w @ w))


def householder(x):
    """Reflector I - gamma y y^T with (I - gamma y y^T) x = rho e_1 (Alg. 1, n = 1),
    LAPACK dlarfg sign convention."""
    x = np.asarray(x, dtype=np.float64)
    alpha = float(x[0])
    xnorm = _scaled_norm(x[1:])
    y = np.zeros_like(x)
    y[0] = 1.0
    if xnorm == 0.0:
        return y, 0.0, alpha
    h = math.hypot(alpha, xnorm)
    beta = -math.copysign(h, alpha)
    gamma = (beta - alpha) / beta
    y[1:] = x[1:] / (alpha - beta)
    return y, gamma, beta


def block_qr(A):
    """Recursive block QR of Elmroth & Gustavson (Alg. 1), recursion down to single
    columns.  A is m x n with m >= n.  Returns Y (m x n, unit lower trapezoidal),
    T (n x n upper), R (n x n upper) with A = (I - Y T Y^T) [R; 0]."""
    A = np.array(A, dtype=np.float64)
    m, n = A.shape
    if m < n:
        raise ValueError("block_qr needs m >= n")
    if n == 1:
        y, gamma, rho = householder(A[:, 0])
        return y[:, None], np.array([[gamma]]), np.array([[rho]])
    n1 = n // 2
    Y1, T1, R1 = block_qr(A[:, :n1])
    A2 = A[:, n1:]
    A2 = A2 - Y1 @ (T1.T @ (Y1.T @ A2))            # Q_1^T A_2
    Y2, T2, R2 = block_qr(A2[n1:, :])
    Y2t = np.vstack([np.zeros((n1, n - n1)), Y2])
    T12 = -T1 @ (Y1.T @ Y2t) @ T2
    Y = np.hstack([Y1, Y2t])
    T = np.block([[T1, T12], [np.zeros((n - n1, n1)), T2]])
    R = np.block([[R1, A2[:n1]], [np.zeros((n - n1, n1)), R2]])
    return Y, T, R


def dense_qr_flops(h, w):
    """Algorithmic flops of a dense Householder QR of h x w with its T factor."""
    return int(2 * h * w * w - 2 * w ** 3 / 3) + int(h * w * w - w ** 3 / 3)


# --------------------------------------------------------------------------------------
# hQR (Alg. 2)
# --------------------------------------------------------------------------------------
def hqr_node(At: HNode, BL, BR, C, epsA, epsT):
    """One call  [Y, T, R] = hQR(A~, B, C)  of Alg. 2.

    At : HODLR node A~ (m x m); consumed (its storage is reused for the result).
    BL, BR : factors of B = BL @ BR (p x r1, r1 x m), or None when B is void.
    C  : r2 x m dense rows.
    Returns (YR, YBt, YC, T, BLq):
      YR  — one HODLR node holding Y_A (strictly lower leaves + lower blocks, unit diagonal
            implied) and R (upper-triangular leaves + upper blocks), LAPACK-style;
            the lower block of YR at each node is Y_{A,21} = B_L(orthonormal) @ Y~_B.
      YBt — Y~_B (r1 x m), so that Y_B = BLq @ YBt;  YC — Y_C (r2 x m);
      T   — upper-triangular HODLR node;  BLq — the orthonormalized B_L (or None).
    """
    m = At.m
    C = np.zeros((0, m)) if C is None else np.asarray(C, dtype=np.float64)
    if BL is not None:
        BL, BR = left_orthogonalize(BL, np.asarray(BR, dtype=np.float64).T)   # Alg. 2, first step
        BR = BR.T
    else:
        BR = np.zeros((0, m))
    r1 = BR.shape[0]
    if At.leaf:                                                            # lowest level
        Ht = np.vstack([At.D, BR, C])
        Y, T, R = block_qr(Ht)
        FLOPS["a4_leaf_qr"] += dense_qr_flops(Ht.shape[0], m)
        YR = HNode.make_leaf(np.triu(R) + np.tril(Y[:m], -1))
        return YR, Y[m:m + r1], Y[m + r1:], HNode.make_leaf(T), BL
    m1 = At.c1.m
    m2 = m - m1
    U12, V12, U21, V21 = At.U12, At.V12, At.U21, At.V21
    BR1, BR2 = BR[:, :m1], BR[:, m1:]
    C1, C2 = C[:, :m1], C[:, m1:]
    # first block column, recursively:  hQR(A~11, A~21, [B_R1; C1])
    YR11, Yt21, YC1s, T1, BL21 = hqr_node(At.c1, U21, V21.T, np.vstack([BR1, C1]), epsA, epsT)
    YBR1, YCC1 = YC1s[:r1], YC1s[r1:]
    # S~ = T_{eps||A||}( Y_A11^T A~12 + Y_A21^T A~22 + Y_BR1^T B_R2 + Y_C1^T C2 )
    #   Y_A11^T A~12 = (Y_A11^T U12) V12^T;  Y_A21^T A~22 = Y~_B^T (A~22^T B_L21)^T
    L = np.hstack([matmat(YR11, U12, True, "unit_lower", "a5_S"), Yt21.T, YBR1.T, YCC1.T])
    Rt = np.hstack([V12, matmat(At.c2, BL21, True, "full", "a5_S"), BR2.T, C2.T])
    SL, SRt = truncate(L, Rt, epsA, "a5_S")
    # S = T1^T S~
    SL = matmat(T1, SL, True, "upper", "a6_TS")
    # update of the second block column
    U12n, V12n = truncate(np.hstack([U12, -matmat(YR11, SL, False, "unit_lower", "a7_update")]),
                          np.hstack([V12, SRt]), epsA, "a7_update")
    Yt21SL = _mm(Yt21, SL, "a7_update")
    A22 = At.c2
    lr_update(A22, _mm(BL21, Yt21SL, "a7_update"), SRt, epsA, "a7_update")
    BR2 = BR2 - _mm(_mm(YBR1, SL, "a7_update"), SRt.T, "a7_update")
    C2 = C2 - _mm(_mm(YCC1, SL, "a7_update"), SRt.T, "a7_update")
    # second block column, recursively:  hQR(A^22, [], [B^_R2; C^2])
    YR22, _, YC2s, T2, _ = hqr_node(A22, None, None, np.vstack([BR2, C2]), epsA, epsT)
    YBR2, YCC2 = YC2s[:r1], YC2s[r1:]
    # T~12 = T_eps( Y_A21^T Y_A22 + Y_BR1^T Y_BR2 + Y_C1^T Y_C2 ),  T12 = -T1 T~12 T2
    L = np.hstack([Yt21.T, YBR1.T, YCC1.T])
    Rt = np.hstack([matmat(YR22, BL21, True, "unit_lower", "a8_T12"), YBR2.T, YCC2.T])
    TL, TRt = truncate(L, Rt, epsT, "a8_T12")
    T12U = -matmat(T1, TL, False, "upper", "a8_T12")
    T12V = matmat(T2, TRt, True, "upper", "a8_T12")
    YR = HNode.make_internal(YR11, YR22, U12n, V12n, BL21, Yt21.T)
    T = HNode.make_internal(T1, T2, T12U, T12V, np.zeros((m2, 0)), np.zeros((m1, 0)))
    return YR, np.hstack([YBR1, YBR2]), np.hstack([YCC1, YCC2]), T, BL


def norm2_estimate(H: HNode, iters=POWER_ITERS) -> float:
    """||A||_2 by power iteration on A^T A from the normalized all-ones vector (the paper
    does not say how ||A||_2 is obtained)."""
    x = np.ones((H.m, 1)) / math.sqrt(H.m)
    for _ in range(iters):
        z = matmat(H, matmat(H, x, False, "full", "a2_norm"), True, "full", "a2_norm")
        s = float(np.linalg.norm(z))
        if s == 0.0:
            return 0.0
        x = z / s
    return float(np.linalg.norm(matmat(H, x, False, "full", "a2_norm")))


class QRResult:
    """Y and R share one HODLR tree (YR), T is a second tree; anorm is the ||A||_2 used."""

    def __init__(self, YR, T, anorm, tol):
        self.YR, self.T, self.anorm, self.tol = YR, T, anorm, tol

    def Y_dense(self):
        return to_dense(self.YR, "unit_lower")

    def R_dense(self):
        return to_dense(self.YR, "upper")

    def T_dense(self):
        return to_dense(self.T, "upper")

    def Q_dense(self):
        Y, T = self.Y_dense(), self.T_dense()
        return np.eye(Y.shape[0]) - Y @ T @ Y.T


def hqr(A: HNode, tol: float, anorm: float | None = None) -> QRResult:
    """QR decomposition A = (I - Y T Y^T) R of a HODLR matrix by Alg. 2 applied with
    A~ = A and void B, C.  A is not modified."""
    A = A.copy()
    if anorm is None or anorm <= 0:
        anorm = norm2_estimate(A)
    YR, _, _, T, _ = hqr_node(A, None, None, None, tol * anorm, tol)
    return QRResult(YR, T, anorm, tol)


# --------------------------------------------------------------------------------------
# Apply / solve (Q = I - Y T Y^T, Sec. 1; HODLR triangular solve, Table 1)
# --------------------------------------------------------------------------------------
def apply_qt(res: QRResult, B):
    """Q^T B = B - Y T^T Y^T B."""
    W = matmat(res.YR, B, True, "unit_lower", "a10_apply")
    W = matmat(res.T, W, True, "upper", "a10_apply")
    return B - matmat(res.YR, W, False, "unit_lower", "a10_apply")


def apply_q(res: QRResult, B):
    """Q B = B - Y T Y^T B."""
    W = matmat(res.YR, B, True, "unit_lower", "a10_apply")
    W = matmat(res.T, W, False, "upper", "a10_apply")
    return B - matmat(res.YR, W, False, "unit_lower", "a10_apply")


def upper_solve(R: HNode, B):
    """Back-substitution with the upper-triangular HODLR matrix R (upper part of R):
    x2 = R22^{-1} b2,  x1 = R11^{-1} (b1 - R12 x2)."""
    if R.leaf:
        FLOPS["a10_solve"] += R.m * R.m * B.shape[1]
        return scipy.linalg.solve_triangular(np.triu(R.D), B, lower=False)
    m1 = R.c1.m
    x2 = upper_solve(R.c2, B[m1:])
    b1 = B[:m1] - _mm(R.U12, _mm(R.V12.T, x2, "a10_solve"), "a10_solve")
    x1 = upper_solve(R.c1, b1)
    return np.vstack([x1, x2])


def solve(res: QRResult, B):
    """x = R^{-1} Q^T B."""
    return upper_solve(res.YR, apply_qt(res, np.asarray(B, dtype=np.float64)))


# --------------------------------------------------------------------------------------
# Accuracy measures (Sec. 5):  e_orth = ||Q^T Q - I||_2,  e_acc = ||Q R - A||_2
# --------------------------------------------------------------------------------------
def errors_dense(res: QRResult, A_dense):
    Q = res.Q_dense()
    R = res.R_dense()
    n = Q.shape[0]
    e_orth = float(np.linalg.norm(Q.T @ Q - np.eye(n), 2))
    e_acc = float(np.linalg.norm(Q @ R - A_dense, 2))
    return e_orth, e_acc


def errors_power(res: QRResult, A: HNode, iters=40, seed=0):
    """e_orth and e_acc by power iteration with HODLR operations only (large n)."""
    n = A.m
    rng = np.random.default_rng(seed)

    def orth_op(x):
        return apply_qt(res, apply_q(res, x)) - x

    def acc_op(x, t):
        if not t:
            return apply_q(res, matmat(res.YR, x, False, "upper")) - matmat(A, x)
        return matmat(res.YR, apply_qt(res, x), True, "upper") - matmat(A, x, True)

    x = rng.standard_normal((n, 1)); x /= np.linalg.norm(x)
    e_orth = 0.0
    for _ in range(iters):
        y = orth_op(x)
        e_orth = float(np.linalg.norm(y))
        if e_orth == 0:
            break
        x = y / e_orth
    x = rng.standard_normal((n, 1)); x /= np.linalg.norm(x)
    e_acc = 0.0
    for _ in range(iters):
        z = acc_op(acc_op(x, False), True)
        s = float(np.linalg.norm(z))
        if s == 0:
            break
        x = z / s
    e_acc = float(np.linalg.norm(acc_op(x, False)))
    return e_orth, e_acc
