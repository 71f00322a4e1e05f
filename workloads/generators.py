"""Seeded synthetic HODLR inputs shaped like the workloads of Kressner & Susnjara,
"Fast QR decomposition of HODLR matrices" (arXiv:1809.10585).

This module only draws random numbers and lays them out as a HODLR input description.
It contains none of the QR method's arithmetic, so both the CPU oracle and the CUDA path
can consume its output without sharing any numerical code.

Layout of a HODLR input (the integer partition of Sec. 2.1, Eq. (2), and the factored
off-diagonal blocks of Eq. (3)):

* ``leaf_sizes``: the partition ``n = n_1 + ... + n_{2^l}``.
* Nodes of the cluster tree are numbered in heap order: root 0, children of ``v`` are
  ``2v+1`` (rows/columns first) and ``2v+2``. Internal nodes are ``0 .. 2^l - 2``.
* ``leaves[j]``: dense ``n_j x n_j`` diagonal block ``j`` (float64, C or F order).
* For internal node ``v`` with children ``c1``, ``c2`` of sizes ``m1``, ``m2``:
  ``U12[v] (m1 x r)``, ``V12[v] (m2 x r)`` give the upper block ``A12 = U12 @ V12.T``;
  ``U21[v] (m2 x r)``, ``V21[v] (m1 x r)`` give the lower block ``A21 = U21 @ V21.T``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class HodlrInput:
    n: int
    leaf_sizes: list
    leaves: list
    U12: list
    V12: list
    U21: list
    V21: list
    name: str = ""

    @property
    def levels(self) -> int:
        return int(round(math.log2(len(self.leaf_sizes))))


def balanced_leaf_sizes(n: int, nmin: int) -> list:
    """Balanced integer partition: the smallest level l with ceil(n / 2^l) <= nmin, each
    split giving floor(m/2) to the first half (the 'nearly equal' advice of Sec. 2.1)."""
    if n <= 0 or nmin <= 0:
        raise ValueError("n and nmin must be positive")
    levels = 0
    while -(-n // (1 << levels)) > nmin:
        levels += 1
    sizes = [n]
    for _ in range(levels):
        nxt = []
        for m in sizes:
            nxt += [m // 2, m - m // 2]
        sizes = nxt
    return sizes


def node_ranges(leaf_sizes) -> list:
    """(lo, hi) for every heap-ordered node of the cluster tree defined by leaf_sizes."""
    nleaf = len(leaf_sizes)
    levels = int(round(math.log2(nleaf)))
    if (1 << levels) != nleaf:
        raise ValueError("number of leaves must be a power of two")
    nnodes = 2 * nleaf - 1
    rng = [None] * nnodes
    off = 0
    for j, s in enumerate(leaf_sizes):
        rng[nleaf - 1 + j] = (off, off + s)
        off += s
    for v in range(nleaf - 2, -1, -1):
        rng[v] = (rng[2 * v + 1][0], rng[2 * v + 2][1])
    return rng


def random_hodlr(n, nmin, k, seed=0, leaf_shift=4.0, factor_scale=None, leaf_sizes=None,
                 col_scale_decades=0.0, rank_fn=None, name="") -> HodlrInput:
    """Random HODLR matrix: dense N(0,1) leaves plus ``leaf_shift * I`` and off-diagonal
    blocks U V^T with i.i.d. N(0,1)/sqrt(n) factors of rank k (the random HODLR matrices of
    Example 5.1, with rank k instead of 1).

    ``col_scale_decades = d`` additionally scales column j by 10^(-d j/(n-1)) (this keeps every
    off-diagonal rank: only the right factors and the leaves change).  ``rank_fn(v, which)``
    may override the rank of a block.
    """
    rng = np.random.default_rng(seed)
    sizes = list(leaf_sizes) if leaf_sizes is not None else balanced_leaf_sizes(n, nmin)
    if sum(sizes) != n:
        raise ValueError("leaf sizes must sum to n")
    ranges = node_ranges(sizes)
    nleaf = len(sizes)
    fs = (1.0 / math.sqrt(n)) if factor_scale is None else factor_scale
    if col_scale_decades:
        dcol = 10.0 ** (-col_scale_decades * np.arange(n) / max(n - 1, 1))
    else:
        dcol = None
    leaves = []
    for j in range(nleaf):
        lo, hi = ranges[nleaf - 1 + j]
        m = hi - lo
        D = rng.standard_normal((m, m)) + leaf_shift * np.eye(m)
        if dcol is not None:
            D = D * dcol[lo:hi][None, :]
        leaves.append(np.asfortranarray(D))
    U12, V12, U21, V21 = [], [], [], []
    for v in range(nleaf - 1):
        lo1, hi1 = ranges[2 * v + 1]
        lo2, hi2 = ranges[2 * v + 2]
        m1, m2 = hi1 - lo1, hi2 - lo2
        r12 = k if rank_fn is None else rank_fn(v, "12")
        r21 = k if rank_fn is None else rank_fn(v, "21")
        u12 = rng.standard_normal((m1, r12)) * fs
        v12 = rng.standard_normal((m2, r12)) * fs
        u21 = rng.standard_normal((m2, r21)) * fs
        v21 = rng.standard_normal((m1, r21)) * fs
        if dcol is not None:
            v12 = v12 * dcol[lo2:hi2][:, None]
            v21 = v21 * dcol[lo1:hi1][:, None]
        U12.append(np.asfortranarray(u12)); V12.append(np.asfortranarray(v12))
        U21.append(np.asfortranarray(u21)); V21.append(np.asfortranarray(v21))
    return HodlrInput(n, sizes, leaves, U12, V12, U21, V21, name=name)


def config0(seed=0) -> HodlrInput:
    """Plain HODLR QR workload: n=1024, nmin=128 (3 levels), rank 5 Gaussian factors
    scaled by 1/sqrt(n), leaves N(0,1) + 4 I."""
    return random_hodlr(1024, 128, 5, seed=seed, name="n1024_nmin128_k5")


def config1(seed=0) -> HodlrInput:
    """Ill-conditioned HODLR QR workload: n=8192, nmin=256, rank 10, then columns scaled by
    10^(-14 j/(n-1)) (condition number about 1e14)."""
    return random_hodlr(8192, 256, 10, seed=seed, col_scale_decades=14.0,
                        name="n8192_nmin256_k10_colscaled1e-14")


def scaled_config1(n, nmin, k=10, seed=0, decades=14.0) -> HodlrInput:
    """Same family as config1 at another size (parity cases the oracle finishes quickly)."""
    return random_hodlr(n, nmin, k, seed=seed, col_scale_decades=decades,
                        name=f"n{n}_nmin{nmin}_k{k}_colscaled1e-{decades:g}")


def rank1_example(n, nmin=250, seed=0) -> HodlrInput:
    """Example 5.1: dense random leaves, every off-diagonal block an outer product of two
    random vectors.  Distributions are not stated in the paper; N(0,1) entries are used."""
    return random_hodlr(n, nmin, 1, seed=seed, leaf_shift=0.0, factor_scale=1.0,
                        name=f"rank1_n{n}")


def zero_rank(n, nmin, seed=0) -> HodlrInput:
    """Block-diagonal HODLR matrix (every off-diagonal rank zero)."""
    return random_hodlr(n, nmin, 0, seed=seed, name=f"zero_rank_n{n}")


def cauchy_points(which: int, n=2000, seed=0):
    """Points of the Cauchy matrices A_1..A_3 of Example 5.2: n equally spaced points on I_x
    and I_y, each perturbed by +-2e-2 with a random sign (Rademacher draws from ``seed``)."""
    ix = (-1.25, 998.25)
    iy = {1: (-0.7, 998.9), 2: (-0.45, 999.15), 3: (-0.15, 999.45)}[which]
    rng = np.random.default_rng(seed)
    sx = rng.choice([-1.0, 1.0], size=n)
    sy = rng.choice([-1.0, 1.0], size=n)
    x = np.linspace(ix[0], ix[1], n) + 2e-2 * sx
    y = np.linspace(iy[0], iy[1], n) + 2e-2 * sy
    return x, y


def cauchy_dense(which: int, n=2000, seed=0) -> np.ndarray:
    """Dense Cauchy matrix (x_i - y_j)^{-1} of Example 5.2."""
    x, y = cauchy_points(which, n, seed)
    return 1.0 / (x[:, None] - y[None, :])


def kernel_points(n, seed=0):
    """Points for the kernel-generated nonsymmetric workload A_ij = 1/(x_i - y_j): x sorted
    uniform on [0, 1], y_j = x_j + 0.5/n."""
    rng = np.random.default_rng(seed)
    x = np.sort(rng.uniform(0.0, 1.0, n))
    y = x + 0.5 / n
    return x, y


def dense_to_hodlr_input(A, nmin, eps, leaf_sizes=None, name="") -> HodlrInput:
    """Lay a dense matrix out as a HODLR input by truncated SVD of every off-diagonal block,
    keeping the singular triplets with sigma > eps (the construction of Sec. 2.1.1).  Used only
    to prepare inputs such as the Cauchy matrices; the QR method never calls it."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    sizes = list(leaf_sizes) if leaf_sizes is not None else balanced_leaf_sizes(n, nmin)
    ranges = node_ranges(sizes)
    nleaf = len(sizes)
    leaves = []
    for j in range(nleaf):
        lo, hi = ranges[nleaf - 1 + j]
        leaves.append(np.asfortranarray(A[lo:hi, lo:hi]))
    U12, V12, U21, V21 = [], [], [], []
    for v in range(nleaf - 1):
        lo1, hi1 = ranges[2 * v + 1]
        lo2, hi2 = ranges[2 * v + 2]
        for (rlo, rhi, clo, chi, Ul, Vl) in ((lo1, hi1, lo2, hi2, U12, V12),
                                             (lo2, hi2, lo1, hi1, U21, V21)):
            u, s, vt = np.linalg.svd(A[rlo:rhi, clo:chi], full_matrices=False)
            k = int(np.sum(s > eps))
            Ul.append(np.asfortranarray(u[:, :k]))
            Vl.append(np.asfortranarray(vt[:k].T * s[:k][None, :]))
    return HodlrInput(n, sizes, leaves, U12, V12, U21, V21, name=name)


def kernel_hodlr(n, nmin, eps=1e-12, seed=0, shift=None, samples=64, device="cpu", name="") -> HodlrInput:
    """Kernel-generated nonsymmetric workload: A_ij = 1/(x_i - y_j) with the points of
    ``kernel_points``, ``shift`` (default n) added to the diagonal, every off-diagonal block
    replaced by its singular triplets with sigma > eps * sigma_1(block).

    Blocks are never held whole: each is sampled by a randomized range finder (Halko, Martinsson
    and Tropp, SIAM Review 2011, Alg. 4.1) from row panels generated on the fly, and the SVD of
    the projected block gives the truncation; the sample count doubles until the smallest
    captured singular value falls below eps * sigma_1.  The arithmetic runs in torch float64 on
    ``device`` (input preparation only; the QR method never calls this)."""
    import torch
    dev = torch.device(device)
    x_np, y_np = kernel_points(n, seed)
    x = torch.from_numpy(x_np).to(dev)
    y = torch.from_numpy(y_np).to(dev)
    shift = float(n) if shift is None else float(shift)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1000003 * seed + 7)
    sizes = balanced_leaf_sizes(n, nmin)
    ranges = node_ranges(sizes)
    nleaf = len(sizes)
    leaves = []
    for j in range(nleaf):
        lo, hi = ranges[nleaf - 1 + j]
        D = 1.0 / (x[lo:hi, None] - y[None, lo:hi])
        D += shift * torch.eye(hi - lo, dtype=torch.float64, device=dev)
        leaves.append(np.asfortranarray(D.cpu().numpy()))

    def panel_rows(m2):
        return max(1, min(1 << 14, (1 << 25) // max(m2, 1)))

    def compress(rlo, rhi, clo, chi):
        m1, m2 = rhi - rlo, chi - clo
        xs, ys = x[rlo:rhi], y[clo:chi]
        p = min(samples, m1, m2)
        while True:
            Om = torch.randn(m2, p, dtype=torch.float64, device=dev, generator=gen)
            Y = torch.empty(m1, p, dtype=torch.float64, device=dev)
            step = panel_rows(m2)
            for a in range(0, m1, step):
                Y[a:a + step] = (1.0 / (xs[a:a + step, None] - ys[None, :])) @ Om
            Q, _ = torch.linalg.qr(Y)
            Bt = torch.zeros(p, m2, dtype=torch.float64, device=dev)      # Q^T B
            for a in range(0, m1, step):
                Bt += Q[a:a + step].T @ (1.0 / (xs[a:a + step, None] - ys[None, :]))
            Ub, sv, Vh = torch.linalg.svd(Bt, full_matrices=False)
            if sv[-1] <= eps * sv[0] or p >= min(m1, m2):
                break
            p = min(2 * p, m1, m2)
        k = int((sv > eps * sv[0]).sum().item())
        U = (Q @ Ub[:, :k]).cpu().numpy()
        V = (Vh[:k].T * sv[:k][None, :]).cpu().numpy()
        return np.asfortranarray(U), np.asfortranarray(V)

    U12, V12, U21, V21 = [], [], [], []
    for v in range(nleaf - 1):
        lo1, hi1 = ranges[2 * v + 1]
        lo2, hi2 = ranges[2 * v + 2]
        u, w = compress(lo1, hi1, lo2, hi2)
        U12.append(u); V12.append(w)
        u, w = compress(lo2, hi2, lo1, hi1)
        U21.append(u); V21.append(w)
    return HodlrInput(n, sizes, leaves, U12, V12, U21, V21, name=name or f"kernel_n{n}_nmin{nmin}")


def banded_hodlr(n, b=8, nmin=256, seed=0, name="") -> HodlrInput:
    """Symmetric banded matrix: entries N(0,1) for 0 < |i - j| <= b (mirrored), N(0,1) + 2b on
    the diagonal.  An off-diagonal block of the HODLR partition is nonzero only in the b x b
    corner next to the diagonal, so it is stored exactly with rank b: a selection of b rows
    times those rows of the block."""
    if b < 0 or nmin <= b:
        raise ValueError("need 0 <= b < nmin")
    rng = np.random.default_rng(seed)
    diag = rng.standard_normal(n) + 2.0 * b
    off = rng.standard_normal((b, n))            # off[k-1, i] = A[i, i+k] = A[i+k, i]

    def entry_block(r0, r1, c0, c1):
        B = np.zeros((r1 - r0, c1 - c0))
        for i in range(r0, r1):
            for j in range(max(c0, i - b), min(c1, i + b + 1)):
                if i == j:
                    B[i - r0, j - c0] = diag[i]
                else:
                    lo = min(i, j)
                    B[i - r0, j - c0] = off[abs(i - j) - 1, lo]
        return B

    sizes = balanced_leaf_sizes(n, nmin)
    ranges = node_ranges(sizes)
    nleaf = len(sizes)
    leaves = []
    for j in range(nleaf):
        lo, hi = ranges[nleaf - 1 + j]
        leaves.append(np.asfortranarray(entry_block(lo, hi, lo, hi)))
    U12, V12, U21, V21 = [], [], [], []
    for v in range(nleaf - 1):
        lo1, hi1 = ranges[2 * v + 1]
        lo2, hi2 = ranges[2 * v + 2]
        m1, m2 = hi1 - lo1, hi2 - lo2
        # A12: rows hi1-b..hi1-1 of the first child against the columns of the second
        S = np.zeros((m1, b)); S[m1 - b:, :] = np.eye(b)
        C = entry_block(hi1 - b, hi1, lo2, hi2)                    # b x m2
        U12.append(np.asfortranarray(S)); V12.append(np.asfortranarray(C.T))
        # A21 = A12^T
        U21.append(np.asfortranarray(C.T.copy())); V21.append(np.asfortranarray(S.copy()))
    return HodlrInput(n, sizes, leaves, U12, V12, U21, V21, name=name or f"banded_n{n}_b{b}")


def batched_family(count=256, seed0=0, nmin_choices=(128, 256), n_lo=2048, n_hi=32768):
    """Cross-matrix batch: n log-uniform in [n_lo, n_hi] rounded to nmin * 2^l, nmin from
    nmin_choices, ranks uniform in [5, 20], every second matrix column-scaled to kappa ~ 1e10."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        nmin = int(rng.choice(nmin_choices))
        n_target = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        lev = max(0, int(round(math.log2(n_target / nmin))))
        n = nmin * (1 << lev)
        k = int(rng.integers(5, 21))
        dec = 10.0 if (i % 2 == 1) else 0.0
        out.append(random_hodlr(n, nmin, k, seed=seed0 + i, col_scale_decades=dec,
                                name=f"batch{i}_n{n}_nmin{nmin}_k{k}"))
    return out


def rhs(n, nrhs, seed=0) -> np.ndarray:
    """Right-hand sides with N(0,1) entries, column-major."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((n, nrhs)))


def to_dense(h: HodlrInput) -> np.ndarray:
    """Assemble the dense matrix described by a HODLR input (a plain layout step)."""
    A = np.zeros((h.n, h.n))
    ranges = node_ranges(h.leaf_sizes)
    nleaf = len(h.leaf_sizes)
    for j in range(nleaf):
        lo, hi = ranges[nleaf - 1 + j]
        A[lo:hi, lo:hi] = h.leaves[j]
    for v in range(nleaf - 1):
        lo1, hi1 = ranges[2 * v + 1]
        lo2, hi2 = ranges[2 * v + 2]
        A[lo1:hi1, lo2:hi2] = h.U12[v] @ h.V12[v].T
        A[lo2:hi2, lo1:hi1] = h.U21[v] @ h.V21[v].T
    return A


@dataclasses.dataclass
class RectHodlrInput:
    """Rectangular HODLR input (Sec. 6): row partition ``m_sizes`` and column partition
    ``n_sizes`` (equal length 2^l, m_j >= n_j); leaf j is the dense m_j x n_j block; for internal
    node v with children c1, c2: ``U12[v]`` (rows of c1 x r), ``V12[v]`` (columns of c2 x r),
    ``U21[v]`` (rows of c2 x r), ``V21[v]`` (columns of c1 x r)."""
    m_sizes: list
    n_sizes: list
    leaves: list
    U12: list
    V12: list
    U21: list
    V21: list
    name: str = ""

    @property
    def m(self):
        return int(sum(self.m_sizes))

    @property
    def n(self):
        return int(sum(self.n_sizes))


def random_rect_hodlr(m, n, nmin, k, seed=0, name="") -> RectHodlrInput:
    """Random rectangular HODLR matrix shaped like Example 6.2: the column partition is the
    balanced partition of n with leaves of at most ``nmin`` columns, the row partition splits m
    the same number of times (floor(m/2) first), every leaf is N(0,1) of size m_j x n_j and every
    off-diagonal block is U V^T with N(0,1) factors of rank k."""
    n_sizes = balanced_leaf_sizes(n, nmin)
    L = len(n_sizes)
    m_sizes = [m]
    while len(m_sizes) < L:
        m_sizes = [x for s in m_sizes for x in (s // 2, s - s // 2)]
    if any(a < b for a, b in zip(m_sizes, n_sizes)):
        raise ValueError("every leaf needs m_j >= n_j")
    rng = np.random.default_rng(seed)
    rr, cr = node_ranges(m_sizes), node_ranges(n_sizes)
    leaves = [np.asfortranarray(rng.standard_normal((m_sizes[j], n_sizes[j]))) for j in range(L)]
    U12, V12, U21, V21 = [], [], [], []
    for v in range(L - 1):
        a, b = 2 * v + 1, 2 * v + 2
        ma, mb = rr[a][1] - rr[a][0], rr[b][1] - rr[b][0]
        na, nb = cr[a][1] - cr[a][0], cr[b][1] - cr[b][0]
        U12.append(np.asfortranarray(rng.standard_normal((ma, k))))
        V12.append(np.asfortranarray(rng.standard_normal((nb, k))))
        U21.append(np.asfortranarray(rng.standard_normal((mb, k))))
        V21.append(np.asfortranarray(rng.standard_normal((na, k))))
    return RectHodlrInput(m_sizes, n_sizes, leaves, U12, V12, U21, V21,
                          name=name or f"rect_m{m}_n{n}_nmin{nmin}_k{k}")


def rect_to_dense(h: RectHodlrInput) -> np.ndarray:
    """Assemble the dense m x n matrix of a rectangular HODLR input (a plain layout step)."""
    A = np.zeros((h.m, h.n))
    rr, cr = node_ranges(h.m_sizes), node_ranges(h.n_sizes)
    L = len(h.m_sizes)
    for j in range(L):
        v = L - 1 + j
        A[rr[v][0]:rr[v][1], cr[v][0]:cr[v][1]] = h.leaves[j]
    for v in range(L - 1):
        a, b = 2 * v + 1, 2 * v + 2
        A[rr[a][0]:rr[a][1], cr[b][0]:cr[b][1]] = h.U12[v] @ h.V12[v].T
        A[rr[b][0]:rr[b][1], cr[a][0]:cr[a][1]] = h.U21[v] @ h.V21[v].T
    return A
