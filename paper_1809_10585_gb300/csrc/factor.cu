// Cluster-cooperative FP64 factorizations of the hQR hot path:
//
//  * qr_dsmem_kernel — Householder QR in compact WY form (Alg. 1 semantics: one
//    reflector per column, LAPACK dlarfg sign convention) of one dense h x w matrix per
//    thread-block cluster.  Columns are dealt cyclically to the CTAs of the cluster; for
//    column j its owner builds the reflector, one cluster barrier publishes it, and every CTA
//    applies it to its own later columns (one warp per column, warp-shuffle reductions).  The
//    T factor is then built from G = Y^T Y: 16 x 16 diagonal blocks by the column recurrence
//    of the compact WY form, and larger blocks by T12 = -T1 G12 T2 (Sec. 3, Eq. (10)).
//    Used for the compressed leaf columns (Alg. 2, lowest level), the left-orthogonalization
//    (Sec. 2.1) and the two QRs inside T_eps (Sec. 2.1.1).
//
//  * jacobi_dsmem_kernel — one-sided (Hestenes) Jacobi on the columns of the K x K core of
//    T_eps, round-robin pair ordering, pairs spread over all warps of the cluster, one
//    cluster barrier per round; plane rotations in scaled form (two FMAs per row and pair).
//
// On GB300 a single SM retires about 2 FP64 FMA per clock, so a K^3 factorization on one SM
// takes milliseconds for K ~ 100; a cluster of up to 16 CTAs (one per SM) multiplies the FP64
// rate at the cost of one hardware cluster barrier per step.  Both kernels pick their form
// from the actual (device-side) sizes: columns in the shared memory of the cluster's CTAs,
// exchanged through distributed shared memory, when they fit; otherwise in global memory
// (L2-resident at these sizes), read with ld.global.cg so that values published by other CTAs
// of the cluster after a barrier are never served stale from L1.
#include <cooperative_groups.h>

#include <atomic>

#include <cstdio>
#include <cstdlib>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace hq {

constexpr int QT = 256;            // threads per CTA
constexpr int QW = QT / 32;        // warps per CTA
constexpr int TNB = 16;            // diagonal block size of the T build
constexpr int kJacobiRegs = 8;     // column elements per lane held in registers (q1 <= 256)
constexpr int kQRRegs = 16;        // QR: column elements per lane in registers (h <= 512)
constexpr int kJacobiMaxCols = 4096;

__device__ inline double warp_sum2(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v, double* red) {
  v = warp_sum2(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = (threadIdx.x < QW) ? red[threadIdx.x] : 0.0;
  if (w == 0) t = warp_sum2(t);
  if (threadIdx.x == 0) red[QW] = t;
  __syncthreads();
  return red[QW];
}

__device__ double block_max(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = (threadIdx.x < QW) ? red[threadIdx.x] : 0.0;
  if (w == 0)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
  if (threadIdx.x == 0) red[QW] = t;
  __syncthreads();
  return red[QW];
}

// Reflector norms of the QR kernels.  The pivot column's squared norm s = |a(j+1:h)|^2 arrives
// as a plain sum of squares; it is used as is while s and alpha^2 stay far from the overflow
// and underflow thresholds.  Otherwise (entries beyond about 1e+-150) the whole owner CTA
// recomputes |(alpha, a(j+1:h))| with the column scaled by a power of two, as LAPACK's dnrm2
// and dlapy2 do inside dlarfg, so R and the reflectors keep full accuracy at any scale.
constexpr double kSumHuge = 0x1p960, kSumTiny = 0x1p-960, kAlphaHuge = 0x1p480;
__device__ __forceinline__ bool norm_needs_scaling(double s, double alpha) {
  return !(s >= kSumTiny && s <= kSumHuge && fabs(alpha) <= kAlphaHuge);
}
// |(alpha, x(lo:h))| with power-of-two scaling; every thread of the CTA calls it with the same
// arguments (x in shared memory, or in global memory read with ld.global.cg when GLOBAL).
// *xzero = 1 when x(lo:h) is exactly zero (no reflector, dlarfg's tau = 0).
template <bool GLOBAL>
__device__ double scaled_column_norm(const double* x, int lo, int h, double alpha, double* red, bool* xzero) {
  double m = threadIdx.x == 0 ? fabs(alpha) : 0.0;
  for (int i = lo + threadIdx.x; i < h; i += QT) m = fmax(m, fabs(GLOBAL ? __ldcg(&x[i]) : x[i]));
  m = block_max(m, red);
  if (m == 0.0) {
    *xzero = true;
    return 0.0;
  }
  int e = 0;
  frexp(m, &e);
  const double sc = ldexp(1.0, -e);                     // m * sc in [0.5, 1): exact scaling
  double ss = 0.0;
  for (int i = lo + threadIdx.x; i < h; i += QT) {
    const double v = (GLOBAL ? __ldcg(&x[i]) : x[i]) * sc;
    ss = fma(v, v, ss);
  }
  ss = block_sum(ss, red);
  *xzero = ss == 0.0;
  const double a = alpha * sc;
  return ldexp(sqrt(fma(a, a, ss)), e);
}

// Cluster barrier and distributed-shared-memory mapping, or their one-CTA forms.
template <bool SOLO>
__device__ __forceinline__ void csync(cg::cluster_group& cl) {
  if (SOLO) __syncthreads();
  else cl.sync();
}
template <bool SOLO, class T>
__device__ __forceinline__ T* rmt(cg::cluster_group& cl, T* p, int rank) {
  return SOLO ? p : cl.map_shared_rank(p, rank);
}

// Sums of acc[0..15] over the 32 lanes of a warp by halving exchanges (after the step with
// offset o a lane keeps half of its values, summed with the partner's): 16 additions per lane
// instead of 16 x 5.  Lane l returns the sum of value l >> 1.
__device__ __forceinline__ double halving_sum16(double acc[16], int lane) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const bool hi = lane & 16;
    const double send = hi ? acc[q] : acc[q + 8];
    const double keep = hi ? acc[q + 8] : acc[q];
    acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const bool hi = lane & 8;
    const double send = hi ? acc[q] : acc[q + 4];
    const double keep = hi ? acc[q + 4] : acc[q];
    acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const bool hi = lane & 4;
    const double send = hi ? acc[q] : acc[q + 2];
    const double keep = hi ? acc[q + 2] : acc[q];
    acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  {
    const bool hi = lane & 2;
    const double send = hi ? acc[0] : acc[1];
    const double keep = hi ? acc[1] : acc[0];
    acc[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  return acc[0] + __shfl_xor_sync(0xffffffffu, acc[0], 1);
}

// One TNB x TNB diagonal block of T by the column recurrence of the compact WY form
// T(0:c, c) = -tau_c T(0:c, 0:c) G(0:c, c), T(c, c) = tau_c (Sec. 3), one warp: g holds
// G(q, c) = y_q^T y_c for q < c (zeros for columns beyond the block's), tl is tau of column
// `lane` (0 beyond the block), and lane l receives row l of the block in trow (zeros below the
// diagonal).  The block's rows stay in registers, so the dependent chain touches no memory.
__device__ __forceinline__ void t_block_rows(const double (*g)[TNB + 1], double tl, int lane, double trow[TNB]) {
#pragma unroll
  for (int c = 0; c < TNB; ++c) trow[c] = 0.0;
#pragma unroll
  for (int c = 0; c < TNB; ++c) {
    const double tc = __shfl_sync(0xffffffffu, tl, c);
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int q = 0; q < c; ++q) {
      if (q & 1) s1 = fma(trow[q], g[q][c], s1);
      else s0 = fma(trow[q], g[q][c], s0);
    }
    trow[c] = lane < c ? -tc * (s0 + s1) : (lane == c ? tc : 0.0);
  }
}

// T of the compact WY form from the Householder vectors stored below the diagonal of A
// (unit diagonal implied): G = Y^T Y (strictly upper part), 16 x 16 diagonal blocks by the
// column recurrence T(0:i,i) = -tau_i T(0:i,0:i) G(0:i,i), then T12 = -T1 G12 T2 (Sec. 3, Eq. (10))
// for blocks of doubling size.  A and tau must be final and visible to every CTA of the cluster.
// `solo`: one CTA alone (block barriers instead of cluster barriers).  `diag_done`: the
// diagonal blocks of T are already stored (the blocked form builds them panel by panel), so
// only G's off-diagonal blocks and the merges remain.  Not a template, so that all forms share
// the one static staging area.
__device__ void qr_build_T(const QRDesc& d, const double* A, const size_t lda, const int h, const int kmax,
                           const int C, const int crank, cg::cluster_group& cl, const bool solo,
                           const bool diag_done = false) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // staging area: 16 x 16 blocks of G per warp for the diagonal blocks, then the two 16 x 32
  // operand tiles of the merges
  __shared__ double gsm[QW][TNB][TNB + 1];
  static_assert(QW * TNB * (TNB + 1) >= 2 * 16 * 33, "merge tiles must fit in the staging area");
  if (d.T == nullptr || kmax == 0) return;

  // ---- T from G = Y^T Y (strictly upper part), Y unit lower trapezoidal
  double* G = d.G;
  const size_t ldg = d.ldg;
  double* T = d.T;
  const size_t ldt = d.ldt;
  if (solo) __syncthreads(); else cl.sync();   // all columns final
  {
    // G in 4 x 4 tiles of (i, jj) column blocks, one warp per tile: every lane walks its share of
    // the rows once for 16 dot products (16 FMA per 8 loads instead of 1 per 2), then the 16 sums
    // are reduced across the warp by halving exchanges (16 adds instead of 80).
    const int gw = warp * C + crank, nw = C * QW;   // consecutive items on different SMs
    const int nb4 = (kmax + 3) / 4;
    const long ntiles = (long)nb4 * (nb4 + 1) / 2;
    for (long p = gw; p < ntiles; p += nw) {
      // decode p -> (I, J) with I <= J, J-major
      int J = (int)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
      while ((long)J * (J + 1) / 2 > p) --J;
      while ((long)(J + 1) * (J + 2) / 2 <= p) ++J;
      const int I = (int)(p - (long)J * (J + 1) / 2);
      if (diag_done && (I >> 2) == (J >> 2)) continue;   // inside a diagonal block: not needed
      const int i0 = 4 * I, j0 = 4 * J;
      double acc[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) acc[q] = 0.0;
      for (int r = j0 + lane; r < h; r += 32) {
        double yi[4], yj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int ci = i0 + u, cj = j0 + u;
          // unit lower trapezoidal Y: 0 above the diagonal, 1 on it
          yi[u] = (ci < kmax && r >= ci) ? (r == ci ? 1.0 : __ldcg(&A[r + (size_t)ci * lda])) : 0.0;
          yj[u] = (cj < kmax && r >= cj) ? (r == cj ? 1.0 : __ldcg(&A[r + (size_t)cj * lda])) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[4 * u + v] = fma(yi[u], yj[v], acc[4 * u + v]);
      }
      const double v = halving_sum16(acc, lane);        // lane l: value l >> 1
      const int q = lane >> 1;
      const int i = i0 + q / 4, jj = j0 + q % 4;
      if ((lane & 1) == 0 && i < jj && jj < kmax) G[i + (size_t)jj * ldg] = v;
    }
    // zero T's strictly lower part, then diagonal blocks by the column recurrence
    for (long e = (long)crank * QT + threadIdx.x; e < (long)kmax * kmax; e += (long)C * QT) {
      int i = (int)(e % kmax), jj = (int)(e / kmax);
      if (i > jj) T[i + jj * ldt] = 0.0;
    }
  }
  if (solo) __syncthreads(); else cl.sync();
  if (!diag_done) {
    // Diagonal 16 x 16 blocks, one warp per block: the block of G is staged in shared memory and
    // lane l keeps row l of the block of T in registers, so the column recurrence runs without
    // global memory in its dependent chain.
    const int gw = warp * C + crank, nw = C * QW;   // consecutive items on different SMs
    const int nblk = (kmax + TNB - 1) / TNB;
    for (int b = gw; b < nblk; b += nw) {
      const int b0 = b * TNB, nbk = min(kmax, b0 + TNB) - b0;
      for (int e = lane; e < TNB * TNB; e += 32) {
        const int r = e % TNB, c = e / TNB;
        gsm[warp][r][c] = (r < c && c < nbk) ? __ldcg(&G[(b0 + r) + (size_t)(b0 + c) * ldg]) : 0.0;
      }
      const double tl = lane < nbk ? __ldcg(&d.tau[b0 + lane]) : 0.0;
      __syncwarp();
      double trow[TNB];
      t_block_rows(gsm[warp], tl, lane, trow);
      if (lane < nbk) {
#pragma unroll
        for (int c = 0; c < TNB; ++c)
          if (c < nbk && c >= lane) T[(b0 + lane) + (size_t)(b0 + c) * ldt] = trow[c];
      }
      __syncwarp();
    }
  }
  // ---- merges: T12 = -T1 G12 T2 for adjacent blocks of size s, as two triangular products in
  // 32 x 32 output tiles (one CTA per tile, operands staged through shared memory in chunks of
  // 16; 2 x 2 outputs per thread): X = T1 G12 is kept transposed in G's strictly lower part,
  // then T12 = -X T2.
  double (*As)[33] = reinterpret_cast<double (*)[33]>(&gsm[0][0][0]);          // [16][33]
  double (*Bs)[33] = reinterpret_cast<double (*)[33]>(&gsm[0][0][0] + 16 * 33);  // [16][33]
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  for (int s = TNB; s < kmax; s *= 2) {
    const int npair = (kmax + 2 * s - 1) / (2 * s);
    if (s < 32) {
      // 16 x 16 blocks: one output per thread is cheaper than a padded 32 x 32 tile
      const long tid = (long)crank * QT + threadIdx.x, nt = (long)C * QT;
      if (solo) __syncthreads(); else cl.sync();
      for (long e = tid; e < (long)npair * s * s; e += nt) {
        const int q = (int)(e / ((long)s * s)), rem = (int)(e % ((long)s * s));
        const int i = rem % s, jj = rem / s, a = 2 * q * s, b = a + s;
        if (b + jj >= kmax) continue;
        double acc = 0.0;
        for (int l = i; l < s; ++l) acc = fma(__ldcg(&T[(a + i) + (size_t)(a + l) * ldt]), __ldcg(&G[(a + l) + (size_t)(b + jj) * ldg]), acc);
        G[(b + jj) + (size_t)(a + i) * ldg] = acc;
      }
      if (solo) __syncthreads(); else cl.sync();
      for (long e = tid; e < (long)npair * s * s; e += nt) {
        const int q = (int)(e / ((long)s * s)), rem = (int)(e % ((long)s * s));
        const int i = rem % s, jj = rem / s, a = 2 * q * s, b = a + s;
        if (b + jj >= kmax) continue;
        double acc = 0.0;
        for (int l = 0; l <= jj; ++l) acc = fma(__ldcg(&G[(b + l) + (size_t)(a + i) * ldg]), __ldcg(&T[(b + l) + (size_t)(b + jj) * ldt]), acc);
        T[(a + i) + (size_t)(b + jj) * ldt] = -acc;
      }
      continue;
    }
    const int tpd = (s + 31) / 32;                        // tiles per dimension of one pair
    for (int pass = 0; pass < 2; ++pass) {
      if (solo) __syncthreads(); else cl.sync();
      for (int tile = crank; tile < npair * tpd * tpd; tile += C) {
        const int q = tile / (tpd * tpd), rem = tile % (tpd * tpd);
        const int i0 = 32 * (rem % tpd), j0 = 32 * (rem / tpd);
        const int a = 2 * q * s, b = a + s;
        const int bs = min(s, kmax - b);                  // width of the second block
        if (bs <= 0 || j0 >= bs) continue;                // uniform over the CTA
        double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
        // pass 0: X(i, jj) = sum_{l >= i} T1(i, l) G12(l, jj);  pass 1: T12(i, jj) = -sum_{l <= jj} X(i, l) T2(l, jj)
        const int lbeg = pass == 0 ? i0 : 0;
        const int lend = pass == 0 ? s : min(bs, j0 + 32);
        for (int l0 = lbeg; l0 < lend; l0 += 16) {
          for (int e = threadIdx.x; e < 32 * 16; e += QT) {
            const int ii = e % 32, ll = e / 32;
            const int i = i0 + ii, l = l0 + ll;
            double va = 0.0;
            if (i < s && l < lend) {
              if (pass == 0) va = (l >= i) ? __ldcg(&T[(a + i) + (size_t)(a + l) * ldt]) : 0.0;
              else va = __ldcg(&G[(b + l) + (size_t)(a + i) * ldg]);
            }
            As[ll][ii] = va;
          }
          for (int e = threadIdx.x; e < 16 * 32; e += QT) {
            const int ll = e % 16, jj2 = e / 16;
            const int l = l0 + ll, jj = j0 + jj2;
            double vb = 0.0;
            if (jj < bs && l < lend) {
              if (pass == 0) vb = __ldcg(&G[(a + l) + (size_t)(b + jj) * ldg]);
              else vb = (l <= jj) ? __ldcg(&T[(b + l) + (size_t)(b + jj) * ldt]) : 0.0;
            }
            Bs[ll][jj2] = vb;
          }
          __syncthreads();
#pragma unroll
          for (int ll = 0; ll < 16; ++ll) {
            const double a0 = As[ll][ty], a1 = As[ll][ty + 16];
            const double b0 = Bs[ll][tx], b1 = Bs[ll][tx + 16];
            acc[0][0] = fma(a0, b0, acc[0][0]);
            acc[0][1] = fma(a0, b1, acc[0][1]);
            acc[1][0] = fma(a1, b0, acc[1][0]);
            acc[1][1] = fma(a1, b1, acc[1][1]);
          }
          __syncthreads();
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            const int i = i0 + ty + 16 * u, jj = j0 + tx + 16 * v;
            if (i < s && jj < bs) {
              if (pass == 0) G[(b + jj) + (size_t)(a + i) * ldg] = acc[u][v];
              else T[(a + i) + (size_t)(b + jj) * ldt] = -acc[u][v];
            }
          }
      }
    }
  }
}

// Global-memory form of the cluster QR: the columns stay in global memory (L2-resident),
// the reflector is staged in `ysm` (shared memory of `stage_rows` doubles) when it fits.
__device__ __forceinline__ void qr_global_impl(const QRDesc* __restrict__ descs, const int* __restrict__ di,
                                               double* flops, double* ysm, int stage_rows) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int crank = (int)cl.block_rank();
  const QRDesc& d = descs[blockIdx.y];
  const int h = dimv(d.h, d.href, di), w = dimv(d.w, d.wref, di);
  const int kmax = min(h, w);
  double* A = d.A;
  const size_t lda = d.lda;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ double red[QW + 1];

  if (crank == 0 && threadIdx.x == 0 && flops && kmax > 0) {
    if (d.step >= 0) {
      double f;
      if (d.fmode == 0) {   // dense QR with its T factor
        f = 2.0 * h * (double)w * w - 2.0 * (double)w * w * w / 3.0 + (double)h * w * w - (double)w * w * w / 3.0;
      } else {              // economy QR with Q formed
        double q = kmax;
        f = 4.0 * h * (double)w * q - 4.0 * q * q * q / 3.0;
      }
      atomicAdd(&flops[d.step], f);
    }
    // work of this launch: Householder QR (reflectors applied to all w columns) and T
    const double q = kmax;
    double g = 2.0 * h * (double)w * q - q * q * (double)w - q * q * q / 3.0 + (double)w * q * q / 3.0;
    if (g < 0) g = 0;
    if (d.T) g += (double)h * q * q - q * q * q / 3.0;
    atomicAdd(&flops[kKindSlot + 2], g);
  }

  // Column j's owner forms its reflector v = [1; a(j+1:h, j) / (alpha - beta)] in place before
  // the cluster barrier that publishes it, so every product with v is taken with the scaled
  // vector (an unscaled column of magnitude 1e150 times another such column would overflow).
  // The norm of the next pivot column is produced by the warp that applies the current
  // reflector to it.
  __shared__ double xn_next;
  if (crank == 0 && kmax > 0) {
    double s = 0.0;
    for (int i = 1 + threadIdx.x; i < h; i += QT) {
      double v = __ldcg(&A[i]);
      s = fma(v, v, s);
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) xn_next = s;
  }
  __syncthreads();
  const bool staged = h <= stage_rows;
  const bool in_regs = h <= 32 * kQRRegs;
  for (int j = 0; j < kmax; ++j) {
    if ((j % C) == crank) {
      double s = xn_next;
      const double alpha = __ldcg(&A[j + j * lda]);
      double hn = 0.0;
      if (norm_needs_scaling(s, alpha)) {                // uniform over the owner CTA
        bool xz = false;
        hn = scaled_column_norm<true>(A + (size_t)j * lda, j + 1, h, alpha, red, &xz);
        s = xz ? 0.0 : 1.0;
        __syncthreads();                                 // red is read above, written below
      } else if (threadIdx.x == 0) {
        hn = sqrt(fma(alpha, alpha, s));                 // s: plain sum of squares
      }
      __syncthreads();                                   // every thread has read alpha
      if (threadIdx.x == 0) {
        double tau = 0.0, scal = 0.0;
        if (s > 0.0) {
          const double beta = -copysign(hn, alpha);
          tau = (beta - alpha) / beta;
          scal = 1.0 / (alpha - beta);
          A[j + j * lda] = beta;
        }
        d.tau[j] = tau;
        red[QW] = scal;
      }
      __syncthreads();
      const double scal = red[QW];
      if (scal != 0.0)
        for (int i = j + 1 + threadIdx.x; i < h; i += QT) A[i + (size_t)j * lda] = __ldcg(&A[i + (size_t)j * lda]) * scal;
    }
    cl.sync();
    const double tau = __ldcg(&d.tau[j]);
    const double* y = A + j * lda;
    if (staged && tau != 0.0) {
      for (int i = j + 1 + threadIdx.x; i < h; i += QT) ysm[i] = __ldcg(&y[i]);
      __syncthreads();
    }
    const int first = j + 1;
    const int c0 = first + ((crank - first % C) + C) % C;
    for (int c = c0 + warp * C; c < w; c += QW * C) {
      double* a = A + c * lda;
      double nn = 0.0;   // squared norm of a(j+2:h) after the update (next pivot only)
      if (tau != 0.0) {
        if (in_regs) {
          double r[kQRRegs];
          double t = 0.0;
          const int nq = (h - j - 1 + 31) >> 5;   // warp-uniform live register slots
#pragma unroll
          for (int q = 0; q < kQRRegs; ++q) {
            if (q < nq) {
              const int i = j + 1 + lane + 32 * q;
              r[q] = i < h ? __ldcg(&a[i]) : 0.0;
              if (i < h) t = fma(staged ? ysm[i] : __ldcg(&y[i]), r[q], t);
            }
          }
          t = warp_sum2(t);
          const double wv = tau * (t + __ldcg(&a[j]));
          const bool pivot = c == j + 1;          // next pivot: its norm below row j + 1 too
#pragma unroll
          for (int q = 0; q < kQRRegs; ++q) {
            if (q < nq) {
              const int i = j + 1 + lane + 32 * q;
              if (i < h) {
                const double v = fma(-wv, staged ? ysm[i] : __ldcg(&y[i]), r[q]);
                a[i] = v;
                if (pivot && i > j + 1) nn = fma(v, v, nn);
              }
            }
          }
          if (lane == 0) a[j] = __ldcg(&a[j]) - wv;
        } else {
          double t = 0.0;
          for (int i = j + 1 + lane; i < h; i += 32) t = fma(staged ? ysm[i] : __ldcg(&y[i]), __ldcg(&a[i]), t);
          t = warp_sum2(t);
          const double wv = tau * (t + __ldcg(&a[j]));
          const bool pivot = c == j + 1;
          for (int i = j + 1 + lane; i < h; i += 32) {
            const double v = fma(-wv, staged ? ysm[i] : __ldcg(&y[i]), __ldcg(&a[i]));
            a[i] = v;
            if (pivot && i > j + 1) nn = fma(v, v, nn);
          }
          if (lane == 0) a[j] = __ldcg(&a[j]) - wv;
        }
      } else if (c == j + 1) {
        for (int i = j + 2 + lane; i < h; i += 32) {
          const double v = __ldcg(&a[i]);
          nn = fma(v, v, nn);
        }
      }
      if (c == j + 1) {
        nn = warp_sum2(nn);
        if (lane == 0) xn_next = nn;
      }
    }
    __syncthreads();
  }
  cl.sync();
  qr_build_T(d, A, lda, h, kmax, C, crank, cl, false);
}

__global__ void __launch_bounds__(QT) jacobi_cluster_kernel(const JacobiDesc* __restrict__ descs);

template <bool kOwner>
__global__ void __launch_bounds__(QT, 2) jacobi_dsmem_kernel(const JacobiDesc* __restrict__ descs,
                                                          int q1cap, int q2cap, int smem_bytes, int solo_cols);
constexpr size_t kJacobiSmemMax = 200 * 1024;


// Householder QR with the matrix held in distributed shared memory: column c lives in the
// shared memory of CTA c % C (slot c / C).  The owner of column j forms and scales its
// reflector in place, one cluster barrier publishes it, and every CTA copies it once through
// DSMEM into a local buffer before updating its own columns (one warp per column, the warp
// that updates the next pivot also returns that column's norm).  The factored columns are
// written back to global memory and T is built as in the global-memory form.  The layout
// follows the actual size h x w: `nloc` slots of h doubles and a reflector buffer of h.
template <bool SOLO>
__device__ __forceinline__ void qr_dsmem_impl(const QRDesc* __restrict__ descs, const int* __restrict__ di,
                                              double* flops, int h, int w, double* qsm) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = SOLO ? 1 : (int)cl.num_blocks();
  const int crank = SOLO ? 0 : (int)cl.block_rank();
  const QRDesc& d = descs[blockIdx.y];
  const int kmax = min(h, w);
  double* A = d.A;
  const size_t lda = d.lda;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nloc = (w + C - 1) / C;
  const size_t ldc = h;
  double* cols = qsm;                                   // nloc x h
  double* ybuf = cols + (size_t)nloc * ldc;             // h
  __shared__ double red[QW + 1];
  __shared__ double sh_tau, xn_next;

  if (crank == 0 && threadIdx.x == 0 && flops && kmax > 0) {
    if (d.step >= 0) {
      double f;
      if (d.fmode == 0) {
        f = 2.0 * h * (double)w * w - 2.0 * (double)w * w * w / 3.0 + (double)h * w * w - (double)w * w * w / 3.0;
      } else {
        double q = kmax;
        f = 4.0 * h * (double)w * q - 4.0 * q * q * q / 3.0;
      }
      atomicAdd(&flops[d.step], f);
    }
    const double q = kmax;
    double g = 2.0 * h * (double)w * q - q * q * (double)w - q * q * q / 3.0 + (double)w * q * q / 3.0;
    if (g < 0) g = 0;
    if (d.T) g += (double)h * q * q - q * q * q / 3.0;
    atomicAdd(&flops[kKindSlot + 2], g);
  }
  for (int sl = 0; sl < nloc; ++sl) {
    const int c = crank + sl * C;
    if (c >= w) break;
    for (int i = threadIdx.x; i < h; i += QT) cols[(size_t)sl * ldc + i] = A[i + (size_t)c * lda];
  }
  csync<SOLO>(cl);                                       // all CTAs running before any DSMEM access
  if (crank == 0 && kmax > 0) {
    double s = 0.0;
    for (int i = 1 + threadIdx.x; i < h; i += QT) s = fma(cols[i], cols[i], s);
    s = block_sum(s, red);
    if (threadIdx.x == 0) xn_next = s;
  }
  __syncthreads();
  const bool in_regs = h <= 32 * kQRRegs;
  for (int j = 0; j < kmax; ++j) {
    const int owner = j % C;
    if (owner == crank) {
      double* cj = cols + (size_t)(j / C) * ldc;
      double s = xn_next;
      const double alpha = cj[j];
      double hn = 0.0;
      if (norm_needs_scaling(s, alpha)) {                // uniform over the owner CTA
        bool xz = false;
        hn = scaled_column_norm<false>(cj, j + 1, h, alpha, red, &xz);
        s = xz ? 0.0 : 1.0;
        __syncthreads();                                 // red is read above, written below
      } else if (threadIdx.x == 0) {
        hn = sqrt(fma(alpha, alpha, s));                 // s: plain sum of squares
      }
      double beta = alpha;
      if (threadIdx.x == 0) {
        double tau = 0.0, scal = 0.0;
        if (s > 0.0) {
          beta = -copysign(hn, alpha);
          tau = (beta - alpha) / beta;
          scal = 1.0 / (alpha - beta);
        }
        sh_tau = tau;
        red[QW] = scal;
        d.tau[j] = tau;
      }
      __syncthreads();                                   // every thread has read alpha
      const double scal = red[QW];
      if (threadIdx.x == 0) cj[j] = beta;
      if (scal != 0.0)
        for (int i = j + 1 + threadIdx.x; i < h; i += QT) cj[i] *= scal;
    }
    csync<SOLO>(cl);
    const double tau = *rmt<SOLO>(cl, &sh_tau, owner);
    const double* yref = ybuf;                         // the reflector of column j
    if (SOLO) {
      yref = cols + (size_t)j * ldc;                   // local, and only read until the next step
    } else if (tau != 0.0) {
      const double* yj = cl.map_shared_rank(cols, owner) + (size_t)(j / C) * ldc;
      for (int i = j + 1 + threadIdx.x; i < h; i += QT) ybuf[i] = yj[i];
      __syncthreads();
    }
    const int first = j + 1;
    const int c0 = first + ((crank - first % C) + C) % C;
    // A warp updates two columns at once, c and c + QW C: one load of the reflector serves both
    // dot products, and the two warp reductions share their first level (lanes 0-15 finish the
    // sum of c, lanes 16-31 that of c + QW C), which saves FP64 instructions on short columns.
    for (int c = c0 + warp * C; c < w; c += 2 * QW * C) {
      const int c2 = c + QW * C;
      if (tau != 0.0 && c2 < w) {
        double* aA = cols + (size_t)(c / C) * ldc;
        double* aB = cols + (size_t)(c2 / C) * ldc;
        const int nq = (h - j - 1 + 31) >> 5;     // warp-uniform row slots
        double tA0 = 0.0, tA1 = 0.0, tB0 = 0.0, tB1 = 0.0;
        int q = 0;
        for (; q + 1 < nq; q += 2) {
          const int i0 = j + 1 + lane + 32 * q, i1 = i0 + 32;   // i0 < h here
          const double y0 = yref[i0];
          tA0 = fma(y0, aA[i0], tA0);
          tB0 = fma(y0, aB[i0], tB0);
          if (i1 < h) {
            const double y1 = yref[i1];
            tA1 = fma(y1, aA[i1], tA1);
            tB1 = fma(y1, aB[i1], tB1);
          }
        }
        if (q < nq) {
          const int i0 = j + 1 + lane + 32 * q;
          if (i0 < h) {
            const double y0 = yref[i0];
            tA0 = fma(y0, aA[i0], tA0);
            tB0 = fma(y0, aB[i0], tB0);
          }
        }
        const bool lo = lane < 16;
        const double tA = tA0 + tA1, tB = tB0 + tB1;
        double tm = (lo ? tA : tB) + __shfl_xor_sync(0xffffffffu, lo ? tB : tA, 16);
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) tm += __shfl_xor_sync(0xffffffffu, tm, o);
        double* ac = lo ? aA : aB;
        const double wv = tau * (tm + ac[j]);
        const double wA = __shfl_sync(0xffffffffu, wv, 0), wB = __shfl_sync(0xffffffffu, wv, 16);
        if (c == j + 1) {                         // next pivot: its norm below row j + 1 too
          double nn = 0.0;
          for (int qq = 0; qq < nq; ++qq) {
            const int i = j + 1 + lane + 32 * qq;
            if (i < h) {
              const double yv = yref[i];
              const double v = fma(-wA, yv, aA[i]);
              aA[i] = v;
              aB[i] = fma(-wB, yv, aB[i]);
              if (i > j + 1) nn = fma(v, v, nn);
            }
          }
          nn = warp_sum2(nn);
          if (lane == 0) xn_next = nn;
        } else {
          for (int qq = 0; qq < nq; ++qq) {
            const int i = j + 1 + lane + 32 * qq;
            if (i < h) {
              const double yv = yref[i];
              aA[i] = fma(-wA, yv, aA[i]);
              aB[i] = fma(-wB, yv, aB[i]);
            }
          }
        }
        __syncwarp();
        if ((lane & 15) == 0) ac[j] -= wv;       // lane 0: column c, lane 16: column c + QW C
        continue;
      }
      double* a = cols + (size_t)(c / C) * ldc;
      double nn = 0.0;
      if (tau != 0.0) {
        if (in_regs) {
          double r[kQRRegs];
          double t0 = 0.0, t1 = 0.0;             // two chains: half the dependent FMA latency
          const int nq = (h - j - 1 + 31) >> 5;   // warp-uniform live register slots
#pragma unroll
          for (int q = 0; q < kQRRegs; ++q) {
            if (q < nq) {
              const int i = j + 1 + lane + 32 * q;
              r[q] = i < h ? a[i] : 0.0;
              if (i < h) {
                if (q & 1) t1 = fma(yref[i], r[q], t1);
                else t0 = fma(yref[i], r[q], t0);
              }
            }
          }
          double t = warp_sum2(t0 + t1);
          const double wv = tau * (t + a[j]);
          if (c == j + 1) {                       // next pivot: its norm below row j + 1 too
            double nn1 = 0.0;
#pragma unroll
            for (int q = 0; q < kQRRegs; ++q) {
              if (q < nq) {
                const int i = j + 1 + lane + 32 * q;
                if (i < h) {
                  const double v = fma(-wv, yref[i], r[q]);
                  a[i] = v;
                  if (i > j + 1) {
                    if (q & 1) nn1 = fma(v, v, nn1);
                    else nn = fma(v, v, nn);
                  }
                }
              }
            }
            nn += nn1;
          } else {
#pragma unroll
            for (int q = 0; q < kQRRegs; ++q) {
              if (q < nq) {
                const int i = j + 1 + lane + 32 * q;
                if (i < h) a[i] = fma(-wv, yref[i], r[q]);
              }
            }
          }
          __syncwarp();
          if (lane == 0) a[j] -= wv;
        } else {
          double t = 0.0;
          for (int i = j + 1 + lane; i < h; i += 32) t = fma(yref[i], a[i], t);
          t = warp_sum2(t);
          const double wv = tau * (t + a[j]);
          if (c == j + 1) {
            for (int i = j + 1 + lane; i < h; i += 32) {
              const double v = fma(-wv, yref[i], a[i]);
              a[i] = v;
              if (i > j + 1) nn = fma(v, v, nn);
            }
          } else {
            for (int i = j + 1 + lane; i < h; i += 32) a[i] = fma(-wv, yref[i], a[i]);
          }
          __syncwarp();
          if (lane == 0) a[j] -= wv;
        }
      } else if (c == j + 1) {
        for (int i = j + 2 + lane; i < h; i += 32) nn = fma(a[i], a[i], nn);
      }
      if (c == j + 1) {
        nn = warp_sum2(nn);
        if (lane == 0) xn_next = nn;
      }
      // (tau = 0: no reflector, the second column c + QW C is unchanged and is never the pivot)
    }
    // One cluster barrier per column suffices.  sh_tau of a CTA is rewritten only when it owns
    // a column again, C >= 2 columns later, after every CTA has arrived at the barrier of the
    // column before that one, i.e. after every CTA finished reading this reflector; the rows of
    // column j read remotely are final; ybuf and xn_next are private to the CTA.
    __syncthreads();
  }
  for (int sl = 0; sl < nloc; ++sl) {
    const int c = crank + sl * C;
    if (c >= w) break;
    for (int i = threadIdx.x; i < h; i += QT) A[i + (size_t)c * lda] = cols[(size_t)sl * ldc + i];
  }
  qr_build_T(d, A, lda, h, kmax, C, crank, cl, SOLO);   // starts with a barrier
}

// Blocked Householder QR (Alg. 1 with panels of QNB columns: the reflectors of a panel are
// formed one by one, then applied together to the columns to its right) of one h x w matrix
// held in global memory (L2-resident), for matrices whose columns do not fit in the cluster's
// shared memory.  Column block q (columns q QNB .. q QNB + QNB - 1) belongs to CTA q % C.  For
// panel p its owner loads the panel into shared memory, factors it there with block barriers
// only (reflector norms by block reductions, scaled when needed), writes it back and publishes
// it with one cluster barrier.  Every CTA then holds the panel's reflectors in shared memory
// (unit lower trapezoidal), together with the panel's diagonal block T_p of T (built by the
// owner from the panel's block of G = Y^T Y before the barrier), and applies
// Q_p^T = I - Y_p T_p^T Y_p^T to each of its own later columns (Sec. 3, Eq. (10)), one warp per
// column with the column in registers (qr_apply_panel): a column is read and written once per
// panel, and the cluster waits once per panel instead of once per column.  The rest of T (the
// off-diagonal blocks of G and the merges) is built afterwards as in the other forms.
constexpr int QNB = 16;

// Shared memory of the blocked form: the panel (h x QNB) followed by three TNB x (TNB + 1)
// staging blocks (the owner's block of G, the owner's T_p, this CTA's copy of T_p).
constexpr int kQRTBlk = TNB * (TNB + 1);
__host__ __device__ inline size_t qr_blocked_bytes(int h) {
  return ((size_t)h * QNB + 3 * kQRTBlk) * sizeof(double) + 64;
}

// Q_p^T = I - Y_p T_p^T Y_p^T applied to one column a (rows j0 .. h-1) by one warp, the column
// in NR registers per lane (nq <= NR of them in use): the lane partials of the nbp products
// Y_p^T a are summed across the warp together (halving_sum16: 16 additions per lane instead of
// 16 reductions of 5), W = T_p^T (Y_p^T a) is formed on lanes 2j, 2j + 1, and a -= Y_p W.
template <int NR>
__device__ __forceinline__ void qr_apply_panel(double* a, int h, int j0, int nq, int nbp, const double* Ys,
                                               const double (*tq)[TNB + 1], int lane) {
  double r[NR];
#pragma unroll
  for (int u = 0; u < NR; ++u) {
    const int i = j0 + lane + 32 * u;
    r[u] = (u < nq && i < h) ? __ldcg(&a[i]) : 0.0;
  }
  double acc[QNB];
#pragma unroll
  for (int k = 0; k < QNB; ++k) {
    double t = 0.0;
    if (k < nbp) {
      const double* yk = Ys + (size_t)k * h;
#pragma unroll
      for (int u = 0; u < NR; ++u) {
        const int i = j0 + lane + 32 * u;
        if (u < nq && i < h) t = fma(yk[i], r[u], t);
      }
    }
    acc[k] = t;
  }
  const double wv = halving_sum16(acc, lane);
  const int jq = lane >> 1;
  double wt = 0.0;
#pragma unroll
  for (int k = 0; k < QNB; ++k) wt = fma(tq[k][jq], __shfl_sync(0xffffffffu, wv, 2 * k), wt);
#pragma unroll
  for (int k = 0; k < QNB; ++k) {
    const double wk = __shfl_sync(0xffffffffu, wt, 2 * k);
    if (k < nbp) {
      const double* yk = Ys + (size_t)k * h;
#pragma unroll
      for (int u = 0; u < NR; ++u) {
        const int i = j0 + lane + 32 * u;
        if (u < nq && i < h) r[u] = fma(-wk, yk[i], r[u]);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < NR; ++u) {
    const int i = j0 + lane + 32 * u;
    if (u < nq && i < h) a[i] = r[u];
  }
}

__device__ __forceinline__ void qr_blocked_impl(const QRDesc& d, int h, int w, double* flops, double* Ys) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int crank = (int)cl.block_rank();
  const int kmax = min(h, w);
  double* A = d.A;
  const size_t lda = d.lda;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __shared__ double red[QW + 1];
  __shared__ double ptau[QNB];
  // after the panel in the dynamic shared memory (same offsets in every CTA of the cluster)
  double (*gp)[TNB + 1] = reinterpret_cast<double (*)[TNB + 1]>(Ys + (size_t)h * QNB);   // owner's G block
  double (*tp)[TNB + 1] = gp + TNB;                      // the owner's T_p (read by every CTA)
  double (*tq)[TNB + 1] = tp + TNB;                      // this CTA's copy of T_p
  static_assert(QNB == TNB, "panels and diagonal blocks of T coincide");

  if (crank == 0 && tid == 0 && flops && kmax > 0) {
    if (d.step >= 0) {
      double f;
      if (d.fmode == 0) {
        f = 2.0 * h * (double)w * w - 2.0 * (double)w * w * w / 3.0 + (double)h * w * w - (double)w * w * w / 3.0;
      } else {
        const double q = kmax;
        f = 4.0 * h * (double)w * q - 4.0 * q * q * q / 3.0;
      }
      atomicAdd(&flops[d.step], f);
    }
    const double q = kmax;
    double g = 2.0 * h * (double)w * q - q * q * (double)w - q * q * q / 3.0 + (double)w * q * q / 3.0;
    if (g < 0) g = 0;
    if (d.T) g += (double)h * q * q - q * q * q / 3.0;
    atomicAdd(&flops[kKindSlot + 2], g);
  }

  const int npanel = (kmax + QNB - 1) / QNB;
  for (int p = 0; p < npanel; ++p) {
    const int j0 = p * QNB, nbp = min(QNB, kmax - j0), rows = h - j0;
    const int owner = p % C;
    if (crank == owner) {
      __syncthreads();                                   // own columns updated by all threads
      for (int e = tid; e < rows * nbp; e += QT) {
        const int i = j0 + e % rows, c = e / rows;
        Ys[i + (size_t)c * h] = __ldcg(&A[i + (size_t)(j0 + c) * lda]);
      }
      __syncthreads();
      for (int jj = 0; jj < nbp; ++jj) {
        const int j = j0 + jj;
        double* y = Ys + (size_t)jj * h;
        double s = 0.0;
        for (int i = j + 1 + tid; i < h; i += QT) s = fma(y[i], y[i], s);
        s = block_sum(s, red);
        const double alpha = y[j];
        double hn = 0.0;
        if (norm_needs_scaling(s, alpha)) {              // uniform over the CTA
          bool xz = false;
          hn = scaled_column_norm<false>(y, j + 1, h, alpha, red, &xz);
          s = xz ? 0.0 : 1.0;
        } else if (tid == 0) {
          hn = sqrt(fma(alpha, alpha, s));
        }
        __syncthreads();                                 // every thread has read alpha and red
        if (tid == 0) {
          double tau = 0.0, scal = 0.0, beta = alpha;
          if (s > 0.0) {
            beta = -copysign(hn, alpha);
            tau = (beta - alpha) / beta;
            scal = 1.0 / (alpha - beta);
          }
          ptau[jj] = tau;
          red[QW] = scal;
          d.tau[j] = tau;
          y[j] = beta;
        }
        __syncthreads();
        const double scal = red[QW], tau = ptau[jj];
        if (scal != 0.0)
          for (int i = j + 1 + tid; i < h; i += QT) y[i] *= scal;
        __syncthreads();
        if (tau != 0.0) {
          for (int c = jj + 1 + warp; c < nbp; c += QW) {  // the rest of the panel
            double* a = Ys + (size_t)c * h;
            double t0 = 0.0, t1 = 0.0;
            int i = j + 1 + lane;
            for (; i + 32 < h; i += 64) {
              t0 = fma(y[i], a[i], t0);
              t1 = fma(y[i + 32], a[i + 32], t1);
            }
            if (i < h) t0 = fma(y[i], a[i], t0);
            const double wv = tau * (warp_sum2(t0 + t1) + a[j]);
            for (int r = j + 1 + lane; r < h; r += 32) a[r] = fma(-wv, y[r], a[r]);
            __syncwarp();
            if (lane == 0) a[j] -= wv;
          }
        }
        __syncthreads();
      }
      // the factored panel back to global memory (R above the diagonal, reflectors below)
      for (int e = tid; e < rows * nbp; e += QT) {
        const int i = j0 + e % rows, c = e / rows;
        A[i + (size_t)(j0 + c) * lda] = Ys[i + (size_t)c * h];
      }
      __syncthreads();
      // unit lower trapezoidal form of the reflectors for the update of later columns
      for (int e = tid; e < nbp * nbp; e += QT) {
        const int r = e % nbp, c = e / nbp;
        if (r <= c) Ys[j0 + r + (size_t)c * h] = (r == c) ? 1.0 : 0.0;
      }
      __syncthreads();
      // the panel's block of G (strictly upper; ten 4 x 4 tiles, one warp each), then T_p
      for (int tile = warp; tile < 10; tile += QW) {
        int J = 0;
        while ((J + 1) * (J + 2) / 2 <= tile) ++J;
        const int I = tile - J * (J + 1) / 2, i0 = 4 * I, c0 = 4 * J;
        double acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = 0.0;
        for (int r = j0 + c0 + lane; r < h; r += 32) {
          double yi[4], yj[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            yi[u] = i0 + u < nbp ? Ys[r + (size_t)(i0 + u) * h] : 0.0;
            yj[u] = c0 + u < nbp ? Ys[r + (size_t)(c0 + u) * h] : 0.0;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[4 * u + v] = fma(yi[u], yj[v], acc[4 * u + v]);
        }
        const double v = halving_sum16(acc, lane);
        const int q = lane >> 1, i = i0 + q / 4, jj = c0 + q % 4;
        if ((lane & 1) == 0) gp[i][jj] = (i < jj && jj < nbp) ? v : 0.0;
      }
      __syncthreads();
      if (warp == 0) {
        double trow[TNB];
        t_block_rows(gp, lane < nbp ? ptau[lane] : 0.0, lane, trow);
        if (lane < TNB) {
#pragma unroll
          for (int c = 0; c < TNB; ++c) tp[lane][c] = trow[c];
        }
        if (d.T && lane < nbp) {
#pragma unroll
          for (int c = 0; c < TNB; ++c)
            if (c < nbp && c >= lane) d.T[(j0 + lane) + (size_t)(j0 + c) * d.ldt] = trow[c];
        }
      }
    }
    cl.sync();                                           // panel p, its tau and T_p published
    if (crank != owner) {
      for (int e = tid; e < rows * nbp; e += QT) {
        const int i = j0 + e % rows, c = e / rows;
        const double v = __ldcg(&A[i + (size_t)(j0 + c) * lda]);
        Ys[i + (size_t)c * h] = i < j0 + c ? 0.0 : (i == j0 + c ? 1.0 : v);
      }
      if (tid < nbp) ptau[tid] = __ldcg(&d.tau[j0 + tid]);
    }
    {
      // T_p from the owner's shared memory; the owner writes it again only for panel p + C,
      // after the next cluster barrier, which every CTA passes after this copy
      const double* src = cl.map_shared_rank(&tp[0][0], owner);
      for (int e = tid; e < TNB * (TNB + 1); e += QT) (&tq[0][0])[e] = src[e];
    }
    __syncthreads();
    // apply the panel's reflectors in order to this CTA's columns beyond the panel
    const int qfirst = p + 1 + ((crank - (p + 1) % C) + C) % C;   // first own block after p
    const int nown = [&] {
      int c = 0;
      for (int q = qfirst; q * QNB < w; q += C) c += min(QNB, w - q * QNB);
      return c;
    }();
    const int nq = (rows + 31) >> 5;
    for (int idx = warp; idx < nown; idx += QW) {
      const int q = qfirst + (idx / QNB) * C;             // blocks before the last are full
      const int c = q * QNB + idx % QNB;
      double* a = A + (size_t)c * lda;
      if (nq <= 12) {
        qr_apply_panel<12>(a, h, j0, nq, nbp, Ys, tq, lane);
      } else if (nq <= kQRRegs) {
        // longer columns (h - j0 <= 512): the reflectors one after another, column in registers
        // (the level-3 form would not fit the register budget)
        double r[kQRRegs];
#pragma unroll
        for (int u = 0; u < kQRRegs; ++u) {
          const int i = j0 + lane + 32 * u;
          r[u] = (u < nq && i < h) ? __ldcg(&a[i]) : 0.0;
        }
        for (int k = 0; k < nbp; ++k) {
          const double tk = ptau[k];
          if (tk == 0.0) continue;
          const double* yk = Ys + (size_t)k * h;
          double t0 = 0.0, t1 = 0.0;
#pragma unroll
          for (int u = 0; u < kQRRegs; ++u) {
            const int i = j0 + lane + 32 * u;
            if (u < nq && i < h) {
              if (u & 1) t1 = fma(yk[i], r[u], t1);
              else t0 = fma(yk[i], r[u], t0);
            }
          }
          const double wv = tk * warp_sum2(t0 + t1);
#pragma unroll
          for (int u = 0; u < kQRRegs; ++u) {
            const int i = j0 + lane + 32 * u;
            if (u < nq && i < h) r[u] = fma(-wv, yk[i], r[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < kQRRegs; ++u) {
          const int i = j0 + lane + 32 * u;
          if (u < nq && i < h) a[i] = r[u];
        }
      } else {
        // long columns: each reflector streams the column from L2
        for (int k = 0; k < nbp; ++k) {
          const double tk = ptau[k];
          if (tk == 0.0) continue;
          const double* yk = Ys + (size_t)k * h;
          double t = 0.0;
          for (int i = j0 + k + lane; i < h; i += 32) t = fma(yk[i], __ldcg(&a[i]), t);
          const double wv = tk * warp_sum2(t);
          for (int i = j0 + k + lane; i < h; i += 32) a[i] = fma(-wv, yk[i], __ldcg(&a[i]));
          __syncwarp();
        }
      }
    }
  }
  // the rest of T: off-diagonal blocks of G and the merges (starts with a cluster barrier:
  // every column and every T_p final everywhere)
  qr_build_T(d, A, lda, h, kmax, C, crank, cl, false, true);
}

// Bytes of shared memory of the distributed form for an h x w matrix on C CTAs.
__host__ __device__ inline size_t qr_dsmem_bytes(int h, int w, int cluster) {
  const size_t nloc = (w + cluster - 1) / cluster;
  return (nloc + 1) * (size_t)h * sizeof(double) + 64;
}

// The form is chosen from the matrix's actual size (every CTA of the cluster reads the same
// descriptor): distributed shared memory when its columns fit in the launch's shared memory,
// the global-memory form otherwise (reflector staged in the same shared memory).
__global__ void __launch_bounds__(QT) qr_dsmem_kernel(const QRDesc* __restrict__ descs,
                                                      int hcap, int wcap, int smem_bytes, int solo_cols) {
  const QRDesc& d = descs[blockIdx.y];
  const int* di = d.di;
  double* flops = d.fl;
  const int h = min(dimv(d.h, d.href, di), hcap), w = min(dimv(d.w, d.wref, di), wcap);
  const int C = (int)cg::this_cluster().num_blocks();
  extern __shared__ double qsm[];
  if (w <= solo_cols && qr_dsmem_bytes(h, w, 1) <= (size_t)smem_bytes) {
    if (cg::this_cluster().block_rank() != 0) return;   // one CTA; no cluster barrier follows
    qr_dsmem_impl<true>(descs, di, flops, h, w, qsm);
  } else if (qr_dsmem_bytes(h, w, C) <= (size_t)smem_bytes) {
    qr_dsmem_impl<false>(descs, di, flops, h, w, qsm);
  } else if (w > QNB && qr_blocked_bytes(h) <= (size_t)smem_bytes) {
    qr_blocked_impl(d, h, w, flops, qsm);
  } else {
    qr_global_impl(descs, di, flops, qsm, smem_bytes / (int)sizeof(double));
  }
}

constexpr size_t kQRSmemMax = 200 * 1024;
constexpr int kQRSoloCols = 32;

// Largest cluster size both cluster kernels can be launched with (16 needs the non-portable
// attribute and enough SMs per GPC), probed once per process (thread-safe: the first caller
// runs the probe, concurrent callers wait for it); attributes are set here, never during stream
// capture.
static int probe_max_cluster() {
  int v = 8;
  bool ok = cudaFuncSetAttribute(qr_dsmem_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
            cudaFuncSetAttribute(qr_dsmem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kQRSmemMax) == cudaSuccess &&
            cudaFuncSetAttribute(jacobi_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
  if (ok) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(QT, 1, 1);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    cfg.dynamicSmemBytes = kQRSmemMax;
    if (cudaOccupancyMaxActiveClusters(&nclusters, qr_dsmem_kernel, &cfg) == cudaSuccess && nclusters > 0) {
      cfg.dynamicSmemBytes = 0;
      int nj = 0;
      if (cudaOccupancyMaxActiveClusters(&nj, jacobi_cluster_kernel, &cfg) == cudaSuccess && nj > 0) v = 16;
    }
  }
  cudaGetLastError();
  cudaFuncSetAttribute(jacobi_dsmem_kernel<false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaFuncSetAttribute(jacobi_dsmem_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kJacobiSmemMax);
  cudaFuncSetAttribute(jacobi_dsmem_kernel<true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaFuncSetAttribute(jacobi_dsmem_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kJacobiSmemMax);
  cudaGetLastError();
  return v;
}

int qr_max_cluster() {
  static const int cached = probe_max_cluster();
  return cached;
}

cudaError_t launch_qr(const QRDesc* h, int n, QRDesc* d, int cluster, size_t smem_cap, cudaStream_t s,
                      int cluster_large) {
  if (n <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster, n, 1);
  cfg.blockDim = dim3(QT, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int hcap = 1, wcap = 1;
  for (int i = 0; i < n; ++i) {
    hcap = max(hcap, h[i].h);
    wcap = max(wcap, h[i].w);
  }
  // A matrix whose columns fit neither the cluster's shared memory nor, as one panel, a CTA's
  // (a tall truncation or left-orthogonalization input) would take the level-2 global-memory
  // form: it is large by nature, so it gets the context's cluster size for large problems.
  const size_t cap = std::min(kQRSmemMax, smem_cap);
  if (cluster_large > cluster && qr_dsmem_bytes(hcap, wcap, cluster) > cap && qr_blocked_bytes(hcap) > cap) {
    cluster = cluster_large;
    cfg.gridDim = dim3(cluster, n, 1);
    attr[0].val.clusterDim.x = cluster;
  }
  // shared memory for the capacities, up to the per-CTA limit; the kernel picks its form from
  // the actual sizes
  const size_t smem = std::min(qr_dsmem_bytes(hcap, wcap, cluster), cap);
  cfg.dynamicSmemBytes = smem;
  // matrices of at most this many columns are factored by one CTA of the cluster (the others
  // exit at once): no cluster barrier per column; more of them while other factorizations
  // share the SMs
  const int solo = smem_cap < kQRSmemMax ? 2 * kQRSoloCols : kQRSoloCols;
  return cudaLaunchKernelEx(&cfg, qr_dsmem_kernel, (const QRDesc*)d, hcap, wcap, (int)smem, solo);
}

// --------------------------------------------------------------------------------- Jacobi
// 2^k as a double, for -1022 <= k <= 1023 (exact).
__device__ inline double pow2i(int k) { return __longlong_as_double((long long)(k + 1023) << 52); }

// Plane rotation of one column pair of one-sided Jacobi from alpha = |x|^2 > 0, beta = |y|^2 > 0
// and gamma = x.y.  Returns false when the pair is orthogonal to the relative tolerance tol
// (gamma^2 <= tol^2 alpha beta).  Otherwise t = tan(theta) is the root of magnitude <= 1 of
// gamma t^2 + (beta - alpha) t - gamma = 0 and (c, s) = (1, t) / sqrt(1 + t^2).
//
// FP64 instructions are the scarce resource here (an SM retires one FP64 warp instruction per
// ~16 cycles, each with ~67 cycles of latency; divide and square root are sequences of
// 450-700 cycles), so only what needs FP64 uses it.  The inputs are scaled by one power of two
// to O(1) (exact; the test and t are scale-invariant), the test and t are formed in FP32, and
// (c, s) are taken from FP32 values c0, s0 and normalized in FP64 with the series
// (1 + d)^(-1/2) = 1 - d/2 + 3 d^2 / 8, d = c0^2 + s0^2 - 1 = O(1e-7), so that c^2 + s^2 = 1
// to FP64 rounding: the rotation is orthogonal to working precision, only the angle carries the
// FP32 error (a slightly less effective rotation, never a less accurate one).  Pairs whose
// scaled values leave the normal FP32 range (norms more than ~1e30 apart, or gamma below
// 1e-30 max(alpha, beta)) take the plain FP64 formulas.
__device__ inline bool jacobi_rotation(double al, double be, double g, double tol2, float tolf, double& c,
                                       double& s, double& t) {
  const long long im = max(__double_as_longlong(al), __double_as_longlong(be));  // order of
  int ex = (int)(im >> 52) - 1023;                                                // positive doubles
  ex = min(max(ex, -1000), 1000);
  const double sc = pow2i(-ex);
  const double a2 = al * sc, b2 = be * sc, g2 = g * sc;
  const float af = (float)a2, bf = (float)b2, gf = (float)g2;
  if (fminf(af, bf) > 1e-30f && fabsf(gf) > 1e-30f) {
    // |g| > tol sqrt(a) sqrt(b): every factor stays in the normal FP32 range here (a squared
    // form would underflow for columns far apart in norm and wrongly stop rotations)
    if (!(fabsf(gf) > tolf * sqrtf(af) * sqrtf(bf))) return false;
    const float zf = __fdividef(bf - af, 2.0f * gf);
    float tf;
    if (fabsf(zf) > 1e18f) tf = __fdividef(0.5f, zf);
    else tf = __fdividef(copysignf(1.0f, zf), fabsf(zf) + sqrtf(fmaf(zf, zf, 1.0f)));
    const float cf = rsqrtf(fmaf(tf, tf, 1.0f));
    const double c0 = (double)cf, s0 = (double)(cf * tf);
    const double dd = fma(c0, c0, fma(s0, s0, -1.0));
    const double pc = fma(fma(0.375, dd, -0.5), dd, 1.0);
    c = c0 * pc;
    s = s0 * pc;
    t = (double)tf;
    return true;
  }
  if (!(g2 * g2 > tol2 * a2 * b2)) return false;
  const double zeta = (b2 - a2) / (2.0 * g2);
  if (fabs(zeta) > 1e100) t = 0.5 / zeta;
  else t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  c = 1.0 / sqrt(1.0 + t * t);
  s = c * t;
  return true;
}

// The same rotation for the scaled form of the sweep (jacobi_solo_impl): returns t exactly as it
// is applied and c = 1 / sqrt(1 + t^2) to FP64 rounding.  In the FP32 branch c0 = rsqrtf(1 + tf^2)
// is corrected in FP64 with the series above, d = c0^2 (1 + t^2) - 1, where c0 t is exact in
// FP64 (two 24-bit significands).
__device__ inline bool jacobi_rotation_ct(double al, double be, double g, double tol2, float tolf, double& c,
                                          double& t) {
  const long long im = max(__double_as_longlong(al), __double_as_longlong(be));
  int ex = (int)(im >> 52) - 1023;
  ex = min(max(ex, -1000), 1000);
  const double sc = pow2i(-ex);
  const double a2 = al * sc, b2 = be * sc, g2 = g * sc;
  const float af = (float)a2, bf = (float)b2, gf = (float)g2;
  if (fminf(af, bf) > 1e-30f && fabsf(gf) > 1e-30f) {
    if (!(fabsf(gf) > tolf * sqrtf(af) * sqrtf(bf))) return false;
    const float zf = __fdividef(bf - af, 2.0f * gf);
    float tf;
    if (fabsf(zf) > 1e18f) tf = __fdividef(0.5f, zf);
    else tf = __fdividef(copysignf(1.0f, zf), fabsf(zf) + sqrtf(fmaf(zf, zf, 1.0f)));
    const float cf = rsqrtf(fmaf(tf, tf, 1.0f));
    const double c0 = (double)cf;
    t = (double)tf;
    const double s0 = c0 * t;
    const double dd = fma(c0, c0, fma(s0, s0, -1.0));
    c = c0 * fma(fma(0.375, dd, -0.5), dd, 1.0);
    return true;
  }
  if (!(g2 * g2 > tol2 * a2 * b2)) return false;
  const double zeta = (b2 - a2) / (2.0 * g2);
  if (fabs(zeta) > 1e100) t = 0.5 / zeta;
  else t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  c = 1.0 / sqrt(1.0 + t * t);
  return true;
}

__device__ inline void rr_pair(int r, int i, int P, int& a, int& b) {
  // round-robin (circle) schedule on P (even) players, round r in [0, P-1); r, i < P - 1
  if (i == 0) {
    a = P - 1;
    b = r;
  } else {
    const int m = P - 1;
    a = r + i;
    if (a >= m) a -= m;
    b = r - i;
    if (b < 0) b += m;
  }
}

__device__ __forceinline__ void jacobi_global_impl(const JacobiDesc* __restrict__ descs,
                                                   const int* __restrict__ di, double* flops) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int crank = (int)cl.block_rank();
  const JacobiDesc& d = descs[blockIdx.y];
  const int q1 = dimv(d.q1, d.q1ref, di), q2 = dimv(d.q2, d.q2ref, di);
  if (crank == 0 && threadIdx.x == 0 && flops && q1 > 0 && q2 > 0) {
    // algorithmic count of an SVD of the q1 x q2 core (R-SVD, Golub & Van Loan)
    double p = max(q1, q2), q = min(q1, q2);
    atomicAdd(&flops[kKindSlot + 3], 4.0 * p * p * q + 8.0 * p * q * q + 9.0 * q * q * q);
  }
  double* M = d.M;
  const size_t ldm = d.ldm;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = warp * C + crank, nw = C * QW;   // consecutive items on different SMs
  // relative orthogonality threshold for a pair: 4 eps sqrt(q1) sits above the rounding noise of
  // a computed cosine (about eps sqrt(q1)), so converged pairs stop, and keeps the kept basis
  // orthogonal enough that the reconstruction error tol * sigma_1 stays far below thr
  const double tol = fmin(1e-13, fmax(1e-15, 8.8e-16 * sqrt((double)q1)));
  // Columns whose squared norm is below dfl are left out of the rotations: they stay below
  // the truncation threshold and together change the core by at most 1e-2 * thr.
  double thr = d.thr;
  if (d.thr_ref) thr *= *d.thr_ref;
  const double dth = 1e-2 * thr / sqrt((double)max(q2, 1));
  const double dfl = dth * dth;
  __shared__ int act[kJacobiMaxCols];
  __shared__ int nact;

  if (crank == 0)
    for (int i = threadIdx.x; i < kMaxSweeps; i += QT) d.rot[i] = 0;
  for (int j = gw; j < q2; j += nw) {
    double s = 0.0;
    for (int i = lane; i < q1; i += 32) {
      double v = M[i + j * ldm];
      s = fma(v, v, s);
    }
    s = warp_sum2(s);
    if (lane == 0) d.nrm[j] = s;
  }
  cl.sync();
  if (q2 < 2 || q1 == 0 || q2 > kJacobiMaxCols) return;
  const bool in_regs = q1 <= 32 * kJacobiRegs;
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    // active columns of this sweep (identical in every CTA: all read the published norms)
    if (threadIdx.x == 0) {
      int c = 0;
      for (int j = 0; j < q2; ++j)
        if (__ldcg(&d.nrm[j]) > dfl) act[c++] = j;
      nact = c;
    }
    // every CTA must have read the norms before any CTA rotates (keeps the lists identical)
    cl.sync();
    const int Ka = nact;
    if (Ka < 2) break;
    const int P = Ka + (Ka & 1);
    int local = 0;
    for (int r = 0; r < P - 1; ++r) {
      for (int pi = gw; pi < P / 2; pi += nw) {
        int ia, ib;
        rr_pair(r, pi, P, ia, ib);
        if (ia >= Ka || ib >= Ka) continue;
        const int a = act[ia], b = act[ib];
        double* ca = M + a * ldm;
        double* cb = M + b * ldm;
        const double al = __ldcg(&d.nrm[a]), be = __ldcg(&d.nrm[b]);
        if (al <= dfl || be <= dfl) continue;
        double na = 0.0, nb = 0.0;
        if (in_regs) {
          // the pair is read once into registers (q1 <= 32 * kJacobiRegs)
          double x[kJacobiRegs], y[kJacobiRegs];
          double g = 0.0;
#pragma unroll
          for (int t = 0; t < kJacobiRegs; ++t) {
            const int i = lane + 32 * t;
            x[t] = i < q1 ? __ldcg(&ca[i]) : 0.0;
            y[t] = i < q1 ? __ldcg(&cb[i]) : 0.0;
            g = fma(x[t], y[t], g);
          }
          g = warp_sum2(g);
          double c, sn, tt;
          if (!(al > 0.0 && be > 0.0) || !jacobi_rotation(al, be, g, tol * tol, (float)tol, c, sn, tt)) continue;
#pragma unroll
          for (int t = 0; t < kJacobiRegs; ++t) {
            const int i = lane + 32 * t;
            const double xn = c * x[t] - sn * y[t];
            const double yn = sn * x[t] + c * y[t];
            na = fma(xn, xn, na);
            nb = fma(yn, yn, nb);
            if (i < q1) {
              ca[i] = xn;
              cb[i] = yn;
            }
          }
        } else {
          // long columns: two passes over L2
          double g = 0.0;
          for (int i = lane; i < q1; i += 32) g = fma(__ldcg(&ca[i]), __ldcg(&cb[i]), g);
          g = warp_sum2(g);
          double c, sn, tt;
          if (!(al > 0.0 && be > 0.0) || !jacobi_rotation(al, be, g, tol * tol, (float)tol, c, sn, tt)) continue;
          for (int i = lane; i < q1; i += 32) {
            const double xv = __ldcg(&ca[i]), yv = __ldcg(&cb[i]);
            const double xn = c * xv - sn * yv;
            const double yn = sn * xv + c * yv;
            ca[i] = xn;
            cb[i] = yn;
            na = fma(xn, xn, na);
            nb = fma(yn, yn, nb);
          }
        }
        na = warp_sum2(na);
        nb = warp_sum2(nb);
        if (lane == 0) {
          d.nrm[a] = na;
          d.nrm[b] = nb;
        }
        ++local;
      }
      cl.sync();
    }
    if (lane == 0 && local) atomicAdd(&d.rot[sweep], local);
    cl.sync();
    if (*(volatile int*)&d.rot[sweep] == 0) break;
  }
}

__global__ void __launch_bounds__(QT) jacobi_cluster_kernel(const JacobiDesc* __restrict__ descs) {
  jacobi_global_impl(descs, descs[blockIdx.y].di, descs[blockIdx.y].fl);
}

// One-sided Jacobi with the core held in distributed shared memory: column j lives in the
// shared memory of CTA j % C.  Each warp rotates 32 / LG column pairs at once, one pair per
// group of LG lanes (LG = 4 or 8, chosen by the dispatcher): the FP64 instructions that form
// the rotation (the scarce resource, see jacobi_rotation) are then shared by several pairs, and
// the dot product needs only log2(LG) shuffle levels.  Control
// flow stays warp-uniform: a group whose pair is converged, deflated or absent applies the
// identity and stores nothing; a warp none of whose pairs rotates skips the application.  Pair
// (a, b) reads and writes both columns through DSMEM; per round that is one remote load, one
// remote store and one cluster barrier.  Rotations take the scaled form of jacobi_solo_impl
// (two FMAs per row; the scales d_j, e_j live with the column's owner and are folded into the
// columns at every sweep start and every 16 rounds).  Same pair schedule, thresholds and
// deflation as jacobi_cluster_kernel.  Columns longer than LG * kJacobiRegs (q1 > 64 for
// LG = 8) are streamed from shared memory twice instead of held in registers.
template <int LG>
__device__ __forceinline__ void jacobi_dsmem_impl(const JacobiDesc* __restrict__ descs, const int* __restrict__ di,
                                                  double* flops, int q1cap, int q2cap) {
  constexpr int PPW = 32 / LG;                            // pairs per warp and step
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int crank = (int)cl.block_rank();
  const JacobiDesc& d = descs[blockIdx.y];
  const int q1 = min(dimv(d.q1, d.q1ref, di), q1cap), q2 = min(dimv(d.q2, d.q2ref, di), q2cap);
  if (crank == 0 && threadIdx.x == 0 && flops && q1 > 0 && q2 > 0) {
    double p = max(q1, q2), q = min(q1, q2);
    atomicAdd(&flops[kKindSlot + 3], 4.0 * p * p * q + 8.0 * p * q * q + 9.0 * q * q * q);
  }
  extern __shared__ double jsm[];
  const int nloc = (q2 + C - 1) / C;                     // laid out by the actual core size
  const int ldc = max(q1, 1);
  double* cols = jsm;                                    // nloc x ldc, slot s = column crank + s*C
  double* cn = cols + (size_t)nloc * ldc;                // current squared norms of own columns
  double* dsc = cn + nloc;                               // scales d_j of own columns
  double* esc = dsc + nloc;                              // e_j ~ 1 / d_j
  double* nall = esc + nloc;                             // squared norms of all columns (sweep start)
  int* act = reinterpret_cast<int*>(nall + q2);          // active columns of the sweep
  __shared__ int nact;
  double* M = d.M;
  const size_t ldm = d.ldm;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane / LG, gl = lane % LG;             // pair slot in the warp, lane in the group
  const double tol = fmin(1e-13, fmax(1e-15, 8.8e-16 * sqrt((double)q1)));   // as jacobi_cluster_kernel
  const double tol2 = tol * tol;
  const float tolf = (float)tol;
  double thr = d.thr;
  if (d.thr_ref) thr *= *d.thr_ref;
  const double dth = 1e-2 * thr / sqrt((double)max(q2, 1));
  const double dfl = dth * dth;
  const long long dfl_bits = __double_as_longlong(dfl);

  if (crank == 0)
    for (int i = threadIdx.x; i < kMaxSweeps; i += QT) d.rot[i] = 0;
  for (int sl = 0; sl < nloc; ++sl) {
    const int j = crank + sl * C;
    if (j >= q2) break;
    for (int i = threadIdx.x; i < q1; i += QT) cols[(size_t)sl * ldc + i] = M[i + (size_t)j * ldm];
  }
  for (int sl = threadIdx.x; sl < nloc; sl += QT) dsc[sl] = 1.0;
  // every CTA of the cluster must be running before any distributed shared memory access
  cl.sync();

  const int gw = warp * C + crank, nw = C * QW;   // consecutive items on different SMs
  const int nreg = (q1 + LG - 1) / LG;                   // register slots in use (uniform)
  const bool inreg = nreg <= kJacobiRegs;
  for (int sweep = 0; sweep <= kMaxSweeps; ++sweep) {
    // fold the scales into own columns; exact squared norms, broadcast into every CTA's copy
    for (int sl = warp; sl < nloc; sl += QW) {
      const int j = crank + sl * C;
      if (j >= q2) break;
      const double s = dsc[sl];
      double v = 0.0;
      for (int i = lane; i < q1; i += 32) {
        const double x = cols[(size_t)sl * ldc + i] * s;
        cols[(size_t)sl * ldc + i] = x;
        v = fma(x, x, v);
      }
      v = warp_sum2(v);
      if (lane < C) cl.map_shared_rank(nall, lane)[j] = v;
      if (lane == 0) {
        cn[sl] = v;
        d.nrm[j] = v;
        dsc[sl] = 1.0;
        esc[sl] = 1.0;
      }
    }
    cl.sync();
    if (sweep == kMaxSweeps || q2 < 2 || q1 == 0) break;
    if (threadIdx.x == 0) {
      int c = 0;
      for (int j = 0; j < q2; ++j)
        if (nall[j] > dfl) act[c++] = j;
      nact = c;
    }
    __syncthreads();
    const int Ka = nact;
    if (Ka < 2) break;
    const int P = Ka + (Ka & 1);
    int local = 0;
    for (int r = 0; r < P - 1; ++r) {
      if (r > 0 && r % 16 == 0) {
        // fold own scales (true norms are tracked unchanged); the previous round's barrier
        // ordered every remote access to these columns
        for (int sl = warp; sl < nloc; sl += QW) {
          if (crank + sl * C >= q2) break;
          const double s = dsc[sl];
          for (int i = lane; i < q1; i += 32) cols[(size_t)sl * ldc + i] *= s;
          __syncwarp();
          if (lane == 0) {
            dsc[sl] = 1.0;
            esc[sl] = 1.0;
          }
        }
        cl.sync();
      }
      for (int pb = gw * PPW; pb < P / 2; pb += nw * PPW) {
        const int pi = pb + sub;
        int ia = 0, ib = 0;
        bool valid = pi < P / 2;
        if (valid) {
          rr_pair(r, pi, P, ia, ib);
          valid = ia < Ka && ib < Ka;
        }
        const int a = valid ? act[ia] : 0, b = valid ? act[ib] : 0;
        double* xa = cl.map_shared_rank(cols, a % C) + (size_t)(a / C) * ldc;
        double* yb = cl.map_shared_rank(cols, b % C) + (size_t)(b / C) * ldc;
        // per-column scalars of the owners (pointers are formed again for the stores: fewer live
        // registers)
        const int ao = a % C, as = a / C, bo = b % C, bs = b / C;
        const double al = valid ? cl.map_shared_rank(cn, ao)[as] : 0.0;
        const double be = valid ? cl.map_shared_rank(cn, bo)[bs] : 0.0;
        const double da = valid ? cl.map_shared_rank(dsc, ao)[as] : 1.0;
        const double db = valid ? cl.map_shared_rank(dsc, bo)[bs] : 1.0;
        double x[kJacobiRegs], y[kJacobiRegs];
        double g0 = 0.0, g1 = 0.0;
        if (inreg) {
#pragma unroll
          for (int t = 0; t < kJacobiRegs; ++t) {
            if (t < nreg) {
              const int i = gl + LG * t;
              const bool in = valid && i < q1;
              x[t] = in ? xa[i] : 0.0;
              y[t] = in ? yb[i] : 0.0;
              if (t & 1) g1 = fma(x[t], y[t], g1);
              else g0 = fma(x[t], y[t], g0);
            }
          }
        } else if (valid) {
          for (int i = gl; i < q1; i += 2 * LG) {
            g0 = fma(xa[i], yb[i], g0);
            if (i + LG < q1) g1 = fma(xa[i + LG], yb[i + LG], g1);
          }
        }
        double gw2 = g0 + g1;
#pragma unroll
        for (int o = LG / 2; o > 0; o >>= 1) gw2 += __shfl_xor_sync(0xffffffffu, gw2, o);
        const double g = da * db * gw2;                   // gamma of the true columns
        // every lane of a group holds g and forms the same rotation (an FP64 instruction costs
        // the same for one lane as for 32); the deflation test runs on the bit patterns
        double c = 1.0, tt = 0.0;
        const bool doit = valid && __double_as_longlong(al) > dfl_bits && __double_as_longlong(be) > dfl_bits &&
                          jacobi_rotation_ct(al, be, g, tol2, tolf, c, tt);
        if (!doit) {
          c = 1.0;
          tt = 0.0;
        }
        const double ea = doit ? cl.map_shared_rank(esc, ao)[as] : 1.0;
        const double eb = doit ? cl.map_shared_rank(esc, bo)[bs] : 1.0;
        const double mu = doit ? tt * db * ea : 0.0, nu = doit ? tt * da * eb : 0.0;
        // alpha' = alpha - t gamma, beta' = beta + t gamma; the shrinking column's norm is summed
        // exactly when it loses more than half of its mass (cancellation)
        const double tg = tt * g;
        const bool a_shrinks = tg > 0.0;
        const bool exact = doit && (a_shrinks ? (tg > 0.5 * al) : (-tg > 0.5 * be));
        const bool any_exact = __any_sync(0xffffffffu, exact);
        const bool any_doit = __any_sync(0xffffffffu, doit);   // else the warp's pairs are final
        // the pair's scalars are stored before the columns (no other pair of the round reads
        // them), so that they are not live across the application; an exact norm replaces the
        // tracked one afterwards
        const double dsh = c * (a_shrinks ? da : db);     // new scale of the shrinking column
        if (doit && gl == 0) {
          const double rc = fma(tt, tt, 1.0) * c;         // 1 / c
          cl.map_shared_rank(cn, ao)[as] = fma(-tt, g, al);
          cl.map_shared_rank(cn, bo)[bs] = fma(tt, g, be);
          cl.map_shared_rank(esc, ao)[as] = ea * rc;
          cl.map_shared_rank(esc, bo)[bs] = eb * rc;
          cl.map_shared_rank(dsc, ao)[as] = c * da;
          cl.map_shared_rank(dsc, bo)[bs] = c * db;
          ++local;
        }
        double s0 = 0.0, s1 = 0.0;
        if (inreg && any_doit) {
#pragma unroll
          for (int t = 0; t < kJacobiRegs; ++t) {
            if (t < nreg) {
              const double xn = fma(-mu, y[t], x[t]);
              const double yn = fma(nu, x[t], y[t]);
              const int i = gl + LG * t;
              if (doit && i < q1) {
                xa[i] = xn;
                yb[i] = yn;
              }
              if (any_exact) {
                const double v = a_shrinks ? xn : yn;
                if (t & 1) s1 = fma(v, v, s1);
                else s0 = fma(v, v, s0);
              }
            }
          }
        } else if (doit) {
          for (int i = gl; i < q1; i += LG) {
            const double xv = xa[i], yv = yb[i];
            const double xn = fma(-mu, yv, xv);
            const double yn = fma(nu, xv, yv);
            xa[i] = xn;
            yb[i] = yn;
            const double v = a_shrinks ? xn : yn;
            s0 = fma(v, v, s0);
          }
        }
        double ss = s0 + s1;
        if (any_exact) {
#pragma unroll
          for (int o = LG / 2; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        }
        if (exact && gl == 0) {
          if (a_shrinks) cl.map_shared_rank(cn, ao)[as] = dsh * dsh * ss;
          else cl.map_shared_rank(cn, bo)[bs] = dsh * dsh * ss;
        }
      }
      cl.sync();
    }
    if (local) atomicAdd(&d.rot[sweep], local);
    cl.sync();
    if (*(volatile int*)&d.rot[sweep] == 0) sweep = kMaxSweeps - 1;   // converged: final norms next pass
  }
  // write the rotated columns back (the rank selection reads them from global memory)
  for (int sl = 0; sl < nloc; ++sl) {
    const int j = crank + sl * C;
    if (j >= q2) break;
    for (int i = threadIdx.x; i < q1; i += QT) M[i + (size_t)j * ldm] = cols[(size_t)sl * ldc + i];
  }
  cl.sync();   // no CTA may exit while others still access its shared memory
}

// One-sided Jacobi, owner-computes form.  Column j lives in the shared memory of CTA j % C, in
// two buffers: round r reads buffer r & 1 and writes buffer (r + 1) & 1.  For every pair (a, b)
// of a round, the CTA owning a and the CTA owning b both form the same rotation from the same
// data (identical instruction sequences on identical inputs give identical results) and each
// writes only its own column and norm, into its own shared memory.  Remote traffic is therefore
// loads only; the one cluster barrier per round orders the round's writes before the next
// round's reads and the round's reads before the buffer is written again.  A column without a
// partner in a round is copied to the other buffer.  Rotations take the scaled form of
// jacobi_solo_impl (the owner's new column is one FMA per row; scales are double-buffered with
// the columns and folded at every sweep start and every 16 rounds).  Lane groups, thresholds,
// deflation and the exact-norm rule as in jacobi_dsmem_impl.
template <int LG, bool SOLO>
__device__ __forceinline__ void jacobi_owner_impl(const JacobiDesc* __restrict__ descs, const int* __restrict__ di,
                                                  double* flops, int q1cap, int q2cap) {
  constexpr int PPW = 32 / LG;                            // pair tasks per warp and step
  cg::cluster_group cl = cg::this_cluster();
  const int C = SOLO ? 1 : (int)cl.num_blocks();
  const int crank = SOLO ? 0 : (int)cl.block_rank();
  const JacobiDesc& d = descs[blockIdx.y];
  const int q1 = min(dimv(d.q1, d.q1ref, di), q1cap), q2 = min(dimv(d.q2, d.q2ref, di), q2cap);
  if (crank == 0 && threadIdx.x == 0 && flops && q1 > 0 && q2 > 0) {
    double p = max(q1, q2), q = min(q1, q2);
    atomicAdd(&flops[kKindSlot + 3], 4.0 * p * p * q + 8.0 * p * q * q + 9.0 * q * q * q);
  }
  extern __shared__ double jsm[];
  // laid out by the core's actual size (ranks are known only here), which the caller checked
  // against the shared memory of the launch
  const int nloc = (q2 + C - 1) / C;
  const int ldc = max(q1, 1);
  const int q2n = q2;
  double* cols0 = jsm;                                   // [2][nloc][ldc], slot s = column crank + s*C
  double* cn0 = cols0 + 2 * (size_t)nloc * ldc;          // [2][nloc] tracked squared norms
  double* sc0 = cn0 + 2 * nloc;                          // [2][nloc] scales d_j
  double* ec0 = sc0 + 2 * nloc;                          // [2][nloc] e_j ~ 1 / d_j
  double* nall = ec0 + 2 * nloc;                         // squared norms of all columns (sweep start)
  int* act = reinterpret_cast<int*>(nall + q2n);         // active columns of the sweep
  int* own = act + q2n;                                // positions (in act) of own active columns
  __shared__ int nact, nown;
  double* M = d.M;
  const size_t ldm = d.ldm;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane / LG, gl = lane % LG;
  const double tol = fmin(1e-13, fmax(1e-15, 8.8e-16 * sqrt((double)q1)));   // as jacobi_cluster_kernel
  const double tol2 = tol * tol;
  const float tolf = (float)tol;
  double thr = d.thr;
  if (d.thr_ref) thr *= *d.thr_ref;
  const double dth = 1e-2 * thr / sqrt((double)max(q2, 1));
  const double dfl = dth * dth;
  const long long dfl_bits = __double_as_longlong(dfl);
  const size_t bufstride = (size_t)nloc * ldc;

  if (crank == 0)
    for (int i = threadIdx.x; i < kMaxSweeps; i += QT) d.rot[i] = 0;
  for (int sl = 0; sl < nloc; ++sl) {
    const int j = crank + sl * C;
    if (j >= q2) break;
    for (int i = threadIdx.x; i < q1; i += QT) cols0[(size_t)sl * ldc + i] = M[i + (size_t)j * ldm];
  }
  for (int sl = threadIdx.x; sl < nloc; sl += QT) sc0[sl] = 1.0;
  // every CTA of the cluster must be running before any distributed shared memory access
  csync<SOLO>(cl);

  const int nreg = (q1 + LG - 1) / LG;
  const bool inreg = nreg <= kJacobiRegs;
  int cur = 0;                                           // buffer holding the current columns
  for (int sweep = 0; sweep <= kMaxSweeps; ++sweep) {
    double* cols = cols0 + cur * bufstride;
    double* cn = cn0 + cur * nloc;
    // fold the scales into own columns; exact squared norms, broadcast into every CTA's copy
    for (int sl = warp; sl < nloc; sl += QW) {
      const int j = crank + sl * C;
      if (j >= q2) break;
      const double s = sc0[cur * nloc + sl];
      double v = 0.0;
      for (int i = lane; i < q1; i += 32) {
        const double x = cols[(size_t)sl * ldc + i] * s;
        cols[(size_t)sl * ldc + i] = x;
        v = fma(x, x, v);
      }
      v = warp_sum2(v);
      if (lane < C) rmt<SOLO>(cl, nall, lane)[j] = v;
      if (lane == 0) {
        cn[sl] = v;
        d.nrm[j] = v;
        sc0[cur * nloc + sl] = 1.0;
        ec0[cur * nloc + sl] = 1.0;
      }
    }
    csync<SOLO>(cl);
    if (sweep == kMaxSweeps || q2 < 2 || q1 == 0) break;
    if (threadIdx.x == 0) {
      // act[x] packs (slot << 5) | owner CTA of the x-th active column, so the round loop needs
      // no integer division by the cluster size
      int c = 0, o = 0;
      for (int j = 0; j < q2; ++j)
        if (nall[j] > dfl) {
          const int ow = j % C;
          if (ow == crank) own[o++] = c;
          act[c++] = ((j / C) << 5) | ow;
        }
      nact = c;
      nown = o;
    }
    __syncthreads();
    const int Ka = nact, No = nown;
    if (Ka < 2) break;
    const int P = Ka + (Ka & 1), m = P - 1;
    int local = 0;
    for (int r = 0; r < P - 1; ++r) {
      if (r > 0 && r % 16 == 0) {
        // fold the scales of own active columns in the buffer this round reads (the previous
        // round's barrier ordered every access to it)
        for (int t = warp; t < No; t += QW) {
          const int sl = act[own[t]] >> 5;
          const double s = sc0[cur * nloc + sl];
          for (int i = lane; i < q1; i += 32) cols0[cur * bufstride + (size_t)sl * ldc + i] *= s;
          __syncwarp();
          if (lane == 0) {
            sc0[cur * nloc + sl] = 1.0;
            ec0[cur * nloc + sl] = 1.0;
          }
        }
        csync<SOLO>(cl);
      }
      const int rb = cur, wb = cur ^ 1;                  // read / write buffers of this round
      for (int tb = warp * PPW; tb < No; tb += QW * PPW) {
        const int t = tb + sub;
        const bool task = t < No;
        const int x = task ? own[t] : 0;
        // partner of player x in round r of the circle schedule on P players: 2r - x mod m
        int y = 2 * r - x;
        y += (y < 0) ? m : 0;
        y -= (y >= m) ? m : 0;
        y = (x == m) ? r : (x == r ? m : y);
        const bool valid = task && y < Ka;
        const int lo = min(x, y), hi = max(x, y);
        const int pa = valid ? act[lo] : 0, pb = valid ? act[hi] : 0;
        const int ao = pa & 31, as = pa >> 5, bo = pb & 31, bs = pb >> 5;
        const bool mine_a = x == lo;                     // this task writes column a (else b)
        const int ms = task ? (act[x] >> 5) : 0;         // own slot
        const double* xa = rmt<SOLO>(cl, cols0, ao) + rb * bufstride + (size_t)as * ldc;
        const double* yb = rmt<SOLO>(cl, cols0, bo) + rb * bufstride + (size_t)bs * ldc;
        const double al = valid ? rmt<SOLO>(cl, cn0, ao)[rb * nloc + as] : 0.0;
        const double be = valid ? rmt<SOLO>(cl, cn0, bo)[rb * nloc + bs] : 0.0;
        const double da = valid ? rmt<SOLO>(cl, sc0, ao)[rb * nloc + as] : 1.0;
        const double db = valid ? rmt<SOLO>(cl, sc0, bo)[rb * nloc + bs] : 1.0;
        double* dst = cols0 + wb * bufstride + (size_t)ms * ldc;
        const double* src = cols0 + rb * bufstride + (size_t)ms * ldc;
        double xr[kJacobiRegs], yr[kJacobiRegs];
        double g0 = 0.0, g1 = 0.0;
        if (inreg) {
#pragma unroll
          for (int u = 0; u < kJacobiRegs; ++u) {
            if (u < nreg) {
              const int i = gl + LG * u;
              const bool in = valid && i < q1;
              xr[u] = in ? xa[i] : 0.0;
              yr[u] = in ? yb[i] : 0.0;
              if (u & 1) g1 = fma(xr[u], yr[u], g1);
              else g0 = fma(xr[u], yr[u], g0);
            }
          }
        } else if (valid) {
          for (int i = gl; i < q1; i += 2 * LG) {
            g0 = fma(xa[i], yb[i], g0);
            if (i + LG < q1) g1 = fma(xa[i + LG], yb[i + LG], g1);
          }
        }
        double gw2 = g0 + g1;
#pragma unroll
        for (int o = LG / 2; o > 0; o >>= 1) gw2 += __shfl_xor_sync(0xffffffffu, gw2, o);
        const double g = da * db * gw2;                   // gamma of the true columns
        double c = 1.0, tt = 0.0;
        const bool doit = valid && __double_as_longlong(al) > dfl_bits && __double_as_longlong(be) > dfl_bits &&
                          jacobi_rotation_ct(al, be, g, tol2, tolf, c, tt);
        if (!doit) {
          c = 1.0;
          tt = 0.0;
        }
        // own new column: w_a - (t d_b e_a) w_b (a) or w_b + (t d_a e_b) w_a (b)
        const double eown = ec0[rb * nloc + (task ? ms : 0)];
        const double m1 = mine_a ? -tt * db * eown : tt * da * eown;
        const double tg = tt * g;
        const bool a_shrinks = tg > 0.0;
        const bool exact = doit && (mine_a == a_shrinks) && (a_shrinks ? (tg > 0.5 * al) : (-tg > 0.5 * be));
        const bool any_exact = __any_sync(0xffffffffu, exact);
        const bool any_doit = __any_sync(0xffffffffu, doit);
        // own scalars of the next buffer are stored before the column (only this task writes
        // them), so that they are not live across the application
        const double dnew = c * (mine_a ? da : db);
        if (task && gl == 0) {
          const int sl = ms;
          cn0[wb * nloc + sl] = doit ? (mine_a ? fma(-tt, g, al) : fma(tt, g, be)) : cn0[rb * nloc + sl];
          sc0[wb * nloc + sl] = doit ? dnew : sc0[rb * nloc + sl];
          ec0[wb * nloc + sl] = doit ? eown * (fma(tt, tt, 1.0) * c) : eown;
          if (doit && mine_a) ++local;
        }
        double s0 = 0.0, s1 = 0.0;
        if (inreg && any_doit) {
#pragma unroll
          for (int u = 0; u < kJacobiRegs; ++u) {
            if (u < nreg) {
              const int i = gl + LG * u;
              const double v = doit ? fma(m1, mine_a ? yr[u] : xr[u], mine_a ? xr[u] : yr[u]) : 0.0;
              if (task && i < q1) dst[i] = doit ? v : src[i];
              if (any_exact) {
                if (u & 1) s1 = fma(v, v, s1);
                else s0 = fma(v, v, s0);
              }
            }
          }
        } else if (inreg) {
          // no pair of the warp rotates: carry the own columns over (no arithmetic)
#pragma unroll
          for (int u = 0; u < kJacobiRegs; ++u) {
            if (u < nreg) {
              const int i = gl + LG * u;
              if (task && i < q1) dst[i] = src[i];
            }
          }
        } else if (task) {
          for (int i = gl; i < q1; i += LG) {
            const double v = doit ? fma(m1, mine_a ? yb[i] : xa[i], mine_a ? xa[i] : yb[i]) : src[i];
            dst[i] = v;
            s0 = fma(v, v, s0);
          }
        }
        double ss = s0 + s1;
        if (any_exact) {
#pragma unroll
          for (int o = LG / 2; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        }
        if (exact && gl == 0) cn0[wb * nloc + ms] = dnew * dnew * ss;
      }
      csync<SOLO>(cl);
      cur ^= 1;
    }
    if (local) atomicAdd(&d.rot[sweep], local);
    // inactive (deflated) own columns: bring them into the current buffer before the norm pass
    for (int sl = 0; sl < nloc; ++sl) {
      const int j = crank + sl * C;
      if (j >= q2) break;
      if (!(nall[j] > dfl) && ((P - 1) & 1)) {
        for (int i = threadIdx.x; i < q1; i += QT) cols0[cur * bufstride + (size_t)sl * ldc + i] =
                                                      cols0[(cur ^ 1) * bufstride + (size_t)sl * ldc + i];
        if (threadIdx.x == 0) sc0[cur * nloc + sl] = sc0[(cur ^ 1) * nloc + sl];
      }
    }
    csync<SOLO>(cl);
    if (*(volatile int*)&d.rot[sweep] == 0) sweep = kMaxSweeps - 1;   // converged: final norms next pass
  }
  // write the rotated columns back (the rank selection reads them from global memory)
  for (int sl = 0; sl < nloc; ++sl) {
    const int j = crank + sl * C;
    if (j >= q2) break;
    for (int i = threadIdx.x; i < q1; i += QT) M[i + (size_t)j * ldm] = cols0[cur * bufstride + (size_t)sl * ldc + i];
  }
  csync<SOLO>(cl);   // no CTA may exit while others still access its shared memory
}

// Shared memory of the one-CTA scaled Jacobi (jacobi_solo_impl) for a q1 x q2 core.
__host__ __device__ inline size_t jacobi_solo_bytes(int q1, int q2) {
  return (size_t)q2 * max(q1, 1) * sizeof(double) + 3 * (size_t)q2 * sizeof(double) + (size_t)q2 * sizeof(int) + 64;
}

// One-sided Jacobi on one CTA with scaled rotations.  Column j is held as w_j with the true
// column d_j w_j; the CTA also keeps e_j ~ 1 / d_j and the true squared norm.  A rotation of
// the pair (a, b) with tangent t and cosine c (jacobi_rotation_ct) is applied as
//     w_a <- w_a - (t d_b e_a) w_b,   w_b <- w_b + (t d_a e_b) w_a,   d_a, d_b <- c d_a, c d_b,
// which is the plane rotation c [1, -t; t, 1] of the true columns with two FMAs per row instead
// of two multiplications and two FMAs (Rutishauser's scaled form of the rotation).  The scales
// are folded into the columns at the start of every sweep and every 16 rounds, which bounds
// both the growth of w (c >= 1 / sqrt 2) and the drift of d_j e_j away from 1.  One group of
// LG lanes rotates one pair; pairs of a round are disjoint, so columns are updated in place
// and one block barrier separates the rounds.  Pair schedule, thresholds, deflation and the
// exact-norm rule as in the other forms.
template <int LG>
__device__ __forceinline__ void jacobi_solo_impl(const JacobiDesc* __restrict__ descs, const int* __restrict__ di,
                                                 double* flops, int q1cap, int q2cap) {
  constexpr int PPW = 32 / LG;                            // pairs per warp and step
  constexpr int kFold = 16;                               // rounds between folds of the scales
  const JacobiDesc& d = descs[blockIdx.y];
  const int q1 = min(dimv(d.q1, d.q1ref, di), q1cap), q2 = min(dimv(d.q2, d.q2ref, di), q2cap);
  if (threadIdx.x == 0 && flops && q1 > 0 && q2 > 0) {
    double p = max(q1, q2), q = min(q1, q2);
    atomicAdd(&flops[kKindSlot + 3], 4.0 * p * p * q + 8.0 * p * q * q + 9.0 * q * q * q);
  }
  extern __shared__ double jsm[];
  const int ldc = max(q1, 1);
  double* cols = jsm;                                     // q2 x ldc: w
  double* cn = cols + (size_t)q2 * ldc;                   // true squared norms
  double* dsc = cn + q2;                                  // d_j
  double* esc = dsc + q2;                                 // e_j
  int* act = reinterpret_cast<int*>(esc + q2);            // active columns of the sweep
  __shared__ int nact, nrot;
  double* M = d.M;
  const size_t ldm = d.ldm;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane / LG, gl = lane % LG;
  const double tol = fmin(1e-13, fmax(1e-15, 8.8e-16 * sqrt((double)q1)));   // as jacobi_cluster_kernel
  const double tol2 = tol * tol;
  const float tolf = (float)tol;
  double thr = d.thr;
  if (d.thr_ref) thr *= *d.thr_ref;
  const double dth = 1e-2 * thr / sqrt((double)max(q2, 1));
  const double dfl = dth * dth;
  const long long dfl_bits = __double_as_longlong(dfl);

  for (int j = 0; j < q2; ++j)
    for (int i = threadIdx.x; i < q1; i += QT) cols[(size_t)j * ldc + i] = M[i + (size_t)j * ldm];
  for (int j = threadIdx.x; j < q2; j += QT) dsc[j] = 1.0;
  __syncthreads();

  const int nreg = (q1 + LG - 1) / LG;
  const bool inreg = nreg <= kJacobiRegs;
  for (int sweep = 0; sweep <= kMaxSweeps; ++sweep) {
    // fold the scales into the columns and take exact squared norms
    for (int j = warp; j < q2; j += QW) {
      const double s = dsc[j];
      double v = 0.0;
      for (int i = lane; i < q1; i += 32) {
        const double x = cols[(size_t)j * ldc + i] * s;
        cols[(size_t)j * ldc + i] = x;
        v = fma(x, x, v);
      }
      v = warp_sum2(v);
      if (lane == 0) {
        cn[j] = v;
        d.nrm[j] = v;
        dsc[j] = 1.0;
        esc[j] = 1.0;
      }
    }
    __syncthreads();
    if (sweep == kMaxSweeps || q2 < 2 || q1 == 0) break;
    if (threadIdx.x == 0) {
      int c = 0;
      for (int j = 0; j < q2; ++j)
        if (cn[j] > dfl) act[c++] = j;
      nact = c;
      nrot = 0;
    }
    __syncthreads();
    const int Ka = nact;
    if (Ka < 2) break;
    const int P = Ka + (Ka & 1);
    int local = 0;
    for (int r = 0; r < P - 1; ++r) {
      if (r > 0 && r % kFold == 0) {
        // fold the scales of the active columns (their true norms are tracked unchanged)
        for (int x = warp; x < Ka; x += QW) {
          const int j = act[x];
          const double s = dsc[j];
          for (int i = lane; i < q1; i += 32) cols[(size_t)j * ldc + i] *= s;
          __syncwarp();
          if (lane == 0) {
            dsc[j] = 1.0;
            esc[j] = 1.0;
          }
        }
        __syncthreads();
      }
      for (int pb = warp * PPW; pb < P / 2; pb += QW * PPW) {
        const int pi = pb + sub;
        int ia = 0, ib = 0;
        bool valid = pi < P / 2;
        if (valid) {
          rr_pair(r, pi, P, ia, ib);
          valid = ia < Ka && ib < Ka;
        }
        const int a = valid ? act[ia] : 0, b = valid ? act[ib] : 0;
        double* xa = cols + (size_t)a * ldc;
        double* yb = cols + (size_t)b * ldc;
        const double al = valid ? cn[a] : 0.0, be = valid ? cn[b] : 0.0;
        const double da = dsc[a], db = dsc[b];
        double x[kJacobiRegs], y[kJacobiRegs];
        double g0 = 0.0, g1 = 0.0;
        if (inreg) {
#pragma unroll
          for (int u = 0; u < kJacobiRegs; ++u) {
            if (u < nreg) {
              const int i = gl + LG * u;
              const bool in = valid && i < q1;
              x[u] = in ? xa[i] : 0.0;
              y[u] = in ? yb[i] : 0.0;
              if (u & 1) g1 = fma(x[u], y[u], g1);
              else g0 = fma(x[u], y[u], g0);
            }
          }
        } else if (valid) {
          for (int i = gl; i < q1; i += 2 * LG) {
            g0 = fma(xa[i], yb[i], g0);
            if (i + LG < q1) g1 = fma(xa[i + LG], yb[i + LG], g1);
          }
        }
        double gw = g0 + g1;
#pragma unroll
        for (int o = LG / 2; o > 0; o >>= 1) gw += __shfl_xor_sync(0xffffffffu, gw, o);
        const double g = da * db * gw;                    // gamma of the true columns
        double c = 1.0, tt = 0.0;
        const bool doit = valid && __double_as_longlong(al) > dfl_bits && __double_as_longlong(be) > dfl_bits &&
                          jacobi_rotation_ct(al, be, g, tol2, tolf, c, tt);
        if (!doit) {
          c = 1.0;
          tt = 0.0;
        }
        const double mu = tt * db * esc[a], nu = tt * da * esc[b];
        const double tg = tt * g;
        const bool a_shrinks = tg > 0.0;
        const bool exact = doit && (a_shrinks ? (tg > 0.5 * al) : (-tg > 0.5 * be));
        const bool any_exact = __any_sync(0xffffffffu, exact);
        const bool any_doit = __any_sync(0xffffffffu, doit);
        double s0 = 0.0, s1 = 0.0;
        if (inreg && any_doit) {
#pragma unroll
          for (int u = 0; u < kJacobiRegs; ++u) {
            if (u < nreg) {
              const double xn = fma(-mu, y[u], x[u]);
              const double yn = fma(nu, x[u], y[u]);
              const int i = gl + LG * u;
              if (doit && i < q1) {
                xa[i] = xn;
                yb[i] = yn;
              }
              if (any_exact) {
                const double v = a_shrinks ? xn : yn;
                if (u & 1) s1 = fma(v, v, s1);
                else s0 = fma(v, v, s0);
              }
            }
          }
        } else if (doit) {
          for (int i = gl; i < q1; i += LG) {
            const double xv = xa[i], yv = yb[i];
            const double xn = fma(-mu, yv, xv);
            const double yn = fma(nu, xv, yv);
            xa[i] = xn;
            yb[i] = yn;
            const double v = a_shrinks ? xn : yn;
            s0 = fma(v, v, s0);
          }
        }
        double ss = s0 + s1;
        if (any_exact) {
#pragma unroll
          for (int o = LG / 2; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        }
        if (doit && gl == 0) {
          const double dan = c * da, dbn = c * db;
          const double rc = fma(tt, tt, 1.0) * c;         // 1 / c
          double na = fma(-tt, g, al), nb = fma(tt, g, be);
          if (exact) {
            if (a_shrinks) na = dan * dan * ss;
            else nb = dbn * dbn * ss;
          }
          cn[a] = na;
          cn[b] = nb;
          dsc[a] = dan;
          dsc[b] = dbn;
          esc[a] *= rc;
          esc[b] *= rc;
          ++local;
        }
      }
      __syncthreads();
    }
    if (local) atomicAdd(&nrot, local);
    __syncthreads();
    if (threadIdx.x == 0) d.rot[sweep] = nrot;
    if (nrot == 0) sweep = kMaxSweeps - 1;                // converged: final norms next pass
    __syncthreads();                                      // nrot is read before it is reset
  }
  for (int j = 0; j < q2; ++j)
    for (int i = threadIdx.x; i < q1; i += QT) M[i + (size_t)j * ldm] = cols[(size_t)j * ldc + i];
}

// Shared memory of the remote-store Jacobi (jacobi_dsmem_impl) for a core of at most q1cap x q2cap.
__host__ __device__ inline size_t jacobi_dsmem_bytes(int q1cap, int q2cap, int cluster) {
  const size_t nloc = (q2cap + cluster - 1) / cluster;
  return nloc * (q1cap + 3) * sizeof(double) + (size_t)q2cap * sizeof(double) + (size_t)q2cap * sizeof(int) + 64;
}
// Shared memory of the owner-computes Jacobi for a core of at most q1cap x q2cap on `cluster` CTAs.
__host__ __device__ inline size_t jacobi_owner_bytes(int q1cap, int q2cap, int cluster) {
  const size_t nloc = (q2cap + cluster - 1) / cluster;
  return 2 * nloc * (q1cap + 3) * sizeof(double) + (size_t)q2cap * sizeof(double) +
         ((size_t)q2cap + nloc) * sizeof(int) + 64;
}
constexpr int kJacobiSoloCols = 32;   // cores up to this many columns run on one CTA (twice as
                                      // many while factorizations share the SMs)

// Lane-group width from the actual column length of this cluster's core (ranks are known only
// on the device; every CTA of the cluster reads the same descriptor, so the choice is uniform):
// 4 lanes per pair up to 32 rows, else 8, with columns longer than 64 rows streamed from
// shared memory.  Wider groups would hold longer columns in registers, but the rotation's
// scalar FP64 work (scales, tangent, cosine: about 18 instructions per group) is shared by the
// 32 / LG pairs of a warp, and with 32 lanes per pair it costs as much as the rows themselves.
// kOwner: the instantiation launched on clusters of 8 or more CTAs for a factorization alone on
// the GPU, the only launches where the owner-computes form is chosen (each instantiation gets
// its own register allocation); that form keeps the wider groups, since alone on the GPU the
// round's latency matters more than its FP64 instructions.
template <bool kOwner>
__global__ void __launch_bounds__(QT, 2) jacobi_dsmem_kernel(const JacobiDesc* __restrict__ descs,
                                                          int q1cap, int q2cap, int smem_bytes, int solo_cols) {
  // The form is chosen from the core's actual size (every CTA of the cluster reads the same
  // descriptor): one CTA for small cores; on clusters of 8 or more CTAs owner-computes when its
  // two column buffers fit in the shared memory of the launch; else remote-store when one buffer
  // fits; global memory otherwise (owner-computes needs more shared memory than remote-store,
  // so it is never the fallback).
  const JacobiDesc& d = descs[blockIdx.y];
  const int* di = d.di;
  double* flops = d.fl;
  const int q1 = min(dimv(d.q1, d.q1ref, di), q1cap);
  const int q2 = min(dimv(d.q2, d.q2ref, di), q2cap);
  const int C = (int)cg::this_cluster().num_blocks();
  const size_t avail = (size_t)smem_bytes;
  if (q2 <= solo_cols && jacobi_solo_bytes(q1, q2) <= avail) {
    if (cg::this_cluster().block_rank() != 0) return;
    if (q1 <= 4 * kJacobiRegs) jacobi_solo_impl<4>(descs, di, flops, q1cap, q2cap);
    else jacobi_solo_impl<8>(descs, di, flops, q1cap, q2cap);
  } else if (kOwner && C >= 8 && jacobi_owner_bytes(q1, q2, C) <= avail) {
    // owner-computes shortens the round (only loads cross SMs) but computes every pair on both
    // owners: it pays off on large clusters, where a round is latency-bound, not on small ones,
    // where the SM's FP64 issue rate is the limit
    if (q1 <= 4 * kJacobiRegs) jacobi_owner_impl<4, false>(descs, di, flops, q1cap, q2cap);
    else if (q1 <= 8 * kJacobiRegs) jacobi_owner_impl<8, false>(descs, di, flops, q1cap, q2cap);
    else if (q1 <= 16 * kJacobiRegs) jacobi_owner_impl<16, false>(descs, di, flops, q1cap, q2cap);
    else jacobi_owner_impl<32, false>(descs, di, flops, q1cap, q2cap);
  } else if (jacobi_dsmem_bytes(q1, q2, C) <= avail) {
    if (q1 <= 4 * kJacobiRegs) jacobi_dsmem_impl<4>(descs, di, flops, q1cap, q2cap);
    else jacobi_dsmem_impl<8>(descs, di, flops, q1cap, q2cap);
  } else {
    jacobi_global_impl(descs, di, flops);
  }
}




cudaError_t launch_jacobi(const JacobiDesc* h, int n, JacobiDesc* d, int cluster, size_t smem_cap,
                          cudaStream_t s, int cluster_large) {
  if (n <= 0) return cudaSuccess;
  const int cluster_max = cluster;
  int q1cap = 0, q2cap = 0;
  for (int i = 0; i < n; ++i) {
    q1cap = max(q1cap, h[i].q1);
    q2cap = max(q2cap, h[i].q2);
  }
  q1cap = max(q1cap, 1);
  q2cap = max(q2cap, 1);
  // Cluster size for this launch: enough CTAs that each has about two warps of pair groups per
  // round (more CTAs only add barrier cost: a round is one dependent chain per pair), at most
  // the context's size, and enough that the columns fit in shared memory.
  // pairs per warp: lane groups of 4 or 8 (up to 32 for long columns alone on the GPU, where the
  // owner-computes form takes them)
  const bool alone = smem_cap >= kJacobiSmemMax;
  const int ppw = q1cap <= 4 * kJacobiRegs ? 8
                  : (q1cap <= 8 * kJacobiRegs || !alone ? 4 : (q1cap <= 16 * kJacobiRegs ? 2 : 1));
  const int pairs = (q2cap + 1) / 2;
  cluster = max(1, min(cluster, (pairs + 2 * ppw - 1) / (2 * ppw)));
  // a core whose columns do not fit the context's cluster in distributed shared memory grows
  // the cluster, up to the context's size for large problems and, for a factorization alone on
  // the GPU, at least to 8 CTAs (the portable limit), instead of falling back to the
  // global-memory form, which costs more than twice the FP64 instructions per rotation; small
  // actual cores still run on one CTA of it (the others exit).  While factorizations share the
  // SMs the larger clusters cost more than they save (measured on the batched n = 8192
  // workload: 54.7 against 62.9 factorizations/s).
  const size_t jcap = std::min(kJacobiSmemMax, smem_cap);
  const int jgrow = smem_cap >= kJacobiSmemMax ? std::min(8, qr_max_cluster()) : 0;
  const int jmax = std::max(std::max(cluster_max, cluster_large), jgrow);
  while (cluster < jmax && jacobi_dsmem_bytes(q1cap, q2cap, cluster) > jcap) ++cluster;
  const size_t smem = jacobi_dsmem_bytes(q1cap, q2cap, cluster);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster, n, 1);
  cfg.blockDim = dim3(QT, 1, 1);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // shared memory for the owner-computes form at the capacities, at most the per-CTA limit; the
  // kernel picks its form from the actual core size, which is usually far below the capacities
  const size_t smem2 = std::min(jacobi_owner_bytes(q1cap, q2cap, cluster), std::min(kJacobiSmemMax, smem_cap));
  if (q2cap <= kJacobiMaxCols) {
    cfg.dynamicSmemBytes = smem2;
    // cores of at most this many columns run on one CTA; more of them while other factorizations
    // share the SMs (throughput over latency)
    const int solo = smem_cap < kJacobiSmemMax ? 2 * kJacobiSoloCols : kJacobiSoloCols;
    // owner-computes (every pair formed on both owners) only for a factorization alone on the
    // GPU: with several in flight the FP64 issue rate, not the round's latency, is the limit
    if (cluster >= 8 && smem_cap >= kJacobiSmemMax)
      return cudaLaunchKernelEx(&cfg, jacobi_dsmem_kernel<true>, (const JacobiDesc*)d, q1cap, q2cap,
                                (int)smem2, solo);
    return cudaLaunchKernelEx(&cfg, jacobi_dsmem_kernel<false>, (const JacobiDesc*)d, q1cap, q2cap,
                              (int)smem2, solo);
  }
  return cudaLaunchKernelEx(&cfg, jacobi_cluster_kernel, (const JacobiDesc*)d);
}

}  // namespace hq

// ----------------------------------------------------------------- allocation-free dense QR
// Scratch of hodlr_dense_qr_noalloc: the launch descriptor, tau (kNoAllocMaxK) and the
// G = Y^T Y work area (kNoAllocMaxK^2), in one file-scope device array.  Every GPU that loads
// the library holds it (about 0.5 MiB) until the process exits.
namespace hq {
constexpr int kNoAllocMaxK = 256;
constexpr size_t kNoAllocDescDoubles = (sizeof(QRDesc) + 255) / 256 * 256 / sizeof(double);
constexpr size_t kNoAllocDoubles = kNoAllocDescDoubles + kNoAllocMaxK + (size_t)kNoAllocMaxK * kNoAllocMaxK;
constexpr int kNoAllocMaxDevices = 64;
cudaStream_t ctx_stream(hodlr_ctx* ctx);
int ctx_cluster(hodlr_ctx* ctx);
int ctx_device(hodlr_ctx* ctx);
}  // namespace hq

static __device__ __align__(256) double g_noalloc_scratch[hq::kNoAllocDoubles];

extern "C" int hodlr_dense_qr_noalloc(hodlr_ctx* ctx, int h, int w, double* A, int lda, double* T, int ldt) {
  using namespace hq;
  if (!ctx || !A || !T || h < 1 || w < 1 || w > 1024 || lda < h) return 1;  // HODLR_EINVAL
  const int k = h < w ? h : w;
  if (k > kNoAllocMaxK || ldt < k) return 1;                                // beyond the scratch size
  // the array, the stream and the caller's buffers all belong to the context's device
  const int dev = ctx_device(ctx);
  if (dev < 0 || dev >= kNoAllocMaxDevices) return 1;
  HQ_CUDA_OK(cudaSetDevice(dev));
  // once per device, with that device current: the device address of the scratch array.  The
  // table is shared by host threads; a lookup that two threads make at once stores the same
  // address twice.
  static std::atomic<double*> scratch_addr[kNoAllocMaxDevices] = {};
  double* base = scratch_addr[dev].load(std::memory_order_acquire);
  if (!base) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, __FILE__, __LINE__);
    base = static_cast<double*>(p);
    scratch_addr[dev].store(base, std::memory_order_release);
  }
  QRDesc q = {};
  q.A = A; q.lda = lda; q.h = h; q.w = w; q.href = -1; q.wref = -1;
  q.tau = base + kNoAllocDescDoubles;
  q.G = q.tau + kNoAllocMaxK;
  q.ldg = k;
  q.T = T; q.ldt = ldt; q.step = kStepNone; q.fmode = 0;
  cudaStream_t s = ctx_stream(ctx);
  QRDesc* dq = reinterpret_cast<QRDesc*>(base);
  // every entry of tau and G is written by the kernel before it is read: nothing to clear
  cudaError_t e = cudaMemcpyAsync(dq, &q, sizeof(QRDesc), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_qr(&q, 1, dq, ctx_cluster(ctx), (size_t)-1, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, __FILE__, __LINE__);
  return 0;
}
