// FP64 kernels of the hQR hot path that are not factorizations: a descriptor-driven batched
// GEMM (every HODLR-times-block product, low-rank product and WY application of Alg. 2),
// column concatenation for the truncation inputs, the gather/scatter of the compressed leaf
// column (Sec. 4, Eq. (12)), rank selection after the Jacobi SVD (Sec. 2.1.1, k_eps) and small
// utilities.  GB300 has about 2 FP64 FMA per clock per SM, so these kernels are FP64-issue
// bound; they are written to spread work over all 152 SMs rather than to stage operands.
#include <algorithm>
#include <cstdio>

#include "common.cuh"

namespace hq {

int cuda_fail(cudaError_t e, const char* file, int line) {
  fprintf(stderr, "hodlr_qr: CUDA error %s at %s:%d\n", cudaGetErrorString(e), file, line);
  return 6;  // HODLR_ECUDA
}

__device__ inline double ldcg(const double* p) { return __ldcg(p); }

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ----------------------------------------------------------------------------------- GEMM
// Tiles of BM x BN outputs, k in chunks of BK, GT threads.  Each thread owns a register
// micro-tile of MR x NR outputs (MR consecutive rows, NR consecutive columns).
constexpr int BM = kGemmBM, BN = kGemmBN, BK = 16, GT = 256, MR = 4, NR = 2;
constexpr int LDA_S = BM + 2, LDB_S = BN + 2;   // shared row strides: 16-byte aligned, few conflicts
static_assert(BM * BN == GT * MR * NR, "one micro-tile per thread covers the tile");

__device__ inline double masked(const double* M, int ld, int r, int c, int mask) {
  if (mask == kMaskNone) return M[r + (size_t)c * ld];
  if (mask == kMaskUpper) return r <= c ? M[r + (size_t)c * ld] : 0.0;
  if (mask == kMaskLower) return r >= c ? M[r + (size_t)c * ld] : 0.0;
  // unit lower
  if (r > c) return M[r + (size_t)c * ld];
  return r == c ? 1.0 : 0.0;
}

// One work item (an output tile and a k split of one descriptor).  Called by every thread of
// the CTA with the same item, so control flow and block barriers are uniform.
__device__ __forceinline__ void gemm_item(const GemmDesc* __restrict__ descs, int ndesc, int item,
                                          double (*As)[LDA_S], double (*Bs)[LDB_S], int& last) {
  // Locate the descriptor (work items are contiguous per descriptor, work0 strictly increasing):
  // each warp samples 32 first items at stride s = ceil(ndesc / 32) in one load and votes, then
  // scans the chosen stretch of s descriptors 32 at a time: two dependent loads instead of
  // log2(ndesc) of a binary search.
  const int lane = threadIdx.x & 31;
  const int stride = (ndesc + 31) >> 5;
  int lo;
  {
    const int idx = lane * stride;
    const bool le = idx < ndesc && __ldg(&descs[idx].work0) <= item;
    lo = (31 - __clz(__ballot_sync(0xffffffffu, le))) * stride;   // lane 0 always votes yes
  }
  if (stride > 1) {
    const int end = min(lo + stride, ndesc);
    for (int b = lo; b < end; b += 32) {
      const int idx = b + lane;
      const bool le = idx < end && __ldg(&descs[idx].work0) <= item;
      const unsigned m = __ballot_sync(0xffffffffu, le);
      lo = b + 31 - __clz(m);                         // bit 0 is set: descs[b].work0 <= item
      if (m != 0xffffffffu) break;
    }
  }
  const GemmDesc& d = descs[lo];
  const int* di = d.di;
  double* flops = d.fl;
  int local = item - d.work0;
  int tiles = d.tiles_m * d.tiles_n;
  int split = local / tiles;
  int t = local - split * tiles;
  int tm = t % d.tiles_m, tn = t / d.tiles_m;
  const int m = dimv(d.m, d.mref, di), n = dimv(d.n, d.nref, di), k = dimv(d.k, d.kref, di);
  if (local == 0 && threadIdx.x == 0 && flops) {
    double f = (double)m * n * k * (d.fmode == 1 ? 1.0 : 2.0);
    if (f > 0) {
      if (d.step >= 0 && d.fmode >= 0) atomicAdd(&flops[d.step], f);
      atomicAdd(&flops[kKindSlot + 0], f);
    }
  }
  const int row0 = tm * BM, col0 = tn * BN;
  const bool to_part = d.ksplit > 1;
  if (row0 >= m || col0 >= n) return;   // nothing to compute (partial slots beyond k unused)
  int kchunk = (k + d.ksplit - 1) / d.ksplit;
  kchunk = (kchunk + BK - 1) / BK * BK;
  int k0 = split * kchunk;
  int k1 = min(k, k0 + kchunk);
  {
    // a triangular operand is zero outside a band of k set by the tile's rows (A) or columns
    // (B): products there are skipped (they would add exact zeros)
    const int ma0 = min(BM, m - row0), na0 = min(BN, n - col0);
    const bool lowa = d.mska == kMaskLower || d.mska == kMaskUnitLower;
    const bool lowb = d.mskb == kMaskLower || d.mskb == kMaskUnitLower;
    if ((d.mska == kMaskUpper && !d.ta) || (lowa && d.ta)) k0 = max(k0, row0);        // l >= i
    if ((d.mska == kMaskUpper && d.ta) || (lowa && !d.ta)) k1 = min(k1, row0 + ma0);   // l <= i
    if ((d.mskb == kMaskUpper && d.tb) || (lowb && !d.tb)) k0 = max(k0, col0);        // l >= j
    if ((d.mskb == kMaskUpper && !d.tb) || (lowb && d.tb)) k1 = min(k1, col0 + na0);   // l <= j
  }

  // The outputs of this tile that exist (ma x na) are known only on the device; most products
  // here multiply by a block of a few columns, so most tiles are sparse.  GB300 retires one
  // 32-lane FP64 FMA instruction per 64 cycles on each of an SM's four sub-partitions, so FP64
  // work must reach all of them, i.e. all warps of the CTA:
  //  * dense form (ma x na <= 4 GT): the outputs are dealt to the threads in column-major
  //    order, one per thread per pass (at most four passes), two FMA chains per output; only
  //    the last warp of a pass carries idle lanes;
  //  * micro-tile form (larger tiles): each thread owns MR x NR outputs (MR consecutive rows,
  //    NR consecutive columns), eight independent chains, six shared loads per eight FMAs.
  // A warp none of whose outputs exist issues no FMA.
  const int ma = min(BM, m - row0), na = min(BN, n - col0);
  const int nout = ma * na;
  const bool dense = nout <= 4 * GT;                        // uniform over the CTA
  const int tid = threadIdx.x;
  const int wbase = tid & ~31;
  const int mrow = (ma + MR - 1) / MR, mcol = (na + NR - 1) / NR;
  const int nmic = mrow * mcol;
  // micro-tile form: the thread's micro-tile; dense form: its output of each pass u (packed)
  int r0 = 0, c0 = 0;
  int oij[4];
  if (dense) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int o = min(tid + GT * u, nout - 1);
      const int oj = o / ma;
      oij[u] = ((o - oj * ma) << 8) | oj;                   // row << 8 | column (both < 256)
    }
  } else {
    const int mi = tid < nmic ? tid % mrow : 0, nj = tid < nmic ? tid / mrow : 0;
    r0 = mi * MR;
    c0 = nj * NR;
  }
  double acc[MR][NR];
#pragma unroll
  for (int u = 0; u < MR; ++u)
#pragma unroll
    for (int v = 0; v < NR; ++v) acc[u][v] = 0.0;
  // Operand tiles pass through registers: the loads of chunk kk + BK are in flight while chunk
  // kk is multiplied.  Element e = tid + GT p of each tile is mapped so that consecutive
  // threads read consecutive addresses of the stored (possibly transposed) operand.
  constexpr int PA = BM * BK / GT, PB = BN * BK / GT;
  double pa[PA], pb[PB];
  auto fetch = [&](int kk) {
    const int kl = min(BK, k1 - kk);
#pragma unroll
    for (int p = 0; p < PA; ++p) {
      const int e = tid + GT * p;
      const int i = d.ta ? e / BK : e % BM, l = d.ta ? e % BK : e / BM;
      double v = 0.0;
      if (i < ma && l < kl)
        v = d.ta ? masked(d.A, d.lda, kk + l, row0 + i, d.mska) : masked(d.A, d.lda, row0 + i, kk + l, d.mska);
      pa[p] = v;
    }
#pragma unroll
    for (int p = 0; p < PB; ++p) {
      const int e = tid + GT * p;
      const int j = d.tb ? e % BN : e / BK, lb = d.tb ? e / BN : e % BK;
      double w = 0.0;
      if (j < na && lb < kl)
        w = d.tb ? masked(d.B, d.ldb, col0 + j, kk + lb, d.mskb) : masked(d.B, d.ldb, kk + lb, col0 + j, d.mskb);
      pb[p] = w;
    }
  };
  fetch(k0);
  for (int kk = k0; kk < k1; kk += BK) {
    const int kl = min(BK, k1 - kk);
#pragma unroll
    for (int p = 0; p < PA; ++p) {
      const int e = tid + GT * p;
      const int i = d.ta ? e / BK : e % BM, l = d.ta ? e % BK : e / BM;
      As[l][i] = pa[p];
    }
#pragma unroll
    for (int p = 0; p < PB; ++p) {
      const int e = tid + GT * p;
      const int j = d.tb ? e % BN : e / BK, lb = d.tb ? e / BN : e % BK;
      Bs[lb][j] = pb[p];
    }
    __syncthreads();
    if (kk + BK < k1) fetch(kk + BK);
    if (dense) {
      // dense form: acc[u][0] / acc[u][1] are the even / odd k chains of pass u's output
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (wbase + GT * u < nout) {                          // warp-uniform
          const int i = oij[u] >> 8, j = oij[u] & 255;
          int l = 0;
          for (; l + 1 < kl; l += 2) {
            acc[u][0] = fma(As[l][i], Bs[l][j], acc[u][0]);
            acc[u][1] = fma(As[l + 1][i], Bs[l + 1][j], acc[u][1]);
          }
          if (l < kl) acc[u][0] = fma(As[l][i], Bs[l][j], acc[u][0]);
        }
      }
    } else if (wbase < nmic) {
      // rows / columns beyond ma / na hold zeros: a partial micro-tile computes zeros there
#pragma unroll 8
      for (int l = 0; l < kl; ++l) {
        const double2 a01 = *reinterpret_cast<const double2*>(&As[l][r0]);
        const double2 a23 = *reinterpret_cast<const double2*>(&As[l][r0 + 2]);
        const double2 b01 = *reinterpret_cast<const double2*>(&Bs[l][c0]);
        acc[0][0] = fma(a01.x, b01.x, acc[0][0]);
        acc[1][0] = fma(a01.y, b01.x, acc[1][0]);
        acc[2][0] = fma(a23.x, b01.x, acc[2][0]);
        acc[3][0] = fma(a23.y, b01.x, acc[3][0]);
        acc[0][1] = fma(a01.x, b01.y, acc[0][1]);
        acc[1][1] = fma(a01.y, b01.y, acc[1][1]);
        acc[2][1] = fma(a23.x, b01.y, acc[2][1]);
        acc[3][1] = fma(a23.y, b01.y, acc[3][1]);
      }
    }
    __syncthreads();
  }
  double alpha = d.alpha;
  if (d.alpha_ref) alpha *= *d.alpha_ref;
  auto emit = [&](int r, int c, double v) {
    const int gi = row0 + r, gj = col0 + c;
    if (to_part) {
      d.part[(size_t)split * d.m * d.n + gi + (size_t)gj * d.m] = v;
    } else {
      double* cp = d.C + gi + (size_t)gj * d.ldc;
      double val = alpha * v;
      if (d.beta != 0.0) val = fma(d.beta, *cp, val);
      *cp = val;
    }
  };
  if (dense) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (tid + GT * u < nout) emit(oij[u] >> 8, oij[u] & 255, acc[u][0] + acc[u][1]);
  } else if (tid < nmic) {
#pragma unroll
    for (int v = 0; v < NR; ++v)
#pragma unroll
      for (int u = 0; u < MR; ++u)
        if (r0 + u < ma && c0 + v < na) emit(r0 + u, c0 + v, acc[u][v]);
  }
  if (!to_part || d.tile_count == nullptr) return;
  // split-K: the last split to finish this tile sums the partials in split order (the result
  // does not depend on arrival order) and resets the counter for the next use
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    int* cnt = d.tile_count + t;
    last = (atomicAdd(cnt, 1) == d.ksplit - 1);
    if (last) *cnt = 0;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  int nsp = 0;
  for (int sp = 0; sp < d.ksplit; ++sp)
    if (sp * kchunk < k) nsp = sp + 1;
  for (int o = tid; o < ma * na; o += GT) {
    const int gi = row0 + o % ma, gj = col0 + o / ma;
    double sacc = 0.0;
    for (int sp = 0; sp < nsp; ++sp) sacc += __ldcg(&d.part[(size_t)sp * d.m * d.n + gi + (size_t)gj * d.m]);
    double* c = d.C + gi + (size_t)gj * d.ldc;
    double val = alpha * sacc;
    if (d.beta != 0.0) val = fma(d.beta, *c, val);
    *c = val;
  }
}

// Persistent over the launch's work items: CTA b takes items b, b + grid, b + 2 grid, ...
// (a static queue: which CTA computes an item never changes its result).  Most products here
// have capacity tiles that are empty at run time (their rank is below the capacity); a CTA
// skips those in a few instructions instead of the launch paying a CTA for each.
__global__ void __launch_bounds__(GT, 3) gemm_kernel(const GemmDesc* __restrict__ descs, int ndesc, int total) {
  __shared__ __align__(16) double As[BK][LDA_S];
  __shared__ __align__(16) double Bs[BK][LDB_S];
  __shared__ int last;
  for (int item = blockIdx.x; item < total; item += gridDim.x) gemm_item(descs, ndesc, item, As, Bs, last);
}

// Sum split-K partials: C = alpha * sum_s part_s + beta * C.  One block per 256 outputs.
__global__ void gemm_reduce_kernel(const GemmDesc* __restrict__ descs, const int* __restrict__ rd, int nred) {
  int item = blockIdx.x;
  // rd: pairs (desc index, first block) sorted by first block
  int lo = 0, hi = nred - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (rd[2 * mid + 1] <= item) lo = mid; else hi = mid - 1;
  }
  const GemmDesc& d = descs[rd[2 * lo]];
  const int* di = d.di;
  int e = (item - rd[2 * lo + 1]) * blockDim.x + threadIdx.x;
  const int m = dimv(d.m, d.mref, di), n = dimv(d.n, d.nref, di), k = dimv(d.k, d.kref, di);
  if (e >= d.m * d.n) return;
  int i = e % d.m, j = e / d.m;
  if (i >= m || j >= n) return;
  int kchunk = (k + d.ksplit - 1) / d.ksplit;
  kchunk = (kchunk + BK - 1) / BK * BK;
  double s = 0.0;
  for (int sp = 0; sp < d.ksplit; ++sp) {
    if (sp * kchunk >= k) break;   // splits beyond k never wrote their slot
    s += d.part[(size_t)sp * d.m * d.n + i + (size_t)j * d.m];
  }
  double alpha = d.alpha;
  if (d.alpha_ref) alpha *= *d.alpha_ref;
  double* c = d.C + i + (size_t)j * d.ldc;
  double v = alpha * s;
  if (d.beta != 0.0) v = fma(d.beta, *c, v);
  *c = v;
}

// SM count of the device, queried once per process (thread-safe static initialisation).
static int device_sms() {
  static const int sms = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        v <= 0)
      v = 152;
    cudaGetLastError();
    return v;
  }();
  return sms;
}

cudaError_t launch_gemm(GemmDesc* h, int n, GemmDesc* d, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int total = h[n - 1].work0 + h[n - 1].tiles_m * h[n - 1].tiles_n * h[n - 1].ksplit;
  if (total <= 0) return cudaSuccess;
  const int grid = std::min(total, 6 * device_sms());    // two waves of 3 resident CTAs per SM
  gemm_kernel<<<grid, GT, 0, s>>>(d, n, total);
  return cudaGetLastError();
}

// Reduction launch helper: `rd` is a device array of (desc index, first block) pairs,
// `nblocks` the total number of blocks.
cudaError_t launch_gemm_reduce(const GemmDesc* d, const int* rd, int nred, int nblocks, cudaStream_t s) {
  if (nred <= 0 || nblocks <= 0) return cudaSuccess;
  gemm_reduce_kernel<<<nblocks, 256, 0, s>>>(d, rd, nred);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------- concat
__global__ void concat_kernel(const ConcatDesc* __restrict__ descs) {
  const ConcatDesc& d = descs[blockIdx.y];
  int* di = d.di;
  int off = 0;
  for (int s = 0; s < d.nseg; ++s) {
    const ConcatSeg& g = d.seg[s];
    int c = dimv(g.cols, g.colsref, di);
    if (off + c > d.cap) c = d.cap - off;
    const int rows = d.rows;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * c; e += gridDim.x * blockDim.x) {
      int i = e % rows, j = e / rows;
      d.dst[i + (size_t)(off + j) * d.ldd] = g.alpha * g.src[i + (size_t)j * g.lds];
    }
    off += c;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && d.kout_ref >= 0) {
    di[d.kout_ref] = off;
    di[d.kout_ref + 1] = off < d.rows ? off : d.rows;
  }
}

cudaError_t launch_concat(const ConcatDesc* h, int n, ConcatDesc* d, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int maxrows = 0;
  for (int i = 0; i < n; ++i) maxrows = max(maxrows, h[i].rows);
  int gx = min(64, max(1, maxrows * 8 / 256));
  concat_kernel<<<dim3(gx, n), 256, 0, s>>>(d);
  return cudaGetLastError();
}

// -------------------------------------------------------------------- leaf panel gather
__global__ void panel_gather_kernel(const PanelDesc* __restrict__ descs) {
  const PanelDesc& d = descs[blockIdx.y];
  int* di = d.di;
  const int w = d.w;
  // leaf block
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < w * w; e += gridDim.x * blockDim.x) {
    int i = e % w, j = e / w;
    d.P[i + (size_t)j * d.ldP] = d.D[i + (size_t)j * d.ldD];
  }
  int off = w;
  for (int s = 0; s < d.nsrc; ++s) {
    int r = dimv(d.rcap[s], d.rref[s], di);
    // rows off..off+r-1 of the panel are row i of B_R = column i of V21 (transposed)
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * w; e += gridDim.x * blockDim.x) {
      int c = e % w, i = e / w;
      d.P[(off + i) + (size_t)c * d.ldP] = d.src[s][c + (size_t)i * d.lds[s]];
    }
    off += r;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) di[d.href] = off;
}

__global__ void panel_scatter_kernel(const PanelDesc* __restrict__ descs) {
  const PanelDesc& d = descs[blockIdx.y];
  const int* di = d.di;
  const int w = d.w;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < w * w; e += gridDim.x * blockDim.x) {
    int i = e % w, j = e / w;
    d.D[i + (size_t)j * d.ldD] = d.P[i + (size_t)j * d.ldP];
  }
  int off = w;
  for (int s = 0; s < d.nsrc; ++s) {
    int r = dimv(d.rcap[s], d.rref[s], di);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * w; e += gridDim.x * blockDim.x) {
      int c = e % w, i = e / w;
      d.src[s][c + (size_t)i * d.lds[s]] = d.P[(off + i) + (size_t)c * d.ldP];
    }
    off += r;
  }
}

cudaError_t launch_panel_gather(const PanelDesc* h, int n, PanelDesc* d, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int gx = min(64, max(1, h[0].w * h[0].w / 1024));
  panel_gather_kernel<<<dim3(gx, n), 256, 0, s>>>(d);
  return cudaGetLastError();
}
cudaError_t launch_panel_scatter(const PanelDesc* h, int n, PanelDesc* d, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int gx = min(64, max(1, h[0].w * h[0].w / 1024));
  panel_scatter_kernel<<<dim3(gx, n), 256, 0, s>>>(d);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------- rank selection
// One block per truncation problem.  k_eps = #{sigma_i > thr} (Sec. 2.1.1); the kept columns
// of W = M J are normalized to the left singular vectors and sorted by sigma descending.
__global__ void select_kernel(const SelectDesc* __restrict__ descs) {
  const SelectDesc& d = descs[blockIdx.x];
  int* di = d.di;
  double* flops = d.fl;
  const int q1 = dimv(d.q1, d.q1ref, di), q2 = dimv(d.q2, d.q2ref, di);
  double thr = d.thr;
  if (d.thr_ref) thr *= *d.thr_ref;
  extern __shared__ int sh[];
  int* order = sh;           // q2 entries: output slot of column j, or -1
  __shared__ int kcount;
  __shared__ unsigned long long nmax_bits;
  if (threadIdx.x == 0) {
    kcount = 0;
    nmax_bits = 0ull;
  }
  __syncthreads();
  // largest squared column norm (non-negative doubles order like their bit patterns)
  for (int j = threadIdx.x; j < q2; j += blockDim.x)
    atomicMax(&nmax_bits, (unsigned long long)__double_as_longlong(fmax(d.nrm[j], 0.0)));
  __syncthreads();
  // Columns below 4.4e-16 sqrt(q1) sigma_1 are numerically zero: their directions are rounding
  // noise (a rank-deficient core drives them even to denormal size), so they are dropped even
  // when thr is smaller; this changes the block by at most that much per column.
  const double floor_ = 4.4e-16 * sqrt((double)max(q1, 1)) * sqrt(__longlong_as_double((long long)nmax_bits));
  const double keep = fmax(thr, floor_);
  for (int j = threadIdx.x; j < q2; j += blockDim.x) {
    double nj = d.nrm[j];
    int slot = -1;
    if (sqrt(nj) > keep) {
      int rank = 0;
      for (int l = 0; l < q2; ++l) {
        double nl = d.nrm[l];
        if (sqrt(nl) > keep && (nl > nj || (nl == nj && l < j))) ++rank;
      }
      slot = rank;
      atomicAdd(&kcount, 1);
    }
    order[j] = slot;
  }
  __syncthreads();
  int k = kcount;
  if (k > d.kcap) {
    if (threadIdx.x == 0 && d.status) atomicMax(d.status, 3);
    k = d.kcap;
  }
  for (int j = 0; j < q2; ++j) {
    int slot = order[j];
    if (slot < 0 || slot >= k) continue;
    double inv = 1.0 / sqrt(d.nrm[j]);
    for (int i = threadIdx.x; i < q1; i += blockDim.x)
      d.U[i + (size_t)slot * d.ldu] = d.W[i + (size_t)j * d.ldw] * inv;
  }
  if (threadIdx.x == 0) {
    di[d.kref] = k;
    if (flops && d.step >= 0) {
      // the oracle's count of one T_eps: two economy QRs with Q formed, the core product,
      // an R-SVD of the q1 x q2 core and the two reconstructions
      int K = d.Kref >= 0 ? di[d.Kref] : 0;
      double f = 0;
      if (K > 0 && d.nL > 0 && d.nR > 0) {
        double a = min(d.nL, K), b = min(d.nR, K);
        f += 4.0 * d.nL * K * a - 4.0 * a * a * a / 3.0;
        f += 4.0 * d.nR * K * b - 4.0 * b * b * b / 3.0;
        f += 2.0 * a * K * b;
        double p = max(a, b), q = min(a, b);
        f += 4.0 * p * p * q + 8.0 * p * q * q + 9.0 * q * q * q;
        f += 2.0 * d.nL * a * k + 2.0 * d.nR * b * k;
      }
      atomicAdd(&flops[d.step], f);
    }
  }
}

cudaError_t launch_select(const SelectDesc* h, int n, SelectDesc* d, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int maxq2 = 0;
  for (int i = 0; i < n; ++i) maxq2 = max(maxq2, h[i].q2);
  select_kernel<<<n, 256, sizeof(int) * (maxq2 + 1), s>>>(d);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------------- copy
__global__ void copy_kernel(const CopyDesc* __restrict__ descs) {
  const CopyDesc& d = descs[blockIdx.y];
  const int* di = d.di;
  int cols = dimv(d.cols, d.colsref, di);
  int rs = dimv(d.rows_src, d.rows_src_ref, di);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)d.rows * cols;
       e += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(e % d.rows), j = (int)(e / d.rows);
    double v = (i < rs && d.src) ? d.alpha * d.src[i + (size_t)j * d.lds] : 0.0;
    d.dst[i + (size_t)j * d.ldd] = v;
  }
}

cudaError_t launch_copy(const CopyDesc* h, int n, CopyDesc* d, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int maxe = 0;
  for (int i = 0; i < n; ++i) maxe = max(maxe, h[i].rows * h[i].cols);
  int gx = min(128, max(1, maxe / 1024));
  copy_kernel<<<dim3(gx, n), 256, 0, s>>>(d);
  return cudaGetLastError();
}

// ------------------------------------------------------------- small descriptor operations
__global__ void small_kernel(const SmallDesc* __restrict__ descs) {
  const SmallDesc& d = descs[blockIdx.y];
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (d.kind == kSmallFill) {
    for (long long i = t0; i < d.cnt; i += stride) d.p[i] = d.v;
  } else if (d.kind == kSmallIFill) {
    const int iv = (int)d.v;
    for (long long i = t0; i < d.cnt; i += stride) d.ip[i] = iv;
  } else if (d.kind == kSmallIdent) {
    const long long tot = (long long)d.rows * d.cols;
    for (long long e = t0; e < tot; e += stride) {
      const int i = (int)(e % d.rows), j = (int)(e / d.rows);
      d.p[i + (size_t)j * d.ld] = (i == j) ? 1.0 : 0.0;
    }
  } else if (d.kind == kSmallTri) {
    const long long tot = (long long)d.rows * d.cols;
    for (long long e = t0; e < tot; e += stride) {
      const int i = (int)(e % d.rows), j = (int)(e / d.rows);
      const double a = d.p[i + (size_t)j * d.ld];
      d.out[i + (size_t)j * d.cnt] = d.scale ? (i <= j ? a : 0.0) : (i > j ? a : (i == j ? 1.0 : 0.0));
    }
  }
}

cudaError_t launch_small(const SmallDesc* h, int n, SmallDesc* d, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long mx = 1;
  for (int i = 0; i < n; ++i)
    mx = std::max(mx, (h[i].kind == kSmallIdent || h[i].kind == kSmallTri) ? (long long)h[i].rows * h[i].cols
                                                                               : h[i].cnt);
  const int gx = (int)std::min<long long>(256, std::max<long long>(1, mx / 1024));
  small_kernel<<<dim3(gx, n), 256, 0, s>>>(d);
  return cudaGetLastError();
}

// ||x||_2 of one vector per block (blockIdx.x = descriptor).
__global__ void norms_kernel(const SmallDesc* __restrict__ descs) {
  const SmallDesc& d = descs[blockIdx.x];
  __shared__ double red[32];
  double s = 0.0;
  for (long long i = threadIdx.x; i < d.cnt; i += blockDim.x) s = fma(d.p[i], d.p[i], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) red[0] = sqrt(v);
  }
  __syncthreads();
  const double nrm = red[0];
  if (threadIdx.x == 0) *d.out = nrm;
  if (d.scale && nrm > 0.0) {
    const double inv = 1.0 / nrm;
    for (long long i = threadIdx.x; i < d.cnt; i += blockDim.x) d.p[i] *= inv;
  }
}

cudaError_t launch_norms(const SmallDesc* h, int n, SmallDesc* d, cudaStream_t s) {
  (void)h;
  if (n <= 0) return cudaSuccess;
  norms_kernel<<<n, 1024, 0, s>>>(d);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------- utilities
__global__ void fill_kernel(double* p, size_t n, double v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    p[i] = v;
}
cudaError_t launch_fill(double* p, size_t n, double v, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  size_t gb = (n + 255) / 256;
  int g = (int)(gb < 1024 ? gb : 1024);
  fill_kernel<<<g, 256, 0, s>>>(p, n, v);
  return cudaGetLastError();
}

// Standard normal samples for a randomized range finder.  Element i of stream `seed` hashes the
// counter seed * 2^32 + i with SplitMix64 (Steele, Lea and Flood, OOPSLA 2014); two 24-bit
// uniforms of the hash give one normal by the Box-Muller transform, evaluated in FP32 (a sketch
// needs independent Gaussian-like entries, not FP64 accuracy).
__device__ inline unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__global__ void gauss_kernel(double* p, size_t n, unsigned long long seed) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const unsigned long long z = splitmix64((seed << 32) + i);
    const float u1 = ((float)(z >> 40) + 1.0f) * 0x1p-24f;              // (0, 1]
    const float u2 = (float)((z >> 16) & 0xFFFFFFull) * 0x1p-24f;        // [0, 1)
    p[i] = (double)(sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2));
  }
}
cudaError_t launch_gauss(double* p, size_t n, unsigned long long seed, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  size_t gb = (n + 255) / 256;
  int g = (int)(gb < 2048 ? gb : 2048);
  gauss_kernel<<<g, 256, 0, s>>>(p, n, seed);
  return cudaGetLastError();
}

__global__ void set_diag_identity_kernel(double* p, int ld, int rows, int cols) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * cols; e += gridDim.x * blockDim.x) {
    int i = e % rows, j = e / rows;
    p[i + (size_t)j * ld] = (i == j) ? 1.0 : 0.0;
  }
}
cudaError_t launch_set_diag_identity(double* p, int ld, int rows, int cols, cudaStream_t s) {
  int g = min(256, max(1, rows * cols / 256));
  set_diag_identity_kernel<<<g, 256, 0, s>>>(p, ld, rows, cols);
  return cudaGetLastError();
}

// ||x||_2 of an n-vector (one block).  mode 0: x <- x / ||x|| and out = ||x||;
// mode 1: out = ||x|| only.  A zero vector is left unchanged and out = 0.
__global__ void norm_scale_kernel(double* x, int n, double* out, int mode) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s = fma(x[i], x[i], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) red[0] = sqrt(v);
  }
  __syncthreads();
  double nrm = red[0];
  if (threadIdx.x == 0) *out = nrm;
  if (mode == 0 && nrm > 0.0) {
    double inv = 1.0 / nrm;
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] *= inv;
  }
}
cudaError_t launch_norm_scale(double* x, int n, double* out, int mode, cudaStream_t s) {
  norm_scale_kernel<<<1, 1024, 0, s>>>(x, n, out, mode);
  return cudaGetLastError();
}

__global__ void check_finite_kernel(const double* p, int ld, int rows, int cols, int* flag) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * cols; e += gridDim.x * blockDim.x) {
    int i = e % rows, j = e / rows;
    double v = p[i + (size_t)j * ld];
    if (!isfinite(v)) { atomicExch(flag, 1); return; }
  }
}
cudaError_t launch_check_finite(const double* p, int ld, int rows, int cols, int* flag, cudaStream_t s) {
  int g = min(256, max(1, rows * cols / 256));
  check_finite_kernel<<<g, 256, 0, s>>>(p, ld, rows, cols, flag);
  return cudaGetLastError();
}

// Dense upper-triangular back-substitution R x = b at one leaf, one warp per right-hand side.
__global__ void trsm_leaf_kernel(const double* __restrict__ R, int ldr, int w, double* B, int ldb, int nrhs) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= nrhs) return;
  double* b = B + (size_t)warp * ldb;
  for (int i = w - 1; i >= 0; --i) {
    double xi = 0.0;
    if (lane == 0) xi = b[i] / R[i + (size_t)i * ldr];
    xi = __shfl_sync(0xffffffffu, xi, 0);
    __syncwarp();
    if (lane == 0) b[i] = xi;
    for (int r = lane; r < i; r += 32) b[r] = fma(-R[r + (size_t)i * ldr], xi, b[r]);
    __syncwarp();
  }
}
cudaError_t launch_trsm_leaf(const double* R, int ldr, int w, double* B, int ldb, int nrhs, cudaStream_t s) {
  int threads = 128;
  int blocks = (nrhs * 32 + threads - 1) / threads;
  trsm_leaf_kernel<<<blocks, threads, 0, s>>>(R, ldr, w, B, ldb, nrhs);
  return cudaGetLastError();
}

}  // namespace hq
