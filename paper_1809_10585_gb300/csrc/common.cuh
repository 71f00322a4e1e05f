// Shared definitions of the hQR CUDA library (FP64, sm_103a).
//
// Data-dependent sizes.  Off-diagonal ranks are produced on the device by the truncation
// T_eps (Sec. 2.1.1) and never read back during a factorization.  Every descriptor therefore
// carries each size twice: a literal that is also the capacity used to size the grid, and a
// reference `*ref` into a device int table ("devints"); a reference >= 0 overrides the
// literal at run time.  Kernels clamp to the capacity.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

struct hodlr_ctx;

namespace hq {

constexpr int kMaxSweeps = 40;      // one-sided Jacobi sweep cap
constexpr int kMaxSegs = 12;        // segments of one column concatenation
constexpr int kMaxRowSrc = 24;      // ancestor row sources of one compressed leaf column

// Flop-counter slots (algorithmic FP64 flops per step of the hot path).
enum Step { kStepNorm = 0, kStepLeftOrth = 1, kStepLeafQR = 2, kStepS = 3, kStepTS = 4,
            kStepUpdate = 5, kStepT12 = 6, kStepNone = -1 };
// Per-kernel-kind algorithmic flops live after the step slots: flops[kKindSlot + kind],
// kinds 0 GEMM, 2 cluster QR, 3 cluster Jacobi.
constexpr int kKindSlot = 7;

__host__ __device__ inline int dimv(int lit, int ref, const int* di) {
  if (ref < 0) return lit;
  int v = di[ref];
  return v < 0 ? 0 : (v > lit ? lit : v);
}

// Output tile of the batched GEMM (rows x columns); the planner sizes the grid with it.
constexpr int kGemmBM = 64, kGemmBN = 32;

// C = alpha * op(mask(A)) * op(mask(B)) + beta * C.  Masks act on the stored matrices.
enum Mask { kMaskNone = 0, kMaskUpper = 1, kMaskUnitLower = 2, kMaskLower = 3 };
// flop accounting mode: 0 = 2mnk, 1 = mnk (one triangular factor), -1 = not counted
// Every descriptor names the rank table (`di`, the devints of its matrix) and, where the kernel
// counts algorithmic flops, the flop counters (`fl`) of its matrix, so that one launch may
// carry descriptors of several matrices.
struct GemmDesc {
  const int* di;
  double* fl;
  const double* A;
  const double* B;
  double* C;
  int lda, ldb, ldc;
  int m, n, k;
  int mref, nref, kref;
  int ta, tb;
  int mska, mskb;
  double alpha, beta;
  const double* alpha_ref;  // if set, alpha *= *alpha_ref
  int ksplit;               // >= 1
  double* part;             // ksplit * m * n partials when ksplit > 1
  int* tile_count;          // per-tile arrival counters when ksplit > 1 (zero between uses)
  int work0;                // first work item of this descriptor in the launch
  int tiles_m, tiles_n;     // grid of tiles (capacity)
  int step, fmode;
};

// Column concatenation  dst = [alpha_0 S_0 | alpha_1 S_1 | ...]  with run-time widths.
struct ConcatSeg {
  const double* src;
  int lds;
  int cols, colsref;
  double alpha;
};
struct ConcatDesc {
  int* di;
  double* dst;
  int ldd, rows;            // rows is a literal (block sizes are static)
  int cap;                  // column capacity of dst
  int nseg;
  ConcatSeg seg[kMaxSegs];
  int kout_ref;             // devints[kout_ref] = total width K, devints[kout_ref+1] = min(rows, K)
};

// Compressed leaf column (Sec. 4, Eq. (12)): panel = [leaf; B_R; C] with the B_R / C rows
// taken from right factors V21 of ancestor lower blocks (stored transposed).
struct PanelDesc {
  int* di;
  double* D;                // leaf block w x w, ld ldD
  int ldD, w;
  double* P;                // panel, ld ldP
  int ldP;
  int nsrc;
  double* src[kMaxRowSrc];  // V21 of the ancestor, already offset to this leaf's columns
  int lds[kMaxRowSrc];
  int rref[kMaxRowSrc];     // rank of each source (devints)
  int rcap[kMaxRowSrc];
  int href;                 // devints[href] = panel height
};

// Householder QR of one dense h x w matrix by a thread-block cluster (Alg. 1 semantics).
struct QRDesc {
  const int* di;
  double* fl;
  double* A;
  int lda;
  int h, w, href, wref;
  double* tau;              // min(h,w)
  double* T;                // min(h,w) x min(h,w) upper, ld ldt
  int ldt;
  double* G;                // scratch, ld ldg, >= min(h,w)^2
  int ldg;
  int step;                 // flop slot (kStepNone: not counted)
  int fmode;                // 0: QR + T (dense_qr_flops), 1: economy QR with Q formed
};

// One-sided Jacobi on the columns of M (q1 x q2), in place.
struct JacobiDesc {
  const int* di;
  double* fl;
  double* M;
  int ldm;
  int q1, q2, q1ref, q2ref;
  double* nrm;              // q2 squared column norms on exit
  int* rot;                 // kMaxSweeps counters (scratch)
  double thr;               // truncation threshold of the caller (thr_ref scales it)
  const double* thr_ref;
};

// Rank selection after Jacobi: keep columns with norm > thr, sorted by norm descending,
// normalized, into U (q1 x kcap, ld ldu).  Writes k to devints[kref].
struct SelectDesc {
  int* di;
  double* fl;
  const double* W;
  int ldw;
  const double* nrm;
  int q1, q2, q1ref, q2ref;
  double thr;
  const double* thr_ref;    // if set, thr *= *thr_ref
  double* U;
  int ldu;
  int kcap;
  int kref;
  int* status;              // set HODLR_ERANK (3) if more than kcap values exceed thr
  // algorithmic flop accounting of the whole truncation (the oracle's counts)
  int nL, nR, Kref;
  int step;
};

// Y(rows) = alpha * X(rows) with dynamic columns, optional zero padding of rows [r0, rows).
struct CopyDesc {
  const int* di;
  const double* src;
  int lds;
  double* dst;
  int ldd;
  int rows, rows_src;       // rows of dst written; rows_src (dynamic via ref) copied, rest zero
  int rows_src_ref;
  int cols, colsref;
  double alpha;
};

// Small element-wise operations, one descriptor per array, so that one launch may carry many:
//   kSmallFill  p[0..cnt) = v;   kSmallIFill  ip[0..cnt) = (int)v;
//   kSmallIdent p (ld, rows x cols) = [I; 0];
//   kSmallNorm  *out = ||p[0..cnt)||_2, and p /= *out when scale (a zero vector is kept);
//   kSmallTri   out (leading dimension cnt, rows x cols) = the unit lower trapezoidal part of
//               p (ld) when scale == 0 (ones on the diagonal), its upper part when scale == 1.
enum SmallKind { kSmallFill = 0, kSmallIFill = 1, kSmallIdent = 2, kSmallNorm = 3, kSmallTri = 4 };
struct SmallDesc {
  int kind;
  double* p;
  int* ip;
  double* out;
  long long cnt;
  int ld, rows, cols, scale;
  double v;
};

}  // namespace hq

#define HQ_CUDA_OK(call)                                           \
  do {                                                             \
    cudaError_t e__ = (call);                                      \
    if (e__ != cudaSuccess) return hq::cuda_fail(e__, __FILE__, __LINE__); \
  } while (0)

namespace hq {
int cuda_fail(cudaError_t e, const char* file, int line);

// Host launchers (kernels.cu / factor.cu).  All queue work on `s`.
cudaError_t launch_gemm(GemmDesc* h_descs, int n, GemmDesc* d_descs, cudaStream_t s);
cudaError_t launch_concat(const ConcatDesc* h, int n, ConcatDesc* d, cudaStream_t s);
cudaError_t launch_panel_gather(const PanelDesc* h, int n, PanelDesc* d, cudaStream_t s);
cudaError_t launch_panel_scatter(const PanelDesc* h, int n, PanelDesc* d, cudaStream_t s);
// The cluster kernels reserve shared memory for the capacities of their launch, at most
// `smem_cap` bytes (the per-CTA limit when larger), and pick their form from the actual sizes.
// kClusterSmemShared is the cap while several factorizations run concurrently: two CTAs per SM
// (their register use, ~126 per thread at 256 threads, allows no more), each with up to 18 KB
// of static shared memory, out of the SM's 228 KB.
constexpr size_t kClusterSmemShared = 92 * 1024;
// cluster_large (<= the device maximum): the cluster size for problems whose capacity does not
// fit the shared memory of `cluster` CTAs (0: no growth).
cudaError_t launch_qr(const QRDesc* h, int n, QRDesc* d, int cluster, size_t smem_cap, cudaStream_t s,
                      int cluster_large = 0);
cudaError_t launch_jacobi(const JacobiDesc* h, int n, JacobiDesc* d, int cluster, size_t smem_cap, cudaStream_t s,
                          int cluster_large = 0);
cudaError_t launch_select(const SelectDesc* h, int n, SelectDesc* d, cudaStream_t s);
cudaError_t launch_copy(const CopyDesc* h, int n, CopyDesc* d, cudaStream_t s);
// fills and identities (kinds 0-2) of one record; norms (kind 3) of one record
cudaError_t launch_small(const SmallDesc* h, int n, SmallDesc* d, cudaStream_t s);
cudaError_t launch_norms(const SmallDesc* h, int n, SmallDesc* d, cudaStream_t s);
cudaError_t launch_set_ints(int* devints, const int* idx_vals, int n, int* scratch, cudaStream_t s);
cudaError_t launch_fill(double* p, size_t n, double v, cudaStream_t s);
cudaError_t launch_gauss(double* p, size_t n, unsigned long long seed, cudaStream_t s);
cudaError_t launch_norm_scale(double* x, int n, double* out_norm, int mode, cudaStream_t s);
cudaError_t launch_set_diag_identity(double* p, int ld, int rows, int cols, cudaStream_t s);
cudaError_t launch_check_finite(const double* p, int ld, int rows, int cols, int* flag, cudaStream_t s);
cudaError_t launch_trsm_leaf(const double* R, int ldr, int w, double* B, int ldb, int nrhs, cudaStream_t s);
int qr_max_cluster();

}  // namespace hq
