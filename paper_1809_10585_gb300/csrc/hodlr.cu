// Host side of the hQR library: the device-resident HODLR container, the recursion
// scheduler of Alg. 2, apply/solve, and the C ABI declared in include/hodlr_qr.h.
//
// Scheduling model.  The recursion of Alg. 2 depends only on the cluster tree, never on the
// ranks, so a factorization is planned once per matrix: the planner walks the recursion and
// emits a flat list of kernel launches whose descriptors (pointers, capacities and
// references to ranks kept in device memory) are uploaded once.  Running a factorization
// replays that list on one stream, and hodlr_qr_graph captures it as a single CUDA graph.
// Ranks produced by T_eps stay on the device; kernels read them and size nothing on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <unordered_map>
#include <vector>

#include "../../include/hodlr_qr.h"
#include "common.cuh"

using namespace hq;

namespace hq {
cudaStream_t ctx_stream(hodlr_ctx* ctx);
int ctx_cluster(hodlr_ctx* ctx);
int ctx_device(hodlr_ctx* ctx);
void* ctx_alloc(hodlr_ctx* ctx, size_t bytes);
void ctx_free(hodlr_ctx* ctx, void* p, size_t bytes);
cudaError_t launch_gemm_reduce(const GemmDesc* d, const int* rd, int nred, int nblocks, cudaStream_t s);
}

// ------------------------------------------------------------------------------- objects
// Device bytes held through one context (its matrices with their plans, arenas and snapshots),
// against an optional limit set by the caller.  Matrices keep the account alive, so freeing a
// matrix after its context is destroyed stays correct.
// A device memory pool reserved once (one cudaMalloc) and carved up on the host: first fit
// over a free list ordered by offset, 256-byte granules, neighbours merged on release.  Taking
// and returning memory makes no CUDA call, so it never synchronizes the device.
struct DevPool {
  char* base = nullptr;
  size_t size = 0;
  std::map<size_t, size_t> free_;               // offset -> bytes
  std::map<size_t, size_t> used_;               // offset -> bytes
  std::mutex mu;
  void* take(size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    std::lock_guard<std::mutex> g(mu);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, rest = it->second - bytes;
      free_.erase(it);
      if (rest) free_[off + bytes] = rest;
      used_[off] = bytes;
      return base + off;
    }
    return nullptr;
  }
  void give(void* p) {
    std::lock_guard<std::mutex> g(mu);
    auto u = used_.find((size_t)((char*)p - base));
    if (u == used_.end()) return;
    size_t off = u->first, bytes = u->second;
    used_.erase(u);
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + bytes == next->first) {
      bytes += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }
  bool owns(void* p) const { return base && (char*)p >= base && (char*)p < base + size; }
};

struct MemAcct {
  std::atomic<long long> used{0};
  std::atomic<long long> limit{0};   // 0: no limit
  std::shared_ptr<DevPool> pool;     // set: every allocation of the account comes from it
  ~MemAcct() {
    if (pool && pool->base) cudaFree(pool->base);
  }
};

struct BatchGroup;

struct hodlr_ctx {
  std::shared_ptr<MemAcct> mem = std::make_shared<MemAcct>();
  int dev = 0;
  cudaStream_t own = nullptr;
  cudaStream_t s = nullptr;
  cudaStream_t side = nullptr;   // second stream for work off the critical path
  int cluster = 8;
  int cluster_large = 0;         // cluster size for problems that do not fit `cluster` (0: none)
  // stream pairs of batched factorizations (one pair per matrix of a batch)
  std::vector<std::pair<cudaStream_t, cudaStream_t>> pool;
  // CUDA graph of the last batched factorization captured with hodlr_qr_batched_graph
  cudaGraphExec_t bgraph = nullptr;
  std::vector<hodlr_mat*> bmats;
  double btol = -1, banorm = -2;
  int bcluster = 0;
  int concurrency = 1;           // factorizations in flight, as set by the caller
  int concurrent = 1;            // factorizations in flight on the pool's streams (batch size)
  int batch_group = 0;           // most matrices per merged launch sequence (0: no limit)
  // merged plans of cross-matrix batches (one per group of matrices with the same structure),
  // their device descriptor blobs owned by `batch_owner` (charged to this context's account)
  std::vector<BatchGroup*> groups;
  hodlr_mat* batch_owner = nullptr;
  int bconc = 0;
  int bgroup = -1;
};

// Shared memory a cluster kernel may reserve per CTA: the per-CTA limit for one factorization at
// a time; with several in flight, a cap that lets CTAs of other factorizations share the SM.
static size_t smem_cap(const hodlr_ctx* ctx) {
  return std::max(ctx->concurrent, ctx->concurrency) > 1 ? kClusterSmemShared : (size_t)-1;
}

enum RecType { R_GEMM, R_REDUCE, R_CONCAT, R_GATHER, R_SCATTER, R_QR, R_JACOBI, R_SELECT, R_COPY,
               R_SMALL, R_NORMS, R_TRSM, R_EVREC, R_EVWAIT, R_GAUSS };

struct Rec {
  int type;
  int stream;     // 0: main stream, 1: side stream
  int n;          // descriptors
  size_t off;     // byte offset of the descriptors in the blob
  int extra0, extra1;
  double* p0;
  int* ip;
  double v;
  size_t cnt;
  int i0, i1, i2, i3;
};

struct Plan {
  std::vector<Rec> recs;
  int nevents = 0;
  std::vector<cudaEvent_t> events;
  std::vector<char> blob;
  char* dblob = nullptr;
  size_t dblob_bytes = 0;
  int* counters = nullptr;       // split-K tile counters of this plan (zero between uses)
  size_t counters_n = 0;
  // host copies of descriptors needed for launch-time grid sizing live inside blob
};

// A group of matrices of one structure and the merged plan that factors them together.
struct BatchGroup {
  std::vector<hodlr_mat*> mats;
  std::vector<long> versions;    // plan_version of each member when the plan was merged
  Plan plan;
};

struct View {
  // HODLR storage view: leaves and per-node factor pointers (device), rank refs
  double* D;
  int ldl;
  const std::vector<double*>* U12;
  const std::vector<double*>* V12;
  const std::vector<double*>* U21;
  const std::vector<double*>* V21;
  int r12_base, r21_base;  // -1 = block absent
};

struct hodlr_mat {
  std::shared_ptr<MemAcct> mem;                 // account of the context that built it
  std::unordered_map<void*, size_t> allocs;     // live device allocations and their sizes
  long long held = 0;                           // their total
  int n = 0, nleaf = 0, levels = 0, kc = 0, ldl = 0, nn = 0;
  std::vector<int> leaf_sizes, lo, hi;  // per heap node
  // device storage
  double* store = nullptr;
  size_t store_doubles = 0, a_doubles = 0;
  double* D = nullptr;
  double* TD = nullptr;
  std::vector<double*> U12, V12, U21, V21, TU, TV;
  int* devints = nullptr;
  int n_devints = 0;
  double* dscal = nullptr;   // [0] anorm, [1..8] flops
  int* dstatus = nullptr;
  double* snapshot = nullptr;
  int* snap_ints = nullptr;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  char* arena2 = nullptr;      // never-reused scratch of side-stream work
  size_t arena2_bytes = 0;
  // cached plan of hodlr_solve_async (own arenas, so factorization plans are never disturbed)
  Plan splan;
  int splan_nrhs = 0;
  double* sbuf = nullptr;      // n x splan_nrhs staging buffer of the right-hand sides
  char* pack = nullptr;        // device staging of hodlr_download_compact (grown on demand)
  size_t pack_bytes = 0;
  char* sarena = nullptr;
  size_t sarena_bytes = 0;
  char* sarena2 = nullptr;
  size_t sarena2_bytes = 0;
  // plan of the factorization
  Plan plan;
  bool planned = false;
  long plan_version = 0;         // unique serial of the current `plan`, new on every rebuild
  double plan_tol = -1, plan_anorm = -2;
  cudaGraphExec_t gexec = nullptr;
  double g_tol = -1, g_anorm = -2;
  int g_cluster = 0;
  int g_conc = 0;
  bool factored = false;
};

// Return device memory: to the account's pool (no CUDA call), else cudaFree.
static void release_device(MemAcct* a, void* p) {
  if (a && a->pool && a->pool->owns(p)) a->pool->give(p);
  else cudaFree(p);
}

// Device allocation on behalf of matrix M, charged to its context's account.  HODLR_ENOMEM when
// the account's limit would be exceeded or cudaMalloc fails (*p is then nullptr).
static int mat_malloc(hodlr_mat* M, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  MemAcct* a = M->mem.get();
  if (a) {
    const long long lim = a->limit.load();
    const long long before = a->used.fetch_add((long long)bytes);
    if (lim > 0 && before + (long long)bytes > lim) {
      a->used.fetch_sub((long long)bytes);
      return HODLR_ENOMEM;
    }
  }
  if (a && a->pool) {
    *p = a->pool->take(bytes);
    if (!*p) {
      a->used.fetch_sub((long long)bytes);
      return HODLR_ENOMEM;
    }
  } else if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    if (a) a->used.fetch_sub((long long)bytes);
    return HODLR_ENOMEM;
  }
  M->allocs[*p] = bytes;
  M->held += (long long)bytes;
  return HODLR_OK;
}
template <class T>
static int mat_alloc(hodlr_mat* M, T** p, size_t bytes) {
  void* q = nullptr;
  int rc = mat_malloc(M, &q, bytes);
  *p = static_cast<T*>(q);
  return rc;
}
static void mat_free(hodlr_mat* M, void* p) {
  if (!p) return;
  size_t b = 0;
  auto it = M->allocs.find(p);
  if (it != M->allocs.end()) {
    b = it->second;
    M->allocs.erase(it);
  }
  release_device(M->mem.get(), p);
  M->held -= (long long)b;
  if (M->mem) M->mem->used.fetch_sub((long long)b);
}

// Device buffers outside any matrix (the server's right-hand sides), from the context's
// account: its pool when it has one.
void* hq::ctx_alloc(hodlr_ctx* ctx, size_t bytes) {
  MemAcct* a = ctx->mem.get();
  void* p = nullptr;
  if (a->pool) {
    p = a->pool->take(bytes);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) a->used.fetch_add((long long)((bytes + 255) & ~size_t(255)));
  return p;
}
void hq::ctx_free(hodlr_ctx* ctx, void* p, size_t bytes) {
  if (!p) return;
  release_device(ctx->mem.get(), p);
  ctx->mem->used.fetch_sub((long long)((bytes + 255) & ~size_t(255)));
}

cudaStream_t hq::ctx_stream(hodlr_ctx* ctx) { return ctx->s; }
int hq::ctx_cluster(hodlr_ctx* ctx) { return ctx->cluster; }
int hq::ctx_device(hodlr_ctx* ctx) { return ctx->dev; }

// ----------------------------------------------------------------------------- planner
struct Planner {
  hodlr_mat* M;
  Plan* P;
  // Scratch regions.  The main stream's work uses a LIFO arena (mark/release); the side
  // stream's work uses a second LIFO arena of its own (its work is ordered on its stream, so
  // one node's side work reuses the memory of the previous one, and the two streams never
  // alias); buffers that the main stream writes and the side stream reads later (hand-offs)
  // come from a third region that is never reused.
  size_t top = 0, high = 0;      // main-stream arena bump pointer
  char* base;                    // arena base (nullptr in the measuring pass)
  size_t top2 = 0;               // never-reused hand-off region
  char* base2 = nullptr;
  size_t top3 = 0, high3 = 0;    // side-stream arena
  char* base3 = nullptr;
  int stream = 0;                // stream of the records being emitted
  bool fresh = false;            // route alloc() to the never-reused hand-off region
  int int_top;                   // devints bump pointer
  int int_high;
  size_t cnt_top = 0;            // split-K tile counters (never reused, zero between uses)
  int* cnt_base = nullptr;
  int cluster;
  double tol;

  template <class T>
  T* alloc(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    if (fresh) {
      size_t off2 = top2;
      top2 += bytes;
      return reinterpret_cast<T*>(base2 + off2);
    }
    if (stream == 1) {
      size_t off3 = top3;
      top3 += bytes;
      high3 = std::max(high3, top3);
      return reinterpret_cast<T*>(base3 + off3);
    }
    size_t off = top;
    top += bytes;
    high = std::max(high, top);
    return reinterpret_cast<T*>(base + off);
  }
  // mark / release act on the arena of the stream whose records are being emitted
  size_t mark() const { return stream == 1 ? top3 : top; }
  void release(size_t m) {
    if (stream == 1) top3 = m;
    else top = m;
  }
  int event() { return P->nevents++; }
  void ev_record(int st, int ev) {
    Rec r = {};
    r.type = R_EVREC; r.stream = st; r.i0 = ev;
    P->recs.push_back(r);
  }
  void ev_wait(int st, int ev) {
    Rec r = {};
    r.type = R_EVWAIT; r.stream = st; r.i0 = ev;
    P->recs.push_back(r);
  }
  int ints(int n) {
    int r = int_top;
    int_top += n;
    int_high = std::max(int_high, int_top);
    return r;
  }

  // small operations as one-descriptor records (fill, int fill, identity, norm)
  void fill(double* p, size_t cnt, double v) {
    SmallDesc d = {};
    d.kind = kSmallFill; d.p = p; d.cnt = (long long)cnt; d.v = v;
    rec(R_SMALL, 1, put(std::vector<SmallDesc>{d}));
  }
  void ifill(int* p, size_t cnt, int v) {
    SmallDesc d = {};
    d.kind = kSmallIFill; d.ip = p; d.cnt = (long long)cnt; d.v = v;
    rec(R_SMALL, 1, put(std::vector<SmallDesc>{d}));
  }
  void ident(double* p, int ld, int rows, int cols) {
    SmallDesc d = {};
    d.kind = kSmallIdent; d.p = p; d.ld = ld; d.rows = rows; d.cols = cols;
    rec(R_SMALL, 1, put(std::vector<SmallDesc>{d}));
  }
  void norm(double* x, int n, double* out, bool scale) {
    SmallDesc d = {};
    d.kind = kSmallNorm; d.p = x; d.cnt = n; d.out = out; d.scale = scale ? 1 : 0;
    rec(R_NORMS, 1, put(std::vector<SmallDesc>{d}));
  }

  // every descriptor carries its matrix's rank table and flop counters
  void stamp(GemmDesc& d) const { d.di = M->devints; d.fl = M->dscal ? M->dscal + 1 : nullptr; }
  void stamp(ConcatDesc& d) const { d.di = M->devints; }
  void stamp(PanelDesc& d) const { d.di = M->devints; }
  void stamp(QRDesc& d) const { d.di = M->devints; d.fl = M->dscal ? M->dscal + 1 : nullptr; }
  void stamp(JacobiDesc& d) const { d.di = M->devints; d.fl = M->dscal ? M->dscal + 1 : nullptr; }
  void stamp(SelectDesc& d) const { d.di = M->devints; d.fl = M->dscal ? M->dscal + 1 : nullptr; }
  void stamp(CopyDesc& d) const { d.di = M->devints; }
  void stamp(SmallDesc&) const {}
  void stamp(int&) const {}

  template <class D>
  size_t put(std::vector<D> v) {
    for (auto& d : v) stamp(d);
    size_t off = (P->blob.size() + 15) & ~size_t(15);
    P->blob.resize(off + v.size() * sizeof(D));
    memcpy(P->blob.data() + off, v.data(), v.size() * sizeof(D));
    return off;
  }
  void rec(int type, int n, size_t off) {
    Rec r = {};
    r.type = type;
    r.n = n;
    r.off = off;
    r.stream = stream;
    P->recs.push_back(r);
  }
  void push(Rec r) {
    r.stream = stream;
    P->recs.push_back(r);
  }

  // ---------------------------------------------------------------- GEMM batches
  // Add a batch of GEMMs that may run concurrently (no output overlaps).
  void gemm(std::vector<GemmDesc> ds) {
    std::vector<GemmDesc> out;
    int work = 0;
    std::vector<int> red;
    int redblocks = 0;
    for (auto d : ds) {
      if (d.m <= 0 || d.n <= 0) continue;
      d.tiles_m = (d.m + kGemmBM - 1) / kGemmBM;
      d.tiles_n = (d.n + kGemmBN - 1) / kGemmBN;
      int tiles = d.tiles_m * d.tiles_n;
      d.ksplit = 1;
      d.part = nullptr;
      // A tile retires a few thousand flops per k on one SM (~7 GFLOP/s of FP64): split the
      // reduction so that one launch spreads over the whole GPU and each CTA runs >= 64 k.  Only
      // a literal k is split: a k set by a rank at run time (kref >= 0) is usually far below its
      // capacity, where splits would only add partial sums and their scratch.
      if (d.k >= 128 && d.kref < 0 && tiles < 608) {
        int ks = (608 + tiles - 1) / tiles;
        ks = std::min(ks, d.k / 64);
        ks = std::min(ks, 16);                   // partial sums: at most 16 x m x n scratch
        if (ks >= 2) d.ksplit = ks;
      }
      d.tile_count = nullptr;
      if (d.ksplit > 1) {
        d.part = alloc<double>((size_t)d.ksplit * d.m * d.n);
        d.tile_count = cnt_base + cnt_top;
        cnt_top += tiles;
      }
      d.work0 = work;
      work += tiles * d.ksplit;
      out.push_back(d);
    }
    if (out.empty()) return;
    size_t off = put(out);
    rec(R_GEMM, (int)out.size(), off);
    (void)redblocks;
    if (!red.empty()) {
      size_t roff = put(red);
      Rec r = {};
      r.type = R_REDUCE;
      r.n = (int)red.size() / 2;
      r.off = roff;
      r.extra0 = redblocks;
      r.extra1 = (int)off;   // offset of the GEMM descriptors
      push(r);
    }
  }

  static GemmDesc gd(const double* A, int lda, int ta, int mska, const double* B, int ldb, int tb,
                     int mskb, double* C, int ldc, int m, int mref, int n, int nref, int k, int kref,
                     double alpha, double beta, int step, int fmode) {
    GemmDesc d = {};
    d.A = A; d.lda = lda; d.ta = ta; d.mska = mska;
    d.B = B; d.ldb = ldb; d.tb = tb; d.mskb = mskb;
    d.C = C; d.ldc = ldc;
    d.m = m; d.mref = mref; d.n = n; d.nref = nref; d.k = k; d.kref = kref;
    d.alpha = alpha; d.beta = beta; d.alpha_ref = nullptr;
    d.step = step; d.fmode = fmode;
    return d;
  }

  // ------------------------------------------------------------------- tree helpers
  bool is_leaf(int v) const { return v >= M->nleaf - 1; }
  int m1(int v) const { return M->hi[2 * v + 1] - M->lo[2 * v + 1]; }
  int m2(int v) const { return M->hi[2 * v + 2] - M->lo[2 * v + 2]; }
  int size(int v) const { return M->hi[v] - M->lo[v]; }
  int r12(int v) const { return v; }
  int r21(int v) const { return M->nn + v; }
  int rT(int v) const { return 2 * M->nn + v; }
  void subtree_nodes(int s, std::vector<int>& internal, std::vector<int>& leaves, std::vector<int>& depth) const {
    std::vector<std::pair<int, int>> st = {{s, 0}};
    while (!st.empty()) {
      auto [v, d] = st.back();
      st.pop_back();
      if (is_leaf(v)) {
        leaves.push_back(v);
      } else {
        internal.push_back(v);
        depth.push_back(d);
        st.push_back({2 * v + 2, d + 1});
        st.push_back({2 * v + 1, d + 1});
      }
    }
  }
  // ancestors u (closest first) whose left subtree contains v: their lower blocks' right
  // factors supply the B_R / C rows of v's compressed column
  std::vector<int> rowsrc(int v) const {
    std::vector<int> out;
    int x = v;
    while (x > 0) {
      int p = (x - 1) / 2;
      if (x == 2 * p + 1) out.push_back(p);
      x = p;
    }
    return out;
  }

  View aview() const {
    return View{M->D, M->ldl, &M->U12, &M->V12, &M->U21, &M->V21, 0, M->nn};
  }
  View tview() const {
    return View{M->TD, M->ldl, &M->TU, &M->TV, nullptr, nullptr, 2 * M->nn, -1};
  }

  // ------------------------------------------------------------- HODLR x block (Table 1)
  // Y = alpha * op(part(H_s)) X + beta * Y (beta acts on the leaf products; block parts add).
  // part: 0 full, 1 unit lower, 2 upper.
  void matvec(const View& H, int s, int part, int trans, const double* X, int ldx, double* Y, int ldy,
              int pcap, int pref, double alpha, double beta, int step) {
    const int los = M->lo[s];
    std::vector<int> internal, leaves, depth;
    subtree_nodes(s, internal, leaves, depth);
    const int kc = M->kc;
    int mask = part == 0 ? kMaskNone : (part == 1 ? kMaskUnitLower : kMaskUpper);
    int fm = part == 0 ? 0 : 1;
    std::vector<GemmDesc> lv;
    for (int v : leaves) {
      int j = v - (M->nleaf - 1);
      int w = size(v), off = M->lo[v] - los;
      lv.push_back(gd(H.D + (size_t)j * H.ldl * H.ldl, H.ldl, trans, mask, X + off, ldx, 0, kMaskNone,
                      Y + off, ldy, w, -1, pcap, pref, w, -1, alpha, beta, step, fm));
    }
    gemm(lv);
    if (internal.empty()) return;
    size_t mk = mark();
    std::vector<GemmDesc> zd;
    struct Up { GemmDesc d; int depth; };
    std::vector<Up> ups;
    for (size_t q = 0; q < internal.size(); ++q) {
      int u = internal[q];
      int c1lo = M->lo[2 * u + 1] - los, c2lo = M->lo[2 * u + 2] - los;
      int a = m1(u), b = m2(u);
      bool up = (part == 0 || part == 2) && H.r12_base >= 0;
      bool lo = (part == 0 || part == 1) && H.r21_base >= 0;
      if (up) {
        double* Z = alloc<double>((size_t)kc * pcap);
        int rref = H.r12_base + u;
        if (!trans) {
          zd.push_back(gd((*H.V12)[u], b, 1, 0, X + c2lo, ldx, 0, 0, Z, kc, kc, rref, pcap, pref, b, -1, 1.0, 0.0, step, 0));
          ups.push_back({gd((*H.U12)[u], a, 0, 0, Z, kc, 0, 0, Y + c1lo, ldy, a, -1, pcap, pref, kc, rref, alpha, 1.0, step, 0), depth[q]});
        } else {
          zd.push_back(gd((*H.U12)[u], a, 1, 0, X + c1lo, ldx, 0, 0, Z, kc, kc, rref, pcap, pref, a, -1, 1.0, 0.0, step, 0));
          ups.push_back({gd((*H.V12)[u], b, 0, 0, Z, kc, 0, 0, Y + c2lo, ldy, b, -1, pcap, pref, kc, rref, alpha, 1.0, step, 0), depth[q]});
        }
      }
      if (lo) {
        double* Z = alloc<double>((size_t)kc * pcap);
        int rref = H.r21_base + u;
        if (!trans) {
          zd.push_back(gd((*H.V21)[u], a, 1, 0, X + c1lo, ldx, 0, 0, Z, kc, kc, rref, pcap, pref, a, -1, 1.0, 0.0, step, 0));
          ups.push_back({gd((*H.U21)[u], b, 0, 0, Z, kc, 0, 0, Y + c2lo, ldy, b, -1, pcap, pref, kc, rref, alpha, 1.0, step, 0), depth[q]});
        } else {
          zd.push_back(gd((*H.U21)[u], b, 1, 0, X + c2lo, ldx, 0, 0, Z, kc, kc, rref, pcap, pref, b, -1, 1.0, 0.0, step, 0));
          ups.push_back({gd((*H.V21)[u], a, 0, 0, Z, kc, 0, 0, Y + c1lo, ldy, a, -1, pcap, pref, kc, rref, alpha, 1.0, step, 0), depth[q]});
        }
      }
    }
    gemm(zd);
    int maxd = 0;
    for (auto& u : ups) maxd = std::max(maxd, u.depth);
    for (int dd = 0; dd <= maxd; ++dd) {
      std::vector<GemmDesc> g;
      for (auto& u : ups)
        if (u.depth == dd) g.push_back(u.d);
      gemm(g);
    }
    release(mk);
  }

  // ---------------------------------------------------------------- T_eps (Sec. 2.1.1)
  bool too_wide = false;
  struct Trunc {
    int nL, nR;
    std::vector<ConcatSeg> L, R;
    double thr;
    const double* thr_ref;
    double* Uout; int ldu;
    double* Vout; int ldv;
    int kout_ref;
    int step;
  };
  static ConcatSeg seg(const double* src, int lds, int cols, int colsref, double alpha) {
    ConcatSeg g;
    g.src = src; g.lds = lds; g.cols = cols; g.colsref = colsref; g.alpha = alpha;
    return g;
  }

  void truncate(std::vector<Trunc>& ps) {
    if (ps.empty()) return;
    size_t mk = mark();
    const int kc = M->kc;
    int np = (int)ps.size();
    std::vector<ConcatDesc> cds;
    std::vector<QRDesc> qds;
    std::vector<GemmDesc> gM, gP1, gZ, gP2, gP3, gF;
    std::vector<JacobiDesc> jds;
    std::vector<SelectDesc> sds;
    std::vector<CopyDesc> cps;
    for (auto& p : ps) {
      int Kcap = 0;
      for (auto& g : p.L) Kcap += g.cols;
      int KcapR = 0;
      for (auto& g : p.R) KcapR += g.cols;
      Kcap = std::max(Kcap, KcapR);
      if (Kcap == 0) Kcap = 1;
      if (std::min(p.nR, Kcap) > 4096) too_wide = true;   // beyond the Jacobi kernel's column list
      int q1c = std::min(p.nL, Kcap), q2c = std::min(p.nR, Kcap);
      double* Lb = alloc<double>((size_t)p.nL * Kcap);
      double* Rb = alloc<double>((size_t)p.nR * Kcap);
      double* tauL = alloc<double>(Kcap);
      double* tauR = alloc<double>(Kcap);
      double* TL = alloc<double>((size_t)q1c * q1c);
      double* TR = alloc<double>((size_t)q2c * q2c);
      double* GL = alloc<double>((size_t)q1c * q1c);
      double* GR = alloc<double>((size_t)q2c * q2c);
      double* Mb = alloc<double>((size_t)q1c * q2c);
      double* nrm = alloc<double>(q2c);
      int* rot = alloc<int>(kMaxSweeps);
      double* Uk = alloc<double>((size_t)q1c * kc);
      double* P1 = alloc<double>((size_t)Kcap * kc);
      double* Zb = alloc<double>((size_t)q2c * kc);
      double* P2 = alloc<double>((size_t)q1c * kc);
      double* P3 = alloc<double>((size_t)q1c * kc);
      double* P2r = alloc<double>((size_t)q2c * kc);
      double* P3r = alloc<double>((size_t)q2c * kc);
      int iL = ints(2), iR = ints(2);   // (K, q) for each side
      int kref = p.kout_ref;
      ConcatDesc c = {};
      c.dst = Lb; c.ldd = p.nL; c.rows = p.nL; c.cap = Kcap; c.nseg = (int)p.L.size();
      for (int i = 0; i < c.nseg; ++i) c.seg[i] = p.L[i];
      c.kout_ref = iL;
      cds.push_back(c);
      c = {};
      c.dst = Rb; c.ldd = p.nR; c.rows = p.nR; c.cap = Kcap; c.nseg = (int)p.R.size();
      for (int i = 0; i < c.nseg; ++i) c.seg[i] = p.R[i];
      c.kout_ref = iR;
      cds.push_back(c);
      QRDesc q = {};
      q.A = Lb; q.lda = p.nL; q.h = p.nL; q.w = Kcap; q.href = -1; q.wref = iL;
      q.tau = tauL; q.T = TL; q.ldt = q1c; q.G = GL; q.ldg = q1c; q.step = kStepNone; q.fmode = 1;
      qds.push_back(q);
      q.A = Rb; q.lda = p.nR; q.h = p.nR; q.wref = iR; q.tau = tauR; q.T = TR; q.ldt = q2c; q.G = GR; q.ldg = q2c;
      qds.push_back(q);
      // M = R1 R2^T  (q1 x q2)
      gM.push_back(gd(Lb, p.nL, 0, kMaskUpper, Rb, p.nR, 1, kMaskUpper, Mb, q1c, q1c, iL + 1, q2c, iR + 1,
                      Kcap, iL, 1.0, 0.0, kStepNone, -1));
      JacobiDesc jd = {};
      jd.M = Mb; jd.ldm = q1c; jd.q1 = q1c; jd.q2 = q2c; jd.q1ref = iL + 1; jd.q2ref = iR + 1;
      jd.nrm = nrm; jd.rot = rot; jd.thr = p.thr; jd.thr_ref = p.thr_ref;
      jds.push_back(jd);
      SelectDesc sd = {};
      sd.W = Mb; sd.ldw = q1c; sd.nrm = nrm; sd.q1 = q1c; sd.q2 = q2c; sd.q1ref = iL + 1; sd.q2ref = iR + 1;
      sd.thr = p.thr; sd.thr_ref = p.thr_ref; sd.U = Uk; sd.ldu = q1c; sd.kcap = kc; sd.kref = kref;
      sd.status = M->dstatus; sd.nL = p.nL; sd.nR = p.nR; sd.Kref = iL; sd.step = p.step;
      sds.push_back(sd);
      // Z = R2 (R1^T Uk)
      gP1.push_back(gd(Lb, p.nL, 1, kMaskUpper, Uk, q1c, 0, 0, P1, Kcap, Kcap, iL, kc, kref, q1c, iL + 1, 1.0, 0.0, kStepNone, -1));
      gZ.push_back(gd(Rb, p.nR, 0, kMaskUpper, P1, Kcap, 0, 0, Zb, q2c, q2c, iR + 1, kc, kref, Kcap, iR, 1.0, 0.0, kStepNone, -1));
      // outputs: Q1 [Uk; 0] and Q2 [Z; 0] with Q = I - Y T Y^T
      CopyDesc cp = {};
      cp.src = Uk; cp.lds = q1c; cp.dst = p.Uout; cp.ldd = p.ldu; cp.rows = p.nL; cp.rows_src = q1c;
      cp.rows_src_ref = iL + 1; cp.cols = kc; cp.colsref = kref; cp.alpha = 1.0;
      cps.push_back(cp);
      cp.src = Zb; cp.lds = q2c; cp.dst = p.Vout; cp.ldd = p.ldv; cp.rows = p.nR; cp.rows_src = q2c;
      cp.rows_src_ref = iR + 1;
      cps.push_back(cp);
      gP2.push_back(gd(Lb, p.nL, 1, kMaskUnitLower, Uk, q1c, 0, 0, P2, q1c, q1c, iL + 1, kc, kref, q1c, iL + 1, 1.0, 0.0, kStepNone, -1));
      gP2.push_back(gd(Rb, p.nR, 1, kMaskUnitLower, Zb, q2c, 0, 0, P2r, q2c, q2c, iR + 1, kc, kref, q2c, iR + 1, 1.0, 0.0, kStepNone, -1));
      gP3.push_back(gd(TL, q1c, 0, kMaskUpper, P2, q1c, 0, 0, P3, q1c, q1c, iL + 1, kc, kref, q1c, iL + 1, 1.0, 0.0, kStepNone, -1));
      gP3.push_back(gd(TR, q2c, 0, kMaskUpper, P2r, q2c, 0, 0, P3r, q2c, q2c, iR + 1, kc, kref, q2c, iR + 1, 1.0, 0.0, kStepNone, -1));
      gF.push_back(gd(Lb, p.nL, 0, kMaskUnitLower, P3, q1c, 0, 0, p.Uout, p.ldu, p.nL, -1, kc, kref, q1c, iL + 1, -1.0, 1.0, kStepNone, -1));
      gF.push_back(gd(Rb, p.nR, 0, kMaskUnitLower, P3r, q2c, 0, 0, p.Vout, p.ldv, p.nR, -1, kc, kref, q2c, iR + 1, -1.0, 1.0, kStepNone, -1));
    }
    rec(R_CONCAT, (int)cds.size(), put(cds));
    rec(R_QR, (int)qds.size(), put(qds));
    gemm(gM);
    rec(R_JACOBI, (int)jds.size(), put(jds));
    rec(R_SELECT, (int)sds.size(), put(sds));
    gemm(gP1);
    gemm(gZ);
    rec(R_COPY, (int)cps.size(), put(cps));
    gemm(gP2);
    gemm(gP3);
    gemm(gF);
    (void)np;
    release(mk);
  }

  // ------------------------------ HODLR approximation of a dense device matrix (Sec. 2.1.1)
  // Leaves are copied.  Every off-diagonal block B (m x q) is sampled by a randomized range
  // finder (Halko, Martinsson and Tropp, SIAM Review 2011, Alg. 4.1): Y = B Omega with
  // p = min(kc + 16, m, q) Gaussian columns, Q = orth(Y) by Householder QR, Z = B^T Q, and
  // T_eps(Q Z^T) gives the stored factors and the rank (device rank table).  The kept rank is at
  // most kc (else HODLR_ERANK), so at least 16 columns of oversampling remain and the range error
  // stays at the level of sigma_{k+1} (when p = q the sample spans B exactly).
  void compress_dense(const double* A, int lda, double thr, unsigned long long seed) {
    const int kc = M->kc;
    std::vector<CopyDesc> cps;
    for (int j = 0; j < M->nleaf; ++j) {
      const int v = M->nleaf - 1 + j, lo = M->lo[v], w = size(v);
      CopyDesc cp = {};
      cp.src = A + lo + (size_t)lo * lda; cp.lds = lda;
      cp.dst = M->D + (size_t)j * M->ldl * M->ldl; cp.ldd = M->ldl;
      cp.rows = w; cp.rows_src = w; cp.rows_src_ref = -1; cp.cols = w; cp.colsref = -1; cp.alpha = 1.0;
      cps.push_back(cp);
    }
    rec(R_COPY, (int)cps.size(), put(cps));
    for (int l = 0; l < M->levels; ++l) {
      size_t mk = mark();
      std::vector<QRDesc> qds;
      std::vector<GemmDesc> gY, gP2, gP3, gQ, gZ;
      std::vector<Trunc> ts;
      std::vector<Rec> pre;
      std::vector<SmallDesc> idents;
      for (int v = (1 << l) - 1; v < (2 << l) - 1; ++v) {
        for (int which = 0; which < 2; ++which) {
          const int rlo = M->lo[which == 0 ? 2 * v + 1 : 2 * v + 2];
          const int clo = M->lo[which == 0 ? 2 * v + 2 : 2 * v + 1];
          const int m = which == 0 ? m1(v) : m2(v);
          const int q = which == 0 ? m2(v) : m1(v);
          const int p = std::min(std::min(kc + 16, m), q);
          const double* B = A + rlo + (size_t)clo * lda;
          double* Om = alloc<double>((size_t)q * p);
          double* Y = alloc<double>((size_t)m * p);
          double* tau = alloc<double>(p);
          double* T = alloc<double>((size_t)p * p);
          double* G = alloc<double>((size_t)p * p);
          double* Q = alloc<double>((size_t)m * p);
          double* P2 = alloc<double>((size_t)p * p);
          double* P3 = alloc<double>((size_t)p * p);
          double* Z = alloc<double>((size_t)q * p);
          const unsigned long long stream = seed * (unsigned long long)(2 * M->nn + 2) + 2 * v + which;
          Rec g = {};
          g.type = R_GAUSS; g.p0 = Om; g.cnt = (size_t)q * p;
          g.i0 = (int)(unsigned)(stream & 0xffffffffull); g.i1 = (int)(unsigned)(stream >> 32);
          pre.push_back(g);
          SmallDesc sd = {};
          sd.kind = kSmallIdent; sd.p = Q; sd.ld = m; sd.rows = m; sd.cols = p;
          idents.push_back(sd);
          gY.push_back(gd(B, lda, 0, 0, Om, q, 0, 0, Y, m, m, -1, p, -1, q, -1, 1.0, 0.0, kStepNone, -1));
          QRDesc qd = {};
          qd.A = Y; qd.lda = m; qd.h = m; qd.w = p; qd.href = -1; qd.wref = -1; qd.tau = tau; qd.T = T;
          qd.ldt = p; qd.G = G; qd.ldg = p; qd.step = kStepNone; qd.fmode = 1;
          qds.push_back(qd);
          // Q = (I - Y T Y^T) [I; 0]
          gP2.push_back(gd(Y, m, 1, kMaskUnitLower, Q, m, 0, 0, P2, p, p, -1, p, -1, p, -1, 1.0, 0.0, kStepNone, -1));
          gP3.push_back(gd(T, p, 0, kMaskUpper, P2, p, 0, 0, P3, p, p, -1, p, -1, p, -1, 1.0, 0.0, kStepNone, -1));
          gQ.push_back(gd(Y, m, 0, kMaskUnitLower, P3, p, 0, 0, Q, m, m, -1, p, -1, p, -1, -1.0, 1.0, kStepNone, -1));
          gZ.push_back(gd(B, lda, 1, 0, Q, m, 0, 0, Z, q, q, -1, p, -1, m, -1, 1.0, 0.0, kStepNone, -1));
          Trunc t;
          t.nL = m; t.nR = q;
          t.L.push_back(seg(Q, m, p, -1, 1.0));
          t.R.push_back(seg(Z, q, p, -1, 1.0));
          t.thr = thr; t.thr_ref = nullptr;
          t.Uout = which == 0 ? M->U12[v] : M->U21[v]; t.ldu = m;
          t.Vout = which == 0 ? M->V12[v] : M->V21[v]; t.ldv = q;
          t.kout_ref = which == 0 ? r12(v) : r21(v);
          t.step = kStepNone;
          ts.push_back(t);
        }
      }
      for (auto& r : pre) push(r);
      rec(R_SMALL, (int)idents.size(), put(idents));
      gemm(gY);
      rec(R_QR, (int)qds.size(), put(qds));
      gemm(gP2);
      gemm(gP3);
      gemm(gQ);
      gemm(gZ);
      truncate(ts);
      release(mk);
    }
  }

  // ------------------------------------------- rectangular HODLR and the permuted QR (Sec. 6)
  // Row blocks moved by a row permutation: rows src .. src + len - 1 of the source go to rows
  // dst .. dst + len - 1 of the destination (inverse: the other way round).
  struct RowSeg {
    int src, dst, len;
  };
  void copy_rows(const double* S, int lds, double* D, int ldd, int cols, const std::vector<RowSeg>& segs,
                 bool inverse) {
    std::vector<CopyDesc> cps;
    for (const auto& g : segs) {
      if (g.len <= 0 || cols <= 0) continue;
      CopyDesc c = {};
      c.src = S + (inverse ? g.dst : g.src); c.lds = lds;
      c.dst = D + (inverse ? g.src : g.dst); c.ldd = ldd;
      c.rows = g.len; c.rows_src = g.len; c.rows_src_ref = -1; c.cols = cols; c.colsref = -1; c.alpha = 1.0;
      cps.push_back(c);
    }
    if (!cps.empty()) rec(R_COPY, (int)cps.size(), put(cps));
  }

  // Householder QR of the dense h x w matrix W (h >= w) in place, in the LAPACK layout (R on and
  // above the diagonal, the unit lower trapezoidal Y below it), with the w x w upper T of the
  // compact WY form (Alg. 1 blocked by panels of kRectNB columns): each panel is factored by
  // the cluster QR kernel (its own T block), the columns to its right are updated with
  // Q_p^T = I - Y_p T_p^T Y_p^T by three GEMMs, and the off-diagonal blocks of T are formed
  // afterwards by T(0:j0, panel) = -T(0:j0, 0:j0) (Y(:, 0:j0)^T Y_p) T_p (Sec. 3, Eq. (10)).
  static constexpr int kRectNB = 64;
  void dense_qr(double* W, int ldw, int h, int w, double* T, int ldt, double* tau) {
    const int nb = kRectNB;
    double* G = alloc<double>((size_t)nb * nb);
    double* X = alloc<double>((size_t)nb * w);
    double* X2 = alloc<double>((size_t)nb * w);
    {
      CopyDesc z = {};                                     // T starts at zero (upper part written)
      z.src = nullptr; z.dst = T; z.ldd = ldt; z.rows = w; z.rows_src = 0; z.rows_src_ref = -1;
      z.cols = w; z.colsref = -1;
      rec(R_COPY, 1, put(std::vector<CopyDesc>{z}));
    }
    for (int j0 = 0; j0 < w; j0 += nb) {
      const int nbp = std::min(nb, w - j0), rest = w - j0 - nbp, hp = h - j0;
      double* Yp = W + j0 + (size_t)j0 * ldw;
      double* Tp = T + j0 + (size_t)j0 * ldt;
      QRDesc q = {};
      q.A = Yp; q.lda = ldw; q.h = hp; q.w = nbp; q.href = -1; q.wref = -1; q.tau = tau + j0;
      q.T = Tp; q.ldt = ldt; q.G = G; q.ldg = nb; q.step = kStepNone; q.fmode = 0;
      rec(R_QR, 1, put(std::vector<QRDesc>{q}));
      if (rest == 0) continue;
      double* Cp = W + j0 + (size_t)(j0 + nbp) * ldw;
      gemm({gd(Yp, ldw, 1, kMaskUnitLower, Cp, ldw, 0, 0, X, nb, nbp, -1, rest, -1, hp, -1, 1.0, 0.0, kStepNone, -1)});
      gemm({gd(Tp, ldt, 1, kMaskUpper, X, nb, 0, 0, X2, nb, nbp, -1, rest, -1, nbp, -1, 1.0, 0.0, kStepNone, -1)});
      gemm({gd(Yp, ldw, 0, kMaskUnitLower, X2, nb, 0, 0, Cp, ldw, hp, -1, rest, -1, nbp, -1, -1.0, 1.0, kStepNone, -1)});
    }
    if (w <= nb) return;
    // Y(:, 0:j0)^T Y_p for every later panel at once (rows above j0 of Y_p are zero)
    double* Gx = alloc<double>((size_t)w * w);
    std::vector<GemmDesc> gg;
    for (int j0 = nb; j0 < w; j0 += nb) {
      const int nbp = std::min(nb, w - j0);
      gg.push_back(gd(W + j0, ldw, 1, 0, W + j0 + (size_t)j0 * ldw, ldw, 0, kMaskUnitLower, Gx + (size_t)j0 * w, w,
                      j0, -1, nbp, -1, h - j0, -1, 1.0, 0.0, kStepNone, -1));
    }
    gemm(gg);
    double* Xt = alloc<double>((size_t)w * nb);
    for (int j0 = nb; j0 < w; j0 += nb) {                 // in order: each needs T(0:j0, 0:j0)
      const int nbp = std::min(nb, w - j0);
      gemm({gd(T, ldt, 0, kMaskUpper, Gx + (size_t)j0 * w, w, 0, 0, Xt, w, j0, -1, nbp, -1, j0, -1, 1.0, 0.0,
               kStepNone, -1)});
      gemm({gd(Xt, w, 0, 0, T + j0 + (size_t)j0 * ldt, ldt, 0, kMaskUpper, T + (size_t)j0 * ldt, ldt, j0, -1, nbp,
               -1, nbp, -1, -1.0, 0.0, kStepNone, -1)});
    }
  }

  // ||A||_2 of a dense m x n matrix by power iteration on A^T A from the normalized all-ones
  // vector (the reading used for HODLR matrices), written to *out.
  void dense_norm2(const double* A, int lda, int m, int n, double* out, int iters) {
    double* x = alloc<double>(n);
    double* z = alloc<double>(m);
    fill(x, n, 1.0 / std::sqrt((double)n));
    for (int it = 0; it < iters; ++it) {
      gemm({gd(A, lda, 0, 0, x, n, 0, 0, z, m, m, -1, 1, -1, n, -1, 1.0, 0.0, kStepNone, -1)});
      gemm({gd(A, lda, 1, 0, z, m, 0, 0, x, n, n, -1, 1, -1, m, -1, 1.0, 0.0, kStepNone, -1)});
      norm(x, n, out, true);
    }
    gemm({gd(A, lda, 0, 0, x, n, 0, 0, z, m, m, -1, 1, -1, n, -1, 1.0, 0.0, kStepNone, -1)});
    norm(z, m, out, false);
  }

  // Rectangular HODLR approximation (Sec. 2.1.1 on a row and a column partition) of the dense
  // matrix A, as compress_dense: leaves copied, every off-diagonal block sampled by the
  // randomized range finder and truncated by T_eps at thr (times *thr_ref when given).  rr / cr:
  // row / column range of every heap-ordered node; the factors go to the matrix's U12, V12, U21,
  // V21 (ranks in its rank table), leaf j to leaf[j] (ld = its rows).
  void compress_rect(const double* A, int lda, const std::vector<std::pair<int, int>>& rr,
                     const std::vector<std::pair<int, int>>& cr, const std::vector<double*>& leaf, double thr,
                     const double* thr_ref, unsigned long long seed) {
    const int kc = M->kc, nleaf = M->nleaf;
    std::vector<CopyDesc> cps;
    for (int j = 0; j < nleaf; ++j) {
      const int v = nleaf - 1 + j, mr = rr[v].second - rr[v].first, nc = cr[v].second - cr[v].first;
      CopyDesc cp = {};
      cp.src = A + rr[v].first + (size_t)cr[v].first * lda; cp.lds = lda;
      cp.dst = leaf[j]; cp.ldd = std::max(mr, 1);
      cp.rows = mr; cp.rows_src = mr; cp.rows_src_ref = -1; cp.cols = nc; cp.colsref = -1; cp.alpha = 1.0;
      cps.push_back(cp);
    }
    rec(R_COPY, (int)cps.size(), put(cps));
    for (int l = 0; l < M->levels; ++l) {
      size_t mk = mark();
      std::vector<QRDesc> qds;
      std::vector<GemmDesc> gY, gP2, gP3, gQ, gZ;
      std::vector<Trunc> ts;
      std::vector<Rec> pre;
      std::vector<SmallDesc> idents;
      for (int v = (1 << l) - 1; v < (2 << l) - 1; ++v) {
        for (int which = 0; which < 2; ++which) {
          const int a = which == 0 ? 2 * v + 1 : 2 * v + 2, b = which == 0 ? 2 * v + 2 : 2 * v + 1;
          const int rlo = rr[a].first, clo = cr[b].first;
          const int m = rr[a].second - rr[a].first, q = cr[b].second - cr[b].first;
          const int p = std::min(std::min(kc + 16, m), q);
          if (m == 0 || q == 0 || p == 0) continue;
          const double* B = A + rlo + (size_t)clo * lda;
          double* Om = alloc<double>((size_t)q * p);
          double* Y = alloc<double>((size_t)m * p);
          double* tau = alloc<double>(p);
          double* T = alloc<double>((size_t)p * p);
          double* G = alloc<double>((size_t)p * p);
          double* Q = alloc<double>((size_t)m * p);
          double* P2 = alloc<double>((size_t)p * p);
          double* P3 = alloc<double>((size_t)p * p);
          double* Z = alloc<double>((size_t)q * p);
          const unsigned long long stream = seed * (unsigned long long)(2 * M->nn + 2) + 2 * v + which;
          Rec g = {};
          g.type = R_GAUSS; g.p0 = Om; g.cnt = (size_t)q * p;
          g.i0 = (int)(unsigned)(stream & 0xffffffffull); g.i1 = (int)(unsigned)(stream >> 32);
          pre.push_back(g);
          SmallDesc sd = {};
          sd.kind = kSmallIdent; sd.p = Q; sd.ld = m; sd.rows = m; sd.cols = p;
          idents.push_back(sd);
          gY.push_back(gd(B, lda, 0, 0, Om, q, 0, 0, Y, m, m, -1, p, -1, q, -1, 1.0, 0.0, kStepNone, -1));
          QRDesc qd = {};
          qd.A = Y; qd.lda = m; qd.h = m; qd.w = p; qd.href = -1; qd.wref = -1; qd.tau = tau; qd.T = T;
          qd.ldt = p; qd.G = G; qd.ldg = p; qd.step = kStepNone; qd.fmode = 1;
          qds.push_back(qd);
          gP2.push_back(gd(Y, m, 1, kMaskUnitLower, Q, m, 0, 0, P2, p, p, -1, p, -1, p, -1, 1.0, 0.0, kStepNone, -1));
          gP3.push_back(gd(T, p, 0, kMaskUpper, P2, p, 0, 0, P3, p, p, -1, p, -1, p, -1, 1.0, 0.0, kStepNone, -1));
          gQ.push_back(gd(Y, m, 0, kMaskUnitLower, P3, p, 0, 0, Q, m, m, -1, p, -1, p, -1, -1.0, 1.0, kStepNone, -1));
          gZ.push_back(gd(B, lda, 1, 0, Q, m, 0, 0, Z, q, q, -1, p, -1, m, -1, 1.0, 0.0, kStepNone, -1));
          Trunc t;
          t.nL = m; t.nR = q;
          t.L.push_back(seg(Q, m, p, -1, 1.0));
          t.R.push_back(seg(Z, q, p, -1, 1.0));
          t.thr = thr; t.thr_ref = thr_ref;
          t.Uout = which == 0 ? M->U12[v] : M->U21[v]; t.ldu = m;
          t.Vout = which == 0 ? M->V12[v] : M->V21[v]; t.ldv = q;
          t.kout_ref = which == 0 ? r12(v) : r21(v);
          t.step = kStepNone;
          ts.push_back(t);
        }
      }
      for (auto& r : pre) push(r);
      if (!idents.empty()) rec(R_SMALL, (int)idents.size(), put(idents));
      gemm(gY);
      if (!qds.empty()) rec(R_QR, (int)qds.size(), put(qds));
      gemm(gP2);
      gemm(gP3);
      gemm(gQ);
      gemm(gZ);
      truncate(ts);
      release(mk);
    }
  }

  // Dense m x n matrix (ld) of a rectangular HODLR matrix: leaves copied, every off-diagonal
  // block formed as U V^T at its stored rank.
  void rect_to_dense(const std::vector<std::pair<int, int>>& rr, const std::vector<std::pair<int, int>>& cr,
                     const std::vector<double*>& leaf, double* out, int ld) {
    const int nleaf = M->nleaf, kc = M->kc;
    std::vector<CopyDesc> cps;
    for (int j = 0; j < nleaf; ++j) {
      const int v = nleaf - 1 + j, mr = rr[v].second - rr[v].first, nc = cr[v].second - cr[v].first;
      CopyDesc cp = {};
      cp.src = leaf[j]; cp.lds = std::max(mr, 1);
      cp.dst = out + rr[v].first + (size_t)cr[v].first * ld; cp.ldd = ld;
      cp.rows = mr; cp.rows_src = mr; cp.rows_src_ref = -1; cp.cols = nc; cp.colsref = -1; cp.alpha = 1.0;
      cps.push_back(cp);
    }
    rec(R_COPY, (int)cps.size(), put(cps));
    std::vector<GemmDesc> g;
    for (int v = 0; v < M->nn; ++v) {
      for (int which = 0; which < 2; ++which) {
        const int a = which == 0 ? 2 * v + 1 : 2 * v + 2, b = which == 0 ? 2 * v + 2 : 2 * v + 1;
        const int m = rr[a].second - rr[a].first, q = cr[b].second - cr[b].first;
        if (m == 0 || q == 0) continue;
        double* C = out + rr[a].first + (size_t)cr[b].first * ld;
        const double* U = which == 0 ? M->U12[v] : M->U21[v];
        const double* V = which == 0 ? M->V12[v] : M->V21[v];
        // C = U V^T at the stored rank (k = 0 writes zeros)
        g.push_back(gd(U, m, 0, 0, V, q, 1, 0, C, ld, m, -1, q, -1, kc, which == 0 ? r12(v) : r21(v), 1.0, 0.0,
                       kStepNone, -1));
      }
    }
    gemm(g);
  }

  // --------------------------------------------------------- left-orthogonal form (Sec. 2.1)
  void left_orth(int p) {
    size_t mk = mark();
    const int kc = M->kc;
    int a = m1(p), b = m2(p);          // U21: b x r, V21: a x r
    int rr = r21(p);
    double* S = alloc<double>((size_t)b * kc);
    double* Vt = alloc<double>((size_t)a * kc);
    int kq = std::min(b, kc);
    double* tau = alloc<double>(kc);
    double* T = alloc<double>((size_t)kq * kq);
    double* G = alloc<double>((size_t)kq * kq);
    double* P2 = alloc<double>((size_t)kc * kc);
    double* P3 = alloc<double>((size_t)kc * kc);
    std::vector<CopyDesc> cps(2);
    cps[0] = {}; cps[0].src = M->U21[p]; cps[0].lds = b; cps[0].dst = S; cps[0].ldd = b; cps[0].rows = b;
    cps[0].rows_src = b; cps[0].rows_src_ref = -1; cps[0].cols = kc; cps[0].colsref = rr; cps[0].alpha = 1.0;
    cps[1] = {}; cps[1].src = M->V21[p]; cps[1].lds = a; cps[1].dst = Vt; cps[1].ldd = a; cps[1].rows = a;
    cps[1].rows_src = a; cps[1].rows_src_ref = -1; cps[1].cols = kc; cps[1].colsref = rr; cps[1].alpha = 1.0;
    rec(R_COPY, 2, put(cps));
    QRDesc q = {};
    q.A = S; q.lda = b; q.h = b; q.w = kc; q.href = -1; q.wref = rr; q.tau = tau; q.T = T; q.ldt = kq;
    q.G = G; q.ldg = kq; q.step = kStepLeftOrth; q.fmode = 1;
    rec(R_QR, 1, put(std::vector<QRDesc>{q}));
    // U21 <- Q = (I - Y T Y^T) [I; 0]
    ident(M->U21[p], b, b, kc);
    gemm({gd(S, b, 1, kMaskUnitLower, M->U21[p], b, 0, 0, P2, kc, kc, rr, kc, rr, kc, rr, 1.0, 0.0, kStepNone, -1)});
    gemm({gd(T, kq, 0, kMaskUpper, P2, kc, 0, 0, P3, kc, kq, rr, kc, rr, kq, rr, 1.0, 0.0, kStepNone, -1)});
    gemm({gd(S, b, 0, kMaskUnitLower, P3, kc, 0, 0, M->U21[p], b, b, -1, kc, rr, kq, rr, -1.0, 1.0, kStepNone, -1),
          // V21 <- V21 R^T  (B_R <- R B_R)
          gd(Vt, a, 0, 0, S, b, 1, kMaskUpper, M->V21[p], a, a, -1, kc, rr, kc, rr, 1.0, 0.0, kStepLeftOrth, 0)});
    release(mk);
  }

  // ------------------------------------------------------ lowest level of Alg. 2 at a leaf
  void leaf(int v) {
    size_t mk = mark();
    const int kc = M->kc;
    int j = v - (M->nleaf - 1);
    int w = size(v);
    std::vector<int> rs = rowsrc(v);
    int hcap = w + (int)rs.size() * kc;
    double* Pn = alloc<double>((size_t)hcap * w);
    double* tau = alloc<double>(w);
    double* G = alloc<double>((size_t)w * w);
    int href = ints(1);
    PanelDesc pd = {};
    pd.D = M->D + (size_t)j * M->ldl * M->ldl; pd.ldD = M->ldl; pd.w = w; pd.P = Pn; pd.ldP = hcap;
    pd.nsrc = (int)rs.size();
    for (size_t i = 0; i < rs.size(); ++i) {
      int u = rs[i];
      int off = M->lo[v] - M->lo[2 * u + 1];
      pd.src[i] = M->V21[u] + off;
      pd.lds[i] = m1(u);
      pd.rref[i] = r21(u);
      pd.rcap[i] = kc;
    }
    pd.href = href;
    rec(R_GATHER, 1, put(std::vector<PanelDesc>{pd}));
    QRDesc q = {};
    q.A = Pn; q.lda = hcap; q.h = hcap; q.w = w; q.href = href; q.wref = -1; q.tau = tau;
    q.T = M->TD + (size_t)j * M->ldl * M->ldl; q.ldt = M->ldl; q.G = G; q.ldg = w;
    q.step = kStepLeafQR; q.fmode = 0;
    rec(R_QR, 1, put(std::vector<QRDesc>{q}));
    rec(R_SCATTER, 1, put(std::vector<PanelDesc>{pd}));
    release(mk);
  }

  // ----------------------------------------------------------------- Alg. 2 recursion
  // tdone[v]: event (side stream) after which T of subtree v is complete; -1 for leaves
  std::vector<int> tdone;

  void node(int v) {
    if (tdone.empty()) tdone.assign(2 * M->nleaf - 1, -1);
    if (v != 0 && v == 2 * ((v - 1) / 2) + 1) left_orth((v - 1) / 2);   // B of v is A21 of its parent
    if (is_leaf(v)) {
      leaf(v);
      return;
    }
    const int kc = M->kc;
    const int c1 = 2 * v + 1, c2 = 2 * v + 2;
    const int a = m1(v), b = m2(v);
    node(c1);
    View A = aview(), T = tview();
    std::vector<int> rs = rowsrc(v);
    const double* anorm = M->dscal;
    size_t mk = mark();
    // S~ = T_{eps ||A||}( Y11^T A12 + Y21^T A22 + Y_BR1^T B_R2 + Y_C1^T C2 )
    double* X1 = alloc<double>((size_t)a * kc);
    double* X2 = alloc<double>((size_t)b * kc);
    matvec(A, c1, 1, 1, M->U12[v], a, X1, a, kc, r12(v), 1.0, 0.0, kStepS);
    matvec(A, c2, 0, 1, M->U21[v], b, X2, b, kc, r21(v), 1.0, 0.0, kStepS);
    double* SL = alloc<double>((size_t)a * kc);
    fresh = true;                                  // read later by the side stream
    double* SR = alloc<double>((size_t)b * kc);
    double* X3 = alloc<double>((size_t)a * kc);
    fresh = false;
    int kS = ints(1);
    {
      Trunc t;
      t.nL = a; t.nR = b;
      t.L = {seg(X1, a, kc, r12(v), 1.0), seg(M->V21[v], a, kc, r21(v), 1.0)};
      t.R = {seg(M->V12[v], b, kc, r12(v), 1.0), seg(X2, b, kc, r21(v), 1.0)};
      for (int u : rs) {
        int off = M->lo[v] - M->lo[2 * u + 1];
        t.L.push_back(seg(M->V21[u] + off, m1(u), kc, r21(u), 1.0));
        t.R.push_back(seg(M->V21[u] + off + a, m1(u), kc, r21(u), 1.0));
      }
      t.thr = tol; t.thr_ref = anorm; t.Uout = SL; t.ldu = a; t.Vout = SR; t.ldv = b; t.kout_ref = kS;
      t.step = kStepS;
      std::vector<Trunc> ts = {t};
      truncate(ts);
    }
    // S = T1^T S~   (T of subtree c1 is finished on the side stream)
    if (tdone[c1] >= 0) ev_wait(0, tdone[c1]);
    double* SL2 = alloc<double>((size_t)a * kc);
    matvec(T, c1, 2, 1, SL, a, SL2, a, kc, kS, 1.0, 0.0, kStepTS);
    // Y11 S (input of A^12), then A^12 = T_{eps ||A||}(A12 - Y11 S) on the side stream:
    // nothing later in the recursion reads R12 of this node
    matvec(A, c1, 1, 0, SL2, a, X3, a, kc, kS, 1.0, 0.0, kStepUpdate);
    int e_x3 = event();
    ev_record(0, e_x3);
    {
      stream = 1;                                  // side-stream arena
      ev_wait(1, e_x3);
      Trunc t;
      t.nL = a; t.nR = b;
      t.L = {seg(M->U12[v], a, kc, r12(v), 1.0), seg(X3, a, kc, kS, -1.0)};
      t.R = {seg(M->V12[v], b, kc, r12(v), 1.0), seg(SR, b, kc, kS, 1.0)};
      t.thr = tol; t.thr_ref = anorm; t.Uout = M->U12[v]; t.ldu = a; t.Vout = M->V12[v]; t.ldv = b;
      t.kout_ref = r12(v); t.step = kStepUpdate;
      std::vector<Trunc> ts = {t};
      truncate(ts);
      stream = 0;
    }
    // A^22 = A~22 -_H (B_L21 (Y~_B S_L)) S_R^T
    double* Pm = alloc<double>((size_t)kc * kc);
    double* Uu = alloc<double>((size_t)b * kc);
    gemm({gd(M->V21[v], a, 1, 0, SL2, a, 0, 0, Pm, kc, kc, r21(v), kc, kS, a, -1, 1.0, 0.0, kStepUpdate, 0)});
    gemm({gd(M->U21[v], b, 0, 0, Pm, kc, 0, 0, Uu, b, b, -1, kc, kS, kc, r21(v), 1.0, 0.0, kStepUpdate, 0)});
    lr_update(c2, Uu, b, SR, b, kS);
    // B^_R2 = B_R2 - Y_BR1 S,  C^2 = C2 - Y_C1 S   (rows stored transposed in ancestors' V21)
    if (!rs.empty()) {
      std::vector<GemmDesc> g1, g2;
      for (int u : rs) {
        int off = M->lo[v] - M->lo[2 * u + 1];
        double* Pu = alloc<double>((size_t)kc * kc);
        g1.push_back(gd(SL2, a, 1, 0, M->V21[u] + off, m1(u), 0, 0, Pu, kc, kc, kS, kc, r21(u), a, -1, 1.0, 0.0, kStepUpdate, 0));
        g2.push_back(gd(SR, b, 0, 0, Pu, kc, 0, 0, M->V21[u] + off + a, m1(u), b, -1, kc, r21(u), kc, kS, -1.0, 1.0, kStepUpdate, 0));
      }
      gemm(g1);
      gemm(g2);
    }
    release(mk);
    node(c2);
    // T~12 = T_eps( Y21^T Y22 + Y_BR1^T Y_BR2 + Y_C1^T Y_C2 ),  T12 = -T1 T~12 T2, on the side
    // stream once the second block column is factored; its inputs are final from here on
    int e_c2 = event();
    ev_record(0, e_c2);
    stream = 1;                                    // side-stream arena, reused node to node
    const size_t mk3 = mark();
    ev_wait(1, e_c2);
    {
      double* X4 = alloc<double>((size_t)b * kc);
      matvec(A, c2, 1, 1, M->U21[v], b, X4, b, kc, r21(v), 1.0, 0.0, kStepT12);
      double* TLb = alloc<double>((size_t)a * kc);
      double* TRb = alloc<double>((size_t)b * kc);
      Trunc t;
      t.nL = a; t.nR = b;
      t.L = {seg(M->V21[v], a, kc, r21(v), 1.0)};
      t.R = {seg(X4, b, kc, r21(v), 1.0)};
      for (int u : rs) {
        int off = M->lo[v] - M->lo[2 * u + 1];
        t.L.push_back(seg(M->V21[u] + off, m1(u), kc, r21(u), 1.0));
        t.R.push_back(seg(M->V21[u] + off + a, m1(u), kc, r21(u), 1.0));
      }
      t.thr = tol; t.thr_ref = nullptr; t.Uout = TLb; t.ldu = a; t.Vout = TRb; t.ldv = b; t.kout_ref = rT(v);
      t.step = kStepT12;
      std::vector<Trunc> ts = {t};
      truncate(ts);
      matvec(T, c1, 2, 0, TLb, a, M->TU[v], a, kc, rT(v), -1.0, 0.0, kStepT12);
      matvec(T, c2, 2, 1, TRb, b, M->TV[v], b, kc, rT(v), 1.0, 0.0, kStepT12);
    }
    int e_t = event();
    ev_record(1, e_t);
    tdone[v] = e_t;
    release(mk3);
    stream = 0;
  }

  // HODLR low-rank update  H_s <- H_s -_H U V^T  (Table 1)
  void lr_update(int s, const double* U, int ldu, const double* V, int ldv, int kref) {
    const int kc = M->kc;
    std::vector<int> internal, leaves, depth;
    subtree_nodes(s, internal, leaves, depth);
    const int los = M->lo[s];
    std::vector<GemmDesc> g;
    for (int v : leaves) {
      int j = v - (M->nleaf - 1);
      int w = size(v), off = M->lo[v] - los;
      g.push_back(gd(U + off, ldu, 0, 0, V + off, ldv, 1, 0, M->D + (size_t)j * M->ldl * M->ldl, M->ldl,
                     w, -1, w, -1, kc, kref, -1.0, 1.0, kStepUpdate, 0));
    }
    gemm(g);
    // The truncations of one depth of the subtree form one batch; the batches run depth after
    // depth, so that each reuses the scratch of the previous one (truncate releases its
    // scratch) and the arena holds one depth's worth, not the whole subtree's.
    int maxdep = 0;
    for (int dd : depth) maxdep = std::max(maxdep, dd);
    for (int dep = 0; dep <= maxdep; ++dep) {
      std::vector<Trunc> ts;
      for (size_t q = 0; q < internal.size(); ++q) {
        if (depth[q] != dep) continue;
        const int u = internal[q];
        int a = m1(u), b = m2(u);
        int c1lo = M->lo[2 * u + 1] - los, c2lo = M->lo[2 * u + 2] - los;
        Trunc t;
        t.nL = a; t.nR = b;
        t.L = {seg(M->U12[u], a, kc, r12(u), 1.0), seg(U + c1lo, ldu, kc, kref, -1.0)};
        t.R = {seg(M->V12[u], b, kc, r12(u), 1.0), seg(V + c2lo, ldv, kc, kref, 1.0)};
        t.thr = tol; t.thr_ref = M->dscal; t.Uout = M->U12[u]; t.ldu = a; t.Vout = M->V12[u]; t.ldv = b;
        t.kout_ref = r12(u); t.step = kStepUpdate;
        ts.push_back(t);
        Trunc t2;
        t2.nL = b; t2.nR = a;
        t2.L = {seg(M->U21[u], b, kc, r21(u), 1.0), seg(U + c2lo, ldu, kc, kref, -1.0)};
        t2.R = {seg(M->V21[u], a, kc, r21(u), 1.0), seg(V + c1lo, ldv, kc, kref, 1.0)};
        t2.thr = tol; t2.thr_ref = M->dscal; t2.Uout = M->U21[u]; t2.ldu = b; t2.Vout = M->V21[u]; t2.ldv = a;
        t2.kout_ref = r21(u); t2.step = kStepUpdate;
        ts.push_back(t2);
      }
      truncate(ts);
    }
  }

  // ||A||_2 by power iteration on A^T A (device), result into dscal[0]
  void norm_estimate(int iters) {
    size_t mk = mark();
    const int n = M->n;
    double* x = alloc<double>(n);
    double* y = alloc<double>(n);
    double* z = alloc<double>(n);
    double* tmp = alloc<double>(1);
    fill(x, n, 1.0 / std::sqrt((double)n));
    View A = aview();
    for (int it = 0; it < iters; ++it) {
      matvec(A, 0, 0, 0, x, n, y, n, 1, -1, 1.0, 0.0, kStepNorm);
      matvec(A, 0, 0, 1, y, n, z, n, 1, -1, 1.0, 0.0, kStepNorm);
      norm(z, n, tmp, true);
      std::swap(x, z);
    }
    matvec(A, 0, 0, 0, x, n, y, n, 1, -1, 1.0, 0.0, kStepNorm);
    norm(y, n, M->dscal, false);
    release(mk);
  }
};

// ------------------------------------------------------------------------------ executor
// kernel kind of a record (profiling): 0 GEMM, 1 reduce, 2 QR, 3 Jacobi, 4 select,
// 5 data movement, 6 norm, 7 other, -1 not a kernel
static int rec_kind(int t) {
  switch (t) {
    case R_GEMM: return 0;
    case R_REDUCE: return 1;
    case R_QR: return 2;
    case R_JACOBI: return 3;
    case R_SELECT: return 4;
    case R_CONCAT: case R_GATHER: case R_SCATTER: case R_COPY: case R_SMALL: return 5;
    case R_NORMS: return 6;
    case R_TRSM: case R_GAUSS: return 7;
    default: return -1;
  }
}

struct Profiler {
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind;
};

static int run_plan_on(hodlr_ctx* ctx, hodlr_mat* M, Plan& P, Profiler* prof, cudaStream_t mainst,
                       cudaStream_t sidest) {
  char* db = P.dblob;
  bool two = !P.events.empty();
  cudaEvent_t fork = nullptr, join = nullptr;
  if (two) {
    // the side stream starts after everything queued before the plan on the main stream
    HQ_CUDA_OK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    HQ_CUDA_OK(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
    HQ_CUDA_OK(cudaEventRecord(fork, mainst));
    HQ_CUDA_OK(cudaStreamWaitEvent(sidest, fork, 0));
  }
  for (const Rec& r : P.recs) {
    cudaStream_t s = r.stream ? sidest : mainst;
    int kd = rec_kind(r.type);
    if (prof && kd >= 0) {
      cudaEvent_t e0;
      cudaEventCreate(&e0);
      cudaEventRecord(e0, s);
      prof->ev.push_back(e0);
      prof->kind.push_back(kd);
    }
    const char* hb = P.blob.data() + r.off;
    char* dp = db + r.off;
    cudaError_t e = cudaSuccess;
    switch (r.type) {
      case R_GEMM:
        e = launch_gemm((GemmDesc*)hb, r.n, (GemmDesc*)dp, s);
        break;
      case R_REDUCE:
        e = launch_gemm_reduce((const GemmDesc*)(db + r.extra1), (const int*)dp, r.n, r.extra0, s);
        break;
      case R_CONCAT: e = launch_concat((const ConcatDesc*)hb, r.n, (ConcatDesc*)dp, s); break;
      case R_GATHER: e = launch_panel_gather((const PanelDesc*)hb, r.n, (PanelDesc*)dp, s); break;
      case R_SCATTER: e = launch_panel_scatter((const PanelDesc*)hb, r.n, (PanelDesc*)dp, s); break;
      case R_QR:
        e = launch_qr((const QRDesc*)hb, r.n, (QRDesc*)dp, ctx->cluster, smem_cap(ctx), s, ctx->cluster_large);
        break;
      case R_JACOBI:
        e = launch_jacobi((const JacobiDesc*)hb, r.n, (JacobiDesc*)dp, ctx->cluster, smem_cap(ctx), s,
                          ctx->cluster_large);
        break;
      case R_SELECT: e = launch_select((const SelectDesc*)hb, r.n, (SelectDesc*)dp, s); break;
      case R_COPY: e = launch_copy((const CopyDesc*)hb, r.n, (CopyDesc*)dp, s); break;
      case R_SMALL: e = launch_small((const SmallDesc*)hb, r.n, (SmallDesc*)dp, s); break;
      case R_NORMS: e = launch_norms((const SmallDesc*)hb, r.n, (SmallDesc*)dp, s); break;
      case R_GAUSS:
        e = launch_gauss(r.p0, r.cnt, ((unsigned long long)(unsigned)r.i1 << 32) | (unsigned)r.i0, s);
        break;

      case R_TRSM: e = launch_trsm_leaf(r.p0, r.i0, r.i1, reinterpret_cast<double*>(r.ip), r.i2, r.i3, s); break;
      case R_EVREC: e = cudaEventRecord(P.events[r.i0], s); break;
      case R_EVWAIT: e = cudaStreamWaitEvent(s, P.events[r.i0], 0); break;
      default: e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return cuda_fail(e, __FILE__, __LINE__);
    if (prof && kd >= 0) {
      cudaEvent_t e1;
      cudaEventCreate(&e1);
      cudaEventRecord(e1, s);
      prof->ev.push_back(e1);
    }
  }
  if (two) {
    // the main stream waits for the side stream's last work (joins it back)
    HQ_CUDA_OK(cudaEventRecord(join, sidest));
    HQ_CUDA_OK(cudaStreamWaitEvent(mainst, join, 0));
    cudaEventDestroy(fork);
    cudaEventDestroy(join);
  }
  return HODLR_OK;
}

static int run_plan(hodlr_ctx* ctx, hodlr_mat* M, Plan& P, Profiler* prof = nullptr) {
  return run_plan_on(ctx, M, P, prof, ctx->s, ctx->side);
}

static int upload_plan(hodlr_mat* M, Plan& P) {
  for (auto e : P.events) cudaEventDestroy(e);
  P.events.assign(P.nevents, nullptr);
  for (auto& e : P.events)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return HODLR_ECUDA;
  mat_free(M, P.dblob);
  P.dblob = nullptr;
  P.dblob_bytes = std::max<size_t>(P.blob.size(), 16);
  if (int rc = mat_alloc(M, &P.dblob, P.dblob_bytes)) return rc;
  if (!P.blob.empty()) HQ_CUDA_OK(cudaMemcpy(P.dblob, P.blob.data(), P.blob.size(), cudaMemcpyHostToDevice));
  // a pageable upload may still be in flight when cudaMemcpy returns, and the context's streams
  // do not wait for the legacy stream: finish it before any launch reads the descriptors
  HQ_CUDA_OK(cudaStreamSynchronize(cudaStreamLegacy));
  return HODLR_OK;
}

// Device bytes of a plan's scratch, measured by the planner's first (measuring) pass: the
// main-stream arena, the hand-off region followed by the side-stream arena, the split-K tile
// counters and the descriptor blob.
struct PlanSizes {
  size_t arena = 0, hand = 0, side = 0, counters = 0, blob = 0;
  size_t arena_bytes() const { return arena + 4096; }
  size_t arena2_bytes() const { return hand + side + 4096; }
  size_t counter_bytes() const { return sizeof(int) * counters; }
  size_t blob_bytes() const { return std::max<size_t>(blob, 16); }
};

template <class F>
static int measure_plan(hodlr_mat* M, Plan& P, double tol, F&& body, PlanSizes* out) {
  P.recs.clear();
  P.blob.clear();
  Planner pl;
  pl.M = M; pl.P = &P; pl.base = nullptr; pl.base2 = nullptr; pl.base3 = nullptr; pl.cnt_base = nullptr;
  P.nevents = 0;
  pl.int_top = 3 * M->nn; pl.int_high = pl.int_top;
  pl.cluster = 0; pl.tol = tol;
  body(pl);
  if (pl.int_high > M->n_devints) return HODLR_ENOMEM;
  if (pl.too_wide) return HODLR_EINVAL;
  out->arena = pl.high;
  out->hand = (pl.top2 + 255) & ~size_t(255);
  out->side = pl.high3;
  out->counters = pl.cnt_top;
  out->blob = P.blob.size();
  return HODLR_OK;
}

// Build a plan: measure its scratch, allocate what is missing, plan again for real.
template <class F>
static int build_plan(hodlr_mat* M, Plan& P, int cluster, double tol, F&& body, bool solve_arenas = false) {
  char** ar1 = solve_arenas ? &M->sarena : &M->arena;
  size_t* ar1b = solve_arenas ? &M->sarena_bytes : &M->arena_bytes;
  char** ar2 = solve_arenas ? &M->sarena2 : &M->arena2;
  size_t* ar2b = solve_arenas ? &M->sarena2_bytes : &M->arena2_bytes;
  PlanSizes ps;
  if (int rc = measure_plan(M, P, tol, body, &ps)) return rc;
  if (ps.arena_bytes() > *ar1b) {
    mat_free(M, *ar1);
    *ar1 = nullptr;
    *ar1b = 0;
    if (int rc = mat_alloc(M, ar1, ps.arena_bytes())) return rc;
    *ar1b = ps.arena_bytes();
  }
  if (ps.counters > P.counters_n) {
    mat_free(M, P.counters);
    P.counters = nullptr;
    P.counters_n = 0;
    if (int rc = mat_alloc(M, &P.counters, ps.counter_bytes())) return rc;
    P.counters_n = ps.counters;
    HQ_CUDA_OK(cudaMemset(P.counters, 0, ps.counter_bytes()));
    HQ_CUDA_OK(cudaStreamSynchronize(cudaStreamLegacy));
  }
  if (ps.arena2_bytes() > *ar2b) {
    mat_free(M, *ar2);
    *ar2 = nullptr;
    *ar2b = 0;
    if (int rc = mat_alloc(M, ar2, ps.arena2_bytes())) return rc;
    *ar2b = ps.arena2_bytes();
  }
  P.recs.clear();
  P.blob.clear();
  Planner pl;
  pl.M = M; pl.P = &P; pl.base = *ar1;
  pl.base2 = *ar2;
  pl.base3 = *ar2 + ps.hand;
  pl.cnt_base = P.counters;
  P.nevents = 0;
  pl.int_top = 3 * M->nn; pl.int_high = pl.int_top;
  pl.cluster = cluster; pl.tol = tol;
  body(pl);
  return upload_plan(M, P);
}

static void free_plan(hodlr_mat* M, Plan& P) {
  for (auto e : P.events) cudaEventDestroy(e);
  P.events.clear();
  P.nevents = 0;
  mat_free(M, P.dblob);
  P.dblob = nullptr;
  mat_free(M, P.counters);
  P.counters = nullptr;
  P.counters_n = 0;
  P.recs.clear();
  P.blob.clear();
}

static void free_groups(hodlr_ctx* ctx);

// =============================================================================== C ABI
extern "C" {

const char* hodlr_strerror(int code) {
  switch (code) {
    case HODLR_OK: return "ok";
    case HODLR_EINVAL: return "invalid argument";
    case HODLR_ENOMEM: return "out of memory";
    case HODLR_ERANK: return "rank capacity exceeded (result truncated)";
    case HODLR_ESINGULAR: return "singular triangular factor";
    case HODLR_ETIMEOUT: return "device wait timed out";
    case HODLR_ECUDA: return "CUDA error";
    case HODLR_ESTATE: return "invalid state";
    default: return "unknown error";
  }
}

int hodlr_ctx_create(int device, hodlr_ctx** out) {
  if (!out) return HODLR_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return HODLR_EINVAL;
  }
  HQ_CUDA_OK(cudaSetDevice(device));
  hodlr_ctx* c = new (std::nothrow) hodlr_ctx();
  if (!c) return HODLR_ENOMEM;
  c->dev = device;
  if (cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return HODLR_ECUDA;
  }
  c->s = c->own;
  if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess) {
    cudaStreamDestroy(c->own);
    delete c;
    return HODLR_ECUDA;
  }
  c->cluster = qr_max_cluster();
  *out = c;
  return HODLR_OK;
}

void hodlr_ctx_destroy(hodlr_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->dev);
  if (ctx->own) {
    cudaStreamSynchronize(ctx->own);
    cudaStreamDestroy(ctx->own);
  }
  if (ctx->side) {
    cudaStreamSynchronize(ctx->side);
    cudaStreamDestroy(ctx->side);
  }
  for (auto& pr : ctx->pool) {
    cudaStreamSynchronize(pr.first);
    cudaStreamSynchronize(pr.second);
    cudaStreamDestroy(pr.first);
    cudaStreamDestroy(pr.second);
  }
  if (ctx->bgraph) cudaGraphExecDestroy(ctx->bgraph);
  free_groups(ctx);
  if (ctx->batch_owner) hodlr_free(ctx->batch_owner);
  delete ctx;
}

int hodlr_ctx_set_stream(hodlr_ctx* ctx, void* stream) {
  if (!ctx) return HODLR_EINVAL;
  ctx->s = stream ? (cudaStream_t)stream : ctx->own;
  return HODLR_OK;
}

int hodlr_ctx_set_cluster(hodlr_ctx* ctx, int cluster) {
  if (!ctx) return HODLR_EINVAL;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  if (cluster < 1 || cluster > qr_max_cluster()) return HODLR_EINVAL;
  ctx->cluster = cluster;
  return HODLR_OK;
}

int hodlr_ctx_set_cluster_large(hodlr_ctx* ctx, int cluster) {
  if (!ctx) return HODLR_EINVAL;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  if (cluster < 0 || cluster > qr_max_cluster()) return HODLR_EINVAL;
  ctx->cluster_large = cluster;
  return HODLR_OK;
}

int hodlr_ctx_get_cluster(hodlr_ctx* ctx, int* cluster) {
  if (!ctx || !cluster) return HODLR_EINVAL;
  *cluster = ctx->cluster;
  return HODLR_OK;
}

int hodlr_ctx_set_concurrency(hodlr_ctx* ctx, int factorizations) {
  if (!ctx || factorizations < 1) return HODLR_EINVAL;
  ctx->concurrency = factorizations;
  return HODLR_OK;
}

int hodlr_ctx_set_batch_group(hodlr_ctx* ctx, int max_matrices) {
  if (!ctx || max_matrices < 0) return HODLR_EINVAL;
  ctx->batch_group = max_matrices;
  return HODLR_OK;
}

int hodlr_ctx_get_concurrency(hodlr_ctx* ctx, int* factorizations) {
  if (!ctx || !factorizations) return HODLR_EINVAL;
  *factorizations = ctx->concurrency;
  return HODLR_OK;
}

int hodlr_sync(hodlr_ctx* ctx) {
  if (!ctx) return HODLR_EINVAL;
  HQ_CUDA_OK(cudaStreamSynchronize(ctx->s));
  return HODLR_OK;
}

static int upload_values(hodlr_ctx* ctx, hodlr_mat* M, const double* const* leaves,
                         const double* const* U12, const double* const* V12, const int* r12,
                         const double* const* U21, const double* const* V21, const int* r21) {
  for (int v = 0; v < M->nn; ++v) {
    int a = M->hi[2 * v + 1] - M->lo[2 * v + 1], b = M->hi[2 * v + 2] - M->lo[2 * v + 2];
    if (r12[v] < 0 || r21[v] < 0 || r12[v] > M->kc || r21[v] > M->kc || r12[v] > std::min(a, b) ||
        r21[v] > std::min(a, b))
      return HODLR_EINVAL;
    if ((r12[v] && (!U12 || !V12 || !U12[v] || !V12[v])) || (r21[v] && (!U21 || !V21 || !U21[v] || !V21[v])))
      return HODLR_EINVAL;
  }
  for (int j = 0; j < M->nleaf; ++j)
    if (!leaves || !leaves[j]) return HODLR_EINVAL;
  // every value must be finite: a NaN or infinity would spread through the whole factorization
  auto finite = [](const double* p, size_t cnt) {
    for (size_t i = 0; i < cnt; ++i)
      if (!std::isfinite(p[i])) return false;
    return true;
  };
  for (int j = 0; j < M->nleaf; ++j) {
    const size_t w = M->leaf_sizes[j];
    if (!finite(leaves[j], w * w)) return HODLR_EINVAL;
  }
  for (int v = 0; v < M->nn; ++v) {
    const size_t a = M->hi[2 * v + 1] - M->lo[2 * v + 1], b = M->hi[2 * v + 2] - M->lo[2 * v + 2];
    if (r12[v] && (!finite(U12[v], a * r12[v]) || !finite(V12[v], b * r12[v]))) return HODLR_EINVAL;
    if (r21[v] && (!finite(U21[v], b * r21[v]) || !finite(V21[v], a * r21[v]))) return HODLR_EINVAL;
  }
  cudaStream_t s = ctx->s;
  for (int j = 0; j < M->nleaf; ++j) {
    int w = M->leaf_sizes[j];
    HQ_CUDA_OK(cudaMemcpy2DAsync(M->D + (size_t)j * M->ldl * M->ldl, sizeof(double) * M->ldl, leaves[j],
                                 sizeof(double) * w, sizeof(double) * w, w, cudaMemcpyHostToDevice, s));
  }
  for (int v = 0; v < M->nn; ++v) {
    int a = M->hi[2 * v + 1] - M->lo[2 * v + 1], b = M->hi[2 * v + 2] - M->lo[2 * v + 2];
    if (r12[v]) {
      HQ_CUDA_OK(cudaMemcpyAsync(M->U12[v], U12[v], sizeof(double) * a * r12[v], cudaMemcpyHostToDevice, s));
      HQ_CUDA_OK(cudaMemcpyAsync(M->V12[v], V12[v], sizeof(double) * b * r12[v], cudaMemcpyHostToDevice, s));
    }
    if (r21[v]) {
      HQ_CUDA_OK(cudaMemcpyAsync(M->U21[v], U21[v], sizeof(double) * b * r21[v], cudaMemcpyHostToDevice, s));
      HQ_CUDA_OK(cudaMemcpyAsync(M->V21[v], V21[v], sizeof(double) * a * r21[v], cudaMemcpyHostToDevice, s));
    }
  }
  std::vector<int> ranks(3 * M->nn, 0);
  for (int v = 0; v < M->nn; ++v) {
    ranks[v] = r12[v];
    ranks[M->nn + v] = r21[v];
  }
  if (M->nn) {
    HQ_CUDA_OK(cudaMemcpyAsync(M->devints, ranks.data(), sizeof(int) * 3 * M->nn, cudaMemcpyHostToDevice, s));
  }
  HQ_CUDA_OK(cudaStreamSynchronize(s));
  M->factored = false;
  return HODLR_OK;
}

void hodlr_free(hodlr_mat* M) {
  if (!M) return;
  if (M->gexec) cudaGraphExecDestroy(M->gexec);
  free_plan(M, M->plan);
  free_plan(M, M->splan);
  for (auto& kv : M->allocs) release_device(M->mem.get(), kv.first);   // storage, tables, arenas, buffers
  if (M->mem) M->mem->used.fetch_sub(M->held);
  M->allocs.clear();
  delete M;
}

}  // extern "C"

// Sizes, cluster tree and storage layout of a matrix of the given partition (host only).
static int layout_mat(hodlr_mat* M, int n, int nleaf, const int* leaf_sizes, int rank_cap) {
  if (!leaf_sizes || n <= 0 || nleaf <= 0 || (nleaf & (nleaf - 1)) || rank_cap < 1 || rank_cap > 256)
    return HODLR_EINVAL;
  long sum = 0;
  int maxw = 0;
  for (int j = 0; j < nleaf; ++j) {
    if (leaf_sizes[j] <= 0 || leaf_sizes[j] > 4096) return HODLR_EINVAL;
    sum += leaf_sizes[j];
    maxw = std::max(maxw, leaf_sizes[j]);
  }
  if (sum != n) return HODLR_EINVAL;
  M->n = n; M->nleaf = nleaf; M->kc = rank_cap; M->ldl = maxw; M->nn = nleaf - 1;
  int lev = 0;
  while ((1 << lev) < nleaf) ++lev;
  M->levels = lev;
  M->leaf_sizes.assign(leaf_sizes, leaf_sizes + nleaf);
  int nnodes = 2 * nleaf - 1;
  M->lo.assign(nnodes, 0);
  M->hi.assign(nnodes, 0);
  int off = 0;
  for (int j = 0; j < nleaf; ++j) {
    M->lo[nleaf - 1 + j] = off;
    off += leaf_sizes[j];
    M->hi[nleaf - 1 + j] = off;
  }
  for (int v = nleaf - 2; v >= 0; --v) {
    M->lo[v] = M->lo[2 * v + 1];
    M->hi[v] = M->hi[2 * v + 2];
  }
  // storage: [A leaves][A factors][T leaves][T factors]
  size_t leafd = (size_t)nleaf * maxw * maxw;
  size_t afac = 0, tfac = 0;
  for (int v = 0; v < M->nn; ++v) {
    size_t a = M->hi[2 * v + 1] - M->lo[2 * v + 1], b = M->hi[2 * v + 2] - M->lo[2 * v + 2];
    afac += 2 * (a + b) * rank_cap;
    tfac += (a + b) * rank_cap;
  }
  M->a_doubles = leafd + afac;
  M->store_doubles = 2 * leafd + afac + tfac;
  M->n_devints = 3 * M->nn + 64 * nleaf + 4096;
  return HODLR_OK;
}

// Pointers of the leaf and factor pools inside the storage block starting at `store`.
static void place_mat(hodlr_mat* M, double* store) {
  const int rank_cap = M->kc;
  const size_t leafd = (size_t)M->nleaf * M->ldl * M->ldl;
  double* p = store;
  M->store = store;
  M->D = p;
  p += leafd;
  M->U12.resize(M->nn); M->V12.resize(M->nn); M->U21.resize(M->nn); M->V21.resize(M->nn);
  M->TU.resize(M->nn); M->TV.resize(M->nn);
  for (int v = 0; v < M->nn; ++v) {
    size_t a = M->hi[2 * v + 1] - M->lo[2 * v + 1], b = M->hi[2 * v + 2] - M->lo[2 * v + 2];
    M->U12[v] = p; p += a * rank_cap;
    M->V12[v] = p; p += b * rank_cap;
    M->U21[v] = p; p += b * rank_cap;
    M->V21[v] = p; p += a * rank_cap;
  }
  M->TD = p;
  p += leafd;
  for (int v = 0; v < M->nn; ++v) {
    size_t a = M->hi[2 * v + 1] - M->lo[2 * v + 1], b = M->hi[2 * v + 2] - M->lo[2 * v + 2];
    M->TU[v] = p; p += a * rank_cap;
    M->TV[v] = p; p += b * rank_cap;
  }
}

// Allocate a matrix of the given partition with all values and ranks zero.
static int alloc_mat(hodlr_ctx* ctx, int n, int nleaf, const int* leaf_sizes, int rank_cap, hodlr_mat** out) {
  if (!ctx || !out) return HODLR_EINVAL;
  hodlr_mat* M = new (std::nothrow) hodlr_mat();
  if (!M) return HODLR_ENOMEM;
  int rc = layout_mat(M, n, nleaf, leaf_sizes, rank_cap);
  if (rc != HODLR_OK) {
    delete M;
    return rc;
  }
  if (cudaSetDevice(ctx->dev) != cudaSuccess) {
    delete M;
    return cuda_fail(cudaGetLastError(), __FILE__, __LINE__);
  }
  M->mem = ctx->mem;
  double* store = nullptr;
  if (mat_alloc(M, &store, M->store_doubles * sizeof(double)) != HODLR_OK) {
    hodlr_free(M);
    return HODLR_ENOMEM;
  }
  cudaMemsetAsync(store, 0, M->store_doubles * sizeof(double), ctx->s);
  place_mat(M, store);
  if (mat_alloc(M, &M->devints, sizeof(int) * M->n_devints) != HODLR_OK ||
      mat_alloc(M, &M->dscal, sizeof(double) * 32) != HODLR_OK ||
      mat_alloc(M, &M->dstatus, sizeof(int) * 4) != HODLR_OK) {
    hodlr_free(M);
    return HODLR_ENOMEM;
  }
  cudaMemsetAsync(M->devints, 0, sizeof(int) * M->n_devints, ctx->s);
  cudaMemsetAsync(M->dscal, 0, sizeof(double) * 32, ctx->s);
  cudaMemsetAsync(M->dstatus, 0, sizeof(int) * 4, ctx->s);
  *out = M;
  return HODLR_OK;
}

extern "C" {

int hodlr_build(hodlr_ctx* ctx, int n, int nleaf, const int* leaf_sizes, const double* const* leaves,
                const double* const* U12, const double* const* V12, const int* r12,
                const double* const* U21, const double* const* V21, const int* r21, int rank_cap,
                hodlr_mat** out) {
  if (nleaf > 1 && (!r12 || !r21)) return HODLR_EINVAL;
  if (!leaves) return HODLR_EINVAL;
  hodlr_mat* M = nullptr;
  int rc = alloc_mat(ctx, n, nleaf, leaf_sizes, rank_cap, &M);
  if (rc) return rc;
  std::vector<int> z12(std::max(1, M->nn), 0), z21(std::max(1, M->nn), 0);
  rc = upload_values(ctx, M, leaves, U12, V12, r12 ? r12 : z12.data(), U21, V21, r21 ? r21 : z21.data());
  if (rc != HODLR_OK) {
    hodlr_free(M);
    return rc;
  }
  *out = M;
  return HODLR_OK;
}

int hodlr_upload(hodlr_ctx* ctx, hodlr_mat* A, const double* const* leaves, const double* const* U12,
                 const double* const* V12, const int* r12, const double* const* U21, const double* const* V21,
                 const int* r21) {
  if (!ctx || !A) return HODLR_EINVAL;
  std::vector<int> z(std::max(1, A->nn), 0);
  // clear the factor columns beyond the new ranks is not needed: kernels read only r columns
  return upload_values(ctx, A, leaves, U12, V12, r12 ? r12 : z.data(), U21, V21, r21 ? r21 : z.data());
}

int hodlr_snapshot(hodlr_ctx* ctx, hodlr_mat* A) {
  if (!ctx || !A) return HODLR_EINVAL;
  if (!A->snapshot) {
    if (mat_alloc(A, &A->snapshot, A->a_doubles * sizeof(double)) != HODLR_OK ||
        mat_alloc(A, &A->snap_ints, sizeof(int) * std::max(1, 3 * A->nn)) != HODLR_OK) {
      mat_free(A, A->snapshot);
      A->snapshot = nullptr;
      return HODLR_ENOMEM;
    }
  }
  HQ_CUDA_OK(cudaMemcpyAsync(A->snapshot, A->store, A->a_doubles * sizeof(double), cudaMemcpyDeviceToDevice, ctx->s));
  if (A->nn)
    HQ_CUDA_OK(cudaMemcpyAsync(A->snap_ints, A->devints, sizeof(int) * 3 * A->nn, cudaMemcpyDeviceToDevice, ctx->s));
  return HODLR_OK;
}

int hodlr_restore(hodlr_ctx* ctx, hodlr_mat* A) {
  if (!ctx || !A) return HODLR_EINVAL;
  if (!A->snapshot) return HODLR_ESTATE;
  HQ_CUDA_OK(cudaMemcpyAsync(A->store, A->snapshot, A->a_doubles * sizeof(double), cudaMemcpyDeviceToDevice, ctx->s));
  if (A->nn)
    HQ_CUDA_OK(cudaMemcpyAsync(A->devints, A->snap_ints, sizeof(int) * 3 * A->nn, cudaMemcpyDeviceToDevice, ctx->s));
  A->factored = false;
  return HODLR_OK;
}

// The factorization: clear the flop counters and status, estimate ||A||_2 unless given, Alg. 2.
static void plan_qr(Planner& pl, hodlr_mat* A, bool estimate_norm) {
  pl.fill(A->dscal + 1, 16, 0.0);
  pl.ifill(A->dstatus, 4, 0);
  if (estimate_norm) pl.norm_estimate(30);
  pl.node(0);
}

static int ensure_plan(hodlr_ctx* ctx, hodlr_mat* A, double tol, double anorm) {
  bool est = !(anorm > 0);
  if (A->planned && A->plan_tol == tol && ((A->plan_anorm > 0) == !est)) return HODLR_OK;
  free_plan(A, A->plan);
  if (A->gexec) {
    cudaGraphExecDestroy(A->gexec);
    A->gexec = nullptr;
  }
  int rc = build_plan(A, A->plan, ctx->cluster, tol, [&](Planner& pl) { plan_qr(pl, A, est); });
  if (rc != HODLR_OK) return rc;
  A->planned = true;
  // process-wide unique, so a merged plan can never be taken for the plan of another matrix
  // that later lives at the same address
  static std::atomic<long> plan_serial{0};
  A->plan_version = ++plan_serial;
  A->plan_tol = tol;
  A->plan_anorm = est ? -1.0 : 1.0;
  return HODLR_OK;
}

static int qr_launch_on(hodlr_ctx* ctx, hodlr_mat* A, double tol, double anorm, cudaStream_t m, cudaStream_t sd) {
  (void)tol;
  // anorm given: set it on the device with a kernel (capturable); else the plan estimates it
  if (anorm > 0) HQ_CUDA_OK(launch_fill(A->dscal, 1, anorm, m));
  return run_plan_on(ctx, A, A->plan, nullptr, m, sd);
}

static int qr_launch(hodlr_ctx* ctx, hodlr_mat* A, double tol, double anorm) {
  return qr_launch_on(ctx, A, tol, anorm, ctx->s, ctx->side);
}

int hodlr_qr(hodlr_ctx* ctx, hodlr_mat* A, double tol, double anorm) {
  if (!ctx || !A || !(tol >= 0)) return HODLR_EINVAL;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  int rc = ensure_plan(ctx, A, tol, anorm);
  if (rc) return rc;
  rc = qr_launch(ctx, A, tol, anorm);
  if (rc) return rc;
  A->factored = true;
  return HODLR_OK;
}

int hodlr_qr_graph(hodlr_ctx* ctx, hodlr_mat* A, double tol, double anorm) {
  if (!ctx || !A || !(tol >= 0)) return HODLR_EINVAL;
  if (!A->snapshot) return HODLR_ESTATE;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  int rc = ensure_plan(ctx, A, tol, anorm);
  if (rc) return rc;
  if (!A->gexec || A->g_tol != tol || A->g_anorm != anorm || A->g_cluster != ctx->cluster * 64 + ctx->cluster_large ||
      A->g_conc != ctx->concurrency) {
    if (A->gexec) cudaGraphExecDestroy(A->gexec);
    A->gexec = nullptr;
    cudaGraph_t g;
    HQ_CUDA_OK(cudaStreamBeginCapture(ctx->s, cudaStreamCaptureModeThreadLocal));
    int r1 = hodlr_restore(ctx, A);
    int r2 = r1 ? r1 : qr_launch(ctx, A, tol, anorm);
    cudaError_t e = cudaStreamEndCapture(ctx->s, &g);
    if (r2) return r2;
    if (e != cudaSuccess) return cuda_fail(e, __FILE__, __LINE__);
    e = cudaGraphInstantiate(&A->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, __FILE__, __LINE__);
    A->g_tol = tol;
    A->g_anorm = anorm;
    A->g_cluster = ctx->cluster * 64 + ctx->cluster_large;
    A->g_conc = ctx->concurrency;
  }
  HQ_CUDA_OK(cudaGraphLaunch(A->gexec, ctx->s));
  A->factored = true;
  return HODLR_OK;
}

int hodlr_qr_profile(hodlr_ctx* ctx, hodlr_mat* A, double tol, double anorm, double* ms, int* launches,
                     double* flops) {
  if (!ctx || !A || !ms || !launches || !flops || !(tol >= 0)) return HODLR_EINVAL;
  if (!A->snapshot) return HODLR_ESTATE;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  int rc = ensure_plan(ctx, A, tol, anorm);
  if (rc) return rc;
  rc = hodlr_restore(ctx, A);
  if (rc) return rc;
  Profiler prof;
  if (anorm > 0) HQ_CUDA_OK(launch_fill(A->dscal, 1, anorm, ctx->s));
  rc = run_plan(ctx, A, A->plan, &prof);
  cudaError_t e = cudaStreamSynchronize(ctx->s);
  for (int k = 0; k < 8; ++k) {
    ms[k] = 0;
    launches[k] = 0;
    flops[k] = 0;
  }
  for (size_t i = 0; i < prof.kind.size(); ++i) {
    float t = 0;
    if (e == cudaSuccess && !rc) cudaEventElapsedTime(&t, prof.ev[2 * i], prof.ev[2 * i + 1]);
    ms[prof.kind[i]] += t;
    launches[prof.kind[i]] += 1;
  }
  for (auto ev : prof.ev) cudaEventDestroy(ev);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(e, __FILE__, __LINE__);
  double f[16];
  HQ_CUDA_OK(cudaMemcpy(f, A->dscal + 1, sizeof(double) * 16, cudaMemcpyDeviceToHost));
  for (int k = 0; k < 8 && kKindSlot + k < 16; ++k) flops[k] = f[kKindSlot + k];
  A->factored = true;
  return HODLR_OK;
}

static int ensure_pool(hodlr_ctx* ctx, int count) {
  while ((int)ctx->pool.size() < count) {
    cudaStream_t a, b;
    HQ_CUDA_OK(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
    if (cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking) != cudaSuccess) {
      cudaStreamDestroy(a);
      return HODLR_ECUDA;
    }
    ctx->pool.push_back({a, b});
  }
  return HODLR_OK;
}

}  // extern "C"

// ----------------------------------------------------------- cross-matrix batched plans
// The planner's records depend only on a matrix's partition, rank capacity and whether ||A||_2
// is estimated (ranks are data on the device), so matrices that share these have plans with the
// same records.  One merged plan replays such a group: each of its launches carries the
// descriptors of every matrix of the group (each descriptor names its own matrix's memory, rank
// table and counters), so a batch of B matrices costs the launches of one factorization.
static bool same_structure(const hodlr_mat* a, const hodlr_mat* b) {
  return a->n == b->n && a->kc == b->kc && a->leaf_sizes == b->leaf_sizes &&
         (a->plan_anorm > 0) == (b->plan_anorm > 0);
}

template <class D>
static void merge_descs(const std::vector<hodlr_mat*>& mats, size_t r, Plan& out, Rec& rr) {
  int total = 0;
  for (auto* m : mats) total += m->plan.recs[r].n;
  const size_t off = (out.blob.size() + 15) & ~size_t(15);
  out.blob.resize(off + (size_t)total * sizeof(D));
  char* dst = out.blob.data() + off;
  for (auto* m : mats) {
    const Rec& src = m->plan.recs[r];
    memcpy(dst, m->plan.blob.data() + src.off, (size_t)src.n * sizeof(D));
    dst += (size_t)src.n * sizeof(D);
  }
  rr.n = total;
  rr.off = off;
}

static int merge_plans(const std::vector<hodlr_mat*>& mats, Plan& out) {
  const Plan& P0 = mats[0]->plan;
  const size_t R = P0.recs.size();
  for (auto* m : mats)
    if (m->plan.recs.size() != R || m->plan.nevents != P0.nevents) return HODLR_EINVAL;
  out.recs.clear();
  out.blob.clear();
  out.nevents = P0.nevents;
  for (size_t r = 0; r < R; ++r) {
    Rec rr = P0.recs[r];
    for (auto* m : mats) {
      const Rec& q = m->plan.recs[r];
      if (q.type != rr.type || q.stream != rr.stream || q.i0 != rr.i0) return HODLR_EINVAL;
    }
    switch (rr.type) {
      case R_EVREC: case R_EVWAIT: break;
      case R_GEMM: {
        merge_descs<GemmDesc>(mats, r, out, rr);
        GemmDesc* g = reinterpret_cast<GemmDesc*>(out.blob.data() + rr.off);
        int work = 0;                                   // work items contiguous per descriptor
        for (int i = 0; i < rr.n; ++i) {
          g[i].work0 = work;
          work += g[i].tiles_m * g[i].tiles_n * g[i].ksplit;
        }
        break;
      }
      case R_CONCAT: merge_descs<ConcatDesc>(mats, r, out, rr); break;
      case R_GATHER: case R_SCATTER: merge_descs<PanelDesc>(mats, r, out, rr); break;
      case R_QR: merge_descs<QRDesc>(mats, r, out, rr); break;
      case R_JACOBI: merge_descs<JacobiDesc>(mats, r, out, rr); break;
      case R_SELECT: merge_descs<SelectDesc>(mats, r, out, rr); break;
      case R_COPY: merge_descs<CopyDesc>(mats, r, out, rr); break;
      case R_SMALL: case R_NORMS: merge_descs<SmallDesc>(mats, r, out, rr); break;
      default: return HODLR_EINVAL;                      // not part of a factorization plan
    }
    out.recs.push_back(rr);
  }
  return HODLR_OK;
}

// The groups of a batch, in order of first appearance: matrices of one structure, at most
// ctx->batch_group per group.  A group of one matrix runs that matrix's own plan.
static std::vector<std::vector<hodlr_mat*>> batch_groups(hodlr_ctx* ctx, int count, hodlr_mat* const* A) {
  std::vector<std::vector<hodlr_mat*>> gs;
  for (int i = 0; i < count; ++i) {
    bool placed = false;
    for (auto& g : gs) {
      if (same_structure(g[0], A[i]) && (ctx->batch_group <= 0 || (int)g.size() < ctx->batch_group)) {
        g.push_back(A[i]);
        placed = true;
        break;
      }
    }
    if (!placed) gs.push_back({A[i]});
  }
  return gs;
}

static void free_groups(hodlr_ctx* ctx) {
  for (auto* g : ctx->groups) {
    if (ctx->batch_owner) free_plan(ctx->batch_owner, g->plan);
    delete g;
  }
  ctx->groups.clear();
}

// The merged plan of group `mats`, built (or rebuilt after a member's plan changed) on demand.
static int group_plan(hodlr_ctx* ctx, const std::vector<hodlr_mat*>& mats, Plan** out) {
  std::vector<long> vers;
  for (auto* m : mats) vers.push_back(m->plan_version);
  for (auto* g : ctx->groups)
    if (g->mats == mats && g->versions == vers) {
      *out = &g->plan;
      return HODLR_OK;
    }
  if (!ctx->batch_owner) {
    ctx->batch_owner = new (std::nothrow) hodlr_mat();
    if (!ctx->batch_owner) return HODLR_ENOMEM;
    ctx->batch_owner->mem = ctx->mem;
  }
  for (size_t i = 0; i < ctx->groups.size(); ++i)
    if (ctx->groups[i]->mats == mats) {                 // stale: a member was re-planned
      free_plan(ctx->batch_owner, ctx->groups[i]->plan);
      delete ctx->groups[i];
      ctx->groups.erase(ctx->groups.begin() + i);
      break;
    }
  BatchGroup* g = new (std::nothrow) BatchGroup();
  if (!g) return HODLR_ENOMEM;
  g->mats = mats;
  g->versions = vers;
  int rc = merge_plans(mats, g->plan);
  if (!rc) rc = upload_plan(ctx->batch_owner, g->plan);
  if (rc) {
    free_plan(ctx->batch_owner, g->plan);
    delete g;
    return rc;
  }
  ctx->groups.push_back(g);
  *out = &g->plan;
  return HODLR_OK;
}

// Drop cached merged plans that the batch being recorded does not use, once there are many.
static void trim_groups(hodlr_ctx* ctx, const std::vector<std::vector<hodlr_mat*>>& keep) {
  if (ctx->groups.size() <= 64) return;
  std::vector<BatchGroup*> kept;
  for (auto* g : ctx->groups) {
    bool used = false;
    for (auto& k : keep) used = used || g->mats == k;
    if (used) {
      kept.push_back(g);
    } else {
      free_plan(ctx->batch_owner, g->plan);
      delete g;
    }
  }
  ctx->groups = kept;
}

// Queue restore (optional) + factorization of every matrix: one merged plan per group of
// matrices with the same structure, each group on its own stream pair, forked from and joined
// back into the context stream.
struct BatchSetup {
  std::vector<std::vector<hodlr_mat*>> groups;
  std::vector<Plan*> plans;
};

// Everything that allocates (merged plans and their device blobs, streams) happens here, before
// any stream capture begins.
static int batch_prepare(hodlr_ctx* ctx, int count, hodlr_mat* const* A, BatchSetup* b) {
  b->groups = batch_groups(ctx, count, A);
  trim_groups(ctx, b->groups);
  b->plans.assign(b->groups.size(), nullptr);
  for (size_t i = 0; i < b->groups.size(); ++i) {
    if (b->groups[i].size() == 1) {
      b->plans[i] = &b->groups[i][0]->plan;
    } else if (int rc = group_plan(ctx, b->groups[i], &b->plans[i])) {
      return rc;
    }
  }
  return ensure_pool(ctx, (int)b->groups.size());
}

static int batch_launch(hodlr_ctx* ctx, const BatchSetup& b, double anorm, bool restore) {
  const auto& gs = b.groups;
  const auto& plans = b.plans;
  const int count = [&] { int c = 0; for (auto& g : gs) c += (int)g.size(); return c; }();
  cudaEvent_t fork;
  HQ_CUDA_OK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  HQ_CUDA_OK(cudaEventRecord(fork, ctx->s));
  std::vector<cudaEvent_t> joins(gs.size(), nullptr);
  int rc = HODLR_OK;
  ctx->concurrent = count;
  for (size_t i = 0; i < gs.size() && !rc; ++i) {
    cudaStream_t m = ctx->pool[i].first, sd = ctx->pool[i].second;
    if (cudaStreamWaitEvent(m, fork, 0) != cudaSuccess) rc = HODLR_ECUDA;
    for (hodlr_mat* X : gs[i]) {
      if (rc) break;
      if (restore &&
          (cudaMemcpyAsync(X->store, X->snapshot, X->a_doubles * sizeof(double), cudaMemcpyDeviceToDevice, m) != cudaSuccess ||
           (X->nn && cudaMemcpyAsync(X->devints, X->snap_ints, sizeof(int) * 3 * X->nn, cudaMemcpyDeviceToDevice, m) != cudaSuccess)))
        rc = HODLR_ECUDA;
      if (!rc && anorm > 0 && launch_fill(X->dscal, 1, anorm, m) != cudaSuccess) rc = HODLR_ECUDA;
    }
    if (!rc) rc = run_plan_on(ctx, gs[i][0], *plans[i], nullptr, m, sd);
    if (!rc && (cudaEventCreateWithFlags(&joins[i], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventRecord(joins[i], m) != cudaSuccess || cudaStreamWaitEvent(ctx->s, joins[i], 0) != cudaSuccess))
      rc = HODLR_ECUDA;
  }
  ctx->concurrent = 1;
  cudaEventDestroy(fork);
  for (auto e : joins)
    if (e) cudaEventDestroy(e);
  return rc;
}

extern "C" {

int hodlr_qr_batched(hodlr_ctx* ctx, int count, hodlr_mat* const* A, double tol, double anorm) {
  if (!ctx || !A || count < 1 || !(tol >= 0)) return HODLR_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (!A[i]) return HODLR_EINVAL;
    for (int j = 0; j < i; ++j)
      if (A[j] == A[i]) return HODLR_EINVAL;
  }
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  int rc = HODLR_OK;
  for (int i = 0; i < count && !rc; ++i) rc = ensure_plan(ctx, A[i], tol, anorm);
  if (rc) return rc;
  BatchSetup b;
  rc = batch_prepare(ctx, count, A, &b);
  if (!rc) rc = batch_launch(ctx, b, anorm, false);
  if (rc) return rc;
  for (int i = 0; i < count; ++i) A[i]->factored = true;
  return HODLR_OK;
}

int hodlr_qr_batched_graph(hodlr_ctx* ctx, int count, hodlr_mat* const* A, double tol, double anorm) {
  if (!ctx || !A || count < 1 || !(tol >= 0)) return HODLR_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (!A[i]) return HODLR_EINVAL;
    if (!A[i]->snapshot) return HODLR_ESTATE;
    for (int j = 0; j < i; ++j)
      if (A[j] == A[i]) return HODLR_EINVAL;
  }
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  int rc = HODLR_OK;
  bool replan = false;
  for (int i = 0; i < count && !rc; ++i) {
    bool had = A[i]->planned && A[i]->plan_tol == tol && ((A[i]->plan_anorm > 0) == (anorm > 0));
    rc = ensure_plan(ctx, A[i], tol, anorm);
    if (!had) replan = true;
  }
  if (rc) return rc;
  std::vector<hodlr_mat*> key(A, A + count);
  if (!ctx->bgraph || replan || key != ctx->bmats || ctx->btol != tol || ctx->banorm != anorm ||
      ctx->bcluster != ctx->cluster * 64 + ctx->cluster_large || ctx->bconc != ctx->concurrency ||
      ctx->bgroup != ctx->batch_group) {
    if (ctx->bgraph) cudaGraphExecDestroy(ctx->bgraph);
    ctx->bgraph = nullptr;
    BatchSetup b;
    if (int r1 = batch_prepare(ctx, count, A, &b)) return r1;
    cudaGraph_t g;
    HQ_CUDA_OK(cudaStreamBeginCapture(ctx->s, cudaStreamCaptureModeThreadLocal));
    int r2 = batch_launch(ctx, b, anorm, true);
    cudaError_t e = cudaStreamEndCapture(ctx->s, &g);
    if (r2) return r2;
    if (e != cudaSuccess) return cuda_fail(e, __FILE__, __LINE__);
    e = cudaGraphInstantiate(&ctx->bgraph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, __FILE__, __LINE__);
    ctx->bmats = key;
    ctx->btol = tol;
    ctx->banorm = anorm;
    ctx->bcluster = ctx->cluster * 64 + ctx->cluster_large;
    ctx->bconc = ctx->concurrency;
    ctx->bgroup = ctx->batch_group;
  }
  HQ_CUDA_OK(cudaGraphLaunch(ctx->bgraph, ctx->s));
  for (int i = 0; i < count; ++i) A[i]->factored = true;
  return HODLR_OK;
}

int hodlr_autotune_batched(hodlr_ctx* ctx, int count, hodlr_mat* const* A, double tol, double anorm, int reps,
                           int* best_cluster, int* best_group, double* best_ms) {
  if (!ctx || !A || count < 1 || reps < 1) return HODLR_EINVAL;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  const int cmax = qr_max_cluster();
  std::vector<int> clusters;
  for (int c : {2, 3, 4, 8, cmax})
    if (c <= cmax && std::find(clusters.begin(), clusters.end(), c) == clusters.end()) clusters.push_back(c);
  std::vector<int> groups = {1, 4};
  const int c0 = ctx->cluster, g0 = ctx->batch_group;
  cudaEvent_t e0, e1;
  HQ_CUDA_OK(cudaEventCreate(&e0));
  HQ_CUDA_OK(cudaEventCreate(&e1));
  double best = -1.0;
  int bc = c0, bg = g0, rc = HODLR_OK;
  for (int c : clusters) {
    for (int g : groups) {
      if (g > 1 && count < 2 * g) continue;
      ctx->cluster = c;
      ctx->batch_group = g;
      rc = hodlr_qr_batched_graph(ctx, count, A, tol, anorm);     // records the graph
      if (!rc && cudaStreamSynchronize(ctx->s) != cudaSuccess) rc = HODLR_ECUDA;
      double mn = -1.0;
      for (int r = 0; r < reps && !rc; ++r) {
        cudaEventRecord(e0, ctx->s);
        rc = hodlr_qr_batched_graph(ctx, count, A, tol, anorm);
        cudaEventRecord(e1, ctx->s);
        if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = HODLR_ECUDA;
        float ms = 0.0f;
        if (!rc) cudaEventElapsedTime(&ms, e0, e1);
        if (!rc && (mn < 0 || ms < mn)) mn = ms;
      }
      if (rc) break;
      if (best < 0 || mn < best) {
        best = mn;
        bc = c;
        bg = g;
      }
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->cluster = rc ? c0 : bc;
  ctx->batch_group = rc ? g0 : bg;
  if (rc) return rc;
  if (best_cluster) *best_cluster = bc;
  if (best_group) *best_group = bg;
  if (best_ms) *best_ms = best;
  return HODLR_OK;
}

int hodlr_status(hodlr_ctx* ctx, hodlr_mat* A, int* status, double* anorm_used) {
  if (!ctx || !A) return HODLR_EINVAL;
  HQ_CUDA_OK(cudaStreamSynchronize(ctx->s));
  int st = 0;
  double an = 0;
  HQ_CUDA_OK(cudaMemcpy(&st, A->dstatus, sizeof(int), cudaMemcpyDeviceToHost));
  HQ_CUDA_OK(cudaMemcpy(&an, A->dscal, sizeof(double), cudaMemcpyDeviceToHost));
  if (status) *status = st;
  if (anorm_used) *anorm_used = an;
  return HODLR_OK;
}

int hodlr_ranks(hodlr_ctx* ctx, const hodlr_mat* A, int* r12, int* r21, int* rT) {
  if (!ctx || !A) return HODLR_EINVAL;
  HQ_CUDA_OK(cudaStreamSynchronize(ctx->s));
  if (A->nn == 0) return HODLR_OK;
  std::vector<int> h(3 * A->nn);
  HQ_CUDA_OK(cudaMemcpy(h.data(), A->devints, sizeof(int) * 3 * A->nn, cudaMemcpyDeviceToHost));
  if (r12) memcpy(r12, h.data(), sizeof(int) * A->nn);
  if (r21) memcpy(r21, h.data() + A->nn, sizeof(int) * A->nn);
  if (rT) memcpy(rT, h.data() + 2 * A->nn, sizeof(int) * A->nn);
  return HODLR_OK;
}

int hodlr_flops(hodlr_ctx* ctx, const hodlr_mat* A, double* out) {
  if (!ctx || !A || !out) return HODLR_EINVAL;
  HQ_CUDA_OK(cudaStreamSynchronize(ctx->s));
  double f[8];
  HQ_CUDA_OK(cudaMemcpy(f, A->dscal + 1, sizeof(double) * 8, cudaMemcpyDeviceToHost));
  double tot = 0;
  for (int i = 0; i < 7; ++i) {
    out[i] = f[i];
    tot += f[i];
  }
  out[7] = tot;
  return HODLR_OK;
}

}  // extern "C"

static int run_temp_plan(hodlr_ctx* ctx, hodlr_mat* A, Plan& P) {
  int rc = run_plan(ctx, A, P);
  cudaError_t e = cudaStreamSynchronize(ctx->s);
  free_plan(A, P);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(e, __FILE__, __LINE__);
  return HODLR_OK;
}

// Temporary plans share the matrix arena: they are built with measuring + real pass.
template <class F>
static int temp_plan(hodlr_ctx* ctx, hodlr_mat* A, F&& body) {
  Plan P;
  // a temporary plan must not shrink the arena the factorization plan uses; build_plan only grows it
  // but would rewrite pointers of the cached factorization plan if it reallocates: drop that plan then.
  char* before = A->arena;
  char* before2 = A->arena2;
  int rc = build_plan(A, P, ctx->cluster, 0.0, body);
  if (rc) {
    free_plan(A, P);
    return rc;
  }
  if ((A->arena != before || A->arena2 != before2) && A->planned) {
    free_plan(A, A->plan);
    A->planned = false;
    if (A->gexec) {
      cudaGraphExecDestroy(A->gexec);
      A->gexec = nullptr;
    }
  }
  return run_temp_plan(ctx, A, P);
}

extern "C" {

int hodlr_to_dense(hodlr_ctx* ctx, const hodlr_mat* Ac, int which, double* out, int ld) {
  hodlr_mat* A = const_cast<hodlr_mat*>(Ac);
  if (!ctx || !A || !out || ld < A->n || which < 0 || which > 3) return HODLR_EINVAL;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  // dense = op(part) I: use the HODLR x block product with an identity block
  return temp_plan(ctx, A, [&](Planner& pl) {
    double* I = pl.alloc<double>((size_t)A->n * A->n);
    pl.ident(I, A->n, A->n, A->n);
    View v = which == 3 ? pl.tview() : pl.aview();
    int part = which == 0 ? 0 : (which == 1 ? 1 : 2);
    pl.matvec(v, 0, part, 0, I, A->n, out, ld, A->n, -1, 1.0, 0.0, kStepNone);
  });
}

int hodlr_matvec(hodlr_ctx* ctx, const hodlr_mat* Ac, int which, int trans, int nrhs, const double* X, int ldx,
                 double* Y, int ldy) {
  hodlr_mat* A = const_cast<hodlr_mat*>(Ac);
  if (!ctx || !A || !X || !Y || nrhs <= 0 || ldx < A->n || ldy < A->n || which < 0 || which > 3)
    return HODLR_EINVAL;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  return temp_plan(ctx, A, [&](Planner& pl) {
    View v = which == 3 ? pl.tview() : pl.aview();
    int part = which == 0 ? 0 : (which == 1 ? 1 : 2);
    pl.matvec(v, 0, part, trans ? 1 : 0, X, ldx, Y, ldy, nrhs, -1, 1.0, 0.0, kStepNone);
  });
}

static void plan_apply(Planner& pl, hodlr_mat* A, int nrhs, double* B, int ldb, bool transposed_q) {
  const int n = A->n;
  double* W1 = pl.alloc<double>((size_t)n * nrhs);
  double* W2 = pl.alloc<double>((size_t)n * nrhs);
  View Y = pl.aview(), T = pl.tview();
  pl.matvec(Y, 0, 1, 1, B, ldb, W1, n, nrhs, -1, 1.0, 0.0, kStepNone);                 // Y^T B
  pl.matvec(T, 0, 2, transposed_q ? 1 : 0, W1, n, W2, n, nrhs, -1, 1.0, 0.0, kStepNone);  // T^T or T
  pl.matvec(Y, 0, 1, 0, W2, n, B, ldb, nrhs, -1, -1.0, 1.0, kStepNone);                // B -= Y W2
}

int hodlr_apply_q(hodlr_ctx* ctx, const hodlr_mat* Ac, int nrhs, double* B, int ldb) {
  hodlr_mat* A = const_cast<hodlr_mat*>(Ac);
  if (!ctx || !A || !B || nrhs <= 0 || ldb < A->n) return HODLR_EINVAL;
  if (!A->factored) return HODLR_ESTATE;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  return temp_plan(ctx, A, [&](Planner& pl) { plan_apply(pl, A, nrhs, B, ldb, false); });
}

int hodlr_apply_qt(hodlr_ctx* ctx, const hodlr_mat* Ac, int nrhs, double* B, int ldb) {
  hodlr_mat* A = const_cast<hodlr_mat*>(Ac);
  if (!ctx || !A || !B || nrhs <= 0 || ldb < A->n) return HODLR_EINVAL;
  if (!A->factored) return HODLR_ESTATE;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  return temp_plan(ctx, A, [&](Planner& pl) { plan_apply(pl, A, nrhs, B, ldb, true); });
}

static void plan_upper_solve(Planner& pl, hodlr_mat* A, int v, double* B, int ldb, int nrhs) {
  if (pl.is_leaf(v)) {
    int j = v - (A->nleaf - 1);
    Rec r = {};
    r.type = R_TRSM; r.p0 = A->D + (size_t)j * A->ldl * A->ldl; r.i0 = A->ldl; r.i1 = pl.size(v);
    r.ip = reinterpret_cast<int*>(B + A->lo[v]); r.i2 = ldb; r.i3 = nrhs;
    pl.P->recs.push_back(r);
    return;
  }
  int c1 = 2 * v + 1, c2 = 2 * v + 2;
  plan_upper_solve(pl, A, c2, B, ldb, nrhs);
  size_t mk = pl.mark();
  const int kc = A->kc;
  double* Z = pl.alloc<double>((size_t)kc * nrhs);
  int a = pl.m1(v), b = pl.m2(v);
  pl.gemm({Planner::gd(A->V12[v], b, 1, 0, B + A->lo[c2], ldb, 0, 0, Z, kc, kc, v, nrhs, -1, b, -1, 1.0, 0.0, kStepNone, -1)});
  pl.gemm({Planner::gd(A->U12[v], a, 0, 0, Z, kc, 0, 0, B + A->lo[c1], ldb, a, -1, nrhs, -1, kc, v, -1.0, 1.0, kStepNone, -1)});
  pl.release(mk);
  plan_upper_solve(pl, A, c1, B, ldb, nrhs);
}

int hodlr_solve(hodlr_ctx* ctx, const hodlr_mat* Ac, int nrhs, double* B, int ldb) {
  hodlr_mat* A = const_cast<hodlr_mat*>(Ac);
  if (!ctx || !A || !B || nrhs <= 0 || ldb < A->n) return HODLR_EINVAL;
  if (!A->factored) return HODLR_ESTATE;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  int rc = temp_plan(ctx, A, [&](Planner& pl) {
    plan_apply(pl, A, nrhs, B, ldb, true);
    plan_upper_solve(pl, A, 0, B, ldb, nrhs);
  });
  if (rc) return rc;
  int* flag = A->dstatus + 2;                      // status word 2: non-finite solution seen
  HQ_CUDA_OK(cudaMemsetAsync(flag, 0, sizeof(int), ctx->s));
  HQ_CUDA_OK(launch_check_finite(B, ldb, A->n, nrhs, flag, ctx->s));
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->s);
  if (e != cudaSuccess) return cuda_fail(e, __FILE__, __LINE__);
  return h ? HODLR_ESINGULAR : HODLR_OK;
}

int hodlr_solve_async(hodlr_ctx* ctx, hodlr_mat* A, int nrhs, double* B, int ldb) {
  if (!ctx || !A || !B || nrhs <= 0 || nrhs > 1024 || ldb < A->n) return HODLR_EINVAL;
  if (!A->factored) return HODLR_ESTATE;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  const int n = A->n;
  if (!A->splan.dblob || A->splan_nrhs < nrhs) {
    free_plan(A, A->splan);
    mat_free(A, A->sbuf);
    A->sbuf = nullptr;
    int cap = std::max(nrhs, std::max(1, A->splan_nrhs));
    if (int rc = mat_alloc(A, &A->sbuf, sizeof(double) * (size_t)n * cap)) return rc;
    int rc = build_plan(A, A->splan, ctx->cluster, 0.0, [&](Planner& pl) {
      plan_apply(pl, A, cap, A->sbuf, n, true);
      plan_upper_solve(pl, A, 0, A->sbuf, n, cap);
    }, true);
    if (rc) return rc;
    A->splan_nrhs = cap;
  }
  // stage B (unused columns are zero: they solve to zero), solve in place, copy back
  HQ_CUDA_OK(cudaMemsetAsync(A->sbuf, 0, sizeof(double) * (size_t)n * A->splan_nrhs, ctx->s));
  HQ_CUDA_OK(cudaMemcpy2DAsync(A->sbuf, sizeof(double) * n, B, sizeof(double) * ldb, sizeof(double) * n, nrhs,
                               cudaMemcpyDeviceToDevice, ctx->s));
  int rc = run_plan(ctx, A, A->splan);
  if (rc) return rc;
  HQ_CUDA_OK(cudaMemcpy2DAsync(B, sizeof(double) * ldb, A->sbuf, sizeof(double) * n, sizeof(double) * n, nrhs,
                               cudaMemcpyDeviceToDevice, ctx->s));
  return HODLR_OK;
}

int hodlr_ready(hodlr_ctx* ctx, int* ready) {
  if (!ctx || !ready) return HODLR_EINVAL;
  cudaError_t e = cudaStreamQuery(ctx->s);
  if (e == cudaSuccess) {
    *ready = 1;
    return HODLR_OK;
  }
  if (e == cudaErrorNotReady) {
    cudaGetLastError();
    *ready = 0;
    return HODLR_OK;
  }
  return cuda_fail(e, __FILE__, __LINE__);
}

int hodlr_norm2_estimate(hodlr_ctx* ctx, const hodlr_mat* Ac, int iters, double* out) {
  hodlr_mat* A = const_cast<hodlr_mat*>(Ac);
  if (!ctx || !A || !out || iters < 0) return HODLR_EINVAL;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  int rc = temp_plan(ctx, A, [&](Planner& pl) { pl.norm_estimate(iters); });
  if (rc) return rc;
  HQ_CUDA_OK(cudaMemcpy(out, A->dscal, sizeof(double), cudaMemcpyDeviceToHost));
  return HODLR_OK;
}

size_t hodlr_storage_bytes(const hodlr_mat* A) {
  if (!A) return 0;
  return A->store_doubles * sizeof(double) + sizeof(int) * 3 * A->nn;
}

int hodlr_download(hodlr_ctx* ctx, const hodlr_mat* A, void* host, size_t bytes) {
  if (!ctx || !A || !host || bytes < hodlr_storage_bytes(A)) return HODLR_EINVAL;
  HQ_CUDA_OK(cudaMemcpyAsync(host, A->store, A->store_doubles * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
  if (A->nn)
    HQ_CUDA_OK(cudaMemcpyAsync((char*)host + A->store_doubles * sizeof(double), A->devints, sizeof(int) * 3 * A->nn,
                               cudaMemcpyDeviceToHost, ctx->s));
  HQ_CUDA_OK(cudaStreamSynchronize(ctx->s));
  return HODLR_OK;
}

}  // extern "C"

// Compact layout of a factorization (hodlr_download_compact): a header of ints, then the dense
// leaves of A (Y and R) and of T, then per internal node the factors at their stored ranks.
struct CompactLayout {
  std::vector<int> ranks;                       // r12, r21, rT (3 nn)
  size_t header = 0, total = 0;                 // bytes
  std::vector<CopyDesc> copies;                 // device -> staging, dst as an offset in bytes
};

static int compact_layout(hodlr_ctx* ctx, const hodlr_mat* A, CompactLayout* L) {
  L->ranks.assign(3 * A->nn, 0);
  HQ_CUDA_OK(cudaStreamSynchronize(ctx->s));
  if (A->nn) HQ_CUDA_OK(cudaMemcpy(L->ranks.data(), A->devints, sizeof(int) * 3 * A->nn, cudaMemcpyDeviceToHost));
  L->header = ((4 + (size_t)A->nleaf + 3 * (size_t)A->nn) * sizeof(int) + 7) & ~size_t(7);
  size_t off = L->header;
  L->copies.clear();
  auto add = [&](const double* src, int lds, int rows, int cols) {
    if (rows <= 0 || cols <= 0) return;
    CopyDesc c = {};
    c.src = src; c.lds = lds; c.dst = reinterpret_cast<double*>(off); c.ldd = rows;
    c.rows = rows; c.rows_src = rows; c.rows_src_ref = -1; c.cols = cols; c.colsref = -1; c.alpha = 1.0;
    L->copies.push_back(c);
    off += (size_t)rows * cols * sizeof(double);
  };
  for (int pass = 0; pass < 2; ++pass)                      // leaves of A (Y, R), then of T
    for (int j = 0; j < A->nleaf; ++j) {
      const int w = A->leaf_sizes[j];
      add((pass ? A->TD : A->D) + (size_t)j * A->ldl * A->ldl, A->ldl, w, w);
    }
  for (int v = 0; v < A->nn; ++v) {
    const int a = A->hi[2 * v + 1] - A->lo[2 * v + 1], b = A->hi[2 * v + 2] - A->lo[2 * v + 2];
    const int r12 = L->ranks[v], r21 = L->ranks[A->nn + v], rT = L->ranks[2 * A->nn + v];
    add(A->U12[v], a, a, r12);
    add(A->V12[v], b, b, r12);
    add(A->U21[v], b, b, r21);
    add(A->V21[v], a, a, r21);
    add(A->TU[v], a, a, rT);
    add(A->TV[v], b, b, rT);
  }
  L->total = off;
  return HODLR_OK;
}

extern "C" {

int hodlr_compact_bytes(hodlr_ctx* ctx, const hodlr_mat* A, size_t* bytes) {
  if (!ctx || !A || !bytes) return HODLR_EINVAL;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  CompactLayout L;
  if (int rc = compact_layout(ctx, A, &L)) return rc;
  *bytes = L.total;
  return HODLR_OK;
}

int hodlr_download_compact(hodlr_ctx* ctx, const hodlr_mat* Ac, void* host, size_t bytes) {
  hodlr_mat* A = const_cast<hodlr_mat*>(Ac);
  if (!ctx || !A || !host) return HODLR_EINVAL;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  CompactLayout L;
  if (int rc = compact_layout(ctx, A, &L)) return rc;
  if (bytes < L.total) return HODLR_EINVAL;
  // header on the host
  int* hh = static_cast<int*>(host);
  hh[0] = A->n; hh[1] = A->nleaf; hh[2] = A->nn; hh[3] = 0;
  for (int j = 0; j < A->nleaf; ++j) hh[4 + j] = A->leaf_sizes[j];
  for (int i = 0; i < 3 * A->nn; ++i) hh[4 + A->nleaf + i] = L.ranks[i];
  // pack the blocks into a device staging buffer (descriptors after the data), one copy back
  const size_t data = L.total - L.header;
  const size_t dbytes = L.copies.size() * sizeof(CopyDesc);
  const size_t need = ((data + 255) & ~size_t(255)) + dbytes + 256;
  if (need > A->pack_bytes) {
    mat_free(A, A->pack);
    A->pack = nullptr;
    A->pack_bytes = 0;
    if (int rc = mat_alloc(A, &A->pack, need)) return rc;
    A->pack_bytes = need;
  }
  char* stage = A->pack;
  CopyDesc* dd = reinterpret_cast<CopyDesc*>(stage + ((data + 255) & ~size_t(255)));
  for (auto& c : L.copies) c.dst = reinterpret_cast<double*>(stage + (reinterpret_cast<size_t>(c.dst) - L.header));
  if (!L.copies.empty()) {
    HQ_CUDA_OK(cudaMemcpyAsync(dd, L.copies.data(), dbytes, cudaMemcpyHostToDevice, ctx->s));
    HQ_CUDA_OK(launch_copy(L.copies.data(), (int)L.copies.size(), dd, ctx->s));
    HQ_CUDA_OK(cudaMemcpyAsync(static_cast<char*>(host) + L.header, stage, data, cudaMemcpyDeviceToHost, ctx->s));
  }
  HQ_CUDA_OK(cudaStreamSynchronize(ctx->s));
  return HODLR_OK;
}

// ------------------------------------------------------------------------- primitives
int hodlr_dense_qr(hodlr_ctx* ctx, int h, int w, double* A, int lda, double* T, int ldt) {
  if (!ctx || !A || !T || h < 1 || w < 1 || w > 1024 || lda < h || ldt < std::min(h, w)) return HODLR_EINVAL;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  int k = std::min(h, w);
  double *tau, *G;
  QRDesc* dq;
  HQ_CUDA_OK(cudaMalloc(&tau, sizeof(double) * k));
  HQ_CUDA_OK(cudaMalloc(&G, sizeof(double) * k * k));
  HQ_CUDA_OK(cudaMalloc(&dq, sizeof(QRDesc)));
  QRDesc q = {};
  q.A = A; q.lda = lda; q.h = h; q.w = w; q.href = -1; q.wref = -1; q.tau = tau; q.T = T; q.ldt = ldt;
  q.G = G; q.ldg = k; q.step = kStepNone; q.fmode = 0;
  cudaError_t e = cudaMemcpyAsync(dq, &q, sizeof(QRDesc), cudaMemcpyHostToDevice, ctx->s);
  if (e == cudaSuccess) e = launch_qr(&q, 1, dq, ctx->cluster, smem_cap(ctx), ctx->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->s);
  cudaFree(tau);
  cudaFree(G);
  cudaFree(dq);
  if (e != cudaSuccess) return cuda_fail(e, __FILE__, __LINE__);
  return HODLR_OK;
}

int hodlr_truncate(hodlr_ctx* ctx, int nL, int nR, int K, const double* L, const double* Rt, double thr,
                   int kmax, double* Lout, double* Rout, int* k_out) {
  if (!ctx || nL < 1 || nR < 1 || K < 0 || K > 256 || kmax < 1 || kmax > 256 || !k_out || (K && (!L || !Rt)) ||
      !Lout || !Rout || !(thr >= 0))
    return HODLR_EINVAL;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  // a one-node shell matrix provides devints, status and arena
  hodlr_mat M;
  M.n = nL; M.nleaf = 1; M.nn = 0; M.kc = kmax; M.ldl = 1;
  M.n_devints = 64;
  M.mem = ctx->mem;
  int rc = HODLR_OK;
  if (mat_alloc(&M, &M.devints, sizeof(int) * 64) != HODLR_OK || mat_alloc(&M, &M.dstatus, sizeof(int) * 4) != HODLR_OK ||
      mat_alloc(&M, &M.dscal, sizeof(double) * 32) != HODLR_OK)
    rc = HODLR_ENOMEM;
  Plan P;
  if (!rc) {
    cudaMemsetAsync(M.devints, 0, sizeof(int) * 64, ctx->s);
    cudaMemsetAsync(M.dstatus, 0, sizeof(int) * 4, ctx->s);
    cudaMemsetAsync(M.dscal, 0, sizeof(double) * 32, ctx->s);
    rc = build_plan(&M, P, ctx->cluster, thr, [&](Planner& pl) {
      Planner::Trunc t;
      t.nL = nL; t.nR = nR;
      t.L = {Planner::seg(L, nL, K, -1, 1.0)};
      t.R = {Planner::seg(Rt, nR, K, -1, 1.0)};
      t.thr = thr; t.thr_ref = nullptr; t.Uout = Lout; t.ldu = nL; t.Vout = Rout; t.ldv = nR;
      t.kout_ref = pl.ints(1); t.step = kStepNone;
      std::vector<Planner::Trunc> ts = {t};
      if (K > 0) pl.truncate(ts);
    });
  }
  if (!rc && K > 0) rc = run_plan(ctx, &M, P);
  if (!rc) {
    cudaStreamSynchronize(ctx->s);
    int st = 0, k = 0;
    cudaMemcpy(&k, M.devints, sizeof(int), cudaMemcpyDeviceToHost);
    cudaMemcpy(&st, M.dstatus, sizeof(int), cudaMemcpyDeviceToHost);
    *k_out = K > 0 ? k : 0;
    if (cudaGetLastError() != cudaSuccess) rc = HODLR_ECUDA;
    else if (st == HODLR_ERANK) rc = HODLR_ERANK;
  }
  free_plan(&M, P);
  for (auto& kv : M.allocs) release_device(M.mem.get(), kv.first);    // tables and arenas of the shell
  if (M.mem) M.mem->used.fetch_sub(M.held);
  M.allocs.clear();
  return rc;
}


int hodlr_build_dense(hodlr_ctx* ctx, int n, int nleaf, const int* leaf_sizes, const double* A_dev, int lda,
                      double tol, int rank_cap, unsigned long long seed, hodlr_mat** out) {
  if (!ctx || !out || !A_dev || lda < n || !(tol >= 0)) return HODLR_EINVAL;
  hodlr_mat* M = nullptr;
  int rc = alloc_mat(ctx, n, nleaf, leaf_sizes, rank_cap, &M);
  if (rc) return rc;
  rc = temp_plan(ctx, M, [&](Planner& pl) { pl.compress_dense(A_dev, lda, tol, seed); });
  int st = 0;
  if (!rc) {
    if (cudaMemcpy(&st, M->dstatus, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = HODLR_ECUDA;
    else if (st == HODLR_ERANK) rc = HODLR_ERANK;
  }
  if (rc) {
    hodlr_free(M);
    return rc;
  }
  *out = M;
  return HODLR_OK;
}

int hodlr_ctx_set_memory_limit(hodlr_ctx* ctx, size_t bytes) {
  if (!ctx) return HODLR_EINVAL;
  ctx->mem->limit.store((long long)bytes);
  return HODLR_OK;
}

int hodlr_ctx_set_memory_pool(hodlr_ctx* ctx, size_t bytes) {
  if (!ctx || bytes == 0) return HODLR_EINVAL;
  if (ctx->mem->pool || ctx->mem->used.load() != 0) return HODLR_ESTATE;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  auto pool = std::make_shared<DevPool>();
  pool->size = (bytes + 255) & ~size_t(255);
  if (cudaMalloc(&pool->base, pool->size) != cudaSuccess) {
    cudaGetLastError();
    return HODLR_ENOMEM;
  }
  pool->free_[0] = pool->size;
  ctx->mem->pool = pool;
  return HODLR_OK;
}

int hodlr_ctx_share_memory(hodlr_ctx* ctx, hodlr_ctx* from) {
  if (!ctx || !from || ctx->dev != from->dev) return HODLR_EINVAL;
  if (ctx->mem->used.load() != 0) return HODLR_ESTATE;
  ctx->mem = from->mem;
  return HODLR_OK;
}

int hodlr_ctx_memory_used(hodlr_ctx* ctx, size_t* bytes) {
  if (!ctx || !bytes) return HODLR_EINVAL;
  const long long u = ctx->mem->used.load();
  *bytes = u > 0 ? (size_t)u : 0;
  return HODLR_OK;
}

int hodlr_device_bytes(const hodlr_mat* A, size_t* bytes) {
  if (!A || !bytes) return HODLR_EINVAL;
  *bytes = A->held > 0 ? (size_t)A->held : 0;
  return HODLR_OK;
}

int hodlr_footprint(int n, int nleaf, const int* leaf_sizes, int rank_cap, int estimate_norm, int with_snapshot,
                    int nrhs, size_t* bytes) {
  if (!bytes || nrhs < 0 || nrhs > 1024) return HODLR_EINVAL;
  // A host-only shell of the matrix: its pools are laid out from a fixed, never dereferenced base,
  // so the planner's measuring pass sees the same sizes as for a real matrix.
  hodlr_mat S;
  int rc = layout_mat(&S, n, nleaf, leaf_sizes, rank_cap);
  if (rc) return rc;
  static double fake[1];
  place_mat(&S, fake);
  S.devints = reinterpret_cast<int*>(fake);
  S.dscal = fake;
  S.dstatus = reinterpret_cast<int*>(fake);
  size_t total = S.store_doubles * sizeof(double) + sizeof(int) * S.n_devints + sizeof(double) * 32 + sizeof(int) * 4;
  if (with_snapshot) total += S.a_doubles * sizeof(double) + sizeof(int) * std::max(1, 3 * S.nn);
  Plan P;
  PlanSizes ps;
  rc = measure_plan(&S, P, 1.0, [&](Planner& pl) { plan_qr(pl, &S, estimate_norm != 0); }, &ps);
  if (rc) return rc;
  total += ps.arena_bytes() + ps.arena2_bytes() + (ps.counters ? ps.counter_bytes() : 0) + ps.blob_bytes();
  if (nrhs > 0) {
    // hodlr_solve_async: staging buffer, its own arenas and plan
    S.sbuf = fake;
    Plan Q;
    PlanSizes qs;
    rc = measure_plan(&S, Q, 0.0, [&](Planner& pl) {
      plan_apply(pl, &S, nrhs, S.sbuf, S.n, true);
      plan_upper_solve(pl, &S, 0, S.sbuf, S.n, nrhs);
    }, &qs);
    if (rc) return rc;
    total += sizeof(double) * (size_t)S.n * nrhs + qs.arena_bytes() + qs.arena2_bytes() +
             (qs.counters ? qs.counter_bytes() : 0) + qs.blob_bytes();
  }
  *bytes = total;
  return HODLR_OK;
}

int hodlr_stats(hodlr_ctx* ctx, const hodlr_mat* A, int* max_rank_Y, int* max_rank_T, int* max_rank_R,
                size_t* bytes) {
  if (!ctx || !A) return HODLR_EINVAL;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  HQ_CUDA_OK(cudaStreamSynchronize(ctx->s));
  std::vector<int> h(std::max(1, 3 * A->nn), 0);
  if (A->nn) HQ_CUDA_OK(cudaMemcpy(h.data(), A->devints, sizeof(int) * 3 * A->nn, cudaMemcpyDeviceToHost));
  int mr = 0, my = 0, mt = 0;
  for (int v = 0; v < A->nn; ++v) {
    mr = std::max(mr, h[v]);
    my = std::max(my, h[A->nn + v]);
    mt = std::max(mt, h[2 * A->nn + v]);
  }
  if (max_rank_R) *max_rank_R = mr;
  if (max_rank_Y) *max_rank_Y = my;
  if (max_rank_T) *max_rank_T = mt;
  if (bytes) *bytes = A->store_doubles * sizeof(double) + sizeof(int) * 3 * A->nn;
  return HODLR_OK;
}

}  // extern "C"

// ============================================= rectangular HODLR and the permuted QR (Sec. 6)
// A rectangular HODLR matrix on the device: a shell hodlr_mat owns the storage (leaves, factors
// at the rank capacity, rank table, status, scratch arenas) and the two partitions give the row
// and column range of every heap-ordered node.
struct hodlr_rect {
  hodlr_mat* S = nullptr;
  int m = 0, n = 0;
  std::vector<int> m_sizes, n_sizes;
  std::vector<std::pair<int, int>> rr, cr;
  std::vector<double*> leaf;
};

namespace {

// Node ranges of a partition (heap order), or empty when it is not a power-of-two partition of
// positive sizes.
std::vector<std::pair<int, int>> node_ranges_of(int nleaf, const int* sizes) {
  std::vector<std::pair<int, int>> r;
  if (nleaf < 1 || (nleaf & (nleaf - 1)) || !sizes) return r;
  r.assign(2 * nleaf - 1, {0, 0});
  int off = 0;
  for (int j = 0; j < nleaf; ++j) {
    if (sizes[j] < 1) return {};
    r[nleaf - 1 + j] = {off, off + sizes[j]};
    off += sizes[j];
  }
  for (int v = nleaf - 2; v >= 0; --v) r[v] = {r[2 * v + 1].first, r[2 * v + 2].second};
  return r;
}

// A shell matrix for plans that are not one square HODLR matrix: rank table (2 (nleaf - 1)
// ranks followed by the planner's integer slots), status, scalars; no storage.
int make_shell(hodlr_ctx* ctx, int n, int nleaf, int kc, hodlr_mat** out) {
  hodlr_mat* M = new (std::nothrow) hodlr_mat();
  if (!M) return HODLR_ENOMEM;
  M->mem = ctx->mem;
  M->n = n; M->nleaf = nleaf; M->nn = nleaf - 1; M->kc = kc; M->ldl = 1;
  int lv = 0;
  while ((1 << lv) < nleaf) ++lv;
  M->levels = lv;
  M->n_devints = 3 * M->nn + 16 * (2 * M->nn + 1) + 64;
  if (mat_alloc(M, &M->devints, sizeof(int) * M->n_devints) != HODLR_OK ||
      mat_alloc(M, &M->dscal, sizeof(double) * 32) != HODLR_OK || mat_alloc(M, &M->dstatus, sizeof(int) * 4) != HODLR_OK) {
    hodlr_free(M);
    return HODLR_ENOMEM;
  }
  cudaMemsetAsync(M->devints, 0, sizeof(int) * M->n_devints, ctx->s);
  cudaMemsetAsync(M->dscal, 0, sizeof(double) * 32, ctx->s);
  cudaMemsetAsync(M->dstatus, 0, sizeof(int) * 4, ctx->s);
  *out = M;
  return HODLR_OK;
}

// Row blocks of the permutation of Sec. 6: the first n_j rows of every row block j, in order,
// then the remaining rows of every block.
std::vector<Planner::RowSeg> perm_segments(int nleaf, const int* m_sizes, const int* n_sizes) {
  std::vector<Planner::RowSeg> segs;
  int src = 0, dst = 0;
  for (int j = 0; j < nleaf; ++j) {
    segs.push_back({src, dst, n_sizes[j]});
    dst += n_sizes[j];
    src += m_sizes[j];
  }
  src = 0;
  for (int j = 0; j < nleaf; ++j) {
    segs.push_back({src + n_sizes[j], dst, m_sizes[j] - n_sizes[j]});
    dst += m_sizes[j] - n_sizes[j];
    src += m_sizes[j];
  }
  return segs;
}

bool rect_args_ok(int m, int n, int nleaf, const int* m_sizes, const int* n_sizes) {
  if (m < 1 || n < 1 || nleaf < 1 || (nleaf & (nleaf - 1)) || !m_sizes || !n_sizes) return false;
  long sm = 0, sn = 0;
  for (int j = 0; j < nleaf; ++j) {
    if (n_sizes[j] < 1 || m_sizes[j] < n_sizes[j]) return false;
    sm += m_sizes[j];
    sn += n_sizes[j];
  }
  return sm == m && sn == n;
}

// Dense permuted QR on the shell S: A (m x n, lda) is copied in permuted row order to W
// (m x n, scratch of S), factored there, and written back to A in the original row order; T
// (n x n, ldt).  anorm_out (device, may be null): ||A||_2 by power iteration, taken first.
int plan_permuted_qr(hodlr_ctx* ctx, hodlr_mat* S, int m, int n, int nleaf, const int* m_sizes, const int* n_sizes,
                     double* A, int lda, double* T, int ldt, double* W, double* anorm_out, double* Ysplit,
                     double* Rsplit) {
  const auto segs = perm_segments(nleaf, m_sizes, n_sizes);
  Plan P;
  int rc = build_plan(S, P, ctx->cluster, 0.0, [&](Planner& pl) {
    if (anorm_out) pl.dense_norm2(A, lda, m, n, anorm_out, 30);
    pl.copy_rows(A, lda, W, m, n, segs, false);
    double* tau = pl.alloc<double>(n);
    pl.dense_qr(W, m, m, n, T, ldt, tau);
    if (Ysplit && Rsplit) {
      // unit lower trapezoidal Y~ and upper R~ in the permuted order, then both back to the
      // original row order (Y = P^T Y~, R = P^T [R~; 0])
      double* Yt = pl.alloc<double>((size_t)m * n);
      double* Rt = pl.alloc<double>((size_t)m * n);
      SmallDesc a = {}, b = {};
      a.kind = kSmallTri; a.p = W; a.ld = m; a.out = Yt; a.cnt = m; a.rows = m; a.cols = n; a.scale = 0;
      b = a; b.out = Rt; b.scale = 1;
      pl.rec(R_SMALL, 2, pl.put(std::vector<SmallDesc>{a, b}));
      pl.copy_rows(Yt, m, Ysplit, m, n, segs, true);
      pl.copy_rows(Rt, m, Rsplit, m, n, segs, true);
    } else {
      pl.copy_rows(W, m, A, lda, n, segs, true);
    }
  });
  if (rc) {
    free_plan(S, P);
    return rc;
  }
  return run_temp_plan(ctx, S, P);
}

int new_rect(hodlr_ctx* ctx, int m, int n, int nleaf, const int* m_sizes, const int* n_sizes, int kc, hodlr_rect** out) {
  hodlr_rect* R = new (std::nothrow) hodlr_rect();
  if (!R) return HODLR_ENOMEM;
  R->m = m; R->n = n;
  R->m_sizes.assign(m_sizes, m_sizes + nleaf);
  R->n_sizes.assign(n_sizes, n_sizes + nleaf);
  R->rr = node_ranges_of(nleaf, m_sizes);
  R->cr = node_ranges_of(nleaf, n_sizes);
  int rc = make_shell(ctx, std::max(m, n), nleaf, kc, &R->S);
  if (rc) {
    delete R;
    return rc;
  }
  hodlr_mat* S = R->S;
  S->U12.assign(S->nn, nullptr); S->V12.assign(S->nn, nullptr); S->U21.assign(S->nn, nullptr); S->V21.assign(S->nn, nullptr);
  auto fail = [&]() {
    hodlr_free(S);
    delete R;
    return HODLR_ENOMEM;
  };
  for (int j = 0; j < nleaf; ++j) {
    double* p = nullptr;
    if (mat_alloc(S, &p, sizeof(double) * (size_t)m_sizes[j] * n_sizes[j]) != HODLR_OK) return fail();
    R->leaf.push_back(p);
  }
  for (int v = 0; v < S->nn; ++v) {
    const int a = 2 * v + 1, b = 2 * v + 2;
    const size_t ma = R->rr[a].second - R->rr[a].first, mb = R->rr[b].second - R->rr[b].first;
    const size_t na = R->cr[a].second - R->cr[a].first, nb = R->cr[b].second - R->cr[b].first;
    if (mat_alloc(S, &S->U12[v], sizeof(double) * ma * kc) != HODLR_OK ||
        mat_alloc(S, &S->V12[v], sizeof(double) * nb * kc) != HODLR_OK ||
        mat_alloc(S, &S->U21[v], sizeof(double) * mb * kc) != HODLR_OK ||
        mat_alloc(S, &S->V21[v], sizeof(double) * na * kc) != HODLR_OK)
      return fail();
  }
  *out = R;
  return HODLR_OK;
}

// Compress the dense A (device, lda) into R at thr (times *thr_ref when given); HODLR_ERANK
// when a block needs more than the rank capacity.
int rect_compress_into(hodlr_ctx* ctx, hodlr_rect* R, const double* A, int lda, double thr, const double* thr_ref,
                       unsigned long long seed) {
  int rc = temp_plan(ctx, R->S, [&](Planner& pl) { pl.compress_rect(A, lda, R->rr, R->cr, R->leaf, thr, thr_ref, seed); });
  if (rc) return rc;
  int st = 0;
  if (cudaMemcpy(&st, R->S->dstatus, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return HODLR_ECUDA;
  return st == HODLR_ERANK ? HODLR_ERANK : HODLR_OK;
}

}  // namespace

extern "C" {

int hodlr_permuted_qr(hodlr_ctx* ctx, int m, int n, int nleaf, const int* m_sizes, const int* n_sizes, double* A_dev,
                      int lda, double* T_dev, int ldt) {
  if (!ctx || !A_dev || !T_dev || !rect_args_ok(m, n, nleaf, m_sizes, n_sizes) || lda < m || ldt < n)
    return HODLR_EINVAL;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  hodlr_mat* S = nullptr;
  int rc = make_shell(ctx, m, 1, 1, &S);
  if (rc) return rc;
  double* W = nullptr;
  if (mat_alloc(S, &W, sizeof(double) * (size_t)m * n) != HODLR_OK) rc = HODLR_ENOMEM;
  if (!rc) rc = plan_permuted_qr(ctx, S, m, n, nleaf, m_sizes, n_sizes, A_dev, lda, T_dev, ldt, W, nullptr, nullptr, nullptr);
  hodlr_free(S);
  return rc;
}

int hodlr_rect_compress(hodlr_ctx* ctx, int m, int n, int nleaf, const int* m_sizes, const int* n_sizes,
                        const double* A_dev, int lda, double thr, int rank_cap, unsigned long long seed, hodlr_rect** out) {
  if (!ctx || !out || !A_dev || lda < m || !(thr >= 0) || rank_cap < 1 || rank_cap > 256) return HODLR_EINVAL;
  // the compression itself needs no m_j >= n_j; it needs two power-of-two partitions
  if (m < 1 || n < 1 || nleaf < 1 || (nleaf & (nleaf - 1)) || node_ranges_of(nleaf, m_sizes).empty() ||
      node_ranges_of(nleaf, n_sizes).empty() || node_ranges_of(nleaf, m_sizes)[0].second != m ||
      node_ranges_of(nleaf, n_sizes)[0].second != n)
    return HODLR_EINVAL;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  hodlr_rect* R = nullptr;
  int rc = new_rect(ctx, m, n, nleaf, m_sizes, n_sizes, rank_cap, &R);
  if (rc) return rc;
  rc = rect_compress_into(ctx, R, A_dev, lda, thr, nullptr, seed);
  if (rc && rc != HODLR_ERANK) {
    hodlr_rect_free(R);
    return rc;
  }
  *out = R;
  return rc;
}

int hodlr_rect_qr(hodlr_ctx* ctx, int m, int n, int nleaf, const int* m_sizes, const int* n_sizes,
                  const double* A_dev, int lda, double tol, double anorm, int rank_cap, unsigned long long seed,
                  hodlr_rect** Y, hodlr_rect** T, hodlr_rect** R, double* anorm_used) {
  if (!ctx || !A_dev || !Y || !T || !R || !rect_args_ok(m, n, nleaf, m_sizes, n_sizes) || lda < m || !(tol >= 0) ||
      rank_cap < 1 || rank_cap > 256)
    return HODLR_EINVAL;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  *Y = *T = *R = nullptr;
  hodlr_mat* S = nullptr;
  int rc = make_shell(ctx, m, 1, 1, &S);
  if (rc) return rc;
  // dense factors, in the original row order, kept until the three compressions are done
  double *A = nullptr, *W = nullptr, *Td = nullptr, *Yd = nullptr, *Rd = nullptr;
  if (mat_alloc(S, &A, sizeof(double) * (size_t)m * n) != HODLR_OK || mat_alloc(S, &W, sizeof(double) * (size_t)m * n) != HODLR_OK ||
      mat_alloc(S, &Td, sizeof(double) * (size_t)n * n) != HODLR_OK || mat_alloc(S, &Yd, sizeof(double) * (size_t)m * n) != HODLR_OK ||
      mat_alloc(S, &Rd, sizeof(double) * (size_t)m * n) != HODLR_OK)
    rc = HODLR_ENOMEM;
  if (!rc && cudaMemcpy2DAsync(A, sizeof(double) * m, A_dev, sizeof(double) * lda, sizeof(double) * m, n,
                               cudaMemcpyDeviceToDevice, ctx->s) != cudaSuccess)
    rc = HODLR_ECUDA;
  double* dnorm = S->dscal;                                // [0]: ||A||_2 used for R's threshold
  if (!rc && anorm > 0 && cudaMemcpyAsync(dnorm, &anorm, sizeof(double), cudaMemcpyHostToDevice, ctx->s) != cudaSuccess)
    rc = HODLR_ECUDA;
  if (!rc)
    rc = plan_permuted_qr(ctx, S, m, n, nleaf, m_sizes, n_sizes, A, m, Td, n, W, anorm > 0 ? nullptr : dnorm, Yd, Rd);
  hodlr_rect *y = nullptr, *t = nullptr, *r = nullptr;
  int rank_rc = HODLR_OK;
  if (!rc) rc = new_rect(ctx, m, n, nleaf, m_sizes, n_sizes, rank_cap, &y);
  if (!rc) rc = new_rect(ctx, n, n, nleaf, n_sizes, n_sizes, rank_cap, &t);
  if (!rc) rc = new_rect(ctx, m, n, nleaf, m_sizes, n_sizes, rank_cap, &r);
  // thresholds as in the square case: plain tol for the scale-free Y and T, tol ||A||_2 for R
  for (int which = 0; which < 3 && !rc; ++which) {
    const int c = which == 0 ? rect_compress_into(ctx, y, Yd, m, tol, nullptr, seed)
                 : which == 1 ? rect_compress_into(ctx, t, Td, n, tol, nullptr, seed + 1)
                              : rect_compress_into(ctx, r, Rd, m, tol, dnorm, seed + 2);
    if (c == HODLR_ERANK) rank_rc = HODLR_ERANK;
    else rc = c;
  }
  double an = anorm;
  if (!rc && cudaMemcpy(&an, dnorm, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) rc = HODLR_ECUDA;
  hodlr_free(S);
  if (rc) {
    hodlr_rect_free(y);
    hodlr_rect_free(t);
    hodlr_rect_free(r);
    return rc;
  }
  if (anorm_used) *anorm_used = an;
  *Y = y; *T = t; *R = r;
  return rank_rc;
}

int hodlr_rect_permutation(int nleaf, const int* m_sizes, const int* n_sizes, int* p) {
  if (!p || nleaf < 1 || !m_sizes || !n_sizes) return HODLR_EINVAL;
  int m = 0, n = 0;
  for (int j = 0; j < nleaf; ++j) {
    m += m_sizes[j];
    n += n_sizes[j];
  }
  if (!rect_args_ok(m, n, nleaf, m_sizes, n_sizes)) return HODLR_EINVAL;
  for (const auto& g : perm_segments(nleaf, m_sizes, n_sizes))
    for (int i = 0; i < g.len; ++i) p[g.dst + i] = g.src + i;
  return HODLR_OK;
}

int hodlr_rect_to_dense(hodlr_ctx* ctx, const hodlr_rect* Rc, double* out_dev, int ld) {
  hodlr_rect* R = const_cast<hodlr_rect*>(Rc);
  if (!ctx || !R || !out_dev || ld < R->m) return HODLR_EINVAL;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  return temp_plan(ctx, R->S, [&](Planner& pl) { pl.rect_to_dense(R->rr, R->cr, R->leaf, out_dev, ld); });
}

int hodlr_rect_ranks(hodlr_ctx* ctx, const hodlr_rect* R, int* r12, int* r21) {
  if (!ctx || !R || !r12 || !r21) return HODLR_EINVAL;
  HQ_CUDA_OK(cudaSetDevice(ctx->dev));
  HQ_CUDA_OK(cudaStreamSynchronize(ctx->s));
  const int nn = R->S->nn;
  std::vector<int> h(std::max(1, 2 * nn), 0);
  if (nn) HQ_CUDA_OK(cudaMemcpy(h.data(), R->S->devints, sizeof(int) * 2 * nn, cudaMemcpyDeviceToHost));
  for (int v = 0; v < nn; ++v) {
    r12[v] = h[v];
    r21[v] = h[nn + v];
  }
  return HODLR_OK;
}

void hodlr_rect_free(hodlr_rect* R) {
  if (!R) return;
  hodlr_free(R->S);
  delete R;
}

}  // extern "C"
