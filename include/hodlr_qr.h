/*
 * hodlr_qr.h — C ABI of a GB300 (sm_103a) FP64 implementation of hQR, the recursive
 * Householder QR decomposition of HODLR matrices of Kressner & Susnjara, "Fast QR
 * decomposition of HODLR matrices" (arXiv:1809.10585).
 *
 * A = Q R with Q = I - Y T Y^T in compact WY form (Sec. 1, Eq. (9)); Y (unit lower
 * triangular), T and R (upper triangular) are HODLR matrices of the same partition as A, and
 * every block update runs in HODLR arithmetic with truncation (Alg. 2).
 *
 * Conventions for every entry point below:
 *  - All floating point data is IEEE double, column-major.
 *  - "host" pointers point to CPU memory, "dev" pointers to memory of the context's device.
 *    The caller owns every array it passes; the library owns the opaque handles.
 *  - Work is queued on the context's stream and is asynchronous unless stated otherwise;
 *    hodlr_sync() waits for it.  Calls on one context must not overlap from several threads.
 *  - Every function returns HODLR_OK (0) or one of the error codes; on an error nothing that
 *    the call would have written is guaranteed, and the handles stay valid.
 *  - HODLR partition (Sec. 2.1, Eq. (2)): n = n_1 + ... + n_{2^l}.  Cluster-tree nodes are
 *    numbered in heap order (root 0, children of v are 2v+1 and 2v+2); the internal nodes are
 *    0 .. 2^l - 2.  For an internal node v with children c1 (size m1) and c2 (size m2), the
 *    upper block is A12 = U12 V12^T (U12: m1 x r, V12: m2 x r) and the lower block is
 *    A21 = U21 V21^T (U21: m2 x r, V21: m1 x r)  (Eq. (3) with A_L = U, A_R = V^T).
 */
#ifndef HODLR_QR_H
#define HODLR_QR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HODLR_OK 0
#define HODLR_EINVAL 1     /* malformed argument (sizes, partition, rank > block size ...)  */
#define HODLR_ENOMEM 2     /* device or host allocation failed                               */
#define HODLR_ERANK 3      /* a truncated rank exceeded the rank capacity: result truncated  */
#define HODLR_ESINGULAR 4  /* zero diagonal entry of R met in a triangular solve             */
#define HODLR_ETIMEOUT 5   /* reserved for a device-side wait that gave up; no entry point
                              waits on the device today, so none returns it                  */
#define HODLR_ECUDA 6      /* a CUDA runtime call failed                                     */
#define HODLR_ESTATE 7     /* call not valid in the object's state (e.g. solve before qr)    */

typedef struct hodlr_ctx hodlr_ctx;   /* device, stream, workspace                          */
typedef struct hodlr_mat hodlr_mat;   /* device-resident HODLR matrix and, after hodlr_qr,
                                         its factors: Y and R in place of A, plus T           */

const char* hodlr_strerror(int code);

/* Context on CUDA device `device`; creates its own non-blocking stream. */
int hodlr_ctx_create(int device, hodlr_ctx** out);
void hodlr_ctx_destroy(hodlr_ctx* ctx);
/* Use `stream` (a cudaStream_t, or NULL for the context's own stream) for later work. */
int hodlr_ctx_set_stream(hodlr_ctx* ctx, void* stream);
/* Thread-block cluster size (number of CTAs, 1..16) of the Householder QR and Jacobi kernels
 * launched from this context from now on.  The default is the largest size the device can
 * co-schedule (16 on GB300).  A single factorization is fastest with the default; several
 * factorizations in flight at once (hodlr_qr_batched, concurrent contexts) reach more throughput
 * with smaller clusters, since more of them are resident on the SMs at the same time.  Results
 * depend on the size at the level of rounding only: partial sums are split over the cluster's
 * CTAs.  Graphs captured earlier are re-captured on their next call.  HODLR_EINVAL for a size
 * below 1 or above the device's maximum. */
int hodlr_ctx_set_cluster(hodlr_ctx* ctx, int cluster);
/* Cluster size for large problems: a QR whose columns fit neither the shared memory of the
 * context's cluster nor, as one 16-column panel, that of one CTA, and a Jacobi core whose
 * columns do not fit the cluster's shared memory, run on up to this many CTAs instead (so that
 * they avoid the slower global-memory forms).  0 (the default) keeps every launch at the
 * context's cluster size.  Results depend on it at the level of rounding only.  HODLR_EINVAL
 * above the device's maximum. */
int hodlr_ctx_set_cluster_large(hodlr_ctx* ctx, int cluster);
int hodlr_ctx_get_cluster(hodlr_ctx* ctx, int* cluster);
/* Number of factorizations the caller runs on the GPU at the same time through this and other
 * contexts (default 1).  Above 1, the QR and Jacobi kernels reserve less shared memory per CTA
 * (two CTAs per SM instead of one), so that CTAs of different factorizations share SMs, and run
 * QRs of up to 64 columns and Jacobi cores of up to 64 columns on one CTA (32 otherwise);
 * hodlr_qr_batched applies this by itself for the duration of a batch of two or more.  Results
 * depend on the setting at the level of rounding only (a matrix whose columns no longer fit in
 * the cluster's shared memory is factored in the global-memory form).  Graphs captured earlier
 * are re-captured on their next call.  HODLR_EINVAL for a value below 1. */
int hodlr_ctx_set_concurrency(hodlr_ctx* ctx, int factorizations);
/* Largest number of matrices of one structure that hodlr_qr_batched and hodlr_qr_batched_graph
 * factor with one merged schedule (0, the default: no limit).  Smaller groups run as several
 * schedules side by side on separate streams.  Results do not depend on it.  HODLR_EINVAL below 0. */
int hodlr_ctx_set_batch_group(hodlr_ctx* ctx, int max_matrices);
int hodlr_ctx_get_concurrency(hodlr_ctx* ctx, int* factorizations);
/* Block until all queued work on the context's stream is done. */
int hodlr_sync(hodlr_ctx* ctx);

/*
 * Device memory accounting (not in the paper; admission control for batched and served use).
 * Every device allocation the library makes for a matrix built through this context (storage,
 * rank tables, snapshot, the factorization and solve plans with their scratch arenas) is charged
 * to the context's account and released by hodlr_free.  With a limit set (bytes > 0), an
 * allocation that would take the account above it fails with HODLR_ENOMEM instead, and the call
 * that needed it (hodlr_build, hodlr_snapshot, hodlr_qr ...) returns HODLR_ENOMEM with the
 * handles still valid; a later call may succeed after memory is freed or the limit raised.
 * bytes = 0 removes the limit.  hodlr_ctx_memory_used reports the account's current total.
 */
int hodlr_ctx_set_memory_limit(hodlr_ctx* ctx, size_t bytes);
int hodlr_ctx_memory_used(hodlr_ctx* ctx, size_t* bytes);
/* Reserve `bytes` of device memory once (one cudaMalloc) as the pool of the context's account:
 * every later device allocation for matrices built through the context is carved from it on the
 * host, and hodlr_free returns it to the pool, without any CUDA call.  cudaMalloc and cudaFree
 * wait for the whole device, so a pool keeps work of other streams (other requests) running
 * while matrices come and go.  With a pool, hodlr_free does not wait for the device: free a
 * matrix only after its work has completed (hodlr_sync, hodlr_ready).  An allocation that does
 * not fit the pool fails with HODLR_ENOMEM.  HODLR_ESTATE if the context already has a pool or
 * holds memory.  The pool is released when the last context and matrix using it are gone. */
int hodlr_ctx_set_memory_pool(hodlr_ctx* ctx, size_t bytes);
/* Make `ctx` use the memory account (limit, pool) of `from` (same device; ctx must hold no
 * memory yet, else HODLR_ESTATE). */
int hodlr_ctx_share_memory(hodlr_ctx* ctx, hodlr_ctx* from);

/*
 * hodlr_build — allocate a device-resident HODLR matrix and upload it (Sec. 2.1, Eq. (3)).
 *   n, nleaf        : order, number of leaves (a power of two, >= 1).
 *   leaf_sizes      : host, nleaf entries n_j > 0 summing to n.
 *   leaves          : host, nleaf pointers; leaves[j] is n_j x n_j, leading dimension n_j.
 *   U12, V12, U21, V21 : host, nleaf-1 pointers each (NULL allowed where the rank is 0),
 *                     layouts as in the header comment, leading dimension = row count.
 *   r12, r21        : host, nleaf-1 ranks, 0 <= r <= min(m1, m2) and r <= rank_cap.
 *   rank_cap        : storage capacity per off-diagonal block (ranks of Y, T and R produced
 *                     by hodlr_qr must fit; 8 <= rank_cap <= 256).
 * Errors: HODLR_EINVAL on bad sizes or a non-finite value (NaN, infinity) in any leaf or
 * factor; HODLR_ENOMEM when an allocation fails or the context's memory limit would be
 * exceeded.  The copies complete before return.
 */
int hodlr_build(hodlr_ctx* ctx, int n, int nleaf, const int* leaf_sizes,
                const double* const* leaves,
                const double* const* U12, const double* const* V12, const int* r12,
                const double* const* U21, const double* const* V21, const int* r21,
                int rank_cap, hodlr_mat** out);
void hodlr_free(hodlr_mat* A);

/* Re-upload new values into an existing matrix of the same partition (no allocation;
 * the arguments have the meaning of hodlr_build).  Asynchronous w.r.t. the host only if the
 * host arrays are pinned. */
int hodlr_upload(hodlr_ctx* ctx, hodlr_mat* A, const double* const* leaves,
                 const double* const* U12, const double* const* V12, const int* r12,
                 const double* const* U21, const double* const* V21, const int* r21);

/* Keep a device copy of the current A (snapshot) / copy it back (restore), so that A can be
 * factored again after hodlr_qr overwrote it.  restore is a device-to-device copy. */
int hodlr_snapshot(hodlr_ctx* ctx, hodlr_mat* A);
int hodlr_restore(hodlr_ctx* ctx, hodlr_mat* A);

/*
 * hodlr_qr — hQR (Alg. 2 applied with A~ = A and void B, C): A = (I - Y T Y^T) R.
 *   tol   : truncation tolerance eps.  Truncations that carry A's scale (S~, A^12 and the
 *           HODLR update of A^22) use eps * anorm, T~12 uses eps (Alg. 2).
 *   anorm : ||A||_2 to scale thresholds; <= 0 means estimate it on the device by
 *           30 power iterations on A^T A from the normalized all-ones vector.
 * A is overwritten: its storage then holds Y (strictly lower leaves and lower blocks) and R
 * (upper leaves and upper blocks); T is stored alongside.  Asynchronous; the device-side
 * status (e.g. HODLR_ERANK) is returned by hodlr_status.
 */
int hodlr_qr(hodlr_ctx* ctx, hodlr_mat* A, double tol, double anorm);

/* Record hodlr_restore + hodlr_qr(tol, anorm) into a CUDA graph held by A (first call), and
 * launch that graph (every call).  Same results as restore followed by hodlr_qr. */
int hodlr_qr_graph(hodlr_ctx* ctx, hodlr_mat* A, double tol, double anorm);

/*
 * hodlr_qr_profile — hodlr_restore followed by hodlr_qr(tol, anorm), run eagerly with a CUDA
 * event pair around every kernel launch (needs a prior hodlr_snapshot).  For each kernel kind
 * k in 0..7 = {batched GEMM, split-K reduction, cluster Householder QR, cluster Jacobi SVD,
 * rank selection, data movement (concat/copy/gather/scatter), vector norm, other} it returns
 * the summed event time ms[k] (milliseconds), the launch count launches[k] and the
 * algorithmic FP64 flops flops[k] those launches performed (standard counts per primitive:
 * 2mnk per product, 2hk^2 - 2k^3/3 per QR plus hk^2 - k^3/3 when T is built, the R-SVD count
 * 4p^2q + 8pq^2 + 9q^3 per Jacobi core).  Synchronous; results equal those of hodlr_qr.
 */
int hodlr_qr_profile(hodlr_ctx* ctx, hodlr_mat* A, double tol, double anorm, double* ms,
                     int* launches, double* flops);

/*
 * hodlr_qr_batched — cross-matrix batching: factor `count` distinct matrices A[0..count-1]
 * (any partitions, ranks and sizes), each as hodlr_qr(tol, anorm) would up to rounding (while
 * the batch runs, the kernels take the forms of hodlr_ctx_set_concurrency(count)), concurrently
 * on the device.  Matrices with the same partition and rank capacity form a group: the recursion
 * of Alg. 2 depends only on the partition, so the group is factored by one merged schedule whose
 * every launch carries the descriptors of all its matrices (at most hodlr_ctx_set_batch_group
 * matrices per group).  Each group runs on its own pair of streams owned by the context; the
 * pairs are forked from and joined back into the context's stream, so later work on that stream
 * sees all results.  Asynchronous.  HODLR_EINVAL if a pointer repeats.
 *
 * hodlr_qr_batched_graph — the same with hodlr_restore of every matrix first (each needs a
 * snapshot), recorded once into one CUDA graph held by the context and launched on every call;
 * the graph is re-recorded when the list of matrices, tol or anorm changes.  A matrix must not
 * be freed while the context still holds a graph that names it (call with a new list first).
 * Not in the paper: it batches independent problems (no data moves between matrices).
 */
int hodlr_qr_batched(hodlr_ctx* ctx, int count, hodlr_mat* const* A, double tol, double anorm);
int hodlr_qr_batched_graph(hodlr_ctx* ctx, int count, hodlr_mat* const* A, double tol, double anorm);

/*
 * hodlr_autotune_batched — choose the launch shapes of a batch by measurement: for each cluster
 * size of the QR and Jacobi kernels in {2, 3, 4, 8, device maximum} and each batch group size in
 * {1, 4} (merged schedules, hodlr_ctx_set_batch_group), hodlr_qr_batched_graph of the given
 * matrices is recorded and timed `reps` times with CUDA events on the context's stream; the
 * fastest pair is kept on the context and returned (*best_ms: its best time per batch).  The
 * matrices need snapshots (each timed run restores them first); they end up factored.  The
 * choice depends on the workload (sizes, ranks, how many matrices) and on the GPU, and results
 * depend on it at the level of rounding only.  Synchronous.  Not in the paper.
 */
int hodlr_autotune_batched(hodlr_ctx* ctx, int count, hodlr_mat* const* A, double tol, double anorm, int reps,
                           int* best_cluster, int* best_group, double* best_ms);

/* Synchronize and return the status word of the last factorization in *status, and the
 * ||A||_2 used for the thresholds eps ||A||_2 of Alg. 2 (S~ and the update of the second block
 * column) in *anorm_used (either may be NULL).  The status is HODLR_OK, or HODLR_ERANK when a
 * truncation T_eps (Sec. 2.1.1) kept more singular values than the rank capacity. */
int hodlr_status(hodlr_ctx* ctx, hodlr_mat* A, int* status, double* anorm_used);

/* Copy the current off-diagonal ranks (the k of Eq. (3), A_off = A_L A_R with A_L of k columns)
 * to host arrays of nleaf-1 entries, heap order (any may be NULL): r12/r21 of the A/Y/R storage
 * (before hodlr_qr the ranks of A; after it, r12 those of R and r21 those of Y) and rT of T's
 * upper blocks; these are the quantities of Table 3.  Synchronous. */
int hodlr_ranks(hodlr_ctx* ctx, const hodlr_mat* A, int* r12, int* r21, int* rT);

/* Algorithmic FP64 flop counts of the last hodlr_qr, per step of the hot path, into
 * out[0..7] = {norm estimate, left-orthogonalization, leaf QR, S~, S, update, T12, total}
 * (standard counts per primitive computed from the sizes each kernel met).  Synchronous. */
int hodlr_flops(hodlr_ctx* ctx, const hodlr_mat* A, double* out);

/*
 * hodlr_build_dense — HODLR approximation of a dense n x n matrix held on the device (Sec. 2.1.1,
 * the construction of a HODLR matrix by truncated SVDs of the off-diagonal blocks).
 *   A_dev: column-major n x n FP64 device array, leading dimension lda >= n (read only, owned
 *   by the caller).  Partition and rank capacity as in hodlr_build.  Diagonal leaf blocks are
 *   copied.  Every off-diagonal block B of the cluster tree is sampled by a randomized range
 *   finder (Halko, Martinsson and Tropp 2011, Alg. 4.1) with min(rank_cap + 16, rows, cols)
 *   Gaussian columns drawn from the counter-based stream `seed`, orthonormalized by Householder
 *   QR, and the sampled block Q Q^T B is truncated to its singular triplets with sigma > tol
 *   (absolute), as T_eps does.  With at least 16 columns of oversampling beyond the kept rank
 *   the sampling error stays at the level of the first discarded singular value.
 * Synchronous.  HODLR_ERANK (nothing allocated) if a block keeps more than rank_cap terms;
 * HODLR_EINVAL for bad arguments; HODLR_ENOMEM.  The result is an ordinary matrix handle.
 */
int hodlr_build_dense(hodlr_ctx* ctx, int n, int nleaf, const int* leaf_sizes, const double* A_dev, int lda,
                      double tol, int rank_cap, unsigned long long seed, hodlr_mat** out);

/* Device bytes currently held by matrix A: its storage, tables, snapshot and plans. */
int hodlr_device_bytes(const hodlr_mat* A, size_t* bytes);

/*
 * hodlr_footprint — the device bytes that hodlr_build of a matrix with this partition
 * (n, nleaf, leaf_sizes) and rank capacity, followed by hodlr_snapshot when with_snapshot, by
 * hodlr_qr (estimate_norm: anorm <= 0, i.e. ||A||_2 estimated on the device) and, when
 * nrhs > 0, by hodlr_solve_async with nrhs right-hand sides, allocate in total.  Computed on
 * the host by the planner's measuring pass, without a device; equal to hodlr_device_bytes
 * after those calls.  The factorization's storage is O(k n log n) (Sec. 2.1) at k = rank_cap;
 * its scratch does not depend on the ranks.  HODLR_EINVAL for a bad partition or nrhs > 1024.
 */
int hodlr_footprint(int n, int nleaf, const int* leaf_sizes, int rank_cap, int estimate_norm, int with_snapshot,
                    int nrhs, size_t* bytes);

/* Largest stored rank of the lower blocks (Y's after hodlr_qr, A's before), of T and of the
 * upper blocks (R's after hodlr_qr), and the device bytes of the matrix storage (the paper's
 * Table 3 quantities).  Any pointer may be NULL.  Synchronous. */
int hodlr_stats(hodlr_ctx* ctx, const hodlr_mat* A, int* max_rank_Y, int* max_rank_T, int* max_rank_R,
                size_t* bytes);

/*
 * Dense n x n copy of a part of the stored matrix into out_dev (leading dimension ld >= n):
 * which = 0: A as stored (full), 1: Y (unit lower part), 2: R (upper part), 3: T.
 */
int hodlr_to_dense(hodlr_ctx* ctx, const hodlr_mat* A, int which, double* out_dev, int ld);

/* Y_dev = op(M) X_dev for M = part `which` (as in hodlr_to_dense), op = transpose if trans;
 * X and Y are n x nrhs (Table 1, matrix-vector multiplication, with nrhs vectors at once). */
int hodlr_matvec(hodlr_ctx* ctx, const hodlr_mat* A, int which, int trans, int nrhs,
                 const double* X_dev, int ldx, double* Y_dev, int ldy);

/* B_dev <- Q B or Q^T B with Q = I - Y T Y^T (Sec. 1), B is n x nrhs.  Needs hodlr_qr. */
int hodlr_apply_q(hodlr_ctx* ctx, const hodlr_mat* A, int nrhs, double* B_dev, int ldb);
int hodlr_apply_qt(hodlr_ctx* ctx, const hodlr_mat* A, int nrhs, double* B_dev, int ldb);

/* B_dev <- R^{-1} Q^T B: the solution of A x = b by the QR decomposition (Sec. 1: x = R^{-1}
 * Q^T b), i.e. Q^T b = b - Y T^T Y^T b followed by the HODLR back-substitution with the upper
 * triangular R (Table 1, triangular solve: x2 = R22^{-1} b2, x1 = R11^{-1} (b1 - R12 x2),
 * dense triangular solves at the leaves).  B is n x nrhs, leading dimension ldb >= n, owned by
 * the caller and overwritten.  Needs hodlr_qr.  A zero diagonal entry of R makes the result
 * non-finite; hodlr_solve then returns HODLR_ESINGULAR (synchronous). */
int hodlr_solve(hodlr_ctx* ctx, const hodlr_mat* A, int nrhs, double* B_dev, int ldb);

/*
 * hodlr_solve_async — B_dev <- R^{-1} Q^T B as hodlr_solve, queued without synchronizing and
 * without reading anything back (no HODLR_ESINGULAR detection: a zero diagonal entry of R
 * gives non-finite results).  The first call on a matrix, or a call with more right-hand sides
 * than any earlier one, plans the solve and allocates its buffers; every later call allocates
 * nothing.  Calls on one matrix must not overlap on the device.  1 <= nrhs <= 1024.
 */
int hodlr_solve_async(hodlr_ctx* ctx, hodlr_mat* A, int nrhs, double* B_dev, int ldb);

/* *ready = 1 if all work queued on the context's stream (which joins every stream the
 * context uses) has finished, else 0.  Never blocks. */
int hodlr_ready(hodlr_ctx* ctx, int* ready);

/* ||A||_2 estimate as used by hodlr_qr (power iteration, `iters` steps).  Synchronous. */
int hodlr_norm2_estimate(hodlr_ctx* ctx, const hodlr_mat* A, int iters, double* out);

/* Size in bytes of the compact device storage of A (factors, T, ranks) and a synchronous
 * copy of it into host memory (for moving a factorization off the device). */
size_t hodlr_storage_bytes(const hodlr_mat* A);
int hodlr_download(hodlr_ctx* ctx, const hodlr_mat* A, void* host, size_t bytes);

/*
 * Compact copy of a factorization (or of an unfactored matrix) into host memory, with every
 * off-diagonal factor at its stored rank instead of the rank capacity (the O(k n log n) storage
 * of Sec. 2.1 at the actual k).  hodlr_compact_bytes returns the size (synchronous: it reads
 * the ranks).  Layout, all column-major with leading dimension = rows:
 *   int header[4 + nleaf + 3 nn] = {n, nleaf, nn = nleaf - 1, 0, leaf_sizes[nleaf],
 *                                   r12[nn], r21[nn], rT[nn]}, padded to 8 bytes;
 *   the nleaf dense leaves of the A/Y/R storage (n_j x n_j each), then the nleaf leaves of T;
 *   per internal node v (heap order): U12 (m1 x r12), V12 (m2 x r12), U21 (m2 x r21),
 *   V21 (m1 x r21), TU (m1 x rT), TV (m2 x rT), where T12 = TU TV^T.
 * The blocks are packed on the device into a staging buffer held by A (allocated on the first
 * call, charged to the context's account) and copied back once.  HODLR_EINVAL if bytes is too
 * small.  Synchronous.
 */
int hodlr_compact_bytes(hodlr_ctx* ctx, const hodlr_mat* A, size_t* bytes);
int hodlr_download_compact(hodlr_ctx* ctx, const hodlr_mat* A, void* host, size_t bytes);

/*
 * Primitives of the hot path, exposed for testing kernel by kernel.
 *
 * hodlr_dense_qr — Householder QR in compact WY form of one dense h x w device matrix
 * (Alg. 1; h >= 1, 1 <= w <= 1024): on return A holds R in its upper triangle and the
 * Householder vectors (unit diagonal implied) below it, T_dev (w x w, leading dimension ldt)
 * the upper-triangular T with Q = I - Y T Y^T.  LAPACK dlarfg sign convention.  The kernel form
 * follows the context's cluster size and concurrency setting, like the factorization's QRs.
 */
int hodlr_dense_qr(hodlr_ctx* ctx, int h, int w, double* A_dev, int lda, double* T_dev, int ldt);

/*
 * hodlr_truncate — recompression T_thr of the low-rank product L Rt^T (Sec. 2.1.1):
 * L_dev (nL x K, ld nL), Rt_dev (nR x K, ld nR); keeps the singular triplets with
 * sigma > thr.  Writes Lout_dev (nL x k, ld nL, orthonormal columns) and Rout_dev
 * (nR x k, ld nR) with k <= min(K, kmax), and k to *k_out (host).  Synchronous.
 * K <= 256.  Returns HODLR_ERANK if more than kmax singular values exceed thr.
 */
int hodlr_truncate(hodlr_ctx* ctx, int nL, int nR, int K, const double* L_dev,
                   const double* Rt_dev, double thr, int kmax, double* Lout_dev,
                   double* Rout_dev, int* k_out);

/*
 * Rectangular HODLR matrices and their permuted QR (Sec. 6, Fig. 6.1-6.3).
 *
 * A rectangular HODLR matrix (m x n) has a row partition m_sizes and a column partition
 * n_sizes of equal power-of-two length nleaf; the 2 x 2 splitting of Sec. 2.1 splits rows by
 * the first and columns by the second, so leaf j is the dense m_j x n_j block and every
 * off-diagonal block of an internal node is stored as U V^T (U: rows of the first child, V:
 * columns of the second for A12, and the other way round for A21), at most rank_cap columns.
 *
 * hodlr_permuted_qr — Householder QR (Alg. 1, LAPACK sign convention, compact WY) of the dense
 *   m x n matrix A_dev (device, column-major, lda >= m; m_j >= n_j for every j) that reduces
 *   block column j to a triangle in the first n_j rows of row block j (Sec. 6: "situated on top
 *   of the dense diagonal block"; everything else of the unreduced rows becomes zero).  This is
 *   the QR of P A, where P lists the first n_j rows of every row block first, then all other
 *   rows, each group in order: on return A_dev[P^T (...)] holds LAPACK's layout of that QR, i.e.
 *   row p_i of A_dev holds row i of [R~ above the diagonal | Y~ below, unit diagonal implied],
 *   so that Y = P^T Y~, R = P^T [R~; 0] and A = (I - Y T Y^T) R.  T_dev (n x n, ldt >= n) gets
 *   the upper triangular T (zeros below the diagonal).  Panels of 64 columns by the cluster QR
 *   kernel, trailing updates and the off-diagonal blocks of T by GEMMs (Sec. 3, Eq. (10)).
 *   Scratch of m x n doubles plus n x n comes from the context's account (HODLR_ENOMEM).
 *   Synchronous.  HODLR_EINVAL on inconsistent partitions or leading dimensions.
 *
 * hodlr_rect_compress — rectangular HODLR approximation of the dense device matrix A_dev: leaves
 *   copied, every off-diagonal block by the randomized range finder and T_eps at the absolute
 *   threshold thr (Sec. 2.1.1), Gaussian sketches from `seed`.  The partitions need not satisfy
 *   m_j >= n_j.  Returns HODLR_ERANK (with *out valid, blocks truncated to rank_cap) when a
 *   block keeps more than rank_cap singular values.
 *
 * hodlr_rect_qr — the Sec. 6 factorization as the paper evaluates it (Ex. 6.1, 6.2: "a dense
 *   version of the algorithm", factors compressed afterwards into the formats of Fig. 6.3):
 *   hodlr_permuted_qr of a copy of A_dev (A_dev is not modified), then Y (m x n) and R (m x n)
 *   compressed in the rectangular format of A and T (n x n) in the square format of n_sizes.
 *   Thresholds as in hQR: tol for Y and T (scale-free), tol ||A||_2 for R; anorm > 0 is used as
 *   ||A||_2, else it is estimated by 30 power iterations on A^T A from the normalized all-ones
 *   vector (*anorm_used, may be NULL, receives the value).  Outputs three new matrices owned by
 *   the caller (hodlr_rect_free).  HODLR_ERANK (outputs valid) when a compression hit rank_cap.
 *
 * hodlr_rect_permutation — host only, no device: the row permutation of hodlr_permuted_qr,
 *   p[i] = the row of A that is row i of P A (the first n_j rows of every row block j in block
 *   order, then the remaining rows of every block), for the m = sum(m_sizes) entries of p.
 *   HODLR_EINVAL unless nleaf is a power of two and 1 <= n_j <= m_j for every j.
 *
 * hodlr_rect_to_dense — the dense m x n matrix of R into out_dev (ld >= m).  hodlr_rect_ranks —
 * the stored ranks of A12 (r12[v]) and A21 (r21[v]) for the nleaf - 1 internal nodes (heap
 * order), synchronous.  hodlr_rect_free — release a matrix (NULL is ignored).
 */
typedef struct hodlr_rect hodlr_rect;
int hodlr_permuted_qr(hodlr_ctx* ctx, int m, int n, int nleaf, const int* m_sizes, const int* n_sizes,
                      double* A_dev, int lda, double* T_dev, int ldt);
int hodlr_rect_compress(hodlr_ctx* ctx, int m, int n, int nleaf, const int* m_sizes, const int* n_sizes,
                        const double* A_dev, int lda, double thr, int rank_cap, unsigned long long seed,
                        hodlr_rect** out);
int hodlr_rect_qr(hodlr_ctx* ctx, int m, int n, int nleaf, const int* m_sizes, const int* n_sizes,
                  const double* A_dev, int lda, double tol, double anorm, int rank_cap, unsigned long long seed,
                  hodlr_rect** Y, hodlr_rect** T, hodlr_rect** R, double* anorm_used);
int hodlr_rect_permutation(int nleaf, const int* m_sizes, const int* n_sizes, int* p);
int hodlr_rect_to_dense(hodlr_ctx* ctx, const hodlr_rect* R, double* out_dev, int ld);
int hodlr_rect_ranks(hodlr_ctx* ctx, const hodlr_rect* R, int* r12, int* r21);
void hodlr_rect_free(hodlr_rect* R);

/*
 * hodlr_dense_qr_noalloc — the same compact-WY Householder QR as hodlr_dense_qr, for callers
 * that must not allocate device memory: cudaMalloc and cudaFree synchronize the whole device
 * and can stall unrelated streams, and some callers (latency-critical loops, services that
 * reserve all their memory at start-up, hosts that route every allocation through their own
 * pool) forbid allocation after initialization.  The paper has no counterpart: this is a
 * deployment variant of one kernel of the hot path.
 *
 * It calls no cudaMalloc, cudaFree or allocating library routine.  Its scratch (the launch
 * descriptor, tau and the G = Y^T Y work area) lives in one static device array of about
 * 0.5 MiB that every GPU loading this library holds until the process exits.  Limits:
 * min(h, w) <= 256 and, as for hodlr_dense_qr, w <= 1024 (HODLR_EINVAL beyond them, with
 * nothing written); other arguments as in hodlr_dense_qr.  The call makes the context's device
 * current (A_dev and T_dev must live there).  The first call on a device looks up the array's
 * device address on that device; make that first call before any stream capture.  The address
 * table is safe to fill from several host threads at once.  All calls share the one array and
 * it keeps the last call's contents (every entry is written before it is read, so nothing needs
 * clearing); calls that overlap on the GPU, e.g. from two contexts, streams or host threads,
 * race on it.  Synchronous.
 */
int hodlr_dense_qr_noalloc(hodlr_ctx* ctx, int h, int w, double* A_dev, int lda, double* T_dev,
                           int ldt);

/*
 * Continuously batched factorize/solve service (the serving workload of the benchmark; the
 * paper has no service).  A server owns `slots` contexts on device `device`; every admitted
 * request runs in a slot of its own, so requests that arrive while others are on the GPU start
 * as soon as a slot and memory free up and their work overlaps on the device.
 *   hbm_budget : device bytes that running requests and resident factors may hold.  A request
 *                is charged its exact footprint (hodlr_footprint of build + factorization +
 *                solve, plus its right-hand sides); least recently used resident factors that
 *                no running request uses are evicted to make room; a request that cannot fit
 *                even with nothing else on the device fails with HODLR_ENOMEM.
 *   rank_cap   : rank capacity of every factorization (as in hodlr_build).
 * Order: first come, first served, except that a solve whose factors are not ready (still being
 * factored, busy with another request, or about to be replaced) lets later requests pass.
 * Requests are progressed by every call on the server (submit, poll, stats), none of which waits
 * for the device: every slot has a host worker thread that issues its request (upload, build,
 * factorization, solve, copy of the solution back), so the device work of requests in
 * different slots overlaps even though issuing one factorization's launches can block its
 * issuing thread.  All device memory of the server comes from one pool of
 * hbm_budget + hbm_budget / 8 bytes reserved at creation (hodlr_ctx_set_memory_pool), so
 * requests that come and go never wait for the device.  Calls on one server from several
 * threads are serialized by the server; hodlr_server_destroy must not overlap any other call,
 * and waits for the requests on the device to finish.
 */
typedef struct hodlr_server hodlr_server;
int hodlr_server_create(int device, int slots, size_t hbm_budget, int rank_cap, hodlr_server** out);
void hodlr_server_destroy(hodlr_server* S);
/* Factorize + solve: A described as for hodlr_build (host arrays, copied by the call), hQR with
 * truncation tolerance tol and ||A||_2 estimated on the device (Alg. 2), then x = R^{-1} Q^T b
 * for nrhs right-hand sides B_host (n x nrhs, leading dimension ldb >= n, copied; 1..1024).
 * keep_key >= 0 keeps the factors resident under that key for hodlr_server_submit_solve
 * (replacing older factors under the same key); -1 frees them after the solve.  *request is
 * the request's id.  HODLR_EINVAL for a bad partition or arguments. */
int hodlr_server_submit(hodlr_server* S, int n, int nleaf, const int* leaf_sizes, const double* const* leaves,
                        const double* const* U12, const double* const* V12, const int* r12,
                        const double* const* U21, const double* const* V21, const int* r21, double tol,
                        int nrhs, const double* B_host, int ldb, long long keep_key, long long* request);
/* Solve with the resident factors under `key` (Sec. 1: x = R^{-1} Q^T b), nrhs right-hand sides
 * (copied).  HODLR_ESTATE if no factorization was ever submitted under the key. */
int hodlr_server_submit_solve(hodlr_server* S, long long key, int nrhs, const double* B_host, int ldb,
                              long long* request);
/* Progress the server without blocking and report request `request`: *state = 0 waiting,
 * 1 on the GPU, 2 done, or -code when it failed (HODLR_ENOMEM: can never fit the budget,
 * HODLR_ESTATE: its factors will never exist, HODLR_ERANK: rank capacity exceeded ...).
 * *latency_s (may be NULL) is the time from submission to completion (to now while pending).
 * When the request is done and X_host is not NULL, the solution (n x nrhs, leading dimension
 * ldx >= n) is copied there and the request's record is released (HODLR_ESTATE if it was
 * already taken); a failed request's record is released when reported. */
int hodlr_server_poll(hodlr_server* S, long long request, int* state, double* X_host, int ldx, double* latency_s);
/* Progress the server, then report the waiting and running requests, resident factorizations
 * and the bytes charged against the budget (any pointer may be NULL). */
int hodlr_server_stats(hodlr_server* S, int* waiting, int* running, int* resident, size_t* bytes_used);

/*
 * hodlr_fp64_peak — measured FP64 throughput of device `device`, the roofline denominator for
 * the kernels above (they are bound by FP64 arithmetic).  Not part of the paper's method: a
 * measurement utility.  Two paths are timed with CUDA events, best of `reps` launches after one
 * warm-up launch, on a grid of 4 CTAs of 256 threads per SM:
 *   dfma_tflops : fused multiply-add (8 independent chains per thread, 2 flops each);
 *   dmma_tflops : the FP64 tensor-core instruction mma.sync.m8n8k4.f64 (512 flops each).
 * `iters` sets the launch length (128 iterations of 16 x 8 operations per thread each).
 * Allocates a few bytes and a stream, synchronous.  HODLR_EINVAL on bad arguments.
 */
int hodlr_fp64_peak(int device, int iters, int reps, double* dfma_tflops, double* dmma_tflops);

#ifdef __cplusplus
}
#endif

#endif /* HODLR_QR_H */
