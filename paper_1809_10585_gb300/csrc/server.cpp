// The continuously batched factorize/solve service behind hodlr_server_* (include/hodlr_qr.h).
// Scheduling policy: serve_sched.h.  Every slot is a library context with its own streams and a
// host worker thread that issues the slot's requests, so the work of requests admitted while
// others run overlaps on the device: issuing a factorization of thousands of launches can block
// the issuing thread until the device has drained most of them, and with one issuing thread the
// requests would run one after another.  Admission charges a request with its exact device
// footprint (hodlr_footprint: storage, plans and scratch of build + factorization + solve) plus
// its right-hand sides.  The caller's thread only submits, admits and collects (never waits for
// the device).  Host-side code only: all numerics run in the library's kernels.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/hodlr_qr.h"
#include "serve_sched.h"

namespace hq {
cudaStream_t ctx_stream(hodlr_ctx* ctx);
void* ctx_alloc(hodlr_ctx* ctx, size_t bytes);
void ctx_free(hodlr_ctx* ctx, void* p, size_t bytes);
}

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Job {
  int kind = 0;
  long long key = -1;
  // factorize requests: a copy of the matrix description (hodlr_build's arguments)
  int n = 0;
  std::vector<int> leaf_sizes, r12, r21;
  std::vector<std::vector<double>> leaves, U12, V12, U21, V21;
  double tol = 0.0;
  // right-hand sides (n x nrhs, packed) and, when done, the solution
  int nrhs = 0;
  std::vector<double> B, X;
  bool taken = false;            // the solution was handed out
  double t_submit = 0.0, t_done = 0.0;
};

}  // namespace

// One slot: a library context, its reusable right-hand-side buffer and the worker thread that
// runs the slot's requests.  Fields below `th` are guarded by hodlr_server::mu.
struct Slot {
  hodlr_ctx* ctx = nullptr;
  double* buf = nullptr;           // n x nrhs staging of right-hand sides, grown on demand
  size_t buf_doubles = 0;
  std::thread th;
  int state = 0;                   // 0 idle, 1 request assigned, 2 request finished (rc valid)
  long long id = -1;
  Job* job = nullptr;
  hodlr_mat* M = nullptr;          // solve: the resident factors; factorization: set by the worker
  int rc = 0;
};

struct hodlr_server {
  int dev = 0;
  int rank_cap = 128;
  std::vector<Slot> slots;
  hq::ServeScheduler* sched = nullptr;
  std::map<long long, Job> jobs;
  std::map<long long, hodlr_mat*> resident;     // key -> factored matrix
  // All device memory of the server (matrices, plans, scratch, right-hand sides) comes from one
  // pool reserved at creation and shared by the slots' contexts: cudaMalloc and cudaFree wait
  // for the whole device, and would serialize the requests.
  size_t budget = 0;
  std::mutex mu;                   // API calls and the workers' hand-offs
  std::condition_variable work;    // a slot was given a request, or the server is closing
  bool quit = false;
};

namespace {

void evict(hodlr_server* S, long long key) {
  auto it = S->resident.find(key);
  if (it == S->resident.end()) return;
  hodlr_free(it->second);                          // back to the pool; nothing waits
  S->resident.erase(it);
}

// Run one request on slot `slot` (the slot's worker thread, without the server lock): build and
// factor, or take the resident factors; stage the right-hand sides, solve, wait for the slot's
// stream and copy the solution back.
int run_request(hodlr_server* S, Slot& sl, Job& j, hodlr_mat** Mout) {
  hodlr_ctx* ctx = sl.ctx;
  cudaStream_t st = hq::ctx_stream(ctx);
  if (cudaSetDevice(S->dev) != cudaSuccess) return HODLR_ECUDA;
  int rc = HODLR_OK;
  hodlr_mat* M = *Mout;
  if (j.kind == 0) {
    const int nleaf = (int)j.leaf_sizes.size(), nn = nleaf - 1;
    std::vector<const double*> lv(nleaf), u12(std::max(1, nn)), v12(std::max(1, nn)), u21(std::max(1, nn)),
        v21(std::max(1, nn));
    for (int i = 0; i < nleaf; ++i) lv[i] = j.leaves[i].data();
    for (int v = 0; v < nn; ++v) {
      u12[v] = j.U12[v].empty() ? nullptr : j.U12[v].data();
      v12[v] = j.V12[v].empty() ? nullptr : j.V12[v].data();
      u21[v] = j.U21[v].empty() ? nullptr : j.U21[v].data();
      v21[v] = j.V21[v].empty() ? nullptr : j.V21[v].data();
    }
    rc = hodlr_build(ctx, j.n, nleaf, j.leaf_sizes.data(), lv.data(), u12.data(), v12.data(),
                     nn ? j.r12.data() : nullptr, u21.data(), v21.data(), nn ? j.r21.data() : nullptr,
                     S->rank_cap, &M);
    if (rc) return rc;
    *Mout = M;
    rc = hodlr_qr(ctx, M, j.tol, 0.0);
  }
  const size_t nb = (size_t)j.n * j.nrhs;
  if (!rc && sl.buf_doubles < nb) {
    // the slot's buffer grows (its old contents are not needed: the slot is idle)
    hq::ctx_free(ctx, sl.buf, sizeof(double) * sl.buf_doubles);
    sl.buf = static_cast<double*>(hq::ctx_alloc(ctx, sizeof(double) * nb));
    sl.buf_doubles = sl.buf ? nb : 0;
    if (!sl.buf) rc = HODLR_ENOMEM;
  }
  if (!rc && cudaMemcpyAsync(sl.buf, j.B.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, st) != cudaSuccess)
    rc = HODLR_ECUDA;
  if (!rc) rc = hodlr_solve_async(ctx, M, j.nrhs, sl.buf, j.n);
  if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = HODLR_ECUDA;
  if (!rc && j.kind == 0) {
    int status = 0;
    rc = hodlr_status(ctx, M, &status, nullptr);
    if (!rc && status) rc = status;
  }
  if (!rc) {
    j.X.resize(nb);
    if (cudaMemcpy(j.X.data(), sl.buf, sizeof(double) * nb, cudaMemcpyDeviceToHost) != cudaSuccess) rc = HODLR_ECUDA;
  }
  return rc;
}

void worker(hodlr_server* S, int slot) {
  Slot& sl = S->slots[slot];
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->work.wait(lk, [&] { return S->quit || sl.state == 1; });
    if (sl.state != 1) return;                    // closing, nothing assigned
    Job* j = sl.job;
    hodlr_mat* M = sl.M;
    lk.unlock();
    const int rc = run_request(S, sl, *j, &M);
    const double t = now_s();
    lk.lock();
    j->t_done = t;
    sl.M = M;
    sl.rc = rc;
    sl.state = 2;
  }
}

// Hand an admitted request to its slot's worker (server lock held).
int start(hodlr_server* S, const hq::ServeScheduler::Request& r) {
  Slot& sl = S->slots[r.slot];
  Job& j = S->jobs[r.id];
  hodlr_mat* M = nullptr;
  if (r.kind == hq::ServeScheduler::kSolve) {
    auto it = S->resident.find(r.key);
    if (it == S->resident.end()) return HODLR_ESTATE;
    M = it->second;
  }
  sl.id = r.id;
  sl.job = &j;
  sl.M = M;
  sl.rc = 0;
  sl.state = 1;
  S->work.notify_all();
  return HODLR_OK;
}

// Complete the requests the workers finished, then admit waiting ones (server lock held; never
// waits for the device).
int progress(hodlr_server* S) {
  if (cudaSetDevice(S->dev) != cudaSuccess) return HODLR_ECUDA;
  auto ev = [S](long long key) { evict(S, key); };
  for (Slot& sl : S->slots) {
    if (sl.state != 2) continue;
    const long long id = sl.id;
    Job& j = S->jobs[id];
    const hq::ServeScheduler::Request* r = S->sched->find(id);
    const int err = sl.rc;
    hodlr_mat* M = sl.M;
    sl.state = 0;
    sl.id = -1;
    sl.job = nullptr;
    sl.M = nullptr;
    // the description was uploaded; keep only the solution
    j.leaves.clear(); j.U12.clear(); j.V12.clear(); j.U21.clear(); j.V21.clear();
    j.B.clear();
    if (err) j.X.clear();
    size_t held = 0;
    if (r->kind == hq::ServeScheduler::kFactor) {
      if (!err && r->key >= 0) {
        hodlr_device_bytes(M, &held);
        S->sched->finish(id, 0, held, ev);           // may evict older factors under the key
        S->resident[r->key] = M;
      } else {
        if (M) hodlr_free(M);                         // back to the pool; the slot's stream is idle
        S->sched->finish(id, err, 0, ev);
      }
    } else {
      S->sched->finish(id, err, 0, ev);
      if (S->resident.count(j.key)) {
        hodlr_device_bytes(S->resident[j.key], &held);   // a solve plan may have grown
        S->sched->resize_resident(j.key, held);
      }
    }
  }
  S->sched->admit([S](const hq::ServeScheduler::Request& r) { return start(S, r); }, ev);
  return HODLR_OK;
}

}  // namespace

extern "C" {

int hodlr_server_create(int device, int slots, size_t hbm_budget, int rank_cap, hodlr_server** out) {
  if (!out || slots < 1 || slots > 256 || hbm_budget == 0 || rank_cap < 1 || rank_cap > 256) return HODLR_EINVAL;
  hodlr_server* S = new (std::nothrow) hodlr_server();
  if (!S) return HODLR_ENOMEM;
  S->dev = device;
  S->rank_cap = rank_cap;
  S->budget = hbm_budget;
  S->slots.resize(slots);                          // fixed from here on: workers hold references
  for (int s = 0; s < slots; ++s) {
    hodlr_ctx* c = nullptr;
    int rc = hodlr_ctx_create(device, &c);
    if (!rc) rc = hodlr_ctx_set_concurrency(c, slots);   // factorizations share the SMs
    // one pool for all slots: the budget plus an eighth for fragmentation
    if (!rc) rc = s == 0 ? hodlr_ctx_set_memory_pool(c, hbm_budget + hbm_budget / 8)
                         : hodlr_ctx_share_memory(c, S->slots[0].ctx);
    if (rc) {
      if (c) hodlr_ctx_destroy(c);
      hodlr_server_destroy(S);
      return rc;
    }
    S->slots[s].ctx = c;
  }
  S->sched = new (std::nothrow) hq::ServeScheduler(slots, hbm_budget);
  if (!S->sched) {
    hodlr_server_destroy(S);
    return HODLR_ENOMEM;
  }
  try {
    for (int s = 0; s < slots; ++s) S->slots[s].th = std::thread(worker, S, s);
  } catch (...) {
    hodlr_server_destroy(S);
    return HODLR_ENOMEM;
  }
  *out = S;
  return HODLR_OK;
}

void hodlr_server_destroy(hodlr_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->quit = true;                                // workers finish the request they hold, then stop
  }
  S->work.notify_all();
  for (Slot& sl : S->slots)
    if (sl.th.joinable()) sl.th.join();
  cudaSetDevice(S->dev);
  for (Slot& sl : S->slots) {
    if (!sl.ctx) continue;
    hodlr_sync(sl.ctx);
    if (sl.M && sl.job && sl.job->kind == 0) hodlr_free(sl.M);   // finished, never collected
  }
  for (auto& kv : S->resident) hodlr_free(kv.second);
  for (Slot& sl : S->slots)
    if (sl.ctx) hq::ctx_free(sl.ctx, sl.buf, sizeof(double) * sl.buf_doubles);
  for (Slot& sl : S->slots)
    if (sl.ctx) hodlr_ctx_destroy(sl.ctx);
  delete S->sched;
  delete S;
}

int hodlr_server_submit(hodlr_server* S, int n, int nleaf, const int* leaf_sizes, const double* const* leaves,
                        const double* const* U12, const double* const* V12, const int* r12,
                        const double* const* U21, const double* const* V21, const int* r21, double tol,
                        int nrhs, const double* B_host, int ldb, long long keep_key, long long* request) {
  if (!S) return HODLR_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  if (!S || !request || !leaves || !B_host || nrhs < 1 || nrhs > 1024 || ldb < n || !(tol >= 0) || keep_key < -1)
    return HODLR_EINVAL;
  size_t need = 0;
  if (int rc = hodlr_footprint(n, nleaf, leaf_sizes, S->rank_cap, 1, 0, nrhs, &need)) return rc;
  const int nn = nleaf - 1;
  if (nn > 0 && (!r12 || !r21)) return HODLR_EINVAL;
  Job j;
  j.kind = 0;
  j.key = keep_key;
  j.n = n;
  j.tol = tol;
  j.nrhs = nrhs;
  j.leaf_sizes.assign(leaf_sizes, leaf_sizes + nleaf);
  std::vector<int> lo(2 * nleaf - 1), hi(2 * nleaf - 1);
  int off = 0;
  for (int i = 0; i < nleaf; ++i) {
    lo[nleaf - 1 + i] = off;
    off += leaf_sizes[i];
    hi[nleaf - 1 + i] = off;
    if (!leaves[i]) return HODLR_EINVAL;
    j.leaves.emplace_back(leaves[i], leaves[i] + (size_t)leaf_sizes[i] * leaf_sizes[i]);
  }
  for (int v = nleaf - 2; v >= 0; --v) {
    lo[v] = lo[2 * v + 1];
    hi[v] = hi[2 * v + 2];
  }
  for (int v = 0; v < nn; ++v) {
    const size_t a = hi[2 * v + 1] - lo[2 * v + 1], b = hi[2 * v + 2] - lo[2 * v + 2];
    if (r12[v] < 0 || r21[v] < 0) return HODLR_EINVAL;
    auto cp = [](const double* const* arr, int v, size_t cnt, std::vector<std::vector<double>>& dst) {
      if (cnt == 0) {
        dst.emplace_back();
        return true;
      }
      if (!arr || !arr[v]) return false;
      dst.emplace_back(arr[v], arr[v] + cnt);
      return true;
    };
    if (!cp(U12, v, a * r12[v], j.U12) || !cp(V12, v, b * r12[v], j.V12) || !cp(U21, v, b * r21[v], j.U21) ||
        !cp(V21, v, a * r21[v], j.V21))
      return HODLR_EINVAL;
    j.r12.push_back(r12[v]);
    j.r21.push_back(r21[v]);
  }
  j.B.resize((size_t)n * nrhs);
  for (int c = 0; c < nrhs; ++c) memcpy(j.B.data() + (size_t)c * n, B_host + (size_t)c * ldb, sizeof(double) * n);
  j.t_submit = now_s();
  need += sizeof(double) * (size_t)n * nrhs;
  const long long id = S->sched->submit(hq::ServeScheduler::kFactor, keep_key, need);
  S->jobs[id] = std::move(j);
  *request = id;
  return progress(S);
}

int hodlr_server_submit_solve(hodlr_server* S, long long key, int nrhs, const double* B_host, int ldb,
                              long long* request) {
  if (!S) return HODLR_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  if (!S || !request || !B_host || key < 0 || nrhs < 1 || nrhs > 1024) return HODLR_EINVAL;
  // the order n comes from the resident matrix or from the waiting factorization producing it
  int n = -1;
  std::vector<int> leaf_sizes;
  for (auto& kv : S->jobs)
    if (kv.second.kind == 0 && kv.second.key == key) {
      n = kv.second.n;
      leaf_sizes = kv.second.leaf_sizes;
    }
  if (n < 0) return HODLR_ESTATE;                    // no factors under key, none coming
  if (ldb < n) return HODLR_EINVAL;
  size_t with = 0, without = 0;
  hodlr_footprint(n, (int)leaf_sizes.size(), leaf_sizes.data(), S->rank_cap, 1, 0, nrhs, &with);
  hodlr_footprint(n, (int)leaf_sizes.size(), leaf_sizes.data(), S->rank_cap, 1, 0, 0, &without);
  Job j;
  j.kind = 1;
  j.key = key;
  j.n = n;
  j.leaf_sizes = leaf_sizes;
  j.nrhs = nrhs;
  j.B.resize((size_t)n * nrhs);
  for (int c = 0; c < nrhs; ++c) memcpy(j.B.data() + (size_t)c * n, B_host + (size_t)c * ldb, sizeof(double) * n);
  j.t_submit = now_s();
  // right-hand sides plus, at most, a solve plan of this width
  const size_t need = sizeof(double) * (size_t)n * nrhs + (with - without);
  const long long id = S->sched->submit(hq::ServeScheduler::kSolve, key, need);
  S->jobs[id] = std::move(j);
  *request = id;
  return progress(S);
}

int hodlr_server_poll(hodlr_server* S, long long request, int* state, double* X_host, int ldx, double* latency_s) {
  if (!S) return HODLR_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  if (!S || !state) return HODLR_EINVAL;
  if (int rc = progress(S)) return rc;
  const hq::ServeScheduler::Request* r = S->sched->find(request);
  auto it = S->jobs.find(request);
  if (!r || it == S->jobs.end()) return HODLR_EINVAL;
  Job& j = it->second;
  if (r->state == hq::ServeScheduler::kFailed) {
    *state = -r->error;
  } else {
    *state = r->state == hq::ServeScheduler::kDone ? 2 : r->state;
  }
  if (latency_s) *latency_s = (r->state == hq::ServeScheduler::kDone || r->state == hq::ServeScheduler::kFailed)
                                  ? j.t_done - j.t_submit : now_s() - j.t_submit;
  const bool finished = r->state == hq::ServeScheduler::kDone || r->state == hq::ServeScheduler::kFailed;
  if (r->state == hq::ServeScheduler::kDone && X_host) {
    if (ldx < j.n) return HODLR_EINVAL;
    if (j.taken) return HODLR_ESTATE;              // handed out by an earlier poll
    for (int c = 0; c < j.nrhs; ++c)
      memcpy(X_host + (size_t)c * ldx, j.X.data() + (size_t)c * j.n, sizeof(double) * j.n);
  }
  // a finished request's record is released once its result was taken (or it failed), except
  // that a factorization stays known while solves may still name its key
  if (finished && (X_host || r->state == hq::ServeScheduler::kFailed)) {
    const bool keep_record = j.kind == 0 && j.key >= 0 && S->sched->is_resident(j.key);
    if (!keep_record) {
      S->sched->forget(request);
      S->jobs.erase(it);
    } else if (X_host) {
      j.taken = true;
      j.X.clear();
      j.X.shrink_to_fit();
    }
  }
  return HODLR_OK;
}

int hodlr_server_stats(hodlr_server* S, int* waiting, int* running, int* resident, size_t* bytes_used) {
  if (!S) return HODLR_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  if (!S) return HODLR_EINVAL;
  if (int rc = progress(S)) return rc;
  if (waiting) *waiting = S->sched->waiting();
  if (running) *running = S->sched->running();
  if (resident) *resident = S->sched->resident_count();
  if (bytes_used) *bytes_used = S->sched->used();
  return HODLR_OK;
}

}  // extern "C"
