// serve.cu -- the request server of include/faco_serve.h: admission by a
// device-memory pool, per-request set-up on a side stream, continuous
// iteration rounds (the batch launches of multi.h), results to pinned host
// memory.  Active requests are grouped into cohorts by roulette width and
// size; each cohort iterates in rounds of its own on a stream of its own,
// so a small request is not held to the pace of a large one and the
// cohorts' kernels share the GPU.  The scheduler is a host thread; every
// step of the method runs in the library's kernels.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "faco_serve.h"
#include "multi.h"

using namespace faco;

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// First-fit allocator over one device block, 256-byte granules; freed
// ranges merge with their free neighbours.
class Pool {
 public:
  void init(char* b, size_t n) {
    base_ = b;
    size_ = n & ~(size_t)255;
    free_.clear();
    if (size_) free_[0] = size_;
    in_use_ = 0;
  }
  char* get(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, len = it->second;
      free_.erase(it);
      if (len > bytes) free_[off + bytes] = len - bytes;
      in_use_ += bytes;
      return base_ + off;
    }
    return nullptr;
  }
  void put(char* p, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    size_t off = (size_t)(p - base_);
    in_use_ -= bytes;
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
  size_t size() const { return size_; }
  size_t in_use() const { return in_use_; }

 private:
  char* base_ = nullptr;
  size_t size_ = 0, in_use_ = 0;
  std::map<size_t, size_t> free_;  // offset -> length
};

enum class St { Queued, SettingUp, Active, Finishing, Done };

struct Request {
  uint64_t id = 0;
  int n = 0, k = 0, ants = 0, budget = 0;
  uint64_t seed = 0;
  std::vector<int32_t> coords;
  int64_t t_submit = 0, t_done = 0;
  St st = St::Queued;
  int status = FACO_PENDING;
  Group g;
  AntSet a;
  char* block = nullptr;
  size_t bytes = 0;
  int iters = 0, variant = kVarArr8, cohort = 0;
  cudaEvent_t ev = nullptr;  // set-up complete, later: result copied
  char* pinned = nullptr;    // tour (n int32), length (int64), error flags (int32)
  std::vector<int32_t> tour;
  int64_t length = 0;
};

// Host-side shape of a request: its colony group and ant buffers.
int plan_request(Request& r, const faco_params& prm, size_t smem_blk) {
  faco_params p = prm;
  p.seed = r.seed;
  int rc = group_init(r.g, &r.n, 1, r.k, p, nullptr);
  if (rc != FACO_OK) return rc;
  antset_layout(r.a, r.g, r.ants, smem_blk, prm.seg_cap, nullptr);
  r.bytes = ((r.g.bytes + 255) & ~(size_t)255) + r.a.bytes;
  return FACO_OK;
}

}  // namespace

// Cohorts: roulette width (16, 32) x size (n <= 4096, <= 32768, larger).
constexpr int kSizeBuckets = 3;
constexpr int kCohorts = 2 * kSizeBuckets;

struct faco_server {
  faco_params prm{};
  int device = 0;
  size_t smem_blk[2] = {0, 0};  // roulette width 16, 32
  cudaStream_t setup = nullptr;
  cudaStream_t lane[kCohorts] = {};  // each cohort's rounds and result copies
  char* pool_mem = nullptr;
  Pool pool;
  std::mutex mu;
  std::condition_variable cv;
  std::thread thr;
  bool stop = false;
  uint64_t next_id = 1;
  std::map<uint64_t, std::unique_ptr<Request>> reqs;
  std::deque<Request*> queue;
  // owned by the scheduler thread
  std::vector<Request*> setting, active[kCohorts], finishing;
  Runner runner[kCohorts];
  bool dirty[kCohorts] = {true, true, true, true, true, true};
  cudaEvent_t round_ev[kCohorts][2] = {};
  bool round_pending[kCohorts][2] = {};
  int round_par[kCohorts] = {};
  faco_server_stats stats{};
};

namespace {

#define CKS(expr)                                                          \
  do {                                                                     \
    cudaError_t e_ = (expr);                                               \
    if (e_ != cudaSuccess) {                                               \
      (void)cudaGetLastError();                                            \
      return e_ == cudaErrorMemoryAllocation ? FACO_E_NOMEM : FACO_E_CUDA; \
    }                                                                      \
  } while (0)

int wslot(const Request* r) { return r->g.kw == 32 ? 1 : 0; }

int cohort_of(const Request* r) {
  const int b = r->n <= 4096 ? 0 : (r->n <= 32768 ? 1 : 2);
  return wslot(r) * kSizeBuckets + b;
}

// Marks r done with `status` and returns its memory (scheduler thread).
void finish(faco_server* s, Request* r, int status) {
  if (r->ev) cudaEventDestroy(r->ev);
  r->ev = nullptr;
  if (r->pinned) cudaFreeHost(r->pinned);
  r->pinned = nullptr;
  std::lock_guard<std::mutex> lk(s->mu);
  if (r->block) s->pool.put(r->block, r->bytes);
  r->block = nullptr;
  r->status = status;
  r->t_done = now_ns();
  r->st = St::Done;
  r->coords.clear();
  r->coords.shrink_to_fit();
  s->stats.completed++;
  s->cv.notify_all();
}

int start_setup(faco_server* s, Request* r) {
  r->cohort = cohort_of(r);
  char* base = r->block;
  group_layout(r->g, base);
  const size_t gb = (r->g.bytes + 255) & ~(size_t)255;
  antset_layout(r->a, r->g, r->ants, s->smem_blk[wslot(r)], s->prm.seg_cap, base + gb);
  CKS(cudaHostAlloc(reinterpret_cast<void**>(&r->pinned), sizeof(int32_t) * (size_t)r->n + 16,
                    cudaHostAllocDefault));
  CKS(cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming));
  const int32_t* xy = r->coords.data();
  int rc = group_setup(r->g, &xy, s->setup);
  if (rc != FACO_OK) return rc;
  rc = antset_zero(r->a, s->setup);
  if (rc != FACO_OK) return rc;
  s->stats.kernel_launches += 15;
  CKS(cudaEventRecord(r->ev, s->setup));
  return FACO_OK;
}

std::vector<RunEntry> entries(const std::vector<Request*>& list) {
  std::vector<RunEntry> e;
  e.reserve(list.size());
  for (Request* r : list) e.push_back(RunEntry{&r->g, 0, &r->a, r->variant});
  return e;
}

// The kernel of a request whose set-up is complete (tuned once per size
// class and ant count for the request's own latency, then cached).
int choose_variant(faco_server* s, Request* r) {
  const int cls = size_class(r->n);
  int v = tuner_get(cls, r->ants, r->g.kw, kTuneLatency);
  if (v < 0) {
    std::vector<RunEntry> e{RunEntry{&r->g, 0, &r->a, kVarArr8}};
    cudaStream_t st = s->lane[r->cohort];
    int rc = tuner_run(e, s->smem_blk[wslot(r)], st, kTuneLatency);
    if (rc != FACO_OK) return rc;
    rc = antset_zero(r->a, st);  // counters of the trial launches
    if (rc != FACO_OK) return rc;
    v = tuner_get(cls, r->ants, r->g.kw, kTuneLatency);
  }
  if (v < 0 || (v == kVarTable && r->a.cap[0] <= 0)) v = kVarArr8;
  r->variant = v;
  return FACO_OK;
}

int enqueue_result_copy(faco_server* s, Request* r) {
  const Colony& C = r->g.hC[0];
  cudaStream_t st = s->lane[r->cohort];
  CKS(cudaMemcpyAsync(r->pinned, C.gb_route, sizeof(int32_t) * (size_t)r->n, cudaMemcpyDeviceToHost, st));
  char* tail = r->pinned + sizeof(int32_t) * (size_t)r->n;
  CKS(cudaMemcpyAsync(tail, reinterpret_cast<char*>(C.st) + offsetof(DevState, gb_len), sizeof(int64_t),
                      cudaMemcpyDeviceToHost, st));
  CKS(cudaMemcpyAsync(tail + 8, reinterpret_cast<char*>(C.st) + offsetof(DevState, error), sizeof(int32_t),
                      cudaMemcpyDeviceToHost, st));
  CKS(cudaEventRecord(r->ev, st));
  return FACO_OK;
}

// One iteration of every active request of each cohort that has fewer than
// two rounds in flight; requests whose budget is spent leave with their
// result copy in flight.  *queued: some cohort got a round.
int run_rounds(faco_server* s, bool* queued) {
  int64_t nact = 0;
  for (int c = 0; c < kCohorts; ++c) nact += (int64_t)s->active[c].size();
  if (nact > s->stats.peak_active) s->stats.peak_active = nact;
  for (int c = 0; c < kCohorts; ++c) {
    std::vector<Request*>& act = s->active[c];
    if (act.empty()) continue;
    // the cohort's round before last must be done before another is queued:
    // the host stays at most one round ahead of the GPU
    const int p = s->round_par[c];
    if (s->round_pending[c][p]) {
      const cudaError_t q = cudaEventQuery(s->round_ev[c][p]);
      if (q == cudaErrorNotReady) continue;
      CKS(q);
      s->round_pending[c][p] = false;
    }
    *queued = true;
    cudaStream_t st = s->lane[c];
    if (s->dirty[c]) {
      int rc = s->runner[c].build(entries(act), s->smem_blk[c / kSizeBuckets], st);
      if (rc != FACO_OK) return rc;
      s->dirty[c] = false;
    }
    int rc = s->runner[c].enqueue(st, 3);
    if (rc != FACO_OK) return rc;
    s->stats.kernel_launches += s->runner[c].kernels_per_iteration();
    s->stats.rounds++;
    std::vector<Request*> keep;
    for (Request* r : act) {
      if (++r->iters < r->budget) {
        keep.push_back(r);
        continue;
      }
      rc = enqueue_result_copy(s, r);
      if (rc != FACO_OK) return rc;
      r->st = St::Finishing;
      s->finishing.push_back(r);
      s->dirty[c] = true;
    }
    act.swap(keep);
    CKS(cudaEventRecord(s->round_ev[c][p], st));
    s->round_pending[c][p] = true;
    s->round_par[c] = p ^ 1;
  }
  return FACO_OK;
}

void fail_all(faco_server* s, int status) {
  std::vector<Request*> all;
  for (Request* r : s->setting) all.push_back(r);
  for (int c = 0; c < kCohorts; ++c)
    for (Request* r : s->active[c]) all.push_back(r);
  for (Request* r : s->finishing) all.push_back(r);
  s->setting.clear();
  for (int c = 0; c < kCohorts; ++c) {
    s->active[c].clear();
    s->dirty[c] = true;
    s->round_pending[c][0] = s->round_pending[c][1] = false;
  }
  s->finishing.clear();
  for (int c = 0; c < kCohorts; ++c) cudaStreamSynchronize(s->lane[c]);
  cudaStreamSynchronize(s->setup);
  (void)cudaGetLastError();
  for (Request* r : all) finish(s, r, status);
}

void scheduler(faco_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<Request*> admit;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      bool busy = !s->setting.empty() || !s->finishing.empty();
      for (int c = 0; c < kCohorts; ++c) busy = busy || !s->active[c].empty();
      if (!busy && s->queue.empty()) {
        if (s->stop) break;
        s->cv.wait_for(lk, std::chrono::milliseconds(5));
        continue;
      }
      while (!s->queue.empty()) {  // arrival order; the head waits for memory
        Request* r = s->queue.front();
        char* blk = s->pool.get(r->bytes);
        if (!blk) break;
        r->block = blk;
        r->st = St::SettingUp;
        s->queue.pop_front();
        admit.push_back(r);
      }
    }
    for (Request* r : admit) {
      const int rc = start_setup(s, r);
      if (rc != FACO_OK)
        finish(s, r, rc);
      else
        s->setting.push_back(r);
    }
    // set-up complete: the request joins the next round
    for (size_t i = 0; i < s->setting.size();) {
      Request* r = s->setting[i];
      const cudaError_t q = cudaEventQuery(r->ev);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      s->setting.erase(s->setting.begin() + (long)i);
      int rc = q == cudaSuccess ? choose_variant(s, r) : FACO_E_CUDA;
      (void)cudaGetLastError();
      if (rc != FACO_OK) {
        finish(s, r, rc);
        continue;
      }
      r->st = St::Active;
      s->active[r->cohort].push_back(r);
      s->dirty[r->cohort] = true;
    }
    bool queued = false;
    const int rc = run_rounds(s, &queued);
    if (rc != FACO_OK) {
      fail_all(s, rc);
      continue;
    }
    for (size_t i = 0; i < s->finishing.size();) {
      Request* r = s->finishing[i];
      const cudaError_t q = cudaEventQuery(r->ev);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      s->finishing.erase(s->finishing.begin() + (long)i);
      int st = FACO_E_CUDA;
      if (q == cudaSuccess) {
        const char* tail = r->pinned + sizeof(int32_t) * (size_t)r->n;
        int32_t err = 0;
        std::memcpy(&r->length, tail, sizeof(int64_t));
        std::memcpy(&err, tail + 8, sizeof(int32_t));
        r->tour.assign(reinterpret_cast<const int32_t*>(r->pinned),
                       reinterpret_cast<const int32_t*>(r->pinned) + r->n);
        st = err & kErrTimeout ? FACO_E_TIMEOUT : (err & kErrCapacity ? FACO_E_CAPACITY : (err ? FACO_E_CUDA : FACO_OK));
      }
      (void)cudaGetLastError();
      finish(s, r, st);
    }
    // nothing queued this pass (every cohort two rounds ahead, or only
    // set-ups and result copies in flight): let the GPU catch up
    if (!queued) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

}  // namespace

extern "C" {

int64_t faco_server_request_bytes(int32_t n, int32_t k, int32_t ants, const faco_params* p) {
  faco_params prm;
  faco_params_default(&prm);
  if (p) prm = *p;
  if (ants < 1) return -1;
  Request r;
  r.n = n;
  r.k = k;
  r.ants = ants;
  r.seed = prm.seed;
  const int kk = k < n - 1 ? k : n - 1;
  const size_t smem = batch_smem_blk(kk <= 16 ? 16 : 32);
  if (plan_request(r, prm, smem) != FACO_OK) return -1;
  return (int64_t)r.bytes;
}

int faco_server_create(size_t device_bytes, const faco_params* p, faco_server** out) {
  if (!out || device_bytes < 4096) return FACO_E_ARG;
  faco_params prm;
  faco_params_default(&prm);
  if (p) prm = *p;
  int rc = check_faco_params(prm);
  if (rc != FACO_OK) return rc;
  if (prm.keep_ant_tours || prm.keep_pre_ls || prm.seg_cap > 0) return FACO_E_ARG;
  prm.stream = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    (void)cudaGetLastError();
    return FACO_E_CUDA;
  }
  faco_server* s = new (std::nothrow) faco_server();
  if (!s) return FACO_E_NOMEM;
  s->prm = prm;
  rc = [&]() -> int {
    CKS(cudaGetDevice(&s->device));
    s->smem_blk[0] = batch_smem_blk(16);
    s->smem_blk[1] = batch_smem_blk(32);
    CKS(cudaStreamCreateWithFlags(&s->setup, cudaStreamNonBlocking));
    for (int c = 0; c < kCohorts; ++c) {
      CKS(cudaStreamCreateWithFlags(&s->lane[c], cudaStreamNonBlocking));
      CKS(cudaEventCreateWithFlags(&s->round_ev[c][0], cudaEventDisableTiming));
      CKS(cudaEventCreateWithFlags(&s->round_ev[c][1], cudaEventDisableTiming));
    }
    CKS(cudaMalloc(&s->pool_mem, device_bytes));
    s->pool.init(s->pool_mem, device_bytes);
    s->stats.pool_bytes = (int64_t)s->pool.size();
    return FACO_OK;
  }();
  if (rc != FACO_OK) {
    if (s->pool_mem) cudaFree(s->pool_mem);
    for (int c = 0; c < kCohorts; ++c) {
      for (cudaEvent_t e : s->round_ev[c])
        if (e) cudaEventDestroy(e);
      if (s->lane[c]) cudaStreamDestroy(s->lane[c]);
    }
    if (s->setup) cudaStreamDestroy(s->setup);
    delete s;
    return rc;
  }
  s->thr = std::thread(scheduler, s);
  *out = s;
  return FACO_OK;
}

int faco_server_submit(faco_server* s, const int32_t* coords_xy, int32_t n, int32_t k, int32_t ants,
                       int32_t budget, uint64_t seed, uint64_t* ticket) {
  if (!s || !coords_xy || !ticket || n < 3 || k < 2 || k > kMaxK || ants < 1 || budget < 1) return FACO_E_ARG;
  if (n > kMultiMaxN) return FACO_E_SIZE;
  for (int64_t j = 0; j < 2 * (int64_t)n; ++j)
    if (coords_xy[j] < 0 || coords_xy[j] >= (1 << 24)) return FACO_E_ARG;
  std::unique_ptr<Request> r(new (std::nothrow) Request());
  if (!r) return FACO_E_NOMEM;
  r->n = n;
  r->k = k;
  r->ants = ants;
  r->budget = budget;
  r->seed = seed;
  const int kk = k < n - 1 ? k : n - 1;
  int rc = plan_request(*r, s->prm, s->smem_blk[kk <= 16 ? 0 : 1]);
  if (rc != FACO_OK) return rc;
  if (r->bytes > s->pool.size()) return FACO_E_NOMEM;
  r->coords.assign(coords_xy, coords_xy + 2 * (size_t)n);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return FACO_E_STATE;
  r->id = s->next_id++;
  r->t_submit = now_ns();
  *ticket = r->id;
  s->queue.push_back(r.get());
  s->reqs[r->id] = std::move(r);
  s->stats.submitted++;
  s->cv.notify_all();
  return FACO_OK;
}

int faco_server_poll(faco_server* s, uint64_t ticket, int32_t* tour, int32_t len, int64_t* length_out,
                     int64_t* t_submit_ns, int64_t* t_done_ns) {
  if (!s) return FACO_E_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return FACO_E_ARG;
  Request* r = it->second.get();
  if (t_submit_ns) *t_submit_ns = r->t_submit;
  if (r->st != St::Done) return FACO_PENDING;
  if (r->status == FACO_OK) {
    if (tour) {
      if (len < r->n) return FACO_E_SIZE;
      std::memcpy(tour, r->tour.data(), sizeof(int32_t) * (size_t)r->n);
    }
    if (length_out) *length_out = r->length;
  }
  if (t_done_ns) *t_done_ns = r->t_done;
  return r->status;
}

int faco_server_wait(faco_server* s, uint64_t ticket, int32_t timeout_ms) {
  if (!s) return FACO_E_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return FACO_E_ARG;
  Request* r = it->second.get();
  s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                 [&] { return r->st == St::Done; });
  return r->st == St::Done ? r->status : FACO_PENDING;
}

int faco_server_release(faco_server* s, uint64_t ticket) {
  if (!s) return FACO_E_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return FACO_E_ARG;
  if (it->second->st != St::Done) return FACO_E_STATE;
  s->reqs.erase(it);
  return FACO_OK;
}

int faco_server_stats_get(faco_server* s, faco_server_stats* st) {
  if (!s || !st) return FACO_E_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *st = s->stats;
  st->queued = (int64_t)s->queue.size();
  int64_t setting = 0, active = 0;
  for (auto& kv : s->reqs) {
    setting += kv.second->st == St::SettingUp;
    active += kv.second->st == St::Active;
  }
  st->setting_up = setting;
  st->active = active;
  st->pool_in_use = (int64_t)s->pool.in_use();
  return FACO_OK;
}

int faco_test_pool(int64_t pool_bytes, const int64_t* ops, int32_t count, int64_t* out) {
  if (pool_bytes < 0 || pool_bytes > ((int64_t)1 << 26) || count < 0 || (count > 0 && (!ops || !out)))
    return FACO_E_ARG;
  std::vector<char> mem((size_t)pool_bytes + 1);
  Pool pool;
  pool.init(mem.data(), (size_t)pool_bytes);
  std::vector<char*> got((size_t)count, nullptr);
  std::vector<size_t> got_bytes((size_t)count, 0);
  for (int32_t i = 0; i < count; ++i) {
    const int64_t a = ops[2 * (size_t)i], b = ops[2 * (size_t)i + 1];
    if (a > 0) {
      char* p = pool.get((size_t)a);
      got[i] = p;
      got_bytes[i] = (size_t)a;
      out[2 * (size_t)i] = p ? (int64_t)(p - mem.data()) : -1;
    } else if (a == 0 && b >= 0 && b < i && got[b]) {
      pool.put(got[b], got_bytes[b]);
      got[b] = nullptr;
      out[2 * (size_t)i] = 0;
    } else {
      return FACO_E_ARG;
    }
    out[2 * (size_t)i + 1] = (int64_t)pool.in_use();
  }
  return FACO_OK;
}

void faco_server_destroy(faco_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (Request* r : s->queue) {  // queued requests are dropped
      r->status = FACO_E_STATE;
      r->st = St::Done;
      r->t_done = now_ns();
    }
    s->queue.clear();
    s->cv.notify_all();
  }
  if (s->thr.joinable()) s->thr.join();
  for (int c = 0; c < kCohorts; ++c) cudaStreamSynchronize(s->lane[c]);
  cudaStreamSynchronize(s->setup);
  for (auto& kv : s->reqs) {
    Request* r = kv.second.get();
    if (r->ev) cudaEventDestroy(r->ev);
    if (r->pinned) cudaFreeHost(r->pinned);
  }
  s->reqs.clear();
  for (int c = 0; c < kCohorts; ++c) {
    for (cudaEvent_t e : s->round_ev[c])
      if (e) cudaEventDestroy(e);
  }
  if (s->pool_mem) cudaFree(s->pool_mem);
  for (int c = 0; c < kCohorts; ++c) cudaStreamDestroy(s->lane[c]);
  cudaStreamDestroy(s->setup);
  delete s;
}

}  // extern "C"
