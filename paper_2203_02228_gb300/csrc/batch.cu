// batch.cu -- the C ABI of include/faco_batch.h: many independent colonies
// through the same launches (group set-up, tuned per-ant kernels, the whole
// iteration budget replayed as one CUDA graph).  Host code only plans,
// allocates and launches.
#include <cstring>
#include <new>
#include <vector>

#include "faco_batch.h"
#include "multi.h"

using namespace faco;

struct faco_batch {
  Group g;
  AntSet a;
  Runner r;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int plan_mode = -1;              // -1 tuned, 0 segment tables, 1 arrays
  int seg_mode = -1;               // params.seg_cap: -1 tables where they fit, 0 never
  std::vector<int32_t> variant;    // per colony, -1 before planning
  bool planned = false;
  size_t smem_blk = 0;
  cudaGraphExec_t gexec = nullptr;
  int graph_budget = -1;
  int64_t launches = 0;
  int32_t* pack_tours = nullptr;   // packed results
  int64_t* pack_lens = nullptr;
  int32_t* pack_err = nullptr;
};

namespace {

#define CK(expr)                                                           \
  do {                                                                     \
    cudaError_t e_ = (expr);                                               \
    if (e_ != cudaSuccess) {                                               \
      (void)cudaGetLastError();                                            \
      return e_ == cudaErrorMemoryAllocation ? FACO_E_NOMEM : FACO_E_CUDA; \
    }                                                                      \
  } while (0)

void drop_graph(faco_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  b->graph_budget = -1;
}

void free_batch(faco_batch* b) {
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graph(b);
  if (b->a.base) cudaFree(b->a.base);
  b->a.base = nullptr;
  if (b->g.base) cudaFree(b->g.base);
  b->g.base = nullptr;
  if (b->pack_tours) cudaFree(b->pack_tours);
  if (b->pack_lens) cudaFree(b->pack_lens);
  if (b->pack_err) cudaFree(b->pack_err);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  b->stream = nullptr;
}

std::vector<RunEntry> entries_of(faco_batch* b) {
  std::vector<RunEntry> e(b->g.count);
  for (int i = 0; i < b->g.count; ++i) e[i] = RunEntry{&b->g, i, &b->a, b->variant[i] < 0 ? 0 : b->variant[i]};
  return e;
}

// Per-ant buffers for `m` ants and the kernel plan; leaves the ant
// counters zeroed.
int plan(faco_batch* b, int m) {
  if (b->a.m != m) {
    CK(cudaStreamSynchronize(b->stream));
    drop_graph(b);
    if (b->a.base) cudaFree(b->a.base);
    b->a = AntSet{};
    AntSet a;
    antset_layout(a, b->g, m, b->smem_blk, b->seg_mode, nullptr);
    char* base = nullptr;
    CK(cudaMalloc(&base, a.bytes));
    antset_layout(a, b->g, m, b->smem_blk, b->seg_mode, base);
    b->a = a;
    CK(cudaMemsetAsync(base, 0, a.zero_bytes, b->stream));
    b->planned = false;
  }
  if (b->planned) return FACO_OK;
  drop_graph(b);
  const int C = b->g.count;
  b->variant.assign(C, 0);
  if (b->plan_mode < 0) {
    std::vector<RunEntry> e = entries_of(b);
    int rc = tuner_run(e, b->smem_blk, b->stream);
    if (rc != FACO_OK) return rc;
    for (int i = 0; i < C; ++i) {
      const int v = tuner_get(size_class(b->g.n[i]), m, b->g.kw);
      b->variant[i] = v >= 0 ? v : 0;
    }
  } else {
    for (int i = 0; i < C; ++i) b->variant[i] = b->plan_mode;
  }
  for (int i = 0; i < C; ++i)
    if (b->a.cap[i] <= 0 && b->variant[i] == kVarTable) b->variant[i] = kVarArr2;
  int rc = antset_zero(b->a, b->stream);  // counters written by trial launches
  if (rc != FACO_OK) return rc;
  rc = b->r.build(entries_of(b), b->smem_blk, b->stream);
  if (rc != FACO_OK) return rc;
  b->planned = true;
  return FACO_OK;
}

int capture(faco_batch* b, int budget) {
  drop_graph(b);
  cudaGraph_t gr = nullptr;
  CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  int rc = FACO_OK;
  for (int it = 0; it < budget && rc == FACO_OK; ++it) rc = b->r.enqueue(b->stream, 3);
  cudaError_t e = cudaStreamEndCapture(b->stream, &gr);
  if (rc != FACO_OK) {
    if (gr) cudaGraphDestroy(gr);
    return rc;
  }
  CK(e);
  e = cudaGraphInstantiate(&b->gexec, gr, 0);
  cudaGraphDestroy(gr);
  CK(e);
  b->graph_budget = budget;
  return FACO_OK;
}

int sync_check(faco_batch* b, int64_t* lens_host) {
  CK(launch_pack_batch(b->g.dC, b->g.count, b->g.map256, b->g.nmap256, b->g.d_node_off, nullptr, b->pack_lens,
                       b->pack_err, b->stream));
  int32_t err = 0;
  CK(cudaMemcpyAsync(&err, b->pack_err, sizeof(err), cudaMemcpyDeviceToHost, b->stream));
  if (lens_host)
    CK(cudaMemcpyAsync(lens_host, b->pack_lens, sizeof(int64_t) * b->g.count, cudaMemcpyDeviceToHost, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  if (err & kErrTimeout) return FACO_E_TIMEOUT;
  if (err & kErrCapacity) return FACO_E_CAPACITY;
  if (err) return FACO_E_CUDA;
  return FACO_OK;
}

}  // namespace

extern "C" {

int faco_batch_create(const int32_t* const* coords_xy, const int32_t* ns, int32_t count, int32_t k,
                      const faco_params* p, const uint64_t* seeds, faco_batch** out) {
  if (!coords_xy || !ns || !out) return FACO_E_ARG;
  faco_params prm;
  faco_params_default(&prm);
  if (p) prm = *p;
  faco_batch* b = new (std::nothrow) faco_batch();
  if (!b) return FACO_E_NOMEM;
  int rc = [&]() -> int {
    // arguments first, on the host
    int r = group_init(b->g, ns, count, k, prm, seeds);
    if (r != FACO_OK) return r;
    r = group_check_coords(b->g, coords_xy);
    if (r != FACO_OK) return r;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
      (void)cudaGetLastError();
      return FACO_E_CUDA;
    }
    b->seg_mode = prm.seg_cap;
    b->variant.assign(count, -1);
    if (prm.stream) {
      b->stream = static_cast<cudaStream_t>(prm.stream);
    } else {
      CK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
      b->own_stream = true;
    }
    b->smem_blk = batch_smem_blk(b->g.kw);
    char* base = nullptr;
    CK(cudaMalloc(&base, b->g.bytes));
    group_layout(b->g, base);
    CK(cudaMalloc(&b->pack_tours, sizeof(int32_t) * (size_t)b->g.node_off[count]));
    CK(cudaMalloc(&b->pack_lens, sizeof(int64_t) * (size_t)count));
    CK(cudaMalloc(&b->pack_err, sizeof(int32_t)));
    r = group_setup(b->g, coords_xy, b->stream);
    if (r != FACO_OK) return r;
    b->launches += 15;  // set-up: grid 3, candidate lists 4, initial tour 2, colony state 6
    return FACO_OK;
  }();
  if (rc != FACO_OK) {
    free_batch(b);
    delete b;
    return rc;
  }
  *out = b;
  return FACO_OK;
}

int faco_batch_iterate(faco_batch* b, int32_t ants, int32_t budget) {
  if (!b || ants < 1 || budget < 0) return FACO_E_ARG;
  if (budget == 0) return FACO_OK;
  int rc = plan(b, ants);
  if (rc != FACO_OK) return rc;
  if (!b->gexec || b->graph_budget != budget) {
    rc = capture(b, budget);
    if (rc != FACO_OK) return rc;
  }
  CK(cudaGraphLaunch(b->gexec, b->stream));
  b->launches += (int64_t)budget * b->r.kernels_per_iteration();
  return FACO_OK;
}

int faco_batch_sync(faco_batch* b) {
  if (!b) return FACO_E_ARG;
  return sync_check(b, nullptr);
}

int faco_batch_best(faco_batch* b, int32_t i, int32_t* tour, int32_t len, int64_t* length_out) {
  if (!b || i < 0 || i >= b->g.count) return FACO_E_ARG;
  if (tour && len < b->g.n[i]) return FACO_E_SIZE;
  int rc = sync_check(b, nullptr);
  if (rc != FACO_OK) return rc;
  if (tour) CK(cudaMemcpy(tour, b->g.hC[i].gb_route, sizeof(int32_t) * b->g.n[i], cudaMemcpyDeviceToHost));
  if (length_out)
    CK(cudaMemcpy(length_out, reinterpret_cast<char*>(b->g.hC[i].st) + offsetof(DevState, gb_len),
                  sizeof(int64_t), cudaMemcpyDeviceToHost));
  return FACO_OK;
}

int faco_batch_tours(faco_batch* b, int32_t* tours, int64_t* lengths) {
  if (!b) return FACO_E_ARG;
  CK(launch_pack_batch(b->g.dC, b->g.count, b->g.map256, b->g.nmap256, b->g.d_node_off,
                       tours ? b->pack_tours : nullptr, b->pack_lens, b->pack_err, b->stream));
  int rc = sync_check(b, lengths);
  if (rc != FACO_OK) return rc;
  if (tours)
    CK(cudaMemcpy(tours, b->pack_tours, sizeof(int32_t) * (size_t)b->g.node_off[b->g.count],
                  cudaMemcpyDeviceToHost));
  return FACO_OK;
}

int faco_batch_stats(faco_batch* b, int32_t i, faco_stats* s) {
  if (!b || !s || i < 0 || i >= b->g.count) return FACO_E_ARG;
  int rc = sync_check(b, nullptr);
  if (rc != FACO_OK) return rc;
  DevState h;
  CK(cudaMemcpy(&h, b->g.hC[i].st, sizeof(h), cudaMemcpyDeviceToHost));
  std::memset(s, 0, sizeof(*s));
  s->iteration = h.iter;
  s->best_length = h.gb_len;
  s->initial_length = h.init_len;
  s->source_length = h.src_len;
  s->n = b->g.n[i];
  s->k = b->g.k[i];
  s->bl = b->g.bl[i];
  s->ants = b->a.m;
  if (b->a.m > 0 && h.iter > 0) {
    std::vector<int64_t> st((size_t)b->a.m * kNStats);
    CK(cudaMemcpy(st.data(), b->a.hA[i].stats, sizeof(int64_t) * st.size(), cudaMemcpyDeviceToHost));
    for (int a = 0; a < b->a.m; ++a) {
      const int64_t* r = st.data() + (size_t)a * kNStats;
      s->aco_steps += r[kStAco];
      s->new_edges += r[kStNew];
      s->backup_picks += r[kStBackup];
      s->global_picks += r[kStGlobal];
      s->ls_pops += r[kStPops];
      s->moves_2opt += r[kStMoves2];
      s->moves_or += r[kStMovesOr];
      s->flip_elems += r[kStFlip];
      s->redone_ants += r[kStRedo];
    }
  }
  s->kernel_launches = b->launches;
  s->seg_cap = (b->variant.empty() || b->variant[i] != kVarTable) ? 0 : (b->a.m > 0 ? b->a.cap[i] : 0);
  return FACO_OK;
}

int faco_batch_tau(faco_batch* b, int32_t i, float* tau) {
  if (!b || !tau || i < 0 || i >= b->g.count) return FACO_E_ARG;
  int rc = sync_check(b, nullptr);
  if (rc != FACO_OK) return rc;
  CK(cudaMemcpy(tau, b->g.hC[i].tau, sizeof(float) * (size_t)b->g.n[i] * b->g.k[i], cudaMemcpyDeviceToHost));
  return FACO_OK;
}

int faco_batch_set_plan(faco_batch* b, int32_t mode) {
  if (!b || mode < -1 || mode >= kNVariants) return FACO_E_ARG;
  if (mode != b->plan_mode) {
    b->plan_mode = mode;
    b->planned = false;
  }
  return FACO_OK;
}

int faco_batch_get_plan(faco_batch* b, int32_t* variants) {
  if (!b || !variants) return FACO_E_ARG;
  for (int i = 0; i < b->g.count; ++i) variants[i] = b->planned ? b->variant[i] : -1;
  return FACO_OK;
}

int faco_batch_tuner_report(double* rows, int32_t max_rows, int32_t* count) {
  if (!count || max_rows < 0 || (max_rows > 0 && !rows)) return FACO_E_ARG;
  *count = tuner_report(rows, max_rows);
  return FACO_OK;
}

void faco_batch_destroy(faco_batch* b) {
  if (!b) return;
  free_batch(b);
  delete b;
}

}  // extern "C"
