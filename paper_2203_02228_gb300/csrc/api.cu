// api.cu -- the C ABI declared in include/faco.h: colony set-up (Alg 2
// lines before the main loop), the graph-captured iteration, results and
// inspection.  Host code only marshals, allocates and launches; every step
// of the method runs in the kernels of ants.cu, colony.cu, knn.cu, tour.cu.
#include <cmath>
#include <cstddef>
#include <cstring>
#include <new>
#include <vector>

#include "faco.h"
#include "launch.h"
#include "multi.h"

using namespace faco;

struct faco_ctx {
  int n = 0, k = 0, bl = 0, kw = 16;
  faco_params prm{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  double c_min = 0;
  int2* xy = nullptr;
  int32_t* cand = nullptr;
  int32_t* backup = nullptr;
  float* eta = nullptr;
  float* tau = nullptr;
  int32_t *src_route = nullptr, *src_pos = nullptr, *gb_route = nullptr, *gb_pos = nullptr;
  float* Wsrc = nullptr;
  int32_t* Csrc = nullptr;
  int32_t* Dcsrc = nullptr;
  int32_t* dcand = nullptr;
  int2* XYsrc = nullptr;
  int32_t* Dsrc = nullptr;
  int64_t* Psrc = nullptr;
  DevState* st = nullptr;
  int64_t* hist = nullptr;
  int64_t hist_cap = 0;
  int32_t* init_route = nullptr;
  int64_t init_len = 0;
  int64_t* len_tmp = nullptr;
  int32_t* tmp_route = nullptr;          // iteration-best tour, materialised
  int32_t* tmp_pos = nullptr;
  Grid grid{};                           // point grid (candidate lists, nearest unvisited)
  int32_t* cell_start = nullptr;
  int32_t* cell_pts = nullptr;
  int4* cell_src = nullptr;
  Ants A{};
  std::vector<void*> ant_allocs;
  cudaGraphExec_t gexec = nullptr;       // whole iteration
  cudaGraphExec_t gexec_ants = nullptr;  // per-ant kernel only (profiling)
  cudaGraphExec_t gexec_rest = nullptr;  // colony update only (profiling)
  int graph_ants = -1;
  bool profiling = false;
  std::vector<cudaEvent_t> events;       // pairs around the per-ant kernel
  size_t events_used = 0;
  int64_t iters_enqueued = 0;
  int64_t launches = 0;                  // kernels launched (graph nodes counted)
  std::vector<void*> allocs;
};

// Kernels per iteration: ants (segment tables), ants (arrays), best,
// best tour, source, rows, prefix sums; one fewer without segment tables.
constexpr int kItersKernels = 7;
// Kernels of the set-up: bbox, cell count, cell scan, cell fill, kNN,
// nearest-neighbour tour, positions, relabel, initial local search,
// unlabel, tour length, state, positions (source), positions (best), rows,
// prefix sums.
constexpr int kSetupKernels = 16;

namespace {

#define CK(expr)                                 \
  do {                                           \
    cudaError_t e_ = (expr);                     \
    if (e_ != cudaSuccess) {                     \
      (void)cudaGetLastError();                  \
      return e_ == cudaErrorMemoryAllocation ? FACO_E_NOMEM : FACO_E_CUDA; \
    }                                            \
  } while (0)

template <typename T>
int dalloc(std::vector<void*>& list, T** p, size_t count) {
  void* q = nullptr;
  const size_t bytes = count * sizeof(T) > 0 ? count * sizeof(T) : 16;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? FACO_E_NOMEM : FACO_E_CUDA;
  }
  list.push_back(q);
  *p = static_cast<T*>(q);
  return FACO_OK;
}

#define DA(list, ptr, count)                       \
  do {                                             \
    int rc_ = dalloc(list, &(ptr), (size_t)(count)); \
    if (rc_ != FACO_OK) return rc_;                \
  } while (0)

Colony colony_view(const faco_ctx* c) {
  Colony C;
  C.n = c->n; C.k = c->k; C.bl = c->bl; C.kw = c->kw;
  C.seed = c->prm.seed; C.rho = c->prm.rho; C.min_new_edges = c->prm.min_new_edges;
  C.oropt = c->prm.oropt; C.verify = c->prm.verify_pass; C.ls = c->prm.local_search;
  C.init3 = c->prm.init_3opt;
  C.c_min = c->c_min; C.p_src_gb = c->prm.p_source_gb;
  C.xy = c->xy; C.cand = c->cand; C.backup = c->backup; C.eta = c->eta; C.tau = c->tau;
  C.src_route = c->src_route; C.src_pos = c->src_pos; C.gb_route = c->gb_route; C.gb_pos = c->gb_pos;
  C.Wsrc = c->Wsrc; C.Csrc = c->Csrc; C.XYsrc = c->XYsrc; C.Dsrc = c->Dsrc; C.Psrc = c->Psrc;
  C.Dcsrc = c->Dcsrc; C.dcand = c->dcand;
  C.st = c->st;
  C.grid = c->grid;
  C.cell_start = c->cell_start;
  C.cell_pts = c->cell_pts;
  C.cell_src = c->cell_src;
  C.tmp_route = c->tmp_route;
  C.tmp_pos = c->tmp_pos;
  return C;
}

void free_ants(faco_ctx* c) {
  for (void* p : c->ant_allocs) cudaFree(p);
  c->ant_allocs.clear();
  c->A = Ants{};
  for (cudaGraphExec_t* g : {&c->gexec, &c->gexec_ants, &c->gexec_rest}) {
    if (*g) cudaGraphExecDestroy(*g);
    *g = nullptr;
  }
  c->graph_ants = -1;
}

void free_all(faco_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_ants(c);
  for (cudaEvent_t e : c->events) cudaEventDestroy(e);
  c->events.clear();
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  c->stream = nullptr;
}

int set_hist(faco_ctx* c) {
  CK(cudaMemcpyAsync(reinterpret_cast<char*>(c->st) + offsetof(DevState, hist), &c->hist,
                     sizeof(c->hist), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(reinterpret_cast<char*>(c->st) + offsetof(DevState, hist_cap), &c->hist_cap,
                     sizeof(c->hist_cap), cudaMemcpyHostToDevice, c->stream));
  return cudaStreamSynchronize(c->stream) == cudaSuccess ? FACO_OK : FACO_E_CUDA;
}

int grow_hist(faco_ctx* c, int64_t rows) {
  if (rows <= c->hist_cap) return FACO_OK;
  int64_t cap = c->hist_cap > 0 ? c->hist_cap : 1024;
  while (cap < rows) cap *= 2;
  int64_t* h = nullptr;
  CK(cudaMalloc(&h, sizeof(int64_t) * 4 * cap));
  CK(cudaMemsetAsync(h, 0, sizeof(int64_t) * 4 * cap, c->stream));
  if (c->hist) {
    CK(cudaMemcpyAsync(h, c->hist, sizeof(int64_t) * 4 * c->hist_cap, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    cudaFree(c->hist);
  }
  c->hist = h;
  c->hist_cap = cap;
  return set_hist(c);
}

int create_common(const int32_t* coords, int32_t n, int32_t k, const faco_params* p, bool on_device,
                  faco_ctx** out) {
  if (!coords || !out || n < 3 || k < 2 || k > kMaxK) return FACO_E_ARG;
  faco_params prm;
  faco_params_default(&prm);
  if (p) prm = *p;
  int rc = check_faco_params(prm);
  if (rc != FACO_OK) return rc;
  if (!on_device) {
    for (int64_t i = 0; i < 2 * (int64_t)n; ++i)
      if (coords[i] < 0 || coords[i] >= (1 << 24)) return FACO_E_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    (void)cudaGetLastError();
    return FACO_E_CUDA;
  }
  faco_ctx* c = new (std::nothrow) faco_ctx();
  if (!c) return FACO_E_NOMEM;
  c->prm = prm;
  c->n = n;
  c->k = k < n - 1 ? k : n - 1;
  c->bl = prm.bl_size < n - 1 - c->k ? prm.bl_size : n - 1 - c->k;
  if (c->bl < 0) c->bl = 0;
  c->kw = c->k <= 16 ? 16 : 32;
  const double pr = std::pow(prm.p_best, 1.0 / (double)n);
  c->c_min = (1.0 - pr) / ((double)(c->k - 1) * pr);

  rc = [&]() -> int {
    if (prm.stream) {
      c->stream = static_cast<cudaStream_t>(prm.stream);
    } else {
      CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
      c->own_stream = true;
    }
    auto& L = c->allocs;
    const int K = c->k + c->bl;
    (void)K;
    DA(L, c->xy, n);
    DA(L, c->cand, (size_t)n * c->k);
    DA(L, c->backup, (size_t)n * (c->bl > 0 ? c->bl : 1));
    DA(L, c->eta, (size_t)n * c->k);
    DA(L, c->tau, (size_t)n * c->k);
    DA(L, c->src_route, n);
    DA(L, c->src_pos, n);
    DA(L, c->gb_route, n);
    DA(L, c->gb_pos, n);
    DA(L, c->Wsrc, (size_t)n * c->kw);
    DA(L, c->Csrc, (size_t)n * c->kw);
    DA(L, c->Dcsrc, (size_t)n * c->kw);
    DA(L, c->dcand, (size_t)n * c->k);
    DA(L, c->XYsrc, n);
    DA(L, c->Dsrc, n);
    DA(L, c->Psrc, (size_t)n + 1);
    DA(L, c->st, 1);
    DA(L, c->init_route, n);
    DA(L, c->len_tmp, 1);
    DA(L, c->tmp_route, n);
    DA(L, c->tmp_pos, n);
    CK(cudaMemsetAsync(c->st, 0, sizeof(DevState), c->stream));
    cudaStream_t s = c->stream;
    CK(cudaMemcpyAsync(c->xy, coords, sizeof(int2) * (size_t)n,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    // bounding box (and the range check for device coordinates)
    int32_t* bb = nullptr;
    std::vector<void*> tmp;
    auto free_tmp = [&]() {
      for (void* q : tmp) cudaFree(q);
      tmp.clear();
    };
    int r2 = dalloc(tmp, &bb, 5);
    if (r2 != FACO_OK) return r2;
    int32_t hb[5];
    if (launch_bbox_check(c->xy, n, bb, s) != cudaSuccess ||
        cudaMemcpyAsync(hb, bb, sizeof(hb), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      free_tmp();
      return FACO_E_CUDA;
    }
    if (hb[4]) {
      free_tmp();
      return FACO_E_ARG;
    }
    Grid g;
    g.minx = hb[0];
    g.miny = hb[1];
    const int64_t ext = (int64_t)(hb[2] - hb[0] > hb[3] - hb[1] ? hb[2] - hb[0] : hb[3] - hb[1]) + 1;
    int64_t G = (int64_t)std::ceil(std::sqrt((double)n / 2.0));
    if (G < 1) G = 1;
    g.cs = (int32_t)((ext + G - 1) / G);
    if (g.cs < 1) g.cs = 1;
    g.gx = (hb[2] - hb[0]) / g.cs + 1;
    g.gy = (hb[3] - hb[1]) / g.cs + 1;
    const int64_t cells = (int64_t)g.gx * g.gy;
    int32_t* cc = nullptr;
    if ((r2 = dalloc(tmp, &cc, cells)) != FACO_OK || (r2 = dalloc(c->allocs, &c->cell_start, cells + 1)) != FACO_OK ||
        (r2 = dalloc(c->allocs, &c->cell_pts, n)) != FACO_OK || (r2 = dalloc(c->allocs, &c->cell_src, n)) != FACO_OK) {
      free_tmp();
      return r2;
    }
    c->grid = g;
    int32_t *cs = c->cell_start, *cp = c->cell_pts;
    if (build_lists(c->xy, n, c->k, c->bl, g, cc, cs, cp, c->cell_src, c->cand, c->backup, c->eta, c->dcand, s) !=
        cudaSuccess) {
      free_tmp();
      return FACO_E_CUDA;
    }
    // initial tour: nearest neighbour, then local search with every node queued
    const size_t vis_bytes = (size_t)((n + 31) >> 5) * sizeof(uint32_t);
    uint32_t* vis_g = nullptr;
    if (vis_bytes > 200 * 1024 && (r2 = dalloc(tmp, &vis_g, (n + 31) >> 5)) != FACO_OK) {
      free_tmp();
      return r2;
    }
    int32_t *q = nullptr, *lg = nullptr;
    uint8_t* fl = nullptr;
    // the search runs on copies named by nearest-neighbour tour position
    int2* xy_t = nullptr;
    int32_t *cand_t = nullptr, *dcand_t = nullptr, *route_t = nullptr, *pos_t = nullptr;
    const size_t nk = (size_t)n * c->k;
    if ((r2 = dalloc(tmp, &q, n)) != FACO_OK || (r2 = dalloc(tmp, &lg, n)) != FACO_OK ||
        (r2 = dalloc(tmp, &fl, n)) != FACO_OK || (r2 = dalloc(tmp, &xy_t, n)) != FACO_OK ||
        (r2 = dalloc(tmp, &cand_t, nk)) != FACO_OK || (r2 = dalloc(tmp, &dcand_t, nk)) != FACO_OK ||
        (r2 = dalloc(tmp, &route_t, n)) != FACO_OK || (r2 = dalloc(tmp, &pos_t, n)) != FACO_OK) {
      free_tmp();
      return r2;
    }
    cudaError_t e = launch_nn_tour(c->xy, n, c->cand, c->k, c->backup, c->bl, c->init_route, vis_g, g,
                                   c->cell_start, c->cell_src, s);
    if (e == cudaSuccess) e = launch_positions(c->init_route, c->src_pos, n, s);
    if (e == cudaSuccess)
      e = launch_relabel(c->init_route, c->src_pos, c->xy, c->cand, c->dcand, n, c->k, xy_t, cand_t, dcand_t,
                         route_t, pos_t, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(fl, 0, n, s);
    if (e == cudaSuccess)
      e = launch_init_ls(xy_t, n, cand_t, dcand_t, c->k, prm.oropt, prm.verify_pass, prm.init_3opt, route_t, pos_t,
                         q, fl, lg, s);
    // back to node ids (through tmp_route: init_route is the map's source)
    if (e == cudaSuccess) e = launch_unlabel(c->init_route, route_t, c->tmp_route, n, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->init_route, c->tmp_route, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = launch_tour_length(c->xy, c->init_route, n, c->len_tmp, s);
    Colony C = colony_view(c);
    if (e == cudaSuccess) e = launch_state_init(C, c->len_tmp, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->src_route, c->init_route, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->gb_route, c->init_route, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = launch_positions(c->src_route, c->src_pos, n, s);
    if (e == cudaSuccess) e = launch_positions(c->gb_route, c->gb_pos, n, s);
    if (e == cudaSuccess) e = launch_rows(C, 0, s);
    if (e == cudaSuccess) e = launch_scan_P(C, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&c->init_len, c->len_tmp, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    free_tmp();
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return FACO_E_CUDA;
    }
    c->launches += kSetupKernels;
    return grow_hist(c, 1024);
  }();
  if (rc != FACO_OK) {
    free_all(c);
    delete c;
    return rc;
  }
  *out = c;
  return FACO_OK;
}

// Segments per ant table (one ant per block): the requested size, or (auto)
// the largest table, up to 1024 segments, that still lets every ant of an
// iteration be resident at once; with fewer blocks per SM when the visited
// bits alone are too large for that.  0 (arrays only) when not even 64 fit.
int seg_capacity(int n, int m, int requested) {
  if (requested >= 0) return requested;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t base = ants_smem_per_warp(n, 0, true);
  const size_t per_seg = ants_smem_per_warp(n, 1, true) - base;
  const size_t total = 225 * 1024, fixed = 2 * 1024;  // usable per SM; static + reserved per block
  const int want = (m + sms - 1) / (sms > 0 ? sms : 1);
  for (int bps = want; bps >= 1; --bps) {
    const size_t budget = total / bps - fixed;
    if (budget <= base) continue;
    size_t cap = (budget - base) / per_seg;
    cap = cap > 1024 ? 1024 : (cap & ~(size_t)31);
    if (cap >= 256 || (bps == 1 && cap >= 64)) return (int)cap;
  }
  return 0;
}

int ensure_ants(faco_ctx* c, int m) {
  if (c->A.m == m) return FACO_OK;
  CK(cudaStreamSynchronize(c->stream));
  free_ants(c);
  const int n = c->n;
  const size_t words = (size_t)((n + 31) >> 5);
  auto& L = c->ant_allocs;
  Ants A{};
  A.m = m;
  const size_t mn = (size_t)m * n;
  DA(L, A.route, mn);
  DA(L, A.pos, mn);
  DA(L, A.chk, mn);
  DA(L, A.len, m);
  DA(L, A.stats, (size_t)m * kNStats);
  DA(L, A.queue, mn);
  DA(L, A.flags, mn);
  DA(L, A.logb, mn);
  CK(cudaMemsetAsync(A.flags, 0, mn, c->stream));
  CK(cudaMemsetAsync(A.stats, 0, sizeof(int64_t) * m * kNStats, c->stream));
  // array kernel: visited bits in shared memory when four warps' worth fits
  const size_t smem_arr = 4 * ants_smem_per_warp(n, 0, false);
  A.smem_vis = smem_arr <= 200 * 1024 ? 1 : 0;
  if (!A.smem_vis) DA(L, A.vis_g, (size_t)m * words);
  // segment-table kernel: one ant per block, bits + table in shared memory
  A.seg_cap = seg_capacity(n, m, c->prm.seg_cap);
  A.seg_cap_ls = ants_seg_cap_ls(n, A.seg_cap);
  const size_t smem_seg = A.seg_cap > 0 ? ants_smem_per_warp(n, A.seg_cap, true) : 0;
  if (A.seg_cap > 0) {
    DA(L, A.segs, (size_t)m * A.seg_cap_ls);
    DA(L, A.nseg, m);
    DA(L, A.redo, m);
    CK(cudaMemsetAsync(A.redo, 0, sizeof(int32_t) * m, c->stream));
  }
  A.keep_tours = c->prm.keep_ant_tours;
  CK(prepare_ants_kernel(c->kw, smem_seg, A.smem_vis ? smem_arr : 0));
  if (c->prm.keep_pre_ls) {
    DA(L, A.pre_route, mn);
    DA(L, A.pre_len, m);
    DA(L, A.pre_chk, mn);
    DA(L, A.pre_nchk, m);
  }
  c->A = A;
  return FACO_OK;
}

// part 1: the per-ant kernel; part 2: best, source, pheromone rows, prefix sums.
int enqueue_iteration(faco_ctx* c, int parts) {
  const Colony C = colony_view(c);
  if (parts & 1) CK(launch_ants(C, c->A, c->stream));
  if (parts & 2) {
    CK(launch_best(C, c->A, c->stream));
    CK(launch_source(C, c->A, c->stream));
    CK(launch_rows(C, 1, c->stream));
    CK(launch_scan_P(C, c->stream));
  }
  return FACO_OK;
}

int capture(faco_ctx* c, int parts, cudaGraphExec_t* out) {
  if (*out) {
    cudaGraphExecDestroy(*out);
    *out = nullptr;
  }
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  const int rc = enqueue_iteration(c, parts);
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (rc != FACO_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  CK(e);
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  CK(e);
  return FACO_OK;
}

int ensure_graph(faco_ctx* c) {
  if (c->gexec && c->gexec_ants && c->gexec_rest && c->graph_ants == c->A.m) return FACO_OK;
  int rc = capture(c, 3, &c->gexec);
  if (rc == FACO_OK) rc = capture(c, 1, &c->gexec_ants);
  if (rc == FACO_OK) rc = capture(c, 2, &c->gexec_rest);
  if (rc != FACO_OK) return rc;
  c->graph_ants = c->A.m;
  return FACO_OK;
}

int sync_and_check(faco_ctx* c) {
  CK(cudaStreamSynchronize(c->stream));
  int32_t err = 0;
  CK(cudaMemcpy(&err, reinterpret_cast<char*>(c->st) + offsetof(DevState, error), sizeof(err),
                cudaMemcpyDeviceToHost));
  if (err & kErrTimeout) return FACO_E_TIMEOUT;
  if (err & kErrCapacity) return FACO_E_CAPACITY;
  if (err) return FACO_E_CUDA;
  return FACO_OK;
}

}  // namespace

extern "C" {

int faco_params_default(faco_params* p) {
  if (!p) return FACO_E_ARG;
  std::memset(p, 0, sizeof(*p));
  p->seed = 1;
  p->rho = 0.5f;
  p->min_new_edges = 8;
  p->bl_size = 64;
  p->p_best = 0.05;
  p->p_source_gb = 0.01;
  p->oropt = 1;
  p->verify_pass = 1;
  p->keep_ant_tours = 0;
  p->keep_pre_ls = 0;
  p->seg_cap = -1;
  p->local_search = 1;
  p->init_3opt = 0;
  p->stream = nullptr;
  return FACO_OK;
}

int faco_create(const int32_t* coords_xy, int32_t n, int32_t k, faco_ctx** out) {
  return create_common(coords_xy, n, k, nullptr, false, out);
}

int faco_create_ex(const int32_t* coords_xy, int32_t n, int32_t k, const faco_params* p, faco_ctx** out) {
  return create_common(coords_xy, n, k, p, false, out);
}

int faco_create_device(const int32_t* coords_xy, int32_t n, int32_t k, const faco_params* p,
                       faco_ctx** out) {
  return create_common(coords_xy, n, k, p, true, out);
}

int faco_iterate(faco_ctx* c, int32_t ants, int32_t budget) {
  if (!c || ants < 1 || budget < 0) return FACO_E_ARG;
  if (budget == 0) return FACO_OK;
  int rc = ensure_ants(c, ants);
  if (rc != FACO_OK) return rc;
  rc = grow_hist(c, c->iters_enqueued + budget);
  if (rc != FACO_OK) return rc;
  rc = ensure_graph(c);
  if (rc != FACO_OK) return rc;
  if (!c->profiling) {
    for (int32_t b = 0; b < budget; ++b) CK(cudaGraphLaunch(c->gexec, c->stream));
  } else {
    while (c->events.size() < c->events_used + 2 * (size_t)budget) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      c->events.push_back(e);
    }
    for (int32_t b = 0; b < budget; ++b) {
      CK(cudaEventRecord(c->events[c->events_used], c->stream));
      CK(cudaGraphLaunch(c->gexec_ants, c->stream));
      CK(cudaEventRecord(c->events[c->events_used + 1], c->stream));
      CK(cudaGraphLaunch(c->gexec_rest, c->stream));
      c->events_used += 2;
    }
  }
  c->iters_enqueued += budget;
  c->launches += (int64_t)(c->A.seg_cap > 0 ? kItersKernels : kItersKernels - 1) * budget;
  return FACO_OK;
}

int faco_profile_enable(faco_ctx* c, int on) {
  if (!c) return FACO_E_ARG;
  c->profiling = on != 0;
  return FACO_OK;
}

int faco_profile_read(faco_ctx* c, double* ants_ms, int64_t* launches) {
  if (!c || !ants_ms || !launches) return FACO_E_ARG;
  CK(cudaStreamSynchronize(c->stream));
  double sum = 0;
  for (size_t i = 0; i + 1 < c->events_used; i += 2) {
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, c->events[i], c->events[i + 1]));
    sum += ms;
  }
  *ants_ms = sum;
  *launches = (int64_t)(c->events_used / 2);
  c->events_used = 0;
  return FACO_OK;
}

int faco_sync(faco_ctx* c) {
  if (!c) return FACO_E_ARG;
  return sync_and_check(c);
}

int faco_best(faco_ctx* c, int32_t* tour, int32_t len, int64_t* length_out) {
  if (!c) return FACO_E_ARG;
  if (tour && len < c->n) return FACO_E_SIZE;
  int rc = sync_and_check(c);
  if (rc != FACO_OK) return rc;
  if (tour) CK(cudaMemcpy(tour, c->gb_route, sizeof(int32_t) * c->n, cudaMemcpyDeviceToHost));
  if (length_out)
    CK(cudaMemcpy(length_out, reinterpret_cast<char*>(c->st) + offsetof(DevState, gb_len),
                  sizeof(int64_t), cudaMemcpyDeviceToHost));
  return FACO_OK;
}

int faco_best_device(faco_ctx* c, int32_t* tour_dev, int64_t* length_dev) {
  if (!c || !tour_dev || !length_dev) return FACO_E_ARG;
  CK(cudaMemcpyAsync(tour_dev, c->gb_route, sizeof(int32_t) * c->n, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(length_dev, reinterpret_cast<char*>(c->st) + offsetof(DevState, gb_len),
                     sizeof(int64_t), cudaMemcpyDeviceToDevice, c->stream));
  return FACO_OK;
}

int faco_stats_get(faco_ctx* c, faco_stats* s) {
  if (!c || !s) return FACO_E_ARG;
  int rc = sync_and_check(c);
  if (rc != FACO_OK) return rc;
  DevState h;
  CK(cudaMemcpy(&h, c->st, sizeof(h), cudaMemcpyDeviceToHost));
  std::memset(s, 0, sizeof(*s));
  s->iteration = h.iter;
  s->best_length = h.gb_len;
  s->initial_length = h.init_len;
  s->source_length = h.src_len;
  s->n = c->n;
  s->k = c->k;
  s->bl = c->bl;
  s->ants = c->A.m;
  if (c->A.m > 0 && h.iter > 0) {
    std::vector<int64_t> st((size_t)c->A.m * kNStats);
    CK(cudaMemcpy(st.data(), c->A.stats, sizeof(int64_t) * st.size(), cudaMemcpyDeviceToHost));
    for (int a = 0; a < c->A.m; ++a) {
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
  s->kernel_launches = c->launches;
  s->seg_cap = c->A.seg_cap;
  return FACO_OK;
}

void faco_destroy(faco_ctx* c) {
  if (!c) return;
  free_all(c);
  if (c->hist) cudaFree(c->hist);
  delete c;
}

const char* faco_strerror(int status) {
  switch (status) {
    case FACO_OK: return "ok";
    case FACO_E_ARG: return "invalid argument";
    case FACO_E_SIZE: return "buffer too small";
    case FACO_E_NOMEM: return "out of memory";
    case FACO_E_CUDA: return "CUDA error";
    case FACO_E_TIMEOUT: return "device wait timed out";
    case FACO_E_STATE: return "invalid state for this call";
    case FACO_E_CAPACITY: return "device capacity exceeded";
    default: return "unknown status";
  }
}

int faco_get_lists(faco_ctx* c, int32_t* cand, int32_t* backup, float* eta) {
  if (!c) return FACO_E_ARG;
  int rc = sync_and_check(c);
  if (rc != FACO_OK) return rc;
  const size_t n = (size_t)c->n;
  if (cand) CK(cudaMemcpy(cand, c->cand, sizeof(int32_t) * n * c->k, cudaMemcpyDeviceToHost));
  if (backup && c->bl > 0) CK(cudaMemcpy(backup, c->backup, sizeof(int32_t) * n * c->bl, cudaMemcpyDeviceToHost));
  if (eta) CK(cudaMemcpy(eta, c->eta, sizeof(float) * n * c->k, cudaMemcpyDeviceToHost));
  return FACO_OK;
}

int faco_get_tau(faco_ctx* c, float* tau) {
  if (!c || !tau) return FACO_E_ARG;
  int rc = sync_and_check(c);
  if (rc != FACO_OK) return rc;
  CK(cudaMemcpy(tau, c->tau, sizeof(float) * (size_t)c->n * c->k, cudaMemcpyDeviceToHost));
  return FACO_OK;
}

int faco_get_limits(faco_ctx* c, double* out4) {
  if (!c || !out4) return FACO_E_ARG;
  int rc = sync_and_check(c);
  if (rc != FACO_OK) return rc;
  DevState h;
  CK(cudaMemcpy(&h, c->st, sizeof(h), cudaMemcpyDeviceToHost));
  out4[0] = h.tmax_d;
  out4[1] = h.tmin_d;
  out4[2] = h.tmax;
  out4[3] = h.tmin;
  return FACO_OK;
}

int faco_get_source(faco_ctx* c, int32_t* route, int64_t* length_out) {
  if (!c) return FACO_E_ARG;
  int rc = sync_and_check(c);
  if (rc != FACO_OK) return rc;
  if (route) CK(cudaMemcpy(route, c->src_route, sizeof(int32_t) * c->n, cudaMemcpyDeviceToHost));
  if (length_out)
    CK(cudaMemcpy(length_out, reinterpret_cast<char*>(c->st) + offsetof(DevState, src_len),
                  sizeof(int64_t), cudaMemcpyDeviceToHost));
  return FACO_OK;
}

int faco_get_initial(faco_ctx* c, int32_t* route, int64_t* length_out) {
  if (!c) return FACO_E_ARG;
  int rc = sync_and_check(c);
  if (rc != FACO_OK) return rc;
  if (route) CK(cudaMemcpy(route, c->init_route, sizeof(int32_t) * c->n, cudaMemcpyDeviceToHost));
  if (length_out) *length_out = c->init_len;
  return FACO_OK;
}

int faco_get_history(faco_ctx* c, int64_t* hist, int64_t max_iters, int64_t* rows) {
  if (!c || !hist || !rows || max_iters < 0) return FACO_E_ARG;
  int rc = sync_and_check(c);
  if (rc != FACO_OK) return rc;
  int64_t it = 0;
  CK(cudaMemcpy(&it, c->st, sizeof(int64_t), cudaMemcpyDeviceToHost));
  int64_t r = it < max_iters ? it : max_iters;
  if (r > c->hist_cap) r = c->hist_cap;
  if (r > 0) CK(cudaMemcpy(hist, c->hist, sizeof(int64_t) * 4 * r, cudaMemcpyDeviceToHost));
  *rows = r;
  return FACO_OK;
}

int faco_get_ant_tours(faco_ctx* c, int32_t* tours, int64_t* lens) {
  if (!c) return FACO_E_ARG;
  if (!c->prm.keep_ant_tours || c->A.m == 0) return FACO_E_STATE;
  int rc = sync_and_check(c);
  if (rc != FACO_OK) return rc;
  const size_t mn = (size_t)c->A.m * c->n;
  if (tours) CK(cudaMemcpy(tours, c->A.route, sizeof(int32_t) * mn, cudaMemcpyDeviceToHost));
  if (lens) CK(cudaMemcpy(lens, c->A.len, sizeof(int64_t) * c->A.m, cudaMemcpyDeviceToHost));
  return FACO_OK;
}

int faco_get_ant_pre(faco_ctx* c, int32_t* tours, int64_t* lens, int32_t* checklists, int32_t* nchecks) {
  if (!c) return FACO_E_ARG;
  if (!c->prm.keep_pre_ls || c->A.m == 0) return FACO_E_STATE;
  int rc = sync_and_check(c);
  if (rc != FACO_OK) return rc;
  const size_t mn = (size_t)c->A.m * c->n;
  if (tours) CK(cudaMemcpy(tours, c->A.pre_route, sizeof(int32_t) * mn, cudaMemcpyDeviceToHost));
  if (lens) CK(cudaMemcpy(lens, c->A.pre_len, sizeof(int64_t) * c->A.m, cudaMemcpyDeviceToHost));
  if (checklists) CK(cudaMemcpy(checklists, c->A.pre_chk, sizeof(int32_t) * mn, cudaMemcpyDeviceToHost));
  if (nchecks) CK(cudaMemcpy(nchecks, c->A.pre_nchk, sizeof(int32_t) * c->A.m, cudaMemcpyDeviceToHost));
  return FACO_OK;
}

int faco_get_ant_stats(faco_ctx* c, int64_t* stats) {
  if (!c || !stats) return FACO_E_ARG;
  if (c->A.m == 0) return FACO_E_STATE;
  int rc = sync_and_check(c);
  if (rc != FACO_OK) return rc;
  CK(cudaMemcpy(stats, c->A.stats, sizeof(int64_t) * kNStats * c->A.m, cudaMemcpyDeviceToHost));
  return FACO_OK;
}

// Device self-tests used by the test-suite: host buffers in and out.
int faco_test_device(int what, const void* in, size_t in_bytes, void* out, size_t out_bytes, int count,
                     int width, uint64_t seed) {
  if (!in || !out || count < 0 || what < 0 || what > 2) return FACO_E_ARG;
  void *din = nullptr, *dout = nullptr;
  CK(cudaMalloc(&din, in_bytes > 0 ? in_bytes : 16));
  cudaError_t e = cudaMalloc(&dout, out_bytes > 0 ? out_bytes : 16);
  if (e == cudaSuccess) e = cudaMemcpy(din, in, in_bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && count > 0) e = launch_test_kernels(what, din, dout, count, width, seed, 0);
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, out_bytes, cudaMemcpyDeviceToHost);
  cudaFree(din);
  if (dout) cudaFree(dout);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return FACO_E_CUDA;
  }
  return FACO_OK;
}

}  // extern "C"
