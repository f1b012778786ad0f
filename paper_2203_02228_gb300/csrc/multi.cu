// multi.cu -- host side of running many colonies through the same launches:
// group set-up in one arena, per-ant buffers, the per-iteration runner with
// its block maps, and the per-size-class kernel tuner.  Every step of the
// method runs in the batch kernels of ants.cu, colony.cu, knn.cu, tour.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "multi.h"

namespace faco {

int check_faco_params(const faco_params& p) {
  if (!(p.rho > 0.0f && p.rho < 1.0f)) return FACO_E_ARG;
  if (!(p.p_best > 0.0 && p.p_best < 1.0)) return FACO_E_ARG;
  if (!(p.p_source_gb >= 0.0 && p.p_source_gb <= 1.0)) return FACO_E_ARG;
  if (p.min_new_edges < 1 || p.bl_size < 0 || p.bl_size > 128) return FACO_E_ARG;
  if (p.seg_cap < -1 || (p.seg_cap > 0 && p.seg_cap < 8) || p.seg_cap > 4096) return FACO_E_ARG;
  if (p.local_search != 0 && p.local_search != 1) return FACO_E_ARG;
  if (p.init_3opt != 0 && p.init_3opt != 1) return FACO_E_ARG;
  return FACO_OK;
}

namespace {

#define CK(expr)                                                           \
  do {                                                                     \
    cudaError_t e_ = (expr);                                               \
    if (e_ != cudaSuccess) {                                               \
      (void)cudaGetLastError();                                            \
      return e_ == cudaErrorMemoryAllocation ? FACO_E_NOMEM : FACO_E_CUDA; \
    }                                                                      \
  } while (0)

// Bump layout: every piece starts on a 256-byte boundary.
struct Bump {
  char* base;
  size_t size = 0;
  explicit Bump(char* b) : base(b) {}
  template <typename T>
  T* take(size_t count) {
    const size_t off = (size + 255) & ~(size_t)255;
    const size_t bytes = count * sizeof(T);
    size = off + (bytes > 0 ? bytes : 16);
    return base ? reinterpret_cast<T*>(base + off) : nullptr;
  }
};

int grid_side(int n) {
  const int64_t G = (int64_t)std::ceil(std::sqrt((double)n / 2.0));
  return G < 1 ? 1 : (int)G;
}

void add_blocks(std::vector<int2>& map, int c, int64_t items, int per) {
  const int nb = (int)((items + per - 1) / per);
  for (int b = 0; b < nb; ++b) map.push_back(make_int2(c, b));
}

size_t vis_bytes_of(int n) { return ((size_t)((n + 31) >> 5) * 4 + 15) & ~(size_t)15; }

}  // namespace

// ---------------------------------------------------------------------
// Group
// ---------------------------------------------------------------------
int group_init(Group& g, const int32_t* ns, int count, int k, const faco_params& prm, const uint64_t* seeds) {
  if (!ns || count < 1 || count > 65535 || k < 2 || k > kMaxK) return FACO_E_ARG;
  int rc = check_faco_params(prm);
  if (rc != FACO_OK) return rc;
  if (prm.keep_ant_tours || prm.keep_pre_ls || prm.seg_cap > 0) return FACO_E_ARG;
  g = Group{};
  g.count = count;
  g.prm = prm;
  g.n.resize(count);
  g.k.resize(count);
  g.bl.resize(count);
  g.seed.resize(count);
  g.node_off.assign(count + 1, 0);
  int kw = -1;
  for (int i = 0; i < count; ++i) {
    const int n = ns[i];
    if (n < 3) return FACO_E_ARG;
    if (n > kMultiMaxN) return FACO_E_SIZE;
    const int kk = k < n - 1 ? k : n - 1;
    int bl = prm.bl_size < n - 1 - kk ? prm.bl_size : n - 1 - kk;
    if (bl < 0) bl = 0;
    const int w = kk <= 16 ? 16 : 32;
    if (kw >= 0 && w != kw) return FACO_E_ARG;  // one roulette width per group
    kw = w;
    g.n[i] = n;
    g.k[i] = kk;
    g.bl[i] = bl;
    g.seed[i] = seeds ? seeds[i] : prm.seed;
    g.node_off[i + 1] = g.node_off[i] + n;
    g.max_n = std::max(g.max_n, n);
  }
  g.kw = kw;
  group_layout(g, nullptr);
  return FACO_OK;
}

void group_layout(Group& g, char* base) {
  Bump B(base);
  const int C = g.count;
  g.hC.assign(C, Colony{});
  g.hS.assign(C, ColonySetup{});
  // zeroed on set-up: states, lengths, cell counts, local-search flags
  std::vector<DevState*> st(C);
  for (int i = 0; i < C; ++i) st[i] = B.take<DevState>(1);
  for (int i = 0; i < C; ++i) g.hS[i].len = B.take<int64_t>(1);
  for (int i = 0; i < C; ++i) {
    const int G = grid_side(g.n[i]);
    g.hS[i].cell_cnt = B.take<int32_t>((size_t)G * G);
  }
  for (int i = 0; i < C; ++i) g.hS[i].flags = B.take<uint8_t>(g.n[i]);
  g.zero_bytes = (B.size + 255) & ~(size_t)255;
  // tables
  std::vector<int2> m256, m128;
  for (int i = 0; i < C; ++i) {
    add_blocks(m256, i, g.n[i], 256);
    add_blocks(m128, i, g.n[i], 128);
  }
  g.nmap256 = (int)m256.size();
  g.nmap128 = (int)m128.size();
  g.dC = B.take<Colony>(C);
  g.dS = B.take<ColonySetup>(C);
  g.map256 = B.take<int2>(m256.size());
  g.map128 = B.take<int2>(m128.size());
  g.d_node_off = B.take<int64_t>(C + 1);
  for (int i = 0; i < C; ++i) g.hS[i].bb = B.take<int32_t>(5);
  // per-colony arrays, type by type
  for (int i = 0; i < C; ++i) {
    Colony& c = g.hC[i];
    const int n = g.n[i];
    c.n = n;
    c.k = g.k[i];
    c.bl = g.bl[i];
    c.kw = g.kw;
    c.seed = g.seed[i];
    c.rho = g.prm.rho;
    c.min_new_edges = g.prm.min_new_edges;
    c.oropt = g.prm.oropt;
    c.verify = g.prm.verify_pass;
    c.ls = g.prm.local_search;
    c.init3 = g.prm.init_3opt;
    const double pr = std::pow(g.prm.p_best, 1.0 / (double)n);
    c.c_min = (1.0 - pr) / ((double)(c.k - 1) * pr);
    c.p_src_gb = g.prm.p_source_gb;
    c.st = st[i];
    c.grid = Grid{0, 0, 1, 1, 1};
  }
  for (int i = 0; i < C; ++i) g.hC[i].xy = B.take<int2>(g.n[i]);
  for (int i = 0; i < C; ++i) {
    g.hS[i].cand = B.take<int32_t>((size_t)g.n[i] * g.k[i]);
    g.hC[i].cand = g.hS[i].cand;
  }
  for (int i = 0; i < C; ++i) {
    g.hS[i].backup = B.take<int32_t>((size_t)g.n[i] * (g.bl[i] > 0 ? g.bl[i] : 1));
    g.hC[i].backup = g.hS[i].backup;
  }
  for (int i = 0; i < C; ++i) {
    g.hS[i].eta = B.take<float>((size_t)g.n[i] * g.k[i]);
    g.hC[i].eta = g.hS[i].eta;
  }
  for (int i = 0; i < C; ++i) {
    g.hS[i].dcand = B.take<int32_t>((size_t)g.n[i] * g.k[i]);
    g.hC[i].dcand = g.hS[i].dcand;
  }
  for (int i = 0; i < C; ++i) g.hC[i].tau = B.take<float>((size_t)g.n[i] * g.k[i]);
  for (int i = 0; i < C; ++i) g.hC[i].src_route = B.take<int32_t>(g.n[i]);
  for (int i = 0; i < C; ++i) g.hC[i].src_pos = B.take<int32_t>(g.n[i]);
  for (int i = 0; i < C; ++i) g.hC[i].gb_route = B.take<int32_t>(g.n[i]);
  for (int i = 0; i < C; ++i) g.hC[i].gb_pos = B.take<int32_t>(g.n[i]);
  for (int i = 0; i < C; ++i) g.hC[i].Wsrc = B.take<float>((size_t)g.n[i] * g.kw);
  for (int i = 0; i < C; ++i) g.hC[i].Csrc = B.take<int32_t>((size_t)g.n[i] * g.kw);
  for (int i = 0; i < C; ++i) g.hC[i].Dcsrc = B.take<int32_t>((size_t)g.n[i] * g.kw);
  for (int i = 0; i < C; ++i) g.hC[i].XYsrc = B.take<int2>(g.n[i]);
  for (int i = 0; i < C; ++i) g.hC[i].Dsrc = B.take<int32_t>(g.n[i]);
  for (int i = 0; i < C; ++i) g.hC[i].Psrc = B.take<int64_t>((size_t)g.n[i] + 1);
  for (int i = 0; i < C; ++i) g.hC[i].tmp_route = B.take<int32_t>(g.n[i]);
  for (int i = 0; i < C; ++i) g.hC[i].tmp_pos = B.take<int32_t>(g.n[i]);
  for (int i = 0; i < C; ++i) {
    const int G = grid_side(g.n[i]);
    g.hS[i].cell_start = B.take<int32_t>((size_t)G * G + 1);
    g.hC[i].cell_start = g.hS[i].cell_start;
  }
  for (int i = 0; i < C; ++i) {
    g.hS[i].cell_pts = B.take<int32_t>(g.n[i]);
    g.hC[i].cell_pts = g.hS[i].cell_pts;
  }
  for (int i = 0; i < C; ++i) {
    g.hS[i].cell_src = B.take<int4>(g.n[i]);
    g.hC[i].cell_src = g.hS[i].cell_src;
  }
  for (int i = 0; i < C; ++i) g.hS[i].init_route = B.take<int32_t>(g.n[i]);
  for (int i = 0; i < C; ++i) g.hS[i].queue = B.take<int32_t>(g.n[i]);
  for (int i = 0; i < C; ++i) g.hS[i].logb = B.take<int32_t>(g.n[i]);
  g.bytes = (B.size + 255) & ~(size_t)255;
  g.base = base;
}

int group_check_coords(const Group& g, const int32_t* const* coords) {
  if (!coords) return FACO_E_ARG;
  for (int i = 0; i < g.count; ++i) {
    const int32_t* xy = coords[i];
    if (!xy) return FACO_E_ARG;
    for (int64_t j = 0; j < 2 * (int64_t)g.n[i]; ++j)
      if (xy[j] < 0 || xy[j] >= (1 << 24)) return FACO_E_ARG;
  }
  return FACO_OK;
}

int group_setup(Group& g, const int32_t* const* coords, cudaStream_t s) {
  if (!g.base) return FACO_E_ARG;
  int rc = group_check_coords(g, coords);
  if (rc != FACO_OK) return rc;
  CK(cudaMemsetAsync(g.base, 0, g.zero_bytes, s));
  for (int i = 0; i < g.count; ++i)
    CK(cudaMemcpyAsync(const_cast<int2*>(g.hC[i].xy), coords[i], sizeof(int2) * (size_t)g.n[i],
                       cudaMemcpyHostToDevice, s));
  std::vector<int2> m256, m128;
  for (int i = 0; i < g.count; ++i) {
    add_blocks(m256, i, g.n[i], 256);
    add_blocks(m128, i, g.n[i], 128);
  }
  // pageable sources: each copy has been staged when the call returns
  CK(cudaMemcpyAsync(g.dC, g.hC.data(), sizeof(Colony) * g.count, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(g.dS, g.hS.data(), sizeof(ColonySetup) * g.count, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(g.map256, m256.data(), sizeof(int2) * m256.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(g.map128, m128.data(), sizeof(int2) * m128.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(g.d_node_off, g.node_off.data(), sizeof(int64_t) * (g.count + 1), cudaMemcpyHostToDevice, s));
  CK(launch_grid_batch(g.dC, g.dS, g.count, g.map256, g.nmap256, s));
  CK(build_lists_batch(g.dC, g.dS, g.count, g.map256, g.nmap256, g.map128, g.nmap128, s));
  CK(launch_init_tour_batch(g.dC, g.dS, g.count, g.max_n, 0, s));       // nearest-neighbour tours
  CK(launch_colony_init_batch(g.dC, g.dS, g.count, g.map256, g.nmap256, 0, s));
  CK(launch_init_tour_batch(g.dC, g.dS, g.count, g.max_n, 1, s));       // their local search
  CK(launch_colony_init_batch(g.dC, g.dS, g.count, g.map256, g.nmap256, 1, s));
  return FACO_OK;
}

// ---------------------------------------------------------------------
// Per-ant buffers
// ---------------------------------------------------------------------
int ant_cap(int n, size_t smem_blk, int seg_mode) {
  if (seg_mode == 0) return 0;
  const size_t base = ants_smem_per_warp(n, 0, true);  // visited bits + fixed part of a table
  const size_t per_seg = ants_smem_per_warp(n, 1, true) - base;
  if (smem_blk <= base) return 0;
  size_t cap = (smem_blk - base) / per_seg;
  cap = cap > 1024 ? 1024 : (cap & ~(size_t)31);
  return cap >= 64 ? (int)cap : 0;
}

void antset_layout(AntSet& a, const Group& g, int m, size_t smem_blk, int seg_mode, char* base) {
  Bump B(base);
  const int C = g.count;
  a.m = m;
  a.hA.assign(C, Ants{});
  a.cap.assign(C, 0);
  for (int i = 0; i < C; ++i) a.hA[i].flags = B.take<uint8_t>((size_t)m * g.n[i]);
  for (int i = 0; i < C; ++i) a.hA[i].stats = B.take<int64_t>((size_t)m * kNStats);
  for (int i = 0; i < C; ++i) a.hA[i].redo = B.take<int32_t>(m);
  a.zero_bytes = (B.size + 255) & ~(size_t)255;
  for (int i = 0; i < C; ++i) a.hA[i].route = B.take<int32_t>((size_t)m * g.n[i]);
  for (int i = 0; i < C; ++i) a.hA[i].pos = B.take<int32_t>((size_t)m * g.n[i]);
  for (int i = 0; i < C; ++i) a.hA[i].chk = B.take<int32_t>((size_t)m * g.n[i]);
  for (int i = 0; i < C; ++i) a.hA[i].queue = B.take<int32_t>((size_t)m * g.n[i]);
  for (int i = 0; i < C; ++i) a.hA[i].logb = B.take<int32_t>((size_t)m * g.n[i]);
  for (int i = 0; i < C; ++i) a.hA[i].len = B.take<int64_t>(m);
  for (int i = 0; i < C; ++i) a.hA[i].nseg = B.take<int32_t>(m);
  for (int i = 0; i < C; ++i) {
    a.cap[i] = ant_cap(g.n[i], smem_blk, seg_mode);
    a.hA[i].seg_cap_ls = ants_seg_cap_ls(g.n[i], a.cap[i]);
    a.hA[i].segs = B.take<int4>((size_t)m * (a.cap[i] > 0 ? a.hA[i].seg_cap_ls : 1));
  }
  for (int i = 0; i < C; ++i) {
    Ants& A = a.hA[i];
    A.m = m;
    A.vis_g = nullptr;
    A.smem_vis = 1;
    A.seg_cap = a.cap[i];
    A.keep_tours = 0;
    A.pre_route = nullptr;
    A.pre_len = nullptr;
    A.pre_chk = nullptr;
    A.pre_nchk = nullptr;
  }
  a.bytes = (B.size + 255) & ~(size_t)255;
  a.base = base;
}

int antset_zero(const AntSet& a, cudaStream_t s) {
  CK(cudaMemsetAsync(a.base, 0, a.zero_bytes, s));
  return FACO_OK;
}

// ---------------------------------------------------------------------
// Runner
// ---------------------------------------------------------------------
Runner::~Runner() {
  if (mem) cudaFree(mem);
  for (int v = 0; v < kNVariants; ++v) {
    if (side[v]) cudaStreamDestroy(side[v]);
    if (join[v]) cudaEventDestroy(join[v]);
  }
  if (fork) cudaEventDestroy(fork);
}

int Runner::build(const std::vector<RunEntry>& entries, size_t smem, cudaStream_t s) {
  const int C = (int)entries.size();
  if (C < 1) return FACO_E_ARG;
  count = C;
  kw = entries[0].g->kw;
  smem_blk = smem;
  std::vector<Ants> hA(C);
  std::vector<int> order(C);
  per_warp = 16;
  int64_t redo_cap = 1;
  for (int j = 0; j < C; ++j) {
    const RunEntry& e = entries[j];
    if (e.g->kw != kw) return FACO_E_ARG;
    Ants A = e.a->hA[e.i];
    if (e.variant != kVarTable || A.seg_cap <= 0) {
      A.seg_cap = 0;
      A.seg_cap_ls = 0;
      A.segs = nullptr;
      A.nseg = nullptr;
      A.redo = nullptr;
    } else {
      redo_cap += A.m;
    }
    hA[j] = A;
    order[j] = j;
    per_warp = std::max(per_warp, vis_bytes_of(e.g->n[e.i]));
  }
  // longest instances first: their ants start in the first wave
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return entries[x].g->n[entries[x].i] > entries[y].g->n[entries[y].i];
  });
  std::vector<int2> mblk, marr[kNVariants], m256;
  for (int j : order) {
    const int m = hA[j].m;
    if (hA[j].segs) {
      for (int a = 0; a < m; ++a) mblk.push_back(make_int2(j, a));
    } else {
      int v = entries[j].variant;
      if (v < kVarArr2 || v >= kNVariants) v = kVarArr2;
      for (int a = 0; a < m; a += 4) marr[v].push_back(make_int2(j, a));
    }
  }
  for (int j = 0; j < C; ++j) add_blocks(m256, j, entries[j].g->n[entries[j].i], 256);
  nblk = (int)mblk.size();
  for (int v = 0; v < kNVariants; ++v) narr[v] = (int)marr[v].size();
  nmap256 = (int)m256.size();
  redo_blocks = nblk > 0 ? kRedoBlocks : 0;  // a launch of its own, after the segment-table launch
  // one device block: tables, maps, redo list and count
  Bump B(nullptr);
  B.take<Colony>(C);
  B.take<Ants>(C);
  B.take<int2>(mblk.size());
  for (int v = 0; v < kNVariants; ++v) B.take<int2>(marr[v].size());
  B.take<int2>(m256.size());
  B.take<int2>((size_t)redo_cap);
  B.take<int32_t>(1);
  if (B.size > mem_bytes) {
    // a runner rebuilt for changing sets (the server's cohorts) grows
    // geometrically: a free waits for the whole device
    const size_t want = mem_bytes ? std::max(B.size, 2 * mem_bytes) : B.size;
    if (mem) {
      CK(cudaStreamSynchronize(s));
      cudaFree(mem);
      mem = nullptr;
      mem_bytes = 0;
    }
    CK(cudaMalloc(&mem, want));
    mem_bytes = want;
  }
  Bump D(mem);
  dC = D.take<Colony>(C);
  dA = D.take<Ants>(C);
  map_blk = D.take<int2>(mblk.size());
  for (int v = 0; v < kNVariants; ++v) map_arr[v] = D.take<int2>(marr[v].size());
  map256 = D.take<int2>(m256.size());
  redo_list = D.take<int2>((size_t)redo_cap);
  redo_n = D.take<int32_t>(1);
  // colony descriptors: device to device (their grids were set on the device),
  // one copy per run of consecutive colonies of a group
  for (int j = 0; j < C;) {
    int r = j + 1;
    while (r < C && entries[r].g == entries[j].g && entries[r].i == entries[r - 1].i + 1) ++r;
    CK(cudaMemcpyAsync(dC + j, entries[j].g->dC + entries[j].i, sizeof(Colony) * (r - j),
                       cudaMemcpyDeviceToDevice, s));
    j = r;
  }
  CK(cudaMemcpyAsync(dA, hA.data(), sizeof(Ants) * C, cudaMemcpyHostToDevice, s));
  if (!mblk.empty())
    CK(cudaMemcpyAsync(map_blk, mblk.data(), sizeof(int2) * mblk.size(), cudaMemcpyHostToDevice, s));
  for (int v = 0; v < kNVariants; ++v)
    if (!marr[v].empty())
      CK(cudaMemcpyAsync(map_arr[v], marr[v].data(), sizeof(int2) * marr[v].size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(map256, m256.data(), sizeof(int2) * m256.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(redo_n, 0, sizeof(int32_t), s));
  CK(prepare_ants_batch(kw, smem_blk, 4 * per_warp));
  if (!fork) {
    CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    for (int v = 0; v < kNVariants; ++v) {
      CK(cudaStreamCreateWithFlags(&side[v], cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&join[v], cudaEventDisableTiming));
    }
  }
  return FACO_OK;
}

int Runner::enqueue(cudaStream_t s, int parts) const {
  if (parts & 1) {
    // every per-ant launch on its own branch; the redo list after the
    // segment-table launch that fills it
    int used[kNVariants];
    int nused = 0;
    for (int v = 0; v < kNVariants; ++v)
      if (v == kVarTable ? nblk > 0 : narr[v] > 0) used[nused++] = v;
    if (nused > 1) CK(cudaEventRecord(fork, s));
    for (int u = 0; u < nused; ++u) {
      const int v = used[u];
      cudaStream_t q = u == 0 ? s : side[v];
      if (u > 0) CK(cudaStreamWaitEvent(q, fork, 0));
      if (v == kVarTable) {
        CK(launch_ants_blk_batch(kw, dC, dA, map_blk, nblk, redo_list, redo_n, smem_blk, q));
        CK(launch_ants_arr_batch(kw, 2, dC, dA, nullptr, 0, redo_blocks, redo_list, redo_n, per_warp, q));
      } else {
        CK(launch_ants_arr_batch(kw, kArrMinBlocks[v], dC, dA, map_arr[v], narr[v], 0, redo_list, redo_n,
                                 per_warp, q));
      }
      if (u > 0) CK(cudaEventRecord(join[v], q));
    }
    for (int u = 1; u < nused; ++u) CK(cudaStreamWaitEvent(s, join[used[u]], 0));
  }
  if (parts & 2) CK(launch_colony_update_batch(dC, dA, count, map256, nmap256, redo_n, s));
  return FACO_OK;
}

int Runner::kernels_per_iteration() const {
  int k = (nblk > 0 ? 2 : 0) + 5;
  for (int v = kVarArr2; v < kNVariants; ++v) k += narr[v] > 0;
  return k;
}

// ---------------------------------------------------------------------
// Tuner
// ---------------------------------------------------------------------
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, int> g_tune;  // (device, class, m, kw, goal) -> variant
// the timings behind each choice, per variant (ms, scaled as the goal says;
// negative: not tried)
std::map<std::tuple<int, int, int, int, int>, std::vector<float>> g_tune_ms;

int cur_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}
}  // namespace

int size_class(int n) {
  int c = 0;
  for (int v = n; v >= 512; v >>= 2) ++c;
  return c;  // [3, 512), [512, 2048), [2048, 8192), ...
}

int tuner_get(int cls, int m, int kw, int goal) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(std::make_tuple(cur_device(), cls, m, kw, goal));
  return it == g_tune.end() ? -1 : it->second;
}

void tuner_put(int cls, int m, int kw, int variant, int goal) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[std::make_tuple(cur_device(), cls, m, kw, goal)] = variant;
}

int tuner_run(const std::vector<RunEntry>& entries, size_t smem, cudaStream_t s, int goal) {
  // the untuned classes, and up to 64 colonies of each (spread over the
  // class when it has more)
  std::map<std::pair<int, int>, std::vector<RunEntry>> cls;
  for (const RunEntry& e : entries) {
    const int c = size_class(e.g->n[e.i]);
    const int m = e.a->m;
    if (tuner_get(c, m, e.g->kw, goal) >= 0) continue;
    cls[std::make_pair(c, m)].push_back(e);
  }
  for (auto& kv : cls) {
    std::vector<RunEntry>& v = kv.second;
    if (v.size() <= 64) continue;
    std::vector<RunEntry> pick;
    for (int j = 0; j < 64; ++j) pick.push_back(v[(size_t)j * v.size() / 64]);
    v.swap(pick);
  }
  if (cls.empty()) return FACO_OK;
  cudaEvent_t ev[2];
  CK(cudaEventCreate(&ev[0]));
  cudaError_t ce = cudaEventCreate(&ev[1]);
  if (ce != cudaSuccess) {
    cudaEventDestroy(ev[0]);
    CK(ce);
  }
  int rc = FACO_OK;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cur_device());
  for (auto& kv : cls) {
    std::vector<RunEntry>& v = kv.second;
    bool any_tab = false;
    for (const RunEntry& e : v) any_tab |= e.a->cap[e.i] > 0;
    int best = kVarArr2;
    float t_rec[kNVariants];
    for (int variant = 0; variant < kNVariants; ++variant) t_rec[variant] = -1.0f;
    {
      float t[kNVariants];
      for (int variant = 0; variant < kNVariants && rc == FACO_OK; ++variant) {
        t[variant] = 1e30f;
        if (variant == kVarTable && !any_tab) continue;
        for (RunEntry& e : v) e.variant = variant;
        Runner r;
        rc = r.build(v, smem, s);
        float tmin = 1e30f;
        for (int rep = 0; rep < 2 && rc == FACO_OK; ++rep) {
          if (cudaEventRecord(ev[0], s) != cudaSuccess) rc = FACO_E_CUDA;
          if (rc == FACO_OK) rc = r.enqueue(s, 1);
          if (rc == FACO_OK && cudaEventRecord(ev[1], s) != cudaSuccess) rc = FACO_E_CUDA;
          if (rc == FACO_OK && cudaEventSynchronize(ev[1]) != cudaSuccess) rc = FACO_E_CUDA;
          float ms = 0;
          if (rc == FACO_OK && cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess) rc = FACO_E_CUDA;
          tmin = std::min(tmin, ms);
        }
        if (rc == FACO_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = FACO_E_CUDA;
        // A class that does not fill the GPU's resident ant slots leaves the
        // rest to the other classes of a batch: its cost there is the time
        // measured alone times the fraction of slots it holds.
        int ants = 0;
        for (const RunEntry& e : v) ants += e.a->m;
        const int per_sm = ants_batch_resident(variant, v[0].g->kw,
                                               variant == kVarTable ? r.smem_blk : 4 * r.per_warp);
        const double slots = (double)per_sm * sms;
        const double frac = goal == kTuneBatch && slots > 0 ? std::min(1.0, ants / slots) : 1.0;
        t[variant] = (float)(tmin * frac);
      }
      if (rc != FACO_OK) break;
      for (int variant = 0; variant < kNVariants; ++variant) {
        if (t[variant] < t[best]) best = variant;
        if (t[variant] < 1e29f) t_rec[variant] = t[variant];
      }
    }
    tuner_put(kv.first.first, kv.first.second, v[0].g->kw, best, goal);
    if (rc == FACO_OK) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      std::vector<float>& rec =
          g_tune_ms[std::make_tuple(cur_device(), kv.first.first, kv.first.second, v[0].g->kw, goal)];
      rec.assign(kNVariants, -1.0f);
      for (int variant = 0; variant < kNVariants; ++variant) rec[variant] = t_rec[variant];
    }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (rc != FACO_OK) (void)cudaGetLastError();
  return rc;
}

int tuner_report(double* out, int max_rows) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const int dev = cur_device();
  int r = 0;
  for (const auto& kv : g_tune_ms) {
    if (std::get<0>(kv.first) != dev) continue;
    if (r < max_rows && out) {
      double* row = out + (size_t)r * (5 + kNVariants);
      row[0] = std::get<1>(kv.first);
      row[1] = std::get<2>(kv.first);
      row[2] = std::get<3>(kv.first);
      row[3] = std::get<4>(kv.first);
      auto it = g_tune.find(kv.first);
      row[4] = it == g_tune.end() ? -1 : it->second;
      for (int v = 0; v < kNVariants; ++v) row[5 + v] = kv.second[v];
    }
    ++r;
  }
  return r;
}

size_t batch_smem_blk(int kw) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, size_t> cache;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair(cur_device(), kw);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  const size_t S = ants_blk_batch_smem(kw);
  cache[key] = S;
  return S;
}

}  // namespace faco
