// colony.cu -- per-iteration colony kernels of Alg 2 after the ants:
// iteration best and global best with the trail limits of Sec. 4.5, the
// source choice (global best with probability p_source_gb, Sec. 5.2),
// the pheromone update of Eq. 2 on candidate edges (Sec. 4.2), and the
// source-ordered rows that the next iteration's ants read.
#include "common.cuh"
#include "launch.h"

namespace faco {

namespace {

// Eq. 2 for every stored entry of the node at source position p, fused with
// the emission of that node's row in source order for the next iteration:
//   tau' = max(tau_min, min(tau_max, fmaf(rho, tau, delta * [edge in source])))
//   Wsrc[p][s] = tau' * eta,  Csrc[p][s] = source position of cand[u][s].
// update = 0 only sets tau = tau_max (Alg 2 set-up).
// The source node at p and its two source neighbours, and the trail
// parameters of this update.
struct RowCtx {
  int u, pn, pp;
  float tmax, tmin, delta;
};

__device__ __forceinline__ RowCtx row_ctx(const Colony& C, int p) {
  const int n = C.n;
  RowCtx r;
  r.u = C.src_route[p];
  r.pn = C.src_route[p + 1 == n ? 0 : p + 1];
  r.pp = C.src_route[p == 0 ? n - 1 : p - 1];
  r.tmax = C.st->tmax;
  r.tmin = C.st->tmin;
  r.delta = C.st->delta;
  return r;
}

// Entry s of row p (s < kw).
__device__ __forceinline__ void rows_entry(const Colony& C, const RowCtx& r, int p, int s, int update) {
  const int k = C.k, kw = C.kw;
  const size_t o = (size_t)p * kw + s;
  if (s >= k) {
    C.Wsrc[o] = 0.0f;
    C.Csrc[o] = -1;
    C.Dcsrc[o] = 0;
    return;
  }
  const size_t idx = (size_t)r.u * k + s;
  const int v = C.cand[idx];
  float t;
  if (update) {
    const float dep = (v == r.pn || v == r.pp) ? r.delta : 0.0f;
    t = __fmaf_rn(C.rho, C.tau[idx], dep);
    t = t < r.tmax ? t : r.tmax;
    t = t > r.tmin ? t : r.tmin;
  } else {
    t = r.tmax;
  }
  C.tau[idx] = t;
  C.Wsrc[o] = __fmul_rn(t, C.eta[idx]);
  C.Csrc[o] = C.src_pos[v];
  C.Dcsrc[o] = C.dcand[idx];
}

// The per-node parts of row p: coordinates, source edge length, and the
// grid's point record p with the new source positions.
__device__ __forceinline__ void rows_node(const Colony& C, const RowCtx& r, int p) {
  const int2 xu = C.xy[r.u];
  C.XYsrc[p] = xu;
  C.Dsrc[p] = euc2d(xu, C.xy[r.pn]);
  const int v = C.cell_pts[p];
  const int2 xv = C.xy[v];
  C.cell_src[p] = make_int4(C.src_pos[v], xv.x, xv.y, v);
}

// Exclusive prefix sums of the source edge lengths (one block).
__device__ __forceinline__ void scan_P_body(const Colony& C) {
  // tiles of 8 consecutive edges per thread, read and written coalesced,
  // with the running total carried from tile to tile
  constexpr int E = 8;
  __shared__ int64_t warp_tot[32];
  __shared__ int64_t s_carry;
  const int n = C.n, t = threadIdx.x, T = blockDim.x;
  const int lane = t & 31, w = t >> 5, nw = T >> 5;
  if (t == 0) s_carry = 0;
  for (int base = 0; base < n; base += E * T) {
    const int i0 = base + E * t;
    int d[E];
#pragma unroll
    for (int u = 0; u < E; ++u) d[u] = i0 + u < n ? C.Dsrc[i0 + u] : 0;
    int64_t s = 0;
#pragma unroll
    for (int u = 0; u < E; ++u) s += d[u];
    // block inclusive scan of s
    int64_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = shfl64_up(incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
      int64_t v = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = shfl64_up(v, o);
        if (lane >= o) v += y;
      }
      warp_tot[lane] = v;  // inclusive over warps
    }
    __syncthreads();
    const int64_t carry = s_carry;
    int64_t run = carry + (incl - s) + (w > 0 ? warp_tot[w - 1] : 0);
#pragma unroll
    for (int u = 0; u < E; ++u) {
      if (i0 + u < n) C.Psrc[i0 + u] = run;
      run += d[u];
    }
    const int64_t tile = warp_tot[nw - 1];
    __syncthreads();  // every thread has read the carry and the warp totals
    if (t == 0) s_carry = carry + tile;
  }
  __syncthreads();
  if (t == 0) C.Psrc[n] = s_carry;
}

__device__ __forceinline__ void set_limits(const Colony& C, DevState* st, int64_t L) {
  st->tmax_d = 1.0 / ((double)L * (1.0 - (double)C.rho));
  st->tmin_d = st->tmax_d * C.c_min;
  st->tmax = __double2float_rn(st->tmax_d);
  st->tmin = __double2float_rn(st->tmin_d);
}

// Iteration best (shortest, lowest ant on ties), global best + limits,
// source choice, deposit amount, history row (one block).
__device__ __forceinline__ void best_body(const Colony& C, const Ants& A) {
  __shared__ int64_t sl[32];
  __shared__ int32_t sa[32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  int64_t bl = INT64_MAX;
  int32_t ba = INT32_MAX;
  for (int a = t; a < A.m; a += blockDim.x) {
    const int64_t L = A.len[a];
    if (L < bl || (L == bl && a < ba)) {
      bl = L;
      ba = a;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int64_t l2 = shfl64_xor(bl, o);
    const int32_t a2 = __shfl_xor_sync(kFull, ba, o);
    if (l2 < bl || (l2 == bl && a2 < ba)) {
      bl = l2;
      ba = a2;
    }
  }
  if (lane == 0) {
    sl[w] = bl;
    sa[w] = ba;
  }
  __syncthreads();
  if (t != 0) return;
  for (int i = 1; i < (int)(blockDim.x >> 5); ++i)
    if (sl[i] < bl || (sl[i] == bl && sa[i] < ba)) {
      bl = sl[i];
      ba = sa[i];
    }
  DevState* st = C.st;
  const int64_t iter = st->iter + 1;
  const int improved = bl < st->gb_len;
  if (improved) {
    st->gb_len = bl;
    set_limits(C, st, bl);
  }
  const float u = u01(draw(C.seed, 0, 0, (uint32_t)iter, 1));
  const int use_gb = (double)u < C.p_src_gb;
  st->src_len = use_gb ? st->gb_len : bl;
  st->delta = __double2float_rn(1.0 / (double)st->src_len);
  st->it_best_len = bl;
  st->it_best_ant = ba;
  st->gb_improved = improved;
  st->use_gb = use_gb;
  st->iter = iter;
  if (iter - 1 < st->hist_cap) {
    int64_t* h = st->hist + 4 * (iter - 1);
    h[0] = bl;
    h[1] = ba;
    h[2] = st->gb_len;
    h[3] = use_gb;
  }
}

// The iteration-best tour as explicit route/pos (into tmp): from its
// segment table (source positions -> node ids of the current source), or
// from the ant's arrays when it was built with them.  Skipped when neither
// the global best nor the source will take it.
__device__ __forceinline__ void best_tour_body(const Colony& C, const Ants& A, int t) {
  int32_t* tmp_route = C.tmp_route;
  int32_t* tmp_pos = C.tmp_pos;
  const int n = C.n;
  const DevState* st = C.st;
  if (t >= n || (!st->gb_improved && st->use_gb)) return;
  const int a = st->it_best_ant;
  int node;
  const int S = A.nseg ? A.nseg[a] : -1;
  if (S == -1) {  // node ids
    node = A.route[(size_t)a * n + t];
  } else if (S < 0) {  // source positions
    node = C.src_route[A.route[(size_t)a * n + t]];
  } else {
    const int4* sg = A.segs + (size_t)a * A.seg_cap_ls;
    int lo = 0, hi = S - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sg[mid].z <= t)
        lo = mid;
      else
        hi = mid - 1;
    }
    const int4 s = sg[lo];
    const int d = t - s.z;
    int q = s.w ? s.x + s.y - 1 - d : s.x + d;
    if ((unsigned)q >= (unsigned)n) {  // inconsistent table: a library bug, flagged
      atomicOr(&C.st->error, kErrInternal);
      q = 0;
    }
    node = C.src_route[q];
  }
  tmp_route[t] = node;
  tmp_pos[node] = t;
}

// Global best <- iteration best when improved; source <- global best or
// iteration best (routes and positions).
__device__ __forceinline__ void source_body(const Colony& C, int i) {
  const int32_t* tmp_route = C.tmp_route;
  const int32_t* tmp_pos = C.tmp_pos;
  const int n = C.n;
  if (i >= n) return;
  const DevState* st = C.st;
  if (st->gb_improved) {
    C.gb_route[i] = tmp_route[i];
    C.gb_pos[i] = tmp_pos[i];
  }
  if (st->use_gb) {
    C.src_route[i] = C.gb_route[i];
    C.src_pos[i] = C.gb_pos[i];
  } else {
    C.src_route[i] = tmp_route[i];
    C.src_pos[i] = tmp_pos[i];
  }
}

__device__ __forceinline__ void state_init_body(const Colony& C, const int64_t* len) {
  DevState* st = C.st;
  const int64_t L = *len;
  st->iter = 0;
  st->init_len = L;
  st->gb_len = L;
  st->src_len = L;
  st->it_best_len = L;
  st->it_best_ant = 0;
  st->use_gb = 1;
  st->gb_improved = 0;
  st->error = 0;
  set_limits(C, st, L);
  st->delta = __double2float_rn(1.0 / (double)L);
}

// ---------------------------------------------------------------------
// Kernels of one colony (descriptor by value) and of a batch (each block
// reads its colony, and its block within the colony, from a block map).
// ---------------------------------------------------------------------
// A thread per row entry: consecutive threads write consecutive entries.
__global__ void k_rows(Colony C, int update) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = (int)(t / C.kw), s = (int)(t % C.kw);
  if (p >= C.n) return;
  const RowCtx r = row_ctx(C, p);
  rows_entry(C, r, p, s, update);
  if (s == 0) rows_node(C, r, p);
}

__global__ void __launch_bounds__(1024) k_scan_P(Colony C) { scan_P_body(C); }

__global__ void __launch_bounds__(1024) k_best(Colony C, Ants A) { best_body(C, A); }

__global__ void k_best_tour(Colony C, Ants A) { best_tour_body(C, A, blockIdx.x * blockDim.x + threadIdx.x); }

__global__ void k_source(Colony C) { source_body(C, blockIdx.x * blockDim.x + threadIdx.x); }

__global__ void k_state_init(Colony C, const int64_t* len) {
  if (threadIdx.x == 0 && blockIdx.x == 0) state_init_body(C, len);
}

// Block e.y of colony e.x covers the rows of nodes e.y * blockDim.x onward
// (as many as threads); its threads take the row entries in order, so that
// consecutive threads write consecutive entries.
__global__ void k_rows_b(const Colony* cols, const int2* map, int update) {
  const int2 e = map[blockIdx.x];
  const Colony C = cols[e.x];
  const int p0 = e.y * blockDim.x;
  const int rows = min((int)blockDim.x, C.n - p0);
  if (rows <= 0) return;
  const int kw = C.kw;
  for (int q = threadIdx.x; q < rows * kw; q += blockDim.x) {
    const int p = p0 + q / kw, s = q % kw;
    const RowCtx r = row_ctx(C, p);
    rows_entry(C, r, p, s, update);
    if (s == 0) rows_node(C, r, p);
  }
}

__global__ void __launch_bounds__(1024) k_scan_P_b(const Colony* cols) {
  const Colony C = cols[blockIdx.x];
  scan_P_body(C);
}

// Also empties the redo list of the batch's per-ant kernels (they have all
// finished when this kernel runs).
__global__ void __launch_bounds__(1024) k_best_b(const Colony* cols, const Ants* ants, int32_t* redo_n) {
  const Colony C = cols[blockIdx.x];
  const Ants A = ants[blockIdx.x];
  if (blockIdx.x == 0 && threadIdx.x == 0 && redo_n) *redo_n = 0;
  best_body(C, A);
}

__global__ void k_best_tour_b(const Colony* cols, const Ants* ants, const int2* map) {
  const int2 e = map[blockIdx.x];
  const Colony C = cols[e.x];
  const Ants A = ants[e.x];
  best_tour_body(C, A, e.y * blockDim.x + threadIdx.x);
}

__global__ void k_source_b(const Colony* cols, const int2* map) {
  const int2 e = map[blockIdx.x];
  const Colony C = cols[e.x];
  source_body(C, e.y * blockDim.x + threadIdx.x);
}

// Batch set-up: positions of the initial tour (into src_pos, the local
// search's position array), its length, the colony state, and source and
// global best <- initial tour.
__global__ void k_init_pos_b(const Colony* cols, const ColonySetup* sets, const int2* map) {
  const int2 e = map[blockIdx.x];
  const int i = e.y * blockDim.x + threadIdx.x;
  const Colony C = cols[e.x];
  if (i < C.n) C.src_pos[sets[e.x].init_route[i]] = i;
}

__global__ void k_init_len_b(const Colony* cols, const ColonySetup* sets, const int2* map) {
  const int2 e = map[blockIdx.x];
  const int i = e.y * blockDim.x + threadIdx.x;
  const Colony C = cols[e.x];
  const int32_t* route = sets[e.x].init_route;
  int64_t d = 0;
  if (i < C.n) d = euc2d(C.xy[route[i]], C.xy[route[i + 1 == C.n ? 0 : i + 1]]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += shfl64_xor(d, o);
  if ((threadIdx.x & 31) == 0 && d)
    atomicAdd(reinterpret_cast<unsigned long long*>(sets[e.x].len), (unsigned long long)d);
}

__global__ void k_state_init_b(const Colony* cols, const ColonySetup* sets, int count) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= count) return;
  const Colony C = cols[c];
  state_init_body(C, sets[c].len);
}

__global__ void k_init_routes_b(const Colony* cols, const ColonySetup* sets, const int2* map) {
  const int2 e = map[blockIdx.x];
  const int i = e.y * blockDim.x + threadIdx.x;
  const Colony C = cols[e.x];
  if (i >= C.n) return;
  const int v = sets[e.x].init_route[i];
  C.src_route[i] = v;
  C.gb_route[i] = v;
  C.src_pos[v] = i;
  C.gb_pos[v] = i;
}

// Batch results: every colony's global-best tour packed at node_off[c];
// lengths and the union of the device error flags.
__global__ void k_pack_tours_b(const Colony* cols, const int2* map, const int64_t* node_off, int32_t* out) {
  const int2 e = map[blockIdx.x];
  const int i = e.y * blockDim.x + threadIdx.x;
  const Colony C = cols[e.x];
  if (i < C.n) out[node_off[e.x] + i] = C.gb_route[i];
}

__global__ void k_pack_state_b(const Colony* cols, int count, int64_t* lens, int32_t* err) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= count) return;
  const DevState* st = cols[c].st;
  lens[c] = st->gb_len;
  if (st->error) atomicOr(err, st->error);
}

__global__ void k_positions(const int32_t* route, int32_t* pos, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) pos[route[i]] = i;
}

__global__ void k_tour_length(const int2* xy, const int32_t* route, int n, unsigned long long* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int64_t d = 0;
  if (i < n) d = euc2d(xy[route[i]], xy[route[i + 1 == n ? 0 : i + 1]]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += shfl64_xor(d, o);
  if ((threadIdx.x & 31) == 0 && d) atomicAdd(out, (unsigned long long)d);
}

}  // namespace

cudaError_t launch_rows(const Colony& C, int update, cudaStream_t s) {
  k_rows<<<(unsigned)(((int64_t)C.n * C.kw + 255) / 256), 256, 0, s>>>(C, update);
  return cudaGetLastError();
}

cudaError_t launch_scan_P(const Colony& C, cudaStream_t s) {
  k_scan_P<<<1, 1024, 0, s>>>(C);
  return cudaGetLastError();
}

cudaError_t launch_best(const Colony& C, const Ants& A, cudaStream_t s) {
  k_best<<<1, 1024, 0, s>>>(C, A);
  return cudaGetLastError();
}

cudaError_t launch_source(const Colony& C, const Ants& A, cudaStream_t s) {
  k_best_tour<<<(C.n + 255) / 256, 256, 0, s>>>(C, A);
  k_source<<<(C.n + 255) / 256, 256, 0, s>>>(C);
  return cudaGetLastError();
}

cudaError_t launch_colony_update_batch(const Colony* cols, const Ants* ants, int count, const int2* map256,
                                       int nmap256, int32_t* redo_n, cudaStream_t s) {
  k_best_b<<<count, 256, 0, s>>>(cols, ants, redo_n);
  k_best_tour_b<<<nmap256, 256, 0, s>>>(cols, ants, map256);
  k_source_b<<<nmap256, 256, 0, s>>>(cols, map256);
  k_rows_b<<<nmap256, 256, 0, s>>>(cols, map256, 1);
  k_scan_P_b<<<count, 256, 0, s>>>(cols);
  return cudaGetLastError();
}

cudaError_t launch_pack_batch(const Colony* cols, int count, const int2* map256, int nmap256,
                              const int64_t* node_off, int32_t* tours, int64_t* lens, int32_t* err,
                              cudaStream_t s) {
  if (tours) k_pack_tours_b<<<nmap256, 256, 0, s>>>(cols, map256, node_off, tours);
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  k_pack_state_b<<<(count + 127) / 128, 128, 0, s>>>(cols, count, lens, err);
  return cudaGetLastError();
}

cudaError_t launch_colony_init_batch(const Colony* cols, const ColonySetup* sets, int count, const int2* map256,
                                     int nmap256, int stage, cudaStream_t s) {
  if (stage == 0) {  // positions of the initial tour, before its local search
    k_init_pos_b<<<nmap256, 256, 0, s>>>(cols, sets, map256);
  } else {  // after it: length, state, source and global best, rows, prefix sums
    k_init_len_b<<<nmap256, 256, 0, s>>>(cols, sets, map256);
    k_state_init_b<<<(count + 127) / 128, 128, 0, s>>>(cols, sets, count);
    k_init_routes_b<<<nmap256, 256, 0, s>>>(cols, sets, map256);
    k_rows_b<<<nmap256, 256, 0, s>>>(cols, map256, 0);
    k_scan_P_b<<<count, 256, 0, s>>>(cols);
  }
  return cudaGetLastError();
}

cudaError_t launch_state_init(const Colony& C, const int64_t* len, cudaStream_t s) {
  k_state_init<<<1, 32, 0, s>>>(C, len);
  return cudaGetLastError();
}

cudaError_t launch_positions(const int32_t* route, int32_t* pos, int n, cudaStream_t s) {
  k_positions<<<(n + 255) / 256, 256, 0, s>>>(route, pos, n);
  return cudaGetLastError();
}

cudaError_t launch_tour_length(const int2* xy, const int32_t* route, int n, int64_t* out,
                               cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int64_t), s);
  if (e != cudaSuccess) return e;
  k_tour_length<<<(n + 255) / 256, 256, 0, s>>>(xy, route, n, reinterpret_cast<unsigned long long*>(out));
  return cudaGetLastError();
}

}  // namespace faco
