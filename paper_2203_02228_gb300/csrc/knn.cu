// knn.cu -- candidate and backup lists (Sec. 4.1) with a uniform grid.
//
// For every node u the k + bl nearest other nodes ordered by (squared
// distance, node id): the first k form the candidate list, the next bl the
// backup list; eta = 1/d for the candidates (Sec. 2.1, d = EUC_2D cost).
// Points are bucketed into square cells (about two points per cell); a
// query scans rings of cells around its own cell and stops once the current
// k+bl-th key is strictly below the squared distance to the nearest point
// that could lie outside the scanned block, so the result is exact.
#include <climits>

#include "common.cuh"
#include "launch.h"

namespace faco {

namespace {

__device__ __forceinline__ void bbox_add(int2 p, int& mnx, int& mny, int& mxx, int& mxy, int& bad) {
  mnx = min(mnx, p.x); mny = min(mny, p.y); mxx = max(mxx, p.x); mxy = max(mxy, p.y);
  bad |= (p.x < 0 || p.y < 0 || p.x >= (1 << 24) || p.y >= (1 << 24));
}

// Warp reduction of a partial bounding box into out5 (atomics).
__device__ __forceinline__ void bbox_flush(int mnx, int mny, int mxx, int mxy, int bad, int32_t* out5) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mnx = min(mnx, __shfl_xor_sync(kFull, mnx, o));
    mny = min(mny, __shfl_xor_sync(kFull, mny, o));
    mxx = max(mxx, __shfl_xor_sync(kFull, mxx, o));
    mxy = max(mxy, __shfl_xor_sync(kFull, mxy, o));
    bad |= __shfl_xor_sync(kFull, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&out5[0], mnx);
    atomicMin(&out5[1], mny);
    atomicMax(&out5[2], mxx);
    atomicMax(&out5[3], mxy);
    if (bad) atomicOr(&out5[4], 1);
  }
}

__global__ void k_bbox_check(const int2* xy, int n, int32_t* out5) {
  int mnx = INT_MAX, mny = INT_MAX, mxx = INT_MIN, mxy = INT_MIN, bad = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    bbox_add(xy[i], mnx, mny, mxx, mxy, bad);
  bbox_flush(mnx, mny, mxx, mxy, bad, out5);
}

__device__ __forceinline__ int cell_of(const Grid& g, int2 p) {
  return ((p.y - g.miny) / g.cs) * g.gx + (p.x - g.minx) / g.cs;
}

__global__ void k_cell_count(const int2* xy, int n, Grid g, int32_t* count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&count[cell_of(g, xy[i])], 1);
}

// Exclusive scan of `count` into `start` (start[len] = total), one block;
// also into `cursor` when given (which may be `count` itself).
__device__ __forceinline__ void scan_i32_body(int32_t* count, int32_t* start, int len, int32_t* cursor) {
  __shared__ int32_t warp_tot[32];
  const int t = threadIdx.x, T = blockDim.x;
  const int chunk = (len + T - 1) / T;
  const int lo = min(len, t * chunk), hi = min(len, lo + chunk);
  int32_t s = 0;
  for (int i = lo; i < hi; ++i) s += count[i];
  const int lane = t & 31, w = t >> 5;
  int32_t incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    int32_t v = lane < (T >> 5) ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(kFull, v, o);
      if (lane >= o) v += y;
    }
    warp_tot[lane] = v;
  }
  __syncthreads();
  int32_t run = (incl - s) + (w > 0 ? warp_tot[w - 1] : 0);
  for (int i = lo; i < hi; ++i) {
    const int32_t ci = count[i];
    start[i] = run;
    if (cursor) cursor[i] = run;
    run += ci;
  }
  if (t == T - 1) start[len] = warp_tot[(T >> 5) - 1];
}

__global__ void __launch_bounds__(1024) k_scan_i32(int32_t* count, int32_t* start, int len) {
  scan_i32_body(count, start, len, nullptr);
}

__global__ void k_cell_fill(const int2* xy, int n, Grid g, int32_t* cursor, int32_t* pts, int4* recs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int2 p = xy[i];
  const int j = atomicAdd(&cursor[cell_of(g, p)], 1);
  pts[j] = i;
  if (recs) recs[j] = make_int4(i, p.x, p.y, i);
}

__device__ __forceinline__ void knn_body(const int2* xy, int n, const Grid& g, const int32_t* start,
                                         const int32_t* pts, int k, int bl, int32_t* cand, int32_t* backup,
                                         float* eta, int32_t* dcand, int u) {
  if (u >= n) return;
  const int K = k + bl;
  uint64_t bm[kMaxKnn];
  int32_t bi[kMaxKnn];
  int cnt = 0;
  const int2 q = xy[u];
  const int cx = (q.x - g.minx) / g.cs, cy = (q.y - g.miny) / g.cs;
  for (int r = 0;; ++r) {
    const int x0 = cx - r, x1 = cx + r, y0 = cy - r, y1 = cy + r;
    for (int yy = max(y0, 0); yy <= min(y1, g.gy - 1); ++yy) {
      const bool edge_row = (yy == y0 || yy == y1);
      for (int xx = max(x0, 0); xx <= min(x1, g.gx - 1); ++xx) {
        if (!edge_row && xx != x0 && xx != x1) {
          xx = x1 - 1;  // interior of the ring: jump to its right column
          continue;
        }
        const int c = yy * g.gx + xx;
        for (int j = start[c]; j < start[c + 1]; ++j) {
          const int v = pts[j];
          if (v == u) continue;
          const uint64_t m = sqdist(q, xy[v]);
          int pos;
          if (cnt < K) {
            pos = cnt++;
          } else if (m < bm[K - 1] || (m == bm[K - 1] && v < bi[K - 1])) {
            pos = K - 1;
          } else {
            continue;
          }
          while (pos > 0 && (m < bm[pos - 1] || (m == bm[pos - 1] && v < bi[pos - 1]))) {
            bm[pos] = bm[pos - 1];
            bi[pos] = bi[pos - 1];
            --pos;
          }
          bm[pos] = m;
          bi[pos] = v;
        }
      }
    }
    const bool lin = x0 <= 0, rin = x1 >= g.gx - 1, din = y0 <= 0, uin = y1 >= g.gy - 1;
    if (lin && rin && din && uin) break;  // every cell scanned
    if (cnt == K) {
      int64_t dmin = INT64_MAX;
      if (!lin) dmin = min(dmin, (int64_t)q.x - ((int64_t)g.minx + (int64_t)x0 * g.cs) + 1);
      if (!rin) dmin = min(dmin, ((int64_t)g.minx + (int64_t)(x1 + 1) * g.cs) - q.x);
      if (!din) dmin = min(dmin, (int64_t)q.y - ((int64_t)g.miny + (int64_t)y0 * g.cs) + 1);
      if (!uin) dmin = min(dmin, ((int64_t)g.miny + (int64_t)(y1 + 1) * g.cs) - q.y);
      if (bm[K - 1] < (uint64_t)(dmin * dmin)) break;
    }
  }
  for (int s = 0; s < k; ++s) {
    cand[(size_t)u * k + s] = bi[s];
    const int32_t d = euc2d_m(bm[s]);
    eta[(size_t)u * k + s] = d > 0 ? __fdiv_rn(1.0f, (float)d) : 1.0f;
    if (dcand) dcand[(size_t)u * k + s] = d;
  }
  for (int j = 0; j < bl; ++j) backup[(size_t)u * bl + j] = bi[k + j];
}

__global__ void __launch_bounds__(128) k_knn(const int2* xy, int n, Grid g, const int32_t* start,
                                             const int32_t* pts, int k, int bl, int32_t* cand,
                                             int32_t* backup, float* eta, int32_t* dcand) {
  knn_body(xy, n, g, start, pts, k, bl, cand, backup, eta, dcand, blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------
// Batch: the same steps for every colony of a batch; each block reads its
// colony and its block within the colony from a block map.
// ---------------------------------------------------------------------
__global__ void k_bbox_init_b(const ColonySetup* sets, int count) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= count) return;
  int32_t* b = sets[c].bb;
  b[0] = INT_MAX; b[1] = INT_MAX; b[2] = INT_MIN; b[3] = INT_MIN; b[4] = 0;
}

__global__ void k_bbox_b(const Colony* cols, const ColonySetup* sets, const int2* map) {
  const int2 e = map[blockIdx.x];
  const int i = e.y * blockDim.x + threadIdx.x;
  const int n = cols[e.x].n;
  int mnx = INT_MAX, mny = INT_MAX, mxx = INT_MIN, mxy = INT_MIN, bad = 0;
  if (i < n) bbox_add(cols[e.x].xy[i], mnx, mny, mxx, mxy, bad);
  bbox_flush(mnx, mny, mxx, mxy, bad, sets[e.x].bb);
}

// Grid of each colony from its bounding box, by the rule of the one-colony
// set-up: G = ceil(sqrt(n / 2)) cells per side of the square of the larger
// extent, so gx, gy <= G.
__global__ void k_grid_b(Colony* cols, const ColonySetup* sets, int count) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= count) return;
  const int32_t* b = sets[c].bb;
  const int n = cols[c].n;
  const int64_t ext = (int64_t)max(b[2] - b[0], b[3] - b[1]) + 1;
  int64_t G = (int64_t)ceil(sqrt((double)n / 2.0));
  if (G < 1) G = 1;
  Grid g;
  g.minx = b[0];
  g.miny = b[1];
  g.cs = (int32_t)((ext + G - 1) / G);
  if (g.cs < 1) g.cs = 1;
  g.gx = (b[2] - b[0]) / g.cs + 1;
  g.gy = (b[3] - b[1]) / g.cs + 1;
  cols[c].grid = g;
}

__global__ void k_cell_count_b(const Colony* cols, const ColonySetup* sets, const int2* map) {
  const int2 e = map[blockIdx.x];
  const int i = e.y * blockDim.x + threadIdx.x;
  const Colony C = cols[e.x];
  if (i < C.n) atomicAdd(&sets[e.x].cell_cnt[cell_of(C.grid, C.xy[i])], 1);
}

__global__ void __launch_bounds__(1024) k_cell_scan_b(const Colony* cols, const ColonySetup* sets) {
  const ColonySetup S = sets[blockIdx.x];
  const Grid g = cols[blockIdx.x].grid;
  scan_i32_body(S.cell_cnt, S.cell_start, g.gx * g.gy, S.cell_cnt);
}

__global__ void k_cell_fill_b(const Colony* cols, const ColonySetup* sets, const int2* map) {
  const int2 e = map[blockIdx.x];
  const int i = e.y * blockDim.x + threadIdx.x;
  const Colony C = cols[e.x];
  if (i >= C.n) return;
  const ColonySetup& S = sets[e.x];
  const int2 p = C.xy[i];
  const int j = atomicAdd(&S.cell_cnt[cell_of(C.grid, p)], 1);
  S.cell_pts[j] = i;
  S.cell_src[j] = make_int4(i, p.x, p.y, i);
}

__global__ void __launch_bounds__(128) k_knn_b(const Colony* cols, const ColonySetup* sets, const int2* map) {
  const int2 e = map[blockIdx.x];
  const Colony C = cols[e.x];
  const ColonySetup S = sets[e.x];
  knn_body(C.xy, C.n, C.grid, S.cell_start, S.cell_pts, C.k, C.bl, S.cand, S.backup, S.eta, S.dcand,
           e.y * blockDim.x + threadIdx.x);
}

}  // namespace

cudaError_t launch_grid_batch(Colony* cols, const ColonySetup* sets, int count, const int2* map256, int nmap256,
                              cudaStream_t s) {
  k_bbox_init_b<<<(count + 127) / 128, 128, 0, s>>>(sets, count);
  k_bbox_b<<<nmap256, 256, 0, s>>>(cols, sets, map256);
  k_grid_b<<<(count + 127) / 128, 128, 0, s>>>(cols, sets, count);
  return cudaGetLastError();
}

// The cell counts must be zero on entry.
cudaError_t build_lists_batch(const Colony* cols, const ColonySetup* sets, int count, const int2* map256,
                              int nmap256, const int2* map128, int nmap128, cudaStream_t s) {
  k_cell_count_b<<<nmap256, 256, 0, s>>>(cols, sets, map256);
  k_cell_scan_b<<<count, 256, 0, s>>>(cols, sets);
  k_cell_fill_b<<<nmap256, 256, 0, s>>>(cols, sets, map256);
  k_knn_b<<<nmap128, 128, 0, s>>>(cols, sets, map128);
  return cudaGetLastError();
}

cudaError_t launch_bbox_check(const int2* xy, int n, int32_t* out5, cudaStream_t s) {
  const int32_t init[5] = {INT_MAX, INT_MAX, INT_MIN, INT_MIN, 0};
  cudaError_t e = cudaMemcpyAsync(out5, init, sizeof(init), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const int blocks = min(1024, (n + 255) / 256);
  k_bbox_check<<<blocks, 256, 0, s>>>(xy, n, out5);
  return cudaGetLastError();
}

cudaError_t build_lists(const int2* xy, int n, int k, int bl, const Grid& g, int32_t* cell_count,
                        int32_t* cell_start, int32_t* cell_pts, int4* cell_src, int32_t* cand, int32_t* backup,
                        float* eta, int32_t* dcand, cudaStream_t s) {
  const int cells = g.gx * g.gy;
  cudaError_t e = cudaMemsetAsync(cell_count, 0, sizeof(int32_t) * cells, s);
  if (e != cudaSuccess) return e;
  k_cell_count<<<(n + 255) / 256, 256, 0, s>>>(xy, n, g, cell_count);
  k_scan_i32<<<1, 1024, 0, s>>>(cell_count, cell_start, cells);
  e = cudaMemcpyAsync(cell_count, cell_start, sizeof(int32_t) * cells, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  k_cell_fill<<<(n + 255) / 256, 256, 0, s>>>(xy, n, g, cell_count, cell_pts, cell_src);
  k_knn<<<(n + 127) / 128, 128, 0, s>>>(xy, n, g, cell_start, cell_pts, k, bl, cand, backup, eta, dcand);
  return cudaGetLastError();
}

}  // namespace faco
