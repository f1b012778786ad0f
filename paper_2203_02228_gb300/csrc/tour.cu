// tour.cu -- the initial solution of Alg 2 (Sec. 4.3): nearest-neighbour
// tour from node 0 -- first unvisited candidate, else first unvisited backup
// entry, else the globally nearest unvisited node by (squared distance, id)
// -- improved by the local search with every node queued in tour order.
// Both steps are sequential by definition; each runs on one warp.
//
// Also: small device self-test kernels (Philox, EUC_2D, roulette) that the
// tests call through the library to compare with their own expectations.
#include <climits>

#include "common.cuh"
#include "launch.h"
#include "ls.cuh"
#include "nearest.cuh"

namespace faco {

namespace {

__device__ __forceinline__ void nn_tour_body(const int2* xy, int n, const int32_t* cand, int k,
                                             const int32_t* backup, int bl, int32_t* route, uint32_t* vis,
                                             const Grid& g, const int32_t* cstart, const int32_t* cpts) {
  const int lane = lane_id();
  const int words = (n + 31) >> 5;
  for (int i = lane; i < words; i += 32) vis[i] = 0;
  __syncwarp();
  if (lane == 0) {
    route[0] = 0;
    vis[0] = 1u;
  }
  __syncwarp();
  int u = 0;
  for (int i = 1; i < n; ++i) {
    int v = -1;
    {
      const int c = lane < k ? cand[(size_t)u * k + lane] : -1;
      const bool ok = c >= 0 && !((vis[c >> 5] >> (c & 31)) & 1u);
      const unsigned bal = __ballot_sync(kFull, ok);
      if (bal) v = __shfl_sync(kFull, c, __ffs(bal) - 1);
    }
    for (int j0 = 0; v < 0 && j0 < bl; j0 += 32) {
      const int j = j0 + lane;
      const int c = j < bl ? backup[(size_t)u * bl + j] : -1;
      const bool ok = c >= 0 && !((vis[c >> 5] >> (c & 31)) & 1u);
      const unsigned bal = __ballot_sync(kFull, ok);
      if (bal) v = __shfl_sync(kFull, c, __ffs(bal) - 1);
    }
    if (v < 0) {
      // global nearest unvisited node: rings of grid cells, else a scan of
      // the visited words that skips full ones
      const int2 xu = xy[u];
      v = ring_nearest(xy, g, cstart, cpts, xu, 24,
                       [&](int x) { return ((vis[x >> 5] >> (x & 31)) & 1u) != 0; });
    }
    if (v < 0) {
      const int2 xu = xy[u];
      uint64_t bk = ~0ull;
      int32_t bi = INT_MAX;
      for (int wi = lane; wi < words; wi += 32) {
        uint32_t fr = ~vis[wi];
        if (wi == words - 1 && (n & 31)) fr &= (1u << (n & 31)) - 1u;
        while (fr) {
          const int w = wi * 32 + __ffs(fr) - 1;
          fr &= fr - 1;
          const uint64_t m = sqdist(xu, xy[w]);
          if (m < bk || (m == bk && w < bi)) {
            bk = m;
            bi = w;
          }
        }
      }
      warp_min_key(bk, bi);
      v = (bi >= 0 && bi < n) ? bi : 0;  // bi is valid while a node is unvisited
    }
    if (lane == 0) {
      route[i] = v;
      vis[v >> 5] |= 1u << (v & 31);
    }
    __syncwarp();
    u = v;
  }
}

__global__ void __launch_bounds__(32) k_nn_tour(const int2* xy, int n, const int32_t* cand, int k,
                                                const int32_t* backup, int bl, int32_t* route,
                                                uint32_t* vis_g, Grid g, const int32_t* cstart,
                                                const int32_t* cpts) {
  extern __shared__ uint32_t sv[];
  nn_tour_body(xy, n, cand, k, backup, bl, route, vis_g ? vis_g : sv, g, cstart, cpts);
}

// Batch: one warp per colony, visited bits in shared memory.
__global__ void __launch_bounds__(32) k_nn_tour_b(const Colony* cols, const ColonySetup* sets) {
  extern __shared__ uint32_t sv[];
  const Colony C = cols[blockIdx.x];
  const ColonySetup S = sets[blockIdx.x];
  nn_tour_body(C.xy, C.n, S.cand, C.k, S.backup, C.bl, S.init_route, sv, C.grid, S.cell_start, S.cell_pts);
}

// Reverse the forward span x..y (or its complement) with the whole block.
__device__ void cta_flip(ArrTour& T, int x, int y) {
  const int n = T.n;
  __syncthreads();
  int i = T.pos[x], j = T.pos[y];
  __syncthreads();  // every thread has read i, j before any position moves
  int L = j - i;
  if (L < 0) L += n;
  L += 1;
  if (2 * L > n) {
    const int i2 = (j + 1 == n) ? 0 : j + 1;
    const int j2 = (i == 0) ? n - 1 : i - 1;
    i = i2;
    j = j2;
    L = n - L;
  }
  const int half = L >> 1;
  for (int t = threadIdx.x; t < half; t += blockDim.x) {
    int ia = i + t;
    if (ia >= n) ia -= n;
    int ib = j - t;
    if (ib < 0) ib += n;
    const int va = T.route[ia], vb = T.route[ib];
    T.route[ia] = vb;
    T.route[ib] = va;
    T.pos[vb] = ia;
    T.pos[va] = ib;
  }
  __syncthreads();
}

__device__ void cta_move2(ArrTour& T, int n1, int n2, int n3, int n4) {
  const bool fwd = T.succ(n1) == n2;
  if (fwd)
    cta_flip(T, n2, n3);
  else
    cta_flip(T, n1, n4);
}

// The local search of ls_array.cuh with every node queued (the initial
// tour), run by one block of 32 warps.  Each round, warp w evaluates the
// w-th queued node on the current tour; the entries are then popped in
// queue order up to and including the first one that found a move, which
// is applied.  Nothing changes the tour between the confirmed evaluations,
// so the result is exactly that of popping one node at a time.
__device__ __forceinline__ void init_ls_body(const int2* xy, int n, const int32_t* cand, int k, int oropt,
                                             int verify, int32_t* route, int32_t* pos, int32_t* queue,
                                             uint8_t* flags, int32_t* logb) {
  __shared__ int64_t s_gain[32];
  __shared__ int s_mv[32][8];
  __shared__ int s_qh, s_qn, s_nlog, s_changes, s_moves_round, s_win;
  LsEnv E{n, oropt, verify, queue, flags, logb};
  ArrTour T{n, k, route, pos, xy, cand, k};
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  for (int i = tid; i < n; i += blockDim.x) {
    const int x = route[i];
    queue[i] = x;
    flags[x] = 1;
  }
  if (tid == 0) {
    s_qh = 0; s_qn = n; s_nlog = 0; s_changes = 0; s_moves_round = 0;
  }
  __syncthreads();
  for (;;) {
    const int qh = s_qh, qn = s_qn;
    if (qn == 0 || s_changes >= n) {
      if (s_changes >= n || !verify || s_moves_round == 0) break;
      const int nl = s_nlog;  // verify round: queue again the nodes popped
      for (int i = tid; i < nl; i += blockDim.x) {
        const int x = logb[i];
        queue[i] = x;
        flags[x] = 1;
      }
      __syncthreads();
      if (tid == 0) {
        s_qh = 0; s_qn = nl; s_nlog = 0; s_moves_round = 0;
      }
      __syncthreads();
      continue;
    }
    const int W = qn < 32 ? qn : 32;
    if (w < W) {
      int idx = qh + w;
      if (idx >= n) idx -= n;
      const int a = queue[idx];
      int mv2[4], mvo[7];
      int64_t g2, go;
      eval_both(T, a, oropt != 0, g2, mv2, go, mvo);
      if (lane == 0) {
        if (g2 > 0) {
          s_gain[w] = g2;
          for (int t = 0; t < 4; ++t) s_mv[w][t] = mv2[t];
          s_mv[w][7] = 0;
        } else {
          s_gain[w] = go > 0 ? go : 0;
          for (int t = 0; t < 7; ++t) s_mv[w][t] = mvo[t];
          s_mv[w][7] = 1;
        }
      }
    }
    __syncthreads();
    if (w == 0) {
      const unsigned bal = __ballot_sync(kFull, lane < W && s_gain[lane] > 0);
      const int first = bal ? __ffs(bal) - 1 : W;
      const int cnt = bal ? first + 1 : W;  // queue entries popped this round
      int a = -1;
      bool first_pop = false;
      if (lane < cnt) {
        int idx = qh + lane;
        if (idx >= n) idx -= n;
        a = queue[idx];
        const uint8_t f = flags[a];
        first_pop = !(f & 2);
        flags[a] = (uint8_t)((f & ~1) | 2);
      }
      const unsigned fb = __ballot_sync(kFull, first_pop);
      if (first_pop) logb[s_nlog + __popc(fb & ((1u << lane) - 1u))] = a;
      __syncwarp();
      if (lane == 0) {
        s_nlog += __popc(fb);
        int h = qh + cnt;
        if (h >= n) h -= n;
        s_qh = h;
        s_qn = qn - cnt;
        s_win = bal ? first : -1;
      }
    }
    __syncthreads();
    const int win = s_win;
    if (win >= 0) {
      int mv[8];
      for (int t = 0; t < 8; ++t) mv[t] = s_mv[win][t];
      if (mv[7] == 0) {
        cta_flip(T, mv[1], mv[2]);
      } else {
        cta_move2(T, mv[0], mv[1], mv[4], mv[5]);
        cta_move2(T, mv[0], mv[4], mv[3], mv[2]);
        if (mv[6]) cta_move2(T, mv[4], mv[2], mv[1], mv[5]);
      }
      if (w == 0) {
        const int qn2 = ls_push_warp(E, mv, mv[7] == 0 ? 4 : 6, s_qh, s_qn);
        if (lane == 0) {
          s_qn = qn2;
          s_changes++;
          s_moves_round++;
        }
      }
      __syncthreads();
    }
  }
  __syncthreads();
  const int qh = s_qh, qn = s_qn, nl = s_nlog;
  for (int t = tid; t < qn; t += blockDim.x) {
    int i = qh + t;
    if (i >= n) i -= n;
    flags[queue[i]] = 0;
  }
  for (int i = tid; i < nl; i += blockDim.x) flags[logb[i]] = 0;
}

__global__ void __launch_bounds__(1024) k_init_ls(const int2* xy, int n, const int32_t* cand, int k,
                                                  int oropt, int verify, int32_t* route, int32_t* pos,
                                                  int32_t* queue, uint8_t* flags, int32_t* logb) {
  init_ls_body(xy, n, cand, k, oropt, verify, route, pos, queue, flags, logb);
}

// Batch: one block per colony; positions of the initial tour in src_pos.
__global__ void __launch_bounds__(1024) k_init_ls_b(const Colony* cols, const ColonySetup* sets) {
  const Colony C = cols[blockIdx.x];
  const ColonySetup S = sets[blockIdx.x];
  init_ls_body(C.xy, C.n, S.cand, C.k, C.oropt, C.verify, S.init_route, C.src_pos, S.queue, S.flags, S.logb);
}

// what = 0: Philox draws   in: uint32 [count][4] = (idx, ant, iter, tag) -> out uint32
// what = 1: EUC_2D         in: int32 [count][4] = (x1, y1, x2, y2)       -> out int32
// what = 2: roulette       in: float [count][width + 1] (weights, u)     -> out int32
__global__ void k_tests(int what, const void* in, void* out, int count, int width, uint64_t seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  if (what == 0) {
    const uint32_t* a = static_cast<const uint32_t*>(in) + 4 * i;
    static_cast<uint32_t*>(out)[i] = draw(seed, a[0], a[1], a[2], a[3]);
  } else if (what == 1) {
    const int32_t* a = static_cast<const int32_t*>(in) + 4 * i;
    static_cast<int32_t*>(out)[i] = euc2d(make_int2(a[0], a[1]), make_int2(a[2], a[3]));
  } else {
    const float* a = static_cast<const float*>(in) + (size_t)(width + 1) * i;
    int r;
    if (width == 16) {
      float w[16];
      for (int s = 0; s < 16; ++s) w[s] = a[s];
      r = roulette<16>(w, a[16]);
    } else {
      float w[32];
      for (int s = 0; s < 32; ++s) w[s] = a[s];
      r = roulette<32>(w, a[32]);
    }
    static_cast<int32_t*>(out)[i] = r;
  }
}

}  // namespace

cudaError_t launch_nn_tour(const int2* xy, int n, const int32_t* cand, int k, const int32_t* backup,
                           int bl, int32_t* route, uint32_t* vis_g, const Grid& g, const int32_t* cstart,
                           const int32_t* cpts, cudaStream_t s) {
  const size_t smem = vis_g ? 0 : (size_t)((n + 31) >> 5) * sizeof(uint32_t);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_nn_tour, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_nn_tour<<<1, 32, smem, s>>>(xy, n, cand, k, backup, bl, route, vis_g, g, cstart, cpts);
  return cudaGetLastError();
}

cudaError_t launch_init_ls(const int2* xy, int n, const int32_t* cand, int k, int oropt, int verify,
                           int32_t* route, int32_t* pos, int32_t* queue, uint8_t* flags,
                           int32_t* logb, cudaStream_t s) {
  k_init_ls<<<1, 1024, 0, s>>>(xy, n, cand, k, oropt, verify, route, pos, queue, flags, logb);
  return cudaGetLastError();
}

cudaError_t launch_init_tour_batch(const Colony* cols, const ColonySetup* sets, int count, int max_n, int stage,
                                   cudaStream_t s) {
  if (stage == 0) {
    const size_t smem = (size_t)((max_n + 31) >> 5) * sizeof(uint32_t);
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_nn_tour_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    k_nn_tour_b<<<count, 32, smem, s>>>(cols, sets);
  } else {
    k_init_ls_b<<<count, 1024, 0, s>>>(cols, sets);
  }
  return cudaGetLastError();
}

cudaError_t launch_test_kernels(int what, const void* in, void* out, int count, int width,
                                uint64_t seed, cudaStream_t s) {
  k_tests<<<(count + 127) / 128, 128, 0, s>>>(what, in, out, count, width, seed);
  return cudaGetLastError();
}

}  // namespace faco
