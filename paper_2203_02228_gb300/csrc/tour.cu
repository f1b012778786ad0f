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
                                             const Grid& g, const int32_t* cstart, const int4* recs) {
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
      // the next node is most often one of these: their own lists start on
      // their way to L1 now, off the chain of dependent steps
      if (c >= 0) prefetch_l1(cand + (size_t)c * k);
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
      int h;
      v = ring_nearest(recs, g, cstart, xu, 24,
                       [&](const int4& P) { return ((vis[P.w >> 5] >> (P.w & 31)) & 1u) != 0; }, h);
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
                                                const int4* recs) {
  extern __shared__ uint32_t sv[];
  nn_tour_body(xy, n, cand, k, backup, bl, route, vis_g ? vis_g : sv, g, cstart, recs);
}

// Batch: one warp per colony, visited bits in shared memory.
__global__ void __launch_bounds__(32) k_nn_tour_b(const Colony* cols, const ColonySetup* sets) {
  extern __shared__ uint32_t sv[];
  const Colony C = cols[blockIdx.x];
  const ColonySetup S = sets[blockIdx.x];
  nn_tour_body(C.xy, C.n, S.cand, C.k, S.backup, C.bl, S.init_route, sv, C.grid, S.cell_start, S.cell_src);
}

// Positions reversed by one move (at most three flips): first position and
// length of each reversed span, appended by thread 0.
struct SpanLog {
  int2 span[3];
  int count;
};

// The initial search's tour with its positions in shared memory (n up to
// about 106k nodes fits): the low 16 bits of each position in lo[n], bit 16
// in the bitmap hi.  Otherwise the same lookups as ArrTour.
struct SmemPosTour {
  int n, k;
  int32_t* route;
  uint16_t* lo;
  uint32_t* hi;
  const int2* xy;
  const int32_t* cn;
  const int32_t* cd;
  __device__ __forceinline__ int pos_of(int x) const {
    return (int)lo[x] | (int)(((hi[x >> 5] >> (x & 31)) & 1u) << 16);
  }
  // x moves from position `from` to `to`; each node moves by one thread at a
  // time, but the 32 nodes of a bitmap word may move together
  __device__ __forceinline__ void move_pos(int x, int from, int to) {
    lo[x] = (uint16_t)to;
    if ((from ^ to) >> 16) atomicXor(&hi[x >> 5], 1u << (x & 31));
  }
  __device__ __forceinline__ int at_off(int p, int d) const {
    p += d;
    if (p >= n) p -= n;
    if (p < 0) p += n;
    return route[p];
  }
  __device__ __forceinline__ int succ(int x) const { return at_off(pos_of(x), 1); }
  __device__ __forceinline__ int adj(int x, bool up) const { return at_off(pos_of(x), up ? 1 : -1); }
  __device__ __forceinline__ void nbrs(int x, int& p, int& s) const {
    const int t = pos_of(x);
    p = at_off(t, -1);
    s = at_off(t, 1);
  }
  __device__ __forceinline__ void walk(int a, int& p, int& s1, int& s2, int& s3) const {
    const int t = pos_of(a);
    p = at_off(t, -1);
    s1 = at_off(t, 1);
    s2 = at_off(t, 2);
    s3 = at_off(t, 3);
  }
  __device__ __forceinline__ int2 coord(int x) const { return xy[x]; }
  __device__ __forceinline__ int cand(int x, int s) const { return cn[(size_t)x * k + s]; }
  __device__ __forceinline__ int cdist(int x, int s) const { return cd[(size_t)x * k + s]; }
};

// Shared-memory bytes of an n-node SmemPosTour.
__host__ __device__ __forceinline__ size_t smem_pos_bytes(int n) {
  return (((size_t)n * 2 + 15) & ~(size_t)15) + (size_t)((n + 31) >> 5) * 4;
}

__device__ __forceinline__ SmemPosTour smem_pos_tour(unsigned char* sm, int n, int k, int32_t* route,
                                                     const int2* xy, const int32_t* cand, const int32_t* dcand) {
  SmemPosTour T;
  T.n = n;
  T.k = k;
  T.route = route;
  T.lo = reinterpret_cast<uint16_t*>(sm);
  T.hi = reinterpret_cast<uint32_t*>(sm + (((size_t)n * 2 + 15) & ~(size_t)15));
  T.xy = xy;
  T.cn = cand;
  T.cd = dcand;
  return T;
}

// Positions of the tour `route` into T (block).
__device__ __forceinline__ void smem_pos_load(SmemPosTour& T) {
  const int n = T.n;
  for (int w = threadIdx.x; w < ((n + 31) >> 5); w += blockDim.x) T.hi[w] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int x = T.route[i];
    T.lo[x] = (uint16_t)i;
    if (i >> 16) atomicOr(&T.hi[x >> 5], 1u << (x & 31));
  }
  __syncthreads();
}

// Reverse the forward span x..y (or its complement) with the whole block;
// the span actually reversed goes to the log.  Every caller reaches it
// after a block barrier that follows the last write to the tour.
template <class TT>
__device__ void cta_flip(TT& T, int x, int y, SpanLog& log) {
  const int n = T.n;
  int i = T.pos_of(x), j = T.pos_of(y);
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
  if (threadIdx.x == 0 && log.count < 3) log.span[log.count++] = make_int2(i, L);
  const int half = L >> 1;
  for (int t = threadIdx.x; t < half; t += blockDim.x) {
    int ia = i + t;
    if (ia >= n) ia -= n;
    int ib = j - t;
    if (ib < 0) ib += n;
    const int va = T.route[ia], vb = T.route[ib];
    T.route[ia] = vb;
    T.route[ib] = va;
    T.move_pos(vb, ib, ia);
    T.move_pos(va, ia, ib);
  }
  __syncthreads();
}

template <class TT>
__device__ void cta_move2(TT& T, int n1, int n2, int n3, int n4, SpanLog& log) {
  const bool fwd = T.succ(n1) == n2;
  if (fwd)
    cta_flip(T, n2, n3, log);
  else
    cta_flip(T, n1, n4, log);
}

// true when position p lies in the cyclic span (first position i, length L).
__device__ __forceinline__ bool in_span(int p, int2 sp, int n) {
  int d = p - sp.x;
  if (d < 0) d += n;
  return d < sp.y;
}

// The local search with every node queued (the initial tour), run by one
// block of 32 warps over a window of the next 32 queued nodes.  Each window
// entry keeps its evaluation -- the best 2-opt / Or-opt move from its node
// on the tour as it was -- together with the tour positions that evaluation
// read (the node's, the next three and the previous one; each candidate's
// and its two neighbours').  A move reverses spans of positions; an entry
// whose positions meet none of them would evaluate to the same result, so
// it is kept, the others are dropped.  Each round pops entries in queue
// order up to and including the first one whose evaluation found a move,
// which is applied.  An evaluation runs only when an entry without one
// comes before the first improving entry (all entries without one are then
// evaluated, a warp each).  The pops, moves and queue are exactly those of
// popping one node at a time.
constexpr int kWin = 32;

template <class TT>
__device__ __forceinline__ void init_ls_body(TT& T, int oropt, int verify, int init3, int32_t* queue, uint8_t* flags,
                                             int32_t* logb) {
  __shared__ int64_t s_gain[kWin];
  __shared__ int s_mv[kWin][8];
  __shared__ int s_any[kWin];             // 1: the evaluation read beyond s_dep (3-opt scan): any move drops it
  __shared__ int s_node[kWin];            // node whose evaluation the slot holds, -1: none
  __shared__ int s_dep[kWin][kMaxK + 1];  // [0]: its position, [1 + s]: candidate s's position
  __shared__ SpanLog s_log;
  __shared__ int s_qh, s_qn, s_nlog, s_changes, s_moves_round, s_win, s_base;
  const int n = T.n, k = T.k;
  int32_t* route = T.route;
  LsEnv E{n, oropt, verify, queue, flags, logb};
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  for (int i = tid; i < n; i += blockDim.x) {
    const int x = route[i];
    queue[i] = x;
    flags[x] = 1;
  }
  if (tid < kWin) s_node[tid] = -1;
  if (tid == 0) {
    s_qh = 0; s_qn = n; s_nlog = 0; s_changes = 0; s_moves_round = 0; s_base = 0;
  }
  __syncthreads();
  for (;;) {
    const int qh = s_qh, qn = s_qn, base = s_base;
    if (qn == 0 || s_changes >= n) {
      if (s_changes >= n || !verify || s_moves_round == 0) break;
      const int nl = s_nlog;  // verify round: queue again the nodes popped
      for (int i = tid; i < nl; i += blockDim.x) {
        const int x = logb[i];
        queue[i] = x;
        flags[x] = 1;
      }
      __syncthreads();
      if (tid < kWin) s_node[tid] = -1;  // the queue changed: no evaluation carries over
      if (tid == 0) {
        s_qh = 0; s_qn = nl; s_nlog = 0; s_moves_round = 0; s_base = 0;
      }
      __syncthreads();
      continue;
    }
    // window offset `lane` of every warp: its node, slot, and whether its
    // evaluation is there and improves
    const int R = qn < kWin ? qn : kWin;
    const int slot = (base + lane) & (kWin - 1);
    int node = -1;
    bool have = false, impr = false;
    if (lane < R) {
      int idx = qh + lane;
      if (idx >= n) idx -= n;
      node = queue[idx];
      have = s_node[slot] == node;
      impr = have && s_gain[slot] > 0;
    }
    const unsigned bimp = __ballot_sync(kFull, impr);
    const unsigned bmiss = __ballot_sync(kFull, lane < R && !have);
    const int f = bimp ? __ffs(bimp) - 1 : R;
    const unsigned before = f >= 32 ? kFull : ((1u << f) - 1u);
    __syncthreads();  // every warp has decided (from the same slots) before any slot is written
    if (bmiss & before) {  // an entry without an evaluation comes first: evaluate every such entry
      const int my_node = __shfl_sync(kFull, node, w & 31);
      const int my_slot = (base + w) & (kWin - 1);
      if (w < R && ((bmiss >> w) & 1u)) {
        int mv2[4], mvo[7], mv3[6];
        int64_t g2, go, g3 = 0;
        eval_both(T, my_node, oropt != 0, g2, mv2, go, mvo);
        // the 3-opt exchange only when neither 2-opt nor Or-opt improves
        // (g2, go are the warp's reductions: the branch is warp-uniform)
        const bool try3 = init3 && !(g2 > 0) && !(go > 0);
        if (try3) g3 = eval_or3(T, my_node, mv3);
        if (lane < k) s_dep[my_slot][1 + lane] = T.pos_of(T.cand(my_node, lane));
        if (lane == 0) {
          s_dep[my_slot][0] = T.pos_of(my_node);
          if (g2 > 0) {
            s_gain[my_slot] = g2;
            for (int t = 0; t < 4; ++t) s_mv[my_slot][t] = mv2[t];
            s_mv[my_slot][7] = 0;
          } else if (g3 > 0) {
            s_gain[my_slot] = g3;
            for (int t = 0; t < 6; ++t) s_mv[my_slot][t] = mv3[t];
            s_mv[my_slot][7] = 2;
          } else {
            s_gain[my_slot] = go > 0 ? go : 0;
            for (int t = 0; t < 7; ++t) s_mv[my_slot][t] = mvo[t];
            s_mv[my_slot][7] = 1;
          }
          s_any[my_slot] = try3 ? 1 : 0;
          s_node[my_slot] = my_node;
        }
      }
      __syncthreads();
    }
    if (w == 0) {
      const unsigned bal = __ballot_sync(kFull, lane < R && s_gain[slot] > 0);
      const int first = bal ? __ffs(bal) - 1 : R;
      const int cnt = bal ? first + 1 : R;  // queue entries popped this round
      bool first_pop = false;
      if (lane < cnt) {
        const uint8_t fl = flags[node];
        first_pop = !(fl & 2);
        flags[node] = (uint8_t)((fl & ~1) | 2);
      }
      const unsigned fb = __ballot_sync(kFull, first_pop);
      if (first_pop) logb[s_nlog + __popc(fb & ((1u << lane) - 1u))] = node;
      const int win_slot = (base + first) & (kWin - 1);
      __syncwarp();
      if (lane < cnt && lane != first) s_node[slot] = -1;  // popped: the slots are free
      if (lane == 0) {
        s_nlog += __popc(fb);
        int h = qh + cnt;
        if (h >= n) h -= n;
        s_qh = h;
        s_qn = qn - cnt;
        s_base = (base + cnt) & (kWin - 1);
        s_win = bal ? win_slot : -1;
        s_log.count = 0;
      }
    }
    __syncthreads();
    const int win = s_win;
    if (win >= 0) {
      int mv[8];
      for (int t = 0; t < 8; ++t) mv[t] = s_mv[win][t];
      // the slot is free (its move is not overwritten before the next
      // evaluation phase, several barriers on); the warp checking it below
      // may still read the old node, which leaves the slot free either way
      if (tid == 0) s_node[win] = -1;
      if (mv[7] == 0) {
        cta_flip(T, mv[1], mv[2], s_log);
      } else if (mv[7] == 1) {
        cta_move2(T, mv[0], mv[1], mv[4], mv[5], s_log);
        cta_move2(T, mv[0], mv[4], mv[3], mv[2], s_log);
        if (mv[6]) cta_move2(T, mv[4], mv[2], mv[1], mv[5], s_log);
      } else {  // 3-opt exchange {a, t2, b, b', c, c'} as three edge exchanges
        cta_move2(T, mv[0], mv[1], mv[2], mv[3], s_log);  // {a,t2},{b,b'} -> {a,b},{t2,b'}
        cta_move2(T, mv[0], mv[2], mv[4], mv[5], s_log);  // {a,b},{c,c'} -> {a,c},{b,c'}
        cta_move2(T, mv[0], mv[4], mv[3], mv[1], s_log);  // {a,c},{b',t2} -> {a,b'},{c,t2}
      }
      // drop the evaluations that read a reversed position (warp w checks slot w)
      {
        const int sn = s_node[w];
        if (sn >= 0) {
          const int ns = s_log.count;
          bool hit = s_any[w] != 0;
          if (lane < k) {
            const int tb = s_dep[w][1 + lane];
            for (int q = 0; q < ns && !hit; ++q) {
              const int2 sp = s_log.span[q];
              hit = in_span(tb, sp, n) || in_span(tb == 0 ? n - 1 : tb - 1, sp, n) ||
                    in_span(tb + 1 == n ? 0 : tb + 1, sp, n);
            }
          }
          if (lane == 31 && !hit) {
            const int t0 = s_dep[w][0];
            for (int q = 0; q < ns && !hit; ++q) {
              const int2 sp = s_log.span[q];
              for (int d = -1; d <= 3 && !hit; ++d) {
                int p = t0 + d;
                if (p < 0) p += n;
                if (p >= n) p -= n;
                hit = in_span(p, sp, n);
              }
            }
          }
          if (__any_sync(kFull, hit) && lane == 0) s_node[w] = -1;
        }
      }
      if (w == 0) {
        const int qn2 = ls_push_warp(E, mv, mv[7] == 0 ? 4 : 6, s_qh, s_qn);  // 2-opt: 4 ends, else 6
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

// SP: the positions live in shared memory during the search (launched with
// smem_pos_bytes(n) of it) and are written to `pos` at the end; otherwise
// the search works on `pos` in global memory.
template <bool SP>
__device__ __forceinline__ void init_ls_run(const int2* xy, int n, const int32_t* cand, const int32_t* dcand, int k,
                                            int oropt, int verify, int init3, int32_t* route, int32_t* pos,
                                            int32_t* queue, uint8_t* flags, int32_t* logb) {
  if constexpr (SP) {
    extern __shared__ __align__(16) unsigned char s_pos[];
    SmemPosTour T = smem_pos_tour(s_pos, n, k, route, xy, cand, dcand);
    smem_pos_load(T);
    init_ls_body(T, oropt, verify, init3, queue, flags, logb);
    __syncthreads();
    for (int x = threadIdx.x; x < n; x += blockDim.x) pos[x] = T.pos_of(x);
  } else {
    ArrTour T{n, k, route, pos, xy, cand, k, dcand};
    init_ls_body(T, oropt, verify, init3, queue, flags, logb);
  }
}

template <bool SP>
__global__ void __launch_bounds__(1024) k_init_ls(const int2* xy, int n, const int32_t* cand,
                                                  const int32_t* dcand, int k, int oropt, int verify, int init3,
                                                  int32_t* route, int32_t* pos, int32_t* queue, uint8_t* flags,
                                                  int32_t* logb) {
  init_ls_run<SP>(xy, n, cand, dcand, k, oropt, verify, init3, route, pos, queue, flags, logb);
}

// Batch: one block per colony; positions of the initial tour in src_pos.
template <bool SP>
__global__ void __launch_bounds__(1024) k_init_ls_b(const Colony* cols, const ColonySetup* sets) {
  const Colony C = cols[blockIdx.x];
  const ColonySetup S = sets[blockIdx.x];
  init_ls_run<SP>(C.xy, C.n, S.cand, S.dcand, C.k, C.oropt, C.verify, C.init3, S.init_route, C.src_pos, S.queue, S.flags,
                  S.logb);
}

// Shared memory for positions of up to n nodes if kernel f can take it,
// else 0 (the positions then stay in global memory).
size_t init_ls_pos_smem(const void* f, int n) {
  const size_t b = smem_pos_bytes(n);
  if (allow_dyn_smem(f, b) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return b;
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

// The initial search names nodes by their position in the nearest-
// neighbour tour: node i of the copies is route0[i], and a candidate list
// names its entries the same way.  Lists keep their order and coordinates
// their values, so every decision of the search is the same; what changes is
// where things lie in memory -- consecutive names are neighbours on the walk,
// so a node's coordinates, lists and tour neighbours share cache lines with
// those of the nodes around it.  One thread per list entry.
__global__ void k_relabel(const int32_t* __restrict__ route0, const int32_t* __restrict__ pos0,
                          const int2* __restrict__ xy, const int32_t* __restrict__ cand,
                          const int32_t* __restrict__ dcand, int n, int k, int2* __restrict__ xy_t,
                          int32_t* __restrict__ cand_t, int32_t* __restrict__ dcand_t,
                          int32_t* __restrict__ route_t, int32_t* __restrict__ pos_t) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)n * k) return;
  const int i = (int)(e / k), s = (int)(e - (size_t)i * k);
  const int u = route0[i];
  const int c = cand[(size_t)u * k + s];
  cand_t[e] = c >= 0 ? pos0[c] : c;
  dcand_t[e] = dcand[(size_t)u * k + s];
  if (s == 0) {
    xy_t[i] = xy[u];
    route_t[i] = i;
    pos_t[i] = i;
  }
}

// route[t] = route0[route_t[t]]: the searched tour back in node ids.
__global__ void k_unlabel(const int32_t* __restrict__ route0, const int32_t* __restrict__ route_t,
                          int32_t* __restrict__ route, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) route[t] = route0[route_t[t]];
}

}  // namespace

cudaError_t launch_nn_tour(const int2* xy, int n, const int32_t* cand, int k, const int32_t* backup,
                           int bl, int32_t* route, uint32_t* vis_g, const Grid& g, const int32_t* cstart,
                           const int4* recs, cudaStream_t s) {
  const size_t smem = vis_g ? 0 : (size_t)((n + 31) >> 5) * sizeof(uint32_t);
  if (smem > 48 * 1024) {
    cudaError_t e = allow_dyn_smem(reinterpret_cast<const void*>(k_nn_tour), smem);
    if (e != cudaSuccess) return e;
  }
  k_nn_tour<<<1, 32, smem, s>>>(xy, n, cand, k, backup, bl, route, vis_g, g, cstart, recs);
  return cudaGetLastError();
}

cudaError_t launch_relabel(const int32_t* route0, const int32_t* pos0, const int2* xy, const int32_t* cand,
                           const int32_t* dcand, int n, int k, int2* xy_t, int32_t* cand_t, int32_t* dcand_t,
                           int32_t* route_t, int32_t* pos_t, cudaStream_t s) {
  const size_t e = (size_t)n * k;
  k_relabel<<<(unsigned)((e + 255) / 256), 256, 0, s>>>(route0, pos0, xy, cand, dcand, n, k, xy_t, cand_t, dcand_t,
                                                        route_t, pos_t);
  return cudaGetLastError();
}

cudaError_t launch_unlabel(const int32_t* route0, const int32_t* route_t, int32_t* route, int n, cudaStream_t s) {
  k_unlabel<<<(n + 255) / 256, 256, 0, s>>>(route0, route_t, route, n);
  return cudaGetLastError();
}

cudaError_t launch_init_ls(const int2* xy, int n, const int32_t* cand, const int32_t* dcand, int k, int oropt,
                           int verify, int init3, int32_t* route, int32_t* pos, int32_t* queue, uint8_t* flags,
                           int32_t* logb, cudaStream_t s) {
  const size_t sm = init_ls_pos_smem(reinterpret_cast<const void*>(k_init_ls<true>), n);
  if (sm > 0)
    k_init_ls<true><<<1, 1024, sm, s>>>(xy, n, cand, dcand, k, oropt, verify, init3, route, pos, queue, flags, logb);
  else
    k_init_ls<false><<<1, 1024, 0, s>>>(xy, n, cand, dcand, k, oropt, verify, init3, route, pos, queue, flags, logb);
  return cudaGetLastError();
}

cudaError_t launch_init_tour_batch(const Colony* cols, const ColonySetup* sets, int count, int max_n, int stage,
                                   cudaStream_t s) {
  if (stage == 0) {
    const size_t smem = (size_t)((max_n + 31) >> 5) * sizeof(uint32_t);
    if (smem > 48 * 1024) {
      cudaError_t e = allow_dyn_smem(reinterpret_cast<const void*>(k_nn_tour_b), smem);
      if (e != cudaSuccess) return e;
    }
    k_nn_tour_b<<<count, 32, smem, s>>>(cols, sets);
  } else {
    const size_t sm = init_ls_pos_smem(reinterpret_cast<const void*>(k_init_ls_b<true>), max_n);
    if (sm > 0)
      k_init_ls_b<true><<<count, 1024, sm, s>>>(cols, sets);
    else
      k_init_ls_b<false><<<count, 1024, 0, s>>>(cols, sets);
  }
  return cudaGetLastError();
}

cudaError_t launch_test_kernels(int what, const void* in, void* out, int count, int width,
                                uint64_t seed, cudaStream_t s) {
  k_tests<<<(count + 127) / 128, 128, 0, s>>>(what, in, out, count, width, seed);
  return cudaGetLastError();
}

}  // namespace faco
