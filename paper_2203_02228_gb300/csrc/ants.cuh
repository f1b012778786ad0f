// ants.cuh -- device code of the per-ant kernels (one warp per ant, or one block per ant): focused tour construction (Sec. 4.3, Alg 2)
// followed by the checklist-seeded local search (Sec. 4.4, Alg 3).
//
// Construction works in the SOURCE solution's position space: the colony
// keeps, per iteration, the candidate rows re-ordered by source position
// (Wsrc = tau*eta, Csrc = the candidates' source positions), so that an ant
// walking along the source reads consecutive rows, and the visited set is a
// bit per source position (shared memory).  Because the pheromone contrast
// makes the roulette follow the source edge almost always, a warp evaluates
// the next 32 roulette steps speculatively, one per lane: lane t assumes the
// ant reached p_t = pc + t*dir by following the source, treats p_1..p_t as
// visited, and draws its own Philox number (draw index = route index).  The
// first lane whose pick leaves the source ends the confirmed prefix; its own
// pick is the ant's next step.  The result equals the sequential walk step
// for step.
//
// The tour is a sequence of runs of the source.  The main kernel keeps it
// that way -- a segment table in shared memory (seg.cuh) on which the local
// search runs -- so an ant never writes n-entry arrays.  If an ant's table
// fills up, the ant is marked and redone by the array kernel, which writes
// route[]/pos[] explicitly; both give the same tour.
//
// Readings (shared with the oracle, decided there independently):
//   start node   floor(x * n / 2^32) of draw 0;
//   roulette     Eq. 1 with alpha = beta = 1 (see common.cuh);
//   fallbacks    first unvisited node of the backup list, else the unvisited
//                node nearest by (squared distance, node id);
//   new edge     v is neither source successor nor predecessor of u;
//   completion   once new_edges >= min_new_edges: copy the source forward
//                from the current end while unvisited, then backward while
//                unvisited, then resume the ACO rule;
//   checklist    the head v of every new edge, in order.
#pragma once

#include "common.cuh"
#include "launch.h"
#include "ls.cuh"
#include "nearest.cuh"
#include "seg.cuh"

namespace faco {

namespace {

__device__ __forceinline__ bool vis_get(const uint32_t* w, int q) { return (w[q >> 5] >> (q & 31)) & 1u; }

// Set visited bits for the linear range [a, b] (a <= b) with the warp.
__device__ __forceinline__ void vis_set_linear(uint32_t* w, int a, int b) {
  const int wa = a >> 5, wb = b >> 5;
  for (int x = wa + lane_id(); x <= wb; x += 32) {
    uint32_t m = 0xffffffffu;
    if (x == wa) m &= 0xffffffffu << (a & 31);
    if (x == wb) m &= 0xffffffffu >> (31 - (b & 31));
    w[x] |= m;
  }
}

// Set visited bits for the c positions pc+dir, ..., pc+c*dir (cyclic).
__device__ __forceinline__ void vis_set_run(uint32_t* w, int n, int pc, int dir, int c) {
  int a, b;
  if (dir > 0) {
    a = pc + 1;
    b = pc + c;
  } else {
    a = pc - c;
    b = pc - 1;
  }
  if (a < 0) {
    vis_set_linear(w, a + n, n - 1);
    vis_set_linear(w, 0, b);
  } else if (b >= n) {
    vis_set_linear(w, a, n - 1);
    vis_set_linear(w, 0, b - n);
  } else {
    vis_set_linear(w, a, b);
  }
  __syncwarp();
}

// First visited position in [a, b) ascending, or -1.
__device__ __forceinline__ int first_set_up(const uint32_t* w, int a, int b) {
  if (a >= b) return -1;
  const int wa = a >> 5, wb = (b - 1) >> 5;
  for (int base = wa; base <= wb; base += 32) {
    const int x = base + lane_id();
    uint32_t m = 0;
    if (x <= wb) {
      m = w[x];
      if (x == wa) m &= 0xffffffffu << (a & 31);
      if (x == wb) m &= 0xffffffffu >> (31 - ((b - 1) & 31));
    }
    const unsigned bal = __ballot_sync(kFull, m != 0);
    if (bal) {
      const int l = __ffs(bal) - 1;
      const uint32_t ml = __shfl_sync(kFull, m, l);
      return (base + l) * 32 + __ffs(ml) - 1;
    }
  }
  return -1;
}

// Last visited position in [a, b] descending, or -1.
__device__ __forceinline__ int last_set_down(const uint32_t* w, int a, int b) {
  if (a > b) return -1;
  const int wa = a >> 5, wb = b >> 5;
  for (int top = wb; top >= wa; top -= 32) {
    const int x = top - lane_id();
    uint32_t m = 0;
    if (x >= wa) {
      m = w[x];
      if (x == wa) m &= 0xffffffffu << (a & 31);
      if (x == wb) m &= 0xffffffffu >> (31 - (b & 31));
    }
    const unsigned bal = __ballot_sync(kFull, m != 0);
    if (bal) {
      const int l = __ffs(bal) - 1;
      const uint32_t ml = __shfl_sync(kFull, m, l);
      return (top - l) * 32 + 31 - __clz(ml);
    }
  }
  return -1;
}

// Number of consecutive unvisited positions s, s+dir, s+2dir, ... (cyclic);
// at least one position is visited, so the result is < n.
__device__ __forceinline__ int unvisited_run(const uint32_t* w, int n, int s, int dir) {
  if (dir > 0) {
    int p = first_set_up(w, s, n);
    if (p >= 0) return p - s;
    p = first_set_up(w, 0, s);
    return (n - s) + p;
  }
  int p = last_set_down(w, 0, s);
  if (p >= 0) return s - p;
  p = last_set_down(w, s + 1, n - 1);
  return s + (n - p);
}

// Sum of the source edge lengths covered by a run of `len` nodes starting
// at source position `first` and moving in direction `dir`.
__device__ __forceinline__ int64_t run_sum(const Colony& C, int first, int dir, int len) {
  if (len <= 1) return 0;
  const int n = C.n, cnt = len - 1;
  const int lo = dir > 0 ? first : wrapn(first - cnt, n);
  const int hi = lo + cnt;
  if (hi <= n) return C.Psrc[hi] - C.Psrc[lo];
  return (C.Psrc[n] - C.Psrc[lo]) + C.Psrc[hi - n];
}

// Shared state of a nearest-unvisited search run by a whole ant block:
// warp 0 posts the request (cmd 1, the current source position), the other
// warps wait for it at a block barrier; cmd 0 ends their loop.
struct FbBlock {
  int cmd, pc;             // cmd 1: nearest unvisited of pc; 2: speculative roulette steps
  int dir, kf;             // cmd 2: direction and tour length at pc
  int stop[32], sany[32], sq[32];  // cmd 2, per warp: first step that does not follow, its roulette
  uint64_t key[32];      // cmd 1, per warp: nearest unvisited (squared distance, node id)
  int32_t idx[32];
};

// The nearest unvisited node of source position fb.pc by (squared
// distance, node id), with every thread of the block: the visited words
// are split over the threads, each unvisited position is measured, and
// the block's minimum wins.  (A search over grid rings around fb.pc, one
// barrier per ring, took 11-14 rings on average at the points where
// construction needs this search -- late in the walk, with few nodes left
// -- and cost several times the scan.)  Must be called by every thread of
// the block; returns the source position (the same on every thread).
__device__ __noinline__ int block_nearest(const Colony& C, const uint32_t* vis, FbBlock& fb) {
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  const int n = C.n;
  const int pc = fb.pc;
  const int2 xu = C.XYsrc[pc];
  uint64_t bk = ~0ull;
  int32_t bi = INT_MAX;
  const int words = (n + 31) >> 5;
  for (int wi = tid; wi < words; wi += blockDim.x) {
    uint32_t fr = ~vis[wi];
    if (wi == words - 1 && (n & 31)) fr &= (1u << (n & 31)) - 1u;
    while (fr) {
      const int q = wi * 32 + __ffs(fr) - 1;
      fr &= fr - 1;
      const uint64_t m = sqdist(xu, C.XYsrc[q]);
      if (m <= bk) {  // the node id only decides ties
        const int32_t nd = C.src_route[q];
        if (m < bk || nd < bi) {
          bk = m;
          bi = nd;
        }
      }
    }
  }
  warp_min_key(bk, bi);
  if (lane == 0) {
    fb.key[w] = bk;
    fb.idx[w] = bi;
  }
  __syncthreads();
  uint64_t best_k = ~0ull;
  int32_t best_i = INT_MAX;
  for (int v = 0; v < nw; ++v) {
    const uint64_t k2 = fb.key[v];
    const int32_t i2 = fb.idx[v];
    if (k2 < best_k || (k2 == best_k && i2 < best_i)) {
      best_k = k2;
      best_i = i2;
    }
  }
  // (the next request reaches the slots only after the barrier that posts
  // it, which every thread passes after these reads)
  if (best_i < 0 || best_i >= n) {  // cannot happen while a node is unvisited
    if (tid == 0) atomicOr(&C.st->error, kErrInternal);
    return pc == 0 ? n - 1 : pc - 1;
  }
  return C.src_pos[best_i];
}

struct Walk {
  int kf;          // route entries filled
  int pc;          // source position of the current end
  int dir;         // direction of the current run (0: single node)
  int run_first;   // source position where the current run starts
  int run_len;
  int first_q;     // source position of route[0]
  int new_edges, nchk;
  int64_t len;     // length of the closed runs and connecting edges
  int64_t aco, backup, global;
  int64_t fall_ns;  // time in global nearest-unvisited scans
  bool segs;       // emit a segment table instead of route/pos arrays
  bool overflow;   // the segment table is full
  SegTab tab;
};

// Closes the current run: appends its segment(s) to the table.  The run
// occupies ant positions [kf - run_len, kf).
__device__ __forceinline__ void close_run(const Colony& C, Walk& W) {
  if (!W.segs || W.overflow) return;
  const int n = C.n, len = W.run_len, off = W.kf - len;
  const int S = *W.tab.S;
  if (S + 2 > W.tab.cap) {
    W.overflow = true;
    return;
  }
  if (lane_id() == 0) {
    Seg* sg = W.tab.sg;
    int add = 1;
    if (W.dir >= 0) {
      const int f = W.run_first;
      if (f + len <= n) {
        sg[S] = Seg{f, len, off, 0};
      } else {
        const int l1 = n - f;
        sg[S] = Seg{f, l1, off, 0};
        sg[S + 1] = Seg{0, len - l1, off + l1, 0};
        add = 2;
      }
    } else {
      const int f = W.run_first;
      if (f - len + 1 >= 0) {
        sg[S] = Seg{f - len + 1, len, off, 1};
      } else {
        const int l1 = f + 1;
        sg[S] = Seg{0, l1, off, 1};
        sg[S + 1] = Seg{n - (len - l1), len - l1, off + l1, 1};
        add = 2;
      }
    }
    W.tab.A[S] = (uint16_t)S;
    if (add == 2) W.tab.A[S + 1] = (uint16_t)(S + 1);
    *W.tab.S = S + add;
  }
  __syncwarp();
}

// Writes route/pos for the c positions following pc in direction dir.
__device__ __forceinline__ void place_run(const Colony& C, int32_t* route, int32_t* pos, const Walk& W,
                                          int dir, int c) {
  if (W.segs) return;
  const int n = C.n, lane = lane_id();
  constexpr int U = 8;
  for (int i0 = 0; i0 < c; i0 += 32 * U) {
    int nd[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + lane + 32 * u;
      nd[u] = -1;
      if (i < c) nd[u] = C.src_route[wrapn(W.pc + dir * (i + 1), n)];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + lane + 32 * u;
      if (i < c) {
        route[W.kf + i] = nd[u];
        pos[nd[u]] = W.kf + i;
      }
    }
  }
}

// Backup list, then global nearest unvisited node (warp).  Returns the
// source position of the chosen node.
__device__ __noinline__ int fallback_pick(const Colony& C, const uint32_t* vis, int pc, Walk& W, FbBlock* fb) {
  const int n = C.n, lane = lane_id();
  const int u = C.src_route[pc];
  for (int j0 = 0; j0 < C.bl; j0 += 32) {
    const int j = j0 + lane;
    int q = -1;
    if (j < C.bl) {
      q = C.src_pos[C.backup[(size_t)u * C.bl + j]];
      if (vis_get(vis, q)) q = -1;
    }
    const unsigned bal = __ballot_sync(kFull, q >= 0);
    if (bal) {
      W.backup++;
      return __shfl_sync(kFull, q, __ffs(bal) - 1);
    }
  }
  // global nearest unvisited node: rings of grid cells around u, else a
  // scan of the visited words that skips full ones
  const uint64_t t0 = global_ns();
  if (fb) {  // with the whole block (the block kernel: the other warps wait for this)
    if (lane == 0) {
      fb->cmd = 1;
      fb->pc = pc;
    }
    __syncwarp();
    __syncthreads();
    const int q = block_nearest(C, vis, *fb);
    W.global++;
    W.fall_ns += (int64_t)(global_ns() - t0);
    return q;
  }
  const int2 xu = C.XYsrc[pc];
  int qn;
  const int near = ring_nearest(C.cell_src, C.grid, C.cell_start, xu, 24,
                                [&](const int4& P) { return vis_get(vis, P.x); }, qn);
  if (near >= 0) {
    W.global++;
    W.fall_ns += (int64_t)(global_ns() - t0);
    return qn;
  }
  uint64_t bk = ~0ull;
  int32_t bi = INT_MAX;
  const int words = (n + 31) >> 5;
  for (int wi = lane; wi < words; wi += 32) {
    uint32_t fr = ~vis[wi];
    if (wi == words - 1 && (n & 31)) fr &= (1u << (n & 31)) - 1u;
    while (fr) {  // two unvisited positions of the word in flight
      const int q0 = wi * 32 + __ffs(fr) - 1;
      fr &= fr - 1;
      int q1 = -1;
      if (fr) {
        q1 = wi * 32 + __ffs(fr) - 1;
        fr &= fr - 1;
      }
      const int2 x0 = C.XYsrc[q0];
      const int32_t n0 = C.src_route[q0];
      int2 x1 = x0;
      int32_t n1 = n0;
      if (q1 >= 0) {
        x1 = C.XYsrc[q1];
        n1 = C.src_route[q1];
      }
      const uint64_t m0 = sqdist(xu, x0), m1 = sqdist(xu, x1);
      if (m0 < bk || (m0 == bk && n0 < bi)) {
        bk = m0;
        bi = n0;
      }
      if (m1 < bk || (m1 == bk && n1 < bi)) {
        bk = m1;
        bi = n1;
      }
    }
  }
  warp_min_key(bk, bi);
  W.global++;
  W.fall_ns += (int64_t)(global_ns() - t0);
  if (bi < 0 || bi >= n) {  // cannot happen while a node is unvisited
    if (lane == 0) atomicOr(&C.st->error, kErrInternal);
    return pc == 0 ? n - 1 : pc - 1;
  }
  return C.src_pos[bi];
}

// One ACO step (already chosen source position q) from the current end.
__device__ __forceinline__ void place_step(const Colony& C, int32_t* route, int32_t* pos, uint32_t* vis,
                                           int32_t* chk, Walk& W, int q) {
  const int n = C.n, lane = lane_id();
  const int up = W.pc + 1 == n ? 0 : W.pc + 1;
  const int dn = W.pc == 0 ? n - 1 : W.pc - 1;
  if (q != up && q != dn) {  // new edge: the current run ends here
    W.len += run_sum(C, W.run_first, W.dir, W.run_len) + euc2d(C.XYsrc[W.pc], C.XYsrc[q]);
    close_run(C, W);
    if (lane == 0) chk[W.nchk] = W.segs ? q : C.src_route[q];
    W.nchk++;
    W.new_edges++;
    W.run_first = q;
    W.run_len = 1;
    W.dir = 0;
  } else {
    if (W.dir == 0) W.dir = (q == up) ? 1 : -1;
    W.run_len++;
  }
  if (lane == 0) {
    if (!W.segs) {
      const int node = C.src_route[q];
      route[W.kf] = node;
      pos[node] = W.kf;
    }
    vis[q >> 5] |= 1u << (q & 31);
  }
  __syncwarp();
  W.kf++;
  W.pc = q;
}

// The roulette of the step taken o steps after source position pc (tour
// length kf there), in a walk along the source in direction dir, on the
// assumption that the o steps before it follow the source: the nodes they
// visit count as visited.  valid: the step exists.  Returns whether it
// picks the source successor; any: some candidate is unvisited, q: the pick.
template <int KW>
__device__ __forceinline__ bool spec_step(const Colony& C, const uint32_t* vis, int pc, int dir, int kf, int o,
                                          bool valid, uint32_t ant, uint32_t iter, bool& any, int& q) {
  const int n = C.n;
  const int pt = wrapn(pc + o * dir, n);
  any = false;
  q = -1;
  if (valid) {
    float w[KW];
    int c[KW];
    const float4* wr = reinterpret_cast<const float4*>(C.Wsrc + (size_t)pt * KW);
    const int4* cr = reinterpret_cast<const int4*>(C.Csrc + (size_t)pt * KW);
#pragma unroll
    for (int v = 0; v < KW / 4; ++v) {
      const float4 a = wr[v];
      const int4 b = cr[v];
      w[4 * v] = a.x; w[4 * v + 1] = a.y; w[4 * v + 2] = a.z; w[4 * v + 3] = a.w;
      c[4 * v] = b.x; c[4 * v + 1] = b.y; c[4 * v + 2] = b.z; c[4 * v + 3] = b.w;
    }
#pragma unroll
    for (int s = 0; s < KW; ++s) {
      bool seen = c[s] < 0;
      if (!seen) {
        seen = vis_get(vis, c[s]);
        if (!seen && dir != 0) {
          int off = (c[s] - pc) * dir;
          if (off < 0) off += n;
          seen = off >= 1 && off <= o;  // visited earlier in this speculative run
        }
      }
      if (seen) w[s] = 0.0f;
      any |= w[s] > 0.0f;
    }
    if (any) {
      const float u = u01(draw(C.seed, (uint32_t)(kf + o), ant, iter, 0));
      q = c[roulette<KW>(w, u)];
    }
  }
  return valid && any && dir != 0 && q == wrapn(pt + dir, n);
}

// cmd 2 with the whole block: warp w takes the steps 32w .. 32w+31 after
// fb.pc and records the first one that does not follow the source.  Must
// be called by every thread of the block.
template <int KW>
__device__ __forceinline__ void block_spec(const Colony& C, const uint32_t* vis, FbBlock& fb, uint32_t ant,
                                           uint32_t iter) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int o = w * 32 + lane;
  bool any;
  int q;
  const bool fol = spec_step<KW>(C, vis, fb.pc, fb.dir, fb.kf, o, fb.kf + o < C.n, ant, iter, any, q);
  const unsigned stop = __ballot_sync(kFull, !fol);
  const int l = stop ? __ffs(stop) - 1 : 0;
  const int anyl = __shfl_sync(kFull, (int)any, l), ql = __shfl_sync(kFull, q, l);
  if (lane == 0) {
    fb.stop[w] = stop ? l : 32;
    fb.sany[w] = anyl;
    fb.sq[w] = ql;
  }
  __syncthreads();
}

// Up to `nspec` roulette steps, lane t taking the step at pc + t*dir; with
// the block (fb) and a known direction, up to 32 steps per warp.
template <int KW>
__device__ __forceinline__ void aco_steps(const Colony& C, int32_t* route, int32_t* pos, uint32_t* vis,
                                          int32_t* chk, Walk& W, int nspec, uint32_t ant,
                                          uint32_t iter, FbBlock* fb) {
  const int n = C.n, lane = lane_id();
  int f, anyf, qf;
  if (fb && W.dir != 0 && nspec == 32) {
    const int nw = blockDim.x >> 5;
    nspec = 32 * nw;
    if (lane == 0) {
      fb->cmd = 2;
      fb->pc = W.pc;
      fb->dir = W.dir;
      fb->kf = W.kf;
    }
    __syncwarp();
    __syncthreads();  // the other warps take their share
    block_spec<KW>(C, vis, *fb, ant, iter);
    int ws = 0;
    while (ws < nw && fb->stop[ws] == 32) ++ws;
    f = ws < nw ? 32 * ws + fb->stop[ws] : nspec;
    anyf = ws < nw ? fb->sany[ws] : 0;
    qf = ws < nw ? fb->sq[ws] : -1;
  } else {
    bool any;
    int q;
    const bool follows = spec_step<KW>(C, vis, W.pc, W.dir, W.kf, lane, lane < nspec && W.kf + lane < n, ant,
                                       iter, any, q);
    const unsigned stop = __ballot_sync(kFull, !follows);
    f = stop ? __ffs(stop) - 1 : 32;
    anyf = __shfl_sync(kFull, (int)any, f & 31);
    qf = __shfl_sync(kFull, q, f & 31);
  }
  if (f > 0) {
    place_run(C, route, pos, W, W.dir, f);
    vis_set_run(vis, n, W.pc, W.dir, f);
    W.pc = wrapn(W.pc + f * W.dir, n);
    W.run_len += f;
    W.kf += f;
    W.aco += f;
  }
  if (f < nspec && W.kf < n) {
    if (!anyf) qf = fallback_pick(C, vis, W.pc, W, fb);
    W.aco++;
    place_step(C, route, pos, vis, chk, W, qf);
  }
}

// Focused construction of one ant.  Returns the tour length.
// fb: the block's shared state when the whole block helps with nearest-
// unvisited searches and speculative roulette steps (the caller then posts
// cmd 0 when it is done), or null.
template <int KW>
__device__ __forceinline__ int64_t construct(const Colony& C, int32_t* route, int32_t* pos, uint32_t* vis,
                                             int32_t* chk, Walk& W, uint32_t ant, uint32_t iter,
                                             FbBlock* fb = nullptr) {
  const int n = C.n, lane = lane_id();
  const int words = (n + 31) >> 5;
  for (int i = lane; i < words; i += 32) vis[i] = 0;
  __syncwarp();
  const uint32_t x0 = draw(C.seed, 0, ant, iter, 0);
  const int s0 = (int)(((uint64_t)x0 * (uint64_t)n) >> 32);
  const int q0 = C.src_pos[s0];
  if (lane == 0) {
    if (!W.segs) {
      route[0] = s0;
      pos[s0] = 0;
    }
    vis[q0 >> 5] |= 1u << (q0 & 31);
  }
  __syncwarp();
  W.kf = 1; W.pc = q0; W.dir = 0; W.run_first = q0; W.run_len = 1; W.first_q = q0;
  W.new_edges = 0; W.nchk = 0; W.len = 0; W.aco = 0; W.backup = 0; W.global = 0;
  W.overflow = false;
  while (W.kf < n && !W.overflow) {
    if (W.new_edges >= C.min_new_edges) {
      // complete along the source: forward, then backward
      int c = unvisited_run(vis, n, W.pc + 1 == n ? 0 : W.pc + 1, 1);
      if (c > 0) {
        if (W.dir == 0) W.dir = 1;
        place_run(C, route, pos, W, 1, c);
        vis_set_run(vis, n, W.pc, 1, c);
        W.pc = wrapn(W.pc + c, n);
        W.run_len += c;
        W.kf += c;
      }
      c = unvisited_run(vis, n, W.pc == 0 ? n - 1 : W.pc - 1, -1);
      if (c > 0) {
        if (W.dir == 0) W.dir = -1;
        place_run(C, route, pos, W, -1, c);
        vis_set_run(vis, n, W.pc, -1, c);
        W.pc = wrapn(W.pc - c, n);
        W.run_len += c;
        W.kf += c;
      }
      if (W.kf >= n) break;
      aco_steps<KW>(C, route, pos, vis, chk, W, 1, ant, iter, fb);
    } else {
      aco_steps<KW>(C, route, pos, vis, chk, W, W.dir != 0 ? 32 : 1, ant, iter, fb);
    }
  }
  const int64_t L = W.len + run_sum(C, W.run_first, W.dir, W.run_len) +
                    euc2d(C.XYsrc[W.pc], C.XYsrc[W.first_q]);
  close_run(C, W);
  return L;
}

// Writes the table's tour as node ids (source order -> node ids).
__device__ void seg_materialize(const Colony& C, const SegTab& T, int32_t* route) {
  const int S = *T.S;
  const int n = C.n;
  for (int r = 0; r < S; ++r) {
    const Seg s = T.sg[T.A[r]];
    for (int d = lane_id(); d < s.len; d += 32) {
      const int q = s.rev ? s.lo + s.len - 1 - d : s.lo + d;
      const int t = s.off + d;
      if ((unsigned)q < (unsigned)n && (unsigned)t < (unsigned)n) route[t] = C.src_route[q];
    }
  }
  __syncwarp();
}

// B = ids by lo (ranks by counting: lo values are distinct); keys.
__device__ void seg_finish_construction(const SegTab& T) {
  const int S = *T.S;
  for (int id = lane_id(); id < S; id += 32) {
    const int lo = T.sg[id].lo;
    int r = 0;
    for (int o = 0; o < S; ++o) r += T.sg[o].lo < lo;
    T.B[r] = (uint16_t)id;
  }
  __syncwarp();
  segtab_keys(T);
}

// Array kernel body: one warp runs ant `ant` with explicit route/pos;
// `mine` is the warp's own shared memory (visited bits, and the segment
// table when SEGS).
template <int KW, bool SEGS>
__device__ __forceinline__ void ants_arr_body(const Colony& C, const Ants& A, int ant, char* mine) {
  const int lane = lane_id();
  if (ant >= A.m) return;
  if (!SEGS && A.redo && !A.redo[ant]) return;  // array kernel: only the ants the table could not hold
  const int n = C.n;
  const int words = (n + 31) >> 5;
  const size_t vis_bytes = ((size_t)words * 4 + 15) & ~(size_t)15;
  uint32_t* vis = (SEGS || A.smem_vis) ? reinterpret_cast<uint32_t*>(mine) : A.vis_g + (size_t)ant * words;
  const uint32_t iter = (uint32_t)(C.st->iter + 1);
  const uint64_t t_start = global_ns();
  int32_t* route = A.route + (size_t)ant * n;
  int32_t* pos = A.pos + (size_t)ant * n;
  int32_t* chk = A.chk + (size_t)ant * n;

  Walk W;
  W.segs = SEGS;
  if (SEGS) {
    W.tab = segtab_at(mine + vis_bytes, A.seg_cap);
    if (lane == 0) *W.tab.S = 0;
    __syncwarp();
  }
  W.fall_ns = 0;
  const int64_t pre_len = construct<KW>(C, route, pos, vis, chk, W, (uint32_t)ant, iter);
  const uint64_t t_cons = global_ns();
  if (SEGS && W.overflow) {
    if (lane == 0) A.redo[ant] = 1;
    return;
  }
  if (SEGS) seg_finish_construction(W.tab);
  if (A.pre_route) {
    if (SEGS) {
      seg_materialize(C, W.tab, A.pre_route + (size_t)ant * n);
      for (int i = lane; i < W.nchk; i += 32) A.pre_chk[(size_t)ant * n + i] = C.src_route[chk[i]];
    } else {
      for (int i = lane; i < n; i += 32) A.pre_route[(size_t)ant * n + i] = route[i];
      for (int i = lane; i < W.nchk; i += 32) A.pre_chk[(size_t)ant * n + i] = chk[i];
    }
    if (lane == 0) {
      A.pre_len[ant] = pre_len;
      A.pre_nchk[ant] = W.nchk;
    }
  }
  // local search seeded with the checklist
  LsEnv E{n, C.oropt, C.verify, A.queue + (size_t)ant * n, A.flags + (size_t)ant * n,
          A.logb + (size_t)ant * n};
  LsStats S{0, 0, 0, 0, 0};
  int64_t gain;
  if (SEGS) {
    SegTour T{n, C.k, C.kw, W.tab, C.XYsrc, C.Csrc, C.Dcsrc};
    gain = C.ls ? ls_run(E, T, chk, W.nchk, S) : 0;
    if (gain < 0) {  // the table filled up during the search
      if (lane == 0) A.redo[ant] = 1;
      return;
    }
    // hand the tour over: segments in ant order
    const int Sn = *W.tab.S;
    int4* out = A.segs + (size_t)ant * A.seg_cap_ls;
    for (int r = lane; r < Sn; r += 32) {
      const Seg s = W.tab.sg[W.tab.A[r]];
      out[r] = make_int4(s.lo, s.len, s.off, s.rev);
    }
    if (lane == 0) A.nseg[ant] = Sn;
    if (A.keep_tours) seg_materialize(C, W.tab, route);
  } else {
    ArrTour T{n, C.k, route, pos, C.xy, C.cand, C.k, C.dcand};
    gain = C.ls ? ls_run(E, T, chk, W.nchk, S) : 0;
    if (lane == 0 && A.nseg) A.nseg[ant] = -1;  // tour is in route/pos
  }
  if (lane == 0) {
    A.len[ant] = pre_len - gain;
    if (A.redo) A.redo[ant] = 0;
    int64_t* st = A.stats + (size_t)ant * kNStats;
    // counters accumulate over iterations (zeroed when the ant buffers are made)
    st[kStAco] += W.aco; st[kStNew] += W.new_edges; st[kStBackup] += W.backup;
    st[kStGlobal] += W.global; st[kStCheck] += W.nchk; st[kStPops] += S.pops;
    st[kStMoves2] += S.moves2; st[kStMovesOr] += S.movesor; st[kStFlip] += S.flip;
    st[kStVerify] += S.verify;
    if (!SEGS && A.segs) st[kStRedo] += 1;
    st[kStStartNs] = (int64_t)t_start;
    st[kStDurNs] = (int64_t)(global_ns() - t_start);
    st[kStConsNs] = (int64_t)(t_cons - t_start);
    st[kStFallNs] = W.fall_ns;
  }
}

// One block of kAntWarps warps per ant, tour as a segment table in shared
// memory: warp 0 constructs, then all warps run the local search with
// speculative in-order pops (ls_run_block).  An ant whose table fills up is
// marked and redone by the array kernel.  A launch lasts as long as its
// slowest ant; wider blocks speculate deeper, so the slowest ants finish
// sooner, while fewer blocks fit an SM (with 64 registers, four blocks of
// eight warps: 608 of 1,024 ants start at once, the rest as the quick ones
// finish).  Measured best of 4..12 warps and 40..72 registers.
constexpr int kAntWarps = 8;
constexpr int kAntMaxRegs = 64;

__device__ __forceinline__ void st_redo_add(const Ants& A, int ant) {
  A.stats[(size_t)ant * kNStats + kStRedo] += 1;
}


// ---------------------------------------------------------------------
// Kernels.  One colony: the Colony and Ants descriptors are kernel
// parameters.  A batch of colonies: every block reads its (colony, ant)
// from a block map and the colony's descriptors from device tables into
// shared memory; the bodies are the same.
// ---------------------------------------------------------------------
template <int KW, bool SEGS>
__global__ void __launch_bounds__(128, 1) k_ants(Colony C, Ants A) {
  extern __shared__ __align__(16) char smem[];
  const int wib = threadIdx.x >> 5;
  const int ant = blockIdx.x * (blockDim.x >> 5) + wib;
  const size_t vis_bytes = ((size_t)((C.n + 31) >> 5) * 4 + 15) & ~(size_t)15;
  const size_t per_warp = SEGS ? vis_bytes + segtab_bytes(A.seg_cap) : (A.smem_vis ? vis_bytes : 0);
  ants_arr_body<KW, SEGS>(C, A, ant, smem + (size_t)wib * per_warp);
}

template <int KW>
__global__ void __maxnreg__(kAntMaxRegs) k_ants_blk(Colony C, Ants A) {
  const int ant = blockIdx.x;
  if (ant >= A.m) return;
#define ANTS_BLK_OVERFLOW (void)0
#include "ants_blk_body.inc"
#undef ANTS_BLK_OVERFLOW
}

// Copies `bytes` (a multiple of 4) with the threads lo..lo+cnt-1.
__device__ __forceinline__ void copy_words(void* dst, const void* src, size_t bytes, int lo, int cnt) {
  const int nw = (int)(bytes >> 2);
  for (int i = (int)threadIdx.x - lo; i < nw; i += cnt)
    static_cast<int32_t*>(dst)[i] = static_cast<const int32_t*>(src)[i];
}

// Batch: block b runs ant map[b].y of colony map[b].x; an ant whose table
// filled up is appended to the redo list.
template <int KW>
__global__ void __maxnreg__(kAntMaxRegs)
    k_ants_blk_b(const Colony* cols, const Ants* ants, const int2* map, int2* redo_list, int32_t* redo_n) {
  __shared__ Colony sC;
  __shared__ Ants sA;
  const int2 e = map[blockIdx.x];
  copy_words(&sC, cols + e.x, sizeof(Colony), 0, blockDim.x);
  copy_words(&sA, ants + e.x, sizeof(Ants), 0, blockDim.x);
  __syncthreads();
  const Colony& C = sC;
  const Ants& A = sA;
  const int ant = e.y;
  if (ant >= A.m) return;
#define ANTS_BLK_OVERFLOW \
  if (tid == 0) redo_list[atomicAdd(redo_n, 1)] = e
#include "ants_blk_body.inc"
#undef ANTS_BLK_OVERFLOW
}

// Batch, arrays: blocks below nmap run the four ants map[b].y + warp of
// colony map[b].x; the remaining blocks run the redo list, one entry per
// warp in turn.  per_warp is the shared-memory stride of a warp.
template <int KW, int MB>
__global__ void __launch_bounds__(128, MB)
    k_ants_b(const Colony* cols, const Ants* ants, const int2* map, int nmap, const int2* redo_list,
             const int32_t* redo_n, size_t per_warp) {
  extern __shared__ __align__(16) char smem[];
  __shared__ Colony sC[4];
  __shared__ Ants sA[4];
  const int wib = threadIdx.x >> 5;
  const bool mapped = (int)blockIdx.x < nmap;
  const int stride = mapped ? 0 : ((int)gridDim.x - nmap) * 4;
  for (int r = mapped ? 0 : ((int)blockIdx.x - nmap) * 4 + wib;; r += stride) {
    int2 e;
    if (mapped) {
      e = map[blockIdx.x];
      e.y += wib;
    } else {
      if (r >= *redo_n) break;
      e = redo_list[r];
    }
    copy_words(&sC[wib], cols + e.x, sizeof(Colony), wib * 32, 32);
    copy_words(&sA[wib], ants + e.x, sizeof(Ants), wib * 32, 32);
    __syncwarp();
    ants_arr_body<KW, false>(sC[wib], sA[wib], e.y, smem + (size_t)wib * per_warp);
    __syncwarp();
    if (mapped) break;
  }
}

}  // namespace
}  // namespace faco
