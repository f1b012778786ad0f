// common.cuh -- device helpers and shared structures of the GB300 FACO library.
//
// Independent of the CPU oracle: nothing here is shared with it.  The
// arithmetic follows the paper (Sec. 2.1 costs, Eq. 1 weights, Eq. 2 update)
// and the readings documented in the library header.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace faco {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxK = 32;        // candidate list length supported (Sec. 4.1: 16)
constexpr int kMaxKnn = 160;     // k + backup length supported by the list builder

// Device error flags (bitwise or into DevState::error).
enum : int32_t {
  kErrCapacity = 1,
  kErrTimeout = 2,
  kErrInternal = 4,
};

// Per-ant counters (row of Ants::stats).
enum : int {
  kStAco = 0, kStNew, kStBackup, kStGlobal, kStCheck, kStPops, kStMoves2, kStMovesOr,
  kStFlip, kStVerify, kStRedo,
  kStStartNs,  // device time (ns) when the ant's warp started, last iteration
  kStDurNs,    // its duration (ns), last iteration
  kStConsNs,   // of which construction (ns), last iteration
  kStFallNs,   // of which global nearest-unvisited scans (ns), last iteration
  kStEvalNs,   // local search: evaluation rounds (ns), last iteration
  kStConfNs,   //   confirming pops (ns)
  kStFlipNs,   //   applying moves (ns)
  kStPushNs,   //   queueing endpoints (ns)
  kNStats = 24
};

// Colony scalars that change on the device (read by graph-replayed kernels).
struct DevState {
  int64_t iter;          // iterations completed
  int64_t gb_len;        // global-best length
  int64_t src_len;       // length of the current source solution
  int64_t it_best_len;   // iteration-best length of the last iteration
  int64_t init_len;
  double tmax_d, tmin_d; // trail limits (Sec. 4.5)
  float tmax, tmin;      // the same, stored in FP32
  float delta;           // deposit amount for the current source
  int32_t it_best_ant;
  int32_t use_gb;        // the current source is the global best
  int32_t gb_improved;   // the last iteration improved the global best
  int32_t error;         // kErr* flags
  int32_t pad;
  int64_t* hist;         // per-iteration history, 4 int64 per row
  int64_t hist_cap;      // rows available
};

// Uniform grid over the points: square cells of side cs from (minx, miny).
struct Grid {
  int32_t minx, miny, cs, gx, gy;
};

// Device pointers and sizes of one colony (passed by value).
struct Colony {
  int32_t n, k, bl, kw;  // kw = roulette width: 16 if k <= 16, else 32
  uint64_t seed;
  float rho;
  int32_t min_new_edges;
  int32_t oropt, verify;
  int32_t ls;            // 1: local search on every new tour; 0: base FACO
  int32_t init3;         // 1: the initial tour's search also tries 3-opt segment exchanges
  double c_min;          // tau_min / tau_max ratio
  double p_src_gb;
  const int2* xy;        // [n] coordinates, node order
  const int32_t* cand;   // [n][k] candidate lists
  const int32_t* backup; // [n][bl] backup lists
  const float* eta;      // [n][k] 1/d
  const int32_t* dcand;  // [n][k] d, the EUC_2D cost of each candidate edge
  float* tau;            // [n][k] pheromone on candidate edges
  int32_t* src_route;    // [n] source solution
  int32_t* src_pos;      // [n] its inverse
  int32_t* gb_route;     // [n] global best
  int32_t* gb_pos;       // [n]
  float* Wsrc;           // [n][kw] tau*eta in source order, 0 beyond k
  int32_t* Csrc;         // [n][kw] source position of each candidate, -1 beyond k
  int32_t* Dcsrc;        // [n][kw] cost of each candidate edge in source order, 0 beyond k
  int2* XYsrc;           // [n] coordinates in source order
  int32_t* Dsrc;         // [n] length of source edge (p, p+1)
  int64_t* Psrc;         // [n+1] exclusive prefix sums of Dsrc
  DevState* st;
  Grid grid;             // point grid of the candidate-list build
  const int32_t* cell_start;  // [cells+1]
  const int32_t* cell_pts;    // [n] node ids by cell
  int4* cell_src;        // [n] the same points: (source position, x, y, node id); source positions
                         //     refreshed with each iteration's rows
  int32_t* tmp_route;    // [n] iteration-best tour, materialised
  int32_t* tmp_pos;      // [n]
};

// Set-up buffers of one colony of a batch: the candidate lists and the
// initial tour of every colony are built by the same launches.
struct ColonySetup {
  int32_t* cell_cnt;     // [cells] counts, then the fill cursor
  int32_t* cell_start;   // [cells+1]
  int32_t* cell_pts;     // [n]
  int4* cell_src;        // [n] (node id, x, y, node id) until the first rows are written
  int32_t* cand;         // [n][k]
  int32_t* backup;       // [n][bl]
  float* eta;            // [n][k]
  int32_t* dcand;        // [n][k]
  int32_t* init_route;   // [n] nearest-neighbour tour, then locally optimal
  int32_t* queue;        // [n] local search of the initial tour
  uint8_t* flags;        // [n]
  int32_t* logb;         // [n]
  int64_t* len;          // length of the initial tour
  int32_t* bb;           // [5] min x, min y, max x, max y, out-of-range flag
};

// Per-ant buffers of one ant count.
struct Ants {
  int32_t m;             // ants per iteration
  int32_t* route;        // [m][n]
  int32_t* pos;          // [m][n]
  int32_t* chk;          // [m][n] checklist (node ids)
  int64_t* len;          // [m]
  int64_t* stats;        // [m][kNStats]
  int32_t* queue;        // [m][n] local-search FIFO
  uint8_t* flags;        // [m][n] bit0 queued, bit1 popped this round (kept zero between uses)
  int32_t* logb;         // [m][n] nodes popped this round, first pop order
  uint32_t* vis_g;       // [m][words] visited bits when they do not fit shared memory
  int32_t smem_vis;      // 1: visited bits live in shared memory (array kernel)
  int32_t seg_cap;       // segments per ant table during construction (0: arrays only)
  int32_t seg_cap_ls;    // during the local search, which also takes the visited bits' room;
                         // the stride of segs
  int4* segs;            // [m][seg_cap] final tours as (lo, len, off, rev), or null
  int32_t* nseg;         // [m] segment count, -1 when the tour is in route/pos
  int32_t* redo;         // [m] 1: the table overflowed, the array kernel redoes the ant
  int32_t keep_tours;    // 1: also write every tour to route[] (inspection)
  int32_t* pre_route;    // [m][n] optional: tours before local search
  int64_t* pre_len;      // [m]
  int32_t* pre_chk;      // [m][n]
  int32_t* pre_nchk;     // [m]
};

// ---------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its definition:
// ten rounds of two 32x32->64 multiplies with the Weyl key schedule.
// ---------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Draw `idx` of stream (ant, iter, tag): word idx%4 of counter (idx/4, ant, iter, tag).
__device__ __forceinline__ uint32_t draw(uint64_t seed, uint32_t idx, uint32_t ant, uint32_t iter,
                                         uint32_t tag) {
  const uint4 o = philox4x32_10(make_uint4(idx >> 2, ant, iter, tag), (uint32_t)seed,
                                (uint32_t)(seed >> 32));
  const uint32_t w = idx & 3u;
  return w == 0 ? o.x : (w == 1 ? o.y : (w == 2 ? o.z : o.w));
}

// Top 24 bits times 2^-24: exact, in [0, 1).
__device__ __forceinline__ float u01(uint32_t x) {
  return __uint2float_rn(x >> 8) * (1.0f / 16777216.0f);
}

// ---------------------------------------------------------------------
// EUC_2D: nint(sqrt(dx^2 + dy^2)) for coordinates in [0, 2^24).  The FP32
// square root is only an estimate (off by at most 2); integer corrections
// make r = floor(sqrt(m)) exactly, and sqrt(m) >= r + 1/2 <=> m - r^2 > r.
// ---------------------------------------------------------------------
__device__ __forceinline__ uint64_t sqdist(int2 a, int2 b) {
  const int64_t dx = (int64_t)a.x - b.x, dy = (int64_t)a.y - b.y;
  return (uint64_t)(dx * dx + dy * dy);
}

__device__ __forceinline__ int32_t euc2d_m(uint64_t m) {
  // a first guess from the hardware reciprocal square root (close for the
  // short edges that dominate; any guess works), then exact integer steps
  // to floor(sqrt(m))
  const float x = __ull2float_rn(m);
  uint32_t r = m ? (uint32_t)(x * rsqrtf(x)) : 0u;
  uint64_t rr = (uint64_t)r * r;
  while (rr > m) {
    --r;
    rr = (uint64_t)r * r;
  }
  while (rr + 2ull * r + 1ull <= m) {
    rr += 2ull * r + 1ull;
    ++r;
  }
  return (int32_t)(r + ((m - rr) > r ? 1u : 0u));
}

// The same cost of two points, on a short dependency chain.  An FP32
// estimate d of sqrt(dx^2 + dy^2) is accepted when the exact integer test
// d^2 - d < m <= d^2 + d holds, which says (d - 1/2)^2 < m < (d + 1/2)^2,
// i.e. d = nint(sqrt(m)); otherwise the exact integer steps of euc2d_m
// decide.  The estimate: |dx|, |dy| < 2^22 convert to FP32 exactly by the
// 1.5 * 2^23 bias (an add on the bit pattern and a float subtract), the
// hardware's approximate square root (sqrt.approx.f32) follows, and an
// estimate below 2^22 rounds to the nearest integer by the same bias.  Its
// relative error is about 2^-21, so the test fails only for costs above
// ~10^6, next to a half-integer, or with |dx| or |dy| >= 2^22 (where the
// bias tricks do not hold and the estimate is meaningless): those, and
// m = 0 (d = 0 fails the test), take the exact path.
__device__ __forceinline__ float i2f_biased(int32_t v) {  // exact for |v| < 2^22
  return __fsub_rn(__int_as_float(v + 0x4B400000), 12582912.0f);
}

__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ int32_t euc2d(int2 a, int2 b) {
  const int32_t dx = a.x - b.x, dy = a.y - b.y;  // |dx|, |dy| < 2^24
  const uint64_t m = (uint64_t)((int64_t)dx * dx) + (uint64_t)((int64_t)dy * dy);
  const float fx = i2f_biased(dx), fy = i2f_biased(dy);
  const float mf = __fmaf_rn(fx, fx, __fmul_rn(fy, fy));
  const uint32_t d = (uint32_t)(__float_as_int(__fadd_rn(sqrt_approx(mf), 12582912.0f)) - 0x4B400000);
  const uint64_t dd = (uint64_t)d * d;
  if (m > dd - d && m <= dd + d) return (int32_t)d;
  return euc2d_m(m);
}

// ---------------------------------------------------------------------
// Roulette of Eq. 1 over W slots (weights tau*eta, zero when visited or
// padding): inclusive Kogge-Stone scan (level `off` adds the value `off`
// slots to the left), r = u * total, the first slot with positive weight
// whose prefix exceeds r, else the last slot with positive weight.
// ---------------------------------------------------------------------
template <int W>
__device__ __forceinline__ int roulette(const float (&w)[W], float u) {
  float s[W];
#pragma unroll
  for (int i = 0; i < W; ++i) s[i] = w[i];
#pragma unroll
  for (int off = 1; off < W; off <<= 1) {
#pragma unroll
    for (int i = W - 1; i >= off; --i) s[i] = __fadd_rn(s[i - off], s[i]);
  }
  const float r = __fmul_rn(u, s[W - 1]);
  int pick = -1;
#pragma unroll
  for (int i = W - 1; i >= 0; --i)
    if (w[i] > 0.0f && s[i] > r) pick = i;
  if (pick < 0) {
#pragma unroll
    for (int i = 0; i < W; ++i)
      if (w[i] > 0.0f) pick = i;
  }
  return pick;
}

// ---------------------------------------------------------------------
// Small warp helpers.
// ---------------------------------------------------------------------
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int64_t shfl64(int64_t v, int src) {
  return (int64_t)__shfl_sync(kFull, (unsigned long long)v, src);
}

__device__ __forceinline__ int64_t shfl64_xor(int64_t v, int o) {
  return (int64_t)__shfl_xor_sync(kFull, (unsigned long long)v, o);
}

__device__ __forceinline__ int64_t shfl64_up(int64_t v, int o) {
  return (int64_t)__shfl_up_sync(kFull, (unsigned long long)v, o);
}

// Starts bringing the cache line holding p into L1 (no value returned).
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Lexicographic minimum of (key, idx) over the warp, for idx >= 0; every
// lane gets it.  Three warp reductions: the key's high word, its low word
// among the lanes with that high word, the index among the lanes with that
// key.
__device__ __forceinline__ void warp_min_key(uint64_t& key, int32_t& idx) {
  const unsigned kh = (unsigned)(key >> 32);
  const unsigned hi = __reduce_min_sync(kFull, kh);
  const unsigned lo = __reduce_min_sync(kFull, kh == hi ? (unsigned)key : 0xFFFFFFFFu);
  const uint64_t km = ((uint64_t)hi << 32) | lo;
  idx = (int32_t)__reduce_min_sync(kFull, key == km ? (unsigned)idx : 0xFFFFFFFFu);
  key = km;
}

// Maximum gain, ties to the smallest order index; every lane gets it.
// For gains >= 0 and indices >= 0: two warp reductions (the largest gain,
// then the smallest index among the lanes holding it).
__device__ __forceinline__ void warp_max_gain(int32_t& g, int32_t& idx) {
  const int32_t gm = __reduce_max_sync(kFull, g);
  idx = (int32_t)__reduce_min_sync(kFull, g == gm ? (unsigned)idx : 0xFFFFFFFFu);
  g = gm;
}

__device__ __forceinline__ void warp_max_gain(int64_t& g, int32_t& idx) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int64_t g2 = shfl64_xor(g, o);
    const int32_t i2 = __shfl_xor_sync(kFull, idx, o);
    if (g2 > g || (g2 == g && i2 < idx)) {
      g = g2;
      idx = i2;
    }
  }
}

__device__ __forceinline__ int wrapn(int x, int n) {  // x in (-n, 2n)
  return x < 0 ? x + n : (x >= n ? x - n : x);
}

}  // namespace faco
