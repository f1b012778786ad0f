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
#include "ls_array.cuh"

namespace faco {

namespace {

__global__ void __launch_bounds__(32) k_nn_tour(const int2* xy, int n, const int32_t* cand, int k,
                                                const int32_t* backup, int bl, int32_t* route,
                                                uint32_t* vis_g) {
  extern __shared__ uint32_t sv[];
  uint32_t* vis = vis_g ? vis_g : sv;
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
      const int2 xu = xy[u];
      uint64_t bk = ~0ull;
      int32_t bi = INT_MAX;
      for (int w = lane; w < n; w += 32) {
        if (!((vis[w >> 5] >> (w & 31)) & 1u)) {
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

__global__ void __launch_bounds__(32) k_init_ls(const int2* xy, int n, const int32_t* cand, int k,
                                                int oropt, int verify, int32_t* route, int32_t* pos,
                                                int32_t* queue, uint8_t* flags, int32_t* logb) {
  LsEnv E;
  E.n = n; E.k = k; E.oropt = oropt; E.verify = verify; E.xy = xy; E.cand = cand;
  E.queue = queue; E.flags = flags; E.logb = logb;
  ArrTour T{n, route, pos};
  LsStats S{0, 0, 0, 0, 0};
  ls_array_run(E, T, route, n, S);
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
                           int bl, int32_t* route, uint32_t* vis_g, cudaStream_t s) {
  const size_t smem = vis_g ? 0 : (size_t)((n + 31) >> 5) * sizeof(uint32_t);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_nn_tour, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_nn_tour<<<1, 32, smem, s>>>(xy, n, cand, k, backup, bl, route, vis_g);
  return cudaGetLastError();
}

cudaError_t launch_init_ls(const int2* xy, int n, const int32_t* cand, int k, int oropt, int verify,
                           int32_t* route, int32_t* pos, int32_t* queue, uint8_t* flags,
                           int32_t* logb, cudaStream_t s) {
  k_init_ls<<<1, 32, 0, s>>>(xy, n, cand, k, oropt, verify, route, pos, queue, flags, logb);
  return cudaGetLastError();
}

cudaError_t launch_test_kernels(int what, const void* in, void* out, int count, int width,
                                uint64_t seed, cudaStream_t s) {
  k_tests<<<(count + 127) / 128, 128, 0, s>>>(what, in, out, count, width, seed);
  return cudaGetLastError();
}

}  // namespace faco
