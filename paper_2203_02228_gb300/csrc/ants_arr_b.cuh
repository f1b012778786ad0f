// ants_arr_b.cuh -- the batch array kernel (one warp per ant) at a given
// residency bound MB (blocks per SM the register allocation must allow):
// a lower bound gives each warp more registers, a higher one keeps more
// ants in flight per SM to hide the latency of their dependent loads.
// Each bound is instantiated in its own translation unit (ants_arr_bMB.cu).
#pragma once

#include "ants.cuh"

namespace faco {
namespace {

template <int MB>
cudaError_t launch_arr_b_mb(int kw, const Colony* cols, const Ants* ants, const int2* map, int nmap,
                            int redo_blocks, const int2* redo_list, const int32_t* redo_n, size_t per_warp,
                            cudaStream_t s) {
  const int blocks = nmap + redo_blocks;
  if (blocks <= 0) return cudaSuccess;
  const size_t smem = 4 * per_warp;
  if (kw == 16)
    k_ants_b<16, MB><<<blocks, 128, smem, s>>>(cols, ants, map, nmap, redo_list, redo_n, per_warp);
  else
    k_ants_b<32, MB><<<blocks, 128, smem, s>>>(cols, ants, map, nmap, redo_list, redo_n, per_warp);
  return cudaGetLastError();
}

template <int MB>
cudaError_t prepare_arr_b_mb(int kw, size_t smem) {
  const void* f = kw == 16 ? reinterpret_cast<const void*>(k_ants_b<16, MB>)
                           : reinterpret_cast<const void*>(k_ants_b<32, MB>);
  return allow_dyn_smem(f, smem);
}

template <int MB>
int occupancy_arr_b_mb(int kw, size_t smem) {
  const void* f = kw == 16 ? reinterpret_cast<const void*>(k_ants_b<16, MB>)
                           : reinterpret_cast<const void*>(k_ants_b<32, MB>);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, 128, smem) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return nb;
}

}  // namespace
}  // namespace faco
