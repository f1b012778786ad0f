// ants.cu -- host launchers of the per-ant kernels of ants.cuh: the
// one-colony kernels (segment-table block per ant, then arrays for the ants
// whose table filled up) and the batch segment-table kernel.  The batch
// array kernel is instantiated in ants_arr_b.cu.
#include <mutex>
#include <set>
#include <utility>

#include "ants.cuh"

namespace faco {

cudaError_t allow_dyn_smem(const void* f, size_t need) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, f);
  if (e != cudaSuccess) return e;
  const size_t limit = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
  if (need > limit) return cudaErrorInvalidValue;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair(dev, f);
  if (done.count(key)) return cudaSuccess;
  e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit);
  if (e == cudaSuccess) done.insert(key);
  return e;
}

int ants_seg_cap_ls(int n, int seg_cap) {
  if (seg_cap <= 0) return 0;
  const size_t vis_bytes = ((size_t)((n + 31) >> 5) * 4 + 15) & ~(size_t)15;
  return segtab_cap_ls(vis_bytes, seg_cap);
}

size_t ants_smem_per_warp(int n, int seg_cap, bool segs) {
  const size_t vis_bytes = ((size_t)((n + 31) >> 5) * 4 + 15) & ~(size_t)15;
  return segs ? vis_bytes + segtab_bytes(seg_cap) : vis_bytes;
}

cudaError_t launch_ants(const Colony& C, const Ants& A, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (A.segs) {  // one block per ant on segment tables, then arrays for the marked ants
    const size_t smem = ants_smem_per_warp(C.n, A.seg_cap, true);
    if (C.kw == 16)
      k_ants_blk<16><<<A.m, 32 * kAntWarps, smem, s>>>(C, A);
    else
      k_ants_blk<32><<<A.m, 32 * kAntWarps, smem, s>>>(C, A);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int warps = 4;
  const dim3 grid((A.m + warps - 1) / warps), block(32 * warps);
  const size_t smem = A.smem_vis ? warps * ants_smem_per_warp(C.n, 0, false) : 0;
  if (C.kw == 16)
    k_ants<16, false><<<grid, block, smem, s>>>(C, A);
  else
    k_ants<32, false><<<grid, block, smem, s>>>(C, A);
  return cudaGetLastError();
}

cudaError_t launch_ants_blk_batch(int kw, const Colony* cols, const Ants* ants, const int2* map, int blocks,
                                  int2* redo_list, int32_t* redo_n, size_t smem, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  if (kw == 16)
    k_ants_blk_b<16><<<blocks, 32 * kAntWarps, smem, s>>>(cols, ants, map, redo_list, redo_n);
  else
    k_ants_blk_b<32><<<blocks, 32 * kAntWarps, smem, s>>>(cols, ants, map, redo_list, redo_n);
  return cudaGetLastError();
}

// Dynamic shared memory of the batch segment-table kernel that still lets
// as many blocks reside per SM as its registers allow.
size_t ants_blk_batch_smem(int kw) {
  const void* f = kw == 16 ? reinterpret_cast<const void*>(k_ants_blk_b<16>)
                           : reinterpret_cast<const void*>(k_ants_blk_b<32>);
  int dev = 0, smem_sm = 0, reserved = 0, regs_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, f) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  const int threads = 32 * kAntWarps;
  int blocks = regs_sm / (fa.numRegs > 0 ? fa.numRegs * threads : threads);
  if (blocks < 1) blocks = 1;
  if (allow_dyn_smem(f, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  for (; blocks >= 1; --blocks) {
    long long S = (long long)smem_sm / blocks - reserved - (long long)fa.sharedSizeBytes;
    S &= ~127LL;
    for (int tries = 0; tries < 8 && S > 0; ++tries, S -= 256) {
      int nb = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, threads, (size_t)S) != cudaSuccess) {
        (void)cudaGetLastError();
        continue;
      }
      if (nb >= blocks) return (size_t)S;
    }
  }
  return 0;
}

cudaError_t launch_ants_arr_batch(int kw, int minb, const Colony* cols, const Ants* ants, const int2* map, int nmap,
                                  int redo_blocks, const int2* redo_list, const int32_t* redo_n,
                                  size_t per_warp, cudaStream_t s) {
  switch (minb) {
    case 2: return launch_ants_arr_batch_2(kw, cols, ants, map, nmap, redo_blocks, redo_list, redo_n, per_warp, s);
    case 4: return launch_ants_arr_batch_4(kw, cols, ants, map, nmap, redo_blocks, redo_list, redo_n, per_warp, s);
    case 8: return launch_ants_arr_batch_8(kw, cols, ants, map, nmap, redo_blocks, redo_list, redo_n, per_warp, s);
    default: return cudaErrorInvalidValue;
  }
}

int ants_batch_resident(int variant, int kw, size_t smem) {
  if (variant == 0) {
    const void* f = kw == 16 ? reinterpret_cast<const void*>(k_ants_blk_b<16>)
                             : reinterpret_cast<const void*>(k_ants_blk_b<32>);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, 32 * kAntWarps, smem) != cudaSuccess) {
      (void)cudaGetLastError();
      return 0;
    }
    return nb;
  }
  const int per_block = 4;  // ants (warps) per block of the array kernel
  switch (variant) {
    case 1: return per_block * occupancy_ants_arr_batch_2(kw, smem);
    case 2: return per_block * occupancy_ants_arr_batch_4(kw, smem);
    case 3: return per_block * occupancy_ants_arr_batch_8(kw, smem);
    default: return 0;
  }
}

cudaError_t prepare_ants_batch(int kw, size_t smem_blk, size_t smem_arr) {
  const void* f = kw == 16 ? reinterpret_cast<const void*>(k_ants_blk_b<16>)
                           : reinterpret_cast<const void*>(k_ants_blk_b<32>);
  cudaError_t e = allow_dyn_smem(f, smem_blk);
  if (e == cudaSuccess) e = prepare_ants_arr_batch_2(kw, smem_arr);
  if (e == cudaSuccess) e = prepare_ants_arr_batch_4(kw, smem_arr);
  if (e == cudaSuccess) e = prepare_ants_arr_batch_8(kw, smem_arr);
  return e;
}

cudaError_t prepare_ants_kernel(int kw, size_t smem_seg, size_t smem_arr) {
  cudaError_t e;
  if (kw == 16) {
    e = allow_dyn_smem(reinterpret_cast<const void*>(k_ants_blk<16>), smem_seg);
    if (e == cudaSuccess) e = allow_dyn_smem(reinterpret_cast<const void*>(k_ants<16, false>), smem_arr);
  } else {
    e = allow_dyn_smem(reinterpret_cast<const void*>(k_ants_blk<32>), smem_seg);
    if (e == cudaSuccess) e = allow_dyn_smem(reinterpret_cast<const void*>(k_ants<32, false>), smem_arr);
  }
  return e;
}

}  // namespace faco
