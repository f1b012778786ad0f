// launch.h -- host-side launchers shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace faco {

// ants.cu
cudaError_t launch_ants(const Colony& C, const Ants& A, cudaStream_t s);
cudaError_t prepare_ants_kernel(int kw, size_t smem_seg, size_t smem_arr);
// Lets kernel f take as much dynamic shared memory as the device allows
// beside its static shared memory.  Set once per kernel and device and
// never lowered, so a launch stays valid whoever prepared the kernel last
// (colonies, batches and a server's cohorts share the kernels, from any
// host thread).  cudaErrorInvalidValue if `need` bytes exceed that limit.
cudaError_t allow_dyn_smem(const void* f, size_t need);
size_t ants_smem_per_warp(int n, int seg_cap, bool segs);
// Segments per ant table during the local search (the visited bits' room added).
int ants_seg_cap_ls(int n, int seg_cap);
cudaError_t launch_ants_blk_batch(int kw, const Colony* cols, const Ants* ants, const int2* map, int blocks,
                                  int2* redo_list, int32_t* redo_n, size_t smem, cudaStream_t s);
// batch array kernel: minb = 2, 4 or 8 blocks per SM (registers per thread
// 255, 128, 64); one translation unit per bound (ants_arr_bMB.cu)
cudaError_t launch_ants_arr_batch(int kw, int minb, const Colony* cols, const Ants* ants, const int2* map, int nmap,
                                  int redo_blocks, const int2* redo_list, const int32_t* redo_n,
                                  size_t per_warp, cudaStream_t s);
#define FACO_ARR_B_DECL(MB)                                                                                   \
  cudaError_t launch_ants_arr_batch_##MB(int kw, const Colony* cols, const Ants* ants, const int2* map,       \
                                         int nmap, int redo_blocks, const int2* redo_list,                    \
                                         const int32_t* redo_n, size_t per_warp, cudaStream_t s);             \
  cudaError_t prepare_ants_arr_batch_##MB(int kw, size_t smem);                                                \
  int occupancy_ants_arr_batch_##MB(int kw, size_t smem);
FACO_ARR_B_DECL(2)
FACO_ARR_B_DECL(4)
FACO_ARR_B_DECL(8)
#undef FACO_ARR_B_DECL
cudaError_t prepare_ants_batch(int kw, size_t smem_blk, size_t smem_arr);
size_t ants_blk_batch_smem(int kw);
// Ants resident per SM for a batch per-ant kernel: variant 0 = segment-table
// block (smem = its dynamic shared memory), 1..3 = array kernel with 2, 4, 8
// blocks per SM (smem = four warps' visited bits).
int ants_batch_resident(int variant, int kw, size_t smem);

// colony.cu
cudaError_t launch_rows(const Colony& C, int update, cudaStream_t s);
cudaError_t launch_scan_P(const Colony& C, cudaStream_t s);
cudaError_t launch_best(const Colony& C, const Ants& A, cudaStream_t s);
cudaError_t launch_source(const Colony& C, const Ants& A, cudaStream_t s);
cudaError_t launch_state_init(const Colony& C, const int64_t* len, cudaStream_t s);
cudaError_t launch_positions(const int32_t* route, int32_t* pos, int n, cudaStream_t s);
cudaError_t launch_colony_update_batch(const Colony* cols, const Ants* ants, int count, const int2* map256,
                                       int nmap256, int32_t* redo_n, cudaStream_t s);
cudaError_t launch_colony_init_batch(const Colony* cols, const ColonySetup* sets, int count, const int2* map256,
                                     int nmap256, int stage, cudaStream_t s);
cudaError_t launch_pack_batch(const Colony* cols, int count, const int2* map256, int nmap256,
                              const int64_t* node_off, int32_t* tours, int64_t* lens, int32_t* err,
                              cudaStream_t s);
cudaError_t launch_tour_length(const int2* xy, const int32_t* route, int n, int64_t* out,
                               cudaStream_t s);

// knn.cu
cudaError_t launch_bbox_check(const int2* xy, int n, int32_t* out5, cudaStream_t s);
cudaError_t build_lists(const int2* xy, int n, int k, int bl, const Grid& g, int32_t* cell_count,
                        int32_t* cell_start, int32_t* cell_pts, int4* cell_src, int32_t* cand, int32_t* backup,
                        float* eta, int32_t* dcand, cudaStream_t s);

cudaError_t launch_grid_batch(Colony* cols, const ColonySetup* sets, int count, const int2* map256, int nmap256,
                              cudaStream_t s);
cudaError_t build_lists_batch(const Colony* cols, const ColonySetup* sets, int count, const int2* map256,
                              int nmap256, const int2* map128, int nmap128, cudaStream_t s);

// tour.cu
cudaError_t launch_nn_tour(const int2* xy, int n, const int32_t* cand, int k, const int32_t* backup,
                           int bl, int32_t* route, uint32_t* vis_g, const Grid& g, const int32_t* cstart,
                           const int4* recs, cudaStream_t s);
// Copies of the coordinates and lists named by nearest-neighbour tour
// position (route0, pos0: that tour and its inverse) with the identity tour
// in route_t/pos_t; and the searched tour mapped back to node ids.
cudaError_t launch_relabel(const int32_t* route0, const int32_t* pos0, const int2* xy, const int32_t* cand,
                           const int32_t* dcand, int n, int k, int2* xy_t, int32_t* cand_t, int32_t* dcand_t,
                           int32_t* route_t, int32_t* pos_t, cudaStream_t s);
cudaError_t launch_unlabel(const int32_t* route0, const int32_t* route_t, int32_t* route, int n, cudaStream_t s);
cudaError_t launch_init_ls(const int2* xy, int n, const int32_t* cand, const int32_t* dcand, int k, int oropt,
                           int verify, int init3, int32_t* route, int32_t* pos, int32_t* queue, uint8_t* flags,
                           int32_t* logb, cudaStream_t s);
cudaError_t launch_init_tour_batch(const Colony* cols, const ColonySetup* sets, int count, int max_n, int stage,
                                   cudaStream_t s);
cudaError_t launch_test_kernels(int what, const void* in, void* out, int count, int width,
                                uint64_t seed, cudaStream_t s);

}  // namespace faco
