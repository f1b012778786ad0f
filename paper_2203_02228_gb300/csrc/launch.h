// launch.h -- host-side launchers shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace faco {

// ants.cu
cudaError_t launch_ants(const Colony& C, const Ants& A, cudaStream_t s);
cudaError_t prepare_ants_kernel(int kw, size_t smem_seg, size_t smem_arr);
size_t ants_smem_per_warp(int n, int seg_cap, bool segs);

// colony.cu
cudaError_t launch_rows(const Colony& C, int update, cudaStream_t s);
cudaError_t launch_scan_P(const Colony& C, cudaStream_t s);
cudaError_t launch_best(const Colony& C, const Ants& A, cudaStream_t s);
cudaError_t launch_source(const Colony& C, const Ants& A, int32_t* tmp_route, int32_t* tmp_pos,
                          cudaStream_t s);
cudaError_t launch_state_init(const Colony& C, const int64_t* len, cudaStream_t s);
cudaError_t launch_positions(const int32_t* route, int32_t* pos, int n, cudaStream_t s);
cudaError_t launch_tour_length(const int2* xy, const int32_t* route, int n, int64_t* out,
                               cudaStream_t s);

// knn.cu
cudaError_t launch_bbox_check(const int2* xy, int n, int32_t* out5, cudaStream_t s);
cudaError_t build_lists(const int2* xy, int n, int k, int bl, const Grid& g, int32_t* cell_count,
                        int32_t* cell_start, int32_t* cell_pts, int32_t* cand, int32_t* backup,
                        float* eta, cudaStream_t s);

// tour.cu
cudaError_t launch_nn_tour(const int2* xy, int n, const int32_t* cand, int k, const int32_t* backup,
                           int bl, int32_t* route, uint32_t* vis_g, const Grid& g, const int32_t* cstart,
                           const int32_t* cpts, cudaStream_t s);
cudaError_t launch_init_ls(const int2* xy, int n, const int32_t* cand, int k, int oropt, int verify,
                           int32_t* route, int32_t* pos, int32_t* queue, uint8_t* flags,
                           int32_t* logb, cudaStream_t s);
cudaError_t launch_test_kernels(int what, const void* in, void* out, int count, int width,
                                uint64_t seed, cudaStream_t s);

}  // namespace faco
