// ants_arr_b8.cu -- the batch array kernel with residency bound 8 (ants_arr_b.cuh).
#include "ants_arr_b.cuh"

namespace faco {

cudaError_t launch_ants_arr_batch_8(int kw, const Colony* cols, const Ants* ants, const int2* map, int nmap,
                                    int redo_blocks, const int2* redo_list, const int32_t* redo_n,
                                    size_t per_warp, cudaStream_t s) {
  return launch_arr_b_mb<8>(kw, cols, ants, map, nmap, redo_blocks, redo_list, redo_n, per_warp, s);
}

cudaError_t prepare_ants_arr_batch_8(int kw, size_t smem) { return prepare_arr_b_mb<8>(kw, smem); }

int occupancy_ants_arr_batch_8(int kw, size_t smem) { return occupancy_arr_b_mb<8>(kw, smem); }

}  // namespace faco
