// noalloc.cu -- candidate/backup lists without any device allocation.
//
// Some callers cannot let a library call cudaMalloc: an application whose
// memory manager owns every byte of the device (a serving process with a
// fixed pool, a framework caching allocator) or a latency-critical loop in
// which cudaMalloc/cudaFree would synchronise the device and stall other
// streams.  faco_lists_noalloc serves them: the caller passes device input
// and output buffers, and the only scratch -- the point grid of the list
// builder -- lives in the file-scope array below, reserved once when the
// library is loaded and kept by every GPU that loads it until exit.
#include <cmath>

#include "faco.h"
#include "launch.h"

using namespace faco;

namespace {

// Largest instance accepted, and the scratch it needs: bounding box (8
// ints), per-cell counts and starts for a grid of at most (G+1)^2 cells,
// G = ceil(sqrt(n/2)), and the points sorted by cell.
constexpr int kNoAllocMaxN = 1 << 18;
constexpr int kNoAllocMaxG = 363;  // ceil(sqrt(2^17))
constexpr int64_t kNoAllocMaxCells = (int64_t)(kNoAllocMaxG + 1) * (kNoAllocMaxG + 1);
constexpr int64_t kScratchInts = 8 + kNoAllocMaxCells + (kNoAllocMaxCells + 1) + kNoAllocMaxN;

__device__ __align__(256) int32_t g_list_scratch[kScratchInts];

// Device address of g_list_scratch on the current device.  Looked up on
// every call (cheap beside the stream synchronisation the call makes
// anyway), so that the address stays right after a cudaDeviceReset, which
// loads the module again, possibly elsewhere.
int scratch_for_current_device(int32_t** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_list_scratch) != cudaSuccess || !p) {
    (void)cudaGetLastError();
    return FACO_E_CUDA;
  }
  *out = static_cast<int32_t*>(p);
  return FACO_OK;
}

}  // namespace

extern "C" int faco_lists_noalloc(const int32_t* coords_dev, int32_t n, int32_t k, int32_t bl,
                                  int32_t* cand_dev, int32_t* backup_dev, float* eta_dev,
                                  void* stream) {
  if (!coords_dev || !cand_dev || !eta_dev || n < 3 || k < 2 || k > kMaxK || bl < 0 || bl > 128)
    return FACO_E_ARG;
  if (n > kNoAllocMaxN) return FACO_E_SIZE;
  const int ke = k < n - 1 ? k : n - 1;
  const int ble = bl < n - 1 - ke ? bl : n - 1 - ke;
  if (ble > 0 && !backup_dev) return FACO_E_ARG;
  int32_t* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != FACO_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int32_t* bbox = scratch;
  int32_t* counts = scratch + 8;
  int32_t* starts = counts + kNoAllocMaxCells;
  int32_t* pts = starts + (kNoAllocMaxCells + 1);

  // bounding box and range check (the box is re-initialised every call)
  int32_t hb[5];
  if (launch_bbox_check(reinterpret_cast<const int2*>(coords_dev), n, bbox, s) != cudaSuccess ||
      cudaMemcpyAsync(hb, bbox, sizeof(hb), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    (void)cudaGetLastError();
    return FACO_E_CUDA;
  }
  if (hb[4]) return FACO_E_ARG;
  // square cells, about two points per cell (as in faco_create)
  Grid g;
  g.minx = hb[0];
  g.miny = hb[1];
  const int64_t ext = (int64_t)(hb[2] - hb[0] > hb[3] - hb[1] ? hb[2] - hb[0] : hb[3] - hb[1]) + 1;
  int64_t G = (int64_t)std::ceil(std::sqrt((double)n / 2.0));
  if (G < 1) G = 1;
  g.cs = (int32_t)((ext + G - 1) / G);
  if (g.cs < 1) g.cs = 1;
  g.gx = (hb[2] - hb[0]) / g.cs + 1;
  g.gy = (hb[3] - hb[1]) / g.cs + 1;
  if ((int64_t)g.gx * g.gy > kNoAllocMaxCells) return FACO_E_SIZE;
  // counts are cleared inside build_lists; starts and points are overwritten
  if (build_lists(reinterpret_cast<const int2*>(coords_dev), n, ke, ble, g, counts, starts, pts, nullptr, cand_dev,
                  ble > 0 ? backup_dev : cand_dev, eta_dev, nullptr, s) != cudaSuccess) {
    (void)cudaGetLastError();
    return FACO_E_CUDA;
  }
  return FACO_OK;
}
