// probe.cu -- an L2 read-bandwidth probe: the denominator against which the
// per-ant kernel's L2 traffic (ncu lts__t_bytes) is reported.  The paper
// has no counterpart; the method's hot path never needs it.
//
// A buffer small enough to stay resident in L2 is read `reps` times by a
// grid of a few blocks per SM, 16 bytes per load with the L1-bypassing
// ld.global.cg, so that every load is an L2 transaction.  The bytes read
// over the kernel's CUDA-event duration is the achievable L2 read rate.
#include <cstdint>

#include "common.cuh"
#include "faco.h"

namespace {

__global__ void __launch_bounds__(512) k_l2_read(const uint4* __restrict__ buf, size_t n16, int reps,
                                                 uint32_t* __restrict__ sink) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  uint32_t acc = 0;
  for (int r = 0; r < reps; ++r) {
    // consecutive threads read consecutive 16-byte words (coalesced); every
    // pass reads each word once, from a starting offset that moves with r
    const size_t off = ((size_t)r * 4096u) % n16;
    for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < n16; j += stride) {
      size_t i = j + off;
      if (i >= n16) i -= n16;
      const uint4 v = __ldcg(buf + i);
      acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
  }
  // one word per block keeps the loads live
  acc = __reduce_xor_sync(faco::kFull, acc);
  if ((threadIdx.x & 31) == 0) atomicXor(sink + blockIdx.x, acc);
}

__global__ void k_fill(uint4* buf, size_t n16) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x)
    buf[i] = make_uint4((uint32_t)i, (uint32_t)(i >> 7), 0x9E3779B9u, (uint32_t)i * 3u);
}

}  // namespace

extern "C" int faco_l2_probe(size_t bytes, int32_t reps, double* gbs) {
  if (!gbs || bytes < (1u << 20) || bytes > ((size_t)1 << 30) || reps < 1 || reps > 100000) return FACO_E_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return FACO_E_CUDA;
  }
  const size_t n16 = bytes / 16;
  const int blocks = sms * 4;
  uint4* buf = nullptr;
  uint32_t* sink = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = FACO_OK;
  float ms = 0.0f;
  if (cudaMalloc(&buf, n16 * 16) != cudaSuccess || cudaMalloc(&sink, sizeof(uint32_t) * blocks) != cudaSuccess) {
    rc = FACO_E_NOMEM;
    goto done;
  }
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = FACO_E_CUDA;
    goto done;
  }
  k_fill<<<blocks, 256, 0, s>>>(buf, n16);
  cudaMemsetAsync(sink, 0, sizeof(uint32_t) * blocks, s);
  k_l2_read<<<blocks, 512, 0, s>>>(buf, n16, 2, sink);  // warm: the buffer comes into L2
  cudaEventRecord(e0, s);
  k_l2_read<<<blocks, 512, 0, s>>>(buf, n16, reps, sink);
  cudaEventRecord(e1, s);
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.0f) {
    rc = FACO_E_CUDA;
    goto done;
  }
  *gbs = (double)n16 * 16.0 * reps / (ms * 1e-3) / 1e9;
done:
  (void)cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (buf) cudaFree(buf);
  if (sink) cudaFree(sink);
  return rc;
}
