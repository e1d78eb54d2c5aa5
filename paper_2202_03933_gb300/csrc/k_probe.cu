// Measurement utility (not part of the method): FP64 fused multiply-add
// throughput of the device, used as the denominator of the FP64 roofline.
// Each thread runs 8 independent dependency chains of `iters` DFMAs; lanes at
// or above `active_lanes` in each warp skip the loop, which shows whether
// partially populated warps still occupy the FP64 pipe.
#include "context.h"

namespace {

__global__ void k_dfma(int64_t iters, int active_lanes, double* __restrict__ sink) {
  const int lane = threadIdx.x & 31;
  double a0 = 1.0 + 1e-9 * threadIdx.x, a1 = a0 + 1e-3, a2 = a0 + 2e-3, a3 = a0 + 3e-3;
  double a4 = a0 + 4e-3, a5 = a0 + 5e-3, a6 = a0 + 6e-3, a7 = a0 + 7e-3;
  const double b = 0.999999999, c = 1e-12;
  if (lane < active_lanes) {
    for (int64_t i = 0; i < iters; ++i) {
      a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
      a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
    }
  }
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
}

}  // namespace

extern "C" int mortar_probe_dfma(void* stream, int32_t blocks, int32_t threads, int64_t iters, int32_t active_lanes,
                                 double* sink) {
  if (blocks < 1 || threads < 32 || threads > 1024 || iters < 0 || active_lanes < 1 || active_lanes > 32 || !sink)
    return MORTAR_ERR_INVALID_ARG;
  k_dfma<<<blocks, threads, 0, (cudaStream_t)stream>>>(iters, active_lanes, sink);
  return cudaGetLastError() == cudaSuccess ? MORTAR_OK : MORTAR_ERR_CUDA;
}
