// Device-wide exclusive prefix sum of int32 counts into int64 offsets.
//
// Three stream-ordered kernels (tile sums, scan of tile sums in one block,
// tile-local scan plus carry).  The element count may live on the device (it
// is produced by an earlier kernel of the same run), so the grid is sized for
// a host-side maximum and surplus blocks exit at once.  The result is
// deterministic (integer arithmetic) and out[n] receives the total.
#include "context.h"

namespace mortar {

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 16;
constexpr int kTile = kThreads * kPerThread;

__device__ __forceinline__ int64_t count_of(const int64_t* n_dev, int64_t n_max) {
  return n_dev ? *n_dev : n_max;
}

__device__ __forceinline__ int64_t block_sum(int64_t v) {
  __shared__ int64_t warp_sums[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = v;
  __syncthreads();
  int64_t t = 0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < kThreads / 32 ? warp_sums[threadIdx.x] : 0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

// Exclusive block scan; returns this thread's exclusive prefix.
__device__ __forceinline__ int64_t block_exclusive(int64_t v) {
  __shared__ int64_t warp_tot[kThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    int64_t t = lane < kThreads / 32 ? warp_tot[lane] : 0;
    int64_t ti = t;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < kThreads / 32) warp_tot[lane] = ti - t;
  }
  __syncthreads();
  return inc - v + warp_tot[w];
}

__global__ void __launch_bounds__(kThreads) k_tile_sums(const int32_t* __restrict__ in, const int64_t* n_dev,
                                                        int64_t n_max, int64_t* __restrict__ tmp) {
  const int64_t n = count_of(n_dev, n_max);
  const int64_t base = (int64_t)blockIdx.x * kTile;
  if (base >= n) return;
  int64_t s = 0;
  for (int k = 0; k < kPerThread; ++k) {
    const int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
    if (i < n) s += in[i];
  }
  s = block_sum(s);
  if (threadIdx.x == 0) tmp[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(int64_t* __restrict__ tmp, const int64_t* n_dev, int64_t n_max,
                                                     int64_t* __restrict__ out) {
  const int64_t n = count_of(n_dev, n_max);
  const int64_t nt = (n + kTile - 1) / kTile;
  __shared__ int64_t warp_tot[32];
  __shared__ int64_t carry_s;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t b0 = 0; b0 < nt; b0 += 1024) {
    const int64_t i = b0 + threadIdx.x;
    const int64_t v = i < nt ? tmp[i] : 0;
    int64_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
      int64_t t = warp_tot[lane], ti = t;
      for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, ti, o);
        if (lane >= o) ti += y;
      }
      warp_tot[lane] = ti - t;
    }
    __syncthreads();
    const int64_t carry = carry_s;
    const int64_t excl = inc - v + warp_tot[w] + carry;
    if (i < nt) tmp[i] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry_s = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry_s;
}

__global__ void __launch_bounds__(kThreads) k_tile_scan(const int32_t* __restrict__ in, const int64_t* n_dev,
                                                        int64_t n_max, const int64_t* __restrict__ tmp,
                                                        int64_t* __restrict__ out) {
  const int64_t n = count_of(n_dev, n_max);
  const int64_t base = (int64_t)blockIdx.x * kTile;
  if (base >= n) return;
  // each thread owns kPerThread consecutive elements
  const int64_t my0 = base + (int64_t)threadIdx.x * kPerThread;
  int32_t v[kPerThread];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const int64_t i = my0 + k;
    v[k] = i < n ? in[i] : 0;
    s += v[k];
  }
  int64_t run = block_exclusive(s) + tmp[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const int64_t i = my0 + k;
    if (i < n) out[i] = run;
    run += v[k];
  }
}

}  // namespace

int64_t scan_temp_words(int64_t n_max) { return (n_max + kTile - 1) / kTile + 1; }

void launch_exclusive_scan_i32(const int32_t* in, int64_t* out, const int64_t* n_dev, int64_t n_max,
                               int64_t* tmp, cudaStream_t st) {
  const int64_t nb = (n_max + kTile - 1) / kTile;
  if (nb > 0) k_tile_sums<<<(unsigned)nb, kThreads, 0, st>>>(in, n_dev, n_max, tmp);
  k_scan_tiles<<<1, 1024, 0, st>>>(tmp, n_dev, n_max, out);
  if (nb > 0) k_tile_scan<<<(unsigned)nb, kThreads, 0, st>>>(in, n_dev, n_max, tmp, out);
}

}  // namespace mortar
