// Shared device-side definitions of the GB300 mortar library (sm_103a).
//
// Geometry conventions (Mayr & Popp, arXiv 2202.03933, Sec. 2.2-2.3):
//   quad4 shape functions N_a(xi) = 1/4 (1 + xi xi_a)(1 + eta eta_a) with
//   corners (-1,-1), (1,-1), (1,1), (-1,1); tri3 N = (1 - xi - eta, xi, eta).
//   One auxiliary plane per slave element: point x0 = x(xi_c), unit normal n0
//   at xi_c (Fig. 1), in-plane basis t1 = normalised projected first edge,
//   t2 = n0 x t1.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mortar {

constexpr int kMaxPoly = 16;   // polygon vertex cap; convex quad vs quad needs <= 8
// Largest block of the pair kernels.  They hold up to 255 registers per
// thread, so 256 threads already fill the 64 K register file of an SM; a
// 512-thread block would cap them at 128 registers and spill.
constexpr int kMaxPairBlock = 256;
constexpr size_t kMaxDynSmem = 227 * 1024;   // dynamic shared memory per block on sm_103a
constexpr int kMaxRow = 256;   // CSR entries gathered per row before the slow path

// Per-run numeric parameters, passed by value to the kernels.
struct RunParams {
  int32_t lm;
  int32_t d_domain;
  int32_t newton_max_iter;
  int32_t pad;
  double newton_tol;
  double clip_tol_rel;
  double merge_tol_rel;
  double area_tol_rel;
  double delta;
  double bin_margin;
  int32_t integration;    // 0 segment-based, 1 element-based
  int32_t rule_n;         // element-based rule: points per direction
  int32_t facing;         // facing test on candidate pairs
  int32_t watchdog_us;    // per-CTA time budget of the persistent pair kernels (0 = none)
};

// Slave element record (FP64 words).  Written once per evaluation by the
// precompute kernel, read by every pair of that element.
enum SlaveRec : int {
  SR_X0 = 0,      // x0 (3)
  SR_T1 = 3,      // t1 (3)
  SR_T2 = 6,      // t2 (3)
  SR_N0 = 9,      // n0 (3)
  SR_C = 12,      // bilinear coefficients of the projected slave element c0..c3 (8)
  SR_PS = 20,     // projected slave nodes in window (CCW) order (8)
  SR_EPSIN = 28,  // inside tolerance
  SR_EPSM2 = 29,  // squared merge distance
  SR_EPSA = 30,   // area threshold
  SR_REV = 31,    // 1 if the window order is the reverse of the node order
  SR_A = 32,      // LM coefficients A[a][b] (16)
  SR_BINV = 48,   // inverse of [c1 c2] (row-major 2x2): xi = Binv (x - c0) for affine maps
  SR_AFF = 52,    // 1 if the projected slave map is affine (c3 negligible)
  SR_STRIDE = 56
};

// Device-side counters and sizes of one run (read back once per run).
struct DevStatus {
  unsigned long long n_pairs;
  unsigned long long nnz_D;
  unsigned long long nnz_M;
  unsigned long long n_bins;
  unsigned long long nonempty;
  unsigned long long gauss_points;
  unsigned long long cells;
  unsigned long long newton_fail;
  unsigned long long xi_oor;
  unsigned long long clip_overflow;
  unsigned long long over_pairs;   // pair buffer too small (needed size in n_pairs)
  unsigned long long over_nnz;     // CSR buffer too small
  unsigned long long over_bins;    // bin table too small
  unsigned long long degenerate;
  unsigned long long timeout;
  unsigned long long row_slow;     // rows assembled by the slow (unbuffered) path
  unsigned long long over_mlist;   // master pair-list buffer too small
  unsigned long long work_ctr;     // work counter of the persistent integration kernel
  unsigned long long work_ctr2;    // work counter of the persistent adjoint kernel
  unsigned long long work_ctr3;    // work counter of the linearisation pair kernel
  unsigned long long nnzb_K;       // 3x3 blocks of the linearisation
  unsigned long long over_K;       // linearisation block buffer too small
  unsigned long long nonfinite;    // elements with a non-finite node coordinate
  double J;
};

// Per-interface search grid.
struct GridParams {
  double org[3];
  double beta[3];
  int32_t nb[3];
  int32_t pad;
  int64_t bin_off;   // first bin of this interface in the global bin table
  int64_t n_bins;
};

// ---------------------------------------------------------------------------
// small math
// ---------------------------------------------------------------------------
__device__ __forceinline__ double cross2(double au, double av, double bu, double bv) {
  return au * bv - av * bu;
}

// Side of a signed distance d with respect to the inside band [-eps, eps]
// (eps finite, >= 0): 1 if d > eps, -1 if d < -eps, 0 inside the band, 2 for
// NaN.  Decided with integer compares on the IEEE bit patterns (sign and
// magnitude order equal the numeric order for finite values), so the result
// is exactly that of the FP64 comparisons while keeping them off the FP64 pipe.
__device__ __forceinline__ int band_side(double d, long long eps_bits) {
  const long long b = __double_as_longlong(d);
  const long long mag = b & 0x7fffffffffffffffLL;
  if (mag > 0x7ff0000000000000LL) return 2;
  if (mag <= eps_bits) return 0;
  return b < 0 ? -1 : 1;
}

// Conversions between FP64 and FP32 by integer operations, which keeps them
// off the FP64 pipe (a conversion instruction with an FP64 operand issues
// there, at the FP64 rate):
//  * f32_trunc: FP64 -> FP32 with the mantissa truncated (signed zero below
//    the FP32 normal range, infinity above it) -- for FP32 seeds and sort keys;
//  * f64_of_f32: FP32 -> FP64, exact for normal numbers and zero (FP32
//    subnormals become signed zero; infinity and NaN keep their class).
__device__ __forceinline__ float f32_trunc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((unsigned)e << 23) | (unsigned)((b >> 29) & 0x7fffffull));
}

__device__ __forceinline__ double f64_of_f32(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0) return __longlong_as_double((long long)sign);
  const unsigned long long e64 = e == 0xffu ? 0x7ffull : (unsigned long long)(e + 896u);
  return __longlong_as_double((long long)(sign | (e64 << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}

template <int NEN>
__device__ __forceinline__ void shape_fn(double xi, double eta, double N[4]) {
  if constexpr (NEN == 4) {
    const double a = 1.0 - xi, b = 1.0 + xi, c = 1.0 - eta, d = 1.0 + eta;
    N[0] = 0.25 * a * c;
    N[1] = 0.25 * b * c;
    N[2] = 0.25 * b * d;
    N[3] = 0.25 * a * d;
  } else {
    N[0] = 1.0 - xi - eta;
    N[1] = xi;
    N[2] = eta;
    N[3] = 0.0;
  }
}

// Bilinear (quad4) or affine (tri3) map of an element in the auxiliary plane:
//   x(xi, eta) = c0 + c1 xi + c2 eta + c3 xi eta    (c3 = 0 for tri3)
struct PlaneMap {
  double c0u, c0v, c1u, c1v, c2u, c2v, c3u, c3v;
};

template <int NEN>
__device__ __forceinline__ PlaneMap plane_map(const double* pu, const double* pv) {
  PlaneMap m;
  if constexpr (NEN == 4) {
    m.c0u = 0.25 * ((pu[0] + pu[1]) + (pu[2] + pu[3]));
    m.c0v = 0.25 * ((pv[0] + pv[1]) + (pv[2] + pv[3]));
    m.c1u = 0.25 * ((pu[1] - pu[0]) + (pu[2] - pu[3]));
    m.c1v = 0.25 * ((pv[1] - pv[0]) + (pv[2] - pv[3]));
    m.c2u = 0.25 * ((pu[2] - pu[1]) + (pu[3] - pu[0]));
    m.c2v = 0.25 * ((pv[2] - pv[1]) + (pv[3] - pv[0]));
    m.c3u = 0.25 * ((pu[0] - pu[1]) + (pu[2] - pu[3]));
    m.c3v = 0.25 * ((pv[0] - pv[1]) + (pv[2] - pv[3]));
  } else {
    m.c0u = pu[0];
    m.c0v = pv[0];
    m.c1u = pu[1] - pu[0];
    m.c1v = pv[1] - pv[0];
    m.c2u = pu[2] - pu[0];
    m.c2v = pv[2] - pv[0];
    m.c3u = 0.0;
    m.c3v = 0.0;
  }
  return m;
}

// Back-projection chi_h: solve x(xi) = (xu, xv).  quad4: Newton from xi = 0,
// stop once |dxi|_inf <= tol and apply one more update; tri3: one linear solve.
// Returns false if Newton did not converge within max_iter updates.
template <int NEN>
__device__ __forceinline__ bool invert_plane_map(const PlaneMap& m, double xu, double xv, double tol,
                                                 int max_iter, double& xi, double& eta) {
  if constexpr (NEN == 3) {
    const double ru = xu - m.c0u, rv = xv - m.c0v;
    const double det = m.c1u * m.c2v - m.c2u * m.c1v;
    const double inv = 1.0 / det;
    xi = (ru * m.c2v - m.c2u * rv) * inv;
    eta = (m.c1u * rv - ru * m.c1v) * inv;
    return true;
  } else {
    xi = 0.0;
    eta = 0.0;
    bool last = false;
    for (int it = 0; it < max_iter; ++it) {
      const double ru = m.c0u + m.c1u * xi + m.c2u * eta + m.c3u * xi * eta - xu;
      const double rv = m.c0v + m.c1v * xi + m.c2v * eta + m.c3v * xi * eta - xv;
      const double j00 = m.c1u + m.c3u * eta, j01 = m.c2u + m.c3u * xi;
      const double j10 = m.c1v + m.c3v * eta, j11 = m.c2v + m.c3v * xi;
      const double inv = 1.0 / (j00 * j11 - j01 * j10);
      const double d0 = -(j11 * ru - j01 * rv) * inv;
      const double d1 = -(j00 * rv - j10 * ru) * inv;
      xi += d0;
      eta += d1;
      if (last) return true;
      if (fmax(fabs(d0), fabs(d1)) <= tol) last = true;
    }
    return false;
  }
}

// A projected quad4 map is treated as affine when its bilinear coefficient is
// below 1e-15 of the linear ones (rounding level for parallelograms): the
// affine solve then differs from the bilinear one by less than 1e-15 in xi.
__device__ __forceinline__ bool map_is_affine(const PlaneMap& m) {
  return fabs(m.c3u) + fabs(m.c3v) <= 1e-15 * (fabs(m.c1u) + fabs(m.c1v) + fabs(m.c2u) + fabs(m.c2v));
}

template <int NEN>
__device__ __forceinline__ bool xi_out_of_range(double xi, double eta) {
  const double lim = 1.0 + 1e-8;
  if constexpr (NEN == 4) {
    return fabs(xi) > lim || fabs(eta) > lim;
  } else {
    return xi < -1e-8 || eta < -1e-8 || xi + eta > lim;
  }
}

// 7-point degree-5 triangle rule (Radon; Stroud T2:5-1): barycentric
// (l0, l1, l2) and weights summing to one.
struct Tri7 {
  static constexpr double a1 = 0.10128650732345633, b1 = 0.7974269853530872, w1 = 0.12593918054482717;
  static constexpr double a2 = 0.47014206410511505, b2 = 0.05971587178976981, w2 = 0.13239415278850616;
  static constexpr double w0 = 0.225;
};

__device__ __forceinline__ void tri7_point(int q, double& l1, double& l2, double& w) {
  // point 0: centroid; 1-3: orbit (a1,a1,b1); 4-6: orbit (a2,a2,b2);
  // (l0, l1, l2) = (a,a,b), (a,b,a), (b,a,a)
  switch (q) {
    case 0: l1 = 1.0 / 3.0; l2 = 1.0 / 3.0; w = Tri7::w0; break;
    case 1: l1 = Tri7::a1; l2 = Tri7::b1; w = Tri7::w1; break;
    case 2: l1 = Tri7::b1; l2 = Tri7::a1; w = Tri7::w1; break;
    case 3: l1 = Tri7::a1; l2 = Tri7::a1; w = Tri7::w1; break;
    case 4: l1 = Tri7::a2; l2 = Tri7::b2; w = Tri7::w2; break;
    case 5: l1 = Tri7::b2; l2 = Tri7::a2; w = Tri7::w2; break;
    default: l1 = Tri7::a2; l2 = Tri7::a2; w = Tri7::w2; break;
  }
}

// 1 / n for the vertex counts of a clip polygon (the vertex-mean centroid of
// the fan): a constant-memory load and a multiplication instead of an
// integer-to-FP64 conversion and a division on the FP64 pipe
static __constant__ double kInvCount[17] = {0.0,       1.0,       1.0 / 2,  1.0 / 3,  1.0 / 4,  1.0 / 5,
                                            1.0 / 6,   1.0 / 7,   1.0 / 8,  1.0 / 9,  1.0 / 10, 1.0 / 11,
                                            1.0 / 12,  1.0 / 13,  1.0 / 14, 1.0 / 15, 1.0 / 16};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Watchdog of the persistent pair kernels: a warp stops fetching work once
// its CTA has run longer than the budget (watchdog_us > 0) and flags
// st->timeout; the host then reports MORTAR_ERR_TIMEOUT and the context stays
// usable (every run starts from cleared counters).
struct Watchdog {
  unsigned long long t0, budget_ns;
  __device__ __forceinline__ explicit Watchdog(int32_t us)
      : t0(global_ns()), budget_ns(us > 0 ? 1000ull * (unsigned long long)us : 0ull) {}
  // warp-uniform: true if the budget ran out (lane 0 reads the clock)
  __device__ __forceinline__ bool expired(unsigned long long* timeout_flag) const {
    if (budget_ns == 0) return false;
    int out = 0;
    if ((threadIdx.x & 31) == 0 && global_ns() - t0 > budget_ns) {
      out = 1;
      atomicAdd(timeout_flag, 1ull);
    }
    return __shfl_sync(0xffffffffu, out, 0) != 0;
  }
};

// Busy interval of this CTA of a persistent kernel (first / last thread
// activity), recorded only when cta_t is non-null.
__device__ __forceinline__ void cta_mark(unsigned long long* cta_t, int which) {
  if (cta_t && threadIdx.x == 0) cta_t[2 * blockIdx.x + which] = global_ns();
}

// Block-wide sum of an unsigned counter, one atomic per block.
__device__ __forceinline__ void block_count_add(unsigned long long* dst, unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

}  // namespace mortar
