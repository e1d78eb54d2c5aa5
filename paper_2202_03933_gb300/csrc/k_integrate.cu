// Per-pair segment-based mortar integration (Algorithm 1 body, Sec. 2.3).
//
// For one slave/master pair: project the master nodes onto the slave
// element's auxiliary plane (Fig. 1: x0, n0), clip the master polygon by the
// slave polygon (Sutherland-Hodgman with an absolute inside band eps_in),
// merge near-duplicate vertices, discard slivers, split the clip polygon
// into a centroid fan of triangular cells, and integrate with the 7-point
// degree-5 rule.  At every quadrature point both elements are inverted
// (chi_h: the element map in the plane solved for xi) and
//     G[c][l] += W N_c(xi_s) N_l(xi_m),   H[c][b] += W N_c(xi_s) N_b(xi_s)
// so that M_pair = A G and D_pair = A H with the slave element's LM
// coefficients A (Phi_a = sum_c A[a][c] N_c, Eq. AnsatzDiscretizationLagrangeMult).
//
// GB300 has two FP64 lanes per SM and clock, and a warp-wide FP64 instruction
// costs the same with 1 or 32 active lanes, so the kernels are written to
// issue few FP64 instructions with full warps:
//
//  * variant 0 (default): each warp takes a batch of up to 32 R pairs
//    (guided self-scheduling).  Phase A clips one pair per lane in FP32 for
//    a sort key (cell count and edge intersections); the warp sorts its
//    pairs by key (ballot counting sort) and phase B clips in FP64 and
//    integrates them in rounds of 32 lanes of similar cost.  Affine element
//    maps are inverted with
//    one precomputed 2x2 inverse; bilinear ones by Newton in FP32 on
//    power-of-two-scaled coordinates, then one Newton step with an FP64
//    residual and the FP32 Jacobian inverse (the converged xi agrees with a
//    full FP64 Newton to rounding; MapInverse in clip.cuh).
//  * variant 1: one pair per thread, FP64 Newton from xi = 0 at every point
//    (the oracle's iteration), kept as the reference schedule.
//
// Both are persistent grids taking work from a global counter; the loops are
// bounded by the pair count.
#include <type_traits>

#include "clip.cuh"
#include "context.h"

namespace mortar {

namespace {

struct PairCounters {
  unsigned long long nonempty = 0, gp = 0, cells = 0, newton_fail = 0, xi_oor = 0, clip_over = 0;
};

// Writes M = A G (and D = A H) for pair p.
template <int NS, int NM, bool SEG>
__device__ __forceinline__ void write_blocks(int64_t p, const double* __restrict__ r, const double G[4][4],
                                             const double H[4][4], bool dual, double* __restrict__ Mblk,
                                             double* __restrict__ Dblk) {
  double* mo = Mblk + 16 * p;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      double v = 0.0;
      if (a < NS && l < NM) {
        if (dual) {
#pragma unroll
          for (int c = 0; c < NS; ++c) v += r[SR_A + 4 * a + c] * G[c][l];
        } else {
          v = G[a][l];
        }
      }
      mo[4 * a + l] = v;
    }
  if (SEG) {
    double* dout = Dblk + 16 * p;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        double v = 0.0;
        if (a < NS && b < NS) {
          if (dual) {
#pragma unroll
            for (int c = 0; c < NS; ++c) v += r[SR_A + 4 * a + c] * H[c][b];
          } else {
            v = H[a][b];
          }
        }
        dout[4 * a + b] = v;
      }
  }
}

__device__ __forceinline__ void write_zero_blocks(int64_t p, bool seg, double* __restrict__ Mblk,
                                                  double* __restrict__ Dblk) {
  double2* mo = reinterpret_cast<double2*>(Mblk + 16 * p);
#pragma unroll
  for (int k = 0; k < 8; ++k) mo[k] = make_double2(0.0, 0.0);
  if (seg) {
    double2* dout = reinterpret_cast<double2*>(Dblk + 16 * p);
#pragma unroll
    for (int k = 0; k < 8; ++k) dout[k] = make_double2(0.0, 0.0);
  }
}

// ---------------------------------------------------------------- variant 1
template <int NS, int NM, bool SEG>
__device__ __forceinline__ void integrate_one(int64_t p, const int32_t* __restrict__ ps,
                                              const int32_t* __restrict__ pm, const double* __restrict__ srec,
                                              const double* __restrict__ xm, const int32_t* __restrict__ conn_m,
                                              const RunParams& rp, double* __restrict__ Mblk,
                                              double* __restrict__ Dblk, uint8_t* __restrict__ flag,
                                              PairCounters& ctr) {
  const int32_t s = ps[p], m = pm[p];
  const double* r = srec + (int64_t)SR_STRIDE * s;
  double G[4][4], H[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { G[a][b] = 0.0; H[a][b] = 0.0; }
  PlaneMap mmap;
  double Pu[kMaxPoly], Pv[kMaxPoly];
  const int nr = clip_polygon<NS, NM, kMaxPoly>(r, xm, conn_m, m, mmap, Pu, Pv, ctr.clip_over);
  if (nr == 0) {
    write_zero_blocks(p, SEG, Mblk, Dblk);
    flag[p] = 0;
    return;
  }
  PlaneMap smap;
  smap.c0u = r[SR_C + 0]; smap.c0v = r[SR_C + 1]; smap.c1u = r[SR_C + 2]; smap.c1v = r[SR_C + 3];
  smap.c2u = r[SR_C + 4]; smap.c2v = r[SR_C + 5]; smap.c3u = r[SR_C + 6]; smap.c3v = r[SR_C + 7];
  double cu, cv;
  int ncell;
  if (nr == 3) {
    ncell = 1;
    cu = Pu[0]; cv = Pv[0];
  } else {
    ncell = nr;
    double su = 0.0, sv = 0.0;
    for (int k = 0; k < nr; ++k) { su += Pu[k]; sv += Pv[k]; }
    cu = su / (double)nr;
    cv = sv / (double)nr;
  }
  ctr.cells += ncell;
  ctr.nonempty++;
  for (int cI = 0; cI < ncell; ++cI) {
    double au, av, bu, bv, wu, wv;
    if (nr == 3) {
      au = Pu[0]; av = Pv[0]; bu = Pu[1]; bv = Pv[1]; wu = Pu[2]; wv = Pv[2];
    } else {
      const int k1 = cI + 1 == nr ? 0 : cI + 1;
      au = cu; av = cv; bu = Pu[cI]; bv = Pv[cI]; wu = Pu[k1]; wv = Pv[k1];
    }
    const double e1u = bu - au, e1v = bv - av, e2u = wu - au, e2v = wv - av;
    const double area = 0.5 * fabs(cross2(e1u, e1v, e2u, e2v));
#pragma unroll 1
    for (int q = 0; q < 7; ++q) {
      double l1, l2, w;
      tri7_point(q, l1, l2, w);
      const double xu = au + l1 * e1u + l2 * e2u;
      const double xv = av + l1 * e1v + l2 * e2v;
      const double W = w * area;
      double xs1, xs2, xm1, xm2;
      if (!invert_plane_map<NS>(smap, xu, xv, rp.newton_tol, rp.newton_max_iter, xs1, xs2)) ctr.newton_fail++;
      if (!invert_plane_map<NM>(mmap, xu, xv, rp.newton_tol, rp.newton_max_iter, xm1, xm2)) ctr.newton_fail++;
      if (xi_out_of_range<NS>(xs1, xs2)) ctr.xi_oor++;
      if (xi_out_of_range<NM>(xm1, xm2)) ctr.xi_oor++;
      double Ns[4], Nm[4];
      shape_fn<NS>(xs1, xs2, Ns);
      shape_fn<NM>(xm1, xm2, Nm);
#pragma unroll
      for (int a = 0; a < NS; ++a) {
        const double wn = W * Ns[a];
#pragma unroll
        for (int l = 0; l < NM; ++l) G[a][l] += wn * Nm[l];
        if (SEG) {
#pragma unroll
          for (int b = 0; b < NS; ++b) H[a][b] += wn * Ns[b];
        }
      }
      ctr.gp++;
    }
  }
  write_blocks<NS, NM, SEG>(p, r, G, H, rp.lm == 1, Mblk, Dblk);
  flag[p] = 1;
}

template <int NS, int NM, bool SEG>
__global__ void __launch_bounds__(kMaxPairBlock) k_integrate(const int32_t* __restrict__ ps, const int32_t* __restrict__ pm,
                                                   const double* __restrict__ srec, const double* __restrict__ xm,
                                                   const int32_t* __restrict__ conn_m, RunParams rp,
                                                   double* __restrict__ Mblk, double* __restrict__ Dblk,
                                                   uint8_t* __restrict__ flag, int64_t pair_cap, int32_t chunk,
                                                   DevStatus* st) {
  PairCounters ctr;
  const int lane = threadIdx.x & 31;
  const bool ok = st->over_pairs == 0 && st->over_bins == 0;
  const int64_t n = ok ? (int64_t)min((unsigned long long)pair_cap, st->n_pairs) : 0;
  const Watchdog wd(rp.watchdog_us);
  // bounded work loop: the counter only grows, so at most n / chunk fetches succeed
  for (;;) {
    if (wd.expired(&st->timeout)) break;
    int64_t base = 0;
    if (lane == 0) base = (int64_t)atomicAdd(&st->work_ctr, (unsigned long long)chunk);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= n) break;
    const int64_t end = min(base + (int64_t)chunk, n);
    for (int64_t p = base + lane; p < end; p += 32)
      integrate_one<NS, NM, SEG>(p, ps, pm, srec, xm, conn_m, rp, Mblk, Dblk, flag, ctr);
  }
  block_count_add(&st->nonempty, ctr.nonempty);
  block_count_add(&st->gauss_points, ctr.gp);
  block_count_add(&st->cells, ctr.cells);
  block_count_add(&st->newton_fail, ctr.newton_fail);
  block_count_add(&st->xi_oor, ctr.xi_oor);
  block_count_add(&st->clip_overflow, ctr.clip_over);
}

// ---------------------------------------------------------------- variant 0
// Shared memory of a warp: the sort keys of its batch, the sorted order and
// the set of key values present.
template <int R>
struct BatchSmem {
  static constexpr int B = 32 * R;
  using PermT = typename std::conditional<(B > 256), uint16_t, uint8_t>::type;
  static constexpr int kBytes = B * (1 + (int)sizeof(PermT)) + 8 * 4;
};

// One pair of a sorted round: FP64 clip, then the 7-point rule on the
// centroid fan with the map inversions of MapInverse.
template <int NS, int NM, bool SEG>
__device__ __forceinline__ void integrate_pair_sorted(int64_t p, const int32_t* __restrict__ ps,
                                                      const int32_t* __restrict__ pm,
                                                      const double* __restrict__ srec, const double* __restrict__ xm,
                                                      const int32_t* __restrict__ conn_m, const RunParams& rp,
                                                      double* __restrict__ Mblk, double* __restrict__ Dblk,
                                                      uint8_t* __restrict__ flag, PairCounters& ctr) {
  const double* r = srec + (int64_t)SR_STRIDE * ps[p];
  PlaneMap mmap;
  double pu[kPolyS], pv[kPolyS];
  const int nr = clip_polygon<NS, NM, kPolyS>(r, xm, conn_m, pm[p], mmap, pu, pv, ctr.clip_over);
  if (nr == 0) {
    write_zero_blocks(p, SEG, Mblk, Dblk);
    flag[p] = 0;
    return;
  }
  MapInverse mi;
  mi.setup(mmap, NM == 3 || map_is_affine(mmap));
  MapInverse si;
  {
    PlaneMap smap;
    smap.c0u = r[SR_C + 0]; smap.c0v = r[SR_C + 1]; smap.c1u = r[SR_C + 2]; smap.c1v = r[SR_C + 3];
    smap.c2u = r[SR_C + 4]; smap.c2v = r[SR_C + 5]; smap.c3u = r[SR_C + 6]; smap.c3v = r[SR_C + 7];
    if (r[SR_AFF] != 0.0) {
      si.m = smap;
      si.affine = true;
      si.i00 = r[SR_BINV]; si.i01 = r[SR_BINV + 1]; si.i10 = r[SR_BINV + 2]; si.i11 = r[SR_BINV + 3];
    } else {
      si.setup(smap, false);
    }
  }
  double G[4][4], H[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { G[a][b] = 0.0; H[a][b] = 0.0; }
  const int ncell = nr == 3 ? 1 : nr;
  double cu = pu[0], cv = pv[0];
  if (nr > 3) {
    double su = 0.0, sv = 0.0;
    for (int k = 0; k < nr; ++k) { su += pu[k]; sv += pv[k]; }
    cu = su * kInvCount[nr];
    cv = sv * kInvCount[nr];
  }
  ctr.cells += ncell;
  ctr.nonempty++;
  // the quad4 factors 1/4 of both sides are folded into the weight
  constexpr double km = NM == 4 ? 0.25 : 1.0;
  constexpr double kw = km * (NS == 4 ? 0.25 : 1.0);
  for (int cI = 0; cI < ncell; ++cI) {
    const int ib = nr == 3 ? 1 : cI;
    const int iw = nr == 3 ? 2 : (cI + 1 == nr ? 0 : cI + 1);
    const double e1u = pu[ib] - cu, e1v = pv[ib] - cv, e2u = pu[iw] - cu, e2v = pv[iw] - cv;
    const double area = 0.5 * fabs(cross2(e1u, e1v, e2u, e2v));
#pragma unroll 1
    for (int q = 0; q < 7; ++q) {
      double l1, l2, w;
      tri7_point(q, l1, l2, w);
      const double xu = cu + l1 * e1u + l2 * e2u;
      const double xv = cv + l1 * e1v + l2 * e2v;
      double xs1, xs2, xm1, xm2;
      if (!si.solve(xu, xv, xs1, xs2)) ctr.newton_fail++;
      if (!mi.solve(xu, xv, xm1, xm2)) ctr.newton_fail++;
      const double wk = kw * (w * area);
      double Ns[4], Nm[4];   // Ns = (kw W) N_s / ks, Nm = N_m / km
      if constexpr (NS == 4) {   // (1 -+ xi)(1 -+ eta) products as FMAs
        const double qa = fma(-wk, xs1, wk), qb = fma(wk, xs1, wk);
        Ns[0] = fma(-qa, xs2, qa); Ns[1] = fma(-qb, xs2, qb); Ns[2] = fma(qb, xs2, qb); Ns[3] = fma(qa, xs2, qa);
      } else {
        Ns[1] = wk * xs1; Ns[2] = wk * xs2; Ns[0] = wk - Ns[1] - Ns[2]; Ns[3] = 0.0;
      }
      if constexpr (NM == 4) {
        const double a = 1.0 - xm1, b = 1.0 + xm1;
        Nm[0] = fma(-a, xm2, a); Nm[1] = fma(-b, xm2, b); Nm[2] = fma(b, xm2, b); Nm[3] = fma(a, xm2, a);
      } else {
        shape_fn<NM>(xm1, xm2, Nm);
      }
#pragma unroll
      for (int a = 0; a < NS; ++a)
#pragma unroll
        for (int l = 0; l < NM; ++l) G[a][l] = fma(Ns[a], Nm[l], G[a][l]);
      if (SEG) {   // H = sum W N_s N_s^T = sum Ns (N_s / km)
        double Nu[4];
        if constexpr (NS == 4 && NM == 4) {
          const double a = 1.0 - xs1, b = 1.0 + xs1;
          Nu[0] = fma(-a, xs2, a); Nu[1] = fma(-b, xs2, b); Nu[2] = fma(b, xs2, b); Nu[3] = fma(a, xs2, a);
        } else {
          shape_fn<NS>(xs1, xs2, Nu);
          if (NM == 4)
            for (int b = 0; b < NS; ++b) Nu[b] *= 4.0;
        }
#pragma unroll
        for (int a = 0; a < NS; ++a)
#pragma unroll
          for (int b = 0; b < NS; ++b) H[a][b] = fma(Ns[a], Nu[b], H[a][b]);
      }
      ctr.gp++;
    }
  }
  write_blocks<NS, NM, SEG>(p, r, G, H, rp.lm == 1, Mblk, Dblk);
  flag[p] = 1;
}

template <int NS, int NM, bool SEG, int R>
__global__ void __launch_bounds__(kMaxPairBlock) k_integrate_batched(
    const int32_t* __restrict__ ps, const int32_t* __restrict__ pm, const double* __restrict__ srec,
    const double* __restrict__ xm, const int32_t* __restrict__ conn_m, RunParams rp, double* __restrict__ Mblk,
    double* __restrict__ Dblk, uint8_t* __restrict__ flag, int64_t pair_cap, DevStatus* st,
    unsigned long long* cta_t) {
  cta_mark(cta_t, 0);
  using L = BatchSmem<R>;
  using PermT = typename L::PermT;
  constexpr int B = L::B;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* my = smem_raw + (size_t)warp * L::kBytes;
  unsigned* pres = reinterpret_cast<unsigned*>(my);
  PermT* perm = reinterpret_cast<PermT*>(my + 32);
  uint8_t* keys = reinterpret_cast<uint8_t*>(perm + B);

  PairCounters ctr;
  const bool ok = st->over_pairs == 0 && st->over_bins == 0;
  const int64_t n = ok ? (int64_t)min((unsigned long long)pair_cap, st->n_pairs) : 0;
  const unsigned lt_mask = (1u << lane) - 1u;
  const Watchdog wd(rp.watchdog_us);
  // guided self-scheduling: a warp takes half an even share of the pairs
  // left (at most B, at least 32, a multiple of 32)
  const int64_t share = 2 * (int64_t)gridDim.x * (blockDim.x >> 5);
  for (;;) {   // bounded: the shared counter only grows
    if (wd.expired(&st->timeout)) break;
    int64_t base = 0;
    int fetch = B;
    if (lane == 0) {
      const unsigned long long seen = *reinterpret_cast<volatile unsigned long long*>(&st->work_ctr);
      const int64_t f = (n - (int64_t)seen) / share;
      fetch = f >= B ? B : (f < 32 ? 32 : (int)(f & ~31ll));
      base = (int64_t)atomicAdd(&st->work_ctr, (unsigned long long)fetch);
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    fetch = __shfl_sync(0xffffffffu, fetch, 0);
    if (base >= n) break;
    const int64_t lim = min(n, base + (int64_t)fetch);
    const int rounds = (fetch + 31) >> 5;
    // ---- phase A: sort key of each pair from an FP32 clip: 1 + 16 x its
    //      cell count + its edge intersections (0 = no pair); a cost
    //      estimate only, the FP64 clip of phase B decides
    if (lane < 8) pres[lane] = 0u;
    __syncwarp();
#pragma unroll 1
    for (int rr = 0; rr < rounds; ++rr) {
      const int64_t p = base + rr * 32 + lane;
      int key = 0;
      if (p < lim) {
        int n_int = 0;
        const int nr = clip_count_f32<NS, NM>(srec + (int64_t)SR_STRIDE * ps[p], xm, conn_m, pm[p], n_int);
        key = 1 + 16 * (nr == 0 ? 0 : (nr == 3 ? 1 : min(nr, kPolyS))) + min(n_int, 15);
        atomicOr(&pres[key >> 5], 1u << (key & 31));
      }
      keys[rr * 32 + lane] = (uint8_t)key;
    }
    __syncwarp();
    // ---- sort by key, descending, over the key values present (ballots)
    int basecnt = 0;
#pragma unroll 1
    for (int w = 7; w >= 0; --w) {
      unsigned bits = pres[w];
      while (bits != 0u) {   // uniform across the warp
        const int b = 31 - __clz(bits);
        bits &= ~(1u << b);
        const int v = 32 * w + b;
        int before = 0;
#pragma unroll 1
        for (int rr = 0; rr < rounds; ++rr) {
          const int slot = rr * 32 + lane;
          const bool hit = keys[slot] == v;
          const unsigned mk = __ballot_sync(0xffffffffu, hit);
          if (hit) perm[basecnt + before + __popc(mk & lt_mask)] = (PermT)slot;
          before += __popc(mk);
        }
        basecnt += before;
      }
    }
    const int n_live = basecnt;
    __syncwarp();
    // ---- phase B: one pair per lane, rounds of similar cost
    for (int i0 = 0; i0 < n_live; i0 += 32) {
      const int i = i0 + lane;
      if (i < n_live)
        integrate_pair_sorted<NS, NM, SEG>(base + perm[i], ps, pm, srec, xm, conn_m, rp, Mblk, Dblk, flag, ctr);
    }
    __syncwarp();
  }
  block_count_add(&st->nonempty, ctr.nonempty);
  block_count_add(&st->gauss_points, ctr.gp);
  block_count_add(&st->cells, ctr.cells);
  block_count_add(&st->newton_fail, ctr.newton_fail);
  block_count_add(&st->xi_oor, ctr.xi_oor);
  block_count_add(&st->clip_overflow, ctr.clip_over);
  __syncthreads();
  cta_mark(cta_t, 1);
}

#ifdef MORTAR_PAIR_NS
template <int NS, int NM, bool SEG, int R>
void launch_batched_t(const IntegrateArgs& a, const RunParams& rp, int n_sm, int kWarps) {
  const size_t shm = (size_t)kWarps * BatchSmem<R>::kBytes;
  auto kern = k_integrate_batched<NS, NM, SEG, R>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarps * 32, shm);
  if (per_sm < 1) per_sm = 1;
  const unsigned grid = (unsigned)(n_sm * per_sm);
  if (a.grid_out) *a.grid_out = (int)grid;
  kern<<<grid, kWarps * 32, shm, a.stream>>>(a.ps, a.pm, a.srec, a.xm, a.conn_m, rp, a.Mblk, a.Dblk, a.flag,
                                             a.pair_cap, a.st, a.cta_t);
}

template <int NS, int NM, bool SEG>
void launch_batched_r(const IntegrateArgs& a, const RunParams& rp, int n_sm, int rounds, int warps) {
  if (rounds <= 1) launch_batched_t<NS, NM, SEG, 1>(a, rp, n_sm, warps);
  else if (rounds == 2) launch_batched_t<NS, NM, SEG, 2>(a, rp, n_sm, warps);
  else if (rounds == 4) launch_batched_t<NS, NM, SEG, 4>(a, rp, n_sm, warps);
  else if (rounds == 8) launch_batched_t<NS, NM, SEG, 8>(a, rp, n_sm, warps);
  else if (rounds == 16) launch_batched_t<NS, NM, SEG, 16>(a, rp, n_sm, warps);
  else launch_batched_t<NS, NM, SEG, 32>(a, rp, n_sm, warps);
}

template <int NS, int NM, bool SEG>
void launch_one_pair_per_thread(const IntegrateArgs& a, const RunParams& rp, int n_sm, int block, int chunk) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_integrate<NS, NM, SEG>, block, 0);
  if (per_sm < 1) per_sm = 1;
  const unsigned grid = (unsigned)(n_sm * per_sm);
  k_integrate<NS, NM, SEG><<<grid, block, 0, a.stream>>>(a.ps, a.pm, a.srec, a.xm, a.conn_m, rp, a.Mblk, a.Dblk,
                                                         a.flag, a.pair_cap, chunk, a.st);
}

}  // namespace

template <int NS, int NM>
void integrate_nsnm(const IntegrateArgs& a, const RunParams& rp, int n_sm, int variant, int block, int chunk,
                    int rounds) {
  const bool seg = rp.d_domain == 1;
  if (variant == 1) {
    if (seg) launch_one_pair_per_thread<NS, NM, true>(a, rp, n_sm, block, chunk);
    else launch_one_pair_per_thread<NS, NM, false>(a, rp, n_sm, block, chunk);
    return;
  }
  if (seg) launch_batched_r<NS, NM, true>(a, rp, n_sm, rounds, block / 32);
  else launch_batched_r<NS, NM, false>(a, rp, n_sm, rounds, block / 32);
}
template void integrate_nsnm<MORTAR_PAIR_NS, MORTAR_PAIR_NM>(const IntegrateArgs&, const RunParams&, int, int, int,
                                                              int, int);
#else   // the main part: dispatch

void launch_dispatch(const IntegrateArgs& a, const RunParams& rp, int nen_s, int nen_m, int n_sm, int variant,
                     int block, int chunk, int rounds) {
  if (nen_s == 4 && nen_m == 4) integrate_nsnm<4, 4>(a, rp, n_sm, variant, block, chunk, rounds);
  else if (nen_s == 4 && nen_m == 3) integrate_nsnm<4, 3>(a, rp, n_sm, variant, block, chunk, rounds);
  else if (nen_s == 3 && nen_m == 4) integrate_nsnm<3, 4>(a, rp, n_sm, variant, block, chunk, rounds);
  else integrate_nsnm<3, 3>(a, rp, n_sm, variant, block, chunk, rounds);
}

}  // namespace

bool integrate_batched_fits(int rounds, int block) {
  const size_t per_warp = (size_t)BatchSmem<32>::kBytes;   // the largest batch
  (void)rounds;
  return block >= 32 && block <= kMaxPairBlock && (size_t)(block / 32) * per_warp <= kMaxDynSmem;
}

int integrate_rounds(int rounds, int block) {
  (void)block;
  return rounds <= 1 ? 1 : (rounds >= 32 ? 32 : rounds);
}

void launch_integrate_raw(const IntegrateArgs& a, const RunParams& rp, int nen_s, int nen_m, int n_sm) {
  launch_dispatch(a, rp, nen_s, nen_m, n_sm, 0, 128, 32, 2);
}

void launch_integrate(mortar_ctx* c, const RunParams& rp) {
  if (quadratic_slave(c)) {
    launch_integrate_quadratic(c, rp);
    return;
  }
  if (rp.integration == 1) {
    c->pair_grid = 0;
    launch_integrate_element_based(c, rp);
    return;
  }
  IntegrateArgs a{c->pairs_s.as<int32_t>(), c->pairs_m.as<int32_t>(), c->srec.as<double>(), c->xm.as<double>(),
                  c->conn_m.as<int32_t>(), c->Mblk.as<double>(), c->Dblk.as<double>(), c->flag.as<uint8_t>(),
                  c->pair_cap, c->dstat.as<DevStatus>(), c->stream};
  c->pair_grid = 0;
  if (c->timing && c->cta_t.p) {
    a.cta_t = c->cta_t.as<unsigned long long>();
    a.grid_out = &c->pair_grid;
  }
  const int block = c->block_size > 0 ? c->block_size : 128;
  const int chunk = c->chunk_pairs > 0 ? c->chunk_pairs : 32;
  const int rounds = integrate_rounds(c->rounds > 0 ? c->rounds : 2, block);
  launch_dispatch(a, rp, c->nen_s, c->nen_m, c->n_sm, c->variant, block, chunk, rounds);
}
#endif  // MORTAR_PAIR_NS

}  // namespace mortar
