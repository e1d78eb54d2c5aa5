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
//  * variant 0 (default): each warp takes a batch of 32 R consecutive pairs.
//    Phase A clips one pair per lane and leaves the merged polygon and the
//    master map in shared memory; the warp then sorts its pairs by cell count
//    (ballot counting sort) and phase B integrates them in rounds of 32 lanes
//    with (nearly) equal cell counts.  Affine element maps are inverted with
//    one precomputed 2x2 inverse; bilinear ones by Newton in FP32 on
//    power-of-two-scaled coordinates, then one FP64 Newton step with an
//    FP64 residual (the converged xi agrees with a full FP64 Newton to
//    rounding; MapInverse in clip.cuh).
//  * variant 1: one pair per thread, FP64 Newton from xi = 0 at every point
//    (the oracle's iteration), kept as the reference schedule.
//
// Both are persistent grids taking work from a global counter; the loops are
// bounded by the pair count.
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
template <int R>
struct BatchSmem {   // per-warp shared layout for 32 R pairs
  static constexpr int B = 32 * R;
  static constexpr int kPu = 0;
  static constexpr int kPv = kPu + B * kPolyS;
  static constexpr int kCen = kPv + B * kPolyS;
  static constexpr int kMap = kCen + B * 2;
  static constexpr int kDoubles = kMap + B * 8;
  static constexpr int kBytes = kDoubles * 8 + B * 4 * 2 + B * 2;   // + pidx, sidx (int32), nr/perm (int8)
};

template <int NS, int NM, bool SEG, int R>
__global__ void __launch_bounds__(kMaxPairBlock) k_integrate_batched(
    const int32_t* __restrict__ ps, const int32_t* __restrict__ pm, const double* __restrict__ srec,
    const double* __restrict__ xm, const int32_t* __restrict__ conn_m, RunParams rp, double* __restrict__ Mblk,
    double* __restrict__ Dblk, uint8_t* __restrict__ flag, int64_t pair_cap, DevStatus* st,
    unsigned long long* cta_t) {
  cta_mark(cta_t, 0);
  using L = BatchSmem<R>;
  constexpr int B = L::B;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* my = smem_raw + (size_t)warp * L::kBytes;
  double* sd = reinterpret_cast<double*>(my);
  double* Pu = sd + L::kPu;
  double* Pv = sd + L::kPv;
  double* Cen = sd + L::kCen;
  double* Map = sd + L::kMap;
  int32_t* pidx = reinterpret_cast<int32_t*>(sd + L::kDoubles);
  int32_t* sidx = pidx + B;
  int8_t* nrs = reinterpret_cast<int8_t*>(sidx + B);
  uint8_t* perm = reinterpret_cast<uint8_t*>(nrs + B);

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
    // ---- phase A: clip one pair per lane, results to shared memory
    int key[R];
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      const int slot = rr * 32 + lane;
      const int64_t p = base + slot;
      int nr = 0;
      if (p < lim) {
        const int32_t s = ps[p];
        const double* r = srec + (int64_t)SR_STRIDE * s;
        PlaneMap mm;
        nr = clip_polygon<NS, NM, kPolyS>(r, xm, conn_m, pm[p], mm, Pu + slot * kPolyS, Pv + slot * kPolyS,
                                          ctr.clip_over);
        if (nr == 0) {
          write_zero_blocks(p, SEG, Mblk, Dblk);
          flag[p] = 0;
        } else {
          double* mp = Map + slot * 8;
          mp[0] = mm.c0u; mp[1] = mm.c0v; mp[2] = mm.c1u; mp[3] = mm.c1v;
          mp[4] = mm.c2u; mp[5] = mm.c2v; mp[6] = mm.c3u; mp[7] = mm.c3v;
          if (nr > 3) {
            double su = 0.0, sv = 0.0;
            for (int k = 0; k < nr; ++k) { su += Pu[slot * kPolyS + k]; sv += Pv[slot * kPolyS + k]; }
            Cen[2 * slot] = su / (double)nr;
            Cen[2 * slot + 1] = sv / (double)nr;
          }
          pidx[slot] = (int32_t)p;
          sidx[slot] = s;
        }
      }
      nrs[slot] = (int8_t)nr;
      key[rr] = nr == 0 ? 0 : (nr == 3 ? 1 : nr);   // cells of the pair
    }
    // ---- sort slots by cell count, descending (ballot counting sort)
    int pos[R];
    int basecnt = 0;
#pragma unroll 1
    for (int v = kPolyS; v >= 1; --v) {
      int before = 0;
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        const unsigned mk = __ballot_sync(0xffffffffu, key[rr] == v);
        if (key[rr] == v) pos[rr] = basecnt + before + __popc(mk & lt_mask);
        before += __popc(mk);
      }
      basecnt += before;
    }
    const int n_live = basecnt;
#pragma unroll
    for (int rr = 0; rr < R; ++rr)
      if (key[rr] > 0) perm[pos[rr]] = (uint8_t)(rr * 32 + lane);
    __syncwarp();
    // ---- phase B: integrate, one pair per lane, rounds of similar cell counts
    for (int i0 = 0; i0 < n_live; i0 += 32) {
      const int i = i0 + lane;
      if (i >= n_live) continue;
      const int slot = perm[i];
      const int nr = nrs[slot];
      const int64_t p = pidx[slot];
      const double* r = srec + (int64_t)SR_STRIDE * sidx[slot];
      const double* mp = Map + slot * 8;
      PlaneMap mmap;
      mmap.c0u = mp[0]; mmap.c0v = mp[1]; mmap.c1u = mp[2]; mmap.c1v = mp[3];
      mmap.c2u = mp[4]; mmap.c2v = mp[5]; mmap.c3u = mp[6]; mmap.c3v = mp[7];
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
      const double* pu = Pu + slot * kPolyS;
      const double* pv = Pv + slot * kPolyS;
      const int ncell = nr == 3 ? 1 : nr;
      const double cu = nr == 3 ? pu[0] : Cen[2 * slot], cv = nr == 3 ? pv[0] : Cen[2 * slot + 1];
      ctr.cells += ncell;
      ctr.nonempty++;
      for (int cI = 0; cI < ncell; ++cI) {
        const int ib = nr == 3 ? 1 : cI;
        const int iw = nr == 3 ? 2 : (cI + 1 == nr ? 0 : cI + 1);
        const double au = cu, av = cv;
        const double e1u = pu[ib] - au, e1v = pv[ib] - av, e2u = pu[iw] - au, e2v = pv[iw] - av;
        const double area = 0.5 * fabs(cross2(e1u, e1v, e2u, e2v));
#pragma unroll 1
        for (int q = 0; q < 7; ++q) {
          double l1, l2, w;
          tri7_point(q, l1, l2, w);
          const double xu = au + l1 * e1u + l2 * e2u;
          const double xv = av + l1 * e1v + l2 * e2v;
          double xs1, xs2, xm1, xm2;
          if (!si.solve(xu, xv, xs1, xs2)) ctr.newton_fail++;
          if (!mi.solve(xu, xv, xm1, xm2)) ctr.newton_fail++;
          const double w4 = 0.25 * (w * area);
          double Ns[4], Nm[4];
          if constexpr (NS == 4) {   // W * N_s
            const double qa = w4 * (1.0 - xs1), qb = w4 * (1.0 + xs1), c = 1.0 - xs2, dd = 1.0 + xs2;
            Ns[0] = qa * c; Ns[1] = qb * c; Ns[2] = qb * dd; Ns[3] = qa * dd;
          } else {
            const double W = 4.0 * w4;
            Ns[0] = W * (1.0 - xs1 - xs2); Ns[1] = W * xs1; Ns[2] = W * xs2; Ns[3] = 0.0;
          }
          shape_fn<NM>(xm1, xm2, Nm);
#pragma unroll
          for (int a = 0; a < NS; ++a) {
#pragma unroll
            for (int l = 0; l < NM; ++l) G[a][l] = fma(Ns[a], Nm[l], G[a][l]);
          }
          if (SEG) {   // H = sum W N_s N_s^T = sum (W N_s) N_s^T, N_s = (W N_s) / W
            double Nu[4];
            shape_fn<NS>(xs1, xs2, Nu);
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
  else launch_batched_t<NS, NM, SEG, 4>(a, rp, n_sm, warps);
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
  const size_t per_warp = rounds <= 1 ? BatchSmem<1>::kBytes : (rounds == 2 ? BatchSmem<2>::kBytes : BatchSmem<4>::kBytes);
  return block >= 32 && block <= kMaxPairBlock && (size_t)(block / 32) * per_warp <= kMaxDynSmem;
}

int integrate_rounds(int rounds, int block) {
  // the integration kernel keeps each batch's polygons in shared memory:
  // at most 4 rounds (128 pairs per warp), fewer where 8 warps would not fit
  int r = rounds <= 1 ? 1 : (rounds == 2 ? 2 : 4);
  while (r > 1 && !integrate_batched_fits(r, block)) r >>= 1;
  return r;
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
