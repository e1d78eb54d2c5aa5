// Segment-based integration of quadratic slave elements (tri6, quad8; the
// paper's isoparametric discretisation, Eq. AnsatzDiscretization, with
// quadratic shape functions and standard Lagrange multipliers).
//
// The slave surface is integrated on its piecewise flat approximation
// (Sec. 2.3): every quadratic element is split into four linear sub-elements
// (precomputed records 4 s + k: auxiliary plane, window, map), and for a pair
// (s, m) each sub-element runs the body of Algorithm 1 against the master
// element -- project, clip, centroid fan, 7-point rule, back-projection.  A
// quadrature point's sub-element parameters map affinely to the parent's,
// where the quadratic shape functions are evaluated:
//     M_pair[a][l] += W N_a(xi_parent) N_l(xi_m)      (8 x 4 block per pair).
// D is the element-domain integral of the precomputation.
//
// Work unit = (pair, sub-element), u = 4 p + k: the four sub-elements of a
// pair overlap the master element in different cell counts (often none), so
// one pair per lane would leave most lanes idle.  A persistent grid takes
// batches of units (guided self-scheduling), sorts each batch by the cell
// count and edge intersections of an FP32 clip, and runs the units in rounds
// of similar cost: FP64 clip, quadrature into the unit's 8 x 4 block.  A
// second kernel sums the four unit blocks of every pair in the fixed order
// k = 0..3 (bitwise reproducible) into the pair block and its flag.
#include <type_traits>

#include "clip.cuh"
#include "context.h"
#include "quadratic.cuh"

namespace mortar {

namespace {

constexpr int kQThreads = 128;
constexpr int kQRounds = 16;   // units per warp batch: 32 x 16

struct QCounters {
  unsigned long long gp = 0, cells = 0, newton_fail = 0, clip_over = 0;
};

// One unit: sub-element k of pair p.  Writes the unit's 8 x 4 block and flag.
template <int NP, int NM>
__device__ void integrate_unit(int64_t u, const int32_t* __restrict__ ps, const int32_t* __restrict__ pm,
                               const double* __restrict__ srec, const double* __restrict__ xm,
                               const int32_t* __restrict__ conn_m, double* __restrict__ U,
                               uint8_t* __restrict__ uflag, QCounters& ctr) {
  constexpr int NSUB = NP == 8 ? 4 : 3;
  const int64_t p = u >> 2;
  const int k = (int)(u & 3);
  const int32_t s = ps[p], m = pm[p];
  const double* r = srec + (int64_t)SR_STRIDE * (4 * (int64_t)s + k);
  double2* out = reinterpret_cast<double2*>(U + 32 * u);
  PlaneMap mmap;
  double Pu[kPolyS], Pv[kPolyS];
  const int nr = clip_polygon<NSUB, NM, kPolyS>(r, xm, conn_m, m, mmap, Pu, Pv, ctr.clip_over);
  if (nr == 0) {
#pragma unroll
    for (int i = 0; i < 16; ++i) __stcs(out + i, make_double2(0.0, 0.0));
    uflag[u] = 0;
    return;
  }
  double Mq[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int l = 0; l < 4; ++l) Mq[a][l] = 0.0;
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
  double cu = Pu[0], cv = Pv[0];
  int ncell = 1;
  if (nr > 3) {
    double su = 0.0, sv = 0.0;
    for (int j = 0; j < nr; ++j) { su += Pu[j]; sv += Pv[j]; }
    cu = su * kInvCount[nr];
    cv = sv * kInvCount[nr];
    ncell = nr;
  }
  ctr.cells += ncell;
  for (int cI = 0; cI < ncell; ++cI) {
    const int ib = nr == 3 ? 1 : cI;
    const int iw = nr == 3 ? 2 : (cI + 1 == nr ? 0 : cI + 1);
    const double e1u = Pu[ib] - cu, e1v = Pv[ib] - cv, e2u = Pu[iw] - cu, e2v = Pv[iw] - cv;
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
      double xp, ep;
      sub_to_parent<NP>(k, xs1, xs2, xp, ep);
      double Np[8], WNm[4];   // W folded into the master side (4 products instead of NP)
      shape_quadratic<NP>(xp, ep, Np);
      if constexpr (NM == 4) {   // 1/4 of the quad4 shape functions folded into W
        const double wq = 0.25 * (w * area);
        const double qa = fma(-wq, xm1, wq), qb = fma(wq, xm1, wq);
        WNm[0] = fma(-qa, xm2, qa); WNm[1] = fma(-qb, xm2, qb); WNm[2] = fma(qb, xm2, qb); WNm[3] = fma(qa, xm2, qa);
      } else {
        const double W = w * area;
        WNm[1] = W * xm1; WNm[2] = W * xm2; WNm[0] = W - WNm[1] - WNm[2]; WNm[3] = 0.0;
      }
#pragma unroll
      for (int a = 0; a < NP; ++a)
#pragma unroll
        for (int l = 0; l < NM; ++l) Mq[a][l] = fma(Np[a], WNm[l], Mq[a][l]);
      ctr.gp++;
    }
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    __stcs(out + 2 * a, make_double2(Mq[a][0], Mq[a][1]));
    __stcs(out + 2 * a + 1, make_double2(Mq[a][2], NM == 4 ? Mq[a][3] : 0.0));
  }
  uflag[u] = 1;
}

template <int NP, int NM>
__global__ void __launch_bounds__(kQThreads) k_integrate_quadratic(
    const int32_t* __restrict__ ps, const int32_t* __restrict__ pm, const double* __restrict__ srec,
    const double* __restrict__ xm, const int32_t* __restrict__ conn_m, RunParams rp, double* __restrict__ U,
    uint8_t* __restrict__ uflag, int64_t pair_cap, DevStatus* st) {
  constexpr int NSUB = NP == 8 ? 4 : 3;
  constexpr int B = 32 * kQRounds;
  using PermT = typename std::conditional<(B > 256), uint16_t, uint8_t>::type;
  __shared__ PermT perm_s[kQThreads / 32][B];
  __shared__ uint8_t key_s[kQThreads / 32][B];
  __shared__ unsigned pres_s[kQThreads / 32][8];
  PermT* perm = perm_s[threadIdx.x >> 5];
  uint8_t* keys = key_s[threadIdx.x >> 5];
  unsigned* pres = pres_s[threadIdx.x >> 5];
  QCounters ctr;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const bool ok = st->over_pairs == 0 && st->over_bins == 0;
  const int64_t n = ok ? 4 * (int64_t)min((unsigned long long)pair_cap, st->n_pairs) : 0;   // units
  const int64_t share = 2 * (int64_t)gridDim.x * (blockDim.x >> 5);
  const Watchdog wd(rp.watchdog_us);
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
    // phase A: sort key of each unit from an FP32 clip of its sub-element
    if (lane < 8) pres[lane] = 0u;
    __syncwarp();
#pragma unroll 1
    for (int rr = 0; rr < rounds; ++rr) {
      const int64_t u = base + rr * 32 + lane;
      int key = 0;
      if (u < lim) {
        const int64_t p = u >> 2;
        const double* r = srec + (int64_t)SR_STRIDE * (4 * (int64_t)ps[p] + (u & 3));
        int n_int = 0;
        const int nr = clip_count_f32<NSUB, NM>(r, xm, conn_m, pm[p], n_int);
        key = 1 + 16 * (nr == 0 ? 0 : (nr == 3 ? 1 : min(nr, kPolyS))) + min(n_int, 15);
        atomicOr(&pres[key >> 5], 1u << (key & 31));
      }
      keys[rr * 32 + lane] = (uint8_t)key;
    }
    __syncwarp();
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
    // phase B: one unit per lane, rounds of similar cost
    for (int i0 = 0; i0 < n_live; i0 += 32) {
      const int i = i0 + lane;
      if (i < n_live) integrate_unit<NP, NM>(base + perm[i], ps, pm, srec, xm, conn_m, U, uflag, ctr);
    }
    __syncwarp();
  }
  block_count_add(&st->gauss_points, ctr.gp);
  block_count_add(&st->cells, ctr.cells);
  block_count_add(&st->newton_fail, ctr.newton_fail);
  block_count_add(&st->clip_overflow, ctr.clip_over);
}

// Pair block = sum of its four unit blocks in the order k = 0..3; flag = any.
// Sixteen threads per pair, thread j summing the j-th 16-byte pair of entries
// of the four blocks: every load and store of a half-warp is one contiguous
// 256-byte segment.
__global__ void __launch_bounds__(256) k_quadratic_reduce(const double* __restrict__ U,
                                                          const uint8_t* __restrict__ uflag, int64_t pair_cap,
                                                          double* __restrict__ Mblk, uint8_t* __restrict__ flag,
                                                          DevStatus* st) {
  const bool ok = st->over_pairs == 0 && st->over_bins == 0;
  const int64_t n = ok ? (int64_t)min((unsigned long long)pair_cap, st->n_pairs) : 0;
  const int j = threadIdx.x & 15;
  unsigned long long ne = 0;
  for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 4; p < n;
       p += ((int64_t)gridDim.x * blockDim.x) >> 4) {
    const double2* u0 = reinterpret_cast<const double2*>(U + 128 * p) + j;
    double2 acc = __ldcs(u0);
#pragma unroll
    for (int k = 1; k < 4; ++k) {
      const double2 t = __ldcs(u0 + 16 * k);
      acc.x += t.x;
      acc.y += t.y;
    }
    __stcs(reinterpret_cast<double2*>(Mblk + 32 * p) + j, acc);
    if (j == 0) {
      const uint32_t f = *reinterpret_cast<const uint32_t*>(uflag + 4 * p);
      flag[p] = f != 0u ? 1 : 0;
      ne += f != 0u ? 1ull : 0ull;
    }
  }
  block_count_add(&st->nonempty, ne);
}

template <int NP, int NM>
void launch_q(mortar_ctx* c, const RunParams& rp) {
  auto kern = k_integrate_quadratic<NP, NM>;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kQThreads, 0);
  if (per_sm < 1) per_sm = 1;
  kern<<<(unsigned)(c->n_sm * per_sm), kQThreads, 0, c->stream>>>(
      c->pairs_s.as<int32_t>(), c->pairs_m.as<int32_t>(), c->srec.as<double>(), c->xm.as<double>(),
      c->conn_m.as<int32_t>(), rp, c->Qunit.as<double>(), c->Qflag.as<uint8_t>(), c->pair_cap,
      c->dstat.as<DevStatus>());
  k_quadratic_reduce<<<(unsigned)(c->n_sm * 8), 256, 0, c->stream>>>(c->Qunit.as<double>(), c->Qflag.as<uint8_t>(),
                                                                     c->pair_cap, c->Mblk.as<double>(),
                                                                     c->flag.as<uint8_t>(), c->dstat.as<DevStatus>());
}

}  // namespace

void launch_integrate_quadratic(mortar_ctx* c, const RunParams& rp) {
  c->pair_grid = 0;
  if (c->nen_s == 8 && c->nen_m == 4) launch_q<8, 4>(c, rp);
  else if (c->nen_s == 8) launch_q<8, 3>(c, rp);
  else if (c->nen_m == 4) launch_q<6, 4>(c, rp);
  else launch_q<6, 3>(c, rp);
}

}  // namespace mortar
