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
// D is the element-domain integral of the precomputation.  One pair per
// thread in a persistent grid taking 32-pair chunks from a work counter.
#include "clip.cuh"
#include "context.h"
#include "quadratic.cuh"

namespace mortar {

namespace {

constexpr int kQThreads = 128;

struct QCounters {
  unsigned long long nonempty = 0, gp = 0, cells = 0, newton_fail = 0, clip_over = 0;
};

template <int NP, int NM>
__device__ void integrate_quadratic_one(int64_t p, const int32_t* __restrict__ ps, const int32_t* __restrict__ pm,
                                        const double* __restrict__ srec, const double* __restrict__ xm,
                                        const int32_t* __restrict__ conn_m, double* __restrict__ Mblk,
                                        uint8_t* __restrict__ flag, QCounters& ctr) {
  constexpr int NSUB = NP == 8 ? 4 : 3;
  const int32_t s = ps[p], m = pm[p];
  double Mq[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int l = 0; l < 4; ++l) Mq[a][l] = 0.0;
  bool any = false;
#pragma unroll 1
  for (int k = 0; k < 4; ++k) {
    const double* r = srec + (int64_t)SR_STRIDE * (4 * (int64_t)s + k);
    PlaneMap mmap;
    double Pu[kMaxPoly], Pv[kMaxPoly];
    const int nr = clip_polygon<NSUB, NM, kMaxPoly>(r, xm, conn_m, m, mmap, Pu, Pv, ctr.clip_over);
    if (nr == 0) continue;
    any = true;
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
      cu = su / (double)nr;
      cv = sv / (double)nr;
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
        double Np[8], Nm[4];
        shape_quadratic<NP>(xp, ep, Np);
        shape_fn<NM>(xm1, xm2, Nm);
        const double W = w * area;
#pragma unroll
        for (int a = 0; a < NP; ++a) {
          const double wn = W * Np[a];
#pragma unroll
          for (int l = 0; l < NM; ++l) Mq[a][l] = fma(wn, Nm[l], Mq[a][l]);
        }
        ctr.gp++;
      }
    }
  }
  double2* out = reinterpret_cast<double2*>(Mblk + 32 * p);
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    out[2 * a] = make_double2(Mq[a][0], Mq[a][1]);
    out[2 * a + 1] = make_double2(Mq[a][2], NM == 4 ? Mq[a][3] : 0.0);
  }
  flag[p] = any ? 1 : 0;
  if (any) ctr.nonempty++;
}

template <int NP, int NM>
__global__ void __launch_bounds__(kQThreads) k_integrate_quadratic(
    const int32_t* __restrict__ ps, const int32_t* __restrict__ pm, const double* __restrict__ srec,
    const double* __restrict__ xm, const int32_t* __restrict__ conn_m, RunParams rp, double* __restrict__ Mblk,
    uint8_t* __restrict__ flag, int64_t pair_cap, DevStatus* st) {
  QCounters ctr;
  const int lane = threadIdx.x & 31;
  const bool ok = st->over_pairs == 0 && st->over_bins == 0;
  const int64_t n = ok ? (int64_t)min((unsigned long long)pair_cap, st->n_pairs) : 0;
  const Watchdog wd(rp.watchdog_us);
  for (;;) {   // bounded: the shared counter only grows
    if (wd.expired(&st->timeout)) break;
    int64_t base = 0;
    if (lane == 0) base = (int64_t)atomicAdd(&st->work_ctr, 32ull);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= n) break;
    const int64_t p = base + lane;
    if (p < n) integrate_quadratic_one<NP, NM>(p, ps, pm, srec, xm, conn_m, Mblk, flag, ctr);
  }
  block_count_add(&st->nonempty, ctr.nonempty);
  block_count_add(&st->gauss_points, ctr.gp);
  block_count_add(&st->cells, ctr.cells);
  block_count_add(&st->newton_fail, ctr.newton_fail);
  block_count_add(&st->clip_overflow, ctr.clip_over);
}

template <int NP, int NM>
void launch_q(mortar_ctx* c, const RunParams& rp) {
  auto kern = k_integrate_quadratic<NP, NM>;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kQThreads, 0);
  if (per_sm < 1) per_sm = 1;
  kern<<<(unsigned)(c->n_sm * per_sm), kQThreads, 0, c->stream>>>(
      c->pairs_s.as<int32_t>(), c->pairs_m.as<int32_t>(), c->srec.as<double>(), c->xm.as<double>(),
      c->conn_m.as<int32_t>(), rp, c->Mblk.as<double>(), c->flag.as<uint8_t>(), c->pair_cap,
      c->dstat.as<DevStatus>());
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
