// Per-pair segment-based mortar integration (Algorithm 1 body, Sec. 2.3).
//
// For one slave/master pair: project the master nodes onto the slave
// element's auxiliary plane (Fig. 1: x0, n0), clip the master polygon by the
// slave polygon (Sutherland-Hodgman with an absolute inside band eps_in),
// merge near-duplicate vertices, discard slivers, split the clip polygon
// into a centroid fan of triangular cells, and integrate with the 7-point
// degree-5 rule.  At every quadrature point both elements are inverted
// (chi_h: Newton on the bilinear map in the plane) and
//     G[c][l] += W N_c(xi_s) N_l(xi_m),   H[c][b] += W N_c(xi_s) N_b(xi_s)
// so that M_pair = A G and D_pair = A H with the slave element's LM
// coefficients A (Phi_a = sum_c A[a][c] N_c, Eq. AnsatzDiscretizationLagrangeMult).
//
// Execution: a persistent grid; each warp takes 32 consecutive pairs at a time
// from a global work counter (one pair per lane), so uneven pair costs and
// uneven interfaces of a batch balance across the chip.  The loop is bounded
// by the pair count.  All arithmetic is FP64.
#include "context.h"

namespace mortar {

namespace {

struct PairCounters {
  unsigned long long nonempty = 0, gp = 0, cells = 0, newton_fail = 0, xi_oor = 0, clip_over = 0;
};

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
  bool nonempty = false;
  const double eps_in = r[SR_EPSIN];
  if (eps_in >= 0.0) {
    const double x0x = r[SR_X0], x0y = r[SR_X0 + 1], x0z = r[SR_X0 + 2];
    const double t1x = r[SR_T1], t1y = r[SR_T1 + 1], t1z = r[SR_T1 + 2];
    const double t2x = r[SR_T2], t2y = r[SR_T2 + 1], t2z = r[SR_T2 + 2];
    // ---- project master nodes onto the auxiliary plane (in-plane coords)
    double mu[4], mv[4];
#pragma unroll
    for (int l = 0; l < NM; ++l) {
      const int64_t n = conn_m[(int64_t)NM * m + l];
      const double dx = xm[3 * n] - x0x, dy = xm[3 * n + 1] - x0y, dz = xm[3 * n + 2] - x0z;
      mu[l] = dx * t1x + dy * t1y + dz * t1z;
      mv[l] = dx * t2x + dy * t2y + dz * t2z;
    }
    const PlaneMap mmap = plane_map<NM>(mu, mv);
    PlaneMap smap;
    smap.c0u = r[SR_C + 0]; smap.c0v = r[SR_C + 1]; smap.c1u = r[SR_C + 2]; smap.c1v = r[SR_C + 3];
    smap.c2u = r[SR_C + 4]; smap.c2v = r[SR_C + 5]; smap.c3u = r[SR_C + 6]; smap.c3v = r[SR_C + 7];
    double ma2 = 0.0;
#pragma unroll
    for (int l = 0; l < NM; ++l) ma2 += cross2(mu[l], mv[l], mu[(l + 1) % NM], mv[(l + 1) % NM]);
    // ---- subject polygon (master, CCW)
    double Pu[kMaxPoly], Pv[kMaxPoly], Qu[kMaxPoly], Qv[kMaxPoly], d[kMaxPoly];
#pragma unroll
    for (int l = 0; l < NM; ++l) {
      const int src = ma2 < 0.0 ? NM - 1 - l : l;
      Pu[l] = mu[src];
      Pv[l] = mv[src];
    }
    int n = NM;
    // ---- Sutherland-Hodgman against each slave edge (window CCW)
    for (int i = 0; i < NS && n > 0; ++i) {
      const int i1 = i + 1 == NS ? 0 : i + 1;
      const double au = r[SR_PS + 2 * i], av = r[SR_PS + 2 * i + 1];
      const double eu = r[SR_PS + 2 * i1] - au, ev = r[SR_PS + 2 * i1 + 1] - av;
      for (int k = 0; k < n; ++k) d[k] = cross2(eu, ev, Pu[k] - au, Pv[k] - av);
      int o = 0;
      for (int k = 0; k < n; ++k) {
        const int k1 = k + 1 == n ? 0 : k + 1;
        const double dp = d[k], dq = d[k1];
        if ((dp > eps_in && dq < -eps_in) || (dp < -eps_in && dq > eps_in)) {
          const double t = dp / (dp - dq);
          if (o < kMaxPoly) {
            Qu[o] = Pu[k] + t * (Pu[k1] - Pu[k]);
            Qv[o] = Pv[k] + t * (Pv[k1] - Pv[k]);
          }
          ++o;
        }
        if (dq >= -eps_in) {
          if (o < kMaxPoly) { Qu[o] = Pu[k1]; Qv[o] = Pv[k1]; }
          ++o;
        }
      }
      if (o > kMaxPoly) { ctr.clip_over++; o = kMaxPoly; }
      for (int k = 0; k < o; ++k) { Pu[k] = Qu[k]; Pv[k] = Qv[k]; }
      n = o;
    }
    // ---- merge consecutive (cyclic) vertices closer than eps_merge
    const double em2 = r[SR_EPSM2];
    int nr = 0;
    for (int k = 0; k < n; ++k) {
      if (nr > 0) {
        const double du = Pu[k] - Pu[nr - 1], dv = Pv[k] - Pv[nr - 1];
        if (du * du + dv * dv < em2) continue;
      }
      Pu[nr] = Pu[k];
      Pv[nr] = Pv[k];
      ++nr;
    }
    while (nr > 1) {
      const double du = Pu[nr - 1] - Pu[0], dv = Pv[nr - 1] - Pv[0];
      if (du * du + dv * dv < em2) --nr; else break;
    }
    double pa2 = 0.0;
    for (int k = 0; k < nr; ++k) {
      const int k1 = k + 1 == nr ? 0 : k + 1;
      pa2 += cross2(Pu[k], Pv[k], Pu[k1], Pv[k1]);
    }
    if (nr >= 3 && !(0.5 * fabs(pa2) < r[SR_EPSA])) {
      nonempty = true;
      // ---- centroid fan (a triangle stays one cell)
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
      for (int cI = 0; cI < ncell; ++cI) {
        double au, av, bu, bv, wu, wv;   // cell vertices a, b, c(=w)
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
    }
  }
  if (nonempty) ctr.nonempty++;
  // ---- M = A G, D = A H
  double A[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) A[a][b] = r[SR_A + 4 * a + b];
  double* mo = Mblk + 16 * p;
  const bool dual = rp.lm == 1;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      double v = 0.0;
      if (a < NS && l < NM) {
        if (dual) {
#pragma unroll
          for (int c = 0; c < NS; ++c) v += A[a][c] * G[c][l];
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
            for (int c = 0; c < NS; ++c) v += A[a][c] * H[c][b];
          } else {
            v = H[a][b];
          }
        }
        dout[4 * a + b] = v;
      }
  }
  flag[p] = nonempty ? 1 : 0;
}

template <int NS, int NM, bool SEG>
__global__ void __launch_bounds__(128) k_integrate(const int32_t* __restrict__ ps, const int32_t* __restrict__ pm,
                                                   const double* __restrict__ srec, const double* __restrict__ xm,
                                                   const int32_t* __restrict__ conn_m, RunParams rp,
                                                   double* __restrict__ Mblk, double* __restrict__ Dblk,
                                                   uint8_t* __restrict__ flag, int64_t pair_cap, int32_t chunk,
                                                   DevStatus* st) {
  PairCounters ctr;
  const int lane = threadIdx.x & 31;
  const bool ok = st->over_pairs == 0 && st->over_bins == 0;
  const int64_t n = ok ? (int64_t)min((unsigned long long)pair_cap, st->n_pairs) : 0;
  // bounded work loop: the counter only grows, so at most n / chunk fetches succeed
  for (;;) {
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

template <int NS, int NM>
void launch_nsnm(mortar_ctx* c, const RunParams& rp, unsigned grid, unsigned block, int32_t chunk) {
  DevStatus* st = c->dstat.as<DevStatus>();
  if (rp.d_domain == 1)
    k_integrate<NS, NM, true><<<grid, block, 0, c->stream>>>(
        c->pairs_s.as<int32_t>(), c->pairs_m.as<int32_t>(), c->srec.as<double>(), c->xm.as<double>(),
        c->conn_m.as<int32_t>(), rp, c->Mblk.as<double>(), c->Dblk.as<double>(), c->flag.as<uint8_t>(), c->pair_cap,
        chunk, st);
  else
    k_integrate<NS, NM, false><<<grid, block, 0, c->stream>>>(
        c->pairs_s.as<int32_t>(), c->pairs_m.as<int32_t>(), c->srec.as<double>(), c->xm.as<double>(),
        c->conn_m.as<int32_t>(), rp, c->Mblk.as<double>(), c->Dblk.as<double>(), c->flag.as<uint8_t>(), c->pair_cap,
        chunk, st);
}

template <int NS, int NM>
void launch_raw_nsnm(const IntegrateArgs& a, const RunParams& rp, unsigned grid, unsigned block, int32_t chunk) {
  if (rp.d_domain == 1)
    k_integrate<NS, NM, true><<<grid, block, 0, a.stream>>>(a.ps, a.pm, a.srec, a.xm, a.conn_m, rp, a.Mblk, a.Dblk,
                                                           a.flag, a.pair_cap, chunk, a.st);
  else
    k_integrate<NS, NM, false><<<grid, block, 0, a.stream>>>(a.ps, a.pm, a.srec, a.xm, a.conn_m, rp, a.Mblk, a.Dblk,
                                                            a.flag, a.pair_cap, chunk, a.st);
}

}  // namespace

void launch_integrate_raw(const IntegrateArgs& a, const RunParams& rp, int nen_s, int nen_m, int n_sm) {
  const unsigned block = 128u;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_integrate<4, 4, false>, (int)block, 0);
  if (per_sm < 1) per_sm = 1;
  const unsigned grid = (unsigned)(n_sm * per_sm);
  if (nen_s == 4 && nen_m == 4) launch_raw_nsnm<4, 4>(a, rp, grid, block, 32);
  else if (nen_s == 4 && nen_m == 3) launch_raw_nsnm<4, 3>(a, rp, grid, block, 32);
  else if (nen_s == 3 && nen_m == 4) launch_raw_nsnm<3, 4>(a, rp, grid, block, 32);
  else launch_raw_nsnm<3, 3>(a, rp, grid, block, 32);
}

void launch_integrate(mortar_ctx* c, const RunParams& rp) {
  const unsigned block = c->block_size > 0 ? (unsigned)c->block_size : 128u;
  const int32_t chunk = c->chunk_pairs > 0 ? c->chunk_pairs : 32;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_integrate<4, 4, false>, (int)block, 0);
  if (per_sm < 1) per_sm = 1;
  const unsigned grid = (unsigned)(c->n_sm * per_sm);
  if (c->nen_s == 4 && c->nen_m == 4) launch_nsnm<4, 4>(c, rp, grid, block, chunk);
  else if (c->nen_s == 4 && c->nen_m == 3) launch_nsnm<4, 3>(c, rp, grid, block, chunk);
  else if (c->nen_s == 3 && c->nen_m == 4) launch_nsnm<3, 4>(c, rp, grid, block, chunk);
  else launch_nsnm<3, 3>(c, rp, grid, block, chunk);
}

}  // namespace mortar
