// Adjoint (reverse-mode gradient) of the weighted gap functional
//     J = sum_j lambda_j . ( (D X_s)_j - (M X_m)_j )
// with respect to every slave and master nodal coordinate -- the consistent
// linearisation of the mortar terms (Sec. 1 of arXiv 2202.03933).
//
// Per pair, J_pair = sum over quadrature points of W * Lh . q with
//   Lh = sum_c Lambda_c N_c(xi_s),  Lambda_c = sum_a A[a][c] lambda_a,
//   q  = [segment D] x_s(xi_s) - x_m(xi_m)   (x_s, x_m: isoparametric
//        interpolation of the ORIGINAL 3D nodes).
// The kernel recomputes the pair's geometry (nothing is stored between the
// forward and the adjoint) while recording the clip (every intersection vertex
// with its two parent vertices and its clip edge), then runs the reverse sweep:
//   quadrature point -> back-projection (implicit function theorem at the
//   converged xi: dxi = J^-1 (dx - d map)) -> cell vertices and cell area ->
//   centroid fan -> merge (selection) -> clipping stages (vertex copies and
//   edge intersections x = p + t (q - p), t = d_p / (d_p - d_q)) -> in-plane
//   coordinates u = (X - x0).t1, v = (X - x0).t2 -> auxiliary plane (x0, n0,
//   t1, t2 as functions of the slave nodes).
// The LM coefficients A (dual basis, A = Dh Me^-1) depend on the slave
// element only: each pair emits dJ/dA, a per-element kernel sums it over the
// element's pairs, adds the element-domain D term and propagates both through
// A and the element integrals to the slave nodes.  Per-pair and per-element
// gradient blocks are then gathered per node in a fixed order (no floating
// point atomics), and J is reduced with a fixed tree: results are bitwise
// reproducible.
#include <algorithm>
#include <type_traits>

#include "clip.cuh"
#include "context.h"
#include "reverse.cuh"

namespace mortar {

namespace {

constexpr int kThreads = 128;


// Reverse of the back-projection at a converged xi: accumulates the adjoint of
// the query point (xb) and of the map coefficients (cb[8] = c0u c0v c1u c1v ...).
__device__ __forceinline__ void invert_map_reverse(const PlaneMap& m, double xi, double eta, double xib0,
                                                   double xib1, double& xbu, double& xbv, double* cb) {
  const double j00 = m.c1u + m.c3u * eta, j01 = m.c2u + m.c3u * xi;
  const double j10 = m.c1v + m.c3v * eta, j11 = m.c2v + m.c3v * xi;
  const double inv = 1.0 / (j00 * j11 - j01 * j10);
  const double mu = (j11 * xib0 - j10 * xib1) * inv;   // mu = J^-T xib
  const double mv = (-j01 * xib0 + j00 * xib1) * inv;
  xbu += mu;
  xbv += mv;
  const double xe = xi * eta;
  cb[0] -= mu;      cb[1] -= mv;
  cb[2] -= xi * mu; cb[3] -= xi * mv;
  cb[4] -= eta * mu; cb[5] -= eta * mv;
  cb[6] -= xe * mu; cb[7] -= xe * mv;
}

struct AdjCounters {
  unsigned long long clip_over = 0, newton_fail = 0, nonempty = 0, cells = 0, gp = 0;
};

// Forward outputs written by the fused kernel (M, D blocks and flags).
struct FwdOut {
  double* Mblk;
  double* Dblk;
  uint8_t* flag;
};

template <int NS, int NM, bool SEG, bool DUAL>
__device__ void adjoint_one(int64_t p, const int32_t* __restrict__ ps, const int32_t* __restrict__ pm,
                            const double* __restrict__ srec, const double* __restrict__ xs,
                            const double* __restrict__ xm, const int32_t* __restrict__ conn_s,
                            const int32_t* __restrict__ conn_m, const double* __restrict__ lambda,
                            const RunParams& rp, double* __restrict__ gs_out, double* __restrict__ gm_out,
                            double* __restrict__ ab_out, double* __restrict__ J_out, AdjCounters& ctr) {
  const int32_t s = ps[p], m = pm[p];
  const double* r = srec + (int64_t)SR_STRIDE * s;
  double gX[4][3], gY[4][3], Lb[4][3];
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 3; ++k) { gX[a][k] = 0.0; gY[a][k] = 0.0; Lb[a][k] = 0.0; }
  double Jp = 0.0;
  const double eps_in = r[SR_EPSIN];
  bool nonempty = false;
  V3 X[4], Y[4], lam[4], Lam[4];
  if (eps_in >= 0.0) {
    for (int a = 0; a < NS; ++a) {
      const int64_t n = conn_s[(int64_t)NS * s + a];
      X[a] = v3(xs[3 * n], xs[3 * n + 1], xs[3 * n + 2]);
      lam[a] = v3(lambda[3 * n], lambda[3 * n + 1], lambda[3 * n + 2]);
    }
    for (int l = 0; l < NM; ++l) {
      const int64_t n = conn_m[(int64_t)NM * m + l];
      Y[l] = v3(xm[3 * n], xm[3 * n + 1], xm[3 * n + 2]);
    }
    const V3 x0 = v3(r[SR_X0], r[SR_X0 + 1], r[SR_X0 + 2]);
    const V3 t1 = v3(r[SR_T1], r[SR_T1 + 1], r[SR_T1 + 2]);
    const V3 t2 = v3(r[SR_T2], r[SR_T2 + 1], r[SR_T2 + 2]);
    // ---- forward: projection, maps, orientation (as in the integration kernel)
    double mu[4], mv[4];
    for (int l = 0; l < NM; ++l) {
      const double dx = Y[l].x - x0.x, dy = Y[l].y - x0.y, dz = Y[l].z - x0.z;
      mu[l] = dx * t1.x + dy * t1.y + dz * t1.z;
      mv[l] = dx * t2.x + dy * t2.y + dz * t2.z;
    }
    const PlaneMap mmap = plane_map<NM>(mu, mv);
    PlaneMap smap;
    smap.c0u = r[SR_C + 0]; smap.c0v = r[SR_C + 1]; smap.c1u = r[SR_C + 2]; smap.c1v = r[SR_C + 3];
    smap.c2u = r[SR_C + 4]; smap.c2v = r[SR_C + 5]; smap.c3u = r[SR_C + 6]; smap.c3v = r[SR_C + 7];
    double ma2 = 0.0;
    for (int l = 0; l < NM; ++l) ma2 += cross2(mu[l], mv[l], mu[(l + 1) % NM], mv[(l + 1) % NM]);
    const bool mrev = ma2 < 0.0;
    const bool srev = r[SR_REV] != 0.0;
    // ---- forward clip with recorded stages and merge
    ClipRec<NS> cr;
    nonempty = cr.template run<NM>(r, mu, mv, mrev, ctr.clip_over);
    const int nr = cr.nr;
    if (nonempty) {
      // LM-weighted multipliers Lambda_c
      double A[4][4];
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) A[a][b] = r[SR_A + 4 * a + b];
      for (int c = 0; c < NS; ++c) {
        if (DUAL) {
          V3 acc = v3(0, 0, 0);
          for (int a = 0; a < NS; ++a) acc = acc + A[a][c] * lam[a];
          Lam[c] = acc;
        } else {
          Lam[c] = lam[c];
        }
      }
      double Ru[kPolyA], Rv[kPolyA], Rbu[kPolyA], Rbv[kPolyA];
      for (int k = 0; k < nr; ++k) {
        Ru[k] = cr.pu(k);
        Rv[k] = cr.pv(k);
        Rbu[k] = 0.0;
        Rbv[k] = 0.0;
      }
      double cu = 0.0, cv = 0.0, cbu = 0.0, cbv = 0.0;
      int ncell = 1;
      if (nr > 3) {
        double su = 0.0, sv = 0.0;
        for (int k = 0; k < nr; ++k) { su += Ru[k]; sv += Rv[k]; }
        cu = su / (double)nr;
        cv = sv / (double)nr;
        ncell = nr;
      }
      double smb[8] = {0, 0, 0, 0, 0, 0, 0, 0}, mmb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int cI = 0; cI < ncell; ++cI) {
        int ib, iw;
        double au, av;
        if (nr == 3) {
          au = Ru[0]; av = Rv[0]; ib = 1; iw = 2;
        } else {
          au = cu; av = cv; ib = cI; iw = cI + 1 == nr ? 0 : cI + 1;
        }
        const double e1u = Ru[ib] - au, e1v = Rv[ib] - av, e2u = Ru[iw] - au, e2v = Rv[iw] - av;
        const double cr = cross2(e1u, e1v, e2u, e2v);
        const double area = 0.5 * fabs(cr);
        double area_b = 0.0, e1bu = 0.0, e1bv = 0.0, e2bu = 0.0, e2bv = 0.0, abu = 0.0, abv = 0.0;
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
          double Ns[4], Nm[4];
          shape_fn<NS>(xs1, xs2, Ns);
          shape_fn<NM>(xm1, xm2, Nm);
          V3 Lh = v3(0, 0, 0), xsI = v3(0, 0, 0), xmI = v3(0, 0, 0);
          for (int c = 0; c < NS; ++c) Lh = Lh + Ns[c] * Lam[c];
          if (SEG)
            for (int b = 0; b < NS; ++b) xsI = xsI + Ns[b] * X[b];
          for (int l = 0; l < NM; ++l) xmI = xmI + Nm[l] * Y[l];
          const V3 qv = xsI - xmI;
          const double f = dot(Lh, qv);
          Jp += W * f;
          // ---- reverse of this quadrature point
          area_b += w * f;
          const V3 Lhb = W * qv, qb = W * Lh;
          double Nsb[4] = {0, 0, 0, 0}, Nmb[4] = {0, 0, 0, 0};
          for (int c = 0; c < NS; ++c) {
            Lb[c][0] += Ns[c] * Lhb.x; Lb[c][1] += Ns[c] * Lhb.y; Lb[c][2] += Ns[c] * Lhb.z;
            Nsb[c] += dot(Lam[c], Lhb);
          }
          if (SEG)
            for (int b = 0; b < NS; ++b) {
              gX[b][0] += Ns[b] * qb.x; gX[b][1] += Ns[b] * qb.y; gX[b][2] += Ns[b] * qb.z;
              Nsb[b] += dot(X[b], qb);
            }
          for (int l = 0; l < NM; ++l) {
            gY[l][0] -= Nm[l] * qb.x; gY[l][1] -= Nm[l] * qb.y; gY[l][2] -= Nm[l] * qb.z;
            Nmb[l] -= dot(Y[l], qb);
          }
          double dNs[4][2], dNm[4][2];
          shape_grad<NS>(xs1, xs2, dNs);
          shape_grad<NM>(xm1, xm2, dNm);
          double xsb0 = 0.0, xsb1 = 0.0, xmb0 = 0.0, xmb1 = 0.0;
          for (int c = 0; c < NS; ++c) { xsb0 += Nsb[c] * dNs[c][0]; xsb1 += Nsb[c] * dNs[c][1]; }
          for (int l = 0; l < NM; ++l) { xmb0 += Nmb[l] * dNm[l][0]; xmb1 += Nmb[l] * dNm[l][1]; }
          double xbu = 0.0, xbv = 0.0;
          invert_map_reverse(smap, xs1, xs2, xsb0, xsb1, xbu, xbv, smb);
          invert_map_reverse(mmap, xm1, xm2, xmb0, xmb1, xbu, xbv, mmb);
          abu += xbu; abv += xbv;
          e1bu += l1 * xbu; e1bv += l1 * xbv;
          e2bu += l2 * xbu; e2bv += l2 * xbv;
        }
        // area = |cr| / 2
        const double crb = 0.5 * (cr < 0.0 ? -area_b : area_b);
        e1bu += crb * e2v; e1bv -= crb * e2u;
        e2bu -= crb * e1v; e2bv += crb * e1u;
        Rbu[ib] += e1bu; Rbv[ib] += e1bv;
        Rbu[iw] += e2bu; Rbv[iw] += e2bv;
        abu -= e1bu + e2bu;
        abv -= e1bv + e2bv;
        if (nr == 3) { Rbu[0] += abu; Rbv[0] += abv; } else { cbu += abu; cbv += abv; }
      }
      if (nr > 3) {
        const double inv = 1.0 / (double)nr;
        for (int k = 0; k < nr; ++k) { Rbu[k] += cbu * inv; Rbv[k] += cbv * inv; }
      }
      // ---- reverse merge and clipping stages, projection, auxiliary plane
      double sbu[4] = {0, 0, 0, 0}, sbv[4] = {0, 0, 0, 0}, mbu[4] = {0, 0, 0, 0}, mbv[4] = {0, 0, 0, 0};
      cr.template reverse<NM>(r, Rbu, Rbv, srev, mrev, sbu, sbv, mbu, mbv);
      map_coeff_reverse<NS>(smb, sbu, sbv);
      map_coeff_reverse<NM>(mmb, mbu, mbv);
      const V3 n0 = v3(r[SR_N0], r[SR_N0 + 1], r[SR_N0 + 2]);
      plane_reverse<NS, NM>(X, Y, x0, t1, t2, n0, sbu, sbv, mbu, mbv, gX, gY);
    }
  }
  double* go = gs_out + 12 * p;
  double* gmo = gm_out + 12 * p;
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 3; ++k) {
      go[3 * a + k] = gX[a][k];
      gmo[3 * a + k] = gY[a][k];
    }
  if (DUAL) {
    double* ab = ab_out + 16 * p;
    for (int a = 0; a < 4; ++a)
      for (int c = 0; c < 4; ++c)
        ab[4 * a + c] = (nonempty && a < NS && c < NS)
                            ? lam[a].x * Lb[c][0] + lam[a].y * Lb[c][1] + lam[a].z * Lb[c][2]
                            : 0.0;
  }
  J_out[p] = Jp;
}

template <int NS, int NM, bool SEG, bool DUAL>
__global__ void __launch_bounds__(kMaxPairBlock) k_adjoint_pairs(
    const int32_t* __restrict__ ps, const int32_t* __restrict__ pm, const double* __restrict__ srec,
    const double* __restrict__ xs, const double* __restrict__ xm, const int32_t* __restrict__ conn_s,
    const int32_t* __restrict__ conn_m, const double* __restrict__ lambda, RunParams rp, int64_t pair_cap,
    int32_t chunk, double* __restrict__ gs_out, double* __restrict__ gm_out, double* __restrict__ ab_out,
    double* __restrict__ J_out, DevStatus* st) {
  AdjCounters ctr;
  const int lane = threadIdx.x & 31;
  const bool ok = st->over_pairs == 0 && st->over_bins == 0;
  const int64_t n = ok ? (int64_t)min((unsigned long long)pair_cap, st->n_pairs) : 0;
  const Watchdog wd(rp.watchdog_us);
  for (;;) {   // bounded: the shared counter only grows
    if (wd.expired(&st->timeout)) break;
    int64_t base = 0;
    if (lane == 0) base = (int64_t)atomicAdd(&st->work_ctr2, (unsigned long long)chunk);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= n) break;
    const int64_t end = min(base + (int64_t)chunk, n);
    for (int64_t p = base + lane; p < end; p += 32)
      adjoint_one<NS, NM, SEG, DUAL>(p, ps, pm, srec, xs, xm, conn_s, conn_m, lambda, rp, gs_out, gm_out, ab_out,
                                     J_out, ctr);
  }
  block_count_add(&st->clip_overflow, ctr.clip_over);
  block_count_add(&st->newton_fail, ctr.newton_fail);
}

// ---------------------------------------------------------------- variant 0
// Same functional, reorganised for the FP64 pipe:
//  * the per-point work is written in the monomial basis of the shape
//    functions, N = T m with m = (1, xi, eta, xi eta) (quad4) or (1, xi, eta)
//    (tri3).  With the monomial coefficients LM_i = sum_c T_s[c][i] Lambda_c,
//    YM_j = sum_l T_m[l][j] Y_l and XM_j = sum_b T_s[b][j] X_b (per pair),
//      f = Lh . q = [seg] m_s^T CX m_s - m_s^T CY m_m,
//      CY[i][j] = LM_i . YM_j,  CX[i][j] = LM_i . XM_j,
//    so a point needs v = CY m_m, u = CY^T m_s (and [seg] w = (CX + CX^T) m_s):
//      f = [seg] m_s^T w / 2 - m_s^T v,
//      W df/dxi_s = W (dm_s/dxi_s)^T (w - v),  W df/dxi_m = -W (dm_m/dxi_m)^T u;
//  * the terms that hold the shape functions fixed come from the forward
//    accumulators G = sum W N Nm^T and H = sum W N N^T (summed in the nodal
//    basis: non-negative terms keep small entries accurate) at the end:
//      dJ/dY_l |direct = -sum_c G[c][l] Lambda_c,  dJ/dX_b |direct = sum_c H[c][b] Lambda_c,
//      dJ/dLambda_c = sum_b H[c][b] X_b - sum_l G[c][l] Y_l,  J = sum_c Lambda_c . dJ/dLambda_c;
//  * element maps are inverted as in the batched integration kernel (affine
//    2x2 inverse, or FP32 Newton + one Newton step on the FP64 residual), and the
//    implicit-function step applies the FP64 inverse Jacobian at the
//    converged xi (MapInverse::jinvT);
//  * the clip is recorded as a compact vertex pool (ClipPool);
//  * a warp sorts its batch of pairs by the cell count and edge
//    intersections of an FP32 clip before the sweep.
template <int NS, int NM, bool SEG, bool DUAL, bool FWD>
__device__ void adjoint_pair_fast(int64_t p, const int32_t* __restrict__ ps, const int32_t* __restrict__ pm,
                                  const double* __restrict__ srec, const double* __restrict__ xs,
                                  const double* __restrict__ xm, const int32_t* __restrict__ conn_s,
                                  const int32_t* __restrict__ conn_m, const double* __restrict__ lambda,
                                  double* __restrict__ gs_out, double* __restrict__ gm_out,
                                  double* __restrict__ ab_out, double* __restrict__ J_out,
                                  const FwdOut& fo, AdjCounters& ctr, double* __restrict__ csh, int cstride) {
  constexpr int KS = NS, KM = NM;   // monomials per side (quad4: 4, tri3: 3)
  // CY (and [seg] SX) live in this thread's slice of shared memory, entry k
  // at csh[k * cstride] (interleaved across the block's threads: no bank
  // conflicts); they are read at every quadrature point and would otherwise
  // hold 32 (64) registers through the loop
  auto CYs = [&](int i, int j) -> double& { return csh[(4 * i + j) * cstride]; };
  auto SXs = [&](int i, int j) -> double& { return csh[(16 + 4 * i + j) * cstride]; };
  const int32_t s = ps[p], m = pm[p];
  const double* r = srec + (int64_t)SR_STRIDE * s;
  const int32_t* cs = conn_s + (int64_t)NS * s;
  const int32_t* cm = conn_m + (int64_t)NM * m;
  // Node coordinates and multipliers are read here for the set-up and read
  // again (from L1/L2) after the quadrature loop: keeping them in registers
  // across the loop would spill.
  auto load_nodes = [&](V3* X, V3* Y, V3* lam) {
    for (int a = 0; a < NS; ++a) {
      const int64_t n = cs[a];
      X[a] = v3(xs[3 * n], xs[3 * n + 1], xs[3 * n + 2]);
      lam[a] = v3(lambda[3 * n], lambda[3 * n + 1], lambda[3 * n + 2]);
    }
    for (int l = 0; l < NM; ++l) {
      const int64_t n = cm[l];
      Y[l] = v3(xm[3 * n], xm[3 * n + 1], xm[3 * n + 2]);
    }
  };
  auto lm_weights = [&](const V3* lam, V3* Lam) {   // Lambda_c = sum_a A[a][c] lambda_a (dual), lambda_c
    for (int c = 0; c < NS; ++c) {
      if (DUAL) {
        V3 acc = v3(0, 0, 0);
        for (int a = 0; a < NS; ++a) acc = acc + r[SR_A + 4 * a + c] * lam[a];
        Lam[c] = acc;
      } else {
        Lam[c] = lam[c];
      }
    }
  };
  const V3 x0 = v3(r[SR_X0], r[SR_X0 + 1], r[SR_X0 + 2]);
  const V3 t1 = v3(r[SR_T1], r[SR_T1 + 1], r[SR_T1 + 2]);
  const V3 t2 = v3(r[SR_T2], r[SR_T2 + 1], r[SR_T2 + 2]);
  double mu[4], mv[4];
  for (int l = 0; l < NM; ++l) {
    const int64_t n = cm[l];
    const double dx = xm[3 * n] - x0.x, dy = xm[3 * n + 1] - x0.y, dz = xm[3 * n + 2] - x0.z;
    mu[l] = dx * t1.x + dy * t1.y + dz * t1.z;
    mv[l] = dx * t2.x + dy * t2.y + dz * t2.z;
  }
  const PlaneMap mmap = plane_map<NM>(mu, mv);
  PlaneMap smap;
  smap.c0u = r[SR_C + 0]; smap.c0v = r[SR_C + 1]; smap.c1u = r[SR_C + 2]; smap.c1v = r[SR_C + 3];
  smap.c2u = r[SR_C + 4]; smap.c2v = r[SR_C + 5]; smap.c3u = r[SR_C + 6]; smap.c3v = r[SR_C + 7];
  double ma2 = 0.0;
  for (int l = 0; l < NM; ++l) ma2 += cross2(mu[l], mv[l], mu[(l + 1) % NM], mv[(l + 1) % NM]);
  const bool mrev = ma2 < 0.0;
  const bool srev = r[SR_REV] != 0.0;
  // ---- forward clip recorded as a vertex pool, and merge (same decisions as clip_polygon)
  ClipPool<NS, NM> cp;
  const bool nonempty = cp.run(r, mu, mv, mrev, ctr.clip_over);
  const int nr = cp.nr;
  double Jp = 0.0;
  V3 Lb[4];
  if (nonempty) {
    // monomial coefficients and the pair's bilinear forms
    {
      V3 X[4], Y[4], lam[4], Lam[4], LM[4], YM[4];
      load_nodes(X, Y, lam);
      lm_weights(lam, Lam);
      nodal_to_mono<NS>(Lam, LM);
      nodal_to_mono<NM>(Y, YM);
#pragma unroll
      for (int i = 0; i < KS; ++i)
#pragma unroll
        for (int j = 0; j < KM; ++j) CYs(i, j) = dot(LM[i], YM[j]);
      if (SEG) {
        V3 XM[4];
        nodal_to_mono<NS>(X, XM);
        double CX[4][4];
#pragma unroll
        for (int i = 0; i < KS; ++i)
#pragma unroll
          for (int j = 0; j < KS; ++j) CX[i][j] = dot(LM[i], XM[j]);
#pragma unroll
        for (int i = 0; i < KS; ++i)
#pragma unroll
          for (int j = 0; j < KS; ++j) SXs(i, j) = CX[i][j] + CX[j][i];
      }
    }
    MapInverse mi;
    mi.setup(mmap, NM == 3 || map_is_affine(mmap));
    MapInverse si;
    if (r[SR_AFF] != 0.0) {
      si.m = smap;
      si.affine = true;
      si.i00 = r[SR_BINV]; si.i01 = r[SR_BINV + 1]; si.i10 = r[SR_BINV + 2]; si.i11 = r[SR_BINV + 3];
    } else {
      si.setup(smap, false);
    }
    // polygon vertex adjoints, kept at the vertices' pool slots
    double Bu[ClipPool<NS, NM>::kSlots], Bv[ClipPool<NS, NM>::kSlots];
    for (int k = 0; k < cp.nv; ++k) { Bu[k] = 0.0; Bv[k] = 0.0; }
    double cu = 0.0, cv = 0.0, cbu = 0.0, cbv = 0.0;
    int ncell = 1;
    if (nr > 3) {
      double su = 0.0, sv = 0.0;
      for (int k = 0; k < nr; ++k) { su += cp.u(k); sv += cp.v(k); }
      cu = su * kInvCount[nr];
      cv = sv * kInvCount[nr];
      ncell = nr;
    }
    // forward accumulators G = sum W N_s N_m^T, H = sum W N_s N_s^T, summed
    // from the nodal shape functions: all terms are non-negative, so small
    // entries keep their relative accuracy (monomial moments would cancel)
    double G[4][4], H[4][4];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) { G[a][b] = 0.0; H[a][b] = 0.0; }
    double smb[8] = {0, 0, 0, 0, 0, 0, 0, 0}, mmb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int cI = 0; cI < ncell; ++cI) {
      int ib, iw;
      double au, av;
      if (nr == 3) {
        au = cp.u(0); av = cp.v(0); ib = 1; iw = 2;
      } else {
        au = cu; av = cv; ib = cI; iw = cI + 1 == nr ? 0 : cI + 1;
      }
      const int sb = cp.id(ib), sw = cp.id(iw);
      const double e1u = cp.pu[sb] - au, e1v = cp.pv[sb] - av, e2u = cp.pu[sw] - au, e2v = cp.pv[sw] - av;
      const double cr = cross2(e1u, e1v, e2u, e2v);
      const double area = 0.5 * fabs(cr);
      double area_b = 0.0, e1bu = 0.0, e1bv = 0.0, e2bu = 0.0, e2bv = 0.0, abu = 0.0, abv = 0.0;
      if (FWD) { ctr.cells++; ctr.gp += 7; }
#pragma unroll 1
      for (int q = 0; q < 7; ++q) {
        double l1, l2, w;
        tri7_point(q, l1, l2, w);
        const double xu = au + l1 * e1u + l2 * e2u;
        const double xv = av + l1 * e1v + l2 * e2v;
        const double W = w * area;
        double xs1, xs2, xm1, xm2;
        if (!si.solve(xu, xv, xs1, xs2)) ctr.newton_fail++;
        if (!mi.solve(xu, xv, xm1, xm2)) ctr.newton_fail++;
        const double xs12 = xs1 * xs2, xm12 = xm1 * xm2;
        // v = CY m_m (rows 1.. only: the derivative in xi_s needs no v_0),
        // u = CY^T m_s, and m_s^T CY m_m = u . m_m
        double v[4], u[4];
#pragma unroll
        for (int i = 1; i < KS; ++i) {
          double t = fma(CYs(i, 2), xm2, fma(CYs(i, 1), xm1, CYs(i, 0)));
          if (KM == 4) t = fma(CYs(i, 3), xm12, t);
          v[i] = t;
        }
#pragma unroll
        for (int j = 0; j < KM; ++j) {
          double t = fma(CYs(2, j), xs2, fma(CYs(1, j), xs1, CYs(0, j)));
          if (KS == 4) t = fma(CYs(3, j), xs12, t);
          u[j] = t;
        }
        // g = [seg] (CX + CX^T) m_s - v;  f = [seg] m_s^T w / 2 - m_s^T v
        double g[4], f;
        {
          double fv = fma(u[2], xm2, fma(u[1], xm1, u[0]));
          if (KM == 4) fv = fma(u[3], xm12, fv);
          if (SEG) {
            double fw = 0.0;
#pragma unroll
            for (int i = 0; i < KS; ++i) {
              double t = fma(SXs(i, 2), xs2, fma(SXs(i, 1), xs1, SXs(i, 0)));
              if (KS == 4) t = fma(SXs(i, 3), xs12, t);
              if (i > 0) g[i] = t - v[i];
              fw = i == 0 ? t : fma(i == 1 ? xs1 : (i == 2 ? xs2 : xs12), t, fw);
            }
            f = fma(0.5, fw, -fv);
          } else {
#pragma unroll
            for (int i = 1; i < KS; ++i) g[i] = -v[i];
            f = -fv;
          }
        }
        area_b = fma(w, f, area_b);
        // W df/dxi on both sides
        double xsb0, xsb1, xmb0, xmb1;
        if (KS == 4) {
          xsb0 = W * fma(xs2, g[3], g[1]);
          xsb1 = W * fma(xs1, g[3], g[2]);
        } else {
          xsb0 = W * g[1];
          xsb1 = W * g[2];
        }
        if (KM == 4) {
          xmb0 = -W * fma(xm2, u[3], u[1]);
          xmb1 = -W * fma(xm1, u[3], u[2]);
        } else {
          xmb0 = -W * u[1];
          xmb1 = -W * u[2];
        }
        // forward accumulators (nodal shape functions).  The factors 1/4 of
        // quad4 shape functions are folded into W: with ks, km = 1/4 for a
        // quad4 side (1 for tri3), WNs = (ks km W) N_s / ks and Nm = N_m / km,
        // so that WNs Nm = W N_s N_m
        {
          constexpr double km = NM == 4 ? 0.25 : 1.0;
          constexpr double kw = km * (NS == 4 ? 0.25 : 1.0);
          double WNs[4], Nm[4];
          const double wk = kw * W;
          if constexpr (NS == 4) {
            // products of (1 -+ xi)(1 -+ eta) as FMAs: q (1 -+ eta) = q -+ q eta
            const double qa = fma(-wk, xs1, wk), qb = fma(wk, xs1, wk);
            WNs[0] = fma(-qa, xs2, qa); WNs[1] = fma(-qb, xs2, qb); WNs[2] = fma(qb, xs2, qb);
            WNs[3] = fma(qa, xs2, qa);
          } else {
            WNs[1] = wk * xs1; WNs[2] = wk * xs2; WNs[0] = wk - WNs[1] - WNs[2]; WNs[3] = 0.0;
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
            for (int l = 0; l < NM; ++l) G[a][l] = fma(WNs[a], Nm[l], G[a][l]);
          if (SEG) {   // H = sum W N_s N_s^T = sum WNs (N_s / km)
            double Ns[4];
            if constexpr (NS == 4 && NM == 4) {
              const double a = 1.0 - xs1, b = 1.0 + xs1;
              Ns[0] = fma(-a, xs2, a); Ns[1] = fma(-b, xs2, b); Ns[2] = fma(b, xs2, b); Ns[3] = fma(a, xs2, a);
            } else {
              shape_fn<NS>(xs1, xs2, Ns);
              if (NM == 4)
                for (int b = 0; b < NS; ++b) Ns[b] *= 4.0;
            }
#pragma unroll
            for (int a = 0; a < NS; ++a)
#pragma unroll
              for (int b = 0; b < NS; ++b) H[a][b] = fma(WNs[a], Ns[b], H[a][b]);
          }
        }
        double msu, msv, mmu, mmv;   // J^-T xib on both sides
        si.jinvT(xs1, xs2, xsb0, xsb1, msu, msv);
        mi.jinvT(xm1, xm2, xmb0, xmb1, mmu, mmv);
        smb[0] -= msu; smb[1] -= msv;
        smb[2] = fma(-xs1, msu, smb[2]); smb[3] = fma(-xs1, msv, smb[3]);
        smb[4] = fma(-xs2, msu, smb[4]); smb[5] = fma(-xs2, msv, smb[5]);
        smb[6] = fma(-xs12, msu, smb[6]); smb[7] = fma(-xs12, msv, smb[7]);
        mmb[0] -= mmu; mmb[1] -= mmv;
        mmb[2] = fma(-xm1, mmu, mmb[2]); mmb[3] = fma(-xm1, mmv, mmb[3]);
        mmb[4] = fma(-xm2, mmu, mmb[4]); mmb[5] = fma(-xm2, mmv, mmb[5]);
        mmb[6] = fma(-xm12, mmu, mmb[6]); mmb[7] = fma(-xm12, mmv, mmb[7]);
        const double xbu = msu + mmu, xbv = msv + mmv;
        abu += xbu; abv += xbv;
        e1bu = fma(l1, xbu, e1bu); e1bv = fma(l1, xbv, e1bv);
        e2bu = fma(l2, xbu, e2bu); e2bv = fma(l2, xbv, e2bv);
      }
      const double crb = 0.5 * (cr < 0.0 ? -area_b : area_b);
      e1bu += crb * e2v; e1bv -= crb * e2u;
      e2bu -= crb * e1v; e2bv += crb * e1u;
      Bu[sb] += e1bu; Bv[sb] += e1bv;
      Bu[sw] += e2bu; Bv[sw] += e2bv;
      abu -= e1bu + e2bu;
      abv -= e1bv + e2bv;
      if (nr == 3) { const int s0 = cp.id(0); Bu[s0] += abu; Bv[s0] += abv; } else { cbu += abu; cbv += abv; }
    }
    if (nr > 3) {
      const double inv = kInvCount[nr];
      for (int k = 0; k < nr; ++k) { const int sk = cp.id(k); Bu[sk] += cbu * inv; Bv[sk] += cbv * inv; }
    }
    // Outputs go out with streaming (evict-first) stores: each is written once
    // and read by a later kernel, and L2 keeps the threads' stack lines instead.
    if (FWD) {   // fused forward: M = A G, D = A H of this pair
      ctr.nonempty++;
      double* mo = fo.Mblk + 16 * p;
      for (int a = 0; a < 4; ++a)
        for (int l = 0; l < 4; ++l) {
          double v = 0.0;
          if (a < NS && l < NM) {
            if (DUAL)
              for (int c = 0; c < NS; ++c) v += r[SR_A + 4 * a + c] * G[c][l];
            else
              v = G[a][l];
          }
          __stcs(mo + 4 * a + l, v);
        }
      if (SEG) {
        double* dout = fo.Dblk + 16 * p;
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) {
            double v = 0.0;
            if (a < NS && b < NS) {
              if (DUAL)
                for (int c = 0; c < NS; ++c) v += r[SR_A + 4 * a + c] * H[c][b];
              else
                v = H[a][b];
            }
            __stcs(dout + 4 * a + b, v);
          }
      }
      __stcs(fo.flag + p, (uint8_t)1);
    }
    // ---- reverse merge and clipping (vertex pool) and the element maps
    double sbu[4] = {0, 0, 0, 0}, sbv[4] = {0, 0, 0, 0}, mbu[4] = {0, 0, 0, 0}, mbv[4] = {0, 0, 0, 0};
    cp.reverse(r, Bu, Bv, srev, mrev, sbu, sbv, mbu, mbv);
    map_coeff_reverse<NS>(smb, sbu, sbv);
    map_coeff_reverse<NM>(mmb, mbu, mbv);
    // ---- direct terms and J from the forward accumulators, then the
    //      reverse of the projection onto the auxiliary plane
    V3 X[4], Y[4], lam[4], Lam[4];
    load_nodes(X, Y, lam);
    lm_weights(lam, Lam);
    double gX[4][3], gY[4][3];
    for (int a = 0; a < 4; ++a)
      for (int k = 0; k < 3; ++k) { gX[a][k] = 0.0; gY[a][k] = 0.0; }
    for (int c = 0; c < NS; ++c) {
      V3 acc = v3(0, 0, 0);
      if (SEG)
        for (int b = 0; b < NS; ++b) acc = acc + H[c][b] * X[b];
      for (int l = 0; l < NM; ++l) acc = acc - G[c][l] * Y[l];
      Lb[c] = acc;
      Jp += dot(Lam[c], acc);
    }
    for (int l = 0; l < NM; ++l) {
      V3 acc = v3(0, 0, 0);
      for (int c = 0; c < NS; ++c) acc = acc + G[c][l] * Lam[c];
      gY[l][0] -= acc.x; gY[l][1] -= acc.y; gY[l][2] -= acc.z;
    }
    if (SEG)
      for (int b = 0; b < NS; ++b) {
        V3 acc = v3(0, 0, 0);
        for (int c = 0; c < NS; ++c) acc = acc + H[c][b] * Lam[c];
        gX[b][0] += acc.x; gX[b][1] += acc.y; gX[b][2] += acc.z;
      }
    const V3 n0 = v3(r[SR_N0], r[SR_N0 + 1], r[SR_N0 + 2]);
    plane_reverse<NS, NM>(X, Y, x0, t1, t2, n0, sbu, sbv, mbu, mbv, gX, gY);
    double* go = gs_out + 12 * p;
    double* gmo = gm_out + 12 * p;
    for (int a = 0; a < 4; ++a)
      for (int k = 0; k < 3; ++k) {
        __stcs(go + 3 * a + k, gX[a][k]);
        __stcs(gmo + 3 * a + k, gY[a][k]);
      }
    if (DUAL) {
      double* ab = ab_out + 16 * p;
      for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 4; ++c) __stcs(ab + 4 * a + c, (a < NS && c < NS) ? dot(lam[a], Lb[c]) : 0.0);
    }
  } else {
    double2* g1 = reinterpret_cast<double2*>(gs_out + 12 * p);
    double2* g2 = reinterpret_cast<double2*>(gm_out + 12 * p);
    for (int k = 0; k < 6; ++k) { __stcs(g1 + k, make_double2(0.0, 0.0)); __stcs(g2 + k, make_double2(0.0, 0.0)); }
    if (DUAL) {
      double2* a2 = reinterpret_cast<double2*>(ab_out + 16 * p);
      for (int k = 0; k < 8; ++k) __stcs(a2 + k, make_double2(0.0, 0.0));
    }
    if (FWD) {
      double2* mo = reinterpret_cast<double2*>(fo.Mblk + 16 * p);
      for (int k = 0; k < 8; ++k) __stcs(mo + k, make_double2(0.0, 0.0));
      if (SEG) {
        double2* dd = reinterpret_cast<double2*>(fo.Dblk + 16 * p);
        for (int k = 0; k < 8; ++k) __stcs(dd + k, make_double2(0.0, 0.0));
      }
      __stcs(fo.flag + p, (uint8_t)0);
    }
  }
  __stcs(J_out + p, Jp);
}

// shared-memory coefficients per thread of the batched adjoint kernel: CY and [seg] SX
template <bool SEG>
constexpr int kAdjCoef = SEG ? 32 : 16;

template <int NS, int NM, bool SEG, bool DUAL, bool FWD, int R>
__global__ void __launch_bounds__(kMaxPairBlock) k_adjoint_batched(
    const int32_t* __restrict__ ps, const int32_t* __restrict__ pm, const double* __restrict__ srec,
    const double* __restrict__ xs, const double* __restrict__ xm, const int32_t* __restrict__ conn_s,
    const int32_t* __restrict__ conn_m, const double* __restrict__ lambda, int64_t pair_cap,
    double* __restrict__ gs_out, double* __restrict__ gm_out, double* __restrict__ ab_out,
    double* __restrict__ J_out, FwdOut fo, DevStatus* st, unsigned long long* cta_t, int32_t watchdog_us) {
  cta_mark(cta_t, 0);
  constexpr int B = 32 * R;
  using PermT = typename std::conditional<(B > 256), uint16_t, uint8_t>::type;
  __shared__ PermT perm_s[kMaxPairBlock / 32][B];
  __shared__ uint8_t key_s[kMaxPairBlock / 32][B];
  __shared__ unsigned pres_s[kMaxPairBlock / 32][8];   // key values present in the batch (256 bits)
  extern __shared__ double adj_coef[];   // kAdjCoef doubles per thread, interleaved
  PermT* perm = perm_s[threadIdx.x >> 5];
  uint8_t* keys = key_s[threadIdx.x >> 5];
  unsigned* pres = pres_s[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  AdjCounters ctr;
  const bool ok = st->over_pairs == 0 && st->over_bins == 0;
  const int64_t n = ok ? (int64_t)min((unsigned long long)pair_cap, st->n_pairs) : 0;
  // guided self-scheduling: a warp takes half an even share of the pairs
  // left (at most B, at least 32, a multiple of 32), so batches are full
  // while there is plenty of work and shrink towards the end of the queue
  const int64_t share = 2 * (int64_t)gridDim.x * (blockDim.x >> 5);
  const Watchdog wd(watchdog_us);
  for (;;) {   // bounded: the shared counter only grows
    if (wd.expired(&st->timeout)) break;
    int64_t base = 0;
    int fetch = B;
    if (lane == 0) {
      const unsigned long long seen = *reinterpret_cast<volatile unsigned long long*>(&st->work_ctr2);
      const int64_t f = (n - (int64_t)seen) / share;
      fetch = f >= B ? B : (f < 32 ? 32 : (int)(f & ~31ll));
      base = (int64_t)atomicAdd(&st->work_ctr2, (unsigned long long)fetch);
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    fetch = __shfl_sync(0xffffffffu, fetch, 0);
    if (base >= n) break;
    const int64_t lim = min(n, base + (int64_t)fetch);
    const int rounds = (fetch + 31) >> 5;
    // phase A: sort key of each pair from an FP32 clip: 1 + 16 x its cell
    // count + its edge intersections (cells 0 = empty in FP32; key 0 = no
    // pair).  The cell count sets the quadrature work, the intersections the
    // divergent clip and reverse-clip work.  Every pair goes through phase B,
    // where the FP64 clip decides what it contributes.
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
    // counting sort of the batch by key, descending, over the key values
    // present (ballots per value)
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
    // phase B: full adjoint of each pair, rounds of similar cost
    for (int i0 = 0; i0 < n_live; i0 += 32) {
      const int i = i0 + lane;
      if (i < n_live)
        adjoint_pair_fast<NS, NM, SEG, DUAL, FWD>(base + perm[i], ps, pm, srec, xs, xm, conn_s, conn_m, lambda,
                                                  gs_out, gm_out, ab_out, J_out, fo, ctr, adj_coef + threadIdx.x,
                                                  (int)blockDim.x);
    }
    __syncwarp();
  }
  block_count_add(&st->clip_overflow, ctr.clip_over);
  block_count_add(&st->newton_fail, ctr.newton_fail);
  if (FWD) {
    block_count_add(&st->nonempty, ctr.nonempty);
    block_count_add(&st->cells, ctr.cells);
    block_count_add(&st->gauss_points, ctr.gp);
  }
  __syncthreads();
  cta_mark(cta_t, 1);
}

// Constant tables of a flat element with dual LMs.  There Dh_a = d for every
// a, Me = d Mref and A is the constant matrix ac (quad4: 4 on the diagonal,
// -2 for edge neighbours, 1 across; tri3: 3 and -1), so the adjoint of the
// element integrals through A = Dh Me^-1 is Meb = -(1/d) ac Ab ac.  The flat
// reverse below needs Meb only through weighted sums sum_ab w_ab Meb_ab, which
// equal -(1/d) sum_cd Ab_cd (ac w ac)_cd: w[k] holds ac w_k ac for the weights
// of the closed-form reference integrals (quad4: the three of S1 / S2; tri3:
// int N_a N_b).
struct FlatDualTables {
  double ac[4][4];
  double w[3][4][4];
};

template <int NS>
constexpr FlatDualTables flat_dual_tables() {
  FlatDualTables t{};
  const double cx[4] = {-1.0, 1.0, 1.0, -1.0}, cy[4] = {-1.0, -1.0, 1.0, 1.0};
  double wk[3][4][4] = {};
  for (int a = 0; a < NS; ++a)
    for (int b = 0; b < NS; ++b) {
      if (NS == 4) {
        const int dd = (a - b + 4) % 4;
        t.ac[a][b] = dd == 0 ? 4.0 : (dd == 2 ? 1.0 : -2.0);
        const double px = 2.0 + (2.0 / 3.0) * cx[a] * cx[b], py = 2.0 + (2.0 / 3.0) * cy[a] * cy[b];
        wk[0][a][b] = px * py;
        wk[1][a][b] = px * (cy[a] + cy[b]);
        wk[2][a][b] = py * (cx[a] + cx[b]);
      } else {
        t.ac[a][b] = a == b ? 3.0 : -1.0;
        wk[0][a][b] = a == b ? 1.0 / 12.0 : 1.0 / 24.0;
      }
    }
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < NS; ++c)
      for (int d = 0; d < NS; ++d) {
        double v = 0.0;
        for (int a = 0; a < NS; ++a)
          for (int b = 0; b < NS; ++b) v += t.ac[a][c] * wk[k][a][b] * t.ac[d][b];
        t.w[k][c][d] = v;
      }
  return t;
}

// The tables' ac is the dual matrix of the reference element: ac Mref = dref I
// (quad4: Mref = (4, 2, 1) / 9 by node distance, dref = 1; tri3: Mref = 1/12 on
// the diagonal, 1/24 off it, dref = 1/6).
template <int NS>
constexpr bool flat_dual_biorthogonal() {
  const FlatDualTables t = flat_dual_tables<NS>();
  for (int a = 0; a < NS; ++a)
    for (int c = 0; c < NS; ++c) {
      double v = 0.0;
      for (int b = 0; b < NS; ++b) {
        const int dd = (b - c + NS) % NS;
        const double mref = NS == 4 ? (dd == 0 ? 4.0 / 9.0 : (dd == 2 ? 1.0 / 9.0 : 2.0 / 9.0))
                                    : (dd == 0 ? 1.0 / 12.0 : 1.0 / 24.0);
        v += t.ac[a][b] * mref;
      }
      const double want = a == c ? (NS == 4 ? 1.0 : 1.0 / 6.0) : 0.0;
      const double err = v - want;
      if (err > 1e-14 || err < -1e-14) return false;
    }
  return true;
}
static_assert(flat_dual_biorthogonal<4>() && flat_dual_biorthogonal<3>(),
              "flat-element dual coefficients are not the reference element's dual matrix");

// Per slave element: sum dJ/dA over its pairs, add the element-domain D term,
// propagate through A = Dh Me^-1 and the element integrals to the nodes.
template <int NS, bool DUAL, bool ELEMD>
__global__ void __launch_bounds__(kThreads) k_adjoint_elems(
    const double* __restrict__ xs, const int32_t* __restrict__ conn_s, const double* __restrict__ lambda,
    const double* __restrict__ srec, const double* __restrict__ De, const int64_t* __restrict__ pair_off,
    const double* __restrict__ ab_pair, int64_t Es, double* __restrict__ ge, const DevStatus* st) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Es) return;
  double* out = ge + 16 * e;
  for (int k = 0; k < 16; ++k) out[k] = 0.0;
  const double* r = srec + (int64_t)SR_STRIDE * e;
  if (r[SR_EPSIN] < 0.0 || st->over_pairs) return;
  V3 X[4], lam[4];
  for (int a = 0; a < NS; ++a) {
    const int64_t n = conn_s[(int64_t)NS * e + a];
    X[a] = v3(xs[3 * n], xs[3 * n + 1], xs[3 * n + 2]);
    lam[a] = v3(lambda[3 * n], lambda[3 * n + 1], lambda[3 * n + 2]);
  }
  double A[4][4], Ab[4][4], Meb[4][4], Dhb[4];
  for (int a = 0; a < 4; ++a) {
    Dhb[a] = 0.0;
    for (int b = 0; b < 4; ++b) { A[a][b] = r[SR_A + 4 * a + b]; Ab[a][b] = 0.0; Meb[a][b] = 0.0; }
  }
  if (DUAL) {
    const int64_t p0 = pair_off[e], p1 = pair_off[e + 1];
    for (int64_t p = p0; p < p1; ++p)
      for (int a = 0; a < NS; ++a)
        for (int b = 0; b < NS; ++b) Ab[a][b] += ab_pair[16 * p + 4 * a + b];
  }
  V3 Xb[4];
  for (int a = 0; a < 4; ++a) Xb[a] = v3(0, 0, 0);
  double Je = 0.0;
  constexpr int nq = NS == 4 ? 9 : 7;
  // element integrals Me, Dh (recomputed).  A flat element (negligible
  // bilinear term: parallelograms, every tri3) has constant tangents g1, g2
  // and Jacobian J0, so Me = J0 Mref and Dh = J0 dref, and in the reverse
  // sweep below the Jacobian's gradient directions are the same at every
  // quadrature point.
  double Me[4][4], Dh[4];
  for (int a = 0; a < 4; ++a) {
    Dh[a] = 0.0;
    for (int b = 0; b < 4; ++b) Me[a][b] = 0.0;
  }
  V3 g1c, g2c;
  bool flat;
  if constexpr (NS == 4) {
    g1c = 0.25 * ((X[1] - X[0]) + (X[2] - X[3]));
    g2c = 0.25 * ((X[2] - X[1]) + (X[3] - X[0]));
    const V3 d3 = 0.25 * ((X[0] - X[1]) + (X[2] - X[3]));
    const double s3 = fabs(d3.x) + fabs(d3.y) + fabs(d3.z);
    const double s12 = fabs(g1c.x) + fabs(g1c.y) + fabs(g1c.z) + fabs(g2c.x) + fabs(g2c.y) + fabs(g2c.z);
    flat = s3 <= 1e-15 * s12;
  } else {
    g1c = X[1] - X[0];
    g2c = X[2] - X[0];
    flat = true;
  }
  const V3 nc = cross(g1c, g2c);
  const double J0 = sqrt(dot(nc, nc));
  if (flat) {
    if constexpr (NS == 4) {
      const double m4 = J0 * (4.0 / 9.0), m2 = J0 * (2.0 / 9.0), m1 = J0 * (1.0 / 9.0);
      for (int a = 0; a < 4; ++a) {
        Dh[a] = J0;
        for (int b = 0; b < 4; ++b) {
          const int dd = (a - b + 4) % 4;
          Me[a][b] = dd == 0 ? m4 : (dd == 2 ? m1 : m2);
        }
      }
    } else {
      for (int a = 0; a < 3; ++a) {
        Dh[a] = J0 * (1.0 / 6.0);
        for (int b = 0; b < 3; ++b) Me[a][b] = J0 * (a == b ? 1.0 / 12.0 : 1.0 / 24.0);
      }
    }
  }
  for (int q = 0; q < nq && !flat; ++q) {
    double xi, eta, w;
    elem_point_a<NS>(q, xi, eta, w);
    double N[4], dN[4][2];
    shape_fn<NS>(xi, eta, N);
    shape_grad<NS>(xi, eta, dN);
    V3 g1 = v3(0, 0, 0), g2 = v3(0, 0, 0);
    for (int a = 0; a < NS; ++a) { g1 = g1 + dN[a][0] * X[a]; g2 = g2 + dN[a][1] * X[a]; }
    const V3 nq3 = cross(g1, g2);
    const double wj = w * sqrt(dot(nq3, nq3));
    for (int a = 0; a < NS; ++a) {
      Dh[a] += wj * N[a];
      for (int b = 0; b < NS; ++b) Me[a][b] += wj * N[a] * N[b];
    }
  }
  if (ELEMD && DUAL) {
    // dual LMs: De = A Me = diag(Dh) exactly, J_e = sum_a Dh_a (lam_a . X_a)
    for (int a = 0; a < NS; ++a) {
      const double dla = dot(lam[a], X[a]);
      const double dab = De[16 * e + 5 * a];
      Je += dab * dla;
      Xb[a] = Xb[a] + dab * lam[a];
      Dhb[a] += dla;
    }
  } else if (ELEMD) {
    // J_e = sum_ab (lam_a . X_b) De_ab with De = A Me
    for (int a = 0; a < NS; ++a)
      for (int b = 0; b < NS; ++b) {
        const double dab = De[16 * e + 4 * a + b];
        Je += dab * dot(lam[a], X[b]);
        Xb[b] = Xb[b] + dab * lam[a];
        const double deb = dot(lam[a], X[b]);
        for (int c = 0; c < NS; ++c) {
          Ab[a][c] += deb * Me[c][b];
          Meb[c][b] += A[a][c] * deb;
        }
      }
  }
  constexpr FlatDualTables kFD = flat_dual_tables<NS>();
  const bool flat_dual = DUAL && flat;
  const double inv_d = flat_dual ? 1.0 / Dh[0] : 0.0;
  if (flat_dual) {
    // Dhb_a += sum_b Ab_ab K_ab with K = ac / d; Meb enters below as weighted sums
#pragma unroll
    for (int a = 0; a < NS; ++a) {
      double t = 0.0;
#pragma unroll
      for (int b = 0; b < NS; ++b) t = fma(kFD.ac[a][b], Ab[a][b], t);
      Dhb[a] = fma(t, inv_d, Dhb[a]);
    }
  } else if (DUAL) {
    // A = Dh K, K = Me^-1 = Dh^-1 A
    double K[4][4], Kb[4][4];
    for (int a = 0; a < NS; ++a) {
      const double inv = 1.0 / Dh[a];   // one division per row
      for (int b = 0; b < NS; ++b) {
        K[a][b] = A[a][b] * inv;
        Kb[a][b] = Dh[a] * Ab[a][b];
      }
    }
    for (int a = 0; a < NS; ++a) {
      double s = 0.0;
      for (int b = 0; b < NS; ++b) s += Ab[a][b] * K[a][b];
      Dhb[a] += s;
    }
    // Meb -= K Kb K
    double T[4][4];
    for (int a = 0; a < NS; ++a)
      for (int b = 0; b < NS; ++b) {
        double s = 0.0;
        for (int c = 0; c < NS; ++c) s += K[a][c] * Kb[c][b];
        T[a][b] = s;
      }
    for (int a = 0; a < NS; ++a)
      for (int b = 0; b < NS; ++b) {
        double s = 0.0;
        for (int c = 0; c < NS; ++c) s += T[a][c] * K[c][b];
        Meb[a][b] -= s;
      }
  }
  // element integrals -> nodes.  The adjoint of the surface Jacobian at a
  // point is jb = sum_ab (Dhb_a + Meb_ab N_b) N_a; a flat element only needs
  // S1_c = int jb dN_c/dxi and S2_c = int jb dN_c/deta over the reference
  // element, which are exact polynomial integrals:
  //   quad4 (corners (xi_a, eta_a) = (-1,-1), (1,-1), (1,1), (-1,1)):
  //     int N_a dN_c/dxi         = xi_c / 4 (1 + eta_a eta_c / 3)
  //     int N_a N_b dN_c/dxi     = xi_c / 64 (2 + 2/3 xi_a xi_b)(2 + 2/3 (eta_a eta_b + eta_c (eta_a + eta_b)))
  //   (and the same with xi and eta exchanged for dN_c/deta);
  //   tri3: dN_c constant, int N_a = 1/6, int N_a N_b = 1/12 (a = b) or 1/24.
  double S1[4] = {0, 0, 0, 0}, S2[4] = {0, 0, 0, 0};
  if (flat) {
    if constexpr (NS == 4) {
      constexpr double cx[4] = {-1.0, 1.0, 1.0, -1.0}, cy[4] = {-1.0, -1.0, 1.0, 1.0};
      double A0 = 0.0, A1 = 0.0, C1 = 0.0, B0 = 0.0, Bx = 0.0, By = 0.0;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        B0 += Dhb[a];
        Bx = fma(cx[a], Dhb[a], Bx);
        By = fma(cy[a], Dhb[a], By);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if (flat_dual) {
            A0 = fma(kFD.w[0][a][b], Ab[a][b], A0);
            A1 = fma(kFD.w[1][a][b], Ab[a][b], A1);
            C1 = fma(kFD.w[2][a][b], Ab[a][b], C1);
          } else {
            const double px = 2.0 + (2.0 / 3.0) * cx[a] * cx[b], py = 2.0 + (2.0 / 3.0) * cy[a] * cy[b];
            A0 = fma(px * py, Meb[a][b], A0);
            A1 = fma(px * (cy[a] + cy[b]), Meb[a][b], A1);
            C1 = fma(py * (cx[a] + cx[b]), Meb[a][b], C1);
          }
        }
      }
      if (flat_dual) { A0 *= -inv_d; A1 *= -inv_d; C1 *= -inv_d; }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        S1[c] = cx[c] * fma(1.0 / 64.0, fma((2.0 / 3.0) * cy[c], A1, A0), 0.25 * fma(cy[c] / 3.0, By, B0));
        S2[c] = cy[c] * fma(1.0 / 64.0, fma((2.0 / 3.0) * cx[c], C1, A0), 0.25 * fma(cx[c] / 3.0, Bx, B0));
      }
    } else {
      double T = 0.0, Tm = 0.0;
      for (int a = 0; a < 3; ++a) {
        T = fma(1.0 / 6.0, Dhb[a], T);
        for (int b = 0; b < 3; ++b)
          Tm = flat_dual ? fma(kFD.w[0][a][b], Ab[a][b], Tm) : fma(a == b ? 1.0 / 12.0 : 1.0 / 24.0, Meb[a][b], Tm);
      }
      T = flat_dual ? fma(-inv_d, Tm, T) : T + Tm;
      S1[0] = -T; S1[1] = T; S1[2] = 0.0;
      S2[0] = -T; S2[1] = 0.0; S2[2] = T;
    }
  }
  for (int q = 0; q < nq && !flat; ++q) {
    double xi, eta, w;
    elem_point_a<NS>(q, xi, eta, w);
    double N[4], dN[4][2];
    shape_fn<NS>(xi, eta, N);
    shape_grad<NS>(xi, eta, dN);
    double jb = 0.0;
    for (int a = 0; a < NS; ++a) {
      double v = Dhb[a];
      for (int b = 0; b < NS; ++b) v = fma(Meb[a][b], N[b], v);
      jb = fma(v, N[a], jb);
    }
    jb *= w;
    if (jb == 0.0) continue;
    V3 g1 = v3(0, 0, 0), g2 = v3(0, 0, 0);
    for (int a = 0; a < NS; ++a) { g1 = g1 + dN[a][0] * X[a]; g2 = g2 + dN[a][1] * X[a]; }
    const V3 nq3 = cross(g1, g2);
    const double J = sqrt(dot(nq3, nq3));
    const V3 nb = (jb / J) * nq3;
    const V3 g1b = cross(g2, nb), g2b = cross(nb, g1);
    for (int a = 0; a < NS; ++a) Xb[a] = Xb[a] + dN[a][0] * g1b + dN[a][1] * g2b;
  }
  if (flat && J0 > 0.0) {   // d J / d g1 = g2 x n / J, d J / d g2 = n / J x g1 (same at every point)
    const V3 nu = (1.0 / J0) * nc;
    const V3 d1 = cross(g2c, nu), d2 = cross(nu, g1c);
    for (int a = 0; a < NS; ++a) Xb[a] = Xb[a] + S1[a] * d1 + S2[a] * d2;
  }
  for (int a = 0; a < NS; ++a) {
    out[3 * a] = Xb[a].x;
    out[3 * a + 1] = Xb[a].y;
    out[3 * a + 2] = Xb[a].z;
  }
  out[12] = Je;
}

#ifndef MORTAR_PAIR_NS
// master element -> pairs (non-empty ones), counting sort + per-element sort
__global__ void k_mp_count(const int32_t* __restrict__ pm, const uint8_t* __restrict__ flag, int64_t pair_cap,
                           int32_t* __restrict__ cnt, const DevStatus* st) {
  const int64_t n = st->over_pairs ? 0 : (int64_t)min((unsigned long long)pair_cap, st->n_pairs);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    if (flag[p]) atomicAdd(&cnt[pm[p]], 1);
}

__global__ void k_mp_fill(const int32_t* __restrict__ pm, const uint8_t* __restrict__ flag, int64_t pair_cap,
                          const int64_t* __restrict__ off, int32_t* __restrict__ cnt, int32_t* __restrict__ list,
                          const DevStatus* st) {
  const int64_t n = st->over_pairs ? 0 : (int64_t)min((unsigned long long)pair_cap, st->n_pairs);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    if (flag[p]) {
      const int32_t m = pm[p];
      const int32_t slot = atomicSub(&cnt[m], 1) - 1;
      list[off[m] + slot] = (int32_t)p;
    }
}

__global__ void k_mp_sort(const int64_t* __restrict__ off, int64_t Em, int32_t* __restrict__ list) {
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= Em) return;
  const int64_t b0 = off[f], b1 = off[f + 1];
  for (int64_t a = b0 + 1; a < b1; ++a) {
    const int32_t v = list[a];
    int64_t b = a - 1;
    while (b >= b0 && list[b] > v) { list[b + 1] = list[b]; --b; }
    list[b + 1] = v;
  }
}

__global__ void k_grad_slave(const int64_t* __restrict__ n2e_ptr, const int64_t* __restrict__ n2e_ent,
                             const int64_t* __restrict__ pair_off, const uint8_t* __restrict__ flag,
                             const double* __restrict__ gs_pair, const double* __restrict__ ge, int64_t Ns,
                             double* __restrict__ grad, const DevStatus* st) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Ns) return;
  double g0 = 0.0, g1 = 0.0, g2 = 0.0;
  if (!st->over_pairs)
    for (int64_t q = n2e_ptr[j]; q < n2e_ptr[j + 1]; ++q) {
      const int64_t e = n2e_ent[q] >> 2;
      const int a = (int)(n2e_ent[q] & 3);
      g0 += ge[16 * e + 3 * a]; g1 += ge[16 * e + 3 * a + 1]; g2 += ge[16 * e + 3 * a + 2];
      for (int64_t p = pair_off[e]; p < pair_off[e + 1]; ++p) {
        if (!flag[p]) continue;
        g0 += gs_pair[12 * p + 3 * a]; g1 += gs_pair[12 * p + 3 * a + 1]; g2 += gs_pair[12 * p + 3 * a + 2];
      }
    }
  grad[3 * j] = g0;
  grad[3 * j + 1] = g1;
  grad[3 * j + 2] = g2;
}

__global__ void k_grad_master(const int64_t* __restrict__ n2e_ptr, const int64_t* __restrict__ n2e_ent,
                              const int64_t* __restrict__ mp_off, const int32_t* __restrict__ mp_list,
                              const double* __restrict__ gm_pair, int64_t Nm, double* __restrict__ grad,
                              const DevStatus* st) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Nm) return;
  double g0 = 0.0, g1 = 0.0, g2 = 0.0;
  if (!st->over_pairs)
    for (int64_t q = n2e_ptr[j]; q < n2e_ptr[j + 1]; ++q) {
      const int64_t f = n2e_ent[q] >> 2;
      const int l = (int)(n2e_ent[q] & 3);
      for (int64_t k = mp_off[f]; k < mp_off[f + 1]; ++k) {
        const int64_t p = mp_list[k];
        g0 += gm_pair[12 * p + 3 * l]; g1 += gm_pair[12 * p + 3 * l + 1]; g2 += gm_pair[12 * p + 3 * l + 2];
      }
    }
  grad[3 * j] = g0;
  grad[3 * j + 1] = g1;
  grad[3 * j + 2] = g2;
}

constexpr int kJBlocks = 256;

// Fixed-shape reduction of J over pairs and elements (deterministic).
__global__ void __launch_bounds__(256) k_J_partial(const double* __restrict__ J_pair, int64_t pair_cap,
                                                   const double* __restrict__ ge, int64_t Es,
                                                   double* __restrict__ part, const DevStatus* st) {
  const int64_t np = st->over_pairs ? 0 : (int64_t)min((unsigned long long)pair_cap, st->n_pairs);
  const int64_t total = np + Es;
  const int64_t per = (total + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = per * blockIdx.x, b1 = min(total, b0 + per);
  double s = 0.0;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) s += i < np ? J_pair[i] : ge[16 * (i - np) + 12];
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(256) k_J_final(const double* __restrict__ part, DevStatus* st) {
  __shared__ double sh[256];
  sh[threadIdx.x] = part[threadIdx.x];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) st->J = sh[0];
}
#endif  // !MORTAR_PAIR_NS

#ifdef MORTAR_PAIR_NS
template <int NS, int NM, bool SEG, bool DUAL>
void launch_pairs_t(mortar_ctx* c, const RunParams& rp, unsigned grid, unsigned block, int32_t chunk) {
  if (grid == 0) {   // persistent grid: every SM filled to the kernel's occupancy
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adjoint_pairs<NS, NM, SEG, DUAL>, (int)block, 0);
    grid = (unsigned)(c->n_sm * (per_sm < 1 ? 1 : per_sm));
  }
  k_adjoint_pairs<NS, NM, SEG, DUAL><<<grid, block, 0, c->stream>>>(
      c->pairs_s.as<int32_t>(), c->pairs_m.as<int32_t>(), c->srec.as<double>(), c->xs.as<double>(),
      c->xm.as<double>(), c->conn_s.as<int32_t>(), c->conn_m.as<int32_t>(), c->lambda.as<double>(), rp, c->pair_cap,
      chunk, c->gs_pair.as<double>(), c->gm_pair.as<double>(), c->abar_pair.as<double>(), c->J_pair.as<double>(),
      c->dstat.as<DevStatus>());
}

template <int NS, int NM, bool SEG, bool DUAL, bool FWD>
void launch_batched_f(mortar_ctx* c, int rounds) {
  const FwdOut fo{c->Mblk.as<double>(), c->Dblk.as<double>(), c->flag.as<uint8_t>()};
  unsigned long long* cta_t = (FWD && c->timing && c->cta_t.p) ? c->cta_t.as<unsigned long long>() : nullptr;
  const int block = c->block_size > 0 ? c->block_size : 128;
  const size_t shm = (size_t)block * kAdjCoef<SEG> * sizeof(double);
  auto go = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);   // > 48 KB at 256 threads
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, shm);
    if (per_sm < 1) per_sm = 1;
    const unsigned grid = (unsigned)(c->n_sm * per_sm);
    if (cta_t) c->pair_grid = (int)grid;
    kern<<<grid, block, shm, c->stream>>>(
        c->pairs_s.as<int32_t>(), c->pairs_m.as<int32_t>(), c->srec.as<double>(), c->xs.as<double>(),
        c->xm.as<double>(), c->conn_s.as<int32_t>(), c->conn_m.as<int32_t>(), c->lambda.as<double>(), c->pair_cap,
        c->gs_pair.as<double>(), c->gm_pair.as<double>(), c->abar_pair.as<double>(), c->J_pair.as<double>(), fo,
        c->dstat.as<DevStatus>(), cta_t, c->watchdog_us);
  };
  if (rounds <= 1) go(k_adjoint_batched<NS, NM, SEG, DUAL, FWD, 1>);
  else if (rounds == 2) go(k_adjoint_batched<NS, NM, SEG, DUAL, FWD, 2>);
  else if (rounds == 4) go(k_adjoint_batched<NS, NM, SEG, DUAL, FWD, 4>);
  else if (rounds == 8) go(k_adjoint_batched<NS, NM, SEG, DUAL, FWD, 8>);
  else if (rounds == 16) go(k_adjoint_batched<NS, NM, SEG, DUAL, FWD, 16>);
  else go(k_adjoint_batched<NS, NM, SEG, DUAL, FWD, 32>);
}

// The warp-batched adjoint always produces the forward blocks as well (the
// run pipeline fuses the two whenever the batched schedule is selected); a
// non-fused call only rewrites the same blocks.
template <int NS, int NM, bool SEG, bool DUAL>
void launch_batched_t(mortar_ctx* c, int rounds, bool) {
  launch_batched_f<NS, NM, SEG, DUAL, true>(c, rounds);
}

}  // namespace

template <int NS, int NM>
void adjoint_pairs_nsnm(mortar_ctx* c, const RunParams& rp, unsigned grid, unsigned block, int32_t chunk,
                        bool fused) {
  const bool seg = rp.d_domain == 1, dual = rp.lm == 1;
  if (c->variant == 1) {
    if (seg && dual) launch_pairs_t<NS, NM, true, true>(c, rp, grid, block, chunk);
    else if (seg) launch_pairs_t<NS, NM, true, false>(c, rp, grid, block, chunk);
    else if (dual) launch_pairs_t<NS, NM, false, true>(c, rp, grid, block, chunk);
    else launch_pairs_t<NS, NM, false, false>(c, rp, grid, block, chunk);
    return;
  }
  const int rounds = c->rounds > 0 ? c->rounds : 2;
  if (seg && dual) launch_batched_t<NS, NM, true, true>(c, rounds, fused);
  else if (seg) launch_batched_t<NS, NM, true, false>(c, rounds, fused);
  else if (dual) launch_batched_t<NS, NM, false, true>(c, rounds, fused);
  else launch_batched_t<NS, NM, false, false>(c, rounds, fused);
}
template void adjoint_pairs_nsnm<MORTAR_PAIR_NS, MORTAR_PAIR_NM>(mortar_ctx*, const RunParams&, unsigned, unsigned,
                                                                  int32_t, bool);
#else   // the main part: element adjoint, gathers, J, dispatch

template <int NS>
void launch_elems_ns(mortar_ctx* c, const RunParams& rp) {
  const unsigned g = (unsigned)((c->Es + kThreads - 1) / kThreads);
  if (c->Es == 0) return;
  const bool elemd = rp.d_domain == 0, dual = rp.lm == 1;
  auto args = [&](auto kern) {
    kern<<<g, kThreads, 0, c->stream>>>(c->xs.as<double>(), c->conn_s.as<int32_t>(), c->lambda.as<double>(),
                                        c->srec.as<double>(), c->De.as<double>(), c->pair_off.as<int64_t>(),
                                        c->abar_pair.as<double>(), c->Es, c->ge_elem.as<double>(),
                                        c->dstat.as<DevStatus>());
  };
  if (dual && elemd) args(k_adjoint_elems<NS, true, true>);
  else if (dual) args(k_adjoint_elems<NS, true, false>);
  else if (elemd) args(k_adjoint_elems<NS, false, true>);
  else args(k_adjoint_elems<NS, false, false>);
}

}  // namespace

int prepare_adjoint_buffers(mortar_ctx* c) {
  const size_t P = (size_t)std::max<int64_t>(c->pair_cap, 1);
  int r;
  if ((r = buf_reserve(c->gs_pair, P * 12 * 8)) != MORTAR_OK) return r;
  if ((r = buf_reserve(c->gm_pair, P * 12 * 8)) != MORTAR_OK) return r;
  if ((r = buf_reserve(c->J_pair, P * 8)) != MORTAR_OK) return r;
  if (c->opt.lm == MORTAR_LM_DUAL && (r = buf_reserve(c->abar_pair, P * 16 * 8)) != MORTAR_OK) return r;
  if ((r = buf_reserve(c->mp_list, P * 4)) != MORTAR_OK) return r;
  const size_t Es = (size_t)std::max<int64_t>(c->Es, 1), Em = (size_t)std::max<int64_t>(c->Em, 1);
  if ((r = buf_reserve(c->ge_elem, Es * 16 * 8)) != MORTAR_OK) return r;
  if ((r = buf_reserve(c->mp_cnt, Em * 4)) != MORTAR_OK) return r;
  if ((r = buf_reserve(c->mp_off, (Em + 1) * 8)) != MORTAR_OK) return r;
  if ((r = buf_reserve(c->grad_s, (size_t)std::max<int64_t>(c->Ns, 1) * 24)) != MORTAR_OK) return r;
  if ((r = buf_reserve(c->grad_m, (size_t)std::max<int64_t>(c->Nm, 1) * 24)) != MORTAR_OK) return r;
  if ((r = buf_reserve(c->J_part, kJBlocks * 8)) != MORTAR_OK) return r;
  if ((r = buf_reserve(c->lambda, (size_t)std::max<int64_t>(c->Ns, 1) * 24)) != MORTAR_OK) return r;
  return MORTAR_OK;
}

bool adjoint_fuses_forward(const mortar_ctx* c) { return c->variant == 0; }

void launch_adjoint_pairs(mortar_ctx* c, const RunParams& rp, bool fused) {
  const unsigned block = c->block_size > 0 ? (unsigned)c->block_size : 128u;
  const int32_t chunk = c->chunk_pairs > 0 ? c->chunk_pairs : 32;
  const unsigned grid = 0;   // the one-pair-per-thread kernels size their own grid
  if (c->nen_s == 4 && c->nen_m == 4) adjoint_pairs_nsnm<4, 4>(c, rp, grid, block, chunk, fused);
  else if (c->nen_s == 4 && c->nen_m == 3) adjoint_pairs_nsnm<4, 3>(c, rp, grid, block, chunk, fused);
  else if (c->nen_s == 3 && c->nen_m == 4) adjoint_pairs_nsnm<3, 4>(c, rp, grid, block, chunk, fused);
  else adjoint_pairs_nsnm<3, 3>(c, rp, grid, block, chunk, fused);
}

void launch_adjoint_rest(mortar_ctx* c, const RunParams& rp) {
  DevStatus* st = c->dstat.as<DevStatus>();
  if (c->nen_s == 4) launch_elems_ns<4>(c, rp); else launch_elems_ns<3>(c, rp);
  // master element -> pair lists
  cudaMemsetAsync(c->mp_cnt.p, 0, (size_t)std::max<int64_t>(c->Em, 1) * 4, c->stream);
  const unsigned pg = (unsigned)(c->n_sm * 8);
  k_mp_count<<<pg, 256, 0, c->stream>>>(c->pairs_m.as<int32_t>(), c->flag.as<uint8_t>(), c->pair_cap,
                                        c->mp_cnt.as<int32_t>(), st);
  launch_exclusive_scan_i32(c->mp_cnt.as<int32_t>(), c->mp_off.as<int64_t>(), nullptr, c->Em,
                            c->scan_tmp.as<int64_t>(), c->stream);
  k_mp_fill<<<pg, 256, 0, c->stream>>>(c->pairs_m.as<int32_t>(), c->flag.as<uint8_t>(), c->pair_cap,
                                       c->mp_off.as<int64_t>(), c->mp_cnt.as<int32_t>(), c->mp_list.as<int32_t>(), st);
  if (c->Em > 0)
    k_mp_sort<<<(unsigned)((c->Em + kThreads - 1) / kThreads), kThreads, 0, c->stream>>>(
        c->mp_off.as<int64_t>(), c->Em, c->mp_list.as<int32_t>());
  if (c->Ns > 0)
    k_grad_slave<<<(unsigned)((c->Ns + kThreads - 1) / kThreads), kThreads, 0, c->stream>>>(
        c->n2e_s_ptr.as<int64_t>(), c->n2e_s_ent.as<int64_t>(), c->pair_off.as<int64_t>(), c->flag.as<uint8_t>(),
        c->gs_pair.as<double>(), c->ge_elem.as<double>(), c->Ns, c->grad_s.as<double>(), st);
  if (c->Nm > 0)
    k_grad_master<<<(unsigned)((c->Nm + kThreads - 1) / kThreads), kThreads, 0, c->stream>>>(
        c->n2e_m_ptr.as<int64_t>(), c->n2e_m_ent.as<int64_t>(), c->mp_off.as<int64_t>(), c->mp_list.as<int32_t>(),
        c->gm_pair.as<double>(), c->Nm, c->grad_m.as<double>(), st);
  k_J_partial<<<kJBlocks, 256, 0, c->stream>>>(c->J_pair.as<double>(), c->pair_cap, c->ge_elem.as<double>(), c->Es,
                                               c->J_part.as<double>(), st);
  k_J_final<<<1, 256, 0, c->stream>>>(c->J_part.as<double>(), st);
}
#endif  // MORTAR_PAIR_NS

}  // namespace mortar
