// Linearisation of the mortar coupling terms (Sec. 1: the consistent
// linearisation of D and M enters every nonlinear iteration):
//     K = d/dX [ (D (x) I3) ys - (M (x) I3) ym ],   ys, ym held fixed,
// a block-sparse matrix of 3x3 blocks: block rows = slave nodes, block
// columns = slave nodes, then master nodes.
//
// Per pair (s, m), in the standard basis N_e of the slave element,
//     O_e,c = sum over quadrature points of W N_e(xi_s) Z_c,
//     Z_c   = [segment D] sum_b N_b(xi_s) ys_b,c - sum_l N_l(xi_m) ym_l,c,
// and the pair's rows are sum_e A[a][e] O_e,c (A = I for standard LMs).
// Three lanes own one pair, one component c each, and run the reverse sweep
// of the four outputs O_0..3,c together: each lane computes every third
// quadrature point's back-projections and shape functions and shares them
// with the other two through shared memory, the per-point adjoints of the
// four seeds are accumulated side by side (their map-coefficient adjoints in
// shared memory), and only the reverse of the clip and of the projection runs
// once per seed.  The derivatives through A (dual LMs) and of
// the element-domain D depend on the slave element alone: a per-element
// kernel pushes the pair sums of O and the D term through A = Dh Me^-1 and
// the element integrals in forward mode over the 12 slave coordinates.  Rows
// are gathered per slave node in a fixed order into BSR with no
// floating-point atomics: bitwise reproducible.
#include <algorithm>

#include "clip.cuh"
#include "context.h"
#include "reverse.cuh"

namespace mortar {

namespace {

constexpr int kTanWarps = 4;
constexpr int kTanThreads = 32 * kTanWarps;
constexpr int kThreads = 128;
// map-coefficient adjoints of 4 seeds per thread, then 32 exchange slots per warp
constexpr size_t kTanSmem = sizeof(double) * 16 * 4 * kTanThreads + 32 * kTanWarps * 28 * sizeof(double);

struct TanArgs {
  const int32_t* ps;
  const int32_t* pm;
  const double* srec;
  const double* xs;
  const double* xm;
  const int32_t* conn_s;
  const int32_t* conn_m;
  const double* ys;
  const double* ym;
  double* Kp;          // per pair 288: [a][c][k][d], k < 4 slave node, k >= 4 master node k - 4
  double* Op;          // per pair 12: O_e,c (dual LMs)
  const uint8_t* flag; // per pair: non-empty in the forward run (FP64 clip)
  int64_t pair_cap;
  DevStatus* st;
  int32_t watchdog_us;
};

// Quadrature-point data one lane computes and the other two lanes of its
// pair group read (shared memory): back-projections, shape-function state of
// both sides and both inverse Jacobians.
struct GPX {
  double xs1, xs2, xm1, xm2;
  double sN[4], sq[4], mN[4], mq[4];
  double a[4], b[4];
};

// Pair p, component cp, for the lanes of one pair group (lanes 3g, 3g + 1,
// 3g + 2 hold components 0, 1, 2 of the same pair).  Every lane of the warp
// calls this with the same control flow around the exchanges: lanes with
// live = false (no pair) take part in the loops and exchanges without work.
// acc: this thread's shared-memory accumulators, entry i at acc[i * kTanThreads];
// gx: the warp's 32 exchange slots.
template <int NS, int NM, bool SEG, bool DUAL>
__device__ void tangent_pair(const TanArgs& g, int64_t p, int cp, bool live, double* __restrict__ acc,
                             GPX* __restrict__ gx, unsigned long long& clip_over, unsigned long long& newton_fail) {
  const int lane = threadIdx.x & 31;
  const int32_t s = g.ps[p], m = g.pm[p];
  const double* r = g.srec + (int64_t)SR_STRIDE * s;
  const int32_t* cs = g.conn_s + (int64_t)NS * s;
  const int32_t* cm = g.conn_m + (int64_t)NM * m;
  double yS[4] = {0, 0, 0, 0}, yM[4] = {0, 0, 0, 0};
  for (int a = 0; a < NS; ++a) yS[a] = g.ys[3 * (int64_t)cs[a] + cp];
  for (int l = 0; l < NM; ++l) yM[l] = g.ym[3 * (int64_t)cm[l] + cp];
  const V3 x0 = v3(r[SR_X0], r[SR_X0 + 1], r[SR_X0 + 2]);
  const V3 t1 = v3(r[SR_T1], r[SR_T1 + 1], r[SR_T1 + 2]);
  const V3 t2 = v3(r[SR_T2], r[SR_T2 + 1], r[SR_T2 + 2]);
  double mu[4], mv[4];
  for (int l = 0; l < NM; ++l) {
    const int64_t n = cm[l];
    const double dx = g.xm[3 * n] - x0.x, dy = g.xm[3 * n + 1] - x0.y, dz = g.xm[3 * n + 2] - x0.z;
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
  ClipPool<NS, NM> clip;   // compact record: master corners + intersections
  unsigned long long clip_dummy = 0;
  const bool nonempty = clip.run(r, mu, mv, mrev, live ? clip_over : clip_dummy);
  // row a at + 72 a; written with streaming (evict-first) stores, so that L2
  // keeps the threads' stack lines rather than these write-once blocks
  double* kout = g.Kp + 288 * p + 24 * cp;
  const int nr = nonempty ? clip.nr : 0;
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
  // per-seed adjoints of the polygon vertices, kept at the vertices' pool slots
  constexpr int kSlots = ClipPool<NS, NM>::kSlots;
  double Rbu[4][kSlots], Rbv[4][kSlots];
  for (int k = 0; k < clip.nv; ++k)
    for (int e = 0; e < NS; ++e) { Rbu[e][k] = 0.0; Rbv[e][k] = 0.0; }
  double cu = 0.0, cv = 0.0;
  int ncell = nr >= 3 ? 1 : 0;
  if (nr > 3) {
    double su = 0.0, sv = 0.0;
    for (int k = 0; k < nr; ++k) { su += clip.u(k); sv += clip.v(k); }
    cu = su * kInvCount[nr];
    cv = sv * kInvCount[nr];
    ncell = nr;
  }
  if (!live) ncell = 0;
  for (int i = 0; i < 16 * NS; ++i) acc[i * kTanThreads] = 0.0;
  double O[4] = {0, 0, 0, 0}, cbu[4] = {0, 0, 0, 0}, cbv[4] = {0, 0, 0, 0};
  const int ncell_w = __reduce_max_sync(0xffffffffu, ncell);
  const int gbase = 3 * (lane / 3);
  for (int cI = 0; cI < ncell_w; ++cI) {
    const bool cell_ok = cI < ncell;
    int ib = 0, iw = 0;   // pool slots of the cell's two polygon vertices
    double au = 0.0, av = 0.0;
    if (cell_ok) {
      if (nr == 3) {
        au = clip.u(0); av = clip.v(0); ib = clip.id(1); iw = clip.id(2);
      } else {
        au = cu; av = cv; ib = clip.id(cI); iw = clip.id(cI + 1 == nr ? 0 : cI + 1);
      }
    }
    const double e1u = cell_ok ? clip.pu[ib] - au : 0.0, e1v = cell_ok ? clip.pv[ib] - av : 0.0;
    const double e2u = cell_ok ? clip.pu[iw] - au : 0.0, e2v = cell_ok ? clip.pv[iw] - av : 0.0;
    const double crs = cross2(e1u, e1v, e2u, e2v);
    const double area = 0.5 * fabs(crs);
    double arb[4], e1bu[4], e1bv[4], e2bu[4], e2bv[4], xbu_c[4], xbv_c[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      arb[e] = 0.0; e1bu[e] = 0.0; e1bv[e] = 0.0; e2bu[e] = 0.0; e2bv[e] = 0.0; xbu_c[e] = 0.0; xbv_c[e] = 0.0;
    }
#pragma unroll 1
    for (int rr = 0; rr < 3; ++rr) {
      // this lane's quadrature point of the round (component cp computes point 3 rr + cp)
      const int qo = 3 * rr + cp;
      if (cell_ok && qo < 7) {
        double l1, l2, w;
        tri7_point(qo, l1, l2, w);
        const double xu = au + l1 * e1u + l2 * e2u;
        const double xv = av + l1 * e1v + l2 * e2v;
        GPX& o = gx[lane];
        double xs1, xs2, xm1, xm2;
        if (!si.solve(xu, xv, xs1, xs2)) newton_fail++;
        if (!mi.solve(xu, xv, xm1, xm2)) newton_fail++;
        ShapeAD<NS> SA;
        ShapeAD<NM> MA;
        SA.eval(xs1, xs2);
        MA.eval(xm1, xm2);
        o.xs1 = xs1; o.xs2 = xs2; o.xm1 = xm1; o.xm2 = xm2;
#pragma unroll
        for (int k = 0; k < 4; ++k) { o.sN[k] = SA.N[k]; o.mN[k] = MA.N[k]; }
        o.sq[0] = SA.qa; o.sq[1] = SA.qb; o.sq[2] = SA.qc; o.sq[3] = SA.qd;
        o.mq[0] = MA.qa; o.mq[1] = MA.qb; o.mq[2] = MA.qc; o.mq[3] = MA.qd;
        si.jinv(xs1, xs2, o.a[0], o.a[1], o.a[2], o.a[3]);
        mi.jinv(xm1, xm2, o.b[0], o.b[1], o.b[2], o.b[3]);
      }
      __syncwarp();
#pragma unroll 1
      for (int jj = 0; jj < 3; ++jj) {
        const int q = 3 * rr + jj;
        if (!(cell_ok && q < 7)) continue;
        const GPX& x = gx[gbase + jj];
        double l1, l2, w;
        tri7_point(q, l1, l2, w);
        const double W = w * area;
        const double xs1 = x.xs1, xs2 = x.xs2, xm1 = x.xm1, xm2 = x.xm2;
        ShapeAD<NS> SA;
        ShapeAD<NM> MA;
#pragma unroll
        for (int k = 0; k < 4; ++k) { SA.N[k] = x.sN[k]; MA.N[k] = x.mN[k]; }
        SA.qa = x.sq[0]; SA.qb = x.sq[1]; SA.qc = x.sq[2]; SA.qd = x.sq[3];
        MA.qa = x.mq[0]; MA.qb = x.mq[1]; MA.qc = x.mq[2]; MA.qd = x.mq[3];
        double Z = 0.0;
        if (SEG)
#pragma unroll
          for (int b = 0; b < NS; ++b) Z = fma(SA.N[b], yS[b], Z);
#pragma unroll
        for (int l = 0; l < NM; ++l) Z = fma(-MA.N[l], yM[l], Z);
        // gradients in the plane: J_s^-T grad_xi N_e, J^-T grad_xi of the interpolated y
        const double a00 = x.a[0], a01 = x.a[1], a10 = x.a[2], a11 = x.a[3];
        double dx[4], de[4];
        if constexpr (NS == 4) {
          dx[0] = -SA.qc; dx[1] = SA.qc; dx[2] = SA.qd; dx[3] = -SA.qd;
          de[0] = -SA.qa; de[1] = -SA.qb; de[2] = SA.qb; de[3] = SA.qa;
        } else {
          dx[0] = -1.0; dx[1] = 1.0; dx[2] = 0.0; dx[3] = 0.0;
          de[0] = -1.0; de[1] = 0.0; de[2] = 1.0; de[3] = 0.0;
        }
        // gu_e = J_s^-T grad N_e = (a00 dx_e + a10 de_e, a01 dx_e + a11 de_e) enters
        // only scaled by W Z (and, segment mode, through sum_e yS_e gu_e): the
        // scale is folded into the coefficients once per point
        const double WZ = W * Z, wZ = w * Z;
        const double p00 = WZ * a00, p10 = WZ * a10, p01 = WZ * a01, p11 = WZ * a11;
        double WgYsu = 0.0, WgYsv = 0.0;
        if (SEG) {
          double sdx = 0.0, sde = 0.0;
#pragma unroll
          for (int e = 0; e < NS; ++e) { sdx = fma(yS[e], dx[e], sdx); sde = fma(yS[e], de[e], sde); }
          WgYsu = W * fma(a00, sdx, a10 * sde);
          WgYsv = W * fma(a01, sdx, a11 * sde);
        }
        double ym0, ym1;
        MA.pull(yM, ym0, ym1);
        const double b00 = x.b[0], b01 = x.b[1], b10 = x.b[2], b11 = x.b[3];
        const double mWu = -W * fma(b00, ym0, b10 * ym1), mWv = -W * fma(b01, ym0, b11 * ym1);
        const double s12 = xs1 * xs2, m12 = xm1 * xm2;
#pragma unroll
        for (int e = 0; e < NS; ++e) {
          const double ne = SA.N[e];
          O[e] = fma(ne, WZ, O[e]);
          arb[e] = fma(wZ, ne, arb[e]);
          double su = fma(p00, dx[e], p10 * de[e]), sv = fma(p01, dx[e], p11 * de[e]);   // J_s^-T (adjoint of xi_s)
          if (SEG) { su = fma(ne, WgYsu, su); sv = fma(ne, WgYsv, sv); }
          const double tu = ne * mWu, tv = ne * mWv;   // J_m^-T (adjoint of xi_m)
          double* A = acc + (16 * e) * kTanThreads;
          A[0 * kTanThreads] -= su;
          A[1 * kTanThreads] -= sv;
          A[2 * kTanThreads] = fma(-xs1, su, A[2 * kTanThreads]);
          A[3 * kTanThreads] = fma(-xs1, sv, A[3 * kTanThreads]);
          A[4 * kTanThreads] = fma(-xs2, su, A[4 * kTanThreads]);
          A[5 * kTanThreads] = fma(-xs2, sv, A[5 * kTanThreads]);
          A[6 * kTanThreads] = fma(-s12, su, A[6 * kTanThreads]);
          A[7 * kTanThreads] = fma(-s12, sv, A[7 * kTanThreads]);
          A[8 * kTanThreads] -= tu;
          A[9 * kTanThreads] -= tv;
          A[10 * kTanThreads] = fma(-xm1, tu, A[10 * kTanThreads]);
          A[11 * kTanThreads] = fma(-xm1, tv, A[11 * kTanThreads]);
          A[12 * kTanThreads] = fma(-xm2, tu, A[12 * kTanThreads]);
          A[13 * kTanThreads] = fma(-xm2, tv, A[13 * kTanThreads]);
          A[14 * kTanThreads] = fma(-m12, tu, A[14 * kTanThreads]);
          A[15 * kTanThreads] = fma(-m12, tv, A[15 * kTanThreads]);
          const double xbu = su + tu, xbv = sv + tv;
          xbu_c[e] += xbu; xbv_c[e] += xbv;
          e1bu[e] = fma(l1, xbu, e1bu[e]); e1bv[e] = fma(l1, xbv, e1bv[e]);
          e2bu[e] = fma(l2, xbu, e2bu[e]); e2bv[e] = fma(l2, xbv, e2bv[e]);
        }
      }
      __syncwarp();   // the slots are rewritten by the next three points
    }
    if (cell_ok) {
#pragma unroll
      for (int e = 0; e < NS; ++e) {   // area = |cross| / 2, cell vertices, centroid
        const double crb = 0.5 * (crs < 0.0 ? -arb[e] : arb[e]);
        e1bu[e] += crb * e2v; e1bv[e] -= crb * e2u;
        e2bu[e] -= crb * e1v; e2bv[e] += crb * e1u;
        Rbu[e][ib] += e1bu[e]; Rbv[e][ib] += e1bv[e];
        Rbu[e][iw] += e2bu[e]; Rbv[e][iw] += e2bv[e];
        const double abu = xbu_c[e] - (e1bu[e] + e2bu[e]), abv = xbv_c[e] - (e1bv[e] + e2bv[e]);
        if (nr == 3) {
          const int s0 = clip.id(0);
          Rbu[e][s0] += abu; Rbv[e][s0] += abv;
        } else {
          cbu[e] += abu; cbv[e] += abv;
        }
      }
    }
  }
  if (!live) return;
  if (!nonempty) {   // not reached for pairs the count pass found non-empty; blocks stay defined
    for (int a = 0; a < 4; ++a)
      for (int k = 0; k < 24; ++k) __stcs(kout + 72 * a + k, 0.0);
    if (DUAL)
      for (int e = 0; e < 4; ++e) __stcs(g.Op + 12 * p + 3 * e + cp, 0.0);
    return;
  }
  if (nr > 3) {
    const double inv = kInvCount[nr];
    for (int e = 0; e < NS; ++e)
      for (int k = 0; k < nr; ++k) {
        const int sk = clip.id(k);
        Rbu[e][sk] += cbu[e] * inv; Rbv[e][sk] += cbv[e] * inv;
      }
  }
  // ---- per seed: clip and merge, map coefficients, projection and plane;
  //      node coordinates read again here (L1/L2) rather than held through
  //      the quadrature loop
  const V3 n0 = v3(r[SR_N0], r[SR_N0 + 1], r[SR_N0 + 2]);
  V3 X[4], Y[4];
  for (int a = 0; a < NS; ++a) {
    const int64_t n = cs[a];
    X[a] = v3(g.xs[3 * n], g.xs[3 * n + 1], g.xs[3 * n + 2]);
  }
  for (int l = 0; l < NM; ++l) {
    const int64_t n = cm[l];
    Y[l] = v3(g.xm[3 * n], g.xm[3 * n + 1], g.xm[3 * n + 2]);
  }
  double Ks[DUAL ? 4 : 1][24];   // seed rows, combined through A at the end (dual LMs)
  for (int e = 0; e < NS; ++e) {
    double sbu[4] = {0, 0, 0, 0}, sbv[4] = {0, 0, 0, 0}, mbu[4] = {0, 0, 0, 0}, mbv[4] = {0, 0, 0, 0};
    clip.reverse(r, Rbu[e], Rbv[e], srev, mrev, sbu, sbv, mbu, mbv);
    double smb[8], mmb[8];
    for (int k = 0; k < 8; ++k) {
      smb[k] = acc[(16 * e + k) * kTanThreads];
      mmb[k] = acc[(16 * e + 8 + k) * kTanThreads];
    }
    map_coeff_reverse<NS>(smb, sbu, sbv);
    map_coeff_reverse<NM>(mmb, mbu, mbv);
    double gX[4][3], gY[4][3];
    for (int a = 0; a < 4; ++a)
      for (int d = 0; d < 3; ++d) { gX[a][d] = 0.0; gY[a][d] = 0.0; }
    plane_reverse<NS, NM>(X, Y, x0, t1, t2, n0, sbu, sbv, mbu, mbv, gX, gY);
    if (DUAL) {
      for (int a = 0; a < 4; ++a)
        for (int d = 0; d < 3; ++d) {
          Ks[DUAL ? e : 0][3 * a + d] = gX[a][d];
          Ks[DUAL ? e : 0][12 + 3 * a + d] = gY[a][d];
        }
    } else {   // standard LMs: seed e is row e
      for (int a = 0; a < 4; ++a)
        for (int d = 0; d < 3; ++d) {
          __stcs(kout + 72 * e + 3 * a + d, gX[a][d]);
          __stcs(kout + 72 * e + 12 + 3 * a + d, gY[a][d]);
        }
    }
  }
  if (DUAL) {
    for (int a = 0; a < 4; ++a)
      for (int k = 0; k < 24; ++k) {
        double v = 0.0;
        if (a < NS)
          for (int e = 0; e < NS; ++e) v = fma(r[SR_A + 4 * a + e], Ks[e][k], v);
        __stcs(kout + 72 * a + k, v);
      }
  } else {
    for (int a = NS; a < 4; ++a)
      for (int k = 0; k < 24; ++k) __stcs(kout + 72 * a + k, 0.0);
  }
  if (DUAL)
    for (int e = 0; e < 4; ++e) __stcs(g.Op + 12 * p + 3 * e + cp, e < NS ? O[e] : 0.0);
}

// Persistent kernel over warp batches of 32 R pairs, each sorted by the cell
// count and edge intersections of an FP32 clip (ballot counting sort) and
// swept in rounds of 10 pairs x 3 components.
template <int NS, int NM, bool SEG, bool DUAL, int R>
__global__ void __launch_bounds__(kTanThreads) k_tangent_pairs(TanArgs g) {
  extern __shared__ double tan_acc[];
  constexpr int B = 32 * R;
  __shared__ uint8_t perm_s[kTanWarps][B];
  __shared__ unsigned pres_s[kTanWarps][8];   // key values present in the batch (256 bits)
  uint8_t* perm = perm_s[threadIdx.x >> 5];
  unsigned* pres = pres_s[threadIdx.x >> 5];
  double* acc = tan_acc + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  unsigned long long clip_over = 0, newton_fail = 0;
  DevStatus* st = g.st;
  const bool ok = st->over_pairs == 0 && st->over_bins == 0;
  const int64_t n = ok ? (int64_t)min((unsigned long long)g.pair_cap, st->n_pairs) : 0;
  const int64_t items = (n + B - 1) / B;
  GPX* gx = reinterpret_cast<GPX*>(tan_acc + 16 * 4 * kTanThreads) + 32 * (threadIdx.x >> 5);
  const Watchdog wd(g.watchdog_us);
  for (;;) {   // bounded: the shared counter only grows
    if (wd.expired(&st->timeout)) break;
    int64_t item = 0;
    if (lane == 0) item = (int64_t)atomicAdd(&st->work_ctr3, 1ull);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= items) break;
    const int64_t base = item * B;
    // sort key: 0 for pairs the forward run found empty (their blocks are
    // never read), else 1 + 16 x the cell count + the edge intersections of
    // an FP32 clip (a cost estimate only; the FP64 clip of the pair kernel
    // decides)
    if (lane < 8) pres[lane] = 0u;
    __syncwarp();
    int key[R];
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      const int64_t p = base + rr * 32 + lane;
      int k = 0;
      if (p < n && g.flag[p]) {
        int n_int = 0;
        const int nr = clip_count_f32<NS, NM>(g.srec + (int64_t)SR_STRIDE * g.ps[p], g.xm, g.conn_m, g.pm[p],
                                              n_int);
        k = 1 + 16 * (nr == 0 ? 0 : (nr == 3 ? 1 : min(nr, kPolyS))) + min(n_int, 15);
        atomicOr(&pres[k >> 5], 1u << (k & 31));
      }
      key[rr] = k;
    }
    __syncwarp();
    int pos[R];
    int basecnt = 0;
#pragma unroll 1
    for (int w = 7; w >= 0; --w) {
      unsigned bits = pres[w];
      while (bits != 0u) {   // uniform across the warp
        const int b = 31 - __clz(bits);
        bits &= ~(1u << b);
        const int v = 32 * w + b;
        int before = 0;
#pragma unroll
        for (int rr = 0; rr < R; ++rr) {
          const unsigned mk = __ballot_sync(0xffffffffu, key[rr] == v);
          if (key[rr] == v) pos[rr] = basecnt + before + __popc(mk & lt_mask);
          before += __popc(mk);
        }
        basecnt += before;
      }
    }
    const int n_live = basecnt;
#pragma unroll
    for (int rr = 0; rr < R; ++rr)
      if (key[rr] > 0) perm[pos[rr]] = (uint8_t)(rr * 32 + lane);
    __syncwarp();
    // rounds of 10 pairs: lanes 3 g .. 3 g + 2 take components 0..2 of pair g
    const int grp = lane / 3, cp = lane - 3 * (lane / 3);
    for (int i0 = 0; i0 < n_live; i0 += 10) {
      const int i = i0 + grp;
      const bool live = lane < 30 && i < n_live;
      const int64_t p = base + perm[live ? i : i0];
      tangent_pair<NS, NM, SEG, DUAL>(g, p, cp, live, acc, gx, clip_over, newton_fail);
      __syncwarp();
    }
    __syncwarp();
  }
  (void)clip_over;     // both counted once already by the forward pass
  (void)newton_fail;
}

// Per slave element (forward mode over its 12 coordinates X_b,d):
//   Ke[a][c][b][d] = sum_e dA[a][e]/dX_bd S[e][c]                     (dual LMs)
//                  + sum_b' dDe[a][b']/dX_bd ys_b',c                  (element D)
// with S = sum of O over the element's non-empty pairs, A = Dh Me^-1 (so
// dA S = dDh T - A dMe T, T = Me^-1 S = Dh^-1 A S) and De = A Me (dual:
// De = Dh, dDe = dDh; standard: dDe = dMe).  Every element integral is
// sum_q w f(q) J(q), and dJ(q)/dX_bd = dN_b/dxi (g2 x n)_d + dN_b/deta (n x g1)_d,
// so Ke[a][c][b][d] = sum_q rho[a][c](q) dJ(q)/dX_bd with
//   rho[a][c] = w (N_a T[a][c] - Phi_a tau_c) + [element D] w N_a yD_a,c,
//   tau_c = sum_j N_j T[j][c], Phi_a = sum_i A[a][i] N_i,
//   yD_a,c = ys_a,c (dual) or sum_b N_b ys_b,c (standard).
template <int NS, bool DUAL, bool ELEMD>
__global__ void __launch_bounds__(kThreads) k_tangent_elems(
    const double* __restrict__ xs, const int32_t* __restrict__ conn_s, const double* __restrict__ ys,
    const double* __restrict__ srec, const int64_t* __restrict__ pair_off, const uint8_t* __restrict__ flag,
    const double* __restrict__ Op, int64_t Es, double* __restrict__ Ke, const DevStatus* st) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Es) return;
  double* out = Ke + 144 * e;
  for (int k = 0; k < 144; ++k) out[k] = 0.0;
  const double* r = srec + (int64_t)SR_STRIDE * e;
  if (r[SR_EPSIN] < 0.0 || st->over_pairs) return;
  V3 X[4];
  double yS[4][3];
  for (int a = 0; a < 4; ++a) {
    X[a] = v3(0, 0, 0);
    yS[a][0] = yS[a][1] = yS[a][2] = 0.0;
  }
  for (int a = 0; a < NS; ++a) {
    const int64_t n = conn_s[(int64_t)NS * e + a];
    X[a] = v3(xs[3 * n], xs[3 * n + 1], xs[3 * n + 2]);
    for (int c = 0; c < 3; ++c) yS[a][c] = ys[3 * n + c];
  }
  double A[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) A[a][b] = r[SR_A + 4 * a + b];
  constexpr int nq = NS == 4 ? 9 : 7;
  double T[4][3];
  for (int a = 0; a < 4; ++a) T[a][0] = T[a][1] = T[a][2] = 0.0;
  if (DUAL) {
    double S[4][3];
    for (int a = 0; a < 4; ++a) S[a][0] = S[a][1] = S[a][2] = 0.0;
    for (int64_t p = pair_off[e]; p < pair_off[e + 1]; ++p) {
      if (!flag[p]) continue;
      for (int a = 0; a < NS; ++a)
        for (int c = 0; c < 3; ++c) S[a][c] += Op[12 * p + 3 * a + c];
    }
    double Dh[4] = {0, 0, 0, 0};
    for (int q = 0; q < nq; ++q) {
      double xi, eta, w;
      elem_point_a<NS>(q, xi, eta, w);
      double N[4], dN[4][2];
      shape_fn<NS>(xi, eta, N);
      shape_grad<NS>(xi, eta, dN);
      V3 g1 = v3(0, 0, 0), g2 = v3(0, 0, 0);
      for (int a = 0; a < NS; ++a) { g1 = g1 + dN[a][0] * X[a]; g2 = g2 + dN[a][1] * X[a]; }
      const V3 nq3 = cross(g1, g2);
      const double wj = w * sqrt(dot(nq3, nq3));
      for (int a = 0; a < NS; ++a) Dh[a] += wj * N[a];
    }
    for (int j = 0; j < NS; ++j)
      for (int c = 0; c < 3; ++c) {
        double v = 0.0;
        for (int k = 0; k < NS; ++k) v = fma(A[j][k], S[k][c], v);
        T[j][c] = v / Dh[j];
      }
  }
  // flat element (parallelogram, every tri3): constant tangents g1, g2, so
  // dJ/dX_bd = dN_b/dxi c1_d + dN_b/deta c2_d with constant c1, c2, and the
  // point sums of rho dN_b are taken first (96 sums instead of 144 per point)
  bool flat;
  V3 g1c, g2c;
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
  if (flat) {
    const V3 ncv = cross(g1c, g2c);
    const V3 nu = (1.0 / sqrt(dot(ncv, ncv))) * ncv;
    const V3 c1 = cross(g2c, nu), c2 = cross(nu, g1c);
    const double c1d[3] = {c1.x, c1.y, c1.z}, c2d[3] = {c2.x, c2.y, c2.z};
    double P1[4][3][4], P2[4][3][4];
    for (int a = 0; a < 4; ++a)
      for (int c = 0; c < 3; ++c)
        for (int b = 0; b < 4; ++b) { P1[a][c][b] = 0.0; P2[a][c][b] = 0.0; }
    for (int q = 0; q < nq; ++q) {
      double xi, eta, w;
      elem_point_a<NS>(q, xi, eta, w);
      double N[4], dN[4][2];
      shape_fn<NS>(xi, eta, N);
      shape_grad<NS>(xi, eta, dN);
      double tau[3] = {0, 0, 0}, yq[3] = {0, 0, 0};
      for (int j = 0; j < NS; ++j)
        for (int c = 0; c < 3; ++c) {
          tau[c] = fma(N[j], T[j][c], tau[c]);
          yq[c] = fma(N[j], yS[j][c], yq[c]);
        }
      for (int a = 0; a < NS; ++a) {
        double phi = 0.0;
        for (int i = 0; i < NS; ++i) phi = fma(A[a][i], N[i], phi);
        for (int c = 0; c < 3; ++c) {
          double rho = 0.0;
          if (DUAL) rho = w * (N[a] * T[a][c] - phi * tau[c]);
          if (ELEMD) rho = fma(w * N[a], DUAL ? yS[a][c] : yq[c], rho);
          for (int b = 0; b < NS; ++b) {
            P1[a][c][b] = fma(rho, dN[b][0], P1[a][c][b]);
            P2[a][c][b] = fma(rho, dN[b][1], P2[a][c][b]);
          }
        }
      }
    }
    for (int a = 0; a < NS; ++a)
      for (int c = 0; c < 3; ++c)
        for (int b = 0; b < NS; ++b)
          for (int d = 0; d < 3; ++d)
            out[36 * a + 12 * c + 3 * b + d] = fma(P1[a][c][b], c1d[d], P2[a][c][b] * c2d[d]);
    return;
  }
  for (int q = 0; q < nq; ++q) {
    double xi, eta, w;
    elem_point_a<NS>(q, xi, eta, w);
    double N[4], dN[4][2];
    shape_fn<NS>(xi, eta, N);
    shape_grad<NS>(xi, eta, dN);
    V3 g1 = v3(0, 0, 0), g2 = v3(0, 0, 0);
    for (int a = 0; a < NS; ++a) { g1 = g1 + dN[a][0] * X[a]; g2 = g2 + dN[a][1] * X[a]; }
    const V3 nq3 = cross(g1, g2);
    const V3 nu = (1.0 / sqrt(dot(nq3, nq3))) * nq3;
    const V3 c1 = cross(g2, nu), c2 = cross(nu, g1);
    const double c1d[3] = {c1.x, c1.y, c1.z}, c2d[3] = {c2.x, c2.y, c2.z};
    double tau[3] = {0, 0, 0}, yq[3] = {0, 0, 0};
    for (int j = 0; j < NS; ++j)
      for (int c = 0; c < 3; ++c) {
        tau[c] = fma(N[j], T[j][c], tau[c]);
        yq[c] = fma(N[j], yS[j][c], yq[c]);
      }
    for (int a = 0; a < NS; ++a) {
      double phi = 0.0;
      for (int i = 0; i < NS; ++i) phi = fma(A[a][i], N[i], phi);
      for (int c = 0; c < 3; ++c) {
        double rho = 0.0;
        if (DUAL) rho = w * (N[a] * T[a][c] - phi * tau[c]);
        if (ELEMD) rho = fma(w * N[a], DUAL ? yS[a][c] : yq[c], rho);
        if (rho == 0.0) continue;
        double* o = out + 36 * a + 12 * c;
        for (int b = 0; b < NS; ++b) {
          const double u = rho * dN[b][0], v = rho * dN[b][1];
          for (int d = 0; d < 3; ++d) o[3 * b + d] = fma(u, c1d[d], fma(v, c2d[d], o[3 * b + d]));
        }
      }
    }
  }
}

// Sources of one block row j, visited in a fixed order: the slave elements
// around j (sorted), for each its non-empty pairs in (s, m) order, then the
// element block.  f(col, block pointer, row stride of the block, diagonal add).
template <int NS, int NM, bool SEG, bool DUAL, bool ELEMD>
struct TanRowSource {
  const int64_t* n2e_ptr;
  const int64_t* n2e_ent;
  const int64_t* pair_off;
  const int32_t* pm;
  const uint8_t* flag;
  const int32_t* conn_s;
  const int32_t* conn_m;
  const double* Kp;
  const double* Ke;
  const double* Mblk;
  const double* Dblk;
  const double* De;
  int64_t Ns;
  int direct;

  template <class F>
  __device__ __forceinline__ void visit(int64_t j, F&& f) const {
    for (int64_t q = n2e_ptr[j]; q < n2e_ptr[j + 1]; ++q) {
      const int64_t ee = n2e_ent[q];
      const int64_t e = ee >> 2;
      const int a = (int)(ee & 3);
      bool any = false;
      for (int64_t p = pair_off[e]; p < pair_off[e + 1]; ++p) {
        if (!flag[p]) continue;
        any = true;
        const double* kb = Kp + 288 * p + 72 * a;
        for (int k = 0; k < NS; ++k)
          f(conn_s[(int64_t)NS * e + k], kb + 3 * k, 24, (SEG && direct) ? Dblk[16 * p + 4 * a + k] : 0.0);
        const int64_t m = pm[p];
        for (int l = 0; l < NM; ++l)
          f((int32_t)(Ns + conn_m[(int64_t)NM * m + l]), kb + 12 + 3 * l, 24,
            direct ? -Mblk[16 * p + 4 * a + l] : 0.0);
      }
      if (ELEMD || (DUAL && any)) {
        const double* kb = Ke + 144 * e + 36 * a;
        for (int k = 0; k < NS; ++k)
          f(conn_s[(int64_t)NS * e + k], kb + 3 * k, 12, (ELEMD && direct) ? De[16 * e + 4 * a + k] : 0.0);
      }
    }
  }
};

// Sorted unique column ids of a row (block columns).
template <int CAP>
struct RowKeys {
  int32_t col[CAP];
  int u = 0;
  bool over = false;
  __device__ __forceinline__ void add(int32_t c) {
    int lo = 0, hi = u;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (col[mid] < c) lo = mid + 1; else hi = mid;
    }
    if (lo < u && col[lo] == c) return;
    if (u == CAP) { over = true; return; }
    for (int k = u; k > lo; --k) col[k] = col[k - 1];
    col[lo] = c;
    ++u;
  }
};

constexpr int kRowCap = 64;

// One thread per block row.  MODE 0: count the unique block columns.
// MODE 1: write them, sorted (the values follow in k_tangent_rows_warp).
template <int MODE, class Src>
__global__ void __launch_bounds__(kThreads) k_tangent_rows(Src src, int64_t N, int32_t* __restrict__ cnt,
                                                           const int64_t* __restrict__ rp, int64_t cap,
                                                           int32_t* __restrict__ col, double* __restrict__ val,
                                                           DevStatus* st) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  if (st->over_pairs) {
    if (MODE == 0) cnt[j] = 0;
    return;
  }
  if (MODE == 1 && rp[N] > cap) {
    if (j == 0) atomicMax(&st->over_K, 1ull);
    return;
  }
  RowKeys<kRowCap> keys;
  src.visit(j, [&](int32_t c, const double*, int, double) { keys.add(c); });
  int u = keys.u;
  const int64_t o = MODE == 1 ? rp[j] : 0;
  if (keys.over) {   // long row: repeated selection of the next column
    u = 0;
    int32_t last = -1;
    for (;;) {
      int32_t next = 0x7fffffff;
      src.visit(j, [&](int32_t c, const double*, int, double) { if (c > last && c < next) next = c; });
      if (next == 0x7fffffff) break;
      if (MODE == 1) col[o + u] = next;
      ++u;
      last = next;
    }
  } else if (MODE == 1) {
    for (int k = 0; k < u; ++k) col[o + k] = keys.col[k];
  }
  if (MODE == 0) cnt[j] = u;
  (void)val;
}

// Value pass, one warp per block row: the row's sorted columns (written by
// k_tangent_rows<1>) go to shared memory, then the row's sources are visited
// in the fixed order and each source's
// entries (72 of a pair row, 36 of an element row, contiguous in memory) are
// read by the 32 lanes together and added to the row's blocks held in shared
// memory.  Within one source no two entries share a block entry, and sources
// follow each other after a warp barrier, so every block entry is summed in
// the same order (sources in visit order).  Rows with more than kRowCap
// columns are summed by lane 0 alone in global memory, in the same order.
constexpr int kRowWarps = 4;

template <int NS, int NM, bool SEG, bool DUAL, bool ELEMD>
__global__ void __launch_bounds__(32 * kRowWarps) k_tangent_rows_warp(TanRowSource<NS, NM, SEG, DUAL, ELEMD> src,
                                                                      int64_t N, const int64_t* __restrict__ rp,
                                                                      int64_t cap, int32_t* __restrict__ col,
                                                                      double* __restrict__ val, DevStatus* st) {
  __shared__ int32_t keys_s[kRowWarps][kRowCap];
  __shared__ double acc_s[kRowWarps][kRowCap * 9];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* keys = keys_s[w];
  double* acc = acc_s[w];
  if (st->over_pairs) return;
  if (rp[N] > cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicMax(&st->over_K, 1ull);
    return;
  }
  const int64_t nw = (int64_t)gridDim.x * kRowWarps;
  for (int64_t j = (int64_t)blockIdx.x * kRowWarps + w; j < N; j += nw) {
    const int64_t o = rp[j];
    const int u = (int)(rp[j + 1] - o);
    if (u > kRowCap) {   // long row: lane 0 accumulates in global memory, in the same order
      if (lane == 0) {
        double* vrow = val + 9 * o;
        for (int k = 0; k < 9 * u; ++k) vrow[k] = 0.0;
        const int32_t* crow = col + o;
        src.visit(j, [&](int32_t c, const double* blk, int stride, double diag) {
          int lo = 0, hi = u;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (crow[mid] < c) lo = mid + 1; else hi = mid;
          }
          double* vb = vrow + 9 * lo;
          for (int cc = 0; cc < 3; ++cc)
            for (int d = 0; d < 3; ++d) vb[3 * cc + d] += blk[stride * cc + d] + (cc == d ? diag : 0.0);
        });
      }
      __syncwarp();
      continue;
    }
    for (int k = lane; k < u; k += 32) keys[k] = col[o + k];
    for (int k = lane; k < 9 * u; k += 32) acc[k] = 0.0;
    __syncwarp();
    auto find = [&](int32_t c) {
      int lo = 0, hi = u;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (keys[mid] < c) lo = mid + 1; else hi = mid;
      }
      return lo;
    };
    for (int64_t q = src.n2e_ptr[j]; q < src.n2e_ptr[j + 1]; ++q) {
      const int64_t ee = src.n2e_ent[q];
      const int64_t e = ee >> 2;
      const int a = (int)(ee & 3);
      bool any = false;
      for (int64_t p = src.pair_off[e]; p < src.pair_off[e + 1]; ++p) {
        if (!src.flag[p]) continue;
        any = true;
        const int64_t m = src.pm[p];
        int mypos = 0;   // lanes 0..7: block position of the pair's node k = lane
        if (lane < NS) mypos = find(src.conn_s[(int64_t)NS * e + lane]);
        else if (lane >= 4 && lane < 4 + NM) mypos = find((int32_t)(src.Ns + src.conn_m[(int64_t)NM * m + lane - 4]));
        const double* kb = src.Kp + 288 * p + 72 * a;
        for (int it = 0; it < 3; ++it) {   // entries lane, lane + 32, lane + 64 (< 72)
          const int idx = lane + 32 * it;
          const int ic = idx < 72 ? idx : 0;
          const int c = ic / 24, rem = ic - 24 * c, k = rem / 3, d = rem - 3 * k;
          const int pos = __shfl_sync(0xffffffffu, mypos, k);   // every lane takes part
          const bool valid = idx < 72 && (k < NS || (k >= 4 && k - 4 < NM));
          if (!valid) continue;
          double v = kb[idx];
          if (src.direct && c == d)
            v += k < 4 ? (SEG ? src.Dblk[16 * p + 4 * a + k] : 0.0) : -src.Mblk[16 * p + 4 * a + (k - 4)];
          acc[9 * pos + 3 * c + d] += v;
        }
        __syncwarp();
      }
      if (ELEMD || (DUAL && any)) {
        int mypos = 0;
        if (lane < NS) mypos = find(src.conn_s[(int64_t)NS * e + lane]);
        const double* kb = src.Ke + 144 * e + 36 * a;
        for (int it = 0; it < 2; ++it) {   // entries lane, lane + 32 (< 36)
          const int idx = lane + 32 * it;
          const int ic = idx < 36 ? idx : 0;
          const int c = ic / 12, rem = ic - 12 * c, k = rem / 3, d = rem - 3 * k;
          const int pos = __shfl_sync(0xffffffffu, mypos, k);   // every lane takes part
          if (idx >= 36 || k >= NS) continue;
          double v = kb[idx];
          if (ELEMD && src.direct && c == d) v += src.De[16 * e + 4 * a + k];
          acc[9 * pos + 3 * c + d] += v;
        }
        __syncwarp();
      }
    }
    double* vrow = val + 9 * o;
    for (int k = lane; k < 9 * u; k += 32) vrow[k] = acc[k];
    __syncwarp();
  }
}

#ifdef MORTAR_PAIR_NS
__global__ void k_tangent_nnzb(const int64_t* __restrict__ rp, int64_t N, DevStatus* st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) st->nnzb_K = (unsigned long long)rp[N];
}

template <int NS, int NM, bool SEG, bool DUAL>
void launch_pairs_t(mortar_ctx* c) {
  TanArgs g{c->pairs_s.as<int32_t>(), c->pairs_m.as<int32_t>(), c->srec.as<double>(), c->xs.as<double>(),
            c->xm.as<double>(), c->conn_s.as<int32_t>(), c->conn_m.as<int32_t>(), c->tan_ys.as<double>(),
            c->tan_ym.as<double>(), c->tan_Kp.as<double>(), c->tan_Op.as<double>(), c->flag.as<uint8_t>(),
            c->tan_pair_cap, c->dstat.as<DevStatus>(), c->watchdog_us};
  // batches of 160 pairs: 16 full rounds of 10 pair groups (lanes 30, 31 idle)
  auto kern = k_tangent_pairs<NS, NM, SEG, DUAL, 5>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTanSmem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTanThreads, kTanSmem);
  if (per_sm < 1) per_sm = 1;
  kern<<<(unsigned)(c->n_sm * per_sm), kTanThreads, kTanSmem, c->stream>>>(g);
}

template <int NS, int NM, bool SEG, bool DUAL, bool ELEMD>
void rows_t(mortar_ctx* c, int mode) {
  TanRowSource<NS, NM, SEG, DUAL, ELEMD> src{
      c->n2e_s_ptr.as<int64_t>(), c->n2e_s_ent.as<int64_t>(), c->pair_off.as<int64_t>(), c->pairs_m.as<int32_t>(),
      c->flag.as<uint8_t>(), c->conn_s.as<int32_t>(), c->conn_m.as<int32_t>(), c->tan_Kp.as<double>(),
      c->tan_Ke.as<double>(), c->Mblk.as<double>(), c->Dblk.as<double>(), c->De.as<double>(), c->Ns,
      c->tan_direct};
  const int64_t N = c->Ns;
  const unsigned g = (unsigned)((N + kThreads - 1) / kThreads);
  DevStatus* st = c->dstat.as<DevStatus>();
  if (mode == 0) {
    if (N > 0)
      k_tangent_rows<0><<<g, kThreads, 0, c->stream>>>(src, N, c->row_cnt.as<int32_t>(), nullptr, 0, nullptr,
                                                       nullptr, st);
    launch_exclusive_scan_i32(c->row_cnt.as<int32_t>(), c->tan_rowptr.as<int64_t>(), nullptr, N,
                              c->scan_tmp.as<int64_t>(), c->stream);
    k_tangent_nnzb<<<1, 32, 0, c->stream>>>(c->tan_rowptr.as<int64_t>(), N, st);
  } else if (N > 0) {
    k_tangent_rows<1><<<g, kThreads, 0, c->stream>>>(src, N, nullptr, c->tan_rowptr.as<int64_t>(), c->tan_nnzb_cap,
                                                     c->tan_col.as<int32_t>(), nullptr, st);
    const int64_t blocks = std::min<int64_t>((N + kRowWarps - 1) / kRowWarps, (int64_t)c->n_sm * 64);
    k_tangent_rows_warp<NS, NM, SEG, DUAL, ELEMD><<<(unsigned)blocks, 32 * kRowWarps, 0, c->stream>>>(
        src, N, c->tan_rowptr.as<int64_t>(), c->tan_nnzb_cap, c->tan_col.as<int32_t>(), c->tan_val.as<double>(), st);
  }
}

}  // namespace

template <int NS, int NM>
void tangent_pairs_nsnm(mortar_ctx* c, const RunParams& rp) {
  const bool seg = rp.d_domain == 1, dual = rp.lm == 1;
  if (seg && dual) launch_pairs_t<NS, NM, true, true>(c);
  else if (seg) launch_pairs_t<NS, NM, true, false>(c);
  else if (dual) launch_pairs_t<NS, NM, false, true>(c);
  else launch_pairs_t<NS, NM, false, false>(c);
}

template <int NS, int NM>
void tangent_rows_nsnm(mortar_ctx* c, const RunParams& rp, int mode) {
  const bool seg = rp.d_domain == 1, dual = rp.lm == 1;
  if (seg && dual) rows_t<NS, NM, true, true, false>(c, mode);
  else if (seg) rows_t<NS, NM, true, false, false>(c, mode);
  else if (dual) rows_t<NS, NM, false, true, true>(c, mode);
  else rows_t<NS, NM, false, false, true>(c, mode);
}

template void tangent_pairs_nsnm<MORTAR_PAIR_NS, MORTAR_PAIR_NM>(mortar_ctx*, const RunParams&);
template void tangent_rows_nsnm<MORTAR_PAIR_NS, MORTAR_PAIR_NM>(mortar_ctx*, const RunParams&, int);
#else   // the main part: element blocks, dispatch

template <int NS, bool DUAL, bool ELEMD>
void launch_elems_t(mortar_ctx* c) {
  if (c->Es == 0) return;
  k_tangent_elems<NS, DUAL, ELEMD><<<(unsigned)((c->Es + kThreads - 1) / kThreads), kThreads, 0, c->stream>>>(
      c->xs.as<double>(), c->conn_s.as<int32_t>(), c->tan_ys.as<double>(), c->srec.as<double>(),
      c->pair_off.as<int64_t>(), c->flag.as<uint8_t>(), c->tan_Op.as<double>(), c->Es, c->tan_Ke.as<double>(),
      c->dstat.as<DevStatus>());
}

}  // namespace

bool tangent_needs_elems(const mortar_ctx* c) {
  return c->opt.lm == MORTAR_LM_DUAL || c->opt.d_domain == MORTAR_D_ELEMENT;
}

void launch_tangent_blocks(mortar_ctx* c, const RunParams& rp) {
  if (c->nen_s == 4 && c->nen_m == 4) tangent_pairs_nsnm<4, 4>(c, rp);
  else if (c->nen_s == 4 && c->nen_m == 3) tangent_pairs_nsnm<4, 3>(c, rp);
  else if (c->nen_s == 3 && c->nen_m == 4) tangent_pairs_nsnm<3, 4>(c, rp);
  else tangent_pairs_nsnm<3, 3>(c, rp);
  if (!tangent_needs_elems(c)) return;
  const bool elemd = rp.d_domain == 0, dual = rp.lm == 1;
  if (c->nen_s == 4) {
    if (dual && elemd) launch_elems_t<4, true, true>(c);
    else if (dual) launch_elems_t<4, true, false>(c);
    else launch_elems_t<4, false, true>(c);
  } else {
    if (dual && elemd) launch_elems_t<3, true, true>(c);
    else if (dual) launch_elems_t<3, true, false>(c);
    else launch_elems_t<3, false, true>(c);
  }
}

void launch_tangent_rows(mortar_ctx* c, const RunParams& rp, int mode) {
  if (c->nen_s == 4 && c->nen_m == 4) tangent_rows_nsnm<4, 4>(c, rp, mode);
  else if (c->nen_s == 4 && c->nen_m == 3) tangent_rows_nsnm<4, 3>(c, rp, mode);
  else if (c->nen_s == 3 && c->nen_m == 4) tangent_rows_nsnm<3, 4>(c, rp, mode);
  else tangent_rows_nsnm<3, 3>(c, rp, mode);
}
#endif  // MORTAR_PAIR_NS

}  // namespace mortar
