// Element-based integration of the mortar matrices (Sec. 1 and Sec. 2.3 set
// it against the segment-based Algorithm 1: no clipping or triangulation; a
// higher-order rule on the slave element copes with the kinks of the
// integrand at master element edges, at lower accuracy).
//
// One thread per slave element (points outermost, see the kernel).  Rule: n x n
// Gauss-Legendre points on quad4
// (collapsed n x n points on tri3), mapped into the element's auxiliary plane
// by the projected slave map, weights w |det J_s|.  The element's candidate
// pairs are visited in pair order; each takes the points not taken yet whose
// back-projection onto its projected master element converges inside it
// (|xi|, |eta| <= 1 + 1e-10 on quad4, barycentric >= -1e-10 on tri3) and adds
//     M_p[a][l] += W Phi_a(xi_s) N_l(xi_m),   D_p[a][b] += W Phi_a N_b(xi_s) (segment D).
// Points no master covers contribute nothing.  Ownership is a bit mask per
// thread.  The blocks keep the layout of the segment-based ones, so the
// assembly is shared.
#include <cmath>
#include <vector>

#include "clip.cuh"
#include "context.h"

namespace mortar {

namespace {

constexpr int kThreads = 128;
constexpr int kMaxRule = 16;
constexpr double kInsideTol = 1e-10;

constexpr int kChunk = 8;   // candidate pairs held per pass over the points

// One thread per slave element, points outermost: for each rule point the
// element's candidate pairs (a chunk of up to kChunk, with their projected
// master maps kept in thread-local memory) are tried in pair order with a box
// reject and the FP32 Newton iterate, and only the owner's FP64 step and the
// point's contribution are computed.  The FP64 work then runs once per point
// on every lane (interior elements own all points), instead of once per
// (pair, point) behind lane-divergent tests.  Contributions are added into
// the owner's block in global memory (this thread's own blocks, L1-resident)
// in point order.  Elements with more than kChunk pairs take further passes
// over the points not yet owned, so "first covering pair in pair order" holds.
// NODAL (dual LMs only): accumulate G = sum W N_s N_m^T in the nodal basis and
// apply A once per pair, instead of forming the dual basis at every point;
// chosen for rules with about ten or more points per pair (n >= 6).
template <int NS, int NM, bool SEG, bool DUAL, bool NODAL>
__global__ void __launch_bounds__(kThreads) k_integrate_elembased(
    const int64_t* __restrict__ pair_off, const int32_t* __restrict__ pm, const double* __restrict__ srec,
    const double* __restrict__ xm, const int32_t* __restrict__ conn_m, const double* __restrict__ rule, int n,
    int64_t Es, double* __restrict__ Mblk, double* __restrict__ Dblk, uint8_t* __restrict__ flag,
    DevStatus* st) {
  unsigned long long n_live = 0, n_gp = 0;
  const bool ok = st->over_pairs == 0 && st->over_bins == 0;
  const int nq = n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ok && e < Es;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p0 = pair_off[e], p1 = pair_off[e + 1];
    if (p0 == p1) continue;
    const double* r = srec + (int64_t)SR_STRIDE * e;
    const bool live = r[SR_EPSIN] >= 0.0;
    PlaneMap smap;
    smap.c0u = r[SR_C + 0]; smap.c0v = r[SR_C + 1]; smap.c1u = r[SR_C + 2]; smap.c1v = r[SR_C + 3];
    smap.c2u = r[SR_C + 4]; smap.c2v = r[SR_C + 5]; smap.c3u = r[SR_C + 6]; smap.c3v = r[SR_C + 7];
    const double x0x = r[SR_X0], x0y = r[SR_X0 + 1], x0z = r[SR_X0 + 2];
    const double t1x = r[SR_T1], t1y = r[SR_T1 + 1], t1z = r[SR_T1 + 2];
    const double t2x = r[SR_T2], t2y = r[SR_T2 + 1], t2z = r[SR_T2 + 2];
    double Phi_c[4][4];   // dual: Phi_a = sum_c A[a][c] N_c
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) Phi_c[a][c] = r[SR_A + 4 * a + c];
    uint32_t taken[kMaxRule * kMaxRule / 32];
#pragma unroll
    for (int k = 0; k < kMaxRule * kMaxRule / 32; ++k) taken[k] = 0u;
    for (int64_t c0 = p0; c0 < p1; c0 += kChunk) {
      const int kc = (int)min((int64_t)kChunk, p1 - c0);
      MapInverse mic[kChunk];
      float box[kChunk][4];
      int got[kChunk];
      for (int k = 0; k < kc; ++k) {
        got[k] = 0;
        const int64_t p = c0 + k;
        double* mo = Mblk + 16 * p;
        for (int t = 0; t < 16; ++t) mo[t] = 0.0;
        if (SEG) {
          double* dout = Dblk + 16 * p;
          for (int t = 0; t < 16; ++t) dout[t] = 0.0;
        }
        const int32_t m = pm[p];
        double mu[4], mv[4];
        double lo_u = 1e300, hi_u = -1e300, lo_v = 1e300, hi_v = -1e300;
#pragma unroll
        for (int l = 0; l < NM; ++l) {
          const int64_t nd = conn_m[(int64_t)NM * m + l];
          const double dx = xm[3 * nd] - x0x, dy = xm[3 * nd + 1] - x0y, dz = xm[3 * nd + 2] - x0z;
          mu[l] = dx * t1x + dy * t1y + dz * t1z;
          mv[l] = dx * t2x + dy * t2y + dz * t2z;
          lo_u = fmin(lo_u, mu[l]); hi_u = fmax(hi_u, mu[l]);
          lo_v = fmin(lo_v, mv[l]); hi_v = fmax(hi_v, mv[l]);
        }
        // box of the projected master element in FP32, widened far beyond the
        // inside tolerance and the FP32 rounding of the test point: a quick reject only
        const double band = 1e-4 * fmax(hi_u - lo_u, hi_v - lo_v);
        box[k][0] = f32_trunc(lo_u - band); box[k][1] = f32_trunc(hi_u + band);
        box[k][2] = f32_trunc(lo_v - band); box[k][3] = f32_trunc(hi_v + band);
        const PlaneMap mmap = plane_map<NM>(mu, mv);
        mic[k].setup(mmap, NM == 3 || map_is_affine(mmap));
      }
      if (live) {
        for (int q = 0; q < nq; ++q) {
          if ((taken[q >> 5] >> (q & 31)) & 1u) continue;
          const int i = q / n, j = q - (q / n) * n;
          double xi, eta, wq;
          if constexpr (NS == 4) {
            xi = rule[i]; eta = rule[j];
            wq = rule[n + i] * rule[n + j];
          } else {
            const double s = 0.5 * (rule[i] + 1.0), tt = 0.5 * (rule[j] + 1.0);
            xi = s; eta = tt * (1.0 - s);
            wq = 0.25 * rule[n + i] * rule[n + j] * (1.0 - s);
          }
          const double xe = xi * eta;
          const double xu = smap.c0u + smap.c1u * xi + smap.c2u * eta + smap.c3u * xe;
          const double xv = smap.c0v + smap.c1v * xi + smap.c2v * eta + smap.c3v * xe;
          const float fu = f32_trunc(xu), fv = f32_trunc(xv);
          // Owner search in two parts: an FP32 scan (box reject, FP32 Newton
          // iterate within 1e-5 of the element) finds the next candidate, then
          // its FP64 step and inside test run for all lanes together; a
          // candidate that fails the FP64 test (a point within 1e-5 of a
          // master edge) resumes the scan after it.  Same owner as testing
          // the candidates one by one in pair order.
          int owner = -1;
          double m1 = 0.0, m2 = 0.0;
          int k = 0;
          while (owner < 0 && k < kc) {
            int kn = -1, mode = 0;   // 1: affine (solved), 2: FP32 iterate near, 3: FP32 did not settle
            double a1 = 0.0, a2 = 0.0;
            CoarseInv ci;
            for (; k < kc; ++k) {
              if (fu < box[k][0] || fu > box[k][1] || fv < box[k][2] || fv > box[k][3]) continue;
              const MapInverse& mk = mic[k];
              if (mk.affine) { mode = 1; kn = k; break; }
              if (mk.coarse(xu, xv, a1, a2, ci)) {   // points clearly outside skip the FP64 step
                const bool near = NM == 4
                    ? (fabs(a1) <= 1.0 + 1e-5 && fabs(a2) <= 1.0 + 1e-5)
                    : (a1 >= -1e-5 && a2 >= -1e-5 && a1 + a2 <= 1.0 + 1e-5);
                if (!near) continue;
                mode = 2;
              } else {
                mode = 3;
              }
              kn = k;
              break;
            }
            if (kn < 0) break;
            k = kn + 1;
            MapInverse& mi = mic[kn];
            if (mode == 1) {
              mi.solve(xu, xv, a1, a2);
            } else if (mode == 2) {
              mi.polish(xu, xv, a1, a2, ci);
            } else if (!mi.newton64(xu, xv, a1, a2)) {   // FP32 did not settle: FP64 Newton from its iterate
              continue;
            }
            const bool inside = NM == 4
                ? (fabs(a1) <= 1.0 + kInsideTol && fabs(a2) <= 1.0 + kInsideTol)
                : (a1 >= -kInsideTol && a2 >= -kInsideTol && a1 + a2 <= 1.0 + kInsideTol);
            if (!inside) continue;
            owner = kn;
            m1 = a1;
            m2 = a2;
          }
          if (owner < 0) continue;
          taken[q >> 5] |= 1u << (q & 31);
          got[owner] += 1;
          const double j00 = smap.c1u + smap.c3u * eta, j01 = smap.c2u + smap.c3u * xi;
          const double j10 = smap.c1v + smap.c3v * eta, j11 = smap.c2v + smap.c3v * xi;
          const double W = wq * fabs(j00 * j11 - j01 * j10);
          // dual LMs: Phi_a = A N_s per point, or (NODAL) G = sum W N_s N_m^T
          // and H = sum W N_s N_s^T in the nodal basis, turned into A G, A H
          // once the chunk is done
          double Ns[4], Nm[4], Phi[4];
          shape_fn<NS>(xi, eta, Ns);
          shape_fn<NM>(m1, m2, Nm);
#pragma unroll
          for (int a = 0; a < NS; ++a) {
            double v = Ns[a];
            if (DUAL && !NODAL) {
              v = 0.0;
#pragma unroll
              for (int c = 0; c < NS; ++c) v = fma(Phi_c[a][c], Ns[c], v);
            }
            Phi[a] = W * v;
          }
          double* mo = Mblk + 16 * (c0 + owner);
#pragma unroll
          for (int a = 0; a < NS; ++a)
#pragma unroll
            for (int l = 0; l < NM; ++l) mo[4 * a + l] = fma(Phi[a], Nm[l], mo[4 * a + l]);
          if (SEG) {
            double* dout = Dblk + 16 * (c0 + owner);
#pragma unroll
            for (int a = 0; a < NS; ++a)
#pragma unroll
              for (int b = 0; b < NS; ++b) dout[4 * a + b] = fma(Phi[a], Ns[b], dout[4 * a + b]);
          }
        }
        if (DUAL && NODAL)   // every point of this chunk's pairs is in: M = A G, D = A H
          for (int k = 0; k < kc; ++k) {
            if (got[k] == 0) continue;
            double* mo = Mblk + 16 * (c0 + k);
            double G[4][4];
#pragma unroll
            for (int c = 0; c < NS; ++c)
#pragma unroll
              for (int l = 0; l < NM; ++l) G[c][l] = mo[4 * c + l];
#pragma unroll
            for (int a = 0; a < NS; ++a)
#pragma unroll
              for (int l = 0; l < NM; ++l) {
                double v = 0.0;
#pragma unroll
                for (int c = 0; c < NS; ++c) v = fma(Phi_c[a][c], G[c][l], v);
                mo[4 * a + l] = v;
              }
            if (SEG) {
              double* dout = Dblk + 16 * (c0 + k);
#pragma unroll
              for (int c = 0; c < NS; ++c)
#pragma unroll
                for (int b = 0; b < NS; ++b) G[c][b] = dout[4 * c + b];
#pragma unroll
              for (int a = 0; a < NS; ++a)
#pragma unroll
                for (int b = 0; b < NS; ++b) {
                  double v = 0.0;
#pragma unroll
                  for (int c = 0; c < NS; ++c) v = fma(Phi_c[a][c], G[c][b], v);
                  dout[4 * a + b] = v;
                }
            }
          }
      }
      for (int k = 0; k < kc; ++k) {
        flag[c0 + k] = got[k] > 0 ? 1 : 0;
        n_live += got[k] > 0 ? 1 : 0;
        n_gp += (unsigned long long)got[k];
      }
    }
  }
  block_count_add(&st->nonempty, n_live);
  block_count_add(&st->gauss_points, n_gp);
}

template <int NS, int NM>
void launch_nsnm(mortar_ctx* c, const RunParams& rp, unsigned grid) {
  const bool seg = rp.d_domain == 1, dual = rp.lm == 1;
  auto go = [&](auto kern) {
    kern<<<grid, kThreads, 0, c->stream>>>(c->pair_off.as<int64_t>(), c->pairs_m.as<int32_t>(), c->srec.as<double>(),
                                           c->xm.as<double>(), c->conn_m.as<int32_t>(), c->rule_1d.as<double>(),
                                           c->rule_1d_n, c->Es, c->Mblk.as<double>(), c->Dblk.as<double>(),
                                           c->flag.as<uint8_t>(), c->dstat.as<DevStatus>());
  };
  const bool nodal = c->rule_1d_n >= 6;
  if (seg && dual && nodal) go(k_integrate_elembased<NS, NM, true, true, true>);
  else if (seg && dual) go(k_integrate_elembased<NS, NM, true, true, false>);
  else if (seg) go(k_integrate_elembased<NS, NM, true, false, false>);
  else if (dual && nodal) go(k_integrate_elembased<NS, NM, false, true, true>);
  else if (dual) go(k_integrate_elembased<NS, NM, false, true, false>);
  else go(k_integrate_elembased<NS, NM, false, false, false>);
}

}  // namespace

// n-point Gauss-Legendre rule on [-1, 1] (points ascending, then weights):
// roots of P_n by Newton from cos(pi (i + 3/4) / (n + 1/2)), P_n and P_n' by
// the three-term recurrence, weights 2 / ((1 - x^2) P_n'(x)^2).
int upload_gauss_legendre(mortar_ctx* c, int n) {
  std::vector<double> h(2 * (size_t)n);
  const double pi = std::acos(-1.0);
  for (int i = 0; i < n; ++i) {
    double x = std::cos(pi * (n - i - 0.25) / (n + 0.5));   // ascending order
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double pk = 1.0, pk1 = 0.0;   // P_k, P_{k-1}
      for (int k = 1; k <= n; ++k) {
        const double pn = ((2.0 * k - 1.0) * x * pk - (k - 1.0) * pk1) / k;
        pk1 = pk;
        pk = pn;
      }
      dp = n * (x * pk - pk1) / (x * x - 1.0);
      const double dx = pk / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    double pk = 1.0, pk1 = 0.0;
    for (int k = 1; k <= n; ++k) {
      const double pn = ((2.0 * k - 1.0) * x * pk - (k - 1.0) * pk1) / k;
      pk1 = pk;
      pk = pn;
    }
    dp = n * (x * pk - pk1) / (x * x - 1.0);
    h[i] = x;
    h[n + i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  int r = buf_reserve(c->rule_1d, h.size() * sizeof(double));
  if (r != MORTAR_OK) return r;
  if (cudaMemcpy(c->rule_1d.p, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return MORTAR_ERR_CUDA;
  }
  c->rule_1d_n = n;
  return MORTAR_OK;
}

void launch_integrate_element_based(mortar_ctx* c, const RunParams& rp) {
  if (c->Es == 0) return;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_integrate_elembased<4, 4, false, true, false>, kThreads, 0);
  if (per_sm < 1) per_sm = 1;
  const int64_t need = (c->Es + kThreads - 1) / kThreads;
  const unsigned grid = (unsigned)std::min<int64_t>(need, (int64_t)c->n_sm * per_sm * 8);
  if (c->nen_s == 4 && c->nen_m == 4) launch_nsnm<4, 4>(c, rp, grid);
  else if (c->nen_s == 4 && c->nen_m == 3) launch_nsnm<4, 3>(c, rp, grid);
  else if (c->nen_s == 3 && c->nen_m == 4) launch_nsnm<3, 4>(c, rp, grid);
  else launch_nsnm<3, 3>(c, rp, grid);
}

}  // namespace mortar
