// Element-level precomputation and the per-interface search grid.
//
//  * Slave elements (one thread each): auxiliary plane x0, n0 and in-plane
//    basis t1, t2 (Sec. 2.3, Fig. 1), projected slave polygon and its bilinear
//    map, clipping tolerances, LM coefficients A (standard: identity; dual:
//    A = Dh Me^-1, biorthogonal to N, Sec. 2.2) and the element-domain D
//    block; inflated bounding box and diameter for the search.
//  * Master elements: inflated bounding box and diameter.
//  * Search grid per interface (Sec. 3.5): bounding box of the interface,
//    minimal bin size beta_min = (1 + 1e-9) max diameter + 2 delta (+ the
//    velocity margin of moving interfaces), box
//    expanded by beta_min, n_d = max(1, floor(L_d / beta_min)) bins per
//    direction (bins grow by 1.25x while an interface would exceed its bin
//    capacity).
#include <cfloat>

#include "context.h"
#include "quadratic.cuh"

namespace mortar {

namespace {

constexpr int kThreads = 128;

struct V3 {
  double x, y, z;
};
__device__ __forceinline__ V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Surface Jacobian |x,xi x x,eta| of an element at (xi, eta).
template <int NEN>
__device__ double surface_jac(const V3* X, double xi, double eta) {
  V3 g1, g2;
  if constexpr (NEN == 4) {
    const double em = 0.25 * (1.0 - eta), ep = 0.25 * (1.0 + eta);
    const double xm = 0.25 * (1.0 - xi), xp = 0.25 * (1.0 + xi);
    g1 = {-em * X[0].x + em * X[1].x + ep * X[2].x - ep * X[3].x,
          -em * X[0].y + em * X[1].y + ep * X[2].y - ep * X[3].y,
          -em * X[0].z + em * X[1].z + ep * X[2].z - ep * X[3].z};
    g2 = {-xm * X[0].x - xp * X[1].x + xp * X[2].x + xm * X[3].x,
          -xm * X[0].y - xp * X[1].y + xp * X[2].y + xm * X[3].y,
          -xm * X[0].z - xp * X[1].z + xp * X[2].z + xm * X[3].z};
  } else {
    g1 = sub(X[1], X[0]);
    g2 = sub(X[2], X[0]);
  }
  V3 n = cross(g1, g2);
  return sqrt(dot(n, n));
}

// Element rule point k: 3x3 Gauss-Legendre (quad4, weights sum 4) or the
// 7-point triangle rule (tri3, weights sum 1/2).
template <int NEN>
__device__ __forceinline__ void elem_point(int k, double& xi, double& eta, double& w) {
  if constexpr (NEN == 4) {
    const double g = 0.7745966692414834;
    const double p[3] = {-g, 0.0, g};
    const double ww[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
    xi = p[k / 3];
    eta = p[k % 3];
    w = ww[k / 3] * ww[k % 3];
  } else {
    tri7_point(k, xi, eta, w);
    w *= 0.5;
  }
}

// Auxiliary plane and clip window of one linear element (or linear
// sub-element of a quadratic one) with nodes X: writes the record fields x0,
// t1, t2, n0, the projected map, the window polygon, the tolerances, the
// orientation flag, the inverse of the affine part and the affine flag, marks
// a degenerate element (eps_in < 0); returns |g1 x g2| at the centre and the
// diameter h, and the centre tangents g1, g2.
template <int NS>
__device__ __forceinline__ void slave_record(const V3* X, const RunParams& rp, double* r, double& ln, double& h,
                                             V3& g1, V3& g2, bool& degenerate) {
  // ---- auxiliary plane at the element centre
  V3 x0;
  if constexpr (NS == 4) {
    x0 = {0.25 * ((X[0].x + X[1].x) + (X[2].x + X[3].x)), 0.25 * ((X[0].y + X[1].y) + (X[2].y + X[3].y)),
          0.25 * ((X[0].z + X[1].z) + (X[2].z + X[3].z))};
    g1 = {0.25 * ((X[1].x - X[0].x) + (X[2].x - X[3].x)), 0.25 * ((X[1].y - X[0].y) + (X[2].y - X[3].y)),
          0.25 * ((X[1].z - X[0].z) + (X[2].z - X[3].z))};
    g2 = {0.25 * ((X[2].x - X[1].x) + (X[3].x - X[0].x)), 0.25 * ((X[2].y - X[1].y) + (X[3].y - X[0].y)),
          0.25 * ((X[2].z - X[1].z) + (X[3].z - X[0].z))};
  } else {
    const double t = 1.0 / 3.0;
    x0 = {t * (X[0].x + X[1].x + X[2].x), t * (X[0].y + X[1].y + X[2].y), t * (X[0].z + X[1].z + X[2].z)};
    g1 = sub(X[1], X[0]);
    g2 = sub(X[2], X[0]);
  }
  V3 n = cross(g1, g2);
  ln = sqrt(dot(n, n));
  const V3 n0 = {n.x / ln, n.y / ln, n.z / ln};
  const V3 ed = sub(X[1], X[0]);
  const double en = dot(ed, n0);
  const V3 ep = {ed.x - en * n0.x, ed.y - en * n0.y, ed.z - en * n0.z};
  const double le = sqrt(dot(ep, ep));
  const V3 t1 = {ep.x / le, ep.y / le, ep.z / le};
  const V3 t2 = cross(n0, t1);
  r[SR_X0] = x0.x; r[SR_X0 + 1] = x0.y; r[SR_X0 + 2] = x0.z;
  r[SR_T1] = t1.x; r[SR_T1 + 1] = t1.y; r[SR_T1 + 2] = t1.z;
  r[SR_T2] = t2.x; r[SR_T2 + 1] = t2.y; r[SR_T2 + 2] = t2.z;
  r[SR_N0] = n0.x; r[SR_N0 + 1] = n0.y; r[SR_N0 + 2] = n0.z;
  // ---- projected slave polygon
  double pu[4] = {0, 0, 0, 0}, pv[4] = {0, 0, 0, 0};
  for (int a = 0; a < NS; ++a) {
    const V3 d = sub(X[a], x0);
    pu[a] = dot(d, t1);
    pv[a] = dot(d, t2);
  }
  const PlaneMap pm = plane_map<NS>(pu, pv);
  r[SR_C + 0] = pm.c0u; r[SR_C + 1] = pm.c0v; r[SR_C + 2] = pm.c1u; r[SR_C + 3] = pm.c1v;
  r[SR_C + 4] = pm.c2u; r[SR_C + 5] = pm.c2v; r[SR_C + 6] = pm.c3u; r[SR_C + 7] = pm.c3v;
  double area2 = 0.0;
  for (int a = 0; a < NS; ++a) area2 += cross2(pu[a], pv[a], pu[(a + 1) % NS], pv[(a + 1) % NS]);
  for (int a = 0; a < NS; ++a) {
    const int src = area2 < 0.0 ? NS - 1 - a : a;
    r[SR_PS + 2 * a] = pu[src];
    r[SR_PS + 2 * a + 1] = pv[src];
  }
  if (NS == 3) { r[SR_PS + 6] = 0.0; r[SR_PS + 7] = 0.0; }
  r[SR_REV] = area2 < 0.0 ? 1.0 : 0.0;
  {
    const double det = pm.c1u * pm.c2v - pm.c2u * pm.c1v;
    const double id = 1.0 / det;
    r[SR_BINV + 0] = pm.c2v * id;
    r[SR_BINV + 1] = -pm.c2u * id;
    r[SR_BINV + 2] = -pm.c1v * id;
    r[SR_BINV + 3] = pm.c1u * id;
    r[SR_AFF] = (NS == 3 || map_is_affine(pm)) ? 1.0 : 0.0;
    r[SR_AFF + 1] = 0.0; r[SR_AFF + 2] = 0.0; r[SR_AFF + 3] = 0.0;
  }
  // ---- tolerances: diameter and projected area
  double h2 = 0.0;
  for (int a = 0; a < NS; ++a)
    for (int b = a + 1; b < NS; ++b) {
      const V3 d = sub(X[a], X[b]);
      h2 = fmax(h2, dot(d, d));
    }
  h = sqrt(h2);
  const double em = rp.merge_tol_rel * h;
  r[SR_EPSIN] = rp.clip_tol_rel * h * h;
  r[SR_EPSM2] = em * em;
  r[SR_EPSA] = rp.area_tol_rel * (0.5 * fabs(area2));
  // an inverted (folded) quad4: its projected corners do not form a convex
  // polygon of one orientation, and its Jacobian changes sign inside
  bool folded = false;
  if constexpr (NS == 4) {
    for (int a = 0; a < 4; ++a) {
      const int a1 = (a + 1) & 3, a2 = (a + 2) & 3;
      const double c = cross2(pu[a1] - pu[a], pv[a1] - pv[a], pu[a2] - pu[a1], pv[a2] - pv[a1]);
      folded |= !(c * area2 > 0.0);
    }
  }
  degenerate = !(ln > 0.0) || !(le > 0.0) || !(fabs(area2) > 0.0) || !isfinite(h) || folded;
  if (degenerate) r[SR_EPSIN] = -1.0;   // marks the element; its pairs integrate to nothing
}

// An element with a non-finite node coordinate gets an all-NaN box: every
// box-overlap test (closed <= compares) is false for it, so it has no pairs,
// and the grid's min / max reductions (fmin / fmax) skip it.
__device__ __forceinline__ void set_nan_box(double* b) {
  const double q = __longlong_as_double(0x7ff8000000000000LL);
  for (int k = 0; k < 7; ++k) b[k] = q;
}

template <int NS>
__global__ void __launch_bounds__(kThreads) k_slave_precompute(
    const double* __restrict__ xs, const int32_t* __restrict__ conn, int64_t Es, RunParams rp,
    double* __restrict__ srec, double* __restrict__ De, double* __restrict__ box, DevStatus* st) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool degenerate = false, bad = false;
  if (e < Es) {
    V3 X[4];
    for (int a = 0; a < NS; ++a) {
      const int64_t n = conn[NS * e + a];
      X[a] = {xs[3 * n], xs[3 * n + 1], xs[3 * n + 2]};
      bad |= !(isfinite(X[a].x) && isfinite(X[a].y) && isfinite(X[a].z));
    }
    double* r = srec + (int64_t)SR_STRIDE * e;
    double ln = 0.0, h = 0.0;
    V3 g1, g2;
    slave_record<NS>(X, rp, r, ln, h, g1, g2, degenerate);
    // ---- element integrals Me[a][b] = int N_a N_b, Dh[a] = int N_a (surface measure)
    // An element whose bilinear term is negligible (parallelogram, any tri3) has a
    // constant surface Jacobian J0, and then Me = J0 Mref, Dh = J0 dref exactly.
    double Me[4][4], Dh[4];
    for (int a = 0; a < 4; ++a) {
      Dh[a] = 0.0;
      for (int b = 0; b < 4; ++b) Me[a][b] = 0.0;
    }
    bool flat_jac = NS == 3;
    if constexpr (NS == 4) {
      const V3 d3 = {0.25 * ((X[0].x - X[1].x) + (X[2].x - X[3].x)), 0.25 * ((X[0].y - X[1].y) + (X[2].y - X[3].y)),
                     0.25 * ((X[0].z - X[1].z) + (X[2].z - X[3].z))};
      const double s3 = fabs(d3.x) + fabs(d3.y) + fabs(d3.z);
      const double s12 = fabs(g1.x) + fabs(g1.y) + fabs(g1.z) + fabs(g2.x) + fabs(g2.y) + fabs(g2.z);
      flat_jac = s3 <= 1e-15 * s12;
    }
    if (flat_jac) {
      if constexpr (NS == 4) {
        const double J0 = ln;   // |g1 x g2| at the centre = the constant Jacobian
        const double m4 = J0 * (4.0 / 9.0), m2 = J0 * (2.0 / 9.0), m1 = J0 * (1.0 / 9.0);
        for (int a = 0; a < 4; ++a) {
          Dh[a] = J0;
          for (int b = 0; b < 4; ++b) {
            const int dd = (a - b + 4) % 4;
            Me[a][b] = dd == 0 ? m4 : (dd == 2 ? m1 : m2);
          }
        }
      } else {
        const double J0 = ln;   // twice the triangle area
        for (int a = 0; a < 3; ++a) {
          Dh[a] = J0 * (1.0 / 6.0);
          for (int b = 0; b < 3; ++b) Me[a][b] = J0 * (a == b ? 1.0 / 12.0 : 1.0 / 24.0);
        }
      }
    } else {
      constexpr int nq = NS == 4 ? 9 : 7;
      for (int q = 0; q < nq; ++q) {
        double xi, eta, w;
        elem_point<NS>(q, xi, eta, w);
        double N[4];
        shape_fn<NS>(xi, eta, N);
        const double wj = w * surface_jac<NS>(X, xi, eta);
        for (int a = 0; a < NS; ++a) {
          const double wn = wj * N[a];
          Dh[a] += wn;
          for (int b = 0; b < NS; ++b) Me[a][b] += wn * N[b];
        }
      }
    }
    // ---- LM coefficients: standard A = I; dual A = Dh Me^-1 (Me A^T = diag(Dh))
    double A[4][4];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) A[a][b] = a == b ? 1.0 : 0.0;
    if (rp.lm == 1 && !degenerate && flat_jac) {
      // constant Jacobian: Me = J0 Mref, Dh = J0 dref, so A = dref Mref^-1 is a
      // constant -- the tensor product of the 1D duals 2 N_1 - N_2 on a
      // parallelogram (4 on the diagonal, -2 for edge neighbours, 1 across),
      // Phi_a = 3 N_a - N_b - N_c on a triangle
      for (int a = 0; a < NS; ++a)
        for (int b = 0; b < NS; ++b) {
          const int dd = (a - b + NS) % NS;
          A[a][b] = NS == 4 ? (dd == 0 ? 4.0 : (dd == 2 ? 1.0 : -2.0)) : (dd == 0 ? 3.0 : -1.0);
        }
    } else if (rp.lm == 1 && !degenerate) {
      double K[4][4], B[4][4];
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          K[a][b] = Me[a][b];
          B[a][b] = (a == b && a < NS) ? Dh[a] : 0.0;
        }
      for (int c = 0; c < NS; ++c) {   // Gauss-Jordan with partial pivoting
        int piv = c;
        for (int rr = c + 1; rr < NS; ++rr)
          if (fabs(K[rr][c]) > fabs(K[piv][c])) piv = rr;
        if (piv != c)
          for (int k = 0; k < 4; ++k) {
            double t = K[c][k]; K[c][k] = K[piv][k]; K[piv][k] = t;
            t = B[c][k]; B[c][k] = B[piv][k]; B[piv][k] = t;
          }
        const double inv = 1.0 / K[c][c];
        for (int k = 0; k < 4; ++k) { K[c][k] *= inv; B[c][k] *= inv; }
        for (int rr = 0; rr < NS; ++rr) {
          if (rr == c) continue;
          const double f = K[rr][c];
          for (int k = 0; k < 4; ++k) {
            K[rr][k] -= f * K[c][k];
            B[rr][k] -= f * B[c][k];
          }
        }
      }
      for (int a = 0; a < NS; ++a)
        for (int b = 0; b < NS; ++b) A[a][b] = B[b][a];
    }
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) r[SR_A + 4 * a + b] = A[a][b];
    // ---- element-domain D: De = sum_q w J Phi_a N_b = A Me; with dual LMs
    //      this is diag(Dh) exactly (biorthogonality), stored as such
    double* d = De + 16 * e;
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        double v = 0.0;
        if (rp.lm == 1) {
          v = a == b ? Dh[a] : 0.0;
        } else {
          for (int c = 0; c < NS; ++c) v += A[a][c] * Me[c][b];
        }
        d[4 * a + b] = (a < NS && b < NS) ? v : 0.0;
      }
    // ---- search box (delta-inflated) and diameter
    double lo[3] = {X[0].x, X[0].y, X[0].z}, hi[3] = {X[0].x, X[0].y, X[0].z};
    for (int a = 1; a < NS; ++a) {
      lo[0] = fmin(lo[0], X[a].x); hi[0] = fmax(hi[0], X[a].x);
      lo[1] = fmin(lo[1], X[a].y); hi[1] = fmax(hi[1], X[a].y);
      lo[2] = fmin(lo[2], X[a].z); hi[2] = fmax(hi[2], X[a].z);
    }
    double* b = box + 8 * e;
    for (int k = 0; k < 3; ++k) {
      b[k] = lo[k] - rp.delta;
      b[3 + k] = hi[k] + rp.delta;
    }
    b[6] = h;
    b[7] = 0.0;
    if (bad) {
      set_nan_box(b);
      r[SR_EPSIN] = -1.0;
      degenerate = true;
    }
  }
  block_count_add(&st->degenerate, degenerate ? 1ull : 0ull);
  block_count_add(&st->nonfinite, bad ? 1ull : 0ull);
}

// Quadratic slave element (tri6, quad8; standard LMs): the records of its
// four linear sub-elements (record 4 e + k; the piecewise flat approximation
// of the slave surface, Sec. 2.3, whose clip windows and auxiliary planes the
// pairs use), the element-domain D with the quadratic isoparametric Jacobian
// (3x3 Gauss-Legendre on quad8, the 7-point rule on tri6; 8 x 8 block per
// element) and the search box over all its nodes.
template <int NP>
__global__ void __launch_bounds__(kThreads) k_slave_precompute_quadratic(
    const double* __restrict__ xs, const int32_t* __restrict__ conn, int64_t Es, RunParams rp,
    double* __restrict__ srec, double* __restrict__ De, double* __restrict__ box, DevStatus* st) {
  constexpr int NSUB = NP == 8 ? 4 : 3;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool degenerate = false, bad = false;
  if (e < Es) {
    V3 X[8];
    for (int a = 0; a < NP; ++a) {
      const int64_t n = conn[(int64_t)NP * e + a];
      X[a] = {xs[3 * n], xs[3 * n + 1], xs[3 * n + 2]};
      bad |= !(isfinite(X[a].x) && isfinite(X[a].y) && isfinite(X[a].z));
    }
    V3 xc = {0.0, 0.0, 0.0};
    if constexpr (NP == 8) {   // x(0, 0): corners weigh -1/4, mid-sides 1/2
      for (int a = 0; a < 8; ++a) {
        const double w = a < 4 ? -0.25 : 0.5;
        xc = {xc.x + w * X[a].x, xc.y + w * X[a].y, xc.z + w * X[a].z};
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      V3 Xs[4];
#pragma unroll
      for (int j = 0; j < NSUB; ++j) {
        const int a = sub_node<NP>(k, j);
        Xs[j] = a < 0 ? xc : X[a];
      }
      double* r = srec + (int64_t)SR_STRIDE * (4 * e + k);
      double ln = 0.0, h = 0.0;
      V3 g1, g2;
      bool dg = false;
      slave_record<NSUB>(Xs, rp, r, ln, h, g1, g2, dg);
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) r[SR_A + 4 * a + b] = a == b ? 1.0 : 0.0;
      degenerate |= dg;
      if (bad) r[SR_EPSIN] = -1.0;
    }
    if (degenerate)   // a degenerate sub-element makes the whole element contribute nothing
      for (int k = 0; k < 4; ++k) srec[(int64_t)SR_STRIDE * (4 * e + k) + SR_EPSIN] = -1.0;
    // element-domain D, standard LMs: De[a][b] = sum_q w J N_a N_b
    double D[8][8];
    for (int a = 0; a < 8; ++a)
      for (int b = 0; b < 8; ++b) D[a][b] = 0.0;
    constexpr int nq = NP == 8 ? 9 : 7;
    for (int q = 0; q < nq; ++q) {
      double xi, eta, w;
      elem_point<NP == 8 ? 4 : 3>(q, xi, eta, w);
      double N[8], dN[8][2];
      shape_quadratic<NP>(xi, eta, N);
      shape_quadratic_grad<NP>(xi, eta, dN);
      V3 g1 = {0.0, 0.0, 0.0}, g2 = g1;
      for (int a = 0; a < NP; ++a) {
        g1 = {g1.x + dN[a][0] * X[a].x, g1.y + dN[a][0] * X[a].y, g1.z + dN[a][0] * X[a].z};
        g2 = {g2.x + dN[a][1] * X[a].x, g2.y + dN[a][1] * X[a].y, g2.z + dN[a][1] * X[a].z};
      }
      const V3 nq3 = cross(g1, g2);
      const double wj = w * sqrt(dot(nq3, nq3));
      for (int a = 0; a < NP; ++a)
        for (int b = 0; b < NP; ++b) D[a][b] += wj * N[a] * N[b];
    }
    double* d = De + 64 * e;
    for (int a = 0; a < 8; ++a)
      for (int b = 0; b < 8; ++b) d[8 * a + b] = D[a][b];
    // search box (delta-inflated) and diameter over all nodes
    double lo[3] = {X[0].x, X[0].y, X[0].z}, hi[3] = {X[0].x, X[0].y, X[0].z};
    for (int a = 1; a < NP; ++a) {
      lo[0] = fmin(lo[0], X[a].x); hi[0] = fmax(hi[0], X[a].x);
      lo[1] = fmin(lo[1], X[a].y); hi[1] = fmax(hi[1], X[a].y);
      lo[2] = fmin(lo[2], X[a].z); hi[2] = fmax(hi[2], X[a].z);
    }
    double h2 = 0.0;
    for (int a = 0; a < NP; ++a)
      for (int b = a + 1; b < NP; ++b) {
        const V3 dd = sub(X[a], X[b]);
        h2 = fmax(h2, dot(dd, dd));
      }
    double* b = box + 8 * e;
    for (int k = 0; k < 3; ++k) {
      b[k] = lo[k] - rp.delta;
      b[3 + k] = hi[k] + rp.delta;
    }
    b[6] = sqrt(h2);
    b[7] = 0.0;
    if (bad) {
      set_nan_box(b);
      degenerate = true;
    }
  }
  block_count_add(&st->degenerate, degenerate ? 1ull : 0ull);
  block_count_add(&st->nonfinite, bad ? 1ull : 0ull);
}

template <int NM>
__global__ void __launch_bounds__(kThreads) k_master_boxes(const double* __restrict__ xm,
                                                            const int32_t* __restrict__ conn, int64_t Em,
                                                            double delta, double* __restrict__ box,
                                                            double* __restrict__ nrm, DevStatus* st) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  if (e < Em) {
  V3 X[4];
  for (int a = 0; a < NM; ++a) {
    const int64_t n = conn[NM * e + a];
    X[a] = {xm[3 * n], xm[3 * n + 1], xm[3 * n + 2]};
    bad |= !(isfinite(X[a].x) && isfinite(X[a].y) && isfinite(X[a].z));
  }
  double lo[3] = {X[0].x, X[0].y, X[0].z}, hi[3] = {X[0].x, X[0].y, X[0].z};
  double h2 = 0.0;
  for (int a = 1; a < NM; ++a) {
    lo[0] = fmin(lo[0], X[a].x); hi[0] = fmax(hi[0], X[a].x);
    lo[1] = fmin(lo[1], X[a].y); hi[1] = fmax(hi[1], X[a].y);
    lo[2] = fmin(lo[2], X[a].z); hi[2] = fmax(hi[2], X[a].z);
  }
  for (int a = 0; a < NM; ++a)
    for (int b = a + 1; b < NM; ++b) {
      const V3 d = sub(X[a], X[b]);
      h2 = fmax(h2, dot(d, d));
    }
  double* b = box + 8 * e;
  for (int k = 0; k < 3; ++k) {
    b[k] = lo[k] - delta;
    b[3 + k] = hi[k] + delta;
  }
  b[6] = sqrt(h2);
  b[7] = 0.0;
  if (nrm) {   // unit normal at the element centre (facing test)
    V3 g1, g2;
    if constexpr (NM == 4) {
      const V3 d10 = sub(X[1], X[0]), d23 = sub(X[2], X[3]), d21 = sub(X[2], X[1]), d30 = sub(X[3], X[0]);
      g1 = {0.25 * (d10.x + d23.x), 0.25 * (d10.y + d23.y), 0.25 * (d10.z + d23.z)};
      g2 = {0.25 * (d21.x + d30.x), 0.25 * (d21.y + d30.y), 0.25 * (d21.z + d30.z)};
    } else {
      g1 = sub(X[1], X[0]);
      g2 = sub(X[2], X[0]);
    }
    const V3 n = {g1.y * g2.z - g1.z * g2.y, g1.z * g2.x - g1.x * g2.z, g1.x * g2.y - g1.y * g2.x};
    const double l = sqrt(dot(n, n));
    nrm[3 * e] = n.x / l;
    nrm[3 * e + 1] = n.y / l;
    nrm[3 * e + 2] = n.z / l;
  }
  if (bad) set_nan_box(b);
  }
  block_count_add(&st->nonfinite, bad ? 1ull : 0ull);
}

// One block per chunk: min of lo, max of hi, max of h over its elements.
__global__ void __launch_bounds__(256) k_chunk_reduce(const Chunk* __restrict__ chunks,
                                                      const double* __restrict__ box_s,
                                                      const double* __restrict__ box_m,
                                                      double* __restrict__ red) {
  const Chunk c = chunks[blockIdx.x];
  const double* box = c.side == 0 ? box_s : box_m;
  double v[7] = {DBL_MAX, DBL_MAX, DBL_MAX, -DBL_MAX, -DBL_MAX, -DBL_MAX, 0.0};
  for (int64_t e = c.begin + threadIdx.x; e < c.end; e += blockDim.x) {
    const double* b = box + 8 * e;
    for (int k = 0; k < 3; ++k) {
      v[k] = fmin(v[k], b[k]);
      v[3 + k] = fmax(v[3 + k], b[3 + k]);
    }
    v[6] = fmax(v[6], b[6]);
  }
  __shared__ double sh[8][7];
  for (int k = 0; k < 7; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_down_sync(0xffffffffu, x, o);
      x = k < 3 ? fmin(x, y) : fmax(x, y);
    }
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][k] = x;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    const int k = threadIdx.x;
    double x = sh[0][k];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) x = k < 3 ? fmin(x, sh[w][k]) : fmax(x, sh[w][k]);
    red[8 * blockIdx.x + k] = x;
  }
}

// One block per interface: combine its chunks and set up the bin grid.
__global__ void __launch_bounds__(256) k_grid_params(const int32_t* __restrict__ chunk_ptr,
                                                     const double* __restrict__ red,
                                                     const int64_t* __restrict__ bin_cap_off, double delta,
                                                     double margin, GridParams* __restrict__ grid) {
  const int i = blockIdx.x;
  const int32_t c0 = chunk_ptr[i], c1 = chunk_ptr[i + 1];
  double v[7] = {DBL_MAX, DBL_MAX, DBL_MAX, -DBL_MAX, -DBL_MAX, -DBL_MAX, 0.0};
  for (int32_t c = c0 + threadIdx.x; c < c1; c += blockDim.x)
    for (int k = 0; k < 7; ++k) v[k] = k < 3 ? fmin(v[k], red[8 * c + k]) : fmax(v[k], red[8 * c + k]);
  __shared__ double sh[8][7];
  for (int k = 0; k < 7; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_down_sync(0xffffffffu, x, o);
      x = k < 3 ? fmin(x, y) : fmax(x, y);
    }
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][k] = x;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int k = 0; k < 7; ++k)
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) sh[0][k] = k < 3 ? fmin(sh[0][k], sh[w][k]) : fmax(sh[0][k], sh[w][k]);
  GridParams g;
  const int64_t cap = bin_cap_off[i + 1] - bin_cap_off[i];
  if (c1 <= c0 || !(sh[0][0] <= sh[0][3])) {   // empty interface
    for (int k = 0; k < 3; ++k) { g.org[k] = 0.0; g.beta[k] = 1.0; g.nb[k] = 1; }
  } else {
    double beta_min = (1.0 + 1e-9) * sh[0][6] + 2.0 * delta + margin;
    if (!(beta_min > 0.0)) beta_min = 1.0;
    for (int attempt = 0; attempt < 200; ++attempt) {
      int64_t tot = 1;
      for (int k = 0; k < 3; ++k) {
        g.org[k] = sh[0][k] - beta_min;
        const double L = (sh[0][3 + k] + beta_min) - g.org[k];
        double nbd = floor(L / beta_min);
        nbd = fmin(fmax(nbd, 1.0), 1.0e6);
        g.nb[k] = (int32_t)nbd;
        g.beta[k] = L / nbd;
        tot *= g.nb[k];
      }
      if (tot <= cap) break;
      beta_min *= 1.25;
    }
  }
  g.pad = 0;
  g.n_bins = (int64_t)g.nb[0] * g.nb[1] * g.nb[2];
  g.bin_off = 0;
  grid[i] = g;
}

// Exclusive scan of n_bins over interfaces (single block); total -> status.
__global__ void __launch_bounds__(1024) k_bin_offsets(GridParams* __restrict__ grid, int32_t n_if,
                                                      int64_t bin_cap, DevStatus* st) {
  __shared__ int64_t warp_tot[32];
  __shared__ int64_t carry_s;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int b0 = 0; b0 < n_if; b0 += 1024) {
    const int i = b0 + threadIdx.x;
    const int64_t v = i < n_if ? grid[i].n_bins : 0;
    int64_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
      const int64_t t = warp_tot[lane];
      int64_t ti = t;
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, ti, o);
        if (lane >= o) ti += y;
      }
      warp_tot[lane] = ti - t;
    }
    __syncthreads();
    const int64_t excl = inc - v + warp_tot[w] + carry_s;
    if (i < n_if) grid[i].bin_off = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry_s = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    st->n_bins = (unsigned long long)carry_s;
    if (carry_s > bin_cap) st->over_bins = (unsigned long long)carry_s;
  }
}

}  // namespace

RunParams run_params(const mortar_ctx* c) {
  RunParams rp;
  rp.lm = c->opt.lm;
  rp.d_domain = c->opt.d_domain;
  rp.newton_max_iter = c->opt.newton_max_iter;
  rp.pad = 0;
  rp.newton_tol = c->opt.newton_tol;
  rp.clip_tol_rel = c->opt.clip_tol_rel;
  rp.merge_tol_rel = c->opt.merge_tol_rel;
  rp.area_tol_rel = c->opt.area_tol_rel;
  rp.delta = c->opt.search_inflation;
  rp.bin_margin = c->opt.bin_margin;
  rp.integration = c->opt.integration;
  rp.rule_n = c->opt.element_rule_n;
  rp.facing = c->opt.facing_test;
  rp.watchdog_us = c->watchdog_us;
  return rp;
}

void launch_slave_precompute(mortar_ctx* c, const RunParams& rp) {
  if (c->Es == 0) return;
  const unsigned g = (unsigned)((c->Es + kThreads - 1) / kThreads);
  DevStatus* st = c->dstat.as<DevStatus>();
  if (c->nen_s == 8 || c->nen_s == 6) {
    auto kern = c->nen_s == 8 ? k_slave_precompute_quadratic<8> : k_slave_precompute_quadratic<6>;
    kern<<<g, kThreads, 0, c->stream>>>(c->xs.as<double>(), c->conn_s.as<int32_t>(), c->Es, rp, c->srec.as<double>(),
                                        c->De.as<double>(), c->box_s.as<double>(), st);
    return;
  }
  if (c->nen_s == 4)
    k_slave_precompute<4><<<g, kThreads, 0, c->stream>>>(c->xs.as<double>(), c->conn_s.as<int32_t>(), c->Es, rp,
                                                          c->srec.as<double>(), c->De.as<double>(),
                                                          c->box_s.as<double>(), st);
  else
    k_slave_precompute<3><<<g, kThreads, 0, c->stream>>>(c->xs.as<double>(), c->conn_s.as<int32_t>(), c->Es, rp,
                                                          c->srec.as<double>(), c->De.as<double>(),
                                                          c->box_s.as<double>(), st);
}

void launch_slave_precompute_raw(const double* xs, const int32_t* conn_s, int64_t Es, int nen_s,
                                 const RunParams& rp, double* srec, double* De, double* box, DevStatus* st,
                                 cudaStream_t stream) {
  if (Es == 0) return;
  const unsigned g = (unsigned)((Es + kThreads - 1) / kThreads);
  if (nen_s == 4)
    k_slave_precompute<4><<<g, kThreads, 0, stream>>>(xs, conn_s, Es, rp, srec, De, box, st);
  else
    k_slave_precompute<3><<<g, kThreads, 0, stream>>>(xs, conn_s, Es, rp, srec, De, box, st);
}

void launch_master_boxes(mortar_ctx* c, const RunParams& rp) {
  if (c->Em == 0) return;
  const unsigned g = (unsigned)((c->Em + kThreads - 1) / kThreads);
  if (c->nen_m == 4)
    k_master_boxes<4><<<g, kThreads, 0, c->stream>>>(c->xm.as<double>(), c->conn_m.as<int32_t>(), c->Em, rp.delta,
                                                     c->box_m.as<double>(), rp.facing ? c->nrm_m.as<double>() : nullptr,
                                                     c->dstat.as<DevStatus>());
  else
    k_master_boxes<3><<<g, kThreads, 0, c->stream>>>(c->xm.as<double>(), c->conn_m.as<int32_t>(), c->Em, rp.delta,
                                                     c->box_m.as<double>(), rp.facing ? c->nrm_m.as<double>() : nullptr,
                                                     c->dstat.as<DevStatus>());
}

void launch_grid_params(mortar_ctx* c, const RunParams& rp) {
  if (c->n_chunks > 0)
    k_chunk_reduce<<<(unsigned)c->n_chunks, 256, 0, c->stream>>>(c->chunks.as<Chunk>(), c->box_s.as<double>(),
                                                                 c->box_m.as<double>(), c->chunk_red.as<double>());
  k_grid_params<<<(unsigned)c->n_if, 256, 0, c->stream>>>(c->chunk_ptr.as<int32_t>(), c->chunk_red.as<double>(),
                                                          c->bin_cap_off.as<int64_t>(), rp.delta, rp.bin_margin,
                                                          c->grid.as<GridParams>());
  k_bin_offsets<<<1, 1024, 0, c->stream>>>(c->grid.as<GridParams>(), c->n_if, c->bin_cap,
                                           c->dstat.as<DevStatus>());
}

}  // namespace mortar
