// TEST INFRASTRUCTURE ONLY -- the CPU oracle for segment-based mortar integration.
//
// A plain, slow, step-by-step CPU restatement of what Mayr & Popp, "Scalable
// computational kernels for mortar finite element methods" (arXiv 2202.03933)
// compute on the hot path.  Only the test-suite, the smoke check and the CPU
// baseline of the benchmark call it; the product path never does.  It shares no
// code with the CUDA library.
//
// What it follows:
//   * Eq. (AnsatzDiscretization), Sec. 2.2: isoparametric quad4 / tri3 shape
//     functions on slave and master surfaces.
//   * Eq. (AnsatzDiscretizationLagrangeMult), Sec. 2.2: Lagrange multiplier
//     shape functions, standard (Phi = N) or dual (biorthogonal to N, which
//     makes D diagonal).
//   * Eq. (DiscreteWeakFormInterfaceFlux), Sec. 2.2: D[j,k] = int Phi_j N_k and
//     M[j,l] = int Phi_j (N_l o chi_h), both over the discrete slave surface.
//   * Sec. 2.3: integration on a piecewise flat approximation of the slave
//     surface (one auxiliary plane per slave element with point x_0 and normal
//     n_0, Fig. 1), projection along n_0, mortar segments = clip polygons.
//   * Algorithm 1: for each slave element and each nearby master element --
//     project, clip, triangulate into cells, quadrature.
//   * Sec. 3.5 / Algorithm 2: Cartesian bins covering the interface's bounding
//     box, elements sorted into bins, neighbours of a bin searched.
//   * Sec. 1 (consistent linearisation): derivatives of the weighted gap
//     functional by forward-mode dual numbers (exact to rounding).
//
// Readings where the paper is silent (each also listed in the design notes):
// Sutherland-Hodgman clipping of the master polygon by the slave window with an
// absolute inside tolerance eps_in = clip_tol_rel * h_s^2; merge of consecutive
// vertices closer than merge_tol_rel * h_s; discard of polygons with fewer than
// 3 vertices or area < area_tol_rel * A_s; centroid-fan triangulation; the
// 7-point degree-5 triangle rule; Newton back-projection from xi = 0 with
// one extra update after |dxi|_inf <= tol; dual basis built on the whole slave
// element with a 3x3 Gauss-Legendre rule (quad4) or the 7-point rule (tri3).
//
// Scalar type T is double or Dual<N> (forward-mode derivatives).  All branch
// decisions use val(x).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <array>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {

// --------------------------------------------------------------------------
// scalar types
// --------------------------------------------------------------------------
inline double val(double x) { return x; }

template <int N>
struct Dual {
  double v;
  double d[N];
  Dual() : v(0) { for (int i = 0; i < N; ++i) d[i] = 0; }
  Dual(double x) : v(x) { for (int i = 0; i < N; ++i) d[i] = 0; }
  static Dual seed(double x, int k) { Dual r(x); r.d[k] = 1.0; return r; }
};
template <int N> inline double val(const Dual<N>& x) { return x.v; }
template <int N> inline Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v + b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r;
}
template <int N> inline Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v - b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i]; return r;
}
template <int N> inline Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r; r.v = -a.v; for (int i = 0; i < N; ++i) r.d[i] = -a.d[i]; return r;
}
template <int N> inline Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v * b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r;
}
template <int N> inline Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v / b.v;
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v;
  return r;
}
template <int N> inline Dual<N> sqrt(const Dual<N>& a) {
  Dual<N> r; r.v = std::sqrt(a.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / (2.0 * r.v); return r;
}
template <int N> inline Dual<N>& operator+=(Dual<N>& a, const Dual<N>& b) { a = a + b; return a; }
template <int N> inline Dual<N>& operator-=(Dual<N>& a, const Dual<N>& b) { a = a - b; return a; }
template <int N> inline Dual<N> operator+(double a, const Dual<N>& b) { return Dual<N>(a) + b; }
template <int N> inline Dual<N> operator+(const Dual<N>& a, double b) { return a + Dual<N>(b); }
template <int N> inline Dual<N> operator-(double a, const Dual<N>& b) { return Dual<N>(a) - b; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, double b) { return a - Dual<N>(b); }
template <int N> inline Dual<N> operator*(double a, const Dual<N>& b) {
  Dual<N> r; r.v = a * b.v; for (int i = 0; i < N; ++i) r.d[i] = a * b.d[i]; return r;
}
template <int N> inline Dual<N> operator*(const Dual<N>& a, double b) { return b * a; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, double b) { return a / Dual<N>(b); }
template <int N> inline Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }

using std::sqrt;

template <class T> inline T tabs(const T& x) { return val(x) < 0 ? -x : x; }

// --------------------------------------------------------------------------
// options and small geometry helpers
// --------------------------------------------------------------------------
struct Opts {
  int32_t lm;            // 0 standard, 1 dual
  int32_t d_domain;      // 0 element (D over the whole slave surface), 1 segment
  int32_t tri_rule;      // 7 = 7-point degree-5 rule, 25 = collapsed 5x5 Gauss-Legendre
  int32_t fan;           // 0 = centroid fan, 1 = ear fan from vertex 0
  int32_t newton_max_iter;
  int32_t n_threads;
  int32_t terms;         // weighted gap terms: bit 0 = lambda.D Xs, bit 1 = lambda.M Xm
  int32_t pad;
  double delta;          // search inflation
  double newton_tol;
  double clip_tol_rel, merge_tol_rel, area_tol_rel;
};

template <class T> struct V3 { T x, y, z; };
template <class T> struct V2 { T u, v; };

template <class T> inline V3<T> sub(const V3<T>& a, const V3<T>& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> inline T dot(const V3<T>& a, const V3<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> inline V3<T> cross(const V3<T>& a, const V3<T>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class T> inline V3<T> scale(const T& s, const V3<T>& a) { return {s * a.x, s * a.y, s * a.z}; }
template <class T> inline T cross2(const V2<T>& a, const V2<T>& b) { return a.u * b.v - a.v * b.u; }
template <class T> inline V2<T> sub2(const V2<T>& a, const V2<T>& b) { return {a.u - b.u, a.v - b.v}; }

// --------------------------------------------------------------------------
// shape functions (Eq. AnsatzDiscretization)
// quad4 corners (-1,-1), (1,-1), (1,1), (-1,1); tri3 N = (1-xi-eta, xi, eta)
// --------------------------------------------------------------------------
static const double kQuadCorner[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};

template <class T> void shape(int nen, const T& xi, const T& eta, T N[4]) {
  if (nen == 4) {
    for (int a = 0; a < 4; ++a)
      N[a] = 0.25 * (1.0 + kQuadCorner[a][0] * xi) * (1.0 + kQuadCorner[a][1] * eta);
  } else {
    N[0] = 1.0 - xi - eta; N[1] = xi; N[2] = eta; N[3] = T(0.0);
  }
}
template <class T> void shape_deriv(int nen, const T& xi, const T& eta, T dN[4][2]) {
  if (nen == 4) {
    for (int a = 0; a < 4; ++a) {
      dN[a][0] = 0.25 * kQuadCorner[a][0] * (1.0 + kQuadCorner[a][1] * eta);
      dN[a][1] = 0.25 * kQuadCorner[a][1] * (1.0 + kQuadCorner[a][0] * xi);
    }
  } else {
    dN[0][0] = T(-1.0); dN[0][1] = T(-1.0);
    dN[1][0] = T(1.0);  dN[1][1] = T(0.0);
    dN[2][0] = T(0.0);  dN[2][1] = T(1.0);
    dN[3][0] = T(0.0);  dN[3][1] = T(0.0);
  }
}

// --------------------------------------------------------------------------
// quadrature rules
// --------------------------------------------------------------------------
struct TriPoint { double l0, l1, l2, w; };  // barycentric point, weight (sum 1)

// 7-point degree-5 rule on a triangle (Radon 1948; Stroud T2:5-1): centroid
// plus two 3-point orbits with abscissae built from sqrt(15).
static std::vector<TriPoint> rule_tri7() {
  const double r = std::sqrt(15.0);
  const double a1 = (6.0 - r) / 21.0, b1 = (9.0 + 2.0 * r) / 21.0, w1 = (155.0 - r) / 1200.0;
  const double a2 = (6.0 + r) / 21.0, b2 = (9.0 - 2.0 * r) / 21.0, w2 = (155.0 + r) / 1200.0;
  return {{1.0 / 3, 1.0 / 3, 1.0 / 3, 9.0 / 40.0},
          {a1, a1, b1, w1}, {a1, b1, a1, w1}, {b1, a1, a1, w1},
          {a2, a2, b2, w2}, {a2, b2, a2, w2}, {b2, a2, a2, w2}};
}

// n-point Gauss-Legendre on [-1, 1]: Newton on P_n from the Chebyshev guess.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0); w.assign(n, 0.0);
  const double pi = std::acos(-1.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) { double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) { double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Collapsed (Duffy) n x n Gauss-Legendre rule on a triangle: exact for
// polynomials of total degree <= 2n - 2.  Used only to cross-check the
// 7-point rule where integrands are polynomial.
static std::vector<TriPoint> rule_tri_duffy(int n) {
  std::vector<double> x, w;
  gauss_legendre(n, x, w);
  std::vector<TriPoint> out;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.5 * (x[i] + 1.0), t = 0.5 * (x[j] + 1.0);
      double l1 = s, l2 = t * (1.0 - s);
      // area of reference triangle is 1/2 -> normalised weight = 2 * (w/4) * (1-s)
      out.push_back({1.0 - l1 - l2, l1, l2, 2.0 * 0.25 * w[i] * w[j] * (1.0 - s)});
    }
  return out;
}

// Element rule on the parameter domain: points (xi, eta) and weights summing
// to the parameter-domain area (4 for quad4, 1/2 for tri3).
struct ElemPoint { double xi, eta, w; };
static std::vector<ElemPoint> element_rule(int nen) {
  std::vector<ElemPoint> r;
  if (nen == 4) {
    const double g = std::sqrt(0.6);
    const double p[3] = {-g, 0.0, g}, w[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) r.push_back({p[i], p[j], w[i] * w[j]});
  } else {
    for (const TriPoint& q : rule_tri7()) r.push_back({q.l1, q.l2, 0.5 * q.w});
  }
  return r;
}

// --------------------------------------------------------------------------
// slave element data: auxiliary plane, dual basis, element D
// --------------------------------------------------------------------------
template <class T> struct SlaveData {
  int nen;
  V3<T> X[4];           // nodes
  V3<T> x0, n0, t1, t2; // auxiliary plane and in-plane basis
  T A[4][4];            // LM coefficients: Phi_a = sum_b A[a][b] N_b
};

template <class T>
void slave_frame(SlaveData<T>& S) {
  const int nen = S.nen;
  T N[4], dN[4][2];
  const double xc = nen == 4 ? 0.0 : 1.0 / 3.0;
  shape<T>(nen, T(xc), T(xc), N);
  shape_deriv<T>(nen, T(xc), T(xc), dN);
  V3<T> x0{T(0.0), T(0.0), T(0.0)}, g1 = x0, g2 = x0;
  for (int a = 0; a < nen; ++a) {
    x0 = {x0.x + N[a] * S.X[a].x, x0.y + N[a] * S.X[a].y, x0.z + N[a] * S.X[a].z};
    g1 = {g1.x + dN[a][0] * S.X[a].x, g1.y + dN[a][0] * S.X[a].y, g1.z + dN[a][0] * S.X[a].z};
    g2 = {g2.x + dN[a][1] * S.X[a].x, g2.y + dN[a][1] * S.X[a].y, g2.z + dN[a][1] * S.X[a].z};
  }
  V3<T> n = cross(g1, g2);
  T ln = sqrt(dot(n, n));
  S.x0 = x0;
  S.n0 = {n.x / ln, n.y / ln, n.z / ln};
  V3<T> e = sub(S.X[1], S.X[0]);
  T en = dot(e, S.n0);
  V3<T> ep = sub(e, scale(en, S.n0));
  T le = sqrt(dot(ep, ep));
  S.t1 = {ep.x / le, ep.y / le, ep.z / le};
  S.t2 = cross(S.n0, S.t1);
}

// Gaussian elimination with partial pivoting: solve K X = B (n x n, n rhs).
template <class T>
void solve_dense(int n, T K[4][4], T B[4][4]) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(val(K[r][c])) > std::fabs(val(K[piv][c]))) piv = r;
    if (piv != c)
      for (int k = 0; k < n; ++k) { std::swap(K[c][k], K[piv][k]); std::swap(B[c][k], B[piv][k]); }
    for (int r = c + 1; r < n; ++r) {
      T f = K[r][c] / K[c][c];
      for (int k = c; k < n; ++k) K[r][k] = K[r][k] - f * K[c][k];
      for (int k = 0; k < n; ++k) B[r][k] = B[r][k] - f * B[c][k];
    }
  }
  for (int c = n - 1; c >= 0; --c)
    for (int k = 0; k < n; ++k) {
      T s = B[c][k];
      for (int j = c + 1; j < n; ++j) s = s - K[c][j] * B[j][k];
      B[c][k] = s / K[c][c];
    }
}

template <class T>
T surface_jacobian(int nen, const V3<T> X[4], const T dN[4][2]) {
  V3<T> g1{T(0.0), T(0.0), T(0.0)}, g2 = g1;
  for (int a = 0; a < nen; ++a) {
    g1 = {g1.x + dN[a][0] * X[a].x, g1.y + dN[a][0] * X[a].y, g1.z + dN[a][0] * X[a].z};
    g2 = {g2.x + dN[a][1] * X[a].x, g2.y + dN[a][1] * X[a].y, g2.z + dN[a][1] * X[a].z};
  }
  V3<T> n = cross(g1, g2);
  return sqrt(dot(n, n));
}

// LM coefficients.  Standard: A = I.  Dual (biorthogonal, Sec. 2.2): with
// Me[a][b] = int_e N_a N_b and Dh = diag(int_e N_a), A = Dh Me^{-1}, so that
// int_e Phi_a N_b = delta_ab int_e N_b.
template <class T>
void lm_coefficients(SlaveData<T>& S, int lm) {
  const int n = S.nen;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) S.A[a][b] = T(a == b ? 1.0 : 0.0);
  if (lm == 0) return;
  T Me[4][4], Dh[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) { Me[a][b] = T(0.0); Dh[a][b] = T(0.0); }
  for (const ElemPoint& q : element_rule(n)) {
    T N[4], dN[4][2];
    shape<T>(n, T(q.xi), T(q.eta), N);
    shape_deriv<T>(n, T(q.xi), T(q.eta), dN);
    T wj = q.w * surface_jacobian<T>(n, S.X, dN);
    for (int a = 0; a < n; ++a) {
      Dh[a][a] = Dh[a][a] + wj * N[a];
      for (int b = 0; b < n; ++b) Me[a][b] = Me[a][b] + wj * N[a] * N[b];
    }
  }
  // Me symmetric: Me A^T = Dh  ->  solve for A^T column by column
  solve_dense<T>(n, Me, Dh);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) S.A[a][b] = Dh[b][a];
}

// Element-domain D (Eq. DiscreteWeakFormInterfaceFlux integrated over the whole
// slave element): De[a][b] = sum_q w_q J(xi_q) Phi_a(xi_q) N_b(xi_q).
template <class T>
void element_D(const SlaveData<T>& S, T De[4][4]) {
  const int n = S.nen;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) De[a][b] = T(0.0);
  for (const ElemPoint& q : element_rule(n)) {
    T N[4], dN[4][2];
    shape<T>(n, T(q.xi), T(q.eta), N);
    shape_deriv<T>(n, T(q.xi), T(q.eta), dN);
    T wj = q.w * surface_jacobian<T>(n, S.X, dN);
    for (int a = 0; a < n; ++a) {
      T phi = T(0.0);
      for (int c = 0; c < n; ++c) phi = phi + S.A[a][c] * N[c];
      for (int b = 0; b < n; ++b) De[a][b] = De[a][b] + wj * phi * N[b];
    }
  }
}

// --------------------------------------------------------------------------
// back-projection chi_h: solve sum_a N_a(xi) p_a = x in the auxiliary plane
// --------------------------------------------------------------------------
struct Stats {
  int64_t pairs = 0, nonempty = 0, gauss_points = 0, newton_fail = 0, xi_out_of_range = 0,
          clip_overflow = 0, cells = 0;
};

template <class T>
void invert_map(int nen, const V2<T> p[4], const V2<T>& x, const Opts& o, T xi[2], Stats& st) {
  if (nen == 3) {
    V2<T> e1 = sub2(p[1], p[0]), e2 = sub2(p[2], p[0]), r = sub2(x, p[0]);
    T det = e1.u * e2.v - e2.u * e1.v;
    xi[0] = (r.u * e2.v - e2.u * r.v) / det;
    xi[1] = (e1.u * r.v - r.u * e1.v) / det;
  } else {
    xi[0] = T(0.0); xi[1] = T(0.0);
    bool converged = false, last = false;
    for (int it = 0; it < o.newton_max_iter; ++it) {
      T N[4], dN[4][2];
      shape<T>(4, xi[0], xi[1], N);
      shape_deriv<T>(4, xi[0], xi[1], dN);
      T ru = -x.u, rv = -x.v, J00 = T(0.0), J01 = T(0.0), J10 = T(0.0), J11 = T(0.0);
      for (int a = 0; a < 4; ++a) {
        ru = ru + N[a] * p[a].u;
        rv = rv + N[a] * p[a].v;
        J00 = J00 + dN[a][0] * p[a].u; J01 = J01 + dN[a][1] * p[a].u;
        J10 = J10 + dN[a][0] * p[a].v; J11 = J11 + dN[a][1] * p[a].v;
      }
      T det = J00 * J11 - J01 * J10;
      T d0 = -(J11 * ru - J01 * rv) / det;
      T d1 = -(J00 * rv - J10 * ru) / det;
      xi[0] = xi[0] + d0;
      xi[1] = xi[1] + d1;
      if (last) { converged = true; break; }
      if (std::max(std::fabs(val(d0)), std::fabs(val(d1))) <= o.newton_tol) last = true;
    }
    if (!converged) st.newton_fail++;
  }
  double lim = 1.0 + 1e-8;
  if (nen == 4) {
    if (std::fabs(val(xi[0])) > lim || std::fabs(val(xi[1])) > lim) st.xi_out_of_range++;
  } else {
    if (val(xi[0]) < -1e-8 || val(xi[1]) < -1e-8 || val(xi[0]) + val(xi[1]) > lim) st.xi_out_of_range++;
  }
}

// --------------------------------------------------------------------------
// one slave/master pair (Algorithm 1 body)
// --------------------------------------------------------------------------
template <class T> struct PairOut {
  bool nonempty = false;
  int nverts = 0;
  T M[4][4];
  T D[4][4];
};

template <class T>
T polygon_signed_area2(const std::vector<V2<T>>& P) {  // twice the signed area
  T s = T(0.0);
  const size_t n = P.size();
  for (size_t k = 0; k < n; ++k) s = s + cross2(P[k], P[(k + 1) % n]);
  return s;
}

template <class T> struct Cell { V2<T> a, b, c; };

// Steps (1)-(4) of Algorithm 1 for one slave/master pair: projection onto the
// slave element's auxiliary plane, clipping, merge, triangulation.  Writes the
// projected slave and master polygons (element node order) and the cells;
// returns false (no cells) when the pair contributes nothing.
template <class T>
bool pair_cells(const SlaveData<T>& S, const V3<T> Xm[4], int nen_m, const Opts& o, Stats& st, V2<T> ps[4],
                V2<T> pm[4], std::vector<Cell<T>>& cells, int& nverts) {
  const int nen_s = S.nen;
  cells.clear();
  nverts = 0;

  // tolerances from the real slave geometry (diameter, projected area)
  double h_s = 0.0;
  for (int a = 0; a < nen_s; ++a)
    for (int b = a + 1; b < nen_s; ++b) {
      double dx = val(S.X[a].x) - val(S.X[b].x), dy = val(S.X[a].y) - val(S.X[b].y),
             dz = val(S.X[a].z) - val(S.X[b].z);
      h_s = std::max(h_s, std::sqrt(dx * dx + dy * dy + dz * dz));
    }
  const double eps_in = o.clip_tol_rel * h_s * h_s;
  const double eps_merge = o.merge_tol_rel * h_s;

  // (1) project all nodes onto the auxiliary plane; in-plane coordinates
  for (int a = 0; a < nen_s; ++a) {
    V3<T> d = sub(S.X[a], S.x0);
    ps[a] = {dot(d, S.t1), dot(d, S.t2)};
  }
  for (int l = 0; l < nen_m; ++l) {
    V3<T> d = sub(Xm[l], S.x0);
    pm[l] = {dot(d, S.t1), dot(d, S.t2)};
  }
  std::vector<V2<T>> win(ps, ps + nen_s), poly(pm, pm + nen_m);
  T as2 = polygon_signed_area2(win);
  if (val(as2) < 0) std::reverse(win.begin(), win.end());
  if (val(polygon_signed_area2(poly)) < 0) std::reverse(poly.begin(), poly.end());
  const double A_s = 0.5 * std::fabs(val(as2));
  const double eps_area = o.area_tol_rel * A_s;

  // (2) clip: Sutherland-Hodgman, master polygon against the slave window
  for (int i = 0; i < nen_s && !poly.empty(); ++i) {
    const V2<T>& a = win[i];
    const V2<T>& b = win[(i + 1) % nen_s];
    V2<T> e = sub2(b, a);
    std::vector<V2<T>> next;
    const size_t n = poly.size();
    for (size_t k = 0; k < n; ++k) {
      const V2<T>& p = poly[k];
      const V2<T>& q = poly[(k + 1) % n];
      T dp = cross2(e, sub2(p, a));
      T dq = cross2(e, sub2(q, a));
      double vp = val(dp), vq = val(dq);
      if ((vp > eps_in && vq < -eps_in) || (vp < -eps_in && vq > eps_in)) {
        T t = dp / (dp - dq);
        next.push_back({p.u + t * (q.u - p.u), p.v + t * (q.v - p.v)});
      }
      if (vq >= -eps_in) next.push_back(q);
    }
    poly.swap(next);
  }
  if (poly.size() > 16) st.clip_overflow++;

  // (3) merge consecutive (cyclic) vertices closer than eps_merge
  std::vector<V2<T>> P;
  const double em2 = eps_merge * eps_merge;
  auto close = [&](const V2<T>& x, const V2<T>& y) {
    double du = val(x.u) - val(y.u), dv = val(x.v) - val(y.v);
    return du * du + dv * dv < em2;
  };
  for (const V2<T>& v : poly)
    if (P.empty() || !close(v, P.back())) P.push_back(v);
  while (P.size() > 1 && close(P.back(), P.front())) P.pop_back();
  if (P.size() < 3) return false;
  if (0.5 * std::fabs(val(polygon_signed_area2(P))) < eps_area) return false;
  nverts = (int)P.size();
  st.nonempty++;

  // (4) triangulate into integration cells
  const size_t nv = P.size();
  if (nv == 3) {
    cells.push_back({P[0], P[1], P[2]});
  } else if (o.fan == 1) {
    for (size_t i = 1; i + 1 < nv; ++i) cells.push_back({P[0], P[i], P[i + 1]});
  } else {
    V2<T> c{T(0.0), T(0.0)};
    for (const V2<T>& v : P) { c.u = c.u + v.u; c.v = c.v + v.v; }
    c.u = c.u / double(nv);
    c.v = c.v / double(nv);
    for (size_t i = 0; i < nv; ++i) cells.push_back({c, P[i], P[(i + 1) % nv]});
  }
  st.cells += (int64_t)cells.size();
  return true;
}

template <class T>
void integrate_pair(const SlaveData<T>& S, const V3<T> Xm[4], int nen_m, const Opts& o,
                    PairOut<T>& out, Stats& st) {
  const int nen_s = S.nen;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) { out.M[a][b] = T(0.0); out.D[a][b] = T(0.0); }
  out.nonempty = false;
  out.nverts = 0;
  st.pairs++;
  V2<T> ps[4], pm[4];
  std::vector<Cell<T>> cells;
  if (!pair_cells<T>(S, Xm, nen_m, o, st, ps, pm, cells, out.nverts)) return;
  out.nonempty = true;

  // (5) quadrature on each cell with back-projection to both elements
  const std::vector<TriPoint> rule = o.tri_rule == 25 ? rule_tri_duffy(5) : rule_tri7();
  for (const Cell<T>& C : cells) {
    T ar2 = cross2(sub2(C.b, C.a), sub2(C.c, C.a));
    T area = 0.5 * tabs(ar2);
    for (const TriPoint& q : rule) {
      V2<T> xg{q.l0 * C.a.u + q.l1 * C.b.u + q.l2 * C.c.u, q.l0 * C.a.v + q.l1 * C.b.v + q.l2 * C.c.v};
      T W = q.w * area;
      T xs[2], xm[2];
      invert_map<T>(nen_s, ps, xg, o, xs, st);
      invert_map<T>(nen_m, pm, xg, o, xm, st);
      T Ns[4], Nm[4], Phi[4];
      shape<T>(nen_s, xs[0], xs[1], Ns);
      shape<T>(nen_m, xm[0], xm[1], Nm);
      for (int a = 0; a < nen_s; ++a) {
        Phi[a] = T(0.0);
        for (int c = 0; c < nen_s; ++c) Phi[a] = Phi[a] + S.A[a][c] * Ns[c];
      }
      for (int a = 0; a < nen_s; ++a) {
        T wp = W * Phi[a];
        for (int l = 0; l < nen_m; ++l) out.M[a][l] = out.M[a][l] + wp * Nm[l];
        if (o.d_domain == 1)
          for (int b = 0; b < nen_s; ++b) out.D[a][b] = out.D[a][b] + wp * Ns[b];
      }
      st.gauss_points++;
    }
  }
}

// --------------------------------------------------------------------------
// quadratic slave elements (tri6, quad8), standard Lagrange multipliers
// --------------------------------------------------------------------------
// quad8 (serendipity): corners 0..3 at (-1,-1), (1,-1), (1,1), (-1,1), mid-side
// nodes 4..7 at (0,-1), (1,0), (0,1), (-1,0):
//   corner:   N = (1 + xi xi_a)(1 + eta eta_a)(xi xi_a + eta eta_a - 1) / 4,
//   xi_a = 0: N = (1 - xi^2)(1 + eta eta_a) / 2,  eta_a = 0: N = (1 + xi xi_a)(1 - eta^2) / 2.
// tri6: corners 0..2 at (0,0), (1,0), (0,1), mid-side nodes 3 (edge 0-1),
// 4 (edge 1-2), 5 (edge 2-0); with L = (1 - xi - eta, xi, eta):
//   corner i: N = L_i (2 L_i - 1),  mid-side (i, j): N = 4 L_i L_j.
static const double kQ8Node[8][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}, {0, -1}, {1, 0}, {0, 1}, {-1, 0}};

inline void shape_quadratic(int nen, double xi, double eta, double N[8], double dN[8][2]) {
  if (nen == 8) {
    for (int a = 0; a < 8; ++a) {
      const double xa = kQ8Node[a][0], ea = kQ8Node[a][1];
      if (a < 4) {
        N[a] = 0.25 * (1.0 + xi * xa) * (1.0 + eta * ea) * (xi * xa + eta * ea - 1.0);
        dN[a][0] = 0.25 * xa * (1.0 + eta * ea) * (2.0 * xi * xa + eta * ea);
        dN[a][1] = 0.25 * ea * (1.0 + xi * xa) * (xi * xa + 2.0 * eta * ea);
      } else if (xa == 0.0) {
        N[a] = 0.5 * (1.0 - xi * xi) * (1.0 + eta * ea);
        dN[a][0] = -xi * (1.0 + eta * ea);
        dN[a][1] = 0.5 * ea * (1.0 - xi * xi);
      } else {
        N[a] = 0.5 * (1.0 + xi * xa) * (1.0 - eta * eta);
        dN[a][0] = 0.5 * xa * (1.0 - eta * eta);
        dN[a][1] = -eta * (1.0 + xi * xa);
      }
    }
  } else {
    const double L[3] = {1.0 - xi - eta, xi, eta};
    const double dL[3][2] = {{-1.0, -1.0}, {1.0, 0.0}, {0.0, 1.0}};
    for (int i = 0; i < 3; ++i) {
      N[i] = L[i] * (2.0 * L[i] - 1.0);
      dN[i][0] = (4.0 * L[i] - 1.0) * dL[i][0];
      dN[i][1] = (4.0 * L[i] - 1.0) * dL[i][1];
    }
    const int edge[3][2] = {{0, 1}, {1, 2}, {2, 0}};
    for (int k = 0; k < 3; ++k) {
      const int i = edge[k][0], j = edge[k][1];
      N[3 + k] = 4.0 * L[i] * L[j];
      dN[3 + k][0] = 4.0 * (L[j] * dL[i][0] + L[i] * dL[j][0]);
      dN[3 + k][1] = 4.0 * (L[j] * dL[i][1] + L[i] * dL[j][1]);
    }
    for (int a = 6; a < 8; ++a) { N[a] = 0.0; dN[a][0] = 0.0; dN[a][1] = 0.0; }
  }
}

// The four linear sub-elements of a quadratic element: their corners (parent
// local nodes; -1 = the quad8 centre xi = eta = 0) and the corners' parent
// parameter coordinates, counter-clockwise like the parent.  quad8 -> four
// quad4 (corner, mid-side, centre, mid-side); tri6 -> four tri3 (three corner
// triangles and the middle one).
struct SubElement { int nen; int node[4]; double ref[4][2]; };

inline void sub_elements(int nen_p, SubElement sub[4]) {
  if (nen_p == 8) {
    const SubElement q[4] = {
        {4, {0, 4, -1, 7}, {{-1, -1}, {0, -1}, {0, 0}, {-1, 0}}},
        {4, {4, 1, 5, -1}, {{0, -1}, {1, -1}, {1, 0}, {0, 0}}},
        {4, {-1, 5, 2, 6}, {{0, 0}, {1, 0}, {1, 1}, {0, 1}}},
        {4, {7, -1, 6, 3}, {{-1, 0}, {0, 0}, {0, 1}, {-1, 1}}}};
    for (int k = 0; k < 4; ++k) sub[k] = q[k];
  } else {
    const SubElement t[4] = {
        {3, {0, 3, 5, 0}, {{0, 0}, {0.5, 0}, {0, 0.5}, {0, 0}}},
        {3, {3, 1, 4, 0}, {{0.5, 0}, {1, 0}, {0.5, 0.5}, {0, 0}}},
        {3, {5, 4, 2, 0}, {{0, 0.5}, {0.5, 0.5}, {0, 1}, {0, 0}}},
        {3, {3, 4, 5, 0}, {{0.5, 0}, {0.5, 0.5}, {0, 0.5}, {0, 0}}}};
    for (int k = 0; k < 4; ++k) sub[k] = t[k];
  }
}

// Element-domain D of a quadratic element, standard LMs (Eq.
// DiscreteWeakFormInterfaceFlux over the whole element): De[a][b] =
// sum_q w_q J(xi_q) N_a N_b with the 3x3 Gauss-Legendre rule (quad8) or the
// 7-point rule (tri6), exact for flat elements (N_a N_b of degree <= 4 per
// direction).
inline void element_D_quadratic(int nen, const V3<double> X[8], double De[8][8]) {
  for (int a = 0; a < 8; ++a)
    for (int b = 0; b < 8; ++b) De[a][b] = 0.0;
  for (const ElemPoint& q : element_rule(nen == 8 ? 4 : 3)) {
    double N[8], dN[8][2];
    shape_quadratic(nen, q.xi, q.eta, N, dN);
    V3<double> g1{0.0, 0.0, 0.0}, g2 = g1;
    for (int a = 0; a < nen; ++a) {
      g1 = {g1.x + dN[a][0] * X[a].x, g1.y + dN[a][0] * X[a].y, g1.z + dN[a][0] * X[a].z};
      g2 = {g2.x + dN[a][1] * X[a].x, g2.y + dN[a][1] * X[a].y, g2.z + dN[a][1] * X[a].z};
    }
    const V3<double> n = cross(g1, g2);
    const double wj = q.w * std::sqrt(dot(n, n));
    for (int a = 0; a < nen; ++a)
      for (int b = 0; b < nen; ++b) De[a][b] += wj * N[a] * N[b];
  }
}

// One quadratic slave element against one master element: steps (1)-(4) of
// Algorithm 1 on each linear sub-element (the piecewise flat approximation of
// the slave surface, Sec. 2.3), the 7-point rule on every cell, and at every
// point the sub-element parameters mapped to the parent's, where the
// quadratic shape functions are evaluated:
//   M[a][l] += W N_a(xi_parent) N_l(xi_m).
inline void integrate_pair_quadratic(int nen_p, const V3<double> Xp[8], const V3<double> Xm[4], int nen_m,
                                     const Opts& o, double M[8][4], bool& nonempty, Stats& st) {
  for (int a = 0; a < 8; ++a)
    for (int l = 0; l < 4; ++l) M[a][l] = 0.0;
  nonempty = false;
  st.pairs++;
  SubElement sub[4];
  sub_elements(nen_p, sub);
  V3<double> xc{0.0, 0.0, 0.0};
  if (nen_p == 8) {   // the centre point of the quad8
    double N[8], dN[8][2];
    shape_quadratic(8, 0.0, 0.0, N, dN);
    for (int a = 0; a < 8; ++a) xc = {xc.x + N[a] * Xp[a].x, xc.y + N[a] * Xp[a].y, xc.z + N[a] * Xp[a].z};
  }
  const std::vector<TriPoint> rule = rule_tri7();
  for (int k = 0; k < 4; ++k) {
    const SubElement& se = sub[k];
    SlaveData<double> S;
    S.nen = se.nen;
    for (int j = 0; j < 4; ++j) S.X[j] = {0.0, 0.0, 0.0};
    for (int j = 0; j < se.nen; ++j) S.X[j] = se.node[j] < 0 ? xc : Xp[se.node[j]];
    slave_frame<double>(S);
    Stats sk;
    V2<double> ps[4], pm[4];
    std::vector<Cell<double>> cells;
    int nv = 0;
    if (!pair_cells<double>(S, Xm, nen_m, o, sk, ps, pm, cells, nv)) {
      st.clip_overflow += sk.clip_overflow;
      continue;
    }
    nonempty = true;
    st.cells += sk.cells;
    st.clip_overflow += sk.clip_overflow;
    for (const Cell<double>& C : cells) {
      const double area = 0.5 * std::fabs(cross2(sub2(C.b, C.a), sub2(C.c, C.a)));
      for (const TriPoint& q : rule) {
        V2<double> xg{q.l0 * C.a.u + q.l1 * C.b.u + q.l2 * C.c.u, q.l0 * C.a.v + q.l1 * C.b.v + q.l2 * C.c.v};
        const double W = q.w * area;
        double xs[2], xm[2];
        invert_map<double>(se.nen, ps, xg, o, xs, st);
        invert_map<double>(nen_m, pm, xg, o, xm, st);
        double Nsub[4], Nm[4];
        shape<double>(se.nen, xs[0], xs[1], Nsub);
        shape<double>(nen_m, xm[0], xm[1], Nm);
        double xp = 0.0, ep = 0.0;   // parent parameters (an affine map of the sub-element's)
        for (int j = 0; j < se.nen; ++j) { xp += Nsub[j] * se.ref[j][0]; ep += Nsub[j] * se.ref[j][1]; }
        double Np[8], dNp[8][2];
        shape_quadratic(nen_p, xp, ep, Np, dNp);
        for (int a = 0; a < nen_p; ++a) {
          const double wn = W * Np[a];
          for (int l = 0; l < nen_m; ++l) M[a][l] += wn * Nm[l];
        }
        st.gauss_points++;
      }
    }
  }
  if (nonempty) st.nonempty++;
}

// --------------------------------------------------------------------------
// contact search
// --------------------------------------------------------------------------
struct Box { double lo[3], hi[3]; };

static Box element_box(const double* X, const int32_t* conn, int nen, double delta) {
  Box b;
  for (int d = 0; d < 3; ++d) { b.lo[d] = X[3 * conn[0] + d]; b.hi[d] = b.lo[d]; }
  for (int a = 1; a < nen; ++a)
    for (int d = 0; d < 3; ++d) {
      double x = X[3 * conn[a] + d];
      b.lo[d] = std::min(b.lo[d], x);
      b.hi[d] = std::max(b.hi[d], x);
    }
  for (int d = 0; d < 3; ++d) { b.lo[d] = b.lo[d] - delta; b.hi[d] = b.hi[d] + delta; }
  return b;
}

static bool boxes_overlap(const Box& a, const Box& b) {
  for (int d = 0; d < 3; ++d)
    if (!(a.lo[d] <= b.hi[d] && b.lo[d] <= a.hi[d])) return false;
  return true;
}

static double element_diameter(const double* X, const int32_t* conn, int nen) {
  double h = 0.0;
  for (int a = 0; a < nen; ++a)
    for (int b = a + 1; b < nen; ++b) {
      double s = 0.0;
      for (int d = 0; d < 3; ++d) { double t = X[3 * conn[a] + d] - X[3 * conn[b] + d]; s += t * t; }
      h = std::max(h, std::sqrt(s));
    }
  return h;
}

}  // namespace orc

using namespace orc;

namespace {

template <class T>
void load_slave(SlaveData<T>& S, const double* xs, const int32_t* cs, int nen, int64_t e, int lm) {
  S.nen = nen;
  for (int a = 0; a < nen; ++a) {
    const double* p = xs + 3 * (int64_t)cs[nen * e + a];
    S.X[a] = {T(p[0]), T(p[1]), T(p[2])};
  }
  for (int a = nen; a < 4; ++a) S.X[a] = {T(0.0), T(0.0), T(0.0)};
  slave_frame<T>(S);
  lm_coefficients<T>(S, lm);
}

void add_stats(int64_t* out, const Stats& s) {
  out[0] += s.pairs; out[1] += s.nonempty; out[2] += s.gauss_points; out[3] += s.newton_fail;
  out[4] += s.xi_out_of_range; out[5] += s.clip_overflow; out[6] += s.cells;
}

}  // namespace

extern "C" {

// Brute-force candidate search (the definition): all (s, m) whose
// delta-inflated bounding boxes overlap, closed comparison, sorted by (s, m).
// Returns the number of pairs; writes at most `cap` of them.
int64_t oracle_search_bruteforce(const double* xs, int64_t Ns, const int32_t* cs, int64_t Es, int32_t nen_s,
                                 const double* xm, int64_t Nm, const int32_t* cm, int64_t Em, int32_t nen_m,
                                 double delta, int32_t* s_out, int32_t* m_out, int64_t cap) {
  (void)Ns; (void)Nm;
  std::vector<Box> bm(Em);
  for (int64_t m = 0; m < Em; ++m) bm[m] = element_box(xm, cm + nen_m * m, nen_m, delta);
  int64_t n = 0;
  for (int64_t s = 0; s < Es; ++s) {
    Box b = element_box(xs, cs + nen_s * s, nen_s, delta);
    for (int64_t m = 0; m < Em; ++m)
      if (boxes_overlap(b, bm[m])) {
        if (n < cap) { s_out[n] = (int32_t)s; m_out[n] = (int32_t)m; }
        ++n;
      }
  }
  return n;
}

// Binned candidate search (Algorithm 2 on one device): Cartesian bins over the
// interface's bounding box, expanded by the minimal bin size
//   beta_min = (1 + 1e-9) * max element diameter (both sides) + 2 * delta;
// n_d = max(1, floor(L_d / beta_min)) bins per direction.  Each element is
// binned by its bounding-box centre; each slave element tests the master
// elements of its own bin and its 26 neighbours.  Same result as brute force.
int64_t oracle_search_binned(const double* xs, int64_t Ns, const int32_t* cs, int64_t Es, int32_t nen_s,
                             const double* xm, int64_t Nm, const int32_t* cm, int64_t Em, int32_t nen_m,
                             double delta, int32_t* s_out, int32_t* m_out, int64_t cap) {
  double lo[3], hi[3];
  for (int d = 0; d < 3; ++d) { lo[d] = INFINITY; hi[d] = -INFINITY; }
  for (int64_t i = 0; i < Ns; ++i)
    for (int d = 0; d < 3; ++d) { lo[d] = std::min(lo[d], xs[3 * i + d]); hi[d] = std::max(hi[d], xs[3 * i + d]); }
  for (int64_t i = 0; i < Nm; ++i)
    for (int d = 0; d < 3; ++d) { lo[d] = std::min(lo[d], xm[3 * i + d]); hi[d] = std::max(hi[d], xm[3 * i + d]); }
  double hmax = 0.0;
  for (int64_t e = 0; e < Es; ++e) hmax = std::max(hmax, element_diameter(xs, cs + nen_s * e, nen_s));
  for (int64_t e = 0; e < Em; ++e) hmax = std::max(hmax, element_diameter(xm, cm + nen_m * e, nen_m));
  const double beta_min = (1.0 + 1e-9) * hmax + 2.0 * delta;
  int64_t nb[3];
  double beta[3], org[3];
  for (int d = 0; d < 3; ++d) {
    org[d] = lo[d] - beta_min;
    double L = (hi[d] + beta_min) - org[d];
    nb[d] = std::max<int64_t>(1, (int64_t)std::floor(L / beta_min));
    beta[d] = L / (double)nb[d];
  }
  auto bin_of = [&](const Box& b, int64_t ijk[3]) {
    for (int d = 0; d < 3; ++d) {
      double c = 0.5 * (b.lo[d] + b.hi[d]);
      int64_t i = (int64_t)std::floor((c - org[d]) / beta[d]);
      ijk[d] = std::min<int64_t>(std::max<int64_t>(i, 0), nb[d] - 1);
    }
  };
  std::vector<Box> bm(Em);
  // sparse bins: sorted (bin id, element) list
  std::vector<std::pair<int64_t, int32_t>> keyed(Em);
  for (int64_t m = 0; m < Em; ++m) {
    bm[m] = element_box(xm, cm + nen_m * m, nen_m, delta);
    int64_t ijk[3];
    bin_of(bm[m], ijk);
    keyed[m] = {(ijk[2] * nb[1] + ijk[1]) * nb[0] + ijk[0], (int32_t)m};
  }
  std::sort(keyed.begin(), keyed.end());
  int64_t n = 0;
  std::vector<int32_t> found;
  for (int64_t s = 0; s < Es; ++s) {
    Box b = element_box(xs, cs + nen_s * s, nen_s, delta);
    int64_t ijk[3];
    bin_of(b, ijk);
    found.clear();
    for (int64_t dz = -1; dz <= 1; ++dz)
      for (int64_t dy = -1; dy <= 1; ++dy)
        for (int64_t dx = -1; dx <= 1; ++dx) {
          int64_t i = ijk[0] + dx, j = ijk[1] + dy, k = ijk[2] + dz;
          if (i < 0 || j < 0 || k < 0 || i >= nb[0] || j >= nb[1] || k >= nb[2]) continue;
          int64_t key = (k * nb[1] + j) * nb[0] + i;
          auto it = std::lower_bound(keyed.begin(), keyed.end(), std::make_pair(key, (int32_t)-1));
          for (; it != keyed.end() && it->first == key; ++it)
            if (boxes_overlap(b, bm[it->second])) found.push_back(it->second);
        }
    std::sort(found.begin(), found.end());
    for (int32_t m : found) {
      if (n < cap) { s_out[n] = (int32_t)s; m_out[n] = m; }
      ++n;
    }
  }
  return n;
}

// Per-slave-element LM coefficients A (Es x 16, row-major 4x4) and
// element-domain D blocks (Es x 16).
int oracle_element_blocks(const double* xs, const int32_t* cs, int64_t Es, int32_t nen_s, int32_t lm,
                          double* A_out, double* De_out) {
  for (int64_t e = 0; e < Es; ++e) {
    SlaveData<double> S;
    load_slave<double>(S, xs, cs, nen_s, e, lm);
    double De[4][4];
    element_D<double>(S, De);
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        if (A_out) A_out[16 * e + 4 * a + b] = S.A[a][b];
        if (De_out) De_out[16 * e + 4 * a + b] = De[a][b];
      }
  }
  return 0;
}

// Per-pair integration (Algorithm 1 body) for an explicit pair list.
// M_out, D_out: P x 16 (row a = slave local node, column = master / slave
// local node); nonempty: P bytes; stats: 7 counters
// (pairs, nonempty, gauss points, newton failures, xi out of range,
//  clip overflow, cells).
int oracle_pair_blocks(const double* xs, const int32_t* cs, int32_t nen_s,
                       const double* xm, const int32_t* cm, int32_t nen_m,
                       const Opts* o, const int32_t* ps, const int32_t* pm, int64_t P,
                       double* M_out, double* D_out, uint8_t* nonempty, int64_t* stats) {
  for (int k = 0; k < 7; ++k) stats[k] = 0;
  int nt = o->n_threads > 0 ? o->n_threads : 1;
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
  {
    Stats st;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 256)
#endif
    for (int64_t p = 0; p < P; ++p) {
      SlaveData<double> S;
      load_slave<double>(S, xs, cs, nen_s, ps[p], o->lm);
      V3<double> Xm[4];
      for (int l = 0; l < 4; ++l) Xm[l] = {0.0, 0.0, 0.0};
      for (int l = 0; l < nen_m; ++l) {
        const double* q = xm + 3 * (int64_t)cm[(int64_t)nen_m * pm[p] + l];
        Xm[l] = {q[0], q[1], q[2]};
      }
      PairOut<double> r;
      integrate_pair<double>(S, Xm, nen_m, *o, r, st);
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          M_out[16 * p + 4 * a + b] = r.M[a][b];
          if (D_out) D_out[16 * p + 4 * a + b] = r.D[a][b];
        }
      nonempty[p] = r.nonempty ? 1 : 0;
    }
#ifdef _OPENMP
#pragma omp critical
#endif
    add_stats(stats, st);
  }
  (void)nt;
  return 0;
}

// Element-based integration (Sec. 1 and Sec. 2.3: no clipping or
// triangulation; a higher-order rule on the slave element copes with the
// kinks of the integrand at master element edges, at lower accuracy than the
// segment-based rule).  Per slave element: an n x n Gauss-Legendre rule on
// quad4 (collapsed n x n rule on tri3) in the element's auxiliary plane; each
// quadrature point x_q is back-projected onto the master elements of the
// element's candidate pairs in pair order, and the first whose map inverse
// converges with the point inside (|xi|, |eta| <= 1 + 1e-10 on quad4,
// barycentric >= -1e-10 on tri3) receives it:
//   M_p[a][l] += w_q |det J_s(xi_q)| Phi_a(xi_q) N_l(xi_m),
//   D_p[a][b] += w_q |det J_s(xi_q)| Phi_a(xi_q) N_b(xi_q)   (segment D).
// Points no master covers contribute nothing.  Pairs must be sorted by slave
// element.  flag[p] = 1 if pair p received a point.
int oracle_element_based_blocks(const double* xs, const int32_t* cs, int32_t nen_s,
                                const double* xm, const int32_t* cm, int32_t nen_m,
                                const Opts* o, const int32_t* ps, const int32_t* pm, int64_t P,
                                int32_t n_rule, double* M_out, double* D_out, uint8_t* flag) {
  std::vector<double> gx, gw;
  gauss_legendre(n_rule, gx, gw);
  struct SP { double xi, eta, w; };   // slave parameter points, weights summing to the parameter area
  std::vector<SP> rule;
  if (nen_s == 4) {
    for (int i = 0; i < n_rule; ++i)
      for (int j = 0; j < n_rule; ++j) rule.push_back({gx[i], gx[j], gw[i] * gw[j]});
  } else {
    for (const TriPoint& q : rule_tri_duffy(n_rule)) rule.push_back({q.l1, q.l2, 0.5 * q.w});
  }
  const double tol_in = 1e-10;
  for (int64_t p = 0; p < P; ++p) {
    flag[p] = 0;
    for (int k = 0; k < 16; ++k) { M_out[16 * p + k] = 0.0; if (D_out) D_out[16 * p + k] = 0.0; }
  }
  // runs of pairs with the same slave element
  std::vector<int64_t> starts;
  for (int64_t p = 0; p < P; ++p)
    if (p == 0 || ps[p] != ps[p - 1]) starts.push_back(p);
  starts.push_back(P);
  const int nt = o->n_threads > 0 ? o->n_threads : 1;
  const int64_t n_runs = (int64_t)starts.size() - 1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
#endif
  for (int64_t r = 0; r < n_runs; ++r) {
    const int64_t p0 = starts[r], p1 = starts[r + 1];
    SlaveData<double> S;
    load_slave<double>(S, xs, cs, nen_s, ps[p0], o->lm);
    V2<double> pss[4];
    for (int a = 0; a < nen_s; ++a) {
      V3<double> d = sub(S.X[a], S.x0);
      pss[a] = {dot(d, S.t1), dot(d, S.t2)};
    }
    // projected master elements of the candidate pairs
    std::vector<std::array<V2<double>, 4>> pmm(p1 - p0);
    for (int64_t p = p0; p < p1; ++p)
      for (int l = 0; l < nen_m; ++l) {
        const double* q = xm + 3 * (int64_t)cm[(int64_t)nen_m * pm[p] + l];
        V3<double> d = sub(V3<double>{q[0], q[1], q[2]}, S.x0);
        pmm[p - p0][l] = {dot(d, S.t1), dot(d, S.t2)};
      }
    for (const SP& g : rule) {
      double N[4], dN[4][2];
      shape<double>(nen_s, g.xi, g.eta, N);
      shape_deriv<double>(nen_s, g.xi, g.eta, dN);
      V2<double> x{0.0, 0.0};
      double J00 = 0.0, J01 = 0.0, J10 = 0.0, J11 = 0.0;
      for (int a = 0; a < nen_s; ++a) {
        x.u = x.u + N[a] * pss[a].u;
        x.v = x.v + N[a] * pss[a].v;
        J00 = J00 + dN[a][0] * pss[a].u; J01 = J01 + dN[a][1] * pss[a].u;
        J10 = J10 + dN[a][0] * pss[a].v; J11 = J11 + dN[a][1] * pss[a].v;
      }
      const double W = g.w * std::fabs(J00 * J11 - J01 * J10);
      double Phi[4];
      for (int a = 0; a < nen_s; ++a) {
        Phi[a] = 0.0;
        for (int c = 0; c < nen_s; ++c) Phi[a] = Phi[a] + S.A[a][c] * N[c];
      }
      for (int64_t p = p0; p < p1; ++p) {
        Stats st;
        double xim[2];
        invert_map<double>(nen_m, pmm[p - p0].data(), x, *o, xim, st);
        if (st.newton_fail) continue;
        const bool inside = nen_m == 4
            ? (std::fabs(xim[0]) <= 1.0 + tol_in && std::fabs(xim[1]) <= 1.0 + tol_in)
            : (xim[0] >= -tol_in && xim[1] >= -tol_in && xim[0] + xim[1] <= 1.0 + tol_in);
        if (!inside) continue;
        double Nm[4];
        shape<double>(nen_m, xim[0], xim[1], Nm);
        for (int a = 0; a < nen_s; ++a) {
          const double wp = W * Phi[a];
          for (int l = 0; l < nen_m; ++l) M_out[16 * p + 4 * a + l] += wp * Nm[l];
          if (D_out && o->d_domain == 1)
            for (int b = 0; b < nen_s; ++b) D_out[16 * p + 4 * a + b] += wp * N[b];
        }
        flag[p] = 1;
        break;
      }
    }
  }
  return 0;
}

// Weighted gap functional J = sum_j lambda_j . ((D X_s)_j - (M X_m)_j) and its
// gradient with respect to every slave and master coordinate (or of one of the
// two terms alone, selected by Opts::terms), by forward-mode
// dual numbers: Dual<24> over the 8 nodes of each pair, Dual<12> over the
// slave nodes for the element-domain D.  Contributions are summed in pair
// order, then element order.
int oracle_weighted_gap_grad(const double* xs, int64_t Ns, const int32_t* cs, int64_t Es, int32_t nen_s,
                             const double* xm, int64_t Nm, const int32_t* cm, int32_t nen_m,
                             const Opts* o, const int32_t* ps, const int32_t* pm, int64_t P,
                             const double* lambda, double* J_out, double* gs, double* gm) {
  for (int64_t i = 0; i < 3 * Ns; ++i) gs[i] = 0.0;
  for (int64_t i = 0; i < 3 * Nm; ++i) gm[i] = 0.0;
  typedef Dual<24> D24;
  const int nt = o->n_threads > 0 ? o->n_threads : 1;
  // per-pair value and 24 derivatives, computed independently
  std::vector<double> blk((size_t)P * 25, 0.0);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
#endif
  for (int64_t p = 0; p < P; ++p) {
    Stats st;
    const int32_t s = ps[p], m = pm[p];
    SlaveData<D24> S;
    S.nen = nen_s;
    V3<D24> Xm[4];
    for (int a = 0; a < 4; ++a) S.X[a] = {D24(0.0), D24(0.0), D24(0.0)};
    for (int l = 0; l < 4; ++l) Xm[l] = {D24(0.0), D24(0.0), D24(0.0)};
    for (int a = 0; a < nen_s; ++a) {
      const double* q = xs + 3 * (int64_t)cs[(int64_t)nen_s * s + a];
      S.X[a] = {D24::seed(q[0], 3 * a), D24::seed(q[1], 3 * a + 1), D24::seed(q[2], 3 * a + 2)};
    }
    for (int l = 0; l < nen_m; ++l) {
      const double* q = xm + 3 * (int64_t)cm[(int64_t)nen_m * m + l];
      Xm[l] = {D24::seed(q[0], 12 + 3 * l), D24::seed(q[1], 12 + 3 * l + 1), D24::seed(q[2], 12 + 3 * l + 2)};
    }
    slave_frame<D24>(S);
    lm_coefficients<D24>(S, o->lm);
    PairOut<D24> r;
    integrate_pair<D24>(S, Xm, nen_m, *o, r, st);
    if (!r.nonempty) continue;
    D24 Jp(0.0);
    for (int a = 0; a < nen_s; ++a) {
      const double* lam = lambda + 3 * (int64_t)cs[(int64_t)nen_s * s + a];
      if (o->terms & 2)
        for (int l = 0; l < nen_m; ++l) {
          D24 g = lam[0] * Xm[l].x + lam[1] * Xm[l].y + lam[2] * Xm[l].z;
          Jp = Jp - r.M[a][l] * g;
        }
      if (o->d_domain == 1 && (o->terms & 1))
        for (int b = 0; b < nen_s; ++b) {
          D24 g = lam[0] * S.X[b].x + lam[1] * S.X[b].y + lam[2] * S.X[b].z;
          Jp = Jp + r.D[a][b] * g;
        }
    }
    double* out = blk.data() + 25 * p;
    out[0] = Jp.v;
    for (int k = 0; k < 24; ++k) out[1 + k] = Jp.d[k];
  }
  double J = 0.0;
  for (int64_t p = 0; p < P; ++p) {
    const double* b = blk.data() + 25 * p;
    const int32_t s = ps[p], m = pm[p];
    J += b[0];
    for (int a = 0; a < nen_s; ++a)
      for (int c = 0; c < 3; ++c) gs[3 * (int64_t)cs[(int64_t)nen_s * s + a] + c] += b[1 + 3 * a + c];
    for (int l = 0; l < nen_m; ++l)
      for (int c = 0; c < 3; ++c) gm[3 * (int64_t)cm[(int64_t)nen_m * m + l] + c] += b[13 + 3 * l + c];
  }
  if (o->d_domain == 0 && (o->terms & 1)) {
    typedef Dual<12> D12;
    std::vector<double> eb((size_t)Es * 13, 0.0);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) num_threads(nt)
#endif
    for (int64_t e = 0; e < Es; ++e) {
      SlaveData<D12> S;
      S.nen = nen_s;
      for (int a = 0; a < 4; ++a) S.X[a] = {D12(0.0), D12(0.0), D12(0.0)};
      for (int a = 0; a < nen_s; ++a) {
        const double* q = xs + 3 * (int64_t)cs[(int64_t)nen_s * e + a];
        S.X[a] = {D12::seed(q[0], 3 * a), D12::seed(q[1], 3 * a + 1), D12::seed(q[2], 3 * a + 2)};
      }
      slave_frame<D12>(S);
      lm_coefficients<D12>(S, o->lm);
      D12 De[4][4];
      element_D<D12>(S, De);
      D12 Je(0.0);
      for (int a = 0; a < nen_s; ++a) {
        const double* lam = lambda + 3 * (int64_t)cs[(int64_t)nen_s * e + a];
        for (int b = 0; b < nen_s; ++b) {
          D12 g = lam[0] * S.X[b].x + lam[1] * S.X[b].y + lam[2] * S.X[b].z;
          Je = Je + De[a][b] * g;
        }
      }
      double* out = eb.data() + 13 * e;
      out[0] = Je.v;
      for (int k = 0; k < 12; ++k) out[1 + k] = Je.d[k];
    }
    for (int64_t e = 0; e < Es; ++e) {
      const double* b = eb.data() + 13 * e;
      J += b[0];
      for (int a = 0; a < nen_s; ++a)
        for (int c = 0; c < 3; ++c) gs[3 * (int64_t)cs[(int64_t)nen_s * e + a] + c] += b[1 + 3 * a + c];
    }
  }
  *J_out = J;
  return 0;
}

// Linearisation of the mortar coupling terms (Sec. 1: every nonlinear
// iteration needs the consistent derivatives of D and M), contracted with
// nodal fields ys (Ns x 3) and ym (Nm x 3) that are held fixed:
//   K = d/dX [ (D (x) I3) ys - (M (x) I3) ym ].
// Returned as the dense blocks of its sources, by forward-mode dual numbers
// (Dual<24> over the 8 nodes of a pair, Dual<12> over the nodes of a slave
// element), so that the LM coefficients A (dual basis), the auxiliary plane,
// the clip polygon and the back-projections all carry derivatives:
//   kp[p][a][c][k][d] = [segment D] sum_b dD_p[a][b]/dX_kd ys_b[c]
//                       - sum_l dM_p[a][l]/dX_kd ym_l[c]
//     (a: local slave node = row, c: component, k < 4: slave node k,
//      k >= 4: master node k - 4, d: coordinate direction);
//   ke[e][a][c][k][d] = [element D] sum_b dDe[a][b]/dX_kd ys_b[c]  (k < 4).
// flag[p] = 1 for pairs with a non-empty clip polygon (the structural ones).
int oracle_tangent_blocks(const double* xs, const int32_t* cs, int64_t Es, int32_t nen_s,
                          const double* xm, const int32_t* cm, int32_t nen_m, const Opts* o,
                          const int32_t* ps, const int32_t* pm, int64_t P, const double* ys,
                          const double* ym, double* kp, double* ke, uint8_t* flag) {
  typedef Dual<24> D24;
  const int nt = o->n_threads > 0 ? o->n_threads : 1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
#endif
  for (int64_t p = 0; p < P; ++p) {
    Stats st;
    const int32_t s = ps[p], m = pm[p];
    double* out = kp + 288 * p;
    for (int k = 0; k < 288; ++k) out[k] = 0.0;
    SlaveData<D24> S;
    S.nen = nen_s;
    V3<D24> Xm[4];
    for (int a = 0; a < 4; ++a) S.X[a] = {D24(0.0), D24(0.0), D24(0.0)};
    for (int l = 0; l < 4; ++l) Xm[l] = {D24(0.0), D24(0.0), D24(0.0)};
    for (int a = 0; a < nen_s; ++a) {
      const double* q = xs + 3 * (int64_t)cs[(int64_t)nen_s * s + a];
      S.X[a] = {D24::seed(q[0], 3 * a), D24::seed(q[1], 3 * a + 1), D24::seed(q[2], 3 * a + 2)};
    }
    for (int l = 0; l < nen_m; ++l) {
      const double* q = xm + 3 * (int64_t)cm[(int64_t)nen_m * m + l];
      Xm[l] = {D24::seed(q[0], 12 + 3 * l), D24::seed(q[1], 12 + 3 * l + 1), D24::seed(q[2], 12 + 3 * l + 2)};
    }
    slave_frame<D24>(S);
    lm_coefficients<D24>(S, o->lm);
    PairOut<D24> r;
    integrate_pair<D24>(S, Xm, nen_m, *o, r, st);
    flag[p] = r.nonempty ? 1 : 0;
    if (!r.nonempty) continue;
    for (int a = 0; a < nen_s; ++a)
      for (int c = 0; c < 3; ++c)
        for (int k = 0; k < 24; ++k) {
          double v = 0.0;
          if (o->d_domain == 1)
            for (int b = 0; b < nen_s; ++b)
              v += r.D[a][b].d[k] * ys[3 * (int64_t)cs[(int64_t)nen_s * s + b] + c];
          for (int l = 0; l < nen_m; ++l)
            v -= r.M[a][l].d[k] * ym[3 * (int64_t)cm[(int64_t)nen_m * m + l] + c];
          out[72 * a + 24 * c + k] = v;
        }
  }
  if (o->d_domain == 0) {
    typedef Dual<12> D12;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) num_threads(nt)
#endif
    for (int64_t e = 0; e < Es; ++e) {
      double* out = ke + 144 * e;
      for (int k = 0; k < 144; ++k) out[k] = 0.0;
      SlaveData<D12> S;
      S.nen = nen_s;
      for (int a = 0; a < 4; ++a) S.X[a] = {D12(0.0), D12(0.0), D12(0.0)};
      for (int a = 0; a < nen_s; ++a) {
        const double* q = xs + 3 * (int64_t)cs[(int64_t)nen_s * e + a];
        S.X[a] = {D12::seed(q[0], 3 * a), D12::seed(q[1], 3 * a + 1), D12::seed(q[2], 3 * a + 2)};
      }
      slave_frame<D12>(S);
      lm_coefficients<D12>(S, o->lm);
      D12 De[4][4];
      element_D<D12>(S, De);
      for (int a = 0; a < nen_s; ++a)
        for (int c = 0; c < 3; ++c)
          for (int k = 0; k < 12; ++k) {
            double v = 0.0;
            for (int b = 0; b < nen_s; ++b)
              v += De[a][b].d[k] * ys[3 * (int64_t)cs[(int64_t)nen_s * e + b] + c];
            out[36 * a + 12 * c + k] = v;
          }
    }
  }
  return 0;
}

// Averaged nodal normals of a surface mesh (the continuous normal field of
// Sec. 2.2 used by contact formulations): at each node, the sum over the
// adjacent elements (element order) of each element's unit normal at that
// node's parametric position, normalised.  out: N x 3 (zero for unused nodes).
int oracle_nodal_normals(const double* x, int64_t N, const int32_t* conn, int64_t E, int32_t nen, double* out) {
  for (int64_t i = 0; i < 3 * N; ++i) out[i] = 0.0;
  static const double tri_pts[3][2] = {{0.0, 0.0}, {1.0, 0.0}, {0.0, 1.0}};
  for (int64_t e = 0; e < E; ++e) {
    V3<double> X[4];
    for (int a = 0; a < nen; ++a) {
      const double* q = x + 3 * (int64_t)conn[(int64_t)nen * e + a];
      X[a] = {q[0], q[1], q[2]};
    }
    for (int a = 0; a < nen; ++a) {
      const double xi = nen == 4 ? kQuadCorner[a][0] : tri_pts[a][0];
      const double eta = nen == 4 ? kQuadCorner[a][1] : tri_pts[a][1];
      double dN[4][2];
      shape_deriv<double>(nen, xi, eta, dN);
      V3<double> g1{0.0, 0.0, 0.0}, g2{0.0, 0.0, 0.0};
      for (int b = 0; b < nen; ++b) {
        g1 = {g1.x + dN[b][0] * X[b].x, g1.y + dN[b][0] * X[b].y, g1.z + dN[b][0] * X[b].z};
        g2 = {g2.x + dN[b][1] * X[b].x, g2.y + dN[b][1] * X[b].y, g2.z + dN[b][1] * X[b].z};
      }
      V3<double> n = cross(g1, g2);
      const double ln = std::sqrt(dot(n, n));
      double* o = out + 3 * (int64_t)conn[(int64_t)nen * e + a];
      o[0] += n.x / ln; o[1] += n.y / ln; o[2] += n.z / ln;
    }
  }
  for (int64_t i = 0; i < N; ++i) {
    double* o = out + 3 * i;
    const double l = std::sqrt(o[0] * o[0] + o[1] * o[1] + o[2] * o[2]);
    if (l > 0.0) { o[0] /= l; o[1] /= l; o[2] /= l; }
  }
  return 0;
}

// Unit normal of every element at its centre (quad4 xi = (0, 0), tri3 the
// constant normal): E x 3.
int oracle_element_normals(const double* x, const int32_t* conn, int64_t E, int32_t nen, double* out) {
  for (int64_t e = 0; e < E; ++e) {
    V3<double> X[4];
    for (int a = 0; a < nen; ++a) {
      const double* q = x + 3 * (int64_t)conn[(int64_t)nen * e + a];
      X[a] = {q[0], q[1], q[2]};
    }
    const double xc = nen == 4 ? 0.0 : 1.0 / 3.0;
    double dN[4][2];
    shape_deriv<double>(nen, xc, xc, dN);
    V3<double> g1{0.0, 0.0, 0.0}, g2{0.0, 0.0, 0.0};
    for (int b = 0; b < nen; ++b) {
      g1 = {g1.x + dN[b][0] * X[b].x, g1.y + dN[b][0] * X[b].y, g1.z + dN[b][0] * X[b].z};
      g2 = {g2.x + dN[b][1] * X[b].x, g2.y + dN[b][1] * X[b].y, g2.z + dN[b][1] * X[b].z};
    }
    V3<double> n = cross(g1, g2);
    const double ln = std::sqrt(dot(n, n));
    out[3 * e] = n.x / ln; out[3 * e + 1] = n.y / ln; out[3 * e + 2] = n.z / ln;
  }
  return 0;
}

// Slave auxiliary planes (x0, n0, t1, t2) per element: Es x 12.
int oracle_slave_frames(const double* xs, const int32_t* cs, int64_t Es, int32_t nen_s, double* out) {
  for (int64_t e = 0; e < Es; ++e) {
    SlaveData<double> S;
    load_slave<double>(S, xs, cs, nen_s, e, 0);
    double* o = out + 12 * e;
    o[0] = S.x0.x; o[1] = S.x0.y; o[2] = S.x0.z;
    o[3] = S.n0.x; o[4] = S.n0.y; o[5] = S.n0.z;
    o[6] = S.t1.x; o[7] = S.t1.y; o[8] = S.t1.z;
    o[9] = S.t2.x; o[10] = S.t2.y; o[11] = S.t2.z;
  }
  return 0;
}

// Quadrature rules as used above, for unit checks: which = 7 or 25.
int oracle_tri_rule(int32_t which, double* out, int32_t cap) {
  std::vector<TriPoint> r = which == 25 ? rule_tri_duffy(5) : rule_tri7();
  int n = (int)r.size();
  for (int i = 0; i < n && i < cap; ++i) {
    out[4 * i] = r[i].l0; out[4 * i + 1] = r[i].l1; out[4 * i + 2] = r[i].l2; out[4 * i + 3] = r[i].w;
  }
  return n;
}

// Back-projection on its own (for the Newton pin): p: 4 (or 3) in-plane nodes
// (u, v), x: query point; writes xi[2]; returns 1 if converged.
int oracle_invert_map(int32_t nen, const double* p, const double* x, const Opts* o, double* xi) {
  V2<double> q[4];
  for (int a = 0; a < 4; ++a) q[a] = {0.0, 0.0};
  for (int a = 0; a < nen; ++a) q[a] = {p[2 * a], p[2 * a + 1]};
  Stats st;
  invert_map<double>(nen, q, V2<double>{x[0], x[1]}, *o, xi, st);
  return st.newton_fail == 0 ? 1 : 0;
}


// Quadratic slave elements (tri6, quad8; standard LMs, element-domain D):
// element D blocks (Es x 64, row-major 8 x 8) ...
int oracle_quadratic_element_D(const double* xs, const int32_t* cs, int64_t Es, int32_t nen, double* De) {
  if (nen != 6 && nen != 8) return -1;
  for (int64_t e = 0; e < Es; ++e) {
    V3<double> X[8];
    for (int a = 0; a < 8; ++a) X[a] = {0.0, 0.0, 0.0};
    for (int a = 0; a < nen; ++a) {
      const double* p = xs + 3 * (int64_t)cs[(int64_t)nen * e + a];
      X[a] = {p[0], p[1], p[2]};
    }
    double D[8][8];
    element_D_quadratic(nen, X, D);
    for (int a = 0; a < 8; ++a)
      for (int b = 0; b < 8; ++b) De[64 * e + 8 * a + b] = D[a][b];
  }
  return 0;
}

// ... and per-pair M blocks (P x 32, row-major 8 x 4), nonempty flags, counters.
int oracle_quadratic_pair_blocks(const double* xs, const int32_t* cs, int32_t nen_s, const double* xm,
                                 const int32_t* cm, int32_t nen_m, const Opts* o, const int32_t* ps,
                                 const int32_t* pm, int64_t P, double* M_out, uint8_t* nonempty, int64_t* stats) {
  if (nen_s != 6 && nen_s != 8) return -1;
  for (int k = 0; k < 7; ++k) stats[k] = 0;
  int nt = o->n_threads > 0 ? o->n_threads : 1;
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
  {
    Stats st;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 256)
#endif
    for (int64_t p = 0; p < P; ++p) {
      V3<double> Xp[8], Xm[4];
      for (int a = 0; a < 8; ++a) Xp[a] = {0.0, 0.0, 0.0};
      for (int a = 0; a < nen_s; ++a) {
        const double* q = xs + 3 * (int64_t)cs[(int64_t)nen_s * ps[p] + a];
        Xp[a] = {q[0], q[1], q[2]};
      }
      for (int l = 0; l < 4; ++l) Xm[l] = {0.0, 0.0, 0.0};
      for (int l = 0; l < nen_m; ++l) {
        const double* q = xm + 3 * (int64_t)cm[(int64_t)nen_m * pm[p] + l];
        Xm[l] = {q[0], q[1], q[2]};
      }
      double M[8][4];
      bool ne = false;
      integrate_pair_quadratic(nen_s, Xp, Xm, nen_m, *o, M, ne, st);
      for (int a = 0; a < 8; ++a)
        for (int l = 0; l < 4; ++l) M_out[32 * p + 4 * a + l] = M[a][l];
      nonempty[p] = ne ? 1 : 0;
    }
#ifdef _OPENMP
#pragma omp critical
#endif
    add_stats(stats, st);
  }
  (void)nt;
  return 0;
}

// Quadratic shape functions and their parameter derivatives at one point
// (N: 8, dN: 16 row-major [a][xi, eta]; tri6 fills 6).
int oracle_quadratic_shape(int32_t nen, double xi, double eta, double* N, double* dN) {
  if (nen != 6 && nen != 8) return -1;
  double n[8], d[8][2];
  shape_quadratic(nen, xi, eta, n, d);
  for (int a = 0; a < 8; ++a) { N[a] = n[a]; dN[2 * a] = d[a][0]; dN[2 * a + 1] = d[a][1]; }
  return 0;
}
}  // extern "C"
