// Per-pair geometry shared by the integration and adjoint kernels, so that
// both take identical decisions: projection and clipping of one slave/master
// pair (Sec. 2.3, Algorithm 1: project the master element onto the slave
// element's auxiliary plane, find the intersection by clipping) and the
// inverse of an element map in that plane (chi_h).
#pragma once

#include "common.cuh"

namespace mortar {

constexpr int kPolyS = 10;   // stored clip-polygon vertices (convex quad vs quad: <= 8)

// Projection of the master element, its map, and the clipped, merged polygon
// (Pu, Pv, nr vertices; nr = 0 when the pair contributes nothing).
template <int NS, int NM, int CAP>
__device__ __forceinline__ int clip_polygon(const double* __restrict__ r, const double* __restrict__ xm,
                                            const int32_t* __restrict__ conn_m, int32_t m, PlaneMap& mmap,
                                            double* Pu, double* Pv,
                                            unsigned long long& clip_over) {
  const double eps_in = r[SR_EPSIN];
  if (!(eps_in >= 0.0)) return 0;
  const long long eps_bits = __double_as_longlong(eps_in);
  const double x0x = r[SR_X0], x0y = r[SR_X0 + 1], x0z = r[SR_X0 + 2];
  const double t1x = r[SR_T1], t1y = r[SR_T1 + 1], t1z = r[SR_T1 + 2];
  const double t2x = r[SR_T2], t2y = r[SR_T2 + 1], t2z = r[SR_T2 + 2];
  double mu[4], mv[4];
#pragma unroll
  for (int l = 0; l < NM; ++l) {
    const int64_t n = conn_m[(int64_t)NM * m + l];
    const double dx = xm[3 * n] - x0x, dy = xm[3 * n + 1] - x0y, dz = xm[3 * n + 2] - x0z;
    mu[l] = dx * t1x + dy * t1y + dz * t1z;
    mv[l] = dx * t2x + dy * t2y + dz * t2z;
  }
  mmap = plane_map<NM>(mu, mv);
  double ma2 = 0.0;
#pragma unroll
  for (int l = 0; l < NM; ++l) ma2 += cross2(mu[l], mv[l], mu[(l + 1) % NM], mv[(l + 1) % NM]);
  double Qu[kMaxPoly], Qv[kMaxPoly], d[kMaxPoly];
  double Wu[kMaxPoly], Wv[kMaxPoly];   // working polygon
#pragma unroll
  for (int l = 0; l < NM; ++l) {
    const int src = ma2 < 0.0 ? NM - 1 - l : l;
    Wu[l] = mu[src];
    Wv[l] = mv[src];
  }
  int n = NM;
  for (int i = 0; i < NS && n > 0; ++i) {
    const int i1 = i + 1 == NS ? 0 : i + 1;
    const double au = r[SR_PS + 2 * i], av = r[SR_PS + 2 * i + 1];
    const double eu = r[SR_PS + 2 * i1] - au, ev = r[SR_PS + 2 * i1 + 1] - av;
    int side[kMaxPoly];
    for (int k = 0; k < n; ++k) {
      d[k] = cross2(eu, ev, Wu[k] - au, Wv[k] - av);
      side[k] = band_side(d[k], eps_bits);
    }
    int o = 0;
    for (int k = 0; k < n; ++k) {
      const int k1 = k + 1 == n ? 0 : k + 1;
      const double dp = d[k], dq = d[k1];
      const int sp = side[k], sq = side[k1];
      if ((sp == 1 && sq == -1) || (sp == -1 && sq == 1)) {   // dp, dq beyond the band on both sides
        const double t = dp / (dp - dq);
        if (o < kMaxPoly) {
          Qu[o] = Wu[k] + t * (Wu[k1] - Wu[k]);
          Qv[o] = Wv[k] + t * (Wv[k1] - Wv[k]);
        }
        ++o;
      }
      if (sq == 0 || sq == 1) {   // dq >= -eps_in
        if (o < kMaxPoly) { Qu[o] = Wu[k1]; Qv[o] = Wv[k1]; }
        ++o;
      }
    }
    if (o > kMaxPoly) { clip_over++; o = kMaxPoly; }
    for (int k = 0; k < o; ++k) { Wu[k] = Qu[k]; Wv[k] = Qv[k]; }
    n = o;
  }
  // merge consecutive (cyclic) vertices closer than eps_merge
  const double em2 = r[SR_EPSM2];
  int nr = 0;
  for (int k = 0; k < n; ++k) {
    if (nr > 0) {
      const double du = Wu[k] - Wu[nr - 1], dv = Wv[k] - Wv[nr - 1];
      if (du * du + dv * dv < em2) continue;
    }
    Wu[nr] = Wu[k];
    Wv[nr] = Wv[k];
    ++nr;
  }
  while (nr > 1) {
    const double du = Wu[nr - 1] - Wu[0], dv = Wv[nr - 1] - Wv[0];
    if (du * du + dv * dv < em2) --nr; else break;
  }
  double pa2 = 0.0;
  for (int k = 0; k < nr; ++k) {
    const int k1 = k + 1 == nr ? 0 : k + 1;
    pa2 += cross2(Wu[k], Wv[k], Wu[k1], Wv[k1]);
  }
  if (nr < 3 || 0.5 * fabs(pa2) < r[SR_EPSA]) return 0;
  if (nr > CAP) {   // cannot happen for convex elements; reported, pair dropped
    clip_over++;
    return 0;
  }
  for (int k = 0; k < nr; ++k) { Pu[k] = Wu[k]; Pv[k] = Wv[k]; }
  return nr;
}

// Vertex count of a pair's clipped and merged polygon, computed in FP32 with
// the steps of clip_polygon (0 when the FP32 polygon is empty), and the number
// of edge intersections the clip created (n_int).  Used only as the key that
// groups pairs of similar cost: the FP64 clip decides what a pair contributes.
// Coordinates are O(element size) apart, so FP32 keeps them to ~1e-4 of an
// element; near-degenerate pairs may get other counts.
template <int NS, int NM>
__device__ __forceinline__ int clip_count_f32(const double* __restrict__ r, const double* __restrict__ xm,
                                              const int32_t* __restrict__ conn_m, int32_t m, int& n_int) {
  n_int = 0;
  const double eps_in = r[SR_EPSIN];
  if (!(eps_in >= 0.0)) return 0;
  const float ein = f32_trunc(eps_in);
  const float x0x = f32_trunc(r[SR_X0]), x0y = f32_trunc(r[SR_X0 + 1]), x0z = f32_trunc(r[SR_X0 + 2]);
  const float t1x = f32_trunc(r[SR_T1]), t1y = f32_trunc(r[SR_T1 + 1]), t1z = f32_trunc(r[SR_T1 + 2]);
  const float t2x = f32_trunc(r[SR_T2]), t2y = f32_trunc(r[SR_T2 + 1]), t2z = f32_trunc(r[SR_T2 + 2]);
  constexpr int CAP = 12;
  float Wu[CAP], Wv[CAP], Qu[CAP], Qv[CAP], d[CAP];
  float mu[4], mv[4];
#pragma unroll
  for (int l = 0; l < NM; ++l) {
    const int64_t n = conn_m[(int64_t)NM * m + l];
    const float dx = f32_trunc(xm[3 * n]) - x0x, dy = f32_trunc(xm[3 * n + 1]) - x0y,
                dz = f32_trunc(xm[3 * n + 2]) - x0z;
    mu[l] = fmaf(dz, t1z, fmaf(dy, t1y, dx * t1x));
    mv[l] = fmaf(dz, t2z, fmaf(dy, t2y, dx * t2x));
  }
  float ma2 = 0.0f;
#pragma unroll
  for (int l = 0; l < NM; ++l) {
    const int l1 = (l + 1) % NM;
    ma2 += mu[l] * mv[l1] - mv[l] * mu[l1];
  }
#pragma unroll
  for (int l = 0; l < NM; ++l) {
    const int src = ma2 < 0.0f ? NM - 1 - l : l;
    Wu[l] = mu[src];
    Wv[l] = mv[src];
  }
  int n = NM;
  for (int i = 0; i < NS && n > 0; ++i) {
    const int i1 = i + 1 == NS ? 0 : i + 1;
    const float au = f32_trunc(r[SR_PS + 2 * i]), av = f32_trunc(r[SR_PS + 2 * i + 1]);
    const float eu = f32_trunc(r[SR_PS + 2 * i1]) - au, ev = f32_trunc(r[SR_PS + 2 * i1 + 1]) - av;
    for (int k = 0; k < n; ++k) d[k] = eu * (Wv[k] - av) - ev * (Wu[k] - au);
    int o = 0;
    for (int k = 0; k < n; ++k) {
      const int k1 = k + 1 == n ? 0 : k + 1;
      const float dp = d[k], dq = d[k1];
      if ((dp > ein && dq < -ein) || (dp < -ein && dq > ein)) {
        const float t = dp / (dp - dq);
        if (o < CAP) { Qu[o] = fmaf(t, Wu[k1] - Wu[k], Wu[k]); Qv[o] = fmaf(t, Wv[k1] - Wv[k], Wv[k]); }
        ++o;
        ++n_int;
      }
      if (dq >= -ein) {
        if (o < CAP) { Qu[o] = Wu[k1]; Qv[o] = Wv[k1]; }
        ++o;
      }
    }
    if (o > CAP) o = CAP;
    for (int k = 0; k < o; ++k) { Wu[k] = Qu[k]; Wv[k] = Qv[k]; }
    n = o;
  }
  const float em2 = f32_trunc(r[SR_EPSM2]);
  int nr = 0;
  for (int k = 0; k < n; ++k) {
    if (nr > 0) {
      const float du = Wu[k] - Wu[nr - 1], dv = Wv[k] - Wv[nr - 1];
      if (du * du + dv * dv < em2) continue;
    }
    Wu[nr] = Wu[k];
    Wv[nr] = Wv[k];
    ++nr;
  }
  while (nr > 1) {
    const float du = Wu[nr - 1] - Wu[0], dv = Wv[nr - 1] - Wv[0];
    if (du * du + dv * dv < em2) --nr; else break;
  }
  float pa2 = 0.0f;
  for (int k = 0; k < nr; ++k) {
    const int k1 = k + 1 == nr ? 0 : k + 1;
    pa2 += Wu[k] * Wv[k1] - Wv[k] * Wu[k1];
  }
  if (nr < 3 || 0.5f * fabsf(pa2) < f32_trunc(r[SR_EPSA])) return 0;
  return nr;
}

// The FP32 Newton iteration's last Jacobian inverse of a bilinear map, in the
// map's own (unscaled) units, and the FP32 reciprocal of its scaled
// determinant.
struct CoarseInv {
  float g00, g01, g10, g11;
  float idf;
};

// Inverse of an element map in the plane for many query points: affine maps
// by a 2x2 inverse, bilinear ones by FP32 Newton on coordinates scaled by a
// power of two (error e0 ~ 1e-7 in xi), then one Newton step with the FP64
// residual and the FP32 iteration's last Jacobian inverse (relative error
// d ~ 1e-7): the step leaves ~d e0 + |c3|/|J| e0^2 ~ 1e-14 in xi, the same
// converged value as a full FP64 Newton to rounding.  The reverse sweep's
// Jacobian inverse at the converged xi uses the FP64 Jacobian there, with
// 1 / det one Newton-Raphson reciprocal step from the FP32 reciprocal
// (~1e-14).  Conversions between FP32 and FP64 are integer operations
// (f32_trunc, f64_of_f32): a conversion instruction with an FP64 operand
// issues on the FP64 pipe.
struct MapInverse {
  PlaneMap m;
  bool affine;
  double i00, i01, i10, i11;        // affine: exact inverse of [c1 c2]
  double sc, sc2;                   // power-of-two scale and its square
  float scf;                        // the scale in FP32
  float f1u, f1v, f2u, f2v, f3u, f3v;
  float b00, b01, b10, b11;         // FP32 inverse of the scaled [c1 c2]
  double id_seed;                   // 1 / det J near the last solve's point, to ~1e-7 (seed for jinv, jinvT)

  __device__ __forceinline__ void setup(const PlaneMap& mp, bool is_affine) {
    m = mp;
    affine = is_affine;
    if (affine) {
      const double id = 1.0 / (m.c1u * m.c2v - m.c2u * m.c1v);
      i00 = m.c2v * id; i01 = -m.c2u * id; i10 = -m.c1v * id; i11 = m.c1u * id;
      return;
    }
    const double L = fmax(fmax(fabs(m.c1u), fabs(m.c1v)), fmax(fabs(m.c2u), fabs(m.c2v)));
    int e = 0;
    frexp(L, &e);
    sc = ldexp(1.0, -e);   // exact power of two, L * sc in [0.5, 1)
    sc2 = sc * sc;
    scf = ldexpf(1.0f, -e);   // the same scale in FP32 (exact)
    f1u = f32_trunc(m.c1u) * scf; f1v = f32_trunc(m.c1v) * scf;
    f2u = f32_trunc(m.c2u) * scf; f2v = f32_trunc(m.c2v) * scf;
    f3u = f32_trunc(m.c3u) * scf; f3v = f32_trunc(m.c3v) * scf;
    const float fd = 1.0f / (f1u * f2v - f2u * f1v);
    b00 = f2v * fd; b01 = -f2u * fd; b10 = -f1v * fd; b11 = f1u * fd;
  }

  // Inverse of the Jacobian at the (xi, eta) of the last solve to ~1e-13 (the
  // reverse sweep's implicit-function step); 1 / det as in jinvT
  __device__ __forceinline__ void jinv(double xi, double eta, double& a00, double& a01, double& a10,
                                       double& a11) const {
    if (affine) {
      a00 = i00; a01 = i01; a10 = i10; a11 = i11;
      return;
    }
    const double j00 = fma(m.c3u, eta, m.c1u), j01 = fma(m.c3u, xi, m.c2u);
    const double j10 = fma(m.c3v, eta, m.c1v), j11 = fma(m.c3v, xi, m.c2v);
    const double det = fma(j00, j11, -j01 * j10);
    const double id = fma(id_seed, fma(-det, id_seed, 1.0), id_seed);
    a00 = j11 * id; a01 = -j01 * id; a10 = -j10 * id; a11 = j00 * id;
  }

  // J^-T b at the (xi, eta) of the last solve (the implicit-function step of
  // a reverse sweep): (j11 b0 - j10 b1, j00 b1 - j01 b0) / det, without
  // forming the inverse.  1 / det is one Newton-Raphson reciprocal iteration
  // from id_seed (the FP32 iteration's last reciprocal, ~1e-7 relative
  // error, which the iteration squares to ~1e-14).
  __device__ __forceinline__ void jinvT(double xi, double eta, double b0, double b1, double& mu,
                                        double& mv) const {
    if (affine) {
      mu = fma(i00, b0, i10 * b1);
      mv = fma(i01, b0, i11 * b1);
      return;
    }
    const double j00 = fma(m.c3u, eta, m.c1u), j01 = fma(m.c3u, xi, m.c2u);
    const double j10 = fma(m.c3v, eta, m.c1v), j11 = fma(m.c3v, xi, m.c2v);
    const double det = fma(j00, j11, -j01 * j10);
    const double id = fma(id_seed, fma(-det, id_seed, 1.0), id_seed);
    mu = id * fma(j11, b0, -j10 * b1);
    mv = id * fma(j00, b1, -j01 * b0);
  }

  // FP32 Newton of a bilinear map (error ~1e-7 in xi); false if it did not
  // settle.  ci: the last iteration's FP32 Jacobian inverse (taken at a point
  // within that iteration's step, <= 3e-7, of the returned xi) and 1 / det.
  __device__ __forceinline__ bool coarse(double xu, double xv, double& xi, double& eta, CoarseInv& ci) const {
    const double du = xu - m.c0u, dv = xv - m.c0v;
    const float tu = f32_trunc(du) * scf, tv = f32_trunc(dv) * scf;
    float x = b00 * tu + b01 * tv, y = b10 * tu + b11 * tv;
    float j00 = f1u, j01 = f2u, j10 = f1v, j11 = f2v, id = 0.0f;
    bool conv = false;
#pragma unroll 1
    for (int it = 0; it < 16; ++it) {
      const float ru = fmaf(f3u * x, y, fmaf(f1u, x, fmaf(f2u, y, -tu)));
      const float rv = fmaf(f3v * x, y, fmaf(f1v, x, fmaf(f2v, y, -tv)));
      j00 = fmaf(f3u, y, f1u); j01 = fmaf(f3u, x, f2u);
      j10 = fmaf(f3v, y, f1v); j11 = fmaf(f3v, x, f2v);
      id = __frcp_rn(j00 * j11 - j01 * j10);
      const float d0 = (j11 * ru - j01 * rv) * id, d1 = (j00 * rv - j10 * ru) * id;
      x -= d0;
      y -= d1;
      if (fabsf(d0) + fabsf(d1) <= 3e-7f) { conv = true; break; }
    }
    // the scaled map is scf J: J^-1 = scf (scf J)^-1 (scf a power of two)
    const float is = id * scf;
    ci.g00 = j11 * is; ci.g01 = -j01 * is; ci.g10 = -j10 * is; ci.g11 = j00 * is;
    ci.idf = id;
    xi = f64_of_f32(x);
    eta = f64_of_f32(y);
    return conv;
  }

  // One Newton step of a bilinear map from the FP32 iterate (xi, eta): FP64
  // residual r = (c1 + c3 eta) xi + c2 eta - d, step G r with G the FP32
  // iteration's last Jacobian inverse.  G differs from J(xi, eta)^-1 by a
  // relative ~1e-7 (FP32 rounding, and the last FP32 step <= 3e-7), so the
  // step leaves an error of ~1e-7 x the iterate's own ~1e-7 error, the same
  // order as the quadratic term of an exact-Jacobian step.
  __device__ __forceinline__ void polish(double xu, double xv, double& xi, double& eta, const CoarseInv& ci) {
    const double du = xu - m.c0u, dv = xv - m.c0v;
    const double j00 = fma(m.c3u, eta, m.c1u), j10 = fma(m.c3v, eta, m.c1v);
    const double ru = fma(j00, xi, fma(m.c2u, eta, -du));
    const double rv = fma(j10, xi, fma(m.c2v, eta, -dv));
    const double g00 = f64_of_f32(ci.g00), g01 = f64_of_f32(ci.g01);
    const double g10 = f64_of_f32(ci.g10), g11 = f64_of_f32(ci.g11);
    xi = fma(-g00, ru, fma(-g01, rv, xi));
    eta = fma(-g10, ru, fma(-g11, rv, eta));
    id_seed = f64_of_f32(ci.idf) * sc2;
  }

  // FP64 Newton from the current (xi, eta), with the oracle's stopping rule:
  // stop once |dxi|_inf <= 1e-14, then apply one more update; at most 20
  // updates.  Taken only when the FP32 iteration did not settle (strongly
  // distorted elements: a corner angle near 180 degrees makes the FP32
  // Jacobian too inaccurate for its 3e-7 step test).
  __device__ __forceinline__ bool newton64(double xu, double xv, double& xi, double& eta) {
    const double du = xu - m.c0u, dv = xv - m.c0v;
    bool last = false;
    for (int it = 0; it < 20; ++it) {
      const double j00 = fma(m.c3u, eta, m.c1u), j01 = fma(m.c3u, xi, m.c2u);
      const double j10 = fma(m.c3v, eta, m.c1v), j11 = fma(m.c3v, xi, m.c2v);
      const double ru = fma(j00, xi, fma(m.c2u, eta, -du));
      const double rv = fma(j10, xi, fma(m.c2v, eta, -dv));
      const double id = 1.0 / (j00 * j11 - j01 * j10);
      id_seed = id;
      const double d0 = (j11 * ru - j01 * rv) * id, d1 = (j00 * rv - j10 * ru) * id;
      xi -= d0;
      eta -= d1;
      if (last) return true;
      if (fmax(fabs(d0), fabs(d1)) <= 1e-14) last = true;
    }
    return false;
  }

  // Converged xi of a point; false only if the FP64 fallback did not converge
  // either (xi then is the last iterate).
  __device__ __forceinline__ bool solve(double xu, double xv, double& xi, double& eta) {
    if (affine) {
      const double du = xu - m.c0u, dv = xv - m.c0v;
      xi = i00 * du + i01 * dv;
      eta = i10 * du + i11 * dv;
      return true;
    }
    CoarseInv ci;
    if (!coarse(xu, xv, xi, eta, ci)) return newton64(xu, xv, xi, eta);
    polish(xu, xv, xi, eta, ci);
    return true;
  }
};

// Shape functions and the pull-back of a shape-function adjoint to xi:
// quad4 with a = 1 - xi, b = 1 + xi, c = 1 - eta, d = 1 + eta:
//   N = (a c, b c, b d, a d) / 4,  dN/dxi = (-c, c, d, -d) / 4,  dN/deta = (-a, -b, b, a) / 4.
template <int NEN>
struct ShapeAD {
  double N[4];
  double qa, qb, qc, qd;
  __device__ __forceinline__ void eval(double xi, double eta) {
    if constexpr (NEN == 4) {
      qa = 0.25 * (1.0 - xi); qb = 0.25 * (1.0 + xi);
      const double c = 1.0 - eta, d = 1.0 + eta;
      qc = 0.25 * c; qd = 0.25 * d;
      N[0] = qa * c; N[1] = qb * c; N[2] = qb * d; N[3] = qa * d;
    } else {
      N[0] = 1.0 - xi - eta; N[1] = xi; N[2] = eta; N[3] = 0.0;
    }
  }
  // (dxi, deta) += sum_k Nb[k] grad N_k
  __device__ __forceinline__ void pull(const double* Nb, double& g0, double& g1) const {
    if constexpr (NEN == 4) {
      g0 = fma(qc, Nb[1] - Nb[0], qd * (Nb[2] - Nb[3]));
      g1 = fma(qa, Nb[3] - Nb[0], qb * (Nb[2] - Nb[1]));
    } else {
      g0 = Nb[1] - Nb[0];
      g1 = Nb[2] - Nb[0];
    }
  }
};

}  // namespace mortar
