// Pieces of the pair geometry shared by the reverse-mode kernels (adjoint of
// the weighted gap, linearisation of D and M): the Sutherland-Hodgman clip
// with its stages recorded (Sec. 2.3, Algorithm 1: master polygon clipped by
// the slave window in the slave element's auxiliary plane), the reverse sweep
// through the clip and merge, and the reverse of the projection onto the
// auxiliary plane (x0, n0, t1, t2 as functions of the slave nodes).  The
// forward decisions are the ones clip_polygon takes, so every kernel agrees on
// which pairs contribute.
#pragma once

#include "common.cuh"

namespace mortar {

constexpr int kPolyA = 10;   // vertex cap per recorded clipping stage (convex polygons need <= 8)

struct V3 {
  double x, y, z;
};
__device__ __forceinline__ V3 v3(double x, double y, double z) { return {x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

template <int NEN>
__device__ __forceinline__ void shape_grad(double xi, double eta, double dN[4][2]) {
  if constexpr (NEN == 4) {
    dN[0][0] = -0.25 * (1.0 - eta); dN[0][1] = -0.25 * (1.0 - xi);
    dN[1][0] = 0.25 * (1.0 - eta);  dN[1][1] = -0.25 * (1.0 + xi);
    dN[2][0] = 0.25 * (1.0 + eta);  dN[2][1] = 0.25 * (1.0 + xi);
    dN[3][0] = -0.25 * (1.0 + eta); dN[3][1] = 0.25 * (1.0 - xi);
  } else {
    dN[0][0] = -1.0; dN[0][1] = -1.0;
    dN[1][0] = 1.0;  dN[1][1] = 0.0;
    dN[2][0] = 0.0;  dN[2][1] = 1.0;
    dN[3][0] = 0.0;  dN[3][1] = 0.0;
  }
}

// Element quadrature point k (same rule as the precomputation).
template <int NEN>
__device__ __forceinline__ void elem_point_a(int k, double& xi, double& eta, double& w) {
  if constexpr (NEN == 4) {
    const double g = 0.7745966692414834;
    const double pp[3] = {-g, 0.0, g};
    const double ww[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
    xi = pp[k / 3];
    eta = pp[k % 3];
    w = ww[k / 3] * ww[k % 3];
  } else {
    tri7_point(k, xi, eta, w);
    w *= 0.5;
  }
}

// Map-coefficient adjoint (c0u c0v c1u c1v c2u c2v c3u c3v) -> in-plane node adjoints.
template <int NEN>
__device__ __forceinline__ void map_coeff_reverse(const double* cb, double* pbu, double* pbv) {
  if constexpr (NEN == 4) {
    const double s1[4] = {-1.0, 1.0, 1.0, -1.0}, s2[4] = {-1.0, -1.0, 1.0, 1.0};
    for (int a = 0; a < 4; ++a) {
      pbu[a] += 0.25 * (cb[0] + s1[a] * cb[2] + s2[a] * cb[4] + s1[a] * s2[a] * cb[6]);
      pbv[a] += 0.25 * (cb[1] + s1[a] * cb[3] + s2[a] * cb[5] + s1[a] * s2[a] * cb[7]);
    }
  } else {
    pbu[0] += cb[0] - cb[2] - cb[4];
    pbv[0] += cb[1] - cb[3] - cb[5];
    pbu[1] += cb[2]; pbv[1] += cb[3];
    pbu[2] += cb[4]; pbv[2] += cb[5];
  }
}

// Clip of one pair with every stage recorded, and its reverse.
template <int NS>
struct ClipRec {
  double Vu[NS + 1][kPolyA], Vv[NS + 1][kPolyA], tt[NS][kPolyA];
  int8_t src[NS][kPolyA];   // output vertex o of stage i: input edge k; +64 if an intersection
  int nv[NS + 1];
  int last = 0, nl = 0, nr = 0;
  int sel[kPolyA];          // merged polygon: vertices of the last stage

  // Master polygon (in-plane coordinates, reversed to CCW if mrev) clipped by
  // the slave window of record r, then merged.  Returns true for a non-empty
  // polygon (same decisions as clip_polygon).
  template <int NM>
  __device__ __forceinline__ bool run(const double* __restrict__ r, const double* mu, const double* mv, bool mrev,
                                      unsigned long long& clip_over) {
    const double eps_in = r[SR_EPSIN];
    const long long eps_bits = __double_as_longlong(eps_in >= 0.0 ? eps_in : 0.0);
    for (int k = 0; k < NM; ++k) {
      const int l = mrev ? NM - 1 - k : k;
      Vu[0][k] = mu[l];
      Vv[0][k] = mv[l];
    }
    nv[0] = NM;
    last = 0;
    for (int i = 0; i < NS; ++i) {
      const int n = nv[i];
      if (n == 0) break;
      const int i1 = i + 1 == NS ? 0 : i + 1;
      const double au = r[SR_PS + 2 * i], av = r[SR_PS + 2 * i + 1];
      const double eu = r[SR_PS + 2 * i1] - au, ev = r[SR_PS + 2 * i1 + 1] - av;
      double d[kPolyA];
      int side[kPolyA];
      for (int k = 0; k < n; ++k) {
        d[k] = cross2(eu, ev, Vu[i][k] - au, Vv[i][k] - av);
        side[k] = band_side(d[k], eps_bits);
      }
      int o = 0;
      for (int k = 0; k < n; ++k) {
        const int k1 = k + 1 == n ? 0 : k + 1;
        const double dp = d[k], dq = d[k1];
        const int sp = side[k], sq = side[k1];
        if ((sp == 1 && sq == -1) || (sp == -1 && sq == 1)) {   // dp, dq beyond the band on both sides
          const double t = dp / (dp - dq);
          if (o < kPolyA) {
            Vu[i + 1][o] = Vu[i][k] + t * (Vu[i][k1] - Vu[i][k]);
            Vv[i + 1][o] = Vv[i][k] + t * (Vv[i][k1] - Vv[i][k]);
            tt[i][o] = t;
            src[i][o] = (int8_t)(k + 64);
          }
          ++o;
        }
        if (sq == 0 || sq == 1) {   // dq >= -eps_in
          if (o < kPolyA) {
            Vu[i + 1][o] = Vu[i][k1];
            Vv[i + 1][o] = Vv[i][k1];
            src[i][o] = (int8_t)k;
          }
          ++o;
        }
      }
      if (o > kPolyA) { clip_over++; o = kPolyA; }
      nv[i + 1] = o;
      last = i + 1;
    }
    // merge consecutive (cyclic) vertices closer than eps_merge: a selection
    const double em2 = r[SR_EPSM2];
    nr = 0;
    nl = nv[last];
    const bool clipped = last == NS;
    for (int k = 0; clipped && k < nl; ++k) {
      if (nr > 0) {
        const double du = Vu[last][k] - Vu[last][sel[nr - 1]], dv = Vv[last][k] - Vv[last][sel[nr - 1]];
        if (du * du + dv * dv < em2) continue;
      }
      sel[nr++] = k;
    }
    while (nr > 1) {
      const double du = Vu[last][sel[nr - 1]] - Vu[last][sel[0]], dv = Vv[last][sel[nr - 1]] - Vv[last][sel[0]];
      if (du * du + dv * dv < em2) --nr; else break;
    }
    double pa2 = 0.0;
    for (int k = 0; k < nr; ++k) {
      const int k1 = k + 1 == nr ? 0 : k + 1;
      pa2 += cross2(Vu[last][sel[k]], Vv[last][sel[k]], Vu[last][sel[k1]], Vv[last][sel[k1]]);
    }
    return eps_in >= 0.0 && clipped && nr >= 3 && !(0.5 * fabs(pa2) < r[SR_EPSA]);
  }

  __device__ __forceinline__ double pu(int k) const { return Vu[last][sel[k]]; }
  __device__ __forceinline__ double pv(int k) const { return Vv[last][sel[k]]; }

  // Reverse of merge and clip: adjoints (Rbu, Rbv) of the nr merged vertices
  // are ADDED to the in-plane adjoints of the slave nodes (sbu, sbv; element
  // node order) and of the master nodes (mbu, mbv).
  template <int NM>
  __device__ __forceinline__ void reverse(const double* __restrict__ r, const double* Rbu, const double* Rbv,
                                          bool srev, bool mrev, double* sbu, double* sbv, double* mbu,
                                          double* mbv) const {
    double Bu[NS + 1][kPolyA], Bv[NS + 1][kPolyA];
    for (int k = 0; k < nl; ++k) { Bu[last][k] = 0.0; Bv[last][k] = 0.0; }
    for (int k = 0; k < nr; ++k) { Bu[last][sel[k]] += Rbu[k]; Bv[last][sel[k]] += Rbv[k]; }
    double Wbu[4] = {0, 0, 0, 0}, Wbv[4] = {0, 0, 0, 0};
    for (int i = NS - 1; i >= 0; --i) {
      const int n = nv[i];
      const int i1 = i + 1 == NS ? 0 : i + 1;
      const double au = r[SR_PS + 2 * i], av = r[SR_PS + 2 * i + 1];
      const double eu = r[SR_PS + 2 * i1] - au, ev = r[SR_PS + 2 * i1 + 1] - av;
      for (int k = 0; k < n; ++k) { Bu[i][k] = 0.0; Bv[i][k] = 0.0; }
      double abu2 = 0.0, abv2 = 0.0, ebu = 0.0, ebv = 0.0;
      for (int o = 0; o < nv[i + 1]; ++o) {
        const double gbu = Bu[i + 1][o], gbv = Bv[i + 1][o];
        const int code = src[i][o];
        const int k = code & 63;
        const int k1 = k + 1 == n ? 0 : k + 1;
        if (code < 64) {   // copied vertex
          Bu[i][k1] += gbu;
          Bv[i][k1] += gbv;
          continue;
        }
        // intersection x = p + t (q - p), t = d_p / (d_p - d_q),
        // d = eu (y_v - a_v) - ev (y_u - a_u) for y = p, q
        const double tk = tt[i][o];
        const double pu_ = Vu[i][k], pv_ = Vv[i][k], qu = Vu[i][k1], qv = Vv[i][k1];
        Bu[i][k] += (1.0 - tk) * gbu; Bv[i][k] += (1.0 - tk) * gbv;
        Bu[i][k1] += tk * gbu;        Bv[i][k1] += tk * gbv;
        const double tb = gbu * (qu - pu_) + gbv * (qv - pv_);
        const double dp = cross2(eu, ev, pu_ - au, pv_ - av);
        const double dq = cross2(eu, ev, qu - au, qv - av);
        const double den = dp - dq;
        const double i2 = 1.0 / (den * den);
        const double dpb = -tb * dq * i2, dqb = tb * dp * i2;
        Bu[i][k] += -ev * dpb;  Bv[i][k] += eu * dpb;
        Bu[i][k1] += -ev * dqb; Bv[i][k1] += eu * dqb;
        abu2 += ev * (dpb + dqb);
        abv2 += -eu * (dpb + dqb);
        ebu += (pv_ - av) * dpb + (qv - av) * dqb;
        ebv += -(pu_ - au) * dpb - (qu - au) * dqb;
      }
      Wbu[i] += abu2 - ebu; Wbv[i] += abv2 - ebv;
      Wbu[i1] += ebu;       Wbv[i1] += ebv;
    }
    for (int k = 0; k < NS; ++k) {
      const int a = srev ? NS - 1 - k : k;
      sbu[a] += Wbu[k];
      sbv[a] += Wbv[k];
    }
    for (int k = 0; k < NM; ++k) {
      const int l = mrev ? NM - 1 - k : k;
      mbu[l] += Bu[0][k];
      mbv[l] += Bv[0][k];
    }
  }
};

// Compact clip record: the same Sutherland-Hodgman clip and merge as
// ClipRec (identical arithmetic and decisions), recorded as a pool of
// vertices instead of whole stages.  Pool slots [0, NM) are the master
// polygon's vertices (counter-clockwise), every later slot is an edge
// intersection x = p + t (q - p) made at stage i from pool slots p and q; a
// copied vertex keeps its slot.  The working polygon of a stage is a list of
// 4-bit slot ids packed into 64 bits.  Reverse: slots are visited from the
// last intersection down, so that each slot's adjoint is complete before it
// is passed on to its two parents and to the clip edge.
template <int NS, int NM>
struct ClipPool {
  static constexpr int kSlots = 12;   // master vertices + intersections (convex quads: <= 4 + 8)
  double pu[kSlots], pv[kSlots], tt[kSlots];
  uint16_t meta[kSlots];              // intersection: p | q << 4 | stage << 8
  int nv = 0, nr = 0;
  uint64_t poly = 0;                  // merged polygon: slot ids, 4 bits each

  __device__ __forceinline__ int id(int k) const { return (int)((poly >> (4 * k)) & 15); }
  __device__ __forceinline__ double u(int k) const { return pu[id(k)]; }
  __device__ __forceinline__ double v(int k) const { return pv[id(k)]; }

  __device__ __forceinline__ bool run(const double* __restrict__ r, const double* mu, const double* mv, bool mrev,
                                      unsigned long long& clip_over) {
    const double eps_in = r[SR_EPSIN];
    const long long eps_bits = __double_as_longlong(eps_in >= 0.0 ? eps_in : 0.0);
    uint64_t cur = 0;
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      const int l = mrev ? NM - 1 - k : k;
      pu[k] = mu[l];
      pv[k] = mv[l];
      cur |= (uint64_t)k << (4 * k);
    }
    nv = NM;
    int n = NM;
    bool over = false;
    for (int i = 0; i < NS && n > 0; ++i) {
      const int i1 = i + 1 == NS ? 0 : i + 1;
      const double au = r[SR_PS + 2 * i], av = r[SR_PS + 2 * i + 1];
      const double eu = r[SR_PS + 2 * i1] - au, ev = r[SR_PS + 2 * i1 + 1] - av;
      const int id0 = (int)(cur & 15);
      const double d0 = cross2(eu, ev, pu[id0] - au, pv[id0] - av);
      const int s0 = band_side(d0, eps_bits);
      double dp = d0;
      int sp = s0, idp = id0;
      uint64_t nxt = 0;
      int o = 0;
      for (int k = 0; k < n; ++k) {
        const int k1 = k + 1 == n ? 0 : k + 1;
        const int idq = (int)((cur >> (4 * k1)) & 15);
        double dq;
        int sq;
        if (k1 == 0) {
          dq = d0;
          sq = s0;
        } else {
          dq = cross2(eu, ev, pu[idq] - au, pv[idq] - av);
          sq = band_side(dq, eps_bits);
        }
        if ((sp == 1 && sq == -1) || (sp == -1 && sq == 1)) {   // dp, dq beyond the band on both sides
          const double t = dp / (dp - dq);
          if (nv < kSlots && o < 16) {
            pu[nv] = pu[idp] + t * (pu[idq] - pu[idp]);
            pv[nv] = pv[idp] + t * (pv[idq] - pv[idp]);
            tt[nv] = t;
            meta[nv] = (uint16_t)(idp | (idq << 4) | (i << 8));
            nxt |= (uint64_t)nv << (4 * o);
            ++nv;
            ++o;
          } else {
            over = true;
          }
        }
        if (sq == 0 || sq == 1) {   // dq >= -eps_in
          if (o < 16) {
            nxt |= (uint64_t)idq << (4 * o);
            ++o;
          } else {
            over = true;
          }
        }
        dp = dq;
        sp = sq;
        idp = idq;
      }
      cur = nxt;
      n = o;
    }
    if (over) {   // cannot happen for convex elements; reported, pair dropped
      clip_over++;
      nr = 0;
      return false;
    }
    // merge consecutive (cyclic) vertices closer than eps_merge: a selection
    const double em2 = r[SR_EPSM2];
    nr = 0;
    poly = 0;
    int last_id = -1, first_id = -1;
    for (int k = 0; k < n; ++k) {
      const int q = (int)((cur >> (4 * k)) & 15);
      if (nr > 0) {
        const double du = pu[q] - pu[last_id], dv = pv[q] - pv[last_id];
        if (du * du + dv * dv < em2) continue;
      } else {
        first_id = q;
      }
      poly |= (uint64_t)q << (4 * nr);
      last_id = q;
      ++nr;
    }
    while (nr > 1) {
      const int q = id(nr - 1);
      const double du = pu[q] - pu[first_id], dv = pv[q] - pv[first_id];
      if (du * du + dv * dv < em2) {
        --nr;
        poly &= ~((uint64_t)15 << (4 * nr));
      } else {
        break;
      }
    }
    double pa2 = 0.0;
    for (int k = 0; k < nr; ++k) {
      const int a = id(k), b = id(k + 1 == nr ? 0 : k + 1);
      pa2 += cross2(pu[a], pv[a], pu[b], pv[b]);
    }
    return eps_in >= 0.0 && nr >= 3 && !(0.5 * fabs(pa2) < r[SR_EPSA]);
  }

  // Reverse of merge and clip.  Bu, Bv (kSlots, caller-owned) hold on entry
  // the adjoints of the merged polygon's vertices ADDED at their slots (all
  // other slots zero); the in-plane adjoints of the slave window vertices
  // (element node order) and of the master nodes are ADDED to sbu, sbv, mbu, mbv.
  __device__ __forceinline__ void reverse(const double* __restrict__ r, double* Bu, double* Bv, bool srev,
                                          bool mrev, double* sbu, double* sbv, double* mbu, double* mbv) const {
    double Wbu[NS], Wbv[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) { Wbu[k] = 0.0; Wbv[k] = 0.0; }
    for (int w = nv - 1; w >= NM; --w) {
      const double gbu = Bu[w], gbv = Bv[w];
      const int p = meta[w] & 15, q = (meta[w] >> 4) & 15, i = meta[w] >> 8;
      const int i1 = i + 1 == NS ? 0 : i + 1;
      const double au = r[SR_PS + 2 * i], av = r[SR_PS + 2 * i + 1];
      const double eu = r[SR_PS + 2 * i1] - au, ev = r[SR_PS + 2 * i1 + 1] - av;
      // intersection x = p + t (q - p), t = d_p / (d_p - d_q),
      // d = eu (y_v - a_v) - ev (y_u - a_u) for y = p, q
      const double tk = tt[w];
      const double pu_ = pu[p], pv_ = pv[p], qu = pu[q], qv = pv[q];
      const double tb = gbu * (qu - pu_) + gbv * (qv - pv_);
      const double dp = cross2(eu, ev, pu_ - au, pv_ - av);
      const double dq = cross2(eu, ev, qu - au, qv - av);
      const double den = dp - dq;
      const double i2 = 1.0 / (den * den);
      const double dpb = -tb * dq * i2, dqb = tb * dp * i2;
      Bu[p] += (1.0 - tk) * gbu - ev * dpb;
      Bv[p] += (1.0 - tk) * gbv + eu * dpb;
      Bu[q] += tk * gbu - ev * dqb;
      Bv[q] += tk * gbv + eu * dqb;
      const double abu2 = ev * (dpb + dqb), abv2 = -eu * (dpb + dqb);
      const double ebu = (pv_ - av) * dpb + (qv - av) * dqb;
      const double ebv = -(pu_ - au) * dpb - (qu - au) * dqb;
#pragma unroll
      for (int s = 0; s < NS; ++s) {   // window vertices i and i + 1 (registers, no indexed array)
        const int s1 = s + 1 == NS ? 0 : s + 1;
        if (s == i) {
          Wbu[s] += abu2 - ebu;
          Wbv[s] += abv2 - ebv;
          Wbu[s1] += ebu;
          Wbv[s1] += ebv;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const int a = srev ? NS - 1 - k : k;
      sbu[a] += Wbu[k];
      sbv[a] += Wbv[k];
    }
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      const int l = mrev ? NM - 1 - k : k;
      mbu[l] += Bu[k];
      mbv[l] += Bv[k];
    }
  }
};

// Reverse of the projection u = (P - x0).t1, v = (P - x0).t2 of every node of
// the pair and of the auxiliary plane (x0 = element centre, n0 = unit normal
// there, t1 = normalised projected first edge, t2 = n0 x t1) as functions of
// the slave nodes X.  In-plane node adjoints (sbu, sbv, mbu, mbv) in; 3D
// coordinate adjoints ADDED to gX (slave) and gY (master).
template <int NS, int NM>
__device__ __forceinline__ void plane_reverse(const V3* X, const V3* Y, V3 x0, V3 t1, V3 t2, V3 n0,
                                              const double* sbu, const double* sbv, const double* mbu,
                                              const double* mbv, double gX[4][3], double gY[4][3]) {
  V3 x0b = v3(0, 0, 0), t1b = v3(0, 0, 0), t2b = v3(0, 0, 0);
  for (int a = 0; a < NS; ++a) {
    const V3 dd = X[a] - x0;
    const V3 db = sbu[a] * t1 + sbv[a] * t2;
    gX[a][0] += db.x; gX[a][1] += db.y; gX[a][2] += db.z;
    x0b = x0b - db;
    t1b = t1b + sbu[a] * dd;
    t2b = t2b + sbv[a] * dd;
  }
  for (int l = 0; l < NM; ++l) {
    const V3 dd = Y[l] - x0;
    const V3 db = mbu[l] * t1 + mbv[l] * t2;
    gY[l][0] += db.x; gY[l][1] += db.y; gY[l][2] += db.z;
    x0b = x0b - db;
    t1b = t1b + mbu[l] * dd;
    t2b = t2b + mbv[l] * dd;
  }
  V3 g1, g2;
  if constexpr (NS == 4) {
    g1 = 0.25 * ((X[1] - X[0]) + (X[2] - X[3]));
    g2 = 0.25 * ((X[2] - X[1]) + (X[3] - X[0]));
  } else {
    g1 = X[1] - X[0];
    g2 = X[2] - X[0];
  }
  const V3 nn = cross(g1, g2);
  const double ln = sqrt(dot(nn, nn));
  const V3 ed = X[1] - X[0];
  const double en = dot(ed, n0);
  const V3 ep = ed - en * n0;
  const double le = sqrt(dot(ep, ep));
  V3 n0b = cross(t1, t2b);   // t2 = n0 x t1
  t1b = t1b + cross(t2b, n0);
  const V3 epb = (1.0 / le) * (t1b - dot(t1, t1b) * t1);
  V3 edb = epb;
  const double enb = -dot(epb, n0);
  n0b = n0b - en * epb;
  edb = edb + enb * n0;
  n0b = n0b + enb * ed;
  const V3 nb = (1.0 / ln) * (n0b - dot(n0, n0b) * n0);
  const V3 g1b = cross(g2, nb), g2b = cross(nb, g1);
  V3 Xb[4];
  for (int a = 0; a < 4; ++a) Xb[a] = v3(0, 0, 0);
  Xb[1] = Xb[1] + edb;
  Xb[0] = Xb[0] - edb;
  if constexpr (NS == 4) {
    const V3 a1 = 0.25 * g1b, a2 = 0.25 * g2b, ax = 0.25 * x0b;
    Xb[0] = Xb[0] - a1 - a2 + ax;
    Xb[1] = Xb[1] + a1 - a2 + ax;
    Xb[2] = Xb[2] + a1 + a2 + ax;
    Xb[3] = Xb[3] - a1 + a2 + ax;
  } else {
    const V3 ax = (1.0 / 3.0) * x0b;
    Xb[0] = Xb[0] - g1b - g2b + ax;
    Xb[1] = Xb[1] + g1b + ax;
    Xb[2] = Xb[2] + g2b + ax;
  }
  for (int a = 0; a < NS; ++a) {
    gX[a][0] += Xb[a].x; gX[a][1] += Xb[a].y; gX[a][2] += Xb[a].z;
  }
}

// Monomial form of the element shape functions, N(xi) = T m(xi): quad4
// m = (1, xi, eta, xi eta) and row a of T is (1, xi_a, eta_a, xi_a eta_a) / 4
// with the corners (xi_a, eta_a) = (-1,-1), (1,-1), (1,1), (-1,1); tri3
// m = (1, xi, eta) and N = (1 - xi - eta, xi, eta).  A bilinear form
// N_s^T P N_m of nodal quantities equals m_s^T (T_s^T P T_m) m_m, which a
// quadrature point evaluates without forming N.

// out_i = sum_a T[a][i] in_a: monomial coefficients of the nodal field `in`.
template <int NEN>
__device__ __forceinline__ void nodal_to_mono(const V3* in, V3* out) {
  if constexpr (NEN == 4) {
    const V3 s02 = in[0] + in[2], s13 = in[1] + in[3], d20 = in[2] - in[0], d13 = in[1] - in[3];
    out[0] = 0.25 * (s02 + s13);
    out[1] = 0.25 * (d20 + d13);
    out[2] = 0.25 * (d20 - d13);
    out[3] = 0.25 * (s02 - s13);
  } else {
    out[0] = in[0];
    out[1] = in[1] - in[0];
    out[2] = in[2] - in[0];
  }
}

}  // namespace mortar
