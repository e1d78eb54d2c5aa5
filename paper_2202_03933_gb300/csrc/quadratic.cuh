// Quadratic slave elements (tri6, quad8) on the device: shape functions and
// the four linear sub-elements of the piecewise flat approximation of the
// slave surface (Sec. 2.3), with the affine maps from a sub-element's
// parameters to the parent element's.
//
// quad8 (serendipity): corners 0..3 at (-1,-1), (1,-1), (1,1), (-1,1),
// mid-side nodes 4..7 at (0,-1), (1,0), (0,1), (-1,0):
//   corner:   N = (1 + xi xi_a)(1 + eta eta_a)(xi xi_a + eta eta_a - 1) / 4,
//   xi_a = 0: N = (1 - xi^2)(1 + eta eta_a) / 2,  eta_a = 0: N = (1 + xi xi_a)(1 - eta^2) / 2.
// tri6: corners 0..2 at (0,0), (1,0), (0,1), mid-side nodes 3 (edge 0-1),
// 4 (edge 1-2), 5 (edge 2-0); with L = (1 - xi - eta, xi, eta):
//   corner i: N = L_i (2 L_i - 1),  mid-side (i, j): N = 4 L_i L_j.
// Sub-elements, counter-clockwise like the parent (-1 = the quad8 centre):
//   quad8 -> quad4 (0, 4, c, 7), (4, 1, 5, c), (c, 5, 2, 6), (7, c, 6, 3);
//   tri6  -> tri3  (0, 3, 5), (3, 1, 4), (5, 4, 2), (3, 4, 5).
#pragma once

#include "common.cuh"

namespace mortar {

template <int NP>
__device__ __forceinline__ void shape_quadratic(double xi, double eta, double N[8]) {
  if constexpr (NP == 8) {
    const double xm = 1.0 - xi, xp = 1.0 + xi, em = 1.0 - eta, ep = 1.0 + eta;
    N[0] = 0.25 * xm * em * (-xi - eta - 1.0);
    N[1] = 0.25 * xp * em * (xi - eta - 1.0);
    N[2] = 0.25 * xp * ep * (xi + eta - 1.0);
    N[3] = 0.25 * xm * ep * (-xi + eta - 1.0);
    const double bx = 0.5 * (1.0 - xi * xi), by = 0.5 * (1.0 - eta * eta);
    N[4] = bx * em;
    N[5] = xp * by;
    N[6] = bx * ep;
    N[7] = xm * by;
  } else {
    const double L0 = 1.0 - xi - eta, L1 = xi, L2 = eta;
    N[0] = L0 * (2.0 * L0 - 1.0);
    N[1] = L1 * (2.0 * L1 - 1.0);
    N[2] = L2 * (2.0 * L2 - 1.0);
    N[3] = 4.0 * L0 * L1;
    N[4] = 4.0 * L1 * L2;
    N[5] = 4.0 * L2 * L0;
    N[6] = 0.0;
    N[7] = 0.0;
  }
}

// Parameter derivatives dN[a][0] = dN_a/dxi, dN[a][1] = dN_a/deta.
template <int NP>
__device__ __forceinline__ void shape_quadratic_grad(double xi, double eta, double dN[8][2]) {
  if constexpr (NP == 8) {
    const double xm = 1.0 - xi, xp = 1.0 + xi, em = 1.0 - eta, ep = 1.0 + eta;
    dN[0][0] = 0.25 * em * (2.0 * xi + eta);   dN[0][1] = 0.25 * xm * (xi + 2.0 * eta);
    dN[1][0] = 0.25 * em * (2.0 * xi - eta);   dN[1][1] = 0.25 * xp * (2.0 * eta - xi);
    dN[2][0] = 0.25 * ep * (2.0 * xi + eta);   dN[2][1] = 0.25 * xp * (xi + 2.0 * eta);
    dN[3][0] = 0.25 * ep * (2.0 * xi - eta);   dN[3][1] = 0.25 * xm * (2.0 * eta - xi);
    dN[4][0] = -xi * em;                       dN[4][1] = -0.5 * (1.0 - xi * xi);
    dN[5][0] = 0.5 * (1.0 - eta * eta);        dN[5][1] = -eta * xp;
    dN[6][0] = -xi * ep;                       dN[6][1] = 0.5 * (1.0 - xi * xi);
    dN[7][0] = -0.5 * (1.0 - eta * eta);       dN[7][1] = -eta * xm;
  } else {
    const double L0 = 1.0 - xi - eta, L1 = xi, L2 = eta;
    dN[0][0] = -(4.0 * L0 - 1.0);   dN[0][1] = -(4.0 * L0 - 1.0);
    dN[1][0] = 4.0 * L1 - 1.0;      dN[1][1] = 0.0;
    dN[2][0] = 0.0;                 dN[2][1] = 4.0 * L2 - 1.0;
    dN[3][0] = 4.0 * (L0 - L1);     dN[3][1] = -4.0 * L1;
    dN[4][0] = 4.0 * L2;            dN[4][1] = 4.0 * L1;
    dN[5][0] = -4.0 * L2;           dN[5][1] = 4.0 * (L0 - L2);
    dN[6][0] = dN[6][1] = dN[7][0] = dN[7][1] = 0.0;
  }
}

// Corner j of sub-element k: parent local node, or -1 for the quad8 centre.
template <int NP>
__device__ __forceinline__ int sub_node(int k, int j) {
  if constexpr (NP == 8) {
    constexpr int t[4][4] = {{0, 4, -1, 7}, {4, 1, 5, -1}, {-1, 5, 2, 6}, {7, -1, 6, 3}};
    return t[k][j];
  } else {
    constexpr int t[4][3] = {{0, 3, 5}, {3, 1, 4}, {5, 4, 2}, {3, 4, 5}};
    return t[k][j];
  }
}

// Parent parameters of the point with parameters (xs, es) of sub-element k.
template <int NP>
__device__ __forceinline__ void sub_to_parent(int k, double xs, double es, double& xp, double& ep) {
  if constexpr (NP == 8) {
    const double sx = (k == 1 || k == 2) ? 1.0 : -1.0, sy = k >= 2 ? 1.0 : -1.0;
    xp = 0.5 * (xs + sx);
    ep = 0.5 * (es + sy);
  } else {
    switch (k) {
      case 0: xp = 0.5 * xs;        ep = 0.5 * es; break;
      case 1: xp = 0.5 + 0.5 * xs;  ep = 0.5 * es; break;
      case 2: xp = 0.5 * xs;        ep = 0.5 + 0.5 * es; break;
      default: xp = 0.5 - 0.5 * es; ep = 0.5 * (xs + es); break;
    }
  }
}

}  // namespace mortar
