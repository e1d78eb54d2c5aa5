// Contact-specific terms on top of the mortar matrices (Sec. 2.1: the
// Hertz-Signorini-Moreau conditions gap >= 0, pressure <= 0,
// gap * pressure = 0, with the gap measured along a continuous normal field):
//   * averaged nodal normals of the slave surface: at each node the sum, over
//     its elements in element order, of the element's unit normal at that
//     node's parametric position, normalised;
//   * weighted normal gap g_j = -n_j . ((D X_s)_j - (M X_m)_j) from the
//     assembled CSR rows (one thread per row, sums in column order);
//   * active set lambda_j + c g_j < 0 and complementarity residual
//     C_j = lambda_j - min(0, lambda_j + c g_j).
// One thread per slave node, fixed summation orders: reproducible.
#include "context.h"

namespace mortar {

namespace {

constexpr int kThreads = 128;

template <int NEN>
__global__ void __launch_bounds__(kThreads) k_nodal_normals(const double* __restrict__ xs,
                                                            const int32_t* __restrict__ conn,
                                                            const int64_t* __restrict__ n2e_ptr,
                                                            const int64_t* __restrict__ n2e_ent, int64_t N,
                                                            double* __restrict__ nrm) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double sx = 0.0, sy = 0.0, sz = 0.0;
  for (int64_t q = n2e_ptr[j]; q < n2e_ptr[j + 1]; ++q) {
    const int64_t e = n2e_ent[q] >> 2;
    const int a = (int)(n2e_ent[q] & 3);
    double X[4][3];
    for (int b = 0; b < NEN; ++b) {
      const int64_t n = conn[(int64_t)NEN * e + b];
      X[b][0] = xs[3 * n]; X[b][1] = xs[3 * n + 1]; X[b][2] = xs[3 * n + 2];
    }
    // tangents at the node's corner of the parameter domain
    double g1[3], g2[3];
    if constexpr (NEN == 4) {
      // quad4 corners (-1,-1), (1,-1), (1,1), (-1,1): at a corner the
      // parametric derivatives reduce to half the differences along the two
      // element edges through it
      // along xi: edge (0-1) at corners 0 and 1, edge (3-2) at corners 3 and 2
      const int x0 = (a == 0 || a == 1) ? 0 : 3, x1 = (a == 0 || a == 1) ? 1 : 2;
      // along eta: edge (0-3) at corners 0 and 3, edge (1-2) at corners 1 and 2
      const int y0 = (a == 0 || a == 3) ? 0 : 1, y1 = (a == 0 || a == 3) ? 3 : 2;
      for (int k = 0; k < 3; ++k) {
        g1[k] = 0.5 * (X[x1][k] - X[x0][k]);
        g2[k] = 0.5 * (X[y1][k] - X[y0][k]);
      }
    } else {
      for (int k = 0; k < 3; ++k) {
        g1[k] = X[1][k] - X[0][k];
        g2[k] = X[2][k] - X[0][k];
      }
    }
    const double nx = g1[1] * g2[2] - g1[2] * g2[1];
    const double ny = g1[2] * g2[0] - g1[0] * g2[2];
    const double nz = g1[0] * g2[1] - g1[1] * g2[0];
    const double l = sqrt(nx * nx + ny * ny + nz * nz);
    sx += nx / l;
    sy += ny / l;
    sz += nz / l;
  }
  const double l = sqrt(sx * sx + sy * sy + sz * sz);
  const double inv = l > 0.0 ? 1.0 / l : 0.0;
  nrm[3 * j] = sx * inv;
  nrm[3 * j + 1] = sy * inv;
  nrm[3 * j + 2] = sz * inv;
}

__global__ void __launch_bounds__(kThreads) k_weighted_gap(
    const int64_t* __restrict__ rpD, const int32_t* __restrict__ ciD, const double* __restrict__ vaD,
    const int64_t* __restrict__ rpM, const int32_t* __restrict__ ciM, const double* __restrict__ vaM,
    const double* __restrict__ xs, const double* __restrict__ xm, const double* __restrict__ nrm, int64_t N,
    double* __restrict__ gap, const double* __restrict__ lam, double cpen, uint8_t* __restrict__ active,
    double* __restrict__ ncp) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double vx = 0.0, vy = 0.0, vz = 0.0;
  for (int64_t q = rpD[j]; q < rpD[j + 1]; ++q) {
    const int64_t k = ciD[q];
    const double d = vaD[q];
    vx += d * xs[3 * k]; vy += d * xs[3 * k + 1]; vz += d * xs[3 * k + 2];
  }
  for (int64_t q = rpM[j]; q < rpM[j + 1]; ++q) {
    const int64_t l = ciM[q];
    const double mm = vaM[q];
    vx -= mm * xm[3 * l]; vy -= mm * xm[3 * l + 1]; vz -= mm * xm[3 * l + 2];
  }
  const double g = -(nrm[3 * j] * vx + nrm[3 * j + 1] * vy + nrm[3 * j + 2] * vz);
  gap[j] = g;
  if (lam) {
    const double t = __dadd_rn(lam[j], __dmul_rn(cpen, g));   // no contraction: the decision is reproducible
    active[j] = t < 0.0 ? 1 : 0;
    ncp[j] = lam[j] - fmin(0.0, t);
  }
}

}  // namespace

void launch_contact_terms(mortar_ctx* c, bool with_ncp, double cpen) {
  const int64_t N = c->Ns;
  if (N == 0) return;
  const unsigned g = (unsigned)((N + kThreads - 1) / kThreads);
  if (c->nen_s == 4)
    k_nodal_normals<4><<<g, kThreads, 0, c->stream>>>(c->xs.as<double>(), c->conn_s.as<int32_t>(),
                                                      c->n2e_s_ptr.as<int64_t>(), c->n2e_s_ent.as<int64_t>(), N,
                                                      c->cn_normals.as<double>());
  else
    k_nodal_normals<3><<<g, kThreads, 0, c->stream>>>(c->xs.as<double>(), c->conn_s.as<int32_t>(),
                                                      c->n2e_s_ptr.as<int64_t>(), c->n2e_s_ent.as<int64_t>(), N,
                                                      c->cn_normals.as<double>());
  k_weighted_gap<<<g, kThreads, 0, c->stream>>>(
      c->rowptr_D.as<int64_t>(), c->col_D.as<int32_t>(), c->val_D.as<double>(), c->rowptr_M.as<int64_t>(),
      c->col_M.as<int32_t>(), c->val_M.as<double>(), c->xs.as<double>(), c->xm.as<double>(),
      c->cn_normals.as<double>(), N, c->cn_gap.as<double>(), with_ncp ? c->cn_lam.as<double>() : nullptr, cpen,
      with_ncp ? c->cn_active.as<uint8_t>() : nullptr, with_ncp ? c->cn_ncp.as<double>() : nullptr);
}

}  // namespace mortar
