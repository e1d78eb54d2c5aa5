// Binned contact search (Sec. 3.5, Algorithm 2, restated for one device).
//
// Master elements are sorted into the bins of their interface's grid by the
// centre of their inflated bounding box (counting sort: per-bin counts, a
// device-wide scan, an atomic fill).  Each slave element then tests the
// master elements in its own bin and the 26 neighbouring bins and keeps those
// whose delta-inflated boxes overlap (closed comparison; only min/max/add and
// compares, so the decision is bitwise the same as the brute-force
// definition).  Candidate counts are scanned into per-slave offsets and each
// slave element writes its master ids sorted ascending, so pairs come out
// sorted by (s, m) regardless of the fill order within a bin.
#include "context.h"

namespace mortar {

namespace {

constexpr int kThreads = 128;
constexpr int kLocalCand = 64;

__device__ __forceinline__ int32_t iface_of(const int64_t* __restrict__ off, int32_t n_if, int64_t e) {
  int32_t lo = 0, hi = n_if - 1;   // last interface whose offset <= e
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void bin_coords(const GridParams& g, const double* b, int32_t ijk[3]) {
  for (int k = 0; k < 3; ++k) {
    const double c = 0.5 * (b[k] + b[3 + k]);
    double t = floor((c - g.org[k]) / g.beta[k]);
    t = fmin(fmax(t, 0.0), (double)(g.nb[k] - 1));
    ijk[k] = (int32_t)t;
  }
}

__global__ void k_zero_i32(int32_t* __restrict__ p, const unsigned long long* n_dev) {
  const int64_t n = (int64_t)*n_dev;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0;
}

__global__ void __launch_bounds__(kThreads) k_master_keys(const double* __restrict__ box_m,
                                                          const int64_t* __restrict__ me_off, int32_t n_if,
                                                          int64_t Em, const GridParams* __restrict__ grid,
                                                          int64_t* __restrict__ key, int32_t* __restrict__ cnt,
                                                          const DevStatus* st) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= Em || st->over_bins) return;
  const int32_t i = iface_of(me_off, n_if, m);
  const GridParams g = grid[i];
  int32_t ijk[3];
  bin_coords(g, box_m + 8 * m, ijk);
  const int64_t k = g.bin_off + ((int64_t)ijk[2] * g.nb[1] + ijk[1]) * g.nb[0] + ijk[0];
  key[m] = k;
  atomicAdd(&cnt[k], 1);
}

__global__ void __launch_bounds__(kThreads) k_master_fill(const int64_t* __restrict__ key, int64_t Em,
                                                          const int64_t* __restrict__ start,
                                                          int32_t* __restrict__ cnt, int32_t* __restrict__ elems,
                                                          const DevStatus* st) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= Em || st->over_bins) return;
  const int64_t k = key[m];
  const int32_t slot = atomicSub(&cnt[k], 1) - 1;
  elems[start[k] + slot] = (int32_t)m;
}

__device__ __forceinline__ bool overlap(const double* a, const double* b) {
  return a[0] <= b[3] && b[0] <= a[3] && a[1] <= b[4] && b[1] <= a[4] && a[2] <= b[5] && b[2] <= a[5];
}

// Visits the candidates of slave element s; mode 0 counts, mode 1 writes.
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_candidates(
    const double* __restrict__ box_s, const double* __restrict__ box_m, const int64_t* __restrict__ se_off,
    int32_t n_if, int64_t Es, const GridParams* __restrict__ grid, const int64_t* __restrict__ start,
    const int32_t* __restrict__ elems, int32_t* __restrict__ cnt, const int64_t* __restrict__ pair_off,
    int64_t pair_cap, int32_t* __restrict__ ps, int32_t* __restrict__ pm, const double* __restrict__ srec,
    const double* __restrict__ nrm_m, DevStatus* st) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Es || st->over_bins) return;
  if (MODE == 1 && pair_off[Es] > pair_cap) {
    if (s == 0) st->over_pairs = (unsigned long long)pair_off[Es];
    return;
  }
  const int32_t i = iface_of(se_off, n_if, s);
  const GridParams g = grid[i];
  double bs[6];
  for (int k = 0; k < 6; ++k) bs[k] = box_s[8 * s + k];
  int32_t ijk[3];
  bin_coords(g, box_s + 8 * s, ijk);
  // facing test (optional): slave normal n0 of the element record vs the master centre normal
  double nsx = 0.0, nsy = 0.0, nsz = 0.0;
  if (nrm_m) {
    const double* r = srec + (int64_t)SR_STRIDE * s;
    nsx = r[SR_N0]; nsy = r[SR_N0 + 1]; nsz = r[SR_N0 + 2];
  }
  int32_t local[kLocalCand];
  int32_t n = 0;
  const int64_t base = MODE == 1 ? pair_off[s] : 0;
  for (int dz = -1; dz <= 1; ++dz) {
    const int32_t kz = ijk[2] + dz;
    if (kz < 0 || kz >= g.nb[2]) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int32_t ky = ijk[1] + dy;
      if (ky < 0 || ky >= g.nb[1]) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int32_t kx = ijk[0] + dx;
        if (kx < 0 || kx >= g.nb[0]) continue;
        const int64_t bin = g.bin_off + ((int64_t)kz * g.nb[1] + ky) * g.nb[0] + kx;
        const int64_t b0 = start[bin], b1 = start[bin + 1];
        for (int64_t q = b0; q < b1; ++q) {
          const int32_t m = elems[q];
          if (!overlap(bs, box_m + 8 * (int64_t)m)) continue;
          if (nrm_m) {
            const double* q = nrm_m + 3 * (int64_t)m;
            if (!(nsx * q[0] + nsy * q[1] + nsz * q[2] < 0.0)) continue;
          }
          if (MODE == 1) {
            if (n < kLocalCand) local[n] = m;
            pm[base + n] = m;   // also written in place for the long-list path
          }
          ++n;
        }
      }
    }
  }
  if (MODE == 0) {
    cnt[s] = n;
    return;
  }
  if (n <= kLocalCand) {
    for (int a = 1; a < n; ++a) {   // insertion sort, ascending master id
      const int32_t v = local[a];
      int b = a - 1;
      while (b >= 0 && local[b] > v) { local[b + 1] = local[b]; --b; }
      local[b + 1] = v;
    }
    for (int a = 0; a < n; ++a) {
      pm[base + a] = local[a];
      ps[base + a] = (int32_t)s;
    }
  } else {
    for (int a = 1; a < n; ++a) {
      const int32_t v = pm[base + a];
      int b = a - 1;
      while (b >= 0 && pm[base + b] > v) { pm[base + b + 1] = pm[base + b]; --b; }
      pm[base + b + 1] = v;
    }
    for (int a = 0; a < n; ++a) ps[base + a] = (int32_t)s;
  }
}

__global__ void k_pairs_total(const int64_t* __restrict__ pair_off, int64_t Es, DevStatus* st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) st->n_pairs = (unsigned long long)pair_off[Es];
}

}  // namespace

void launch_bin_masters(mortar_ctx* c) {
  DevStatus* st = c->dstat.as<DevStatus>();
  const unsigned zg = (unsigned)(c->n_sm * 8);
  k_zero_i32<<<zg, 256, 0, c->stream>>>(c->bin_cnt.as<int32_t>(), &st->n_bins);
  if (c->Em > 0)
    k_master_keys<<<(unsigned)((c->Em + kThreads - 1) / kThreads), kThreads, 0, c->stream>>>(
        c->box_m.as<double>(), c->me_off.as<int64_t>(), c->n_if, c->Em, c->grid.as<GridParams>(),
        c->mkey.as<int64_t>(), c->bin_cnt.as<int32_t>(), st);
  launch_exclusive_scan_i32(c->bin_cnt.as<int32_t>(), c->bin_start.as<int64_t>(),
                            reinterpret_cast<const int64_t*>(&st->n_bins), c->bin_cap, c->scan_tmp.as<int64_t>(),
                            c->stream);
  if (c->Em > 0)
    k_master_fill<<<(unsigned)((c->Em + kThreads - 1) / kThreads), kThreads, 0, c->stream>>>(
        c->mkey.as<int64_t>(), c->Em, c->bin_start.as<int64_t>(), c->bin_cnt.as<int32_t>(),
        c->bin_elems.as<int32_t>(), st);
}

void launch_candidates(mortar_ctx* c) {
  DevStatus* st = c->dstat.as<DevStatus>();
  const unsigned g = (unsigned)((c->Es + kThreads - 1) / kThreads);
  if (c->Es > 0)
    k_candidates<0><<<g, kThreads, 0, c->stream>>>(
        c->box_s.as<double>(), c->box_m.as<double>(), c->se_off.as<int64_t>(), c->n_if, c->Es,
        c->grid.as<GridParams>(), c->bin_start.as<int64_t>(), c->bin_elems.as<int32_t>(), c->cand_cnt.as<int32_t>(),
        nullptr, 0, nullptr, nullptr, c->srec.as<double>(), c->opt.facing_test ? c->nrm_m.as<double>() : nullptr,
        st);
  launch_exclusive_scan_i32(c->cand_cnt.as<int32_t>(), c->pair_off.as<int64_t>(), nullptr, c->Es,
                            c->scan_tmp.as<int64_t>(), c->stream);
  k_pairs_total<<<1, 32, 0, c->stream>>>(c->pair_off.as<int64_t>(), c->Es, st);
  if (c->Es > 0)
    k_candidates<1><<<g, kThreads, 0, c->stream>>>(
        c->box_s.as<double>(), c->box_m.as<double>(), c->se_off.as<int64_t>(), c->n_if, c->Es,
        c->grid.as<GridParams>(), c->bin_start.as<int64_t>(), c->bin_elems.as<int32_t>(), nullptr,
        c->pair_off.as<int64_t>(), c->pair_cap, c->pairs_s.as<int32_t>(), c->pairs_m.as<int32_t>(),
        c->srec.as<double>(), c->opt.facing_test ? c->nrm_m.as<double>() : nullptr, st);
}

}  // namespace mortar
