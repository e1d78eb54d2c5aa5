// Deterministic assembly of D and M into CSR (Eq. DiscreteWeakFormInterfaceFlux:
// the matrices are assembled from nodal blocks).
//
// Rows are slave nodes.  One thread gathers every contribution to its row --
// from the slave elements around the node (node -> element adjacency, sorted
// by element), and for each such element from its pairs (contiguous, in
// (s, m) order) -- sorts the column ids stably and sums equal columns in
// gather order.  There are no floating-point atomics, so results are bitwise
// reproducible run to run.  A count pass sizes the rows, a scan builds
// rowptr, a write pass fills colidx / vals.
//
// Topology (node -> element adjacency of each side) is built once per
// interface with a counting sort plus a per-node sort of the short lists.
#include "context.h"

namespace mortar {

namespace {

constexpr int kThreads = 128;

template <int NEN>
__global__ void k_adj_count(const int32_t* __restrict__ conn, int64_t E, int32_t* __restrict__ cnt) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  for (int a = 0; a < NEN; ++a) atomicAdd(&cnt[conn[NEN * e + a]], 1);
}

template <int NEN>
__global__ void k_adj_fill(const int32_t* __restrict__ conn, int64_t E, const int64_t* __restrict__ ptr,
                           int32_t* __restrict__ cnt, int64_t* __restrict__ ent) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  for (int a = 0; a < NEN; ++a) {
    const int32_t n = conn[NEN * e + a];
    const int32_t slot = atomicSub(&cnt[n], 1) - 1;
    ent[ptr[n] + slot] = e * 4 + a;
  }
}

__global__ void k_adj_sort(const int64_t* __restrict__ ptr, int64_t N, int64_t* __restrict__ ent) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t b0 = ptr[i], b1 = ptr[i + 1];
  for (int64_t a = b0 + 1; a < b1; ++a) {
    const int64_t v = ent[a];
    int64_t b = a - 1;
    while (b >= b0 && ent[b] > v) { ent[b + 1] = ent[b]; --b; }
    ent[b + 1] = v;
  }
}

// Entry source of one row.  WHICH: 0 = element-domain D, 1 = segment D, 2 = M.
template <int WHICH, int NS, int NM>
struct RowSource {
  const int64_t* n2e_ptr;
  const int64_t* n2e_ent;
  const int64_t* pair_off;
  const int32_t* pm;
  const uint8_t* flag;
  const double* blk;       // De (per element) or Dblk / Mblk (per pair)
  const int32_t* conn_s;
  const int32_t* conn_m;

  template <class F>
  __device__ __forceinline__ void visit(int64_t j, F&& f) const {
    const int64_t q0 = n2e_ptr[j], q1 = n2e_ptr[j + 1];
    for (int64_t q = q0; q < q1; ++q) {
      const int64_t ee = n2e_ent[q];
      const int64_t e = ee >> 2;
      const int a = (int)(ee & 3);
      if (WHICH == 0) {
        for (int b = 0; b < NS; ++b) f(conn_s[NS * e + b], blk[16 * e + 4 * a + b]);
      } else {
        const int64_t p0 = pair_off[e], p1 = pair_off[e + 1];
        for (int64_t p = p0; p < p1; ++p) {
          if (!flag[p]) continue;
          if (WHICH == 1) {
            for (int b = 0; b < NS; ++b) f(conn_s[NS * e + b], blk[16 * p + 4 * a + b]);
          } else {
            const int64_t m = pm[p];
            for (int l = 0; l < NM; ++l) f(conn_m[NM * m + l], blk[16 * p + 4 * a + l]);
          }
        }
      }
    }
  }
};

// MODE 0: count unique columns of each row; MODE 1: write the row.
template <int MODE, class Src>
__global__ void __launch_bounds__(kThreads) k_rows(Src src, int64_t N, int32_t* __restrict__ row_cnt,
                                                   const int64_t* __restrict__ rowptr, int64_t nnz_cap,
                                                   int32_t* __restrict__ col_out, double* __restrict__ val_out,
                                                   DevStatus* st, int which_over) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  if (st->over_pairs) {   // pair buffers incomplete: the run is repeated with larger ones
    if (MODE == 0) row_cnt[j] = 0;
    return;
  }
  if (MODE == 1 && rowptr[N] > nnz_cap) {
    if (j == 0) atomicMax(&st->over_nnz, (unsigned long long)rowptr[N]);
    return;
  }
  int32_t col[kMaxRow];
  double val[kMaxRow];
  int k = 0;
  src.visit(j, [&](int32_t c, double v) {
    if (k < kMaxRow) {   // stable insertion by column
      int b = k - 1;
      while (b >= 0 && col[b] > c) { col[b + 1] = col[b]; val[b + 1] = val[b]; --b; }
      col[b + 1] = c;
      val[b + 1] = v;
    }
    ++k;
  });
  int64_t out = MODE == 1 ? rowptr[j] : 0;
  if (k <= kMaxRow) {
    int u = 0;
    for (int a = 0; a < k;) {
      const int32_t c = col[a];
      double s = 0.0;
      while (a < k && col[a] == c) s += val[a++];
      if (MODE == 1) { col_out[out + u] = c; val_out[out + u] = s; }
      ++u;
    }
    if (MODE == 0) row_cnt[j] = u;
    return;
  }
  // long row: repeated selection of the next column, sums in gather order
  if (MODE == 0 && which_over == 0) atomicAdd(&st->row_slow, 1ull);
  int u = 0;
  int32_t last = -1;
  for (;;) {
    int32_t next = 0x7fffffff;
    src.visit(j, [&](int32_t c, double) { if (c > last && c < next) next = c; });
    if (next == 0x7fffffff) break;
    double s = 0.0;
    src.visit(j, [&](int32_t c, double v) { if (c == next) s += v; });
    if (MODE == 1) { col_out[out + u] = next; val_out[out + u] = s; }
    ++u;
    last = next;
  }
  if (MODE == 0) row_cnt[j] = u;
}

__global__ void k_finalize(const int64_t* __restrict__ rpD, const int64_t* __restrict__ rpM, int64_t N,
                           DevStatus* st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    st->nnz_D = (unsigned long long)rpD[N];
    st->nnz_M = (unsigned long long)rpM[N];
  }
}

template <int WHICH, int NS, int NM>
void assemble_one(mortar_ctx* c, const double* blk, mortar::DevBuf& rowptr, mortar::DevBuf& col,
                  mortar::DevBuf& val, int64_t cap, int which_over) {
  RowSource<WHICH, NS, NM> src{c->n2e_s_ptr.as<int64_t>(), c->n2e_s_ent.as<int64_t>(), c->pair_off.as<int64_t>(),
                               c->pairs_m.as<int32_t>(), c->flag.as<uint8_t>(), blk, c->conn_s.as<int32_t>(),
                               c->conn_m.as<int32_t>()};
  DevStatus* st = c->dstat.as<DevStatus>();
  const int64_t N = c->Ns;
  const unsigned g = (unsigned)((N + kThreads - 1) / kThreads);
  if (N > 0)
    k_rows<0><<<g, kThreads, 0, c->stream>>>(src, N, c->row_cnt.as<int32_t>(), nullptr, 0, nullptr, nullptr, st,
                                              which_over);
  launch_exclusive_scan_i32(c->row_cnt.as<int32_t>(), rowptr.as<int64_t>(), nullptr, N, c->scan_tmp.as<int64_t>(),
                            c->stream);
  if (N > 0)
    k_rows<1><<<g, kThreads, 0, c->stream>>>(src, N, nullptr, rowptr.as<int64_t>(), cap, col.as<int32_t>(),
                                              val.as<double>(), st, which_over);
}

template <int NS, int NM>
void assemble_nsnm(mortar_ctx* c, const RunParams& rp) {
  if (rp.d_domain == 1)
    assemble_one<1, NS, NM>(c, c->Dblk.as<double>(), c->rowptr_D, c->col_D, c->val_D, c->nnz_cap_D, 0);
  else
    assemble_one<0, NS, NM>(c, c->De.as<double>(), c->rowptr_D, c->col_D, c->val_D, c->nnz_cap_D, 0);
  assemble_one<2, NS, NM>(c, c->Mblk.as<double>(), c->rowptr_M, c->col_M, c->val_M, c->nnz_cap_M, 1);
}

}  // namespace

void launch_topology(mortar_ctx* c) {
  for (int side = 0; side < 2; ++side) {
    const int64_t N = side == 0 ? c->Ns : c->Nm;
    const int64_t E = side == 0 ? c->Es : c->Em;
    const int nen = side == 0 ? c->nen_s : c->nen_m;
    const int32_t* conn = (side == 0 ? c->conn_s : c->conn_m).as<int32_t>();
    DevBuf& ptr = side == 0 ? c->n2e_s_ptr : c->n2e_m_ptr;
    DevBuf& ent = side == 0 ? c->n2e_s_ent : c->n2e_m_ent;
    int32_t* cnt = c->row_cnt.as<int32_t>();
    cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)(N > 0 ? N : 1), c->stream);
    const unsigned ge = (unsigned)((E + kThreads - 1) / kThreads);
    if (E > 0) {
      if (nen == 4) k_adj_count<4><<<ge, kThreads, 0, c->stream>>>(conn, E, cnt);
      else k_adj_count<3><<<ge, kThreads, 0, c->stream>>>(conn, E, cnt);
    }
    launch_exclusive_scan_i32(cnt, ptr.as<int64_t>(), nullptr, N, c->scan_tmp.as<int64_t>(), c->stream);
    if (E > 0) {
      if (nen == 4) k_adj_fill<4><<<ge, kThreads, 0, c->stream>>>(conn, E, ptr.as<int64_t>(), cnt, ent.as<int64_t>());
      else k_adj_fill<3><<<ge, kThreads, 0, c->stream>>>(conn, E, ptr.as<int64_t>(), cnt, ent.as<int64_t>());
    }
    if (N > 0)
      k_adj_sort<<<(unsigned)((N + kThreads - 1) / kThreads), kThreads, 0, c->stream>>>(ptr.as<int64_t>(), N,
                                                                                        ent.as<int64_t>());
  }
}

void launch_assemble(mortar_ctx* c, const RunParams& rp) {
  if (c->nen_s == 4 && c->nen_m == 4) assemble_nsnm<4, 4>(c, rp);
  else if (c->nen_s == 4 && c->nen_m == 3) assemble_nsnm<4, 3>(c, rp);
  else if (c->nen_s == 3 && c->nen_m == 4) assemble_nsnm<3, 4>(c, rp);
  else assemble_nsnm<3, 3>(c, rp);
}

void launch_finalize_status(mortar_ctx* c) {
  k_finalize<<<1, 32, 0, c->stream>>>(c->rowptr_D.as<int64_t>(), c->rowptr_M.as<int64_t>(), c->Ns,
                                      c->dstat.as<DevStatus>());
}

}  // namespace mortar
