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
  for (int a = 0; a < NEN; ++a) atomicAdd(&cnt[conn[(int64_t)NEN * e + a]], 1);
}

// Entry of the adjacency: element e, local node a, as e << kLocalBits(NEN) | a.
template <int NEN>
constexpr int kLocalBits = NEN > 4 ? 3 : 2;

template <int NEN>
__global__ void k_adj_fill(const int32_t* __restrict__ conn, int64_t E, const int64_t* __restrict__ ptr,
                           int32_t* __restrict__ cnt, int64_t* __restrict__ ent) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  for (int a = 0; a < NEN; ++a) {
    const int32_t n = conn[(int64_t)NEN * e + a];
    const int32_t slot = atomicSub(&cnt[n], 1) - 1;
    ent[ptr[n] + slot] = (e << kLocalBits<NEN>) | a;
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
// Blocks: linear slave elements 4 x 4 (16 per element or pair); quadratic
// slave elements 8 x 8 element D (64) and 8 x 4 pair M (32).
template <int WHICH, int NS, int NM>
struct RowSource {
  static constexpr int kRowW = NS > 4 ? 8 : 4;   // slave-side block row width
  const int64_t* n2e_ptr;
  const int64_t* n2e_ent;
  const int64_t* pair_off;
  const int32_t* pm;
  const uint8_t* flag;
  const double* blk;       // De (per element) or Dblk / Mblk (per pair)
  const int32_t* conn_s;
  const int32_t* conn_m;
  int diag_only;          // element-domain D with dual LMs: the diagonal only (biorthogonality)

  template <class F>
  __device__ __forceinline__ void visit(int64_t j, F&& f) const {
    const int64_t q0 = n2e_ptr[j], q1 = n2e_ptr[j + 1];
    for (int64_t q = q0; q < q1; ++q) {
      const int64_t ee = n2e_ent[q];
      const int64_t e = ee >> kLocalBits<NS>;
      const int a = (int)(ee & ((1 << kLocalBits<NS>) - 1));
      if (WHICH == 0) {
        const double* de = blk + (int64_t)kRowW * kRowW * e + kRowW * a;
        if (diag_only)
          f(conn_s[NS * e + a], de[a]);
        else
          for (int b = 0; b < NS; ++b) f(conn_s[NS * e + b], de[b]);
      } else {
        const int64_t p0 = pair_off[e], p1 = pair_off[e + 1];
        for (int64_t p = p0; p < p1; ++p) {
          if (!flag[p]) continue;
          if (WHICH == 1) {
            for (int b = 0; b < NS; ++b) f(conn_s[NS * e + b], blk[16 * p + 4 * a + b]);
          } else {
            const int64_t m = pm[p];
            for (int l = 0; l < NM; ++l) f(conn_m[NM * m + l], blk[4 * kRowW * p + 4 * a + l]);
          }
        }
      }
    }
  }
};

// Sorted list of unique columns with running sums: inserting (c, v) adds v to
// column c's sum (sums in insertion order, i.e. gather order) or opens c.
template <int CAP>
struct RowAcc {
  int32_t col[CAP];
  double val[CAP];
  int u = 0;
  bool over = false;
  __device__ __forceinline__ void add(int32_t c, double v) {
    int lo = 0, hi = u;   // first index with col >= c
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (col[mid] < c) lo = mid + 1; else hi = mid;
    }
    if (lo < u && col[lo] == c) {
      val[lo] += v;
      return;
    }
    if (u == CAP) {
      over = true;
      return;
    }
    for (int k = u; k > lo; --k) { col[k] = col[k - 1]; val[k] = val[k - 1]; }
    col[lo] = c;
    val[lo] = v;
    ++u;
  }
};

// Long row (more unique columns than the accumulator holds): repeated
// selection of the next column, sums in gather order.  Returns the count.
template <int MODE, class Src>
__device__ int row_slow(const Src& src, int64_t j, int64_t out, int32_t* __restrict__ col_out,
                        double* __restrict__ val_out) {
  int u = 0;
  int32_t last = -1;
  for (;;) {
    int32_t next = 0x7fffffff;
    src.visit(j, [&](int32_t c, double) { if (c > last && c < next) next = c; });
    if (next == 0x7fffffff) break;
    bool first = true;
    double s = 0.0;
    src.visit(j, [&](int32_t c, double v) {
      if (c == next) {
        s = first ? v : s + v;
        first = false;
      }
    });
    if (MODE == 1) { col_out[out + u] = next; val_out[out + u] = s; }
    ++u;
    last = next;
  }
  return u;
}

// One thread per slave node (row): both D and M.  MODE 0 counts the unique
// columns of each row, MODE 1 writes the rows.
template <int MODE, class SrcD, class SrcM>
__global__ void __launch_bounds__(kThreads) k_rows(SrcD srcD, SrcM srcM, int64_t N, int32_t* __restrict__ cntD,
                                                   int32_t* __restrict__ cntM, const int64_t* __restrict__ rpD,
                                                   const int64_t* __restrict__ rpM, int64_t capD, int64_t capM,
                                                   int32_t* __restrict__ colD, double* __restrict__ valD,
                                                   int32_t* __restrict__ colM, double* __restrict__ valM,
                                                   DevStatus* st) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  if (st->over_pairs) {   // pair buffers incomplete: the run is repeated with larger ones
    if (MODE == 0) { cntD[j] = 0; cntM[j] = 0; }
    return;
  }
  if (MODE == 1 && (rpD[N] > capD || rpM[N] > capM)) {
    if (j == 0) atomicMax(&st->over_nnz, 1ull);
    return;
  }
  {
    RowAcc<32> acc;
    srcD.visit(j, [&](int32_t c, double v) { acc.add(c, v); });
    int u = acc.u;
    const int64_t out = MODE == 1 ? rpD[j] : 0;
    if (!acc.over) {
      if (MODE == 1)
        for (int k = 0; k < u; ++k) { colD[out + k] = acc.col[k]; valD[out + k] = acc.val[k]; }
    } else {
      if (MODE == 0) atomicAdd(&st->row_slow, 1ull);
      u = row_slow<MODE>(srcD, j, out, colD, valD);
    }
    if (MODE == 0) cntD[j] = u;
  }
  {
    RowAcc<64> acc;
    srcM.visit(j, [&](int32_t c, double v) { acc.add(c, v); });
    int u = acc.u;
    const int64_t out = MODE == 1 ? rpM[j] : 0;
    if (!acc.over) {
      if (MODE == 1)
        for (int k = 0; k < u; ++k) { colM[out + k] = acc.col[k]; valM[out + k] = acc.val[k]; }
    } else {
      if (MODE == 0) atomicAdd(&st->row_slow, 1ull);
      u = row_slow<MODE>(srcM, j, out, colM, valM);
    }
    if (MODE == 0) cntM[j] = u;
  }
}

__global__ void k_finalize(const int64_t* __restrict__ rpD, const int64_t* __restrict__ rpM, int64_t N,
                           DevStatus* st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    st->nnz_D = (unsigned long long)rpD[N];
    st->nnz_M = (unsigned long long)rpM[N];
  }
}

template <int WHICHD, int NS, int NM>
void assemble_t(mortar_ctx* c, const double* blkD) {
  RowSource<WHICHD, NS, NM> srcD{c->n2e_s_ptr.as<int64_t>(), c->n2e_s_ent.as<int64_t>(), c->pair_off.as<int64_t>(),
                                 c->pairs_m.as<int32_t>(), c->flag.as<uint8_t>(), blkD, c->conn_s.as<int32_t>(),
                                 c->conn_m.as<int32_t>(), WHICHD == 0 && c->opt.lm == MORTAR_LM_DUAL};
  RowSource<2, NS, NM> srcM{c->n2e_s_ptr.as<int64_t>(), c->n2e_s_ent.as<int64_t>(), c->pair_off.as<int64_t>(),
                            c->pairs_m.as<int32_t>(), c->flag.as<uint8_t>(), c->Mblk.as<double>(),
                            c->conn_s.as<int32_t>(), c->conn_m.as<int32_t>(), 0};
  DevStatus* st = c->dstat.as<DevStatus>();
  const int64_t N = c->Ns;
  const unsigned g = (unsigned)((N + kThreads - 1) / kThreads);
  int32_t* cntD = c->row_cnt.as<int32_t>();
  int32_t* cntM = c->row_cnt2.as<int32_t>();
  if (N > 0)
    k_rows<0><<<g, kThreads, 0, c->stream>>>(srcD, srcM, N, cntD, cntM, nullptr, nullptr, 0, 0, nullptr, nullptr,
                                              nullptr, nullptr, st);
  launch_exclusive_scan_i32(cntD, c->rowptr_D.as<int64_t>(), nullptr, N, c->scan_tmp.as<int64_t>(), c->stream);
  launch_exclusive_scan_i32(cntM, c->rowptr_M.as<int64_t>(), nullptr, N, c->scan_tmp.as<int64_t>(), c->stream);
  if (N > 0)
    k_rows<1><<<g, kThreads, 0, c->stream>>>(srcD, srcM, N, nullptr, nullptr, c->rowptr_D.as<int64_t>(),
                                              c->rowptr_M.as<int64_t>(), c->nnz_cap_D, c->nnz_cap_M,
                                              c->col_D.as<int32_t>(), c->val_D.as<double>(), c->col_M.as<int32_t>(),
                                              c->val_M.as<double>(), st);
}

template <int NS, int NM>
void assemble_nsnm(mortar_ctx* c, const RunParams& rp) {
  if (NS <= 4 && rp.d_domain == 1) assemble_t<1, NS, NM>(c, c->Dblk.as<double>());
  else assemble_t<0, NS, NM>(c, c->De.as<double>());
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
      else if (nen == 3) k_adj_count<3><<<ge, kThreads, 0, c->stream>>>(conn, E, cnt);
      else if (nen == 8) k_adj_count<8><<<ge, kThreads, 0, c->stream>>>(conn, E, cnt);
      else k_adj_count<6><<<ge, kThreads, 0, c->stream>>>(conn, E, cnt);
    }
    launch_exclusive_scan_i32(cnt, ptr.as<int64_t>(), nullptr, N, c->scan_tmp.as<int64_t>(), c->stream);
    if (E > 0) {
      int64_t* en = ent.as<int64_t>();
      if (nen == 4) k_adj_fill<4><<<ge, kThreads, 0, c->stream>>>(conn, E, ptr.as<int64_t>(), cnt, en);
      else if (nen == 3) k_adj_fill<3><<<ge, kThreads, 0, c->stream>>>(conn, E, ptr.as<int64_t>(), cnt, en);
      else if (nen == 8) k_adj_fill<8><<<ge, kThreads, 0, c->stream>>>(conn, E, ptr.as<int64_t>(), cnt, en);
      else k_adj_fill<6><<<ge, kThreads, 0, c->stream>>>(conn, E, ptr.as<int64_t>(), cnt, en);
    }
    if (N > 0)
      k_adj_sort<<<(unsigned)((N + kThreads - 1) / kThreads), kThreads, 0, c->stream>>>(ptr.as<int64_t>(), N,
                                                                                        ent.as<int64_t>());
  }
}

void launch_assemble(mortar_ctx* c, const RunParams& rp) {
  if (c->nen_s == 8 && c->nen_m == 4) assemble_nsnm<8, 4>(c, rp);
  else if (c->nen_s == 8) assemble_nsnm<8, 3>(c, rp);
  else if (c->nen_s == 6 && c->nen_m == 4) assemble_nsnm<6, 4>(c, rp);
  else if (c->nen_s == 6) assemble_nsnm<6, 3>(c, rp);
  else if (c->nen_s == 4 && c->nen_m == 4) assemble_nsnm<4, 4>(c, rp);
  else if (c->nen_s == 4 && c->nen_m == 3) assemble_nsnm<4, 3>(c, rp);
  else if (c->nen_s == 3 && c->nen_m == 4) assemble_nsnm<3, 4>(c, rp);
  else assemble_nsnm<3, 3>(c, rp);
}

void launch_finalize_status(mortar_ctx* c) {
  k_finalize<<<1, 32, 0, c->stream>>>(c->rowptr_D.as<int64_t>(), c->rowptr_M.as<int64_t>(), c->Ns,
                                      c->dstat.as<DevStatus>());
}

}  // namespace mortar
