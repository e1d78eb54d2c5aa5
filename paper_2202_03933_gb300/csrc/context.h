// Host-side context of the mortar library: device workspaces, sizes, and the
// launchers of every kernel (implemented in the k_*.cu translation units).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/mortar.h"
#include "common.cuh"

namespace mortar {

// Grow-only device buffer.  Contents are not preserved on growth.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  template <class T>
  T* as() const { return static_cast<T*>(p); }
};

int buf_reserve(DevBuf& b, size_t bytes);   // MORTAR_OK or MORTAR_ERR_OOM / CUDA
void buf_free(DevBuf& b);

struct Chunk {          // contiguous element range of one interface and side
  int32_t iface;
  int32_t side;         // 0 slave, 1 master
  int64_t begin, end;
};

}  // namespace mortar

struct mortar_ctx {
  mortar_options opt{};
  cudaStream_t stream = nullptr;
  bool owns_stream = false;
  int device = 0;
  int n_sm = 0;
  bool timing = false;
  int32_t variant = 0;        // integration kernel: 0 batched + sorted (default), 1 one pair per thread
  int32_t block_size = 0;     // pair kernels (0 = default)
  int32_t chunk_pairs = 0;    // pairs per work item of the one-pair-per-thread kernels (0 = default)
  int32_t rounds = 0;         // batched kernel: 32 * rounds pairs per warp batch (0 = default)
  int32_t watchdog_us = 0;    // per-CTA time budget of the persistent pair kernels (0 = none)

  // ---- interface definition
  bool have_interface = false;
  int32_t n_if = 0;
  int32_t nen_s = 4, nen_m = 4;
  int64_t Ns = 0, Es = 0, Nm = 0, Em = 0;
  std::vector<int64_t> h_sn_off, h_se_off, h_mn_off, h_me_off;
  mortar::DevBuf xs, xm, conn_s, conn_m;
  mortar::DevBuf se_off, me_off;            // element offsets per interface (int64, n_if+1)
  mortar::DevBuf elem_if_s;                 // interface id of each slave element (int32)
  mortar::DevBuf chunks;                    // mortar::Chunk[n_chunks]
  mortar::DevBuf chunk_ptr;                 // per interface: first chunk (int32, n_if+1)
  int64_t n_chunks = 0;
  mortar::DevBuf bin_cap_off;               // per interface bin capacity offsets (int64, n_if+1)
  int64_t bin_cap = 0;

  // topology: node -> (element, local index) adjacency, sorted by element
  mortar::DevBuf n2e_s_ptr, n2e_s_ent, n2e_m_ptr, n2e_m_ent;

  // ---- per-evaluation workspaces
  mortar::DevBuf srec, De, box_s, box_m;    // slave records, element D, boxes (lo3 hi3 h pad)
  mortar::DevBuf chunk_red;                 // per chunk: lo3 hi3 hmax pad
  mortar::DevBuf grid;                      // GridParams per interface
  mortar::DevBuf mkey;                      // master bin key (int64)
  mortar::DevBuf bin_cnt, bin_start;        // int32 counts, int64 starts (bin_cap + 1)
  mortar::DevBuf bin_elems;                 // int32 (Em)
  mortar::DevBuf cand_cnt, pair_off;        // int32 (Es), int64 (Es + 1)
  mortar::DevBuf pairs_s, pairs_m;          // int32 (pair_cap)
  int64_t pair_cap = 0;
  mortar::DevBuf Mblk, Dblk, flag;          // FP64 16/pair (quadratic slaves 32), uint8/pair
  mortar::DevBuf Qunit, Qflag;              // quadratic slaves: per (pair, sub-element) 32 FP64, uint8
  mortar::DevBuf row_cnt, row_cnt2;         // int32 (max(Ns, Nm)), int32 (Ns)
  mortar::DevBuf rowptr_D, col_D, val_D;
  mortar::DevBuf rowptr_M, col_M, val_M;
  int64_t nnz_cap_D = 0, nnz_cap_M = 0;
  mortar::DevBuf scan_tmp;                  // block partials of the scans
  mortar::DevBuf cta_t;                     // per-CTA busy intervals of the pair kernel (timing)
  int pair_grid = 0;                        // CTAs of the last batched pair kernel (timing)
  std::vector<unsigned long long> h_cta_t;

  // ---- adjoint workspaces
  mortar::DevBuf lambda;                    // Ns x 3
  mortar::DevBuf gs_pair, gm_pair, abar_pair, J_pair;   // per pair
  mortar::DevBuf ge_elem;                   // per slave element 4x3 + J
  mortar::DevBuf mp_cnt, mp_off, mp_list;   // master element -> pairs
  mortar::DevBuf grad_s, grad_m;            // Ns x 3, Nm x 3
  mortar::DevBuf J_part;                    // block partial sums of J

  // ---- linearisation workspaces
  mortar::DevBuf tan_ys, tan_ym;            // contracted fields, Ns x 3 and Nm x 3
  mortar::DevBuf tan_Kp, tan_Op;            // per pair: 288 block entries, 12 (dual LMs)
  mortar::DevBuf tan_Ke;                    // per slave element: 144 block entries
  mortar::DevBuf tan_rowptr, tan_col, tan_val;   // BSR of 3x3 blocks
  int64_t tan_pair_cap = 0, tan_nnzb_cap = 0, nnzb_K = 0;
  int32_t tan_direct = 0;
  bool tan_valid = false;

  // ---- status / bookkeeping
  mortar::DevBuf nrm_m;                     // master element centre normals (facing test), Em x 3
  mortar::DevBuf cn_normals, cn_gap, cn_lam, cn_active, cn_ncp;   // contact terms per slave node
  mortar::DevBuf rule_1d;                   // element-based rule: Gauss-Legendre points and weights
  int32_t rule_1d_n = 0;
  mortar::DevBuf dstat;                     // mortar::DevStatus
  mortar::DevStatus* hstat = nullptr;       // pinned host copy
  bool search_valid = false;
  bool eval_valid = false;
  bool grad_valid = false;
  int64_t n_pairs = 0, nnz_D = 0, nnz_M = 0;
  mortar_stats stats{};
  cudaEvent_t ev[8] = {};

  // ---- graph
  cudaGraphExec_t graph_exec = nullptr;
  bool graph_with_adjoint = false;
  bool graph_timing = false;
};

namespace mortar {

// ---- launchers (all stream-ordered on ctx->stream) ----
// k_scan.cu
int64_t scan_temp_words(int64_t n_max);
void launch_exclusive_scan_i32(const int32_t* in, int64_t* out, const int64_t* n_dev, int64_t n_max,
                               int64_t* tmp, cudaStream_t st);

// k_precompute.cu
void launch_slave_precompute(mortar_ctx* c, const RunParams& rp);
void launch_master_boxes(mortar_ctx* c, const RunParams& rp);
void launch_grid_params(mortar_ctx* c, const RunParams& rp);

// k_search.cu
void launch_bin_masters(mortar_ctx* c);
void launch_candidates(mortar_ctx* c);

// k_integrate.cu
void launch_integrate(mortar_ctx* c, const RunParams& rp);
bool integrate_batched_fits(int rounds, int block);   // shared memory of the batched kernel fits
int integrate_rounds(int rounds, int block);          // rounds the integration kernel uses for a setting

// k_contact.cu
void launch_contact_terms(mortar_ctx* c, bool with_ncp, double cpen);   // normals, gap (+ active, ncp)

// k_elembased.cu
int upload_gauss_legendre(mortar_ctx* c, int n);   // element-based rule table (host, at create)
void launch_integrate_element_based(mortar_ctx* c, const RunParams& rp);

// k_assemble.cu
void launch_topology(mortar_ctx* c);
void launch_assemble(mortar_ctx* c, const RunParams& rp);
void launch_finalize_status(mortar_ctx* c);

// k_adjoint.cu
int prepare_adjoint_buffers(mortar_ctx* c);   // sizes per-pair adjoint buffers from n_pairs
bool adjoint_fuses_forward(const mortar_ctx* c);   // the adjoint pair kernel also writes M/D blocks
void launch_adjoint_pairs(mortar_ctx* c, const RunParams& rp, bool fused);
void launch_adjoint_rest(mortar_ctx* c, const RunParams& rp);   // element adjoint, gathers, J

// k_tangent.cu
bool tangent_needs_elems(const mortar_ctx* c);   // dual LMs or element-domain D: per-element blocks
void launch_tangent_blocks(mortar_ctx* c, const RunParams& rp);   // per-pair and per-element blocks
void launch_tangent_rows(mortar_ctx* c, const RunParams& rp, int mode);   // 0: count + rowptr, 1: write

RunParams run_params(const mortar_ctx* c);

// Quadratic slave elements (tri6, quad8): forward path only, 8 x 4 pair blocks.
inline bool quadratic_slave(const mortar_ctx* c) { return c->nen_s > 4; }
inline int mblk_stride(const mortar_ctx* c) { return quadratic_slave(c) ? 32 : 16; }

// k_quadratic.cu
void launch_integrate_quadratic(mortar_ctx* c, const RunParams& rp);

// Per element-type combination (slave NS, master NM nodes) parts of the pair
// kernels.  Each is built as an object of its own from the same source file
// with MORTAR_PAIR_NS / MORTAR_PAIR_NM defined, so the large kernel templates
// compile in parallel; the main part of each file only dispatches to them.
struct IntegrateArgs;
template <int NS, int NM>
void integrate_nsnm(const IntegrateArgs& a, const RunParams& rp, int n_sm, int variant, int block, int chunk,
                    int rounds);
template <int NS, int NM>
void adjoint_pairs_nsnm(mortar_ctx* c, const RunParams& rp, unsigned grid, unsigned block, int32_t chunk, bool fused);
template <int NS, int NM>
void tangent_pairs_nsnm(mortar_ctx* c, const RunParams& rp);
template <int NS, int NM>
void tangent_rows_nsnm(mortar_ctx* c, const RunParams& rp, int mode);

// Launchers on explicit pointers (no context), used by the no-allocation entry point.
struct IntegrateArgs {
  const int32_t* ps;
  const int32_t* pm;
  const double* srec;
  const double* xm;
  const int32_t* conn_m;
  double* Mblk;
  double* Dblk;
  uint8_t* flag;
  int64_t pair_cap;
  DevStatus* st;
  cudaStream_t stream;
  unsigned long long* cta_t = nullptr;   // per-CTA busy interval (timing only)
  int* grid_out = nullptr;               // receives the grid size used
};
void launch_slave_precompute_raw(const double* xs, const int32_t* conn_s, int64_t Es, int nen_s,
                                 const RunParams& rp, double* srec, double* De, double* box, DevStatus* st,
                                 cudaStream_t stream);
void launch_integrate_raw(const IntegrateArgs& a, const RunParams& rp, int nen_s, int nen_m, int n_sm);
void record_event(cudaEvent_t ev, cudaStream_t st);   // api.cu

}  // namespace mortar
