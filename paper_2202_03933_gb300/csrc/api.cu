// C ABI of the mortar library (declared in include/mortar.h): context and
// workspace management, the stream-ordered run pipeline and result copies.
//
// One run = precompute -> grid -> binning -> candidates -> integration ->
// assembly (-> adjoint), all on the context's stream with sizes that live on
// the device; the host reads one small status block at the end.  When a
// workspace turned out too small (pairs, CSR entries) the run is repeated
// once with grown buffers; buffers only grow.
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "context.h"

using namespace mortar;

namespace {
// NVTX range for tracing tools (Nsight Systems, ncu --nvtx): a named host
// range around every public call and each phase of an enqueued run.  Without
// an attached tool the push / pop are no-ops.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace

namespace mortar {

int buf_reserve(DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return MORTAR_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return e == cudaErrorMemoryAllocation ? MORTAR_ERR_OOM : MORTAR_ERR_CUDA;
  }
  b.bytes = bytes;
  return MORTAR_OK;
}

void buf_free(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

}  // namespace mortar

namespace {

#define MORTAR_TRY(x)                 \
  do {                                \
    int _st = (x);                    \
    if (_st != MORTAR_OK) return _st; \
  } while (0)

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return MORTAR_OK;
  if (e == cudaErrorMemoryAllocation) return MORTAR_ERR_OOM;
  return MORTAR_ERR_CUDA;
}

int check_cuda() { return cuda_status(cudaGetLastError()); }

int copy_in(void* dst, const void* src, size_t bytes, int on_device, cudaStream_t st) {
  if (bytes == 0) return MORTAR_OK;
  if (!src) return MORTAR_ERR_INVALID_ARG;
  return cuda_status(
      cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
}

int copy_out(void* dst, const void* src, size_t bytes, int on_device, cudaStream_t st) {
  if (bytes == 0) return MORTAR_OK;
  if (!dst) return MORTAR_ERR_INVALID_ARG;
  return cuda_status(
      cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
}

// ---- connectivity check: every id inside its interface's node range
__global__ void k_check_conn(const int32_t* __restrict__ conn, int nen, const int64_t* __restrict__ eoff,
                             const int64_t* __restrict__ noff, int32_t n_if, int64_t E,
                             unsigned long long* __restrict__ bad) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  int32_t lo = 0, hi = n_if - 1;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (eoff[mid] <= e) lo = mid; else hi = mid - 1;
  }
  const int64_t n0 = noff[lo], n1 = noff[lo + 1];
  for (int a = 0; a < nen; ++a) {
    const int64_t n = conn[nen * e + a];
    if (n < n0 || n >= n1) atomicAdd(bad, 1ull);
  }
}

int alloc_pair_buffers(mortar_ctx* c, int64_t cap) {
  const size_t n = (size_t)std::max<int64_t>(cap, 1);
  MORTAR_TRY(buf_reserve(c->pairs_s, n * 4));
  MORTAR_TRY(buf_reserve(c->pairs_m, n * 4));
  MORTAR_TRY(buf_reserve(c->Mblk, n * mblk_stride(c) * 8));
  if (quadratic_slave(c)) {   // four sub-element blocks per pair, summed into Mblk
    MORTAR_TRY(buf_reserve(c->Qunit, n * 4 * 32 * 8));
    MORTAR_TRY(buf_reserve(c->Qflag, n * 4));
  }
  if (c->opt.d_domain == MORTAR_D_SEGMENT) MORTAR_TRY(buf_reserve(c->Dblk, n * 16 * 8));
  MORTAR_TRY(buf_reserve(c->flag, n));
  c->pair_cap = cap;
  return MORTAR_OK;
}

int alloc_csr_buffers(mortar_ctx* c, int64_t capD, int64_t capM) {
  MORTAR_TRY(buf_reserve(c->col_D, (size_t)std::max<int64_t>(capD, 1) * 4));
  MORTAR_TRY(buf_reserve(c->val_D, (size_t)std::max<int64_t>(capD, 1) * 8));
  MORTAR_TRY(buf_reserve(c->col_M, (size_t)std::max<int64_t>(capM, 1) * 4));
  MORTAR_TRY(buf_reserve(c->val_M, (size_t)std::max<int64_t>(capM, 1) * 8));
  c->nnz_cap_D = capD;
  c->nnz_cap_M = capM;
  return MORTAR_OK;
}

void invalidate(mortar_ctx* c) {
  c->search_valid = c->eval_valid = c->grad_valid = c->tan_valid = false;
  if (c->graph_exec) {
    cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
  }
}

struct Phases {
  bool search = true, integrate = true, assemble = true, adjoint = false;
};

}  // namespace

namespace mortar {
// Phase event; inside a stream capture it becomes an event-record node of the
// graph (cudaEventRecordExternal), so replays still time their phases.
void record_event(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  cudaEventRecordWithFlags(ev, st, cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0);
}
}  // namespace mortar

namespace {

// Launch one run (no host synchronisation inside).
void enqueue_run(mortar_ctx* c, const Phases& ph) {
  const RunParams rp = run_params(c);
  cudaStream_t st = c->stream;
  cudaMemsetAsync(c->dstat.p, 0, sizeof(DevStatus), st);
  c->pair_grid = 0;
  if (c->timing) record_event(c->ev[0], st);
  {
    NvtxRange nv("mortar:search");
    launch_slave_precompute(c, rp);
    launch_master_boxes(c, rp);
    launch_grid_params(c, rp);
    launch_bin_masters(c);
    launch_candidates(c);
  }
  if (c->timing) record_event(c->ev[1], st);
  // with the adjoint, the batched adjoint pair kernel also produces the
  // forward blocks (one pass over the pairs instead of two)
  const bool fused = ph.adjoint && ph.integrate && adjoint_fuses_forward(c);
  {
    NvtxRange nv(fused ? "mortar:pairs(forward+adjoint)" : "mortar:pairs(forward)");
    if (fused) launch_adjoint_pairs(c, rp, true);
    else if (ph.integrate) launch_integrate(c, rp);
  }
  if (c->timing) record_event(c->ev[2], st);
  if (ph.assemble) {
    NvtxRange nv("mortar:assemble");
    launch_assemble(c, rp);
    launch_finalize_status(c);
  }
  if (c->timing) record_event(c->ev[3], st);
  if (ph.adjoint) {
    NvtxRange nv("mortar:adjoint");
    if (!fused) launch_adjoint_pairs(c, rp, false);
    if (c->timing) record_event(c->ev[5], st);
    launch_adjoint_rest(c, rp);
  }
  if (c->timing) record_event(c->ev[4], st);
  c->stats.fused = fused ? 1 : 0;
  cudaMemcpyAsync(c->hstat, c->dstat.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, st);
}

// Read back the status of an enqueued run; grow buffers if needed.
// Returns MORTAR_OK, or 1 if the run must be repeated.
int finish_run(mortar_ctx* c, const Phases& ph) {
  MORTAR_TRY(cuda_status(cudaStreamSynchronize(c->stream)));
  MORTAR_TRY(check_cuda());
  const DevStatus& h = *c->hstat;
  bool again = false;
  if (h.over_pairs) {
    MORTAR_TRY(alloc_pair_buffers(c, (int64_t)(h.over_pairs + h.over_pairs / 8 + 1024)));
    again = true;
  }
  if (ph.assemble && h.over_nnz) {
    const int64_t needD = (int64_t)h.nnz_D, needM = (int64_t)h.nnz_M;
    MORTAR_TRY(alloc_csr_buffers(c, std::max(c->nnz_cap_D, needD + needD / 8 + 64),
                                 std::max(c->nnz_cap_M, needM + needM / 8 + 64)));
    again = true;
  }
  if (ph.adjoint && h.over_mlist) again = true;   // list buffers are sized from n_pairs below
  if (h.over_bins) return MORTAR_ERR_CAPACITY;
  if (h.timeout) return MORTAR_ERR_TIMEOUT;
  if (again) {
    if (c->graph_exec) {
      cudaGraphExecDestroy(c->graph_exec);
      c->graph_exec = nullptr;
    }
    return 1;
  }
  c->n_pairs = (int64_t)h.n_pairs;
  c->nnz_D = (int64_t)h.nnz_D;
  c->nnz_M = (int64_t)h.nnz_M;
  mortar_stats& s = c->stats;
  s.n_interfaces = c->n_if;
  s.n_pairs = c->n_pairs;
  s.n_nonempty = (int64_t)h.nonempty;
  s.n_gauss_points = (int64_t)h.gauss_points;
  s.n_cells = (int64_t)h.cells;
  s.n_newton_fail = (int64_t)h.newton_fail;
  s.n_xi_out_of_range = (int64_t)h.xi_oor;
  s.n_clip_overflow = (int64_t)h.clip_overflow;
  s.nnz_D = c->nnz_D;
  s.nnz_M = c->nnz_M;
  s.n_bins = (int64_t)h.n_bins;
  if (c->timing) {
    cudaEventElapsedTime(&s.ms_search, c->ev[0], c->ev[1]);
    cudaEventElapsedTime(&s.ms_integrate, c->ev[1], c->ev[2]);
    cudaEventElapsedTime(&s.ms_assemble, c->ev[2], c->ev[3]);
    cudaEventElapsedTime(&s.ms_adjoint, c->ev[3], c->ev[4]);
    cudaEventElapsedTime(&s.ms_total, c->ev[0], c->ev[4]);
    s.ms_adjoint_pairs = 0.0f;
    if (ph.adjoint) cudaEventElapsedTime(&s.ms_adjoint_pairs, c->ev[3], c->ev[5]);
    s.eta_t = 0.0f;
    const int g = c->pair_grid;
    if (g > 0 && (size_t)g * 16 <= c->cta_t.bytes) {   // CTA busy-time imbalance of the pair kernel
      c->h_cta_t.resize(2 * (size_t)g);
      if (cudaMemcpy(c->h_cta_t.data(), c->cta_t.p, 16 * (size_t)g, cudaMemcpyDeviceToHost) == cudaSuccess) {
        unsigned long long lo = ~0ull, hi = 0;
        for (int b = 0; b < g; ++b) {
          const unsigned long long d = c->h_cta_t[2 * b + 1] - c->h_cta_t[2 * b];
          lo = std::min(lo, d);
          hi = std::max(hi, d);
        }
        if (lo > 0) s.eta_t = (float)((double)hi / (double)lo);
      }
      cudaGetLastError();
    }
  }
  return MORTAR_OK;
}

// Status of a completed run: non-finite coordinates first, then Newton
// failures, then degenerate slave elements.
int run_status(const DevStatus& h, const Phases& ph) {
  if (h.nonfinite) return MORTAR_ERR_INVALID_ARG;
  if (ph.integrate && h.newton_fail) return MORTAR_ERR_NEWTON;
  if (h.degenerate) return MORTAR_ERR_DEGENERATE;
  return MORTAR_OK;
}

int run(mortar_ctx* c, const Phases& ph) {
  if (!c->have_interface) return MORTAR_ERR_STATE;
  if (ph.adjoint && (c->opt.integration != MORTAR_INTEGRATE_SEGMENT || quadratic_slave(c))) return MORTAR_ERR_INVALID_ARG;
  c->stats.reruns = 0;
  for (int attempt = 0; attempt < 4; ++attempt) {
    if (ph.adjoint) MORTAR_TRY(prepare_adjoint_buffers(c));
    enqueue_run(c, ph);
    const int r = finish_run(c, ph);
    if (r == MORTAR_OK) {
      c->search_valid = true;
      c->tan_valid = false;
      c->eval_valid = ph.integrate && ph.assemble;
      c->grad_valid = ph.adjoint;
      return run_status(*c->hstat, ph);
    }
    if (r != 1) return r;
    c->stats.reruns++;
  }
  return MORTAR_ERR_CAPACITY;
}

int set_common(mortar_ctx* c, int32_t n_if, const int64_t* sn_off, const int64_t* se_off, const int64_t* mn_off,
               const int64_t* me_off, const double* xs, const int32_t* conn_s, int32_t type_s, const double* xm,
               const int32_t* conn_m, int32_t type_m, int32_t on_device) {
  if (!c || n_if < 1) return MORTAR_ERR_INVALID_ARG;
  const bool quad_s = type_s == MORTAR_TRI6 || type_s == MORTAR_QUAD8;
  if ((type_s != MORTAR_QUAD4 && type_s != MORTAR_TRI3 && !quad_s) ||
      (type_m != MORTAR_QUAD4 && type_m != MORTAR_TRI3))
    return MORTAR_ERR_INVALID_ARG;
  // quadratic slave elements: standard multipliers, element-domain D,
  // segment-based integration, no facing test (the forward path only)
  if (quad_s && (c->opt.lm != MORTAR_LM_STANDARD || c->opt.d_domain != MORTAR_D_ELEMENT ||
                 c->opt.integration != MORTAR_INTEGRATE_SEGMENT || c->opt.facing_test != 0))
    return MORTAR_ERR_INVALID_ARG;
  for (int i = 0; i < n_if; ++i)
    if (sn_off[i + 1] < sn_off[i] || se_off[i + 1] < se_off[i] || mn_off[i + 1] < mn_off[i] ||
        me_off[i + 1] < me_off[i])
      return MORTAR_ERR_INVALID_ARG;
  if (sn_off[0] != 0 || se_off[0] != 0 || mn_off[0] != 0 || me_off[0] != 0) return MORTAR_ERR_INVALID_ARG;
  invalidate(c);
  c->have_interface = false;
  c->n_if = n_if;
  c->nen_s = type_s;
  c->nen_m = type_m;
  c->Ns = sn_off[n_if];
  c->Es = se_off[n_if];
  c->Nm = mn_off[n_if];
  c->Em = me_off[n_if];
  if (c->Ns >= INT32_MAX || c->Nm >= INT32_MAX || c->Es >= INT32_MAX || c->Em >= INT32_MAX)
    return MORTAR_ERR_INVALID_ARG;
  c->h_sn_off.assign(sn_off, sn_off + n_if + 1);
  c->h_se_off.assign(se_off, se_off + n_if + 1);
  c->h_mn_off.assign(mn_off, mn_off + n_if + 1);
  c->h_me_off.assign(me_off, me_off + n_if + 1);
  cudaStream_t st = c->stream;
  const size_t Ns = (size_t)c->Ns, Nm = (size_t)c->Nm, Es = (size_t)c->Es, Em = (size_t)c->Em;
  MORTAR_TRY(buf_reserve(c->xs, Ns * 24));
  MORTAR_TRY(buf_reserve(c->xm, Nm * 24));
  MORTAR_TRY(buf_reserve(c->conn_s, Es * 4 * type_s));
  MORTAR_TRY(buf_reserve(c->conn_m, Em * 4 * type_m));
  MORTAR_TRY(copy_in(c->xs.p, xs, Ns * 24, on_device, st));
  MORTAR_TRY(copy_in(c->xm.p, xm, Nm * 24, on_device, st));
  MORTAR_TRY(copy_in(c->conn_s.p, conn_s, Es * 4 * type_s, on_device, st));
  MORTAR_TRY(copy_in(c->conn_m.p, conn_m, Em * 4 * type_m, on_device, st));
  // interface tables
  std::vector<int64_t> sn(sn_off, sn_off + n_if + 1), mn(mn_off, mn_off + n_if + 1);
  MORTAR_TRY(buf_reserve(c->se_off, (size_t)(n_if + 1) * 8));
  MORTAR_TRY(buf_reserve(c->me_off, (size_t)(n_if + 1) * 8));
  DevBuf sn_d, mn_d;
  MORTAR_TRY(buf_reserve(sn_d, (size_t)(n_if + 1) * 8));
  MORTAR_TRY(buf_reserve(mn_d, (size_t)(n_if + 1) * 8));
  cudaMemcpyAsync(c->se_off.p, c->h_se_off.data(), (n_if + 1) * 8, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(c->me_off.p, c->h_me_off.data(), (n_if + 1) * 8, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(sn_d.p, sn.data(), (n_if + 1) * 8, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(mn_d.p, mn.data(), (n_if + 1) * 8, cudaMemcpyHostToDevice, st);
  // chunks for the grid reductions
  constexpr int64_t kChunk = 4096;
  std::vector<Chunk> ch;
  std::vector<int32_t> cptr(n_if + 1, 0);
  std::vector<int64_t> capoff(n_if + 1, 0);
  for (int i = 0; i < n_if; ++i) {
    cptr[i] = (int32_t)ch.size();
    for (int side = 0; side < 2; ++side) {
      const int64_t b = side == 0 ? se_off[i] : me_off[i], e = side == 0 ? se_off[i + 1] : me_off[i + 1];
      for (int64_t x = b; x < e; x += kChunk) ch.push_back(Chunk{i, side, x, std::min(e, x + kChunk)});
    }
    capoff[i + 1] = capoff[i] + 32 * (me_off[i + 1] - me_off[i]) + 4096;
  }
  cptr[n_if] = (int32_t)ch.size();
  c->n_chunks = (int64_t)ch.size();
  c->bin_cap = capoff[n_if];
  MORTAR_TRY(buf_reserve(c->chunks, std::max<size_t>(ch.size(), 1) * sizeof(Chunk)));
  MORTAR_TRY(buf_reserve(c->chunk_ptr, (size_t)(n_if + 1) * 4));
  MORTAR_TRY(buf_reserve(c->bin_cap_off, (size_t)(n_if + 1) * 8));
  if (!ch.empty()) cudaMemcpyAsync(c->chunks.p, ch.data(), ch.size() * sizeof(Chunk), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(c->chunk_ptr.p, cptr.data(), (n_if + 1) * 4, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(c->bin_cap_off.p, capoff.data(), (n_if + 1) * 8, cudaMemcpyHostToDevice, st);
  // per-element workspaces
  // quadratic slave elements: four sub-element records and an 8 x 8 D block each
  MORTAR_TRY(buf_reserve(c->srec, Es * (quad_s ? 4 : 1) * SR_STRIDE * 8));
  MORTAR_TRY(buf_reserve(c->De, Es * (quad_s ? 64 : 16) * 8));
  MORTAR_TRY(buf_reserve(c->box_s, Es * 8 * 8));
  MORTAR_TRY(buf_reserve(c->box_m, Em * 8 * 8));
  if (c->opt.facing_test) MORTAR_TRY(buf_reserve(c->nrm_m, Em * 3 * 8));
  MORTAR_TRY(buf_reserve(c->chunk_red, std::max<size_t>(ch.size(), 1) * 8 * 8));
  MORTAR_TRY(buf_reserve(c->grid, (size_t)n_if * sizeof(GridParams)));
  MORTAR_TRY(buf_reserve(c->mkey, Em * 8));
  MORTAR_TRY(buf_reserve(c->bin_cnt, (size_t)c->bin_cap * 4));
  MORTAR_TRY(buf_reserve(c->bin_start, (size_t)(c->bin_cap + 1) * 8));
  MORTAR_TRY(buf_reserve(c->bin_elems, Em * 4));
  MORTAR_TRY(buf_reserve(c->cand_cnt, Es * 4));
  MORTAR_TRY(buf_reserve(c->pair_off, (Es + 1) * 8));
  MORTAR_TRY(buf_reserve(c->row_cnt, std::max(Ns, Nm) * 4));
  MORTAR_TRY(buf_reserve(c->row_cnt2, std::max<size_t>(Ns, 1) * 4));
  MORTAR_TRY(buf_reserve(c->rowptr_D, (Ns + 1) * 8));
  MORTAR_TRY(buf_reserve(c->rowptr_M, (Ns + 1) * 8));
  MORTAR_TRY(buf_reserve(c->n2e_s_ptr, (Ns + 1) * 8));
  MORTAR_TRY(buf_reserve(c->n2e_m_ptr, (Nm + 1) * 8));
  MORTAR_TRY(buf_reserve(c->n2e_s_ent, Es * type_s * 8));
  MORTAR_TRY(buf_reserve(c->n2e_m_ent, Em * type_m * 8));
  const int64_t scan_n = std::max<int64_t>({c->bin_cap, c->Es, c->Ns, c->Nm, c->Em, 1});
  MORTAR_TRY(buf_reserve(c->scan_tmp, (size_t)scan_temp_words(scan_n) * 8));
  if (c->pair_cap < 8 * c->Es + 1024 || c->Mblk.bytes < (size_t)c->pair_cap * mblk_stride(c) * 8 ||
      (quad_s && c->Qunit.bytes < (size_t)c->pair_cap * 4 * 32 * 8))
    MORTAR_TRY(alloc_pair_buffers(c, std::max<int64_t>(c->pair_cap, 8 * c->Es + 1024)));
  if (c->nnz_cap_D < 9 * c->Ns + 64 || c->nnz_cap_M < 16 * c->Ns + 64)
    MORTAR_TRY(alloc_csr_buffers(c, std::max(c->nnz_cap_D, 9 * c->Ns + 64), std::max(c->nnz_cap_M, 16 * c->Ns + 64)));
  // validation
  cudaMemsetAsync(c->dstat.p, 0, sizeof(DevStatus), st);
  unsigned long long* bad = &c->dstat.as<DevStatus>()->degenerate;
  if (c->Es)
    k_check_conn<<<(unsigned)((c->Es + 127) / 128), 128, 0, st>>>(c->conn_s.as<int32_t>(), type_s,
                                                                  c->se_off.as<int64_t>(), sn_d.as<int64_t>(), n_if,
                                                                  c->Es, bad);
  if (c->Em)
    k_check_conn<<<(unsigned)((c->Em + 127) / 128), 128, 0, st>>>(c->conn_m.as<int32_t>(), type_m,
                                                                  c->me_off.as<int64_t>(), mn_d.as<int64_t>(), n_if,
                                                                  c->Em, bad);
  cudaMemcpyAsync(c->hstat, c->dstat.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, st);
  MORTAR_TRY(cuda_status(cudaStreamSynchronize(st)));
  buf_free(sn_d);
  buf_free(mn_d);
  if (c->hstat->degenerate) return MORTAR_ERR_INVALID_ARG;
  launch_topology(c);
  MORTAR_TRY(cuda_status(cudaStreamSynchronize(st)));
  MORTAR_TRY(check_cuda());
  c->have_interface = true;
  return MORTAR_OK;
}

}  // namespace

extern "C" {

int mortar_default_options(mortar_options* o) {
  if (!o) return MORTAR_ERR_INVALID_ARG;
  std::memset(o, 0, sizeof(*o));
  o->lm = MORTAR_LM_STANDARD;
  o->d_domain = MORTAR_D_ELEMENT;
  o->newton_max_iter = 20;
  o->block_size = 0;
  o->search_inflation = 1e-9;
  o->newton_tol = 1e-14;
  o->clip_tol_rel = 1e-12;
  o->merge_tol_rel = 1e-10;
  o->area_tol_rel = 1e-14;
  o->bin_margin = 0.0;
  o->integration = MORTAR_INTEGRATE_SEGMENT;
  o->element_rule_n = 8;
  o->facing_test = 0;
  o->watchdog_us = 0;
  return MORTAR_OK;
}

int mortar_create(mortar_ctx** out, const mortar_options* o, void* stream) {
  if (!out) return MORTAR_ERR_INVALID_ARG;
  *out = nullptr;
  mortar_ctx* c = new mortar_ctx();
  if (o) c->opt = *o; else mortar_default_options(&c->opt);
  if ((c->opt.lm != 0 && c->opt.lm != 1) || (c->opt.d_domain != 0 && c->opt.d_domain != 1) ||
      c->opt.newton_max_iter < 1 || !(c->opt.search_inflation >= 0.0) || !(c->opt.bin_margin >= 0.0) ||
      (c->opt.integration != MORTAR_INTEGRATE_SEGMENT && c->opt.integration != MORTAR_INTEGRATE_ELEMENT) ||
      c->opt.element_rule_n < 1 || c->opt.element_rule_n > 16 || (c->opt.facing_test != 0 && c->opt.facing_test != 1) ||
      c->opt.block_size < 0 || c->opt.block_size > kMaxPairBlock || (c->opt.block_size % 32) != 0 ||
      c->opt.watchdog_us < 0) {
    delete c;
    return MORTAR_ERR_INVALID_ARG;
  }
  c->block_size = c->opt.block_size;
  c->watchdog_us = c->opt.watchdog_us;
  int r = cuda_status(cudaGetDevice(&c->device));
  if (r == MORTAR_OK) r = cuda_status(cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device));
  if (r == MORTAR_OK) {
    if (stream) c->stream = (cudaStream_t)stream;
    else r = cuda_status(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)), c->owns_stream = true;
  }
  if (r == MORTAR_OK) r = buf_reserve(c->dstat, sizeof(DevStatus));
  if (r == MORTAR_OK && c->opt.integration == MORTAR_INTEGRATE_ELEMENT)
    r = upload_gauss_legendre(c, c->opt.element_rule_n);
  if (r == MORTAR_OK) r = buf_reserve(c->cta_t, (size_t)c->n_sm * 64 * 2 * sizeof(unsigned long long));
  if (r == MORTAR_OK) r = cuda_status(cudaMallocHost((void**)&c->hstat, sizeof(DevStatus)));
  for (int i = 0; i < 8 && r == MORTAR_OK; ++i) r = cuda_status(cudaEventCreate(&c->ev[i]));
  if (r != MORTAR_OK) {
    mortar_destroy(c);
    return r;
  }
  std::memset(c->hstat, 0, sizeof(DevStatus));
  *out = c;
  return MORTAR_OK;
}

void mortar_destroy(mortar_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  DevBuf* bufs[] = {&c->xs, &c->xm, &c->conn_s, &c->conn_m, &c->se_off, &c->me_off, &c->elem_if_s, &c->chunks,
                    &c->chunk_ptr, &c->bin_cap_off, &c->n2e_s_ptr, &c->n2e_s_ent, &c->n2e_m_ptr, &c->n2e_m_ent,
                    &c->srec, &c->De, &c->box_s, &c->box_m, &c->chunk_red, &c->grid, &c->mkey, &c->bin_cnt,
                    &c->bin_start, &c->bin_elems, &c->cand_cnt, &c->pair_off, &c->pairs_s, &c->pairs_m, &c->Mblk,
                    &c->Dblk, &c->flag, &c->row_cnt, &c->row_cnt2, &c->rowptr_D, &c->col_D, &c->val_D, &c->rowptr_M,
                    &c->col_M, &c->val_M, &c->scan_tmp, &c->lambda, &c->gs_pair, &c->gm_pair, &c->abar_pair,
                    &c->J_pair, &c->ge_elem, &c->mp_cnt, &c->mp_off, &c->mp_list, &c->grad_s, &c->grad_m,
                    &c->J_part, &c->dstat, &c->cta_t, &c->tan_ys, &c->tan_ym, &c->tan_Kp, &c->tan_Op,
                    &c->tan_Ke, &c->tan_rowptr, &c->tan_col, &c->tan_val, &c->rule_1d, &c->nrm_m,
                    &c->cn_normals, &c->cn_gap, &c->cn_lam, &c->cn_active, &c->cn_ncp, &c->Qunit, &c->Qflag};
  for (DevBuf* b : bufs) buf_free(*b);
  if (c->hstat) cudaFreeHost(c->hstat);
  for (int i = 0; i < 8; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  if (c->owns_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

int mortar_set_interface(mortar_ctx* c, const double* xs, int64_t Ns, const int32_t* conn_s, int64_t Es,
                         int32_t type_s, const double* xm, int64_t Nm, const int32_t* conn_m, int64_t Em,
                         int32_t type_m, int32_t on_device) {
  NvtxRange nv_call("mortar_set_interface");
  if (Ns < 0 || Es < 0 || Nm < 0 || Em < 0) return MORTAR_ERR_INVALID_ARG;
  const int64_t sn[2] = {0, Ns}, se[2] = {0, Es}, mn[2] = {0, Nm}, me[2] = {0, Em};
  return set_common(c, 1, sn, se, mn, me, xs, conn_s, type_s, xm, conn_m, type_m, on_device);
}

int mortar_set_batch(mortar_ctx* c, int32_t n_if, const int64_t* sn, const int64_t* se, const int64_t* mn,
                     const int64_t* me, const double* xs, const int32_t* conn_s, int32_t type_s, const double* xm,
                     const int32_t* conn_m, int32_t type_m, int32_t on_device) {
  NvtxRange nv_call("mortar_set_batch");
  if (!sn || !se || !mn || !me) return MORTAR_ERR_INVALID_ARG;
  return set_common(c, n_if, sn, se, mn, me, xs, conn_s, type_s, xm, conn_m, type_m, on_device);
}

int mortar_set_coordinates(mortar_ctx* c, const double* xs, const double* xm, int32_t on_device) {
  if (!c || !c->have_interface) return MORTAR_ERR_STATE;
  if (xs) MORTAR_TRY(copy_in(c->xs.p, xs, (size_t)c->Ns * 24, on_device, c->stream));
  if (xm) MORTAR_TRY(copy_in(c->xm.p, xm, (size_t)c->Nm * 24, on_device, c->stream));
  c->search_valid = c->eval_valid = c->grad_valid = c->tan_valid = false;   // graph stays valid: same buffers
  return MORTAR_OK;
}

int mortar_search(mortar_ctx* c, int64_t* n_pairs) {
  NvtxRange nv_call("mortar_search");
  if (!c) return MORTAR_ERR_INVALID_ARG;
  Phases ph;
  ph.integrate = ph.assemble = false;
  const int r = run(c, ph);
  if (r != MORTAR_OK && r != MORTAR_ERR_DEGENERATE) return r;
  if (n_pairs) *n_pairs = c->n_pairs;
  return r;
}

int mortar_get_pairs(mortar_ctx* c, int32_t* s_ids, int32_t* m_ids, int64_t capacity, int32_t on_device) {
  if (!c) return MORTAR_ERR_INVALID_ARG;
  if (!c->search_valid) return MORTAR_ERR_STATE;
  if (capacity < c->n_pairs) return MORTAR_ERR_CAPACITY;
  MORTAR_TRY(copy_out(s_ids, c->pairs_s.p, (size_t)c->n_pairs * 4, on_device, c->stream));
  MORTAR_TRY(copy_out(m_ids, c->pairs_m.p, (size_t)c->n_pairs * 4, on_device, c->stream));
  return cuda_status(cudaStreamSynchronize(c->stream));
}

int mortar_evaluate(mortar_ctx* c) {
  NvtxRange nv_call("mortar_evaluate");
  if (!c) return MORTAR_ERR_INVALID_ARG;
  Phases ph;
  return run(c, ph);
}

int mortar_csr_size(mortar_ctx* c, int32_t which, int64_t* nrows, int64_t* ncols, int64_t* nnz) {
  if (!c || (which != 0 && which != 1)) return MORTAR_ERR_INVALID_ARG;
  if (!c->eval_valid) return MORTAR_ERR_STATE;
  if (nrows) *nrows = c->Ns;
  if (ncols) *ncols = which == 0 ? c->Ns : c->Nm;
  if (nnz) *nnz = which == 0 ? c->nnz_D : c->nnz_M;
  return MORTAR_OK;
}

int mortar_csr_copy(mortar_ctx* c, int32_t which, int64_t* rowptr, int32_t* colidx, double* vals,
                    int64_t capacity_nnz, int32_t on_device) {
  NvtxRange nv_call("mortar_csr_copy");
  if (!c || (which != 0 && which != 1)) return MORTAR_ERR_INVALID_ARG;
  if (!c->eval_valid) return MORTAR_ERR_STATE;
  const int64_t nnz = which == 0 ? c->nnz_D : c->nnz_M;
  if (capacity_nnz < nnz) return MORTAR_ERR_CAPACITY;
  const DevBuf& rp = which == 0 ? c->rowptr_D : c->rowptr_M;
  const DevBuf& ci = which == 0 ? c->col_D : c->col_M;
  const DevBuf& va = which == 0 ? c->val_D : c->val_M;
  MORTAR_TRY(copy_out(rowptr, rp.p, (size_t)(c->Ns + 1) * 8, on_device, c->stream));
  MORTAR_TRY(copy_out(colidx, ci.p, (size_t)nnz * 4, on_device, c->stream));
  MORTAR_TRY(copy_out(vals, va.p, (size_t)nnz * 8, on_device, c->stream));
  return cuda_status(cudaStreamSynchronize(c->stream));
}

int mortar_get_pair_blocks(mortar_ctx* c, double* M_blocks, double* D_blocks, uint8_t* nonempty, int64_t capacity,
                           int32_t on_device) {
  if (!c) return MORTAR_ERR_INVALID_ARG;
  if (!c->eval_valid) return MORTAR_ERR_STATE;
  if (capacity < c->n_pairs) return MORTAR_ERR_CAPACITY;
  const size_t P = (size_t)c->n_pairs;
  if (M_blocks) MORTAR_TRY(copy_out(M_blocks, c->Mblk.p, P * mblk_stride(c) * 8, on_device, c->stream));
  if (D_blocks) {
    if (c->opt.d_domain != MORTAR_D_SEGMENT) return MORTAR_ERR_STATE;
    MORTAR_TRY(copy_out(D_blocks, c->Dblk.p, P * 128, on_device, c->stream));
  }
  if (nonempty) MORTAR_TRY(copy_out(nonempty, c->flag.p, P, on_device, c->stream));
  return cuda_status(cudaStreamSynchronize(c->stream));
}

int mortar_weighted_gap_grad(mortar_ctx* c, const double* lambda, double* J, double* grad_xs, double* grad_xm,
                             int32_t on_device) {
  NvtxRange nv_call("mortar_weighted_gap_grad");
  if (!c || !lambda) return MORTAR_ERR_INVALID_ARG;
  if (!c->have_interface) return MORTAR_ERR_STATE;
  MORTAR_TRY(buf_reserve(c->lambda, (size_t)std::max<int64_t>(c->Ns, 1) * 24));
  MORTAR_TRY(copy_in(c->lambda.p, lambda, (size_t)c->Ns * 24, on_device, c->stream));
  Phases ph;
  ph.adjoint = true;
  const int r = run(c, ph);
  if (r != MORTAR_OK && r != MORTAR_ERR_NEWTON && r != MORTAR_ERR_DEGENERATE) return r;
  MORTAR_TRY(mortar_get_gradient(c, J, grad_xs, grad_xm, on_device));
  return r;
}

int mortar_tangent(mortar_ctx* c, const double* ys, const double* ym, int32_t add_direct, int32_t on_device,
                   int64_t* nnzb) {
  NvtxRange nv_call("mortar_tangent");
  if (!c || !ys || !ym) return MORTAR_ERR_INVALID_ARG;
  if (c->opt.integration != MORTAR_INTEGRATE_SEGMENT) return MORTAR_ERR_INVALID_ARG;
  if (!c->have_interface) return MORTAR_ERR_STATE;
  if (quadratic_slave(c)) return MORTAR_ERR_INVALID_ARG;
  MORTAR_TRY(buf_reserve(c->tan_ys, (size_t)std::max<int64_t>(c->Ns, 1) * 24));
  MORTAR_TRY(buf_reserve(c->tan_ym, (size_t)std::max<int64_t>(c->Nm, 1) * 24));
  MORTAR_TRY(copy_in(c->tan_ys.p, ys, (size_t)c->Ns * 24, on_device, c->stream));
  MORTAR_TRY(copy_in(c->tan_ym.p, ym, (size_t)c->Nm * 24, on_device, c->stream));
  int r0 = MORTAR_OK;
  if (!c->eval_valid) {   // forward blocks, flags and pairs of the current coordinates
    Phases ph;
    r0 = run(c, ph);
    if (r0 != MORTAR_OK && r0 != MORTAR_ERR_NEWTON && r0 != MORTAR_ERR_DEGENERATE) return r0;
  }
  c->tan_valid = false;
  // per-pair and per-element blocks, sized from the pair count of the forward run
  const size_t P = (size_t)std::max<int64_t>(c->n_pairs, 1);
  MORTAR_TRY(buf_reserve(c->tan_Kp, P * 288 * 8));
  if (c->opt.lm == MORTAR_LM_DUAL) MORTAR_TRY(buf_reserve(c->tan_Op, P * 12 * 8));
  if (tangent_needs_elems(c)) MORTAR_TRY(buf_reserve(c->tan_Ke, (size_t)std::max<int64_t>(c->Es, 1) * 144 * 8));
  MORTAR_TRY(buf_reserve(c->tan_rowptr, (size_t)(c->Ns + 1) * 8));
  c->tan_pair_cap = c->n_pairs;
  c->tan_direct = add_direct ? 1 : 0;
  const RunParams rp = run_params(c);
  DevStatus* dst = c->dstat.as<DevStatus>();
  cudaMemsetAsync(&dst->work_ctr3, 0, 3 * sizeof(unsigned long long), c->stream);   // work_ctr3, nnzb_K, over_K
  if (c->timing) record_event(c->ev[6], c->stream);
  launch_tangent_blocks(c, rp);
  launch_tangent_rows(c, rp, 0);
  cudaMemcpyAsync(c->hstat, c->dstat.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream);
  MORTAR_TRY(cuda_status(cudaStreamSynchronize(c->stream)));
  MORTAR_TRY(check_cuda());
  const int64_t need = (int64_t)c->hstat->nnzb_K;
  if (need > c->tan_nnzb_cap) {
    const int64_t cap = need + need / 16 + 64;
    MORTAR_TRY(buf_reserve(c->tan_col, (size_t)cap * 4));
    MORTAR_TRY(buf_reserve(c->tan_val, (size_t)cap * 72));
    c->tan_nnzb_cap = cap;
  }
  launch_tangent_rows(c, rp, 1);
  if (c->timing) record_event(c->ev[7], c->stream);
  cudaMemcpyAsync(c->hstat, c->dstat.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream);
  MORTAR_TRY(cuda_status(cudaStreamSynchronize(c->stream)));
  MORTAR_TRY(check_cuda());
  if (c->hstat->over_K || c->hstat->over_pairs) return MORTAR_ERR_CAPACITY;
  c->nnzb_K = need;
  c->stats.nnzb_K = need;
  c->stats.ms_tangent = 0.0f;
  if (c->timing) cudaEventElapsedTime(&c->stats.ms_tangent, c->ev[6], c->ev[7]);
  c->tan_valid = true;
  if (nnzb) *nnzb = need;
  return r0;
}

int mortar_contact_terms(mortar_ctx* c, const double* lambda_n, double cpen, double* normals, double* gap,
                         uint8_t* active, double* ncp, int32_t on_device) {
  NvtxRange nv_call("mortar_contact_terms");
  if (!c) return MORTAR_ERR_INVALID_ARG;
  if (!c->have_interface) return MORTAR_ERR_STATE;
  if (lambda_n && !(cpen > 0.0)) return MORTAR_ERR_INVALID_ARG;
  if (quadratic_slave(c)) return MORTAR_ERR_INVALID_ARG;
  int r0 = MORTAR_OK;
  if (!c->eval_valid) {
    Phases ph;
    r0 = run(c, ph);
    if (r0 != MORTAR_OK && r0 != MORTAR_ERR_NEWTON && r0 != MORTAR_ERR_DEGENERATE) return r0;
  }
  const size_t Ns = (size_t)std::max<int64_t>(c->Ns, 1);
  MORTAR_TRY(buf_reserve(c->cn_normals, Ns * 24));
  MORTAR_TRY(buf_reserve(c->cn_gap, Ns * 8));
  if (lambda_n) {
    MORTAR_TRY(buf_reserve(c->cn_lam, Ns * 8));
    MORTAR_TRY(buf_reserve(c->cn_active, Ns));
    MORTAR_TRY(buf_reserve(c->cn_ncp, Ns * 8));
    MORTAR_TRY(copy_in(c->cn_lam.p, lambda_n, (size_t)c->Ns * 8, on_device, c->stream));
  }
  launch_contact_terms(c, lambda_n != nullptr, cpen);
  MORTAR_TRY(check_cuda());
  if (normals) MORTAR_TRY(copy_out(normals, c->cn_normals.p, (size_t)c->Ns * 24, on_device, c->stream));
  if (gap) MORTAR_TRY(copy_out(gap, c->cn_gap.p, (size_t)c->Ns * 8, on_device, c->stream));
  if (lambda_n && active) MORTAR_TRY(copy_out(active, c->cn_active.p, (size_t)c->Ns, on_device, c->stream));
  if (lambda_n && ncp) MORTAR_TRY(copy_out(ncp, c->cn_ncp.p, (size_t)c->Ns * 8, on_device, c->stream));
  MORTAR_TRY(cuda_status(cudaStreamSynchronize(c->stream)));
  return r0;
}

int mortar_tangent_copy(mortar_ctx* c, int64_t* rowptr, int32_t* colidx, double* vals, int64_t capacity_nnzb,
                        int32_t on_device) {
  if (!c) return MORTAR_ERR_INVALID_ARG;
  if (!c->tan_valid) return MORTAR_ERR_STATE;
  if (capacity_nnzb < c->nnzb_K) return MORTAR_ERR_CAPACITY;
  MORTAR_TRY(copy_out(rowptr, c->tan_rowptr.p, (size_t)(c->Ns + 1) * 8, on_device, c->stream));
  MORTAR_TRY(copy_out(colidx, c->tan_col.p, (size_t)c->nnzb_K * 4, on_device, c->stream));
  MORTAR_TRY(copy_out(vals, c->tan_val.p, (size_t)c->nnzb_K * 72, on_device, c->stream));
  return cuda_status(cudaStreamSynchronize(c->stream));
}

int mortar_get_gradient(mortar_ctx* c, double* J, double* grad_xs, double* grad_xm, int32_t on_device) {
  NvtxRange nv_call("mortar_get_gradient");
  if (!c) return MORTAR_ERR_INVALID_ARG;
  if (!c->grad_valid) return MORTAR_ERR_STATE;
  if (J) *J = c->hstat->J;
  if (grad_xs) MORTAR_TRY(copy_out(grad_xs, c->grad_s.p, (size_t)c->Ns * 24, on_device, c->stream));
  if (grad_xm) MORTAR_TRY(copy_out(grad_xm, c->grad_m.p, (size_t)c->Nm * 24, on_device, c->stream));
  return cuda_status(cudaStreamSynchronize(c->stream));
}

int mortar_run_graph(mortar_ctx* c, const double* lambda, int32_t on_device) {
  NvtxRange nv_call("mortar_run_graph");
  if (!c) return MORTAR_ERR_INVALID_ARG;
  if (!c->have_interface) return MORTAR_ERR_STATE;
  Phases ph;
  ph.adjoint = lambda != nullptr;
  if (lambda) {
    MORTAR_TRY(buf_reserve(c->lambda, (size_t)std::max<int64_t>(c->Ns, 1) * 24));
    MORTAR_TRY(copy_in(c->lambda.p, lambda, (size_t)c->Ns * 24, on_device, c->stream));
  }
  if (c->graph_exec && c->graph_with_adjoint != ph.adjoint) {
    cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
  }
  if (!c->graph_exec) {
    // eager run first: sizes every buffer for this input
    const int r = run(c, ph);
    if (r != MORTAR_OK && r != MORTAR_ERR_NEWTON && r != MORTAR_ERR_DEGENERATE) return r;
    if (ph.adjoint) MORTAR_TRY(prepare_adjoint_buffers(c));
    cudaGraph_t g = nullptr;
    MORTAR_TRY(cuda_status(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal)));
    enqueue_run(c, ph);   // phase events (if timing) become event-record nodes
    MORTAR_TRY(cuda_status(cudaStreamEndCapture(c->stream, &g)));
    c->graph_timing = c->timing;
    size_t n_nodes = 0;
    cudaGraphGetNodes(g, nullptr, &n_nodes);
    std::vector<cudaGraphNode_t> nodes(n_nodes);
    if (n_nodes) cudaGraphGetNodes(g, nodes.data(), &n_nodes);
    int64_t nk = 0;
    for (cudaGraphNode_t nd : nodes) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
    }
    c->stats.graph_kernels = nk;
    const int r2 = cuda_status(cudaGraphInstantiate(&c->graph_exec, g, 0));
    cudaGraphDestroy(g);
    MORTAR_TRY(r2);
    c->graph_with_adjoint = ph.adjoint;
    return r;
  }
  MORTAR_TRY(cuda_status(cudaGraphLaunch(c->graph_exec, c->stream)));
  const bool timing = c->timing;
  c->timing = c->graph_timing;   // the captured graph records the phase events
  int r = finish_run(c, ph);
  c->timing = timing;
  if (r == 1) {   // grown: rerun eagerly, the graph is re-captured on the next call
    c->stats.reruns++;
    r = run(c, ph);
  } else if (r == MORTAR_OK) {
    c->search_valid = true;
    c->eval_valid = true;
    c->grad_valid = ph.adjoint;
    r = run_status(*c->hstat, ph);
  }
  return r;
}

int mortar_get_stats(mortar_ctx* c, mortar_stats* out) {
  if (!c || !out) return MORTAR_ERR_INVALID_ARG;
  *out = c->stats;
  return MORTAR_OK;
}

int mortar_set_timing(mortar_ctx* c, int32_t enabled) {
  if (!c) return MORTAR_ERR_INVALID_ARG;
  c->timing = enabled != 0;
  if (c->graph_exec && c->graph_timing != c->timing) {
    cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
  }
  return MORTAR_OK;
}

int mortar_set_watchdog(mortar_ctx* c, int32_t watchdog_us) {
  if (!c || watchdog_us < 0) return MORTAR_ERR_INVALID_ARG;
  c->watchdog_us = watchdog_us;
  if (c->graph_exec) {   // the budget is a kernel argument of the captured launches
    cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
  }
  return MORTAR_OK;
}

int mortar_set_launch(mortar_ctx* c, int32_t variant, int32_t block_size, int32_t chunk_pairs, int32_t rounds) {
  if (!c || variant < 0 || variant > 1 || block_size < 0 || block_size > kMaxPairBlock || (block_size % 32) != 0 ||
      chunk_pairs < 0 ||
      (rounds != 0 && rounds != 1 && rounds != 2 && rounds != 4 && rounds != 8 && rounds != 16 && rounds != 32))
    return MORTAR_ERR_INVALID_ARG;
  c->variant = variant;
  c->block_size = block_size;
  c->chunk_pairs = chunk_pairs;
  c->rounds = rounds;
  if (c->graph_exec) {
    cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
  }
  return MORTAR_OK;
}

int mortar_autotune(mortar_ctx* c, const double* lambda, int32_t on_device, int32_t* variant, int32_t* rounds,
                    int32_t* block_size, float* best_ms) {
  NvtxRange nv_call("mortar_autotune");
  if (!c) return MORTAR_ERR_INVALID_ARG;
  if (!c->have_interface) return MORTAR_ERR_STATE;
  if (quadratic_slave(c)) return MORTAR_ERR_INVALID_ARG;   // one launch shape: nothing to tune
  Phases ph;
  ph.adjoint = lambda != nullptr;
  if (lambda) {
    MORTAR_TRY(buf_reserve(c->lambda, (size_t)std::max<int64_t>(c->Ns, 1) * 24));
    MORTAR_TRY(copy_in(c->lambda.p, lambda, (size_t)c->Ns * 24, on_device, c->stream));
  }
  // candidate launch shapes: the warp-batched kernels with 32 R pairs per
  // warp batch (R = rounds 1, 2, 4, 8, 16, 32) and 2, 4 or 8 warps per block, and
  // the one-pair-per-thread kernels with 64, 128 or 256 threads per block and
  // 32 or 128 pairs per work-counter fetch
  struct Cand { int32_t variant, rounds, block, chunk; };
  std::vector<Cand> cands;
  for (int32_t r : {1, 2, 4, 8, 16, 32})
    for (int32_t b : {64, 128, 256})
      if (integrate_batched_fits(r, b)) cands.push_back({0, r, b, 0});
  for (int32_t b : {64, 128, 256})
    for (int32_t k : {32, 128}) cands.push_back({1, 0, b, k});
  const bool timing = c->timing;
  c->timing = true;
  float best = 1e30f;
  Cand pick = {0, 2, 128, 0};
  int r = MORTAR_OK;
  for (const Cand& k : cands) {
    c->variant = k.variant;
    c->rounds = k.rounds;
    c->block_size = k.block;
    c->chunk_pairs = k.chunk;
    float t_best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {   // first run sizes buffers and warms up
      r = run(c, ph);
      if (r != MORTAR_OK && r != MORTAR_ERR_NEWTON && r != MORTAR_ERR_DEGENERATE) break;
      const float t = c->stats.ms_integrate + (ph.adjoint ? c->stats.ms_adjoint_pairs : 0.0f);
      if (rep > 0) t_best = std::min(t_best, t);
    }
    if (r != MORTAR_OK && r != MORTAR_ERR_NEWTON && r != MORTAR_ERR_DEGENERATE) break;
    if (t_best < best) {
      best = t_best;
      pick = k;
    }
  }
  c->timing = timing;
  c->variant = pick.variant;
  c->rounds = pick.rounds;
  c->block_size = pick.block;
  c->chunk_pairs = pick.chunk;
  if (c->graph_exec) {
    cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
  }
  if (variant) *variant = pick.variant;
  if (rounds) *rounds = pick.rounds;
  if (block_size) *block_size = pick.block;
  if (best_ms) *best_ms = best;
  return (r == MORTAR_ERR_NEWTON || r == MORTAR_ERR_DEGENERATE) ? MORTAR_OK : r;
}

const char* mortar_status_string(int s) {
  switch (s) {
    case MORTAR_OK: return "MORTAR_OK";
    case MORTAR_ERR_INVALID_ARG: return "MORTAR_ERR_INVALID_ARG";
    case MORTAR_ERR_DEGENERATE: return "MORTAR_ERR_DEGENERATE";
    case MORTAR_ERR_NEWTON: return "MORTAR_ERR_NEWTON";
    case MORTAR_ERR_CAPACITY: return "MORTAR_ERR_CAPACITY";
    case MORTAR_ERR_CUDA: return "MORTAR_ERR_CUDA";
    case MORTAR_ERR_OOM: return "MORTAR_ERR_OOM";
    case MORTAR_ERR_TIMEOUT: return "MORTAR_ERR_TIMEOUT";
    case MORTAR_ERR_STATE: return "MORTAR_ERR_STATE";
    case MORTAR_ERR_NOT_BUILT: return "MORTAR_ERR_NOT_BUILT";
    default: return "MORTAR_ERR_UNKNOWN";
  }
}

}  // extern "C"
