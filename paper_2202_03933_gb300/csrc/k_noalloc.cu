// Entry point that allocates no device memory: slave-element precomputation
// plus per-pair integration over a caller-supplied pair list, with all scratch
// in one file-scope static device array.
//
// Some callers cannot call cudaMalloc: code inside a device-memory
// allocator's own callback (an allocation there re-enters the allocator), and
// processes whose device memory is reserved up front by a pool or a fixed
// budget (a new allocation fails or breaks the budget).  They pass inputs and
// outputs; everything else the kernels need lives in g_static_scratch below.
// Each call synchronises its stream once, to read the id check back before
// any kernel dereferences an id.
//
// Scratch layout (FP64 words): [DevStatus | slave records | element D blocks |
// slave boxes], sized for kStaticMaxSlave slave elements.  The array exists on
// every device that loads this library until the process exits.  Every call
// shares it and it keeps the last call's contents: the status block (counters,
// pair count, work counter) is cleared by each call, the per-element parts are
// fully rewritten for the call's slave elements.  Calls whose work overlaps on
// the GPU (different streams, or another thread) race on the array.
#include <mutex>

#include "context.h"

namespace mortar {

namespace {

constexpr int64_t kStaticMaxSlave = 8192;
constexpr int64_t kStatusWords = 32;                        // >= sizeof(DevStatus) / 8
constexpr int64_t kSrecWords = kStaticMaxSlave * SR_STRIDE;
constexpr int64_t kDeWords = kStaticMaxSlave * 16;
constexpr int64_t kBoxWords = kStaticMaxSlave * 8;
constexpr int64_t kStaticWords = kStatusWords + kSrecWords + kDeWords + kBoxWords;
static_assert(sizeof(DevStatus) <= kStatusWords * 8, "status block does not fit");

static __device__ __align__(256) double g_static_scratch[kStaticWords];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};   // device address of g_static_scratch, per device
int g_n_sm[kMaxDevices] = {};

__global__ void k_static_reset(DevStatus* st, int64_t n_pairs) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    unsigned long long* w = reinterpret_cast<unsigned long long*>(st);
    for (size_t i = 0; i < sizeof(DevStatus) / 8; ++i) w[i] = 0ull;
    st->n_pairs = (unsigned long long)n_pairs;
  }
}

// Every id the geometry kernels dereference must be in range; a bad id is
// counted in st->degenerate (read back by the host before those kernels run).
__global__ void k_static_check(const int32_t* __restrict__ conn_s, int64_t Es, int nen_s, int64_t Ns,
                               const int32_t* __restrict__ conn_m, int64_t Em, int nen_m, int64_t Nm,
                               const int32_t* __restrict__ ps, const int32_t* __restrict__ pm, int64_t P,
                               DevStatus* st) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long bad = 0;
  for (int64_t i = t0; i < Es * nen_s; i += stride) bad += (conn_s[i] < 0 || conn_s[i] >= Ns);
  for (int64_t i = t0; i < Em * nen_m; i += stride) bad += (conn_m[i] < 0 || conn_m[i] >= Nm);
  for (int64_t i = t0; i < P; i += stride) bad += (ps[i] < 0 || ps[i] >= Es || pm[i] < 0 || pm[i] >= Em);
  if (bad) atomicAdd(&st->degenerate, bad);
}

// Once per device, with that device current: look up the device address of
// the static array (the host-side symbol is only a stand-in) and the SM count.
int static_setup(int dev, double** ptr, int* n_sm) {
  if (dev < 0 || dev >= kMaxDevices) return MORTAR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return MORTAR_ERR_CUDA;
    }
    int sm = 0;
    if (cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sm < 1) {
      cudaGetLastError();
      return MORTAR_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
    g_n_sm[dev] = sm;
  }
  *ptr = g_scratch_ptr[dev];
  *n_sm = g_n_sm[dev];
  return MORTAR_OK;
}

}  // namespace

}  // namespace mortar

using namespace mortar;

extern "C" int mortar_integrate_pairs_static(const mortar_options* o, void* stream, const double* xs,
                                             int64_t n_slave_nodes, const int32_t* conn_s, int64_t n_slave_elems,
                                             int32_t type_s, const double* xm, int64_t n_master_nodes,
                                             const int32_t* conn_m, int64_t n_master_elems, int32_t type_m,
                                             const int32_t* pair_s, const int32_t* pair_m, int64_t n_pairs,
                                             double* M_blocks, double* D_blocks, uint8_t* nonempty) {
  if (n_slave_elems > kStaticMaxSlave) return MORTAR_ERR_CAPACITY;
  if (!o || n_slave_elems < 0 || n_pairs < 0 || n_slave_nodes < 0 || n_master_nodes < 0 || n_master_elems < 0)
    return MORTAR_ERR_INVALID_ARG;
  if ((type_s != MORTAR_QUAD4 && type_s != MORTAR_TRI3) || (type_m != MORTAR_QUAD4 && type_m != MORTAR_TRI3))
    return MORTAR_ERR_INVALID_ARG;
  if ((o->lm != 0 && o->lm != 1) || (o->d_domain != 0 && o->d_domain != 1) || o->newton_max_iter < 1)
    return MORTAR_ERR_INVALID_ARG;
  if ((n_slave_elems > 0 && (!xs || !conn_s)) || (n_master_elems > 0 && (!xm || !conn_m)))
    return MORTAR_ERR_INVALID_ARG;
  if (n_pairs > 0 && (!pair_s || !pair_m || !M_blocks || !nonempty)) return MORTAR_ERR_INVALID_ARG;
  if (n_pairs > 0 && o->d_domain == MORTAR_D_SEGMENT && !D_blocks) return MORTAR_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return MORTAR_ERR_CUDA;
  }
  double* base = nullptr;
  int n_sm = 0;
  const int r = static_setup(dev, &base, &n_sm);
  if (r != MORTAR_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  DevStatus* status = reinterpret_cast<DevStatus*>(base);
  double* srec = base + kStatusWords;
  double* De = srec + kSrecWords;
  double* box = De + kDeWords;
  // clear the status block, validate ids, read the verdict into host stack memory
  k_static_reset<<<1, 32, 0, st>>>(status, n_pairs);
  k_static_check<<<(unsigned)(n_sm * 4), 256, 0, st>>>(conn_s, n_slave_elems, type_s, n_slave_nodes, conn_m,
                                                       n_master_elems, type_m, n_master_nodes, pair_s, pair_m,
                                                       n_pairs, status);
  unsigned long long bad = 0;
  if (cudaMemcpyAsync(&bad, &status->degenerate, sizeof(bad), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return MORTAR_ERR_CUDA;
  }
  if (bad) return MORTAR_ERR_INVALID_ARG;
  RunParams rp;
  rp.lm = o->lm;
  rp.d_domain = o->d_domain;
  rp.newton_max_iter = o->newton_max_iter;
  rp.pad = 0;
  rp.newton_tol = o->newton_tol;
  rp.clip_tol_rel = o->clip_tol_rel;
  rp.merge_tol_rel = o->merge_tol_rel;
  rp.area_tol_rel = o->area_tol_rel;
  rp.delta = o->search_inflation;
  rp.bin_margin = o->bin_margin;
  rp.integration = 0;   // segment-based only: element-based integration needs the pair offsets of a search
  rp.rule_n = 0;
  rp.facing = 0;
  rp.watchdog_us = 0;
  launch_slave_precompute_raw(xs, conn_s, n_slave_elems, type_s, rp, srec, De, box, status, st);
  if (n_pairs > 0) {
    IntegrateArgs a{pair_s, pair_m, srec, xm, conn_m, M_blocks, D_blocks, nonempty, n_pairs, status, st};
    launch_integrate_raw(a, rp, type_s, type_m, n_sm);
  }
  return cudaGetLastError() == cudaSuccess ? MORTAR_OK : MORTAR_ERR_CUDA;
}
