/*
 * mortar.h -- C ABI of the GB300 mortar-integration library.
 *
 * Computes the mortar coupling matrices of a non-matching 3D surface interface
 * (Mayr & Popp, arXiv 2202.03933, Sec. 2.2, Eq. DiscreteWeakFormInterfaceFlux):
 *
 *   D[j,k] = int_{Gamma_s,h} Phi_j N_k  dGamma      (slave x slave)
 *   M[j,l] = int_{Gamma_s,h} Phi_j (N_l o chi_h) dGamma (slave x master)
 *
 * with isoparametric quad4/tri3 shape functions N (Eq. AnsatzDiscretization),
 * standard or dual Lagrange-multiplier shape functions Phi
 * (Eq. AnsatzDiscretizationLagrangeMult), segment-based integration on one
 * auxiliary plane per slave element (Sec. 2.3, Algorithm 1: project, clip,
 * triangulate, quadrature), a binned contact search (Sec. 3.5, Algorithm 2),
 * and the gradient of the weighted gap functional
 *   J = sum_j lambda_j . ( (D X_s)_j - (M X_m)_j )
 * with respect to every slave and master nodal coordinate (the consistent
 * linearisation the method needs, Sec. 1).
 *
 * Conventions shared by every call:
 *  - All functions return an int status: MORTAR_OK (0) or a negative
 *    mortar_status code; mortar_status_string() names it.
 *  - Coordinates are FP64, row-major (N x 3): x0 y0 z0 x1 y1 z1 ...
 *  - Connectivity is int32, row-major (E x nen), nen = 4 (quad4) or 3 (tri3),
 *    0-based node ids, nodes counter-clockwise about the surface normal
 *    (quad4 corners in the order of the parameter corners (-1,-1), (1,-1),
 *    (1,1), (-1,1)).  Master elements may have either orientation.
 *  - `on_device` = 1: the pointer is CUDA device memory of the current device;
 *    0: host memory.  Input buffers are only read during the call; the
 *    library keeps its own copies.  Output buffers belong to the caller.
 *  - All device work runs on the stream given to mortar_create() (NULL = a
 *    non-blocking stream the context creates and owns).  Calls returning host
 *    data synchronise that stream only.
 *  - The library owns the context, its device workspaces and any captured
 *    CUDA graph; mortar_destroy() releases them.
 *  - Calls on one context are not thread-safe; distinct contexts are
 *    independent.
 */
#ifndef MORTAR_H
#define MORTAR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mortar_status {
  MORTAR_OK = 0,
  MORTAR_ERR_INVALID_ARG = -1, /* null pointer, bad element type, node id out of range, bad size;
                                  from a run: a non-finite node coordinate (elements touching it get
                                  no pairs, the rest is still computed) */
  MORTAR_ERR_DEGENERATE = -2,  /* zero-area, non-finite or inverted slave element */
  MORTAR_ERR_NEWTON = -3,      /* a back-projection did not converge; results are still written */
  MORTAR_ERR_CAPACITY = -4,    /* caller buffer too small; nothing written */
  MORTAR_ERR_CUDA = -5,        /* a CUDA runtime call failed */
  MORTAR_ERR_OOM = -6,         /* device allocation failed */
  MORTAR_ERR_TIMEOUT = -7,     /* a bounded device loop hit its cap */
  MORTAR_ERR_STATE = -8,       /* call out of order (e.g. copy before evaluate) */
  MORTAR_ERR_NOT_BUILT = -9    /* functionality not available in this build */
} mortar_status;

/* Element types (number of nodes).  Linear: tri3, quad4 (both sides).
 * Quadratic (slave side only; Sec. 2.3 admits higher-order interpolation):
 * tri6 = corners 0-2 at (0,0), (1,0), (0,1), mid-side nodes 3 (edge 0-1),
 * 4 (edge 1-2), 5 (edge 2-0); quad8 (serendipity) = corners 0-3 at (-1,-1),
 * (1,-1), (1,1), (-1,1), mid-side nodes 4-7 at (0,-1), (1,0), (0,1), (-1,0).
 * A quadratic slave element is integrated on its piecewise flat
 * approximation (four linear sub-elements, each clipped against the master
 * element), with the quadratic shape functions evaluated at the parent
 * parameters of every quadrature point.  Quadratic slave elements support the
 * forward path only: standard multipliers, element-domain D, segment-based
 * integration, no facing test (other options: MORTAR_ERR_INVALID_ARG at
 * mortar_set_interface / mortar_set_batch); the adjoint, the linearisation,
 * the contact terms and the autotuner return MORTAR_ERR_INVALID_ARG. */
enum { MORTAR_TRI3 = 3, MORTAR_QUAD4 = 4, MORTAR_TRI6 = 6, MORTAR_QUAD8 = 8 };
enum { MORTAR_LM_STANDARD = 0, MORTAR_LM_DUAL = 1 };
/* Domain of D: ELEMENT integrates D over the whole slave element (the
 * definition in Eq. DiscreteWeakFormInterfaceFlux, so sum(D) is the slave
 * area); SEGMENT integrates it over the clip polygons inside the pair loop of
 * Algorithm 1 (then sum(D) = sum(M)). */
enum { MORTAR_D_ELEMENT = 0, MORTAR_D_SEGMENT = 1 };
enum { MORTAR_MATRIX_D = 0, MORTAR_MATRIX_M = 1 };
/* Integration of M (and of D in segment mode): SEGMENT = Algorithm 1 (clip,
 * triangulate, 7-point rule per cell; exact up to the Newton tolerance for
 * affine masters); ELEMENT = element-based integration (Sec. 1, Sec. 2.3): an
 * n x n Gauss-Legendre rule on each slave element (collapsed n x n on tri3),
 * every point assigned to the first master element of its candidate pairs
 * (pair order) that contains its projection, no clipping; cheaper and less
 * accurate (kinks of the integrand at master edges, coverage ends inside
 * elements).  The gradient and the linearisation need SEGMENT. */
enum { MORTAR_INTEGRATE_SEGMENT = 0, MORTAR_INTEGRATE_ELEMENT = 1 };

typedef struct mortar_options {
  int32_t lm;               /* MORTAR_LM_STANDARD or MORTAR_LM_DUAL */
  int32_t d_domain;         /* MORTAR_D_ELEMENT (default) or MORTAR_D_SEGMENT */
  int32_t newton_max_iter;  /* back-projection Newton cap (20) */
  int32_t block_size;       /* threads per block of the pair kernels: 0 (default 128) or a multiple of
                               32 up to 256 */
  double search_inflation;  /* delta: absolute AABB inflation of the search (1e-9) */
  double newton_tol;        /* stop when |dxi|_inf <= tol, then one more update (1e-14) */
  double clip_tol_rel;      /* inside tolerance eps_in = clip_tol_rel * h_s^2 (1e-12) */
  double merge_tol_rel;     /* vertex merge distance = merge_tol_rel * h_s (1e-10) */
  double area_tol_rel;      /* discard polygons below area_tol_rel * slave area (1e-14) */
  double bin_margin;        /* added to the minimal bin size: the 2 dt |mean interface velocity| term
                               of Sec. 3.5 for moving interfaces (0); bins are rebuilt every run */
  int32_t integration;      /* MORTAR_INTEGRATE_SEGMENT (default) or MORTAR_INTEGRATE_ELEMENT */
  int32_t element_rule_n;   /* points per direction of the element-based rule, 1..16 (8) */
  int32_t facing_test;      /* 1: keep only candidate pairs whose slave and master element normals (at
                               the element centres) point against each other, n_s . n_m < 0 (0) */
  int32_t watchdog_us;      /* time budget of the persistent pair kernels in microseconds, 0 = none (0):
                               a kernel whose thread blocks run longer stops taking work and the call
                               returns MORTAR_ERR_TIMEOUT (results not valid; the context stays usable) */
} mortar_options;

typedef struct mortar_stats {
  int64_t n_interfaces;
  int64_t n_pairs;          /* candidate pairs from the search */
  int64_t n_nonempty;       /* pairs with a non-empty clip polygon */
  int64_t n_gauss_points;
  int64_t n_cells;
  int64_t n_newton_fail;
  int64_t n_xi_out_of_range;
  int64_t n_clip_overflow;
  int64_t nnz_D, nnz_M;
  int64_t n_bins;
  int64_t reruns;           /* capacity-driven re-executions of the last run */
  int64_t graph_kernels;    /* kernel nodes in the captured graph (0 before capture) */
  int64_t fused;            /* 1: one pair kernel produced both the forward blocks and the adjoint */
  /* phase times of the last run (CUDA events on the context's stream, also
   * inside replayed graphs; 0 unless mortar_set_timing(ctx, 1)):
   * search = precompute + grid + binning + candidates; integrate = the
   * per-pair kernel producing the forward blocks (when fused = 1 that kernel
   * also runs the adjoint's per-pair reverse sweep); assemble = CSR assembly;
   * adjoint = the remaining adjoint kernels, of which adjoint_pairs is the
   * separate per-pair reverse sweep (0 when fused). */
  float ms_search, ms_integrate, ms_assemble, ms_adjoint, ms_adjoint_pairs, ms_total;
  /* CTA busy-time imbalance max/min of the batched pair kernel in the last run
   * (timing on; the measure eta_t of the paper's load-balancing trigger,
   * Sec. 4.4, taken over CTAs instead of processes); 0 if not measured */
  float eta_t;
  /* linearisation (mortar_tangent): time of its kernels (timing on) and 3x3 blocks */
  float ms_tangent;
  int64_t nnzb_K;
} mortar_stats;

typedef struct mortar_ctx mortar_ctx;

/* Fill `o` with the defaults listed above. */
int mortar_default_options(mortar_options* o);

/* Create a context.  `stream` is a cudaStream_t that every later call on this
 * context uses (NULL: the context creates its own non-blocking stream).  Uses
 * the current CUDA device. */
int mortar_create(mortar_ctx** ctx, const mortar_options* o, void* stream);

/* Release the context, its workspaces and graphs.  NULL is ignored. */
void mortar_destroy(mortar_ctx* ctx);

/* Define one interface (Eq. AnsatzDiscretization: slave and master node
 * coordinates and connectivity).  type_s: MORTAR_QUAD4, MORTAR_TRI3,
 * MORTAR_QUAD8 or MORTAR_TRI6; type_m: MORTAR_QUAD4 or MORTAR_TRI3.  Copies the data; node ids are checked against the node
 * counts (MORTAR_ERR_INVALID_ARG).  Empty meshes are allowed. */
int mortar_set_interface(mortar_ctx* ctx,
                         const double* xs, int64_t n_slave_nodes,
                         const int32_t* conn_s, int64_t n_slave_elems, int32_t type_s,
                         const double* xm, int64_t n_master_nodes,
                         const int32_t* conn_m, int64_t n_master_elems, int32_t type_m,
                         int32_t on_device);

/* Define a batch of independent interfaces, integrated together.  The
 * arrays are the interfaces' arrays concatenated; offsets have
 * n_interfaces + 1 entries (node and element offsets of each side), and
 * connectivity holds GLOBAL node ids into the concatenated node arrays, each
 * element referencing only nodes of its own interface.  Pairs never cross
 * interfaces.  D and M of the batch are block diagonal over interfaces. */
int mortar_set_batch(mortar_ctx* ctx, int32_t n_interfaces,
                     const int64_t* slave_node_off, const int64_t* slave_elem_off,
                     const int64_t* master_node_off, const int64_t* master_elem_off,
                     const double* xs, const int32_t* conn_s, int32_t type_s,
                     const double* xm, const int32_t* conn_m, int32_t type_m,
                     int32_t on_device);

/* Replace node coordinates (same topology), e.g. for a moved configuration.
 * Either pointer may be NULL to keep that side. */
int mortar_set_coordinates(mortar_ctx* ctx, const double* xs, const double* xm, int32_t on_device);

/* Contact search (Algorithm 2 on one device): element bounding boxes, uniform
 * bins per interface, candidate pairs (s, m) whose search_inflation-inflated
 * boxes overlap, sorted by (s, m).  Writes the pair count. */
int mortar_search(mortar_ctx* ctx, int64_t* n_pairs);

/* Copy the candidate pairs of the last search (slave element, master element
 * ids).  capacity < n_pairs -> MORTAR_ERR_CAPACITY. */
int mortar_get_pairs(mortar_ctx* ctx, int32_t* s_ids, int32_t* m_ids, int64_t capacity,
                     int32_t on_device);

/* Segment-based integration (Algorithm 1) over all pairs and deterministic
 * assembly of D and M into CSR.  Runs the search first if the coordinates
 * changed since the last search.  Returns MORTAR_ERR_NEWTON (results still
 * valid) if a back-projection failed to converge. */
int mortar_evaluate(mortar_ctx* ctx);

/* Size of D (which = MORTAR_MATRIX_D: n_slave_nodes^2) or M
 * (MORTAR_MATRIX_M: n_slave_nodes x n_master_nodes) of the last evaluation. */
int mortar_csr_size(mortar_ctx* ctx, int32_t which, int64_t* nrows, int64_t* ncols, int64_t* nnz);

/* Copy a CSR matrix: rowptr (nrows + 1, int64), colidx (nnz, int32, sorted
 * within each row), vals (nnz, FP64).  capacity_nnz < nnz ->
 * MORTAR_ERR_CAPACITY.  A structural entry exists iff some non-empty pair
 * (or, for element-domain D, some slave element) touches it; element-domain D
 * with dual LMs holds the diagonal only (int Phi_a N_b = delta_ab int N_b). */
int mortar_csr_copy(mortar_ctx* ctx, int32_t which, int64_t* rowptr, int32_t* colidx, double* vals,
                    int64_t capacity_nnz, int32_t on_device);

/* Per-pair blocks of the last evaluation, in pair order: M_blocks and D_blocks
 * are (n_pairs x 16) FP64, row a = slave local node, column = master (or
 * slave) local node, 4x4 padded with zeros; nonempty is n_pairs bytes.
 * D_blocks is filled only in segment mode (may be NULL).  Quadratic slave
 * elements: M_blocks is (n_pairs x 32), 8 x 4 rows of slave local nodes
 * padded with zeros, and D_blocks must be NULL. */
int mortar_get_pair_blocks(mortar_ctx* ctx, double* M_blocks, double* D_blocks, uint8_t* nonempty,
                           int64_t capacity, int32_t on_device);

/* Weighted gap J = sum_j lambda_j . ((D X_s)_j - (M X_m)_j) and its gradient
 * (adjoint kernel: per-pair forward recomputation, reverse sweep through
 * quadrature, back-projection, triangulation, clipping, projection and the
 * dual basis).  lambda: n_slave_nodes x 3.  grad_xs: n_slave_nodes x 3,
 * grad_xm: n_master_nodes x 3 (overwritten).  J: one double.  Uses the pairs
 * of the last evaluation (evaluates first if needed). */
int mortar_weighted_gap_grad(mortar_ctx* ctx, const double* lambda, double* J,
                             double* grad_xs, double* grad_xm, int32_t on_device);

/* Consistent linearisation of the mortar coupling terms (Sec. 1: every
 * nonlinear iteration needs the derivatives of D and M with respect to the
 * nodal coordinates; Eq. DiscreteWeakFormInterfaceFlux defines D and M):
 *     K = d/dX [ (D (x) I3) ys - (M (x) I3) ym ]
 * with the nodal fields ys (n_slave_nodes x 3) and ym (n_master_nodes x 3)
 * held fixed.  With add_direct != 0 the blocks [D (x) I3 | -M (x) I3] are
 * added, so that ys = X_s, ym = X_m gives the Jacobian of the weighted gap
 * vector g = (D (x) I3) X_s - (M (x) I3) X_m.  Derivatives pass through the
 * auxiliary plane, the clip polygon, the back-projections and the dual basis
 * A = Dh Me^-1 (and the element-domain D).
 * K is block sparse with 3x3 blocks: block rows = slave nodes, block columns
 * = slave nodes [0, n_slave_nodes) then master nodes [n_slave_nodes,
 * n_slave_nodes + n_master_nodes); block (j, k)[c][d] = d g_j[c] / d X_k[d].
 * A block is structural iff some non-empty pair has slave node j and node k
 * among its 8 nodes, or (element-domain D) some slave element has both.
 * Evaluates first if the last evaluation is stale (its status, e.g.
 * MORTAR_ERR_NEWTON, is returned).  *nnzb (may be NULL) receives the block
 * count.  Per-pair workspace: 2.3 KB per candidate pair (device). */
int mortar_tangent(mortar_ctx* ctx, const double* ys, const double* ym, int32_t add_direct, int32_t on_device,
                   int64_t* nnzb);

/* Copy the linearisation of the last mortar_tangent call: rowptr
 * (n_slave_nodes + 1, int64), colidx (nnzb, int32, ascending within a row),
 * vals (nnzb x 9 FP64, each block row-major).  MORTAR_ERR_CAPACITY if
 * capacity_nnzb < nnzb (nothing written); MORTAR_ERR_STATE before a
 * mortar_tangent call or after a coordinate change. */
int mortar_tangent_copy(mortar_ctx* ctx, int64_t* rowptr, int32_t* colidx, double* vals, int64_t capacity_nnzb,
                        int32_t on_device);

/* Contact-specific terms of the last evaluation (Sec. 2.1: Hertz-Signorini-
 * Moreau conditions gap >= 0, pressure <= 0, gap * pressure = 0; the gap is
 * measured along a continuous field of normals):
 *   normals (n_slave_nodes x 3): averaged nodal normals -- at each slave node
 *     the sum, over its elements in element order, of the element's unit
 *     normal at that node, normalised;
 *   gap (n_slave_nodes): weighted normal gap g_j = -n_j . ((D X_s)_j - (M X_m)_j),
 *     positive where the master lies beyond the slave along n_j;
 *   with lambda_n (n_slave_nodes normal multipliers, compression negative) and
 *   c > 0: active (bytes) = lambda_n + c g < 0, ncp = lambda_n - min(0, lambda_n + c g)
 *   (zero exactly where the conditions hold).
 * Any output may be NULL; lambda_n NULL skips active / ncp.  Evaluates first
 * if the last evaluation is stale (its status, e.g. MORTAR_ERR_NEWTON, is
 * returned).  Caller-owned buffers; on_device says where all of them live.
 * MORTAR_ERR_INVALID_ARG for lambda_n with c <= 0 (or NaN), MORTAR_ERR_STATE
 * without an interface.  The facing test (mortar_options.facing_test) acts
 * on the candidate pairs of the search and so on D and M themselves. */
int mortar_contact_terms(mortar_ctx* ctx, const double* lambda_n, double c, double* normals, double* gap,
                         uint8_t* active, double* ncp, int32_t on_device);

/* Run search + integration + assembly (+ the adjoint if lambda != NULL) as
 * one stream-ordered sequence with device-side sizes, captured once into a
 * CUDA graph and replayed on later calls.  Buffers grow and the graph is
 * re-captured when a capacity is exceeded.  Results are read with the calls
 * above (mortar_csr_copy, mortar_get_gradient). */
int mortar_run_graph(mortar_ctx* ctx, const double* lambda, int32_t on_device);

/* Gradient and J of the last adjoint run (mortar_run_graph with lambda). */
int mortar_get_gradient(mortar_ctx* ctx, double* J, double* grad_xs, double* grad_xm, int32_t on_device);

/* Counters and phase timings of the last run. */
int mortar_get_stats(mortar_ctx* ctx, mortar_stats* out);

/* Enable (1) / disable (0) CUDA-event phase timing (default 0). */
int mortar_set_timing(mortar_ctx* ctx, int32_t enabled);

/* Change the pair kernels' time budget (mortar_options.watchdog_us; 0 = none).
 * A captured graph is re-captured on its next run.  MORTAR_ERR_INVALID_ARG
 * for a negative budget. */
int mortar_set_watchdog(mortar_ctx* ctx, int32_t watchdog_us);

/* Launch shape of the pair kernels (used by the autotuner; 0 = default):
 * variant 0 = integration and adjoint in warp batches of up to 32 * rounds
 * pairs sorted by their clip's cell count and edge intersections (rounds 1,
 * 2, 4, 8, 16 or 32), variant 1 = one pair per thread; block_size = threads per block of either variant (a
 * multiple of 32 up to 256; default 128); chunk_pairs = pairs per
 * work-counter fetch of variant 1 (default 32).  MORTAR_ERR_INVALID_ARG for
 * other values. */
int mortar_set_launch(mortar_ctx* ctx, int32_t variant, int32_t block_size, int32_t chunk_pairs, int32_t rounds);

/* Per-pair integration without any device allocation.  The paper has no
 * counterpart to this call.  It exists for callers that cannot call
 * cudaMalloc: code inside a device-memory allocator's own callback (an
 * allocation there re-enters the allocator), and processes whose device
 * memory is reserved up front by a pool or a fixed budget (a new allocation
 * fails or breaks the budget).
 *
 * Computes, for a caller-given pair list, the per-pair blocks that
 * mortar_evaluate computes (the slave-element precomputation, then the
 * segment-based integration of each pair): M_blocks / D_blocks (n_pairs x 16
 * FP64, layout of mortar_get_pair_blocks; D_blocks only in segment mode, may be
 * NULL otherwise) and nonempty (n_pairs bytes).  All pointers are device
 * memory of the current device, owned by the caller; ids are 0-based
 * (pair_s < n_slave_elems, pair_m < n_master_elems).
 *
 * Scratch lives in one static device array of this library (room for
 * 8192 slave elements, 5.2 MB, held on every device that loads the library
 * until the process exits): n_slave_elems > 8192 returns MORTAR_ERR_CAPACITY
 * and nothing runs.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress) with that device current.  Every call shares
 * the array and clears its counters itself; calls whose work overlaps on the
 * GPU (other streams, other threads) race on it.
 *
 * Always segment-based (o->integration is ignored).  Every call first checks
 * all ids on the GPU and reads the verdict back, so it synchronises `stream`
 * once: ids out of range return MORTAR_ERR_INVALID_ARG before any geometry
 * kernel runs.  After that the precomputation and the integration are
 * enqueued on `stream` and the call returns MORTAR_OK without waiting for
 * them.  Unlike mortar_evaluate, this call does not report degenerate slave
 * elements or back-projection failures: a degenerate slave element gives
 * nonempty = 0 and zero blocks for its pairs, and nothing else is signalled. */
int mortar_integrate_pairs_static(const mortar_options* o, void* stream,
                                  const double* xs, int64_t n_slave_nodes,
                                  const int32_t* conn_s, int64_t n_slave_elems, int32_t type_s,
                                  const double* xm, int64_t n_master_nodes,
                                  const int32_t* conn_m, int64_t n_master_elems, int32_t type_m,
                                  const int32_t* pair_s, const int32_t* pair_m, int64_t n_pairs,
                                  double* M_blocks, double* D_blocks, uint8_t* nonempty);

/* Autotuner (the batched persistent schedule of many uneven interfaces picks
 * its launch shape on the workload itself): runs the context's workload three
 * times per candidate shape -- warp batches of 32 to 1024 pairs (rounds 1, 2,
 * 4, 8, 16, 32) with 64,
 * 128 or 256 threads per block, and one pair per thread with 64, 128 or 256
 * threads per block and 32 or 128 pairs per work fetch --
 * times the pair kernels (integration, plus the adjoint's per-pair kernel when
 * lambda != NULL) with CUDA events, and keeps the fastest shape for later
 * calls.  Writes the choice (any output pointer may be NULL) and its time in
 * ms. */
int mortar_autotune(mortar_ctx* ctx, const double* lambda, int32_t on_device, int32_t* variant,
                    int32_t* rounds, int32_t* block_size, float* best_ms);

/* Name of a status code. */
const char* mortar_status_string(int status);

/* Measurement utility, not part of the method: runs a chain of FP64 fused
 * multiply-adds (`iters` per thread, 8 independent chains) over `blocks` x
 * `threads` threads on `stream` and writes one value per thread to `sink`
 * (device, blocks*threads doubles) so that nothing is optimised away.
 * active_lanes (1..32) masks lanes per warp to test divergence cost. */
int mortar_probe_dfma(void* stream, int32_t blocks, int32_t threads, int64_t iters,
                      int32_t active_lanes, double* sink);

#ifdef __cplusplus
}
#endif

#endif /* MORTAR_H */
