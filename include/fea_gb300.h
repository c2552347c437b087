/*
 * fea_gb300.h -- C-ABI of the GB300 (sm_103a) finite element assembly engine.
 *
 * The engine runs the element loop of the MPI+X assembly paper (Alg.
 * "sequential assembly", Sec. 2.1.1): for every element e it computes the
 * element matrix A^e and right-hand side b^e by Gauss quadrature and
 * scatter-adds them into one CSR system, A += P_e^T A^e P_e, b += P_e^T b^e.
 * The system is the square "partial-row" local matrix of Sec. 3.1: every
 * node the mesh holds has its own rows, and the matrix is assembled from the
 * elements of this mesh only.
 *
 * Conventions shared by every entry point
 *  - Every function returns an int status: FEA_OK (0) or a negative
 *    fea_status code; fea_last_error() then returns a message (thread-local).
 *  - Pointers named *_d are DEVICE pointers (cudaMalloc or torch tensors on
 *    the current device); the caller owns them and the library never frees or
 *    keeps them beyond the call.  Pointers named *_h are host pointers.
 *  - Every call that launches work takes a cudaStream_t (passed as void*,
 *    NULL = legacy default stream) and is stream-ordered; it returns as soon
 *    as the work is enqueued.  Calls documented as "synchronous" wait for the
 *    stream.
 *  - Errors found on the device (an inverted element, a row wider than the
 *    builder supports) are latched in a per-mesh status word and reported by
 *    the next synchronous call on that mesh or by fea_check().
 *  - A mesh handle is library-owned device memory; it is used by one stream
 *    at a time (calls on the same handle from two streams must be ordered by
 *    the caller).
 *
 * Element types and local node order (the reference elements):
 *  FEA_TET4   simplex, nodes (0,0,0) (1,0,0) (0,1,0) (0,0,1)
 *  FEA_PYR5   base [-1,1]^2 at zeta=0 counter-clockwise seen from the apex,
 *             then the apex (0,0,1); rational basis
 *  FEA_PRISM6 triangle (0,0) (1,0) (0,1) at zeta=-1, then the same at +1
 *  FEA_HEX8   [-1,1]^3, (000,100,110,010,001,101,111,011)
 * Jacobian J_ij = dx_i/dxi_j must have det J > 0 at every quadrature point.
 */
#ifndef FEA_GB300_H
#define FEA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FEA_ABI_VERSION 3

typedef enum {
  FEA_OK = 0,
  FEA_ERR_ARG = -1,              /* invalid argument (checked on the host)       */
  FEA_ERR_OOM = -2,              /* a library allocation failed                  */
  FEA_ERR_CUDA = -3,             /* a CUDA runtime call failed                   */
  FEA_ERR_INVERTED_ELEMENT = -4, /* det J <= 0 at a quadrature point             */
  FEA_ERR_NO_CONVERGENCE = -5,   /* a local Newton iteration did not converge    */
  FEA_ERR_TIMEOUT = -6,          /* a bounded device-side wait gave up           */
  FEA_ERR_INDEX_OVERFLOW = -7,   /* a count does not fit the index type          */
  FEA_ERR_UNSUPPORTED = -8       /* valid input beyond a documented limit        */
} fea_status;

typedef enum { FEA_TET4 = 0, FEA_PYR5 = 1, FEA_PRISM6 = 2, FEA_HEX8 = 3 } fea_elem_type;

typedef enum {
  FEA_OP_DIFFUSION = 0,  /* scalar, 1 dof/node: A_ab = int k(x) grad N_a . grad N_b, b_a = int f N_a */
  FEA_OP_ELASTICITY = 1, /* 3 dofs/node, isotropic small strain: A = int B^T D B, b = int f N        */
  FEA_OP_J2 = 2,         /* 3 dofs/node, small-strain J2 plasticity with Voce hardening (the Gauss-point
                            constitutive update of the solid element loop, Sec. 2.2 / 5.2): radial return
                            from the committed state, A = int B^T D_ep B with the consistent tangent,
                            b = f_int = int B^T sigma; see the J2 fields of fea_operator */
  FEA_OP_NEOHOOKE = 3    /* 3 dofs/node, finite strain in the reference configuration (Sec. 2.2: first
                            Piola-Kirchhoff stress P, Newton-Raphson on the Newmark-discretised momentum
                            balance), compressible neo-Hookean solid (Bonet and Wood 2008, Sec. 6.4.3):
                            Psi = mu/2 (F:F - 3) - mu ln J + lam/2 (ln J)^2, F = I + grad0 u at each Gauss
                            point;  A = int grad0 N (dP/dF) grad0 N + mass int N N I  (the Jacobian),
                            b = f_int = int P grad0 N.  Needs u_d; young, poisson, mass as documented in
                            fea_operator; tet4 always 4-point; ATOMIC or COLOR scatter, per-type launches.
                            det J0 <= 0 or det F <= 0 at a point latches FEA_ERR_INVERTED_ELEMENT. */
} fea_op_kind;

typedef enum {
  FEA_FP64 = 0,           /* geometry, integration and accumulation in FP64 */
  FEA_FP32_INTEGRATE = 1, /* element integration in FP32, accumulation into A and b in FP64;
                             J, its cofactors and det J in FP64 for every element (every
                             non-affine element counts as distorted); J^{-1} = C^T / det J and
                             the physical gradients are formed in FP32 from the rounded FP64
                             cofactors and determinant */
  FEA_FP32_ADAPTIVE = 2   /* as FEA_FP32_INTEGRATE, but the geometry is FP32 (on node
                             coordinates relative to node 0, subtracted in FP64) unless the
                             element is distorted: Frobenius condition number of J above
                             FEA_KAPPA_FP64 at some quadrature point, or a det J FP32 cannot
                             trust; such elements are redone in FP64 */
} fea_precision;

#define FEA_KAPPA_FP64 12.0

typedef enum {
  FEA_SCATTER_ATOMIC = 0, /* FP64 atomic adds into A and b (the paper's Alg. "no coloring") */
  FEA_SCATTER_COLOR = 1,  /* element coloring, plain read-modify-write per color (Alg. "coloring") */
  FEA_SCATTER_BLOCK = 2,  /* locality blocks accumulated in shared memory, block-boundary
                             entries resolved globally (Alg. "local partitioning" / "multideps") */
  FEA_SCATTER_ROWS = 3,   /* owner-computes full rows (Sec. 3.1 full-row decomposition with halo
                             elements, applied per CTA): each CTA owns a block of nodes along a
                             Morton curve, recomputes the geometry of the elements touching them and
                             writes every entry of its rows once with plain stores -- no atomics, no
                             zero fill, bitwise reproducible.  The first call per (mesh, ndof) builds
                             the block plan on the host (synchronous); later calls are stream-ordered. */
  FEA_SCATTER_MULTIDEP = 4 /* commutative multidependences (Sec. 3.2.2, Alg. "multideps"): the
                             elements are cut into subdomains of `chunk` consecutive elements of one
                             type (the work items of fea_work_items); one persistent launch in which
                             a CTA runs a subdomain only while it holds a lock on every subdomain of
                             the subdomain's neighbour list (the subdomains sharing a node with it,
                             itself included), so two subdomains whose lists meet never run at the
                             same time, in no fixed order.  Locks are taken by bounded try-locks
                             (all or none), subdomains with more neighbours first.  A subdomain's
                             elements run in local color classes (no two elements of a class share
                             a node) and add into A and b by plain read-modify-write: no atomics.
                             A CTA that finds no subdomain it can take for lock_timeout_us latches
                             FEA_ERR_TIMEOUT and exits.  The first call per (mesh, chunk) builds the
                             plan on the host (synchronous).  Diffusion and elasticity only. */
} fea_scatter;

/* Scheduling of the element loop (the GPU counterpart of the paper's dynamic
 * load balancing, Sec. 4: the cost of an element is not known beforehand).
 * A work item is a run of at most `chunk` consecutive elements of one type:
 * for each type t in enum order, the elements of type t in upload order are
 * cut into ceil(n_t / chunk) items (fea_work_items lists them). */
typedef enum {
  FEA_SCHED_PER_TYPE = 0, /* one launch per element type (per color class for FEA_SCATTER_COLOR) */
  FEA_SCHED_STEAL = 1,    /* one persistent launch over every type: n_ctas CTAs take items from a
                             global counter (dynamic work stealing), in list order, or in the order
                             queue_d gives when queue_d is set and queue_off_d is NULL (a permutation
                             of all items, e.g. by decreasing predicted cost) */
  FEA_SCHED_QUEUES = 2,   /* one persistent launch: CTA c processes exactly the items
                             queue_d[queue_off_d[c] .. queue_off_d[c+1]) in that order (static
                             queues packed by the caller, e.g. longest-processing-time first on
                             predicted costs); no stealing */
  FEA_SCHED_QUEUES_STEAL = 3 /* as FEA_SCHED_QUEUES, then a CTA whose queue is empty takes the
                             next item of the other queues (c+1, c+2, ... in turn), so the static
                             packing is the plan and stealing corrects what it mispredicted */
} fea_schedule;

/* Mesh description for fea_mesh_upload.  coords is xyz per node (AoS,
 * float64 [3*n_nodes]); element e has type types[e] and nodes
 * conn[conn_offsets[e] .. conn_offsets[e+1]) in the local order above.
 * on_device = 0: the five arrays are host pointers; 1: device pointers. */
typedef struct {
  int64_t n_nodes;
  int64_t n_elems;
  const double* coords;
  const uint8_t* types;
  const int64_t* conn_offsets;
  const int32_t* conn;
  int32_t on_device;
  int32_t reserved;
} fea_mesh_desc;

/* The operator to assemble.
 *  kind       fea_op_kind
 *  precision  fea_precision
 *  scatter    fea_scatter
 *  tet_rule   0: tet4 uses the 1-point centroid rule, 1: the 4-point degree-2 rule.
 *             pyr5 always uses 8 points (2x2 Gauss x 2-point Gauss-Jacobi on the
 *             collapsed cube), prism6 6 points (3-point triangle x 2-point Gauss),
 *             hex8 2x2x2 Gauss.
 *  diffusion  k(x) = k0 + k2 * x^2 (x = physical x-coordinate), source f
 *  elasticity young, poisson, body_force[3]
 *  events     optional profiling hook (NULL to skip): cudaEvent_t handles the
 *             call records on its stream -- events[0] before zeroing A and b,
 *             events[1] after zeroing, events[2 + j] after the j-th kernel it
 *             launches (only those with index < n_events are recorded).
 *  schedule   fea_schedule (FEA_SCATTER_ATOMIC only for the persistent ones)
 *  chunk      elements per work item (persistent schedules) and per subdomain
 *             (FEA_SCATTER_MULTIDEP); 0 = 128
 *  n_ctas     persistent grid size (0 = the resident-CTA count); the queue schedules need it
 *  queue_d, queue_off_d  FEA_SCHED_QUEUES*: int32 item ids and int64 [n_ctas + 1]
 *             offsets (device); every item must appear exactly once (not checked)
 *  item_ns_d  optional uint64 [n_items] (device): per item, the %globaltimer
 *             nanoseconds its CTA spent on it (persistent schedules)
 *  item_cta_d optional int32 [n_items] (device): the CTA that processed the item
 *  J2 (kind FEA_OP_J2; young and poisson as for elasticity, tet4 always 4-point):
 *   sigma_y(alpha) = sigma0 + hardening alpha + (sigma_inf - sigma0)(1 - exp(-delta alpha));
 *   the Newton iteration on the consistency condition stops when |g| <= tol_g
 *   sigma_y(alpha_n) or after an update of at most tol_step; more than max_iter
 *   updates latches FEA_ERR_NO_CONVERGENCE.
 *   u_d          float64 [n_nodes][3] nodal displacements (device)
 *   state_in_d   float64 [n_elems][8][7] committed state per (element, point slot):
 *                plastic strain (xx, yy, zz, xy, yz, xz tensor components), alpha;
 *                NULL = virgin material.  Slots past the rule's point count are unused.
 *   state_out_d  float64 [n_elems][8][7] updated state (may be NULL; not in place)
 *   yield_out_d  uint8 [n_elems][8]: 1 where the point yielded (may be NULL)
 *   iters_out_d  uint8 [n_elems][8]: Newton updates of the point (may be NULL)
 *   Elements are indexed by original (upload) id.
 */
typedef struct {
  int32_t kind;
  int32_t precision;
  int32_t scatter;
  int32_t tet_rule;
  double k0, k2, source;
  double young, poisson;
  double body_force[3];
  void** events;
  int32_t n_events;
  int32_t reserved;
  /* scheduling */
  int32_t schedule;
  int32_t chunk;
  int32_t n_ctas;
  int32_t reserved2;
  const int32_t* queue_d;
  const int64_t* queue_off_d;
  uint64_t* item_ns_d;
  int32_t* item_cta_d;
  /* J2 */
  double sigma0, sigma_inf, delta, hardening, tol_g, tol_step;
  int32_t max_iter;
  int32_t reserved3;
  const double* u_d;
  const double* state_in_d;
  double* state_out_d;
  uint8_t* yield_out_d;
  uint8_t* iters_out_d;
  /* FEA_SCATTER_MULTIDEP */
  int32_t lock_timeout_us;   /* bounded wait of a CTA that finds no subdomain to take (0 = 1 s) */
  int32_t reserved4;
  uint64_t* span_d;          /* optional uint64 [n_subdomains][2] (device): the %globaltimer
                                nanoseconds at which each subdomain's locks were taken and at which
                                its last add was done, before the release */
  /* FEA_OP_NEOHOOKE */
  double mass;               /* m >= 0 of the Newmark Jacobian term m int N_a N_b I
                                (m = rho0 / (beta dt^2); 0: a static Newton step) */
} fea_operator;

/* Launch parameters of an assembly on one mesh, as fea_autotune chose them. */
typedef struct fea_tuning {
  int32_t block_elems;      /* elements per block of FEA_SCATTER_BLOCK */
  int32_t producer_warps;   /* geometry-producer warps (of 16) of the pipelined block-task kernel */
  int32_t rows_block_nodes; /* nodes per block of FEA_SCATTER_ROWS */
  int32_t chunk;            /* elements per work item (FEA_SCHED_STEAL) or per subdomain (MULTIDEP) */
  float ms;                 /* median time of one assembly with these parameters */
  int32_t candidates;       /* configurations timed */
} fea_tuning;

typedef struct fea_mesh fea_mesh;

/* Message of the last failing call on this thread ("" if none).  A service
 * of the library; no passage of the paper defines it. */
const char* fea_last_error(void);

/* FEA_ABI_VERSION of the loaded library (service). */
int fea_abi_version(void);

/* Copy a mesh to the device and prepare it: the mesh of one subdomain, whose
 * elements the loop of Alg. "sequential assembly" visits (Sec. 3.1).  The
 * handle holds the element lists per type in input order, the packed per-type
 * connectivity and the offsets of the element-to-nonzero map.  Checks on the host that every type is known, that
 * conn_offsets matches the node count of each type and that node ids are in
 * range (host input), or on the device (device input; then synchronous).
 * n_nodes < 2^31, n_elems < 2^31.  *out receives the handle.
 * Synchronous. */
int fea_mesh_upload(const fea_mesh_desc* desc, void* stream, fea_mesh** out);

/* Replace the node coordinates of a mesh (moving meshes, Newton updates):
 * coords is float64 [3*n_nodes], a device pointer if on_device else a host
 * pointer.  Stream-ordered (a pageable host source is copied before return). */
int fea_mesh_set_coords(fea_mesh* mesh, const double* coords, int on_device, void* stream);

/* Free a handle and every device buffer it owns (synchronizes the device).
 * Service. */
int fea_mesh_destroy(fea_mesh* mesh);

/* Sizes: nodes, elements, and map_len = sum over elements of n_e^2 (the
 * length of node_map).  Service; host call, no device work. */
int fea_mesh_info(const fea_mesh* mesh, int64_t* n_nodes, int64_t* n_elems, int64_t* map_len);

/* Build the node graph of the mesh inside the handle (Sec. 3.1: nodes i and j
 * couple iff some element holds both, diagonal included; rows sorted
 * ascending) and return the number of scalar nonzeros for ndof interleaved
 * dofs per node: *nnz = ndof^2 * (node nonzeros).  ndof in {1, 3}.
 * Synchronous (the count is read back).  FEA_ERR_UNSUPPORTED if a node
 * gathers more than 1024 (element, node) incidences. */
int fea_pattern_size(fea_mesh* mesh, int ndof, int64_t* nnz, void* stream);

/* Write the scalar CSR pattern and the element-to-nonzero map (needs a
 * preceding fea_pattern_size with the same ndof).  The map gives the
 * positions the scatter A += P_e^T A^e P_e of Alg. "sequential assembly"
 * writes, in the square local matrix of Sec. 3.1.
 *  row_ptr_d  int64 [n_nodes*ndof + 1]  row d*i+c starts at row_ptr_d[d*i+c]
 *  col_idx_d  int32 [nnz]               row d*i+c holds columns d*j+c' for the
 *                                       node neighbours j ascending, c' = 0..d-1
 *  node_map_d int32 [map_len]           node_map_d[off(e) + a*n_e + b] = k, the
 *                                       rank of node conn[e][b] among the sorted
 *                                       neighbours of node conn[e][a]; off(e) =
 *                                       sum_{e'<e} n_{e'}^2 over ORIGINAL ids.
 *                                       Entry (d*i+c, d*j+c') of A sits at
 *                                       row_ptr_d[d*i+c] + d*k + c'.
 * col_idx_d or node_map_d may be NULL to skip them.  Stream-ordered.
 * Positions are int64 (row_ptr), columns int32: ndof*n_nodes must be < 2^31
 * (checked by fea_pattern_size, FEA_ERR_INDEX_OVERFLOW). */
int fea_build_csr_pattern(fea_mesh* mesh, int ndof, int64_t* row_ptr_d, int32_t* col_idx_d,
                          int32_t* node_map_d, void* stream);

/* Assemble (Alg. "sequential assembly", parallelised per fea_scatter):
 * OVERWRITES A_vals_d (float64 [nnz]) and b_d (float64 [n_nodes*ndof]) with
 * sum_e P_e^T A^e P_e and sum_e P_e^T b^e, using the pattern and map written
 * by fea_build_csr_pattern for ndof = 1 (diffusion) or 3 (elasticity).
 * A_vals_d must be 16-byte aligned (cudaMalloc and PyTorch allocations are)
 * and b_d 8-byte aligned, else -1 (FEA_ERR_ARG) before any work.
 * Stream-ordered; an inverted element is latched in the mesh status and
 * reported by fea_check (the values are then unspecified). */
int fea_assemble(const fea_operator* op, fea_mesh* mesh, const int64_t* row_ptr_d,
                 const int32_t* node_map_d, double* A_vals_d, double* b_d, void* stream);

/* Work items of the persistent schedules (fea_schedule), the counterpart of
 * the chunks of elements the paper's loop scheduling hands to threads (Sec.
 * 3.2.1; their size is studied in Sec. 5.2): for each element type t in enum
 * order, the elements of type t in upload order cut into runs
 * of at most chunk elements (chunk 0 = 128).  Item i covers the elements of
 * type type_h[i] with in-type ranks first_h[i] .. first_h[i] + count_h[i] - 1.
 * *n_items receives the count; the three host arrays (each may be NULL) need
 * *n_items entries.  Host call, no device work. */
int fea_work_items(const fea_mesh* mesh, int chunk, int64_t* n_items, int32_t* type_h, int32_t* first_h,
                   int32_t* count_h);

/* Grid size of the persistent launch of op on mesh (the workers that share
 * the items, Sec. 4): op->n_ctas if positive,
 * else the number of CTAs resident at once (occupancy x SM count), which is
 * how many queues a FEA_SCHED_QUEUES packing should fill.  Host call. */
int fea_persistent_grid(const fea_operator* op, fea_mesh* mesh, int* n_ctas);

/* The element-wise loop without a scatter (the paper's second measured loop:
 * the subgrid-scale update of Sec. 2.1.3, timed in Sec. 5.3, is a loop over
 * the elements that updates per-element quantities and assembles nothing).  For op->kind == FEA_OP_J2 it runs the Gauss-point
 * update of every element -- strain, radial return from state_in_d -- and
 * writes state_out_d, yield_out_d, iters_out_d (fea_operator layout) and
 * stress_d (float64 [n_elems][8][6], Cauchy stress tensor components xx, yy,
 * zz, xy, yz, xz per point slot; may be NULL).  The mesh needs no pattern.
 * op->schedule selects per-type launches or a persistent schedule (items,
 * queues and item timings as for fea_assemble).  Stream-ordered; a failed
 * return map latches FEA_ERR_NO_CONVERGENCE. */
int fea_element_loop(const fea_operator* op, fea_mesh* mesh, double* stress_d, void* stream);

/* Grid size of the persistent element loop (as fea_persistent_grid, Sec. 4). */
int fea_element_loop_grid(const fea_operator* op, fea_mesh* mesh, int* n_ctas);

/* Product of an assembled system with a vector, and the partial-row form of
 * Sec. 3.1: with the elements partitioned into subdomains that each assemble
 * the square local matrix of their own elements, y = sum_p P_p^T A_p P_p x,
 * the interface rows being summed over the subdomains that hold the node.
 *  mesh, ndof   the mesh (its node graph built for ndof by fea_pattern_size)
 *  row_ptr_d, A_d  its assembled system (fea_build_csr_pattern / fea_assemble)
 *  x_d, y_d     float64 vectors, ndof values per node (device)
 *  glob_d       NULL: x and y are numbered like the mesh, y is overwritten.
 *               Else int32 [n_nodes] local -> global node ids: x is gathered
 *               and y scattered by them, and
 *  shared_d     uint8 [n_nodes] (needed with glob_d): 1 for a node held by
 *               other subdomains too -- its rows are added to y with FP64
 *               atomics (y must hold 0 there before the first subdomain) --
 *               0 for a node of this subdomain only, whose rows are stored.
 * The matrix is read through the mesh's node graph (no scalar column array).
 * Stream-ordered. */
int fea_spmv(fea_mesh* mesh, int ndof, const int64_t* row_ptr_d, const double* A_d, const double* x_d, double* y_d,
             const int32_t* glob_d, const uint8_t* shared_d, void* stream);

/* ---------------------------------------------------------------------------
 * Learned cost model (the GPU counterpart of the paper's dynamic load
 * balancing, Sec. 4: element costs are not known a priori).  A small MLP,
 * n_in features -> 32 tanh -> 32 tanh -> 1, trained by mean squared error and
 * full-batch Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the standardised
 * features and target (training-set mean and population standard deviation;
 * a zero deviation is replaced by 1).  All tensors are FP32, device memory,
 * row-major: X [n][n_in], y [n].  Parameter vector (n_params = 32 n_in + 1,121):
 * W1 [32][n_in], b1 [32], W2 [32][32], b2 [32], w3 [32], b3.
 * ------------------------------------------------------------------------- */
typedef struct fea_costmodel fea_costmodel;

/* New model with the given initial parameters (host, n_params floats);
 * 1 <= n_in <= 8.  Synchronous. */
int fea_costmodel_create(int n_in, const float* params_h, fea_costmodel** out);
int fea_costmodel_destroy(fea_costmodel* model);

/* Current parameters (n_params floats) and scaler (x mean [n_in], x std
 * [n_in], y mean, y std); either pointer may be NULL.  Synchronous. */
int fea_costmodel_get_params(const fea_costmodel* model, float* params_h, float* scaler_h);

/* Fit the scaler to a training set.  Stream-ordered. */
int fea_costmodel_fit_scaler(fea_costmodel* model, const float* X_d, const float* y_d, int64_t n, void* stream);

/* Full-batch gradient (grad_d [n_params]) and loss (loss_d [1], may be NULL)
 * at the current parameters, no update.  Stream-ordered. */
int fea_costmodel_grad(fea_costmodel* model, const float* X_d, const float* y_d, int64_t n, float* grad_d,
                       float* loss_d, void* stream);

/* `epochs` full-batch Adam steps with learning rate lr; loss_d (may be NULL)
 * receives the loss of the last epoch before its update.  Stream-ordered. */
int fea_costmodel_train(fea_costmodel* model, const float* X_d, const float* y_d, int64_t n, int epochs, float lr,
                        float* loss_d, void* stream);

/* Predictions in target units, y_d [n].  Stream-ordered. */
int fea_costmodel_predict(const fea_costmodel* model, const float* X_d, int64_t n, float* y_d, void* stream);

/* Features of the work items of fea_work_items(mesh, chunk): X_d [n_items][6]
 * float = per item, the mean over its elements of the one-hot element type
 * (4), the fraction of the element's Gauss points whose committed equivalent
 * plastic strain (state_in_d, fea_operator layout) is positive, and the
 * Frobenius norm of sym(grad u) (u_d [n_nodes][3]) at the element's reference
 * centroid.  u_d and state_in_d may be NULL (feature 0).  Synchronous. */
int fea_item_features(fea_mesh* mesh, int chunk, const double* u_d, const double* state_in_d, float* X_d,
                      void* stream);

/* Longest-processing-time-first packing (Graham 1969) of n_items items with
 * costs cost_h into n_queues queues: items in decreasing cost (ties: lower id
 * first), each onto the queue with the least load so far (ties: lower queue).
 * Output, host: queue_h [n_items] item ids queue by queue in assignment order,
 * queue_off_h [n_queues + 1], load_h [n_queues] (may be NULL).  The result
 * feeds FEA_SCHED_QUEUES.  Host call. */
int fea_pack_lpt(const double* cost_h, int64_t n_items, int n_queues, int32_t* queue_h, int64_t* queue_off_h,
                 double* load_h);

/* ---------------------------------------------------------------------------
 * Batches: many independent meshes of uneven sizes (the uneven per-unit work
 * that the load balancing of Sec. 4 evens out) assembled by one
 * persistent launch (a zeroing kernel, then CTAs that take work items of any
 * (mesh, element type) by work stealing), optionally captured once as a CUDA
 * graph and replayed.  Each entry names a mesh whose pattern and map were
 * built for the operator's ndof and the caller-owned device buffers of its
 * system; they must stay valid for the life of the batch.
 * ------------------------------------------------------------------------- */
typedef struct fea_batch fea_batch;

typedef struct {
  fea_mesh* mesh;
  const int64_t* row_ptr_d;
  const int32_t* node_map_d;
  double* A_d;  /* overwritten by every fea_batch_assemble */
  double* b_d;
} fea_batch_entry;

/* op: FEA_OP_DIFFUSION or FEA_OP_ELASTICITY (schedule and scatter fields are
 * ignored: the batch always uses work stealing and the ATOMIC scatter; the
 * items are listed mesh by mesh, fewest elements first, which minimises the
 * mean per-mesh latency);
 * op->chunk (0 = 128) and op->n_ctas (0 = resident CTAs) give the initial
 * configuration.  1 <= n_meshes <= 32767.  Synchronous. */
int fea_batch_create(const fea_operator* op, int n_meshes, const fea_batch_entry* entries_h, fea_batch** out);
int fea_batch_destroy(fea_batch* batch);

/* Change the work-item size and grid (synchronizes the device; drops a
 * captured graph). */
int fea_batch_set_config(fea_batch* batch, int chunk, int n_ctas);

/* Items, chunk size and grid of the current configuration.  Host call. */
int fea_batch_info(const fea_batch* batch, int64_t* n_items, int* chunk, int* grid);

/* Time chunk sizes 16..512 and grids of k x SM-count CTAs up to the resident
 * count (median of reps runs each, CUDA events on stream), keep the fastest
 * and return it.  Synchronous; the batch's systems are overwritten. */
int fea_batch_autotune(fea_batch* batch, int reps, void* stream, int* chunk_out, int* n_ctas_out, float* ms_out);

/* Capture one assembly of the batch as a CUDA graph (on an internal stream);
 * later fea_batch_assemble calls replay it.  Synchronous. */
int fea_batch_capture(fea_batch* batch, void* stream);

/* Assemble every system of the batch (overwrite semantics).  Stream-ordered. */
int fea_batch_assemble(fea_batch* batch, void* stream);

/* Per-mesh latency of the last assembly, ns: the %globaltimer at which the
 * mesh's last work item finished minus the start of the persistent launch.
 * Synchronizes the stream. */
int fea_batch_latency(fea_batch* batch, uint64_t* mesh_ns_h, void* stream);

/* CSR row pointers from row lengths, allocating nothing on the device.
 * The paper has no counterpart: this is a service for callers that cannot let
 * a library allocate device memory -- applications that reserve all of the
 * GPU's memory for their own pool at start-up, or that run this step where an
 * allocation would have to go through their allocator or would synchronize
 * the device.  The same scan inside fea_pattern_size takes its scratch from a
 * stream-ordered allocation; this entry point instead uses a fixed 128 KB
 * array compiled into the library, which every GPU that loads the library
 * holds until the process exits.
 *  counts_d   int32 [n] row lengths (device)
 *  row_ptr_d  int64 [n + 1] output (device): row_ptr_d[0] = 0,
 *             row_ptr_d[i + 1] = counts_d[0] + ... + counts_d[i]
 *  n          0 <= n <= 67,108,864 (16,384 tiles of 4,096 rows); larger n is
 *             rejected with FEA_ERR_UNSUPPORTED before any work is queued
 * Stream-ordered.  The first call on a device looks up the scratch array's
 * device address (once per device, with that device current); make that
 * first call before any stream capture.  Every call shares the one scratch
 * array, so calls whose work overlaps on the GPU (different streams, or
 * different host threads on one device) race: order them.  The scratch needs
 * no clearing between calls (every slot read is written first in the same
 * call). */
int fea_row_ptr_from_counts_noalloc(const int32_t* counts_d, int64_t n, int64_t* row_ptr_d, void* stream);

/* Nodes per CTA block of FEA_SCATTER_ROWS (the full-row decomposition of Sec.
 * 3.1 applied per CTA; default 64; 1..512).  A change
 * drops the current plan; the next ROWS assembly rebuilds it.  Host call. */
int fea_mesh_set_rows_block(fea_mesh* mesh, int block_nodes);

/* Elements per block of FEA_SCATTER_BLOCK (the local partitioning of Sec.
 * 3.2.1; default 64; 1..108, the blocks'
 * geometry is staged in shared memory).  A change drops the current plan.
 * Host call. */
int fea_mesh_set_block_elems(fea_mesh* mesh, int block_elems);

/* Producer warps (4..8 of the 16) of the pipelined block-task kernel, which
 * FEA_SCATTER_BLOCK uses for hex meshes in FEA_FP32_INTEGRATE: they compute
 * the next block's geometry while the others run the current block's tasks
 * (the local partitioning of Sec. 3.2.1 with its element work split in two
 * stages).  Default 6.  Host call. */
int fea_mesh_set_pipe_split(fea_mesh* mesh, int producer_warps);

/* Autotuner of the assembly's launch parameters on this mesh.  The paper
 * tunes the chunk size of its task-based assembly by hand (Sec. 5.2, the
 * study of elements per task); here every candidate of the parameters that
 * op's path uses is timed -- the median of `reps` assemblies with CUDA events
 * on `stream`, after one untimed call that builds any plan -- and the fastest
 * is kept:
 *   FEA_SCATTER_MULTIDEP        subdomain size (op->chunk) 64, 128, 256
 *   FEA_SCHED_STEAL             work-item size (op->chunk) 16 .. 256
 *   FEA_SCATTER_ROWS            nodes per block 32, 64, 96, 128
 *   FEA_SCATTER_BLOCK           elements per block 32, 48, 64, 80 (x producer
 *                               warps 4 .. 8 where the pipelined kernel runs)
 * (other paths: the current configuration is timed).  The mesh's setters and
 * op->chunk are left at the choice, and A and b hold an assembly with it.
 * The values are assembled by the same arithmetic under every candidate; only
 * the FP64 summation order of an entry's contributions may change.
 * Synchronous; host work for plan rebuilds. */
int fea_autotune(fea_operator* op, fea_mesh* mesh, const int64_t* row_ptr_d, const int32_t* node_map_d, double* A_d,
                 double* b_d, int reps, void* stream, fea_tuning* out);

/* Statistics of the current FEA_SCATTER_ROWS plan (Sec. 3.1; zeros if none):
 * info[0] blocks, [1] nodes per block, [2] max local nodes of a block,
 * [3] max halo elements of a block, [4] entry tasks, [5] element
 * contributions, [6] halo elements (with repeats), [7] plan bytes on the
 * device.  Host call. */
int fea_rows_plan_info(const fea_mesh* mesh, int64_t info[8]);

/* The FEA_SCATTER_MULTIDEP plan for subdomains of `chunk` elements (0 = 128),
 * built if the mesh holds none for that chunk (host work, synchronous): the
 * subdomains and their neighbour lists that the commutative multidependences
 * of Sec. 3.2.2 (Alg. "multideps") exclude each other by.
 *  info        int64 [4]: subdomains, neighbour-list entries, largest list,
 *              most local colors of a subdomain
 *  nb_off_h    NULL or int64 [subdomains + 1] (host): offsets into nb_h
 *  nb_h        NULL or int32 [entries] (host): the neighbour list of each
 *              subdomain, ascending, itself included (the locks it takes)
 *  order_h     NULL or int32 [subdomains] (host): the priority order
 *              (neighbour count descending; ties in a hashed order)
 *  color_h     NULL or int32 [n_elems] (host): local color of each element
 *              (original id) inside its subdomain
 * Subdomain k is work item k of fea_work_items(chunk).  FEA_ERR_UNSUPPORTED
 * if a subdomain would need more than 64 local colors. */
int fea_multidep_plan(fea_mesh* mesh, int chunk, int64_t info[4], int64_t* nb_off_h, int32_t* nb_h, int32_t* order_h,
                      int32_t* color_h);

/* Hold (held = 1) or free (0) the lock of one subdomain of the mesh's
 * FEA_SCATTER_MULTIDEP plan (Sec. 3.2.2) in every later launch, as if a CTA that never
 * finishes owned it: the subdomains whose lists contain it can then never
 * run, and the CTAs give up after lock_timeout_us with FEA_ERR_TIMEOUT.  For
 * tests of the bounded wait.  Host call; FEA_ERR_ARG without a plan or for a
 * subdomain out of range. */
int fea_multidep_hold(fea_mesh* mesh, int subdomain, int held);

/* The element coloring of FEA_SCATTER_COLOR (Sec. 3.2.1, Alg. "coloring";
 * built by the first COLOR assembly): *n_colors classes, and, if colors_h is not NULL, the class of
 * every element (int32 [n_elems], host).  No two elements of one class share
 * a node.  Host call; FEA_ERR_ARG if no coloring exists yet. */
int fea_color_info(const fea_mesh* mesh, int32_t* colors_h, int* n_colors);

/* Number of kernels one fea_assemble call with this operator launches on this
 * mesh (after its pattern is built).  Service; host call. */
int fea_assemble_launches(const fea_operator* op, const fea_mesh* mesh, int* n_kernels);

/* Wait for the stream and return the mesh's latched device status (and clear
 * it).  Service.  FEA_ERR_INVERTED_ELEMENT names the first element id found in the
 * message.  Synchronous. */
int fea_check(fea_mesh* mesh, void* stream);

/* Measured arithmetic peak of the current device: the FP64 (kind 0) or FP32
 * (kind 1) rate of fused multiply-adds, in flop/s (an FMA is 2 flop).  The
 * paper has no counterpart: it is the microbenchmark behind the FP64 and FP32
 * denominators of the assembly roofline (T_roof = max(FP64 flop / P64, FP32
 * flop / P32, bytes / HBM bandwidth)).  Every SM runs 8 independent FMA
 * chains per thread for `iters` (>= 4) steps, after a shorter warm-up launch;
 * the rate is taken over the CUDA-event time of the timed launch on `stream`.
 * Allocates a small scratch buffer.  Synchronous. */
int fea_peak_probe(int kind, int64_t iters, double* flops, void* stream);

/* The precision conversions of the FP32-integrate kernels, elementwise on n
 * device values: dir 0 widens FP32 `in` to FP64 `out` exactly (every FP32
 * contribution enters the FP64 accumulation this way); dir 1 rounds FP64 `in`
 * to FP32 `out` to nearest, ties to even (FP64 geometry to FP32 records).  Both
 * use integer instructions instead of the FP64 pipe, and both must equal the
 * IEEE 754 conversions bit for bit (NaN: a NaN).  The paper has no counterpart:
 * it exists so that the conversions can be checked.  Asynchronous on
 * `stream`; n = 0 does nothing.  -1 for a bad dir, n < 0 or a null buffer. */
int fea_convert(int dir, const void* in_d, void* out_d, int64_t n, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FEA_GB300_H */
