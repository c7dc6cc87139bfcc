/*
 * sso.h -- C-ABI of the GB300 structural-FEM hot path (arXiv 2407.20026,
 * "JAX-SSO: Differentiable Finite Element Analysis Solver for Structural
 * Optimization").
 *
 * What the library computes, with the passage that defines it:
 *   - element stiffness matrices k_e(x) of 3D beam-columns and MITC-4 quad
 *     shells from nodal coordinates and section/material data (Sec. 2.2.1;
 *     the beam's six numbers E, G, Iy, Iz, J, A are those of Listing 1, the
 *     quad's t, E, nu, kappa_x, kappa_y those of the attribute vector a_quad);
 *   - their assembly into the global stiffness K of K u = f (Eq. 1), stored as
 *     6x6-block sparse rows (one block row per node);
 *   - the supports V u = b with b = 0 (Eqs. 2-3), imposed by eliminating the
 *     fixed DOFs (identity rows/columns in K, zero load), which gives the same
 *     u as the Lagrange-multiplier system K_aug u_aug = f_aug;
 *   - the solve of K u = f by Jacobi / block-Jacobi preconditioned CG, in FP64,
 *     in FP32 inside FP64 iterative refinement, or (small systems, one CTA
 *     each) in double-float arithmetic; optionally with a two-level
 *     preconditioner (rigid-body modes of node aggregates), or, for chains of
 *     beams (block-tridiagonal K), by a direct block cyclic reduction;
 *   - compliance C = f^T u and the adjoint sensitivity of
 *     J = w C + g^T u (Eqs. 5-6): K^T lambda = dJ/du,
 *     dJ/dp = dJ/dp|explicit - lambda^T (dK/dp u - df/dp), for p = the z
 *     coordinate of every node (NodeParameter(node, 2), Listing 2) and the
 *     thickness of every quad (Sec. 3.3).
 *
 * Conventions shared by every call:
 *   - DOF order per node is (ux, uy, uz, rx, ry, rz) (Listing 1); vectors of
 *     DOFs are node-major, length 6 * n_nodes, FP64.
 *   - Input arrays may live in host memory or in device memory of the current
 *     CUDA device; the library detects which (cudaPointerGetAttributes) and
 *     copies what it needs.  Inputs stay owned by the caller and are not
 *     referenced after the call returns.  Outputs are caller-allocated and may
 *     also be host or device memory.
 *   - Every call returns an sso_status and never aborts.  A description of
 *     the last failure on the calling thread is available from
 *     sso_last_error().  A handle whose call failed with SSO_ERR_CUDA may hold
 *     inconsistent device state and should be destroyed.
 *   - A model or batch runs all its work on the CUDA stream given at creation.
 *     Calls that return results to the caller synchronise that stream; the
 *     element-level calls (sso_*_stiffness) and a gradient without g only
 *     enqueue work (later calls and sso_model_get are ordered after it).
 *   - Handles are not thread-safe; use one handle from one thread at a time.
 */
#ifndef SSO_H_
#define SSO_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SSO_OK = 0,
  SSO_ERR_INVALID = 1,       /* bad argument, index out of range, degenerate element */
  SSO_ERR_OOM = 2,           /* device allocation failed or over the memory budget */
  SSO_ERR_SINGULAR = 3,      /* CG breakdown: p^T K p <= 0 or non-finite (K not SPD, e.g. a mechanism) */
  SSO_ERR_NOT_CONVERGED = 4, /* iteration or refinement-sweep cap reached before rtol, or
                                 the FP64 residual no longer falls (rtol below what K and
                                 FP64 resolve) */
  SSO_ERR_TIMEOUT = 5,       /* wall-clock cap reached */
  SSO_ERR_CUDA = 6,          /* a CUDA runtime call failed */
  SSO_ERR_NOT_READY = 7      /* result not available yet (serving poll) */
} sso_status;

/* A structural model (Listing 1: nodes, elements, supports, loads). */
typedef struct {
  int32_t n_nodes;
  const double* xyz;          /* [n_nodes*3] node coordinates (m) */
  int32_t n_beams;
  const int32_t* beam_conn;   /* [n_beams*2] end nodes i, j */
  const double* beam_props;   /* [n_beams*6] E, G, Iy, Iz, J, A */
  int32_t n_quads;
  const int32_t* quad_conn;   /* [n_quads*4] counter-clockwise about the normal */
  const double* quad_props;   /* [n_quads*5] t, E, nu, kappa_x, kappa_y */
  const uint8_t* fixed;       /* [n_nodes*6] 1 = DOF fixed (b = 0) */
  const double* nodal_load;   /* [n_nodes*6] applied nodal forces/moments */
  double pressure;            /* area load on every quad (Pa), along -Z */
  double gamma;               /* self-weight density (N/m^3); quad e carries gamma*t_e along -Z */
} sso_mesh;

/* SSO_F32X2: the whole CG of each system in one CTA and one launch, in
 * double-float arithmetic (every value an unevaluated sum of two FP32
 * numbers, about 48 significant bits, on the FP32 pipes); K is read as its
 * FP32 rounding plus the FP32 rounding of the remainder (K64 - K32).  For
 * small systems (up to a few thousand DOF), whose solve is otherwise
 * dominated by launch and synchronisation latency: one SM works per system,
 * so a large system is slow.  Jacobi, block-Jacobi or two-level (the coarse
 * correction applied inside the same CTA; it pays on systems of a few
 * hundred nodes and more, not on the smallest, whose coarse set-up costs more
 * than the iterations it saves); batches and models (not the server).  Convergence is tested on the residual b - K u recomputed
 * in FP64 from the FP64 K; the CG restarts from it while it is above rtol
 * (max_sweeps caps the restarts, and a restart that lowers the residual less
 * than 2x ends the solve). */
typedef enum { SSO_FP64 = 0, SSO_FP32_IR = 1, SSO_F32X2 = 2 } sso_precision;
/* SSO_TWO_LEVEL: block-Jacobi plus a coarse correction over the rigid-body
 * modes of node aggregates (z = M_b^-1 r + P A_c^-1 P^T r, A_c = P^T K P);
 * FP32_IR (batches, models and the server) or F32X2 (batches and models).
 * SSO_CHAIN: no CG: K u = f is solved exactly by block cyclic reduction in
 * FP64 (K factored once per assembly, every solve and adjoint solve reusing
 * the factors).  Only for a block-tridiagonal K, i.e. every element joins
 * nodes numbered consecutively (a chain of beam-columns: arches, multi-span
 * bridges, cantilevers); other models return SSO_ERR_INVALID.  FP64 only;
 * batches and models (not the server).  While the FP64 residual is above
 * rtol the solution is refined with the same factors (u += K^-1 (f - K u)),
 * up to max_sweeps times or until the residual stops falling; the stats
 * report 0 CG iterations, the refinements as sweeps, and the residual. */
typedef enum {
  SSO_JACOBI = 0, SSO_BLOCK_JACOBI = 1, SSO_TWO_LEVEL = 2, SSO_CHAIN = 3
} sso_precond;

/* Solver options.  Convergence is ||f - K u||_2 <= rtol ||f||_2 over all DOFs,
 * with the residual recomputed in FP64 from the FP64 K. */
typedef struct {
  int32_t precision;         /* sso_precision */
  int32_t precond;           /* sso_precond */
  double rtol;               /* outer relative residual target */
  double inner_rtol;         /* FP32 inner CG: residual reduction per refinement sweep (a
                                sweep that lowers the FP64 residual less than 4x makes the
                                system's later sweeps 10x tighter, down to 1e-6; after that
                                such a sweep ends the solve with SSO_ERR_NOT_CONVERGED) */
  int32_t max_iter;          /* cap on CG iterations summed over sweeps */
  int32_t max_sweeps;        /* cap on refinement sweeps (FP64 residual recomputations) */
  int32_t iters_per_launch;  /* CG iterations per captured CUDA-graph launch */
  int32_t warm_start;        /* 1: start from the model's current u instead of 0 */
  double timeout_ms;         /* wall-clock cap, <= 0 for none */
} sso_options;

typedef struct {
  int32_t status;            /* sso_status of this system */
  int32_t iterations;        /* CG iterations, all sweeps */
  int32_t sweeps;            /* FP64 residual recomputations */
  double rel_residual;       /* ||f - K u|| / ||f|| at exit, from the FP64 K */
  double ms;                 /* wall-clock of the call (same for every system of a batch) */
} sso_stats;

typedef struct sso_model sso_model;
typedef struct sso_batch sso_batch;

/* Defaults: FP32_IR, block-Jacobi, rtol 1e-8, inner_rtol 2e-3,
 * max_iter 200000, max_sweeps 40, iters_per_launch 32, cold start, no timeout. */
void sso_default_options(sso_options* opts);

/* Message of the last failure on this thread ("" if none).  Valid until the
 * next failing call on the same thread. */
const char* sso_last_error(void);

/* Library version string. */
const char* sso_version(void);

/* Number of CUDA kernel launches this library has issued in this process
 * (graph launches count every kernel node they run).  For accounting only. */
unsigned long long sso_kernel_launches(void);

/* ---------------------------------------------------------------------------
 * Element-level kernels (Sec. 2.2.1, element_K_bc_local / element_K_quad_local).
 * All pointers are DEVICE pointers; work is enqueued on `stream`
 * (cudaStream_t, NULL = legacy default stream) and not waited for.
 *
 * Output layout: node-pair blocks, ke[e][a][b][r][c] = k_e[6a+r][6b+c] in
 * global axes, row-major, FP64.  Beams: a, b in {0,1} (144 doubles per
 * element); quads: a, b in {0..3} (576 doubles per element).
 */
sso_status sso_beam_stiffness(int32_t n_beams, const double* d_xyz, const int32_t* d_beam_conn,
                              const double* d_beam_props, double* d_ke, void* stream);
sso_status sso_quad_stiffness(int32_t n_quads, const double* d_xyz, const int32_t* d_quad_conn,
                              const double* d_quad_props, double* d_ke, void* stream);

/* y = K x and *xty = x^T y for a 6x6-block sparse K (the product K u of
 * Eq. 1 for an assembled K, e.g. from sso_model_get_stiffness).  All pointers
 * are DEVICE pointers: row_ptr [n_nodes+1], col [n_blocks], K [n_blocks*36]
 * row-major FP64 blocks, x and y [6*n_nodes], xty [1].  x^T y is summed in a
 * fixed order (bit-reproducible).  Scratch memory (8 bytes per 32 nodes) is
 * allocated and freed stream-ordered on `stream` (cudaMallocAsync); the call
 * only enqueues work.  Indices in col must be < n_nodes. */
sso_status sso_bsr_spmv(int32_t n_nodes, const int32_t* d_row_ptr, const int32_t* d_col,
                        const double* d_K, const double* d_x, double* d_y, double* d_xty,
                        void* stream);

/* The same product as sso_bsr_spmv for callers that cannot allocate device
 * memory: a plug-in that its host application gives a fixed device-memory
 * budget and forbids to allocate beyond it, a real-time loop that cannot take
 * the allocator's latency or the synchronisation that cudaMalloc / cudaFree
 * may imply, or an application whose device memory all belongs to its own
 * pool allocator.  The paper has no counterpart; it is an interface for such
 * callers.
 *
 * Nothing is allocated: the partial sums live in a fixed array compiled into
 * the library (about 512 KiB, held on every GPU that loads the library until
 * the process exits), which limits n_nodes to 2,097,152 (larger n_nodes
 * returns SSO_ERR_INVALID with a message).  Every call looks up that array's
 * device address (cudaGetSymbolAddress, with the caller's device current); the
 * first call in a context may load the library's device code there, so make
 * that first call before any stream capture.  Every call shares the array and
 * it keeps the last call's contents (the completion counter is cleared by each
 * call): calls whose kernels overlap on the GPU -- different streams or host
 * threads -- race and must be serialised by the caller.  Results are
 * bit-identical to sso_bsr_spmv (same kernel, same fixed summation order).
 * Only enqueues work on `stream`. */
sso_status sso_bsr_spmv_noalloc(int32_t n_nodes, const int32_t* d_row_ptr, const int32_t* d_col,
                                const double* d_K, const double* d_x, double* d_y,
                                double* d_xty, void* stream);

/* ---------------------------------------------------------------------------
 * Models.  A model owns the device copy of one structure, its block-sparse
 * pattern (built once on the host from the connectivity: K's block rows are
 * nodes, a block (i, j) exists when some element joins nodes i and j, and the
 * list of element blocks summed into every K block is sorted by element so
 * that assembly is a fixed-order sum, bit-reproducible without atomics), and
 * the solver state.  Device memory is allocated with cudaMalloc at creation.
 */
sso_status sso_model_create(const sso_mesh* mesh, void* stream, sso_model** out);
void sso_model_destroy(sso_model* model);

/* Replace the design: z [n_nodes] node z coordinates and/or t [n_quads]
 * thicknesses (either may be NULL to keep the current values). */
sso_status sso_model_set_design(sso_model* model, const double* z, const double* t);

/* The node aggregates of the two-level preconditioner (host only, no device
 * needed): agg_of_node [n_nodes] (host memory) receives each node's aggregate
 * in [0, *n_aggregates).  Aggregates grow breadth-first over the node
 * adjacency from the lowest-numbered free node to ~max(16, n_nodes / 39)
 * nodes; small leftovers join their best-linked neighbour. */
sso_status sso_aggregate(const sso_mesh* mesh, int32_t* agg_of_node, int32_t* n_aggregates);

/* SIMP topology variables (Sec. 3.5, Eq. simp_eq): E_j = rho_j^penal E*_j for
 * every quad, E* the moduli the model was created with.  rho [n_quads] (host
 * or device) in (0, 1], penal >= 1; rho NULL restores E*.  Afterwards every
 * gradient call also yields dJ/drho (sso_model_get_topology_gradient):
 * -(penal / rho_j) lambda_e^T k_e u_e, the stiffness term of Eq. 6 for this
 * variable (loads do not depend on rho).  Errors: SSO_ERR_INVALID for a
 * density outside (0, 1], a penalty below 1, or rho on a model without quads. */
sso_status sso_model_set_topology(sso_model* model, const double* rho, double penal);
/* dJ/drho [n_quads] of the last gradient call (host or device output). */
sso_status sso_model_get_topology_gradient(sso_model* model, double* drho);

/* Element matrices -> K (FP64, and its FP32 rounding) -> supports ->
 * preconditioner -> loads -> CG / iterative refinement.  Results stay on the
 * device; read them with sso_model_get.  `stats` may be NULL. */
sso_status sso_model_solve(sso_model* model, const sso_options* opts, sso_stats* stats);

/* Adjoint sensitivity of J = w C + g^T u after a successful solve (Eqs. 5-6).
 * g is NULL or [6*n_nodes] (host or device).  With g == NULL, lambda = w u and
 * no second solve is made (K is symmetric); otherwise K lambda = w f + g is
 * solved with the same options as the last solve.  Fills dJ/dz and dJ/dt.
 * Without g the call returns once the contraction kernels are queued: the
 * caller's stream, later calls on the model and sso_model_get are ordered
 * after them (with g, the adjoint solve's status has been read first). */
sso_status sso_model_gradient(sso_model* model, double w, const double* g, sso_stats* stats);

/* Copy results out; any pointer may be NULL.  u [6*n_nodes], C [1],
 * dz [n_nodes], dt [n_quads], lam [6*n_nodes] (adjoint vector). */
sso_status sso_model_get(sso_model* model, double* u, double* C, double* dz, double* dt,
                         double* lam);

/* Material volume of the quads, W = sum_e A_e t_e (Sec. 3.3: the volume term
 * of the size-optimisation objective, without its minimum-thickness
 * penalty), at the model's current design, with A_e the area of the
 * element's flat facet (the 2 x 2 Gauss integral used for area loads).
 * Outputs (any may be NULL; host or device): V [1], dVdz [n_nodes]
 * (dW/dz_i, every node), dVdt [n_quads] (dW/dt_e = A_e).  Beams add nothing.
 * Ordered on the model's stream; returns when the outputs are written.
 * The sum over elements has a fixed order, so W is reproducible. */
sso_status sso_model_volume(sso_model* model, double* V, double* dVdz, double* dVdt);

/* Sizes of the model: n_blocks of K and the number of element blocks. */
sso_status sso_model_info(const sso_model* model, int32_t* n_nodes, int32_t* n_blocks,
                          int32_t* n_elem_blocks);

/* Copy the assembled K (after a solve), supports applied: row_ptr
 * [n_nodes+1], col [n_blocks], K64 [n_blocks*36] and K32 [n_blocks*36],
 * blocks row-major.  Any pointer may be NULL. */
sso_status sso_model_get_stiffness(sso_model* model, int32_t* row_ptr, int32_t* col,
                                   double* K64, float* K32);

/* The full load vector f [6*n_nodes] (nodal + consistent area loads, zero on
 * fixed DOFs) after a solve. */
sso_status sso_model_get_load(sso_model* model, double* f);

/* ---------------------------------------------------------------------------
 * Batches: several models (any mix of sizes and topologies, all on the same
 * device) solved together.  Every CG iteration is one pass of two kernels over
 * all systems that are still iterating; each system keeps its own scalars,
 * refinement state and convergence test, and its reductions follow a fixed
 * tiling of its own rows, so its result does not depend on which other systems
 * share the batch.  The batch runs on the stream of models[0].  A batch of 32
 * or more models runs its CG as 2 to 4 parts at once (about 18,000 tiles of 30
 * nodes per part), on the streams of their first models and on as many host
 * threads (the first part on the calling thread); each part's kernel ramps and
 * tails overlap the others' work.  The results are the same bits as without
 * the split (sso_batch_set_parts changes the count).
 */
sso_status sso_batch_create(sso_model* const* models, int32_t n_models, sso_batch** out);

/* Runs the batch's CG as `parts` concurrent parts of contiguous models (1 =
 * one part; at most 16 and at most one model per part), replacing the default
 * split.  Each part has its own stream (its first model's), CUDA graphs and
 * host thread; the results do not change.  Waits for the batch's work. */
sso_status sso_batch_set_parts(sso_batch* batch, int32_t parts);
void sso_batch_destroy(sso_batch* batch);
/* Solve every model; stats is NULL or [n_models].  Returns the first
 * non-OK per-system status (if any) after all systems finished. */
sso_status sso_batch_solve(sso_batch* batch, const sso_options* opts, sso_stats* stats);
/* Gradients of J_i = w[i] C_i + g[i]^T u_i for every model.  w NULL means
 * all 1; g NULL, or g[i] NULL, means no g term for that system. */
sso_status sso_batch_gradient(sso_batch* batch, const double* w, const double* const* g,
                              sso_stats* stats);

/* Kernel timing of the CG engine, for roofline measurements: while enabled,
 * every CG kernel launch of this batch (kernel A: SpMV + p^T K p or the FP64
 * residual; kernel B: update + preconditioner) is bracketed by CUDA events on
 * the batch's stream and the durations are summed.  Enabling resets the sums.
 * launches counts the (A, B) pairs timed. */
sso_status sso_batch_set_profiling(sso_batch* batch, int32_t enable);
sso_status sso_batch_kernel_times(const sso_batch* batch, double* ms_a, double* ms_b,
                                  int64_t* launches);
/* Set-up and adjoint timing while profiling is enabled (same switch and
 * reset).  sso_batch_solve sets up all its models with one launch per stage:
 * element matrices (Sec. 2.2), assembly of K (Eq. 1), preconditioner + load
 * vector.  ms_elements, ms_assembly and ms_precond are the device
 * milliseconds of those launches (CUDA events on the batch's stream), summed
 * over solves; ms_setup_wall is the elapsed time of the whole set-up phase
 * (the two-level coarse spaces included), summed over solves.  ms_adjoint is
 * the elapsed time of every contraction pass of sso_batch_gradient (the
 * adjoint sum of Eq. 6 and the per-node gather, all models, on a pool of up
 * to 16 streams).  setups counts model set-ups timed, gradients the gradient
 * calls.  Any pointer may be NULL. */
sso_status sso_batch_setup_times(const sso_batch* batch, double* ms_elements,
                                 double* ms_assembly, double* ms_precond, double* ms_adjoint,
                                 double* ms_setup_wall, int64_t* setups, int64_t* gradients);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of design evaluations.  Each request is one
 * structure (any size, any topology) whose solve and adjoint gradient of
 * J = w C (compliance, Sec. 2.3; dJ/dz per node, dJ/dt per quad, Eqs. 5-6)
 * are wanted.  A server keeps up to max_systems requests resident on the GPU
 * (their patterns, K, preconditioners and solver state), within
 * hbm_budget_bytes of per-request device memory and max_tiles tiles of 30
 * nodes.  Every sso_server_step runs one captured CUDA graph of CG iterations
 * over the resident systems; meanwhile it admits waiting requests as slots,
 * tiles and budget allow (their element matrices, assembly and preconditioner
 * run on a second stream and overlap the CG), and when a system has converged
 * it computes its gradient, stores the result on the host and releases its
 * memory.  A request's result is bit-identical to solving it alone with the
 * same options (sso_model_solve + sso_model_gradient(w, NULL)).  Every
 * preconditioner but SSO_CHAIN is served (SSO_TWO_LEVEL: the coarse set-up
 * runs with the request's other set-up kernels).  The server runs on streams
 * of its own; every call returns with the host-visible state
 * up to date.  Not thread-safe.
 */
typedef struct sso_server sso_server;

sso_status sso_server_create(const sso_options* opts, size_t hbm_budget_bytes,
                             int32_t max_systems, int32_t max_tiles, sso_server** out);

/* A server of `lanes` (1..8) independent lanes: each lane is a server with
 * 1/lanes of the budget, slots and tiles; each request goes to the lane with
 * the fewest nodes still to finish, and sso_server_step steps every lane at
 * once (the first on the calling thread, the others on helper threads the
 * server owns), so that the lanes' CG launches fill one another's ramps and
 * tails.  Tickets, completion lists, polls and phase times (summed over the
 * lanes) behave as for one server; a request's result is still bit-identical
 * to solving it alone.  lanes = 1 is sso_server_create. */
sso_status sso_server_create_lanes(const sso_options* opts, size_t hbm_budget_bytes,
                                   int32_t max_systems, int32_t max_tiles, int32_t lanes,
                                   sso_server** out);
void sso_server_destroy(sso_server* server);

/* Queue a request; the mesh (host or device arrays) is copied, and worker
 * threads of the server start building its scatter map at once.  A NULL or
 * incomplete mesh is rejected here (SSO_ERR_INVALID); a mesh whose contents
 * are invalid (node indices, non-finite values) is reported by the request's
 * result status, as is one that can never fit the budget (SSO_ERR_OOM). */
sso_status sso_server_submit(sso_server* server, const sso_mesh* mesh, double w,
                             uint64_t* ticket);

/* One round: a graph launch of CG iterations, admissions, harvesting.
 * n_resident = requests on the GPU, n_waiting = requests queued.  A CUDA
 * error (SSO_ERR_CUDA) is fatal for the server: destroy it.  With
 * SSO_DEBUG_SYNC=1 in the environment every model's scatter map is checked
 * on the host and each phase of the step is synchronised, so that an error
 * names the phase it came from. */
sso_status sso_server_step(sso_server* server, int32_t* n_resident, int32_t* n_waiting);

/* Tickets whose results became ready since the last call (in completion
 * order), at most `capacity` of them; *n receives the count.  Results stay
 * available to sso_server_poll until polled. */
sso_status sso_server_completed(sso_server* server, uint64_t* tickets, int32_t capacity,
                                int32_t* n);

/* Host time spent in each phase of sso_server_step since creation (ms[8]):
 * ms[0] admission (model build, set-up kernels enqueued), ms[1] system-table
 * uploads, ms[2] waiting for the CG graph, ms[3] harvest (adjoint
 * contraction, results to host, freeing the model); parts of ms[0]: ms[4]
 * waiting for the worker threads' preparation, ms[5] arena allocation and
 * upload, ms[6] set-up kernel launches; ms[7] reserved (0).  counts[2]:
 * steps, CG graph launches.  Either pointer may be NULL. */
sso_status sso_server_info(const sso_server* server, double* ms, int64_t* counts);

/* Result of a finished request: SSO_ERR_NOT_READY while it is queued or
 * running; otherwise SSO_OK, the outputs are filled (any pointer may be NULL;
 * u [6*n_nodes], C [1], dz [n_nodes], dt [n_quads], host or device), stats
 * holds the request's status and CG statistics, latency_ms the time from
 * submission to result, and the request is forgotten. */
sso_status sso_server_poll(sso_server* server, uint64_t ticket, double* u, double* C,
                           double* dz, double* dt, sso_stats* stats, double* latency_ms);

#ifdef __cplusplus
}
#endif

#endif /* SSO_H_ */
