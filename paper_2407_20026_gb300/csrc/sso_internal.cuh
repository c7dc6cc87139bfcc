// Internal declarations shared by the CUDA translation units of libsso.
//
// Data layout in device memory (one structure = one "system"):
//   DOF vectors      node-major, 6 entries per node, length 6 * n_nodes
//   K (BSR)          one block row per node; row_ptr [n_nodes+1], col [n_blocks],
//                    values [n_blocks][6][6] row-major (FP64 K64 and FP32 K32)
//   element blocks   ke[eb][6][6] FP64, eb = 4 e + 2 a + b for beam e,
//                    eb = 4 n_beams + 16 e + 4 a + b for quad e
//   node slots       s = 2 e + a for beam e (node a), s = 2 n_beams + 4 e + a
//                    for quad e; per-slot gradient and load values are summed
//                    per node in slot order
//   preconditioner   block-Jacobi: [n_nodes][6][6] inverse diagonal blocks;
//                    Jacobi: [n_nodes*6] inverse diagonal entries
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sso.h"

namespace sso {

// PCG tiling: a tile is TILE consecutive nodes of one system, processed by one
// CTA of WARPS warps; each warp owns NODES_PER_WARP whole nodes, one lane per
// scalar row (6 * NODES_PER_WARP = 30 lanes, two idle).
constexpr int NODES_PER_WARP = 5;
constexpr int WARPS = 6;
constexpr int TILE = NODES_PER_WARP * WARPS;  // 30 nodes
constexpr int NT = 32 * WARPS;                // 192 threads
// Tiling of the stateless BSR product (spmv.cu): SPMV_TILE nodes per CTA of
// 6 * SPMV_TILE threads.
constexpr int SPMV_TILE = 32;

// FOLD (FP32 mode only): the sweep's FP32 correction is added to the FP64
// solution before the FP64 residual pass.
enum SysState : int { ST_INIT = 0, ST_PCG = 1, ST_RESID = 2, ST_DONE = 3, ST_FOLD = 4 };

// Per-system solver scalars (device memory, one per system).
struct SysScalars {
  int state;        // SysState
  int parity;       // which p buffer holds the current direction
  int iters;        // CG iterations, all sweeps
  int inner;        // CG iterations in the current sweep
  int sweeps;       // FP64 residual recomputations after the first
  int status;       // sso_status
  unsigned int cnt_a, cnt_b;  // chunk-completion counters (last-chunk reduction)
  double rz;        // r^T z of the current iteration
  double beta;      // rz_new / rz_old
  double pq;        // p^T K p
  double alpha;     // rz / pq
  double rr;        // ||r||^2 of the recursive (inner) residual
  double rr_start;  // ||r||^2 at the start of the sweep
  double rr64;      // ||b - K64 x||^2, FP64
  double rr64_prev; // rr64 at the start of the previous sweep (stagnation test)
  double ff;        // ||b||^2
  double scale;     // ||b - K64 x|| at the start of the sweep (inner rhs scale)
  double inner_thr; // inner stop: rr <= inner_thr
  double rtol2;     // outer: rr64 <= rtol2 * ff
  double inner_rtol2;
  int max_iter;
  int max_sweeps;
  // two-level preconditioner: kernel B leaves r^T z_b and r^T r here and sets
  // coarse_pending; the coarse kernel adds w^T y and updates the scalars
  int coarse_pending;
  unsigned int coarse_cnt;  // row blocks of the coarse solve done (last-block reduction)
  double rz_b, rr_b;
};

// Static description of one tile of a batch (device memory, built once per
// batch on the host).  The K rows of a tile are the contiguous blocks
// [j0, j0 + nblk); the columns they read lie in the node range of the halo.
// The *_b fields give 16-byte aligned runs for bulk copies.
// A tile's halo (the z / p entries its rows read) is staged as at most this
// many runs of consecutive nodes: the rows above, at and below a tile of a
// row-major grid.
constexpr int HALO_RUNS = 3;

struct TileDesc {
  int sys;     // system index in the batch
  int node0;   // first node of the tile
  int nn;      // nodes in the tile
  int j0;      // row_ptr[node0]
  int nblk;    // row_ptr[node0 + nn] - j0
  int cb;      // first column index to copy (multiple of 4)
  int ncb;     // column indices to copy (multiple of 4)
  int vlo[HALO_RUNS];  // first node of each halo run (even), ascending
  int nv[HALO_RUNS];   // nodes of each halo run (even; 0: unused)
  int rb;      // first row_ptr entry to copy (multiple of 4)
  int nrb;     // row_ptr entries to copy (multiple of 4)
  int stage;   // 1 when the FP32 slab, columns, halo and row_ptr fit the staging buffers
  int stage_k; // 1 when the FP32 slab, columns and row_ptr fit (the halo may not)
};

// Per-system pointers (device memory, one per system of a batch).
struct SysDesc {
  int n_nodes;
  int tile0;        // first tile of this system in the batch tile list
  int n_tiles;
  int precond;      // sso_precond
  const int* row_ptr;
  const int* col;
  // per block: the slot (in nodes) of its column in the staged halo of its
  // row's tile (tiles with stage = 1; fixed by the mesh, built on the host)
  const int* hslot;
  const float* K32;
  const double* K64;
  const float* M32;  // block-Jacobi: packed upper triangle, M32_PACK per node; Jacobi: 6 per node
  const double* M64;
  const double* b;  // right-hand side (FP64)
  double* x;        // solution (FP64)
  void* dx;         // FP32 mode: correction of the current sweep (x += scale dx at its end)
  double* r64;      // FP64 residual
  void* r;          // inner vectors, float or double
  void* z;
  void* p0;
  void* p1;
  void* q;
  double* part_a;   // [2 * WARPS * n_tiles]
  double* part_b;   // [2 * WARPS * n_tiles]
  // two-level reductions: the system's tiles fall in fixed chunks of CHUNK;
  // the kernel that completes a chunk sums its partials, the one that
  // completes the last chunk sums the chunk sums
  int n_chunks;
  unsigned* chunk_cnt;  // [2 * n_chunks]: tiles counted per chunk, kernel A then kernel B
  double* chunk_part;   // [4 * n_chunks]: two sums per chunk, kernel A then kernel B
  // two-level preconditioner (precond == SSO_TWO_LEVEL, FP32 CG):
  // z = z_b + P A_c^-1 P^T r with z_b the block-Jacobi part and P the rigid-body
  // modes of each node aggregate
  int n_agg;              // aggregates; the coarse problem has 6 n_agg unknowns
  const int* agg_ptr;     // [n_agg + 1] node lists of the aggregates
  const int* agg_nodes;   // [n_nodes]
  const int* agg_of;      // [n_nodes]
  const uint8_t* fixed;   // [6 n_nodes] 1 = fixed DOF
  const float* node_rf;   // [n_nodes][4] node position minus its aggregate's centroid
  const float* Aci;       // [6 n_agg][6 n_agg] inverse of the coarse matrix
  float* w;               // [6 n_agg] P^T r
  float* y;               // [6 n_agg] A_c^-1 w
  double* cdot;           // [COARSE_ROW_BLOCKS] w^T y per row block of the coarse solve
  void* zb;               // [6 n_nodes] z_b (FP32)
  // double-float CG (precision SSO_F32X2, small.cu): the low parts of K,
  // K64 - K32 rounded to FP32, [n_blocks * 36] (the element-block scratch)
  float* klo;
  SysScalars* sc;
};

#ifdef __CUDACC__
// Double-float sums of FP32 products: an unevaluated sum hi + lo of two
// floats, formed only with error-free transformations (the exact product
// a b = p + fma(a, b, -p); Knuth's two-sum; a fast two-sum to renormalise),
// so a dot product of FP32 vectors is accumulated to about 48 significant
// bits on the FP32 pipes.  The FP32 CG kernels sum a warp's terms this way
// and convert once to FP64, where every later sum (tiles, chunks) happens:
// on this GPU an FP64 instruction costs a warp about 64 FP32 ones.
// (Also the arithmetic of the one-CTA double-float CG, small.cu.)
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float v = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float hi = __fadd_rn(s, e);
  return {hi, __fsub_rn(e, __fsub_rn(hi, s))};
}
// Fixed-shape tree over the warp; the sum is in lane 0.
__device__ __forceinline__ DF df_warp_sum(DF x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DF y;
    y.hi = __shfl_down_sync(0xffffffffu, x.hi, o);
    y.lo = __shfl_down_sync(0xffffffffu, x.lo, o);
    x = df_add(x, y);
  }
  return x;
}
__device__ __forceinline__ double df_double(DF x) { return (double)x.hi + (double)x.lo; }

// double -> float rounded to nearest even, with integer operations when the
// result is a normal float (every stiffness entry here), else the hardware
// conversion.  GB300 runs double -> float conversions on its FP64 pipe (about
// 2 per clock per SM), which limited assembly; these are ~12 integer ops.
// The 52-bit mantissa keeps its top 23 bits; the 29 dropped bits round up
// above half and at half when the kept part is odd; a carry out of the
// mantissa moves into the exponent (and to infinity past the largest float),
// as rounding does.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const int E = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;  // float biased exponent
  if (E >= 1 && E <= 254) {
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1fffffffu;
    unsigned r = (hi & 0x80000000u) | ((unsigned)E << 23) | m;
    r += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
    return __uint_as_float(r);
  }
  if (((hi & 0x7fffffffu) | lo) == 0u) return __uint_as_float(hi);  // signed zero
  return __double2float_rn(x);
}

// ---------------------------------------------------------------------------
// mbarrier and bulk-copy (1-D TMA) helpers (CG kernels, assembly).  Every
// wait is bounded.
constexpr long long kWaitPolls = 1LL << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// Announces `bytes` more of asynchronous copies in the current phase without
// arriving (the phase then also waits for a later arrival).
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity) {
  for (long long i = 0; i < kWaitPolls; ++i)
    if (mbar_test(bar, parity)) return true;
  return false;
}

#endif

// ---------------------------------------------------------------------------
// Tiles per reduction chunk.  A chunk's kernel-A partials (CHUNK * WARPS)
// are CHUNK_PER_THREAD contiguous ones per thread of a CTA, its kernel-B
// partials (CHUNK) as many per lane of a warp: one round of loads each.
constexpr int CHUNK = 256;
constexpr int CHUNK_PER_THREAD = 8;
static_assert(CHUNK * WARPS == NT * CHUNK_PER_THREAD, "kernel-A chunk: 8 partials per thread");
static_assert(CHUNK == 32 * CHUNK_PER_THREAD, "kernel-B chunk: 8 partials per lane");

// Two-level preconditioner: at most this many node aggregates per system.  The
// coarse solve reads all of A_c^-1 (FP32, [6 n_agg]^2, here <= 219 KB) in every
// CG iteration and holds w in shared memory and 8 columns of two rows per lane
// in registers, so the coarse space stays small.
constexpr int COARSE_MAX_AGG = 39;
constexpr int COARSE_MAX_N = 6 * COARSE_MAX_AGG;
// The coarse solve y = A_c^-1 w of a system is split into row blocks, one CTA each.
constexpr int COARSE_ROWS_PER_BLOCK = 16;
constexpr int COARSE_ROW_BLOCKS = (COARSE_MAX_N + COARSE_ROWS_PER_BLOCK - 1) / COARSE_ROWS_PER_BLOCK;

// Packed symmetric 6x6 (upper triangle by rows, 21 values, 3 zeros of
// padding so that every node starts on a 16-byte boundary).
constexpr int M32_PACK = 24;
__host__ __device__ constexpr int sym6(int a, int c) {
  return a <= c ? a * 6 - a * (a - 1) / 2 + (c - a) : c * 6 - c * (c - 1) / 2 + (a - c);
}

// ---------------------------------------------------------------------------
// Set-up of one structure: element matrices and area-load shares, assembly of
// K64 and K32, the (block-)Jacobi preconditioner, the load vector.  The
// element kernels write every 6x6 element block to its place in assembly
// order (epos: element block -> position, the inverse of the sorted scatter
// map), so the blocks summed into K block b are kes[cptr[b] .. cptr[b+1]),
// contiguous, and assembly reads one stream.  Set-up kernels take an array of
// jobs and run one job per grid row (blockIdx.y): one launch per stage sets
// up a whole batch.
struct SetupJob {
  const double* xyz;
  const int* beam_conn;
  const double* beam_props;
  const int* quad_conn;
  const double* quad_props;
  int n_beams, n_quads, n_nodes, n_blocks;
  double pressure, gamma;
  const int* epos;        // [4 n_beams + 16 n_quads]
  double* kes;            // element blocks in assembly order [n_eb][36]
  double* fslot;          // area-load share per (element, node) slot
  const int* cptr;        // [n_blocks + 1]
  // supports of every block: bits 0-5 fixed rows of its row node, 6-11 fixed
  // columns of its column node, 12 a diagonal block (fixed by the mesh)
  const uint16_t* bmask;
  const uint8_t* fixed;   // [6 n_nodes]
  double* K64;
  float* K32;
  int* err;               // set by a non-positive preconditioner pivot
  const int* diag;        // diagonal block of every node
  double* M64;
  float* M32;
  const int* nptr;        // node incidence (slots by node)
  const int* nsrc;
  const double* nodal_load;
  double* f;
};

// Launchers (set-up stages; elements.cu and assembly.cu).  max_*: the largest
// count over the jobs (the grid's x extent).  n_jobs <= 65535.
cudaError_t launch_store_setup_job(SetupJob* dst, const SetupJob& job, cudaStream_t s);
cudaError_t launch_setup_beams(const SetupJob* jobs, int n_jobs, int max_beams, cudaStream_t s);
cudaError_t launch_setup_quads(const SetupJob* jobs, int n_jobs, int max_quads, cudaStream_t s);
cudaError_t launch_setup_assemble(const SetupJob* jobs, int n_jobs, int max_blocks,
                                  cudaStream_t s);
cudaError_t launch_setup_precond(const SetupJob* jobs, int n_jobs, int max_nodes, int kind,
                                 cudaStream_t s);
cudaError_t launch_setup_loads(const SetupJob* jobs, int n_jobs, int max_nodes, cudaStream_t s);

// ---------------------------------------------------------------------------
// Launchers (elements.cu)
cudaError_t launch_beam_stiffness(int n_beams, const double* xyz, const int* conn,
                                  const double* props, double* ke, cudaStream_t s);
cudaError_t launch_quad_volume(int n_quads, const double* xyz, const int* conn,
                               const double* props, double* vslot, double* dt, double* vol,
                               cudaStream_t s);
cudaError_t launch_ordered_sum(int n, const double* v, double* out, cudaStream_t s);
cudaError_t launch_quad_stiffness(int n_quads, const double* xyz, const int* conn,
                                  const double* props, double pressure, double gamma,
                                  double* ke, double* fslot, cudaStream_t s);
cudaError_t launch_beam_adjoint(int n_beams, const double* xyz, const int* conn,
                                const double* props, const double* u, const double* lam,
                                double lam_scale, double* gslot, cudaStream_t s);
cudaError_t launch_quad_adjoint(int n_quads, const double* xyz, const int* conn,
                                const double* props, double pressure, double gamma,
                                const double* u, const double* lam, double lam_scale,
                                double w, double* gslot, double* dt, cudaStream_t s,
                                const double* rho = nullptr, double penal = 1.0,
                                double* drho = nullptr);
cudaError_t launch_simp(int n_quads, const double* rho, const double* E0, double penal,
                        double* props, cudaStream_t s);

// Launchers (assembly.cu)
cudaError_t launch_precond(int n_nodes, int kind, const int* diag_idx, const double* K64,
                           double* M64, float* M32, int* err_flag, cudaStream_t s);
cudaError_t launch_node_gather(int n_nodes, const int* nptr, const int* nsrc, int slot_quad0,
                               const double* fslot, const double* gslot,
                               const double* nodal_load, const uint8_t* fixed, double* f,
                               double* dz, cudaStream_t s);
cudaError_t launch_axpby(int n, double a, const double* x, const double* y, const uint8_t* fixed,
                         double* out, cudaStream_t s);

// Launchers (pcg.cu)
// flags[0] = systems still iterating, flags[1] = device-side failure (a bounded
// wait that gave up); grid sizes from pcg_grid_limits.  Kernel A's grid may be
// grid_mult times the resident CTA count (its tile ranges then shorten).
cudaError_t launch_pcg_a(bool fp64, const TileDesc* tiles, const int* n_tiles,
                         const SysDesc* sys, int* flags, int grid, int grid_mult,
                         cudaStream_t s);
cudaError_t launch_pcg_b(bool fp64, const TileDesc* tiles, const int* n_tiles,
                         const SysDesc* sys, int* flags, int grid, cudaStream_t s);
// Staging-buffer limits of the FP32 kernel A (a tile is staged when it fits).
constexpr int STAGE_SLAB_K = 40 * 1024;  // K rows (bytes)
constexpr int STAGE_SLAB_C = 1280;       // column indices (bytes)
constexpr int STAGE_SLAB_V = 6144;       // one vector halo (bytes)
constexpr int STAGE_SLAB_R = 256;        // row_ptr run (bytes)
cudaError_t launch_dot(int n_sys, const SysDesc* sys, double* out, cudaStream_t s);

// Launchers (small.cu): the whole double-float CG of each listed system in
// one CTA (systems sys[list[0 .. n_list)]); threads a multiple of 32, <= 1024.
cudaError_t launch_small_cg(const SysDesc* sys, const int* list, int n_list, int threads,
                            int max_nodes, bool two_level, cudaStream_t s);
// The coarse correction of the two-level preconditioner, after kernel B:
// restriction (one warp per (system, aggregate) of `aggs`), coarse solve and
// scalar update (COARSE_ROW_BLOCKS work items per system of `csys`),
// prolongation (the tiles).  The list lengths are read from the device
// (*n_aggs, *n_csys); `grid` CTAs loop over the items.
struct AggRef {
  int sys, agg;
};
cudaError_t launch_coarse_restrict(const AggRef* aggs, const int* n_aggs, int grid,
                                   const SysDesc* sys, cudaStream_t s);
cudaError_t launch_coarse_solve(const int* csys, const int* n_csys, int grid, const SysDesc* sys,
                                int* flags, cudaStream_t s);
cudaError_t launch_coarse_prolong(const TileDesc* tiles, const int* n_tiles, const SysDesc* sys,
                                  int grid, cudaStream_t s);

// Coarse set-up of one model (coarse.cu): aggregate geometry, Galerkin matrix
// A_c = P^T K P (FP64, dense [6 n_agg]^2), its FP32 inverse.  W: scratch of
// 2 coarse_padded_n(n_agg)^2 floats; coarse_setup_launches(n_agg) kernels.
int coarse_padded_n(int n_agg);
int coarse_setup_launches(int n_agg);
cudaError_t launch_coarse_setup(int n_nodes, int n_agg, int n_blocks, const int* agg_ptr,
                                const int* agg_nodes, const int* brow, const int* col,
                                const int* cg_ptr, const int* cg_src, const double* xyz,
                                const uint8_t* fixed, const double* K64, double* node_r64,
                                float* node_rf, double* T, double* Ac, float* W, float* Aci,
                                cudaStream_t s);

// Direct solve of a block-tridiagonal K by block cyclic reduction (chain.cu).
// ws: chain_workspace_doubles(n) doubles; up[i]: index of block (i, i+1) in
// the BSR arrays or -1; err set on a non-positive pivot.
size_t chain_workspace_doubles(int n);
cudaError_t launch_chain_factor(int n, const int* diag, const int* up, const double* K64,
                                double* ws, int* err, cudaStream_t s);
cudaError_t launch_chain_solve(int n, double* ws, const double* b, double* x, int* err,
                               cudaStream_t s);
// r = b - K64 x (if r is not NULL), out[0] = ||r||^2, out[1] = ||b||^2 (FP64,
// fixed order); part: residual_partials(n) doubles of scratch.
size_t residual_partials(int n);
cudaError_t launch_residual_norms(int n, const int* row_ptr, const int* col, const double* K64,
                                  const double* x, const double* b, double* r, double* part,
                                  double* out, cudaStream_t s);

// Launchers (spmv.cu): y = K x, *xty = x^T y; partials [ceil(n_nodes/TILE)],
// counter must be 0 on entry and is 0 again on exit.
cudaError_t launch_bsr_spmv(int n_nodes, const int* row_ptr, const int* col, const double* K,
                            const double* x, double* y, double* xty, double* partials,
                            unsigned int* counter, cudaStream_t s);
void pcg_grid_limits(bool fp64, int* grid_a, int* grid_b);

}  // namespace sso
