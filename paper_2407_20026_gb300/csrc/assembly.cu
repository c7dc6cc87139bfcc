// Assembly of K (Eq. 1) from element blocks, supports (Eqs. 2-3 with b = 0,
// by elimination), the (block-)Jacobi preconditioner and per-node gathers.
//
// Assembly is a segmented sum over one contiguous stream: the element kernels
// wrote every element block to its place in assembly order (sorted by K block,
// then by element block id, once per topology), so K block b is the sum of
// kes[cptr[b] .. cptr[b+1]) in that order -- fixed, hence bit-reproducible
// without atomics.  A chunk of consecutive K blocks therefore reads one
// contiguous range, which a CTA brings into shared memory with a single bulk
// copy; its K64 / K32 stores are contiguous runs too.  The kernel is bound by
// HBM.  A batch of structures is set up by one launch per stage (one
// structure per grid row).
#include <math.h>

#include "sso_internal.cuh"

namespace sso {
namespace {

// Pairs of entries per 6x6 block (36 doubles = 18 double2).
constexpr int PAIRS = 18;
// K blocks per CTA, and the shared-memory slab that receives their element
// blocks in one bulk copy (a quad mesh's chunk holds ~1.8 contributions per
// block, at most 4; a chunk whose range does not fit -- a hub node's
// diagonal block -- is summed straight from global memory).
constexpr int ASM_CHUNK = 64;
constexpr int ASM_SLAB = 40 * 1024;
constexpr int ASM_THREADS = 256;

// One CTA per chunk of ASM_CHUNK consecutive K blocks of job blockIdx.y.  The
// chunk's element blocks are the contiguous range kes[cptr[b0] .. cptr[b0 +
// n)): thread 0 copies it into shared memory with one bulk copy (the copy
// engine keeps many KB in flight per SM without registers), while the
// threads stage the chunk's cptr, block rows and columns; then each thread
// sums (block, pair) items from shared memory in cptr order and writes K64
// and its FP32 rounding K32.  Supports turn fixed rows / columns into identity
// rows / columns.  The wait for the copy is bounded: a CTA that gives up sets
// *err = 2 (reported as a CUDA failure) and writes nothing.
__global__ void __launch_bounds__(ASM_THREADS, 5) assemble_bulk_kernel(
    const SetupJob* __restrict__ jobs) {
  extern __shared__ __align__(16) unsigned char asm_slab[];
  __shared__ __align__(8) unsigned long long bar;
  __shared__ int s_cptr[ASM_CHUNK + 1], s_mask[ASM_CHUNK];
  __shared__ int s_staged;
  const SetupJob& J = jobs[blockIdx.y];
  const int b0 = blockIdx.x * ASM_CHUNK;
  const int t = threadIdx.x;
  if (blockIdx.x == 0 && t == 0) *J.err = 0;  // the preconditioner runs next
  if (b0 >= J.n_blocks) return;  // uniform over the CTA
  const int nb = min(ASM_CHUNK, J.n_blocks - b0);
  if (t == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
    const int c0 = __ldg(J.cptr + b0), c1 = __ldg(J.cptr + b0 + nb);
    const uint32_t bytes = (uint32_t)(c1 - c0) * 288u;
    const bool fits = (long long)(c1 - c0) * 288 <= ASM_SLAB;
    s_staged = fits;
    fence_proxy_async();
    if (fits && bytes > 0) {
      mbar_arrive_tx(&bar, bytes);
      bulk_g2s(asm_slab, J.kes + (size_t)c0 * 36, bytes, &bar);
    } else {
      mbar_arrive(&bar);
    }
  }
  if (t <= nb) s_cptr[t] = __ldg(J.cptr + b0 + t);
  if (t < nb) s_mask[t] = __ldg(J.bmask + b0 + t);
  __syncthreads();
  const bool staged = s_staged != 0;
  if (!mbar_wait(&bar, 0)) {
    if (t == 0) atomicExch(J.err, 2);
    mbar_wait(&bar, 0);  // the copy may still land; give it one more bounded wait
    return;
  }
  const int cbase = s_cptr[0];
  const double2* slab = reinterpret_cast<const double2*>(asm_slab);
  const double2* gsrc = reinterpret_cast<const double2*>(J.kes);
  double2* K64 = reinterpret_cast<double2*>(J.K64) + (size_t)b0 * PAIRS;
  float2* K32 = reinterpret_cast<float2*>(J.K32) + (size_t)b0 * PAIRS;
  for (int item = t; item < nb * PAIRS; item += ASM_THREADS) {
    const int lb = item / PAIRS;
    const int p = item - lb * PAIRS;
    const int c0 = s_cptr[lb], c1 = s_cptr[lb + 1];
    // the sum starts from the first contribution (no 0 + v: GB300's FP64 pipe
    // issues about 2 operations per clock per SM, and is this kernel's limit)
    double sx = 0.0, sy = 0.0;
    for (int c = c0; c < c1; ++c) {
      const double2 v = staged ? slab[(size_t)(c - cbase) * PAIRS + p]
                               : __ldcs(gsrc + (size_t)c * PAIRS + p);
      if (c == c0) {
        sx = v.x;
        sy = v.y;
      } else {
        sx += v.x;
        sy += v.y;
      }
    }
    const int r = p / 3, cc = 2 * (p - 3 * r);
    const int m = s_mask[lb];
    const bool fr = (m >> r) & 1, diag = (m >> 12) & 1;
    if (fr || ((m >> (6 + cc)) & 1)) sx = (diag && r == cc) ? 1.0 : 0.0;
    if (fr || ((m >> (7 + cc)) & 1)) sy = (diag && r == cc + 1) ? 1.0 : 0.0;
    K64[item] = make_double2(sx, sy);
    K32[item] = make_float2(f64_to_f32_rn(sx), f64_to_f32_rn(sy));
  }
}

// Block-Jacobi: Cholesky-invert the 6x6 diagonal block of every node (FP64).
// Jacobi: invert the diagonal entries.  A non-positive pivot sets *err.
// Layouts: M64 [n][6][6] (Jacobi: [n][6]); M32 packed [n][M32_PACK]
// (Jacobi: [n][6]).
__device__ __forceinline__ void precond_node(int n, int kind, const int* __restrict__ diag_idx,
                                             const double* __restrict__ K64,
                                             double* __restrict__ M64, float* __restrict__ M32,
                                             int* __restrict__ err) {
  const double* B = K64 + (size_t)diag_idx[n] * 36;
  if (kind == SSO_JACOBI) {
    for (int i = 0; i < 6; ++i) {
      const double d = B[7 * i];
      const double inv = d > 0.0 ? 1.0 / d : 0.0;
      if (!(d > 0.0)) atomicMax(err, 1);
      M64[6 * n + i] = inv;
      M32[6 * n + i] = (float)inv;
    }
    return;
  }
  double L[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) L[i][j] = 0.0;
  bool ok = true;
  for (int j = 0; j < 6; ++j) {
    double s = B[7 * j];
    for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
    if (!(s > 0.0)) {
      ok = false;
      s = 1.0;
    }
    L[j][j] = ::sqrt(s);
    for (int i = j + 1; i < 6; ++i) {
      double t = B[6 * i + j];
      for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
      L[i][j] = t / L[j][j];
    }
  }
  if (!ok) atomicMax(err, 1);
  // inverse of L (lower), then M = L^-T L^-1
  double Li[6][6];
  for (int j = 0; j < 6; ++j) {
    for (int i = 0; i < 6; ++i) Li[i][j] = 0.0;
    Li[j][j] = 1.0 / L[j][j];
    for (int i = j + 1; i < 6; ++i) {
      double t = 0.0;
      for (int k = j; k < i; ++k) t -= L[i][k] * Li[k][j];
      Li[i][j] = t / L[i][i];
    }
  }
  // M64 full; M32 packed (upper triangle, M32_PACK floats per node): the
  // product is symmetric term by term, so nothing is lost
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double t = 0.0;
      for (int k = (i > j ? i : j); k < 6; ++k) t += Li[k][i] * Li[k][j];
      M64[(size_t)n * 36 + 6 * i + j] = t;
      if (i <= j) M32[(size_t)n * M32_PACK + sym6(i, j)] = (float)t;
    }
  for (int k = 21; k < M32_PACK; ++k) M32[(size_t)n * M32_PACK + k] = 0.f;
}

// 32-thread CTAs: FP64-bound per node, spread over SMs for small models
__global__ void __launch_bounds__(128) precond_setup_kernel(const SetupJob* __restrict__ jobs,
                                                            int kind) {
  const SetupJob& J = jobs[blockIdx.y];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < J.n_nodes) precond_node(n, kind, J.diag, J.K64, J.M64, J.M32, J.err);
}

// Per node, in slot order: f = nodal load + area-load shares (uz only; quad
// slots s >= slot_quad0 of fslot), zero on fixed DOFs; dz = sum of the per-slot
// gradient values gslot[s].  Either output may be NULL.  One thread per node.
__device__ __forceinline__ void node_gather(int n, const int* __restrict__ nptr,
                                            const int* __restrict__ nsrc, int slot_quad0,
                                            const double* __restrict__ fslot,
                                            const double* __restrict__ gslot,
                                            const double* __restrict__ nodal_load,
                                            const uint8_t* __restrict__ fixed,
                                            double* __restrict__ f, double* __restrict__ dz) {
  const int s0 = nptr[n], s1 = nptr[n + 1];
  if (f) {
    double fz = nodal_load[6 * n + 2];
    for (int i = s0; i < s1; ++i) {
      const int s = nsrc[i];
      if (s >= slot_quad0) fz += fslot[s];
    }
    for (int d = 0; d < 6; ++d) {
      const double v = d == 2 ? fz : nodal_load[6 * n + d];
      f[6 * n + d] = fixed[6 * n + d] ? 0.0 : v;
    }
  }
  if (dz) {
    double g = 0.0;
    for (int i = s0; i < s1; ++i) g += gslot[nsrc[i]];
    dz[n] = g;
  }
}

__global__ void __launch_bounds__(128) node_gather_kernel(
    int n_nodes, const int* __restrict__ nptr, const int* __restrict__ nsrc, int slot_quad0,
    const double* __restrict__ fslot, const double* __restrict__ gslot,
    const double* __restrict__ nodal_load, const uint8_t* __restrict__ fixed,
    double* __restrict__ f, double* __restrict__ dz) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < n_nodes) node_gather(n, nptr, nsrc, slot_quad0, fslot, gslot, nodal_load, fixed, f, dz);
}

__global__ void __launch_bounds__(128) loads_setup_kernel(const SetupJob* __restrict__ jobs) {
  const SetupJob& J = jobs[blockIdx.y];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < J.n_nodes)
    node_gather(n, J.nptr, J.nsrc, 2 * J.n_beams, J.fslot, nullptr, J.nodal_load, J.fixed, J.f,
                nullptr);
}

__global__ void axpby_kernel(int n, double a, const double* __restrict__ x,
                             const double* __restrict__ y, const uint8_t* __restrict__ fixed,
                             double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = a * x[i] + (y ? y[i] : 0.0);
  out[i] = fixed[i] ? 0.0 : v;
}

}  // namespace

cudaError_t launch_setup_assemble(const SetupJob* jobs, int n_jobs, int max_blocks,
                                  cudaStream_t s) {
  if (n_jobs <= 0 || max_blocks <= 0) return cudaSuccess;
  if (n_jobs > 65535) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(assemble_bulk_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, ASM_SLAB);
    // all of the SM's shared memory for the slabs: five CTAs per SM
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(assemble_bulk_kernel,
                               cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const unsigned chunks = (unsigned)((max_blocks + ASM_CHUNK - 1) / ASM_CHUNK);
  assemble_bulk_kernel<<<dim3(chunks, n_jobs), ASM_THREADS, ASM_SLAB, s>>>(jobs);
  return cudaGetLastError();
}

cudaError_t launch_setup_precond(const SetupJob* jobs, int n_jobs, int max_nodes, int kind,
                                 cudaStream_t s) {
  if (n_jobs <= 0 || max_nodes <= 0) return cudaSuccess;
  if (n_jobs > 65535) return cudaErrorInvalidValue;
  precond_setup_kernel<<<dim3((max_nodes + 31) / 32, n_jobs), 32, 0, s>>>(jobs, kind);
  return cudaGetLastError();
}

cudaError_t launch_setup_loads(const SetupJob* jobs, int n_jobs, int max_nodes, cudaStream_t s) {
  if (n_jobs <= 0 || max_nodes <= 0) return cudaSuccess;
  if (n_jobs > 65535) return cudaErrorInvalidValue;
  loads_setup_kernel<<<dim3((max_nodes + 127) / 128, n_jobs), 128, 0, s>>>(jobs);
  return cudaGetLastError();
}

cudaError_t launch_node_gather(int n_nodes, const int* nptr, const int* nsrc, int slot_quad0,
                               const double* fslot, const double* gslot,
                               const double* nodal_load, const uint8_t* fixed, double* f,
                               double* dz, cudaStream_t s) {
  if (n_nodes <= 0) return cudaSuccess;
  node_gather_kernel<<<(n_nodes + 127) / 128, 128, 0, s>>>(n_nodes, nptr, nsrc, slot_quad0,
                                                            fslot, gslot, nodal_load, fixed, f,
                                                            dz);
  return cudaGetLastError();
}

cudaError_t launch_axpby(int n, double a, const double* x, const double* y, const uint8_t* fixed,
                         double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  axpby_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, a, x, y, fixed, out);
  return cudaGetLastError();
}

}  // namespace sso
