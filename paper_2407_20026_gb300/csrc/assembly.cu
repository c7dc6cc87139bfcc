// Assembly of K (Eq. 1) from element blocks, supports (Eqs. 2-3 with b = 0,
// by elimination), the (block-)Jacobi preconditioner and per-node gathers.
//
// Assembly is a gather: K block b is the sum of the element blocks listed in
// csrc[cptr[b] .. cptr[b+1]), in that (increasing element-block) order.  The
// list is built once per topology, so the sum order is fixed and the result is
// bit-reproducible without atomics.  One thread per (block, entry): a warp
// reads 32 consecutive doubles of one or two element blocks, so reads and the
// K64/K32 writes are coalesced; the kernel is bound by HBM.
#include <math.h>

#include "sso_internal.cuh"

namespace sso {
namespace {

__global__ void __launch_bounds__(256) assemble_kernel(
    int n_blocks, const int* __restrict__ cptr, const int* __restrict__ csrc,
    const double* __restrict__ ke, const int* __restrict__ brow, const int* __restrict__ col,
    const uint8_t* __restrict__ fixed, double* __restrict__ K64, float* __restrict__ K32) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n_blocks * 36) return;
  const int b = (int)(idx / 36);
  const int k = (int)(idx - (long long)b * 36);
  const int r = k / 6, c = k - 6 * (k / 6);
  double s = 0.0;
  const int c1 = cptr[b + 1];
  for (int i = cptr[b]; i < c1; ++i) s += ke[(size_t)csrc[i] * 36 + k];
  const int ni = brow[b], nj = col[b];
  if (fixed[6 * ni + r] || fixed[6 * nj + c]) s = (ni == nj && r == c) ? 1.0 : 0.0;
  K64[idx] = s;
  K32[idx] = (float)s;
}

// Block-Jacobi: Cholesky-invert the 6x6 diagonal block of every node (FP64).
// Jacobi: invert the diagonal entries.  A non-positive pivot sets *err.
// Layouts: M64 [n][6][6] (Jacobi: [n][6]); M32 packed [n][M32_PACK]
// (Jacobi: [n][6]).
__global__ void __launch_bounds__(128) precond_kernel(int n_nodes, int kind,
                                                      const int* __restrict__ diag_idx,
                                                      const double* __restrict__ K64,
                                                      double* __restrict__ M64,
                                                      float* __restrict__ M32,
                                                      int* __restrict__ err) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
  const double* B = K64 + (size_t)diag_idx[n] * 36;
  if (kind == SSO_JACOBI) {
    for (int i = 0; i < 6; ++i) {
      const double d = B[7 * i];
      const double inv = d > 0.0 ? 1.0 / d : 0.0;
      if (!(d > 0.0)) atomicExch(err, 1);
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
  if (!ok) atomicExch(err, 1);
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

// Per node, in slot order: f = nodal load + area-load shares (uz only; quad
// slots s >= slot_quad0 of fslot), zero on fixed DOFs; dz = sum of the per-slot
// gradient values gslot[s].  Either output may be NULL.  One thread per node.
__global__ void __launch_bounds__(128) node_gather_kernel(
    int n_nodes, const int* __restrict__ nptr, const int* __restrict__ nsrc, int slot_quad0,
    const double* __restrict__ fslot, const double* __restrict__ gslot,
    const double* __restrict__ nodal_load, const uint8_t* __restrict__ fixed,
    double* __restrict__ f, double* __restrict__ dz) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
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

__global__ void axpby_kernel(int n, double a, const double* __restrict__ x,
                             const double* __restrict__ y, const uint8_t* __restrict__ fixed,
                             double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = a * x[i] + (y ? y[i] : 0.0);
  out[i] = fixed[i] ? 0.0 : v;
}

}  // namespace

cudaError_t launch_assemble(int n_blocks, const int* cptr, const int* csrc, const double* ke,
                            const int* brow, const int* col, const uint8_t* fixed,
                            double* K64, float* K32, cudaStream_t s) {
  const long long n = (long long)n_blocks * 36;
  if (n <= 0) return cudaSuccess;
  assemble_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n_blocks, cptr, csrc, ke, brow,
                                                                col, fixed, K64, K32);
  return cudaGetLastError();
}

cudaError_t launch_precond(int n_nodes, int kind, const int* diag_idx, const double* K64,
                           double* M64, float* M32, int* err_flag, cudaStream_t s) {
  if (n_nodes <= 0) return cudaSuccess;
  precond_kernel<<<(n_nodes + 127) / 128, 128, 0, s>>>(n_nodes, kind, diag_idx, K64, M64, M32,
                                                        err_flag);
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
