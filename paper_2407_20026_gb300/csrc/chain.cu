// Exact solve of K u = b (Eq. 1) for a block-tridiagonal K: every K block
// couples node i with itself or with i +- 1, as for a chain of beam-columns
// numbered along its length (arches, multi-span bridges, cantilevers).
//
// Block cyclic reduction in FP64.  A level holds a chain of n nodes with
// diagonal blocks A_i, couplings B_i = K(i, i+1) (K(i+1, i) = B_i^T) and a
// right-hand side b.  Each odd node i is eliminated through its own
// equation, x_i = A_i^-1 (b_i - B_{i-1}^T x_{i-1} - B_i x_{i+1}), which
// leaves a chain on the even nodes j = 2k:
//   A'_k = A_j - B_{j-1}^T A_{j-1}^-1 B_{j-1} - B_j A_{j+1}^-1 B_j^T
//   B'_k = -B_j A_{j+1}^-1 B_{j+1}
//   b'_k = b_j - B_{j-1}^T A_{j-1}^-1 b_{j-1} - B_j A_{j+1}^-1 b_{j+1}.
// Levels halve the chain down to one node; the solution is recovered level
// by level in reverse with the equation of each odd node.  Every thread
// works on one node of one level in a fixed order, so results are
// reproducible.  The reduced diagonal blocks are Schur complements of an SPD
// matrix, hence SPD: they are inverted by Cholesky, and a non-positive pivot
// sets the error flag.
#include <math.h>

#include "sso_internal.cuh"

namespace sso {
namespace {

constexpr int kChainThreads = 128;

__device__ __forceinline__ void ld36(const double* __restrict__ p, double* m) {
#pragma unroll
  for (int k = 0; k < 36; ++k) m[k] = p[k];
}

// Inverse of an SPD 6x6 block by Cholesky (A = L L^T, A^-1 = L^-T L^-1).
__device__ bool spd_inv6(const double* A, double* Ai) {
  double L[36];
#pragma unroll
  for (int k = 0; k < 36; ++k) L[k] = 0.0;
  for (int j = 0; j < 6; ++j) {
    double d = A[7 * j];
    for (int k = 0; k < j; ++k) d -= L[6 * j + k] * L[6 * j + k];
    if (!(d > 0.0)) return false;
    const double ljj = sqrt(d);
    L[7 * j] = ljj;
    for (int i = j + 1; i < 6; ++i) {
      double s = A[6 * i + j];
      for (int k = 0; k < j; ++k) s -= L[6 * i + k] * L[6 * j + k];
      L[6 * i + j] = s / ljj;
    }
  }
  // W = L^-1 (lower triangular)
  double W[36];
#pragma unroll
  for (int k = 0; k < 36; ++k) W[k] = 0.0;
  for (int c = 0; c < 6; ++c) {
    W[7 * c] = 1.0 / L[7 * c];
    for (int i = c + 1; i < 6; ++i) {
      double s = 0.0;
      for (int k = c; k < i; ++k) s += L[6 * i + k] * W[6 * k + c];
      W[6 * i + c] = -s / L[7 * i];
    }
  }
  // A^-1 = W^T W
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double s = 0.0;
      for (int k = (i > j ? i : j); k < 6; ++k) s += W[6 * k + i] * W[6 * k + j];
      Ai[6 * i + j] = s;
    }
  return true;
}

// Z = X Y, Z = X^T Y, Z = X Y^T (6x6 row-major)
__device__ __forceinline__ void mm(const double* X, const double* Y, double* Z) {
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) s = fma(X[6 * i + k], Y[6 * k + j], s);
      Z[6 * i + j] = s;
    }
}
__device__ __forceinline__ void mtm(const double* X, const double* Y, double* Z) {
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) s = fma(X[6 * k + i], Y[6 * k + j], s);
      Z[6 * i + j] = s;
    }
}
__device__ __forceinline__ void mmt(const double* X, const double* Y, double* Z) {
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) s = fma(X[6 * i + k], Y[6 * j + k], s);
      Z[6 * i + j] = s;
    }
}

// Level 0 from K64: A_i = K(i, i), B_i = K(i, i+1) (zero where absent).
__global__ void __launch_bounds__(kChainThreads) chain_extract_kernel(
    int n, const int* __restrict__ diag, const int* __restrict__ up,
    const double* __restrict__ K64, double* __restrict__ A, double* __restrict__ B) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 36LL * n) return;
  const int i = (int)(idx / 36), e = (int)(idx - 36LL * i);
  A[idx] = K64[(size_t)diag[i] * 36 + e];
  B[idx] = up[i] >= 0 ? K64[(size_t)up[i] * 36 + e] : 0.0;
}

// Inverses of the odd nodes' diagonal blocks: Ainv[k] = A_{2k+1}^-1.
__global__ void __launch_bounds__(kChainThreads) chain_invert_kernel(
    int n, const double* __restrict__ A, double* __restrict__ Ainv, int* __restrict__ err) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = 2 * k + 1;
  if (i >= n) return;
  double a[36], ai[36];
  ld36(A + (size_t)i * 36, a);
  if (!spd_inv6(a, ai)) {
    atomicMax(err, 1);
#pragma unroll
    for (int q = 0; q < 36; ++q) ai[q] = 0.0;
  }
  double* o = Ainv + (size_t)k * 36;
#pragma unroll
  for (int q = 0; q < 36; ++q) o[q] = ai[q];
}

// The even nodes' chain: A'_k, B'_k of node j = 2k.
__global__ void __launch_bounds__(kChainThreads) chain_reduce_kernel(
    int n, const double* __restrict__ A, const double* __restrict__ B,
    const double* __restrict__ Ainv, double* __restrict__ An, double* __restrict__ Bn) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = 2 * k;
  if (j >= n) return;
  double a[36], X[36], T[36], U[36];
  ld36(A + (size_t)j * 36, a);
  if (j >= 1) {  // odd neighbour j - 1: a -= B_{j-1}^T A_{j-1}^-1 B_{j-1}
    ld36(Ainv + (size_t)((j - 1) / 2) * 36, X);
    ld36(B + (size_t)(j - 1) * 36, U);
    mm(X, U, T);
    mtm(U, T, X);
#pragma unroll
    for (int q = 0; q < 36; ++q) a[q] -= X[q];
  }
  double bn[36];
#pragma unroll
  for (int q = 0; q < 36; ++q) bn[q] = 0.0;
  if (j + 1 < n) {  // odd neighbour j + 1: a -= B_j A_{j+1}^-1 B_j^T; B' = -B_j A_{j+1}^-1 B_{j+1}
    ld36(Ainv + (size_t)((j + 1) / 2) * 36, X);
    ld36(B + (size_t)j * 36, U);
    mm(U, X, T);  // T = B_j A_{j+1}^-1
    mmt(T, U, X);
#pragma unroll
    for (int q = 0; q < 36; ++q) a[q] -= X[q];
    if (j + 2 < n) {
      ld36(B + (size_t)(j + 1) * 36, U);
      mm(T, U, X);
#pragma unroll
      for (int q = 0; q < 36; ++q) bn[q] = -X[q];
    }
  }
  double* oa = An + (size_t)k * 36;
  double* ob = Bn + (size_t)k * 36;
#pragma unroll
  for (int q = 0; q < 36; ++q) {
    oa[q] = a[q];
    ob[q] = bn[q];
  }
}

// The even nodes' right-hand side b'_k.
__global__ void __launch_bounds__(kChainThreads) chain_rhs_kernel(
    int n, const double* __restrict__ B, const double* __restrict__ Ainv,
    const double* __restrict__ b, double* __restrict__ bn) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = 2 * k;
  if (j >= n) return;
  double r[6], t[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) r[q] = b[6 * (size_t)j + q];
  if (j >= 1) {  // r -= B_{j-1}^T A_{j-1}^-1 b_{j-1}
    const double* X = Ainv + (size_t)((j - 1) / 2) * 36;
    const double* bb = b + 6 * (size_t)(j - 1);
    for (int p = 0; p < 6; ++p) {
      double s = 0.0;
      for (int q = 0; q < 6; ++q) s = fma(X[6 * p + q], bb[q], s);
      t[p] = s;
    }
    const double* U = B + (size_t)(j - 1) * 36;
    for (int p = 0; p < 6; ++p) {
      double s = 0.0;
      for (int q = 0; q < 6; ++q) s = fma(U[6 * q + p], t[q], s);
      r[p] -= s;
    }
  }
  if (j + 1 < n) {  // r -= B_j A_{j+1}^-1 b_{j+1}
    const double* X = Ainv + (size_t)((j + 1) / 2) * 36;
    const double* bb = b + 6 * (size_t)(j + 1);
    for (int p = 0; p < 6; ++p) {
      double s = 0.0;
      for (int q = 0; q < 6; ++q) s = fma(X[6 * p + q], bb[q], s);
      t[p] = s;
    }
    const double* U = B + (size_t)j * 36;
    for (int p = 0; p < 6; ++p) {
      double s = 0.0;
      for (int q = 0; q < 6; ++q) s = fma(U[6 * p + q], t[q], s);
      r[p] -= s;
    }
  }
#pragma unroll
  for (int q = 0; q < 6; ++q) bn[6 * (size_t)k + q] = r[q];
}

// One node left: x = A^-1 b.
__global__ void chain_last_kernel(const double* __restrict__ A, const double* __restrict__ b,
                                  double* __restrict__ x, int* __restrict__ err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a[36], ai[36];
  ld36(A, a);
  if (!spd_inv6(a, ai)) {
    atomicMax(err, 1);
    for (int q = 0; q < 6; ++q) x[q] = 0.0;
    return;
  }
  for (int p = 0; p < 6; ++p) {
    double s = 0.0;
    for (int q = 0; q < 6; ++q) s = fma(ai[6 * p + q], b[q], s);
    x[p] = s;
  }
}

// Back substitution of one level: even nodes from the reduced chain, odd
// nodes x_i = A_i^-1 (b_i - B_{i-1}^T x_{i-1} - B_i x_{i+1}).
__global__ void __launch_bounds__(kChainThreads) chain_back_kernel(
    int n, const double* __restrict__ B, const double* __restrict__ Ainv,
    const double* __restrict__ b, const double* __restrict__ xn, double* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if ((i & 1) == 0) {
#pragma unroll
    for (int q = 0; q < 6; ++q) x[6 * (size_t)i + q] = xn[6 * (size_t)(i / 2) + q];
    return;
  }
  double r[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) r[q] = b[6 * (size_t)i + q];
  {  // left neighbour i - 1 (even, always present)
    const double* U = B + (size_t)(i - 1) * 36;
    const double* xl = xn + 6 * (size_t)((i - 1) / 2);
    for (int p = 0; p < 6; ++p) {
      double s = 0.0;
      for (int q = 0; q < 6; ++q) s = fma(U[6 * q + p], xl[q], s);
      r[p] -= s;
    }
  }
  if (i + 1 < n) {
    const double* U = B + (size_t)i * 36;
    const double* xr = xn + 6 * (size_t)((i + 1) / 2);
    for (int p = 0; p < 6; ++p) {
      double s = 0.0;
      for (int q = 0; q < 6; ++q) s = fma(U[6 * p + q], xr[q], s);
      r[p] -= s;
    }
  }
  const double* X = Ainv + (size_t)(i / 2) * 36;
  for (int p = 0; p < 6; ++p) {
    double s = 0.0;
    for (int q = 0; q < 6; ++q) s = fma(X[6 * p + q], r[q], s);
    x[6 * (size_t)i + p] = s;
  }
}

unsigned blocks_for(long long n) { return (unsigned)((n + kChainThreads - 1) / kChainThreads); }

}  // namespace

size_t chain_workspace_doubles(int n) {
  size_t total = 0;
  for (long long m = n; m >= 1; m = (m + 1) / 2) {
    total += (size_t)m * (36 + 36 + 6 + 6) + (size_t)(m / 2) * 36;
    if (m == 1) break;
  }
  return total;
}

namespace {
// The level arrays, carved from the workspace in level order.
struct ChainLevel {
  int n;
  double *A, *B, *Ainv, *b, *x;
};
int chain_levels(int n, double* ws, ChainLevel* lv, int max_levels) {
  int L = 0;
  for (long long m = n; L < max_levels; m = (m + 1) / 2) {
    ChainLevel& c = lv[L++];
    c.n = (int)m;
    c.A = ws;
    ws += m * 36;
    c.B = ws;
    ws += m * 36;
    c.b = ws;
    ws += m * 6;
    c.x = ws;
    ws += m * 6;
    c.Ainv = ws;
    ws += (m / 2) * 36;
    if (m == 1) break;
  }
  return L;
}
constexpr int kMaxLevels = 40;
}  // namespace

cudaError_t launch_chain_factor(int n, const int* diag, const int* up, const double* K64,
                                double* ws, int* err, cudaStream_t s) {
  if (n <= 0) return cudaErrorInvalidValue;
  ChainLevel lv[kMaxLevels];
  const int L = chain_levels(n, ws, lv, kMaxLevels);
  chain_extract_kernel<<<blocks_for(36LL * n), kChainThreads, 0, s>>>(n, diag, up, K64, lv[0].A,
                                                                       lv[0].B);
  cudaError_t e = cudaGetLastError();
  for (int l = 0; l + 1 < L && e == cudaSuccess; ++l) {
    const ChainLevel& c = lv[l];
    chain_invert_kernel<<<blocks_for(c.n / 2), kChainThreads, 0, s>>>(c.n, c.A, c.Ainv, err);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    chain_reduce_kernel<<<blocks_for((c.n + 1) / 2), kChainThreads, 0, s>>>(
        c.n, c.A, c.B, c.Ainv, lv[l + 1].A, lv[l + 1].B);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t launch_chain_solve(int n, double* ws, const double* b, double* x, int* err,
                               cudaStream_t s) {
  if (n <= 0) return cudaErrorInvalidValue;
  ChainLevel lv[kMaxLevels];
  const int L = chain_levels(n, ws, lv, kMaxLevels);
  cudaError_t e = cudaMemcpyAsync(lv[0].b, b, sizeof(double) * 6 * (size_t)n,
                                  cudaMemcpyDeviceToDevice, s);
  for (int l = 0; l + 1 < L && e == cudaSuccess; ++l) {
    const ChainLevel& c = lv[l];
    chain_rhs_kernel<<<blocks_for((c.n + 1) / 2), kChainThreads, 0, s>>>(c.n, c.B, c.Ainv, c.b,
                                                                         lv[l + 1].b);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  chain_last_kernel<<<1, 32, 0, s>>>(lv[L - 1].A, lv[L - 1].b, lv[L - 1].x, err);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int l = L - 2; l >= 0 && e == cudaSuccess; --l) {
    const ChainLevel& c = lv[l];
    double* out = l == 0 ? x : c.x;
    chain_back_kernel<<<blocks_for(c.n), kChainThreads, 0, s>>>(c.n, c.B, c.Ainv, c.b,
                                                                lv[l + 1].x, out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && L == 1)
    e = cudaMemcpyAsync(x, lv[0].x, sizeof(double) * 6, cudaMemcpyDeviceToDevice, s);
  return e;
}

// ||b - K64 x||^2 and ||b||^2 of one system, FP64, fixed order: one partial
// pair per CTA, then one CTA sums the partials.
namespace {
constexpr int kResThreads = 192;
__global__ void __launch_bounds__(kResThreads) residual_partials_kernel(
    int n, const int* __restrict__ row_ptr, const int* __restrict__ col,
    const double* __restrict__ K, const double* __restrict__ x, const double* __restrict__ b,
    double* __restrict__ r_out, double* __restrict__ part) {
  __shared__ double red[2][kResThreads / 32];
  const long long i = (long long)blockIdx.x * kResThreads + threadIdx.x;
  double rr = 0.0, bb = 0.0;
  if (i < 6LL * n) {
    const int node = (int)(i / 6), r = (int)(i - 6LL * node);
    double acc = b[i];
    bb = acc * acc;
    for (int j = row_ptr[node]; j < row_ptr[node + 1]; ++j) {
      const double* Kb = K + (size_t)j * 36 + 6 * r;
      const double* xc = x + 6 * (size_t)col[j];
#pragma unroll
      for (int q = 0; q < 6; ++q) acc = fma(-Kb[q], xc[q], acc);
    }
    rr = acc * acc;
    if (r_out) r_out[i] = acc;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_down_sync(0xffffffffu, rr, o);
    bb += __shfl_down_sync(0xffffffffu, bb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = rr;
    red[1][threadIdx.x >> 5] = bb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int w = 0; w < kResThreads / 32; ++w) {
      a += red[0][w];
      c += red[1][w];
    }
    part[2 * (size_t)blockIdx.x] = a;
    part[2 * (size_t)blockIdx.x + 1] = c;
  }
}
__global__ void __launch_bounds__(256) residual_sum_kernel(int m, const double* __restrict__ part,
                                                           double* __restrict__ out) {
  __shared__ double red[2][256];
  double a = 0.0, c = 0.0;
  for (int k = threadIdx.x; k < m; k += 256) {
    a += part[2 * (size_t)k];
    c += part[2 * (size_t)k + 1];
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = c;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      red[0][threadIdx.x] += red[0][threadIdx.x + h];
      red[1][threadIdx.x] += red[1][threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = red[0][0];
    out[1] = red[1][0];
  }
}
}  // namespace

size_t residual_partials(int n) { return 2 * (size_t)((6LL * n + kResThreads - 1) / kResThreads); }

cudaError_t launch_residual_norms(int n, const int* row_ptr, const int* col, const double* K64,
                                  const double* x, const double* b, double* r, double* part,
                                  double* out, cudaStream_t s) {
  const int m = (int)((6LL * n + kResThreads - 1) / kResThreads);
  residual_partials_kernel<<<m, kResThreads, 0, s>>>(n, row_ptr, col, K64, x, b, r, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  residual_sum_kernel<<<1, 256, 0, s>>>(m, part, out);
  return cudaGetLastError();
}

}  // namespace sso
