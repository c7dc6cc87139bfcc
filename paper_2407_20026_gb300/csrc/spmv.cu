// Stateless FP64 6x6-block sparse product y = K x with the dot product x^T y
// (the K u of Eq. 1 for an assembled K), behind sso_bsr_spmv.
//
// One CTA per tile of TILE nodes, one thread per scalar row; every tile writes
// its partial of x^T y to scratch, and the CTA completing the last tile sums
// the partials in tile order (deterministic; no float atomics).  The scratch
// (n_tiles doubles + a counter) is allocated per call, stream-ordered.
#include <math.h>

#include "sso_internal.cuh"

namespace sso {

__device__ __forceinline__ void spmv_load6(const double* p, double v[6]) {
  const double2* q = reinterpret_cast<const double2*>(p);
  const double2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
}

__global__ void __launch_bounds__(6 * SPMV_TILE) bsr_spmv_kernel(int n_nodes, const int* __restrict__ row_ptr,
                                                      const int* __restrict__ col,
                                                      const double* __restrict__ K,
                                                      const double* __restrict__ x,
                                                      double* __restrict__ y,
                                                      double* __restrict__ xty,
                                                      double* __restrict__ partials,
                                                      unsigned int* __restrict__ counter) {
  __shared__ double red[6 * SPMV_TILE / 32];
  __shared__ int s_last;
  const int t = threadIdx.x;
  const int ln = t / 6, rr = t - 6 * (t / 6);
  const int node = blockIdx.x * SPMV_TILE + ln;
  double part = 0.0;
  if (node < n_nodes) {
    const int i = 6 * node + rr;
    double acc = 0.0;
    const int j1 = __ldg(row_ptr + node + 1);
    for (int j = __ldg(row_ptr + node); j < j1; ++j) {
      const int c = __ldg(col + j);
      double kv[6], xv[6];
      spmv_load6(K + (size_t)j * 36 + rr * 6, kv);
      spmv_load6(x + (size_t)c * 6, xv);
#pragma unroll
      for (int k = 0; k < 6; ++k) acc = fma(kv[k], xv[k], acc);
    }
    y[i] = acc;
    part = x[i] * acc;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((t & 31) == 0) red[t >> 5] = part;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < 6 * SPMV_TILE / 32; ++w) s += red[w];
    partials[blockIdx.x] = s;
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    s_last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    double v = 0.0;
    for (int k = t; k < (int)gridDim.x; k += 6 * SPMV_TILE) v += __ldcg(partials + k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((t & 31) == 0) red[t >> 5] = v;
    __syncthreads();
    if (t == 0) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < 6 * SPMV_TILE / 32; ++w) s += red[w];
      *xty = s;
      *counter = 0u;
    }
  }
}

cudaError_t launch_bsr_spmv(int n_nodes, const int* row_ptr, const int* col, const double* K,
                            const double* x, double* y, double* xty, double* partials,
                            unsigned int* counter, cudaStream_t s) {
  const int tiles = (n_nodes + SPMV_TILE - 1) / SPMV_TILE;
  if (tiles <= 0) return cudaSuccess;
  bsr_spmv_kernel<<<tiles, 6 * SPMV_TILE, 0, s>>>(n_nodes, row_ptr, col, K, x, y, xty, partials, counter);
  return cudaGetLastError();
}

}  // namespace sso
