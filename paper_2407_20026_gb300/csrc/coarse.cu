// Coarse level of the two-level preconditioner (set-up, once per design).
//
// The nodes of a system are split into aggregates (host, per topology).  The
// six rigid-body modes of an aggregate -- translations t and rotations theta
// about its centroid, u_i = t + theta x r_i at node i, rotation theta -- are
// the columns of P: node i's 6x6 block is B_i = [[I, X_i], [0, I]] with
// X_i theta = theta x r_i, its rows of fixed DOFs zeroed.  The coarse matrix
// A_c = P^T K P is formed from the FP64 K block by block (Galerkin) and summed
// per aggregate pair in a fixed order; its inverse is formed in FP32 by
// Gauss-Jordan elimination in one CTA's shared memory (A_c is SPD; modes with
// no stiffness -- an aggregate whose DOFs are all fixed -- are dropped).
#include "sso_internal.cuh"

namespace sso {
namespace {

// One warp per aggregate: the centroid of its nodes (lane-strided partial
// sums, fixed-shape tree), then every node's offset from it.
__global__ void coarse_geom_kernel(int n_agg, const int* __restrict__ agg_ptr,
                                   const int* __restrict__ agg_nodes,
                                   const double* __restrict__ xyz, double* __restrict__ node_r64,
                                   float* __restrict__ node_rf) {
  const int g = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (g >= n_agg) return;
  const int b = agg_ptr[g], e = agg_ptr[g + 1];
  double c[3] = {0.0, 0.0, 0.0};
  for (int k = b + lane; k < e; k += 32) {
    const int i = agg_nodes[k];
#pragma unroll
    for (int d = 0; d < 3; ++d) c[d] += xyz[3 * i + d];
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c[d] += __shfl_down_sync(0xffffffffu, c[d], o);
    c[d] = __shfl_sync(0xffffffffu, c[d], 0) / (double)(e - b);
  }
  for (int k = b + lane; k < e; k += 32) {
    const int i = agg_nodes[k];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double r = xyz[3 * i + d] - c[d];
      node_r64[3 * i + d] = r;
      node_rf[4 * i + d] = (float)r;
    }
    node_rf[4 * i + 3] = 0.f;
  }
}

// One thread per K block (i, j): T = B_i^T (D_i K_ij D_j) B_j, D the free-DOF
// masks, with B = [[I, X], [0, I]], X v = v x r:
//   K B_j = [K[:,0:3], K[:,0:3] X_j + K[:,3:6]],  B_i^T M = [M[0:3,:]; X_i^T M[0:3,:] + M[3:6,:]].
__global__ void __launch_bounds__(128) galerkin_product_kernel(
    int nb, const int* __restrict__ brow, const int* __restrict__ col,
    const double* __restrict__ K64, const uint8_t* __restrict__ fixed,
    const double* __restrict__ node_r64, double* __restrict__ T) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int i = brow[b], j = col[b];
  double K[6][6];
#pragma unroll
  for (int r = 0; r < 6; ++r)
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const bool live = !fixed[6 * i + r] && !fixed[6 * j + c];
      K[r][c] = live ? K64[(size_t)b * 36 + 6 * r + c] : 0.0;
    }
  const double ri[3] = {node_r64[3 * i], node_r64[3 * i + 1], node_r64[3 * i + 2]};
  const double rj[3] = {node_r64[3 * j], node_r64[3 * j + 1], node_r64[3 * j + 2]};
  // X = matrix of v -> v x r: X = [[0, r2, -r1], [-r2, 0, r0], [r1, -r0, 0]]
  const double Xj[3][3] = {{0.0, rj[2], -rj[1]}, {-rj[2], 0.0, rj[0]}, {rj[1], -rj[0], 0.0}};
  const double Xi[3][3] = {{0.0, ri[2], -ri[1]}, {-ri[2], 0.0, ri[0]}, {ri[1], -ri[0], 0.0}};
  double KB[6][6];
#pragma unroll
  for (int r = 0; r < 6; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c) KB[r][c] = K[r][c];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double s = K[r][3 + c];
#pragma unroll
      for (int m = 0; m < 3; ++m) s = fma(K[r][m], Xj[m][c], s);
      KB[r][3 + c] = s;
    }
  }
  double* out = T + (size_t)b * 36;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
#pragma unroll
    for (int r = 0; r < 3; ++r) out[6 * r + c] = KB[r][c];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      double s = KB[3 + r][c];
#pragma unroll
      for (int m = 0; m < 3; ++m) s = fma(Xi[m][r], KB[m][c], s);
      out[6 * (3 + r) + c] = s;
    }
  }
}

// One thread per entry of an aggregate pair's 6x6 block of A_c: the sum of
// that entry over the pair's K blocks, in the order of the host-built list.
__global__ void galerkin_gather_kernel(int n_agg, const int* __restrict__ cg_ptr,
                                       const int* __restrict__ cg_src,
                                       const double* __restrict__ T, double* __restrict__ Ac) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long pairs = (long long)n_agg * n_agg;
  if (t >= pairs * 36) return;
  const int p = (int)(t / 36), e = (int)(t - 36LL * p);
  const int g = p / n_agg, h = p - g * n_agg;
  double s = 0.0;
  for (int k = cg_ptr[p]; k < cg_ptr[p + 1]; ++k) s += T[(size_t)cg_src[k] * 36 + e];
  const int nc = 6 * n_agg;
  Ac[(size_t)(6 * g + e / 6) * nc + 6 * h + e % 6] = s;
}

// One CTA: A_c^-1 in FP32 by Gauss-Jordan elimination in shared memory.
constexpr int kInvThreads = 1024;
__global__ void __launch_bounds__(kInvThreads) coarse_invert_kernel(int nc,
                                                                    const double* __restrict__ Ac,
                                                                    float* __restrict__ Aci) {
  extern __shared__ float A[];  // nc * nc
  __shared__ float f[COARSE_MAX_N];
  __shared__ int dead[COARSE_MAX_N];
  __shared__ float dmax;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  for (int k = tid; k < nc * nc; k += blockDim.x) A[k] = (float)Ac[k];
  __syncthreads();
  if (tid == 0) {
    float m = 0.f;
    for (int k = 0; k < nc; ++k) m = fmaxf(m, A[k * nc + k]);
    dmax = m;
  }
  __syncthreads();
  for (int k = tid; k < nc; k += blockDim.x) dead[k] = !(A[k * nc + k] > 1e-9f * dmax);
  __syncthreads();
  for (int r = warp; r < nc; r += nw)
    for (int c = lane; c < nc; c += 32)
      if (dead[r] || dead[c]) A[r * nc + c] = r == c ? 1.f : 0.f;
  __syncthreads();
  for (int kk = 0; kk < nc; ++kk) {
    for (int r = tid; r < nc; r += blockDim.x) f[r] = A[r * nc + kk];
    __syncthreads();
    const float inv = 1.f / f[kk];
    for (int c = tid; c < nc; c += blockDim.x)
      A[kk * nc + c] = c == kk ? inv : A[kk * nc + c] * inv;
    __syncthreads();
    for (int r = warp; r < nc; r += nw) {
      if (r == kk) continue;
      const float fr = f[r];
      for (int c = lane; c < nc; c += 32)
        A[r * nc + c] = c == kk ? -fr * inv : fmaf(-fr, A[kk * nc + c], A[r * nc + c]);
    }
    __syncthreads();
  }
  for (int r = warp; r < nc; r += nw)
    for (int c = lane; c < nc; c += 32) {
      float v = 0.5f * (A[r * nc + c] + A[c * nc + r]);
      if (dead[r] || dead[c]) v = 0.f;
      Aci[(size_t)r * nc + c] = v;
    }
}

}  // namespace

cudaError_t launch_coarse_setup(int n_nodes, int n_agg, int n_blocks, const int* agg_ptr,
                                const int* agg_nodes, const int* brow, const int* col,
                                const int* cg_ptr, const int* cg_src, const double* xyz,
                                const uint8_t* fixed, const double* K64, double* node_r64,
                                float* node_rf, double* T, double* Ac, float* Aci,
                                cudaStream_t s) {
  if (n_agg <= 0 || n_agg > COARSE_MAX_AGG || n_nodes <= 0) return cudaErrorInvalidValue;
  static bool attr = false;
  const int nc = 6 * n_agg;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(coarse_invert_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         COARSE_MAX_N * COARSE_MAX_N * (int)sizeof(float));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  coarse_geom_kernel<<<(n_agg * 32 + 127) / 128, 128, 0, s>>>(n_agg, agg_ptr, agg_nodes, xyz,
                                                               node_r64, node_rf);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  galerkin_product_kernel<<<(n_blocks + 127) / 128, 128, 0, s>>>(n_blocks, brow, col, K64, fixed,
                                                                  node_r64, T);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const long long entries = 36LL * n_agg * n_agg;
  galerkin_gather_kernel<<<(unsigned)((entries + 255) / 256), 256, 0, s>>>(n_agg, cg_ptr, cg_src,
                                                                           T, Ac);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  coarse_invert_kernel<<<1, kInvThreads, (size_t)nc * nc * sizeof(float), s>>>(nc, Ac, Aci);
  return cudaGetLastError();
}

}  // namespace sso
