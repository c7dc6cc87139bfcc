// Coarse level of the two-level preconditioner (set-up, once per design).
//
// The nodes of a system are split into aggregates (host, per topology).  The
// six rigid-body modes of an aggregate -- translations t and rotations theta
// about its centroid, u_i = t + theta x r_i at node i, rotation theta -- are
// the columns of P: node i's 6x6 block is B_i = [[I, X_i], [0, I]] with
// X_i theta = theta x r_i, its rows of fixed DOFs zeroed.  The coarse matrix
// A_c = P^T K P is formed from the FP64 K block by block (Galerkin) and summed
// per aggregate pair in a fixed order; its inverse is formed in FP32 by
// blocked Gauss-Jordan elimination without pivoting (A_c is SPD, so every
// pivot block -- a diagonal block of a Schur complement -- is SPD too; modes
// with no stiffness -- an aggregate whose DOFs are all fixed -- are dropped).
#include <algorithm>

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

// One CTA per aggregate pair: its 6x6 block of A_c, each entry the sum of
// that entry over the pair's K blocks.  Group q of 36 threads (one per entry)
// sums the list's blocks q, q + G, q + 2G, ... (four running sums, loads in
// flight together), then the group sums are added in group order.
constexpr int kGatherGroups = 14;
__global__ void __launch_bounds__(36 * kGatherGroups) galerkin_gather_kernel(
    int n_agg, const int* __restrict__ cg_ptr, const int* __restrict__ cg_src,
    const double* __restrict__ T, double* __restrict__ Ac) {
  constexpr int G = kGatherGroups;
  __shared__ double part[G][36];
  const int p = blockIdx.x, g = p / n_agg, h = p - g * n_agg;
  const int t = threadIdx.x, q = t / 36, ent = t - 36 * q;
  const int b = cg_ptr[p], e = cg_ptr[p + 1];
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int k = b + q;
  for (; k + 3 * G < e; k += 4 * G) {
    const int s0 = cg_src[k], s1 = cg_src[k + G], s2 = cg_src[k + 2 * G], s3 = cg_src[k + 3 * G];
    a0 += T[(size_t)s0 * 36 + ent];
    a1 += T[(size_t)s1 * 36 + ent];
    a2 += T[(size_t)s2 * 36 + ent];
    a3 += T[(size_t)s3 * 36 + ent];
  }
  for (; k < e; k += G) a0 += T[(size_t)cg_src[k] * 36 + ent];
  part[q][ent] = (a0 + a1) + (a2 + a3);
  __syncthreads();
  if (t < 36) {
    double sum = 0.0;
#pragma unroll
    for (int j = 0; j < G; ++j) sum += part[j][t];
    const int nc = 6 * n_agg;
    Ac[(size_t)(6 * g + t / 6) * nc + 6 * h + t % 6] = sum;
  }
}

// Blocked Gauss-Jordan inverse of A_c in FP32.  The work matrix W is A_c
// padded to np = 32 nb rows with the identity, and with the rows and columns
// of dead modes (diagonal <= 1e-9 of the largest) replaced by the identity.
// Block step k (one launch, one CTA per 32x32 tile (i, j), reading W_in and
// writing W_out):
//   P = W_kk^-1                       (each CTA, unblocked Gauss-Jordan)
//   R_j = P W_kj (j != k), R_k = P
//   W_kj <- R_j;   W_ij <- [j != k] W_ij - W_ik R_j  (i != k)
// After the nb steps W = A_c^-1 (the standard in-place block Gauss-Jordan
// inversion); Aci = its symmetric part, zero on dead modes.
constexpr int GJ = 32;
constexpr int GJ_THREADS = 256;

// The largest FP32 diagonal entry of A_c (every thread of the CTA gets it).
__device__ float coarse_diag_max(int nc, const double* __restrict__ Ac, float* red) {
  const int tid = threadIdx.x;
  float m = 0.f;
  for (int k = tid; k < nc; k += blockDim.x) m = fmaxf(m, (float)Ac[(size_t)k * nc + k]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) red[tid >> 5] = m;
  __syncthreads();
  m = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
  return m;
}

__device__ __forceinline__ bool coarse_dead(int nc, const double* __restrict__ Ac, int k,
                                            float dmax) {
  return !((float)Ac[(size_t)k * nc + k] > 1e-9f * dmax);
}

__global__ void __launch_bounds__(GJ_THREADS) coarse_gj_load_kernel(int nc, int np,
                                                                    const double* __restrict__ Ac,
                                                                    float* __restrict__ W) {
  __shared__ float red[GJ_THREADS / 32];
  __shared__ int dead_r[GJ], dead_c[GJ];
  const float dmax = coarse_diag_max(nc, Ac, red);
  const int r0 = GJ * blockIdx.y, c0 = GJ * blockIdx.x, tid = threadIdx.x;
  if (tid < GJ) {
    const int r = r0 + tid, c = c0 + tid;
    dead_r[tid] = r >= nc || coarse_dead(nc, Ac, r, dmax);
    dead_c[tid] = c >= nc || coarse_dead(nc, Ac, c, dmax);
  }
  __syncthreads();
  for (int e = tid; e < GJ * GJ; e += GJ_THREADS) {
    const int lr = e / GJ, lc = e % GJ, r = r0 + lr, c = c0 + lc;
    float v;
    if (dead_r[lr] || dead_c[lc])
      v = r == c ? 1.f : 0.f;
    else
      v = (float)Ac[(size_t)r * nc + c];
    W[(size_t)r * np + c] = v;
  }
}

__global__ void __launch_bounds__(GJ_THREADS) coarse_gj_step_kernel(int np, int k,
                                                                    const float* __restrict__ Win,
                                                                    float* __restrict__ Wout) {
  __shared__ float P[GJ][GJ + 1], X[GJ][GJ + 1], Y[GJ][GJ + 1], R[GJ][GJ + 1];
  __shared__ float f[GJ], prow[GJ];
  const int bi = blockIdx.y, bj = blockIdx.x, tid = threadIdx.x;
  const int lc = tid % GJ, lr0 = tid / GJ;  // rows lr0 + 8u, column lc
  constexpr int RPT = GJ * GJ / GJ_THREADS;
  const size_t kk0 = (size_t)GJ * k;
#pragma unroll
  for (int u = 0; u < RPT; ++u) {
    const int lr = lr0 + (GJ_THREADS / GJ) * u;
    P[lr][lc] = Win[(kk0 + lr) * np + kk0 + lc];
    if (bj != k) X[lr][lc] = Win[(kk0 + lr) * np + (size_t)GJ * bj + lc];
    if (bi != k) Y[lr][lc] = Win[((size_t)GJ * bi + lr) * np + kk0 + lc];
  }
  float wij[RPT];
#pragma unroll
  for (int u = 0; u < RPT; ++u) {
    const int lr = lr0 + (GJ_THREADS / GJ) * u;
    wij[u] = (bi != k && bj != k) ? Win[((size_t)GJ * bi + lr) * np + (size_t)GJ * bj + lc] : 0.f;
  }
  __syncthreads();
  // P <- P^-1: per pivot m, the pivot row scaled by 1/p_mm, every other row
  // r less f_r times it (f: column m before the step)
  for (int m = 0; m < GJ; ++m) {
    if (tid < GJ)
      f[tid] = P[tid][m];
    else if (tid < 2 * GJ)
      prow[tid - GJ] = P[m][tid - GJ];
    __syncthreads();
    const float inv = 1.f / f[m];
    const float pr = lc == m ? inv : prow[lc] * inv;
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      const int lr = lr0 + (GJ_THREADS / GJ) * u;
      P[lr][lc] = lr == m ? pr : fmaf(-f[lr], pr, lc == m ? 0.f : P[lr][lc]);
    }
    __syncthreads();
  }
  // R = P X (or P)
#pragma unroll
  for (int u = 0; u < RPT; ++u) {
    const int lr = lr0 + (GJ_THREADS / GJ) * u;
    float acc = 0.f;
    if (bj == k) {
      acc = P[lr][lc];
    } else {
#pragma unroll 8
      for (int m = 0; m < GJ; ++m) acc = fmaf(P[lr][m], X[m][lc], acc);
    }
    R[lr][lc] = acc;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < RPT; ++u) {
    const int lr = lr0 + (GJ_THREADS / GJ) * u;
    float v;
    if (bi == k) {
      v = R[lr][lc];
    } else {
      v = wij[u];
#pragma unroll 8
      for (int m = 0; m < GJ; ++m) v = fmaf(-Y[lr][m], R[m][lc], v);
    }
    Wout[((size_t)GJ * bi + lr) * np + (size_t)GJ * bj + lc] = v;
  }
}

__global__ void __launch_bounds__(GJ_THREADS) coarse_gj_store_kernel(int nc, int np,
                                                                     const double* __restrict__ Ac,
                                                                     const float* __restrict__ W,
                                                                     float* __restrict__ Aci) {
  __shared__ float red[GJ_THREADS / 32];
  __shared__ int dead_r[GJ], dead_c[GJ];
  const float dmax = coarse_diag_max(nc, Ac, red);
  const int r0 = GJ * blockIdx.y, c0 = GJ * blockIdx.x, tid = threadIdx.x;
  if (tid < GJ) {
    const int r = r0 + tid, c = c0 + tid;
    dead_r[tid] = r >= nc || coarse_dead(nc, Ac, r, dmax);
    dead_c[tid] = c >= nc || coarse_dead(nc, Ac, c, dmax);
  }
  __syncthreads();
  for (int e = tid; e < GJ * GJ; e += GJ_THREADS) {
    const int lr = e / GJ, lc = e % GJ, r = r0 + lr, c = c0 + lc;
    if (r >= nc || c >= nc) continue;
    float v = 0.5f * (W[(size_t)r * np + c] + W[(size_t)c * np + r]);
    if (dead_r[lr] || dead_c[lc]) v = 0.f;
    Aci[(size_t)r * nc + c] = v;
  }
}

}  // namespace

int coarse_padded_n(int n_agg) { return GJ * ((6 * std::max(n_agg, 1) + GJ - 1) / GJ); }

int coarse_setup_launches(int n_agg) { return 5 + coarse_padded_n(n_agg) / GJ; }

cudaError_t launch_coarse_setup(int n_nodes, int n_agg, int n_blocks, const int* agg_ptr,
                                const int* agg_nodes, const int* brow, const int* col,
                                const int* cg_ptr, const int* cg_src, const double* xyz,
                                const uint8_t* fixed, const double* K64, double* node_r64,
                                float* node_rf, double* T, double* Ac, float* W, float* Aci,
                                cudaStream_t s) {
  if (n_agg <= 0 || n_agg > COARSE_MAX_AGG || n_nodes <= 0) return cudaErrorInvalidValue;
  const int nc = 6 * n_agg, np = coarse_padded_n(n_agg), nb = np / GJ;
  coarse_geom_kernel<<<(n_agg * 32 + 127) / 128, 128, 0, s>>>(n_agg, agg_ptr, agg_nodes, xyz,
                                                               node_r64, node_rf);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  galerkin_product_kernel<<<(n_blocks + 127) / 128, 128, 0, s>>>(n_blocks, brow, col, K64, fixed,
                                                                  node_r64, T);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  galerkin_gather_kernel<<<n_agg * n_agg, 36 * kGatherGroups, 0, s>>>(n_agg, cg_ptr, cg_src, T,
                                                                      Ac);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const dim3 tiles(nb, nb);
  float* w[2] = {W, W + (size_t)np * np};
  coarse_gj_load_kernel<<<tiles, GJ_THREADS, 0, s>>>(nc, np, Ac, w[0]);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int k = 0; k < nb; ++k) {
    coarse_gj_step_kernel<<<tiles, GJ_THREADS, 0, s>>>(np, k, w[k & 1], w[(k + 1) & 1]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  coarse_gj_store_kernel<<<tiles, GJ_THREADS, 0, s>>>(nc, np, Ac, w[nb & 1], Aci);
  return cudaGetLastError();
}

}  // namespace sso
