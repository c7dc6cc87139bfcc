// Batched preconditioned CG with FP64 iterative refinement.
//
// One CG iteration over every system of a batch is two kernels, A then B.
// The rows of every system are cut into tiles of TILE consecutive nodes; a
// warp owns NODES_PER_WARP whole nodes of a tile (lane = 6 * node + row, two
// lanes idle) and a CTA of WARPS warps owns a tile.  Each CTA walks a
// contiguous range of tiles.  Every system runs its own state machine, stored
// in its SysScalars:
//
//   INIT   A: r64 = b, ||b||^2             B: start sweep 1 (or finish if b = 0)
//   RESID  A: r64 = b - K64 x (FP64 SpMV), B: finish if ||r64|| <= rtol ||b||,
//             ||r64||^2, ||b||^2              else r = r64 / ||r64||, z = M^-1 r,
//                                             start a new inner sweep
//   PCG    A: p = z + beta p (formed on    B: x += scale alpha p (FP64),
//             the fly for every column       r -= alpha q, z = M^-1 r,
//             read), q = K p, p^T q           r^T z, ||r||^2; beta; end the
//                                             sweep when ||r||^2 <= inner_thr
//   DONE   skipped
//
// In FP32_IR mode r, z, p, q and K are FP32 (K32 = round(K64)); x, r64 and
// every dot product are FP64.  In FP64 mode everything is FP64 and the RESID
// step only confirms the true residual.
//
// Reductions: every warp reduces its rows with shuffles and stores one
// partial per (tile, warp); there is no CTA barrier per tile.  When a CTA has
// finished its run of consecutive tiles of one system it adds the run length
// to the system's completion counter (one integer atomic per run); the CTA
// that brings the counter to the system's tile count sums all of that
// system's partials in (tile, warp) order and updates the scalars.  The
// grouping into tiles and warps depends only on the system itself, so its
// iterates are bit-identical whether it runs alone or inside any batch.
// There are no spin-waits.
#include <math.h>

#include "sso_internal.cuh"

namespace sso {
namespace {

__device__ __forceinline__ void load6(const float* p, float v[6]) {
  const float2* q = reinterpret_cast<const float2*>(p);
  const float2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
}
__device__ __forceinline__ void load6(const double* p, double v[6]) {
  const double2* q = reinterpret_cast<const double2*>(p);
  const double2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
}
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }

template <typename T> struct MatOf;
template <> struct MatOf<float> {
  static __device__ __forceinline__ const float* K(const SysDesc& S) { return S.K32; }
  static __device__ __forceinline__ const float* M(const SysDesc& S) { return S.M32; }
};
template <> struct MatOf<double> {
  static __device__ __forceinline__ const double* K(const SysDesc& S) { return S.K64; }
  static __device__ __forceinline__ const double* M(const SysDesc& S) { return S.M64; }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the NT threads of the CTA in a fixed order; valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < WARPS; ++w) s += red[w];
  }
  __syncthreads();
  return s;
}

// Ordered sum of n values part[k * stride + off]; valid in thread 0.
__device__ __forceinline__ double ordered_sum(const double* part, int n, int stride, int off,
                                              double* red) {
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += NT) v += __ldcg(part + (size_t)k * stride + off);
  return block_sum(v, red);
}

// sum_j K[j][rr][:] . (z + beta pold)[col[j]] over j in [j0, j1), in j order.
// Column indices of a chunk first, then every K-row / z / p load of the chunk
// (indices past the row end are clamped to its last block and their FMAs
// skipped), then the FMAs: the loads of a chunk are in flight together.
template <typename T, int CH>
__device__ __forceinline__ T row_dot(const T* __restrict__ K, const int* __restrict__ col,
                                     int j0, int j1, int rr, const T* __restrict__ z,
                                     const T* __restrict__ pold, T beta) {
  T acc = T(0);
  for (int jb = j0; jb < j1; jb += CH) {
    int cc[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) cc[u] = __ldg(col + min(jb + u, j1 - 1));
    T kv[CH][6], zv[CH][6], pv[CH][6];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      load6(K + (size_t)min(jb + u, j1 - 1) * 36 + rr * 6, kv[u]);
      load6(z + (size_t)cc[u] * 6, zv[u]);
      load6(pold + (size_t)cc[u] * 6, pv[u]);
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      if (jb + u < j1) {
#pragma unroll
        for (int k = 0; k < 6; ++k) acc = fmaT(kv[u][k], fmaT(beta, pv[u][k], zv[u][k]), acc);
      }
    }
  }
  return acc;
}

// The CTA's contiguous range of tiles.
__device__ __forceinline__ void tile_range(int n_tiles, int& begin, int& end) {
  const int per = (n_tiles + (int)gridDim.x - 1) / (int)gridDim.x;
  begin = (int)blockIdx.x * per;
  end = min(n_tiles, begin + per);
}

template <typename T>
__global__ void __launch_bounds__(NT, 4) pcg_a_kernel(const int2* __restrict__ tiles,
                                                      const int* __restrict__ n_tiles_ptr,
                                                      const SysDesc* __restrict__ sys,
                                                      int* __restrict__ flags) {
  __shared__ double red[WARPS];
  __shared__ int s_last;
  int* n_active = flags;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int ln = w * NODES_PER_WARP + lane / 6, rr = lane % 6;
  int begin, end;
  tile_range(*n_tiles_ptr, begin, end);
  int run = 0;  // tiles of the current system done by this CTA since the last count
  for (int tile = begin; tile < end; ++tile) {
    const int2 tl = tiles[tile];
    const SysDesc& S = sys[tl.x];
    SysScalars* sc = S.sc;
    const int state = *(volatile int*)&sc->state;
    if (state == ST_DONE) continue;
    const int node = tl.y + ln;
    const bool act = lane < 6 * NODES_PER_WARP && node < S.n_nodes;
    const int i = 6 * node + rr;
    double part = 0.0, part_b = 0.0;
    if (state == ST_PCG) {
      const T* __restrict__ z = (const T*)S.z;
      const int par = sc->parity;
      const T* pold = (const T*)(par ? S.p1 : S.p0);
      T* pnew = (T*)(par ? S.p0 : S.p1);
      // first iteration of a sweep: p = z, written as z + 0 * z (exact for
      // finite z) so that one code path serves every iteration
      const bool first = sc->inner == 0;
      const T beta = first ? T(0) : (T)sc->beta;
      if (first) pold = z;
      if (act) {
        constexpr int CH = sizeof(T) == 4 ? 3 : 2;
        const int j0 = __ldg(S.row_ptr + node), j1 = __ldg(S.row_ptr + node + 1);
        const T acc = row_dot<T, CH>(MatOf<T>::K(S), S.col, j0, j1, rr, z, pold, beta);
        const T pi = fmaT(beta, pold[i], z[i]);
        pnew[i] = pi;
        ((T*)S.q)[i] = acc;
        part = (double)pi * (double)acc;
      }
    } else {  // ST_INIT or ST_RESID: r64 = b - K64 x in FP64
      if (act) {
        const double bi = S.b[i];
        double acc = bi;
        part_b = bi * bi;
        if (state == ST_RESID) {
          const int j0 = __ldg(S.row_ptr + node), j1 = __ldg(S.row_ptr + node + 1);
          acc -= row_dot<double, 2>(S.K64, S.col, j0, j1, rr, S.x, S.x, 0.0);
        }
        S.r64[i] = acc;
        part = acc * acc;
      }
    }
    part = warp_sum(part);
    part_b = warp_sum(part_b);
    if (lane == 0) {
      double* dst = S.part_a + 2 * ((size_t)(tile - S.tile0) * WARPS + w);
      dst[0] = part;
      dst[1] = part_b;
      __threadfence();
    }
    ++run;
    // end of this CTA's run of the system: count it
    if (tile + 1 < end && tiles[tile + 1].x == tl.x) continue;
    __syncthreads();
    if (t == 0) {
      __threadfence();
      const unsigned prev = atomicAdd(&sc->cnt_a, (unsigned)run);
      s_last = (prev + (unsigned)run == (unsigned)S.n_tiles);
    }
    run = 0;
    __syncthreads();
    if (s_last) {
      __threadfence();
      const int n_part = S.n_tiles * WARPS;
      const double sum = ordered_sum(S.part_a, n_part, 2, 0, red);
      const double sum_b = state == ST_PCG ? 0.0 : ordered_sum(S.part_a, n_part, 2, 1, red);
      if (t == 0) {
        if (state == ST_PCG) {
          sc->pq = sum;
          if (!(sum > 0.0) || !isfinite(sum)) {
            sc->status = SSO_ERR_SINGULAR;
            sc->state = ST_DONE;
            atomicSub(n_active, 1);
          } else {
            sc->alpha = sc->rz / sum;
            sc->parity ^= 1;
          }
        } else {
          sc->rr64 = sum;
          sc->ff = sum_b;
        }
        sc->cnt_a = 0u;
      }
      __syncthreads();
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(NT, 4) pcg_b_kernel(const int2* __restrict__ tiles,
                                                      const int* __restrict__ n_tiles_ptr,
                                                      const SysDesc* __restrict__ sys,
                                                      int* __restrict__ flags) {
  __shared__ double red[WARPS];
  __shared__ int s_last;
  int* n_active = flags;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int ln = w * NODES_PER_WARP + lane / 6, rr = lane % 6;
  const int node_lane0 = lane - rr;  // lane of row 0 of this lane's node
  int begin, end;
  tile_range(*n_tiles_ptr, begin, end);
  int run = 0;
  for (int tile = begin; tile < end; ++tile) {
    const int2 tl = tiles[tile];
    const SysDesc& S = sys[tl.x];
    SysScalars* sc = S.sc;
    const int state = *(volatile int*)&sc->state;
    if (state == ST_DONE) continue;
    const int node = tl.y + ln;
    const bool act = lane < 6 * NODES_PER_WARP && node < S.n_nodes;
    const int i = 6 * node + rr;
    T* r = (T*)S.r;
    const T* __restrict__ M = MatOf<T>::M(S);
    const bool block = S.precond == SSO_BLOCK_JACOBI;
    bool work = true;
    T ri = T(0);
    T mv[6];
    if (state == ST_PCG) {
      const T alpha = (T)sc->alpha;
      const double ua = sc->alpha * sc->scale;
      const T* p = (const T*)(sc->parity ? S.p1 : S.p0);
      if (act) {
        if (block) load6(M + (size_t)node * 36 + rr * 6, mv);
        else mv[0] = M[i];
        S.x[i] = fma(ua, (double)p[i], S.x[i]);
        ri = fmaT(-alpha, ((const T*)S.q)[i], r[i]);
        r[i] = ri;
      }
    } else {
      const double rr64 = sc->rr64;
      work = isfinite(rr64) && !(rr64 <= sc->rtol2 * sc->ff);
      if (work && act) {
        if (block) load6(M + (size_t)node * 36 + rr * 6, mv);
        else mv[0] = M[i];
        ri = (T)(S.r64[i] * (1.0 / ::sqrt(rr64)));
        r[i] = ri;
      }
    }
    double v1 = 0.0, v2 = 0.0;
    if (work) {
      // z = M^-1 r: the node's six residual rows are lanes node_lane0 .. +5
      T zi = T(0);
      if (block) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const T rk = __shfl_sync(0xffffffffu, ri, (node_lane0 + k) & 31);
          zi = fmaT(mv[k], rk, zi);
        }
      } else {
        zi = mv[0] * ri;
      }
      if (act) {
        ((T*)S.z)[i] = zi;
        v1 = (double)ri * (double)zi;
        v2 = (double)ri * (double)ri;
      }
    }
    v1 = warp_sum(v1);
    v2 = warp_sum(v2);
    if (lane == 0) {
      double* dst = S.part_b + 2 * ((size_t)(tile - S.tile0) * WARPS + w);
      dst[0] = v1;
      dst[1] = v2;
      __threadfence();
    }
    ++run;
    if (tile + 1 < end && tiles[tile + 1].x == tl.x) continue;
    __syncthreads();
    if (t == 0) {
      __threadfence();
      const unsigned prev = atomicAdd(&sc->cnt_b, (unsigned)run);
      s_last = (prev + (unsigned)run == (unsigned)S.n_tiles);
    }
    run = 0;
    __syncthreads();
    if (s_last) {
      __threadfence();
      const int n_part = S.n_tiles * WARPS;
      const double s1 = ordered_sum(S.part_b, n_part, 2, 0, red);
      const double s2 = ordered_sum(S.part_b, n_part, 2, 1, red);
      if (t == 0) {
        if (state == ST_PCG) {
          sc->iters += 1;
          sc->inner += 1;
          if (!isfinite(s1) || !isfinite(s2)) {
            sc->status = SSO_ERR_SINGULAR;
            sc->state = ST_DONE;
            atomicSub(n_active, 1);
          } else {
            sc->beta = s1 / sc->rz;
            sc->rz = s1;
            sc->rr = s2;
            if (s2 <= sc->inner_thr || sc->iters >= sc->max_iter) sc->state = ST_RESID;
          }
        } else {
          const double rr64 = sc->rr64;
          if (!isfinite(rr64)) {
            sc->status = SSO_ERR_INVALID;
            sc->state = ST_DONE;
            atomicSub(n_active, 1);
          } else if (rr64 <= sc->rtol2 * sc->ff) {
            sc->status = SSO_OK;
            sc->state = ST_DONE;
            atomicSub(n_active, 1);
          } else if (sc->iters >= sc->max_iter || sc->sweeps >= sc->max_sweeps ||
                     (sc->sweeps >= 2 && rr64 > 0.0625 * sc->rr64_prev)) {
            // cap reached, or the FP64 residual fell by less than 4x over the
            // last sweep (rtol below what this K and FP64 can resolve)
            sc->status = SSO_ERR_NOT_CONVERGED;
            sc->state = ST_DONE;
            atomicSub(n_active, 1);
          } else if (!(s1 > 0.0)) {
            sc->status = SSO_ERR_SINGULAR;  // preconditioner not positive definite
            sc->state = ST_DONE;
            atomicSub(n_active, 1);
          } else {
            sc->rz = s1;
            sc->rr = s2;
            sc->rr_start = s2;
            sc->scale = ::sqrt(rr64);
            sc->rr64_prev = rr64;
            sc->inner_thr = s2 * fmax(sc->inner_rtol2, 0.25 * sc->rtol2 * sc->ff / rr64);
            sc->inner = 0;
            sc->sweeps += 1;
            sc->state = ST_PCG;
          }
        }
        sc->cnt_b = 0u;
      }
      __syncthreads();
    }
  }
}

// out[s] = b_s^T x_s for every system, one CTA per system, fixed order.
__global__ void __launch_bounds__(NT) dot_kernel(const SysDesc* __restrict__ sys,
                                                 double* __restrict__ out) {
  __shared__ double red[WARPS];
  const SysDesc& S = sys[blockIdx.x];
  const int n = 6 * S.n_nodes;
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += NT) v = fma(S.b[i], S.x[i], v);
  const double s = block_sum(v, red);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

}  // namespace

cudaError_t launch_pcg_a(bool fp64, const int2* tiles, const int* n_tiles, const SysDesc* sys,
                         int* flags, int grid, cudaStream_t s) {
  if (fp64)
    pcg_a_kernel<double><<<grid, NT, 0, s>>>(tiles, n_tiles, sys, flags);
  else
    pcg_a_kernel<float><<<grid, NT, 0, s>>>(tiles, n_tiles, sys, flags);
  return cudaGetLastError();
}

cudaError_t launch_pcg_b(bool fp64, const int2* tiles, const int* n_tiles, const SysDesc* sys,
                         int* flags, int grid, cudaStream_t s) {
  if (fp64)
    pcg_b_kernel<double><<<grid, NT, 0, s>>>(tiles, n_tiles, sys, flags);
  else
    pcg_b_kernel<float><<<grid, NT, 0, s>>>(tiles, n_tiles, sys, flags);
  return cudaGetLastError();
}

cudaError_t launch_dot(int n_sys, const SysDesc* sys, double* out, cudaStream_t s) {
  if (n_sys <= 0) return cudaSuccess;
  dot_kernel<<<n_sys, NT, 0, s>>>(sys, out);
  return cudaGetLastError();
}

// CTAs resident on the whole device for each PCG kernel (the range loops
// never need more).
void pcg_grid_limits(bool fp64, int* grid_a, int* grid_b) {
  int dev = 0, sms = 0, per_sm_a = 0, per_sm_b = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (fp64) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_a, pcg_a_kernel<double>, NT, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, pcg_b_kernel<double>, NT, 0);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_a, pcg_a_kernel<float>, NT, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, pcg_b_kernel<float>, NT, 0);
  }
  if (sms < 1) sms = 1;
  *grid_a = sms * (per_sm_a < 1 ? 1 : per_sm_a);
  *grid_b = sms * (per_sm_b < 1 ? 1 : per_sm_b);
}

}  // namespace sso
