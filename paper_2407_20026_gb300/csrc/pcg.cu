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
//   PCG    A: p = z + beta p (formed on    B: x += scale alpha p (FP64; in
//             the fly for every column       FP32 mode dx += alpha p), r -= alpha q,
//             read), q = K p, p^T q           z = M^-1 r, r^T z, ||r||^2; beta;
//                                             end the sweep when ||r||^2 <= inner_thr
//   FOLD   A: skipped                      B: x += scale dx, dx = 0 (FP32 mode)
//   DONE   skipped
//
// In FP32_IR mode r, z, p, q, dx and K are FP32 (K32 = round(K64)); x, r64
// and every dot product are FP64, and a sweep ends PCG -> FOLD -> RESID.  In
// FP64 mode everything is FP64, x is updated directly and the RESID step only
// confirms the true residual.
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
#include <climits>
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
template <> struct MatOf<double> {
  static __device__ __forceinline__ const double* K(const SysDesc& S) { return S.K64; }
  static __device__ __forceinline__ const double* M(const SysDesc& S) { return S.M64; }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Programmatic dependent launch: a CG kernel lets the next kernel of the
// stream begin launching as soon as all of its own CTAs run (its grids are one
// wave, so waiting CTAs never hold back its own), and waits for the previous
// kernel's completion and memory before its first read of solver state.
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

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

// The CTA's contiguous range of tiles.  A grid of `mult` CTAs per resident
// CTA slot cuts a long list into short ranges that the block scheduler hands
// out as SMs free up; a range is never cut below kMinTilesPerCta tiles (a
// CTA's fixed costs would dominate), nor made longer than one wave of the
// resident slots would make it.  With mult = 1 this is the even split.
constexpr int kMinTilesPerCta = 16;
__device__ __forceinline__ void tile_range(int n_tiles, int& begin, int& end, int mult = 1) {
  const int g = (int)gridDim.x, res = max(1, g / max(mult, 1));
  const int per_all = (n_tiles + g - 1) / g, per_res = (n_tiles + res - 1) / res;
  const int per = min(per_res, max(per_all, kMinTilesPerCta));
  begin = (int)blockIdx.x * per;
  end = min(n_tiles, begin + per);
}

// Dynamic state of one system as the kernels of one launch see it: it only
// changes at the very end of a launch (by the CTA that completes the system),
// so a CTA reads it once per run of consecutive tiles of that system.
struct RunState {
  int state;
  int parity;
  int first;
  double beta, alpha, scale, rr64, ff, rtol2;
};

__device__ __forceinline__ RunState read_state(const SysScalars* sc) {
  RunState r;
  r.state = *(volatile const int*)&sc->state;
  r.parity = sc->parity;
  r.first = sc->inner == 0;
  r.beta = sc->beta;
  r.alpha = sc->alpha;
  r.scale = sc->scale;
  r.rr64 = sc->rr64;
  r.ff = sc->ff;
  r.rtol2 = sc->rtol2;
  return r;
}

// Scalar update of kernel A for one system (one thread): sum = p^T q in a CG
// iteration, else ||r64||^2; sum_b = ||b||^2.
__device__ __forceinline__ void finish_a_scalars(SysScalars* sc, int state, double sum,
                                                 double sum_b, int* n_active) {
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

// Sums of the pairs p[2e], p[2e + 1] for e in [e0, min(e0 + CHUNK_PER_THREAD, e1)),
// in e order; every load is issued before the first add.
__device__ __forceinline__ void sum_pairs(const double* p, int e0, int e1, double& a,
                                          double& b) {
  double x[CHUNK_PER_THREAD], y[CHUNK_PER_THREAD];
#pragma unroll
  for (int u = 0; u < CHUNK_PER_THREAD; ++u) {
    const int e = e0 + u;
    x[u] = e < e1 ? __ldcg(p + 2 * (size_t)e) : 0.0;
    y[u] = e < e1 ? __ldcg(p + 2 * (size_t)e + 1) : 0.0;
  }
  a = 0.0;
  b = 0.0;
#pragma unroll
  for (int u = 0; u < CHUNK_PER_THREAD; ++u) {
    a += x[u];
    b += y[u];
  }
}

// Kernel A, end of a CTA's run of the system-local tiles [r0, r1) (their
// partials written): the run is counted into its chunks; a chunk completed
// here is summed (CHUNK_PER_THREAD contiguous partials per thread), and the
// chunk that completes the system leads to the sum of the chunk sums and the
// scalar update.  Every grouping depends on the system alone.  sync() is a
// barrier over the NT threads running this, bsum() their fixed-order sum
// (valid in thread 0); flag is shared scratch; count = false (an aborted CTA)
// counts nothing.
template <typename Sync, typename BSum>
__device__ __forceinline__ void a_count_run(const SysDesc& S, SysScalars* sc, int state, int r0,
                                            int r1, int t, int* n_active, int* flag, bool count,
                                            Sync sync, BSum bsum) {
  for (int c = r0 / CHUNK; c * CHUNK < r1; ++c) {
    const int lo = max(r0, c * CHUNK), hi = min(r1, (c + 1) * CHUNK);
    const int m = min(CHUNK, S.n_tiles - c * CHUNK);
    if (t == 0) {
      int done = 0;
      if (count) {
        __threadfence();
        const unsigned prev = atomicAdd(&S.chunk_cnt[c], (unsigned)(hi - lo));
        done = prev + (unsigned)(hi - lo) == (unsigned)m;
      }
      *flag = done;
    }
    sync();
    const bool done = *flag != 0;
    sync();
    if (!done) continue;
    __threadfence();
    double v, vb;
    sum_pairs(S.part_a + 2 * (size_t)c * CHUNK * WARPS, CHUNK_PER_THREAD * t, m * WARPS, v, vb);
    const double ca = bsum(v);
    const double cb = bsum(vb);
    if (S.n_chunks == 1) {  // the chunk is the system
      if (t == 0) {
        S.chunk_cnt[c] = 0u;
        finish_a_scalars(sc, state, ca, cb, n_active);
      }
      sync();
      continue;
    }
    if (t == 0) {
      S.chunk_part[2 * c] = ca;
      S.chunk_part[2 * c + 1] = cb;
      S.chunk_cnt[c] = 0u;
      __threadfence();
      const unsigned prev = atomicAdd(&sc->cnt_a, 1u);
      *flag = prev + 1u == (unsigned)S.n_chunks;
    }
    sync();
    const bool last = *flag != 0;
    sync();
    if (!last) continue;
    __threadfence();
    double sa = 0.0, sb = 0.0;
    for (int q = t; q < S.n_chunks; q += NT) {
      sa += __ldcg(S.chunk_part + 2 * (size_t)q);
      sb += __ldcg(S.chunk_part + 2 * (size_t)q + 1);
    }
    const double A = bsum(sa);
    const double Bs = bsum(sb);
    if (t == 0) finish_a_scalars(sc, state, A, Bs, n_active);
    sync();
  }
}

// Kernel A, FP64 CG (and any system kernel A reads from global memory).
template <typename T>
__global__ void __launch_bounds__(NT, 3) pcg_a_kernel(const TileDesc* __restrict__ tiles,
                                                      const int* __restrict__ n_tiles_ptr,
                                                      const SysDesc* __restrict__ sys,
                                                      int* __restrict__ flags, int grid_mult) {
  __shared__ double red[WARPS];
  __shared__ int s_last;
  pdl_trigger();
  int* n_active = flags;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int ln = w * NODES_PER_WARP + lane / 6, rr = lane % 6;
  int begin, end;
  tile_range(*n_tiles_ptr, begin, end, grid_mult);
  pdl_wait();
  int run = 0, cur = -1;
  RunState R;
  R.state = ST_DONE;
  for (int tile = begin; tile < end; ++tile) {
    const int sid = tiles[tile].sys;
    const int node0 = tiles[tile].node0;
    const SysDesc& S = sys[sid];
    SysScalars* sc = S.sc;
    if (sid != cur) {
      cur = sid;
      R = read_state(sc);
    }
    if (R.state == ST_DONE || R.state == ST_FOLD) continue;
    const int state = R.state;
    const int node = node0 + ln;
    const bool act = lane < 6 * NODES_PER_WARP && node < S.n_nodes;
    const int i = 6 * node + rr;
    double part = 0.0, part_b = 0.0;
    if (state == ST_PCG) {
      const T* __restrict__ z = (const T*)S.z;
      const T* pold = R.first ? z : (const T*)(R.parity ? S.p1 : S.p0);
      T* pnew = (T*)(R.parity ? S.p0 : S.p1);
      // first iteration of a sweep: p = z, written as z + 0 * z (exact for
      // finite z) so that one code path serves every iteration
      const T beta = R.first ? T(0) : (T)R.beta;
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
    }
    ++run;
    // end of this CTA's run of the system: count it
    if (tile + 1 < end && tiles[tile + 1].sys == sid) continue;
    const int r1 = tile - S.tile0 + 1;
    __syncthreads();
    a_count_run(S, sc, state, r1 - run, r1, t, n_active, &s_last, true,
                [] { __syncthreads(); }, [&](double v) { return block_sum(v, red); });
    run = 0;
  }
}

// Kernel B of the FP64 CG.  Pure streaming per node (no neighbours): one thread owns one
// node (all six rows), so z = M^-1 r is a 6x6 product in registers and every
// vector is read as 24- or 48-byte runs.  Warp w of a CTA takes every
// WARPS-th tile of the CTA's range; a tile (TILE nodes) is one warp.  The
// warp reduces the tile's r^T z and r^T r with shuffles, lane 0 stores the
// tile's partials and adds 1 to the system's completion counter; the warp that
// completes the system sums all of its tile partials in tile order and updates
// the scalars.  No CTA barriers; the grouping depends on the system only, so
// results are bit-identical alone and in any batch.
__device__ __forceinline__ void ld4x9(const double* p, double m[36]) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int k = 0; k < 18; ++k) {
    const double2 v = __ldg(q + k);
    m[2 * k] = v.x; m[2 * k + 1] = v.y;
  }
}
__device__ __forceinline__ void ld6rw(const float* p, float v[6]) {
  const float2* q = reinterpret_cast<const float2*>(p);
  const float2 a = q[0], b = q[1], c = q[2];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
}
__device__ __forceinline__ void ld6rw(const double* p, double v[6]) {
  const double2* q = reinterpret_cast<const double2*>(p);
  const double2 a = q[0], b = q[1], c = q[2];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
}
__device__ __forceinline__ void st6(float* p, const float v[6]) {
  float2* q = reinterpret_cast<float2*>(p);
  q[0] = make_float2(v[0], v[1]);
  q[1] = make_float2(v[2], v[3]);
  q[2] = make_float2(v[4], v[5]);
}
__device__ __forceinline__ void st6(double* p, const double v[6]) {
  double2* q = reinterpret_cast<double2*>(p);
  q[0] = make_double2(v[0], v[1]);
  q[1] = make_double2(v[2], v[3]);
  q[2] = make_double2(v[4], v[5]);
}

// Scalar update of kernel B for one system, by one thread, once every tile of
// the system has been counted.  s1 = r^T z, s2 = r^T r.
__device__ __forceinline__ void finish_b(SysScalars* sc, int state, double s1, double s2,
                                         int* n_active, bool fold) {
  if (state == ST_FOLD) {  // the correction has been added to x by every tile
    sc->state = ST_RESID;
  } else if (state == ST_PCG) {
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
      if (s2 <= sc->inner_thr || sc->iters >= sc->max_iter) sc->state = fold ? ST_FOLD : ST_RESID;
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
               (sc->sweeps >= 2 && rr64 > 0.0625 * sc->rr64_prev &&
                !(sc->inner_rtol2 > 1e-12))) {
      // cap reached, or the FP64 residual fell by less than 4x over the last
      // sweep although the inner solve was already run to 1e-6 (rtol below
      // what this K and FP64 can resolve)
      sc->status = SSO_ERR_NOT_CONVERGED;
      sc->state = ST_DONE;
      atomicSub(n_active, 1);
    } else if (!(s1 > 0.0)) {
      sc->status = SSO_ERR_SINGULAR;  // preconditioner not positive definite
      sc->state = ST_DONE;
      atomicSub(n_active, 1);
    } else {
      // a sweep that gained less than 4x: the inner FP32 solve stopped before
      // its own residual was trustworthy; run the following sweeps 10x tighter
      if (sc->sweeps >= 2 && rr64 > 0.0625 * sc->rr64_prev) sc->inner_rtol2 *= 0.01;
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

// Two-level preconditioner: kernel B has only z_b = M_b^-1 r; it leaves
// r^T z_b and r^T r for the coarse kernel, which adds w^T y and updates the
// scalars (finish_b).
__device__ __forceinline__ void defer_b(SysScalars* sc, double rz_b, double rr) {
  sc->rz_b = rz_b;
  sc->rr_b = rr;
  sc->coarse_pending = 1;
  sc->cnt_b = 0u;
}

// Kernel B, warp level: adds n of this warp's tiles to chunk c of system S.
// The warp that completes a chunk sums the chunk's tile partials
// (CHUNK_PER_THREAD contiguous ones per lane); the one that completes the last chunk sums the chunk sums in order
// and updates the scalars.  Every grouping depends on the system alone.
__device__ __forceinline__ void b_count(const SysDesc& S, SysScalars* sc, int state, int c, int n,
                                        int lane, int* n_active, bool fold, bool defer = false) {
  const int m = min(CHUNK, S.n_tiles - c * CHUNK);
  unsigned* cnt = S.chunk_cnt + S.n_chunks;
  double* cpart = S.chunk_part + 2 * (size_t)S.n_chunks;
  int done = 0;
  if (lane == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&cnt[c], (unsigned)n);
    done = prev + (unsigned)n == (unsigned)m;
  }
  if (!__shfl_sync(0xffffffffu, done, 0)) return;
  __threadfence();
  double v1, v2;
  sum_pairs(S.part_b + 2 * (size_t)c * CHUNK, CHUNK_PER_THREAD * lane, m, v1, v2);
  v1 = warp_sum(v1);
  v2 = warp_sum(v2);
  if (S.n_chunks == 1) {  // the chunk is the system
    if (lane == 0) {
      cnt[c] = 0u;
      if (defer)
        defer_b(sc, v1, v2);
      else
        finish_b(sc, state, v1, v2, n_active, fold);
    }
    return;
  }
  int last = 0;
  if (lane == 0) {
    cpart[2 * c] = v1;
    cpart[2 * c + 1] = v2;
    cnt[c] = 0u;
    __threadfence();
    const unsigned prev = atomicAdd(&sc->cnt_b, 1u);
    last = prev + 1u == (unsigned)S.n_chunks;
  }
  if (!__shfl_sync(0xffffffffu, last, 0)) return;
  __threadfence();
  double a1 = 0.0, a2 = 0.0;
  for (int q = lane; q < S.n_chunks; q += 32) {
    a1 += __ldcg(cpart + 2 * (size_t)q);
    a2 += __ldcg(cpart + 2 * (size_t)q + 1);
  }
  a1 = warp_sum(a1);
  a2 = warp_sum(a2);
  if (lane == 0) {
    if (defer)
      defer_b(sc, a1, a2);
    else
      finish_b(sc, state, a1, a2, n_active, fold);
  }
}

template <typename T>
__global__ void __launch_bounds__(NT, 4) pcg_b_kernel(const TileDesc* __restrict__ tiles,
                                                      const int* __restrict__ n_tiles_ptr,
                                                      const SysDesc* __restrict__ sys,
                                                      int* __restrict__ flags) {
  pdl_trigger();
  int* n_active = flags;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int begin, end;
  tile_range(*n_tiles_ptr, begin, end);
  pdl_wait();
  int cur = -1;
  RunState R;
  R.state = ST_DONE;
  bool work = false, block = true;
  double inv_norm = 0.0, ua = 0.0;
  T alpha = T(0);
  int pend_c = -1, pend_n = 0;
  for (int tile = begin + w; tile < end; tile += WARPS) {
    const TileDesc& td = tiles[tile];
    const int sid = td.sys;
    const SysDesc& S = sys[sid];
    SysScalars* sc = S.sc;
    if (sid != cur) {
      cur = sid;
      R = read_state(sc);
      work = R.state == ST_PCG || (isfinite(R.rr64) && !(R.rr64 <= R.rtol2 * R.ff));
      inv_norm = R.state == ST_PCG ? 0.0 : 1.0 / ::sqrt(R.rr64);
      alpha = (T)R.alpha;
      ua = R.alpha * R.scale;
      block = S.precond != SSO_JACOBI;
    }
    if (R.state == ST_DONE) continue;
    const int state = R.state;
    const int node = td.node0 + lane;
    double v1 = 0.0, v2 = 0.0;
    if (lane < td.nn && work) {
      const size_t i0 = 6 * (size_t)node;
      T* r = (T*)S.r + i0;
      const T* M = MatOf<T>::M(S);
      T rv[6];
      if (state == ST_PCG) {
        T pv[6], qv[6];
        double xv[6];
        load6((const T*)(R.parity ? S.p1 : S.p0) + i0, pv);
        load6((const T*)S.q + i0, qv);
        ld6rw(r, rv);
        ld6rw(S.x + i0, xv);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          xv[k] = fma(ua, (double)pv[k], xv[k]);
          rv[k] = fmaT(-alpha, qv[k], rv[k]);
        }
        st6(S.x + i0, xv);
      } else {
        double gv[6];
        ld6rw(S.r64 + i0, gv);
#pragma unroll
        for (int k = 0; k < 6; ++k) rv[k] = (T)(gv[k] * inv_norm);
      }
      st6(r, rv);
      T zv[6];
      if (block) {
        T mv[36];
        ld4x9(M + 36 * (size_t)node, mv);
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          T s = T(0);
#pragma unroll
          for (int c = 0; c < 6; ++c) s = fmaT(mv[6 * a + c], rv[c], s);
          zv[a] = s;
        }
      } else {
        T mv[6];
        load6(M + i0, mv);
#pragma unroll
        for (int a = 0; a < 6; ++a) zv[a] = mv[a] * rv[a];
      }
      st6((T*)S.z + i0, zv);
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        v1 += (double)rv[a] * (double)zv[a];
        v2 += (double)rv[a] * (double)rv[a];
      }
    }
    v1 = warp_sum(v1);
    v2 = warp_sum(v2);
    const int lt = tile - S.tile0;
    if (lane == 0) {
      double* dst = S.part_b + 2 * (size_t)lt;
      dst[0] = v1;
      dst[1] = v2;
    }
    // count the warp's tiles per chunk, flushing when the chunk or the run ends
    if (lt / CHUNK != pend_c) {
      if (pend_n) b_count(S, sc, state, pend_c, pend_n, lane, n_active, false);
      pend_c = lt / CHUNK;
      pend_n = 0;
    }
    ++pend_n;
    if (!(tile + WARPS < end && tiles[tile + WARPS].sys == sid)) {
      b_count(S, sc, state, pend_c, pend_n, lane, n_active, false);
      pend_c = -1;
      pend_n = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// Kernel B for the FP32 CG.  A warp owns a tile (TILE nodes) at a time and
// works from its own two-stage slice of shared memory.  While it computes one
// tile, lane 0 has already issued the bulk copies (cp.async.bulk) of the
// warp's next tile into the other stage: the tile's packed preconditioner
// blocks (M32_PACK floats per node; Jacobi: 6) and its p, q, r and dx runs.
// One thread per node then computes
//   dx += alpha p,  r -= alpha q,  z = M^-1 r,  r^T z,  r^T r
// from shared memory, and r, z and dx go back out as coalesced runs.  The
// solution update of a CG sweep accumulates in dx (FP32, in units of the
// sweep's scaled system); when the sweep ends the system passes through FOLD,
// where x += scale dx in FP64 (and dx = 0) before the FP64 residual pass.
// Every stage completes one mbarrier phase per tile (a plain arrival when
// the tile needs no copy), and every wait is bounded: a warp whose wait gives
// up raises the error flag and runs its remaining tiles without work.
// Reductions: one partial per tile; a warp counts its run of consecutive tiles
// of one system with a single atomic, and the warp that completes the system
// sums the partials in tile order.
constexpr int B32_M = M32_PACK * TILE;   // floats of preconditioner per stage
constexpr int B32_V = 6 * TILE;          // floats per vector run of a tile
constexpr int B32_STAGE = B32_M + 4 * B32_V;
constexpr int B32_SMEM = WARPS * 2 * B32_STAGE * (int)sizeof(float);

__device__ __forceinline__ uint32_t round16(uint32_t b) { return (b + 15u) & ~15u; }

__device__ __forceinline__ void store_run(float* dst, const float* src, int n2, int lane) {
  float2* g = reinterpret_cast<float2*>(dst);
  const float2* d = reinterpret_cast<const float2*>(src);
  for (int k = lane; k < n2; k += 32) g[k] = d[k];
}

// What a warp knows about one of its tiles before it touches the data.
struct BJob {
  int tile, sid, node0, nn;
  const SysDesc* S;
  RunState R;
  bool work, block;
  int kind;  // 2: PCG (M and four vectors staged), 1: INIT / RESID (M staged), 0: none
};

// The fields of a tile descriptor a warp of kernel B needs, loaded a tile
// ahead of their use.
struct BTile {
  int sys, node0, nn;
};
__device__ __forceinline__ BTile load_btile(const TileDesc* __restrict__ tiles, int tile) {
  const TileDesc& td = tiles[tile];
  return BTile{td.sys, td.node0, td.nn};
}

__device__ __forceinline__ BJob make_bjob(const BTile& td, const SysDesc* __restrict__ sys,
                                          int tile, const BJob* prev) {
  BJob J;
  J.tile = tile;
  J.sid = td.sys;
  J.node0 = td.node0;
  J.nn = td.nn;
  J.S = sys + J.sid;
  if (prev && prev->sid == J.sid) {
    J.R = prev->R;
    J.work = prev->work;
    J.block = prev->block;
  } else {
    // a system's state cannot change while this warp still holds uncounted
    // tiles of it, so it may be read ahead
    J.R = read_state(J.S->sc);
    J.work = J.R.state == ST_PCG || J.R.state == ST_FOLD ||
             (isfinite(J.R.rr64) && !(J.R.rr64 <= J.R.rtol2 * J.R.ff));
    J.block = J.S->precond != SSO_JACOBI;
  }
  J.kind = !J.work ? 0 : J.R.state == ST_PCG ? 2
                       : (J.R.state == ST_INIT || J.R.state == ST_RESID) ? 1 : 0;
  return J;
}

// Lane 0: start the copies of job J into stage buffer st (mbarrier bar).
__device__ __forceinline__ void issue_bjob(const BJob& J, float* st, unsigned long long* bar) {
  if (J.kind == 0) {
    mbar_arrive(bar);
    return;
  }
  const SysDesc& S = *J.S;
  const size_t v0 = 6 * (size_t)J.node0;
  const uint32_t mb = J.block ? (uint32_t)J.nn * (M32_PACK * 4u) : round16((uint32_t)J.nn * 24u);
  const uint32_t vb = round16((uint32_t)J.nn * 24u);
  fence_proxy_async();
  mbar_arrive_tx(bar, mb + (J.kind == 2 ? 4u * vb : 0u));
  bulk_g2s(st, J.block ? S.M32 + (size_t)J.node0 * M32_PACK : S.M32 + v0, mb, bar);
  if (J.kind == 2) {
    bulk_g2s(st + B32_M, (const float*)(J.R.parity ? S.p1 : S.p0) + v0, vb, bar);
    bulk_g2s(st + B32_M + B32_V, (const float*)S.q + v0, vb, bar);
    bulk_g2s(st + B32_M + 2 * B32_V, (const float*)S.r + v0, vb, bar);
    bulk_g2s(st + B32_M + 3 * B32_V, (const float*)S.dx + v0, vb, bar);
  }
}

__global__ void __launch_bounds__(NT, 3) pcg_b32_kernel(const TileDesc* __restrict__ tiles,
                                                        const int* __restrict__ n_tiles_ptr,
                                                        const SysDesc* __restrict__ sys,
                                                        int* __restrict__ flags) {
  extern __shared__ __align__(128) float b32_smem[];
  __shared__ __align__(8) unsigned long long full[WARPS][2];
  pdl_trigger();
  int* n_active = flags;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* stages = b32_smem + w * 2 * B32_STAGE;
  if (lane == 0) {
    mbar_init(&full[w][0], 1);
    mbar_init(&full[w][1], 1);
    fence_barrier_init();
  }
  __syncwarp();
  int begin, end;
  tile_range(*n_tiles_ptr, begin, end);
  // The preconditioner blocks do not change during a solve: the first tile's
  // copy of them is issued before waiting for kernel A and overlaps its tail.
  // That stage announces the four vector runs too, which follow the wait
  // (kernel A writes p and q) whatever the system's state turns out to be.
  BTile first;
  if (begin + w < end) {
    first = load_btile(tiles, begin + w);
    if (lane == 0) {
      const SysDesc& S0 = sys[first.sys];
      const bool blk = S0.precond != SSO_JACOBI;
      const uint32_t mb =
          blk ? (uint32_t)first.nn * (M32_PACK * 4u) : round16((uint32_t)first.nn * 24u);
      const uint32_t vb = round16((uint32_t)first.nn * 24u);
      fence_proxy_async();
      mbar_arrive_tx(&full[w][0], mb + 4u * vb);
      bulk_g2s(stages, blk ? S0.M32 + (size_t)first.node0 * M32_PACK
                           : S0.M32 + 6 * (size_t)first.node0,
               mb, &full[w][0]);
    }
  }
  pdl_wait();
  int k = 0, pend_c = -1, pend_n = 0, last_k[2] = {-1, -1};
  bool dry = false;
  BJob J;
  BTile pf;  // descriptor of the warp's tile after next
  if (begin + w < end) {
    J = make_bjob(first, sys, begin + w, nullptr);
    if (lane == 0) {
      const size_t v0 = 6 * (size_t)J.node0;
      const uint32_t vb = round16((uint32_t)J.nn * 24u);
      const SysDesc& S0 = *J.S;
      const float* pv = (const float*)(J.R.parity ? S0.p1 : S0.p0);
      bulk_g2s(stages + B32_M, pv + v0, vb, &full[w][0]);
      bulk_g2s(stages + B32_M + B32_V, (const float*)S0.q + v0, vb, &full[w][0]);
      bulk_g2s(stages + B32_M + 2 * B32_V, (const float*)S0.r + v0, vb, &full[w][0]);
      bulk_g2s(stages + B32_M + 3 * B32_V, (const float*)S0.dx + v0, vb, &full[w][0]);
    }
    last_k[0] = 0;
    if (begin + w + WARPS < end) pf = load_btile(tiles, begin + w + WARPS);
  }
  for (int tile = begin + w; tile < end; tile += WARPS, ++k) {
    const int s = k & 1;
    const int nxt = tile + WARPS;
    BJob JN;
    if (nxt < end) {
      JN = make_bjob(pf, sys, nxt, &J);
      if (nxt + WARPS < end) pf = load_btile(tiles, nxt + WARPS);
      if (dry) JN.kind = 0;
      if (lane == 0) issue_bjob(JN, stages + (s ^ 1) * B32_STAGE, &full[w][s ^ 1]);
      last_k[s ^ 1] = k + 1;
    }
    if (!dry) {
      const bool ok = mbar_wait(&full[w][s], (k >> 1) & 1);
      if (__any_sync(0xffffffffu, !ok)) {
        dry = true;
        if (lane == 0) atomicExch(flags + 1, 1);
      }
    }
    const SysDesc& S = *J.S;
    SysScalars* sc = S.sc;
    const int state = J.R.state;
    // two-level: this kernel writes z_b; the coarse kernels finish z and the scalars
    const bool defer = S.precond == SSO_TWO_LEVEL && state != ST_FOLD;
    if (state != ST_DONE) {
      const int nn = J.nn;
      const size_t v0 = 6 * (size_t)J.node0;
      DF d1 = {0.f, 0.f}, d2 = {0.f, 0.f};  // r^T z, r^T r terms of the thread's node
      if (state == ST_FOLD) {
        if (!dry) {
          double* x = S.x + v0;
          float* dx = (float*)S.dx + v0;
          for (int i = lane; i < 6 * nn; i += 32) {
            x[i] = fma(J.R.scale, (double)dx[i], x[i]);
            dx[i] = 0.f;
          }
        }
      } else if (J.work && !dry) {
        float* st = stages + s * B32_STAGE;
        float* Vp = st + B32_M;
        float* Vq = Vp + B32_V;
        float* Vr = Vq + B32_V;
        float* Vd = Vr + B32_V;
        if (lane < nn) {
          float rv[6];
          if (state == ST_PCG) {
            const float alpha = (float)J.R.alpha;
            float pv[6], qv[6], dv[6];
            ld6rw(Vp + 6 * lane, pv);
            ld6rw(Vq + 6 * lane, qv);
            ld6rw(Vr + 6 * lane, rv);
            ld6rw(Vd + 6 * lane, dv);
#pragma unroll
            for (int c = 0; c < 6; ++c) {
              dv[c] = fmaf(alpha, pv[c], dv[c]);
              rv[c] = fmaf(-alpha, qv[c], rv[c]);
            }
            st6(Vd + 6 * lane, dv);
          } else {
            const double inv_norm = 1.0 / ::sqrt(J.R.rr64);
            double gv[6];
            ld6rw(S.r64 + v0 + 6 * lane, gv);
#pragma unroll
            for (int c = 0; c < 6; ++c) rv[c] = (float)(gv[c] * inv_norm);
          }
          st6(Vr + 6 * lane, rv);
          float zv[6];
          if (J.block) {
            float m[M32_PACK];
            const float4* mp = reinterpret_cast<const float4*>(st + lane * M32_PACK);
#pragma unroll
            for (int c = 0; c < M32_PACK / 4; ++c) {
              const float4 v = mp[c];
              m[4 * c] = v.x; m[4 * c + 1] = v.y; m[4 * c + 2] = v.z; m[4 * c + 3] = v.w;
            }
#pragma unroll
            for (int a = 0; a < 6; ++a) {
              float acc = 0.f;
#pragma unroll
              for (int c = 0; c < 6; ++c) acc = fmaf(m[sym6(a, c)], rv[c], acc);
              zv[a] = acc;
            }
          } else {
            float m[6];
            ld6rw(st + 6 * lane, m);
#pragma unroll
            for (int a = 0; a < 6; ++a) zv[a] = m[a] * rv[a];
          }
          st6(Vq + 6 * lane, zv);  // q is consumed: its slot now holds z
          d1 = df_prod(rv[0], zv[0]);
          d2 = df_prod(rv[0], rv[0]);
#pragma unroll
          for (int a = 1; a < 6; ++a) {
            d1 = df_add(d1, df_prod(rv[a], zv[a]));
            d2 = df_add(d2, df_prod(rv[a], rv[a]));
          }
        }
        __syncwarp();
        store_run((float*)S.r + v0, Vr, 3 * nn, lane);
        store_run((float*)(defer ? S.zb : S.z) + v0, Vq, 3 * nn, lane);
        if (state == ST_PCG) store_run((float*)S.dx + v0, Vd, 3 * nn, lane);
      }
      // the stage is free for the copies of the tile after next
      __syncwarp();
      const double v1 = df_double(df_warp_sum(d1));
      const double v2 = df_double(df_warp_sum(d2));
      const int lt = tile - S.tile0;
      if (lane == 0) {
        double* dst = S.part_b + 2 * (size_t)lt;
        dst[0] = v1;
        dst[1] = v2;
      }
      // count the warp's tiles per chunk, flushing when the chunk or the run ends
      if (lt / CHUNK != pend_c) {
        if (pend_n) b_count(S, sc, state, pend_c, pend_n, lane, n_active, true, defer);
        pend_c = lt / CHUNK;
        pend_n = 0;
      }
      ++pend_n;
      if (!(nxt < end && JN.sid == J.sid)) {
        b_count(S, sc, state, pend_c, pend_n, lane, n_active, true, defer);
        pend_c = -1;
        pend_n = 0;
      }
    }
    if (nxt < end) J = JN;
  }
  // copies still in flight land before the shared memory is released
  if (dry && lane == 0)
    for (int st = 0; st < 2; ++st)
      if (last_k[st] >= 0) mbar_wait(&full[w][st], (last_k[st] >> 1) & 1);
}

// ---------------------------------------------------------------------------
// Coarse correction of the two-level preconditioner, after kernel B (which
// wrote z_b = M_b^-1 r and left r^T z_b, r^T r):
//   restriction   w = P^T r            one warp per (system, aggregate)
//   coarse solve  y = A_c^-1 w          one CTA per system; r^T z = r^T z_b + w^T y,
//                                       then the scalar update of kernel B
//   prolongation  z = z_b + P y         one warp per tile, one thread per node
// P's block at node i: u = t + theta x r_i, rotation theta (r_i: the node's
// offset from its aggregate's centroid), zero on fixed DOFs.  FP32 vectors,
// fixed-order warp trees, w^T y in FP64.
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(256) coarse_restrict_kernel(const AggRef* __restrict__ aggs,
                                                              const int* __restrict__ n_aggs_ptr,
                                                              const SysDesc* __restrict__ sys) {
  pdl_trigger();
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const int n_aggs = *n_aggs_ptr, stride = (int)((gridDim.x * blockDim.x) >> 5);
  for (int k = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); k < n_aggs; k += stride) {
    const AggRef a = aggs[k];
    const SysDesc& S = sys[a.sys];
    if (S.precond != SSO_TWO_LEVEL || *(volatile const int*)&S.sc->coarse_pending != 1) continue;
    const int b = S.agg_ptr[a.agg], e = S.agg_ptr[a.agg + 1];
    const float* r = (const float*)S.r;
    const float4* rf = reinterpret_cast<const float4*>(S.node_rf);
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    constexpr int U = 4;  // members per lane whose loads are in flight together
    for (int q0 = b + lane; q0 < e; q0 += 32 * U) {
      int idx[U];
#pragma unroll
      for (int u = 0; u < U; ++u) idx[u] = q0 + 32 * u < e ? S.agg_nodes[q0 + 32 * u] : -1;
      float4 o[U];
      float v[U][6];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (idx[u] >= 0) {
          o[u] = rf[idx[u]];
          ld6rw(r + 6 * (size_t)idx[u], v[u]);
        }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (idx[u] >= 0) {
          // B_i^T v: translations v_u; rotations o x v_u + v_theta
          acc[0] += v[u][0];
          acc[1] += v[u][1];
          acc[2] += v[u][2];
          acc[3] += fmaf(o[u].y, v[u][2], fmaf(-o[u].z, v[u][1], v[u][3]));
          acc[4] += fmaf(o[u].z, v[u][0], fmaf(-o[u].x, v[u][2], v[u][4]));
          acc[5] += fmaf(o[u].x, v[u][1], fmaf(-o[u].y, v[u][0], v[u][5]));
        }
    }
#pragma unroll
    for (int d = 0; d < 6; ++d) acc[d] = warp_sum_f(acc[d]);
    if (lane == 0)
#pragma unroll
      for (int d = 0; d < 6; ++d) S.w[6 * a.agg + d] = acc[d];
  }
}

// Work item (system, row block): COARSE_ROWS_PER_BLOCK rows of y = A_c^-1 w
// (two rows per warp, the column loads of both in flight together) and that
// block's w^T y; the CTA that completes the system's row blocks sums the
// partials in block order and updates the scalars.  The item count is read
// from the device (a server's list changes between launches of one graph);
// each CTA takes items blockIdx.x, blockIdx.x + gridDim.x, ...
__global__ void __launch_bounds__(256) coarse_solve_kernel(const int* __restrict__ csys,
                                                           const int* __restrict__ n_csys_ptr,
                                                           const SysDesc* __restrict__ sys,
                                                           int* __restrict__ flags) {
  __shared__ float ws[COARSE_MAX_N];
  __shared__ double red[8];
  __shared__ int s_last;
  pdl_trigger();
  pdl_wait();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_items = *n_csys_ptr * COARSE_ROW_BLOCKS;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int si = item / COARSE_ROW_BLOCKS, rb = item - si * COARSE_ROW_BLOCKS;
    const SysDesc& S = sys[csys[si]];
    SysScalars* sc = S.sc;
    if (S.precond != SSO_TWO_LEVEL || *(volatile const int*)&sc->coarse_pending != 1) continue;
    const int nc = 6 * S.n_agg;
    const int row0 = rb * COARSE_ROWS_PER_BLOCK;
    if (row0 >= nc) continue;
    const int n_blocks = (nc + COARSE_ROWS_PER_BLOCK - 1) / COARSE_ROWS_PER_BLOCK;
    __syncthreads();  // ws, red and s_last of the CTA's previous item are consumed
    for (int k = tid; k < nc; k += blockDim.x) ws[k] = S.w[k];
    __syncthreads();
    constexpr int CPL = (COARSE_MAX_N + 31) / 32;  // columns per lane
    const int ra = row0 + 2 * warp, rbb = ra + 1;
    float xa[CPL], xb[CPL];
#pragma unroll
    for (int u = 0; u < CPL; ++u) {
      const int c = lane + 32 * u;
      xa[u] = (ra < nc && c < nc) ? S.Aci[(size_t)ra * nc + c] : 0.f;
      xb[u] = (rbb < nc && c < nc) ? S.Aci[(size_t)rbb * nc + c] : 0.f;
    }
    float aa = 0.f, ab = 0.f;
#pragma unroll
    for (int u = 0; u < CPL; ++u) {
      const int c = lane + 32 * u;
      const float wc = c < nc ? ws[c] : 0.f;
      aa = fmaf(xa[u], wc, aa);
      ab = fmaf(xb[u], wc, ab);
    }
    aa = warp_sum_f(aa);
    ab = warp_sum_f(ab);
    double dot = 0.0;
    if (lane == 0) {
      if (ra < nc) {
        S.y[ra] = aa;
        dot += (double)aa * (double)ws[ra];
      }
      if (rbb < nc) {
        S.y[rbb] = ab;
        dot += (double)ab * (double)ws[rbb];
      }
      red[warp] = dot;
    }
    __syncthreads();
    if (tid == 0) {
      double part = 0.0;
#pragma unroll
      for (int k = 0; k < 8; ++k) part += red[k];
      S.cdot[rb] = part;
      __threadfence();
      const unsigned prev = atomicAdd(&sc->coarse_cnt, 1u);
      s_last = prev + 1u == (unsigned)n_blocks;
    }
    __syncthreads();
    if (s_last && tid == 0) {
      __threadfence();
      double wy = 0.0;
      for (int k = 0; k < n_blocks; ++k) wy += __ldcg(S.cdot + k);
      sc->coarse_cnt = 0u;
      sc->coarse_pending = 0;
      finish_b(sc, sc->state, sc->rz_b + wy, sc->rr_b, flags, true);
    }
  }
}

__global__ void __launch_bounds__(NT) coarse_prolong_kernel(const TileDesc* __restrict__ tiles,
                                                            const int* __restrict__ n_tiles_ptr,
                                                            const SysDesc* __restrict__ sys) {
  pdl_trigger();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int begin, end;
  tile_range(*n_tiles_ptr, begin, end);
  pdl_wait();
  for (int tile = begin + w; tile < end; tile += WARPS) {
    const TileDesc& td = tiles[tile];
    const SysDesc& S = sys[td.sys];
    // after the coarse solve a system in CG needs z (a sweep that just began
    // or one more iteration); FOLD and DONE do not
    if (S.precond != SSO_TWO_LEVEL || *(volatile const int*)&S.sc->state != ST_PCG) continue;
    if (lane >= td.nn) continue;
    const int i = td.node0 + lane;
    const int g = S.agg_of[i];
    const float4 o = reinterpret_cast<const float4*>(S.node_rf)[i];
    const float* y = S.y + 6 * g;
    const float t0 = y[0], t1 = y[1], t2 = y[2], w0 = y[3], w1 = y[4], w2 = y[5];
    // u = t + theta x o, rotation theta
    float c[6] = {fmaf(w1, o.z, fmaf(-w2, o.y, t0)), fmaf(w2, o.x, fmaf(-w0, o.z, t1)),
                  fmaf(w0, o.y, fmaf(-w1, o.x, t2)), w0, w1, w2};
    const uint8_t* fx = S.fixed + 6 * (size_t)i;
    float zb[6];
    ld6rw((const float*)S.zb + 6 * (size_t)i, zb);
#pragma unroll
    for (int d = 0; d < 6; ++d) zb[d] += fx[d] ? 0.f : c[d];
    st6((float*)S.z + 6 * (size_t)i, zb);
  }
}

// ---------------------------------------------------------------------------
// Kernel A for the FP32 CG, warp-specialised.  Everything a tile reads is
// contiguous in memory -- its K rows are one slab of the BSR value array, its
// column indices and its row_ptr entries one run each, and the z / p entries
// its columns touch lie in one node range (the tile's halo) -- and their
// extents are fixed by the mesh (TileDesc, built on the host).  A producer
// warp streams these five pieces of each tile into a two-stage shared-memory
// ring with bulk copies (cp.async.bulk, the 1-D form of the TMA engine) and
// passes the system's scalars along; six consumer warps compute the tile from
// shared memory with no global loads.  full[s] / empty[s] mbarriers hand each
// stage over; every wait is bounded.  Tiles that do not fit (scattered
// numbering) and the FP64 residual passes read global memory instead; a tile
// whose halo alone does not fit (long grid rows) stages everything but the
// halo and gathers z and p from global memory.
constexpr int ST_SLAB_K = STAGE_SLAB_K;
constexpr int ST_SLAB_C = STAGE_SLAB_C;
constexpr int ST_SLAB_V = STAGE_SLAB_V;
constexpr int ST_SLAB_R = STAGE_SLAB_R;
constexpr int ST_OFF_C = ST_SLAB_K;
constexpr int ST_OFF_Z = ST_OFF_C + ST_SLAB_C;
constexpr int ST_OFF_P = ST_OFF_Z + ST_SLAB_V;
constexpr int ST_OFF_R = ST_OFF_P + ST_SLAB_V;
constexpr int ST_STAGE = ST_OFF_R + ST_SLAB_R;
constexpr int ST_STAGES = 2;
constexpr int ST_SMEM = ST_STAGES * ST_STAGE;
constexpr int ST_THREADS = NT + 32;  // six consumer warps + one producer warp
// barrier among the 192 consumer threads only (the producer warp runs ahead)
__device__ __forceinline__ void consumer_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}
__device__ __forceinline__ double consumer_block_sum(double v, double* red) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  consumer_sync();
  double s = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < WARPS; ++w) s += red[w];
  }
  consumer_sync();
  return s;
}
__device__ __forceinline__ void ld6s(const float* p, float v[6]) {
  const float2* q = reinterpret_cast<const float2*>(p);
  const float2 a = q[0], b = q[1], c = q[2];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
}

// What the producer hands the consumers with each stage.
struct StageInfo {
  int state, mode, first, parity;  // mode 1: the tile's data is in the stage
  float beta;
  int sys, node0, nn, j0, cb, rb;
  int run_end;  // the next tile of the CTA's range belongs to another system (or there is none)
  // where the consumers write (read once per system by the producer, so that
  // no consumer waits on its system's descriptor)
  float* pnew;   // p of this iteration
  float* q;
  double* part;  // this tile's kernel-A partials
  // halo runs in the stage: column c sits at slot c + shift[k] (nodes) for the
  // last run k whose first node is <= c (first nodes of unused runs: INT_MAX)
  int v1, v2, sh0, sh1, sh2;
};

__global__ void __launch_bounds__(ST_THREADS, 2) pcg_a_staged_kernel(
    const TileDesc* __restrict__ tiles, const int* __restrict__ n_tiles_ptr,
    const SysDesc* __restrict__ sys, int* __restrict__ flags, int grid_mult) {
  extern __shared__ __align__(128) unsigned char ring[];
  __shared__ __align__(8) unsigned long long full[ST_STAGES], empty[ST_STAGES];
  __shared__ StageInfo info[ST_STAGES];
  __shared__ double red[WARPS];
  __shared__ int s_last, s_abort;
  pdl_trigger();
  int* n_active = flags;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  int begin, end;
  tile_range(*n_tiles_ptr, begin, end, grid_mult);
  if (t == 0) {
    for (int s = 0; s < ST_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], WARPS);
    }
    fence_barrier_init();
    s_abort = 0;
  }
  __syncthreads();
  if (w != WARPS) pdl_wait();

  if (w == WARPS) {
    // ---------------- producer warp (lane 0) ----------------
    if (lane != 0) return;
    // K rows, columns and row_ptr do not change during a solve, so the first
    // stages' copies of them are issued before waiting for the previous
    // kernel and overlap its tail; the halo copies (vectors that kernel
    // writes) follow the wait.  All of a stage's bytes are announced up
    // front, but its one arrival comes only after its StageInfo is written,
    // so no consumer can see the phase complete before that.
    int pre = 0;
    for (; pre < ST_STAGES && begin + pre < end; ++pre) {
      const TileDesc t = tiles[begin + pre];
      if (!t.stage_k) break;
      const SysDesc* S = sys + t.sys;
      uint32_t vb = 0u;
      if (t.stage)
        for (int r = 0; r < HALO_RUNS; ++r) vb += (uint32_t)t.nv[r] * 24u;
      const uint32_t kb = (uint32_t)t.nblk * 144u, cb = (uint32_t)t.ncb * 4u;
      const uint32_t rb = (uint32_t)t.nrb * 4u;
      unsigned char* st = ring + pre * ST_STAGE;
      fence_proxy_async();
      mbar_expect_tx(&full[pre], kb + cb + 2 * vb + rb);
      bulk_g2s(st, S->K32 + (size_t)t.j0 * 36, kb, &full[pre]);
      // a tile staged whole reads its columns as halo slots
      bulk_g2s(st + ST_OFF_C, (t.stage ? S->hslot : S->col) + t.cb, cb, &full[pre]);
      bulk_g2s(st + ST_OFF_R, S->row_ptr + t.rb, rb, &full[pre]);
    }
    pdl_wait();
    int cur = -1, issued = 0;
    RunState R;
    R.state = ST_DONE;
    // the system's arrays, read once per run of tiles of one system
    struct {
      const float *z, *K32;
      float *p0, *p1, *q;
      const int *col, *hslot, *row_ptr;
      double* part_a;
      int tile0;
    } P = {};
    // each tile's descriptor is loaded one tile ahead, so that its latency
    // overlaps the wait for a free stage
    TileDesc td_next;
    if (begin < end) td_next = tiles[begin];
    for (int tile = begin, k = 0; tile < end; ++tile, ++k) {
      const int s = k % ST_STAGES, use = k / ST_STAGES;
      const TileDesc td = td_next;
      if (tile + 1 < end) td_next = tiles[tile + 1];
      if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1)) {
        atomicExch(flags + 1, 1);
        break;
      }
      const SysDesc* S = sys + td.sys;
      if (td.sys != cur) {
        cur = td.sys;
        R = read_state(S->sc);
        P.z = (const float*)S->z;
        P.K32 = S->K32;
        P.p0 = (float*)S->p0;
        P.p1 = (float*)S->p1;
        P.q = (float*)S->q;
        P.col = S->col;
        P.hslot = S->hslot;
        P.row_ptr = S->row_ptr;
        P.part_a = S->part_a;
        P.tile0 = S->tile0;
      }
      StageInfo inf;
      inf.state = R.state;
      inf.mode = 0;
      inf.first = R.first;
      inf.parity = R.parity;
      inf.beta = R.first ? 0.f : (float)R.beta;
      inf.sys = td.sys;
      inf.node0 = td.node0;
      inf.nn = td.nn;
      inf.j0 = td.j0;
      inf.cb = td.cb;
      inf.rb = td.rb;
      inf.run_end = tile + 1 >= end || td_next.sys != td.sys;
      inf.pnew = R.parity ? P.p0 : P.p1;
      inf.q = P.q;
      inf.part = P.part_a + 2 * (size_t)(tile - P.tile0) * WARPS;
      inf.v1 = td.nv[1] ? td.vlo[1] : INT_MAX;
      inf.v2 = td.nv[2] ? td.vlo[2] : INT_MAX;
      inf.sh0 = -td.vlo[0];
      inf.sh1 = td.nv[0] - td.vlo[1];
      inf.sh2 = td.nv[0] + td.nv[1] - td.vlo[2];
      ++issued;
      if (k < pre) {
        // K, columns and row_ptr already on their way; the halo (copied
        // whatever the state, since the stage expects its bytes)
        inf.mode = R.state == ST_PCG ? (td.stage ? 1 : 2) : 0;
        info[s] = inf;
        if (td.stage) {
          const float* z = P.z;
          const float* pold = R.state == ST_PCG && !R.first ? (R.parity ? P.p1 : P.p0) : z;
          unsigned char* st = ring + s * ST_STAGE;
          uint32_t off = 0u;
          for (int r = 0; r < HALO_RUNS; ++r) {
            if (!td.nv[r]) continue;
            const uint32_t b = (uint32_t)td.nv[r] * 24u;
            bulk_g2s(st + ST_OFF_Z + off, z + (size_t)td.vlo[r] * 6, b, &full[s]);
            bulk_g2s(st + ST_OFF_P + off, pold + (size_t)td.vlo[r] * 6, b, &full[s]);
            off += b;
          }
        }
        mbar_arrive(&full[s]);  // after info[s]: the phase can complete now
      } else if (R.state == ST_PCG && td.stage_k) {
        // mode 1: K rows, columns, row_ptr and both vector halos; mode 2: the
        // halo does not fit, the consumers gather z and p from global memory
        inf.mode = td.stage ? 1 : 2;
        info[s] = inf;
        const float* z = P.z;
        const float* pold = R.first ? z : (R.parity ? P.p1 : P.p0);
        const uint32_t kb = (uint32_t)td.nblk * 144u, cb = (uint32_t)td.ncb * 4u;
        const uint32_t rb = (uint32_t)td.nrb * 4u;
        uint32_t vb = 0u;
        if (td.stage)
          for (int k = 0; k < HALO_RUNS; ++k) vb += (uint32_t)td.nv[k] * 24u;
        unsigned char* st = ring + s * ST_STAGE;
        fence_proxy_async();
        mbar_arrive_tx(&full[s], kb + cb + 2 * vb + rb);
        bulk_g2s(st, P.K32 + (size_t)td.j0 * 36, kb, &full[s]);
        bulk_g2s(st + ST_OFF_C, (td.stage ? P.hslot : P.col) + td.cb, cb, &full[s]);
        if (td.stage) {
          uint32_t off = 0u;  // bytes into each vector slab
          for (int k = 0; k < HALO_RUNS; ++k) {
            if (!td.nv[k]) continue;
            const uint32_t b = (uint32_t)td.nv[k] * 24u;
            bulk_g2s(st + ST_OFF_Z + off, z + (size_t)td.vlo[k] * 6, b, &full[s]);
            bulk_g2s(st + ST_OFF_P + off, pold + (size_t)td.vlo[k] * 6, b, &full[s]);
            off += b;
          }
        }
        bulk_g2s(st + ST_OFF_R, P.row_ptr + td.rb, rb, &full[s]);
      } else {
        info[s] = inf;
        mbar_arrive(&full[s]);
      }
    }
    // let the copies in flight land before the CTA's shared memory is released
    for (int k = issued - ST_STAGES; k < issued; ++k)
      if (k >= 0) mbar_wait(&full[k % ST_STAGES], (k / ST_STAGES) & 1);
    return;
  }

  // ---------------- consumer warps ----------------
  // A warp whose wait gives up sets the error flag and runs the rest of its
  // tiles dry (no waits, no work) so that every consumer warp still reaches
  // the same named barriers; the host then fails the solve.
  const int ln = w * NODES_PER_WARP + lane / 6, rr = lane % 6;
  int run = 0;
  bool dry = false;
  for (int tile = begin, k = 0; tile < end; ++tile, ++k) {
    const int s = k % ST_STAGES, use = k / ST_STAGES;
    if (!dry && !mbar_wait(&full[s], use & 1)) {
      dry = true;
      s_abort = 1;
      atomicExch(flags + 1, 1);
    }
    // a dry warp takes nothing from the stage (it may never have been
    // written): the system and its state come from global memory, as the
    // producer read them, so the warp keeps the others' barrier pattern
    StageInfo inf = info[s];
    if (dry) {
      inf.sys = tiles[tile].sys;
      inf.state = read_state(sys[inf.sys].sc).state;
      inf.run_end = tile + 1 >= end || tiles[tile + 1].sys != inf.sys;
    }

    const SysDesc& S = sys[inf.sys];
    SysScalars* sc = S.sc;
    const int real_state = inf.state;
    const bool skip = real_state == ST_DONE || real_state == ST_FOLD;
    const int state = dry || skip ? ST_DONE : real_state;
    const int node = inf.node0 + ln;
    const bool act = lane < 6 * NODES_PER_WARP && ln < inf.nn;
    const int i = 6 * node + rr;
    double part = 0.0, part_b = 0.0;
    DF dpart = {0.f, 0.f};  // CG state: the warp's p^T q terms
    if (state == ST_PCG) {
      float* pnew = inf.pnew;
      const float beta = inf.beta;
      if (act) {
        float acc = 0.f, zi = 0.f, pi_old = 0.f;
        if (inf.mode == 1) {
          const unsigned char* st = ring + s * ST_STAGE;
          const int* Rs = reinterpret_cast<const int*>(st + ST_OFF_R) - inf.rb;
          const int j0 = Rs[node], j1 = Rs[node + 1];
          const float* Ks = reinterpret_cast<const float*>(st) + (size_t)(j0 - inf.j0) * 36 + rr * 6;
          // each block's column slot in the staged halo comes precomputed
          const int* Hs = reinterpret_cast<const int*>(st + ST_OFF_C) - inf.cb;
          const float* Zs = reinterpret_cast<const float*>(st + ST_OFF_Z);
          const float* Ps = reinterpret_cast<const float*>(st + ST_OFF_P);
          const int v1 = inf.v1, v2 = inf.v2, sh0 = inf.sh0, sh1 = inf.sh1, sh2 = inf.sh2;
          for (int j = j0; j < j1; ++j) {
            const int o = 6 * Hs[j];
            float kv[6], zv[6], pv[6];
            ld6s(Ks, kv);
            ld6s(Zs + o, zv);
            ld6s(Ps + o, pv);
            Ks += 36;
#pragma unroll
            for (int q = 0; q < 6; ++q) acc = fmaf(kv[q], fmaf(beta, pv[q], zv[q]), acc);
          }
          const int oi = 6 * (node + (node >= v2 ? sh2 : (node >= v1 ? sh1 : sh0))) + rr;
          zi = Zs[oi];
          pi_old = Ps[oi];
        } else if (inf.mode == 2) {
          // K rows, columns and row_ptr from the stage; z and p gathered from
          // global memory, three columns in flight at a time
          const unsigned char* st = ring + s * ST_STAGE;
          const int* Rs = reinterpret_cast<const int*>(st + ST_OFF_R) - inf.rb;
          const int j0 = Rs[node], j1 = Rs[node + 1];
          const float* Kt = reinterpret_cast<const float*>(st) - (size_t)inf.j0 * 36 + rr * 6;
          const int* Cs = reinterpret_cast<const int*>(st + ST_OFF_C) - inf.cb;
          const float* z = (const float*)S.z;
          const float* pold = inf.first ? z : (const float*)(inf.parity ? S.p1 : S.p0);
          constexpr int CH = 3;
          for (int jb = j0; jb < j1; jb += CH) {
            int cc[CH];
#pragma unroll
            for (int u = 0; u < CH; ++u) cc[u] = Cs[min(jb + u, j1 - 1)];
            float kv[CH][6], zv[CH][6], pv[CH][6];
#pragma unroll
            for (int u = 0; u < CH; ++u) {
              ld6s(Kt + (size_t)min(jb + u, j1 - 1) * 36, kv[u]);
              load6(z + (size_t)cc[u] * 6, zv[u]);
              load6(pold + (size_t)cc[u] * 6, pv[u]);
            }
#pragma unroll
            for (int u = 0; u < CH; ++u)
              if (jb + u < j1) {
#pragma unroll
                for (int q = 0; q < 6; ++q)
                  acc = fmaf(kv[u][q], fmaf(beta, pv[u][q], zv[u][q]), acc);
              }
          }
          zi = z[i];
          pi_old = pold[i];
        } else {
          const float* z = (const float*)S.z;
          const float* pold = inf.first ? z : (const float*)(inf.parity ? S.p1 : S.p0);
          const int j0 = __ldg(S.row_ptr + node), j1 = __ldg(S.row_ptr + node + 1);
          acc = row_dot<float, 3>(S.K32, S.col, j0, j1, rr, z, pold, beta);
          zi = z[i];
          pi_old = pold[i];
        }
        const float pi = fmaf(beta, pi_old, zi);
        pnew[i] = pi;
        inf.q[i] = acc;
        dpart = df_prod(pi, acc);
      }
    } else if (state != ST_DONE) {  // ST_INIT or ST_RESID: r64 = b - K64 x in FP64
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
    // stage s is consumed: hand it back to the producer
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    if (skip) continue;
    if (real_state == ST_PCG) {
      part = df_double(df_warp_sum(dpart));
    } else {
      part = warp_sum(part);
      part_b = warp_sum(part_b);
    }
    if (lane == 0) {
      // a dry warp may hold a stage descriptor that was never written
      double* dst = dry ? S.part_a + 2 * ((size_t)(tile - S.tile0) * WARPS + w)
                        : inf.part + 2 * w;
      dst[0] = part;
      dst[1] = part_b;
    }
    ++run;
    if (!inf.run_end) continue;
    const int r1 = tile - S.tile0 + 1;
    consumer_sync();
    const bool count = !s_abort;
    consumer_sync();
    a_count_run(S, sc, real_state, r1 - run, r1, t, n_active, &s_last, count,
                [] { consumer_sync(); }, [&](double v) { return consumer_block_sum(v, red); });
    run = 0;
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

static cudaError_t staged_attributes() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(pcg_a_staged_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, ST_SMEM);
  if (e == cudaSuccess) done = true;
  return e;
}

static cudaError_t b32_attributes() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(pcg_b32_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, B32_SMEM);
  if (e == cudaSuccess) done = true;
  return e;
}

// A CG kernel launched with programmatic stream serialisation (see pdl_wait).
template <typename... Args>
static cudaError_t launch_cg_kernel(void (*kernel)(Args...), int grid, int threads, int smem,
                                    cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

cudaError_t launch_pcg_a(bool fp64, const TileDesc* tiles, const int* n_tiles,
                         const SysDesc* sys, int* flags, int grid, int grid_mult,
                         cudaStream_t s) {
  if (fp64)
    return launch_cg_kernel<const TileDesc*, const int*, const SysDesc*, int*, int>(
        pcg_a_kernel<double>, grid, NT, 0, s, tiles, n_tiles, sys, flags, grid_mult);
  cudaError_t e = staged_attributes();
  if (e != cudaSuccess) return e;
  return launch_cg_kernel<const TileDesc*, const int*, const SysDesc*, int*, int>(
      pcg_a_staged_kernel, grid, ST_THREADS, ST_SMEM, s, tiles, n_tiles, sys, flags, grid_mult);
}

cudaError_t launch_pcg_b(bool fp64, const TileDesc* tiles, const int* n_tiles,
                         const SysDesc* sys, int* flags, int grid, cudaStream_t s) {
  if (fp64)
    return launch_cg_kernel<const TileDesc*, const int*, const SysDesc*, int*>(
        pcg_b_kernel<double>, grid, NT, 0, s, tiles, n_tiles, sys, flags);
  cudaError_t e = b32_attributes();
  if (e != cudaSuccess) return e;
  return launch_cg_kernel<const TileDesc*, const int*, const SysDesc*, int*>(
      pcg_b32_kernel, grid, NT, B32_SMEM, s, tiles, n_tiles, sys, flags);
}

template <typename... Args>
static cudaError_t launch_pdl(void (*kernel)(Args...), int grid, int threads, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

cudaError_t launch_coarse_restrict(const AggRef* aggs, const int* n_aggs, int grid,
                                   const SysDesc* sys, cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  return launch_pdl(coarse_restrict_kernel, grid, 256, s, aggs, n_aggs, sys);
}

cudaError_t launch_coarse_solve(const int* csys, const int* n_csys, int grid, const SysDesc* sys,
                                int* flags, cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  return launch_pdl(coarse_solve_kernel, grid, 256, s, csys, n_csys, sys, flags);
}

cudaError_t launch_coarse_prolong(const TileDesc* tiles, const int* n_tiles, const SysDesc* sys,
                                  int grid, cudaStream_t s) {
  return launch_pdl(coarse_prolong_kernel, grid, NT, s, tiles, n_tiles, sys);
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
    staged_attributes();
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_a, pcg_a_staged_kernel, ST_THREADS,
                                                  ST_SMEM);
    b32_attributes();
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, pcg_b32_kernel, NT, B32_SMEM);
  }
  if (sms < 1) sms = 1;
  *grid_a = sms * (per_sm_a < 1 ? 1 : per_sm_a);
  *grid_b = sms * (per_sm_b < 1 ? 1 : per_sm_b);
}

}  // namespace sso
