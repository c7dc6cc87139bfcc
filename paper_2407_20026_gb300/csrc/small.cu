// Double-float CG in one CTA per system (precision SSO_F32X2): the whole
// preconditioned CG of K u = b (Eq. 1 under the supports of Eqs. 2-3) in a
// single launch, for small systems whose solve time is otherwise launch and
// host-synchronisation latency (the 600-DOF grid-shell: ~100 iterations).
//
// Arithmetic.  GB300 issues an FP64 instruction at about 1/64 of the FP32
// rate, and one SM does all of a system's work here, so every vector and
// every product is kept as an unevaluated sum hi + lo of two floats (about 48
// significant bits) and computed on the FP32 pipes with error-free
// transformations: K = K32 + Klo with Klo = K64 - K32 rounded to FP32 (exact
// to ~2^-48 relative), row products accumulated as compensated dot products
// (a running two-sum plus an FP32 error term, the "Dot2" scheme of Ogita,
// Rump and Oishi, 2005, with the cross terms of the low parts added), vector
// updates by double-float multiply and add.  The scalars alpha, beta and the
// convergence tests are double-float too (quotients refined once by their
// remainder): every thread forms them, and an FP64 instruction per thread
// would cost more than the matrix product of the iteration.  The
// preconditioner (Jacobi or block-Jacobi, FP32 inverse blocks) is applied to
// the double-float residual with double-float products; with the two-level
// preconditioner the coarse correction P A_c^-1 P^T r (rigid-body modes of the
// node aggregates, FP32 inverse of the coarse matrix) is added in the same
// CTA: each row's share of P^T r, the sums per aggregate in node order, the
// coarse product, the prolongation -- three barriers more per iteration.
//
// Recurrences: the Chronopoulos-Gear form of preconditioned CG (1989), which
// carries s = K p by s = w + beta s with w = K u, u = M^-1 r, so that one
// matrix product and ONE reduction point (r^T u, w^T u and r^T r together)
// make an iteration; in one CTA a reduction costs two barriers and a warp
// tree per warp, as much as a third of the iteration.
//
// Layout of the work: warps own groups of 5 nodes, one lane per scalar row
// (30 lanes, two idle), as in the batched CG kernels; every reduction is a
// fixed-shape warp tree, then the partials of the warps that own rows summed
// in warp order by warp 0, so each system's iterates are the same alone or in
// a batch.  The six vectors (x, r, u, w, p, s as float2 hi, lo) live in shared
// memory for systems of up to 512 nodes, else in the system's scratch
// vectors; the matrix is read through the read-only cache, so a small K stays
// in the SM's L1.
//
// Convergence: when the recursive residual satisfies ||r|| <= rtol ||b||, the
// residual b - K64 x is recomputed in FP64 (the refinement residual: FP64 only
// there, a few microseconds per sweep on one SM); above rtol the CG restarts
// from it (a "sweep", at most max_sweeps), below it the system is done.
// Exits: converged (SSO_OK), p^T K p <= 0 or non-finite (SSO_ERR_SINGULAR),
// max_iter or max_sweeps reached (SSO_ERR_NOT_CONVERGED).
#include "sso_internal.cuh"

namespace sso {
namespace {

constexpr int MAX_WARPS = 32;
// a CTA of at most 20 warps (640 threads: 100 nodes at a time), which leaves
// each thread ~100 registers; larger systems loop over their node groups
constexpr int SMALL_MAX_THREADS = 640;
// six double-float vectors of 6 entries per node in shared memory
constexpr int SMALL_BYTES_PER_NODE = 6 * 6 * 8;
constexpr int SMALL_BYTES_PER_NODE_2L = 7 * 6 * 8;  // and the restriction shares
constexpr int SMALL_SMEM_NODES = 512;  // 144 KB; the rest of the SM's 256 KB stays L1 for K

__device__ __forceinline__ DF df_split(double v) {
  const float hi = __double2float_rn(v);
  return {hi, __double2float_rn(v - (double)hi)};
}
// a * b for double-float a, b (the lo * lo term, below 2^-48 |a b|, dropped)
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float hi = __fadd_rn(p, e);
  return {hi, __fsub_rn(e, __fsub_rn(hi, p))};
}
__device__ __forceinline__ DF df_neg(DF a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ DF ld_df(const float2* p) {
  const float2 v = *p;
  return {v.x, v.y};
}
__device__ __forceinline__ void st_df(float2* p, DF v) { *p = make_float2(v.hi, v.lo); }

// Compensated accumulation of products: s carries the running sum, c the
// FP32 sum of every rounding error (two-product and two-sum) and cross term.
struct Acc {
  float s = 0.f, c = 0.f;
};
__device__ __forceinline__ void acc_prod(Acc& A, DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, pe);
  pe = __fmaf_rn(a.lo, b.hi, pe);
  const float t = __fadd_rn(A.s, p);
  const float z = __fsub_rn(t, A.s);
  const float se = __fadd_rn(__fsub_rn(A.s, __fsub_rn(t, z)), __fsub_rn(p, z));
  A.s = t;
  A.c = __fadd_rn(A.c, __fadd_rn(pe, se));
}
__device__ __forceinline__ DF acc_value(const Acc& A) {
  const float hi = __fadd_rn(A.s, A.c);
  return {hi, __fsub_rn(A.c, __fsub_rn(hi, A.s))};
}

// Sum over the CTA of each lane's (a, b, c) in a fixed order; every thread
// gets the three totals.  Warps >= nw hold no rows: the tree over 32 warp
// slots sees zeros there whatever the CTA's size, so a system's sums do not
// depend on the launch's block size.  buf: 3 * MAX_WARPS + 3 DF of shared
// memory, not written again before the next __syncthreads of the caller.
__device__ __forceinline__ void block_sum3(DF a, DF b, DF c, DF* buf, int nw, DF& sa, DF& sb,
                                           DF& sc) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  a = df_warp_sum(a);
  b = df_warp_sum(b);
  c = df_warp_sum(c);
  if (lane == 0 && w < nw) {
    buf[w] = a;
    buf[MAX_WARPS + w] = b;
    buf[2 * MAX_WARPS + w] = c;
  }
  __syncthreads();
  if (w == 0) {
    DF x = lane < nw ? buf[lane] : DF{0.f, 0.f};
    DF y = lane < nw ? buf[MAX_WARPS + lane] : DF{0.f, 0.f};
    DF z = lane < nw ? buf[2 * MAX_WARPS + lane] : DF{0.f, 0.f};
    x = df_warp_sum(x);
    y = df_warp_sum(y);
    z = df_warp_sum(z);
    if (lane == 0) {
      buf[3 * MAX_WARPS] = x;
      buf[3 * MAX_WARPS + 1] = y;
      buf[3 * MAX_WARPS + 2] = z;
    }
  }
  __syncthreads();
  sa = buf[3 * MAX_WARPS];
  sb = buf[3 * MAX_WARPS + 1];
  sc = buf[3 * MAX_WARPS + 2];
}

// a / b in double-float: an FP32 quotient, corrected once by the double-float
// remainder a - q b (about 44 significant bits).  Every thread computes the
// CG scalars this way, on the FP32 pipes.
__device__ __forceinline__ DF df_div(DF a, DF b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const DF r = df_add(a, df_neg(df_mul(DF{q1, 0.f}, b)));
  const float q2 = __fdiv_rn(r.hi, b.hi);
  const float hi = __fadd_rn(q1, q2);
  return {hi, __fsub_rn(q2, __fsub_rn(hi, q1))};
}
// a <= b for normalised double-float values
__device__ __forceinline__ bool df_le(DF a, DF b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo);
}
__device__ __forceinline__ bool df_finite(DF a) { return isfinite(a.hi) && isfinite(a.lo); }

// One CG iteration's reduction point and scalar update (Chronopoulos-Gear):
// the block sums of (gamma_n, delta_n, r^T r) as block_sum3, after which one
// thread (warp 0, lane 0) takes the decisions and forms the new scalars
//   beta = gamma_n / gamma, alpha = gamma_n / (delta_n - beta gamma_n / alpha)
// and every thread reads them after the barrier: the same arithmetic in the
// same order as if every thread formed them, without 20 warps issuing it.
// Returns 0 to go on, 1 when K is found not positive definite or a value is
// not finite, 2 when the recursive residual reached thr.
__device__ __forceinline__ int cg_step(DF a, DF b, DF c, DF* buf, int nw, DF thr, DF& alpha,
                                       DF& beta, DF& gamma) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  a = df_warp_sum(a);
  b = df_warp_sum(b);
  c = df_warp_sum(c);
  if (lane == 0 && w < nw) {
    buf[w] = a;
    buf[MAX_WARPS + w] = b;
    buf[2 * MAX_WARPS + w] = c;
  }
  __syncthreads();
  int* code = reinterpret_cast<int*>(buf + 3 * MAX_WARPS + 3);
  if (w == 0) {
    DF gn = lane < nw ? buf[lane] : DF{0.f, 0.f};
    DF dn = lane < nw ? buf[MAX_WARPS + lane] : DF{0.f, 0.f};
    DF rrn = lane < nw ? buf[2 * MAX_WARPS + lane] : DF{0.f, 0.f};
    gn = df_warp_sum(gn);
    dn = df_warp_sum(dn);
    rrn = df_warp_sum(rrn);
    if (lane == 0) {
      int k = 0;
      DF al = alpha, be = beta, ga = gamma;
      if (!df_finite(rrn) || !df_finite(gn) || !df_finite(dn)) {
        k = 1;
      } else if (df_le(rrn, thr)) {
        k = 2;
      } else {
        const DF bn = df_div(gn, gamma);
        const DF den = df_add(dn, df_neg(df_div(df_mul(bn, gn), alpha)));
        if (!(den.hi > 0.f)) {  // p^T K p <= 0: K is not positive definite
          k = 1;
        } else {
          al = df_div(gn, den);
          be = bn;
          ga = gn;
        }
      }
      buf[3 * MAX_WARPS] = al;
      buf[3 * MAX_WARPS + 1] = be;
      buf[3 * MAX_WARPS + 2] = ga;
      *code = k;
    }
  }
  __syncthreads();
  alpha = buf[3 * MAX_WARPS];
  beta = buf[3 * MAX_WARPS + 1];
  gamma = buf[3 * MAX_WARPS + 2];
  return *code;
}

struct Small {
  const int* row_ptr;
  const int* col;
  const float* KH;
  const float* KL;
  const float* M;
  bool block;
  int n;
};

// (K v)[6 node + r] for a double-float vector v
// Two accumulators, one for the even and one for the odd columns of every
// block: two independent dependency chains per lane (the sum order is fixed
// by the row alone).
__device__ __forceinline__ DF row_product(const Small& G, const float2* v, int node, int r) {
  Acc A0, A1;
  const int j1 = __ldg(G.row_ptr + node + 1);
#pragma unroll 2
  for (int j = __ldg(G.row_ptr + node); j < j1; ++j) {
    const int c0 = 6 * __ldg(G.col + j);
    // the row's 6 entries of both parts as 8-byte loads (24-byte rows)
    const float2* kh = reinterpret_cast<const float2*>(G.KH + (size_t)j * 36 + 6 * r);
    const float2* kl = reinterpret_cast<const float2*>(G.KL + (size_t)j * 36 + 6 * r);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 h = __ldg(kh + c), l = __ldg(kl + c);
      acc_prod(A0, DF{h.x, l.x}, ld_df(v + c0 + 2 * c));
      acc_prod(A1, DF{h.y, l.y}, ld_df(v + c0 + 2 * c + 1));
    }
  }
  return df_add(acc_value(A0), acc_value(A1));
}

// z = M^-1 r for the lane's row; every lane of the warp calls it (shuffles).
// rv: this lane's residual entry; node / r: its row (valid or not).
__device__ __forceinline__ DF apply_precond(const Small& G, DF rv, int node, int r, bool ok) {
  const int lane = threadIdx.x & 31;
  const int base = lane - r;  // first lane of the node
  Acc A;
  if (G.block) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      DF rc;
      rc.hi = __shfl_sync(0xffffffffu, rv.hi, (base + c) & 31);
      rc.lo = __shfl_sync(0xffffffffu, rv.lo, (base + c) & 31);
      const float m = ok ? __ldg(G.M + (size_t)node * M32_PACK + sym6(r, c)) : 0.f;
      acc_prod(A, DF{m, 0.f}, rc);
    }
  } else {
    const float m = ok ? __ldg(G.M + 6 * (size_t)node + r) : 0.f;
    acc_prod(A, DF{m, 0.f}, rv);
  }
  return acc_value(A);
}

// Two-level preconditioner (precond SSO_TWO_LEVEL): u = M_bj^-1 r + P A_c^-1 P^T r
// with P the rigid-body modes of each node aggregate about its centroid (node
// offset o).  Row r of node i contributes to w_a = P^T r (a = agg_of[i]):
//   translations  w[d] += r_i[d]                      (d < 3)
//   rotations     w[3 + d] += (o x r_i,t)[d] + r_i[3 + d]
// The lane's share is returned; every lane of the warp calls it (shuffles).
__device__ __forceinline__ DF restrict_share(const SysDesc& S, DF rv, int node, int r, bool ok) {
  const int lane = threadIdx.x & 31, base = lane - r;
  DF rc[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    rc[c].hi = __shfl_sync(0xffffffffu, rv.hi, (base + c) & 31);
    rc[c].lo = __shfl_sync(0xffffffffu, rv.lo, (base + c) & 31);
  }
  if (!ok) return DF{0.f, 0.f};
  if (r < 3) return rv;
  const float4 o = reinterpret_cast<const float4*>(S.node_rf)[node];
  // (o x v)_x = o.y v_z - o.z v_y, (o x v)_y = o.z v_x - o.x v_z, (o x v)_z = o.x v_y - o.y v_x
  const float oa = r == 3 ? o.y : (r == 4 ? o.z : o.x);
  const float ob = r == 3 ? o.z : (r == 4 ? o.x : o.y);
  const DF va = r == 3 ? rc[2] : (r == 4 ? rc[0] : rc[1]);
  const DF vb = r == 3 ? rc[1] : (r == 4 ? rc[2] : rc[0]);
  return df_add(df_add(df_mul(DF{oa, 0.f}, va), df_neg(df_mul(DF{ob, 0.f}, vb))), rv);
}

// The coarse step between two barriers of the caller: Wc holds each row's
// restriction share (6 n DF).  Thread t < 6 n_agg sums w_t over its
// aggregate's nodes in their stored order; after a barrier, thread t forms
// y_t = sum_c A_c^-1[t][c] w_c (FP32 inverse entries, double-float sums).
// Cw, Cy: 6 n_agg DF of shared memory.  Every thread calls it.
__device__ __forceinline__ void coarse_solve_cta(const SysDesc& S, const float2* Wc, DF* Cw,
                                                 DF* Cy) {
  const int nc = 6 * S.n_agg;
  for (int t = threadIdx.x; t < nc; t += blockDim.x) {
    const int a = t / 6, d = t - 6 * a;
    DF acc{0.f, 0.f};
    for (int k = S.agg_ptr[a]; k < S.agg_ptr[a + 1]; ++k)
      acc = df_add(acc, ld_df(Wc + 6 * S.agg_nodes[k] + d));
    Cw[t] = acc;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nc; t += blockDim.x) {
    Acc A;
    const float* row = S.Aci + (size_t)t * nc;
    for (int c = 0; c < nc; ++c) acc_prod(A, DF{__ldg(row + c), 0.f}, Cw[c]);
    Cy[t] = acc_value(A);
  }
  __syncthreads();
}

// Row r of node i of P y (zero on a fixed DOF).
__device__ __forceinline__ DF prolong_row(const SysDesc& S, const DF* Cy, int node, int r) {
  if (S.fixed[6 * (size_t)node + r]) return DF{0.f, 0.f};
  const DF* y = Cy + 6 * S.agg_of[node];
  if (r >= 3) return y[r];
  // u = t + theta x o: (theta x o)_x = th_y o_z - th_z o_y, ...
  const float4 o = reinterpret_cast<const float4*>(S.node_rf)[node];
  const float oa = r == 0 ? o.z : (r == 1 ? o.x : o.y);
  const float ob = r == 0 ? o.y : (r == 1 ? o.z : o.x);
  const DF ta = r == 0 ? y[4] : (r == 1 ? y[5] : y[3]);
  const DF tb = r == 0 ? y[5] : (r == 1 ? y[3] : y[4]);
  return df_add(y[r], df_add(df_mul(ta, DF{oa, 0.f}), df_neg(df_mul(tb, DF{ob, 0.f}))));
}

// (b - K64 x)[i] for row i = 6 node + r in FP64 (x the FP64 solution)
__device__ __forceinline__ double residual64(const SysDesc& S, int node, int r, int i) {
  double acc = S.b[i];
  const int j1 = __ldg(S.row_ptr + node + 1);
  for (int j = __ldg(S.row_ptr + node); j < j1; ++j) {
    const int c0 = 6 * __ldg(S.col + j);
    const double* k = S.K64 + (size_t)j * 36 + 6 * r;
#pragma unroll
    for (int c = 0; c < 6; ++c) acc = fma(-__ldg(k + c), S.x[c0 + c], acc);
  }
  return acc;
}

__global__ void __launch_bounds__(1024) split_k_kernel(const SysDesc* __restrict__ sys,
                                                       const int* __restrict__ list) {
  const SysDesc& S = sys[list[blockIdx.y]];
  const long long n = (long long)S.row_ptr[S.n_nodes] * 36;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    S.klo[i] = __double2float_rn(S.K64[i] - (double)S.K32[i]);
}

// kSmem: the six double-float vectors in dynamic shared memory (systems of
// up to SMALL_SMEM_NODES nodes), else in the system's scratch vectors.
template <bool kSmem>
__global__ void __launch_bounds__(SMALL_MAX_THREADS) small_cg_kernel(const SysDesc* __restrict__ sys,
                                                        const int* __restrict__ list) {
  extern __shared__ __align__(16) float2 small_vec[];
  // warp partials and totals of the block sums, and cg_step's decision
  __shared__ DF red[3 * MAX_WARPS + 4];
  const SysDesc& S = sys[list[blockIdx.x]];
  SysScalars* sc = S.sc;
  const int n = S.n_nodes;
  const int groups = (n + NODES_PER_WARP - 1) / NODES_PER_WARP;
  // warps that own rows: min(32, groups) whatever the launch's block size (a
  // batch launches for its largest system), so the order of every sum is the
  // system's own
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = min(min((int)(blockDim.x >> 5), MAX_WARPS), groups);
  const Small G{S.row_ptr, S.col, S.K32, S.klo, S.M32, S.precond != SSO_JACOBI, n};
  // x, r, u = M^-1 r, w = K u, p, s = K p (double-float)
  float2 *X, *R, *U, *W, *P, *Sv;
  // two-level: each row's restriction share (Wc), w = P^T r and y = A_c^-1 w
  const bool two = S.precond == SSO_TWO_LEVEL;
  float2* Wc;
  DF *Cw, *Cy;
  if (kSmem) {
    const int nd = 6 * n;
    X = small_vec;
    R = X + nd;
    U = R + nd;
    W = U + nd;
    P = W + nd;
    Sv = P + nd;
    Wc = Sv + nd;
    Cw = reinterpret_cast<DF*>(Wc + nd);
  } else {
    X = reinterpret_cast<float2*>(S.dx);
    R = reinterpret_cast<float2*>(S.r);
    U = reinterpret_cast<float2*>(S.z);
    W = reinterpret_cast<float2*>(S.q);
    P = reinterpret_cast<float2*>(S.p0);
    Sv = reinterpret_cast<float2*>(S.p1);
    Wc = reinterpret_cast<float2*>(S.zb);
    Cw = reinterpret_cast<DF*>(small_vec);
  }
  Cy = Cw + COARSE_MAX_N;
  const bool warm = sc->state == ST_RESID;
  const double rtol2 = sc->rtol2;
  const int max_iter = sc->max_iter, max_sweeps = sc->max_sweeps;
  const int r6 = lane % 6;
  const DF zero{0.f, 0.f};
  // rows of group g: node 5 g + lane / 6, row lane % 6 (lanes 30, 31 idle);
  // the loop over groups is uniform over a warp
#define SMALL_ROWS(BODY)                                                  \
  for (int g = w; w < nw && g < groups; g += nw) {                        \
    const int node = NODES_PER_WARP * g + lane / 6;                       \
    const bool ok = lane < 6 * NODES_PER_WARP && node < n;               \
    const int i = 6 * node + r6;                                          \
    BODY                                                                  \
  }

  // x0 (warm start: the current solution) and ||b||^2
  DF ff_p = zero;
  SMALL_ROWS({
    if (ok) {
      const DF bi = df_split(S.b[i]);
      st_df(X + i, warm ? df_split(S.x[i]) : zero);
      ff_p = df_add(ff_p, df_mul(bi, bi));
    }
  })
  DF ff, dummy, dummy2;
  block_sum3(ff_p, zero, zero, red, nw, ff, dummy, dummy2);
  // convergence threshold rtol^2 ||b||^2 (the only FP64 scalar arithmetic, once)
  const DF thr = df_split(rtol2 * df_double(ff));

  // Every decision below is taken from block sums that all threads hold
  // alike, so the control flow (and every __syncthreads) is uniform.  The
  // scalars are double-float: an FP64 instruction per thread of the CTA
  // would cost more than the iteration's matrix product.
  int iters = 0, sweeps = 0, status = SSO_ERR_NOT_CONVERGED;
  DF rr64 = zero, rr64_prev = zero;
  for (;;) {
    // the refinement residual r = b - K64 x in FP64 (x = hi + lo), then
    // u = M^-1 r, w = K u and p = s = 0 in double-float
    for (int k = threadIdx.x; k < 6 * n; k += blockDim.x) {
      const float2 v = X[k];
      S.x[k] = (double)v.x + (double)v.y;
    }
    __syncthreads();
    DF rr_p = zero, ga_p = zero;
    SMALL_ROWS({
      DF rv = zero;
      if (ok) rv = df_split(residual64(S, node, r6, i));
      const DF uv = apply_precond(G, rv, node, r6, ok);
      const DF wc = two ? restrict_share(S, rv, node, r6, ok) : zero;
      if (ok) {
        st_df(R + i, rv);
        st_df(U + i, uv);
        st_df(P + i, zero);
        st_df(Sv + i, zero);
        rr_p = df_add(rr_p, df_mul(rv, rv));
        if (two)
          st_df(Wc + i, wc);
        else
          ga_p = df_add(ga_p, df_mul(rv, uv));
      }
    })
    if (two) {  // u += P A_c^-1 P^T r, then r^T u
      __syncthreads();
      coarse_solve_cta(S, Wc, Cw, Cy);
      SMALL_ROWS({
        if (ok) {
          const DF uv = df_add(ld_df(U + i), prolong_row(S, Cy, node, r6));
          st_df(U + i, uv);
          ga_p = df_add(ga_p, df_mul(ld_df(R + i), uv));
        }
      })
    }
    __syncthreads();  // U complete before K u
    DF de_p = zero;
    SMALL_ROWS({
      if (ok) {
        const DF wv = row_product(G, U, node, r6);
        st_df(W + i, wv);
        de_p = df_add(de_p, df_mul(wv, ld_df(U + i)));
      }
    })
    DF gamma, delta, rr;
    block_sum3(ga_p, de_p, rr_p, red, nw, gamma, delta, rr);
    rr64 = rr;
    if (!df_finite(rr) || !df_finite(delta)) {
      status = SSO_ERR_SINGULAR;
      break;
    }
    if (df_le(rr, thr)) {
      status = SSO_OK;
      break;
    }
    // out of iterations or sweeps, or the last sweep lowered the residual
    // less than 2x (rtol below what K and this arithmetic resolve)
    if (iters >= max_iter || sweeps >= max_sweeps ||
        (iters > 0 && df_le(DF{0.25f * rr64_prev.hi, 0.25f * rr64_prev.lo}, rr)))
      break;
    if (iters > 0) ++sweeps;
    rr64_prev = rr;
    if (!(delta.hi > 0.f)) {
      status = SSO_ERR_SINGULAR;
      break;
    }
    // Chronopoulos-Gear recurrences: one reduction point per iteration
    // (gamma = r^T u, delta = w^T u and r^T r together), s = K p carried by
    // s = w + beta s instead of a second product
    DF alpha = df_div(gamma, delta), beta = zero;
    while (iters < max_iter) {
      // p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, u = M^-1 r
      DF ga_n = zero, rr_n = zero;
      SMALL_ROWS({
        DF rv = zero;
        if (ok) {
          const DF pv = df_add(ld_df(U + i), df_mul(beta, ld_df(P + i)));
          const DF sv = df_add(ld_df(W + i), df_mul(beta, ld_df(Sv + i)));
          st_df(P + i, pv);
          st_df(Sv + i, sv);
          st_df(X + i, df_add(ld_df(X + i), df_mul(alpha, pv)));
          rv = df_add(ld_df(R + i), df_neg(df_mul(alpha, sv)));
          st_df(R + i, rv);
        }
        const DF uv = apply_precond(G, rv, node, r6, ok);
        const DF wc = two ? restrict_share(S, rv, node, r6, ok) : zero;
        if (ok) {
          st_df(U + i, uv);
          rr_n = df_add(rr_n, df_mul(rv, rv));
          if (two)
            st_df(Wc + i, wc);
          else
            ga_n = df_add(ga_n, df_mul(rv, uv));
        }
      })
      if (two) {  // u += P A_c^-1 P^T r, then r^T u
        __syncthreads();
        coarse_solve_cta(S, Wc, Cw, Cy);
        SMALL_ROWS({
          if (ok) {
            const DF uv = df_add(ld_df(U + i), prolong_row(S, Cy, node, r6));
            st_df(U + i, uv);
            ga_n = df_add(ga_n, df_mul(ld_df(R + i), uv));
          }
        })
      }
      __syncthreads();  // U complete before K u
      DF de_n = zero;
      SMALL_ROWS({
        if (ok) {
          const DF wv = row_product(G, U, node, r6);
          st_df(W + i, wv);
          de_n = df_add(de_n, df_mul(wv, ld_df(U + i)));
        }
      })
      const int code = cg_step(ga_n, de_n, rr_n, red, nw, thr, alpha, beta, gamma);
      ++iters;
      if (code == 1) {
        status = SSO_ERR_SINGULAR;
        break;
      }
      if (code == 2) break;  // the recursive residual: check the true one
    }
    if (status == SSO_ERR_SINGULAR) break;
    __syncthreads();  // X complete before the residual pass
  }
#undef SMALL_ROWS
  __syncthreads();
  // the solution in FP64
  for (int k = threadIdx.x; k < 6 * n; k += blockDim.x) {
    const float2 v = X[k];
    S.x[k] = (double)v.x + (double)v.y;
  }
  if (threadIdx.x == 0) {
    sc->iters = iters;
    sc->sweeps = sweeps;
    sc->rr64 = df_double(rr64);
    sc->ff = df_double(ff);
    sc->status = status;
    sc->state = ST_DONE;
  }
}

}  // namespace

cudaError_t launch_small_cg(const SysDesc* sys, const int* list, int n_list, int threads,
                            int max_nodes, bool two_level, cudaStream_t s) {
  if (n_list <= 0) return cudaSuccess;
  if (threads < 32 || threads % 32 || n_list > 65535) return cudaErrorInvalidValue;
  threads = threads < SMALL_MAX_THREADS ? threads : SMALL_MAX_THREADS;
  split_k_kernel<<<dim3(64, n_list), 256, 0, s>>>(sys, list);  // FP64: spread over SMs
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // two-level: a seventh vector (the rows' restriction shares) and w, y
  const size_t coarse = two_level ? 2 * COARSE_MAX_N * sizeof(DF) : 0;
  if (max_nodes <= SMALL_SMEM_NODES) {
    static bool attr = false;
    if (!attr) {
      e = cudaFuncSetAttribute(small_cg_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               SMALL_SMEM_NODES * SMALL_BYTES_PER_NODE_2L +
                                   (int)(2 * COARSE_MAX_N * sizeof(DF)));
      if (e != cudaSuccess) return e;
      attr = true;
    }
    const size_t smem =
        (size_t)max_nodes * (two_level ? SMALL_BYTES_PER_NODE_2L : SMALL_BYTES_PER_NODE) + coarse;
    small_cg_kernel<true><<<n_list, threads, smem, s>>>(sys, list);
  } else {
    small_cg_kernel<false><<<n_list, threads, coarse, s>>>(sys, list);
  }
  return cudaGetLastError();
}

}  // namespace sso
