// C-ABI of libsso (include/sso.h): models, batches, the host-side scatter-map
// builder and the batched CG driver.
//
// Streams: every model owns an internal non-blocking stream.  Each call first
// makes that stream wait for the caller's stream (event), does its work there
// and, before returning, makes the caller's stream wait for it.  The internal
// stream is what CUDA-graph capture needs (the legacy default stream cannot be
// captured).
//
// Memory: one cudaMalloc arena per model, carved into the arrays listed in
// ModelLayout; one per batch for its tables.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <cstring>
#include <deque>
#include <unordered_map>
#include <string>
#include <vector>
#include <map>
#include <memory>
#include <condition_variable>
#include <mutex>
#include <thread>

#include "sso_internal.cuh"

using namespace sso;

namespace {

thread_local std::string g_last_error;
std::atomic<unsigned long long> g_launches{0};

sso_status fail(sso_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

sso_status cuda_fail(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(SSO_ERR_OOM, buf);
  }
  return fail(SSO_ERR_CUDA, buf);
}

// SSO_DEBUG_SYNC=1 in the environment: every model's scatter map is checked
// on the host before upload, and the server synchronises after each of its
// phases and reports the phase in which a CUDA error appeared.
bool debug_sync() {
  static const bool on = [] {
    const char* v = std::getenv("SSO_DEBUG_SYNC");
    return v && v[0] == '1';
  }();
  return on;
}

#define CK(expr)                                         \
  do {                                                   \
    cudaError_t e_ = (expr);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr);  \
  } while (0)

#define CL(expr, n)                                      \
  do {                                                   \
    cudaError_t e_ = (expr);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr);  \
    g_launches += (n);                                   \
  } while (0)

// True when p is device (or managed) memory.  A pointer CUDA does not know,
// or a machine without a usable device, means host memory.
// Host memory the GPU cannot reach directly (not pinned, not managed).
bool is_pageable_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeUnregistered;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copy from a host or device source into host memory.
cudaError_t to_host(void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return cudaSuccess;
  if (!is_device_ptr(src)) {
    std::memcpy(dst, src, bytes);
    return cudaSuccess;
  }
  return cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost);
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Carves typed arrays out of one allocation (256-byte aligned).
// Carves 256-byte-aligned arrays out of one allocation; with a null base the
// pointers it returns are the arrays' byte offsets.
struct Carver {
  uintptr_t base;
  size_t off = 0;
  explicit Carver(void* b) : base(reinterpret_cast<uintptr_t>(b)) {}
  template <class T>
  T* take(size_t n) {
    off = align_up(off, 256);
    T* p = reinterpret_cast<T*>(base + off);
    off += n * sizeof(T);
    return p;
  }
};

// A vector whose resize leaves new elements uninitialised: the mesh arrays
// are overwritten by the caller's data right after, and zero-filling them
// first doubled the host time of queuing a large stream of requests.
template <class T>
struct NoInitAlloc : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = NoInitAlloc<U>;
  };
  NoInitAlloc() = default;
  template <class U>
  NoInitAlloc(const NoInitAlloc<U>&) {}
  template <class U>
  void construct(U* p) {
    ::new (static_cast<void*>(p)) U;
  }
  template <class U, class... A>
  void construct(U* p, A&&... a) {
    ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
  }
};
template <class T>
using RawVec = std::vector<T, NoInitAlloc<T>>;

struct HostMesh {
  int n_nodes = 0, n_beams = 0, n_quads = 0;
  RawVec<double> xyz, beam_props, quad_props, nodal_load;
  RawVec<int> beam_conn, quad_conn;
  RawVec<uint8_t> fixed;
  double pressure = 0.0, gamma = 0.0;
};

struct HostTopo {
  std::vector<int> row_ptr, col, brow, diag, cptr, csrc, nptr, nsrc;
  // epos[eb]: position of element block eb in assembly order (inverse of csrc)
  std::vector<int> epos;
  // two-level preconditioner: node aggregates and, per aggregate pair (g, h),
  // the K blocks (i, j) with i in g and j in h, in block order
  int n_agg = 0;
  std::vector<int> agg_of, agg_ptr, agg_nodes, cg_ptr, cg_src;
  // block (i, i+1) of every node or -1, and whether every block lies within
  // one of the diagonal (a chain)
  std::vector<int> chain_up;
  bool is_chain = false;
};

// Largest per-model counts of a set of models (the set-up grids' x extents).
struct SetupExtent {
  int beams = 0, quads = 0, blocks = 0, nodes = 0;
  template <class Model>
  void add(const Model* M) {
    beams = std::max(beams, M->n_beams);
    quads = std::max(quads, M->n_quads);
    blocks = std::max(blocks, M->n_blocks);
    nodes = std::max(nodes, M->n_nodes);
  }
};

}  // namespace

struct sso_model {
  int device = 0;
  cudaStream_t user_stream = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int n_nodes = 0, n_beams = 0, n_quads = 0, n_blocks = 0, n_eb = 0, n_slots = 0, n_tiles = 0;
  int n_agg = 0;  // node aggregates of the two-level preconditioner
  double pressure = 0.0, gamma = 0.0;
  std::vector<int> h_row_ptr, h_col;
  void* arena = nullptr;
  size_t arena_bytes = 0;  // size of the arena (fixed at creation)
  bool own_arena = true;   // false: the arena belongs to a server's pool
  // topology
  int *d_beam_conn, *d_quad_conn, *d_row_ptr, *d_col, *d_hslot, *d_brow, *d_diag, *d_cptr,
      *d_epos,
      *d_nptr, *d_nsrc;
  uint8_t* d_fixed;
  // design
  double *d_xyz, *d_beam_props, *d_quad_props, *d_nodal_load;
  // element and global arrays
  double *d_ke, *d_fslot, *d_gslot, *d_K64, *d_M64, *d_f, *d_u, *d_dx, *d_lam, *d_rhs, *d_r64;
  float *d_K32, *d_M32;
  void *d_r, *d_z, *d_p0, *d_p1, *d_q;
  double *d_part_a, *d_part_b, *d_dz, *d_dt, *d_C;
  unsigned* d_chunk_cnt;
  double* d_chunk_part;
  // material volume (Sec. 3.3): per-quad A t, per-slot t dA/dz (beam slots
  // stay 0), dW/dz, dW/dt, W
  double *d_vol, *d_vslot, *d_vdz, *d_vdt, *d_V;
  // SIMP topology (Eq. simp_eq): reference moduli E*, densities, dJ/drho
  double *d_E0, *d_rho, *d_drho;
  // two-level preconditioner: aggregate lists (per topology), per-design
  // node offsets, coarse matrix and its inverse, coarse vectors, z_b
  int *d_agg_of, *d_agg_ptr, *d_agg_nodes, *d_cg_ptr, *d_cg_src;
  double *d_node_r64, *d_Ac;
  float *d_node_rf, *d_Aci, *d_cw, *d_cy, *d_gj;
  double* d_cdot;
  double* d_zb;
  bool has_topology = false;
  double penal = 1.0;
  // SSO_CHAIN: the pattern is block-tridiagonal; workspace of the factors
  // (allocated on first use), assembly count when they were formed
  bool is_chain = false;
  int* d_chain_up;        // [n_nodes] block (i, i+1) or -1
  double* d_chain_ws = nullptr;
  long long assembly_gen = 0, chain_gen = -1;
  int* d_err;
  // the set-up stages' view of this model (device copy, written at creation)
  SetupJob* d_job;
  uint16_t* d_bmask;  // per block: supports of its row and column nodes
  // pinned staging of results bound for pageable host memory (sso_model_get)
  double* h_stage = nullptr;
  size_t h_stage_n = 0;
  bool assembled = false, solved = false;
  int assembled_precond = -1;
  sso_options last_opts;
  sso_batch* self_batch = nullptr;
};

struct sso_batch {
  std::vector<sso_model*> models;
  cudaStream_t stream = nullptr;  // models[0]'s internal stream
  int n_sys = 0, n_tiles = 0;
  void* arena = nullptr;
  SysDesc* d_sys = nullptr;
  SysScalars* d_sc = nullptr;
  TileDesc* d_tiles = nullptr;
  int* d_n_tiles = nullptr;
  int* d_n_active = nullptr;
  double* d_dots = nullptr;
  std::vector<SysDesc> h_sys;
  // the full tile list; while a solve runs, the device list may hold only the
  // tiles of systems still iterating (compacted), with tile0 moved to match
  std::vector<TileDesc> h_tiles;
  std::vector<int> h_tile0;
  std::vector<TileDesc> h_work;  // compacted list being uploaded (kept alive until synced)
  int n_listed = 0;              // systems whose tiles the device list holds
  int n_work = 0;                // tiles in h_work (uploaded from here)
  bool compacted = false;
  SysScalars* h_sc = nullptr;   // pinned, n_sys
  int* h_flag = nullptr;        // pinned: [0..1] upload, [2..3] read back
  // CG graphs: [0] FP32, [1] FP64, [2] FP32 with the two-level coarse kernels
  cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};
  int exec_iters[3] = {0, 0, 0};
  int exec_prof[3] = {0, 0, 0};
  int grid_a[3] = {0, 0, 0};
  int grid_b[3] = {0, 0, 0};
  int mult_a[3] = {1, 1, 1};  // kernel A's waves (grid_a / resident CTAs)
  // kernel A's CTAs per resident CTA slot.  A server's systems are in
  // different states at once (FP32 CG tiles next to FP64 residual and
  // initial tiles, which cost several times more), so a contiguous split of
  // its tile list leaves some CTAs with far more work than others; with 8x as
  // many CTAs as fit, each one short, the hardware block scheduler evens the
  // load out (each CTA still takes at least 16 tiles while more than one wave
  // of the resident slots is busy).  A batch's systems move in step, but each
  // enters its FP64 residual passes at its own iterations, so a batch uses 4x
  // (kBatchGridMult); the server 8x.
  int grid_a_mult = 1;
  std::chrono::steady_clock::time_point run_t0;  // start of the last batch_run
  // two-level work lists: every (system, aggregate), every system; their
  // lengths on the device (d_ccount[0], [1]) and the CTAs of their kernels
  AggRef* d_aggs = nullptr;
  int n_aggs = 0;
  int* d_csys = nullptr;
  int* d_ccount = nullptr;
  int grid_restrict = 0, grid_csolve = 0;
  // A large batch runs its CG as two to four parts on as many streams at once,
  // one host thread each: each part's kernel ramps and tails overlap the
  // others' work (128 shell designs: +8 % in 2 parts; 256: +14 % in 3).
  // parts[k] holds the systems [part0[k], part0[k + 1]); a part is a batch of
  // its own (tile list, scalars, CUDA graphs) on its first model's stream.
  std::vector<sso_batch*> parts;
  std::vector<int> part0;
  std::vector<cudaEvent_t> part_ev;
  // the models' set-up jobs (one launch per set-up stage for the whole batch)
  SetupJob* d_jobs = nullptr;
  // SSO_F32X2: the systems being solved (one CTA each)
  int* d_list = nullptr;
  std::vector<int> h_list;
  SetupExtent extent;
  cudaEvent_t ev = nullptr;
  // kernel timing (sso_batch_set_profiling): events around every A and B
  // launch inside the captured graph
  int profiling = 0;
  std::vector<cudaEvent_t> pev;
  double prof_ms_a = 0.0, prof_ms_b = 0.0;
  long long prof_launches = 0;
  // set-up and adjoint timing: 4 events per model around its element,
  // assembly and preconditioner + load kernels, 2 around the contraction pass
  std::vector<cudaEvent_t> sev;
  // per-model set-up and adjoint kernels run on a pool of streams (models
  // are independent), forked from and joined back to the batch stream
  std::vector<cudaStream_t> aux;
  std::vector<cudaEvent_t> aux_ev;
  cudaEvent_t ev_fork = nullptr;
  double prof_ms_el = 0.0, prof_ms_asm = 0.0, prof_ms_pre = 0.0, prof_ms_adj = 0.0;
  double prof_ms_setup = 0.0;  // fork-to-join wall time of the set-ups
  long long prof_setups = 0, prof_grads = 0;
};

namespace {

// ---------------------------------------------------------------------------
// Validation and the scatter map (Sec. 2.2.1 element_K_*_indices, as a sorted
// gather list).
sso_status validate(const HostMesh& m) {
  const int n = m.n_nodes;
  for (size_t k = 0; k < m.xyz.size(); ++k)
    if (!std::isfinite(m.xyz[k])) return fail(SSO_ERR_INVALID, "non-finite node coordinate");
  for (size_t k = 0; k < m.nodal_load.size(); ++k)
    if (!std::isfinite(m.nodal_load[k])) return fail(SSO_ERR_INVALID, "non-finite nodal load");
  if (!std::isfinite(m.pressure) || !std::isfinite(m.gamma))
    return fail(SSO_ERR_INVALID, "non-finite area load");
  char buf[200];
  for (int e = 0; e < m.n_beams; ++e) {
    const int i = m.beam_conn[2 * e], j = m.beam_conn[2 * e + 1];
    if (i < 0 || i >= n || j < 0 || j >= n) {
      snprintf(buf, sizeof(buf), "beam %d: node index out of range", e);
      return fail(SSO_ERR_INVALID, buf);
    }
    double L2 = 0.0;
    for (int k = 0; k < 3; ++k) {
      const double d = m.xyz[3 * j + k] - m.xyz[3 * i + k];
      L2 += d * d;
    }
    if (i == j || !(L2 > 0.0)) {
      snprintf(buf, sizeof(buf), "beam %d: zero length", e);
      return fail(SSO_ERR_INVALID, buf);
    }
    for (int k = 0; k < 6; ++k)
      if (!(m.beam_props[6 * e + k] > 0.0) || !std::isfinite(m.beam_props[6 * e + k])) {
        snprintf(buf, sizeof(buf), "beam %d: section/material value %d must be > 0", e, k);
        return fail(SSO_ERR_INVALID, buf);
      }
  }
  for (int e = 0; e < m.n_quads; ++e) {
    int nd[4];
    for (int a = 0; a < 4; ++a) {
      nd[a] = m.quad_conn[4 * e + a];
      if (nd[a] < 0 || nd[a] >= n) {
        snprintf(buf, sizeof(buf), "quad %d: node index out of range", e);
        return fail(SSO_ERR_INVALID, buf);
      }
    }
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b)
        if (nd[a] == nd[b]) {
          snprintf(buf, sizeof(buf), "quad %d: repeated node", e);
          return fail(SSO_ERR_INVALID, buf);
        }
    const double* p = &m.quad_props[5 * e];
    if (!(p[0] > 0.0) || !(p[1] > 0.0) || !(p[2] > -1.0 && p[2] < 0.5) || !(p[3] > 0.0) ||
        !(p[4] > 0.0)) {
      snprintf(buf, sizeof(buf), "quad %d: need t > 0, E > 0, -1 < nu < 0.5, kappa > 0", e);
      return fail(SSO_ERR_INVALID, buf);
    }
    // convex, consistently oriented about the diagonal normal
    double X[4][3];
    for (int a = 0; a < 4; ++a)
      for (int k = 0; k < 3; ++k) X[a][k] = m.xyz[3 * nd[a] + k];
    double d13[3], d24[3], nrm[3];
    for (int k = 0; k < 3; ++k) {
      d13[k] = X[2][k] - X[0][k];
      d24[k] = X[3][k] - X[1][k];
    }
    nrm[0] = d13[1] * d24[2] - d13[2] * d24[1];
    nrm[1] = d13[2] * d24[0] - d13[0] * d24[2];
    nrm[2] = d13[0] * d24[1] - d13[1] * d24[0];
    for (int a = 0; a < 4; ++a) {
      const double* P0 = X[a];
      const double* P1 = X[(a + 1) % 4];
      const double* P2 = X[(a + 2) % 4];
      double u[3], v[3];
      for (int k = 0; k < 3; ++k) {
        u[k] = P1[k] - P0[k];
        v[k] = P2[k] - P1[k];
      }
      const double c = (u[1] * v[2] - u[2] * v[1]) * nrm[0] + (u[2] * v[0] - u[0] * v[2]) * nrm[1] +
                       (u[0] * v[1] - u[1] * v[0]) * nrm[2];
      if (!(c > 0.0)) {
        snprintf(buf, sizeof(buf), "quad %d: not convex or degenerate", e);
        return fail(SSO_ERR_INVALID, buf);
      }
    }
  }
  return SSO_OK;
}

// Element-block eb -> (row node, col node).
void build_topology(const HostMesh& m, HostTopo& T) {
  const int n = m.n_nodes;
  // node adjacency (with the node itself) in flat arrays: count, prefix,
  // fill, then sort and deduplicate each short row in place
  std::vector<int> cnt(n + 1, 0);
  for (int i = 0; i < n; ++i) cnt[i + 1] = 1;
  for (int e = 0; e < m.n_beams; ++e)
    for (int a = 0; a < 2; ++a) cnt[m.beam_conn[2 * e + a] + 1] += 2;
  for (int e = 0; e < m.n_quads; ++e)
    for (int a = 0; a < 4; ++a) cnt[m.quad_conn[4 * e + a] + 1] += 4;
  for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  std::vector<int> flat(cnt[n]);
  std::vector<int> fill(cnt.begin(), cnt.end() - 1);
  for (int i = 0; i < n; ++i) flat[fill[i]++] = i;
  for (int e = 0; e < m.n_beams; ++e)
    for (int a = 0; a < 2; ++a) {
      const int r = m.beam_conn[2 * e + a];
      for (int b = 0; b < 2; ++b) flat[fill[r]++] = m.beam_conn[2 * e + b];
    }
  for (int e = 0; e < m.n_quads; ++e)
    for (int a = 0; a < 4; ++a) {
      const int r = m.quad_conn[4 * e + a];
      for (int b = 0; b < 4; ++b) flat[fill[r]++] = m.quad_conn[4 * e + b];
    }
  T.row_ptr.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    int* b = flat.data() + cnt[i];
    const int len = cnt[i + 1] - cnt[i];
    for (int k = 1; k < len; ++k) {  // insertion sort: rows are short
      const int v = b[k];
      int j = k - 1;
      while (j >= 0 && b[j] > v) {
        b[j + 1] = b[j];
        --j;
      }
      b[j + 1] = v;
    }
    int u = 0;
    for (int k = 0; k < len; ++k)
      if (u == 0 || b[k] != b[u - 1]) b[u++] = b[k];
    T.row_ptr[i + 1] = T.row_ptr[i] + u;
  }
  const int nb = T.row_ptr[n];
  T.col.resize(nb);
  T.brow.resize(nb);
  T.diag.resize(n);
  for (int i = 0; i < n; ++i) {
    const int* b = flat.data() + cnt[i];
    for (int k = T.row_ptr[i]; k < T.row_ptr[i + 1]; ++k) {
      T.col[k] = b[k - T.row_ptr[i]];
      T.brow[k] = i;
      if (T.col[k] == i) T.diag[i] = k;
    }
  }
  auto block_of = [&](int i, int j) {
    const int* b = T.col.data() + T.row_ptr[i];
    const int* e = T.col.data() + T.row_ptr[i + 1];
    return (int)(std::lower_bound(b, e, j) - T.col.data());
  };
  const int n_eb = 4 * m.n_beams + 16 * m.n_quads;
  std::vector<int> target(n_eb);
  for (int e = 0; e < m.n_beams; ++e)
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        target[4 * e + 2 * a + b] = block_of(m.beam_conn[2 * e + a], m.beam_conn[2 * e + b]);
  const int q0 = 4 * m.n_beams;
  for (int e = 0; e < m.n_quads; ++e)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b)
        target[q0 + 16 * e + 4 * a + b] = block_of(m.quad_conn[4 * e + a], m.quad_conn[4 * e + b]);
  // counting sort by target block, stable in element-block order
  T.cptr.assign(nb + 1, 0);
  for (int k = 0; k < n_eb; ++k) T.cptr[target[k] + 1]++;
  for (int b = 0; b < nb; ++b) T.cptr[b + 1] += T.cptr[b];
  T.csrc.resize(n_eb);
  {
    std::vector<int> fill(T.cptr.begin(), T.cptr.end() - 1);
    for (int k = 0; k < n_eb; ++k) T.csrc[fill[target[k]]++] = k;
  }
  T.epos.resize(n_eb);
  for (int k = 0; k < n_eb; ++k) T.epos[T.csrc[k]] = k;
  // node incidence: slots 2e+a (beams), 2 n_beams + 4e + a (quads), by node, stable
  const int n_slots = 2 * m.n_beams + 4 * m.n_quads;
  std::vector<int> slot_node(n_slots);
  for (int e = 0; e < m.n_beams; ++e)
    for (int a = 0; a < 2; ++a) slot_node[2 * e + a] = m.beam_conn[2 * e + a];
  for (int e = 0; e < m.n_quads; ++e)
    for (int a = 0; a < 4; ++a) slot_node[2 * m.n_beams + 4 * e + a] = m.quad_conn[4 * e + a];
  T.nptr.assign(n + 1, 0);
  for (int s = 0; s < n_slots; ++s) T.nptr[slot_node[s] + 1]++;
  for (int i = 0; i < n; ++i) T.nptr[i + 1] += T.nptr[i];
  T.nsrc.resize(n_slots);
  {
    std::vector<int> fill(T.nptr.begin(), T.nptr.end() - 1);
    for (int s = 0; s < n_slots; ++s) T.nsrc[fill[slot_node[s]]++] = s;
  }
}

// Aggregation of the nodes for the two-level preconditioner: greedy
// breadth-first growth from the lowest-numbered free node over the block
// adjacency (the rows of K), each aggregate stopping at `target` nodes;
// aggregates of fewer than target / 4 nodes are then merged into the
// neighbouring aggregate they share most block links with (lowest index on a
// tie).  Deterministic; returns the number of aggregates, agg_of[n] in
// [0, n_agg) numbered in order of their seeds.
int aggregate_nodes(int n, const std::vector<int>& row_ptr, const std::vector<int>& col,
                    int target, std::vector<int>& agg_of) {
  agg_of.assign(n, -1);
  std::vector<int> queue;
  queue.reserve(target);
  int n_agg = 0;
  for (int seed = 0; seed < n; ++seed) {
    if (agg_of[seed] >= 0) continue;
    queue.clear();
    queue.push_back(seed);
    agg_of[seed] = n_agg;
    for (size_t h = 0; h < queue.size() && (int)queue.size() < target; ++h) {
      const int v = queue[h];
      for (int b = row_ptr[v]; b < row_ptr[v + 1] && (int)queue.size() < target; ++b) {
        const int u = col[b];
        if (agg_of[u] < 0) {
          agg_of[u] = n_agg;
          queue.push_back(u);
        }
      }
    }
    ++n_agg;
  }
  // merge the small ones
  std::vector<int> size(n_agg, 0);
  for (int i = 0; i < n; ++i) size[agg_of[i]]++;
  std::vector<int> remap(n_agg);
  for (int g = 0; g < n_agg; ++g) remap[g] = g;
  std::vector<int> links(n_agg, 0);
  for (int g = 0; g < n_agg; ++g) {
    if (size[g] * 4 >= target || n_agg == 1) continue;
    std::vector<int> touched;
    for (int i = 0; i < n; ++i) {
      if (agg_of[i] != g) continue;
      for (int b = row_ptr[i]; b < row_ptr[i + 1]; ++b) {
        int h = agg_of[col[b]];
        while (remap[h] != h) h = remap[h];
        if (h == g) continue;
        if (links[h]++ == 0) touched.push_back(h);
      }
    }
    int best = -1;
    for (int h : touched)
      if (best < 0 || links[h] > links[best] || (links[h] == links[best] && h < best)) best = h;
    for (int h : touched) links[h] = 0;
    if (best >= 0) remap[g] = best;
  }
  std::vector<int> renum(n_agg, -1);
  int m = 0;
  for (int g = 0; g < n_agg; ++g) {
    int h = g;
    while (remap[h] != h) h = remap[h];
    if (h == g) renum[g] = m++;
  }
  for (int i = 0; i < n; ++i) {
    int h = agg_of[i];
    while (remap[h] != h) h = remap[h];
    agg_of[i] = renum[h];
  }
  return m;
}

// Aggregate size for a mesh of n nodes: at most kMaxAggregates aggregates
// (coarse problems of at most 6 kMaxAggregates = 234 unknowns, whose FP32
// inverse is read in every CG iteration), at least 16 nodes each.
constexpr int kMaxAggregates = COARSE_MAX_AGG;
int aggregate_target(int n) {
  return std::max(16, (n + kMaxAggregates - 1) / kMaxAggregates);
}

// Every index the set-up and CG kernels follow, checked against the extents
// of the arrays it indexes (the SSO_DEBUG_SYNC check).
bool topology_consistent(const HostMesh& m, const HostTopo& T) {
  const int n = m.n_nodes;
  const long long nb = (long long)T.col.size(), n_eb = (long long)T.csrc.size();
  const long long n_slots = (long long)T.nsrc.size();
  if ((long long)T.row_ptr.size() != n + 1 || T.row_ptr[0] != 0 || T.row_ptr[n] != nb) return false;
  for (int i = 0; i < n; ++i) {
    if (T.row_ptr[i + 1] <= T.row_ptr[i]) return false;
    const int d = T.diag[i];
    if (d < T.row_ptr[i] || d >= T.row_ptr[i + 1] || T.col[d] != i) return false;
    for (int b = T.row_ptr[i]; b < T.row_ptr[i + 1]; ++b)
      if (T.col[b] < 0 || T.col[b] >= n || T.brow[b] != i) return false;
  }
  if ((long long)T.cptr.size() != nb + 1 || T.cptr[0] != 0 || T.cptr[nb] != n_eb) return false;
  for (long long b = 0; b < nb; ++b)
    if (T.cptr[b + 1] < T.cptr[b]) return false;
  std::vector<char> seen(n_eb, 0);
  for (long long k = 0; k < n_eb; ++k) {
    const int e = T.csrc[k];
    if (e < 0 || e >= n_eb || seen[e]) return false;
    seen[e] = 1;
  }
  if (n_eb != 4LL * m.n_beams + 16LL * m.n_quads) return false;
  if ((long long)T.nptr.size() != n + 1 || T.nptr[0] != 0 || T.nptr[n] != n_slots) return false;
  for (int i = 0; i < n; ++i)
    if (T.nptr[i + 1] < T.nptr[i]) return false;
  std::vector<char> seen2(n_slots, 0);
  for (long long k = 0; k < n_slots; ++k) {
    const int q = T.nsrc[k];
    if (q < 0 || q >= n_slots || seen2[q]) return false;
    seen2[q] = 1;
  }
  for (int v : m.beam_conn)
    if (v < 0 || v >= n) return false;
  for (int v : m.quad_conn)
    if (v < 0 || v >= n) return false;
  return true;
}

int n_chunks_of(const sso_model* M) { return (M->n_tiles + CHUNK - 1) / CHUNK; }

// Lays out (base == nullptr: sizes only) every device array of a model.
size_t layout_model(sso_model* M, void* base) {
  Carver c(base);
  const size_t n = M->n_nodes, ndof = 6 * n;
  M->d_beam_conn = c.take<int>(2 * (size_t)M->n_beams);
  M->d_quad_conn = c.take<int>(4 * (size_t)M->n_quads);
  M->d_row_ptr = c.take<int>(n + 1);
  M->d_col = c.take<int>(M->n_blocks);
  M->d_hslot = c.take<int>(M->n_blocks);
  M->d_brow = c.take<int>(M->n_blocks);
  M->d_diag = c.take<int>(n);
  M->d_cptr = c.take<int>((size_t)M->n_blocks + 1);
  M->d_bmask = c.take<uint16_t>(M->n_blocks);
  M->d_epos = c.take<int>(M->n_eb);
  M->d_nptr = c.take<int>(n + 1);
  M->d_nsrc = c.take<int>(M->n_slots);
  M->d_fixed = c.take<uint8_t>(ndof);
  M->d_xyz = c.take<double>(3 * n);
  M->d_beam_props = c.take<double>(6 * (size_t)M->n_beams);
  M->d_quad_props = c.take<double>(5 * (size_t)M->n_quads);
  M->d_nodal_load = c.take<double>(ndof);
  M->d_E0 = c.take<double>(M->n_quads > 0 ? M->n_quads : 1);
  M->d_rho = c.take<double>(M->n_quads > 0 ? M->n_quads : 1);
  const size_t na = (size_t)std::max(M->n_agg, 1);
  M->d_agg_of = c.take<int>(n);
  M->d_agg_ptr = c.take<int>(na + 1);
  M->d_agg_nodes = c.take<int>(n);
  M->d_cg_ptr = c.take<int>(na * na + 1);
  M->d_cg_src = c.take<int>(M->n_blocks);
  M->d_chain_up = c.take<int>(n);
  // element blocks; after assembly also the Galerkin block products
  M->d_ke = c.take<double>((size_t)std::max(M->n_eb, M->n_blocks) * 36);
  M->d_fslot = c.take<double>(M->n_slots);
  M->d_gslot = c.take<double>(M->n_slots);
  M->d_K64 = c.take<double>((size_t)M->n_blocks * 36);
  M->d_K32 = c.take<float>((size_t)M->n_blocks * 36);
  M->d_M64 = c.take<double>(36 * n);
  M->d_M32 = c.take<float>(36 * n);
  M->d_f = c.take<double>(ndof);
  M->d_u = c.take<double>(ndof);
  M->d_dx = c.take<double>(ndof);
  M->d_lam = c.take<double>(ndof);
  M->d_rhs = c.take<double>(ndof);
  M->d_r64 = c.take<double>(ndof);
  M->d_r = c.take<double>(ndof);
  M->d_z = c.take<double>(ndof);
  M->d_p0 = c.take<double>(ndof);
  M->d_p1 = c.take<double>(ndof);
  M->d_q = c.take<double>(ndof);
  M->d_part_a = c.take<double>(2 * (size_t)WARPS * M->n_tiles);
  M->d_part_b = c.take<double>(2 * (size_t)WARPS * M->n_tiles);
  M->d_chunk_cnt = c.take<unsigned>(2 * (size_t)n_chunks_of(M));
  M->d_chunk_part = c.take<double>(4 * (size_t)n_chunks_of(M));
  M->d_dz = c.take<double>(n);
  M->d_dt = c.take<double>(M->n_quads > 0 ? M->n_quads : 1);
  M->d_C = c.take<double>(1);
  M->d_vol = c.take<double>(M->n_quads > 0 ? M->n_quads : 1);
  M->d_vslot = c.take<double>(M->n_slots);
  M->d_vdz = c.take<double>(n);
  M->d_vdt = c.take<double>(M->n_quads > 0 ? M->n_quads : 1);
  M->d_V = c.take<double>(1);
  M->d_drho = c.take<double>(M->n_quads > 0 ? M->n_quads : 1);
  M->d_node_r64 = c.take<double>(3 * n);
  M->d_node_rf = c.take<float>(4 * n);
  M->d_Ac = c.take<double>(36 * na * na);
  M->d_Aci = c.take<float>(36 * na * na);
  M->d_gj = c.take<float>(2 * (size_t)coarse_padded_n((int)na) * coarse_padded_n((int)na));
  M->d_cw = c.take<float>(6 * na);
  M->d_cy = c.take<float>(6 * na);
  M->d_cdot = c.take<double>(COARSE_ROW_BLOCKS);
  M->d_zb = c.take<double>(ndof);
  M->d_err = c.take<int>(1);
  M->d_job = c.take<SetupJob>(1);
  return align_up(c.off, 256);
}

sso_status check_options(const sso_options* o) {
  if (!o) return fail(SSO_ERR_INVALID, "options is NULL");
  if (o->precision != SSO_FP64 && o->precision != SSO_FP32_IR && o->precision != SSO_F32X2)
    return fail(SSO_ERR_INVALID, "precision must be SSO_FP64, SSO_FP32_IR or SSO_F32X2");
  if (o->precision == SSO_F32X2 && o->precond != SSO_JACOBI && o->precond != SSO_BLOCK_JACOBI &&
      o->precond != SSO_TWO_LEVEL)
    return fail(SSO_ERR_INVALID, "SSO_F32X2 needs SSO_JACOBI, SSO_BLOCK_JACOBI or SSO_TWO_LEVEL");
  if (o->precond != SSO_JACOBI && o->precond != SSO_BLOCK_JACOBI && o->precond != SSO_TWO_LEVEL &&
      o->precond != SSO_CHAIN)
    return fail(SSO_ERR_INVALID,
                "precond must be SSO_JACOBI, SSO_BLOCK_JACOBI, SSO_TWO_LEVEL or SSO_CHAIN");
  if (o->precond == SSO_TWO_LEVEL && o->precision == SSO_FP64)
    return fail(SSO_ERR_INVALID, "SSO_TWO_LEVEL needs SSO_FP32_IR or SSO_F32X2");
  if (o->precond == SSO_CHAIN && o->precision != SSO_FP64)
    return fail(SSO_ERR_INVALID, "SSO_CHAIN needs SSO_FP64");
  if (!(o->rtol > 0.0) || !(o->inner_rtol >= 0.0) || o->inner_rtol >= 1.0)
    return fail(SSO_ERR_INVALID, "need rtol > 0 and 0 <= inner_rtol < 1");
  if (o->max_iter <= 0 || o->max_sweeps <= 0)
    return fail(SSO_ERR_INVALID, "max_iter and max_sweeps must be > 0");
  if (o->iters_per_launch <= 0 || o->iters_per_launch > 4096)
    return fail(SSO_ERR_INVALID, "iters_per_launch must be in [1, 4096]");
  return SSO_OK;
}

// Work on the model's internal stream ordered after the caller's stream.
sso_status enter(sso_model* M) {
  CK(cudaSetDevice(M->device));
  CK(cudaEventRecord(M->ev_in, M->user_stream));
  CK(cudaStreamWaitEvent(M->stream, M->ev_in, 0));
  return SSO_OK;
}
sso_status leave(sso_model* M) {
  CK(cudaEventRecord(M->ev_out, M->stream));
  CK(cudaStreamWaitEvent(M->user_stream, M->ev_out, 0));
  return SSO_OK;
}

// The set-up stages' view of a model's arrays.
SetupJob make_setup_job(const sso_model* M) {
  SetupJob J;
  J.xyz = M->d_xyz;
  J.beam_conn = M->d_beam_conn;
  J.beam_props = M->d_beam_props;
  J.quad_conn = M->d_quad_conn;
  J.quad_props = M->d_quad_props;
  J.n_beams = M->n_beams;
  J.n_quads = M->n_quads;
  J.n_nodes = M->n_nodes;
  J.n_blocks = M->n_blocks;
  J.pressure = M->pressure;
  J.gamma = M->gamma;
  J.epos = M->d_epos;
  J.kes = M->d_ke;
  J.fslot = M->d_fslot;
  J.cptr = M->d_cptr;
  J.bmask = M->d_bmask;
  J.fixed = M->d_fixed;
  J.K64 = M->d_K64;
  J.K32 = M->d_K32;
  J.err = M->d_err;
  J.diag = M->d_diag;
  J.M64 = M->d_M64;
  J.M32 = M->d_M32;
  J.nptr = M->d_nptr;
  J.nsrc = M->d_nsrc;
  J.nodal_load = M->d_nodal_load;
  J.f = M->d_f;
  return J;
}

// Element matrices, K, preconditioner and loads of the n models whose jobs
// are jobs[0 .. n), one launch per stage.  ev (or NULL): four events recorded
// before the element kernels, after them, after the assembly and at the end.
sso_status setup_stages(const SetupJob* jobs, int n, const SetupExtent& x, int precond,
                        cudaStream_t s, const cudaEvent_t* ev = nullptr) {
  if (ev) CK(cudaEventRecord(ev[0], s));
  CL(launch_setup_beams(jobs, n, x.beams, s), x.beams > 0);
  CL(launch_setup_quads(jobs, n, x.quads, s), x.quads > 0);
  if (ev) CK(cudaEventRecord(ev[1], s));
  CL(launch_setup_assemble(jobs, n, x.blocks, s), 1);
  if (ev) CK(cudaEventRecord(ev[2], s));
  CL(launch_setup_precond(jobs, n, x.nodes, precond == SSO_JACOBI ? SSO_JACOBI : SSO_BLOCK_JACOBI,
                          s),
     1);
  CL(launch_setup_loads(jobs, n, x.nodes, s), 1);
  if (ev) CK(cudaEventRecord(ev[3], s));
  return SSO_OK;
}

// The two-level coarse space of one assembled model.
sso_status setup_coarse(sso_model* M, cudaStream_t s) {
  CL(launch_coarse_setup(M->n_nodes, M->n_agg, M->n_blocks, M->d_agg_ptr, M->d_agg_nodes,
                         M->d_brow, M->d_col, M->d_cg_ptr, M->d_cg_src, M->d_xyz, M->d_fixed,
                         M->d_K64, M->d_node_r64, M->d_node_rf, M->d_ke, M->d_Ac, M->d_gj,
                         M->d_Aci, s),
     coarse_setup_launches(M->n_agg));
  return SSO_OK;
}

void mark_assembled(sso_model* M, int precond) {
  M->assembled = true;
  M->assembled_precond = precond;
  ++M->assembly_gen;
}

// Element matrices, K, preconditioner and loads of one model (its own job).
sso_status setup_model(sso_model* M, int precond, cudaStream_t s) {
  SetupExtent x;
  x.add(M);
  sso_status st = setup_stages(M->d_job, 1, x, precond, s);
  if (st != SSO_OK) return st;
  if (precond == SSO_TWO_LEVEL && (st = setup_coarse(M, s)) != SSO_OK) return st;
  mark_assembled(M, precond);
  return SSO_OK;
}

sso_status batch_graph(sso_batch* B, bool fp64, int iters, bool two_level = false) {
  const int k = fp64 ? 1 : two_level ? 2 : 0;
  if (B->exec[k] && B->exec_iters[k] == iters && B->exec_prof[k] == B->profiling) return SSO_OK;
  if (B->exec[k]) {
    cudaGraphExecDestroy(B->exec[k]);
    B->exec[k] = nullptr;
  }
  if (B->grid_a[k] == 0) {
    int ga = 1, gb = 1;
    pcg_grid_limits(fp64, &ga, &gb);  // CTAs resident at once
    B->grid_a[k] = std::max(1, std::min(B->n_tiles, ga * B->grid_a_mult));
    B->grid_b[k] = std::max(1, std::min(B->n_tiles, gb));
    // the multiplier kernel A splits its ranges by: the waves its grid really
    // has, so that a batch of fewer tiles than resident CTAs keeps one tile
    // per CTA instead of gathering them on a quarter of the SMs
    B->mult_a[k] = std::max(1, B->grid_a[k] / std::max(1, ga));
  }
  if (B->profiling) {
    while ((int)B->pev.size() < 2 * iters + 1) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      B->pev.push_back(e);
    }
  }
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = cudaSuccess;
  if (B->profiling)
    err = cudaEventRecordWithFlags(B->pev[0], B->stream, cudaEventRecordExternal);
  for (int it = 0; it < iters && err == cudaSuccess; ++it) {
    err = launch_pcg_a(fp64, B->d_tiles, B->d_n_tiles, B->d_sys, B->d_n_active, B->grid_a[k],
                       B->mult_a[k], B->stream);
    if (err == cudaSuccess && B->profiling)
      err = cudaEventRecordWithFlags(B->pev[2 * it + 1], B->stream, cudaEventRecordExternal);
    if (err == cudaSuccess)
      err = launch_pcg_b(fp64, B->d_tiles, B->d_n_tiles, B->d_sys, B->d_n_active, B->grid_b[k],
                         B->stream);
    if (err == cudaSuccess && two_level) {
      err = launch_coarse_restrict(B->d_aggs, B->d_ccount, B->grid_restrict, B->d_sys,
                                   B->stream);
      if (err == cudaSuccess)
        err = launch_coarse_solve(B->d_csys, B->d_ccount + 1, B->grid_csolve, B->d_sys,
                                  B->d_n_active, B->stream);
      if (err == cudaSuccess)
        err = launch_coarse_prolong(B->d_tiles, B->d_n_tiles, B->d_sys,
                                    std::max(1, std::min(B->n_tiles, 152 * 8)), B->stream);
    }
    if (err == cudaSuccess && B->profiling)
      err = cudaEventRecordWithFlags(B->pev[2 * it + 2], B->stream, cudaEventRecordExternal);
  }
  cudaError_t e2 = cudaStreamEndCapture(B->stream, &g);
  if (err != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(err, "capturing the CG graph");
  }
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
  err = cudaGraphInstantiate(&B->exec[k], g, 0);
  cudaGraphDestroy(g);
  if (err != cudaSuccess) return cuda_fail(err, "cudaGraphInstantiate");
  B->exec_iters[k] = iters;
  B->exec_prof[k] = B->profiling;
  return SSO_OK;
}

// At least n timing events in B->sev.
sso_status ensure_setup_events(sso_batch* B, size_t n) {
  while (B->sev.size() < n) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    B->sev.push_back(e);
  }
  return SSO_OK;
}

constexpr int kAuxStreams = 16;

// Forks B's pool of streams off its stream (created on first use).
sso_status fork_aux(sso_batch* B) {
  if (B->aux.empty()) {
    const int k = std::min(kAuxStreams, B->n_sys);
    CK(cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming));
    for (int i = 0; i < k; ++i) {
      cudaStream_t st;
      cudaEvent_t ev;
      CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      B->aux.push_back(st);
      CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      B->aux_ev.push_back(ev);
    }
  }
  CK(cudaEventRecord(B->ev_fork, B->stream));
  for (cudaStream_t st : B->aux) CK(cudaStreamWaitEvent(st, B->ev_fork, 0));
  return SSO_OK;
}

// Orders B's stream after everything issued on the pool.
sso_status join_aux(sso_batch* B) {
  for (size_t i = 0; i < B->aux.size(); ++i) {
    CK(cudaEventRecord(B->aux_ev[i], B->aux[i]));
    CK(cudaStreamWaitEvent(B->stream, B->aux_ev[i], 0));
  }
  return SSO_OK;
}

float elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  return cudaEventElapsedTime(&ms, a, b) == cudaSuccess ? ms : 0.f;
}

// Adds the kernel durations of the last graph launch (after it completed).
sso_status accumulate_profile(sso_batch* B, int iters) {
  for (int it = 0; it < iters; ++it) {
    float a = 0.f, b = 0.f;
    CK(cudaEventElapsedTime(&a, B->pev[2 * it], B->pev[2 * it + 1]));
    CK(cudaEventElapsedTime(&b, B->pev[2 * it + 1], B->pev[2 * it + 2]));
    B->prof_ms_a += a;
    B->prof_ms_b += b;
  }
  B->prof_launches += iters;
  return SSO_OK;
}

// Runs the batched CG over the systems with active[s] != 0, solving
// K x = b with b = (adjoint ? rhs : f), x = (adjoint ? lam : u).
// SSO_CHAIN: every active system solved directly (factors formed once per
// assembly); while its FP64 residual is above rtol, refined with the same
// factors (x += K^-1 (b - K x)), at most max_sweeps times or until the
// residual stops falling.
sso_status chain_run(sso_batch* B, const sso_options* o, bool adjoint,
                     const std::vector<char>& active, sso_stats* stats) {
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<double> norms(2 * (size_t)B->n_sys, 0.0);
  std::vector<int> sweeps(B->n_sys, 0);
  for (int s = 0; s < B->n_sys; ++s) {
    sso_model* M = B->models[s];
    SysDesc& D = B->h_sys[s];
    D.precond = o->precond;
    D.b = adjoint ? M->d_rhs : M->d_f;
    D.x = adjoint ? M->d_lam : M->d_u;
    if (!active[s]) continue;
    if (!M->is_chain)
      return fail(SSO_ERR_INVALID, "SSO_CHAIN needs a block-tridiagonal K (every element joining "
                                   "consecutively numbered nodes)");
    const int n = M->n_nodes;
    if (!M->d_chain_ws) {
      const size_t bytes = sizeof(double) * (chain_workspace_doubles(n) + residual_partials(n) + 2);
      cudaError_t e = cudaMalloc(&M->d_chain_ws, bytes);
      if (e != cudaSuccess) {
        M->d_chain_ws = nullptr;
        return cuda_fail(e, "cudaMalloc(chain workspace)");
      }
    }
    double* part = M->d_chain_ws + chain_workspace_doubles(n);
    double* out = part + residual_partials(n);
    if (M->chain_gen != M->assembly_gen) {
      CL(launch_chain_factor(n, M->d_diag, M->d_chain_up, M->d_K64, M->d_chain_ws, M->d_err,
                             B->stream),
         1);
      M->chain_gen = M->assembly_gen;
    }
    CL(launch_chain_solve(n, M->d_chain_ws, D.b, D.x, M->d_err, B->stream), 1);
    double prev = HUGE_VAL;
    for (;;) {
      CL(launch_residual_norms(n, M->d_row_ptr, M->d_col, M->d_K64, D.x, D.b, M->d_r64, part, out,
                               B->stream),
         2);
      CK(cudaMemcpyAsync(&norms[2 * (size_t)s], out, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                         B->stream));
      CK(cudaStreamSynchronize(B->stream));
      const double rr = norms[2 * (size_t)s], bb = norms[2 * (size_t)s + 1];
      if (!(rr > o->rtol * o->rtol * bb) || !(rr < 0.25 * prev) || sweeps[s] >= o->max_sweeps)
        break;
      prev = rr;
      ++sweeps[s];
      CL(launch_chain_solve(n, M->d_chain_ws, M->d_r64, M->d_dx, M->d_err, B->stream), 1);
      CL(launch_axpby(6 * n, 1.0, M->d_dx, D.x, M->d_fixed, D.x, B->stream), 1);
    }
  }
  CK(cudaMemcpyAsync(B->d_sys, B->h_sys.data(), sizeof(SysDesc) * B->n_sys,
                     cudaMemcpyHostToDevice, B->stream));
  CK(cudaStreamSynchronize(B->stream));
  const double ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  sso_status first_bad = SSO_OK;
  for (int s = 0; s < B->n_sys; ++s) {
    if (!active[s]) continue;
    const double rr = norms[2 * (size_t)s], bb = norms[2 * (size_t)s + 1];
    const bool ok = std::isfinite(rr) && rr <= o->rtol * o->rtol * bb;
    const sso_status st = ok ? SSO_OK : SSO_ERR_NOT_CONVERGED;
    if (st != SSO_OK && first_bad == SSO_OK) first_bad = st;
    if (stats) {
      stats[s].status = st;
      stats[s].iterations = 0;
      stats[s].sweeps = sweeps[s];
      stats[s].rel_residual = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
      stats[s].ms = ms;
    }
  }
  if (first_bad != SSO_OK) g_last_error = "direct chain solve above rtol (loss of accuracy)";
  return first_bad;
}

sso_status finish_run(sso_batch* B, const std::vector<char>& active, sso_stats* stats);

// defer: return after queuing the copy of the scalars, without waiting (the
// caller synchronises the stream and calls finish_run).
sso_status batch_run(sso_batch* B, const sso_options* o, bool adjoint,
                     const std::vector<char>& active, sso_stats* stats, bool defer = false) {
  if (o->precond == SSO_CHAIN) return chain_run(B, o, adjoint, active, stats);
  const auto t0 = std::chrono::steady_clock::now();
  const bool fp64 = o->precision == SSO_FP64;
  const double inner = fp64 ? 0.0 : o->inner_rtol;
  if (B->compacted) {  // the previous solve left a compacted list: restore the full one
    CK(cudaMemcpyAsync(B->d_tiles, B->h_tiles.data(), B->h_tiles.size() * sizeof(TileDesc),
                       cudaMemcpyHostToDevice, B->stream));
    CK(cudaMemcpyAsync(B->d_n_tiles, &B->n_tiles, sizeof(int), cudaMemcpyHostToDevice,
                       B->stream));
    for (int s = 0; s < B->n_sys; ++s) B->h_sys[s].tile0 = B->h_tile0[s];
    B->compacted = false;
  }
  int n_act = 0;
  for (int s = 0; s < B->n_sys; ++s) {
    sso_model* M = B->models[s];
    SysDesc& D = B->h_sys[s];
    D.precond = o->precond;
    D.b = adjoint ? M->d_rhs : M->d_f;
    D.x = adjoint ? M->d_lam : M->d_u;
    SysScalars& S = B->h_sc[s];
    std::memset(&S, 0, sizeof(S));
    const bool warm = !adjoint && o->warm_start && M->solved;
    S.state = active[s] ? (warm ? ST_RESID : ST_INIT) : ST_DONE;
    S.status = active[s] ? SSO_ERR_NOT_CONVERGED : SSO_OK;
    S.rtol2 = o->rtol * o->rtol;
    S.inner_rtol2 = inner * inner;
    S.max_iter = o->max_iter;
    S.max_sweeps = o->max_sweeps;
    // the one-CTA double-float CG sets its own x and scratch and counts no
    // chunks: three fewer operations ahead of its launch
    if (active[s]) {
      ++n_act;
      if (o->precision != SSO_F32X2) {
        if (!warm)
          CK(cudaMemsetAsync(D.x, 0, sizeof(double) * 6 * (size_t)M->n_nodes, B->stream));
        CK(cudaMemsetAsync(M->d_dx, 0, sizeof(double) * 6 * (size_t)M->n_nodes, B->stream));
        CK(cudaMemsetAsync(M->d_chunk_cnt, 0, sizeof(unsigned) * 2 * (size_t)n_chunks_of(M),
                           B->stream));
      }
    }
  }
  CK(cudaMemcpyAsync(B->d_sys, B->h_sys.data(), sizeof(SysDesc) * B->n_sys,
                     cudaMemcpyHostToDevice, B->stream));
  CK(cudaMemcpyAsync(B->d_sc, B->h_sc, sizeof(SysScalars) * B->n_sys, cudaMemcpyHostToDevice,
                     B->stream));
  B->n_listed = B->n_sys;
  B->h_flag[0] = n_act;
  B->h_flag[1] = 0;
  CK(cudaMemcpyAsync(B->d_n_active, B->h_flag, 2 * sizeof(int), cudaMemcpyHostToDevice,
                     B->stream));
  if (n_act > 0 && o->precision == SSO_F32X2) {
    // every active system's whole CG in one CTA of one launch
    B->h_list.clear();
    int groups = 1, max_nodes = 1;
    for (int s = 0; s < B->n_sys; ++s)
      if (active[s]) {
        B->h_list.push_back(s);
        groups = std::max(groups, (B->models[s]->n_nodes + NODES_PER_WARP - 1) / NODES_PER_WARP);
        max_nodes = std::max(max_nodes, B->models[s]->n_nodes);
      }
    CK(cudaMemcpyAsync(B->d_list, B->h_list.data(), B->h_list.size() * sizeof(int),
                       cudaMemcpyHostToDevice, B->stream));
    const int threads = 32 * std::min(32, groups);
    CL(launch_small_cg(B->d_sys, B->d_list, (int)B->h_list.size(), threads, max_nodes,
                       o->precond == SSO_TWO_LEVEL, B->stream),
       2);
  } else if (n_act > 0) {
    const bool two_level = o->precond == SSO_TWO_LEVEL;
    sso_status st = batch_graph(B, fp64, o->iters_per_launch, two_level);
    if (st != SSO_OK) return st;
    const int k = fp64 ? 1 : two_level ? 2 : 0;
    const long long max_launches = (long long)o->max_iter * 2 / o->iters_per_launch + 4LL * o->max_sweeps + 8;
    long long launches = 0;
    for (;;) {
      CK(cudaGraphLaunch(B->exec[k], B->stream));
      g_launches += (two_level ? 5ull : 2ull) * (unsigned long long)o->iters_per_launch;
      CK(cudaMemcpyAsync(B->h_flag + 2, B->d_n_active, 2 * sizeof(int),
                         cudaMemcpyDeviceToHost, B->stream));
      CK(cudaEventRecord(B->ev, B->stream));
      CK(cudaEventSynchronize(B->ev));
      if (B->profiling) {
        sso_status ps = accumulate_profile(B, o->iters_per_launch);
        if (ps != SSO_OK) return ps;
      }
      ++launches;
      if (B->h_flag[3] != 0)
        return fail(SSO_ERR_CUDA, "CG kernel gave up waiting for a bulk copy (device fault?)");
      if (B->h_flag[2] <= 0) break;
      if (o->timeout_ms > 0.0) {
        const double ms = std::chrono::duration<double, std::milli>(
                              std::chrono::steady_clock::now() - t0).count();
        if (ms > o->timeout_ms) break;
      }
      if (launches > max_launches) break;  // caps are enforced on the device; belt and braces
      // Systems have left since the tile list was last built: list only the
      // tiles of those still iterating, so that every CTA keeps working on
      // them instead of a few CTAs holding all of the remaining ones.  Each
      // system's tiles stay contiguous and in order (tile0 moves with them),
      // so its results do not change.
      const int n_now = B->h_flag[2];
      if (B->n_listed - n_now >= std::max(1, B->n_listed / 16)) {
        CK(cudaMemcpyAsync(B->h_sc, B->d_sc, sizeof(SysScalars) * B->n_sys,
                           cudaMemcpyDeviceToHost, B->stream));
        CK(cudaStreamSynchronize(B->stream));
        B->h_work.clear();
        int listed = 0;
        for (int s = 0; s < B->n_sys; ++s) {
          if (B->h_sc[s].state == ST_DONE) continue;
          B->h_sys[s].tile0 = (int)B->h_work.size();
          const int t0s = B->h_tile0[s], nt = B->models[s]->n_tiles;
          B->h_work.insert(B->h_work.end(), B->h_tiles.begin() + t0s,
                           B->h_tiles.begin() + t0s + nt);
          ++listed;
        }
        B->n_work = (int)B->h_work.size();
        if (B->n_work > 0)
          CK(cudaMemcpyAsync(B->d_tiles, B->h_work.data(), B->h_work.size() * sizeof(TileDesc),
                             cudaMemcpyHostToDevice, B->stream));
        CK(cudaMemcpyAsync(B->d_n_tiles, &B->n_work, sizeof(int), cudaMemcpyHostToDevice,
                           B->stream));
        CK(cudaMemcpyAsync(B->d_sys, B->h_sys.data(), sizeof(SysDesc) * B->n_sys,
                           cudaMemcpyHostToDevice, B->stream));
        B->compacted = true;
        B->n_listed = listed;
      }
    }
  }
  CK(cudaMemcpyAsync(B->h_sc, B->d_sc, sizeof(SysScalars) * B->n_sys, cudaMemcpyDeviceToHost,
                     B->stream));
  B->run_t0 = t0;
  if (defer) return SSO_OK;  // the caller synchronises, then calls finish_run
  CK(cudaStreamSynchronize(B->stream));
  return finish_run(B, active, stats);
}

// Per-system status and statistics of the last batch_run, from the scalars
// it copied to the host (after the stream has been synchronised).
sso_status finish_run(sso_batch* B, const std::vector<char>& active, sso_stats* stats) {
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() -
                                                              B->run_t0)
                        .count();
  sso_status first_bad = SSO_OK;
  for (int s = 0; s < B->n_sys; ++s) {
    const SysScalars& S = B->h_sc[s];
    int st = S.state == ST_DONE ? S.status : SSO_ERR_TIMEOUT;
    if (!active[s]) st = SSO_OK;
    if (st != SSO_OK && first_bad == SSO_OK) first_bad = (sso_status)st;
    if (stats && active[s]) {
      stats[s].status = st;
      stats[s].iterations = S.iters;
      stats[s].sweeps = S.sweeps;
      stats[s].rel_residual = S.ff > 0.0 ? std::sqrt(S.rr64 / S.ff) : 0.0;
      stats[s].ms = ms;
    }
  }
  if (first_bad != SSO_OK) {
    char buf[160];
    snprintf(buf, sizeof(buf), "CG finished with status %d in at least one system",
             (int)first_bad);
    g_last_error = buf;
  }
  return first_bad;
}

// The CG of a batch's active systems: batch_run, or for a split batch its
// parts at once, each on its own stream and host thread.  While profiling, the
// batch runs whole (one graph over every system), so that the events around
// each kernel time it alone at the batch's full size.  The parts start after
// the work already on the batch's stream, which then waits for them.
sso_status run_cg(sso_batch* B, const sso_options* o, bool adjoint,
                  const std::vector<char>& active, sso_stats* stats, bool* deferred = nullptr) {
  if (B->parts.empty() || B->profiling) {
    // one launch and no host loop (double-float CG): the caller may fold
    // the wait for it into its own
    const bool defer = deferred && o->precision == SSO_F32X2 && o->precond != SSO_CHAIN;
    if (deferred) *deferred = defer;
    return batch_run(B, o, adjoint, active, stats, defer);
  }
  if (deferred) *deferred = false;
  const int np = (int)B->parts.size();
  CK(cudaEventRecord(B->part_ev[0], B->stream));
  for (int k = 1; k < np; ++k) CK(cudaStreamWaitEvent(B->parts[k]->stream, B->part_ev[0], 0));
  std::vector<sso_status> res(np, SSO_OK);
  std::vector<std::string> msg(np);
  auto work = [&](int k) {
    const std::vector<char> act(active.begin() + B->part0[k], active.begin() + B->part0[k + 1]);
    res[k] = batch_run(B->parts[k], o, adjoint, act, stats ? stats + B->part0[k] : nullptr);
    if (res[k] != SSO_OK) msg[k] = g_last_error;
  };
  std::vector<std::thread> threads;
  try {
    for (int k = 1; k < np; ++k) threads.emplace_back(work, k);
  } catch (const std::exception&) {
    // no thread: the remaining parts run after the first, in this thread
  }
  work(0);
  for (std::thread& t : threads) t.join();
  for (int k = 1 + (int)threads.size(); k < np; ++k) work(k);
  for (int k = 1; k < np; ++k) {
    CK(cudaEventRecord(B->part_ev[k], B->parts[k]->stream));
    CK(cudaStreamWaitEvent(B->stream, B->part_ev[k], 0));
  }
  int worst = -1;
  for (int k = 0; k < np; ++k)
    if (res[k] != SSO_OK && (worst < 0 || res[k] == SSO_ERR_CUDA || res[k] == SSO_ERR_OOM))
      worst = k;
  if (worst < 0) return SSO_OK;
  g_last_error = msg[worst];
  return res[worst];
}

// Tile k of model M (system s of a batch): its block range, the aligned runs
// of column indices and row_ptr entries, and the node range (halo) of the
// vector entries its rows read; stage = 1 when all of it fits the FP32
// staging buffers of kernel A.
TileDesc make_tile(const sso_model* M, int s, int k) {
  TileDesc d;
  d.sys = s;
  d.node0 = k * TILE;
  d.nn = std::min(TILE, M->n_nodes - d.node0);
  d.j0 = M->h_row_ptr[d.node0];
  const int j1 = M->h_row_ptr[d.node0 + d.nn];
  d.nblk = j1 - d.j0;
  d.cb = d.j0 & ~3;
  d.ncb = ((j1 + 3) & ~3) - d.cb;
  // halo: the sorted column nodes, cut into runs at gaps longer than 8 nodes
  // (a gap shorter than that costs less to copy than a run of its own), each
  // run widened to even bounds (16-byte bulk copies of 24-byte nodes); a
  // single run covering everything is used whenever it fits
  std::vector<int> cols(M->h_col.begin() + d.j0, M->h_col.begin() + j1);
  std::sort(cols.begin(), cols.end());
  cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
  for (int k = 0; k < HALO_RUNS; ++k) d.vlo[k] = d.nv[k] = 0;
  int halo_nodes = 0, runs = 0;
  if (!cols.empty()) {
    const int lo = cols.front() & ~1, hi = cols.back() | 1;
    if ((long long)(hi - lo + 1) * 24 <= STAGE_SLAB_V) {
      d.vlo[0] = lo;
      d.nv[0] = hi - lo + 1;
      runs = 1;
    } else {
      std::vector<std::pair<int, int>> seg;  // [first, last] nodes, even / odd bounds
      for (int c : cols) {
        const int a = c & ~1, b = c | 1;
        if (!seg.empty() && a <= seg.back().second + 9)
          seg.back().second = std::max(seg.back().second, b);
        else
          seg.push_back({a, b});
      }
      runs = (int)seg.size();
      for (int k = 0; k < runs && k < HALO_RUNS; ++k) {
        d.vlo[k] = seg[k].first;
        d.nv[k] = seg[k].second - seg[k].first + 1;
      }
    }
    for (int k = 0; k < HALO_RUNS; ++k) halo_nodes += d.nv[k];
  }
  d.rb = d.node0 & ~3;
  d.nrb = ((d.node0 + d.nn + 1 + 3) & ~3) - d.rb;
  d.stage_k = d.nblk > 0 && (long long)d.nblk * 144 <= STAGE_SLAB_K &&
              d.ncb * 4 <= STAGE_SLAB_C && d.nrb * 4 <= STAGE_SLAB_R;
  d.stage = d.stage_k && runs >= 1 && runs <= HALO_RUNS &&
            (long long)halo_nodes * 24 <= STAGE_SLAB_V;
  return d;
}

// Host half of a model: the mesh, validated, and its scatter map, node
// incidence and tile descriptors, plus the packed image of every array the
// device arena starts with.  Built without CUDA calls, so any thread may run
// it.
struct ModelPrep {
  // node aggregates of the two-level preconditioner (a server whose
  // preconditioner is another skips them: they cost most of the preparation)
  bool aggregates = true;
  HostMesh hm;
  HostTopo T;
  sso_model* M = nullptr;  // counts, host copies and arena offsets (base 0)
  std::vector<TileDesc> tiles;  // sys = -1
  std::vector<unsigned char> image;  // arena bytes [0, prefix)
  size_t bytes = 0, prefix = 0;
  std::string error;
  ~ModelPrep() { delete M; }
};

// Copies a mesh (host or device arrays) into P.hm after the argument checks.
sso_status mesh_to_prep(const sso_mesh* mesh, ModelPrep& P) {
  if (!mesh) return fail(SSO_ERR_INVALID, "mesh is NULL");
  if (mesh->n_nodes <= 0 || mesh->n_beams < 0 || mesh->n_quads < 0)
    return fail(SSO_ERR_INVALID, "need n_nodes > 0, n_beams >= 0, n_quads >= 0");
  if (mesh->n_beams + mesh->n_quads == 0) return fail(SSO_ERR_INVALID, "no elements");
  if (!mesh->xyz || !mesh->fixed || !mesh->nodal_load)
    return fail(SSO_ERR_INVALID, "xyz, fixed and nodal_load are required");
  if (mesh->n_beams > 0 && (!mesh->beam_conn || !mesh->beam_props))
    return fail(SSO_ERR_INVALID, "beam arrays missing");
  if (mesh->n_quads > 0 && (!mesh->quad_conn || !mesh->quad_props))
    return fail(SSO_ERR_INVALID, "quad arrays missing");
  const long long eb = 4LL * mesh->n_beams + 16LL * mesh->n_quads;
  if (eb >= (1LL << 31) || 6LL * mesh->n_nodes >= (1LL << 31))
    return fail(SSO_ERR_INVALID, "mesh too large for 32-bit block indices");
  HostMesh& hm = P.hm;
  hm.n_nodes = mesh->n_nodes;
  hm.n_beams = mesh->n_beams;
  hm.n_quads = mesh->n_quads;
  hm.pressure = mesh->pressure;
  hm.gamma = mesh->gamma;
  hm.xyz.resize(3 * (size_t)hm.n_nodes);
  hm.nodal_load.resize(6 * (size_t)hm.n_nodes);
  hm.fixed.resize(6 * (size_t)hm.n_nodes);
  hm.beam_conn.resize(2 * (size_t)hm.n_beams);
  hm.beam_props.resize(6 * (size_t)hm.n_beams);
  hm.quad_conn.resize(4 * (size_t)hm.n_quads);
  hm.quad_props.resize(5 * (size_t)hm.n_quads);
  CK(to_host(hm.xyz.data(), mesh->xyz, hm.xyz.size() * sizeof(double)));
  CK(to_host(hm.nodal_load.data(), mesh->nodal_load, hm.nodal_load.size() * sizeof(double)));
  CK(to_host(hm.fixed.data(), mesh->fixed, hm.fixed.size()));
  CK(to_host(hm.beam_conn.data(), mesh->beam_conn, hm.beam_conn.size() * sizeof(int)));
  CK(to_host(hm.beam_props.data(), mesh->beam_props, hm.beam_props.size() * sizeof(double)));
  CK(to_host(hm.quad_conn.data(), mesh->quad_conn, hm.quad_conn.size() * sizeof(int)));
  CK(to_host(hm.quad_props.data(), mesh->quad_props, hm.quad_props.size() * sizeof(double)));
  for (auto& f : hm.fixed) f = f ? 1 : 0;
  return SSO_OK;
}

// Validation, scatter map, tile descriptors and the arena image.  On failure
// the message is in P.error (this may run off the calling thread).
sso_status prepare_model(ModelPrep& P) {
  const HostMesh& hm = P.hm;
  sso_status st = validate(hm);
  if (st != SSO_OK) {
    P.error = g_last_error;
    return st;
  }
  build_topology(hm, P.T);
  if (debug_sync() && !topology_consistent(hm, P.T)) {
    P.error = "scatter map inconsistent (internal error)";
    return SSO_ERR_INVALID;
  }
  HostTopo& Tm = P.T;
  if (P.aggregates) {
    const int n = hm.n_nodes;
    // at most COARSE_MAX_AGG aggregates (the coarse inverse is read every iteration)
    for (int target = aggregate_target(n);; target += std::max(1, target / 4)) {
      Tm.n_agg = aggregate_nodes(n, Tm.row_ptr, Tm.col, target, Tm.agg_of);
      if (Tm.n_agg <= COARSE_MAX_AGG) break;
    }
    const int na = Tm.n_agg;
    Tm.agg_ptr.assign(na + 1, 0);
    for (int i = 0; i < n; ++i) Tm.agg_ptr[Tm.agg_of[i] + 1]++;
    for (int g = 0; g < na; ++g) Tm.agg_ptr[g + 1] += Tm.agg_ptr[g];
    Tm.agg_nodes.resize(n);
    std::vector<int> fillg(Tm.agg_ptr.begin(), Tm.agg_ptr.end() - 1);
    for (int i = 0; i < n; ++i) Tm.agg_nodes[fillg[Tm.agg_of[i]]++] = i;
    const int nb = (int)Tm.col.size();
    Tm.cg_ptr.assign((size_t)na * na + 1, 0);
    std::vector<int> key(nb);
    for (int b = 0; b < nb; ++b) {
      key[b] = Tm.agg_of[Tm.brow[b]] * na + Tm.agg_of[Tm.col[b]];
      Tm.cg_ptr[key[b] + 1]++;
    }
    for (size_t q = 0; q < (size_t)na * na; ++q) Tm.cg_ptr[q + 1] += Tm.cg_ptr[q];
    Tm.cg_src.resize(nb);
    std::vector<int> fillp(Tm.cg_ptr.begin(), Tm.cg_ptr.end() - 1);
    for (int b = 0; b < nb; ++b) Tm.cg_src[fillp[key[b]]++] = b;
  }
  {
    const int n = hm.n_nodes;
    Tm.chain_up.assign(n, -1);
    Tm.is_chain = true;
    for (int i = 0; i < n; ++i)
      for (int b = Tm.row_ptr[i]; b < Tm.row_ptr[i + 1]; ++b) {
        const int j = Tm.col[b];
        if (j > i + 1 || j < i - 1) Tm.is_chain = false;
        if (j == i + 1) Tm.chain_up[i] = b;
      }
  }
  const HostTopo& T = P.T;
  sso_model* M = new sso_model();
  P.M = M;
  M->is_chain = T.is_chain;
  M->n_agg = T.n_agg;
  M->n_nodes = hm.n_nodes;
  M->n_beams = hm.n_beams;
  M->n_quads = hm.n_quads;
  M->n_blocks = (int)T.col.size();
  M->n_eb = (int)T.csrc.size();
  M->n_slots = (int)T.nsrc.size();
  M->n_tiles = (hm.n_nodes + TILE - 1) / TILE;
  M->pressure = hm.pressure;
  M->gamma = hm.gamma;
  M->h_row_ptr = T.row_ptr;
  M->h_col = T.col;
  sso_default_options(&M->last_opts);
  P.tiles.reserve(M->n_tiles);
  for (int t = 0; t < M->n_tiles; ++t) P.tiles.push_back(make_tile(M, -1, t));
  // every block's column slot in its tile's staged halo (the runs laid end
  // to end; the same rule as the consumers' slot of their own node)
  std::vector<int> hslot(T.col.size(), 0);
  for (const TileDesc& d : P.tiles) {
    if (!d.stage) continue;
    const int v1 = d.nv[1] ? d.vlo[1] : INT_MAX, v2 = d.nv[2] ? d.vlo[2] : INT_MAX;
    const int sh0 = -d.vlo[0], sh1 = d.nv[0] - d.vlo[1], sh2 = d.nv[0] + d.nv[1] - d.vlo[2];
    for (int j = d.j0; j < d.j0 + d.nblk; ++j) {
      const int c = T.col[j];
      hslot[j] = c + (c >= v2 ? sh2 : (c >= v1 ? sh1 : sh0));
    }
  }
  // arena offsets (base 0) and the image of the arrays that start it
  P.bytes = layout_model(M, nullptr);
  P.prefix = (size_t)reinterpret_cast<uintptr_t>(M->d_ke);
  P.image.assign(P.prefix, 0);
  auto put = [&](const void* dev_off, const void* src, size_t b) {
    if (b) std::memcpy(P.image.data() + reinterpret_cast<uintptr_t>(dev_off), src, b);
  };
  put(M->d_beam_conn, hm.beam_conn.data(), hm.beam_conn.size() * 4);
  put(M->d_quad_conn, hm.quad_conn.data(), hm.quad_conn.size() * 4);
  put(M->d_row_ptr, T.row_ptr.data(), T.row_ptr.size() * 4);
  put(M->d_col, T.col.data(), T.col.size() * 4);
  put(M->d_hslot, hslot.data(), hslot.size() * 4);
  put(M->d_brow, T.brow.data(), T.brow.size() * 4);
  put(M->d_diag, T.diag.data(), T.diag.size() * 4);
  put(M->d_cptr, T.cptr.data(), T.cptr.size() * 4);
  {
    std::vector<uint16_t> bm(T.col.size());
    for (size_t b = 0; b < T.col.size(); ++b) {
      const int ni = T.brow[b], nj = T.col[b];
      int m = ni == nj ? 1 << 12 : 0;
      for (int d = 0; d < 6; ++d) {
        m |= (hm.fixed[6 * (size_t)ni + d] != 0) << d;
        m |= (hm.fixed[6 * (size_t)nj + d] != 0) << (6 + d);
      }
      bm[b] = (uint16_t)m;
    }
    put(M->d_bmask, bm.data(), bm.size() * 2);
  }
  put(M->d_epos, T.epos.data(), T.epos.size() * 4);
  put(M->d_nptr, T.nptr.data(), T.nptr.size() * 4);
  put(M->d_nsrc, T.nsrc.data(), T.nsrc.size() * 4);
  put(M->d_fixed, hm.fixed.data(), hm.fixed.size());
  put(M->d_xyz, hm.xyz.data(), hm.xyz.size() * 8);
  put(M->d_beam_props, hm.beam_props.data(), hm.beam_props.size() * 8);
  put(M->d_quad_props, hm.quad_props.data(), hm.quad_props.size() * 8);
  put(M->d_nodal_load, hm.nodal_load.data(), hm.nodal_load.size() * 8);
  put(M->d_agg_of, T.agg_of.data(), T.agg_of.size() * 4);
  put(M->d_agg_ptr, T.agg_ptr.data(), T.agg_ptr.size() * 4);
  put(M->d_agg_nodes, T.agg_nodes.data(), T.agg_nodes.size() * 4);
  put(M->d_cg_ptr, T.cg_ptr.data(), T.cg_ptr.size() * 4);
  put(M->d_cg_src, T.cg_src.data(), T.cg_src.size() * 4);
  put(M->d_chain_up, T.chain_up.data(), T.chain_up.size() * 4);
  {
    std::vector<double> e0(hm.n_quads), one(hm.n_quads, 1.0);
    for (int e = 0; e < hm.n_quads; ++e) e0[e] = hm.quad_props[5 * (size_t)e + 1];
    put(M->d_E0, e0.data(), e0.size() * 8);
    put(M->d_rho, one.data(), one.size() * 8);
  }
  return SSO_OK;
}

// Device half: arena (arena != NULL: given, e.g. from a server pool, and
// not freed with the model), one upload of the image (from `image`, a pinned
// copy of P.image, when given), the rest zeroed.  own_stream:
// the model gets its own stream and events (ordered after user_stream) and the
// call returns with the upload done; otherwise everything is ordered on s
// and the model has no stream of its own (server models).  Takes P.M.
sso_status create_model_device(ModelPrep& P, cudaStream_t user_stream, bool own_stream,
                               cudaStream_t s, sso_model** out, void* arena = nullptr,
                               const void* image = nullptr) {
  sso_model* M = P.M;
  P.M = nullptr;
  auto cleanup = [&](sso_status st) {
    sso_model_destroy(M);
    return st;
  };
  cudaError_t e = cudaGetDevice(&M->device);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaGetDevice"));
  M->user_stream = user_stream;
  if (own_stream) {
    e = cudaStreamCreateWithFlags(&M->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&M->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&M->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "stream/event creation"));
    s = M->stream;
  }
  M->arena_bytes = P.bytes;
  if (arena) {
    M->arena = arena;
    M->own_arena = false;
  } else {
    e = cudaMalloc(&M->arena, P.bytes);
    if (e != cudaSuccess) {
      M->arena = nullptr;
      return cleanup(cuda_fail(e, "cudaMalloc(model arena)"));
    }
  }
  layout_model(M, M->arena);
  e = cudaMemcpyAsync(M->arena, image ? image : P.image.data(), P.prefix,
                      cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(static_cast<unsigned char*>(M->arena) + P.prefix, 0, P.bytes - P.prefix,
                        s);
  if (e == cudaSuccess) {
    e = launch_store_setup_job(M->d_job, make_setup_job(M), s);
    g_launches += 1;
  }
  if (e == cudaSuccess && own_stream) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "uploading the model"));
  *out = M;
  return SSO_OK;
}

sso_status ensure_self_batch(sso_model* M) {
  if (M->self_batch) return SSO_OK;
  sso_model* ms[1] = {M};
  return sso_batch_create(ms, 1, &M->self_batch);
}

}  // namespace

namespace sso {
sso_status record_failure(sso_status st, const char* msg) { return fail(st, msg); }
void count_launches(unsigned long long n) { g_launches += n; }
}  // namespace sso

// ===========================================================================
extern "C" {

void sso_default_options(sso_options* o) {
  if (!o) return;
  o->precision = SSO_FP32_IR;
  o->precond = SSO_BLOCK_JACOBI;
  o->rtol = 1e-8;
  o->inner_rtol = 2e-3;
  o->max_iter = 200000;
  o->max_sweeps = 40;
  o->iters_per_launch = 32;
  o->warm_start = 0;
  o->timeout_ms = 0.0;
}

const char* sso_last_error(void) { return g_last_error.c_str(); }

const char* sso_version(void) { return "sso 0.1 (sm_103a)"; }

unsigned long long sso_kernel_launches(void) { return g_launches.load(); }

sso_status sso_beam_stiffness(int32_t n_beams, const double* d_xyz, const int32_t* d_beam_conn,
                              const double* d_beam_props, double* d_ke, void* stream) {
  if (n_beams < 0) return fail(SSO_ERR_INVALID, "n_beams < 0");
  if (n_beams > 0 && (!d_xyz || !d_beam_conn || !d_beam_props || !d_ke))
    return fail(SSO_ERR_INVALID, "NULL pointer");
  CL(launch_beam_stiffness(n_beams, d_xyz, d_beam_conn, d_beam_props, d_ke,
                           (cudaStream_t)stream),
     n_beams > 0);
  return SSO_OK;
}

sso_status sso_quad_stiffness(int32_t n_quads, const double* d_xyz, const int32_t* d_quad_conn,
                              const double* d_quad_props, double* d_ke, void* stream) {
  if (n_quads < 0) return fail(SSO_ERR_INVALID, "n_quads < 0");
  if (n_quads > 0 && (!d_xyz || !d_quad_conn || !d_quad_props || !d_ke))
    return fail(SSO_ERR_INVALID, "NULL pointer");
  CL(launch_quad_stiffness(n_quads, d_xyz, d_quad_conn, d_quad_props, 0.0, 0.0, d_ke, nullptr,
                           (cudaStream_t)stream),
     n_quads > 0);
  return SSO_OK;
}

sso_status sso_bsr_spmv(int32_t n_nodes, const int32_t* d_row_ptr, const int32_t* d_col,
                        const double* d_K, const double* d_x, double* d_y, double* d_xty,
                        void* stream) {
  if (n_nodes < 0) return fail(SSO_ERR_INVALID, "n_nodes < 0");
  if (n_nodes == 0) return SSO_OK;
  if (!d_row_ptr || !d_col || !d_K || !d_x || !d_y || !d_xty)
    return fail(SSO_ERR_INVALID, "NULL pointer");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t tiles = (size_t)(n_nodes + SPMV_TILE - 1) / SPMV_TILE;
  void* scratch = nullptr;
  CK(cudaMallocAsync(&scratch, tiles * sizeof(double) + 256, s));
  unsigned int* counter = (unsigned int*)((char*)scratch + align_up(tiles * sizeof(double), 16));
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess)
    e = launch_bsr_spmv(n_nodes, d_row_ptr, d_col, d_K, d_x, d_y, d_xty, (double*)scratch,
                        counter, s);
  if (e == cudaSuccess) g_launches += 1;
  cudaError_t e2 = cudaFreeAsync(scratch, s);
  if (e != cudaSuccess) return cuda_fail(e, "sso_bsr_spmv");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
  return SSO_OK;
}

sso_status sso_model_create(const sso_mesh* mesh, void* stream, sso_model** out) {
  if (!out) return fail(SSO_ERR_INVALID, "out is NULL");
  *out = nullptr;
  ModelPrep P;
  sso_status st = mesh_to_prep(mesh, P);
  if (st != SSO_OK) return st;
  if ((st = prepare_model(P)) != SSO_OK) return fail(st, P.error);
  return create_model_device(P, (cudaStream_t)stream, true, nullptr, out);
}

void sso_model_destroy(sso_model* M) {
  if (!M) return;
  if (M->self_batch) sso_batch_destroy(M->self_batch);
  if (M->stream) cudaStreamSynchronize(M->stream);
  if (M->arena && M->own_arena) cudaFree(M->arena);
  if (M->d_chain_ws) cudaFree(M->d_chain_ws);
  if (M->h_stage) cudaFreeHost(M->h_stage);
  if (M->ev_in) cudaEventDestroy(M->ev_in);
  if (M->ev_out) cudaEventDestroy(M->ev_out);
  if (M->stream) cudaStreamDestroy(M->stream);
  delete M;
}

sso_status sso_model_set_design(sso_model* M, const double* z, const double* t) {
  if (!M) return fail(SSO_ERR_INVALID, "model is NULL");
  sso_status st = enter(M);
  if (st != SSO_OK) return st;
  if (z)
    CK(cudaMemcpy2DAsync(M->d_xyz + 2, 3 * sizeof(double), z, sizeof(double), sizeof(double),
                         M->n_nodes, cudaMemcpyDefault, M->stream));
  if (t && M->n_quads > 0)
    CK(cudaMemcpy2DAsync(M->d_quad_props, 5 * sizeof(double), t, sizeof(double), sizeof(double),
                         M->n_quads, cudaMemcpyDefault, M->stream));
  if (z || t) M->assembled = false;
  return leave(M);
}

sso_status sso_model_solve(sso_model* M, const sso_options* opts, sso_stats* stats) {
  if (!M) return fail(SSO_ERR_INVALID, "model is NULL");
  sso_status st = ensure_self_batch(M);
  if (st != SSO_OK) return st;
  return sso_batch_solve(M->self_batch, opts, stats);
}

sso_status sso_model_gradient(sso_model* M, double w, const double* g, sso_stats* stats) {
  if (!M) return fail(SSO_ERR_INVALID, "model is NULL");
  sso_status st = ensure_self_batch(M);
  if (st != SSO_OK) return st;
  const double* gs[1] = {g};
  return sso_batch_gradient(M->self_batch, &w, gs, stats);
}

sso_status sso_model_get(sso_model* M, double* u, double* C, double* dz, double* dt,
                         double* lam) {
  if (!M) return fail(SSO_ERR_INVALID, "model is NULL");
  sso_status st = enter(M);
  if (st != SSO_OK) return st;
  const size_t ndof = 6 * (size_t)M->n_nodes;
  struct Out {
    double* dst;
    const double* src;
    size_t n;
  } outs[5] = {{u, M->d_u, ndof},
               {C, M->d_C, 1},
               {dz, M->d_dz, (size_t)M->n_nodes},
               {dt, M->d_dt, M->n_quads > 0 ? (size_t)M->n_quads : 0},
               {lam, M->d_lam, ndof}};
  // Outputs in pageable host memory go through one pinned staging buffer, so
  // their copies run together and the call waits once (a copy into pageable
  // memory would each wait for the stream); device and pinned outputs are
  // copied straight.
  size_t staged = 0;
  bool pageable[5] = {};
  for (int k = 0; k < 5; ++k)
    if (outs[k].dst && outs[k].n && is_pageable_host(outs[k].dst)) {
      pageable[k] = true;
      staged += outs[k].n;
    }
  if (staged > M->h_stage_n) {
    if (M->h_stage) cudaFreeHost(M->h_stage);
    M->h_stage = nullptr;
    M->h_stage_n = 0;
    CK(cudaMallocHost(&M->h_stage, staged * sizeof(double)));
    M->h_stage_n = staged;
  }
  size_t off = 0;
  for (int k = 0; k < 5; ++k) {
    if (!outs[k].dst || !outs[k].n) continue;
    double* to = pageable[k] ? M->h_stage + off : outs[k].dst;
    CK(cudaMemcpyAsync(to, outs[k].src, outs[k].n * 8, cudaMemcpyDefault, M->stream));
    if (pageable[k]) off += outs[k].n;
  }
  CK(cudaStreamSynchronize(M->stream));
  off = 0;
  for (int k = 0; k < 5; ++k)
    if (pageable[k]) {
      std::memcpy(outs[k].dst, M->h_stage + off, outs[k].n * 8);
      off += outs[k].n;
    }
  return leave(M);
}

sso_status sso_aggregate(const sso_mesh* mesh, int32_t* agg_of_node, int32_t* n_aggregates) {
  if (!agg_of_node || !n_aggregates) return fail(SSO_ERR_INVALID, "NULL argument");
  ModelPrep P;
  sso_status st = mesh_to_prep(mesh, P);
  if (st != SSO_OK) return st;
  if ((st = validate(P.hm)) != SSO_OK) return st;
  build_topology(P.hm, P.T);
  std::vector<int> agg;
  for (int target = aggregate_target(P.hm.n_nodes);; target += std::max(1, target / 4)) {
    *n_aggregates = aggregate_nodes(P.hm.n_nodes, P.T.row_ptr, P.T.col, target, agg);
    if (*n_aggregates <= COARSE_MAX_AGG) break;
  }
  std::copy(agg.begin(), agg.end(), agg_of_node);
  return SSO_OK;
}

sso_status sso_model_set_topology(sso_model* M, const double* rho, double penal) {
  if (!M) return fail(SSO_ERR_INVALID, "model is NULL");
  if (rho && !(penal >= 1.0 && std::isfinite(penal)))
    return fail(SSO_ERR_INVALID, "need a finite penalty factor >= 1");
  if (M->n_quads == 0) return rho ? fail(SSO_ERR_INVALID, "the model has no quads") : SSO_OK;
  sso_status st = enter(M);
  if (st != SSO_OK) return st;
  if (rho) {
    std::vector<double> h(M->n_quads);
    CK(to_host(h.data(), rho, h.size() * sizeof(double)));
    for (double v : h)
      if (!(v > 0.0 && v <= 1.0)) return fail(SSO_ERR_INVALID, "densities must lie in (0, 1]");
    CK(cudaMemcpyAsync(M->d_rho, h.data(), h.size() * 8, cudaMemcpyHostToDevice, M->stream));
    CK(cudaStreamSynchronize(M->stream));  // h is a temporary
    M->penal = penal;
    M->has_topology = true;
  } else {
    const std::vector<double> one(M->n_quads, 1.0);
    CK(cudaMemcpyAsync(M->d_rho, one.data(), one.size() * 8, cudaMemcpyHostToDevice, M->stream));
    CK(cudaStreamSynchronize(M->stream));
    M->penal = 1.0;
    M->has_topology = false;
  }
  CL(launch_simp(M->n_quads, M->d_rho, M->d_E0, M->penal, M->d_quad_props, M->stream), 1);
  M->assembled = false;
  M->solved = false;
  return leave(M);
}

sso_status sso_model_get_topology_gradient(sso_model* M, double* drho) {
  if (!M || !drho) return fail(SSO_ERR_INVALID, "NULL argument");
  if (!M->has_topology) return fail(SSO_ERR_INVALID, "no topology densities set");
  sso_status st = enter(M);
  if (st != SSO_OK) return st;
  CK(cudaMemcpyAsync(drho, M->d_drho, M->n_quads * 8, cudaMemcpyDefault, M->stream));
  CK(cudaStreamSynchronize(M->stream));
  return leave(M);
}

sso_status sso_model_volume(sso_model* M, double* V, double* dVdz, double* dVdt) {
  if (!M) return fail(SSO_ERR_INVALID, "model is NULL");
  sso_status st = enter(M);
  if (st != SSO_OK) return st;
  cudaStream_t s = M->stream;
  if (M->n_quads > 0) {
    CL(launch_quad_volume(M->n_quads, M->d_xyz, M->d_quad_conn, M->d_quad_props,
                          M->d_vslot + 2 * (size_t)M->n_beams, M->d_vdt, M->d_vol, s),
       1);
    CL(launch_ordered_sum(M->n_quads, M->d_vol, M->d_V, s), 1);
  } else {
    CK(cudaMemsetAsync(M->d_V, 0, sizeof(double), s));
  }
  CL(launch_node_gather(M->n_nodes, M->d_nptr, M->d_nsrc, 2 * M->n_beams, nullptr, M->d_vslot,
                        nullptr, M->d_fixed, nullptr, M->d_vdz, s),
     1);
  if (V) CK(cudaMemcpyAsync(V, M->d_V, 8, cudaMemcpyDefault, s));
  if (dVdz) CK(cudaMemcpyAsync(dVdz, M->d_vdz, M->n_nodes * 8, cudaMemcpyDefault, s));
  if (dVdt && M->n_quads > 0)
    CK(cudaMemcpyAsync(dVdt, M->d_vdt, M->n_quads * 8, cudaMemcpyDefault, s));
  CK(cudaStreamSynchronize(s));
  return leave(M);
}

sso_status sso_model_info(const sso_model* M, int32_t* n_nodes, int32_t* n_blocks,
                          int32_t* n_elem_blocks) {
  if (!M) return fail(SSO_ERR_INVALID, "model is NULL");
  if (n_nodes) *n_nodes = M->n_nodes;
  if (n_blocks) *n_blocks = M->n_blocks;
  if (n_elem_blocks) *n_elem_blocks = M->n_eb;
  return SSO_OK;
}

sso_status sso_model_get_stiffness(sso_model* M, int32_t* row_ptr, int32_t* col, double* K64,
                                   float* K32) {
  if (!M) return fail(SSO_ERR_INVALID, "model is NULL");
  if ((K64 || K32) && !M->assembled) return fail(SSO_ERR_INVALID, "K not assembled yet");
  sso_status st = enter(M);
  if (st != SSO_OK) return st;
  if (row_ptr)
    CK(cudaMemcpyAsync(row_ptr, M->h_row_ptr.data(), M->h_row_ptr.size() * 4, cudaMemcpyDefault,
                       M->stream));
  if (col)
    CK(cudaMemcpyAsync(col, M->h_col.data(), M->h_col.size() * 4, cudaMemcpyDefault, M->stream));
  if (K64)
    CK(cudaMemcpyAsync(K64, M->d_K64, (size_t)M->n_blocks * 36 * 8, cudaMemcpyDefault,
                       M->stream));
  if (K32)
    CK(cudaMemcpyAsync(K32, M->d_K32, (size_t)M->n_blocks * 36 * 4, cudaMemcpyDefault,
                       M->stream));
  CK(cudaStreamSynchronize(M->stream));
  return leave(M);
}

sso_status sso_model_get_load(sso_model* M, double* f) {
  if (!M || !f) return fail(SSO_ERR_INVALID, "NULL argument");
  if (!M->assembled) return fail(SSO_ERR_INVALID, "loads not assembled yet");
  sso_status st = enter(M);
  if (st != SSO_OK) return st;
  CK(cudaMemcpyAsync(f, M->d_f, 6 * (size_t)M->n_nodes * 8, cudaMemcpyDefault, M->stream));
  CK(cudaStreamSynchronize(M->stream));
  return leave(M);
}

}  // extern "C"

namespace {
// Batches of at least this many systems run their CG as concurrent parts.
constexpr int kSplitMin = 32;
constexpr int kTilesPerPart = 18000;
// Kernel A of a batch launches this many times the CTAs that fit at once,
// each with a shorter range of tiles, so that the block scheduler evens out
// ranges that cost more: an FP64 residual pass reads K64 through global
// memory at the FP64 rate, and a system's tiles are contiguous.  Measured on
// 256 designs of the 64 x 64 shell (designs/s over the timed steps, kernel A's
// fraction of HBM over the profiled step): 1x 62.5 / 0.75, 2x 64.3 / 0.79,
// 4x 64.8 / 0.82, 8x 64.0 / 0.83 (4x and 8x in 2 parts).
constexpr int kBatchGridMult = 4;
sso_status make_parts(sso_batch* B, int k);

sso_status create_batch(sso_model* const* models, int32_t n, sso_batch** out, bool split) {
  if (!out) return fail(SSO_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!models || n <= 0) return fail(SSO_ERR_INVALID, "need at least one model");
  for (int s = 0; s < n; ++s)
    if (!models[s]) return fail(SSO_ERR_INVALID, "NULL model in batch");
  for (int s = 1; s < n; ++s)
    if (models[s]->device != models[0]->device)
      return fail(SSO_ERR_INVALID, "models of a batch must be on one device");
  sso_batch* B = new sso_batch();
  B->models.assign(models, models + n);
  B->grid_a_mult = kBatchGridMult;
  B->stream = models[0]->stream;
  B->n_sys = n;
  std::vector<TileDesc> tiles;
  B->h_sys.resize(n);
  for (int s = 0; s < n; ++s) {
    sso_model* M = models[s];
    SysDesc& D = B->h_sys[s];
    D.n_nodes = M->n_nodes;
    D.tile0 = (int)tiles.size();
    D.n_tiles = M->n_tiles;
    D.precond = SSO_BLOCK_JACOBI;
    D.row_ptr = M->d_row_ptr;
    D.col = M->d_col;
    D.hslot = M->d_hslot;
    D.K32 = M->d_K32;
    D.K64 = M->d_K64;
    D.M32 = M->d_M32;
    D.M64 = M->d_M64;
    D.b = M->d_f;
    D.x = M->d_u;
    D.dx = M->d_dx;
    D.r64 = M->d_r64;
    D.r = M->d_r;
    D.z = M->d_z;
    D.p0 = M->d_p0;
    D.p1 = M->d_p1;
    D.q = M->d_q;
    D.part_a = M->d_part_a;
    D.part_b = M->d_part_b;
    D.n_chunks = n_chunks_of(M);
    D.chunk_cnt = M->d_chunk_cnt;
    D.chunk_part = M->d_chunk_part;
    D.n_agg = M->n_agg;
    D.agg_ptr = M->d_agg_ptr;
    D.agg_nodes = M->d_agg_nodes;
    D.agg_of = M->d_agg_of;
    D.fixed = M->d_fixed;
    D.node_rf = M->d_node_rf;
    D.Aci = M->d_Aci;
    D.w = M->d_cw;
    D.y = M->d_cy;
    D.cdot = M->d_cdot;
    D.zb = M->d_zb;
    D.klo = reinterpret_cast<float*>(M->d_ke);
    for (int k = 0; k < M->n_tiles; ++k) tiles.push_back(make_tile(M, s, k));
  }
  B->n_tiles = (int)tiles.size();
  B->h_tiles = tiles;
  B->h_tile0.resize(n);
  for (int s = 0; s < n; ++s) B->h_tile0[s] = B->h_sys[s].tile0;
  std::vector<AggRef> aggs;
  std::vector<int> csys(n);
  for (int s = 0; s < n; ++s) {
    csys[s] = s;
    for (int g = 0; g < models[s]->n_agg; ++g) aggs.push_back({s, g});
  }
  B->n_aggs = (int)aggs.size();
  Carver c(nullptr);
  c.take<SysDesc>(n);
  c.take<SysScalars>(n);
  c.take<TileDesc>(tiles.size());
  c.take<int>(1);
  c.take<int>(2);
  c.take<double>(n);
  c.take<AggRef>(std::max<size_t>(aggs.size(), 1));
  c.take<int>(n);
  c.take<int>(2);
  c.take<SetupJob>(n);
  c.take<int>(n);
  const size_t bytes = align_up(c.off, 256);
  std::vector<SetupJob> jobs(n);
  for (int s = 0; s < n; ++s) {
    jobs[s] = make_setup_job(models[s]);
    B->extent.add(models[s]);
  }
  if (n > 65535) {
    delete B;
    return fail(SSO_ERR_INVALID, "a batch holds at most 65535 models");
  }
  cudaError_t e = cudaMalloc(&B->arena, bytes);
  if (e != cudaSuccess) {
    delete B;
    return cuda_fail(e, "cudaMalloc(batch arena)");
  }
  Carver d(B->arena);
  B->d_sys = d.take<SysDesc>(n);
  B->d_sc = d.take<SysScalars>(n);
  B->d_tiles = d.take<TileDesc>(tiles.size());
  B->d_n_tiles = d.take<int>(1);
  B->d_n_active = d.take<int>(2);
  B->d_dots = d.take<double>(n);
  B->d_aggs = d.take<AggRef>(std::max<size_t>(aggs.size(), 1));
  B->d_csys = d.take<int>(n);
  B->d_ccount = d.take<int>(2);
  B->d_jobs = d.take<SetupJob>(n);
  B->d_list = d.take<int>(n);
  B->grid_restrict = (B->n_aggs + 7) / 8;  // one warp per (system, aggregate)
  B->grid_csolve = n * COARSE_ROW_BLOCKS;  // one CTA per work item
  const int ccount[2] = {B->n_aggs, n};
  for (int s = 0; s < n; ++s) B->h_sys[s].sc = B->d_sc + s;
  e = cudaMallocHost(&B->h_sc, sizeof(SysScalars) * n);
  if (e == cudaSuccess) e = cudaMallocHost(&B->h_flag, 4 * sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemsetAsync(B->arena, 0, bytes, B->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->d_tiles, tiles.data(), tiles.size() * sizeof(TileDesc),
                        cudaMemcpyHostToDevice, B->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->d_n_tiles, &B->n_tiles, sizeof(int), cudaMemcpyHostToDevice,
                        B->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->d_sys, B->h_sys.data(), sizeof(SysDesc) * n, cudaMemcpyHostToDevice,
                        B->stream);
  if (e == cudaSuccess && !aggs.empty())
    e = cudaMemcpyAsync(B->d_aggs, aggs.data(), aggs.size() * sizeof(AggRef),
                        cudaMemcpyHostToDevice, B->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->d_csys, csys.data(), csys.size() * sizeof(int), cudaMemcpyHostToDevice,
                        B->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->d_ccount, ccount, sizeof(ccount), cudaMemcpyHostToDevice, B->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->d_jobs, jobs.data(), sizeof(SetupJob) * n, cudaMemcpyHostToDevice,
                        B->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
  if (e != cudaSuccess) {
    sso_batch_destroy(B);
    return cuda_fail(e, "batch set-up");
  }
  if (split && n >= kSplitMin) {
    // about 18,000 tiles per part, 2 to 4 parts (measured on 64 x 64 shells
    // with kernel A at 4x: 256 designs 64.8 designs/s in 2 parts, 63.5 in 3,
    // 59.1 whole)
    const int k = std::min(4, std::max(2, (B->n_tiles + kTilesPerPart / 2) / kTilesPerPart));
    sso_status st = make_parts(B, k);
    if (st != SSO_OK) {
      sso_batch_destroy(B);
      return st;
    }
  }
  *out = B;
  return SSO_OK;
}

// Splits B's CG into k concurrent parts of contiguous systems (k <= 1: none).
sso_status make_parts(sso_batch* B, int k) {
  for (sso_batch* P : B->parts) sso_batch_destroy(P);
  for (cudaEvent_t e : B->part_ev) cudaEventDestroy(e);
  B->parts.clear();
  B->part_ev.clear();
  B->part0.clear();
  if (k <= 1) return SSO_OK;
  for (int i = 0; i <= k; ++i) B->part0.push_back((int)((long long)B->n_sys * i / k));
  for (int i = 0; i < k; ++i) {
    sso_batch* P = nullptr;
    sso_status st = create_batch(B->models.data() + B->part0[i], B->part0[i + 1] - B->part0[i],
                                 &P, false);
    if (st != SSO_OK) return st;
    B->parts.push_back(P);
    P->profiling = B->profiling;
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "batch part event");
    B->part_ev.push_back(ev);
  }
  return SSO_OK;
}
}  // namespace

extern "C" {

sso_status sso_batch_create(sso_model* const* models, int32_t n, sso_batch** out) {
  return create_batch(models, n, out, true);
}

sso_status sso_batch_set_parts(sso_batch* B, int32_t parts) {
  if (!B) return fail(SSO_ERR_INVALID, "batch is NULL");
  if (parts < 1 || parts > 16 || parts > B->n_sys)
    return fail(SSO_ERR_INVALID, "parts must be in [1, min(16, models)]");
  CK(cudaStreamSynchronize(B->stream));
  for (sso_batch* P : B->parts) CK(cudaStreamSynchronize(P->stream));
  return make_parts(B, parts);
}


void sso_batch_destroy(sso_batch* B) {
  if (!B) return;
  for (sso_batch* P : B->parts) sso_batch_destroy(P);
  for (cudaEvent_t e : B->part_ev) cudaEventDestroy(e);
  if (B->stream) cudaStreamSynchronize(B->stream);
  for (int k = 0; k < 3; ++k)
    if (B->exec[k]) cudaGraphExecDestroy(B->exec[k]);
  for (cudaEvent_t e : B->pev) cudaEventDestroy(e);
  for (cudaEvent_t e : B->sev) cudaEventDestroy(e);
  for (cudaStream_t st : B->aux) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (cudaEvent_t e : B->aux_ev) cudaEventDestroy(e);
  if (B->ev_fork) cudaEventDestroy(B->ev_fork);
  if (B->arena) cudaFree(B->arena);
  if (B->h_sc) cudaFreeHost(B->h_sc);
  if (B->h_flag) cudaFreeHost(B->h_flag);
  if (B->ev) cudaEventDestroy(B->ev);
  delete B;
}

sso_status sso_batch_set_profiling(sso_batch* B, int32_t enable) {
  if (!B) return fail(SSO_ERR_INVALID, "batch is NULL");
  for (sso_batch* P : B->parts) sso_batch_set_profiling(P, enable);
  B->profiling = enable ? 1 : 0;
  B->prof_ms_a = B->prof_ms_b = 0.0;
  B->prof_launches = 0;
  B->prof_ms_el = B->prof_ms_asm = B->prof_ms_pre = B->prof_ms_adj = B->prof_ms_setup = 0.0;
  B->prof_setups = B->prof_grads = 0;
  return SSO_OK;
}

sso_status sso_batch_setup_times(const sso_batch* B, double* ms_elements, double* ms_assembly,
                                 double* ms_precond, double* ms_adjoint, double* ms_setup_wall,
                                 int64_t* setups, int64_t* gradients) {
  if (!B) return fail(SSO_ERR_INVALID, "batch is NULL");
  if (ms_setup_wall) *ms_setup_wall = B->prof_ms_setup;
  if (ms_elements) *ms_elements = B->prof_ms_el;
  if (ms_assembly) *ms_assembly = B->prof_ms_asm;
  if (ms_precond) *ms_precond = B->prof_ms_pre;
  if (ms_adjoint) *ms_adjoint = B->prof_ms_adj;
  if (setups) *setups = B->prof_setups;
  if (gradients) *gradients = B->prof_grads;
  return SSO_OK;
}

sso_status sso_batch_kernel_times(const sso_batch* B, double* ms_a, double* ms_b,
                                  int64_t* launches) {
  if (!B) return fail(SSO_ERR_INVALID, "batch is NULL");
  double a = B->prof_ms_a, b = B->prof_ms_b;
  long long n = B->prof_launches;
  for (const sso_batch* P : B->parts) {
    a += P->prof_ms_a;
    b += P->prof_ms_b;
    n += P->prof_launches;
  }
  if (ms_a) *ms_a = a;
  if (ms_b) *ms_b = b;
  if (launches) *launches = n;
  return SSO_OK;
}

sso_status sso_batch_solve(sso_batch* B, const sso_options* opts, sso_stats* stats) {
  if (!B) return fail(SSO_ERR_INVALID, "batch is NULL");
  sso_status st = check_options(opts);
  if (st != SSO_OK) return st;
  sso_model* M0 = B->models[0];
  st = enter(M0);
  if (st != SSO_OK) return st;
  // other models' callers' streams also order before this work
  for (int s = 1; s < B->n_sys; ++s) {
    sso_model* M = B->models[s];
    CK(cudaEventRecord(M->ev_in, M->user_stream));
    CK(cudaStreamWaitEvent(B->stream, M->ev_in, 0));
  }
  const bool prof = B->profiling != 0;
  // set-up: one launch per stage for the whole batch (events: before the
  // element kernels, after them, after assembly, after the preconditioner and
  // loads, after the two-level coarse set-ups)
  if (prof && (st = ensure_setup_events(B, 5)) != SSO_OK) return st;
  st = setup_stages(B->d_jobs, B->n_sys, B->extent, opts->precond, B->stream,
                    prof ? B->sev.data() : nullptr);
  if (st != SSO_OK) return st;
  if (opts->precond == SSO_TWO_LEVEL) {
    // coarse spaces per model, on a pool of streams (they are independent)
    if ((st = fork_aux(B)) != SSO_OK) return st;
    for (int s = 0; s < B->n_sys; ++s)
      if ((st = setup_coarse(B->models[s], B->aux[s % B->aux.size()])) != SSO_OK) return st;
    if ((st = join_aux(B)) != SSO_OK) return st;
  }
  if (prof) CK(cudaEventRecord(B->sev[4], B->stream));
  for (int s = 0; s < B->n_sys; ++s) mark_assembled(B->models[s], opts->precond);
  std::vector<char> active(B->n_sys, 1);
  bool deferred = false;
  sso_status run = run_cg(B, opts, false, active, stats, &deferred);
  if (run == SSO_ERR_CUDA || run == SSO_ERR_OOM) return run;
  // compliance C = f^T u, and the preconditioner check
  CL(launch_dot(B->n_sys, B->d_sys, B->d_dots, B->stream), 1);
  for (int s = 0; s < B->n_sys; ++s) {
    sso_model* M = B->models[s];
    CK(cudaMemcpyAsync(M->d_C, B->d_dots + s, sizeof(double), cudaMemcpyDeviceToDevice,
                       B->stream));
  }
  std::vector<int> errs(B->n_sys, 0);
  for (int s = 0; s < B->n_sys; ++s)
    CK(cudaMemcpyAsync(&errs[s], B->models[s]->d_err, sizeof(int), cudaMemcpyDeviceToHost,
                       B->stream));
  CK(cudaStreamSynchronize(B->stream));
  if (deferred) run = finish_run(B, active, stats);
  if (prof) {
    const cudaEvent_t* e = B->sev.data();
    B->prof_ms_el += elapsed_ms(e[0], e[1]);
    B->prof_ms_asm += elapsed_ms(e[1], e[2]);
    B->prof_ms_pre += elapsed_ms(e[2], e[3]);
    B->prof_ms_setup += elapsed_ms(e[0], e[4]);
    B->prof_setups += B->n_sys;
  }
  for (int s = 0; s < B->n_sys; ++s) {
    sso_model* M = B->models[s];
    M->solved = true;
    M->last_opts = *opts;
    if (errs[s] >= 2) {
      if (stats) stats[s].status = SSO_ERR_CUDA;
      run = fail(SSO_ERR_CUDA, "assembly gave up waiting for a bulk copy (device fault?)");
    } else if (errs[s]) {
      if (stats) stats[s].status = SSO_ERR_SINGULAR;
      if (run == SSO_OK) run = fail(SSO_ERR_SINGULAR, "a diagonal block of K is not positive "
                                                      "definite (unsupported mechanism?)");
    }
  }
  for (int s = 0; s < B->n_sys; ++s) {
    sso_model* M = B->models[s];
    CK(cudaEventRecord(M->ev_out, B->stream));
    CK(cudaStreamWaitEvent(M->user_stream, M->ev_out, 0));
  }
  return run;
}

sso_status sso_batch_gradient(sso_batch* B, const double* w, const double* const* g,
                              sso_stats* stats) {
  if (!B) return fail(SSO_ERR_INVALID, "batch is NULL");
  for (int s = 0; s < B->n_sys; ++s)
    if (!B->models[s]->solved || !B->models[s]->assembled)
      return fail(SSO_ERR_INVALID, "gradient needs a current solve of every model");
  sso_model* M0 = B->models[0];
  sso_status st = enter(M0);
  if (st != SSO_OK) return st;
  for (int s = 1; s < B->n_sys; ++s) {
    sso_model* M = B->models[s];
    CK(cudaEventRecord(M->ev_in, M->user_stream));
    CK(cudaStreamWaitEvent(B->stream, M->ev_in, 0));
  }
  std::vector<char> active(B->n_sys, 0);
  bool any = false;
  for (int s = 0; s < B->n_sys; ++s) {
    sso_model* M = B->models[s];
    const double ws = w ? w[s] : 1.0;
    const double* gs = g ? g[s] : nullptr;
    const int ndof = 6 * M->n_nodes;
    if (gs) {
      // rhs = w f + g, zero on fixed DOFs (g may be host memory)
      CK(cudaMemcpyAsync(M->d_rhs, gs, (size_t)ndof * 8, cudaMemcpyDefault, B->stream));
      CL(launch_axpby(ndof, ws, M->d_f, M->d_rhs, M->d_fixed, M->d_rhs, B->stream), 1);
      active[s] = 1;
      any = true;
    }
  }
  sso_status run = SSO_OK;
  if (any) {
    // the adjoint solve reuses K, the preconditioner and the last options
    sso_options o = B->models[0]->last_opts;
    run = run_cg(B, &o, true, active, stats);
    if (run == SSO_ERR_CUDA || run == SSO_ERR_OOM) return run;
  }
  const bool prof = B->profiling != 0;
  const size_t e0 = 5;  // after the solve's set-up events
  if (prof) {
    if ((st = ensure_setup_events(B, e0 + 2)) != SSO_OK) return st;
    CK(cudaEventRecord(B->sev[e0], B->stream));
  }
  // models' contractions on a pool of streams (one model: its own stream)
  const bool pool = B->n_sys > 1;
  if (pool && (st = fork_aux(B)) != SSO_OK) return st;
  for (int s = 0; s < B->n_sys; ++s) {
    sso_model* M = B->models[s];
    cudaStream_t as = pool ? B->aux[s % B->aux.size()] : B->stream;
    const double ws = w ? w[s] : 1.0;
    const bool has_g = active[s] != 0;
    const double* lam = has_g ? M->d_lam : M->d_u;
    const double lam_scale = has_g ? 1.0 : ws;
    if (!has_g)
      CL(launch_axpby(6 * M->n_nodes, ws, M->d_u, nullptr, M->d_fixed, M->d_lam, as), 1);
    CL(launch_beam_adjoint(M->n_beams, M->d_xyz, M->d_beam_conn, M->d_beam_props, M->d_u, lam,
                           lam_scale, M->d_gslot, as),
       M->n_beams > 0);
    CL(launch_quad_adjoint(M->n_quads, M->d_xyz, M->d_quad_conn, M->d_quad_props, M->pressure,
                           M->gamma, M->d_u, lam, lam_scale, ws,
                           M->d_gslot + 2 * (size_t)M->n_beams, M->d_dt, as,
                           M->d_rho, M->penal, M->has_topology ? M->d_drho : nullptr),
       M->n_quads > 0);
    CL(launch_node_gather(M->n_nodes, M->d_nptr, M->d_nsrc, 2 * M->n_beams, nullptr, M->d_gslot,
                          nullptr, M->d_fixed, nullptr, M->d_dz, as),
       1);
    if (stats && !has_g) {
      stats[s].status = SSO_OK;
      stats[s].iterations = 0;
      stats[s].sweeps = 0;
      stats[s].rel_residual = 0.0;
      stats[s].ms = 0.0;
    }
  }
  if (pool && (st = join_aux(B)) != SSO_OK) return st;
  // The contractions stay queued: the caller's streams wait on them through
  // ev_out below, and sso_model_get synchronises; only a
  // profiled call waits here, to read its events.
  if (prof) {
    CK(cudaEventRecord(B->sev[e0 + 1], B->stream));
    CK(cudaStreamSynchronize(B->stream));
    B->prof_ms_adj += elapsed_ms(B->sev[e0], B->sev[e0 + 1]);
    B->prof_grads += 1;
  }
  for (int s = 0; s < B->n_sys; ++s) {
    sso_model* M = B->models[s];
    CK(cudaEventRecord(M->ev_out, B->stream));
    CK(cudaStreamWaitEvent(M->user_stream, M->ev_out, 0));
  }
  return run;
}

}  // extern "C"

// ===========================================================================
// Serving: continuous batching of design evaluations (solve + adjoint z / t
// gradient of J = w C).  A server owns a batch sized for its capacity
// (max_systems systems, max_tiles tiles) whose system table and tile list
// are rewritten between CUDA-graph launches of the CG engine: finished
// systems leave, newly admitted ones join, without waiting for the others.
// Admission is by free slot, free tiles and an HBM budget; a request's model
// (its pattern, K, preconditioner and solver state) stays resident until its
// result has been produced.

namespace {

// A server's device memory: one allocation of its HBM budget, carved into
// model arenas first-fit, with freed ranges merged with their neighbours.
struct DevPool {
  unsigned char* base = nullptr;
  size_t size = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  void* alloc(size_t n) {
    n = align_up(n, 256);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      const size_t off = it->first, rem = it->second - n;
      free_.erase(it);
      if (rem) free_[off + n] = rem;
      return base + off;
    }
    return nullptr;
  }
  void release(void* p, size_t n) {
    size_t off = (size_t)(static_cast<unsigned char*>(p) - base);
    n = align_up(n, 256);
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + n == next->first) {
      n += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += n;
        return;
      }
    }
    free_[off] = n;
  }
};

// Pinned staging for model uploads: images are copied into a ring of pinned
// host memory and uploaded from there asynchronously; a region is reused
// once the event recorded after its upload has completed.
struct PinnedRing {
  unsigned char* base = nullptr;
  size_t size = 0, head = 0;
  struct Use {
    size_t begin, end;
    cudaEvent_t ev;
  };
  std::deque<Use> busy;
  std::vector<cudaEvent_t> spare;
  // A region of n bytes (16-byte aligned start), or nullptr if n exceeds the
  // ring.  Regions are handed out in order, so the ones in use span
  // [oldest begin, head) circularly; the oldest are waited for until n fits.
  unsigned char* take(size_t n, cudaError_t& err) {
    err = cudaSuccess;
    if (n > size) return nullptr;
    size_t a = 0;
    for (;;) {
      if (busy.empty()) {
        a = 0;
        break;
      }
      const size_t tail = busy.front().begin, h = align_up(head, 16);
      if (h > tail) {  // in use: [tail, h)
        if (h + n <= size) {
          a = h;
          break;
        }
        if (n <= tail) {
          a = 0;
          break;
        }
      } else if (h + n <= tail) {  // in use: [tail, size) and [0, h)
        a = h;
        break;
      }
      err = cudaEventSynchronize(busy.front().ev);
      if (err != cudaSuccess) return nullptr;
      spare.push_back(busy.front().ev);
      busy.pop_front();
    }
    head = a + n;
    return base + a;
  }
  // Marks [p, p + n) busy until stream s passes this point.
  cudaError_t mark(unsigned char* p, size_t n, cudaStream_t s) {
    cudaEvent_t ev;
    if (!spare.empty()) {
      ev = spare.back();
      spare.pop_back();
    } else {
      cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e != cudaSuccess) return e;
    }
    busy.push_back({(size_t)(p - base), (size_t)(p - base) + n, ev});
    return cudaEventRecord(ev, s);
  }
  void release_all() {
    for (auto& u : busy) cudaEventDestroy(u.ev);
    for (auto ev : spare) cudaEventDestroy(ev);
    busy.clear();
    spare.clear();
    if (base) cudaFreeHost(base);
    base = nullptr;
  }
};

struct ServerReq {
  uint64_t ticket = 0;
  std::unique_ptr<ModelPrep> prep;  // host half of the model, built by a worker thread
  bool prep_done = false;           // guarded by the server's mutex
  sso_status prep_status = SSO_OK;
  double w = 1.0;
  double t_submit = 0.0, t_done = 0.0;  // ms since the server was created
  int slot = -1;
  int phase = 0;  // 0 queued, 1 setting up, 2 in CG, 3 result ready
  sso_model* M = nullptr;
  size_t bytes = 0;
  cudaEvent_t ev_setup = nullptr;
  sso_stats stats{};
  std::vector<double> u, dz, dt;
  double C = 0.0;
};

// A batch with room for max_sys systems and max_tiles tiles and no models,
// running on `stream`.
sso_status batch_with_capacity(cudaStream_t stream, int max_sys, int max_tiles,
                               sso_batch** out) {
  sso_batch* B = new sso_batch();
  B->stream = stream;
  B->n_sys = max_sys;
  B->n_tiles = max_tiles;  // sizes the graph's grids; the live count is on the device
  B->grid_a_mult = 8;
  B->h_sys.assign(max_sys, SysDesc{});
  Carver c(nullptr);
  c.take<SysDesc>(max_sys);
  c.take<SysScalars>(max_sys);
  c.take<TileDesc>(max_tiles);
  c.take<int>(1);
  c.take<int>(2);
  c.take<double>(max_sys);
  c.take<AggRef>((size_t)max_sys * COARSE_MAX_AGG);
  c.take<int>(max_sys);
  c.take<int>(2);
  const size_t bytes = align_up(c.off, 256);
  cudaError_t e = cudaMalloc(&B->arena, bytes);
  if (e != cudaSuccess) {
    delete B;
    return cuda_fail(e, "cudaMalloc(server tables)");
  }
  Carver d(B->arena);
  B->d_sys = d.take<SysDesc>(max_sys);
  B->d_sc = d.take<SysScalars>(max_sys);
  B->d_tiles = d.take<TileDesc>(max_tiles);
  B->d_n_tiles = d.take<int>(1);
  B->d_n_active = d.take<int>(2);
  B->d_dots = d.take<double>(max_sys);
  // two-level lists of the running systems (lengths on the device, rewritten
  // with the tile list); the coarse kernels loop over them on a fixed grid
  B->d_aggs = d.take<AggRef>((size_t)max_sys * COARSE_MAX_AGG);
  B->d_csys = d.take<int>(max_sys);
  B->d_ccount = d.take<int>(2);
  B->n_aggs = max_sys * COARSE_MAX_AGG;
  {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    sms = std::max(sms, 1);
    B->grid_restrict = std::min((B->n_aggs + 7) / 8, 8 * sms);
    B->grid_csolve = std::min(max_sys * COARSE_ROW_BLOCKS, 4 * sms);
  }
  for (int s = 0; s < max_sys; ++s) B->h_sys[s].sc = B->d_sc + s;
  e = cudaMallocHost(&B->h_sc, sizeof(SysScalars) * max_sys);
  if (e == cudaSuccess) e = cudaMallocHost(&B->h_flag, 4 * sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemsetAsync(B->arena, 0, bytes, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    sso_batch_destroy(B);
    return cuda_fail(e, "server tables");
  }
  *out = B;
  return SSO_OK;
}

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct sso_server {
  sso_options opts;
  size_t budget = 0, used = 0;
  int max_sys = 0, max_tiles = 0;
  cudaStream_t cg_stream = nullptr;
  // set-up streams, taken in turn by admitted requests so that their set-up
  // kernels (element matrices, assembly, preconditioner, coarse space)
  // overlap one another
  std::vector<cudaStream_t> setup_streams;
  int next_setup = 0;
  sso_batch* B = nullptr;
  DevPool pool;                // model arenas
  PinnedRing ring;             // upload staging
  SysScalars* h_up = nullptr;  // pinned upload staging, one per slot
  std::deque<ServerReq*> queue;
  std::unordered_map<uint64_t, ServerReq*> reqs;
  std::vector<ServerReq*> slot_req;
  std::vector<int> running, pending;
  std::vector<std::vector<TileDesc>> slot_tiles;  // tile descriptors of each slot's model
  int tiles_used = 0;  // tiles of running + pending systems
  uint64_t next_ticket = 1;
  std::chrono::steady_clock::time_point t0;
  bool dirty = false;
  // host time per phase of sso_server_step (ms): admission (model build and
  // set-up enqueue), table upload, wait for the CG graph, harvest
  double ms_admit = 0.0, ms_upload = 0.0, ms_wait = 0.0, ms_harvest = 0.0;
  // parts of the admission time: waiting for a worker's preparation, arena
  // allocation and upload, set-up kernel launches
  double ms_admit_prep = 0.0, ms_admit_device = 0.0, ms_admit_setup = 0.0;
  long long steps = 0, graph_launches = 0;
  std::vector<uint64_t> completed;  // tickets finished since the last sso_server_completed
  // worker threads preparing submitted requests (scatter map, tiles, arena image)
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<ServerReq*> prep_queue;
  bool stop = false;
  // Lanes (sso_server_create_lanes): this server only routes requests to
  // independent lane servers, each with its share of the budget, slots and
  // tiles, and steps them at once, one host thread each, so that each lane's
  // CG launches fill the others' ramps and tails.  Tickets are this server's
  // own, mapped to (lane, the lane's ticket).
  std::vector<sso_server*> lanes;
  std::unordered_map<uint64_t, std::pair<int, uint64_t>> lane_of;
  std::vector<std::unordered_map<uint64_t, uint64_t>> global_of;
  std::vector<long long> lane_nodes;  // nodes of each lane's unfinished requests
  std::unordered_map<uint64_t, int> ticket_nodes;
  // one helper thread per lane after the first, woken for every step
  std::vector<std::thread> lane_threads;
  std::mutex lane_mu;
  std::condition_variable lane_cv;
  long long lane_round = 0;
  int lane_pending = 0;
  bool lane_stop = false;
  std::vector<sso_status> lane_status;
  std::vector<std::string> lane_msg;
  std::vector<int32_t> lane_running, lane_waiting;
};

namespace {
constexpr int kIdleAdmit = 16;  // requests admitted per step while no CG graph runs
constexpr int kSetupStreams = 8;  // set-up streams of a server
constexpr size_t kRingBytes = 64u << 20;  // pinned upload staging of a server

void prep_worker(sso_server* S) {
  for (;;) {
    ServerReq* R;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [S] { return S->stop || !S->prep_queue.empty(); });
      if (S->stop) return;
      R = S->prep_queue.front();
      S->prep_queue.pop_front();
    }
    const sso_status st = prepare_model(*R->prep);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      R->prep_status = st;
      R->prep_done = true;
    }
    S->cv_done.notify_all();
  }
}
}  // namespace

namespace {

// With SSO_DEBUG_SYNC set: synchronise s and name the phase of any CUDA error.
sso_status debug_check(cudaStream_t s, const char* phase) {
  if (!debug_sync()) return SSO_OK;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, phase);
  return SSO_OK;
}

// Tile list and system table of the running systems, in slot order.
sso_status server_upload_tables(sso_server* S, std::vector<std::vector<TileDesc>>& tile_cache) {
  sso_batch* B = S->B;
  std::sort(S->running.begin(), S->running.end());
  // every index the kernels will follow, checked before it reaches the device
  for (int slot : S->running) {
    const ServerReq* R = (slot >= 0 && slot < S->max_sys) ? S->slot_req[slot] : nullptr;
    const sso_model* M = R ? R->M : nullptr;
    const SysDesc& D = B->h_sys[slot];
    bool ok = M && (int)tile_cache[slot].size() == M->n_tiles && D.n_nodes == M->n_nodes &&
              D.n_tiles == M->n_tiles && D.x == M->d_u && D.b == M->d_f && D.K32 == M->d_K32 &&
              D.col == M->d_col && D.row_ptr == M->d_row_ptr && D.sc == B->d_sc + slot;
    for (const TileDesc& td : tile_cache[slot])
      ok = ok && td.sys == slot && td.node0 >= 0 && td.nn > 0 && td.node0 + td.nn <= M->n_nodes &&
           td.j0 == M->h_row_ptr[td.node0] &&
           td.j0 + td.nblk == M->h_row_ptr[td.node0 + td.nn];
    if (!ok) return fail(SSO_ERR_INVALID, "server tables inconsistent (internal error)");
  }
  std::vector<TileDesc> tiles;
  tiles.reserve(S->tiles_used);
  for (int slot : S->running) {
    B->h_sys[slot].tile0 = (int)tiles.size();
    tiles.insert(tiles.end(), tile_cache[slot].begin(), tile_cache[slot].end());
  }
  const int n = (int)tiles.size();
  if (n > 0)
    CK(cudaMemcpyAsync(B->d_tiles, tiles.data(), n * sizeof(TileDesc), cudaMemcpyHostToDevice,
                       B->stream));
  CK(cudaMemcpyAsync(B->d_n_tiles, &n, sizeof(int), cudaMemcpyHostToDevice, B->stream));
  std::vector<AggRef> aggs;
  int ccount[2] = {0, 0};
  if (S->opts.precond == SSO_TWO_LEVEL) {
    for (int slot : S->running)
      for (int g = 0; g < S->slot_req[slot]->M->n_agg; ++g) aggs.push_back({slot, g});
    ccount[0] = (int)aggs.size();
    ccount[1] = (int)S->running.size();
    if (!aggs.empty())
      CK(cudaMemcpyAsync(B->d_aggs, aggs.data(), aggs.size() * sizeof(AggRef),
                         cudaMemcpyHostToDevice, B->stream));
    if (!S->running.empty())
      CK(cudaMemcpyAsync(B->d_csys, S->running.data(), S->running.size() * sizeof(int),
                         cudaMemcpyHostToDevice, B->stream));
  }
  CK(cudaMemcpyAsync(B->d_ccount, ccount, sizeof(ccount), cudaMemcpyHostToDevice, B->stream));
  CK(cudaMemcpyAsync(B->d_sys, B->h_sys.data(), sizeof(SysDesc) * S->max_sys,
                     cudaMemcpyHostToDevice, B->stream));
  CK(cudaStreamSynchronize(B->stream));  // the host vectors above are temporaries
  S->dirty = false;
  return SSO_OK;
}

void fill_sysdesc(SysDesc& D, sso_model* M, int precond) {
  D.n_nodes = M->n_nodes;
  D.n_tiles = M->n_tiles;
  D.precond = precond;
  D.row_ptr = M->d_row_ptr;
  D.col = M->d_col;
  D.hslot = M->d_hslot;
  D.K32 = M->d_K32;
  D.K64 = M->d_K64;
  D.M32 = M->d_M32;
  D.M64 = M->d_M64;
  D.b = M->d_f;
  D.x = M->d_u;
  D.dx = M->d_dx;
  D.r64 = M->d_r64;
  D.r = M->d_r;
  D.z = M->d_z;
  D.p0 = M->d_p0;
  D.p1 = M->d_p1;
  D.q = M->d_q;
  D.part_a = M->d_part_a;
  D.part_b = M->d_part_b;
  D.n_chunks = n_chunks_of(M);
  D.chunk_cnt = M->d_chunk_cnt;
  D.chunk_part = M->d_chunk_part;
  D.n_agg = M->n_agg;
  D.agg_ptr = M->d_agg_ptr;
  D.agg_nodes = M->d_agg_nodes;
  D.agg_of = M->d_agg_of;
  D.fixed = M->d_fixed;
  D.node_rf = M->d_node_rf;
  D.Aci = M->d_Aci;
  D.w = M->d_cw;
  D.y = M->d_cy;
  D.cdot = M->d_cdot;
  D.zb = M->d_zb;
  D.klo = reinterpret_cast<float*>(M->d_ke);
}

void init_scalars(SysScalars& S, const sso_options& o) {
  std::memset(&S, 0, sizeof(S));
  const double inner = o.precision == SSO_FP64 ? 0.0 : o.inner_rtol;
  S.state = ST_INIT;
  S.status = SSO_ERR_NOT_CONVERGED;
  S.rtol2 = o.rtol * o.rtol;
  S.inner_rtol2 = inner * inner;
  S.max_iter = o.max_iter;
  S.max_sweeps = o.max_sweeps;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {
// A lane's helper thread: one sso_server_step of lane k per round.
void lane_loop(sso_server* S, int k) {
  long long seen = 0;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(S->lane_mu);
      S->lane_cv.wait(lk, [&] { return S->lane_stop || S->lane_round != seen; });
      if (S->lane_stop) return;
      seen = S->lane_round;
    }
    int32_t r = 0, w = 0;
    const sso_status st = sso_server_step(S->lanes[k], &r, &w);
    const std::string msg = st != SSO_OK ? g_last_error : std::string();
    {
      std::lock_guard<std::mutex> lk(S->lane_mu);
      S->lane_status[k] = st;
      S->lane_msg[k] = msg;
      S->lane_running[k] = r;
      S->lane_waiting[k] = w;
      --S->lane_pending;
    }
    S->lane_cv.notify_all();
  }
}

void stop_lanes(sso_server* S) {
  {
    std::lock_guard<std::mutex> lk(S->lane_mu);
    S->lane_stop = true;
  }
  S->lane_cv.notify_all();
  for (std::thread& t : S->lane_threads) t.join();
  S->lane_threads.clear();
  for (sso_server* L : S->lanes) sso_server_destroy(L);
  S->lanes.clear();
}

sso_status router_step(sso_server* S, int32_t* n_running, int32_t* n_waiting) {
  const int nl = (int)S->lanes.size();
  {
    std::lock_guard<std::mutex> lk(S->lane_mu);
    ++S->lane_round;
    S->lane_pending = nl - 1;
  }
  S->lane_cv.notify_all();
  int32_t r = 0, w = 0;
  S->lane_status[0] = sso_server_step(S->lanes[0], &r, &w);
  if (S->lane_status[0] != SSO_OK) S->lane_msg[0] = g_last_error;
  S->lane_running[0] = r;
  S->lane_waiting[0] = w;
  {
    std::unique_lock<std::mutex> lk(S->lane_mu);
    S->lane_cv.wait(lk, [S] { return S->lane_pending == 0; });
  }
  ++S->steps;
  int32_t tr = 0, tw = 0;
  int bad = -1;
  for (int k = 0; k < nl; ++k) {
    tr += S->lane_running[k];
    tw += S->lane_waiting[k];
    if (S->lane_status[k] != SSO_OK && (bad < 0 || S->lane_status[k] == SSO_ERR_CUDA)) bad = k;
  }
  if (n_running) *n_running = tr;
  if (n_waiting) *n_waiting = tw;
  if (bad < 0) return SSO_OK;
  g_last_error = S->lane_msg[bad];
  return S->lane_status[bad];
}
}  // namespace

extern "C" {

sso_status sso_server_create_lanes(const sso_options* opts, size_t hbm_budget_bytes,
                                   int32_t max_systems, int32_t max_tiles, int32_t lanes,
                                   sso_server** out) {
  if (!out) return fail(SSO_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (lanes < 1 || lanes > 8) return fail(SSO_ERR_INVALID, "lanes must be in [1, 8]");
  if (lanes == 1) return sso_server_create(opts, hbm_budget_bytes, max_systems, max_tiles, out);
  if (max_systems < lanes || max_tiles < lanes || hbm_budget_bytes < (size_t)lanes)
    return fail(SSO_ERR_INVALID, "need max_systems, max_tiles and budget of at least one per lane");
  sso_server* S = new sso_server();
  S->t0 = std::chrono::steady_clock::now();
  for (int k = 0; k < lanes; ++k) {
    sso_server* L = nullptr;
    const sso_status st = sso_server_create(opts, hbm_budget_bytes / lanes, max_systems / lanes,
                                            max_tiles / lanes, &L);
    if (st != SSO_OK) {
      stop_lanes(S);
      delete S;
      return st;
    }
    S->lanes.push_back(L);
  }
  S->global_of.resize(lanes);
  S->lane_nodes.assign(lanes, 0);
  S->lane_status.assign(lanes, SSO_OK);
  S->lane_msg.assign(lanes, std::string());
  S->lane_running.assign(lanes, 0);
  S->lane_waiting.assign(lanes, 0);
  try {
    for (int k = 1; k < lanes; ++k) S->lane_threads.emplace_back(lane_loop, S, k);
  } catch (const std::exception&) {
    stop_lanes(S);
    delete S;
    return fail(SSO_ERR_INVALID, "could not start the lanes' threads");
  }
  *out = S;
  return SSO_OK;
}

sso_status sso_server_create(const sso_options* opts, size_t hbm_budget_bytes,
                             int32_t max_systems, int32_t max_tiles, sso_server** out) {
  if (!out) return fail(SSO_ERR_INVALID, "out is NULL");
  *out = nullptr;
  sso_status st = check_options(opts);
  if (st != SSO_OK) return st;
  if (opts->precond == SSO_CHAIN)
    return fail(SSO_ERR_INVALID, "the server runs the CG preconditioners only (not SSO_CHAIN)");
  if (opts->precision == SSO_F32X2)
    return fail(SSO_ERR_INVALID, "the server runs SSO_FP64 or SSO_FP32_IR (not SSO_F32X2)");
  if (max_systems <= 0 || max_tiles <= 0 || hbm_budget_bytes == 0)
    return fail(SSO_ERR_INVALID, "need max_systems > 0, max_tiles > 0, budget > 0");
  sso_server* S = new sso_server();
  S->opts = *opts;
  S->opts.warm_start = 0;
  S->budget = hbm_budget_bytes;
  S->max_sys = max_systems;
  S->max_tiles = max_tiles;
  S->slot_req.assign(max_systems, nullptr);
  S->slot_tiles.assign(max_systems, {});
  S->t0 = std::chrono::steady_clock::now();
  const unsigned hw = std::thread::hardware_concurrency();
  const int n_workers = (int)std::min(8u, std::max(1u, hw));
  for (int k = 0; k < n_workers; ++k) S->workers.emplace_back(prep_worker, S);
  cudaError_t e = cudaStreamCreateWithFlags(&S->cg_stream, cudaStreamNonBlocking);
  for (int k = 0; k < kSetupStreams && e == cudaSuccess; ++k) {
    cudaStream_t st2 = nullptr;
    e = cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking);
    if (e == cudaSuccess) S->setup_streams.push_back(st2);
  }
  if (e == cudaSuccess) e = cudaMallocHost(&S->h_up, sizeof(SysScalars) * max_systems);
  if (e != cudaSuccess) {
    sso_server_destroy(S);
    return cuda_fail(e, "server streams");
  }
  e = cudaMalloc(&S->pool.base, hbm_budget_bytes);
  if (e != cudaSuccess) {
    S->pool.base = nullptr;
    sso_server_destroy(S);
    return cuda_fail(e, "cudaMalloc(server HBM budget)");
  }
  S->pool.size = hbm_budget_bytes;
  S->pool.free_[0] = hbm_budget_bytes;
  S->ring.size = kRingBytes;
  e = cudaMallocHost(&S->ring.base, kRingBytes);
  if (e != cudaSuccess) {
    S->ring.base = nullptr;
    sso_server_destroy(S);
    return cuda_fail(e, "cudaMallocHost(upload staging)");
  }
  st = batch_with_capacity(S->cg_stream, max_systems, max_tiles, &S->B);
  if (st != SSO_OK) {
    sso_server_destroy(S);
    return st;
  }
  *out = S;
  return SSO_OK;
}

void sso_server_destroy(sso_server* S) {
  if (!S) return;
  if (!S->lanes.empty()) {
    stop_lanes(S);
    delete S;
    return;
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (std::thread& t : S->workers) t.join();
  if (S->cg_stream) cudaStreamSynchronize(S->cg_stream);
  for (cudaStream_t st2 : S->setup_streams) cudaStreamSynchronize(st2);
  for (auto& kv : S->reqs) {
    ServerReq* R = kv.second;
    if (R->M) sso_model_destroy(R->M);
    if (R->ev_setup) cudaEventDestroy(R->ev_setup);
    delete R;
  }
  if (S->B) sso_batch_destroy(S->B);
  if (S->pool.base) cudaFree(S->pool.base);
  S->ring.release_all();
  if (S->h_up) cudaFreeHost(S->h_up);
  if (S->cg_stream) cudaStreamDestroy(S->cg_stream);
  for (cudaStream_t st2 : S->setup_streams) cudaStreamDestroy(st2);
  delete S;
}

sso_status sso_server_submit(sso_server* S, const sso_mesh* mesh, double w, uint64_t* ticket) {
  if (!S || !ticket) return fail(SSO_ERR_INVALID, "NULL argument");
  if (!S->lanes.empty()) {
    // the lane with the fewest nodes still to finish
    int k = 0;
    for (int j = 1; j < (int)S->lanes.size(); ++j)
      if (S->lane_nodes[j] < S->lane_nodes[k]) k = j;
    uint64_t lt = 0;
    const sso_status st = sso_server_submit(S->lanes[k], mesh, w, &lt);
    if (st != SSO_OK) return st;
    const uint64_t g = S->next_ticket++;
    S->lane_of[g] = {k, lt};
    S->global_of[k][lt] = g;
    const int nn = mesh ? mesh->n_nodes : 0;
    S->ticket_nodes[g] = nn;
    S->lane_nodes[k] += nn;
    *ticket = g;
    return SSO_OK;
  }
  ServerReq* R = new ServerReq();
  R->prep.reset(new ModelPrep());
  R->prep->aggregates = S->opts.precond == SSO_TWO_LEVEL;
  sso_status st = mesh_to_prep(mesh, *R->prep);
  if (st != SSO_OK) {
    delete R;
    return st;
  }
  R->ticket = S->next_ticket++;
  R->w = w;
  R->t_submit = ms_since(S->t0);
  S->reqs[R->ticket] = R;
  S->queue.push_back(R);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->prep_queue.push_back(R);
  }
  S->cv_work.notify_one();
  *ticket = R->ticket;
  return SSO_OK;
}

sso_status sso_server_step(sso_server* S, int32_t* n_running, int32_t* n_waiting) {
  if (!S) return fail(SSO_ERR_INVALID, "server is NULL");
  if (!S->lanes.empty()) return router_step(S, n_running, n_waiting);
  sso_batch* B = S->B;
  const bool fp64 = S->opts.precision == SSO_FP64;
  const bool two_level = S->opts.precond == SSO_TWO_LEVEL;
  const int k = fp64 ? 1 : two_level ? 2 : 0;
  const int iters = S->opts.iters_per_launch;
  sso_status st;
  // 1. one graph launch of CG iterations over the running systems
  bool launched = false;
  ++S->steps;
  auto tick = std::chrono::steady_clock::now();
  auto lap = [&tick](double& acc) {
    const auto now = std::chrono::steady_clock::now();
    acc += std::chrono::duration<double, std::milli>(now - tick).count();
    tick = now;
  };
  if (!S->running.empty()) {
    if (S->dirty && (st = server_upload_tables(S, S->slot_tiles)) != SSO_OK) return st;
    lap(S->ms_upload);
    ++S->graph_launches;
    B->h_flag[0] = (int)S->running.size();
    B->h_flag[1] = 0;
    CK(cudaMemcpyAsync(B->d_n_active, B->h_flag, 2 * sizeof(int), cudaMemcpyHostToDevice,
                       B->stream));
    if ((st = batch_graph(B, fp64, iters, two_level)) != SSO_OK) return st;
    CK(cudaGraphLaunch(B->exec[k], B->stream));
    g_launches += (two_level ? 5ull : 2ull) * (unsigned long long)iters;
    if ((st = debug_check(B->stream, "server: CG graph")) != SSO_OK) return st;
    CK(cudaMemcpyAsync(B->h_flag + 2, B->d_n_active, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                       B->stream));
    CK(cudaMemcpyAsync(B->h_sc, B->d_sc, sizeof(SysScalars) * S->max_sys,
                       cudaMemcpyDeviceToHost, B->stream));
    CK(cudaEventRecord(B->ev, B->stream));
    launched = true;
  }
  tick = std::chrono::steady_clock::now();
  // 2. admission while the GPU iterates: build models, set them up on the
  //    set-up stream (their kernels overlap the CG graph).  With a graph in
  //    flight the host admits until it completes; with the GPU idle it admits
  //    a few requests and returns, so that CG starts on them at once.
  int admitted = 0;
  while (!S->queue.empty()) {
    if (launched ? cudaEventQuery(B->ev) != cudaErrorNotReady : admitted >= kIdleAdmit) break;
    int slot = -1;
    for (int s2 = 0; s2 < S->max_sys; ++s2)
      if (!S->slot_req[s2]) {
        slot = s2;
        break;
      }
    if (slot < 0) break;
    ServerReq* R = S->queue.front();
    auto ta = std::chrono::steady_clock::now();
    auto lap2 = [&ta](double& acc) {
      const auto now = std::chrono::steady_clock::now();
      acc += std::chrono::duration<double, std::milli>(now - ta).count();
      ta = now;
    };
    {
      // The request's host half is built by a worker thread after submission.
      // Wait for it only while there is nothing else to do: with a graph in
      // flight, until the graph completes (then harvest, and admit at the
      // next step); with systems set up and waiting to join, not at all; with
      // the GPU idle and nothing pending, as long as it takes.
      std::unique_lock<std::mutex> lk(S->mu);
      if (launched) {
        while (!R->prep_done && cudaEventQuery(B->ev) == cudaErrorNotReady)
          S->cv_done.wait_for(lk, std::chrono::microseconds(50));
      } else if (S->running.empty() && S->pending.empty()) {
        S->cv_done.wait(lk, [R] { return R->prep_done; });
      }
      if (!R->prep_done) {
        lk.unlock();
        lap2(S->ms_admit_prep);
        break;
      }
    }
    lap2(S->ms_admit_prep);
    if (R->prep_status != SSO_OK) {  // invalid request: its result is the error
      S->queue.pop_front();
      R->stats.status = R->prep_status;
      R->phase = 3;
      S->completed.push_back(R->ticket);
      R->t_done = ms_since(S->t0);
      R->prep.reset();
      continue;
    }
    const size_t bytes = R->prep->bytes;
    const int n_tiles = (int)R->prep->tiles.size();
    const bool idle = S->running.empty() && S->pending.empty();
    if (S->tiles_used + n_tiles > S->max_tiles || S->used + bytes > S->budget) {
      if (!idle) break;  // wait for finished systems to free room
      S->queue.pop_front();
      R->stats.status = SSO_ERR_OOM;  // can never fit
      R->phase = 3;
      S->completed.push_back(R->ticket);
      R->t_done = ms_since(S->t0);
      R->prep.reset();
      continue;
    }
    void* arena = S->pool.alloc(bytes);
    if (!arena) {  // fragmented: wait for finished systems, unless none is left
      if (!idle) break;
      S->queue.pop_front();
      R->stats.status = SSO_ERR_OOM;
      R->phase = 3;
      S->completed.push_back(R->ticket);
      R->t_done = ms_since(S->t0);
      R->prep.reset();
      continue;
    }
    cudaError_t re;
    unsigned char* staged = S->ring.take(R->prep->prefix, re);
    if (re != cudaSuccess) return cuda_fail(re, "upload staging");
    if (staged) std::memcpy(staged, R->prep->image.data(), R->prep->prefix);
    sso_model* M = nullptr;
    cudaStream_t ss = S->setup_streams[S->next_setup];
    S->next_setup = (S->next_setup + 1) % (int)S->setup_streams.size();
    st = create_model_device(*R->prep, nullptr, false, ss, &M, arena, staged);
    if (staged) CK(S->ring.mark(staged, R->prep->prefix, ss));
    lap2(S->ms_admit_device);
    if (st != SSO_OK) S->pool.release(arena, bytes);
    if (st == SSO_ERR_CUDA) return st;  // the device, not the request, failed
    if (st != SSO_OK) {  // could not be set up
      S->queue.pop_front();
      R->stats.status = st;
      R->phase = 3;
      S->completed.push_back(R->ticket);
      R->t_done = ms_since(S->t0);
      R->prep.reset();
      continue;
    }
    S->queue.pop_front();
    if ((st = debug_check(ss, "server: before set-up")) != SSO_OK) return st;
    if ((st = setup_model(M, S->opts.precond, ss)) != SSO_OK) return st;
    CK(cudaMemsetAsync(M->d_u, 0, sizeof(double) * 6 * (size_t)M->n_nodes, ss));
    if ((st = debug_check(ss, "server: set-up kernels")) != SSO_OK) return st;
    CK(cudaEventCreateWithFlags(&R->ev_setup, cudaEventDisableTiming));
    CK(cudaEventRecord(R->ev_setup, ss));
    lap2(S->ms_admit_setup);
    R->M = M;
    R->bytes = bytes;
    R->slot = slot;
    R->phase = 1;
    S->slot_req[slot] = R;
    S->slot_tiles[slot].swap(R->prep->tiles);
    for (TileDesc& td : S->slot_tiles[slot]) td.sys = slot;
    R->prep.reset();
    fill_sysdesc(B->h_sys[slot], M, S->opts.precond);
    S->tiles_used += M->n_tiles;
    S->used += bytes;
    S->pending.push_back(slot);
    ++admitted;
  }
  lap(S->ms_admit);
  // 3. wait for the launch; harvest the systems that finished
  if (launched) {
    CK(cudaEventSynchronize(B->ev));
    lap(S->ms_wait);
    if (B->h_flag[3] != 0)
      return fail(SSO_ERR_CUDA, "CG kernel gave up waiting for a bulk copy (device fault?)");
    std::vector<int> done;
    for (int slot : S->running)
      if (B->h_sc[slot].state == ST_DONE) done.push_back(slot);
    for (int slot : done) {
      ServerReq* R = S->slot_req[slot];
      sso_model* M = R->M;
      const size_t ndof = 6 * (size_t)M->n_nodes;
      cudaStream_t s2 = B->stream;
      CL(launch_axpby((int)ndof, R->w, M->d_u, nullptr, M->d_fixed, M->d_lam, s2), 1);
      CL(launch_beam_adjoint(M->n_beams, M->d_xyz, M->d_beam_conn, M->d_beam_props, M->d_u,
                             M->d_u, R->w, M->d_gslot, s2),
         M->n_beams > 0);
      CL(launch_quad_adjoint(M->n_quads, M->d_xyz, M->d_quad_conn, M->d_quad_props,
                             M->pressure, M->gamma, M->d_u, M->d_u, R->w, R->w,
                             M->d_gslot + 2 * (size_t)M->n_beams, M->d_dt, s2),
         M->n_quads > 0);
      CL(launch_node_gather(M->n_nodes, M->d_nptr, M->d_nsrc, 2 * M->n_beams, nullptr,
                            M->d_gslot, nullptr, M->d_fixed, nullptr, M->d_dz, s2),
         1);
      CL(launch_dot(1, B->d_sys + slot, B->d_dots + slot, s2), 1);
      R->u.resize(ndof);
      R->dz.resize(M->n_nodes);
      R->dt.resize(M->n_quads);
      CK(cudaMemcpyAsync(R->u.data(), M->d_u, ndof * 8, cudaMemcpyDeviceToHost, s2));
      CK(cudaMemcpyAsync(R->dz.data(), M->d_dz, M->n_nodes * 8, cudaMemcpyDeviceToHost, s2));
      if (M->n_quads > 0)
        CK(cudaMemcpyAsync(R->dt.data(), M->d_dt, M->n_quads * 8, cudaMemcpyDeviceToHost, s2));
      CK(cudaMemcpyAsync(&R->C, B->d_dots + slot, 8, cudaMemcpyDeviceToHost, s2));
    }
    if (!done.empty()) CK(cudaStreamSynchronize(B->stream));
    if ((st = debug_check(B->stream, "server: gradients")) != SSO_OK) return st;
    const double now = ms_since(S->t0);
    for (int slot : done) {
      ServerReq* R = S->slot_req[slot];
      const SysScalars& sc = B->h_sc[slot];
      int err = 0;
      CK(cudaMemcpy(&err, R->M->d_err, sizeof(int), cudaMemcpyDeviceToHost));
      R->stats.status = err >= 2 ? SSO_ERR_CUDA : err ? SSO_ERR_SINGULAR : sc.status;
      R->stats.iterations = sc.iters;
      R->stats.sweeps = sc.sweeps;
      R->stats.rel_residual = sc.ff > 0.0 ? std::sqrt(sc.rr64 / sc.ff) : 0.0;
      R->stats.ms = now - R->t_submit;
      R->t_done = now;
      R->phase = 3;
      S->completed.push_back(R->ticket);
      S->used -= R->bytes;
      S->tiles_used -= R->M->n_tiles;
      void* arena = R->M->arena;
      sso_model_destroy(R->M);
      S->pool.release(arena, R->bytes);
      R->M = nullptr;
      S->slot_req[slot] = nullptr;
      S->running.erase(std::find(S->running.begin(), S->running.end(), slot));
      S->dirty = true;
    }
    lap(S->ms_harvest);
  }
  // 4. systems whose set-up has finished join the CG
  for (size_t i = 0; i < S->pending.size();) {
    const int slot = S->pending[i];
    ServerReq* R = S->slot_req[slot];
    cudaError_t q = cudaEventQuery(R->ev_setup);
    if (q == cudaErrorNotReady) {
      ++i;
      continue;
    }
    if (q != cudaSuccess) return cuda_fail(q, "set-up of an admitted request");
    init_scalars(S->h_up[slot], S->opts);
    CK(cudaMemcpyAsync(B->d_sc + slot, S->h_up + slot, sizeof(SysScalars),
                       cudaMemcpyHostToDevice, B->stream));
    R->phase = 2;
    S->running.push_back(slot);
    S->pending.erase(S->pending.begin() + i);
    S->dirty = true;
  }
  if (n_running) *n_running = (int)(S->running.size() + S->pending.size());
  if (n_waiting) *n_waiting = (int)S->queue.size();
  return SSO_OK;
}

sso_status sso_server_completed(sso_server* S, uint64_t* tickets, int32_t capacity,
                                int32_t* n) {
  if (!S || !n || (capacity > 0 && !tickets)) return fail(SSO_ERR_INVALID, "NULL argument");
  if (!S->lanes.empty()) {
    int got = 0;
    for (int k = 0; k < (int)S->lanes.size() && got < capacity; ++k) {
      int32_t m = 0;
      const sso_status st = sso_server_completed(S->lanes[k], tickets + got, capacity - got, &m);
      if (st != SSO_OK) return st;
      int kept = got;
      for (int j = got; j < got + m; ++j) {
        auto it = S->global_of[k].find(tickets[j]);
        if (it == S->global_of[k].end()) continue;  // polled already
        const uint64_t g = it->second;
        tickets[kept++] = g;
        auto nn = S->ticket_nodes.find(g);
        if (nn != S->ticket_nodes.end()) {
          S->lane_nodes[k] -= nn->second;
          S->ticket_nodes.erase(nn);
        }
      }
      got = kept;
    }
    *n = got;
    return SSO_OK;
  }
  const int k = std::min<int>(std::max(capacity, 0), (int)S->completed.size());
  std::copy(S->completed.begin(), S->completed.begin() + k, tickets);
  S->completed.erase(S->completed.begin(), S->completed.begin() + k);
  *n = k;
  return SSO_OK;
}

sso_status sso_server_info(const sso_server* S, double* ms, int64_t* counts) {
  if (!S) return fail(SSO_ERR_INVALID, "server is NULL");
  if (!S->lanes.empty()) {
    // phases summed over the lanes (they run at once); steps are this server's
    double acc[8] = {};
    int64_t cnt[2] = {0, 0};
    for (const sso_server* L : S->lanes) {
      double m[8];
      int64_t c[2];
      sso_server_info(L, m, c);
      for (int j = 0; j < 8; ++j) acc[j] += m[j];
      cnt[1] += c[1];
    }
    if (ms) std::copy(acc, acc + 8, ms);
    if (counts) {
      counts[0] = S->steps;
      counts[1] = cnt[1];
    }
    return SSO_OK;
  }
  if (ms) {
    ms[0] = S->ms_admit;
    ms[1] = S->ms_upload;
    ms[2] = S->ms_wait;
    ms[3] = S->ms_harvest;
    ms[4] = S->ms_admit_prep;
    ms[5] = S->ms_admit_device;
    ms[6] = S->ms_admit_setup;
    ms[7] = 0.0;
  }
  if (counts) {
    counts[0] = S->steps;
    counts[1] = S->graph_launches;
  }
  return SSO_OK;
}

sso_status sso_server_poll(sso_server* S, uint64_t ticket, double* u, double* C, double* dz,
                           double* dt, sso_stats* stats, double* latency_ms) {
  if (!S) return fail(SSO_ERR_INVALID, "server is NULL");
  if (!S->lanes.empty()) {
    auto lt = S->lane_of.find(ticket);
    if (lt == S->lane_of.end()) return fail(SSO_ERR_INVALID, "unknown ticket");
    const sso_status st = sso_server_poll(S->lanes[lt->second.first], lt->second.second, u, C,
                                          dz, dt, stats, latency_ms);
    if (st != SSO_ERR_NOT_READY) {
      const int k = lt->second.first;
      S->global_of[k].erase(lt->second.second);
      auto nn = S->ticket_nodes.find(ticket);
      if (nn != S->ticket_nodes.end()) {
        S->lane_nodes[k] -= nn->second;
        S->ticket_nodes.erase(nn);
      }
      S->lane_of.erase(lt);
    }
    return st;
  }
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return fail(SSO_ERR_INVALID, "unknown ticket");
  ServerReq* R = it->second;
  if (R->phase != 3) return SSO_ERR_NOT_READY;
  if (u && !R->u.empty()) CK(cudaMemcpy(u, R->u.data(), R->u.size() * 8, cudaMemcpyDefault));
  if (C) CK(cudaMemcpy(C, &R->C, 8, cudaMemcpyDefault));
  if (dz && !R->dz.empty())
    CK(cudaMemcpy(dz, R->dz.data(), R->dz.size() * 8, cudaMemcpyDefault));
  if (dt && !R->dt.empty())
    CK(cudaMemcpy(dt, R->dt.data(), R->dt.size() * 8, cudaMemcpyDefault));
  if (stats) *stats = R->stats;
  if (latency_ms) *latency_ms = R->t_done - R->t_submit;
  if (R->ev_setup) cudaEventDestroy(R->ev_setup);
  S->reqs.erase(it);
  delete R;
  return SSO_OK;
}

}  // extern "C"
