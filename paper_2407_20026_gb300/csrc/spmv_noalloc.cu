// sso_bsr_spmv_noalloc: the product y = K x with x^T y of sso_bsr_spmv, for
// callers that must not allocate device memory.
//
// Who needs it: callers that cannot call cudaMalloc or cudaMallocAsync.  A
// plug-in hosted by an application that hands it a fixed device-memory budget
// and forbids allocating beyond it; a real-time control or co-simulation loop
// that cannot take the allocator's latency or the synchronisation a
// cudaMalloc/cudaFree may imply; an application whose device memory all
// belongs to its own pool allocator.  They still pass their inputs and
// outputs; the per-tile partial sums the kernel needs live in a fixed array
// compiled into this library instead of being allocated per call.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (about 512 KiB) until the process exits.  Its size bounds
// the problem: at most kNoAllocMaxNodes nodes (larger inputs are rejected).
// Every call shares it, and the last call's partial sums stay in it; the
// completion counter is cleared by each call before the kernel runs.  Two
// calls whose kernels overlap on the GPU (different streams, or different host
// threads) race on the array and give wrong results: serialise them.
#include <cstdio>

#include "sso_internal.cuh"

namespace {

constexpr int kNoAllocMaxTiles = 65536;
constexpr int kNoAllocMaxNodes = kNoAllocMaxTiles * sso::SPMV_TILE;  // 2,097,152 nodes
constexpr size_t kCounterOffset = (size_t)kNoAllocMaxTiles * sizeof(double);

// partial sums [kNoAllocMaxTiles] doubles, then the completion counter
static __device__ __align__(256) unsigned char g_noalloc_scratch[kCounterOffset + 256];

// The device address of g_noalloc_scratch in the current context.  In host
// code the array's name is only a host-side stand-in, so the address is looked
// up with cudaGetSymbolAddress -- a host query that allocates nothing -- on
// every call, with the caller's device current.  It is not cached: after a
// cudaDeviceReset, or under another context of the same device, the array has
// a different address (the module is loaded anew).  On the first call in a
// context the query may load this library's device code (lazy module loading).
cudaError_t scratch_in_current_context(void** out) {
  return cudaGetSymbolAddress(out, g_noalloc_scratch);
}

}  // namespace

namespace sso {
// capi.cu: records the message returned by sso_last_error(); counts launches
sso_status record_failure(sso_status st, const char* msg);
void count_launches(unsigned long long n);
}  // namespace sso

extern "C" sso_status sso_bsr_spmv_noalloc(int32_t n_nodes, const int32_t* d_row_ptr,
                                            const int32_t* d_col, const double* d_K,
                                            const double* d_x, double* d_y, double* d_xty,
                                            void* stream) {
  if (n_nodes < 0) return sso::record_failure(SSO_ERR_INVALID, "n_nodes < 0");
  if (n_nodes > kNoAllocMaxNodes)
    return sso::record_failure(SSO_ERR_INVALID,
                             "sso_bsr_spmv_noalloc: n_nodes exceeds the fixed scratch "
                             "(at most 2097152 nodes); use sso_bsr_spmv");
  if (n_nodes == 0) return SSO_OK;
  if (!d_row_ptr || !d_col || !d_K || !d_x || !d_y || !d_xty)
    return sso::record_failure(SSO_ERR_INVALID, "NULL pointer");
  void* base = nullptr;
  cudaError_t e = scratch_in_current_context(&base);
  if (e != cudaSuccess) {
    char msg[256];
    snprintf(msg, sizeof msg, "sso_bsr_spmv_noalloc: cudaGetSymbolAddress of the fixed scratch "
             "failed: %s", cudaGetErrorString(e));
    return sso::record_failure(SSO_ERR_CUDA, msg);
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* partials = (double*)base;
  unsigned int* counter = (unsigned int*)((char*)base + kCounterOffset);
  e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess)
    e = sso::launch_bsr_spmv(n_nodes, d_row_ptr, d_col, d_K, d_x, d_y, d_xty, partials, counter,
                             s);
  if (e != cudaSuccess) return sso::record_failure(SSO_ERR_CUDA, cudaGetErrorString(e));
  sso::count_launches(1);
  return SSO_OK;
}
