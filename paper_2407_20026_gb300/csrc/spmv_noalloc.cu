// sso_bsr_spmv_noalloc: the product y = K x with x^T y of sso_bsr_spmv, for
// callers that must not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc / cudaMallocAsync is not
// allowed or not wanted -- inside a framework's region that forbids new
// allocations (for example while another component records a CUDA graph of
// its own work and treats any allocation as an error), in a real-time loop
// that cannot afford the implicit synchronisation or the latency of the
// allocator, or in an application whose device memory is entirely owned by its
// own pool.  Such callers still pass their inputs and outputs; the per-tile
// partial sums the kernel needs live in a fixed array compiled into this
// library instead of being allocated per call.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (about 512 KiB) until the process exits.  Its size bounds the
// problem: at most kNoAllocMaxNodes nodes.  Every call shares it, and the
// last call's partial sums stay in it; the completion counter is cleared by
// each call before the kernel runs.  Two calls whose kernels overlap on the
// GPU (different streams, or different host threads) race on the array and
// give wrong results: serialise them.
#include <mutex>

#include "sso_internal.cuh"

namespace {

constexpr int kNoAllocMaxTiles = 65536;
constexpr int kNoAllocMaxNodes = kNoAllocMaxTiles * sso::SPMV_TILE;  // 2,097,152 nodes
constexpr size_t kCounterOffset = (size_t)kNoAllocMaxTiles * sizeof(double);

// partial sums [kNoAllocMaxTiles] doubles, then the completion counter
static __device__ __align__(256) unsigned char g_noalloc_scratch[kCounterOffset + 256];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// The device address of g_noalloc_scratch on the current device.  The name of
// the array in host code is only a host-side stand-in, so the address is
// looked up once per device (with that device current) and cached.
cudaError_t scratch_on_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
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
  cudaError_t e = scratch_on_current_device(&base);
  if (e != cudaSuccess)
    return sso::record_failure(SSO_ERR_CUDA, "cudaGetSymbolAddress of the fixed scratch failed");
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
