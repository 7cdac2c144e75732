// pic_diag_static: the Gauss-law / field-energy diagnostic of pic_diag with
// its charge-density scratch in a file-scope device array instead of memory
// allocated on first use.
//
// Who needs it: code that may not allocate device memory when it asks for a
// diagnostic -- a step loop being recorded into a CUDA graph (cudaMalloc is
// not allowed while a stream is capturing), hosts whose device memory is
// owned by a pool allocator that forbids side allocations, or real-time loops
// where an allocation's latency or failure is not acceptable.  pic_diag
// allocates its scratch lazily on the first call; this entry point never
// allocates.
//
// The array holds kStaticRhoMax doubles (64 MiB) on every GPU where the
// library is loaded, until the process exits.  All calls share it and it
// keeps the contents of the last call, so every call clears it first; two
// calls that overlap on the GPU (different streams or contexts at the same
// time) race on it.
#include <cuda_runtime.h>

#include "../../include/picpml.h"
#include "picpml_internal.cuh"

namespace picpml {

// 8,388,608 nodes: enough for a 200^3-node grid.
constexpr long long kStaticRhoMax = 1LL << 23;

static __device__ __align__(256) double g_static_rho[kStaticRhoMax];
static __device__ __align__(256) double g_static_out[8];

namespace {
constexpr int kMaxDevices = 64;
double* g_rho_ptr[kMaxDevices] = {nullptr};
double* g_out_ptr[kMaxDevices] = {nullptr};
}  // namespace

// Device address of the static arrays for the current device; resolved once
// per device (cudaGetSymbolAddress), which is why the first call on a device
// should not happen while a stream is being captured.
cudaError_t static_diag_buffers(double** rho, double** out, long long* cap) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!g_rho_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_rho);
    if (e != cudaSuccess) return e;
    void* q = nullptr;
    e = cudaGetSymbolAddress(&q, g_static_out);
    if (e != cudaSuccess) return e;
    g_rho_ptr[dev] = static_cast<double*>(p);
    g_out_ptr[dev] = static_cast<double*>(q);
  }
  *rho = g_rho_ptr[dev];
  *out = g_out_ptr[dev];
  *cap = kStaticRhoMax;
  return cudaSuccess;
}

}  // namespace picpml
