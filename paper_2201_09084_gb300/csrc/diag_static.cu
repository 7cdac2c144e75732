// pic_diag_static: the Gauss-law / field-energy diagnostic of pic_diag with
// its charge-density scratch in a file-scope device array instead of memory
// allocated on first use.
//
// Who needs it: code that may not allocate device memory when it asks for a
// diagnostic -- hosts whose device memory is owned by a pool allocator that
// forbids side allocations, or real-time loops where an allocation's latency
// or failure is not acceptable.  pic_diag allocates its scratch lazily on the
// first call; this entry point never allocates.  Like pic_diag it reads the
// three results back to the host and synchronises the context's stream.
//
// The array holds kStaticRhoMax doubles (64 MiB) on every GPU where the
// library is loaded, until the process exits.  All calls share it and it
// keeps the contents of the last call, so every call clears it first; two
// calls that overlap on the GPU (different streams or contexts at the same
// time) race on it.
#include <cuda_runtime.h>

#include <atomic>

#include "../../include/picpml.h"
#include "picpml_internal.cuh"

namespace picpml {

// 8,388,608 nodes: enough for a 200^3-node grid.
constexpr long long kStaticRhoMax = 1LL << 23;

static __device__ __align__(256) double g_static_rho[kStaticRhoMax];
static __device__ __align__(256) double g_static_out[8];

namespace {
constexpr int kMaxDevices = 64;
// Per-device cache of the arrays' device addresses.  Threads that race on the
// first call of a device all store the same values, and the atomics make each
// store and load whole.  The cache assumes one (primary) context per device
// for the life of the process: after cudaDeviceReset the cached addresses
// would be stale, so the library does not support a reset while it is loaded.
std::atomic<double*> g_rho_ptr[kMaxDevices];
std::atomic<double*> g_out_ptr[kMaxDevices];
}  // namespace

// Device address of the static arrays for the current device; resolved on
// the first call on each device (cudaGetSymbolAddress), which is why that
// first call should come before any stream capture.
cudaError_t static_diag_buffers(double** rho, double** out, long long* cap) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  double* r = g_rho_ptr[dev].load(std::memory_order_acquire);
  double* o = g_out_ptr[dev].load(std::memory_order_acquire);
  if (!r || !o) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_rho);
    if (e != cudaSuccess) return e;
    void* q = nullptr;
    e = cudaGetSymbolAddress(&q, g_static_out);
    if (e != cudaSuccess) return e;
    r = static_cast<double*>(p);
    o = static_cast<double*>(q);
    g_out_ptr[dev].store(o, std::memory_order_release);
    g_rho_ptr[dev].store(r, std::memory_order_release);
  }
  *rho = r;
  *out = o;
  *cap = kStaticRhoMax;
  return cudaSuccess;
}

}  // namespace picpml
