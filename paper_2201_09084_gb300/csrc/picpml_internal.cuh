// Internal definitions of libpicpml (not part of the ABI).
//
// Field normalisation used by every kernel: E' = E (V/m), B' = c B (V/m),
// J' = J dt / eps0 (V/m).  The Yee update is then
//   E' += S_a (B'_+ - B'_-) - J',   B' -= S_a (E'_+ - E'_-),
// with Courant numbers S_a = c dt / Delta_a, and the Boris push uses the one
// constant ke = q dt / (2 m c) for both E' and B' (Sec. II.B: the alpha terms
// leave the usual FDTD discretisation unchanged).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace picpml {

constexpr double kC = 299792458.0;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kMu0 = 1.0 / (kEps0 * kC * kC);

// Packed cell index: i | j << 10 | k << 20; -1 marks a removed particle.
__host__ __device__ inline int cell_i(int c) { return c & 1023; }
__host__ __device__ inline int cell_j(int c) { return (c >> 10) & 1023; }
__host__ __device__ inline int cell_k(int c) { return (c >> 20) & 2047; }
__host__ __device__ inline int pack_cell(int i, int j, int k) { return i | (j << 10) | (k << 20); }

// Grid geometry, passed by value to kernels.
struct Geom {
  int dim;
  int N[3];        // total cells per axis (physical + PML); N[1] = 0 in 2D
  int nn[3];       // nodes per axis stored: N + 1 (1 for y in 2D)
  int px;          // x pitch of the field arrays (elements)
  long long sy;    // stride of j
  long long sz;    // stride of k
  long long size;  // elements per field array
  double S[3];     // Courant numbers c dt / d_a
  float Sf[3];     // the same as a float-float pair (hi, lo), so kernels need no FP64
  float Sfl[3];
  int plo[3];      // PML cells on the low face
  int nph[3];      // physical cells
  int rmin[3], rmax[3];  // a particle at X = i + f stays while rmin <= X <= rmax
  // weight damping (alpha mode PML_ALPHA_WEIGHT): dt sigma/eps0 at depth d
  // cells into a face is wk[a] (d / delta)^wexp, wk[a] = coef c dt / d_a
  int wdamp;
  double wk[3];
  double winv_delta, wexp;
  __host__ __device__ long long idx(int i, int j, int k) const {
    return (long long)i + sy * j + sz * k;
  }
};

// Per-axis 1-D coefficient tables (device pointers), Sec. II.B: sigma and
// alpha at the nodes and the cell centres of the staggered grid.
struct Tables {
  // exponential differencing of d/dt F = R - s F over dt, normalised so that
  // F <- ea F + eb (R dt):  ea = exp(-s dt), eb = (1 - ea)/(s dt) (1 if s = 0)
  const double* ea_n[3];
  const double* eb_n[3];
  const double* sdt_n[3];   // s dt at the nodes (to pick the source split)
  const double* ea_c[3];
  const double* eb_c[3];
  const double* sdt_c[3];
  const float* sdtf_n[3];   // s dt as float (only compared: which split part
  const float* sdtf_c[3];   //   is damped and which takes the source)
  const float2* ea2_n[3];   // ea, eb as float-float pairs (hi, lo) for the
  const float2* eb2_n[3];   //   float-float split parts
  const float2* ea2_c[3];
  const float2* eb2_c[3];
  const float* al_nf[3];    // alpha at nodes / centres, FP32 copy
  const float* al_cf[3];
  const double* al_nd[3];   // FP64 copy
  const double* al_cd[3];
  int al1_lo[3], al1_hi[3]; // alpha is exactly 1 at nodes and centres al1_lo .. al1_hi
};

template <typename T>
struct FieldPtrs {
  T* E[3];
  T* Bh[3];   // B'^{n+1/2}
  T* Bp[3];   // B'^{n-1/2} (overwritten with B'^{n+3/2} by the B pass)
  T* J[3];    // J' (dt/eps0 units)
  double* Es[3][2];
  double* Bs[3][2];
  long long* Jq[3];   // deterministic mode: int64 current sums (else null)
  T* Bn[3];           // B at the integer time, (B^{n-1/2} + B^{n+1/2})/2, written by the B pass (else null)
};

// Particle data of one species for a kernel.
template <typename T>
struct SpeciesPtrs {
  void* pos;
  void* mom;
  const long long* n_dev;   // live count on the device (upper bound of indices)
  long long capacity;
  T ke;                     // q dt / (2 m c)
  T cj[3];                  // J' per unit weight: -q/(eps0 d_b d_c) (3D)
  T cjy2d;                  // 2D out-of-plane: q dt c /(eps0 dx dz Ly)
  int immobile;
  double qn;                // charge in elementary charges (deterministic mode)
  float4* save_pos;         // scratch of push(): x^n (FP32 layout)
  float4* save_mom;
};

// Species of one launch of the tile-resident particle kernel (3D FP32,
// order 1): each with the end offset of every sort tile's particles at the
// species' last sort (device array of one entry per tile).
constexpr int kTileMaxSpecies = 8;
struct TileSpecies {
  SpeciesPtrs<float> sp;
  const long long* tile_end;
};
struct TileLaunch {
  int nsp;
  int prescribed;
  int arr_E[3], arr_Bh[3], arr_Bp[3], arr_Bn[3];   // field array of each component (4th tensor-map coordinate)
  TileSpecies s[kTileMaxSpecies];
};

// 32-byte aligned quadruple of doubles (FP64 particle layout).
struct __align__(32) dbl4 {
  double x, y, z, w;
};

// Deterministic deposition: shape quantum 2^-kFixShapeBits; one integer
// current unit is e / (6 * 2^24) of charge crossing a cell face, reached from
// the exact integer Esirkepov sums (units 2^-60 of the particle charge, times
// 6) by the factor w q/e 2^-36.  The factor is the integer
// Wq = rint(w q/e 2^kFixWqBits) of the particle, and each sum's contribution
// is (sum * Wq) 2^-(36 + kFixWqBits) rounded to the nearest integer (halves
// up), formed exactly in 128-bit integer arithmetic (fix_scale).
constexpr int kFixShapeBits = 20;
constexpr int kFixWqBits = 28;
constexpr double kFixWqScale = 268435456.0;        // 2^kFixWqBits
constexpr double kFixUnit = 6.0 * 16777216.0;      // 6 * 2^24
constexpr double kFixMaxWq = 4294967296.0;         // |w q/e| above 2^32 is refused

#ifdef __CUDACC__
// round(acc * Wq / 2^S), halves up, from the exact 128-bit product
// (|acc| < 2^63, |Wq| <= 2^60, 0 < S <= 64).
template <int S>
__device__ __forceinline__ long long fix_scale(long long acc, long long Wq) {
  const unsigned long long lo = (unsigned long long)acc * (unsigned long long)Wq;
  long long hi = __mul64hi(acc, Wq);
  const unsigned long long lo2 = lo + (1ull << (S - 1));
  hi += lo2 < lo ? 1 : 0;
  if constexpr (S == 64)
    return hi;
  else
    return (long long)(((unsigned long long)hi << (64 - S)) | (lo2 >> S));
}
#endif
constexpr double kQe = 1.602176634e-19;

// Raises a kernel's dynamic shared-memory limit to `bytes` on the current
// device, once per device (the attribute belongs to the device's context;
// `done` holds one bit per device ordinal < 64, shared by the callers of one
// kernel).  Threads racing on the first launch may both set it: harmless.
template <typename K>
inline cudaError_t smem_limit_once(K kernel, int bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
  return e;
}

// Device status word bits.
enum : unsigned { ST_BAD_PARTICLE = 1u, ST_FIXED_OVERFLOW = 2u, ST_INJECT_OVERFLOW = 4u, ST_TIMEOUT = 8u };

}  // namespace picpml
