// Yee field update with the split-field PML (Eqs. MaxwellE, MaxwellB,
// MaxwellSum), in the normalised units of picpml_internal.cuh.
//
// One thread per node (i,j,k) updates the three components staggered from
// that node; threads are laid out along x so every array access of a warp is
// one contiguous run (coalesced).  A component location is "split" when the
// conductivity of either axis it is split along is nonzero there; its two
// parts then advance by exponential differencing,
//   F <- e^{-s dt} F + (1 - e^{-s dt})/(s dt) (R dt),
// and their sum is written to the field array.  The source -alpha j goes to the
// part with the larger conductivity (first axis on ties), which for a pure
// z-PML is exactly Eq. MaxwellE; J was multiplied by alpha when deposited.
//
// Split parts are accumulated in one of two FP64-class representations:
//   SPL = 0: IEEE FP64;
//   SPL = 1: float-float pairs (hi + lo, about 48 significant bits) updated
//            with error-free FP32 transformations.  GB300's FP64 pipe runs at
//            a small fraction of its FP32 rate, and with FP64 parts the E pass
//            was FP64-pipe bound; the pairs keep the accumulation precision at
//            FP32 instruction cost and the same 8 bytes per part.
// Conductivity tests and Courant numbers use float copies, so FP32 fields need
// no FP64 instruction outside the FP64 parts.
#include "picpml_internal.cuh"

namespace picpml {

namespace {

// ---- float-float arithmetic (Dekker / Knuth error-free transformations) ----
struct ff {
  float h, l;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff ff_quick(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = ff_two_sum(a.h, b.h);
  const float e = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  return ff_quick(s.h, e);
}
__device__ __forceinline__ ff ff_mul(float2 a, ff b) {
  const float p = __fmul_rn(a.x, b.h);
  float e = __fmaf_rn(a.x, b.h, -p);
  e = __fmaf_rn(a.x, b.l, __fmaf_rn(a.y, b.h, e));
  return ff_quick(p, e);
}

// ---- split-part advance, FP64 parts ----
template <typename T>
__device__ __forceinline__ T adv64(double* p0, double* p1, long long id, T r0, T r1, T src, double ea0, double eb0,
                                   double ea1, double eb1, bool into1) {
  double e0 = p0[id], e1 = p1[id];
  e0 = ea0 * e0 + eb0 * ((double)r0 + (into1 ? 0.0 : (double)src));
  e1 = ea1 * e1 + eb1 * ((double)r1 + (into1 ? (double)src : 0.0));
  p0[id] = e0;
  p1[id] = e1;
  return (T)(e0 + e1);
}

// ---- split-part advance, float-float parts ----
__device__ __forceinline__ float advff(float2* p0, float2* p1, long long id, float r0, float r1, float src, float2 ea0,
                                       float2 eb0, float2 ea1, float2 eb1, bool into1) {
  const float2 a = p0[id], b = p1[id];
  ff e0 = ff_add(ff_mul(ea0, ff{a.x, a.y}), ff_mul(eb0, ff_two_sum(r0, into1 ? 0.f : src)));
  ff e1 = ff_add(ff_mul(ea1, ff{b.x, b.y}), ff_mul(eb1, ff_two_sum(r1, into1 ? src : 0.f)));
  p0[id] = make_float2(e0.h, e0.l);
  p1[id] = make_float2(e1.h, e1.l);
  const ff t = ff_add(e0, e1);
  return __fadd_rn(t.h, t.l);
}

// Advances one split location with parts along axes (A, B) at table indices
// (ia, ib); node tables for E, centre tables for B.  Returns the new total.
template <typename T, int SPL, bool CENT>
__device__ __forceinline__ T advance(const Tables& tb, double* const* parts, long long id, int A, int ia, int B,
                                     int ib, T r0, T r1, T src, float sA, float sB) {
  const bool into1 = sB > sA;
  if (SPL == 1) {
    const float2 one = make_float2(1.f, 0.f);
    const float2 ea0 = A >= 0 ? (CENT ? tb.ea2_c[A][ia] : tb.ea2_n[A][ia]) : one;
    const float2 eb0 = A >= 0 ? (CENT ? tb.eb2_c[A][ia] : tb.eb2_n[A][ia]) : one;
    const float2 ea1 = B >= 0 ? (CENT ? tb.ea2_c[B][ib] : tb.ea2_n[B][ib]) : one;
    const float2 eb1 = B >= 0 ? (CENT ? tb.eb2_c[B][ib] : tb.eb2_n[B][ib]) : one;
    return (T)advff(reinterpret_cast<float2*>(parts[0]), reinterpret_cast<float2*>(parts[1]), id, (float)r0,
                    (float)r1, (float)src, ea0, eb0, ea1, eb1, into1);
  } else {
    const double ea0 = A >= 0 ? (CENT ? tb.ea_c[A][ia] : tb.ea_n[A][ia]) : 1.0;
    const double eb0 = A >= 0 ? (CENT ? tb.eb_c[A][ia] : tb.eb_n[A][ia]) : 1.0;
    const double ea1 = B >= 0 ? (CENT ? tb.ea_c[B][ib] : tb.ea_n[B][ib]) : 1.0;
    const double eb1 = B >= 0 ? (CENT ? tb.eb_c[B][ib] : tb.eb_n[B][ib]) : 1.0;
    return adv64<T>(parts[0], parts[1], id, r0, r1, src, ea0, eb0, ea1, eb1, into1);
  }
}

template <typename T>
__device__ __forceinline__ T courant(const Geom& g, int a) {
  return sizeof(T) == 4 ? T(g.Sf[a]) : T(g.S[a]);
}

// Nodes per thread along z (3D): a thread marches KZ nodes upward in z and
// carries the z-neighbour values of the previous node in registers; its KZ
// nodes' loads are independent, so more memory requests are in flight.
constexpr int KZ = 4;

template <typename T, int DIM, int SPL>
__global__ void __launch_bounds__(256) k_field_E(Geom g, Tables tb, FieldPtrs<T> f) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = DIM == 3 ? blockIdx.y * blockDim.y + threadIdx.y : 0;
  const int k0 = DIM == 3 ? blockIdx.z * KZ : (blockIdx.y * blockDim.y + threadIdx.y) * KZ;
  if (i >= g.nn[0] || j >= g.nn[1] || k0 >= g.nn[2]) return;
  const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2];
  const T Sx = courant<T>(g, 0), Sy = courant<T>(g, 1), Sz = courant<T>(g, 2);
  const T* __restrict__ Bx = f.Bh[0];
  const T* __restrict__ By = f.Bh[1];
  const T* __restrict__ Bz = f.Bh[2];
  const bool jin = DIM == 2 || (j >= 1 && j <= N1 - 1);
  const bool iin = i >= 1 && i <= N0 - 1;
  const float sxn = tb.sdtf_n[0][i];
  const float syn = DIM == 3 ? tb.sdtf_n[1][j] : 0.f;
  long long id = g.idx(i, j, k0);
  // values at k-1 carried from the previous node
  T by_m = k0 >= 1 ? By[id - g.sz] : T(0);
  T bx_m = k0 >= 1 ? Bx[id - g.sz] : T(0);
#pragma unroll
  for (int kk = 0; kk < KZ; ++kk, id += g.sz) {
    const int k = k0 + kk;
    if (k >= g.nn[2]) break;
    const bool kin = k >= 1 && k <= N2 - 1;
    const T by0 = By[id], bx0 = Bx[id], bz0 = Bz[id];
    // J' is consumed here: read once, zeroed where it was nonzero (most of
    // the grid carries no current, so most threads write nothing back).
    const T jx = f.J[0][id], jy = f.J[1][id], jz = f.J[2][id];
    if (jx != T(0)) f.J[0][id] = T(0);
    if (jy != T(0)) f.J[1][id] = T(0);
    if (jz != T(0)) f.J[2][id] = T(0);
    const float szn = tb.sdtf_n[2][k];
    // Ex(i+1/2, j, k): parts along y (sigma_y at node j) and z (sigma_z at node k)
    if (i <= N0 - 1 && jin && kin) {
      const T r0 = DIM == 3 ? Sy * (bz0 - Bz[id - g.sy]) : T(0);
      const T r1 = -Sz * (by0 - by_m);
      if (syn > 0.f || szn > 0.f)
        f.E[0][id] = advance<T, SPL, false>(tb, f.Es[0], id, DIM == 3 ? 1 : -1, j, 2, k, r0, r1, -jx, syn, szn);
      else
        f.E[0][id] += r0 + r1 - jx;
    }
    // Ey(i, j+1/2, k): parts along x (sigma_x at node i) and z
    if (iin && (DIM == 2 || j <= N1 - 1) && kin) {
      const T r0 = -Sx * (bz0 - Bz[id - 1]);
      const T r1 = Sz * (bx0 - bx_m);
      if (sxn > 0.f || szn > 0.f)
        f.E[1][id] = advance<T, SPL, false>(tb, f.Es[1], id, 0, i, 2, k, r0, r1, -jy, sxn, szn);
      else
        f.E[1][id] += r0 + r1 - jy;
    }
    // Ez(i, j, k+1/2): parts along x and y
    if (iin && jin && k <= N2 - 1) {
      const T r0 = Sx * (by0 - By[id - 1]);
      const T r1 = DIM == 3 ? -Sy * (bx0 - Bx[id - g.sy]) : T(0);
      if (sxn > 0.f || syn > 0.f)
        f.E[2][id] = advance<T, SPL, false>(tb, f.Es[2], id, 0, i, DIM == 3 ? 1 : -1, j, r0, r1, -jz, sxn, syn);
      else
        f.E[2][id] += r0 + r1 - jz;
    }
    by_m = by0;
    bx_m = bx0;
  }
}

template <typename T, int DIM, int SPL>
__global__ void __launch_bounds__(256) k_field_B(Geom g, Tables tb, FieldPtrs<T> f) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = DIM == 3 ? blockIdx.y * blockDim.y + threadIdx.y : 0;
  const int k0 = DIM == 3 ? blockIdx.z * KZ : (blockIdx.y * blockDim.y + threadIdx.y) * KZ;
  if (i >= g.nn[0] || j >= g.nn[1] || k0 >= g.nn[2]) return;
  const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2];
  const T Sx = courant<T>(g, 0), Sy = courant<T>(g, 1), Sz = courant<T>(g, 2);
  const T* __restrict__ Ex = f.E[0];
  const T* __restrict__ Ey = f.E[1];
  const T* __restrict__ Ez = f.E[2];
  const bool jc = DIM == 2 || j <= N1 - 1;   // j is a cell-centre index
  const bool ic = i <= N0 - 1;
  const float sxc = ic ? tb.sdtf_c[0][i] : 0.f;
  const float syc = DIM == 3 && jc ? tb.sdtf_c[1][j] : 0.f;
  long long id = g.idx(i, j, k0);
  // values at k carried from the previous node (its k+1 neighbours)
  T ex0 = Ex[id], ey0 = Ey[id];
#pragma unroll
  for (int kk = 0; kk < KZ; ++kk, id += g.sz) {
    const int k = k0 + kk;
    if (k >= g.nn[2]) break;
    const bool kc = k <= N2 - 1;
    const T ex_p = kc ? Ex[id + g.sz] : T(0);
    const T ey_p = kc ? Ey[id + g.sz] : T(0);
    const T ez0 = Ez[id];
    const float szc = kc ? tb.sdtf_c[2][k] : 0.f;
    // Bx(i, j+1/2, k+1/2): parts along y (sigma_y at centre j) and z (centre k)
    if (jc && kc) {
      const T r0 = DIM == 3 ? -Sy * (Ez[id + g.sy] - ez0) : T(0);
      const T r1 = Sz * (ey_p - ey0);
      if (syc > 0.f || szc > 0.f)
        f.Bp[0][id] = advance<T, SPL, true>(tb, f.Bs[0], id, DIM == 3 ? 1 : -1, j, 2, k, r0, r1, T(0), syc, szc);
      else
        f.Bp[0][id] = f.Bh[0][id] + (r0 + r1);
    }
    // By(i+1/2, j, k+1/2): parts along x (centre i) and z (centre k)
    if (ic && kc) {
      const T r0 = Sx * (Ez[id + 1] - ez0);
      const T r1 = -Sz * (ex_p - ex0);
      if (sxc > 0.f || szc > 0.f)
        f.Bp[1][id] = advance<T, SPL, true>(tb, f.Bs[1], id, 0, i, 2, k, r0, r1, T(0), sxc, szc);
      else
        f.Bp[1][id] = f.Bh[1][id] + (r0 + r1);
    }
    // Bz(i+1/2, j+1/2, k): parts along x (centre i) and y (centre j)
    if (ic && jc) {
      const T r0 = -Sx * (Ey[id + 1] - ey0);
      const T r1 = DIM == 3 ? Sy * (Ex[id + g.sy] - ex0) : T(0);
      if (sxc > 0.f || syc > 0.f)
        f.Bp[2][id] = advance<T, SPL, true>(tb, f.Bs[2], id, 0, i, DIM == 3 ? 1 : -1, j, r0, r1, T(0), sxc, syc);
      else
        f.Bp[2][id] = f.Bh[2][id] + (r0 + r1);
    }
    ex0 = ex_p;
    ey0 = ey_p;
  }
}

template <typename T, int SPL>
cudaError_t launch_E(const Geom& g, const Tables& tb, const FieldPtrs<T>& f, cudaStream_t s) {
  if (g.dim == 3) {
    dim3 blk(32, 8, 1), grd((g.nn[0] + 31) / 32, (g.nn[1] + 7) / 8, (g.nn[2] + KZ - 1) / KZ);
    k_field_E<T, 3, SPL><<<grd, blk, 0, s>>>(g, tb, f);
  } else {
    dim3 blk(32, 8, 1), grd((g.nn[0] + 31) / 32, ((g.nn[2] + KZ - 1) / KZ + 7) / 8, 1);
    k_field_E<T, 2, SPL><<<grd, blk, 0, s>>>(g, tb, f);
  }
  return cudaGetLastError();
}

template <typename T, int SPL>
cudaError_t launch_B(const Geom& g, const Tables& tb, const FieldPtrs<T>& f, cudaStream_t s) {
  if (g.dim == 3) {
    dim3 blk(32, 8, 1), grd((g.nn[0] + 31) / 32, (g.nn[1] + 7) / 8, (g.nn[2] + KZ - 1) / KZ);
    k_field_B<T, 3, SPL><<<grd, blk, 0, s>>>(g, tb, f);
  } else {
    dim3 blk(32, 8, 1), grd((g.nn[0] + 31) / 32, ((g.nn[2] + KZ - 1) / KZ + 7) / 8, 1);
    k_field_B<T, 2, SPL><<<grd, blk, 0, s>>>(g, tb, f);
  }
  return cudaGetLastError();
}

}  // namespace

// split_ff: 1 = float-float split parts (FP32 fields only), 0 = FP64 parts.
template <typename T>
cudaError_t launch_field_E(const Geom& g, const Tables& tb, const FieldPtrs<T>& f, int split_ff, cudaStream_t s) {
  if (sizeof(T) == 4 && split_ff) return launch_E<T, 1>(g, tb, f, s);
  return launch_E<T, 0>(g, tb, f, s);
}

template <typename T>
cudaError_t launch_field_B(const Geom& g, const Tables& tb, const FieldPtrs<T>& f, int split_ff, cudaStream_t s) {
  if (sizeof(T) == 4 && split_ff) return launch_B<T, 1>(g, tb, f, s);
  return launch_B<T, 0>(g, tb, f, s);
}

template cudaError_t launch_field_E<float>(const Geom&, const Tables&, const FieldPtrs<float>&, int, cudaStream_t);
template cudaError_t launch_field_E<double>(const Geom&, const Tables&, const FieldPtrs<double>&, int, cudaStream_t);
template cudaError_t launch_field_B<float>(const Geom&, const Tables&, const FieldPtrs<float>&, int, cudaStream_t);
template cudaError_t launch_field_B<double>(const Geom&, const Tables&, const FieldPtrs<double>&, int, cudaStream_t);

}  // namespace picpml
