// Per-node Yee/PML updates shared by the field kernels of one box
// (field.cu) and of the batched runs (batch2d.cu).  See field.cu for the
// scheme; the functions here update the three components staggered from node
// (i,j,k), given the z-neighbour values (k-1 for E, k+1 for B) by the caller.
#pragma once

#include "ff.cuh"
#include "picpml_internal.cuh"

namespace picpml {
namespace fn {

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


// Whether a node (centre: the point i + 1/2) lies in the PML along axis a,
// from the box geometry: there sigma > 0 whenever the profile's coefficient
// is (Eq. conductivity vanishes only at depth 0).
__device__ __forceinline__ bool pml_node(const Geom& g, int a, int i) {
  return i < g.plo[a] || i > g.plo[a] + g.nph[a];
}
__device__ __forceinline__ bool pml_cent(const Geom& g, int a, int i) {
  return i < g.plo[a] || i >= g.plo[a] + g.nph[a];
}

// E^{n+1} at node (i,j,k).  by_m, bx_m: By, Bx at (i,j,k-1).  GEO: decide
// the split locations from the box geometry (single boxes), so the split
// parts' loads need not wait for the conductivity tables; else from the
// tables (batched runs).
template <typename T, int DIM, int SPL, bool GEO = false>
__device__ __forceinline__ void e_update(const Geom& g, const Tables& tb, const FieldPtrs<T>& f, int i, int j, int k,
                                         long long id, T by_m, T bx_m, T by0, T bx0, T bz0) {
  const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2];
  const T Sx = courant<T>(g, 0), Sy = courant<T>(g, 1), Sz = courant<T>(g, 2);
  const bool jin = DIM == 2 || (j >= 1 && j <= N1 - 1);
  const bool iin = i >= 1 && i <= N0 - 1;
  const bool kin = k >= 1 && k <= N2 - 1;
  const float sxn = tb.sdtf_n[0][i];
  const float syn = DIM == 3 ? tb.sdtf_n[1][j] : 0.f;
  const float szn = tb.sdtf_n[2][k];
  const bool px = GEO ? pml_node(g, 0, i) : sxn > 0.f;
  const bool py = DIM == 3 && (GEO ? pml_node(g, 1, j) : syn > 0.f);
  const bool pz = GEO ? pml_node(g, 2, k) : szn > 0.f;
  // J' is consumed here: read once, zeroed where it was nonzero (most of the
  // grid carries no current, so most threads write nothing back).
  const T jx = f.J[0][id], jy = f.J[1][id], jz = f.J[2][id];
  if (jx != T(0)) f.J[0][id] = T(0);
  if (jy != T(0)) f.J[1][id] = T(0);
  if (jz != T(0)) f.J[2][id] = T(0);
  const T* __restrict__ Bx = f.Bh[0];
  const T* __restrict__ By = f.Bh[1];
  const T* __restrict__ Bz = f.Bh[2];
  // Ex(i+1/2, j, k): parts along y (sigma_y at node j) and z (sigma_z at node k)
  if (i <= N0 - 1 && jin && kin) {
    const T r0 = DIM == 3 ? Sy * (bz0 - Bz[id - g.sy]) : T(0);
    const T r1 = -Sz * (by0 - by_m);
    if (py || pz)
      f.E[0][id] = advance<T, SPL, false>(tb, f.Es[0], id, DIM == 3 ? 1 : -1, j, 2, k, r0, r1, -jx, syn, szn);
    else
      f.E[0][id] += r0 + r1 - jx;
  }
  // Ey(i, j+1/2, k): parts along x (sigma_x at node i) and z
  if (iin && (DIM == 2 || j <= N1 - 1) && kin) {
    const T r0 = -Sx * (bz0 - Bz[id - 1]);
    const T r1 = Sz * (bx0 - bx_m);
    if (px || pz)
      f.E[1][id] = advance<T, SPL, false>(tb, f.Es[1], id, 0, i, 2, k, r0, r1, -jy, sxn, szn);
    else
      f.E[1][id] += r0 + r1 - jy;
  }
  // Ez(i, j, k+1/2): parts along x and y
  if (iin && jin && k <= N2 - 1) {
    const T r0 = Sx * (by0 - By[id - 1]);
    const T r1 = DIM == 3 ? -Sy * (bx0 - Bx[id - g.sy]) : T(0);
    if (px || py)
      f.E[2][id] = advance<T, SPL, false>(tb, f.Es[2], id, 0, i, DIM == 3 ? 1 : -1, j, r0, r1, -jz, sxn, syn);
    else
      f.E[2][id] += r0 + r1 - jz;
  }
}

// B^{n+3/2} at node (i,j,k) into Bp.  ex_p, ey_p: Ex, Ey at (i,j,k+1) (any
// value when k = N2); ex0, ey0, ez0: values at (i,j,k).
template <typename T, int DIM, int SPL, bool GEO = false>
__device__ __forceinline__ void b_update(const Geom& g, const Tables& tb, const FieldPtrs<T>& f, int i, int j, int k,
                                         long long id, T ex_p, T ey_p, T ex0, T ey0, T ez0) {
  const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2];
  const T Sx = courant<T>(g, 0), Sy = courant<T>(g, 1), Sz = courant<T>(g, 2);
  const T* __restrict__ Ex = f.E[0];
  const T* __restrict__ Ey = f.E[1];
  const T* __restrict__ Ez = f.E[2];
  const bool jc = DIM == 2 || j <= N1 - 1;   // j is a cell-centre index
  const bool ic = i <= N0 - 1;
  const bool kc = k <= N2 - 1;
  const float sxc = ic ? tb.sdtf_c[0][i] : 0.f;
  const float syc = DIM == 3 && jc ? tb.sdtf_c[1][j] : 0.f;
  const float szc = kc ? tb.sdtf_c[2][k] : 0.f;
  const bool px = GEO ? (ic && pml_cent(g, 0, i)) : sxc > 0.f;
  const bool py = DIM == 3 && (GEO ? (jc && pml_cent(g, 1, j)) : syc > 0.f);
  const bool pz = GEO ? (kc && pml_cent(g, 2, k)) : szc > 0.f;
  // Bx(i, j+1/2, k+1/2): parts along y (sigma_y at centre j) and z (centre k)
  if (jc && kc) {
    const T r0 = DIM == 3 ? -Sy * (Ez[id + g.sy] - ez0) : T(0);
    const T r1 = Sz * (ey_p - ey0);
    if (py || pz)
      f.Bp[0][id] = advance<T, SPL, true>(tb, f.Bs[0], id, DIM == 3 ? 1 : -1, j, 2, k, r0, r1, T(0), syc, szc);
    else
      f.Bp[0][id] = f.Bh[0][id] + (r0 + r1);
  }
  // By(i+1/2, j, k+1/2): parts along x (centre i) and z (centre k)
  if (ic && kc) {
    const T r0 = Sx * (Ez[id + 1] - ez0);
    const T r1 = -Sz * (ex_p - ex0);
    if (px || pz)
      f.Bp[1][id] = advance<T, SPL, true>(tb, f.Bs[1], id, 0, i, 2, k, r0, r1, T(0), sxc, szc);
    else
      f.Bp[1][id] = f.Bh[1][id] + (r0 + r1);
  }
  // Bz(i+1/2, j+1/2, k): parts along x (centre i) and y (centre j)
  if (ic && jc) {
    const T r0 = -Sx * (Ey[id + 1] - ey0);
    const T r1 = DIM == 3 ? Sy * (Ex[id + g.sy] - ex0) : T(0);
    if (px || py)
      f.Bp[2][id] = advance<T, SPL, true>(tb, f.Bs[2], id, 0, i, DIM == 3 ? 1 : -1, j, r0, r1, T(0), sxc, syc);
    else
      f.Bp[2][id] = f.Bh[2][id] + (r0 + r1);
  }
}

}  // namespace fn
}  // namespace picpml
