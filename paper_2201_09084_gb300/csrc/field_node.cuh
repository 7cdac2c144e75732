// Per-node Yee/PML updates shared by the field kernels of one box
// (field.cu) and of the batched runs (batch2d.cu).  See field.cu for the
// scheme; the functions here update the three components staggered from node
// (i,j,k), given the z-neighbour values (k-1 for E, k+1 for B) by the caller.
#pragma once

#include "ff.cuh"
#include "picpml_internal.cuh"

namespace picpml {
namespace fn {

// A split location's two parts, held in registers between their load and
// their store (FP64 parts, or float-float pairs).
template <int SPL>
struct Parts;
template <>
struct Parts<1> {
  float2 a, b;
};
template <>
struct Parts<0> {
  double a, b;
};

template <int SPL>
__device__ __forceinline__ Parts<SPL> load_parts(double* const* parts, long long id) {
  if constexpr (SPL == 1)
    return {reinterpret_cast<const float2*>(parts[0])[id], reinterpret_cast<const float2*>(parts[1])[id]};
  else
    return {parts[0][id], parts[1][id]};
}

template <int SPL>
__device__ __forceinline__ void store_parts(double* const* parts, long long id, const Parts<SPL>& pv) {
  if constexpr (SPL == 1) {
    reinterpret_cast<float2*>(parts[0])[id] = pv.a;
    reinterpret_cast<float2*>(parts[1])[id] = pv.b;
  } else {
    parts[0][id] = pv.a;
    parts[1][id] = pv.b;
  }
}

// Advances one split location's parts (in registers) along axes (A, B) at
// table indices (ia, ib); node tables for E, centre tables for B.  Each part
// F <- e^{-s dt} F + (1 - e^{-s dt})/(s dt) (r + source), the source going to
// the part with the larger conductivity.  Returns the new total.
template <typename T, int SPL, bool CENT>
__device__ __forceinline__ T advance(const Tables& tb, Parts<SPL>& pv, int A, int ia, int B, int ib, T r0, T r1,
                                     T src, float sA, float sB) {
  const bool into1 = sB > sA;
  if constexpr (SPL == 1) {
    const float2 one = make_float2(1.f, 0.f);
    const float2 ea0 = A >= 0 ? (CENT ? tb.ea2_c[A][ia] : tb.ea2_n[A][ia]) : one;
    const float2 eb0 = A >= 0 ? (CENT ? tb.eb2_c[A][ia] : tb.eb2_n[A][ia]) : one;
    const float2 ea1 = B >= 0 ? (CENT ? tb.ea2_c[B][ib] : tb.ea2_n[B][ib]) : one;
    const float2 eb1 = B >= 0 ? (CENT ? tb.eb2_c[B][ib] : tb.eb2_n[B][ib]) : one;
    const float s = (float)src;
    const ff e0 = ff_add(ff_mul(ea0, ff{pv.a.x, pv.a.y}), ff_mul(eb0, ff_two_sum((float)r0, into1 ? 0.f : s)));
    const ff e1 = ff_add(ff_mul(ea1, ff{pv.b.x, pv.b.y}), ff_mul(eb1, ff_two_sum((float)r1, into1 ? s : 0.f)));
    pv.a = make_float2(e0.h, e0.l);
    pv.b = make_float2(e1.h, e1.l);
    const ff t = ff_add(e0, e1);
    return (T)__fadd_rn(t.h, t.l);
  } else if constexpr (sizeof(T) == 4) {
    // FP32 fields, IEEE FP64 parts: the increment eb (r + source) is formed in
    // FP32 from its FP32 inputs (eb rounded to FP32: the hi word of its
    // float-float pair) and added to the decayed part in FP64, so a part costs
    // one conversion and one FP64 FMA on GB300's narrow FP64 pipe.
    const float eb0 = A >= 0 ? (CENT ? tb.eb2_c[A][ia].x : tb.eb2_n[A][ia].x) : 1.0f;
    const float eb1 = B >= 0 ? (CENT ? tb.eb2_c[B][ib].x : tb.eb2_n[B][ib].x) : 1.0f;
    const double ea0 = A >= 0 ? (CENT ? tb.ea_c[A][ia] : tb.ea_n[A][ia]) : 1.0;
    const double ea1 = B >= 0 ? (CENT ? tb.ea_c[B][ib] : tb.ea_n[B][ib]) : 1.0;
    const float i0 = eb0 * ((float)r0 + (into1 ? 0.0f : (float)src));
    const float i1 = eb1 * ((float)r1 + (into1 ? (float)src : 0.0f));
    const double e0 = fma(ea0, pv.a, (double)i0);
    const double e1 = fma(ea1, pv.b, (double)i1);
    pv.a = e0;
    pv.b = e1;
    return (T)(e0 + e1);
  } else {
    const double ea0 = A >= 0 ? (CENT ? tb.ea_c[A][ia] : tb.ea_n[A][ia]) : 1.0;
    const double eb0 = A >= 0 ? (CENT ? tb.eb_c[A][ia] : tb.eb_n[A][ia]) : 1.0;
    const double ea1 = B >= 0 ? (CENT ? tb.ea_c[B][ib] : tb.ea_n[B][ib]) : 1.0;
    const double eb1 = B >= 0 ? (CENT ? tb.eb_c[B][ib] : tb.eb_n[B][ib]) : 1.0;
    const double e0 = ea0 * pv.a + eb0 * ((double)r0 + (into1 ? 0.0 : (double)src));
    const double e1 = ea1 * pv.b + eb1 * ((double)r1 + (into1 ? (double)src : 0.0));
    pv.a = e0;
    pv.b = e1;
    return (T)(e0 + e1);
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
// the split locations from the box geometry (the split parts' loads then need
// no table load first); else from the conductivity tables.  Every load of the
// node comes before any of its stores (the compiler cannot reorder loads
// across stores to arrays that might alias), so a thread has all its memory
// requests in flight at once.
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
  // Ex(i+1/2, j, k): parts along y (sigma_y at node j) and z (sigma_z at node k);
  // Ey(i, j+1/2, k): parts along x and z; Ez(i, j, k+1/2): parts along x and y
  const bool okx = i <= N0 - 1 && jin && kin;
  const bool oky = iin && (DIM == 2 || j <= N1 - 1) && kin;
  const bool okz = iin && jin && k <= N2 - 1;
  const bool spx = okx && (py || pz), spy = oky && (px || pz), spz = okz && (px || py);
  const T* __restrict__ Bx = f.Bh[0];
  const T* __restrict__ By = f.Bh[1];
  const T* __restrict__ Bz = f.Bh[2];
  // ---- loads: J' (consumed here), the B neighbours, E or the split parts ----
  const T jx = f.J[0][id], jy = f.J[1][id], jz = f.J[2][id];
  const T bz_ym = DIM == 3 && okx ? Bz[id - g.sy] : T(0);
  const T bz_xm = oky ? Bz[id - 1] : T(0);
  const T by_xm = okz ? By[id - 1] : T(0);
  const T bx_ym = DIM == 3 && okz ? Bx[id - g.sy] : T(0);
  T ex = okx && !spx ? f.E[0][id] : T(0);
  T ey = oky && !spy ? f.E[1][id] : T(0);
  T ez = okz && !spz ? f.E[2][id] : T(0);
  Parts<SPL> qx{}, qy{}, qz{};
  if (spx) qx = load_parts<SPL>(f.Es[0], id);
  if (spy) qy = load_parts<SPL>(f.Es[1], id);
  if (spz) qz = load_parts<SPL>(f.Es[2], id);
  // ---- update ----
  if (okx) {
    const T r0 = DIM == 3 ? Sy * (bz0 - bz_ym) : T(0);
    const T r1 = -Sz * (by0 - by_m);
    ex = spx ? advance<T, SPL, false>(tb, qx, DIM == 3 ? 1 : -1, j, 2, k, r0, r1, -jx, syn, szn) : ex + (r0 + r1 - jx);
  }
  if (oky) {
    const T r0 = -Sx * (bz0 - bz_xm);
    const T r1 = Sz * (bx0 - bx_m);
    ey = spy ? advance<T, SPL, false>(tb, qy, 0, i, 2, k, r0, r1, -jy, sxn, szn) : ey + (r0 + r1 - jy);
  }
  if (okz) {
    const T r0 = Sx * (by0 - by_xm);
    const T r1 = DIM == 3 ? -Sy * (bx0 - bx_ym) : T(0);
    ez = spz ? advance<T, SPL, false>(tb, qz, 0, i, DIM == 3 ? 1 : -1, j, r0, r1, -jz, sxn, syn) : ez + (r0 + r1 - jz);
  }
  // ---- stores; J' is zeroed where it was nonzero (most of the grid carries
  //      no current, so most threads write nothing back) ----
  if (okx) f.E[0][id] = ex;
  if (oky) f.E[1][id] = ey;
  if (okz) f.E[2][id] = ez;
  if (spx) store_parts<SPL>(f.Es[0], id, qx);
  if (spy) store_parts<SPL>(f.Es[1], id, qy);
  if (spz) store_parts<SPL>(f.Es[2], id, qz);
  if (jx != T(0)) f.J[0][id] = T(0);
  if (jy != T(0)) f.J[1][id] = T(0);
  if (jz != T(0)) f.J[2][id] = T(0);
}

// B^{n+3/2} at node (i,j,k) into Bp.  ex_p, ey_p: Ex, Ey at (i,j,k+1) (any
// value when k = N2); ex0, ey0, ez0: values at (i,j,k).  Loads before stores
// as in e_update.
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
  // Bx(i, j+1/2, k+1/2): parts along y (centre j) and z (centre k);
  // By(i+1/2, j, k+1/2): parts along x and z; Bz(i+1/2, j+1/2, k): x and y
  const bool okx = jc && kc, oky = ic && kc, okz = ic && jc;
  const bool spx = okx && (py || pz), spy = oky && (px || pz), spz = okz && (px || py);
  // ---- loads ----
  const T ez_yp = DIM == 3 && okx ? Ez[id + g.sy] : T(0);
  const T ez_xp = oky ? Ez[id + 1] : T(0);
  const T ey_xp = okz ? Ey[id + 1] : T(0);
  const T ex_yp = DIM == 3 && okz ? Ex[id + g.sy] : T(0);
  T bx = okx && !spx ? f.Bh[0][id] : T(0);
  T by = oky && !spy ? f.Bh[1][id] : T(0);
  T bz = okz && !spz ? f.Bh[2][id] : T(0);
  Parts<SPL> qx{}, qy{}, qz{};
  if (spx) qx = load_parts<SPL>(f.Bs[0], id);
  if (spy) qy = load_parts<SPL>(f.Bs[1], id);
  if (spz) qz = load_parts<SPL>(f.Bs[2], id);
  // B at the integer time for the particle push, (old + new)/2, where asked
  // for: the old totals (split nodes hold them only as parts)
  const bool avg = f.Bn[0] != nullptr;
  T bx0 = bx, by0 = by, bz0 = bz;
  if (avg) {
    if (spx) bx0 = f.Bh[0][id];
    if (spy) by0 = f.Bh[1][id];
    if (spz) bz0 = f.Bh[2][id];
  }
  // ---- update ----
  if (okx) {
    const T r0 = DIM == 3 ? -Sy * (ez_yp - ez0) : T(0);
    const T r1 = Sz * (ey_p - ey0);
    bx = spx ? advance<T, SPL, true>(tb, qx, DIM == 3 ? 1 : -1, j, 2, k, r0, r1, T(0), syc, szc) : bx + (r0 + r1);
  }
  if (oky) {
    const T r0 = Sx * (ez_xp - ez0);
    const T r1 = -Sz * (ex_p - ex0);
    by = spy ? advance<T, SPL, true>(tb, qy, 0, i, 2, k, r0, r1, T(0), sxc, szc) : by + (r0 + r1);
  }
  if (okz) {
    const T r0 = -Sx * (ey_xp - ey0);
    const T r1 = DIM == 3 ? Sy * (ex_yp - ex0) : T(0);
    bz = spz ? advance<T, SPL, true>(tb, qz, 0, i, DIM == 3 ? 1 : -1, j, r0, r1, T(0), sxc, syc) : bz + (r0 + r1);
  }
  // ---- stores ----
  if (okx) f.Bp[0][id] = bx;
  if (oky) f.Bp[1][id] = by;
  if (okz) f.Bp[2][id] = bz;
  if (avg) {
    if (okx) f.Bn[0][id] = T(0.5) * (bx0 + bx);
    if (oky) f.Bn[1][id] = T(0.5) * (by0 + by);
    if (okz) f.Bn[2][id] = T(0.5) * (bz0 + bz);
  }
  if (spx) store_parts<SPL>(f.Bs[0], id, qx);
  if (spy) store_parts<SPL>(f.Bs[1], id, qy);
  if (spz) store_parts<SPL>(f.Bs[2], id, qz);
}

// ---------------------------------------------------------------------------
// Cole-Karkkainen (CK) solver (App. A: the paper's single-particle and LWFA
// runs; the scheme of Cole 1997/2002 and Karkkainen et al. 2006): Faraday's
// law takes each difference of E averaged over the two transverse axes with
// weights (1/4, 1/2, 1/4) per axis; Ampere's law (e_update) is Yee's.  Next
// to the conducting outer walls the averages read E's images: odd across a
// wall the component is tangential to, even across a wall it is normal to.
// ---------------------------------------------------------------------------

// E_c at index (i, j, k) of the grid or of its images (|offset| <= 1 cell
// beyond a wall).
template <typename T, int DIM>
__device__ __forceinline__ T e_img(const Geom& g, const T* __restrict__ E, int c, int i, int j, int k) {
  int x[3] = {i, j, k};
  bool neg = false;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    if (DIM == 2 && b == 1) {
      x[1] = 0;
      continue;
    }
    const int N = g.N[b];
    if (b == c) {              // centred along its own axis: even images
      if (x[b] < 0) x[b] = -1 - x[b];
      else if (x[b] > N - 1) x[b] = 2 * N - 1 - x[b];
    } else {                   // on the nodes of the other axes: odd images
      if (x[b] < 0) {
        x[b] = -x[b];
        neg = !neg;
      } else if (x[b] > N) {
        x[b] = 2 * N - x[b];
        neg = !neg;
      }
    }
  }
  const T v = E[g.idx(x[0], x[1], x[2])];
  return neg ? -v : v;
}

// CK difference of E_c along axis a at the B location of index (i, j, k).
template <typename T, int DIM>
__device__ __forceinline__ T ck_diff(const Geom& g, const T* __restrict__ E, int c, int a, int i, int j, int k) {
  const int b = (a + 1) % 3, d = (a + 2) % 3;
  T acc = T(0);
#pragma unroll
  for (int p = -1; p <= 1; ++p)
#pragma unroll
    for (int q = -1; q <= 1; ++q) {
      const bool flat_b = DIM == 2 && b == 1, flat_d = DIM == 2 && d == 1;
      if ((flat_b && p != 0) || (flat_d && q != 0)) continue;
      const T w = (flat_b ? T(1) : (p == 0 ? T(0.5) : T(0.25))) * (flat_d ? T(1) : (q == 0 ? T(0.5) : T(0.25)));
      int n0[3] = {i, j, k};
      n0[b] += p;
      n0[d] += q;
      int n1[3] = {n0[0], n0[1], n0[2]};
      n1[a] += 1;
      acc += w * (e_img<T, DIM>(g, E, c, n1[0], n1[1], n1[2]) - e_img<T, DIM>(g, E, c, n0[0], n0[1], n0[2]));
    }
  return acc;
}

// B^{n+3/2} at node (i,j,k) into Bp with the CK differences (b_update's
// split-field treatment otherwise), and (B^{n+1/2} + B^{n+3/2})/2 into Bn
// where asked for.
template <typename T, int DIM, int SPL>
__device__ __forceinline__ void b_update_ck(const Geom& g, const Tables& tb, const FieldPtrs<T>& f, int i, int j,
                                            int k, long long id) {
  const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2];
  const T Sx = courant<T>(g, 0), Sy = courant<T>(g, 1), Sz = courant<T>(g, 2);
  const bool jc = DIM == 2 || j <= N1 - 1;
  const bool ic = i <= N0 - 1;
  const bool kc = k <= N2 - 1;
  const float sxc = ic ? tb.sdtf_c[0][i] : 0.f;
  const float syc = DIM == 3 && jc ? tb.sdtf_c[1][j] : 0.f;
  const float szc = kc ? tb.sdtf_c[2][k] : 0.f;
  const bool px = ic && pml_cent(g, 0, i);
  const bool py = DIM == 3 && jc && pml_cent(g, 1, j);
  const bool pz = kc && pml_cent(g, 2, k);
  const bool okx = jc && kc, oky = ic && kc, okz = ic && jc;
  const bool spx = okx && (py || pz), spy = oky && (px || pz), spz = okz && (px || py);
  const T* __restrict__ Ex = f.E[0];
  const T* __restrict__ Ey = f.E[1];
  const T* __restrict__ Ez = f.E[2];
  if (okx) {
    const T r0 = DIM == 3 ? -Sy * ck_diff<T, DIM>(g, Ez, 2, 1, i, j, k) : T(0);
    const T r1 = Sz * ck_diff<T, DIM>(g, Ey, 1, 2, i, j, k);
    if (spx) {
      Parts<SPL> q = load_parts<SPL>(f.Bs[0], id);
      const T b1 = advance<T, SPL, true>(tb, q, DIM == 3 ? 1 : -1, j, 2, k, r0, r1, T(0), syc, szc);
      f.Bp[0][id] = b1;
      store_parts<SPL>(f.Bs[0], id, q);
      if (f.Bn[0]) f.Bn[0][id] = T(0.5) * (f.Bh[0][id] + b1);
    } else {
      const T b0 = f.Bh[0][id], b1 = b0 + (r0 + r1);
      f.Bp[0][id] = b1;
      if (f.Bn[0]) f.Bn[0][id] = T(0.5) * (b0 + b1);
    }
  }
  if (oky) {
    const T r0 = Sx * ck_diff<T, DIM>(g, Ez, 2, 0, i, j, k);
    const T r1 = -Sz * ck_diff<T, DIM>(g, Ex, 0, 2, i, j, k);
    if (spy) {
      Parts<SPL> q = load_parts<SPL>(f.Bs[1], id);
      const T b1 = advance<T, SPL, true>(tb, q, 0, i, 2, k, r0, r1, T(0), sxc, szc);
      f.Bp[1][id] = b1;
      store_parts<SPL>(f.Bs[1], id, q);
      if (f.Bn[0]) f.Bn[1][id] = T(0.5) * (f.Bh[1][id] + b1);
    } else {
      const T b0 = f.Bh[1][id], b1 = b0 + (r0 + r1);
      f.Bp[1][id] = b1;
      if (f.Bn[0]) f.Bn[1][id] = T(0.5) * (b0 + b1);
    }
  }
  if (okz) {
    const T r0 = -Sx * ck_diff<T, DIM>(g, Ey, 1, 0, i, j, k);
    const T r1 = DIM == 3 ? Sy * ck_diff<T, DIM>(g, Ex, 0, 1, i, j, k) : T(0);
    if (spz) {
      Parts<SPL> q = load_parts<SPL>(f.Bs[2], id);
      const T b1 = advance<T, SPL, true>(tb, q, 0, i, DIM == 3 ? 1 : -1, j, r0, r1, T(0), sxc, syc);
      f.Bp[2][id] = b1;
      store_parts<SPL>(f.Bs[2], id, q);
      if (f.Bn[0]) f.Bn[2][id] = T(0.5) * (f.Bh[2][id] + b1);
    } else {
      const T b0 = f.Bh[2][id], b1 = b0 + (r0 + r1);
      f.Bp[2][id] = b1;
      if (f.Bn[0]) f.Bn[2][id] = T(0.5) * (b0 + b1);
    }
  }
}

}  // namespace fn
}  // namespace picpml
