// Device helpers shared by the particle kernels: record I/O, B-spline
// weights, gather, Boris rotation, the float-float move, Esirkepov shape
// arrays and the alpha tables.
#pragma once

#include "picpml_internal.cuh"

namespace picpml {
namespace pc {

template <typename T>
struct PIO;

template <>
struct PIO<float> {
  __device__ static void load(const void* pos, const void* mom, long long p, float o[3], float& w,
                              float u[3], int& cell) {
    float4 a = reinterpret_cast<const float4*>(pos)[p];
    float4 b = reinterpret_cast<const float4*>(mom)[p];
    o[0] = a.x; o[1] = a.y; o[2] = a.z; w = a.w;
    u[0] = b.x; u[1] = b.y; u[2] = b.z; cell = __float_as_int(b.w);
  }
  __device__ static void store(void* pos, void* mom, long long p, const float o[3], float w,
                               const float u[3], int cell) {
    reinterpret_cast<float4*>(pos)[p] = make_float4(o[0], o[1], o[2], w);
    reinterpret_cast<float4*>(mom)[p] = make_float4(u[0], u[1], u[2], __int_as_float(cell));
  }
  __device__ static void save(void* sv, long long p, const float o[3], int cell) {
    reinterpret_cast<float4*>(sv)[p] = make_float4(o[0], o[1], o[2], __int_as_float(cell));
  }
  __device__ static void restore(const void* sv, long long p, float o[3], int& cell) {
    float4 a = reinterpret_cast<const float4*>(sv)[p];
    o[0] = a.x; o[1] = a.y; o[2] = a.z; cell = __float_as_int(a.w);
  }
};

template <>
struct PIO<double> {
  __device__ static void load(const void* pos, const void* mom, long long p, double o[3], double& w,
                              double u[3], int& cell) {
    dbl4 a = reinterpret_cast<const dbl4*>(pos)[p];
    dbl4 b = reinterpret_cast<const dbl4*>(mom)[p];
    o[0] = a.x; o[1] = a.y; o[2] = a.z; w = a.w;
    u[0] = b.x; u[1] = b.y; u[2] = b.z; cell = (int)__double_as_longlong(b.w);
  }
  __device__ static void store(void* pos, void* mom, long long p, const double o[3], double w,
                               const double u[3], int cell) {
    dbl4 a; a.x = o[0]; a.y = o[1]; a.z = o[2]; a.w = w;
    dbl4 b; b.x = u[0]; b.y = u[1]; b.z = u[2]; b.w = __longlong_as_double((long long)cell);
    reinterpret_cast<dbl4*>(pos)[p] = a;
    reinterpret_cast<dbl4*>(mom)[p] = b;
  }
  __device__ static void save(void* sv, long long p, const double o[3], int cell) {
    dbl4 a; a.x = o[0]; a.y = o[1]; a.z = o[2]; a.w = __longlong_as_double((long long)cell);
    reinterpret_cast<dbl4*>(sv)[p] = a;
  }
  __device__ static void restore(const void* sv, long long p, double o[3], int& cell) {
    dbl4 a = reinterpret_cast<const dbl4*>(sv)[p];
    o[0] = a.x; o[1] = a.y; o[2] = a.z; cell = (int)__double_as_longlong(a.w);
  }
};

// False for NaN and infinities (and values beyond 1e30, which no momentum or
// weight of a run reaches).
template <typename T>
__device__ __forceinline__ bool finite_value(T v) { return fabs(v) < T(1e30); }

// B-spline weights of the ORDER+1 nodes around a point at offset f in [0,1)
// from node `base` (nodes base - (ORDER==3) ... base - (ORDER==3) + ORDER).
template <int ORDER, typename T>
__device__ __forceinline__ void bspline(T f, T* w) {
  if (ORDER == 1) {
    w[0] = T(1) - f;
    w[1] = f;
  } else {
    const T g = T(1) - f;
    w[0] = g * g * g * T(1.0 / 6.0);
    w[1] = T(2.0 / 3.0) - f * f + T(0.5) * f * f * f;
    w[2] = T(2.0 / 3.0) - g * g + T(0.5) * g * g * g;
    w[3] = f * f * f * T(1.0 / 6.0);
  }
}

// Gather weights along one axis for stagger 0 (nodes) and 1/2 (centres):
// lowest node index and ORDER+1 weights.
template <int ORDER, typename T>
__device__ __forceinline__ void axis_weights(int ic, T f, int& b0, T* w0, int& bh, T* wh) {
  constexpr int lo = ORDER == 3 ? 1 : 0;
  b0 = ic - lo;
  bspline<ORDER, T>(f, w0);
  if (f >= T(0.5)) {
    bh = ic - lo;
    bspline<ORDER, T>(f - T(0.5), wh);
  } else {
    bh = ic - 1 - lo;
    bspline<ORDER, T>(f + T(0.5), wh);
  }
}

template <int ORDER, int DIM, typename T>
__device__ __forceinline__ T interp(const Geom& g, const T* __restrict__ F, int bx, const T* wx, int by,
                                    const T* wy, int bz, const T* wz) {
  constexpr int W = ORDER + 1;
  T acc = T(0);
#pragma unroll
  for (int tz = 0; tz < W; ++tz) {
#pragma unroll
    for (int ty = 0; ty < (DIM == 3 ? W : 1); ++ty) {
      const T wyz = (DIM == 3 ? wy[ty] : T(1)) * wz[tz];
      const long long row = g.idx(bx, DIM == 3 ? by + ty : 0, bz + tz);
      T racc = T(0);
#pragma unroll
      for (int tx = 0; tx < W; ++tx) racc += wx[tx] * __ldg(F + row + tx);
      acc += wyz * racc;
    }
  }
  return acc;
}

// B^n = (B^{n-1/2} + B^{n+1/2})/2 at the particle.
template <int ORDER, int DIM, typename T>
__device__ __forceinline__ T interp_avg(const Geom& g, const T* __restrict__ F1, const T* __restrict__ F2,
                                        int bx, const T* wx, int by, const T* wy, int bz, const T* wz) {
  return T(0.5) * (interp<ORDER, DIM, T>(g, F1, bx, wx, by, wy, bz, wz) +
                   interp<ORDER, DIM, T>(g, F2, bx, wx, by, wy, bz, wz));
}

__device__ __forceinline__ float inv_sqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double inv_sqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float fast_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fast_div(double a, double b) { return a / b; }

// Boris rotation for u = p/(mc), ke = q dt/(2 m c), fields E' and B' = cB.
// FP32 uses the hardware reciprocal square root and division (a few ulp;
// the rotation is norm-preserving for any t, so these round-offs do not
// accumulate systematically).
template <typename T>
__device__ __forceinline__ void boris(T u[3], const T E[3], const T B[3], T ke) {
  T um[3], t[3], s[3], uq[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) um[a] = u[a] + ke * E[a];
  const T kb = ke * inv_sqrt(T(1) + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
#pragma unroll
  for (int a = 0; a < 3; ++a) t[a] = kb * B[a];
  const T t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  const T f2 = fast_div(T(2), T(1) + t2);
#pragma unroll
  for (int a = 0; a < 3; ++a) s[a] = f2 * t[a];
  uq[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
  uq[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
  uq[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
  u[0] = um[0] + (uq[1] * s[2] - uq[2] * s[1]) + ke * E[0];
  u[1] = um[1] + (uq[2] * s[0] - uq[0] * s[2]) + ke * E[1];
  u[2] = um[2] + (uq[0] * s[1] - uq[1] * s[0]) + ke * E[2];
}

// Error-free transformations for the FP32 move (Dekker/Knuth): the displacement
// S u / gamma is formed in float-float arithmetic so the in-cell offset only
// carries the final rounding, not a systematic per-step error that would
// accumulate along a trajectory with nearly constant u.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// New offset o + S u / gamma for FP32 (float-float), plain for FP64.
template <typename T>
struct Mover;

template <>
struct Mover<float> {
  float ih, il;  // 1/gamma as a float-float pair
  __device__ __forceinline__ Mover(const float u[3]) {
    float sh = 1.0f, sl = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float p, e, t, f;
      two_prod(u[a], u[a], p, e);
      two_sum(sh, p, t, f);
      sh = t;
      sl = __fadd_rn(sl, __fadd_rn(f, e));
    }
    // 1/gamma = (sh + sl)^(-1/2): hardware estimate plus one Newton step with
    // the residual r = 1 - s y^2 formed from exact products, so the pair
    // (ih, il) carries about twice the FP32 precision.
    const float y = rsqrtf(sh);
    float y2, y2e;
    two_prod(y, y, y2, y2e);
    float r = __fmaf_rn(-sh, y2, 1.0f);
    r = __fmaf_rn(-sh, y2e, r);
    r = __fmaf_rn(-sl, y2, r);
    ih = y;
    il = __fmul_rn(__fmul_rn(0.5f, y), r);
  }
  // returns the displacement S u / gamma as a float-float pair
  __device__ __forceinline__ void disp(float Sh, float Sl, float ua, float& dh, float& dl) const {
    float suh, sul;
    two_prod(Sh, ua, suh, sul);
    sul = __fmaf_rn(Sl, ua, sul);
    float p, e;
    two_prod(suh, ih, p, e);
    dh = p;
    dl = __fadd_rn(e, __fadd_rn(__fmul_rn(suh, il), __fmul_rn(sul, ih)));
  }
  __device__ __forceinline__ float advance(float o, float Sh, float Sl, float ua) const {
    float dh, dl, s, e;
    disp(Sh, Sl, ua, dh, dl);
    two_sum(o, dh, s, e);
    return __fadd_rn(s, __fadd_rn(e, dl));
  }
  __device__ __forceinline__ float inv_gamma() const { return __fadd_rn(ih, il); }
};

template <>
struct Mover<double> {
  double ig;
  __device__ __forceinline__ Mover(const double u[3]) {
    ig = 1.0 / sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  }
  __device__ __forceinline__ double advance(double o, double Sh, double, double ua) const {
    return o + Sh * ua * ig;
  }
  __device__ __forceinline__ double inv_gamma() const { return ig; }
};

template <typename T>
__device__ __forceinline__ const T* al_node(const Tables& tb, int a);
template <>
__device__ __forceinline__ const float* al_node<float>(const Tables& tb, int a) { return tb.al_nf[a]; }
template <>
__device__ __forceinline__ const double* al_node<double>(const Tables& tb, int a) { return tb.al_nd[a]; }
template <typename T>
__device__ __forceinline__ const T* al_cent(const Tables& tb, int a);
template <>
__device__ __forceinline__ const float* al_cent<float>(const Tables& tb, int a) { return tb.al_cf[a]; }
template <>
__device__ __forceinline__ const double* al_cent<double>(const Tables& tb, int a) { return tb.al_cd[a]; }

// Weight damping (the alternative scheme of the paper's discussion of
// limitations): alpha = 1 in the deposit, and a macroparticle's weight decays
// as w exp(-int sigma(x(t))/eps0 dt) along its own path, summed over the
// faces.  Per step the integral is the trapezoid rule on the straight move,
// I = (dt s(x0) + dt s(x1)) / 2; the step's current uses w exp(-I/2), the
// weight then becomes w exp(-I).  Depths in cells from cell index + offset.
template <typename T>
__device__ __forceinline__ T pml_depth(const Geom& g, int a, int c, T o) {
  const int lo = g.plo[a], hi = g.plo[a] + g.nph[a];
  if (c < lo) return T(lo - c) - o;
  if (c >= hi) return T(c - hi) + o;
  return T(0);
}
template <typename T>
__device__ __forceinline__ T sdt_at_depth(const Geom& g, int a, T d) {
  if (!(d > T(0))) return T(0);
  const T x = d * T(g.winv_delta);
  const T p = T(g.wexp);
  const T xp = p == T(2) ? x * x : (p == T(1) ? x : (p == T(0) ? T(1) : pow(x, p)));
  return T(g.wk[a]) * xp;
}
template <typename T>
__device__ __forceinline__ T weight_exponent(const Geom& g, const int c0[3], const T o0[3], const int c1[3],
                                             const T o1[3]) {
  T sum = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (g.dim == 2 && a == 1) continue;
    sum += sdt_at_depth<T>(g, a, pml_depth<T>(g, a, c0[a], o0[a]));
    sum += sdt_at_depth<T>(g, a, pml_depth<T>(g, a, c1[a], o1[a]));
  }
  return T(0.5) * sum;
}

// Old (S0) and new (S1) shape values on the ORDER+2 nodes starting at
// min(i0,i1) - (ORDER==3).
template <int ORDER, typename T>
__device__ __forceinline__ void esk_axis(int i0, T f0, int i1, T f1, int& lo, T* S0, T* DS) {
  constexpr int W = ORDER + 2;
  const int b = min(i0, i1);
  lo = b - (ORDER == 3 ? 1 : 0);
  T w0[ORDER + 1], w1[ORDER + 1];
  bspline<ORDER, T>(f0, w0);
  bspline<ORDER, T>(f1, w1);
  const bool s0 = i0 != b, s1 = i1 != b;
#pragma unroll
  for (int t = 0; t < W; ++t) {
    T a = s0 ? (t >= 1 ? w0[t - 1] : T(0)) : (t <= ORDER ? w0[t] : T(0));
    T c = s1 ? (t >= 1 ? w1[t - 1] : T(0)) : (t <= ORDER ? w1[t] : T(0));
    S0[t] = a;
    DS[t] = c - a;
  }
}

// Esirkepov deposition of one move, damped by alpha at each component's
// staggered location, accumulated with global atomics.
template <int ORDER, int DIM, typename T>
__device__ __forceinline__ void deposit_one(const Geom& g, const Tables& tb, const FieldPtrs<T>& f,
                                            const SpeciesPtrs<T>& sp, const int c0[3], const T o0[3],
                                            const int c1[3], const T o1[3], T w, T vy) {
  constexpr int W = ORDER + 2;
  int lo[3];
  T S0[3][W], DS[3][W];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (DIM == 2 && a == 1) {
      lo[1] = 0;
#pragma unroll
      for (int t = 0; t < W; ++t) S0[1][t] = DS[1][t] = T(0);
      continue;
    }
    esk_axis<ORDER, T>(c0[a], o0[a], c1[a], o1[a], lo[a], S0[a], DS[a]);
  }
  const T* anx = al_node<T>(tb, 0);
  const T* acx = al_cent<T>(tb, 0);
  const T* any = al_node<T>(tb, 1);
  const T* acy = al_cent<T>(tb, 1);
  const T* anz = al_node<T>(tb, 2);
  const T* acz = al_cent<T>(tb, 2);
  // transverse factor S0 S0' + DS S0'/2 + S0 DS'/2 + DS DS'/3 = M M' + Q DS'
  // with the mid-move shape M = S0 + DS/2 and Q = DS/12 (1/3 = 1/4 + 1/12)
  T M[3][W], Q[3][W];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int t = 0; t < W; ++t) {
      M[a][t] = (DIM == 2 && a == 1) ? T(t == 0) : S0[a][t] + T(0.5) * DS[a][t];
      Q[a][t] = (DIM == 2 && a == 1) ? T(0) : T(1.0 / 12.0) * DS[a][t];
    }
  if (DIM == 3) {
    const T qx = sp.cj[0] * w, qy = sp.cj[1] * w, qz = sp.cj[2] * w;
    // J_x: prefix sums along x of W_x = DSx (S0y S0z + DSy S0z/2 + S0y DSz/2 + DSy DSz/3)
#pragma unroll
    for (int kz = 0; kz < W; ++kz)
#pragma unroll
      for (int jy = 0; jy < W; ++jy) {
        const T Tl = M[1][jy] * M[2][kz] + Q[1][jy] * DS[2][kz];
        if (Tl == T(0)) continue;
        const T line = qx * Tl * any[lo[1] + jy] * anz[lo[2] + kz];
        const long long row = g.idx(lo[0], lo[1] + jy, lo[2] + kz);
        T acc = T(0);
#pragma unroll
        for (int ix = 0; ix < W - 1; ++ix) {
          acc += DS[0][ix];
          if (acc != T(0)) atomicAdd(f.J[0] + row + ix, line * acc * acx[lo[0] + ix]);
        }
      }
    // J_y
#pragma unroll
    for (int kz = 0; kz < W; ++kz)
#pragma unroll
      for (int ix = 0; ix < W; ++ix) {
        const T Tl = M[0][ix] * M[2][kz] + Q[0][ix] * DS[2][kz];
        if (Tl == T(0)) continue;
        const T line = qy * Tl * anx[lo[0] + ix] * anz[lo[2] + kz];
        T acc = T(0);
#pragma unroll
        for (int jy = 0; jy < W - 1; ++jy) {
          acc += DS[1][jy];
          if (acc != T(0))
            atomicAdd(f.J[1] + g.idx(lo[0] + ix, lo[1] + jy, lo[2] + kz), line * acc * acy[lo[1] + jy]);
        }
      }
    // J_z
#pragma unroll
    for (int jy = 0; jy < W; ++jy)
#pragma unroll
      for (int ix = 0; ix < W; ++ix) {
        const T Tl = M[0][ix] * M[1][jy] + Q[0][ix] * DS[1][jy];
        if (Tl == T(0)) continue;
        const T line = qz * Tl * anx[lo[0] + ix] * any[lo[1] + jy];
        T acc = T(0);
#pragma unroll
        for (int kz = 0; kz < W - 1; ++kz) {
          acc += DS[2][kz];
          if (acc != T(0))
            atomicAdd(f.J[2] + g.idx(lo[0] + ix, lo[1] + jy, lo[2] + kz), line * acc * acz[lo[2] + kz]);
        }
      }
  } else {
    const T qx = sp.cj[0] * w, qz = sp.cj[2] * w, qy = sp.cjy2d * w * vy;
    // J_x: prefix along x of W_x = DSx (S0z + DSz/2)
#pragma unroll
    for (int kz = 0; kz < W; ++kz) {
      const T Tl = M[2][kz];
      if (Tl == T(0)) continue;
      const T line = qx * Tl * anz[lo[2] + kz];
      const long long row = g.idx(lo[0], 0, lo[2] + kz);
      T acc = T(0);
#pragma unroll
      for (int ix = 0; ix < W - 1; ++ix) {
        acc += DS[0][ix];
        if (acc != T(0)) atomicAdd(f.J[0] + row + ix, line * acc * acx[lo[0] + ix]);
      }
    }
    // J_z: prefix along z of W_z = DSz (S0x + DSx/2)
#pragma unroll
    for (int ix = 0; ix < W; ++ix) {
      const T Tl = M[0][ix];
      if (Tl == T(0)) continue;
      const T line = qz * Tl * anx[lo[0] + ix];
      T acc = T(0);
#pragma unroll
      for (int kz = 0; kz < W - 1; ++kz) {
        acc += DS[2][kz];
        if (acc != T(0)) atomicAdd(f.J[2] + g.idx(lo[0] + ix, 0, lo[2] + kz), line * acc * acz[lo[2] + kz]);
      }
    }
    // J_y (out of plane): v_y times the time-averaged shape
    if (qy != T(0)) {
#pragma unroll
      for (int kz = 0; kz < W; ++kz)
#pragma unroll
        for (int ix = 0; ix < W; ++ix) {
          const T Wy = M[0][ix] * M[2][kz] + Q[0][ix] * DS[2][kz];
          if (Wy != T(0))
            atomicAdd(f.J[1] + g.idx(lo[0] + ix, 0, lo[2] + kz), qy * Wy * anx[lo[0] + ix] * anz[lo[2] + kz]);
        }
    }
  }
}


// ---------------------------------------------------------------------------
// Deterministic deposition (3D): the only floating-point decisions are per
// particle and in a fixed operation order (explicitly rounded intrinsics, no
// contraction), so the int64 sums do not depend on the order in which
// particles reach the grid.
//   1. Shape values of the old and new offsets in FP32, quantised to
//      2^-20: S = rint(s 2^20); one node per axis (the node at offset f for
//      order 1, the second node for order 3) takes 2^20 minus the others so
//      every shape sums to 2^20 exactly.
//   2. Esirkepov's decomposition in exact integers, scaled by 6:
//      6 W_x = DSx (6 S0y S0z + 3 DSy S0z + 3 S0y DSz + 2 DSy DSz), prefix
//      sums along x (likewise y, z); the continuity equation then holds
//      exactly in integers.
//   3. One rounding per node, in integers: with the particle's
//      Wq = rint((w q/e) 2^28) (one FP64 product, rounded once),
//      val = round((acc Wq) 2^-64), halves up, from the exact 128-bit
//      product (fix_scale), added with an int64 atomic.
// ---------------------------------------------------------------------------
template <int ORDER>
__device__ __forceinline__ void fixed_shape(float f, long long* w) {
  const float scale = (float)(1 << kFixShapeBits);
  const long long one = 1LL << kFixShapeBits;
  if (ORDER == 1) {
    w[1] = __float2ll_rn(__fmul_rn(f, scale));
    w[0] = one - w[1];
  } else {
    const float g = __fsub_rn(1.0f, f);
    const float sixth = (float)(1.0 / 6.0), twothird = (float)(2.0 / 3.0);
    const float s0 = __fmul_rn(__fmul_rn(__fmul_rn(g, g), g), sixth);
    const float s2 = __fadd_rn(__fsub_rn(twothird, __fmul_rn(g, g)), __fmul_rn(__fmul_rn(__fmul_rn(0.5f, g), g), g));
    const float s3 = __fmul_rn(__fmul_rn(__fmul_rn(f, f), f), sixth);
    w[0] = __float2ll_rn(__fmul_rn(s0, scale));
    w[2] = __float2ll_rn(__fmul_rn(s2, scale));
    w[3] = __float2ll_rn(__fmul_rn(s3, scale));
    w[1] = one - w[0] - w[2] - w[3];
  }
}

template <int ORDER>
__device__ __forceinline__ int fixed_axis(int c0, float f0, int c1, float f1, long long* S0, long long* DS) {
  constexpr int W = ORDER + 2;
  const int b = min(c0, c1);
  long long w0[ORDER + 1], w1[ORDER + 1];
  fixed_shape<ORDER>(f0, w0);
  fixed_shape<ORDER>(f1, w1);
  const bool s0 = c0 != b, s1 = c1 != b;
#pragma unroll
  for (int t = 0; t < W; ++t) {
    const long long a = s0 ? (t >= 1 ? w0[t - 1] : 0) : (t <= ORDER ? w0[t] : 0);
    const long long c = s1 ? (t >= 1 ? w1[t - 1] : 0) : (t <= ORDER ? w1[t] : 0);
    S0[t] = a;
    DS[t] = c - a;
  }
  return b - (ORDER == 3 ? 1 : 0);
}

template <int ORDER>
__device__ __forceinline__ void deposit_fixed(const Geom& g, const FieldPtrs<float>& f, double qn, const int c0[3],
                                              const float o0[3], const int c1[3], const float o1[3], float w,
                                              unsigned* status) {
  constexpr int W = ORDER + 2;
  long long S0[3][W], DS[3][W];
  int lo[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) lo[a] = fixed_axis<ORDER>(c0[a], o0[a], c1[a], o1[a], S0[a], DS[a]);
  const double wq = __dmul_rn((double)w, qn);
  if (!(fabs(wq) <= kFixMaxWq)) {
    atomicOr(status, ST_FIXED_OVERFLOW);
    return;
  }
  const long long Wq = __double2ll_rn(__dmul_rn(wq, kFixWqScale));
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int b = c == 0 ? 1 : 0, d = c == 2 ? 1 : 2;   // transverse axes, b < d
#pragma unroll
    for (int tb = 0; tb < W; ++tb)
#pragma unroll
      for (int td = 0; td < W; ++td) {
        const long long T = 6 * S0[b][tb] * S0[d][td] + 3 * DS[b][tb] * S0[d][td] + 3 * S0[b][tb] * DS[d][td] +
                            2 * DS[b][tb] * DS[d][td];
        if (T == 0) continue;
        long long acc = 0;
#pragma unroll
        for (int ta = 0; ta < W - 1; ++ta) {
          acc += DS[c][ta] * T;
          if (acc == 0) continue;
          int idx[3];
          idx[c] = lo[c] + ta;
          idx[b] = lo[b] + tb;
          idx[d] = lo[d] + td;
          const long long v = fix_scale<36 + kFixWqBits>(acc, Wq);
          atomicAdd(reinterpret_cast<unsigned long long*>(f.Jq[c] + g.idx(idx[0], idx[1], idx[2])),
                    static_cast<unsigned long long>(v));
        }
      }
  }
}

// The 2D (x, z) form: J_x and J_z from the in-plane integer sums,
// 6 W_x = DSx (6 S0z + 3 DSz) (units 2^-40, so the scale is 2^-16 for the
// same unit e/(6 2^24): val = round((acc Wq) 2^-44)); J_y (out of the plane) from the mid-move
// shape product 6 S0x S0z + 3 DSx S0z + 3 S0x DSz + 2 DSx DSz times v_y/c,
// which is formed in FP64 from the FP32 momentum with correctly rounded
// operations in a fixed order, u_y / sqrt(((1 + u_x^2) + u_y^2) + u_z^2).
template <int ORDER>
__device__ __forceinline__ void deposit_fixed2d(const Geom& g, const FieldPtrs<float>& f, double qn, const int c0[3],
                                                const float o0[3], const int c1[3], const float o1[3], float w,
                                                const float u[3], unsigned* status) {
  constexpr int W = ORDER + 2;
  constexpr double kDown2 = 1.0 / 65536.0;   // 2^-16
  long long S0[2][W], DS[2][W];
  const int lox = fixed_axis<ORDER>(c0[0], o0[0], c1[0], o1[0], S0[0], DS[0]);
  const int loz = fixed_axis<ORDER>(c0[2], o0[2], c1[2], o1[2], S0[1], DS[1]);
  const double wq = __dmul_rn((double)w, qn);
  if (!(fabs(wq) <= kFixMaxWq)) {
    atomicOr(status, ST_FIXED_OVERFLOW);
    return;
  }
  const long long Wq = __double2ll_rn(__dmul_rn(wq, kFixWqScale));
  const double ux = u[0], uy = u[1], uz = u[2];
  const double g2 = __dadd_rn(__dadd_rn(__dadd_rn(1.0, __dmul_rn(ux, ux)), __dmul_rn(uy, uy)), __dmul_rn(uz, uz));
  const double vyc = __ddiv_rn(uy, __dsqrt_rn(g2));
  auto add = [&](int c, int i, int k, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(f.Jq[c] + g.idx(i, 0, k)), static_cast<unsigned long long>(v));
  };
#pragma unroll
  for (int tk = 0; tk < W; ++tk) {   // J_x: prefix sums along x
    const long long T = 6 * S0[1][tk] + 3 * DS[1][tk];
    long long acc = 0;
#pragma unroll
    for (int ti = 0; ti < W - 1; ++ti) {
      acc += DS[0][ti] * T;
      if (acc != 0) add(0, lox + ti, loz + tk, fix_scale<16 + kFixWqBits>(acc, Wq));
    }
  }
#pragma unroll
  for (int ti = 0; ti < W; ++ti) {   // J_z: prefix sums along z
    const long long T = 6 * S0[0][ti] + 3 * DS[0][ti];
    long long acc = 0;
#pragma unroll
    for (int tk = 0; tk < W - 1; ++tk) {
      acc += DS[1][tk] * T;
      if (acc != 0) add(2, lox + ti, loz + tk, fix_scale<16 + kFixWqBits>(acc, Wq));
    }
  }
  if (vyc == 0.0) return;
#pragma unroll
  for (int tk = 0; tk < W; ++tk)     // J_y: mid-move shape product
#pragma unroll
    for (int ti = 0; ti < W; ++ti) {
      const long long T = 6 * S0[0][ti] * S0[1][tk] + 3 * DS[0][ti] * S0[1][tk] + 3 * S0[0][ti] * DS[1][tk] +
                          2 * DS[0][ti] * DS[1][tk];
      if (T == 0) continue;
      const double v = __dmul_rn(__dmul_rn(__dmul_rn(__ll2double_rn(T), wq), vyc), kDown2);
      add(1, lox + ti, loz + tk, __double2ll_rn(v));
    }
}

// Deposit of one 2D particle of a batched run (same arithmetic).
template <int ORDER, typename T>
__device__ __forceinline__ void deposit_run_particle(const Geom& g, const Tables& tb, const FieldPtrs<T>& f,
                                                     const SpeciesPtrs<T>& sp, const int c0[3], const T o0[3],
                                                     const int c1[3], const T o1[3], T w, T vy) {
  deposit_one<ORDER, 2, T>(g, tb, f, sp, c0, o0, c1, o1, w, vy);
}

}  // namespace pc
}  // namespace picpml
