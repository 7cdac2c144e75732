// Particle stages of the PIC step: field gather, Boris push, move, and
// charge-conserving Esirkepov deposition with the PML damping alpha applied
// in the flush to the grid (Eq. MaxwellE source term, Eq. alpha, Sec. II.B).
//
// Positions are an int32 cell index (packed i | j<<10 | k<<20) and an
// in-cell offset in [0,1) per axis, so FP32 keeps a uniform resolution of
// 2^-24 cell over the whole grid.  A move is shorter than one cell (Courant
// condition), so the cell index changes by at most one per axis per step and
// the Esirkepov stencil of a move spans ORDER+2 nodes per axis starting at
// min(old cell, new cell) - (ORDER-1)/2.
#include "picpml_internal.cuh"

namespace picpml {

namespace {

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

// Boris rotation for u = p/(mc), ke = q dt/(2 m c), fields E' and B' = cB.
template <typename T>
__device__ __forceinline__ void boris(T u[3], const T E[3], const T B[3], T ke) {
  T um[3], t[3], s[3], uq[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) um[a] = u[a] + ke * E[a];
  const T gm = sqrt(T(1) + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
  const T kb = ke / gm;
#pragma unroll
  for (int a = 0; a < 3; ++a) t[a] = kb * B[a];
  const T t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  const T f2 = T(2) / (T(1) + t2);
#pragma unroll
  for (int a = 0; a < 3; ++a) s[a] = f2 * t[a];
  uq[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
  uq[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
  uq[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
  u[0] = um[0] + (uq[1] * s[2] - uq[2] * s[1]) + ke * E[0];
  u[1] = um[1] + (uq[2] * s[0] - uq[0] * s[2]) + ke * E[1];
  u[2] = um[2] + (uq[0] * s[1] - uq[1] * s[0]) + ke * E[2];
}

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
  const T third = T(1.0 / 3.0);
  if (DIM == 3) {
    const T qx = sp.cj[0] * w, qy = sp.cj[1] * w, qz = sp.cj[2] * w;
    // J_x: prefix sums along x of W_x = DSx (S0y S0z + DSy S0z/2 + S0y DSz/2 + DSy DSz/3)
#pragma unroll
    for (int kz = 0; kz < W; ++kz)
#pragma unroll
      for (int jy = 0; jy < W; ++jy) {
        const T Tl = S0[1][jy] * S0[2][kz] + T(0.5) * DS[1][jy] * S0[2][kz] +
                     T(0.5) * S0[1][jy] * DS[2][kz] + third * DS[1][jy] * DS[2][kz];
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
        const T Tl = S0[0][ix] * S0[2][kz] + T(0.5) * DS[0][ix] * S0[2][kz] +
                     T(0.5) * S0[0][ix] * DS[2][kz] + third * DS[0][ix] * DS[2][kz];
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
        const T Tl = S0[0][ix] * S0[1][jy] + T(0.5) * DS[0][ix] * S0[1][jy] +
                     T(0.5) * S0[0][ix] * DS[1][jy] + third * DS[0][ix] * DS[1][jy];
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
      const T Tl = S0[2][kz] + T(0.5) * DS[2][kz];
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
      const T Tl = S0[0][ix] + T(0.5) * DS[0][ix];
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
          const T Wy = S0[0][ix] * S0[2][kz] + T(0.5) * DS[0][ix] * S0[2][kz] +
                       T(0.5) * S0[0][ix] * DS[2][kz] + third * DS[0][ix] * DS[2][kz];
          if (Wy != T(0))
            atomicAdd(f.J[1] + g.idx(lo[0] + ix, 0, lo[2] + kz), qy * Wy * anx[lo[0] + ix] * anz[lo[2] + kz]);
        }
    }
  }
}

// MODE 0: push only (saves x^n); MODE 1: deposit only (from saved x^n);
// MODE 2: fused push + deposit.
template <int ORDER, int DIM, typename T, int MODE>
__global__ void __launch_bounds__(256) k_particles(Geom g, Tables tb, FieldPtrs<T> f, SpeciesPtrs<T> sp,
                                                   int prescribed, unsigned* status,
                                                   unsigned long long* pushed_total) {
  const long long n = *sp.n_dev;
  const long long stride = (long long)gridDim.x * blockDim.x;
  unsigned pushed = 0;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    T o[3], u[3], w;
    int cell;
    PIO<T>::load(sp.pos, sp.mom, p, o, w, u, cell);
    if (MODE == 1) {
      int cell0;
      T o0[3];
      PIO<T>::restore(sp.save_pos, p, o0, cell0);
      if (cell < 0 || cell0 < 0) continue;
      const int c0[3] = {cell_i(cell0), cell_j(cell0), cell_k(cell0)};
      const int c1[3] = {cell_i(cell), cell_j(cell), cell_k(cell)};
      const T g2 = sqrt(T(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
      deposit_one<ORDER, DIM, T>(g, tb, f, sp, c0, o0, c1, o, w, u[1] / g2);
      continue;
    }
    if (cell < 0) {
      if (MODE == 0) PIO<T>::save(sp.save_pos, p, o, -1);
      continue;
    }
    int c[3] = {cell_i(cell), cell_j(cell), cell_k(cell)};
    bool bad = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (DIM == 2 && a == 1) continue;
      if (c[a] < g.rmin[a] || c[a] > g.rmax[a] || !(o[a] >= T(0) && o[a] < T(1))) bad = true;
    }
    if (bad) {
      atomicOr(status, ST_BAD_PARTICLE);
      if (MODE == 0) PIO<T>::save(sp.save_pos, p, o, -1);
      continue;
    }
    if (sp.immobile) {
      if (MODE == 0) PIO<T>::save(sp.save_pos, p, o, -1);
      continue;
    }
    if (!prescribed) {
      constexpr int WN = ORDER + 1;
      int b0[3], bh[3];
      T w0[3][WN], wh[3][WN];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (DIM == 2 && a == 1) {
          b0[1] = bh[1] = 0;
#pragma unroll
          for (int t = 0; t < WN; ++t) w0[1][t] = wh[1][t] = T(t == 0);
          continue;
        }
        axis_weights<ORDER, T>(c[a], o[a], b0[a], w0[a], bh[a], wh[a]);
      }
      T E[3], B[3];
      E[0] = interp<ORDER, DIM, T>(g, f.E[0], bh[0], wh[0], b0[1], w0[1], b0[2], w0[2]);
      E[1] = interp<ORDER, DIM, T>(g, f.E[1], b0[0], w0[0], bh[1], wh[1], b0[2], w0[2]);
      E[2] = interp<ORDER, DIM, T>(g, f.E[2], b0[0], w0[0], b0[1], w0[1], bh[2], wh[2]);
      B[0] = interp_avg<ORDER, DIM, T>(g, f.Bh[0], f.Bp[0], b0[0], w0[0], bh[1], wh[1], bh[2], wh[2]);
      B[1] = interp_avg<ORDER, DIM, T>(g, f.Bh[1], f.Bp[1], bh[0], wh[0], b0[1], w0[1], bh[2], wh[2]);
      B[2] = interp_avg<ORDER, DIM, T>(g, f.Bh[2], f.Bp[2], bh[0], wh[0], bh[1], wh[1], b0[2], w0[2]);
      boris<T>(u, E, B, sp.ke);
    }
    ++pushed;
    const T gam = sqrt(T(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const T ig = T(1) / gam;
    int c1[3] = {c[0], c[1], c[2]};
    T o1[3] = {o[0], o[1], o[2]};
    bool out = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (DIM == 2 && a == 1) continue;
      T x = o[a] + T(g.S[a]) * u[a] * ig;
      if (x >= T(1)) {
        x -= T(1);
        c1[a] += 1;
      } else if (x < T(0)) {
        x += T(1);
        c1[a] -= 1;
        if (x >= T(1)) {  // x was a tiny negative number: stay on the node
          x = T(0);
          c1[a] += 1;
        }
      }
      o1[a] = x;
      if (c1[a] < g.rmin[a] || c1[a] > g.rmax[a] || (c1[a] == g.rmax[a] && x > T(0))) out = true;
    }
    const int cell1 = out ? -1 : pack_cell(c1[0], c1[1], c1[2]);
    if (MODE == 0) PIO<T>::save(sp.save_pos, p, o, out ? -1 : cell);
    PIO<T>::store(sp.pos, sp.mom, p, out ? o : o1, w, u, cell1);
    if (MODE == 2 && !out) deposit_one<ORDER, DIM, T>(g, tb, f, sp, c, o, c1, o1, w, u[1] * ig);
  }
  // particles pushed this launch: warp sum, one atomic per warp
  if (MODE != 1 && pushed_total) {
    const unsigned wsum = __reduce_add_sync(0xffffffffu, pushed);
    if ((threadIdx.x & 31) == 0 && wsum) atomicAdd(pushed_total, (unsigned long long)wsum);
  }
}

template <int ORDER, int DIM, typename T>
cudaError_t launch_mode(int mode, const Geom& g, const Tables& tb, const FieldPtrs<T>& f,
                        const SpeciesPtrs<T>& sp, int prescribed, unsigned* status,
                        unsigned long long* pushed, int nsm, cudaStream_t s) {
  long long cap = sp.capacity;
  if (cap <= 0) return cudaSuccess;
  const int threads = 256;
  long long want = (cap + threads - 1) / threads;
  long long maxb = (long long)nsm * 8;
  int blocks = (int)(want < maxb ? want : maxb);
  if (blocks < 1) blocks = 1;
  if (mode == 0)
    k_particles<ORDER, DIM, T, 0><<<blocks, threads, 0, s>>>(g, tb, f, sp, prescribed, status, pushed);
  else if (mode == 1)
    k_particles<ORDER, DIM, T, 1><<<blocks, threads, 0, s>>>(g, tb, f, sp, prescribed, status, pushed);
  else
    k_particles<ORDER, DIM, T, 2><<<blocks, threads, 0, s>>>(g, tb, f, sp, prescribed, status, pushed);
  return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_particles(int mode, int order, const Geom& g, const Tables& tb, const FieldPtrs<T>& f,
                             const SpeciesPtrs<T>& sp, int prescribed, unsigned* status,
                             unsigned long long* pushed, int nsm, cudaStream_t s) {
  if (order == 1) {
    return g.dim == 3 ? launch_mode<1, 3, T>(mode, g, tb, f, sp, prescribed, status, pushed, nsm, s)
                      : launch_mode<1, 2, T>(mode, g, tb, f, sp, prescribed, status, pushed, nsm, s);
  }
  return g.dim == 3 ? launch_mode<3, 3, T>(mode, g, tb, f, sp, prescribed, status, pushed, nsm, s)
                    : launch_mode<3, 2, T>(mode, g, tb, f, sp, prescribed, status, pushed, nsm, s);
}

template cudaError_t launch_particles<float>(int, int, const Geom&, const Tables&, const FieldPtrs<float>&,
                                             const SpeciesPtrs<float>&, int, unsigned*, unsigned long long*, int,
                                             cudaStream_t);
template cudaError_t launch_particles<double>(int, int, const Geom&, const Tables&, const FieldPtrs<double>&,
                                              const SpeciesPtrs<double>&, int, unsigned*, unsigned long long*, int,
                                              cudaStream_t);

}  // namespace picpml
