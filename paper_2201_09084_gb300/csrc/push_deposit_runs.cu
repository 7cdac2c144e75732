// Fused gather + Boris + move + Esirkepov deposit + alpha-damped flush for
// shape order 1, over particles sorted by cell.
//
// A block takes a chunk of 256*P consecutive particles.  The chunk is loaded
// into shared memory with coalesced 16-byte loads (structure of arrays, rows
// padded to P+1 words so the strided per-thread reads are bank-conflict
// free), every thread then processes its own run of P consecutive particles,
// and the updated records go back with coalesced stores.
//
// Deposit: consecutive particles of a sorted run mostly share the Esirkepov
// stencil anchor (per-axis min(old cell, new cell)); the order-1 current of a
// move spans 3 nodes per axis, i.e. 2x3x3 prefix values per component, 54 in
// all.  A thread accumulates them in registers while the anchor stays the same
// and flushes only when it changes.  Because alpha (Eq. alpha) and the charge
// factor depend only on the node, they are applied once per flush, which is
// the "damping fused into the flush to the grid" of Eq. MaxwellE's source
// term.  At the end of a run the lanes of a warp that share one anchor sum
// their accumulators with shuffles, so a dense beam core costs one set of
// global atomics per warp instead of one per particle.
#include "particle_common.cuh"

namespace picpml {

namespace {

using namespace pc;

template <typename T>
__device__ __forceinline__ T cell_to_bits(int c);
template <>
__device__ __forceinline__ float cell_to_bits<float>(int c) { return __int_as_float(c); }
template <>
__device__ __forceinline__ double cell_to_bits<double>(int c) { return __longlong_as_double((long long)c); }
template <typename T>
__device__ __forceinline__ int bits_to_cell(T v);
template <>
__device__ __forceinline__ int bits_to_cell<float>(float v) { return __float_as_int(v); }
template <>
__device__ __forceinline__ int bits_to_cell<double>(double v) { return (int)__double_as_longlong(v); }

// Register accumulator of the order-1 current of a run (values are
// w * (shape factor) sums; the charge factor and alpha are applied at flush).
template <typename T, int DIM>
struct Acc1 {
  static constexpr int NX = DIM == 3 ? 18 : 6;   // Jx: 2 x 3 (x 3)
  static constexpr int NY = DIM == 3 ? 18 : 9;   // Jy: 3 x 2 x 3 (3D) / 3 x 3 (2D, out of plane)
  static constexpr int NZ = DIM == 3 ? 18 : 6;
  T vx[NX], vy[NY], vz[NZ];

  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int t = 0; t < NX; ++t) vx[t] = T(0);
#pragma unroll
    for (int t = 0; t < NY; ++t) vy[t] = T(0);
#pragma unroll
    for (int t = 0; t < NZ; ++t) vz[t] = T(0);
  }

  // 3D layout: vx[ix*9 + jy*3 + kz], vy[ix*6 + jy*3 + kz], vz[ix*6 + jy*2 + kz].
  // Esirkepov's transverse factor S0 S0' + DS S0'/2 + S0 DS'/2 + DS DS'/3 is
  // evaluated as M M' + DS DS'/12 with the mid-move shape M = S0 + DS/2 (the
  // same polynomial, since 1/3 = 1/4 + 1/12); a component whose prefix sums
  // vanish (no motion along its axis) adds nothing and is skipped.
  __device__ __forceinline__ void add(const T S0[3][3], const T DS[3][3], T w, T wvy) {
    const T c12 = T(1.0 / 12.0);
    T M[3][3], Q[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        M[a][t] = S0[a][t] + T(0.5) * DS[a][t];
        Q[a][t] = c12 * DS[a][t];
      }
    if (DIM == 3) {
      const T ax0 = w * DS[0][0], ax1 = w * (DS[0][0] + DS[0][1]);
      if (ax0 != T(0) || ax1 != T(0)) {
#pragma unroll
        for (int jy = 0; jy < 3; ++jy)
#pragma unroll
          for (int kz = 0; kz < 3; ++kz) {
            const T Tl = M[1][jy] * M[2][kz] + Q[1][jy] * DS[2][kz];
            vx[0 * 9 + jy * 3 + kz] += ax0 * Tl;
            vx[1 * 9 + jy * 3 + kz] += ax1 * Tl;
          }
      }
      const T ay0 = w * DS[1][0], ay1 = w * (DS[1][0] + DS[1][1]);
      if (ay0 != T(0) || ay1 != T(0)) {
#pragma unroll
        for (int ix = 0; ix < 3; ++ix)
#pragma unroll
          for (int kz = 0; kz < 3; ++kz) {
            const T Tl = M[0][ix] * M[2][kz] + Q[0][ix] * DS[2][kz];
            vy[ix * 6 + 0 * 3 + kz] += ay0 * Tl;
            vy[ix * 6 + 1 * 3 + kz] += ay1 * Tl;
          }
      }
      const T az0 = w * DS[2][0], az1 = w * (DS[2][0] + DS[2][1]);
      if (az0 != T(0) || az1 != T(0)) {
#pragma unroll
        for (int ix = 0; ix < 3; ++ix)
#pragma unroll
          for (int jy = 0; jy < 3; ++jy) {
            const T Tl = M[0][ix] * M[1][jy] + Q[0][ix] * DS[1][jy];
            vz[ix * 6 + jy * 2 + 0] += az0 * Tl;
            vz[ix * 6 + jy * 2 + 1] += az1 * Tl;
          }
      }
    } else {
      // 2D layout: vx[ix*3 + kz], vz[ix*2 + kz], vy[ix*3 + kz]
      const T ax0 = w * DS[0][0], ax1 = w * (DS[0][0] + DS[0][1]);
#pragma unroll
      for (int kz = 0; kz < 3; ++kz) {
        vx[0 * 3 + kz] += ax0 * M[2][kz];
        vx[1 * 3 + kz] += ax1 * M[2][kz];
      }
      const T az0 = w * DS[2][0], az1 = w * (DS[2][0] + DS[2][1]);
#pragma unroll
      for (int ix = 0; ix < 3; ++ix) {
        vz[ix * 2 + 0] += az0 * M[0][ix];
        vz[ix * 2 + 1] += az1 * M[0][ix];
      }
      if (wvy != T(0)) {
#pragma unroll
        for (int ix = 0; ix < 3; ++ix)
#pragma unroll
          for (int kz = 0; kz < 3; ++kz) vy[ix * 3 + kz] += wvy * (M[0][ix] * M[2][kz] + Q[0][ix] * DS[2][kz]);
      }
    }
  }

  __device__ __forceinline__ void warp_sum() {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int t = 0; t < NX; ++t) vx[t] += __shfl_xor_sync(0xffffffffu, vx[t], off);
#pragma unroll
      for (int t = 0; t < NY; ++t) vy[t] += __shfl_xor_sync(0xffffffffu, vy[t], off);
#pragma unroll
      for (int t = 0; t < NZ; ++t) vz[t] += __shfl_xor_sync(0xffffffffu, vz[t], off);
    }
  }

  // Adds the run's current, times the charge factors and alpha, to the grid.
  __device__ __forceinline__ void flush(const Geom& g, const Tables& tb, const FieldPtrs<T>& f,
                                        const SpeciesPtrs<T>& sp, int key) const {
    const int ax = cell_i(key), ay = DIM == 3 ? cell_j(key) : 0, az = cell_k(key);
    const T* anx = al_node<T>(tb, 0);
    const T* acx = al_cent<T>(tb, 0);
    const T* any = al_node<T>(tb, 1);
    const T* acy = al_cent<T>(tb, 1);
    const T* anz = al_node<T>(tb, 2);
    const T* acz = al_cent<T>(tb, 2);
    if (DIM == 3) {
#pragma unroll
      for (int ix = 0; ix < 2; ++ix)
#pragma unroll
        for (int jy = 0; jy < 3; ++jy)
#pragma unroll
          for (int kz = 0; kz < 3; ++kz) {
            const T v = vx[ix * 9 + jy * 3 + kz];
            if (v != T(0))
              atomicAdd(f.J[0] + g.idx(ax + ix, ay + jy, az + kz),
                        sp.cj[0] * v * acx[ax + ix] * any[ay + jy] * anz[az + kz]);
          }
#pragma unroll
      for (int ix = 0; ix < 3; ++ix)
#pragma unroll
        for (int jy = 0; jy < 2; ++jy)
#pragma unroll
          for (int kz = 0; kz < 3; ++kz) {
            const T v = vy[ix * 6 + jy * 3 + kz];
            if (v != T(0))
              atomicAdd(f.J[1] + g.idx(ax + ix, ay + jy, az + kz),
                        sp.cj[1] * v * anx[ax + ix] * acy[ay + jy] * anz[az + kz]);
          }
#pragma unroll
      for (int ix = 0; ix < 3; ++ix)
#pragma unroll
        for (int jy = 0; jy < 3; ++jy)
#pragma unroll
          for (int kz = 0; kz < 2; ++kz) {
            const T v = vz[ix * 6 + jy * 2 + kz];
            if (v != T(0))
              atomicAdd(f.J[2] + g.idx(ax + ix, ay + jy, az + kz),
                        sp.cj[2] * v * anx[ax + ix] * any[ay + jy] * acz[az + kz]);
          }
    } else {
#pragma unroll
      for (int ix = 0; ix < 2; ++ix)
#pragma unroll
        for (int kz = 0; kz < 3; ++kz) {
          const T v = vx[ix * 3 + kz];
          if (v != T(0))
            atomicAdd(f.J[0] + g.idx(ax + ix, 0, az + kz), sp.cj[0] * v * acx[ax + ix] * anz[az + kz]);
        }
#pragma unroll
      for (int ix = 0; ix < 3; ++ix)
#pragma unroll
        for (int kz = 0; kz < 2; ++kz) {
          const T v = vz[ix * 2 + kz];
          if (v != T(0))
            atomicAdd(f.J[2] + g.idx(ax + ix, 0, az + kz), sp.cj[2] * v * anx[ax + ix] * acz[az + kz]);
        }
#pragma unroll
      for (int ix = 0; ix < 3; ++ix)
#pragma unroll
        for (int kz = 0; kz < 3; ++kz) {
          const T v = vy[ix * 3 + kz];
          if (v != T(0))
            atomicAdd(f.J[1] + g.idx(ax + ix, 0, az + kz), sp.cjy2d * v * anx[ax + ix] * anz[az + kz]);
        }
    }
  }
};

constexpr int kNT = 256;

template <typename T, int DIM, int P>
__global__ void __launch_bounds__(kNT, sizeof(T) == 4 ? 2 : 1) k_pd1(Geom g, Tables tb, FieldPtrs<T> f, SpeciesPtrs<T> sp, int prescribed,
                                             unsigned* status, unsigned long long* pushed_total) {
  constexpr int PP = P + 1;          // padded row: conflict-free strided reads
  constexpr int ROW = kNT * PP;      // one component array in shared memory
  constexpr int C = kNT * P;         // particles per chunk
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const long long n = *sp.n_dev;
  const long long nchunks = (n + C - 1) / C;
  const int lane = threadIdx.x & 31;
  unsigned pushed = 0;
  for (long long ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const long long base = ch * C;
    __syncthreads();
    for (int q = threadIdx.x; q < C; q += kNT) {
      const long long gp = base + q;
      if (gp >= n) break;
      T o[3], u[3], w;
      int cell;
      PIO<T>::load(sp.pos, sp.mom, gp, o, w, u, cell);
      const int slot = (q / P) * PP + (q % P);
      sm[0 * ROW + slot] = o[0];
      sm[1 * ROW + slot] = o[1];
      sm[2 * ROW + slot] = o[2];
      sm[3 * ROW + slot] = w;
      sm[4 * ROW + slot] = u[0];
      sm[5 * ROW + slot] = u[1];
      sm[6 * ROW + slot] = u[2];
      sm[7 * ROW + slot] = cell_to_bits<T>(cell);
    }
    __syncthreads();

    Acc1<T, DIM> acc;
    acc.zero();
    int key = -1;
    for (int i = 0; i < P; ++i) {
      const long long gp = base + (long long)threadIdx.x * P + i;
      if (gp >= n) break;
      const int slot = threadIdx.x * PP + i;
      T o[3] = {sm[0 * ROW + slot], sm[1 * ROW + slot], sm[2 * ROW + slot]};
      const T w = sm[3 * ROW + slot];
      T u[3] = {sm[4 * ROW + slot], sm[5 * ROW + slot], sm[6 * ROW + slot]};
      const int cell = bits_to_cell<T>(sm[7 * ROW + slot]);
      if (cell < 0) continue;
      int c[3] = {cell_i(cell), cell_j(cell), cell_k(cell)};
      bool bad = false;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (DIM == 2 && a == 1) continue;
        if (c[a] < g.rmin[a] || c[a] > g.rmax[a] || !(o[a] >= T(0) && o[a] < T(1))) bad = true;
      }
      if (bad) {
        atomicOr(status, ST_BAD_PARTICLE);
        continue;
      }
      if (!prescribed) {
        int b0[3], bh[3];
        T w0[3][2], wh[3][2];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (DIM == 2 && a == 1) {
            b0[1] = bh[1] = 0;
            w0[1][0] = wh[1][0] = T(1);
            w0[1][1] = wh[1][1] = T(0);
            continue;
          }
          axis_weights<1, T>(c[a], o[a], b0[a], w0[a], bh[a], wh[a]);
        }
        T E[3], B[3];
        E[0] = interp<1, DIM, T>(g, f.E[0], bh[0], wh[0], b0[1], w0[1], b0[2], w0[2]);
        E[1] = interp<1, DIM, T>(g, f.E[1], b0[0], w0[0], bh[1], wh[1], b0[2], w0[2]);
        E[2] = interp<1, DIM, T>(g, f.E[2], b0[0], w0[0], b0[1], w0[1], bh[2], wh[2]);
        B[0] = interp_avg<1, DIM, T>(g, f.Bh[0], f.Bp[0], b0[0], w0[0], bh[1], wh[1], bh[2], wh[2]);
        B[1] = interp_avg<1, DIM, T>(g, f.Bh[1], f.Bp[1], bh[0], wh[0], b0[1], w0[1], bh[2], wh[2]);
        B[2] = interp_avg<1, DIM, T>(g, f.Bh[2], f.Bp[2], bh[0], wh[0], bh[1], wh[1], b0[2], w0[2]);
        boris<T>(u, E, B, sp.ke);
      }
      ++pushed;
      const Mover<T> mv(u);
      int c1[3] = {c[0], c[1], c[2]};
      T o1[3] = {o[0], o[1], o[2]};
      bool out = false;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (DIM == 2 && a == 1) continue;
        const T Sh = sizeof(T) == 4 ? T(g.Sf[a]) : T(g.S[a]);
        const T Sl = sizeof(T) == 4 ? T(g.Sfl[a]) : T(0);
        T x = mv.advance(o[a], Sh, Sl, u[a]);
        if (x >= T(1)) {
          x -= T(1);
          c1[a] += 1;
        } else if (x < T(0)) {
          x += T(1);
          c1[a] -= 1;
          if (x >= T(1)) {
            x = T(0);
            c1[a] += 1;
          }
        }
        o1[a] = x;
        if (c1[a] < g.rmin[a] || c1[a] > g.rmax[a] || (c1[a] == g.rmax[a] && x > T(0))) out = true;
      }
      sm[4 * ROW + slot] = u[0];
      sm[5 * ROW + slot] = u[1];
      sm[6 * ROW + slot] = u[2];
      if (out) {
        sm[7 * ROW + slot] = cell_to_bits<T>(-1);
        continue;
      }
      sm[0 * ROW + slot] = o1[0];
      sm[1 * ROW + slot] = o1[1];
      sm[2 * ROW + slot] = o1[2];
      sm[7 * ROW + slot] = cell_to_bits<T>(pack_cell(c1[0], c1[1], c1[2]));
      // Esirkepov shape arrays on the 3-node stencil from min(old, new) per axis
      int lo[3] = {0, 0, 0};
      T S0[3][3], DS[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (DIM == 2 && a == 1) {
          S0[1][0] = T(1); S0[1][1] = S0[1][2] = T(0);
          DS[1][0] = DS[1][1] = DS[1][2] = T(0);
          continue;
        }
        esk_axis<1, T>(c[a], o[a], c1[a], o1[a], lo[a], S0[a], DS[a]);
      }
      const int k = pack_cell(lo[0], lo[1], lo[2]);
      if (k != key) {
        if (key >= 0) acc.flush(g, tb, f, sp, key);
        acc.zero();
        key = k;
      }
      acc.add(S0, DS, w, w * u[1] * mv.inv_gamma());
    }
    // end of the run: lanes sharing one anchor reduce with shuffles first
    const unsigned same = __match_any_sync(0xffffffffu, key);
    if (same == 0xffffffffu) {
      if (key >= 0) {
        acc.warp_sum();
        if (lane == 0) acc.flush(g, tb, f, sp, key);
      }
    } else if (key >= 0) {
      acc.flush(g, tb, f, sp, key);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < C; q += kNT) {
      const long long gp = base + q;
      if (gp >= n) break;
      const int slot = (q / P) * PP + (q % P);
      const T o[3] = {sm[0 * ROW + slot], sm[1 * ROW + slot], sm[2 * ROW + slot]};
      const T u[3] = {sm[4 * ROW + slot], sm[5 * ROW + slot], sm[6 * ROW + slot]};
      PIO<T>::store(sp.pos, sp.mom, gp, o, sm[3 * ROW + slot], u, bits_to_cell<T>(sm[7 * ROW + slot]));
    }
  }
  if (pushed_total) {
    const unsigned wsum = __reduce_add_sync(0xffffffffu, pushed);
    if (lane == 0 && wsum) atomicAdd(pushed_total, (unsigned long long)wsum);
  }
}

template <typename T, int DIM, int P>
cudaError_t launch_pd1_p(const Geom& g, const Tables& tb, const FieldPtrs<T>& f, const SpeciesPtrs<T>& sp,
                         int prescribed, unsigned* status, unsigned long long* pushed, int nsm, int blocks_per_sm,
                         cudaStream_t s) {
  const size_t smem = (size_t)8 * kNT * (P + 1) * sizeof(T);
  static bool configured = false;  // per template instance, once per process
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_pd1<T, DIM, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const long long C = (long long)kNT * P;
  long long chunks = (sp.capacity + C - 1) / C;
  long long maxb = (long long)nsm * blocks_per_sm;
  int blocks = (int)(chunks < maxb ? chunks : maxb);
  if (blocks < 1) blocks = 1;
  k_pd1<T, DIM, P><<<blocks, kNT, smem, s>>>(g, tb, f, sp, prescribed, status, pushed);
  return cudaGetLastError();
}

}  // namespace

// Particles per thread P of the run kernel; 0 selects the default.
template <typename T>
cudaError_t launch_push_deposit_runs(int ppt, const Geom& g, const Tables& tb, const FieldPtrs<T>& f,
                                     const SpeciesPtrs<T>& sp, int prescribed, unsigned* status,
                                     unsigned long long* pushed, int nsm, cudaStream_t s) {
  if (sp.capacity <= 0) return cudaSuccess;
  const bool d3 = g.dim == 3;
  if (sizeof(T) == 8) {
    if (ppt == 0) ppt = 4;
    if (ppt <= 4) return d3 ? launch_pd1_p<T, 3, 4>(g, tb, f, sp, prescribed, status, pushed, nsm, 2, s)
                            : launch_pd1_p<T, 2, 4>(g, tb, f, sp, prescribed, status, pushed, nsm, 2, s);
    return d3 ? launch_pd1_p<T, 3, 8>(g, tb, f, sp, prescribed, status, pushed, nsm, 1, s)
              : launch_pd1_p<T, 2, 8>(g, tb, f, sp, prescribed, status, pushed, nsm, 1, s);
  }
  if (ppt == 0) ppt = 8;
  if (ppt <= 4) return d3 ? launch_pd1_p<T, 3, 4>(g, tb, f, sp, prescribed, status, pushed, nsm, 3, s)
                          : launch_pd1_p<T, 2, 4>(g, tb, f, sp, prescribed, status, pushed, nsm, 3, s);
  if (ppt <= 8) return d3 ? launch_pd1_p<T, 3, 8>(g, tb, f, sp, prescribed, status, pushed, nsm, 2, s)
                          : launch_pd1_p<T, 2, 8>(g, tb, f, sp, prescribed, status, pushed, nsm, 2, s);
  return d3 ? launch_pd1_p<T, 3, 16>(g, tb, f, sp, prescribed, status, pushed, nsm, 1, s)
            : launch_pd1_p<T, 2, 16>(g, tb, f, sp, prescribed, status, pushed, nsm, 1, s);
}

template cudaError_t launch_push_deposit_runs<float>(int, const Geom&, const Tables&, const FieldPtrs<float>&,
                                                     const SpeciesPtrs<float>&, int, unsigned*, unsigned long long*,
                                                     int, cudaStream_t);
template cudaError_t launch_push_deposit_runs<double>(int, const Geom&, const Tables&, const FieldPtrs<double>&,
                                                      const SpeciesPtrs<double>&, int, unsigned*, unsigned long long*,
                                                      int, cudaStream_t);

}  // namespace picpml
