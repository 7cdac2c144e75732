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

  // Sums the accumulators of each contiguous run of lanes with equal segment
  // id towards the run's first lane (shuffle-down segmented reduction).
  __device__ __forceinline__ void seg_sum(int segid, int lane) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int so = __shfl_down_sync(0xffffffffu, segid, off);
      const bool take = lane + off < 32 && so == segid;
#pragma unroll
      for (int t = 0; t < NX; ++t) {
        const T o = __shfl_down_sync(0xffffffffu, vx[t], off);
        if (take) vx[t] += o;
      }
#pragma unroll
      for (int t = 0; t < NY; ++t) {
        const T o = __shfl_down_sync(0xffffffffu, vy[t], off);
        if (take) vy[t] += o;
      }
#pragma unroll
      for (int t = 0; t < NZ; ++t) {
        const T o = __shfl_down_sync(0xffffffffu, vz[t], off);
        if (take) vz[t] += o;
      }
    }
  }

  // Adds the run's sums into the shared-memory current box (local anchor
  // (ax, ay, az), box row lengths bx, by; arrays J0, J1, J2).
  __device__ __forceinline__ void flush_box(T* J0, T* J1, T* J2, int ax, int ay, int az, int bx, int bxy) const {
    if (DIM == 3) {
#pragma unroll
      for (int ix = 0; ix < 2; ++ix)
#pragma unroll
        for (int jy = 0; jy < 3; ++jy)
#pragma unroll
          for (int kz = 0; kz < 3; ++kz) {
            const T v = vx[ix * 9 + jy * 3 + kz];
            if (v != T(0)) atomicAdd(J0 + (ax + ix) + bx * (ay + jy) + bxy * (az + kz), v);
          }
#pragma unroll
      for (int ix = 0; ix < 3; ++ix)
#pragma unroll
        for (int jy = 0; jy < 2; ++jy)
#pragma unroll
          for (int kz = 0; kz < 3; ++kz) {
            const T v = vy[ix * 6 + jy * 3 + kz];
            if (v != T(0)) atomicAdd(J1 + (ax + ix) + bx * (ay + jy) + bxy * (az + kz), v);
          }
#pragma unroll
      for (int ix = 0; ix < 3; ++ix)
#pragma unroll
        for (int jy = 0; jy < 3; ++jy)
#pragma unroll
          for (int kz = 0; kz < 2; ++kz) {
            const T v = vz[ix * 6 + jy * 2 + kz];
            if (v != T(0)) atomicAdd(J2 + (ax + ix) + bx * (ay + jy) + bxy * (az + kz), v);
          }
    } else {
#pragma unroll
      for (int ix = 0; ix < 2; ++ix)
#pragma unroll
        for (int kz = 0; kz < 3; ++kz) {
          const T v = vx[ix * 3 + kz];
          if (v != T(0)) atomicAdd(J0 + (ax + ix) + bxy * (az + kz), v);
        }
#pragma unroll
      for (int ix = 0; ix < 3; ++ix)
#pragma unroll
        for (int kz = 0; kz < 2; ++kz) {
          const T v = vz[ix * 2 + kz];
          if (v != T(0)) atomicAdd(J2 + (ax + ix) + bxy * (az + kz), v);
        }
#pragma unroll
      for (int ix = 0; ix < 3; ++ix)
#pragma unroll
        for (int kz = 0; kz < 3; ++kz) {
          const T v = vy[ix * 3 + kz];
          if (v != T(0)) atomicAdd(J1 + (ax + ix) + bxy * (az + kz), v);
        }
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

constexpr int kNT = 128;

// Shared memory of one block: the staged chunk (8 words per particle, rows
// padded to P+1), the field/current box (E, time-averaged B, J: 9 arrays of
// NBMAX nodes), the per-cell counters and the permutation of the chunk sort.
template <typename T, int P>
struct Plan {
  static constexpr int PP = P + 1;
  static constexpr int ROW = kNT * PP;
  static constexpr int C = kNT * P;
  static constexpr int NBMAX = sizeof(T) == 4 ? 768 : 384;
  static constexpr size_t stage = (size_t)8 * ROW * sizeof(T);
  static constexpr size_t box = (size_t)9 * NBMAX * sizeof(T);
  static constexpr size_t cnt = (size_t)(NBMAX + 1) * sizeof(int);
  static constexpr size_t perm = (size_t)C * sizeof(unsigned short);
  static constexpr size_t total = stage + box + cnt + perm;
};

// Order-1 interpolation from a shared-memory box (local base indices).
template <int DIM, typename T>
__device__ __forceinline__ T interp_box(const T* F, int bx, int bxy, int li, const T* wx, int lj, const T* wy, int lk,
                                        const T* wz) {
  T acc = T(0);
#pragma unroll
  for (int tz = 0; tz < 2; ++tz)
#pragma unroll
    for (int ty = 0; ty < (DIM == 3 ? 2 : 1); ++ty) {
      const T* row = F + li + bx * (lj + ty) + bxy * (lk + tz);
      acc += (DIM == 3 ? wy[ty] : T(1)) * wz[tz] * (wx[0] * row[0] + wx[1] * row[1]);
    }
  return acc;
}

__device__ __forceinline__ int warp_min(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <typename T, int DIM, int P>
__global__ void __launch_bounds__(kNT, sizeof(T) == 4 ? 3 : 2)
    k_pd1(Geom g, Tables tb, FieldPtrs<T> f, SpeciesPtrs<T> sp, int prescribed, unsigned* status,
          unsigned long long* pushed_total) {
  using PL = Plan<T, P>;
  constexpr int PP = PL::PP, ROW = PL::ROW, C = PL::C, NBMAX = PL::NBMAX;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* stg = reinterpret_cast<T*>(smraw);
  T* bx_ = reinterpret_cast<T*>(smraw + PL::stage);
  int* cnt = reinterpret_cast<int*>(smraw + PL::stage + PL::box);
  unsigned short* perm = reinterpret_cast<unsigned short*>(smraw + PL::stage + PL::box + PL::cnt);
  __shared__ int s_red[6][kNT / 32];
  __shared__ int s_geo[8];   // origin x,y,z; box dims x, y, z; cells per row x, y (of the sort key)
  __shared__ int s_use_box;
  __shared__ int s_scan[kNT / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long n = *sp.n_dev;
  const long long nchunks = (n + C - 1) / C;
  unsigned pushed = 0;

  for (long long ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const long long base = ch * C;
    __syncthreads();
    // ---- 1. stage the chunk (coalesced), mark empty slots ----
    for (int q = tid; q < C; q += kNT) {
      const long long gp = base + q;
      const int slot = (q / P) * PP + (q % P);
      if (gp < n) {
        T o[3], u[3], w;
        int cell;
        PIO<T>::load(sp.pos, sp.mom, gp, o, w, u, cell);
        stg[0 * ROW + slot] = o[0];
        stg[1 * ROW + slot] = o[1];
        stg[2 * ROW + slot] = o[2];
        stg[3 * ROW + slot] = w;
        stg[4 * ROW + slot] = u[0];
        stg[5 * ROW + slot] = u[1];
        stg[6 * ROW + slot] = u[2];
        stg[7 * ROW + slot] = cell_to_bits<T>(cell);
      } else {
        stg[7 * ROW + slot] = cell_to_bits<T>(-1);
      }
    }
    __syncthreads();
    // ---- 2. validate, bounding box of the current cells ----
    int mn[3] = {1 << 30, 1 << 30, 1 << 30}, mx[3] = {-1, -1, -1};
    for (int i = 0; i < P; ++i) {
      const int slot = tid * PP + i;
      const int cell = bits_to_cell<T>(stg[7 * ROW + slot]);
      if (cell < 0) continue;
      const int c[3] = {cell_i(cell), cell_j(cell), cell_k(cell)};
      bool bad = false;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (DIM == 2 && a == 1) continue;
        const T o = stg[a * ROW + slot];
        if (c[a] < g.rmin[a] || c[a] > g.rmax[a] || !(o >= T(0) && o < T(1))) bad = true;
      }
      if (bad || (sp.immobile)) {
        if (bad) {
          atomicOr(status, ST_BAD_PARTICLE);
          stg[7 * ROW + slot] = cell_to_bits<T>(-1);  // removed
        }
        continue;
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        mn[a] = min(mn[a], c[a]);
        mx[a] = max(mx[a], c[a]);
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int lo = warp_min(mn[a]), hi = warp_max(mx[a]);
      if (lane == 0) {
        s_red[a][warp] = lo;
        s_red[3 + a][warp] = hi;
      }
    }
    __syncthreads();
    if (tid == 0) {
      int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-1, -1, -1};
      for (int w8 = 0; w8 < kNT / 32; ++w8)
        for (int a = 0; a < 3; ++a) {
          lo[a] = min(lo[a], s_red[a][w8]);
          hi[a] = max(hi[a], s_red[3 + a][w8]);
        }
      int use = hi[0] >= 0;
      if (DIM == 2) lo[1] = hi[1] = 0;
      const int dx = hi[0] - lo[0] + 4, dy = DIM == 3 ? hi[1] - lo[1] + 4 : 1, dz = hi[2] - lo[2] + 4;
      if (use && (long long)dx * dy * dz > NBMAX) use = 0;
      s_use_box = use;
      s_geo[0] = lo[0] - 1;
      s_geo[1] = DIM == 3 ? lo[1] - 1 : 0;
      s_geo[2] = lo[2] - 1;
      s_geo[3] = dx;
      s_geo[4] = dy;
      s_geo[5] = dz;
    }
    __syncthreads();
    const int use_box = s_use_box;
    const int ox = s_geo[0], oy = s_geo[1], oz = s_geo[2];
    const int bdx = s_geo[3], bdy = s_geo[4], bdz = s_geo[5];
    const int bxy = bdx * bdy;
    const int NB = bdx * bdy * bdz;
    T* const BE0 = bx_;
    T* const BE1 = bx_ + NBMAX;
    T* const BE2 = bx_ + 2 * NBMAX;
    T* const BB0 = bx_ + 3 * NBMAX;
    T* const BB1 = bx_ + 4 * NBMAX;
    T* const BB2 = bx_ + 5 * NBMAX;
    T* const BJ0 = bx_ + 6 * NBMAX;
    T* const BJ1 = bx_ + 7 * NBMAX;
    T* const BJ2 = bx_ + 8 * NBMAX;
    // the sort key is the box-local node of the particle's cell
    if (use_box) {
      // ---- 3. load E and the time-averaged B of the box, zero the J box ----
      for (int t = tid; t < NB; t += kNT) {
        const int li = t % bdx, r = t / bdx, lj = r % bdy, lk = r / bdy;
        const long long gi = g.idx(ox + li, oy + lj, oz + lk);
        BE0[t] = f.E[0][gi];
        BE1[t] = f.E[1][gi];
        BE2[t] = f.E[2][gi];
        BB0[t] = T(0.5) * (f.Bh[0][gi] + f.Bp[0][gi]);
        BB1[t] = T(0.5) * (f.Bh[1][gi] + f.Bp[1][gi]);
        BB2[t] = T(0.5) * (f.Bh[2][gi] + f.Bp[2][gi]);
        BJ0[t] = BJ1[t] = BJ2[t] = T(0);
      }
      for (int t = tid; t <= NB; t += kNT) cnt[t] = 0;
      __syncthreads();
      // ---- 4. counting sort of the chunk by box-local cell (warp-aggregated) ----
      for (int k = 0; k < P; ++k) {
        const int q = tid + k * kNT;
        const int slot = (q / P) * PP + (q % P);
        const int cell = bits_to_cell<T>(stg[7 * ROW + slot]);
        const int key = cell < 0 ? NB : (cell_i(cell) - ox) + bdx * ((DIM == 3 ? cell_j(cell) - oy : 0) + bdy * (cell_k(cell) - oz));
        const unsigned m = __match_any_sync(0xffffffffu, key);
        if (lane == __ffs(m) - 1) atomicAdd(cnt + key, __popc(m));
      }
      __syncthreads();
      // exclusive scan of cnt[0..NB]
      {
        const int per = (NB + 1 + kNT - 1) / kNT;
        const int b0 = tid * per;
        int loc = 0;
        for (int t = 0; t < per; ++t)
          if (b0 + t <= NB) loc += cnt[b0 + t];
        int inc = loc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= o) inc += v;
        }
        if (lane == 31) s_scan[warp] = inc;
        __syncthreads();
        int wofs = 0;
        for (int w8 = 0; w8 < warp; ++w8) wofs += s_scan[w8];
        int run = wofs + inc - loc;
        for (int t = 0; t < per; ++t)
          if (b0 + t <= NB) {
            const int c0 = cnt[b0 + t];
            cnt[b0 + t] = run;
            run += c0;
          }
      }
      __syncthreads();
      for (int k = 0; k < P; ++k) {
        const int q = tid + k * kNT;
        const int slot = (q / P) * PP + (q % P);
        const int cell = bits_to_cell<T>(stg[7 * ROW + slot]);
        const int key = cell < 0 ? NB : (cell_i(cell) - ox) + bdx * ((DIM == 3 ? cell_j(cell) - oy : 0) + bdy * (cell_k(cell) - oz));
        const unsigned m = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(m) - 1;
        int b = 0;
        if (lane == leader) b = atomicAdd(cnt + key, __popc(m));
        b = __shfl_sync(0xffffffffu, b, leader);
        perm[b + __popc(m & ((1u << lane) - 1u))] = (unsigned short)slot;
      }
      __syncthreads();
    }

    // ---- 5. push and deposit one run of P particles per thread ----
    Acc1<T, DIM> acc;
    acc.zero();
    int key = -1;
    for (int i = 0; i < P; ++i) {
      const int slot = use_box ? (int)perm[tid * P + i] : tid * PP + i;
      const int cell = bits_to_cell<T>(stg[7 * ROW + slot]);
      if (cell < 0 || sp.immobile) continue;
      T o[3] = {stg[0 * ROW + slot], stg[1 * ROW + slot], stg[2 * ROW + slot]};
      const T w = stg[3 * ROW + slot];
      T u[3] = {stg[4 * ROW + slot], stg[5 * ROW + slot], stg[6 * ROW + slot]};
      int c[3] = {cell_i(cell), cell_j(cell), cell_k(cell)};
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
        if (use_box) {
          const int l0x = b0[0] - ox, lhx = bh[0] - ox, l0y = b0[1] - oy, lhy = bh[1] - oy, l0z = b0[2] - oz,
                    lhz = bh[2] - oz;
          E[0] = interp_box<DIM, T>(BE0, bdx, bxy, lhx, wh[0], l0y, w0[1], l0z, w0[2]);
          E[1] = interp_box<DIM, T>(BE1, bdx, bxy, l0x, w0[0], lhy, wh[1], l0z, w0[2]);
          E[2] = interp_box<DIM, T>(BE2, bdx, bxy, l0x, w0[0], l0y, w0[1], lhz, wh[2]);
          B[0] = interp_box<DIM, T>(BB0, bdx, bxy, l0x, w0[0], lhy, wh[1], lhz, wh[2]);
          B[1] = interp_box<DIM, T>(BB1, bdx, bxy, lhx, wh[0], l0y, w0[1], lhz, wh[2]);
          B[2] = interp_box<DIM, T>(BB2, bdx, bxy, lhx, wh[0], lhy, wh[1], l0z, w0[2]);
        } else {
          E[0] = interp<1, DIM, T>(g, f.E[0], bh[0], wh[0], b0[1], w0[1], b0[2], w0[2]);
          E[1] = interp<1, DIM, T>(g, f.E[1], b0[0], w0[0], bh[1], wh[1], b0[2], w0[2]);
          E[2] = interp<1, DIM, T>(g, f.E[2], b0[0], w0[0], b0[1], w0[1], bh[2], wh[2]);
          B[0] = interp_avg<1, DIM, T>(g, f.Bh[0], f.Bp[0], b0[0], w0[0], bh[1], wh[1], bh[2], wh[2]);
          B[1] = interp_avg<1, DIM, T>(g, f.Bh[1], f.Bp[1], bh[0], wh[0], b0[1], w0[1], bh[2], wh[2]);
          B[2] = interp_avg<1, DIM, T>(g, f.Bh[2], f.Bp[2], bh[0], wh[0], bh[1], wh[1], b0[2], w0[2]);
        }
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
      stg[4 * ROW + slot] = u[0];
      stg[5 * ROW + slot] = u[1];
      stg[6 * ROW + slot] = u[2];
      if (out) {
        stg[7 * ROW + slot] = cell_to_bits<T>(-1);
        continue;
      }
      stg[0 * ROW + slot] = o1[0];
      stg[1 * ROW + slot] = o1[1];
      stg[2 * ROW + slot] = o1[2];
      stg[7 * ROW + slot] = cell_to_bits<T>(pack_cell(c1[0], c1[1], c1[2]));
      int lo[3] = {0, 0, 0};
      T S0[3][3], DS[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (DIM == 2 && a == 1) {
          S0[1][0] = T(1);
          S0[1][1] = S0[1][2] = T(0);
          DS[1][0] = DS[1][1] = DS[1][2] = T(0);
          continue;
        }
        esk_axis<1, T>(c[a], o[a], c1[a], o1[a], lo[a], S0[a], DS[a]);
      }
      // anchor key: box-local in the box path, global otherwise
      const int k = use_box ? pack_cell(lo[0] - ox, DIM == 3 ? lo[1] - oy : 0, lo[2] - oz)
                            : pack_cell(lo[0], lo[1], lo[2]);
      if (k != key) {
        if (key >= 0) {
          if (use_box)
            acc.flush_box(BJ0, BJ1, BJ2, cell_i(key), cell_j(key), cell_k(key), bdx, bxy);
          else
            acc.flush(g, tb, f, sp, key);
        }
        acc.zero();
        key = k;
      }
      acc.add(S0, DS, w, w * u[1] * mv.inv_gamma());
    }
    // ---- 6. end of the runs: warp-level reduction, flush ----
    if (use_box) {
      const int up = __shfl_up_sync(0xffffffffu, key, 1);
      const bool head = lane == 0 || up != key;
      const unsigned hm = __ballot_sync(0xffffffffu, head);
      const int segid = __popc(hm & ((2u << lane) - 1u));
      acc.seg_sum(segid, lane);
      if (head && key >= 0) acc.flush_box(BJ0, BJ1, BJ2, cell_i(key), cell_j(key), cell_k(key), bdx, bxy);
    } else {
      const unsigned same = __match_any_sync(0xffffffffu, key);
      if (same == 0xffffffffu) {
        if (key >= 0) {
          acc.warp_sum();
          if (lane == 0) acc.flush(g, tb, f, sp, key);
        }
      } else if (key >= 0) {
        acc.flush(g, tb, f, sp, key);
      }
    }
    __syncthreads();
    // ---- 7. flush the J box to the grid with the charge factor and alpha ----
    if (use_box) {
      const T* anx = al_node<T>(tb, 0);
      const T* acx = al_cent<T>(tb, 0);
      const T* any = al_node<T>(tb, 1);
      const T* acy = al_cent<T>(tb, 1);
      const T* anz = al_node<T>(tb, 2);
      const T* acz = al_cent<T>(tb, 2);
      const T qy = DIM == 3 ? sp.cj[1] : sp.cjy2d;
      for (int t = tid; t < NB; t += kNT) {
        const T j0 = BJ0[t], j1 = BJ1[t], j2 = BJ2[t];
        if (j0 == T(0) && j1 == T(0) && j2 == T(0)) continue;
        const int li = t % bdx, r = t / bdx, lj = r % bdy, lk = r / bdy;
        const int gi = ox + li, gj = oy + lj, gk = oz + lk;
        const long long id = g.idx(gi, gj, gk);
        const T ay_n = DIM == 3 ? any[gj] : T(1), ay_c = DIM == 3 ? acy[gj] : T(1);
        if (j0 != T(0)) atomicAdd(f.J[0] + id, sp.cj[0] * j0 * acx[gi] * ay_n * anz[gk]);
        if (j1 != T(0)) atomicAdd(f.J[1] + id, qy * j1 * anx[gi] * ay_c * anz[gk]);
        if (j2 != T(0)) atomicAdd(f.J[2] + id, sp.cj[2] * j2 * anx[gi] * ay_n * acz[gk]);
      }
    }
    // ---- 8. write the chunk back (coalesced) ----
    for (int q = tid; q < C; q += kNT) {
      const long long gp = base + q;
      if (gp >= n) break;
      const int slot = (q / P) * PP + (q % P);
      const T o[3] = {stg[0 * ROW + slot], stg[1 * ROW + slot], stg[2 * ROW + slot]};
      const T u[3] = {stg[4 * ROW + slot], stg[5 * ROW + slot], stg[6 * ROW + slot]};
      PIO<T>::store(sp.pos, sp.mom, gp, o, stg[3 * ROW + slot], u, bits_to_cell<T>(stg[7 * ROW + slot]));
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
  const size_t smem = Plan<T, P>::total;
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
    return d3 ? launch_pd1_p<T, 3, 4>(g, tb, f, sp, prescribed, status, pushed, nsm, 2, s)
              : launch_pd1_p<T, 2, 4>(g, tb, f, sp, prescribed, status, pushed, nsm, 2, s);
  }
  if (ppt == 4)
    return d3 ? launch_pd1_p<T, 3, 4>(g, tb, f, sp, prescribed, status, pushed, nsm, 4, s)
              : launch_pd1_p<T, 2, 4>(g, tb, f, sp, prescribed, status, pushed, nsm, 4, s);
  return d3 ? launch_pd1_p<T, 3, 8>(g, tb, f, sp, prescribed, status, pushed, nsm, 3, s)
            : launch_pd1_p<T, 2, 8>(g, tb, f, sp, prescribed, status, pushed, nsm, 3, s);
}

template cudaError_t launch_push_deposit_runs<float>(int, const Geom&, const Tables&, const FieldPtrs<float>&,
                                                     const SpeciesPtrs<float>&, int, unsigned*, unsigned long long*,
                                                     int, cudaStream_t);
template cudaError_t launch_push_deposit_runs<double>(int, const Geom&, const Tables&, const FieldPtrs<double>&,
                                                      const SpeciesPtrs<double>&, int, unsigned*, unsigned long long*,
                                                      int, cudaStream_t);

}  // namespace picpml
