// Fused gather + Boris + move + Esirkepov deposit + alpha-damped flush for
// cubic (order-3) shapes in 3D, over particles sorted by tile.
//
// An order-3 move touches 4 x 5 x 5 prefix values per current component
// (300 in all), too many to accumulate in registers, so the deposit goes
// through shared memory.  A block takes a chunk of 128*P consecutive
// particles:
//   1. stage the chunk (coalesced) and find the bounding box of its cells;
//   2. load E and the time-averaged B of that box with fixed strides
//      (nodes lo-2 .. hi+3 per axis: the cubic gather reaches two nodes
//      below the cell, the deposit stencil of a move three above);
//   A. push every particle (64-point gather per component from the box),
//      write its record back and keep old and new positions in the stage;
//   C. every thread takes its P particles' moves into registers; the stage
//      and the dead field box become K private copies of a compact current
//      box over the chunk's nodes, and every thread adds its particles'
//      Esirkepov values into copy (lane mod K) with shared-memory atomics, so
//      lanes of a dense cell collide K times less often;
//   D. sum the copies and add them to the grid with the charge factor and
//      alpha at each component's staggered location (Eq. alpha, Sec. II.B),
//      once per node: the damping of Eq. MaxwellE's source in the flush.
// A chunk whose box does not fit (sparse particles) takes a per-particle
// path with global loads and atomics.
#include "chunk_common.cuh"

namespace picpml {

namespace {

using namespace pc;
using namespace chunk;

constexpr int kNT3 = 128;

template <typename T, int P>
struct Plan3 {
  static constexpr int PP = P + 1;
  static constexpr int ROW = kNT3 * PP;
  static constexpr int C = kNT3 * P;
  static constexpr int NW = 9;   // 0-2 old offsets, 3 weight, 4-6 u then new offsets, 7 old cell, 8 new cell
  static constexpr int BX = 14, BY = 10, BZ = 10;   // up to 8 cells along x (two 4-cell tiles), 4 along y, z
  static constexpr int BXY = BX * BY;
  static constexpr int NBOX = BXY * BZ;
  static constexpr int KMAX = 16;                    // most private current copies
  static constexpr size_t stage = (size_t)NW * ROW * sizeof(T);
  static constexpr size_t box = (size_t)6 * NBOX * sizeof(T);
  static constexpr size_t total = stage + box;
};

// Cubic interpolation from the fixed-stride box; b: box index of the lowest
// of the 4 x 4 x 4 nodes.
template <int BX, int BXY, typename T>
__device__ __forceinline__ T interp3_box(const T* F, int b, const T* wx, const T* wy, const T* wz) {
  T acc = T(0);
#pragma unroll
  for (int tz = 0; tz < 4; ++tz)
#pragma unroll
    for (int ty = 0; ty < 4; ++ty) {
      const T* row = F + b + BX * ty + BXY * tz;
      acc += wy[ty] * wz[tz] * (wx[0] * row[0] + wx[1] * row[1] + wx[2] * row[2] + wx[3] * row[3]);
    }
  return acc;
}

// Esirkepov values of one order-3 move added into a current box copy J
// (component arrays nb apart, strides 1, sy, sz; lo: box-local first node).
// The transverse factor S0 S0' + DS S0'/2 + S0 DS'/2 + DS DS'/3 is evaluated
// as M M' + Q DS' with M = S0 + DS/2, Q = DS/12.
template <typename T>
__device__ __forceinline__ void deposit3_box(T* J, int nb, int sy, int sz, const int lo[3], const T S0[3][5],
                                             const T DS[3][5], T w) {
  T M[3][5], Q[3][5];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      M[a][t] = S0[a][t] + T(0.5) * DS[a][t];
      Q[a][t] = T(1.0 / 12.0) * DS[a][t];
    }
  const int st[3] = {1, sy, sz};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int b = c == 0 ? 1 : 0, d = c == 2 ? 1 : 2;   // transverse axes
    T* Jc = J + c * nb;
#pragma unroll
    for (int td = 0; td < 5; ++td)
#pragma unroll
      for (int tb = 0; tb < 5; ++tb) {
        const T Tl = M[b][tb] * M[d][td] + Q[b][tb] * DS[d][td];
        if (Tl == T(0)) continue;
        const T line = w * Tl;
        T* row = Jc + (lo[b] + tb) * st[b] + (lo[d] + td) * st[d] + lo[c] * st[c];
        T acc = T(0);
#pragma unroll
        for (int ta = 0; ta < 4; ++ta) {
          acc += DS[c][ta];
          if (acc != T(0)) atomicAdd(row + ta * st[c], line * acc);
        }
      }
  }
}

// The whole step of one particle from global memory (chunks whose box does
// not fit): gather, push, move, deposit with global atomics; writes the
// record back.  Returns 1 if the particle was pushed.
template <typename T>
__device__ __noinline__ unsigned particle3_global(const Geom& g, const Tables& tb, const FieldPtrs<T>& f,
                                                  const SpeciesPtrs<T>& sp, int prescribed, const T* stg, int slot,
                                                  int ROW, long long gp) {
  const int cell = bits_to_cell<T>(stg[7 * ROW + slot]);
  const T o[3] = {stg[0 * ROW + slot], stg[1 * ROW + slot], stg[2 * ROW + slot]};
  const T w = stg[3 * ROW + slot];
  T u[3] = {stg[4 * ROW + slot], stg[5 * ROW + slot], stg[6 * ROW + slot]};
  if (cell < 0) {
    PIO<T>::store(sp.pos, sp.mom, gp, o, w, u, -1);
    return 0;
  }
  const int c[3] = {cell_i(cell), cell_j(cell), cell_k(cell)};
  if (!prescribed) {
    int b0[3], bh[3];
    T w0[3][4], wh[3][4];
#pragma unroll
    for (int a = 0; a < 3; ++a) axis_weights<3, T>(c[a], o[a], b0[a], w0[a], bh[a], wh[a]);
    T E[3], B[3];
    E[0] = interp<3, 3, T>(g, f.E[0], bh[0], wh[0], b0[1], w0[1], b0[2], w0[2]);
    E[1] = interp<3, 3, T>(g, f.E[1], b0[0], w0[0], bh[1], wh[1], b0[2], w0[2]);
    E[2] = interp<3, 3, T>(g, f.E[2], b0[0], w0[0], b0[1], w0[1], bh[2], wh[2]);
    B[0] = interp_avg<3, 3, T>(g, f.Bh[0], f.Bp[0], b0[0], w0[0], bh[1], wh[1], bh[2], wh[2]);
    B[1] = interp_avg<3, 3, T>(g, f.Bh[1], f.Bp[1], bh[0], wh[0], b0[1], w0[1], bh[2], wh[2]);
    B[2] = interp_avg<3, 3, T>(g, f.Bh[2], f.Bp[2], bh[0], wh[0], bh[1], wh[1], b0[2], w0[2]);
    boris<T>(u, E, B, sp.ke);
  }
  int c1[3];
  T o1[3], ig;
  const bool in = move_particle<3, T>(g, o, c, u, c1, o1, ig);
  T wd = w, wn = w;
  if (g.wdamp && in) {
    const T I = weight_exponent<T>(g, c, o, c1, o1);
    wd = w * exp(T(-0.5) * I);
    wn = w * exp(-I);
  }
  PIO<T>::store(sp.pos, sp.mom, gp, in ? o1 : o, wn, u, in ? pack_cell(c1[0], c1[1], c1[2]) : -1);
  if (in) deposit_one<3, 3, T>(g, tb, f, sp, c, o, c1, o1, wd, T(0));
  return 1;
}

template <typename T, int P>
__global__ void __launch_bounds__(kNT3, sizeof(T) == 4 ? 3 : 2)
    k_pd3(const __grid_constant__ Geom g, const __grid_constant__ Tables tb, const __grid_constant__ FieldPtrs<T> f,
          const __grid_constant__ SpeciesPtrs<T> sp, int prescribed, unsigned* status,
          unsigned long long* pushed_total) {
  using PL = Plan3<T, P>;
  constexpr int PP = PL::PP, ROW = PL::ROW, C = PL::C;
  constexpr int BX = PL::BX, BY = PL::BY, BZ = PL::BZ, BXY = PL::BXY, NBOX = PL::NBOX;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* stg = reinterpret_cast<T*>(smraw);
  T* bx_ = reinterpret_cast<T*>(smraw + PL::stage);
  __shared__ int s_lo[3], s_hi[3];
  const int tid = threadIdx.x, lane = tid & 31;
  const long long n = *sp.n_dev;
  const long long nchunks = (n + C - 1) / C;
  unsigned pushed = 0;
  if (sp.immobile) return;

  for (long long ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const long long base = ch * C;
    __syncthreads();
    stage_chunk<T, 3, P, kNT3>(g, sp, base, n, base + (long long)gridDim.x * C, stg, ROW, status, s_lo, s_hi);
    const int ox = s_lo[0] - 2, oy = s_lo[1] - 2, oz = s_lo[2] - 2;
    const int bdx = s_hi[0] - s_lo[0] + 6, bdy = s_hi[1] - s_lo[1] + 6, bdz = s_hi[2] - s_lo[2] + 6;
    if (s_hi[0] >= 0 && bdx <= BX && bdy <= BY && bdz <= BZ) {
      const int NB = bdx * bdy * bdz;
      // ---- 2. E and the time-averaged B of the box ----
      for (int t = tid; t < NB; t += kNT3) {
        const int li = t % bdx, r = t / bdx, lj = r % bdy, lk = r / bdy;
        const long long gi = g.idx(ox + li, oy + lj, oz + lk);
        const int bi = li + BX * lj + BXY * lk;
        bx_[0 * NBOX + bi] = f.E[0][gi];
        bx_[1 * NBOX + bi] = f.E[1][gi];
        bx_[2 * NBOX + bi] = f.E[2][gi];
        bx_[3 * NBOX + bi] = T(0.5) * (f.Bh[0][gi] + f.Bp[0][gi]);
        bx_[4 * NBOX + bi] = T(0.5) * (f.Bh[1][gi] + f.Bp[1][gi]);
        bx_[5 * NBOX + bi] = T(0.5) * (f.Bh[2][gi] + f.Bp[2][gi]);
      }
      __syncthreads();
      // ---- A. gather, push, move; records straight back to global memory ----
      for (int i = 0; i < P; ++i) {
        const int slot = tid * PP + i;
        const long long gp = base + tid * P + i;
        const int cell = bits_to_cell<T>(stg[7 * ROW + slot]);
        const T o[3] = {stg[0 * ROW + slot], stg[1 * ROW + slot], stg[2 * ROW + slot]};
        const T w = stg[3 * ROW + slot];
        T u[3] = {stg[4 * ROW + slot], stg[5 * ROW + slot], stg[6 * ROW + slot]};
        if (cell < 0) {
          stg[8 * ROW + slot] = cell_to_bits<T>(-1);
          if (gp < n) PIO<T>::store(sp.pos, sp.mom, gp, o, w, u, -1);
          continue;
        }
        const int c[3] = {cell_i(cell), cell_j(cell), cell_k(cell)};
        if (!prescribed) {
          int b0[3], bh[3];
          T w0[3][4], wh[3][4];
#pragma unroll
          for (int a = 0; a < 3; ++a) axis_weights<3, T>(c[a], o[a], b0[a], w0[a], bh[a], wh[a]);
          const int sx0 = b0[0] - ox, sxh = bh[0] - ox;
          const int sy0 = BX * (b0[1] - oy), syh = BX * (bh[1] - oy);
          const int sz0 = BXY * (b0[2] - oz), szh = BXY * (bh[2] - oz);
          T E[3], B[3];
          E[0] = interp3_box<BX, BXY, T>(bx_ + 0 * NBOX, sxh + sy0 + sz0, wh[0], w0[1], w0[2]);
          E[1] = interp3_box<BX, BXY, T>(bx_ + 1 * NBOX, sx0 + syh + sz0, w0[0], wh[1], w0[2]);
          E[2] = interp3_box<BX, BXY, T>(bx_ + 2 * NBOX, sx0 + sy0 + szh, w0[0], w0[1], wh[2]);
          B[0] = interp3_box<BX, BXY, T>(bx_ + 3 * NBOX, sx0 + syh + szh, w0[0], wh[1], wh[2]);
          B[1] = interp3_box<BX, BXY, T>(bx_ + 4 * NBOX, sxh + sy0 + szh, wh[0], w0[1], wh[2]);
          B[2] = interp3_box<BX, BXY, T>(bx_ + 5 * NBOX, sxh + syh + sz0, wh[0], wh[1], w0[2]);
          boris<T>(u, E, B, sp.ke);
        }
        ++pushed;
        int c1[3];
        T o1[3], ig;
        const bool in = move_particle<3, T>(g, o, c, u, c1, o1, ig);
        const int cell1 = in ? pack_cell(c1[0], c1[1], c1[2]) : -1;
        T wn = w;
        if (g.wdamp && in) {  // weight damping: mid-step weight for this step's current
          const T I = weight_exponent<T>(g, c, o, c1, o1);
          stg[3 * ROW + slot] = w * exp(T(-0.5) * I);
          wn = w * exp(-I);
        }
        PIO<T>::store(sp.pos, sp.mom, gp, in ? o1 : o, wn, u, cell1);
        stg[4 * ROW + slot] = o1[0];
        stg[5 * ROW + slot] = o1[1];
        stg[6 * ROW + slot] = o1[2];
        stg[8 * ROW + slot] = cell_to_bits<T>(cell1);
      }
      __syncthreads();
      // ---- C. private current copies over the chunk's nodes (compact strides) ----
      // Each thread keeps its own P particles' moves in registers, so the
      // stage and the dead field box together hold the copies.
      int mc0[P], mc1[P];
      T mo0[P][3], mo1[P][3], mw[P];
#pragma unroll
      for (int i = 0; i < P; ++i) {
        const int slot = tid * PP + i;
        mc0[i] = bits_to_cell<T>(stg[7 * ROW + slot]);
        mc1[i] = bits_to_cell<T>(stg[8 * ROW + slot]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          mo0[i][a] = stg[a * ROW + slot];
          mo1[i][a] = stg[(4 + a) * ROW + slot];
        }
        mw[i] = stg[3 * ROW + slot];
      }
      __syncthreads();
      constexpr int kRoom = (int)((PL::stage + PL::box) / sizeof(T));
      int K = 1;
      while (K < PL::KMAX && 2 * K * 3 * NB <= kRoom) K *= 2;
      T* const BJ = stg;
      for (int t = tid; t < K * 3 * NB; t += kNT3) BJ[t] = T(0);
      __syncthreads();
      T* const Jmine = BJ + (lane & (K - 1)) * 3 * NB;
#pragma unroll 1
      for (int i = 0; i < P; ++i) {
        if (mc1[i] < 0 || mc0[i] < 0) continue;
        const int c0[3] = {cell_i(mc0[i]), cell_j(mc0[i]), cell_k(mc0[i])};
        const int c1[3] = {cell_i(mc1[i]), cell_j(mc1[i]), cell_k(mc1[i])};
        const int org[3] = {ox, oy, oz};
        int lo[3];
        T S0[3][5], DS[3][5];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          esk_axis<3, T>(c0[a], mo0[i][a], c1[a], mo1[i][a], lo[a], S0[a], DS[a]);
          lo[a] -= org[a];
        }
        deposit3_box<T>(Jmine, NB, bdx, bdx * bdy, lo, S0, DS, mw[i]);
      }
      __syncthreads();
      // ---- D. sum the copies, add to the grid with the charge factor and alpha ----
      const T* anx = al_node<T>(tb, 0);
      const T* acx = al_cent<T>(tb, 0);
      const T* any = al_node<T>(tb, 1);
      const T* acy = al_cent<T>(tb, 1);
      const T* anz = al_node<T>(tb, 2);
      const T* acz = al_cent<T>(tb, 2);
      for (int t = tid; t < NB; t += kNT3) {
        T j0 = T(0), j1 = T(0), j2 = T(0);
        for (int k = 0; k < K; ++k) {
          j0 += BJ[k * 3 * NB + t];
          j1 += BJ[k * 3 * NB + NB + t];
          j2 += BJ[k * 3 * NB + 2 * NB + t];
        }
        if (j0 == T(0) && j1 == T(0) && j2 == T(0)) continue;
        const int li = t % bdx, r = t / bdx, lj = r % bdy, lk = r / bdy;
        const int gi = ox + li, gj = oy + lj, gk = oz + lk;
        const long long id = g.idx(gi, gj, gk);
        if (j0 != T(0)) atomicAdd(f.J[0] + id, sp.cj[0] * j0 * acx[gi] * any[gj] * anz[gk]);
        if (j1 != T(0)) atomicAdd(f.J[1] + id, sp.cj[1] * j1 * anx[gi] * acy[gj] * anz[gk]);
        if (j2 != T(0)) atomicAdd(f.J[2] + id, sp.cj[2] * j2 * anx[gi] * any[gj] * acz[gk]);
      }
    } else {
      for (int i = 0; i < P; ++i) {
        const long long gp = base + tid * P + i;
        if (gp < n) pushed += particle3_global<T>(g, tb, f, sp, prescribed, stg, tid * PP + i, ROW, gp);
      }
    }
  }
  if (pushed_total) {
    const unsigned wsum = __reduce_add_sync(0xffffffffu, pushed);
    if (lane == 0 && wsum) atomicAdd(pushed_total, (unsigned long long)wsum);
  }
}

template <typename T, int P>
cudaError_t launch_pd3_p(const Geom& g, const Tables& tb, const FieldPtrs<T>& f, const SpeciesPtrs<T>& sp,
                         int prescribed, unsigned* status, unsigned long long* pushed, int nsm, int blocks_per_sm,
                         cudaStream_t s) {
  const size_t smem = Plan3<T, P>::total;
  static bool configured = false;  // per template instance, once per process
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_pd3<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const long long C = (long long)kNT3 * P;
  long long chunks = (sp.capacity + C - 1) / C;
  long long maxb = (long long)nsm * blocks_per_sm;
  int blocks = (int)(chunks < maxb ? chunks : maxb);
  if (blocks < 1) blocks = 1;
  k_pd3<T, P><<<blocks, kNT3, smem, s>>>(g, tb, f, sp, prescribed, status, pushed);
  return cudaGetLastError();
}

}  // namespace

// Order-3 3D fused kernel; ppt 8 selects 8 particles per thread, else 4.
template <typename T>
cudaError_t launch_push_deposit_o3(int ppt, const Geom& g, const Tables& tb, const FieldPtrs<T>& f,
                                   const SpeciesPtrs<T>& sp, int prescribed, unsigned* status,
                                   unsigned long long* pushed, int nsm, cudaStream_t s) {
  if (sp.capacity <= 0) return cudaSuccess;
  if (g.dim != 3) return cudaErrorInvalidValue;
  if constexpr (sizeof(T) == 8) {
    return launch_pd3_p<T, 4>(g, tb, f, sp, prescribed, status, pushed, nsm, 2, s);
  } else {
    if (ppt == 8) return launch_pd3_p<T, 8>(g, tb, f, sp, prescribed, status, pushed, nsm, 2, s);
    return launch_pd3_p<T, 4>(g, tb, f, sp, prescribed, status, pushed, nsm, 3, s);
  }
}

template cudaError_t launch_push_deposit_o3<float>(int, const Geom&, const Tables&, const FieldPtrs<float>&,
                                                   const SpeciesPtrs<float>&, int, unsigned*, unsigned long long*,
                                                   int, cudaStream_t);
template cudaError_t launch_push_deposit_o3<double>(int, const Geom&, const Tables&, const FieldPtrs<double>&,
                                                    const SpeciesPtrs<double>&, int, unsigned*,
                                                    unsigned long long*, int, cudaStream_t);

}  // namespace picpml
