// Fused gather + Boris + move + Esirkepov deposit + alpha-damped flush for
// shape order 1, over particles sorted by tile.
//
// A block takes a chunk of 128*P consecutive particles and works in phases,
// all from shared memory:
//   1. stage the chunk with coalesced 16-byte loads (structure of arrays, rows
//      padded to P+1 words so a thread's strided reads are bank-conflict free)
//      and find the bounding box of its cells; the block's next chunk is
//      prefetched into L2 meanwhile;
//   2. load E and the time-averaged B of that box (+ guard nodes);
//   A. push: every thread gathers, rotates and moves its own P particles and
//      keeps old and new positions in the stage;
//   B. counting-sort the chunk by Esirkepov anchor (the per-axis minimum of
//      old and new cell, where the order-1 current stencil of the move
//      starts) and cut each anchor's particles into runs of at most L
//      (P, or more when the chunk holds few anchors, so that there is still
//      about one run per thread); the E/B box is dead now and becomes the
//      current box;
//   C. deposit: each thread takes a run, which shares one anchor, and
//      accumulates the 2x3x3 prefix values of each component (54 in 3D) in
//      registers; then, for each anchor held by lanes of a warp (every
//      group, however small), the warp sums those lanes' values with a
//      reduce-scatter of shuffles (each lane ends with two sums) and adds
//      them to the box with two shared-memory atomics per lane;
//   D. add the box to the grid with the charge factor and alpha (Eq. alpha,
//      at each component's staggered location): the damping of Eq. MaxwellE's
//      source term applied once per node in the flush.
// The pushed records are written back from phase A directly (a thread's P
// particles are consecutive, so a warp's stores cover whole lines over its P
// iterations and merge in L2).
// A chunk whose box does not fit in shared memory (sparse particles) takes a
// per-particle path with global loads and atomics.
#include "chunk_common.cuh"

namespace picpml {

namespace {

using namespace pc;
using namespace chunk;

// Register accumulator of the order-1 current of a run: w * (Esirkepov shape
// factor) prefix sums; the charge factor and alpha are applied at the flush.
// Flat layout, 3D: Jx [ix*9 + jy*3 + kz] (ix < 2), Jy 18 + [ix*6 + jy*3 + kz]
// (jy < 2), Jz 36 + [ix*6 + jy*2 + kz] (kz < 2); 2D: Jx [ix*3 + kz],
// Jy (out of plane) 6 + [ix*3 + kz], Jz 15 + [ix*2 + kz].
template <typename T, int DIM, int BX, int BXY, int NBOX>
struct Acc1 {
  static constexpr int NX = DIM == 3 ? 18 : 6;
  static constexpr int NY = DIM == 3 ? 18 : 9;
  static constexpr int NV = DIM == 3 ? 54 : 21;
  static constexpr int NVP = DIM == 3 ? 64 : 32;   // padded to 32 * 2^k for the reduce-scatter
  T v[NV];

  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int t = 0; t < NV; ++t) v[t] = T(0);
  }

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
            v[0 * 9 + jy * 3 + kz] += ax0 * Tl;
            v[1 * 9 + jy * 3 + kz] += ax1 * Tl;
          }
      }
      const T ay0 = w * DS[1][0], ay1 = w * (DS[1][0] + DS[1][1]);
      if (ay0 != T(0) || ay1 != T(0)) {
#pragma unroll
        for (int ix = 0; ix < 3; ++ix)
#pragma unroll
          for (int kz = 0; kz < 3; ++kz) {
            const T Tl = M[0][ix] * M[2][kz] + Q[0][ix] * DS[2][kz];
            v[NX + ix * 6 + 0 * 3 + kz] += ay0 * Tl;
            v[NX + ix * 6 + 1 * 3 + kz] += ay1 * Tl;
          }
      }
      const T az0 = w * DS[2][0], az1 = w * (DS[2][0] + DS[2][1]);
      if (az0 != T(0) || az1 != T(0)) {
#pragma unroll
        for (int ix = 0; ix < 3; ++ix)
#pragma unroll
          for (int jy = 0; jy < 3; ++jy) {
            const T Tl = M[0][ix] * M[1][jy] + Q[0][ix] * DS[1][jy];
            v[NX + NY + ix * 6 + jy * 2 + 0] += az0 * Tl;
            v[NX + NY + ix * 6 + jy * 2 + 1] += az1 * Tl;
          }
      }
    } else {
      const T ax0 = w * DS[0][0], ax1 = w * (DS[0][0] + DS[0][1]);
#pragma unroll
      for (int kz = 0; kz < 3; ++kz) {
        v[0 * 3 + kz] += ax0 * M[2][kz];
        v[1 * 3 + kz] += ax1 * M[2][kz];
      }
      const T az0 = w * DS[2][0], az1 = w * (DS[2][0] + DS[2][1]);
#pragma unroll
      for (int ix = 0; ix < 3; ++ix) {
        v[NX + NY + ix * 2 + 0] += az0 * M[0][ix];
        v[NX + NY + ix * 2 + 1] += az1 * M[0][ix];
      }
      if (wvy != T(0)) {
#pragma unroll
        for (int ix = 0; ix < 3; ++ix)
#pragma unroll
          for (int kz = 0; kz < 3; ++kz) v[NX + ix * 3 + kz] += wvy * (M[0][ix] * M[2][kz] + Q[0][ix] * DS[2][kz]);
      }
    }
  }

  // Component and node offsets of flat index idx.
  __device__ __forceinline__ static void node_of(int idx, int& comp, int& ix, int& jy, int& kz) {
    if (DIM == 3) {
      if (idx < 18) {
        comp = 0; ix = idx / 9; jy = (idx / 3) % 3; kz = idx % 3;
      } else if (idx < 36) {
        const int t = idx - 18;
        comp = 1; ix = t / 6; jy = (t / 3) % 2; kz = t % 3;
      } else {
        const int t = idx - 36;
        comp = 2; ix = t / 6; jy = (t / 2) % 3; kz = t % 2;
      }
    } else {
      jy = 0;
      if (idx < 6) {
        comp = 0; ix = idx / 3; kz = idx % 3;
      } else if (idx < 15) {
        const int t = idx - 6;
        comp = 1; ix = t / 3; kz = t % 3;
      } else {
        const int t = idx - 15;
        comp = 2; ix = t / 2; kz = t % 2;
      }
    }
  }

  // Box offset of flat index idx (component array comp * NBOX + node offset)
  // in a box with row length BX and plane size BXY.
  __device__ __forceinline__ static int box_offset(int idx) {
    int comp, ix, jy, kz;
    node_of(idx, comp, ix, jy, kz);
    return comp * NBOX + ix + BX * jy + BXY * kz;
  }


  // Sums the accumulators of the lanes with member == true (one anchor) by a
  // reduce-scatter of shuffles into a scratch array: after five halving steps
  // lane L holds the group's sums of flat indices K L .. K L + K - 1
  // (K = NVP / 32), which it adds to the box at offsets goff (precomputed per
  // lane, -1 past the last index).  Every lane takes part (lanes outside the
  // group contribute zeros and carry partial sums) and keeps its own
  // accumulators for its own group.
  template <bool ALL>
  __device__ __forceinline__ void group_flush(bool member, int lane, T* J, int a, const int* goff) const {
    constexpr int H = NVP / 2;
    T t[H];
    {
      const bool up = (lane & 16) != 0;
#pragma unroll
      for (int i = 0; i < H; ++i) {
        const T lo = (i < NV && (ALL || member)) ? v[i < NV ? i : 0] : T(0);
        const T hi = (i + H < NV && (ALL || member)) ? v[i + H < NV ? i + H : 0] : T(0);
        t[i] = (up ? hi : lo) + __shfl_xor_sync(0xffffffffu, up ? lo : hi, 16);
      }
    }
#pragma unroll
    for (int lev = 1; lev < 5; ++lev) {
      const int o = 16 >> lev;
      const int h = H >> lev;
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int i = 0; i < h; ++i) {
        const T lo = t[i], hi = t[i + h];
        t[i] = (up ? hi : lo) + __shfl_xor_sync(0xffffffffu, up ? lo : hi, o);
      }
    }
    constexpr int K = NVP / 32;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (goff[k] >= 0 && t[k] != T(0)) atomicAdd(J + a + goff[k], t[k]);
  }
};

// An accumulator with the lane's precomputed reduce-scatter offsets, in the
// form flush_warp_runs takes.
template <class AC>
struct WithOffsets {
  const AC& acc;
  const int* goff;
  template <bool ALL, typename T>
  __device__ __forceinline__ void group_flush(bool member, int lane, T* J, int a) const {
    acc.template group_flush<ALL>(member, lane, J, a, goff);
  }
};

constexpr int kNT = 128;
// Fewest lanes of one anchor that a warp sums by reduce-scatter (about 330
// instructions per anchor).  With runs cut at anchor boundaries every group,
// even a single lane, takes the reduce-scatter: the per-lane flush (54
// shared atomics) was slower on the 4M beam (0.322 vs 0.300 ms per step) and
// its code is not needed.
constexpr int kMinGroupLanes = 1;

// Shared memory of one block: the staged chunk (NW words per particle, rows
// padded to P+1), the field box (E and time-averaged B, 6 arrays of NBOX
// nodes with fixed strides BX, BX*BY, so every gather and deposit offset is a
// compile-time constant; its first 3 arrays are the current box after the
// push), the counters and the permutation of the anchor sort, and the runs
// (in 3D inside the box's last 3 arrays, which the push leaves dead).  The box holds
// nodes lo-1 .. hi+2 of a chunk whose cells span lo .. hi: up to 9 cells
// along x (two x-adjacent 4-cell sort tiles) and 5 along y and z.  (A box
// for 11 and 6 cells, which keeps the chunks of a thermal plasma whose
// particles leave their tiles on both sides, made the dense beam 10 % slower.)
// Stage words: 0-2 old offsets, 3 weight, 4-6 u (replaced by the new offsets
// once the particle is pushed and its record written back), 7 old cell,
// 8 new cell (-1: removed or deposits nothing), 9 (2D) w v_y/c.
template <typename T, int DIM, int P>
struct Plan {
  static constexpr int PP = P + 1;
  static constexpr int ROW = kNT * PP;
  static constexpr int C = kNT * P;
  static constexpr int NW = DIM == 3 ? 9 : 10;
  static constexpr int BX = 12, BY = DIM == 3 ? 8 : 1, BZ = 8;
  static constexpr int BXY = BX * BY;
  static constexpr int NBOX = BXY * BZ;
  static constexpr size_t stage = (size_t)NW * ROW * sizeof(T);
  static constexpr size_t box = (size_t)6 * NBOX * sizeof(T);
  static constexpr size_t cnt = (size_t)(NBOX + 1) * sizeof(int);   // anchor counters
  static constexpr size_t perm = (size_t)C * sizeof(unsigned short);
  static constexpr size_t runs = (size_t)C * sizeof(unsigned short);  // run descriptors
  // the sort arrays live in the box's last three arrays (the time-averaged
  // B, dead after the push) where they fit (3D), else after the box
  static constexpr bool sort_in_box = cnt + perm + runs <= (size_t)3 * NBOX * sizeof(T);
  static constexpr size_t sort_at = stage + (sort_in_box ? (size_t)3 * NBOX * sizeof(T) : box);
  static constexpr size_t total = stage + box + (sort_in_box ? 0 : cnt + perm + runs);
};

// Order-1 interpolation from a shared-memory box with fixed strides; b is
// the box index of the lowest of the 8 (4 in 2D) nodes.
template <int DIM, int BX, int BXY, typename T>
__device__ __forceinline__ T interp_box(const T* F, int b, const T* wx, const T* wy, const T* wz) {
  T acc = T(0);
#pragma unroll
  for (int tz = 0; tz < 2; ++tz)
#pragma unroll
    for (int ty = 0; ty < (DIM == 3 ? 2 : 1); ++ty) {
      const T* row = F + b + BX * ty + BXY * tz;
      acc += (DIM == 3 ? wy[ty] : T(1)) * wz[tz] * (wx[0] * row[0] + wx[1] * row[1]);
    }
  return acc;
}

// The whole step of one particle from global memory (chunks whose box does
// not fit in shared memory): gather, push, move, deposit with global atomics
// (charge factor and alpha per contribution), and the particle's record is
// written back.  Returns 1 if the particle was pushed.
template <typename T, int DIM>
__device__ __noinline__ unsigned particle_global(const Geom& g, const Tables& tb, const FieldPtrs<T>& f,
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
  int c1[3];
  T o1[3], ig;
  const bool in = move_particle<DIM, T>(g, o, c, u, c1, o1, ig);
  T wd = w, wn = w;
  if (g.wdamp && in) {
    const T I = weight_exponent<T>(g, c, o, c1, o1);
    wd = w * exp(T(-0.5) * I);
    wn = w * exp(-I);
  }
  PIO<T>::store(sp.pos, sp.mom, gp, in ? o1 : o, wn, u, in ? pack_cell(c1[0], c1[1], c1[2]) : -1);
  if (in) deposit_one<1, DIM, T>(g, tb, f, sp, c, o, c1, o1, wd, u[1] * ig);
  return 1;
}

template <typename T, int DIM, int P>
__global__ void __launch_bounds__(kNT, sizeof(T) == 4 ? (P >= 8 ? 3 : 4) : 2)
    k_pd1(const __grid_constant__ Geom g, const __grid_constant__ Tables tb, const __grid_constant__ FieldPtrs<T> f,
          const __grid_constant__ SpeciesPtrs<T> sp, int prescribed, unsigned* status,
          unsigned long long* pushed_total) {
  using PL = Plan<T, DIM, P>;
  using AC = Acc1<T, DIM, PL::BX, PL::BXY, PL::NBOX>;
  constexpr int PP = PL::PP, ROW = PL::ROW, C = PL::C;
  constexpr int BX = PL::BX, BY = PL::BY, BZ = PL::BZ, BXY = PL::BXY, NBOX = PL::NBOX;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* stg = reinterpret_cast<T*>(smraw);
  T* bx_ = reinterpret_cast<T*>(smraw + PL::stage);
  int* cnt = reinterpret_cast<int*>(smraw + PL::sort_at);
  unsigned short* perm = reinterpret_cast<unsigned short*>(smraw + PL::sort_at + PL::cnt);
  __shared__ int s_lo[3], s_hi[3];
  __shared__ int s_scan[kNT / 32];
  __shared__ int s_nanchor;
  __shared__ int s_nrun;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long n = *sp.n_dev;
  const long long nchunks = (n + C - 1) / C;
  unsigned pushed = 0;
  if (sp.immobile) return;
  unsigned short* runs = reinterpret_cast<unsigned short*>(smraw + PL::sort_at + PL::cnt + PL::perm);
  // box offsets of the two (2D: one) reduce-scatter results this lane adds
  constexpr int K = AC::NVP / 32;
  int goff[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int idx = k + K * lane;
    goff[k] = idx < AC::NV ? AC::box_offset(idx) : -1;
  }

  for (long long ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const long long base = ch * C;
    __syncthreads();
    // ---- 1. stage the chunk (and prefetch the next), bounding box of its cells ----
    stage_chunk<T, DIM, P, kNT>(g, sp, base, n, base + (long long)gridDim.x * C, stg, ROW, status, s_lo, s_hi);
    // nodes lo-1 .. hi+2 per axis: the gather reads from the cell's lower
    // node minus one (half-staggered components) to its upper node, the
    // deposit stencil of a move spans min(old, new cell) .. + 2
    const int ox = s_lo[0] - 1, oy = DIM == 3 ? s_lo[1] - 1 : 0, oz = s_lo[2] - 1;
    const int bdx = s_hi[0] - s_lo[0] + 4, bdy = DIM == 3 ? s_hi[1] - s_lo[1] + 4 : 1, bdz = s_hi[2] - s_lo[2] + 4;
    if (s_hi[0] >= 0 && bdx <= BX && bdy <= BY && bdz <= BZ) {
      const int NB = bdx * bdy * bdz;   // nodes of the chunk's region (row length bdx)
      // ---- 2. E and the time-averaged B of the box ----
      for (int t = tid; t < NB; t += kNT) {
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
      // ---- A. gather, push and move this thread's P particles; the new
      //      records go straight back to global memory ----
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
          const int l0x = b0[0] - ox, lhx = bh[0] - ox, l0y = b0[1] - oy, lhy = bh[1] - oy, l0z = b0[2] - oz,
                    lhz = bh[2] - oz;
          T E[3], B[3];
          // box index of the lowest node per (x, y, z) stagger combination
          const int sx0 = l0x, sxh = lhx, sy0 = BX * l0y, syh = BX * lhy, sz0 = BXY * l0z, szh = BXY * lhz;
          E[0] = interp_box<DIM, BX, BXY, T>(bx_ + 0 * NBOX, sxh + sy0 + sz0, wh[0], w0[1], w0[2]);
          E[1] = interp_box<DIM, BX, BXY, T>(bx_ + 1 * NBOX, sx0 + syh + sz0, w0[0], wh[1], w0[2]);
          E[2] = interp_box<DIM, BX, BXY, T>(bx_ + 2 * NBOX, sx0 + sy0 + szh, w0[0], w0[1], wh[2]);
          B[0] = interp_box<DIM, BX, BXY, T>(bx_ + 3 * NBOX, sx0 + syh + szh, w0[0], wh[1], wh[2]);
          B[1] = interp_box<DIM, BX, BXY, T>(bx_ + 4 * NBOX, sxh + sy0 + szh, wh[0], w0[1], wh[2]);
          B[2] = interp_box<DIM, BX, BXY, T>(bx_ + 5 * NBOX, sxh + syh + sz0, wh[0], wh[1], w0[2]);
          boris<T>(u, E, B, sp.ke);
        }
        ++pushed;
        int c1[3];
        T o1[3], ig;
        const bool in = move_particle<DIM, T>(g, o, c, u, c1, o1, ig);
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
        if constexpr (DIM == 2) stg[9 * ROW + slot] = stg[3 * ROW + slot] * u[1] * ig;
      }
      __syncthreads();
      // ---- B. counting sort of the chunk by anchor, runs ----
      // (keys are compact indices of the anchor cells, key nk collects the
      // particles that deposit nothing; the E/B box is dead: its first three
      // arrays become the current box)
      T* const BJ = bx_;
      {
        // 16-byte stores, then the values of a last partial group
        float4* z = reinterpret_cast<float4*>(BJ);
        constexpr int PER = (int)(sizeof(float4) / sizeof(T));
        constexpr int NZ = 3 * NBOX / PER;
        for (int t = tid; t < NZ; t += kNT) z[t] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int t = NZ * PER + tid; t < 3 * NBOX; t += kNT) BJ[t] = T(0);
      }
      // key: the anchor cell min(old, new) per axis, from s_lo - 1 to s_hi
      const int kdx = bdx - 2, kdy = DIM == 3 ? bdy - 2 : 1, nk = kdx * kdy * (bdz - 2);
      for (int t = tid; t <= nk; t += kNT) cnt[t] = 0;
      if (tid == 0) {
        s_nanchor = 0;
        s_nrun = 0;
      }
      __syncthreads();
      int keys[P];
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const int q = tid + k * kNT;
        const int slot = (q / P) * PP + (q % P);
        const int c0 = bits_to_cell<T>(stg[7 * ROW + slot]);
        const int c1 = bits_to_cell<T>(stg[8 * ROW + slot]);
        if (c0 < 0 || c1 < 0) {
          keys[k] = nk;
        } else {
          const int ax = min(cell_i(c0), cell_i(c1)) - ox;
          const int ay = DIM == 3 ? min(cell_j(c0), cell_j(c1)) - oy : 0;
          const int az = min(cell_k(c0), cell_k(c1)) - oz;
          keys[k] = ax + kdx * (ay + kdy * az);
        }
      }
      sort_runs<P, kNT>(keys, nk, cnt, perm, runs, s_scan, &s_nanchor, &s_nrun);
      // ---- C. deposit the runs, one per thread at a time ----
      // Shape factors of a slot's move; returns the box offset of its anchor.
      auto prepare = [&](int slot, T (&S0)[3][3], T (&DS)[3][3]) -> int {
        const int cell1 = bits_to_cell<T>(stg[8 * ROW + slot]);
        const int cell0 = bits_to_cell<T>(stg[7 * ROW + slot]);
        const int c0[3] = {cell_i(cell0), cell_j(cell0), cell_k(cell0)};
        const int c1[3] = {cell_i(cell1), cell_j(cell1), cell_k(cell1)};
        int lo[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (DIM == 2 && a == 1) {
            S0[1][0] = T(1);
            S0[1][1] = S0[1][2] = T(0);
            DS[1][0] = DS[1][1] = DS[1][2] = T(0);
            continue;
          }
          esk_axis<1, T>(c0[a], stg[a * ROW + slot], c1[a], stg[(4 + a) * ROW + slot], lo[a], S0[a], DS[a]);
        }
        return (lo[0] - ox) + BX * (DIM == 3 ? lo[1] - oy : 0) + BXY * (lo[2] - oz);
      };
      auto wvy_of = [&](int slot) -> T {
        if constexpr (DIM == 2) return stg[9 * ROW + slot];
        return T(0);
      };
      const int R = s_nrun;
      for (int rb = warp * 32; rb < R; rb += kNT) {
        AC acc;
        acc.zero();
        int key = -1;
        if (rb + lane < R) {
          const unsigned d = runs[rb + lane];
          const int st = d & 0x7ff, len = d >> 11;
          for (int i = 0; i < len; ++i) {
            const int slot = perm[st + i];
            T S0[3][3], DS[3][3];
            key = prepare(slot, S0, DS);
            acc.add(S0, DS, stg[3 * ROW + slot], wvy_of(slot));
          }
        }
        flush_warp_runs<kMinGroupLanes>(WithOffsets<AC>{acc, goff}, key, lane, BJ);
      }
      __syncthreads();
      // ---- D. add the current box to the grid with the charge factor and alpha ----
      const T* anx = al_node<T>(tb, 0);
      const T* acx = al_cent<T>(tb, 0);
      const T* any = al_node<T>(tb, 1);
      const T* acy = al_cent<T>(tb, 1);
      const T* anz = al_node<T>(tb, 2);
      const T* acz = al_cent<T>(tb, 2);
      const T qy = DIM == 3 ? sp.cj[1] : sp.cjy2d;
      // axes along which the whole region lies where alpha is 1 skip its tables
      const bool one_x = ox >= tb.al1_lo[0] && ox + bdx - 1 <= tb.al1_hi[0];
      const bool one_y = DIM == 2 || (oy >= tb.al1_lo[1] && oy + bdy - 1 <= tb.al1_hi[1]);
      const bool one_z = oz >= tb.al1_lo[2] && oz + bdz - 1 <= tb.al1_hi[2];
      for (int t = tid; t < NB; t += kNT) {
        const int li = t % bdx, r = t / bdx, lj = r % bdy, lk = r / bdy;
        const int bi = li + BX * lj + BXY * lk;
        const T j0 = BJ[bi], j1 = BJ[NBOX + bi], j2 = BJ[2 * NBOX + bi];
        if (j0 == T(0) && j1 == T(0) && j2 == T(0)) continue;
        const int gi = ox + li, gj = oy + lj, gk = oz + lk;
        const long long id = g.idx(gi, gj, gk);
        const T ax_n = one_x ? T(1) : anx[gi], ax_c = one_x ? T(1) : acx[gi];
        const T ay_n = one_y ? T(1) : any[gj], ay_c = one_y ? T(1) : acy[gj];
        const T az_n = one_z ? T(1) : anz[gk], az_c = one_z ? T(1) : acz[gk];
        if (j0 != T(0)) atomicAdd(f.J[0] + id, sp.cj[0] * j0 * ax_c * ay_n * az_n);
        if (j1 != T(0)) atomicAdd(f.J[1] + id, qy * j1 * ax_n * ay_c * az_n);
        if (j2 != T(0)) atomicAdd(f.J[2] + id, sp.cj[2] * j2 * ax_n * ay_n * az_c);
      }
    } else {
      // sparse chunk: one particle at a time from global memory
      for (int i = 0; i < P; ++i) {
        const long long gp = base + tid * P + i;
        if (gp < n) pushed += particle_global<T, DIM>(g, tb, f, sp, prescribed, stg, tid * PP + i, ROW, gp);
      }
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
  const size_t smem = Plan<T, DIM, P>::total;
  static std::atomic<unsigned long long> configured{0};   // devices whose limit is set
  {
    cudaError_t e = smem_limit_once(k_pd1<T, DIM, P>, (int)smem, configured);
    if (e != cudaSuccess) return e;
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

// Particles per thread P of the run kernel: 8, else 4 (FP64: always 4).
template <typename T>
cudaError_t launch_push_deposit_runs(int ppt, const Geom& g, const Tables& tb, const FieldPtrs<T>& f,
                                     const SpeciesPtrs<T>& sp, int prescribed, unsigned* status,
                                     unsigned long long* pushed, int nsm, cudaStream_t s) {
  if (sp.capacity <= 0) return cudaSuccess;
  const bool d3 = g.dim == 3;
  if constexpr (sizeof(T) == 8) {
    return d3 ? launch_pd1_p<T, 3, 4>(g, tb, f, sp, prescribed, status, pushed, nsm, 2, s)
              : launch_pd1_p<T, 2, 4>(g, tb, f, sp, prescribed, status, pushed, nsm, 2, s);
  } else {
    if (ppt == 8)
      return d3 ? launch_pd1_p<T, 3, 8>(g, tb, f, sp, prescribed, status, pushed, nsm, 3, s)
                : launch_pd1_p<T, 2, 8>(g, tb, f, sp, prescribed, status, pushed, nsm, 3, s);
    return d3 ? launch_pd1_p<T, 3, 4>(g, tb, f, sp, prescribed, status, pushed, nsm, 4, s)
              : launch_pd1_p<T, 2, 4>(g, tb, f, sp, prescribed, status, pushed, nsm, 4, s);
  }
}

template cudaError_t launch_push_deposit_runs<float>(int, const Geom&, const Tables&, const FieldPtrs<float>&,
                                                     const SpeciesPtrs<float>&, int, unsigned*, unsigned long long*,
                                                     int, cudaStream_t);
template cudaError_t launch_push_deposit_runs<double>(int, const Geom&, const Tables&, const FieldPtrs<double>&,
                                                      const SpeciesPtrs<double>&, int, unsigned*, unsigned long long*,
                                                      int, cudaStream_t);

}  // namespace picpml
