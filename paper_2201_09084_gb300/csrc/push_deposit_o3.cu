// Fused gather + Boris + move + Esirkepov deposit + alpha-damped flush for
// cubic (order-3) shapes in 3D, over particles sorted by tile.
//
// An order-3 move adds 4 x 5 x 5 prefix values to each current component
// (300 in all).  A block takes a chunk of 128*P consecutive particles:
//   1. stage the chunk (coalesced) and find the bounding box of its cells;
//   2. load E and the time-averaged B of that box with fixed strides
//      (nodes lo-2 .. hi+3 per axis: the cubic gather reaches two nodes
//      below the cell, the deposit stencil of a move three above);
//   A. push every particle (64-point gather per component from the box),
//      write its record back and keep old and new positions in the stage;
//   B. counting-sort the chunk by anchor cell (the per-axis minimum of old and
//      new cell) and cut each anchor's particles into runs (about one per
//      thread); the E/B box is dead and becomes the current box;
//   C. for each current component in turn, every thread accumulates the 100
//      values of its run's moves in registers (the transverse factor as
//      M M' + Q DS' with M = S0 + DS/2, Q = DS/12, times the prefix sums of
//      DS along the component); a warp's lanes that share an anchor then sum
//      their values by reduce-scatters of shuffles and add them to the box
//      (every group, however small: a per-lane flush of 100 atomics made the
//      kernel's code large enough to stall on instruction fetch);
//   D. add the box to the grid with the charge factor and alpha at each
//      component's staggered location (Eq. alpha, Sec. II.B), once per node:
//      the damping of Eq. MaxwellE's source in the flush.
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
  static constexpr size_t stage = (size_t)NW * ROW * sizeof(T);
  static constexpr size_t box = (size_t)6 * NBOX * sizeof(T);
  // anchor counters, permutation and runs, in the box's last three arrays
  // (the time-averaged B, dead after the push)
  static constexpr int NKEY = (BX - 4) * (BY - 4) * (BZ - 4) + 1;
  static constexpr size_t cnt = (size_t)NKEY * sizeof(int);
  static constexpr size_t perm = (size_t)C * sizeof(unsigned short);
  static_assert(cnt + 2 * perm <= (size_t)3 * NBOX * sizeof(T), "sort arrays exceed the dead box");
  static constexpr size_t sort_at = stage + (size_t)3 * NBOX * sizeof(T);
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

// Register accumulator of one current component c of a run of order-3
// moves: w * (Esirkepov factor) prefix sums, 4 x 5 x 5 values with flat
// index q = (td * 5 + tb) * 4 + ta: ta along c (the prefix sums of DS),
// tb and td along the transverse axes b < d.  The transverse factor
// S0 S0' + DS S0'/2 + S0 DS'/2 + DS DS'/3 is evaluated as M M' + Q DS' with
// M = S0 + DS/2, Q = DS/12.  The component is a run-time value, so one copy
// of the code serves all three: its box offsets are c NBOX + ta sc + tb sb +
// td sd with the strides (1, BX, BXY) of axes c, b, d.
template <typename T>
struct Acc3 {
  static constexpr int NV = 100;
  T v[NV];
  int oc, sc, sb, sd;

  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = T(0);
  }

  // One move: DSc along the component, (Sb, DSb) and (Sd, DSd) along b, d.
  __device__ __forceinline__ void add(const T* DSc, const T* Sb, const T* DSb, const T* Sd, const T* DSd, T w) {
    T A[4];
    T run = T(0);
#pragma unroll
    for (int ta = 0; ta < 4; ++ta) {
      run += DSc[ta];
      A[ta] = w * run;
    }
#pragma unroll
    for (int td = 0; td < 5; ++td) {
      const T Md = Sd[td] + T(0.5) * DSd[td];
#pragma unroll
      for (int tb = 0; tb < 5; ++tb) {
        const T Mb = Sb[tb] + T(0.5) * DSb[tb];
        const T Tl = Mb * Md + T(1.0 / 12.0) * DSb[tb] * DSd[td];
#pragma unroll
        for (int ta = 0; ta < 4; ++ta) v[(td * 5 + tb) * 4 + ta] += A[ta] * Tl;
      }
    }
  }

  __device__ __forceinline__ int box_offset(int q) const {
    const int ta = q & 3, tb = (q >> 2) % 5, td = q / 20;
    return oc + ta * sc + tb * sb + td * sd;
  }

  // Sums the values of the lanes with member == true (one anchor) by four
  // reduce-scatters of 32 values each: after five halving steps lane L holds
  // the group's sum of flat index 32 k + L of block k, which it adds to the
  // box.  Every lane takes part and keeps its own values.
  template <bool ALL>
  __device__ __forceinline__ void group_flush(bool member, int lane, T* J, int a) const {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      T t[16];
      const bool up = (lane & 16) != 0;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int ql = 32 * k + i, qh = 32 * k + 16 + i;
        const T lo = (ql < NV && (ALL || member)) ? v[ql < NV ? ql : 0] : T(0);
        const T hi = (qh < NV && (ALL || member)) ? v[qh < NV ? qh : 0] : T(0);
        t[i] = (up ? hi : lo) + __shfl_xor_sync(0xffffffffu, up ? lo : hi, 16);
      }
#pragma unroll
      for (int lev = 1; lev < 5; ++lev) {
        const int o = 16 >> lev;
        const bool u2 = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
          const T lo = t[i], hi = t[i + o];
          t[i] = (u2 ? hi : lo) + __shfl_xor_sync(0xffffffffu, u2 ? lo : hi, o);
        }
      }
      const int q = 32 * k + lane;
      if (q < NV && t[0] != T(0)) atomicAdd(J + a + box_offset(q), t[0]);
    }
  }
};

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
  int* cnt = reinterpret_cast<int*>(smraw + PL::sort_at);
  unsigned short* perm = reinterpret_cast<unsigned short*>(smraw + PL::sort_at + PL::cnt);
  unsigned short* runs = reinterpret_cast<unsigned short*>(smraw + PL::sort_at + PL::cnt + PL::perm);
  __shared__ int s_lo[3], s_hi[3];
  __shared__ int s_scan[kNT3 / 32];
  __shared__ int s_nanchor;
  __shared__ int s_nrun;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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
          // one copy of the 64-point gather serves the six components (their
          // half-node staggers chosen at run time: E_x, E_y, E_z are half a
          // cell along x, y, z; B_x, B_y, B_z along the other two axes)
          T E[3], B[3];
#pragma unroll 1
          for (int comp = 0; comp < 6; ++comp) {
            const bool hx = comp == 0 || comp == 4 || comp == 5;
            const bool hy = comp == 1 || comp == 3 || comp == 5;
            const bool hz = comp == 2 || comp == 3 || comp == 4;
            T wx[4], wy[4], wz[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              wx[t] = hx ? wh[0][t] : w0[0][t];
              wy[t] = hy ? wh[1][t] : w0[1][t];
              wz[t] = hz ? wh[2][t] : w0[2][t];
            }
            const T v = interp3_box<BX, BXY, T>(bx_ + comp * NBOX, (hx ? sxh : sx0) + (hy ? syh : sy0) + (hz ? szh : sz0),
                                                wx, wy, wz);
            if (comp == 0) E[0] = v;
            if (comp == 1) E[1] = v;
            if (comp == 2) E[2] = v;
            if (comp == 3) B[0] = v;
            if (comp == 4) B[1] = v;
            if (comp == 5) B[2] = v;
          }
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
      // ---- B. counting sort by anchor cell, runs ----
      // (key: the anchor cell min(old, new) per axis, from s_lo - 1 to s_hi;
      // key nk collects the particles that deposit nothing; the E/B box is
      // dead: its first three arrays become the current box)
      T* const BJ = bx_;
      {
        // 16-byte stores, then the values of a last partial group
        float4* z = reinterpret_cast<float4*>(BJ);
        constexpr int PER = (int)(sizeof(float4) / sizeof(T));
        constexpr int NZ = 3 * NBOX / PER;
        for (int t = tid; t < NZ; t += kNT3) z[t] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int t = NZ * PER + tid; t < 3 * NBOX; t += kNT3) BJ[t] = T(0);
      }
      const int kdx = bdx - 4, kdy = bdy - 4, nk = kdx * kdy * (bdz - 4);
      for (int t = tid; t <= nk; t += kNT3) cnt[t] = 0;
      if (tid == 0) {
        s_nanchor = 0;
        s_nrun = 0;
      }
      __syncthreads();
      int keys[P];
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const int q = tid + k * kNT3;
        const int slot = (q / P) * PP + (q % P);
        const int c0 = bits_to_cell<T>(stg[7 * ROW + slot]);
        const int c1 = bits_to_cell<T>(stg[8 * ROW + slot]);
        if (c0 < 0 || c1 < 0) {
          keys[k] = nk;
        } else {
          const int ax = min(cell_i(c0), cell_i(c1)) - ox - 1;
          const int ay = min(cell_j(c0), cell_j(c1)) - oy - 1;
          const int az = min(cell_k(c0), cell_k(c1)) - oz - 1;
          keys[k] = ax + kdx * (ay + kdy * az);
        }
      }
      sort_runs<P, kNT3>(keys, nk, cnt, perm, runs, s_scan, &s_nanchor, &s_nrun);
      // ---- C. deposit the runs, one component at a time ----
      const int R = s_nrun;
#pragma unroll 1
      for (int c = 0; c < 3; ++c) {
        Acc3<T> acc;
        const int b = c == 0 ? 1 : 0, dd = c == 2 ? 1 : 2;   // transverse axes
        acc.oc = c * NBOX;
        acc.sc = c == 0 ? 1 : (c == 1 ? BX : BXY);
        acc.sb = b == 0 ? 1 : BX;
        acc.sd = dd == 1 ? BX : BXY;
        for (int rb = warp * 32; rb < R; rb += kNT3) {
          acc.zero();
          int key = -1;
          if (rb + lane < R) {
            const unsigned d = runs[rb + lane];
            const int st0 = d & 0x7ff, len = d >> 11;
            for (int i = 0; i < len; ++i) {
              const int slot = perm[st0 + i];
              const int cell0 = bits_to_cell<T>(stg[7 * ROW + slot]);
              const int cell1 = bits_to_cell<T>(stg[8 * ROW + slot]);
              const int c0[3] = {cell_i(cell0), cell_j(cell0), cell_k(cell0)};
              const int c1[3] = {cell_i(cell1), cell_j(cell1), cell_k(cell1)};
              // box offset of the first stencil node (the anchor minus one)
              key = (min(c0[0], c1[0]) - 1 - ox) + BX * (min(c0[1], c1[1]) - 1 - oy) +
                    BXY * (min(c0[2], c1[2]) - 1 - oz);
              auto pick = [](int a, int x, int y, int z) { return a == 0 ? x : (a == 1 ? y : z); };
              int lo;
              T Sc[5], DSc[5], Sb[5], DSb[5], Sd[5], DSd[5];
              esk_axis<3, T>(pick(c, c0[0], c0[1], c0[2]), stg[c * ROW + slot], pick(c, c1[0], c1[1], c1[2]),
                             stg[(4 + c) * ROW + slot], lo, Sc, DSc);
              esk_axis<3, T>(pick(b, c0[0], c0[1], c0[2]), stg[b * ROW + slot], pick(b, c1[0], c1[1], c1[2]),
                             stg[(4 + b) * ROW + slot], lo, Sb, DSb);
              esk_axis<3, T>(pick(dd, c0[0], c0[1], c0[2]), stg[dd * ROW + slot], pick(dd, c1[0], c1[1], c1[2]),
                             stg[(4 + dd) * ROW + slot], lo, Sd, DSd);
              acc.add(DSc, Sb, DSb, Sd, DSd, stg[3 * ROW + slot]);
            }
          }
          flush_warp_runs<1>(acc, key, lane, BJ);
        }
      }
      __syncthreads();
      // ---- D. add the current box to the grid with the charge factor and alpha ----
      const T* anx = al_node<T>(tb, 0);
      const T* acx = al_cent<T>(tb, 0);
      const T* any = al_node<T>(tb, 1);
      const T* acy = al_cent<T>(tb, 1);
      const T* anz = al_node<T>(tb, 2);
      const T* acz = al_cent<T>(tb, 2);
      for (int t = tid; t < NB; t += kNT3) {
        const int li = t % bdx, r = t / bdx, lj = r % bdy, lk = r / bdy;
        const int bi = li + BX * lj + BXY * lk;
        const T j0 = BJ[bi], j1 = BJ[NBOX + bi], j2 = BJ[2 * NBOX + bi];
        if (j0 == T(0) && j1 == T(0) && j2 == T(0)) continue;
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
  static std::atomic<unsigned long long> configured{0};   // devices whose limit is set
  {
    cudaError_t e = smem_limit_once(k_pd3<T, P>, (int)smem, configured);
    if (e != cudaSuccess) return e;
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
