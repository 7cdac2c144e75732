// Tile-resident fused gather + Boris + move + Esirkepov deposit + alpha-damped
// flush for 3D FP32 runs of shape order 1 whose species have been sorted by
// tile (the thermal plasmas of the benchmark: a few particles per cell that
// move a small fraction of a cell per step and fill the whole grid).
//
// Work unit: two sort tiles along x, i.e. 16 x 4 x 4 cells, and the particles
// of every species that sat in those cells at the last sort (one contiguous
// index range per species).  A block (persistent, two per SM) takes units
// round-robin and, per unit:
//   1. one thread issues six TMA tensor copies (cp.async.bulk.tensor, one
//      mbarrier) of the unit's field box -- E^n and B^n (the field step's
//      average of the two B half steps) over 24 x 8 x 8 nodes, i.e. the unit
//      plus every node a particle that has drifted up to one cell out of it
//      can gather from or deposit to -- and prefetches the next unit's box
//      and particle records into L2;
//   2. each thread takes about 8 consecutive particles of a species (about
//      one cell: the sort orders cells inside a tile x fastest, so the 32
//      lanes of a warp sit in one 8 x 4 layer of cells and their gathers hit
//      distinct shared-memory banks), gathers from the box, pushes, moves,
//      writes the record back, and deposits: a move that stays in its cell
//      (almost all of them) adds its 12 Esirkepov values (4 per component)
//      to one of the thread's two runs in registers (no atomics; a move in
//      a third cell sends the run used less recently to the grid and takes
//      its place), flushed once per pass to the grid with the damping
//      alpha_c at each component's staggered location (Eq. alpha, Eq.
//      MaxwellE source term); a move across a cell face is queued per
//      warp and deposited, one lane per entry, with global atomics and
//      alpha_c; a particle outside the box gathers and deposits through
//      global memory.
// Particles injected after the last sort (beyond the sorted range) are pushed
// one per thread through global memory after the units.
//
// The deterministic form (int64 deposition) loads both B half steps and
// averages after the interpolation, as the one-thread kernel does, so its
// particles move and deposit bit for bit as there.
#include <cuda.h>

#include "chunk_common.cuh"

namespace picpml {

namespace {

using namespace pc;
using namespace chunk;

// sort tile (cells) and unit
constexpr int TX = 8, TY = 4, TZ = 4;
constexpr int UXT = 2;                    // sort tiles per unit along x
constexpr int UX = TX * UXT;              // 16 cells
// box (nodes) and its origin relative to the unit's first cell
constexpr int BX = 24, BY = 8, BZ = 8;
constexpr int BXY = BX * BY, BN = BXY * BZ;
constexpr int OX = 4, OY = 2, OZ = 2;
constexpr int NT = 256;                   // threads per block (a power of two)
constexpr int PT = 12;                    // most particles per thread in one pass
constexpr int kQWords = 11;               // words of a queue entry
// Shared memory (floats): the field box (E, B^n; the deterministic form
// keeps B^{n+1/2} and B^{n-1/2}: 9 arrays), the alpha tables (node and
// centre per axis: 2 (BX + BY + BZ)), the
// warps' queues, then the mbarrier, the species' live counts and two
// buffers of the species' index ranges of a unit.
template <bool FIX>
struct Smem {
  static constexpr int box = (FIX ? 9 : 6) * BN;
  static constexpr int al = 2 * (BX + BY + BZ);
  static constexpr int queue = FIX ? 0 : (NT / 32) * kQWords * 32;
  static constexpr int floats = box + al + queue;
  static constexpr int bytes = floats * 4 + 16 + 8 * kTileMaxSpecies + 2 * 16 * kTileMaxSpecies;
  static constexpr unsigned box_bytes = (unsigned)box * 4u;
};
static_assert(Smem<false>::bytes <= 113 * 1024, "two blocks per SM");
static_assert(2 * (BX + BY + BZ) <= NT, "one thread per alpha-table entry");
static_assert((NT & (NT - 1)) == 0 && NT % 32 == 0, "thread ranks wrap with a mask");

// A particle whose cell (local to the box) lies in [OX-1, OX+UX] x [OY-1, OY+TY]
// x [OZ-1, OZ+TZ] gathers from nodes l-1 .. l+1 and deposits to nodes l .. l+1
// (l .. l+2 from the lower cell of a move across a face): all inside the box.
static_assert(OX >= 2 && OX + UX + 2 <= BX && OX % 4 == 0, "box x range");
static_assert(OY >= 2 && OY + TY + 2 <= BY && OZ >= 2 && OZ + TZ + 2 <= BZ, "box y, z range");

__device__ __forceinline__ bool in_box(int lx, int ly, int lz) {
  return (unsigned)(lx - (OX - 1)) <= (unsigned)(UX + 1) && (unsigned)(ly - (OY - 1)) <= (unsigned)(TY + 1) &&
         (unsigned)(lz - (OZ - 1)) <= (unsigned)(TZ + 1);
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits for the mbarrier phase with the given parity; gives up after 2 s of
// wall time (a copy that never lands) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* b, unsigned parity) {
  if (mbar_try_wait(b, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(b, parity))
    if (global_ns() - t0 > 2000000000ull) return false;
  return true;
}
__device__ __forceinline__ void tma_box(float* dst, const CUtensorMap* map, int x, int y, int z, int a,
                                        unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(a), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_prefetch_box(const CUtensorMap* map, int x, int y, int z, int a) {
  asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];" ::"l"(map), "r"(x), "r"(y),
               "r"(z), "r"(a)
               : "memory");
}
__device__ __forceinline__ void prefetch_l2(const void* p, long long bytes) {
  // one bulk prefetch covers at most 2^31 - 16 bytes; the ranges here are far smaller
  if (bytes > 0 && bytes < (1LL << 30))
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"((unsigned)bytes) : "memory");
}

// Trilinear interpolation in a box array from the lower corner (x, y, z)
// with fractions (fx, fy, fz): the order-1 B-spline gather.
__device__ __forceinline__ float tri(const float* F, int x, float fx, int y, float fy, int z, float fz) {
  const float* p = F + x + BX * y + BXY * z;
  const float a0 = p[0], a1 = p[1], b0 = p[BX], b1 = p[BX + 1];
  const float c0 = p[BXY], c1 = p[BXY + 1], d0 = p[BXY + BX], d1 = p[BXY + BX + 1];
  const float a = fmaf(fx, a1 - a0, a0), b = fmaf(fx, b1 - b0, b0);
  const float c = fmaf(fx, c1 - c0, c0), d = fmaf(fx, d1 - d0, d0);
  const float e = fmaf(fy, b - a, a), h = fmaf(fy, d - c, c);
  return fmaf(fz, h - e, e);
}

// The order-1 gather of the one-thread kernel (interp(): the same weights and
// the same order of the sums) from a box array, local indices: the
// deterministic form uses it so that a particle moves bit for bit as it does
// in the other kernels, whichever kernel pushes it.
__device__ __forceinline__ float interp_box(const float* F, int bx, const float* wx, int by, const float* wy, int bz,
                                            const float* wz) {
  float acc = 0.0f;
#pragma unroll
  for (int tz = 0; tz < 2; ++tz)
#pragma unroll
    for (int ty = 0; ty < 2; ++ty) {
      const float wyz = wy[ty] * wz[tz];
      const float* row = F + bx + BX * (by + ty) + BXY * (bz + tz);
      float racc = 0.0f;
#pragma unroll
      for (int tx = 0; tx < 2; ++tx) racc += wx[tx] * row[tx];
      acc += wyz * racc;
    }
  return acc;
}

// Index range [beg, end) of species s in the unit whose first sort tile is t0
// (nt tiles), clamped to the live count.
__device__ __forceinline__ void unit_range(const TileSpecies& S, long long t0, int nt, long long n, long long& beg,
                                           long long& end) {
  beg = t0 > 0 ? S.tile_end[t0 - 1] : 0;
  end = S.tile_end[t0 + nt - 1];
  if (end > n) end = n;
  if (beg > end) beg = end;
}

// Runs of in-cell moves: each thread keeps the 12 Esirkepov values of the
// charge-scaled current J' (4 per component) at two box cells (its particles
// span one or two sort cells) in registers, so no atomics are needed until
// the flush at the end of the pass, or until a move in a third cell evicts
// the run used less recently.  (Runs in per-thread shared memory freed
// the registers but were slower: they add six 16-byte shared accesses per
// particle to a shared-memory pipe the gather already loads heavily.)
struct Runs {
  int cell[2];   // local linear cell index, -1 when free
  float v[2][12];
  __device__ __forceinline__ void clear() {
    cell[0] = cell[1] = -1;
#pragma unroll
    for (int t = 0; t < 12; ++t) v[0][t] = v[1][t] = 0.0f;
  }
};

// Adds the 12 values v of local box cell L to the grid's current with native
// global float reductions (in L2).  The node's damping alpha_c (Eq. alpha, at
// the component's staggered location) multiplies the value unless the unit's
// whole box lies where alpha = 1.  al: the unit's alpha tables (x node,
// x centre, y node, y centre, z node, z centre); org: the box origin in grid
// cells.  Slots: J_x at (x centre, y node +b, z node +c): v[b + 2c]; J_y at
// (x node +a, y centre, z node +c): v[4 + a + 2c]; J_z at (x node +a, y node
// +b, z centre): v[8 + a + 2b].
__device__ __forceinline__ void red_cell(const float v[12], int L, const Geom& g, const FieldPtrs<float>& f,
                                         const int org[3], const float* al, bool alpha_one) {
  const int lx = L % BX, ly = (L / BX) % BY, lz = L / BXY;
  const long long base = g.idx(org[0] + lx, org[1] + ly, org[2] + lz);
  const int lc[3] = {lx, ly, lz};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int e1 = c == 0 ? 1 : 0, e2 = c == 2 ? 1 : 2;   // axes of the +1, +2 slots
    const long long s1 = e1 == 0 ? 1 : (e1 == 1 ? g.sy : g.sz);
    const long long s2 = e2 == 1 ? g.sy : g.sz;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float x = v[4 * c + t];
      if (!alpha_one) {
        int n[3] = {lc[0], lc[1], lc[2]};
        n[e1] += t & 1;
        n[e2] += t >> 1;
        const float ax = c == 0 ? al[BX + n[0]] : al[n[0]];
        const float ay = c == 1 ? al[2 * BX + BY + n[1]] : al[2 * BX + n[1]];
        const float az = c == 2 ? al[2 * BX + 2 * BY + BZ + n[2]] : al[2 * BX + 2 * BY + n[2]];
        x *= ax * ay * az;
      }
      atomicAdd(f.J[c] + base + (t & 1) * s1 + (t >> 1) * s2, x);
    }
  }
}

// Adds the runs to the grid's current (red_cell): the 32 lanes of a warp
// hold runs at distinct cells of one 8 x 4 layer, so each reduction
// instruction covers a few sectors.
__device__ __forceinline__ void flush_runs(const Runs& R, const Geom& g, const FieldPtrs<float>& f,
                                           const int org[3], const float* al, bool alpha_one) {
#pragma unroll
  for (int r = 0; r < 2; ++r)
    if (R.cell[r] >= 0) red_cell(R.v[r], R.cell[r], g, f, org, al, alpha_one);
}

// Esirkepov current of a move that stays in its cell (Esirkepov's density
// decomposition with S1 - S0 nonzero only on the cell's two nodes per axis):
// J'_x(b, c) = cj_x w (-d_x) (M_y[b] M_z[c] + (-1)^{b+c} d_y d_z / 12) with
// the mid-move shape M = (1 - m, m), m = (o0 + o1)/2, d = o1 - o0 (the
// transverse factor S0 S0' + DS S0'/2 + S0 DS'/2 + DS DS'/3 = M M' + DS DS'/12).
// add_in_cell: the 12 values (slots as in red_cell) added s0 times to run 0
// and s1 times to run 1 (s0, s1 in {0, 1}).
__device__ __forceinline__ void add_in_cell(Runs& r, const float o0[3], const float o1[3], const float qw[3],
                                            float s0, float s1) {
  float d[3], m[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    d[a] = o1[a] - o0[a];
    m[a] = 0.5f * (o0[a] + o1[a]);
  }
  const float c12 = 1.0f / 12.0f;
  const float eyz = c12 * d[1] * d[2], exz = c12 * d[0] * d[2], exy = c12 * d[0] * d[1];
  const float mx0 = 1.0f - m[0], my0 = 1.0f - m[1], mz0 = 1.0f - m[2];
  float T[12];
  T[0] = fmaf(my0, mz0, eyz);
  T[1] = fmaf(m[1], mz0, -eyz);
  T[2] = fmaf(my0, m[2], -eyz);
  T[3] = fmaf(m[1], m[2], eyz);
  T[4] = fmaf(mx0, mz0, exz);
  T[5] = fmaf(m[0], mz0, -exz);
  T[6] = fmaf(mx0, m[2], -exz);
  T[7] = fmaf(m[0], m[2], exz);
  T[8] = fmaf(mx0, my0, exy);
  T[9] = fmaf(m[0], my0, -exy);
  T[10] = fmaf(mx0, m[1], -exy);
  T[11] = fmaf(m[0], m[1], exy);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float a = -qw[c] * d[c];
    const float a0 = s0 * a, a1 = s1 * a;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      r.v[0][4 * c + t] = fmaf(a0, T[4 * c + t], r.v[0][4 * c + t]);
      r.v[1][4 * c + t] = fmaf(a1, T[4 * c + t], r.v[1][4 * c + t]);
    }
  }
}

// Deferred deposits of one warp (moves across a cell face): structure of
// arrays of 32 entries, grid cells (packed) and offsets before and after,
// and the charge-scaled weight per component.
struct Queue {
  float* q;   // kQWords * 32 floats of this warp
  __device__ __forceinline__ void put(int k, int C0, const float o0[3], int C1, const float o1[3],
                                      const float qw[3]) {
    q[0 * 32 + k] = __int_as_float(C0);
    q[1 * 32 + k] = o0[0];
    q[2 * 32 + k] = o0[1];
    q[3 * 32 + k] = o0[2];
    q[4 * 32 + k] = __int_as_float(C1);
    q[5 * 32 + k] = o1[0];
    q[6 * 32 + k] = o1[1];
    q[7 * 32 + k] = o1[2];
    q[8 * 32 + k] = qw[0];
    q[9 * 32 + k] = qw[1];
    q[10 * 32 + k] = qw[2];
  }
};

// Deposits the first n entries of a warp's queue, lane k entry k, with the
// global Esirkepov deposit and alpha_c at each staggered location (every lane
// of the warp calls it: at the end of a unit, or when the queue fills).
// Inlined: a call from the particle loop would make the loop keep its values
// across the call (measured slower).
__device__ __forceinline__ void drain_queue(const float* q, int n, const Geom& g, const Tables& tb,
                                            const FieldPtrs<float>& f) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  if (lane < n) {
    const int C0 = __float_as_int(q[lane]), C1 = __float_as_int(q[4 * 32 + lane]);
    const int c0[3] = {cell_i(C0), cell_j(C0), cell_k(C0)};
    const int c1[3] = {cell_i(C1), cell_j(C1), cell_k(C1)};
    const float o0[3] = {q[1 * 32 + lane], q[2 * 32 + lane], q[3 * 32 + lane]};
    const float o1[3] = {q[5 * 32 + lane], q[6 * 32 + lane], q[7 * 32 + lane]};
    SpeciesPtrs<float> sq{};
    sq.cj[0] = q[8 * 32 + lane];
    sq.cj[1] = q[9 * 32 + lane];
    sq.cj[2] = q[10 * 32 + lane];
    deposit_one<1, 3, float>(g, tb, f, sq, c0, o0, c1, o1, 1.0f, 0.0f);
  }
  __syncwarp();
}

// Gather from global memory, push, move and deposit with global atomics: the
// path of a particle outside its unit's box.
template <bool FIX>
__device__ __forceinline__ void particle_global(const Geom& g, const Tables& tb, const FieldPtrs<float>& f,
                                                const SpeciesPtrs<float>& sp, long long p, int prescribed,
                                                unsigned* status, unsigned* pushed) {
  float4* P = reinterpret_cast<float4*>(sp.pos);
  float4* Mo = reinterpret_cast<float4*>(sp.mom);
  const float4 a = P[p], b = Mo[p];
  const int cell = __float_as_int(b.w);
  if (cell < 0) return;
  const int c[3] = {cell_i(cell), cell_j(cell), cell_k(cell)};
  float o[3] = {a.x, a.y, a.z}, u[3] = {b.x, b.y, b.z};
  const float w = a.w;
  bool bad = !finite_value(w);
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    if (!finite_value(u[ax])) bad = true;
    if (c[ax] < g.rmin[ax] || c[ax] > g.rmax[ax] || !(o[ax] >= 0.0f && o[ax] < 1.0f)) bad = true;
  }
  if (bad) {
    atomicOr(status, ST_BAD_PARTICLE);
    Mo[p] = make_float4(b.x, b.y, b.z, __int_as_float(-1));
    return;
  }
  if (!prescribed) {
    int b0[3], bh[3];
    float w0[3][2], wh[3][2], E[3], B[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) axis_weights<1, float>(c[ax], o[ax], b0[ax], w0[ax], bh[ax], wh[ax]);
    E[0] = interp<1, 3, float>(g, f.E[0], bh[0], wh[0], b0[1], w0[1], b0[2], w0[2]);
    E[1] = interp<1, 3, float>(g, f.E[1], b0[0], w0[0], bh[1], wh[1], b0[2], w0[2]);
    E[2] = interp<1, 3, float>(g, f.E[2], b0[0], w0[0], b0[1], w0[1], bh[2], wh[2]);
    B[0] = interp_avg<1, 3, float>(g, f.Bh[0], f.Bp[0], b0[0], w0[0], bh[1], wh[1], bh[2], wh[2]);
    B[1] = interp_avg<1, 3, float>(g, f.Bh[1], f.Bp[1], bh[0], wh[0], b0[1], w0[1], bh[2], wh[2]);
    B[2] = interp_avg<1, 3, float>(g, f.Bh[2], f.Bp[2], bh[0], wh[0], bh[1], wh[1], b0[2], w0[2]);
    boris<float>(u, E, B, sp.ke);
  }
  *pushed += 1;
  int c1[3];
  float o1[3], ig;
  const bool ok = move_particle<3, float>(g, o, c, u, c1, o1, ig);
  float wd = w, wn = w;
  if (g.wdamp && ok) {
    const float I = weight_exponent<float>(g, c, o, c1, o1);
    wd = w * expf(-0.5f * I);
    wn = w * expf(-I);
  }
  P[p] = ok ? make_float4(o1[0], o1[1], o1[2], wn) : a;
  Mo[p] = make_float4(u[0], u[1], u[2], __int_as_float(ok ? pack_cell(c1[0], c1[1], c1[2]) : -1));
  if (!ok) return;
  if constexpr (FIX)
    deposit_fixed<1>(g, f, sp.qn, c, o, c1, o1, wd, status);
  else
    deposit_one<1, 3, float>(g, tb, f, sp, c, o, c1, o1, wd, 0.0f);
}

// The values of a species the box path reads per particle, held in registers
// (the species table itself lives in the kernel's parameter space).
struct Hot {
  float4* pos;
  float4* mom;
  float ke, cj0, cj1, cj2;
  double qn;   // charge in elementary charges (deterministic deposit)
};

// What the box path leaves for the deposit: nothing (removed or refused), an
// in-cell move, a move across a face inside the box, or the whole particle
// for the global path (its cell, or its new cell, lies outside the box; the
// record is then left as it was).
enum : int { DEP_NONE = 0, DEP_IN_CELL = 1, DEP_ACROSS = 2, DEP_OUT = 3 };

// One particle of the box path: checks, gather from the box, Boris push,
// move, record write-back.  Returns the deposit kind with the local cell L0,
// the packed grid cells C0 (before) and C1 (after), the offsets o (before)
// and o1 (after) and the mid-step weight.
//
// FIX: the deterministic form.  The gather reads E, B^{n+1/2} and B^{n-1/2}
// from the box with the one-thread kernel's arithmetic (interp_box, B^n
// averaged after the interpolation), the move is always the float-float one,
// and the particle deposits its integer Esirkepov sums with int64 atomics
// (deposit_fixed) straight away: the result does not depend on the kernel,
// the particle order or the launch shape.
template <bool FIX>
__device__ __forceinline__ int box_particle(const Geom& g, const Hot& h, const FieldPtrs<float>& f, long long p,
                                            float4 a, float4 b, const float* F, const int org[3], int prescribed,
                                            unsigned* status, unsigned& pushed, int& L0, int& C0, int& C1,
                                            float o[3], float o1[3], float& wd) {
  const int cell = __float_as_int(b.w);
  if (cell < 0) return DEP_NONE;
  const int c[3] = {cell_i(cell), cell_j(cell), cell_k(cell)};
  const int l[3] = {c[0] - org[0], c[1] - org[1], c[2] - org[2]};
  if (!in_box(l[0], l[1], l[2])) return DEP_OUT;   // drifted out of the unit's box since the sort
  o[0] = a.x; o[1] = a.y; o[2] = a.z;
  float u[3] = {b.x, b.y, b.z};
  const float w = a.w;
  bool bad = !finite_value(w);
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    if (!finite_value(u[ax])) bad = true;
    if (c[ax] < g.rmin[ax] || c[ax] > g.rmax[ax] || !(o[ax] >= 0.0f && o[ax] < 1.0f)) bad = true;
  }
  float4* P = h.pos;
  float4* Mo = h.mom;
  if (bad) {
    atomicOr(status, ST_BAD_PARTICLE);
    Mo[p] = make_float4(b.x, b.y, b.z, __int_as_float(-1));
    return DEP_NONE;
  }
  if (FIX && !prescribed) {
    int b0[3], bh[3];
    float w0[3][2], wh[3][2], E[3], B[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      axis_weights<1, float>(c[ax], o[ax], b0[ax], w0[ax], bh[ax], wh[ax]);
      b0[ax] -= org[ax];
      bh[ax] -= org[ax];
    }
    E[0] = interp_box(F + 0 * BN, bh[0], wh[0], b0[1], w0[1], b0[2], w0[2]);
    E[1] = interp_box(F + 1 * BN, b0[0], w0[0], bh[1], wh[1], b0[2], w0[2]);
    E[2] = interp_box(F + 2 * BN, b0[0], w0[0], b0[1], w0[1], bh[2], wh[2]);
    B[0] = 0.5f * (interp_box(F + 3 * BN, b0[0], w0[0], bh[1], wh[1], bh[2], wh[2]) +
                   interp_box(F + 6 * BN, b0[0], w0[0], bh[1], wh[1], bh[2], wh[2]));
    B[1] = 0.5f * (interp_box(F + 4 * BN, bh[0], wh[0], b0[1], w0[1], bh[2], wh[2]) +
                   interp_box(F + 7 * BN, bh[0], wh[0], b0[1], w0[1], bh[2], wh[2]));
    B[2] = 0.5f * (interp_box(F + 5 * BN, bh[0], wh[0], bh[1], wh[1], b0[2], w0[2]) +
                   interp_box(F + 8 * BN, bh[0], wh[0], bh[1], wh[1], b0[2], w0[2]));
    boris<float>(u, E, B, h.ke);
  } else if (!prescribed) {
    int bc[3];
    float wc[3], E[3], B[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const bool low = o[ax] < 0.5f;
      bc[ax] = l[ax] - (low ? 1 : 0);
      wc[ax] = low ? o[ax] + 0.5f : o[ax] - 0.5f;
    }
    E[0] = tri(F + 0 * BN, bc[0], wc[0], l[1], o[1], l[2], o[2]);
    E[1] = tri(F + 1 * BN, l[0], o[0], bc[1], wc[1], l[2], o[2]);
    E[2] = tri(F + 2 * BN, l[0], o[0], l[1], o[1], bc[2], wc[2]);
    B[0] = tri(F + 3 * BN, l[0], o[0], bc[1], wc[1], bc[2], wc[2]);
    B[1] = tri(F + 4 * BN, bc[0], wc[0], l[1], o[1], bc[2], wc[2]);
    B[2] = tri(F + 5 * BN, bc[0], wc[0], bc[1], wc[1], l[2], o[2]);
    boris<float>(u, E, B, h.ke);
  }
  int c1[3];
  bool ok;
  {
    // A displacement below 1/16 cell (slow particles) is formed in FP32: its
    // rounding error (a few 2^-24 of at most 1/16 cell) is far below the
    // offset's own rounding.  Longer ones need the float-float move, so that
    // a fast particle's position carries no systematic per-step error; the
    // box path leaves them to the global path (the record is not written
    // yet), which keeps the float-float move out of the particle loop.  The
    // deterministic form always takes the float-float move.
    if (FIX) {
      float igg;
      ok = move_particle<3, float>(g, o, c, u, c1, o1, igg);
    } else {
      const float ig = rsqrtf(1.0f + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
      float d[3];
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) d[ax] = g.Sf[ax] * u[ax] * ig;
      if (!(fmaxf(fabsf(d[0]), fmaxf(fabsf(d[1]), fabsf(d[2]))) < 0.0625f)) return DEP_OUT;
      bool outside = false;
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        c1[ax] = c[ax];
        float x = o[ax] + d[ax];
        if (x >= 1.0f) {
          x -= 1.0f;
          c1[ax] += 1;
        } else if (x < 0.0f) {
          x += 1.0f;
          c1[ax] -= 1;
          if (x >= 1.0f) {   // x was a tiny negative number: stay on the node
            x = 0.0f;
            c1[ax] += 1;
          }
        }
        o1[ax] = x;
        if (c1[ax] < g.rmin[ax] || c1[ax] > g.rmax[ax] || (c1[ax] == g.rmax[ax] && x > 0.0f)) outside = true;
      }
      ok = !outside;
    }
  }
  if (!FIX && ok && !in_box(c1[0] - org[0], c1[1] - org[1], c1[2] - org[2])) return DEP_OUT;
  ++pushed;
  float wn = w;
  wd = w;
  if (g.wdamp && ok) {   // weight damping: mid-step weight for the current, then decay
    const float I = weight_exponent<float>(g, c, o, c1, o1);
    wd = w * expf(-0.5f * I);
    wn = w * expf(-I);
  }
  const int cell1 = pack_cell(c1[0], c1[1], c1[2]);
  // streaming stores: the records are not read again in this launch, so they
  // need not displace the next unit's prefetched box and records in L2
  __stcs(P + p, ok ? make_float4(o1[0], o1[1], o1[2], wn) : a);
  __stcs(Mo + p, make_float4(u[0], u[1], u[2], __int_as_float(ok ? cell1 : -1)));
  if (!ok) return DEP_NONE;
  if constexpr (FIX) {
    deposit_fixed<1>(g, f, h.qn, c, o, c1, o1, wd, status);
    return DEP_NONE;
  }
  L0 = l[0] + BX * l[1] + BXY * l[2];
  C0 = cell;
  C1 = cell1;
  return cell1 == cell ? DEP_IN_CELL : DEP_ACROSS;
}

// One thread's consecutive particles [p0, p1) of a species, at most `iters`
// (every lane of the warp calls it with the same `iters`): box path, runs,
// deferred queue, then the flush of the runs.  Particles outside the box go
// through the global path after the loop.
template <bool FIX>
__device__ __forceinline__ void thread_pass(const Geom& g, const Tables& tb, const FieldPtrs<float>& f,
                                            const SpeciesPtrs<float>& sp, long long p0, long long p1, int iters,
                                            const float* F, Queue& Q, int& qn, const int org[3],
                                            const float* al, bool alpha_one, int prescribed, unsigned* status,
                                            unsigned& pushed) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const Hot h = {reinterpret_cast<float4*>(sp.pos), reinterpret_cast<float4*>(sp.mom), sp.ke, sp.cj[0], sp.cj[1],
                 sp.cj[2], sp.qn};
  const float4* P = h.pos;
  const float4* Mo = h.mom;
  Runs R;
  R.clear();
  int mru = 0;        // the run used last
  unsigned out = 0;   // particles of this thread for the global path
  float4 na = make_float4(0.f, 0.f, 0.f, 0.f), nb = na;
  if (p0 < p1) {
    na = P[p0];
    nb = Mo[p0];
  }
  for (int i = 0; i < iters; ++i) {
    const long long p = p0 + i;
    const float4 a = na, b = nb;
    if (p + 1 < p1) {   // the next record is loaded while this one is worked on
      na = P[p + 1];
      nb = Mo[p + 1];
    }
    int L0 = -1, C0 = 0, C1 = 0, kind = DEP_NONE;
    float o[3], o1[3], wd = 0.0f;
    if (p < p1)
      kind = box_particle<FIX>(g, h, f, p, a, b, F, org, prescribed, status, pushed, L0, C0, C1, o, o1, wd);
    if (kind == DEP_OUT) out |= 1u << i;
    if (FIX) continue;
    const bool toq = kind == DEP_ACROSS;
    if (kind == DEP_IN_CELL) {
      bool r0 = R.cell[0] == L0 || R.cell[0] < 0;
      bool r1 = !r0 && (R.cell[1] == L0 || R.cell[1] < 0);
      if (!r0 && !r1) {
        // a third cell: the run used less recently goes to the grid and
        // takes this cell, so the particles of each cell visited in turn
        // (the thread's next sorted cell after a particle that had moved)
        // still accumulate in registers
        const bool v1 = mru == 0;
        float v[12];
#pragma unroll
        for (int t = 0; t < 12; ++t) v[t] = v1 ? R.v[1][t] : R.v[0][t];
        red_cell(v, v1 ? R.cell[1] : R.cell[0], g, f, org, al, alpha_one);
#pragma unroll
        for (int t = 0; t < 12; ++t) {
          R.v[0][t] = v1 ? R.v[0][t] : 0.0f;
          R.v[1][t] = v1 ? 0.0f : R.v[1][t];
        }
        r0 = !v1;
        r1 = v1;
      }
      if (r0) R.cell[0] = L0;
      if (r1) R.cell[1] = L0;
      mru = r0 ? 0 : 1;
      const float qw[3] = {h.cj0 * wd, h.cj1 * wd, h.cj2 * wd};
      add_in_cell(R, o, o1, qw, r0 ? 1.0f : 0.0f, r0 ? 0.0f : 1.0f);
    }
    const unsigned m = __ballot_sync(0xffffffffu, toq);
    if (m) {
      if (qn + __popc(m) > 32) {
        drain_queue(Q.q, qn, g, tb, f);
        qn = 0;
      }
      if (toq) {
        const float qw[3] = {h.cj0 * wd, h.cj1 * wd, h.cj2 * wd};
        Q.put(qn + __popc(m & lt), C0, o, C1, o1, qw);
      }
      qn += __popc(m);
    }
  }
  if (!FIX) flush_runs(R, g, f, org, al, alpha_one);
  while (out) {
    const int i = __ffs(out) - 1;
    out &= out - 1;
    particle_global<FIX>(g, tb, f, sp, p0 + i, prescribed, status, &pushed);
  }
}

template <bool FIX>
__global__ void __launch_bounds__(NT, 2)
    k_tile(const __grid_constant__ Geom g, const __grid_constant__ Tables tb,
           const __grid_constant__ FieldPtrs<float> f, const __grid_constant__ TileLaunch L,
           const __grid_constant__ CUtensorMap tmap, unsigned* status, unsigned long long* pushed_total) {
  using S = Smem<FIX>;
  extern __shared__ __align__(128) float smem[];
  float* F = smem;   // E (3), then B^n (3), or B^{n+1/2} (3) and B^{n-1/2} (3) in the deterministic form
  const int tid = threadIdx.x;
  float* al = smem + S::box;   // alpha at the box's nodes / centres: x n, x c, y n, y c, z n, z c
  Queue Q;
  Q.q = al + S::al + (tid >> 5) * (kQWords * 32);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + S::floats);

  const int tx = (g.N[0] + TX - 1) / TX, ty = (g.N[1] + TY - 1) / TY, tz = (g.N[2] + TZ - 1) / TZ;
  const int ux = (tx + UXT - 1) / UXT;
  const long long nunits = (long long)ux * ty * tz;
  long long* nlive = reinterpret_cast<long long*>(bar + 1);   // live count of each species
  // [beg, end) of every species in a unit, two buffers: thread 0 fills the
  // other buffer with the block's next unit while this one is worked on, so
  // a unit starts without waiting on global loads of the tile ends
  long long* urange = nlive + kTileMaxSpecies;
  if (tid < L.nsp) nlive[tid] = *L.s[tid].sp.n_dev;
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  unsigned parity = 0, pushed = 0;
  bool alive = true;
  // tensor-map arrays of the box: E, then B^n (or B^{n+1/2}, B^{n-1/2})
  int arr[9];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    arr[c] = L.arr_E[c];
    arr[3 + c] = FIX ? L.arr_Bh[c] : L.arr_Bn[c];
    arr[6 + c] = L.arr_Bp[c];
  }
  constexpr int kArrays = FIX ? 9 : 6;

  int buf = 0;          // the urange buffer of the current unit
  bool ahead = false;   // it was filled during the previous unit
  for (long long u = blockIdx.x; u < nunits && alive; u += gridDim.x) {
    const int iu = (int)(u % ux);
    const long long r = u / ux;
    const int jt = (int)(r % ty), kt = (int)(r / ty);
    const long long t0 = (long long)iu * UXT + (long long)tx * (jt + (long long)ty * kt);
    const int nt = min(UXT, tx - iu * UXT);
    long long* ur = urange + buf * 2 * kTileMaxSpecies;
    if (!ahead) {
      if (tid < L.nsp) unit_range(L.s[tid], t0, nt, nlive[tid], ur[2 * tid], ur[2 * tid + 1]);
      __syncthreads();
    }
    long long total = 0;
    for (int s = 0; s < L.nsp; ++s) total += ur[2 * s + 1] - ur[2 * s];
    if (total == 0) {   // uniform across the block; the next unit fills the other buffer
      buf ^= 1;
      ahead = false;
      continue;
    }
    const int org[3] = {iu * UX - OX, jt * TY - OY, kt * TZ - OZ};
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(bar, S::box_bytes);
#pragma unroll
      for (int c = 0; c < kArrays; ++c) tma_box(F + c * BN, &tmap, org[0], org[1], org[2], arr[c], bar);
      // the block's next unit: its field box and particle records into L2
      const long long un = u + gridDim.x;
      if (un < nunits) {
        const int iu2 = (int)(un % ux);
        const long long r2 = un / ux;
        const int jt2 = (int)(r2 % ty), kt2 = (int)(r2 / ty);
        const long long t2 = (long long)iu2 * UXT + (long long)tx * (jt2 + (long long)ty * kt2);
        const int nt2 = min(UXT, tx - iu2 * UXT);
        long long tot2 = 0;
        long long* ur2 = urange + (buf ^ 1) * 2 * kTileMaxSpecies;
        for (int s = 0; s < L.nsp; ++s) {
          long long b, e;
          unit_range(L.s[s], t2, nt2, nlive[s], b, e);
          ur2[2 * s] = b;
          ur2[2 * s + 1] = e;
          tot2 += e - b;
          prefetch_l2(reinterpret_cast<const float4*>(L.s[s].sp.pos) + b, (e - b) * 16);
          prefetch_l2(reinterpret_cast<const float4*>(L.s[s].sp.mom) + b, (e - b) * 16);
        }
        if (tot2 > 0) {
          const int x2 = iu2 * UX - OX, y2 = jt2 * TY - OY, z2 = kt2 * TZ - OZ;
#pragma unroll
          for (int c = 0; c < kArrays; ++c) tma_prefetch_box(&tmap, x2, y2, z2, arr[c]);
        }
      }
    }
    // alpha tables of this box (0 outside the grid, where no current lands)
    if (tid < S::al) {
      int ax, i, stag;
      if (tid < 2 * BX) { ax = 0; i = tid % BX; stag = tid / BX; }
      else if (tid < 2 * (BX + BY)) { ax = 1; i = (tid - 2 * BX) % BY; stag = (tid - 2 * BX) / BY; }
      else { ax = 2; i = (tid - 2 * (BX + BY)) % BZ; stag = (tid - 2 * (BX + BY)) / BZ; }
      const int gi = org[ax] + i;
      float v = 0.0f;
      if (gi >= 0 && gi < g.nn[ax]) v = stag ? tb.al_cf[ax][gi] : tb.al_nf[ax][gi];
      al[tid] = v;
    }
    // alpha = 1 over the whole box (nodes and centres org .. org + extent - 1 on every axis)
    const bool alpha_one = org[0] >= tb.al1_lo[0] && org[0] + BX - 1 <= tb.al1_hi[0] && org[1] >= tb.al1_lo[1] &&
                           org[1] + BY - 1 <= tb.al1_hi[1] && org[2] >= tb.al1_lo[2] &&
                           org[2] + BZ - 1 <= tb.al1_hi[2];
    const bool got = mbar_wait_bounded(bar, parity);
    parity ^= 1u;
    if (!__syncthreads_and(got)) {
      // give the late copy (it lands in this block's shared memory) one more
      // bounded wait before the block leaves
      if (tid == 0) {
        atomicOr(status, ST_TIMEOUT);
        (void)mbar_wait_bounded(bar, parity ^ 1u);
      }
      __syncthreads();
      alive = false;
      break;
    }
    int qn = 0;   // entries in this warp's queue (the same in every lane)
    int xs = 0;   // first thread of the next pass's extra particles (a multiple of 32)
    for (int s = 0; s < L.nsp; ++s) {
      const TileSpecies& Sp = L.s[s];
      const long long beg = ur[2 * s], end = ur[2 * s + 1];
      // passes of at most NT * PT particles; in a pass of m particles the
      // thread of rank t = (tid - xs) mod NT takes q or q + 1 consecutive
      // ones (q = m / NT, ranks below m % NT one more), so only the warps
      // holding the extra particles run the extra iteration; the extras of
      // the next pass start at the warp after them, which spreads the extra
      // iterations of a unit's passes over its warps
      const long long npass = (end - beg + NT * PT - 1) / (NT * PT);
      for (long long k = 0; k < npass; ++k) {
        const long long b0 = beg + (end - beg) * k / npass, b1 = beg + (end - beg) * (k + 1) / npass;
        const int m = (int)(b1 - b0);
        const int q = m / NT, rem = m % NT;
        const int t = (tid - xs) & (NT - 1);
        const long long p0 = b0 + (long long)q * t + min(t, rem);
        const long long p1 = p0 + q + (t < rem ? 1 : 0);
        thread_pass<FIX>(g, tb, f, Sp.sp, p0, p1, q + ((t & ~31) < rem ? 1 : 0), F, Q, qn, org, al, alpha_one,
                         L.prescribed, status, pushed);
        xs = (xs + ((rem + 31) & ~31)) & (NT - 1);
      }
    }
    if (!FIX && qn) drain_queue(Q.q, qn, g, tb, f);
    __syncthreads();   // the next unit's copy may overwrite the box: every thread is past it
    buf ^= 1;
    ahead = u + gridDim.x < nunits;   // thread 0 filled the other buffer with it
  }
  // particles added after the last sort: one per thread, through global memory
  if (alive) {
    const long long ntiles = (long long)tx * ty * tz;
    for (int s = 0; s < L.nsp; ++s) {
      const long long b = L.s[s].tile_end[ntiles - 1];
      for (long long p = b + (long long)blockIdx.x * NT + tid; p < nlive[s]; p += (long long)gridDim.x * NT)
        particle_global<FIX>(g, tb, f, L.s[s].sp, p, L.prescribed, status, &pushed);
    }
  }
  const unsigned wsum = __reduce_add_sync(0xffffffffu, pushed);
  if ((tid & 31) == 0 && wsum) atomicAdd(pushed_total, (unsigned long long)wsum);
}

// End offset of every sort tile's particles: the scattered cursor of a
// tile's last key (the keys of a tile are consecutive).
__global__ void k_tile_ends(const unsigned* cursor, long long ntiles, int keys_per_tile, long long* tile_end) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < ntiles;
       t += (long long)gridDim.x * blockDim.x)
    tile_end[t] = cursor[(t + 1) * keys_per_tile - 1];
}

}  // namespace

long long tile_count(const Geom& g) {
  if (g.dim != 3) return 0;
  return (long long)((g.N[0] + TX - 1) / TX) * ((g.N[1] + TY - 1) / TY) * ((g.N[2] + TZ - 1) / TZ);
}

cudaError_t launch_tile_ends(const Geom& g, const unsigned* cursor, long long* tile_end, cudaStream_t s) {
  const long long nt = tile_count(g);
  if (nt <= 0) return cudaSuccess;
  long long blocks = (nt + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_tile_ends<<<(unsigned)blocks, 256, 0, s>>>(cursor, nt, TX * TY * TZ, tile_end);
  return cudaGetLastError();
}

// Tensor map of the field allocation from its first FP32 array on, as
// `arrays` arrays of `size` FP32 elements (E, B^{n+1/2}, B^{n-1/2}, J per
// component; the FP64 split parts; B^n per component where present): one 4D
// tensor (x, y, z, array) whose boxes are the 24 x 8 x 8-node field boxes of
// the tile kernel.  Out-of-grid parts of a box read as zero.
cudaError_t make_tile_tensor_map(const Geom& g, const float* base, int arrays, void* map_out) {
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<Encode>(fn);
  }
  const cuuint64_t dims[4] = {(cuuint64_t)g.nn[0], (cuuint64_t)g.nn[1], (cuuint64_t)g.nn[2], (cuuint64_t)arrays};
  const cuuint64_t strides[3] = {(cuuint64_t)g.sy * 4, (cuuint64_t)g.sz * 4, (cuuint64_t)g.size * 4};
  const cuuint32_t box[4] = {BX, BY, BZ, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = encode(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                      const_cast<float*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int tile_map_bytes() { return (int)sizeof(CUtensorMap); }

// B at the integer time from the two B half steps, (Bh + Bp)/2 per node, for
// the box path when B was set from outside the field step.
__global__ void k_bn_average(FieldPtrs<float> f, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < 3; ++c) f.Bn[c][i] = 0.5f * (f.Bh[c][i] + f.Bp[c][i]);
}

cudaError_t launch_bn_average(const Geom& g, const FieldPtrs<float>& f, cudaStream_t s) {
  if (!f.Bn[0]) return cudaErrorInvalidValue;
  long long blocks = (g.size + 255) / 256;
  if (blocks > 65536) blocks = 65536;
  k_bn_average<<<(unsigned)blocks, 256, 0, s>>>(f, g.size);
  return cudaGetLastError();
}

cudaError_t launch_tile(const Geom& g, const Tables& tb, const FieldPtrs<float>& f, const TileLaunch& L,
                        const void* map, unsigned* status, unsigned long long* pushed, int nsm, cudaStream_t s) {
  if (L.nsp <= 0) return cudaSuccess;
  const bool fix = f.Jq[0] != nullptr;   // the deterministic (int64) form
  if (!fix && !f.Bn[0]) return cudaErrorInvalidValue;   // the box path reads B^n
  auto kern = fix ? k_tile<true> : k_tile<false>;
  const int smem = fix ? Smem<true>::bytes : Smem<false>::bytes;
  static std::atomic<unsigned long long> configured[2];   // devices whose limit is set, per form
  {
    cudaError_t e = smem_limit_once(kern, smem, configured[fix ? 1 : 0]);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const long long tx = (g.N[0] + TX - 1) / TX, ty = (g.N[1] + TY - 1) / TY, tz = (g.N[2] + TZ - 1) / TZ;
  const long long nunits = ((tx + UXT - 1) / UXT) * ty * tz;
  long long blocks = (long long)nsm * per_sm;
  if (blocks > nunits) blocks = nunits;
  if (blocks < 1) blocks = 1;
  kern<<<(unsigned)blocks, NT, smem, s>>>(g, tb, f, L, *reinterpret_cast<const CUtensorMap*>(map), status,
                                                  pushed);
  return cudaGetLastError();
}

}  // namespace picpml
