// Pieces shared by the chunked particle kernels (order 1 and order 3): a
// block stages a chunk of consecutive particles in shared memory, finds the
// bounding box of their cells, pushes them against a shared-memory field box
// and deposits through a shared-memory current box.
#pragma once

#include "particle_common.cuh"

namespace picpml {
namespace chunk {

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

// Move of one particle with its new u; returns false when the particle leaves
// its allowed cells.  c1, o1: new cell and offsets.
template <int DIM, typename T>
__device__ __forceinline__ bool move_particle(const Geom& g, const T o[3], const int c[3], const T u[3], int c1[3],
                                              T o1[3], T& inv_gamma) {
  const Mover<T> mv(u);
  inv_gamma = mv.inv_gamma();
  bool out = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    c1[a] = c[a];
    o1[a] = o[a];
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
      if (x >= T(1)) {  // x was a tiny negative number: stay on the node
        x = T(0);
        c1[a] += 1;
      }
    }
    o1[a] = x;
    if (c1[a] < g.rmin[a] || c1[a] > g.rmax[a] || (c1[a] == g.rmax[a] && x > T(0))) out = true;
  }
  return !out;
}

// Hints L2 to fetch the records of particles [base, base + count) (the
// block's next chunk) while the current one is being worked on.
template <typename T>
__device__ __forceinline__ void prefetch_records(const SpeciesPtrs<T>& sp, long long base, long long count) {
  if (count <= 0) return;
  const unsigned bytes = (unsigned)(count * (long long)sizeof(T) * 4);   // multiple of 16
  const char* p0 = reinterpret_cast<const char*>(sp.pos) + base * (long long)sizeof(T) * 4;
  const char* p1 = reinterpret_cast<const char*>(sp.mom) + base * (long long)sizeof(T) * 4;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p0), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p1), "r"(bytes) : "memory");
}

// Stages particles [base, base + NT*P) with coalesced loads into the stage
// (words 0-2 offsets, 3 weight, 4-6 u, 7 cell; row length ROW, particle q at
// slot (q / P) * (P + 1) + q % P), removes and reports particles outside
// their allowed cells or with a non-finite momentum or weight, and leaves the bounding box of the live particles'
// cells in s_lo / s_hi (s_hi[0] < 0: no live particle).  The records of the
// block's next chunk (from next_base) are prefetched into L2.  The caller
// must not read s_lo / s_hi of the previous chunk after its last barrier
// before this call.  Ends with a barrier.
template <typename T, int DIM, int P, int NT>
__device__ __forceinline__ void stage_chunk(const Geom& g, const SpeciesPtrs<T>& sp, long long base, long long n,
                                            long long next_base, T* stg, int ROW, unsigned* status, int* s_lo,
                                            int* s_hi) {
  constexpr int PP = P + 1, C = NT * P;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      s_lo[a] = 1 << 30;
      s_hi[a] = -1;
    }
    const long long left = n - next_base;
    prefetch_records<T>(sp, next_base, left < C ? left : C);
  }
  for (int q = tid; q < C; q += NT) {
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
  int mn[3] = {1 << 30, 1 << 30, 1 << 30}, mx[3] = {-1, -1, -1};
  for (int i = 0; i < P; ++i) {
    const int slot = tid * PP + i;
    const int cell = bits_to_cell<T>(stg[7 * ROW + slot]);
    if (cell < 0) continue;
    const int c[3] = {cell_i(cell), cell_j(cell), cell_k(cell)};
    // (a non-finite momentum or weight would poison the current: refused too)
    bool bad = !finite_value(stg[3 * ROW + slot]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (!finite_value(stg[(4 + a) * ROW + slot])) bad = true;
      if (DIM == 2 && a == 1) continue;
      const T o = stg[a * ROW + slot];
      if (c[a] < g.rmin[a] || c[a] > g.rmax[a] || !(o >= T(0) && o < T(1))) bad = true;
    }
    if (bad) {
      atomicOr(status, ST_BAD_PARTICLE);
      stg[7 * ROW + slot] = cell_to_bits<T>(-1);  // removed
      continue;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      mn[a] = min(mn[a], c[a]);
      mx[a] = max(mx[a], c[a]);
    }
  }
  if (DIM == 2) {  // one cell layer in y
    mn[1] = 0;
    mx[1] = mx[0] < 0 ? -1 : 0;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int lo = warp_min(mn[a]), hi = warp_max(mx[a]);
    if (lane == 0 && hi >= 0) {
      atomicMin(s_lo + a, lo);
      atomicMax(s_hi + a, hi);
    }
  }
  __syncthreads();
}

// Counting sort of a chunk's particles by anchor key, and the cut of each
// anchor's particles into runs.  keys[k] is the key of particle
// q = tid + k NT (stage slot (q / P) (P + 1) + q % P), nk for a particle that
// deposits nothing.  cnt holds nk + 1 counters that the caller zeroed before
// a barrier, together with *s_nanchor and *s_nrun.  Leaves perm (the slots in
// key order) and runs[0 .. *s_nrun): descriptors start | length << 11 of
// runs of consecutive sorted particles that share one key.  The runs are at
// most L long: P, or more when the chunk holds few keys, so that there is
// still about one run per thread.  Each key's runs are contiguous in runs[].
// Ends with a barrier.
template <int P, int NT>
__device__ __forceinline__ void sort_runs(const int (&keys)[P], int nk, int* cnt, unsigned short* perm,
                                          unsigned short* runs, int* s_scan, int* s_nanchor, int* s_nrun) {
  constexpr int PP = P + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // count pass: each particle's rank among the chunk's particles of its key
  // (warp-aggregated counter increments)
  int ranks[P];
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const unsigned m = __match_any_sync(0xffffffffu, keys[k]);
    const int leader = __ffs(m) - 1;
    int b = 0;
    if (lane == leader) b = atomicAdd(cnt + keys[k], __popc(m));
    ranks[k] = __shfl_sync(0xffffffffu, b, leader) + __popc(m & ((1u << lane) - 1u));
  }
  __syncthreads();
  const int per = (nk + 1 + NT - 1) / NT;   // counters scanned per thread
  const int b0 = tid * per;
  {  // exclusive scan of cnt[0..nk]; number of keys present
    int loc = 0, nz = 0;
    for (int t = 0; t < per; ++t)
      if (b0 + t <= nk) {
        const int c = cnt[b0 + t];
        loc += c;
        nz += b0 + t < nk && c != 0;
      }
    nz = __reduce_add_sync(0xffffffffu, nz);
    if (lane == 0 && nz) atomicAdd(s_nanchor, nz);
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
      if (b0 + t <= nk) {
        const int c0 = cnt[b0 + t];
        cnt[b0 + t] = run;
        run += c0;
      }
  }
  __syncthreads();
  // scatter pass: the scan turned the counters into each key's start
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const int q = tid + k * NT;
    perm[cnt[keys[k]] + ranks[k]] = (unsigned short)((q / P) * PP + (q % P));
  }
  const int nlive = cnt[nk], nanc = *s_nanchor;
  int L = P;
  if (2 * nanc < NT) {
    const int l = (nlive + NT - nanc - 1) / (NT - nanc);
    L = l > P ? l : P;
  }
  for (int t = 0; t < per; ++t) {
    const int b = b0 + t;
    if (b >= nk) break;
    const int st = cnt[b], cb = cnt[b + 1] - st;
    if (cb == 0) continue;
    const int r = (cb + L - 1) / L;
    const int rb = atomicAdd(s_nrun, r);
    for (int j = 0; j < r; ++j) {
      const int len = min(L, cb - j * L);
      runs[rb + j] = (unsigned short)((st + j * L) | (len << 11));
    }
  }
  __syncthreads();
}

// Adds the lanes' run accumulators of one warp to the shared current box J:
// lanes that share an anchor (key >= 0) hold consecutive runs; a group of at
// least MIN_LANES lanes sums its accumulators with one reduce-scatter
// (acc.group_flush), the lanes of smaller groups add their own (acc.flush_box)
// where few lanes meet on an address.  MIN_LANES = 1: every group takes the
// reduce-scatter (no flush_box needed).  A warp holding one anchor in every
// lane takes the same masked reduce-scatter: a mask-free copy of it made the
// code larger and the kernels slower.
template <int MIN_LANES, class ACC, typename T>
__device__ __forceinline__ void flush_warp_runs(const ACC& acc, int key, int lane, T* J) {
  const int up = __shfl_up_sync(0xffffffffu, key, 1);
  const bool head = key >= 0 && (lane == 0 || up != key);
  const unsigned heads = __ballot_sync(0xffffffffu, head);
  const unsigned live = __ballot_sync(0xffffffffu, key >= 0);

  const unsigned below = heads & ((2u << lane) - 1u);     // heads at or before this lane
  const unsigned above = (heads | ~live) & ~((2u << lane) - 1u);
  const int first = below ? 31 - __clz(below) : 0;
  const int next = above ? __ffs(above) - 1 : 32;
  const bool big = key >= 0 && next - first >= MIN_LANES;
  unsigned pend = __ballot_sync(0xffffffffu, head && big);
  while (pend) {
    const int leader = __ffs(pend) - 1;
    pend &= pend - 1;
    const int gk = __shfl_sync(0xffffffffu, key, leader);
    acc.template group_flush<false>(key == gk, lane, J, gk);
  }
  if constexpr (MIN_LANES > 1) {
    if (key >= 0 && !big) acc.flush_box(J, key);
  }
}

}  // namespace chunk
}  // namespace picpml
