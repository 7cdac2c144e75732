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
#include "particle_common.cuh"

namespace picpml {

namespace {

using namespace pc;

// MODE 0: push only (saves x^n); MODE 1: deposit only (from saved x^n);
// MODE 2: fused push + deposit.  FIX: deterministic int64 deposition (FP32
// only) instead of the floating-point one.
template <int ORDER, int DIM, typename T, int MODE, bool FIX = false>
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
      T wd = w;
      if (g.wdamp) {  // weight damping: mid-step weight for the current, then decay
        const T I = weight_exponent<T>(g, c0, o0, c1, o);
        wd = w * exp(T(-0.5) * I);
        PIO<T>::store(sp.pos, sp.mom, p, o, w * exp(-I), u, cell);
      }
      if constexpr (FIX) {
        if constexpr (DIM == 3)
          deposit_fixed<ORDER>(g, f, sp.qn, c0, o0, c1, o, wd, status);
        else
          deposit_fixed2d<ORDER>(g, f, sp.qn, c0, o0, c1, o, wd, u, status);
      } else {
        const T g2 = sqrt(T(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        deposit_one<ORDER, DIM, T>(g, tb, f, sp, c0, o0, c1, o, wd, u[1] / g2);
      }
      continue;
    }
    if (cell < 0) {
      if (MODE == 0) PIO<T>::save(sp.save_pos, p, o, -1);
      continue;
    }
    int c[3] = {cell_i(cell), cell_j(cell), cell_k(cell)};
    bool bad = !finite_value(w);   // (a non-finite momentum or weight is refused too)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (!finite_value(u[a])) bad = true;
      if (DIM == 2 && a == 1) continue;
      if (c[a] < g.rmin[a] || c[a] > g.rmax[a] || !(o[a] >= T(0) && o[a] < T(1))) bad = true;
    }
    if (bad) {  // removed, as the chunk kernels do: cell -1 in the record
      atomicOr(status, ST_BAD_PARTICLE);
      if (MODE == 0) PIO<T>::save(sp.save_pos, p, o, -1);
      PIO<T>::store(sp.pos, sp.mom, p, o, w, u, -1);
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
    const Mover<T> mv(u);
    const T ig = mv.inv_gamma();
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
    // weight damping (fused step only; the stage call deposit() applies it)
    T wd = w, wn = w;
    if (MODE == 2 && g.wdamp && !out) {
      const T I = weight_exponent<T>(g, c, o, c1, o1);
      wd = w * exp(T(-0.5) * I);
      wn = w * exp(-I);
    }
    PIO<T>::store(sp.pos, sp.mom, p, out ? o : o1, wn, u, cell1);
    if constexpr (MODE == 2 && FIX) {
      if (!out) {
        if constexpr (DIM == 3)
          deposit_fixed<ORDER>(g, f, sp.qn, c, o, c1, o1, wd, status);
        else
          deposit_fixed2d<ORDER>(g, f, sp.qn, c, o, c1, o1, wd, u, status);
      }
    } else if (MODE == 2 && !out) {
      deposit_one<ORDER, DIM, T>(g, tb, f, sp, c, o, c1, o1, wd, u[1] * ig);
    }
  }
  // particles pushed this launch: warp sum, one atomic per warp
  if (MODE != 1 && pushed_total) {
    const unsigned wsum = __reduce_add_sync(0xffffffffu, pushed);
    if ((threadIdx.x & 31) == 0 && wsum) atomicAdd(pushed_total, (unsigned long long)wsum);
  }
}

template <int ORDER, int DIM, typename T, bool FIX = false>
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
    k_particles<ORDER, DIM, T, 1, FIX><<<blocks, threads, 0, s>>>(g, tb, f, sp, prescribed, status, pushed);
  else
    k_particles<ORDER, DIM, T, 2, FIX><<<blocks, threads, 0, s>>>(g, tb, f, sp, prescribed, status, pushed);
  return cudaGetLastError();
}

// Deterministic mode, after all species have deposited: the damped current
// J'_c = alpha_c K_c Jq_c with K_c the value of one unit of component c's
// integer sum (in 3D -e / (eps0 d_a d_b) / (6 2^24), a and b the axes
// transverse to c; in 2D the host's per-component 2D units, j = 0) and
// alpha_c at the component's staggered location
// (Eq. alpha, Sec. II.B), one thread per node; J' is overwritten, the integer
// sums are kept until the next deposit clears them.  |Jq| above 2^62 is
// reported as an overflow.
__global__ void __launch_bounds__(256) k_fixed_flush(Geom g, Tables tb, FieldPtrs<float> f, double K0, double K1,
                                                     double K2, unsigned* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, k = blockIdx.z;
  if (i >= g.nn[0]) return;
  const long long id = g.idx(i, j, k);
  const double anx = tb.al_nd[0][i], acx = tb.al_cd[0][i];
  const double any = tb.al_nd[1][j], acy = tb.al_cd[1][j];
  const double anz = tb.al_nd[2][k], acz = tb.al_cd[2][k];
  const double al[3] = {acx * any * anz, anx * acy * anz, anx * any * acz};
  const double K[3] = {K0, K1, K2};
  bool big = false;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const long long v = f.Jq[c][id];
    big |= v > (1LL << 62) || v < -(1LL << 62);
    f.J[c][id] = (float)(((double)v * K[c]) * al[c]);
  }
  if (big) atomicOr(status, ST_FIXED_OVERFLOW);
}

}  // namespace

template <typename T>
cudaError_t launch_particles(int mode, int order, const Geom& g, const Tables& tb, const FieldPtrs<T>& f,
                             const SpeciesPtrs<T>& sp, int prescribed, unsigned* status,
                             unsigned long long* pushed, int nsm, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (f.Jq[0]) {
      if (g.dim == 3)
        return order == 1 ? launch_mode<1, 3, T, true>(mode, g, tb, f, sp, prescribed, status, pushed, nsm, s)
                          : launch_mode<3, 3, T, true>(mode, g, tb, f, sp, prescribed, status, pushed, nsm, s);
      return order == 1 ? launch_mode<1, 2, T, true>(mode, g, tb, f, sp, prescribed, status, pushed, nsm, s)
                        : launch_mode<3, 2, T, true>(mode, g, tb, f, sp, prescribed, status, pushed, nsm, s);
    }
  }
  if (order == 1) {
    return g.dim == 3 ? launch_mode<1, 3, T>(mode, g, tb, f, sp, prescribed, status, pushed, nsm, s)
                      : launch_mode<1, 2, T>(mode, g, tb, f, sp, prescribed, status, pushed, nsm, s);
  }
  return g.dim == 3 ? launch_mode<3, 3, T>(mode, g, tb, f, sp, prescribed, status, pushed, nsm, s)
                    : launch_mode<3, 2, T>(mode, g, tb, f, sp, prescribed, status, pushed, nsm, s);
}

cudaError_t launch_fixed_flush(const Geom& g, const Tables& tb, const FieldPtrs<float>& f, const double K[3],
                               unsigned* status, cudaStream_t s) {
  if (!f.Jq[0]) return cudaErrorInvalidValue;
  dim3 blk(128, 1, 1), grd((g.nn[0] + 127) / 128, g.nn[1], g.nn[2]);
  k_fixed_flush<<<grd, blk, 0, s>>>(g, tb, f, K[0], K[1], K[2], status);
  return cudaGetLastError();
}

template cudaError_t launch_particles<float>(int, int, const Geom&, const Tables&, const FieldPtrs<float>&,
                                             const SpeciesPtrs<float>&, int, unsigned*, unsigned long long*, int,
                                             cudaStream_t);
template cudaError_t launch_particles<double>(int, int, const Geom&, const Tables&, const FieldPtrs<double>&,
                                              const SpeciesPtrs<double>&, int, unsigned*, unsigned long long*, int,
                                              cudaStream_t);

}  // namespace picpml
