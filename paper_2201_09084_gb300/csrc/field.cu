// Yee field update with the split-field PML (Eqs. MaxwellE, MaxwellB,
// MaxwellSum), in the normalised units of picpml_internal.cuh.
//
// One thread per node (i,j,k) updates the three components staggered from
// that node; threads are laid out along x (then y) so every array access of a
// warp is one contiguous run (coalesced).  A component location is "split"
// when it lies in the PML along either axis it is split along (decided from
// the box geometry, so the parts' loads do not wait for a table load); its
// two parts then advance by exponential differencing,
//   F <- e^{-s dt} F + (1 - e^{-s dt})/(s dt) (R dt),
// and their sum is written to the field array.  The source -alpha j goes to the
// part with the larger conductivity (first axis on ties), which for a pure
// z-PML is exactly Eq. MaxwellE; J was multiplied by alpha when deposited.
//
// Split parts are accumulated in one of two FP64-class representations:
//   SPL = 0: IEEE FP64 (with FP32 fields the increment eb (r dt + source) is
//            formed in FP32 from its FP32 inputs and added to the decayed
//            part with one FP64 FMA);
//   SPL = 1: float-float pairs (hi + lo, about 48 significant bits) updated
//            with error-free FP32 transformations.  GB300's FP64 pipe runs at
//            a small fraction of its FP32 rate, and with FP64 parts the E pass
//            was FP64-pipe bound; the pairs keep the accumulation precision at
//            FP32 instruction cost and the same 8 bytes per part.
// Conductivity comparisons and Courant numbers use float copies, so FP32
// fields need no FP64 instruction outside the FP64 parts.  Launch bounds ask
// for 6 blocks of 256 per SM for FP32 (one node per thread) to keep more
// loads in flight (the passes are memory-latency bound), 4 for FP64, whose
// node update needs more registers.
#include "field_node.cuh"

namespace picpml {

namespace {

// KZ: nodes per thread along z.  A thread marches KZ nodes upward in z and
// carries the z-neighbour values of the previous node in registers (fewer
// loads, fewer resident warps); chosen by the autotuner, 1 by default.
// Threads cover the (x, y) node plane as one flat range (x fastest), so no
// thread idles in a partial row block; blockIdx.y walks z in steps of KZ (in
// 2D the flat range is the (x, z/KZ) plane).
template <int DIM>
__device__ __forceinline__ bool node_of_thread(const Geom& g, int KZ, int& i, int& j, int& k0) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (DIM == 3) {
    if (t >= g.nn[0] * g.nn[1]) return false;
    i = t % g.nn[0];
    j = t / g.nn[0];
    k0 = blockIdx.y * KZ;
  } else {  // 2D: the (x, z/KZ) plane is the flat range
    const int nk = (g.nn[2] + KZ - 1) / KZ;
    if (t >= g.nn[0] * nk) return false;
    i = t % g.nn[0];
    j = 0;
    k0 = (t / g.nn[0]) * KZ;
  }
  return k0 < g.nn[2];
}

template <typename T, int DIM, int SPL, int KZ>
__global__ void __launch_bounds__(256, KZ == 1 && sizeof(T) == 4 ? 6 : 4) k_field_E(Geom g, Tables tb, FieldPtrs<T> f) {
  int i, j, k0;
  if (!node_of_thread<DIM>(g, KZ, i, j, k0)) return;
  long long id = g.idx(i, j, k0);
  T by_m = k0 >= 1 ? f.Bh[1][id - g.sz] : T(0);
  T bx_m = k0 >= 1 ? f.Bh[0][id - g.sz] : T(0);
#pragma unroll
  for (int kk = 0; kk < KZ; ++kk, id += g.sz) {
    const int k = k0 + kk;
    if (k >= g.nn[2]) break;
    const T by0 = f.Bh[1][id], bx0 = f.Bh[0][id], bz0 = f.Bh[2][id];
    fn::e_update<T, DIM, SPL, true>(g, tb, f, i, j, k, id, by_m, bx_m, by0, bx0, bz0);
    by_m = by0;
    bx_m = bx0;
  }
}

template <typename T, int DIM, int SPL, int KZ>
__global__ void __launch_bounds__(256, KZ == 1 && sizeof(T) == 4 ? 6 : 4) k_field_B(Geom g, Tables tb, FieldPtrs<T> f) {
  int i, j, k0;
  if (!node_of_thread<DIM>(g, KZ, i, j, k0)) return;
  long long id = g.idx(i, j, k0);
  T ex0 = f.E[0][id], ey0 = f.E[1][id];
#pragma unroll
  for (int kk = 0; kk < KZ; ++kk, id += g.sz) {
    const int k = k0 + kk;
    if (k >= g.nn[2]) break;
    const bool kc = k <= g.N[2] - 1;
    const T ex_p = kc ? f.E[0][id + g.sz] : T(0);
    const T ey_p = kc ? f.E[1][id + g.sz] : T(0);
    fn::b_update<T, DIM, SPL, true>(g, tb, f, i, j, k, id, ex_p, ey_p, ex0, ey0, f.E[2][id]);
    ex0 = ex_p;
    ey0 = ey_p;
  }
}

// The B pass of the Cole-Karkkainen solver (one node per thread; each B
// component reads a 3 x 3 transverse neighbourhood of two E components).
template <typename T, int DIM, int SPL>
__global__ void __launch_bounds__(256) k_field_B_ck(Geom g, Tables tb, FieldPtrs<T> f) {
  int i, j, k0;
  if (!node_of_thread<DIM>(g, 1, i, j, k0)) return;
  fn::b_update_ck<T, DIM, SPL>(g, tb, f, i, j, k0, g.idx(i, j, k0));
}

// Zeroed-field (perfect conductor) cells: after the E pass every E
// component on the 12 edges of a marked cell (8 in 2D) is set to zero, with
// both split parts of the location (the parts arrays exist everywhere; where
// a location is not split its parts are unused, and zero).  One thread per
// marked cell; neighbouring cells share edges and write the same zero.
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_conductor(Geom g, FieldPtrs<T> f, const int* cells, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int lin = cells[t];
  const int N0 = g.N[0], N1 = DIM == 3 ? g.N[1] : 1;
  const int i = lin % N0, j = (lin / N0) % N1, k = lin / (N0 * N1);
  auto zero = [&](int c, int a, int b, int d) {
    const long long id = g.idx(a, b, d);
    f.E[c][id] = T(0);
    f.Es[c][0][id] = 0.0;
    f.Es[c][1][id] = 0.0;
  };
  const int jt = DIM == 3 ? 1 : 0;
  for (int b = 0; b <= jt; ++b)
    for (int c = 0; c <= 1; ++c) zero(0, i, j + b, k + c);   // Ex(i+1/2, ., .)
  for (int a = 0; a <= 1; ++a)
    for (int c = 0; c <= 1; ++c) zero(1, i + a, j, k + c);   // Ey(., j+1/2, .)
  for (int a = 0; a <= 1; ++a)
    for (int b = 0; b <= jt; ++b) zero(2, i + a, j + b, k);  // Ez(., ., k+1/2)
}

inline dim3 field_grid(const Geom& g, int KZ) {
  const long long nk = (g.nn[2] + KZ - 1) / KZ;
  if (g.dim == 3) return dim3((unsigned)(((long long)g.nn[0] * g.nn[1] + 255) / 256), (unsigned)nk, 1);
  return dim3((unsigned)(((long long)g.nn[0] * nk + 255) / 256), 1, 1);
}

template <typename T, int SPL, int KZ>
cudaError_t launch_E(const Geom& g, const Tables& tb, const FieldPtrs<T>& f, cudaStream_t s) {
  if (g.dim == 3)
    k_field_E<T, 3, SPL, KZ><<<field_grid(g, KZ), 256, 0, s>>>(g, tb, f);
  else
    k_field_E<T, 2, SPL, KZ><<<field_grid(g, KZ), 256, 0, s>>>(g, tb, f);
  return cudaGetLastError();
}

template <typename T, int SPL, int KZ>
cudaError_t launch_B(const Geom& g, const Tables& tb, const FieldPtrs<T>& f, cudaStream_t s) {
  if (g.dim == 3)
    k_field_B<T, 3, SPL, KZ><<<field_grid(g, KZ), 256, 0, s>>>(g, tb, f);
  else
    k_field_B<T, 2, SPL, KZ><<<field_grid(g, KZ), 256, 0, s>>>(g, tb, f);
  return cudaGetLastError();
}

// Binomial filter of the deposited current (App. A: applied before the field
// update; Birdsall and Langdon's (1, 2, 1)/4 stencil along each axis, values
// beyond the node arrays counting as zero).  One thread per node and
// component set, x fastest (coalesced).  k_filter_x does the x pass from J
// into the scratch arrays O; k_filter_yz does the y and z passes together
// (the outer product of the two stencils) from O back into J.
template <typename T>
__global__ void __launch_bounds__(256) k_filter_x(Geom g, FieldPtrs<T> f, T* O0, T* O1, T* O2) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long plane = (long long)g.nn[0] * g.nn[1];
  if (t >= plane * g.nn[2]) return;
  const int i = (int)(t % g.nn[0]);
  const long long r = t / g.nn[0];
  const int j = (int)(r % g.nn[1]), k = (int)(r / g.nn[1]);
  const long long id = g.idx(i, j, k);
  T* const out[3] = {O0, O1, O2};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T* J = f.J[c];
    const T lo = i > 0 ? J[id - 1] : T(0), hi = i + 1 < g.nn[0] ? J[id + 1] : T(0);
    out[c][id] = T(0.25) * lo + T(0.5) * J[id] + T(0.25) * hi;
  }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_filter_yz(Geom g, FieldPtrs<T> f, const T* I0, const T* I1, const T* I2) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long plane = (long long)g.nn[0] * g.nn[1];
  if (t >= plane * g.nn[2]) return;
  const int i = (int)(t % g.nn[0]);
  const long long r = t / g.nn[0];
  const int j = (int)(r % g.nn[1]), k = (int)(r / g.nn[1]);
  const T w[3] = {T(0.25), T(0.5), T(0.25)};
  const T* const in[3] = {I0, I1, I2};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T acc = T(0);
#pragma unroll
    for (int dk = -1; dk <= 1; ++dk) {
      if (k + dk < 0 || k + dk >= g.nn[2]) continue;
      T row = T(0);
#pragma unroll
      for (int dj = (DIM == 3 ? -1 : 0); dj <= (DIM == 3 ? 1 : 0); ++dj) {
        if (j + dj < 0 || j + dj >= g.nn[1]) continue;
        row += (DIM == 3 ? w[dj + 1] : T(1)) * in[c][g.idx(i, j + dj, k + dk)];
      }
      acc += w[dk + 1] * row;
    }
    f.J[c][g.idx(i, j, k)] = acc;
  }
}

}  // namespace

// One pass of the binomial current filter: J -> O (x), O -> J (y, z).
template <typename T>
cudaError_t launch_filter_J(const Geom& g, const FieldPtrs<T>& f, T* const O[3], cudaStream_t s) {
  const long long n = (long long)g.nn[0] * g.nn[1] * g.nn[2];
  const unsigned blocks = (unsigned)((n + 255) / 256);
  k_filter_x<T><<<blocks, 256, 0, s>>>(g, f, O[0], O[1], O[2]);
  if (g.dim == 3)
    k_filter_yz<T, 3><<<blocks, 256, 0, s>>>(g, f, O[0], O[1], O[2]);
  else
    k_filter_yz<T, 2><<<blocks, 256, 0, s>>>(g, f, O[0], O[1], O[2]);
  return cudaGetLastError();
}

template cudaError_t launch_filter_J<float>(const Geom&, const FieldPtrs<float>&, float* const[3], cudaStream_t);
template cudaError_t launch_filter_J<double>(const Geom&, const FieldPtrs<double>&, double* const[3], cudaStream_t);

// split_ff: 1 = float-float split parts (FP32 fields only), 0 = FP64 parts;
// kz: nodes per thread along z (1, 2 or 4).
template <typename T>
cudaError_t launch_field_E(const Geom& g, const Tables& tb, const FieldPtrs<T>& f, int split_ff, int kz,
                           cudaStream_t s) {
  if (sizeof(T) == 4 && split_ff) {
    if (kz == 4) return launch_E<T, 1, 4>(g, tb, f, s);
    if (kz == 2) return launch_E<T, 1, 2>(g, tb, f, s);
    return launch_E<T, 1, 1>(g, tb, f, s);
  }
  if (kz == 4) return launch_E<T, 0, 4>(g, tb, f, s);
  if (kz == 2) return launch_E<T, 0, 2>(g, tb, f, s);
  return launch_E<T, 0, 1>(g, tb, f, s);
}

template <typename T>
cudaError_t launch_field_B(const Geom& g, const Tables& tb, const FieldPtrs<T>& f, int split_ff, int kz,
                           cudaStream_t s) {
  if (sizeof(T) == 4 && split_ff) {
    if (kz == 4) return launch_B<T, 1, 4>(g, tb, f, s);
    if (kz == 2) return launch_B<T, 1, 2>(g, tb, f, s);
    return launch_B<T, 1, 1>(g, tb, f, s);
  }
  if (kz == 4) return launch_B<T, 0, 4>(g, tb, f, s);
  if (kz == 2) return launch_B<T, 0, 2>(g, tb, f, s);
  return launch_B<T, 0, 1>(g, tb, f, s);
}

// Zeroes the edges of the n marked cells (device list of linear cell
// indices i + N0 (j + N1 k), N1 = 1 in 2D).
template <typename T>
cudaError_t launch_conductor(const Geom& g, const FieldPtrs<T>& f, const int* cells, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (g.dim == 3) k_conductor<T, 3><<<blocks, 256, 0, s>>>(g, f, cells, n);
  else k_conductor<T, 2><<<blocks, 256, 0, s>>>(g, f, cells, n);
  return cudaGetLastError();
}

template cudaError_t launch_conductor<float>(const Geom&, const FieldPtrs<float>&, const int*, long long,
                                             cudaStream_t);
template cudaError_t launch_conductor<double>(const Geom&, const FieldPtrs<double>&, const int*, long long,
                                              cudaStream_t);

// The CK B pass (Faraday's law with the transversely averaged differences).
template <typename T>
cudaError_t launch_field_B_ck(const Geom& g, const Tables& tb, const FieldPtrs<T>& f, int split_ff, cudaStream_t s) {
  const dim3 grd = field_grid(g, 1);
  if (sizeof(T) == 4 && split_ff) {
    if (g.dim == 3) k_field_B_ck<T, 3, 1><<<grd, 256, 0, s>>>(g, tb, f);
    else k_field_B_ck<T, 2, 1><<<grd, 256, 0, s>>>(g, tb, f);
  } else {
    if (g.dim == 3) k_field_B_ck<T, 3, 0><<<grd, 256, 0, s>>>(g, tb, f);
    else k_field_B_ck<T, 2, 0><<<grd, 256, 0, s>>>(g, tb, f);
  }
  return cudaGetLastError();
}

template cudaError_t launch_field_B_ck<float>(const Geom&, const Tables&, const FieldPtrs<float>&, int, cudaStream_t);
template cudaError_t launch_field_B_ck<double>(const Geom&, const Tables&, const FieldPtrs<double>&, int,
                                               cudaStream_t);
template cudaError_t launch_field_E<float>(const Geom&, const Tables&, const FieldPtrs<float>&, int, int,
                                           cudaStream_t);
template cudaError_t launch_field_E<double>(const Geom&, const Tables&, const FieldPtrs<double>&, int, int,
                                            cudaStream_t);
template cudaError_t launch_field_B<float>(const Geom&, const Tables&, const FieldPtrs<float>&, int, int,
                                           cudaStream_t);
template cudaError_t launch_field_B<double>(const Geom&, const Tables&, const FieldPtrs<double>&, int, int,
                                            cudaStream_t);

}  // namespace picpml
