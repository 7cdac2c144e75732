// Yee field update with the split-field PML (Eqs. MaxwellE, MaxwellB,
// MaxwellSum), in the normalised units of picpml_internal.cuh.
//
// One thread per node (i,j,k) updates the three components staggered from
// that node; threads are laid out along x so every array access of a warp is
// one contiguous run (coalesced).  A component location is "split" when the
// conductivity of either axis it is split along is nonzero there; its two
// FP64 parts then advance by exponential differencing and their sum is
// written to the FP32 total.  The source -alpha j goes to the part with the
// larger conductivity (first axis on ties), which for a pure z-PML is exactly
// Eq. MaxwellE.  J was already multiplied by alpha when it was deposited.
#include "picpml_internal.cuh"

namespace picpml {

namespace {

// Advances a split location; returns the new total.
__device__ __forceinline__ double adv_split(double* p0, double* p1, long long id, double r0,
                                            double r1, double src, double ea0, double eb0,
                                            double ea1, double eb1, bool into1) {
  double e0 = p0[id], e1 = p1[id];
  e0 = ea0 * e0 + eb0 * (r0 + (into1 ? 0.0 : src));
  e1 = ea1 * e1 + eb1 * (r1 + (into1 ? src : 0.0));
  p0[id] = e0;
  p1[id] = e1;
  return e0 + e1;
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_field_E(Geom g, Tables tb, FieldPtrs<T> f) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = DIM == 3 ? blockIdx.y * blockDim.y + threadIdx.y : 0;
  const int k = DIM == 3 ? blockIdx.z : blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.nn[0] || j >= g.nn[1] || k >= g.nn[2]) return;
  const long long id = g.idx(i, j, k);
  const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2];
  const T Sx = (T)g.S[0], Sy = (T)g.S[1], Sz = (T)g.S[2];
  const T* Bx = f.Bh[0];
  const T* By = f.Bh[1];
  const T* Bz = f.Bh[2];
  const bool jin = DIM == 2 || (j >= 1 && j <= N1 - 1);
  const bool kin = k >= 1 && k <= N2 - 1;
  const bool iin = i >= 1 && i <= N0 - 1;
  // J' is consumed here: read once, zeroed where it was nonzero (most of the
  // grid carries no current, so most threads write nothing back).
  const T jx = f.J[0][id], jy = f.J[1][id], jz = f.J[2][id];
  if (jx != T(0)) f.J[0][id] = T(0);
  if (jy != T(0)) f.J[1][id] = T(0);
  if (jz != T(0)) f.J[2][id] = T(0);

  // Ex(i+1/2, j, k): parts along y (sigma_y at node j) and z (sigma_z at node k)
  if (i <= N0 - 1 && jin && kin) {
    T r0 = DIM == 3 ? Sy * (Bz[id] - Bz[id - g.sy]) : T(0);
    T r1 = -Sz * (By[id] - By[id - g.sz]);
    T src = -jx;
    const double sA = DIM == 3 ? tb.sdt_n[1][j] : 0.0, sB = tb.sdt_n[2][k];
    if (sA > 0.0 || sB > 0.0) {
      const double ea0 = DIM == 3 ? tb.ea_n[1][j] : 1.0, eb0 = DIM == 3 ? tb.eb_n[1][j] : 1.0;
      f.E[0][id] = (T)adv_split(f.Es[0][0], f.Es[0][1], id, (double)r0, (double)r1, (double)src, ea0,
                                eb0, tb.ea_n[2][k], tb.eb_n[2][k], sB > sA);
    } else {
      f.E[0][id] += r0 + r1 + src;
    }
  }
  // Ey(i, j+1/2, k): parts along x (sigma_x at node i) and z
  if (iin && (DIM == 2 || j <= N1 - 1) && kin) {
    T r0 = -Sx * (Bz[id] - Bz[id - 1]);
    T r1 = Sz * (Bx[id] - Bx[id - g.sz]);
    T src = -jy;
    const double sA = tb.sdt_n[0][i], sB = tb.sdt_n[2][k];
    if (sA > 0.0 || sB > 0.0) {
      f.E[1][id] = (T)adv_split(f.Es[1][0], f.Es[1][1], id, (double)r0, (double)r1, (double)src,
                                tb.ea_n[0][i], tb.eb_n[0][i], tb.ea_n[2][k], tb.eb_n[2][k], sB > sA);
    } else {
      f.E[1][id] += r0 + r1 + src;
    }
  }
  // Ez(i, j, k+1/2): parts along x and y
  if (iin && jin && k <= N2 - 1) {
    T r0 = Sx * (By[id] - By[id - 1]);
    T r1 = DIM == 3 ? -Sy * (Bx[id] - Bx[id - g.sy]) : T(0);
    T src = -jz;
    const double sA = tb.sdt_n[0][i], sB = DIM == 3 ? tb.sdt_n[1][j] : 0.0;
    if (sA > 0.0 || sB > 0.0) {
      const double ea1 = DIM == 3 ? tb.ea_n[1][j] : 1.0, eb1 = DIM == 3 ? tb.eb_n[1][j] : 1.0;
      f.E[2][id] = (T)adv_split(f.Es[2][0], f.Es[2][1], id, (double)r0, (double)r1, (double)src,
                                tb.ea_n[0][i], tb.eb_n[0][i], ea1, eb1, sB > sA);
    } else {
      f.E[2][id] += r0 + r1 + src;
    }
  }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_field_B(Geom g, Tables tb, FieldPtrs<T> f) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = DIM == 3 ? blockIdx.y * blockDim.y + threadIdx.y : 0;
  const int k = DIM == 3 ? blockIdx.z : blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.nn[0] || j >= g.nn[1] || k >= g.nn[2]) return;
  const long long id = g.idx(i, j, k);
  const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2];
  const T Sx = (T)g.S[0], Sy = (T)g.S[1], Sz = (T)g.S[2];
  const T* Ex = f.E[0];
  const T* Ey = f.E[1];
  const T* Ez = f.E[2];
  const bool jc = DIM == 2 || j <= N1 - 1;   // j is a cell-centre index
  const bool kc = k <= N2 - 1;
  const bool ic = i <= N0 - 1;

  // Bx(i, j+1/2, k+1/2): parts along y (sigma_y at centre j) and z (centre k)
  if (jc && kc) {
    T r0 = DIM == 3 ? -Sy * (Ez[id + g.sy] - Ez[id]) : T(0);
    T r1 = Sz * (Ey[id + g.sz] - Ey[id]);
    const double sA = DIM == 3 ? tb.sdt_c[1][j] : 0.0, sB = tb.sdt_c[2][k];
    if (sA > 0.0 || sB > 0.0) {
      const double ea0 = DIM == 3 ? tb.ea_c[1][j] : 1.0, eb0 = DIM == 3 ? tb.eb_c[1][j] : 1.0;
      f.Bp[0][id] = (T)adv_split(f.Bs[0][0], f.Bs[0][1], id, (double)r0, (double)r1, 0.0, ea0, eb0,
                                 tb.ea_c[2][k], tb.eb_c[2][k], false);
    } else {
      f.Bp[0][id] = f.Bh[0][id] + (r0 + r1);
    }
  }
  // By(i+1/2, j, k+1/2): parts along x (centre i) and z (centre k)
  if (ic && kc) {
    T r0 = Sx * (Ez[id + 1] - Ez[id]);
    T r1 = -Sz * (Ex[id + g.sz] - Ex[id]);
    const double sA = tb.sdt_c[0][i], sB = tb.sdt_c[2][k];
    if (sA > 0.0 || sB > 0.0) {
      f.Bp[1][id] = (T)adv_split(f.Bs[1][0], f.Bs[1][1], id, (double)r0, (double)r1, 0.0,
                                 tb.ea_c[0][i], tb.eb_c[0][i], tb.ea_c[2][k], tb.eb_c[2][k], false);
    } else {
      f.Bp[1][id] = f.Bh[1][id] + (r0 + r1);
    }
  }
  // Bz(i+1/2, j+1/2, k): parts along x (centre i) and y (centre j)
  if (ic && jc) {
    T r0 = -Sx * (Ey[id + 1] - Ey[id]);
    T r1 = DIM == 3 ? Sy * (Ex[id + g.sy] - Ex[id]) : T(0);
    const double sA = tb.sdt_c[0][i], sB = DIM == 3 ? tb.sdt_c[1][j] : 0.0;
    if (sA > 0.0 || sB > 0.0) {
      const double ea1 = DIM == 3 ? tb.ea_c[1][j] : 1.0, eb1 = DIM == 3 ? tb.eb_c[1][j] : 1.0;
      f.Bp[2][id] = (T)adv_split(f.Bs[2][0], f.Bs[2][1], id, (double)r0, (double)r1, 0.0,
                                 tb.ea_c[0][i], tb.eb_c[0][i], ea1, eb1, false);
    } else {
      f.Bp[2][id] = f.Bh[2][id] + (r0 + r1);
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_field_E(const Geom& g, const Tables& tb, const FieldPtrs<T>& f, cudaStream_t s) {
  if (g.dim == 3) {
    dim3 blk(32, 8, 1), grd((g.nn[0] + 31) / 32, (g.nn[1] + 7) / 8, g.nn[2]);
    k_field_E<T, 3><<<grd, blk, 0, s>>>(g, tb, f);
  } else {
    dim3 blk(32, 8, 1), grd((g.nn[0] + 31) / 32, (g.nn[2] + 7) / 8, 1);
    k_field_E<T, 2><<<grd, blk, 0, s>>>(g, tb, f);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_field_B(const Geom& g, const Tables& tb, const FieldPtrs<T>& f, cudaStream_t s) {
  if (g.dim == 3) {
    dim3 blk(32, 8, 1), grd((g.nn[0] + 31) / 32, (g.nn[1] + 7) / 8, g.nn[2]);
    k_field_B<T, 3><<<grd, blk, 0, s>>>(g, tb, f);
  } else {
    dim3 blk(32, 8, 1), grd((g.nn[0] + 31) / 32, (g.nn[2] + 7) / 8, 1);
    k_field_B<T, 2><<<grd, blk, 0, s>>>(g, tb, f);
  }
  return cudaGetLastError();
}

template cudaError_t launch_field_E<float>(const Geom&, const Tables&, const FieldPtrs<float>&, cudaStream_t);
template cudaError_t launch_field_E<double>(const Geom&, const Tables&, const FieldPtrs<double>&, cudaStream_t);
template cudaError_t launch_field_B<float>(const Geom&, const Tables&, const FieldPtrs<float>&, cudaStream_t);
template cudaError_t launch_field_B<double>(const Geom&, const Tables&, const FieldPtrs<double>&, cudaStream_t);

}  // namespace picpml
