// Diagnostics (not on the timed path): charge density on the nodes, the
// Gauss-law residual div E - rho/eps0 (FP64 reduction), field energy, and the
// conversion of fields between the kernels' normalised units and SI.
#include "picpml_internal.cuh"

namespace picpml {

namespace {

__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

template <int ORDER, typename T>
__device__ __forceinline__ void bsp(T f, double* w) {
  double x = (double)f;
  if (ORDER == 1) {
    w[0] = 1.0 - x; w[1] = x;
  } else {
    double g = 1.0 - x;
    w[0] = g * g * g / 6.0;
    w[1] = 2.0 / 3.0 - x * x + 0.5 * x * x * x;
    w[2] = 2.0 / 3.0 - g * g + 0.5 * g * g * g;
    w[3] = x * x * x / 6.0;
  }
}

// rho/eps0 at the nodes (V/m^2), FP64 atomics.
template <int ORDER, int DIM, typename T>
__global__ void k_rho(Geom g, const void* pos, const void* mom, const long long* n_dev, double qoe,
                      double* rho) {
  const long long n = *n_dev;
  constexpr int W = ORDER + 1;
  constexpr int lo = ORDER == 3 ? 1 : 0;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    T o[3], w;
    int cell;
    if (sizeof(T) == 4) {
      float4 a = reinterpret_cast<const float4*>(pos)[p];
      float4 b = reinterpret_cast<const float4*>(mom)[p];
      o[0] = a.x; o[1] = a.y; o[2] = a.z; w = a.w; cell = __float_as_int(b.w);
    } else {
      dbl4 a = reinterpret_cast<const dbl4*>(pos)[p];
      dbl4 b = reinterpret_cast<const dbl4*>(mom)[p];
      o[0] = (T)a.x; o[1] = (T)a.y; o[2] = (T)a.z; w = (T)a.w; cell = (int)__double_as_longlong(b.w);
    }
    if (cell < 0) continue;
    double wx[W], wy[W], wz[W];
    bsp<ORDER, T>(o[0], wx);
    bsp<ORDER, T>(o[2], wz);
    if (DIM == 3) bsp<ORDER, T>(o[1], wy);
    const int i = cell_i(cell) - lo, j = DIM == 3 ? cell_j(cell) - lo : 0, k = cell_k(cell) - lo;
    // skip a record whose stencil would leave the node arrays
    if (i < 0 || k < 0 || j < 0 || i + W - 1 > g.N[0] || k + W - 1 > g.N[2] ||
        (DIM == 3 && j + W - 1 > g.N[1]))
      continue;
    for (int tz = 0; tz < W; ++tz)
      for (int ty = 0; ty < (DIM == 3 ? W : 1); ++ty)
        for (int tx = 0; tx < W; ++tx)
          atomicAdd(rho + g.idx(i + tx, j + ty, k + tz),
                    qoe * (double)w * wx[tx] * (DIM == 3 ? wy[ty] : 1.0) * wz[tz]);
  }
}

// Gauss residual on nodes at least one cell inside the physical region, and
// the field energy over the whole grid.  out[0] = max residual, out[1] = max
// |rho/eps0| there, out[2] = energy.
template <typename T, int DIM>
__global__ void k_gauss_energy(Geom g, FieldPtrs<T> f, const double* rho, double inv_d0, double inv_d1,
                               double inv_d2, double vol, double* out) {
  const long long total = (long long)g.nn[0] * g.nn[1] * g.nn[2];
  double en = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nn[0]);
    const long long r = t / g.nn[0];
    const int j = (int)(r % g.nn[1]);
    const int k = (int)(r / g.nn[1]);
    const long long id = g.idx(i, j, k);
    double e2 = 0.0, b2 = 0.0;
    for (int c = 0; c < 3; ++c) {
      double e = (double)f.E[c][id];
      double b = 0.5 * ((double)f.Bh[c][id] + (double)f.Bp[c][id]);
      e2 += e * e;
      b2 += b * b;
    }
    en += 0.5 * kEps0 * (e2 + b2) * vol;
    bool inside = i >= g.plo[0] + 1 && i <= g.plo[0] + g.nph[0] - 1 && k >= g.plo[2] + 1 &&
                  k <= g.plo[2] + g.nph[2] - 1;
    if (DIM == 3) inside = inside && j >= g.plo[1] + 1 && j <= g.plo[1] + g.nph[1] - 1;
    if (inside) {
      double div = ((double)f.E[0][id] - (double)f.E[0][id - 1]) * inv_d0 +
                   ((double)f.E[2][id] - (double)f.E[2][id - g.sz]) * inv_d2;
      if (DIM == 3) div += ((double)f.E[1][id] - (double)f.E[1][id - g.sy]) * inv_d1;
      atomic_max_pos(out + 0, fabs(div - rho[id]));
      atomic_max_pos(out + 1, fabs(rho[id]));
    }
  }
  // block reduction of the energy
  __shared__ double red[256];
  red[threadIdx.x] = en;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out + 2, red[0]);
}

// Copies a normalised field array into a tight SI array (scale applied).
template <typename T, typename U>
__global__ void k_export(Geom g, const T* a, const T* b, double scale, U* dst) {
  const long long total = (long long)g.nn[0] * g.nn[1] * g.nn[2];
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nn[0]);
    const long long r = t / g.nn[0];
    const long long id = g.idx(i, (int)(r % g.nn[1]), (int)(r / g.nn[1]));
    double v = (double)a[id];
    if (b) v = 0.5 * (v + (double)b[id]);
    dst[t] = (U)(v * scale);
  }
}

template <typename T, typename U>
__global__ void k_import(Geom g, const U* src, double scale, T* a, double* split0, double* split1, int ff) {
  const long long total = (long long)g.nn[0] * g.nn[1] * g.nn[2];
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % g.nn[0]);
    const long long r = t / g.nn[0];
    const long long id = g.idx(i, (int)(r % g.nn[1]), (int)(r / g.nn[1]));
    const double v = (double)src[t] * scale;
    a[id] = (T)v;
    if (split0 && ff) {  // float-float parts: (hi, lo) pairs
      const float h = (float)v;
      reinterpret_cast<float2*>(split0)[id] = make_float2(h, (float)(v - (double)h));
      reinterpret_cast<float2*>(split1)[id] = make_float2(0.f, 0.f);
    } else if (split0) {
      split0[id] = v;
      split1[id] = 0.0;
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_rho(int order, const Geom& g, const void* pos, const void* mom, const long long* n_dev,
                       long long cap, double qoe, double* rho, cudaStream_t s) {
  if (cap <= 0) return cudaSuccess;
  int blocks = (int)((cap + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (order == 1) {
    if (g.dim == 3) k_rho<1, 3, T><<<blocks, 256, 0, s>>>(g, pos, mom, n_dev, qoe, rho);
    else k_rho<1, 2, T><<<blocks, 256, 0, s>>>(g, pos, mom, n_dev, qoe, rho);
  } else {
    if (g.dim == 3) k_rho<3, 3, T><<<blocks, 256, 0, s>>>(g, pos, mom, n_dev, qoe, rho);
    else k_rho<3, 2, T><<<blocks, 256, 0, s>>>(g, pos, mom, n_dev, qoe, rho);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gauss(const Geom& g, const FieldPtrs<T>& f, const double* rho, const double* d,
                         double* out, cudaStream_t s) {
  double vol = d[0] * d[2] * (g.dim == 3 ? d[1] : 1.0);
  if (g.dim == 3)
    k_gauss_energy<T, 3><<<1024, 256, 0, s>>>(g, f, rho, 1.0 / d[0], 1.0 / d[1], 1.0 / d[2], vol, out);
  else
    k_gauss_energy<T, 2><<<1024, 256, 0, s>>>(g, f, rho, 1.0 / d[0], 0.0, 1.0 / d[2], vol, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_export(const Geom& g, const T* a, const T* b, double scale, void* dst, int as_double,
                          cudaStream_t s) {
  if (as_double) k_export<T, double><<<1024, 256, 0, s>>>(g, a, b, scale, (double*)dst);
  else k_export<T, float><<<1024, 256, 0, s>>>(g, a, b, scale, (float*)dst);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_import(const Geom& g, const void* src, int as_double, double scale, T* a, double* s0,
                          double* s1, int ff, cudaStream_t s) {
  if (as_double) k_import<T, double><<<1024, 256, 0, s>>>(g, (const double*)src, scale, a, s0, s1, ff);
  else k_import<T, float><<<1024, 256, 0, s>>>(g, (const float*)src, scale, a, s0, s1, ff);
  return cudaGetLastError();
}

#define INST(T)                                                                                          \
  template cudaError_t launch_rho<T>(int, const Geom&, const void*, const void*, const long long*,     \
                                     long long, double, double*, cudaStream_t);                        \
  template cudaError_t launch_gauss<T>(const Geom&, const FieldPtrs<T>&, const double*, const double*, \
                                       double*, cudaStream_t);                                         \
  template cudaError_t launch_export<T>(const Geom&, const T*, const T*, double, void*, int,           \
                                        cudaStream_t);                                                 \
  template cudaError_t launch_import<T>(const Geom&, const void*, int, double, T*, double*, double*,   \
                                        int, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace picpml
