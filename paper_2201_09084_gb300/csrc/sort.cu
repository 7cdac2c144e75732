// Counting sort of one species by cell, dropping removed particles.  The key
// is tile-major: 8x4x4-cell tiles in x,y,z order (4x4 in 2D), then the cell
// inside the tile.  Consecutive particles then share their cell, and any run of them
// covers a compact 3D block of cells, which keeps the shared-memory field
// and current box of the particle kernel small.
//   1. histogram of the linear cell index (atomics, one per cell present in
//      a warp: the lanes that share a cell add their count together),
//   2. exclusive scan of the histogram (block scans + recursive carry),
//   3. scatter into scratch arrays (the same warp-aggregated atomics hand
//      out the places; the order within a cell is not kept across warps),
//   4. copy back, live count := number of kept particles.
#include "picpml_internal.cuh"

namespace picpml {

namespace {

// Tile-major key.  3D: tiles of 8 x 4 x 4 cells (x, y, z) in x, y, z order,
// then the cell inside the tile, x fastest: 32 consecutive cells are one
// 8 x 4 layer of a tile.  2D: 4 x 4 tiles of the (x, z) plane.
__device__ __forceinline__ long long lin_cell(const Geom& g, int cell) {
  const int i = cell_i(cell), j = cell_j(cell), k = cell_k(cell);
  if (g.dim == 3) {
    const long long tx = (g.N[0] + 7) >> 3, ty = (g.N[1] + 3) >> 2;
    const long long tile = (i >> 3) + tx * ((j >> 2) + ty * (k >> 2));
    return tile * 128 + ((i & 7) + 8 * ((j & 3) + 4 * (k & 3)));
  }
  const long long tx = (g.N[0] + 3) >> 2;
  const long long tile = (i >> 2) + tx * (k >> 2);
  return tile * 16 + ((i & 3) + 4 * (k & 3));
}

template <int PB>
__device__ __forceinline__ int read_cell(const void* mom, long long p) {
  if (PB == 16) return __float_as_int(reinterpret_cast<const float4*>(mom)[p].w);
  return (int)__double_as_longlong(reinterpret_cast<const dbl4*>(mom)[p].w);
}

// Warp-aggregated counting: the lanes of a warp that share a key (particles
// of one cell, consecutive after an earlier sort) take one atomic together,
// issued by their lowest lane; *rank is the lane's place among them.
// key < 0: no particle.  Every lane of the warp calls it.
__device__ __forceinline__ unsigned warp_count(unsigned* cnt, long long key, unsigned* rank) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned m = __match_any_sync(0xffffffffu, key);
  const int leader = __ffs(m) - 1;
  unsigned base = 0;
  if (key >= 0 && lane == (unsigned)leader) base = atomicAdd(cnt + key, (unsigned)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  *rank = (unsigned)__popc(m & ((1u << lane) - 1u));
  return base;
}

template <int PB>
__global__ void k_hist(Geom g, const void* mom, const long long* n_dev, unsigned* cnt) {
  const long long n = *n_dev;
  // whole warps step together (blockDim is a multiple of 32)
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long pw = w0; pw < n; pw += stride) {
    const long long p = pw + (threadIdx.x & 31);
    const int c = p < n ? read_cell<PB>(mom, p) : -1;
    unsigned rank;
    warp_count(cnt, c >= 0 ? lin_cell(g, c) : -1LL, &rank);
  }
}

// Exclusive scan of 2*blockDim elements per block; block totals to sums.
__global__ void k_scan_block(unsigned* data, long long n, unsigned* sums) {
  extern __shared__ unsigned sh[];
  const int t = threadIdx.x, B = blockDim.x;
  const long long base = (long long)blockIdx.x * 2 * B;
  sh[t] = base + t < n ? data[base + t] : 0u;
  sh[t + B] = base + t + B < n ? data[base + t + B] : 0u;
  // up-sweep
  int off = 1;
  for (int d = B; d > 0; d >>= 1) {
    __syncthreads();
    if (t < d) {
      int ai = off * (2 * t + 1) - 1, bi = off * (2 * t + 2) - 1;
      sh[bi] += sh[ai];
    }
    off <<= 1;
  }
  if (t == 0) {
    if (sums) sums[blockIdx.x] = sh[2 * B - 1];
    sh[2 * B - 1] = 0;
  }
  // down-sweep
  for (int d = 1; d < 2 * B; d <<= 1) {
    off >>= 1;
    __syncthreads();
    if (t < d) {
      int ai = off * (2 * t + 1) - 1, bi = off * (2 * t + 2) - 1;
      unsigned v = sh[ai];
      sh[ai] = sh[bi];
      sh[bi] += v;
    }
  }
  __syncthreads();
  if (base + t < n) data[base + t] = sh[t];
  if (base + t + B < n) data[base + t + B] = sh[t + B];
}

__global__ void k_add_carry(unsigned* data, long long n, const unsigned* sums) {
  const long long base = (long long)blockIdx.x * 2 * blockDim.x;
  const unsigned c = sums[blockIdx.x];
  for (int q = 0; q < 2; ++q) {
    long long t = base + threadIdx.x + q * blockDim.x;
    if (t < n) data[t] += c;
  }
}

template <int PB>
__global__ void k_scatter(Geom g, const void* pos, const void* mom, const long long* n_dev, unsigned* cursor,
                          void* pos_out, void* mom_out) {
  const long long n = *n_dev;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long pw = w0; pw < n; pw += stride) {
    const long long p = pw + (threadIdx.x & 31);
    const int c = p < n ? read_cell<PB>(mom, p) : -1;
    unsigned rank;
    const unsigned d0 = warp_count(cursor, c >= 0 ? lin_cell(g, c) : -1LL, &rank);
    if (c < 0) continue;
    const unsigned d = d0 + rank;
    if (PB == 16) {
      reinterpret_cast<float4*>(pos_out)[d] = reinterpret_cast<const float4*>(pos)[p];
      reinterpret_cast<float4*>(mom_out)[d] = reinterpret_cast<const float4*>(mom)[p];
    } else {
      reinterpret_cast<dbl4*>(pos_out)[d] = reinterpret_cast<const dbl4*>(pos)[p];
      reinterpret_cast<dbl4*>(mom_out)[d] = reinterpret_cast<const dbl4*>(mom)[p];
    }
  }
}

// Appends `count` records after the n live ones (n read from the device
// before k_inject_count advances it); records past the capacity are dropped
// and flagged.
template <int PB>
__global__ void k_inject(void* pos, void* mom, const long long* n_dev, long long cap, const void* ipos,
                         const void* imom, long long count, unsigned* status) {
  const long long n = *n_dev;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const long long d = n + i;
    if (d >= cap) {
      atomicOr(status, ST_INJECT_OVERFLOW);
      continue;
    }
    if (PB == 16) {
      reinterpret_cast<float4*>(pos)[d] = reinterpret_cast<const float4*>(ipos)[i];
      reinterpret_cast<float4*>(mom)[d] = reinterpret_cast<const float4*>(imom)[i];
    } else {
      reinterpret_cast<dbl4*>(pos)[d] = reinterpret_cast<const dbl4*>(ipos)[i];
      reinterpret_cast<dbl4*>(mom)[d] = reinterpret_cast<const dbl4*>(imom)[i];
    }
  }
}

__global__ void k_inject_count(long long* n_dev, long long cap, long long count) {
  const long long n = *n_dev + count;
  *n_dev = n < cap ? n : cap;
}

// After the scatter every cursor holds the end offset of its cell, so the
// last one is the number of kept particles.
__global__ void k_set_count(const unsigned* cursor, long long ncell, long long* n_dev) {
  *n_dev = (long long)cursor[ncell - 1];
}

constexpr int kScanT = 512;

cudaError_t scan(unsigned* data, long long n, unsigned* tmp, cudaStream_t s) {
  const long long per = 2LL * kScanT;
  const long long nb = (n + per - 1) / per;
  unsigned* sums = tmp;
  k_scan_block<<<(unsigned)nb, kScanT, 2 * kScanT * sizeof(unsigned), s>>>(data, n, nb > 1 ? sums : nullptr);
  if (nb > 1) {
    cudaError_t e = scan(sums, nb, tmp + nb, s);
    if (e != cudaSuccess) return e;
    k_add_carry<<<(unsigned)nb, kScanT, 0, s>>>(data, n, sums);
  }
  return cudaGetLastError();
}

}  // namespace

// Kernels one sort launches: histogram, the scan levels with their carry
// passes, scatter, count.
int sort_launches(long long ncell) {
  int k = 3;
  long long n = ncell;
  for (;;) {
    const long long nb = (n + 2LL * kScanT - 1) / (2LL * kScanT);
    k += 1;
    if (nb <= 1) break;
    k += 1;
    n = nb;
  }
  return k;
}

// Scratch needed: hist (ncell+1) + scan carries (< ncell/512) unsigned.
long long sort_scratch_words(long long ncell) { return ncell + 1 + ncell / 512 + 64; }

// Number of sort keys (cells padded to whole tiles).
long long sort_keys(const Geom& g) {
  if (g.dim == 3) {
    const long long tx = (g.N[0] + 7) >> 3, ty = (g.N[1] + 3) >> 2, tz = (g.N[2] + 3) >> 2;
    return tx * ty * tz * 128;
  }
  const long long tx = (g.N[0] + 3) >> 2, tz = (g.N[2] + 3) >> 2;
  return tx * tz * 16;
}

cudaError_t launch_sort(const Geom& g, int pbytes, void* pos, void* mom, long long* n_dev, long long cap,
                        unsigned* scratch, void* tmp_pos, void* tmp_mom, cudaStream_t s) {
  const long long ncell = sort_keys(g);
  unsigned* hist = scratch;
  unsigned* carry = scratch + ncell + 1;
  cudaError_t e = cudaMemsetAsync(hist, 0, (ncell + 1) * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  int blocks = (int)((cap + 255) / 256);
  if (blocks > 8192) blocks = 8192;
  if (blocks < 1) blocks = 1;
  if (pbytes == 16) k_hist<16><<<blocks, 256, 0, s>>>(g, mom, n_dev, hist);
  else k_hist<32><<<blocks, 256, 0, s>>>(g, mom, n_dev, hist);
  e = scan(hist, ncell, carry, s);
  if (e != cudaSuccess) return e;
  if (pbytes == 16) k_scatter<16><<<blocks, 256, 0, s>>>(g, pos, mom, n_dev, hist, tmp_pos, tmp_mom);
  else k_scatter<32><<<blocks, 256, 0, s>>>(g, pos, mom, n_dev, hist, tmp_pos, tmp_mom);
  k_set_count<<<1, 1, 0, s>>>(hist, ncell, n_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(pos, tmp_pos, cap * pbytes, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(mom, tmp_mom, cap * pbytes, cudaMemcpyDeviceToDevice, s);
}

cudaError_t launch_inject(int pbytes, void* pos, void* mom, long long* n_dev, long long cap, const void* ipos,
                          const void* imom, long long count, unsigned* status, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  long long blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (pbytes == 16) k_inject<16><<<(unsigned)blocks, 256, 0, s>>>(pos, mom, n_dev, cap, ipos, imom, count, status);
  else k_inject<32><<<(unsigned)blocks, 256, 0, s>>>(pos, mom, n_dev, cap, ipos, imom, count, status);
  k_inject_count<<<1, 1, 0, s>>>(n_dev, cap, count);
  return cudaGetLastError();
}

}  // namespace picpml
