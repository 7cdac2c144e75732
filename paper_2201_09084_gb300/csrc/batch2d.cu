// Batched independent 2D runs: thousands of small (x,z) boxes, each with its
// own size and PML width and one exiting macroparticle (the paper's
// single-particle studies, Sec. III, swept over incidence angle and gamma),
// advanced by ONE persistent kernel launch per time step.
//
// A block takes the next run from a work queue ordered largest first (so the
// uneven run sizes balance across SMs) and does the whole step of that run:
// gather + Boris + move + Esirkepov deposit (alpha-damped) of the run's
// particle by one thread, then the E pass and the B pass over the run's grid
// with the same per-node split-field PML updates as a single box
// (field_node.cuh).  __syncthreads separates the stages; runs never interact.
// The launches of a step pair (the two B buffers swap every step) are
// captured once into a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/picpml.h"
#include "field_node.cuh"
#include "particle_common.cuh"
#include <nvtx3/nvToolsExt.h>

namespace picpml {

// Axis tables of one box, built from the closed forms of Eq. conductivity and
// Eq. alpha, and the alpha mode of a face (defined in api.cu).
void build_axis_table(const pml_desc& p, int axis, double Delta, double dt, int plo, int nph, int nn, bool active,
                      double* ea_n, double* eb_n, double* sdt_n, double* ea_c, double* eb_c, double* sdt_c,
                      double* al_n, double* al_c);
int face_alpha_mode(const pml_desc& p, int face);

namespace {

using namespace pc;

struct RunInfo {
  int N0, N2;          // total cells along x and z
  int nn0, nn2;        // nodes
  int rmin0, rmax0, rmin2, rmax2;
  int p, nx, nz;       // PML cells on each face, physical cells along x and z
  long long off;       // first element of this run in every field array
  int tx, tz;          // first entry of this run's x and z tables
};

// One table family laid out for all runs (x tables then z tables per run).
struct BatchTables {
  const double *ea_n, *eb_n, *sdt_n, *ea_c, *eb_c, *sdt_c, *al_nd, *al_cd;
  const float *sdtf_n, *sdtf_c, *al_nf, *al_cf;
  const float2 *ea2_n, *eb2_n, *ea2_c, *eb2_c;
};

template <typename T>
struct BatchArgs {
  const RunInfo* runs;
  const int* order;
  int* queue;
  int nruns;
  T* E[3];
  T* B0[3];
  T* B1[3];
  T* J[3];
  double* parts[12];   // E parts (c,h) then B parts (c,h); 8-byte words
  BatchTables tb;
  const double* dummy_d;   // one-entry y tables: sigma 0, alpha 1, ea 1, eb 1
  const float* dummy_f0;
  const float* dummy_f1;
  const float2* dummy_f2;
  void* pos;
  void* mom;
  T ke, cjx, cjz, cjy;
  double S[3];
  float Sf[3], Sfl[3];
  int wdamp;                 // weight damping (PML_ALPHA_WEIGHT): see Geom
  double wk[3], winv_delta, wexp;
  unsigned* status;
  unsigned long long* pushed;
  int prescribed;
};

template <typename T>
__device__ __forceinline__ Tables run_tables(const BatchArgs<T>& a, const RunInfo& r) {
  Tables t;
  const BatchTables& b = a.tb;
  const int off[3] = {r.tx, 0, r.tz};
  for (int ax = 0; ax < 3; ax += 2) {
    const int o = off[ax];
    t.ea_n[ax] = b.ea_n + o; t.eb_n[ax] = b.eb_n + o; t.sdt_n[ax] = b.sdt_n + o;
    t.ea_c[ax] = b.ea_c + o; t.eb_c[ax] = b.eb_c + o; t.sdt_c[ax] = b.sdt_c + o;
    t.al_nd[ax] = b.al_nd + o; t.al_cd[ax] = b.al_cd + o;
    t.sdtf_n[ax] = b.sdtf_n + o; t.sdtf_c[ax] = b.sdtf_c + o;
    t.al_nf[ax] = b.al_nf + o; t.al_cf[ax] = b.al_cf + o;
    t.ea2_n[ax] = b.ea2_n + o; t.eb2_n[ax] = b.eb2_n + o; t.ea2_c[ax] = b.ea2_c + o; t.eb2_c[ax] = b.eb2_c + o;
  }
  t.ea_n[1] = t.eb_n[1] = t.ea_c[1] = t.eb_c[1] = a.dummy_d + 1;   // 1.0
  t.sdt_n[1] = t.sdt_c[1] = a.dummy_d;                               // 0.0
  t.al_nd[1] = t.al_cd[1] = a.dummy_d + 1;
  t.sdtf_n[1] = t.sdtf_c[1] = a.dummy_f0;                            // 0.f
  t.al_nf[1] = t.al_cf[1] = a.dummy_f1;                              // 1.f
  t.ea2_n[1] = t.eb2_n[1] = t.ea2_c[1] = t.eb2_c[1] = a.dummy_f2;    // (1, 0)
  for (int ax = 0; ax < 3; ++ax) {  // no alpha-is-one ranges: tables always read
    t.al1_lo[ax] = 1;
    t.al1_hi[ax] = 0;
  }
  return t;
}

template <typename T, int ORDER, int SPL, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_batch_step(BatchArgs<T> a, int parity) {
  __shared__ int s_run;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_run = atomicAdd(a.queue, 1);
    __syncthreads();
    const int rq = s_run;
    if (rq >= a.nruns) break;
    const int run = a.order[rq];
    const RunInfo ri = a.runs[run];
    Geom g;
    g.dim = 2;
    g.N[0] = ri.N0; g.N[1] = 0; g.N[2] = ri.N2;
    g.nn[0] = ri.nn0; g.nn[1] = 1; g.nn[2] = ri.nn2;
    g.px = ri.nn0;
    g.sy = ri.nn0;
    g.sz = ri.nn0;
    g.size = (long long)ri.nn0 * ri.nn2;
    for (int ax = 0; ax < 3; ++ax) {
      g.S[ax] = a.S[ax];
      g.Sf[ax] = a.Sf[ax];
      g.Sfl[ax] = a.Sfl[ax];
    }
    g.wdamp = a.wdamp;
    for (int ax = 0; ax < 3; ++ax) g.wk[ax] = a.wk[ax];
    g.winv_delta = a.winv_delta;
    g.wexp = a.wexp;
    g.plo[0] = ri.p; g.nph[0] = ri.nx;
    g.plo[1] = 0; g.nph[1] = 0;
    g.plo[2] = ri.p; g.nph[2] = ri.nz;
    g.rmin[0] = ri.rmin0; g.rmax[0] = ri.rmax0;
    g.rmin[1] = 0; g.rmax[1] = 1 << 30;
    g.rmin[2] = ri.rmin2; g.rmax[2] = ri.rmax2;
    const Tables tb = run_tables(a, ri);
    FieldPtrs<T> f{};
    for (int c = 0; c < 3; ++c) {
      f.E[c] = a.E[c] + ri.off;
      f.Bh[c] = (parity ? a.B1[c] : a.B0[c]) + ri.off;
      f.Bp[c] = (parity ? a.B0[c] : a.B1[c]) + ri.off;
      f.J[c] = a.J[c] + ri.off;
      for (int h = 0; h < 2; ++h) {
        f.Es[c][h] = a.parts[c * 2 + h] + ri.off;
        f.Bs[c][h] = a.parts[6 + c * 2 + h] + ri.off;
      }
    }
    // ---- the run's particle: gather, push, move, deposit (one thread) ----
    if (threadIdx.x == 0) {
      T o[3], u[3], w;
      int cell;
      PIO<T>::load(a.pos, a.mom, run, o, w, u, cell);
      if (cell >= 0) {
        int c[3] = {cell_i(cell), 0, cell_k(cell)};
        bool bad = !finite_value(w) || !finite_value(u[0]) || !finite_value(u[1]) || !finite_value(u[2]);
        for (int ax = 0; ax < 3; ax += 2)
          if (c[ax] < g.rmin[ax] || c[ax] > g.rmax[ax] || !(o[ax] >= T(0) && o[ax] < T(1))) bad = true;
        if (bad) {
          atomicOr(a.status, ST_BAD_PARTICLE);
          PIO<T>::store(a.pos, a.mom, run, o, w, u, -1);
        } else {
          if (!a.prescribed) {
            constexpr int WN = ORDER + 1;
            int b0[3], bh[3];
            T w0[3][WN], wh[3][WN];
            b0[1] = bh[1] = 0;
            for (int t = 0; t < WN; ++t) w0[1][t] = wh[1][t] = T(t == 0);
            axis_weights<ORDER, T>(c[0], o[0], b0[0], w0[0], bh[0], wh[0]);
            axis_weights<ORDER, T>(c[2], o[2], b0[2], w0[2], bh[2], wh[2]);
            T E[3], B[3];
            E[0] = interp<ORDER, 2, T>(g, f.E[0], bh[0], wh[0], 0, w0[1], b0[2], w0[2]);
            E[1] = interp<ORDER, 2, T>(g, f.E[1], b0[0], w0[0], 0, wh[1], b0[2], w0[2]);
            E[2] = interp<ORDER, 2, T>(g, f.E[2], b0[0], w0[0], 0, w0[1], bh[2], wh[2]);
            B[0] = interp_avg<ORDER, 2, T>(g, f.Bh[0], f.Bp[0], b0[0], w0[0], 0, wh[1], bh[2], wh[2]);
            B[1] = interp_avg<ORDER, 2, T>(g, f.Bh[1], f.Bp[1], bh[0], wh[0], 0, w0[1], bh[2], wh[2]);
            B[2] = interp_avg<ORDER, 2, T>(g, f.Bh[2], f.Bp[2], bh[0], wh[0], 0, wh[1], b0[2], w0[2]);
            boris<T>(u, E, B, a.ke);
          }
          atomicAdd(a.pushed, 1ull);
          const Mover<T> mv(u);
          int c1[3] = {c[0], 0, c[2]};
          T o1[3] = {o[0], T(0), o[2]};
          bool out = false;
          for (int ax = 0; ax < 3; ax += 2) {
            const T Sh = sizeof(T) == 4 ? T(g.Sf[ax]) : T(g.S[ax]);
            const T Sl = sizeof(T) == 4 ? T(g.Sfl[ax]) : T(0);
            T x = mv.advance(o[ax], Sh, Sl, u[ax]);
            if (x >= T(1)) {
              x -= T(1);
              c1[ax] += 1;
            } else if (x < T(0)) {
              x += T(1);
              c1[ax] -= 1;
              if (x >= T(1)) {
                x = T(0);
                c1[ax] += 1;
              }
            }
            o1[ax] = x;
            if (c1[ax] < g.rmin[ax] || c1[ax] > g.rmax[ax] || (c1[ax] == g.rmax[ax] && x > T(0))) out = true;
          }
          const int cc0[3] = {c[0], 0, c[2]};
          T wd = w, wn = w;
          if (g.wdamp && !out) {  // weight damping: mid-step weight for the current, then decay
            const T I = weight_exponent<T>(g, cc0, o, c1, o1);
            wd = w * exp(T(-0.5) * I);
            wn = w * exp(-I);
          }
          PIO<T>::store(a.pos, a.mom, run, out ? o : o1, wn, u, out ? -1 : pack_cell(c1[0], 0, c1[2]));
          if (!out) {
            SpeciesPtrs<T> sp{};
            sp.cj[0] = a.cjx;
            sp.cj[2] = a.cjz;
            sp.cjy2d = a.cjy;
            deposit_run_particle<ORDER, T>(g, tb, f, sp, cc0, o, c1, o1, wd, u[1] * mv.inv_gamma());
          }
        }
      }
    }
    __syncthreads();
    // ---- E pass over the run's grid ----
    const int nnode = ri.nn0 * ri.nn2;
    for (int t = threadIdx.x; t < nnode; t += blockDim.x) {
      const int i = t % ri.nn0, k = t / ri.nn0;
      const long long id = t;
      const T by_m = k >= 1 ? f.Bh[1][id - g.sz] : T(0);
      const T bx_m = k >= 1 ? f.Bh[0][id - g.sz] : T(0);
      fn::e_update<T, 2, SPL, true>(g, tb, f, i, 0, k, id, by_m, bx_m, f.Bh[1][id], f.Bh[0][id], f.Bh[2][id]);
    }
    __syncthreads();
    // ---- B pass ----
    for (int t = threadIdx.x; t < nnode; t += blockDim.x) {
      const int i = t % ri.nn0, k = t / ri.nn0;
      const long long id = t;
      const bool kc = k <= g.N[2] - 1;
      const T ex_p = kc ? f.E[0][id + g.sz] : T(0);
      const T ey_p = kc ? f.E[1][id + g.sz] : T(0);
      fn::b_update<T, 2, SPL, true>(g, tb, f, i, 0, k, id, ex_p, ey_p, f.E[0][id], f.E[1][id], f.E[2][id]);
    }
  }
}

}  // namespace
}  // namespace picpml

// ============================================================================
// host side
// ============================================================================
namespace picpml {
template <typename T>
cudaError_t launch_export(const Geom&, const T*, const T*, double, void*, int, cudaStream_t);
double sigma_eps0_face(const pml_desc& p, double Delta, double dc);
}  // namespace picpml

using namespace picpml;

struct pic_batch {
  pic_batch_desc d{};
  pml_desc pml{};
  int prec = PIC_FP32;
  int order = 1;
  double dt = 0;
  cudaStream_t stream = nullptr;      // caller's stream
  cudaStream_t capture = nullptr;     // private stream used only to record the graph
  int nsm = 148, blocks = 0;
  int cfg = 0;                         // block shape chosen by the autotuner (index into kShapes)
  std::vector<float> tune_ms;          // measured ms per step of every candidate
  std::vector<RunInfo> runs;
  std::vector<void*> allocs;
  BatchArgs<float> af{};
  BatchArgs<double> ad{};
  cudaGraphExec_t pair = nullptr;     // two steps (both B-buffer parities)
  long long steps_done = 0;
  std::string err;
};

namespace {

int bfail(pic_batch* b, int code, const std::string& m) {
  if (b) b->err = m;
  return code;
}

#define BCK(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return bfail(b, PIC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

void* balloc(pic_batch* b, size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) return nullptr;
  b->allocs.push_back(p);
  return p;
}

template <typename T>
BatchArgs<T>& args(pic_batch* b);
template <>
BatchArgs<float>& args<float>(pic_batch* b) { return b->af; }
template <>
BatchArgs<double>& args<double>(pic_batch* b) { return b->ad; }

// Block shapes the autotuner chooses from: (threads, minimum blocks per SM).
// (256, 6) and (256, 8) cap registers (42 and 32 per thread) for more
// resident warps in the FP32 field passes; the particle stage of a run, one
// thread's work, may then spill.  (256, 3) leaves the FP64 node update its
// registers (about 85) at 24 warps per SM.
constexpr int kNumShapes = 7;
constexpr int kShapes[kNumShapes][2] = {{512, 1}, {256, 2}, {512, 2}, {1024, 1}, {256, 6}, {256, 8}, {256, 3}};

template <typename T, int ORDER, int SPL, int NT, int MINB>
cudaError_t launch_shape(pic_batch* b, BatchArgs<T>& a, int parity, cudaStream_t s) {
  static int per_sm = 0;   // resident blocks per SM of this instance (queried once)
  if (per_sm == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_step<T, ORDER, SPL, NT, MINB>, NT, 0) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
  const int blocks = std::max(1, std::min(b->nsm * per_sm, b->d.nruns));
  k_batch_step<T, ORDER, SPL, NT, MINB><<<blocks, NT, 0, s>>>(a, parity);
  return cudaGetLastError();
}

template <typename T, int ORDER, int SPL>
cudaError_t launch_cfg(pic_batch* b, BatchArgs<T>& a, int parity, cudaStream_t s) {
  switch (b->cfg) {
    case 1: return launch_shape<T, ORDER, SPL, 256, 2>(b, a, parity, s);
    case 2: return launch_shape<T, ORDER, SPL, 512, 2>(b, a, parity, s);
    case 3: return launch_shape<T, ORDER, SPL, 1024, 1>(b, a, parity, s);
    case 4: return launch_shape<T, ORDER, SPL, 256, 6>(b, a, parity, s);
    case 5: return launch_shape<T, ORDER, SPL, 256, 8>(b, a, parity, s);
    case 6: return launch_shape<T, ORDER, SPL, 256, 3>(b, a, parity, s);
    default: return launch_shape<T, ORDER, SPL, 512, 1>(b, a, parity, s);
  }
}

template <typename T>
cudaError_t launch_step(pic_batch* b, int parity, cudaStream_t s) {
  BatchArgs<T>& a = args<T>(b);
  cudaError_t e = cudaMemsetAsync(a.queue, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const bool ff = sizeof(T) == 4;
  if (b->order == 1) return ff ? launch_cfg<T, 1, 1>(b, a, parity, s) : launch_cfg<T, 1, 0>(b, a, parity, s);
  return ff ? launch_cfg<T, 3, 1>(b, a, parity, s) : launch_cfg<T, 3, 0>(b, a, parity, s);
}

cudaError_t launch_any(pic_batch* b, int parity, cudaStream_t s) {
  return b->prec == PIC_FP64 ? launch_step<double>(b, parity, s) : launch_step<float>(b, parity, s);
}

template <typename T>
int setup_args(pic_batch* b, long long total, const std::vector<double>& tabd, const std::vector<float>& tabf,
               const std::vector<float2>& tab2, size_t ntab) {
  BatchArgs<T>& a = args<T>(b);
  const size_t es = sizeof(T);
  char* fm = (char*)balloc(b, (size_t)total * (12 * es + 12 * 8));
  if (!fm) return bfail(b, PIC_ENOMEM, "batch fields");
  BCK(cudaMemsetAsync(fm, 0, (size_t)total * (12 * es + 12 * 8), b->stream));
  char* q = fm;
  for (int c = 0; c < 3; ++c) {
    a.E[c] = (T*)q; q += total * es;
    a.B0[c] = (T*)q; q += total * es;
    a.B1[c] = (T*)q; q += total * es;
    a.J[c] = (T*)q; q += total * es;
  }
  for (int t = 0; t < 12; ++t) { a.parts[t] = (double*)q; q += total * 8; }
  double* td = (double*)balloc(b, tabd.size() * 8);
  float* tf = (float*)balloc(b, tabf.size() * 4);
  float2* t2 = (float2*)balloc(b, tab2.size() * 8);
  double* dd = (double*)balloc(b, 64);
  if (!td || !tf || !t2 || !dd) return bfail(b, PIC_ENOMEM, "batch tables");
  BCK(cudaMemcpyAsync(td, tabd.data(), tabd.size() * 8, cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemcpyAsync(tf, tabf.data(), tabf.size() * 4, cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemcpyAsync(t2, tab2.data(), tab2.size() * 8, cudaMemcpyHostToDevice, b->stream));
  const double dummy_d[2] = {0.0, 1.0};
  const float dummy_f[2] = {0.f, 1.f};
  const float2 dummy_2 = make_float2(1.f, 0.f);
  BCK(cudaMemcpyAsync(dd, dummy_d, sizeof(dummy_d), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemcpyAsync((char*)dd + 16, dummy_f, sizeof(dummy_f), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemcpyAsync((char*)dd + 32, &dummy_2, sizeof(dummy_2), cudaMemcpyHostToDevice, b->stream));
  a.dummy_d = dd;
  a.dummy_f0 = (const float*)((char*)dd + 16);
  a.dummy_f1 = (const float*)((char*)dd + 20);
  a.dummy_f2 = (const float2*)((char*)dd + 32);
  BatchTables& t = a.tb;
  t.ea_n = td + 0 * ntab; t.eb_n = td + 1 * ntab; t.sdt_n = td + 2 * ntab; t.ea_c = td + 3 * ntab;
  t.eb_c = td + 4 * ntab; t.sdt_c = td + 5 * ntab; t.al_nd = td + 6 * ntab; t.al_cd = td + 7 * ntab;
  t.al_nf = tf + 0 * ntab; t.al_cf = tf + 1 * ntab; t.sdtf_n = tf + 2 * ntab; t.sdtf_c = tf + 3 * ntab;
  t.ea2_n = t2 + 0 * ntab; t.eb2_n = t2 + 1 * ntab; t.ea2_c = t2 + 2 * ntab; t.eb2_c = t2 + 3 * ntab;
  return PIC_OK;
}

template <typename T>
void set_constants(pic_batch* b, const RunInfo* runs_dev, const int* order_dev, int* queue, unsigned* status,
                   unsigned long long* pushed) {
  BatchArgs<T>& a = args<T>(b);
  const double dx = b->d.d[0], dz = b->d.d[1], q = b->d.q, m = b->d.m, dt = b->dt, Ly = 1.0;
  a.runs = runs_dev;
  a.order = order_dev;
  a.queue = queue;
  a.nruns = b->d.nruns;
  a.pos = b->d.pos;
  a.mom = b->d.mom;
  a.ke = (T)(q * dt / (2.0 * m * kC));
  a.cjx = (T)(-q / (kEps0 * dz * Ly));
  a.cjz = (T)(-q / (kEps0 * dx * Ly));
  a.cjy = (T)(q * dt * kC / (kEps0 * dx * dz * Ly));
  const double S[3] = {kC * dt / dx, 0.0, kC * dt / dz};
  for (int ax = 0; ax < 3; ++ax) {
    a.S[ax] = S[ax];
    a.Sf[ax] = (float)S[ax];
    a.Sfl[ax] = (float)(S[ax] - (double)a.Sf[ax]);
  }
  a.status = status;
  a.pushed = pushed;
  a.prescribed = 0;
  a.wdamp = b->d.pml.alpha_mode == PML_ALPHA_WEIGHT ? 1 : 0;
  for (int ax = 0; ax < 3; ++ax) a.wk[ax] = b->d.pml.sigma_max_coef * S[ax];
  a.winv_delta = 1.0 / b->d.pml.delta_cells;
  a.wexp = b->d.pml.exponent;
}

}  // namespace

extern "C" {

int pic_batch_init(pic_batch** out, const pic_batch_desc* d, void* stream) {
  if (!out || !d) return PIC_EINVAL;
  *out = nullptr;
  pic_batch* b = new pic_batch();
  *out = b;
  b->d = *d;
  b->pml = d->pml;
  b->prec = d->prec;
  b->order = d->shape_order;
  b->stream = (cudaStream_t)stream;
  if (d->nruns < 1 || !d->nx || !d->nz || !d->npml) return bfail(b, PIC_EINVAL, "nruns and per-run arrays");
  if (d->shape_order != 1 && d->shape_order != 3) return bfail(b, PIC_EINVAL, "shape_order must be 1 or 3");
  if (d->prec != PIC_FP32 && d->prec != PIC_FP64) return bfail(b, PIC_EINVAL, "prec must be PIC_FP32 or PIC_FP64");
  if (!(d->d[0] > 0 && d->d[1] > 0) || !(d->m > 0) || !d->pos || !d->mom)
    return bfail(b, PIC_EINVAL, "cell sizes, mass and particle arrays");
  if (d->pml.alpha_mode < 0 || d->pml.alpha_mode > 3 || !(d->pml.delta_cells > 0))
    return bfail(b, PIC_EINVAL, "PML profile");
  if (d->pml.face_alpha_set) {
    if (d->pml.alpha_mode == PML_ALPHA_WEIGHT) return bfail(b, PIC_EINVAL, "per-face modes with weight damping");
    for (int f = 0; f < 6; ++f)
      if (d->pml.face_alpha[f] < PML_ALPHA_ZERO || d->pml.face_alpha[f] > PML_ALPHA_DAMPED)
        return bfail(b, PIC_EINVAL, "per-face alpha modes are zero, one or damped");
  }
  const double lim = 1.0 / (kC * std::sqrt(1.0 / (d->d[0] * d->d[0]) + 1.0 / (d->d[1] * d->d[1])));
  double dt = d->dt;
  if (!(dt > 0)) {
    if (!(d->cfl > 0 && d->cfl <= 1)) return bfail(b, PIC_EINVAL, "dt <= 0 needs 0 < cfl <= 1");
    dt = d->cfl * lim;
  }
  if (dt > lim * (1 + 1e-12)) return bfail(b, PIC_ECFL, "dt above the Yee Courant limit");
  b->dt = dt;
  const int margin = d->shape_order == 1 ? 2 : 3;
  const int n = d->nruns;
  b->runs.resize(n);
  long long total = 0;
  size_t ntab = 0;
  for (int r = 0; r < n; ++r) {
    const int nx = d->nx[r], nz = d->nz[r], p = d->npml[r];
    if (nx < 1 || nz < 1 || p < 0) return bfail(b, PIC_EINVAL, "run " + std::to_string(r) + ": bad size");
    RunInfo& ri = b->runs[r];
    ri.N0 = nx + 2 * p;
    ri.N2 = nz + 2 * p;
    if (ri.N0 > 1023 || ri.N2 > 2047) return bfail(b, PIC_EINVAL, "run " + std::to_string(r) + ": too large");
    ri.nn0 = ri.N0 + 1;
    ri.nn2 = ri.N2 + 1;
    int r0 = margin, r1 = ri.N0 - margin, z0 = margin, z1 = ri.N2 - margin;
    if (face_alpha_mode(d->pml, 0) == PML_ALPHA_ZERO) r0 = std::max(r0, p);   // removed at the interface
    if (face_alpha_mode(d->pml, 1) == PML_ALPHA_ZERO) r1 = std::min(r1, p + nx);
    if (face_alpha_mode(d->pml, 4) == PML_ALPHA_ZERO) z0 = std::max(z0, p);
    if (face_alpha_mode(d->pml, 5) == PML_ALPHA_ZERO) z1 = std::min(z1, p + nz);
    if (r1 <= r0 || z1 <= z0) return bfail(b, PIC_EINVAL, "run " + std::to_string(r) + ": too small for the shape");
    ri.rmin0 = r0; ri.rmax0 = r1; ri.rmin2 = z0; ri.rmax2 = z1;
    ri.p = p; ri.nx = nx; ri.nz = nz;
    ri.off = total;
    total += ((long long)ri.nn0 * ri.nn2 + 31) / 32 * 32;
    ri.tx = (int)ntab;
    ntab += ri.nn0;
    ri.tz = (int)ntab;
    ntab += ri.nn2;
  }
  // tables: 8 double families, 4 float families, 4 float2 families, each ntab long
  std::vector<double> tabd(8 * ntab);
  std::vector<float> tabf(4 * ntab);
  std::vector<float2> tab2(4 * ntab);
  auto split2 = [](double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
  };
  for (int r = 0; r < n; ++r) {
    const RunInfo& ri = b->runs[r];
    const int p = d->npml[r];
    const int starts[2] = {ri.tx, ri.tz}, nns[2] = {ri.nn0, ri.nn2}, nph[2] = {d->nx[r], d->nz[r]};
    const double Dl[2] = {d->d[0], d->d[1]};
    for (int ax = 0; ax < 2; ++ax) {
      const int o = starts[ax], nn = nns[ax];
      std::vector<double> t8(8 * (size_t)nn);
      double* q8 = t8.data();
      build_axis_table(d->pml, ax == 0 ? 0 : 2, Dl[ax], dt, p, nph[ax], nn, true, q8, q8 + nn, q8 + 2 * nn, q8 + 3 * nn,
                       q8 + 4 * nn, q8 + 5 * nn, q8 + 6 * nn, q8 + 7 * nn);
      for (int i = 0; i < nn; ++i) {
        for (int f = 0; f < 8; ++f) tabd[f * ntab + o + i] = q8[f * nn + i];
        tabf[0 * ntab + o + i] = (float)q8[6 * nn + i];   // alpha nodes
        tabf[1 * ntab + o + i] = (float)q8[7 * nn + i];   // alpha centres
        tabf[2 * ntab + o + i] = (float)q8[2 * nn + i];   // s dt nodes
        tabf[3 * ntab + o + i] = (float)q8[5 * nn + i];   // s dt centres
        tab2[0 * ntab + o + i] = split2(q8[0 * nn + i]);
        tab2[1 * ntab + o + i] = split2(q8[1 * nn + i]);
        tab2[2 * ntab + o + i] = split2(q8[3 * nn + i]);
        tab2[3 * ntab + o + i] = split2(q8[4 * nn + i]);
      }
    }
  }
  // work queue order: largest run first
  std::vector<int> order(n);
  for (int r = 0; r < n; ++r) order[r] = r;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return (long long)b->runs[x].nn0 * b->runs[x].nn2 > (long long)b->runs[y].nn0 * b->runs[y].nn2;
  });
  RunInfo* runs_dev = (RunInfo*)balloc(b, n * sizeof(RunInfo));
  int* order_dev = (int*)balloc(b, n * sizeof(int));
  char* misc = (char*)balloc(b, 256);
  if (!runs_dev || !order_dev || !misc) return bfail(b, PIC_ENOMEM, "batch run tables");
  BCK(cudaMemcpyAsync(runs_dev, b->runs.data(), n * sizeof(RunInfo), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemcpyAsync(order_dev, order.data(), n * sizeof(int), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemsetAsync(misc, 0, 256, b->stream));
  int r = b->prec == PIC_FP64 ? setup_args<double>(b, total, tabd, tabf, tab2, ntab)
                              : setup_args<float>(b, total, tabd, tabf, tab2, ntab);
  if (r) return r;
  int* queue = (int*)misc;
  unsigned* status = (unsigned*)(misc + 64);
  unsigned long long* pushed = (unsigned long long*)(misc + 128);
  if (b->prec == PIC_FP64) set_constants<double>(b, runs_dev, order_dev, queue, status, pushed);
  else set_constants<float>(b, runs_dev, order_dev, queue, status, pushed);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  // autotune the block shape: a few steps per candidate from the initial
  // state, which is then restored (fields zeroed, particle records copied back)
  {
    const size_t pb = (size_t)n * (b->prec == PIC_FP64 ? 32 : 16);
    void* save = balloc(b, 2 * pb);
    if (!save) return bfail(b, PIC_ENOMEM, "autotune scratch");
    BCK(cudaMemcpyAsync(save, d->pos, pb, cudaMemcpyDeviceToDevice, b->stream));
    BCK(cudaMemcpyAsync((char*)save + pb, d->mom, pb, cudaMemcpyDeviceToDevice, b->stream));
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_cfg = 0;
    for (int c = 0; c < kNumShapes; ++c) {
      b->cfg = c;
      BCK(launch_any(b, 0, b->stream));   // warm-up (first launch of this shape)
      BCK(cudaEventRecord(e0, b->stream));
      for (int t = 0; t < 3; ++t) BCK(launch_any(b, (t + 1) & 1, b->stream));
      BCK(cudaEventRecord(e1, b->stream));
      BCK(cudaEventSynchronize(e1));
      float ms = 0.f;
      BCK(cudaEventElapsedTime(&ms, e0, e1));
      b->tune_ms.push_back(ms / 3);
      if (ms < best) {
        best = ms;
        best_cfg = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->cfg = best_cfg;
    // restore the initial state
    const size_t es = b->prec == PIC_FP64 ? 8 : 4;
    char* fm = b->prec == PIC_FP64 ? (char*)b->ad.E[0] : (char*)b->af.E[0];
    BCK(cudaMemsetAsync(fm, 0, (size_t)total * (12 * es + 12 * 8), b->stream));
    BCK(cudaMemcpyAsync(d->pos, save, pb, cudaMemcpyDeviceToDevice, b->stream));
    BCK(cudaMemcpyAsync(d->mom, (char*)save + pb, pb, cudaMemcpyDeviceToDevice, b->stream));
    BCK(cudaMemsetAsync(misc, 0, 256, b->stream));
  }
  // record the two-step graph on a private stream (no work runs during capture)
  BCK(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  BCK(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
  cudaError_t e0 = launch_any(b, 0, b->capture);
  cudaError_t e1 = launch_any(b, 1, b->capture);
  cudaError_t ec = cudaStreamEndCapture(b->capture, &graph);
  if (e0 != cudaSuccess || e1 != cudaSuccess || ec != cudaSuccess)
    return bfail(b, PIC_ECUDA, "graph capture failed");
  BCK(cudaGraphInstantiate(&b->pair, graph, 0));
  cudaGraphDestroy(graph);
  BCK(cudaStreamSynchronize(b->stream));
  return PIC_OK;
}

static int batch_step_impl(pic_batch* b, int n);

int pic_batch_step(pic_batch* b, int n) {
  nvtxRangePushA("picpml pic_batch_step");
  const int r_ = batch_step_impl(b, n);
  nvtxRangePop();
  return r_;
}

static int batch_step_impl(pic_batch* b, int n) {
  if (!b || !b->pair) return bfail(b, PIC_ESTATE, "batch not initialised");
  if (n < 0) return bfail(b, PIC_EINVAL, "negative step count");
  while (n > 0) {
    const int parity = (int)(b->steps_done & 1);
    if (parity == 0 && n >= 2) {
      BCK(cudaGraphLaunch(b->pair, b->stream));
      b->steps_done += 2;
      n -= 2;
    } else {
      BCK(launch_any(b, parity, b->stream));
      b->steps_done += 1;
      n -= 1;
    }
  }
  return PIC_OK;
}

int pic_batch_get_field(pic_batch* b, int run, int which, void* dst, int as_double) {
  if (!b || !b->pair) return bfail(b, PIC_ESTATE, "batch not initialised");
  if (run < 0 || run >= b->d.nruns || which < 0 || which > 8 || !dst) return bfail(b, PIC_EINVAL, "bad arguments");
  const RunInfo& ri = b->runs[run];
  Geom g{};
  g.dim = 2;
  g.N[0] = ri.N0; g.N[2] = ri.N2;
  g.nn[0] = ri.nn0; g.nn[1] = 1; g.nn[2] = ri.nn2;
  g.px = ri.nn0; g.sy = ri.nn0; g.sz = ri.nn0;
  g.size = (long long)ri.nn0 * ri.nn2;
  const int c = which % 3, kind = which / 3;
  const double scale = kind == 0 ? 1.0 : kind == 2 ? kEps0 / b->dt : 1.0 / kC;
  const int parity = (int)(b->steps_done & 1);   // B^{n+1/2} is in B0 after an even number of steps
  if (b->prec == PIC_FP64) {
    BatchArgs<double>& a = b->ad;
    const double* bh = (parity ? a.B1[c] : a.B0[c]) + ri.off;
    const double* bp = (parity ? a.B0[c] : a.B1[c]) + ri.off;
    const double* src = kind == 0 ? a.E[c] + ri.off : kind == 2 ? a.J[c] + ri.off : bh;
    BCK(launch_export<double>(g, src, kind == 1 ? bp : nullptr, scale, dst, as_double, b->stream));
  } else {
    BatchArgs<float>& a = b->af;
    const float* bh = (parity ? a.B1[c] : a.B0[c]) + ri.off;
    const float* bp = (parity ? a.B0[c] : a.B1[c]) + ri.off;
    const float* src = kind == 0 ? a.E[c] + ri.off : kind == 2 ? a.J[c] + ri.off : bh;
    BCK(launch_export<float>(g, src, kind == 1 ? bp : nullptr, scale, dst, as_double, b->stream));
  }
  return PIC_OK;
}

int pic_batch_set_prescribed(pic_batch* b, int flag) {
  if (!b || !b->pair) return bfail(b, PIC_ESTATE, "batch not initialised");
  b->af.prescribed = b->ad.prescribed = flag ? 1 : 0;
  // the recorded graph holds the kernel arguments: record it again
  cudaGraphExecDestroy(b->pair);
  b->pair = nullptr;
  cudaGraph_t graph = nullptr;
  BCK(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
  cudaError_t e0 = launch_any(b, 0, b->capture);
  cudaError_t e1 = launch_any(b, 1, b->capture);
  cudaError_t ec = cudaStreamEndCapture(b->capture, &graph);
  if (e0 != cudaSuccess || e1 != cudaSuccess || ec != cudaSuccess) return bfail(b, PIC_ECUDA, "graph capture failed");
  BCK(cudaGraphInstantiate(&b->pair, graph, 0));
  cudaGraphDestroy(graph);
  return PIC_OK;
}

int pic_batch_particle_steps(pic_batch* b, long long* n) {
  if (!b || !b->pair || !n) return bfail(b, PIC_EINVAL, "bad arguments");
  unsigned long long v = 0;
  unsigned long long* p = b->prec == PIC_FP64 ? b->ad.pushed : b->af.pushed;
  BCK(cudaMemcpyAsync(&v, p, sizeof(v), cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  *n = (long long)v;
  return PIC_OK;
}

int pic_batch_sync(pic_batch* b) {
  if (!b || !b->pair) return bfail(b, PIC_ESTATE, "batch not initialised");
  BCK(cudaStreamSynchronize(b->stream));
  unsigned st = 0;
  BCK(cudaMemcpy(&st, b->prec == PIC_FP64 ? b->ad.status : b->af.status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st & ST_BAD_PARTICLE) return bfail(b, PIC_EPARTICLE, "a particle was outside its allowed cells (removed)");
  return PIC_OK;
}

int pic_batch_tuning(pic_batch* b, int* threads, int* min_blocks, float* ms_per_step, int ncand) {
  if (!b || !b->pair) return bfail(b, PIC_ESTATE, "batch not initialised");
  if (threads) *threads = kShapes[b->cfg][0];
  if (min_blocks) *min_blocks = kShapes[b->cfg][1];
  for (int c = 0; c < ncand && c < (int)b->tune_ms.size(); ++c) ms_per_step[c] = b->tune_ms[c];
  return PIC_OK;
}

int pic_batch_info(pic_batch* b, double* dt, long long* cells) {
  if (!b || !b->pair) return bfail(b, PIC_ESTATE, "batch not initialised");
  if (dt) *dt = b->dt;
  if (cells) {
    long long c = 0;
    for (const RunInfo& ri : b->runs) c += (long long)ri.N0 * ri.N2;
    *cells = c;
  }
  return PIC_OK;
}

const char* pic_batch_last_error(pic_batch* b) { return b ? b->err.c_str() : "null batch"; }

void pic_batch_destroy(pic_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->pair) cudaGraphExecDestroy(b->pair);
  if (b->capture) cudaStreamDestroy(b->capture);
  for (void* p : b->allocs) cudaFree(p);
  delete b;
}

}  // extern "C"
