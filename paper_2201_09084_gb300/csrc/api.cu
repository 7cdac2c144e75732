// Host side of libpicpml: the C ABI of include/picpml.h.
//
// The context owns the fields (E, B at two half steps, J), the FP64 PML split
// parts, the per-axis coefficient tables and scratch; particle arrays belong
// to the caller.  Every entry point validates, enqueues kernels on the
// context's stream and returns a pic_status.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/picpml.h"
#include "picpml_internal.cuh"
#include <nvtx3/nvToolsExt.h>

namespace picpml {
template <typename T>
cudaError_t launch_field_E(const Geom&, const Tables&, const FieldPtrs<T>&, int split_ff, int kz, cudaStream_t);
template <typename T>
cudaError_t launch_field_B(const Geom&, const Tables&, const FieldPtrs<T>&, int split_ff, int kz, cudaStream_t);
template <typename T>
cudaError_t launch_field_B_ck(const Geom&, const Tables&, const FieldPtrs<T>&, int split_ff, cudaStream_t);
template <typename T>
cudaError_t launch_conductor(const Geom&, const FieldPtrs<T>&, const int* cells, long long n, cudaStream_t);
template <typename T>
cudaError_t launch_filter_J(const Geom&, const FieldPtrs<T>&, T* const O[3], cudaStream_t);
template <typename T>
cudaError_t launch_particles(int mode, int order, const Geom&, const Tables&, const FieldPtrs<T>&,
                             const SpeciesPtrs<T>&, int prescribed, unsigned* status, unsigned long long* pushed,
                             int nsm, cudaStream_t);
template <typename T>
cudaError_t launch_rho(int order, const Geom&, const void*, const void*, const long long*, long long, double,
                       double*, cudaStream_t);
template <typename T>
cudaError_t launch_gauss(const Geom&, const FieldPtrs<T>&, const double*, const double*, double*, cudaStream_t);
template <typename T>
cudaError_t launch_export(const Geom&, const T*, const T*, double, void*, int, cudaStream_t);
template <typename T>
cudaError_t launch_import(const Geom&, const void*, int, double, T*, double*, double*, int split_ff, cudaStream_t);
template <typename T>
cudaError_t launch_push_deposit_runs(int ppt, const Geom&, const Tables&, const FieldPtrs<T>&, const SpeciesPtrs<T>&,
                                     int prescribed, unsigned* status, unsigned long long* pushed, int nsm,
                                     cudaStream_t);
cudaError_t launch_fixed_flush(const Geom&, const Tables&, const FieldPtrs<float>&, const double K[3], unsigned*,
                               cudaStream_t);
template <typename T>
cudaError_t launch_push_deposit_o3(int ppt, const Geom&, const Tables&, const FieldPtrs<T>&, const SpeciesPtrs<T>&,
                                   int prescribed, unsigned* status, unsigned long long* pushed, int nsm,
                                   cudaStream_t);
long long sort_scratch_words(long long ncell);
int sort_launches(long long ncell);
long long sort_keys(const Geom& g);
cudaError_t launch_inject(int pbytes, void* pos, void* mom, long long* n_dev, long long cap, const void* ipos,
                          const void* imom, long long count, unsigned* status, cudaStream_t s);
cudaError_t static_diag_buffers(double** rho, double** out, long long* cap);
cudaError_t launch_sort(const Geom&, int pbytes, void* pos, void* mom, long long* n_dev, long long cap,
                        unsigned* scratch, void* tmp_pos, void* tmp_mom, cudaStream_t);
long long tile_count(const Geom&);
cudaError_t launch_tile_ends(const Geom&, const unsigned* cursor, long long* tile_end, cudaStream_t);
cudaError_t make_tile_tensor_map(const Geom&, const float* base, int arrays, void* map_out);
cudaError_t launch_bn_average(const Geom&, const FieldPtrs<float>&, cudaStream_t);
int tile_map_bytes();
cudaError_t launch_tile(const Geom&, const Tables&, const FieldPtrs<float>&, const TileLaunch&, const void* map,
                        unsigned* status, unsigned long long* pushed, int nsm, cudaStream_t);
}  // namespace picpml

namespace picpml {
double sigma_eps0_face(const pml_desc& p, double Delta, double dc);
double alpha_face(const pml_desc& p, int face, double dc);
int face_alpha_mode(const pml_desc& p, int face);

// Per-axis coefficient tables of one box at the nodes i and centres i+1/2
// (Sec. II.B): exponential-differencing factors, s dt and alpha, from the
// closed forms of Eq. conductivity and Eq. alpha.  axis: 0, 1, 2 (its faces
// 2 axis and 2 axis + 1 pick the alpha mode below and above the physical
// box); plo, nph: PML cells below and physical cells along the axis;
// `active` false for the absent y axis of 2D boxes (no PML, alpha = 1).
void build_axis_table(const pml_desc& p, int axis, double Delta, double dt, int plo, int nph, int nn, bool active,
                      double* ea_n, double* eb_n, double* sdt_n, double* ea_c, double* eb_c, double* sdt_c,
                      double* al_n, double* al_c) {
  for (int i = 0; i < nn; ++i) {
    for (int stag = 0; stag < 2; ++stag) {
      const double x = i + 0.5 * stag;
      double dc = 0.0;
      if (active) {
        const double lo = plo, hi = plo + nph;
        dc = x < lo ? lo - x : (x > hi ? x - hi : 0.0);
      }
      const double sdt = sigma_eps0_face(p, Delta, dc) * dt;
      const double ea = std::exp(-sdt);
      const double eb = sdt > 0 ? -std::expm1(-sdt) / sdt : 1.0;
      const double al = alpha_face(p, x < plo ? 2 * axis : 2 * axis + 1, dc);
      (stag ? ea_c : ea_n)[i] = ea;
      (stag ? eb_c : eb_n)[i] = eb;
      (stag ? sdt_c : sdt_n)[i] = sdt;
      (stag ? al_c : al_n)[i] = al;
    }
  }
}
}  // namespace picpml

using namespace picpml;

namespace {

struct Species {
  pic_species desc{};
  long long* n_dev = nullptr;
  void* save = nullptr;      // x^n saved by push() for deposit() (allocated at the first stage call)
  long long* tile_end = nullptr;   // per sort tile: end of its particles at the last sort (3D)
  bool tiled = false;              // sorted since registration: tile_end is valid
  void* tmp_pos = nullptr;   // sort scratch, allocated at the first sort
  void* tmp_mom = nullptr;
  double ke = 0, cj[3] = {0, 0, 0}, cjy2d = 0;
  double qn = 0;             // charge in elementary charges (deterministic mode)
};

thread_local std::string g_init_error;

}  // namespace

namespace {
// A named NVTX range around a host entry point (shown by a timeline profiler;
// a no-op when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

struct picpml_ctx {
  pic_grid_desc gd{};
  pml_desc pd{};
  bool ready = false;
  cudaStream_t stream = nullptr;
  int nsm = 148;
  double dt = 0;
  Geom g{};
  Tables tb{};
  FieldPtrs<float> ff{};
  FieldPtrs<double> fd{};
  std::vector<void*> allocs;
  unsigned* status = nullptr;
  unsigned long long* pushed = nullptr;  // particles pushed since pml_init
  double* diag = nullptr;
  double* rho = nullptr;
  unsigned* sort_scratch = nullptr;
  void* filter_tmp[3] = {nullptr, nullptr, nullptr};   // binomial filter scratch (x pass)
  std::vector<Species> sp;
  int prescribed = 0;
  int ppt = 0;        // particles per thread of the shared-memory chunk kernels (order 1; order 3
                      // in 3D): 4 or 8 (0 = default 4), or 1 = one thread per particle with
                      // global atomics, or PIC_TUNING_TILE = the tile-resident kernel (3D FP32
                      // order 1, sorted species)
  int* cond = nullptr;                   // zeroed-field cells (device list of linear indices)
  long long ncond = 0;
  long long cond_cap = 0;
  alignas(64) unsigned char tmap[128];   // TMA tensor map of the FP32 field arrays (3D)
  bool tmap_ok = false;
  bool bn_stale = true;   // ff.Bn does not hold (Bh + Bp)/2 of the current B arrays
  size_t field_bytes = 0;   // the field allocation (state arrays, then ff.Bn where present)
  int kz = 1;         // nodes per thread along z in the field kernels
  long long steps_done = 0;
  long long launches = 0;
  std::string err;
  int elem() const { return gd.prec == PIC_FP64 ? 8 : 4; }
  int pbytes() const { return gd.prec == PIC_FP64 ? 32 : 16; }
  int split_ff() const { return gd.prec != PIC_FP64 && !gd.split_fp64; }
  bool fixed() const { return gd.prec == PIC_FP32_FIXED64; }
};

namespace {

int fail(picpml_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  else g_init_error = msg;
  return code;
}

int cuda_fail(picpml_ctx* c, cudaError_t e, const char* where) {
  return fail(c, PIC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                   \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);       \
  } while (0)

void* dev_alloc(picpml_ctx* ctx, size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) return nullptr;
  ctx->allocs.push_back(p);
  return p;
}

// Courant limit of the field solver: Yee 1/(c sqrt(sum 1/d_a^2)); the
// Cole-Karkkainen scheme min(d_a)/c (its averaged differences keep the
// amplification of every Fourier mode within that of a 1D wave).
double courant_limit(const pic_grid_desc& g) {
  if (g.solver == PIC_SOLVER_CK) {
    double m = std::min(g.d[0], g.d[2]);
    if (g.dim == 3) m = std::min(m, g.d[1]);
    return m / kC;
  }
  double s = 1.0 / (g.d[0] * g.d[0]) + 1.0 / (g.d[2] * g.d[2]);
  if (g.dim == 3) s += 1.0 / (g.d[1] * g.d[1]);
  return 1.0 / (kC * std::sqrt(s));
}

}  // namespace

// sigma/eps0 at depth dc cells into a face (Eq. conductivity generalised)
double picpml::sigma_eps0_face(const pml_desc& p, double Delta, double dc) {
  if (dc <= 0.0) return 0.0;
  return p.sigma_max_coef * kC / Delta * std::pow(dc / p.delta_cells, p.exponent);
}

// Eq. alpha in closed form for the power-law profile: the exponent is
// int_0^d sigma/(eps0 v) dz = coef (c/v) delta (d/delta)^{p+1}/(p+1), d in cells.
int picpml::face_alpha_mode(const pml_desc& p, int face) {
  return p.face_alpha_set ? p.face_alpha[face] : p.alpha_mode;
}

double picpml::alpha_face(const pml_desc& p, int face, double dc) {
  if (dc <= 0.0) return 1.0;
  const int mode = face_alpha_mode(p, face);
  if (mode == PML_ALPHA_ZERO) return 0.0;
  if (mode == PML_ALPHA_ONE || mode == PML_ALPHA_WEIGHT) return 1.0;
  const double v = p.v_assumed > 0 ? p.v_assumed : kC;
  const double e = p.sigma_max_coef * (kC / v) * p.delta_cells *
                   std::pow(dc / p.delta_cells, p.exponent + 1.0) / (p.exponent + 1.0);
  return std::exp(-e);
}

namespace {

template <typename T>
FieldPtrs<T>& fields(picpml_ctx* c);
template <>
FieldPtrs<float>& fields<float>(picpml_ctx* c) { return c->ff; }
template <>
FieldPtrs<double>& fields<double>(picpml_ctx* c) { return c->fd; }

template <typename T>
SpeciesPtrs<T> species_ptrs(picpml_ctx* ctx, Species& s) {
  SpeciesPtrs<T> p{};
  p.pos = s.desc.pos;
  p.mom = s.desc.mom;
  p.n_dev = s.n_dev;
  p.capacity = s.desc.capacity;
  p.ke = (T)s.ke;
  for (int a = 0; a < 3; ++a) p.cj[a] = (T)s.cj[a];
  p.cjy2d = (T)s.cjy2d;
  p.immobile = s.desc.immobile;
  p.qn = s.qn;
  p.save_pos = reinterpret_cast<float4*>(s.save);
  p.save_mom = nullptr;
  return p;
}

// The tile-resident kernel serves 3D order-1 boxes with FP32 fields (its
// deterministic form for PIC_FP32_FIXED64).
bool tile_capable(picpml_ctx* ctx) {
  return ctx->gd.dim == 3 && ctx->gd.prec != PIC_FP64 && ctx->gd.shape_order == 1 && ctx->tmap_ok;
}

// x^n scratch of the stage calls push() / deposit(), allocated on first use.
int ensure_save(picpml_ctx* ctx, Species& s) {
  if (s.save) return PIC_OK;
  s.save = dev_alloc(ctx, (size_t)std::max<long long>(s.desc.capacity, 1) * ctx->pbytes());
  return s.save ? PIC_OK : fail(ctx, PIC_ENOMEM, "species scratch");
}

// One launch of the tile-resident kernel for every sorted mobile species (up
// to kTileMaxSpecies); the others are marked in `done` as not handled.
int run_tile(picpml_ctx* ctx, std::vector<char>& done) {
  TileLaunch L{};
  L.prescribed = ctx->prescribed;
  const FieldPtrs<float>& f = ctx->ff;
  const float* base = f.E[0];
  for (int c = 0; c < 3; ++c) {
    L.arr_E[c] = (int)((f.E[c] - base) / ctx->g.size);
    L.arr_Bh[c] = (int)((f.Bh[c] - base) / ctx->g.size);
    L.arr_Bp[c] = (int)((f.Bp[c] - base) / ctx->g.size);
    L.arr_Bn[c] = f.Bn[c] ? (int)((f.Bn[c] - base) / ctx->g.size) : 0;
  }
  for (size_t i = 0; i < ctx->sp.size(); ++i) {
    Species& s = ctx->sp[i];
    if (s.desc.immobile || s.desc.capacity <= 0 || !s.tiled || L.nsp >= kTileMaxSpecies) continue;
    L.s[L.nsp].sp = species_ptrs<float>(ctx, s);
    L.s[L.nsp].tile_end = s.tile_end;
    ++L.nsp;
    done[i] = 1;
  }
  if (L.nsp == 0) return PIC_OK;
  if (!ctx->fixed() && ctx->bn_stale) {   // B^n for the box path, after B was set from outside
    CK(launch_bn_average(ctx->g, f, ctx->stream));
    ctx->launches += 1;
    ctx->bn_stale = false;
  }
  CK(launch_tile(ctx->g, ctx->tb, f, L, ctx->tmap, ctx->status, ctx->pushed, ctx->nsm, ctx->stream));
  ctx->launches += 1;
  return PIC_OK;
}

template <typename T>
int run_particles(picpml_ctx* ctx, int mode) {
  const bool fixed = ctx->fixed() && mode != 0;
  if (fixed) {
    // the integer sums of the previous deposit stay readable until here
    const size_t jb = (size_t)ctx->g.size * sizeof(long long);
    for (int c = 0; c < 3; ++c) CK(cudaMemsetAsync(ctx->ff.Jq[c], 0, jb, ctx->stream));
  }
  std::vector<char> done(ctx->sp.size(), 0);
  const bool tile = mode == 2 && ctx->ppt == PIC_TUNING_TILE && tile_capable(ctx);
  if (tile) {
    int r = run_tile(ctx, done);
    if (r) return r;
  }
  for (size_t i = 0; i < ctx->sp.size(); ++i) {
    Species& s = ctx->sp[i];
    if (done[i]) continue;
    if (s.desc.immobile && mode != 0) continue;
    if (mode != 2 && s.desc.capacity > 0) {
      int r = ensure_save(ctx, s);
      if (r) return r;
    }
    SpeciesPtrs<T> p = species_ptrs<T>(ctx, s);
    if (s.desc.capacity <= 0) continue;
    if (tile)   // a species not sorted since it was added: one thread per particle
      CK(launch_particles<T>(mode, ctx->gd.shape_order, ctx->g, ctx->tb, fields<T>(ctx), p, ctx->prescribed,
                             ctx->status, ctx->pushed, ctx->nsm, ctx->stream));
    else if (mode == 2 && ctx->gd.shape_order == 1 && ctx->ppt != 1 && !ctx->fixed())
      CK(launch_push_deposit_runs<T>(ctx->ppt, ctx->g, ctx->tb, fields<T>(ctx), p, ctx->prescribed, ctx->status,
                                     ctx->pushed, ctx->nsm, ctx->stream));
    else if (mode == 2 && ctx->gd.shape_order == 3 && ctx->gd.dim == 3 && ctx->ppt != 1 && !ctx->fixed())
      CK(launch_push_deposit_o3<T>(ctx->ppt, ctx->g, ctx->tb, fields<T>(ctx), p, ctx->prescribed, ctx->status,
                                   ctx->pushed, ctx->nsm, ctx->stream));
    else
      CK(launch_particles<T>(mode, ctx->gd.shape_order, ctx->g, ctx->tb, fields<T>(ctx), p, ctx->prescribed,
                             ctx->status, ctx->pushed, ctx->nsm, ctx->stream));
    ctx->launches += 1;
  }
  if (fixed) {
    const double* d = ctx->gd.d;
    // Every integer sum already carries the particle's charge number q/e.
    // J_x, J_z (and 3D J_y) are minus the prefix sums of Esirkepov's W, one
    // unit being e/(6 2^24) of charge crossing a cell face (in 2D the faces
    // are 1 m long along y): K_c = -e/(eps0 face area)/(6 2^24) of J' = J dt/eps0.
    // The 2D J_y sums shape products times v_y/c: K_y = +e c dt/(eps0 dx dz Ly)/(6 2^24).
    const double Ly = 1.0;
    const double K[3] = {ctx->gd.dim == 3 ? -kQe / (kEps0 * d[1] * d[2]) / kFixUnit : -kQe / (kEps0 * d[2] * Ly) / kFixUnit,
                         ctx->gd.dim == 3 ? -kQe / (kEps0 * d[0] * d[2]) / kFixUnit
                                          : kQe * ctx->dt * kC / (kEps0 * d[0] * d[2] * Ly) / kFixUnit,
                         ctx->gd.dim == 3 ? -kQe / (kEps0 * d[0] * d[1]) / kFixUnit : -kQe / (kEps0 * d[0] * Ly) / kFixUnit};
    CK(launch_fixed_flush(ctx->g, ctx->tb, ctx->ff, K, ctx->status, ctx->stream));
    ctx->launches += 1;
  }
  return PIC_OK;
}

template <typename T>
int run_field(picpml_ctx* ctx) {
  FieldPtrs<T>& f = fields<T>(ctx);
  for (int p = 0; p < ctx->gd.filter_passes; ++p) {   // App. A: the current is filtered first
    T* const O[3] = {(T*)ctx->filter_tmp[0], (T*)ctx->filter_tmp[1], (T*)ctx->filter_tmp[2]};
    CK(launch_filter_J<T>(ctx->g, f, O, ctx->stream));
    ctx->launches += 2;
  }
  CK(launch_field_E<T>(ctx->g, ctx->tb, f, ctx->split_ff(), ctx->kz, ctx->stream));
  if (ctx->ncond > 0) {   // zeroed-field cells: their edges' E after the E pass
    CK(launch_conductor<T>(ctx->g, f, ctx->cond, ctx->ncond, ctx->stream));
    ctx->launches += 1;
  }
  if (ctx->gd.solver == PIC_SOLVER_CK)
    CK(launch_field_B_ck<T>(ctx->g, ctx->tb, f, ctx->split_ff(), ctx->stream));
  else
    CK(launch_field_B<T>(ctx->g, ctx->tb, f, ctx->split_ff(), ctx->kz, ctx->stream));
  ctx->launches += 2;
  for (int c = 0; c < 3; ++c) std::swap(f.Bh[c], f.Bp[c]);
  ctx->bn_stale = f.Bn[0] == nullptr;   // the B pass wrote Bn where it exists
  return PIC_OK;
}

int check_ready(picpml_ctx* ctx) {
  if (!ctx) return fail(nullptr, PIC_EINVAL, "null context");
  if (!ctx->ready) return fail(ctx, PIC_ESTATE, "pml_init has not been called");
  return PIC_OK;
}

template <typename T>
int do_sort(picpml_ctx* ctx) {
  const long long ncell = sort_keys(ctx->g);
  if (!ctx->sort_scratch) {
    ctx->sort_scratch = (unsigned*)dev_alloc(ctx, sort_scratch_words(ncell) * sizeof(unsigned));
    if (!ctx->sort_scratch) return fail(ctx, PIC_ENOMEM, "sort scratch");
  }
  for (auto& s : ctx->sp) {
    if (!s.tmp_pos) {
      s.tmp_pos = dev_alloc(ctx, (size_t)s.desc.capacity * ctx->pbytes());
      s.tmp_mom = dev_alloc(ctx, (size_t)s.desc.capacity * ctx->pbytes());
      if (!s.tmp_pos || !s.tmp_mom) return fail(ctx, PIC_ENOMEM, "sort buffers");
    }
    CK(launch_sort(ctx->g, ctx->pbytes(), s.desc.pos, s.desc.mom, s.n_dev, s.desc.capacity, ctx->sort_scratch,
                   s.tmp_pos, s.tmp_mom, ctx->stream));
    ctx->launches += sort_launches(ncell);
    const long long nt = tile_count(ctx->g);
    if (nt > 0) {   // 3D: where each sort tile's particles end (the tile kernel's work ranges)
      if (!s.tile_end) {
        s.tile_end = (long long*)dev_alloc(ctx, (size_t)nt * sizeof(long long));
        if (!s.tile_end) return fail(ctx, PIC_ENOMEM, "tile offsets");
      }
      CK(launch_tile_ends(ctx->g, ctx->sort_scratch, s.tile_end, ctx->stream));
      ctx->launches += 1;
      s.tiled = true;
    }
  }
  return PIC_OK;
}

}  // namespace

extern "C" {

int pic_init(picpml_ctx** out, const pic_grid_desc* g, void* stream) {
  if (!out || !g) return fail(nullptr, PIC_EINVAL, "null argument");
  *out = nullptr;
  if (g->dim != 2 && g->dim != 3) return fail(nullptr, PIC_EINVAL, "dim must be 2 or 3");
  if (g->shape_order != 1 && g->shape_order != 3) return fail(nullptr, PIC_EINVAL, "shape_order must be 1 or 3");
  if (g->prec != PIC_FP32 && g->prec != PIC_FP64 && g->prec != PIC_FP32_FIXED64)
    return fail(nullptr, PIC_EINVAL, "bad prec");
  if (g->filter_passes < 0 || g->filter_passes > 8) return fail(nullptr, PIC_EINVAL, "filter_passes must be 0..8");
  if (g->solver != PIC_SOLVER_YEE && g->solver != PIC_SOLVER_CK)
    return fail(nullptr, PIC_EINVAL, "solver must be PIC_SOLVER_YEE or PIC_SOLVER_CK");
  for (int a = 0; a < 3; ++a) {
    if (g->dim == 2 && a == 1) continue;
    if (g->n[a] < 1 || !(g->d[a] > 0)) return fail(nullptr, PIC_EINVAL, "cells and cell sizes must be positive");
  }
  pic_grid_desc gd = *g;
  if (gd.dim == 2) {
    gd.n[1] = 0;
    gd.d[1] = 1.0;
  }
  const double lim = courant_limit(gd);
  double dt = gd.dt;
  if (!(dt > 0)) {
    if (!(gd.cfl > 0 && gd.cfl <= 1.0)) return fail(nullptr, PIC_EINVAL, "dt <= 0 needs 0 < cfl <= 1");
    dt = gd.cfl * lim;
  }
  if (dt > lim * (1 + 1e-12)) return fail(nullptr, PIC_ECFL, "dt above the field solver's Courant limit");
  picpml_ctx* ctx = new picpml_ctx();
  ctx->gd = gd;
  ctx->dt = dt;
  ctx->stream = (cudaStream_t)stream;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, dev);
  *out = ctx;
  return PIC_OK;
}

int pml_init(picpml_ctx* ctx, const pml_desc* p) {
  if (!ctx || !p) return fail(ctx, PIC_EINVAL, "null argument");
  if (ctx->ready) return fail(ctx, PIC_ESTATE, "pml_init called twice");
  if (p->alpha_mode < 0 || p->alpha_mode > 3) return fail(ctx, PIC_EINVAL, "bad alpha_mode");
  if (p->face_alpha_set) {
    if (p->alpha_mode == PML_ALPHA_WEIGHT) return fail(ctx, PIC_EINVAL, "per-face modes with weight damping");
    for (int f = 0; f < 6; ++f)
      if (p->face_alpha[f] < PML_ALPHA_ZERO || p->face_alpha[f] > PML_ALPHA_DAMPED)
        return fail(ctx, PIC_EINVAL, "per-face alpha modes are zero, one or damped");
  }
  if (p->sigma_max_coef < 0 || !(p->delta_cells > 0) || p->exponent < 0)
    return fail(ctx, PIC_EINVAL, "bad conductivity profile");
  const pic_grid_desc& gd = ctx->gd;
  ctx->pd = *p;
  Geom& g = ctx->g;
  g.dim = gd.dim;
  const int margin = gd.shape_order == 1 ? 2 : 3;
  for (int a = 0; a < 3; ++a) {
    if (gd.dim == 2 && a == 1) {
      g.N[1] = 0; g.nn[1] = 1; g.plo[1] = 0; g.nph[1] = 0; g.rmin[1] = 0; g.rmax[1] = 1 << 30;
      g.S[1] = 0.0;
      g.Sf[1] = g.Sfl[1] = 0.f;
      continue;
    }
    const int lo = p->ncell[2 * a], hi = p->ncell[2 * a + 1];
    if (lo < 0 || hi < 0) return fail(ctx, PIC_EINVAL, "negative PML width");
    g.plo[a] = lo;
    g.nph[a] = gd.n[a];
    g.N[a] = gd.n[a] + lo + hi;
    g.nn[a] = g.N[a] + 1;
    g.S[a] = kC * ctx->dt / gd.d[a];
    g.Sf[a] = (float)g.S[a];
    g.Sfl[a] = (float)(g.S[a] - (double)g.Sf[a]);
    int rmin = margin, rmax = g.N[a] - margin;
    if (face_alpha_mode(*p, 2 * a) == PML_ALPHA_ZERO) rmin = std::max(rmin, lo);   // removed at the interface
    if (face_alpha_mode(*p, 2 * a + 1) == PML_ALPHA_ZERO) rmax = std::min(rmax, lo + gd.n[a]);
    g.rmin[a] = rmin;
    g.rmax[a] = rmax;
    if (rmax <= rmin) return fail(ctx, PIC_EINVAL, "grid too small for the particle shape");
  }
  if (g.N[0] > 1023 || g.N[1] > 1023 || g.N[2] > 2047)
    return fail(ctx, PIC_EINVAL, "grid too large for the packed cell index (1023 x 1023 x 2047 cells)");
  g.wdamp = p->alpha_mode == PML_ALPHA_WEIGHT ? 1 : 0;
  for (int a = 0; a < 3; ++a) g.wk[a] = (gd.dim == 2 && a == 1) ? 0.0 : p->sigma_max_coef * g.S[a];
  g.winv_delta = 1.0 / p->delta_cells;
  g.wexp = p->exponent;
  g.px = (g.nn[0] + 7) / 8 * 8;
  g.sy = g.px;
  g.sz = (long long)g.px * g.nn[1];
  g.size = g.sz * g.nn[2];

  // per-axis tables at nodes and centres
  std::vector<double> host;
  const int nt = 10;  // ea_n eb_n sdt_n ea_c eb_c sdt_c al_nd al_cd (+2 float arrays packed after)
  size_t total = 0;
  for (int a = 0; a < 3; ++a) total += (size_t)g.nn[a];
  host.assign(total * nt, 0.0);
  std::vector<float> hostf(total * 4, 0.f);      // alpha (n, c), s dt (n, c) as float
  std::vector<float2> host2(total * 4);           // ea, eb (n, c) as float-float pairs
  double* td = (double*)dev_alloc(ctx, host.size() * sizeof(double));
  float* tf = (float*)dev_alloc(ctx, hostf.size() * sizeof(float));
  float2* t2 = (float2*)dev_alloc(ctx, host2.size() * sizeof(float2));
  if (!td || !tf || !t2) return fail(ctx, PIC_ENOMEM, "tables");
  auto split2 = [](double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
  };
  size_t off = 0;
  for (int a = 0; a < 3; ++a) {
    const int nn = g.nn[a];
    std::vector<double> t8(8 * (size_t)nn);
    double* q8 = t8.data();
    build_axis_table(*p, a, gd.d[a], ctx->dt, g.plo[a], g.nph[a], nn, !(gd.dim == 2 && a == 1), q8, q8 + nn,
                     q8 + 2 * nn, q8 + 3 * nn, q8 + 4 * nn, q8 + 5 * nn, q8 + 6 * nn, q8 + 7 * nn);
    for (int i = 0; i < nn; ++i) {
      for (int stag = 0; stag < 2; ++stag) {
        const double ea = q8[(stag * 3 + 0) * nn + i], eb = q8[(stag * 3 + 1) * nn + i];
        const double sdt = q8[(stag * 3 + 2) * nn + i], al = q8[(6 + stag) * nn + i];
        const size_t base = off + i;
        host[(stag * 3 + 0) * total + base] = ea;
        host[(stag * 3 + 1) * total + base] = eb;
        host[(stag * 3 + 2) * total + base] = sdt;
        host[(6 + stag) * total + base] = al;
        hostf[stag * total + base] = (float)al;
        hostf[(2 + stag) * total + base] = (float)sdt;
        host2[(stag * 2 + 0) * total + base] = split2(ea);
        host2[(stag * 2 + 1) * total + base] = split2(eb);
      }
    }
    {  // the run of nodes (and their centres) where alpha is exactly 1
      const double* aln = q8 + 6 * nn;
      const double* alc = q8 + 7 * nn;
      int lo = 0;
      while (lo < nn && !(aln[lo] == 1.0 && alc[lo] == 1.0)) ++lo;
      int hi = lo;
      while (hi + 1 < nn && aln[hi + 1] == 1.0 && alc[hi + 1] == 1.0) ++hi;
      ctx->tb.al1_lo[a] = lo < nn ? lo : 1;
      ctx->tb.al1_hi[a] = lo < nn ? hi : 0;   // empty when alpha is nowhere 1
    }
    ctx->tb.ea_n[a] = td + 0 * total + off;
    ctx->tb.eb_n[a] = td + 1 * total + off;
    ctx->tb.sdt_n[a] = td + 2 * total + off;
    ctx->tb.ea_c[a] = td + 3 * total + off;
    ctx->tb.eb_c[a] = td + 4 * total + off;
    ctx->tb.sdt_c[a] = td + 5 * total + off;
    ctx->tb.al_nd[a] = td + 6 * total + off;
    ctx->tb.al_cd[a] = td + 7 * total + off;
    ctx->tb.al_nf[a] = tf + off;
    ctx->tb.al_cf[a] = tf + total + off;
    ctx->tb.sdtf_n[a] = tf + 2 * total + off;
    ctx->tb.sdtf_c[a] = tf + 3 * total + off;
    ctx->tb.ea2_n[a] = t2 + 0 * total + off;
    ctx->tb.eb2_n[a] = t2 + 1 * total + off;
    ctx->tb.ea2_c[a] = t2 + 2 * total + off;
    ctx->tb.eb2_c[a] = t2 + 3 * total + off;
    off += nn;
  }
  CK(cudaMemcpyAsync(td, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(tf, hostf.data(), hostf.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(t2, host2.data(), host2.size() * sizeof(float2), cudaMemcpyHostToDevice, ctx->stream));

  // fields: 12 arrays of the field type + 12 FP64 split arrays, then, for
  // the tile kernel's box path (3D, FP32, order 1), the 3 FP32 arrays of B at
  // the integer time; zeroed
  const size_t es = ctx->elem();
  const bool bn = gd.dim == 3 && gd.prec == PIC_FP32 && gd.shape_order == 1;
  const size_t fbytes = (size_t)g.size * (12 * es + 12 * 8 + (bn ? 12 : 0));
  ctx->field_bytes = fbytes;
  char* fm = (char*)dev_alloc(ctx, fbytes);
  if (!fm) return fail(ctx, PIC_ENOMEM, "fields");
  CK(cudaMemsetAsync(fm, 0, fbytes, ctx->stream));
  char* q = fm;
  for (int c = 0; c < 3; ++c) {
    void* arr[4];
    for (int t = 0; t < 4; ++t) { arr[t] = q; q += (size_t)g.size * es; }
    if (gd.prec == PIC_FP64) {
      ctx->fd.E[c] = (double*)arr[0]; ctx->fd.Bh[c] = (double*)arr[1];
      ctx->fd.Bp[c] = (double*)arr[2]; ctx->fd.J[c] = (double*)arr[3];
    } else {
      ctx->ff.E[c] = (float*)arr[0]; ctx->ff.Bh[c] = (float*)arr[1];
      ctx->ff.Bp[c] = (float*)arr[2]; ctx->ff.J[c] = (float*)arr[3];
    }
  }
  for (int c = 0; c < 3; ++c)
    for (int h = 0; h < 2; ++h) {
      double* e = (double*)q; q += (size_t)g.size * 8;
      double* b = (double*)q; q += (size_t)g.size * 8;
      ctx->ff.Es[c][h] = ctx->fd.Es[c][h] = e;
      ctx->ff.Bs[c][h] = ctx->fd.Bs[c][h] = b;
    }
  if (bn)
    for (int c = 0; c < 3; ++c) {
      ctx->ff.Bn[c] = (float*)q;
      q += (size_t)g.size * 4;
    }
  ctx->bn_stale = true;
  if (gd.filter_passes > 0) {
    char* ft = (char*)dev_alloc(ctx, (size_t)g.size * 3 * es);
    if (!ft) return fail(ctx, PIC_ENOMEM, "filter scratch");
    CK(cudaMemsetAsync(ft, 0, (size_t)g.size * 3 * es, ctx->stream));
    for (int c = 0; c < 3; ++c) ctx->filter_tmp[c] = ft + (size_t)c * g.size * es;
  }
  if (ctx->fixed()) {
    long long* jq = (long long*)dev_alloc(ctx, (size_t)g.size * 3 * sizeof(long long));
    if (!jq) return fail(ctx, PIC_ENOMEM, "fixed-point current");
    CK(cudaMemsetAsync(jq, 0, (size_t)g.size * 3 * sizeof(long long), ctx->stream));
    for (int c = 0; c < 3; ++c) ctx->ff.Jq[c] = jq + (size_t)c * g.size;
  }
  if (gd.dim == 3 && gd.prec != PIC_FP64 && tile_map_bytes() <= (int)sizeof(ctx->tmap))
    ctx->tmap_ok = make_tile_tensor_map(g, ctx->ff.E[0], (int)(fbytes / ((size_t)g.size * 4)), ctx->tmap) ==
                   cudaSuccess;
  ctx->status = (unsigned*)dev_alloc(ctx, 64);
  ctx->pushed = (unsigned long long*)(ctx->status + 8);
  ctx->diag = (double*)dev_alloc(ctx, 8 * sizeof(double));
  if (!ctx->status || !ctx->diag) return fail(ctx, PIC_ENOMEM, "status");
  CK(cudaMemsetAsync(ctx->status, 0, 64, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->ready = true;
  return PIC_OK;
}

int pic_add_species(picpml_ctx* ctx, const pic_species* s, int* sid) {
  int r = check_ready(ctx);
  if (r) return r;
  if (!s || !sid) return fail(ctx, PIC_EINVAL, "null argument");
  if (s->n < 0 || s->capacity < s->n || (s->capacity > 0 && (!s->pos || !s->mom)))
    return fail(ctx, PIC_EINVAL, "bad particle arrays");
  if (!(s->m > 0)) return fail(ctx, PIC_EINVAL, "mass must be positive");
  if ((reinterpret_cast<uintptr_t>(s->pos) | reinterpret_cast<uintptr_t>(s->mom)) % ctx->pbytes())
    return fail(ctx, PIC_EINVAL, "particle arrays must be aligned to one particle record");
  Species sp;
  sp.desc = *s;
  sp.n_dev = (long long*)dev_alloc(ctx, sizeof(long long));
  if (!sp.n_dev) return fail(ctx, PIC_ENOMEM, "species scratch");
  CK(cudaMemcpyAsync(sp.n_dev, &s->n, sizeof(long long), cudaMemcpyHostToDevice, ctx->stream));
  const pic_grid_desc& gd = ctx->gd;
  const double q = s->q, dt = ctx->dt;
  sp.ke = q * dt / (2.0 * s->m * kC);
  sp.qn = q / kQe;
  if (gd.dim == 3) {
    sp.cj[0] = -q / (kEps0 * gd.d[1] * gd.d[2]);
    sp.cj[1] = -q / (kEps0 * gd.d[0] * gd.d[2]);
    sp.cj[2] = -q / (kEps0 * gd.d[0] * gd.d[1]);
  } else {
    const double Ly = 1.0;  // a 2D macroparticle is a line charge of 1 m along y
    sp.cj[0] = -q / (kEps0 * gd.d[2] * Ly);
    sp.cj[2] = -q / (kEps0 * gd.d[0] * Ly);
    sp.cjy2d = q * dt * kC / (kEps0 * gd.d[0] * gd.d[2] * Ly);
  }
  ctx->sp.push_back(sp);
  *sid = (int)ctx->sp.size() - 1;
  CK(cudaStreamSynchronize(ctx->stream));
  return PIC_OK;
}

int push(picpml_ctx* ctx) {
  NvtxRange nvtx_("picpml push");
  int r = check_ready(ctx);
  if (r) return r;
  return ctx->gd.prec == PIC_FP64 ? run_particles<double>(ctx, 0) : run_particles<float>(ctx, 0);
}

int deposit(picpml_ctx* ctx) {
  NvtxRange nvtx_("picpml deposit");
  int r = check_ready(ctx);
  if (r) return r;
  return ctx->gd.prec == PIC_FP64 ? run_particles<double>(ctx, 1) : run_particles<float>(ctx, 1);
}

int field_step(picpml_ctx* ctx) {
  NvtxRange nvtx_("picpml field_step");
  int r = check_ready(ctx);
  if (r) return r;
  return ctx->gd.prec == PIC_FP64 ? run_field<double>(ctx) : run_field<float>(ctx);
}

int pic_sort(picpml_ctx* ctx) {
  NvtxRange nvtx_("picpml pic_sort");
  int r = check_ready(ctx);
  if (r) return r;
  return ctx->gd.prec == PIC_FP64 ? do_sort<double>(ctx) : do_sort<float>(ctx);
}

int push_deposit(picpml_ctx* ctx) {
  NvtxRange nvtx_("picpml push_deposit");
  int r = check_ready(ctx);
  if (r) return r;
  return ctx->gd.prec == PIC_FP64 ? run_particles<double>(ctx, 2) : run_particles<float>(ctx, 2);
}

int pic_particle_steps(picpml_ctx* ctx, long long* n) {
  int r = check_ready(ctx);
  if (r) return r;
  if (!n) return fail(ctx, PIC_EINVAL, "null argument");
  unsigned long long v = 0;
  CK(cudaMemcpyAsync(&v, ctx->pushed, sizeof(v), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  *n = (long long)v;
  return PIC_OK;
}

namespace {
struct Snapshot {
  std::vector<std::pair<void*, size_t>> items;   // (source, bytes)
  std::vector<void*> copies;
};
}  // namespace

// Times the particle kernel for each particles-per-thread choice and the field
// kernels for each z-nodes-per-thread choice over `steps` steps each, starting
// every candidate from the same state (a device-side snapshot of the fields,
// the particle records and the counters, restored afterwards), and keeps the
// fastest.  The result does not depend on the choice beyond round-off order.
int pic_autotune(picpml_ctx* ctx, int steps, int* ppt, int* kz) {
  NvtxRange nvtx_("picpml pic_autotune");
  int r = check_ready(ctx);
  if (r) return r;
  if (steps < 1) steps = 3;
  const bool f64 = ctx->gd.prec == PIC_FP64;
  Snapshot sn;
  const size_t es = ctx->elem();
  void* fm = f64 ? (void*)ctx->fd.E[0] : (void*)ctx->ff.E[0];
  sn.items.push_back({fm, ctx->field_bytes});
  (void)es;
  const bool bn_stale0 = ctx->bn_stale;
  for (auto& s : ctx->sp) {
    sn.items.push_back({s.desc.pos, (size_t)s.desc.capacity * ctx->pbytes()});
    sn.items.push_back({s.desc.mom, (size_t)s.desc.capacity * ctx->pbytes()});
    sn.items.push_back({s.n_dev, sizeof(long long)});
  }
  sn.items.push_back({ctx->status, 64});
  for (auto& it : sn.items) {
    void* c = nullptr;
    if (cudaMalloc(&c, it.second) != cudaSuccess) {
      for (void* q : sn.copies) cudaFree(q);
      return fail(ctx, PIC_ENOMEM, "autotune snapshot");
    }
    sn.copies.push_back(c);
    CK(cudaMemcpyAsync(c, it.first, it.second, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  auto restore = [&]() -> cudaError_t {
    for (size_t t = 0; t < sn.items.size(); ++t) {
      cudaError_t e = cudaMemcpyAsync(sn.items[t].first, sn.copies[t], sn.items[t].second,
                                      cudaMemcpyDeviceToDevice, ctx->stream);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  // the field kernels write B into the "previous" buffer: keep the pointer order
  FieldPtrs<float> ff0 = ctx->ff;
  FieldPtrs<double> fd0 = ctx->fd;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // A particle candidate is timed over whole steps (push + deposit, then the
  // field step, which is not timed): the fields the particles see then evolve
  // as in a run; without the field steps they stay at their start values,
  // which favoured the wrong launch shape for a beam starting in vacuum.
  auto time_it = [&](bool particles, float* ms) -> int {
    int rr = 0;
    *ms = 0.f;
    // warm-up step, then the timed ones
    for (int t = 0; t <= steps; ++t) {
      if (t >= 1) CK(cudaEventRecord(e0, ctx->stream));
      rr = particles ? (f64 ? run_particles<double>(ctx, 2) : run_particles<float>(ctx, 2))
                     : (f64 ? run_field<double>(ctx) : run_field<float>(ctx));
      if (rr) return rr;
      if (t >= 1) {
        CK(cudaEventRecord(e1, ctx->stream));
        CK(cudaEventSynchronize(e1));
        float one = 0.f;
        CK(cudaEventElapsedTime(&one, e0, e1));
        *ms += one;
      }
      if (particles) {
        rr = f64 ? run_field<double>(ctx) : run_field<float>(ctx);
        if (rr) return rr;
      }
    }
    *ms /= steps;
    CK(restore());
    ctx->ff = ff0;
    ctx->fd = fd0;
    ctx->bn_stale = bn_stale0;
    return PIC_OK;
  };
  const long long launches0 = ctx->launches;
  int best_p = ctx->ppt, best_k = ctx->kz;
  if ((ctx->gd.shape_order == 1 || ctx->gd.dim == 3) && !ctx->fixed()) {
    float best = 1e30f;
    bool all_tiled = tile_capable(ctx);
    for (auto& s : ctx->sp)
      if (!s.desc.immobile && s.desc.capacity > 0 && !s.tiled) all_tiled = false;
    for (int p : {1, PIC_TUNING_TILE, 4, 8}) {
      if (f64 && p == 8) continue;
      if (p == PIC_TUNING_TILE && !all_tiled) continue;
      ctx->ppt = p;
      float ms = 0;
      r = time_it(true, &ms);
      if (r) return r;
      if (ms < best) { best = ms; best_p = p; }
    }
  }
  {
    float best = 1e30f;
    for (int k : {1, 2, 4}) {
      ctx->kz = k;
      float ms = 0;
      r = time_it(false, &ms);
      if (r) return r;
      if (ms < best) { best = ms; best_k = k; }
    }
  }
  ctx->ppt = best_p;
  ctx->kz = best_k;
  ctx->launches = launches0;
  CK(cudaStreamSynchronize(ctx->stream));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (void* q : sn.copies) cudaFree(q);
  if (ppt) *ppt = ctx->ppt;
  if (kz) *kz = ctx->kz;
  return PIC_OK;
}

int pic_set_tuning(picpml_ctx* ctx, int ppt, int kz) {
  if (!ctx) return fail(nullptr, PIC_EINVAL, "null context");
  if (!(ppt == 0 || ppt == 1 || ppt == PIC_TUNING_TILE || ppt == 4 || ppt == 8) || !(kz == 1 || kz == 2 || kz == 4))
    return fail(ctx, PIC_EINVAL,
                "particles per thread must be 0, 1, 2 (tile kernel), 4 or 8; z nodes per thread 1, 2 or 4");
  ctx->ppt = ppt;
  ctx->kz = kz;
  return PIC_OK;
}

int pic_launch_count(picpml_ctx* ctx, long long* n) {
  if (!ctx || !n) return fail(ctx, PIC_EINVAL, "null argument");
  *n = ctx->launches;
  return PIC_OK;
}

int step_n(picpml_ctx* ctx, int n) {
  NvtxRange nvtx_("picpml step_n");
  int r = check_ready(ctx);
  if (r) return r;
  if (n < 0) return fail(ctx, PIC_EINVAL, "negative step count");
  const bool f64 = ctx->gd.prec == PIC_FP64;
  for (int s = 0; s < n; ++s) {
    if (ctx->gd.sort_every > 0 && ctx->steps_done % ctx->gd.sort_every == 0) {
      r = f64 ? do_sort<double>(ctx) : do_sort<float>(ctx);
      if (r) return r;
    }
    r = f64 ? run_particles<double>(ctx, 2) : run_particles<float>(ctx, 2);
    if (r) return r;
    r = f64 ? run_field<double>(ctx) : run_field<float>(ctx);
    if (r) return r;
    ctx->steps_done++;
  }
  return PIC_OK;
}

int pic_set_old_positions(picpml_ctx* ctx, int sid, const void* src) {
  int r = check_ready(ctx);
  if (r) return r;
  if (sid < 0 || sid >= (int)ctx->sp.size() || !src) return fail(ctx, PIC_EINVAL, "bad species id or source");
  Species& s = ctx->sp[sid];
  if (s.desc.capacity > 0) {
    r = ensure_save(ctx, s);
    if (r) return r;
  }
  if (s.desc.capacity > 0)
    CK(cudaMemcpyAsync(s.save, src, (size_t)s.desc.capacity * ctx->pbytes(), cudaMemcpyDeviceToDevice,
                       ctx->stream));
  return PIC_OK;
}

int pic_get_current_fixed(picpml_ctx* ctx, int comp, long long* dst) {
  int r = check_ready(ctx);
  if (r) return r;
  if (!ctx->fixed()) return fail(ctx, PIC_ESTATE, "the context does not use fixed-point deposition");
  if (comp < 0 || comp > 2 || !dst) return fail(ctx, PIC_EINVAL, "bad component or destination");
  const Geom& g = ctx->g;
  CK(cudaMemcpy2DAsync(dst, (size_t)g.nn[0] * sizeof(long long), ctx->ff.Jq[comp], (size_t)g.px * sizeof(long long),
                       (size_t)g.nn[0] * sizeof(long long), (size_t)g.nn[1] * g.nn[2], cudaMemcpyDeviceToDevice,
                       ctx->stream));
  return PIC_OK;
}

int pic_grid_info(picpml_ctx* ctx, int* nn3, double* dt) {
  int r = check_ready(ctx);
  if (r) return r;
  if (nn3) for (int a = 0; a < 3; ++a) nn3[a] = ctx->g.nn[a];
  if (dt) *dt = ctx->dt;
  return PIC_OK;
}

int pic_get_field(picpml_ctx* ctx, int which, void* dst, int as_double) {
  int r = check_ready(ctx);
  if (r) return r;
  if (!dst || which < 0 || which > 14) return fail(ctx, PIC_EINVAL, "bad field selector");
  const int c = which % 3, kind = which / 3;
  const double scale = kind == 0 ? 1.0 : kind == 2 ? kEps0 / ctx->dt : 1.0 / kC;
  if (ctx->gd.prec == PIC_FP64) {
    FieldPtrs<double>& f = ctx->fd;
    const double* a = kind == 0 ? f.E[c] : kind == 2 ? f.J[c] : kind == 4 ? f.Bp[c] : f.Bh[c];
    const double* b = kind == 1 ? f.Bp[c] : nullptr;
    CK(launch_export<double>(ctx->g, a, b, scale, dst, as_double, ctx->stream));
  } else {
    FieldPtrs<float>& f = ctx->ff;
    const float* a = kind == 0 ? f.E[c] : kind == 2 ? f.J[c] : kind == 4 ? f.Bp[c] : f.Bh[c];
    const float* b = kind == 1 ? f.Bp[c] : nullptr;
    CK(launch_export<float>(ctx->g, a, b, scale, dst, as_double, ctx->stream));
  }
  return PIC_OK;
}

int pic_set_field(picpml_ctx* ctx, int which, const void* src, int as_double) {
  int r = check_ready(ctx);
  if (r) return r;
  if (!src || !(which / 3 == 0 || which / 3 == 3 || which / 3 == 4)) return fail(ctx, PIC_EINVAL, "bad field selector");
  const int c = which % 3, kind = which / 3;
  const double scale = kind == 0 ? 1.0 : kC;
  double* s0 = kind == 0 ? ctx->fd.Es[c][0] : kind == 3 ? ctx->fd.Bs[c][0] : nullptr;
  double* s1 = kind == 0 ? ctx->fd.Es[c][1] : kind == 3 ? ctx->fd.Bs[c][1] : nullptr;
  if (ctx->gd.prec == PIC_FP64) {
    double* a = kind == 0 ? ctx->fd.E[c] : kind == 3 ? ctx->fd.Bh[c] : ctx->fd.Bp[c];
    CK(launch_import<double>(ctx->g, src, as_double, scale, a, s0, s1, 0, ctx->stream));
  } else {
    float* a = kind == 0 ? ctx->ff.E[c] : kind == 3 ? ctx->ff.Bh[c] : ctx->ff.Bp[c];
    CK(launch_import<float>(ctx->g, src, as_double, scale, a, s0, s1, ctx->split_ff(), ctx->stream));
  }
  if (kind != 0) ctx->bn_stale = true;
  return PIC_OK;
}

int pic_set_conductor(picpml_ctx* ctx, const unsigned char* mask) {
  int r = check_ready(ctx);
  if (r) return r;
  if (!mask) {
    ctx->ncond = 0;
    return PIC_OK;
  }
  const Geom& g = ctx->g;
  const long long N0 = g.N[0], N1 = g.dim == 3 ? g.N[1] : 1, N2 = g.N[2];
  std::vector<int> cells;
  for (long long t = 0; t < N0 * N1 * N2; ++t)
    if (mask[t]) cells.push_back((int)t);
  if ((long long)cells.size() > ctx->cond_cap) {
    ctx->cond = (int*)dev_alloc(ctx, cells.size() * sizeof(int));
    if (!ctx->cond) return fail(ctx, PIC_ENOMEM, "conductor cells");
    ctx->cond_cap = (long long)cells.size();
  }
  if (!cells.empty())
    CK(cudaMemcpyAsync(ctx->cond, cells.data(), cells.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->ncond = (long long)cells.size();
  return PIC_OK;
}

int pic_set_prescribed(picpml_ctx* ctx, int flag) {
  if (!ctx) return fail(nullptr, PIC_EINVAL, "null context");
  ctx->prescribed = flag ? 1 : 0;
  return PIC_OK;
}

int pic_num_particles(picpml_ctx* ctx, int sid, long long* n) {
  int r = check_ready(ctx);
  if (r) return r;
  if (sid < 0 || sid >= (int)ctx->sp.size() || !n) return fail(ctx, PIC_EINVAL, "bad species id");
  CK(cudaMemcpyAsync(n, ctx->sp[sid].n_dev, sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return PIC_OK;
}

int pic_sync(picpml_ctx* ctx) {
  int r = check_ready(ctx);
  if (r) return r;
  CK(cudaStreamSynchronize(ctx->stream));
  unsigned st = 0;
  CK(cudaMemcpy(&st, ctx->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (st & ST_BAD_PARTICLE)
    return fail(ctx, PIC_EPARTICLE, "a particle was outside its allowed cells or not finite (removed)");
  if (st & ST_FIXED_OVERFLOW) return fail(ctx, PIC_EOVERFLOW, "fixed-point current overflow");
  if (st & ST_INJECT_OVERFLOW) return fail(ctx, PIC_EOVERFLOW, "injected particles beyond the species capacity (dropped)");
  if (st & ST_TIMEOUT) return fail(ctx, PIC_ETIMEOUT, "a kernel gave up waiting for its field box copy (2 s)");
  return PIC_OK;
}

int pic_inject(picpml_ctx* ctx, int sid, const void* pos, const void* mom, long long count) {
  NvtxRange nvtx_("picpml pic_inject");
  int r = check_ready(ctx);
  if (r) return r;
  if (sid < 0 || sid >= (int)ctx->sp.size()) return fail(ctx, PIC_EINVAL, "bad species id");
  if (count < 0 || (count > 0 && (!pos || !mom))) return fail(ctx, PIC_EINVAL, "bad particle arrays");
  if ((reinterpret_cast<uintptr_t>(pos) | reinterpret_cast<uintptr_t>(mom)) % ctx->pbytes())
    return fail(ctx, PIC_EINVAL, "particle arrays must be aligned to one particle record");
  Species& s = ctx->sp[sid];
  CK(launch_inject(ctx->pbytes(), s.desc.pos, s.desc.mom, s.n_dev, s.desc.capacity, pos, mom, count, ctx->status,
                   ctx->stream));
  ctx->launches += count > 0 ? 2 : 0;
  return PIC_OK;
}

}  // extern "C"

namespace {
// The Gauss-law residual, charge-density scale and field energy of the
// current state into out[0..2] with rho as charge-density scratch (zeroed
// here), read back to the host.  Shared by pic_diag (scratch allocated on
// first use) and pic_diag_static (file-scope scratch).
int diag_into(picpml_ctx* ctx, double* rho, double* out, double* gauss, double* rho_scale, double* energy) {
  CK(cudaMemsetAsync(rho, 0, (size_t)ctx->g.size * sizeof(double), ctx->stream));
  CK(cudaMemsetAsync(out, 0, 3 * sizeof(double), ctx->stream));
  const pic_grid_desc& gd = ctx->gd;
  const double V = gd.d[0] * gd.d[2] * (gd.dim == 3 ? gd.d[1] : 1.0);
  for (auto& s : ctx->sp) {
    const double qoe = s.desc.q / (kEps0 * V);
    if (gd.prec == PIC_FP64)
      CK(launch_rho<double>(gd.shape_order, ctx->g, s.desc.pos, s.desc.mom, s.n_dev, s.desc.capacity, qoe, rho,
                            ctx->stream));
    else
      CK(launch_rho<float>(gd.shape_order, ctx->g, s.desc.pos, s.desc.mom, s.n_dev, s.desc.capacity, qoe, rho,
                           ctx->stream));
  }
  if (gd.prec == PIC_FP64) CK(launch_gauss<double>(ctx->g, ctx->fd, rho, gd.d, out, ctx->stream));
  else CK(launch_gauss<float>(ctx->g, ctx->ff, rho, gd.d, out, ctx->stream));
  double h[3];
  CK(cudaMemcpyAsync(h, out, 3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (gauss) *gauss = h[0];
  if (rho_scale) *rho_scale = h[1];
  if (energy) *energy = h[2];
  return pic_sync(ctx);
}
}  // namespace

extern "C" {

int pic_diag(picpml_ctx* ctx, double* gauss, double* rho_scale, double* energy) {
  NvtxRange nvtx_("picpml pic_diag");
  int r = check_ready(ctx);
  if (r) return r;
  if (!ctx->rho) {
    ctx->rho = (double*)dev_alloc(ctx, (size_t)ctx->g.size * sizeof(double));
    if (!ctx->rho) return fail(ctx, PIC_ENOMEM, "rho");
  }
  return diag_into(ctx, ctx->rho, ctx->diag, gauss, rho_scale, energy);
}

int pic_diag_static(picpml_ctx* ctx, double* gauss, double* rho_scale, double* energy) {
  NvtxRange nvtx_("picpml pic_diag_static");
  int r = check_ready(ctx);
  if (r) return r;
  double* rho = nullptr;
  double* out = nullptr;
  long long cap = 0;
  CK(static_diag_buffers(&rho, &out, &cap));
  if (ctx->g.size > cap)
    return fail(ctx, PIC_EINVAL,
                "pic_diag_static: the grid needs " + std::to_string(ctx->g.size) +
                    " scratch nodes (x rows padded to 8); the static scratch holds " + std::to_string(cap));
  // the shared array keeps the last call's contents: diag_into clears what accumulates
  return diag_into(ctx, rho, out, gauss, rho_scale, energy);
}

int pic_state_size(picpml_ctx* ctx, long long* bytes) {
  int r = check_ready(ctx);
  if (r) return r;
  if (!bytes) return fail(ctx, PIC_EINVAL, "null argument");
  *bytes = (long long)ctx->g.size * (12 * ctx->elem() + 12 * 8);
  return PIC_OK;
}

}  // extern "C"

namespace {
template <typename T>
void state_arrays(picpml_ctx* ctx, FieldPtrs<T>& f, std::vector<std::pair<void*, size_t>>& v) {
  const size_t n = (size_t)ctx->g.size;
  for (int c = 0; c < 3; ++c) {
    v.push_back({f.E[c], n * sizeof(T)});
    v.push_back({f.Bh[c], n * sizeof(T)});
    v.push_back({f.Bp[c], n * sizeof(T)});
    v.push_back({f.J[c], n * sizeof(T)});
  }
  for (int c = 0; c < 3; ++c)
    for (int h = 0; h < 2; ++h) {
      v.push_back({f.Es[c][h], n * 8});
      v.push_back({f.Bs[c][h], n * 8});
    }
}
}  // namespace

extern "C" {

int pic_get_state(picpml_ctx* ctx, void* host_dst) {
  int r = check_ready(ctx);
  if (r) return r;
  if (!host_dst) return fail(ctx, PIC_EINVAL, "null argument");
  std::vector<std::pair<void*, size_t>> v;
  if (ctx->gd.prec == PIC_FP64) state_arrays(ctx, ctx->fd, v);
  else state_arrays(ctx, ctx->ff, v);
  char* q = (char*)host_dst;
  for (auto& a : v) {
    CK(cudaMemcpyAsync(q, a.first, a.second, cudaMemcpyDeviceToHost, ctx->stream));
    q += a.second;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return PIC_OK;
}

int pic_set_state(picpml_ctx* ctx, const void* host_src) {
  int r = check_ready(ctx);
  if (r) return r;
  if (!host_src) return fail(ctx, PIC_EINVAL, "null argument");
  std::vector<std::pair<void*, size_t>> v;
  if (ctx->gd.prec == PIC_FP64) state_arrays(ctx, ctx->fd, v);
  else state_arrays(ctx, ctx->ff, v);
  const char* q = (const char*)host_src;
  for (auto& a : v) {
    CK(cudaMemcpyAsync(a.first, q, a.second, cudaMemcpyHostToDevice, ctx->stream));
    q += a.second;
  }
  ctx->bn_stale = true;
  CK(cudaStreamSynchronize(ctx->stream));
  return PIC_OK;
}

const char* pic_last_error(picpml_ctx* ctx) { return ctx ? ctx->err.c_str() : g_init_error.c_str(); }

void pic_destroy(picpml_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (void* p : ctx->allocs) cudaFree(p);
  delete ctx;
}

}  // extern "C"
