/*
 * picpml_oracle.c -- plain, slow, FP64 CPU reference of the electromagnetic PIC
 * time step with the damped-current PML of Lehe et al. (arXiv:2201.09084).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle against which the CUDA
 * path is checked.  Only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py may load it.  It shares no code, header, table or
 * constant generator with the CUDA library, and the CUDA library never calls it.
 *
 * What it computes, in the paper's order and notation (one time step):
 *   1. gather E^n and B^n = (B^{n-1/2}+B^{n+1/2})/2 at each macroparticle with
 *      the same B-spline shape order as the deposit, at each component's
 *      staggered Yee location;
 *   2. Boris push u^{n-1/2} -> u^{n+1/2} (u = p/mc), then move
 *      x^{n+1} = x^n + dt c u/gamma; particles that leave the allowed region are
 *      removed and deposit nothing for this step (Sec. I: the standard scheme
 *      removes a particle as soon as it enters the PML);
 *   3. charge-conserving Esirkepov deposition of J^{n+1/2} (shape order 1 or 3;
 *      App. A cites Esirkepov's scheme);
 *   4. damping of the deposited current, J_c <- alpha_c J_c, with alpha taken at
 *      each component's staggered location (Eq. alpha, Sec. II.B);
 *   5. E^{n+1} = E^n + dt (c^2 curl B^{n+1/2} - J/eps0), then
 *      B^{n+3/2} = B^{n+1/2} - dt curl E^{n+1}, with the split-field PML of
 *      Eqs. MaxwellE, MaxwellB, MaxwellSum in every location where a damping
 *      conductivity is nonzero.
 *
 * Readings of points the paper leaves open:
 *   - B lives at half-integer times; the push uses the time average of the two
 *     B half steps that bracket t^n (the classic Yee/Boris leapfrog).
 *   - The split components with d/dt F = R - s F, s = sigma/eps0, advance by
 *     exponential differencing F <- e^{-s dt} F + (1 - e^{-s dt})/s R; the
 *     -alpha j/eps0 source sits inside R of one split (Sec. II.A leaves the time
 *     discretisation of the damping terms to "usual FDTD").
 *   - Every face can carry a PML: component c is split into c,d for the two
 *     axes d != c (Berenger); each split is damped by sigma_d.  The source
 *     alpha j_c goes to the split whose sigma is larger (ties: first axis in
 *     x,y,z order); for a pure z-PML this is exactly Eq. MaxwellE.  alpha is
 *     the product of the per-face alpha(depth) values.
 *   - The interface is the last physical node plane; sigma and alpha are
 *     evaluated at nodes and cell centres from their closed forms (Sec. II.B).
 *   - Outer termination: perfect conductor (tangential E = 0 on the last plane).
 *   - 2D is the (x,z) plane with d/dy = 0 (Sec. II.A, last paragraph); a 2D
 *     macroparticle is a line charge of length 1 m along y.
 *   - Removal: alpha = 0 mode removes at the physical-domain boundary; the
 *     other modes remove a particle once its shape support would reach the
 *     outer PML edge.
 *
 * Positions are absolute FP64, in cell units measured from the outer lower
 * corner of the whole grid (physical cells plus PML cells).
 *
 * Parity pins: see tests/test_oracle_*.py (alpha closed form and ODE, Fourier
 * ansatz condition, Yee cavity eigenmode frequency, split == unsplit for a
 * zero-conductivity PML, Esirkepov continuity and quadrature flux, Boris
 * rotation and E x B drift, Gauss law, boosted Coulomb field, PML attenuation,
 * superposition, exiting-particle error ordering).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_C 299792458.0
#define ORA_EPS0 8.8541878128e-12

/* Host threads of the particle and field loops (1 = the plain serial loops,
 * the default; the tests run that way).  With T > 1 the push and field loops
 * split their independent iterations over T threads, and the deposit gives
 * each thread its own current arrays for a contiguous share of the
 * particles, summed afterwards in thread order: the result is deterministic
 * for a given T and equals the serial one up to the summation order. */
static int g_threads = 1;

int ora_set_threads(int n) {
#ifdef _OPENMP
  if (n < 1) n = omp_get_num_procs();
  g_threads = n;
#else
  (void)n;
  g_threads = 1;
#endif
  return g_threads;
}

typedef struct ora_sim {
  int dim, order, alpha_mode, prescribed;
  int filter_passes;                /* binomial passes on J before each E update */
  int ck;                           /* 1: Cole-Karkkainen differences in Faraday's law */
  int face_mode[6];                 /* alpha mode of each face (-x,+x,-y,+y,-z,+z) */
  int n[3], plo[3], phi[3], N[3];   /* physical cells, PML cells low/high, total cells */
  long nn[3];                       /* nodes per axis in the arrays (1 for y in 2D) */
  long ntot;
  double d[3], dt;
  double sig_coef, delta, sig_exp, v_assumed;
  double *E[3], *Bh[3], *Bp[3], *J[3];   /* Bh = B^{n+1/2}, Bp = B^{n-1/2} */
  double *Es[3][2], *Bs[3][2];           /* split parts, for the two axes != c */
  double *s_node[3], *s_cent[3], *a_node[3], *a_cent[3];
  long np, cap;
  double *X[3], *X0[3], *u[3], *w, *q, *m;
  int *alive, *immobile, *moved;
  unsigned char* cond;              /* conductor cells (NULL: none), i + N0 (j + N1 k) */
  double* jt;                       /* per-thread current arrays of the threaded deposit */
  int jt_threads;
} ora_sim;

/* ------------------------------------------------------------------------- */
/* PML profiles: Eq. conductivity and Eq. alpha                              */
/* ------------------------------------------------------------------------- */

/* sigma/eps0 at depth dcells (cells) into a face: (coef c/Delta) (d/delta)^p,
 * Eq. conductivity with coef = 4, delta = 6 cells, p = 2. */
double ora_sigma_over_eps0(double dcells, double Delta, double coef, double delta,
                           double p) {
  if (dcells <= 0.0) return 0.0;
  return coef * ORA_C / Delta * pow(dcells / delta, p);
}

/* alpha(d) = exp(-int_0^d sigma/(eps0 v) dz'), Eq. alpha, integrated in closed
 * form for the power-law profile:  int_0^d (coef c/Delta)(z/delta)^p dz' (z in
 * metres, z = zc Delta) = coef c delta (d/delta)^{p+1}/(p+1) with d, delta in
 * cells.  mode 0: alpha = 0 inside the PML (Berenger, no source); mode 1:
 * alpha = 1 (undamped deposition); mode 2: Eq. alpha; mode 3: alpha = 1, the
 * macroparticle weights are damped instead (ora_weight_integral). */
double ora_alpha(double dcells, double coef, double delta, double p, double v,
                 int mode) {
  if (dcells <= 0.0) return 1.0;
  if (mode == 0) return 0.0;
  if (mode == 1 || mode == 3) return 1.0;
  double integral = coef * (ORA_C / v) * delta * pow(dcells / delta, p + 1.0) / (p + 1.0);
  return exp(-integral);
}

/* Depth (cells) of coordinate x beyond the physical box along axis a; the
 * interface is the last physical node plane, depth 0 inside (Sec. II.B). */
static double depth_of(const ora_sim* s, int a, double x) {
  double lo = (double)s->plo[a], hi = (double)(s->plo[a] + s->n[a]);
  if (x < lo) return lo - x;
  if (x > hi) return x - hi;
  return 0.0;
}

/* The face of axis a that position x lies beyond (its low face below the
 * physical box, else its high face). */
static int face_of(const ora_sim* s, int a, double x) {
  return x < (double)s->plo[a] ? 2 * a : 2 * a + 1;
}

/* Per-axis tables at nodes and cell centres: sigma/eps0 from
 * Eq. conductivity and alpha from Eq. alpha at each location's depth, with
 * the face's own alpha mode (Sec. II.B staggering: E and j_x, j_y at nodes,
 * B and j_z at centres along the damping axis). */
static void build_tables(ora_sim* s) {
  for (int a = 0; a < 3; ++a) {
    long nn = s->nn[a];
    s->s_node[a] = calloc(nn, sizeof(double));
    s->a_node[a] = calloc(nn, sizeof(double));
    s->s_cent[a] = calloc(nn, sizeof(double));
    s->a_cent[a] = calloc(nn, sizeof(double));
    int active = !(s->dim == 2 && a == 1);
    for (long i = 0; i < nn; ++i) {
      double dn = active ? depth_of(s, a, (double)i) : 0.0;
      double dc = active ? depth_of(s, a, (double)i + 0.5) : 0.0;
      s->s_node[a][i] = ora_sigma_over_eps0(dn, s->d[a], s->sig_coef, s->delta, s->sig_exp);
      s->s_cent[a][i] = ora_sigma_over_eps0(dc, s->d[a], s->sig_coef, s->delta, s->sig_exp);
      int fn = s->face_mode[face_of(s, a, (double)i)];
      int fc = s->face_mode[face_of(s, a, (double)i + 0.5)];
      s->a_node[a][i] = ora_alpha(dn, s->sig_coef, s->delta, s->sig_exp, s->v_assumed, fn);
      s->a_cent[a][i] = ora_alpha(dc, s->sig_coef, s->delta, s->sig_exp, s->v_assumed, fc);
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Construction                                                              */
/* ------------------------------------------------------------------------- */

ora_sim* ora_create(int dim, const int* nphys, const int* pml, const double* d,
                    double dt, int order, int alpha_mode, double sig_coef,
                    double delta, double sig_exp, double v_assumed) {
  if ((dim != 2 && dim != 3) || (order != 1 && order != 3)) return NULL;
  ora_sim* s = calloc(1, sizeof(ora_sim));
  s->dim = dim; s->order = order; s->alpha_mode = alpha_mode;
  for (int f = 0; f < 6; ++f) s->face_mode[f] = alpha_mode;
  s->dt = dt; s->sig_coef = sig_coef; s->delta = delta; s->sig_exp = sig_exp;
  s->v_assumed = v_assumed > 0 ? v_assumed : ORA_C;
  for (int a = 0; a < 3; ++a) {
    s->d[a] = d[a];
    if (dim == 2 && a == 1) { s->n[a] = 0; s->plo[a] = s->phi[a] = 0; }
    else { s->n[a] = nphys[a]; s->plo[a] = pml[2 * a]; s->phi[a] = pml[2 * a + 1]; }
    s->N[a] = s->n[a] + s->plo[a] + s->phi[a];
    s->nn[a] = s->N[a] + 1;
  }
  s->ntot = s->nn[0] * s->nn[1] * s->nn[2];
  for (int c = 0; c < 3; ++c) {
    s->E[c] = calloc(s->ntot, sizeof(double));
    s->Bh[c] = calloc(s->ntot, sizeof(double));
    s->Bp[c] = calloc(s->ntot, sizeof(double));
    s->J[c] = calloc(s->ntot, sizeof(double));
    for (int h = 0; h < 2; ++h) {
      s->Es[c][h] = calloc(s->ntot, sizeof(double));
      s->Bs[c][h] = calloc(s->ntot, sizeof(double));
    }
  }
  build_tables(s);
  return s;
}

void ora_destroy(ora_sim* s) {
  if (!s) return;
  for (int c = 0; c < 3; ++c) {
    free(s->E[c]); free(s->Bh[c]); free(s->Bp[c]); free(s->J[c]);
    for (int h = 0; h < 2; ++h) { free(s->Es[c][h]); free(s->Bs[c][h]); }
    free(s->s_node[c]); free(s->s_cent[c]); free(s->a_node[c]); free(s->a_cent[c]);
    free(s->X[c]); free(s->X0[c]); free(s->u[c]);
  }
  free(s->w); free(s->q); free(s->m); free(s->alive); free(s->immobile); free(s->moved);
  free(s->cond);
  free(s->jt);
  free(s);
}

void ora_set_prescribed(ora_sim* s, int flag) { s->prescribed = flag; }

/* Per-face deposition schemes (the paper's cavity discussion, Sec. III: the
 * undamped scheme on the face where particles enter, the damped one on the
 * face where they leave).  modes[f] in {0, 1, 2} (alpha = 0, 1 or Eq. alpha
 * inside face f) replaces the box's mode on that face: its alpha values and,
 * for mode 0, the removal of particles at that face's interface.  Weight
 * damping (mode 3) is a property of the macroparticles, not of a face: a box
 * in mode 3 takes no per-face modes.  Returns 0, or -1 (nothing changed). */
int ora_set_face_alpha(ora_sim* s, const int* modes) {
  if (s->alpha_mode == 3) return -1;
  for (int f = 0; f < 6; ++f)
    if (modes[f] < 0 || modes[f] > 2) return -1;
  for (int f = 0; f < 6; ++f) s->face_mode[f] = modes[f];
  for (int a = 0; a < 3; ++a) {
    free(s->s_node[a]); free(s->s_cent[a]); free(s->a_node[a]); free(s->a_cent[a]);
  }
  build_tables(s);
  return 0;
}

static inline long IX(const ora_sim* s, long i, long j, long k) {
  return i + s->nn[0] * (j + s->nn[1] * k);
}

/* Removal margin in cells from the outer edge: the Esirkepov stencil of a move
 * shorter than one cell then stays inside the node arrays. */
static double margin(const ora_sim* s) { return s->order == 1 ? 2.0 : 3.0; }

static int outside_allowed(const ora_sim* s, const double* X) {
  for (int a = 0; a < 3; ++a) {
    if (s->dim == 2 && a == 1) continue;
    if (s->face_mode[2 * a] == 0 && X[a] < (double)s->plo[a]) return 1;
    if (s->face_mode[2 * a + 1] == 0 && X[a] > (double)(s->plo[a] + s->n[a])) return 1;
    double m = margin(s);
    if (X[a] < m || X[a] > (double)s->N[a] - m) return 1;
  }
  return 0;
}

/* Adds n macroparticles of one species (charge q, mass m); positions in cell
 * units.  Returns the number of particles refused because they start outside
 * the allowed region (these are not added), or -1 on bad input. */
long ora_add_particles(ora_sim* s, long n, const double* X, const double* Y,
                       const double* Z, const double* ux, const double* uy,
                       const double* uz, const double* w, double q, double m,
                       int immobile) {
  if (n < 0) return -1;
  long need = s->np + n;
  if (need > s->cap) {
    long cap = need * 2 + 16;
    for (int a = 0; a < 3; ++a) {
      s->X[a] = realloc(s->X[a], cap * sizeof(double));
      s->X0[a] = realloc(s->X0[a], cap * sizeof(double));
      s->u[a] = realloc(s->u[a], cap * sizeof(double));
    }
    s->w = realloc(s->w, cap * sizeof(double));
    s->q = realloc(s->q, cap * sizeof(double));
    s->m = realloc(s->m, cap * sizeof(double));
    s->alive = realloc(s->alive, cap * sizeof(int));
    s->immobile = realloc(s->immobile, cap * sizeof(int));
    s->moved = realloc(s->moved, cap * sizeof(int));
    s->cap = cap;
  }
  long refused = 0;
  for (long i = 0; i < n; ++i) {
    long p = s->np;
    double P[3] = {X[i], s->dim == 3 ? Y[i] : 0.0, Z[i]};
    if (outside_allowed(s, P)) { ++refused; continue; }
    for (int a = 0; a < 3; ++a) { s->X[a][p] = P[a]; s->X0[a][p] = P[a]; }
    s->u[0][p] = ux[i]; s->u[1][p] = uy[i]; s->u[2][p] = uz[i];
    s->w[p] = w[i]; s->q[p] = q; s->m[p] = m;
    s->alive[p] = 1; s->immobile[p] = immobile; s->moved[p] = 0;
    s->np++;
  }
  return refused;
}

long ora_num_particles(const ora_sim* s) { return s->np; }

/* Copies particle state out: X,Y,Z (cell units), ux,uy,uz, alive. */
void ora_get_particles(const ora_sim* s, double* X, double* Y, double* Z,
                       double* ux, double* uy, double* uz, int* alive) {
  for (long p = 0; p < s->np; ++p) {
    X[p] = s->X[0][p]; Y[p] = s->X[1][p]; Z[p] = s->X[2][p];
    ux[p] = s->u[0][p]; uy[p] = s->u[1][p]; uz[p] = s->u[2][p];
    alive[p] = s->alive[p];
  }
}

void ora_get_weights(const ora_sim* s, double* w) {
  for (long p = 0; p < s->np; ++p) w[p] = s->w[p];
}

/* ------------------------------------------------------------------------- */
/* Shape factors (B-splines of order 1 and 3)                                */
/* ------------------------------------------------------------------------- */

/* Value of the centred B-spline of the given order at distance r (cells). */
double ora_shape(int order, double r) {
  double a = fabs(r);
  if (order == 1) return a < 1.0 ? 1.0 - a : 0.0;
  if (a < 1.0) return 2.0 / 3.0 - a * a + 0.5 * a * a * a;
  if (a < 2.0) { double b = 2.0 - a; return b * b * b / 6.0; }
  return 0.0;
}

/* Lowest node touched by the shape of a point at xi. */
static long shape_lo(int order, double xi) {
  return (long)floor(xi) - (order == 3 ? 1 : 0);
}
static int shape_width(int order) { return order + 1; }

/* ------------------------------------------------------------------------- */
/* Gather                                                                    */
/* ------------------------------------------------------------------------- */

/* Interpolates the node array F, staggered by (o0,o1,o2) half cells, at X. */
static double gather_one(const ora_sim* s, const double* F, const double* o,
                         const double* X) {
  int W = shape_width(s->order);
  long lo[3]; double wt[3][4];
  for (int a = 0; a < 3; ++a) {
    if (s->dim == 2 && a == 1) { lo[a] = 0; wt[a][0] = 1.0; continue; }
    double xi = X[a] - o[a];
    lo[a] = shape_lo(s->order, xi);
    for (int t = 0; t < W; ++t) wt[a][t] = ora_shape(s->order, xi - (double)(lo[a] + t));
  }
  int Wy = (s->dim == 2) ? 1 : W;
  double acc = 0.0;
  for (int tk = 0; tk < W; ++tk)
    for (int tj = 0; tj < Wy; ++tj)
      for (int ti = 0; ti < W; ++ti) {
        long i = lo[0] + ti, j = lo[1] + tj, k = lo[2] + tk;
        if (i < 0 || i >= s->nn[0] || j < 0 || j >= s->nn[1] || k < 0 || k >= s->nn[2]) continue;
        acc += wt[0][ti] * wt[1][tj] * wt[2][tk] * F[IX(s, i, j, k)];
      }
  return acc;
}

/* Staggering of each component in half cells: Ex(i+1/2,j,k), Ey(i,j+1/2,k),
 * Ez(i,j,k+1/2), Bx(i,j+1/2,k+1/2), By(i+1/2,j,k+1/2), Bz(i+1/2,j+1/2,k). */
static const double STAG_E[3][3] = {{0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 0.5}};
static const double STAG_B[3][3] = {{0, 0.5, 0.5}, {0.5, 0, 0.5}, {0.5, 0.5, 0}};

/* E^n and B^n = (B^{n-1/2} + B^{n+1/2})/2 at absolute position X (cells),
 * each component interpolated at its own staggered points with the
 * B-spline of the deposit's order (App. A shape order; energy-conserving
 * gather). */
void ora_gather(const ora_sim* s, const double* X, double* Eout, double* Bout) {
  for (int c = 0; c < 3; ++c) {
    Eout[c] = gather_one(s, s->E[c], STAG_E[c], X);
    Bout[c] = 0.5 * (gather_one(s, s->Bh[c], STAG_B[c], X) +
                     gather_one(s, s->Bp[c], STAG_B[c], X));
  }
}

/* ------------------------------------------------------------------------- */
/* Boris push                                                                */
/* ------------------------------------------------------------------------- */

/* Boris rotation for u = p/(mc): half electric kick, magnetic rotation, half
 * electric kick.  E in V/m, B in T. */
void ora_boris(double* u, const double* E, const double* B, double q, double m,
               double dt) {
  double ke = q * dt / (2.0 * m * ORA_C);
  double um[3], up[3], t[3], sv[3], uq[3];
  for (int a = 0; a < 3; ++a) um[a] = u[a] + ke * E[a];
  double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
  double kb = q * dt / (2.0 * m * gm);
  for (int a = 0; a < 3; ++a) t[a] = kb * B[a];
  double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  for (int a = 0; a < 3; ++a) sv[a] = 2.0 * t[a] / (1.0 + t2);
  /* u' = u- + u- x t */
  uq[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
  uq[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
  uq[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
  /* u+ = u- + u' x s */
  up[0] = um[0] + (uq[1] * sv[2] - uq[2] * sv[1]);
  up[1] = um[1] + (uq[2] * sv[0] - uq[0] * sv[2]);
  up[2] = um[2] + (uq[0] * sv[1] - uq[1] * sv[0]);
  for (int a = 0; a < 3; ++a) u[a] = up[a] + ke * E[a];
}

/* Gather + Boris + move + removal for every live particle. */
void ora_push(ora_sim* s) {
#pragma omp parallel for num_threads(g_threads) schedule(static) if (g_threads > 1)
  for (long p = 0; p < s->np; ++p) {
    s->moved[p] = 0;
    if (!s->alive[p]) continue;
    double X[3] = {s->X[0][p], s->X[1][p], s->X[2][p]};
    for (int a = 0; a < 3; ++a) s->X0[a][p] = X[a];
    if (s->immobile[p]) continue;
    double u[3] = {s->u[0][p], s->u[1][p], s->u[2][p]};
    if (!s->prescribed) {
      double E[3], B[3];
      ora_gather(s, X, E, B);
      ora_boris(u, E, B, s->q[p], s->m[p], s->dt);
    }
    double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double Xn[3];
    for (int a = 0; a < 3; ++a) {
      if (s->dim == 2 && a == 1) { Xn[a] = X[a]; continue; }
      Xn[a] = X[a] + s->dt * ORA_C * u[a] / (g * s->d[a]);
    }
    for (int a = 0; a < 3; ++a) s->u[a][p] = u[a];
    if (outside_allowed(s, Xn)) { s->alive[p] = 0; continue; }
    for (int a = 0; a < 3; ++a) s->X[a][p] = Xn[a];
    s->moved[p] = 1;
  }
}

/* ------------------------------------------------------------------------- */
/* Esirkepov deposition                                                      */
/* ------------------------------------------------------------------------- */

/* Shape values of the old (S0) and new (S1) positions on the common node range
 * lo .. lo+W-1 along one axis. */
static int esk_axis(int order, double x0, double x1, long* lo, double* S0, double* S1) {
  long l0 = shape_lo(order, x0), l1 = shape_lo(order, x1);
  long lmin = l0 < l1 ? l0 : l1, lmax = l0 > l1 ? l0 : l1;
  int W = (int)(lmax - lmin) + shape_width(order);
  *lo = lmin;
  for (int t = 0; t < W; ++t) {
    S0[t] = ora_shape(order, x0 - (double)(lmin + t));
    S1[t] = ora_shape(order, x1 - (double)(lmin + t));
  }
  return W;
}

/* Adds the current density of one macroparticle (charge qw) moving from X0 to
 * X1 (cell units, |X1-X0| < 1 per axis) during dt, to Jx, Jy, Jz (node arrays
 * with the Yee staggering).  3D: Esirkepov's density decomposition
 *   W_x = DSx (S0y S0z + DSy S0z/2 + S0y DSz/2 + DSy DSz/3)  (and cyclic),
 *   J_x(i+1/2) - J_x(i-1/2) = -(qw/(dy dz dt)) W_x(i).
 * 2D (x,z): W_x = DSx (S0z + DSz/2), W_z = DSz (S0x + DSx/2) with the same
 * prefix sums, and J_y = qw v_y (S0x S0z + DSx S0z/2 + S0x DSz/2 + DSx DSz/3)/V
 * for the out-of-plane component.  V uses a 1 m depth in 2D. */
static void esirkepov_into(const ora_sim* s, double* const* J, const double* X0, const double* X1, double qw,
                           double vy);

void ora_esirkepov(ora_sim* s, const double* X0, const double* X1, double qw,
                   double vy) {
  esirkepov_into(s, s->J, X0, X1, qw, vy);
}

/* ora_esirkepov adding into the arrays J[0..2] instead of the sim's own. */
static void esirkepov_into(const ora_sim* s, double* const* J, const double* X0, const double* X1, double qw,
                           double vy) {
  int order = s->order;
  long lo[3]; int W[3];
  double S0[3][6], S1[3][6], DS[3][6];
  for (int a = 0; a < 3; ++a) {
    if (s->dim == 2 && a == 1) { lo[a] = 0; W[a] = 1; S0[a][0] = S1[a][0] = 1.0; DS[a][0] = 0.0; continue; }
    W[a] = esk_axis(order, X0[a], X1[a], &lo[a], S0[a], S1[a]);
    for (int t = 0; t < W[a]; ++t) DS[a][t] = S1[a][t] - S0[a][t];
  }
  double dx = s->d[0], dy = s->d[1], dz = s->d[2], dt = s->dt;
  if (s->dim == 3) {
    double cx = -qw / (dy * dz * dt), cy = -qw / (dx * dz * dt), cz = -qw / (dx * dy * dt);
    /* J_x: prefix sum along x for every (j,k) line */
    for (int tk = 0; tk < W[2]; ++tk)
      for (int tj = 0; tj < W[1]; ++tj) {
        double T = S0[1][tj] * S0[2][tk] + 0.5 * DS[1][tj] * S0[2][tk] +
                   0.5 * S0[1][tj] * DS[2][tk] + DS[1][tj] * DS[2][tk] / 3.0;
        double acc = 0.0;
        for (int ti = 0; ti < W[0]; ++ti) {
          acc += DS[0][ti] * T;
          J[0][IX(s, lo[0] + ti, lo[1] + tj, lo[2] + tk)] += cx * acc;
        }
      }
    for (int tk = 0; tk < W[2]; ++tk)
      for (int ti = 0; ti < W[0]; ++ti) {
        double T = S0[0][ti] * S0[2][tk] + 0.5 * DS[0][ti] * S0[2][tk] +
                   0.5 * S0[0][ti] * DS[2][tk] + DS[0][ti] * DS[2][tk] / 3.0;
        double acc = 0.0;
        for (int tj = 0; tj < W[1]; ++tj) {
          acc += DS[1][tj] * T;
          J[1][IX(s, lo[0] + ti, lo[1] + tj, lo[2] + tk)] += cy * acc;
        }
      }
    for (int tj = 0; tj < W[1]; ++tj)
      for (int ti = 0; ti < W[0]; ++ti) {
        double T = S0[0][ti] * S0[1][tj] + 0.5 * DS[0][ti] * S0[1][tj] +
                   0.5 * S0[0][ti] * DS[1][tj] + DS[0][ti] * DS[1][tj] / 3.0;
        double acc = 0.0;
        for (int tk = 0; tk < W[2]; ++tk) {
          acc += DS[2][tk] * T;
          J[2][IX(s, lo[0] + ti, lo[1] + tj, lo[2] + tk)] += cz * acc;
        }
      }
  } else {
    double Ly = 1.0;
    double cx = -qw / (dz * Ly * dt), cz = -qw / (dx * Ly * dt);
    double cyy = qw * vy / (dx * dz * Ly);
    for (int tk = 0; tk < W[2]; ++tk) {
      double T = S0[2][tk] + 0.5 * DS[2][tk];
      double acc = 0.0;
      for (int ti = 0; ti < W[0]; ++ti) {
        acc += DS[0][ti] * T;
        J[0][IX(s, lo[0] + ti, 0, lo[2] + tk)] += cx * acc;
      }
    }
    for (int ti = 0; ti < W[0]; ++ti) {
      double T = S0[0][ti] + 0.5 * DS[0][ti];
      double acc = 0.0;
      for (int tk = 0; tk < W[2]; ++tk) {
        acc += DS[2][tk] * T;
        J[2][IX(s, lo[0] + ti, 0, lo[2] + tk)] += cz * acc;
      }
    }
    for (int tk = 0; tk < W[2]; ++tk)
      for (int ti = 0; ti < W[0]; ++ti) {
        double Wy = S0[0][ti] * S0[2][tk] + 0.5 * DS[0][ti] * S0[2][tk] +
                    0.5 * S0[0][ti] * DS[2][tk] + DS[0][ti] * DS[2][tk] / 3.0;
        J[1][IX(s, lo[0] + ti, 0, lo[2] + tk)] += cyy * Wy;
      }
  }
}

void ora_zero_J(ora_sim* s) {
  for (int c = 0; c < 3; ++c) memset(s->J[c], 0, s->ntot * sizeof(double));
}

/* Weight damping (alpha mode 3; the scheme of the paper's discussion of
 * limitations, Sec. II): alpha = 1 in the deposit and each macroparticle's
 * weight decays as w' = w exp(-int sigma(x(t'))/eps0 dt') along its own path,
 * so the damping matches every particle's actual velocity.  In corners and
 * edges the exponent is the sum over the faces (the product of the per-face
 * factors, as for alpha).  Over one step the integral is taken by the
 * trapezoid rule on the straight move:
 *   I = dt (s(X0) + s(X1)) / 2,  s(X) = sum_a sigma_a(depth_a(X)) / eps0,
 * sigma from Eq. conductivity at the particle's position.  The step's
 * current uses the mid-step weight w exp(-I/2); the weight then becomes
 * w exp(-I). */
double ora_weight_integral(const ora_sim* s, const double* X0, const double* X1) {
  double sum = 0.0;
  for (int a = 0; a < 3; ++a) {
    if (s->dim == 2 && a == 1) continue;
    sum += ora_sigma_over_eps0(depth_of(s, a, X0[a]), s->d[a], s->sig_coef, s->delta, s->sig_exp);
    sum += ora_sigma_over_eps0(depth_of(s, a, X1[a]), s->d[a], s->sig_coef, s->delta, s->sig_exp);
  }
  return 0.5 * s->dt * sum;
}

/* Step 3 of the time step: J^{n+1/2} of every particle moved by ora_push
 * (with weight damping: at the mid-step weight, then the weight decays). */
/* One particle's share of the deposit (with weight damping: at the
 * mid-step weight, then the weight decays). */
static void deposit_particle(ora_sim* s, double* const* J, long p) {
  double X0[3] = {s->X0[0][p], s->X0[1][p], s->X0[2][p]};
  double X1[3] = {s->X[0][p], s->X[1][p], s->X[2][p]};
  double g = sqrt(1.0 + s->u[0][p] * s->u[0][p] + s->u[1][p] * s->u[1][p] + s->u[2][p] * s->u[2][p]);
  double vy = ORA_C * s->u[1][p] / g;
  double wd = s->w[p];
  double I = 0.0;
  if (s->alpha_mode == 3) {
    I = ora_weight_integral(s, X0, X1);
    wd *= exp(-0.5 * I);
  }
  esirkepov_into(s, J, X0, X1, s->q[p] * wd, vy);
  if (s->alpha_mode == 3) s->w[p] *= exp(-I);
}

void ora_deposit_raw(ora_sim* s) {
  ora_zero_J(s);
  const int T = g_threads;
  if (T <= 1) {
    for (long p = 0; p < s->np; ++p)
      if (s->moved[p]) deposit_particle(s, s->J, p);
    return;
  }
  if (s->jt_threads != T) {
    free(s->jt);
    s->jt = (double*)malloc(sizeof(double) * 3 * (size_t)s->ntot * (size_t)T);
    s->jt_threads = s->jt ? T : 0;
    if (!s->jt) { /* no room for the per-thread arrays: the serial loop */
      for (long p = 0; p < s->np; ++p)
        if (s->moved[p]) deposit_particle(s, s->J, p);
      return;
    }
  }
#pragma omp parallel num_threads(T)
  {
#ifdef _OPENMP
    const int t = omp_get_thread_num();
#else
    const int t = 0;
#endif
    double* Jt[3];
    for (int c = 0; c < 3; ++c) {
      Jt[c] = s->jt + ((size_t)t * 3 + c) * (size_t)s->ntot;
      memset(Jt[c], 0, sizeof(double) * (size_t)s->ntot);
    }
    const long p0 = s->np * t / T, p1 = s->np * (t + 1) / T;
    for (long p = p0; p < p1; ++p)
      if (s->moved[p]) deposit_particle(s, Jt, p);
#pragma omp barrier
#pragma omp for schedule(static)
    for (long id = 0; id < s->ntot; ++id)
      for (int c = 0; c < 3; ++c) {
        double v = 0.0;
        for (int q = 0; q < T; ++q) v += s->jt[((size_t)q * 3 + c) * (size_t)s->ntot + id];
        s->J[c][id] = v;
      }
  }
}

/* Step 4: J_c <- alpha_c J_c at each component's staggered location. */
void ora_damp_J(ora_sim* s) {
#pragma omp parallel for num_threads(g_threads) schedule(static) if (g_threads > 1)
  for (long k = 0; k < s->nn[2]; ++k)
    for (long j = 0; j < s->nn[1]; ++j)
      for (long i = 0; i < s->nn[0]; ++i) {
        long id = IX(s, i, j, k);
        double ax_n = s->a_node[0][i], ay_n = s->a_node[1][j], az_n = s->a_node[2][k];
        double ax_c = s->a_cent[0][i], ay_c = s->a_cent[1][j], az_c = s->a_cent[2][k];
        if (s->dim == 2) { ay_n = 1.0; ay_c = 1.0; }
        s->J[0][id] *= ax_c * ay_n * az_n;
        s->J[1][id] *= ax_n * ay_c * az_n;
        s->J[2][id] *= ax_n * ay_n * az_c;
      }
}

/* Esirkepov deposit of every moving particle, then J_c <- alpha_c J_c at
 * each component's staggered location (App. A, Eq. alpha, Sec. II.B). */
void ora_deposit(ora_sim* s) { ora_deposit_raw(s); ora_damp_J(s); }

/* ------------------------------------------------------------------------- */
/* Field update: Yee leapfrog with the split-field PML                      */
/* ------------------------------------------------------------------------- */

/* Exponential differencing of d/dt F = R - s F over tau. */
static inline double ed_a(double s, double tau) { return exp(-s * tau); }
static inline double ed_b(double s, double tau) { return s > 0.0 ? -expm1(-s * tau) / s : tau; }

/* Advance one field location.  R[0], R[1] are the curl parts from the
 * derivatives along the two axes != c (in increasing axis order); sA, sB their
 * conductivities; src the source term (-alpha j/eps0 for E, 0 for B).  Returns
 * the new total. */
static double advance(double old, double* sp0, double* sp1, const double* R,
                      double sA, double sB, double src, double tau) {
  if (sA > 0.0 || sB > 0.0) {
    int into1 = sB > sA;
    *sp0 = ed_a(sA, tau) * (*sp0) + ed_b(sA, tau) * (R[0] + (into1 ? 0.0 : src));
    *sp1 = ed_a(sB, tau) * (*sp1) + ed_b(sB, tau) * (R[1] + (into1 ? src : 0.0));
    return *sp0 + *sp1;
  }
  return old + tau * (R[0] + R[1] + src);
}

/* E^{n+1} = E^n + dt (c^2 curl B^{n+1/2} - J/eps0)  (Eqs. MaxwellE, MaxwellSum). */
/* Binomial filter of the deposited current (App. A: the paper's runs smooth
 * the current with a binomial filter, after Birdsall and Langdon, before the
 * field update): one pass replaces every J value by
 * (J[i-1] + 2 J[i] + J[i+1])/4 along x, then along y (3D), then along z,
 * for each component at its own staggered points; values beyond the arrays
 * count as zero. */
void ora_filter_J(ora_sim* s) {
  double* tmp = malloc(s->ntot * sizeof(double));
  const long nn[3] = {s->nn[0], s->nn[1], s->nn[2]};
  for (int c = 0; c < 3; ++c)
    for (int a = 0; a < 3; ++a) {
      if (nn[a] < 2) continue;   /* the absent y axis of 2D boxes */
      for (long k = 0; k < nn[2]; ++k)
        for (long j = 0; j < nn[1]; ++j)
          for (long i = 0; i < nn[0]; ++i) {
            long x[3] = {i, j, k};
            double lo = 0.0, hi = 0.0;
            if (x[a] > 0) { x[a] -= 1; lo = s->J[c][IX(s, x[0], x[1], x[2])]; x[a] += 1; }
            if (x[a] < nn[a] - 1) { x[a] += 1; hi = s->J[c][IX(s, x[0], x[1], x[2])]; x[a] -= 1; }
            tmp[IX(s, i, j, k)] = 0.25 * lo + 0.5 * s->J[c][IX(s, i, j, k)] + 0.25 * hi;
          }
      memcpy(s->J[c], tmp, s->ntot * sizeof(double));
    }
  free(tmp);
}

/* Number of binomial passes applied to J at the start of each E update. */
void ora_set_filter(ora_sim* s, int passes) { s->filter_passes = passes > 0 ? passes : 0; }

/* Field solver: 0 = Yee, 1 = Cole-Karkkainen (the solver of the paper's
 * single-particle and LWFA runs, App. A).  The CK scheme (Cole 1997, 2002;
 * Karkkainen et al. 2006) keeps Yee's staggering and Ampere's law and
 * replaces each difference of E in Faraday's law by its average over the two
 * transverse axes with the weights (1/4, 1/2, 1/4) per axis.  The discrete
 * curl of a Fourier mode then carries, for the derivative along a, the factor
 * prod_{b != a} cos^2(k_b d_b / 2), which gives the dispersion relation
 *   sin^2(w dt/2) = (c dt)^2 sum_a sin^2(k_a d_a/2)/d_a^2 prod_{b!=a} cos^2(k_b d_b/2):
 * stable up to c dt = min d_a, and free of dispersion along an axis at
 * c dt = d_a (cubic cells: along every axis at c dt = d). */
void ora_set_solver(ora_sim* s, int ck) { s->ck = ck ? 1 : 0; }

/* E_c at index (i, j, k), continued beyond the grid by its images across the
 * conducting outer walls: odd across a wall the component is tangential to
 * (a node axis b != c: E(-m) = -E(m), E(N_b + m) = -E(N_b - m)), even across
 * a wall it is normal to (its own, centred axis: E(-1) = E(0),
 * E(N_c) = E(N_c - 1)).  The CK averages read these images next to the
 * walls; a PEC cavity eigenmode is then an exact discrete eigenmode. */
static double e_img(const ora_sim* s, int c, long i, long j, long k) {
  long x[3] = {i, j, k};
  double sign = 1.0;
  for (int b = 0; b < 3; ++b) {
    if (s->dim == 2 && b == 1) { x[1] = 0; continue; }
    const long N = s->N[b];
    if (b == c) {
      if (x[b] < 0) x[b] = -1 - x[b];
      else if (x[b] > N - 1) x[b] = 2 * N - 1 - x[b];
    } else {
      if (x[b] < 0) { x[b] = -x[b]; sign = -sign; }
      else if (x[b] > N) { x[b] = 2 * N - x[b]; sign = -sign; }
    }
  }
  return sign * s->E[c][IX(s, x[0], x[1], x[2])];
}

/* CK difference of E_c along axis a at the B location of index (i, j, k):
 * sum over p, q in {-1, 0, 1} of w_p w_q [E_c(n + e_a) - E_c(n)] with
 * n = (i, j, k) + p e_b + q e_d, (b, d) the two other axes, w = (1/4, 1/2,
 * 1/4); in 2D the y axis is not averaged. */
static double ck_diff(const ora_sim* s, int c, int a, long i, long j, long k) {
  static const double w[3] = {0.25, 0.5, 0.25};
  const int b = (a + 1) % 3, d = (a + 2) % 3;
  double acc = 0.0;
  for (int p = -1; p <= 1; ++p)
    for (int q = -1; q <= 1; ++q) {
      const int flat_b = s->dim == 2 && b == 1, flat_d = s->dim == 2 && d == 1;
      if ((flat_b && p != 0) || (flat_d && q != 0)) continue;
      const double wt = (flat_b ? 1.0 : w[p + 1]) * (flat_d ? 1.0 : w[q + 1]);
      long n0[3] = {i, j, k};
      n0[b] += p;
      n0[d] += q;
      long n1[3] = {n0[0], n0[1], n0[2]};
      n1[a] += 1;
      acc += wt * (e_img(s, c, n1[0], n1[1], n1[2]) - e_img(s, c, n0[0], n0[1], n0[2]));
    }
  return acc;
}

/* Zeroed-field cells (the cavity run of Sec. III has cells where E and B
 * are zero; the paper gives no geometry).  A marked cell is a perfect
 * conductor: every E component on its 12 edges is zero after each E update,
 * so E is tangentially zero on its faces and B inside it keeps its initial
 * value.  mask: one byte per cell of the whole grid (PML included), laid out
 * i + N0 (j + N1 k) (N1 = 1 in 2D); NULL removes all.  Returns 0. */
int ora_set_conductor(ora_sim* s, const unsigned char* mask) {
  free(s->cond);
  s->cond = NULL;
  if (!mask) return 0;
  const long N1 = s->dim == 3 ? s->N[1] : 1;
  const long nc = (long)s->N[0] * N1 * s->N[2];
  s->cond = malloc(nc);
  memcpy(s->cond, mask, nc);
  return 0;
}

static void zero_E(ora_sim* s, int c, long i, long j, long k) {
  const long id = IX(s, i, j, k);
  s->E[c][id] = 0.0;
  s->Es[c][0][id] = 0.0;
  s->Es[c][1][id] = 0.0;
}

static void apply_conductor(ora_sim* s) {
  const int d3 = s->dim == 3;
  const long N0 = s->N[0], N1 = d3 ? s->N[1] : 1, N2 = s->N[2];
  for (long k = 0; k < N2; ++k)
    for (long j = 0; j < N1; ++j)
      for (long i = 0; i < N0; ++i) {
        if (!s->cond[i + N0 * (j + N1 * k)]) continue;
        const long jt = d3 ? 1 : 0;   /* the y nodes of the cell: j, j + 1 (2D: 0) */
        for (long b = 0; b <= jt; ++b)
          for (long c = 0; c <= 1; ++c) zero_E(s, 0, i, j + b, k + c);       /* Ex(i+1/2, ., .) */
        for (long a = 0; a <= 1; ++a)
          for (long c = 0; c <= 1; ++c) zero_E(s, 1, i + a, j, k + c);       /* Ey(., j+1/2, .) */
        for (long a = 0; a <= 1; ++a)
          for (long b = 0; b <= jt; ++b) zero_E(s, 2, i + a, j + b, k);      /* Ez(., ., k+1/2) */
      }
}

/* E^{n+1} from E^n, B^{n+1/2} and the damped (and filtered) J^{n+1/2}
 * (Eqs. MaxwellE, MaxwellSum; split parts in PML cells, Sec. II.B), then the
 * conductor cells' edges set to zero. */
void ora_field_E(ora_sim* s) {
  for (int f = 0; f < s->filter_passes; ++f) ora_filter_J(s);
  const double c2 = ORA_C * ORA_C, dt = s->dt;
  const double dx = s->d[0], dy = s->d[1], dz = s->d[2];
  const int d3 = s->dim == 3;
  const long N0 = s->N[0], N1 = s->N[1], N2 = s->N[2];
  double *Bx = s->Bh[0], *By = s->Bh[1], *Bz = s->Bh[2];
  long j0 = d3 ? 1 : 0, j1 = d3 ? N1 - 1 : 0;
  /* Ex(i+1/2, j, k): splits (xy, xz) */
#pragma omp parallel for num_threads(g_threads) schedule(static) if (g_threads > 1)
  for (long k = 1; k <= N2 - 1; ++k)
    for (long j = j0; j <= j1; ++j)
      for (long i = 0; i <= N0 - 1; ++i) {
        long id = IX(s, i, j, k);
        double R[2];
        R[0] = d3 ? c2 * (Bz[id] - Bz[IX(s, i, j - 1, k)]) / dy : 0.0;
        R[1] = -c2 * (By[id] - By[IX(s, i, j, k - 1)]) / dz;
        double sA = d3 ? s->s_node[1][j] : 0.0, sB = s->s_node[2][k];
        s->E[0][id] = advance(s->E[0][id], &s->Es[0][0][id], &s->Es[0][1][id], R, sA, sB,
                              -s->J[0][id] / ORA_EPS0, dt);
      }
  /* Ey(i, j+1/2, k): splits (yx, yz) */
  long jy1 = d3 ? N1 - 1 : 0;
#pragma omp parallel for num_threads(g_threads) schedule(static) if (g_threads > 1)
  for (long k = 1; k <= N2 - 1; ++k)
    for (long j = 0; j <= jy1; ++j)
      for (long i = 1; i <= N0 - 1; ++i) {
        long id = IX(s, i, j, k);
        double R[2];
        R[0] = -c2 * (Bz[id] - Bz[IX(s, i - 1, j, k)]) / dx;
        R[1] = c2 * (Bx[id] - Bx[IX(s, i, j, k - 1)]) / dz;
        double sA = s->s_node[0][i], sB = s->s_node[2][k];
        s->E[1][id] = advance(s->E[1][id], &s->Es[1][0][id], &s->Es[1][1][id], R, sA, sB,
                              -s->J[1][id] / ORA_EPS0, dt);
      }
  /* Ez(i, j, k+1/2): splits (zx, zy) */
#pragma omp parallel for num_threads(g_threads) schedule(static) if (g_threads > 1)
  for (long k = 0; k <= N2 - 1; ++k)
    for (long j = j0; j <= j1; ++j)
      for (long i = 1; i <= N0 - 1; ++i) {
        long id = IX(s, i, j, k);
        double R[2];
        R[0] = c2 * (By[id] - By[IX(s, i - 1, j, k)]) / dx;
        R[1] = d3 ? -c2 * (Bx[id] - Bx[IX(s, i, j - 1, k)]) / dy : 0.0;
        double sA = s->s_node[0][i], sB = d3 ? s->s_node[1][j] : 0.0;
        s->E[2][id] = advance(s->E[2][id], &s->Es[2][0][id], &s->Es[2][1][id], R, sA, sB,
                              -s->J[2][id] / ORA_EPS0, dt);
      }
  if (s->cond) apply_conductor(s);
}

/* B^{n+3/2} = B^{n+1/2} - dt curl E^{n+1}  (Eqs. MaxwellB, MaxwellSum); with
 * the CK solver the differences of E are the transversely averaged ones of
 * ck_diff. */
void ora_field_B(ora_sim* s) {
  const double dt = s->dt;
  const int ck = s->ck;
  const double dx = s->d[0], dy = s->d[1], dz = s->d[2];
  const int d3 = s->dim == 3;
  const long N0 = s->N[0], N1 = s->N[1], N2 = s->N[2];
  double *Ex = s->E[0], *Ey = s->E[1], *Ez = s->E[2];
  long jc1 = d3 ? N1 - 1 : 0, jn1 = d3 ? N1 : 0;
  /* Bx(i, j+1/2, k+1/2): splits (xy, xz) */
#pragma omp parallel for num_threads(g_threads) schedule(static) if (g_threads > 1)
  for (long k = 0; k <= N2 - 1; ++k)
    for (long j = 0; j <= jc1; ++j)
      for (long i = 0; i <= N0; ++i) {
        long id = IX(s, i, j, k);
        double R[2];
        if (ck) {
          R[0] = d3 ? -ck_diff(s, 2, 1, i, j, k) / dy : 0.0;
          R[1] = ck_diff(s, 1, 2, i, j, k) / dz;
        } else {
          R[0] = d3 ? -(Ez[IX(s, i, j + 1, k)] - Ez[id]) / dy : 0.0;
          R[1] = (Ey[IX(s, i, j, k + 1)] - Ey[id]) / dz;
        }
        double sA = d3 ? s->s_cent[1][j] : 0.0, sB = s->s_cent[2][k];
        s->Bp[0][id] = advance(s->Bh[0][id], &s->Bs[0][0][id], &s->Bs[0][1][id], R, sA, sB, 0.0, dt);
      }
  /* By(i+1/2, j, k+1/2): splits (yx, yz) */
#pragma omp parallel for num_threads(g_threads) schedule(static) if (g_threads > 1)
  for (long k = 0; k <= N2 - 1; ++k)
    for (long j = 0; j <= jn1; ++j)
      for (long i = 0; i <= N0 - 1; ++i) {
        long id = IX(s, i, j, k);
        double R[2];
        if (ck) {
          R[0] = ck_diff(s, 2, 0, i, j, k) / dx;
          R[1] = -ck_diff(s, 0, 2, i, j, k) / dz;
        } else {
          R[0] = (Ez[IX(s, i + 1, j, k)] - Ez[id]) / dx;
          R[1] = -(Ex[IX(s, i, j, k + 1)] - Ex[id]) / dz;
        }
        double sA = s->s_cent[0][i], sB = s->s_cent[2][k];
        s->Bp[1][id] = advance(s->Bh[1][id], &s->Bs[1][0][id], &s->Bs[1][1][id], R, sA, sB, 0.0, dt);
      }
  /* Bz(i+1/2, j+1/2, k): splits (zx, zy) */
#pragma omp parallel for num_threads(g_threads) schedule(static) if (g_threads > 1)
  for (long k = 0; k <= N2; ++k)
    for (long j = 0; j <= jc1; ++j)
      for (long i = 0; i <= N0 - 1; ++i) {
        long id = IX(s, i, j, k);
        double R[2];
        if (ck) {
          R[0] = -ck_diff(s, 1, 0, i, j, k) / dx;
          R[1] = d3 ? ck_diff(s, 0, 1, i, j, k) / dy : 0.0;
        } else {
          R[0] = -(Ey[IX(s, i + 1, j, k)] - Ey[id]) / dx;
          R[1] = d3 ? (Ex[IX(s, i, j + 1, k)] - Ex[id]) / dy : 0.0;
        }
        double sA = s->s_cent[0][i], sB = d3 ? s->s_cent[1][j] : 0.0;
        s->Bp[2][id] = advance(s->Bh[2][id], &s->Bs[2][0][id], &s->Bs[2][1][id], R, sA, sB, 0.0, dt);
      }
  /* the freshly written array now holds B^{n+3/2}; the other one B^{n+1/2} */
  for (int c = 0; c < 3; ++c) { double* t = s->Bh[c]; s->Bh[c] = s->Bp[c]; s->Bp[c] = t; }
}

/* One full time step. */
void ora_step(ora_sim* s, int nsteps) {
  for (int n = 0; n < nsteps; ++n) {
    ora_push(s);
    ora_deposit(s);
    ora_field_E(s);
    ora_field_B(s);
  }
}

/* ------------------------------------------------------------------------- */
/* Field access and diagnostics                                              */
/* ------------------------------------------------------------------------- */

/* which: 0-2 E^n; 3-5 B^n = (B^{n-1/2}+B^{n+1/2})/2; 6-8 J (last deposit,
 * damped); 9-11 B^{n+1/2}; 12-14 B^{n-1/2}.  out holds ntot doubles laid out
 * i + nx (j + ny k) with nx = N0+1, ny = N1+1 (1 in 2D). */
int ora_get_field(const ora_sim* s, int which, double* out) {
  int c = which % 3;
  for (long t = 0; t < s->ntot; ++t) {
    switch (which / 3) {
      case 0: out[t] = s->E[c][t]; break;
      case 1: out[t] = 0.5 * (s->Bh[c][t] + s->Bp[c][t]); break;
      case 2: out[t] = s->J[c][t]; break;
      case 3: out[t] = s->Bh[c][t]; break;
      case 4: out[t] = s->Bp[c][t]; break;
      default: return -1;
    }
  }
  return 0;
}

/* Sets E^n (which 0-2), the current J (6-8), B^{n+1/2} (9-11) or B^{n-1/2}
 * (12-14).  Splits at a split location take the whole value in their first
 * part. */
int ora_set_field(ora_sim* s, int which, const double* in) {
  int c = which % 3;
  double* dst;
  double** sp;
  switch (which / 3) {
    case 0: dst = s->E[c]; sp = s->Es[c]; break;
    case 2: dst = s->J[c]; sp = NULL; break;
    case 3: dst = s->Bh[c]; sp = s->Bs[c]; break;
    case 4: dst = s->Bp[c]; sp = NULL; break;
    default: return -1;
  }
  for (long t = 0; t < s->ntot; ++t) {
    dst[t] = in[t];
    if (sp) { sp[0][t] = in[t]; sp[1][t] = 0.0; }
  }
  return 0;
}

/* Charge density at the nodes: rho = sum q w S(X-i) S(Y-j) S(Z-k) / V. */
void ora_rho(const ora_sim* s, double* rho) {
  memset(rho, 0, s->ntot * sizeof(double));
  double V = s->d[0] * s->d[2] * (s->dim == 3 ? s->d[1] : 1.0);
  int W = shape_width(s->order);
  for (long p = 0; p < s->np; ++p) {
    if (!s->alive[p]) continue;
    long lo[3]; double wt[3][4];
    for (int a = 0; a < 3; ++a) {
      if (s->dim == 2 && a == 1) { lo[a] = 0; wt[a][0] = 1.0; continue; }
      lo[a] = shape_lo(s->order, s->X[a][p]);
      for (int t = 0; t < W; ++t) wt[a][t] = ora_shape(s->order, s->X[a][p] - (double)(lo[a] + t));
    }
    int Wy = s->dim == 2 ? 1 : W;
    for (int tk = 0; tk < W; ++tk)
      for (int tj = 0; tj < Wy; ++tj)
        for (int ti = 0; ti < W; ++ti)
          rho[IX(s, lo[0] + ti, lo[1] + tj, lo[2] + tk)] +=
              s->q[p] * s->w[p] * wt[0][ti] * wt[1][tj] * wt[2][tk] / V;
  }
}

/* Discrete divergence of E at the nodes (zero on the outer node planes). */
void ora_divE(const ora_sim* s, double* div) {
  memset(div, 0, s->ntot * sizeof(double));
  const int d3 = s->dim == 3;
  long j0 = d3 ? 1 : 0, j1 = d3 ? s->N[1] - 1 : 0;
  for (long k = 1; k <= s->N[2] - 1; ++k)
    for (long j = j0; j <= j1; ++j)
      for (long i = 1; i <= s->N[0] - 1; ++i) {
        long id = IX(s, i, j, k);
        double v = (s->E[0][id] - s->E[0][IX(s, i - 1, j, k)]) / s->d[0] +
                   (s->E[2][id] - s->E[2][IX(s, i, j, k - 1)]) / s->d[2];
        if (d3) v += (s->E[1][id] - s->E[1][IX(s, i, j - 1, k)]) / s->d[1];
        div[id] = v;
      }
}

/* Table access for tests: which 0 s_node, 1 s_cent, 2 a_node, 3 a_cent. */
void ora_get_table(const ora_sim* s, int which, int axis, double* out) {
  const double* src = which == 0 ? s->s_node[axis] : which == 1 ? s->s_cent[axis]
                    : which == 2 ? s->a_node[axis] : s->a_cent[axis];
  memcpy(out, src, s->nn[axis] * sizeof(double));
}

void ora_dims(const ora_sim* s, long* nn) { nn[0] = s->nn[0]; nn[1] = s->nn[1]; nn[2] = s->nn[2]; }

/* ------------------------------------------------------------------------- */
/* Deterministic (int64 fixed-point) deposition, 3D                         */
/* ------------------------------------------------------------------------- */
/* The deterministic mode takes its only floating-point decisions per
 * particle, in a fixed order, so the integers it adds are independent of the
 * order in which particles reach the grid:
 *   1. the B-spline shape values of the old and new offsets, in FP32 with the
 *      operation order below (this file is compiled without contraction), are
 *      quantised S_int = rint(S * 2^20), except one node per axis that takes
 *      2^20 minus the others (the node at offset f for order 1, the second
 *      node for order 3), so every quantised shape sums to 2^20 exactly and
 *      the decomposition conserves the integer charge exactly;
 *   2. Esirkepov's decomposition (the charge-conserving W of Esirkepov 2001,
 *      App. A) is then exact integer arithmetic.  Scaled by 6 so the 1/2 and
 *      1/3 weights stay integral, for the x component
 *        6 W_x = DSx (6 S0y S0z + 3 DSy S0z + 3 S0y DSz + 2 DSy DSz),
 *      and acc_x(i) = sum_{i' <= i} 6 W_x(i') (likewise y, z), in units of
 *      2^-60 of the macroparticle's charge; sum_c 6 W_c = 6 (S1 S1 S1 - S0 S0 S0)
 *      holds exactly;
 *   3. each nonzero acc becomes one integer contribution in units of
 *      e / (6 * 2^24) per cell face: with the particle's integer charge factor
 *        Wq = rint( (double(w) * qn) * 2^28 ),
 *      qn = q / e (the charge in units of the elementary charge),
 *        val = floor( (acc * Wq + 2^63) / 2^64 ),
 *      i.e. acc * w q/e * 2^-36 rounded to the nearest integer (halves up),
 *      formed exactly in 128-bit integer arithmetic; the sum over particles
 *      is exact.
 * The physical current is J_x = -(e / (dy dz dt)) val_x / (6 * 2^24) before
 * the PML damping (likewise for y, z).  raw != 0 skips step 3 and adds acc
 * itself (for the continuity check; weights and qn are ignored).
 * Moves: cell0/cell1 (i, j, k) and FP32 offsets off0/off1 in [0,1) per axis,
 * three per particle; the cell changes by at most one per axis.  Output:
 * int64 sums (+=) in the node layout i + nx (j + ny k); nodes outside the
 * arrays are skipped. */

#define FIX_QB 20
#define FIX_WQB 28

/* round(acc * Wq / 2^s), halves up, exactly (|acc| < 2^63, |Wq| <= 2^60). */
static long long fix_scale(long long acc, long long Wq, int s) {
  const __int128 P = (__int128)acc * (__int128)Wq + ((__int128)1 << (s - 1));
  return (long long)(P >> s);
}

/* The particle's integer charge factor rint(w q/e 2^28). */
static long long fix_wq(float w, double qn) { return llrint(ldexp((double)w * qn, FIX_WQB)); }

/* B-spline shape values of an in-cell offset f, computed in FP32 and
 * quantised to 2^-20 with the remainder on one node so the values sum to
 * 2^20 exactly (order 1: 2 nodes, order 3: 4 nodes). */
static void fixed_shape(int order, float f, long long* w) {
  const float scale = (float)(1 << FIX_QB);
  const long long one = 1LL << FIX_QB;
  if (order == 1) {
    w[1] = (long long)nearbyintf(f * scale);
    w[0] = one - w[1];
    return;
  }
  const float g = 1.0f - f;
  const float sixth = (float)(1.0 / 6.0), twothird = (float)(2.0 / 3.0);
  const float s0 = ((g * g) * g) * sixth;
  const float s2 = (twothird - (g * g)) + (((0.5f * g) * g) * g);
  const float s3 = ((f * f) * f) * sixth;
  w[0] = (long long)nearbyintf(s0 * scale);
  w[2] = (long long)nearbyintf(s2 * scale);
  w[3] = (long long)nearbyintf(s3 * scale);
  w[1] = one - w[0] - w[2] - w[3];
}

/* Old shape S0 and change DS on the order+2 nodes starting at
 * min(c0, c1) - (order == 3); returns that first node. */
static int fixed_axis(int order, int c0, float f0, int c1, float f1, long long* S0, long long* DS) {
  const int b = c0 < c1 ? c0 : c1;
  long long w0[4], w1[4], S1[5] = {0, 0, 0, 0, 0};
  fixed_shape(order, f0, w0);
  fixed_shape(order, f1, w1);
  for (int t = 0; t < order + 2; ++t) S0[t] = 0;
  for (int t = 0; t <= order; ++t) {
    S0[c0 - b + t] = w0[t];
    S1[c1 - b + t] = w1[t];
  }
  for (int t = 0; t < order + 2; ++t) DS[t] = S1[t] - S0[t];
  return b - (order == 3 ? 1 : 0);
}

void ora_fixed_deposit3d(int order, long long n, const int* cell0, const float* off0, const int* cell1,
                         const float* off1, const float* w, double qn, int raw, long long nx, long long ny,
                         long long nz, long long* Jx, long long* Jy, long long* Jz) {
  const int W = order + 2;
  for (long long p = 0; p < n; ++p) {
    long long S0[3][5], DS[3][5];
    int lo[3];
    for (int a = 0; a < 3; ++a)
      lo[a] = fixed_axis(order, cell0[3 * p + a], off0[3 * p + a], cell1[3 * p + a], off1[3 * p + a], S0[a], DS[a]);
    const long long Wq = fix_wq(w[p], qn);
    for (int c = 0; c < 3; ++c) {
      /* component c: prefix sums along axis c; the two transverse axes b < d */
      const int b = c == 0 ? 1 : 0, d = c == 2 ? 1 : 2;
      long long* J = c == 0 ? Jx : (c == 1 ? Jy : Jz);
      for (int tb = 0; tb < W; ++tb)
        for (int td = 0; td < W; ++td) {
          const long long T = 6 * S0[b][tb] * S0[d][td] + 3 * DS[b][tb] * S0[d][td] +
                              3 * S0[b][tb] * DS[d][td] + 2 * DS[b][tb] * DS[d][td];
          long long acc = 0;
          for (int ta = 0; ta < W - 1; ++ta) {
            acc += DS[c][ta] * T;
            if (acc == 0) continue;
            long long idx[3];
            idx[c] = lo[c] + ta;
            idx[b] = lo[b] + tb;
            idx[d] = lo[d] + td;
            if (idx[0] < 0 || idx[0] >= nx || idx[1] < 0 || idx[1] >= ny || idx[2] < 0 || idx[2] >= nz) continue;
            const long long v = raw ? acc : fix_scale(acc, Wq, 36 + FIX_WQB);
            J[idx[0] + nx * (idx[1] + ny * idx[2])] += v;
          }
        }
    }
  }
}

/* The replay for 2D (x, z) boxes (d/dy = 0).  J_x and J_z come from the
 * integer Esirkepov sums of the two in-plane axes, 6 W_x = DS_x (6 S0_z +
 * 3 DS_z) (prefix sums along x; likewise z), in units 2^-40, so one rounding
 * val = floor((acc Wq + 2^43) / 2^44) (acc w q/e 2^-16 to the nearest integer, halves up;
 * Wq as in the 3D replay) gives the unit of the 3D replay, e/(6 2^24).
 * J_y (out of the plane) is the mid-move shape product 6 S0_x S0_z +
 * 3 DS_x S0_z + 3 S0_x DS_z + 2 DS_x DS_z times v_y/c, which is formed in
 * FP64 from the FP32 momentum with correctly rounded operations in a fixed
 * order, v_y/c = u_y / sqrt(((1 + u_x^2) + u_y^2) + u_z^2), and rounded once:
 * val = rint(((T w q/e) v_y/c) 2^-16).  u: 3 floats per particle.  Arrays
 * are laid out i + nx k.  raw = 1 stores the unrounded integers (J_y without
 * the weight and velocity). */
void ora_fixed_deposit2d(int order, long long n, const int* cell0, const float* off0, const int* cell1,
                         const float* off1, const float* w, const float* u, double qn, int raw, long long nx,
                         long long nz, long long* Jx, long long* Jy, long long* Jz) {
  const int W = order + 2;
  const double down = ldexp(1.0, -16);
  for (long long p = 0; p < n; ++p) {
    long long S0[3][5], DS[3][5];
    int lo[3] = {0, 0, 0};
    for (int a = 0; a < 3; a += 2)
      lo[a] = fixed_axis(order, cell0[3 * p + a], off0[3 * p + a], cell1[3 * p + a], off1[3 * p + a], S0[a], DS[a]);
    const double wq = (double)w[p] * qn;
    const long long Wq = fix_wq(w[p], qn);
    const double ux = u[3 * p], uy = u[3 * p + 1], uz = u[3 * p + 2];
    const double vyc = uy / sqrt(((1.0 + ux * ux) + uy * uy) + uz * uz);
    for (int tk = 0; tk < W; ++tk) {        /* J_x: prefix sums along x */
      const long long T = 6 * S0[2][tk] + 3 * DS[2][tk];
      long long acc = 0;
      for (int ti = 0; ti < W - 1; ++ti) {
        acc += DS[0][ti] * T;
        const long long i = lo[0] + ti, k = lo[2] + tk;
        if (acc == 0 || i < 0 || i >= nx || k < 0 || k >= nz) continue;
        Jx[i + nx * k] += raw ? acc : fix_scale(acc, Wq, 16 + FIX_WQB);
      }
    }
    for (int ti = 0; ti < W; ++ti) {        /* J_z: prefix sums along z */
      const long long T = 6 * S0[0][ti] + 3 * DS[0][ti];
      long long acc = 0;
      for (int tk = 0; tk < W - 1; ++tk) {
        acc += DS[2][tk] * T;
        const long long i = lo[0] + ti, k = lo[2] + tk;
        if (acc == 0 || i < 0 || i >= nx || k < 0 || k >= nz) continue;
        Jz[i + nx * k] += raw ? acc : fix_scale(acc, Wq, 16 + FIX_WQB);
      }
    }
    for (int tk = 0; tk < W; ++tk)          /* J_y: mid-move shape product */
      for (int ti = 0; ti < W; ++ti) {
        const long long T = 6 * S0[0][ti] * S0[2][tk] + 3 * DS[0][ti] * S0[2][tk] + 3 * S0[0][ti] * DS[2][tk] +
                            2 * DS[0][ti] * DS[2][tk];
        const long long i = lo[0] + ti, k = lo[2] + tk;
        if (T == 0 || i < 0 || i >= nx || k < 0 || k >= nz) continue;
        Jy[i + nx * k] += raw ? T : llrint((((double)T * wq) * vyc) * down);
      }
  }
}

/* Integer node charge of 2D boxes, 6 S_int,x S_int,z (units 2^-40). */
void ora_fixed_rho2d(int order, long long n, const int* cell, const float* off, long long nx, long long nz,
                     long long* rho) {
  const int lo = order == 3 ? 1 : 0;
  for (long long p = 0; p < n; ++p) {
    long long w[3][4];
    fixed_shape(order, off[3 * p], w[0]);
    fixed_shape(order, off[3 * p + 2], w[2]);
    for (int tk = 0; tk <= order; ++tk)
      for (int ti = 0; ti <= order; ++ti) {
        const long long i = cell[3 * p] - lo + ti, k = cell[3 * p + 2] - lo + tk;
        if (i < 0 || i >= nx || k < 0 || k >= nz) continue;
        rho[i + nx * k] += 6 * w[0][ti] * w[2][tk];
      }
  }
}

/* Integer node charge 6 S_int,x S_int,y S_int,z (units 2^-60 of the particle
 * charge): the quantity whose change the raw integer currents carry exactly. */
void ora_fixed_rho3d(int order, long long n, const int* cell, const float* off, long long nx, long long ny,
                     long long nz, long long* rho) {
  const int lo = order == 3 ? 1 : 0;
  for (long long p = 0; p < n; ++p) {
    long long w[3][4];
    for (int a = 0; a < 3; ++a) fixed_shape(order, off[3 * p + a], w[a]);
    for (int tk = 0; tk <= order; ++tk)
      for (int tj = 0; tj <= order; ++tj)
        for (int ti = 0; ti <= order; ++ti) {
          const long long i = cell[3 * p] - lo + ti, j = cell[3 * p + 1] - lo + tj, k = cell[3 * p + 2] - lo + tk;
          if (i < 0 || i >= nx || j < 0 || j >= ny || k < 0 || k >= nz) continue;
          rho[i + nx * (j + ny * k)] += 6 * w[0][ti] * w[1][tj] * w[2][tk];
        }
  }
}
