/*
 * picpml.h -- C ABI of the GB300 (sm_103a) electromagnetic PIC step with the
 * damped-current perfectly matched layer of Lehe et al., "Absorption of
 * charged particles in Perfectly-Matched-Layers by optimal damping of the
 * deposited current" (arXiv:2201.09084).
 *
 * One time step (Sec. II.A-B of the paper, App. A for the scheme choices):
 *   gather E^n, B^n at each macroparticle (B-spline shape of order 1 or 3),
 *   Boris push u^{n-1/2} -> u^{n+1/2} and move x^n -> x^{n+1},
 *   charge-conserving Esirkepov deposition of J^{n+1/2},
 *   damping of the current deposited in PML cells, J_c <- alpha_c J_c, with
 *     alpha(z) = exp(-int_0^z sigma/(eps0 v) dz')              (Eq. alpha)
 *     evaluated at each component's staggered Yee location (Sec. II.B),
 *   Yee update E^{n+1} = E^n + dt (c^2 curl B^{n+1/2} - J/eps0) and
 *     B^{n+3/2} = B^{n+1/2} - dt curl E^{n+1}, with the split-field PML of
 *     Eqs. MaxwellE, MaxwellB, MaxwellSum in cells where sigma > 0.
 *
 * Conventions for every entry point:
 *   - Returns a pic_status (0 = success, < 0 = error); nothing is thrown
 *     across the ABI.  pic_last_error(ctx) gives a one-line message.
 *   - Work is enqueued on the context's CUDA stream (given at pic_init) and is
 *     asynchronous unless stated.  Device-side faults of the method (a particle
 *     outside the grid, a fixed-point overflow) set a status word that is
 *     reported by pic_sync() and pic_diag().
 *   - Memory: particle arrays are CALLER-owned device memory registered with
 *     pic_add_species and must outlive the context; fields, PML split
 *     components, coefficient tables and scratch are LIBRARY-owned (allocated
 *     at pml_init / pic_add_species, freed by pic_destroy).
 *   - Units: SI (metres, seconds, V/m, tesla, A/m^2, coulomb, kilogram).
 *     Momenta are u = p/(m c).  Positions are an int32 cell index plus an
 *     in-cell offset in [0,1) per axis, in units of the cell size.
 *   - 2D runs are the (x,z) plane with d/dy = 0 (Sec. II.A, last paragraph);
 *     a 2D macroparticle is a line charge 1 m long along y.
 */
#ifndef PICPML_H
#define PICPML_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct picpml_ctx picpml_ctx; /* opaque, library-owned */

typedef enum {
  PIC_OK = 0,
  PIC_EINVAL = -1,      /* bad argument or description */
  PIC_ENOMEM = -2,      /* device allocation failed */
  PIC_ECUDA = -3,       /* a CUDA runtime call failed */
  PIC_ECFL = -4,        /* dt above the Yee Courant limit */
  PIC_EOVERFLOW = -5,   /* fixed-point current accumulator overflow, or an
                           injection past a species' capacity */
  PIC_ETIMEOUT = -6,    /* a bounded device wait gave up: the tile kernel
                           (PIC_TUNING_TILE) waits at most 2 s for the TMA
                           copy of a field box, then stops and reports this
                           at pic_sync */
  PIC_ENOTIMPL = -7,    /* combination not built (reserved: pic_init takes
                           every dim, order, precision and alpha mode; the
                           batch API takes FP32 and FP64 and answers
                           PIC_EINVAL to the fixed-point mode) */
  PIC_ESTATE = -8,      /* call out of order (e.g. push before pml_init) */
  PIC_EPARTICLE = -9    /* a particle record was invalid (outside its allowed
                           cells, an offset outside [0,1), or a momentum or
                           weight that is not finite); it was removed before
                           it touched the fields */
} pic_status;

typedef enum {
  PIC_FP32 = 0,         /* FP32 fields, momenta and offsets; PML split parts
                           as float-float pairs, or IEEE FP64 with
                           pic_grid_desc.split_fp64 = 1 */
  PIC_FP64 = 1,         /* everything FP64 (the plain FP64 form) */
  PIC_FP32_FIXED64 = 2  /* as PIC_FP32, current accumulated in int64 fixed
                           point: deterministic, bit-identical J (3D and 2D;
                           see pic_get_current_fixed) */
} pic_prec;

typedef enum {
  PML_ALPHA_ZERO = 0,   /* alpha = 0 in the PML: Berenger's PML, particles
                           removed on entering it (Sec. I, Eq. MaxwellE) */
  PML_ALPHA_ONE = 1,    /* alpha = 1: undamped deposition in the PML */
  PML_ALPHA_DAMPED = 2, /* alpha of Eq. alpha (the paper's scheme) */
  PML_ALPHA_WEIGHT = 3  /* alpha = 1 in the deposit; instead each
                           macroparticle's weight decays as
                           w exp(-int sigma(x(t))/eps0 dt) along its own path
                           (the alternative scheme of the paper's discussion
                           of limitations, Sec. II): per step the trapezoid
                           rule I = dt (s(x^n) + s(x^{n+1}))/2, s summed over
                           the faces; the step's current uses w exp(-I/2) and
                           the stored weight becomes w exp(-I) */
} pml_alpha_mode;

/* Field solvers (pic_grid_desc.solver). */
typedef enum {
  PIC_SOLVER_YEE = 0,   /* Yee leapfrog; Courant limit 1/(c sqrt(sum 1/d_i^2)) */
  PIC_SOLVER_CK = 1     /* Cole-Karkkainen (the solver of the paper's
                           single-particle and LWFA runs, App. A; Cole
                           1997/2002, Karkkainen et al. 2006): Faraday's law
                           takes every difference of E averaged over the two
                           transverse axes with weights (1/4, 1/2, 1/4) per
                           axis (images across the conducting outer walls:
                           odd for a tangential component, even for a normal
                           one); Ampere's law is Yee's.  Courant limit
                           min(d_i)/c; no numerical dispersion along an axis
                           at c dt = d on cubic cells */
} pic_solver;

/* Grid description.  n[] counts PHYSICAL cells (the PML cells of pml_desc
 * are added outside them); n[1] is ignored in 2D.  dt <= 0 selects
 * cfl * (the solver's Courant limit). */
typedef struct pic_grid_desc {
  int dim;              /* 2 or 3 */
  int n[3];             /* physical cells per axis */
  double d[3];          /* cell sizes (m) */
  double dt;            /* time step (s), or <= 0 for cfl * Courant limit */
  double cfl;           /* used when dt <= 0, e.g. 0.99 */
  int shape_order;      /* 1 (linear) or 3 (cubic spline), App. A */
  int prec;             /* pic_prec */
  int sort_every;       /* step_n sorts particles by cell every this many
                           steps (0 = never) */
  int split_fp64;       /* PIC_FP32 only: 1 = PML split parts in IEEE FP64
                           (each step's increment formed in FP32 from its
                           FP32 inputs, added with one FP64 FMA);
                           0 (default) = float-float pairs (hi + lo, ~48-bit
                           significand, 8 bytes) computed on the FP32 pipes */
  int filter_passes;    /* 0 (default): none.  n = 1..8: field_step first
                           filters the deposited current n times with the
                           binomial (1, 2, 1)/4 stencil along each axis (App.
                           A; values beyond the node arrays count as zero);
                           the field then conserves the filtered charge */
  int solver;           /* pic_solver: PIC_SOLVER_YEE (0, default) or
                           PIC_SOLVER_CK */
} pic_grid_desc;

/* PML description: conductivity sigma(d) = coef eps0 c / Delta (d/delta)^p at
 * depth d into a face (Eq. conductivity: coef 4, delta 6 cells, p 2).  alpha
 * in a corner is the product of the faces' alpha values. */
typedef struct pml_desc {
  int ncell[6];         /* PML cells on the -x,+x,-y,+y,-z,+z faces */
  double sigma_max_coef;/* coef */
  double delta_cells;   /* delta, in cells */
  double exponent;      /* p */
  int alpha_mode;       /* pml_alpha_mode */
  double v_assumed;     /* v of Eq. alpha (m/s); <= 0 selects c */
  int face_alpha_set;   /* 0: every face uses alpha_mode.  1: face f uses
                           face_alpha[f] instead (PML_ALPHA_ZERO, _ONE or
                           _DAMPED; the paper's cavity discussion, Sec. III,
                           suggests the undamped scheme on the face where
                           particles enter and the damped one where they
                           leave).  A face in PML_ALPHA_ZERO removes particles
                           at its own interface only.  PIC_EINVAL for another
                           mode, or with alpha_mode PML_ALPHA_WEIGHT (weight
                           damping belongs to the particles, not a face). */
  int face_alpha[6];    /* per-face modes, -x,+x,-y,+y,-z,+z */
} pml_desc;

/* A species: caller-owned device arrays of `capacity` particles, n of them
 * live.  PIC_FP32 / PIC_FP32_FIXED64: pos = float4 (ox, oy, oz, w), mom =
 * float4 (ux, uy, uz, cell) where cell is an int32 stored in the float's
 * bits: i | j << 10 | k << 20 (i, j < 1024, k < 2048; -1 = removed).
 * PIC_FP64: the same fields as four doubles each (cell as int64 bits).
 * q, m: charge and mass of one physical particle; w is the macroparticle
 * weight. */
typedef struct pic_species {
  void* pos;
  void* mom;
  long long n;
  long long capacity;
  double q;
  double m;
  int immobile;         /* 1: never pushed (e.g. the motionless partner of
                           App. A); deposits no current */
} pic_species;

/* Creates a context on the current CUDA device.  stream: a cudaStream_t (NULL
 * = legacy default stream).  Validates the description (PIC_EINVAL, PIC_ECFL)
 * and allocates nothing on the device yet. */
int pic_init(picpml_ctx** ctx, const pic_grid_desc* grid, void* stream);

/* Builds the sigma / alpha / exponential-differencing tables per axis at
 * nodes and cell centres (Eq. conductivity, Eq. alpha; Sec. II.B: closed
 * forms evaluated at the staggered points) and allocates the fields (zeroed).
 * Must be called once, after pic_init.  A PML of 0 cells on a face gives a
 * perfectly conducting wall there. */
int pml_init(picpml_ctx* ctx, const pml_desc* pml);

/* Registers caller-owned particle arrays (see pic_species); returns the
 * species id in *sid.  The library allocates per-species scratch (the
 * positions saved by push() for a later deposit()). */
int pic_add_species(picpml_ctx* ctx, const pic_species* sp, int* sid);

/* Gather + Boris push + move of every live particle of every species; a
 * particle whose new position leaves the allowed region is removed (cell set
 * to -1): at the physical-domain boundary in PML_ALPHA_ZERO mode (Sec. I),
 * else once its shape would reach the outer PML edge.  Saves x^n for
 * deposit(). */
int push(picpml_ctx* ctx);

/* Esirkepov deposition of J^{n+1/2} from the positions saved by push() to the
 * current ones, with the PML damping alpha_c applied in the flush to the grid
 * (Eq. MaxwellE source term, Eq. alpha).  Accumulates into J, which the next
 * field_step() consumes and zeroes. */
int deposit(picpml_ctx* ctx);

/* Sets x^n, the positions deposit() moves from (what push() saves), for a
 * species: src is a caller-owned device buffer of `capacity` records, float4
 * (ox, oy, oz, cell bits) (PIC_FP64: four doubles, cell as int64 bits; a cell
 * of -1 deposits nothing).  With it, deposit() deposits any prescribed moves
 * from src to the species' current positions (each move shorter than one
 * cell per axis). */
int pic_set_old_positions(picpml_ctx* ctx, int sid, const void* src);

/* PIC_FP32_FIXED64 only (else PIC_ESTATE): copies the int64 current sums of
 * the last deposit() / push_deposit() / step into dst (caller-owned device
 * buffer of nx*ny*nz int64, index i + nx (j + ny k)), before the PML damping.
 * Deterministic mode, per particle and in a fixed operation order:
 *   shape values of the old and new offsets (B-spline of Sec. II.A's PIC,
 *   order 1 or 3) in FP32, quantised to 2^-20, one node per axis taking the
 *   remainder so every shape sums to 1 exactly;
 *   Esirkepov's decomposition (App. A) in exact integers, scaled by 6:
 *   6 W_x = DSx (6 S0y S0z + 3 DSy S0z + 3 S0y DSz + 2 DSy DSz), prefix sums
 *   along x (y, z likewise), so continuity holds exactly in integers;
 *   per node one rounding, rint(acc * (w q/e) * 2^-36), added with int64
 *   atomics (order-independent).
 * Units: one integer is e / (6 * 2^24) of charge crossing the component's
 * cell face, i.e. J_x = -(e / (dy dz dt)) Jq_x / (6 * 2^24) in A/m^2 before
 * damping.  The deposit then writes J = alpha_c * that (Eq. alpha) over the
 * whole grid (replacing, not adding to, J).  2D boxes: J_x and J_z from the
 * in-plane sums 6 W_x = DSx (6 S0z + 3 DSz), rounded as rint(acc (w q/e)
 * 2^-16) (the same unit, with faces 1 m long along y); J_y from the
 * mid-move shape product 6 S0x S0z + 3 DSx S0z + 3 S0x DSz + 2 DSx DSz times
 * v_y/c, formed in FP64 from the FP32 momentum with correctly rounded
 * operations, u_y / sqrt(((1 + u_x^2) + u_y^2) + u_z^2), rounded as
 * rint(((T (w q/e)) v_y/c) 2^-16): one integer is e c / (6 2^24 dx dz) of
 * J_y.  Limits: |w q/e| <= 2^32 per particle and |Jq| <= 2^62 per node, else
 * PIC_EOVERFLOW at pic_sync. */
int pic_get_current_fixed(picpml_ctx* ctx, int comp, long long* dst);

/* Field update: E^{n+1} = E^n + dt (c^2 curl B^{n+1/2} - J/eps0), then
 * B^{n+3/2} = B^{n+1/2} - dt curl E^{n+1} (with PIC_SOLVER_CK the curl of E
 * takes the Cole-Karkkainen differences); split-field PML components in
 * every location with sigma > 0 (Eqs. MaxwellE, MaxwellB, MaxwellSum), their
 * parts in IEEE FP64 (PIC_FP64, or PIC_FP32 with split_fp64 = 1) or as
 * float-float pairs (PIC_FP32 by default).  Consumes and zeroes J. */
int field_step(picpml_ctx* ctx);

/* The particle half of a time step in one fused kernel per species: gather,
 * Boris push, move (+ removal), Esirkepov deposition and the alpha-damped
 * flush into J.  step_n() is push_deposit() followed by field_step(). */
int push_deposit(picpml_ctx* ctx);

/* n full time steps: fused gather/push/move/deposit/damp kernel per species,
 * then field_step; particles are sorted by cell every sort_every steps. */
int step_n(picpml_ctx* ctx, int n);

/* Sorts every species by cell (counting sort on a tile-major key: 8x4x4-cell
 * tiles in 3D, 4x4 in 2D, then the cell inside the tile, x fastest; the
 * order within a cell is not kept) and drops removed particles; the live
 * count is updated on the device.  In 3D it also records where each tile's
 * particles end, the work ranges of the tile kernel (PIC_TUNING_TILE). */
int pic_sort(picpml_ctx* ctx);

/* Node counts of the field arrays (nx, ny, nz): N+1 per axis (ny = 1 in 2D),
 * N = physical + PML cells. */
int pic_grid_info(picpml_ctx* ctx, int* nn3, double* dt);

/* Copies one field component into dst (caller-owned device buffer of
 * nx*ny*nz elements, index i + nx (j + ny k)), as double if as_double else
 * float.  which: 0-2 E^n; 3-5 B^n = (B^{n-1/2}+B^{n+1/2})/2; 6-8 the last
 * deposited current (damped, A/m^2; zero after field_step); 9-11 B^{n+1/2};
 * 12-14 B^{n-1/2}.  SI units. */
int pic_get_field(picpml_ctx* ctx, int which, void* dst, int as_double);

/* Sets one field component from src (same layout as pic_get_field).  which:
 * 0-2 E^n, 9-11 B^{n+1/2}, 12-14 B^{n-1/2}.  At a split PML location the
 * whole value goes into the first split part. */
int pic_set_field(picpml_ctx* ctx, int which, const void* src, int as_double);

/* Zeroed-field (perfect conductor) cells, e.g. the walls of the cavity run
 * of Sec. III (the paper zeroes the fields in some cells and gives no
 * geometry): mask is a host array of N0*N1*N2 bytes over the cells of the
 * whole grid (physical + PML; N1 = 1 in 2D), index i + N0 (j + N1 k), nonzero
 * for a conductor cell.  After every E update of field_step the E components
 * on the 12 edges of each marked cell (8 in 2D) are zero, with their split
 * parts, so E is tangentially zero on the cell's faces.  Particles are not
 * stopped by conductor cells; the caller keeps them out.  NULL removes the
 * conductor.  Copies the cell list to the device (allocating when it grows)
 * and synchronises the stream. */
int pic_set_conductor(picpml_ctx* ctx, const unsigned char* mask);

/* 1: particles keep their momentum (no gather/push; they still move and
 * deposit), for prescribed-trajectory studies. */
int pic_set_prescribed(picpml_ctx* ctx, int flag);

/* Live particle count of a species (synchronises the stream). */
int pic_num_particles(picpml_ctx* ctx, int sid, long long* n);

/* Appends `count` particles to species sid, between steps: pos and mom are
 * device arrays of `count` records in the species' layout (as in
 * pic_species, same alignment), copied after the species' live particles.
 * This is the continuous injection of a beam through a face (Sec. III: the
 * cavity beam is injected on one side and absorbed on the other; particles
 * may start inside the entry face's PML).  The live count is read and
 * advanced on the device, so the call does not synchronise; the caller keeps
 * pos/mom valid until the stream has run the copy.  Records beyond the
 * capacity are dropped and pic_sync then reports PIC_EOVERFLOW.  Particles
 * outside their allowed cells are removed at the next push and reported like
 * any other (PIC_EPARTICLE).  PIC_EINVAL for a bad species id, count < 0 or
 * misaligned arrays. */
int pic_inject(picpml_ctx* ctx, int sid, const void* pos, const void* mom, long long count);

/* Diagnostics (synchronise the stream).  gauss: max |div E - rho/eps0| over
 * nodes at least one cell inside the physical region, in V/m^2; rho_scale:
 * max |rho/eps0| there; energy: field energy integral of
 * (eps0 E^2 + B^2/mu0)/2 over the whole grid (J per m in 2D). */
int pic_diag(picpml_ctx* ctx, double* gauss, double* rho_scale, double* energy);

/* Autotuner: times the fused particle kernel for each particles-per-thread
 * choice (order 1, and order 3 in 3D: 1, 4, 8; FP64: 1, 4) over `steps`
 * whole steps (the field step runs between them, untimed, so the particles
 * see evolving fields), and the field kernels for each z-nodes-per-thread
 * choice, each candidate from the same state (a device snapshot, restored
 * afterwards; the call allocates that snapshot), keeps the fastest and
 * returns the choices.  Results do not depend on the choice beyond the
 * summation order of the current. */
int pic_autotune(picpml_ctx* ctx, int steps, int* particles_per_thread, int* z_nodes_per_thread);

/* Sets the launch shapes directly (e.g. the result of pic_autotune in
 * another context).  Particles per thread (order 1; order 3 in 3D): 4 or 8
 * = the shared-memory chunk kernel with that many particles per thread
 * (dense particles), 1 = one thread per particle with global atomics (a few
 * particles per cell), 0 = default (4; FP64 uses 4 for 8), PIC_TUNING_TILE
 * = the tile-resident kernel: 3D PIC_FP32 boxes of shape order 1 only (else
 * the default), one launch for every species sorted since it was added
 * (pic_sort or sort_every; the others run one thread per particle): a block
 * per 16x4x4-cell unit loads the unit's E and B box with TMA, pushes the
 * particles that sat in the unit at the last sort, keeps the current of
 * moves inside a cell in two register runs per thread and queues moves
 * across a face per warp, and adds both to J with global reductions, damped
 * by alpha (a thermal plasma's few particles per cell and short moves).  z
 * nodes per thread of the field kernels: 1, 2 or 4. */
#define PIC_TUNING_TILE 2
int pic_set_tuning(picpml_ctx* ctx, int particles_per_thread, int z_nodes_per_thread);

/* Particle-steps done so far: the number of live particles each push has
 * moved, summed over all pushes since pml_init (synchronises the stream). */
int pic_particle_steps(picpml_ctx* ctx, long long* n);

/* Number of CUDA kernels this context has launched so far. */
int pic_launch_count(picpml_ctx* ctx, long long* n);

/* Same results as pic_diag, but allocates no device memory, ever.  The paper
 * has no counterpart: this serves callers that cannot allocate when they ask
 * for a diagnostic -- a host whose device memory belongs to a pool
 * allocator, a real-time loop that must not pay for or fail on an
 * allocation.  pic_diag allocates its charge-density scratch on first use;
 * this variant uses a file-scope device array of 8,388,608 doubles (64 MiB)
 * that every GPU loading the library holds until the process exits.  Grids
 * whose padded node count (x rows padded to 8) exceeds that return
 * PIC_EINVAL.  The first call on a device looks up the array's device
 * address; make that first call before any stream capture.  All calls share
 * the array (each call clears it first): calls that overlap on the GPU race
 * and their results are undefined.  Like pic_diag it reads the results back
 * and synchronises the stream. */
int pic_diag_static(picpml_ctx* ctx, double* gauss, double* rho_scale, double* energy);

/* Waits for the stream and reports any device-side status word. */
int pic_sync(picpml_ctx* ctx);

/* Checkpoint: bytes needed for the field state (fields, both B half steps,
 * PML split parts); copy it to / from caller-owned host memory.  Particles
 * are caller-owned and saved by the caller. */
int pic_state_size(picpml_ctx* ctx, long long* bytes);
int pic_get_state(picpml_ctx* ctx, void* host_dst);
int pic_set_state(picpml_ctx* ctx, const void* host_src);

/* ------------------------------------------------------------------------ */
/* Batched independent 2D runs (the single-particle studies of Sec. III,    */
/* swept over incidence angle and gamma): one persistent kernel launch per  */
/* step advances every run; launches are replayed from a captured CUDA      */
/* graph.  Runs share the cell size, time step, shape order, precision and  */
/* PML profile; each has its own physical size, PML width (on its four      */
/* faces) and one macroparticle.                                            */
/* ------------------------------------------------------------------------ */
typedef struct pic_batch pic_batch; /* opaque, library-owned */

typedef struct pic_batch_desc {
  int nruns;
  const int* nx;        /* host arrays of nruns entries: physical cells along x, */
  const int* nz;        /*   along z,                                             */
  const int* npml;      /*   PML cells on each of the run's four faces            */
  double d[2];          /* cell sizes dx, dz (m), shared by all runs */
  double dt;            /* s; <= 0 selects cfl * Courant limit */
  double cfl;
  int shape_order;      /* 1 or 3 */
  int prec;             /* PIC_FP32 (float-float PML parts) or PIC_FP64 */
  pml_desc pml;         /* profile and alpha mode (ncell is ignored) */
  double q, m;          /* charge and mass of the macroparticles */
  void* pos;            /* caller-owned device arrays of nruns particle */
  void* mom;            /*   records (layout of pic_species); record r lives in
                           run r, its cell index relative to run r's grid */
} pic_batch_desc;

/* Validates the description, builds per-run coefficient tables (Eq.
 * conductivity, Eq. alpha at nodes and centres), allocates and zeroes the
 * fields of every run, autotunes the kernel's block shape by timing a few
 * steps of every candidate from the initial state (then restored), and
 * records the two-step CUDA graph.  The first
 * call on a device must not happen while that stream is being captured. */
int pic_batch_init(pic_batch** b, const pic_batch_desc* d, void* stream);
/* n time steps of every run (graph replay; one kernel launch per step). */
int pic_batch_step(pic_batch* b, int n);
/* One field component of one run into dst (device buffer of
 * (nx+2p+1)*(nz+2p+1) elements, i fastest); which: 0-2 E^n, 3-5 B^n,
 * 6-8 the current not yet consumed (zero after a step).  SI units. */
int pic_batch_get_field(pic_batch* b, int run, int which, void* dst, int as_double);
/* 1: particles keep their momentum (prescribed trajectories). */
int pic_batch_set_prescribed(pic_batch* b, int flag);
/* Live particles pushed so far, summed over steps (synchronises). */
int pic_batch_particle_steps(pic_batch* b, long long* n);
/* Block shape the batch autotuner chose at pic_batch_init (threads per
 * block, minimum resident blocks per SM) and the measured ms per step of the
 * ncand candidates (threads, min blocks) = (512,1), (256,2), (512,2),
 * (1024,1), (256,6), (256,8), (256,3). */
int pic_batch_tuning(pic_batch* b, int* threads, int* min_blocks, float* ms_per_step, int ncand);
/* dt in use and the total number of cells of all runs. */
int pic_batch_info(pic_batch* b, double* dt, long long* cells);
int pic_batch_sync(pic_batch* b);
const char* pic_batch_last_error(pic_batch* b);
void pic_batch_destroy(pic_batch* b);

/* Last error message of this context (or of the last failed pic_init when
 * ctx is NULL).  Valid until the next call on the context. */
const char* pic_last_error(picpml_ctx* ctx);

/* Frees all library-owned device memory; does not touch particle arrays. */
void pic_destroy(picpml_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PICPML_H */
