/*
 * s2.h -- C ABI of the GB300 STREAmS-2 solver (libs2.so).
 *
 * The library advances the 3-D compressible Navier-Stokes equations of an
 * ideal gas, calorically or thermally perfect, on a Cartesian grid,
 * stretched in y, with
 * the method of the paper's Sec. 2 ("Numerical Methods"): hybrid
 * convective discretisation (energy-preserving split-form central flux of
 * 6th order; at interfaces flagged by a modified Ducros shock sensor, a
 * WENO5/WENO7 reconstruction of characteristic fluxes with Lax-Friedrichs
 * splitting, projected on the right eigenvectors), 6th-order viscous terms
 * in Laplacian form, and a third-order low-storage Runge-Kutta scheme.
 * The call sequence follows the program flow of Sec. 3.1 (create grid,
 * metrics, gas, boundaries -> initialise -> time loop) and the single
 * host-to-device copy of the initial field before the loop (Sec. 3.2,
 * Listing 3); afterwards the state stays resident on the GPU.
 *
 * Units: reference density, velocity, temperature and length are 1; the
 * gas constant is R = 1/(gamma mach_ref^2), p = rho R T,
 * E = e(T) + |u|^2/2, mu = (T/t_ref)^visc_exp / re_ref; e(T) = c_v T with
 * c_v = R/(gamma-1) for a calorically perfect gas (s2_gas below gives the
 * thermally perfect e(T)).
 *
 * State layout across the ABI: w[v][k][j][i], v = 0..4 = (rho, rho u,
 * rho v, rho w, rho E), interior points only, i (x) fastest: 5*nx*ny*nz
 * doubles, the order of the paper's (x, y, z, v) device array (Sec. 3.2,
 * Listing 2) without its ghost layers.
 *
 * Errors: every int-returning call returns S2_OK (0) or a negative code;
 * s2_strerror names it.  Handles are not thread-safe; each solver issues
 * its work on one CUDA stream (s2_stream_states adds two copy streams of
 * its own, synchronised before it returns).  No call allocates device memory except
 * s2_create (which allocates everything up front), s2_batch_create (its
 * work-list tables) and the first s2_stream_states (its staging buffers).
 */
#ifndef S2_H
#define S2_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define S2_OK 0
#define S2_EINVAL -1      /* bad argument or unsupported configuration */
#define S2_ENOMEM -2      /* device or host allocation failed */
#define S2_ECUDA -3       /* a CUDA runtime call failed */
#define S2_ENONFINITE -4  /* non-positive density/temperature or NaN met */
#define S2_ETIMEOUT -5    /* a bounded device wait gave up */
#define S2_EBUSY -6       /* solver busy (reserved) */
#define S2_ETOOBIG -7     /* larger than the fixed scratch of s2_cfl_dt_noalloc */
#define S2_EBOUNDS -8     /* an index left its array (bounds-checked build libs2_checked.so only) */

#define S2_BC_PERIODIC 0
#define S2_BC_ISOTHERMAL_WALL 1

#define S2_HOST 0
#define S2_DEVICE 1

#define S2_FP64 0   /* all arithmetic and storage in double precision */
#define S2_MIXED 1  /* single-precision primitives, flux, WENO and viscous arithmetic;
                       double-precision state, RK accumulation and E -> T recovery */

typedef struct s2_solver s2_solver; /* opaque; owned by the library */

/* Interior points and box size.  x in [0, lx), z in [0, lz) are periodic;
 * y spans ly (periodic, or walls at y = -ly/2 and +ly/2). */
typedef struct {
  int nx, ny, nz;
  double lx, ly, lz;
} s2_grid;

/* Node ordinates in y (Sec. 3.1: the Grid object evaluates the metrics).
 * y: host pointer to ny increasing values, read during s2_create only;
 * NULL = uniform nodes y_j = -ly/2 + (j + 1/2) ly/ny.  With walls the
 * nodes lie strictly inside (-ly/2, ly/2) and the walls sit half way
 * between the outermost node and its mirror image.  The library derives
 * eta_y = 1/y_eta and eta_yy from the 6th-order stencil. */
typedef struct {
  const double *y;
} s2_metrics;

/* Gas (Sec. 2: ideal gas, calorically or thermally perfect).  re_ref <= 0
 * = inviscid.  gamma (with mach_ref) fixes the gas constant R.
 *
 * cp_coeffs: NULL for a calorically perfect gas (c_p = gamma R/(gamma-1)).
 * Otherwise a thermally perfect gas whose specific heat follows the NASA
 * Glenn 9-coefficient polynomial (Sec. 2: "NASA polynomials", McBride et
 * al. 2002): host pointer to 7 doubles a_{-2}, a_{-1}, a_0, ..., a_4 with
 * c_p(T)/R = sum_l a_l T^l, T in reference units (scale dimensional
 * coefficients by T_ref^l).  Read during the call only.  The internal
 * energy is the antiderivative of c_v = c_p - R with zero constant,
 * e(T)/R = -a_{-2}/T + a_{-1} ln T + (a_0 - 1) T + a_1 T^2/2 + a_2 T^3/3
 * + a_3 T^4/4 + a_4 T^5/5 (the calorically perfect e when only a_0 is
 * set); states passed in and out use this e.  T follows from e by Newton's
 * method, the sound speed is sqrt(gamma(T) R T) with gamma(T) = c_p/c_v,
 * the conductivity mu c_p(T)/Pr.  The coefficients must be finite and
 * give c_v > 0 at T = 1, at t_ref and at the wall temperature (else
 * S2_EINVAL); c_v must stay
 * positive over the temperatures the flow visits (an inversion that
 * fails to converge is reported as S2_ENONFINITE). */
typedef struct {
  double gamma, prandtl, mach_ref, re_ref, visc_exp, t_ref;
  const double *cp_coeffs;
} s2_gas;

/* Boundaries: x and z must be S2_BC_PERIODIC; y periodic or isothermal
 * no-slip walls at temperature t_wall.  force_mass_flow = 1 adds the
 * uniform x body force that keeps the bulk rho*u constant (force_rhs_1 of
 * Table 2). */
typedef struct {
  int x, y, z;
  double t_wall;
  int force_mass_flow;
} s2_bcs;

/* Scheme (paper Sec. 2: central schemes up to 8th order, WENO up to 7th).
 * central_order: 2, 4, 6 or 8 for the central convective flux;
 * visc_order: 2, 4, 6 or 8 for the viscous terms and the sensor's
 * derivatives (the y metric uses the higher of the two).  weno_order: 0
 * (central everywhere), 1, 3, 5 or 7.  An interface is WENO iff the sensor's maximum over
 * its stencil exceeds sensor_threshold (strictly).  precision: S2_FP64 or
 * S2_MIXED (the sensor then decides in single precision).
 * dt: if cfl > 0 it is recomputed from the CFL condition (compute_dt of
 * Table 2) at every step whose counter is a multiple of dt_every and
 * frozen within a step; otherwise dt_fixed is used.
 * keep: the central flux (Sec. 2).  0: the energy-preserving split form
 * (Pirozzoli 2010), two-point flux {rho}{u_n}{phi} with phi = 1, u, v, w,
 * H.  n >= 1: KEEP-n, the kinetic-energy and entropy preserving flux of
 * the same flux-differencing form with the two-point flux
 * <rho>{u_n} (1, {u}, c_v/<1/T> + (u_a . u_b)/2) plus the pressure terms
 * {p} n and (p_a u_n,b + p_b u_n,a)/2 ({.} arithmetic, <.> logarithmic
 * means), its logarithmic means from the first n terms of their series in
 * (a-b)/(a+b) (entropy error of order ((a-b)/(a+b))^2n per pair); -1:
 * the same with exact logarithmic means (entropy conserved to rounding in
 * smooth inviscid flow).  KEEP needs a calorically perfect gas (else
 * S2_EINVAL).  A field at the end of the struct: code that zero-fills or
 * omits it gets the split form. */
typedef struct {
  int central_order, weno_order, visc_order;
  double sensor_threshold;
  int precision;
  double cfl, dt_fixed;
  int dt_every;
  int keep;
} s2_scheme;

/* Device options.  alloc/free: optional allocator callbacks (device
 * memory, blocks aligned to at least 256 bytes as cudaMalloc's are;
 * s2_create fails with S2_EINVAL otherwise), both NULL =
 * cudaMalloc/cudaFree.  stream: a cudaStream_t or
 * NULL for the legacy default stream.  device: CUDA ordinal, or -1 for
 * the current device. */
typedef struct {
  void *(*alloc)(size_t bytes, void *ctx);
  void (*free)(void *ptr, void *ctx);
  void *ctx;
  void *stream;
  int device;
} s2_device;

/* Monitoring (paper Sec. 3.2 residual, Listings 7-8; Table 2 reductions).
 * Volume integrals use dV = dx dz / eta_y. */
typedef struct {
  double t;             /* simulated time */
  long long step;       /* completed RK3 steps */
  double dt;            /* current time step */
  double mass;          /* integral of rho */
  double mom[3];        /* integrals of rho u, rho v, rho w */
  double energy;        /* integral of rho E */
  double kinetic;       /* integral of rho |u|^2 / 2 */
  double residual_rhou; /* sqrt(mean(R_rhou^2)) of the last RHS evaluation */
  double weno_frac;     /* flagged interfaces / (3 N) in the last RHS evaluation */
  double forcing;       /* body force of the last RHS evaluation */
  long long launches;   /* kernels launched by s2_step so far (all graph nodes that are kernels) */
  int status;           /* S2_OK or the first error met on the device */
} s2_stats_t;

/* Create a solver; allocates all device memory (state, RK register, RHS,
 * primitive and auxiliary fields with ghost layers) and computes the
 * metrics.  dev may be NULL.  On success *out owns the solver; release it
 * with s2_destroy.  S2_EINVAL for unsupported settings, and for grids with
 * (nx+1)(ny+1)(nz+1) > 2^31 - 1 (point and interface indices are split
 * in 32-bit arithmetic; such a grid would not fit in device memory). */
int s2_create(const s2_grid *grid, const s2_metrics *metrics, const s2_gas *gas, const s2_bcs *bcs,
              const s2_scheme *scheme, const s2_device *dev, s2_solver **out);

/* Copy a state in (layout above).  where = S2_HOST: w is host memory
 * (pageable or pinned); S2_DEVICE: w is device memory on the solver's
 * device.  The caller keeps ownership; the copy is complete when the call
 * returns.  The clock (t, step, dt) is left unchanged. */
int s2_set_state(s2_solver *s, const double *w, int where);

/* Copy the state out; synchronises the solver's stream first.  Returns
 * S2_ENONFINITE if the device recorded an invalid state. */
int s2_get_state(s2_solver *s, double *w, int where);

/* Set the state from primitive fields prim[v][k][j][i], v = 0..4 = (rho,
 * u, v, w, T), interior points only (5*nx*ny*nz doubles), host or device
 * memory per where.  The conversion runs on the device with the solver's
 * gas: E = e(T) + |u|^2/2, the thermally perfect e(T) when s2_gas gives
 * c_p coefficients.  Otherwise as s2_set_state (clock unchanged, RK
 * register cleared).  Returns S2_ENONFINITE, with the state set as given,
 * if some rho or T is not positive and finite. */
int s2_set_primitives(s2_solver *s, const double *prim, int where);

/* Primitive fields (rho, u, v, w, T) of the current state, same layout,
 * into host or device memory per where; T from e by the solver's gas in
 * double precision (Newton's method for a thermally perfect gas).
 * Synchronises.  The state is unchanged. */
int s2_get_primitives(s2_solver *s, double *prim, int where);

/* Advance n full RK3 steps (3 stages each).  Asynchronous on the solver's
 * stream: the call enqueues the work (a captured CUDA graph per step) and
 * returns; an invalid state met on the device is reported by the next
 * synchronising call (s2_get_state, s2_stats, s2_sync). */
int s2_step(s2_solver *s, int n);

/* Wait for the solver's stream; returns the device status. */
int s2_sync(s2_solver *s);

/* Stream count independent states through the solver (Sec. 3.2,
 * Listing 3: the state crosses the host link once in and once out, the
 * steps in between stay on the device).  For j = 0 .. count-1: state j is copied in from
 * w_in + j*in_stride, advanced by nsteps RK3 steps, and copied out to
 * w_out + j*out_stride (strides in doubles, >= 0; a stride of 0 reuses one
 * buffer; layout of each state as s2_set_state).  w_in and w_out may be
 * host (pinned or pageable) or device memory.  The copy-in of state j+1
 * and the copy-out of result j run on two streams of the solver beside
 * the steps of state j, through two device staging buffers of one state
 * each (allocated at the first call through the s2_device allocator,
 * released by s2_destroy); pinned host memory lets them overlap.  Each
 * state starts as after s2_set_state (RK register cleared; the clock runs
 * on from state to state).  The call returns when every result is in
 * w_out; w_in must stay unchanged until then, and w_out must not overlap
 * w_in.  Returns S2_ENONFINITE if any state met an invalid value (its
 * result and the following ones are still copied out), S2_ENOMEM if the
 * staging buffers cannot be allocated, S2_EINVAL for a NULL pointer or a
 * negative count, step count or stride. */
int s2_stream_states(s2_solver *s, const double *w_in, long long in_stride, double *w_out, long long out_stride,
                     int count, int nsteps);

/* Flux tile shape per direction: tiles[d] = 0 (64x4 points for x, 32x8
 * for y and z) or 1 (narrower along the direction: 32x8 for x, 16x16 for y
 * and z, for small boxes); single precision doubles each tile along one
 * axis.  Default: (0, 0, 0) for S2_FP64, (0, 1, 1) for S2_MIXED.  Chosen
 * per grid by the autotuner (paper_2304_05494_gb300/autotune.py, the tile
 * knobs of the paper's launch-bounds study, Table 3).  Takes effect at the
 * next s2_step; batches created earlier keep the previous choice.  Results
 * do not depend on it. */
int s2_set_tiles(s2_solver *s, const int *tiles);

/* Launch shape of the kernels, the knobs of the paper's block-shape study
 * (Table 3) and of its translator's configuration (Sec. 3.3), searched by
 * the autotuner (paper_2304_05494_gb300/autotune.py).  tiles: as
 * s2_set_tiles.  flux_ctas_per_sm[d]: CTAs per multiprocessor of the
 * persistent single-precision flux grid of direction d (0: as many as
 * fit, up to 16).
 * z_planes: z-planes each CTA of the mixed path's z-marching gradient and
 * viscous passes walks (0: 12; else 4, 8, 16 or 24, compiled variants).  weno_ctas_per_sm: cap of the
 * WENO kernels' 64-thread CTAs per multiprocessor (0: 16; else 1..64).
 * Takes effect at the next s2_step; results do not depend on it, except
 * that with channel forcing in S2_MIXED the viscous pass sums the forcing
 * per CTA, so z_planes changes the order of that sum (single-precision
 * rounding). */
typedef struct {
  int tiles[3];
  int flux_ctas_per_sm[3];
  int z_planes;
  int weno_ctas_per_sm;
} s2_tuning;
int s2_set_tuning(s2_solver *s, const s2_tuning *t);
int s2_get_tuning(const s2_solver *s, s2_tuning *t);

/* Restore the clock (for a restart from a saved state). */
int s2_set_clock(s2_solver *s, double t, long long step, double dt);

/* Reductions over the current state; synchronises. */
int s2_stats(s2_solver *s, s2_stats_t *out);

/* Diagnostics: evaluate the right-hand side R(w) of the current state
 * (all terms, forcing included) into rhs (same layout as the state; host
 * or device pointer per where).  Synchronises.  The state is unchanged. */
int s2_rhs(s2_solver *s, double *rhs, int where);

/* Diagnostics: per-interface WENO flags of the last RHS evaluation (the
 * last stage of s2_step, or s2_rhs), as bytes
 * 0/1, host pointers: fx (nz, ny, nx+1), fy (nz, ny+1, nx), fz (nz+1, ny,
 * nx); slot p along the direction is the interface between points p-1 and
 * p.  Any pointer may be NULL. */
int s2_get_flags(s2_solver *s, unsigned char *fx, unsigned char *fy, unsigned char *fz);

/* Tracing: kernel classes timed by s2_profile. */
#define S2_PROF_PRIMS 0     /* primitive recovery (+ CFL partials) */
#define S2_PROF_DT 1        /* CFL max reduction, compute_dt of Table 2 */
#define S2_PROF_GHOST 2     /* ghost faces of the primitives */
#define S2_PROF_GRAD 3      /* velocity gradients, divergence, shock sensor */
#define S2_PROF_GHOST_AUX 4 /* ghost faces of divergence and sensor */
#define S2_PROF_FLUX_X 5    /* euler_x (central + WENO) */
#define S2_PROF_FLUX_Y 6    /* euler_y */
#define S2_PROF_FLUX_Z 7    /* euler_z */
#define S2_PROF_VISC 8      /* visflx */
#define S2_PROF_FORCE 9     /* force_rhs_1 (two kernels) */
#define S2_PROF_UPDATE 10   /* RK3 update */
#define S2_PROF_WENO 11     /* WENO flux corrections at flagged interfaces (3 kernels) */
#define S2_PROF_APPLY 12    /* adding the WENO corrections (inviscid runs; fused into visc otherwise) */
#define S2_PROF_KINDS 13

/* Advance n steps launching every kernel directly (no graph) with CUDA
 * events around each class on the solver's stream; ms[k] receives the
 * summed device time of class k over the n steps and launches[k] its
 * kernel count (arrays of S2_PROF_KINDS, host memory; either may be NULL).
 * The state advances exactly as with s2_step.  Synchronises. */
int s2_profile(s2_solver *s, int n, double *ms, long long *launches);

/* Name of a kernel class ("prims", "flux_y", ...); NULL if out of range. */
const char *s2_profile_name(int kind);

/* Measurement aid (the paper has no counterpart): the issue-limited
 * fused multiply-add rate of the GPU, in GFLOP/s (2 flops per FMA), in
 * double (precision = S2_FP64) or single precision (S2_MIXED), from a
 * register-only loop of independent FMA chains on every SM for a few
 * hundred milliseconds.  The double-precision path of this library is
 * bound by that unit; this is the denominator of its roofline, taken at
 * the clock the GPU runs at.  device: CUDA ordinal or -1 for the current
 * one.  Allocates no memory; synchronises. */
int s2_fma_rate(int precision, int device, double *gflops);

/* Release everything; NULL is accepted. */
void s2_destroy(s2_solver *s);

/* Batched stepping, for many independent boxes (ensembles, serving).  A
 * batch groups count distinct solvers created on the same device;
 * s2_batch_step advances every member by n RK3 steps, each step one CUDA
 * graph launch, so that boxes too small to fill the GPU alone (the paper
 * finds ~2M points are needed, Sec. 4.1) fill it together.
 *
 * Work-list mode (S2_BATCH_WORKLIST, the default of s2_batch_create):
 * members that share their kernels (same precision, orders, WENO order,
 * tile shapes, gas model and viscous / WENO / forcing / CFL switches) form
 * a group, and each kernel of an RK stage is one launch for the whole
 * group: a work list in device memory gives every CTA of the launch its
 * box and its tile in that box, the box's parameters come from a table in
 * device memory, and the persistent single-precision flux grids are
 * shared out over the boxes by their tile counts.  A step costs the same
 * ~40 launches for 1 box or 100.  Members of S2_BATCH_SOLO_POINTS points
 * or more fill enough of the GPU on their own, and groups of fewer than
 * S2_BATCH_MIN_GROUP members save too few launches: those keep their own
 * launch sequence (S2_BATCH_WORKLIST_ALL puts every member in a group).  Groups and such members run as concurrent branches of the
 * step graph.  Branch mode (S2_BATCH_BRANCHES): every member's own
 * launch sequence is a concurrent branch.  Either way each box's
 * arithmetic is exactly that of its solo run (results identical bit for
 * bit), members keep their own state, parameters, streams and clocks, and
 * no buffer is shared.
 *
 * stream: the batch's cudaStream_t, or NULL for a private one.  Creation
 * waits for the members' pending work; in work-list mode it allocates the
 * groups' tables (a few KB per member, through the first member's
 * allocator callbacks if it has them), released by s2_batch_destroy.
 * Members' parameters (s2_set_tiles, the clock's dt switch) are taken at
 * creation.  s2_batch_step is asynchronous on the batch stream;
 * s2_batch_sync waits for it and returns the first member error.  Do not
 * step a member on its own while its batch is in flight, and destroy the
 * batch before any of its members. */
#define S2_BATCH_WORKLIST 0
#define S2_BATCH_BRANCHES 1
#define S2_BATCH_WORKLIST_ALL 2   /* work list for every member, whatever its size */
#define S2_BATCH_SOLO_POINTS 262144 /* 64^3 */
#define S2_BATCH_MIN_GROUP 4        /* smaller groups keep their members' own launches */
typedef struct s2_batch s2_batch;
int s2_batch_create(s2_solver *const *members, int count, void *stream, s2_batch **out);
int s2_batch_create_ex(s2_solver *const *members, int count, void *stream, int mode, s2_batch **out);
/* Kernel launches per batch step (all groups or branches); -1 for NULL. */
long long s2_batch_launches(const s2_batch *b);
int s2_batch_step(s2_batch *b, int n);
int s2_batch_sync(s2_batch *b);
void s2_batch_destroy(s2_batch *b);

/* Allocation-free CFL time step.  The paper has no counterpart: this entry
 * point serves callers that must not allocate device memory when they need
 * a step size -- a serving loop whose memory is owned by a pooling
 * allocator it does not control, code running while another framework
 * holds the device's memory, or a latency-bound loop that cannot afford
 * cudaMalloc's implicit synchronisation.  It returns the dt that s2_step
 * computes from the same state (cfl / max over the points of the
 * convective plus viscous spectral radius) without a solver object.
 *
 * w: device pointer, the state in the ABI layout (5*nx*ny*nz doubles).
 * eta_y: device pointer to ny values of deta/dy, or NULL for uniform nodes
 * (ny/ly).  dt: device pointer; one double is written.  stream: a
 * cudaStream_t or NULL.  The call is asynchronous on that stream.  A point
 * that s2_step would report as invalid (density or temperature not
 * positive and finite, or a non-finite velocity) makes *dt = 0.
 *
 * Its only scratch is a fixed array of 65536 doubles (512 KiB) compiled
 * into the library, present on every GPU that loads it until the process
 * exits; nothing is allocated (no cudaMalloc, cudaFree or allocating
 * library call).  Grids above 65536 * 4096 = 268,435,456 points return
 * S2_ETOOBIG (each extent is checked before it is multiplied).  The first
 * call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and caches it with the
 * identifier of the current context; make that first call before any
 * stream capture.  A later call that finds another context current (after
 * cudaDeviceReset, say) looks the address up again, so it too should not
 * be the first call inside a capture.  All calls on a device share the
 * array and every call rewrites the entries it reads, so nothing needs
 * clearing; calls that overlap on the GPU (different streams without
 * ordering) race on it and must be serialised by the caller. */
int s2_cfl_dt_noalloc(const s2_grid *grid, const s2_gas *gas, const double *w, const double *eta_y, double cfl,
                      double *dt, void *stream);

/* Static description of an error code. */
const char *s2_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* S2_H */
