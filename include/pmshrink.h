/*
 * pmshrink — shrinking-domain particle-mesh step on one GB300 (sm_103a).
 *
 * C ABI of the library libpmshrink.so.  The method is Llinares (2017),
 * "The shrinking domain framework I" (arXiv:1709.04703):
 *   - equations of motion dx/dtau = p/a, dp/dtau = -a grad(Phi)      Sec. 2.1, Eqs. 1-2
 *   - Poisson's equation lap(Phi) = (3 H0^2 Om / 2a) delta           Sec. 2.1, Eq. 3
 *   - synchronised (drift-kick-drift) leapfrog                        Sec. 2.2
 *   - CIC mass assignment and force interpolation (same kernel)       Sec. 2.4
 *   - active cells / particles restricted to the observer's past
 *     lightcone, recomputed at the end of every step                 Sec. 2.4, Table 2
 *   - periodic boundaries until the lightcone reaches the box edge,
 *     open boundaries afterwards                                      Sec. 3, Table 1
 *
 * Units.  Positions are in cells of the n_mesh^3 mesh measured from the mesh
 * corner (cell (i,j,k) is centred at (i+.5, j+.5, k+.5)); conformal time in
 * 1/H0; momentum p = a dx/dtau in cells*H0; the potential in (cells*H0)^2.
 * Grids are row-major [z][y][x].
 *
 * Particle records are float4:  pos4 = (x, y, z, id) with the int32 particle
 * id stored bit-for-bit in .w;  mom4 = (px, py, pz, a_cross) where a_cross is
 * only meaningful in lightcone records (expansion factor at which the particle
 * left the domain).
 *
 * Errors.  Every call returns a pm_status; nothing throws or aborts.
 * pm_last_error(ctx) gives a text description of the last failure of that
 * context (pm_last_error(NULL) the last failure of a context-free call).
 *
 * Streams.  Calls that take a context are ordered on the CUDA stream given to
 * pm_init; calls that return host scalars synchronise that stream.
 */
#ifndef PMSHRINK_H
#define PMSHRINK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PM_OK = 0,
  PM_EINVAL = 1,     /* bad argument or configuration */
  PM_ENOMEM = 2,     /* device or pinned-host allocation failed */
  PM_ECUDA = 3,      /* a CUDA call or kernel launch failed */
  PM_ENOCONV = 4,    /* a Poisson solve did not reach rtol in max_vcycles */
  PM_EOVERFLOW = 5,  /* a fixed-point cell count exceeded 2^62 */
  PM_ETIMEOUT = 6,   /* a bounded device-side wait gave up */
  PM_EIO = 7         /* a checkpoint file could not be written or read */
} pm_status;

enum { PM_MIXED = 0, PM_FP32_PLAIN = 1, PM_FP64_PLAIN = 2,
       PM_MIXED_FP64 = 3 };                          /* pm_config.precision */
enum { PM_GUESS_WARM = 0, PM_GUESS_ZERO = 1, PM_GUESS_LEARNED = 2 };  /* pm_config.guess */
enum { PM_GRAVITY_POISSON = 0, PM_GRAVITY_DIFFUSION = 1,
       PM_GRAVITY_DIFFUSION_ADE = 2 };                                 /* pm_config.gravity */
enum { PM_BC_PAPER = 0, PM_BC_OPEN = 1, PM_BC_PERIODIC = 2 };  /* pm_config.bc */
enum { PM_SHRINK_OFF = 0, PM_SHRINK_ON = 1, PM_SHRINK_RECORD = 2 };  /* pm_config.shrink */
enum { PM_ASSIGN_CIC = 0, PM_ASSIGN_TSC = 1 };                  /* pm_config.assignment */
enum { PM_DOMAIN_CUBE = 0, PM_DOMAIN_SPHERE = 1, PM_DOMAIN_BALL = 2 };  /* pm_config.domain */

typedef struct {
  int32_t n_mesh;        /* cells per side, of the form 2^j or 3*2^j, 4..1024 */
  int64_t n_particles;   /* particle count N at the start of the run */
  double box_mpch;       /* comoving side of the initial box, Mpc/h */
  double omega_m;        /* flat background: omega_m + omega_l = 1 expected;
                            omega_m >= 1e-6 (PM_EINVAL below) */
  double omega_l;
  double a_init;         /* first expansion factor */
  double a_final;        /* last expansion factor */
  int32_t n_steps;       /* steps uniform in a (Sec. 3) */
  double rtol;           /* relative residual ||f - A Phi||_2 / ||f||_2 per solve */
  int32_t max_vcycles;   /* V-cycles allowed per solve before PM_ENOCONV */
  int32_t precision;     /* PM_MIXED: FP32 V-cycles inside a double-float
                            defect-correction loop; PM_FP32_PLAIN: FP32 only;
                            PM_FP64_PLAIN: potential, source and every
                            multigrid level in FP64 (one-colour sweeps, a
                            one-CTA bottom of 64 sweeps), Poisson gravity
                            without the learned guess only: the cost of FP64
                            on the device, for comparison;
                            PM_MIXED_FP64: the FP32 V-cycles of PM_MIXED
                            inside a defect correction in FP64 arithmetic:
                            the potential is FP64 for the whole run, and
                            r = f - A Phi and Phi += e are evaluated in FP64
                            (Poisson gravity, warm or zero start) */
  int32_t guess;         /* PM_GUESS_WARM: previous step's Phi; PM_GUESS_ZERO;
                            PM_GUESS_LEARNED: the warm start corrected by the
                            network attached with pm_set_guess */
  int32_t bc;            /* PM_BC_PAPER: periodic until the lightcone reaches
                            the box edge, open afterwards; PM_BC_OPEN /
                            PM_BC_PERIODIC force one kind for the whole run */
  int32_t shrink;        /* PM_SHRINK_ON: drop particles that leave the keep
                            cube (into the lightcone buffer; needs open
                            boundaries, i.e. bc != PM_BC_PERIODIC);
                            PM_SHRINK_OFF: keep everything, record nothing;
                            PM_SHRINK_RECORD: keep and integrate every
                            particle (the fixed-box run the paper compares
                            against, Sec. 3.3) and copy each one, with
                            a_cross, into the lightcone buffer at the end of
                            the first step after which it lies outside the
                            keep cube, with the rule and order of the shrink.
                            In this mode an active particle's mom.w is its
                            record mark (0: not yet recorded; pm_init
                            clears it) */
  double buffer_cells;   /* keep half-width R = chi(a)/cell + buffer_cells */
  int32_t store_forces;  /* 1: keep grad(Phi) at each particle of the last step */
  int32_t gravity;       /* PM_GRAVITY_POISSON: static Eq. 3 every step;
                            PM_GRAVITY_DIFFUSION: the diffusion equation (Eq. 4,
                            Sec. 2.3) advanced by two implicit half-substeps
                            per step in the Table 2 order (see pm_step);
                            PM_GRAVITY_DIFFUSION_ADE: the same equation and
                            order with the paper's alternating-direction
                            explicit scheme (see pm_step) */
  double c_eff_factor;   /* diffusion only: c_eff = factor * cell (Mpc/h) * c,
                            0.019 in Sec. 3.1.1 */
  int32_t assignment;    /* PM_ASSIGN_CIC or PM_ASSIGN_TSC (Sec. 2.4 footnote:
                            the same scheme for the density and the force);
                            TSC needs PM_GRAVITY_POISSON and widens the open
                            cube by one cell (half-width ceil(R) + 2) */
  int32_t domain;        /* keep region: PM_DOMAIN_CUBE (max_d |x_d - c| <= R,
                            the loop-bounded domain of Sec. 2.4) or
                            PM_DOMAIN_SPHERE (|x - c| <= R, Table 1, in FP64:
                            ((x-c)^2 + (y-c)^2) + (z-c)^2 <= R^2); the solve
                            stays on the cube; with the sphere the mean-density
                            term is the CIC image of the ball (exact chord
                            integral, 16-point Gauss-Legendre over the tents);
                            the sphere needs PM_ASSIGN_CIC.  PM_DOMAIN_BALL:
                            the sphere's keep rule and mean-density term; in
                            the open phase the solve runs only on the cells
                            whose centre lies within R + 2 of c (the cube
                            reaches ceil(R) + 3).  Every
                            smoothing, restriction, prolongation and defect
                            pass skips the other cells, which take the
                            multipole values (Dirichlet ghosts next to the
                            ball); coarse levels keep the cells whose centre
                            lies in the ball, with the finest level's
                            boundary.  Needs PM_ASSIGN_CIC, PM_MIXED, Poisson
                            gravity and the warm or zero start */
  int32_t sort_every;    /* 0: the particle arrays keep their order (the
                            initial order, compacted stably by the shrink);
                            k > 0: at the start of every k-th step (step
                            index a multiple of k) the active particles are
                            reordered by the mesh cell of their CIC base
                            node, as pm_sort_particles.  No result of a
                            particle changes, only the order of the arrays
                            and hence of the lightcone records; it keeps
                            the deposit's atomics and the gather's loads
                            coherent once clustering has scattered the
                            initial order.  Single contexts only (a batch
                            rejects k > 0) */
  int32_t inner_vcycles; /* PM_MIXED / PM_MIXED_FP64: FP32 V-cycles run on one
                            correction equation A e = r before the next
                            defect r = f - A Phi (1, the default: a defect
                            after every V-cycle; m > 1: while the solver runs
                            the V-cycles it expects to need without reading
                            the residual, up to m of them share one defect,
                            the first from zero, the others from the
                            iterate, driven by the V-cycle's own FP32
                            residual).  0..16 (0 acts as 1); a batch needs
                            <= 1 */
} pm_config;

/* Fill *cfg with defaults: 32^3 mesh and particles, 250 Mpc/h, Om=0.3,
 * OL=0.7, a 0.02 -> 1 in 20 steps, rtol 1e-7, 50 V-cycles, mixed precision,
 * warm start, paper boundary conditions, shrinking on, buffer 1 cell. */
void pm_config_default(pm_config* cfg);

typedef struct pm_ctx pm_ctx;

/* Checkpoint and resume (not in the paper).  pm_save writes, at a step
 * boundary, everything the following steps depend on: the configuration,
 * the step index, the active particles and the lightcone records (in array
 * order), the potential pair and the previous solution that the warm start
 * extrapolates from, the active cube, the solver's counters and history and
 * the cumulative statistics.  pm_load restores that state into a context
 * created by pm_init with the same configuration (every pm_config field
 * equal, else PM_EINVAL); the steps after it then give the same bits as an
 * uninterrupted run.  The file is a fixed header followed by raw
 * little-endian arrays; it is read back only by this library.  Both calls
 * synchronise the context's stream.  Errors: PM_EINVAL (NULL argument,
 * another configuration, not a checkpoint of this library), PM_EIO (open,
 * write or short read), PM_ECUDA. */
pm_status pm_save(pm_ctx* ctx, const char* path);
pm_status pm_load(pm_ctx* ctx, const char* path);

/* Create a simulation context.  pos4/mom4 hold cfg->n_particles float4
 * records (layout above); they are copied (host_mem = 1: host pointers,
 * pinned or pageable; host_mem = 0: device pointers).  The context owns all
 * device state it allocates; stream is a cudaStream_t (NULL = legacy default
 * stream).  The step schedule (a_k, dtau_k, a_half_k, chi_k) is computed here
 * on the host in FP64.  Errors: PM_EINVAL (n_mesh not 2^j / 3*2^j, N = 0,
 * positions not representable), PM_ENOMEM, PM_ECUDA.  *out is NULL on error. */
pm_status pm_init(const pm_config* cfg, const float* pos4, const float* mom4,
                  int32_t host_mem, void* stream, pm_ctx** out);

/* Advance n_steps steps in the order of Table 2 (Sec. 2.4): half drift,
 * CIC deposit, Poisson solve (Sec. 2.1, Eq. 3), gradient + CIC gather, kick,
 * half drift, lightcone shrink (Sec. 2.4).  With PM_GRAVITY_DIFFUSION the
 * solve is replaced by Table 2's right column: the field is advanced from t
 * to t+dt/2 before the gradient and from t+dt/2 to t+dt after the second
 * half drift, each half-substep one backward-Euler step of Eq. 4,
 * (A - sig) Phi = S delta - sig Phi_old with sig = 3 H / (c_eff^2 dtau/2),
 * H = a E(a) and S at the substep's end, the density of t+dt/2 for both,
 * solved by the same multigrid with a diagonal shift to rtol of
 * ||g - (A - sig) Phi|| / ||g||; the field starts from the static solution
 * of the initial density.  With PM_GRAVITY_DIFFUSION_ADE each half-substep
 * is instead one sweep of the paper's alternating-direction explicit scheme
 * (Sec. 2.3, Saul'yev form) with lam = 1/sig:
 *   Phi_c (1 + lam m) = Phi_c,old (1 - lam (6 - m)) + lam (sum_q Phi_q - S delta)
 * over the cells in lexicographic order, upward in the first half-substep
 * and downward in the second, Phi_q as already updated by the sweep (m of
 * the six) or not; no solve.  Stops early with PM_EINVAL past the last step
 * of the schedule, PM_ENOCONV if a solve fails to converge, PM_EOVERFLOW on
 * fixed-point overflow.  Synchronises the stream for the solver's residual
 * reads (after a run of V-cycles as long as the previous solve's, less one,
 * then after each) and once per shrink (new active count). */
pm_status pm_step(pm_ctx* ctx, int32_t n_steps);

/* Drop particles outside the keep cube of expansion factor a (Sec. 2.4:
 * max_d |x_d - c| > chi(a)/cell + buffer, c the box centre), appending them,
 * in their current order, to the lightcone buffer with a_cross = a; the
 * survivors keep their relative order.  A no-op while the keep cube still
 * covers the periodic box.  Writes the new active count to *n_active_out
 * (may be NULL).  Synchronises the stream. */
pm_status pm_shrink(pm_ctx* ctx, double a, int64_t* n_active_out);

/* Solve sum_nb(Phi) - 6 Phi = S(a) delta on the context's whole n^3 mesh
 * (Sec. 2.1, Eq. 3; S = 3 Om / (2a), cell units) with bc = PM_BC_OPEN
 * (Dirichlet values from the monopole+dipole+quadrupole expansion about the
 * box centre at one layer of ghost-cell centres) or PM_BC_PERIODIC (zero-mean
 * gauge on output).  delta_dev: n^3 doubles [z][y][x] (device).  phi_out_dev:
 * n^3 floats (device), the FP32 rounding of the solution; phi64_out_dev
 * (device, may be NULL): the same as doubles (hi + lo of the double-float
 * state).  Starts from zero and iterates to the context's rtol with its
 * precision setting; *vcycles_out and *resid_out (may be NULL) receive the
 * V-cycles used and the final relative residual.  Does not touch the
 * particles; overwrites the context's potential, which the next pm_step then
 * takes as its warm start.  Errors: PM_EINVAL, PM_ENOCONV, PM_ECUDA. */
pm_status pm_potential(pm_ctx* ctx, const double* delta_dev, double a, int32_t bc,
                       float* phi_out_dev, double* phi64_out_dev,
                       int32_t* vcycles_out, double* resid_out);

/* Power spectrum of n particles (pos4_dev, device) with positions in cells of
 * an n_mesh^3 periodic mesh of side box (Mpc/h): int64 fixed-point CIC
 * density, R2C FFT, |delta_k|^2 L^3/Ng^6 divided by the squared CIC window
 * prod_d sinc^2(k_d h/2), minus the shot noise L^3/n (Sec. 2.4: power
 * spectrum with discreteness correction).  Linear bins of width
 * k_f = 2 pi/L: bin b holds |k|/k_f in [b+.5, b+1.5).  Host outputs of n_bins
 * entries: mean |k| (h/Mpc), mean P ((Mpc/h)^3), number of modes.  Allocates
 * its own scratch; synchronises stream.  subtract_shot = 0 omits the L^3/n
 * term (lattice-based particle sets). */
pm_status pm_power_spectrum(const float* pos4_dev, int64_t n, double box,
                            int32_t n_mesh, int32_t n_bins, int32_t subtract_shot,
                            double* k_out, double* pk_out, double* modes_out,
                            void* stream);

/* The same spectrum with the full alias correction of Jing (2005), the
 * discreteness correction Sec. 2.4 names.  The FFT at k (|k_d| <= k_N) holds
 * every alias k + 2 k_N v (v an integer vector) weighted by the CIC window W:
 *   P_obs(k) = sum_v W^2(k + 2k_N v) P(|k + 2k_N v|) + (L^3/n) C1(k),
 *   C1 = prod_d [1 - (2/3) sin^2(k_d h/2)]  (closed form of sum_v W^2);
 * with P a local power law of slope nu,
 *   P(k) = (P_obs(k) - (L^3/n) C1(k)) / sum_v W^2(k + 2k_N v) (|k + 2k_N v|/|k|)^nu,
 * the sum over v in [-alias_range, alias_range]^3 (1..3).  Each mode takes the
 * slope of its bin; the slopes start from the first-order estimate and are
 * re-measured from the corrected binned spectrum (centred difference of ln P
 * in ln k over the neighbouring bins, clipped to [-6, 4]) until they move by
 * less than tol, at most max_iter passes.  Bins as pm_power_spectrum;
 * nu_out (host, n_bins, may be NULL) receives the slopes, *passes_out (may
 * be NULL) the passes made.  Allocates its own scratch; synchronises stream
 * once per pass.  subtract_shot = 0 drops the (L^3/n) C1 term. */
pm_status pm_power_spectrum_jing(const float* pos4_dev, int64_t n, double box,
                                 int32_t n_mesh, int32_t n_bins, int32_t subtract_shot,
                                 int32_t alias_range, int32_t max_iter, double tol,
                                 double* k_out, double* pk_out, double* modes_out,
                                 double* nu_out, int32_t* passes_out, void* stream);

/* Fixed-point CIC deposit of n particles into rho_dev (n_mesh^3 int64,
 * device, accumulated into: clear it first) over the cube [lo, lo+side)^3
 * (Sec. 2.4 footnote: CIC).  On the float position u per axis:
 * i = floor(u - .5), dq = floor((u - .5) 2^16) - i 2^16; weights 2^16 - dq on
 * node i and dq on node i+1; their product is added as an int64.  periodic=1
 * wraps nodes mod n_mesh (then lo = 0, side = n_mesh); otherwise a particle
 * with a node outside the cube deposits nothing and is counted in
 * *escaped_out (host, may be NULL).  If mom4_dev is not NULL the particles
 * are first drifted in place, x = fl(x + fl(p * drift_coef)) in float32
 * (Sec. 2.2, first DKD line), wrapped into [0, n_mesh) when periodic.
 * Synchronises stream only when escaped_out is not NULL. */
pm_status pm_deposit(float* pos4_dev, const float* mom4_dev, int64_t n,
                     float drift_coef, int32_t n_mesh, int32_t lo, int32_t side,
                     int32_t periodic, int64_t* rho_dev, int64_t* escaped_out,
                     void* stream);

/* The same deposit with the TSC weights (Sec. 2.4 footnote): per axis the
 * cell i = floor(u) and q = floor(u 2^16) - i 2^16 give nodes i-1, i, i+1
 * the weights (2^16 - q)^2 >> 17, the remainder, q^2 >> 17 (exactly 2^16 in
 * total); their products are added as int64.  Open: a particle with a node
 * outside [lo, lo+side) deposits nothing and is counted as escaped.
 * Arguments, drift and synchronisation as pm_deposit. */
pm_status pm_deposit_tsc(float* pos4_dev, const float* mom4_dev, int64_t n,
                         float drift_coef, int32_t n_mesh, int32_t lo, int32_t side,
                         int32_t periodic, int64_t* rho_dev, int64_t* escaped_out,
                         void* stream);

/* Reorder n particles by the mesh cell of their CIC base node: key
 * ((k n + j) n + i) with i = floor(u_x - 1/2) mod n_mesh (likewise j, k;
 * float32 subtraction, non-finite coordinates give 0), a stable sort (equal
 * keys keep their input order), so the result is unique.  pos4_out and
 * mom4_out (device, n float4 each, caller-owned, not overlapping the inputs)
 * receive the records in that order; mom4_dev may be NULL (then mom4_out is
 * not written).  An order of the data only: the deposit of the particles is
 * unchanged (its integer sums do not depend on the order).  Work space is
 * allocated and freed inside the call.  n_mesh in [1, 1024], n in
 * [0, 2^31).  Synchronises stream. */
pm_status pm_sort_particles(const float* pos4_dev, const float* mom4_dev, int64_t n,
                            int32_t n_mesh, float* pos4_out, float* mom4_out, void* stream);

typedef struct {
  int32_t step;          /* steps completed */
  double a;              /* current expansion factor */
  int64_t n_active;      /* particles inside the domain */
  int64_t n_lightcone;   /* particles in the lightcone buffer */
  int32_t cube_lo;       /* active mesh cube of the last step: [lo, lo+side)^3 */
  int32_t cube_side;
  int32_t periodic;      /* boundary kind of the last step */
  int32_t vcycles_last;  /* V-cycles of the last solve */
  int64_t vcycles_total; /* V-cycles since pm_init */
  double resid_last;     /* final relative residual of the last solve */
  int64_t escaped;       /* particle-steps skipped because a CIC node left the cube */
  int64_t particle_steps;/* sum over completed steps of the active count */
  int32_t guess_used_last;  /* 1 if the network corrected the last solve's start */
  int64_t guess_used_total; /* solves started from the network's correction */
  double resid_start;       /* relative residual of the last solve's start */
  double resid_guess;       /* ... after the network's correction (= resid_start
                               when the network did not run) */
} pm_stats_t;

pm_status pm_stats(pm_ctx* ctx, pm_stats_t* out);

/* The fused smoother's launch shape per level side, as pm_init picked it by
 * timing (the multigrid solve's red-black smoothing, two sweeps in one
 * pass; every shape gives the same bits).  Host arrays of cap entries each
 * (any may be NULL): sides[i], the CTA tile height (16, 24 or 32) and the
 * planes per CTA.  *count (required) = the number of sides tuned (0: all
 * levels smaller than 192, or the ball solve, which keeps height 16); at
 * most cap entries are written.  NULL ctx or count, cap < 0: PM_EINVAL. */
pm_status pm_smoother_tiles(pm_ctx* ctx, int32_t* sides, int32_t* tile_height,
                            int32_t* z_chunk, int32_t cap, int32_t* count);

/* Copy the schedule (n_steps + 1 entries each, host arrays, any may be NULL):
 * a_k, dtau_k (conformal step k -> k+1, last entry 0), a_half_k (a at the
 * conformal midpoint of step k, last entry 0), chi_k (Mpc/h). */
pm_status pm_schedule(pm_ctx* ctx, double* a, double* dtau, double* a_half,
                      double* chi);

/* Active particles (n_active float4 records each) to host (host_mem = 1) or
 * device buffers; either pointer may be NULL.  Synchronises the stream. */
pm_status pm_get_particles(pm_ctx* ctx, float* pos4, float* mom4,
                           int32_t host_mem, int64_t* n_active_out);

/* Replace the active particles by n records (n <= cfg.n_particles). */
pm_status pm_set_particles(pm_ctx* ctx, const float* pos4, const float* mom4,
                           int64_t n, int32_t host_mem);

/* Lightcone records (pos4, mom4 with .w = a_cross). */
pm_status pm_get_lightcone(pm_ctx* ctx, float* pos4, float* mom4,
                           int32_t host_mem, int64_t* n_out);

/* grad(Phi) at each active particle of the last step (float4, .w unused),
 * in the particle order at the end of that step's kick, before the shrink.
 * Needs cfg.store_forces = 1. */
pm_status pm_get_forces(pm_ctx* ctx, float* f4, int32_t host_mem, int64_t* n_out);

/* Copy the current potential on the active cube plus its ghost layer,
 * (side+2)^3 doubles [z][y][x], to host (hi + lo of the double-float state). */
pm_status pm_get_potential(pm_ctx* ctx, double* phi_host, int32_t* lo_out,
                           int32_t* side_out);

/* Per-kernel-class timing with CUDA events recorded on the context's stream
 * around the launches of each class, read back at the step's existing sync
 * points.  Classes: */
enum {
  PM_PROF_DEPOSIT = 0,  /* half drift + CIC deposit                         */
  PM_PROF_SOURCE,       /* counts -> double-float source (+ moments)        */
  PM_PROF_BOUNDARY,     /* open-boundary ghost layer                        */
  PM_PROF_SMOOTH0,      /* red-black sweeps on the finest level             */
  PM_PROF_TRANSFER0,    /* finest-level residual+restriction, prolongation  */
  PM_PROF_COARSE,       /* everything on levels >= 1                        */
  PM_PROF_DEFECT,       /* double-float residual + norm                     */
  PM_PROF_CORRECT,      /* Phi += e                                         */
  PM_PROF_GATHER,       /* gradient + gather + kick + drift + keep flags    */
  PM_PROF_COMPACT,      /* scan + stable scatter                            */
  PM_PROF_GUESS,        /* learned initial guess (network forward)          */
  PM_PROF_ADE,          /* explicit diffusion sweeps (PM_GRAVITY_DIFFUSION_ADE) */
  PM_PROF_SORT,         /* particle order by cell (sort_every)              */
  PM_PROF_N
};
/* enable = 1 starts (and zeroes) the counters, 0 stops them. */
pm_status pm_profile(pm_ctx* ctx, int32_t enable);
/* Accumulated device time (ms), timed launch groups, and algorithmic bytes
 * (the minimal DRAM traffic of those launches) of one class. */
pm_status pm_profile_read(pm_ctx* ctx, int32_t cls, double* ms, int64_t* groups,
                          double* bytes);

/* ---------------------------------------------------------------------------
 * Batched step: many independent realisations (each its own configuration,
 * mesh size, particles and lightcone schedule; Sec. 2.4 applied to each)
 * advance together.  Every phase of pm_step runs as one kernel launch over
 * all realisations (a device table maps each block to a realisation).  The
 * solve (Sec. 2.1: defect, convergence test, V-cycle, repeated) is decided
 * on the device: the convergence test runs in a kernel after each batched
 * defect, a realisation that has converged is masked out of further passes,
 * and the host reads nothing until the step ends.  By default the solve is
 * one CUDA graph whose V-cycle loop is a conditional while node; a
 * persistent cooperative kernel is the other form (pm_batch_set_solve).
 * Results equal those of separate contexts bit for bit.
 * Requirements: 1 <= n_real <= 64, precision PM_MIXED, all realisations on
 * the same number of steps and a_init/a_final (one schedule of a, each with
 * its own chi(a)/cell), stream not NULL.
 * pos4[r] / mom4[r]: cfgs[r].n_particles records each (host_mem as in
 * pm_init).  Errors as pm_init / pm_step; pm_batch_last_error() explains.
 * ------------------------------------------------------------------------- */
typedef struct pm_batch pm_batch;
pm_status pm_batch_init(int32_t n_real, const pm_config* cfgs, const float* const* pos4,
                        const float* const* mom4, int32_t host_mem, void* stream,
                        pm_batch** out);
pm_status pm_batch_step(pm_batch* b, int32_t n_steps);
pm_status pm_batch_stats(pm_batch* b, int32_t r, pm_stats_t* out);
pm_status pm_batch_get_particles(pm_batch* b, int32_t r, float* pos4, float* mom4,
                                 int32_t host_mem, int64_t* n_active_out);
pm_status pm_batch_get_lightcone(pm_batch* b, int32_t r, float* pos4, float* mom4,
                                 int32_t host_mem, int64_t* n_out);
/* grad(Phi) at each active particle of realisation r in the last batched
 * step, as pm_get_forces (needs cfgs[r].store_forces = 1). */
pm_status pm_batch_get_forces(pm_batch* b, int32_t r, float* f4, int32_t host_mem,
                              int64_t* n_out);
/* How a batch solves.  persistent = 0 (the default): the graph above.
 * persistent = 1: one persistent cooperative launch per solve, its passes
 * separated by a grid-wide barrier, every block taking the same convergence
 * decisions from the residual norms (the two give the same bits).
 * wait_seconds (> 0, finite; default 2): the longest wait at one grid
 * barrier; when it runs out the kernel sets an error word, every block
 * leaves, and pm_batch_step returns PM_ETIMEOUT (the batch's state is then
 * undefined: destroy it).  extra_arrivals: 0; a value > 0 makes every
 * barrier wait for arrivals that never come, which tests the time limit.
 * PM_EINVAL on bad arguments, or persistent = 1 where the kernel's grid
 * cannot be resident. */
pm_status pm_batch_set_solve(pm_batch* b, int32_t persistent, double wait_seconds,
                             int32_t extra_arrivals);
const char* pm_batch_last_error(const pm_batch* b);
void pm_batch_destroy(pm_batch* b);

/* Allocation-free lightcone compaction.  The paper has no counterpart: this
 * is a variant of pm_shrink's compaction for callers that cannot allocate
 * device memory — host programs that hand the library a fixed memory budget
 * and forbid further allocation, and loops that cannot afford the implicit
 * device synchronisation of cudaMalloc/cudaFree.  It calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *
 * Takes n float4 particle records on the device (pos4_in, mom4_in, layout as
 * above) and writes, in their input order, the survivors of the keep cube of
 * expansion factor a (the rule of pm_shrink with PM_BC_PAPER: keep iff
 * max_d |x_d - n_mesh/2| <= chi(a)/(box_mpch/n_mesh) + buffer_cells, and
 * everything is kept while that half-width exceeds n_mesh/2 - 1) to
 * pos4_keep/mom4_keep and the leavers to pos4_leave/mom4_leave with
 * mom.w = a.  Output buffers are caller-owned, n records each, and must not
 * overlap the inputs.  *n_keep_out receives the survivor count; the stream
 * (cudaStream_t, NULL = legacy default stream) is synchronised.
 *
 * Scratch: a static device array for at most PM_SHRINK_STATIC_MAX_PARTICLES
 * particles (~4.1 MB, held on every GPU that loads the library until exit);
 * larger n is rejected with PM_EINVAL.  The first call on a device looks up
 * that array's device address (set-up), so make the first call before any
 * stream capture.  All calls on a device share the one array: calls that
 * overlap on the GPU (different streams or threads) race and must be
 * serialised by the caller.  Non-finite box_mpch, omega_m, omega_l,
 * buffer_cells or a give PM_EINVAL.  pm_shrink_static_error() describes the
 * calling thread's last failure; the returned text stays valid until that
 * thread's next failing call. */
#define PM_SHRINK_STATIC_MAX_PARTICLES (1 << 22)
pm_status pm_shrink_static(const float* pos4_in, const float* mom4_in, int64_t n,
                           int32_t n_mesh, double box_mpch, double omega_m, double omega_l,
                           double buffer_cells, double a, float* pos4_keep, float* mom4_keep,
                           float* pos4_leave, float* mom4_leave, int64_t* n_keep_out,
                           void* stream);
const char* pm_shrink_static_error(void);

/* ---------------------------------------------------------------------------
 * Learned initial guess (not in the paper; a build requirement): a BF16
 * convolutional network on the tensor cores (tcgen05, FP32 accumulation in
 * tensor memory) that maps a source to a potential guess for the solver.
 * ------------------------------------------------------------------------- */

/* Failure-detection self-test of the bounded wait used by the tensor-core
 * kernels (an mbarrier polled with an iteration limit; on giving up a
 * kernel sets an error word that the host maps to PM_ETIMEOUT).  One warp
 * initialises an mbarrier for one arrival; arrive = 1: a thread arrives and
 * the wait completes (PM_OK); arrive = 0: nothing arrives and the wait gives
 * up after `polls` polls (PM_ETIMEOUT).  Nothing asynchronous is in flight,
 * and the context stays usable.  polls in [1, 1e9], else PM_EINVAL.
 * Synchronises stream. */
pm_status pm_selftest_wait(int32_t arrive, int64_t polls, void* stream);

/* The multigrid smoother of the Poisson solve (Sec. 2.1, Eq. 3 as the
 * 7-point system h^-2 (sum_nb u - diag u) = b): two red-black SOR sweeps
 * (red = (i+j+k) even first, then black, twice), u_out = S(u_in).
 * Arrays are padded (s+2)^3 FP32 device arrays, [z][y][x], one ghost layer
 * (read, never written).  periodic = 1 wraps instead; gam > 0 adds gam per
 * ghost face to the diagonal 6 (the coarse-level open boundary).
 * zero_start: u_in is taken as zero (ghosts included) and not read.
 * Each update is red-black SOR: the cell moves from its old value u_old
 * towards the Gauss-Seidel value g = (sum_nb u - h2 b) / diag by the factor
 * PM_MG_OMEGA, u = u_old + PM_MG_OMEGA (g - u_old) (one fused multiply-add
 * in FP32); every multigrid smoothing pass of the solver does the same.
 * fused = 1: one pass over the grid (u_in and u_out distinct unless
 * zero_start) in 32 x 16 tiles; fused = 16, 24 or 32: the same pass in
 * 32 x fused tiles; fused = 0: four one-colour passes in place on u_out
 * after copying u_in.  All give the same bits.  zchunk: planes per CTA of
 * the fused pass (0 = default).  s even, >= 4.  Other values of fused:
 * PM_EINVAL.  Synchronises stream. */
/* The smoother's over-relaxation factor (1 would be Gauss-Seidel). */
#define PM_MG_OMEGA 1.25f

pm_status pm_mg_smooth(const float* u_in, float* u_out, const float* b, int32_t s,
                       int32_t periodic, float h2, float gam, int32_t zero_start, int32_t fused,
                       int32_t zchunk, void* stream);

/* The multigrid transfers of the same solve, on padded (s+2)^3 FP32 device
 * arrays [z][y][x] (s even, >= 4; coarse side s/2, padded likewise).
 * pm_mg_restrict: bc = 1/8 of the sum over the 8 children of the residual
 * b - (sum_nb u - diag u) / h2 (diag as pm_mg_smooth: 6, plus gam per ghost
 * face when open); uc is zeroed (interiors only).  pm_mg_prolong: u += P uc,
 * trilinear with weights 3/4 on the parent and 1/4 on the next coarse cell
 * per axis; periodic wraps, open takes the next cell outside the coarse
 * grid as -gam_c times the parent.  Synchronise stream. */
pm_status pm_mg_restrict(const float* u, const float* b, int32_t s, int32_t periodic, float h2,
                         float gam, float* uc, float* bc, void* stream);
pm_status pm_mg_prolong(const float* uc, float* u, int32_t s, int32_t periodic, float gam_c,
                        void* stream);

/* C[M x N] (FP32, row-major) = A[M x K] B[N x K]^T with A, B row-major BF16
 * device matrices; M % 128 == 0, K % 64 == 0, N in {16, 32, 64, 128}.  The
 * tile engine under every convolution of the learned guess.  PM_ETIMEOUT if
 * an MMA completion wait gave up.  Synchronises stream. */
pm_status pm_nn_gemm_bf16(const void* A, const void* B, float* C, int32_t M, int32_t N,
                          int32_t K, void* stream);

/* The network.  levels L in 1..4, channels 8 * 2^l per level: encoder of
 * 3x3x3 convolutions + ReLU with 2x average pooling between levels, decoder
 * of nearest 2x upsampling, concatenation with the encoder output of the
 * same level, convolution + ReLU, and a final linear 3x3x3 convolution to
 * 8 channels whose first is the guess.  The input is the source scaled to
 * unit RMS per sample; the guess is rescaled by RMS(source) * out_scale.
 * Activations BF16 channels-last, accumulation FP32 in tensor memory,
 * parameters FP32 masters (per convolution, encoder then decoder then
 * output: weights [cout][27 cin] with tap index (dz+1)*9+(dy+1)*3+(dx+1),
 * then biases [cout]).  Zero padding outside each sample. */
typedef struct pm_guess pm_guess;
pm_status pm_guess_create(int32_t levels, void* stream, pm_guess** out);
int64_t pm_guess_num_params(const pm_guess* g);
/* Host parameters in, Adam state reset. */
pm_status pm_guess_set_params(pm_guess* g, const float* params_host, float out_scale);
/* Parameters and the gradient of the last pm_guess_loss_grad (host; either
 * may be NULL). */
pm_status pm_guess_get_params(pm_guess* g, float* params_host, float* grad_host);
/* guess[b] for B sources of side S (device FP32 arrays B*S^3, [b][z][y][x]);
 * S a multiple of 2^(L-1). */
pm_status pm_guess_forward(pm_guess* g, const float* src_dev, int32_t B, int32_t S,
                           int32_t periodic, float* guess_dev);
/* Loss between the network output y and t = target / (RMS(source) *
 * out_scale), and its gradient with respect to the parameters (kept for
 * pm_guess_adam / pm_guess_get_params).  loss_kind 0: mean over voxels of
 * (y - t)^2; 1: mean of (A (y - t))^2 with A the 7-point Laplacian (zero
 * outside each sample unless periodic), i.e. the residual the guess leaves.
 * periodic = 1 makes every convolution and A wrap around each sample. */
pm_status pm_guess_loss_grad(pm_guess* g, const float* src_dev, const float* target_dev,
                             int32_t B, int32_t S, int32_t periodic, int32_t loss_kind,
                             double* loss_out);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) with learning rate lr. */
pm_status pm_guess_adam(pm_guess* g, float lr);
const char* pm_guess_last_error(const pm_guess* g);
void pm_guess_destroy(pm_guess* g);

/* Attach a network (or NULL) to a context for PM_GUESS_LEARNED.  In every
 * solve whose cube side is >= 16 and a multiple of 2^(levels-1), the
 * residual r of the warm start is fed to the network and its output, a
 * correction e ~ A^-1 r, is added to the start before the V-cycles, which
 * still iterate to rtol.  The context does not own the network; the
 * network's parameters must not change while a step runs.  Allocates two
 * n_mesh^3 FP32 scratch fields.  Not in the paper. */
pm_status pm_set_guess(pm_ctx* ctx, pm_guess* net);
/* Training pairs from the solver: while armed (r_dev, e_dev non-NULL, device
 * arrays of n_mesh^3 floats), every solve writes the residual of its warm
 * start (r) and the correction that the solve added to it (e = Phi - start)
 * as dense side^3 arrays [z][y][x], side = pm_stats cube_side.  PM_MIXED
 * only.  NULLs disarm.  Not in the paper. */
pm_status pm_capture(pm_ctx* ctx, float* r_dev, float* e_dev);

/* Kernel launches made by this library in this process so far. */
int64_t pm_launch_count(void);

/* CTAs per thread-block cluster of the coarse multigrid levels (the levels
 * of side <= 64, 32 or 16 for 16, 8 or 1 CTAs run in one cluster's
 * distributed shared memory, Sec. 2.1's V-cycle below the launched levels),
 * set at pm_init: 1 by default (the fastest measured), 8 or 16 when the
 * environment variable PM_CMG_CLUSTER asks for it and the GPU can hold such
 * a cluster, 1 whenever PM_NO_CLUSTER is set.  The results do not depend
 * on it. */
int32_t pm_mg_cluster_size(void);

const char* pm_last_error(const pm_ctx* ctx);
void pm_destroy(pm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* PMSHRINK_H */
