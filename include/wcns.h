/*
 * wcns.h - C ABI of the GB300 PP-WCNS-IS solver for the five-equation
 * (Allaire) two-phase model with an ideal-gas phase and a stiffened-gas
 * liquid phase.
 *
 * Method: Wong, Angel, Barad & Kiris, "A positivity-preserving high-order
 * weighted compact nonlinear scheme for compressible gas-liquid flows"
 * (arXiv 2102.05287).  Section numbers below refer to that paper.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Phase 1 is the liquid (stiffened gas: gamma_l, pinf_l >= 0), phase 2 the
 *    gas (ideal: gamma_g, pinf = 0), as in the paper's fluid table (Sec. 6).
 *  - State layout: conservative vector W = (a1r1, a2r2, rho*u_1 .. rho*u_ndim,
 *    E, alpha1) (Sec. 2), nf = ndim + 4 fields, stored structure-of-arrays as
 *    a contiguous double array [nf][n_z][n_y][n_x] (x fastest, interior cells
 *    only; lower-dimensional grids drop the leading axes).
 *  - Pointers named W / dWdt are DEVICE pointers owned by the caller (for
 *    example torch CUDA tensors), 8-byte aligned.  The handle owns all
 *    scratch it needs, allocated once in wcns_create; rhs / step / advance
 *    calls allocate nothing (the one exception: the first
 *    wcns_advance_steps_host call allocates the device copy of a host
 *    state, which the handle then keeps).
 *  - Work is ordered on the stream set with wcns_set_options (default: the
 *    legacy default stream).  Calls returning host values synchronise that
 *    stream.
 *  - Every call returns a status code (WCNS_OK = 0, or a WCNS_E_* value);
 *    nothing throws or aborts.  wcns_strerror gives a message.  Device-side
 *    problems (non-finite values, inadmissible input, limiter hard switches)
 *    are counted in the handle's statistics (wcns_get_stats), never trapped.
 *    The calls that synchronise at their end (wcns_advance_steps,
 *    wcns_advance_to, wcns_advance_steps_host, wcns_batch_advance) also read
 *    those counters back and return WCNS_E_NONFINITE when an update of
 *    theirs was not finite, else WCNS_E_INADMISSIBLE when a stage input
 *    state (the initial state included) had a cell outside G: a negative
 *    partial density, alpha1 outside [0, 1], rho ctilde^2 <= 0 or a
 *    non-finite value (Sec. 2).  The state is left as the device computed
 *    it; the kernels always run to completion.  Asynchronous calls
 *    (wcns_rhs, wcns_rk3_step, wcns_rk3_step_noalloc) only count.
 */
#ifndef WCNS_H
#define WCNS_H

#ifdef __cplusplus
extern "C" {
#endif

/* A handle (wcns_handle or wcns_batch) is not thread-safe: calls on one
 * handle must not run concurrently. */
typedef struct wcns_handle wcns_handle;

/* Status codes. */
enum {
  WCNS_OK = 0,
  WCNS_E_INVALID_ARG = 1,   /* bad argument (null pointer, size, parameter) */
  WCNS_E_CUDA = 2,          /* a CUDA runtime call failed */
  WCNS_E_INADMISSIBLE = 3,  /* a stage input state outside the admissible set G (Sec. 2) */
  WCNS_E_NONFINITE = 4,     /* a non-finite value appeared */
                            /* 5 is not used: no call waits on the device with a time limit */
  WCNS_E_UNSUPPORTED = 6,   /* option combination not provided */
  WCNS_E_TOO_LARGE = 7      /* problem exceeds the fixed no-allocation scratch */
};

/* Boundary conditions per face (three ghost layers, Sec. 6 "extrapolation"):
 *   TRANSMISSIVE - zero-gradient copy of the boundary cell;
 *   PERIODIC     - wrap-around (both faces of an axis must be periodic);
 *   SYMMETRY     - mirror image with the normal momentum negated (n >= 3);
 *   DIRICHLET    - a fixed conservative state given in wcns_bcs.dirichlet. */
enum { WCNS_BC_TRANSMISSIVE = 0, WCNS_BC_PERIODIC = 1, WCNS_BC_SYMMETRY = 2, WCNS_BC_DIRICHLET = 3 };

/* Uniform Cartesian grid on [lo, hi] (Sec. 3: cells of width (hi-lo)/n). */
typedef struct {
  int ndim;       /* 1, 2 or 3 */
  int n[3];       /* cells per axis (entries beyond ndim ignored), each >= 1 */
  double lo[3];
  double hi[3];
} wcns_grid;

typedef struct {
  int kind[3][2];              /* [axis][0 = low face, 1 = high face] */
  double dirichlet[3][2][7];   /* conservative ghost state for DIRICHLET faces */
} wcns_bcs;

/* Precision of the hot path. */
enum {
  WCNS_FP64 = 0,   /* every step in FP64 */
  WCNS_MIXED = 1   /* FP32 characteristic projection, WCNS-IS interpolation and
                      HLLC fluxes; FP64 pressure / sound speed, limiter
                      blending-coefficient solve and state accumulation */
};

/* Spatial scheme. */
enum {
  WCNS_SCHEME_PP_WCNS_IS = 0,  /* WCNS-IS with both PP limiters (Secs. 4-5) */
  WCNS_SCHEME_HLLC1 = 1,       /* first-order HLLC scheme (Sec. 3) */
  WCNS_SCHEME_WCNS_IS = 2      /* WCNS-IS with the limiters switched off */
};

typedef struct {
  int precision;        /* WCNS_FP64 (default) or WCNS_MIXED */
  int scheme;           /* WCNS_SCHEME_* (default PP-WCNS-IS) */
  double eps_is;        /* epsilon of the IS nonlinear weights (Sec. 4.3; the paper
                           does not print it): default 1e-40 (FP64), the FP32
                           stages of the mixed path use max(eps_is, 1e-30) */
  double eps_ar, eps_a, eps_rc;  /* limiter tolerances, Sec. 5.1: 1e-10, 1e-10, 1e-8 */
  double hs_ar, hs_a, hs_rc;     /* hard-switch tolerances, Sec. 5.1: 1e-11, 1e-11, 1e-9;
                                    all six finite and >= 0, else WCNS_E_INVALID_ARG */
  void *stream;         /* cudaStream_t for all work of this handle (NULL = default) */
} wcns_options;

/* Counters accumulated on the device since the last reset. */
typedef struct {
  long long interp_limited;  /* interpolated states with some theta < 1 (Algs. 1-3) */
  long long interp_hard;     /* interpolation hard switches (Sec. 5.1) */
  long long flux_limited;    /* midpoints with some flux-limiter theta < 1 (Algs. 4-6) */
  long long flux_hard;       /* flux hard switches (Sec. 5.2) */
  long long nonfinite;       /* cells whose update was not finite */
  long long inadmissible;    /* input cells outside G (Sec. 2) */
  long long midpoints;       /* midpoint fluxes evaluated */
  long long fp64_fallbacks;  /* interpolated states and midpoints whose
                                limiter could not be certified in FP32 and
                                ran in FP64 (both precisions certify) */
} wcns_stats;

/* Create a solver for one grid, boundary set and fluid pair.
 * gamma_g > 1, gamma_l > 1, pinf_l >= 0 and gamma_g <= gamma_l (Lemma 1,
 * Sec. 2: the admissible set is convex only then).  Periodic axes need both
 * faces periodic; symmetry needs n >= 3 on that axis.  Launch-grid limits
 * (65535 blocks in grid y and z): in 2D and 3D n[0] <= 524,280 and
 * n[1] <= 131,070; in 3D also n[1], n[2] <= 65,535.  Allocates the
 * handle's device scratch on the current device: three states (8 nf bytes
 * a cell each) and, in 2D and 3D, a 24-byte-per-cell node cache the mixed
 * precision sweeps of one RHS share.
 * Returns WCNS_E_INVALID_ARG on a bad argument, WCNS_E_CUDA on allocation
 * failure; *out is NULL on error. */
int wcns_create(const wcns_grid *grid, const wcns_bcs *bcs, double gamma_g, double gamma_l,
                double pinf_l, wcns_handle **out);

/* Default options (FP64, PP-WCNS-IS, paper tolerances, default stream). */
void wcns_default_options(wcns_options *opt);
int wcns_set_options(wcns_handle *h, const wcns_options *opt);
int wcns_get_options(const wcns_handle *h, wcns_options *opt);

/* A Dirichlet state that varies along a face (Sec. 6, Mach 100 water jet:
 * the inflow state depends on the position along the left boundary).
 * W_face is a HOST array of nf * (ncells / n[axis]) doubles, conservative
 * states laid out [nf][face cells], the face cells ordered by the remaining
 * axes in increasing order with the lower axis fastest; the three ghost
 * layers of each line normal to the face take that line's state.  The face
 * must have kind WCNS_BC_DIRICHLET (else WCNS_E_INVALID_ARG).  The first
 * call allocates a device copy owned by the handle (later calls overwrite
 * it in place); W_face = NULL frees it and the face returns to the uniform
 * state of wcns_bcs.dirichlet.  Synchronises the handle's stream. */
int wcns_set_dirichlet_face(wcns_handle *h, int axis, int side, const double *W_face);

/* Semi-discrete right-hand side L(W) = dW/dt of Sec. 4 (eq. for dW/dt with
 * G^{x,-}_{i+1/2} - G^{x,+}_{i-1/2}, including the alpha1 div(u) term),
 * summed over the ndim directions.  dt is the Euler step the flux limiter
 * protects (Sec. 5.2): lambda_d = dt / (dx_d sigma_d), sigma_d = tau_d /
 * sum(tau) with tau_d = max(|u_d| + c)/dx_d of W and the Dirichlet ghost
 * states (Sec. 3.3).  dt must be finite and >= 0 (else WCNS_E_INVALID_ARG);
 * dt = 0 is taken as a vanishing step (1e-300), for which the flux limiter's
 * half states are the cell states themselves.
 * W and dWdt are device arrays of nf * ncells doubles; they must not
 * overlap.  Asynchronous on the handle's stream. */
int wcns_rhs(wcns_handle *h, const double *W, double *dWdt, double dt);

/* max over cells of (|u_d| + c) for each direction d < ndim (Sec. 3.3);
 * out[d] = 0 for d >= ndim.  Dirichlet ghost states (uniform or per face)
 * count as cells: they enter the boundary midpoints' fluxes, so their wave
 * speeds bound dt as well.  out is a HOST array of 3 doubles; synchronises. */
int wcns_max_wavespeed(wcns_handle *h, const double *W, double out[3]);

/* One SSPRK3 (Shu-Osher) step of size dt, in place on the device array W
 * (Sec. 5.3: each stage is a convex combination of Euler steps).
 * Asynchronous. */
int wcns_rk3_step(wcns_handle *h, double *W, double dt);

/* Stage tracing (verification aid, not part of the method): with W1_out
 * and W2_out non-NULL device arrays of the state's size, every SSPRK3 step
 * of this handle also copies its intermediate stage states W^(1) and W^(2)
 * there (device-to-device on the handle's stream, no allocation); a later
 * step overwrites them.  NULL, NULL switches tracing off. */
int wcns_set_stage_trace(wcns_handle *h, double *W1_out, double *W2_out);

/* Advance W in place by nsteps SSPRK3 steps.  With dt_fixed > 0 every step
 * uses dt_fixed; otherwise dt = cfl / sum_d tau_d from the state at the
 * start of each step (Sec. 3.3), computed and kept on the device.
 * *t_io (host, may be NULL) holds the start time on entry and the final
 * time on exit.  One step (dt kernel and all sweeps) is captured once into
 * a CUDA graph per (W, dt_fixed, cfl) and replayed on the handle's private
 * stream, ordered after the caller's pending work; per-kernel timing
 * disables the graph.  Synchronises once at the end and returns
 * WCNS_E_NONFINITE / WCNS_E_INADMISSIBLE as described at the top (all
 * nsteps steps are taken either way). */
int wcns_advance_steps(wcns_handle *h, double *W, int nsteps, double cfl, double dt_fixed,
                       double *t_io);

/* Advance W in place from t0 to t_end with CFL-limited steps (dt as above,
 * the last step clipped to land on t_end).  Returns the end time and the
 * number of steps taken in the host outputs (either may be NULL).  The host
 * checks the device step control and counters every 8-256 steps: a
 * non-finite time step (a state whose wave speed is not finite) or a
 * non-finite update ends the call with WCNS_E_NONFINITE, an inadmissible
 * stage input with WCNS_E_INADMISSIBLE, W holding the state of that moment
 * and the outputs the time and steps reached. */
int wcns_advance_to(wcns_handle *h, double *W, double t0, double t_end, double cfl,
                    double *t_out, long *steps_out);

/* As wcns_advance_steps, but W_host is a HOST array (pageable or pinned):
 * it is copied to a device state owned by the handle (allocated by the
 * first call, 8 nf bytes a cell, freed by wcns_destroy), advanced, and
 * copied back, all on the handle's stream.  Synchronises.  Returns
 * WCNS_E_CUDA if that allocation fails; the state is copied back also when
 * the steps return WCNS_E_NONFINITE or WCNS_E_INADMISSIBLE. */
int wcns_advance_steps_host(wcns_handle *h, double *W_host, int nsteps, double cfl,
                            double dt_fixed, double *t_io);

/* Statistics counted on the device since creation or the last reset;
 * synchronises. */
int wcns_get_stats(wcns_handle *h, wcns_stats *out);
int wcns_reset_stats(wcns_handle *h);

/* Number of fields nf = ndim + 4 and of cells of the handle's grid. */
int wcns_nfields(const wcns_handle *h);
long long wcns_ncells(const wcns_handle *h);

/* Kernel launches issued by this handle since creation (host-side count). */
long long wcns_launch_count(const wcns_handle *h);

/* One SSPRK3 step that allocates nothing (the paper has no counterpart:
 * this is a deployment aid).  Some callers cannot call cudaMalloc:
 * real-time loops, where an allocation can synchronise the whole device and
 * break the loop's deadline; host applications that hand a plugin a fixed
 * device-memory budget and forbid it to allocate more; and code that must
 * not create per-solver state at all (no handle to keep, no scratch to
 * free).  This entry point takes the grid, boundary set, fluids and
 * options directly (no handle) and advances the caller's device array W in
 * place by one step of size dt, exactly like wcns_rk3_step.  Its scratch (two stage states,
 * the RHS accumulator, the node cache in 2D/3D, step control and counters)
 * lives in one file-scope device array of WCNS_NOALLOC_MAX_DOUBLES doubles
 * (64 MiB) that every GPU loading the library holds until the process
 * exits; a problem needs 3 * nf * ncells doubles of it in 1D and
 * (3 * nf + 3) * ncells in 2D/3D (up to 559,240 cells in 1D, 399,457 in
 * 2D, 349,525 in 3D) and larger ones are rejected with WCNS_E_TOO_LARGE
 * before any GPU work.
 * The first call on a device looks the array's device address up once
 * (cudaGetSymbolAddress with that device current); make that first call
 * before any stream capture.  Every call shares the one array and finds
 * the previous call's contents there: the counters are cleared on entry,
 * the rest is overwritten before it is read.  Calls whose work overlaps on
 * the GPU (other streams, other host threads) race on the array and must
 * be serialised by the caller.  opt may be NULL (defaults).  Asynchronous
 * on opt->stream: no host memory is read by the device and nothing is
 * waited for (uniform Dirichlet states travel as kernel arguments). */
#define WCNS_NOALLOC_MAX_DOUBLES (8ll * 1024 * 1024)
int wcns_rk3_step_noalloc(const wcns_grid *grid, const wcns_bcs *bcs, double gamma_g, double gamma_l,
                          double pinf_l, const wcns_options *opt, double *W, double dt);

/* Per-kernel timing (tracing aid, not part of the method).  When enabled,
 * every directional sweep launch is bracketed by CUDA events on the
 * handle's stream; wcns_profile_read synchronises, sums the durations per
 * sweep direction since the previous read, and clears them.  capacity is
 * the number of launches that can be recorded between reads (events are
 * created here, once); 0 disables.  Returns WCNS_E_CUDA if the events
 * cannot be created. */
typedef struct {
  long long launches[3];  /* sweep launches per direction x, y, z */
  double ms[3];           /* summed device time per direction, milliseconds */
  long long dropped;      /* launches beyond capacity, not timed */
} wcns_profile;
int wcns_profile_enable(wcns_handle *h, int capacity);
int wcns_profile_read(wcns_handle *h, wcns_profile *out);

/* Verification aid (not part of the method; the paper has no
 * counterpart): q[i] = a[i] / b[i] for n elements of the DEVICE arrays a,
 * b, q, computed with the FP64 sweeps' own division routine (an FP32
 * reciprocal seed, one Newton-Raphson step and one remainder correction,
 * within one unit in the last place of the IEEE quotient; IEEE division
 * outside its range), so that tests can compare it with CUDA's division.
 * Asynchronous on `stream` (a cudaStream_t, NULL = default). */
int wcns_check_division(const double *a, const double *b, double *q, long long n, void *stream);

/* Verification aid (not part of the method): the FP64 sweeps skip the
 * limiters of Secs. 5.1-5.2 (Algorithms 1-6) where an FP32 test from
 * truncated operands, with a rigorous error margin, certifies that every
 * threshold test passes.  This call evaluates that certification and the
 * FP64 limiter on the same inputs, n cases, NF = ndim + 4 conservative
 * components (a1r1, a2r2, momentum, E, a1), tolerances eps_ar, eps_a,
 * eps_rc (hard-switch tolerances equal to them), mixture EOS as in
 * wcns_create:
 *   kind 0, interpolation limiter: row i = W_node | W_interp (2 NF
 *     doubles); exact[i] = 1 if Algorithms 1-3 and the hard switch leave
 *     W_interp unchanged;
 *   kind 1, flux limiter with a given first-order flux: row i = W_i |
 *     W_{i+1} | F_i | F_{i+1} | G^{HLLC,-} | G^{HLLC,+} | G^- | G^+ |
 *     lambda (8 NF + 1 doubles; the alpha components of F are taken as 0,
 *     the other components of G^{HLLC,+} and G^+ from G^{HLLC,-} and G^-,
 *     as the sweeps form them; the certification takes G^HLLC to within
 *     its FP32 truncation); exact[i] = 1 if Algorithms 4-6 and the hard
 *     switch leave G^-, G^+ unchanged;
 *   kind 2, flux limiter from node states, as the sweeps run it: row i =
 *     node i | node i+1 | F_i | F_{i+1} | G | G^-_alpha | G^+_alpha |
 *     lambda, a node being W (NF), velocity (ndim), p, c (2 (NF + ndim
 *     + 2) + 3 NF + 3 doubles; G: the shared components of G^- and G^+,
 *     its alpha component unused; the flux direction is the last axis).
 *     The sweeps' certification evaluates the first-order HLLC flux (Sec.
 *     3.2) in FP32 with error bounds; exact[i] = 1 if the FP64 flux and
 *     Algorithms 4-6 with the hard switch leave G^-, G^+ unchanged;
 *   cert[i] = 1 if the sweeps' certification skips that limiter.
 * Sound means cert[i] = 1 implies exact[i] = 1.  rows, cert, exact: DEVICE
 * arrays (n rows; n ints each).  Asynchronous on `stream` (a cudaStream_t,
 * NULL = default).  Returns WCNS_E_INVALID_ARG for ndim outside 1..3, kind
 * outside 0..2, n < 0, null arrays with n > 0, tolerances negative or not
 * finite, or an EOS that wcns_create rejects. */
int wcns_check_limiter_cert(int ndim, int kind, const double *rows, long long n, double eps_ar, double eps_a,
                            double eps_rc, double gamma_g, double gamma_l, double pinf_l, int *cert, int *exact,
                            void *stream);

const char *wcns_strerror(int status);
void wcns_destroy(wcns_handle *h);

/* ------------------------------------------------------------------------
 * Batched mode: many independent 1D or 2D problems advanced together.
 * In 1D each problem k has ncells[k] cells on [lo[k], hi[k]] with the boundary
 * kinds bc_lo / bc_hi (TRANSMISSIVE, PERIODIC or SYMMETRY), and shares the fluid
 * pair.  States are packed one after another: the packed device array has
 * 5 rows of total = sum(ncells) doubles (SoA [5][total]); problem k
 * occupies columns offsets[k] .. offsets[k] + ncells[k] - 1 with
 * offsets[k] = sum_{j<k} ncells[j].  Every problem takes its own CFL time
 * step dt_k = cfl * dx_k / max(|u| + c) (Sec. 3.3, 1D).
 * ------------------------------------------------------------------------ */
typedef struct wcns_batch wcns_batch;

/* ncells: host array of nprob sizes (each >= 1); lo/hi: host arrays of
 * nprob doubles; bc_lo/bc_hi: TRANSMISSIVE, PERIODIC (both periodic or
 * neither) or SYMMETRY (then every problem needs >= 3 cells).  Copies the problem table and one (problem, tile) work list per
 * candidate tile length to the device and allocates the stage states and a
 * tuning copy (four packed states in all). */
int wcns_batch_create(int nprob, const int *ncells, const double *lo, const double *hi, int bc_lo,
                      int bc_hi, double gamma_g, double gamma_l, double pinf_l, wcns_batch **out);
/* Problems of one or two dimensions (Sec. 3.3: each problem takes its own
 * CFL step dt_k = cfl / sum_d max(|u_d| + c)/dx_{k,d} and its own
 * directional split lambda_d).  n, lo and hi are HOST arrays of
 * nprob * ndim values, problem-major (n[k * ndim + d]; d = 0 is x), each
 * n >= 1 (and <= 2^20 an axis in 2D), hi > lo.  bcs holds one boundary set
 * for every problem: TRANSMISSIVE, PERIODIC (both faces of an axis) or
 * SYMMETRY (n >= 3 on that axis); DIRICHLET is not provided in batches
 * (WCNS_E_INVALID_ARG).  Packed state: nf = ndim + 4 rows of total =
 * sum_k prod_d n[k][d] doubles; problem k occupies columns offsets[k] ..
 * offsets[k] + prod_d n[k][d] - 1 (offsets[k] = the cells of the problems
 * before it), stored x fastest like a single grid's state.  ndim = 1 is
 * wcns_batch_create with the axis-0 kinds of bcs; ndim = 3 returns
 * WCNS_E_UNSUPPORTED.  In 2D every stage is one persistent launch per
 * direction over a work list of (problem, tile) (x tiles of 4 rows x 58
 * cells, y tiles of 8 columns x 26 cells), and the device holds the
 * problem tables, three packed states and the RHS accumulator besides the
 * caller's, a tuning copy, and the mixed sweeps' node cache (24 bytes a
 * cell).  A problem advanced in a batch equals the same problem advanced
 * alone through wcns_create / wcns_advance_steps, step for step. */
int wcns_batch_create_grids(int ndim, int nprob, const int *n, const double *lo, const double *hi,
                            const wcns_bcs *bcs, double gamma_g, double gamma_l, double pinf_l,
                            wcns_batch **out);
int wcns_batch_set_options(wcns_batch *b, const wcns_options *opt);
/* Advance every problem by nsteps SSPRK3 steps in place (device array
 * W_packed).  Each stage is one persistent launch over all problems; one
 * step (dt update + three stages) is captured once into a CUDA graph and
 * replayed.  The first call tunes the tile length (63, 127 or 255 cells)
 * and the persistent grid (1, 2, 4 or 8 blocks per SM; 2D: 1 up to the
 * occupancy limit) by timing trial steps on the tuning copy; make it
 * before any stream capture of the
 * caller's.  t_out: optional DEVICE array of nprob doubles; each problem's
 * step sizes are added to it.  Ordered after the caller's pending work on
 * the options' stream, and that stream waits for it; synchronises once at
 * the end and returns WCNS_E_NONFINITE / WCNS_E_INADMISSIBLE as described
 * at the top (every problem takes all nsteps steps either way). */
int wcns_batch_advance(wcns_batch *b, double *W_packed, int nsteps, double cfl, double *t_out);
/* The autotuner's choice: cells per tile and persistent grid size (2D:
 * the cells of an x tile and the blocks of the persistent sweeps before
 * the cap by their work lists); WCNS_E_UNSUPPORTED before the first
 * advance. */
int wcns_batch_tuning(const wcns_batch *b, int *tile_cells, int *grid);
int wcns_batch_get_stats(wcns_batch *b, wcns_stats *out);
long long wcns_batch_total_cells(const wcns_batch *b);
long long wcns_batch_launch_count(const wcns_batch *b);
void wcns_batch_destroy(wcns_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* WCNS_H */
