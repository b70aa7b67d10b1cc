/*
 * m1.h -- C ABI of libm1: one implicit time step of the gray M1 moment model
 * for radiative transfer, solved on one GB300 GPU by the nonlinear FAS
 * geometric multigrid of Bloch, Tremblin, Gonzalez & Audit, "Towards a
 * multigrid method for the M1 model for radiative transfer" (arXiv:2208.14703).
 *
 * The unknowns per cell are the radiative energy E, the radiative flux
 * F = (Fx, Fy) and the gas temperature T (Section 2.1, Eq. (3)); the scheme is
 * the backward-Euler Rusanov (HLL with speeds +-c) finite volume scheme of
 * Section 2.2, Eq. (6), on a uniform Cartesian grid, plus backward-Euler
 * absorption (sigma_a) / scattering (sigma_s) sources coupling E to T.  The
 * paper itself sets every opacity to zero; with sigma_a = sigma_s = 0 the
 * operator is exactly its Eq. (6).
 *
 * Conventions for every entry point:
 *  - Arrays are row-major [ny][nx] (index j*nx + i), FP64, one array per field.
 *    In 1D (dim = 1) ny must be 1 and Fy may be NULL.
 *  - `on_device` = 0: host pointers (any host memory; pinned is faster);
 *    `on_device` = 1: CUDA device pointers on the grid's device, read or
 *    written in stream order on the grid's stream.
 *  - Input arrays are copied; the caller keeps ownership of every pointer it
 *    passes.  The grid owns all device memory it allocates and frees it in
 *    m1_destroy_grid.  The library never frees caller memory.
 *  - Every call returns an m1_status; nothing is thrown across the ABI.
 *  - A grid is used by one host thread at a time (calls on one grid are not
 *    thread safe); different grids are independent.
 */
#ifndef M1_H
#define M1_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct m1_grid* m1_grid_t;

typedef enum {
    M1_OK = 0,
    M1_PENDING = 1,
    M1_ERR_INVALID_ARG = -1,          /* bad size, pointer, level count or parameter */
    M1_ERR_NONADMISSIBLE_INPUT = -2,  /* E <= 0, T <= 0, |F| > c E, sigma < 0 or non-finite */
    M1_ERR_OOM = -3,                  /* device allocation failed */
    M1_ERR_NOT_CONVERGED = -4,        /* max_cycles reached; the last iterate is kept */
    M1_ERR_CUDA = -5,                 /* a CUDA call failed (see m1_last_error) */
    M1_ERR_TIMEOUT = -6,
    M1_ERR_REJECTED = -7
} m1_status;

/* Boundary conditions per wall (west, east, south, north).  The paper only asks
 * for "appropriate boundary conditions" (Section 4.2); each is one ghost cell:
 *   PERIODIC wrap; REFLECT mirror cell with the wall-normal flux negated;
 *   NEUMANN copy of the boundary cell; INFLOW prescribed (E, Fx, Fy) set by
 *   m1_set_inflow (T copied from the boundary cell). */
typedef enum { M1_BC_PERIODIC = 0, M1_BC_REFLECT = 1, M1_BC_NEUMANN = 2, M1_BC_INFLOW = 3 } m1_bc;

/* M1_FP64: every level in FP64.  M1_MIXED: the iterate, the right-hand side,
 * the opacities and the solution stay in FP64 at the fine level; each cycle
 * forms the fine defect r = b - A(v), runs one FP32 V-cycle for the correction
 * e of A(w + e) - A(w) = r around the base w = fl32(v) (correction form), and
 * adds v += e in FP64 with the damping of Eq. (34).  The defect of the cycles is
 * formed in double-word FP32 (about 48 bits) when tol ||r_0|| > 5e-12 diag ||b||,
 * where its noise (measured at most ~3e-14 diag ||b||) stays below 1% of the stop
 * test's threshold, and in FP64 otherwise; the defect of the step's start is
 * FP64.  The stop test, the dtau control and the result are FP64 quantities. */
typedef enum { M1_FP64 = 0, M1_MIXED = 1 } m1_precision;

/* Grid description.  lx, ly: domain lengths (cells hx = lx/nx, hy = ly/ny);
 * lmax: number of multigrid levels counting the fine grid (Section 5, "L_max";
 * lmax = 1 is plain Jacobi); nx (and ny in 2D) must be divisible by 2^(lmax-1).
 * c, a_r, c_v: speed of light, radiation constant, gas heat capacity. */
typedef struct {
    int dim, nx, ny;
    double lx, ly;
    int bc[4];
    int lmax;
    double c, a_r, c_v;
    int precision;   /* m1_precision */
} m1_grid_desc;

/* Solver parameters of Algorithm 4 (Appendix A).  Section 5 fixes nu0 = 3 (fine
 * pre/post smoothing sweeps), nu_l = 1 (Jacobi sweeps per pseudo-time step on
 * coarse levels), m_pseudo = 3 (pseudo-time steps), dtau0 = 1e-3.  The paper
 * leaves the rest open; defaults (m1_default_params): m_coarse = 3, grow 1.1,
 * shrink 0.5 (Algorithm 4), eps_i = 1e-2, eps_d = 1e-4, tol = 1e-8 (relative to
 * the initial residual), dtau clamped to [1e-12, 1e6], theta_ex = 0.5 (fraction
 * of the admissible explicit pseudo-time step), theta_c = 0.5 (damping of an
 * inadmissible prolongated cell), max_cycles = 20000, dtau_rule = M1_DTAU_ABS,
 * cycle = M1_CYCLE_V.
 * dtau_rule selects the residual change that drives dtau after each cycle:
 *   M1_DTAU_ABS     delta = | ||r_k|| - ||r_{k-1}|| | / ||r_0|| (as Algorithm 4
 *                   prints it): a fast-growing residual also grows dtau;
 *   M1_DTAU_SIGNED  delta = (||r_{k-1}|| - ||r_k||) / ||r_0||, the decrease (as
 *                   Section 4 words the rule: increase dtau when the residual
 *                   decreases fast enough, decrease it when it decreases slowly),
 *                   so a growing residual halves dtau.
 * Then dtau *= grow if delta > eps_i, dtau *= shrink if delta < eps_d.
 * cycle selects the cycle shape (default M1_CYCLE_V, the paper's; Section 6.3
 * names W- and F-cycles as alternatives).  The coarse-grid corrections of level
 * l are one visit of level l + 1 (V), two visits, the second continuing from
 * the corrected iterate with the same FAS right-hand side (W), or an F-visit
 * followed by such a repeated V-visit (F); the coarsest level is visited once
 * per correction, so with lmax <= 2 the shapes coincide.  Each visit of a
 * coarse level smooths m_pseudo pseudo-time steps before and after its
 * corrections (the coarsest: m_coarse); the fine level is visited once per
 * cycle whatever the shape. */
enum { M1_DTAU_ABS = 0, M1_DTAU_SIGNED = 1 };
enum { M1_CYCLE_V = 0, M1_CYCLE_W = 1, M1_CYCLE_F = 2 };
typedef struct {
    int nu0, nu_l, m_pseudo, m_coarse;
    double dtau0, grow, shrink, eps_i, eps_d, tol, dtau_min, dtau_max, theta_ex, theta_c;
    int max_cycles;
    int dtau_rule;
    int cycle;
} m1_solve_params;

/* Statistics of one implicit step.  res0/res: ||r|| before the first and after
 * the last cycle, ||r||^2 = sum over cells h^d (rE^2 + |rF|^2/c^2 + rT^2);
 * sweeps: fine-level Jacobi sweeps; ms: device time of the step. */
typedef struct {
    int cycles;
    double res0, res, dtau_final;
    long long sweeps;
    double ms;
    int status;
    unsigned int newton_fail, damped;
    long long launches;   /* kernels this call launched (cycles queued past convergence included) */
} m1_step_stats;

/* Fills *p with the defaults listed above. */
m1_status m1_default_params(m1_solve_params* p);

/* Allocates the level hierarchy of `desc` on the current CUDA device.
 * cuda_stream: a cudaStream_t to run on, or NULL for a stream owned by the grid.
 * Errors: INVALID_ARG (sizes, lmax, dim), OOM, CUDA. */
m1_status m1_create_grid(const m1_grid_desc* desc, void* cuda_stream, m1_grid_t* out);
m1_status m1_destroy_grid(m1_grid_t g);

/* Sets the state v^n (E, Fx, Fy, T per cell) and the opacities sigma_a,
 * sigma_s (constant during a step; restricted by full weighting to the coarse
 * levels).  Checks admissibility (Eq. (7): E > 0, |F| <= c E; and T > 0,
 * sigma >= 0, all finite): NONADMISSIBLE_INPUT leaves the grid unchanged.
 * sig_a / sig_s may be NULL to keep the previous opacities. */
m1_status m1_set_state(m1_grid_t g, const double* E, const double* Fx, const double* Fy,
                       const double* T, const double* sig_a, const double* sig_s, int on_device);

/* Prescribed ghost state of an inflow wall (side 0..3 = W, E, S, N): host
 * arrays of length ny (W/E) or nx (S/N).  The coarse levels see its
 * full-weighting restriction along the wall. */
m1_status m1_set_inflow(m1_grid_t g, int side, const double* E, const double* Fx, const double* Fy);

/* Copies the current state out (v^{n+1} after a step). Fy may be NULL. */
m1_status m1_get_state(m1_grid_t g, double* E, double* Fx, double* Fy, double* T, int on_device);

/* One implicit time step of length dt (Algorithm 4): b = (E^n, F^n, C_v T^n),
 * cycles (of the shape params->cycle) until ||r|| <= tol ||r_0||, the state becomes v^{n+1}; no cycle at all
 * when ||r_0|| <= 1e-14 (1 + c dt/hx + c dt/hy) ||b|| (already solved to the
 * rounding of A, e.g. an equilibrium state E = a_r T^4, F = 0), the state
 * becomes v^{n+1}.  params may be NULL for the defaults; stats may be NULL.
 * Returns NOT_CONVERGED after max_cycles with the last (admissible) iterate
 * kept as the state.  Blocks until the step is done. */
m1_status m1_implicit_step(m1_grid_t g, double dt, const m1_solve_params* params,
                           m1_step_stats* stats);

/* Algorithm 1 alone (the Jacobi method of Section 3, timed in the paper's
 * Table 1): b = (E, F, C_v T) of the current state, then `sweeps` nonlinear
 * Jacobi sweeps of A(v) = b starting from the current state, which becomes the
 * result.  Asynchronous: the sweeps are queued on the grid's stream and the call
 * returns; synchronise that stream before reading the state from another stream.
 * On a MIXED grid the sweeps run in FP32 on the correction equation
 * A(w + e) - A(w) = r (w = the state rounded to FP32, r = b - A(v) in FP64,
 * e = 0 at the start), and the state becomes v + e in FP64 (damped like the
 * prolongation, Eq. (34), where v + e is not admissible). */
m1_status m1_jacobi(m1_grid_t g, double dt, int sweeps);

/* ||b - A(v)|| (the norm above) of the current state v for a step of length dt,
 * with b the right-hand side of the last implicit step taken on this grid with
 * the same dt, or b = (E, F, C_v T) of the current state if there was none. */
m1_status m1_residual_norm(m1_grid_t g, double dt, double* out);

/* Residual history of the last step: hist[k] = ||r_k||, k = 0..cycles (up to
 * len entries); dtau[k] = implicit pseudo-time step used in cycle k+1. */
m1_status m1_step_history(m1_grid_t g, double* hist, double* dtau, int len);

/* ---- batches: many independent instances stepped together ---------------------
 * A batch holds `count` instances (grids) that share lmax and precision; sizes,
 * dimension (1D and 2D may mix), walls, constants and time steps are per
 * instance.  One persistent launch per level and kernel serves all instances
 * (their strips of cells are items of a device work list), one CUDA graph holds the
 * V-cycle, and each instance keeps its own dtau_im, residual norms and stop flag
 * (Algorithm 4 per instance): an instance's result is the same alone and in a
 * batch.  Index arguments are 0 .. count-1. */
typedef struct m1_batch* m1_batch_t;
m1_status m1_create_batch(const m1_grid_desc* descs, int count, void* cuda_stream, m1_batch_t* out);
m1_status m1_destroy_batch(m1_batch_t b);
m1_status m1_batch_set_state(m1_batch_t b, int index, const double* E, const double* Fx,
                             const double* Fy, const double* T, const double* sig_a,
                             const double* sig_s, int on_device);
m1_status m1_batch_set_inflow(m1_batch_t b, int index, int side, const double* E, const double* Fx,
                              const double* Fy);
m1_status m1_batch_get_state(m1_batch_t b, int index, double* E, double* Fx, double* Fy, double* T,
                             int on_device);
/* One implicit step of every instance; dt[count]; stats[count] (may be NULL).
 * Returns when every instance has converged (or reached max_cycles:
 * NOT_CONVERGED if any did). */
m1_status m1_batch_implicit_step(m1_batch_t b, const double* dt, const m1_solve_params* params,
                                 m1_step_stats* stats);

/* ---- serving: many simulations stepping on one GPU with continuous batching ----
 * A server holds two lanes, each an engine of max_slots slots (level count
 * lmax, precision FP64 or MIXED; the structural solver parameters nu0,
 * m_pseudo, m_coarse are fixed at creation, the others are per request) with a
 * scheduler thread and a CUDA stream of its own: requests of at most
 * small_cells fine cells go to the small lane (a stream the server creates at
 * the highest priority), the others to the large lane (cuda_stream, or a
 * stream of the server's when NULL); small_cells = 0 puts every request in the
 * large lane.  A small request's V-cycles thus never wait for the levels of
 * the largest instances.  m1_serve_submit queues a caller's grid (its state
 * set, same lmax and precision) for nsteps implicit steps of length dt.  Each
 * lane admits its queued requests in arrival order into free slots while the
 * level hierarchies of both lanes fit hbm_budget_bytes, copies the state in on
 * the device (it stays resident for all steps), and launches V-cycle graphs
 * over every active slot, one cycle at a time; while a cycle runs it reads the
 * control blocks left by the previous one: a slot whose step converged starts
 * its next step (behind the running cycle), and a finished request's state is
 * copied back into its grid and its slot and budget are freed, all between
 * V-cycles, so requests arriving while others run join the running batch.
 * The caller must not use a submitted grid until its ticket completes.
 * Submit, poll, wait and stats are thread safe.  Step latency is the host time
 * from the start of a step to the reading that sees it converged. */
typedef struct m1_server* m1_server_t;
typedef struct {
    long long requests_done, steps_done, cycles;
    double wall_s;          /* from the first admission to the last completed step */
    double solves_per_s;    /* steps_done / wall_s */
    double p50_ms, p99_ms, mean_ms;   /* step latency */
    int active, queued;
    long long bytes_in_use, bytes_peak;   /* budgeted device bytes of admitted requests */
} m1_server_stats;
/* INVALID_ARG: max_slots < 1, lmax outside 1..20, a zero budget, small_cells < 0,
 * an unknown precision or invalid structural parameters. */
m1_status m1_server_create(size_t hbm_budget_bytes, int max_slots, int lmax, int precision,
                           const m1_solve_params* structure, long long small_cells,
                           void* cuda_stream, m1_server_t* out);
/* REJECTED: the grid alone exceeds the budget; INVALID_ARG: precision, lmax or
 * structural parameters differ from the server's. */
m1_status m1_serve_submit(m1_server_t s, m1_grid_t g, int nsteps, double dt,
                          const m1_solve_params* params, unsigned long long* ticket);
/* PENDING while queued or running; then OK, NOT_CONVERGED (a step reached
 * max_cycles; the request stops there) or the server's error. */
m1_status m1_serve_poll(m1_server_t s, unsigned long long ticket, int* steps_done,
                        m1_step_stats* last);
/* Blocks until the ticket completes or timeout_s passes (TIMEOUT). */
m1_status m1_serve_wait(m1_server_t s, unsigned long long ticket, double timeout_s);
m1_status m1_server_get_stats(m1_server_t s, m1_server_stats* out);
/* Finishes every submitted request, then stops the scheduler and frees the engine. */
m1_status m1_server_destroy(m1_server_t s);

/* ---- autotuning of the sweep kernels' strip shape ----
 * The Jacobi and pseudo-time sweeps (Algorithm 1, Algorithm 3) of a 2D level
 * give each warp a strip of 30 columns and `strip_rows` rows.  m1_autotune
 * times one sweep of a synthetic admissible n x n level (n = 16 .. 2048; the
 * FP32 correction form also 4096) for
 * strip heights 1, 2, 4, 8, 12, 16, 24, 32, 48, 64, 96, 128 (at most n), for
 * FP64 (kind 0) and for the FP32
 * correction form of the mixed path (kind 1, also both row stagings), and keeps
 * the fastest shape per size class (grids of about the same cell count) in a
 * process-wide table that grids, batches and servers created afterwards use.
 * Before any tuning the height is ny / 64 (between 1 and 16), registers.  The height does not change any
 * arithmetic (results are bitwise identical for every height); the two FP32
 * stagings are two kernels whose FP32 roundings may differ in the last bit, so
 * mixed-precision results agree to rounding.  Runs on `cuda_stream`
 * (NULL: a stream of its own) and blocks; takes well under a second.  Writes up
 * to max_entries entries (one per kind and size) to `out` and their count to
 * *n_entries. */
typedef struct {
    int kind;            /* 0: FP64, 1: FP32 correction form */
    int n;               /* level size n x n */
    int strip_rows;      /* chosen height */
    int staging;         /* kind 1: 0 = rows loaded into registers one row ahead,
                            1 = rows copied asynchronously into a shared-memory ring
                            three rows ahead (fine-level sweeps); kind 0: 0 */
    double ms;           /* time of one sweep with the chosen shape */
    double ms_default;   /* time with the untuned shape (NAN if not a candidate) */
} m1_tune_entry;
m1_status m1_autotune(void* cuda_stream, m1_tune_entry* out, int max_entries, int* n_entries);
/* Installs entries (e.g. restored from an earlier m1_autotune); strip_rows = 0
 * restores the default for that kind and size class; INVALID_ARG for a height
 * above 256, an unknown kind or staging. */
m1_status m1_set_tuning(const m1_tune_entry* in, int n);
/* The strip height a new nx x ny level of the given kind would take. */
m1_status m1_strip_rows(int kind, int nx, int ny, int* rows);

/* ---- arithmetic peak probe (a roofline denominator; not a step of the method) ----
 * The FP64 kernels of this library are bound by the FP64 pipe, not by HBM; this
 * call measures that pipe's ceiling on the current device.  A kernel of
 * independent fused multiply-add chains (8 per thread, no chain waits on
 * another; 152 x 8 blocks of 256 threads, 4096 rounds) runs `reps` timed
 * launches after one untimed one, each timed with CUDA events on cuda_stream
 * (NULL: the legacy default stream); *ops_per_s = FMA instructions per second
 * summed over lanes (one FMA is one pipe operation, two flops) of the median
 * launch.  precision M1_FP64: DFMA; M1_MIXED: FP32 FFMA.  Allocates and frees a
 * small output buffer.  INVALID_ARG: NULL output, reps < 1 or an unknown
 * precision; CUDA: a failed allocation, launch or event (m1_last_error). */
m1_status m1_probe_fma_peak(int precision, void* cuda_stream, int reps, double* ops_per_s);

/* ---- FP64 <-> double-word FP32 conversions (host runs of the device code) ----
 * The mixed path keeps double-word copies (hi + lo, two FP32 numbers) of its
 * fine-level FP64 arrays and widens the FP32 cycle's correction to FP64.  It
 * does both with integer and FP32 operations on the bit patterns instead of
 * conversion instructions, which GB300 issues at the FP64 rate (1/64 of FP32).
 * These entry points run the same inline functions on the host, so that they
 * can be checked without a GPU:
 *   m1_dw_split:  hi[i] = fl32(x[i]), lo[i] = fl32(x[i] - hi[i]), both rounded
 *                 to nearest even (x[i] - hi[i] is exact in FP64);
 *   m1_f32_widen: y[i] = (double)x[i].
 * Host pointers to n >= 0 elements; nothing is allocated.  INVALID_ARG: n < 0,
 * or a NULL pointer with n > 0. */
m1_status m1_dw_split(const double* x, long long n, float* hi, float* lo);
m1_status m1_f32_widen(const float* x, long long n, double* y);

/* ---- the kernels' per-element arithmetic on the device (for checks) ----
 * y[i] = f(x[i]) for 0 <= i < n, computed on the device by the inline functions
 * the kernels call, so that tests can hold them against correctly rounded
 * results (IEEE division and square root, IEEE conversions):
 *   M1_FN_RCP64     double -> double: 1/x, the hardware estimate with one
 *                   third-order correction (positive normal x);
 *   M1_FN_SQRT64    double -> double: sqrt(x), the same construction;
 *   M1_FN_RCP32     float -> float: the approximate FP32 reciprocal;
 *   M1_FN_SQRT32    float -> float: the approximate FP32 square root;
 *   M1_FN_DW_SPLIT  double -> float pairs: y[2i] = hi, y[2i+1] = lo (as m1_dw_split);
 *   M1_FN_WIDEN     float -> double (as m1_f32_widen).
 * x and y are device pointers (y holds n results, 2n floats for the split);
 * one launch on cuda_stream (NULL: the legacy default stream), and the call
 * returns after synchronising that stream.  INVALID_ARG: n < 0, a NULL pointer
 * with n > 0, or an unknown fn; CUDA: the launch or the kernel failed
 * (m1_last_error). */
enum { M1_FN_RCP64 = 0, M1_FN_SQRT64 = 1, M1_FN_RCP32 = 2, M1_FN_SQRT32 = 3, M1_FN_DW_SPLIT = 4,
       M1_FN_WIDEN = 5 };
m1_status m1_op_elementwise(int fn, const void* x, long long n, void* y, void* cuda_stream);

/* ---- single-kernel entry points (one kernel on caller data, for checks) ----
 * Stateless: each call allocates its own device buffers for `desc` (lmax is
 * ignored; precision selects FP64 or FP32 arithmetic), runs one kernel on the
 * current device and copies the result to host memory.  Host arrays are planar
 * [4][ny*nx] (E, Fx, Fy, T) for states and [2][ny*nx] (sigma_a, sigma_s) for
 * opacities; inflow is [4 walls][3 fields][max(nx, ny)] or NULL.
 *
 * m1_op_level modes:
 *   M1_OP_APPLY     out = A(state)                         (Eq. (12) + sources)
 *   M1_OP_RESIDUAL  out = rhs - A(state), *norm = ||out||  (Eq. (13))
 *   M1_OP_FAS_RHS   out = A(state) + rhs                   (Eq. (24))
 *   M1_OP_JACOBI    out = one Jacobi sweep of A(u) = rhs from u = state
 *                                                          (Algorithm 1)
 *   M1_OP_PSEUDO    out = one pseudo-time step with source f = rhs: explicit
 *                   limited half then one Jacobi sweep of u + dtau A(u) = u~
 *                   (Eq. (30), Algorithm 3), theta_ex = theta
 *   M1_OP_RESIDUAL_DW  as M1_OP_RESIDUAL, evaluated in double-word FP32 (pairs
 *                   hi + lo of FP32 numbers, about 48 bits; FP64 descriptors
 *                   only): the arithmetic of the mixed path's defect when its
 *                   tolerance lies far above that format's noise floor
 * For M1_OP_JACOBI and M1_OP_PSEUDO, *norm (if not NULL) receives the number of
 * cells whose local E-T solve did not converge to a finite positive T. */
enum { M1_OP_APPLY = 0, M1_OP_RESIDUAL = 1, M1_OP_FAS_RHS = 2, M1_OP_JACOBI = 3, M1_OP_PSEUDO = 4,
       M1_OP_RESIDUAL_DW = 5 };
m1_status m1_op_level(const m1_grid_desc* desc, const double* inflow, double dt, const double* sig,
                      const double* state, const double* rhs, int mode, double dtau, double theta,
                      double* out, double* norm);

/* ---- 3D single-level operators (one pass on caller data, for checks) ----
 * A 3D grid of nx x ny x nz cells on [0,lx] x [0,ly] x [0,lz]; walls bc[6] =
 * (x low, x high, y low, y high, z low, z high), each periodic, reflecting or
 * Neumann (m1_op_level3 takes no inflow wall; the 3D grids below do).  States are planar [5][nz*ny*nx] doubles
 * (E, Fx, Fy, Fz, T; index (k*ny + j)*nx + i), opacities [2][nz*ny*nx]
 * (sigma_a, sigma_s).  The operator is the 2D one on three axes: the Rusanov
 * faces of Eq. (6) with the 3x3 closure of Eq. (5), transport diagonal
 * 1 + c dt (1/hx + 1/hy + 1/hz), the same sources and local E-T solve.
 *   M1_OP3_APPLY     out = A(state)
 *   M1_OP3_RESIDUAL  out = rhs - A(state)
 *   M1_OP3_JACOBI    out = `sweeps` Jacobi sweeps of A(u) = rhs from u = state
 *                    (Algorithm 1)
 * on_device = 0: host arrays (copied in and out; the call returns when done);
 * 1: device arrays, stream-ordered on cuda_stream (the call still waits for its
 * own work).  Each call allocates its own device buffers.  ms (may be NULL):
 * device time of the operator passes alone (closure + operator per sweep).
 * INVALID_ARG: a size < 1 or above 2^31 cells, a non-positive length, dt or
 * constant, an inflow or unknown wall, an unknown mode, sweeps < 1 for JACOBI,
 * a NULL array the mode needs.  The state must be admissible. */
typedef struct {
    int nx, ny, nz;
    double lx, ly, lz;
    m1_bc bc[6];
    double c, a_r, c_v;
} m1_grid3_desc;
enum { M1_OP3_APPLY = 0, M1_OP3_RESIDUAL = 1, M1_OP3_JACOBI = 2 };
m1_status m1_op_level3(const m1_grid3_desc* desc, double dt, const double* sig,
                       const double* state, const double* rhs, int mode, int sweeps,
                       double* out, int on_device, void* cuda_stream, double* ms);

/* ---- 3D grids: one implicit step of Algorithm 4 (Appendix A) in three
 * dimensions.  Section 4.2 writes the transfers for d = 1, 2, 3 (R = 2^-d P^T);
 * the operator, closure, sources, local solve, pseudo-time smoother, damping,
 * norm and dtau_im control are those of the 2D grid on three axes (Rusanov
 * faces of Eq. (6) on x, y and z, the 3x3 closure of Eq. (5), 27-point full
 * weighting, tensor-product prolongation with the damping of Eq. (34)).  FP64.
 *
 * m1_create_grid3: levels 0 .. lmax-1 of `desc` (lmax counts the grids; nx, ny
 *   and nz divisible by 2^(lmax-1)) on the current device; every wall periodic
 *   (in pairs), reflecting, Neumann or inflow; cuda_stream NULL: a stream of its
 *   own.  INVALID_ARG: sizes, lengths or constants out of range, an unknown or
 *   unpaired periodic wall, more than 2^31 cells; OOM.
 * m1_grid3_set_state: v^n from planar [5][nz*ny*nx] doubles (E, Fx, Fy, Fz, T;
 *   index (k*ny + j)*nx + i) and opacities [2][nz*ny*nx] (sigma_a, sigma_s),
 *   host arrays (on_device = 0) or device arrays on the grid's stream (1); both
 *   are copied.  NONADMISSIBLE_INPUT: some E <= 0, T <= 0, |F| > c E, negative
 *   opacity or non-finite value (the state is then not usable for a step).
 * m1_grid3_set_inflow: the prescribed E, Fx, Fy, Fz of every inflow wall's face
 *   cells, host array [6 walls][4 fields][F], F = max(ny*nz, nx*nz, nx*ny), the
 *   face of a wall on axis d indexed b * n_a + a over its two other axes a < b;
 *   T of an inflow ghost is the mirror cell's.  Coarse levels take the
 *   full-weighting restriction of the face (1/4, 1/2, 1/4, ends copied) along
 *   each tangential axis.  Required before a step when a wall is an inflow wall;
 *   INVALID_ARG when none is.
 * m1_grid3_get_state: the current state into planar [5][nz*ny*nx] (host or device).
 * m1_grid3_implicit_step: v^n -> v^{n+1} in place, V-, W- or F-cycles to
 *   ||r|| <= tol ||r_0|| (params NULL: the defaults of m1_default_params;
 *   nu_l must be 1); stats as for m1_implicit_step.  NOT_CONVERGED after
 *   max_cycles (the last iterate kept); INVALID_ARG: dt <= 0, bad parameters,
 *   no state set, or a missing inflow profile.
 * m1_grid3_step_history: ||r_kappa|| for kappa = 0 .. cycles and the dtau_im of
 *   each cycle of the last step (first `len` entries).
 * A grid is used by one thread and stream at a time. */
typedef struct m1_grid3* m1_grid3_t;
m1_status m1_create_grid3(const m1_grid3_desc* desc, int lmax, void* cuda_stream, m1_grid3_t* out);
m1_status m1_destroy_grid3(m1_grid3_t g);
m1_status m1_grid3_set_state(m1_grid3_t g, const double* state, const double* sig, int on_device);
m1_status m1_grid3_set_inflow(m1_grid3_t g, const double* faces);
m1_status m1_grid3_get_state(m1_grid3_t g, double* state, int on_device);
m1_status m1_grid3_implicit_step(m1_grid3_t g, double dt, const m1_solve_params* params,
                                 m1_step_stats* stats);
m1_status m1_grid3_step_history(m1_grid3_t g, double* hist, double* dtau, int len);

/* Full weighting (Section 4.2, Eq. (21)/(22)) of a fine state (STATE ghosts) and
 * a fine residual (DIFF ghosts: zero at inflow walls) to the coarse grid
 * (nx/2 x ny/2; ny stays 1 in 1D).  Outputs are planar [4][coarse cells]. */
m1_status m1_op_restrict(const m1_grid_desc* fine, const double* inflow, const double* state,
                         const double* resid, double* coarse_state, double* coarse_resid);

/* Prolongation of the coarse correction uc - vc onto the fine iterate uf with
 * the damping of inadmissible cells (Eq. (18), Eq. (34), theta_c = theta);
 * *damped = number of damped cells. */
m1_status m1_op_prolong_correct(const m1_grid_desc* fine, const double* uc, const double* vc,
                                const double* uf, double theta, double* out, int* damped);

/* Residual norm without allocating device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc
 * where they need the norm -- a framework whose own pool owns all device
 * memory, or a latency-critical loop in which a cudaMalloc (which can
 * synchronise the whole device) is not allowed.
 * Computes ||b - A(v)|| (the norm of m1_step_stats) for a step of length dt on
 * the grid `desc` (lmax and precision ignored; FP64), from caller-owned device
 * arrays: state [4][ny*nx] planar (E, Fx, Fy, T), rhs [4][ny*nx], sig [2][ny*nx]
 * (sigma_a, sigma_s), inflow [4 walls][3][max(nx, ny)] (may be NULL when no wall
 * is INFLOW), and writes the norm to *norm_out, a device pointer.  Queued on
 * `cuda_stream` (NULL: the legacy default stream); returns without waiting.
 * It allocates nothing: the per-tile partial sums go to a fixed array of 65536
 * doubles (512 KiB) in the library's own device memory, which every GPU that
 * loads the library holds until the process exits.  A grid needing more than
 * 65536 tiles (32 x 8 cells in 2D, 256 in 1D; so at most 4096 x 4096 cells in
 * 2D) is rejected with INVALID_ARG and a message in m1_last_error.  Each call
 * overwrites the entries it reads, so nothing needs clearing, but all calls
 * share the array: calls whose kernels overlap on the GPU (unordered streams)
 * race on it.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call before
 * any stream capture. */
m1_status m1_residual_norm_noalloc(const m1_grid_desc* desc, double dt, const double* state,
                                   const double* rhs, const double* sig, const double* inflow,
                                   double* norm_out, void* cuda_stream);

/* Text of the last CUDA error seen by this thread's calls (static storage). */
const char* m1_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* M1_H */
