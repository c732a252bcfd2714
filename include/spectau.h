/*
 * spectau.h -- C ABI of the GB300 (sm_103a) IMEX spectral-tau timestep.
 *
 * The library advances first-order problems  M dt(X) + L X = F(X)  on a
 * Fourier(x) x Chebyshev(z) domain with the sparse generalized tau method
 * (paper Sec. "A general sparse tau method", Sec. "Initial value solver",
 * Eq. ivp).  Coefficient space splits into independent pencils, one per
 * Fourier wavenumber k_x (Sec. "Linear boundary value solver": the pencil
 * systems couple only through F).  Each pencil holds S variables x N_z
 * Chebyshev modes, n = S N_z unknowns.
 *
 * Conventions for every entry point:
 *  - every call returns an sp_status; on failure sp_last_error() returns a
 *    message describing the first error of the last call;
 *  - host arrays passed in are copied before the call returns; the caller
 *    keeps ownership;
 *  - device memory owned by the library is released by sp_destroy;
 *  - work is queued on the context's CUDA stream and runs asynchronously;
 *    device-side failures (singular pivot, non-finite state, bounded wait
 *    expiry) are latched in a device status word read by sp_sync_status;
 *  - a pointer passed with on_device = 1 must be device memory of the
 *    context's device, valid until the stream reaches the queued work;
 *  - there is no CPU fallback: without a usable CUDA device sp_create fails.
 *
 * Layouts (all little-endian, C order):
 *  - coefficient layout 'c': complex FP64 interleaved (re, im), indexed
 *    [p][m], p = 0 .. P-1 the stored k_x >= 0 modes (k_x = 2 pi p / L_x,
 *    Nyquist dropped, Sec. "Fourier basis"), m = 0 .. N_z-1 the Chebyshev
 *    mode (Sec. "Chebyshev basis");
 *    (3D: p = i_y N_x/2 + i_x, see sp_add_problem);
 *  - grid layout 'g': real FP64 indexed [iz][ix] (3D: [iz][iy][ix]) on the
 *    Gauss-Chebyshev nodes z_i = a + (b - a)(1 - cos(pi (i + 1/2) / N_gz)) / 2
 *    (ascending) and the Fourier nodes x_i = L_x i / N_gx, y_i = L_y i / N_gy.
 */
#ifndef SPECTAU_H
#define SPECTAU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sp_ctx sp_ctx;

typedef enum {
  SP_OK = 0,
  SP_ERR_ARG = -1,           /* invalid argument (checked on the host)        */
  SP_ERR_CUDA = -2,          /* a CUDA runtime call failed                    */
  SP_ERR_OOM = -3,           /* device allocation failed                      */
  SP_ERR_SINGULAR = -4,      /* zero pivot in a pencil factorization          */
  SP_ERR_NOT_FACTORED = -5,  /* sp_step with a dt that was not factored       */
  SP_ERR_NONFINITE = -6,     /* NaN or Inf in the state after a step          */
  SP_ERR_TIMEOUT = -7,       /* a bounded device wait expired                 */
  SP_ERR_STATE = -8          /* call out of order (e.g. step before setup)    */
} sp_status;

typedef enum { SP_FOURIER = 0, SP_CHEBYSHEV = 1 } sp_basis_kind;

/* One axis (Sec. "Spectral bases"): kind, coefficient count N_c, interval
 * [a, b] (Fourier: length b - a), dealias scale num/den (Sec. "Scaled
 * transforms & dealiasing"; 3/2 dealiases quadratic products). */
typedef struct {
  int32_t kind;
  int32_t n_coeff;
  double a, b;
  int32_t dealias_num, dealias_den;
} sp_basis;

/* IMEX schemes (Sec. "Timesteppers"): RK222 = ARS(2,2,2), RK111 and
 * RK443 = ARS(4,4,3) (third order, four stages, implicit diagonal 1/2: one
 * factorization serves every stage) of Ascher, Ruuth & Spiteri (1997);
 * SBDF1 .. SBDF4 of Wang & Ruuth (2008), constant step.  SBDFq takes its
 * first q - 1 steps at the orders the history allows (SBDF1, SBDF2, ...)
 * and keeps one factorization per order.  CNAB1 and CNAB2 (Crank-Nicolson
 * Adams-Bashforth, the same family and paper; Sec. "Multistep IMEX
 * integrators"): (M~ + dt/2 L~) X^{n+1} = (M~ - dt/2 L~) X^n
 * + dt (3/2 F^n - 1/2 F^{n-1}) (CNAB1: dt F^n, CNAB2's first step), one
 * factorization for both orders.  The adjoint entry points support RK222
 * and RK111; batched stepping every scheme. */
typedef enum {
  SP_RK222 = 0, SP_SBDF1 = 1, SP_SBDF2 = 2, SP_RK111 = 3, SP_RK443 = 4, SP_SBDF3 = 5, SP_SBDF4 = 6,
  SP_CNAB1 = 7, SP_CNAB2 = 8
} sp_scheme;

/* FP64: every stage in FP64.  MIXED: transforms and grid products in FP32,
 * pencil factorization, right-hand-side assembly and solves in FP64. */
typedef enum { SP_PREC_FP64 = 0, SP_PREC_MIXED = 1 } sp_precision;

/* Operators in bilinear right-hand-side terms (DY: three-dimensional
 * problems only). */
typedef enum { SP_OP_ID = 0, SP_OP_DX = 1, SP_OP_DY = 2 } sp_op;

/* Create a context on CUDA device `device`, queueing work on `cuda_stream`
 * (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream; NULL = the
 * legacy default stream).  *out receives the handle. */
sp_status sp_create(sp_ctx** out, int device, void* cuda_stream);

/* Synchronize the stream and release every resource of the context. */
sp_status sp_destroy(sp_ctx* ctx);

/* Message of the last failing call on this context ("" if none).  The
 * string is owned by the context and valid until its next call. */
const char* sp_last_error(const sp_ctx* ctx);

/* Declare a problem (Sec. "Domains", Sec. "Problems").  ndim = 2:
 * bases[0] Fourier (x), bases[1] Chebyshev (z, the coupled axis, last);
 * ndim = 3: bases[0] Fourier (x, real data), bases[1] Fourier (y, complex
 * axis), bases[2] Chebyshev (z).  Pencils: one per stored Fourier mode,
 * P = N_x/2 (2D) or P = N_y N_x/2 (3D, pencil p = i_y N_x/2 + i_x, i_y the
 * y slot in FFT order: mode i_y for i_y < N_y/2, i_y - N_y above, the
 * Nyquist slot N_y/2 held at zero by the transforms).
 * nvars = S = number of first-order variables = number of equations.
 * Sizes supported by the kernels: N_x, N_y even with N_gx = N_x * scale and
 * N_gy of the form 2^k or 3*2^k (16 <= N_gx <= 4096, 4 <= N_gy <= 4096),
 * N_z with N_gz likewise (8 <= N_gz <= 1536), S <= 16.  Batched stepping,
 * the adjoint entry points and sp_transform_backward_static take 2D
 * problems only (SP_ERR_ARG otherwise).  *problem_id receives the handle. */
sp_status sp_add_problem(sp_ctx* ctx, int ndim, const sp_basis* bases, int nvars,
                         int scheme, int precision, int* problem_id);

/* Pencil layout and preconditioners (Sec. "Matrix construction",
 * Sec. "Linear boundary value solver", Appendix "Dirichlet recombination
 * matrices"):
 *  col_map[v*N_z + m]  column of variable v, mode m in the pencil system;
 *  row_map[e*N_z + m]  row that receives mode m of equation e's
 *                      left-preconditioned right-hand side, or -1 for a
 *                      dropped tau row;
 *  var_recombine[v]    1: the solved coefficients are in the Dirichlet
 *                      basis D_n = T_n - T_{n-2}, so x_m = x~_m - x~_{m+2};
 *  var_phase[v]        q: true coefficient = i^q x solved coefficient;
 *  eq_differential[e]  1: equation rows are T-to-U converted,
 *                      (P^L f)_m = f_m/(2 - delta_m0) - f_{m+2}/2;
 *  eq_phase[e]         q: equation rows are multiplied by i^(-q);
 *  bc_rows[q], q < nbc rows holding boundary conditions;
 *  bc_values[(p*nbc + q)*2 + {0,1}]  complex value of boundary row q on
 *                      pencil p (already multiplied by its row phase).
 * Row and column indices are in [0, n) and must form a permutation. */
sp_status sp_set_layout(sp_ctx* ctx, int problem, const int32_t* col_map,
                        const int32_t* row_map, const int32_t* var_recombine,
                        const int32_t* var_phase, const int32_t* eq_differential,
                        const int32_t* eq_phase, int nbc, const int32_t* bc_rows,
                        const double* bc_values);

/* Preconditioned pencil matrices M~_p = P^L M_p P^R and L~_p = P^L L_p P^R
 * (Sec. "Linear boundary value solver"), real, for pencils
 * [first_pencil, first_pencil + count), on one CSR pattern shared by all
 * pencils (the union of the M and L patterns, Sec. "Matrix construction"):
 * indptr[n+1], indices[nnz] (sorted, unique per row), M_values and L_values
 * [count][nnz].  Every pencil must be set, with the same pattern, before
 * sp_factor.  The band widths kl, ku are taken from the pattern. */
sp_status sp_set_pencils(sp_ctx* ctx, int problem, int64_t first_pencil, int64_t count,
                         int n, int64_t nnz, const int32_t* indptr, const int32_t* indices,
                         const double* M_values, const double* L_values);

/* Quadratic right-hand side as a sum of terms (Sec. "Arithmetic
 * operators", products evaluated on the dealiased grid):
 *   F[eq[t]] += coef[t] * op_a[t](var_a[t]) * op_b[t](var_b[t]),
 * op in sp_op (DX = i k_x on the true coefficients). */
sp_status sp_set_bilinear_rhs(sp_ctx* ctx, int problem, int nterms, const int32_t* eq,
                              const double* coef, const int32_t* op_a, const int32_t* var_a,
                              const int32_t* op_b, const int32_t* var_b);

/* Factor every pencil for step size dt with banded LU and partial pivoting in
 * FP64 (Sec. "Matrix solvers": factorize once, reuse while dt is fixed):
 * RK schemes: M~ + dt H_ii L~ (one matrix, H_ii equal for all stages);
 * SBDF2: (M~ + dt L~) for its first step and (3/2 M~ + dt L~) afterwards;
 * SBDF1: M~ + dt L~.  A zero pivot latches SP_ERR_SINGULAR (read it with
 * sp_sync_status, which also reports the first failing pencil). */
sp_status sp_factor(sp_ctx* ctx, int problem, double dt);

/* Linear boundary value solve (Sec. "Linear boundary value solver"):
 * L~_p X~_p = P^L_p F_p with the boundary values, X_p = P^R X~_p, for every
 * pencil, into the problem's state (read it with sp_get_field).  M~ is not
 * used.  The first call (and the first after sp_factor or sp_eig_target)
 * factors L~ alone, replacing any stepping factorization (sp_step then
 * needs sp_factor again).  F: host, nslots blocks [P][N_z] complex FP64 of
 * T coefficients, block q the right-hand side of equation eqs[q] (other
 * equations' right-hand sides are zero); differential equations get the
 * T-to-U conversion and lose their tau row in the kernel, as the stepping
 * right-hand sides do.  Synchronous.  SP_ERR_ARG for bad slots or equation
 * indices, SP_ERR_SINGULAR if a pencil's L~ is singular. */
sp_status sp_solve_lbvp(sp_ctx* ctx, int problem, int nslots, const int32_t* eqs, const void* F_host);

/* Set / get one variable of the state (Sec. "Initial conditions").
 * layout 'c': P*N_z complex (re, im) doubles [p][m], true coefficients;
 * layout 'g': N_z*N_x (3D: N_z*N_y*N_x) real doubles [iz][ix] ([iz][iy][ix])
 * on the scale-1 grid
 * (forward-transformed on the device).  Setting a variable restarts
 * multistep history (the next SBDF2 step is an SBDF1 step). */
sp_status sp_set_field(sp_ctx* ctx, int problem, int var, const void* data, int on_device,
                       char layout);
sp_status sp_get_field(sp_ctx* ctx, int problem, int var, void* data, int on_device,
                       char layout);

/* dst_var := d/dz src_var in coefficient space, with the O(N) Chebyshev
 * recurrence (Appendix "Differentiation and conversion matrices"; used to
 * make first-order initial conditions consistent, Sec. "Initial
 * conditions"). */
sp_status sp_dz(sp_ctx* ctx, int problem, int src_var, int dst_var);

/* Advance nsteps steps of size dt (Sec. "Time evolution").  dt must equal
 * the dt of the last sp_factor (else SP_ERR_NOT_FACTORED).  Asynchronous. */
sp_status sp_step(sp_ctx* ctx, int problem, double dt, int nsteps);

/* Same as sp_step, but the stream work for the nsteps steps is recorded once
 * into a CUDA graph and replayed; the graph is cached per (problem, dt,
 * nsteps) and rebuilt when any of them changes. */
sp_status sp_step_graph(sp_ctx* ctx, int problem, double dt, int nsteps);

/* Advance a batch of independent problems together (uneven sizes, Rayleigh
 * numbers and step sizes; one scheme and precision for all).  Each stage
 * launches each kernel type once for the whole batch: the work of every
 * problem is listed (largest items first) in one grid, so small problems
 * fill the SMs left idle by large ones.  dts[q] must equal problem q's
 * factored dt.  Problems not yet in their steady schedule (fresh state,
 * SBDF2 first step) are first stepped one by one.  On the first call for a
 * set of ids the pencil tile of the z-transform kernels is autotuned (4, 8
 * or 16 columns per CTA, fastest kept; sp_batch_tile reports it).
 * use_graph = 1 records blocks of up to 16 batch steps in CUDA graphs and
 * replays them.  Asynchronous. */
sp_status sp_step_batched(sp_ctx* ctx, int nproblems, const int* problem_ids, const double* dts,
                          int nsteps, int use_graph);
sp_status sp_batch_tile(sp_ctx* ctx, int nproblems, const int* problem_ids, int* tile);

/* Launch shape the batch autotuner chose for these problems on their first
 * batched step: *persistent = 1 when the batched transform kernels run as
 * persistent grids (as many CTAs as the GPU holds at once) pulling (problem,
 * tile) work items from a device counter, largest items first; 0 when each
 * work item has a CTA of its own.  The batched pencil solves always take one
 * CTA per pencil.  The autotuner times one batch step of
 * each shape (with the z tile it picked) on a saved copy of every buffer a
 * step writes, then restores them.  SP_ERR_STATE before that step. */
sp_status sp_batch_persistent(sp_ctx* ctx, int nproblems, const int* problem_ids, int* persistent);
/* Fix the launch shape of these problems' batched steps (mode 1:
 * persistent grids, 0: one CTA per work item) or hand it back to the
 * autotuner (-1); takes effect at the next sp_step_batched. */
sp_status sp_set_batch_persistent(sp_ctx* ctx, int nproblems, const int* problem_ids, int mode);

/* Discrete adjoint of the step (Sec. "Runge-Kutta IMEX integrators": the
 * transpose of each stage equation), for the RK222 and RK111 schemes.  The
 * state space is that of sp_set_field/sp_get_field ('c' layout, all S
 * variables, [v][p][m] complex), with the real inner product of the
 * (re, im) components.
 * sp_adjoint_init: after sp_factor, factors the transposed pencils
 *   A~^T = M~^T + dt H_ii L~^T (banded LU with partial pivoting, FP64) and
 *   allocates the adjoint work buffers; for problems on the partitioned
 *   substitution it also computes the transposed factor's back-substitution
 *   coupling matrices (the transposed solves substitute forward whole-row,
 *   since kl' = ku is wider than the partitioned forward windows, and back
 *   in blocks) and zeroes their inflow guesses.
 * sp_step_adjoint: given the states of one forward step (states_dev,
 *   device, nstates consecutive arrays of S*P*N_z complex: X^n alone
 *   (nstates = 1; the first stage is then recomputed from X^n) or X^n
 *   followed by the stage states as sp_step_record writes them (nstates =
 *   number of stages)) and lambda = dJ/dX^{n+1} (lambda_dev, device, one
 *   state), overwrites lambda with dJ/dX^n.  It solves the transposed stage
 *   systems and applies the transposes of the dealiased transforms and
 *   products (in the problem's transform precision).  The problem's state
 *   buffers are used as scratch: set the state again before stepping
 *   forward.  dt must be the factored dt; other nstates give SP_ERR_ARG.
 * sp_step_record: nsteps forward steps exactly as sp_step, also writing,
 *   for step k, X^{n+k} and its stage states (RK222: X^{n+k} and X^1; RK111:
 *   X^{n+k}) to states_dev + k * (number of stages) * S*P*N_z complex
 *   (device, caller-owned), the input of sp_step_adjoint.  Asynchronous.
 * sp_transform_adjoint: transpose of sp_transform (direction -1: grid
 *   adjoint in, coefficient adjoint out; +1: coefficient adjoint in, grid
 *   adjoint out), FP64.
 * sp_dz_adjoint: src_bar += D^T dst_bar for the Chebyshev derivative of
 *   sp_dz (device arrays of P*N_z complex). */
sp_status sp_adjoint_init(sp_ctx* ctx, int problem);
sp_status sp_step_adjoint(sp_ctx* ctx, int problem, double dt, const void* states_dev, int nstates,
                          void* lambda_dev);
sp_status sp_step_record(sp_ctx* ctx, int problem, double dt, int nsteps, void* states_dev);
sp_status sp_transform_adjoint(sp_ctx* ctx, int problem, const void* in, void* out, int nfields,
                               int direction, int scale_num, int scale_den, int on_device);
sp_status sp_dz_adjoint(sp_ctx* ctx, int problem, const void* dst_bar_dev, void* src_bar_dev);

/* Wait for the stream and return the latched device status (SP_OK,
 * SP_ERR_SINGULAR, SP_ERR_NONFINITE or SP_ERR_TIMEOUT); the latch is
 * cleared.  *pencil (may be NULL) receives the first failing pencil or -1. */
sp_status sp_sync_status(sp_ctx* ctx, int64_t* pencil);

/* Transform nfields fields between coefficient and grid space at scale
 * scale_num/scale_den along every axis (Sec. "Scaled transforms &
 * dealiasing"): direction -1 = backward (in: 'c' layout [f][p][m] complex,
 * out: grid [f][iz][ix] (3D: [f][iz][iy][ix]) real, N_g = scale * N_c with
 * zero padding; order z, y, x),
 * direction +1 = forward (in: grid, out: 'c', truncation to N_c).
 * Arithmetic in the problem's transform precision; in/out are host
 * (on_device = 0) or device (on_device = 1) FP64 arrays. */
sp_status sp_transform(sp_ctx* ctx, int problem, const void* in, void* out, int nfields,
                       int direction, int scale_num, int scale_den, int on_device);

/* Evaluate the bilinear right-hand side of the current state and return its
 * T coefficients per equation with nonlinear terms, [e][p][m] complex, in
 * the order of first appearance in sp_set_bilinear_rhs (for testing). */
sp_status sp_eval_rhs(sp_ctx* ctx, int problem, void* out_host, int* n_eq);

/* Band widths of the pencil pattern: n, kl, ku (U holds kl + ku
 * superdiagonals after pivoting). */
sp_status sp_get_band(sp_ctx* ctx, int problem, int* n, int* kl, int* ku);

/* Eigenmode nearest a target in every pencil at once (Sec. "Eigenvalue
 * solver", sparse solver): for sigma M~ X~ + L~ X~ = 0, the shift-and-invert
 * operator A~ = (L~ + sigma_t M~)^{-1} M~ (its eigenvalue mu belongs to
 * sigma = sigma_t - 1/mu) is applied by the banded pencil solve and iterated
 * `iters` times from x0 -- a power iteration on A~, one mode per pencil
 * (the paper hands A~ to an Arnoldi method for several modes).  mu is the
 * Rayleigh quotient x^H A~ x / x^H x of the last normalized iterate.
 * sigma_t is real (the factorization is real).  The factorization of
 * L~ + sigma_t M~ replaces the step's: call sp_factor before stepping again.
 * x0: host [P][n] complex FP64 start vectors in solve-variable order (NULL:
 * all ones); sigma_re, sigma_im: host [P].  Device errors (a singular
 * shifted pencil) are latched in the status word (sp_sync_status). */
sp_status sp_eig_target(sp_ctx* ctx, int problem, double sigma_t, int iters, const void* x0_host, double* sigma_re,
                        double* sigma_im);

/* Residual of the last sp_eig_target's eigenpairs (the converged iterate x_p
 * and sigma_p of every pencil): residual[p] = ||(L~ + sigma_p M~) x_p|| /
 * (||L~ x_p|| + |sigma_p| ||M~ x_p||) (host, [P]) -- a check of every
 * pencil's pair that needs no other solver (an eigenpair gives rounding
 * level; an unconverged iterate, whose two nearest eigenvalues the
 * iteration has not separated, a larger value).  Several modes per pencil:
 * one sp_eig_target per target (the mode nearest each).  Synchronous.
 * SP_ERR_STATE before any eigensolve. */
sp_status sp_eig_residual(sp_ctx* ctx, int problem, double* residual);

/* CFL frequency of the current state (Sec. "Timestep determination"): the
 * largest over the points of the dealiased grid of
 *     sum_v |v(x)| / dx_{axes[v]}(x),   v = vars[0 .. nvel),
 * the velocity fields vars (state indices) along axes (0: x, 1: y on 3D
 * problems, 2: z), 1 <= nvel <= 3.  Grid spacings: L_x / N_gx, L_y / N_gy,
 * and on z the centred difference of the dealiased Chebyshev nodes
 * (one-sided at the two end nodes).  The velocities are transformed in the
 * problem's precision (FP32 in mixed precision), the sum taken in FP64.
 * Synchronizes the context's stream; *freq_out is host memory.  Scratch
 * for three fields is allocated on the first call and kept. */
sp_status sp_cfl_frequency(sp_ctx* ctx, int problem, int nvel, const int* vars, const int* axes, double* freq_out);

/* CFL timestep from a frequency (Sec. "Timestep determination"), plain
 * host arithmetic: dt = safety / freq (max_dt when freq = 0), bounded to
 * [min_dt, max_dt], then, when dt_prev > 0, to [min_change, max_change] x
 * dt_prev, and kept at dt_prev when |dt - dt_prev| < threshold x dt_prev.
 * A kept step reuses the stored factorization (sp_factor with a new dt is
 * the caller's choice).  SP_ERR_ARG for inconsistent bounds. */
sp_status sp_cfl_dt(double freq, double dt_prev, double safety, double min_dt, double max_dt, double min_change,
                    double max_change, double threshold, double* dt_out);

/* Work of one pencil substitution as the problem's solve kernel performs it
 * (Sec. "Matrix solvers": forward substitution with L, back substitution
 * with U), for the factor that the steady steps use (the last one of
 * sp_factor: SBDF2's, not its SBDF1 start):
 *   fma_per_row   multiply-adds per row and real right-hand side, forward
 *                 plus back.  Window kernel: kl + (kl + ku), every band
 *                 entry.  Lane kernel: kl + the mean number of listed
 *                 superdiagonal entries of U per column (the union of the
 *                 pencils' nonzero patterns); one multiply by 1/U_jj per row
 *                 comes on top in both.
 *   factor_bytes  bytes of stored factor one pencil's substitution reads
 *                 (multipliers, U entries including 1/U_jj, pivot bytes).
 * Either pointer may be NULL.  SP_ERR_NOT_FACTORED before sp_factor. */
sp_status sp_get_solve_work(sp_ctx* ctx, int problem, double* fma_per_row, double* factor_bytes);

/* Launch timing of the pencil-solve kernel (the step's dominant kernel):
 * sp_set_timing reserves CUDA-event pairs for up to max_launches solve
 * launches of sp_step (not of graph replays) and restarts the count
 * (max_launches = 0 disables it); sp_last_solve_time waits for the stream and
 * returns the mean duration in milliseconds of the recorded launches and
 * their number.  Events are recorded on the context stream around each
 * launch. */
sp_status sp_set_timing(sp_ctx* ctx, int problem, int max_launches);

/* Choice of the substitution kernel of the pencil solves (Sec. "Matrix
 * solvers"; the arithmetic is the same, the order of every FMA too, so both
 * give identical results): SP_SOLVE_AUTO picks SP_SOLVE_LANES for problems
 * with at least 4096 pencils when (kl, kl + ku) is (9, 38) or (7, 29), else
 * SP_SOLVE_WINDOW.  WINDOW: one warp per pencil and real/imaginary part,
 * the band across the lanes (latency-bound few-pencil problems).  LANES:
 * one lane per pencil and real/imaginary part (throughput-bound
 * many-pencil problems; SP_ERR_ARG for other band widths).  SPIKE: the
 * partitioned substitution below (few long pencils; SP_ERR_ARG unless
 * kl <= 7 and kl + ku <= 31).  Must precede
 * the first call that moves the problem to the device (sp_factor,
 * sp_set_field, sp_transform): SP_ERR_STATE afterwards. */
typedef enum { SP_SOLVE_AUTO = 0, SP_SOLVE_WINDOW = 1, SP_SOLVE_LANES = 2, SP_SOLVE_SPIKE = 3 } sp_solve_kernel;
sp_status sp_set_solve_kernel(sp_ctx* ctx, int problem, int kind);

/* Partitioned substitution (SP_SOLVE_SPIKE; Sec. "Matrix solvers": the
 * pencil solves are O(n) with the stored factor).  With fewer pencils than
 * the GPU has dependent-chain slots, each pencil's back substitution is cut
 * into nblk blocks of whole 32-row chunks (the forward one into blocks of
 * about 128 rows), substituted in parallel: a pass per block from guessed
 * inflows, a recurrence over blocks with coupling matrices computed at
 * sp_factor (kl x kl forward, (kl+ku) x (kl+ku) backward per block), then a
 * pass with the true inflows.  The back substitution's guesses are the true
 * inflows of the problem's previous solve (zero after sp_factor or
 * sp_set_field, and for a guess that is not finite): exact for any guess,
 * and consecutive time-step solves then correct by small differences, so no
 * rounding is amplified by cancellation.  Results equal the whole-row-order
 * substitution to rounding.  SP_SOLVE_AUTO picks it for 2D problems with
 * fewer than 608 pencils of at least 512 rows when kl <= 7 and kl + ku <= 31.
 * sp_set_spike_blocks sets nblk (0: automatic, about 1024 / P blocks);
 * SP_ERR_ARG if the padded rows do not split into nblk whole 32-row chunks,
 * SP_ERR_STATE once the problem is on the device (like sp_set_solve_kernel).
 * sp_get_spike_blocks returns the block count in use (0: not partitioned,
 * or the problem not yet on the device). */
sp_status sp_set_spike_blocks(sp_ctx* ctx, int problem, int nblk);

/* Chebyshev backward transform of the mixed form (Sec. "Chebyshev basis":
 * g_i = sum_n c_n T_n(x_i)): SP_ZT_FFT, the DCT through a shared-memory FFT
 * in FP32; SP_ZT_MMA, the dense product with the matrix T_n(x_i) on the
 * tensor cores (tcgen05.mma kind::tf32, each operand split into a TF32 head
 * and remainder, three products accumulated in FP32; operands staged by
 * TMA), for N_z a multiple of 32 and N_gz a multiple of 16 up to 256;
 * SP_ZT_AUTO: MMA on three-dimensional mixed problems where it fits, else
 * FFT.  FP64 problems always use the FFT.  SP_ERR_ARG for MMA on sizes or a
 * precision it does not take, SP_ERR_STATE once the problem is on the
 * device.  sp_get_z_transform returns the requested kind before, and the
 * kind in use after, the problem moves to the device. */
typedef enum { SP_ZT_AUTO = 0, SP_ZT_FFT = 1, SP_ZT_MMA = 2 } sp_z_transform;
sp_status sp_set_z_transform(sp_ctx* ctx, int problem, int kind);
sp_status sp_get_z_transform(sp_ctx* ctx, int problem, int* kind);
sp_status sp_get_spike_blocks(sp_ctx* ctx, int problem, int* nblk);
sp_status sp_last_solve_time(sp_ctx* ctx, int problem, double* ms_per_launch, int* launches);

/* Measured fused multiply-add throughput of a device (no paper counterpart;
 * a measurement utility for the ALU rooflines of the FP64 pencil solves and
 * the FP32 transforms).  precision 0: FP64, 1: FP32.  Runs a kernel of
 * independent FMA chains on every SM (about 10 ms, on its own stream, after
 * one warm-up launch) and writes the best of three launches to *tflops
 * (2 flops per FMA).  Synchronous; allocates a small sink buffer; changes no
 * device setting.  SP_ERR_ARG for a bad precision or null output,
 * SP_ERR_CUDA for a device error. */
sp_status sp_measure_fma_peak(int device, int precision, double* tflops);

/* Backward transform without any device allocation.  The paper has no
 * counterpart; this entry point is for callers that cannot call cudaMalloc
 * when they need a transform: code running while a stream is captured into a
 * CUDA graph (allocation is not capturable and may synchronize the device),
 * programs whose device memory all belongs to another allocator, and hosts
 * that must not block on an implicit device synchronization.  It computes
 * the same thing as sp_transform with direction -1 in FP64, with no context:
 *   coef_dev  device, nfields * (n_x/2) * n_z complex FP64 ('c' layout
 *             [f][p][m]), read only;
 *   grid_dev  device, nfields * N_gz * N_gx FP64 ([f][iz][ix]) on the grid of
 *             scale scale_num/scale_den, written;
 *   cuda_stream  stream to queue on (NULL = legacy default stream);
 *   errbuf/errlen  optional caller buffer for a message on failure.
 * Its intermediate data and twiddle tables live in fixed static device
 * arrays that every GPU loading the library keeps until exit: at most
 * nfields * N_gz * (n_x/2) <= 524288 complex values (8 MiB), N_gx <= 4096,
 * N_gz <= 1536, nfields <= 16, and jointly one grid row of every field in a
 * block's shared memory: (2 ceil(nfields/2) + 1) * N_gx * 16 + nfields * N_gx
 * * 8 <= 227 KiB (N_gx <= 3632 for 2 fields, <= 580 for 16); larger requests
 * return SP_ERR_ARG with the reason in errbuf, before anything is queued.
 * The first call on a device (with that device current) looks up the device
 * addresses of those arrays, once per device even under concurrent first
 * calls from several host threads; make it before any stream capture.  All calls share the arrays: calls that may overlap on the GPU
 * (other streams or threads without ordering) race and must be serialized.
 * Each call rewrites everything it reads, so nothing carries over between
 * calls.  Asynchronous: the result is ready when the stream reaches it. */
sp_status sp_transform_backward_static(const double* coef_dev, double* grid_dev, int nfields,
                                       int n_x, int n_z, int scale_num, int scale_den,
                                       void* cuda_stream, char* errbuf, int errlen);

#ifdef __cplusplus
}
#endif

#endif /* SPECTAU_H */
