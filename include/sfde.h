/*
 * sfde.h -- C ABI of the GB300 MGRIT solver for the 2-D Riesz space-fractional diffusion
 * equation (Yue, Shu, Xu, Bu, Pan, arXiv 1805.06688).
 *
 * Problem (Sec. 1, Eq. (1.1)):
 *   u_t = K_x d^{2beta}u/d|x|^{2beta} + K_y d^{2gamma}u/d|y|^{2gamma} + f on (a,b)x(c,d),
 *   u = 0 on the boundary, u(.,0) = psi_0, 1/2 < beta, gamma < 1, K_x, K_y > 0.
 * Discretisation (Sec. 2, Eq. (2.4)): linear elements in space (tensor-product hats; the 1-D
 * stiffness is the symmetric Toeplitz matrix obtained from the paper's element integrals) and
 * continuous-P1 / discontinuous-P0 space-time elements in time, which give the step
 *   S_n U_n = B_n U_{n-1} + F_n,  S_n = M_h + tau_n K,  B_n = M_h - tau_n K,
 *   tau_n = (t_n - t_{n-1})/2,  M_h U = M_y U M_x,  K U = K_x M_y U A_x + K_y A_y U M_x.
 * Solver (Sec. 3, Algorithm 1): MGRIT V-cycle on the block bidiagonal system of Eq. (3.1).
 *
 * Data layout shared by every call.  A spatial field is an N_y x N_x row-major array of
 * doubles, U[j*N_x + i] = u(x_i, y_j), x_i = a + i*h_x (i = 1..N_x), h_x = (b-a)/(N_x+1);
 * a space-time field is N_t+1 such slices, time slowest.  Pointers may be host or device
 * memory: the library asks the CUDA runtime which (cudaPointerGetAttributes) and copies
 * as needed.  All device work runs on the stream given at setup; every call below returns
 * only after that work is finished (synchronous).
 *
 * Errors: every call returns an sfde_status; nothing throws across the ABI (a host
 * allocation or thread start that fails inside a call returns SFDE_ENOMEM).  After
 * SFDE_ECUDA the context must be destroyed.  A context is not thread-safe; distinct
 * contexts are independent.  Ownership: inputs are copied during the call; outputs are
 * caller-allocated; the context owns all internal device memory and frees it in
 * sfde_destroy.
 */
#ifndef SFDE_H
#define SFDE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SFDE_OK = 0,
    SFDE_EINVAL = 1,        /* invalid argument (range, size, NULL, ordering)            */
    SFDE_ENOMEM = 2,        /* a device or host allocation failed                        */
    SFDE_ECUDA = 3,         /* a CUDA runtime call or kernel failed; context unusable    */
    SFDE_ENOCONV = 4,       /* no convergence within max_iter, or a non-finite residual  */
    SFDE_ETIMEOUT = 5,      /* a bounded device wait ran out                             */
    SFDE_EUNSUPPORTED = 6,  /* option or size the library does not provide               */
    SFDE_ESCRATCH = 7       /* request larger than the fixed scratch of sfde_step_batch_noalloc */
} sfde_status;

typedef struct sfde_ctx sfde_ctx;

/* Arithmetic of the fine steps (the MGRIT iterate, residual and norm are FP64 in all forms). */
typedef enum {
    SFDE_PREC_FP64 = 0,        /* every step in FP64                                              */
    SFDE_PREC_MIXED_BF16 = 1,  /* inner V-cycles on BF16 tensor cores (FP32 accumulate), FP64
                                  space-time residual and iterative refinement                    */
    SFDE_PREC_MIXED_TF32 = 2,  /* as above with TF32 operands                                     */
    SFDE_PREC_MIXED_FP32 = 3,  /* as above with FP32 operands and levels: every product formed from
                                  three TF32 tensor-core products (high and low parts of both
                                  operands, about 2^-20 relative), three times the tensor work of
                                  TF32 for corrections about 2^10 times more accurate, so fewer
                                  refinement steps (no counterpart in the paper)                 */
    SFDE_PREC_MIXED_AUTO = 4   /* FP32: with the inner solve held in the step's eigenbasis (the
                                  default for FP32 storage, see sfde_tuning.modal_chains) a
                                  refinement step costs about one FP64 residual, and FP32 corrections
                                  need the fewest of them -- measured faster than the fused BF16
                                  steps too (N = 255, N_t = 1024: 24.8 against 49.1 ms per solve)
                                  (no counterpart in the paper)                                 */
} sfde_precision;

/* Spatial matrices of the fully discrete scheme (2.4). */
typedef enum {
    SFDE_OP_TENSOR = 0,   /* tensor-product (Kronecker) form with the 1-D linear-element matrices:
                             S_n U = M_y U M_x + tau_n (K_x M_y U A_x + K_y A_y U M_x); steps by fast
                             diagonalisation (every precision)                                    */
    SFDE_OP_P1 = 1        /* the P1-triangle matrices printed in Sec. 2: the block-tridiagonal mass
                             M_h (7-point stencil) and the block-Toeplitz A_x^beta, A_y^gamma (the
                             latter through the permutation P_pi); steps by conjugate gradients
                             preconditioned with the tensor-product solve, to 1e-13 relative residual
                             per slice; FP64 precision only                                       */
} sfde_operator;

typedef struct {
    int precision;     /* sfde_precision                                                   */
    void* stream;      /* cudaStream_t for all device work; NULL = the legacy default stream */
    int operator_kind; /* sfde_operator (SFDE_OP_P1 requires SFDE_PREC_FP64, else SFDE_EUNSUPPORTED) */
} sfde_opts;

/*
 * sfde_setup -- build one problem instance (Sec. 2).
 *   beta, gamma : fractional orders, 1/2 < beta, gamma <= 1 (1 gives the classical Laplacian).
 *   kx, ky      : diffusivities K_x, K_y > 0.
 *   omega       : host array {a, b, c, d}, a < b, c < d.
 *   nx, ny      : interior nodes per direction, 1 <= nx, ny <= 4096.
 *   t           : host array t[0..nt], t[0] = 0, strictly increasing (any grid; the fine
 *                 propagator depends on n through t_n - t_{n-1}).
 *   nt          : number of time steps, nt >= 1.
 *   opts        : may be NULL (FP64, default stream).
 *   out         : receives the new context.
 * On the device this computes, in FP64, the Toeplitz coefficients of A_x, A_y from the element
 * integrals (Sec. 2), the dense matrices, the generalised eigenpairs A V = M V diag(lambda)
 * with V^T M V = I (Jacobi rotations on L^{-1} A L^{-T}, M = L L^T), and W = M V.
 * psi_0 defaults to 0 and f to 0.
 */
sfde_status sfde_setup(double beta, double gamma, double kx, double ky, const double omega[4],
                       int nx, int ny, const double* t, int nt, const sfde_opts* opts,
                       sfde_ctx** out);

/* Nodal initial values psi_0^I (Sec. 2, below Eq. (2.4)): N_y x N_x doubles, host or device. */
sfde_status sfde_set_initial(sfde_ctx* ctx, const double* psi0);

/*
 * Separable load vectors (Sec. 2, below Eq. (2.4)):
 *   F_n[j][i] = sum_{r<rank} time_w[(n-1)*rank + r] * by[r*N_y + j] * bx[r*N_x + i], n = 1..N_t,
 * i.e. f = sum_r c_r(t) f_x^r(x) f_y^r(y) with time_w = int_{I_n} c_r dt, bx = (f_x^r, phi_i),
 * by = (f_y^r, phi_j).  0 <= rank <= 4 (rank 0 clears the load).  Host or device arrays.
 */
sfde_status sfde_set_forcing(sfde_ctx* ctx, int rank, const double* time_w, const double* bx,
                             const double* by);

/*
 * Dense (non-separable) load vectors (Sec. 2, below Eq. (2.4)): F holds N_t x N_y x N_x doubles,
 * F[((n-1)*N_y + j)*N_x + i] = (f, phi_i phi_j) integrated over I_n, n = 1..N_t; host or device,
 * copied during the call.  NULL clears the load.  Replaces any load set before (separable or
 * dense), as sfde_set_forcing replaces a dense one.  The library keeps F and its eigenbasis
 * transform V_y^T F_n V_x on the device (2 N_t P_x P_y doubles).  SFDE_ENOMEM if they do not fit.
 */
sfde_status sfde_set_forcing_dense(sfde_ctx* ctx, const double* F);

typedef enum { SFDE_RELAX_FCF = 0, SFDE_RELAX_F = 1 } sfde_relax;
typedef enum {
    SFDE_COARSE_CN = 0,    /* rediscretisation with the same Crank-Nicolson-type step, Eq. (3.4) */
    SFDE_COARSE_BE = 1,    /* L-stable backward-Euler rediscretisation (M_h + dt K)^{-1} M_h      */
    SFDE_COARSE_AUTO = 2   /* CN when Theorem 3.1's two-level bound (Eq. (3.11)) is below 1,
                              otherwise BE; decided at solve time from the eigenvalues            */
} sfde_coarse;

typedef struct {
    int m;               /* coarsening factor, >= 2; 0: chosen per problem by the two-level analysis
                            of Sec. 3.3 (see sfde_choose_coarsening)                          */
    int max_levels;      /* >= 1; levels are added while N_l % m == 0 and N_l/m >= min_coarse   */
    int min_coarse;      /* >= 1                                                              */
    int relax;           /* sfde_relax (Step 1 of Algorithm 1)                                */
    int coarse;          /* sfde_coarse                                                       */
    int max_iter;        /* >= 1                                                              */
    double rel_tol;      /* stop when ||r||_2 <= max(rel_tol*||r_first||_2, abs_tol); r is the  */
    double abs_tol;      /* C-point residual Phi_{km}(u_{km-1}) - u_{km} over all level-0 C-points
                            (or, see stop_kind, the space-time residual)                       */
    uint64_t init_seed;  /* 0: zero initial guess; else SplitMix64 uniform[-1,1) values at
                            t_1..t_N, value index (n*N_y + j)*N_x + i (Sec. 3.2)              */
    int inner_cycles;    /* mixed precision only: low-precision V-cycles per FP64 refinement step
                            (0 = default: 4 for BF16, 5 for TF32, 3 for FP32)                 */
    int skip_first_down; /* 1: the option "skip work on the first down cycle" (Sec. 3.2): the first
                            V-cycle relaxes on no level on its way down -- the coarse right-hand
                            side is the injected C-point residual of the initial guess -- and runs
                            the coarsest solve and the up-cycle as usual.  That iteration applies no
                            stopping test; the C-point reference norm is then the second
                            iteration's.  In the mixed forms it applies to the first V-cycle of every
                            inner solve (each starts from a zero correction).  0: off.          */
    int stop_kind;       /* residual of the stopping test: 0 the form's own (FP64: the C-point
                            residual above; mixed: the space-time residual below); 1 the space-time
                            residual of Eq. (2.4), rho_n = F_n + B_n u_{n-1} - S_n u_n over
                            n = 1..N_t, in FP64, relative to rho of the initial guess -- the same
                            test in every form.  The FP64 form evaluates it after the relaxation,
                            where every F-point's row of Eq. (3.1) holds and rho_{km} = S_{km} r_k. */
} mgrit_opts;

#define SFDE_HISTORY_MAX 512

typedef struct {
    int iters;            /* V-cycles done (outer refinement iterations for mixed precision)    */
    int levels;
    int converged;
    int coarse_used;      /* sfde_coarse actually used (CN or BE)                               */
    double res0, res_final;
    double conv_factor_last5;   /* mean ratio of successive residuals over the last five      */
    double seconds;       /* wall time of the solve on the device (CUDA events), no setup       */
    double tub;           /* Theorem 3.1 bound for the CN coarse propagator (computed for AUTO) */
    long long step_solves;      /* fine/coarse step applications executed, all levels       */
    long long inner_vcycles;    /* low-precision V-cycles (mixed precision only)             */
    double history[SFDE_HISTORY_MAX];  /* residual norm per iteration                         */
    int lp_kind;          /* operand type of the low-precision steps: 0 BF16, 1 TF32, 2 FP32 (three
                             TF32 products); -1 FP64 form                                     */
    int m_used;           /* coarsening factor of the solve (the chosen one when opts.m was 0)   */
} mgrit_stats;

/*
 * Two-level convergence analysis (Sec. 3.3), evaluated on the device over every mode of the
 * problem.
 *
 * sfde_two_level_bound -- Theorem 3.1's bound, Eq. (3.11), for coarsening factor m and the coarse
 * propagator `coarse` (SFDE_COARSE_CN: the paper's rediscretisation, Eq. (3.4); SFDE_COARSE_BE):
 *   max over modes w of (lam+)^m |(lam+)^m - mu++| (1 - (mu*)^{N_c - 1}) / (1 - mu*),
 * with the fine-step eigenvalues of Eq. (3.7) (lam+: their largest magnitude over the fine steps),
 * the coarse propagator's (mu++: smallest, mu*: largest magnitude over the coarse steps),
 * sigma_w = K_x lambda_x + K_y lambda_y from the setup's eigenvalues, N_c = N_t / m.
 * SFDE_EINVAL unless m >= 2 divides N_t with N_t / m >= 2.  *bound is host memory.  For an
 * SFDE_OP_P1 context the modes are those of the tensor-product operator (its preconditioner,
 * spectrally equivalent within a factor of about 4): an estimate, not the P1 spectrum.
 *
 * sfde_choose_coarsening -- the m that mgrit_solve uses when mgrit_opts.m is 0: among
 * m in {2, 4, 8, 16, 32} dividing N_t with at least two coarse intervals, the least estimated work to
 * rel_tol, taking the bound b(m) of the coarse propagator in use (`coarse` as in mgrit_opts; AUTO
 * resolved per m) as the contraction per iteration: ceil(log rel_tol / log b(m)) iterations of about
 * 2 m / (m - 1) step solves per time point.  Candidates with b(m) >= 1 are left out (all of them: the
 * largest valid m); ties go to the larger m.
 */
sfde_status sfde_two_level_bound(sfde_ctx* ctx, int m, int coarse, double* bound);
sfde_status sfde_choose_coarsening(sfde_ctx* ctx, int coarse, double rel_tol, int* m);

/*
 * mgrit_solve -- Algorithm 1: V-cycles of FCF (or F) relaxation, injection of the C-point
 * residual, recursion with zero initial guess, sequential solve on the coarsest level,
 * C-point correction (F-relaxation after the correction on levels >= 1).
 *   opts  : NULL gives m = 2, all levels, FCF, AUTO, max_iter 100, rel_tol 1e-10.
 *   U     : (N_t+1) x N_y x N_x doubles receiving all time points, or NULL.
 *   U_T   : N_y x N_x doubles receiving u at t_N, or NULL.
 *   stats : may be NULL.
 * Returns SFDE_ENOCONV (with U, U_T and stats filled) when max_iter is reached or the
 * residual is not finite.
 */
sfde_status mgrit_solve(sfde_ctx* ctx, const mgrit_opts* opts, double* U, double* U_T,
                        mgrit_stats* stats);

/*
 * sfde_batch_solve -- the batched form: n independent instances (distinct contexts from
 * sfde_setup, any sizes and precisions) solved by Algorithm 1 concurrently on the current GPU.
 * Each instance runs exactly the arithmetic of mgrit_solve on its own stream (a context created
 * with the legacy default stream gets a private non-blocking stream for the call, the quarter with
 * the most work at the highest stream priority), driven by up to 16 host threads that start the
 * instances in order of decreasing work, so results equal those of separate mgrit_solve calls.  No counterpart in the
 * paper (its parallelism is across time on a CPU cluster); it fills the GPU where one instance's
 * coarse levels cannot.
 *   opts   : shared by all instances (NULL: the mgrit_solve defaults).
 *   U_T    : NULL, or n pointers (entries may be NULL) to N_y x N_x doubles receiving u(t_N),
 *            host or device.
 *   stats  : NULL or n entries;  status : NULL or n entries receiving each instance's status.
 * Returns SFDE_EINVAL for n < 1 or NULL / repeated contexts (nothing runs), else the first
 * non-OK instance status (SFDE_OK if all converged).  Synchronous: all instances have finished,
 * outputs written, on return.  Contexts must not be used by other threads during the call.
 */
sfde_status sfde_batch_solve(int n, sfde_ctx* const* ctxs, const mgrit_opts* opts, double* const* U_T,
                             mgrit_stats* stats, sfde_status* status);

/* Sequential time stepping U_n = S_n^{-1}(B_n U_{n-1} + F_n), n = 1..N_t (Eq. (2.4)), one step
 * after another.  U and U_T as in mgrit_solve; seconds (may be NULL) = device time. */
sfde_status seq_timestep(sfde_ctx* ctx, double* U, double* U_T, double* seconds);

/*
 * sfde_step_batch -- apply the fine step Phi_n (Eq. (2.4)) to `batch` fields at once:
 *   out[b] = S_{n_b}^{-1}(B_{n_b} in[b] + F_{n_b}),  n_b = n0 + b*dn,  1 <= n_b <= N_t.
 * in, out: batch x N_y x N_x doubles (host or device, may not overlap).  This is the unit of
 * work every relaxation sweep runs; exposed for testing and benchmarking.
 */
sfde_status sfde_step_batch(sfde_ctx* ctx, int n0, int dn, int batch, const double* in,
                            double* out);

/*
 * sfde_propagate_batch -- the coarse propagators of Algorithm 1 (Sec. 3.1) with a right-hand side,
 * for `batch` fields with their own step sizes (coarse levels of a time-sharded V-cycle):
 *   out[b] = Psi(dts[b]) in[b] + g[b],  Psi(dt) = (M_h + dt/2 K)^{-1} (M_h - dt/2 K)  (scheme
 *   SFDE_COARSE_CN, Eq. (3.4)) or (M_h + dt K)^{-1} M_h  (SFDE_COARSE_BE); no load term.
 * dts: host, batch step sizes > 0; in, g (may be NULL: zero), out: batch x N_y x N_x doubles, host or
 * device, out not overlapping in or g.  Synchronous.  SFDE_EINVAL for another scheme or a step <= 0.
 */
sfde_status sfde_propagate_batch(sfde_ctx* ctx, int scheme, const double* dts, int batch, const double* in,
                                 const double* g, double* out);

/*
 * sfde_step_batch_noalloc -- the same computation as sfde_step_batch, without allocating any device
 * memory (no counterpart in the paper: this exists for callers of the library).
 *
 * Some callers cannot let a library call cudaMalloc or cudaFree: an application whose device memory
 * is held by another allocator (a framework's caching allocator owns the pool, so a new cudaMalloc
 * may fail or force that allocator to give memory back), or a latency-critical loop in which
 * cudaFree would synchronise the whole device.  This entry point keeps its padded staging buffers
 * and step intermediates in one fixed device array of SFDE_NOALLOC_SCRATCH_DOUBLES doubles (10 MiB)
 * that is part of the library image: every GPU that loads the library holds it until exit.
 *
 *   in, out : DEVICE pointers, batch x N_y x N_x doubles each (host pointers -> SFDE_EINVAL).
 *   limit   : 5 * batch * P_x * P_y <= SFDE_NOALLOC_SCRATCH_DOUBLES, where P is the padded extent
 *             of a direction (32 for N <= 32, 64 for N <= 64, else N rounded up to a multiple of 128);
 *             larger requests return SFDE_ESCRATCH before any work is queued.
 * The work is queued on the context's stream and the call returns without waiting: synchronise that
 * stream before reading `out`.  All calls, from every context on a device, share the one array:
 * calls whose work overlaps on the GPU (different streams, or different host threads) race and must
 * be serialised by the caller.  Each call writes every scratch element it reads, so no clearing is
 * needed between calls.  The device that was current when the context was set up must be current
 * for the call (SFDE_EINVAL otherwise): the array's address differs per device.  On the first call
 * for a device the library looks up the array's device address once and caches it; make that first
 * call before any stream capture.  The cached address assumes the device is not reset
 * (cudaDeviceReset) while the library is loaded; a call that fails with SFDE_ECUDA drops the cached
 * address so that the next call looks it up again.  SFDE_OP_P1 contexts: SFDE_EUNSUPPORTED (their
 * conjugate-gradient step needs a workspace).
 */
#define SFDE_NOALLOC_SCRATCH_DOUBLES (5u * 262144u)
sfde_status sfde_step_batch_noalloc(sfde_ctx* ctx, int n0, int dn, int batch, const double* in,
                                    double* out);

/* Read back setup data (for verification).  dir = 0 for x, 1 for y.
 *   coeffs : N doubles a_0..a_{N-1} of the Toeplitz stiffness (may be NULL)
 *   lambda : N generalised eigenvalues (may be NULL)
 *   V      : N x N doubles, V[i*N + k] = component i of eigenvector k (may be NULL)
 * Host pointers.  These are the tensor-product operator's data (for an SFDE_OP_P1 context: those of
 * its preconditioner). */
sfde_status sfde_get_operator(sfde_ctx* ctx, int dir, double* coeffs, double* lambda, double* V);

/*
 * Kernel accounting for roofline reports (no counterpart in the paper).
 * sfde_profile_enable resets the counters; with enable != 0 every launch of the accounted kernels
 * is additionally bracketed by CUDA events on the context's stream, and its device time and
 * algorithmic work (flops of the products with unpadded sizes; bytes each launch must move at
 * least once) are accumulated per kernel class:
 *   0 = FP64 slice GEMM of a step (2 n_R n_C n_out flops per product),
 *   1 = FP64 slice GEMM of the space-time residual (P > 256),
 *   2 = tensor-core slice GEMM of a low-precision step (BF16/TF32; four per step),
 *   3 = fused low-precision step (BF16; 4 n_x n_y (n_x + n_y) flops per slice),
 *   4 = digit-split tensor-core product of the residual (BF16 digit products actually computed:
 *       28 (integer output) or 21 (FP64 output) times 2 n_R n_C n_out),
 *   5 = integer residual assembly (exponents, digit splitting, combination; bytes only),
 *   6 = P1-triangle operator products (FP64; 2 n_y n_x (3 n) flops per direction and slice, n = n_x
 *       or n_y: the block-Toeplitz contraction over three shifted copies of the slice).
 * kernel_launches counts every kernel this library launched on the context.
 */
#define SFDE_PROF_CLASSES 7
typedef struct {
    long long kernel_launches;
    long long launches[SFDE_PROF_CLASSES];
    double ms[SFDE_PROF_CLASSES];
    double flops[SFDE_PROF_CLASSES];
    double bytes[SFDE_PROF_CLASSES];
} sfde_profile;

sfde_status sfde_profile_enable(sfde_ctx* ctx, int enable);
sfde_status sfde_profile_read(sfde_ctx* ctx, sfde_profile* out);

/*
 * Execution choices of the mixed-precision solver.  They change its speed, not its fixed point:
 * every choice solves the same system to the same tolerance (results agree to rounding).
 */
typedef struct {
    int fused_pair;      /* fused BF16 step at P = 256: 1 a CTA pair per slice where 2 x batch <= SMs,
                            else per two slices (default); 2 always per slice; 3 always per two
                            slices; 0 one CTA per slice                                        */
    int modal_chains;    /* F-relaxations in the step's eigenbasis: 1 coarse levels (the
                            default with BF16), 2 every level, 3 every level with BF16 operands,
                            0 none; 4 the whole inner solve in the eigenbasis (the default with
                            TF32/FP32 working precision; as 1 with BF16)                      */
    int inner_cycles;    /* V-cycles per refinement step when mgrit_opts.inner_cycles is 0;
                            0 = 4 (BF16) / 5 (TF32)                                           */
    double ms;           /* measured solve time of this choice (milliseconds; 0 = unmeasured)  */
} sfde_tuning;

/*
 * sfde_set_tuning -- applies t to ctx for the following solves.  SFDE_EINVAL for a NULL argument
 * or a field out of the ranges above (inner_cycles 0..64).
 *
 * sfde_autotune -- picks the fastest of a small fixed set of choices for this context's problem
 * (cache key: padded sizes, fractional orders, K_x, K_y, N_t, T, step spread and a hash of the time
 * points, precision) and the given options: each candidate is applied and
 * timed over one untimed and two timed full solves (device time, the smaller counted); only
 * candidates whose solves converge count.  The winner is applied to ctx and returned in *out (may
 * be NULL).  With cache_path (may be NULL) the choice is first looked up in that text file (lines
 * "<key> <fused_pair> <modal_chains> <inner_cycles> <ms>", the last line for the key counts) and,
 * when measured, appended to it.  The context's iterate is overwritten by the trial solves.  FP64
 * contexts have nothing to tune: *out receives the current settings and SFDE_OK is returned.
 * Returns the status of the last trial when no candidate converged (settings left unchanged).
 *
 * sfde_get_tuning -- writes the choices ctx currently applies to *out (ms = 0).  SFDE_EINVAL for a
 * NULL argument.
 */
sfde_status sfde_set_tuning(sfde_ctx* ctx, const sfde_tuning* t);
sfde_status sfde_get_tuning(const sfde_ctx* ctx, sfde_tuning* out);
sfde_status sfde_autotune(sfde_ctx* ctx, const mgrit_opts* opts, const char* cache_path, sfde_tuning* out);

void sfde_destroy(sfde_ctx* ctx);
const char* sfde_strerror(sfde_status status);

#ifdef __cplusplus
}
#endif
#endif /* SFDE_H */
