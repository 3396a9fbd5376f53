/*
 * sfde_debug.h -- verification hooks of the GB300 SFDE library (not needed to solve problems).
 * No counterpart in the paper.
 */
#ifndef SFDE_DEBUG_H
#define SFDE_DEBUG_H
#include "sfde.h"
#ifdef __cplusplus
extern "C" {
#endif

/*
 * One tensor-core slice GEMM on device buffers, the unit every mixed-precision step is built from:
 *   Out[b] = (X[s0 + b*ds] * Mat)^T,  b = 0..batch-1,
 * X: nslices slices of R x C row-major (R = 32, 64 or a multiple of 128); MatT: Cout x C row-major
 * (Mat transposed, Cout a multiple of 32); Out: batch slices of Cout x R.  kind 0: BF16 operands and
 * output (tcgen05 kind::f16), kind 1: FP32 storage with TF32 products (kind::tf32); FP32
 * accumulation.  All pointers are device pointers, 16-byte aligned.  Synchronous.  *err_out (may be
 * NULL) receives the kernel's error word (non-zero if a bounded wait ran out -> SFDE_ETIMEOUT).
 * If reps > 0 and ms_out != NULL, the product is then repeated `reps` times back to back on the
 * legacy default stream and the average device time per launch (CUDA events) is stored in *ms_out.
 */
sfde_status sfde_debug_tc_gemm(int kind, const void* X, long long nslices, int s0, int ds, int batch,
                               int R, int C, const void* MatT, int Cout, void* Out, int* err_out,
                               int reps, float* ms_out);

/*
 * Failure detection without a fault: one CTA runs the bounded mbarrier wait of the tensor-core
 * kernels (the same primitive, with limit_ns instead of their 2 s) on a barrier that nothing arrives
 * at -- no copy or product is issued -- so the wait runs out, records its error code in a device word
 * and the kernel returns.  1000 <= limit_ns <= 2e9 (SFDE_EINVAL otherwise).  Returns SFDE_ETIMEOUT
 * with *err_out (may be NULL) = the error word and *waited_s (may be NULL) = the device time the wait
 * took; the CUDA context stays usable.  Synchronous (device-wide).
 */
sfde_status sfde_debug_wait_timeout(unsigned long long limit_ns, int* err_out, double* waited_s);

/*
 * One FP64-accurate slice GEMM on the BF16 tensor cores (error-free digit splitting):
 *   Out[b] = (X[b] * Mat)^T,  b = 0..batch-1,  X: batch x R x K doubles, Mat: K x N doubles (row-major),
 *   Out: batch x N x R doubles; R = 32, 64 or a multiple of 128; K, N multiples of 32, K <= 256.
 * Device pointers; synchronous; allocates its own scratch.  Error about 2^-47 of
 * max|X row| * max|Mat column| * K per element, the accuracy of an FP64 GEMM.
 */
sfde_status sfde_debug_oz_gemm(const double* X, int batch, int R, int K, const double* Mat, int N,
                               double* Out, int* err_out);

/*
 * The FP64 space-time residual of the mixed-precision solver for a given iterate (Eq. (2.4)):
 *   rho_n = F_n + B_n U_{n-1} - S_n U_n,  n = 1..N_t,
 * U: (N_t+1) x N_y x N_x doubles (host or device); rho: N_t x N_y x N_x floats (host or device),
 * rounded to TF32 as the solver stores it (plain FP32 for an SFDE_PREC_MIXED_FP32 context);
 * *norm2 = sum of rho_n^2.  use_tensor_cores = 1 (or 7)
 * assembles rho in integer arithmetic around digit-split BF16 tensor-core products with seven
 * digits per operand, 4..6 with that many (operands truncated at about 2^{9-8 nd} of their scales);
 * padded 64 <= P_x, P_y <= 256 or multiples of 256 up to 1024; *norm2 from the stored FP32 values,
 * relative accuracy about 2^-22.  0 uses FP64 arithmetic (*norm2 of the FP64 values).
 * Synchronous; allocates scratch.
 */
sfde_status sfde_debug_residual(sfde_ctx* ctx, const double* U, int use_tensor_cores, float* rho,
                                double* norm2);

/*
 * Digits per operand of the mixed-precision solver's tensor-core residual (Eq. (2.4)): 0 (default)
 * chooses 4 to 7 per outer iteration from the residual's size relative to the first one, always
 * confirming convergence with 7 (exact operands); 4..7 fixes the count.  Takes effect at the next
 * mgrit_solve.
 */
sfde_status sfde_debug_set_residual_digits(sfde_ctx* ctx, int nd);

/*
 * Time points per pass of the tensor-core residual (Eq. (2.4)): 0 (default) the scratch size, else
 * at most that.  Smaller passes keep the digit planes and products of a pass in L2.  Takes effect at
 * the next residual.
 */
sfde_status sfde_debug_set_resid_chunk(sfde_ctx* ctx, int n);

/*
 * Whether the BF16 mixed-precision solver runs each spectral step as one fused kernel (the four
 * products of Sec. 2's fast diagonalisation chained on chip; P_x = P_y in {128, 256}) or as four
 * tensor-core slice GEMMs.  Default 1; the two give the same arithmetic up to the order of FP32
 * accumulation.  Takes effect at the next mgrit_solve.
 */
sfde_status sfde_debug_set_fused_step(sfde_ctx* ctx, int enable);

/*
 * How the fused kernel spreads slices over the GPU (P_x = P_y = 256): 0 one CTA per slice; 1
 * (default) a CTA pair per slice (each CTA holding half the rows of every operand, the products
 * issued over the pair) when twice the number of slices of a launch fits on the SMs, else a CTA
 * pair per two slices (one slice's products run while the other's accumulator is drained); 2 always
 * a pair per slice; 3 always a pair per two slices.  All forms give identical results.  Takes effect
 * at the next mgrit_solve or debug step.
 */
sfde_status sfde_debug_set_fused_pair(sfde_ctx* ctx, int mode);

/*
 * Where the mixed-precision solver's inner V-cycles run F-relaxations and the coarsest level's
 * sequential sweep in the eigenbasis of the step (as mode 3 of sfde_debug_lp_chain: the right-hand
 * sides transformed once per level visit, each sweep one transform of the C-point values, an
 * elementwise FP32 recurrence over the interval and one inverse transform of all F-points) instead
 * of as chained fused steps.  enable 1 (default): the coarse levels l >= 1; 2: every level, the fine
 * one too (its buffers, two more copies of the fine level's low-precision vector, are allocated at
 * the next solve); 3: 2 with BF16 operands (whose chained steps round most), 1 with TF32; 0: none;
 * 4: with FP32 storage (TF32 and FP32 working precisions) the whole inner solve in the eigenbasis:
 * the correction right-hand sides transformed once per refinement step (V_y^T rho_n V_x scaled by
 * 1/(1 + tau_n sigma)), every level's iterate and right-hand side kept as FP32 modal values, every
 * relaxation, residual, correction and coarsest sweep an elementwise recurrence, and the correction
 * transformed back once (with BF16 storage 4 acts as 1).  All forms compute u_{im+j} =
 * Phi(u_{im+j-1}) + g_{im+j} (Algorithm 1's F-relaxation), rounded differently.  Takes effect at the
 * next mgrit_solve; other values give SFDE_EINVAL.
 */
sfde_status sfde_debug_set_modal_chains(sfde_ctx* ctx, int enable);

/*
 * One batched low-precision step of the mixed-precision solver (ctx precision must be MIXED_BF16
 * or MIXED_TF32):  out[b] = Phi(U[b]) + g[b] - ut[b],  b = 0..batch-1, slice b stepped from
 * t_{n0+b-1} to t_{n0+b} (1 <= n0, n0 + batch - 1 <= N_t).
 *   scheme 0: Crank-Nicolson step (Eq. (2.4) with F = 0), 1: backward Euler step (coarse
 *   propagator of Sec. 3), 2: the solve S_{n}^{-1} U alone.
 *   fused  1: the fused kernel (BF16, P_x = P_y in {128, 256}; SFDE_EUNSUPPORTED otherwise),
 *          0: four tensor-core slice GEMMs.
 * U, g, ut, out: batch x N_y x N_x doubles (host or device; g, ut may be NULL), rounded to the
 * operand type on input; *norm2 (may be NULL; used only with ut) = sum over the batch of the squared
 * outputs, formed from the FP32 values before they are rounded (FP32 partial sums of at most 256
 * squares, added in FP64).  Synchronous; allocates scratch.
 */
sfde_status sfde_debug_lp_step(sfde_ctx* ctx, int fused, int scheme, const double* U, int batch, int n0,
                               const double* g, const double* ut, double* out, double* norm2);

/*
 * Host rules of the mixed-precision solver, callable without a GPU.
 *
 * sfde_debug_inner_levels: the time points per level of the inner V-cycles' hierarchy for N_t =
 * nt (Algorithm 1's coarsening by m, levels kept while m divides the level and the coarse level has
 * at least min_coarse points, at most max_levels; a coarse level whose direct sweep of N steps is
 * no longer than relaxing it, 3m - 1 steps, plus the sweep below is the coarsest).  Writes the
 * first min(cap, levels) sizes to `sizes` (host) and the number of levels to *count.
 * SFDE_EINVAL for nt < 1, m < 2, max_levels < 1, min_coarse < 1, cap < 0, count NULL, or sizes NULL
 * with cap > 0.
 *
 * sfde_debug_residual_digits: digits per operand (4..7) of the tensor-core residual of a
 * refinement step whose previous residual norm is prev, the first being res0: the fewest with
 * 2^{9-8 nd} <= 1e-5 prev / res0 (4 when prev or res0 is not positive).  SFDE_EINVAL if nd is NULL.
 */
sfde_status sfde_debug_inner_levels(int nt, int m, int max_levels, int min_coarse, int* sizes, int cap, int* count);

/*
 * Theorem 3.1's two-level bound (Eq. (3.11)) as the solver evaluates it to choose the coarse
 * propagator under SFDE_COARSE_AUTO, without a GPU: the maximum over the modes sigma = K_x lx[i] +
 * K_y ly[j] of (lam+)^m |(lam+)^m - mu++| (1 - (mu*)^{N_c - 1}) / (1 - mu*), with lam+ the largest
 * |fine CN factor| over the steps of t, mu++ the smallest and mu* the largest |coarse factor| over
 * the m-coarsened steps (coarse SFDE_COARSE_CN or SFDE_COARSE_BE), eigenvalues of Eq. (3.7).
 * lx: nx, ly: ny generalised eigenvalues (host); t: nt + 1 increasing time points (host).  *out is
 * +infinity when m does not divide nt or the coarse grid has fewer than two intervals.
 */
sfde_status sfde_debug_tub_bound(const double* lx, int nx, const double* ly, int ny, double kx, double ky,
                                 const double* t, int nt, int m, int coarse, double* out);
sfde_status sfde_debug_residual_digits(double prev, double res0, int* nd);

/*
 * Host parts of sfde_autotune, callable without a GPU.
 * sfde_debug_tune_pick: *best = the index of the candidate with the smallest positive finite ms
 *   (the first on ties), -1 when none has one.  SFDE_EINVAL for n < 0 or NULL pointers (c may be
 *   NULL when n = 0).
 * sfde_debug_tune_cache: store != 0 appends the line for (key, *t) to the text file at path;
 *   store == 0 reads the last valid line for key into *t and sets *found (0 when the file or the
 *   key is missing; malformed lines and out-of-range fields are skipped).  key: 1..255 characters
 *   without white space, else SFDE_EINVAL; SFDE_EINVAL too when the file cannot be written.
 */
sfde_status sfde_debug_tune_pick(const sfde_tuning* c, int n, int* best);
sfde_status sfde_debug_tune_cache(const char* path, const char* key, int store, sfde_tuning* t, int* found);

/*
 * nchain consecutive low-precision steps from each of `batch` slices (ctx precision MIXED_BF16 or
 * MIXED_TF32), as in the F-relaxation of Algorithm 1:
 *   x_0 = U[b],  x_{k+1} = Phi(x_k) + g[b][k],  out[b][k] = x_{k+1},  k = 0..nchain-1,
 * step k of slice b going from t_{n0 + b*nchain + k - 1} to t_{n0 + b*nchain + k}
 * (n0 >= 1, n0 + batch*nchain - 1 <= N_t); scheme 0 Crank-Nicolson, 1 backward Euler.
 *   mode 1: one launch of the fused kernel, each CTA chaining the steps of its slice on chip;
 *   mode 2: nchain launches of the fused kernel (single steps);  mode 0: four slice GEMMs per step;
 *   mode 3: in the eigenbasis of the step (Sec. 2's fast diagonalisation, Phi(X) = V_y [f o
 *   (W_y^T X W_x)] V_x^T): U[b] and every g[b][k] transformed by slice GEMMs (all at once), the
 *   recurrence x^_{k+1} = f_k o x^_k + g^[b][k] run elementwise in FP32, every x^_{k+1}
 *   transformed back -- the chain's latency is that of four batched products, not nchain steps.
 * Modes 1 and 2 need BF16 and P_x = P_y in {128, 256} (else SFDE_EUNSUPPORTED) and give identical
 * results; mode 3 needs batch <= min(N_t, 512).  U: batch x N_y x N_x, g (may be NULL) and out: batch x nchain x N_y x N_x doubles (host
 * or device), rounded to the operand type on input.  Synchronous; allocates scratch.
 */
sfde_status sfde_debug_lp_chain(sfde_ctx* ctx, int mode, int scheme, const double* U, int batch, int nchain,
                                int n0, const double* g, double* out);

/*
 * P1-triangle operator (Sec. 2) hooks.
 * sfde_debug_p1_entries -- the printed Toeplitz entries as the library evaluates them (host only):
 *   a1[l] = a^{1,rho}_{k,k+l}, a2_upper[l] = a^{2,rho}_{k,k+l}, a2_lower[m] = a^{2,rho}_{p+m,p}
 *   (a2_lower[0] = 0), l, m < n; for l >= 16 through a binomial series of the differences.
 * sfde_debug_p1_apply_S -- out_b = (M_h + tau_n K) U_b, n = n0 + b dn, tau_n = (t_n - t_{n-1})/2, for
 *   batch unpadded device slices U (N_y x N_x each) of an SFDE_OP_P1 context; synchronous.
 * sfde_debug_p1_cg_stats -- conjugate-gradient iterations of the last step batch, their total and
 *   the number of step batches solved (any pointer may be NULL).
 */
sfde_status sfde_debug_p1_entries(int n, double rho, double* a1, double* a2_upper, double* a2_lower);
sfde_status sfde_debug_p1_apply_S(sfde_ctx* ctx, const double* U, int batch, int n0, int dn, double* out);
sfde_status sfde_debug_p1_cg_stats(sfde_ctx* ctx, int* last, long long* total, long long* solves);

#ifdef __cplusplus
}
#endif
#endif
