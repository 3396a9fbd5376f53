// Internal declarations of the sm_103a MGRIT solver (not part of the C ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <vector>

#include "../../include/sfde.h"

#define SFDE_MAX_RANK 4

// Round an FP32 value to the nearest TF32 value (10 explicit mantissa bits).  The tensor cores read
// FP32 storage as TF32 by dropping the low 13 bits, a biased truncation that accumulates coherently
// over many time steps; values written for TF32 products are therefore rounded first.
__device__ __forceinline__ float sfde_round_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Return SFDE_ECUDA from the enclosing function on any CUDA error.
#define SFDE_CUDA(call)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) { sfde_set_last_cuda_error(e_, #call, __FILE__, __LINE__); return SFDE_ECUDA; } \
    } while (0)

#define SFDE_TRY(call)                                    \
    do {                                                  \
        sfde_status s_ = (call);                          \
        if (s_ != SFDE_OK) return s_;                     \
    } while (0)

void sfde_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// One spatial direction: N interior nodes padded to P (a multiple of 32, >= 32).
struct SfdeDir {
    int n = 0, P = 0;
    double h = 0, rho = 0;
    double* coeffs = nullptr;  // n Toeplitz coefficients a_k (device)
    double* A = nullptr;       // P x P dense stiffness, zero padded (device)
    double* lam = nullptr;     // P generalised eigenvalues, padding = 1 (device)
    double* V = nullptr;       // P x P eigenvectors, V[i*P + k], zero padded (device)
    double* W = nullptr;       // M V, P x P (device)
    double* VT = nullptr;      // V^T (device)
    double* WT = nullptr;      // W^T (device)
    float* V32 = nullptr;      // low-precision operand copies (mixed precision), see gemm_tc.cu
    float* W32 = nullptr;
};

// Per-level storage of the MGRIT hierarchy.
struct SfdeLevel {
    int N = 0;                  // steps on this level
    std::vector<double> t;      // N+1 times (host)
    double* dt = nullptr;       // N step sizes (device): dt[n-1] = t_n - t_{n-1}
    double* u = nullptr;        // (N+1) x P^2 iterate (level 0: the solution) (device)
    double* g = nullptr;        // (N+1) x P^2 right-hand side, levels >= 1 (device)
};

// Event ring for per-launch kernel timing (see sfde_profile_enable).
struct SfdeProf {
    bool on = false;
    static const int CAP = 512;
    static const int NCLS = SFDE_PROF_CLASSES;
    cudaEvent_t ev[2 * CAP] = {};
    double flops[CAP] = {}, bytes[CAP] = {};
    int cls[CAP] = {};
    int head = 0, count = 0;
    long long launches = 0;
    long long n[NCLS] = {};
    double ms[NCLS] = {}, tot_flops[NCLS] = {}, tot_bytes[NCLS] = {};
};

struct sfde_ctx {
    SfdeDir x, y;
    double kx = 0, ky = 0;
    double omega[4] = {0, 1, 0, 1};
    int nt = 0;
    std::vector<double> t;      // host copy of the time grid
    double* dt0 = nullptr;      // level-0 step sizes (device)
    int precision = SFDE_PREC_FP64;
    cudaStream_t stream = nullptr;
    int device = 0;             // CUDA device that was current at setup (all of the context's memory)
    // data
    double* U0 = nullptr;       // padded psi_0 (device, Py x Px)
    int rank = 0;
    double* time_w = nullptr;   // nt x rank (device)
    double* px = nullptr;       // rank x Px : V_x^T b_x^r (device)
    double* py = nullptr;       // rank x Py : V_y^T b_y^r (device)
    double* bxn = nullptr;      // rank x Px : nodal load factors b_x^r, zero padded (device)
    double* byn = nullptr;      // rank x Py (device)
    double* Fd = nullptr;       // dense load (sfde_set_forcing_dense): N_t padded slices F_n (device)
    double* Fh = nullptr;       // the same in the eigenbasis, V_y^T F_n V_x (device)
    // workspace for batched steps
    size_t ws_slices = 0;
    double* T1 = nullptr;       // ws_slices x P^2 scratch
    double* T2 = nullptr;
    double* T3 = nullptr;
    double* partial = nullptr;  // per-CTA partial sums for deterministic norms
    size_t partial_cap = 0;
    double* scalar = nullptr;   // device scalar (norm^2)
    double* bound_partial = nullptr;  // block maxima of the two-level bound (analysis.cu)
    double* host_scalar = nullptr;  // pinned
    // level hierarchy (built by mgrit_solve)
    std::vector<SfdeLevel> levels;
    int lev_m = 0, lev_max = 0, lev_min = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    struct SfdeMixed* mixed = nullptr;  // tensor-core operands and inner hierarchy (mixed.cu)
    int op_kind = SFDE_OP_TENSOR;       // sfde_operator: the spatial matrices of the steps
    struct SfdeP1* p1 = nullptr;        // P1-triangle matrices and CG workspace (p1.cu)
    int fused_step = 1;         // BF16 steps as one fused kernel where the padded sizes allow it
    int fused_pair = 1;         // fused step form: 0 one CTA per slice, 1 auto (a CTA pair per slice when
                                // 2 batch <= SMs, else per two slices), 2 pair per slice, 3 pair per two slices
    int resid_digits = 0;       // digits of the tensor-core residual: 0 per iteration, else 4..7 fixed
    int resid_chunk = 0;        // time points per pass of the tensor-core residual (0: ws_slices)
    int inner_cycles_tuned = 0; // V-cycles per refinement step when mgrit_opts.inner_cycles is 0
                                // (0: the built-in 4 / 5); set by sfde_set_tuning / sfde_autotune
    int modal_chains = 1;       // 1: coarse-level F-relaxations and coarsest sweeps of the inner
                                // V-cycles in the step's eigenbasis (transforms, elementwise scan,
                                // inverse); 2: the fine level's F-relaxations too; 3: as 2 with BF16
                                // operands, as 1 with TF32; 0: none
    SfdeProf prof;
    size_t P2() const { return (size_t)x.P * (size_t)y.P; }
};

// ---- setup (setup.cu)
sfde_status sfde_setup_direction(SfdeDir& d, int n, double rho, double length, cudaStream_t s);
void sfde_free_direction(SfdeDir& d);
sfde_status sfde_project_forcing(sfde_ctx* c, const double* bx_dev, const double* by_dev);

// ---- FP64 step kernels (step_fp64.cu)
enum SfdeScheme { SCHEME_CN = 0, SCHEME_BE = 1 };

struct StepBatch {
    int batch;                 // number of slices
    const double* src; long long src_stride;   // input slice b at src + b*src_stride (elements)
    double* dst; long long dst_stride;         // output slice b (relax) or residual slice b
    const double* g; long long g_stride;       // coarse right-hand side slice b (or nullptr)
    const double* utgt; long long utgt_stride; // residual mode: u at the target (or nullptr)
    const double* dt;          // step sizes of the level: dt[n_b - 1]
    int n0, dn;                // target time index n_b = n0 + b*dn
    int scheme;                // SfdeScheme
    bool level0;               // add the level-0 load F_n (if rank > 0)
    double* norm_partial;      // residual mode: per-CTA sums of squares (or nullptr)
    // an estimate of the step's result (before g is added), slice b at guess + b*guess_stride, that
    // iterative step solves may start from (or nullptr); guess - g is used when g is set
    const double* guess;
    long long guess_stride;
};

sfde_status sfde_step_fp64(sfde_ctx* c, const StepBatch& sb, int* n_partials);
sfde_status sfde_reduce_partials(sfde_ctx* c, int n_partials, double* host_out);
sfde_status sfde_step_fp64_into(sfde_ctx* c, const StepBatch& sb, double* T1, double* T2, double* T3);
// rho_n = F_n + M_h (U_{n-1} - U_n) - tau_n K (U_{n-1} + U_n), n = n_first .. n_first+count-1, in FP64;
// written as BF16 (out_kind 0), FP32 rounded to TF32 (1) or FP32 (2) to rout (slice stride
// rout_stride elements), with
// per-CTA sums of rho^2 in partial.
sfde_status sfde_residual_fp64(sfde_ctx* c, const double* U, int n_first, int count, void* rout,
                               long long rout_stride, int out_kind, double* partial, int* n_partials);
// X_b = S^{-1} R_b by fast diagonalisation with the tensor-product matrices, S of step scheme
// SCHEME_SOLVE (M + dt/2 K) or SCHEME_SOLVE_BE (M + dt K), dt = dt[n0 + b dn - 1]; batch <= ws_slices
sfde_status sfde_fdm_solve_fp64(sfde_ctx* c, const double* R, long long r_stride, double* X, long long x_stride,
                                int batch, const double* dt, int n0, int dn, int scheme);
// ---- P1-triangle operator (p1.cu)
sfde_status sfde_p1_setup(sfde_ctx* c);
void sfde_p1_free(sfde_ctx* c);
sfde_status sfde_step_p1(sfde_ctx* c, const StepBatch& sb, int* n_partials);
sfde_status sfde_residual_norm2_p1(sfde_ctx* c, const double* U, double* norm2);
sfde_status sfde_apply_S_norm2_p1(sfde_ctx* c, const double* R, long long r_stride, int count, int n0, int dn,
                                  double* norm2);
// the batched FP64 step of the context's operator
inline sfde_status sfde_step_any(sfde_ctx* c, const StepBatch& sb, int* n_partials) {
    return c->op_kind == SFDE_OP_P1 ? sfde_step_p1(c, sb, n_partials) : sfde_step_fp64(c, sb, n_partials);
}
// Out_b = My^T X_b Mx for count padded FP64 slices (Out may not alias X)
sfde_status sfde_two_sided_fp64(sfde_ctx* c, const double* X, int count, const double* Mx, const double* My,
                                double* Out);
// sum over n = 1..N_t of ||rho_n||^2 (the residual above, nothing stored)
sfde_status sfde_residual_norm2_fp64(sfde_ctx* c, const double* U, double* norm2);
// sum over b < count of ||S_{n0 + b dn} R_b||^2, R_b = R + b r_stride (padded slices)
sfde_status sfde_apply_S_norm2(sfde_ctx* c, const double* R, long long r_stride, int count, int n0, int dn,
                               double* norm2);

// ---- tensor-core slice GEMM (gemm_tc.cu)
enum { SCHEME_SOLVE = 2,      // modal factor 1/(1 + dt sigma / 2): the solve S^{-1} alone (CN's S)
       SCHEME_SOLVE_BE = 3 };  // modal factor 1/(1 + dt sigma): the backward-Euler S^{-1} alone
enum { TC_EPI_STORE = 0, TC_EPI_SCALE = 1, TC_EPI_FINAL = 2 };

struct TcEpi {
    const float* lamx; const float* lamy; float kx, ky;   // TC_EPI_SCALE
    const double* dt; int n0, dn, scheme;
    const void* g; long long g_stride;                    // TC_EPI_FINAL
    const void* utgt; long long utgt_stride;
    double* partial;
};

struct TcArgs {
    int R, C, Cout, batch, BN, s0, ds;   // X slices s0 + b*ds, R x C each; Out_b is Cout x R
    void* out; long long out_stride;
    TcEpi e;
    int* err;                            // device error word (bounded waits)
    int oskip;                           // > 0: Out_b goes to slice b + b / oskip + 1 (the F-points
                                         // of intervals of oskip + 1 points), else to slice b
};

// Runs f() and returns its status; a C++ exception from host code (an allocation, a thread that
// cannot start) becomes SFDE_ENOMEM, so nothing throws across the C ABI.
template <typename F>
sfde_status sfde_no_throw(F&& f) noexcept {
    try {
        return f();
    } catch (...) {
        return SFDE_ENOMEM;
    }
}

int sfde_tc_tile_n(int cout);
int sfde_tc_partials_per_tile();   // partial sums of squares the slice GEMM writes per output tile
sfde_status sfde_tc_prepare();
sfde_status sfde_tc_map_slices(CUtensorMap* map, const void* base, int esz, int K, int R, int ds, long long nslices);
sfde_status sfde_tc_map_matrix(CUtensorMap* map, const void* matT, int esz, int K, int N);
// the fixed-matrix operand (Mat^T, N x K) of sfde_tc_gemm of operand kind `kind`: boxes of the
// slice GEMM's tile rows (half of them in its CTA-pair form)
sfde_status sfde_tc_map_gemm_matrix(CUtensorMap* map, const void* matT, int kind, int K, int N);
// as sfde_tc_map_matrix with boxes of `rows` rows (<= 256)
sfde_status sfde_tc_map_matrix_rows(CUtensorMap* map, const void* matT, int esz, int K, int N, int rows);
// kind 0: BF16 operands and storage; 1: FP32 storage rounded to TF32, TF32 products; 2: FP32 storage,
// products from three TF32 products each (Blo: the map of the fixed matrix's low parts, required).
// c may be NULL (no accounting); nr, nc, nout: unpadded extents of one slice product
sfde_status sfde_tc_gemm(sfde_ctx* c, int kind, int epi, const CUtensorMap& A, const CUtensorMap& B, const TcArgs& p,
                         cudaStream_t s, int nr = 0, int nc = 0, int nout = 0, const CUtensorMap* Blo = nullptr);
// dst = lo(src) = src - (src with its 13 low mantissa bits cleared), n FP32 values (kind 2 operands)
sfde_status sfde_tc_lo_parts(const float* src, float* dst, size_t n, cudaStream_t s);

// ---- one whole spectral step per CTA, four chained BF16 products on chip (fused_step.cu)
struct FusedStepArgs {
    int s0, ds, batch;                    // source slices s0 + b*ds (through the slice tensor map)
    int nchain;                           // steps per CTA: step k > 0 starts from step k-1's output
    void* dst; long long dst_stride;      // output of step k for slice b at dst + b*dst_stride +
    long long dst_kstride;                //   k*dst_kstride (elements)
    const void* g; long long g_stride;    // added to the output (or nullptr); step k: + k*g_kstride
    long long g_kstride;
    int g_tma;                            // pair per slice, chained: g also through the tensor map
                                          //   of the g slices (slice b*g_tds + k), staged in shared memory
    int g_tds;
    const void* ut; long long ut_stride;  // subtracted; sum of squares per slice into partial[b]
    double* partial;                      // batch entries (or nullptr)
    const float* lamx; const float* lamy; float kx, ky;
    const double* dt; int n0, dn, scheme; // step k of slice b: dt[n0 + b*dn - 1 + k]; SfdeScheme / SCHEME_SOLVE
    int* err;                             // device error word (bounded waits)
};
bool sfde_fused_supported(int kind, int Px, int Py);
// low-precision operand kind of a mixed-precision context: 0 BF16, 1 TF32, 2 FP32 from three TF32
// products (SFDE_PREC_MIXED_AUTO resolved by size and length, see include/sfde.h)
inline int sfde_mixed_kind(const sfde_ctx* c) {
    if (c->precision == SFDE_PREC_MIXED_BF16) return 0;
    if (c->precision == SFDE_PREC_MIXED_TF32) return 1;
    if (c->precision == SFDE_PREC_MIXED_FP32) return 2;
    return 2;   // SFDE_PREC_MIXED_AUTO
}
sfde_status sfde_fused_prepare();
// O1, O2: W_x^T, W_y^T (V_x^T, V_y^T for the solve); O3, O4: V_x, V_y -- K-major P x P BF16 maps
// with boxes of 64 x P (form 0: one CTA per slice) or 64 x 128 (P = 256, a CTA pair per one slice,
// form 1, or per two slices, form 2).
bool sfde_fused_pair_supported(int P);
sfde_status sfde_fused_step(sfde_ctx* c, int P, int form, const CUtensorMap& U, const CUtensorMap& O1,
                            const CUtensorMap& O2, const CUtensorMap& O3, const CUtensorMap& O4, const CUtensorMap& Gm,
                            const FusedStepArgs& a, cudaStream_t s);

// ---- FP64-accurate slice GEMM on the BF16 tensor cores (ozaki.cu)
#define SFDE_OZ_DIGITS 6
struct OzMatrix {            // a fixed K x N FP64 matrix split into SFDE_OZ_DIGITS BF16 digit planes
    int K = 0, N = 0;
    void* digits = nullptr;  // planes of N x K (K-major)
    int* exps = nullptr;     // one exponent per column (device)
    int e_uniform = 0;       // the common exponent when split with one scale for the whole matrix
    int nd = 0;              // digit planes: 7 with one scale (integer-output product), else 6
    CUtensorMap map;         // tiles of 32 columns
    CUtensorMap map_wide;    // tiles of 64 columns (integer output, N a multiple of 64), if wide
    bool wide = false;
};
// digits of alpha * Mat; uniform: one exponent (max_kn |alpha m_kn| < 2^e) for all columns and seven
// digits (for sfde_oz_gemm_int), else one exponent per column and six digits (for sfde_oz_gemm)
sfde_status sfde_oz_split_matrix(const double* Mat, int K, int N, OzMatrix* out, cudaStream_t s, double alpha,
                                 bool uniform);
void sfde_oz_free_matrix(OzMatrix* m);
size_t sfde_oz_digit_bytes(int R, int K, int batch);
// Out_b = ((X_b [+ X2_b]) Mat)^T in FP64 accuracy; digits (sfde_oz_digit_bytes) and xe (batch x R ints)
// are scratch.  K <= 256.
sfde_status sfde_oz_gemm(sfde_ctx* c, const double* X, const double* X2, long long x_stride, int R, int K,
                         int batch, const OzMatrix& M, void* digits, int* xe, double* out, long long out_stride,
                         int* err, int nr, int nc, int nout);

// The same product on pre-split operand digits (seven planes `plane` elements apart) with the 28 digit
// products p + q <= 8, written as int64 in units of 2^-52 of the operand scales (uniform-exponent
// matrix); exact up to rounding the p + q >= 7 terms to that unit.
int sfde_oz_int_shift(int K);  // the integer product's extra right shift for contraction length K
sfde_status sfde_oz_gemm_int(sfde_ctx* c, void* xdigits, long long plane, int R, int K, int batch,
                             const OzMatrix& M, long long* out, long long out_stride, int* err, int nr, int nc,
                             int nout, int nd);

// ---- the space-time residual of sfde_residual_fp64 in integer arithmetic around two digit-split
// tensor-core products (resid_int.cu), Px, Py <= 1024.  Ax, Ay from sfde_resid_int_matrices; dV, dVt:
// sfde_resid_int_digit_bytes(Px, Py, ws_slices) each (digits of 2V row-major and transposed); En:
// N_t + 1 ints; err: device error word; nd: digits per operand, 4..7 (7: exact operands; fewer
// digits truncate V and the matrices at about 2^{9-8 nd} of their scales); n_zero: U_n = 0 for every
// n >= n_zero - 1 is known (INT_MAX: nothing known), so those pairs are the load alone (the same
// values, no products formed).
bool sfde_resid_int_supported(int Px, int Py);
size_t sfde_resid_int_digit_bytes(int Px, int Py, int batch);
sfde_status sfde_resid_int_matrices(sfde_ctx* c, OzMatrix* Ax, OzMatrix* Ay);
sfde_status sfde_residual_int(sfde_ctx* c, const double* U, int n_first, int count, void* rout,
                              long long rout_stride, int out_kind, double* partial, int* n_partials,
                              const OzMatrix& Ax, const OzMatrix& Ay, void* dV, void* dVt, int* En, int* err,
                              int nd, int n_zero);
void sfde_launch_mass_x_transpose(const double* Un, const double* Um, double* T2, int Px, int Py, double hx,
                                  int nb, cudaStream_t s);

// ---- MGRIT engine (mgrit.cu)
sfde_status sfde_mgrit_fp64(sfde_ctx* c, const mgrit_opts* o, mgrit_stats* st);
sfde_status sfde_seq_fp64(sfde_ctx* c, double* seconds);
sfde_status sfde_ensure_workspace(sfde_ctx* c, size_t slices);
// two-level analysis (analysis.cu): Theorem 3.1's bound on the device, the coarse propagator of
// SFDE_COARSE_AUTO, the coarsening factor of mgrit_opts.m = 0
sfde_status sfde_tub_bound_device(sfde_ctx* c, int m, int coarse, double* out);
sfde_status sfde_choose_coarse(sfde_ctx* c, int m, int requested, int* coarse, double* tub);
sfde_status sfde_choose_m(sfde_ctx* c, int requested_coarse, double rel_tol, int* m_out);

// ---- kernel accounting (api.cu)
int sfde_prof_begin(sfde_ctx* c);                               // slot or -1 when timing is off
void sfde_prof_end(sfde_ctx* c, int slot, int cls, double flops, double bytes);
inline void sfde_count_launch(sfde_ctx* c, int n = 1) { c->prof.launches += n; }

// ---- helpers (api.cu)
bool sfde_is_device_ptr(const void* p);
sfde_status sfde_copy_in(void* dst_dev, const void* src, size_t bytes, cudaStream_t s);
sfde_status sfde_copy_out(void* dst, const void* src_dev, size_t bytes, cudaStream_t s);

// padded <-> unpadded slice copies (setup.cu)
void sfde_launch_pad(const double* src, double* dst, int ny, int nx, int Py, int Px, int slices,
                     cudaStream_t s);
void sfde_launch_unpad(const double* src, double* dst, int ny, int nx, int Py, int Px, int slices,
                       cudaStream_t s);
void sfde_launch_unpad_f32(const float* src, float* dst, int ny, int nx, int Py, int Px, int slices,
                           cudaStream_t s);
sfde_status sfde_level0(sfde_ctx* c, double** u);
void sfde_launch_fill_random(double* u, int nt, int ny, int nx, int Py, int Px, uint64_t seed,
                             cudaStream_t s);
void sfde_launch_axpy_strided(double* y, long long y_stride, const double* x, long long x_stride,
                              int slices, size_t P2, cudaStream_t s);
