// FP64 fine/coarse step on a batch of time slices: the "spectral step" form of one step solve.
//
// For the Kronecker operator of Eq. (2.4) with generalised eigenpairs A V = M V diag(lambda),
// V^T M V = I, W = M V and sigma[j][i] = K_x lambda_x[i] + K_y lambda_y[j], the solution of
// S_n X = B_n U + F_n is
//     X = V_y [ Lt_n o (W_y^T U W_x) + (V_y^T F_n V_x) / (1 + tau_n sigma) ] V_x^T,
//     Lt_n = (1 - tau_n sigma)/(1 + tau_n sigma)   (the eigenvalues of Psi_n, Eq. (3.7)),
// i.e. four dense GEMMs with the fast-diagonalisation scaling fused into the second one; for the
// backward-Euler coarse propagator Lt = 1/(1 + dt sigma).  The load term uses the separable
// factors px = V_x^T b_x, py = V_y^T b_y.
//
// Every GEMM has the form  Out_b = (X_b Mat)^T  for slices b of a batch: X_b is R x C (row-major),
// Mat is C x C' (row-major), Out_b is C' x R.  Storing the transpose lets all four products be
// right-multiplications of stacked slices:
//     T1 = (U W_x)^T,  T2 = (T1 W_y)^T = W_y^T U W_x (scaled),  T3 = (T2 V_x^T)^T,  X = (T3 V_y^T)^T.
// On GB300 FP64 runs at a small fraction of the tensor-core rate, so this kernel is bound by the
// FP64 pipe; tiles are sized so that even a batch of one slice fills all SMs.
#include <cuda_bf16.h>

#include <algorithm>

#include "sfde_internal.cuh"

namespace {

enum Epi { EPI_STORE = 0, EPI_MODAL = 1, EPI_FINAL = 2, EPI_RESID_BF16 = 3, EPI_RESID_F32 = 4, EPI_RESID_NONE = 5,
           EPI_RESID_F32X = 6 };

struct GemmParams {
    const double* X; long long x_stride; int R, C;
    const double* X2;   // optional second operand slice: the A operand is X_b + X2_b (same layout)
    const double* Mat; int Cout;
    double* Out; long long out_stride;
    int batch;
    // EPI_MODAL
    const double* lamx; const double* lamy; double kx, ky;
    const double* dt; int n0, dn, scheme;
    int rank; const double* time_w; const double* px; const double* py;
    const double* Fh;          // dense load in the eigenbasis, V_y^T F_n V_x (slice n-1), or null
    const double* Fd;          // dense nodal load F_n (slice n-1, padded), or null (EPI_RESID_*)
    // EPI_FINAL
    const double* g; long long g_stride;
    const double* utgt; long long utgt_stride;
    double* partial;
    // EPI_RESID_*: space-time residual rho_n = F_n + M_h (U_{n-1} - U_n) - tau_n K (U_{n-1} + U_n)
    // for slice b: U_n = Ucur + b u_stride, U_{n-1} = Uprev + b u_stride (Uprev may be null: zero),
    // n = n0 + b tdn; F_n only when load is set
    const double* t1;          // (V A_x)^T slices, Px x Py
    const double* Ucur; const double* Uprev; long long u_stride; int tdn; int load;
    const double* bxn; const double* byn;   // nodal load factors (padded)
    double hx, hy;
    int Px, Py, nx, ny;
    void* rout;                // residual output (BF16 or FP32), slice b at rout + b * out_stride
};

constexpr int BK = 16;

template <int EPI> struct ResidOut { using T = double; };
template <> struct ResidOut<EPI_RESID_BF16> { using T = __nv_bfloat16; };
template <> struct ResidOut<EPI_RESID_F32> { using T = float; };
template <> struct ResidOut<EPI_RESID_F32X> { using T = float; };
constexpr bool is_resid(int e) {
    return e == EPI_RESID_BF16 || e == EPI_RESID_F32 || e == EPI_RESID_NONE || e == EPI_RESID_F32X;
}

__device__ __forceinline__ void store_as(__nv_bfloat16* p, double v) { *p = __float2bfloat16_rn((float)v); }
__device__ __forceinline__ void store_as(float* p, double v) { *p = sfde_round_tf32((float)v); }
__device__ __forceinline__ void store_as(double* p, double v) { *p = v; }

template <int T, int EPI>
__global__ void __launch_bounds__(256) k_slice_gemm_fp64(GemmParams p) {
    constexpr int MT = T / 16;  // micro-tile edge
    __shared__ double As[BK][T + 1];
    __shared__ double Bs[BK][T + 1];
    __shared__ double red[256];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const long long m0 = (long long)blockIdx.x * T;
    const int n0 = blockIdx.y * T;
    const long long Mtot = (long long)p.batch * p.R;

    double acc[MT][MT];
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < MT; ++j) acc[i][j] = 0.0;

    for (int k0 = 0; k0 < p.C; k0 += BK) {
        for (int e = threadIdx.x; e < T * BK; e += 256) {
            int row = e / BK, kk = e % BK;
            long long m = m0 + row;
            double v = 0.0;
            if (m < Mtot) {
                long long b = m / p.R, r = m % p.R;
                const long long a = b * p.x_stride + r * p.C + k0 + kk;
                v = p.X[a];
                if (p.X2) v += p.X2[a];
            }
            As[kk][row] = v;
        }
        for (int e = threadIdx.x; e < T * BK; e += 256) {
            int kk = e / T, col = e % T;
            Bs[kk][col] = p.Mat[(size_t)(k0 + kk) * p.Cout + n0 + col];
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[MT], bv[MT];
#pragma unroll
            for (int i = 0; i < MT; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < MT; ++j) bv[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < MT; ++i)
#pragma unroll
                for (int j = 0; j < MT; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }

    double sq = 0.0;
#pragma unroll
    for (int i = 0; i < MT; ++i) {
        long long m = m0 + tx + 16 * i;
        if (m >= Mtot) continue;
        long long b = m / p.R;
        int r = (int)(m % p.R);
#pragma unroll
        for (int j = 0; j < MT; ++j) {
            int n = n0 + ty + 16 * j;
            double v = acc[i][j];
            long long o = (long long)n * p.R + r;
            if (EPI == EPI_MODAL) {
                // element (j = n, i = r) of W_y^T U W_x for slice b
                int tn = p.n0 + (int)b * p.dn;            // target time index of this slice
                double dt = p.dt[tn - 1];
                double sig = p.kx * p.lamx[r] + p.ky * p.lamy[n];
                double lt;
                if (p.scheme == SCHEME_CN) {
                    double ts = 0.5 * dt * sig;
                    lt = (1.0 - ts) / (1.0 + ts);
                } else if (p.scheme == SCHEME_SOLVE) {
                    lt = 1.0 / (1.0 + 0.5 * dt * sig);
                } else {   // SCHEME_BE, SCHEME_SOLVE_BE
                    lt = 1.0 / (1.0 + dt * sig);
                }
                v *= lt;
                if (p.rank > 0) {
                    double f = 0.0;
                    for (int q = 0; q < p.rank; ++q)
                        f += p.time_w[(size_t)(tn - 1) * p.rank + q] * p.py[(size_t)q * p.Cout + n] *
                             p.px[(size_t)q * p.R + r];
                    v += f / (1.0 + 0.5 * dt * sig);
                }
                if (p.Fh) v += p.Fh[(size_t)(tn - 1) * ((size_t)p.R * p.Cout) + o] / (1.0 + 0.5 * dt * sig);
            } else if (EPI == EPI_FINAL) {
                if (p.g) v += p.g[b * p.g_stride + o];
                if (p.utgt) {
                    v -= p.utgt[b * p.utgt_stride + o];
                    sq += v * v;
                }
            } else if (is_resid(EPI)) {
                // element (j = n, i = r) of slice b; acc = (A_y (V M_x))[j][i]
                const int i = r, j = n;
                const int tn = p.n0 + (int)b * p.tdn;    // time index of this residual
                const double tau = 0.5 * p.dt[tn - 1];
                const size_t P2 = (size_t)p.Px * p.Py;
                const double* T1 = p.t1 + (size_t)b * P2 + (size_t)i * p.Py;   // row i of (V A_x)^T
                const double my = p.hy / 6.0;
                double y1 = 4.0 * T1[j];
                if (j > 0) y1 += T1[j - 1];
                if (j + 1 < p.Py) y1 += T1[j + 1];
                const double stiff = p.kx * my * y1 + p.ky * v;
                const double* Ua = p.Uprev ? p.Uprev + b * p.u_stride : nullptr;
                const double* Ub = p.Ucur + b * p.u_stride;
                const double wx[3] = {p.hx / 6.0, 4.0 * p.hx / 6.0, p.hx / 6.0};
                const double wy[3] = {my, 4.0 * my, my};
                double mass = 0.0;
#pragma unroll
                for (int a = -1; a <= 1; ++a) {
                    const int jj = j + a;
                    if (jj < 0 || jj >= p.Py) continue;
                    double row = 0.0;
#pragma unroll
                    for (int cc = -1; cc <= 1; ++cc) {
                        const int ii = i + cc;
                        if (ii < 0 || ii >= p.Px) continue;
                        const size_t e = (size_t)jj * p.Px + ii;
                        row += wx[cc + 1] * ((Ua ? Ua[e] : 0.0) - Ub[e]);
                    }
                    mass += wy[a + 1] * row;
                }
                double f = 0.0;
                if (p.load) {
                    for (int q = 0; q < p.rank; ++q)
                        f += p.time_w[(size_t)(tn - 1) * p.rank + q] * p.byn[(size_t)q * p.Py + j] * p.bxn[(size_t)q * p.Px + i];
                    if (p.Fd) f += p.Fd[(size_t)(tn - 1) * P2 + (size_t)j * p.Px + i];
                }
                // padded rows/columns are not unknowns: the stencils above reach one past the last
                // interior node, so the residual is defined as zero there
                const double rho = (i < p.nx && j < p.ny) ? f + mass - tau * stiff : 0.0;
                sq += rho * rho;
                if (EPI == EPI_RESID_F32X) {
                    ((float*)p.rout)[b * p.out_stride + o] = (float)rho;   // FP32, not rounded to TF32
                } else if (EPI != EPI_RESID_NONE) {
                    using OT = typename ResidOut<EPI>::T;
                    store_as((OT*)p.rout + b * p.out_stride + o, rho);
                }
                continue;
            }
            p.Out[b * p.out_stride + o] = v;
        }
    }
    if ((EPI == EPI_FINAL || is_resid(EPI)) && p.partial) {
        red[threadIdx.x] = sq;
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) p.partial[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = red[0];
    }
}

// Fixed-order sum of the per-CTA partials (deterministic norms).  Each thread keeps eight partial
// sums, so eight loads are in flight at a time.
__global__ void k_reduce_partials(const double* partial, int n, double* out) {
    __shared__ double s[1024];
    double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const int step = blockDim.x * 8;
    int i0 = threadIdx.x;
    for (; i0 + 7 * (int)blockDim.x < n; i0 += step)
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] += partial[i0 + k * blockDim.x];
    for (int k = 0; k < 8; ++k)
        if (i0 + k * (int)blockDim.x < n) a[k] += partial[i0 + k * blockDim.x];
    double v = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    s[threadIdx.x] = v;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

int choose_tile(long long rows, int cout, int pmin) {
    const long long target = 2 * 152;
    int T = 64;
    while (T > 16 && (T > pmin || ((rows + T - 1) / T) * (cout / T) < target)) T /= 2;
    return T;
}

// nr, nc, nout: unpadded extents of one slice product (algorithmic work for the profile)
template <int EPI>
void launch_T(sfde_ctx* c, int T, const GemmParams& p, int nr, int nc, int nout) {
    long long rows = (long long)p.batch * p.R;
    dim3 grid((unsigned)((rows + T - 1) / T), p.Cout / T);
    int slot = sfde_prof_begin(c);
    if (T == 64) k_slice_gemm_fp64<64, EPI><<<grid, 256, 0, c->stream>>>(p);
    else if (T == 32) k_slice_gemm_fp64<32, EPI><<<grid, 256, 0, c->stream>>>(p);
    else k_slice_gemm_fp64<16, EPI><<<grid, 256, 0, c->stream>>>(p);
    const double b = p.batch;
    sfde_prof_end(c, slot, (is_resid(EPI) || p.X2) ? 1 : 0, 2.0 * b * nr * nc * nout,
                  8.0 * (b * nr * nc + b * nr * nout + (double)nc * nout + (EPI == EPI_FINAL && p.utgt ? b * nr * nout : 0.0)));
    sfde_count_launch(c);
}

}  // namespace

sfde_status sfde_reduce_partials(sfde_ctx* c, int n_partials, double* host_out) {
    k_reduce_partials<<<1, 1024, 0, c->stream>>>(c->partial, n_partials, c->scalar);
    sfde_count_launch(c);
    SFDE_CUDA(cudaGetLastError());
    SFDE_CUDA(cudaMemcpyAsync(c->host_scalar, c->scalar, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    SFDE_CUDA(cudaStreamSynchronize(c->stream));
    *host_out = *c->host_scalar;
    return SFDE_OK;
}

sfde_status sfde_step_fp64(sfde_ctx* c, const StepBatch& sb, int* n_partials) {
    const int Px = c->x.P, Py = c->y.P;
    const size_t P2 = c->P2();
    const int pmin = Px < Py ? Px : Py;
    int total_partials = 0;
    for (int b0 = 0; b0 < sb.batch; b0 += (int)c->ws_slices) {
        int nb = sb.batch - b0;
        if (nb > (int)c->ws_slices) nb = (int)c->ws_slices;
        GemmParams p{};
        p.batch = nb;
        // G1: T1 = (U W_x)^T
        p.X = sb.src + (long long)b0 * sb.src_stride; p.x_stride = sb.src_stride; p.R = Py; p.C = Px;
        p.Mat = c->x.W; p.Cout = Px; p.Out = c->T1; p.out_stride = (long long)P2;
        launch_T<EPI_STORE>(c, choose_tile((long long)nb * Py, Px, pmin), p, c->y.n, c->x.n, c->x.n);
        // G2: T2 = (T1 W_y)^T, scaled in the modal basis (+ load)
        GemmParams q{};
        q.batch = nb; q.X = c->T1; q.x_stride = (long long)P2; q.R = Px; q.C = Py;
        q.Mat = c->y.W; q.Cout = Py; q.Out = c->T2; q.out_stride = (long long)P2;
        q.lamx = c->x.lam; q.lamy = c->y.lam; q.kx = c->kx; q.ky = c->ky;
        q.dt = sb.dt; q.n0 = sb.n0 + b0 * sb.dn; q.dn = sb.dn; q.scheme = sb.scheme;
        q.rank = (sb.level0 ? c->rank : 0); q.time_w = c->time_w; q.px = c->px; q.py = c->py;
        q.Fh = sb.level0 ? c->Fh : nullptr;
        launch_T<EPI_MODAL>(c, choose_tile((long long)nb * Px, Py, pmin), q, c->x.n, c->y.n, c->y.n);
        // G3: T3 = (T2 V_x^T)^T
        GemmParams r{};
        r.batch = nb; r.X = c->T2; r.x_stride = (long long)P2; r.R = Py; r.C = Px;
        r.Mat = c->x.VT; r.Cout = Px; r.Out = c->T3; r.out_stride = (long long)P2;
        launch_T<EPI_STORE>(c, choose_tile((long long)nb * Py, Px, pmin), r, c->y.n, c->x.n, c->x.n);
        // G4: X = (T3 V_y^T)^T (+ g) (- u_target, squared into partial sums)
        GemmParams f{};
        f.batch = nb; f.X = c->T3; f.x_stride = (long long)P2; f.R = Px; f.C = Py;
        f.Mat = c->y.VT; f.Cout = Py;
        f.Out = sb.dst + (long long)b0 * sb.dst_stride; f.out_stride = sb.dst_stride;
        f.g = sb.g ? sb.g + (long long)b0 * sb.g_stride : nullptr; f.g_stride = sb.g_stride;
        f.utgt = sb.utgt ? sb.utgt + (long long)b0 * sb.utgt_stride : nullptr; f.utgt_stride = sb.utgt_stride;
        int T = choose_tile((long long)nb * Px, Py, pmin);
        long long ctas = (((long long)nb * Px + T - 1) / T) * (Py / T);
        f.partial = sb.norm_partial ? sb.norm_partial + total_partials : nullptr;
        if (sb.norm_partial && (size_t)(total_partials + ctas) > c->partial_cap) return SFDE_EINVAL;
        launch_T<EPI_FINAL>(c, T, f, c->x.n, c->y.n, c->y.n);
        total_partials += (int)ctas;
    }
    SFDE_CUDA(cudaGetLastError());
    if (n_partials) *n_partials = total_partials;
    return SFDE_OK;
}

namespace {

// Launch without event timing or launch accounting (nothing is created or allocated).
template <int EPI>
void launch_plain(int T, const GemmParams& p, cudaStream_t s) {
    long long rows = (long long)p.batch * p.R;
    dim3 grid((unsigned)((rows + T - 1) / T), p.Cout / T);
    if (T == 64) k_slice_gemm_fp64<64, EPI><<<grid, 256, 0, s>>>(p);
    else if (T == 32) k_slice_gemm_fp64<32, EPI><<<grid, 256, 0, s>>>(p);
    else k_slice_gemm_fp64<16, EPI><<<grid, 256, 0, s>>>(p);
}

}  // namespace

// The four products of sfde_step_fp64 for one batch, with caller-provided intermediate buffers
// T1, T2, T3 (batch x P^2 doubles each); no residual or norm.
sfde_status sfde_step_fp64_into(sfde_ctx* c, const StepBatch& sb, double* T1, double* T2, double* T3) {
    const int Px = c->x.P, Py = c->y.P;
    const long long P2 = (long long)c->P2();
    const int pmin = Px < Py ? Px : Py;
    const int nb = sb.batch;
    GemmParams p{};
    p.batch = nb; p.X = sb.src; p.x_stride = sb.src_stride; p.R = Py; p.C = Px;
    p.Mat = c->x.W; p.Cout = Px; p.Out = T1; p.out_stride = P2;
    launch_plain<EPI_STORE>(choose_tile((long long)nb * Py, Px, pmin), p, c->stream);
    GemmParams q{};
    q.batch = nb; q.X = T1; q.x_stride = P2; q.R = Px; q.C = Py;
    q.Mat = c->y.W; q.Cout = Py; q.Out = T2; q.out_stride = P2;
    q.lamx = c->x.lam; q.lamy = c->y.lam; q.kx = c->kx; q.ky = c->ky;
    q.dt = sb.dt; q.n0 = sb.n0; q.dn = sb.dn; q.scheme = sb.scheme;
    q.rank = (sb.level0 ? c->rank : 0); q.time_w = c->time_w; q.px = c->px; q.py = c->py;
    q.Fh = sb.level0 ? c->Fh : nullptr;
    launch_plain<EPI_MODAL>(choose_tile((long long)nb * Px, Py, pmin), q, c->stream);
    GemmParams r{};
    r.batch = nb; r.X = T2; r.x_stride = P2; r.R = Py; r.C = Px;
    r.Mat = c->x.VT; r.Cout = Px; r.Out = T3; r.out_stride = P2;
    launch_plain<EPI_STORE>(choose_tile((long long)nb * Py, Px, pmin), r, c->stream);
    GemmParams f{};
    f.batch = nb; f.X = T3; f.x_stride = P2; f.R = Px; f.C = Py;
    f.Mat = c->y.VT; f.Cout = Py; f.Out = sb.dst; f.out_stride = sb.dst_stride;
    launch_plain<EPI_FINAL>(choose_tile((long long)nb * Px, Py, pmin), f, c->stream);
    SFDE_CUDA(cudaGetLastError());
    return SFDE_OK;
}

namespace {

// T2_b = ((U_n + U_{n-1}) M_x)^T for a batch of slices (stride us; Um may be null: zero): the
// x-direction mass stencil (h_x/6)(v_{i-1} + 4 v_i + v_{i+1}) fused with the sum of two time slices
// and a tile transpose.
__global__ void k_mass_x_transpose(const double* Un, const double* Um, long long us, double* T2, int Px, int Py,
                                   double hx) {
    __shared__ double tile[32][35];
    const size_t P2 = (size_t)Px * Py;
    const size_t sl = blockIdx.z;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const double* a = Un + sl * us;
    const double* b = Um ? Um + sl * us : nullptr;
    // rows j0..j0+31, columns i0-1..i0+32 (halo) into tile[j][1 + i]
    for (int jj = threadIdx.y; jj < 32; jj += blockDim.y) {
        const int j = j0 + jj;
        for (int ii = threadIdx.x; ii < 34; ii += 32) {
            const int i = i0 + ii - 1;
            double v = 0.0;
            if (i >= 0 && i < Px) v = a[(size_t)j * Px + i] + (b ? b[(size_t)j * Px + i] : 0.0);
            tile[jj][ii] = v;
        }
    }
    __syncthreads();
    const double w = hx / 6.0;
    for (int ii = threadIdx.y; ii < 32; ii += blockDim.y) {
        const int jj = threadIdx.x;
        const double v = w * (tile[jj][ii] + 4.0 * tile[jj][ii + 1] + tile[jj][ii + 2]);
        T2[sl * P2 + (size_t)(i0 + ii) * Py + j0 + jj] = v;
    }
}

}  // namespace

void sfde_launch_mass_x_transpose(const double* Un, const double* Um, double* T2, int Px, int Py, double hx,
                                  int nb, cudaStream_t s) {
    k_mass_x_transpose<<<dim3(Px / 32, Py / 32, nb), dim3(32, 8), 0, s>>>(Un, Um, (long long)Px * Py, T2, Px, Py, hx);
}

namespace {

// rho_b = [F_n] + M_h (Uprev_b - Ucur_b) - tau_n K (Uprev_b + Ucur_b) for slices b < count,
// Ucur_b = Ucur + b u_stride, Uprev_b = Uprev + b u_stride (Uprev null: zero), n = n0 + b tdn, in
// chunks of the FP64 workspace; out_kind 0 BF16, 1 FP32 rounded to TF32, 2 FP32, 3 none (sums of
// squares only)
sfde_status resid_general(sfde_ctx* c, const double* Ucur, const double* Uprev, long long u_stride, int n0,
                          int tdn, int count, bool load, void* rout, long long rout_stride, int out_kind,
                          double* partial, int* n_partials) {
    const int Px = c->x.P, Py = c->y.P;
    const size_t P2 = c->P2();
    const int pmin = Px < Py ? Px : Py;
    const size_t esz = out_kind == 0 ? 2 : 4;
    int total = 0;
    for (int b0 = 0; b0 < count; b0 += (int)c->ws_slices) {
        int nb = count - b0;
        if (nb > (int)c->ws_slices) nb = (int)c->ws_slices;
        const double* ucur = Ucur + (size_t)b0 * u_stride;
        const double* uprev = Uprev ? Uprev + (size_t)b0 * u_stride : nullptr;
        // (V A_x)^T with V = U_n + U_{n-1} formed while loading
        GemmParams p{};
        p.batch = nb; p.X = ucur; p.X2 = uprev; p.x_stride = u_stride;
        p.R = Py; p.C = Px; p.Mat = c->x.A; p.Cout = Px; p.Out = c->T1; p.out_stride = (long long)P2;
        launch_T<EPI_STORE>(c, choose_tile((long long)nb * Py, Px, pmin), p, c->y.n, c->x.n, c->x.n);
        // ((U_n + U_{n-1}) M_x)^T
        k_mass_x_transpose<<<dim3(Px / 32, Py / 32, nb), dim3(32, 8), 0, c->stream>>>(ucur, uprev, u_stride, c->T2, Px,
                                                                                        Py, c->x.h);
        sfde_count_launch(c);
        // A_y (V M_x), then the residual epilogue
        GemmParams q{};
        q.batch = nb; q.X = c->T2; q.x_stride = (long long)P2; q.R = Px; q.C = Py;
        q.Mat = c->y.A; q.Cout = Py; q.out_stride = rout_stride;
        q.kx = c->kx; q.ky = c->ky; q.dt = c->dt0; q.n0 = n0 + b0 * tdn; q.tdn = tdn;
        q.load = load ? 1 : 0;
        q.rank = c->rank; q.time_w = c->time_w; q.bxn = c->bxn; q.byn = c->byn; q.Fd = c->Fd;
        q.t1 = c->T1; q.Ucur = ucur; q.Uprev = uprev; q.u_stride = u_stride;
        q.hx = c->x.h; q.hy = c->y.h; q.Px = Px; q.Py = Py;
        q.nx = c->x.n; q.ny = c->y.n;
        q.rout = rout ? (char*)rout + (size_t)b0 * rout_stride * esz : nullptr;
        const int T = choose_tile((long long)nb * Px, Py, pmin);
        const long long ctas = (((long long)nb * Px + T - 1) / T) * (Py / T);
        if ((size_t)(total + ctas) > c->partial_cap) return SFDE_EINVAL;
        q.partial = partial + total;
        if (out_kind == 0) launch_T<EPI_RESID_BF16>(c, T, q, c->x.n, c->y.n, c->y.n);
        else if (out_kind == 1) launch_T<EPI_RESID_F32>(c, T, q, c->x.n, c->y.n, c->y.n);
        else if (out_kind == 2) launch_T<EPI_RESID_F32X>(c, T, q, c->x.n, c->y.n, c->y.n);
        else launch_T<EPI_RESID_NONE>(c, T, q, c->x.n, c->y.n, c->y.n);
        total += (int)ctas;
    }
    SFDE_CUDA(cudaGetLastError());
    if (n_partials) *n_partials = total;
    return SFDE_OK;
}

}  // namespace

sfde_status sfde_residual_fp64(sfde_ctx* c, const double* U, int n_first, int count, void* rout,
                               long long rout_stride, int out_kind, double* partial, int* n_partials) {
    const size_t P2 = c->P2();
    return resid_general(c, U + (size_t)n_first * P2, U + (size_t)(n_first - 1) * P2, (long long)P2, n_first, 1, count,
                         true, rout, rout_stride, out_kind, partial, n_partials);
}

sfde_status sfde_residual_norm2_fp64(sfde_ctx* c, const double* U, double* norm2) {
    if (c->op_kind == SFDE_OP_P1) return sfde_residual_norm2_p1(c, U, norm2);
    const size_t P2 = c->P2();
    double acc = 0.0;
    const int chunk = (int)c->ws_slices;
    for (int n = 1; n <= c->nt; n += chunk) {
        const int cnt = std::min(chunk, c->nt - n + 1);
        int np = 0;
        SFDE_TRY(resid_general(c, U + (size_t)n * P2, U + (size_t)(n - 1) * P2, (long long)P2, n, 1, cnt, true,
                               nullptr, 0, 3, c->partial, &np));
        double r2 = 0.0;
        SFDE_TRY(sfde_reduce_partials(c, np, &r2));
        acc += r2;
    }
    *norm2 = acc;
    return SFDE_OK;
}

sfde_status sfde_apply_S_norm2(sfde_ctx* c, const double* R, long long r_stride, int count, int n0, int dn,
                               double* norm2) {
    if (c->op_kind == SFDE_OP_P1) return sfde_apply_S_norm2_p1(c, R, r_stride, count, n0, dn, norm2);
    double acc = 0.0;
    const int chunk = (int)c->ws_slices;
    for (int b = 0; b < count; b += chunk) {
        const int cnt = std::min(chunk, count - b);
        int np = 0;
        SFDE_TRY(resid_general(c, R + (size_t)b * r_stride, nullptr, r_stride, n0 + b * dn, dn, cnt, false, nullptr, 0,
                               3, c->partial, &np));
        double r2 = 0.0;
        SFDE_TRY(sfde_reduce_partials(c, np, &r2));
        acc += r2;
    }
    *norm2 = acc;
    return SFDE_OK;
}

// X_b = S^{-1} R_b = V_y [ (V_y^T R_b V_x) / (1 + c dt sigma) ] V_x^T (c = 1/2 for SCHEME_SOLVE, 1 for
// SCHEME_SOLVE_BE): the four products of the spectral step with V in place of W on the input side and
// no load; intermediates in the workspace T1..T3 (batch <= ws_slices).
sfde_status sfde_fdm_solve_fp64(sfde_ctx* c, const double* R, long long r_stride, double* X, long long x_stride,
                                int batch, const double* dt, int n0, int dn, int scheme) {
    if (batch > (int)c->ws_slices || (scheme != SCHEME_SOLVE && scheme != SCHEME_SOLVE_BE)) return SFDE_EINVAL;
    const int Px = c->x.P, Py = c->y.P;
    const long long P2 = (long long)c->P2();
    const int pmin = Px < Py ? Px : Py;
    GemmParams p{};
    p.batch = batch; p.X = R; p.x_stride = r_stride; p.R = Py; p.C = Px;
    p.Mat = c->x.V; p.Cout = Px; p.Out = c->T1; p.out_stride = P2;
    launch_T<EPI_STORE>(c, choose_tile((long long)batch * Py, Px, pmin), p, c->y.n, c->x.n, c->x.n);
    GemmParams q{};
    q.batch = batch; q.X = c->T1; q.x_stride = P2; q.R = Px; q.C = Py;
    q.Mat = c->y.V; q.Cout = Py; q.Out = c->T2; q.out_stride = P2;
    q.lamx = c->x.lam; q.lamy = c->y.lam; q.kx = c->kx; q.ky = c->ky;
    q.dt = dt; q.n0 = n0; q.dn = dn; q.scheme = scheme;
    launch_T<EPI_MODAL>(c, choose_tile((long long)batch * Px, Py, pmin), q, c->x.n, c->y.n, c->y.n);
    GemmParams r{};
    r.batch = batch; r.X = c->T2; r.x_stride = P2; r.R = Py; r.C = Px;
    r.Mat = c->x.VT; r.Cout = Px; r.Out = c->T3; r.out_stride = P2;
    launch_T<EPI_STORE>(c, choose_tile((long long)batch * Py, Px, pmin), r, c->y.n, c->x.n, c->x.n);
    GemmParams f{};
    f.batch = batch; f.X = c->T3; f.x_stride = P2; f.R = Px; f.C = Py;
    f.Mat = c->y.VT; f.Cout = Py; f.Out = X; f.out_stride = x_stride;
    launch_T<EPI_FINAL>(c, choose_tile((long long)batch * Px, Py, pmin), f, c->x.n, c->y.n, c->y.n);
    SFDE_CUDA(cudaGetLastError());
    return SFDE_OK;
}

// Out_b = My^T X_b Mx for count padded slices (FP64, two slice products through the workspace T1);
// Out may not alias X.
sfde_status sfde_two_sided_fp64(sfde_ctx* c, const double* X, int count, const double* Mx, const double* My,
                                double* Out) {
    const int Px = c->x.P, Py = c->y.P;
    const long long P2 = (long long)c->P2();
    const int pmin = Px < Py ? Px : Py;
    for (int b0 = 0; b0 < count; b0 += (int)c->ws_slices) {
        const int nb = std::min(count - b0, (int)c->ws_slices);
        GemmParams p{};   // (X Mx)^T
        p.batch = nb; p.X = X + (size_t)b0 * P2; p.x_stride = P2; p.R = Py; p.C = Px;
        p.Mat = Mx; p.Cout = Px; p.Out = c->T1; p.out_stride = P2;
        launch_T<EPI_STORE>(c, choose_tile((long long)nb * Py, Px, pmin), p, c->y.n, c->x.n, c->x.n);
        GemmParams q{};   // ((X Mx)^T My)^T = My^T X Mx
        q.batch = nb; q.X = c->T1; q.x_stride = P2; q.R = Px; q.C = Py;
        q.Mat = My; q.Cout = Py; q.Out = Out + (size_t)b0 * P2; q.out_stride = P2;
        launch_T<EPI_STORE>(c, choose_tile((long long)nb * Px, Py, pmin), q, c->x.n, c->y.n, c->y.n);
    }
    SFDE_CUDA(cudaGetLastError());
    return SFDE_OK;
}
