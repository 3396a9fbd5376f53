// Two-level convergence analysis on the device (Sec. 3.3): the bound of Theorem 3.1, Eq. (3.11),
//   max over modes w of  (lam+_w)^m |(lam+_w)^m - mu++_w| (1 - (mu*_w)^{N_c - 1}) / (1 - mu*_w),
// lam+ = max over the fine steps of |lambda_w| (Eq. (3.7), Crank-Nicolson-type fine step), mu++ the
// smallest and mu* the largest magnitude of the coarse propagator's eigenvalue over the coarse steps,
// for the modes sigma_w = K_x lambda_x[i] + K_y lambda_y[j] of the generalised eigenproblems (3.5).
// |(2 - z)/(2 + z)|, (2 - z)/(2 + z) and 1/(1 + z) are monotone on either side of z = 2, so the
// extremes over the steps of a grid are reached at its smallest or largest step.
//
// One thread per mode, block maxima, the maximum of those on the host (exact: max is associative).
// The bound picks the coarse propagator under SFDE_COARSE_AUTO and, with mgrit_opts.m = 0, the
// coarsening factor (the analysis the paper uses to explain its choice of m, applied per problem).
#include <math.h>

#include <algorithm>
#include <vector>

#include "sfde_internal.cuh"

namespace {

constexpr int BOUND_BLOCKS = 152, BOUND_THREADS = 256;

__device__ __forceinline__ double fine_factor(double z) { return (2.0 - z) / (2.0 + z); }
__device__ __forceinline__ double coarse_factor(double z, int coarse) {
    return coarse == SFDE_COARSE_CN ? (2.0 - z) / (2.0 + z) : 1.0 / (1.0 + z);
}

__global__ void __launch_bounds__(BOUND_THREADS) k_tub_bound(const double* __restrict__ lamx,
                                                             const double* __restrict__ lamy, int nx, int ny, double kx,
                                                             double ky, double f_lo, double f_hi, double c_lo,
                                                             double c_hi, int m, int Nc, int coarse, double* bmax) {
    __shared__ double red[BOUND_THREADS];
    double best = 0.0;
    const long long total = (long long)nx * ny;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(w % nx), j = (int)(w / nx);
        const double s = kx * lamx[i] + ky * lamy[j];
        const double ld = fmax(fabs(fine_factor(f_lo * s)), fabs(fine_factor(f_hi * s)));
        const double mu1 = coarse_factor(c_lo * s, coarse), mu2 = coarse_factor(c_hi * s, coarse);
        const double mdd = fmin(mu1, mu2), mst = fmax(fabs(mu1), fabs(mu2));
        const double lm = pow(ld, (double)m);
        const double geo = mst < 1.0 ? (1.0 - pow(mst, (double)(Nc - 1))) / (1.0 - mst) : (double)(Nc - 1);
        best = fmax(best, lm * fabs(lm - mdd) * geo);
    }
    red[threadIdx.x] = best;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + k]);
        __syncthreads();
    }
    if (threadIdx.x == 0) bmax[blockIdx.x] = red[0];
}

}  // namespace

sfde_status sfde_tub_bound_device(sfde_ctx* c, int m, int coarse, double* out) {
    const int N = c->nt;
    if (m < 2 || N % m != 0 || N / m < 2) { *out = INFINITY; return SFDE_OK; }
    double f_lo = INFINITY, f_hi = 0, c_lo = INFINITY, c_hi = 0;
    for (int n = 1; n <= N; ++n) {
        const double d = c->t[n] - c->t[n - 1];
        f_lo = std::min(f_lo, d);
        f_hi = std::max(f_hi, d);
    }
    for (int k = 1; k <= N / m; ++k) {
        const double d = c->t[(size_t)k * m] - c->t[(size_t)(k - 1) * m];
        c_lo = std::min(c_lo, d);
        c_hi = std::max(c_hi, d);
    }
    if (!c->bound_partial) SFDE_CUDA(cudaMalloc(&c->bound_partial, sizeof(double) * BOUND_BLOCKS));
    k_tub_bound<<<BOUND_BLOCKS, BOUND_THREADS, 0, c->stream>>>(c->x.lam, c->y.lam, c->x.n, c->y.n, c->kx, c->ky, f_lo,
                                                             f_hi, c_lo, c_hi, m, N / m, coarse, c->bound_partial);
    sfde_count_launch(c);
    SFDE_CUDA(cudaGetLastError());
    double h[BOUND_BLOCKS];
    SFDE_CUDA(cudaMemcpyAsync(h, c->bound_partial, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    SFDE_CUDA(cudaStreamSynchronize(c->stream));
    double best = 0.0;
    for (double v : h) best = std::max(best, v);
    *out = best;
    return SFDE_OK;
}

// Coarse propagator for this solve: the requested one, or for AUTO the paper's CN rediscretisation
// when Theorem 3.1's bound (3.11) on the actual eigenvalues is below 1, backward Euler otherwise.
sfde_status sfde_choose_coarse(sfde_ctx* c, int m, int requested, int* coarse, double* tub) {
    SFDE_TRY(sfde_tub_bound_device(c, m, SFDE_COARSE_CN, tub));
    *coarse = requested;
    if (requested == SFDE_COARSE_AUTO) *coarse = (*tub < 1.0) ? SFDE_COARSE_CN : SFDE_COARSE_BE;
    return SFDE_OK;
}

// Coarsening factor for mgrit_opts.m = 0: among m in {2, 4, 8, 16, 32} that divide N_t with at least
// two coarse intervals, the one with the least estimated work to the tolerance -- the two-level bound
// b(m) of the coarse propagator in use taken as the contraction per iteration, so about
// ceil(log(rel_tol) / log b(m)) iterations, each of about 2 m / (m - 1) step solves per time point
// (FCF relaxation, C-point residual, F-relaxation on the coarse level).  Candidates with b(m) >= 1
// are left out; if all are, the largest valid m.  Ties go to the larger m (shorter coarse levels).
sfde_status sfde_choose_m(sfde_ctx* c, int requested_coarse, double rel_tol, int* m_out) {
    const double tol = rel_tol > 0.0 && rel_tol < 1.0 ? rel_tol : 1e-10;
    int best_m = 0, last_valid = 0;
    double best_cost = INFINITY;
    for (int m : {2, 4, 8, 16, 32}) {
        if (c->nt % m != 0 || c->nt / m < 2) continue;
        last_valid = m;
        int coarse = SFDE_COARSE_BE;
        double tub = 0.0, b = 0.0;
        SFDE_TRY(sfde_choose_coarse(c, m, requested_coarse, &coarse, &tub));
        if (coarse == SFDE_COARSE_CN) b = tub;
        else SFDE_TRY(sfde_tub_bound_device(c, m, SFDE_COARSE_BE, &b));
        if (!(b < 1.0)) continue;
        const double iters = b > 0.0 ? std::max(1.0, ceil(log(tol) / log(b))) : 1.0;
        const double cost = iters * 2.0 * m / (m - 1.0);
        if (cost <= best_cost) { best_cost = cost; best_m = m; }
    }
    *m_out = best_m ? best_m : (last_valid ? last_valid : 2);
    return SFDE_OK;
}

extern "C" sfde_status sfde_two_level_bound(sfde_ctx* c, int m, int coarse, double* bound) {
    if (!c || !bound || m < 2 || (coarse != SFDE_COARSE_CN && coarse != SFDE_COARSE_BE)) return SFDE_EINVAL;
    if (c->nt % m != 0 || c->nt / m < 2) return SFDE_EINVAL;
    return sfde_no_throw([&] { return sfde_tub_bound_device(c, m, coarse, bound); });
}

extern "C" sfde_status sfde_choose_coarsening(sfde_ctx* c, int coarse, double rel_tol, int* m) {
    if (!c || !m || coarse < SFDE_COARSE_CN || coarse > SFDE_COARSE_AUTO) return SFDE_EINVAL;
    return sfde_no_throw([&] { return sfde_choose_m(c, coarse, rel_tol, m); });
}
