// MGRIT V-cycle (Algorithm 1) and sequential stepping on the device, FP64 form.
//
// Level l stores its iterate u_l as N_l+1 padded slices (time slowest).  A relaxation sweep is
// one batched step over all coarse intervals at once: F-relaxation runs m-1 batched steps
// (interval k advances from k*m+j-1 to k*m+j for all k together), C-relaxation one.  The
// C-point residual r_k = Phi_{km}(u_{km-1}) - u_{km} is one more batched step whose epilogue
// subtracts u_{km}, writes r_k straight into the next level's right-hand side (injection) and
// accumulates ||r||^2 per CTA for a fixed-order reduction.
#include <math.h>
#include <algorithm>

#include "sfde_internal.cuh"

namespace {

__global__ void k_diff_slice(double* out, const double* a, const double* b, size_t n) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        out[e] = a[e] - b[e];
}

void free_levels(sfde_ctx* c) {
    for (size_t l = 0; l < c->levels.size(); ++l) {
        SfdeLevel& L = c->levels[l];
        if (l > 0) cudaFree(L.dt);
        cudaFree(L.u);
        cudaFree(L.g);
    }
    c->levels.clear();
}

sfde_status build_levels(sfde_ctx* c, int m, int max_levels, int min_coarse) {
    if (!c->levels.empty() && c->lev_m == m && c->lev_max == max_levels && c->lev_min == min_coarse)
        return SFDE_OK;
    free_levels(c);
    c->lev_m = 0;   // set again only once every level is in place: a failed build is never reused
    const size_t P2 = c->P2();
    SfdeLevel L0;
    L0.N = c->nt;
    L0.t = c->t;
    L0.dt = c->dt0;
    c->levels.push_back(L0);
    SFDE_CUDA(cudaMalloc(&c->levels[0].u, sizeof(double) * P2 * (c->nt + 1)));
    while ((int)c->levels.size() < max_levels) {
        const SfdeLevel& F = c->levels.back();
        if (F.N % m != 0 || F.N / m < min_coarse) break;
        SfdeLevel G;
        G.N = F.N / m;
        G.t.resize(G.N + 1);
        for (int k = 0; k <= G.N; ++k) G.t[k] = F.t[(size_t)k * m];
        std::vector<double> dt(G.N);
        for (int k = 0; k < G.N; ++k) dt[k] = G.t[k + 1] - G.t[k];
        c->levels.push_back(G);
        SfdeLevel& Gr = c->levels.back();
        SFDE_CUDA(cudaMalloc(&Gr.dt, sizeof(double) * G.N));
        SFDE_CUDA(cudaMemcpy(Gr.dt, dt.data(), sizeof(double) * G.N, cudaMemcpyHostToDevice));
        SFDE_CUDA(cudaMalloc(&Gr.u, sizeof(double) * P2 * (G.N + 1)));
        SFDE_CUDA(cudaMalloc(&Gr.g, sizeof(double) * P2 * (G.N + 1)));
    }
    c->lev_m = m; c->lev_max = max_levels; c->lev_min = min_coarse;
    return SFDE_OK;
}

struct Engine {
    sfde_ctx* c;
    int m, L, relax, scheme;
    long long steps = 0;
    bool skip = false;   // down-cycle without relaxation (the first iteration with skip_first_down)
    bool warm = false;   // every level's iterate holds valid values: steps may start from them

    size_t P2() const { return c->P2(); }

    sfde_status step(int l, int batch, int src0, int dst0, int stride, int n0, int dn,
                     double* dst_base, long long dst_stride, const double* utgt, double* partial,
                     int* npart) {
        SfdeLevel& Lv = c->levels[l];
        const long long s = (long long)stride * (long long)P2();
        StepBatch sb{};
        sb.batch = batch;
        sb.src = Lv.u + (size_t)src0 * P2(); sb.src_stride = s;
        sb.dst = dst_base ? dst_base : Lv.u + (size_t)dst0 * P2();
        sb.dst_stride = dst_base ? dst_stride : s;
        sb.g = (l > 0) ? Lv.g + (size_t)n0 * P2() : nullptr; sb.g_stride = (long long)dn * P2();
        sb.utgt = utgt; sb.utgt_stride = (long long)dn * P2();
        sb.dt = Lv.dt; sb.n0 = n0; sb.dn = dn;
        sb.scheme = (l == 0) ? SCHEME_CN : scheme;
        sb.level0 = (l == 0);
        sb.norm_partial = partial;
        if (warm) {
            // the value being replaced (relaxation) or the target value (residual): Phi(u) + g is
            // close to it once the iteration converges
            sb.guess = utgt ? utgt : sb.dst;
            sb.guess_stride = utgt ? sb.utgt_stride : sb.dst_stride;
        }
        steps += batch;
        return sfde_step_any(c, sb, npart);
    }

    sfde_status frelax(int l) {
        const int N = c->levels[l].N, nc = N / m;
        for (int j = 1; j < m; ++j)
            SFDE_TRY(step(l, nc, j - 1, j, m, j, m, nullptr, 0, nullptr, nullptr, nullptr));
        return SFDE_OK;
    }

    sfde_status crelax(int l) {
        const int N = c->levels[l].N, nc = N / m;
        return step(l, nc, m - 1, m, m, m, m, nullptr, 0, nullptr, nullptr, nullptr);
    }

    sfde_status relaxation(int l) {
        SFDE_TRY(frelax(l));
        if (relax == SFDE_RELAX_FCF) {
            SFDE_TRY(crelax(l));
            SFDE_TRY(frelax(l));
        }
        return SFDE_OK;
    }

    // r_k into levels[l+1].g[k]; returns the number of partial sums when asked for the norm.
    sfde_status residual(int l, bool want_norm, int* npart) {
        SfdeLevel& Lv = c->levels[l];
        SfdeLevel& Cv = c->levels[l + 1];
        const int nc = Lv.N / m;
        if (l == 0) {
            SFDE_CUDA(cudaMemsetAsync(Cv.g, 0, sizeof(double) * P2(), c->stream));
        } else {
            k_diff_slice<<<64, 256, 0, c->stream>>>(Cv.g, Lv.g, Lv.u, P2());
            sfde_count_launch(c);
        }
        return step(l, nc, m - 1, 0, m, m, m, Cv.g + P2(), (long long)P2(), Lv.u + (size_t)m * P2(),
                    want_norm ? c->partial : nullptr, npart);
    }

    sfde_status coarsest(int l) {
        SfdeLevel& Lv = c->levels[l];
        if (l > 0)
            SFDE_CUDA(cudaMemcpyAsync(Lv.u, Lv.g, sizeof(double) * P2(), cudaMemcpyDeviceToDevice, c->stream));
        for (int n = 1; n <= Lv.N; ++n)
            SFDE_TRY(step(l, 1, n - 1, n, 1, n, 1, nullptr, 0, nullptr, nullptr, nullptr));
        return SFDE_OK;
    }

    sfde_status correct(int l) {
        SfdeLevel& Lv = c->levels[l];
        SfdeLevel& Cv = c->levels[l + 1];
        sfde_launch_axpy_strided(Lv.u, (long long)m * P2(), Cv.u, (long long)P2(), Cv.N + 1, P2(), c->stream);
        sfde_count_launch(c);
        SFDE_CUDA(cudaGetLastError());
        return SFDE_OK;
    }

    sfde_status solve(int l) {
        if (l == L - 1) return coarsest(l);
        if (!skip) SFDE_TRY(relaxation(l));
        SFDE_TRY(residual(l, false, nullptr));
        SFDE_CUDA(cudaMemsetAsync(c->levels[l + 1].u, 0, sizeof(double) * P2() * (c->levels[l + 1].N + 1), c->stream));
        SFDE_TRY(solve(l + 1));
        SFDE_TRY(correct(l));
        return frelax(l);
    }
};

// Theorem 3.1 / Eq. (3.11) for the fine grid and its m-coarsening, over all modes sigma.
// |(2 - z)/(2 + z)| and (2 - z)/(2 + z) are monotone on either side of z = 2, so the
// extremes over the steps of a grid are reached at its smallest or largest step.
double tub_bound_host(const std::vector<double>& lx, const std::vector<double>& ly, int nx, int ny,
                      double kx, double ky, const std::vector<double>& t, int m, int coarse) {
    const int N = (int)t.size() - 1;
    if (N % m != 0 || N / m < 2) return INFINITY;
    double fmin = INFINITY, fmax = 0, cmin = INFINITY, cmax = 0;
    for (int n = 1; n <= N; ++n) { double d = t[n] - t[n - 1]; fmin = std::min(fmin, d); fmax = std::max(fmax, d); }
    for (int k = 1; k <= N / m; ++k) { double d = t[(size_t)k * m] - t[(size_t)(k - 1) * m]; cmin = std::min(cmin, d); cmax = std::max(cmax, d); }
    const int Nc = N / m;
    auto R = [coarse](double z, bool fine) {
        if (fine || coarse == SFDE_COARSE_CN) return (2.0 - z) / (2.0 + z);
        return 1.0 / (1.0 + z);
    };
    double best = 0.0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double s = kx * lx[i] + ky * ly[j];
            double ld = std::max(fabs(R(fmin * s, true)), fabs(R(fmax * s, true)));
            double mu1 = R(cmin * s, false), mu2 = R(cmax * s, false);
            double mdd = std::min(mu1, mu2), mst = std::max(fabs(mu1), fabs(mu2));
            double lm = pow(ld, m);
            double geo = mst < 1.0 ? (1.0 - pow(mst, Nc - 1)) / (1.0 - mst) : (double)(Nc - 1);
            best = std::max(best, lm * fabs(lm - mdd) * geo);
        }
    return best;
}

}  // namespace

sfde_status sfde_ensure_workspace(sfde_ctx* c, size_t slices) {
    if (slices < 1) slices = 1;
    const size_t P2 = c->P2();
    if (c->ws_slices < slices) {
        cudaFree(c->T1); cudaFree(c->T2); cudaFree(c->T3);
        c->T1 = c->T2 = c->T3 = nullptr;
        c->ws_slices = 0;
        SFDE_CUDA(cudaMalloc(&c->T1, sizeof(double) * P2 * slices));
        SFDE_CUDA(cudaMalloc(&c->T2, sizeof(double) * P2 * slices));
        SFDE_CUDA(cudaMalloc(&c->T3, sizeof(double) * P2 * slices));
        c->ws_slices = slices;
    }
    // residual CTAs: at most (slices * Px / 16) * (Py / 16)
    size_t need = slices * (size_t)c->x.P / 16 * (size_t)c->y.P / 16 + 64;
    if (c->partial_cap < need) {
        cudaFree(c->partial);
        c->partial = nullptr;
        SFDE_CUDA(cudaMalloc(&c->partial, sizeof(double) * need));
        c->partial_cap = need;
    }
    return SFDE_OK;
}

void sfde_free_levels(sfde_ctx* c) { free_levels(c); }

// The FP64 level-0 buffer ((N_t+1) padded slices), built on demand; shared by every solver form.
sfde_status sfde_level0(sfde_ctx* c, double** u) {
    if (c->levels.empty()) SFDE_TRY(build_levels(c, 2, 1, 1));
    *u = c->levels[0].u;
    return SFDE_OK;
}

extern "C" sfde_status sfde_debug_tub_bound(const double* lx, int nx, const double* ly, int ny, double kx, double ky,
                                           const double* t, int nt, int m, int coarse, double* out) {
    if (!lx || !ly || !t || !out || nx < 1 || ny < 1 || nt < 1 || m < 2 ||
        (coarse != SFDE_COARSE_CN && coarse != SFDE_COARSE_BE))
        return SFDE_EINVAL;
    return sfde_no_throw([&] {
        *out = tub_bound_host(std::vector<double>(lx, lx + nx), std::vector<double>(ly, ly + ny), nx, ny, kx, ky,
                              std::vector<double>(t, t + nt + 1), m, coarse);
        return SFDE_OK;
    });
}

sfde_status sfde_mgrit_fp64(sfde_ctx* c, const mgrit_opts* o, mgrit_stats* st) {
    SFDE_TRY(build_levels(c, o->m, o->max_levels, o->min_coarse));
    const int L = (int)c->levels.size();
    SFDE_TRY(sfde_ensure_workspace(c, std::max(1, c->nt / o->m)));
    Engine E{c, o->m, L, o->relax, SCHEME_CN};
    E.warm = true;   // level 0 is initialised below, coarse levels are zeroed before each cycle

    int coarse = SFDE_COARSE_BE;
    double tub = 0.0;
    SFDE_TRY(sfde_choose_coarse(c, o->m, o->coarse, &coarse, &tub));
    E.scheme = (coarse == SFDE_COARSE_CN) ? SCHEME_CN : SCHEME_BE;

    const size_t P2 = c->P2();
    SfdeLevel& L0 = c->levels[0];
    SFDE_CUDA(cudaEventRecord(c->ev0, c->stream));
    // initial guess: u_0 = psi_0, zero or SplitMix64 values elsewhere
    SFDE_CUDA(cudaMemcpyAsync(L0.u, c->U0, sizeof(double) * P2, cudaMemcpyDeviceToDevice, c->stream));
    if (o->init_seed) {
        sfde_launch_fill_random(L0.u, c->nt, c->y.n, c->x.n, c->y.P, c->x.P, o->init_seed, c->stream);
        sfde_count_launch(c);
    }
    else
        SFDE_CUDA(cudaMemsetAsync(L0.u + P2, 0, sizeof(double) * P2 * c->nt, c->stream));

    mgrit_stats S{};
    S.levels = L;
    S.coarse_used = coarse;
    S.tub = tub;
    S.lp_kind = -1;
    sfde_status rc = SFDE_OK;
    if (L == 1) {
        rc = E.coarsest(0);
        S.iters = 1;
        S.converged = 1;
    } else {
        // space-time (S-form) stopping test: relative to the residual of the initial guess
        double sref = 0.0;
        if (o->stop_kind == 1) {
            double r2 = 0.0;
            SFDE_TRY(sfde_residual_norm2_fp64(c, L0.u, &r2));
            sref = sqrt(r2);
        }
        const int nc = c->nt / o->m;
        for (int it = 1; it <= o->max_iter; ++it) {
            const bool skip = o->skip_first_down && it == 1;
            if (!skip) SFDE_TRY(E.relaxation(0));
            int np = 0;
            SFDE_TRY(E.residual(0, true, &np));
            double r2 = 0.0;
            SFDE_TRY(sfde_reduce_partials(c, np, &r2));
            if (o->stop_kind == 1) {
                // after a relaxation every F-point's row of Eq. (3.1) holds, so rho vanishes there
                // and rho_{km} = S_{km} r_k at the C-points (r_k was just injected into level 1)
                if (skip) SFDE_TRY(sfde_residual_norm2_fp64(c, L0.u, &r2));
                else SFDE_TRY(sfde_apply_S_norm2(c, c->levels[1].g + P2, (long long)P2, nc, o->m, o->m, &r2));
            }
            const double nrm = sqrt(r2);
            if (it - 1 < SFDE_HISTORY_MAX) S.history[it - 1] = nrm;
            // the reference: the initial guess's space-time residual, or the first C-point norm
            // computed after a relaxation (a skipped iteration's residual is the unrelaxed guess's)
            if (o->stop_kind == 1) S.res0 = sref;
            else if (it == (o->skip_first_down ? 2 : 1)) S.res0 = nrm;
            S.res_final = nrm;
            S.iters = it;
            if (!isfinite(nrm)) { rc = SFDE_ENOCONV; break; }
            if (!skip && nrm <= std::max(o->rel_tol * S.res0, o->abs_tol)) { S.converged = 1; break; }
            SFDE_CUDA(cudaMemsetAsync(c->levels[1].u, 0, sizeof(double) * P2 * (c->levels[1].N + 1), c->stream));
            E.skip = skip;
            SFDE_TRY(E.solve(1));
            E.skip = false;
            SFDE_TRY(E.correct(0));
        }
        if (!S.converged && rc == SFDE_OK) rc = SFDE_ENOCONV;
    }
    SFDE_CUDA(cudaEventRecord(c->ev1, c->stream));
    SFDE_CUDA(cudaEventSynchronize(c->ev1));
    float ms = 0.f;
    SFDE_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    S.seconds = ms * 1e-3;
    S.step_solves = E.steps;
    int nh = std::min(S.iters, SFDE_HISTORY_MAX);
    if (nh >= 2) {
        int k0 = std::max(1, nh - 5);
        double acc = 0; int cnt = 0;
        for (int k = k0; k < nh; ++k) if (S.history[k - 1] > 0) { acc += S.history[k] / S.history[k - 1]; ++cnt; }
        S.conv_factor_last5 = cnt ? acc / cnt : NAN;
    } else {
        S.conv_factor_last5 = NAN;
    }
    if (st) *st = S;
    return rc;
}

sfde_status sfde_seq_fp64(sfde_ctx* c, double* seconds) {
    SFDE_TRY(build_levels(c, c->lev_m ? c->lev_m : 2, c->lev_m ? c->lev_max : 1, c->lev_m ? c->lev_min : 1));
    SFDE_TRY(sfde_ensure_workspace(c, 1));
    Engine E{c, 2, 1, SFDE_RELAX_FCF, SCHEME_CN};
    SfdeLevel& L0 = c->levels[0];
    SFDE_CUDA(cudaEventRecord(c->ev0, c->stream));
    SFDE_CUDA(cudaMemcpyAsync(L0.u, c->U0, sizeof(double) * c->P2(), cudaMemcpyDeviceToDevice, c->stream));
    SFDE_TRY(E.coarsest(0));
    SFDE_CUDA(cudaEventRecord(c->ev1, c->stream));
    SFDE_CUDA(cudaEventSynchronize(c->ev1));
    float ms = 0.f;
    SFDE_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    if (seconds) *seconds = ms * 1e-3;
    return SFDE_OK;
}
