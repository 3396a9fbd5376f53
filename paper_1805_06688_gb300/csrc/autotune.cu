// Autotuner of the mixed-precision solver's execution choices (host code).
//
// The choices -- the fused step's CTA-pair form, where F-relaxations run in the step's eigenbasis,
// the V-cycles per refinement step -- change the time of a solve but not the system it solves, so
// they are picked by measurement: each candidate is applied and timed over full solves of the
// context's own problem (the solver's device-time clock), and the fastest that converges is kept.
// Tensor-core tile shapes follow from the padded size P and are not tuned.  Choices are cached per
// problem key in a plain text file, one line per measurement, the last line for a key counting.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "sfde_internal.cuh"

namespace {

bool tuning_valid(const sfde_tuning& t) {
    return t.fused_pair >= 0 && t.fused_pair <= 3 && t.modal_chains >= 0 && t.modal_chains <= 4 &&
           t.inner_cycles >= 0 && t.inner_cycles <= 64;
}

// index of the smallest positive finite time, the first on ties; -1 if none was measured
int tune_pick(const sfde_tuning* c, int n) {
    int best = -1;
    for (int i = 0; i < n; ++i)
        if (c[i].ms > 0.0 && isfinite(c[i].ms) && (best < 0 || c[i].ms < c[best].ms)) best = i;
    return best;
}

bool key_valid(const char* key) {
    if (!key) return false;
    const size_t n = strlen(key);
    if (n < 1 || n > 255) return false;
    for (size_t i = 0; i < n; ++i)
        if (key[i] == ' ' || key[i] == '\t' || key[i] == '\n' || key[i] == '\r') return false;
    return true;
}

bool cache_read(const char* path, const char* key, sfde_tuning* out) {
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (fgets(line, sizeof line, f)) {
        char k[256];
        sfde_tuning t{};
        if (sscanf(line, "%255s %d %d %d %lf", k, &t.fused_pair, &t.modal_chains, &t.inner_cycles, &t.ms) == 5 &&
            strcmp(k, key) == 0 && tuning_valid(t)) {
            *out = t;
            found = true;
        }
    }
    fclose(f);
    return found;
}

bool cache_append(const char* path, const char* key, const sfde_tuning& t) {
    FILE* f = fopen(path, "a");
    if (!f) return false;
    const int w = fprintf(f, "%s %d %d %d %.6g\n", key, t.fused_pair, t.modal_chains, t.inner_cycles, t.ms);
    return fclose(f) == 0 && w > 0;
}

// what decides the best choice: padded sizes, the operator (fractional orders, diffusivities: they set
// the spectra and so the contraction of the refinement), the time grid (N_t, T, spread of the steps
// and a hash of every time point), precision, and the options that shape the V-cycle and its
// stopping point
std::string tune_key(const sfde_ctx* c, const mgrit_opts& o) {
    double dmin = INFINITY, dmax = 0.0;
    uint64_t h = 1469598103934665603ull;   // FNV-1a over the bytes of t_0..t_N
    for (int n = 0; n <= c->nt; ++n) {
        if (n > 0) {
            const double d = c->t[n] - c->t[n - 1];
            dmin = std::min(dmin, d);
            dmax = std::max(dmax, d);
        }
        unsigned char bytes[sizeof(double)];
        memcpy(bytes, &c->t[n], sizeof(double));
        for (unsigned char by : bytes) { h ^= by; h *= 1099511628211ull; }
    }
    char b[256];
    snprintf(b, sizeof b,
             "P%dx%d_nt%d_T%.6g_dr%.3g_th%016llx_b%.6g_g%.6g_kx%.6g_ky%.6g_p%d_m%d_L%d_c%d_r%d_co%d_tol%.2g_ic%d_sk%d_st%d",
             c->x.P, c->y.P, c->nt, c->t[c->nt], dmax / dmin, (unsigned long long)h, c->x.rho, c->y.rho, c->kx, c->ky,
             c->precision, o.m, o.max_levels, o.min_coarse, o.relax, o.coarse, o.rel_tol, o.inner_cycles,
             o.skip_first_down, o.stop_kind);
    return b;
}

sfde_tuning current(const sfde_ctx* c) {
    sfde_tuning t{};
    t.fused_pair = c->fused_pair;
    t.modal_chains = c->modal_chains;
    t.inner_cycles = c->inner_cycles_tuned;
    return t;
}

void apply(sfde_ctx* c, const sfde_tuning& t) {
    c->fused_pair = t.fused_pair;
    c->modal_chains = t.modal_chains;
    c->inner_cycles_tuned = t.inner_cycles;
}

sfde_status autotune_impl(sfde_ctx* c, const mgrit_opts* opts, const char* cache_path, sfde_tuning* out) {
    if (!c || !opts) return SFDE_EINVAL;
    if (c->precision == SFDE_PREC_FP64) {
        if (out) *out = current(c);
        return SFDE_OK;
    }
    const std::string key = tune_key(c, *opts);
    sfde_tuning t{};
    if (cache_path && cache_read(cache_path, key.c_str(), &t)) {
        apply(c, t);
        if (out) *out = t;
        return SFDE_OK;
    }
    // F-relaxations of the fine level as chained steps or in the eigenbasis (the coarse levels' are
    // always in the eigenbasis), times the default V-cycles per refinement step, 3 or 5 (not when the
    // options fix it); the whole inner solve in the eigenbasis with 3, 5, 8 or the default V-cycles;
    // the CTA-pair forms of the fused step forced either way where that step applies
    std::vector<sfde_tuning> cand;
    for (int mc : {1, 2})
        for (int ic : {0, 3, 5})
            if (ic == 0 || opts->inner_cycles == 0) cand.push_back({1, mc, ic, 0.0});
    // the whole inner solve in the eigenbasis (FP32 or TF32 storage): its V-cycles are elementwise, so more
    // of them per refinement step are worth a trial
    if (sfde_mixed_kind(c) != 0)
        for (int ic : {0, 3, 5, 8})
            if (ic == 0 || opts->inner_cycles == 0) cand.push_back({1, 4, ic, 0.0});
    if (sfde_mixed_kind(c) == 0 && sfde_fused_supported(0, c->x.P, c->y.P) && c->x.P == c->y.P &&
        sfde_fused_pair_supported(c->x.P)) {
        cand.push_back({2, 1, 0, 0.0});
        cand.push_back({3, 1, 0, 0.0});
    }
    const int n = (int)cand.size();
    const sfde_tuning before = current(c);
    sfde_status last = SFDE_OK;
    for (int i = 0; i < n; ++i) {
        apply(c, cand[i]);
        double best = INFINITY;
        bool ok = true;
        for (int r = 0; r < 3 && ok; ++r) {   // one untimed solve (setup, graph capture), two timed
            mgrit_stats st{};
            last = mgrit_solve(c, opts, nullptr, nullptr, &st);
            ok = last == SFDE_OK && st.converged;
            if (ok && r > 0) best = std::min(best, 1e3 * st.seconds);
        }
        if (last != SFDE_OK && last != SFDE_ENOCONV) {   // a CUDA or resource error ends the search
            apply(c, before);
            return last;
        }
        cand[i].ms = ok ? best : 0.0;
    }
    const int b = tune_pick(cand.data(), n);
    if (b < 0) {
        apply(c, before);
        return last == SFDE_OK ? SFDE_ENOCONV : last;
    }
    apply(c, cand[b]);
    if (cache_path) cache_append(cache_path, key.c_str(), cand[b]);
    if (out) *out = cand[b];
    return SFDE_OK;
}

}  // namespace

extern "C" sfde_status sfde_set_tuning(sfde_ctx* c, const sfde_tuning* t) {
    if (!c || !t || !tuning_valid(*t)) return SFDE_EINVAL;
    apply(c, *t);
    return SFDE_OK;
}

extern "C" sfde_status sfde_get_tuning(const sfde_ctx* c, sfde_tuning* out) {
    if (!c || !out) return SFDE_EINVAL;
    *out = current(c);
    return SFDE_OK;
}

extern "C" sfde_status sfde_autotune(sfde_ctx* c, const mgrit_opts* opts, const char* cache_path, sfde_tuning* out) {
    return sfde_no_throw([&] { return autotune_impl(c, opts, cache_path, out); });
}

extern "C" sfde_status sfde_debug_tune_pick(const sfde_tuning* c, int n, int* best) {
    if (n < 0 || !best || (n > 0 && !c)) return SFDE_EINVAL;
    *best = tune_pick(c, n);
    return SFDE_OK;
}

extern "C" sfde_status sfde_debug_tune_cache(const char* path, const char* key, int store, sfde_tuning* t, int* found) {
    if (!path || !key_valid(key) || !t) return SFDE_EINVAL;
    if (store) {
        if (!tuning_valid(*t)) return SFDE_EINVAL;
        return cache_append(path, key, *t) ? SFDE_OK : SFDE_EINVAL;
    }
    if (!found) return SFDE_EINVAL;
    return sfde_no_throw([&] {
        *found = cache_read(path, key, t) ? 1 : 0;
        return SFDE_OK;
    });
}
