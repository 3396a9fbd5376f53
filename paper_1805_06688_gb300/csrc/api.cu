// C ABI entry points (include/sfde.h): argument checks, host/device marshalling, dispatch.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "sfde_internal.cuh"

sfde_status sfde_mgrit_mixed(sfde_ctx* c, const mgrit_opts* o, mgrit_stats* st);  // mixed.cu
void sfde_free_levels(sfde_ctx* c);                                                // mgrit.cu
void sfde_free_mixed(sfde_ctx* c);                                                 // mixed.cu

static thread_local char g_last_error[512];

void sfde_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s:%d)", cudaGetErrorString(e), what, file, line);
}

bool sfde_is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

sfde_status sfde_copy_in(void* dst_dev, const void* src, size_t bytes, cudaStream_t s) {
    SFDE_CUDA(cudaMemcpyAsync(dst_dev, src, bytes,
                              sfde_is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    return SFDE_OK;
}

sfde_status sfde_copy_out(void* dst, const void* src_dev, size_t bytes, cudaStream_t s) {
    SFDE_CUDA(cudaMemcpyAsync(dst, src_dev, bytes,
                              sfde_is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    return SFDE_OK;
}

static void prof_flush_one(sfde_ctx* c, int slot) {
    SfdeProf& P = c->prof;
    cudaEventSynchronize(P.ev[2 * slot + 1]);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, P.ev[2 * slot], P.ev[2 * slot + 1]) != cudaSuccess) ms = 0.f;
    const int k = P.cls[slot];
    if (k >= 0 && k < SfdeProf::NCLS) {
        P.ms[k] += ms;
        P.tot_flops[k] += P.flops[slot];
        P.tot_bytes[k] += P.bytes[slot];
        P.n[k] += 1;
    }
}

int sfde_prof_begin(sfde_ctx* c) {
    SfdeProf& P = c->prof;
    if (!P.on) return -1;
    if (!P.ev[0])
        for (int i = 0; i < 2 * SfdeProf::CAP; ++i) cudaEventCreate(&P.ev[i]);
    int slot = P.head;
    if (P.count == SfdeProf::CAP) {  // reuse the oldest slot: it finished long ago
        prof_flush_one(c, slot);
        P.count--;
    }
    cudaEventRecord(P.ev[2 * slot], c->stream);
    return slot;
}

void sfde_prof_end(sfde_ctx* c, int slot, int cls, double flops, double bytes) {
    if (slot < 0) return;
    SfdeProf& P = c->prof;
    cudaEventRecord(P.ev[2 * slot + 1], c->stream);
    P.cls[slot] = cls;
    P.flops[slot] = flops;
    P.bytes[slot] = bytes;
    P.head = (P.head + 1) % SfdeProf::CAP;
    P.count++;
}

static void prof_flush_all(sfde_ctx* c) {
    SfdeProf& P = c->prof;
    int start = (P.head - P.count + SfdeProf::CAP) % SfdeProf::CAP;
    for (int k = 0; k < P.count; ++k) prof_flush_one(c, (start + k) % SfdeProf::CAP);
    P.count = 0;
}

static void free_ctx(sfde_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    sfde_free_levels(c);
    sfde_free_mixed(c);
    sfde_p1_free(c);
    sfde_free_direction(c->x);
    sfde_free_direction(c->y);
    cudaFree(c->dt0); cudaFree(c->U0); cudaFree(c->time_w); cudaFree(c->px); cudaFree(c->py);
    cudaFree(c->bxn); cudaFree(c->byn); cudaFree(c->Fd); cudaFree(c->Fh);
    cudaFree(c->T1); cudaFree(c->T2); cudaFree(c->T3); cudaFree(c->partial); cudaFree(c->scalar);
    cudaFree(c->bound_partial);
    if (c->host_scalar) cudaFreeHost(c->host_scalar);
    if (c->prof.ev[0])
        for (int i = 0; i < 2 * SfdeProf::CAP; ++i) cudaEventDestroy(c->prof.ev[i]);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    delete c;
}

extern "C" {

const char* sfde_strerror(sfde_status s) {
    switch (s) {
        case SFDE_OK: return "ok";
        case SFDE_EINVAL: return "invalid argument";
        case SFDE_ENOMEM: return "out of memory";
        case SFDE_ECUDA: return g_last_error[0] ? g_last_error : "CUDA error";
        case SFDE_ENOCONV: return "no convergence";
        case SFDE_ETIMEOUT: return "device wait timed out";
        case SFDE_EUNSUPPORTED: return "unsupported option";
        case SFDE_ESCRATCH: return "request exceeds the fixed scratch of sfde_step_batch_noalloc";
    }
    return "unknown status";
}

static sfde_status setup_impl(double beta, double gamma, double kx, double ky, const double omega[4],
                              int nx, int ny, const double* t, int nt, const sfde_opts* opts,
                              sfde_ctx** out) {
    if (!out) return SFDE_EINVAL;
    *out = nullptr;
    if (!(beta > 0.5 && beta <= 1.0) || !(gamma > 0.5 && gamma <= 1.0)) return SFDE_EINVAL;
    if (!(kx > 0.0) || !(ky > 0.0) || !isfinite(kx) || !isfinite(ky)) return SFDE_EINVAL;
    if (nx < 1 || ny < 1 || nx > 4096 || ny > 4096 || nt < 1 || !t) return SFDE_EINVAL;
    double om[4] = {0.0, 1.0, 0.0, 1.0};
    if (omega) memcpy(om, omega, sizeof(om));
    if (!(om[1] > om[0]) || !(om[3] > om[2])) return SFDE_EINVAL;
    if (t[0] != 0.0) return SFDE_EINVAL;
    for (int n = 1; n <= nt; ++n)
        if (!(t[n] > t[n - 1]) || !isfinite(t[n])) return SFDE_EINVAL;
    int prec = opts ? opts->precision : SFDE_PREC_FP64;
    if (prec < SFDE_PREC_FP64 || prec > SFDE_PREC_MIXED_AUTO) return SFDE_EINVAL;
    const int op = opts ? opts->operator_kind : SFDE_OP_TENSOR;
    if (op != SFDE_OP_TENSOR && op != SFDE_OP_P1) return SFDE_EINVAL;
    if (op == SFDE_OP_P1 && prec != SFDE_PREC_FP64) return SFDE_EUNSUPPORTED;

    sfde_ctx* c = new (std::nothrow) sfde_ctx();
    if (!c) return SFDE_ENOMEM;
    c->kx = kx; c->ky = ky; c->nt = nt;
    memcpy(c->omega, om, sizeof(om));
    c->precision = prec;
    c->op_kind = op;
    c->stream = opts ? (cudaStream_t)opts->stream : nullptr;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return SFDE_ECUDA;
    }
    sfde_status st = SFDE_OK;
    try {   // a host allocation that throws frees the partial context before the status is returned
        c->t.assign(t, t + nt + 1);
        do {
            if ((st = sfde_setup_direction(c->x, nx, beta, om[1] - om[0], c->stream)) != SFDE_OK) break;
            if ((st = sfde_setup_direction(c->y, ny, gamma, om[3] - om[2], c->stream)) != SFDE_OK) break;
            if (op == SFDE_OP_P1 && (st = sfde_p1_setup(c)) != SFDE_OK) break;
            // FP32 storage: the inner solve held in the step's eigenbasis by default
            if (prec != SFDE_PREC_FP64 && sfde_mixed_kind(c) != 0) c->modal_chains = 4;
            std::vector<double> dt(nt);
            for (int n = 0; n < nt; ++n) dt[n] = t[n + 1] - t[n];
            cudaError_t e;
#define SC(x) if ((e = (x)) != cudaSuccess) { sfde_set_last_cuda_error(e, #x, __FILE__, __LINE__); st = (e == cudaErrorMemoryAllocation) ? SFDE_ENOMEM : SFDE_ECUDA; break; }
            SC(cudaMalloc(&c->dt0, sizeof(double) * nt));
            SC(cudaMemcpy(c->dt0, dt.data(), sizeof(double) * nt, cudaMemcpyHostToDevice));
            SC(cudaMalloc(&c->U0, sizeof(double) * c->P2()));
            SC(cudaMemsetAsync(c->U0, 0, sizeof(double) * c->P2(), c->stream));
            SC(cudaMalloc(&c->scalar, sizeof(double) * 4));
            SC(cudaMallocHost(&c->host_scalar, sizeof(double) * 4));
            SC(cudaEventCreate(&c->ev0));
            SC(cudaEventCreate(&c->ev1));
            SC(cudaStreamSynchronize(c->stream));
#undef SC
        } while (0);
    } catch (...) {
        free_ctx(c);
        throw;
    }
    if (st != SFDE_OK) {
        free_ctx(c);
        return st;
    }
    *out = c;
    return SFDE_OK;
}

sfde_status sfde_setup(double beta, double gamma, double kx, double ky, const double omega[4],
                       int nx, int ny, const double* t, int nt, const sfde_opts* opts,
                       sfde_ctx** out) {
    return sfde_no_throw([&] { return setup_impl(beta, gamma, kx, ky, omega, nx, ny, t, nt, opts, out); });
}

sfde_status sfde_set_initial(sfde_ctx* c, const double* psi0) {
    if (!c || !psi0) return SFDE_EINVAL;
    double* tmp = nullptr;
    size_t n = (size_t)c->x.n * c->y.n;
    SFDE_CUDA(cudaMalloc(&tmp, sizeof(double) * n));
    sfde_status st = sfde_copy_in(tmp, psi0, sizeof(double) * n, c->stream);
    if (st == SFDE_OK) {
        sfde_launch_pad(tmp, c->U0, c->y.n, c->x.n, c->y.P, c->x.P, 1, c->stream);
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) { sfde_set_last_cuda_error(e, "set_initial", __FILE__, __LINE__); st = SFDE_ECUDA; }
    }
    cudaFree(tmp);
    return st;
}

static sfde_status set_forcing_impl(sfde_ctx* c, int rank, const double* time_w, const double* bx,
                                    const double* by) {
    if (!c || rank < 0 || rank > SFDE_MAX_RANK) return SFDE_EINVAL;
    cudaFree(c->time_w); cudaFree(c->px); cudaFree(c->py); cudaFree(c->bxn); cudaFree(c->byn);
    cudaFree(c->Fd); cudaFree(c->Fh);
    c->time_w = c->px = c->py = c->bxn = c->byn = c->Fd = c->Fh = nullptr;
    c->rank = 0;
    if (rank == 0) return SFDE_OK;
    if (!time_w || !bx || !by) return SFDE_EINVAL;
    double *bxd = nullptr, *byd = nullptr;
    SFDE_CUDA(cudaMalloc(&c->time_w, sizeof(double) * (size_t)c->nt * rank));
    SFDE_CUDA(cudaMalloc(&c->px, sizeof(double) * (size_t)rank * c->x.P));
    SFDE_CUDA(cudaMalloc(&c->py, sizeof(double) * (size_t)rank * c->y.P));
    SFDE_CUDA(cudaMalloc(&bxd, sizeof(double) * (size_t)rank * c->x.n));
    SFDE_CUDA(cudaMalloc(&byd, sizeof(double) * (size_t)rank * c->y.n));
    c->rank = rank;
    sfde_status st = sfde_copy_in(c->time_w, time_w, sizeof(double) * (size_t)c->nt * rank, c->stream);
    if (st == SFDE_OK) st = sfde_copy_in(bxd, bx, sizeof(double) * (size_t)rank * c->x.n, c->stream);
    if (st == SFDE_OK) st = sfde_copy_in(byd, by, sizeof(double) * (size_t)rank * c->y.n, c->stream);
    if (st == SFDE_OK) st = sfde_project_forcing(c, bxd, byd);
    if (st == SFDE_OK) {  // padded nodal factors for the FP64 space-time residual
        cudaError_t e1 = cudaMalloc(&c->bxn, sizeof(double) * (size_t)rank * c->x.P);
        cudaError_t e2 = cudaMalloc(&c->byn, sizeof(double) * (size_t)rank * c->y.P);
        if (e1 != cudaSuccess || e2 != cudaSuccess) st = SFDE_ENOMEM;
        else {
            sfde_launch_pad(bxd, c->bxn, rank, c->x.n, rank, c->x.P, 1, c->stream);
            sfde_launch_pad(byd, c->byn, rank, c->y.n, rank, c->y.P, 1, c->stream);
        }
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (st == SFDE_OK && e != cudaSuccess) { sfde_set_last_cuda_error(e, "set_forcing", __FILE__, __LINE__); st = SFDE_ECUDA; }
    cudaFree(bxd);
    cudaFree(byd);
    return st;
}

sfde_status sfde_set_forcing(sfde_ctx* c, int rank, const double* time_w, const double* bx,
                             const double* by) {
    return sfde_no_throw([&] { return set_forcing_impl(c, rank, time_w, bx, by); });
}

// F_n, n = 1..N_t, padded into c->Fd; V_y^T F_n V_x into c->Fh (the load of the spectral step);
// staged through a temporary of at most 128 unpadded slices
static sfde_status set_forcing_dense_impl(sfde_ctx* c, const double* F) {
    if (!c) return SFDE_EINVAL;
    SFDE_TRY(set_forcing_impl(c, 0, nullptr, nullptr, nullptr));   // drops any load
    if (!F) return SFDE_OK;
    const size_t n2 = (size_t)c->x.n * c->y.n, P2 = c->P2();
    SFDE_TRY(sfde_ensure_workspace(c, std::min<size_t>((size_t)c->nt, 128)));
    const int chunk = (int)std::min<size_t>(c->ws_slices, 128);
    double* tmp = nullptr;
    cudaError_t e = cudaMalloc(&c->Fd, sizeof(double) * P2 * c->nt);
    if (e == cudaSuccess) e = cudaMalloc(&c->Fh, sizeof(double) * P2 * c->nt);
    if (e == cudaSuccess) e = cudaMalloc(&tmp, sizeof(double) * n2 * chunk);
    sfde_status st = e == cudaSuccess ? SFDE_OK : SFDE_ENOMEM;
    for (int n0 = 0; n0 < c->nt && st == SFDE_OK; n0 += chunk) {
        const int nb = std::min(chunk, c->nt - n0);
        st = sfde_copy_in(tmp, F + (size_t)n0 * n2, sizeof(double) * n2 * nb, c->stream);
        if (st == SFDE_OK) sfde_launch_pad(tmp, c->Fd + (size_t)n0 * P2, c->y.n, c->x.n, c->y.P, c->x.P, nb, c->stream);
        // the pad kernel must finish reading tmp before the next chunk's copy overwrites it: both
        // are on the same stream, in order
    }
    if (st == SFDE_OK) st = sfde_two_sided_fp64(c, c->Fd, c->nt, c->x.V, c->y.V, c->Fh);
    const cudaError_t se = cudaStreamSynchronize(c->stream);
    if (st == SFDE_OK && se != cudaSuccess) { sfde_set_last_cuda_error(se, "set_forcing_dense", __FILE__, __LINE__); st = SFDE_ECUDA; }
    cudaFree(tmp);
    if (st != SFDE_OK) {
        cudaFree(c->Fd); cudaFree(c->Fh);
        c->Fd = c->Fh = nullptr;
    }
    return st;
}

sfde_status sfde_set_forcing_dense(sfde_ctx* c, const double* F) {
    return sfde_no_throw([&] { return set_forcing_dense_impl(c, F); });
}

static sfde_status write_outputs(sfde_ctx* c, double* U, double* U_T) {
    const double* u = c->levels[0].u;
    const size_t n2 = (size_t)c->x.n * c->y.n;
    const size_t P2 = c->P2();
    if (U) {
        if (sfde_is_device_ptr(U)) {
            sfde_launch_unpad(u, U, c->y.n, c->x.n, c->y.P, c->x.P, c->nt + 1, c->stream);
        } else {
            double* tmp = nullptr;
            SFDE_CUDA(cudaMalloc(&tmp, sizeof(double) * n2 * (c->nt + 1)));
            sfde_launch_unpad(u, tmp, c->y.n, c->x.n, c->y.P, c->x.P, c->nt + 1, c->stream);
            cudaError_t e = cudaMemcpyAsync(U, tmp, sizeof(double) * n2 * (c->nt + 1), cudaMemcpyDeviceToHost, c->stream);
            cudaError_t e2 = cudaStreamSynchronize(c->stream);
            cudaFree(tmp);
            SFDE_CUDA(e);
            SFDE_CUDA(e2);
        }
    }
    if (U_T) {
        const double* last = u + P2 * (size_t)c->nt;
        if (sfde_is_device_ptr(U_T)) {
            sfde_launch_unpad(last, U_T, c->y.n, c->x.n, c->y.P, c->x.P, 1, c->stream);
        } else {
            // staged in the step workspace when there is one: cudaFree would synchronise the whole
            // device, stalling instances that run concurrently (sfde_batch_solve)
            const bool ws = c->T1 && c->ws_slices >= 1;
            double* tmp = ws ? c->T1 : nullptr;
            if (!ws) SFDE_CUDA(cudaMalloc(&tmp, sizeof(double) * n2));
            sfde_launch_unpad(last, tmp, c->y.n, c->x.n, c->y.P, c->x.P, 1, c->stream);
            cudaError_t e = cudaMemcpyAsync(U_T, tmp, sizeof(double) * n2, cudaMemcpyDeviceToHost, c->stream);
            cudaError_t e2 = cudaStreamSynchronize(c->stream);
            if (!ws) cudaFree(tmp);
            SFDE_CUDA(e);
            SFDE_CUDA(e2);
        }
    }
    SFDE_CUDA(cudaGetLastError());
    SFDE_CUDA(cudaStreamSynchronize(c->stream));
    return SFDE_OK;
}

static sfde_status mgrit_solve_impl(sfde_ctx* c, const mgrit_opts* opts, double* U, double* U_T,
                                    mgrit_stats* stats) {
    if (!c) return SFDE_EINVAL;
    mgrit_opts o;
    if (opts) {
        o = *opts;
    } else {
        o.m = 2; o.max_levels = 64; o.min_coarse = 2; o.relax = SFDE_RELAX_FCF;
        o.coarse = SFDE_COARSE_AUTO; o.max_iter = 100; o.rel_tol = 1e-10; o.abs_tol = 0.0; o.init_seed = 0;
        o.inner_cycles = 0; o.skip_first_down = 0; o.stop_kind = 0;
    }
    if ((o.m != 0 && o.m < 2) || o.max_levels < 1 || o.min_coarse < 1 || o.max_iter < 1) return SFDE_EINVAL;
    if (o.relax != SFDE_RELAX_FCF && o.relax != SFDE_RELAX_F) return SFDE_EINVAL;
    if (o.coarse < SFDE_COARSE_CN || o.coarse > SFDE_COARSE_AUTO) return SFDE_EINVAL;
    if (!(o.rel_tol >= 0.0) || !(o.abs_tol >= 0.0) || o.inner_cycles < 0) return SFDE_EINVAL;
    if (o.skip_first_down != 0 && o.skip_first_down != 1) return SFDE_EINVAL;
    if (o.stop_kind != 0 && o.stop_kind != 1) return SFDE_EINVAL;
    if (o.m == 0) SFDE_TRY(sfde_choose_m(c, o.coarse, o.rel_tol, &o.m));   // two-level analysis picks m
    sfde_status st;
    if (c->precision == SFDE_PREC_FP64)
        st = sfde_mgrit_fp64(c, &o, stats);
    else
        st = sfde_mgrit_mixed(c, &o, stats);
    if (stats) stats->m_used = o.m;
    if (st != SFDE_OK && st != SFDE_ENOCONV) return st;
    sfde_status wo = write_outputs(c, U, U_T);
    return wo != SFDE_OK ? wo : st;
}

sfde_status mgrit_solve(sfde_ctx* c, const mgrit_opts* opts, double* U, double* U_T,
                        mgrit_stats* stats) {
    return sfde_no_throw([&] { return mgrit_solve_impl(c, opts, U, U_T, stats); });
}

static sfde_status seq_timestep_impl(sfde_ctx* c, double* U, double* U_T, double* seconds) {
    if (!c) return SFDE_EINVAL;
    SFDE_TRY(sfde_seq_fp64(c, seconds));
    return write_outputs(c, U, U_T);
}

sfde_status seq_timestep(sfde_ctx* c, double* U, double* U_T, double* seconds) {
    return sfde_no_throw([&] { return seq_timestep_impl(c, U, U_T, seconds); });
}

static sfde_status step_batch_impl(sfde_ctx* c, int n0, int dn, int batch, const double* in, double* out) {
    if (!c || !in || !out || batch < 1) return SFDE_EINVAL;
    long long last = (long long)n0 + (long long)(batch - 1) * dn;
    if (n0 < 1 || n0 > c->nt || last < 1 || last > c->nt) return SFDE_EINVAL;
    const size_t n2 = (size_t)c->x.n * c->y.n, P2 = c->P2();
    SFDE_TRY(sfde_ensure_workspace(c, (size_t)batch));
    double *tin = nullptr, *pin = nullptr, *pout = nullptr, *tout = nullptr;
    sfde_status st = SFDE_OK;
    cudaError_t e;
#define SC(x) if ((e = (x)) != cudaSuccess) { sfde_set_last_cuda_error(e, #x, __FILE__, __LINE__); st = SFDE_ECUDA; goto done; }
    SC(cudaMalloc(&tin, sizeof(double) * n2 * batch));
    SC(cudaMalloc(&tout, sizeof(double) * n2 * batch));
    SC(cudaMalloc(&pin, sizeof(double) * P2 * batch));
    SC(cudaMalloc(&pout, sizeof(double) * P2 * batch));
    if ((st = sfde_copy_in(tin, in, sizeof(double) * n2 * batch, c->stream)) != SFDE_OK) goto done;
    sfde_launch_pad(tin, pin, c->y.n, c->x.n, c->y.P, c->x.P, batch, c->stream);
    {
        StepBatch sb{};
        sb.batch = batch;
        sb.src = pin; sb.src_stride = (long long)P2;
        sb.dst = pout; sb.dst_stride = (long long)P2;
        sb.dt = c->dt0; sb.n0 = n0; sb.dn = dn; sb.scheme = SCHEME_CN; sb.level0 = true;
        if ((st = sfde_step_any(c, sb, nullptr)) != SFDE_OK) goto done;
    }
    sfde_launch_unpad(pout, tout, c->y.n, c->x.n, c->y.P, c->x.P, batch, c->stream);
    if ((st = sfde_copy_out(out, tout, sizeof(double) * n2 * batch, c->stream)) != SFDE_OK) goto done;
    SC(cudaGetLastError());
    SC(cudaStreamSynchronize(c->stream));
done:
#undef SC
    cudaFree(tin); cudaFree(tout); cudaFree(pin); cudaFree(pout);
    return st;
}

sfde_status sfde_step_batch(sfde_ctx* c, int n0, int dn, int batch, const double* in, double* out) {
    return sfde_no_throw([&] { return step_batch_impl(c, n0, dn, batch, in, out); });
}

static sfde_status propagate_batch_impl(sfde_ctx* c, int scheme, const double* dts, int batch, const double* in,
                                        const double* g, double* out) {
    if (!c || !dts || !in || !out || batch < 1 || (scheme != SFDE_COARSE_CN && scheme != SFDE_COARSE_BE))
        return SFDE_EINVAL;
    for (int b = 0; b < batch; ++b)
        if (!(dts[b] > 0.0) || !isfinite(dts[b])) return SFDE_EINVAL;
    const size_t n2 = (size_t)c->x.n * c->y.n, P2 = c->P2();
    SFDE_TRY(sfde_ensure_workspace(c, (size_t)batch));
    double *tin = nullptr, *pin = nullptr, *pout = nullptr, *tout = nullptr, *pg = nullptr, *ddt = nullptr;
    sfde_status st = SFDE_OK;
    cudaError_t e;
#define SC(x) if ((e = (x)) != cudaSuccess) { sfde_set_last_cuda_error(e, #x, __FILE__, __LINE__); st = SFDE_ECUDA; goto done; }
    SC(cudaMalloc(&tin, sizeof(double) * n2 * batch));
    SC(cudaMalloc(&tout, sizeof(double) * n2 * batch));
    SC(cudaMalloc(&pin, sizeof(double) * P2 * batch));
    SC(cudaMalloc(&pout, sizeof(double) * P2 * batch));
    SC(cudaMalloc(&ddt, sizeof(double) * batch));
    SC(cudaMemcpyAsync(ddt, dts, sizeof(double) * batch, cudaMemcpyHostToDevice, c->stream));
    if ((st = sfde_copy_in(tin, in, sizeof(double) * n2 * batch, c->stream)) != SFDE_OK) goto done;
    sfde_launch_pad(tin, pin, c->y.n, c->x.n, c->y.P, c->x.P, batch, c->stream);
    if (g) {
        SC(cudaMalloc(&pg, sizeof(double) * P2 * batch));
        if ((st = sfde_copy_in(tout, g, sizeof(double) * n2 * batch, c->stream)) != SFDE_OK) goto done;
        sfde_launch_pad(tout, pg, c->y.n, c->x.n, c->y.P, c->x.P, batch, c->stream);
    }
    {
        StepBatch sb{};
        sb.batch = batch;
        sb.src = pin; sb.src_stride = (long long)P2;
        sb.dst = pout; sb.dst_stride = (long long)P2;
        sb.g = pg; sb.g_stride = (long long)P2;
        sb.dt = ddt; sb.n0 = 1; sb.dn = 1;   // slice b takes dt[b]
        sb.scheme = scheme == SFDE_COARSE_CN ? SCHEME_CN : SCHEME_BE;
        sb.level0 = false;
        if ((st = sfde_step_any(c, sb, nullptr)) != SFDE_OK) goto done;
    }
    sfde_launch_unpad(pout, tout, c->y.n, c->x.n, c->y.P, c->x.P, batch, c->stream);
    if ((st = sfde_copy_out(out, tout, sizeof(double) * n2 * batch, c->stream)) != SFDE_OK) goto done;
    SC(cudaGetLastError());
    SC(cudaStreamSynchronize(c->stream));
done:
#undef SC
    cudaFree(tin); cudaFree(tout); cudaFree(pin); cudaFree(pout); cudaFree(pg); cudaFree(ddt);
    return st;
}

sfde_status sfde_propagate_batch(sfde_ctx* c, int scheme, const double* dts, int batch, const double* in,
                                 const double* g, double* out) {
    return sfde_no_throw([&] { return propagate_batch_impl(c, scheme, dts, batch, in, g, out); });
}

sfde_status sfde_get_operator(sfde_ctx* c, int dir, double* coeffs, double* lambda, double* V) {
    if (!c || (dir != 0 && dir != 1)) return SFDE_EINVAL;
    SfdeDir& d = dir == 0 ? c->x : c->y;
    if (coeffs) SFDE_CUDA(cudaMemcpy(coeffs, d.coeffs, sizeof(double) * d.n, cudaMemcpyDeviceToHost));
    if (lambda) SFDE_CUDA(cudaMemcpy(lambda, d.lam, sizeof(double) * d.n, cudaMemcpyDeviceToHost));
    if (V) SFDE_CUDA(cudaMemcpy2D(V, sizeof(double) * d.n, d.V, sizeof(double) * d.P,
                                  sizeof(double) * d.n, d.n, cudaMemcpyDeviceToHost));
    return SFDE_OK;
}

sfde_status sfde_profile_enable(sfde_ctx* c, int enable) {
    if (!c) return SFDE_EINVAL;
    SFDE_CUDA(cudaStreamSynchronize(c->stream));
    prof_flush_all(c);
    SfdeProf& P = c->prof;
    P.on = enable != 0;
    P.head = P.count = 0;
    P.launches = 0;
    for (int k = 0; k < SfdeProf::NCLS; ++k) { P.n[k] = 0; P.ms[k] = P.tot_flops[k] = P.tot_bytes[k] = 0.0; }
    return SFDE_OK;
}

sfde_status sfde_profile_read(sfde_ctx* c, sfde_profile* out) {
    if (!c || !out) return SFDE_EINVAL;
    SFDE_CUDA(cudaStreamSynchronize(c->stream));
    prof_flush_all(c);
    const SfdeProf& P = c->prof;
    out->kernel_launches = P.launches;
    for (int k = 0; k < SfdeProf::NCLS; ++k) {
        out->launches[k] = P.n[k];
        out->ms[k] = P.ms[k];
        out->flops[k] = P.tot_flops[k];
        out->bytes[k] = P.tot_bytes[k];
    }
    return SFDE_OK;
}

void sfde_destroy(sfde_ctx* c) { free_ctx(c); }

}  // extern "C"
