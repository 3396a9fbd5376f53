// Mixed-precision MGRIT: FP64 iterative refinement around low-precision tensor-core V-cycles.
//
// The iterate U (all time points) is FP64.  One outer iteration
//   1. forms the space-time residual of Eq. (2.4) to FP64 accuracy,
//          rho_n = F_n + B_n U_{n-1} - S_n U_n = F_n + M_h (U_{n-1} - U_n) - tau_n K (U_{n-1} + U_n),
//      (P <= 256 or a multiple of 256 up to 1024: exact integer arithmetic around two digit-split
//      tensor-core products per time point, resid_int.cu; other P: FP64 slice GEMMs) and its norm,
//      and stores rho in BF16/FP32;
//   2. turns it into the right-hand side of the correction system in Psi form, g_n = S_n^{-1} rho_n
//      (the fast-diagonalisation solve, one batched spectral step in solve mode), so that the
//      correction E solves E_n = Psi_n E_{n-1} + g_n, E_0 = 0 -- the system of Eq. (3.1) again;
//   3. runs K V-cycles of Algorithm 1 on that system (K = 4 BF16, 5 TF32, or mgrit_opts.inner_cycles)
//      with every step a tensor-core spectral step (BF16 or TF32 operands, FP32 accumulation); the
//      coarse levels' sweeps run in the step's eigenbasis;
//   4. adds E to U in FP64.
// The low-precision V-cycles converge to the fixed point of the rounded propagator, whose distance
// from the exact correction (about 2e-2 relative for BF16 and 3e-3 for TF32 at the benchmark sizes)
// is the contraction per outer iteration; the accuracy of the result is set by the FP64 residual.
#include <math.h>

#include <algorithm>
#include <climits>
#include <new>
#include <vector>

#include <cuda_bf16.h>

#include "sfde_internal.cuh"

sfde_status sfde_level0(sfde_ctx* c, double** u);  // mgrit.cu
void sfde_launch_fill_random(double* u, int nt, int ny, int nx, int Py, int Px, uint64_t seed, cudaStream_t s);

namespace {

// Storage of the low-precision levels by operand kind: BF16 (kind 0); FP32 rounded to TF32, the
// values the TF32 tensor cores read (kind 1); FP32 (kind 2, the three-product FP32 form), a 4-byte
// type of its own so that every kernel below stores it without the TF32 rounding.
struct F32 { float v; };
template <typename T> __device__ __forceinline__ T to_lp(double v);
template <> __device__ __forceinline__ __nv_bfloat16 to_lp<__nv_bfloat16>(double v) { return __float2bfloat16_rn((float)v); }
template <> __device__ __forceinline__ float to_lp<float>(double v) { return sfde_round_tf32((float)v); }
template <> __device__ __forceinline__ F32 to_lp<F32>(double v) { return F32{(float)v}; }
__device__ __forceinline__ float lp_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float lp_f(float v) { return v; }
__device__ __forceinline__ float lp_f(F32 v) { return v.v; }

template <typename T>
__global__ void k_to_lp(const double* src, T* dst, size_t n) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        dst[e] = to_lp<T>(src[e]);
}

__global__ void k_to_f32(const double* src, float* dst, size_t n) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        dst[e] = (float)src[e];
}

// out = a - b (one slice)
template <typename T>
__global__ void k_lp_diff(T* out, const T* a, const T* b, size_t n) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        out[e] = to_lp<T>((double)lp_f(a[e]) - (double)lp_f(b[e]));
}

// y[k*ys] += x[k*xs] over `slices` slices of P2 elements (C-point correction)
template <typename T>
__global__ void k_lp_axpy_strided(T* y, long long ys, const T* x, long long xs, size_t P2) {
    const size_t sl = blockIdx.y;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P2; e += (size_t)gridDim.x * blockDim.x)
        y[sl * ys + e] = to_lp<T>((double)lp_f(y[sl * ys + e]) + (double)lp_f(x[sl * xs + e]));
}

// U += E in FP64 for n elements (the refinement update), four per thread and iteration (n a
// multiple of 4, U 16-byte and E 8-byte aligned: whole padded slices)
template <typename T>
__global__ void k_add_correction(double* U, const T* E, size_t n) {
    const size_t n4 = n / 4;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n4; e += (size_t)gridDim.x * blockDim.x) {
        double2* u = (double2*)(U + 4 * e);
        double2 a = u[0], b = u[1];
        float x0, x1, x2, x3;
        if constexpr (sizeof(T) == 2) {
            const uint2 w = __ldg((const uint2*)(E + 4 * e));
            x0 = __uint_as_float(w.x << 16); x1 = __uint_as_float(w.x & 0xFFFF0000u);
            x2 = __uint_as_float(w.y << 16); x3 = __uint_as_float(w.y & 0xFFFF0000u);
        } else {
            const float4 w = __ldg((const float4*)(const void*)(E + 4 * e));
            x0 = w.x; x1 = w.y; x2 = w.z; x3 = w.w;
        }
        a.x += (double)x0; a.y += (double)x1; b.x += (double)x2; b.y += (double)x3;
        u[0] = a;
        u[1] = b;
    }
}

// four consecutive low-precision values <-> FP32 (8-byte BF16 / 16-byte FP32 accesses)
__device__ __forceinline__ void ld4(const __nv_bfloat16* p, float (&v)[4]) {
    const uint2 w = *(const uint2*)p;
    v[0] = __uint_as_float(w.x << 16); v[1] = __uint_as_float(w.x & 0xFFFF0000u);
    v[2] = __uint_as_float(w.y << 16); v[3] = __uint_as_float(w.y & 0xFFFF0000u);
}
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
    const float4 w = *(const float4*)p;
    v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
}
__device__ __forceinline__ void ld4(const F32* p, float (&v)[4]) { ld4((const float*)p, v); }
__device__ __forceinline__ void st4(__nv_bfloat16* p, const float (&v)[4]) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]), b = __floats2bfloat162_rn(v[2], v[3]);
    uint2 w;
    w.x = *(const uint32_t*)&a;
    w.y = *(const uint32_t*)&b;
    *(uint2*)p = w;
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
    *(float4*)p = make_float4(sfde_round_tf32(v[0]), sfde_round_tf32(v[1]), sfde_round_tf32(v[2]), sfde_round_tf32(v[3]));
}
__device__ __forceinline__ void st4(F32* p, const float (&v)[4]) { *(float4*)p = make_float4(v[0], v[1], v[2], v[3]); }

// F-relaxation over intervals of `len` points in the eigenbasis of the step.  Phi(X) = V_y [f o
// (W_y^T X W_x)] V_x^T with W^T V = I (Sec. 2's fast diagonalisation), so u_{il+j} =
// Phi(u_{il+j-1}) + g_{il+j} reads, for transformed values, v_j = f_j o v_{j-1} + g^_{il+j}: one
// recurrence per mode.  v_0 = Uc[i] (the transformed C-point value), g^_{il+j} = G[i gis + j + gj0], f_j the
// modal factor of the step with dt[i dis + j - 1] (backward Euler 1/(1 + dt sigma), Crank-Nicolson
// (1 - dt sigma/2)/(1 + dt sigma/2), sigma = K_x lambda_x + K_y lambda_y of the mode); v_j,
// j = 1 .. len - 1, goes to Y[i (len - 1) + j - 1].  FP32 recurrence; four modes of one row per
// thread (P_x a multiple of 4); grid.y = intervals.
template <typename T>
__global__ void __launch_bounds__(256) k_modal_scan(const T* __restrict__ Uc, const T* __restrict__ G, int gis, int gj0,
                                                    T* __restrict__ Y, int len, int Px, size_t P2,
                                                    const float* __restrict__ lamx, const float* __restrict__ lamy,
                                                    float kx, float ky, const double* __restrict__ dt, int dis,
                                                    int scheme) {
    const size_t i = blockIdx.y;
    const size_t e = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (e >= P2) return;
    const int x = (int)(e % (size_t)Px), y = (int)(e / (size_t)Px);
    const float sy = ky * lamy[y];
    float sg[4], v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) sg[q] = fmaf(kx, lamx[x + q], sy);
    ld4(Uc + i * P2 + e, v);
    const bool be = scheme == SCHEME_BE;
    // eight steps at a time: their right-hand sides are loaded before the first is used, so the
    // load latencies overlap instead of adding up along the recurrence
    for (int j0 = 1; j0 < len; j0 += 8) {
        float gv[8][4], cst[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (j0 + u < len) {
                const float dtj = (float)dt[i * dis + j0 + u - 1];
                cst[u] = be ? dtj : 0.5f * dtj;
                ld4(G + (i * gis + j0 + u + gj0) * P2 + e, gv[u]);
            }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (j0 + u < len) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float f = 1.f / fmaf(cst[u], sg[q], 1.f);
                    if (!be) f = fmaf(2.f, f, -1.f);
                    v[q] = fmaf(f, v[q], gv[u][q]);
                }
                st4(Y + (i * (len - 1) + j0 + u - 1) * P2 + e, v);
            }
    }
}

// The inner solve held in the step's eigenbasis (modal_chains 4, FP32 storage).  With the inner
// solve's levels transformed once, every step is the per-mode recurrence v_j = f_j v_{j-1} + g_j:
// runs over `len` points of `grid.y` groups, v_0 = U[i ucs], g_j = G[i gis + j + gj0], v_j stored to
// Y[i yis + j + yj0], f_j the modal factor of the step with dt[i dis + j - 1] (as k_modal_scan);
// plain FP32 stores (the values stay in the eigenbasis, nothing feeds a TF32 product step by step).
__global__ void __launch_bounds__(256) k_modal_run(const float* __restrict__ U, long long ucs, const float* __restrict__ G,
                                                   long long gis, long long gj0, float* __restrict__ Y, long long yis,
                                                   long long yj0, int len, int Px, size_t P2,
                                                   const float* __restrict__ lamx, const float* __restrict__ lamy,
                                                   float kx, float ky, const double* __restrict__ dt, long long dis,
                                                   int scheme) {
    const long long i = blockIdx.y;
    const size_t e = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (e >= P2) return;
    const int x = (int)(e % (size_t)Px), y = (int)(e / (size_t)Px);
    const float sy = ky * lamy[y];
    float sg[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) sg[q] = fmaf(kx, lamx[x + q], sy);
    float4 v = *(const float4*)(U + (size_t)(i * ucs) * P2 + e);
    const bool be = scheme == SCHEME_BE;
    for (int j0 = 1; j0 < len; j0 += 8) {
        float4 gv[8];
        float cst[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (j0 + u < len) {
                const float dtj = (float)dt[i * dis + j0 + u - 1];
                cst[u] = be ? dtj : 0.5f * dtj;
                gv[u] = *(const float4*)(G + (size_t)(i * gis + j0 + u + gj0) * P2 + e);
            }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (j0 + u < len) {
                float f[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    f[q] = 1.f / fmaf(cst[u], sg[q], 1.f);
                    if (!be) f[q] = fmaf(2.f, f[q], -1.f);
                }
                v.x = fmaf(f[0], v.x, gv[u].x);
                v.y = fmaf(f[1], v.y, gv[u].y);
                v.z = fmaf(f[2], v.z, gv[u].z);
                v.w = fmaf(f[3], v.w, gv[u].w);
                *(float4*)(Y + (size_t)(i * yis + j0 + u + yj0) * P2 + e) = v;
            }
    }
}

// The C-point residuals of the eigenbasis recurrence, injected into the coarse level:
// out[k - 1] = f_{km} u_{km-1} + g_{km} - u_{km}, k = 1 + blockIdx.y (plain FP32 stores)
__global__ void __launch_bounds__(256) k_modal_resid(const float* __restrict__ u, const float* __restrict__ g,
                                                     float* __restrict__ out, int m, int Px, size_t P2,
                                                     const float* __restrict__ lamx, const float* __restrict__ lamy,
                                                     float kx, float ky, const double* __restrict__ dt, int scheme) {
    const long long k = (long long)blockIdx.y + 1, n = k * m;
    const size_t e = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (e >= P2) return;
    const int x = (int)(e % (size_t)Px), y = (int)(e / (size_t)Px);
    const float sy = ky * lamy[y];
    const float dtn = (float)dt[n - 1];
    const bool be = scheme == SCHEME_BE;
    const float cst = be ? dtn : 0.5f * dtn;
    const float4 a = *(const float4*)(u + (size_t)(n - 1) * P2 + e), b = *(const float4*)(u + (size_t)n * P2 + e);
    const float4 gg = *(const float4*)(g + (size_t)n * P2 + e);
    float f[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        f[q] = 1.f / fmaf(cst, fmaf(kx, lamx[x + q], sy), 1.f);
        if (!be) f[q] = fmaf(2.f, f[q], -1.f);
    }
    float4 r;
    r.x = fmaf(f[0], a.x, gg.x) - b.x;
    r.y = fmaf(f[1], a.y, gg.y) - b.y;
    r.z = fmaf(f[2], a.z, gg.z) - b.z;
    r.w = fmaf(f[3], a.w, gg.w) - b.w;
    *(float4*)(out + (size_t)(k - 1) * P2 + e) = r;
}

unsigned grid_for(size_t n) {
    size_t g = (n + 255) / 256;
    return (unsigned)std::min<size_t>(std::max<size_t>(g, 1), 4 * 152);
}

}  // namespace

struct LpLevel {
    int N = 0;
    long long nalloc = 0;      // slices allocated (a multiple of m, > N)
    std::vector<double> t;
    double* dt = nullptr;      // device; level 0 uses ctx->dt0
    void* u = nullptr;         // (nalloc) x P^2 of T
    void* g = nullptr;
    void* gm = nullptr;        // levels >= 1: g transformed to the eigenbasis, (N + 1) x P^2 of T
    bool own_dt = false;
};

struct MapEntry {
    const void* ptr; int R, C, ds; long long ns;
    CUtensorMap map;
};

struct SfdeMixed {
    int kind = -1, esz = 0, m = 0, max_levels = 0, min_coarse = 0;
    void *WTx = nullptr, *WTy = nullptr, *Vx = nullptr, *Vy = nullptr, *VTx = nullptr, *VTy = nullptr;
    float *lamx = nullptr, *lamy = nullptr;
    CUtensorMap mWTx, mWTy, mVx, mVy, mVTx, mVTy;
    // the same matrices as the fixed operand of the slice GEMM (its tile rows per box)
    CUtensorMap gWTx, gWTy, gVx, gVy, gVTx, gVTy;
    // kind 2: their low parts (FP32 products from three TF32 products) and maps
    void *lWTx = nullptr, *lWTy = nullptr, *lVx = nullptr, *lVy = nullptr, *lVTx = nullptr, *lVTy = nullptr;
    CUtensorMap oWTx, oWTy, oVx, oVy, oVTx, oVTy;
    // the same matrices in 128-row boxes: the pair form of the fused step (P = 256)
    bool pair_ok = false;
    int nsm = 0;
    CUtensorMap hWTx, hWTy, hVx, hVy, hVTx, hVTy;
    std::vector<LpLevel> lev;
    void *T1 = nullptr, *T2 = nullptr, *T3 = nullptr;
    size_t ws = 0;
    void* mY = nullptr;        // transformed F-point values of a modal sweep (max N_l, l >= 1, slices)
    int* err = nullptr;
    std::vector<MapEntry> maps;
    // captured inner solve (CUDA graph) and what it contains
    cudaStream_t cap = nullptr;
    // the inner solve in captured parts: prologue, one V-cycle (replayed K-1 times), epilogue, and
    // the first V-cycle without down-cycle relaxation (skip_first_down)
    cudaGraphExec_t inner_exec[4] = {nullptr, nullptr, nullptr, nullptr};
    long long inner_key = -1, inner_launches[4] = {0, 0, 0, 0}, inner_steps[4] = {0, 0, 0, 0};
    // FP64-accurate residual in integer arithmetic around tensor-core products (P <= 256 or a
    // multiple of 256 up to 1024)
    bool use_oz = false;
    OzMatrix oAx, oAy;
    void *oz_dV = nullptr, *oz_dVt = nullptr;
    int* oz_E = nullptr;
    // each BF16 step as one fused four-product kernel (P_x = P_y in {128, 256})
    bool fused = false;
    // the fine level's modal buffers exist (its F-relaxations in the eigenbasis too)
    bool modal_fine = false;
    // every buffer and map of the setup is in place
    bool ready = false;
};

void sfde_free_mixed(sfde_ctx* c) {
    SfdeMixed* M = c->mixed;
    if (!M) return;
    cudaFree(M->WTx); cudaFree(M->WTy); cudaFree(M->Vx); cudaFree(M->Vy); cudaFree(M->VTx); cudaFree(M->VTy);
    cudaFree(M->lWTx); cudaFree(M->lWTy); cudaFree(M->lVx); cudaFree(M->lVy); cudaFree(M->lVTx); cudaFree(M->lVTy);
    cudaFree(M->lamx); cudaFree(M->lamy);
    for (auto& L : M->lev) {
        if (L.own_dt) cudaFree(L.dt);
        cudaFree(L.u); cudaFree(L.g); cudaFree(L.gm);
    }
    cudaFree(M->T1); cudaFree(M->T2); cudaFree(M->T3); cudaFree(M->mY); cudaFree(M->err);
    for (auto& g : M->inner_exec)
        if (g) cudaGraphExecDestroy(g);
    sfde_oz_free_matrix(&M->oAx);
    sfde_oz_free_matrix(&M->oAy);
    cudaFree(M->oz_dV);
    cudaFree(M->oz_dVt);
    cudaFree(M->oz_E);
    if (M->cap) cudaStreamDestroy(M->cap);
    delete M;
    c->mixed = nullptr;
}

namespace {

sfde_status lp_copy(sfde_ctx* c, const double* src, void** dst, size_t n, int kind) {
    const size_t esz = kind == 0 ? 2 : 4;
    SFDE_CUDA(cudaMalloc(dst, esz * n));
    if (kind == 0) k_to_lp<__nv_bfloat16><<<grid_for(n), 256, 0, c->stream>>>(src, (__nv_bfloat16*)*dst, n);
    else if (kind == 1) k_to_lp<float><<<grid_for(n), 256, 0, c->stream>>>(src, (float*)*dst, n);
    else k_to_lp<F32><<<grid_for(n), 256, 0, c->stream>>>(src, (F32*)*dst, n);
    sfde_count_launch(c);
    SFDE_CUDA(cudaGetLastError());
    return SFDE_OK;
}

// kind 2: the low parts of an FP32 operand copy (the third product of the FP32 form)
sfde_status lo_copy(sfde_ctx* c, const void* src, void** dst, size_t n) {
    SFDE_CUDA(cudaMalloc(dst, sizeof(float) * n));
    SFDE_TRY(sfde_tc_lo_parts((const float*)src, (float*)*dst, n, c->stream));
    sfde_count_launch(c);
    return SFDE_OK;
}

// Returns a copy: the cache vector may grow (and move its elements) on a later lookup.
sfde_status map_for(SfdeMixed* M, const void* ptr, int R, int C, int ds, long long ns, CUtensorMap* out) {
    for (const auto& e : M->maps)
        if (e.ptr == ptr && e.R == R && e.C == C && e.ds == ds && e.ns == ns) { *out = e.map; return SFDE_OK; }
    MapEntry e{ptr, R, C, ds, ns, {}};
    SFDE_TRY(sfde_tc_map_slices(&e.map, ptr, M->esz, C, R, ds, ns));
    M->maps.push_back(e);
    *out = e.map;
    return SFDE_OK;
}

// Time points per level of the inner hierarchy: coarsen by m while the level divides, the coarse
// level keeps at least min_coarse points and max_levels allows it.  A coarse level whose direct
// sweep (N steps) is no longer than relaxing it (FCF: 2m - 1 steps, C-point residual: 1, final
// F-relaxation: m - 1) plus the sweep of the level below is the coarsest: the inner V-cycle's
// critical path gets shorter and its coarse solve exact.
std::vector<int> inner_level_sizes(int nt, int m, int max_levels, int min_coarse) {
    std::vector<int> n{nt};
    while ((int)n.size() < max_levels) {
        const int N = n.back();
        if (N % m != 0 || N / m < min_coarse) break;
        if (n.size() > 1 && N <= 3 * m - 1 + N / m) break;
        n.push_back(N / m);
    }
    return n;
}

// Digits per operand of the tensor-core residual: the refinement needs the residual to a fraction
// of its own size only, about 1e-5 ||rho_{k-1}|| (relative to the first residual res0, a wide
// margin); the digit products of nd digits are accurate to about 2^{9-8 nd} of the operands' scale.
// The first residual (prev = 0) takes 4.
int residual_digits_for(double prev, double res0) {
    if (!(prev > 0.0) || !(res0 > 0.0)) return 4;
    const double need = 1e-5 * prev / res0;
    int nd = 4;
    while (nd < 7 && ldexp(1.0, 9 - 8 * nd) > need) ++nd;
    return nd;
}

sfde_status setup_mixed_body(sfde_ctx* c, int kind, int m, int max_levels, int min_coarse);

// Operands, maps and the inner hierarchy for (kind, m, levels), kept while those stay the same.  A
// setup that fails part-way is freed whole, so no later call finds a half-built one.
sfde_status setup_mixed(sfde_ctx* c, int kind, int m, int max_levels, int min_coarse) {
    SfdeMixed* M = c->mixed;
    if (M && M->ready && M->kind == kind && M->m == m && M->max_levels == max_levels &&
        M->min_coarse == min_coarse && M->modal_fine == (c->modal_chains == 2 || (c->modal_chains == 3 && kind == 0)))
        return SFDE_OK;
    sfde_free_mixed(c);
    const sfde_status st = setup_mixed_body(c, kind, m, max_levels, min_coarse);
    if (st == SFDE_OK) c->mixed->ready = true;
    else sfde_free_mixed(c);
    return st;
}

sfde_status setup_mixed_body(sfde_ctx* c, int kind, int m, int max_levels, int min_coarse) {
    SfdeMixed* M = new (std::nothrow) SfdeMixed();
    if (!M) return SFDE_ENOMEM;
    c->mixed = M;
    M->kind = kind; M->esz = kind == 0 ? 2 : 4; M->m = m; M->max_levels = max_levels; M->min_coarse = min_coarse;
    M->modal_fine = c->modal_chains == 2 || (c->modal_chains == 3 && kind == 0);
    SFDE_TRY(sfde_tc_prepare());
    SFDE_TRY(sfde_fused_prepare());
    const int Px = c->x.P, Py = c->y.P;
    const size_t P2 = c->P2();
    SFDE_TRY(lp_copy(c, c->x.WT, &M->WTx, (size_t)Px * Px, kind));
    SFDE_TRY(lp_copy(c, c->y.WT, &M->WTy, (size_t)Py * Py, kind));
    SFDE_TRY(lp_copy(c, c->x.V, &M->Vx, (size_t)Px * Px, kind));
    SFDE_TRY(lp_copy(c, c->y.V, &M->Vy, (size_t)Py * Py, kind));
    SFDE_TRY(lp_copy(c, c->x.VT, &M->VTx, (size_t)Px * Px, kind));
    SFDE_TRY(lp_copy(c, c->y.VT, &M->VTy, (size_t)Py * Py, kind));
    SFDE_CUDA(cudaMalloc(&M->lamx, sizeof(float) * Px));
    SFDE_CUDA(cudaMalloc(&M->lamy, sizeof(float) * Py));
    k_to_f32<<<grid_for(Px), 256, 0, c->stream>>>(c->x.lam, M->lamx, Px);
    k_to_f32<<<grid_for(Py), 256, 0, c->stream>>>(c->y.lam, M->lamy, Py);
    SFDE_CUDA(cudaGetLastError());
    SFDE_TRY(sfde_tc_map_matrix(&M->mWTx, M->WTx, M->esz, Px, Px));
    SFDE_TRY(sfde_tc_map_matrix(&M->mWTy, M->WTy, M->esz, Py, Py));
    SFDE_TRY(sfde_tc_map_matrix(&M->mVx, M->Vx, M->esz, Px, Px));
    SFDE_TRY(sfde_tc_map_matrix(&M->mVy, M->Vy, M->esz, Py, Py));
    SFDE_TRY(sfde_tc_map_matrix(&M->mVTx, M->VTx, M->esz, Px, Px));
    SFDE_TRY(sfde_tc_map_matrix(&M->mVTy, M->VTy, M->esz, Py, Py));
    SFDE_TRY(sfde_tc_map_gemm_matrix(&M->gWTx, M->WTx, M->kind, Px, Px));
    SFDE_TRY(sfde_tc_map_gemm_matrix(&M->gWTy, M->WTy, M->kind, Py, Py));
    SFDE_TRY(sfde_tc_map_gemm_matrix(&M->gVx, M->Vx, M->kind, Px, Px));
    SFDE_TRY(sfde_tc_map_gemm_matrix(&M->gVy, M->Vy, M->kind, Py, Py));
    SFDE_TRY(sfde_tc_map_gemm_matrix(&M->gVTx, M->VTx, M->kind, Px, Px));
    SFDE_TRY(sfde_tc_map_gemm_matrix(&M->gVTy, M->VTy, M->kind, Py, Py));
    if (kind == 2) {
        SFDE_TRY(lo_copy(c, M->WTx, &M->lWTx, (size_t)Px * Px));
        SFDE_TRY(lo_copy(c, M->WTy, &M->lWTy, (size_t)Py * Py));
        SFDE_TRY(lo_copy(c, M->Vx, &M->lVx, (size_t)Px * Px));
        SFDE_TRY(lo_copy(c, M->Vy, &M->lVy, (size_t)Py * Py));
        SFDE_TRY(lo_copy(c, M->VTx, &M->lVTx, (size_t)Px * Px));
        SFDE_TRY(lo_copy(c, M->VTy, &M->lVTy, (size_t)Py * Py));
        SFDE_TRY(sfde_tc_map_gemm_matrix(&M->oWTx, M->lWTx, 2, Px, Px));
        SFDE_TRY(sfde_tc_map_gemm_matrix(&M->oWTy, M->lWTy, 2, Py, Py));
        SFDE_TRY(sfde_tc_map_gemm_matrix(&M->oVx, M->lVx, 2, Px, Px));
        SFDE_TRY(sfde_tc_map_gemm_matrix(&M->oVy, M->lVy, 2, Py, Py));
        SFDE_TRY(sfde_tc_map_gemm_matrix(&M->oVTx, M->lVTx, 2, Px, Px));
        SFDE_TRY(sfde_tc_map_gemm_matrix(&M->oVTy, M->lVTy, 2, Py, Py));
    }
    M->pair_ok = kind == 0 && Px == Py && sfde_fused_pair_supported(Px);
    if (M->pair_ok) {
        SFDE_TRY(sfde_tc_map_matrix_rows(&M->hWTx, M->WTx, M->esz, Px, Px, 128));
        SFDE_TRY(sfde_tc_map_matrix_rows(&M->hWTy, M->WTy, M->esz, Py, Py, 128));
        SFDE_TRY(sfde_tc_map_matrix_rows(&M->hVx, M->Vx, M->esz, Px, Px, 128));
        SFDE_TRY(sfde_tc_map_matrix_rows(&M->hVy, M->Vy, M->esz, Py, Py, 128));
        SFDE_TRY(sfde_tc_map_matrix_rows(&M->hVTx, M->VTx, M->esz, Px, Px, 128));
        SFDE_TRY(sfde_tc_map_matrix_rows(&M->hVTy, M->VTy, M->esz, Py, Py, 128));
    }
    {
        int dev = 0;
        SFDE_CUDA(cudaGetDevice(&dev));
        SFDE_CUDA(cudaDeviceGetAttribute(&M->nsm, cudaDevAttrMultiProcessorCount, dev));
    }
    SFDE_CUDA(cudaMalloc(&M->err, sizeof(int)));
    SFDE_CUDA(cudaMemsetAsync(M->err, 0, sizeof(int), c->stream));
    // inner hierarchy
    const std::vector<int> sizes = inner_level_sizes(c->nt, m, max_levels, min_coarse);
    for (size_t l = 0; l < sizes.size(); ++l) {
        M->lev.emplace_back();
        LpLevel& G = M->lev.back();
        G.N = sizes[l];
        if (l == 0) {
            G.t = c->t;
            G.dt = c->dt0;
            continue;
        }
        const LpLevel& F = M->lev[l - 1];
        G.t.resize(G.N + 1);
        for (int k = 0; k <= G.N; ++k) G.t[k] = F.t[(size_t)k * m];
        std::vector<double> dt(G.N);
        for (int k = 0; k < G.N; ++k) dt[k] = G.t[k + 1] - G.t[k];
        G.own_dt = true;
        SFDE_CUDA(cudaMalloc(&G.dt, sizeof(double) * G.N));
        SFDE_CUDA(cudaMemcpy(G.dt, dt.data(), sizeof(double) * G.N, cudaMemcpyHostToDevice));
    }
    for (auto& L : M->lev) {
        L.nalloc = ((long long)(L.N + 1 + m - 1) / m) * m + m;
        SFDE_CUDA(cudaMalloc(&L.u, M->esz * P2 * L.nalloc));
        SFDE_CUDA(cudaMalloc(&L.g, M->esz * P2 * L.nalloc));
        SFDE_CUDA(cudaMemsetAsync(L.u, 0, M->esz * P2 * L.nalloc, c->stream));
        SFDE_CUDA(cudaMemsetAsync(L.g, 0, M->esz * P2 * L.nalloc, c->stream));
    }
    // modal sweeps of the coarse levels (and of the fine level when asked): transformed right-hand
    // sides per level, one scratch
    {
        int ymax = 0;
        for (size_t l = M->modal_fine ? 0 : 1; l < M->lev.size(); ++l) {
            LpLevel& L = M->lev[l];
            SFDE_CUDA(cudaMalloc(&L.gm, M->esz * P2 * (size_t)(L.N + 1)));
            ymax = std::max(ymax, L.N);
        }
        if (ymax > 0) SFDE_CUDA(cudaMalloc(&M->mY, M->esz * P2 * (size_t)ymax));
    }
    M->ws = (size_t)std::max(1, std::min(c->nt, 512));
    SFDE_CUDA(cudaMalloc(&M->T1, M->esz * P2 * M->ws));
    SFDE_CUDA(cudaMalloc(&M->T2, M->esz * P2 * M->ws));
    SFDE_CUDA(cudaMalloc(&M->T3, M->esz * P2 * M->ws));
    // FP64 scratch for the residual: a chunk of time points at a time
    SFDE_TRY(sfde_ensure_workspace(c, std::min<size_t>(c->nt, 128)));
    // products of the residual on the tensor cores (error-free digit splitting) when K <= 256
    M->use_oz = sfde_resid_int_supported(Px, Py);
    if (M->use_oz) {
        SFDE_TRY(sfde_resid_int_matrices(c, &M->oAx, &M->oAy));
        SFDE_CUDA(cudaMalloc(&M->oz_dV, sfde_resid_int_digit_bytes(Px, Py, (int)c->ws_slices)));
        SFDE_CUDA(cudaMalloc(&M->oz_dVt, sfde_resid_int_digit_bytes(Px, Py, (int)c->ws_slices)));
        SFDE_CUDA(cudaMalloc(&M->oz_E, sizeof(int) * ((size_t)c->nt + 1)));
    }
    size_t need = (size_t)c->nt * (size_t)(c->x.P / 16) * (c->y.P / 16) + 64;
    if (c->partial_cap < need) {
        cudaFree(c->partial);
        c->partial = nullptr;
        SFDE_CUDA(cudaMalloc(&c->partial, sizeof(double) * need));
        c->partial_cap = need;
    }
    SFDE_CUDA(cudaStreamSynchronize(c->stream));
    return SFDE_OK;
}

struct LpEngine {
    sfde_ctx* c;
    SfdeMixed* M;
    int m, L, relax, scheme;
    long long steps = 0;
    bool skip = false;   // down-cycle without relaxation (first V-cycle with skip_first_down)
    bool full = false;   // every level's u and g held in the step's eigenbasis (modal_chains 4)

    size_t P2() const { return c->P2(); }
    char* slice(void* base, long long s) const { return (char*)base + (size_t)s * P2() * M->esz; }

    // One batched spectral step (or solve when `solve`), slices src0 + b*ds of `src` (a buffer of
    // `ns` slices) -> dst slices (stride dst_ds slices); optional g and u-target (stride dn slices).
    sfde_status step(void* src, long long ns, int src0, int ds, int batch, bool solve, int sch,
                     const double* dt, int n0, int dn, void* dst, int dst_ds, const void* g, const void* ut,
                     double* partial, int* npart, int nchain = 1) {
        const int Px = c->x.P, Py = c->y.P;
        const long long P2l = (long long)P2();
        if (M->fused) {
            CUtensorMap a1;
            SFDE_TRY(map_for(M, src, Py, Px, ds, ns, &a1));
            if (partial && (size_t)batch > c->partial_cap) return SFDE_EINVAL;
            FusedStepArgs a{};
            a.s0 = src0; a.ds = ds; a.batch = batch; a.nchain = nchain;
            a.dst = dst; a.dst_stride = (long long)dst_ds * P2l; a.dst_kstride = P2l; a.g_kstride = P2l;
            a.g = g; a.g_stride = (long long)dn * P2l;
            a.ut = ut; a.ut_stride = (long long)dn * P2l;
            a.partial = partial;
            a.lamx = M->lamx; a.lamy = M->lamy; a.kx = (float)c->kx; a.ky = (float)c->ky;
            a.dt = dt; a.n0 = n0; a.dn = dn; a.scheme = solve ? SCHEME_SOLVE : sch;
            a.err = M->err;
            // a CTA pair per slice where the slices leave SMs idle, else a pair per two slices (one
            // slice's products run while the other drains); one CTA per slice when pairs are off
            int form = 0;
            if (M->pair_ok && c->fused_pair != 0)
                form = c->fused_pair == 2 ? 1 : c->fused_pair == 3 ? 2 : (2 * batch <= M->nsm ? 1 : 2);
            // pair per slice, chained with a right-hand side: g through a tensor map of its slices
            // (slice b dn + k from g), staged in shared memory ahead of the drain that adds it
            CUtensorMap gm = a1;
            if (form == 1 && g && nchain > 1) {
                SFDE_TRY(map_for(M, g, Py, Px, 1, (long long)(batch - 1) * dn + nchain, &gm));
                a.g_tma = 1;
                a.g_tds = dn;
            }
            if (form)
                SFDE_TRY(sfde_fused_step(c, Px, form, a1, solve ? M->hVTx : M->hWTx, solve ? M->hVTy : M->hWTy,
                                         M->hVx, M->hVy, gm, a, c->stream));
            else
                SFDE_TRY(sfde_fused_step(c, Px, 0, a1, solve ? M->mVTx : M->mWTx, solve ? M->mVTy : M->mWTy,
                                         M->mVx, M->mVy, gm, a, c->stream));
            steps += (long long)batch * nchain;
            if (npart) *npart = batch;
            return SFDE_OK;
        }
        if (nchain != 1) return SFDE_EINVAL;
        int total = 0;
        for (int b0 = 0; b0 < batch; b0 += (int)M->ws) {
            const int nb = std::min<int>(batch - b0, (int)M->ws);
            CUtensorMap a1, a2, a3, a4;
            SFDE_TRY(map_for(M, src, Py, Px, ds, ns, &a1));
            SFDE_TRY(map_for(M, M->T1, Px, Py, 1, (long long)M->ws, &a2));
            SFDE_TRY(map_for(M, M->T2, Py, Px, 1, (long long)M->ws, &a3));
            SFDE_TRY(map_for(M, M->T3, Px, Py, 1, (long long)M->ws, &a4));
            TcArgs p{};
            p.batch = nb; p.err = M->err;
            // G1: (X W_x)^T  or  (X V_x)^T
            p.R = Py; p.C = Px; p.Cout = Px; p.BN = sfde_tc_tile_n(Px); p.s0 = src0 + b0 * ds; p.ds = ds;
            p.out = M->T1; p.out_stride = P2l;
            SFDE_TRY(sfde_tc_gemm(c, M->kind, TC_EPI_STORE, a1, solve ? M->gVTx : M->gWTx, p, c->stream, c->y.n, c->x.n, c->x.n, M->kind == 2 ? (solve ? &M->oVTx : &M->oWTx) : nullptr));
            // G2: modal scaling
            TcArgs q{};
            q.batch = nb; q.err = M->err;
            q.R = Px; q.C = Py; q.Cout = Py; q.BN = sfde_tc_tile_n(Py); q.s0 = 0; q.ds = 1;
            q.out = M->T2; q.out_stride = P2l;
            q.e.lamx = M->lamx; q.e.lamy = M->lamy; q.e.kx = (float)c->kx; q.e.ky = (float)c->ky;
            q.e.dt = dt; q.e.n0 = n0 + b0 * dn; q.e.dn = dn; q.e.scheme = solve ? SCHEME_SOLVE : sch;
            SFDE_TRY(sfde_tc_gemm(c, M->kind, TC_EPI_SCALE, a2, solve ? M->gVTy : M->gWTy, q, c->stream, c->x.n, c->y.n, c->y.n, M->kind == 2 ? (solve ? &M->oVTy : &M->oWTy) : nullptr));
            // G3: (C V_x^T)^T
            TcArgs r{};
            r.batch = nb; r.err = M->err;
            r.R = Py; r.C = Px; r.Cout = Px; r.BN = sfde_tc_tile_n(Px); r.s0 = 0; r.ds = 1;
            r.out = M->T3; r.out_stride = P2l;
            SFDE_TRY(sfde_tc_gemm(c, M->kind, TC_EPI_STORE, a3, M->gVx, r, c->stream, c->y.n, c->x.n, c->x.n, M->kind == 2 ? &M->oVx : nullptr));
            // G4: (T3 V_y^T)^T + g - u_target
            TcArgs f{};
            f.batch = nb; f.err = M->err;
            f.R = Px; f.C = Py; f.Cout = Py; f.BN = sfde_tc_tile_n(Py); f.s0 = 0; f.ds = 1;
            f.out = slice(dst, 0) + (size_t)b0 * dst_ds * P2() * M->esz; f.out_stride = (long long)dst_ds * P2l;
            f.e.g = g ? (const void*)((const char*)g + (size_t)b0 * dn * P2() * M->esz) : nullptr;
            f.e.g_stride = (long long)dn * P2l;
            f.e.utgt = ut ? (const void*)((const char*)ut + (size_t)b0 * dn * P2() * M->esz) : nullptr;
            f.e.utgt_stride = (long long)dn * P2l;
            // sfde_tc_partials_per_tile() partial sums (one per epilogue warp) per output tile
            const int gx = (int)(((long long)nb * Px + 127) / 128), gy = Py / f.BN;
            const int ppt = sfde_tc_partials_per_tile();
            if (partial && (size_t)(total + ppt * gx * gy) > c->partial_cap) return SFDE_EINVAL;
            f.e.partial = partial ? partial + total : nullptr;
            SFDE_TRY(sfde_tc_gemm(c, M->kind, TC_EPI_FINAL, a4, M->gVy, f, c->stream, c->x.n, c->y.n, c->y.n, M->kind == 2 ? &M->oVy : nullptr));
            total += ppt * gx * gy;
        }
        steps += batch;
        if (npart) *npart = total;
        return SFDE_OK;
    }

    // W_y^T X_b W_x for the slices src0 + b ds (b < batch) of `src` (a buffer of ns slices) -> slice
    // b dst_ds of dst: two slice GEMMs through T1, no modal factor
    sfde_status to_modal(const void* src, long long ns, int src0, int ds, int batch, void* dst, int dst_ds) {
        const int Px = c->x.P, Py = c->y.P;
        const long long P2l = (long long)P2();
        for (int b0 = 0; b0 < batch; b0 += (int)M->ws) {
            const int nb = std::min<int>(batch - b0, (int)M->ws);
            CUtensorMap a1, a2;
            SFDE_TRY(map_for(M, src, Py, Px, ds, ns, &a1));
            SFDE_TRY(map_for(M, M->T1, Px, Py, 1, (long long)M->ws, &a2));
            TcArgs p{};   // (X W_x)^T
            p.batch = nb; p.err = M->err;
            p.R = Py; p.C = Px; p.Cout = Px; p.BN = sfde_tc_tile_n(Px); p.s0 = src0 + b0 * ds; p.ds = ds;
            p.out = M->T1; p.out_stride = P2l;
            SFDE_TRY(sfde_tc_gemm(c, M->kind, TC_EPI_STORE, a1, M->gWTx, p, c->stream, c->y.n, c->x.n, c->x.n, M->kind == 2 ? &M->oWTx : nullptr));
            TcArgs q{};   // (T1 W_y)^T = W_y^T X W_x
            q.batch = nb; q.err = M->err;
            q.R = Px; q.C = Py; q.Cout = Py; q.BN = sfde_tc_tile_n(Py); q.s0 = 0; q.ds = 1;
            q.out = slice(dst, (long long)b0 * dst_ds); q.out_stride = (long long)dst_ds * P2l;
            SFDE_TRY(sfde_tc_gemm(c, M->kind, TC_EPI_STORE, a2, M->gWTy, q, c->stream, c->x.n, c->y.n, c->y.n, M->kind == 2 ? &M->oWTy : nullptr));
        }
        return SFDE_OK;
    }

    // In place, slices n0 .. n0 + batch - 1 of `buf` (ns slices): X -> (V_y^T X V_x) / (1 + tau_n sigma),
    // the right-hand side of S_n^{-1} X in the step's eigenbasis (the first two products of a solve)
    sfde_status to_modal_solve(void* buf, long long ns, int n0, int batch) {
        const int Px = c->x.P, Py = c->y.P;
        const long long P2l = (long long)P2();
        for (int b0 = 0; b0 < batch; b0 += (int)M->ws) {
            const int nb = std::min<int>(batch - b0, (int)M->ws);
            CUtensorMap a1, a2;
            SFDE_TRY(map_for(M, buf, Py, Px, 1, ns, &a1));
            SFDE_TRY(map_for(M, M->T1, Px, Py, 1, (long long)M->ws, &a2));
            TcArgs p{};   // (X V_x)^T
            p.batch = nb; p.err = M->err;
            p.R = Py; p.C = Px; p.Cout = Px; p.BN = sfde_tc_tile_n(Px); p.s0 = n0 + b0; p.ds = 1;
            p.out = M->T1; p.out_stride = P2l;
            SFDE_TRY(sfde_tc_gemm(c, M->kind, TC_EPI_STORE, a1, M->gVTx, p, c->stream, c->y.n, c->x.n, c->x.n,
                                  M->kind == 2 ? &M->oVTx : nullptr));
            TcArgs q{};   // (T1 V_y)^T = V_y^T X V_x, scaled by 1 / (1 + tau_n sigma)
            q.batch = nb; q.err = M->err;
            q.R = Px; q.C = Py; q.Cout = Py; q.BN = sfde_tc_tile_n(Py); q.s0 = 0; q.ds = 1;
            q.out = slice(buf, (long long)n0 + b0); q.out_stride = P2l;
            q.e.lamx = M->lamx; q.e.lamy = M->lamy; q.e.kx = (float)c->kx; q.e.ky = (float)c->ky;
            q.e.dt = c->dt0; q.e.n0 = n0 + b0; q.e.dn = 1; q.e.scheme = SCHEME_SOLVE;
            SFDE_TRY(sfde_tc_gemm(c, M->kind, TC_EPI_SCALE, a2, M->gVTy, q, c->stream, c->x.n, c->y.n, c->y.n,
                                  M->kind == 2 ? &M->oVTy : nullptr));
        }
        return SFDE_OK;
    }

    // k_modal_run over `groups` runs of `len` points (all arrays FP32 slices of the level)
    sfde_status modal_run(const void* U, long long ucs, const void* G, long long gis, long long gj0, void* Y,
                          long long yis, long long yj0, int len, int groups, const double* dt, long long dis,
                          int sch) {
        const size_t P2s = P2();
        dim3 grid((unsigned)((P2s / 4 + 255) / 256), (unsigned)groups);
        k_modal_run<<<grid, 256, 0, c->stream>>>((const float*)U, ucs, (const float*)G, gis, gj0, (float*)Y, yis, yj0,
                                                 len, c->x.P, P2s, M->lamx, M->lamy, (float)c->kx, (float)c->ky, dt,
                                                 dis, sch);
        sfde_count_launch(c);
        SFDE_CUDA(cudaGetLastError());
        return SFDE_OK;
    }

    // V_y Y_b V_x^T for the slices b < batch of `src` (ns slices) -> slice b of dst, or with oskip > 0
    // the b-th F-point, slice b + b / oskip + 1 (intervals of oskip + 1 points): two slice GEMMs
    // through T3, in chunks of whole intervals
    sfde_status from_modal(const void* src, long long ns, int batch, void* dst, int oskip) {
        const int Px = c->x.P, Py = c->y.P;
        const long long P2l = (long long)P2();
        const int chunk = oskip > 0 ? std::max(oskip, ((int)M->ws / oskip) * oskip) : (int)M->ws;
        if (chunk > (int)M->ws) return SFDE_EINVAL;
        for (int b0 = 0; b0 < batch; b0 += chunk) {
            const int nb = std::min(batch - b0, chunk);
            CUtensorMap a3, a4;
            SFDE_TRY(map_for(M, src, Py, Px, 1, ns, &a3));
            SFDE_TRY(map_for(M, M->T3, Px, Py, 1, (long long)M->ws, &a4));
            TcArgs r{};   // (Y V_x^T)^T
            r.batch = nb; r.err = M->err;
            r.R = Py; r.C = Px; r.Cout = Px; r.BN = sfde_tc_tile_n(Px); r.s0 = b0; r.ds = 1;
            r.out = M->T3; r.out_stride = P2l;
            SFDE_TRY(sfde_tc_gemm(c, M->kind, TC_EPI_STORE, a3, M->gVx, r, c->stream, c->y.n, c->x.n, c->x.n, M->kind == 2 ? &M->oVx : nullptr));
            TcArgs f{};   // (T3 V_y^T)^T = V_y Y V_x^T
            f.batch = nb; f.err = M->err;
            f.R = Px; f.C = Py; f.Cout = Py; f.BN = sfde_tc_tile_n(Py); f.s0 = 0; f.ds = 1;
            f.out = slice(dst, oskip > 0 ? (long long)b0 + b0 / oskip : (long long)b0);
            f.out_stride = P2l;
            f.oskip = oskip;
            SFDE_TRY(sfde_tc_gemm(c, M->kind, TC_EPI_STORE, a4, M->gVy, f, c->stream, c->x.n, c->y.n, c->y.n, M->kind == 2 ? &M->oVy : nullptr));
        }
        return SFDE_OK;
    }

    // Y[i (len - 1) + j - 1] = v_j of the eigenbasis recurrence over `nint` intervals (k_modal_scan)
    sfde_status modal_scan(const void* Uc, const void* G, int gis, int gj0, void* Y, int len, int nint,
                           const double* dt, int dis, int sch) {
        const size_t P2s = P2();
        dim3 grid((unsigned)((P2s / 4 + 255) / 256), (unsigned)nint);
        if (M->kind == 0)
            k_modal_scan<__nv_bfloat16><<<grid, 256, 0, c->stream>>>(
                (const __nv_bfloat16*)Uc, (const __nv_bfloat16*)G, gis, gj0, (__nv_bfloat16*)Y, len, c->x.P, P2s, M->lamx,
                M->lamy, (float)c->kx, (float)c->ky, dt, dis, sch);
        else if (M->kind == 1)
            k_modal_scan<float><<<grid, 256, 0, c->stream>>>((const float*)Uc, (const float*)G, gis, gj0, (float*)Y, len,
                                                             c->x.P, P2s, M->lamx, M->lamy, (float)c->kx,
                                                             (float)c->ky, dt, dis, sch);
        else
            k_modal_scan<F32><<<grid, 256, 0, c->stream>>>((const F32*)Uc, (const F32*)G, gis, gj0, (F32*)Y, len, c->x.P,
                                                           P2s, M->lamx, M->lamy, (float)c->kx, (float)c->ky, dt, dis,
                                                           sch);
        sfde_count_launch(c);
        SFDE_CUDA(cudaGetLastError());
        return SFDE_OK;
    }

    // coarse levels sweep in the eigenbasis (F-relaxation, coarsest solve)
    bool modal(int l) const { return c->modal_chains && (l >= 1 || M->modal_fine) && M->lev[l].gm && M->mY; }

    sfde_status lstep(int l, int batch, int src0, int ds, int n0, int dn, void* dst, int dst_ds,
                      const void* ut, double* partial, int* npart) {
        LpLevel& Lv = M->lev[l];
        return step(Lv.u, Lv.nalloc, src0, ds, batch, false, l == 0 ? SCHEME_CN : scheme, Lv.dt, n0, dn,
                    dst, dst_ds, slice(Lv.g, n0), ut, partial, npart);
    }

    // F-relaxation: u_{im+j} = Phi(u_{im+j-1}) + g_{im+j}, j = 1..m-1, all intervals i at once; the
    // fused kernel runs the m-1 steps of an interval in one CTA, each step starting from the last
    sfde_status frelax(int l) {
        LpLevel& Lv = M->lev[l];
        const int nc = Lv.N / m;
        if (full) {   // every interval's F-points from its C-point, in place, per mode
            steps += (long long)nc * (m - 1);
            return modal_run(Lv.u, m, Lv.g, m, 0, Lv.u, m, 0, m, nc, Lv.dt, m, l == 0 ? SCHEME_CN : scheme);
        }
        // (the C-point transforms go to T2, ws slices: more intervals than that keep chained steps)
        if (modal(l) && nc <= (int)M->ws && m - 1 <= (int)M->ws) {
            // C-point values transformed (T2), the interval recurrences, all F-points transformed back
            SFDE_TRY(to_modal(Lv.u, Lv.nalloc, 0, m, nc, M->T2, 1));
            SFDE_TRY(modal_scan(M->T2, Lv.gm, m, 0, M->mY, m, nc, Lv.dt, m, l == 0 ? SCHEME_CN : scheme));
            SFDE_TRY(from_modal(M->mY, (long long)nc * (m - 1), nc * (m - 1), Lv.u, m - 1));
            steps += (long long)nc * (m - 1);
            return SFDE_OK;
        }
        if (M->fused)
            return step(Lv.u, Lv.nalloc, 0, m, nc, false, l == 0 ? SCHEME_CN : scheme, Lv.dt, 1, m, slice(Lv.u, 1), m,
                        slice(Lv.g, 1), nullptr, nullptr, nullptr, m - 1);
        for (int j = 1; j < m; ++j)
            SFDE_TRY(lstep(l, nc, j - 1, m, j, m, slice(Lv.u, j), m, nullptr, nullptr, nullptr));
        return SFDE_OK;
    }

    sfde_status crelax(int l) {
        LpLevel& Lv = M->lev[l];
        if (full) {   // u_{(k+1)m} from u_{(k+1)m-1}: runs of two points starting at the last F-points
            steps += Lv.N / m;
            return modal_run(slice(Lv.u, m - 1), m, slice(Lv.g, m - 1), m, 0, slice(Lv.u, m - 1), m, 0, 2, Lv.N / m,
                             Lv.dt + (m - 1), m, l == 0 ? SCHEME_CN : scheme);
        }
        return lstep(l, Lv.N / m, m - 1, m, m, m, slice(Lv.u, m), m, nullptr, nullptr, nullptr);
    }

    sfde_status relaxation(int l) {
        SFDE_TRY(frelax(l));
        if (relax == SFDE_RELAX_FCF) {
            SFDE_TRY(crelax(l));
            SFDE_TRY(frelax(l));
        }
        return SFDE_OK;
    }

    sfde_status residual(int l, double* partial, int* npart) {
        LpLevel& Lv = M->lev[l];
        LpLevel& Cv = M->lev[l + 1];
        if (M->kind == 0)
            k_lp_diff<__nv_bfloat16><<<grid_for(P2()), 256, 0, c->stream>>>((__nv_bfloat16*)Cv.g, (const __nv_bfloat16*)Lv.g, (const __nv_bfloat16*)Lv.u, P2());
        else if (M->kind == 1)
            k_lp_diff<float><<<grid_for(P2()), 256, 0, c->stream>>>((float*)Cv.g, (const float*)Lv.g, (const float*)Lv.u, P2());
        else
            k_lp_diff<F32><<<grid_for(P2()), 256, 0, c->stream>>>((F32*)Cv.g, (const F32*)Lv.g, (const F32*)Lv.u, P2());
        sfde_count_launch(c);
        if (full) {
            if (partial) return SFDE_EINVAL;   // the inner solve takes no norm
            const size_t P2s = P2();
            dim3 grid((unsigned)((P2s / 4 + 255) / 256), (unsigned)(Lv.N / m));
            k_modal_resid<<<grid, 256, 0, c->stream>>>((const float*)Lv.u, (const float*)Lv.g, (float*)slice(Cv.g, 1), m,
                                                       c->x.P, P2s, M->lamx, M->lamy, (float)c->kx, (float)c->ky,
                                                       Lv.dt, l == 0 ? SCHEME_CN : scheme);
            sfde_count_launch(c);
            steps += Lv.N / m;
            if (npart) *npart = 0;
            SFDE_CUDA(cudaGetLastError());
            return SFDE_OK;
        }
        return lstep(l, Lv.N / m, m - 1, m, m, m, slice(Cv.g, 1), 1, slice(Lv.u, m), partial, npart);
    }

    sfde_status coarsest(int l) {
        LpLevel& Lv = M->lev[l];
        SFDE_CUDA(cudaMemcpyAsync(Lv.u, Lv.g, P2() * M->esz, cudaMemcpyDeviceToDevice, c->stream));
        if (full) {   // u_n = f_n u_{n-1} + g_n, n = 1..N, one run from u_0 = g_0
            steps += Lv.N;
            return modal_run(Lv.g, 0, Lv.g, 0, 0, Lv.u, 0, 0, Lv.N + 1, 1, Lv.dt, 0, l == 0 ? SCHEME_CN : scheme);
        }
        // u_n = Phi(u_{n-1}) + g_n, n = 1..N: one recurrence per mode in the eigenbasis (u_0 = g_0,
        // so its transform is the first transformed right-hand side), or the fused kernel chaining
        // all N steps in one launch
        if (modal(l)) {
            SFDE_TRY(modal_scan(Lv.gm, Lv.gm, Lv.N + 1, 0, M->mY, Lv.N + 1, 1, Lv.dt, Lv.N + 1,
                                l == 0 ? SCHEME_CN : scheme));
            SFDE_TRY(from_modal(M->mY, Lv.N, Lv.N, slice(Lv.u, 1), 0));   // v_j -> u_j, j = 1..N
            steps += Lv.N;
            return SFDE_OK;
        }
        if (M->fused)
            return step(Lv.u, Lv.nalloc, 0, 1, 1, false, l == 0 ? SCHEME_CN : scheme, Lv.dt, 1, 1, slice(Lv.u, 1), 1,
                        slice(Lv.g, 1), nullptr, nullptr, nullptr, Lv.N);
        for (int n = 1; n <= Lv.N; ++n)
            SFDE_TRY(lstep(l, 1, n - 1, 1, n, 1, slice(Lv.u, n), 1, nullptr, nullptr, nullptr));
        return SFDE_OK;
    }

    sfde_status correct(int l) {
        LpLevel& Lv = M->lev[l];
        LpLevel& Cv = M->lev[l + 1];
        dim3 grid(grid_for(P2()) < 64 ? grid_for(P2()) : 64, Cv.N + 1);
        if (M->kind == 0)
            k_lp_axpy_strided<__nv_bfloat16><<<grid, 256, 0, c->stream>>>((__nv_bfloat16*)Lv.u, (long long)m * P2(), (const __nv_bfloat16*)Cv.u, (long long)P2(), P2());
        else if (M->kind == 1 && !full)   // nodal values feed TF32 products: rounded; modal values stay FP32
            k_lp_axpy_strided<float><<<grid, 256, 0, c->stream>>>((float*)Lv.u, (long long)m * P2(), (const float*)Cv.u, (long long)P2(), P2());
        else
            k_lp_axpy_strided<F32><<<grid, 256, 0, c->stream>>>((F32*)Lv.u, (long long)m * P2(), (const F32*)Cv.u, (long long)P2(), P2());
        sfde_count_launch(c);
        SFDE_CUDA(cudaGetLastError());
        return SFDE_OK;
    }

    sfde_status solve(int l) {
        // the level's right-hand sides stay fixed while it is visited: transformed once
        if (!full && modal(l))
            SFDE_TRY(to_modal(M->lev[l].g, M->lev[l].nalloc, 0, 1, M->lev[l].N + 1, M->lev[l].gm, 1));
        if (l == L - 1) return coarsest(l);
        if (!skip) SFDE_TRY(relaxation(l));
        SFDE_TRY(residual(l, nullptr, nullptr));
        SFDE_CUDA(cudaMemsetAsync(M->lev[l + 1].u, 0, P2() * M->esz * (M->lev[l + 1].N + 1), c->stream));
        SFDE_TRY(solve(l + 1));
        SFDE_TRY(correct(l));
        return frelax(l);
    }
};

// Steps 2-4 of one outer iteration, queued on c->stream without any host synchronisation, in
// parts: (0) g_n = S_n^{-1} rho_n (rho already in g_0[1..N]) and E = 0; (1) one V-cycle on
// E_n = Psi_n E_{n-1} + g_n up to the C-point correction; (2) the relaxation of the last V-cycle (so
// E is F-consistent; the sequential solve when there is one level) and U += E in FP64; (3) part 1
// without relaxation on the down-cycle (the first V-cycle under skip_first_down: E = 0, so the
// coarse right-hand sides are the injected g).  K V-cycles are part 0, K-1 times part 1 (the first
// of them part 3 with skip_first_down), part 2.
sfde_status enqueue_inner_part(sfde_ctx* c, SfdeMixed* M, LpEngine& E, double* U, int kind, int part) {
    LpLevel& L0 = M->lev[0];
    const size_t P2 = c->P2();
    if (part == 0) {
        SFDE_CUDA(cudaMemsetAsync(L0.g, 0, P2 * M->esz, c->stream));
        if (E.full) {   // g^_n = (V_y^T rho_n V_x) / (1 + tau_n sigma): the solve, left in the eigenbasis
            SFDE_TRY(E.to_modal_solve(L0.g, L0.nalloc, 1, c->nt));
            SFDE_CUDA(cudaMemsetAsync(L0.u, 0, P2 * M->esz * L0.nalloc, c->stream));
            return SFDE_OK;
        }
        SFDE_TRY(E.step(L0.g, L0.nalloc, 1, 1, c->nt, true, SCHEME_SOLVE, c->dt0, 1, 1, E.slice(L0.g, 1), 1,
                        nullptr, nullptr, nullptr, nullptr));
        SFDE_CUDA(cudaMemsetAsync(L0.u, 0, P2 * M->esz * L0.nalloc, c->stream));
        // fixed for all V-cycles of this refinement step: transformed once
        if (E.modal(0)) SFDE_TRY(E.to_modal(L0.g, L0.nalloc, 0, 1, L0.N + 1, L0.gm, 1));
        return SFDE_OK;
    }
    if (part == 1 || part == 3) {
        E.skip = part == 3;
        sfde_status st = E.skip ? SFDE_OK : E.relaxation(0);
        if (st == SFDE_OK) st = E.residual(0, nullptr, nullptr);
        if (st == SFDE_OK && cudaMemsetAsync(M->lev[1].u, 0, P2 * M->esz * (M->lev[1].N + 1), c->stream) != cudaSuccess)
            st = SFDE_ECUDA;
        if (st == SFDE_OK) st = E.solve(1);
        E.skip = false;
        SFDE_TRY(st);
        return E.correct(0);
    }
    if (E.L == 1) SFDE_TRY(E.coarsest(0));
    else SFDE_TRY(E.relaxation(0));
    const size_t n = P2 * (size_t)c->nt;
    // with the inner solve in the eigenbasis, E_n = V_y e^_n V_x^T into g_0 (no longer needed)
    const void* Ev = E.slice(L0.u, 1);
    if (E.full) {
        SFDE_TRY(E.from_modal(E.slice(L0.u, 1), L0.nalloc - 1, c->nt, E.slice(L0.g, 1), 0));
        Ev = E.slice(L0.g, 1);
    }
    if (kind == 0)
        k_add_correction<__nv_bfloat16><<<grid_for(n), 256, 0, c->stream>>>(U + P2, (const __nv_bfloat16*)Ev, n);
    else   // FP32 storage (kinds 1 and 2) read as FP32
        k_add_correction<float><<<grid_for(n), 256, 0, c->stream>>>(U + P2, (const float*)Ev, n);
    sfde_count_launch(c);
    SFDE_CUDA(cudaGetLastError());
    return SFDE_OK;
}

// Capture part `part` of the inner solve as a CUDA graph (once per configuration).
sfde_status capture_inner_part(sfde_ctx* c, SfdeMixed* M, LpEngine& E, double* U, int kind, int part) {
    if (!M->cap) SFDE_CUDA(cudaStreamCreateWithFlags(&M->cap, cudaStreamNonBlocking));
    cudaStream_t user = c->stream;
    const long long before = c->prof.launches, steps_before = E.steps;
    SFDE_CUDA(cudaStreamBeginCapture(M->cap, cudaStreamCaptureModeThreadLocal));
    c->stream = M->cap;
    const sfde_status cs = enqueue_inner_part(c, M, E, U, kind, part);
    c->stream = user;
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(M->cap, &graph);
    if (cs != SFDE_OK) { if (graph) cudaGraphDestroy(graph); return cs; }
    SFDE_CUDA(ce);
    const cudaError_t ie = cudaGraphInstantiate(&M->inner_exec[part], graph, 0);
    cudaGraphDestroy(graph);
    SFDE_CUDA(ie);
    M->inner_launches[part] = c->prof.launches - before;
    M->inner_steps[part] = E.steps - steps_before;
    c->prof.launches = before;
    E.steps = steps_before;
    return SFDE_OK;
}

sfde_status check_err(SfdeMixed* M, cudaStream_t s) {
    int h = 0;
    SFDE_CUDA(cudaMemcpyAsync(&h, M->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    SFDE_CUDA(cudaStreamSynchronize(s));
    return h ? SFDE_ETIMEOUT : SFDE_OK;
}

}  // namespace

sfde_status sfde_mgrit_mixed(sfde_ctx* c, const mgrit_opts* o, mgrit_stats* st) {
    const int kind = sfde_mixed_kind(c);
    SFDE_TRY(setup_mixed(c, kind, o->m, o->max_levels, o->min_coarse));
    SfdeMixed* M = c->mixed;
    M->fused = c->fused_step && sfde_fused_supported(kind, c->x.P, c->y.P);
    const int L = (int)M->lev.size();
    double* U = nullptr;
    SFDE_TRY(sfde_level0(c, &U));
    const size_t P2 = c->P2();
    int coarse = SFDE_COARSE_BE;
    double tub = 0.0;
    SFDE_TRY(sfde_choose_coarse(c, o->m, o->coarse, &coarse, &tub));
    LpEngine E{c, M, o->m, L, o->relax, coarse == SFDE_COARSE_CN ? SCHEME_CN : SCHEME_BE};
    E.full = c->modal_chains == 4 && kind != 0;   // BF16 storage keeps the nodal levels
    // inner V-cycles per refinement step: enough for the inner error to reach the low-precision
    // floor (about 2e-2 BF16, 3e-3 TF32) at MGRIT contraction ~0.3 per V-cycle; with FP32 products
    // the floor is far lower and 3 V-cycles set the contraction.  (Raising K when the
    // refinement contracts slowly does not help: there the floor itself is high -- rounding
    // accumulated over long stiff runs -- and more V-cycles only add time.)
    const int K = o->inner_cycles > 0 ? o->inner_cycles
                : c->inner_cycles_tuned > 0 ? c->inner_cycles_tuned : (kind == 0 ? 4 : kind == 1 ? 5 : 3);
    // the inner solve is captured once as CUDA graphs and replayed; eager while kernels are timed
    const bool use_graph = !c->prof.on;
    const long long key = ((long long)o->skip_first_down << 32) | ((long long)c->modal_chains << 28) |
                          ((long long)c->fused_pair << 24) | ((long long)M->fused << 20) | ((long long)E.scheme << 4) |
                          (long long)o->relax;
    long long graph_steps = 0;

    mgrit_stats S{};
    S.levels = L;
    S.coarse_used = coarse;
    S.tub = tub;
    S.lp_kind = kind;
    SFDE_CUDA(cudaEventRecord(c->ev0, c->stream));
    SFDE_CUDA(cudaMemcpyAsync(U, c->U0, sizeof(double) * P2, cudaMemcpyDeviceToDevice, c->stream));
    if (o->init_seed) {
        sfde_launch_fill_random(U, c->nt, c->y.n, c->x.n, c->y.P, c->x.P, o->init_seed, c->stream);
        sfde_count_launch(c);
    } else {
        SFDE_CUDA(cudaMemsetAsync(U + P2, 0, sizeof(double) * P2 * c->nt, c->stream));
    }
    LpLevel& L0 = M->lev[0];
    sfde_status rc = SFDE_OK;
    long long inner_total = 0;
    // digits of the tensor-core residual per refinement step (residual_digits_for); a residual that
    // passes the stopping test with fewer than 7 digits is recomputed with all 7
    double prev_nrm = 0.0;
    long long digit_products = 0;
    for (int it = 1; it <= o->max_iter; ++it) {
        // 1. FP64 residual of Eq. (2.4) at n = 1..N_t, stored low precision in g_0[n]
        int nd = c->resid_digits ? c->resid_digits : residual_digits_for(it == 1 ? 0.0 : prev_nrm, S.res0);
        double nrm = 0.0;
        for (;;) {
            int np = 0;
            if (M->use_oz) {
                // the first iterate is psi_0 followed by zeros (unless drawn at random): from the pair
                // (U_1, U_2) on, the residual is the load alone
                SFDE_TRY(sfde_residual_int(c, U, 1, c->nt, E.slice(L0.g, 1), (long long)P2, kind, c->partial, &np,
                                           M->oAx, M->oAy, M->oz_dV, M->oz_dVt, M->oz_E, M->err, nd,
                                           it == 1 && !o->init_seed ? 2 : INT_MAX));
                digit_products += nd * (nd + 1) / 2;
            } else {
                SFDE_TRY(sfde_residual_fp64(c, U, 1, c->nt, E.slice(L0.g, 1), (long long)P2, kind, c->partial, &np));
                nd = 7;
            }
            double r2 = 0.0;
            SFDE_TRY(sfde_reduce_partials(c, np, &r2));
            SFDE_TRY(check_err(M, c->stream));
            nrm = sqrt(r2);
            const double res0 = it == 1 ? nrm : S.res0;
            if (nd == 7 || !(nrm <= std::max(o->rel_tol * res0, o->abs_tol))) break;
            nd = 7;   // apparently converged: confirm with exact operands
        }
        prev_nrm = nrm;
        if (it - 1 < SFDE_HISTORY_MAX) S.history[it - 1] = nrm;
        if (it == 1) S.res0 = nrm;
        S.res_final = nrm;
        S.iters = it;
        if (!isfinite(nrm)) { rc = SFDE_ENOCONV; break; }
        if (nrm <= std::max(o->rel_tol * S.res0, o->abs_tol)) { S.converged = 1; break; }
        // 2-4: correction right-hand side, inner V-cycles, U += E (no host synchronisation inside)
        const int Kr = L == 1 ? 1 : K;
        if (use_graph) {
            if (M->inner_key != key) {
                for (auto& g : M->inner_exec)
                    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
                for (int part = 0; part < 4; ++part)
                    if ((part != 1 || L > 1) && (part != 3 || (L > 1 && o->skip_first_down)))
                        SFDE_TRY(capture_inner_part(c, M, E, U, kind, part));
                M->inner_key = key;
            }
            for (int r = 0; r < Kr + 1; ++r) {
                const int part = r == 0 ? 0 : (r == Kr ? 2 : (r == 1 && o->skip_first_down ? 3 : 1));
                SFDE_CUDA(cudaGraphLaunch(M->inner_exec[part], c->stream));
                sfde_count_launch(c, (int)M->inner_launches[part]);
                graph_steps += M->inner_steps[part];
            }
        } else {
            SFDE_TRY(enqueue_inner_part(c, M, E, U, kind, 0));
            for (int k = 1; k < Kr; ++k)
                SFDE_TRY(enqueue_inner_part(c, M, E, U, kind, k == 1 && o->skip_first_down ? 3 : 1));
            SFDE_TRY(enqueue_inner_part(c, M, E, U, kind, 2));
        }
        inner_total += Kr;
    }
    E.steps += graph_steps;
    if (!S.converged && rc == SFDE_OK) rc = SFDE_ENOCONV;
    SFDE_CUDA(cudaEventRecord(c->ev1, c->stream));
    SFDE_CUDA(cudaEventSynchronize(c->ev1));
    SFDE_TRY(check_err(M, c->stream));
    float ms = 0.f;
    SFDE_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    S.seconds = ms * 1e-3;
    S.step_solves = E.steps;
    S.inner_vcycles = inner_total;
    const int nh = std::min(S.iters, SFDE_HISTORY_MAX);
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

// ---- verification hooks (sfde_debug.h)

namespace {
template <typename T>
__global__ void k_lp_to_f64(const T* src, double* dst, size_t n) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        dst[e] = (double)lp_f(src[e]);
}

// unpadded FP64 slices (host or device) -> padded low-precision device slices
sfde_status load_lp(sfde_ctx* c, const double* in, int batch, double* tmp_unp, double* tmp_pad, void* out, int kind) {
    const size_t n2 = (size_t)c->x.n * c->y.n, P2 = c->P2();
    SFDE_TRY(sfde_copy_in(tmp_unp, in, sizeof(double) * n2 * batch, c->stream));
    SFDE_CUDA(cudaMemsetAsync(tmp_pad, 0, sizeof(double) * P2 * batch, c->stream));
    sfde_launch_pad(tmp_unp, tmp_pad, c->y.n, c->x.n, c->y.P, c->x.P, batch, c->stream);
    const size_t n = P2 * batch;
    if (kind == 0) k_to_lp<__nv_bfloat16><<<grid_for(n), 256, 0, c->stream>>>(tmp_pad, (__nv_bfloat16*)out, n);
    else if (kind == 1) k_to_lp<float><<<grid_for(n), 256, 0, c->stream>>>(tmp_pad, (float*)out, n);
    else k_to_lp<F32><<<grid_for(n), 256, 0, c->stream>>>(tmp_pad, (F32*)out, n);
    SFDE_CUDA(cudaGetLastError());
    return SFDE_OK;
}
}  // namespace

extern "C" sfde_status sfde_debug_set_residual_digits(sfde_ctx* c, int nd) {
    if (!c || (nd != 0 && (nd < 4 || nd > 7))) return SFDE_EINVAL;
    c->resid_digits = nd;
    return SFDE_OK;
}

extern "C" sfde_status sfde_debug_set_fused_step(sfde_ctx* c, int enable) {
    if (!c) return SFDE_EINVAL;
    c->fused_step = enable ? 1 : 0;
    return SFDE_OK;
}

extern "C" sfde_status sfde_debug_set_resid_chunk(sfde_ctx* c, int n) {
    if (!c || n < 0) return SFDE_EINVAL;
    c->resid_chunk = n;
    return SFDE_OK;
}

extern "C" sfde_status sfde_debug_set_fused_pair(sfde_ctx* c, int mode) {
    if (!c || mode < 0 || mode > 3) return SFDE_EINVAL;
    c->fused_pair = mode;
    return SFDE_OK;
}

extern "C" sfde_status sfde_debug_inner_levels(int nt, int m, int max_levels, int min_coarse, int* sizes, int cap,
                                              int* count) {
    if (nt < 1 || m < 2 || max_levels < 1 || min_coarse < 1 || cap < 0 || !count || (cap > 0 && !sizes))
        return SFDE_EINVAL;
    return sfde_no_throw([&] {
        const std::vector<int> n = inner_level_sizes(nt, m, max_levels, min_coarse);
        *count = (int)n.size();
        for (int l = 0; l < std::min(cap, (int)n.size()); ++l) sizes[l] = n[l];
        return SFDE_OK;
    });
}

extern "C" sfde_status sfde_debug_residual_digits(double prev, double res0, int* nd) {
    if (!nd) return SFDE_EINVAL;
    *nd = residual_digits_for(prev, res0);
    return SFDE_OK;
}

extern "C" sfde_status sfde_debug_set_modal_chains(sfde_ctx* c, int enable) {
    if (!c || enable < 0 || enable > 4) return SFDE_EINVAL;
    c->modal_chains = enable;
    return SFDE_OK;
}

extern "C" sfde_status sfde_debug_lp_step(sfde_ctx* c, int fused, int scheme, const double* U, int batch, int n0,
                                         const double* g, const double* ut, double* out, double* norm2) {
    if (!c || !U || !out || batch < 1 || n0 < 1 || (long long)n0 + batch - 1 > c->nt || scheme < 0 || scheme > 2)
        return SFDE_EINVAL;
    if (c->precision == SFDE_PREC_FP64) return SFDE_EINVAL;
    const int kind = sfde_mixed_kind(c);
    if (fused && !sfde_fused_supported(kind, c->x.P, c->y.P)) return SFDE_EUNSUPPORTED;
    if (!c->mixed || c->mixed->kind != kind) SFDE_TRY(setup_mixed(c, kind, 2, 1, 1));
    SfdeMixed* M = c->mixed;
    const size_t P2 = c->P2(), n2 = (size_t)c->x.n * c->y.n, lp = P2 * M->esz * batch;
    double *tu = nullptr, *tp = nullptr;
    void *src = nullptr, *dst = nullptr, *dg = nullptr, *du = nullptr;
    sfde_status st = SFDE_OK;
    const bool saved = M->fused;
    M->fused = fused != 0;
    if (cudaMalloc(&tu, sizeof(double) * n2 * batch) != cudaSuccess ||
        cudaMalloc(&tp, sizeof(double) * P2 * batch) != cudaSuccess || cudaMalloc(&src, lp) != cudaSuccess ||
        cudaMalloc(&dst, lp) != cudaSuccess || cudaMalloc(&dg, lp) != cudaSuccess || cudaMalloc(&du, lp) != cudaSuccess)
        st = SFDE_ENOMEM;
    if (st == SFDE_OK) st = load_lp(c, U, batch, tu, tp, src, kind);
    if (st == SFDE_OK && g) st = load_lp(c, g, batch, tu, tp, dg, kind);
    if (st == SFDE_OK && ut) st = load_lp(c, ut, batch, tu, tp, du, kind);
    if (st == SFDE_OK) {
        LpEngine E{c, M, 2, 1, SFDE_RELAX_FCF, SCHEME_CN};
        int np = 0;
        const int sch = scheme == 0 ? (int)SCHEME_CN : (scheme == 1 ? (int)SCHEME_BE : (int)SCHEME_SOLVE);
        st = E.step(src, batch, 0, 1, batch, scheme == 2, sch, c->dt0, n0, 1, dst, 1, g ? dg : nullptr,
                    ut ? du : nullptr, ut ? c->partial : nullptr, &np);
        if (st == SFDE_OK && ut && norm2) st = sfde_reduce_partials(c, np, norm2);
    }
    if (st == SFDE_OK) {
        const size_t n = P2 * batch;
        if (kind == 0) k_lp_to_f64<__nv_bfloat16><<<grid_for(n), 256, 0, c->stream>>>((const __nv_bfloat16*)dst, tp, n);
        else k_lp_to_f64<float><<<grid_for(n), 256, 0, c->stream>>>((const float*)dst, tp, n);
        sfde_launch_unpad(tp, tu, c->y.n, c->x.n, c->y.P, c->x.P, batch, c->stream);
        st = sfde_copy_out(out, tu, sizeof(double) * n2 * batch, c->stream);
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (st == SFDE_OK && e != cudaSuccess) { sfde_set_last_cuda_error(e, "debug lp step", __FILE__, __LINE__); st = SFDE_ECUDA; }
    if (st == SFDE_OK) st = check_err(M, c->stream);
    M->fused = saved;
    cudaFree(tu); cudaFree(tp); cudaFree(src); cudaFree(dst); cudaFree(dg); cudaFree(du);
    return st;
}

extern "C" sfde_status sfde_debug_lp_chain(sfde_ctx* c, int mode, int scheme, const double* U, int batch, int nchain,
                                          int n0, const double* g, double* out) {
    if (!c || !U || !out || batch < 1 || nchain < 1 || n0 < 1 || scheme < 0 || scheme > 1 ||
        (long long)n0 + (long long)batch * nchain - 1 > c->nt || mode < 0 || mode > 3)
        return SFDE_EINVAL;
    if (c->precision == SFDE_PREC_FP64) return SFDE_EINVAL;
    const int kind = sfde_mixed_kind(c);
    if ((mode == 1 || mode == 2) && !sfde_fused_supported(kind, c->x.P, c->y.P)) return SFDE_EUNSUPPORTED;
    if (!c->mixed || c->mixed->kind != kind) SFDE_TRY(setup_mixed(c, kind, 2, 1, 1));
    SfdeMixed* M = c->mixed;
    if (mode == 3 && (size_t)batch > M->ws) return SFDE_EINVAL;
    const size_t P2 = c->P2(), n2 = (size_t)c->x.n * c->y.n;
    const size_t nout = (size_t)batch * nchain, esz = M->esz;
    double *tu = nullptr, *tp = nullptr;
    void *src = nullptr, *dst = nullptr, *dg = nullptr, *gh = nullptr, *yh = nullptr;
    sfde_status st = SFDE_OK;
    const bool saved = M->fused;
    if (cudaMalloc(&tu, sizeof(double) * n2 * nout) != cudaSuccess ||
        cudaMalloc(&tp, sizeof(double) * P2 * nout) != cudaSuccess || cudaMalloc(&src, P2 * esz * batch) != cudaSuccess ||
        cudaMalloc(&dst, P2 * esz * (nout + nchain)) != cudaSuccess || cudaMalloc(&dg, P2 * esz * nout) != cudaSuccess ||
        (mode == 3 && (cudaMalloc(&gh, P2 * esz * nout) != cudaSuccess || cudaMalloc(&yh, P2 * esz * nout) != cudaSuccess)))
        st = SFDE_ENOMEM;
    if (st == SFDE_OK) st = load_lp(c, U, batch, tu, tp, src, kind);
    if (st == SFDE_OK && g) st = load_lp(c, g, (int)nout, tu, tp, dg, kind);
    if (st == SFDE_OK) {
        LpEngine E{c, M, 2, 1, SFDE_RELAX_FCF, SCHEME_CN};
        const int sch = scheme == 0 ? SCHEME_CN : SCHEME_BE;
        const size_t sl = P2 * esz;
        if (mode == 3) {   // eigenbasis: transforms of all inputs, recurrences, transforms back
            st = E.to_modal(src, batch, 0, 1, batch, M->T2, 1);
            if (st == SFDE_OK && g) st = E.to_modal(dg, (long long)nout, 0, 1, (int)nout, gh, 1);
            if (st == SFDE_OK && !g && cudaMemsetAsync(gh, 0, P2 * esz * nout, c->stream) != cudaSuccess) st = SFDE_ECUDA;
            // interval b: C-point U[b], F-points k = 1..nchain with g[b][k - 1] (slice b nchain + k - 1)
            // and dt[n0 + b nchain + k - 2]
            if (st == SFDE_OK)
                st = E.modal_scan(M->T2, gh, nchain, -1, yh, nchain + 1, batch, c->dt0 + (n0 - 1), nchain, sch);
            if (st == SFDE_OK) st = E.from_modal(yh, (long long)nout, (int)nout, dst, 0);
        } else if (mode == 1) {   // one launch: each CTA runs the nchain steps of its slice
            M->fused = true;
            st = E.step(src, batch, 0, 1, batch, false, sch, c->dt0, n0, nchain, dst, nchain, g ? dg : nullptr,
                        nullptr, nullptr, nullptr, nchain);
        } else {           // nchain launches of single steps (fused kernel or four slice GEMMs)
            M->fused = mode == 2;
            for (int k = 0; k < nchain && st == SFDE_OK; ++k) {
                // step k reads the outputs of step k-1: slices k-1 + b*nchain of dst (allocated with
                // nchain spare slices, so the map over batch*nchain slices from there stays inside)
                void* s = k == 0 ? src : (void*)((char*)dst + (k - 1) * sl);
                const long long ns = k == 0 ? batch : (long long)nout;
                st = E.step(s, ns, 0, k == 0 ? 1 : nchain, batch, false, sch, c->dt0, n0 + k, nchain,
                            (char*)dst + k * sl, nchain, g ? (const void*)((const char*)dg + k * sl) : nullptr,
                            nullptr, nullptr, nullptr);
            }
        }
    }
    if (st == SFDE_OK) {
        const size_t n = P2 * nout;
        if (kind == 0) k_lp_to_f64<__nv_bfloat16><<<grid_for(n), 256, 0, c->stream>>>((const __nv_bfloat16*)dst, tp, n);
        else k_lp_to_f64<float><<<grid_for(n), 256, 0, c->stream>>>((const float*)dst, tp, n);
        sfde_launch_unpad(tp, tu, c->y.n, c->x.n, c->y.P, c->x.P, (int)nout, c->stream);
        st = sfde_copy_out(out, tu, sizeof(double) * n2 * nout, c->stream);
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (st == SFDE_OK && e != cudaSuccess) { sfde_set_last_cuda_error(e, "debug lp chain", __FILE__, __LINE__); st = SFDE_ECUDA; }
    if (st == SFDE_OK) st = check_err(M, c->stream);
    M->fused = saved;
    cudaFree(tu); cudaFree(tp); cudaFree(src); cudaFree(dst); cudaFree(dg); cudaFree(gh); cudaFree(yh);
    return st;
}
