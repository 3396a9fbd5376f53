// One spectral step per CTA with all four products on chip (BF16 operands, FP32 accumulation,
// P_x = P_y = P in {128, 256}).
//
// For a time slice U (P x P, row j = y node, column i = x node) the step
//     X = V_y [ f o (W_y^T U W_x) ] V_x^T  (+ g - u_target)
// is four tcgen05 products D = Op Data^T, Op (M x K) the fixed matrix, Data (N x K) the slice
// operand, both K-major in shared memory.  Each accumulator row is the next product's Data row, so
// the accumulator goes back to shared memory untransposed, in 16-byte vectors:
//   phase 1  D1[a][j] = sum_i Wt_x[a][i] U[j][i]    = (U W_x)[j][a]
//   phase 2  D2[q][a] = sum_j Wt_y[q][j] D1[a][j]   = (W_y^T U W_x)[q][a], then times f(sigma_qa)
//   phase 3  D3[i][q] = sum_a V_x[i][a]  D2[q][a]   = (C V_x^T)[q][i]
//   phase 4  D4[j][i] = sum_q V_y[j][q]  D3[i][q]   = X[j][i]
// (the fast-diagonalisation solve S^{-1} uses V in place of W and f = 1/(1 + tau sigma)).  The
// intermediates are rounded to BF16 exactly as the four-launch chain stores them, so the two forms
// differ only in the order of FP32 accumulation and in how the modal factor is divided out (here
// an approximate reciprocal shared by two modes).  A P x P FP32 accumulator takes P/128 x P TMEM columns (all 512 for
// P = 256); the slice operand (P^2 BF16) stays in shared memory and the fixed matrices stream from
// L2 in 64-wide K-atoms through a two-stage ring.  Per step HBM sees U read once and X written once
// (plus g and u_target), and one launch does what four did.
//
// Pair forms (P = 256, clusters of two CTAs, tcgen05.mma.cta_group::2): CTA r holds rows
// 128r..128r+127 of every operand -- its half of each fixed matrix streams through its ring, its
// half of the slice operand sits in its shared memory -- and the even CTA issues M = N = 256
// products over the pair: rows 128r.. of D land in CTA r's TMEM, which are exactly the Data rows CTA
// r must hold for the next product, so nothing is exchanged.  The loads and drains of both CTAs
// complete on the even CTA's barriers; its commits reach both CTAs (multicast), so no drain
// overwrites Data a product still reads.  With one slice per pair a chained step's right-hand side
// is staged in shared memory by TMA; with two slices per pair (launches with more slices than half
// the SMs) the phases of the two slices alternate, so one slice's products run while the other's
// accumulator is drained.  All forms round the same sums in the same order.
//
// Roles: warps 0-7 drain the accumulator (warp w: TMEM lanes 32 (w % 4).. of every 128-row half,
// one half of the columns; two drain warps per scheduler keep the drain from stalling on latency);
// warp 8 issues TMA (lane 0) and prefetches g / u_target into L2 (all lanes); warp 9 issues the
// MMAs.
// Every wait is bounded; on a timeout the kernel records the error, lets its own copies and
// products finish (bounded), frees TMEM and returns.
#include <cuda_bf16.h>

#include "sfde_internal.cuh"
#include "tc_common.cuh"

namespace {

constexpr int NDRAIN = 8;                       // drain warps 0-7; warp 8 TMA, warp 9 MMA
constexpr int THREADS = 32 * (NDRAIN + 2);
constexpr int HALF_BYTES = 128 * 128;  // 128 rows x 128 bytes: one M-half of a K-atom

template <int P, bool PAIR, int SPP> struct Geo {
    static_assert(SPP == 1 || (PAIR && SPP == 2), "two slices per CTA pair only");
    static constexpr int NH = P / 128;             // 128-row halves of M
    static constexpr int NHL = PAIR ? 1 : NH;      // halves computed by this CTA
    static constexpr int NATOM = P / 64;           // K-atoms of 64 BF16
    static constexpr int ATOM = P * 128;           // bytes of one K-atom of a P-row operand
    static constexpr int DATA = NATOM * ATOM;      // the slice operand, P^2 BF16
    // operand rows held by this CTA per slice: all P, or (pair) its 128-row half, K-atoms of 16 KB
    static constexpr int DATA_L = PAIR ? NATOM * HALF_BYTES : DATA;
    // ring of fixed-matrix K-atoms: two whole atoms, or (pair) this CTA's half of all four
    static constexpr int OSTAGES = PAIR ? NATOM : 2;
    static constexpr int OSTAGE = PAIR ? HALF_BYTES : ATOM;
    static constexpr int RING = OSTAGES * OSTAGE;
    static constexpr int TMEM_COLS = SPP * NHL * P;   // 128, 512, 256 (pair) or 512 (pair, two slices)
    // pair per slice: the right-hand side of a chained step, this CTA's rows, staged by TMA
    static constexpr int GSTAGE = (PAIR && SPP == 1) ? DATA_L : 0;
    static constexpr int STAGE_ROW = P / 2 * 4;    // FP32 output staging: bytes per half-row
    static constexpr int SMEM = 1024 + SPP * DATA_L + RING + GSTAGE + 192 + 2 * P * 4 + SPP * NDRAIN * 8 + 64;
    static_assert(SPP == 2 || NDRAIN * 32 * STAGE_ROW <= DATA_L + RING,
                  "output staging must fit in the operand space");
    static_assert(!PAIR || P == 256, "pair form: two 128-row halves");
    static_assert(2 * OSTAGES + 3 * SPP + 3 <= 23, "barrier block");
};

// byte offset of element (row r, column k) in a K-major, 128-byte-swizzled P-row operand:
// K-atom k/64 is P rows x 128 bytes, rows in 1024-byte groups of 8, 16-byte chunks XOR (r % 8)
template <int P>
__device__ __forceinline__ uint32_t sw128(int r, int k) {
    return (uint32_t)((k >> 6) * (P * 128) + (r >> 3) * 1024 + (r & 7) * 128 +
                      ((((k & 63) >> 3) ^ (r & 7)) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *(const uint32_t*)&v;
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

__device__ __forceinline__ float4 ld_shared_f4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr) : "memory");
    return v;
}

// approximate reciprocal (PTX rcp.approx, about 1 ulp); the result is rounded to BF16 afterwards
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void bf16x8_to_f32(const uint4& u, float (&f)[8]) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        f[2 * i] = __uint_as_float(w[i] << 16);
        f[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
    }
}

template <int P, bool PAIR, int SPP>
__global__ void __launch_bounds__(THREADS, 1)
k_fused_step(const __grid_constant__ CUtensorMap mapU, const __grid_constant__ CUtensorMap mO1,
             const __grid_constant__ CUtensorMap mO2, const __grid_constant__ CUtensorMap mO3,
             const __grid_constant__ CUtensorMap mO4, const __grid_constant__ CUtensorMap mapG, FusedStepArgs p) {
    using G = Geo<P, PAIR, SPP>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sD0 = smem;                                 // slice operands (Data), this CTA's rows, G::DATA_L each
    uint8_t* sO = smem + SPP * G::DATA_L;                // ring of fixed-matrix K-atoms (Op)
    uint8_t* sG = sO + G::RING;                          // pair per slice: staged right-hand side
    uint64_t* bar = (uint64_t*)(sG + G::GSTAGE);
    // pair: the even CTA's ofull, dfull, dready count both CTAs' loads and drains (its MMA thread
    // issues the products of the pair); oempty and accf are signalled to both CTAs
    uint64_t* ofull = bar;                               // [OSTAGES] Op atom landed
    uint64_t* oempty = bar + G::OSTAGES;                 // [OSTAGES] Op atom consumed
    uint64_t* dfull = bar + 2 * G::OSTAGES;              // [SPP] U landed
    uint64_t* dready = dfull + SPP;                      // [SPP] the next Data written by the drain warps
    uint64_t* accf = dready + SPP;                       // [SPP] a phase's products complete
    uint64_t* fin = accf + SPP;                          // error path: outstanding products complete
    uint64_t* gfull = fin + 1;                           // staged right-hand side landed
    uint64_t* gfree = fin + 2;                           // staged right-hand side consumed
    uint32_t* tmem_slot = (uint32_t*)(bar + 23);
    float* s_lx = (float*)(bar + 24);                    // K_x lambda_x[a], P floats
    float* s_ly = s_lx + P;                              // K_y lambda_y[q]
    double* red = (double*)(s_ly + P);                   // [SPP][NDRAIN] partial sums

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rk = PAIR ? (int)tc::cluster_ctarank() : 0;   // pair: the 128-row half of this CTA
    // slices b0 .. b0 + ns - 1 (two per pair: while one slice drains, the other's products run)
    const int b0 = (PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x) * SPP;
    const int ns = min(SPP, p.batch - b0);
    const int nchain = p.nchain;
    const int nphase = 4 * nchain;                       // phases of all chained steps
    const bool gstage = G::GSTAGE > 0 && p.g_tma && p.g && nchain > 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < G::OSTAGES; ++s) { tc::mbar_init(&ofull[s], 1); tc::mbar_init(&oempty[s], 1); }
        for (int s = 0; s < SPP; ++s) {
            tc::mbar_init(&dfull[s], 1);
            tc::mbar_init(&dready[s], (PAIR ? 2 : 1) * 32 * NDRAIN);
            tc::mbar_init(&accf[s], 1);
        }
        tc::mbar_init(fin, 1);
        tc::mbar_init(gfull, 1);
        tc::mbar_init(gfree, NDRAIN);
        tc::mbar_fence_init();
    }
    for (int i = threadIdx.x; i < P; i += THREADS) {
        s_lx[i] = p.kx * p.lamx[i];
        s_ly[i] = p.ky * p.lamy[i];
    }
    if (threadIdx.x < SPP * NDRAIN) red[threadIdx.x] = 0.0;
    if (warp == 0) {
        if constexpr (PAIR) tc::tmem_alloc_pair(tmem_slot, G::TMEM_COLS);
        else tc::tmem_alloc(tmem_slot, G::TMEM_COLS);
    }
    // pair: the peer's barriers are initialised before either CTA signals the other
    if constexpr (PAIR) tc::cluster_sync();
    else __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // slice s, step k of the chain: output dst(s) + k dst_kstride, right-hand side g(s) + k g_kstride,
    // step size dt[n0 + (b0 + s) dn - 1 + k]
    auto gsl = [&](int s) -> const __nv_bfloat16* {
        return p.g ? (const __nv_bfloat16*)p.g + (long long)(b0 + s) * p.g_stride : nullptr;
    };
    auto utsl = [&](int s) -> const __nv_bfloat16* {
        return p.ut ? (const __nv_bfloat16*)p.ut + (long long)(b0 + s) * p.ut_stride : nullptr;
    };
    auto dstsl = [&](int s) -> __nv_bfloat16* { return (__nv_bfloat16*)p.dst + (long long)(b0 + s) * p.dst_stride; };

    if (warp == NDRAIN) {
        if (lane == 0) {
            tc::prefetch_tmap(&mapU);
            for (int s = 0; s < ns; ++s) {
                const int src = p.s0 + (b0 + s) * p.ds;
                uint8_t* sD = sD0 + s * G::DATA_L;
                if (rk == 0) tc::mbar_arrive_expect_tx(&dfull[s], (uint32_t)G::DATA);
                for (int t = 0; t < G::NATOM; ++t)
                    for (int h = 0; h < G::NHL; ++h) {
                        // pair: every load of either CTA completes on the even CTA's barrier
                        if constexpr (PAIR)
                            tc::tma_load_4d_pair(sD + t * HALF_BYTES, &mapU, tc::mapa_shared(tc::smem_u32(&dfull[s]), 0u),
                                                 t * 64, 128 * rk, p.s0 % p.ds, src / p.ds);
                        else
                            tc::tma_load_4d(sD + t * G::ATOM + h * HALF_BYTES, &mapU, &dfull[s], t * 64, h * 128,
                                            p.s0 % p.ds, src / p.ds);
                    }
            }
        }
        __syncwarp();
        // the right-hand sides of the first two steps and u_target are read only by late drains:
        // bring them into L2 now (the drains prefetch the later steps')
        for (int s = 0; s < ns; ++s) {
            const __nv_bfloat16* g0 = gsl(s);
            const __nv_bfloat16* ut = utsl(s);
            for (int e = lane; e < P * P * 2 / 128; e += 32) {
                if (g0) prefetch_l2((const char*)g0 + (size_t)e * 128);
                if (g0 && nchain > 1) prefetch_l2((const char*)(g0 + p.g_kstride) + (size_t)e * 128);
                if (ut) prefetch_l2((const char*)ut + (size_t)e * 128);
            }
        }
        if (lane == 0) {
            const CUtensorMap* maps[4] = {&mO1, &mO2, &mO3, &mO4};
            bool ok = true;
            int issued = 0;
            for (int gi = 0; gi < nphase * G::NATOM && ok; ++gi) {
                const int st = gi % G::OSTAGES, use = gi / G::OSTAGES;
                if (gi >= G::OSTAGES) ok = tc::mbar_wait(&oempty[st], (uint32_t)(use - 1) & 1u, p.err, tc::ERR_WAIT_EMPTY);
                if (!ok) break;
                if constexpr (PAIR) {
                    // rows 128 rk.. of the matrix (a map with 128-row boxes)
                    if (rk == 0) tc::mbar_arrive_expect_tx(&ofull[st], (uint32_t)(2 * G::OSTAGE));
                    tc::tma_load_2d_pair(sO + st * G::OSTAGE, maps[(gi / G::NATOM) & 3],
                                         tc::mapa_shared(tc::smem_u32(&ofull[st]), 0u), (gi % G::NATOM) * 64, 128 * rk);
                } else {
                    tc::mbar_arrive_expect_tx(&ofull[st], (uint32_t)G::OSTAGE);
                    tc::tma_load_2d(sO + st * G::OSTAGE, maps[(gi / G::NATOM) & 3], &ofull[st], (gi % G::NATOM) * 64, 0);
                }
                ++issued;
            }
            // own copies in flight must land before the CTA's shared memory goes away (pair: the
            // even CTA waits for both CTAs' loads, and the odd CTA stays until the even one has)
            if (rk == 0) {
                for (int s = 0; s < ns; ++s) tc::mbar_wait(&dfull[s], 0, p.err, tc::ERR_WAIT_FULL);
                for (int gi = issued - G::OSTAGES < 0 ? 0 : issued - G::OSTAGES; gi < issued; ++gi)
                    tc::mbar_wait(&ofull[gi % G::OSTAGES], (uint32_t)(gi / G::OSTAGES) & 1u, p.err, tc::ERR_WAIT_FULL);
            }
        }
    } else if (warp == NDRAIN + 1) {
        if (lane == 0 && rk == 0) {
            bool ok = true, any = false;
            if constexpr (!PAIR) {
                const uint32_t idesc = tc::idesc_f32acc(1u, 128, P);
                ok = tc::mbar_wait(dfull, 0, p.err, tc::ERR_WAIT_FULL);
                for (int ph = 0; ph < nphase && ok; ++ph) {
                    // the Data of phase ph > 0 is written by the drain of phase ph - 1
                    if (ph > 0) ok = tc::mbar_wait(dready, (uint32_t)(ph - 1) & 1u, p.err, tc::ERR_WAIT_FULL);
                    if (!ok) break;
                    tc::tc_fence_after();
                    for (int t = 0; t < G::NATOM && ok; ++t) {
                        const int gi = ph * G::NATOM + t, st = gi & 1;
                        ok = tc::mbar_wait(&ofull[st], (uint32_t)(gi >> 1) & 1u, p.err, tc::ERR_WAIT_FULL);
                        if (!ok) break;
                        tc::tc_fence_after();
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t bd = tc::smem_desc_sw128(sD0 + t * G::ATOM + kk * 32);
#pragma unroll
                            for (int h = 0; h < G::NH; ++h) {
                                const uint64_t ad = tc::smem_desc_sw128(sO + st * G::ATOM + h * HALF_BYTES + kk * 32);
                                tc::mma<0>(tmem + (uint32_t)(h * P), ad, bd, idesc, (t > 0 || kk > 0) ? 1u : 0u);
                            }
                        }
                        any = true;
                        tc::mma_commit(&oempty[st]);
                    }
                    if (ok) tc::mma_commit(accf);
                }
                if (!ok && any) {  // products still running must finish before TMEM is freed
                    tc::mma_commit(fin);
                    tc::mbar_wait(fin, 0, p.err, tc::ERR_WAIT_ACC);
                }
            } else {
                // the pair's products: D = Op Data^T, M = 256 (rows 128 r.. of Op and of D in CTA r),
                // N = 256 (Data rows 128 r.. in CTA r); each CTA's drain writes exactly its own Data
                // rows, so nothing is exchanged.  With two slices the phases alternate between them
                // (TMEM columns 256 s..), and every fixed-matrix atom serves both.
                const uint32_t idesc = tc::idesc_f32acc(1u, 256, 256);
                for (int ph = 0; ph < nphase && ok; ++ph) {
                    for (int s = 0; s < ns && ok; ++s) {
                        // U (phase 0) or both CTAs' drains of phase ph - 1 of this slice
                        ok = ph == 0 ? tc::mbar_wait_cluster(&dfull[s], 0, p.err, tc::ERR_WAIT_FULL)
                                     : tc::mbar_wait_cluster(&dready[s], (uint32_t)(ph - 1) & 1u, p.err, tc::ERR_WAIT_FULL);
                        if (!ok) break;
                        tc::tc_fence_after();
                        const uint8_t* sD = sD0 + s * G::DATA_L;
                        for (int t = 0; t < G::NATOM && ok; ++t) {
                            if (s == 0) {
                                ok = tc::mbar_wait_cluster(&ofull[t], (uint32_t)ph & 1u, p.err, tc::ERR_WAIT_FULL);
                                if (!ok) break;
                                tc::tc_fence_after();
                            }
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint64_t ad = tc::smem_desc_sw128(sO + t * G::OSTAGE + kk * 32);
                                const uint64_t bd = tc::smem_desc_sw128(sD + t * HALF_BYTES + kk * 32);
                                tc::mma_pair(tmem + (uint32_t)(s * 256), ad, bd, idesc, (t > 0 || kk > 0) ? 1u : 0u);
                            }
                            any = true;
                            if (s == ns - 1) tc::mma_commit_pair_mc(&oempty[t], (uint16_t)3u);
                        }
                        if (ok) tc::mma_commit_pair_mc(&accf[s], (uint16_t)3u);
                    }
                }
                if (!ok && any) {  // products still running must finish before TMEM is freed
                    tc::mma_commit_pair(fin);
                    tc::mbar_wait(fin, 0, p.err, tc::ERR_WAIT_ACC);
                }
            }
        } else if (gstage && lane == 1) {
            // (an arm of its own: neither this loop nor the MMA issue waits for the other to finish)
            // the right-hand side of chained step k (this CTA's 128 rows, 4 K-atoms of 16 KB), once
            // the drain of step k - 1 has read the previous one; the last step reads g directly
            bool ok = true;
            int issued = 0;
            for (int k = 0; k < nchain - 1 && ok; ++k) {
                if (k > 0) ok = tc::mbar_wait(gfree, (uint32_t)(k - 1) & 1u, p.err, tc::ERR_WAIT_EMPTY);
                if (!ok) break;
                tc::mbar_arrive_expect_tx(gfull, (uint32_t)G::GSTAGE);
                for (int t = 0; t < G::NATOM; ++t)
                    tc::tma_load_4d(sG + t * HALF_BYTES, &mapG, gfull, t * 64, 128 * rk, 0, b0 * p.g_tds + k);
                ++issued;
            }
            if (issued > 0) tc::mbar_wait(gfull, (uint32_t)(issued - 1) & 1u, p.err, tc::ERR_WAIT_FULL);
        }
    } else {
        // ---- warps 0-7: accumulator -> next Data operand (phases 1-3 of a step, and phase 4 of a
        // step followed by another) or output (phase 4 of the last step).  Warp w reads TMEM lanes
        // 32 (w % 4).. (the lanes its warp index may access) and columns cb.. cb + CW - 1 of them.
        constexpr int CW = P / 2;                         // accumulator columns per drain warp
        const int lq = warp & 3, cb = (warp >> 2) * CW;
        const bool cn = p.scheme == SCHEME_CN;
        double sq[SPP];
#pragma unroll
        for (int s = 0; s < SPP; ++s) sq[s] = 0.0;
        bool ok = true;
        // byte offset of Data row `row` (a row of this CTA), column k in a slice operand
        auto dofs = [&](int row, int k) -> uint32_t {
            if constexpr (PAIR) return sw128<128>(row - 128 * rk, k);
            else return sw128<P>(row, k);
        };
        // accumulator columns are read 32 at a time (the register budget of ten warps)
        constexpr int CH = 32;
        // right-hand side of a chained step, CH columns of this thread's row, loaded one chunk ahead
        // of its use (the first chunk while the products run): the drain never waits on a load
        uint4 gq[CH / 8];
        auto load_g = [&](const __nv_bfloat16* __restrict__ gk, int h, int c0) {
            const __nv_bfloat16* src = gk + (size_t)((PAIR ? rk : h) * 128 + lq * 32 + lane) * P + cb + c0;
#pragma unroll
            for (int u = 0; u < CH / 8; ++u) gq[u] = __ldg((const uint4*)(src + 8 * u));
        };
        for (int gph = 0; gph < nphase && ok; ++gph) {
            const int ph = gph & 3, k = gph >> 2;
            const bool last = k == nchain - 1;
#pragma unroll 1
            for (int s = 0; s < ns; ++s) {
                const __nv_bfloat16* __restrict__ g0 = gsl(s);
                const __nv_bfloat16* __restrict__ ut = utsl(s);
                __nv_bfloat16* __restrict__ dst0 = dstsl(s);
                const __nv_bfloat16* __restrict__ g = g0 ? g0 + (long long)k * p.g_kstride : nullptr;
                const uint32_t sD_u = tc::smem_u32(sD0 + s * G::DATA_L);
                const bool gsm = gstage && ph == 3 && !last;    // g of this chained step staged in sG
                if (ph == 3 && !last && g && !gsm) load_g(g, 0, 0);
                if (gsm) ok = ok && __all_sync(0xffffffffu, tc::mbar_wait(gfull, (uint32_t)k & 1u, p.err, tc::ERR_WAIT_FULL));
                ok = ok && __all_sync(0xffffffffu, tc::mbar_wait(&accf[s], (uint32_t)gph & 1u, p.err, tc::ERR_WAIT_ACC));
                tc::tc_fence_after();
                if (!ok) break;
                // modal factor of this step: d_qa = 1 + c sigma_qa, sigma_qa = K_x lambda_x[a] + K_y lambda_y[q],
                // c = tau = dt/2 (Crank-Nicolson, solve) or dt (backward Euler); f = 1/d, and
                // 2/d - 1 = (1 - tau sigma)/(1 + tau sigma) for Crank-Nicolson
                const float dtb = (float)p.dt[p.n0 + (b0 + s) * p.dn - 1 + k];
                const float cst = p.scheme == SCHEME_BE ? dtb : 0.5f * dtb;
                for (int h = 0; h < G::NHL; ++h) {
                    const int hh = PAIR ? rk : h;                 // 128-row half of M
                    const int row = hh * 128 + lq * 32 + lane;    // M index held by this thread
                    const uint32_t taddr =
                        tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)((s * G::NHL + h) * P + cb);
                    if (ph < 3) {
                        const float Bq = fmaf(cst, s_ly[row], 1.f);
                        for (int c0 = 0; c0 < CW; c0 += CH) {
                            uint32_t v[CH];
                            tc::tmem_ld32(taddr + (uint32_t)c0, v);
                            float x[CH];
#pragma unroll
                            for (int j = 0; j < CH; ++j) x[j] = __uint_as_float(v[j]);
                            if (ph == 1) {  // D2[q = row][a = cb + c0 + j] times f(sigma_qa)
#pragma unroll
                                for (int j = 0; j < CH; j += 2) {
                                    // one reciprocal for two modes: 1/d0 = d1 / (d0 d1), 1/d1 = d0 / (d0 d1)
                                    const float d0 = fmaf(cst, s_lx[cb + c0 + j], Bq), d1 = fmaf(cst, s_lx[cb + c0 + j + 1], Bq);
                                    const float r = rcp_approx(d0 * d1);
                                    float f0 = d1 * r, f1 = d0 * r;
                                    if (cn) { f0 = fmaf(2.f, f0, -1.f); f1 = fmaf(2.f, f1, -1.f); }
                                    x[j] *= f0;
                                    x[j + 1] *= f1;
                                }
                            }
#pragma unroll
                            for (int u = 0; u < CH / 8; ++u)
                                st_shared_v4(sD_u + dofs(row, cb + c0 + 8 * u), pack_bf16x2(x[8 * u], x[8 * u + 1]),
                                             pack_bf16x2(x[8 * u + 2], x[8 * u + 3]), pack_bf16x2(x[8 * u + 4], x[8 * u + 5]),
                                             pack_bf16x2(x[8 * u + 6], x[8 * u + 7]));
                        }
                    } else if (!last) {
                        // chained: X[j = row][i] + g -> BF16, the next step's Data (row j, K = i) and this
                        // step's output; the output is copied to global memory after the next step starts
                        for (int c0 = 0; c0 < CW; c0 += CH) {
                            uint4 gv[CH / 8];
                            if (gsm) {
                                // staged: same 128-row swizzled layout as the operand (row - 128 rk)
                                const uint32_t gb = tc::smem_u32(sG);
#pragma unroll
                                for (int u = 0; u < CH / 8; ++u)
                                    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                                                 : "=r"(gv[u].x), "=r"(gv[u].y), "=r"(gv[u].z), "=r"(gv[u].w)
                                                 : "r"(gb + dofs(row, cb + c0 + 8 * u)) : "memory");
                            } else {
#pragma unroll
                                for (int u = 0; u < CH / 8; ++u) gv[u] = g ? gq[u] : make_uint4(0, 0, 0, 0);
                                if (g) {
                                    if (c0 + CH < CW) load_g(g, h, c0 + CH);
                                    else if (h + 1 < G::NHL) load_g(g, h + 1, 0);
                                }
                            }
                            uint32_t v[CH];
                            tc::tmem_ld32(taddr + (uint32_t)c0, v);
#pragma unroll
                            for (int u = 0; u < CH / 8; ++u) {
                                float gf[8];
                                bf16x8_to_f32(gv[u], gf);
                                float x[8];
#pragma unroll
                                for (int q = 0; q < 8; ++q) x[q] = __uint_as_float(v[8 * u + q]) + gf[q];
                                st_shared_v4(sD_u + dofs(row, cb + c0 + 8 * u), pack_bf16x2(x[0], x[1]),
                                             pack_bf16x2(x[2], x[3]), pack_bf16x2(x[4], x[5]), pack_bf16x2(x[6], x[7]));
                            }
                        }
                    } else if constexpr (SPP == 2) {
                        // last step, two slices per pair: staged in FP32 through this slice's own
                        // operand space (free once its last products are done; the other slice's
                        // stays in use), 64 columns per round, each warp reading back only what it
                        // staged; then X + g - u_target written with coalesced accesses
                        constexpr int HC = 64;                  // columns per round
                        constexpr int SROW = HC * 4;            // staging bytes per row
                        constexpr int CPR = HC / 8;             // 8-column chunks per row segment
                        constexpr int UNR = 4;
                        static_assert(NDRAIN * 32 * SROW <= G::DATA_L, "staging fits in one slice operand");
                        const uint32_t stg = sD_u + (uint32_t)(warp * 32 * SROW);
                        const int rbase = hh * 128 + lq * 32;
                        __nv_bfloat16* __restrict__ dst = dst0 + (long long)k * p.dst_kstride;
                        const bool want_sq = ut && p.partial;
                        float sqf = 0.f;
                        for (int r2 = 0; r2 < CW / HC; ++r2) {
                            const int cbase = cb + r2 * HC;
                            for (int c0 = 0; c0 < HC; c0 += CH) {
                                uint32_t v[CH];
                                tc::tmem_ld32(taddr + (uint32_t)(r2 * HC + c0), v);
#pragma unroll
                                for (int u = 0; u < CH / 4; ++u) {
                                    const int ch = (c0 >> 2) + u;
                                    st_shared_v4(stg + (uint32_t)(lane * SROW + ((ch ^ (lane & 7)) << 4)), v[4 * u],
                                                 v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
                                }
                            }
                            __syncwarp();
                            for (int i0 = 0; i0 < CPR; i0 += UNR) {   // 32 rows x CPR chunks over 32 lanes
                                uint4 gv[UNR], uv[UNR];
#pragma unroll
                                for (int kk = 0; kk < UNR; ++kk) {
                                    const int e = (i0 + kk) * 32 + lane, rr = e / CPR, cc = e % CPR;
                                    const size_t off = (size_t)(rbase + rr) * P + cbase + cc * 8;
                                    gv[kk] = g ? __ldg((const uint4*)(g + off)) : make_uint4(0, 0, 0, 0);
                                    uv[kk] = ut ? __ldg((const uint4*)(ut + off)) : make_uint4(0, 0, 0, 0);
                                }
#pragma unroll
                                for (int kk = 0; kk < UNR; ++kk) {
                                    const int e = (i0 + kk) * 32 + lane, rr = e / CPR, cc = e % CPR;
                                    const float4 x0 = ld_shared_f4(stg + (uint32_t)(rr * SROW + (((2 * cc) ^ (rr & 7)) << 4)));
                                    const float4 x1 = ld_shared_f4(stg + (uint32_t)(rr * SROW + (((2 * cc + 1) ^ (rr & 7)) << 4)));
                                    float xf[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                                    float gf[8], uf[8];
                                    bf16x8_to_f32(gv[kk], gf);
                                    bf16x8_to_f32(uv[kk], uf);
#pragma unroll
                                    for (int q = 0; q < 8; ++q) xf[q] += gf[q] - uf[q];
                                    if (want_sq) {
#pragma unroll
                                        for (int q = 0; q < 8; ++q) sqf = fmaf(xf[q], xf[q], sqf);
                                    }
                                    uint4 o;
                                    o.x = pack_bf16x2(xf[0], xf[1]);
                                    o.y = pack_bf16x2(xf[2], xf[3]);
                                    o.z = pack_bf16x2(xf[4], xf[5]);
                                    o.w = pack_bf16x2(xf[6], xf[7]);
                                    *(uint4*)(dst + (size_t)(rbase + rr) * P + cbase + cc * 8) = o;
                                }
                            }
                            __syncwarp();
                        }
                        sq[s] += (double)sqf;
                    } else {
                        // stage this warp's 32 rows (j) x CW columns in FP32, 16-byte chunks XOR (row % 8),
                        // then write X + g - u_target with coalesced half-row accesses
                        constexpr int CPR = CW / 8;             // 8-column chunks per half-row
                        constexpr int ITER = CPR;               // 32 rows x CPR chunks over 32 lanes
                        constexpr int UNR = 4;
                        const int rbase = hh * 128 + lq * 32;
                        // g and u_target in groups of UNR chunks, each group loaded one group ahead (the
                        // first before the staging)
                        auto load_grp = [&](int i0, uint4 (&gg)[UNR], uint4 (&uu)[UNR]) {
#pragma unroll
                            for (int kk = 0; kk < UNR; ++kk) {
                                const int e = (i0 + kk) * 32 + lane, rr = e / CPR, cc = e % CPR;
                                const size_t off = (size_t)(rbase + rr) * P + cb + cc * 8;
                                gg[kk] = g ? __ldg((const uint4*)(g + off)) : make_uint4(0, 0, 0, 0);
                                uu[kk] = ut ? __ldg((const uint4*)(ut + off)) : make_uint4(0, 0, 0, 0);
                            }
                        };
                        uint4 gv[UNR], uv[UNR];
                        load_grp(0, gv, uv);
                        const uint32_t stg = tc::smem_u32(sD0) + (uint32_t)(warp * 32 * G::STAGE_ROW);
                        for (int c0 = 0; c0 < CW; c0 += CH) {
                            uint32_t v[CH];
                            tc::tmem_ld32(taddr + (uint32_t)c0, v);
#pragma unroll
                            for (int u = 0; u < CH / 4; ++u) {
                                const int ch = (c0 >> 2) + u;
                                st_shared_v4(stg + (uint32_t)(lane * G::STAGE_ROW + ((ch ^ (lane & 7)) << 4)), v[4 * u],
                                             v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
                            }
                        }
                        __syncwarp();
                        __nv_bfloat16* __restrict__ dst = dst0 + (long long)k * p.dst_kstride;
                        const bool want_sq = ut && p.partial;
                        float sqf = 0.f;   // FP32 over this lane's 8 x ITER values (the FP64 pipe is ~1/64 rate)
                        for (int i0 = 0; i0 < ITER; i0 += UNR) {
                            uint4 gn[UNR], un[UNR];
                            const bool more = i0 + UNR < ITER;
                            if (more) load_grp(i0 + UNR, gn, un);
#pragma unroll
                            for (int kk = 0; kk < UNR; ++kk) {
                                const int e = (i0 + kk) * 32 + lane, rr = e / CPR, cc = e % CPR;
                                const float4 x0 = ld_shared_f4(stg + (uint32_t)(rr * G::STAGE_ROW + (((2 * cc) ^ (rr & 7)) << 4)));
                                const float4 x1 = ld_shared_f4(stg + (uint32_t)(rr * G::STAGE_ROW + (((2 * cc + 1) ^ (rr & 7)) << 4)));
                                float xf[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                                float gf[8], uf[8];
                                bf16x8_to_f32(gv[kk], gf);
                                bf16x8_to_f32(uv[kk], uf);
#pragma unroll
                                for (int q = 0; q < 8; ++q) xf[q] += gf[q] - uf[q];
                                if (want_sq) {
#pragma unroll
                                    for (int q = 0; q < 8; ++q) sqf = fmaf(xf[q], xf[q], sqf);
                                }
                                uint4 o;
                                o.x = pack_bf16x2(xf[0], xf[1]);
                                o.y = pack_bf16x2(xf[2], xf[3]);
                                o.z = pack_bf16x2(xf[4], xf[5]);
                                o.w = pack_bf16x2(xf[6], xf[7]);
                                *(uint4*)(dst + (size_t)(rbase + rr) * P + cb + cc * 8) = o;
                            }
                            if (more) {
#pragma unroll
                                for (int kk = 0; kk < UNR; ++kk) { gv[kk] = gn[kk]; uv[kk] = un[kk]; }
                            }
                        }
                        sq[s] += (double)sqf;
                        __syncwarp();
                    }
                }
                if (ph < 3 || !last) {
                    // generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    tc::tc_fence_before();
                    if (rk == 0) {
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&dready[s])) : "memory");
                    } else {
                        // pair: the odd CTA's rows are read by the even CTA's products
                        tc::mbar_arrive_cluster(tc::mapa_shared(tc::smem_u32(&dready[s]), 0u));
                    }
                }
                if (gsm) {
                    __syncwarp();
                    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(gfree)) : "memory");
                }
                if (ph == 3 && !last) {
                    // while the next step's first product runs: copy this warp's part of the new Data
                    // (exactly this step's BF16 output) to global memory, coalesced half-rows, and bring
                    // the right-hand side two steps ahead into L2
                    __nv_bfloat16* __restrict__ dst = dst0 + (long long)k * p.dst_kstride;
                    constexpr int CPR = CW / 8;
                    for (int h = 0; h < G::NHL; ++h) {
                        const int rbase = (PAIR ? rk : h) * 128 + lq * 32;
#pragma unroll 4
                        for (int e = lane; e < 32 * CPR; e += 32) {
                            const int row = rbase + e / CPR, col = cb + 8 * (e % CPR);
                            uint4 o;
                            asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                                         : "=r"(o.x), "=r"(o.y), "=r"(o.z), "=r"(o.w)
                                         : "r"(sD_u + dofs(row, col)) : "memory");
                            *(uint4*)(dst + (size_t)row * P + col) = o;
                        }
                    }
                    if (g0 && k + 2 < nchain) {
                        const char* gn = (const char*)(g0 + (long long)(k + 2) * p.g_kstride);
                        for (int e = warp * 32 + lane; e < P * P * 2 / 128; e += 32 * NDRAIN) prefetch_l2(gn + (size_t)e * 128);
                    }
                }
            }
        }
#pragma unroll
        for (int s = 0; s < SPP; ++s) {
            double v = sq[s];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[s * NDRAIN + warp] = v;
        }
    }
    tc::tc_fence_before();
    if constexpr (PAIR) {
        // both CTAs' partial sums are final; CTA 0 adds the peer's, which stays valid until the
        // second barrier
        tc::cluster_sync();
        if (p.partial && threadIdx.x == 0 && rk == 0) {
            const uint32_t pr = tc::mapa_shared(tc::smem_u32(red), 1u);
            for (int s = 0; s < ns; ++s) {
                double sp = 0.0;
                for (int w = 0; w < NDRAIN; ++w)
                    sp += red[s * NDRAIN + w] + tc::ld_cluster_f64(pr + 8u * (uint32_t)(s * NDRAIN + w));
                p.partial[b0 + s] = sp;
            }
        }
        tc::cluster_sync();
    } else {
        __syncthreads();
        if (p.partial && threadIdx.x == 0) {
            double sp = 0.0;
            for (int w = 0; w < NDRAIN; ++w) sp += red[w];
            p.partial[b0] = sp;
        }
    }
    if (warp == 0) {
        tc::tc_fence_after();
        if constexpr (PAIR) tc::tmem_dealloc_pair(tmem, G::TMEM_COLS);
        else tc::tmem_dealloc(tmem, G::TMEM_COLS);
    }
}

template <int P, bool PAIR, int SPP>
sfde_status launch(sfde_ctx* c, const CUtensorMap& U, const CUtensorMap& O1, const CUtensorMap& O2,
                   const CUtensorMap& O3, const CUtensorMap& O4, const CUtensorMap& Gm, const FusedStepArgs& a,
                   cudaStream_t s) {
    const int slot = c ? sfde_prof_begin(c) : -1;
    if constexpr (PAIR) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)(2 * ((a.batch + SPP - 1) / SPP)));
        cfg.blockDim = dim3(THREADS);
        cfg.dynamicSmemBytes = Geo<P, PAIR, SPP>::SMEM;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        SFDE_CUDA(cudaLaunchKernelEx(&cfg, k_fused_step<P, PAIR, SPP>, U, O1, O2, O3, O4, Gm, a));
    } else {
        k_fused_step<P, PAIR, SPP><<<a.batch, THREADS, Geo<P, PAIR, SPP>::SMEM, s>>>(U, O1, O2, O3, O4, Gm, a);
    }
    if (c) {
        // per slice: the input once, the output and right-hand side of every chained step
        const double nb = a.batch, nx = c->x.n, ny = c->y.n, nk = a.nchain;
        const double slice = nx * ny;
        const double io = (1.0 + nk * (1.0 + (a.g ? 1.0 : 0.0)) + (a.ut ? 1.0 : 0.0)) * nb * slice;
        sfde_prof_end(c, slot, 3, nk * nb * 4.0 * slice * (nx + ny), 2.0 * (io + 2.0 * nx * nx + 2.0 * ny * ny));
        sfde_count_launch(c);
    }
    SFDE_CUDA(cudaGetLastError());
    return SFDE_OK;
}

}  // namespace

bool sfde_fused_supported(int kind, int Px, int Py) { return kind == 0 && Px == Py && (Px == 128 || Px == 256); }

sfde_status sfde_fused_prepare() {
    SFDE_CUDA(cudaFuncSetAttribute(k_fused_step<128, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   Geo<128, false, 1>::SMEM));
    SFDE_CUDA(cudaFuncSetAttribute(k_fused_step<256, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   Geo<256, false, 1>::SMEM));
    SFDE_CUDA(cudaFuncSetAttribute(k_fused_step<256, true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   Geo<256, true, 1>::SMEM));
    SFDE_CUDA(cudaFuncSetAttribute(k_fused_step<256, true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   Geo<256, true, 2>::SMEM));
    return SFDE_OK;
}

bool sfde_fused_pair_supported(int P) { return P == 256; }

sfde_status sfde_fused_step(sfde_ctx* c, int P, int form, const CUtensorMap& U, const CUtensorMap& O1,
                            const CUtensorMap& O2, const CUtensorMap& O3, const CUtensorMap& O4, const CUtensorMap& Gm,
                            const FusedStepArgs& a, cudaStream_t s) {
    if (a.batch < 1) return SFDE_OK;
    if (!a.dst || !a.dt || !a.lamx || !a.lamy || !a.err || a.nchain < 1 || (a.ut && a.nchain != 1) ||
        a.batch > 65535 * 1024)
        return SFDE_EINVAL;
    if (((uintptr_t)a.dst | (uintptr_t)a.g | (uintptr_t)a.ut) & 15) return SFDE_EINVAL;
    if (form < 0 || form > 2 || (form > 0 && P != 256)) return SFDE_EINVAL;
    if (P == 128) return launch<128, false, 1>(c, U, O1, O2, O3, O4, Gm, a, s);
    if (P == 256) {
        if (form == 1) return launch<256, true, 1>(c, U, O1, O2, O3, O4, Gm, a, s);
        if (form == 2) return launch<256, true, 2>(c, U, O1, O2, O3, O4, Gm, a, s);
        return launch<256, false, 1>(c, U, O1, O2, O3, O4, Gm, a, s);
    }
    return SFDE_EINVAL;
}
