// FP64-accurate slice GEMM on the BF16 tensor cores by error-free operand splitting (the splitting
// scheme of Ozaki, Ogita, Oishi and Rump, restated here for tcgen05).
//
// Out_b = (X_b Mat)^T with FP64 X_b (R x K, row-major) and a fixed FP64 Mat (K x N), as the other
// slice GEMMs.  Each row r of X_b is scaled by 2^{-e_r} (e_r from frexp of the row's max |x|) and
// written as six signed base-256 digits:  x = 2^{e_r} sum_{p=1..6} d_p 2^{-8p} + O(2^{e_r - 49}),
// |d_1| <= 256, |d_p| <= 128 (p >= 2), all exact in BF16.  Mat is split the same way per column n.
// Then  (X Mat)[r][n] = 2^{e_r + e_n} sum_{p,q} 2^{-8(p+q)} sum_k d_p[r][k] d_q[k][n],  and the
// terms with p + q <= 7 (21 digit products) are kept: the dropped ones and the digit truncation are
// below 2^{-47} of 2^{e_r + e_n} K, the accuracy of an FP64 GEMM.
//
// Every digit product is an integer matrix product, accumulated exactly in FP32 TMEM accumulators
// as long as every partial sum stays an integer of magnitude <= 2^24 (the digit plans below).  For
// FP64 output the epilogue combines the accumulators in two int64 words (digit weights
// 2^{-16..-40} and 2^{-48..-56}) and converts to FP64 once per output; for the space-time residual
// (resid_int.cu) it leaves the product as one int64 in units of 2^-52 of the operands' scales, so
// that the residual is assembled in integer arithmetic (the FP64 pipe of this GPU runs at about
// 1/64 of the FP32 rate).
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include <cudaTypedefs.h>

#include "sfde_internal.cuh"
#include "tc_common.cuh"

namespace {

// K chunks of 32 BF16 (64-byte rows, 64-byte swizzle) in a ring of stages: a stage holds every
// digit plane of one chunk of both operands, so loads overlap the products.
constexpr int BM = 128, KC = 32;
constexpr int XTILE = BM * KC * 2;     // 8 KB: one digit plane of the 128-row tile, one K chunk
constexpr int TMEM_COLS = 512;

// Digit plans.  Partial sums of an accumulator must stay integers of magnitude <= 2^24 (exact in
// FP32).
//   FP64 output: 6 digits per operand (|d_1| <= 256, |d_p| <= 128), K <= 256: one (1,1) product,
//     two (1,q)/(p,1) products or four with p, q >= 2 per accumulator; the 21 products with
//     p + q <= 7 in 12 accumulators; tiles of N = 32 columns, K summed in one group.
//   Integer output: 7 digits per operand, all of magnitude <= 128, K summed in groups of 128: every
//     product is at most 128^3 = 2^21 per group, so all (at most 7) products of one digit sum share
//     an accumulator: the 28 products with p + q <= 8 in 7 accumulators of N = 32 columns, twice
//     (2 x 224 of the 512 TMEM columns), so that one K group's products run while the previous
//     group is drained.
template <bool INT_OUT> struct Plan;
template <> struct Plan<false> {
    static constexpr int S = 6, NPROD = 21, NACC = 12, BN = 32, STAGES = 3, KGROUP = 256;
};
template <> struct Plan<true> {
    static constexpr int S = 7, BN = 32, STAGES = 3, KGROUP = 128, NBUF = 2;
};
// Integer output with at most 4 digits per operand (the first refinement steps): 4 accumulators of
// 64 columns, twice, fill the 512 TMEM columns; twice the columns per X tile halve its re-reads.
struct PlanWide {
    static constexpr int S = 4, BN = 64, STAGES = 4, KGROUP = 128, NBUF = 2;
};
template <class PL>
constexpr size_t digit_smem_bytes() { return 1024 + (size_t)PL::STAGES * PL::S * (XTILE + PL::BN * KC * 2) + 256; }

// FP64-output plan: accumulator a -> digit sum d = p + q of its products, and the product list
// (p, q, a), grouped by a (the integer plan needs no table: accumulator d - 2 holds digit sum d)
__constant__ int c6_acc_d[12] = {2, 3, 4, 4, 5, 5, 6, 6, 6, 7, 7, 7};
__constant__ int c6_prod[21][3] = {
    {1, 1, 0},
    {1, 2, 1}, {2, 1, 1},
    {1, 3, 2}, {2, 2, 2}, {3, 1, 3},
    {1, 4, 4}, {2, 3, 4}, {3, 2, 5}, {4, 1, 5},
    {1, 5, 6}, {2, 4, 6}, {3, 3, 7}, {4, 2, 7}, {5, 1, 8},
    {1, 6, 9}, {2, 5, 9}, {3, 4, 10}, {4, 3, 10}, {5, 2, 11}, {6, 1, 11},
};

template <bool INT_OUT>
constexpr int mtile() { return Plan<INT_OUT>::BN * KC * 2; }   // one digit plane of the matrix tile
template <bool INT_OUT>
constexpr size_t smem_bytes() {
    return 1024 + (size_t)Plan<INT_OUT>::STAGES * Plan<INT_OUT>::S * (XTILE + mtile<INT_OUT>()) + 256;
}

struct OzArgs {
    int R, K, N, batch;          // X slice R x K (digits in planes of nslices x R x K), Mat K x N
    const int* xe;               // row exponents, batch x R (FP64 output only)
    const int* me;               // column exponents, N (FP64 output only)
    void* out; long long out_stride;     // Out_b = (X_b Mat)^T, N x R per slice: double or int64
    int zshift;                  // integer output: final right shift (units 2^{zshift-52})
    int nd;                      // integer output: digits used per operand (4..7; p + q <= nd + 1)
    int* err;
};

// Longer K is summed in groups (Plan::KGROUP), each group drained from TMEM into int64 registers
// before the next one starts.

__device__ __forceinline__ double pow2(int e) {  // exact 2^e for normal range
    return __longlong_as_double((long long)(e + 1023) << 52);
}

// FP64 output: sum_{p+q<=7} 2^{-8(p+q)} sum_k d_p c_q scaled by the row and column exponents.
// Roles: warp 4 lane 0 issues TMA, warp 5 lane 0 issues the MMAs, warps 0-3 drain the
// accumulators (TMEM lanes 32w..32w+31).
constexpr int OZ_THREADS = 192;

__global__ void __launch_bounds__(OZ_THREADS, 1)
k_ozaki_slice_gemm(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapM, OzArgs p) {
    constexpr bool INT_OUT = false;
    constexpr int S = Plan<INT_OUT>::S, NPROD = Plan<INT_OUT>::NPROD, NACC = Plan<INT_OUT>::NACC;
    constexpr int BN = Plan<INT_OUT>::BN, STAGES = Plan<INT_OUT>::STAGES, KGROUP = Plan<INT_OUT>::KGROUP;
    constexpr int MTILE = BN * KC * 2;
    constexpr int STAGE = S * (XTILE + MTILE);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // stage st: S X planes (8 KB each) then S matrix planes (BN x 64 bytes each)
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE);
    uint64_t* empty = full + STAGES;
    uint64_t* accf = empty + STAGES;
    uint64_t* fin = accf + 1;
    uint64_t* tfree = fin + 1;                // a K group's accumulators have been drained
    uint32_t* tmem_slot = (uint32_t*)(tfree + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the N tiles of one M tile are neighbours in launch order: they share the X digit planes in L2
    const long long m0 = (long long)blockIdx.y * BM;
    const int n0 = blockIdx.x * BN;
    const long long Mtot = (long long)p.batch * p.R;
    const int nchunks = (p.K + KC - 1) / KC;
    const int nd = S, nprod = NPROD;
    constexpr int CPG = KGROUP / KC;          // chunks per K group (K <= 256: one group)

    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES; ++st) { tc::mbar_init(&full[st], 1); tc::mbar_init(&empty[st], 1); }
        tc::mbar_init(accf, 1);
        tc::mbar_init(fin, 1);
        tc::mbar_init(tfree, 128);
        tc::mbar_fence_init();
        tc::prefetch_tmap(&mapX);
        tc::prefetch_tmap(&mapM);
    }
    if (warp == 0) tc::tmem_alloc(tmem_slot, TMEM_COLS);
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int b0 = (int)(m0 / p.R), r0 = (int)(m0 % p.R);
    bool ok = true;
    if (warp == 4 && lane == 0) {
        int issued = 0;
        for (int c = 0; c < nchunks && ok; ++c) {
            const int st = c % STAGES;
            if (c >= STAGES) ok = tc::mbar_wait(&empty[st], (uint32_t)(c / STAGES - 1) & 1u, p.err, tc::ERR_WAIT_EMPTY);
            if (!ok) break;
            uint8_t* sX = smem + st * STAGE;
            uint8_t* sM = sX + S * XTILE;
            tc::mbar_arrive_expect_tx(&full[st], (uint32_t)(nd * (XTILE + MTILE)));
            for (int d = 0; d < nd; ++d) {
                tc::tma_load_4d(sX + d * XTILE, &mapX, &full[st], c * KC, r0, b0, d);
                tc::tma_load_3d(sM + d * MTILE, &mapM, &full[st], c * KC, n0, d);
            }
            ++issued;
        }
        // own copies in flight must land before the CTA's shared memory goes away
        for (int c = issued - STAGES < 0 ? 0 : issued - STAGES; c < issued; ++c)
            tc::mbar_wait(&full[c % STAGES], (uint32_t)(c / STAGES) & 1u, p.err, tc::ERR_WAIT_FULL);
    } else if (warp == 5 && lane == 0) {
        const uint32_t idesc = tc::idesc_f32acc(1u, BM, BN);
        bool any = false;
        for (int c = 0; c < nchunks && ok; ++c) {
            const int st = c % STAGES, grp = c / CPG;
            const bool group_start = c % CPG == 0;
            // a new K group overwrites the accumulators once the drain warps have read them
            if (group_start && grp > 0) ok = tc::mbar_wait(tfree, (uint32_t)(grp - 1) & 1u, p.err, tc::ERR_WAIT_ACC);
            if (!ok) break;
            ok = tc::mbar_wait(&full[st], (uint32_t)(c / STAGES) & 1u, p.err, tc::ERR_WAIT_FULL);
            if (!ok) break;
            tc::tc_fence_after();
            const uint8_t* sX = smem + st * STAGE;
            const uint8_t* sM = sX + S * XTILE;
            for (int i = 0; i < nprod; ++i) {
                const int dp = c6_prod[i][0] - 1, dq = c6_prod[i][1] - 1;
                const int a = c6_prod[i][2];
                // the first product of an accumulator in a group's first chunk overwrites it
                const bool first = group_start && (i == 0 || c6_prod[i - 1][2] != a);
#pragma unroll
                for (int kk = 0; kk < KC / 16; ++kk) {
                    const uint64_t ad = tc::smem_desc_sw64(sX + dp * XTILE + kk * 32);
                    const uint64_t bd = tc::smem_desc_sw64(sM + dq * MTILE + kk * 32);
                    tc::mma<0>(tmem + (uint32_t)(a * BN), ad, bd, idesc, (first && kk == 0) ? 0u : 1u);
                }
            }
            any = true;
            tc::mma_commit(&empty[st]);
            if (c % CPG == CPG - 1 || c == nchunks - 1) tc::mma_commit(accf);   // group complete
        }
        if (!ok && any) {  // products still running must finish before TMEM is freed
            tc::mma_commit(fin);
            tc::mbar_wait(fin, 0, p.err, tc::ERR_WAIT_ACC);
        }
    }

    if (warp >= 4) {
        // producer and MMA warps: nothing to drain
    } else if (__all_sync(0xffffffffu, tc::mbar_wait(accf, 0, p.err, tc::ERR_WAIT_ACC))) {
        // FP64 output (K <= 256: one group)
        tc::tc_fence_after();
        const long long m = m0 + warp * 32 + lane;
        const bool valid = m < Mtot;
        // z_hi in units of 2^-40 (digit sums d = 2..5), z_lo in units of 2^-56 (d = 6, 7)
        long long zhi[BN], zlo[BN];
#pragma unroll
        for (int j = 0; j < BN; ++j) { zhi[j] = 0; zlo[j] = 0; }
#pragma unroll 1
        for (int a = 0; a < NACC; ++a) {
            uint32_t v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(a * BN), v);
            const int d = c6_acc_d[a];
#pragma unroll
            for (int j = 0; j < BN; ++j) {
                const long long s = (long long)__float2ll_rn(__uint_as_float(v[j]));  // exact integer
                if (d <= 5) zhi[j] += s * (1ll << (8 * (5 - d)));
                else zlo[j] += s * (1ll << (8 * (7 - d)));
            }
        }
        if (valid) {
            const long long b = m / p.R;
            const int r = (int)(m % p.R);
            const int er = p.xe[b * p.R + r];
            double* out = (double*)p.out + b * p.out_stride + r;
#pragma unroll
            for (int j = 0; j < BN; ++j) {
                const int n = n0 + j;
                const int e = er + p.me[n];
                const double y = (double)zhi[j] * pow2(e - 40) + (double)zlo[j] * pow2(e - 56);
                out[(long long)n * p.R] = y;
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, TMEM_COLS);
    }
}

// Integer-output digit GEMM, persistent: CTA c takes tiles c, c + gridDim.x, ... of 128 rows x BN
// columns (columns fastest, so concurrent CTAs share X digit planes in L2).  Warp NDW issues TMA
// and streams chunks across tiles; warp NDW + 1 issues the MMAs; warps 0..NDW-1 drain, warp w
// reading TMEM lanes 32 (w % 4).. (the lanes its warp index may access) and 8 columns.  K groups
// alternate between two accumulator sets: while the drain warps fold group G (and store a finished
// tile), the products of group G + 1 run into the other set, and the producer loads ahead.  With
// 32-column tiles (CW = 8) the drain adds each accumulator into a 32-bit sum per digit sum and
// column (one conversion and one add per value; at most 8 groups of |value| < 2^24) and combines the
// sums into the int64 result once per tile; with 64-column tiles (CW = 16, at most 4 digits: digit
// sums d <= 5) it adds each accumulator into the int64 result directly, shifted exactly.
constexpr int DG_NDW = 16;
constexpr int DG_THREADS = 32 * (DG_NDW + 2);

template <class PL, int CW>
__global__ void __launch_bounds__(DG_THREADS, 1)
k_digit_gemm_int(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapM, OzArgs p) {
    constexpr int S = PL::S, BN = PL::BN, STAGES = PL::STAGES, KGROUP = PL::KGROUP, NBUF = PL::NBUF;
    constexpr int MTILE = BN * KC * 2;
    constexpr int STAGE = S * (XTILE + MTILE);
    constexpr uint32_t SET = S * BN;                    // TMEM columns of one accumulator set
    static_assert(4 * BN / CW == DG_NDW, "four lane quarters x BN / CW column blocks of drain warps");
    static_assert((CW == 8 && S == 7) || (CW == 16 && S <= 4),
                  "32-bit sums of the 7 digit sums, or int64 shifts for d <= 5");
    static_assert(NBUF * SET <= TMEM_COLS && S * BN <= 256, "accumulator sets within TMEM, one product per digit");
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE);
    uint64_t* empty = full + STAGES;
    uint64_t* accf = empty + STAGES;                    // per set: a K group's products complete
    uint64_t* tfree = accf + NBUF;                      // per set: a K group's accumulators have been read
    uint64_t* fin = tfree + NBUF;                       // error path: outstanding products complete
    uint32_t* tmem_slot = (uint32_t*)(fin + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long Mtot = (long long)p.batch * p.R;
    const int ntn = (p.N + BN - 1) / BN;
    const long long ntiles = (long long)ntn * ((Mtot + BM - 1) / BM);
    const int nchunks = (p.K + KC - 1) / KC;
    constexpr int CPG = KGROUP / KC;
    const int ngroups = (nchunks + CPG - 1) / CPG;
    const int nd = p.nd;

    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES; ++st) { tc::mbar_init(&full[st], 1); tc::mbar_init(&empty[st], 1); }
        for (int b = 0; b < NBUF; ++b) { tc::mbar_init(&accf[b], 1); tc::mbar_init(&tfree[b], 32 * DG_NDW); }
        tc::mbar_init(fin, 1);
        tc::mbar_fence_init();
        tc::prefetch_tmap(&mapX);
        tc::prefetch_tmap(&mapM);
    }
    if (warp == 0) tc::tmem_alloc(tmem_slot, TMEM_COLS);
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == DG_NDW) {
        if (lane == 0) {
            bool ok = true;
            long long cnt = 0;
            for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const long long m0 = (t / ntn) * BM;
                const int n0 = (int)(t % ntn) * BN;
                const int b0 = (int)(m0 / p.R), r0 = (int)(m0 % p.R);
                for (int c = 0; c < nchunks && ok; ++c, ++cnt) {
                    const int st = (int)(cnt % STAGES);
                    if (cnt >= STAGES)
                        ok = tc::mbar_wait(&empty[st], (uint32_t)(cnt / STAGES - 1) & 1u, p.err, tc::ERR_WAIT_EMPTY);
                    if (!ok) break;
                    uint8_t* sX = smem + st * STAGE;
                    uint8_t* sM = sX + S * XTILE;
                    tc::mbar_arrive_expect_tx(&full[st], (uint32_t)(nd * (XTILE + MTILE)));
                    for (int d = 0; d < nd; ++d) {
                        tc::tma_load_4d(sX + d * XTILE, &mapX, &full[st], c * KC, r0, b0, d);
                        tc::tma_load_3d(sM + d * MTILE, &mapM, &full[st], c * KC, n0, d);
                    }
                }
            }
            // own copies in flight must land before the CTA's shared memory goes away
            for (long long c = cnt - STAGES < 0 ? 0 : cnt - STAGES; c < cnt; ++c)
                tc::mbar_wait(&full[c % STAGES], (uint32_t)(c / STAGES) & 1u, p.err, tc::ERR_WAIT_FULL);
        }
    } else if (warp == DG_NDW + 1) {
        if (lane == 0) {
            bool ok = true, any = false;
            long long cnt = 0, G = 0;
            for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                for (int c = 0; c < nchunks && ok; ++c, ++cnt) {
                    const int st = (int)(cnt % STAGES);
                    const bool group_start = c % CPG == 0;
                    const int set = (int)(G % NBUF);
                    // a K group overwrites its accumulator set once the drain warps have read the
                    // group NBUF before it (the (G / NBUF)-th completion of that set's barrier)
                    if (group_start && G >= NBUF)
                        ok = tc::mbar_wait(&tfree[set], (uint32_t)(G / NBUF - 1) & 1u, p.err, tc::ERR_WAIT_ACC);
                    if (!ok) break;
                    ok = tc::mbar_wait(&full[st], (uint32_t)(cnt / STAGES) & 1u, p.err, tc::ERR_WAIT_FULL);
                    if (!ok) break;
                    tc::tc_fence_after();
                    const uint8_t* sX = smem + st * STAGE;
                    const uint8_t* sM = sX + S * XTILE;
                    // X digit p against matrix digits 1 .. nd + 1 - p in one product (the matrix
                    // planes lie one after another; accumulator d = p + q sits at columns (d - 2) BN
                    // of the set); the product of p = 1 reaches every accumulator and overwrites the
                    // set at a group's start
                    const uint32_t dset = tmem + (uint32_t)set * SET;
                    for (int pp = 1; pp <= nd; ++pp) {
                        const uint32_t idq = tc::idesc_f32acc(1u, BM, (nd + 1 - pp) * BN);
#pragma unroll
                        for (int kk = 0; kk < KC / 16; ++kk) {
                            const uint64_t ad = tc::smem_desc_sw64(sX + (pp - 1) * XTILE + kk * 32);
                            const uint64_t bd = tc::smem_desc_sw64(sM + kk * 32);
                            tc::mma<0>(dset + (uint32_t)((pp - 1) * BN), ad, bd, idq,
                                       (group_start && pp == 1 && kk == 0) ? 0u : 1u);
                        }
                    }
                    any = true;
                    tc::mma_commit(&empty[st]);
                    if (c % CPG == CPG - 1 || c == nchunks - 1) { tc::mma_commit(&accf[set]); ++G; }
                }
            }
            if (!ok && any) {  // products still running must finish before TMEM is freed
                tc::mma_commit(fin);
                tc::mbar_wait(fin, 0, p.err, tc::ERR_WAIT_ACC);
            }
        }
    } else {
        if constexpr (CW == 8) {
            const int lq = warp & 3, cb = (warp >> 2) * CW;
            const int zs = p.zshift;
            bool ok = true;
            long long G = 0;
            for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const long long m = (t / ntn) * BM + lq * 32 + lane;
                const int n0 = (int)(t % ntn) * BN;
                // acc[a]: the exact sum over the K groups of accumulator a (digit sum d = a + 2), in units
                // of 2^{-8d} (at most 8 groups of |value| < 2^24: below 2^27)
                int acc[S][CW];
#pragma unroll
                for (int a = 0; a < S; ++a)
#pragma unroll
                    for (int j = 0; j < CW; ++j) acc[a][j] = 0;
                // the result in units of 2^-52, formed while the last group is drained: the digit sums
                // d <= 6 exactly (Horner in base 256 from d = 2, whose unit is 2^{36-52}), d = 7 and 8
                // (units 2^-56 and 2^-64) combined exactly and added with one rounding (at most half a
                // unit); the sums past nd are zero
                long long y[CW];
                for (int grp = 0; grp < ngroups; ++grp, ++G) {
                    const bool last = grp == ngroups - 1;
                    const int set = (int)(G % NBUF);
                    ok = __all_sync(0xffffffffu,
                                    tc::mbar_wait(&accf[set], (uint32_t)(G / NBUF) & 1u, p.err, tc::ERR_WAIT_ACC));
                    tc::tc_fence_after();
                    if (!ok) break;
                    // accumulator a's 8 columns (the latency of each load is hidden by the other three drain
                    // warps of the sub-partition)
                    const uint32_t base = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)set * SET + (uint32_t)cb;
#pragma unroll
                    for (int a = 0; a < S; ++a) {
                        if (a < nd) {   // no early exit: the loop unrolls and acc stays in registers
                            uint32_t v[CW];
                            tc::tmem_ld8_async(base + (uint32_t)(a * BN), v);
                            tc::tmem_wait_ld();
                            tc::reg_fence8(v);
#pragma unroll
                            for (int j = 0; j < CW; ++j)   // exact, |value| < 2^24
                                acc[a][j] += __float2int_rn(__uint_as_float(v[j]));
                        }
                        if (last) {
#pragma unroll
                            for (int j = 0; j < CW; ++j) {
                                if (a == 0) y[j] = acc[0][j];
                                else if (a < 5) y[j] = y[j] * 256 + acc[a][j];
                                else if (a == 6)
                                    y[j] = y[j] * 16 + (((long long)acc[5][j] * 256 + acc[6][j] + 2048) >> 12);
                            }
                        }
                    }
                    tc::tc_fence_before();
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&tfree[set]))
                                 : "memory");
                }
                // the next tile's products run while this one is stored
                if (ok && m < Mtot) {
                    const long long b = m / p.R;
                    const int r = (int)(m % p.R);
                    long long* out = (long long*)p.out + b * p.out_stride + r;
#pragma unroll
                    for (int j = 0; j < CW; ++j) {   // N is a multiple of BN: every column exists
                        long long v = y[j];
                        if (zs > 0) v = (v + (1ll << (zs - 1))) >> zs;
                        out[(long long)(n0 + cb + j) * p.R] = v;
                    }
                }
            }
        } else {
            const int lq = warp & 3, cb = (warp >> 2) * CW;
            const int zs = p.zshift;
            bool ok = true;
            long long G = 0;
            for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const long long m = (t / ntn) * BM + lq * 32 + lane;
                const int n0 = (int)(t % ntn) * BN;
                long long zt[CW];   // units of 2^-52: digit sum d = a + 2 <= 5 enters shifted by 52 - 8d, exactly
#pragma unroll
                for (int j = 0; j < CW; ++j) zt[j] = 0;
                for (int grp = 0; grp < ngroups; ++grp, ++G) {
                    const int set = (int)(G % NBUF);
                    ok = __all_sync(0xffffffffu,
                                    tc::mbar_wait(&accf[set], (uint32_t)(G / NBUF) & 1u, p.err, tc::ERR_WAIT_ACC));
                    tc::tc_fence_after();
                    if (!ok) break;
                    const uint32_t base = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)set * SET + (uint32_t)cb;
#pragma unroll
                    for (int a = 0; a < S; ++a) {
                        if (a < nd) {
                            uint32_t v[CW];
                            tc::tmem_ld8_async(base + (uint32_t)(a * BN), v);
                            tc::tmem_ld8_async(base + (uint32_t)(a * BN) + 8u, v + 8);
                            tc::tmem_wait_ld();
                            tc::reg_fence8(v);
                            tc::reg_fence8(v + 8);
#pragma unroll
                            for (int j = 0; j < CW; ++j)   // exact, |value| < 2^24
                                zt[j] += (long long)__float2int_rn(__uint_as_float(v[j])) << (52 - 8 * (a + 2));
                        }
                    }
                    tc::tc_fence_before();
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&tfree[set]))
                                 : "memory");
                }
                if (ok && m < Mtot) {
                    const long long b = m / p.R;
                    const int r = (int)(m % p.R);
                    long long* out = (long long*)p.out + b * p.out_stride + r;
#pragma unroll
                    for (int j = 0; j < CW; ++j) {   // N is a multiple of BN: every column exists
                        long long v = zt[j];
                        if (zs > 0) v = (v + (1ll << (zs - 1))) >> zs;
                        out[(long long)(n0 + cb + j) * p.R] = v;
                    }
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, TMEM_COLS);
    }
}

// Row splitting: X_b (+ X2_b) -> S digit planes (BF16) and one exponent per row.  One warp per row.
__global__ void k_oz_split_rows(const double* X, const double* X2, long long x_stride, int R, int K, int nrows,
                                __nv_bfloat16* digits, long long plane, int* xe) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= nrows) return;
    const long long b = w / R, r = w % R;
    const double* x = X + b * x_stride + r * K;
    const double* x2 = X2 ? X2 + b * x_stride + r * K : nullptr;
    double mx = 0.0;
    for (int k = lane; k < K; k += 32) {
        const double v = x2 ? x[k] + x2[k] : x[k];
        mx = fmax(mx, fabs(v));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);          // mx = f 2^e, f in [0.5, 1)
    if (lane == 0) xe[w] = e;
    const double sc = pow2(-e);
    __nv_bfloat16* out = digits + (long long)w * K;
    for (int k = lane; k < K; k += 32) {
        double v = (x2 ? x[k] + x2[k] : x[k]) * sc;  // in (-1, 1), exact scaling
#pragma unroll
        for (int d = 0; d < Plan<false>::S; ++d) {
            v *= 256.0;
            const double q = rint(v);
            v -= q;                                   // exact: |v| <= 1/2
            out[(long long)d * plane + k] = __float2bfloat16_rn((float)q);   // |q| <= 256, exact
        }
    }
}

// Column splitting of the fixed matrix alpha Mat (K x N, row-major) -> digits stored K-major per
// column (planes of N x K).  k_oz_col_exps: one exponent per column (max_k |alpha m_kn| < 2^e_n);
// k_oz_uniform_exp optionally replaces them by their maximum (one scale for the whole matrix);
// k_oz_split_cols writes the digits with those exponents.  One warp per column; setup time only.
__global__ void k_oz_col_exps(const double* Mat, double alpha, int K, int N, int* me) {
    const int n = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (n >= N) return;
    double mx = 0.0;
    for (int k = lane; k < K; k += 32) mx = fmax(mx, fabs(alpha * Mat[(size_t)k * N + n]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);
    if (lane == 0) me[n] = e;
}

// one exponent for the whole matrix, one above the largest column's: |alpha m / 2^e| < 1/2, so the
// first digit, like every other, lies within [-128, 128] (the integer plan's accumulator bound)
__global__ void k_oz_uniform_exp(int* me, int N) {
    __shared__ int red[256];
    int e = -1074;
    for (int n = threadIdx.x; n < N; n += blockDim.x) e = max(e, me[n]);
    red[threadIdx.x] = e;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    for (int n = threadIdx.x; n < N; n += blockDim.x) me[n] = red[0] + 1;
}

__global__ void k_oz_split_cols(const double* Mat, double alpha, int K, int N, int nd, __nv_bfloat16* digits,
                                const int* me) {
    const int n = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (n >= N) return;
    const double sc = pow2(-me[n]);
    for (int k = lane; k < K; k += 32) {
        double v = alpha * Mat[(size_t)k * N + n] * sc;
        for (int d = 0; d < nd; ++d) {
            v *= 256.0;
            const double q = rint(v);
            v -= q;
            digits[(size_t)d * N * K + (size_t)n * K + k] = __float2bfloat16_rn((float)q);
        }
    }
}

// rho for one 32 x 32 tile of slice b (time n = n0 + b):
//   rho = F_n + M_h (U_{n-1} - U_n) - tau_n (K_x M_y Y1 + K_y Y2'),  Y1 = V A_x given transposed in T1,
//   Y2' = A_y V M_x given in T3 (row j, column i), V = U_{n-1} + U_n;  zero outside the interior nodes.
// Writes rho in BF16/FP32 (kind 0/1) and one sum of rho^2 per block.
template <typename OT>
__global__ void k_resid_combine(const double* __restrict__ T1, const double* __restrict__ T3,
                                const double* __restrict__ U, int n0, int Px, int Py, int nx, int ny, double hx,
                                double hy, double kx, double ky, const double* __restrict__ dt, int rank,
                                const double* __restrict__ time_w, const double* __restrict__ bxn,
                                const double* __restrict__ byn, OT* __restrict__ rout, long long rout_stride,
                                double* __restrict__ partial) {
    __shared__ double t1[32][35];
    __shared__ double red[256];
    const size_t P2 = (size_t)Px * Py;
    const int b = blockIdx.z, tn = n0 + b;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const double* T1b = T1 + (size_t)b * P2;
    for (int ii = threadIdx.y; ii < 32; ii += blockDim.y)
        for (int jj = threadIdx.x; jj < 34; jj += 32) {
            const int j = j0 + jj - 1;
            t1[ii][jj] = (j >= 0 && j < Py) ? T1b[(size_t)(i0 + ii) * Py + j] : 0.0;
        }
    __syncthreads();
    const double tau = 0.5 * dt[tn - 1];
    const double my = hy / 6.0, mx = hx / 6.0;
    const double* Ua = U + (size_t)(tn - 1) * P2;
    const double* Ub = U + (size_t)tn * P2;
    const int ii = threadIdx.x, i = i0 + ii;
    double sq = 0.0;
    for (int jj = threadIdx.y; jj < 32; jj += blockDim.y) {
        const int j = j0 + jj;
        double rho = 0.0;
        if (i < nx && j < ny) {
            const double y1 = my * (t1[ii][jj] + 4.0 * t1[ii][jj + 1] + t1[ii][jj + 2]);
            const double stiff = kx * y1 + ky * T3[(size_t)b * P2 + (size_t)j * Px + i];
            double mass = 0.0;
#pragma unroll
            for (int a = -1; a <= 1; ++a) {
                const int jy = j + a;
                if (jy < 0 || jy >= ny) continue;
                double row = 0.0;
#pragma unroll
                for (int cc = -1; cc <= 1; ++cc) {
                    const int ix = i + cc;
                    if (ix < 0 || ix >= nx) continue;
                    const size_t e = (size_t)jy * Px + ix;
                    row += (cc == 0 ? 4.0 : 1.0) * (Ua[e] - Ub[e]);
                }
                mass += (a == 0 ? 4.0 : 1.0) * row;
            }
            mass *= mx * my;
            double f = 0.0;
            for (int q = 0; q < rank; ++q)
                f += time_w[(size_t)(tn - 1) * rank + q] * byn[(size_t)q * Py + j] * bxn[(size_t)q * Px + i];
            rho = f + mass - tau * stiff;
        }
        sq += rho * rho;
        OT* o = rout + (size_t)b * rout_stride + (size_t)j * Px + i;
        if (sizeof(OT) == 2) *o = (OT)__float2bfloat16_rn((float)rho);
        else *o = (OT)sfde_round_tf32((float)rho);
    }
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    red[t] = sq;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (t < s) red[t] += red[t + s];
        __syncthreads();
    }
    if (t == 0) partial[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = red[0];
}

PFN_cuTensorMapEncodeTiled_v12000 encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    }
    return fn;
}


}  // namespace

sfde_status sfde_oz_split_matrix(const double* Mat, int K, int N, OzMatrix* out, cudaStream_t s, double alpha,
                                 bool uniform) {
    // both plans take tiles of 32 columns (N a multiple of 32)
    const int BN = uniform ? Plan<true>::BN : Plan<false>::BN;
    if (K > (uniform ? 1024 : 256) || K % 32 || N % 32 || N < BN) return SFDE_EUNSUPPORTED;
    // uniform scale: the integer-output product (7 digits); per-column scales: FP64 output (6)
    const int S = uniform ? Plan<true>::S : Plan<false>::S;
    out->K = K; out->N = N; out->nd = S;
    SFDE_CUDA(cudaMalloc(&out->digits, sizeof(__nv_bfloat16) * (size_t)S * N * K));
    SFDE_CUDA(cudaMalloc(&out->exps, sizeof(int) * N));
    const unsigned g = (unsigned)((N * 32 + 255) / 256);
    k_oz_col_exps<<<g, 256, 0, s>>>(Mat, alpha, K, N, out->exps);
    if (uniform) k_oz_uniform_exp<<<1, 256, 0, s>>>(out->exps, N);
    k_oz_split_cols<<<g, 256, 0, s>>>(Mat, alpha, K, N, S, (__nv_bfloat16*)out->digits, out->exps);
    SFDE_CUDA(cudaGetLastError());
    out->e_uniform = 0;
    if (uniform) SFDE_CUDA(cudaMemcpyAsync(&out->e_uniform, out->exps, sizeof(int), cudaMemcpyDeviceToHost, s));
    SFDE_CUDA(cudaStreamSynchronize(s));
    auto fn = encode();
    if (!fn) return SFDE_EUNSUPPORTED;
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)N, (cuuint64_t)S};
    cuuint64_t strides[2] = {(cuuint64_t)K * 2, (cuuint64_t)N * K * 2};
    cuuint32_t box[3] = {(cuuint32_t)KC, (cuuint32_t)BN, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(&out->map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, out->digits, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return SFDE_EINVAL;
    out->wide = false;
    if (uniform && N % PlanWide::BN == 0) {   // 64-column tiles for products of at most 4 digits
        cuuint32_t boxw[3] = {(cuuint32_t)KC, (cuuint32_t)PlanWide::BN, 1};
        r = fn(&out->map_wide, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, out->digits, dims, strides, boxw, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return SFDE_EINVAL;
        out->wide = true;
    }
    SFDE_CUDA(cudaFuncSetAttribute(k_ozaki_slice_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem_bytes<false>()));
    SFDE_CUDA(cudaFuncSetAttribute(k_digit_gemm_int<Plan<true>, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)digit_smem_bytes<Plan<true>>()));
    SFDE_CUDA(cudaFuncSetAttribute(k_digit_gemm_int<PlanWide, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)digit_smem_bytes<PlanWide>()));
    return SFDE_OK;
}

void sfde_oz_free_matrix(OzMatrix* m) {
    cudaFree(m->digits);
    cudaFree(m->exps);
    m->digits = nullptr;
    m->exps = nullptr;
}

size_t sfde_oz_digit_bytes(int R, int K, int batch) { return (size_t)Plan<false>::S * R * K * batch * 2; }

namespace {
// 4-D map over S digit planes of batch x R x K BF16 values: {K, R, batch, plane}
sfde_status map_digit_planes(CUtensorMap* map, void* digits, int R, int K, int batch, long long plane, int S) {
    auto fn = encode();
    if (!fn) return SFDE_EUNSUPPORTED;
    cuuint64_t dims[4] = {(cuuint64_t)K, (cuuint64_t)R, (cuuint64_t)batch, (cuuint64_t)S};
    cuuint64_t strides[3] = {(cuuint64_t)K * 2, (cuuint64_t)R * K * 2, (cuuint64_t)plane * 2};
    cuuint32_t box[4] = {KC, (cuuint32_t)(R < BM ? R : BM), (cuuint32_t)(R < BM ? BM / R : 1), 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, digits, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? SFDE_OK : SFDE_EINVAL;
}

template <bool INT_OUT>
sfde_status launch_oz(sfde_ctx* c, const CUtensorMap& mapX, const OzMatrix& M, const OzArgs& a, cudaStream_t s,
                      int nr, int nc, int nout) {
    const long long mt = ((long long)a.batch * a.R + BM - 1) / BM;
    if (mt > 65535) return SFDE_EINVAL;
    // integer output with at most 4 digits: 64-column tiles where the matrix has them
    const bool wide = INT_OUT && a.nd <= PlanWide::S && M.wide;
    const int bn = INT_OUT ? (wide ? PlanWide::BN : Plan<true>::BN) : Plan<false>::BN;
    const int ntn = (M.N + bn - 1) / bn;
    const int slot = sfde_prof_begin(c);
    if constexpr (INT_OUT) {
        static int nsm = 0;
        if (!nsm) {
            int dev = 0;
            SFDE_CUDA(cudaGetDevice(&dev));
            SFDE_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        }
        const unsigned grid = (unsigned)std::min<long long>(mt * ntn, nsm);
        if (wide)
            k_digit_gemm_int<PlanWide, 16><<<grid, DG_THREADS, digit_smem_bytes<PlanWide>(), s>>>(mapX, M.map_wide, a);
        else
            k_digit_gemm_int<Plan<true>, 8><<<grid, DG_THREADS, digit_smem_bytes<Plan<true>>(), s>>>(mapX, M.map, a);
    } else {
        k_ozaki_slice_gemm<<<dim3(ntn, (unsigned)mt), OZ_THREADS, smem_bytes<false>(), s>>>(mapX, M.map, a);
    }
    // tensor work: the digit products of 2 R K N flops each; bytes: the digit planes of X in use,
    // the matrix digits and the output (8 bytes per element) once
    const int S = INT_OUT ? a.nd : Plan<false>::S;
    const int NPROD = INT_OUT ? a.nd * (a.nd + 1) / 2 : Plan<false>::NPROD;   // digit products
    sfde_prof_end(c, slot, 4, (double)NPROD * 2.0 * a.batch * nr * nc * nout,
                  2.0 * S * ((double)a.batch * nr * nc + (double)nc * nout) + 8.0 * a.batch * nr * nout);
    sfde_count_launch(c);
    SFDE_CUDA(cudaGetLastError());
    return SFDE_OK;
}
}  // namespace

sfde_status sfde_oz_gemm(sfde_ctx* c, const double* X, const double* X2, long long x_stride, int R, int K,
                         int batch, const OzMatrix& M, void* digits, int* xe, double* out, long long out_stride,
                         int* err, int nr, int nc, int nout) {
    if (K != M.K || K > 256 || R % 32 || (R > 128 && R % 128) || M.nd != Plan<false>::S) return SFDE_EUNSUPPORTED;
    const long long plane = (long long)batch * R * K;
    const int nrows = batch * R;
    k_oz_split_rows<<<(nrows * 32 + 255) / 256, 256, 0, c->stream>>>(X, X2, x_stride, R, K, nrows,
                                                                      (__nv_bfloat16*)digits, plane, xe);
    sfde_count_launch(c);
    SFDE_CUDA(cudaGetLastError());
    CUtensorMap mapX;
    SFDE_TRY(map_digit_planes(&mapX, digits, R, K, batch, plane, Plan<false>::S));
    OzArgs a{};
    a.R = R; a.K = K; a.N = M.N; a.batch = batch; a.xe = xe; a.me = M.exps;
    a.out = out; a.out_stride = out_stride; a.err = err;
    return launch_oz<false>(c, mapX, M, a, c->stream, nr, nc, nout);
}

// |sum_k x_k m_k| <= K/4 for |x|, |m| <= 1/2 (units 2^-52): beyond K = 256 the product is scaled
// down by K/256 so that it stays below 2^58, with headroom for the (1,4,1) stencils
int sfde_oz_int_shift(int K) {
    int s = 0;
    while ((256 << s) < K) ++s;
    return s;
}

sfde_status sfde_oz_gemm_int(sfde_ctx* c, void* xdigits, long long plane, int R, int K, int batch,
                             const OzMatrix& M, long long* out, long long out_stride, int* err, int nr, int nc,
                             int nout, int nd) {
    if (K != M.K || K > 1024 || (K > 256 && K % 256) || R % 32 || (R > 128 && R % 128) ||
        plane < (long long)batch * R * K || M.nd != Plan<true>::S || nd < 4 || nd > Plan<true>::S)
        return SFDE_EUNSUPPORTED;
    CUtensorMap mapX;
    SFDE_TRY(map_digit_planes(&mapX, xdigits, R, K, batch, plane, Plan<true>::S));
    OzArgs a{};
    a.R = R; a.K = K; a.N = M.N; a.batch = batch;
    a.out = out; a.out_stride = out_stride; a.err = err;
    a.zshift = sfde_oz_int_shift(K);
    a.nd = nd;
    return launch_oz<true>(c, mapX, M, a, c->stream, nr, nc, nout);
}

extern "C" sfde_status sfde_debug_oz_gemm(const double* X, int batch, int R, int K, const double* Mat, int N,
                                         double* Out, int* err_out) {
    if (!X || !Mat || !Out || batch < 1 || R < 32 || R % 32 || (R > 128 && R % 128) || K < 32 || K % 32 ||
        K > 256 || N < 32 || N % 32)
        return SFDE_EINVAL;
    sfde_ctx* c = new sfde_ctx();
    OzMatrix M;
    void* digits = nullptr;
    int* xe = nullptr;
    int* err = nullptr;
    sfde_status st = SFDE_OK;
    cudaError_t e = cudaSuccess;
    int herr = 0;
    st = sfde_oz_split_matrix(Mat, K, N, &M, nullptr, 1.0, false);
    if (st == SFDE_OK) {
        if ((e = cudaMalloc(&digits, sfde_oz_digit_bytes(R, K, batch))) != cudaSuccess ||
            (e = cudaMalloc(&xe, sizeof(int) * (size_t)batch * R)) != cudaSuccess ||
            (e = cudaMalloc(&err, sizeof(int))) != cudaSuccess || (e = cudaMemset(err, 0, sizeof(int))) != cudaSuccess) {
            sfde_set_last_cuda_error(e, "debug oz gemm alloc", __FILE__, __LINE__);
            st = SFDE_ECUDA;
        }
    }
    if (st == SFDE_OK)
        st = sfde_oz_gemm(c, X, nullptr, (long long)R * K, R, K, batch, M, digits, xe, Out, (long long)N * R, err,
                          R, K, N);
    if (st == SFDE_OK) {
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) { sfde_set_last_cuda_error(e, "debug oz gemm", __FILE__, __LINE__); st = SFDE_ECUDA; }
        else cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    }
    if (err_out) *err_out = herr;
    if (st == SFDE_OK && herr) st = SFDE_ETIMEOUT;
    sfde_oz_free_matrix(&M);
    cudaFree(digits); cudaFree(xe); cudaFree(err);
    delete c;
    return st;
}
