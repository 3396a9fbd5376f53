// Tensor-core slice GEMM for the mixed-precision steps: Out_b = (X_b Mat)^T, as in step_fp64.cu,
// with BF16 (tcgen05.mma kind::f16) or TF32 (kind::tf32) operands and FP32 accumulation in TMEM.
//
// Persistent: the CTAs walk the output tiles of the stacked product (rows = batch slices x R rows
// each) with the N-tiles of one row block next to each other, so the CTAs working at the same time
// share each X row block through L2 (X is read from DRAM once).  Two forms:
//   * N-tiles of 128 or 256 columns: CTA pairs (cta_group::2).  A pair computes a 256 x BN tile as
//     one M = 256 product: each CTA holds 128 rows of X and BN/2 rows of Mat^T per K-block, so a CTA
//     streams 16 + BN/2 x 128 / 1024 KB per K-block instead of 16 + BN/8 KB, and a 6-8 stage ring fits
//     its shared memory; the products are issued by the even CTA, every load completes on its
//     barriers, its commits reach both CTAs;
//   * narrower tiles (P <= 64): one CTA per SM and 128 x BN tiles, four stages.
// Roles (ten warps): warp 0 / lane 0 streams K-blocks of 128 bytes (64 BF16 or 32 FP32 values) of X
// and of Mat^T into the ring of 128-byte-swizzled shared-memory tiles with TMA; warp 1 / lane 0 (of
// the even CTA in a pair) issues four tcgen05.mma (K = 16 BF16 / 8 TF32 each) per K-block into one of
// two TMEM accumulators (2 x BN columns) and releases each stage with tcgen05.commit; warps 2-9 (two
// per TMEM lane quarter, one half of the columns each) read the other accumulator back (tcgen05.ld,
// 32 lanes x 32 columns at a time, the next chunk's load in flight while the current one is stored),
// apply the fused epilogue and store the transposed tile -- lanes hold consecutive rows, so each
// store instruction writes 32 consecutive elements -- while the next tile's products run.  The
// epilogue writes one partial sum of squares per warp and 128-row block.
// X is addressed through a 4-D tensor map {K, R, ds, S/ds} so that a batch of slices taken every
// ds-th time point (a relaxation sweep) is one rectangular box per tile, also when R < 128.
#include <math.h>
#include <string.h>

#include <algorithm>

#include <cudaTypedefs.h>

#include "sfde_internal.cuh"
#include "tc_common.cuh"

namespace {

constexpr int BM = 128;
constexpr int STAGES = 4;                // single-CTA form
constexpr int MAX_PSTAGES = 8;           // pair form: as many stages as 192 KB hold, at most 8
constexpr int PAIR_RING_BYTES = 196608;
constexpr int A_STAGE_BYTES = BM * 128;
constexpr int NEPI = 8;                  // epilogue warp slots: two per TMEM lane quarter (column halves)
constexpr int NTHREADS = 64 + 32 * NEPI; // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue (FP32 products: warps
                                         // 2-5 epilogue, 6-9 split the X tiles into high and low parts)
// epilogue warps of a kind: eight, or four for the three-product FP32 form (the others split)
__host__ __device__ constexpr int n_epi(int kind) { return kind == 2 ? 4 : NEPI; }

// storage of the operands and results by kind: 0 BF16, 1 FP32 rounded to TF32 (the tensor cores read
// FP32 storage as TF32), 2 FP32 (products formed from three TF32 products, see k_split_lo)
template <int KIND> struct StoreT;
template <> struct StoreT<0> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ T from(float v) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ float to(T v) { return __bfloat162float(v); }
};
template <> struct StoreT<1> {
    using T = float;
    static __device__ __forceinline__ T from(float v) { return sfde_round_tf32(v); }
    static __device__ __forceinline__ float to(T v) { return v; }
};
template <> struct StoreT<2> {
    using T = float;
    static __device__ __forceinline__ T from(float v) { return v; }
    static __device__ __forceinline__ float to(T v) { return v; }
};

// FP32 products from TF32 tensor-core products: the tensor cores read an FP32 value x as
// hi(x) = x with its 13 low mantissa bits cleared; lo(x) = x - hi(x) is exact in FP32 and below
// 2^-10 |x|.  Then a b = hi(a) hi(b) + hi(a) lo(b) + lo(a) hi(b) + lo(a) lo(b), each product of TF32
// values exact in FP32; the last is below 2^-20 |a b| and dropped, and the tensor cores' reading of
// lo(.) as TF32 drops at most 2^-21 |x|: products to about 2^-20 relative instead of 2^-10.
__device__ __forceinline__ float tf32_lo(float x) { return x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// lo(.) of a 128-row x 128-byte swizzled tile (16 KB), elementwise (the swizzle only permutes 16-byte
// pieces inside each row, so the same byte offsets hold the low parts in the same layout); the split
// warps (128 threads) each take 32 pieces
__device__ __forceinline__ void split_tile_lo(const uint8_t* src, uint8_t* dst, int t) {
#pragma unroll 4
    for (int k = 0; k < A_STAGE_BYTES / 16 / 128; ++k) {
        const int off = (k * 128 + t) * 16;
        float4 v = *(const float4*)(src + off);
        v.x = tf32_lo(v.x); v.y = tf32_lo(v.y); v.z = tf32_lo(v.z); v.w = tf32_lo(v.w);
        *(float4*)(dst + off) = v;
    }
}

// the products of one K-block: four K-steps of 32 bytes; kind 2 adds hi(A) lo(B) and lo(A) hi(B)
template <int KIND, bool PAIR>
__device__ __forceinline__ void kblock_mmas(uint32_t d, const uint8_t* a, const uint8_t* b, const uint8_t* alo,
                                            const uint8_t* blo, uint32_t idesc, bool first) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint64_t ad = tc::smem_desc_sw128(a + k * 32);
        const uint64_t bd = tc::smem_desc_sw128(b + k * 32);
        const uint32_t acc = (first && k == 0) ? 0u : 1u;
        constexpr int MK = KIND == 0 ? 0 : 1;
        if constexpr (PAIR) tc::mma_pair_kind<MK>(d, ad, bd, idesc, acc);
        else tc::mma<MK>(d, ad, bd, idesc, acc);
        if constexpr (KIND == 2) {
            const uint64_t bld = tc::smem_desc_sw128(blo + k * 32);
            const uint64_t ald = tc::smem_desc_sw128(alo + k * 32);
            if constexpr (PAIR) {
                tc::mma_pair_kind<1>(d, ad, bld, idesc, 1u);
                tc::mma_pair_kind<1>(d, ald, bd, idesc, 1u);
            } else {
                tc::mma<1>(d, ad, bld, idesc, 1u);
                tc::mma<1>(d, ald, bd, idesc, 1u);
            }
        }
    }
}

// TMEM columns of the two accumulators (a power of two >= 32)
__host__ __device__ constexpr uint32_t tmem_cols_for(int BN) {
    return 2 * BN <= 32 ? 32u : 2 * BN <= 64 ? 64u : 2 * BN <= 128 ? 128u : 2 * BN <= 256 ? 256u : 512u;
}

// CTA pairs where they were measured faster: FP32 storage with TF32 products and N >= 512 (P = 512:
// 112 against 121 us per 256-slice product; no gain for BF16, a loss at P = 256), and always for the
// three-product FP32 form with BN >= 128, whose doubled stages only fit a ring as halves
__host__ __device__ inline bool pair_form(int kind, int BN, int Cout) {
    return kind == 2 ? BN >= 128 : (kind == 1 && BN >= 128 && Cout >= 512);
}
// a stage: the X tile and the CTA's Mat^T rows (BN, or BN/2 in a pair), and for kind 2 their low parts
__host__ __device__ inline int b_rows(bool pair, int BN) { return pair ? BN / 2 : BN; }
__host__ __device__ inline int stage_bytes(int kind, bool pair, int BN) {
    return (kind == 2 ? 2 : 1) * (A_STAGE_BYTES + b_rows(pair, BN) * 128);
}
__host__ __device__ inline int n_stages(int kind, bool pair, int BN) {
    if (!pair) return STAGES;
    const int n = PAIR_RING_BYTES / stage_bytes(kind, true, BN);
    return n < MAX_PSTAGES ? n : MAX_PSTAGES;
}

// The epilogue of one 128-row block of the accumulator for epilogue warp (q, h): rows mrow0 + 32 q +
// lane of the stacked product, columns n0 + [cbeg, cend) of the BN columns at TMEM column offset tcol.
// Returns this warp's sum of squares (TC_EPI_FINAL with a target).
template <int KIND, int EPI>
__device__ __forceinline__ double epilogue_block(const TcArgs& p, uint32_t tmem, uint32_t tcol, long long mrow0,
                                                 int n0, int q, int cbeg, int cend, long long Mtot) {
    using T = typename StoreT<KIND>::T;
    const int lane = threadIdx.x & 31;
    double sq = 0.0;
    const long long m = mrow0 + q * 32 + lane;
    const bool valid = m < Mtot;
    const long long b = valid ? m / p.R : 0;
    const int r = valid ? (int)(m % p.R) : 0;
    T* __restrict__ out = (T*)p.out + (p.oskip > 0 ? b + b / p.oskip + 1 : b) * p.out_stride;
    float lx = 0.f;
    float dtf = 0.f;
    if (EPI == TC_EPI_SCALE && valid) {
        lx = p.e.kx * p.e.lamx[r];
        dtf = (float)p.e.dt[p.e.n0 + (int)b * p.e.dn - 1];
    }
    const T* __restrict__ g = (EPI == TC_EPI_FINAL && p.e.g) ? (const T*)p.e.g + b * p.e.g_stride : nullptr;
    const T* __restrict__ ut = (EPI == TC_EPI_FINAL && p.e.utgt) ? (const T*)p.e.utgt + b * p.e.utgt_stride : nullptr;
    // the epilogue of one 32-column chunk held in v
    auto chunk = [&](const uint32_t* v, int c0) {
        if (!valid) return;
        const T* gcol = g ? g + (long long)(n0 + c0) * p.R + r : nullptr;
        const T* ucol = ut ? ut + (long long)(n0 + c0) * p.R + r : nullptr;
        T* ocol = out + (long long)(n0 + c0) * p.R + r;
        // all operand loads of the chunk are issued before any store: they are independent, so
        // their latencies overlap instead of adding up element by element
        float add[32];
        if (EPI == TC_EPI_SCALE) {
#pragma unroll
            for (int j = 0; j < 32; ++j) add[j] = __ldg(p.e.lamy + n0 + c0 + j);
        } else if (EPI == TC_EPI_FINAL) {
#pragma unroll
            for (int j = 0; j < 32; ++j) add[j] = gcol ? StoreT<KIND>::to(gcol[(long long)j * p.R]) : 0.f;
            if (ucol) {
#pragma unroll
                for (int j = 0; j < 32; ++j) add[j] -= StoreT<KIND>::to(ucol[(long long)j * p.R]);
            }
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            float x = __uint_as_float(v[j]);
            if (EPI == TC_EPI_SCALE) {
                const float z = dtf * (lx + p.e.ky * add[j]);
                float f;
                if (p.e.scheme == SCHEME_CN) f = (1.f - 0.5f * z) / (1.f + 0.5f * z);
                else if (p.e.scheme == SCHEME_BE) f = 1.f / (1.f + z);
                else f = 1.f / (1.f + 0.5f * z);  // solve: 1 / (1 + tau sigma)
                x *= f;
            } else if (EPI == TC_EPI_FINAL) {
                x += add[j];
                if (ucol) sq += (double)x * (double)x;
            }
            ocol[(long long)j * p.R] = StoreT<KIND>::from(x);
        }
    };
    // two chunks' TMEM loads in flight: the next chunk is read while this one is stored
    const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + tcol;
    uint32_t va[32], vb[32];
    if (cbeg < cend) {
        tc::tmem_ld32_async(tbase + (uint32_t)cbeg, va);
        tc::tmem_wait_ld();
        tc::reg_fence32(va);
    }
    for (int c0 = cbeg; c0 < cend; c0 += 64) {
        const bool two = c0 + 32 < cend;
        if (two) tc::tmem_ld32_async(tbase + (uint32_t)(c0 + 32), vb);
        chunk(va, c0);
        tc::tmem_wait_ld();
        tc::reg_fence32(vb);
        if (c0 + 64 < cend) tc::tmem_ld32_async(tbase + (uint32_t)(c0 + 64), va);
        if (two) chunk(vb, c0 + 32);
        tc::tmem_wait_ld();
        tc::reg_fence32(va);
    }
    return sq;
}

// X-tile coordinates of the 4-D slice map for stacked row m0
__device__ __forceinline__ void a_coords(const TcArgs& p, long long m0, int& r0, int& c2, int& c3) {
    const int b0 = (int)(m0 / p.R);
    r0 = (int)(m0 % p.R);
    const int s_first = p.s0 + b0 * p.ds;
    c2 = p.s0 % p.ds;
    c3 = s_first / p.ds;
}

// ---------------------------------------------------------------- single-CTA form (BN <= 64)
template <int KIND, int EPI>
__global__ void __launch_bounds__(NTHREADS, 1)
k_tc_slice_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                const __grid_constant__ CUtensorMap mapBlo, TcArgs p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int NE = n_epi(KIND);
    const int BN = p.BN;
    const int B_STAGE_BYTES = BN * 128;
    const int STG = stage_bytes(KIND, false, BN);
    // stage st: X tile, Mat^T tile, then for kind 2 the low parts of both
    auto sA = [&](int st) { return smem + st * STG; };
    auto sB = [&](int st) { return smem + st * STG + A_STAGE_BYTES; };
    auto sAlo = [&](int st) { return smem + st * STG + A_STAGE_BYTES + B_STAGE_BYTES; };
    auto sBlo = [&](int st) { return smem + st * STG + 2 * A_STAGE_BYTES + B_STAGE_BYTES; };
    uint64_t* full = (uint64_t*)(smem + STAGES * STG);
    uint64_t* empty = full + STAGES;
    uint64_t* afull = empty + STAGES;    // kind 2: the X tile landed (the split warps wait for it)
    uint64_t* split = afull + STAGES;    // kind 2: the X tile's low part written
    uint64_t* accf = split + STAGES;     // [2] accumulator b holds a finished tile
    uint64_t* acce = accf + 2;           // [2] accumulator b has been read back (NE epilogue warps)
    uint64_t* fin = acce + 2;            // error path: products in flight have completed
    uint32_t* tmem_slot = (uint32_t*)(fin + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int KB = 128 / 4 * (KIND == 0 ? 2 : 1);  // K elements per stage (128 bytes)
    const int kblocks = (p.C + KB - 1) / KB;
    const long long Mtot = (long long)p.batch * p.R;
    const int mtiles = (int)((Mtot + BM - 1) / BM);
    const int ntiles = p.Cout / BN;
    const int tiles = mtiles * ntiles;
    const uint32_t tcols = tmem_cols_for(BN);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1);
            tc::mbar_init(&afull[s], 1); tc::mbar_init(&split[s], 4);
        }
        for (int b = 0; b < 2; ++b) { tc::mbar_init(&accf[b], 1); tc::mbar_init(&acce[b], NE); }
        tc::mbar_init(fin, 1);
        tc::mbar_fence_init();
        tc::prefetch_tmap(&mapA);
        tc::prefetch_tmap(&mapB);
        if (KIND == 2) tc::prefetch_tmap(&mapBlo);
    }
    if (warp == 0) tc::tmem_alloc(tmem_slot, tcols);
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            bool ok = true;
            long long g = 0;   // K-blocks issued
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
                int r0, c2, c3;
                a_coords(p, (long long)(t / ntiles) * BM, r0, c2, c3);
                const int n0 = (t % ntiles) * BN;
                for (int kb = 0; kb < kblocks; ++kb, ++g) {
                    const int st = (int)(g % STAGES);
                    const uint32_t use = (uint32_t)(g / STAGES);
                    if (g >= STAGES) ok = tc::mbar_wait(&empty[st], (use - 1) & 1u, p.err, tc::ERR_WAIT_EMPTY);
                    if (!ok) break;
                    if constexpr (KIND == 2) {
                        tc::mbar_arrive_expect_tx(&afull[st], (uint32_t)A_STAGE_BYTES);
                        tc::tma_load_4d(sA(st), &mapA, &afull[st], kb * KB, r0, c2, c3);
                        tc::mbar_arrive_expect_tx(&full[st], (uint32_t)(2 * B_STAGE_BYTES));
                        tc::tma_load_2d(sB(st), &mapB, &full[st], kb * KB, n0);
                        tc::tma_load_2d(sBlo(st), &mapBlo, &full[st], kb * KB, n0);
                    } else {
                        tc::mbar_arrive_expect_tx(&full[st], (uint32_t)(A_STAGE_BYTES + B_STAGE_BYTES));
                        tc::tma_load_4d(sA(st), &mapA, &full[st], kb * KB, r0, c2, c3);
                        tc::tma_load_2d(sB(st), &mapB, &full[st], kb * KB, n0);
                    }
                }
            }
            // own copies in flight must land before the CTA's shared memory goes away
            for (long long gi = g - STAGES < 0 ? 0 : g - STAGES; gi < g; ++gi) {
                tc::mbar_wait(&full[gi % STAGES], (uint32_t)(gi / STAGES) & 1u, p.err, tc::ERR_WAIT_FULL);
                if (KIND == 2) tc::mbar_wait(&afull[gi % STAGES], (uint32_t)(gi / STAGES) & 1u, p.err, tc::ERR_WAIT_FULL);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_f32acc(KIND == 0 ? 1u : 2u, BM, BN);
            bool ok = true, any = false;
            long long g = 0;
            int it = 0;
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++it) {
                const int buf = it & 1;
                // the epilogue has read this accumulator's previous tile
                if (it >= 2) ok = tc::mbar_wait(&acce[buf], (uint32_t)((it >> 1) - 1) & 1u, p.err, tc::ERR_WAIT_ACC);
                if (!ok) break;
                tc::tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(buf * BN);
                for (int kb = 0; kb < kblocks; ++kb, ++g) {
                    const int st = (int)(g % STAGES);
                    const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
                    ok = tc::mbar_wait(&full[st], ph, p.err, tc::ERR_WAIT_FULL);
                    if (ok && KIND == 2) ok = tc::mbar_wait(&split[st], ph, p.err, tc::ERR_WAIT_FULL);
                    if (!ok) break;
                    tc::tc_fence_after();
                    kblock_mmas<KIND, false>(d, sA(st), sB(st), sAlo(st), sBlo(st), idesc, kb == 0);
                    any = true;
                    tc::mma_commit(&empty[st]);
                }
                if (ok) tc::mma_commit(&accf[buf]);
            }
            if (!ok && any) {  // products still running must finish before TMEM is freed
                tc::mma_commit(fin);
                tc::mbar_wait(fin, 0, p.err, tc::ERR_WAIT_ACC);
            }
        }
    } else if (warp < 2 + NE) {
        // ---- epilogue warps: TMEM lanes 32 q .. 32 q + 31 (q = warp % 4, the quarter a warp may
        // access), i.e. rows 32 q + lane of each tile, and (eight warps) one half of the columns
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;
        int cbeg = 0, cend = BN;
        if (NE == 8) {
            const int HB = BN >= 64 ? BN / 2 : BN;  // BN = 32: the first half only
            cbeg = h * HB;
            cend = BN >= 64 ? cbeg + HB : (h == 0 ? BN : 0);
        }
        int it = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++it) {
            const int buf = it & 1;
            // tcgen05.ld is warp-collective (.sync.aligned): the whole warp reads the accumulator or
            // none of it, so a lane whose bounded wait ran out makes its warp stop
            const bool acc_ok =
                __all_sync(0xffffffffu, tc::mbar_wait(&accf[buf], (uint32_t)(it >> 1) & 1u, p.err, tc::ERR_WAIT_ACC));
            if (!acc_ok) break;
            tc::tc_fence_after();
            const int mt = t / ntiles, nt = t % ntiles;
            double sq = epilogue_block<KIND, EPI>(p, tmem, (uint32_t)(buf * BN), (long long)mt * BM, nt * BN, q, cbeg,
                                                  cend, Mtot);
            // every tcgen05.ld of this warp has completed: the accumulator may take the tile after next
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acce[buf]);
            // one partial sum per warp slot and 128-row block (no barrier between the epilogue warps:
            // a warp whose wait ran out leaves the loop alone); four warps also clear the other slots
            if (EPI == TC_EPI_FINAL && p.e.partial) {
                for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, off);
                if (lane == 0) {
                    double* pp = p.e.partial + ((size_t)nt * mtiles + mt) * NEPI;
                    pp[h * 4 + q] = sq;
                    if (NE == 4) pp[4 + q] = 0.0;
                }
            }
        }
    } else {
        // ---- kind 2: warps 6-9 write the low parts of each X tile once it has landed
        const int tsp = threadIdx.x - 32 * (2 + NE);
        long long g = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x)
            for (int kb = 0; kb < kblocks && ok; ++kb, ++g) {
                const int st = (int)(g % STAGES);
                ok = __all_sync(0xffffffffu,
                                tc::mbar_wait(&afull[st], (uint32_t)(g / STAGES) & 1u, p.err, tc::ERR_WAIT_FULL));
                if (!ok) break;
                split_tile_lo(sA(st), sAlo(st), tsp);
                // the generic-proxy writes must be visible to the tensor cores' (async proxy) reads
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&split[st]);
            }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, tcols);
    }
}

// ---------------------------------------------------------------- CTA-pair form (BN = 128, 256)
template <int KIND, int EPI>
__global__ void __launch_bounds__(NTHREADS, 1)
k_tc_slice_gemm_pair(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                     const __grid_constant__ CUtensorMap mapBlo, TcArgs p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int NE = n_epi(KIND);
    const int BN = p.BN;
    const int BH = BN / 2;                               // Mat^T rows per CTA
    const int B_STAGE_BYTES = BH * 128;
    const int NST = n_stages(KIND, true, BN);
    const int STG = stage_bytes(KIND, true, BN);
    auto sA = [&](int st) { return smem + st * STG; };
    auto sB = [&](int st) { return smem + st * STG + A_STAGE_BYTES; };
    auto sAlo = [&](int st) { return smem + st * STG + A_STAGE_BYTES + B_STAGE_BYTES; };
    auto sBlo = [&](int st) { return smem + st * STG + 2 * A_STAGE_BYTES + B_STAGE_BYTES; };
    // the even CTA's full barriers count both CTAs' loads (kind 2: of Mat^T only; each CTA's X tile
    // lands on its own afull), its split barriers both CTAs' split warps; empty and accf are signalled
    // to both CTAs by the even CTA's commits; the even CTA's acce counts both CTAs' epilogue warps
    uint64_t* full = (uint64_t*)(smem + NST * STG);
    uint64_t* empty = full + MAX_PSTAGES;
    uint64_t* afull = empty + MAX_PSTAGES;
    uint64_t* split = afull + MAX_PSTAGES;
    uint64_t* accf = split + MAX_PSTAGES;  // [2]
    uint64_t* acce = accf + 2;             // [2]
    uint64_t* fin = acce + 2;
    uint32_t* tmem_slot = (uint32_t*)(fin + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rk = (int)tc::cluster_ctarank();
    constexpr int KB = 128 / 4 * (KIND == 0 ? 2 : 1);
    const int kblocks = (p.C + KB - 1) / KB;
    const long long Mtot = (long long)p.batch * p.R;
    const int mtiles = (int)((Mtot + BM - 1) / BM);           // 128-row blocks
    const int mpairs = (mtiles + 1) / 2;                       // 256-row pair tiles
    const int ntiles = p.Cout / BN;
    const int tiles = mpairs * ntiles;
    const int pair = (int)(blockIdx.x >> 1), npairs = (int)(gridDim.x >> 1);
    const uint32_t tcols = tmem_cols_for(BN);

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1);
            tc::mbar_init(&afull[s], 1); tc::mbar_init(&split[s], 8);
        }
        for (int b = 0; b < 2; ++b) { tc::mbar_init(&accf[b], 1); tc::mbar_init(&acce[b], 2 * NE); }
        tc::mbar_init(fin, 1);
        tc::mbar_fence_init();
        tc::prefetch_tmap(&mapA);
        tc::prefetch_tmap(&mapB);
        if (KIND == 2) tc::prefetch_tmap(&mapBlo);
    }
    if (warp == 0) tc::tmem_alloc_pair(tmem_slot, tcols);
    // the peer's barriers are initialised before either CTA signals the other
    tc::cluster_sync();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            bool ok = true;
            long long g = 0;
            for (int t = pair; t < tiles && ok; t += npairs) {
                int r0, c2, c3;
                a_coords(p, (long long)(t / ntiles) * (2 * BM) + (long long)rk * BM, r0, c2, c3);
                const int n0 = (t % ntiles) * BN + rk * BH;
                for (int kb = 0; kb < kblocks; ++kb, ++g) {
                    const int st = (int)(g % NST);
                    const uint32_t use = (uint32_t)(g / NST);
                    if (g >= NST) ok = tc::mbar_wait(&empty[st], (use - 1) & 1u, p.err, tc::ERR_WAIT_EMPTY);
                    if (!ok) break;
                    const uint32_t fb = tc::mapa_shared(tc::smem_u32(&full[st]), 0u);
                    if constexpr (KIND == 2) {
                        tc::mbar_arrive_expect_tx(&afull[st], (uint32_t)A_STAGE_BYTES);
                        tc::tma_load_4d(sA(st), &mapA, &afull[st], kb * KB, r0, c2, c3);
                        if (rk == 0) tc::mbar_arrive_expect_tx(&full[st], (uint32_t)(4 * B_STAGE_BYTES));
                        tc::tma_load_2d_pair(sB(st), &mapB, fb, kb * KB, n0);
                        tc::tma_load_2d_pair(sBlo(st), &mapBlo, fb, kb * KB, n0);
                    } else {
                        if (rk == 0) tc::mbar_arrive_expect_tx(&full[st], (uint32_t)(2 * (A_STAGE_BYTES + B_STAGE_BYTES)));
                        tc::tma_load_4d_pair(sA(st), &mapA, fb, kb * KB, r0, c2, c3);
                        tc::tma_load_2d_pair(sB(st), &mapB, fb, kb * KB, n0);
                    }
                }
            }
            // both CTAs' copies in flight must land before either CTA's shared memory goes away: the
            // even CTA waits for the pair's, each CTA for its own X tiles (kind 2), and the odd CTA
            // stays until the cluster barrier below
            for (long long gi = g - NST < 0 ? 0 : g - NST; gi < g; ++gi) {
                if (rk == 0)
                    tc::mbar_wait_cluster(&full[gi % NST], (uint32_t)(gi / NST) & 1u, p.err, tc::ERR_WAIT_FULL);
                if (KIND == 2) tc::mbar_wait(&afull[gi % NST], (uint32_t)(gi / NST) & 1u, p.err, tc::ERR_WAIT_FULL);
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && rk == 0) {
            const uint32_t idesc = tc::idesc_f32acc(KIND == 0 ? 1u : 2u, 2 * BM, BN);
            bool ok = true, any = false;
            long long g = 0;
            int it = 0;
            for (int t = pair; t < tiles && ok; t += npairs, ++it) {
                const int buf = it & 1;
                // both CTAs' epilogues have read this accumulator's previous tile
                if (it >= 2)
                    ok = tc::mbar_wait_cluster(&acce[buf], (uint32_t)((it >> 1) - 1) & 1u, p.err, tc::ERR_WAIT_ACC);
                if (!ok) break;
                tc::tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(buf * BN);
                for (int kb = 0; kb < kblocks; ++kb, ++g) {
                    const int st = (int)(g % NST);
                    const uint32_t ph = (uint32_t)(g / NST) & 1u;
                    ok = tc::mbar_wait_cluster(&full[st], ph, p.err, tc::ERR_WAIT_FULL);
                    if (ok && KIND == 2) ok = tc::mbar_wait_cluster(&split[st], ph, p.err, tc::ERR_WAIT_FULL);
                    if (!ok) break;
                    tc::tc_fence_after();
                    kblock_mmas<KIND, true>(d, sA(st), sB(st), sAlo(st), sBlo(st), idesc, kb == 0);
                    any = true;
                    tc::mma_commit_pair_mc(&empty[st], (uint16_t)3u);
                }
                if (ok) tc::mma_commit_pair_mc(&accf[buf], (uint16_t)3u);
            }
            if (!ok && any) {  // products still running must finish before TMEM is freed
                tc::mma_commit_pair(fin);
                tc::mbar_wait(fin, 0, p.err, tc::ERR_WAIT_ACC);
            }
        }
    } else if (warp < 2 + NE) {
        // ---- epilogue warps of both CTAs: this CTA's 128 rows of the pair tile
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;
        const int cbeg = NE == 8 ? h * BH : 0, cend = NE == 8 ? cbeg + BH : BN;
        int it = 0;
        for (int t = pair; t < tiles; t += npairs, ++it) {
            const int buf = it & 1;
            const bool acc_ok =
                __all_sync(0xffffffffu, tc::mbar_wait(&accf[buf], (uint32_t)(it >> 1) & 1u, p.err, tc::ERR_WAIT_ACC));
            if (!acc_ok) break;
            tc::tc_fence_after();
            const int mb = (t / ntiles) * 2 + rk, nt = t % ntiles;
            double sq = epilogue_block<KIND, EPI>(p, tmem, (uint32_t)(buf * BN), (long long)mb * BM, nt * BN, q, cbeg,
                                                  cend, Mtot);
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                if (rk == 0) tc::mbar_arrive(&acce[buf]);
                else tc::mbar_arrive_cluster(tc::mapa_shared(tc::smem_u32(&acce[buf]), 0u));
            }
            // one partial sum per warp slot and 128-row block (a block past the last row writes nothing)
            if (EPI == TC_EPI_FINAL && p.e.partial) {
                for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, off);
                if (lane == 0 && mb < mtiles) {
                    double* pp = p.e.partial + ((size_t)nt * mtiles + mb) * NEPI;
                    pp[h * 4 + q] = sq;
                    if (NE == 4) pp[4 + q] = 0.0;
                }
            }
        }
    } else {
        // ---- kind 2: the split warps of both CTAs write the low parts of their X tiles
        const int tsp = threadIdx.x - 32 * (2 + NE);
        long long g = 0;
        bool ok = true;
        for (int t = pair; t < tiles && ok; t += npairs)
            for (int kb = 0; kb < kblocks && ok; ++kb, ++g) {
                const int st = (int)(g % NST);
                ok = __all_sync(0xffffffffu,
                                tc::mbar_wait(&afull[st], (uint32_t)(g / NST) & 1u, p.err, tc::ERR_WAIT_FULL));
                if (!ok) break;
                split_tile_lo(sA(st), sAlo(st), tsp);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    if (rk == 0) tc::mbar_arrive(&split[st]);
                    else tc::mbar_arrive_cluster(tc::mapa_shared(tc::smem_u32(&split[st]), 0u));
                }
            }
    }
    tc::tc_fence_before();
    // neither CTA frees its shared memory or TMEM while the pair still uses it
    tc::cluster_sync();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc_pair(tmem, tcols);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    }
    return fn;
}

size_t smem_bytes(int kind, bool pair, int BN) {
    // the ring, then at most 37 barriers and the TMEM slot
    return 1024 + (size_t)n_stages(kind, pair, BN) * stage_bytes(kind, pair, BN) + 512;
}

// the largest ring each form of a kind may use (single CTA: BN up to 256 for kinds 0, 1, up to 64 for 2)
size_t smem_max(int kind, bool pair) {
    if (pair) return std::max(smem_bytes(kind, true, 128), smem_bytes(kind, true, 256));
    return smem_bytes(kind, false, kind == 2 ? 64 : 256);
}

// SMs of the current device (one persistent CTA each)
int sm_count() {
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { cudaGetLastError(); return 148; }
    if (!cached[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) { cudaGetLastError(); n = 148; }
        cached[dev] = n;
    }
    return cached[dev];
}

template <int KIND, int EPI>
sfde_status launch(sfde_ctx* c, const CUtensorMap& A, const CUtensorMap& B, const CUtensorMap& Blo, const TcArgs& p,
                   cudaStream_t s, int nr, int nc, int nout) {
    static bool attr = false;   // the dynamic shared-memory limit, once per instantiation
    if (!attr) {
        SFDE_CUDA(cudaFuncSetAttribute(k_tc_slice_gemm<KIND, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_max(KIND, false)));
        SFDE_CUDA(cudaFuncSetAttribute(k_tc_slice_gemm_pair<KIND, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_max(KIND, true)));
        attr = true;
    }
    const long long rows = (long long)p.batch * p.R;
    const long long mtiles = (rows + BM - 1) / BM, ntiles = p.Cout / p.BN;
    const int slot = c ? sfde_prof_begin(c) : -1;
    const bool pair = pair_form(KIND, p.BN, p.Cout);
    if (KIND == 2 && !pair && p.BN > 64) return SFDE_EINVAL;
    if (pair) {
        // one CTA pair per two SMs, at most one per pair tile
        const long long pairs = std::min<long long>(((mtiles + 1) / 2) * ntiles, sm_count() / 2);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(2 * pairs), 1, 1);
        cfg.blockDim = dim3(NTHREADS, 1, 1);
        cfg.dynamicSmemBytes = smem_bytes(KIND, true, p.BN);
        cfg.stream = s;
        cudaLaunchAttribute attr_c[1];
        attr_c[0].id = cudaLaunchAttributeClusterDimension;
        attr_c[0].val.clusterDim.x = 2;
        attr_c[0].val.clusterDim.y = 1;
        attr_c[0].val.clusterDim.z = 1;
        cfg.attrs = attr_c;
        cfg.numAttrs = 1;
        SFDE_CUDA(cudaLaunchKernelEx(&cfg, k_tc_slice_gemm_pair<KIND, EPI>, A, B, Blo, p));
    } else {
        const unsigned grid = (unsigned)std::min<long long>(mtiles * ntiles, sm_count());
        k_tc_slice_gemm<KIND, EPI><<<grid, NTHREADS, smem_bytes(KIND, false, p.BN), s>>>(A, B, Blo, p);
    }
    if (c) {
        const double b = p.batch, esz = KIND == 0 ? 2.0 : 4.0;
        const double extra = EPI == TC_EPI_FINAL ? ((p.e.g ? 1.0 : 0.0) + (p.e.utgt ? 1.0 : 0.0)) * b * nr * nout : 0.0;
        // kind 2 streams the fixed matrix twice (high and low parts)
        sfde_prof_end(c, slot, 2, 2.0 * b * nr * nc * nout,
                      esz * (b * nr * nc + b * nr * nout + (KIND == 2 ? 2.0 : 1.0) * nc * nout + extra));
        sfde_count_launch(c);
    }
    SFDE_CUDA(cudaGetLastError());
    return SFDE_OK;
}

}  // namespace

int sfde_tc_partials_per_tile() { return NEPI; }

int sfde_tc_tile_n(int cout) { return cout <= 256 ? cout : (cout % 256 == 0 ? 256 : 128); }

// Raise the dynamic shared-memory limit of every instantiation up front (outside any stream capture).
template <int KIND, int EPI>
sfde_status prepare_one() {
    SFDE_CUDA(cudaFuncSetAttribute(k_tc_slice_gemm<KIND, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem_max(KIND, false)));
    SFDE_CUDA(cudaFuncSetAttribute(k_tc_slice_gemm_pair<KIND, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem_max(KIND, true)));
    return SFDE_OK;
}

sfde_status sfde_tc_prepare() {
    SFDE_TRY((prepare_one<0, TC_EPI_STORE>()));
    SFDE_TRY((prepare_one<0, TC_EPI_SCALE>()));
    SFDE_TRY((prepare_one<0, TC_EPI_FINAL>()));
    SFDE_TRY((prepare_one<1, TC_EPI_STORE>()));
    SFDE_TRY((prepare_one<1, TC_EPI_SCALE>()));
    SFDE_TRY((prepare_one<1, TC_EPI_FINAL>()));
    SFDE_TRY((prepare_one<2, TC_EPI_STORE>()));
    SFDE_TRY((prepare_one<2, TC_EPI_SCALE>()));
    SFDE_TRY((prepare_one<2, TC_EPI_FINAL>()));
    return SFDE_OK;
}

sfde_status sfde_tc_map_slices(CUtensorMap* map, const void* base, int esz, int K, int R, int ds,
                               long long nslices) {
    auto fn = encode_fn();
    if (!fn) return SFDE_EUNSUPPORTED;
    if (ds < 1 || nslices < ds || ((uintptr_t)base & 15)) return SFDE_EINVAL;
    const CUtensorMapDataType dt = esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    cuuint64_t dims[4] = {(cuuint64_t)K, (cuuint64_t)R, (cuuint64_t)ds, (cuuint64_t)(nslices / ds)};
    cuuint64_t strides[3] = {(cuuint64_t)K * esz, (cuuint64_t)R * K * esz, (cuuint64_t)ds * R * K * esz};
    cuuint32_t box[4] = {(cuuint32_t)(128 / esz), (cuuint32_t)(R < BM ? R : BM), 1u, (cuuint32_t)(R < BM ? BM / R : 1)};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = fn(map, dt, 4, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? SFDE_OK : SFDE_EINVAL;
}

sfde_status sfde_tc_map_matrix(CUtensorMap* map, const void* matT, int esz, int K, int N) {
    return sfde_tc_map_matrix_rows(map, matT, esz, K, N, sfde_tc_tile_n(N));
}

// the B operand of the slice GEMM: BN rows per box, or BN/2 in the CTA-pair form
sfde_status sfde_tc_map_gemm_matrix(CUtensorMap* map, const void* matT, int kind, int K, int N) {
    const int bn = sfde_tc_tile_n(N);
    return sfde_tc_map_matrix_rows(map, matT, kind == 0 ? 2 : 4, K, N, pair_form(kind, bn, N) ? bn / 2 : bn);
}

sfde_status sfde_tc_map_matrix_rows(CUtensorMap* map, const void* matT, int esz, int K, int N, int rows) {
    if (rows < 1 || rows > 256) return SFDE_EINVAL;
    auto fn = encode_fn();
    if (!fn) return SFDE_EUNSUPPORTED;
    const CUtensorMapDataType dt = esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)N};
    cuuint64_t strides[1] = {(cuuint64_t)K * esz};
    cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, dt, 2, const_cast<void*>(matT), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? SFDE_OK : SFDE_EINVAL;
}

sfde_status sfde_tc_gemm(sfde_ctx* c, int kind, int epi, const CUtensorMap& A, const CUtensorMap& B, const TcArgs& p,
                         cudaStream_t s, int nr, int nc, int nout, const CUtensorMap* Blo) {
    if (kind == 2 && !Blo) return SFDE_EINVAL;
    const CUtensorMap& L = Blo ? *Blo : B;
    if (kind == 0) {
        if (epi == TC_EPI_STORE) return launch<0, TC_EPI_STORE>(c, A, B, L, p, s, nr, nc, nout);
        if (epi == TC_EPI_SCALE) return launch<0, TC_EPI_SCALE>(c, A, B, L, p, s, nr, nc, nout);
        return launch<0, TC_EPI_FINAL>(c, A, B, L, p, s, nr, nc, nout);
    }
    if (kind == 1) {
        if (epi == TC_EPI_STORE) return launch<1, TC_EPI_STORE>(c, A, B, L, p, s, nr, nc, nout);
        if (epi == TC_EPI_SCALE) return launch<1, TC_EPI_SCALE>(c, A, B, L, p, s, nr, nc, nout);
        return launch<1, TC_EPI_FINAL>(c, A, B, L, p, s, nr, nc, nout);
    }
    if (epi == TC_EPI_STORE) return launch<2, TC_EPI_STORE>(c, A, B, L, p, s, nr, nc, nout);
    if (epi == TC_EPI_SCALE) return launch<2, TC_EPI_SCALE>(c, A, B, L, p, s, nr, nc, nout);
    return launch<2, TC_EPI_FINAL>(c, A, B, L, p, s, nr, nc, nout);
}

namespace {
// the low parts lo(x) = x - hi(x) of n FP32 values (see tf32_lo)
__global__ void k_tf32_lo(const float* src, float* dst, size_t n) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        dst[e] = tf32_lo(src[e]);
}
}  // namespace

sfde_status sfde_tc_lo_parts(const float* src, float* dst, size_t n, cudaStream_t s) {
    const unsigned grid = (unsigned)std::min<size_t>((n + 255) / 256, 4 * 152);
    k_tf32_lo<<<grid < 1 ? 1 : grid, 256, 0, s>>>(src, dst, n);
    SFDE_CUDA(cudaGetLastError());
    return SFDE_OK;
}

extern "C" sfde_status sfde_debug_tc_gemm(int kind, const void* X, long long nslices, int s0, int ds, int batch,
                                         int R, int C, const void* MatT, int Cout, void* Out, int* err_out,
                                         int reps, float* ms_out) {
    if (kind < 0 || kind > 2 || !X || !MatT || !Out || batch < 1 || R < 32 || R % 32 || C < 1 ||
        Cout < 32 || Cout % 32 || ds < 1 || s0 < 0 || s0 + (long long)(batch - 1) * ds >= nslices)
        return SFDE_EINVAL;
    if (R > 128 && R % 128) return SFDE_EINVAL;
    const int esz = kind == 0 ? 2 : 4;
    CUtensorMap A, B, Bl = {};
    SFDE_TRY(sfde_tc_map_slices(&A, X, esz, C, R, ds, nslices));
    SFDE_TRY(sfde_tc_map_gemm_matrix(&B, MatT, kind, C, Cout));
    float* lo = nullptr;   // kind 2: the low parts of Mat^T
    if (kind == 2) {
        SFDE_CUDA(cudaMalloc(&lo, sizeof(float) * (size_t)Cout * C));
        SFDE_TRY(sfde_tc_lo_parts((const float*)MatT, lo, (size_t)Cout * C, nullptr));
        SFDE_TRY(sfde_tc_map_gemm_matrix(&Bl, lo, kind, C, Cout));
    }
    int* err = nullptr;
    SFDE_CUDA(cudaMalloc(&err, sizeof(int)));
    SFDE_CUDA(cudaMemset(err, 0, sizeof(int)));
    TcArgs p{};
    p.R = R; p.C = C; p.Cout = Cout; p.batch = batch; p.BN = sfde_tc_tile_n(Cout); p.s0 = s0; p.ds = ds;
    p.out = Out; p.out_stride = (long long)Cout * R;
    p.err = err;
    sfde_status st = sfde_tc_gemm(nullptr, kind, TC_EPI_STORE, A, B, p, nullptr, 0, 0, 0, kind == 2 ? &Bl : nullptr);
    cudaError_t e = cudaDeviceSynchronize();
    if (st == SFDE_OK && e == cudaSuccess && ms_out && reps > 0) {
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, nullptr);
        for (int i = 0; i < reps && st == SFDE_OK; ++i)
            st = sfde_tc_gemm(nullptr, kind, TC_EPI_STORE, A, B, p, nullptr, 0, 0, 0, kind == 2 ? &Bl : nullptr);
        cudaEventRecord(e1, nullptr);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        *ms_out = ms / reps;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    int herr = 0;
    cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(err);
    cudaFree(lo);
    if (err_out) *err_out = herr;
    if (e != cudaSuccess) { sfde_set_last_cuda_error(e, "debug tc gemm", __FILE__, __LINE__); return SFDE_ECUDA; }
    if (st == SFDE_OK && herr) return SFDE_ETIMEOUT;
    return st;
}

namespace {

// One CTA waits, with the tensor-core kernels' bounded wait, on an mbarrier that nothing arrives at
// (no copy or product is issued); the wait runs out after limit_ns and records the error code.
__global__ void k_wait_nothing(int* err, unsigned long long limit_ns, unsigned long long* waited_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long t0 = tc::globaltimer();
        const bool ok = tc::mbar_wait_ns(&bar, 0, err, tc::ERR_WAIT_FULL, limit_ns);
        *waited_ns = ok ? 0ull : tc::globaltimer() - t0;
    }
}

}  // namespace

extern "C" sfde_status sfde_debug_wait_timeout(unsigned long long limit_ns, int* err_out, double* waited_s) {
    if (limit_ns < 1000ull || limit_ns > 2000000000ull) return SFDE_EINVAL;
    int* err = nullptr;
    unsigned long long* w = nullptr;
    SFDE_CUDA(cudaMalloc(&err, sizeof(int)));
    cudaError_t e = cudaMalloc(&w, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(int));
    if (e == cudaSuccess) {
        k_wait_nothing<<<1, 32>>>(err, limit_ns, w);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int herr = 0;
    unsigned long long hw = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&hw, w, sizeof(hw), cudaMemcpyDeviceToHost);
    cudaFree(err);
    cudaFree(w);
    if (e != cudaSuccess) { sfde_set_last_cuda_error(e, "debug wait timeout", __FILE__, __LINE__); return SFDE_ECUDA; }
    if (err_out) *err_out = herr;
    if (waited_s) *waited_s = hw * 1e-9;
    return herr ? SFDE_ETIMEOUT : SFDE_OK;
}
