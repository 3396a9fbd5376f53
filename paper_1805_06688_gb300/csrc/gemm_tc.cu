// Tensor-core slice GEMM for the mixed-precision steps: Out_b = (X_b Mat)^T, as in step_fp64.cu,
// with BF16 (tcgen05.mma kind::f16) or TF32 (kind::tf32) operands and FP32 accumulation in TMEM.
//
// One CTA computes a 128 x BN tile of the stacked product (rows = batch slices x R rows each):
//   * warp 0 / lane 0 streams K-blocks of 128 bytes (64 BF16 or 32 FP32 values) of X and of Mat^T
//     into a 4-stage ring of 128-byte-swizzled shared-memory tiles with TMA;
//   * warp 1 / lane 0 issues four tcgen05.mma (K = 16 BF16 / 8 TF32 each) per K-block into the TMEM
//     accumulator and releases the stage with tcgen05.commit;
//   * all four warps read the accumulator back (tcgen05.ld, 32 lanes x 32 columns at a time), apply
//     the fused epilogue and store the transposed tile: lanes hold consecutive rows, so each store
//     instruction writes 32 consecutive elements.
// X is addressed through a 4-D tensor map {K, R, ds, S/ds} so that a batch of slices taken every
// ds-th time point (a relaxation sweep) is one rectangular box per tile, also when R < 128.
#include <math.h>
#include <string.h>

#include <cudaTypedefs.h>

#include "sfde_internal.cuh"
#include "tc_common.cuh"

namespace {

constexpr int BM = 128;
constexpr int STAGES = 4;
constexpr int A_STAGE_BYTES = BM * 128;
constexpr int TMEM_COLS = 256;

template <typename T> struct StoreT;
template <> struct StoreT<__nv_bfloat16> {
    static __device__ __forceinline__ __nv_bfloat16 from(float v) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ float to(__nv_bfloat16 v) { return __bfloat162float(v); }
};
template <> struct StoreT<float> {
    static __device__ __forceinline__ float from(float v) { return sfde_round_tf32(v); }
    static __device__ __forceinline__ float to(float v) { return v; }
};

template <int KIND, typename T, int EPI>
__global__ void __launch_bounds__(128, 1)
k_tc_slice_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcArgs p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int BN = p.BN;
    const int B_STAGE_BYTES = BN * 128;
    uint8_t* sA = smem;
    uint8_t* sB = smem + STAGES * A_STAGE_BYTES;
    uint64_t* full = (uint64_t*)(sB + STAGES * B_STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* accf = empty + STAGES;
    uint32_t* tmem_slot = (uint32_t*)(accf + 1);
    __shared__ double red[4];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int KB = 128 / (int)sizeof(T);          // K elements per stage
    constexpr int KSTEP_BYTES = 32;                   // one MMA consumes 32 bytes of K
    const int kblocks = (p.C + KB - 1) / KB;
    const long long m0 = (long long)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    const long long Mtot = (long long)p.batch * p.R;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
        tc::mbar_init(accf, 1);
        tc::mbar_fence_init();
        tc::prefetch_tmap(&mapA);
        tc::prefetch_tmap(&mapB);
    }
    if (warp == 0) tc::tmem_alloc(tmem_slot, TMEM_COLS);
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // A-tile coordinates: first slice of the tile and row inside it
    const int b0 = (int)(m0 / p.R);
    const int r0 = (int)(m0 % p.R);
    const int s_first = p.s0 + b0 * p.ds;
    const int c2 = p.s0 % p.ds, c3 = s_first / p.ds;

    bool ok = true;
    if (warp == 0 && lane == 0) {
        for (int kb = 0; kb < kblocks && ok; ++kb) {
            const int st = kb % STAGES;
            const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
            if (kb >= STAGES) ok = tc::mbar_wait(&empty[st], ph ^ 1u, p.err, tc::ERR_WAIT_EMPTY);
            if (!ok) break;
            tc::mbar_arrive_expect_tx(&full[st], (uint32_t)(A_STAGE_BYTES + B_STAGE_BYTES));
            tc::tma_load_4d(sA + st * A_STAGE_BYTES, &mapA, &full[st], kb * KB, r0, c2, c3);
            tc::tma_load_2d(sB + st * B_STAGE_BYTES, &mapB, &full[st], kb * KB, n0);
        }
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = tc::idesc_f32acc(KIND == 0 ? 1u : 2u, BM, BN);
        for (int kb = 0; kb < kblocks && ok; ++kb) {
            const int st = kb % STAGES;
            const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
            ok = tc::mbar_wait(&full[st], ph, p.err, tc::ERR_WAIT_FULL);
            if (!ok) break;
            tc::tc_fence_after();
#pragma unroll
            for (int k = 0; k < 128 / KSTEP_BYTES; ++k) {
                const uint64_t ad = tc::smem_desc_sw128(sA + st * A_STAGE_BYTES + k * KSTEP_BYTES);
                const uint64_t bd = tc::smem_desc_sw128(sB + st * B_STAGE_BYTES + k * KSTEP_BYTES);
                tc::mma<KIND>(tmem, ad, bd, idesc, (kb > 0 || k > 0) ? 1u : 0u);
            }
            tc::mma_commit(&empty[st]);
        }
        if (ok) tc::mma_commit(accf);
    }

    // ---- epilogue (all 128 threads)
    // tcgen05.ld is warp-collective (.sync.aligned): the whole warp reads the accumulator or none of
    // it, so a lane whose bounded wait ran out makes its warp skip the epilogue.
    const bool acc_ok = __all_sync(0xffffffffu, tc::mbar_wait(accf, 0, p.err, tc::ERR_WAIT_ACC));
    tc::tc_fence_after();
    double sq = 0.0;
    if (acc_ok) {
        const long long m = m0 + warp * 32 + lane;
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
        for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (!valid) continue;
            const T* gcol = g ? g + (long long)(n0 + c0) * p.R + r : nullptr;
            const T* ucol = ut ? ut + (long long)(n0 + c0) * p.R + r : nullptr;
            T* ocol = out + (long long)(n0 + c0) * p.R + r;
            // all operand loads of the 32-column chunk are issued before any store: they are
            // independent, so their latencies overlap instead of adding up element by element
            float add[32];
            if (EPI == TC_EPI_SCALE) {
#pragma unroll
                for (int j = 0; j < 32; ++j) add[j] = __ldg(p.e.lamy + n0 + c0 + j);
            } else if (EPI == TC_EPI_FINAL) {
#pragma unroll
                for (int j = 0; j < 32; ++j) add[j] = gcol ? StoreT<T>::to(gcol[(long long)j * p.R]) : 0.f;
                if (ucol) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) add[j] -= StoreT<T>::to(ucol[(long long)j * p.R]);
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
                ocol[(long long)j * p.R] = StoreT<T>::from(x);
            }
        }
    }
    if (EPI == TC_EPI_FINAL && p.e.partial) {
        for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, off);
        if (lane == 0) red[warp] = sq;
    }
    tc::tc_fence_before();
    __syncthreads();
    if (EPI == TC_EPI_FINAL && p.e.partial && threadIdx.x == 0)
        p.e.partial[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = red[0] + red[1] + red[2] + red[3];
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, TMEM_COLS);
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

size_t smem_bytes(int BN) { return 1024 + (size_t)STAGES * (A_STAGE_BYTES + (size_t)BN * 128) + 256; }

template <int KIND, typename T, int EPI>
sfde_status launch(sfde_ctx* c, const CUtensorMap& A, const CUtensorMap& B, const TcArgs& p, cudaStream_t s,
                   int nr, int nc, int nout) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_tc_slice_gemm<KIND, T, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes(256));
        attr = true;
    }
    const long long rows = (long long)p.batch * p.R;
    dim3 grid((unsigned)((rows + BM - 1) / BM), p.Cout / p.BN);
    const int slot = c ? sfde_prof_begin(c) : -1;
    k_tc_slice_gemm<KIND, T, EPI><<<grid, 128, smem_bytes(p.BN), s>>>(A, B, p);
    if (c) {
        const double b = p.batch, esz = sizeof(T);
        const double extra = EPI == TC_EPI_FINAL ? ((p.e.g ? 1.0 : 0.0) + (p.e.utgt ? 1.0 : 0.0)) * b * nr * nout : 0.0;
        sfde_prof_end(c, slot, 2, 2.0 * b * nr * nc * nout,
                      esz * (b * nr * nc + b * nr * nout + (double)nc * nout + extra));
        sfde_count_launch(c);
    }
    SFDE_CUDA(cudaGetLastError());
    return SFDE_OK;
}

}  // namespace

int sfde_tc_tile_n(int cout) { return cout <= 256 ? cout : (cout % 256 == 0 ? 256 : 128); }

// Raise the dynamic shared-memory limit of every instantiation up front (outside any stream capture).
sfde_status sfde_tc_prepare() {
    const int bytes = (int)smem_bytes(256);
    SFDE_CUDA(cudaFuncSetAttribute(k_tc_slice_gemm<0, __nv_bfloat16, TC_EPI_STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    SFDE_CUDA(cudaFuncSetAttribute(k_tc_slice_gemm<0, __nv_bfloat16, TC_EPI_SCALE>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    SFDE_CUDA(cudaFuncSetAttribute(k_tc_slice_gemm<0, __nv_bfloat16, TC_EPI_FINAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    SFDE_CUDA(cudaFuncSetAttribute(k_tc_slice_gemm<1, float, TC_EPI_STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    SFDE_CUDA(cudaFuncSetAttribute(k_tc_slice_gemm<1, float, TC_EPI_SCALE>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    SFDE_CUDA(cudaFuncSetAttribute(k_tc_slice_gemm<1, float, TC_EPI_FINAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
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
                         cudaStream_t s, int nr, int nc, int nout) {
    if (kind == 0) {
        if (epi == TC_EPI_STORE) return launch<0, __nv_bfloat16, TC_EPI_STORE>(c, A, B, p, s, nr, nc, nout);
        if (epi == TC_EPI_SCALE) return launch<0, __nv_bfloat16, TC_EPI_SCALE>(c, A, B, p, s, nr, nc, nout);
        return launch<0, __nv_bfloat16, TC_EPI_FINAL>(c, A, B, p, s, nr, nc, nout);
    }
    if (epi == TC_EPI_STORE) return launch<1, float, TC_EPI_STORE>(c, A, B, p, s, nr, nc, nout);
    if (epi == TC_EPI_SCALE) return launch<1, float, TC_EPI_SCALE>(c, A, B, p, s, nr, nc, nout);
    return launch<1, float, TC_EPI_FINAL>(c, A, B, p, s, nr, nc, nout);
}

extern "C" sfde_status sfde_debug_tc_gemm(int kind, const void* X, long long nslices, int s0, int ds, int batch,
                                         int R, int C, const void* MatT, int Cout, void* Out, int* err_out,
                                         int reps, float* ms_out) {
    if ((kind != 0 && kind != 1) || !X || !MatT || !Out || batch < 1 || R < 32 || R % 32 || C < 1 ||
        Cout < 32 || Cout % 32 || ds < 1 || s0 < 0 || s0 + (long long)(batch - 1) * ds >= nslices)
        return SFDE_EINVAL;
    if (R > 128 && R % 128) return SFDE_EINVAL;
    const int esz = kind == 0 ? 2 : 4;
    CUtensorMap A, B;
    SFDE_TRY(sfde_tc_map_slices(&A, X, esz, C, R, ds, nslices));
    SFDE_TRY(sfde_tc_map_matrix(&B, MatT, esz, C, Cout));
    int* err = nullptr;
    SFDE_CUDA(cudaMalloc(&err, sizeof(int)));
    SFDE_CUDA(cudaMemset(err, 0, sizeof(int)));
    TcArgs p{};
    p.R = R; p.C = C; p.Cout = Cout; p.batch = batch; p.BN = sfde_tc_tile_n(Cout); p.s0 = s0; p.ds = ds;
    p.out = Out; p.out_stride = (long long)Cout * R;
    p.err = err;
    sfde_status st = sfde_tc_gemm(nullptr, kind, TC_EPI_STORE, A, B, p, nullptr);
    cudaError_t e = cudaDeviceSynchronize();
    if (st == SFDE_OK && e == cudaSuccess && ms_out && reps > 0) {
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, nullptr);
        for (int i = 0; i < reps && st == SFDE_OK; ++i) st = sfde_tc_gemm(nullptr, kind, TC_EPI_STORE, A, B, p, nullptr);
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
    if (err_out) *err_out = herr;
    if (e != cudaSuccess) { sfde_set_last_cuda_error(e, "debug tc gemm", __FILE__, __LINE__); return SFDE_ECUDA; }
    if (st == SFDE_OK && herr) return SFDE_ETIMEOUT;
    return st;
}
