// The FP64-accurate space-time residual of Eq. (2.4),
//     rho_n = F_n + M_h (U_{n-1} - U_n) - tau_n K (U_{n-1} + U_n),   n = 1..N_t,
// assembled in integer arithmetic around two digit-split BF16 tensor-core products.
//
// The FP64 pipe of this GPU runs at about 1/64 of the FP32 rate, so every FP64 operation per
// element of the space-time grid costs about as much as a whole tensor-core product.  Here the
// iterate is read once as FP64 bit patterns and everything up to the final combination is exact
// integer work:
//   1. per time point, E_n with max |U_n| < 2^{E_n} (an integer max over the bit patterns);
//   2. per pair (n-1, n) with E = max(E_{n-1}, E_n): the fixed-point values fix(u) = round(u 2^{54-E})
//      (|fix| <= 2^54) and V = fix(U_{n-1}) + fix(U_n), exact, written as seven balanced base-256
//      digits of V (BF16-exact, no remainder) in row-major and in transposed order;
//   3. Z1 = V (K_x h_y/6 A_x) and Z2 = (K_y h_x/6 A_y) V on the tensor cores (ozaki.cu, up to 28
//      digit products: 4 to 7 digits per operand as the refinement step needs), each an int64 in
//      units of 2^{-52} of the operands' scales;
//   4. with the mass matrices M = (h/6) tridiag(1, 4, 1) in both directions (they commute with the
//      products: A_y (V M_x) = (A_y V) M_x),
//          K V = (1,4,1)_y Z1 + (1,4,1)_x Z2      (integer, aligned to a common power of two),
//          M_h (U_{n-1} - U_n) = (h_x h_y / 36) (1,4,1)_y (1,4,1)_x du,  du = fix(U_{n-1}) - fix(U_n)
//      (du written by step 2 as int64),
//      and rho = F + c_m S9 - tau c_s S formed exactly in 128-bit integers (the load F formed in
//      FP64 and rounded to the common unit; the FP64 form where it does not fit) and converted to
//      FP32; the sum of rho^2 is taken over the stored FP32 values.
// Pairs of two zero slices (the first iterate's n >= 2) skip steps 2-4: their residual is the load
// alone, written with the values the general form gives them (k_load_resid).
// The fixed-point grid of a pair is 2^{E-54}: values far below the slice maximum keep an absolute
// accuracy of 2^{-55} max|U|, the scale at which an FP64 product's rounding errors enter the residual.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <climits>

#include "f64_round.cuh"
#include "sfde_internal.cuh"

namespace {

// max over one slice of |u| as a bit pattern -> E with max|u| < 2^E (2047 exponent: not finite)
__global__ void __launch_bounds__(256) k_slice_maxexp(const double* __restrict__ U, size_t P2, int* __restrict__ E) {
    const unsigned long long* u = (const unsigned long long*)(U + (size_t)blockIdx.x * P2);
    unsigned long long mx = 0;
    for (size_t e = threadIdx.x * 2; e < P2; e += blockDim.x * 2) {
        const ulonglong2 v = *(const ulonglong2*)(u + e);
        mx = max(mx, max(v.x & 0x7FFFFFFFFFFFFFFFull, v.y & 0x7FFFFFFFFFFFFFFFull));
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __shared__ unsigned long long red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = max(mx, red[w]);
        mx = max(mx, red[0]);
        E[blockIdx.x] = (int)(mx >> 52) - 1022;   // 1.f 2^{ex-1023} < 2^{ex-1022}
    }
}

// round(u 2^{54-E}) for |u| < 2^E from the bit pattern (integer operations only); |result| <= 2^54
__device__ __forceinline__ long long fixp(unsigned long long bits, int E) {
    const int ex = (int)((bits >> 52) & 0x7FF);
    if (ex == 0) return 0;                                    // zero or below 2^-1022
    const long long m = (long long)((bits & 0xFFFFFFFFFFFFFull) | (1ull << 52));
    const int sh = E + 1021 - ex;                             // >= -1 because |u| < 2^E
    long long r;
    if (sh <= 0) r = m << (-sh);
    else if (sh >= 62) r = 0;
    else r = (m + (1ll << (sh - 1))) >> sh;
    return (bits >> 63) ? -r : r;
}

// BF16 bit pattern of a small integer |d| <= 256 (exact): 1.5 2^23 + d is exact in FP32
__device__ __forceinline__ uint16_t bf16_of_int(int d) {
    const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
    return (uint16_t)(__float_as_uint(f) >> 16);
}

constexpr int ND = 7;  // digits per operand

// Balanced base-256 digits of x (|x| <= 2^T, T >= 56): x = d_1 2^{T-8} + sum_{p=2..7} d_p 2^{T-8p} + r
// with d_1 in [-256, 256], d_p in [-128, 127] and |r| <= 2^{T-57} (r = 0 for T = 56).  Adding
// C = sum_{p>=2} 128 2^{T-8p} (+ 2^{T-57} to round) turns every lower digit into an unsigned byte, so
// each digit is one shift and mask.
template <int T>
__device__ __forceinline__ void split7(long long x, uint16_t (&bf)[ND]) {
    static_assert(T >= 56 && T <= 61, "digit frame");
    constexpr unsigned long long C = 128ull * ((1ull << (T - 16)) + (1ull << (T - 24)) + (1ull << (T - 32)) +
                                               (1ull << (T - 40)) + (1ull << (T - 48)) + (1ull << (T - 56))) +
                                     (T > 56 ? (1ull << (T > 56 ? T - 57 : 0)) : 0ull);
    const long long xp = x + (long long)C;
    bf[0] = bf16_of_int((int)(xp >> (T - 8)));
#pragma unroll
    for (int p = 1; p < ND; ++p) bf[p] = bf16_of_int((int)((unsigned long long)(xp >> (T - 8 * (p + 1))) & 255u) - 128);
}

// V = fix(U_{n-1}) + fix(U_n) and du = fix(U_{n-1}) - fix(U_n) for one 32 x 32 tile of pair b
// (n = n0 + b): the digits of V row-major [b][j][i] (rows of the A_x product) and transposed
// [b][i][j] (rows of the A_y product), du as int64 [b][j][i] (the mass term).  Thread t takes four
// consecutive columns 4 (t % 8).. of row t / 8, so every access moves 8 or 16 bytes.
__global__ void __launch_bounds__(256) k_split_pair(const double* __restrict__ U, const int* __restrict__ En, int n0,
                                                    int Px, int Py, uint16_t* __restrict__ dV, uint16_t* __restrict__ dVt,
                                                    long long* __restrict__ du, long long plane, int nd) {
    __shared__ uint16_t dt[ND][32][34];   // digits [p][i][j]
    const int b = blockIdx.z, n = n0 + b;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int q = threadIdx.x & 7, r = threadIdx.x >> 3;
    const int E = max(En[n - 1], En[n]);
    const size_t P2 = (size_t)Px * Py;
    const size_t e = (size_t)(j0 + r) * Px + i0 + 4 * q;
    const ulonglong2* Un = (const ulonglong2*)(U + (size_t)n * P2 + e);
    const ulonglong2* Um = (const ulonglong2*)(U + (size_t)(n - 1) * P2 + e);
    const ulonglong2 n01 = __ldg(Un), n23 = __ldg(Un + 1), m01 = __ldg(Um), m23 = __ldg(Um + 1);
    const unsigned long long un[4] = {n01.x, n01.y, n23.x, n23.y}, um[4] = {m01.x, m01.y, m23.x, m23.y};
    uint16_t bf[4][ND];
    long long d4[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const long long fm = fixp(um[c], E), fn = fixp(un[c], E);
        d4[c] = fm - fn;
        split7<56>(fm + fn, bf[c]);     // |V| <= 2^55: every digit within [-128, 128], exact
    }
    const size_t o = (size_t)b * P2 + e;
    *(longlong2*)(du + o) = make_longlong2(d4[0], d4[1]);
    *(longlong2*)(du + o + 2) = make_longlong2(d4[2], d4[3]);
#pragma unroll
    for (int p = 0; p < ND; ++p)
        if (p < nd) {
            uint2 w;
            w.x = (uint32_t)bf[0][p] | ((uint32_t)bf[1][p] << 16);
            w.y = (uint32_t)bf[2][p] | ((uint32_t)bf[3][p] << 16);
            *(uint2*)(dV + p * plane + o) = w;
#pragma unroll
            for (int c = 0; c < 4; ++c) dt[p][4 * q + c][r] = bf[c][p];
        }
    __syncthreads();
    // transposed: row i = i0 + r, columns j = j0 + 4q .. 4q + 3
    const size_t ot = (size_t)b * P2 + (size_t)(i0 + r) * Py + j0 + 4 * q;
#pragma unroll
    for (int p = 0; p < ND; ++p)
        if (p < nd) {
            const uint32_t* s2 = (const uint32_t*)&dt[p][r][4 * q];
            *(uint2*)(dVt + p * plane + ot) = make_uint2(s2[0], s2[1]);
        }
}

// Exact int64 -> FP64 conversion, round to nearest even, from integer operations (the conversion
// instruction runs on the slow FP64 pipe).
__device__ __forceinline__ double i64_to_f64(long long x) {
    if (x == 0) return 0.0;
    const unsigned long long sgn = (unsigned long long)x & 0x8000000000000000ull;
    const unsigned long long a = x < 0 ? 0ull - (unsigned long long)x : (unsigned long long)x;
    int e = 63 - __clzll((long long)a);                   // a in [2^e, 2^{e+1})
    unsigned long long m;
    if (e <= 52) {
        m = a << (52 - e);
    } else {
        const int sh = e - 52;
        const unsigned long long rem = a & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        m = a >> sh;
        if (rem > half || (rem == half && (m & 1ull))) ++m;
        if (m == (1ull << 53)) { m >>= 1; ++e; }
    }
    return __longlong_as_double((long long)(sgn | ((unsigned long long)(e + 1023) << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

// round(f 2^-ec) as a 128-bit integer from the bit pattern of f (integer operations only); false when
// |f| 2^-ec would reach 2^124 (the caller then keeps the FP64 form) or f is not finite
__device__ __forceinline__ bool f64_to_i128_scaled(double f, int ec, __int128& out) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(f);
    const int ex = (int)((b >> 52) & 0x7FF);
    if (ex == 0) { out = 0; return true; }                  // zero or below 2^-1022
    if (ex == 0x7FF) return false;
    const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | (1ull << 52));   // f = +-m 2^{ex-1075}
    const int sh = ex - 1075 - ec;
    __int128 v;
    if (sh >= 0) {
        if (sh > 70) return false;                          // m 2^sh < 2^123: clear of 2^124
        v = (__int128)m << sh;
    } else if (sh > -64) {
        v = (m + (1ll << (-sh - 1))) >> (-sh);
    } else {
        v = 0;
    }
    out = (b >> 63) ? -v : v;
    return true;
}

// rounding arithmetic right shift (k >= 0)
__device__ __forceinline__ long long rshr(long long x, int k) {
    if (k <= 0) return x;
    if (k >= 62) return 0;
    return (x + (1ll << (k - 1))) >> k;
}

// c = m 2^e exactly (normal c; m a signed integer of at most 53 bits), or m = 0
__device__ __forceinline__ void split_double(double c, long long& m, int& e) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(c);
    const int ex = (int)((b >> 52) & 0x7FF);
    if (ex == 0) { m = 0; e = 0; return; }
    const long long mm = (long long)((b & 0xFFFFFFFFFFFFFull) | (1ull << 52));
    m = (b >> 63) ? -mm : mm;
    e = ex - 1075;
}

// FP32 of x 2^e (x a 128-bit integer, |x| < 2^127; 2^e = s1 s2 given as two FP32 powers of two)
// within 4 ulp: the four 32-bit words of |x| are converted one by one (32-bit conversions; the
// 64-bit ones run on the slow FP64 pipe) and summed by three FMAs from the top word down (all
// terms of one sign: at most seven roundings of 2^-24 each, no cancellation); the powers of two
// scale exactly unless the result leaves the normal range
__device__ __forceinline__ float i128_to_f32(__int128 x, float s1, float s2) {
    const bool neg = x < 0;
    const unsigned __int128 a = neg ? (unsigned __int128)0 - (unsigned __int128)x : (unsigned __int128)x;
    const unsigned long long hi = (unsigned long long)(a >> 64), lo = (unsigned long long)a;
    const float w = 4294967296.0f;   // 2^32
    float r = __uint2float_rn((unsigned)(hi >> 32));
    r = fmaf(r, w, __uint2float_rn((unsigned)hi));
    r = fmaf(r, w, __uint2float_rn((unsigned)(lo >> 32)));
    r = fmaf(r, w, __uint2float_rn((unsigned)lo));
    r = r * s1 * s2;
    return neg ? -r : r;
}

// rho for one 32 x 32 tile of pair b.  Z1 = T1[b][i][j] counts 2^{E+ex-50+zsx} and Z2 = T3[b][j][i]
// counts 2^{E+ey-50+zsy} (V / 2^56 times the matrix over 2^e, in units of 2^{zs-52} with zs the
// product's shift for its contraction length), du = fix(U_{n-1}) - fix(U_n) counts 2^{E-54}.
// |Z| <= 2^58, so (1,4,1) Z stays below 2^61, and both terms are halved at least once before they
// are added.  The mass stencil (1,4,1)_y (1,4,1)_x is applied separably (rows first, in shared
// memory).  Without a load term rho = c_m S9 + c_s S is formed in integers: c_m and c_s are FP64
// numbers, i.e. 53-bit integers times powers of two.  Both are brought to a common power of two
// 2^ec by shifting the mantissa of the coarser one left by up to 10 bits (below 2^63), so both
// products are exact 128-bit integers below 2^126 with no shift per element (when the two units
// differ by more than 2^10 the finer product is shifted right, keeping its bits down to 2^-62 of
// the coarser unit, far below the fixed-point grid's own resolution), added exactly, and converted
// to FP32 within 4 ulp from 32-bit words -- no FP64 arithmetic per element (the FP64 pipe runs at
// about 1/64 of the FP32 rate).  A load term F_n is formed in FP64 (one FMA per separable term, the time weight
// times the y factor taken once per row) and added as round(F 2^-ec), a 128-bit integer in the same
// unit (its rounding, half a unit, lies far below F's own FP64 rounding); where F 2^-ec would not fit,
// or both slices of the pair are zero (no unit: c_m = c_s = 0), the FP64 form F + c_m S9 + c_s S is
// kept.  Writes rho (BF16 or TF32-rounded FP32), zero outside the interior nodes, and one FP64 sum of
// rho^2 per block.
template <typename OT, bool TF32R>
__global__ void __launch_bounds__(256, 4) k_combine_int(
    const long long* __restrict__ T1, const long long* __restrict__ T3, const long long* __restrict__ DU,
    const int* __restrict__ En, int n0, int Px, int Py, int nx, int ny, double cmass, int ex, int ey, int zsx, int zsy,
    const double* __restrict__ dt, int rank, const double* __restrict__ time_w, const double* __restrict__ bxn,
    const double* __restrict__ byn, const double* __restrict__ Fd, OT* __restrict__ rout, long long rout_stride,
    double* __restrict__ partial) {
    __shared__ long long t1[32][35];      // Z1 rows i0.., columns j0-1 .. j0+32
    __shared__ long long t3[32][35];      // Z2 rows j0.., columns i0-1 .. i0+32
    __shared__ long long du[34][35];      // du, rows j0-1.., columns i0-1..
    __shared__ long long rs[34][33];      // (1,4,1)_x du, rows j0-1.., columns i0..
    __shared__ double red[8];
    __shared__ double cst[2];             // c_m 2^{E-54}, -tau 2^u
    __shared__ long long cmi[2];          // their integer mantissas, shifted to the unit 2^ec
    __shared__ int csh[2];                // per term: right shift of the product
    __shared__ float csc[2];              // 2^ec as two FP32 powers of two
    __shared__ int cec;                   // ec
    __shared__ int cdeg;                  // both coefficients zero (two zero slices): no integer unit
    __shared__ double fy[SFDE_MAX_RANK][32];   // time weight x y factor of each load term, per row
    const int b = blockIdx.z, n = n0 + b;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int E = max(En[n - 1], En[n]);
    const size_t P2 = (size_t)Px * Py;
    // all global loads of the block are issued before any of them is used (compile-time trip
    // counts, register staging), so their latencies overlap
    const long long* T1b = T1 + (size_t)b * P2;
    const long long* T3b = T3 + (size_t)b * P2;
    const long long* DUb = DU + (size_t)b * P2;
    long long a1[4][2], a3[4][2], ad[5][2];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = tx + 32 * h;
            const int j = j0 + c - 1, i = i0 + c - 1;
            a1[k][h] = (c < 34 && j >= 0 && j < Py) ? __ldg(T1b + (size_t)(i0 + ty + 8 * k) * Py + j) : 0;
            a3[k][h] = (c < 34 && i >= 0 && i < Px) ? __ldg(T3b + (size_t)(j0 + ty + 8 * k) * Px + i) : 0;
        }
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int rr = ty + 8 * k, c = tx + 32 * h;
            const int j = j0 + rr - 1, i = i0 + c - 1;
            const bool in = rr < 34 && c < 34 && j >= 0 && j < Py && i >= 0 && i < Px;
            ad[k][h] = in ? __ldg(DUb + (size_t)j * Px + i) : 0;     // zero outside the grid
        }
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (tx + 32 * h < 34) {
                t1[ty + 8 * k][tx + 32 * h] = a1[k][h];
                t3[ty + 8 * k][tx + 32 * h] = a3[k][h];
            }
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int rr = ty + 8 * k, c = tx + 32 * h;
            if (rr < 34 && c < 34) du[rr][c] = ad[k][h];
        }
    const int u1 = E + ex - 50 + zsx, u2 = E + ey - 50 + zsy, u = max(u1, u2) + 1;
    if (tx == 0 && ty == 0) {
        cst[0] = ldexp(cmass, E - 54);
        cst[1] = ldexp(-0.5 * dt[n - 1], u);
        // |S9| < 2^61, |S| < 2^62, |m| < 2^53 shifted left by at most 10 bits: products below 2^125
        long long mm, ms;
        int em, es;
        split_double(cst[0], mm, em);
        split_double(cst[1], ms, es);
        cdeg = mm == 0 && ms == 0;
        if (mm == 0) em = es;
        if (ms == 0) es = em;
        const int ec = max(em, es) - 10;
        cmi[0] = em >= ec ? (long long)((unsigned long long)mm << (em - ec)) : mm;
        cmi[1] = es >= ec ? (long long)((unsigned long long)ms << (es - ec)) : ms;
        csh[0] = em >= ec ? 0 : min(ec - em, 127);
        csh[1] = es >= ec ? 0 : min(ec - es, 127);
        const int e1 = min(max(ec, -126), 127);
        csc[0] = ldexpf(1.0f, e1);
        csc[1] = ldexpf(1.0f, min(max(ec - e1, -126), 127));
        cec = ec;
    }
    if (ty == 0)
        for (int q = 0; q < rank; ++q) {
            const int j = j0 + tx;
            fy[q][tx] = j < Py ? time_w[(size_t)(n - 1) * rank + q] * byn[(size_t)q * Py + j] : 0.0;
        }
    __syncthreads();
    for (int rr = ty; rr < 34; rr += 8) rs[rr][tx] = du[rr][tx] + 4 * du[rr][tx + 1] + du[rr][tx + 2];
    __syncthreads();
    const double cm = cst[0], cs = cst[1];
    const long long mm = cmi[0], ms = cmi[1];
    const int rm = csh[0], rsd = csh[1];
    const float sc1 = csc[0], sc2 = csc[1];
    const bool finite = E < 1024;
    const int i = i0 + tx;
    const int ec = cec;
    const bool deg = cdeg != 0;
    double bxi[SFDE_MAX_RANK];
#pragma unroll
    for (int q = 0; q < SFDE_MAX_RANK; ++q) bxi[q] = (q < rank && i < Px) ? bxn[(size_t)q * Px + i] : 0.0;
    float sq = 0.f;   // of the stored values; the norm only decides when the iteration stops
    for (int jj = ty; jj < 32; jj += 8) {
        const int j = j0 + jj;
        float rf = 0.f;
        if (i < nx && j < ny) {
            const long long k1 = t1[tx][jj] + 4 * t1[tx][jj + 1] + t1[tx][jj + 2];
            const long long k2 = t3[jj][tx] + 4 * t3[jj][tx + 1] + t3[jj][tx + 2];
            const long long st = rshr(k1, u - u1) + rshr(k2, u - u2);
            const long long s9 = rs[jj][tx] + 4 * rs[jj + 1][tx] + rs[jj + 2][tx];
            __int128 tm = (__int128)s9 * mm, ts = (__int128)st * ms;
            if (rm) tm >>= rm;     // block-uniform, zero unless the units differ by more than 2^10
            if (rsd) ts >>= rsd;
            __int128 fi = 0;
            bool exact = true;
            if (rank > 0 || Fd) {
                double f = Fd ? Fd[(size_t)(n - 1) * P2 + (size_t)j * Px + i] : 0.0;
#pragma unroll
                for (int q = 0; q < SFDE_MAX_RANK; ++q)
                    if (q < rank) f = fma(fy[q][jj], bxi[q], f);
                exact = !deg && f64_to_i128_scaled(f, ec, fi);
                if (!exact) rf = (float)fma(cm, i64_to_f64(s9), fma(cs, i64_to_f64(st), f));
            }
            if (exact) rf = i128_to_f32(tm + ts + fi, sc1, sc2);
            if (!finite) rf = __int_as_float(0x7FC00000);
        }
        sq = fmaf(rf, rf, sq);
        OT* o = rout + (size_t)b * rout_stride + (size_t)j * Px + i;
        if (sizeof(OT) == 2) *o = (OT)__float2bfloat16_rn(rf);
        else *o = TF32R ? (OT)sfde_round_tf32(rf) : (OT)rf;
    }
    double sqd = sq;
    for (int o = 16; o > 0; o >>= 1) sqd += __shfl_xor_sync(0xffffffffu, sqd, o);
    const int w = (ty * 32 + tx) >> 5;
    if ((tx & 31) == 0) red[w] = sqd;
    __syncthreads();
    if (tx == 0 && ty == 0) {
        double s = 0.0;
        for (int k = 0; k < 8; ++k) s += red[k];
        partial[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
    }
}

// rho_n = F_n for pairs of two zero slices (Z1 = Z2 = du = 0): with no fixed-point unit k_combine_int
// takes its FP64 form there, F_n + 0 S9 + 0 S, i.e. F_n rounded once to FP32 (-0 read as +0); this
// kernel gives the same values from the load alone, on the same tiles and with the same per-block sums
// of rho^2, reading no product.  A rank-1 load without a dense part is one FP64 product per element,
// rounded here in integer arithmetic (mul_f64_to_f32; the FP64 pipe runs at about 1/64 of the FP32
// rate); other loads, and products outside the normal range, take FP64 arithmetic.
template <typename OT, bool TF32R>
__global__ void __launch_bounds__(256) k_load_resid(int n0, int Px, int Py, int nx, int ny, int rank,
                                                    const double* __restrict__ time_w, const double* __restrict__ bxn,
                                                    const double* __restrict__ byn, const double* __restrict__ Fd,
                                                    OT* __restrict__ rout, long long rout_stride,
                                                    double* __restrict__ partial) {
    __shared__ double fy[SFDE_MAX_RANK][32];
    __shared__ double red[8];
    const int b = blockIdx.z, n = n0 + b;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const size_t P2 = (size_t)Px * Py;
    if (ty == 0)
        for (int q = 0; q < rank; ++q) {
            const int j = j0 + tx;
            fy[q][tx] = j < Py ? time_w[(size_t)(n - 1) * rank + q] * byn[(size_t)q * Py + j] : 0.0;
        }
    __syncthreads();
    const int i = i0 + tx;
    double bxi[SFDE_MAX_RANK];
#pragma unroll
    for (int q = 0; q < SFDE_MAX_RANK; ++q) bxi[q] = (q < rank && i < Px) ? bxn[(size_t)q * Px + i] : 0.0;
    float sq = 0.f;
    for (int jj = ty; jj < 32; jj += 8) {
        const int j = j0 + jj;
        float rf = 0.f;
        if (i < nx && j < ny && (rank > 0 || Fd)) {
            float v;
            if (rank == 1 && !Fd && sfde_round::mul_f64_to_f32(fy[0][jj], bxi[0], v)) {
                rf = (__float_as_uint(v) << 1) == 0 ? 0.f : v;   // -0 -> +0
            } else {
                double f = Fd ? Fd[(size_t)(n - 1) * P2 + (size_t)j * Px + i] : 0.0;
#pragma unroll
                for (int q = 0; q < SFDE_MAX_RANK; ++q)
                    if (q < rank) f = fma(fy[q][jj], bxi[q], f);
                if ((__double_as_longlong(f) << 1) == 0) f = 0.0;   // -0 -> +0 (integer test of the bits)
                rf = (float)f;
            }
        }
        sq = fmaf(rf, rf, sq);
        OT* o = rout + (size_t)b * rout_stride + (size_t)j * Px + i;
        if (sizeof(OT) == 2) *o = (OT)__float2bfloat16_rn(rf);
        else *o = TF32R ? (OT)sfde_round_tf32(rf) : (OT)rf;
    }
    double sqd = sq;
    for (int o = 16; o > 0; o >>= 1) sqd += __shfl_xor_sync(0xffffffffu, sqd, o);
    const int w = (ty * 32 + tx) >> 5;
    if ((tx & 31) == 0) red[w] = sqd;
    __syncthreads();
    if (tx == 0 && ty == 0) {
        double s = 0.0;
        for (int k = 0; k < 8; ++k) s += red[k];
        partial[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
    }
}

}  // namespace

// contraction lengths up to 256, or multiples of 256 up to 1024 (the digit product's K groups)
bool sfde_resid_int_supported(int Px, int Py) {
    // the digit products take tiles of 32 output columns and sum K in groups of 128, up to 1024
    // (at least 64: the smallest size the residual's tests and tile shapes cover)
    auto ok = [](int P) { return P >= 64 && (P <= 256 || (P <= 1024 && P % 256 == 0)); };
    return ok(Px) && ok(Py);
}

size_t sfde_resid_int_digit_bytes(int Px, int Py, int batch) { return (size_t)ND * Px * Py * batch * 2; }

sfde_status sfde_resid_int_matrices(sfde_ctx* c, OzMatrix* Ax, OzMatrix* Ay) {
    // K_x M_y (x) A_x = (1,4,1)_y (x) (K_x h_y / 6) A_x and K_y A_y (x) M_x = (K_y h_x / 6) A_y (x) (1,4,1)_x:
    // the (1,4,1) stencils are applied to the exact integer products
    SFDE_TRY(sfde_oz_split_matrix(c->x.A, c->x.P, c->x.P, Ax, c->stream, c->kx * c->y.h / 6.0, true));
    SFDE_TRY(sfde_oz_split_matrix(c->y.A, c->y.P, c->y.P, Ay, c->stream, c->ky * c->x.h / 6.0, true));
    return SFDE_OK;
}

namespace {
// k_combine_int (ZERO: k_load_resid) for one chunk of nb pairs from n0, output kind 0 (BF16),
// 1 (TF32-rounded FP32) or 2 (FP32)
template <bool ZERO>
void launch_combine(sfde_ctx* c, int out_kind, const long long* du, const int* En, int n0, int nb, int ex, int ey,
                    void* ro, long long rout_stride, double* partial) {
    const int Px = c->x.P, Py = c->y.P;
    dim3 grid(Px / 32, Py / 32, nb), block(32, 8);
    const double cmass = c->x.h * c->y.h / 36.0;
    const int zx = sfde_oz_int_shift(Px), zy = sfde_oz_int_shift(Py);
    const long long *T1 = (const long long*)c->T1, *T3 = (const long long*)c->T3;
    if constexpr (ZERO) {
        if (out_kind == 0)
            k_load_resid<__nv_bfloat16, false><<<grid, block, 0, c->stream>>>(
                n0, Px, Py, c->x.n, c->y.n, c->rank, c->time_w, c->bxn, c->byn, c->Fd, (__nv_bfloat16*)ro,
                rout_stride, partial);
        else if (out_kind == 1)
            k_load_resid<float, true><<<grid, block, 0, c->stream>>>(
                n0, Px, Py, c->x.n, c->y.n, c->rank, c->time_w, c->bxn, c->byn, c->Fd, (float*)ro, rout_stride,
                partial);
        else
            k_load_resid<float, false><<<grid, block, 0, c->stream>>>(
                n0, Px, Py, c->x.n, c->y.n, c->rank, c->time_w, c->bxn, c->byn, c->Fd, (float*)ro, rout_stride,
                partial);
        return;
    }
    if (out_kind == 0)
        k_combine_int<__nv_bfloat16, false><<<grid, block, 0, c->stream>>>(
            T1, T3, du, En, n0, Px, Py, c->x.n, c->y.n, cmass, ex, ey, zx, zy, c->dt0, c->rank, c->time_w, c->bxn,
            c->byn, c->Fd, (__nv_bfloat16*)ro, rout_stride, partial);
    else if (out_kind == 1)
        k_combine_int<float, true><<<grid, block, 0, c->stream>>>(
            T1, T3, du, En, n0, Px, Py, c->x.n, c->y.n, cmass, ex, ey, zx, zy, c->dt0, c->rank, c->time_w, c->bxn,
            c->byn, c->Fd, (float*)ro, rout_stride, partial);
    else
        k_combine_int<float, false><<<grid, block, 0, c->stream>>>(
            T1, T3, du, En, n0, Px, Py, c->x.n, c->y.n, cmass, ex, ey, zx, zy, c->dt0, c->rank, c->time_w, c->bxn,
            c->byn, c->Fd, (float*)ro, rout_stride, partial);
}
}  // namespace

sfde_status sfde_residual_int(sfde_ctx* c, const double* U, int n_first, int count, void* rout,
                              long long rout_stride, int out_kind, double* partial, int* n_partials,
                              const OzMatrix& Ax, const OzMatrix& Ay, void* dV, void* dVt, int* En, int* err,
                              int nd, int n_zero) {
    const int Px = c->x.P, Py = c->y.P;
    const size_t P2 = c->P2();
    const size_t esz = out_kind == 0 ? 2 : 4;
    if (!sfde_resid_int_supported(Px, Py) || n_first < 1 || count < 1 || nd < 4 || nd > ND) return SFDE_EINVAL;
    // pairs n >= n_zero (two zero slices) take the load alone; the products run for the others
    const int gcount = (int)std::max<long long>(0, std::min<long long>(count, (long long)n_zero - n_first));
    // accounting (class 5): bytes each kernel must move once, unpadded
    const double nxy = (double)c->x.n * c->y.n;
    const int blocks1 = (Px / 32) * (Py / 32);
    int slot;
    if (gcount > 0) {
        slot = sfde_prof_begin(c);
        k_slice_maxexp<<<gcount + 1, 256, 0, c->stream>>>(U + (size_t)(n_first - 1) * P2, P2, En + (n_first - 1));
        sfde_prof_end(c, slot, 5, 0.0, 8.0 * nxy * (gcount + 1));
        sfde_count_launch(c);
    }
    int total = 0;
    const int chunk = c->resid_chunk > 0 ? std::min(c->resid_chunk, (int)c->ws_slices) : (int)c->ws_slices;
    for (int b0 = 0; b0 < gcount; b0 += chunk) {
        const int nb = std::min(gcount - b0, chunk);
        const int n0 = n_first + b0;
        const long long plane = (long long)nb * Px * Py;
        dim3 grid(Px / 32, Py / 32, nb);
        long long* du = (long long*)c->T2;   // fix(U_{n-1}) - fix(U_n), int64 per element
        slot = sfde_prof_begin(c);
        k_split_pair<<<grid, 256, 0, c->stream>>>(U, En, n0, Px, Py, (uint16_t*)dV, (uint16_t*)dVt, du, plane, nd);
        // U pair in, 2 x nd digit planes and du out
        sfde_prof_end(c, slot, 5, 0.0, (16.0 + 4.0 * nd + 8.0) * nxy * nb);
        sfde_count_launch(c);
        SFDE_TRY(sfde_oz_gemm_int(c, dV, plane, Py, Px, nb, Ax, (long long*)c->T1, (long long)P2, err, c->y.n,
                                  c->x.n, c->x.n, nd));
        SFDE_TRY(sfde_oz_gemm_int(c, dVt, plane, Px, Py, nb, Ay, (long long*)c->T3, (long long)P2, err, c->x.n,
                                  c->y.n, c->y.n, nd));
        const int blocks = blocks1 * nb;
        if ((size_t)(total + blocks) > c->partial_cap) return SFDE_EINVAL;
        slot = sfde_prof_begin(c);
        launch_combine<false>(c, out_kind, du, En, n0, nb, Ax.e_uniform, Ay.e_uniform,
                              (char*)rout + (size_t)b0 * rout_stride * esz, rout_stride, partial + total);
        sfde_prof_end(c, slot, 5, 0.0, (16.0 + 8.0 + (double)esz) * nxy * nb);   // Z1, Z2, du in, rho out
        sfde_count_launch(c);
        total += blocks;
    }
    for (int b0 = gcount; b0 < count; b0 += 65535) {   // grid z <= 65535
        const int nb = std::min(count - b0, 65535);
        const int blocks = blocks1 * nb;
        if ((size_t)(total + blocks) > c->partial_cap) return SFDE_EINVAL;
        slot = sfde_prof_begin(c);
        launch_combine<true>(c, out_kind, (const long long*)c->T2, En, n_first + b0, nb, Ax.e_uniform, Ay.e_uniform,
                             (char*)rout + (size_t)b0 * rout_stride * esz, rout_stride, partial + total);
        sfde_prof_end(c, slot, 5, 0.0, (double)esz * nxy * nb);   // rho out
        sfde_count_launch(c);
        total += blocks;
    }
    SFDE_CUDA(cudaGetLastError());
    if (n_partials) *n_partials = total;
    return SFDE_OK;
}

extern "C" sfde_status sfde_debug_residual(sfde_ctx* c, const double* U, int use_tensor_cores, float* rho,
                                          double* norm2) {
    if (!c || !U || !rho || !norm2) return SFDE_EINVAL;
    const int Px = c->x.P, Py = c->y.P;
    const int nd = use_tensor_cores == 1 ? ND : use_tensor_cores;
    if (use_tensor_cores && (nd < 4 || nd > ND)) return SFDE_EINVAL;
    if (use_tensor_cores && !sfde_resid_int_supported(Px, Py)) return SFDE_EUNSUPPORTED;
    const size_t P2 = c->P2(), n2 = (size_t)c->x.n * c->y.n;
    const int okind = c->precision == SFDE_PREC_MIXED_FP32 ? 2 : 1;   // storage as the solver keeps it
    double* u = nullptr;
    SFDE_TRY(sfde_level0(c, &u));
    SFDE_TRY(sfde_ensure_workspace(c, std::min<size_t>(c->nt, 128)));
    const size_t need = (size_t)c->nt * (Px / 16) * (Py / 16) + 64;
    if (c->partial_cap < need) {
        cudaFree(c->partial);
        c->partial = nullptr;
        SFDE_CUDA(cudaMalloc(&c->partial, sizeof(double) * need));
        c->partial_cap = need;
    }
    double* tmp = nullptr;
    float *rp = nullptr, *ru = nullptr;
    OzMatrix Ax, Ay;
    void *dV = nullptr, *dVt = nullptr;
    int *En = nullptr, *err = nullptr;
    sfde_status st = SFDE_OK;
    int np = 0;
    cudaError_t e;
#define DC(x) if ((e = (x)) != cudaSuccess) { sfde_set_last_cuda_error(e, #x, __FILE__, __LINE__); st = SFDE_ECUDA; goto done; }
    DC(cudaMalloc(&tmp, sizeof(double) * n2 * (c->nt + 1)));
    DC(cudaMalloc(&rp, sizeof(float) * P2 * c->nt));
    DC(cudaMalloc(&ru, sizeof(float) * n2 * c->nt));
    DC(cudaMalloc(&err, sizeof(int)));
    DC(cudaMemset(err, 0, sizeof(int)));
    if ((st = sfde_copy_in(tmp, U, sizeof(double) * n2 * (c->nt + 1), c->stream)) != SFDE_OK) goto done;
    sfde_launch_pad(tmp, u, c->y.n, c->x.n, Py, Px, c->nt + 1, c->stream);
    if (use_tensor_cores) {
        if ((st = sfde_resid_int_matrices(c, &Ax, &Ay)) != SFDE_OK) goto done;
        DC(cudaMalloc(&dV, sfde_resid_int_digit_bytes(Px, Py, (int)c->ws_slices)));
        DC(cudaMalloc(&dVt, sfde_resid_int_digit_bytes(Px, Py, (int)c->ws_slices)));
        DC(cudaMalloc(&En, sizeof(int) * (c->nt + 1)));
        st = sfde_residual_int(c, u, 1, c->nt, rp, (long long)P2, okind, c->partial, &np, Ax, Ay, dV, dVt, En, err,
                               nd, INT_MAX);
    } else {
        st = sfde_residual_fp64(c, u, 1, c->nt, rp, (long long)P2, okind, c->partial, &np);
    }
    if (st != SFDE_OK) goto done;
    if ((st = sfde_reduce_partials(c, np, norm2)) != SFDE_OK) goto done;
    sfde_launch_unpad_f32(rp, ru, c->y.n, c->x.n, Py, Px, c->nt, c->stream);  // one float per interior node
    if ((st = sfde_copy_out(rho, ru, sizeof(float) * n2 * c->nt, c->stream)) != SFDE_OK) goto done;
    DC(cudaStreamSynchronize(c->stream));
    {
        int herr = 0;
        DC(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
        if (herr) st = SFDE_ETIMEOUT;
    }
done:
#undef DC
    sfde_oz_free_matrix(&Ax);
    sfde_oz_free_matrix(&Ay);
    cudaFree(tmp); cudaFree(rp); cudaFree(ru); cudaFree(dV); cudaFree(dVt); cudaFree(En); cudaFree(err);
    return st;
}
