// (float)(a b) for FP64 a, b as FP64 arithmetic gives it -- the exact product rounded to 53 bits,
// then to 24 bits, both to nearest even -- from integer operations, for kernels where the FP64 pipe
// (about 1/64 of the FP32 rate on this GPU) would bound them.  Host and device: the host build is
// what the CPU test checks against FP64 arithmetic.
#pragma once
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define SFDE_HD __host__ __device__ __forceinline__
#else
#define SFDE_HD inline
#endif

namespace sfde_round {

SFDE_HD uint64_t umulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

SFDE_HD uint64_t bits_of(double x) {
    uint64_t u;
    memcpy(&u, &x, 8);
    return u;
}

SFDE_HD float float_of(uint32_t u) {
    float f;
    memcpy(&f, &u, 4);
    return f;
}

// false where an operand is not finite or is subnormal, or a rounded result is not a normal number
// (the caller then uses FP64 arithmetic); a zero factor gives the signed zero of the product
SFDE_HD bool mul_f64_to_f32(double a, double b, float& out) {
    const uint64_t ba = bits_of(a), bb = bits_of(b);
    const uint32_t sgn = (uint32_t)((ba ^ bb) >> 63) << 31;
    const int ea = (int)((ba >> 52) & 0x7FF), eb = (int)((bb >> 52) & 0x7FF);
    if (ea == 0x7FF || eb == 0x7FF) return false;
    if ((ba << 1) == 0 || (bb << 1) == 0) { out = float_of(sgn); return true; }
    if (ea == 0 || eb == 0) return false;
    const uint64_t ma = (ba & 0xFFFFFFFFFFFFFull) | (1ull << 52), mb = (bb & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const uint64_t hi = umulhi64(ma, mb), lo = ma * mb;           // p = hi 2^64 + lo in [2^104, 2^106)
    const int top = (hi >> 41) ? 105 : 104;                       // position of the leading one
    const int sh = top - 52;                                      // bits dropped: 52 or 53, all in lo
    uint64_t m = (hi << (64 - sh)) | (lo >> sh);                  // 53 bits
    const uint64_t rest = lo & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rest > half || (rest == half && (m & 1))) ++m;
    int e = top + ea + eb - 2150;                                 // the value is m 2^(e - 52)
    if (m == (1ull << 53)) { m >>= 1; ++e; }
    if (e + 1023 <= 0 || e + 1023 >= 2047) return false;          // not a normal FP64 number
    const uint64_t r = m & ((1ull << 29) - 1), h2 = 1ull << 28;   // to 24 bits
    uint32_t m24 = (uint32_t)(m >> 29);
    if (r > h2 || (r == h2 && (m24 & 1))) ++m24;
    if (m24 == (1u << 24)) { m24 >>= 1; ++e; }
    if (e + 127 <= 0 || e + 127 >= 255) return false;             // not a normal FP32 number
    out = float_of(sgn | ((uint32_t)(e + 127) << 23) | (m24 & 0x7FFFFF));
    return true;
}

}  // namespace sfde_round
