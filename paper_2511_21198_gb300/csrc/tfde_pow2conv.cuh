// FP64 <-> FP32 conversions with a power-of-two scale, by integer operations
// only.  GB300 issues FP64 at about 2 lanes per clock per SM, so one FP64
// multiply plus one conversion per element bounds an otherwise memory-bound
// vector kernel; with a power-of-two scale both reduce to exponent arithmetic
// on the bit patterns, with results identical to the hardware's
// round-to-nearest-even conversions of the scaled value.
#pragma once
#include <cstdint>

namespace tfde {

#ifdef __CUDACC__
#define TFDE_HD __host__ __device__ __forceinline__
#else
#define TFDE_HD inline
#endif

TFDE_HD float bits_to_f32(uint32_t b) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float f;
    __builtin_memcpy(&f, &b, 4);
    return f;
#endif
}
TFDE_HD uint32_t f32_to_bits(float f) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t b;
    __builtin_memcpy(&b, &f, 4);
    return b;
#endif
}
TFDE_HD double bits_to_f64(unsigned long long b) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double d;
    __builtin_memcpy(&d, &b, 8);
    return d;
#endif
}
TFDE_HD int clz32(uint32_t v) {
#ifdef __CUDA_ARCH__
    return __clz((int)v);
#else
    return v ? __builtin_clz(v) : 32;
#endif
}

// RN(x 2^k) as FP32, x given by its FP64 bit pattern u, |k| < 512: the FP64
// significand rounded to nearest even at FP32 precision (or on the FP32
// subnormal grid); overflow gives infinity, FP64 subnormals give zero.
TFDE_HD float f64_pow2_to_f32(unsigned long long u, int k) {
    const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
    const uint32_t sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu);
    if (e == 0x7FF) return bits_to_f32(sign | 0x7F800000u | (((hi & 0xFFFFFu) | lo) ? 0x400000u : 0u));
    if (e == 0) return bits_to_f32(sign);
    const int E = e - 896 + k;   // FP32 biased exponent (1023 - 127 = 896)
    if (E >= 255) return bits_to_f32(sign | 0x7F800000u);
    if (E > 0) {   // normal: keep 23 of the 52 fraction bits
        const uint32_t frac = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
        const uint32_t rem = lo & 0x1FFFFFFFu;
        const uint32_t up = (rem > 0x10000000u || (rem == 0x10000000u && (frac & 1u))) ? 1u : 0u;
        return bits_to_f32(sign | (((uint32_t)E << 23) + frac + up));   // a carry moves into the exponent
    }
    // subnormal result: the 53-bit significand in units of 2^-149
    const int sh = 30 - E;
    if (sh > 54) return bits_to_f32(sign);
    const unsigned long long M = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const unsigned long long q = M >> sh, rem = M & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    return bits_to_f32(sign | ((uint32_t)q + ((rem > half || (rem == half && (q & 1ull))) ? 1u : 0u)));
}

// (double) f 2^j, exact, for an FP32 f and |j| < 512 (every such value is a
// normal FP64 number); infinities and NaNs keep their class.
TFDE_HD double f32_pow2_to_f64(float f, int j) {
    const uint32_t b = f32_to_bits(f);
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    const uint32_t ex = (b >> 23) & 0xFFu;
    uint32_t frac = b & 0x7FFFFFu;
    if (ex == 0xFFu) return bits_to_f64(sign | 0x7FF0000000000000ull | ((unsigned long long)frac << 29));
    int e = (int)ex;
    if (ex == 0) {
        if (frac == 0) return bits_to_f64(sign);
        const int s = clz32(frac) - 8;   // normalise an FP32 subnormal
        frac = (frac << s) & 0x7FFFFFu;
        e = 1 - s;
    }
    const unsigned long long E = (unsigned long long)(e + 896 + j);
    return bits_to_f64(sign | (E << 52) | ((unsigned long long)frac << 29));
}

// x (FP64 bits u) rounded toward zero to FP32 precision, for sums that need
// only a few digits: values below the FP32 normal range become signed zero,
// values above it (and infinities, NaNs) signed infinity.
TFDE_HD float f64_to_f32_rz(unsigned long long u) {
    const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
    const uint32_t sign = hi & 0x80000000u;
    const int E = (int)((hi >> 20) & 0x7FFu) - 896;
    if (E <= 0) return bits_to_f32(sign);
    if (E >= 255) return bits_to_f32(sign | 0x7F800000u);
    return bits_to_f32(sign | ((uint32_t)E << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}

// k with sc = 2^k exactly and |k| < 512, else false
inline bool pow2_exponent(double sc, int* k) {
    int e = 0;
    const double m = __builtin_frexp(sc, &e);
    if (m != 0.5 || e - 1 <= -512 || e - 1 >= 512) return false;
    *k = e - 1;
    return true;
}

}  // namespace tfde
