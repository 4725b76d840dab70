// Host check of the power-of-two scaled FP64 <-> FP32 conversions used by the
// inner solver's vector kernels, against the host's IEEE round-to-nearest-even
// conversions of the exactly scaled values (ldexp is exact in range).
// Prints the mismatch counts; exit status 1 on any mismatch.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "tfde_pow2conv.cuh"

using namespace tfde;

int main() {
    std::mt19937_64 g(20251203);
    long n64 = 0, bad64 = 0, n32 = 0, bad32 = 0;
    for (int it = 0; it < 4000000; ++it) {
        unsigned long long u = g();
        const int mode = it % 4;
        if (mode == 0) {   // anywhere near the FP32 range
            const int ex = 1023 + (int)(g() % 400) - 200;
            u = (u & 0x800FFFFFFFFFFFFFull) | ((unsigned long long)ex << 52);
        } else if (mode == 1) {   // exact ties at FP32 precision
            const int ex = 1023 + (int)(g() % 300) - 150;
            u = (u & 0x800FFFFFE0000000ull) | 0x10000000ull | ((unsigned long long)ex << 52);
        } else if (mode == 2) {   // results on the FP32 subnormal grid, ties included
            const int ex = 1023 - 126 - (int)(g() % 30);
            u = (u & 0x800FFFFFFFFFFFFFull) | ((unsigned long long)ex << 52);
            if (g() & 1) u = (u & 0xFFFFFFFF00000000ull) | ((g() & 1) ? 0x10000000ull : 0ull);
        }
        double x;
        std::memcpy(&x, &u, 8);
        if (std::isnan(x)) continue;
        const int k = mode == 2 ? (int)(g() % 8) - 4 : (int)(g() % 200) - 100;
        if (x != 0.0 && (std::ilogb(x) + k < -1022 || std::ilogb(x) + k > 1023)) continue;
        const float got = f64_pow2_to_f32(u, k), want = (float)std::ldexp(x, k);
        unsigned a, b;
        std::memcpy(&a, &got, 4);
        std::memcpy(&b, &want, 4);
        ++n64;
        if (a != b) ++bad64;
    }
    for (int it = 0; it < 4000000; ++it) {
        unsigned b = (unsigned)g();
        if (it % 3 == 0) b &= 0x807FFFFFu;   // FP32 subnormals and zeros
        float f;
        std::memcpy(&f, &b, 4);
        if (std::isnan(f)) continue;
        const int j = (int)(g() % 1000) - 500;
        const double got = f32_pow2_to_f64(f, j), want = std::ldexp((double)f, j);
        unsigned long long a, c;
        std::memcpy(&a, &got, 8);
        std::memcpy(&c, &want, 8);
        ++n32;
        if (a != c) ++bad32;
    }
    int k = 0;
    const bool p_ok = pow2_exponent(0.25, &k) && k == -2 && !pow2_exponent(3.0, &k) &&
                      !pow2_exponent(std::ldexp(1.0, 600), &k);
    std::printf("f64_pow2_to_f32 %ld %ld f32_pow2_to_f64 %ld %ld pow2_exponent %d\n", n64, bad64, n32, bad32,
                p_ok ? 1 : 0);
    return (bad64 || bad32 || !p_ok) ? 1 : 0;
}
