// Per-point arithmetic of the chained CN step's right-hand side and
// extrapolated initial guess (Eq. (CN), Eq. (linear_sys)), shared by the
// single-problem kernels (tfde_kernels64.cu) and the batched ones
// (tfde_batch.cu), so that both form the same values.
#pragma once

#include "tfde_pow2conv.cuh"

namespace tfde {

// 2 v by the exponent field (exact; zero, subnormal, huge and non-finite
// values take the FP64 add)
__device__ __forceinline__ double chain_twice(double v) {
    const long long bits = __double_as_longlong(v);
    const unsigned e = (unsigned)(bits >> 52) & 0x7FFu;
    return (e != 0u && e < 0x7FEu) ? __longlong_as_double(bits + (1LL << 52)) : v + v;
}

__device__ __forceinline__ float chain_f32(double v) {
    return f64_to_f32_rz((unsigned long long)__double_as_longlong(v));
}

// The five terms of the minimal-residual correction at one point (FP32 from
// the integer-truncated FP64 values): with a_k = A u^{m-1-k} (a_0 = b - r),
// e1 = a0 - a1, e2 = a0 - 2 a1 + a2 and r_e = b^m - (3 a0 - 3 a1 + a2),
// b^m = 2 A_N u^{m-1} + dt F - a0: e1 e1, e1 e2, e2 e2, e1 r_e, e2 r_e.
__device__ __forceinline__ void chain_mr_terms(double an, const double* F, long long i, float dtf, double b, double r,
                                               double au1, double au2, float s[5]) {
    const float a0 = chain_f32(b) - chain_f32(r), a1 = chain_f32(au1), a2 = chain_f32(au2);
    const float bn = fmaf(2.f, chain_f32(an), F ? dtf * chain_f32(__ldg(F + i)) : 0.f) - a0;
    const float e1 = a0 - a1, e2 = e1 - (a1 - a2);
    const float re = bn - fmaf(3.f, e1, a2);
    s[0] = fmaf(e1, e1, s[0]);
    s[1] = fmaf(e1, e2, s[1]);
    s[2] = fmaf(e2, e2, s[2]);
    s[3] = fmaf(e1, re, s[3]);
    s[4] = fmaf(e2, re, s[4]);
}

// Coefficients g of the corrected guess x0 = g0 u^{m-1} + g1 u^{m-2} +
// g2 u^{m-3} from the five sums m: the order-2 extrapolation 3, -3, 1 plus
// c1 d1 + c2 d2 (d1 = u^{m-1} - u^{m-2}, d2 = u^{m-1} - 2 u^{m-2} + u^{m-3}),
// c solving the 2 x 2 normal equations [m0 m1; m1 m2] c = [m3; m4].  An
// ill-conditioned or non-finite system, or |c| > 1e3, leaves c = 0.
__device__ __forceinline__ void chain_mr_coefficients(const double* m, double* g) {
    double c1 = 0.0, c2 = 0.0;
    bool ok = true;
    for (int q = 0; q < 5; ++q) ok = ok && isfinite(m[q]);
    const double det = m[0] * m[2] - m[1] * m[1];
    if (ok && m[0] > 0.0 && m[2] > 0.0 && det > 1e-12 * m[0] * m[2]) {
        c1 = (m[2] * m[3] - m[1] * m[4]) / det;
        c2 = (m[0] * m[4] - m[1] * m[3]) / det;
        if (!isfinite(c1) || !isfinite(c2) || fabs(c1) > 1e3 || fabs(c2) > 1e3) c1 = c2 = 0.0;
    }
    g[0] = 3.0 + c1 + c2;
    g[1] = -3.0 - c1 - 2.0 * c2;
    g[2] = 1.0 + c2;
}

// One point of the chained step with an extrapolated guess: b^m = 2 A_N u +
// dt F - A u (A u = b - r), x0 and A x0 from the history by the order's
// combination (order 3: g0, g1, g2), r = b^m - A x0; the history's oldest
// slot receives (u, A u).  Returns b^m and r in *bn_out, *rn_out.
__device__ __forceinline__ void chain_extrap_point(long long i, const double* __restrict__ AN,
                                                   const double* __restrict__ F, double dt, double* __restrict__ b,
                                                   double* __restrict__ r, double* __restrict__ u,
                                                   const double* __restrict__ U1, const double* __restrict__ AU1,
                                                   double* __restrict__ U2, double* __restrict__ AU2, int order,
                                                   double g0, double g1, double g2, double* bn_out, double* rn_out) {
    const double ui = u[i];
    const double au = b[i] - r[i];
    const double an2 = chain_twice(AN[i]);
    const double bn = (F ? fma(dt, F[i], an2) : an2) - au;
    double x = ui, ax = au;
    if (order == 1) {
        x = fma(2.0, ui, -U1[i]);
        ax = fma(2.0, au, -AU1[i]);
    } else if (order == 2) {
        x = fma(3.0, ui - U1[i], U2[i]);
        ax = fma(3.0, au - AU1[i], AU2[i]);
    } else if (order >= 3) {
        x = fma(g0, ui, fma(g1, U1[i], g2 * U2[i]));
        ax = fma(g0, au, fma(g1, AU1[i], g2 * AU2[i]));
    }
    const double rn = bn - ax;
    b[i] = bn;
    r[i] = rn;
    u[i] = x;
    U2[i] = ui;
    AU2[i] = au;
    *bn_out = bn;
    *rn_out = rn;
}

}  // namespace tfde
