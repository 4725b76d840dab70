// FP32 / split-BF16 vector kernels of the mixed-precision inner solves.
// A split-BF16 plane pair (hi, lo) stores v ~= hi + lo with
// hi = bf16(v), lo = bf16(v - hi): the B operand format of the tensor-core
// contraction.  Inner products accumulate per thread in compensated FP32 and
// across threads in FP64 (deterministic two-stage reduction).
#include <cuda_bf16.h>

#include "tfde_internal.h"
#include "tfde_stats.h"
#include "tfde_mixed.h"
#include "tfde_pow2conv.cuh"

namespace tfde {
namespace {

constexpr int kT = 256;

__device__ __forceinline__ void split(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// Kahan-compensated FP32 accumulation.
struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

__device__ __forceinline__ double block_sum64(double v) {
    __shared__ double sh[kT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kT / 32; ++w) t += sh[w];
    return t;
}

__device__ __forceinline__ void chunk(long long N, long long& lo, long long& hi) {
    const long long per = (N + gridDim.x - 1) / gridDim.x;
    lo = (long long)blockIdx.x * per;
    hi = lo + per < N ? lo + per : N;
}

__global__ __launch_bounds__(kT) void dot32_kernel(long long N, const float* __restrict__ a,
                                                   const float* __restrict__ b, double* __restrict__ part) {
    long long lo, hi;
    chunk(N, lo, hi);
    KSum k;
    for (long long i = lo + threadIdx.x; i < hi; i += kT) k.add(a[i] * b[i]);
    const double t = block_sum64((double)k.s - (double)k.c);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// alpha = num / den (device scalars, formed once per block); x += alpha p ;
// r -= alpha q ; (rh, rl) = split(r) ; *rr += r.r (compensated per thread,
// FP64 across the block, one atomic add per block)
__global__ __launch_bounds__(kT) void cg_update32_kernel(long long N, const double* __restrict__ num,
                                                         const double* __restrict__ den, const float* __restrict__ p,
                                                         const float* __restrict__ q, float* __restrict__ x,
                                                         float* __restrict__ r, __nv_bfloat16* __restrict__ rh,
                                                         __nv_bfloat16* __restrict__ rl, double* __restrict__ rr) {
    __shared__ float s_alpha;
    if (threadIdx.x == 0) s_alpha = (float)(num[0] / den[0]);
    __syncthreads();
    const float alpha = s_alpha;
    long long lo, hi;
    chunk(N, lo, hi);
    KSum k;
    for (long long i = lo + threadIdx.x; i < hi; i += kT) {
        x[i] = fmaf(alpha, p[i], x[i]);
        const float ri = fmaf(-alpha, q[i], r[i]);
        r[i] = ri;
        split(ri, rh[i], rl[i]);
        k.add(ri * ri);
    }
    const double t = block_sum64((double)k.s - (double)k.c);
    if (threadIdx.x == 0) atomicAdd(rr, t);
}

// alpha = num / den; r -= alpha q ; (rh, rl) = split(r) ; *rr += r.r ; alpha
// (double) to *alpha_out for the later combination of the solution
__global__ __launch_bounds__(kT) void cg_update_r32_kernel(long long N, const double* __restrict__ num,
                                                           const double* __restrict__ den,
                                                           const float* __restrict__ q, float* __restrict__ r,
                                                           __nv_bfloat16* __restrict__ rh,
                                                           __nv_bfloat16* __restrict__ rl, double* __restrict__ rr,
                                                           double* __restrict__ alpha_out, const int* skip) {
    if (skip && *skip) return;
    __shared__ float s_alpha;
    if (threadIdx.x == 0) {
        const double a = num[0] / den[0];
        s_alpha = (float)a;
        if (blockIdx.x == 0) *alpha_out = (double)(float)a;   // the value the update used
    }
    __syncthreads();
    const float alpha = s_alpha;
    long long lo, hi;
    chunk(N, lo, hi);
    KSum k;
    for (long long i = lo + threadIdx.x; i < hi; i += kT) {
        const float ri = fmaf(-alpha, q[i], r[i]);
        r[i] = ri;
        if (rl) split(ri, rh[i], rl[i]);
        else rh[i] = __float2bfloat16_rn(ri);
        k.add(ri * ri);
    }
    const double t = block_sum64((double)k.s - (double)k.c);
    if (threadIdx.x == 0) atomicAdd(rr, t);
}

// The same update four elements at a time (N4 = N / 4 groups; 16-byte
// loads and stores, packed BF16 conversions with the same rounding).
__device__ __forceinline__ uint2 bf16x4_hi(float4 v) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
    return make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
}
__device__ __forceinline__ uint2 bf16x4_lo(float4 v, uint2 h) {
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&h.x);
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&h.y);
    const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    const __nv_bfloat162 la = __floats2bfloat162_rn(v.x - fa.x, v.y - fa.y), lb = __floats2bfloat162_rn(v.z - fb.x, v.w - fb.y);
    return make_uint2(*reinterpret_cast<const uint32_t*>(&la), *reinterpret_cast<const uint32_t*>(&lb));
}
__global__ __launch_bounds__(kT) void cg_update_r32_v4_kernel(long long N4, const double* __restrict__ num,
                                                              const double* __restrict__ den,
                                                              const float4* __restrict__ q, float4* __restrict__ r,
                                                              uint2* __restrict__ rh, uint2* __restrict__ rl,
                                                              double* __restrict__ rr, double* __restrict__ alpha_out,
                                                              const int* skip) {
    if (skip && *skip) return;
    __shared__ float s_alpha;
    if (threadIdx.x == 0) {
        const double a = num[0] / den[0];
        s_alpha = (float)a;
        if (blockIdx.x == 0) *alpha_out = (double)(float)a;
    }
    __syncthreads();
    const float alpha = s_alpha;
    long long lo, hi;
    chunk(N4, lo, hi);
    KSum k;
#pragma unroll 2
    for (long long i = lo + threadIdx.x; i < hi; i += kT) {
        const float4 qv = q[i];
        float4 v = r[i];
        v.x = fmaf(-alpha, qv.x, v.x);
        v.y = fmaf(-alpha, qv.y, v.y);
        v.z = fmaf(-alpha, qv.z, v.z);
        v.w = fmaf(-alpha, qv.w, v.w);
        r[i] = v;
        const uint2 h = bf16x4_hi(v);
        rh[i] = h;
        if (rl) rl[i] = bf16x4_lo(v, h);
        k.add(v.x * v.x);
        k.add(v.y * v.y);
        k.add(v.z * v.z);
        k.add(v.w * v.w);
    }
    const double t = block_sum64((double)k.s - (double)k.c);
    if (threadIdx.x == 0) atomicAdd(rr, t);
}

// ---------------------------------------------- inner PCG in the DST eigenbasis
// Lambda(i, j, k) = ra[k] U[c] + rb[k] V[c], c = i + n1 j (Eq. (diag_tau_pre)):
// the preconditioner is this diagonal once the vectors live in the
// sine-transform eigenbasis.  Launched on a 2-D grid: x over the float4
// groups of one z plane (n1 n2 is a multiple of 4), y over the planes.
struct LamView {
    const float* ra;
    const float* rb;
    const float4* U;
    const float4* V;
    long long nc4;   // n1 n2 / 4
    int n3;
};

__device__ __forceinline__ float4 lam4(const LamView& L, float ra, float rb, long long c4) {
    const float4 u = L.U[c4], v = L.V[c4];
    return make_float4(fmaf(ra, u.x, rb * v.x), fmaf(ra, u.y, rb * v.y), fmaf(ra, u.z, rb * v.z),
                       fmaf(ra, u.w, rb * v.w));
}

// alpha = num / den; r -= alpha q; *rz += <r, r / Lambda>; *rr += <r, r>
__global__ __launch_bounds__(kT) void spec_update_kernel(LamView L, const double* __restrict__ num,
                                                         const double* __restrict__ den, const float4* __restrict__ q,
                                                         float4* __restrict__ r, double* __restrict__ rz,
                                                         double* __restrict__ rr, double* __restrict__ alpha_out,
                                                         const int* skip) {
    if (skip && *skip) return;
    __shared__ float s_alpha;
    if (threadIdx.x == 0) {
        const double a = num[0] / den[0];
        s_alpha = (float)a;
        if (blockIdx.x == 0 && blockIdx.y == 0) *alpha_out = (double)(float)a;
    }
    __syncthreads();
    const float alpha = s_alpha;
    KSum kz, kr;
    for (int k = blockIdx.y; k < L.n3; k += gridDim.y) {
        const float ra = L.ra[k], rb = L.rb[k];
        for (long long c4 = (long long)blockIdx.x * kT + threadIdx.x; c4 < L.nc4; c4 += (long long)gridDim.x * kT) {
            const long long i = (long long)k * L.nc4 + c4;
            const float4 qv = q[i];
            float4 v = r[i];
            v.x = fmaf(-alpha, qv.x, v.x);
            v.y = fmaf(-alpha, qv.y, v.y);
            v.z = fmaf(-alpha, qv.z, v.z);
            v.w = fmaf(-alpha, qv.w, v.w);
            r[i] = v;
            const float4 l = lam4(L, ra, rb, c4);
            kz.add(v.x * (v.x / l.x));
            kz.add(v.y * (v.y / l.y));
            kz.add(v.z * (v.z / l.z));
            kz.add(v.w * (v.w / l.w));
            kr.add(v.x * v.x);
            kr.add(v.y * v.y);
            kr.add(v.z * v.z);
            kr.add(v.w * v.w);
        }
    }
    const double tz = block_sum64((double)kz.s - (double)kz.c);
    const double tr = block_sum64((double)kr.s - (double)kr.c);
    if (threadIdx.x == 0) {
        atomicAdd(rz, tz);
        atomicAdd(rr, tr);
    }
}

// beta = num / den (0 when den is null); p = r / Lambda + beta p_old, written
// in FP32 and as split planes (ph, pl); with rz: *rz += <r, r / Lambda>
__global__ __launch_bounds__(kT) void spec_direction_kernel(LamView L, const double* __restrict__ num,
                                                            const double* __restrict__ den,
                                                            const float4* __restrict__ r,
                                                            const float4* __restrict__ pold, float4* __restrict__ p,
                                                            uint2* __restrict__ ph, uint2* __restrict__ pl,
                                                            double* __restrict__ rz, const int* skip) {
    if (skip && *skip) return;
    __shared__ float s_beta;
    if (threadIdx.x == 0) s_beta = den ? (float)(num[0] / den[0]) : 0.f;
    __syncthreads();
    const float beta = s_beta;
    KSum kz;
    for (int k = blockIdx.y; k < L.n3; k += gridDim.y) {
        const float ra = L.ra[k], rb = L.rb[k];
        for (long long c4 = (long long)blockIdx.x * kT + threadIdx.x; c4 < L.nc4; c4 += (long long)gridDim.x * kT) {
            const long long i = (long long)k * L.nc4 + c4;
            const float4 rv = r[i];
            const float4 l = lam4(L, ra, rb, c4);
            float4 z = make_float4(rv.x / l.x, rv.y / l.y, rv.z / l.z, rv.w / l.w);
            if (rz) {
                kz.add(rv.x * z.x);
                kz.add(rv.y * z.y);
                kz.add(rv.z * z.z);
                kz.add(rv.w * z.w);
            }
            if (pold) {
                const float4 o = pold[i];
                z.x = fmaf(beta, o.x, z.x);
                z.y = fmaf(beta, o.y, z.y);
                z.z = fmaf(beta, o.z, z.z);
                z.w = fmaf(beta, o.w, z.w);
            }
            p[i] = z;
            const uint2 h = bf16x4_hi(z);
            ph[i] = h;
            pl[i] = bf16x4_lo(z, h);
        }
    }
    if (rz) {
        const double t = block_sum64((double)kz.s - (double)kz.c);
        if (threadIdx.x == 0) atomicAdd(rz, t);
    }
}

// d = (x32 when fold) + sum_j alpha_j p_j (FP32, in the order of the
// directions, as the per-iteration update x += alpha p would form it); then
// c64 = sc d and x64 += c64 (c64 set), x64 += sc d (x64 only), or acc32 = d
struct CombineArgs {
    int cnt;
    int fold;
    const float* p[kPRing];
    const double* alpha[kPRing];
};
__global__ void pcg_combine_kernel(long long N, CombineArgs a, const float* __restrict__ x32, double sc,
                                   double* __restrict__ c64, double* __restrict__ x64, float* __restrict__ acc32) {
    __shared__ float s_al[kPRing];
    if (threadIdx.x < a.cnt) s_al[threadIdx.x] = (float)*a.alpha[threadIdx.x];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        float d = a.fold ? x32[i] : 0.f;
#pragma unroll
        for (int j = 0; j < kPRing; ++j)
            if (j < a.cnt) d = fmaf(s_al[j], a.p[j][i], d);
        if (acc32) {
            acc32[i] = d;
        } else if (c64) {
            const double v = sc * (double)d;
            c64[i] = v;
            x64[i] += v;
        } else {
            x64[i] += sc * (double)d;
        }
    }
}

// The same for sc = 2^j (c64 / x64 modes), four elements at a time: sc d
// formed exactly from the FP32 bits (no FP64 multiply or conversion), one
// FP64 addition per element.
__global__ void pcg_combine_pow2_kernel(long long N4, CombineArgs a, const float4* __restrict__ x32, int j,
                                        double2* __restrict__ c64, double2* __restrict__ x64) {
    __shared__ float s_al[kPRing];
    if (threadIdx.x < a.cnt) s_al[threadIdx.x] = (float)*a.alpha[threadIdx.x];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N4; i += (long long)gridDim.x * blockDim.x) {
        float4 d = a.fold ? x32[i] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int t = 0; t < kPRing; ++t)
            if (t < a.cnt) {
                const float4 pv = reinterpret_cast<const float4*>(a.p[t])[i];
                d.x = fmaf(s_al[t], pv.x, d.x);
                d.y = fmaf(s_al[t], pv.y, d.y);
                d.z = fmaf(s_al[t], pv.z, d.z);
                d.w = fmaf(s_al[t], pv.w, d.w);
            }
        const double2 v0 = make_double2(f32_pow2_to_f64(d.x, j), f32_pow2_to_f64(d.y, j));
        const double2 v1 = make_double2(f32_pow2_to_f64(d.z, j), f32_pow2_to_f64(d.w, j));
        if (c64) {
            c64[2 * i] = v0;
            c64[2 * i + 1] = v1;
        }
        double2 x0 = x64[2 * i], x1 = x64[2 * i + 1];
        x0.x += v0.x;
        x0.y += v0.y;
        x1.x += v1.x;
        x1.y += v1.y;
        x64[2 * i] = x0;
        x64[2 * i + 1] = x1;
    }
}

// d = (x32 when fold) + sum_j alpha_j p_j as split planes (h, l) alone, four
// elements at a time (the eigenbasis correction before its sine transform)
__global__ void pcg_combine_split_kernel(long long N4, CombineArgs a, const float4* __restrict__ x32,
                                         uint2* __restrict__ h, uint2* __restrict__ l) {
    __shared__ float s_al[kPRing];
    if (threadIdx.x < a.cnt) s_al[threadIdx.x] = (float)*a.alpha[threadIdx.x];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N4; i += (long long)gridDim.x * blockDim.x) {
        float4 d = a.fold ? x32[i] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int t = 0; t < kPRing; ++t)
            if (t < a.cnt) {
                const float4 pv = reinterpret_cast<const float4*>(a.p[t])[i];
                d.x = fmaf(s_al[t], pv.x, d.x);
                d.y = fmaf(s_al[t], pv.y, d.y);
                d.z = fmaf(s_al[t], pv.z, d.z);
                d.w = fmaf(s_al[t], pv.w, d.w);
            }
        const uint2 hv = bf16x4_hi(d);
        h[i] = hv;
        l[i] = bf16x4_lo(d, hv);
    }
}

// beta = num / den (device scalars); p = z + beta p ; (ph, pl) = split(p)
__global__ void xpay32_kernel(long long N, const double* __restrict__ num, const double* __restrict__ den,
                              const float* __restrict__ z, float* __restrict__ p, __nv_bfloat16* __restrict__ ph,
                              __nv_bfloat16* __restrict__ pl) {
    __shared__ float s_beta;
    if (threadIdx.x == 0) s_beta = (float)(num[0] / den[0]);
    __syncthreads();
    const float beta = s_beta;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const float v = fmaf(beta, p[i], z[i]);
        p[i] = v;
        split(v, ph[i], pl[i]);
    }
}

// r32 = r64 * s ; rh = bf16(r32) (the hi plane alone, for consumers that read no lo plane)
__global__ void scale64to32_hi_kernel(long long N, const double* __restrict__ r64, double s, float* __restrict__ r32,
                                      __nv_bfloat16* __restrict__ rh) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const float v = (float)(r64[i] * s);
        r32[i] = v;
        rh[i] = __float2bfloat16_rn(v);
    }
}

// The same with s = 2^k, four elements at a time (N4 = N / 4 groups): the
// scaled conversion by integer operations (no FP64 arithmetic).
__global__ void scale64to32_hi_pow2_kernel(long long N4, const ulonglong2* __restrict__ r64, int k,
                                           float4* __restrict__ r32, uint2* __restrict__ rh) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N4; i += (long long)gridDim.x * blockDim.x) {
        const ulonglong2 a = r64[2 * i], b = r64[2 * i + 1];
        const float4 v = make_float4(f64_pow2_to_f32(a.x, k), f64_pow2_to_f32(a.y, k), f64_pow2_to_f32(b.x, k),
                                     f64_pow2_to_f32(b.y, k));
        r32[i] = v;
        rh[i] = bf16x4_hi(v);
    }
}

// (rh, rl) = split(r64 2^k), four elements at a time: the scaled conversion
// by integer operations (no FP64 arithmetic), as scale64to32_hi_pow2
__global__ void split64_pow2_kernel(long long N4, const ulonglong2* __restrict__ r64, int k, uint2* __restrict__ rh,
                                    uint2* __restrict__ rl) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N4; i += (long long)gridDim.x * blockDim.x) {
        const ulonglong2 a = r64[2 * i], b = r64[2 * i + 1];
        const float4 v = make_float4(f64_pow2_to_f32(a.x, k), f64_pow2_to_f32(a.y, k), f64_pow2_to_f32(b.x, k),
                                     f64_pow2_to_f32(b.y, k));
        const uint2 h = bf16x4_hi(v);
        rh[i] = h;
        rl[i] = bf16x4_lo(v, h);
    }
}

// r32 = r64 * s ; (rh, rl) = split(r32) ; x32 = 0
__global__ void scale64to32_kernel(long long N, const double* __restrict__ r64, double s, float* __restrict__ r32,
                                   __nv_bfloat16* __restrict__ rh, __nv_bfloat16* __restrict__ rl,
                                   float* __restrict__ x32) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const float v = (float)(r64[i] * s);
        r32[i] = v;
        split(v, rh[i], rl[i]);
        if (x32) x32[i] = 0.f;
    }
}

// (h, l) = split(v)
__global__ void split32_kernel(long long N, const float* __restrict__ v, __nv_bfloat16* __restrict__ h,
                               __nv_bfloat16* __restrict__ l) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        split(v[i], h[i], l[i]);
}

// (h, l) = split((float) v64 * s)
__global__ void split64_kernel(long long N, const double* __restrict__ v, double s, __nv_bfloat16* __restrict__ h,
                               __nv_bfloat16* __restrict__ l) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        split((float)(v[i] * s), h[i], l[i]);
}

// x64 += s * d32
__global__ void add32to64_kernel(long long N, double s, const float* __restrict__ d, double* __restrict__ x) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        x[i] += s * (double)d[i];
}

// c64 = s * d32 ; x64 += c64
__global__ void widen_add32_kernel(long long N, double s, const float* __restrict__ d, double* __restrict__ c,
                                   double* __restrict__ x) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const double v = s * (double)d[i];
        c[i] = v;
        x[i] += v;
    }
}

// y64 = (double) v32 * s
__global__ void widen32_kernel(long long N, const float* __restrict__ v, double s, double* __restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        y[i] = (double)v[i] * s;
}

// coef[0] = num[0] / den[0]  (device-side scalar, no host round trip)
__global__ void ratio_kernel(const double* num, const double* den, double* coef) { coef[0] = num[0] / den[0]; }

// Up to C dot products <V_j, w>, j = m0 .. m0 + mc - 1, per block into part[j * nblk + b].
template <int C>
__global__ __launch_bounds__(kT) void multidot32_kernel(long long N, int m0, int mc, const float* __restrict__ V,
                                                        long long ldv, const float* __restrict__ w,
                                                        double* __restrict__ part) {
    long long lo, hi;
    chunk(N, lo, hi);
    KSum k[C];
    for (long long i = lo + threadIdx.x; i < hi; i += kT) {
        const float wi = w[i];
#pragma unroll
        for (int j = 0; j < C; ++j)
            if (j < mc) k[j].add(V[(long long)(m0 + j) * ldv + i] * wi);
    }
#pragma unroll
    for (int j = 0; j < C; ++j) {
        if (j < mc) {
            const double t = block_sum64((double)k[j].s - (double)k[j].c);
            if (threadIdx.x == 0) part[(long long)(m0 + j) * gridDim.x + blockIdx.x] = t;
        }
    }
}

// w -= sum_{j < m} h[j] V_j   (h: FP64 coefficients on the device, m <= 128)
__global__ void multiaxpy32_kernel(long long N, int m, const float* __restrict__ V, long long ldv,
                                   const double* __restrict__ h, float* __restrict__ w) {
    __shared__ float hs[128];
    for (int j = threadIdx.x; j < m; j += blockDim.x) hs[j] = (float)h[j];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        float acc = w[i];
        for (int j = 0; j < m; ++j)
            if (hs[j] != 0.f) acc = fmaf(-hs[j], V[(long long)j * ldv + i], acc);
        w[i] = acc;
    }
}

// out = sc * in ; (h, l) = split(out)   (in == out allowed)
__global__ void scale_split32_kernel(long long N, float sc, const float* in, float* out, __nv_bfloat16* __restrict__ h,
                                     __nv_bfloat16* __restrict__ l) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const float v = in[i] * sc;
        out[i] = v;
        split(v, h[i], l[i]);
    }
}

// N a multiple of 4 and every (non-null) vector 16-byte aligned: the
// four-element kernels apply
inline bool aligned16(size_t N, const void* a, const void* b, const void* c, const void* d) {
    const uintptr_t m = (uintptr_t)a | (uintptr_t)b | (uintptr_t)c | (uintptr_t)d;
    return N % 4 == 0 && (m & 15) == 0;
}

inline int grid_for(long long N) {
    long long g = (N + kT - 1) / kT;
    if (g > 152LL * 16) g = 152LL * 16;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

void launch_dot32(size_t N, const float* a, const float* b, double* part, int nblk, cudaStream_t s) {
    stats_count_launch();
    dot32_kernel<<<nblk, kT, 0, s>>>((long long)N, a, b, part);
}
void launch_cg_update32(size_t N, const double* num, const double* den, const float* p, const float* q, float* x,
                        float* r, __nv_bfloat16* rh, __nv_bfloat16* rl, double* rr, cudaStream_t s) {
    stats_count_launch();
    cg_update32_kernel<<<grid_for((long long)N), kT, 0, s>>>((long long)N, num, den, p, q, x, r, rh, rl, rr);
}
void launch_cg_update_r32(size_t N, const double* num, const double* den, const float* q, float* r,
                          __nv_bfloat16* rh, __nv_bfloat16* rl, double* rr, double* alpha_out, cudaStream_t s,
                          const int* skip) {
    stats_count_launch();
    if (aligned16(N, q, r, rh, rl)) {
        const long long N4 = (long long)N / 4;
        cg_update_r32_v4_kernel<<<grid_for(N4), kT, 0, s>>>(N4, num, den, reinterpret_cast<const float4*>(q),
                                                            reinterpret_cast<float4*>(r), reinterpret_cast<uint2*>(rh),
                                                            reinterpret_cast<uint2*>(rl), rr, alpha_out, skip);
        return;
    }
    cg_update_r32_kernel<<<grid_for((long long)N), kT, 0, s>>>((long long)N, num, den, q, r, rh, rl, rr, alpha_out,
                                                               skip);
}
// ------------------------------------------------ device-side inner PCG loop
// Control words ctl[0] = iterations done, ctl[1] = done (stop test met or
// maxit reached), ctl[2] = maxit; device scalars d[] in the inner PCG's slots.

// start of an iteration: <r, z> of the last preconditioner application
// becomes the current one; the accumulators start at zero
__global__ void pcg_head_kernel(double* d, int rz, int rzn, int pq, int rr, const int* ctl) {
    if (ctl[1]) return;
    d[rz] = d[rzn];
    d[rzn] = 0.0;
    d[pq] = 0.0;
    d[rr] = 0.0;
}

// after the residual update: count the iteration, take the stop test
// <r, r> <= thr (or maxit, or a non-finite value) and set the loop condition
__global__ void pcg_cond_kernel(cudaGraphConditionalHandle h, const double* rr, const double* thr, int* ctl) {
    if (ctl[1]) {   // an earlier iteration of this body ended the loop
        cudaGraphSetConditional(h, 0u);
        return;
    }
    const int k = ctl[0] + 1;
    ctl[0] = k;
    const double v = *rr;
    const int done = (!(v > *thr) || k >= ctl[2] || !isfinite(v)) ? 1 : 0;
    ctl[1] = done;
    cudaGraphSetConditional(h, done ? 0u : 1u);
}

__global__ void pcg_init_kernel(double* d, int rzn, int thr_slot, double thr, int* ctl, int maxit) {
    d[rzn] = 0.0;
    d[thr_slot] = thr;
    ctl[0] = 0;
    ctl[1] = 0;
    ctl[2] = maxit;
}

// fold of a full window of kPRing directions into x32 (skipped once the loop
// is done: the host combines what is left); the window is the first one
// (x32 = sum) while ctl[0] <= kPRing, else x32 += sum
__global__ void pcg_fold_dev_kernel(long long N4, CombineArgs a, float4* __restrict__ x32, const int* ctl) {
    if (*reinterpret_cast<const volatile int*>(ctl + 1)) return;
    const bool fold = ctl[0] > kPRing;
    __shared__ float s_al[kPRing];
    if (threadIdx.x < kPRing) s_al[threadIdx.x] = (float)*a.alpha[threadIdx.x];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N4; i += (long long)gridDim.x * blockDim.x) {
        float4 d = fold ? x32[i] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int t = 0; t < kPRing; ++t) {
            const float4 pv = reinterpret_cast<const float4*>(a.p[t])[i];
            d.x = fmaf(s_al[t], pv.x, d.x);
            d.y = fmaf(s_al[t], pv.y, d.y);
            d.z = fmaf(s_al[t], pv.z, d.z);
            d.w = fmaf(s_al[t], pv.w, d.w);
        }
        x32[i] = d;
    }
}

// ------------------------------------------------ device-side GMRES cycle
// Control words gctl[0] = j (Arnoldi steps done), gctl[1] = done, gctl[2] =
// the cycle's step limit, gctl[3] = a non-finite value was met; the
// least-squares state gs[] (FP64) at the GS_* offsets of tfde_mixed.h.  The
// step's vector w is the fixed FP32 vector the preconditioner writes; every
// kernel takes the step index from gctl, so one step is the body of the loop.

// the first m = j + 1 inner products <V_i, w>, 8 basis vectors per sweep of w
__global__ __launch_bounds__(kT) void gm_multidot_kernel(long long N, const float* __restrict__ V, long long ldv,
                                                         const float* __restrict__ w, double* __restrict__ part,
                                                         const int* gctl) {
    if (gctl[1]) return;
    const int m = gctl[0] + 1;
    long long lo, hi;
    chunk(N, lo, hi);
    for (int m0 = 0; m0 < m; m0 += 8) {
        const int mc = m - m0 < 8 ? m - m0 : 8;
        KSum k[8];
        for (long long i = lo + threadIdx.x; i < hi; i += kT) {
            const float wi = w[i];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < mc) k[j].add(V[(long long)(m0 + j) * ldv + i] * wi);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j < mc) {
                const double t = block_sum64((double)k[j].s - (double)k[j].c);
                if (threadIdx.x == 0) part[(long long)(m0 + j) * gridDim.x + blockIdx.x] = t;
            }
        }
    }
}

// out[j] = sum of the block partials of result j, j < m (m = mfix, or the
// step's j + 1 when mfix == 0); one warp per result in a fixed order
__global__ void gm_reduce_kernel(const double* __restrict__ part, int nblk, double* __restrict__ out, int mfix,
                                 const int* gctl) {
    if (gctl[1]) return;
    const int m = mfix > 0 ? mfix : gctl[0] + 1;
    const int j = blockIdx.x;
    if (j >= m) return;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) acc += part[(long long)j * nblk + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) out[j] = acc;
}

// The second Gram-Schmidt pass's projections fused with the first pass's
// update: w -= sum_{i <= j} h[i] V_i over the block's chunk, then the first
// m = j + 1 inner products <V_i, w> of the updated chunk (each thread re-reads
// the elements it wrote), 8 basis vectors per sweep; the same arithmetic as
// a plain multi-axpy followed by gm_multidot_kernel.
__global__ __launch_bounds__(kT) void gm_axpy_dot_kernel(long long N, const float* __restrict__ V, long long ldv,
                                                         const double* __restrict__ h, float* __restrict__ w,
                                                         double* __restrict__ part, const int* gctl) {
    if (gctl[1]) return;
    const int m = gctl[0] + 1;
    __shared__ float hs[128];
    for (int j = threadIdx.x; j < m; j += blockDim.x) hs[j] = (float)h[j];
    __syncthreads();
    long long lo, hi;
    chunk(N, lo, hi);
    for (long long i = lo + threadIdx.x; i < hi; i += kT) {
        float acc = w[i];
        for (int j = 0; j < m; ++j) acc = fmaf(-hs[j], V[(long long)j * ldv + i], acc);
        w[i] = acc;
    }
    for (int m0 = 0; m0 < m; m0 += 8) {
        const int mc = m - m0 < 8 ? m - m0 : 8;
        KSum k[8];
        for (long long i = lo + threadIdx.x; i < hi; i += kT) {
            const float wi = w[i];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < mc) k[j].add(V[(long long)(m0 + j) * ldv + i] * wi);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j < mc) {
                const double t = block_sum64((double)k[j].s - (double)k[j].c);
                if (threadIdx.x == 0) part[(long long)(m0 + j) * gridDim.x + blockIdx.x] = t;
            }
        }
    }
}

// The second pass's update fused with ||w||^2: w -= sum_{i <= j} h[i] V_i over
// the block's chunk and the block's partial sum of the updated w^2 (the
// arithmetic of a plain multi-axpy followed by gm_dot_kernel).
__global__ __launch_bounds__(kT) void gm_axpy_norm_kernel(long long N, const float* __restrict__ V, long long ldv,
                                                          const double* __restrict__ h, float* __restrict__ w,
                                                          double* __restrict__ part, const int* gctl) {
    if (gctl[1]) return;
    const int m = gctl[0] + 1;
    __shared__ float hs[128];
    for (int j = threadIdx.x; j < m; j += blockDim.x) hs[j] = (float)h[j];
    __syncthreads();
    long long lo, hi;
    chunk(N, lo, hi);
    KSum k;
    for (long long i = lo + threadIdx.x; i < hi; i += kT) {
        float acc = w[i];
        for (int j = 0; j < m; ++j) acc = fmaf(-hs[j], V[(long long)j * ldv + i], acc);
        w[i] = acc;
        k.add(acc * acc);
    }
    const double t = block_sum64((double)k.s - (double)k.c);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ __launch_bounds__(kT) void gm_dot_kernel(long long N, const float* __restrict__ a, double* __restrict__ part,
                                                    const int* gctl) {
    if (gctl[1]) return;
    long long lo, hi;
    chunk(N, lo, hi);
    KSum k;
    for (long long i = lo + threadIdx.x; i < hi; i += kT) k.add(a[i] * a[i]);
    const double t = block_sum64((double)k.s - (double)k.c);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// Column j of the Hessenberg matrix (h + h2 from the two Gram-Schmidt
// passes, ||w|| below the diagonal) rotated by the previous Givens
// rotations, the new rotation, the residual estimate |g_{j+1}| (Sec. 3.2 left
// preconditioned GMRES), the stop test and the loop condition.
__global__ void gm_givens_kernel(double* gs, const double* h, const double* h2, const double* ww, int* gctl,
                                 cudaGraphConditionalHandle hc) {
    if (gctl[1]) {   // the loop ends whenever its condition kernel runs on a finished cycle
        cudaGraphSetConditional(hc, 0u);
        return;
    }
    const int j = gctl[0];
    double* g = gs + GS_G;
    double* cs = gs + GS_CS;
    double* sn = gs + GS_SN;
    double* R = gs + GS_R + (long long)j * GS_LD;   // column j, entries 0..j+1
    for (int i = 0; i <= j; ++i) R[i] = h[i] + h2[i];
    const double hn = sqrt(*ww);
    R[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
        const double t = cs[i] * R[i] + sn[i] * R[i + 1];
        R[i + 1] = -sn[i] * R[i] + cs[i] * R[i + 1];
        R[i] = t;
    }
    const double den = hypot(R[j], R[j + 1]);
    cs[j] = den > 0.0 ? R[j] / den : 1.0;
    sn[j] = den > 0.0 ? R[j + 1] / den : 0.0;
    R[j] = den;
    R[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    const double est = fabs(g[j + 1]);
    gs[GS_EST] = est;
    gs[GS_INV] = 1.0 / hn;
    const int k = j + 1;
    gctl[0] = k;
    int done = (est <= gs[GS_THR] || hn == 0.0 || k >= gctl[2]) ? 1 : 0;
    if (!isfinite(hn) || !isfinite(est)) {
        gctl[3] = 1;
        done = 1;
    }
    gctl[1] = done;
    cudaGraphSetConditional(hc, done ? 0u : 1u);
}

// V_j (j = the steps done) = w / ||w|| and its split planes, the next
// operator input
__global__ void gm_scale_basis_kernel(long long N, const float* __restrict__ w, float* V, long long ldv,
                                      const double* gs, const int* gctl, __nv_bfloat16* __restrict__ h,
                                      __nv_bfloat16* __restrict__ l) {
    if (gctl[1]) return;
    const float sc = (float)gs[GS_INV];
    float* out = V + (long long)gctl[0] * ldv;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const float v = w[i] * sc;
        out[i] = v;
        split(v, h[i], l[i]);
    }
}

// cycle start: beta = ||P^{-1} r|| (from the reduced dot), g = beta e_1, the
// stop target ptheta beta, control words
__global__ void gm_start_kernel(double* gs, const double* ww, int* gctl, int maxsteps, double ptheta) {
    const double beta = sqrt(*ww);
    gs[GS_BETA] = beta;
    gs[GS_EST] = beta;
    gs[GS_INV] = 1.0 / beta;
    gs[GS_THR] = ptheta * beta;
    for (int i = 0; i <= GS_MAXM; ++i) gs[GS_G + i] = 0.0;
    gs[GS_G] = beta;
    gctl[0] = 0;
    gctl[1] = (!(beta > 0.0) || !isfinite(beta)) ? 1 : 0;
    gctl[2] = maxsteps;
    gctl[3] = isfinite(beta) ? 0 : 1;
}

// -y (the least-squares solution R y = g over the steps done), zero beyond
__global__ void gm_solve_kernel(const double* gs, const int* gctl, double* ny, int maxm) {
    const int k = gctl[0];
    const double* g = gs + GS_G;
    const double* R = gs + GS_R;
    double y[GS_MAXM];
    for (int i = k - 1; i >= 0; --i) {
        double t = g[i];
        for (int j = i + 1; j < k; ++j) t -= R[(long long)j * GS_LD + i] * y[j];
        y[i] = t / R[(long long)i * GS_LD + i];
    }
    for (int i = 0; i < maxm; ++i) ny[i] = i < k ? -y[i] : 0.0;
}

void launch_gm_step(size_t N, const float* V, float* w, double* part, int nblk, double* hbuf, double* h2buf,
                    double* wwbuf, double* gs, int* gctl, cudaGraphConditionalHandle hc, float* Vout,
                    __nv_bfloat16* ph, __nv_bfloat16* pl, int maxm, cudaStream_t s) {
    stats_count_launch(7);
    const long long n = (long long)N;
    // CGS2: <V, w>; w -= V h and <V, w> again (one pass over the block's chunk);
    // w -= V h2 and ||w||^2 (one pass)
    gm_multidot_kernel<<<nblk, kT, 0, s>>>(n, V, n, w, part, gctl);
    gm_reduce_kernel<<<maxm, 32, 0, s>>>(part, nblk, hbuf, 0, gctl);
    gm_axpy_dot_kernel<<<nblk, kT, 0, s>>>(n, V, n, hbuf, w, part, gctl);
    gm_reduce_kernel<<<maxm, 32, 0, s>>>(part, nblk, h2buf, 0, gctl);
    gm_axpy_norm_kernel<<<nblk, kT, 0, s>>>(n, V, n, h2buf, w, part, gctl);
    gm_reduce_kernel<<<1, 32, 0, s>>>(part, nblk, wwbuf, 1, gctl);
    gm_givens_kernel<<<1, 1, 0, s>>>(gs, hbuf, h2buf, wwbuf, gctl, hc);
    (void)Vout;
    stats_count_launch();
    gm_scale_basis_kernel<<<grid_for(n), kT, 0, s>>>(n, w, const_cast<float*>(V), n, gs, gctl, ph, pl);
}
void launch_gm_start(size_t N, const float* w, double* part, int nblk, double* wwbuf, double* gs, int* gctl,
                     int maxsteps, double ptheta, float* V0, __nv_bfloat16* ph, __nv_bfloat16* pl, cudaStream_t s) {
    stats_count_launch(4);
    const long long n = (long long)N;
    // gctl[1] = 0 here (set by the caller's reset) so that the dot and reduce run
    gm_dot_kernel<<<nblk, kT, 0, s>>>(n, w, part, gctl);
    gm_reduce_kernel<<<1, 32, 0, s>>>(part, nblk, wwbuf, 1, gctl);
    gm_start_kernel<<<1, 1, 0, s>>>(gs, wwbuf, gctl, maxsteps, ptheta);
    gm_scale_basis_kernel<<<grid_for(n), kT, 0, s>>>(n, w, V0, n, gs, gctl, ph, pl);
}
void launch_gm_solve(const double* gs, const int* gctl, double* ny, int maxm, cudaStream_t s) {
    stats_count_launch();
    gm_solve_kernel<<<1, 1, 0, s>>>(gs, gctl, ny, maxm);
}

namespace {
LamView lam_view(const float* lam, const int n[3]) {
    const long long nc = (long long)n[0] * n[1];
    LamView L;
    L.ra = lam;
    L.rb = lam + n[2];
    L.U = reinterpret_cast<const float4*>(lam + 2 * n[2]);
    L.V = reinterpret_cast<const float4*>(lam + 2 * n[2] + nc);
    L.nc4 = nc / 4;
    L.n3 = n[2];
    return L;
}
// x over the float4 groups of a plane, y over planes: about 8 blocks of 256 per SM in all
dim3 spec_grid(const LamView& L) {
    long long gx = (L.nc4 + kT - 1) / kT;
    if (gx > 1024) gx = 1024;
    long long gy = (8LL * tc::num_sms() + gx - 1) / gx;
    if (gy > L.n3) gy = L.n3;
    if (gy < 1) gy = 1;
    return dim3((unsigned)gx, (unsigned)gy);
}
}  // namespace

int launch_spec_update(const float* lam, const int n[3], const double* num, const double* den, const float* q,
                       float* r, double* rz, double* rr, double* alpha_out, cudaStream_t s, const int* skip) {
    const long long nc = (long long)n[0] * n[1];
    if (nc % 4 || !aligned16((size_t)nc * n[2], q, r, nullptr, nullptr) || (reinterpret_cast<uintptr_t>(lam) & 15) ||
        (n[2] % 4))
        return set_error(TFDE_EUNSUPPORTED, "spectral update: n1 n2 a multiple of 4 and 16-byte aligned vectors");
    stats_count_launch();
    const LamView L = lam_view(lam, n);
    spec_update_kernel<<<spec_grid(L), kT, 0, s>>>(L, num, den, reinterpret_cast<const float4*>(q),
                                                   reinterpret_cast<float4*>(r), rz, rr, alpha_out, skip);
    return TFDE_OK;
}

int launch_spec_direction(const float* lam, const int n[3], const double* num, const double* den, const float* r,
                          const float* pold, float* p, __nv_bfloat16* ph, __nv_bfloat16* pl, double* rz,
                          cudaStream_t s, const int* skip) {
    const long long nc = (long long)n[0] * n[1];
    if (nc % 4 || !aligned16((size_t)nc * n[2], r, p, ph, pl) || (reinterpret_cast<uintptr_t>(lam) & 15) ||
        (n[2] % 4) || (pold && (reinterpret_cast<uintptr_t>(pold) & 15)))
        return set_error(TFDE_EUNSUPPORTED, "spectral direction: n1 n2 a multiple of 4 and 16-byte aligned vectors");
    stats_count_launch();
    const LamView L = lam_view(lam, n);
    spec_direction_kernel<<<spec_grid(L), kT, 0, s>>>(L, num, den, reinterpret_cast<const float4*>(r),
                                                      reinterpret_cast<const float4*>(pold),
                                                      reinterpret_cast<float4*>(p), reinterpret_cast<uint2*>(ph),
                                                      reinterpret_cast<uint2*>(pl), rz, skip);
    return TFDE_OK;
}

void launch_pcg_head(double* d, int rz, int rzn, int pq, int rr, const int* ctl, cudaStream_t s) {
    stats_count_launch();
    pcg_head_kernel<<<1, 1, 0, s>>>(d, rz, rzn, pq, rr, ctl);
}
void launch_pcg_cond(cudaGraphConditionalHandle h, const double* rr, const double* thr, int* ctl, cudaStream_t s) {
    stats_count_launch();
    pcg_cond_kernel<<<1, 1, 0, s>>>(h, rr, thr, ctl);
}
void launch_pcg_init(double* d, int rzn, int thr_slot, double thr, int* ctl, int maxit, cudaStream_t s) {
    stats_count_launch();
    pcg_init_kernel<<<1, 1, 0, s>>>(d, rzn, thr_slot, thr, ctl, maxit);
}
void launch_pcg_fold_dev(size_t N, const float* const* p, const double* const* alpha, float* x32, const int* ctl,
                         cudaStream_t s) {
    stats_count_launch();
    CombineArgs a;
    a.cnt = kPRing;
    a.fold = 0;
    for (int j = 0; j < kPRing; ++j) {
        a.p[j] = p[j];
        a.alpha[j] = alpha[j];
    }
    const long long N4 = (long long)N / 4;
    pcg_fold_dev_kernel<<<grid_for(N4), kT, 0, s>>>(N4, a, reinterpret_cast<float4*>(x32), ctl);
}

void launch_pcg_combine(size_t N, const PcgPending& pend, const float* x32, double sc, double* c64, double* x64,
                        float* acc32, cudaStream_t s) {
    stats_count_launch();
    CombineArgs a;
    a.cnt = pend.cnt;
    a.fold = pend.fold ? 1 : 0;
    for (int j = 0; j < kPRing; ++j) {
        a.p[j] = j < pend.cnt ? pend.p[j] : nullptr;
        a.alpha[j] = j < pend.cnt ? pend.alpha[j] : nullptr;
    }
    int j = 0;
    bool vec = x64 && !acc32 && pow2_exponent(sc, &j) && aligned16(N, x32, c64, x64, nullptr);
    for (int t = 0; t < pend.cnt; ++t) vec = vec && aligned16(N, pend.p[t], nullptr, nullptr, nullptr);
    if (vec) {
        const long long N4 = (long long)N / 4;
        pcg_combine_pow2_kernel<<<grid_for(N4), kT, 0, s>>>(N4, a, reinterpret_cast<const float4*>(x32), j,
                                                            reinterpret_cast<double2*>(c64),
                                                            reinterpret_cast<double2*>(x64));
        return;
    }
    pcg_combine_kernel<<<grid_for((long long)N), kT, 0, s>>>((long long)N, a, x32, sc, c64, x64, acc32);
}
int launch_pcg_combine_split(size_t N, const PcgPending& pend, const float* x32, __nv_bfloat16* h, __nv_bfloat16* l,
                             cudaStream_t s) {
    bool vec = aligned16(N, x32, h, l, nullptr);
    for (int t = 0; t < pend.cnt; ++t) vec = vec && aligned16(N, pend.p[t], nullptr, nullptr, nullptr);
    if (!vec) return set_error(TFDE_EUNSUPPORTED, "combine to split planes: 16-byte aligned vectors, N % 4 == 0");
    stats_count_launch();
    CombineArgs a;
    a.cnt = pend.cnt;
    a.fold = pend.fold ? 1 : 0;
    for (int j = 0; j < kPRing; ++j) {
        a.p[j] = j < pend.cnt ? pend.p[j] : nullptr;
        a.alpha[j] = j < pend.cnt ? pend.alpha[j] : nullptr;
    }
    const long long N4 = (long long)N / 4;
    pcg_combine_split_kernel<<<grid_for(N4), kT, 0, s>>>(N4, a, reinterpret_cast<const float4*>(x32),
                                                         reinterpret_cast<uint2*>(h), reinterpret_cast<uint2*>(l));
    return TFDE_OK;
}
void launch_scale64to32_hi(size_t N, const double* r64, double sc, float* r32, __nv_bfloat16* rh, cudaStream_t s) {
    stats_count_launch();
    int k = 0;
    if (pow2_exponent(sc, &k) && aligned16(N, r64, r32, rh, nullptr)) {
        const long long N4 = (long long)N / 4;
        scale64to32_hi_pow2_kernel<<<grid_for(N4), kT, 0, s>>>(N4, reinterpret_cast<const ulonglong2*>(r64), k,
                                                               reinterpret_cast<float4*>(r32),
                                                               reinterpret_cast<uint2*>(rh));
        return;
    }
    scale64to32_hi_kernel<<<grid_for((long long)N), kT, 0, s>>>((long long)N, r64, sc, r32, rh);
}
void launch_widen_add32(size_t N, double sc, const float* d, double* c, double* x, cudaStream_t s) {
    stats_count_launch();
    widen_add32_kernel<<<grid_for((long long)N), kT, 0, s>>>((long long)N, sc, d, c, x);
}
void launch_xpay32(size_t N, const double* num, const double* den, const float* z, float* p, __nv_bfloat16* ph,
                   __nv_bfloat16* pl, cudaStream_t s) {
    stats_count_launch();
    xpay32_kernel<<<grid_for((long long)N), kT, 0, s>>>((long long)N, num, den, z, p, ph, pl);
}
void launch_scale64to32(size_t N, const double* r64, double sc, float* r32, __nv_bfloat16* rh, __nv_bfloat16* rl,
                        float* x32, cudaStream_t s) {
    stats_count_launch();
    scale64to32_kernel<<<grid_for((long long)N), kT, 0, s>>>((long long)N, r64, sc, r32, rh, rl, x32);
}
void launch_split32(size_t N, const float* v, __nv_bfloat16* h, __nv_bfloat16* l, cudaStream_t s) {
    stats_count_launch();
    split32_kernel<<<grid_for((long long)N), kT, 0, s>>>((long long)N, v, h, l);
}
void launch_split64(size_t N, const double* v, double sc, __nv_bfloat16* h, __nv_bfloat16* l, cudaStream_t s) {
    stats_count_launch();
    int k = 0;
    if (pow2_exponent(sc, &k) && aligned16(N, v, h, l, nullptr)) {
        const long long N4 = (long long)N / 4;
        split64_pow2_kernel<<<grid_for(N4), kT, 0, s>>>(N4, reinterpret_cast<const ulonglong2*>(v), k,
                                                        reinterpret_cast<uint2*>(h), reinterpret_cast<uint2*>(l));
        return;
    }
    split64_kernel<<<grid_for((long long)N), kT, 0, s>>>((long long)N, v, sc, h, l);
}
void launch_add32to64(size_t N, double sc, const float* d, double* x, cudaStream_t s) {
    stats_count_launch();
    add32to64_kernel<<<grid_for((long long)N), kT, 0, s>>>((long long)N, sc, d, x);
}
void launch_widen32(size_t N, const float* v, double sc, double* y, cudaStream_t s) {
    stats_count_launch();
    widen32_kernel<<<grid_for((long long)N), kT, 0, s>>>((long long)N, v, sc, y);
}
void launch_ratio(const double* num, const double* den, double* coef, cudaStream_t s) {
    stats_count_launch();
    ratio_kernel<<<1, 1, 0, s>>>(num, den, coef);
}

void launch_multidot32(size_t N, int m, const float* V, size_t ldv, const float* w, double* part, int nblk,
                       cudaStream_t s) {
    for (int m0 = 0; m0 < m; m0 += 8) {
        const int mc = (m - m0) < 8 ? (m - m0) : 8;
        stats_count_launch();
        multidot32_kernel<8><<<nblk, kT, 0, s>>>((long long)N, m0, mc, V, (long long)ldv, w, part);
    }
}
void launch_multiaxpy32(size_t N, int m, const float* V, size_t ldv, const double* h, float* w, cudaStream_t s) {
    stats_count_launch();
    multiaxpy32_kernel<<<grid_for((long long)N), kT, 0, s>>>((long long)N, m, V, (long long)ldv, h, w);
}
void launch_scale_split32(size_t N, float sc, const float* in, float* out, __nv_bfloat16* h, __nv_bfloat16* l,
                          cudaStream_t s) {
    stats_count_launch();
    scale_split32_kernel<<<grid_for((long long)N), kT, 0, s>>>((long long)N, sc, in, out, h, l);
}

}  // namespace tfde
