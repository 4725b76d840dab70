// Batched solve of many independent problems of uneven size (the same
// Crank-Nicolson step of Eq. (CN) / Eq. (linear_sys) per problem, Sec. 3.2
// left-preconditioned GMRES per problem).  The problems advance in lock step
// through the Arnoldi iterations; every split-BF16 operator or preconditioner
// pass is ONE persistent tcgen05 launch over a tile work list that spans all
// problems (largest first), every vector step is one launch over a block table
// of all problems, and each problem's Hessenberg column, Givens rotation and
// stop test run on the device (one thread per problem); the host reads only
// the number of problems still iterating, one step late.  A problem whose
// cycle has converged is masked out of the work lists.  The FP64 refinement residual of each problem (the
// exact-integer slice contraction) and the per-problem right-hand sides run
// on a small pool of streams.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "tfde_internal.h"
#include "tfde_mixed.h"
#include "tfde_stats.h"
#include "tfde_chain.cuh"

namespace tfde {

int assemble_problem(const tfde_params* params, int precision, cudaStream_t s, tfde_problem** out);
int destroy_problem(tfde_problem* P);
int cn_prepare(tfde_problem* P, const double* u_prev, const double* F, const double* x0, double* u_next,
               cudaStream_t s, bool chained, bool* r_given, const double* guess, int* used_guess);
int pcg64(const tfde_problem*, const double*, double*, double, int, tfde_info*, cudaStream_t, bool);
int pgmres64(tfde_problem*, const double*, double*, int, double, int, tfde_info*, cudaStream_t, bool);

namespace {

constexpr int kBT = 256;       // threads per block of the vector kernels
constexpr int kCH = 4096;      // elements per block chunk
constexpr int kHS = 192;       // per-problem Hessenberg stride: H (64) | H2 (64) | -y (64)
constexpr int kSS = 16;        // per-problem scalar stride
constexpr int kStreams = 8;    // stream pool of the per-problem work
constexpr int kPcgMaxIt = 100; // inner PCG iterations per refinement sweep at most
// scalar slots (S_RZ .. S_BETA: the batched inner PCG)
enum { S_SC32 = 0, S_SPLIT = 1, S_ADD = 2, S_BB = 3, S_RR = 4, S_WW = 5, S_RZ = 6, S_RZN = 7, S_PQ = 8, S_RR0 = 9,
       S_BETA = 10, S_PRR = 11 };

// Per-problem vector pointers of the batched kernels.
struct BVec {
    long long N;
    float* x32;
    float* r32;
    float* V;          // basis, vector j at V + j N
    __nv_bfloat16* ph;
    __nv_bfloat16* pl;
    __nv_bfloat16* rh;
    __nv_bfloat16* rl;
    __nv_bfloat16* th;   // split planes of the eigenbasis correction (PL_T1)
    __nv_bfloat16* tl;
    float* W;            // the graph-captured cycle's new Arnoldi vector before it joins the basis
    const double* r64;
    double* x64;
    // the batched inner PCG in the eigenbasis: the direction p (FP32, basis
    // slot V_0) and Lambda's factors [ra (n3) | rb (n3) | U (n1 n2) | V (n1 n2)]
    float* p32;
    const float* lam;
    unsigned nc4;        // n1 n2 / 4
    int n3;
    const double* norms; // ||b||^2, ||r_0||^2 of the problem's last cn_prepare
};

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[kBT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kBT / 32; ++w) t += sh[w];
    return t;
}

// The chunk of block b: problem bi[b], elements [bo[b], min(bo[b] + kCH, N)).
#define BK_PROLOGUE                                        \
    const int inst = bi[blockIdx.x];                       \
    if (!act[inst]) return;                                \
    const BVec& v = vt[inst];                              \
    const long long e0 = bo[blockIdx.x];                   \
    const long long e1 = e0 + kCH < v.N ? e0 + kCH : v.N;

// r32 = r64 * sc ; split into (rh, rl) ; x32 = 0
__global__ __launch_bounds__(kBT) void bk_scale64to32(const BVec* __restrict__ vt, const int* __restrict__ bi,
                                                     const long long* __restrict__ bo, const int* __restrict__ act,
                                                     const double* __restrict__ sc) {
    BK_PROLOGUE
    const double f = sc[inst * kSS + S_SC32];
    for (long long e = e0 + threadIdx.x; e < e1; e += kBT) {
        const float x = (float)(v.r64[e] * f);
        v.r32[e] = x;
        split_bf16(x, v.rh[e], v.rl[e]);
        v.x32[e] = 0.f;
    }
}

// <V_{m0+j}, V_jw>, j < mc (<= 8), per block into part[(m0 + j) * NB + b]
__global__ __launch_bounds__(kBT) void bk_multidot(const BVec* __restrict__ vt, const int* __restrict__ bi,
                                                  const long long* __restrict__ bo, const int* __restrict__ act,
                                                  int m0, int mc, int jw, double* __restrict__ part) {
    const int inst = bi[blockIdx.x];
    const bool on = act[inst] != 0;
    KSum k[8];
    if (on) {
        const BVec& v = vt[inst];
        const long long e0 = bo[blockIdx.x];
        const long long e1 = e0 + kCH < v.N ? e0 + kCH : v.N;
        const float* w = v.V + (long long)jw * v.N;
        for (long long e = e0 + threadIdx.x; e < e1; e += kBT) {
            const float we = w[e];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j < mc) k[j].add(v.V[(long long)(m0 + j) * v.N + e] * we);
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (j < mc) {
            const double t = block_sum((double)k[j].s - (double)k[j].c);
            if (threadIdx.x == 0) part[(long long)(m0 + j) * gridDim.x + blockIdx.x] = t;
        }
    }
}

// out[i * ostride + ooff + j] = sum over problem i's blocks of part[(p0 + j) * NB + b], j < m
__global__ void bk_reduce(const double* __restrict__ part, int NB, const int* __restrict__ bstart,
                          const int* __restrict__ act, int p0, double* __restrict__ out, int ostride, int ooff) {
    const int inst = blockIdx.x, j = blockIdx.y;
    if (!act[inst]) return;
    double acc = 0.0;
    for (int b = bstart[inst] + threadIdx.x; b < bstart[inst + 1]; b += 32) acc += part[(long long)(p0 + j) * NB + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) out[inst * ostride + ooff + j] = acc;
}

// target -= sum_{j < m} coef[i * kHS + coff + j] V_j ; target = V_jt (jt >= 0) or x32 (jt < 0)
__global__ __launch_bounds__(kBT) void bk_multiaxpy(const BVec* __restrict__ vt, const int* __restrict__ bi,
                                                   const long long* __restrict__ bo, const int* __restrict__ act,
                                                   int m, int jt, const double* __restrict__ coef, int coff) {
    BK_PROLOGUE
    __shared__ float hs[64];
    for (int j = threadIdx.x; j < m; j += blockDim.x) hs[j] = (float)coef[inst * kHS + coff + j];
    __syncthreads();
    float* w = jt >= 0 ? v.V + (long long)jt * v.N : v.x32;
    for (long long e = e0 + threadIdx.x; e < e1; e += kBT) {
        float acc = w[e];
        for (int j = 0; j < m; ++j) acc = fmaf(-hs[j], v.V[(long long)j * v.N + e], acc);
        w[e] = acc;
    }
}

// V_jw *= sc ; split into (ph, pl)
__global__ __launch_bounds__(kBT) void bk_scale_split(const BVec* __restrict__ vt, const int* __restrict__ bi,
                                                     const long long* __restrict__ bo, const int* __restrict__ act,
                                                     int jw, const double* __restrict__ sc) {
    BK_PROLOGUE
    const float f = (float)sc[inst * kSS + S_SPLIT];
    float* w = v.V + (long long)jw * v.N;
    for (long long e = e0 + threadIdx.x; e < e1; e += kBT) {
        const float x = w[e] * f;
        w[e] = x;
        split_bf16(x, v.ph[e], v.pl[e]);
    }
}

// (th, tl) = split(x32): the cycle's correction in the eigenbasis, before
// its sine transform back to the grid
__global__ __launch_bounds__(kBT) void bk_split_x32(const BVec* __restrict__ vt, const int* __restrict__ bi,
                                                   const long long* __restrict__ bo, const int* __restrict__ act) {
    BK_PROLOGUE
    for (long long e = e0 + threadIdx.x; e < e1; e += kBT) split_bf16(v.x32[e], v.th[e], v.tl[e]);
}

// x64 += sc * x32
__global__ __launch_bounds__(kBT) void bk_add32to64(const BVec* __restrict__ vt, const int* __restrict__ bi,
                                                   const long long* __restrict__ bo, const int* __restrict__ act,
                                                   const double* __restrict__ sc) {
    BK_PROLOGUE
    const double f = sc[inst * kSS + S_ADD];
    for (long long e = e0 + threadIdx.x; e < e1; e += kBT) v.x64[e] += f * (double)v.x32[e];
}

// ---- the batched inner PCG (Sec. 3.1) in the sine-transform eigenbasis,
// where the tau preconditioner is the diagonal Lambda (Eq. (diag_tau_pre)):
// per problem r~ = S_N r (r32), p (p32 and its split planes), x~ (x32),
// q = S_N A S_N p (W); the scalars in the problem's slots.  Elements go four
// at a time (a chunk holds whole groups: N and kCH are multiples of 4).
__device__ __forceinline__ float4 bk_lam4(const BVec& v, unsigned e4) {
    const unsigned k = e4 / v.nc4, c4 = e4 - k * v.nc4;
    const float ra = __ldg(v.lam + k), rb = __ldg(v.lam + v.n3 + k);
    const float4 u = __ldg(reinterpret_cast<const float4*>(v.lam + 2 * v.n3) + c4);
    const float4 w = __ldg(reinterpret_cast<const float4*>(v.lam + 2 * v.n3) + v.nc4 + c4);
    return make_float4(fmaf(ra, u.x, rb * w.x), fmaf(ra, u.y, rb * w.y), fmaf(ra, u.z, rb * w.z),
                       fmaf(ra, u.w, rb * w.w));
}
__device__ __forceinline__ void split4(const float4 z, __nv_bfloat16* hi, __nv_bfloat16* lo, long long e) {
    split_bf16(z.x, hi[e], lo[e]);
    split_bf16(z.y, hi[e + 1], lo[e + 1]);
    split_bf16(z.z, hi[e + 2], lo[e + 2]);
    split_bf16(z.w, hi[e + 3], lo[e + 3]);
}
__device__ __forceinline__ void ksum4(KSum& k, float4 a, float4 b) {
    k.add(a.x * b.x);
    k.add(a.y * b.y);
    k.add(a.z * b.z);
    k.add(a.w * b.w);
}

// ---- the chained steps' right-hand sides and corrected guesses of every
// problem at once (the per-point arithmetic of tfde_chain.cuh, as
// cn_prepare's order-3 path): the five sums of the guess correction, their
// 2 x 2 solve per problem, then b^m, x0 and r = b^m - A x0 with ||b||^2,
// ||r||^2.  Per-problem pointers in a ChainDesc.
struct ChainDesc {
    const double* AN;
    const double* F;
    double* b;
    double* r;
    double* u;
    const double* U1;
    const double* AU1;
    double* U2;
    double* AU2;
    double dt;
};

__global__ __launch_bounds__(kBT) void bkc_mr_dots(const ChainDesc* __restrict__ cd, const BVec* __restrict__ vt,
                                                  const int* __restrict__ bi, const long long* __restrict__ bo,
                                                  const int* __restrict__ act, double* __restrict__ part) {
    BK_PROLOGUE
    const ChainDesc& c = cd[inst];
    const float dtf = (float)c.dt;
    float s5[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (long long e = e0 + threadIdx.x; e < e1; e += kBT)
        chain_mr_terms(__ldg(c.AN + e), c.F, e, dtf, __ldg(c.b + e), __ldg(c.r + e), __ldg(c.AU1 + e),
                       __ldg(c.AU2 + e), s5);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const double t = block_sum((double)s5[q]);
        if (threadIdx.x == 0) part[(long long)q * gridDim.x + blockIdx.x] = t;
    }
}

__global__ void bkc_coef(int C, const double* __restrict__ mr, double* __restrict__ g, const int* __restrict__ act) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < C && act[i]) chain_mr_coefficients(mr + (size_t)i * 8, g + (size_t)i * 4);
}

__global__ __launch_bounds__(kBT) void bkc_chain(const ChainDesc* __restrict__ cd, const BVec* __restrict__ vt,
                                                const int* __restrict__ bi, const long long* __restrict__ bo,
                                                const int* __restrict__ act, const double* __restrict__ g,
                                                double* __restrict__ part) {
    BK_PROLOGUE
    const ChainDesc& c = cd[inst];
    const double g0 = g[(size_t)inst * 4], g1 = g[(size_t)inst * 4 + 1], g2 = g[(size_t)inst * 4 + 2];
    float bb = 0.f, rr = 0.f;
    for (long long e = e0 + threadIdx.x; e < e1; e += kBT) {
        double bn, rn;
        chain_extrap_point(e, c.AN, c.F, c.dt, c.b, c.r, c.u, c.U1, c.AU1, c.U2, c.AU2, 3, g0, g1, g2, &bn, &rn);
        const float bf = chain_f32(bn), rf = chain_f32(rn);
        bb = fmaf(bf, bf, bb);
        rr = fmaf(rf, rf, rr);
    }
    const double t1 = block_sum((double)bb);
    const double t2 = block_sum((double)rr);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = t1;
        part[(long long)gridDim.x + blockIdx.x] = t2;
    }
}

// S_BB, S_RR of every problem from the norms its cn_prepare formed
__global__ void bk_gather_norms(int C, const BVec* __restrict__ vt, double* __restrict__ s) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C) return;
    s[i * kSS + S_BB] = vt[i].norms[0];
    s[i * kSS + S_RR] = vt[i].norms[1];
}

// zero the sums of a new inner solve
__global__ void bkp_reset(int C, double* __restrict__ s, const int* __restrict__ act) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C || !act[i]) return;
    s[i * kSS + S_RZ] = 0.0;
    s[i * kSS + S_RR0] = 0.0;
}

// p = Lambda^{-1} r~ and its split planes; S_RZ += <r~, p>, S_RR0 += <r~, r~>
__global__ __launch_bounds__(kBT) void bkp_first(const BVec* __restrict__ vt, const int* __restrict__ bi,
                                                const long long* __restrict__ bo, const int* __restrict__ act,
                                                double* __restrict__ s) {
    BK_PROLOGUE
    KSum kz, kr;
    const float4* r4 = reinterpret_cast<const float4*>(v.r32);
    float4* p4 = reinterpret_cast<float4*>(v.p32);
    for (long long e = e0 + 4 * threadIdx.x; e < e1; e += 4 * kBT) {
        const unsigned e4 = (unsigned)(e >> 2);
        const float4 rv = r4[e4];
        const float4 l = bk_lam4(v, e4);
        const float4 z = make_float4(rv.x / l.x, rv.y / l.y, rv.z / l.z, rv.w / l.w);
        p4[e4] = z;
        split4(z, v.ph, v.pl, e);
        ksum4(kz, rv, z);
        ksum4(kr, rv, rv);
    }
    const double tz = block_sum((double)kz.s - (double)kz.c);
    const double tr = block_sum((double)kr.s - (double)kr.c);
    if (threadIdx.x == 0) {
        atomicAdd(s + inst * kSS + S_RZ, tz);
        atomicAdd(s + inst * kSS + S_RR0, tr);
    }
}

// alpha = S_RZ / S_PQ; x~ += alpha p; r~ -= alpha q; S_RZN += <r~, Lambda^{-1} r~>,
// S_PRR += <r~, r~>
__global__ __launch_bounds__(kBT) void bkp_update(const BVec* __restrict__ vt, const int* __restrict__ bi,
                                                 const long long* __restrict__ bo, const int* __restrict__ act,
                                                 double* __restrict__ s) {
    BK_PROLOGUE
    const float alpha = (float)(s[inst * kSS + S_RZ] / s[inst * kSS + S_PQ]);
    KSum kz, kr;
    float4* r4 = reinterpret_cast<float4*>(v.r32);
    float4* x4 = reinterpret_cast<float4*>(v.x32);
    const float4* p4 = reinterpret_cast<const float4*>(v.p32);
    const float4* q4 = reinterpret_cast<const float4*>(v.W);
    for (long long e = e0 + 4 * threadIdx.x; e < e1; e += 4 * kBT) {
        const unsigned e4 = (unsigned)(e >> 2);
        const float4 pv = p4[e4], qv = q4[e4];
        float4 xv = x4[e4], rv = r4[e4];
        xv.x = fmaf(alpha, pv.x, xv.x);
        xv.y = fmaf(alpha, pv.y, xv.y);
        xv.z = fmaf(alpha, pv.z, xv.z);
        xv.w = fmaf(alpha, pv.w, xv.w);
        rv.x = fmaf(-alpha, qv.x, rv.x);
        rv.y = fmaf(-alpha, qv.y, rv.y);
        rv.z = fmaf(-alpha, qv.z, rv.z);
        rv.w = fmaf(-alpha, qv.w, rv.w);
        x4[e4] = xv;
        r4[e4] = rv;
        const float4 l = bk_lam4(v, e4);
        ksum4(kz, rv, make_float4(rv.x / l.x, rv.y / l.y, rv.z / l.z, rv.w / l.w));
        ksum4(kr, rv, rv);
    }
    const double tz = block_sum((double)kz.s - (double)kz.c);
    const double tr = block_sum((double)kr.s - (double)kr.c);
    if (threadIdx.x == 0) {
        atomicAdd(s + inst * kSS + S_RZN, tz);
        atomicAdd(s + inst * kSS + S_PRR, tr);
    }
}

// p = Lambda^{-1} r~ + S_BETA p and its split planes
__global__ __launch_bounds__(kBT) void bkp_direction(const BVec* __restrict__ vt, const int* __restrict__ bi,
                                                    const long long* __restrict__ bo, const int* __restrict__ act,
                                                    const double* __restrict__ s) {
    BK_PROLOGUE
    const float beta = (float)s[inst * kSS + S_BETA];
    const float4* r4 = reinterpret_cast<const float4*>(v.r32);
    float4* p4 = reinterpret_cast<float4*>(v.p32);
    for (long long e = e0 + 4 * threadIdx.x; e < e1; e += 4 * kBT) {
        const unsigned e4 = (unsigned)(e >> 2);
        const float4 rv = r4[e4], po = p4[e4];
        const float4 l = bk_lam4(v, e4);
        const float4 z = make_float4(fmaf(beta, po.x, rv.x / l.x), fmaf(beta, po.y, rv.y / l.y),
                                     fmaf(beta, po.z, rv.z / l.z), fmaf(beta, po.w, rv.w / l.w));
        p4[e4] = z;
        split4(z, v.ph, v.pl, e);
    }
}

// ---- the same steps for the graph-captured cycle: the step index j comes
// from *jd (device), the new vector is the fixed per-problem W.
// Block partial sums of <V_{m0+t}, W> for t < min(8, j + 1 - m0), or (ww) of
// <W, W> into row R + 1.
__global__ __launch_bounds__(kBT) void bkg_dots(const BVec* __restrict__ vt, const int* __restrict__ bi,
                                               const long long* __restrict__ bo, const int* __restrict__ act,
                                               int m0, const int* __restrict__ jd, int R, int ww,
                                               double* __restrict__ part) {
    const int inst = bi[blockIdx.x];
    const int j = *jd;
    const int mc = ww ? 1 : min(8, j + 1 - m0);
    if (mc <= 0) return;
    const bool on = act[inst] != 0;
    KSum k[8];
    if (on) {
        const BVec& v = vt[inst];
        const long long e0 = bo[blockIdx.x];
        const long long e1 = e0 + kCH < v.N ? e0 + kCH : v.N;
        for (long long e = e0 + threadIdx.x; e < e1; e += kBT) {
            const float we = v.W[e];
            if (ww) {
                k[0].add(we * we);
                continue;
            }
#pragma unroll
            for (int t = 0; t < 8; ++t)
                if (t < mc) k[t].add(v.V[(long long)(m0 + t) * v.N + e] * we);
        }
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        if (t < mc) {
            const double sum = block_sum((double)k[t].s - (double)k[t].c);
            const int row = ww ? R + 1 : m0 + t;
            if (threadIdx.x == 0) part[(long long)row * gridDim.x + blockIdx.x] = sum;
        }
    }
}

// out[i * ostride + ooff + t] = sum over problem i's blocks, t <= j (rows
// 0 .. j), or (ww) row R + 1 into out[i * ostride + ooff]
__global__ void bkg_reduce(const double* __restrict__ part, int NB, const int* __restrict__ bstart,
                           const int* __restrict__ act, const int* __restrict__ jd, int R, int ww,
                           double* __restrict__ out, int ostride, int ooff) {
    const int inst = blockIdx.x, t = blockIdx.y;
    if (!act[inst] || t > (ww ? 0 : *jd)) return;
    const int row = ww ? R + 1 : t;
    double acc = 0.0;
    for (int b = bstart[inst] + threadIdx.x; b < bstart[inst + 1]; b += 32) acc += part[(long long)row * NB + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) out[inst * ostride + ooff + t] = acc;
}

// The second Gram-Schmidt pass's projections fused with the first pass's
// update: W -= sum_{t <= j} coef[i * kHS + coff + t] V_t over the block's
// chunk, then the block partial sums of <V_t, W> (t <= j) of the updated
// chunk into rows t of part (each thread re-reads the elements it wrote):
// the arithmetic of a plain multi-axpy followed by bkg_dots.
__global__ __launch_bounds__(kBT) void bkg_axpy_dots(const BVec* __restrict__ vt, const int* __restrict__ bi,
                                                    const long long* __restrict__ bo, const int* __restrict__ act,
                                                    const int* __restrict__ jd, const double* __restrict__ coef,
                                                    int coff, double* __restrict__ part) {
    BK_PROLOGUE
    const int m = *jd + 1;
    __shared__ float hs[64];
    for (int t = threadIdx.x; t < m; t += blockDim.x) hs[t] = (float)coef[inst * kHS + coff + t];
    __syncthreads();
    for (long long e = e0 + threadIdx.x; e < e1; e += kBT) {
        float acc = v.W[e];
        for (int t = 0; t < m; ++t) acc = fmaf(-hs[t], v.V[(long long)t * v.N + e], acc);
        v.W[e] = acc;
    }
    for (int m0 = 0; m0 < m; m0 += 8) {
        const int mc = min(8, m - m0);
        KSum k[8];
        for (long long e = e0 + threadIdx.x; e < e1; e += kBT) {
            const float we = v.W[e];
#pragma unroll
            for (int t = 0; t < 8; ++t)
                if (t < mc) k[t].add(v.V[(long long)(m0 + t) * v.N + e] * we);
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            if (t < mc) {
                const double sum = block_sum((double)k[t].s - (double)k[t].c);
                if (threadIdx.x == 0) part[(long long)(m0 + t) * gridDim.x + blockIdx.x] = sum;
            }
        }
    }
}

// The second pass's update fused with ||W||^2: W -= sum_{t <= j} coef V_t and
// the block partial sum of the updated W^2 into row R + 1 of part.
__global__ __launch_bounds__(kBT) void bkg_axpy_ww(const BVec* __restrict__ vt, const int* __restrict__ bi,
                                                  const long long* __restrict__ bo, const int* __restrict__ act,
                                                  const int* __restrict__ jd, const double* __restrict__ coef,
                                                  int coff, int R, double* __restrict__ part) {
    BK_PROLOGUE
    const int m = *jd + 1;
    __shared__ float hs[64];
    for (int t = threadIdx.x; t < m; t += blockDim.x) hs[t] = (float)coef[inst * kHS + coff + t];
    __syncthreads();
    KSum k;
    for (long long e = e0 + threadIdx.x; e < e1; e += kBT) {
        float acc = v.W[e];
        for (int t = 0; t < m; ++t) acc = fmaf(-hs[t], v.V[(long long)t * v.N + e], acc);
        v.W[e] = acc;
        k.add(acc * acc);
    }
    const double sum = block_sum((double)k.s - (double)k.c);
    if (threadIdx.x == 0) part[(long long)(R + 1) * gridDim.x + blockIdx.x] = sum;
}

// V_{j+1} = W sc and its split planes (ph, pl)
__global__ __launch_bounds__(kBT) void bkg_scale_split(const BVec* __restrict__ vt, const int* __restrict__ bi,
                                                      const long long* __restrict__ bo, const int* __restrict__ act,
                                                      const int* __restrict__ jd, const double* __restrict__ sc) {
    BK_PROLOGUE
    const float f = (float)sc[inst * kSS + S_SPLIT];
    float* w = v.V + (long long)(*jd + 1) * v.N;
    for (long long e = e0 + threadIdx.x; e < e1; e += kBT) {
        const float x = v.W[e] * f;
        w[e] = x;
        split_bf16(x, v.ph[e], v.pl[e]);
    }
}

#undef BK_PROLOGUE

// ---- the cycle's least-squares problem on the device, one thread per problem.
// Per-problem state (stride gs_stride(R) doubles): the rotated Hessenberg
// matrix (row q, column j at q R + j, rows 0..R), cs[R], sn[R], g[R + 1], beta.
// The operations are those of GivensLS (tfde_givens.h), in the same order.
__host__ __device__ constexpr int gs_stride(int R) { return (R + 1) * R + 3 * R + 2; }

// start of a cycle: beta = ||P^{-1} r|| from S_WW, g = beta e_1, V_0 scale;
// act[i] (on entry: the problem takes part) stays set when beta > 0
__global__ void bk_cycle_start(int C, int R, double* __restrict__ gs, double* __restrict__ s, int* __restrict__ act,
                               int* __restrict__ its, double* __restrict__ est, int* __restrict__ cnt,
                               int* __restrict__ bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C) return;
    its[i] = 0;
    est[i] = 1.0;
    if (!act[i]) return;
    double* g = gs + (size_t)i * gs_stride(R) + (R + 1) * R + 2 * R;
    const double beta = sqrt(s[i * kSS + S_WW]);
    for (int q = 0; q <= R; ++q) g[q] = 0.0;
    g[0] = beta;
    g[R + 1] = beta;
    if (!isfinite(beta)) {
        atomicOr(bad, 1);
        act[i] = 0;
        return;
    }
    if (beta > 0.0) {
        s[i * kSS + S_SPLIT] = 1.0 / beta;
        atomicAdd(cnt, 1);
    } else {
        act[i] = 0;
    }
}

// Arnoldi step j: column j of the Hessenberg matrix (the two CGS projections
// summed, ||w|| from S_WW) rotated into the least-squares state, the new
// rotation, the residual estimate |g_{j+1}|; the problem leaves the cycle
// when that estimate reaches theta beta, else V_{j+1} gets the scale 1/||w||.
// *cnt counts the problems still in the cycle.
__device__ __forceinline__ void givens_step(int i, int R, int j, double* __restrict__ gs,
                                            const double* __restrict__ h, double* __restrict__ s,
                                            const double* __restrict__ theta, int* __restrict__ act,
                                            int* __restrict__ its, double* __restrict__ est, int* __restrict__ cnt,
                                            int* __restrict__ bad);

__global__ void bk_givens(int C, int R, int j, double* __restrict__ gs, const double* __restrict__ h,
                          double* __restrict__ s, const double* __restrict__ theta, int* __restrict__ act,
                          int* __restrict__ its, double* __restrict__ est, int* __restrict__ cnt,
                          int* __restrict__ bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C || !act[i]) return;
    givens_step(i, R, j, gs, h, s, theta, act, its, est, cnt, bad);
}

// the same with j = *jd, the count into cnt[j + 1]
__global__ void bkg_givens(int C, int R, const int* __restrict__ jd, double* __restrict__ gs,
                           const double* __restrict__ h, double* __restrict__ s, const double* __restrict__ theta,
                           int* __restrict__ act, int* __restrict__ its, double* __restrict__ est,
                           int* __restrict__ cnt, int* __restrict__ bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C || !act[i]) return;
    const int j = *jd;
    givens_step(i, R, j, gs, h, s, theta, act, its, est, cnt + j + 1, bad);
}

// the loop condition of the graph-captured cycle: another step while a
// problem is still in the cycle and the restart length is not reached
__global__ void bkg_next(int* __restrict__ jd, const int* __restrict__ cnt, int R, cudaGraphConditionalHandle hc) {
    const int j = *jd + 1;
    *jd = j;
    cudaGraphSetConditional(hc, (cnt[j] > 0 && j < R) ? 1u : 0u);
}

__device__ __forceinline__ void givens_step(int i, int R, int j, double* __restrict__ gs,
                                            const double* __restrict__ h, double* __restrict__ s,
                                            const double* __restrict__ theta, int* __restrict__ act,
                                            int* __restrict__ its, double* __restrict__ est, int* __restrict__ cnt,
                                            int* __restrict__ bad) {
    double* Rm = gs + (size_t)i * gs_stride(R);
    double* cs = Rm + (R + 1) * R;
    double* sn = cs + R;
    double* g = sn + R;
    const double beta = g[R + 1];
    const double* hc = h + (size_t)i * kHS;
    const double hn = sqrt(s[i * kSS + S_WW]);
    if (!isfinite(hn)) {
        atomicOr(bad, 1);
        act[i] = 0;
        return;
    }
    for (int q = 0; q <= j; ++q) Rm[q * R + j] = hc[q] + hc[64 + q];
    Rm[(j + 1) * R + j] = hn;
    for (int q = 0; q < j; ++q) {
        const double t = cs[q] * Rm[q * R + j] + sn[q] * Rm[(q + 1) * R + j];
        Rm[(q + 1) * R + j] = -sn[q] * Rm[q * R + j] + cs[q] * Rm[(q + 1) * R + j];
        Rm[q * R + j] = t;
    }
    const double den = hypot(Rm[j * R + j], Rm[(j + 1) * R + j]);
    cs[j] = den > 0.0 ? Rm[j * R + j] / den : 1.0;
    sn[j] = den > 0.0 ? Rm[(j + 1) * R + j] / den : 0.0;
    Rm[j * R + j] = den;
    Rm[(j + 1) * R + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    const double e = fabs(g[j + 1]);
    its[i] = j + 1;
    est[i] = e / beta;
    if (e <= theta[i] * beta || hn == 0.0) {
        act[i] = 0;
    } else {
        s[i * kSS + S_SPLIT] = 1.0 / hn;
        atomicAdd(cnt, 1);
    }
}

// end of a cycle: y from the triangular system R y = g (its[i] columns),
// -y into the coefficient slots (the multi-axpy subtracts), zeros after it
__global__ void bk_cycle_solve(int C, int R, const double* __restrict__ gs, const int* __restrict__ its,
                               double* __restrict__ h) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C) return;
    double* y = h + (size_t)i * kHS + 128;
    for (int q = 0; q < 64; ++q) y[q] = 0.0;
    const int k = its[i];
    const double* Rm = gs + (size_t)i * gs_stride(R);
    const double* g = Rm + (R + 1) * R + 2 * R;
    for (int a = k - 1; a >= 0; --a) {
        double t = g[a];
        for (int b = a + 1; b < k; ++b) t -= Rm[a * R + b] * y[b];
        y[a] = t / Rm[a * R + a];
    }
    for (int a = 0; a < k; ++a) y[a] = -y[a];
}

// start of a batched inner PCG: a problem with <r~, Lambda^{-1} r~> > 0 takes
// part (act stays set, *cnt counts it), its sums of the first iteration zeroed
__global__ void bkp_start(int C, double* __restrict__ s, int* __restrict__ act, int* __restrict__ its,
                          double* __restrict__ est, int* __restrict__ cnt, int* __restrict__ bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C) return;
    its[i] = 0;
    est[i] = 1.0;
    if (!act[i]) return;
    double* si = s + (size_t)i * kSS;
    if (!isfinite(si[S_RZ]) || !isfinite(si[S_RR0])) {
        atomicOr(bad, 1);
        act[i] = 0;
        return;
    }
    if (!(si[S_RZ] > 0.0) || !(si[S_RR0] > 0.0)) {
        act[i] = 0;
        return;
    }
    si[S_PQ] = 0.0;
    si[S_RZN] = 0.0;
    si[S_PRR] = 0.0;
    atomicAdd(cnt, 1);
}

// stop test after PCG iteration j: the problem leaves once ||r~|| <= theta
// ||r~_0|| (r~ is S_N r and S_N is orthogonal: the true inner residual) or
// after maxit iterations; else beta = S_RZN / S_RZ for the direction, the
// sums rotated and zeroed for the next iteration, and *cnt counts it
__device__ __forceinline__ void bkp_stop_body(int C, int j, int maxit, double* __restrict__ s,
                                              const double* __restrict__ theta, int* __restrict__ act,
                                              int* __restrict__ its, double* __restrict__ est, int* __restrict__ cnt,
                                              int* __restrict__ bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C || !act[i]) return;
    double* si = s + (size_t)i * kSS;
    const double rr = si[S_PRR], rr0 = si[S_RR0];
    its[i] = j + 1;
    est[i] = sqrt(rr / rr0);
    if (!isfinite(rr) || !isfinite(si[S_RZN]) || !isfinite(si[S_PQ])) {
        atomicOr(bad, 1);
        act[i] = 0;
        return;
    }
    if (rr <= theta[i] * theta[i] * rr0 || j + 1 >= maxit || !(si[S_RZN] > 0.0)) {
        act[i] = 0;
        return;
    }
    si[S_BETA] = si[S_RZN] / si[S_RZ];
    si[S_RZ] = si[S_RZN];
    si[S_RZN] = 0.0;
    si[S_PRR] = 0.0;
    si[S_PQ] = 0.0;
    atomicAdd(cnt, 1);
}
__global__ void bkp_stop(int C, int j, int maxit, double* __restrict__ s, const double* __restrict__ theta,
                         int* __restrict__ act, int* __restrict__ its, double* __restrict__ est,
                         int* __restrict__ cnt, int* __restrict__ bad) {
    bkp_stop_body(C, j, maxit, s, theta, act, its, est, cnt, bad);
}

// bkp_stop with the iteration index j = *jd (the graph-captured loop)
__global__ void bkpg_stop(int C, const int* __restrict__ jd, int maxit, double* __restrict__ s,
                          const double* __restrict__ theta, int* __restrict__ act, int* __restrict__ its,
                          double* __restrict__ est, int* __restrict__ cnt, int* __restrict__ bad) {
    const int j = *jd;
    bkp_stop_body(C, j, maxit, s, theta, act, its, est, cnt + j + 1, bad);
}

using clk = std::chrono::steady_clock;

}  // namespace
}  // namespace tfde

struct tfde_batch {
    int count = 0;
    int restart = 20;
    std::vector<tfde_problem*> P;   // sorted by decreasing size
    std::vector<int> caller;        // sorted position -> caller index
    // grouped descriptors: matvec passes [5][count], preconditioner passes
    // 0..4 [5][count], last preconditioner pass writing V_j [restart+1][count]
    tfde::tc::Params* d_mv = nullptr;
    tfde::tc::Params* d_pc = nullptr;
    tfde::tc::Params* d_pcl = nullptr;
    int mv_axis[5] = {}, pc_axis[6] = {};
    int mv_out[5] = {}, pc_out[6] = {};   // output mode of each pass
    double mv_bytes[5] = {}, mv_flops[5] = {}, pc_bytes[6] = {}, pc_flops[6] = {};
    // the eigenbasis cycle (spectral, default): forward sine transform with
    // Lambda^{-1} fused [3][count] (the z pass writes V_0), the operator's x
    // and y passes [2][count], its z pass writing V_j [restart+1][count], the
    // backward transform [3][count]
    bool spectral = true;
    // the eigenbasis Arnoldi steps as one graph launch per cycle (a while
    // node; the step index on the device, the z pass writing each problem's W)
    bool device_loop = true;
    tfde::tc::Params* d_sopzw = nullptr;   // [count]
    int* d_j = nullptr;
    cudaGraph_t cyc_graph = nullptr;
    cudaGraphExec_t cyc_exec = nullptr;
    bool cyc_failed = false;
    unsigned cyc_tune_gen = 0;
    long long graph_cycles = 0;   // cycles run through the graph (tfde_batch_graph_cycles)
    tfde::tc::Params* d_sfw = nullptr;
    tfde::tc::Params* d_sop = nullptr;
    tfde::tc::Params* d_sopz = nullptr;
    tfde::tc::Params* d_sbw = nullptr;
    double sfw_bytes[3] = {}, sfw_flops[3] = {}, sop_bytes[3] = {}, sop_flops[3] = {}, sbw_bytes[3] = {},
           sbw_flops[3] = {};
    // symmetric problems take the batched inner PCG (Sec. 3.1) in the
    // eigenbasis (tfde_batch_set_symmetric_pcg): the forward transform to
    // S_N r [3][count] and the operator's z pass with <p, q> [count]
    bool sym_pcg = true;
    tfde::tc::Params* d_sfp = nullptr;
    tfde::tc::Params* d_sopq = nullptr;
    double sfp_bytes[3] = {}, sfp_flops[3] = {}, sopq_bytes = 0.0, sopq_flops = 0.0;
    long long pcg_solves = 0;       // problem-sweeps solved by the batched PCG
    // its iterations as one graph launch per sweep (a while node, the
    // iteration index and each problem's stop test on the device)
    cudaGraph_t pcg_graph = nullptr;
    cudaGraphExec_t pcg_exec = nullptr;
    bool pcg_failed = false;
    unsigned pcg_tune_gen = 0;
    long long pcg_graph_launches = 0;
    long long* d_gstart = nullptr;  // [3][count + 1]
    long long gtotal[3] = {};
    // vector kernels: per-problem pointers and the block table
    tfde::BVec* d_vt = nullptr;
    tfde::BVec* h_vt = nullptr;
    int* d_bi = nullptr;
    long long* d_bo = nullptr;
    int* d_bstart = nullptr;
    int NB = 0;
    double* d_part = nullptr;       // max(restart + 2, 5) * NB partial sums
    double* d_h = nullptr;          // count * kHS
    double* d_s = nullptr;          // count * kSS
    double* h_s = nullptr;
    int* d_act = nullptr;
    int* h_act = nullptr;
    int* d_err = nullptr;
    int* h_err = nullptr;
    // the device-side cycle: Givens state, per-problem targets, steps and
    // estimates, the count of problems still active after each step (read
    // by the host one step late), the non-finite flag
    double* d_gs = nullptr;
    double* d_theta = nullptr;
    double* h_theta = nullptr;
    int* d_its = nullptr;
    int* h_its = nullptr;
    double* d_est = nullptr;
    double* h_est = nullptr;
    int* d_cnt = nullptr;           // max(restart, kPcgMaxIt) + 1
    int* h_cnt = nullptr;
    int* d_bad = nullptr;
    int* h_bad = nullptr;
    std::vector<cudaEvent_t> cnt_ev;   // max(restart, kPcgMaxIt) + 1
    cudaStream_t aux[tfde::kStreams] = {};
    cudaEvent_t ev[tfde::kStreams] = {};
    cudaEvent_t fork_ev = nullptr;
    bool chain_ok = false;
    std::vector<double*> chain_u;
    std::vector<int*> own_err;      // each problem's own error flag while it reports to d_err
    tfde::OzBatch* oz = nullptr;    // the exact residuals as grouped launches
    // the chained steps' right-hand sides as grouped launches
    tfde::ChainDesc* d_chain = nullptr;
    tfde::ChainDesc* h_chain = nullptr;
    double* d_mr = nullptr;         // count * 8: the five correction sums per problem
    double* d_g = nullptr;          // count * 4: the guess coefficients per problem
    long long grouped_prepares = 0; // steps whose right-hand sides ran grouped
};

namespace tfde {
namespace {

#define B_TRY(expr)                                                                        \
    do {                                                                                   \
        cudaError_t e__ = (expr);                                                          \
        if (e__ != cudaSuccess)                                                            \
            return set_error(TFDE_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e__)); \
    } while (0)

void fork(tfde_batch* B, cudaStream_t s) {
    cudaEventRecord(B->fork_ev, s);
    for (auto& a : B->aux) cudaStreamWaitEvent(a, B->fork_ev, 0);
}
void join(tfde_batch* B, cudaStream_t s) {
    for (int k = 0; k < kStreams; ++k) {
        cudaEventRecord(B->ev[k], B->aux[k]);
        cudaStreamWaitEvent(s, B->ev[k], 0);
    }
}

int free_batch(tfde_batch* B) {
    if (!B) return TFDE_OK;
    cudaDeviceSynchronize();
    for (size_t i = 0; i < B->P.size(); ++i) {
        if (i < B->own_err.size()) tfde::mixed(B->P[i])->err = B->own_err[i];
        destroy_problem(B->P[i]);
    }
    tfde::oz_batch_destroy(B->oz);
    cudaFree(B->d_chain);
    if (B->h_chain) cudaFreeHost(B->h_chain);
    cudaFree(B->d_mr);
    cudaFree(B->d_g);
    cudaFree(B->d_sopzw);
    cudaFree(B->d_j);
    if (B->cyc_exec) cudaGraphExecDestroy(B->cyc_exec);
    if (B->cyc_graph) cudaGraphDestroy(B->cyc_graph);
    if (B->pcg_exec) cudaGraphExecDestroy(B->pcg_exec);
    if (B->pcg_graph) cudaGraphDestroy(B->pcg_graph);
    cudaFree(B->d_sfw);
    cudaFree(B->d_sop);
    cudaFree(B->d_sopz);
    cudaFree(B->d_sbw);
    cudaFree(B->d_sfp);
    cudaFree(B->d_sopq);
    cudaFree(B->d_mv);
    cudaFree(B->d_pc);
    cudaFree(B->d_pcl);
    cudaFree(B->d_gstart);
    cudaFree(B->d_vt);
    if (B->h_vt) cudaFreeHost(B->h_vt);
    cudaFree(B->d_bi);
    cudaFree(B->d_bo);
    cudaFree(B->d_bstart);
    cudaFree(B->d_part);
    cudaFree(B->d_h);
    cudaFree(B->d_s);
    if (B->h_s) cudaFreeHost(B->h_s);
    cudaFree(B->d_act);
    if (B->h_act) cudaFreeHost(B->h_act);
    cudaFree(B->d_err);
    if (B->h_err) cudaFreeHost(B->h_err);
    cudaFree(B->d_gs);
    cudaFree(B->d_theta);
    if (B->h_theta) cudaFreeHost(B->h_theta);
    cudaFree(B->d_its);
    if (B->h_its) cudaFreeHost(B->h_its);
    cudaFree(B->d_est);
    if (B->h_est) cudaFreeHost(B->h_est);
    cudaFree(B->d_cnt);
    if (B->h_cnt) cudaFreeHost(B->h_cnt);
    cudaFree(B->d_bad);
    if (B->h_bad) cudaFreeHost(B->h_bad);
    for (cudaEvent_t e : B->cnt_ev)
        if (e) cudaEventDestroy(e);
    for (int k = 0; k < kStreams; ++k) {
        if (B->aux[k]) cudaStreamDestroy(B->aux[k]);
        if (B->ev[k]) cudaEventDestroy(B->ev[k]);
    }
    if (B->fork_ev) cudaEventDestroy(B->fork_ev);
    delete B;
    return TFDE_OK;
}

int grouped(tfde_batch* B, const tc::Params* d, int axis, int out_mode, double bytes, double flops, cudaStream_t s) {
    return tc::launch_grouped(d, B->d_gstart + (size_t)axis * (B->count + 1), B->count, B->gtotal[axis],
                              axis == 0 ? 1 : 0, out_mode, B->d_act, B->d_err, s, bytes, flops);
}

// v_j (split planes PL_P of every active problem) -> PL_R = A v_j
int grouped_matvec(tfde_batch* B, cudaStream_t s) {
    for (int k = 0; k < 5; ++k) {
        int st = grouped(B, B->d_mv + (size_t)k * B->count, B->mv_axis[k], B->mv_out[k], B->mv_bytes[k],
                         B->mv_flops[k], s);
        if (st) return st;
    }
    return TFDE_OK;
}

// PL_R -> V_j = P^{-1} (PL_R) in FP32
int grouped_precond(tfde_batch* B, int j, cudaStream_t s) {
    for (int k = 0; k < 5; ++k) {
        int st = grouped(B, B->d_pc + (size_t)k * B->count, B->pc_axis[k], B->pc_out[k], B->pc_bytes[k],
                         B->pc_flops[k], s);
        if (st) return st;
    }
    return grouped(B, B->d_pcl + (size_t)j * B->count, B->pc_axis[5], B->pc_out[5], B->pc_bytes[5],
                   B->pc_flops[5], s);
}

// eigenbasis: the scaled residual planes PL_R -> V_0 = Lambda^{-1} S_N r
int grouped_spec_start(tfde_batch* B, cudaStream_t s) {
    for (int a = 0; a < 3; ++a) {
        int st = grouped(B, B->d_sfw + (size_t)a * B->count, a, a < 2 ? tc::OUT_HILO : tc::OUT_SUM, B->sfw_bytes[a],
                         B->sfw_flops[a], s);
        if (st) return st;
    }
    return TFDE_OK;
}

// eigenbasis: v_j (split planes PL_P) -> V_{j+1} = Lambda^{-1} S_N A S_N v_j
int grouped_spec_step(tfde_batch* B, int j, cudaStream_t s) {
    for (int a = 0; a < 2; ++a) {
        int st = grouped(B, B->d_sop + (size_t)a * B->count, a, tc::OUT_SUM, B->sop_bytes[a], B->sop_flops[a], s);
        if (st) return st;
    }
    return grouped(B, B->d_sopz + (size_t)j * B->count, 2, tc::OUT_SUM, B->sop_bytes[2], B->sop_flops[2], s);
}

// eigenbasis: x32 = S_N x32 for the problems with act set (planes PL_T1 -> PL_T2 -> PL_R -> x32)
int grouped_spec_back(tfde_batch* B, cudaStream_t s) {
    stats_count_launch();
    bk_split_x32<<<B->NB, kBT, 0, s>>>(B->d_vt, B->d_bi, B->d_bo, B->d_act);
    for (int a = 0; a < 3; ++a) {
        int st = grouped(B, B->d_sbw + (size_t)a * B->count, a, a < 2 ? tc::OUT_HILO : tc::OUT_F32, B->sbw_bytes[a],
                         B->sbw_flops[a], s);
        if (st) return st;
    }
    return TFDE_OK;
}

void vec_launch_count() { stats_count_launch(); }

// The eigenbasis Arnoldi step of every problem as the body of a while node:
// the three grouped passes (the z pass into W), CGS2 against V_0 .. V_j with
// the coefficients on the device, ||W||, the Givens update and stop test per
// problem, V_{j+1} = W / ||W|| with its split planes, and the loop condition
// (a problem still in the cycle and j + 1 < restart).  Built once per batch
// (rebuilt when the autotuner's table changes); a failure leaves the host
// loop in use.
int build_cycle_graph(tfde_batch* B, cudaStream_t s) {
    if (B->cyc_exec && B->cyc_tune_gen != tc::tune_generation()) {
        cudaGraphExecDestroy(B->cyc_exec);
        cudaGraphDestroy(B->cyc_graph);
        B->cyc_exec = nullptr;
        B->cyc_graph = nullptr;
    }
    if (B->cyc_exec || B->cyc_failed) return TFDE_OK;
    if (int st = tc::set_attrs()) return st;
    const int C = B->count, R = B->restart;
    const int gb = (C + 63) / 64;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
    cudaGraphConditionalHandle h{};
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    if (ok) ok = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
    }
    if (ok) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        // captured on a stream of its own (the caller's may be the legacy default stream)
        const cudaStream_t s = capture_stream();
        ok = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
             cudaSuccess;
        if (ok) {
            stats_set_capturing(true);
            int st = TFDE_OK;
            for (int a = 0; a < 2 && !st; ++a)
                st = grouped(B, B->d_sop + (size_t)a * C, a, tc::OUT_SUM, B->sop_bytes[a], B->sop_flops[a], s);
            if (!st) st = grouped(B, B->d_sopzw, 2, tc::OUT_SUM, B->sop_bytes[2], B->sop_flops[2], s);
            if (!st) {   // CGS2: <V, W>; W -= V h and <V, W> again (one pass); W -= V h2 and ||W||^2 (one pass)
                for (int m0 = 0; m0 < R; m0 += 8)
                    bkg_dots<<<B->NB, kBT, 0, s>>>(B->d_vt, B->d_bi, B->d_bo, B->d_act, m0, B->d_j, R, 0, B->d_part);
                bkg_reduce<<<dim3((unsigned)C, (unsigned)R), 32, 0, s>>>(B->d_part, B->NB, B->d_bstart, B->d_act,
                                                                         B->d_j, R, 0, B->d_h, kHS, 0);
                bkg_axpy_dots<<<B->NB, kBT, 0, s>>>(B->d_vt, B->d_bi, B->d_bo, B->d_act, B->d_j, B->d_h, 0, B->d_part);
                bkg_reduce<<<dim3((unsigned)C, (unsigned)R), 32, 0, s>>>(B->d_part, B->NB, B->d_bstart, B->d_act,
                                                                         B->d_j, R, 0, B->d_h, kHS, 64);
                bkg_axpy_ww<<<B->NB, kBT, 0, s>>>(B->d_vt, B->d_bi, B->d_bo, B->d_act, B->d_j, B->d_h, 64, R,
                                                  B->d_part);
                bkg_reduce<<<dim3((unsigned)C, 1u), 32, 0, s>>>(B->d_part, B->NB, B->d_bstart, B->d_act, B->d_j, R,
                                                               1, B->d_s, kSS, S_WW);
                bkg_givens<<<gb, 64, 0, s>>>(C, R, B->d_j, B->d_gs, B->d_h, B->d_s, B->d_theta, B->d_act, B->d_its,
                                             B->d_est, B->d_cnt, B->d_bad);
                bkg_scale_split<<<B->NB, kBT, 0, s>>>(B->d_vt, B->d_bi, B->d_bo, B->d_act, B->d_j, B->d_s);
                bkg_next<<<1, 1, 0, s>>>(B->d_j, B->d_cnt, R, h);
            }
            stats_set_capturing(false);
            cudaGraph_t out = nullptr;
            const cudaError_t e = cudaStreamEndCapture(s, &out);
            ok = st == TFDE_OK && e == cudaSuccess;
        }
    }
    if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        B->cyc_failed = true;
        tfde::set_error(TFDE_OK, "");
        return TFDE_OK;
    }
    B->cyc_graph = g;
    B->cyc_exec = ex;
    B->cyc_tune_gen = tc::tune_generation();
    return TFDE_OK;
}

// launches of one captured step: 3 grouped + ceil(R / 8) + 1 (first projections)
// + 4 (fused second pass and norm with their reductions) + 3 (Givens, scale, loop)
unsigned cycle_step_launches(int R) { return 3u + (unsigned)((R + 7) / 8 + 1) + 4u + 3u; }

// The batched PCG iteration of every symmetric problem as the body of a while
// node: the operator's three grouped passes (<p, q> per problem), the update,
// the stop test at j = *d_j, the direction, and the loop condition (a problem
// still iterating and j + 1 < kPcgMaxIt).  Built once per batch (rebuilt
// when the autotuner's table changes); a failure leaves the host loop in use.
int build_pcg_graph(tfde_batch* B) {
    if (B->pcg_exec && B->pcg_tune_gen != tc::tune_generation()) {
        cudaGraphExecDestroy(B->pcg_exec);
        cudaGraphDestroy(B->pcg_graph);
        B->pcg_exec = nullptr;
        B->pcg_graph = nullptr;
    }
    if (B->pcg_exec || B->pcg_failed) return TFDE_OK;
    if (int st = tc::set_attrs()) return st;
    const int C = B->count;
    const int gb = (C + 63) / 64;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
    cudaGraphConditionalHandle h{};
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    if (ok) ok = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
    }
    if (ok) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        // captured on a stream of its own (the caller's may be the legacy default stream)
        const cudaStream_t s = capture_stream();
        ok = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
             cudaSuccess;
        if (ok) {
            stats_set_capturing(true);
            int st = TFDE_OK;
            for (int a = 0; a < 2 && !st; ++a)
                st = grouped(B, B->d_sop + (size_t)a * C, a, tc::OUT_SUM, B->sop_bytes[a], B->sop_flops[a], s);
            if (!st) st = grouped(B, B->d_sopq, 2, tc::OUT_SUM, B->sopq_bytes, B->sopq_flops, s);
            if (!st) {
                bkp_update<<<B->NB, kBT, 0, s>>>(B->d_vt, B->d_bi, B->d_bo, B->d_act, B->d_s);
                bkpg_stop<<<gb, 64, 0, s>>>(C, B->d_j, kPcgMaxIt, B->d_s, B->d_theta, B->d_act, B->d_its, B->d_est,
                                            B->d_cnt, B->d_bad);
                bkp_direction<<<B->NB, kBT, 0, s>>>(B->d_vt, B->d_bi, B->d_bo, B->d_act, B->d_s);
                bkg_next<<<1, 1, 0, s>>>(B->d_j, B->d_cnt, kPcgMaxIt, h);
            }
            stats_set_capturing(false);
            cudaGraph_t out = nullptr;
            const cudaError_t e = cudaStreamEndCapture(s, &out);
            ok = st == TFDE_OK && e == cudaSuccess;
        }
    }
    if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        B->pcg_failed = true;
        tfde::set_error(TFDE_OK, "");
        return TFDE_OK;
    }
    B->pcg_graph = g;
    B->pcg_exec = ex;
    B->pcg_tune_gen = tc::tune_generation();
    return TFDE_OK;
}

// dots <V_{p0+j}, V_jw>, j < m, of every active problem into out (stride, offset)
void bdots(tfde_batch* B, int p0, int m, int jw, double* out, int ostride, int ooff, cudaStream_t s) {
    for (int m0 = p0; m0 < p0 + m; m0 += 8) {
        const int mc = (p0 + m - m0) < 8 ? (p0 + m - m0) : 8;
        vec_launch_count();
        bk_multidot<<<B->NB, kBT, 0, s>>>(B->d_vt, B->d_bi, B->d_bo, B->d_act, m0, mc, jw, B->d_part);
    }
    vec_launch_count();
    bk_reduce<<<dim3((unsigned)B->count, (unsigned)m), 32, 0, s>>>(B->d_part, B->NB, B->d_bstart, B->d_act, p0, out,
                                                                  ostride, ooff);
}

int upload_act_scalars(tfde_batch* B, cudaStream_t s) {
    B_TRY(cudaMemcpyAsync(B->d_act, B->h_act, B->count * sizeof(int), cudaMemcpyHostToDevice, s));
    B_TRY(cudaMemcpyAsync(B->d_s, B->h_s, (size_t)B->count * kSS * sizeof(double), cudaMemcpyHostToDevice, s));
    return TFDE_OK;
}

int read_back(tfde_batch* B, cudaStream_t s) {
    B_TRY(cudaMemcpyAsync(B->h_s, B->d_s, (size_t)B->count * kSS * sizeof(double), cudaMemcpyDeviceToHost, s));
    B_TRY(cudaMemcpyAsync(B->h_err, B->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    B_TRY(cudaStreamSynchronize(s));
    if (*B->h_err) return set_error(TFDE_ETIMEOUT, "tensor-core kernel wait ran out (device error flag set)");
    return TFDE_OK;
}

// One lock-step left-preconditioned GMRES cycle (Sec. 3.2) for every problem
// with outer[i] set: A d_i = r32_i (x32_i = 0 on entry, d_i on exit), stopping
// problem i once its preconditioned residual estimate falls below
// theta[i] * beta_i.  est[i] = final estimate / beta_i; its[i] = steps.
// The Hessenberg columns, their Givens rotations, the stop test and the
// final triangular solve stay on the device; the host only learns how many
// problems are still in the cycle, one step late (it waits for the count of
// step j - 2 while the GPU runs step j - 1), so the GPU never idles on a host
// read, at the price of at most two fully masked steps at the end.  One
// read per cycle brings back every problem's steps and estimate.
int batch_cycle(tfde_batch* B, const std::vector<int>& outer, const std::vector<double>& theta,
                std::vector<double>& est, std::vector<int>& its, cudaStream_t s) {
    const int C = B->count, R = B->restart;
    const int gb = (C + 63) / 64;
    int st;
    for (int i = 0; i < C; ++i) {
        B->h_act[i] = outer[i];
        B->h_theta[i] = theta[i];
    }
    B_TRY(cudaMemcpyAsync(B->d_act, B->h_act, C * sizeof(int), cudaMemcpyHostToDevice, s));
    B_TRY(cudaMemcpyAsync(B->d_theta, B->h_theta, C * sizeof(double), cudaMemcpyHostToDevice, s));
    B_TRY(cudaMemsetAsync(B->d_cnt, 0, (R + 1) * sizeof(int), s));
    B_TRY(cudaMemsetAsync(B->d_bad, 0, sizeof(int), s));
    if ((st = B->spectral ? grouped_spec_start(B, s) : grouped_precond(B, 0, s))) return st;
    bdots(B, 0, 1, 0, B->d_s, kSS, S_WW, s);
    vec_launch_count();
    bk_cycle_start<<<gb, 64, 0, s>>>(C, R, B->d_gs, B->d_s, B->d_act, B->d_its, B->d_est, B->d_cnt, B->d_bad);
    B_TRY(cudaMemcpyAsync(B->h_cnt, B->d_cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
    B_TRY(cudaEventRecord(B->cnt_ev[0], s));
    vec_launch_count();
    bk_scale_split<<<B->NB, kBT, 0, s>>>(B->d_vt, B->d_bi, B->d_bo, B->d_act, 0, B->d_s);
    const bool graph = B->spectral && B->device_loop && !stats_timing();
    if (graph && (st = build_cycle_graph(B, s))) return st;
    if (graph && B->cyc_exec) {
        // every Arnoldi step on the device: one graph launch for the cycle
        B_TRY(cudaMemsetAsync(B->d_j, 0, sizeof(int), s));
        B_TRY(cudaGraphLaunch(B->cyc_exec, s));
        ++B->graph_cycles;
    }
    for (int j = 0; j < R && !(graph && B->cyc_exec); ++j) {
        // stop issuing once no problem is left: the count after step j - 1
        // if it is already in, else the one after step j - 2
        if (cudaEventQuery(B->cnt_ev[j]) == cudaSuccess) {
            if (B->h_cnt[j] == 0) break;
        } else if (j >= 1) {
            B_TRY(cudaEventSynchronize(B->cnt_ev[j - 1]));
            if (B->h_cnt[j - 1] == 0) break;
        }
        if (B->spectral) {
            if ((st = grouped_spec_step(B, j + 1, s))) return st;
        } else {
            if ((st = grouped_matvec(B, s))) return st;
            if ((st = grouped_precond(B, j + 1, s))) return st;
        }
        // CGS2, coefficients on the device
        bdots(B, 0, j + 1, j + 1, B->d_h, kHS, 0, s);
        vec_launch_count();
        bk_multiaxpy<<<B->NB, kBT, 0, s>>>(B->d_vt, B->d_bi, B->d_bo, B->d_act, j + 1, j + 1, B->d_h, 0);
        bdots(B, 0, j + 1, j + 1, B->d_h, kHS, 64, s);
        vec_launch_count();
        bk_multiaxpy<<<B->NB, kBT, 0, s>>>(B->d_vt, B->d_bi, B->d_bo, B->d_act, j + 1, j + 1, B->d_h, 64);
        bdots(B, j + 1, 1, j + 1, B->d_s, kSS, S_WW, s);
        vec_launch_count();
        bk_givens<<<gb, 64, 0, s>>>(C, R, j, B->d_gs, B->d_h, B->d_s, B->d_theta, B->d_act, B->d_its, B->d_est,
                                    B->d_cnt + j + 1, B->d_bad);
        B_TRY(cudaMemcpyAsync(B->h_cnt + j + 1, B->d_cnt + j + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        B_TRY(cudaEventRecord(B->cnt_ev[j + 1], s));
        vec_launch_count();
        bk_scale_split<<<B->NB, kBT, 0, s>>>(B->d_vt, B->d_bi, B->d_bo, B->d_act, j + 1, B->d_s);
    }
    // d_i = V_i y_i
    vec_launch_count();
    bk_cycle_solve<<<gb, 64, 0, s>>>(C, R, B->d_gs, B->d_its, B->d_h);
    B_TRY(cudaMemcpyAsync(B->h_its, B->d_its, C * sizeof(int), cudaMemcpyDeviceToHost, s));
    B_TRY(cudaMemcpyAsync(B->h_est, B->d_est, C * sizeof(double), cudaMemcpyDeviceToHost, s));
    B_TRY(cudaMemcpyAsync(B->h_bad, B->d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    B_TRY(cudaMemcpyAsync(B->h_err, B->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    B_TRY(cudaStreamSynchronize(s));
    if (*B->h_err) return set_error(TFDE_ETIMEOUT, "tensor-core kernel wait ran out (device error flag set)");
    if (*B->h_bad) return set_error(TFDE_ENAN, "non-finite value in a batched GMRES cycle");
    int kmax = 0;
    for (int i = 0; i < C; ++i) kmax = std::max(kmax, outer[i] ? B->h_its[i] : 0);
    if (graph && B->cyc_exec) stats_count_launch((unsigned)(kmax > 0 ? kmax : 1) * cycle_step_launches(R));
    kmax = 0;
    for (int i = 0; i < C; ++i) {
        its[i] = outer[i] ? B->h_its[i] : 0;
        est[i] = outer[i] ? B->h_est[i] : 1.0;
        kmax = std::max(kmax, its[i]);
    }
    if (kmax > 0) {
        for (int i = 0; i < C; ++i) B->h_act[i] = outer[i] && its[i] > 0;
        B_TRY(cudaMemcpyAsync(B->d_act, B->h_act, C * sizeof(int), cudaMemcpyHostToDevice, s));
        vec_launch_count();
        bk_multiaxpy<<<B->NB, kBT, 0, s>>>(B->d_vt, B->d_bi, B->d_bo, B->d_act, kmax, -1, B->d_h, 128);
        if (B->spectral && (st = grouped_spec_back(B, s))) return st;   // back to the grid basis
    }
    return TFDE_OK;
}

// One lock-step inner PCG (Sec. 3.1) for every problem with outer[i] set
// (symmetric problems), in the sine-transform eigenbasis: the scaled residual
// r32 (planes PL_R) goes to r~ = S_N r, PCG with the diagonal Lambda runs on
// S_N A S_N x~ = r~ until ||r~_k|| <= theta[i] ||r~_0|| (r~_k is the true inner
// residual in that basis), and x32 = S_N x~ on return.  Per iteration: the
// operator's three grouped passes over all active problems' tiles (the z pass
// adds <p, q> per problem), then one update, one stop test and one direction
// launch over all of them; the host learns how many problems are left one
// iteration late, as in batch_cycle.  est[i] = ||r~_k|| / ||r~_0||, its[i] =
// iterations.
int batch_pcg(tfde_batch* B, const std::vector<int>& outer, const std::vector<double>& theta,
              std::vector<double>& est, std::vector<int>& its, cudaStream_t s) {
    const int C = B->count;
    const int gb = (C + 63) / 64;
    int st;
    for (int i = 0; i < C; ++i) {
        B->h_act[i] = outer[i];
        B->h_theta[i] = theta[i];
    }
    B_TRY(cudaMemcpyAsync(B->d_act, B->h_act, C * sizeof(int), cudaMemcpyHostToDevice, s));
    B_TRY(cudaMemcpyAsync(B->d_theta, B->h_theta, C * sizeof(double), cudaMemcpyHostToDevice, s));
    B_TRY(cudaMemsetAsync(B->d_cnt, 0, (kPcgMaxIt + 1) * sizeof(int), s));
    B_TRY(cudaMemsetAsync(B->d_bad, 0, sizeof(int), s));
    for (int a = 0; a < 3; ++a)   // r~ = S_N r into r32
        if ((st = grouped(B, B->d_sfp + (size_t)a * C, a, a < 2 ? tc::OUT_HILO : tc::OUT_F32, B->sfp_bytes[a],
                          B->sfp_flops[a], s)))
            return st;
    vec_launch_count();
    bkp_reset<<<gb, 64, 0, s>>>(C, B->d_s, B->d_act);
    vec_launch_count();
    bkp_first<<<B->NB, kBT, 0, s>>>(B->d_vt, B->d_bi, B->d_bo, B->d_act, B->d_s);
    vec_launch_count();
    bkp_start<<<gb, 64, 0, s>>>(C, B->d_s, B->d_act, B->d_its, B->d_est, B->d_cnt, B->d_bad);
    const bool graph = B->device_loop && !stats_timing();
    if (graph && (st = build_pcg_graph(B))) return st;
    if (graph && B->pcg_exec) {
        // every iteration on the device: one graph launch for the solve
        B_TRY(cudaMemsetAsync(B->d_j, 0, sizeof(int), s));
        B_TRY(cudaGraphLaunch(B->pcg_exec, s));
        ++B->pcg_graph_launches;
    } else {
        B_TRY(cudaMemcpyAsync(B->h_cnt, B->d_cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
        B_TRY(cudaEventRecord(B->cnt_ev[0], s));
    }
    for (int j = 0; j < kPcgMaxIt && !(graph && B->pcg_exec); ++j) {
        // stop issuing once no problem is left: the count after iteration j - 1
        // if it is already in, else the one after iteration j - 2
        if (cudaEventQuery(B->cnt_ev[j]) == cudaSuccess) {
            if (B->h_cnt[j] == 0) break;
        } else if (j >= 1) {
            B_TRY(cudaEventSynchronize(B->cnt_ev[j - 1]));
            if (B->h_cnt[j - 1] == 0) break;
        }
        for (int a = 0; a < 2; ++a)
            if ((st = grouped(B, B->d_sop + (size_t)a * C, a, tc::OUT_SUM, B->sop_bytes[a], B->sop_flops[a], s)))
                return st;
        if ((st = grouped(B, B->d_sopq, 2, tc::OUT_SUM, B->sopq_bytes, B->sopq_flops, s))) return st;
        vec_launch_count();
        bkp_update<<<B->NB, kBT, 0, s>>>(B->d_vt, B->d_bi, B->d_bo, B->d_act, B->d_s);
        vec_launch_count();
        bkp_stop<<<gb, 64, 0, s>>>(C, j, kPcgMaxIt, B->d_s, B->d_theta, B->d_act, B->d_its, B->d_est,
                                   B->d_cnt + j + 1, B->d_bad);
        B_TRY(cudaMemcpyAsync(B->h_cnt + j + 1, B->d_cnt + j + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        B_TRY(cudaEventRecord(B->cnt_ev[j + 1], s));
        vec_launch_count();
        bkp_direction<<<B->NB, kBT, 0, s>>>(B->d_vt, B->d_bi, B->d_bo, B->d_act, B->d_s);
    }
    B_TRY(cudaMemcpyAsync(B->h_its, B->d_its, C * sizeof(int), cudaMemcpyDeviceToHost, s));
    B_TRY(cudaMemcpyAsync(B->h_est, B->d_est, C * sizeof(double), cudaMemcpyDeviceToHost, s));
    B_TRY(cudaMemcpyAsync(B->h_bad, B->d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    B_TRY(cudaMemcpyAsync(B->h_err, B->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    B_TRY(cudaStreamSynchronize(s));
    if (*B->h_err) return set_error(TFDE_ETIMEOUT, "tensor-core kernel wait ran out (device error flag set)");
    if (*B->h_bad) return set_error(TFDE_ENAN, "non-finite value in a batched PCG solve");
    int kmax = 0;
    for (int i = 0; i < C; ++i) {
        its[i] = outer[i] ? B->h_its[i] : 0;
        est[i] = outer[i] ? B->h_est[i] : 1.0;
        kmax = std::max(kmax, its[i]);
        if (outer[i]) ++B->pcg_solves;
    }
    if (graph && B->pcg_exec) stats_count_launch(7u * (unsigned)(kmax > 0 ? kmax : 1));   // per body: 3 grouped + 4
    if (kmax > 0) {   // x32 = S_N x~ (a problem without iterations keeps x32 = 0)
        for (int i = 0; i < C; ++i) B->h_act[i] = outer[i] && its[i] > 0;
        B_TRY(cudaMemcpyAsync(B->d_act, B->h_act, C * sizeof(int), cudaMemcpyHostToDevice, s));
        if ((st = grouped_spec_back(B, s))) return st;
    }
    return TFDE_OK;
}

}  // namespace

int batch_create(const tfde_params* params, int count, int restart, cudaStream_t s, tfde_batch** out) {
    *out = nullptr;
    if (!params || count < 1 || count > 1024) return set_error(TFDE_EINVAL, "batch count must lie in [1, 1024]");
    if (restart < 1 || restart > 63) return set_error(TFDE_EINVAL, "batch restart must lie in [1, 63]");
    tfde_batch* B = new tfde_batch();
    B->count = count;
    B->restart = restart;
    int st;
    // problems, sorted by decreasing size (largest tiles first in the work lists)
    std::vector<int> idx(count);
    for (int i = 0; i < count; ++i) idx[i] = i;
    auto sz = [&](int i) { return (long long)params[i].n[0] * params[i].n[1] * params[i].n[2]; };
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return sz(a) > sz(b); });
    B->caller = idx;
    if (cudaMalloc((void**)&B->d_err, sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&B->h_err, sizeof(int)) != cudaSuccess || cudaMemset(B->d_err, 0, sizeof(int)) != cudaSuccess) {
        free_batch(B);
        return set_error(TFDE_ENOMEM, "allocation of the batch error flag failed");
    }
    for (int k = 0; k < count; ++k) {
        tfde_problem* P = nullptr;
        if ((st = assemble_problem(&params[idx[k]], TFDE_MIXED, s, &P))) {
            free_batch(B);
            return st;
        }
        B->P.push_back(P);
        if (!P->mixed) {   // the grouped launches are the tensor-core contraction's
            free_batch(B);
            return set_error(TFDE_EUNSUPPORTED, "tfde_batch_create needs every n_a to be a multiple of 8 and <= 448");
        }
        // every kernel of the batch, per-problem ones included, reports to one flag
        B->own_err.push_back(mixed(P)->err);
        mixed(P)->err = B->d_err;
        if ((st = mixed_prepare_gmres(P, restart))) {
            free_batch(B);
            return st;
        }
    }
    auto fail = [&](int code, const char* what) {
        free_batch(B);
        return set_error(code, what);
    };
    // grouped descriptors
    const size_t C = count, PS = sizeof(tc::Params);
    std::vector<tc::Params> mv(5 * C), pc(5 * C), pcl((size_t)(restart + 1) * C);
    std::vector<tc::Params> sfw(3 * C), sop(2 * C), sopz((size_t)(restart + 1) * C), sbw(3 * C), sopzw(C);
    std::vector<long long> gstart(3 * (C + 1), 0);
    for (size_t i = 0; i < C; ++i) {
        tfde_problem* P = B->P[i];
        MixedState* M = mixed(P);
        tc::Params tmp[6];
        int axes[6];
        double by[6], fl[6];
        fast_pass_descriptors(P, 0, nullptr, tmp, axes, by, fl);
        for (int k = 0; k < 5; ++k) {
            mv[k * C + i] = tmp[k];
            B->mv_axis[k] = axes[k];
            B->mv_out[k] = tmp[k].out_mode;
            B->mv_bytes[k] += by[k];
            B->mv_flops[k] += fl[k];
        }
        for (int j = 0; j <= restart; ++j) {
            fast_pass_descriptors(P, 1, M->V32 + (size_t)j * P->N, tmp, axes, by, fl);
            if (j == 0)
                for (int k = 0; k < 6; ++k) {
                    if (k < 5) pc[k * C + i] = tmp[k];
                    B->pc_axis[k] = axes[k];
                    B->pc_out[k] = tmp[k].out_mode;
                    B->pc_bytes[k] += by[k];
                    B->pc_flops[k] += fl[k];
                }
            pcl[(size_t)j * C + i] = tmp[5];
        }
        spec_pass_descriptors(P, 2, M->V32, tmp, axes, by, fl);
        for (int a = 0; a < 3; ++a) {
            sfw[a * C + i] = tmp[a];
            B->sfw_bytes[a] += by[a];
            B->sfw_flops[a] += fl[a];
        }
        for (int j = 0; j <= restart; ++j) {
            spec_pass_descriptors(P, 3, M->V32 + (size_t)j * P->N, tmp, axes, by, fl);
            if (j == 0)
                for (int a = 0; a < 3; ++a) {
                    if (a < 2) sop[a * C + i] = tmp[a];
                    B->sop_bytes[a] += by[a];
                    B->sop_flops[a] += fl[a];
                }
            sopz[(size_t)j * C + i] = tmp[2];
        }
        spec_pass_descriptors(P, 3, M->f[F_Q], tmp, axes, by, fl);
        sopzw[i] = tmp[2];
        spec_pass_descriptors(P, 4, M->f[F_X], tmp, axes, by, fl);
        for (int a = 0; a < 3; ++a) {
            sbw[a * C + i] = tmp[a];
            B->sbw_bytes[a] += by[a];
            B->sbw_flops[a] += fl[a];
        }
        for (int a = 0; a < 3; ++a) {
            tc::Params g;
            tc::set_geometry(g, P->n, a);
            gstart[a * (C + 1) + i + 1] = gstart[a * (C + 1) + i] + g.ntiles * g.mhalves;
        }
    }
    for (int a = 0; a < 3; ++a) B->gtotal[a] = gstart[a * (C + 1) + C];
    if (cudaMalloc((void**)&B->d_mv, mv.size() * PS) != cudaSuccess ||
        cudaMalloc((void**)&B->d_pc, pc.size() * PS) != cudaSuccess ||
        cudaMalloc((void**)&B->d_pcl, pcl.size() * PS) != cudaSuccess ||
        cudaMalloc((void**)&B->d_gstart, gstart.size() * sizeof(long long)) != cudaSuccess ||
        cudaMalloc((void**)&B->d_sfw, sfw.size() * PS) != cudaSuccess ||
        cudaMalloc((void**)&B->d_sop, sop.size() * PS) != cudaSuccess ||
        cudaMalloc((void**)&B->d_sopz, sopz.size() * PS) != cudaSuccess ||
        cudaMalloc((void**)&B->d_sbw, sbw.size() * PS) != cudaSuccess ||
        cudaMalloc((void**)&B->d_sopzw, sopzw.size() * PS) != cudaSuccess ||
        cudaMalloc((void**)&B->d_j, sizeof(int)) != cudaSuccess)
        return fail(TFDE_ENOMEM, "cudaMalloc of the grouped descriptors failed");
    // block table
    std::vector<int> bstart(C + 1, 0), bi;
    std::vector<long long> bo;
    for (size_t i = 0; i < C; ++i) {
        const long long N = (long long)B->P[i]->N;
        const long long nb = (N + kCH - 1) / kCH;
        for (long long b = 0; b < nb; ++b) {
            bi.push_back((int)i);
            bo.push_back(b * kCH);
        }
        bstart[i + 1] = bstart[i] + (int)nb;
    }
    B->NB = bstart[C];
    const int ncnt = std::max(restart, kPcgMaxIt);
    if (cudaMalloc((void**)&B->d_vt, C * sizeof(BVec)) != cudaSuccess ||
        cudaMallocHost((void**)&B->h_vt, C * sizeof(BVec)) != cudaSuccess ||
        cudaMalloc((void**)&B->d_bi, bi.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&B->d_bo, bo.size() * sizeof(long long)) != cudaSuccess ||
        cudaMalloc((void**)&B->d_bstart, bstart.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&B->d_part, (size_t)std::max(restart + 2, 5) * B->NB * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&B->d_h, C * kHS * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&B->d_s, C * kSS * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void**)&B->h_s, C * kSS * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&B->d_act, C * sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&B->h_act, C * sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&B->d_gs, C * gs_stride(restart) * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&B->d_theta, C * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void**)&B->h_theta, C * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&B->d_its, C * sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&B->h_its, C * sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&B->d_est, C * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void**)&B->h_est, C * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&B->d_cnt, (size_t)(ncnt + 1) * sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&B->h_cnt, (size_t)(ncnt + 1) * sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&B->d_bad, sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&B->h_bad, sizeof(int)) != cudaSuccess)
        return fail(TFDE_ENOMEM, "allocation of the batch workspace failed");
    B->cnt_ev.assign(ncnt + 1, nullptr);
    for (auto& e : B->cnt_ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return fail(TFDE_ECUDA, "event creation failed");
    for (size_t i = 0; i < C; ++i) {
        tfde_problem* P = B->P[i];
        MixedState* M = mixed(P);
        BVec& v = B->h_vt[i];
        v.N = (long long)P->N;
        v.x32 = M->f[F_X];
        v.r32 = M->f[F_R];
        v.V = M->V32;
        v.ph = M->hi[PL_P];
        v.pl = M->lo[PL_P];
        v.rh = M->hi[PL_R];
        v.rl = M->lo[PL_R];
        v.th = M->hi[PL_T1];
        v.tl = M->lo[PL_T1];
        v.W = M->f[F_Q];
        v.r64 = P->w[tfde_problem::W_R];
        v.x64 = nullptr;
        v.p32 = M->V32;
        v.lam = M->lam;
        v.nc4 = (unsigned)((long long)P->n[0] * P->n[1] / 4);
        v.n3 = P->n[2];
        v.norms = P->red_out + kNormsSlot;
    }
    // the batched PCG's descriptors (the z pass adds <p, q> into the problem's S_PQ)
    std::vector<tc::Params> sfp(3 * C), sopq(C);
    for (size_t i = 0; i < C; ++i) {
        tfde_problem* P = B->P[i];
        MixedState* M = mixed(P);
        tc::Params tmp[6];
        int axes[6];
        double by[6], fl[6];
        spec_pass_descriptors(P, 5, M->f[F_R], tmp, axes, by, fl);
        for (int a = 0; a < 3; ++a) {
            sfp[a * C + i] = tmp[a];
            B->sfp_bytes[a] += by[a];
            B->sfp_flops[a] += fl[a];
        }
        spec_pass_descriptors(P, 3, M->f[F_Q], tmp, axes, by, fl, M->V32, B->d_s + i * kSS + S_PQ);
        sopq[i] = tmp[2];
        B->sopq_bytes += by[2];
        B->sopq_flops += fl[2];
    }
    if (cudaMalloc((void**)&B->d_sfp, sfp.size() * PS) != cudaSuccess ||
        cudaMalloc((void**)&B->d_sopq, sopq.size() * PS) != cudaSuccess)
        return fail(TFDE_ENOMEM, "cudaMalloc of the grouped descriptors failed");
    std::memset(B->h_s, 0, C * kSS * sizeof(double));
    if (cudaMemsetAsync(B->d_h, 0, C * kHS * sizeof(double), s) != cudaSuccess)
        return fail(TFDE_ECUDA, "batch workspace initialisation failed");
    if (cudaMemcpyAsync(B->d_mv, mv.data(), mv.size() * PS, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(B->d_pc, pc.data(), pc.size() * PS, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(B->d_pcl, pcl.data(), pcl.size() * PS, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(B->d_sfw, sfw.data(), sfw.size() * PS, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(B->d_sop, sop.data(), sop.size() * PS, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(B->d_sopz, sopz.data(), sopz.size() * PS, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(B->d_sbw, sbw.data(), sbw.size() * PS, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(B->d_sopzw, sopzw.data(), sopzw.size() * PS, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(B->d_sfp, sfp.data(), sfp.size() * PS, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(B->d_sopq, sopq.data(), sopq.size() * PS, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(B->d_gstart, gstart.data(), gstart.size() * sizeof(long long), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(B->d_bi, bi.data(), bi.size() * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(B->d_bo, bo.data(), bo.size() * sizeof(long long), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(B->d_bstart, bstart.data(), bstart.size() * sizeof(int), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemsetAsync(B->d_err, 0, sizeof(int), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return fail(TFDE_ECUDA, "upload of the batch tables failed");
    for (int k = 0; k < kStreams; ++k) {
        if (cudaStreamCreateWithFlags(&B->aux[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->ev[k], cudaEventDisableTiming) != cudaSuccess)
            return fail(TFDE_ECUDA, "stream pool creation failed");
    }
    if (cudaEventCreateWithFlags(&B->fork_ev, cudaEventDisableTiming) != cudaSuccess)
        return fail(TFDE_ECUDA, "event creation failed");
    if (cudaMalloc((void**)&B->d_chain, C * sizeof(ChainDesc)) != cudaSuccess ||
        cudaMallocHost((void**)&B->h_chain, C * sizeof(ChainDesc)) != cudaSuccess ||
        cudaMalloc((void**)&B->d_mr, C * 8 * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&B->d_g, C * 4 * sizeof(double)) != cudaSuccess)
        return fail(TFDE_ENOMEM, "allocation of the batch workspace failed");
    {
        std::vector<double*> norm2(C);
        for (size_t i = 0; i < C; ++i) norm2[i] = B->d_s + i * kSS + S_RR;
        if ((st = oz_batch_create(B->P.data(), count, norm2.data(), &B->oz))) {
            free_batch(B);
            return st;
        }
    }
    *out = B;
    return TFDE_OK;
}

int batch_destroy(tfde_batch* B) { return free_batch(B); }

// The autotuner on the batch's grouped launches (tfde_batch_tune): one
// operator and one preconditioner application over every problem recorded,
// then timed per launch class.
int batch_tune(tfde_batch* B, int reps, cudaStream_t s) {
    if (reps < 1 || reps > 1000) return set_error(TFDE_EINVAL, "reps must lie in [1, 1000]");
    for (int i = 0; i < B->count; ++i) B->h_act[i] = 1;
    B_TRY(cudaMemcpyAsync(B->d_act, B->h_act, B->count * sizeof(int), cudaMemcpyHostToDevice, s));
    tc::tune_record(true);
    int st = grouped_matvec(B, s);
    if (!st) st = grouped_precond(B, 0, s);
    if (!st) st = grouped_spec_start(B, s);
    if (!st) st = grouped_spec_step(B, 1, s);
    tc::tune_record(false);
    if (!st) st = tc::tune_recorded(reps, s);
    if (!st) st = read_back(B, s);
    return st;
}

}  // namespace tfde

extern "C" int tfde_batch_count(const tfde_batch* B) { return B ? B->count : 0; }

extern "C" long long tfde_batch_graph_cycles(const tfde_batch* B) { return B ? B->graph_cycles : 0; }

extern "C" int tfde_batch_set_spectral_inner(tfde_batch* B, int enable) {
    if (!B) return tfde::set_error(TFDE_EINVAL, "NULL batch");
    B->spectral = enable != 0;
    return TFDE_OK;
}

extern "C" int tfde_batch_set_symmetric_pcg(tfde_batch* B, int enable) {
    if (!B) return tfde::set_error(TFDE_EINVAL, "NULL batch");
    B->sym_pcg = enable != 0;
    return TFDE_OK;
}

extern "C" long long tfde_batch_pcg_solves(const tfde_batch* B) { return B ? B->pcg_solves : 0; }

extern "C" long long tfde_batch_pcg_graph_launches(const tfde_batch* B) { return B ? B->pcg_graph_launches : 0; }

extern "C" long long tfde_batch_grouped_prepares(const tfde_batch* B) { return B ? B->grouped_prepares : 0; }

extern "C" int tfde_batch_set_guess_order(tfde_batch* B, int order) {
    if (!B) return tfde::set_error(TFDE_EINVAL, "NULL batch");
    if (order < 0 || order > 3) return tfde::set_error(TFDE_EINVAL, "guess order must be 0, 1, 2 or 3");
    for (tfde_problem* P : B->P) {
        if (order > 0)
            if (int st = tfde::ensure_history(P)) return st;
        P->guess_order = order;
    }
    return TFDE_OK;
}

namespace tfde {

int batch_cn_advance(tfde_batch* B, double* const* u, const double* const* F, int restart_chain, double tol,
                     tfde_info* infos, cudaStream_t s) {
    const auto t0 = clk::now();
    const int C = B->count;
    int st;
    // per-problem pointers (sorted order)
    std::vector<double*> uu(C);
    std::vector<const double*> ff(C, nullptr);
    for (int i = 0; i < C; ++i) {
        uu[i] = u[B->caller[i]];
        if (F) ff[i] = F[B->caller[i]];
        B->h_vt[i].x64 = uu[i];
    }
    const bool chained = !restart_chain && B->chain_ok && B->chain_u == uu;
    B->chain_ok = false;
    B_TRY(cudaMemcpyAsync(B->d_vt, B->h_vt, C * sizeof(BVec), cudaMemcpyHostToDevice, s));
    // right-hand sides and initial residuals.  In the steady state of a chain
    // (every problem has A_N u^{m-1} from its last exact residual and two
    // history levels for the order-3 guess) they run grouped over all
    // problems; otherwise per problem (cn_prepare) on the stream pool
    bool grouped_prep = chained;
    for (int i = 0; i < C && grouped_prep; ++i) {
        const tfde_problem* P = B->P[i];
        grouped_prep = P->an_ready && P->guess_order >= 3 && P->hist >= 2;
    }
    if (grouped_prep) {
        for (int i = 0; i < C; ++i) {
            tfde_problem* P = B->P[i];
            B->h_chain[i] = ChainDesc{P->w[tfde_problem::W_T], ff[i], P->w[tfde_problem::W_B], P->w[tfde_problem::W_R],
                                      uu[i], P->H[0][0], P->H[0][1], P->H[1][0], P->H[1][1], P->p.dt};
            B->h_act[i] = 1;
        }
        B_TRY(cudaMemcpyAsync(B->d_chain, B->h_chain, C * sizeof(ChainDesc), cudaMemcpyHostToDevice, s));
        B_TRY(cudaMemcpyAsync(B->d_act, B->h_act, C * sizeof(int), cudaMemcpyHostToDevice, s));
        const int gb = (C + 63) / 64;
        vec_launch_count();
        bkc_mr_dots<<<B->NB, kBT, 0, s>>>(B->d_chain, B->d_vt, B->d_bi, B->d_bo, B->d_act, B->d_part);
        vec_launch_count();
        bk_reduce<<<dim3((unsigned)C, 5u), 32, 0, s>>>(B->d_part, B->NB, B->d_bstart, B->d_act, 0, B->d_mr, 8, 0);
        vec_launch_count();
        bkc_coef<<<gb, 64, 0, s>>>(C, B->d_mr, B->d_g, B->d_act);
        vec_launch_count();
        bkc_chain<<<B->NB, kBT, 0, s>>>(B->d_chain, B->d_vt, B->d_bi, B->d_bo, B->d_act, B->d_g, B->d_part);
        vec_launch_count();
        bk_reduce<<<dim3((unsigned)C, 2u), 32, 0, s>>>(B->d_part, B->NB, B->d_bstart, B->d_act, 0, B->d_s, kSS, S_BB);
        for (int i = 0; i < C; ++i) {   // as cn_prepare: the mass term is used up, the history moves on
            tfde_problem* P = B->P[i];
            P->an_ready = false;
            std::swap(P->H[0][0], P->H[1][0]);
            std::swap(P->H[0][1], P->H[1][1]);
            P->hist = 2;
        }
        ++B->grouped_prepares;
    } else {
        fork(B, s);
        for (int i = 0; i < C; ++i) {
            bool rg = false;
            if ((st = cn_prepare(B->P[i], uu[i], ff[i], nullptr, uu[i], B->aux[i % kStreams], chained, &rg, nullptr,
                                 nullptr))) {
                join(B, s);
                return st;
            }
        }
        join(B, s);
        // ||b||^2 and ||r_0||^2 as every cn_prepare formed them, into S_BB / S_RR
        vec_launch_count();
        bk_gather_norms<<<(C + 63) / 64, 64, 0, s>>>(C, B->d_vt, B->d_s);
    }
    if ((st = read_back(B, s))) return st;
    std::vector<double> nb(C), nr(C), ratio(C, 1.0), theta(C), est(C);
    std::vector<int> its(C), stall(C, 0), done(C, 0), outer(C, 0);
    std::vector<tfde_info> info(C);
    std::vector<int> status(C, TFDE_ENOCONV);
    for (int i = 0; i < C; ++i) {
        nb[i] = std::sqrt(B->h_s[i * kSS + S_BB]);
        nr[i] = std::sqrt(B->h_s[i * kSS + S_RR]);
        info[i] = tfde_info{};
        info[i].relres0 = nb[i] > 0.0 ? nr[i] / nb[i] : 0.0;
        if (!std::isfinite(nb[i]) || !std::isfinite(nr[i])) return set_error(TFDE_ENAN, "non-finite right-hand side");
    }
    const int max_sweeps = 200;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        int any = 0;
        for (int i = 0; i < C; ++i) {
            outer[i] = 0;
            if (done[i]) continue;
            if (nb[i] == 0.0 || nr[i] <= tol * nb[i]) {
                done[i] = 1;
                status[i] = TFDE_OK;
                continue;
            }
            outer[i] = 1;
            any = 1;
            double th = 0.5 * tol * nb[i] / nr[i] / ratio[i];
            // beyond one sweep's reach (~1e-4): two sweeps share the reduction
            theta[i] = th < 1e-4 ? std::max(1e-4, std::sqrt(th)) : th;
            B->h_s[i * kSS + S_SC32] = 1.0 / nr[i];
            B->h_s[i * kSS + S_ADD] = nr[i];
            B->h_act[i] = 1;
        }
        if (!any) break;
        for (int i = 0; i < C; ++i) B->h_act[i] = outer[i];
        if ((st = upload_act_scalars(B, s))) return st;
        stats_count_launch();
        bk_scale64to32<<<B->NB, kBT, 0, s>>>(B->d_vt, B->d_bi, B->d_bo, B->d_act, B->d_s);
        // symmetric problems: batched PCG; the others: batched GMRES cycles
        std::vector<int> og(C, 0), op(C, 0);
        bool anyg = false, anyp = false;
        for (int i = 0; i < C; ++i) {
            if (!outer[i]) continue;
            if (B->sym_pcg && B->spectral && B->P[i]->symmetric) {
                op[i] = 1;
                anyp = true;
            } else {
                og[i] = 1;
                anyg = true;
            }
        }
        if (anyg) {
            if ((st = batch_cycle(B, og, theta, est, its, s))) return st;
        } else {
            std::fill(est.begin(), est.end(), 1.0);
            std::fill(its.begin(), its.end(), 0);
        }
        if (anyp) {
            std::vector<double> est_p(C, 1.0);
            std::vector<int> its_p(C, 0);
            if ((st = batch_pcg(B, op, theta, est_p, its_p, s))) return st;
            for (int i = 0; i < C; ++i)
                if (op[i]) {
                    est[i] = est_p[i];
                    its[i] = its_p[i];
                }
        }
        for (int i = 0; i < C; ++i) B->h_act[i] = outer[i];
        B_TRY(cudaMemcpyAsync(B->d_act, B->h_act, C * sizeof(int), cudaMemcpyHostToDevice, s));
        stats_count_launch();
        bk_add32to64<<<B->NB, kBT, 0, s>>>(B->d_vt, B->d_bi, B->d_bo, B->d_act, B->d_s);
        // accurate FP64 residuals r = b - A x of every problem still refining,
        // as three grouped slicing and three grouped exact-contraction launches,
        // with their norms (summed in the z pass under the scale 2^shift, shift =
        // -ilogb ||b||, into S_RR) and A_N x (formed exactly in the z-pass
        // slicing, for the next chained step)
        std::vector<int> shift(C, 0);
        std::vector<const double*> xs(uu.begin(), uu.end());
        for (int i = 0; i < C; ++i) {
            if (!outer[i]) continue;
            B->P[i]->an_ready = false;
            shift[i] = -std::ilogb(nb[i]);
        }
        if ((st = oz_batch_residual(B->oz, xs.data(), outer.data(), B->d_act, shift.data(), oz_slices_for_tol(tol), s)))
            return st;
        for (int i = 0; i < C; ++i)
            if (outer[i]) B->P[i]->an_ready = true;
        if ((st = read_back(B, s))) return st;
        for (int i = 0; i < C; ++i) {
            if (!outer[i]) continue;
            const double nr_old = nr[i];
            nr[i] = std::ldexp(std::sqrt(B->h_s[i * kSS + S_RR]), -shift[i]);
            info[i].iters += its[i];
            info[i].restarts++;
            info[i].refine_sweeps++;
            if (!std::isfinite(nr[i])) {
                done[i] = 1;
                status[i] = set_error(TFDE_ENAN, "non-finite residual");
                continue;
            }
            if (est[i] > 0.0) {
                const double observed = (nr[i] / nr_old) / est[i];
                ratio[i] = observed > 1.0 ? observed : 1.0;
            }
            stall[i] = (nr[i] > 0.5 * nr_old) ? stall[i] + 1 : 0;
            if (stall[i] >= 2 && nr[i] > tol * nb[i]) {
                // refinement stopped contracting: finish this problem with FP64 cycles
                tfde_problem* P = B->P[i];
                tfde_info sub{};
                info[i].fallback = 1;
                P->an_ready = false;   // the FP64 cycles move x past the last exact residual
                status[i] = (B->sym_pcg && B->spectral && P->symmetric)
                                ? pcg64(P, P->w[tfde_problem::W_B], uu[i], tol, 10000, &sub, s, false)
                                : pgmres64(P, P->w[tfde_problem::W_B], uu[i], B->restart, tol, 10000, &sub, s, false);
                info[i].iters += sub.iters;
                info[i].restarts += sub.restarts;
                nr[i] = sub.relres * nb[i];
                done[i] = 1;
            }
        }
    }
    const float ms = (float)std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    int worst = TFDE_OK;
    for (int i = 0; i < C; ++i) {
        if (!done[i]) status[i] = TFDE_ENOCONV;
        info[i].relres = nb[i] > 0.0 ? nr[i] / nb[i] : 0.0;
        info[i].ms = ms;
        if (infos) infos[B->caller[i]] = info[i];
        if (status[i] != TFDE_OK && worst == TFDE_OK) worst = status[i];
    }
    if (worst == TFDE_OK) {
        B->chain_ok = true;
        B->chain_u = uu;
    } else if (worst == TFDE_ENOCONV) {
        set_error(TFDE_ENOCONV, "batched solve: a problem reached its sweep limit");
    }
    return worst;
}

}  // namespace tfde
