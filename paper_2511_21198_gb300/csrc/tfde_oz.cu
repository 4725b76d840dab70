// FP64-accurate operator application for the mixed path (Eq. (linear_sys)):
//
//   A x = A3 (A2 (A1 + G1) x + G2 A1 x) + G3 A2 A1 x,   G_a = eta_a B_a,
//
// as three axis passes of the exact-integer slice contraction
// (tfde_oz_kernel.cuh), with no FP64 arithmetic per grid point:
//   x pass: a = (A1 + G1) x,  w = A1 x             (input x sliced along x)
//   y pass: c = A2 a + G2 w,  e = A2 w             (a and w sliced jointly along y)
//   z pass: y = A3 c + G3 e                        (c and e sliced jointly along z)
// The two operators of a two-input pass share one scale per row and the two
// inputs one scale per line, so both land in the same exact accumulators.
#define TFDE_OZ_KERNEL_IMPL
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "tfde_mixed.h"
#include "tfde_oz_kernel.cuh"
#include "tfde_stats.h"

namespace tfde {

namespace {

// ------------------------------------------------------------ digit slicing
// Fixed-point integer round(|x| 2^{7S - E}) with the sign of x, from the FP64
// bits alone (|x| < 2^E): the mantissa m shifted right by r with
// round-half-up, floor((m + 2^{r-1}) / 2^r) = floor((floor(m / 2^{r-1}) + 1) / 2).
template <int S>
__device__ __forceinline__ long long fixed_point(long long bits, int E) {
    const unsigned long long u = (unsigned long long)bits & 0x7FFFFFFFFFFFFFFFull;
    if (u == 0) return 0;
    int e = (int)(u >> 52);
    unsigned long long mant = u & ((1ull << 52) - 1);
    if (e == 0) e = 1; else mant |= (1ull << 52);
    const int r = 1075 - e - 7 * S + E;   // right shift; >= 53 - 7S >= 4 for S <= 7
    long long X;
    if (r > 64) X = 0;
    else if (r <= 0) X = (long long)(mant << (-r));
    else X = (long long)(((mant >> (r - 1)) + 1) >> 1);
    return bits < 0 ? -X : X;
}

// Exponent E with |x| < 2^E for the largest |x| of a line, from the largest
// high word of |x| over the line (bits 20..30: the biased exponent) and the OR
// of the low words (nonzero with a zero high word: a subnormal maximum); 0 for
// an all-zero line.
__device__ __forceinline__ int line_exponent(uint32_t hmax, uint32_t lor) {
    if (hmax == 0) return lor ? -1021 : 0;
    const int e = (int)(hmax >> 20);
    return e == 0 ? -1021 : e - 1022;
}
// high word of |x| 2^sh (exponent field moved by sh) for a normal or zero x
__device__ __forceinline__ uint32_t abs_hi_shifted(unsigned long long bits, int sh) {
    const uint32_t h = (uint32_t)(bits >> 32) & 0x7FFFFFFFu;
    return (h | (uint32_t)bits) ? h + ((uint32_t)sh << 20) : 0u;
}

// Balanced base-128 digits of X (|X| <= 2^{7S}): X = sum_t d_t 128^{S-1-t} with
// d_t in [-64, 63] for t >= 1 and the leading d_0 in [-128, 128].  Adding 64 to
// every digit below the leading one, Y = X + 64 (128^{S-1} - 1) / 127, turns
// them into plain base-128 digits of Y, so d_t = ((Y >> 7 (S-1-t)) & 127) - 64
// for t >= 1 and d_0 = Y >> 7 (S-1) (arithmetic shift): no carry chain.
template <int S>
__host__ __device__ constexpr long long digit_bias() {
    long long b = 0;
    for (int t = 1; t < S; ++t) b = b * 128 + 64;
    return b;
}
// A small integer d (|d| < 2^22) as an FP32 value without a conversion
// instruction: the bit pattern of 1.5 2^23 + d (same binade) minus 1.5 2^23,
// both exact.  The digit field f in [0, 127] gives f - 64 the same way.  The
// BF16 bits of such a value are the top half of its FP32 bits (exact: at most
// 8 significant bits), and two of them pack with one byte permutation.
constexpr uint32_t kMagic = 0x4B400000u;   // 1.5 2^23
__device__ __forceinline__ float small_int_float(int d) { return __int_as_float((int)kMagic + d) - 12582912.0f; }
__device__ __forceinline__ float digit_float(uint32_t f) { return __uint_as_float(kMagic | f) - 12582976.0f; }
__device__ __forceinline__ uint32_t pack_bf16_tops(float a, float b) {
    return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}
// digits of two neighbouring grid points (idx even, idx + 1) as packed BF16 pairs
template <int S>
__device__ __forceinline__ void write_digits2(long long Xa, long long Xb, __nv_bfloat16* planes, long long N,
                                              long long idx) {
    constexpr long long bias = digit_bias<S>();
    const long long Ya = Xa + bias, Yb = Xb + bias;
#pragma unroll
    for (int t = 1; t < S; ++t) {
        const int sh = 7 * (S - 1 - t);
        const float da = digit_float((uint32_t)(Ya >> sh) & 127u);
        const float db = digit_float((uint32_t)(Yb >> sh) & 127u);
        *reinterpret_cast<uint32_t*>(planes + (long long)t * N + idx) = pack_bf16_tops(da, db);
    }
    constexpr int sh0 = 7 * (S - 1);
    *reinterpret_cast<uint32_t*>(planes + idx) =
        pack_bf16_tops(small_int_float((int)(Ya >> sh0)), small_int_float((int)(Yb >> sh0)));
}

// The double Y * 2^s for an integer |Y| < 2^53 (exact; results below the
// normal range are flushed to zero), from the integer bits alone.
__device__ __forceinline__ double i64_ldexp_exact(long long Y, int s) {
    if (Y == 0) return 0.0;
    const unsigned long long neg = Y < 0 ? 1ull : 0ull;
    const unsigned long long mag = (unsigned long long)(Y < 0 ? -Y : Y);
    const int nbits = 64 - __clzll((long long)mag);
    const int be = nbits - 1 + s + 1023;
    if (be <= 0) return 0.0;
    const unsigned long long m = mag << (53 - nbits);
    return __longlong_as_double((long long)((neg << 63) | ((unsigned long long)be << 52) | (m & ((1ull << 52) - 1))));
}

// x axis: one warp per line of n1 contiguous values, each lane taking pairs of
// neighbouring points (16-byte loads, packed BF16 digit pairs).  Writes the
// digit planes of x under its line maximum and, when wout is set,
// w = A_{n1} x along the line from the same fixed-point integers X
// (w_k = (X_{k-1} + 6 X_k + X_{k+1}) 2^{E - 7S - 3}, |sum| < 2^53: exact).
// S (digits) is a template argument: every digit shift is a constant.
template <int S>
__device__ __forceinline__ void slice_x_line(const double* __restrict__ x0, int n1, __nv_bfloat16* __restrict__ p0,
                                             long long N, int* __restrict__ lexp, double* __restrict__ wout, long long l,
                                             int lane) {
    const longlong2* r2 = reinterpret_cast<const longlong2*>(x0 + l * n1);   // n1 even: pairs stay in the line
    const int np = n1 / 2;
    uint32_t hmax = 0, lor = 0;
#pragma unroll 4
    for (int q = lane; q < np; q += 32) {
        const longlong2 v = r2[q];
        hmax = max(hmax, max((uint32_t)((unsigned long long)v.x >> 32) & 0x7FFFFFFFu,
                             (uint32_t)((unsigned long long)v.y >> 32) & 0x7FFFFFFFu));
        lor |= (uint32_t)v.x | (uint32_t)v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        hmax = max(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
        lor |= __shfl_xor_sync(0xffffffffu, lor, o);
    }
    const int E = line_exponent(hmax, lor);
    long long left_carry = 0;   // X just before this iteration's first point
    long long Xa = 0, Xb = 0;
    if (lane < np) {
        const longlong2 v = r2[lane];
        Xa = fixed_point<S>(v.x, E);
        Xb = fixed_point<S>(v.y, E);
    }
    for (int base = 0; base < np; base += 32) {
        const int q = base + lane;
        const int qn = q + 32;
        long long Na = 0, Nb = 0;
        if (qn < np) {
            const longlong2 v = r2[qn];
            Na = fixed_point<S>(v.x, E);
            Nb = fixed_point<S>(v.y, E);
        }
        if (q < np) write_digits2<S>(Xa, Xb, p0, N, l * n1 + 2 * q);
        if (wout) {
            long long left = __shfl_up_sync(0xffffffffu, Xb, 1);
            long long right = __shfl_down_sync(0xffffffffu, Xa, 1);
            const long long first_next = __shfl_sync(0xffffffffu, Na, 0);
            if (lane == 0) left = left_carry;
            if (lane == 31) right = first_next;
            if (q < np) {
                const int sc = E - 7 * S - 3;
                *reinterpret_cast<double2*>(wout + l * n1 + 2 * q) =
                    make_double2(i64_ldexp_exact(left + 6 * Xa + Xb, sc), i64_ldexp_exact(Xa + 6 * Xb + right, sc));
            }
            left_carry = __shfl_sync(0xffffffffu, Xb, 31);
        }
        Xa = Na;
        Xb = Nb;
    }
    if (lane == 0) lexp[l] = E;
}

template <int S>
__global__ void slice_x_kernel(const double* __restrict__ x0, int n1, long long lines,
                               __nv_bfloat16* __restrict__ p0, long long N, int* __restrict__ lexp,
                               double* __restrict__ wout) {
    const int lane = threadIdx.x & 31;
    const long long wg = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long l = wg; l < lines; l += nw) slice_x_line<S>(x0, n1, p0, N, lexp, wout, l, lane);
}

// y / z axes: LB consecutive lines (contiguous in memory) per 512-thread
// block, each thread taking a pair of neighbouring lines.  The block's lines
// of both inputs are copied once into shared memory (16-byte cp.async, all in
// flight together), the joint line maximum of x0 and x1 * 2^sh1 is reduced
// there, and the digits go out as packed BF16 pairs: every input element
// crosses HBM once and every store covers two grid points.  When eout is set,
// e = A_n x1 along the line from the fixed-point integers W of x1 (exact as in
// slice_x_kernel).
constexpr int SL_THREADS = 512;

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

// One group of LB lines starting at line l0 of slice_staged_kernel (the whole
// block; s0 / s1 the staged lines of the two inputs in shared memory).
template <int LB, int S>
__device__ __forceinline__ void slice_staged_group(const double* __restrict__ x0, const double* __restrict__ x1,
                                                   int sh1, const AxisView& v, __nv_bfloat16* __restrict__ p0,
                                                   __nv_bfloat16* __restrict__ p1, long long N,
                                                   int* __restrict__ lexp, double* __restrict__ eout, long long l0,
                                                   unsigned long long* s0, unsigned long long* s1,
                                                   uint32_t (*shmax)[LB], uint32_t (*slor)[LB], int* sexp) {
    constexpr int LP = LB / 2;               // line pairs per block
    constexpr int NKG = SL_THREADS / LP;     // k rows in flight
    const int lp = threadIdx.x % LP, kg = threadIdx.x / LP;
    const int la = 2 * lp;                   // first line of the pair within the block
    const long long* b0 = reinterpret_cast<const long long*>(x0);
    const long long* b1 = reinterpret_cast<const long long*>(x1);
    const long long l = l0 + la;          // lines l, l + 1 (same run: runs hold a multiple of 8 lines)
    const bool valid = l < v.lines;
    const long long off = valid ? (l % v.l_in) * v.s_in + (l / v.l_in) * v.s_out : 0;
    if (valid) {
        for (int k = kg; k < v.n; k += NKG) {
            const long long idx = off + (long long)k * v.stride;
            cp_async16(s0 + k * LB + la, b0 + idx);
            if (b1) cp_async16(s1 + k * LB + la, b1 + idx);
        }
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    uint32_t ha = 0, hb = 0, oa = 0, ob = 0;
    if (valid) {
        for (int k = kg; k < v.n; k += NKG) {
            const unsigned long long wa = s0[k * LB + la], wb = s0[k * LB + la + 1];
            ha = max(ha, (uint32_t)(wa >> 32) & 0x7FFFFFFFu);
            hb = max(hb, (uint32_t)(wb >> 32) & 0x7FFFFFFFu);
            oa |= (uint32_t)wa;
            ob |= (uint32_t)wb;
            if (b1) {
                const unsigned long long ua = s1[k * LB + la], ub = s1[k * LB + la + 1];
                ha = max(ha, abs_hi_shifted(ua, sh1));
                hb = max(hb, abs_hi_shifted(ub, sh1));
                oa |= (uint32_t)ua;
                ob |= (uint32_t)ub;
            }
        }
    }
    shmax[kg][la] = ha;
    shmax[kg][la + 1] = hb;
    slor[kg][la] = oa;
    slor[kg][la + 1] = ob;
    __syncthreads();
    if (threadIdx.x < LB) {
        uint32_t m = shmax[0][threadIdx.x], o = slor[0][threadIdx.x];
#pragma unroll 8
        for (int g = 1; g < NKG; ++g) {
            m = max(m, shmax[g][threadIdx.x]);
            o |= slor[g][threadIdx.x];
        }
        const int E = line_exponent(m, o);
        sexp[threadIdx.x] = E;
        if (l0 + threadIdx.x < v.lines) lexp[l0 + threadIdx.x] = E;
    }
    __syncthreads();
    const int Ea = sexp[la], Eb = sexp[la + 1];
    if (valid) {
        for (int k = kg; k < v.n; k += NKG) {
            const long long idx = off + (long long)k * v.stride;
            write_digits2<S>(fixed_point<S>((long long)s0[k * LB + la], Ea),
                             fixed_point<S>((long long)s0[k * LB + la + 1], Eb), p0, N, idx);
            if (b1) {
                const long long Wa = fixed_point<S>((long long)s1[k * LB + la], Ea - sh1);
                const long long Wb = fixed_point<S>((long long)s1[k * LB + la + 1], Eb - sh1);
                write_digits2<S>(Wa, Wb, p1, N, idx);
                if (eout) {
                    s1[k * LB + la] = (unsigned long long)Wa;
                    s1[k * LB + la + 1] = (unsigned long long)Wb;
                }
            }
        }
    }
    if (eout && b1) {
        __syncthreads();
        if (valid) {
            for (int k = kg; k < v.n; k += NKG) {
                double e2[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int c = la + q;
                    const long long Wp = k > 0 ? (long long)s1[(k - 1) * LB + c] : 0;
                    const long long Wn = k + 1 < v.n ? (long long)s1[(k + 1) * LB + c] : 0;
                    const long long W = (long long)s1[k * LB + c];
                    e2[q] = i64_ldexp_exact(Wp + 6 * W + Wn, (q ? Eb : Ea) - sh1 - 7 * S - 3);
                }
                *reinterpret_cast<double2*>(eout + off + (long long)k * v.stride) = make_double2(e2[0], e2[1]);
            }
        }
    }
    __syncthreads();
}

template <int LB, int S>
__global__ __launch_bounds__(SL_THREADS) void slice_staged_kernel(const double* __restrict__ x0,
                                                                  const double* __restrict__ x1, int sh1, AxisView v,
                                                                  __nv_bfloat16* __restrict__ p0,
                                                                  __nv_bfloat16* __restrict__ p1, long long N,
                                                                  int* __restrict__ lexp, double* __restrict__ eout) {
    constexpr int NKG = SL_THREADS / (LB / 2);
    extern __shared__ unsigned long long sl_smem[];   // [input][k][LB]
    __shared__ uint32_t shmax[NKG][LB];
    __shared__ uint32_t slor[NKG][LB];
    __shared__ int sexp[LB];
    for (long long l0 = (long long)blockIdx.x * LB; l0 < v.lines; l0 += (long long)gridDim.x * LB)
        slice_staged_group<LB, S>(x0, x1, sh1, v, p0, p1, N, lexp, eout, l0, sl_smem, sl_smem + (size_t)v.n * LB, shmax,
                                  slor, sexp);
}

// ---- grouped slicing over the problems of a batch: every problem's lines
// in one launch, the work items (x: lines, y / z: groups of LB lines) of
// problem g at start[g] .. start[g + 1] - 1; problems with act[g] == 0 are
// skipped.
struct SliceDesc {
    const double* x0;
    const double* x1;
    int sh1;
    int n1;
    AxisView v;
    __nv_bfloat16* p0;
    __nv_bfloat16* p1;
    long long N;
    int* lexp;
    double* eout;
};

__device__ __forceinline__ int slice_find(const long long* __restrict__ start, int ng, long long t) {
    int lo = 0, hi = ng - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(start + mid) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int S>
__global__ void slice_x_grouped_kernel(const SliceDesc* __restrict__ d, const long long* __restrict__ start, int ng,
                                       const int* __restrict__ act) {
    const int lane = threadIdx.x & 31;
    const long long wg = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long total = __ldg(start + ng);
    for (long long t = wg; t < total; t += nw) {   // warp-uniform
        const int g = slice_find(start, ng, t);
        if (!__ldg(act + g)) continue;
        const SliceDesc& D = d[g];
        slice_x_line<S>(D.x0, D.n1, D.p0, D.N, D.lexp, D.eout, t - __ldg(start + g), lane);
    }
}

template <int LB, int S>
__global__ __launch_bounds__(SL_THREADS) void slice_staged_grouped_kernel(const SliceDesc* __restrict__ d,
                                                                          const long long* __restrict__ start, int ng,
                                                                          const int* __restrict__ act) {
    constexpr int NKG = SL_THREADS / (LB / 2);
    extern __shared__ unsigned long long sl_smem[];   // [input][k][LB], sized for the longest lines
    __shared__ uint32_t shmax[NKG][LB];
    __shared__ uint32_t slor[NKG][LB];
    __shared__ int sexp[LB];
    const long long total = __ldg(start + ng);
    for (long long t = blockIdx.x; t < total; t += gridDim.x) {   // block-uniform
        const int g = slice_find(start, ng, t);
        if (!__ldg(act + g)) continue;
        const SliceDesc& D = d[g];
        slice_staged_group<LB, S>(D.x0, D.x1, D.sh1, D.v, D.p0, D.p1, D.N, D.lexp, D.eout, (t - __ldg(start + g)) * LB,
                                  sl_smem, sl_smem + (size_t)D.v.n * LB, shmax, slor, sexp);
    }
}

// ------------------------------------------------------- operator slicing
// Digit slices of one or two n x n operators (row-major) under a common
// power-of-two scale per row: slices[op][t][m][k]; returns the row exponents
// and, per operator, the number of leading slices that are not all zero.
void slice_operators_host(const std::vector<const std::vector<double>*>& ops, int n, int S,
                          std::vector<std::vector<__nv_bfloat16>>& slices, std::vector<int>& rexp,
                          std::vector<int>& nonzero) {
    const size_t nn = (size_t)n * n;
    slices.assign(ops.size(), std::vector<__nv_bfloat16>((size_t)S * nn, __float2bfloat16_rn(0.f)));
    nonzero.assign(ops.size(), 0);
    rexp.assign(n, 0);
    for (int m = 0; m < n; ++m) {
        double vmax = 0.0;
        for (const auto* G : ops)
            for (int k = 0; k < n; ++k) vmax = std::fmax(vmax, std::fabs((*G)[(size_t)m * n + k]));
        int E = 0;
        if (vmax > 0.0) std::frexp(vmax, &E);
        rexp[m] = E;
        for (size_t o = 0; o < ops.size(); ++o)
            for (int k = 0; k < n; ++k) {
                long long X = std::llrint(std::ldexp((*ops[o])[(size_t)m * n + k], 7 * S - E));
                for (int t = S - 1; t >= 0; --t) {
                    long long r;
                    if (t > 0) {
                        r = X & 127;
                        if (r >= 64) r -= 128;
                        X = (X - r) >> 7;
                    } else {
                        r = X;
                    }
                    if (r != 0) nonzero[o] = std::max(nonzero[o], t + 1);
                    slices[o][(size_t)t * nn + (size_t)m * n + k] = __float2bfloat16_rn((float)r);
                }
            }
    }
    for (auto& z : nonzero) z = std::max(z, 1);
}

#define OZ_TRY(expr)                                                                       \
    do {                                                                                   \
        cudaError_t e__ = (expr);                                                          \
        if (e__ != cudaSuccess)                                                            \
            return set_error(TFDE_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e__)); \
    } while (0)

bool g_oz_attr = false;
// swizzle of the MN-major input tiles: one atom spans the tile's BN lines
constexpr CUtensorMapSwizzle kMnSwizzle = oz::BN * 2 == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;

// Upload one operator digit set and build its tensor maps.
int upload_set(OzSet& set, const std::vector<__nv_bfloat16>& sl, int n, int S, int na, int rexp_index,
               cudaStream_t s) {
    OZ_TRY(cudaMalloc((void**)&set.dev, sl.size() * sizeof(__nv_bfloat16)));
    OZ_TRY(cudaMemcpyAsync(set.dev, sl.data(), sl.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice, s));
    set.na = na;
    set.rexp_index = rexp_index;
    for (int t = 0; t < S; ++t) {
        int st = tc::make_map_A(&set.amap[t], set.dev + (size_t)t * n * n, n);
        if (st) return st;
        // slices 0..t as one 3-D tensor (k, row, slice)
        const cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)S};
        const cuuint64_t strides[2] = {(cuuint64_t)n * 2, (cuuint64_t)n * n * 2};
        const cuuint32_t box[3] = {(cuuint32_t)tc::BK, (cuuint32_t)tc::BM, (cuuint32_t)(t + 1)};
        // a merged map the driver refuses leaves the per-slice copies in use
        set.amapk_ok[t] = tc::encode_map(&set.amapk[t], set.dev, 3, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_64B) == TFDE_OK;
    }
    return TFDE_OK;
}

}  // namespace

int oz_init(tfde_problem* P, const std::vector<double> etaB[3], cudaStream_t s) {
    MixedState* M = mixed(P);
    const int S = OZ_SLICES;
    const size_t N = P->N;
    auto mass = [](int n) {
        std::vector<double> A((size_t)n * n, 0.0);
        for (int i = 0; i < n; ++i) {
            A[(size_t)i * n + i] = 0.75;
            if (i > 0) A[(size_t)i * n + i - 1] = 0.125;
            if (i + 1 < n) A[(size_t)i * n + i + 1] = 0.125;
        }
        return A;
    };
    auto upload_rexp = [&](const std::vector<int>& r) -> int {
        int* d = nullptr;
        if (cudaMalloc((void**)&d, r.size() * sizeof(int)) != cudaSuccess) return -1;
        cudaMemcpyAsync(d, r.data(), r.size() * sizeof(int), cudaMemcpyHostToDevice, s);
        M->oz_rexp.push_back(d);
        return (int)M->oz_rexp.size() - 1;
    };
    std::vector<std::vector<__nv_bfloat16>> sl;
    std::vector<int> rexp, nz;
    int st;
    // x pass: (A1 + G1), (A1 - G1) and G1, each under its own row scales
    // (A1 x itself comes out of the slicing, exactly)
    {
        const int n = P->n[0];
        const std::vector<double> A1 = mass(n);
        std::vector<double> plus(A1), minus(A1);
        for (size_t i = 0; i < plus.size(); ++i) {
            plus[i] += etaB[0][i];
            minus[i] -= etaB[0][i];
        }
        const std::vector<double>* single[3] = {&plus, &minus, &etaB[0]};
        OzSet* sets[3] = {&M->oz_x_plus, &M->oz_x_minus, &M->oz_x_stiff};
        for (int k = 0; k < 3; ++k) {
            slice_operators_host({single[k]}, n, S, sl, rexp, nz);
            const int ri = upload_rexp(rexp);
            if (ri < 0) return set_error(TFDE_ENOMEM, "cudaMalloc of row exponents failed");
            if ((st = upload_set(*sets[k], sl[0], n, S, nz[0], ri, s))) return st;
        }
    }
    // y and z passes: (A_a | +G_a) and (A_a | -G_a) under common row scales.
    // The second input (A1 x, resp. A2 A1 x) is smaller than the first by about
    // max |G_a|; it is sliced as input * 2^k and G_a is stored as G_a * 2^-k
    // (both exact), so that the two inputs share their line scale without
    // losing bits.
    for (int a = 1; a <= 2; ++a) {
        const int n = P->n[a];
        double gmax = 0.0;
        for (double v : etaB[a]) gmax = std::fmax(gmax, std::fabs(v));
        int k = 0;
        if (gmax > 0.0) std::frexp(gmax, &k);
        M->oz_shift[a] = k;
        std::vector<double> Am = mass(n);
        std::vector<double> pos(etaB[a]), neg(etaB[a]);
        for (auto& v : pos) v = std::ldexp(v, -k);
        for (auto& v : neg) v = -std::ldexp(v, -k);
        slice_operators_host({&Am, &pos, &neg}, n, S, sl, rexp, nz);
        const int ri = upload_rexp(rexp);
        if (ri < 0) return set_error(TFDE_ENOMEM, "cudaMalloc of row exponents failed");
        OzSet* m_set = a == 1 ? &M->oz_y_mass_c : &M->oz_z_mass_c;
        OzSet* p_set = a == 1 ? &M->oz_y_plus : &M->oz_z_plus;
        OzSet* n_set = a == 1 ? &M->oz_y_minus : &M->oz_z_minus;
        if ((st = upload_set(*m_set, sl[0], n, S, nz[0], ri, s))) return st;
        if ((st = upload_set(*p_set, sl[1], n, S, nz[1], ri, s))) return st;
        if ((st = upload_set(*n_set, sl[2], n, S, nz[2], ri, s))) return st;
    }
    OZ_TRY(cudaStreamSynchronize(s));
    // digit planes of two inputs and their maps
    for (int in = 0; in < 2; ++in) {
        OZ_TRY(cudaMalloc((void**)&M->oz_planes[in], (size_t)S * N * sizeof(__nv_bfloat16)));
        for (int t = 0; t < S; ++t)
            for (int a = 0; a < 3; ++a) {
                const __nv_bfloat16* base = M->oz_planes[in] + (size_t)t * N;
                if (a == 0) {
                    st = tc::make_map_B_box(&M->oz_bmap[in][t][a], base, P->n, a, oz::BN);
                } else {
                    // MN-major slice: box {BN lines, BK, 1 plane}, swizzle span BN x 2 bytes
                    const cuuint64_t c1 = P->n[0], c2 = P->n[1], c3 = P->n[2];
                    const cuuint64_t C = a == 1 ? c1 : c1 * c2, K = a == 1 ? c2 : c3, Pl = a == 1 ? c3 : 1;
                    const cuuint64_t dims[3] = {C, K, Pl};
                    const cuuint64_t strides[2] = {C * 2, C * K * 2};
                    const cuuint32_t box[3] = {(cuuint32_t)oz::BN, (cuuint32_t)tc::BK, 1};
                    st = tc::encode_map(&M->oz_bmap[in][t][a], base, 3, dims, strides, box, kMnSwizzle);
                }
                if (st) return st;
                // slices 0..t of input `in` along axis a in one box
                const cuuint64_t n1 = P->n[0], n2 = P->n[1], n3 = P->n[2];
                int es;
                if (a == 0) {
                    const cuuint64_t dims[3] = {n1, n2 * n3, (cuuint64_t)S};
                    const cuuint64_t strides[2] = {n1 * 2, (cuuint64_t)N * 2};
                    const cuuint32_t box[3] = {(cuuint32_t)tc::BK, (cuuint32_t)oz::BN, (cuuint32_t)(t + 1)};
                    es = tc::encode_map(&M->oz_bmapm[in][a][t], M->oz_planes[in], 3, dims, strides, box,
                                        CU_TENSOR_MAP_SWIZZLE_64B);   // K-major rows of BK x 2 = 64 bytes
                } else if (a == 1) {
                    const cuuint64_t dims[4] = {n1, n2, n3, (cuuint64_t)S};
                    const cuuint64_t strides[3] = {n1 * 2, n1 * n2 * 2, (cuuint64_t)N * 2};
                    const cuuint32_t box[4] = {(cuuint32_t)oz::BN, (cuuint32_t)tc::BK, 1, (cuuint32_t)(t + 1)};
                    es = tc::encode_map(&M->oz_bmapm[in][a][t], M->oz_planes[in], 4, dims, strides, box, kMnSwizzle);
                } else {
                    const cuuint64_t dims[3] = {n1 * n2, n3, (cuuint64_t)S};
                    const cuuint64_t strides[2] = {n1 * n2 * 2, (cuuint64_t)N * 2};
                    const cuuint32_t box[3] = {(cuuint32_t)oz::BN, (cuuint32_t)tc::BK, (cuuint32_t)(t + 1)};
                    es = tc::encode_map(&M->oz_bmapm[in][a][t], M->oz_planes[in], 3, dims, strides, box, kMnSwizzle);
                }
                M->oz_bmapm_ok[in][a][t] = es == TFDE_OK;
            }
    }
    long long maxlines = 0;
    for (int a = 0; a < 3; ++a) maxlines = std::max(maxlines, (long long)(N / P->n[a]));
    OZ_TRY(cudaMalloc((void**)&M->oz_lexp, maxlines * sizeof(int)));
    return TFDE_OK;
}

void oz_free(MixedState* M) {
    OzSet* sets[] = {&M->oz_x_plus, &M->oz_x_minus, &M->oz_x_stiff, &M->oz_y_mass_c, &M->oz_y_plus,
                     &M->oz_y_minus, &M->oz_z_mass_c, &M->oz_z_plus, &M->oz_z_minus};
    for (OzSet* z : sets) cudaFree(z->dev);
    for (int* r : M->oz_rexp) cudaFree(r);
    M->oz_rexp.clear();
    cudaFree(M->oz_planes[0]);
    cudaFree(M->oz_planes[1]);
    cudaFree(M->oz_lexp);
}

namespace {

// One y / z slicing launch (grid: the line groups, at most as many blocks as
// fit the SMs' shared memory three times over; blocks loop over groups).
// Measured on GB300: sizing the grid to one wave of resident blocks with the
// largest carve-out (3 blocks per SM instead of 2) was no faster: the
// integer pipe, not latency, bounds these kernels.
template <int LB, int S>
void staged_launch(long long groups, size_t smem, cudaStream_t s, const double* x0, const double* x1, int sh1,
                   const AxisView& v, __nv_bfloat16* p0, __nv_bfloat16* p1, long long N, int* lexp, double* eout) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(slice_staged_kernel<LB, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    const long long per_sm = std::max<long long>(1, (long long)(220 * 1024 / std::max<size_t>(smem, 1)));
    const long long blocks = std::max<long long>(1, std::min<long long>(groups, 152LL * per_sm));
    slice_staged_kernel<LB, S><<<(unsigned)blocks, SL_THREADS, smem, s>>>(x0, x1, sh1, v, p0, p1, N, lexp, eout);
}

// One slicing launch with S digits (see oz_slice).
template <int S>
void oz_slice_s(const tfde_problem* P, int axis, const double* x0, const double* x1, int sh1, double* mass_out,
                cudaStream_t s) {
    MixedState* M = mixed(P);
    const AxisView v = axis_view(P->n, axis);
    const long long N = (long long)P->N;
    if (axis == 0) {
        // one warp per line; up to 16 blocks of 8 warps per SM, warps looping over lines
        const long long blocks = std::max<long long>(1, std::min<long long>((v.lines + 7) / 8, 152LL * 16));
        slice_x_kernel<S><<<(unsigned)blocks, 256, 0, s>>>(x0, P->n[0], v.lines, M->oz_planes[0], N, M->oz_lexp,
                                                          mass_out);
        return;
    }
    // 16 lines per block: with 64 KB of staged lines per block (n = 256, two
    // inputs) three blocks share an SM, so one block's loads overlap another's
    // digit writes; 32-line blocks would fill an SM alone and alternate the
    // two phases.  32 lines only for short lines, where a 16-line block would
    // stage too little to stream well.
    const int nin = x1 ? 2 : 1;
    const bool wide = (size_t)nin * v.n * 16 * 8 < 16 * 1024;
    const int LB = wide ? 32 : 16;
    const size_t smem = (size_t)nin * v.n * LB * 8;
    const long long groups = (v.lines + LB - 1) / LB;
    if (wide) staged_launch<32, S>(groups, smem, s, x0, x1, sh1, v, M->oz_planes[0], M->oz_planes[1], N, M->oz_lexp,
                                   mass_out);
    else staged_launch<16, S>(groups, smem, s, x0, x1, sh1, v, M->oz_planes[0], M->oz_planes[1], N, M->oz_lexp,
                              mass_out);
}

// Slice one or two FP64 inputs along `axis` into the digit planes 0 / 1, the
// second one taken as x1 * 2^sh1; mass_out (optional) receives the mass
// operator along `axis` applied to x1 (x0 on the x axis), exactly from the
// fixed-point integers.  S in [2, OZ_SLICES] (checked by the caller).
void oz_slice(const tfde_problem* P, int axis, const double* x0, const double* x1, int sh1, double* mass_out,
              int S, cudaStream_t s) {
    stats_count_launch();
    switch (S) {
        case 2: oz_slice_s<2>(P, axis, x0, x1, sh1, mass_out, s); break;
        case 3: oz_slice_s<3>(P, axis, x0, x1, sh1, mass_out, s); break;
        case 4: oz_slice_s<4>(P, axis, x0, x1, sh1, mass_out, s); break;
        case 5: oz_slice_s<5>(P, axis, x0, x1, sh1, mass_out, s); break;
        case 6: oz_slice_s<6>(P, axis, x0, x1, sh1, mass_out, s); break;
        default: oz_slice_s<7>(P, axis, x0, x1, sh1, mass_out, s); break;
    }
    static_assert(OZ_SLICES == 7, "one slicing instance per digit count");
}

// out = vsign * sum_seg Op_seg (planes of input seg.input) [+ asign * addend]
struct OzSegSpec {
    const OzSet* op;
    int input;  // digit planes 0 or 1
};

// The descriptor of one exact contraction out = vsign * sum_seg Op_seg (planes
// of input seg.input) [+ asign * addend] along `axis` at S slices; *pairs =
// the digit products per grid point and input.
void oz_params(const tfde_problem* P, int axis, const OzSegSpec* segs, int nseg, int vsign, const double* addend,
               double asign, double* out, int S, double* norm2, int norm_shift, oz::Params& prm, double* pairs) {
    MixedState* M = mixed(P);
    std::memset(&prm, 0, sizeof(prm));
    *pairs = 0.0;
    for (int g = 0; g < nseg; ++g) {
        oz::Segment& G = prm.seg[g];
        G.na = std::min(segs[g].op->na, S);
        G.nb = S;
        G.merged = segs[g].op->amapk_ok[G.na - 1] && M->oz_bmapm_ok[segs[g].input][axis][S - 1] ? 1 : 0;
        G.amapm = segs[g].op->amapk[G.na - 1];
        G.bmapm = M->oz_bmapm[segs[g].input][axis][S - 1];
        for (int t = 0; t < S; ++t) {
            G.amaps[t] = segs[g].op->amap[t];
            G.bmaps[t] = M->oz_bmap[segs[g].input][t][axis];
        }
        for (int sa = 0; sa < G.na; ++sa) *pairs += S - sa;
    }
    prm.nseg = nseg;
    prm.nslices = S;
    const long long n1 = P->n[0], n2 = P->n[1], n3 = P->n[2];
    prm.n = P->n[axis];
    prm.mhalves = (prm.n + oz::BM - 1) / oz::BM;
    prm.n1 = P->n[0];
    if (axis == 0) {
        prm.b_kmajor = 1;
        prm.lines = n2 * n3;
        prm.ntiles = (prm.lines + oz::BN - 1) / oz::BN;
    } else {
        prm.b_kmajor = 0;
        if (axis == 1) { prm.C = (int)n1; prm.P = (int)n3; prm.bm_rank = 4; }
        else { prm.C = (int)(n1 * n2); prm.P = 1; prm.bm_rank = 3; }
        prm.nbc = (prm.C + oz::BN - 1) / oz::BN;
        prm.nblocks = (long long)prm.nbc * prm.P;
        prm.ntiles = prm.nblocks;
        prm.lines = (long long)prm.C * prm.P;
        prm.plane = (long long)prm.C * prm.n;
    }
    prm.row_exp = M->oz_rexp[segs[0].op->rexp_index];
    prm.line_exp = M->oz_lexp;
    prm.value_sign = vsign;
    prm.addend_sign = asign;
    prm.addend = addend;
    prm.out = out;
    prm.norm2 = norm2;
    prm.norm_shift = norm_shift;
    prm.err = M->err;
}

int oz_set_attrs() {
    if (!g_oz_attr) {
        OZ_TRY(cudaFuncSetAttribute(oz::oz_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    oz::SMEM_BYTES));
        OZ_TRY(cudaFuncSetAttribute(oz::oz_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    oz::SMEM_BYTES));
        g_oz_attr = true;
    }
    return TFDE_OK;
}

int oz_contract(const tfde_problem* P, int axis, const OzSegSpec* segs, int nseg, int vsign, const double* addend,
                double asign, double* out, int S, cudaStream_t s, double* norm2 = nullptr, int norm_shift = 0) {
    const long long N = (long long)P->N;
    oz::Params prm;
    double pairs = 0.0;
    oz_params(P, axis, segs, nseg, vsign, addend, asign, out, S, norm2, norm_shift, prm, &pairs);
    if (int st = oz_set_attrs()) return st;
    const long long total = prm.ntiles * prm.mhalves;
    long long grid = total < tc::num_sms() ? total : tc::num_sms();
    void* tok = stats_tc_begin(s, TFDE_KIND_EXACT);
    oz::oz_gemm_kernel<false><<<(unsigned)(grid < 1 ? 1 : grid), oz::NUM_THREADS, oz::SMEM_BYTES, s>>>(
        prm, nullptr, nullptr, 0, nullptr);
    cudaError_t e = cudaGetLastError();
    // algorithmic bytes: digit planes of each input read once, FP64 out (+ addend);
    // flops: 2 n per grid point per digit pair
    const double na = prm.n;
    stats_tc_end(tok, s, TFDE_KIND_EXACT, (2.0 * S * nseg + 8.0 + (addend ? 8.0 : 0.0)) * N, 2.0 * pairs * na * N);
    if (e != cudaSuccess) return set_error(TFDE_ECUDA, std::string("oz_gemm_kernel launch: ") + cudaGetErrorString(e));
    return TFDE_OK;
}

}  // namespace

// y = vsign * (A x | (2 A_N - A) x | (A - A_N) x) [+ asign * addend], FP64-accurate.
int accurate_apply_ex(const tfde_problem* P, int op, const double* x, double* y, int vsign, const double* addend,
                      double asign, cudaStream_t s, int slices, double* norm2, int norm_shift, double* an_out) {
    if (slices < 2 || slices > OZ_SLICES) slices = OZ_SLICES;
    MixedState* M = mixed(P);
    const bool rhs = (op & 1) != 0;
    const bool stiff = (op & TFDE_OP_STIFF) != 0;
    double* ta = P->w[tfde_problem::W_A];
    double* tw = P->w[tfde_problem::W_W];
    double* tc_ = P->w[tfde_problem::W_C];
    double* te = P->w[tfde_problem::W_E];
    int st;
    // x pass: a = (A1 +- G1) x (or G1 x), w = A1 x (in the slicing, exact)
    oz_slice(P, 0, x, nullptr, 0, tw, slices, s);
    const OzSet* xop = stiff ? &M->oz_x_stiff : (rhs ? &M->oz_x_minus : &M->oz_x_plus);
    OzSegSpec sa[1] = {{xop, 0}};
    if ((st = oz_contract(P, 0, sa, 1, (stiff && rhs) ? -1 : 1, nullptr, 0.0, ta, slices, s))) return st;
    // y pass: c = A2 a +- G2 w, e = A2 w (in the slicing, exact)
    oz_slice(P, 1, ta, tw, M->oz_shift[1], te, slices, s);
    OzSegSpec sc[2] = {{&M->oz_y_mass_c, 0}, {rhs ? &M->oz_y_minus : &M->oz_y_plus, 1}};
    if ((st = oz_contract(P, 1, sc, 2, 1, nullptr, 0.0, tc_, slices, s))) return st;
    // z pass: y = A3 c +- G3 e (and, for op = A, A_N x = A3 e in the slicing)
    oz_slice(P, 2, tc_, te, M->oz_shift[2], (op == TFDE_OP_A) ? an_out : nullptr, slices, s);
    OzSegSpec sy[2] = {{&M->oz_z_mass_c, 0}, {rhs ? &M->oz_z_minus : &M->oz_z_plus, 1}};
    if (norm2) OZ_TRY(cudaMemsetAsync(norm2, 0, sizeof(double), s));
    return oz_contract(P, 2, sy, 2, vsign, addend, asign, y, slices, s, norm2, norm_shift);
}

int accurate_apply(const tfde_problem* P, int op, const double* x, double* y, cudaStream_t s) {
    return accurate_apply_ex(P, op, x, y, 1, nullptr, 0.0, s);
}

namespace {
// zero *norm2 of every active problem (the z-pass descriptors carry the pointers)
__global__ void oz_zero_norms(const oz::Params* __restrict__ prm, int C, const int* __restrict__ act) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < C && act[i] && prm[i].norm2) *prm[i].norm2 = 0.0;
}
}  // namespace

struct OzBatch {
    int count = 0;
    std::vector<tfde_problem*> P;
    std::vector<double*> norm2;
    // work-item starts [6][count + 1]: exact contraction x, y, z (row halves of
    // line tiles); slicing x (lines), y and z (groups of 16 lines)
    long long* d_start = nullptr;
    long long total[6] = {};
    int nmax[3] = {};
    oz::Params* d_prm[OZ_SLICES + 1] = {};   // [3][count] per slice count, built on first use
    double flops[OZ_SLICES + 1][3] = {};      // digit-product flops per axis (all problems)
    SliceDesc* d_sd = nullptr;                // [3][count]
    SliceDesc* h_sd = nullptr;
    int* d_shift = nullptr;
    int* h_shift = nullptr;
    cudaEvent_t copied = nullptr;             // the last upload of h_sd / h_shift has been read
};

namespace {
// the segments of the operator A along each axis (as accurate_apply_ex with op = A)
void batch_segs(const MixedState* M, int axis, OzSegSpec* sg, int* nseg) {
    if (axis == 0) {
        sg[0] = {&M->oz_x_plus, 0};
        *nseg = 1;
    } else if (axis == 1) {
        sg[0] = {&M->oz_y_mass_c, 0};
        sg[1] = {&M->oz_y_plus, 1};
        *nseg = 2;
    } else {
        sg[0] = {&M->oz_z_mass_c, 0};
        sg[1] = {&M->oz_z_plus, 1};
        *nseg = 2;
    }
}

int batch_params(OzBatch* ob, int S) {
    if (ob->d_prm[S]) return TFDE_OK;
    const int C = ob->count;
    std::vector<oz::Params> prm((size_t)3 * C);
    for (int i = 0; i < C; ++i) {
        tfde_problem* P = ob->P[i];
        MixedState* M = mixed(P);
        for (int a = 0; a < 3; ++a) {
            OzSegSpec sg[2];
            int nseg;
            batch_segs(M, a, sg, &nseg);
            double pairs = 0.0;
            oz::Params& q = prm[(size_t)a * C + i];
            if (a == 0)
                oz_params(P, 0, sg, nseg, 1, nullptr, 0.0, P->w[tfde_problem::W_A], S, nullptr, 0, q, &pairs);
            else if (a == 1)
                oz_params(P, 1, sg, nseg, 1, nullptr, 0.0, P->w[tfde_problem::W_C], S, nullptr, 0, q, &pairs);
            else
                oz_params(P, 2, sg, nseg, -1, P->w[tfde_problem::W_B], 1.0, P->w[tfde_problem::W_R], S, ob->norm2[i], 0,
                          q, &pairs);
            if (a == 2) q.norm_shift_dev = ob->d_shift + i;
            ob->flops[S][a] += 2.0 * pairs * P->n[a] * (double)P->N;
        }
    }
    OZ_TRY(cudaMalloc((void**)&ob->d_prm[S], prm.size() * sizeof(oz::Params)));
    OZ_TRY(cudaMemcpy(ob->d_prm[S], prm.data(), prm.size() * sizeof(oz::Params), cudaMemcpyHostToDevice));
    return TFDE_OK;
}

template <int S>
void batch_slice(OzBatch* ob, int axis, const int* d_act, cudaStream_t s) {
    const int C = ob->count;
    const long long* start = ob->d_start + (size_t)(3 + axis) * (C + 1);
    const long long tot = ob->total[3 + axis];
    const SliceDesc* d = ob->d_sd + (size_t)axis * C;
    stats_count_launch();
    if (axis == 0) {
        const long long blocks = std::max<long long>(1, std::min<long long>((tot + 7) / 8, 152LL * 16));
        slice_x_grouped_kernel<S><<<(unsigned)blocks, 256, 0, s>>>(d, start, C, d_act);
        return;
    }
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(slice_staged_grouped_kernel<16, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
        attr = true;
    }
    const size_t smem = (size_t)2 * ob->nmax[axis] * 16 * 8;
    const long long per_sm = std::max<long long>(1, (long long)(220 * 1024 / smem));
    const long long blocks = std::max<long long>(1, std::min<long long>(tot, 152LL * per_sm));
    slice_staged_grouped_kernel<16, S><<<(unsigned)blocks, SL_THREADS, smem, s>>>(d, start, C, d_act);
}

void batch_slice_s(OzBatch* ob, int axis, int S, const int* d_act, cudaStream_t s) {
    switch (S) {
        case 2: batch_slice<2>(ob, axis, d_act, s); break;
        case 3: batch_slice<3>(ob, axis, d_act, s); break;
        case 4: batch_slice<4>(ob, axis, d_act, s); break;
        case 5: batch_slice<5>(ob, axis, d_act, s); break;
        case 6: batch_slice<6>(ob, axis, d_act, s); break;
        default: batch_slice<7>(ob, axis, d_act, s); break;
    }
}

int batch_contract(OzBatch* ob, int axis, int S, const int* act, const int* d_act, cudaStream_t s) {
    const int C = ob->count;
    oz::Params p0;
    std::memset(&p0, 0, sizeof(p0));
    p0.nslices = S;
    p0.b_kmajor = axis == 0 ? 1 : 0;
    p0.ntiles = ob->total[axis];
    p0.mhalves = 1;
    p0.err = mixed(ob->P[0])->err;
    if (int st = oz_set_attrs()) return st;
    double bytes = 0.0;
    for (int i = 0; i < C; ++i)
        if (act[i]) bytes += (2.0 * S * (axis == 0 ? 1 : 2) + 8.0 + (axis == 2 ? 8.0 : 0.0)) * (double)ob->P[i]->N;
    const long long grid = std::max<long long>(1, std::min<long long>(ob->total[axis], tc::num_sms()));
    stats_count_launch();
    void* tok = stats_tc_begin(s, TFDE_KIND_EXACT);
    oz::oz_gemm_kernel<true><<<(unsigned)grid, oz::NUM_THREADS, oz::SMEM_BYTES, s>>>(
        p0, ob->d_prm[S] + (size_t)axis * C, ob->d_start + (size_t)axis * (C + 1), C, d_act);
    const cudaError_t e = cudaGetLastError();
    stats_tc_end(tok, s, TFDE_KIND_EXACT, bytes, ob->flops[S][axis]);
    if (e != cudaSuccess) return set_error(TFDE_ECUDA, std::string("grouped oz_gemm_kernel launch: ") + cudaGetErrorString(e));
    return TFDE_OK;
}
}  // namespace

int oz_batch_create(tfde_problem* const* P, int count, double* const* norm2, OzBatch** out) {
    *out = nullptr;
    OzBatch* ob = new OzBatch();
    ob->count = count;
    ob->P.assign(P, P + count);
    ob->norm2.assign(norm2, norm2 + count);
    std::vector<long long> start((size_t)6 * (count + 1), 0);
    for (int i = 0; i < count; ++i) {
        const tfde_problem* Pi = P[i];
        const long long n1 = Pi->n[0], n2 = Pi->n[1], n3 = Pi->n[2];
        long long w[6];
        for (int a = 0; a < 3; ++a) {
            const long long n = Pi->n[a];
            const long long mh = (n + oz::BM - 1) / oz::BM;
            long long tiles;
            if (a == 0) tiles = (n2 * n3 + oz::BN - 1) / oz::BN;
            else if (a == 1) tiles = ((n1 + oz::BN - 1) / oz::BN) * n3;
            else tiles = (n1 * n2 + oz::BN - 1) / oz::BN;
            w[a] = tiles * mh;
            ob->nmax[a] = std::max(ob->nmax[a], (int)n);
        }
        w[3] = n2 * n3;                    // x lines
        w[4] = (n1 * n3 + 15) / 16;        // y groups of 16 lines
        w[5] = (n1 * n2 + 15) / 16;        // z groups of 16 lines
        for (int k = 0; k < 6; ++k) start[(size_t)k * (count + 1) + i + 1] = start[(size_t)k * (count + 1) + i] + w[k];
    }
    for (int k = 0; k < 6; ++k) ob->total[k] = start[(size_t)k * (count + 1) + count];
    auto fail = [&](const char* what) {
        oz_batch_destroy(ob);
        return set_error(TFDE_ENOMEM, what);
    };
    if (cudaMalloc((void**)&ob->d_start, start.size() * sizeof(long long)) != cudaSuccess ||
        cudaMalloc((void**)&ob->d_sd, (size_t)3 * count * sizeof(SliceDesc)) != cudaSuccess ||
        cudaMallocHost((void**)&ob->h_sd, (size_t)3 * count * sizeof(SliceDesc)) != cudaSuccess ||
        cudaMalloc((void**)&ob->d_shift, count * sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&ob->h_shift, count * sizeof(int)) != cudaSuccess ||
        cudaEventCreateWithFlags(&ob->copied, cudaEventDisableTiming) != cudaSuccess)
        return fail("allocation of the batched exact-residual tables failed");
    if (cudaMemcpy(ob->d_start, start.data(), start.size() * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail("upload of the batched exact-residual tables failed");
    *out = ob;
    return TFDE_OK;
}

void oz_batch_destroy(OzBatch* ob) {
    if (!ob) return;
    cudaFree(ob->d_start);
    for (auto* d : ob->d_prm) cudaFree(d);
    cudaFree(ob->d_sd);
    if (ob->h_sd) cudaFreeHost(ob->h_sd);
    cudaFree(ob->d_shift);
    if (ob->h_shift) cudaFreeHost(ob->h_shift);
    if (ob->copied) cudaEventDestroy(ob->copied);
    delete ob;
}

int oz_batch_residual(OzBatch* ob, const double* const* x, const int* act, const int* d_act, const int* shift, int S,
                      cudaStream_t s) {
    if (S < 2 || S > OZ_SLICES) S = OZ_SLICES;
    const int C = ob->count;
    bool any = false;
    for (int i = 0; i < C; ++i) any = any || act[i];
    if (!any) return TFDE_OK;
    if (int st = batch_params(ob, S)) return st;
    OZ_TRY(cudaEventSynchronize(ob->copied));   // the previous call's upload has been read
    for (int i = 0; i < C; ++i) {
        tfde_problem* P = ob->P[i];
        MixedState* M = mixed(P);
        double* const* w = P->w;
        const long long N = (long long)P->N;
        SliceDesc* d = ob->h_sd;
        d[i] = SliceDesc{x[i], nullptr, 0, P->n[0], axis_view(P->n, 0), M->oz_planes[0], M->oz_planes[1], N,
                         M->oz_lexp, w[tfde_problem::W_W]};
        d[C + i] = SliceDesc{w[tfde_problem::W_A], w[tfde_problem::W_W], M->oz_shift[1], P->n[0], axis_view(P->n, 1),
                             M->oz_planes[0], M->oz_planes[1], N, M->oz_lexp, w[tfde_problem::W_E]};
        d[2 * C + i] = SliceDesc{w[tfde_problem::W_C], w[tfde_problem::W_E], M->oz_shift[2], P->n[0],
                                 axis_view(P->n, 2), M->oz_planes[0], M->oz_planes[1], N, M->oz_lexp,
                                 w[tfde_problem::W_T]};
        ob->h_shift[i] = shift[i];
    }
    OZ_TRY(cudaMemcpyAsync(ob->d_sd, ob->h_sd, (size_t)3 * C * sizeof(SliceDesc), cudaMemcpyHostToDevice, s));
    OZ_TRY(cudaMemcpyAsync(ob->d_shift, ob->h_shift, C * sizeof(int), cudaMemcpyHostToDevice, s));
    OZ_TRY(cudaEventRecord(ob->copied, s));
    int st;
    // x pass: a = (A1 + G1) x, w = A1 x; y pass: c = A2 a + G2 w, e = A2 w;
    // z pass: r = b - (A3 c + G3 e), A_N x = A3 e
    batch_slice_s(ob, 0, S, d_act, s);
    if ((st = batch_contract(ob, 0, S, act, d_act, s))) return st;
    batch_slice_s(ob, 1, S, d_act, s);
    if ((st = batch_contract(ob, 1, S, act, d_act, s))) return st;
    batch_slice_s(ob, 2, S, d_act, s);
    stats_count_launch();
    oz_zero_norms<<<(C + 63) / 64, 64, 0, s>>>(ob->d_prm[S] + (size_t)2 * C, C, d_act);
    return batch_contract(ob, 2, S, act, d_act, s);
}

}  // namespace tfde
