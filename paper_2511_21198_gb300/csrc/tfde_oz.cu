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
__global__ void slice_x_kernel(const double* __restrict__ x0, int n1, long long lines,
                               __nv_bfloat16* __restrict__ p0, long long N, int* __restrict__ lexp,
                               double* __restrict__ wout) {
    const int lane = threadIdx.x & 31;
    const long long wg = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long l = wg; l < lines; l += nw) {
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

template <int LB, int S>
__global__ __launch_bounds__(SL_THREADS) void slice_staged_kernel(const double* __restrict__ x0,
                                                                  const double* __restrict__ x1, int sh1, AxisView v,
                                                                  __nv_bfloat16* __restrict__ p0,
                                                                  __nv_bfloat16* __restrict__ p1, long long N,
                                                                  int* __restrict__ lexp, double* __restrict__ eout) {
    constexpr int LP = LB / 2;               // line pairs per block
    constexpr int NKG = SL_THREADS / LP;     // k rows in flight
    extern __shared__ unsigned long long sl_smem[];   // [input][k][LB]
    __shared__ uint32_t shmax[NKG][LB];
    __shared__ uint32_t slor[NKG][LB];
    __shared__ int sexp[LB];
    unsigned long long* s0 = sl_smem;
    unsigned long long* s1 = sl_smem + (size_t)v.n * LB;
    const int lp = threadIdx.x % LP, kg = threadIdx.x / LP;
    const int la = 2 * lp;                   // first line of the pair within the block
    const long long* b0 = reinterpret_cast<const long long*>(x0);
    const long long* b1 = reinterpret_cast<const long long*>(x1);
    for (long long l0 = (long long)blockIdx.x * LB; l0 < v.lines; l0 += (long long)gridDim.x * LB) {
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

int oz_contract(const tfde_problem* P, int axis, const OzSegSpec* segs, int nseg, int vsign, const double* addend,
                double asign, double* out, int S, cudaStream_t s, double* norm2 = nullptr, int norm_shift = 0) {
    MixedState* M = mixed(P);
    const long long N = (long long)P->N;
    oz::Params prm;
    std::memset(&prm, 0, sizeof(prm));
    double pairs = 0.0;
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
        for (int sa = 0; sa < G.na; ++sa) pairs += S - sa;
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
    if (!g_oz_attr) {
        OZ_TRY(cudaFuncSetAttribute(oz::oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, oz::SMEM_BYTES));
        g_oz_attr = true;
    }
    const long long total = prm.ntiles * prm.mhalves;
    long long grid = total < tc::num_sms() ? total : tc::num_sms();
    void* tok = stats_tc_begin(s, TFDE_KIND_EXACT);
    oz::oz_gemm_kernel<<<(unsigned)(grid < 1 ? 1 : grid), oz::NUM_THREADS, oz::SMEM_BYTES, s>>>(prm);
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

}  // namespace tfde
