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
// bits alone (|x| < 2^E): the mantissa shifted right with round-half-up.
__device__ __forceinline__ long long fixed_point(long long bits, int S, int E) {
    const unsigned long long u = (unsigned long long)bits & 0x7FFFFFFFFFFFFFFFull;
    if (u == 0) return 0;
    int e = (int)(u >> 52);
    unsigned long long mant = u & ((1ull << 52) - 1);
    if (e == 0) e = 1; else mant |= (1ull << 52);
    const int r = 1075 - e - 7 * S + E;   // right shift; >= 53 - 7S >= 4 for S <= 7
    long long X;
    if (r >= 64) X = 0;
    else if (r <= 0) X = (long long)(mant << (-r));
    else X = (long long)((mant + (1ull << (r - 1))) >> r);
    return bits < 0 ? -X : X;
}

// Exponent E with |x| < 2^E for the largest |x| of a line (given as the
// biased-exponent field of its bit pattern; 0 for an all-zero line).
__device__ __forceinline__ int line_exponent_from_bits(unsigned long long umax) {
    if (umax == 0) return 0;
    const int e = (int)(umax >> 52);
    return e == 0 ? -1021 : e - 1022;
}

// balanced base-128 digits of X (|X| <= 2^{7S}): planes[t*N + idx] for t = S-1..1 in
// [-64, 63], planes[idx] the remaining leading digit
__device__ __forceinline__ void write_digits(long long X, int S, __nv_bfloat16* planes, long long N, long long idx) {
    for (int t = S - 1; t >= 1; --t) {
        long long r = X & 127;
        if (r >= 64) r -= 128;
        planes[(long long)t * N + idx] = __float2bfloat16_rn((float)r);
        X = (X - r) >> 7;
    }
    planes[idx] = __float2bfloat16_rn((float)X);
}

// |x| bits of x * 2^sh for a normal or zero x (exponent field moved by sh)
__device__ __forceinline__ unsigned long long abs_bits_shifted(long long bits, int sh) {
    const unsigned long long u = (unsigned long long)bits & 0x7FFFFFFFFFFFFFFFull;
    return u == 0 ? 0 : u + ((unsigned long long)(long long)sh << 52);
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

// x axis: one warp per line of n1 contiguous values.  Writes the digit planes
// of x under its line maximum and, when wout is set, w = A_{n1} x along the
// line from the same fixed-point integers X (w_k = (X_{k-1} + 6 X_k +
// X_{k+1}) 2^{E - 7S - 3}, |sum| < 2^53: exact).
__global__ void slice_x_kernel(const double* __restrict__ x0, int n1, long long lines, int S,
                               __nv_bfloat16* __restrict__ p0, long long N, int* __restrict__ lexp,
                               double* __restrict__ wout) {
    const int lane = threadIdx.x & 31;
    const long long wg = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long l = wg; l < lines; l += nw) {
        const long long* r0 = reinterpret_cast<const long long*>(x0 + l * n1);
        unsigned long long umax = 0;
#pragma unroll 4
        for (int k = lane; k < n1; k += 32) umax = max(umax, (unsigned long long)r0[k] & 0x7FFFFFFFFFFFFFFFull);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) umax = max(umax, __shfl_xor_sync(0xffffffffu, umax, o));
        const int E = line_exponent_from_bits(umax);
        long long left_carry = 0;   // X_{base - 1}
        long long Xc = lane < n1 ? fixed_point(r0[lane], S, E) : 0;
        for (int base = 0; base < n1; base += 32) {
            const int k = base + lane;
            const int kn = k + 32;
            const long long Xn = kn < n1 ? fixed_point(r0[kn], S, E) : 0;
            if (k < n1) write_digits(Xc, S, p0, N, l * n1 + k);
            if (wout) {
                long long left = __shfl_up_sync(0xffffffffu, Xc, 1);
                long long right = __shfl_down_sync(0xffffffffu, Xc, 1);
                const long long first_next = __shfl_sync(0xffffffffu, Xn, 0);
                if (lane == 0) left = left_carry;
                if (lane == 31) right = first_next;
                if (k < n1) wout[l * n1 + k] = i64_ldexp_exact(left + 6 * Xc + right, E - 7 * S - 3);
                left_carry = __shfl_sync(0xffffffffu, Xc, 31);
            }
            Xc = Xn;
        }
        if (lane == 0) lexp[l] = E;
    }
}

// y / z axes: LB consecutive lines (contiguous in memory) per 512-thread
// block.  The block's lines of both inputs are copied once into shared memory
// (8-byte cp.async, all in flight together), the joint line maximum of x0 and
// x1 * 2^sh1 is reduced there, and the digits are written from shared memory:
// every input element crosses HBM once.  When eout is set, e = A_n x1 along
// the line from the fixed-point integers W of x1 (exact as in slice_x_kernel).
constexpr int SL_THREADS = 512;

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

template <int LB>
__global__ __launch_bounds__(SL_THREADS) void slice_staged_kernel(const double* __restrict__ x0,
                                                                  const double* __restrict__ x1, int sh1, AxisView v,
                                                                  int S, __nv_bfloat16* __restrict__ p0,
                                                                  __nv_bfloat16* __restrict__ p1, long long N,
                                                                  int* __restrict__ lexp, double* __restrict__ eout) {
    constexpr int NKG = SL_THREADS / LB;
    extern __shared__ unsigned long long sl_smem[];   // [input][k][LB]
    __shared__ unsigned long long smax[NKG][LB];
    __shared__ int sexp[LB];
    unsigned long long* s0 = sl_smem;
    unsigned long long* s1 = sl_smem + (size_t)v.n * LB;
    const int li = threadIdx.x % LB, kg = threadIdx.x / LB;
    const long long* b0 = reinterpret_cast<const long long*>(x0);
    const long long* b1 = reinterpret_cast<const long long*>(x1);
    for (long long l0 = (long long)blockIdx.x * LB; l0 < v.lines; l0 += (long long)gridDim.x * LB) {
        const long long l = l0 + li;
        const bool valid = l < v.lines;
        const long long off = valid ? (l % v.l_in) * v.s_in + (l / v.l_in) * v.s_out : 0;
        if (valid) {
            for (int k = kg; k < v.n; k += NKG) {
                const long long idx = off + (long long)k * v.stride;
                cp_async8(s0 + k * LB + li, b0 + idx);
                if (b1) cp_async8(s1 + k * LB + li, b1 + idx);
            }
        }
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        unsigned long long umax = 0;
        if (valid) {
            for (int k = kg; k < v.n; k += NKG) {
                umax = max(umax, s0[k * LB + li] & 0x7FFFFFFFFFFFFFFFull);
                if (b1) umax = max(umax, abs_bits_shifted((long long)s1[k * LB + li], sh1));
            }
        }
        smax[kg][li] = umax;
        __syncthreads();
        if (kg == 0) {
            unsigned long long m = smax[0][li];
#pragma unroll 8
            for (int g = 1; g < NKG; ++g) m = max(m, smax[g][li]);
            const int E = line_exponent_from_bits(m);
            sexp[li] = E;
            if (valid) lexp[l] = E;
        }
        __syncthreads();
        const int E = sexp[li];
        const int E1 = E - sh1;
        if (valid) {
            for (int k = kg; k < v.n; k += NKG) {
                const long long idx = off + (long long)k * v.stride;
                write_digits(fixed_point((long long)s0[k * LB + li], S, E), S, p0, N, idx);
                if (b1) {
                    const long long W = fixed_point((long long)s1[k * LB + li], S, E1);
                    write_digits(W, S, p1, N, idx);
                    if (eout) s1[k * LB + li] = (unsigned long long)W;
                }
            }
        }
        if (eout && b1) {
            __syncthreads();
            if (valid) {
                for (int k = kg; k < v.n; k += NKG) {
                    const long long Wp = k > 0 ? (long long)s1[(k - 1) * LB + li] : 0;
                    const long long Wn = k + 1 < v.n ? (long long)s1[(k + 1) * LB + li] : 0;
                    const long long W = (long long)s1[k * LB + li];
                    eout[off + (long long)k * v.stride] = i64_ldexp_exact(Wp + 6 * W + Wn, E1 - 7 * S - 3);
                }
            }
        }
        __syncthreads();
    }
}

int grid_for(long long n) {
    long long g = (n + 255) / 256;
    if (g > 152LL * 16) g = 152LL * 16;
    return (int)(g < 1 ? 1 : g);
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
bool g_sl_attr[2] = {false, false};

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
                st = (a == 0) ? tc::make_map_B_box(&M->oz_bmap[in][t][a], base, P->n, a, oz::BN)
                              : tc::make_map_B(&M->oz_bmap[in][t][a], base, P->n, a);
                if (st) return st;
                // slices 0..t of input `in` along axis a in one box
                const cuuint64_t n1 = P->n[0], n2 = P->n[1], n3 = P->n[2];
                int es;
                if (a == 0) {
                    const cuuint64_t dims[3] = {n1, n2 * n3, (cuuint64_t)S};
                    const cuuint64_t strides[2] = {n1 * 2, (cuuint64_t)N * 2};
                    const cuuint32_t box[3] = {(cuuint32_t)tc::BK, (cuuint32_t)oz::BN, (cuuint32_t)(t + 1)};
                    es = tc::encode_map(&M->oz_bmapm[in][a][t], M->oz_planes[in], 3, dims, strides, box,
                                        CU_TENSOR_MAP_SWIZZLE_64B);
                } else if (a == 1) {
                    const cuuint64_t dims[4] = {n1, n2, n3, (cuuint64_t)S};
                    const cuuint64_t strides[3] = {n1 * 2, n1 * n2 * 2, (cuuint64_t)N * 2};
                    const cuuint32_t box[4] = {64, (cuuint32_t)tc::BK, 1, (cuuint32_t)(t + 1)};
                    es = tc::encode_map(&M->oz_bmapm[in][a][t], M->oz_planes[in], 4, dims, strides, box,
                                        CU_TENSOR_MAP_SWIZZLE_128B);
                } else {
                    const cuuint64_t dims[3] = {n1 * n2, n3, (cuuint64_t)S};
                    const cuuint64_t strides[2] = {n1 * n2 * 2, (cuuint64_t)N * 2};
                    const cuuint32_t box[3] = {64, (cuuint32_t)tc::BK, (cuuint32_t)(t + 1)};
                    es = tc::encode_map(&M->oz_bmapm[in][a][t], M->oz_planes[in], 3, dims, strides, box,
                                        CU_TENSOR_MAP_SWIZZLE_128B);
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

// Slice one or two FP64 inputs along `axis` into the digit planes 0 / 1, the
// second one taken as x1 * 2^sh1; mass_out (optional) receives the mass
// operator along `axis` applied to x1 (x0 on the x axis), exactly from the
// fixed-point integers.
void oz_slice(const tfde_problem* P, int axis, const double* x0, const double* x1, int sh1, double* mass_out,
              int S, cudaStream_t s) {
    MixedState* M = mixed(P);
    const AxisView v = axis_view(P->n, axis);
    const long long N = (long long)P->N;
    stats_count_launch();
    if (axis == 0) {
        slice_x_kernel<<<grid_for(v.lines * 32), 256, 0, s>>>(x0, P->n[0], v.lines, S, M->oz_planes[0], N,
                                                               M->oz_lexp, mass_out);
    } else {
        // 32 lines per block while both inputs fit in 200 KB of shared memory, else 16
        const int nin = x1 ? 2 : 1;
        const bool wide = (size_t)nin * v.n * 32 * 8 <= 200 * 1024;
        const int LB = wide ? 32 : 16;
        const size_t smem = (size_t)nin * v.n * LB * 8;
        long long blocks = (v.lines + LB - 1) / LB;
        const long long per_sm = std::max<long long>(1, (long long)(220 * 1024 / std::max<size_t>(smem, 1)));
        if (blocks > 152LL * per_sm) blocks = 152LL * per_sm;
        if (wide) {
            if (!g_sl_attr[0]) {
                cudaFuncSetAttribute(slice_staged_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
                g_sl_attr[0] = true;
            }
            slice_staged_kernel<32><<<(unsigned)blocks, SL_THREADS, smem, s>>>(x0, x1, sh1, v, S, M->oz_planes[0],
                                                                             M->oz_planes[1], N, M->oz_lexp, mass_out);
        } else {
            if (!g_sl_attr[1]) {
                cudaFuncSetAttribute(slice_staged_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
                g_sl_attr[1] = true;
            }
            slice_staged_kernel<16><<<(unsigned)blocks, SL_THREADS, smem, s>>>(x0, x1, sh1, v, S, M->oz_planes[0],
                                                                             M->oz_planes[1], N, M->oz_lexp, mass_out);
        }
    }
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
        prm.nbc = (prm.C + 63) / 64;
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
                      double asign, cudaStream_t s, int slices, double* norm2, int norm_shift) {
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
    // z pass: y = A3 c +- G3 e
    oz_slice(P, 2, tc_, te, M->oz_shift[2], nullptr, slices, s);
    OzSegSpec sy[2] = {{&M->oz_z_mass_c, 0}, {rhs ? &M->oz_z_minus : &M->oz_z_plus, 1}};
    if (norm2) OZ_TRY(cudaMemsetAsync(norm2, 0, sizeof(double), s));
    return oz_contract(P, 2, sy, 2, vsign, addend, asign, y, slices, s, norm2, norm_shift);
}

int accurate_apply(const tfde_problem* P, int op, const double* x, double* y, cudaStream_t s) {
    return accurate_apply_ex(P, op, x, y, 1, nullptr, 0.0, s);
}

}  // namespace tfde
