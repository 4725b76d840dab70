// FP64-accurate operator application for the mixed path (Eq. (linear_sys)):
//
//   A x = A_N x +- [M3 M2 G1 + M3 G2 M1 + G3 M2 M1] x,   G_a = eta_a B_a,
//
// evaluated as  y1 = M1 x;  a = y1 +- G1 x;  c = M2 a +- G2 y1;
//               y  = M3 c +- G3 (M2 y1)
// with the three dense contractions on the tensor cores in exact-integer
// digit slices (tfde_oz_kernel.cuh) and the tridiagonal mass sweeps in FP64.
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

constexpr int kT = 256;

__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// exponent E with |v| < 2^E for the line maximum v (0 for an all-zero line),
// clamped so that the fixed-point scale 2^{7S - E} stays a normal double
__device__ __forceinline__ int line_exponent(double vmax) {
    if (!(vmax > 0.0)) return 0;
    int e;
    frexp(vmax, &e);
    return e < -960 ? -960 : (e > 1000 ? 1000 : e);
}

// balanced base-128 digits of X (|X| < 2^{7S}): d[S-1..1] in [-64, 63], d[0] the rest
__device__ __forceinline__ void write_digits(long long X, int S, __nv_bfloat16* planes, long long N, long long idx) {
    for (int t = S - 1; t >= 1; --t) {
        long long r = X & 127;
        if (r >= 64) r -= 128;
        planes[(long long)t * N + idx] = __float2bfloat16_rn((float)r);
        X = (X - r) >> 7;
    }
    planes[idx] = __float2bfloat16_rn((float)X);
}

// x axis: one warp per line of n1 contiguous values
__global__ void slice_x_kernel(const double* __restrict__ x, int n1, long long lines, int S,
                               __nv_bfloat16* __restrict__ planes, long long N, int* __restrict__ lexp) {
    const int lane = threadIdx.x & 31;
    const long long warp_global = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long l = warp_global; l < lines; l += nwarps) {
        const double* row = x + l * n1;
        double vmax = 0.0;
        for (int k = lane; k < n1; k += 32) vmax = fmax(vmax, fabs(row[k]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        const int E = line_exponent(vmax);
        const double sc = pow2d(7 * S - E);
        for (int k = lane; k < n1; k += 32) write_digits(__double2ll_rn(row[k] * sc), S, planes, N, l * n1 + k);
        if (lane == 0) lexp[l] = E;
    }
}

// y / z axes: one thread per line (consecutive lines are contiguous in memory)
__global__ void slice_strided_kernel(const double* __restrict__ x, AxisView v, int S,
                                     __nv_bfloat16* __restrict__ planes, long long N, int* __restrict__ lexp) {
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < v.lines;
         l += (long long)gridDim.x * blockDim.x) {
        const long long off = (l % v.l_in) * v.s_in + (l / v.l_in) * v.s_out;
        double vmax = 0.0;
        for (int k = 0; k < v.n; ++k) vmax = fmax(vmax, fabs(x[off + (long long)k * v.stride]));
        const int E = line_exponent(vmax);
        const double sc = pow2d(7 * S - E);
        for (int k = 0; k < v.n; ++k) {
            const long long idx = off + (long long)k * v.stride;
            write_digits(__double2ll_rn(x[idx] * sc), S, planes, N, idx);
        }
        lexp[l] = E;
    }
}

int grid_for(long long n) {
    long long g = (n + kT - 1) / kT;
    if (g > 152LL * 16) g = 152LL * 16;
    return (int)(g < 1 ? 1 : g);
}

// Host: digit slices of an n x n operator (row-major) and its row exponents.
void slice_operator_host(const std::vector<double>& G, int n, int S, std::vector<__nv_bfloat16>& slices,
                         std::vector<int>& rexp) {
    slices.assign((size_t)S * n * n, __float2bfloat16_rn(0.f));
    rexp.assign(n, 0);
    for (int m = 0; m < n; ++m) {
        double vmax = 0.0;
        for (int k = 0; k < n; ++k) vmax = std::fmax(vmax, std::fabs(G[(size_t)m * n + k]));
        int E = 0;
        if (vmax > 0.0) std::frexp(vmax, &E);
        rexp[m] = E;
        for (int k = 0; k < n; ++k) {
            long long X = std::llrint(std::ldexp(G[(size_t)m * n + k], 7 * S - E));
            for (int t = S - 1; t >= 1; --t) {
                long long r = X & 127;
                if (r >= 64) r -= 128;
                slices[(size_t)t * n * n + (size_t)m * n + k] = __float2bfloat16_rn((float)r);
                X = (X - r) >> 7;
            }
            slices[(size_t)m * n + k] = __float2bfloat16_rn((float)X);
        }
    }
}

#define OZ_TRY(expr)                                                                       \
    do {                                                                                   \
        cudaError_t e__ = (expr);                                                          \
        if (e__ != cudaSuccess)                                                            \
            return set_error(TFDE_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e__)); \
    } while (0)

bool g_oz_attr = false;

}  // namespace

int oz_init(tfde_problem* P, const std::vector<double> etaB[3], cudaStream_t s) {
    MixedState* M = mixed(P);
    const int S = OZ_SLICES;
    const size_t N = P->N;
    for (int a = 0; a < 3; ++a) {
        const int n = P->n[a];
        std::vector<__nv_bfloat16> sl;
        std::vector<int> rexp;
        slice_operator_host(etaB[a], n, S, sl, rexp);
        OZ_TRY(cudaMalloc((void**)&M->oz_op[a], sl.size() * sizeof(__nv_bfloat16)));
        OZ_TRY(cudaMemcpyAsync(M->oz_op[a], sl.data(), sl.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice, s));
        OZ_TRY(cudaMalloc((void**)&M->oz_rexp[a], n * sizeof(int)));
        OZ_TRY(cudaMemcpyAsync(M->oz_rexp[a], rexp.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
        OZ_TRY(cudaStreamSynchronize(s));
        for (int t = 0; t < S; ++t) {
            int st = tc::make_map_A(&M->oz_amap[a][t], M->oz_op[a] + (size_t)t * n * n, n);
            if (st) return st;
        }
    }
    OZ_TRY(cudaMalloc((void**)&M->oz_planes, (size_t)S * N * sizeof(__nv_bfloat16)));
    long long maxlines = 0;
    for (int a = 0; a < 3; ++a) maxlines = std::max(maxlines, (long long)(N / P->n[a]));
    OZ_TRY(cudaMalloc((void**)&M->oz_lexp, maxlines * sizeof(int)));
    for (int t = 0; t < S; ++t)
        for (int a = 0; a < 3; ++a) {
            const __nv_bfloat16* base = M->oz_planes + (size_t)t * N;
            int st;
            if (a == 0) {
                // x axis: 64-line boxes
                CUtensorMap* m = &M->oz_bmap[t][a];
                st = tc::make_map_B_box(m, base, P->n, a, oz::BN);
            } else {
                st = tc::make_map_B(&M->oz_bmap[t][a], base, P->n, a);
            }
            if (st) return st;
        }
    return TFDE_OK;
}

void oz_free(MixedState* M) {
    for (int a = 0; a < 3; ++a) {
        cudaFree(M->oz_op[a]);
        cudaFree(M->oz_rexp[a]);
    }
    cudaFree(M->oz_planes);
    cudaFree(M->oz_lexp);
}

// out = sign * (G_axis x) + addend, G_axis = eta_a B_a, x sliced along `axis`.
int oz_contract(const tfde_problem* P, int axis, const double* x, double sign, const double* addend, double* out,
                cudaStream_t s) {
    MixedState* M = mixed(P);
    const int S = OZ_SLICES;
    const AxisView v = axis_view(P->n, axis);
    const long long N = (long long)P->N;
    if (axis == 0) {
        stats_count_launch();
        slice_x_kernel<<<grid_for(v.lines * 32), kT, 0, s>>>(x, P->n[0], v.lines, S, M->oz_planes, N, M->oz_lexp);
    } else {
        stats_count_launch();
        slice_strided_kernel<<<grid_for(v.lines), kT, 0, s>>>(x, v, S, M->oz_planes, N, M->oz_lexp);
    }
    oz::Params prm;
    std::memset(&prm, 0, sizeof(prm));
    for (int t = 0; t < S; ++t) {
        prm.amaps[t] = M->oz_amap[axis][t];
        prm.bmaps[t] = M->oz_bmap[t][axis];
    }
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
        if (axis == 1) { prm.C = (int)n1; prm.P = (int)n3; }
        else { prm.C = (int)(n1 * n2); prm.P = 1; }
        prm.nbc = (prm.C + 63) / 64;
        prm.nblocks = (long long)prm.nbc * prm.P;
        prm.ntiles = prm.nblocks;
        prm.lines = (long long)prm.C * prm.P;
        prm.plane = (long long)prm.C * prm.n;
    }
    prm.row_exp = M->oz_rexp[axis];
    prm.line_exp = M->oz_lexp;
    prm.sign = sign;
    prm.addend = addend;
    prm.out = out;
    prm.err = M->err;
    if (!g_oz_attr) {
        OZ_TRY(cudaFuncSetAttribute(oz::oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, oz::SMEM_BYTES));
        g_oz_attr = true;
    }
    const long long total = prm.ntiles * prm.mhalves;
    long long grid = total < tc::num_sms() ? total : tc::num_sms();
    void* tok = stats_tc_begin(s);
    oz::oz_gemm_kernel<<<(unsigned)(grid < 1 ? 1 : grid), oz::NUM_THREADS, oz::SMEM_BYTES, s>>>(prm);
    cudaError_t e = cudaGetLastError();
    // algorithmic bytes: digit slices read + FP64 out (+ addend) ; flops: every digit pair
    const double na = prm.n, pairs = S * (S + 1) / 2;
    stats_tc_end(tok, s, (2.0 * S + 8.0 + (addend ? 8.0 : 0.0)) * N + 2.0 * S * na * na, 2.0 * pairs * na * N);
    if (e != cudaSuccess) return set_error(TFDE_ECUDA, std::string("oz_gemm_kernel launch: ") + cudaGetErrorString(e));
    return TFDE_OK;
}

// y = A x (op A) or (2 A_N - A) x (op RHS), FP64-accurate.
int accurate_apply(const tfde_problem* P, int op, const double* x, double* y, cudaStream_t s) {
    const double sg = (op & 1) ? -1.0 : 1.0;
    const AxisView vx = axis_view(P->n, 0), vy = axis_view(P->n, 1), vz = axis_view(P->n, 2);
    double* t0 = P->w[tfde_problem::W_W];  // y1 = M1 x
    double* t1 = P->w[tfde_problem::W_A];  // a, later y2
    double* t2 = P->w[tfde_problem::W_C];  // M2 a, later M3 c
    double* t3 = P->w[tfde_problem::W_E];  // c
    int st;
    launch_axis_stencil_f64(x, t0, vx, 1.0, nullptr, 0.0, s);
    if ((st = oz_contract(P, 0, x, sg, t0, t1, s))) return st;          // a = y1 +- G1 x
    launch_axis_stencil_f64(t1, t2, vy, 1.0, nullptr, 0.0, s);           // M2 a
    if ((st = oz_contract(P, 1, t0, sg, t2, t3, s))) return st;         // c = M2 a +- G2 y1
    launch_axis_stencil_f64(t0, t1, vy, 1.0, nullptr, 0.0, s);           // y2 = M2 y1
    launch_axis_stencil_f64(t3, t2, vz, 1.0, nullptr, 0.0, s);           // M3 c
    return oz_contract(P, 2, t1, sg, t2, y, s);                           // y = M3 c +- G3 y2
}

}  // namespace tfde
