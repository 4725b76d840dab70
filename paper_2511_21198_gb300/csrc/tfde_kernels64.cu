// FP64 kernels of libtfde: the per-axis dense contraction and tridiagonal mass
// stencil used by the plain-FP64 operator (Eq. (linear_sys)) and DST-I
// preconditioner (Eq. (diag_tau_pre)), and the Krylov vector kernels and
// deterministic reductions shared by both precisions.
#include "tfde_internal.h"
#include "tfde_pow2conv.cuh"
#include "tfde_chain.cuh"
#include "tfde_stats.h"

namespace tfde {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ long long line_offset(const AxisView& v, long long l) {
    return (l % v.l_in) * v.s_in + (l / v.l_in) * v.s_out;
}

// (tridiag(1,6,1)/8 along the axis) Z at position (idx, m): zero exterior data.
__device__ __forceinline__ double mass_stencil(const double* __restrict__ Z, long long idx, int m,
                                               const AxisView& v) {
    double s = 0.75 * Z[idx];
    double nb = 0.0;
    if (m > 0) nb += Z[idx - v.stride];
    if (m + 1 < v.n) nb += Z[idx + v.stride];
    return s + 0.125 * nb;
}

// Tiled FP64 contraction along one axis: each CTA computes a 64 (axis rows)
// x 64 (lines) tile, K in steps of 16, 4x4 outputs per thread.
constexpr int BM = 64, BN = 64, BK = 16;

__global__ __launch_bounds__(kThreads) void axis_gemm_f64_kernel(
    const double* __restrict__ Mat, const double* __restrict__ X, double* __restrict__ Y, AxisView v,
    double alpha, const double* __restrict__ Z, double beta) {
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * BM;
    const long long l0 = (long long)blockIdx.x * BN;
    double acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;

    for (int k0 = 0; k0 < v.n; k0 += BK) {
        for (int e = tid; e < BM * BK; e += kThreads) {
            const int mm = e / BK, kk = e % BK;
            const int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < v.n && gk < v.n) ? Mat[(size_t)gm * v.n + gk] : 0.0;
        }
        if (v.stride == 1) {  // lines are contiguous along k: walk k fastest
            for (int e = tid; e < BN * BK; e += kThreads) {
                const int ll = e / BK, kk = e % BK;
                const long long l = l0 + ll;
                const int gk = k0 + kk;
                Bs[kk][ll] = (l < v.lines && gk < v.n) ? X[line_offset(v, l) + gk] : 0.0;
            }
        } else {              // consecutive lines are contiguous: walk lines fastest
            for (int e = tid; e < BN * BK; e += kThreads) {
                const int kk = e / BN, ll = e % BN;
                const long long l = l0 + ll;
                const int gk = k0 + kk;
                Bs[kk][ll] = (l < v.lines && gk < v.n) ? X[line_offset(v, l) + (long long)gk * v.stride] : 0.0;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int gm = m0 + ty + 16 * r;
        if (gm >= v.n) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const long long l = l0 + tx + 16 * c;
            if (l >= v.lines) continue;
            const long long idx = line_offset(v, l) + (long long)gm * v.stride;
            double val = alpha * acc[r][c];
            if (Z) val += beta * mass_stencil(Z, idx, gm, v);
            Y[idx] = val;
        }
    }
}

// Y = beta (tridiag(1,6,1)/8 along the axis) X + gamma W on a 3-D grid; one
// thread per element of an (i, j, k) block, neighbours along the axis.
__global__ void axis_stencil_f64_kernel(const double* __restrict__ X, double* __restrict__ Y, int n1, int n2,
                                        int n3, int axis, double beta, const double* __restrict__ W,
                                        double gamma) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n1) return;
    // j and k both stride over the grid: gridDim.y is capped at 65535, and on
    // the x axis n2 counts every line (n2 n3 of the grid)
    for (long long j = (long long)blockIdx.y * blockDim.y + threadIdx.y; j < n2; j += (long long)gridDim.y * blockDim.y)
        for (int k = blockIdx.z; k < n3; k += gridDim.z) {
            const long long idx = ((long long)k * n2 + j) * n1 + i;
            long long st;
            long long m, n;
            if (axis == 0) { st = 1; m = i; n = n1; }
            else if (axis == 1) { st = n1; m = j; n = n2; }
            else { st = (long long)n1 * n2; m = k; n = n3; }
            double nb = 0.0;
            if (m > 0) nb += X[idx - st];
            if (m + 1 < n) nb += X[idx + st];
            double val = beta * fma(0.75, X[idx], 0.125 * nb);
            if (W) val = fma(gamma, W[idx], val);
            Y[idx] = val;
        }
}

// Y = (T_{n3} (x) T_{n2} (x) T_{n1}) X, T = tridiag(1,6,1)/8, zero exterior
// data: the three axis sweeps of axis_stencil_f64_kernel in one pass.  A CTA
// owns an MX x MY column of (x, y) points and marches through MZ planes of z
// (plus one halo plane on each side): per plane it stages the (MX+2) x (MY+2)
// tile in shared memory, applies T along x, then along y, and keeps the last
// two results per point in registers to apply T along z.  Each axis applies
// 8 T = tridiag(1,6,1) as fma(6, c, l + r) and the product is scaled by 1/512
// once at the end: two FP64 operations per axis instead of three (the FP64
// pipe, not HBM, bounds this kernel).  Power-of-two scaling commutes with
// rounding, so the result is identical to the three sweeps; X is read about
// once and Y written once (the halo rows and columns come from L2), against
// three reads and three writes for the sweeps.
constexpr int MX = 64, MYT = 4, MY = 8, MZ = 32;   // (MX, MYT) threads, MY / MYT rows each

__device__ __forceinline__ double tri(double l, double c, double r) { return fma(6.0, c, l + r); }

__global__ __launch_bounds__(MX * MYT) void mass3d_f64_kernel(const double* __restrict__ X, double* __restrict__ Y,
                                                              int n1, int n2, int n3) {
    __shared__ double u[MY + 2][MX + 2];   // staged plane, one halo on each side
    __shared__ double a[MY + 2][MX];       // T along x
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * MX + tx;
    const int x0 = blockIdx.x * MX, y0 = blockIdx.y * MY, z0 = blockIdx.z * MZ;
    const int z1 = min(z0 + MZ, n3);
    const long long plane = (long long)n1 * n2;
    const int gx = x0 + tx;
    constexpr int ROWS = (MY + 2 + MYT - 1) / MYT;   // staged rows per thread (interior columns)
    double ri[ROWS], rh = 0.0;                       // the next plane, in flight
    auto load = [&](int k) {
        const bool kin = k >= 0 && k < n3;
        const double* Xk = X + (long long)k * plane;
#pragma unroll
        for (int q = 0; q < ROWS; ++q) {
            const int row = ty + q * MYT, gy = y0 - 1 + row;
            ri[q] = (row < MY + 2 && kin && gx < n1 && gy >= 0 && gy < n2) ? Xk[(long long)gy * n1 + gx] : 0.0;
        }
        if (tid < 2 * (MY + 2)) {   // the two halo columns
            const int row = tid >> 1, gy = y0 - 1 + row;
            const int hx = (tid & 1) ? x0 + MX : x0 - 1;
            rh = (kin && hx >= 0 && hx < n1 && gy >= 0 && gy < n2) ? Xk[(long long)gy * n1 + hx] : 0.0;
        }
    };
    double s1[MY / MYT], s2[MY / MYT];   // T_y T_x X on planes k - 1 and k - 2
#pragma unroll
    for (int q = 0; q < MY / MYT; ++q) s1[q] = s2[q] = 0.0;
    load(z0 - 1);
    for (int k = z0 - 1; k <= z1; ++k) {
#pragma unroll
        for (int q = 0; q < ROWS; ++q) {
            const int row = ty + q * MYT;
            if (row < MY + 2) u[row][tx + 1] = ri[q];
        }
        if (tid < 2 * (MY + 2)) u[tid >> 1][(tid & 1) ? MX + 1 : 0] = rh;
        __syncthreads();
        if (k < z1) load(k + 1);   // overlaps the arithmetic below
#pragma unroll
        for (int q = 0; q < ROWS; ++q) {
            const int row = ty + q * MYT;
            if (row < MY + 2) a[row][tx] = tri(u[row][tx], u[row][tx + 1], u[row][tx + 2]);
        }
        __syncthreads();
        const bool kin = k >= 0 && k < n3;
#pragma unroll
        for (int q = 0; q < MY / MYT; ++q) {
            const int row = 1 + ty + q * MYT;   // tile row of output y0 + ty + q MYT
            const int gy = y0 + ty + q * MYT;
            // T along y of the rows inside the grid (rows outside are zero already)
            const double s0 = kin && gy < n2 ? tri(a[row - 1][tx], a[row][tx], a[row + 1][tx]) : 0.0;
            if (k - 1 >= z0 && gx < n1 && gy < n2)
                Y[(long long)(k - 1) * plane + (long long)gy * n1 + gx] = tri(s2[q], s1[q], s0) * (1.0 / 512.0);
            s2[q] = s1[q];
            s1[q] = s0;
        }
    }
}

__global__ void lambda_scale_f64_kernel(const double* __restrict__ x, double* __restrict__ y,
                                        const double* __restrict__ lam, int n1, int n2, int n3,
                                        double c0, double c1, double c2, int invert) {
    const long long N = (long long)n1 * n2 * n3;
    const double* mx = lam;
    const double* my = mx + n1;
    const double* mz = my + n2;
    const double* tx = mz + n3;
    const double* ty = tx + n1;
    const double* tz = ty + n2;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < N;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % n1);
        const int j = (int)((idx / n1) % n2);
        const int k = (int)(idx / ((long long)n1 * n2));
        const double L = mz[k] * my[j] * mx[i] + c0 * mz[k] * my[j] * tx[i] + c1 * mz[k] * ty[j] * mx[i] +
                         c2 * tz[k] * my[j] * mx[i];
        y[idx] = invert ? x[idx] / L : x[idx] * L;
    }
}

__global__ void axpby_f64_kernel(long long N, double a, const double* __restrict__ x, double b,
                                 double* __restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = a * x[i] + b * y[i];
}

__global__ void axpbypz_f64_kernel(long long N, double a, const double* __restrict__ x, double b,
                                   const double* __restrict__ y, double* __restrict__ z) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x)
        z[i] = a * x[i] + b * y[i];
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < kThreads / 32; ++w) t += sh[w];
    }
    return t;  // valid in thread 0
}

// Contiguous chunk per block keeps the summation order fixed for a given N.
__device__ __forceinline__ void chunk_range(long long N, long long& lo, long long& hi) {
    const long long per = (N + gridDim.x - 1) / gridDim.x;
    lo = (long long)blockIdx.x * per;
    hi = lo + per < N ? lo + per : N;
}

__global__ __launch_bounds__(kThreads) void cg_update_f64_kernel(long long N, double alpha,
                                                                 const double* __restrict__ p,
                                                                 const double* __restrict__ q,
                                                                 double* __restrict__ x,
                                                                 double* __restrict__ r,
                                                                 double* __restrict__ part) {
    long long lo, hi;
    chunk_range(N, lo, hi);
    double acc = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += kThreads) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

template <int C>
__global__ __launch_bounds__(kThreads) void multidot_f64_kernel(long long N, int m0, int mc,
                                                                const double* __restrict__ V, long long ldv,
                                                                const double* __restrict__ w,
                                                                double* __restrict__ part) {
    long long lo, hi;
    chunk_range(N, lo, hi);
    double acc[C];
#pragma unroll
    for (int j = 0; j < C; ++j) acc[j] = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += kThreads) {
        const double wi = w[i];
#pragma unroll
        for (int j = 0; j < C; ++j)
            if (j < mc) acc[j] = fma(V[(long long)(m0 + j) * ldv + i], wi, acc[j]);
    }
#pragma unroll
    for (int j = 0; j < C; ++j) {
        if (j < mc) {
            const double t = block_sum(acc[j]);
            if (threadIdx.x == 0) part[(long long)(m0 + j) * gridDim.x + blockIdx.x] = t;
        }
    }
}

__global__ void multiaxpy_f64_kernel(long long N, int m, const double* __restrict__ V, long long ldv,
                                     const double* __restrict__ h, double* __restrict__ w) {
    __shared__ double hs[128];
    for (int j = threadIdx.x; j < m; j += blockDim.x) hs[j] = h[j];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        double acc = w[i];
        for (int j = 0; j < m; ++j) acc = fma(-hs[j], V[(long long)j * ldv + i], acc);
        w[i] = acc;
    }
}

__global__ void reduce_finish_kernel(const double* __restrict__ part, int nblk, int m, double* __restrict__ out) {
    // one warp per result; fixed order: lane-strided partial sums, then a fixed tree
    const int j = blockIdx.x;
    if (j >= m) return;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) acc += part[(long long)j * nblk + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) out[j] = acc;
}

// F = cP Pz Py Px + cS (Pz Py Sx + Pz Sy Px + Sz Py Px), regrouped per line as
// F = a_jk X1_i + b_jk X2_i with a = Pz Py, b = cS (Pz Sy + Sz Py),
// X1 = cP Px + cS Sx, X2 = Px: the per-line and per-column factors are formed
// once per block in shared memory, so each grid point costs one multiply and
// one fused multiply-add in FP64.  A block covers SRC_LINES lines (j, k).
constexpr int SRC_LINES = 8;
__global__ void source_assemble_f64_kernel(const double* __restrict__ oned, int n1, int n2, int n3,
                                           double cP, double cS, double* __restrict__ F) {
    extern __shared__ double src_sm[];    // X1[n1], X2[n1], a[SRC_LINES], b[SRC_LINES]
    double* X1 = src_sm;
    double* X2 = X1 + n1;
    double* la = X2 + n1;
    double* lb = la + SRC_LINES;
    const double* Px = oned;
    const double* Py = Px + n1;
    const double* Pz = Py + n2;
    const double* Sx = Pz + n3;
    const double* Sy = Sx + n1;
    const double* Sz = Sy + n2;
    const long long lines = (long long)n2 * n3;
    for (int i = threadIdx.x; i < n1; i += blockDim.x) {
        X1[i] = fma(cP, Px[i], cS * Sx[i]);
        X2[i] = Px[i];
    }
    for (long long l0 = (long long)blockIdx.x * SRC_LINES; l0 < lines; l0 += (long long)gridDim.x * SRC_LINES) {
        __syncthreads();
        if (threadIdx.x < SRC_LINES && l0 + threadIdx.x < lines) {
            const long long l = l0 + threadIdx.x;
            const int j = (int)(l % n2), k = (int)(l / n2);
            la[threadIdx.x] = Pz[k] * Py[j];
            lb[threadIdx.x] = cS * fma(Pz[k], Sy[j], Sz[k] * Py[j]);
        }
        __syncthreads();
        const int nl = (int)(lines - l0 < SRC_LINES ? lines - l0 : SRC_LINES);
        for (int e = threadIdx.x; e < nl * n1; e += blockDim.x) {
            const int t = e / n1, i = e - t * n1;
            F[(l0 + t) * n1 + i] = fma(la[t], X1[i], lb[t] * X2[i]);
        }
    }
}

// b = AN - Ku + dt F ;  r = dt F - 2 Ku   (F may be null); with part set,
// per-block sums of b^2 and r^2 into part[block] and part[grid + block]
__global__ void cn_first_kernel(long long N, const double* __restrict__ AN, const double* __restrict__ Ku,
                                const double* __restrict__ F, double dt, double* __restrict__ b,
                                double* __restrict__ r, double* __restrict__ part) {
    double bb = 0.0, rr = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const double f = F ? dt * F[i] : 0.0;
        const double k = Ku[i];
        const double bi = AN[i] - k + f;
        const double ri = fma(-2.0, k, f);
        b[i] = bi;
        r[i] = ri;
        bb = fma(bi, bi, bb);
        rr = fma(ri, ri, rr);
    }
    if (part) {
        const double t1 = block_sum(bb);
        const double t2 = block_sum(rr);
        if (threadIdx.x == 0) {
            part[blockIdx.x] = t1;
            part[gridDim.x + blockIdx.x] = t2;
        }
    }
}

// t = 2 AN + dt F ;  b <- t + r - b ;  r <- b_new + r - b_old  (norm partials as cn_first_kernel)
__global__ void cn_chain_kernel(long long N, const double* __restrict__ AN, const double* __restrict__ F, double dt,
                                double* __restrict__ b, double* __restrict__ r, double* __restrict__ part) {
    double bb = 0.0, rr = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const double t = fma(2.0, AN[i], F ? dt * F[i] : 0.0);
        const double d = r[i] - b[i];
        const double bn = t + d;
        const double rn = bn + d;
        b[i] = bn;
        r[i] = rn;
        bb = fma(bn, bn, bb);
        rr = fma(rn, rn, rr);
    }
    if (part) {
        const double t1 = block_sum(bb);
        const double t2 = block_sum(rr);
        if (threadIdx.x == 0) {
            part[blockIdx.x] = t1;
            part[gridDim.x + blockIdx.x] = t2;
        }
    }
}


// Chained CN step with a polynomial-extrapolation initial guess.  In: u =
// u^{m-1}, AN = A_N u^{m-1}, (b, r) = the previous step's RHS and final true
// residual (so A u^{m-1} = b - r), history H1 = (u^{m-2}, A u^{m-2}) and
// H2 = (u^{m-3}, A u^{m-3}).  Out: b = b^m, u = x0 (extrapolation of the given
// order: 0 u^{m-1}; 1 2u^{m-1} - u^{m-2}; 2 3u^{m-1} - 3u^{m-2} + u^{m-3}),
// r = b^m - A x0 from the same linear combination of the stored A u (no
// operator application), and (u^{m-1}, A u^{m-1}) into the H2 slot, which
// the caller then relabels as H1.
// order 3: x0 = g0 u^{m-1} + g1 u^{m-2} + g2 u^{m-3} with the caller's
// coefficients (the order-2 extrapolation corrected by cn_mr_dots_kernel).
__global__ void cn_chain_extrap_kernel(long long N, const double* __restrict__ AN, const double* __restrict__ F,
                                       double dt, double* __restrict__ b, double* __restrict__ r,
                                       double* __restrict__ u, const double* __restrict__ U1,
                                       const double* __restrict__ AU1, double* __restrict__ U2,
                                       double* __restrict__ AU2, int order, const double* __restrict__ g,
                                       double* __restrict__ part, long long pstride) {
    // GB300 issues FP64 at ~1/64 of its FP32 rate and this pass moves 112
    // bytes per point: it is FP64-bound unless every FP64 operation that is
    // not needed goes.  2 A_N u is formed by the exponent, dt F is fused into
    // the same rounding, and the two norms (which only set the stopping
    // threshold and the first sweep's scale) are summed in FP32 from values
    // truncated by integer operations: 10 FP64 operations per point instead of 13.
    float bb = 0.f, rr = 0.f;
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;   // order 3: the corrected guess's coefficients (device)
    if (order >= 3) {
        g0 = g[0];
        g1 = g[1];
        g2 = g[2];
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        double bn, rn;
        chain_extrap_point(i, AN, F, dt, b, r, u, U1, AU1, U2, AU2, order, g0, g1, g2, &bn, &rn);
        const float bf = f64_to_f32_rz((unsigned long long)__double_as_longlong(bn));
        const float rf = f64_to_f32_rz((unsigned long long)__double_as_longlong(rn));
        bb = fmaf(bf, bf, bb);
        rr = fmaf(rf, rf, rr);
    }
    if (part) {
        const double t1 = block_sum((double)bb);
        const double t2 = block_sum((double)rr);
        if (threadIdx.x == 0) {
            part[blockIdx.x] = t1;
            part[pstride + blockIdx.x] = t2;   // ||r||^2 partials one row below (pstride >= gridDim.x)
        }
    }
}

// Minimal-residual correction of the order-2 extrapolated guess of a chained
// CN step.  With a_k = A u^{m-1-k} (a_0 = b^{m-1} - r^{m-1}, a_1, a_2 from the
// history), the extrapolation's residual is r_e = b^m - (3 a_0 - 3 a_1 + a_2),
// b^m = 2 A_N u^{m-1} + dt F - a_0, and the history differences
// e_1 = a_0 - a_1, e_2 = a_0 - 2 a_1 + a_2 are the operator images of
// d_1 = u^{m-1} - u^{m-2}, d_2 = u^{m-1} - 2 u^{m-2} + u^{m-3}.  Sums over the
// grid: part[q] for q = <e1,e1>, <e1,e2>, <e2,e2>, <e1,r_e>, <e2,r_e>; the
// caller solves the 2 x 2 normal equations for the c minimising
// ||r_e - c1 e1 - c2 e2|| and takes x0 = x_e + c1 d1 + c2 d2 (no operator
// application).  The sums only set two coefficients (their error changes
// the guess, not the solution): every term is formed in FP32 from the FP64
// values truncated by integer operations (no FP64 arithmetic), per-thread
// sums in FP32, the block and grid sums in FP64.
__global__ void cn_mr_dots_kernel(long long N, const double* __restrict__ AN, const double* __restrict__ F, float dtf,
                                  const double* __restrict__ b, const double* __restrict__ r,
                                  const double* __restrict__ AU1, const double* __restrict__ AU2,
                                  double* __restrict__ part) {
    float s[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        chain_mr_terms(__ldg(AN + i), F, i, dtf, __ldg(b + i), __ldg(r + i), __ldg(AU1 + i), __ldg(AU2 + i), s);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const double t = block_sum((double)s[q]);
        if (threadIdx.x == 0) part[(long long)q * gridDim.x + blockIdx.x] = t;
    }
}

// Coefficients g of the corrected guess x0 = g0 u^{m-1} + g1 u^{m-2} +
// g2 u^{m-3} from the five sums m of cn_mr_dots_kernel (one thread): the
// order-2 extrapolation 3, -3, 1 plus c1 d1 + c2 d2 (d1 = u^{m-1} - u^{m-2},
// d2 = u^{m-1} - 2 u^{m-2} + u^{m-3}), c solving the 2 x 2 normal equations
// [m0 m1; m1 m2] c = [m3; m4].  An ill-conditioned or non-finite system, or
// |c| > 1e3, leaves c = 0.
__global__ void cn_mr_coef_kernel(const double* __restrict__ m, double* __restrict__ g) { chain_mr_coefficients(m, g); }

inline int grid_for(long long N) {
    long long g = (N + kThreads - 1) / kThreads;
    if (g > 152LL * 16) g = 152LL * 16;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

int reduction_blocks(size_t N) {
    long long b = ((long long)N + 4 * kThreads - 1) / (4 * kThreads);
    if (b > 1216) b = 1216;  // 8 per SM on 152 SMs
    if (b < 1) b = 1;
    return (int)b;
}

void launch_axis_gemm_f64(const double* Mat, const double* X, double* Y, const AxisView& v, double alpha,
                          const double* Z, double beta, cudaStream_t s) {
    stats_count_launch();
    dim3 grid((unsigned)((v.lines + BN - 1) / BN), (unsigned)((v.n + BM - 1) / BM));
    axis_gemm_f64_kernel<<<grid, kThreads, 0, s>>>(Mat, X, Y, v, alpha, Z, beta);
}

void launch_axis_stencil_f64(const double* X, double* Y, const AxisView& v, double beta, const double* W,
                             double gamma, cudaStream_t s) {
    stats_count_launch();
    // recover (n1, n2, n3) and the axis from the view
    int n1, n2, n3, axis;
    if (v.stride == 1) {
        axis = 0; n1 = v.n; n2 = (int)v.lines; n3 = 1;   // lines of the x axis: any (n2, n3) split works
    } else if (v.s_out != 0) {
        axis = 1; n1 = (int)v.l_in; n2 = v.n; n3 = (int)(v.lines / v.l_in);
    } else {
        axis = 2; n1 = (int)v.l_in; n2 = 1; n3 = v.n;
    }
    dim3 blk(n1 >= 64 ? 64 : 32, 4);
    const long long gy = ((long long)n2 + blk.y - 1) / blk.y;
    dim3 grid((n1 + blk.x - 1) / blk.x, (unsigned)(gy < 65535 ? gy : 65535), n3 < 64 ? n3 : 64);
    axis_stencil_f64_kernel<<<grid, blk, 0, s>>>(X, Y, n1, n2, n3, axis, beta, W, gamma);
}

void launch_mass3d_f64(const double* X, double* Y, const int n[3], cudaStream_t s) {
    stats_count_launch();
    dim3 grid((unsigned)((n[0] + MX - 1) / MX), (unsigned)((n[1] + MY - 1) / MY), (unsigned)((n[2] + MZ - 1) / MZ));
    mass3d_f64_kernel<<<grid, dim3(MX, MYT), 0, s>>>(X, Y, n[0], n[1], n[2]);
}

void launch_lambda_scale_f64(const double* x, double* y, const double* lam, const int n[3], const double c[3],
                             int invert, cudaStream_t s) {
    stats_count_launch();
    const long long N = (long long)n[0] * n[1] * n[2];
    lambda_scale_f64_kernel<<<grid_for(N), kThreads, 0, s>>>(x, y, lam, n[0], n[1], n[2], c[0], c[1], c[2],
                                                              invert);
}

void launch_axpby_f64(size_t N, double a, const double* x, double b, double* y, cudaStream_t s) {
    stats_count_launch();
    axpby_f64_kernel<<<grid_for((long long)N), kThreads, 0, s>>>((long long)N, a, x, b, y);
}

void launch_axpbypz_f64(size_t N, double a, const double* x, double b, const double* y, double* z,
                        cudaStream_t s) {
    stats_count_launch();
    axpbypz_f64_kernel<<<grid_for((long long)N), kThreads, 0, s>>>((long long)N, a, x, b, y, z);
}

void launch_cg_update_f64(size_t N, double alpha, const double* p, const double* q, double* x, double* r,
                          double* part, int nblk, cudaStream_t s) {
    stats_count_launch();
    cg_update_f64_kernel<<<nblk, kThreads, 0, s>>>((long long)N, alpha, p, q, x, r, part);
}

void launch_multidot_f64(size_t N, int m, const double* V, size_t ldv, const double* w, double* part, int nblk,
                         cudaStream_t s) {
    stats_count_launch();
    for (int m0 = 0; m0 < m; m0 += 8) {
        const int mc = (m - m0) < 8 ? (m - m0) : 8;
        if (m0 > 0) stats_count_launch();
        multidot_f64_kernel<8><<<nblk, kThreads, 0, s>>>((long long)N, m0, mc, V, (long long)ldv, w, part);
    }
}

void launch_multiaxpy_f64(size_t N, int m, const double* V, size_t ldv, const double* h, double* w,
                          cudaStream_t s) {
    stats_count_launch();
    multiaxpy_f64_kernel<<<grid_for((long long)N), kThreads, 0, s>>>((long long)N, m, V, (long long)ldv, h, w);
}

void launch_reduce_finish(const double* part, int nblk, int m, double* out, cudaStream_t s) {
    stats_count_launch();
    reduce_finish_kernel<<<m, 32, 0, s>>>(part, nblk, m, out);
}

// ||b||^2 and ||r||^2 of the chain kernels: partials of `grid` blocks -> norms2[0..1]
static void finish_norms(double* part, int grid, double* norms2, cudaStream_t s) {
    if (norms2) launch_reduce_finish(part, grid, 2, norms2, s);
}

void launch_cn_first(size_t N, const double* AN, const double* Ku, const double* F, double dt, double* b, double* r,
                     double* part, double* norms2, cudaStream_t s) {
    stats_count_launch();
    const int g = grid_for((long long)N);
    cn_first_kernel<<<g, kThreads, 0, s>>>((long long)N, AN, Ku, F, dt, b, r, norms2 ? part : nullptr);
    finish_norms(part, g, norms2, s);
}

void launch_cn_chain(size_t N, const double* AN, const double* F, double dt, double* b, double* r, double* part,
                     double* norms2, cudaStream_t s) {
    stats_count_launch();
    const int g = grid_for((long long)N);
    cn_chain_kernel<<<g, kThreads, 0, s>>>((long long)N, AN, F, dt, b, r, norms2 ? part : nullptr);
    finish_norms(part, g, norms2, s);
}

void launch_cn_chain_extrap(size_t N, const double* AN, const double* F, double dt, double* b, double* r, double* u,
                            const double* U1, const double* AU1, double* U2, double* AU2, int order, const double* g,
                            double* part, double* norms2, cudaStream_t s) {
    stats_count_launch();
    const int grid = grid_for((long long)N);
    cn_chain_extrap_kernel<<<grid, kThreads, 0, s>>>((long long)N, AN, F, dt, b, r, u, U1, AU1, U2, AU2,
                                                     order >= 3 && !g ? 2 : order, g, norms2 ? part : nullptr, grid);
    finish_norms(part, grid, norms2, s);
}

void launch_cn_chain_extrap_chunks(size_t N, int nchunks, const cudaEvent_t* ready, const double* AN, const double* F,
                                   double dt, double* b, double* r, double* u, const double* U1, const double* AU1,
                                   double* U2, double* AU2, int order, const double* g, double* part, double* norms2,
                                   cudaStream_t s) {
    const size_t per = (N + nchunks - 1) / nchunks;
    const int grid = grid_for((long long)per);
    const long long pstride = (long long)grid * nchunks;
    for (int k = 0; k < nchunks; ++k) {
        const size_t o = per * k;
        if (o >= N) {   // an empty tail chunk: zero partials, so the sums below stay right
            if (norms2) {
                cudaMemsetAsync(part + (size_t)k * grid, 0, grid * sizeof(double), s);
                cudaMemsetAsync(part + pstride + (size_t)k * grid, 0, grid * sizeof(double), s);
            }
            continue;
        }
        const size_t len = N - o < per ? N - o : per;
        cudaStreamWaitEvent(s, ready[k], 0);
        stats_count_launch();
        cn_chain_extrap_kernel<<<grid, kThreads, 0, s>>>((long long)len, AN + o, F ? F + o : nullptr, dt, b + o, r + o,
                                                         u + o, U1 + o, AU1 + o, U2 + o, AU2 + o,
                                                         order >= 3 && !g ? 2 : order, g,
                                                         norms2 ? part + (size_t)k * grid : nullptr, pstride);
    }
    if (norms2) launch_reduce_finish(part, (int)pstride, 2, norms2, s);
}

void launch_cn_mr_dots(size_t N, const double* AN, const double* F, double dt, const double* b, const double* r,
                       const double* AU1, const double* AU2, double* part, double* out5, cudaStream_t s) {
    stats_count_launch();
    const int grid = grid_for((long long)N);
    cn_mr_dots_kernel<<<grid, kThreads, 0, s>>>((long long)N, AN, F, (float)dt, b, r, AU1, AU2, part);
    launch_reduce_finish(part, grid, 5, out5, s);
}

// The first level of the guess history at a chain's restart: H0 = u,
// AH0 = A u = A_N u + K u (the two products the restart step has formed).
__global__ void history_first_kernel(long long N, const double* __restrict__ u, const double* __restrict__ AN,
                                     const double* __restrict__ Ku, double* __restrict__ H0, double* __restrict__ AH0) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        H0[i] = u[i];
        AH0[i] = AN[i] + Ku[i];
    }
}

void launch_history_first(size_t N, const double* u, const double* AN, const double* Ku, double* H0, double* AH0,
                          cudaStream_t s) {
    stats_count_launch();
    history_first_kernel<<<grid_for((long long)N), kThreads, 0, s>>>((long long)N, u, AN, Ku, H0, AH0);
}

void launch_cn_mr_coefficients(const double* m5, double* g3, cudaStream_t s) {
    stats_count_launch();
    cn_mr_coef_kernel<<<1, 1, 0, s>>>(m5, g3);
}

void launch_source_assemble_f64(const double* oned, const int n[3], double cP, double cS, double* F,
                                cudaStream_t s) {
    stats_count_launch();
    const long long N = (long long)n[0] * n[1] * n[2];
    const long long lines = (long long)n[1] * n[2];
    long long blocks = (lines + SRC_LINES - 1) / SRC_LINES;
    if (blocks > 152LL * 8) blocks = 152LL * 8;
    const size_t smem = (2 * (size_t)n[0] + 2 * SRC_LINES) * sizeof(double);
    (void)N;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(source_assemble_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    source_assemble_f64_kernel<<<(unsigned)blocks, kThreads, smem, s>>>(oned, n[0], n[1], n[2], cP, cS, F);
}

}  // namespace tfde
