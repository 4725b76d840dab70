// Mixed-precision solves on the FFT passes, for the grids the tensor-core
// contraction does not take (an n_a that is not a multiple of 8, n_a > 448,
// and the 2-D problem of Example 1).
//
// The structure is the tensor-core path's: FP64 iterative refinement of
// A u = b (Eq. (linear_sys)) in which every sweep forms the true residual
// r = b - A x with the FP64 FFT-embedded Toeplitz passes and solves the
// correction equation A d = r in FP32, with PCG (Sec. 3.1, symmetric
// problems) or one left-preconditioned GMRES(m) cycle (Sec. 3.2), both with
// the tau preconditioner P^{-1} = S_N Lambda^{-1} S_N (Eq. (diag_tau_pre))
// applied by the FP32 FFT DST-I passes.  The inner operator carries FP32
// rounding only (about 1e-7 relative per product against the split-BF16
// contraction's 2^-16), so one sweep reaches further: the inner floor is
// 1e-5.  Inner products accumulate in FP64; the CG coefficients alpha and
// beta are formed on the device and the host reads one scalar per PCG
// iteration (its stopping test) and two per Arnoldi step (the Hessenberg
// column, whose Givens rotations run on the host as in the FP64 PGMRES).
#include <chrono>
#include <cmath>
#include <vector>

#include "tfde_fft.h"
#include "tfde_givens.h"
#include "tfde_internal.h"
#include "tfde_stats.h"

namespace tfde {

int pcg64(const tfde_problem*, const double*, double*, double, int, tfde_info*, cudaStream_t, bool);
int pgmres64(tfde_problem*, const double*, double*, int, double, int, tfde_info*, cudaStream_t, bool);
void launch_dot32(size_t N, const float* a, const float* b, double* part, int nblk, cudaStream_t s);
void launch_multidot32(size_t N, int m, const float* V, size_t ldv, const float* w, double* part, int nblk,
                       cudaStream_t s);
void launch_multiaxpy32(size_t N, int m, const float* V, size_t ldv, const double* h, float* w, cudaStream_t s);
void launch_add32to64(size_t N, double sc, const float* d, double* x, cudaStream_t s);
void launch_widen32(size_t N, const float* v, double sc, double* y, cudaStream_t s);

namespace {

using clk = std::chrono::steady_clock;

constexpr int kT = 256;
// the inner FP32 solve lowers the true residual by at most about this much
// per sweep (the FP32 operator's accuracy against the problem's conditioning)
constexpr double kInnerFloor32 = 1e-5;
constexpr int kMaxRestart = 120;   // GMRES columns: the reduction scratch holds 128 sums

// FP32 grid functions of the inner solves
enum { V_R, V_Z, V_P, V_Q, V_X, V_A, V_W, V_C, V_E, NV };
// device scalars
enum { S_RZ0 = 0, S_RZ1 = 1, S_PQ = 2, S_RR = 3, S_H = 8, NS = 256 };

struct FftMixed {
    float* v[NV] = {};
    float* V = nullptr;     // GMRES basis, (vcap + 1) vectors
    int vcap = 0;
    double* d = nullptr;    // device scalars
    double* h = nullptr;    // pinned host mirror of d
};

FftMixed* state(const tfde_problem* P) { return static_cast<FftMixed*>(P->fmix); }

#define FM_TRY(call)                                                                     \
    do {                                                                                 \
        if ((call) != cudaSuccess) return set_error(TFDE_ECUDA, "fft mixed: " #call);     \
    } while (0)

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[kT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kT / 32; ++w) t += sh[w];
    return t;
}

// r32 = (float)(sc r64); x32 = 0 (when given)
__global__ void to32_kernel(long long N, const double* __restrict__ r64, double sc, float* __restrict__ r32,
                            float* __restrict__ x32) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        r32[i] = (float)(r64[i] * sc);
        if (x32) x32[i] = 0.f;
    }
}

// alpha = num / den (device); x += alpha p; r -= alpha q; per-block partial
// sums of r.r (FP64 across the block) into part[blockIdx.x]
__global__ __launch_bounds__(kT) void cg_update_kernel(long long N, const double* __restrict__ num,
                                                       const double* __restrict__ den, const float* __restrict__ p,
                                                       const float* __restrict__ q, float* __restrict__ x,
                                                       float* __restrict__ r, double* __restrict__ part) {
    const float alpha = (float)(num[0] / den[0]);
    const long long per = (N + gridDim.x - 1) / gridDim.x;
    const long long lo = (long long)blockIdx.x * per;
    const long long hi = lo + per < N ? lo + per : N;
    double acc = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += kT) {
        x[i] = fmaf(alpha, p[i], x[i]);
        const float ri = fmaf(-alpha, q[i], r[i]);
        r[i] = ri;
        acc += (double)ri * (double)ri;
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// p = z + beta p, beta = num / den (device)
__global__ void xpay_kernel(long long N, const double* __restrict__ num, const double* __restrict__ den,
                            const float* __restrict__ z, float* __restrict__ p) {
    const float beta = (float)(num[0] / den[0]);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        p[i] = fmaf(beta, p[i], z[i]);
}

// v *= sc
__global__ void scale_kernel(long long N, float sc, float* __restrict__ v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        v[i] *= sc;
}

int grid_for(size_t N) {
    long long g = ((long long)N + kT - 1) / kT;
    if (g > 152LL * 16) g = 152LL * 16;
    return (int)(g < 1 ? 1 : g);
}

void launch_to32(size_t N, const double* r64, double sc, float* r32, float* x32, cudaStream_t s) {
    stats_count_launch();
    to32_kernel<<<grid_for(N), kT, 0, s>>>((long long)N, r64, sc, r32, x32);
}

// <a, b> into dev (device, FP64)
void dot_to(const tfde_problem* P, const float* a, const float* b, double* dev, cudaStream_t s) {
    launch_dot32(P->N, a, b, P->red, P->nblk, s);
    launch_reduce_finish(P->red, P->nblk, 1, dev, s);
}

int read_host(const tfde_problem* P, const double* dev, int count, double* out, cudaStream_t s) {
    FftMixed* F = state(P);
    FM_TRY(cudaMemcpyAsync(F->h, dev, count * sizeof(double), cudaMemcpyDeviceToHost, s));
    FM_TRY(cudaStreamSynchronize(s));
    for (int i = 0; i < count; ++i) out[i] = F->h[i];
    return TFDE_OK;
}

int op_A32(const tfde_problem* P, const float* x, float* y, cudaStream_t s) {
    FftMixed* F = state(P);
    return fft::apply_A<float>(P, TFDE_OP_A, x, y, F->v[V_A], F->v[V_W], F->v[V_C], F->v[V_E], s);
}

int op_Pinv32(const tfde_problem* P, const float* r, float* z, cudaStream_t s) {
    FftMixed* F = state(P);
    return fft::apply_Pinv<float>(P, r, z, F->v[V_A], F->v[V_W], s);
}

// Inner PCG in FP32 on A d = r32 (r32 in V_R, d in V_X = 0), until
// ||r|| <= theta ||r_0|| (rr0 = ||r32||^2) or maxit iterations.
int inner_pcg(const tfde_problem* P, double theta, int maxit, double rr0, int* iters, double* reached, cudaStream_t s) {
    FftMixed* F = state(P);
    const size_t N = P->N;
    float* r = F->v[V_R];
    float* z = F->v[V_Z];
    float* p = F->v[V_P];
    float* q = F->v[V_Q];
    double* d = F->d;
    int st;
    *iters = 0;
    *reached = 1.0;
    if (!(rr0 > 0.0)) return TFDE_OK;
    if ((st = op_Pinv32(P, r, p, s))) return st;   // p_0 = z_0 = P^{-1} r_0
    dot_to(P, r, p, d + S_RZ0, s);
    int rz = S_RZ0;
    int k = 0;
    while (k < maxit) {
        if ((st = op_A32(P, p, q, s))) return st;
        dot_to(P, p, q, d + S_PQ, s);
        stats_count_launch();
        cg_update_kernel<<<P->nblk, kT, 0, s>>>((long long)N, d + rz, d + S_PQ, p, q, F->v[V_X], r, P->red);
        launch_reduce_finish(P->red, P->nblk, 1, d + S_RR, s);
        double rr;
        if ((st = read_host(P, d + S_RR, 1, &rr, s))) return st;
        ++k;
        if (!std::isfinite(rr)) return set_error(TFDE_ENAN, "non-finite inner residual");
        *reached = std::sqrt(rr / rr0);
        if (rr <= theta * theta * rr0 || k >= maxit) break;
        const int rzn = rz == S_RZ0 ? S_RZ1 : S_RZ0;
        if ((st = op_Pinv32(P, r, z, s))) return st;
        dot_to(P, r, z, d + rzn, s);
        stats_count_launch();
        xpay_kernel<<<grid_for(N), kT, 0, s>>>((long long)N, d + rzn, d + rz, z, p);   // p = z + beta p
        rz = rzn;
    }
    *iters = k;
    return TFDE_OK;
}

int ensure_basis(const tfde_problem* P, int m) {
    FftMixed* F = state(P);
    if (F->vcap >= m) return TFDE_OK;
    cudaFree(F->V);
    F->V = nullptr;
    F->vcap = 0;
    if (cudaMalloc((void**)&F->V, (size_t)(m + 1) * P->N * sizeof(float)) != cudaSuccess)
        return set_error(TFDE_ENOMEM, "cudaMalloc of the FP32 GMRES basis failed");
    F->vcap = m;
    return TFDE_OK;
}

// One left-preconditioned GMRES(m) cycle in FP32 on A d = r32 (V_R, unit
// norm), d into V_X: Arnoldi on P^{-1} A with classical Gram-Schmidt and one
// re-orthogonalisation (the second projection's sums and ||w||^2 in one
// reduction: ||w - V h2||^2 = ||w||^2 - ||h2||^2 for an orthonormal V),
// stopped when the rotated residual estimate falls to theta of ||P^{-1} r||.
// *est_ratio: that estimate's reduction.
int inner_gmres(const tfde_problem* P, int m, double theta, int maxit, int* iters, double* est_ratio,
                cudaStream_t s) {
    FftMixed* F = state(P);
    const size_t N = P->N;
    float* V = F->V;
    double* d = F->d;
    int st;
    *iters = 0;
    *est_ratio = 1.0;
    auto col = [&](int j) { return V + (size_t)j * N; };
    if ((st = op_Pinv32(P, F->v[V_R], col(0), s))) return st;
    dot_to(P, col(0), col(0), d + S_H, s);
    double beta2;
    if ((st = read_host(P, d + S_H, 1, &beta2, s))) return st;
    const double beta = std::sqrt(beta2);
    if (!std::isfinite(beta)) return set_error(TFDE_ENAN, "non-finite preconditioned residual");
    if (beta == 0.0) return TFDE_OK;
    stats_count_launch();
    scale_kernel<<<grid_for(N), kT, 0, s>>>((long long)N, (float)(1.0 / beta), col(0));
    GivensLS ls(m);
    ls.g[0] = beta;
    std::vector<double> h(m + 2), h2(m + 2);
    int k = 0;
    double res = beta;
    for (int j = 0; j < m && k < maxit; ++j) {
        float* w = col(j + 1);
        if ((st = op_A32(P, col(j), F->v[V_Q], s))) return st;
        if ((st = op_Pinv32(P, F->v[V_Q], w, s))) return st;
        // first projection
        launch_multidot32(N, j + 1, V, N, w, P->red, P->nblk, s);
        launch_reduce_finish(P->red, P->nblk, j + 1, d + S_H, s);
        launch_multiaxpy32(N, j + 1, V, N, d + S_H, w, s);
        if ((st = read_host(P, d + S_H, j + 1, h.data(), s))) return st;
        // second projection, with ||w||^2 (w is column j + 1 of V)
        launch_multidot32(N, j + 2, V, N, w, P->red, P->nblk, s);
        launch_reduce_finish(P->red, P->nblk, j + 2, d + S_H, s);
        launch_multiaxpy32(N, j + 1, V, N, d + S_H, w, s);
        if ((st = read_host(P, d + S_H, j + 2, h2.data(), s))) return st;
        double ww = h2[j + 1];
        for (int i = 0; i <= j; ++i) {
            h[i] += h2[i];
            ww -= h2[i] * h2[i];
        }
        if (!std::isfinite(ww)) return set_error(TFDE_ENAN, "non-finite Arnoldi vector");
        const double hn = std::sqrt(std::fmax(ww, 0.0));
        h[j + 1] = hn;
        if (hn > 0.0) {
            stats_count_launch();
            scale_kernel<<<grid_for(N), kT, 0, s>>>((long long)N, (float)(1.0 / hn), w);
        }
        res = ls.add_column(j, h.data());
        ++k;
        if (res <= theta * beta || hn == 0.0) break;
    }
    // d = V y
    std::vector<double> y;
    ls.solve(k, y);
    for (int i = 0; i < k; ++i) F->h[i] = -y[i];   // multiaxpy subtracts
    FM_TRY(cudaMemcpyAsync(d + S_H, F->h, k * sizeof(double), cudaMemcpyHostToDevice, s));
    FM_TRY(cudaMemsetAsync(F->v[V_X], 0, N * sizeof(float), s));
    launch_multiaxpy32(N, k, V, N, d + S_H, F->v[V_X], s);
    *iters = k;
    *est_ratio = res / beta;
    return TFDE_OK;
}

// r = b - A x (FP64 FFT passes) and ||r||
int true_residual(tfde_problem* P, const double* b, const double* x, double* r, double* nr, cudaStream_t s) {
    double* ax = P->w[tfde_problem::W_Q];
    int st = apply_A64(P, TFDE_OP_A, x, ax, s);
    if (st) return st;
    launch_axpbypz_f64(P->N, 1.0, b, -1.0, ax, r, s);
    double rr;
    if ((st = dots64(P, 1, r, 0, r, &rr, s))) return st;
    *nr = std::sqrt(rr);
    return TFDE_OK;
}

// ||b|| and the starting residual (given in W_R by the CN driver, or formed)
int start(tfde_problem* P, const double* b, double* x, bool r_given, double* nb, double* nr, cudaStream_t s) {
    double* r64 = P->w[tfde_problem::W_R];
    double bb;
    int st = dots64(P, 1, b, 0, b, &bb, s);
    if (st) return st;
    P->norms_ready = false;
    *nb = std::sqrt(bb);
    if (!std::isfinite(*nb)) return set_error(TFDE_ENAN, "non-finite right-hand side");
    if (*nb == 0.0) {
        FM_TRY(cudaMemsetAsync(x, 0, P->N * sizeof(double), s));
        *nr = 0.0;
        return TFDE_OK;
    }
    if (r_given) {
        double rr;
        if ((st = dots64(P, 1, r64, 0, r64, &rr, s))) return st;
        *nr = std::sqrt(rr);
        return TFDE_OK;
    }
    return true_residual(P, b, x, r64, nr, s);
}

}  // namespace

bool fmix_wanted(const tfde_problem* P) {
    if (P->dim2) return true;
    for (int a = 0; a < 3; ++a)
        if (P->n[a] % 8 != 0 || P->n[a] > 448) return true;
    return false;
}

int fmix_init(tfde_problem* P, cudaStream_t s) {
    if (!P->fft) return set_error(TFDE_EUNSUPPORTED, "TFDE_MIXED on this grid needs the FFT passes (every n_a <= 2048)");
    FftMixed* F = new FftMixed();
    P->fmix = F;
    for (int i = 0; i < NV; ++i) {
        FM_TRY(cudaMalloc((void**)&F->v[i], P->N * sizeof(float)));
        FM_TRY(cudaMemsetAsync(F->v[i], 0, P->N * sizeof(float), s));
    }
    FM_TRY(cudaMalloc((void**)&F->d, NS * sizeof(double)));
    FM_TRY(cudaMemsetAsync(F->d, 0, NS * sizeof(double), s));
    FM_TRY(cudaMallocHost((void**)&F->h, NS * sizeof(double)));
    // the basis of the default restart length (20) up front, larger ones on demand
    return ensure_basis(P, 20);
}

void fmix_free(tfde_problem* P) {
    FftMixed* F = state(P);
    if (!F) return;
    for (float* v : F->v) cudaFree(v);
    cudaFree(F->V);
    cudaFree(F->d);
    if (F->h) cudaFreeHost(F->h);
    delete F;
    P->fmix = nullptr;
}

// y = A x: the FP32 FFT passes (TFDE_OP_FAST) or the FP64 ones
int fmix_apply_A(const tfde_problem* P, int op, const double* x, double* y, cudaStream_t s) {
    if (!(op & TFDE_OP_FAST)) return apply_A64(P, op, x, y, s);
    FftMixed* F = state(P);
    launch_to32(P->N, x, 1.0, F->v[V_P], nullptr, s);
    int st = fft::apply_A<float>(P, op & ~TFDE_OP_FAST, F->v[V_P], F->v[V_Q], F->v[V_A], F->v[V_W], F->v[V_C],
                                 F->v[V_E], s);
    if (st) return st;
    launch_widen32(P->N, F->v[V_Q], 1.0, y, s);
    return TFDE_OK;
}

// z = P^{-1} r with the FP32 FFT DST-I passes
int fmix_apply_Pinv(const tfde_problem* P, const double* r, double* z, cudaStream_t s) {
    FftMixed* F = state(P);
    launch_to32(P->N, r, 1.0, F->v[V_R], nullptr, s);
    int st = op_Pinv32(P, F->v[V_R], F->v[V_Z], s);
    if (st) return st;
    launch_widen32(P->N, F->v[V_Z], 1.0, z, s);
    return TFDE_OK;
}

// FP64 iterative refinement around the FP32 inner PCG.
int fmix_pcg(tfde_problem* P, const double* b, double* x, double tol, int maxit, tfde_info* info, cudaStream_t s,
             bool r_given) {
    const auto t0 = clk::now();
    FftMixed* F = state(P);
    tfde_info loc{};
    double* r64 = P->w[tfde_problem::W_R];
    P->an_ready = false;
    double nb, nr;
    int st = start(P, b, x, r_given, &nb, &nr, s);
    if (st) return st;
    if (nb == 0.0) {
        if (info) *info = loc;
        return TFDE_OK;
    }
    loc.relres0 = nr / nb;
    int status = TFDE_ENOCONV;
    int stall = 0;
    while (true) {
        if (!std::isfinite(nr)) { status = set_error(TFDE_ENAN, "non-finite residual"); break; }
        if (nr <= tol * nb) { status = TFDE_OK; break; }
        if (loc.iters >= maxit) break;
        // inner target: 0.7 of what the sweep must reach; when that lies
        // below what one sweep can deliver, two sweeps share it evenly
        double theta = 0.7 * tol * nb / nr;
        if (theta < kInnerFloor32) theta = std::max(kInnerFloor32, std::sqrt(theta));
        // r32 = r 2^k, ||r32|| in [1/2, 1): an exact power-of-two scale
        const int k = -std::ilogb(nr) - 1;
        const double un = std::ldexp(nr, k);
        launch_to32(P->N, r64, std::ldexp(1.0, k), F->v[V_R], F->v[V_X], s);
        int it = 0;
        double reached = 1.0;
        if ((st = inner_pcg(P, theta, maxit - loc.iters, un * un, &it, &reached, s))) return st;
        loc.iters += it;
        loc.refine_sweeps++;
        launch_add32to64(P->N, std::ldexp(1.0, -k), F->v[V_X], x, s);
        const double nr_old = nr;
        if ((st = true_residual(P, b, x, r64, &nr, s))) return st;
        stall = (nr > 0.5 * nr_old) ? stall + 1 : 0;
        if (stall >= 2) {
            // refinement stopped contracting: finish with FP64 inner solves
            loc.fallback = 1;
            tfde_info sub{};
            status = pcg64(P, b, x, tol, maxit > loc.iters ? maxit - loc.iters : 1, &sub, s, false);
            loc.iters += sub.iters;
            nr = sub.relres * nb;
            break;
        }
    }
    loc.relres = nr / nb;
    if (status == TFDE_ENOCONV) set_error(TFDE_ENOCONV, "mixed PCG reached maxit");
    loc.ms = (float)std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    if (info) *info = loc;
    return status;
}

// FP64 iterative refinement around one FP32 GMRES(restart) cycle per sweep
// (restarted GMRES whose restarts start from the exact FP64 residual).
int fmix_pgmres(tfde_problem* P, const double* b, double* x, int restart, double tol, int maxit, tfde_info* info,
                cudaStream_t s, bool r_given) {
    const auto t0 = clk::now();
    FftMixed* F = state(P);
    tfde_info loc{};
    if (restart < 1 || restart > kMaxRestart) return set_error(TFDE_EINVAL, "restart must lie in 1..120");
    int st = ensure_basis(P, restart);
    if (st) return st;
    double* r64 = P->w[tfde_problem::W_R];
    P->an_ready = false;
    double nb, nr;
    if ((st = start(P, b, x, r_given, &nb, &nr, s))) return st;
    if (nb == 0.0) {
        if (info) *info = loc;
        return TFDE_OK;
    }
    loc.relres0 = nr / nb;
    int status = TFDE_ENOCONV;
    int stall = 0;
    double ratio = 1.0;   // observed true reduction / the preconditioned estimate's
    while (true) {
        if (!std::isfinite(nr)) { status = set_error(TFDE_ENAN, "non-finite residual"); break; }
        if (nr <= tol * nb) { status = TFDE_OK; break; }
        if (loc.iters >= maxit) break;
        double theta = 0.5 * tol * nb / nr / ratio;
        if (theta < kInnerFloor32) theta = std::max(kInnerFloor32, std::sqrt(theta));
        launch_to32(P->N, r64, 1.0 / nr, F->v[V_R], nullptr, s);
        int it = 0;
        double est = 1.0;
        if ((st = inner_gmres(P, restart, theta, maxit - loc.iters, &it, &est, s))) return st;
        loc.iters += it;
        loc.restarts++;
        loc.refine_sweeps++;
        launch_add32to64(P->N, nr, F->v[V_X], x, s);
        const double nr_old = nr;
        if ((st = true_residual(P, b, x, r64, &nr, s))) return st;
        if (est > 0.0) {
            const double observed = (nr / nr_old) / est;
            ratio = observed > 1.0 ? observed : 1.0;
        }
        stall = (nr > 0.5 * nr_old) ? stall + 1 : 0;
        if (stall >= 2) {
            loc.fallback = 1;
            tfde_info sub{};
            status = pgmres64(P, b, x, restart, tol, maxit > loc.iters ? maxit - loc.iters : 1, &sub, s, false);
            loc.iters += sub.iters;
            loc.restarts += sub.restarts;
            nr = sub.relres * nb;
            break;
        }
    }
    loc.relres = nr / nb;
    if (status == TFDE_ENOCONV) set_error(TFDE_ENOCONV, "mixed PGMRES reached maxit");
    loc.ms = (float)std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    if (info) *info = loc;
    return status;
}

}  // namespace tfde
