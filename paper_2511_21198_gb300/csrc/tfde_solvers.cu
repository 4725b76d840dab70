// FP64 operator, preconditioner and Krylov solvers of libtfde, and the
// Crank-Nicolson step driver (Sec. 2 Eq. (CN), Eq. (linear_sys); Sec. 3).
#include <chrono>
#include <cmath>
#include <utility>
#include <vector>

#include "tfde_fft.h"
#include "tfde_internal.h"
#include "tfde_givens.h"

namespace tfde {

#define TFDE_CUDA_TRY(expr)                                                              \
    do {                                                                                  \
        cudaError_t e__ = (expr);                                                         \
        if (e__ != cudaSuccess)                                                           \
            return set_error(TFDE_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e__)); \
    } while (0)

static int check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(TFDE_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return TFDE_OK;
}

// A x (op TFDE_OP_A) or (2 A_N - A) x (op TFDE_OP_RHS), Eq. (linear_sys), as
// three axis passes:  a = (M1 +- eta1 B1) x,  w = M1 x;
//                     c = M2 a +- eta2 B2 w,  e = M2 w;
//                     y = M3 c +- eta3 B3 e.
int apply_A64(const tfde_problem* P, int op, const double* x, double* y, cudaStream_t s) {
    if (P->fft)   // FFT-embedded Toeplitz passes (O(n log n) per line)
        return fft::apply_A<double>(P, op, x, y, P->w[tfde_problem::W_A], P->w[tfde_problem::W_W],
                                    P->w[tfde_problem::W_C], P->w[tfde_problem::W_E], s);
    const bool rhs = (op & 1) != 0;
    const bool stiff = (op & TFDE_OP_STIFF) != 0;   // (A - A_N) x: no mass term in the x pass
    const double sg = rhs ? -1.0 : 1.0;
    const AxisView vx = axis_view(P->n, 0), vy = axis_view(P->n, 1), vz = axis_view(P->n, 2);
    double* a = P->w[tfde_problem::W_A];
    double* w = P->w[tfde_problem::W_W];
    double* c = P->w[tfde_problem::W_C];
    double* e = P->w[tfde_problem::W_E];
    if (stiff) launch_axis_gemm_f64(P->G[0], x, a, vx, sg, nullptr, 0.0, s);
    else launch_axis_gemm_f64(P->Ghat[rhs ? 1 : 0], x, a, vx, 1.0, nullptr, 0.0, s);
    launch_axis_stencil_f64(x, w, vx, 1.0, nullptr, 0.0, s);
    launch_axis_gemm_f64(P->G[1], w, c, vy, sg, a, 1.0, s);
    launch_axis_stencil_f64(w, e, vy, 1.0, nullptr, 0.0, s);
    launch_axis_gemm_f64(P->G[2], e, y, vz, sg, c, 1.0, s);
    return check_launch("apply_A64");
}

// z = S_N Lambda^{-1} S_N r (Eq. (diag_tau_pre)); S_n symmetric, S_n^2 = I.
int apply_Pinv64(const tfde_problem* P, const double* r, double* z, cudaStream_t s) {
    if (P->fft)   // DST-I by FFT (Bluestein), the z pair and Lambda^{-1} in one pass
        return fft::apply_Pinv<double>(P, r, z, P->w[tfde_problem::W_A], P->w[tfde_problem::W_C], s);
    const AxisView vx = axis_view(P->n, 0), vy = axis_view(P->n, 1), vz = axis_view(P->n, 2);
    double* t1 = P->w[tfde_problem::W_A];
    double* t2 = P->w[tfde_problem::W_C];
    launch_axis_gemm_f64(P->S[0], r, t1, vx, 1.0, nullptr, 0.0, s);
    launch_axis_gemm_f64(P->S[1], t1, t2, vy, 1.0, nullptr, 0.0, s);
    launch_axis_gemm_f64(P->S[2], t2, t1, vz, 1.0, nullptr, 0.0, s);
    launch_lambda_scale_f64(t1, t1, P->lam, P->n, P->csum, 1, s);
    launch_axis_gemm_f64(P->S[2], t1, t2, vz, 1.0, nullptr, 0.0, s);
    launch_axis_gemm_f64(P->S[1], t2, t1, vy, 1.0, nullptr, 0.0, s);
    launch_axis_gemm_f64(P->S[0], t1, z, vx, 1.0, nullptr, 0.0, s);
    return check_launch("apply_Pinv64");
}

// out[j] = <V_j, w>, j < m (host output; synchronises the stream).
int dots64(const tfde_problem* P, int m, const double* V, size_t ldv, const double* w, double* out,
           cudaStream_t s) {
    launch_multidot_f64(P->N, m, V, ldv, w, P->red, P->nblk, s);
    launch_reduce_finish(P->red, P->nblk, m, P->red_out, s);
    TFDE_CUDA_TRY(cudaGetLastError());
    TFDE_CUDA_TRY(cudaMemcpyAsync(P->red_host, P->red_out, m * sizeof(double), cudaMemcpyDeviceToHost, s));
    TFDE_CUDA_TRY(cudaStreamSynchronize(s));
    for (int j = 0; j < m; ++j) out[j] = P->red_host[j];
    return TFDE_OK;
}

static int dot(const tfde_problem* P, const double* a, const double* b, double* out, cudaStream_t s) {
    return dots64(P, 1, a, 0, b, out, s);
}

// The (u, A u) history of the extrapolated initial guess: allocated by
// tfde_set_guess_order / tfde_batch_set_guess_order (order > 0), not by a solve.
int ensure_history(tfde_problem* P) {
    if (P->H[0][0]) return TFDE_OK;
    for (auto& hk : P->H)
        for (auto& v : hk)
            if (cudaMalloc((void**)&v, P->N * sizeof(double)) != cudaSuccess)
                return set_error(TFDE_ENOMEM, "cudaMalloc of the extrapolation history failed");
    P->hist = 0;
    return TFDE_OK;
}

int ensure_gmres_basis(tfde_problem* P, int restart) {
    if (P->gmres_cap >= restart) return TFDE_OK;
    cudaFree(P->V);
    P->V = nullptr;
    P->gmres_cap = 0;
    if (cudaMalloc((void**)&P->V, (size_t)(restart + 1) * P->N * sizeof(double)) != cudaSuccess)
        return set_error(TFDE_ENOMEM, "cudaMalloc of the GMRES basis failed");
    P->gmres_cap = restart;
    return TFDE_OK;
}

namespace {

using clk = std::chrono::steady_clock;

double ms_since(clk::time_point t0) {
    return std::chrono::duration<double, std::milli>(clk::now() - t0).count();
}

// r = b - A x into `r`; returns ||r||.
int true_residual(const tfde_problem* P, const double* b, const double* x, double* r, double* nrm,
                  cudaStream_t s) {
    double* q = P->w[tfde_problem::W_Q];
    int st = apply_A64(P, TFDE_OP_A, x, q, s);
    if (st) return st;
    launch_axpbypz_f64(P->N, 1.0, b, -1.0, q, r, s);
    double rr;
    if ((st = dot(P, r, r, &rr, s))) return st;
    *nrm = std::sqrt(rr);
    return TFDE_OK;
}

}  // namespace

// Preconditioned CG (Sec. 3.1) in FP64, true-residual stopping test.
int pcg64(const tfde_problem* P, const double* b, double* x, double tol, int maxit, tfde_info* info,
          cudaStream_t s, bool r_given) {
    const auto t0 = clk::now();
    tfde_info loc{};
    double* r = P->w[tfde_problem::W_R];
    double* z = P->w[tfde_problem::W_Z];
    double* p = P->w[tfde_problem::W_P];
    double* q = P->w[tfde_problem::W_Q];
    int st;
    double bb;
    if ((st = dot(P, b, b, &bb, s))) return st;
    const double nb = std::sqrt(bb);
    if (!std::isfinite(nb)) return set_error(TFDE_ENAN, "non-finite right-hand side");
    if (nb == 0.0) {
        TFDE_CUDA_TRY(cudaMemsetAsync(x, 0, P->N * sizeof(double), s));
        loc.relres = loc.relres0 = 0.0;
        if (info) *info = loc;
        return TFDE_OK;
    }
    double nr;
    if (r_given) {
        double rr0;
        if ((st = dot(P, r, r, &rr0, s))) return st;
        nr = std::sqrt(rr0);
    } else if ((st = true_residual(P, b, x, r, &nr, s))) {
        return st;
    }
    loc.relres0 = nr / nb;
    int status = TFDE_ENOCONV;
    if (!std::isfinite(nr)) {
        status = set_error(TFDE_ENAN, "non-finite initial residual");
    } else if (nr <= tol * nb) {
        status = TFDE_OK;
        loc.relres = nr / nb;
    } else {
        if ((st = apply_Pinv64(P, r, z, s))) return st;
        TFDE_CUDA_TRY(cudaMemcpyAsync(p, z, P->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
        double rz;
        if ((st = dot(P, r, z, &rz, s))) return st;
        while (loc.iters < maxit) {
            if ((st = apply_A64(P, TFDE_OP_A, p, q, s))) return st;
            double pq;
            if ((st = dot(P, p, q, &pq, s))) return st;
            if (!std::isfinite(pq)) { status = set_error(TFDE_ENAN, "non-finite p.Ap"); break; }
            if (!(pq > 0.0)) { status = set_error(TFDE_EBREAKDOWN, "PCG breakdown: p.Ap <= 0"); break; }
            const double alpha = rz / pq;
            launch_cg_update_f64(P->N, alpha, p, q, x, r, P->red, P->nblk, s);
            launch_reduce_finish(P->red, P->nblk, 1, P->red_out, s);
            TFDE_CUDA_TRY(cudaMemcpyAsync(P->red_host, P->red_out, sizeof(double), cudaMemcpyDeviceToHost, s));
            TFDE_CUDA_TRY(cudaStreamSynchronize(s));
            const double rr = P->red_host[0];
            loc.iters++;
            if (!std::isfinite(rr)) { status = set_error(TFDE_ENAN, "non-finite residual"); break; }
            if (std::sqrt(rr) <= tol * nb) {
                if ((st = true_residual(P, b, x, r, &nr, s))) return st;
                if (nr <= tol * nb) {
                    status = TFDE_OK;
                    loc.relres = nr / nb;
                    break;
                }
                // recursive residual drifted: restart from the true one
                if ((st = apply_Pinv64(P, r, z, s))) return st;
                TFDE_CUDA_TRY(cudaMemcpyAsync(p, z, P->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
                if ((st = dot(P, r, z, &rz, s))) return st;
                continue;
            }
            if ((st = apply_Pinv64(P, r, z, s))) return st;
            double rz_new;
            if ((st = dot(P, r, z, &rz_new, s))) return st;
            const double beta = rz_new / rz;
            rz = rz_new;
            launch_axpby_f64(P->N, 1.0, z, beta, p, s);
        }
        if (status == TFDE_ENOCONV) {
            if ((st = true_residual(P, b, x, r, &nr, s))) return st;
            loc.relres = nr / nb;
            set_error(TFDE_ENOCONV, "PCG reached maxit");
        }
    }
    loc.ms = (float)ms_since(t0);
    if (info) *info = loc;
    return status;
}


// Left-preconditioned restarted GMRES (Sec. 3.2, Eq. (one_side_system)), FP64,
// classical Gram-Schmidt with one re-orthogonalisation.  Converged when the
// true relative residual meets tol; the cycle stops on the preconditioned
// residual estimate, scaled by the observed true/preconditioned ratio.
int pgmres64(tfde_problem* P, const double* b, double* x, int restart, double tol, int maxit, tfde_info* info,
             cudaStream_t s, bool r_given) {
    const auto t0 = clk::now();
    tfde_info loc{};
    int st;
    if ((st = ensure_gmres_basis(P, restart))) return st;
    double* r = P->w[tfde_problem::W_R];
    double* q = P->w[tfde_problem::W_Q];
    double* V = P->V;
    const size_t N = P->N;
    double bb;
    if ((st = dot(P, b, b, &bb, s))) return st;
    const double nb = std::sqrt(bb);
    if (!std::isfinite(nb)) return set_error(TFDE_ENAN, "non-finite right-hand side");
    if (nb == 0.0) {
        TFDE_CUDA_TRY(cudaMemsetAsync(x, 0, N * sizeof(double), s));
        if (info) *info = loc;
        return TFDE_OK;
    }
    double nr;
    if (r_given) {
        double rr0;
        if ((st = dot(P, r, r, &rr0, s))) return st;
        nr = std::sqrt(rr0);
    } else if ((st = true_residual(P, b, x, r, &nr, s))) {
        return st;
    }
    loc.relres0 = nr / nb;
    double ratio = 1.0;  // observed (true relres) / (preconditioned relres)
    int status = TFDE_ENOCONV;
    std::vector<double> h(restart + 2), h2(restart + 2), y;
    double* hdev = P->red_out + 128;
    while (true) {
        if (!std::isfinite(nr)) { status = set_error(TFDE_ENAN, "non-finite residual"); break; }
        if (nr <= tol * nb) { status = TFDE_OK; break; }
        if (loc.iters >= maxit) break;
        // V_0 = P^{-1} r / beta
        if ((st = apply_Pinv64(P, r, V, s))) return st;
        double beta2;
        if ((st = dot(P, V, V, &beta2, s))) return st;
        const double beta = std::sqrt(beta2);
        if (!(beta > 0.0) || !std::isfinite(beta)) { status = set_error(TFDE_EBREAKDOWN, "zero preconditioned residual"); break; }
        launch_axpby_f64(N, 0.0, V, 1.0 / beta, V, s);
        GivensLS ls(restart);
        ls.g[0] = beta;
        // cycle target: ask the preconditioned estimate for half the reduction
        // the true residual still needs, corrected by the ratio observed before
        const double ptarget = beta * (tol * nb / nr) * 0.5 / ratio;
        int k = 0;
        double est = beta;
        for (int j = 0; j < restart && loc.iters < maxit; ++j) {
            double* vj = V + (size_t)j * N;
            double* w = V + (size_t)(j + 1) * N;
            if ((st = apply_A64(P, TFDE_OP_A, vj, q, s))) return st;
            if ((st = apply_Pinv64(P, q, w, s))) return st;
            // CGS2: two rounds of h = V^T w, w -= V h
            if ((st = dots64(P, j + 1, V, N, w, h.data(), s))) return st;
            TFDE_CUDA_TRY(cudaMemcpyAsync(hdev, h.data(), (j + 1) * sizeof(double), cudaMemcpyHostToDevice, s));
            launch_multiaxpy_f64(N, j + 1, V, N, hdev, w, s);
            if ((st = dots64(P, j + 1, V, N, w, h2.data(), s))) return st;
            TFDE_CUDA_TRY(cudaMemcpyAsync(hdev, h2.data(), (j + 1) * sizeof(double), cudaMemcpyHostToDevice, s));
            launch_multiaxpy_f64(N, j + 1, V, N, hdev, w, s);
            for (int i = 0; i <= j; ++i) h[i] += h2[i];
            double ww;
            if ((st = dot(P, w, w, &ww, s))) return st;
            const double hn = std::sqrt(ww);
            h[j + 1] = hn;
            if (!std::isfinite(hn)) { status = set_error(TFDE_ENAN, "non-finite Arnoldi vector"); break; }
            est = ls.add_column(j, h.data());
            loc.iters++;
            k = j + 1;
            if (est <= ptarget || hn == 0.0) break;
            launch_axpby_f64(N, 0.0, w, 1.0 / hn, w, s);
        }
        if (status == TFDE_ENAN) break;
        loc.restarts++;
        if (k > 0) {
            ls.solve(k, y);
            for (int i = 0; i < k; ++i) y[i] = -y[i];
            TFDE_CUDA_TRY(cudaMemcpyAsync(hdev, y.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
            launch_multiaxpy_f64(N, k, V, N, hdev, x, s);  // x += V y
        }
        const double nr_old = nr;
        if ((st = true_residual(P, b, x, r, &nr, s))) return st;
        if (est > 0.0 && nr_old > 0.0) {
            const double observed = (nr / nr_old) / (est / beta);
            ratio = observed > 1.0 ? observed : 1.0;
        }
    }
    loc.relres = nr / nb;
    if (status == TFDE_ENOCONV) set_error(TFDE_ENOCONV, "PGMRES reached maxit");
    loc.ms = (float)ms_since(t0);
    if (info) *info = loc;
    return status;
}

int mixed_pcg(tfde_problem*, const double*, double*, double, int, tfde_info*, cudaStream_t, bool);
int mixed_pgmres(tfde_problem*, const double*, double*, int, double, int, tfde_info*, cudaStream_t, bool);
int accurate_apply(const tfde_problem*, int, const double*, double*, cudaStream_t);
int accurate_apply_ex(const tfde_problem*, int, const double*, double*, int, const double*, double, cudaStream_t, int,
                      double*, int, double*);

// A_N u into `out` (the three tridiagonal sweeps in one pass).
static void mass_apply(const tfde_problem* P, const double* u, double* out, cudaStream_t s) {
    if (P->dim2) {   // A_2 (x) A_1: the x and y sweeps (W_E as the intermediate)
        double* t = P->w[tfde_problem::W_E];
        launch_axis_stencil_f64(u, t, axis_view(P->n, 0), 1.0, nullptr, 0.0, s);
        launch_axis_stencil_f64(t, out, axis_view(P->n, 1), 1.0, nullptr, 0.0, s);
        return;
    }
    launch_mass3d_f64(u, out, P->n, s);
}

void io_wait_input(tfde_problem* P, cudaStream_t s) {
    if (!P->io.in_pending) return;
    cudaStreamWaitEvent(s, P->io.ev_in, 0);
    P->io.in_pending = false;
}

void io_offer_output(tfde_problem* P, const double* x, cudaStream_t s) {
    if (!P->io.out || x != P->io.dev) return;
    cudaEventRecord(P->io.ev_ready, s);
    cudaStreamWaitEvent(P->io.stream, P->io.ev_ready, 0);
    cudaMemcpyAsync(P->io.out, P->io.dev, P->N * sizeof(double), cudaMemcpyDeviceToHost, P->io.stream);
    cudaEventRecord(P->io.ev_out, P->io.stream);
    P->io.out_pending = true;
    P->io.out_valid = true;
}

void io_before_write(tfde_problem* P, const double* x, cudaStream_t s) {
    if (!P->io.out || x != P->io.dev) return;
    io_wait_input(P, s);
    if (P->io.out_pending) {
        cudaStreamWaitEvent(s, P->io.ev_out, 0);
        P->io.out_pending = false;
    }
    P->io.out_valid = false;
}

// Coefficients g of the corrected guess x0 = g0 u^{m-1} + g1 u^{m-2} +
// g2 u^{m-3}, into g (device): the order-2 extrapolation x_e = 3 u^{m-1} -
// 3 u^{m-2} + u^{m-3} plus c1 d1 + c2 d2 (d1 = u^{m-1} - u^{m-2}, d2 =
// u^{m-1} - 2 u^{m-2} + u^{m-3}), c minimising the residual ||r_e - c1 A d1 -
// c2 A d2|| over the stored A u of the history (normal equations of the five
// sums of cn_mr_dots_kernel, solved by one device thread: no host read).  The
// polynomial coefficients are not optimal for the CN transient of the stiff
// modes; the correction uses no operator application.
static void mr_guess_coefficients(tfde_problem* P, const double* an, const double* F, const double* b,
                                  const double* r, double* g, cudaStream_t s) {
    launch_cn_mr_dots(P->N, an, F, P->p.dt, b, r, P->H[0][1], P->H[1][1], P->red, P->red_out + kMrSlot, s);
    launch_cn_mr_coefficients(P->red_out + kMrSlot, g, s);
}

// One CN step (Eq. (CN), Eq. (linear_sys)) for either precision.  `chained`:
// W_B / W_R hold b^{m-1} and the final true residual of u_prev, so that
// A u_prev = b^{m-1} - r^{m-1} replaces the operator application.
// cn_prepare forms b^m in W_B, the initial guess in u_next and (when *r_given)
// its residual in W_R; cn_drive then runs the solver.
int cn_prepare(tfde_problem* P, const double* u_prev, const double* F, const double* x0, double* u_next,
               cudaStream_t s, bool chained, bool* r_given, const double* guess, int* used_guess) {
    double* b = P->w[tfde_problem::W_B];
    double* r = P->w[tfde_problem::W_R];
    double* an = P->w[tfde_problem::W_T];
    const bool mixed_prec = P->mixed != nullptr;   // the tensor-core path's exact-slice products
    const bool guess_is_prev = (x0 == nullptr || x0 == u_prev);
    int st;
    // A_N u_prev: left in W_T by the mixed solver's last (full-width) residual
    // of a chained step, whose z-pass digit slicing forms it exactly; else the
    // fused stencil
    if (!(chained && P->an_ready)) {
        io_wait_input(P, s);
        mass_apply(P, u_prev, an, s);
    }
    P->an_ready = false;
    bool guess_in_place = false;  // x0 already written into u_next, r = b - A x0
    if (used_guess) *used_guess = 0;
    if (chained && P->guess_order > 0 && u_next == u_prev && !guess) {
        if ((st = ensure_history(P))) return st;   // allocated when the order was set
        const int order = P->guess_order < P->hist ? P->guess_order : P->hist;
        double* gp = nullptr;   // device coefficients of the corrected guess
        if (P->guess_order >= 3 && P->hist >= 2) {
            gp = P->red_out + kMrSlot + 5;
            mr_guess_coefficients(P, an, F, b, r, gp, s);   // reads no u: overlaps a host copy of u
        }
        if (P->io.in_pending && P->io.nchunks > 1 && u_next == P->io.dev) {
            // u arrives from the host in pieces: each range starts when its piece is in
            launch_cn_chain_extrap_chunks(P->N, P->io.nchunks, P->io.ev_chunk, an, F, P->p.dt, b, r, u_next,
                                          P->H[0][0], P->H[0][1], P->H[1][0], P->H[1][1],
                                          gp ? 3 : std::min(order, 2), gp, P->red, P->red_out + kNormsSlot, s);
            io_wait_input(P, s);
        } else {
            io_wait_input(P, s);
            launch_cn_chain_extrap(P->N, an, F, P->p.dt, b, r, u_next, P->H[0][0], P->H[0][1], P->H[1][0],
                                   P->H[1][1], gp ? 3 : std::min(order, 2), gp, P->red, P->red_out + kNormsSlot, s);
        }
        std::swap(P->H[0][0], P->H[1][0]);
        std::swap(P->H[0][1], P->H[1][1]);
        P->hist = P->hist < 2 ? P->hist + 1 : 2;
        guess_in_place = true;
    } else if (chained) {
        if (guess) P->hist = 0;
        io_wait_input(P, s);
        launch_cn_chain(P->N, an, F, P->p.dt, b, r, P->red, P->red_out + kNormsSlot, s);
    } else {
        P->hist = 0;
        io_wait_input(P, s);
        double* ku = P->w[tfde_problem::W_Q];
        st = mixed_prec ? accurate_apply(P, TFDE_OP_STIFF, u_prev, ku, s) : apply_A64(P, TFDE_OP_STIFF, u_prev, ku, s);
        if (st) return st;
        launch_cn_first(P->N, an, ku, F, P->p.dt, b, r, P->red, P->red_out + kNormsSlot, s);
        if (P->guess_order > 0 && P->H[0][0] && P->H[0][1]) {
            // the restart has A u^{m-1} = A_N u + K u at hand: it becomes the
            // history's first level, so that the next chained step extrapolates
            launch_history_first(P->N, u_prev, an, ku, P->H[0][0], P->H[0][1], s);
            P->hist = 1;
        }
    }
    const double* start = guess_is_prev ? u_prev : x0;
    io_wait_input(P, s);
    if (!guess_in_place && start != u_next)
        TFDE_CUDA_TRY(cudaMemcpyAsync(u_next, start, P->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    *r_given = guess_is_prev;  // r = b - A x0 is the residual of the initial guess
    P->norms_ready = guess_is_prev;
    if (guess && guess_is_prev) {
        // candidate guess: r_g = r - A (guess - u_prev); keep it if its FP64
        // residual is smaller than that of u_prev (the previous-step guess)
        double* d = P->w[tfde_problem::W_P];
        double* rg = P->w[tfde_problem::W_Z];
        launch_axpbypz_f64(P->N, 1.0, guess, -1.0, u_prev, d, s);
        if (mixed_prec) {
            st = accurate_apply_ex(P, TFDE_OP_A, d, rg, -1, r, 1.0, s, 7, nullptr, 0, nullptr);
        } else {
            st = apply_A64(P, TFDE_OP_A, d, rg, s);
            if (!st) launch_axpby_f64(P->N, 1.0, r, -1.0, rg, s);
        }
        if (st) return st;
        // the point of the line u_prev + c (guess - u_prev) with the least
        // residual: r(c) = (1 - c) r + c r_g, c = <r, r - r_g> / ||r - r_g||^2
        // (c = 1: the candidate itself, c = 0: the previous-step guess)
        double rr[3];
        if ((st = dots64(P, 1, r, 0, r, &rr[0], s)) || (st = dots64(P, 1, rg, 0, rg, &rr[1], s)) ||
            (st = dots64(P, 1, r, 0, rg, &rr[2], s)))
            return st;
        const double den = rr[0] - 2.0 * rr[2] + rr[1];
        double c = den > 0.0 ? (rr[0] - rr[2]) / den : 0.0;
        if (!std::isfinite(c) || c < 0.0 || c > 4.0) c = (std::isfinite(rr[1]) && rr[1] < rr[0]) ? 1.0 : 0.0;
        const double rc2 = (1.0 - c) * (1.0 - c) * rr[0] + 2.0 * c * (1.0 - c) * rr[2] + c * c * rr[1];
        if (c > 0.0 && std::isfinite(rc2) && rc2 < rr[0]) {
            if (c == 1.0) {
                TFDE_CUDA_TRY(cudaMemcpyAsync(u_next, guess, P->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
                TFDE_CUDA_TRY(cudaMemcpyAsync(r, rg, P->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
            } else {
                launch_axpby_f64(P->N, c, guess, 1.0 - c, u_next, s);   // u_next = (1 - c) u_prev + c guess
                launch_axpby_f64(P->N, c, rg, 1.0 - c, r, s);
            }
            P->norms_ready = false;
            if (used_guess) *used_guess = 1;
        }
    }
    return TFDE_OK;
}

int cn_drive(tfde_problem* P, const double* u_prev, const double* F, const double* x0, double* u_next, double tol,
             tfde_info* info, cudaStream_t s, bool chained, const double* guess, int* used_guess) {
    bool rg = false;
    int st = cn_prepare(P, u_prev, F, x0, u_next, s, chained, &rg, guess, used_guess);
    if (st) return st;
    double* b = P->w[tfde_problem::W_B];
    if (P->fmix)
        return P->symmetric ? fmix_pcg(P, b, u_next, tol, 10000, info, s, rg)
                            : fmix_pgmres(P, b, u_next, 20, tol, 10000, info, s, rg);
    const bool mixed_prec = P->prec == TFDE_MIXED;
    if (P->symmetric)
        return mixed_prec ? mixed_pcg(P, b, u_next, tol, 10000, info, s, rg) : pcg64(P, b, u_next, tol, 10000, info, s, rg);
    return mixed_prec ? mixed_pgmres(P, b, u_next, 20, tol, 10000, info, s, rg)
                      : pgmres64(P, b, u_next, 20, tol, 10000, info, s, rg);
}

}  // namespace tfde
