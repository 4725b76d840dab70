// Host-side assembly of a tfde_problem (Sec. 2 and Sec. 3 of the paper):
// generator coefficients, per-axis dense operators, DST-I matrices, the 1-D
// eigenvalue arrays of the tau preconditioner and the 1-D cell averages of
// the Example 2 source.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "tfde_fft.h"
#include "tfde_internal.h"

namespace tfde {

namespace {
thread_local std::string g_err;
}

int set_error(int status, const std::string& msg) {
    g_err = msg;
    return status;
}

const char* last_error_text() { return g_err.c_str(); }

namespace {

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_N).
void gauss_legendre(int N, std::vector<double>& x, std::vector<double>& w) {
    x.assign(N, 0.0);
    w.assign(N, 0.0);
    for (int i = 0; i < (N + 1) / 2; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (N + 0.5));
        double pp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= N; ++j) {
                const double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = N * (z * p1 - p2) / (z * z - 1.0);
            const double dz = p1 / pp;
            z -= dz;
            if (std::fabs(dz) < 1e-17) break;
        }
        x[i] = -z;
        x[N - 1 - i] = z;
        w[i] = w[N - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

// Generator q_k^{(d)}, k = 0..n (Eq. (coef_expression)).  q_0..q_2 come from
// the defining powers in extended precision; for k >= 3 the third difference
// q_k = -[g(k+1/2) - 3g(k-1/2) + 3g(k-3/2) - g(k-5/2)], g(x) = x^d, is
// evaluated without cancellation as -int_0^3 B2(t) g'''(k - 5/2 + t) dt
// (B2: the quadratic B-spline, the Peano kernel of the third difference),
// by 24-point Gauss-Legendre on each polynomial piece of B2.
std::vector<double> generator_q(double d, int n) {
    std::vector<double> q(n + 1, 0.0);
    const long double D = d;
    const long double a = powl(0.5L, D), b = powl(1.5L, D), c = powl(2.5L, D);
    q[0] = (double)(-a);
    if (n >= 1) q[1] = (double)(3.0L * a - b);
    if (n >= 2) q[2] = (double)(3.0L * b - 3.0L * a - c);
    if (n >= 3) {
        std::vector<double> gx, gw;
        gauss_legendre(24, gx, gw);
        const double c3 = d * (d - 1.0) * (d - 2.0);
        for (int k = 3; k <= n; ++k) {
            const double a0 = k - 2.5;
            double sum = 0.0;
            for (int piece = 0; piece < 3; ++piece) {
                for (int g = 0; g < 24; ++g) {
                    const double t = piece + 0.5 * (gx[g] + 1.0);  // node in [piece, piece+1]
                    double bs;
                    if (piece == 0) bs = 0.5 * t * t;
                    else if (piece == 1) bs = 0.5 * (-2.0 * t * t + 6.0 * t - 3.0);
                    else bs = 0.5 * (3.0 - t) * (3.0 - t);
                    sum += 0.5 * gw[g] * bs * std::pow(a0 + t, d - 3.0);
                }
            }
            q[k] = -c3 * sum;
        }
    }
    return q;
}

// sin(pi * r / (n+1)) with r reduced exactly modulo 2(n+1).
double sin_pi_frac(long long r, int n) {
    const long long period = 2LL * (n + 1);
    r %= period;
    if (r < 0) r += period;
    return std::sin(M_PI * (double)r / (double)(n + 1));
}

double cos_pi_frac(long long r, int n) {
    const long long period = 2LL * (n + 1);
    r %= period;
    if (r < 0) r += period;
    return std::cos(M_PI * (double)r / (double)(n + 1));
}

// tau(H(T_n)) eigenvalues (Lemma 1D_tau_SPD), k = 1..n:
//   q_1 + (q_0 + q_2) cos t_k + sum_{j=2}^{n-1} q_{j+1} cos(j t_k),  t_k = k pi/(n+1).
std::vector<double> tau_eigs(const std::vector<double>& q, int n) {
    std::vector<double> lam(n);
    for (int k = 1; k <= n; ++k) {
        double v = q[1];
        if (n >= 2) v += (q[0] + q[2]) * cos_pi_frac(k, n);
        for (int j = 2; j <= n - 1; ++j) v += q[j + 1] * cos_pi_frac((long long)j * k, n);
        lam[k - 1] = v;
    }
    return lam;
}

// Average over [c - h/2, c + h/2] of x^p for c > 0, written as
// c^p * sum_{k>=0} C(p, 2k) u^{2k} / (2k+1) with u = h/(2c) <= 1/2.
double cell_avg_pow(double c, double h, double p) {
    const double u = h / (2.0 * c);
    const double u2 = u * u;
    double term = 1.0, sum = 1.0;  // k = 0
    for (int k = 1; k < 200; ++k) {
        // C(p,2k) = C(p,2k-2) * (p-2k+2)(p-2k+1) / ((2k-1)(2k))
        term *= (p - 2.0 * k + 2.0) * (p - 2.0 * k + 1.0) / ((2.0 * k - 1.0) * (2.0 * k)) * u2;
        const double add = term / (2.0 * k + 1.0);
        sum += add;
        if (std::fabs(add) < 1e-18 * std::fabs(sum)) break;
    }
    return std::pow(c, p) * sum;
}

// Example 2 (Sec. 4): 1-D dual-cell averages of P(x) = x^2 (1-x)^2 and of
// S_d(x) = sum_k (-1)^{2-k} C(2,k) Gamma(5-k)/Gamma(3-k+d) [k+ x^{2-k+d} + k- (1-x)^{2-k+d}].
void example2_1d(int n, double d, double kp, double km, std::vector<double>& P, std::vector<double>& S) {
    const double h = 1.0 / (n + 1);
    P.assign(n, 0.0);
    S.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        const double c = (i + 1) * h;
        // P is a quartic: its cell average is P(c) + (h^2/24) P''(c) + (h^4/1920) P''''(c)
        const double Pc = c * c * (1.0 - c) * (1.0 - c);
        const double P2 = 2.0 - 12.0 * c + 12.0 * c * c;
        P[i] = Pc + h * h / 24.0 * P2 + h * h * h * h / 80.0;
        double s = 0.0;
        for (int k = 0; k <= 2; ++k) {
            const double binom = (k == 1) ? 2.0 : 1.0;
            const double sign = ((2 - k) % 2 == 0) ? 1.0 : -1.0;
            const double coef = sign * binom * std::tgamma(5.0 - k) / std::tgamma(3.0 - k + d);
            const double p = 2.0 - k + d;
            s += coef * (kp * cell_avg_pow(c, h, p) + km * cell_avg_pow(1.0 - c, h, p));
        }
        S[i] = s;
    }
}

template <typename T>
int dalloc(T** p, size_t count) {
    if (cudaMalloc((void**)p, count * sizeof(T)) != cudaSuccess)
        return set_error(TFDE_ENOMEM, "cudaMalloc failed");
    return TFDE_OK;
}

int upload(double* d, const std::vector<double>& h, cudaStream_t s) {
    if (cudaMemcpyAsync(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return set_error(TFDE_ECUDA, "cudaMemcpyAsync H2D failed");
    return cudaStreamSynchronize(s) == cudaSuccess ? TFDE_OK : set_error(TFDE_ECUDA, "stream sync failed");
}

}  // namespace

int validate_params(const tfde_params* p) {
    const int dims = p->n[2] == 0 ? 2 : 3;   // n[2] = 0: the 2-D problem
    for (int a = 0; a < dims; ++a) {
        if (p->n[a] < 1) return set_error(TFDE_EINVAL, "n must be >= 1 on every axis");
        if (!(p->delta[a] > 0.0 && p->delta[a] < 1.0)) return set_error(TFDE_EINVAL, "delta must lie in (0,1)");
        if (!(p->kp[a] > 0.0) || !(p->km[a] > 0.0)) return set_error(TFDE_EINVAL, "k_+ and k_- must be > 0");
        if (!(p->hi[a] > p->lo[a])) return set_error(TFDE_EINVAL, "need lo < hi on every axis");
    }
    if (!(p->dt > 0.0)) return set_error(TFDE_EINVAL, "dt must be > 0");
    const double N = (double)p->n[0] * p->n[1] * (dims == 3 ? p->n[2] : 1);
    if (N > 2.0e9) return set_error(TFDE_EINVAL, "grid too large");
    return TFDE_OK;
}

int mixed_init(tfde_problem* P, cudaStream_t s);   // tfde_mixed.cu
void mixed_free(tfde_problem* P);
int destroy_problem(tfde_problem* P);

int assemble_problem(const tfde_params* params, int precision, cudaStream_t s, tfde_problem** out) {
    *out = nullptr;
    int st = validate_params(params);
    if (st) return st;
    if (precision != TFDE_FP64 && precision != TFDE_MIXED) return set_error(TFDE_EINVAL, "unknown precision");
    tfde_problem* P = new tfde_problem();
    P->p = *params;
    P->prec = precision;
    for (int a = 0; a < 3; ++a) P->n[a] = params->n[a];
    if (params->n[2] == 0) {
        // the 2-D problem: a third axis of one point with an identity mass
        // factor and no stiffness term reproduces the 2-D system exactly
        P->dim2 = true;
        P->n[2] = 1;
        P->p.n[2] = 1;
        P->p.delta[2] = 0.5;
        P->p.kp[2] = P->p.km[2] = 1.0;
        P->p.lo[2] = 0.0;
        P->p.hi[2] = 1.0;
    }
    params = &P->p;
    P->N = (size_t)P->n[0] * P->n[1] * P->n[2];
    P->symmetric = true;
    for (int a = 0; a < 3; ++a) {
        const int n = P->n[a];
        const double d = params->delta[a];
        P->h[a] = (params->hi[a] - params->lo[a]) / (n + 1);
        P->eta[a] = params->dt / (2.0 * std::tgamma(d + 1.0) * std::pow(P->h[a], 2.0 - d));
        if (P->dim2 && a == 2) P->eta[a] = 0.0;
        P->csum[a] = P->eta[a] * (params->kp[a] + params->km[a]);
        if (params->kp[a] != params->km[a]) P->symmetric = false;
        P->q[a] = generator_q(d, n);
        P->lam_tau[a] = tau_eigs(P->q[a], n);
        P->lam_mass[a].resize(n);
        for (int k = 1; k <= n; ++k) P->lam_mass[a][k - 1] = (6.0 + 2.0 * cos_pi_frac(k, n)) / 8.0;
        if (P->dim2 && a == 2) P->lam_mass[a][0] = 1.0;
    }
    P->have_src = true;
    for (int a = 0; a < 3; ++a)
        if (params->lo[a] != 0.0 || params->hi[a] != 1.0) P->have_src = false;
    if (P->have_src)
        for (int a = 0; a < 3; ++a)
            example2_1d(P->n[a], params->delta[a], params->kp[a], params->km[a], P->srcP[a], P->srcS[a]);
    if (P->have_src && P->dim2) {   // Example 1: no third factor
        P->srcP[2].assign(1, 1.0);
        P->srcS[2].assign(1, 0.0);
    }

    auto fail = [&](int code) {
        destroy_problem(P);
        return code;
    };

    // dense operators
    for (int a = 0; a < 3; ++a) {
        const int n = P->n[a];
        const double kp = params->kp[a], km = params->km[a];
        std::vector<double> B((size_t)n * n, 0.0), Sm((size_t)n * n);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double v = 0.0;
                const int m1 = i - j + 1;  // T[i][j] = q_{i-j+1}
                if (m1 >= 0 && m1 <= n) v += kp * P->q[a][m1];
                const int m2 = j - i + 1;  // T^T[i][j] = q_{j-i+1}
                if (m2 >= 0 && m2 <= n) v += km * P->q[a][m2];
                B[(size_t)i * n + j] = P->eta[a] * v;
                Sm[(size_t)i * n + j] = std::sqrt(2.0 / (n + 1)) * sin_pi_frac((long long)(i + 1) * (j + 1), n);
            }
        if ((st = dalloc(&P->G[a], B.size())) || (st = upload(P->G[a], B, s))) return fail(st);
        if ((st = dalloc(&P->S[a], Sm.size())) || (st = upload(P->S[a], Sm, s))) return fail(st);
        if (a == 0) {
            std::vector<double> GA(B), GR(B);
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    double m = (i == j) ? 0.75 : ((i - j == 1 || j - i == 1) ? 0.125 : 0.0);
                    GA[(size_t)i * n + j] = m + B[(size_t)i * n + j];
                    GR[(size_t)i * n + j] = m - B[(size_t)i * n + j];
                }
            if ((st = dalloc(&P->Ghat[0], GA.size())) || (st = upload(P->Ghat[0], GA, s))) return fail(st);
            if ((st = dalloc(&P->Ghat[1], GR.size())) || (st = upload(P->Ghat[1], GR, s))) return fail(st);
        }
    }
    {
        std::vector<double> lam;
        for (int a = 0; a < 3; ++a) lam.insert(lam.end(), P->lam_mass[a].begin(), P->lam_mass[a].end());
        for (int a = 0; a < 3; ++a) lam.insert(lam.end(), P->lam_tau[a].begin(), P->lam_tau[a].end());
        if ((st = dalloc(&P->lam, lam.size())) || (st = upload(P->lam, lam, s))) return fail(st);
    }
    if (P->have_src) {
        std::vector<double> o;
        for (int a = 0; a < 3; ++a) o.insert(o.end(), P->srcP[a].begin(), P->srcP[a].end());
        for (int a = 0; a < 3; ++a) o.insert(o.end(), P->srcS[a].begin(), P->srcS[a].end());
        if ((st = dalloc(&P->src1d, o.size())) || (st = upload(P->src1d, o, s))) return fail(st);
    }
    // FP64 workspace
    for (int k = 0; k < tfde_problem::NW; ++k)
        if ((st = dalloc(&P->w[k], P->N))) return fail(st);
    // the FP64 GMRES basis of the default restart (20) for non-symmetric FP64
    // problems (a longer restart grows it; the mixed paths keep their own)
    if (precision == TFDE_FP64 && !P->symmetric && (st = ensure_gmres_basis(P, 20))) return fail(st);
    P->nblk = reduction_blocks(P->N);
    if ((st = dalloc(&P->red, (size_t)128 * P->nblk)) || (st = dalloc(&P->red_out, 256))) return fail(st);
    if (cudaMallocHost((void**)&P->red_host, 256 * sizeof(double)) != cudaSuccess)
        return fail(set_error(TFDE_ENOMEM, "cudaMallocHost failed"));
    if ((st = fft::init(P, s))) return fail(st);
    if (P->dim2 && !P->fft) return fail(set_error(TFDE_EUNSUPPORTED, "2-D problems need n_a <= 2048"));
    if (precision == TFDE_MIXED) {
        // the tensor-core contraction where the grid suits it, else FP32 FFT
        // inner solves under the same FP64 refinement
        if ((st = fmix_wanted(P) ? fmix_init(P, s) : mixed_init(P, s))) return fail(st);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(set_error(TFDE_ECUDA, "assemble: stream sync failed"));
    *out = P;
    return TFDE_OK;
}

int host_coefficients(const tfde_params* params, int axis, double* q, double* lam_tau, double* lam_mass,
                      double* eta) {
    int st = validate_params(params);
    if (st) return st;
    if (axis < 0 || axis > 2) return set_error(TFDE_EINVAL, "axis must be 0, 1 or 2");
    const int n = params->n[axis];
    const double d = params->delta[axis];
    const std::vector<double> qq = generator_q(d, n);
    if (q)
        for (int k = 0; k <= n; ++k) q[k] = qq[k];
    if (lam_tau) {
        const std::vector<double> l = tau_eigs(qq, n);
        for (int k = 0; k < n; ++k) lam_tau[k] = l[k];
    }
    if (lam_mass)
        for (int k = 1; k <= n; ++k) lam_mass[k - 1] = (6.0 + 2.0 * cos_pi_frac(k, n)) / 8.0;
    if (eta) {
        const double h = (params->hi[axis] - params->lo[axis]) / (n + 1);
        *eta = params->dt / (2.0 * std::tgamma(d + 1.0) * std::pow(h, 2.0 - d));
    }
    return TFDE_OK;
}

int destroy_problem(tfde_problem* P) {
    if (!P) return TFDE_OK;
    cudaDeviceSynchronize();
    mixed_free(P);
    fmix_free(P);
    fft::free_state(P);
    for (auto& g : P->Ghat) cudaFree(g);
    for (int a = 0; a < 3; ++a) {
        cudaFree(P->G[a]);
        cudaFree(P->S[a]);
    }
    cudaFree(P->lam);
    cudaFree(P->src1d);
    if (P->io.stream) cudaStreamDestroy(P->io.stream);
    for (cudaEvent_t e : {P->io.ev_start, P->io.ev_in, P->io.ev_ready, P->io.ev_out})
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : P->io.ev_chunk)
        if (e) cudaEventDestroy(e);
    for (auto& v : P->w) cudaFree(v);
    cudaFree(P->V);
    for (auto& hk : P->H)
        for (auto& v : hk) cudaFree(v);
    cudaFree(P->red);
    cudaFree(P->red_out);
    if (P->red_host) cudaFreeHost(P->red_host);
    delete P;
    return TFDE_OK;
}

}  // namespace tfde
