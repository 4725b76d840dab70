// Spectra of the preconditioned systems at sizes far beyond a dense
// eigensolve (Sec. 3): Lanczos estimates of the extreme eigenvalues of the
// symmetric part P^{-1/2} H(A) P^{-1/2} (Theorem CG_bounded_sprctrum and
// Lemma prop:eigen_S place them in (1/2, 3/2)) and of the spectral radius of
// the skew part P^{-1/2} S(A) P^{-1/2} (Lemma eigen_Skew bounds it by
// varsigma), with the GMRES rate omega of Theorem theorem_main.
//
// H(A) = (A + A^T) / 2 is the operator of Eq. (linear_sys) with
// k_+ = k_- = (k_+ + k_-) / 2 on every axis (B = k_+ T + k_- T^T is linear in
// the two coefficients), and S(A) = A - H(A).  The tau preconditioner depends
// on the coefficients only through k_+ + k_- (Eq. (pre_definition)), so A and
// H(A) share it; P^{-1/2} = S_N Lambda^{-1/2} S_N comes from the same
// diagonalisation.  Every operator application runs on the FP64 FFT passes;
// the Lanczos recurrences use the library's FP64 vector kernels, and the
// extreme eigenvalues of the small tridiagonal matrices are found on the host
// by bisection on Sturm counts.
#include <cmath>
#include <string>
#include <vector>

#include "tfde_fft.h"
#include "tfde_internal.h"

namespace tfde {

int assemble_problem(const tfde_params*, int, cudaStream_t, tfde_problem**);
int destroy_problem(tfde_problem*);

namespace {

// eigenvalues of the symmetric tridiagonal (a, b) below x
int sturm_count(const std::vector<double>& a, const std::vector<double>& b, double x) {
    int c = 0;
    double q = 1.0;
    for (size_t i = 0; i < a.size(); ++i) {
        const double bb = i ? b[i - 1] * b[i - 1] : 0.0;
        q = (a[i] - x) - (i ? bb / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++c;
    }
    return c;
}

// the i-th smallest eigenvalue (0-based) of the tridiagonal by bisection
double tridiag_eig(const std::vector<double>& a, const std::vector<double>& b, int i) {
    double lo = a[0], hi = a[0];
    for (size_t k = 0; k < a.size(); ++k) {   // Gershgorin interval
        const double r = (k ? std::fabs(b[k - 1]) : 0.0) + (k + 1 < a.size() ? std::fabs(b[k]) : 0.0);
        lo = std::fmin(lo, a[k] - r);
        hi = std::fmax(hi, a[k] + r);
    }
    for (int it = 0; it < 200 && hi - lo > 1e-15 * std::fmax(1.0, std::fabs(hi)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(a, b, mid) > i) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

struct Vecs {
    double* v = nullptr;
    double* vp = nullptr;
    double* w = nullptr;
    double* t = nullptr;
    double* u = nullptr;
    ~Vecs() {
        cudaFree(v);
        cudaFree(vp);
        cudaFree(w);
        cudaFree(t);
        cudaFree(u);
    }
};

// Lanczos tridiagonal of the symmetric operator op, `steps` steps from v0
// (no re-orthogonalisation: only the extreme Ritz values are used)
template <typename Op>
int lanczos(tfde_problem* P, Op op, const double* v0, int steps, Vecs& V, std::vector<double>& al,
            std::vector<double>& be, cudaStream_t s) {
    const size_t N = P->N;
    double nv;
    int st = dots64(P, 1, v0, 0, v0, &nv, s);
    if (st) return st;
    nv = std::sqrt(nv);
    if (!(nv > 0.0) || !std::isfinite(nv)) return set_error(TFDE_EINVAL, "the start vector is zero or not finite");
    launch_axpbypz_f64(N, 1.0 / nv, v0, 0.0, v0, V.v, s);
    cudaMemsetAsync(V.vp, 0, N * sizeof(double), s);
    double bprev = 0.0;
    al.clear();
    be.clear();
    for (int j = 0; j < steps; ++j) {
        if ((st = op(V.v, V.w))) return st;
        double a;
        if ((st = dots64(P, 1, V.w, 0, V.v, &a, s))) return st;
        // w = w - a v - bprev vp
        launch_axpby_f64(N, -a, V.v, 1.0, V.w, s);
        launch_axpby_f64(N, -bprev, V.vp, 1.0, V.w, s);
        double bb;
        if ((st = dots64(P, 1, V.w, 0, V.w, &bb, s))) return st;
        if (!std::isfinite(a) || !std::isfinite(bb)) return set_error(TFDE_ENAN, "non-finite Lanczos coefficient");
        al.push_back(a);
        const double b = std::sqrt(bb);
        if (j + 1 == steps || b <= 1e-14 * std::fabs(a)) break;
        be.push_back(b);
        std::swap(V.vp, V.v);                            // vp <- v
        launch_axpbypz_f64(N, 1.0 / b, V.w, 0.0, V.w, V.v, s);   // v <- w / b
        bprev = b;
    }
    be.resize(al.size() > 0 ? al.size() - 1 : 0);
    return TFDE_OK;
}

}  // namespace

int spectrum(const tfde_params* params, int steps, const double* v0, tfde_spectrum_info* out, cudaStream_t s) {
    tfde_problem* PA = nullptr;
    tfde_problem* PH = nullptr;
    tfde_params ph = *params;
    for (int a = 0; a < 3; ++a) ph.kp[a] = ph.km[a] = 0.5 * (params->kp[a] + params->km[a]);
    int st = assemble_problem(params, TFDE_FP64, s, &PA);
    if (!st) st = assemble_problem(&ph, TFDE_FP64, s, &PH);
    if (!st && (!PA->fft || !PH->fft)) st = set_error(TFDE_EUNSUPPORTED, "tfde_spectrum needs every n_a <= 2048");
    Vecs V;
    const size_t N = st ? 0 : PA->N;
    if (!st) {
        for (double** p : {&V.v, &V.vp, &V.w, &V.t, &V.u})
            if (cudaMalloc((void**)p, N * sizeof(double)) != cudaSuccess) {
                st = set_error(TFDE_ENOMEM, "cudaMalloc of the Lanczos vectors failed");
                break;
            }
    }
    tfde_spectrum_info res{};
    std::vector<double> al, be;
    if (!st) {
        // M_H x = P^{-1/2} H(A) P^{-1/2} x
        double* sc1 = PH->w[tfde_problem::W_R];
        double* sc2 = PH->w[tfde_problem::W_Z];
        auto mh = [&](const double* x, double* y) -> int {
            int e = fft::apply_Pinv_half(PH, x, V.t, sc1, sc2, s);
            if (!e) e = apply_A64(PH, TFDE_OP_A, V.t, V.u, s);
            if (!e) e = fft::apply_Pinv_half(PH, V.u, y, sc1, sc2, s);
            return e;
        };
        st = lanczos(PH, mh, v0, steps, V, al, be, s);
        if (!st) {
            res.steps = (int)al.size();
            res.sym_min = tridiag_eig(al, be, 0);
            res.sym_max = tridiag_eig(al, be, (int)al.size() - 1);
        }
    }
    bool skew = false;
    for (int a = 0; a < 3; ++a)
        if (params->kp[a] != params->km[a]) skew = true;
    if (!st && skew) {
        // -M_S^2 (symmetric positive semidefinite), M_S x = P^{-1/2} (A - H(A)) P^{-1/2} x
        double* sc1 = PH->w[tfde_problem::W_R];
        double* sc2 = PH->w[tfde_problem::W_Z];
        double* m1 = PA->w[tfde_problem::W_R];
        auto ms = [&](const double* x, double* y) -> int {
            int e = fft::apply_Pinv_half(PH, x, V.t, sc1, sc2, s);
            if (!e) e = apply_A64(PA, TFDE_OP_A, V.t, V.u, s);
            if (!e) e = apply_A64(PH, TFDE_OP_A, V.t, PA->w[tfde_problem::W_Z], s);
            if (!e) launch_axpby_f64(N, -1.0, PA->w[tfde_problem::W_Z], 1.0, V.u, s);
            if (!e) e = fft::apply_Pinv_half(PH, V.u, y, sc1, sc2, s);
            return e;
        };
        auto msq = [&](const double* x, double* y) -> int {
            int e = ms(x, m1);
            if (!e) e = ms(m1, y);
            if (!e) launch_axpby_f64(N, 0.0, y, -1.0, y, s);   // y = -y
            return e;
        };
        std::vector<double> as, bs;
        st = lanczos(PA, msq, v0, steps, V, as, bs, s);
        if (!st) res.skew_rho = std::sqrt(std::fmax(0.0, tridiag_eig(as, bs, (int)as.size() - 1)));
    }
    if (!st) {
        double vs = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double kp = params->kp[a], km = params->km[a];
            vs = std::fmax(vs, 1.5 * std::tan(0.5 * M_PI * params->delta[a]) * std::fabs(kp - km) / (kp + km));
        }
        res.varsigma = vs;
        res.omega = std::sqrt((2.0 + 4.0 * vs * vs) / (3.0 + 4.0 * vs * vs));
        const double c = res.sym_min, C = res.sym_max, r = res.skew_rho;
        res.omega_est = std::sqrt(std::fmax(0.0, 1.0 - c * c / (c * C + r * r)));
        if (cudaStreamSynchronize(s) != cudaSuccess) st = set_error(TFDE_ECUDA, "tfde_spectrum: stream error");
    }
    destroy_problem(PA);
    destroy_problem(PH);
    if (!st && out) *out = res;
    return st;
}

}  // namespace tfde
