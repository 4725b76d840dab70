// Internal declarations shared by the translation units of libtfde.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tfde.h"

namespace tfde {

// View of a 3-D grid function (x fastest) as a set of 1-D lines along one
// axis: element c of line l sits at  line_offset(l) + c * stride.
//   line_offset(l) = (l % l_in) * s_in + (l / l_in) * s_out
struct AxisView {
    int n;             // length along the axis (= rows and columns of the axis operator)
    long long stride;  // element stride along the axis
    long long lines;   // number of lines (product of the other two extents)
    long long l_in;    // lines per contiguous run
    long long s_in;    // offset step between consecutive lines inside a run
    long long s_out;   // offset step between runs
};

inline AxisView axis_view(const int n[3], int axis) {
    AxisView v{};
    const long long n1 = n[0], n2 = n[1], n3 = n[2];
    if (axis == 0) {
        v.n = n[0]; v.stride = 1; v.lines = n2 * n3; v.l_in = n2 * n3; v.s_in = n1; v.s_out = 0;
    } else if (axis == 1) {
        v.n = n[1]; v.stride = n1; v.lines = n1 * n3; v.l_in = n1; v.s_in = 1; v.s_out = n1 * n2;
    } else {
        v.n = n[2]; v.stride = n1 * n2; v.lines = n1 * n2; v.l_in = n1 * n2; v.s_in = 1; v.s_out = 0;
    }
    return v;
}

// Thread-local error text; set_error returns the status for convenience.
int set_error(int status, const std::string& msg);
// A non-blocking stream of the calling thread on the current device, used to
// capture the device-side loops into CUDA graphs: the caller's stream may be
// the legacy default stream, on which no capture is possible.  The graphs are
// launched on the caller's stream.
cudaStream_t capture_stream();

// ---------------------------------------------------------------- FP64 kernels
// Y = alpha * (Mat along axis) X + beta * (tridiag(1,6,1)/8 along axis) Z  (Z may be null)
void launch_axis_gemm_f64(const double* Mat, const double* X, double* Y, const AxisView& v,
                          double alpha, const double* Z, double beta, cudaStream_t s);
// Y = beta * (tridiag(1,6,1)/8 along axis) X + gamma * W   (W may be null)
void launch_axis_stencil_f64(const double* X, double* Y, const AxisView& v, double beta,
                             const double* W, double gamma, cudaStream_t s);
// Y = A_N X = (T_{n3} (x) T_{n2} (x) T_{n1}) X, T = tridiag(1,6,1)/8: the three
// sweeps of launch_axis_stencil_f64 (x, then y, then z) fused, same result
void launch_mass3d_f64(const double* X, double* Y, const int n[3], cudaStream_t s);
// y[i] = x[i] / Lambda(i,j,k), Lambda from the 1-D arrays (Eq. (diag_tau_pre))
// lam layout: [mass_x | mass_y | mass_z | tau_x | tau_y | tau_z], lengths n1,n2,n3,n1,n2,n3
void launch_lambda_scale_f64(const double* x, double* y, const double* lam, const int n[3],
                             const double c[3], int invert, cudaStream_t s);
// y = a x + b y
void launch_axpby_f64(size_t N, double a, const double* x, double b, double* y, cudaStream_t s);
// z = a x + b y
void launch_axpbypz_f64(size_t N, double a, const double* x, double b, const double* y, double* z,
                        cudaStream_t s);
// x += alpha p ; r -= alpha q ; partial sums of r.r into part[0..nblk)
void launch_cg_update_f64(size_t N, double alpha, const double* p, const double* q, double* x,
                          double* r, double* part, int nblk, cudaStream_t s);
// m dot products <V_j, w>, j < m, V_j = V + j*ldv; partials part[j*nblk + b]
void launch_multidot_f64(size_t N, int m, const double* V, size_t ldv, const double* w,
                         double* part, int nblk, cudaStream_t s);
// w -= sum_j h[j] V_j   (h on device)
void launch_multiaxpy_f64(size_t N, int m, const double* V, size_t ldv, const double* h, double* w,
                          cudaStream_t s);
// deterministic second stage: out[j] = sum_b part[j*nblk + b], j < m
void launch_reduce_finish(const double* part, int nblk, int m, double* out, cudaStream_t s);
int reduction_blocks(size_t N);
// b = AN - Ku + dt F, r = dt F - 2 Ku  (first CN step of a chain); with
// norms2 set, also ||b||^2 and ||r||^2 into norms2[0..1] (device; part =
// scratch of at least 2 * 2432 doubles)
void launch_cn_first(size_t N, const double* AN, const double* Ku, const double* F, double dt, double* b, double* r,
                     double* part, double* norms2, cudaStream_t s);
// t = 2 AN + dt F; b <- t + r - b; r <- b_new + r - b_old  (chained CN step; norms as above)
void launch_cn_chain(size_t N, const double* AN, const double* F, double dt, double* b, double* r, double* part,
                     double* norms2, cudaStream_t s);
// chained CN step with extrapolated initial guess written into u (see
// tfde_kernels64.cu); order 3: x0 = g[0] u + g[1] U1 + g[2] U2 with g in DEVICE
// memory (order 2 when g is null)
void launch_cn_chain_extrap(size_t N, const double* AN, const double* F, double dt, double* b, double* r, double* u,
                            const double* U1, const double* AU1, double* U2, double* AU2, int order, const double* g,
                            double* part, double* norms2, cudaStream_t s);
// the same in `nchunks` consecutive element ranges, range k after event ready[k]
// (the ranges of a host copy of u arriving in pieces); the same norms
void launch_cn_chain_extrap_chunks(size_t N, int nchunks, const cudaEvent_t* ready, const double* AN, const double* F,
                                   double dt, double* b, double* r, double* u, const double* U1, const double* AU1,
                                   double* U2, double* AU2, int order, const double* g, double* part, double* norms2,
                                   cudaStream_t s);
// the five sums of the minimal-residual correction of the order-2 guess into
// out5 (device): <e1,e1>, <e1,e2>, <e2,e2>, <e1,r_e>, <e2,r_e> (see tfde_kernels64.cu)
void launch_cn_mr_dots(size_t N, const double* AN, const double* F, double dt, const double* b, const double* r,
                       const double* AU1, const double* AU2, double* part, double* out5, cudaStream_t s);
// H0 = u, AH0 = AN + Ku: the guess history's first level at a chain's restart
void launch_history_first(size_t N, const double* u, const double* AN, const double* Ku, double* H0, double* AH0,
                          cudaStream_t s);
// g3[0..2] = coefficients of the corrected guess from the five sums m5 (device, one thread)
void launch_cn_mr_coefficients(const double* m5, double* g3, cudaStream_t s);
// F = cP PPP + cS (SPP + PSP + PPS) from 1-D arrays [Px|Py|Pz|Sx|Sy|Sz]
void launch_source_assemble_f64(const double* oned, const int n[3], double cP, double cS, double* F,
                                cudaStream_t s);

}  // namespace tfde

// --------------------------------------------------------------------- problem
struct tfde_problem {
    tfde_params p{};
    int prec = TFDE_FP64;
    int n[3]{};
    size_t N = 0;
    double h[3]{}, eta[3]{}, csum[3]{};
    bool symmetric = false;
    bool dim2 = false;      // params n[2] = 0: the 2-D problem (third axis of extent 1, identity, no stiffness)
    std::vector<double> q[3], lam_tau[3], lam_mass[3];
    std::vector<double> srcP[3], srcS[3];  // 1-D exact cell averages of P and S_delta (if lo=0, hi=1)
    bool have_src = false;

    // device operators (row-major n_a x n_a, [out][in])
    double* Ghat[2] = {nullptr, nullptr};  // x-axis: M1 + eta1 B1 (op A), M1 - eta1 B1 (op RHS)
    double* G[3] = {nullptr, nullptr, nullptr};  // eta_a B_a
    double* S[3] = {nullptr, nullptr, nullptr};  // DST-I matrices
    double* lam = nullptr;                      // [mass x|y|z | tau x|y|z]
    double* src1d = nullptr;                    // [Px|Py|Pz|Sx|Sy|Sz]

    // FP64 workspace: n-vectors
    enum { W_A, W_W, W_C, W_E, W_R, W_Z, W_P, W_Q, W_B, W_T, NW };
    double* w[NW] = {};
    double* V = nullptr;   // GMRES basis, (gmres_cap + 1) vectors
    int gmres_cap = 0;
    double* red = nullptr; // reduction partials (64 * nblk)
    double* red_out = nullptr;  // device results (64)
    double* red_host = nullptr; // pinned host mirror (64)
    int nblk = 0;

    void* mixed = nullptr;  // mixed-precision state (tensor-core path)
    void* fft = nullptr;    // FFT tables of the FFT-embedded passes (tfde_fft.h), null: dense FP64
    void* fmix = nullptr;   // mixed-precision state on the FFT passes (tfde_fftmixed.cu)

    // host copies of a tfde_cn_advance_host step (out == null otherwise): the
    // input goes host -> dev on `stream` while the step starts its work that
    // does not read u; the output goes dev -> host as soon as an iterate that
    // may be final exists (during the residual that decides it), again after
    // any later write of dev
    struct HostIO {
        const double* in = nullptr;
        double* out = nullptr;
        double* dev = nullptr;
        cudaStream_t stream = nullptr;       // copy stream (per problem, created on first use)
        cudaEvent_t ev_start = nullptr, ev_in = nullptr, ev_ready = nullptr, ev_out = nullptr;
        static constexpr int kChunks = 8;    // pieces of the input copy (large grids)
        cudaEvent_t ev_chunk[kChunks] = {};  // piece k has arrived
        int nchunks = 1;
        bool in_pending = false;             // the main stream has not yet waited for the input
        bool out_pending = false;            // an output copy may still read dev
        bool out_valid = false;              // the last output copy was issued after the last write of dev
    } io;

    // chained CN advance: W_B / W_R hold b^{m-1} and its final true residual
    const double* chain_u = nullptr;
    bool chain_ok = false;
    // initial guess of the chained advance: polynomial extrapolation of this
    // order (0: previous step; 3: order 2 with its minimal-residual
    // correction over the history), and the history (u, A u) of the two
    // steps before
    int guess_order = 0;
    // ||b||^2, ||r_0||^2 of the last cn_prepare in red_out[NORMS_SLOT..+1] (device)
    bool norms_ready = false;
    // W_T holds A_N of the mixed solver's final iterate (set by its last
    // full-width residual, cleared by anything else that writes W_T)
    bool an_ready = false;
    int hist = 0;                 // valid history entries (0..2)
    double* H[2][2] = {};         // H[k] = {u^{m-2-k}, A u^{m-2-k}}
};

namespace tfde {
// red_out slot of the fused ||b||^2, ||r_0||^2 of cn_prepare
constexpr int kNormsSlot = 250;
// host copies of tfde_cn_advance_host (tfde_solvers.cu): the main stream s
// waits for the input before the first read of u; an iterate x that may be
// final is offered to the output copy; a write of x first waits for a copy
// still reading it.  No-ops unless x is the step's device state.
void io_wait_input(tfde_problem* P, cudaStream_t s);
void io_offer_output(tfde_problem* P, const double* x, cudaStream_t s);
void io_before_write(tfde_problem* P, const double* x, cudaStream_t s);
// red_out slots of the five sums of the minimal-residual guess correction
constexpr int kMrSlot = 240;
// solver internals (tfde_solvers.cu)
int apply_A64(const tfde_problem* P, int op, const double* x, double* y, cudaStream_t s);
int apply_Pinv64(const tfde_problem* P, const double* r, double* z, cudaStream_t s);
int dots64(const tfde_problem* P, int m, const double* V, size_t ldv, const double* w, double* out,
           cudaStream_t s);
int ensure_gmres_basis(tfde_problem* P, int restart);
int ensure_history(tfde_problem* P);
// TFDE_MIXED on the FFT passes (tfde_fftmixed.cu): grids the tensor-core
// contraction does not take (an n_a not a multiple of 8 or above 448, 2-D)
bool fmix_wanted(const tfde_problem* P);
int fmix_init(tfde_problem* P, cudaStream_t s);
void fmix_free(tfde_problem* P);
int fmix_apply_A(const tfde_problem* P, int op, const double* x, double* y, cudaStream_t s);
int fmix_apply_Pinv(const tfde_problem* P, const double* r, double* z, cudaStream_t s);
int fmix_pcg(tfde_problem* P, const double* b, double* x, double tol, int maxit, tfde_info* info, cudaStream_t s,
             bool r_given);
int fmix_pgmres(tfde_problem* P, const double* b, double* x, int restart, double tol, int maxit, tfde_info* info,
                cudaStream_t s, bool r_given);
}  // namespace tfde
