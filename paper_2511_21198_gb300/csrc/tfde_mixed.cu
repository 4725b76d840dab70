// Mixed-precision path: split-BF16 tcgen05 contractions for the inner
// Krylov solves on FP32 vectors, wrapped in FP64 iterative refinement whose
// residual b - A x is always evaluated accurately (Sec. 2 Eq. (linear_sys),
// Sec. 3 Eq. (diag_tau_pre)).
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "tfde_givens.h"
#include "tfde_mixed.h"
#include "tfde_stats.h"

namespace tfde {

int pcg64(const tfde_problem*, const double*, double*, double, int, tfde_info*, cudaStream_t, bool);
int pgmres64(tfde_problem*, const double*, double*, int, double, int, tfde_info*, cudaStream_t, bool);

namespace {

#define MX_TRY(expr)                                                                       \
    do {                                                                                   \
        cudaError_t e__ = (expr);                                                          \
        if (e__ != cudaSuccess)                                                            \
            return set_error(TFDE_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e__)); \
    } while (0)

using clk = std::chrono::steady_clock;

void to_bf16_pair(double v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn((float)v);
    lo = __float2bfloat16_rn((float)(v - (double)__bfloat162float(hi)));
}

// Dense eta_a B_a (row-major [out][in]) from the generator (Eq. (T_ni), Eq. (stiff_matrix)).
std::vector<double> dense_etaB(const tfde_problem* P, int a) {
    const int n = P->n[a];
    const double kp = P->p.kp[a], km = P->p.km[a];
    std::vector<double> B((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double v = 0.0;
            const int m1 = i - j + 1, m2 = j - i + 1;
            if (m1 >= 0 && m1 <= n) v += kp * P->q[a][m1];
            if (m2 >= 0 && m2 <= n) v += km * P->q[a][m2];
            B[(size_t)i * n + j] = P->eta[a] * v;
        }
    return B;
}

double mass_entry(int i, int j) { return i == j ? 0.75 : ((i - j == 1 || j - i == 1) ? 0.125 : 0.0); }

// S_n of Eq. (diag_tau_pre), S(i, j) = sqrt(2 / (n + 1)) sin(pi (i + 1)(j + 1) / (n + 1))
// (row-major, FP64), the product reduced modulo 2(n + 1) before the sine.
std::vector<double> dst_dense(int n) {
    std::vector<double> S((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            const long long r = ((long long)(i + 1) * (j + 1)) % (2LL * (n + 1));
            S[(size_t)i * n + j] = std::sqrt(2.0 / (n + 1)) * std::sin(M_PI * (double)r / (double)(n + 1));
        }
    return S;
}

struct SegSpec {
    int a_hi, a_lo, plane;  // a_lo < 0: single-term A
};

// Descriptor of one split-BF16 pass: out = alpha * sum_seg (A_seg along axis)
// (plane_seg hi + lo); *bytes / *flops receive its algorithmic traffic and
// tensor-core work.
void gemm_params(const tfde_problem* P, int axis, const SegSpec* segs, int nseg, int out_mode, float alpha,
                 float* out_f32, int out_plane, bool lam_scale, tc::Params& prm, double* bytes, double* flops) {
    MixedState* M = mixed(P);
    std::memset(&prm, 0, sizeof(prm));
    tc::set_geometry(prm, P->n, axis);
    // tensor maps: merged boxes where the allocation allows one copy per operand
    // (hi/lo operator pair; hi/lo plane pair with, on y/z, all line blocks)
    int na = 0, nb = 0;
    for (int g = 0; g < nseg; ++g) {
        tc::Segment& S = prm.seg[g];
        S.nkb = (P->n[axis] + tc::SK - 1) / tc::SK;
        S.amap2 = -1;
        S.bmap2 = -1;
        if (segs[g].a_lo >= 0 && M->has_amap2[segs[g].a_hi]) {
            prm.amaps[na] = M->amap2[segs[g].a_hi];
            S.amap2 = na++;
            S.na = 2;
        } else {
            prm.amaps[na] = M->amap[segs[g].a_hi];
            S.amap[0] = na++;
            S.na = 1;
            if (segs[g].a_lo >= 0) {
                prm.amaps[na] = M->amap[segs[g].a_lo];
                S.amap[1] = na++;
                S.na = 2;
            }
        }
        const int rank = M->bmap2_rank[segs[g].plane][axis];
        if (rank > 0) {
            prm.bmaps[nb] = M->bmap2[segs[g].plane][axis];
            S.bmap2 = nb++;
            prm.b_rank = rank;
        } else {
            prm.bmaps[nb] = M->bmap_hi[segs[g].plane][axis];
            S.bmap[0] = nb++;
            prm.bmaps[nb] = M->bmap_lo[segs[g].plane][axis];
            S.bmap[1] = nb++;
        }
        S.nb = 2;
        S.npair = 0;
        S.pa[S.npair] = 0; S.pb[S.npair++] = 0;   // A_hi * x_hi
        S.pa[S.npair] = 0; S.pb[S.npair++] = 1;   // A_hi * x_lo
        if (S.na == 2) { S.pa[S.npair] = 1; S.pb[S.npair++] = 0; }  // A_lo * x_hi
    }
    prm.nseg = nseg;
    prm.out_mode = out_mode;
    prm.alpha = alpha;
    prm.out_f32 = out_f32;
    if (out_f32) tc::make_out_map(&prm.omap_f32, out_f32, P->n, axis, true);
    if (out_mode == tc::OUT_HILO || out_mode == tc::OUT_XPAY || out_mode == tc::OUT_HI) {
        prm.out_hi = M->hi[out_plane];
        prm.out_lo = M->lo[out_plane];
        prm.omap_hi = M->omap_hi[out_plane][axis];
        prm.omap_hl = M->omap_hl[out_plane][axis];
    }
    if (lam_scale) {
        const long long n1n2 = (long long)P->n[0] * P->n[1];
        prm.lam_ra = M->lam;
        prm.lam_rb = M->lam + P->n[2];
        prm.lam_U = M->lam + 2 * P->n[2];
        prm.lam_V = M->lam + 2 * P->n[2] + n1n2;
    }
    prm.err = M->err;
    // algorithmic traffic: each operand plane pair read once, the output written
    // once (4 bytes per element either way), the operator matrices read once
    const double N = (double)P->N, nax = (double)P->n[axis];
    double by = 4.0 * N, fl = 0.0;
    for (int g = 0; g < nseg; ++g) {
        by += 4.0 * N + 2.0 * nax * nax * prm.seg[g].na;
        fl += 2.0 * prm.seg[g].npair * nax * N;
    }
    *bytes = by;
    *flops = fl;
}

int run_gemm(const tfde_problem* P, int axis, const SegSpec* segs, int nseg, int out_mode, float alpha,
             float* out_f32, int out_plane, bool lam_scale, cudaStream_t s, const float* dot_vec = nullptr,
             double* dot_out = nullptr, const int* skip = nullptr) {
    tc::Params prm;
    double bytes, flops;
    gemm_params(P, axis, segs, nseg, out_mode, alpha, out_f32, out_plane, lam_scale, prm, &bytes, &flops);
    prm.skip = skip;
    if (out_mode == tc::OUT_F32 && dot_out) {
        prm.dot_vec = dot_vec;
        prm.dot_out = dot_out;
    }
    mixed(P)->gemm_launches++;
    return tc::launch(prm, s, bytes, flops);
}

// Pass list of the fast operator and the preconditioner.  Each entry is one
// call of run_gemm; the same list serves the single-problem solvers (launched
// one by one) and the batched solver (descriptors gathered across problems).
struct Pass {
    int axis;
    SegSpec seg[2];
    int nseg;
    int out_mode;
    int out_plane;   // OUT_HILO target plane; OUT_F32 writes the caller's vector
    bool lam;
};

// A (op A) or the RHS operator applied to plane PL_P: 5 passes; the last one
// writes out_plane (split) when out_plane >= 0, else FP32.
int matvec_passes(int op, int out_plane, Pass* ps) {
    const bool rhs = (op & 1) != 0;
    const int gh = rhs ? OM_GHATR_H : OM_GHAT_H, gl = rhs ? OM_GHATR_L : OM_GHAT_L;
    const int yh = rhs ? OM_GYN_H : OM_GY_H, yl = rhs ? OM_GYN_L : OM_GY_L;
    const int zh = rhs ? OM_GZN_H : OM_GZ_H, zl = rhs ? OM_GZN_L : OM_GZ_L;
    ps[0] = {0, {{gh, gl, PL_P}}, 1, tc::OUT_HILO, PL_A, false};
    ps[1] = {0, {{OM_MX, -1, PL_P}}, 1, tc::OUT_HILO, PL_W, false};
    ps[2] = {1, {{OM_MY, -1, PL_A}, {yh, yl, PL_W}}, 2, tc::OUT_HILO, PL_C, false};
    ps[3] = {1, {{OM_MY, -1, PL_W}}, 1, tc::OUT_HILO, PL_E, false};
    ps[4] = {2, {{OM_MZ, -1, PL_C}, {zh, zl, PL_E}}, 2, out_plane >= 0 ? tc::OUT_HILO : tc::OUT_F32,
             out_plane >= 0 ? out_plane : 0, false};
    return 5;
}

// S_N Lambda^{-1} S_N applied to plane PL_R: 6 passes, the last one FP32.
int precond_passes(Pass* ps) {
    ps[0] = {0, {{OM_SX, -1, PL_R}}, 1, tc::OUT_HILO, PL_T1, false};
    ps[1] = {1, {{OM_SY, -1, PL_T1}}, 1, tc::OUT_HILO, PL_T2, false};
    ps[2] = {2, {{OM_SZ, -1, PL_T2}}, 1, tc::OUT_HILO, PL_T1, true};
    ps[3] = {2, {{OM_SZ, -1, PL_T1}}, 1, tc::OUT_HILO, PL_T2, false};
    ps[4] = {1, {{OM_SY, -1, PL_T2}}, 1, tc::OUT_HILO, PL_T1, false};
    ps[5] = {0, {{OM_SX, -1, PL_T1}}, 1, tc::OUT_F32, 0, false};
    return 6;
}

// The last pass's FP32 output may also be dotted with dot_vec into *dot_out
// (accumulated: the caller zeroes it).
int run_passes(const tfde_problem* P, const Pass* ps, int np, float* out_f32, cudaStream_t s,
               const float* dot_vec = nullptr, double* dot_out = nullptr, const int* skip = nullptr) {
    for (int i = 0; i < np; ++i) {
        const Pass& q = ps[i];
        const bool last = i + 1 == np;
        int st = run_gemm(P, q.axis, q.seg, q.nseg, q.out_mode, 1.f, q.out_mode == tc::OUT_F32 ? out_f32 : nullptr,
                          q.out_plane, q.lam, s, last ? dot_vec : nullptr, last ? dot_out : nullptr, skip);
        if (st) return st;
    }
    return TFDE_OK;
}

// q32 = A p (op A) or the RHS operator, p given as the split plane pair PL_P;
// with out_plane >= 0 the result goes to that split plane pair instead.
// The operator's passes 0, 1 (x axis: Ghat p, M_x p) and 2, 3 (y axis:
// M_y a + G_y w, M_y w) are independent pairs along one axis: each pair runs
// as one grouped persistent launch (the tile list of both), so the second
// contraction starts while the first one's last tiles drain.
int ensure_pairs(const tfde_problem* P, cudaStream_t s) {
    MixedState* M = mixed(P);
    if (M->pair_d) return TFDE_OK;
    Pass ps[5];
    matvec_passes(TFDE_OP_A, -1, ps);
    tc::Params prm[4];
    long long gst[6];
    for (int g = 0; g < 2; ++g) {
        gst[3 * g] = 0;
        M->pair_bytes[g] = M->pair_flops[g] = 0.0;
        for (int i = 0; i < 2; ++i) {
            const Pass& q = ps[2 * g + i];
            double by, fl;
            gemm_params(P, q.axis, q.seg, q.nseg, q.out_mode, 1.f, nullptr, q.out_plane, q.lam, prm[2 * g + i], &by, &fl);
            gst[3 * g + i + 1] = gst[3 * g + i] + prm[2 * g + i].ntiles * prm[2 * g + i].mhalves;
            M->pair_bytes[g] += by;
            M->pair_flops[g] += fl;
        }
        M->pair_total[g] = gst[3 * g + 2];
    }
    MX_TRY(cudaMalloc((void**)&M->pair_d, sizeof(prm)));
    MX_TRY(cudaMalloc((void**)&M->pair_gstart, sizeof(gst)));
    MX_TRY(cudaMemcpyAsync(M->pair_d, prm, sizeof(prm), cudaMemcpyHostToDevice, s));
    MX_TRY(cudaMemcpyAsync(M->pair_gstart, gst, sizeof(gst), cudaMemcpyHostToDevice, s));
    MX_TRY(cudaStreamSynchronize(s));   // the host arrays go out of scope
    return TFDE_OK;
}

int fast_matvec(const tfde_problem* P, int op, float* q32, cudaStream_t s, int out_plane = -1,
                const float* dot_vec = nullptr, double* dot_out = nullptr, const int* skip = nullptr) {
    Pass ps[5];
    const int np = matvec_passes(op, out_plane, ps);
    if (op != TFDE_OP_A) return run_passes(P, ps, np, q32, s, dot_vec, dot_out, skip);
    MixedState* M = mixed(P);
    int st;
    if ((st = ensure_pairs(P, s))) return st;
    for (int g = 0; g < 2; ++g) {
        M->gemm_launches++;
        st = tc::launch_grouped(M->pair_d + 2 * g, M->pair_gstart + 3 * g, 2, M->pair_total[g], g == 0 ? 1 : 0,
                                tc::OUT_HILO, nullptr, M->err, s, M->pair_bytes[g], M->pair_flops[g], skip);
        if (st) return st;
    }
    return run_passes(P, ps + 4, 1, q32, s, dot_vec, dot_out, skip);
}

// z32 = S_N Lambda^{-1} S_N r, r given as the split plane pair PL_R.
// z = S_N Lambda^{-1} S_N r (plane PL_R) fused into the CG direction update:
// *rz += <r, z>, accumulated in the Lambda pass as <t, Lambda^{-1} t> with
// t = S_N r (S_N is orthogonal), and p = z + beta p with beta = *num / *den
// (0 when den is null; p_old the previous direction), written by the last
// pass to p32 and to the split planes PL_P: z itself is never stored.
// The passes carry the hi (BF16) plane alone: the inner PCG stops at
// tolerances of ~1e-4 .. 1e-1, far above the ~2^-9 relative perturbation
// that BF16 intermediates give the preconditioner (measured: the same
// iteration counts as with split intermediates), and each pass then moves
// and converts half the data.  The last pass still writes p in FP32 and in
// split planes, for the operator.
int fast_precond_cg(const tfde_problem* P, float* p32, const float* p_old, double* rz, const double* num,
                    const double* den, cudaStream_t s, const int* skip = nullptr) {
    MixedState* M = mixed(P);
    Pass ps[6];
    const int np = precond_passes(ps);
    for (int i = 0; i < np; ++i) {
        const Pass& q = ps[i];
        const bool last = i + 1 == np;
        tc::Params prm;
        double bytes, flops;
        gemm_params(P, q.axis, q.seg, q.nseg, last ? tc::OUT_XPAY : tc::OUT_HI, 1.f, last ? p32 : nullptr,
                    last ? PL_P : q.out_plane, q.lam, prm, &bytes, &flops);
        // one B plane (hi) and one product per pass
        const int pl = q.seg[0].plane;
        tc::Segment& S = prm.seg[0];
        if (S.bmap2 >= 0) {
            if (M->bmap1_rank[pl][q.axis] > 0) {
                prm.bmaps[S.bmap2] = M->bmap1[pl][q.axis];
                prm.b_rank = M->bmap1_rank[pl][q.axis];
            } else {   // the merged box would carry both planes: per-plane boxes, hi alone
                prm.bmaps[S.bmap2] = M->bmap_hi[pl][q.axis];
                S.bmap[0] = S.bmap2;
                S.bmap2 = -1;
            }
        }
        S.nb = 1;
        S.npair = 1;
        bytes -= 2.0 * (double)P->N * (last ? 1.0 : 2.0);   // lo plane neither read nor (but the last) written
        if (q.lam) {
            prm.dot_lam = 1;
            prm.dot_out = rz;
        }
        if (last) {
            prm.xp_num = num;
            prm.xp_den = den;
            prm.xp_old = p_old;
            bytes += 8.0 * (double)P->N;   // the old p in, the split planes out
        }
        prm.skip = skip;
        mixed(P)->gemm_launches++;
        if (int st = tc::launch(prm, s, bytes, flops)) return st;
    }
    return TFDE_OK;
}

int fast_precond(const tfde_problem* P, float* z32, cudaStream_t s, const float* dot_vec = nullptr,
                 double* dot_out = nullptr, const int* skip = nullptr) {
    Pass ps[6];
    const int np = precond_passes(ps);
    return run_passes(P, ps, np, z32, s, dot_vec, dot_out, skip);
}

int check_err(const tfde_problem* P, cudaStream_t s) {
    MixedState* M = mixed(P);
    MX_TRY(cudaMemcpyAsync(M->err_host, M->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MX_TRY(cudaStreamSynchronize(s));
    if (*M->err_host) return set_error(TFDE_ETIMEOUT, "tensor-core kernel wait ran out (device error flag set)");
    return TFDE_OK;
}

double host_scalar(const tfde_problem* P, const double* dev, cudaStream_t s, int* st) {
    *st = TFDE_OK;
    if (cudaMemcpyAsync(P->red_host, dev, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        *st = set_error(TFDE_ECUDA, "scalar read-back failed");
        return 0.0;
    }
    return P->red_host[0];
}

// Device-scalar slots: <p, A p>, <r, r>, and <r, z> of the current / next
// iteration in alternating slots (a kernel that reads one writes the other).
enum { D_PQ = 0, D_RR = 1, D_RZ0 = 2, D_RZ1 = 3 };
// Device / host Hessenberg scratch offsets (MixedState::gm).
enum { GM_H = 0, GM_H2 = 128, GM_WW = 256, GM_Y = 384, GM_SIZE = 512 };

int build_pcg_graph(const tfde_problem* P, cudaStream_t s);
int inner_pcg_graph(const tfde_problem* P, double theta, int maxit, int* iters, PcgPending* pend, cudaStream_t s,
                    double* reached, double rr0);

// Inner PCG on FP32 vectors: A d = r32 (r32 and its split planes prepared by
// the caller, x32 = 0), until ||r|| <= theta ||r32_0|| or maxit.  The inner
// products ride on the kernels that produce their operands (<p, Ap> in the
// operator's last pass, <r, z> in the preconditioner's Lambda pass, <r, r> in
// the update), the coefficients alpha = <r,z>/<p,Ap> and beta =
// <r,z>_new/<r,z> are formed on the device (alpha by the update kernel, beta
// by the preconditioner's last pass, which writes p = z + beta p directly),
// and the host reads <r, r> once per iteration for the stopping test.
// rr0_known > 0: the caller's ||r32||^2 (the refinement scales r by a power
// of two to a norm in [1/2, 1)), which spares a reduction and a host read.  The solution is not
// updated per iteration: the directions p_j and their alpha_j stay in a ring
// of kPRing vectors, folded into F_X when the ring is full, and *pend
// describes what is left (d = fold ? F_X : 0, + sum alpha_j p_j), combined by
// the caller in the same pass that adds the correction to the FP64 solution:
// 12 of the update's 28 bytes per point and iteration are saved.
int inner_pcg(const tfde_problem* P, double theta, int maxit, int* iters, PcgPending* pend, cudaStream_t s,
              double* reached = nullptr, double rr0_known = 0.0) {
    MixedState* M = mixed(P);
    const size_t N = P->N;
    float* r = M->f[F_R];
    float* q = M->f[F_Q];
    double* d = M->dsc;
    int st = TFDE_OK;
    *pend = PcgPending();
    if (!M->pring) MX_TRY(cudaMalloc((void**)&M->pring, (size_t)kPRing * N * sizeof(float)));
    auto pbuf = [&](int j) { return M->pring + (size_t)(j % kPRing) * N; };
    double rr0 = rr0_known;
    if (!(rr0 > 0.0)) {
        launch_dot32(N, r, r, P->red, P->nblk, s);
        launch_reduce_finish(P->red, P->nblk, 1, d + D_RR, s);
        rr0 = host_scalar(P, d + D_RR, s, &st);
        if (st) return st;
    }
    if (reached) *reached = 0.0;
    if (!(rr0 > 0.0) || !std::isfinite(rr0)) return rr0 == 0.0 ? TFDE_OK : set_error(TFDE_ENAN, "non-finite inner residual");
    // device-side loop unless every launch is to be timed on its own
    if (M->device_loop && !stats_timing() && maxit > 0) {
        if ((st = build_pcg_graph(P, s))) return st;
        if (M->pcg_exec) return inner_pcg_graph(P, theta, maxit, iters, pend, s, reached, rr0);
    }
    int rz = D_RZ0;
    MX_TRY(cudaMemsetAsync(d + rz, 0, sizeof(double), s));
    if ((st = fast_precond_cg(P, pbuf(0), nullptr, d + rz, nullptr, nullptr, s))) return st;   // p_0 = z
    int k = 0, j0 = 0;   // directions j0 .. k not yet folded
    bool folded = false;
    while (k < maxit) {
        MX_TRY(cudaMemsetAsync(d + D_PQ, 0, 2 * sizeof(double), s));   // <p, Ap> and <r, r>
        if ((st = fast_matvec(P, TFDE_OP_A, q, s, -1, pbuf(k), d + D_PQ))) return st;
        // the preconditioner reads the hi plane of r alone
        launch_cg_update_r32(N, d + rz, d + D_PQ, q, r, M->hi[PL_R], nullptr, d + D_RR, d + kAlphaSlot + k % kPRing,
                             s);
        const double rr = host_scalar(P, d + D_RR, s, &st);
        if (st) return st;
        ++k;
        if (!std::isfinite(rr)) return set_error(TFDE_ENAN, "non-finite inner residual");
        if (reached) *reached = std::sqrt(rr / rr0);
        if (rr <= theta * theta * rr0 || k >= maxit) break;
        if (k - j0 == kPRing) {
            // the next direction reuses the oldest slot: fold the window into F_X
            PcgPending w;
            w.cnt = kPRing;
            w.fold = folded;
            for (int j = 0; j < kPRing; ++j) {
                w.p[j] = pbuf(j0 + j);
                w.alpha[j] = d + kAlphaSlot + (j0 + j) % kPRing;
            }
            launch_pcg_combine(N, w, M->f[F_X], 0.0, nullptr, nullptr, M->f[F_X], s);
            folded = true;
            j0 = k;
        }
        const int rzn = rz == D_RZ0 ? D_RZ1 : D_RZ0;
        MX_TRY(cudaMemsetAsync(d + rzn, 0, sizeof(double), s));
        // p_k = z + beta p_{k-1}, beta = <r, z>_new / <r, z>
        if ((st = fast_precond_cg(P, pbuf(k), pbuf(k - 1), d + rzn, d + rzn, d + rz, s))) return st;
        rz = rzn;
    }
    pend->cnt = k - j0;
    pend->fold = folded;
    for (int j = 0; j < pend->cnt; ++j) {
        pend->p[j] = pbuf(j0 + j);
        pend->alpha[j] = d + kAlphaSlot + (j0 + j) % kPRing;
    }
    *iters = k;
    return check_err(P, s);
}

// Slots of the device-side loop: <r, z> of the last preconditioner
// application and the stop threshold theta^2 ||r_0||^2.
enum { D_RZN = 4, D_THR = 5 };

// The inner PCG's iterations as one graph: a while node whose body runs
// kPRing iterations (the ring of search directions makes every pointer of a
// body's kernels fixed), each iteration head -> operator (3 split launches,
// <p, Ap> fused) -> residual update -> stop test (sets the loop condition
// and the device flag that turns the rest of the body into no-ops) ->
// preconditioner and direction update (6 split launches, <r, z> and beta
// fused), the body's full window of directions folded into F_X before the
// last direction update.  Built on the first call; a failure to build it
// leaves the host-driven loop in use.
int build_pcg_graph(const tfde_problem* P, cudaStream_t s) {
    MixedState* M = mixed(P);
    if (M->pcg_exec && M->pcg_tune_gen != tc::tune_generation()) {   // launch parameters changed: recapture
        cudaGraphExecDestroy(M->pcg_exec);
        cudaGraphDestroy(M->pcg_graph);
        M->pcg_exec = nullptr;
        M->pcg_graph = nullptr;
    }
    if (M->pcg_exec || M->pcg_graph_failed) return TFDE_OK;
    const size_t N = P->N;
    if (!M->pring) MX_TRY(cudaMalloc((void**)&M->pring, (size_t)kPRing * N * sizeof(float)));
    if (!M->pcg_ctl) {
        MX_TRY(cudaMalloc((void**)&M->pcg_ctl, 4 * sizeof(int)));
        MX_TRY(cudaMallocHost((void**)&M->pcg_ctl_host, 4 * sizeof(int)));
    }
    if (int st = ensure_pairs(P, s)) return st;
    if (int st = tc::set_attrs()) return st;   // kernel attributes are set outside the capture
    float* q = M->f[F_Q];
    float* r = M->f[F_R];
    double* d = M->dsc;
    int* ctl = M->pcg_ctl;
    auto pbuf = [&](int j) { return M->pring + (size_t)(j % kPRing) * N; };
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
    cudaGraphConditionalHandle h{};
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    if (ok) ok = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
    }
    if (ok) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        // captured on a stream of its own (the caller's may be the legacy default stream)
        const cudaStream_t s = capture_stream();
        ok = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
             cudaSuccess;
        if (ok) {
            stats_set_capturing(true);
            int st = TFDE_OK;
            const float* ps[kPRing];
            const double* as[kPRing];
            for (int u = 0; u < kPRing; ++u) {
                ps[u] = pbuf(u);
                as[u] = d + kAlphaSlot + u;
            }
            for (int u = 0; u < kPRing && !st; ++u) {
                launch_pcg_head(d, D_RZ0, D_RZN, D_PQ, D_RR, ctl, s);
                st = fast_matvec(P, TFDE_OP_A, q, s, -1, pbuf(u), d + D_PQ, ctl + 1);
                if (st) break;
                launch_cg_update_r32(N, d + D_RZ0, d + D_PQ, q, r, M->hi[PL_R], nullptr, d + D_RR, d + kAlphaSlot + u,
                                     s, ctl + 1);
                launch_pcg_cond(h, d + D_RR, d + D_THR, ctl, s);
                if (u == kPRing - 1) launch_pcg_fold_dev(N, ps, as, M->f[F_X], ctl, s);
                st = fast_precond_cg(P, pbuf(u + 1), pbuf(u), d + D_RZN, d + D_RZN, d + D_RZ0, s, ctl + 1);
            }
            stats_set_capturing(false);
            cudaGraph_t out = nullptr;
            const cudaError_t e = cudaStreamEndCapture(s, &out);
            ok = st == TFDE_OK && e == cudaSuccess;
        }
    }
    if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();   // the host loop stays in use; clear the capture's error state
        if (g) cudaGraphDestroy(g);
        M->pcg_graph_failed = true;
        set_error(TFDE_OK, "");
        return TFDE_OK;
    }
    M->pcg_graph = g;
    M->pcg_exec = ex;
    M->pcg_tune_gen = tc::tune_generation();
    return TFDE_OK;
}

// inner_pcg (below) with its iterations in the device-side loop: one graph
// launch and one host read per sweep (iterations done and <r, r>).
int inner_pcg_graph(const tfde_problem* P, double theta, int maxit, int* iters, PcgPending* pend, cudaStream_t s,
                    double* reached, double rr0) {
    MixedState* M = mixed(P);
    const size_t N = P->N;
    double* d = M->dsc;
    auto pbuf = [&](int j) { return M->pring + (size_t)(j % kPRing) * N; };
    *pend = PcgPending();
    if (reached) *reached = 0.0;
    launch_pcg_init(d, D_RZN, D_THR, theta * theta * rr0, M->pcg_ctl, maxit, s);
    int st = fast_precond_cg(P, pbuf(0), nullptr, d + D_RZN, nullptr, nullptr, s);   // p_0 = z_0
    if (st) return st;
    MX_TRY(cudaGraphLaunch(M->pcg_exec, s));
    ++M->graph_launches;
    MX_TRY(cudaMemcpyAsync(M->pcg_ctl_host, M->pcg_ctl, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    MX_TRY(cudaMemcpyAsync(P->red_host, d + D_RR, sizeof(double), cudaMemcpyDeviceToHost, s));
    MX_TRY(cudaStreamSynchronize(s));
    const int k = M->pcg_ctl_host[0];
    const double rr = P->red_host[0];
    // launches of the graph: 12 per iteration of a body, the fold once per body
    const int bodies = (k + kPRing - 1) / kPRing;
    stats_count_launch((unsigned)(bodies * (12 * kPRing + 1)));
    *iters = k;
    if (!std::isfinite(rr)) return set_error(TFDE_ENAN, "non-finite inner residual");
    if (reached) *reached = std::sqrt(rr / rr0);
    // the directions of the last (partial or unfolded) window
    const int j0 = kPRing * ((k - 1) / kPRing);
    pend->cnt = k - j0;
    pend->fold = k > kPRing;
    for (int j = 0; j < pend->cnt; ++j) {
        pend->p[j] = pbuf(j0 + j);
        pend->alpha[j] = d + kAlphaSlot + (j0 + j) % kPRing;
    }
    return check_err(P, s);
}

// ------------------------------------------------------------------
// The inner PCG in the sine-transform eigenbasis (symmetric problems).
// S_N = S3 (x) S2 (x) S1 is symmetric and orthogonal and diagonalises both the
// mass operator (A_n = S diag(mu) S, A_n tridiagonal Toeplitz) and the tau
// preconditioner (P = S_N Lambda S_N, Eq. (diag_tau_pre)).  PCG on A c = r
// with P is therefore PCG on (S_N A S_N) c~ = S_N r with the diagonal Lambda,
// c = S_N c~ (the same iterates in exact arithmetic: an orthogonal change of
// basis, Sec. 3.1).  In that basis an iteration is three split contractions
// (one per axis, Kronecker sum with diagonal factors on the other axes) and
// pointwise work: 3 instead of 9 split passes, the preconditioner free.

// out_f32 = S_N v, v the split planes `in`; the x and y passes write split
// planes mid1 and mid2, the z pass FP32.
int spec_transform(const tfde_problem* P, int in, int mid1, int mid2, float* out_f32, cudaStream_t s,
                   const int* skip = nullptr) {
    MixedState* M = mixed(P);
    const SegSpec sx[1] = {{OM_S2X_H, OM_S2X_L, in}}, sy[1] = {{OM_S2Y_H, OM_S2Y_L, mid1}},
                  sz[1] = {{OM_S2Z_H, OM_S2Z_L, mid2}};
    int st;
    if ((st = run_gemm(P, 0, sx, 1, tc::OUT_HILO, 1.f, nullptr, mid1, false, s, nullptr, nullptr, skip))) return st;
    if ((st = run_gemm(P, 1, sy, 1, tc::OUT_HILO, 1.f, nullptr, mid2, false, s, nullptr, nullptr, skip))) return st;
    if ((st = run_gemm(P, 2, sz, 1, tc::OUT_F32, 1.f, out_f32, -1, false, s, nullptr, nullptr, skip))) return st;
    M->spec_transforms++;
    return TFDE_OK;
}

// q = (S_N A S_N) p, p given as the split planes PL_P (and in FP32 as pf for
// the fused <p, q> into *pq):
//   x: s1 = cs_x . ((D1 + Bh1) p)_x ; y: s2 = s1 + cs_y . (Bh2 p)_y ;
//   z: q = s2 + cs_z . (Bh3 p)_z
// with Bh_a = S (eta_a B_a) S, D1 = diag(mu_1) and cs the products of the
// other axes' mass eigenvalues per line (cs_x D1 = D3 D2 D1, the mass part).
// s1, s2 live in F_Z, F_P.
// With lam_div (PGMRES): q = Lambda^{-1} (S_N A S_N) p, no inner product.
int spec_matvec(const tfde_problem* P, const float* pf, float* q, double* pq, cudaStream_t s,
                const int* skip = nullptr, bool lam_div = false) {
    MixedState* M = mixed(P);
    const long long n1 = P->n[0], n2 = P->n[1], n3 = P->n[2];
    const float* cs_x = M->spec;
    const float* cs_y = cs_x + n2 * n3;
    const float* cs_z = cs_y + n1 * n3;
    float* s1 = M->f[F_Z];
    float* s2 = M->f[F_P];
    const double N = (double)P->N;
    for (int a = 0; a < 3; ++a) {
        const SegSpec sg[1] = {{OM_BX_H + 2 * a, OM_BX_L + 2 * a, PL_P}};
        tc::Params prm;
        double bytes, flops;
        float* out = a == 0 ? s1 : (a == 1 ? s2 : q);
        gemm_params(P, a, sg, 1, tc::OUT_SUM, 1.f, out, -1, lam_div && a == 2, prm, &bytes, &flops);
        prm.col_scale = a == 0 ? cs_x : (a == 1 ? cs_y : cs_z);
        if (a > 0) {
            prm.addend = a == 1 ? s1 : s2;
            bytes += 4.0 * N;
        }
        if (a == 2 && !lam_div) {
            prm.dot_vec = pf;
            prm.dot_out = pq;
            bytes += 4.0 * N;
        }
        prm.skip = skip;
        M->gemm_launches++;
        if (int st = tc::launch(prm, s, bytes, flops)) return st;
    }
    return TFDE_OK;
}

int build_pcg_graph_spec(const tfde_problem* P, cudaStream_t s);
int inner_pcg_spec_graph(const tfde_problem* P, double theta, int maxit, int* iters, PcgPending* pend,
                         cudaStream_t s, double* reached, double rr0);

// Inner PCG in the eigenbasis: the caller has written the (scaled) residual as
// the split planes PL_R; on return F_R holds S_N r updated by the iterations
// and *pend the directions (in the eigenbasis) left to combine, as inner_pcg.
int inner_pcg_spec(const tfde_problem* P, double theta, int maxit, int* iters, PcgPending* pend, cudaStream_t s,
                   double* reached, double rr0) {
    MixedState* M = mixed(P);
    const size_t N = P->N;
    float* r = M->f[F_R];
    float* q = M->f[F_Q];
    double* d = M->dsc;
    int st = TFDE_OK;
    *pend = PcgPending();
    if (reached) *reached = 0.0;
    if (!(rr0 > 0.0) || !std::isfinite(rr0)) return rr0 == 0.0 ? TFDE_OK : set_error(TFDE_ENAN, "non-finite inner residual");
    auto pbuf = [&](int j) { return M->pring + (size_t)(j % kPRing) * N; };
    if ((st = spec_transform(P, PL_R, PL_T1, PL_T2, r, s))) return st;   // r~ = S_N r
    if (M->device_loop && !stats_timing() && maxit > 0) {
        if ((st = build_pcg_graph_spec(P, s))) return st;
        if (M->spec_exec) return inner_pcg_spec_graph(P, theta, maxit, iters, pend, s, reached, rr0);
    }
    int rz = D_RZ0;
    MX_TRY(cudaMemsetAsync(d + rz, 0, sizeof(double), s));
    // p_0 = Lambda^{-1} r~, <r~, Lambda^{-1} r~>
    if ((st = launch_spec_direction(M->lam, P->n, nullptr, nullptr, r, nullptr, pbuf(0), M->hi[PL_P], M->lo[PL_P],
                                    d + rz, s)))
        return st;
    int k = 0, j0 = 0;
    bool folded = false;
    while (k < maxit) {
        const int rzn = rz == D_RZ0 ? D_RZ1 : D_RZ0;
        MX_TRY(cudaMemsetAsync(d + D_PQ, 0, 2 * sizeof(double), s));   // <p, Ap> and <r, r>
        MX_TRY(cudaMemsetAsync(d + rzn, 0, sizeof(double), s));
        if ((st = spec_matvec(P, pbuf(k), q, d + D_PQ, s))) return st;
        if ((st = launch_spec_update(M->lam, P->n, d + rz, d + D_PQ, q, r, d + rzn, d + D_RR,
                                     d + kAlphaSlot + k % kPRing, s)))
            return st;
        const double rr = host_scalar(P, d + D_RR, s, &st);
        if (st) return st;
        ++k;
        if (!std::isfinite(rr)) return set_error(TFDE_ENAN, "non-finite inner residual");
        if (reached) *reached = std::sqrt(rr / rr0);
        if (rr <= theta * theta * rr0 || k >= maxit) break;
        if (k - j0 == kPRing) {
            PcgPending w;
            w.cnt = kPRing;
            w.fold = folded;
            for (int j = 0; j < kPRing; ++j) {
                w.p[j] = pbuf(j0 + j);
                w.alpha[j] = d + kAlphaSlot + (j0 + j) % kPRing;
            }
            launch_pcg_combine(N, w, M->f[F_X], 0.0, nullptr, nullptr, M->f[F_X], s);
            folded = true;
            j0 = k;
        }
        // p_k = Lambda^{-1} r~ + beta p_{k-1}, beta = <r, z>_new / <r, z>
        if ((st = launch_spec_direction(M->lam, P->n, d + rzn, d + rz, r, pbuf(k - 1), pbuf(k), M->hi[PL_P],
                                        M->lo[PL_P], nullptr, s)))
            return st;
        rz = rzn;
    }
    pend->cnt = k - j0;
    pend->fold = folded;
    for (int j = 0; j < pend->cnt; ++j) {
        pend->p[j] = pbuf(j0 + j);
        pend->alpha[j] = d + kAlphaSlot + (j0 + j) % kPRing;
    }
    *iters = k;
    return check_err(P, s);
}

// The iterations of inner_pcg_spec as one graph launch per sweep: a while node
// whose body runs kPRing iterations, each head -> the three eigenbasis
// passes (<p, q> fused) -> update (alpha, <r, z>, <r, r>) -> stop test ->
// direction (beta, p and its split planes); the body's window of directions
// folded into F_X before its last direction update.
int build_pcg_graph_spec(const tfde_problem* P, cudaStream_t s) {
    MixedState* M = mixed(P);
    if (M->spec_exec && M->spec_tune_gen != tc::tune_generation()) {
        cudaGraphExecDestroy(M->spec_exec);
        cudaGraphDestroy(M->spec_graph);
        M->spec_exec = nullptr;
        M->spec_graph = nullptr;
    }
    if (M->spec_exec || M->spec_graph_failed) return TFDE_OK;
    const size_t N = P->N;
    if (int st = tc::set_attrs()) return st;
    float* q = M->f[F_Q];
    float* r = M->f[F_R];
    double* d = M->dsc;
    int* ctl = M->pcg_ctl;
    auto pbuf = [&](int j) { return M->pring + (size_t)(j % kPRing) * N; };
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
    cudaGraphConditionalHandle h{};
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    if (ok) ok = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
    }
    if (ok) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        // captured on a stream of its own (the caller's may be the legacy default stream)
        const cudaStream_t s = capture_stream();
        ok = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
             cudaSuccess;
        if (ok) {
            stats_set_capturing(true);
            int st = TFDE_OK;
            const float* ps[kPRing];
            const double* as[kPRing];
            for (int u = 0; u < kPRing; ++u) {
                ps[u] = pbuf(u);
                as[u] = d + kAlphaSlot + u;
            }
            for (int u = 0; u < kPRing && !st; ++u) {
                launch_pcg_head(d, D_RZ0, D_RZN, D_PQ, D_RR, ctl, s);
                st = spec_matvec(P, pbuf(u), q, d + D_PQ, s, ctl + 1);
                if (!st) st = launch_spec_update(M->lam, P->n, d + D_RZ0, d + D_PQ, q, r, d + D_RZN, d + D_RR,
                                                 d + kAlphaSlot + u, s, ctl + 1);
                if (st) break;
                launch_pcg_cond(h, d + D_RR, d + D_THR, ctl, s);
                if (u == kPRing - 1) launch_pcg_fold_dev(N, ps, as, M->f[F_X], ctl, s);
                st = launch_spec_direction(M->lam, P->n, d + D_RZN, d + D_RZ0, r, pbuf(u), pbuf(u + 1), M->hi[PL_P],
                                           M->lo[PL_P], nullptr, s, ctl + 1);
            }
            stats_set_capturing(false);
            cudaGraph_t out = nullptr;
            const cudaError_t e = cudaStreamEndCapture(s, &out);
            ok = st == TFDE_OK && e == cudaSuccess;
        }
    }
    if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        M->spec_graph_failed = true;
        set_error(TFDE_OK, "");
        return TFDE_OK;
    }
    M->spec_graph = g;
    M->spec_exec = ex;
    M->spec_tune_gen = tc::tune_generation();
    return TFDE_OK;
}

int inner_pcg_spec_graph(const tfde_problem* P, double theta, int maxit, int* iters, PcgPending* pend,
                         cudaStream_t s, double* reached, double rr0) {
    MixedState* M = mixed(P);
    const size_t N = P->N;
    double* d = M->dsc;
    auto pbuf = [&](int j) { return M->pring + (size_t)(j % kPRing) * N; };
    launch_pcg_init(d, D_RZN, D_THR, theta * theta * rr0, M->pcg_ctl, maxit, s);
    int st = launch_spec_direction(M->lam, P->n, nullptr, nullptr, M->f[F_R], nullptr, pbuf(0), M->hi[PL_P],
                                   M->lo[PL_P], d + D_RZN, s);   // p_0 = Lambda^{-1} r~
    if (st) return st;
    MX_TRY(cudaGraphLaunch(M->spec_exec, s));
    ++M->graph_launches;
    MX_TRY(cudaMemcpyAsync(M->pcg_ctl_host, M->pcg_ctl, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    MX_TRY(cudaMemcpyAsync(P->red_host, d + D_RR, sizeof(double), cudaMemcpyDeviceToHost, s));
    MX_TRY(cudaStreamSynchronize(s));
    const int k = M->pcg_ctl_host[0];
    const double rr = P->red_host[0];
    // launches of the graph: 7 per iteration of a body (3 of them split), the fold once per body
    const int bodies = (k + kPRing - 1) / kPRing;
    stats_count_launch((unsigned)(bodies * (7 * kPRing + 1)));
    *iters = k;
    if (!std::isfinite(rr)) return set_error(TFDE_ENAN, "non-finite inner residual");
    if (reached) *reached = std::sqrt(rr / rr0);
    const int j0 = kPRing * ((k - 1) / kPRing);
    pend->cnt = k - j0;
    pend->fold = k > kPRing;
    for (int j = 0; j < pend->cnt; ++j) {
        pend->p[j] = pbuf(j0 + j);
        pend->alpha[j] = d + kAlphaSlot + (j0 + j) % kPRing;
    }
    return check_err(P, s);
}

// The eigenbasis solution d~ = (fold ? F_X : 0) + sum alpha_j p_j back to the
// grid: F_X = S_N d~ (the combination and its split planes, then three passes).
int spec_finish(const tfde_problem* P, const PcgPending& pend, cudaStream_t s) {
    MixedState* M = mixed(P);
    if (int st = launch_pcg_combine_split(P->N, pend, M->f[F_X], M->hi[PL_T1], M->lo[PL_T1], s)) return st;
    return spec_transform(P, PL_T1, PL_T2, PL_R, M->f[F_X], s);
}

// ---- left-preconditioned GMRES in the eigenbasis (Sec. 3.2): the Arnoldi
// vectors live in the eigenbasis, Lambda^{-1} S_N A S_N v is three split
// passes with the division fused into the last, and the cycle's correction
// goes back through S_N once.  Inner products and norms are those of the grid
// basis (S_N is orthogonal), so the cycle's iterates are the grid-basis ones.
int build_gmres_graph_spec(const tfde_problem* P, int restart, cudaStream_t s) {
    MixedState* M = mixed(P);
    if (M->gms_graph_failed || restart > GS_MAXM) return TFDE_OK;
    if (M->gms_exec && M->gms_graph_restart == restart && M->gms_tune_gen == tc::tune_generation()) return TFDE_OK;
    if (M->gms_exec) {
        cudaGraphExecDestroy(M->gms_exec);
        cudaGraphDestroy(M->gms_graph);
        M->gms_exec = nullptr;
        M->gms_graph = nullptr;
    }
    if (int st = tc::set_attrs()) return st;
    const size_t N = P->N;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
    cudaGraphConditionalHandle h{};
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    if (ok) ok = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
    }
    if (ok) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        // captured on a stream of its own (the caller's may be the legacy default stream)
        const cudaStream_t s = capture_stream();
        ok = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
             cudaSuccess;
        if (ok) {
            stats_set_capturing(true);
            const int* skip = M->gm_ctl + 1;
            int st = spec_matvec(P, nullptr, M->f[F_Z], nullptr, s, skip, true);   // w = Lambda^{-1} A~ v_j
            if (!st)
                launch_gm_step(N, M->V32, M->f[F_Z], P->red, P->nblk, M->gm + GM_H, M->gm + GM_H2, M->gm + GM_WW,
                               M->gm_state, M->gm_ctl, h, nullptr, M->hi[PL_P], M->lo[PL_P], restart + 1, s);
            stats_set_capturing(false);
            cudaGraph_t out = nullptr;
            const cudaError_t e = cudaStreamEndCapture(s, &out);
            ok = st == TFDE_OK && e == cudaSuccess;
        }
    }
    if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        M->gms_graph_failed = true;
        set_error(TFDE_OK, "");
        return TFDE_OK;
    }
    M->gms_graph = g;
    M->gms_exec = ex;
    M->gms_graph_restart = restart;
    M->gms_tune_gen = tc::tune_generation();
    return TFDE_OK;
}

// One GMRES cycle in the eigenbasis: the caller has written the scaled
// residual as split planes PL_R; on return F_X = S_N d~ (the cycle's
// correction in the grid basis), as inner_gmres leaves d in F_X.
int inner_gmres_spec(const tfde_problem* P, int restart, double ptheta, int maxit, int* iters, double* est_ratio,
                     cudaStream_t s) {
    MixedState* M = mixed(P);
    const size_t N = P->N;
    float* V = M->V32;
    double* g = M->gm;
    int st;
    *iters = 0;
    *est_ratio = 1.0;
    if ((st = spec_transform(P, PL_R, PL_T1, PL_T2, M->f[F_R], s))) return st;   // r~ = S_N r
    // w = Lambda^{-1} r~ (FP32 into F_Z; its planes are overwritten by the cycle start)
    if ((st = launch_spec_direction(M->lam, P->n, nullptr, nullptr, M->f[F_R], nullptr, M->f[F_Z], M->hi[PL_P],
                                    M->lo[PL_P], nullptr, s)))
        return st;
    MX_TRY(cudaMemsetAsync(M->f[F_X], 0, N * sizeof(float), s));
    int k = 0;
    if (M->device_loop && !stats_timing() && maxit > 0 && restart <= GS_MAXM) {
        if ((st = build_gmres_graph_spec(P, restart, s))) return st;
    }
    if (M->device_loop && !stats_timing() && maxit > 0 && M->gms_exec && M->gms_graph_restart == restart) {
        MX_TRY(cudaMemsetAsync(M->gm_ctl, 0, 4 * sizeof(int), s));
        const int maxsteps = restart < maxit ? restart : maxit;
        launch_gm_start(N, M->f[F_Z], P->red, P->nblk, g + GM_WW, M->gm_state, M->gm_ctl, maxsteps, ptheta, V,
                        M->hi[PL_P], M->lo[PL_P], s);
        MX_TRY(cudaGraphLaunch(M->gms_exec, s));
        ++M->graph_launches;
        launch_gm_solve(M->gm_state, M->gm_ctl, g + GM_Y, restart, s);
        launch_multiaxpy32(N, restart, V, N, g + GM_Y, M->f[F_X], s);   // x32 = sum_i y_i v_i
        MX_TRY(cudaMemcpyAsync(M->gm_ctl_host, M->gm_ctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
        MX_TRY(cudaMemcpyAsync(P->red_host, M->gm_state, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        MX_TRY(cudaStreamSynchronize(s));
        k = M->gm_ctl_host[0];
        stats_count_launch((unsigned)(k > 0 ? k : 1) * 11u);   // the graph's launches, 11 per step
        const double beta = P->red_host[GS_BETA], est = P->red_host[GS_EST];
        if (M->gm_ctl_host[3] || !std::isfinite(beta))
            return set_error(TFDE_ENAN, "non-finite preconditioned residual or Arnoldi vector");
        *iters = k;
        *est_ratio = beta > 0.0 ? est / beta : 1.0;
    } else {
        double* gh = M->gm_host;
        MX_TRY(cudaMemcpyAsync(V, M->f[F_Z], N * sizeof(float), cudaMemcpyDeviceToDevice, s));
        launch_dot32(N, V, V, P->red, P->nblk, s);
        launch_reduce_finish(P->red, P->nblk, 1, g + GM_WW, s);
        MX_TRY(cudaMemcpyAsync(gh + GM_WW, g + GM_WW, sizeof(double), cudaMemcpyDeviceToHost, s));
        MX_TRY(cudaStreamSynchronize(s));
        const double beta = std::sqrt(gh[GM_WW]);
        if (!std::isfinite(beta)) return set_error(TFDE_ENAN, "non-finite preconditioned residual");
        if (beta > 0.0) {
            launch_scale_split32(N, (float)(1.0 / beta), V, V, M->hi[PL_P], M->lo[PL_P], s);
            GivensLS ls(restart);
            ls.g[0] = beta;
            std::vector<double> h(restart + 2);
            double est = beta;
            for (int j = 0; j < restart && j < maxit; ++j) {
                float* w = V + (size_t)(j + 1) * N;
                if ((st = spec_matvec(P, nullptr, w, nullptr, s, nullptr, true))) return st;   // w = Lambda^{-1} A~ v_j
                launch_multidot32(N, j + 1, V, N, w, P->red, P->nblk, s);
                launch_reduce_finish(P->red, P->nblk, j + 1, g + GM_H, s);
                launch_multiaxpy32(N, j + 1, V, N, g + GM_H, w, s);
                launch_multidot32(N, j + 1, V, N, w, P->red, P->nblk, s);
                launch_reduce_finish(P->red, P->nblk, j + 1, g + GM_H2, s);
                launch_multiaxpy32(N, j + 1, V, N, g + GM_H2, w, s);
                launch_dot32(N, w, w, P->red, P->nblk, s);
                launch_reduce_finish(P->red, P->nblk, 1, g + GM_WW, s);
                MX_TRY(cudaMemcpyAsync(gh, g, (GM_WW + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
                MX_TRY(cudaStreamSynchronize(s));
                for (int i = 0; i <= j; ++i) h[i] = gh[GM_H + i] + gh[GM_H2 + i];
                const double hn = std::sqrt(gh[GM_WW]);
                if (!std::isfinite(hn)) return set_error(TFDE_ENAN, "non-finite Arnoldi vector");
                h[j + 1] = hn;
                est = ls.add_column(j, h.data());
                k = j + 1;
                if (est <= ptheta * beta || hn == 0.0) break;
                launch_scale_split32(N, (float)(1.0 / hn), w, w, M->hi[PL_P], M->lo[PL_P], s);
            }
            *iters = k;
            *est_ratio = est / beta;
            if (k > 0) {
                std::vector<double> y;
                ls.solve(k, y);
                for (int i = 0; i < k; ++i) gh[GM_Y + i] = -y[i];
                MX_TRY(cudaMemcpyAsync(g + GM_Y, gh + GM_Y, k * sizeof(double), cudaMemcpyHostToDevice, s));
                launch_multiaxpy32(N, k, V, N, g + GM_Y, M->f[F_X], s);   // x32 = sum_i y_i v_i
            }
        }
    }
    // back to the grid basis: F_X = S_N x32
    launch_split32(N, M->f[F_X], M->hi[PL_T1], M->lo[PL_T1], s);
    if ((st = spec_transform(P, PL_T1, PL_T2, PL_R, M->f[F_X], s))) return st;
    return check_err(P, s);
}

// r = b - A x (accurate) and ||r||, the norm accumulated by the last pass of
// the contraction with the terms scaled by 2^-ilogb(nb).
// With an_out, A_N x also goes there (from the z-pass digit slicing).
int accurate_residual(const tfde_problem* P, const double* b, const double* x, double* r, double* nr, double tol,
                      double nb, cudaStream_t s, double* an_out = nullptr) {
    const int shift = nb > 0.0 && std::isfinite(nb) ? -std::ilogb(nb) : 0;
    double* acc = P->red_out + kNormsSlot + 2;
    int st = accurate_apply_ex(P, TFDE_OP_A, x, r, -1, b, 1.0, s, oz_slices_for_tol(tol), acc, shift, an_out);
    if (st) return st;
    MX_TRY(cudaMemcpyAsync(P->red_host, acc, sizeof(double), cudaMemcpyDeviceToHost, s));
    MX_TRY(cudaStreamSynchronize(s));
    *nr = std::ldexp(std::sqrt(P->red_host[0]), -shift);
    return TFDE_OK;
}

// ||b||^2 and (when r_given) ||r_0||^2: from the chain kernels of cn_prepare
// when it left them in red_out, else by FP64 dots.
int initial_norms(tfde_problem* P, const double* b, const double* r, bool r_given, double* bb, double* rr,
                  cudaStream_t s) {
    int st;
    if (r_given && P->norms_ready) {
        P->norms_ready = false;
        MX_TRY(cudaMemcpyAsync(P->red_host, P->red_out + kNormsSlot, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        MX_TRY(cudaStreamSynchronize(s));
        *bb = P->red_host[0];
        *rr = P->red_host[1];
        return TFDE_OK;
    }
    P->norms_ready = false;
    if ((st = dots64(P, 1, b, 0, b, bb, s))) return st;
    if (r_given && (st = dots64(P, 1, r, 0, r, rr, s))) return st;
    return TFDE_OK;
}


int ensure_v32(const tfde_problem* P, int restart) {
    MixedState* M = mixed(P);
    if (!M->gm) {
        MX_TRY(cudaMalloc((void**)&M->gm, GM_SIZE * sizeof(double)));
        MX_TRY(cudaMallocHost((void**)&M->gm_host, GM_SIZE * sizeof(double)));
    }
    if (M->v32_cap >= restart) return TFDE_OK;
    cudaFree(M->V32);
    M->V32 = nullptr;
    M->v32_cap = 0;
    if (cudaMalloc((void**)&M->V32, (size_t)(restart + 1) * P->N * sizeof(float)) != cudaSuccess)
        return set_error(TFDE_ENOMEM, "cudaMalloc of the FP32 GMRES basis failed");
    M->v32_cap = restart;
    return TFDE_OK;
}

// The inner GMRES cycle's Arnoldi steps as one graph: a while node whose
// body is one step -- operator (3 split launches, result in the split planes
// PL_R), preconditioner into the fixed vector F_Z (6), classical Gram-Schmidt
// with one re-orthogonalisation against V_0..V_j, ||w||, the Givens update
// and stop test on the device (the loop condition), V_{j+1} = w / ||w|| --
// with every count and address taken from the control words on the device.
// Built for one restart length; a failure leaves the host-driven cycle in use.
int build_gmres_graph(const tfde_problem* P, int restart, cudaStream_t s) {
    MixedState* M = mixed(P);
    if (M->gm_graph_failed || restart > GS_MAXM) return TFDE_OK;
    if (M->gm_exec && M->gm_graph_restart == restart && M->gm_tune_gen == tc::tune_generation()) return TFDE_OK;
    if (M->gm_exec) {
        cudaGraphExecDestroy(M->gm_exec);
        cudaGraphDestroy(M->gm_graph);
        M->gm_exec = nullptr;
        M->gm_graph = nullptr;
    }
    if (!M->gm_state) {
        MX_TRY(cudaMalloc((void**)&M->gm_state, GS_WORDS * sizeof(double)));
        MX_TRY(cudaMalloc((void**)&M->gm_ctl, 4 * sizeof(int)));
        MX_TRY(cudaMallocHost((void**)&M->gm_ctl_host, 4 * sizeof(int)));
    }
    if (int st = ensure_pairs(P, s)) return st;
    if (int st = tc::set_attrs()) return st;
    const size_t N = P->N;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
    cudaGraphConditionalHandle h{};
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    if (ok) ok = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
    }
    if (ok) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        // captured on a stream of its own (the caller's may be the legacy default stream)
        const cudaStream_t s = capture_stream();
        ok = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
             cudaSuccess;
        if (ok) {
            stats_set_capturing(true);
            const int* skip = M->gm_ctl + 1;
            int st = fast_matvec(P, TFDE_OP_A, nullptr, s, PL_R, nullptr, nullptr, skip);
            if (!st) st = fast_precond(P, M->f[F_Z], s, nullptr, nullptr, skip);
            if (!st)
                launch_gm_step(N, M->V32, M->f[F_Z], P->red, P->nblk, M->gm + GM_H, M->gm + GM_H2, M->gm + GM_WW,
                               M->gm_state, M->gm_ctl, h, nullptr, M->hi[PL_P], M->lo[PL_P], restart + 1, s);
            stats_set_capturing(false);
            cudaGraph_t out = nullptr;
            const cudaError_t e = cudaStreamEndCapture(s, &out);
            ok = st == TFDE_OK && e == cudaSuccess;
        }
    }
    if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        M->gm_graph_failed = true;
        set_error(TFDE_OK, "");
        return TFDE_OK;
    }
    M->gm_graph = g;
    M->gm_exec = ex;
    M->gm_graph_restart = restart;
    M->gm_tune_gen = tc::tune_generation();
    return TFDE_OK;
}

// inner_gmres (below) with the Arnoldi steps in the device-side loop: the
// cycle start, one graph launch, the least-squares solve and x32 = sum y_i v_i
// on the device, one host read per cycle (steps done, residual estimate).
int inner_gmres_graph(const tfde_problem* P, int restart, double ptheta, int maxit, int* iters, double* est_ratio,
                      cudaStream_t s) {
    MixedState* M = mixed(P);
    const size_t N = P->N;
    *iters = 0;
    *est_ratio = 1.0;
    MX_TRY(cudaMemsetAsync(M->gm_ctl, 0, 4 * sizeof(int), s));
    int st = fast_precond(P, M->f[F_Z], s);   // w = P^{-1} r
    if (st) return st;
    const int maxsteps = restart < maxit ? restart : maxit;
    launch_gm_start(N, M->f[F_Z], P->red, P->nblk, M->gm + GM_WW, M->gm_state, M->gm_ctl, maxsteps, ptheta, M->V32,
                    M->hi[PL_P], M->lo[PL_P], s);
    MX_TRY(cudaGraphLaunch(M->gm_exec, s));
    ++M->graph_launches;
    launch_gm_solve(M->gm_state, M->gm_ctl, M->gm + GM_Y, restart, s);
    launch_multiaxpy32(N, restart, M->V32, N, M->gm + GM_Y, M->f[F_X], s);   // x32 = sum_i y_i v_i
    MX_TRY(cudaMemcpyAsync(M->gm_ctl_host, M->gm_ctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    MX_TRY(cudaMemcpyAsync(P->red_host, M->gm_state, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    MX_TRY(cudaStreamSynchronize(s));
    const int k = M->gm_ctl_host[0];
    stats_count_launch((unsigned)(k > 0 ? k : 1) * 17u);   // the graph's launches, 17 per step
    const double beta = P->red_host[GS_BETA], est = P->red_host[GS_EST];
    if (M->gm_ctl_host[3] || !std::isfinite(beta))
        return set_error(TFDE_ENAN, "non-finite preconditioned residual or Arnoldi vector");
    *iters = k;
    *est_ratio = beta > 0.0 ? est / beta : 1.0;
    return check_err(P, s);
}

// One cycle of left-preconditioned GMRES on P^{-1} A d = P^{-1} r32 (Sec. 3.2,
// Eq. (one_side_system)) with FP32 basis vectors, split-BF16 tensor-core
// operator and preconditioner applications, classical Gram-Schmidt with one
// re-orthogonalisation (coefficients stay on the device) and host Givens
// rotations: one host read per Arnoldi step.  r32 and its split planes PL_R
// are prepared by the caller and x32 = 0; on return x32 = d.  The cycle stops
// after `restart` steps or once the preconditioned residual estimate falls
// below ptheta * beta.  *est_ratio = final estimate / beta.
int inner_gmres(const tfde_problem* P, int restart, double ptheta, int maxit, int* iters, double* est_ratio,
                cudaStream_t s) {
    MixedState* M = mixed(P);
    if (M->device_loop && !stats_timing() && maxit > 0 && restart <= GS_MAXM) {
        if (int st = build_gmres_graph(P, restart, s)) return st;
        if (M->gm_exec) return inner_gmres_graph(P, restart, ptheta, maxit, iters, est_ratio, s);
    }
    const size_t N = P->N;
    float* V = M->V32;
    double* g = M->gm;
    double* gh = M->gm_host;
    int st;
    *iters = 0;
    *est_ratio = 1.0;
    // v_0 = P^{-1} r / beta
    if ((st = fast_precond(P, V, s))) return st;
    launch_dot32(N, V, V, P->red, P->nblk, s);
    launch_reduce_finish(P->red, P->nblk, 1, g + GM_WW, s);
    MX_TRY(cudaMemcpyAsync(gh + GM_WW, g + GM_WW, sizeof(double), cudaMemcpyDeviceToHost, s));
    MX_TRY(cudaStreamSynchronize(s));
    const double beta = std::sqrt(gh[GM_WW]);
    if (!std::isfinite(beta)) return set_error(TFDE_ENAN, "non-finite preconditioned residual");
    if (!(beta > 0.0)) return TFDE_OK;
    launch_scale_split32(N, (float)(1.0 / beta), V, V, M->hi[PL_P], M->lo[PL_P], s);
    GivensLS ls(restart);
    ls.g[0] = beta;
    std::vector<double> h(restart + 2);
    double est = beta;
    int k = 0;
    for (int j = 0; j < restart && j < maxit; ++j) {
        float* w = V + (size_t)(j + 1) * N;
        // w = P^{-1} A v_j  (A v_j leaves the contraction as split planes PL_R)
        if ((st = fast_matvec(P, TFDE_OP_A, nullptr, s, PL_R))) return st;
        if ((st = fast_precond(P, w, s))) return st;
        // CGS2 with the coefficients on the device
        launch_multidot32(N, j + 1, V, N, w, P->red, P->nblk, s);
        launch_reduce_finish(P->red, P->nblk, j + 1, g + GM_H, s);
        launch_multiaxpy32(N, j + 1, V, N, g + GM_H, w, s);
        launch_multidot32(N, j + 1, V, N, w, P->red, P->nblk, s);
        launch_reduce_finish(P->red, P->nblk, j + 1, g + GM_H2, s);
        launch_multiaxpy32(N, j + 1, V, N, g + GM_H2, w, s);
        launch_dot32(N, w, w, P->red, P->nblk, s);
        launch_reduce_finish(P->red, P->nblk, 1, g + GM_WW, s);
        MX_TRY(cudaMemcpyAsync(gh, g, (GM_WW + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
        MX_TRY(cudaStreamSynchronize(s));
        for (int i = 0; i <= j; ++i) h[i] = gh[GM_H + i] + gh[GM_H2 + i];
        const double hn = std::sqrt(gh[GM_WW]);
        if (!std::isfinite(hn)) return set_error(TFDE_ENAN, "non-finite Arnoldi vector");
        h[j + 1] = hn;
        est = ls.add_column(j, h.data());
        k = j + 1;
        if (est <= ptheta * beta || hn == 0.0) break;
        launch_scale_split32(N, (float)(1.0 / hn), w, w, M->hi[PL_P], M->lo[PL_P], s);
    }
    *iters = k;
    *est_ratio = est / beta;
    if (k > 0) {
        std::vector<double> y;
        ls.solve(k, y);
        for (int i = 0; i < k; ++i) gh[GM_Y + i] = -y[i];
        MX_TRY(cudaMemcpyAsync(g + GM_Y, gh + GM_Y, k * sizeof(double), cudaMemcpyHostToDevice, s));
        launch_multiaxpy32(N, k, V, N, g + GM_Y, M->f[F_X], s);   // x32 = sum_i y_i v_i
    }
    return check_err(P, s);
}

}  // namespace

int fast_pass_descriptors(const tfde_problem* P, int kind, float* out_f32, tc::Params* prm, int* axes, double* bytes,
                          double* flops) {
    Pass ps[6];
    const int np = kind == 0 ? matvec_passes(TFDE_OP_A, PL_R, ps) : precond_passes(ps);
    for (int i = 0; i < np; ++i) {
        const Pass& q = ps[i];
        gemm_params(P, q.axis, q.seg, q.nseg, q.out_mode, 1.f, q.out_mode == tc::OUT_F32 ? out_f32 : nullptr,
                    q.out_plane, q.lam, prm[i], &bytes[i], &flops[i]);
        axes[i] = q.axis;
    }
    return np;
}

int spec_pass_descriptors(const tfde_problem* P, int kind, float* out_f32, tc::Params* prm, int* axes, double* bytes,
                          double* flops, const float* dot_vec, double* dot_out) {
    MixedState* M = mixed(P);
    const long long n1 = P->n[0], n2 = P->n[1], n3 = P->n[2];
    const double N = (double)P->N;
    for (int a = 0; a < 3; ++a) {
        tc::Params& q = prm[a];
        axes[a] = a;
        if (kind == 3) {
            const SegSpec sg[1] = {{OM_BX_H + 2 * a, OM_BX_L + 2 * a, PL_P}};
            float* out = a == 0 ? M->f[F_Z] : (a == 1 ? M->f[F_P] : out_f32);
            gemm_params(P, a, sg, 1, tc::OUT_SUM, 1.f, out, -1, a == 2 && !dot_out, q, &bytes[a], &flops[a]);
            q.col_scale = M->spec + (a == 0 ? 0 : (a == 1 ? n2 * n3 : n2 * n3 + n1 * n3));
            if (a > 0) {
                q.addend = a == 1 ? M->f[F_Z] : M->f[F_P];
                bytes[a] += 4.0 * N;
            }
            if (a == 2 && dot_out) {
                q.dot_vec = dot_vec;
                q.dot_out = dot_out;
                bytes[a] += 4.0 * N;
            }
        } else {
            const bool fwd = kind == 2 || kind == 5;
            const int in = fwd ? (a == 0 ? PL_R : (a == 1 ? PL_T1 : PL_T2)) : (a == 0 ? PL_T1 : (a == 1 ? PL_T2 : PL_R));
            const int outp = fwd ? (a == 0 ? PL_T1 : PL_T2) : (a == 0 ? PL_T2 : PL_R);
            const SegSpec sg[1] = {{OM_S2X_H + 2 * a, OM_S2X_L + 2 * a, in}};
            const int mode = a < 2 ? tc::OUT_HILO : (kind == 2 ? tc::OUT_SUM : tc::OUT_F32);
            gemm_params(P, a, sg, 1, mode, 1.f, a == 2 ? out_f32 : nullptr, a < 2 ? outp : -1, kind == 2 && a == 2, q,
                        &bytes[a], &flops[a]);
        }
        q.err = M->err;
    }
    return 3;
}

int mixed_prepare_gmres(const tfde_problem* P, int restart) { return ensure_v32(P, restart); }

namespace {
// Device copy of operator matrix om (n x n BF16) with its tensor maps; the lo
// of a hi / lo pair lives in the second half of the pair's allocation, and
// the hi of a pair also gets the merged 3-D box that loads both terms.
int upload_matrix(MixedState* M, int om, const std::vector<__nv_bfloat16>& h, int n, bool pair_hi, bool pair_lo,
                  cudaStream_t s) {
    if (pair_lo) {
        M->mat[om] = M->mat[om - 1] + h.size();
    } else {
        MX_TRY(cudaMalloc((void**)&M->mat[om], (pair_hi ? 2 : 1) * h.size() * sizeof(__nv_bfloat16)));
        M->own_mat[om] = true;
    }
    MX_TRY(cudaMemcpyAsync(M->mat[om], h.data(), h.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice, s));
    MX_TRY(cudaStreamSynchronize(s));
    int st = tc::make_split_map_A(&M->amap[om], M->mat[om], n);
    if (st) return st;
    if (pair_hi) {
        // hi and lo of the pair as one 3-D tensor (k, row, term)
        const cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, 2};
        const cuuint64_t strides[2] = {(cuuint64_t)n * 2, (cuuint64_t)n * n * 2};
        const cuuint32_t box[3] = {(cuuint32_t)tc::SK, (cuuint32_t)tc::BM, 2};
        M->has_amap2[om] = tc::encode_map(&M->amap2[om], M->mat[om], 3, dims, strides, box,
                                          CU_TENSOR_MAP_SWIZZLE_128B) == TFDE_OK;
    }
    return TFDE_OK;
}
}  // namespace

int mixed_init(tfde_problem* P, cudaStream_t s) {
    for (int a = 0; a < 3; ++a)
    {
        if (P->n[a] % 8 != 0)
            return set_error(TFDE_EUNSUPPORTED, "TFDE_MIXED needs every n_a to be a multiple of 8");
        // exact FP32 diagonal sums of the slice contraction: n (36864 + 24576 / n) < 2^24
        if (P->n[a] > 448)
            return set_error(TFDE_EUNSUPPORTED, "TFDE_MIXED supports n_a <= 448");
    }
    MixedState* M = new MixedState();
    P->mixed = M;
    const size_t N = P->N;
    // operator matrices
    for (int om = 0; om < NOM_BASE; ++om) {
        int a;
        if (om <= OM_GHATR_L || om == OM_MX || om == OM_SX) a = 0;
        else if ((om >= OM_GY_H && om <= OM_GYN_L) || om == OM_MY || om == OM_SY) a = 1;
        else a = 2;
        const int n = P->n[a];
        std::vector<__nv_bfloat16> h((size_t)n * n);
        if (om == OM_MX || om == OM_MY || om == OM_MZ) {
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) h[(size_t)i * n + j] = __float2bfloat16_rn((float)mass_entry(i, j));
        } else if (om == OM_SX || om == OM_SY || om == OM_SZ) {
            const std::vector<double> S = dst_dense(n);
            for (size_t e = 0; e < h.size(); ++e) h[e] = __float2bfloat16_rn((float)S[e]);
        } else {
            const std::vector<double> B = dense_etaB(P, a);
            const bool lo = (om == OM_GHAT_L || om == OM_GHATR_L || om == OM_GY_L || om == OM_GYN_L ||
                             om == OM_GZ_L || om == OM_GZN_L);
            double sgn = 1.0, mass = 0.0;
            if (om == OM_GHAT_H || om == OM_GHAT_L) mass = 1.0;
            if (om == OM_GHATR_H || om == OM_GHATR_L) { mass = 1.0; sgn = -1.0; }
            if (om == OM_GYN_H || om == OM_GYN_L || om == OM_GZN_H || om == OM_GZN_L) sgn = -1.0;
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    const double v = mass * mass_entry(i, j) + sgn * B[(size_t)i * n + j];
                    __nv_bfloat16 vh, vl;
                    to_bf16_pair(v, vh, vl);
                    h[(size_t)i * n + j] = lo ? vl : vh;
                }
        }
        const bool pair_hi = om == OM_GHAT_H || om == OM_GHATR_H || om == OM_GY_H || om == OM_GYN_H || om == OM_GZ_H ||
                             om == OM_GZN_H;
        const bool pair_lo = om == OM_GHAT_L || om == OM_GHATR_L || om == OM_GY_L || om == OM_GYN_L || om == OM_GZ_L ||
                             om == OM_GZN_L;
        if (int st = upload_matrix(M, om, h, n, pair_hi, pair_lo, s)) return st;
    }
    // the inner solves in the sine-transform eigenbasis (Sec. 3.1, 3.2): per
    // axis S_n (eta_a B_a) S_n and S_n itself, each split into hi + lo
    {
        for (int a = 0; a < 3; ++a) {
            const int n = P->n[a];
            const std::vector<double> S = dst_dense(n);
            const std::vector<double> E = dense_etaB(P, a);
            std::vector<double> T((size_t)n * n, 0.0), Bh((size_t)n * n, 0.0);
            for (int i = 0; i < n; ++i)          // T = S E
                for (int k = 0; k < n; ++k) {
                    const double sik = S[(size_t)i * n + k];
                    const double* er = E.data() + (size_t)k * n;
                    double* tr = T.data() + (size_t)i * n;
                    for (int j = 0; j < n; ++j) tr[j] += sik * er[j];
                }
            for (int i = 0; i < n; ++i)          // Bh = T S
                for (int k = 0; k < n; ++k) {
                    const double tik = T[(size_t)i * n + k];
                    const double* sr = S.data() + (size_t)k * n;
                    double* br = Bh.data() + (size_t)i * n;
                    for (int j = 0; j < n; ++j) br[j] += tik * sr[j];
                }
            // the x axis also carries the mass eigenvalues mu_1 on its diagonal:
            // its per-line factor mu_2 mu_3 then gives the whole D3 D2 D1 term
            if (a == 0)
                for (int i = 0; i < n; ++i) Bh[(size_t)i * n + i] += P->lam_mass[0][i];
            const int ob = OM_BX_H + 2 * a, os = OM_S2X_H + 2 * a;
            for (int part = 0; part < 2; ++part) {
                const std::vector<double>& src = part == 0 ? Bh : S;
                const int om = part == 0 ? ob : os;
                std::vector<__nv_bfloat16> hh((size_t)n * n), hl((size_t)n * n);
                for (size_t e = 0; e < hh.size(); ++e) to_bf16_pair(src[e], hh[e], hl[e]);
                if (int st = upload_matrix(M, om, hh, n, true, false, s)) return st;
                if (int st = upload_matrix(M, om + 1, hl, n, false, true, s)) return st;
            }
        }
    }
    {
        std::vector<double> etaB[3];
        for (int a = 0; a < 3; ++a) etaB[a] = dense_etaB(P, a);
        int st = oz_init(P, etaB, s);
        if (st) return st;
    }
    // workspace planes and their tensor maps
    for (int pl = 0; pl < NPL; ++pl) {
        MX_TRY(cudaMalloc((void**)&M->hi[pl], 2 * N * sizeof(__nv_bfloat16)));
        M->lo[pl] = M->hi[pl] + N;
        MX_TRY(cudaMemsetAsync(M->hi[pl], 0, 2 * N * sizeof(__nv_bfloat16), s));
        for (int a = 0; a < 3; ++a) {
            int st = tc::make_map_B(&M->bmap_hi[pl][a], M->hi[pl], P->n, a);
            if (!st) st = tc::make_map_B(&M->bmap_lo[pl][a], M->lo[pl], P->n, a);
            if (st) return st;
            M->bmap2_rank[pl][a] = tc::make_map_B_pair(&M->bmap2[pl][a], M->hi[pl], P->n, a);
            M->bmap1_rank[pl][a] = tc::make_map_B_pair(&M->bmap1[pl][a], M->hi[pl], P->n, a, 1);
            if ((st = tc::make_out_map(&M->omap_hi[pl][a], M->hi[pl], P->n, a, false)) ||
                (st = tc::make_out_map_pair(&M->omap_hl[pl][a], M->hi[pl], P->n, a)))
                return st;
        }
    }
    for (int v = 0; v < NF; ++v) {
        MX_TRY(cudaMalloc((void**)&M->f[v], N * sizeof(float)));
        MX_TRY(cudaMemsetAsync(M->f[v], 0, N * sizeof(float), s));
    }
    // z-pass scale: Lambda(i,j,k) = ra[k] U[i + n1 j] + rb[k] V[i + n1 j]  (Eq. (diag_tau_pre))
    {
        const int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2];
        std::vector<float> lam(2 * (size_t)n3 + 2 * (size_t)n1 * n2);
        for (int k = 0; k < n3; ++k) {
            lam[k] = (float)P->lam_mass[2][k];
            lam[n3 + k] = (float)(P->csum[2] * P->lam_tau[2][k]);
        }
        for (int j = 0; j < n2; ++j)
            for (int i = 0; i < n1; ++i) {
                const double a1 = P->lam_mass[0][i], a2 = P->lam_mass[1][j];
                const double l1 = P->lam_tau[0][i], l2 = P->lam_tau[1][j];
                const size_t c = (size_t)i + (size_t)n1 * j;
                lam[2 * (size_t)n3 + c] = (float)(a2 * a1 + P->csum[0] * a2 * l1 + P->csum[1] * l2 * a1);
                lam[2 * (size_t)n3 + (size_t)n1 * n2 + c] = (float)(a2 * a1);
            }
        MX_TRY(cudaMalloc((void**)&M->lam, lam.size() * sizeof(float)));
        MX_TRY(cudaMemcpyAsync(M->lam, lam.data(), lam.size() * sizeof(float), cudaMemcpyHostToDevice, s));
        MX_TRY(cudaStreamSynchronize(s));   // the host array goes out of scope
    }
    // per-line factors of the operator in the sine-transform eigenbasis:
    // S_N A S_N = D3 D2 (D1 + Bh1) + D3 Bh2 D1 + Bh3 D2 D1 (Kronecker
    // products, D_a = diag of the mass eigenvalues, Bh_a = S (eta_a B_a) S),
    // so each axis term is the contraction along its axis scaled by the mass
    // eigenvalues of the other two axes, and D3 D2 D1 is the z term's mass part
    {
        const int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2];
        const std::vector<double>&m1 = P->lam_mass[0], &m2 = P->lam_mass[1], &m3 = P->lam_mass[2];
        std::vector<float> f;
        f.reserve((size_t)n2 * n3 + (size_t)n1 * n3 + (size_t)n1 * n2 + n3);
        for (int k = 0; k < n3; ++k)
            for (int j = 0; j < n2; ++j) f.push_back((float)(m2[j] * m3[k]));   // x lines j + n2 k
        for (int k = 0; k < n3; ++k)
            for (int i = 0; i < n1; ++i) f.push_back((float)(m1[i] * m3[k]));   // y lines i + n1 k
        for (int j = 0; j < n2; ++j)
            for (int i = 0; i < n1; ++i) f.push_back((float)(m1[i] * m2[j]));   // z lines i + n1 j
        for (int k = 0; k < n3; ++k) f.push_back((float)m3[k]);
        MX_TRY(cudaMalloc((void**)&M->spec, f.size() * sizeof(float)));
        MX_TRY(cudaMemcpyAsync(M->spec, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice, s));
        MX_TRY(cudaStreamSynchronize(s));
        M->spectral_ok = true;
        M->spectral = true;
    }
    MX_TRY(cudaMalloc((void**)&M->dsc, 32 * sizeof(double)));
    MX_TRY(cudaMemsetAsync(M->dsc, 0, 32 * sizeof(double), s));
    MX_TRY(cudaMalloc((void**)&M->err, sizeof(int)));
    MX_TRY(cudaMemsetAsync(M->err, 0, sizeof(int), s));
    MX_TRY(cudaMallocHost((void**)&M->err_host, sizeof(int)));
    // the solvers' workspaces up front, so that no solve allocates: the PCG
    // direction ring and loop control, the grouped operator descriptors, the
    // GMRES basis of the default restart (20; a longer restart grows it) and
    // the device-side cycle's state
    MX_TRY(cudaMalloc((void**)&M->pring, (size_t)kPRing * N * sizeof(float)));
    MX_TRY(cudaMalloc((void**)&M->pcg_ctl, 4 * sizeof(int)));
    MX_TRY(cudaMallocHost((void**)&M->pcg_ctl_host, 4 * sizeof(int)));
    MX_TRY(cudaMalloc((void**)&M->gm_state, GS_WORDS * sizeof(double)));
    MX_TRY(cudaMalloc((void**)&M->gm_ctl, 4 * sizeof(int)));
    MX_TRY(cudaMallocHost((void**)&M->gm_ctl_host, 4 * sizeof(int)));
    if (int st = ensure_pairs(P, s)) return st;
    if (int st = ensure_v32(P, 20)) return st;
    MX_TRY(cudaStreamSynchronize(s));
    return TFDE_OK;
}

void mixed_free(tfde_problem* P) {
    MixedState* M = mixed(P);
    if (!M) return;
    for (int om = 0; om < NOM; ++om)
        if (M->own_mat[om]) cudaFree(M->mat[om]);
    for (int pl = 0; pl < NPL; ++pl) cudaFree(M->hi[pl]);   // lo lives in the same allocation
    for (auto& v : M->f) cudaFree(v);
    cudaFree(M->V32);
    cudaFree(M->pring);
    if (M->pcg_exec) cudaGraphExecDestroy(M->pcg_exec);
    if (M->gm_exec) cudaGraphExecDestroy(M->gm_exec);
    if (M->gm_graph) cudaGraphDestroy(M->gm_graph);
    cudaFree(M->gm_state);
    cudaFree(M->gm_ctl);
    if (M->gm_ctl_host) cudaFreeHost(M->gm_ctl_host);
    if (M->pcg_graph) cudaGraphDestroy(M->pcg_graph);
    if (M->spec_exec) cudaGraphExecDestroy(M->spec_exec);
    if (M->spec_graph) cudaGraphDestroy(M->spec_graph);
    if (M->gms_exec) cudaGraphExecDestroy(M->gms_exec);
    if (M->gms_graph) cudaGraphDestroy(M->gms_graph);
    cudaFree(M->pcg_ctl);
    if (M->pcg_ctl_host) cudaFreeHost(M->pcg_ctl_host);
    cudaFree(M->pair_d);
    cudaFree(M->pair_gstart);
    cudaFree(M->gm);
    if (M->gm_host) cudaFreeHost(M->gm_host);
    oz_free(M);
    cudaFree(M->lam);
    cudaFree(M->spec);
    cudaFree(M->dsc);
    cudaFree(M->err);
    if (M->err_host) cudaFreeHost(M->err_host);
    delete M;
    P->mixed = nullptr;
}

int mixed_apply_A(const tfde_problem* P, int op, const double* x, double* y, cudaStream_t s) {
    if (!(op & TFDE_OP_FAST)) return accurate_apply(P, op, x, y, s);
    MixedState* M = mixed(P);
    launch_split64(P->N, x, 1.0, M->hi[PL_P], M->lo[PL_P], s);
    int st = fast_matvec(P, op, M->f[F_Q], s);
    if (st) return st;
    launch_widen32(P->N, M->f[F_Q], 1.0, y, s);
    return TFDE_OK;
}

int mixed_apply_Pinv(const tfde_problem* P, const double* r, double* z, cudaStream_t s) {
    MixedState* M = mixed(P);
    launch_split64(P->N, r, 1.0, M->hi[PL_R], M->lo[PL_R], s);
    int st = fast_precond(P, M->f[F_Z], s);
    if (st) return st;
    launch_widen32(P->N, M->f[F_Z], 1.0, z, s);
    return TFDE_OK;
}

// Measured reduction of the true FP64 residual by one inner split-BF16 solve
// when the inner solve itself goes further (the split operator's accuracy).
constexpr double kInnerFloor = 1e-4;

// b - A x at full width, with A_N x into W_T for the next chained CN step.
int exact_residual(tfde_problem* P, const double* b, const double* x, double* r64, double* nr, double tol, double nb,
                   cudaStream_t s) {
    io_offer_output(P, x, s);   // x may be final: a host copy may leave while its residual is formed
    const int st = accurate_residual(P, b, x, r64, nr, tol, nb, s, P->w[tfde_problem::W_T]);
    P->an_ready = st == TFDE_OK;
    return st;
}

// x += c, c = dsc d (d: the inner solution in F_X for the residual scaled by
// 1/dsc), and the new residual with its norm into r64 / *nr.  A sweep that
// cannot end the solve (predicted true reduction `pred`) updates the
// residual by its correction, r <- r - A c, instead of recomputing b - A x:
// the product is exact-integer at few digits, because c is small (about
// ||r|| / ||A|| against ||x||), so 4 or 5 slices give it far below the next
// sweep's target.  A sweep predicted to end the solve recomputes the true
// residual b - A x at full width, and so does any sweep whose updated
// residual meets the tolerance: the residual that stops the solve, and that
// the next CN step chains on, is always the recomputed one.
int apply_correction(tfde_problem* P, const double* b, double* x, double* r64, double* nr, double pred, double tol,
                     double nb, double dsc, cudaStream_t s, const PcgPending* pend = nullptr) {
    MixedState* M = mixed(P);
    int st;
    double* an = P->w[tfde_problem::W_T];
    io_before_write(P, x, s);
    if (*nr * pred > tol * nb) {
        double* c64 = an;
        P->an_ready = false;
        if (pend) launch_pcg_combine(P->N, *pend, M->f[F_X], dsc, c64, x, nullptr, s);   // c = dsc d, x += c
        else launch_widen_add32(P->N, dsc, M->f[F_X], c64, x, s);
        const int shift = -std::ilogb(nb);
        double* acc = P->red_out + kNormsSlot + 2;
        const int sc = *nr <= 1e-2 * nb ? 4 : (*nr <= nb ? 5 : oz_slices_for_tol(tol));
        if ((st = accurate_apply_ex(P, TFDE_OP_A, c64, r64, -1, r64, 1.0, s, sc, acc, shift))) return st;
        MX_TRY(cudaMemcpyAsync(P->red_host, acc, sizeof(double), cudaMemcpyDeviceToHost, s));
        MX_TRY(cudaStreamSynchronize(s));
        *nr = std::ldexp(std::sqrt(P->red_host[0]), -shift);
        if (*nr <= tol * nb) return exact_residual(P, b, x, r64, nr, tol, nb, s);
        return TFDE_OK;
    }
    if (pend) launch_pcg_combine(P->N, *pend, M->f[F_X], dsc, nullptr, x, nullptr, s);   // x += dsc d
    else launch_add32to64(P->N, dsc, M->f[F_X], x, s);
    return exact_residual(P, b, x, r64, nr, tol, nb, s);
}

// FP64 iterative refinement around the FP32 / split-BF16 inner PCG.
int mixed_pcg(tfde_problem* P, const double* b, double* x, double tol, int maxit, tfde_info* info,
              cudaStream_t s, bool r_given) {
    const auto t0 = clk::now();
    MixedState* M = mixed(P);
    tfde_info loc{};
    double* r64 = P->w[tfde_problem::W_R];
    int st;
    double bb, rr0 = 0.0;
    if ((st = initial_norms(const_cast<tfde_problem*>(P), b, r64, r_given, &bb, &rr0, s))) return st;
    const double nb = std::sqrt(bb);
    if (!std::isfinite(nb)) return set_error(TFDE_ENAN, "non-finite right-hand side");
    if (nb == 0.0) {
        io_before_write(P, x, s);
        MX_TRY(cudaMemsetAsync(x, 0, P->N * sizeof(double), s));
        if (info) *info = loc;
        return TFDE_OK;
    }
    double nr;
    if (r_given) {
        nr = std::sqrt(rr0);
    } else if ((st = exact_residual(P, b, x, r64, &nr, tol, nb, s))) {
        return st;
    }
    loc.relres0 = nr / nb;
    int status = TFDE_ENOCONV;
    int stall = 0;
    while (true) {
        if (!std::isfinite(nr)) { status = set_error(TFDE_ENAN, "non-finite residual"); break; }
        if (nr <= tol * nb) { status = TFDE_OK; break; }
        if (loc.iters >= maxit) break;
        // inner solve of A d = r / ||r|| to a relative theta.  One sweep lowers
        // the true residual by at most ~kInnerFloor (the split operator's
        // accuracy); when the target needs more, two sweeps share it evenly
        // (theta = sqrt of the target, floored) instead of the first one
        // spending iterations below what it can deliver.  The inner target is
        // 0.8 of what the sweep must reach: the split operator's error adds
        // ~1e-4 of ||r|| on top (measured at the n = 256 workload with the
        // eigenbasis inner PCG: final residuals <= 0.76 tol in one sweep, 3.1
        // inner iterations per step against 3.2 with 0.7 and 3.3 with 0.6;
        // 0.9 gives the same counts as 0.8).
        double theta = 0.8 * tol * nb / nr;
        if (theta < kInnerFloor) theta = std::max(kInnerFloor, std::sqrt(theta));
        // r32 = r 2^k with 2^k the power of two nearest below 1 / ||r|| (an
        // exact scale: the conversion and, later, the scale back of the
        // correction need no FP64 arithmetic), so ||r32|| lies in [1/2, 1)
        // up to the FP32 rounding of its elements; the inner PCG reads no lo plane
        const int k = -std::ilogb(nr) - 1;
        const double un = std::ldexp(nr, k);
        int it = 0;
        double reached = 1.0;
        PcgPending pend;
        const bool spec = M->spectral;
        if (spec) {
            // the eigenbasis solve reads the split planes of r and returns S_N d~ in F_X
            launch_split64(P->N, r64, std::ldexp(1.0, k), M->hi[PL_R], M->lo[PL_R], s);
            if ((st = inner_pcg_spec(P, theta, maxit - loc.iters, &it, &pend, s, &reached, un * un))) return st;
            if ((st = spec_finish(P, pend, s))) return st;
        } else {
            launch_scale64to32_hi(P->N, r64, std::ldexp(1.0, k), M->f[F_R], M->hi[PL_R], s);
            if ((st = inner_pcg(P, theta, maxit - loc.iters, &it, &pend, s, &reached, un * un))) return st;
        }
        loc.iters += it;
        loc.refine_sweeps++;
        const double nr_old = nr;
        PcgPending whole;   // eigenbasis: the transformed correction is F_X itself
        whole.fold = true;
        if ((st = apply_correction(P, b, x, r64, &nr, std::max(reached, kInnerFloor), tol, nb, std::ldexp(1.0, -k), s,
                                   spec ? &whole : &pend)))
            return st;
        stall = (nr > 0.5 * nr_old) ? stall + 1 : 0;
        if (stall >= 2) {
            // refinement stopped contracting: finish with FP64 inner solves
            loc.fallback = 1;
            P->an_ready = false;
            tfde_info sub{};
            io_before_write(P, x, s);
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

// FP64 iterative refinement around one FP32 / split-BF16 left-preconditioned
// GMRES cycle per sweep: every sweep restarts from the accurate FP64 residual,
// so the outer loop is restarted GMRES(restart) whose restarts are exact.
int mixed_pgmres(tfde_problem* P, const double* b, double* x, int restart, double tol, int maxit, tfde_info* info,
                 cudaStream_t s, bool r_given) {
    const auto t0 = clk::now();
    MixedState* M = mixed(P);
    tfde_info loc{};
    double* r64 = P->w[tfde_problem::W_R];
    int st;
    if ((st = ensure_v32(P, restart))) return st;
    double bb, rr0 = 0.0;
    if ((st = initial_norms(const_cast<tfde_problem*>(P), b, r64, r_given, &bb, &rr0, s))) return st;
    const double nb = std::sqrt(bb);
    if (!std::isfinite(nb)) return set_error(TFDE_ENAN, "non-finite right-hand side");
    if (nb == 0.0) {
        io_before_write(P, x, s);
        MX_TRY(cudaMemsetAsync(x, 0, P->N * sizeof(double), s));
        if (info) *info = loc;
        return TFDE_OK;
    }
    double nr;
    if (r_given) {
        nr = std::sqrt(rr0);
    } else if ((st = exact_residual(P, b, x, r64, &nr, tol, nb, s))) {
        return st;
    }
    loc.relres0 = nr / nb;
    int status = TFDE_ENOCONV;
    int stall = 0;
    double ratio = 1.0;  // observed (true reduction) / (preconditioned estimate's reduction)
    while (true) {
        if (!std::isfinite(nr)) { status = set_error(TFDE_ENAN, "non-finite residual"); break; }
        if (nr <= tol * nb) { status = TFDE_OK; break; }
        if (loc.iters >= maxit) break;
        double theta = 0.5 * tol * nb / nr / ratio;
        if (theta < kInnerFloor) theta = std::max(kInnerFloor, std::sqrt(theta));   // as in mixed_pcg
        launch_scale64to32(P->N, r64, 1.0 / nr, M->f[F_R], M->hi[PL_R], M->lo[PL_R], M->f[F_X], s);
        int it = 0;
        double est_ratio = 1.0;
        if (M->spectral) {
            if ((st = inner_gmres_spec(P, restart, theta, maxit - loc.iters, &it, &est_ratio, s))) return st;
        } else if ((st = inner_gmres(P, restart, theta, maxit - loc.iters, &it, &est_ratio, s))) {
            return st;
        }
        loc.iters += it;
        loc.restarts++;
        loc.refine_sweeps++;
        const double nr_old = nr;
        const double pred = est_ratio > 0.0 ? std::max(est_ratio * ratio, kInnerFloor) : 1.0;
        if ((st = apply_correction(P, b, x, r64, &nr, pred, tol, nb, nr, s))) return st;
        if (est_ratio > 0.0) {
            const double observed = (nr / nr_old) / est_ratio;
            ratio = observed > 1.0 ? observed : 1.0;
        }
        stall = (nr > 0.5 * nr_old) ? stall + 1 : 0;
        if (stall >= 2) {
            // refinement stopped contracting: finish with FP64 inner cycles
            loc.fallback = 1;
            P->an_ready = false;
            tfde_info sub{};
            io_before_write(P, x, s);
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

// The autotuner on this problem's launch classes: one operator application
// (the two grouped pairs and the z pass) and one preconditioner application
// with the direction update are recorded, then every class is timed over its
// candidate launch parameters and the fastest kept (tfde_tune).  The trials
// overwrite the inner solver's scratch vectors only: call between solves.
int mixed_tune(tfde_problem* P, int reps, cudaStream_t s) {
    MixedState* M = mixed(P);
    if (!M) return set_error(TFDE_EUNSUPPORTED, "only the tensor-core mixed path has tunable launches");
    if (reps < 1 || reps > 1000) return set_error(TFDE_EINVAL, "reps must lie in [1, 1000]");
    double* d = M->dsc;
    const size_t N = P->N;
    tc::tune_record(true);
    int st = fast_matvec(P, TFDE_OP_A, M->f[F_Q], s, -1, M->pring, d + D_PQ);
    if (!st) st = fast_precond_cg(P, M->pring + N, M->pring, d + D_RZ0, nullptr, nullptr, s);
    if (!st && M->spectral_ok) {   // the eigenbasis passes and the sine transform
        st = spec_matvec(P, M->pring, M->f[F_Q], d + D_PQ, s);
        if (!st) st = spec_transform(P, PL_R, PL_T1, PL_T2, M->f[F_R], s);
    }
    tc::tune_record(false);
    if (!st) st = tc::tune_recorded(reps, s);
    if (!st) st = check_err(P, s);
    return st;
}

int mixed_set_spectral(tfde_problem* P, int enable) {
    MixedState* M = mixed(P);
    if (!M || !M->spectral_ok) {
        if (enable) return set_error(TFDE_EUNSUPPORTED, "the eigenbasis inner solves need a TFDE_MIXED problem on the tensor-core path");
        return TFDE_OK;
    }
    M->spectral = enable != 0;
    return TFDE_OK;
}

long long mixed_graph_launches(const tfde_problem* P) {
    const MixedState* M = mixed(P);
    return M ? M->graph_launches : 0;
}

int mixed_set_device_loop(tfde_problem* P, int enable) {
    MixedState* M = mixed(P);
    if (M) M->device_loop = enable != 0;
    return TFDE_OK;
}

}  // namespace tfde
