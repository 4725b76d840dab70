// Mixed-precision state and FP32 / split-BF16 vector kernel launchers.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include <vector>

#include "tfde_internal.h"
#include "tfde_tc.h"

namespace tfde {

constexpr int kPRing = 3;          // inner PCG directions kept before folding into F_X
constexpr int kAlphaSlot = 8;      // device scalars: alpha of direction j at kAlphaSlot + j % kPRing
// Deferred inner solution: d = (fold ? F_X : 0) + sum_{j < cnt} alpha_j p_j.
struct PcgPending {
    int cnt = 0;
    bool fold = false;
    const float* p[kPRing] = {};
    const double* alpha[kPRing] = {};
};

void launch_dot32(size_t N, const float* a, const float* b, double* part, int nblk, cudaStream_t s);
// alpha = *num / *den on the device; x += alpha p; r -= alpha q; split r; *rr += r.r
void launch_cg_update32(size_t N, const double* num, const double* den, const float* p, const float* q, float* x,
                        float* r, __nv_bfloat16* rh, __nv_bfloat16* rl, double* rr, cudaStream_t s);
// r32 = r64 sc; rh = bf16(r32)
void launch_scale64to32_hi(size_t N, const double* r64, double sc, float* r32, __nv_bfloat16* rh, cudaStream_t s);
// alpha = *num / *den on the device (also stored to *alpha_out by one thread);
// r -= alpha q; split r (rl null: the hi plane alone); *rr += r.r  (the
// solution is left to the combination)
void launch_cg_update_r32(size_t N, const double* num, const double* den, const float* q, float* r,
                          __nv_bfloat16* rh, __nv_bfloat16* rl, double* rr, double* alpha_out, cudaStream_t s,
                          const int* skip = nullptr);
// d = (fold ? x32 : 0) + sum_j alpha_j p_j ; with c64: c64 = sc d, x64 += c64 ;
// without: x64 += sc d ; with acc32 (and no x64): acc32 = d (the fold itself)
void launch_pcg_combine(size_t N, const PcgPending& pend, const float* x32, double sc, double* c64, double* x64,
                        float* acc32, cudaStream_t s);
// The inner PCG in the sine-transform eigenbasis, where the tau preconditioner
// is the diagonal Lambda (lam: the [ra | rb | U | V] factors of MixedState).
// Update: alpha = *num / *den (also to *alpha_out); r -= alpha q;
// *rz += <r, r / Lambda>; *rr += <r, r>.
int launch_spec_update(const float* lam, const int n[3], const double* num, const double* den, const float* q,
                       float* r, double* rz, double* rr, double* alpha_out, cudaStream_t s, const int* skip = nullptr);
// Direction: beta = *num / *den (0 when den is null); p = r / Lambda + beta
// pold (pold may be null), in FP32 and as split planes; with rz:
// *rz += <r, r / Lambda>.
int launch_spec_direction(const float* lam, const int n[3], const double* num, const double* den, const float* r,
                          const float* pold, float* p, __nv_bfloat16* ph, __nv_bfloat16* pl, double* rz,
                          cudaStream_t s, const int* skip = nullptr);
// d = (fold ? x32 : 0) + sum_j alpha_j p_j written as split planes (h, l) only
int launch_pcg_combine_split(size_t N, const PcgPending& pend, const float* x32, __nv_bfloat16* h, __nv_bfloat16* l,
                             cudaStream_t s);
// device-side inner PCG loop (see pcg_cond_kernel): iteration head, stop
// test and loop condition, initial control words, fold of a full window
void launch_pcg_head(double* d, int rz, int rzn, int pq, int rr, const int* ctl, cudaStream_t s);
void launch_pcg_cond(cudaGraphConditionalHandle h, const double* rr, const double* thr, int* ctl, cudaStream_t s);
void launch_pcg_init(double* d, int rzn, int thr_slot, double thr, int* ctl, int maxit, cudaStream_t s);
void launch_pcg_fold_dev(size_t N, const float* const* p, const double* const* alpha, float* x32, const int* ctl,
                         cudaStream_t s);
// device-side GMRES cycle: least-squares state layout (FP64 words), for at
// most GS_MAXM Arnoldi steps per cycle
constexpr int GS_MAXM = 64;
constexpr int GS_LD = GS_MAXM + 2;   // leading dimension of a Hessenberg column
enum { GS_BETA = 0, GS_EST = 1, GS_INV = 2, GS_THR = 3, GS_G = 8, GS_CS = GS_G + GS_MAXM + 1,
       GS_SN = GS_CS + GS_MAXM, GS_R = GS_SN + GS_MAXM, GS_WORDS = GS_R + GS_LD * GS_MAXM };
// one Arnoldi step on w (the preconditioner's output): CGS2 against V_0..V_j,
// ||w||, the Givens update and stop test (loop condition hc), V_{j+1} = w/||w||
// with its split planes; every count and address from the control words
void launch_gm_step(size_t N, const float* V, float* w, double* part, int nblk, double* hbuf, double* h2buf,
                    double* wwbuf, double* gs, int* gctl, cudaGraphConditionalHandle hc, float* Vout,
                    __nv_bfloat16* ph, __nv_bfloat16* pl, int maxm, cudaStream_t s);
// cycle start on w = P^{-1} r: beta, g = beta e_1, V_0 = w / beta and its planes
void launch_gm_start(size_t N, const float* w, double* part, int nblk, double* wwbuf, double* gs, int* gctl,
                     int maxsteps, double ptheta, float* V0, __nv_bfloat16* ph, __nv_bfloat16* pl, cudaStream_t s);
// ny = -y of the cycle's least-squares problem (zero beyond the steps done)
void launch_gm_solve(const double* gs, const int* gctl, double* ny, int maxm, cudaStream_t s);
// c64 = sc * d32; x64 += c64
void launch_widen_add32(size_t N, double sc, const float* d, double* c, double* x, cudaStream_t s);
// beta = *num / *den on the device; p = z + beta p; split p
void launch_xpay32(size_t N, const double* num, const double* den, const float* z, float* p, __nv_bfloat16* ph,
                   __nv_bfloat16* pl, cudaStream_t s);
void launch_scale64to32(size_t N, const double* r64, double sc, float* r32, __nv_bfloat16* rh, __nv_bfloat16* rl,
                        float* x32, cudaStream_t s);
void launch_split32(size_t N, const float* v, __nv_bfloat16* h, __nv_bfloat16* l, cudaStream_t s);
void launch_split64(size_t N, const double* v, double sc, __nv_bfloat16* h, __nv_bfloat16* l, cudaStream_t s);
void launch_add32to64(size_t N, double sc, const float* d, double* x, cudaStream_t s);
void launch_widen32(size_t N, const float* v, double sc, double* y, cudaStream_t s);
void launch_ratio(const double* num, const double* den, double* coef, cudaStream_t s);
// m dot products <V_j, w> (FP32 vectors), partials part[j*nblk + b]
void launch_multidot32(size_t N, int m, const float* V, size_t ldv, const float* w, double* part, int nblk,
                       cudaStream_t s);
// w -= sum_j h[j] V_j  (h: FP64 on the device, m <= 128)
void launch_multiaxpy32(size_t N, int m, const float* V, size_t ldv, const double* h, float* w, cudaStream_t s);
// out = sc * in ; (h, l) = split(out)
void launch_scale_split32(size_t N, float sc, const float* in, float* out, __nv_bfloat16* h, __nv_bfloat16* l,
                          cudaStream_t s);

// Split-BF16 plane pairs of the workspace.
enum Plane { PL_P, PL_A, PL_W, PL_C, PL_E, PL_R, PL_T1, PL_T2, NPL };
// FP32 vectors of the inner solver.
enum Vec32 { F_X, F_R, F_Z, F_P, F_Q, NF };
// BF16 operator matrices (n_a x n_a, row-major [out][in]).
enum OpMat {
    OM_GHAT_H, OM_GHAT_L,        // x axis: M1 + eta1 B1
    OM_GHATR_H, OM_GHATR_L,      // x axis: M1 - eta1 B1 (RHS operator)
    OM_GY_H, OM_GY_L, OM_GYN_H, OM_GYN_L,   // +- eta2 B2
    OM_GZ_H, OM_GZ_L, OM_GZN_H, OM_GZN_L,   // +- eta3 B3
    OM_MX, OM_MY, OM_MZ,         // mass A_n (exact in BF16)
    OM_SX, OM_SY, OM_SZ,         // DST-I S_n (rounded once to BF16)
    // the inner PCG in the sine-transform eigenbasis (symmetric problems):
    OM_BX_H, OM_BX_L, OM_BY_H, OM_BY_L, OM_BZ_H, OM_BZ_L,        // S_n (eta_a B_a) S_n, split
    OM_S2X_H, OM_S2X_L, OM_S2Y_H, OM_S2Y_L, OM_S2Z_H, OM_S2Z_L,  // S_n split into hi + lo
    NOM
};
constexpr int NOM_BASE = OM_SZ + 1;   // the matrices every TFDE_MIXED problem carries

// Digit slices of the exact-integer (Ozaki-type) contraction: 7 base-128
// digits, 49 bits below each row / line maximum.
constexpr int OZ_SLICES = 7;

// One operator's digit slices (device) with their tensor maps.
struct OzSet {
    __nv_bfloat16* dev = nullptr;
    CUtensorMap amap[OZ_SLICES];
    CUtensorMap amapk[OZ_SLICES];   // leading k + 1 slices in one box {32, 128, k + 1}
    bool amapk_ok[OZ_SLICES] = {};
    int na = 0;          // leading slices that are not all zero
    int rexp_index = 0;  // row exponents in MixedState::oz_rexp
};

struct MixedState {
    __nv_bfloat16* mat[NOM] = {};   // hi/lo pairs share one allocation (lo = hi + n^2)
    bool own_mat[NOM] = {};
    CUtensorMap amap[NOM];
    CUtensorMap amap2[NOM];          // for the hi of a pair: one 3-D box {64, 128, 2} loads hi and lo
    bool has_amap2[NOM] = {};
    __nv_bfloat16* hi[NPL] = {};   // one allocation per plane pair: lo = hi + N
    __nv_bfloat16* lo[NPL] = {};
    CUtensorMap bmap_hi[NPL][3];
    CUtensorMap bmap_lo[NPL][3];
    CUtensorMap bmap2[NPL][3];     // both planes (and on y/z all four 64-line blocks) in one box
    int bmap2_rank[NPL][3] = {};   // 3 (x), 5 (y/z), 0 = not available
    CUtensorMap bmap1[NPL][3];     // the hi plane alone, same box otherwise
    int bmap1_rank[NPL][3] = {};
    CUtensorMap omap_hi[NPL][3];   // the planes as outputs of the epilogue's tensor stores
    CUtensorMap omap_hl[NPL][3];   // hi and lo as one tensor (lo = hi + N): one store per chunk
    float* f[NF] = {};
    float* lam = nullptr;   // [ra (n3) | rb (n3) | U (n1 n2) | V (n1 n2)]
    // inner solves in the sine-transform eigenbasis: per-line factors of the three axis terms and the z-axis
    // mass eigenvalues, [cs_x (n2 n3) | cs_y (n1 n3) | cs_z (n1 n2) | mu3 (n3)]
    float* spec = nullptr;
    bool spectral_ok = false;    // the matrices and factors exist
    bool spectral = false;       // tfde_set_spectral_inner (default on when available)
    long long spec_transforms = 0;   // sine transforms run (statistics)
    cudaGraph_t gms_graph = nullptr;     // the eigenbasis GMRES cycle's Arnoldi steps as one graph launch
    cudaGraphExec_t gms_exec = nullptr;
    bool gms_graph_failed = false;
    int gms_graph_restart = 0;
    unsigned gms_tune_gen = 0;
    cudaGraph_t spec_graph = nullptr;    // the eigenbasis inner PCG as one graph launch per sweep
    cudaGraphExec_t spec_exec = nullptr;
    bool spec_graph_failed = false;
    unsigned spec_tune_gen = 0;
    double* dsc = nullptr;  // device scalars
    int* err = nullptr;     // device error flag of the tensor-core kernels
    int* err_host = nullptr;
    long long gemm_launches = 0;
    // inner FP32 GMRES: basis (cap + 1 vectors) and device / pinned host
    // Hessenberg scratch [h (128) | h2 (128) | |w|^2 | ... | -y (128)]
    float* V32 = nullptr;
    int v32_cap = 0;
    // inner PCG: the search directions of the current window (the solution is
    // combined from them once per sweep, see inner_pcg)
    float* pring = nullptr;   // kPRing vectors
    // the inner PCG as one graph launch per sweep: a device-side while loop
    // whose body runs kPRing iterations (ctl: iterations, done, maxit)
    int* pcg_ctl = nullptr;
    int* pcg_ctl_host = nullptr;
    cudaGraph_t pcg_graph = nullptr;
    cudaGraphExec_t pcg_exec = nullptr;
    bool pcg_graph_failed = false;
    unsigned pcg_tune_gen = 0;      // autotuner table generation the graphs were captured with
    unsigned gm_tune_gen = 0;
    bool device_loop = true;   // tfde_set_device_loop
    long long graph_launches = 0;   // inner solves run as one graph launch (tfde_device_loop_launches)
    // the inner GMRES cycle's Arnoldi steps as one graph launch (while node)
    double* gm_state = nullptr;   // GS_WORDS
    int* gm_ctl = nullptr;        // 4 control words
    int* gm_ctl_host = nullptr;
    cudaGraph_t gm_graph = nullptr;
    cudaGraphExec_t gm_exec = nullptr;
    int gm_graph_restart = 0;
    bool gm_graph_failed = false;
    // the operator's first four split passes as two grouped launches (device
    // descriptors, tile offsets, totals and algorithmic work per launch)
    tc::Params* pair_d = nullptr;
    long long* pair_gstart = nullptr;   // [2][3]
    long long pair_total[2] = {};
    double pair_bytes[2] = {}, pair_flops[2] = {};
    double* gm = nullptr;
    double* gm_host = nullptr;
    // exact-integer slice path (tfde_oz.cu)
    OzSet oz_x_plus, oz_x_minus, oz_x_stiff;                 // A1 + G1, A1 - G1, G1
    OzSet oz_y_mass_c, oz_y_plus, oz_y_minus;                // (A2 | +-G2) common rows
    OzSet oz_z_mass_c, oz_z_plus, oz_z_minus;                // (A3 | +-G3) common rows
    std::vector<int*> oz_rexp;                               // row exponent arrays
    __nv_bfloat16* oz_planes[2] = {nullptr, nullptr};        // digit planes of two inputs
    CUtensorMap oz_bmap[2][OZ_SLICES][3];
    CUtensorMap oz_bmapm[2][3][OZ_SLICES];                   // leading k + 1 slices of an input in one box
    bool oz_bmapm_ok[2][3][OZ_SLICES] = {};
    int* oz_lexp = nullptr;                                  // joint line exponents
    int oz_shift[3] = {0, 0, 0};                             // exponent shift of the second input
};

inline MixedState* mixed(const tfde_problem* P) { return static_cast<MixedState*>(P->mixed); }

// Descriptors of the split-BF16 passes of one problem, for grouped launches:
// kind 0 = operator A on plane PL_P with the result split into PL_R (5 passes),
// kind 1 = preconditioner on PL_R with FP32 output out_f32 (6 passes).
// Returns the pass count; axes[i], bytes[i], flops[i] per pass.
int fast_pass_descriptors(const tfde_problem* P, int kind, float* out_f32, tc::Params* prm, int* axes, double* bytes,
                          double* flops);
// Descriptors of the eigenbasis passes of one problem (left-preconditioned
// GMRES, Sec. 3.2): kind 2 = forward sine transform of the residual planes
// PL_R with Lambda^{-1} fused, out_f32 = Lambda^{-1} S_N r; kind 3 = the
// preconditioned operator on the basis planes PL_P, out_f32 = Lambda^{-1}
// S_N A S_N v (x and y passes chained through F_Z, F_P); kind 4 = backward
// sine transform of the planes PL_T1, out_f32 = S_N t (through PL_T2, PL_R);
// kind 5 = forward sine transform of PL_R without Lambda, out_f32 = S_N r
// (PCG, Sec. 3.1).  With dot_out set, kind 3's z pass leaves out Lambda^{-1}
// (out_f32 = S_N A S_N v, the PCG operator) and adds <dot_vec, out_f32> into
// *dot_out.  Returns 3 (passes); axes[i], bytes[i], flops[i] per pass.
int spec_pass_descriptors(const tfde_problem* P, int kind, float* out_f32, tc::Params* prm, int* axes, double* bytes,
                          double* flops, const float* dot_vec = nullptr, double* dot_out = nullptr);
// Allocate the FP32 GMRES basis (restart + 1 vectors) and Hessenberg scratch.
int mixed_prepare_gmres(const tfde_problem* P, int restart);

int oz_init(tfde_problem* P, const std::vector<double> etaB[3], cudaStream_t s);
void oz_free(MixedState* M);
int accurate_apply(const tfde_problem* P, int op, const double* x, double* y, cudaStream_t s);
// y = vsign * (operator x) + asign * addend (addend may be null)
// norm2 (optional, device): receives sum_i (y_i 2^norm_shift)^2 accumulated
// in FP32 terms by the last pass (24-bit terms: enough for stopping tests).
// an_out (optional, op = A only): receives A_N x = A3 A2 A1 x, formed exactly
// from the fixed-point digits in the z-pass slicing (error ~2^{-7 slices} of
// the line maxima), at the cost of one extra FP64 write.
int accurate_apply_ex(const tfde_problem* P, int op, const double* x, double* y, int vsign, const double* addend,
                      double asign, cudaStream_t s, int slices = OZ_SLICES, double* norm2 = nullptr,
                      int norm_shift = 0, double* an_out = nullptr);
// Exact residuals of the problems of a batch as grouped launches (tfde_oz.cu).
struct OzBatch;
// norm2[i]: the device double that receives ||r_i||^2 (FP32 terms under the
// call's scale) of problem i.
int oz_batch_create(tfde_problem* const* P, int count, double* const* norm2, OzBatch** out);
void oz_batch_destroy(OzBatch* ob);
// For every problem i with act[i] != 0 (host copy act, device copy d_act):
// r_i = b_i - A_i x_i into W_R, FP64-accurate at S digit slices, with
// sum (r_i 2^shift[i])^2 (FP32 terms) into *norm2[i] and A_N x_i into W_T
// (the next chained step's mass term): three grouped slicing and three
// grouped exact-contraction launches over all problems' lines and tiles.
int oz_batch_residual(OzBatch* ob, const double* const* x, const int* act, const int* d_act, const int* shift, int S,
                      cudaStream_t s);

// Digit slices for a refinement residual at relative tolerance tol: 6 (42
// bits, a worst-case error n 2^-42 < 1.1e-10 of |A||x| for n <= 448) while
// tol >= 1e-9, else 7.
inline int oz_slices_for_tol(double tol) { return tol >= 1e-9 ? 6 : OZ_SLICES; }

}  // namespace tfde
