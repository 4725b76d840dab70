// Mixed-precision state and FP32 / split-BF16 vector kernel launchers.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include <vector>

#include "tfde_internal.h"
#include "tfde_tc.h"

namespace tfde {

void launch_dot32(size_t N, const float* a, const float* b, double* part, int nblk, cudaStream_t s);
void launch_cg_update32(size_t N, const double* coef, const float* p, const float* q, float* x, float* r,
                        __nv_bfloat16* rh, __nv_bfloat16* rl, double* part, int nblk, cudaStream_t s);
void launch_xpay32(size_t N, const double* coef, const float* z, float* p, __nv_bfloat16* ph, __nv_bfloat16* pl,
                   cudaStream_t s);
void launch_scale64to32(size_t N, const double* r64, double sc, float* r32, __nv_bfloat16* rh, __nv_bfloat16* rl,
                        float* x32, cudaStream_t s);
void launch_split32(size_t N, const float* v, __nv_bfloat16* h, __nv_bfloat16* l, cudaStream_t s);
void launch_split64(size_t N, const double* v, double sc, __nv_bfloat16* h, __nv_bfloat16* l, cudaStream_t s);
void launch_add32to64(size_t N, double sc, const float* d, double* x, cudaStream_t s);
void launch_widen32(size_t N, const float* v, double sc, double* y, cudaStream_t s);
void launch_ratio(const double* num, const double* den, double* coef, cudaStream_t s);

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
    NOM
};

// Digit slices of the exact-integer (Ozaki-type) contraction: 7 base-128
// digits, 49 bits below each row / line maximum.
constexpr int OZ_SLICES = 7;

struct MixedState {
    __nv_bfloat16* mat[NOM] = {};
    CUtensorMap amap[NOM];
    __nv_bfloat16* hi[NPL] = {};
    __nv_bfloat16* lo[NPL] = {};
    CUtensorMap bmap_hi[NPL][3];
    CUtensorMap bmap_lo[NPL][3];
    float* f[NF] = {};
    float* lam = nullptr;   // [ra (n3) | rb (n3) | U (n1 n2) | V (n1 n2)]
    double* dsc = nullptr;  // device scalars
    int* err = nullptr;     // device error flag of the tensor-core kernels
    int* err_host = nullptr;
    long long gemm_launches = 0;
    // exact-integer slice path (tfde_oz.cu)
    __nv_bfloat16* oz_op[3] = {};      // per axis: OZ_SLICES digit matrices of eta_a B_a
    int* oz_rexp[3] = {};              // per axis: row exponents
    CUtensorMap oz_amap[3][OZ_SLICES];
    __nv_bfloat16* oz_planes = nullptr;  // OZ_SLICES digit planes of the sliced vector
    int* oz_lexp = nullptr;            // line exponents of the sliced vector
    CUtensorMap oz_bmap[OZ_SLICES][3];
};

inline MixedState* mixed(const tfde_problem* P) { return static_cast<MixedState*>(P->mixed); }

int oz_init(tfde_problem* P, const std::vector<double> etaB[3], cudaStream_t s);
void oz_free(MixedState* M);
int accurate_apply(const tfde_problem* P, int op, const double* x, double* y, cudaStream_t s);

}  // namespace tfde
