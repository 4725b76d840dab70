// FFT-embedded per-axis Toeplitz products and DST-I (tfde_fft.cu).
#pragma once

#include <cuda_runtime.h>

#include "tfde_internal.h"

namespace tfde {
namespace fft {

// Grids with every n_a <= kMaxN (FFT length <= 4096) use the FFT passes.
constexpr int kMaxN = 2048;

// A device table in FP64 and FP32.
struct Table {
    double2* d = nullptr;
    float2* f = nullptr;
};

// Per-problem FFT data (tfde_problem::fft).
struct State {
    int L[3] = {0, 0, 0}, log2L[3] = {0, 0, 0};
    Table tw[3];        // exp(-2 pi i k / L), k < L
    Table G[3];         // spectra / L of eta_a B_a
    Table Ghat[2];      // x axis: M1 + eta1 B1 (op A), M1 - eta1 B1 (op RHS)
    Table pre[3];       // DST phases exp(i pi j^2 / (2(n+1))), j = 1..n
    Table chirp[3];     // spectrum / L of the chirp exp(-i pi m^2 / (2(n+1)))
    double dst_scale[3] = {0, 0, 0};
    float* lamf = nullptr;   // the mass and tau eigenvalues of every axis in FP32 (as tfde_problem::lam)
};

bool available(const int n[3]);
int fft_length(int n);
// Build the tables (no-op when the grid is not available()).
int init(tfde_problem* P, cudaStream_t s);
void free_state(tfde_problem* P);

// y = A x (op TFDE_OP_A), (2 A_N - A) x (TFDE_OP_RHS) or the stiffness terms
// (TFDE_OP_STIFF): three passes; a, w, c, e are workspace grid functions.
template <typename R>
int apply_A(const tfde_problem* P, int op, const R* x, R* y, R* a, R* w, R* c, R* e, cudaStream_t s);
// z = S_N Lambda^{-1} S_N r: five passes (the z pair fused); t1, t2 workspace.
template <typename R>
int apply_Pinv(const tfde_problem* P, const R* r, R* z, R* t1, R* t2, cudaStream_t s);

// z = P^{-1/2} r = S_N Lambda^{-1/2} S_N r (FP64): the symmetric square root
// of the preconditioner's inverse, from the same diagonalisation.
int apply_Pinv_half(const tfde_problem* P, const double* r, double* z, double* t1, double* t2, cudaStream_t s);

}  // namespace fft
}  // namespace tfde
