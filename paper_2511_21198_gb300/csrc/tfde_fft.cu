// FFT-embedded per-axis Toeplitz products and the DST-I by FFT: the fast
// transforms the paper applies its operators with (Introduction: Toeplitz
// matrix-vector products by FFT in O(n log n); Sec. 3: the tau preconditioner
// P^{-1} = S_N Lambda^{-1} S_N of Eq. (diag_tau_pre) with fast sine
// transforms), as CUDA kernels in FP64 (the all-FP64 path) and FP32.
//
// Toeplitz product.  An n x n Toeplitz matrix T (t_d on diagonal d = i - j,
// |d| < n) is the leading block of the circulant of length L >= 2n - 1 whose
// first column is c = (t_0, .., t_{n-1}, 0 .., 0, t_{-(n-1)}, .., t_{-1}), so
// T x = the first n entries of IFFT(FFT(c) . FFT(x padded with zeros)).  T is
// real, so two real lines ride in one complex line (x1 + i x2 -> T x1 + i T x2).
// The inverse transform is the forward one between two conjugations; 1/L is
// folded into the stored spectrum FFT(c) / L.
//
// DST-I.  (S x)_k = s sum_j sin(pi j k / (n+1)) x_j (j, k = 1..n,
// s = sqrt(2/(n+1))).  With jk = (j^2 + k^2 - (k - j)^2) / 2 and theta =
// pi / (n+1):  (S x)_k = s Im[ w_k sum_j g_{k-j} (w_j x_j) ],  w_j =
// exp(i theta j^2 / 2), g_m = exp(-i theta m^2 / 2): a complex symmetric
// Toeplitz product between two diagonal phase scalings (the chirp-z /
// Bluestein form), so it uses the same embedding with L >= 2n - 1.  The
// phases are reduced exactly on the host (j^2 mod 4(n+1)).
//
// FFT.  Complex, length L = 2^m <= 4096, radix-4 Stockham autosort passes
// (a radix-2 pass last when m is odd) in shared memory: a block holds
// 4096 / L complex lines (64 KB in FP64), 256 threads, each pass reads its
// butterflies into registers, synchronises and writes the reordered results.
//
// One launch is one pass along one axis over all lines of the grid:
//   MODE_TOEPLITZ  out0 = alpha T in0 + beta M in1,  out1 = M in0
//                  (M = tridiag(1, 6, 1) / 8, the mass stencil; in1 / out1
//                  optional) -- the three passes of the operator of
//                  Eq. (linear_sys) in the factorisation
//                  A v = M3 [M2 Ghat1 v + G2 (M1 v)] + G3 (M2 M1 v);
//   MODE_DST       out0 = S in0;
//   MODE_DST2      out0 = S Lambda^{-1} S in0 along z (the middle of
//                  Eq. (diag_tau_pre), both z transforms in one pass).
#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include <vector>

#include "tfde_fft.h"
#include "tfde_stats.h"

namespace tfde {
namespace fft {

namespace {

constexpr int NT = 256;        // threads per block
constexpr int ELEMS = 4096;    // complex elements per block (lines x L)

template <typename R>
struct C2;
template <>
struct C2<double> {
    using T = double2;
};
template <>
struct C2<float> {
    using T = float2;
};

template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b) {
    T2 r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename T2>
__device__ __forceinline__ T2 cadd(T2 a, T2 b) {
    a.x += b.x;
    a.y += b.y;
    return a;
}
template <typename T2>
__device__ __forceinline__ T2 csub(T2 a, T2 b) {
    a.x -= b.x;
    a.y -= b.y;
    return a;
}
// a * (-i)
template <typename T2>
__device__ __forceinline__ T2 cmul_mi(T2 a) {
    T2 r;
    r.x = a.y;
    r.y = -a.x;
    return r;
}

struct Pass {
    const void* in0;
    const void* in1;
    void* out0;
    void* out1;
    int n1, n2, n3, axis;
    int n, L, log2L;
    long long lines;
    double alpha, beta;
    const void* spec;   // R2[L]: FFT(c) / L
    const void* tw;     // R2[L]: exp(-2 pi i k / L)
    const void* pre;    // R2[n]: DST phases w_j
    double dst_scale;   // sqrt(2 / (n + 1))
    const double* lam;  // MODE_DST2: [mass x | y | z | tau x | y | z]
    const float* lamf;  // the same in FP32 (the FP32 passes form Lambda in FP32)
    double c0, c1, c2;  // MODE_DST2: eta_a (k+ + k-)
    int half_power;     // MODE_DST2: divide by Lambda^{1/2} instead of Lambda (P^{-1/2})
};

__device__ __forceinline__ long long axis_stride(const Pass& p) {
    return p.axis == 0 ? 1LL : (p.axis == 1 ? (long long)p.n1 : (long long)p.n1 * p.n2);
}

// Offsets of the block's lines l0 + g, g < G, without a 64-bit division per
// element: along y a line is (i, q) = (l % n1, l / n1), taken from the
// block's first line by a carry.
struct LineMap {
    long long l0;
    unsigned i0;
    long long q0;
};
__device__ __forceinline__ LineMap line_map(const Pass& p, long long l0) {
    LineMap m;
    m.l0 = l0;
    m.i0 = 0;
    m.q0 = 0;
    if (p.axis == 1) {
        m.i0 = (unsigned)(l0 % p.n1);
        m.q0 = l0 / p.n1;
    }
    return m;
}
__device__ __forceinline__ long long line_off(const Pass& p, const LineMap& m, int g) {
    if (p.axis == 0) return (m.l0 + g) * (long long)p.n1;
    if (p.axis == 2) return m.l0 + g;
    unsigned i = m.i0 + (unsigned)g;
    long long q = m.q0;
    if (i >= (unsigned)p.n1) {
        q += i / (unsigned)p.n1;
        i %= (unsigned)p.n1;
    }
    return (long long)i + q * (long long)p.n1 * p.n2;
}
// element e of the block's (line g, position j < n) rows: along x j runs
// fastest (a 32-bit division by n), along y / z g does
__device__ __forceinline__ void row_index(int axis, int e, int lgG, int n, int* g, int* j) {
    if (axis == 0) {
        *g = (int)((unsigned)e / (unsigned)n);
        *j = e - *g * n;
    } else {
        *g = e & ((1 << lgG) - 1);
        *j = e >> lgG;
    }
}
// element e of the block's (line g, position j) grid with j < 2^lgJ: along x
// the lines are contiguous, so j runs fastest; along y and z consecutive
// lines are adjacent in memory, so g runs fastest
__device__ __forceinline__ void grid_index(int axis, int e, int lgG, int lgJ, int* g, int* j) {
    if (axis == 0) {
        *g = e >> lgJ;
        *j = e & ((1 << lgJ) - 1);
    } else {
        *g = e & ((1 << lgG) - 1);
        *j = e >> lgG;
    }
}

// Forward DFT of the block's complex lines in place (stride ls between lines).
template <typename R>
__device__ void block_fft(typename C2<R>::T* buf, int ls, int L, int log2L, const typename C2<R>::T* __restrict__ tw) {
    using T2 = typename C2<R>::T;
    int lgNs = 0;
    while (lgNs < log2L) {
        if (log2L - lgNs >= 2) {
            const int lgLr = log2L - 2, Lr = 1 << lgLr;
            const int Ns = 1 << lgNs;
            T2 v[4][4];
            int cc[4], jj[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int b = threadIdx.x + u * NT;   // butterfly of the block: line c, position j
                const int c = b >> lgLr, j = b & (Lr - 1);
                cc[u] = c;
                jj[u] = j;
                const int k = j & (Ns - 1);
                const int step = k << (log2L - lgNs - 2);   // k L / (4 Ns)
                const T2* src = buf + (size_t)c * ls + j;
                T2 x0 = src[0], x1 = src[Lr], x2 = src[2 * Lr], x3 = src[3 * Lr];
                if (k) {
                    x1 = cmul(x1, __ldg(tw + (step & (L - 1))));
                    x2 = cmul(x2, __ldg(tw + ((2 * step) & (L - 1))));
                    x3 = cmul(x3, __ldg(tw + ((3 * step) & (L - 1))));
                }
                const T2 a0 = cadd(x0, x2), a1 = csub(x0, x2);
                const T2 a2 = cadd(x1, x3), a3 = cmul_mi(csub(x1, x3));
                v[u][0] = cadd(a0, a2);
                v[u][1] = cadd(a1, a3);
                v[u][2] = csub(a0, a2);
                v[u][3] = csub(a1, a3);
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = jj[u];
                const int base = ((j >> lgNs) << (lgNs + 2)) + (j & (Ns - 1));
                T2* dst = buf + (size_t)cc[u] * ls + base;
                dst[0] = v[u][0];
                dst[Ns] = v[u][1];
                dst[2 * Ns] = v[u][2];
                dst[3 * Ns] = v[u][3];
            }
            __syncthreads();
            lgNs += 2;
        } else {
            const int lgLr = log2L - 1, Lr = 1 << lgLr;
            const int Ns = 1 << lgNs;
            T2 v[8][2];
            int cc[8], jj[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int b = threadIdx.x + u * NT;
                const int c = b >> lgLr, j = b & (Lr - 1);
                cc[u] = c;
                jj[u] = j;
                const int k = j & (Ns - 1);
                const int step = k << (log2L - lgNs - 1);   // k L / (2 Ns)
                const T2* src = buf + (size_t)c * ls + j;
                T2 x0 = src[0], x1 = src[Lr];
                if (k) x1 = cmul(x1, __ldg(tw + (step & (L - 1))));
                v[u][0] = cadd(x0, x1);
                v[u][1] = csub(x0, x1);
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = jj[u];
                const int base = ((j >> lgNs) << (lgNs + 1)) + (j & (Ns - 1));
                T2* dst = buf + (size_t)cc[u] * ls + base;
                dst[0] = v[u][0];
                dst[Ns] = v[u][1];
            }
            __syncthreads();
            lgNs += 1;
        }
    }
}

// buf <- conj(buf . spec), element-wise over the block's lines.
template <typename R>
__device__ __forceinline__ void block_spectral_scale(typename C2<R>::T* buf, int ls, int L, int log2L,
                                                     const typename C2<R>::T* __restrict__ spec) {
    using T2 = typename C2<R>::T;
    for (int e = threadIdx.x; e < ELEMS; e += NT) {
        const int c = e >> log2L, k = e & (L - 1);
        T2* q = buf + (size_t)c * ls + k;
        T2 v = cmul(*q, __ldg(spec + k));
        v.y = -v.y;
        *q = v;
    }
    __syncthreads();
}

enum { MODE_TOEPLITZ = 0, MODE_DST = 1, MODE_DST2 = 2 };

template <typename R, int MODE>
__global__ void __launch_bounds__(NT) fft_pass_kernel(const Pass p) {
    using T2 = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char fft_smem[];
    T2* buf = reinterpret_cast<T2*>(fft_smem);
    const int L = p.L, lg = p.log2L, n = p.n;
    const int lgCL = 12 - lg;                       // log2(ELEMS / L)
    const int CL = 1 << lgCL;
    const int lgG = MODE == MODE_TOEPLITZ ? lgCL + 1 : lgCL;
    const int G = 1 << lgG;                         // real lines of this block
    const int ls = L + 1;                           // padded line stride (bank spread)
    const long long l0 = (long long)blockIdx.x * G;
    const long long st = axis_stride(p);
    const R* __restrict__ in0 = static_cast<const R*>(p.in0);
    const R* __restrict__ in1 = static_cast<const R*>(p.in1);
    R* __restrict__ out0 = static_cast<R*>(p.out0);
    R* __restrict__ out1 = static_cast<R*>(p.out1);
    const T2* __restrict__ tw = static_cast<const T2*>(p.tw);
    const T2* __restrict__ spec = static_cast<const T2*>(p.spec);
    const T2* __restrict__ pre = static_cast<const T2*>(p.pre);

    const LineMap lm = line_map(p, l0);

    // ---- load (zero padding beyond n and beyond the last line)
    for (int e = threadIdx.x; e < G * L; e += NT) {
        int g, j;
        grid_index(p.axis, e, lgG, lg, &g, &j);
        const long long l = l0 + g;
        R v = R(0);
        if (j < n && l < p.lines) v = in0[line_off(p, lm, g) + j * st];
        if constexpr (MODE == MODE_TOEPLITZ) {
            T2* q = buf + (size_t)(g >> 1) * ls + j;
            if (g & 1) q->y = v; else q->x = v;
        } else {
            T2 w;
            if (j < n) {
                const T2 ph = __ldg(pre + j);
                w.x = ph.x * v;
                w.y = ph.y * v;
            } else {
                w.x = R(0);
                w.y = R(0);
            }
            buf[(size_t)g * ls + j] = w;
        }
    }
    __syncthreads();
    if constexpr (MODE == MODE_TOEPLITZ) {
        // out1 = M in0 along the axis, from the staged values
        if (out1) {
            for (int e = threadIdx.x; e < G * n; e += NT) {
                int g, j;
                row_index(p.axis, e, lgG, n, &g, &j);
                const long long l = l0 + g;
                if (l >= p.lines) continue;
                const T2* q = buf + (size_t)(g >> 1) * ls + j;
                const R c = (g & 1) ? q->y : q->x;
                R nb = R(0);
                if (j > 0) nb += (g & 1) ? q[-1].y : q[-1].x;
                if (j + 1 < n) nb += (g & 1) ? q[1].y : q[1].x;
                out1[line_off(p, lm, g) + j * st] = fma(R(0.75), c, R(0.125) * nb);
            }
        }
        __syncthreads();
    }
    block_fft<R>(buf, ls, L, lg, tw);
    block_spectral_scale<R>(buf, ls, L, lg, spec);
    block_fft<R>(buf, ls, L, lg, tw);
    if constexpr (MODE == MODE_DST2) {
        // t = S in0 (real, k < n), then t / Lambda(i, j, k) re-phased as the
        // input of the second transform; lines along z: l = i + n1 j
        const double* mx = p.lam;
        const double* my = mx + p.n1;
        const double* mz = my + p.n2;
        const double* tx = mz + p.n3;
        const double* ty = tx + p.n1;
        const double* tz = ty + p.n2;
        const R s = (R)p.dst_scale;
        // lines along z: l = i + n1 j, taken from the block's first line by a carry
        const unsigned i0 = (unsigned)(l0 % p.n1);
        const long long j0 = l0 / p.n1;
        const float fc0 = (float)p.c0, fc1 = (float)p.c1, fc2 = (float)p.c2;
        for (int e = threadIdx.x; e < G * L; e += NT) {
            int g, k;
            grid_index(p.axis, e, lgG, lg, &g, &k);
            T2* q = buf + (size_t)g * ls + k;
            T2 w;
            w.x = R(0);
            w.y = R(0);
            const long long l = l0 + g;
            if (k < n && l < p.lines) {
                const T2 ph = __ldg(pre + k);
                const T2 r = *q;   // conj of the product: (r.x, -r.y)
                const R t = s * (ph.y * r.x - ph.x * r.y);
                unsigned i = i0 + (unsigned)g;
                int jy = (int)j0;
                if (i >= (unsigned)p.n1) {
                    jy += (int)(i / (unsigned)p.n1);
                    i %= (unsigned)p.n1;
                }
                R u;
                if constexpr (sizeof(R) == 4) {
                    // Lambda = mz (my (mx + c0 tx) + c1 ty mx) + tz c2 my mx, in FP32
                    const float* fx = p.lamf;
                    const float* fy = fx + p.n1;
                    const float* fz = fy + p.n2;
                    const float* gx = fz + p.n3;
                    const float* gy = gx + p.n1;
                    const float* gz = gy + p.n2;
                    const float mxi = __ldg(fx + i), myj = __ldg(fy + jy);
                    const float U = fmaf(myj, fmaf(fc0, __ldg(gx + i), mxi), fc1 * __ldg(gy + jy) * mxi);
                    const float V = fc2 * myj * mxi;
                    const float lam = fmaf(__ldg(fz + k), U, __ldg(gz + k) * V);
                    u = (R)(t / (p.half_power ? sqrtf(lam) : lam));
                } else {
                    const double lam = mz[k] * my[jy] * mx[i] + p.c0 * mz[k] * my[jy] * tx[i] +
                                       p.c1 * mz[k] * ty[jy] * mx[i] + p.c2 * tz[k] * my[jy] * mx[i];
                    u = (R)((double)t / (p.half_power ? sqrt(lam) : lam));
                }
                w.x = ph.x * u;
                w.y = ph.y * u;
            }
            *q = w;   // each element is read and rewritten by the same thread
        }
        __syncthreads();
        block_fft<R>(buf, ls, L, lg, tw);
        block_spectral_scale<R>(buf, ls, L, lg, spec);
        block_fft<R>(buf, ls, L, lg, tw);
    }

    // ---- store
    for (int e = threadIdx.x; e < G * n; e += NT) {
        int g, j;
        row_index(p.axis, e, lgG, n, &g, &j);
        const long long l = l0 + g;
        if (l >= p.lines) continue;
        const long long o = line_off(p, lm, g) + j * st;
        R v;
        if constexpr (MODE == MODE_TOEPLITZ) {
            const T2 q = buf[(size_t)(g >> 1) * ls + j];
            v = (R)p.alpha * ((g & 1) ? -q.y : q.x);
            if (in1) {
                R nb = R(0);
                if (j > 0) nb += in1[o - st];
                if (j + 1 < n) nb += in1[o + st];
                v = fma((R)p.beta, fma(R(0.75), in1[o], R(0.125) * nb), v);
            }
        } else {
            const T2 ph = __ldg(pre + j);
            const T2 r = buf[(size_t)g * ls + j];
            v = (R)p.dst_scale * (ph.y * r.x - ph.x * r.y);
        }
        out0[o] = v;
    }
}

// ------------------------------------------------------------------- host
using cld = std::complex<long double>;

// In-place forward DFT on the host (iterative radix-2, long double).
void host_fft(std::vector<cld>& a) {
    const size_t L = a.size();
    for (size_t i = 1, j = 0; i < L; ++i) {
        size_t bit = L >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    const long double pi = 3.141592653589793238462643383279502884L;
    for (size_t len = 2; len <= L; len <<= 1) {
        for (size_t i = 0; i < L; i += len)
            for (size_t k = 0; k < len / 2; ++k) {
                const long double ang = -2.0L * pi * (long double)k / (long double)len;
                const cld w(std::cos(ang), std::sin(ang));
                const cld u = a[i + k], v = a[i + k + len / 2] * w;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
    }
}

int log2_exact(int L) {
    int m = 0;
    while ((1 << m) < L) ++m;
    return m;
}

template <typename T>
int dcopy(T** dst, const std::vector<T>& v, cudaStream_t s) {
    if (cudaMalloc((void**)dst, v.size() * sizeof(T)) != cudaSuccess)
        return set_error(TFDE_ENOMEM, "cudaMalloc of FFT tables failed");
    if (cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return set_error(TFDE_ECUDA, "upload of FFT tables failed");
    return TFDE_OK;
}

// Spectrum FFT(c) / L of the circulant embedding of t_d, d in [-(n-1), n-1]
// (t[d + n - 1]), in double and float.
int upload_spectrum(const std::vector<long double>& t, int n, int L, Table* out, cudaStream_t s) {
    std::vector<cld> c(L, cld(0, 0));
    for (int d = 0; d < n; ++d) c[d] = cld(t[d + n - 1], 0);
    for (int d = 1; d < n; ++d) c[L - d] = cld(t[n - 1 - d], 0);
    host_fft(c);
    std::vector<double2> hd(L);
    std::vector<float2> hf(L);
    for (int k = 0; k < L; ++k) {
        const cld v = c[k] / (long double)L;
        hd[k] = make_double2((double)v.real(), (double)v.imag());
        hf[k] = make_float2((float)v.real(), (float)v.imag());
    }
    int st = dcopy(&out->d, hd, s);
    if (!st) st = dcopy(&out->f, hf, s);
    return st;
}

}  // namespace

bool available(const int n[3]) {
    for (int a = 0; a < 3; ++a)
        if (n[a] < 1 || n[a] > kMaxN) return false;
    return true;
}

int fft_length(int n) {
    int L = 2;
    while (L < 2 * n - 1) L <<= 1;
    return L;
}

int init(tfde_problem* P, cudaStream_t s) {
    if (!available(P->n)) return TFDE_OK;   // the dense FP64 contraction stays in use
    State* F = new State();
    P->fft = F;
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int a = 0; a < 3; ++a) {
        const int n = P->n[a];
        const int L = fft_length(n);
        F->L[a] = L;
        F->log2L[a] = log2_exact(L);
        int st;
        {
            std::vector<double2> hd(L);
            std::vector<float2> hf(L);
            for (int k = 0; k < L; ++k) {
                const long double ang = -2.0L * pi * (long double)k / (long double)L;
                hd[k] = make_double2((double)std::cos(ang), (double)std::sin(ang));
                hf[k] = make_float2((float)std::cos(ang), (float)std::sin(ang));
            }
            if ((st = dcopy(&F->tw[a].d, hd, s)) || (st = dcopy(&F->tw[a].f, hf, s))) return st;
        }
        // Toeplitz generators: eta B (d = i - j: k+ q_{d+1} + k- q_{1-d}) and the mass stencil
        const double kp = P->p.kp[a], km = P->p.km[a];
        std::vector<long double> tG(2 * n - 1, 0.0L), tA(2 * n - 1), tR(2 * n - 1);
        for (int d = -(n - 1); d <= n - 1; ++d) {
            long double v = 0.0L;
            if (d + 1 >= 0 && d + 1 <= n) v += (long double)kp * (long double)P->q[a][d + 1];
            if (1 - d >= 0 && 1 - d <= n) v += (long double)km * (long double)P->q[a][1 - d];
            tG[d + n - 1] = (long double)P->eta[a] * v;
        }
        for (int d = -(n - 1); d <= n - 1; ++d) {
            const long double m = d == 0 ? 0.75L : ((d == 1 || d == -1) ? 0.125L : 0.0L);
            tA[d + n - 1] = m + tG[d + n - 1];
            tR[d + n - 1] = m - tG[d + n - 1];
        }
        if ((st = upload_spectrum(tG, n, L, &F->G[a], s))) return st;
        if (a == 0) {
            if ((st = upload_spectrum(tA, n, L, &F->Ghat[0], s)) || (st = upload_spectrum(tR, n, L, &F->Ghat[1], s)))
                return st;
        }
        // DST-I (Bluestein): phases w_j = exp(i pi (j^2 mod 4(n+1)) / (2(n+1))), j = 1..n,
        // chirp g_m = exp(-i pi (m^2 mod 4(n+1)) / (2(n+1))), symmetric in m
        {
            const long long mod = 4LL * (n + 1);
            std::vector<double2> pd(n);
            std::vector<float2> pf(n);
            for (int j = 1; j <= n; ++j) {
                const long double ang = pi * (long double)(((long long)j * j) % mod) / (2.0L * (n + 1));
                pd[j - 1] = make_double2((double)std::cos(ang), (double)std::sin(ang));
                pf[j - 1] = make_float2((float)std::cos(ang), (float)std::sin(ang));
            }
            if ((st = dcopy(&F->pre[a].d, pd, s)) || (st = dcopy(&F->pre[a].f, pf, s))) return st;
            std::vector<cld> c(L, cld(0, 0));
            for (int m = 0; m < n; ++m) {
                const long double ang = -pi * (long double)(((long long)m * m) % mod) / (2.0L * (n + 1));
                const cld g(std::cos(ang), std::sin(ang));
                c[m] = g;
                if (m > 0) c[L - m] = g;
            }
            host_fft(c);
            std::vector<double2> hd(L);
            std::vector<float2> hf(L);
            for (int k = 0; k < L; ++k) {
                const cld v = c[k] / (long double)L;
                hd[k] = make_double2((double)v.real(), (double)v.imag());
                hf[k] = make_float2((float)v.real(), (float)v.imag());
            }
            if ((st = dcopy(&F->chirp[a].d, hd, s)) || (st = dcopy(&F->chirp[a].f, hf, s))) return st;
            F->dst_scale[a] = std::sqrt(2.0 / (n + 1));
        }
    }
    {   // the eigenvalue arrays of Lambda in FP32, layout [mass x | y | z | tau x | y | z]
        std::vector<float> lf;
        for (int a = 0; a < 3; ++a)
            for (double v : P->lam_mass[a]) lf.push_back((float)v);
        for (int a = 0; a < 3; ++a)
            for (double v : P->lam_tau[a]) lf.push_back((float)v);
        if (int st = dcopy(&F->lamf, lf, s)) return st;
    }
    return TFDE_OK;
}

void free_state(tfde_problem* P) {
    State* F = static_cast<State*>(P->fft);
    if (!F) return;
    auto rel = [](Table& t) {
        cudaFree(t.d);
        cudaFree(t.f);
    };
    for (int a = 0; a < 3; ++a) {
        rel(F->tw[a]);
        rel(F->G[a]);
        rel(F->pre[a]);
        rel(F->chirp[a]);
    }
    rel(F->Ghat[0]);
    rel(F->Ghat[1]);
    cudaFree(F->lamf);
    delete F;
    P->fft = nullptr;
}

namespace {

bool g_attr[2][3] = {};

template <typename R, int MODE>
int launch_pass(const Pass& p, cudaStream_t s) {
    using T2 = typename C2<R>::T;
    const int lgCL = 12 - p.log2L;
    const int G = MODE == MODE_TOEPLITZ ? (2 << lgCL) : (1 << lgCL);
    const size_t smem = (size_t)(1 << lgCL) * (p.L + 1) * sizeof(T2);
    const int ti = sizeof(R) == 8 ? 0 : 1;
    if (!g_attr[ti][MODE]) {
        if (cudaFuncSetAttribute(fft_pass_kernel<R, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)((ELEMS + ELEMS) * sizeof(T2))) != cudaSuccess)
            return set_error(TFDE_ECUDA, "cudaFuncSetAttribute(fft_pass_kernel) failed");
        g_attr[ti][MODE] = true;
    }
    const long long blocks = (p.lines + G - 1) / G;
    // algorithmic work: every grid function read and written once; complex
    // transforms of length L at 5 L log2 L flops, 6 L for a spectral product
    const double N = (double)p.lines * p.n;
    const double nio = 2.0 + (p.in1 ? 1.0 : 0.0) + (p.out1 ? 1.0 : 0.0);
    const double cl = MODE == MODE_TOEPLITZ ? (double)p.lines / 2.0 : (double)p.lines;
    const double per = 2.0 * 5.0 * p.L * p.log2L + 6.0 * p.L;
    const double flops = cl * per * (MODE == MODE_DST2 ? 2.0 : 1.0);
    void* tok = stats_tc_begin(s, TFDE_KIND_FFT);
    fft_pass_kernel<R, MODE><<<(unsigned)blocks, NT, smem, s>>>(p);
    const cudaError_t e = cudaGetLastError();
    stats_tc_end(tok, s, TFDE_KIND_FFT, nio * N * sizeof(R), flops);
    if (e != cudaSuccess) return set_error(TFDE_ECUDA, std::string("fft_pass_kernel: ") + cudaGetErrorString(e));
    return TFDE_OK;
}

Pass base_pass(const tfde_problem* P, int axis, bool fp64) {
    const State* F = static_cast<const State*>(P->fft);
    Pass p;
    std::memset(&p, 0, sizeof(p));
    p.n1 = P->n[0];
    p.n2 = P->n[1];
    p.n3 = P->n[2];
    p.axis = axis;
    p.n = P->n[axis];
    p.L = F->L[axis];
    p.log2L = F->log2L[axis];
    p.lines = (long long)P->N / P->n[axis];
    p.tw = fp64 ? (const void*)F->tw[axis].d : (const void*)F->tw[axis].f;
    p.pre = fp64 ? (const void*)F->pre[axis].d : (const void*)F->pre[axis].f;
    p.dst_scale = F->dst_scale[axis];
    return p;
}

template <typename R>
int toeplitz_pass(const tfde_problem* P, int axis, const Table& T, double alpha, const R* in0, const R* in1,
                  double beta, R* out0, R* out1, cudaStream_t s) {
    Pass p = base_pass(P, axis, sizeof(R) == 8);
    p.spec = sizeof(R) == 8 ? (const void*)T.d : (const void*)T.f;
    p.alpha = alpha;
    p.beta = beta;
    p.in0 = in0;
    p.in1 = in1;
    p.out0 = out0;
    p.out1 = out1;
    return launch_pass<R, MODE_TOEPLITZ>(p, s);
}

template <typename R>
int dst_pass(const tfde_problem* P, int axis, const R* in, R* out, bool lambda_pair, cudaStream_t s,
             bool half_power = false) {
    const State* F = static_cast<const State*>(P->fft);
    Pass p = base_pass(P, axis, sizeof(R) == 8);
    p.spec = sizeof(R) == 8 ? (const void*)F->chirp[axis].d : (const void*)F->chirp[axis].f;
    p.in0 = in;
    p.out0 = out;
    if (lambda_pair) {
        p.lam = P->lam;
        p.lamf = F->lamf;
        p.c0 = P->csum[0];
        p.c1 = P->csum[1];
        p.c2 = P->csum[2];
        p.half_power = half_power ? 1 : 0;
        return launch_pass<R, MODE_DST2>(p, s);
    }
    return launch_pass<R, MODE_DST>(p, s);
}

}  // namespace

template <typename R>
int apply_A(const tfde_problem* P, int op, const R* x, R* y, R* a, R* w, R* c, R* e, cudaStream_t s) {
    const State* F = static_cast<const State*>(P->fft);
    const bool rhs = (op & 1) != 0;
    const bool stiff = (op & TFDE_OP_STIFF) != 0;
    const double sg = rhs ? -1.0 : 1.0;
    int st;
    // x: a = Ghat1 x (or sg eta1 B1 x for the stiffness terms alone), w = M1 x
    if (stiff) st = toeplitz_pass<R>(P, 0, F->G[0], sg, x, nullptr, 0.0, a, w, s);
    else st = toeplitz_pass<R>(P, 0, F->Ghat[rhs ? 1 : 0], 1.0, x, nullptr, 0.0, a, w, s);
    if (st) return st;
    // 2-D problem: the y pass gives the result (no third axis)
    if (P->dim2) return toeplitz_pass<R>(P, 1, F->G[1], sg, w, a, 1.0, y, nullptr, s);
    // y: c = sg G2 w + M2 a, e = M2 w
    if ((st = toeplitz_pass<R>(P, 1, F->G[1], sg, w, a, 1.0, c, e, s))) return st;
    // z: y = sg G3 e + M3 c
    return toeplitz_pass<R>(P, 2, F->G[2], sg, e, c, 1.0, y, nullptr, s);
}

template <typename R>
int apply_Pinv(const tfde_problem* P, const R* r, R* z, R* t1, R* t2, cudaStream_t s) {
    int st;
    if ((st = dst_pass<R>(P, 0, r, t1, false, s))) return st;
    if ((st = dst_pass<R>(P, 1, t1, t2, false, s))) return st;
    if ((st = dst_pass<R>(P, 2, t2, t1, true, s))) return st;   // S_z Lambda^{-1} S_z
    if ((st = dst_pass<R>(P, 1, t1, t2, false, s))) return st;
    return dst_pass<R>(P, 0, t2, z, false, s);
}

int apply_Pinv_half(const tfde_problem* P, const double* r, double* z, double* t1, double* t2, cudaStream_t s) {
    int st;
    if ((st = dst_pass<double>(P, 0, r, t1, false, s))) return st;
    if ((st = dst_pass<double>(P, 1, t1, t2, false, s))) return st;
    if ((st = dst_pass<double>(P, 2, t2, t1, true, s, true))) return st;   // S_z Lambda^{-1/2} S_z
    if ((st = dst_pass<double>(P, 1, t1, t2, false, s))) return st;
    return dst_pass<double>(P, 0, t2, z, false, s);
}

template int apply_A<double>(const tfde_problem*, int, const double*, double*, double*, double*, double*, double*,
                             cudaStream_t);
template int apply_A<float>(const tfde_problem*, int, const float*, float*, float*, float*, float*, float*,
                            cudaStream_t);
template int apply_Pinv<double>(const tfde_problem*, const double*, double*, double*, double*, cudaStream_t);
template int apply_Pinv<float>(const tfde_problem*, const float*, float*, float*, float*, cudaStream_t);

}  // namespace fft
}  // namespace tfde
