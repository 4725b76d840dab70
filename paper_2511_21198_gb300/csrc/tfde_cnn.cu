// Warm-start network of the CN solves: four 3x3x3 convolutions with zero
// padding and ReLU between them, mapping per grid point the 11 input channels
//   (u / s, dt F / s, c_1..c_9),   s = max |u^m|,  c = nine problem constants,
// to (u^{m+1} - u^m) / s.  Not part of the paper: a learned initial guess for
// its Krylov solves; the FP64 residual test decides what the solver returns.
//
// Layout.  Activations are BF16, channels last, 16 channels (zero padded), on
// a grid with one layer of zero guard points on every side:
//   slot s = ((z + 1) (n2 + 2) + (y + 1)) R + (x + 1),   R = n1 + 2,
// so that every 3x3x3 tap is a constant shift of the slot index (dz P + dy R
// + dx, P = (n2 + 2) R) and the zero padding is the guard data itself.
//
// Forward / input-gradient convolution (tcgen05 implicit GEMM): a tile is 128
// consecutive slots (M = 128), N = 16 output channels, K = 16 input channels
// per tap, 27 MMAs per tile.  For each of the 9 (dz, dy) rows one TMA box of
// 130 slots x 8 channels per channel half is staged (non-swizzled K-major:
// the two halves are the K-adjacent core matrices); the three dx taps of a
// row are the same staged rows shifted by 16 bytes.  Warps 0..3 load (the 18
// boxes of a tile dealt round-robin), warp 4 issues the MMAs into a
// double-buffered TMEM accumulator, warps 5..8 run the
// epilogue (bias, ReLU or ReLU-gradient mask, BF16 store of interior slots, or
// the FP32 output channel on the plain grid).  Weight gradients and the small
// element-wise steps run on CUDA cores.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "tfde_internal.h"
#include "tfde_stats.h"
#include "tfde_tc.h"
#include "tfde_tc_ptx.cuh"

namespace tfde {
namespace cnn {

constexpr int CH = 16;             // padded channels
constexpr int NL = 4;              // layers
constexpr int NTAP = 27;
constexpr int WSZ = CH * CH * NTAP;  // weights per layer (FP32 master [co][ci][tap])
constexpr int PSZ = WSZ + CH;        // + bias
constexpr int TM = 128;            // slots per tile
constexpr int BOX = TM + 2;        // staged slots per row
constexpr int HALF_BYTES = 2176;   // BOX * 16 B rounded up to 128 B
constexpr int ROW_BYTES = 2 * HALF_BYTES;
constexpr int STAGE_BYTES = 9 * ROW_BYTES;               // 39168
constexpr int STAGES = 2;
constexpr int W_BYTES = NTAP * 2 * CH * 16;              // 13824: [tap][khalf][co][8 ci]
constexpr int NUM_BARS = 2 * STAGES + 5;
constexpr int SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + W_BYTES + NUM_BARS * 8 + 16;
constexpr int PRODUCERS = 4;       // warps 0..3 issue the 18 row boxes of a tile round-robin
constexpr int MMA_WARP = PRODUCERS;
constexpr int NUM_THREADS = 32 * (PRODUCERS + 1 + 4);   // + MMA warp + 4 epilogue warps
constexpr uint32_t TMEM_COLS = 32; // 2 x 16 columns
static_assert(SMEM_BYTES <= 232448, "shared memory budget");

struct ConvParams {
    CUtensorMap amap;              // activations [S_total][16] BF16, box {8, 130}
    const __nv_bfloat16* wts;      // [27][2][16][8] BF16 (B operand layout)
    const float* bias;             // [16] or null
    int relu;                      // apply ReLU after the bias
    const __nv_bfloat16* mask;     // [S_total][16] or null: multiply by (mask > 0)
    __nv_bfloat16* out_act;        // [S_total][16] or null
    float* out_f32;                // plain grid, channel 0, or null
    int n1, n2, n3;
    long long R, P, first, ntiles;
    int* err;
};

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__global__ void __launch_bounds__(NUM_THREADS, 1) conv_kernel(const __grid_constant__ ConvParams p) {
    using namespace tfde::tc;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* stages = smem;
    uint8_t* wsm = smem + STAGES * STAGE_BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(wsm + W_BYTES);
    uint64_t* full = bars;
    uint64_t* empty = bars + STAGES;
    uint64_t* tfull = bars + 2 * STAGES;
    uint64_t* tempty = bars + 2 * STAGES + 2;
    uint64_t* mma_done = bars + 2 * STAGES + 4;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + NUM_BARS);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // weights into shared memory (generic proxy), made visible to the tensor core
    {
        const uint4* src = reinterpret_cast<const uint4*>(p.wts);
        uint4* dst = reinterpret_cast<uint4*>(wsm);
        for (int i = threadIdx.x; i < W_BYTES / 16; i += NUM_THREADS) dst[i] = src[i];
        fence_proxy_async_smem();
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], PRODUCERS);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        mbar_init(mma_done, 1);
        mbar_fence_init();
    }
    if (warp == MMA_WARP) tmem_alloc(tmem_slot, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const long long total = p.ntiles;

    if (warp < PRODUCERS) {
        if (lane == 0) {
            const int pw = warp;
            int s = 0;
            uint32_t ph = 0, filled = 0, last_ph = 0;
            for (long long t = blockIdx.x; t < total; t += gridDim.x) {
                if (!mbar_wait(&empty[s], ph ^ 1u, p.err)) break;
                uint8_t* st = stages + s * STAGE_BYTES;
                uint32_t mine = 0;
                for (int i = pw; i < 18; i += PRODUCERS) mine += BOX * 16u;
                mbar_expect_tx(&full[s], mine);
                const long long s0 = p.first + t * TM;
                for (int i = pw; i < 18; i += PRODUCERS) {
                    const int r = i >> 1, h = i & 1;
                    const int dz = r / 3 - 1, dy = r % 3 - 1;
                    const long long start = s0 - 1 + dz * p.P + dy * p.R;   // >= 0 by the guard planes
                    tma_load_2d(st + r * ROW_BYTES + h * HALF_BYTES, &p.amap, &full[s], 8 * h, (int)start);
                }
                filled |= 1u << s;
                if (ph) last_ph |= 1u << s; else last_ph &= ~(1u << s);
                if (++s == STAGES) { s = 0; ph ^= 1u; }
            }
            for (int i = 0; i < STAGES; ++i)
                if (filled & (1u << i)) mbar_wait(&full[i], (last_ph >> i) & 1u, p.err, false);
        }
    } else if (warp == MMA_WARP) {
        if (lane == 0) {
            const uint32_t idesc = instr_desc(TM, CH, 0);
            // non-swizzled K-major: LBO = K-adjacent core matrix (channel half), SBO = next 8 rows
            const uint64_t a0 = smem_desc(smem_u32(stages), HALF_BYTES, 128, 0);
            const uint64_t b0 = smem_desc(smem_u32(wsm), 256, 128, 0);
            int s = 0;
            uint32_t ph = 0;
            long long it = 0;
            bool ok = true;
            for (long long t = blockIdx.x; t < total && ok; t += gridDim.x, ++it) {
                const int buf = (int)(it & 1);
                const uint32_t use = (uint32_t)(it >> 1);
                if (!mbar_wait(&tempty[buf], (use & 1u) ^ 1u, p.err)) { ok = false; break; }
                if (!mbar_wait(&full[s], ph, p.err)) { ok = false; break; }
                tc_fence_after();
                const uint64_t as = a0 + (uint64_t)((s * STAGE_BYTES) >> 4);
#pragma unroll
                for (int tap = 0; tap < NTAP; ++tap) {
                    const int r = tap / 3, dx = tap % 3;   // tap = (dz+1)*9 + (dy+1)*3 + (dx+1)
                    const uint64_t ad = as + (uint64_t)((r * ROW_BYTES + dx * 16) >> 4);
                    const uint64_t bd = b0 + (uint64_t)((tap * 512) >> 4);
                    umma_bf16(tmem_base + (uint32_t)(buf * CH), ad, bd, idesc, tap > 0 ? 1u : 0u);
                }
                umma_commit(&empty[s]);
                umma_commit(&tfull[buf]);
                if (++s == STAGES) { s = 0; ph ^= 1u; }
            }
            umma_commit(mma_done);
            mbar_wait(mma_done, 0, p.err, false);
        }
    } else {
        const int q = warp & 3;   // TMEM lane quadrant
        long long it = 0;
        const long long plane_slots = p.P;
        for (long long t = blockIdx.x; t < total; t += gridDim.x, ++it) {
            const int buf = (int)(it & 1);
            const uint32_t use = (uint32_t)(it >> 1);
            int ok = 1;
            if (lane == 0) ok = mbar_wait(&tfull[buf], use & 1u, p.err) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            __syncwarp();
            tc_fence_after();
            uint32_t r[16];
            tmem_ld16(tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * CH), r);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
            const long long s = p.first + t * TM + 32 * q + lane;
            const long long x1 = s % p.R, rem = s / p.R;
            const long long y1 = rem % (plane_slots / p.R), z1 = rem / (plane_slots / p.R);
            const bool interior = x1 >= 1 && x1 <= p.n1 && y1 >= 1 && y1 <= p.n2 && z1 >= 1 && z1 <= p.n3;
            if (!interior) continue;
            float v[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                float a = __uint_as_float(r[c]);
                if (p.bias) a += __ldg(p.bias + c);
                if (p.relu) a = fmaxf(a, 0.f);
                v[c] = a;
            }
            if (p.mask) {
                const uint4* mk = reinterpret_cast<const uint4*>(p.mask + s * CH);
                const uint4 m0 = __ldg(mk), m1 = __ldg(mk + 1);
                const __nv_bfloat16* mb0 = reinterpret_cast<const __nv_bfloat16*>(&m0);
                const __nv_bfloat16* mb1 = reinterpret_cast<const __nv_bfloat16*>(&m1);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    if (!(__bfloat162float(mb0[c]) > 0.f)) v[c] = 0.f;
                    if (!(__bfloat162float(mb1[c]) > 0.f)) v[8 + c] = 0.f;
                }
            }
            if (p.out_act) {
                uint4 o0, o1;
                __nv_bfloat162* h0 = reinterpret_cast<__nv_bfloat162*>(&o0);
                __nv_bfloat162* h1 = reinterpret_cast<__nv_bfloat162*>(&o1);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    h0[c] = __floats2bfloat162_rn(v[2 * c], v[2 * c + 1]);
                    h1[c] = __floats2bfloat162_rn(v[8 + 2 * c], v[8 + 2 * c + 1]);
                }
                uint4* dst = reinterpret_cast<uint4*>(p.out_act + s * CH);
                dst[0] = o0;
                dst[1] = o1;
            }
            if (p.out_f32) p.out_f32[((z1 - 1) * p.n2 + (y1 - 1)) * p.n1 + (x1 - 1)] = v[0];
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == MMA_WARP) tmem_dealloc(tmem_base, TMEM_COLS);
}

// ------------------------------------------------------------ CUDA-core kernels
__device__ __forceinline__ long long slot_of(long long p, int n1, int n2, long long R, long long P) {
    const long long x = p % n1, r = p / n1;
    const long long y = r % n2, z = r / n2;
    return (z + 1) * P + (y + 1) * R + (x + 1);
}

// max |u| into *out (one block, deterministic)
__global__ void maxabs_kernel(const double* __restrict__ u, long long N, double* __restrict__ out) {
    __shared__ double sh[256];
    double m = 0.0;
    for (long long i = threadIdx.x; i < N; i += blockDim.x) m = fmax(m, fabs(u[i]));
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0] > 0.0 ? sh[0] : 1.0;
}

// X0[slot] = (u/s, dtF/s, c_0..c_8, d1/s, d2/s, 0...) for every interior grid
// point; d1 = u - u1 and d2 = u - 2 u1 + u2 are the first and second
// differences of the time history (zero channels without it)
__global__ void pack_input_kernel(const double* __restrict__ u, const double* __restrict__ u1,
                                  const double* __restrict__ u2, const double* __restrict__ dtF,
                                  const double* __restrict__ scale, const float* __restrict__ coef, int n1, int n2,
                                  long long N, long long R, long long P, __nv_bfloat16* __restrict__ X) {
    const double inv = 1.0 / scale[0];
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        float v[16];
        v[0] = (float)(u[p] * inv);
        v[1] = dtF ? (float)(dtF[p] * inv) : 0.f;
#pragma unroll
        for (int c = 0; c < 9; ++c) v[2 + c] = coef[c];
        v[11] = u1 ? (float)((u[p] - u1[p]) * inv) : 0.f;
        v[12] = (u1 && u2) ? (float)((u[p] - 2.0 * u1[p] + u2[p]) * inv) : 0.f;
#pragma unroll
        for (int c = 13; c < 16; ++c) v[c] = 0.f;
        uint4 o0, o1;
        __nv_bfloat162* h0 = reinterpret_cast<__nv_bfloat162*>(&o0);
        __nv_bfloat162* h1 = reinterpret_cast<__nv_bfloat162*>(&o1);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            h0[c] = __floats2bfloat162_rn(v[2 * c], v[2 * c + 1]);
            h1[c] = __floats2bfloat162_rn(v[8 + 2 * c], v[8 + 2 * c + 1]);
        }
        uint4* dst = reinterpret_cast<uint4*>(X + slot_of(p, n1, n2, R, P) * CH);
        dst[0] = o0;
        dst[1] = o1;
    }
}

// The base the network corrects: u, or the polynomial extrapolation in time
// of the history (2u - u1 with one level, 3u - 3u1 + u2 with two).
__device__ __forceinline__ double guess_base(const double* u, const double* u1, const double* u2, long long p) {
    if (!u1) return u[p];
    if (!u2) return 2.0 * u[p] - u1[p];
    return 3.0 * u[p] - 3.0 * u1[p] + u2[p];
}

// x0 = base + s * out
__global__ void guess_kernel(const double* __restrict__ u, const double* __restrict__ u1,
                             const double* __restrict__ u2, const float* __restrict__ out,
                             const double* __restrict__ scale, long long N, double* __restrict__ x0) {
    const double s = scale[0];
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x)
        x0[p] = guess_base(u, u1, u2, p) + s * (double)out[p];
}

// loss partials and the output gradient: d = out - (u_next - u)/s ; dZ[slot][0] = 2 d / N
__global__ void loss_grad_kernel(const float* __restrict__ out, const double* __restrict__ u,
                                 const double* __restrict__ u1, const double* __restrict__ u2,
                                 const double* __restrict__ un, const double* __restrict__ scale, int n1, int n2,
                                 long long N, long long R, long long P, __nv_bfloat16* __restrict__ dZ,
                                 double* __restrict__ part) {
    __shared__ double sh[256];
    const double inv = 1.0 / scale[0];
    double acc = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        const double d = (double)out[p] - (un[p] - guess_base(u, u1, u2, p)) * inv;
        acc += d * d;
        dZ[slot_of(p, n1, n2, R, P) * CH] = __float2bfloat16_rn((float)(2.0 * d / (double)N));
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// Weight-gradient partials of one tap over a chunk of slots:
//   part[(chunk * 27 + tap) * 256 + co * 16 + ci] = sum_s dZ[s][co] X[s + off][ci]
// (dZ is zero on guard slots, X is zero there by construction).
constexpr int WG_CHUNK = 256;
__global__ __launch_bounds__(256) void wgrad_kernel(const __nv_bfloat16* __restrict__ dZ,
                                                    const __nv_bfloat16* __restrict__ X, long long first,
                                                    long long count, long long R, long long P,
                                                    float* __restrict__ part) {
    __shared__ float sz[WG_CHUNK][CH + 1];
    __shared__ float sx[WG_CHUNK][CH + 1];
    const int tap = blockIdx.y;
    const long long off = (long long)(tap / 9 - 1) * P + (long long)((tap / 3) % 3 - 1) * R + (tap % 3 - 1);
    const long long s0 = first + (long long)blockIdx.x * WG_CHUNK;
    for (int e = threadIdx.x; e < WG_CHUNK * CH; e += 256) {
        const int i = e / CH, c = e % CH;
        const long long s = s0 + i;
        const bool in = s < first + count;
        sz[i][c] = in ? __bfloat162float(dZ[s * CH + c]) : 0.f;
        sx[i][c] = in ? __bfloat162float(X[(s + off) * CH + c]) : 0.f;
    }
    __syncthreads();
    const int co = threadIdx.x >> 4, ci = threadIdx.x & 15;
    float acc = 0.f;
#pragma unroll 8
    for (int i = 0; i < WG_CHUNK; ++i) acc = fmaf(sz[i][co], sx[i][ci], acc);
    part[((long long)blockIdx.x * NTAP + tap) * 256 + threadIdx.x] = acc;
}

// grad[layer W][co][ci][tap] += sum over chunks; grad bias[co] += sum_s dZ[s][co]
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, int nchunks, float* __restrict__ gW) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;   // (tap, co, ci)
    if (idx >= NTAP * 256) return;
    const int tap = idx / 256, co = (idx / 16) % 16, ci = idx % 16;
    double acc = 0.0;
    for (int c = 0; c < nchunks; ++c) acc += part[((long long)c * NTAP + tap) * 256 + co * 16 + ci];
    gW[(co * CH + ci) * NTAP + tap] += (float)acc;
}

__global__ void bgrad_kernel(const __nv_bfloat16* __restrict__ dZ, long long first, long long count,
                             float* __restrict__ gb) {
    __shared__ float sh[256];
    const int c = blockIdx.x;
    float acc = 0.f;
    for (long long i = threadIdx.x; i < count; i += 256) acc += __bfloat162float(dZ[(first + i) * CH + c]);
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) gb[c] += sh[0];
}

// Forward weights [27][2][16][8] (B operand: N = co, K = ci) and input-gradient
// weights (N = ci, K = co, taps mirrored) from the FP32 master [co][ci][27].
__global__ void pack_weights_kernel(const float* __restrict__ Wm, __nv_bfloat16* __restrict__ fwd,
                                    __nv_bfloat16* __restrict__ bwd) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;   // (tap, h, n, k8)
    if (idx >= NTAP * 256) return;
    const int tap = idx / 256, h = (idx / 128) % 2, n = (idx / 8) % 16, k8 = idx % 8;
    const int k = 8 * h + k8;
    fwd[idx] = __float2bfloat16_rn(Wm[(n * CH + k) * NTAP + tap]);                  // W[co = n][ci = k][tap]
    bwd[idx] = __float2bfloat16_rn(Wm[(k * CH + n) * NTAP + (NTAP - 1 - tap)]);     // W[co = k][ci = n][-tap]
}

// Adam on all parameters (grads averaged over `count` samples), grads zeroed.
__global__ void adam_kernel(float* __restrict__ prm, float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2,
                            float inv_count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i] * inv_count;
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    prm[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    grad[i] = 0.f;
}

bool g_attr = false;

}  // namespace cnn
}  // namespace tfde

struct tfde_cnn {
    int n[3] = {};
    long long N = 0, R = 0, P = 0, S_total = 0, first = 0, count = 0, ntiles = 0;
    float* prm = nullptr;      // FP32 master parameters, NL * PSZ
    float* grad = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    int adam_t = 0;
    int accumulated = 0;
    __nv_bfloat16* wf = nullptr;  // packed forward weights, NL * 27*256
    __nv_bfloat16* wb = nullptr;  // packed input-gradient weights
    __nv_bfloat16* act[tfde::cnn::NL] = {};  // layer inputs X0..X3 (padded slots)
    __nv_bfloat16* dz = nullptr;  // gradient buffers (padded slots), two
    __nv_bfloat16* dz2 = nullptr;
    float* out = nullptr;         // network output, plain grid
    float* coef = nullptr;        // 9 input constants (device)
    double* scale = nullptr;
    float* wpart = nullptr;
    double* lpart = nullptr;
    double* lpart_host = nullptr;
    CUtensorMap amap[tfde::cnn::NL];
    CUtensorMap dmap[2];
    int* err = nullptr;
    int* err_host = nullptr;
    bool packed = false;
};

namespace tfde {
namespace cnn {
namespace {

#define CN_TRY(expr)                                                                       \
    do {                                                                                   \
        cudaError_t e__ = (expr);                                                          \
        if (e__ != cudaSuccess)                                                            \
            return set_error(TFDE_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e__)); \
    } while (0)

int make_act_map(CUtensorMap* m, const __nv_bfloat16* base, long long S_total) {
    const cuuint64_t dims[2] = {(cuuint64_t)CH, (cuuint64_t)S_total};
    const cuuint64_t strides[1] = {(cuuint64_t)CH * 2};
    const cuuint32_t box[2] = {8, (cuuint32_t)BOX};
    return tc::encode_map(m, base, 2, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_NONE);
}

int grid1(long long n) {
    long long g = (n + 255) / 256;
    if (g > 152LL * 8) g = 152LL * 8;
    return (int)(g < 1 ? 1 : g);
}

int conv(tfde_cnn* C, const CUtensorMap& amap, const __nv_bfloat16* w, const float* bias, int relu,
         const __nv_bfloat16* mask, __nv_bfloat16* out_act, float* out_f32, cudaStream_t s) {
    if (!g_attr) {
        CN_TRY(cudaFuncSetAttribute(conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
        g_attr = true;
    }
    ConvParams p;
    std::memset(&p, 0, sizeof(p));
    p.amap = amap;
    p.wts = w;
    p.bias = bias;
    p.relu = relu;
    p.mask = mask;
    p.out_act = out_act;
    p.out_f32 = out_f32;
    p.n1 = C->n[0];
    p.n2 = C->n[1];
    p.n3 = C->n[2];
    p.R = C->R;
    p.P = C->P;
    p.first = C->first;
    p.ntiles = C->ntiles;
    p.err = C->err;
    long long grid = C->ntiles < tc::num_sms() ? C->ntiles : tc::num_sms();
    void* tok = stats_tc_begin(s, TFDE_KIND_CONV);
    conv_kernel<<<(unsigned)(grid < 1 ? 1 : grid), NUM_THREADS, SMEM_BYTES, s>>>(p);
    cudaError_t e = cudaGetLastError();
    // algorithmic: the input activations read once, the output written once
    stats_tc_end(tok, s, TFDE_KIND_CONV, 64.0 * (double)C->N, 2.0 * NTAP * CH * CH * (double)C->N);
    if (e != cudaSuccess) return set_error(TFDE_ECUDA, std::string("conv_kernel launch: ") + cudaGetErrorString(e));
    return TFDE_OK;
}

int ensure_packed(tfde_cnn* C, cudaStream_t s) {
    if (C->packed) return TFDE_OK;
    for (int l = 0; l < NL; ++l) {
        stats_count_launch();
        pack_weights_kernel<<<(NTAP * 256 + 255) / 256, 256, 0, s>>>(C->prm + (size_t)l * PSZ,
                                                                        C->wf + (size_t)l * NTAP * 256,
                                                                        C->wb + (size_t)l * NTAP * 256);
    }
    C->packed = true;
    return TFDE_OK;
}

// forward pass of (u, dtF, coef) into C->out (plain grid, output channel 0)
int forward(tfde_cnn* C, const double* u, const double* u1, const double* u2, const double* dtF,
            const double coef[9], cudaStream_t s) {
    float hc[9];
    for (int i = 0; i < 9; ++i) hc[i] = (float)coef[i];
    CN_TRY(cudaMemcpyAsync(C->coef, hc, sizeof(hc), cudaMemcpyHostToDevice, s));
    int st = ensure_packed(C, s);
    if (st) return st;
    stats_count_launch(2);
    maxabs_kernel<<<1, 256, 0, s>>>(u, C->N, C->scale);
    pack_input_kernel<<<grid1(C->N), 256, 0, s>>>(u, u1, u2, dtF, C->scale, C->coef, C->n[0], C->n[1], C->N, C->R,
                                                    C->P, C->act[0]);
    for (int l = 0; l < NL; ++l) {
        const bool last = l + 1 == NL;
        if ((st = conv(C, C->amap[l], C->wf + (size_t)l * NTAP * 256, C->prm + (size_t)l * PSZ + WSZ, last ? 0 : 1,
                       nullptr, last ? nullptr : C->act[l + 1], last ? C->out : nullptr, s)))
            return st;
    }
    return TFDE_OK;
}

int check(tfde_cnn* C, cudaStream_t s) {
    CN_TRY(cudaMemcpyAsync(C->err_host, C->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CN_TRY(cudaStreamSynchronize(s));
    if (*C->err_host) return set_error(TFDE_ETIMEOUT, "warm-start kernel wait ran out (device error flag set)");
    return TFDE_OK;
}

}  // namespace

int cnn_destroy(tfde_cnn* C);

int cnn_create(const int n[3], tfde_cnn** out) {
    *out = nullptr;
    for (int a = 0; a < 3; ++a)
        if (n[a] < 1) return set_error(TFDE_EINVAL, "grid sizes must be >= 1");
    tfde_cnn* C = new tfde_cnn();
    for (int a = 0; a < 3; ++a) C->n[a] = n[a];
    C->N = (long long)n[0] * n[1] * n[2];
    C->R = n[0] + 2;
    C->P = (long long)(n[1] + 2) * C->R;
    C->S_total = (long long)(n[2] + 2) * C->P;
    C->first = C->P + C->R + 1;
    C->count = C->S_total - 2 * C->first;   // slots from the first to the last interior point
    C->ntiles = (C->count + TM - 1) / TM;
    const size_t act_bytes = (size_t)C->S_total * CH * sizeof(__nv_bfloat16);
    const int nchunks = (int)((C->count + WG_CHUNK - 1) / WG_CHUNK);
    bool ok = cudaMalloc((void**)&C->prm, NL * PSZ * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void**)&C->grad, NL * PSZ * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void**)&C->adam_m, NL * PSZ * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void**)&C->adam_v, NL * PSZ * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void**)&C->wf, NL * NTAP * 256 * sizeof(__nv_bfloat16)) == cudaSuccess &&
              cudaMalloc((void**)&C->wb, NL * NTAP * 256 * sizeof(__nv_bfloat16)) == cudaSuccess &&
              cudaMalloc((void**)&C->dz, act_bytes) == cudaSuccess &&
              cudaMalloc((void**)&C->dz2, act_bytes) == cudaSuccess &&
              cudaMalloc((void**)&C->out, C->N * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void**)&C->coef, 16 * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void**)&C->scale, sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&C->wpart, (size_t)nchunks * NTAP * 256 * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void**)&C->lpart, 1216 * sizeof(double)) == cudaSuccess &&
              cudaMallocHost((void**)&C->lpart_host, 1216 * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&C->err, sizeof(int)) == cudaSuccess &&
              cudaMallocHost((void**)&C->err_host, sizeof(int)) == cudaSuccess;
    for (int l = 0; l < NL && ok; ++l) ok = cudaMalloc((void**)&C->act[l], act_bytes) == cudaSuccess;
    if (!ok) {
        cnn_destroy(C);
        return set_error(TFDE_ENOMEM, "allocation of the warm-start network workspace failed");
    }
    // guard slots must stay zero: every buffer on the padded grid starts zeroed
    bool z = cudaMemset(C->dz, 0, act_bytes) == cudaSuccess && cudaMemset(C->dz2, 0, act_bytes) == cudaSuccess &&
             cudaMemset(C->prm, 0, NL * PSZ * sizeof(float)) == cudaSuccess &&
             cudaMemset(C->grad, 0, NL * PSZ * sizeof(float)) == cudaSuccess &&
             cudaMemset(C->adam_m, 0, NL * PSZ * sizeof(float)) == cudaSuccess &&
             cudaMemset(C->adam_v, 0, NL * PSZ * sizeof(float)) == cudaSuccess &&
             cudaMemset(C->err, 0, sizeof(int)) == cudaSuccess;
    for (int l = 0; l < NL && z; ++l) z = cudaMemset(C->act[l], 0, act_bytes) == cudaSuccess;
    if (!z) {
        cnn_destroy(C);
        return set_error(TFDE_ECUDA, "zeroing of the warm-start workspace failed");
    }
    int st = TFDE_OK;
    for (int l = 0; l < NL && !st; ++l) st = make_act_map(&C->amap[l], C->act[l], C->S_total);
    if (!st) st = make_act_map(&C->dmap[0], C->dz, C->S_total);
    if (!st) st = make_act_map(&C->dmap[1], C->dz2, C->S_total);
    if (st) {
        cnn_destroy(C);
        return st;
    }
    *out = C;
    return TFDE_OK;
}

int cnn_destroy(tfde_cnn* C) {
    if (!C) return TFDE_OK;
    cudaDeviceSynchronize();
    cudaFree(C->prm);
    cudaFree(C->grad);
    cudaFree(C->adam_m);
    cudaFree(C->adam_v);
    cudaFree(C->wf);
    cudaFree(C->wb);
    for (auto* a : C->act) cudaFree(a);
    cudaFree(C->dz);
    cudaFree(C->dz2);
    cudaFree(C->out);
    cudaFree(C->coef);
    cudaFree(C->scale);
    cudaFree(C->wpart);
    cudaFree(C->lpart);
    if (C->lpart_host) cudaFreeHost(C->lpart_host);
    cudaFree(C->err);
    if (C->err_host) cudaFreeHost(C->err_host);
    delete C;
    return TFDE_OK;
}

int cnn_set_params(tfde_cnn* C, const float* host) {
    CN_TRY(cudaMemcpy(C->prm, host, NL * PSZ * sizeof(float), cudaMemcpyHostToDevice));
    CN_TRY(cudaMemset(C->grad, 0, NL * PSZ * sizeof(float)));
    CN_TRY(cudaMemset(C->adam_m, 0, NL * PSZ * sizeof(float)));
    CN_TRY(cudaMemset(C->adam_v, 0, NL * PSZ * sizeof(float)));
    C->adam_t = 0;
    C->accumulated = 0;
    C->packed = false;
    return TFDE_OK;
}

int cnn_get(const tfde_cnn* C, int what, float* host) {
    const float* src = what == 0 ? C->prm : C->grad;
    CN_TRY(cudaMemcpy(host, src, NL * PSZ * sizeof(float), cudaMemcpyDeviceToHost));
    return TFDE_OK;
}

int cnn_predict(tfde_cnn* C, const double* u, const double* u1, const double* u2, const double* dtF,
                const double coef[9], double* x0, cudaStream_t s) {
    int st = forward(C, u, u1, u2, dtF, coef, s);
    if (st) return st;
    stats_count_launch();
    guess_kernel<<<grid1(C->N), 256, 0, s>>>(u, u1, u2, C->out, C->scale, C->N, x0);
    return check(C, s);
}

int cnn_accumulate(tfde_cnn* C, const double* u, const double* u1, const double* u2, const double* dtF,
                   const double coef[9], const double* u_next, double* loss, cudaStream_t s) {
    int st = forward(C, u, u1, u2, dtF, coef, s);
    if (st) return st;
    const int nb = grid1(C->N);
    stats_count_launch();
    CN_TRY(cudaMemsetAsync(C->dz, 0, (size_t)C->S_total * CH * sizeof(__nv_bfloat16), s));
    loss_grad_kernel<<<nb, 256, 0, s>>>(C->out, u, u1, u2, u_next, C->scale, C->n[0], C->n[1], C->N, C->R, C->P,
                                         C->dz, C->lpart);
    const int nchunks = (int)((C->count + WG_CHUNK - 1) / WG_CHUNK);
    __nv_bfloat16* g = C->dz;      // gradient w.r.t. the output of layer l (pre-activation for l < NL - 1 after masking)
    __nv_bfloat16* g2 = C->dz2;
    int gm = 0;
    for (int l = NL - 1; l >= 0; --l) {
        float* gW = C->grad + (size_t)l * PSZ;
        stats_count_launch(3);
        wgrad_kernel<<<dim3((unsigned)nchunks, NTAP), 256, 0, s>>>(g, C->act[l], C->first, C->count, C->R, C->P,
                                                                  C->wpart);
        wgrad_reduce_kernel<<<(NTAP * 256 + 255) / 256, 256, 0, s>>>(C->wpart, nchunks, gW);
        bgrad_kernel<<<CH, 256, 0, s>>>(g, C->first, C->count, gW + WSZ);
        if (l > 0) {
            // gradient w.r.t. the input of layer l, masked by the ReLU of layer l - 1
            if ((st = conv(C, C->dmap[gm], C->wb + (size_t)l * NTAP * 256, nullptr, 0, C->act[l], g2, nullptr, s)))
                return st;
            std::swap(g, g2);
            gm ^= 1;
        }
    }
    C->accumulated++;
    CN_TRY(cudaMemcpyAsync(C->lpart_host, C->lpart, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    if ((st = check(C, s))) return st;
    double acc = 0.0;
    for (int b = 0; b < nb; ++b) acc += C->lpart_host[b];
    if (loss) *loss = acc / (double)C->N;
    return TFDE_OK;
}

int cnn_adam(tfde_cnn* C, float lr, cudaStream_t s) {
    if (C->accumulated == 0) return TFDE_OK;
    C->adam_t++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)C->adam_t), c2 = 1.f - std::pow(b2, (float)C->adam_t);
    const int n = NL * PSZ;
    stats_count_launch();
    adam_kernel<<<(n + 255) / 256, 256, 0, s>>>(C->prm, C->grad, C->adam_m, C->adam_v, n, lr, b1, b2, 1e-8f, c1, c2,
                                                1.f / (float)C->accumulated);
    C->accumulated = 0;
    C->packed = false;
    return check(C, s);
}

}  // namespace cnn
}  // namespace tfde
