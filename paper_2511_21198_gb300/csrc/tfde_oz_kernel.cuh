// Exact-integer slice contraction on tcgen05 (an Ozaki-type splitting) for the
// FP64-accurate apply of one dense per-axis operator G of Eq. (linear_sys):
//
//   out[m, l] = sign * sum_k G[m, k] x[k, l] + addend[m, l]
//
// Row m of G is written as 2^{es[m]} * sum_s g_s[m, :] 2^{-7(s+1)} and line l
// of x as 2^{el[l]} * sum_t x_t[:, l] 2^{-7(t+1)}, with balanced base-128
// digits (|g_0|, |x_0| <= 128, the others <= 64): exact integers in BF16.  For
// every digit pair with s + t <= D the tensor core sums 256 products of at most
// 2^14 in FP32, and a diagonal d = s + t holds at most 2^23 in magnitude, so
// each of the D + 1 accumulators (one per diagonal, in TMEM) is an exact
// integer.  The epilogue recombines the diagonals in 64-bit integers and
// applies the power-of-two scales, giving the contraction with an absolute
// error of about 2^{-7(D+1)} |G| |x| per entry.
//
// One CTA per SM, persistent over tiles of 128 rows x 64 lines; warp 0 TMA,
// warp 1 TMEM allocation + MMA issue (M=128, N=64, K=16), warps 2..5 epilogue.
// Bounded waits as in the split-BF16 kernel.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>

namespace tfde {
namespace oz {

constexpr int BM = 128;
constexpr int BN = 64;
constexpr int BK = 32;
constexpr int MAXS = 7;          // digit slices per operand (D + 1, D <= 6)
constexpr int STAGES = 2;
constexpr int A_TILE_BYTES = BM * BK * 2;                        // 8 KB
constexpr int B_TILE_BYTES = BN * BK * 2;                        // 4 KB
constexpr int STAGE_BYTES = MAXS * (A_TILE_BYTES + B_TILE_BYTES);  // 84 KB
constexpr int NUM_THREADS = 192;
constexpr int EPI_WARPS = 4;
constexpr int NUM_BARS = 2 * STAGES + 3;
constexpr int SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + NUM_BARS * 8 + 16;
constexpr uint32_t TMEM_COLS = 512;                              // (D + 1) x 64 <= 448 columns used
static_assert(SMEM_BYTES <= 232448, "shared memory budget of one CTA");

struct Params {
    CUtensorMap amaps[MAXS];   // operator digit slices g_s: BF16 [n][n], K-major, box {32, 128}, 64B swizzle
    CUtensorMap bmaps[MAXS];   // vector digit slices x_t: x axis box {32, 64} (64B swizzle); y/z {64, 32, 1} (128B)
    int nslices;               // D + 1
    int b_kmajor;
    int mhalves;
    int n;
    long long lines;
    int C, nbc, P;
    long long nblocks;
    long long ntiles;
    int n1;
    long long plane;
    const int* row_exp;        // es[m]
    const int* line_exp;       // el[l], l = line index (x axis: j + n2 k; y: i + n1 k; z: i + n1 j)
    double sign;
    const double* addend;      // may be null
    double* out;
    int* err;
};

#ifdef TFDE_OZ_KERNEL_IMPL
}  // namespace oz
}  // namespace tfde
#include "tfde_tc_ptx.cuh"
namespace tfde {
namespace oz {

using namespace tfde::tc;

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 2^e as a double for -1022 <= e <= 1023, built from its bit pattern.
__device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

__global__ void __launch_bounds__(NUM_THREADS, 1) oz_gemm_kernel(const __grid_constant__ Params p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* stages = smem;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    uint64_t* full = bars;
    uint64_t* empty = bars + STAGES;
    uint64_t* tfull = bars + 2 * STAGES;
    uint64_t* tempty = bars + 2 * STAGES + 1;
    uint64_t* mma_done = bars + 2 * STAGES + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + NUM_BARS);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int S = p.nslices;
    const int D = S - 1;
    const int nkb = (p.n + BK - 1) / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(tfull, 1);
        mbar_init(tempty, EPI_WARPS);
        mbar_init(mma_done, 1);
        mbar_fence_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const long long total = p.ntiles * p.mhalves;

    if (warp == 0) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0, filled = 0, last_ph = 0;
            bool ok = true;
            for (long long t = blockIdx.x; t < total && ok; t += gridDim.x) {
                const long long tile = t / p.mhalves;
                const int mh = (int)(t % p.mhalves);
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!mbar_wait(&empty[s], ph ^ 1u, p.err)) { ok = false; break; }
                    uint8_t* st = stages + s * STAGE_BYTES;
                    mbar_expect_tx(&full[s], (uint32_t)(S * (A_TILE_BYTES + B_TILE_BYTES)));
                    for (int a = 0; a < S; ++a)
                        tma_load_2d(st + a * A_TILE_BYTES, &p.amaps[a], &full[s], kb * BK, mh * BM);
                    for (int b = 0; b < S; ++b) {
                        uint8_t* dst = st + MAXS * A_TILE_BYTES + b * B_TILE_BYTES;
                        if (p.b_kmajor) {
                            tma_load_2d(dst, &p.bmaps[b], &full[s], kb * BK, (int)(tile * BN));
                        } else {
                            const int pl = (int)(tile / p.nbc);
                            const int c0 = (int)(tile % p.nbc) * 64;
                            tma_load_3d(dst, &p.bmaps[b], &full[s], c0, kb * BK, pl);
                        }
                    }
                    filled |= 1u << s;
                    if (ph) last_ph |= 1u << s; else last_ph &= ~(1u << s);
                    if (++s == STAGES) { s = 0; ph ^= 1u; }
                }
            }
            for (int i = 0; i < STAGES; ++i)
                if (filled & (1u << i)) mbar_wait(&full[i], (last_ph >> i) & 1u, p.err, false);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = instr_desc(BM, BN, p.b_kmajor ? 0 : 1);
            int s = 0;
            uint32_t ph = 0;
            bool ok = true;
            long long it = 0;
            for (long long t = blockIdx.x; t < total && ok; t += gridDim.x, ++it) {
                if (!mbar_wait(tempty, ((uint32_t)it & 1u) ^ 1u, p.err)) { ok = false; break; }
                tc_fence_after();
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!mbar_wait(&full[s], ph, p.err)) { ok = false; break; }
                    tc_fence_after();
                    const uint8_t* st = stages + s * STAGE_BYTES;
                    for (int sa = 0; sa < S; ++sa) {
                        const uint32_t a_addr = smem_u32(st + sa * A_TILE_BYTES);
                        for (int tb = 0; tb + sa <= D; ++tb) {
                            const uint32_t b_addr = smem_u32(st + MAXS * A_TILE_BYTES + tb * B_TILE_BYTES);
                            const uint32_t d_tmem = tmem_base + (uint32_t)((sa + tb) * BN);
#pragma unroll
                            for (int k16 = 0; k16 < BK / 16; ++k16) {
                                const uint64_t ad = smem_desc(a_addr + k16 * 32, 16, 512, 4);
                                const uint64_t bd = p.b_kmajor ? smem_desc(b_addr + k16 * 32, 16, 512, 4)
                                                               : smem_desc(b_addr + k16 * 2048, 4096, 1024, 2);
                                // the first product into each diagonal (s = 0, kb = 0, k16 = 0) overwrites it
                                umma_bf16(d_tmem, ad, bd, idesc, (kb > 0 || sa > 0 || k16 > 0) ? 1u : 0u);
                            }
                        }
                    }
                    umma_commit(&empty[s]);
                    if (++s == STAGES) { s = 0; ph ^= 1u; }
                }
                if (ok) umma_commit(tfull);
            }
            umma_commit(mma_done);
            mbar_wait(mma_done, 0, p.err, false);
        }
    } else {
        const int q = warp & 3;
        const int split = D >= 3 ? 3 : S;   // diagonals [0, split) -> hi part, [split, S) -> lo part
        long long it = 0;
        for (long long t = blockIdx.x; t < total; t += gridDim.x, ++it) {
            int ok = 1;
            if (lane == 0) ok = mbar_wait(tfull, (uint32_t)it & 1u, p.err) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            __syncwarp();
            tc_fence_after();
            const long long tile = t / p.mhalves;
            const int mh = (int)(t % p.mhalves);
            const int m = mh * BM + 32 * q + lane;
            const int es = (m < p.n) ? __ldg(p.row_exp + m) : 0;
            const double hi_scale = pow2(7 * (S - split));
            for (int c0 = 0; c0 < BN; c0 += 8) {
                uint32_t r[MAXS][8];
#pragma unroll
                for (int d = 0; d < MAXS; ++d)
                    if (d < S) tmem_ld8(tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(d * BN + c0), r[d]);
                tmem_wait_ld();
                if (m < p.n) {
                    long long ihi[8], ilo[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) ihi[j] = ilo[j] = 0;
#pragma unroll
                    for (int d = 0; d < MAXS; ++d) {
                        if (d >= S) break;
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const long long v = (long long)__float2int_rn(__uint_as_float(r[d][j]));
                            if (d < split) ihi[j] = ihi[j] * 128 + v;
                            else ilo[j] = ilo[j] * 128 + v;
                        }
                    }
                    long long base, lbase;
                    int cbase = 0;
                    if (p.b_kmajor) {
                        lbase = tile * BN + c0;            // line index of column c0
                        base = lbase * p.n1 + m;           // column j at + j * n1
                    } else {
                        const int pl = (int)(tile / p.nbc);
                        cbase = (int)(tile % p.nbc) * 64 + c0;
                        lbase = (long long)pl * p.C + cbase;
                        base = (long long)pl * p.plane + (long long)m * p.C + cbase;   // column j at + j
                    }
                    const double row_scale = p.sign * pow2(es - 7 * (D + 2));
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const bool valid = p.b_kmajor ? (lbase + j < p.lines) : (tile < p.nblocks && cbase + j < p.C);
                        if (!valid) continue;
                        const int el = __ldg(p.line_exp + lbase + j);
                        const double v = fma((double)ihi[j], hi_scale, (double)ilo[j]);
                        const long long idx = p.b_kmajor ? base + (long long)j * p.n1 : base + j;
                        double o = v * row_scale * pow2(el);
                        if (p.addend) o += p.addend[idx];
                        p.out[idx] = o;
                    }
                }
                __syncwarp();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty);
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem_base, TMEM_COLS);
}

#endif  // TFDE_OZ_KERNEL_IMPL

}  // namespace oz
}  // namespace tfde
