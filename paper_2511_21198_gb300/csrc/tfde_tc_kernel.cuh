// tcgen05 (5th-generation tensor core) per-axis contraction for sm_103a.
//
//   Y[m, l] = alpha * sum_{segments} sum_{pairs (a, b)} A_a[m, :] . B_b[:, l]
//
// m runs along one grid axis (the operator's rows), l over the lines of the
// grid function along that axis; A_a are small BF16 operator matrices (the
// split-BF16 parts of eta B, the mass stencil, the DST-I matrix) and B_b BF16
// planes of the operand vector.  This is the dense per-axis contraction of
// Eq. (linear_sys) / Eq. (diag_tau_pre) with the line batch as the GEMM N
// dimension.
//
// Design (one CTA per SM, persistent over tiles of 128 rows x 256 lines):
//   warp 0      TMA producer: A tiles [128 x 32] (K-major, 64B swizzle) and
//               B tiles [32 x 256] (x axis: K-major 64B swizzle; y/z axes:
//               MN-major 128B swizzle, 4 boxes of 64 lines) into a 4-stage ring
//   warp 1      allocates TMEM (2 x 256 FP32 columns) and issues tcgen05.mma
//               (M=128, N=256, K=16, BF16 in, FP32 accumulate) from one thread
//   warps 2..5  epilogue: tcgen05.ld from TMEM, scale, optional Lambda^{-1},
//               store FP32 or split BF16 (hi, lo) with coalesced stores
// Every wait on an mbarrier is bounded by a wall-clock limit; on timeout the
// kernel raises *err, stops issuing work, waits (bounded) for its own copies
// and MMAs in flight, frees its TMEM and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>

namespace tfde {
namespace tc {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int BK = 32;
constexpr int STAGES = 4;
constexpr int MAXA = 2;
constexpr int MAXB = 2;
constexpr int MAXSEG = 2;
constexpr int MAXPAIR = 4;
constexpr int A_TILE_BYTES = BM * BK * 2;                                  // 8 KB
constexpr int B_TILE_BYTES = BN * BK * 2;                                  // 16 KB
constexpr int STAGE_BYTES = MAXA * A_TILE_BYTES + MAXB * B_TILE_BYTES;     // 48 KB
constexpr int NUM_THREADS = 192;
constexpr int EPI_WARPS = 4;
constexpr int EPI_STRIDE = 33;
constexpr int EPI_FLOATS = EPI_WARPS * 32 * EPI_STRIDE;
constexpr int NUM_BARS = 2 * STAGES + 5;
constexpr int SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + EPI_FLOATS * 4 + NUM_BARS * 8 + 16;
constexpr uint32_t TMEM_COLS = 2 * BN;
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;  // 2 s

struct Segment {
    int nkb;                     // k-blocks of BK in this segment
    int na, nb;                  // A / B terms loaded per stage
    int amap[MAXA], bmap[MAXB];  // tensor-map indices
    int npair;
    int pa[MAXPAIR], pb[MAXPAIR];
};

enum { OUT_F32 = 0, OUT_HILO = 1 };

struct Params {
    CUtensorMap amaps[4];
    CUtensorMap bmaps[4];
    Segment seg[MAXSEG];
    int nseg;
    int b_kmajor;        // 1: B stored with k contiguous (x axis); 0: lines contiguous (y, z axes)
    int mhalves;         // ceil(n / 128)
    int n;               // valid rows along the axis
    long long lines;     // valid lines (K-major case)
    int C, nbc, P;       // MN-major: contiguous line extent per plane, 64-blocks per plane, planes
    long long nblocks;   // MN-major: nbc * P
    long long ntiles;    // line tiles of BN
    int n1;              // K-major output: Y[l * n1 + m]
    long long plane;     // MN-major output plane stride (C * n)
    int out_mode;
    float alpha;
    float* out_f32;
    __nv_bfloat16* out_hi;
    __nv_bfloat16* out_lo;
    // optional scale 1 / (ra[m] U[c] + rb[m] V[c]) (z-axis DST pass, MN-major only)
    const float* lam_ra;
    const float* lam_rb;
    const float* lam_U;
    const float* lam_V;
    int* err;
};

#ifdef TFDE_TC_KERNEL_IMPL
// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait.  Returns false when the wait gave up (time limit, or another
// role raised *err and `abort_on_err`).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, bool abort_on_err = true) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (abort_on_err && *reinterpret_cast<volatile int*>(err) != 0) return false;
        if (global_ns() - t0 > WAIT_LIMIT_NS) {
            atomicExch(err, 1);
            return false;
        }
    }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor (tcgen05): start address, leading / stride
// byte offsets (16-byte units), descriptor version 1, swizzle layout code
// (0 none, 2 = 128B, 4 = 64B, 6 = 32B).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)(layout & 7u) << 61;
    return d;
}
// Instruction descriptor for kind::f16: FP32 accumulator, BF16 A and B,
// A K-major, B K-major (0) or MN-major (1), N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N, int b_mn_major) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)b_mn_major << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void store_out(const Params& p, long long idx, float v) {
    if (p.out_mode == OUT_F32) {
        p.out_f32[idx] = v;
    } else {
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        p.out_hi[idx] = hi;
        p.out_lo[idx] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
}

// ---------------------------------------------------------------------- kernel
__global__ void __launch_bounds__(NUM_THREADS, 1) axis_gemm_kernel(const __grid_constant__ Params p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* stages = smem;
    float* epi = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES);
    uint64_t* bars = reinterpret_cast<uint64_t*>(epi + EPI_FLOATS);
    uint64_t* full = bars;
    uint64_t* empty = bars + STAGES;
    uint64_t* tfull = bars + 2 * STAGES;
    uint64_t* tempty = bars + 2 * STAGES + 2;
    uint64_t* mma_done = bars + 2 * STAGES + 4;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + NUM_BARS);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], EPI_WARPS);
        }
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
            // ------------------------------------------------ TMA producer
            int s = 0;
            uint32_t ph = 0;
            uint32_t filled = 0, last_ph = 0;  // per-stage bitmasks
            bool ok = true;
            for (long long t = blockIdx.x; t < total && ok; t += gridDim.x) {
                const long long tile = t / p.mhalves;
                const int mh = (int)(t % p.mhalves);
                for (int sg = 0; sg < p.nseg && ok; ++sg) {
                    const Segment& S = p.seg[sg];
                    for (int kb = 0; kb < S.nkb; ++kb) {
                        if (!mbar_wait(&empty[s], ph ^ 1u, p.err)) { ok = false; break; }
                        uint8_t* st = stages + s * STAGE_BYTES;
                        mbar_expect_tx(&full[s], (uint32_t)(S.na * A_TILE_BYTES + S.nb * B_TILE_BYTES));
                        for (int a = 0; a < S.na; ++a)
                            tma_load_2d(st + a * A_TILE_BYTES, &p.amaps[S.amap[a]], &full[s], kb * BK, mh * BM);
                        for (int b = 0; b < S.nb; ++b) {
                            uint8_t* dst = st + MAXA * A_TILE_BYTES + b * B_TILE_BYTES;
                            if (p.b_kmajor) {
                                tma_load_2d(dst, &p.bmaps[S.bmap[b]], &full[s], kb * BK, (int)(tile * BN));
                            } else {
                                for (int blk = 0; blk < BN / 64; ++blk) {
                                    const long long gb = tile * (BN / 64) + blk;
                                    const int pl = (int)(gb / p.nbc);
                                    const int c0 = (int)(gb % p.nbc) * 64;
                                    tma_load_3d(dst + blk * (64 * BK * 2), &p.bmaps[S.bmap[b]], &full[s], c0,
                                                kb * BK, pl);
                                }
                            }
                        }
                        filled |= 1u << s;
                        if (ph) last_ph |= 1u << s; else last_ph &= ~(1u << s);
                        if (++s == STAGES) { s = 0; ph ^= 1u; }
                    }
                }
            }
            // drain: every issued copy must land before the CTA can exit
            for (int i = 0; i < STAGES; ++i)
                if (filled & (1u << i)) mbar_wait(&full[i], (last_ph >> i) & 1u, p.err, false);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------------------------ MMA issuer
            const uint32_t idesc = instr_desc(BM, BN, p.b_kmajor ? 0 : 1);
            int s = 0;
            uint32_t ph = 0;
            bool ok = true;
            long long it = 0;
            for (long long t = blockIdx.x; t < total && ok; t += gridDim.x, ++it) {
                const int buf = (int)(it & 1);
                const uint32_t use = (uint32_t)(it >> 1);
                if (!mbar_wait(&tempty[buf], (use & 1u) ^ 1u, p.err)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(buf * BN);
                uint32_t acc = 0;
                for (int sg = 0; sg < p.nseg && ok; ++sg) {
                    const Segment& S = p.seg[sg];
                    for (int kb = 0; kb < S.nkb; ++kb) {
                        if (!mbar_wait(&full[s], ph, p.err)) { ok = false; break; }
                        tc_fence_after();
                        const uint8_t* st = stages + s * STAGE_BYTES;
                        for (int pr = 0; pr < S.npair; ++pr) {
                            const uint32_t a_addr = smem_u32(st + S.pa[pr] * A_TILE_BYTES);
                            const uint32_t b_addr = smem_u32(st + MAXA * A_TILE_BYTES + S.pb[pr] * B_TILE_BYTES);
#pragma unroll
                            for (int k16 = 0; k16 < BK / 16; ++k16) {
                                const uint64_t ad = smem_desc(a_addr + k16 * 32, 16, 512, 4);
                                const uint64_t bd = p.b_kmajor ? smem_desc(b_addr + k16 * 32, 16, 512, 4)
                                                               : smem_desc(b_addr + k16 * 2048, 64 * BK * 2, 1024, 2);
                                umma_bf16(d_tmem, ad, bd, idesc, acc);
                                acc = 1;
                            }
                        }
                        umma_commit(&empty[s]);
                        if (++s == STAGES) { s = 0; ph ^= 1u; }
                    }
                }
                if (ok) umma_commit(&tfull[buf]);
            }
            // every MMA issued by this thread has completed once mma_done fires
            umma_commit(mma_done);
            mbar_wait(mma_done, 0, p.err, false);
        }
    } else {
        // ---------------------------------------------------- epilogue warps
        const int q = warp & 3;  // TMEM lane quadrant this warp may access
        float* stg = epi + (warp - 2) * 32 * EPI_STRIDE;
        long long it = 0;
        for (long long t = blockIdx.x; t < total; t += gridDim.x, ++it) {
            const int buf = (int)(it & 1);
            const uint32_t use = (uint32_t)(it >> 1);
            int ok = 1;
            if (lane == 0) ok = mbar_wait(&tfull[buf], use & 1u, p.err) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;  // warp-uniform: the TMEM loads below are .sync.aligned
            __syncwarp();
            tc_fence_after();
            const long long tile = t / p.mhalves;
            const int mh = (int)(t % p.mhalves);
            const int mrow0 = mh * BM + 32 * q;
            const int m = mrow0 + lane;
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t r[32];
                tmem_ld32(tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * BN + c0), r);
                if (p.b_kmajor) {
                    const long long l0 = tile * BN + c0;
                    if (m < p.n) {
#pragma unroll 8
                        for (int j = 0; j < 32; ++j) {
                            const long long l = l0 + j;
                            if (l < p.lines) store_out(p, l * p.n1 + m, p.alpha * __uint_as_float(r[j]));
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) stg[lane * EPI_STRIDE + j] = __uint_as_float(r[j]);
                    __syncwarp();
                    const long long gb = tile * (BN / 64) + c0 / 64;
                    const int pl = (int)(gb / p.nbc);
                    const int c = (int)(gb % p.nbc) * 64 + (c0 & 63) + lane;
                    if (gb < p.nblocks && c < p.C) {
                        float U = 0.f, V = 0.f;
                        if (p.lam_ra) {
                            U = p.lam_U[c];
                            V = p.lam_V[c];
                        }
                        for (int rr = 0; rr < 32; ++rr) {
                            const int mr = mrow0 + rr;
                            if (mr >= p.n) break;
                            float v = p.alpha * stg[rr * EPI_STRIDE + lane];
                            if (p.lam_ra) v = v / (p.lam_ra[mr] * U + p.lam_rb[mr] * V);
                            store_out(p, (long long)pl * p.plane + (long long)mr * p.C + c, v);
                        }
                    }
                    __syncwarp();
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem_base, TMEM_COLS);
}

#endif  // TFDE_TC_KERNEL_IMPL

}  // namespace tc
}  // namespace tfde
