// tcgen05 (5th-generation tensor core) per-axis contraction for sm_103a.
//
//   Y[m, l] = alpha * sum_{segments} sum_{pairs (a, b)} A_a[m, :] . B_b[:, l]
//
// m runs along one grid axis (the operator's rows), l over the lines of the
// grid function along that axis; A_a are small BF16 operator matrices (the
// split-BF16 parts of eta B, the mass matrix, the DST-I matrix) and B_b BF16
// planes of the operand vector.  This is the dense per-axis contraction of
// Eq. (linear_sys) / Eq. (diag_tau_pre) with the line batch as the GEMM N
// dimension.
//
// Design (one CTA per SM, persistent over tiles of 128 rows x 256 lines):
//   warps 0..2  TMA producers: A tiles [128 x 64] (K-major, 128B swizzle; the
//               hi and lo terms of a split operator in one 3-D box) and B
//               tiles [64 x 256] (x axis: K-major 128B swizzle; y/z axes:
//               MN-major 128B swizzle, 4 line blocks of 64 in one box with
//               both planes) into a ring of 192 KB: 2 stages of 96 KB when a
//               segment carries two operator terms and two planes, 4 stages
//               of 48 KB for one term and one plane.  A stage moves 48-96 KB
//               in two copies: the issue cost of a copy (~0.2-0.4 us, measured
//               by an in-kernel timeline) is paid per copy, not per byte, so
//               64-wide k-blocks halve it against 32-wide ones.  The boxes of
//               a stage are dealt round-robin to the issuing threads.
//   warp 3      allocates TMEM (2 x 256 FP32 columns) and issues tcgen05.mma
//               (M=128, N=256, K=16, BF16 in, FP32 accumulate) from one thread
//   warps 4..11 epilogue, two warps per TMEM lane quadrant (one per half of the
//               256 columns), per 32 x 32 chunk: tcgen05.ld, scale, optional
//               Lambda^{-1}, direction update and fused inner products, the
//               chunk written to a swizzled shared-memory slot and sent to
//               global memory by one TMA tensor store per output plane (the
//               tensor map clips rows and columns beyond the grid)
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>

namespace tfde {
namespace tc {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int BK = 32;             // k-block of the exact-slice contraction's operator maps (tfde_oz.cu)
constexpr int SK = 64;             // k-block of this contraction: 128-byte rows of 64 BF16
constexpr int MAXA = 2;
constexpr int MAXB = 2;
constexpr int MAXSEG = 2;
constexpr int MAXPAIR = 4;
constexpr int A_TILE_BYTES = BM * SK * 2;                                  // 16 KB
constexpr int B_TILE_BYTES = BN * SK * 2;                                  // 32 KB
constexpr int RING_BYTES = 2 * (MAXA * A_TILE_BYTES + MAXB * B_TILE_BYTES);  // 192 KB
constexpr int MAX_STAGES = 4;
constexpr int EPI_WARPS = 8;
constexpr int PRODUCERS = 3;           // TMA issuing warps: one box per thread is issued at a time,
constexpr int MMA_WARP = PRODUCERS;    // so several issuers keep more copies in flight
constexpr int EPI_WARP0 = PRODUCERS + 1;
constexpr int NUM_THREADS = 32 * (PRODUCERS + 1 + EPI_WARPS);             // 384: 12 warps (a 13th would cap registers at 128)
constexpr int EPI_SLOT_BYTES = 4096;   // per epilogue warp: one 32 x 32 FP32 chunk, or hi + lo BF16 chunks
constexpr int NUM_BARS = 2 * MAX_STAGES + 5;
constexpr int SMEM_BYTES = 1024 + RING_BYTES + EPI_WARPS * EPI_SLOT_BYTES + NUM_BARS * 8 + 16;
constexpr uint32_t TMEM_COLS = 2 * BN;
static_assert(SMEM_BYTES <= 232448, "shared memory budget of one CTA");

struct Segment {
    int nkb;                     // k-blocks of BK in this segment
    int na, nb;                  // A / B terms loaded per stage
    int amap[MAXA], bmap[MAXB];  // tensor-map indices, one box per term
    int amap2;                   // >= 0: one 3-D box {BK, BM, na} loads all A terms (stored contiguously)
    int bmap2;                   // >= 0: one box loads both B planes (and, on y/z, all BN/64 line blocks)
    int npair;
    int pa[MAXPAIR], pb[MAXPAIR];
};

// OUT_XPAY: p = Y + beta p_old (beta = *xp_num / *xp_den, 0 when xp_den is
// null), written both as FP32 (out_f32) and as the split planes (out_hi,
// out_lo): the CG direction update fused into the last pass of the
// preconditioner.  p_old is xp_old, or out_f32 itself (in place).
// OUT_HI: the BF16 rounding of Y alone (out_hi), for consumers that read
// only the hi plane.
// OUT_SUM: FP32 output (out_f32) of addend + cs[line] Y, optionally dotted
// with dot_vec into *dot_out, cs the per-line factor col_scale (1 when
// null), addend optional: one axis term of
// a Kronecker sum with diagonal factors on the other axes, accumulated pass
// by pass (the operator in the sine-transform eigenbasis); on the z axis
// with lam_ra set, the result is divided by Lambda (the preconditioned
// operator of left-preconditioned GMRES).
enum { OUT_F32 = 0, OUT_HILO = 1, OUT_XPAY = 2, OUT_HI = 3, OUT_SUM = 4 };

struct Params {
    CUtensorMap amaps[4];
    CUtensorMap bmaps[4];
    // output tensor maps (box 32 x 32): FP32 vector, hi plane, lo plane;
    // x axis: {n1, lines}, no swizzle; y/z axes: {C, n, P}, 128B (FP32) /
    // 64B (BF16) swizzle
    CUtensorMap omap_f32, omap_hi, omap_hl;   // FP32 output, hi plane, hi and lo planes as one tensor
    Segment seg[MAXSEG];
    int nseg;
    int b_kmajor;        // 1: B stored with k contiguous (x axis); 0: lines contiguous (y, z axes)
    int b_rank;          // rank of the bmap2 box: 3 (x axis), 5 (y/z axes: blocks, plane, hi/lo)
    int mhalves;         // ceil(n / 128)
    int n;               // valid rows along the axis
    long long lines;     // valid lines (K-major case)
    int C, nbc, P;       // MN-major: contiguous line extent per plane, 64-blocks per plane, planes
    long long nblocks;   // MN-major: nbc * P
    long long ntiles;    // line tiles of BN
    int n1;              // K-major output: Y[l * n1 + m]
    long long plane;     // MN-major output plane stride (C * n)
    int out_mode;
    int nstages;         // ring stages (2 or 4) and their geometry: A terms at 0, B planes at stage_b_off
    int stage_bytes;
    int stage_b_off;
    float alpha;
    float* out_f32;
    __nv_bfloat16* out_hi;
    __nv_bfloat16* out_lo;
    // optional scale 1 / (ra[m] U[c] + rb[m] V[c]) (z-axis DST pass, MN-major only)
    const float* lam_ra;
    const float* lam_rb;
    const float* lam_U;
    const float* lam_V;
    // optional fused inner product (OUT_F32, OUT_SUM): *dot_out += sum out[i] dot_vec[i];
    // a grouped launch adds each group's sum into that group's dot_out
    const float* dot_vec;
    double* dot_out;
    // optional, with lam_ra (z-axis DST pass): *dot_out += sum t[i] (t / Lambda)[i],
    // t the pass's output before the Lambda^{-1} scale: <r, S Lambda^{-1} S r>
    int dot_lam;
    const double* xp_num;   // OUT_XPAY: beta = *xp_num / *xp_den
    const double* xp_den;
    const float* xp_old;    // OUT_XPAY: the old p (null: out_f32 itself, updated in place)
    // OUT_SUM: per-line factor (indexed by the output's line) and an FP32
    // addend in the output's layout
    const float* col_scale;
    const float* addend;
    const int* skip;        // optional: a launch that finds *skip != 0 does no work (device-side loops)
    int* err;
};

#ifdef TFDE_TC_KERNEL_IMPL
}  // namespace tc
}  // namespace tfde
#include "tfde_tc_ptx.cuh"
namespace tfde {
namespace tc {

// Compensated FP32 sum of the fused inner product (one per epilogue thread).
struct DotAcc {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// The 32 values of this thread (row `lane` of a 32 x 32 chunk, columns 0..31)
// into an epilogue slot in the layout of the output tensor map's box:
// x axis (K-major output, element (line, m) at line * 32 + m, rows of 32 m),
// no swizzle -- a warp writes one contiguous row per column; y / z axes
// (MN-major output, element (m, c) at m * 32 + c), swizzled so that the
// 16-byte chunks of 8 consecutive rows fall in distinct banks (FP32: 128-byte
// rows, chunk ^= row & 7; BF16: 64-byte rows, chunk ^= (row >> 1) & 3).
template <bool KMAJ>
__device__ __forceinline__ void slot_f32(uint8_t* slot, int lane, const float (&v)[32]) {
    if constexpr (KMAJ) {
        float* f = reinterpret_cast<float*>(slot);
#pragma unroll
        for (int j = 0; j < 32; ++j) f[j * 32 + lane] = v[j];
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            *reinterpret_cast<float4*>(slot + lane * 128 + ((k ^ (lane & 7)) << 4)) =
                make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    }
}
template <bool KMAJ>
__device__ __forceinline__ void slot_bf16(uint8_t* slot, int lane, const float (&v)[32]) {
    if constexpr (KMAJ) {
        __nv_bfloat16* h = reinterpret_cast<__nv_bfloat16*>(slot);
#pragma unroll
        for (int j = 0; j < 32; ++j) h[j * 32 + lane] = __float2bfloat16_rn(v[j]);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint4 w;
            w.x = pack_bf16(v[8 * k], v[8 * k + 1]);
            w.y = pack_bf16(v[8 * k + 2], v[8 * k + 3]);
            w.z = pack_bf16(v[8 * k + 4], v[8 * k + 5]);
            w.w = pack_bf16(v[8 * k + 6], v[8 * k + 7]);
            *reinterpret_cast<uint4*>(slot + lane * 64 + ((k ^ ((lane >> 1) & 3)) << 4)) = w;
        }
    }
}

// hi = bf16(v) into slot_hi and lo = bf16(v - hi) into slot_lo, same layout.
template <bool KMAJ>
__device__ __forceinline__ void slot_bf16_pair(uint8_t* slot_hi, uint8_t* slot_lo, int lane, const float (&v)[32]) {
    if constexpr (KMAJ) {
        __nv_bfloat16* h = reinterpret_cast<__nv_bfloat16*>(slot_hi);
        __nv_bfloat16* l = reinterpret_cast<__nv_bfloat16*>(slot_lo);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const __nv_bfloat16 hj = __float2bfloat16_rn(v[j]);
            h[j * 32 + lane] = hj;
            l[j * 32 + lane] = __float2bfloat16_rn(v[j] - __bfloat162float(hj));
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[8 * k + 2 * e], v[8 * k + 2 * e + 1]);
                const float2 f2 = __bfloat1622float2(h2);
                const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[8 * k + 2 * e] - f2.x, v[8 * k + 2 * e + 1] - f2.y);
                hw[e] = *reinterpret_cast<const uint32_t*>(&h2);
                lw[e] = *reinterpret_cast<const uint32_t*>(&l2);
            }
            const int off = lane * 64 + ((k ^ ((lane >> 1) & 3)) << 4);
            *reinterpret_cast<uint4*>(slot_hi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4*>(slot_lo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
    }
}

// ---------------------------------------------------------------------- kernel
// Group of tile t in a grouped launch: the largest g with gstart[g] <= t.
__device__ __forceinline__ int find_group(const long long* __restrict__ gstart, int ngroups, long long t) {
    int lo = 0, hi = ngroups - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(gstart + mid) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// GROUPED = false: one contraction described by p0.  GROUPED = true: a work
// list over `ngroups` independent contractions (one per problem of a batch,
// same axis) whose descriptors sit in global memory; tile t belongs to group
// g with gstart[g] <= t < gstart[g+1], and groups with gactive[g] == 0 are
// skipped by all three roles alike.  p0 then carries only the common fields
// (err, the ring geometry) and ntiles = gstart[ngroups], mhalves = 1.  KM
// (= Params::b_kmajor) and OM (= Params::out_mode) are compile-time so that
// each instance carries one straight-line epilogue.
template <bool GROUPED, int KM, int OM>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    axis_gemm_kernel(const __grid_constant__ Params p0, const Params* __restrict__ groups,
                     const long long* __restrict__ gstart, int ngroups, const int* __restrict__ gactive) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* ring = smem;
    uint8_t* epi = smem + RING_BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(epi + EPI_WARPS * EPI_SLOT_BYTES);
    uint64_t* full = bars;
    uint64_t* empty = bars + MAX_STAGES;
    uint64_t* tfull = bars + 2 * MAX_STAGES;
    uint64_t* tempty = bars + 2 * MAX_STAGES + 2;
    uint64_t* mma_done = bars + 2 * MAX_STAGES + 4;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + NUM_BARS);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int nst = p0.nstages;
    const int sbytes = p0.stage_bytes;

    if (threadIdx.x == 0) {
        for (int s = 0; s < MAX_STAGES; ++s) {
            mbar_init(&full[s], PRODUCERS);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], EPI_WARPS);
        }
        mbar_init(mma_done, 1);
        mbar_fence_init();
    }
    if (warp == MMA_WARP) tmem_alloc(tmem_slot, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    // launched with programmatic stream serialisation: the set-up above may
    // overlap the previous kernel, nothing below touches global memory before
    // that kernel has completed; the next kernel may begin its own set-up now
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    // a device-side loop that has converged turns the launch into a no-op
    const long long total = (p0.skip && *reinterpret_cast<const volatile int*>(p0.skip)) ? 0 : p0.ntiles * p0.mhalves;
    int* const err = p0.err;
    constexpr int b_kmajor = KM;

    if (warp < PRODUCERS) {
        if (lane == 0) {
            // ------------------------------------------------ TMA producers
            const int pw = warp;
            const int boff = p0.stage_b_off;
            int s = 0;
            uint32_t ph = 0;
            uint32_t filled = 0, last_ph = 0;  // per-stage bitmasks
            bool ok = true;
            for (long long t = blockIdx.x; t < total && ok; t += gridDim.x) {
                long long lt = t;
                const Params* pp = &p0;
                if (GROUPED) {
                    const int g = find_group(gstart, ngroups, t);
                    if (gactive && !__ldg(gactive + g)) { continue; }
                    pp = groups + g;
                    lt = t - __ldg(gstart + g);
                }
                const Params& p = *pp;
                const long long tile = lt / p.mhalves;
                const int mh = (int)(lt % p.mhalves);
                for (int sg = 0; sg < p.nseg && ok; ++sg) {
                    const Segment& S = p.seg[sg];
                    // boxes of a stage in a fixed order; box i belongs to issuer i % PRODUCERS
                    // merged boxes: one copy for all A terms and one for both B planes
                    const int na_box = S.amap2 >= 0 ? 1 : S.na;
                    const uint32_t abytes = S.amap2 >= 0 ? (uint32_t)(S.na * A_TILE_BYTES) : (uint32_t)A_TILE_BYTES;
                    const int bbox = S.bmap2 >= 0 ? 1 : (b_kmajor ? 1 : BN / 64);
                    const int nb_box = S.bmap2 >= 0 ? 1 : S.nb * bbox;
                    const uint32_t bbytes = S.bmap2 >= 0 ? (uint32_t)(S.nb * B_TILE_BYTES)
                                                         : (b_kmajor ? (uint32_t)B_TILE_BYTES : (uint32_t)(64 * SK * 2));
                    uint32_t mine = 0;
                    for (int i = pw; i < na_box + nb_box; i += PRODUCERS) mine += i < na_box ? abytes : bbytes;
                    for (int kb = 0; kb < S.nkb; ++kb) {
                        if (!mbar_wait(&empty[s], ph ^ 1u, err)) { ok = false; break; }
                        uint8_t* st = ring + s * sbytes;
                        mbar_expect_tx(&full[s], mine);
                        for (int i = pw; i < na_box + nb_box; i += PRODUCERS) {
                            if (i < na_box) {
                                if (S.amap2 >= 0)
                                    tma_load_3d(st, &p.amaps[S.amap2], &full[s], kb * SK, mh * BM, 0);
                                else
                                    tma_load_2d(st + i * A_TILE_BYTES, &p.amaps[S.amap[i]], &full[s], kb * SK, mh * BM);
                                continue;
                            }
                            if (S.bmap2 >= 0) {
                                uint8_t* dstb = st + boff;
                                if (p.b_rank == 3) {
                                    tma_load_3d(dstb, &p.bmaps[S.bmap2], &full[s], kb * SK, (int)(tile * BN), 0);
                                } else {
                                    const long long gb = tile * (BN / 64);
                                    tma_load_5d(dstb, &p.bmaps[S.bmap2], &full[s], 0, kb * SK, (int)(gb % p.nbc),
                                                (int)(gb / p.nbc), 0);
                                }
                                continue;
                            }
                            const int jb = i - na_box;   // B box index in the per-plane enumeration
                            const int b = jb / bbox, blk = jb % bbox;
                            uint8_t* dst = st + boff + b * B_TILE_BYTES;
                            if (b_kmajor) {
                                tma_load_2d(dst, &p.bmaps[S.bmap[b]], &full[s], kb * SK, (int)(tile * BN));
                            } else {
                                const long long gb = tile * (BN / 64) + blk;
                                const int pl = (int)(gb / p.nbc);
                                const int c0 = (int)(gb % p.nbc) * 64;
                                tma_load_3d(dst + blk * (64 * SK * 2), &p.bmaps[S.bmap[b]], &full[s], c0, kb * SK, pl);
                            }
                        }
                        filled |= 1u << s;
                        if (ph) last_ph |= 1u << s; else last_ph &= ~(1u << s);
                        if (++s == nst) { s = 0; ph ^= 1u; }
                    }
                }
            }
            // drain: every issued copy must land before the CTA can exit
            for (int i = 0; i < nst; ++i)
                if (filled & (1u << i)) mbar_wait(&full[i], (last_ph >> i) & 1u, err, false);
        }
    } else if (warp == MMA_WARP) {
        if (lane == 0) {
            // ------------------------------------------------ MMA issuer
            const uint32_t idesc = instr_desc(BM, BN, b_kmajor ? 0 : 1);
            // descriptor templates at stage 0 (128-byte swizzle, 8-row groups
            // 1024 bytes apart; MN-major B: 64-line blocks 64 x SK x 2 bytes
            // apart); in-smem offsets are added to the start-address field
            // (address >> 4, no carry below 256 KB)
            const uint64_t a_desc0 = smem_desc(smem_u32(ring), 16, 1024, 2);
            const uint64_t b_desc0 = b_kmajor ? smem_desc(smem_u32(ring + p0.stage_b_off), 16, 1024, 2)
                                              : smem_desc(smem_u32(ring + p0.stage_b_off), 64 * SK * 2, 1024, 2);
            const uint32_t b_k16 = b_kmajor ? (32u >> 4) : (2048u >> 4);
            int s = 0;
            uint32_t ph = 0;
            bool ok = true;
            long long it = 0;
            for (long long t = blockIdx.x; t < total && ok; t += gridDim.x) {
                long long lt = t;
                const Params* pp = &p0;
                if (GROUPED) {
                    const int g = find_group(gstart, ngroups, t);
                    if (gactive && !__ldg(gactive + g)) { continue; }
                    pp = groups + g;
                    lt = t - __ldg(gstart + g);
                }
                const Params& p = *pp;
                const int buf = (int)(it & 1);
                const uint32_t use = (uint32_t)(it >> 1);
                if (!mbar_wait(&tempty[buf], (use & 1u) ^ 1u, err)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(buf * BN);
                for (int sg = 0; sg < p.nseg && ok; ++sg) {
                    const Segment& S = p.seg[sg];
                    for (int kb = 0; kb < S.nkb; ++kb) {
                        if (!mbar_wait(&full[s], ph, err)) { ok = false; break; }
                        tc_fence_after();
                        const uint64_t ad_s = a_desc0 + (uint64_t)((s * sbytes) >> 4);
                        const uint64_t bd_s = b_desc0 + (uint64_t)((s * sbytes) >> 4);
                        for (int pr = 0; pr < S.npair; ++pr) {
                            const uint64_t ad_p = ad_s + (uint64_t)((S.pa[pr] * A_TILE_BYTES) >> 4);
                            const uint64_t bd_p = bd_s + (uint64_t)((S.pb[pr] * B_TILE_BYTES) >> 4);
#pragma unroll
                            for (int k16 = 0; k16 < SK / 16; ++k16) {
                                const uint32_t acc = (sg == 0 && kb == 0 && pr == 0 && k16 == 0) ? 0u : 1u;
                                umma_bf16(d_tmem, ad_p + (uint64_t)(k16 * (32 >> 4)), bd_p + k16 * b_k16, idesc, acc);
                            }
                        }
                        umma_commit(&empty[s]);
                        if (++s == nst) { s = 0; ph ^= 1u; }
                    }
                }
                if (ok) umma_commit(&tfull[buf]);
                ++it;
            }
            // every MMA issued by this thread has completed once mma_done fires
            umma_commit(mma_done);
            mbar_wait(mma_done, 0, err, false);
        }
    } else {
        // ---------------------------------------------------- epilogue warps
        const int ew = warp - EPI_WARP0;
        const int q = warp & 3;               // TMEM lane quadrant this warp may access
        const int half = ew >> 2;             // which 128 of the 256 columns
        uint8_t* slot = epi + ew * EPI_SLOT_BYTES;
        // the hi-plane output (one 2 KB chunk) alternates between the two
        // halves of the slot, so that a chunk is converted while the previous
        // chunk's store still reads the other half
        int half_sel = 0;
        long long it = 0;
        bool pending = false;                 // a store of this warp may still read the slot
        DotAcc da;                            // fused inner product
        // grouped launches: the destination of da (each group has its own; the
        // tiles of a CTA visit the groups in increasing order, so da is flushed
        // into a group's destination when the next group's first tile comes)
        double* dot_dst = GROUPED ? nullptr : p0.dot_out;
        auto flush_dot = [&]() {
            double t = (double)da.s - (double)da.c;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0 && dot_dst) atomicAdd(dot_dst, t);
            da = DotAcc();
        };
        float xp_beta = 0.f;                  // OUT_XPAY coefficient
        if constexpr (OM == OUT_XPAY) {
            if (p0.xp_den) xp_beta = (float)(__ldg(p0.xp_num) / __ldg(p0.xp_den));
        }
        for (long long t = blockIdx.x; t < total; t += gridDim.x) {
            long long lt = t;
            const Params* pp = &p0;
            if (GROUPED) {
                const int g = find_group(gstart, ngroups, t);
                if (gactive && !__ldg(gactive + g)) { continue; }
                pp = groups + g;
                lt = t - __ldg(gstart + g);
            }
            const Params& p = *pp;
            if (GROUPED && p.dot_out != dot_dst) {   // warp-uniform
                if (dot_dst) flush_dot();
                dot_dst = p.dot_out;
            }
            const int buf = (int)(it & 1);
            const uint32_t use = (uint32_t)(it >> 1);
            int ok = 1;
            if (lane == 0) ok = mbar_wait(&tfull[buf], use & 1u, err) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;  // warp-uniform: the TMEM loads below are .sync.aligned
            __syncwarp();
            tc_fence_after();
            const long long tile = lt / p.mhalves;
            const int mh = (int)(lt % p.mhalves);
            const int mrow0 = mh * BM + 32 * q;   // first row of this warp's quadrant
            const int m = mrow0 + lane;           // this thread's row
            const bool mval = m < p.n;
            const bool lam = !b_kmajor && p.lam_ra != nullptr;
            float ra = 1.f, rb = 0.f;             // Lambda row factors of this row
            if (lam && mval) {
                ra = __ldg(p.lam_ra + m);
                rb = __ldg(p.lam_rb + m);
            }
            for (int cc = 0; cc < BN / 2; cc += 32) {
                const int c0 = half * (BN / 2) + cc;
                // chunk position: x axis -> lines line0 .. line0 + 31 (Y[line * n1 + m]);
                // y / z axes -> plane pl, columns cx .. cx + 31 (Y[pl * plane + m * C + c])
                long long line0 = 0, gb = 0;
                int pl = 0, cx = 0, ncol;
                if (b_kmajor) {
                    line0 = tile * BN + c0;
                    const long long rem = p.lines - line0;
                    ncol = rem >= 32 ? 32 : (rem > 0 ? (int)rem : 0);
                } else {
                    gb = tile * (BN / 64) + c0 / 64;
                    pl = (int)(gb / p.nbc);
                    cx = (int)(gb % p.nbc) * 64 + (c0 & 63);
                    const int rem = p.C - cx;
                    ncol = gb < p.nblocks ? (rem >= 32 ? 32 : (rem > 0 ? rem : 0)) : 0;
                }
                // element (m, column j) of the output in global memory
                const long long gbase = b_kmajor ? line0 * p.n1 + m : (long long)pl * p.plane + (long long)m * p.C + cx;
                const long long gstep = b_kmajor ? (long long)p.n1 : 1LL;
                if constexpr (OM == OUT_SUM) {
                    const bool use_w = p.dot_vec != nullptr;
                    const bool use_ad = p.addend != nullptr;
                    if constexpr (KM != 0) {
                        // x axis (no addend or dot vector): the column factor
                        // of this lane's line, broadcast by shuffles
                        float csl = 1.f;
                        if (p.col_scale && lane < ncol) csl = __ldg(p.col_scale + line0 + lane);
                        if (pending && lane == 0) bulk_wait_read0();
                        __syncwarp();
#pragma unroll
                        for (int hf = 0; hf < 2; ++hf) {
                            uint32_t r[16];
                            tmem_ld16(tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * BN + c0 + 16 * hf), r);
                            float* f = reinterpret_cast<float*>(slot);
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                f[(16 * hf + j) * 32 + lane] =
                                    __shfl_sync(0xffffffffu, csl, 16 * hf + j) * (p.alpha * __uint_as_float(r[j]));
                        }
                    } else {
                        // y / z axes: the chunk's addend and dot vector are read
                        // coalesced (lane l: rows 4i + l / 8, columns 4 (l % 8)
                        // .. + 3, a 128-byte row segment per 8 lanes), issued
                        // before the accumulator read; the accumulator goes
                        // through the slot from its row layout to that one
                        const int rr = lane >> 3, c4 = (lane & 7) * 4;
                        const bool cval = c4 < ncol;
                        const long long cbase = (long long)pl * p.plane + cx + c4;
                        float4 ad4[8], w4[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int row = mrow0 + 4 * i + rr;   // the warp's first row + 4 i + l / 8
                            const bool ok = cval && row < p.n;
                            const long long g = cbase + (long long)row * p.C;
                            ad4[i] = (use_ad && ok) ? __ldg(reinterpret_cast<const float4*>(p.addend + g))
                                                    : make_float4(0.f, 0.f, 0.f, 0.f);
                            w4[i] = (use_w && ok) ? __ldg(reinterpret_cast<const float4*>(p.dot_vec + g))
                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                        float4 cs4 = make_float4(1.f, 1.f, 1.f, 1.f);
                        if (p.col_scale && cval)
                            cs4 = __ldg(reinterpret_cast<const float4*>(p.col_scale + (long long)pl * p.C + cx + c4));
                        // optional Lambda^{-1} (z pass: rows k, columns i + n1 j)
                        const bool ldiv = p.lam_ra != nullptr;
                        if (pending && lane == 0) bulk_wait_read0();
                        __syncwarp();
#pragma unroll
                        for (int hf = 0; hf < 2; ++hf) {
                            uint32_t r[16];
                            tmem_ld16(tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * BN + c0 + 16 * hf), r);
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                *reinterpret_cast<float4*>(slot + lane * 128 + (((4 * hf + k) ^ (lane & 7)) << 4)) =
                                    make_float4(p.alpha * __uint_as_float(r[4 * k]),
                                                p.alpha * __uint_as_float(r[4 * k + 1]),
                                                p.alpha * __uint_as_float(r[4 * k + 2]),
                                                p.alpha * __uint_as_float(r[4 * k + 3]));
                        }
                        __syncwarp();
                        float dacc = 0.f;
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int row = 4 * i + rr;
                            const int grow = mrow0 + row;
                            float4* e = reinterpret_cast<float4*>(slot + row * 128 + (((lane & 7) ^ (row & 7)) << 4));
                            float4 t = *e;
                            t.x = fmaf(cs4.x, t.x, ad4[i].x);
                            t.y = fmaf(cs4.y, t.y, ad4[i].y);
                            t.z = fmaf(cs4.z, t.z, ad4[i].z);
                            t.w = fmaf(cs4.w, t.w, ad4[i].w);
                            if (ldiv) {
                                const float a = grow < p.n ? __ldg(p.lam_ra + grow) : 1.f;
                                const float b = grow < p.n ? __ldg(p.lam_rb + grow) : 0.f;
                                float4 lu4 = make_float4(1.f, 1.f, 1.f, 1.f), lv4 = make_float4(0.f, 0.f, 0.f, 0.f);
                                if (cval) {   // the column factors (L1-resident after the first row)
                                    lu4 = __ldg(reinterpret_cast<const float4*>(p.lam_U + cx + c4));
                                    lv4 = __ldg(reinterpret_cast<const float4*>(p.lam_V + cx + c4));
                                }
                                t.x = __fdividef(t.x, fmaf(a, lu4.x, b * lv4.x));
                                t.y = __fdividef(t.y, fmaf(a, lu4.y, b * lv4.y));
                                t.z = __fdividef(t.z, fmaf(a, lu4.z, b * lv4.z));
                                t.w = __fdividef(t.w, fmaf(a, lu4.w, b * lv4.w));
                            }
                            *e = t;
                            dacc = fmaf(t.x, w4[i].x, dacc);   // w = 0 beyond ncol and below row n
                            dacc = fmaf(t.y, w4[i].y, dacc);
                            dacc = fmaf(t.z, w4[i].z, dacc);
                            dacc = fmaf(t.w, w4[i].w, dacc);
                        }
                        if (use_w) da.add(dacc);
                    }
                    if (ncol == 0) continue;   // warp-uniform
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        if (b_kmajor) tma_store_2d(&p.omap_f32, slot, mrow0, (int)line0);
                        else tma_store_3d(&p.omap_f32, slot, cx, mrow0, pl);
                        bulk_commit();
                    }
                    pending = true;
                    continue;
                }
                // the chunk's other global operand (the old direction of the
                // update, or the vector of the fused inner product), loaded
                // before the accumulator read so that the two latencies overlap
                float w[32];
                bool use_w = false;
                if constexpr (OM == OUT_XPAY) use_w = xp_beta != 0.f;
                if constexpr (OM == OUT_F32) use_w = p.dot_vec != nullptr;
                if (use_w && ncol > 0) {
                    const float* src = OM == OUT_XPAY ? (p.xp_old ? p.xp_old : p.out_f32) : p.dot_vec;
                    if (!mval) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) w[j] = 0.f;
                    } else if (!b_kmajor && ncol == 32) {
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const float4 o4 = OM == OUT_XPAY ? *(reinterpret_cast<const float4*>(src + gbase) + k)
                                                             : __ldg(reinterpret_cast<const float4*>(src + gbase) + k);
                            w[4 * k] = o4.x; w[4 * k + 1] = o4.y; w[4 * k + 2] = o4.z; w[4 * k + 3] = o4.w;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) w[j] = j < ncol ? src[gbase + j * gstep] : 0.f;
                    }
                }
                // the Lambda column factors of the chunk (the same for every
                // row: broadcast loads), ahead of the accumulator read in the
                // hi-only instance (the others have no registers to spare)
                constexpr bool LAM_EARLY = OM == OUT_HI && KM == 0;
                float U[32], V[32];
                if (LAM_EARLY && lam && ncol > 0) {
                    if (ncol == 32) {
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const float4 u4 = __ldg(reinterpret_cast<const float4*>(p.lam_U + cx) + k);
                            const float4 v4 = __ldg(reinterpret_cast<const float4*>(p.lam_V + cx) + k);
                            U[4 * k] = u4.x; U[4 * k + 1] = u4.y; U[4 * k + 2] = u4.z; U[4 * k + 3] = u4.w;
                            V[4 * k] = v4.x; V[4 * k + 1] = v4.y; V[4 * k + 2] = v4.z; V[4 * k + 3] = v4.w;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            U[j] = j < ncol ? __ldg(p.lam_U + cx + j) : 1.f;
                            V[j] = j < ncol ? __ldg(p.lam_V + cx + j) : 0.f;
                        }
                    }
                }
                uint32_t r[32];
                tmem_ld32(tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * BN + c0), r);
                if (ncol == 0) continue;   // warp-uniform
                float v[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = p.alpha * __uint_as_float(r[j]);
                if (lam) {
                    float tl = 0.f;
                    if (!LAM_EARLY) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            U[j] = j < ncol ? __ldg(p.lam_U + cx + j) : 1.f;
                            V[j] = j < ncol ? __ldg(p.lam_V + cx + j) : 0.f;
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float t0 = v[j];
                        v[j] = __fdividef(t0, ra * U[j] + rb * V[j]);
                        if (j < ncol) tl = fmaf(t0, v[j], tl);
                    }
                    if (p.dot_lam && mval) da.add(tl);
                }
                if constexpr (OM == OUT_XPAY) {
                    if (use_w) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = fmaf(xp_beta, w[j], v[j]);
                    }
                }
                if constexpr (OM == OUT_F32) {
                    if (use_w && mval) {
                        float acc = 0.f;
#pragma unroll
                        for (int j = 0; j < 32; ++j) acc = fmaf(v[j], w[j], acc);   // w = 0 beyond ncol
                        da.add(acc);
                    }
                }
                // the slot is free once this warp's previous stores have read
                // it (the hi-only output: the store before the previous one)
                if (pending && lane == 0) {
                    if constexpr (OM == OUT_HI) bulk_wait_read1();
                    else bulk_wait_read0();
                }
                __syncwarp();
                auto store = [&](const CUtensorMap* map, const uint8_t* src) {
                    if (b_kmajor) tma_store_2d(map, src, mrow0, (int)line0);
                    else tma_store_3d(map, src, cx, mrow0, pl);
                };
                // both split planes of the chunk (hi at src, lo 2 KB after it) in one store
                auto store_pair = [&](const CUtensorMap* map, const uint8_t* src) {
                    if (b_kmajor) tma_store_3d(map, src, mrow0, (int)line0, 0);
                    else tma_store_4d(map, src, cx, mrow0, pl, 0);
                };
                if constexpr (OM == OUT_F32 || OM == OUT_XPAY) {
                    slot_f32<KM != 0>(slot, lane, v);
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        store(&p.omap_f32, slot);
                        bulk_commit();
                    }
                    pending = true;
                }
                if constexpr (OM == OUT_XPAY) {
                    if (lane == 0) bulk_wait_read0();
                    __syncwarp();
                }
                if constexpr (OM == OUT_HILO || OM == OUT_XPAY || OM == OUT_HI) {
                    uint8_t* hs = slot;
                    if constexpr (OM == OUT_HI) {
                        hs = slot + half_sel * 2048;
                        half_sel ^= 1;
                        slot_bf16<KM != 0>(hs, lane, v);
                    } else {
                        slot_bf16_pair<KM != 0>(slot, slot + 2048, lane, v);
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        if constexpr (OM == OUT_HI) store(&p.omap_hi, hs);
                        else store_pair(&p.omap_hl, slot);
                        bulk_commit();
                    }
                    pending = true;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
            ++it;
        }
        if (lane == 0) bulk_wait0();   // every store of this warp has completed
        __syncwarp();
        if (dot_dst) flush_dot();
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == MMA_WARP) tmem_dealloc(tmem_base, TMEM_COLS);
}

#endif  // TFDE_TC_KERNEL_IMPL

}  // namespace tc
}  // namespace tfde
