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
//   warps 0..3  TMA producers: A tiles [128 x 32] (K-major, 64B swizzle) and
//               B tiles [32 x 256] (x axis: K-major 64B swizzle; y/z axes:
//               MN-major 128B swizzle, 4 boxes of 64 lines) into a 4-stage ring;
//               the boxes of a stage are dealt round-robin to the four issuing
//               threads (a thread issues one tensor copy at a time, so the copy
//               rate grows with the number of issuers), each of which arrives
//               on the stage barrier with its own byte count
//   warp 4      allocates TMEM (2 x 256 FP32 columns) and issues tcgen05.mma
//               (M=128, N=256, K=16, BF16 in, FP32 accumulate) from one thread
//   warps 5..12 epilogue, two warps per TMEM lane quadrant (one per half of the
//               256 columns): tcgen05.ld, scale, optional Lambda^{-1}, transpose
//               through shared memory, 8- or 16-byte coalesced stores of FP32 or
//               split BF16 (hi, lo) output
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
constexpr int EPI_WARPS = 8;
constexpr int PRODUCERS = 4;           // TMA issuing warps: one box per thread is issued at a time,
constexpr int MMA_WARP = PRODUCERS;    // so several issuers keep more copies in flight
constexpr int EPI_WARP0 = PRODUCERS + 1;
constexpr int NUM_THREADS = 32 * (PRODUCERS + 1 + EPI_WARPS);             // 416
constexpr int EPI_STRIDE = 33;
constexpr int EPI_FLOATS = EPI_WARPS * 32 * EPI_STRIDE;
constexpr int NUM_BARS = 2 * STAGES + 5;
constexpr int SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + EPI_FLOATS * 4 + NUM_BARS * 8 + 16;
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
enum { OUT_F32 = 0, OUT_HILO = 1, OUT_XPAY = 2, OUT_HI = 3 };

struct Params {
    CUtensorMap amaps[4];
    CUtensorMap bmaps[4];
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
    float alpha;
    float* out_f32;
    __nv_bfloat16* out_hi;
    __nv_bfloat16* out_lo;
    // optional scale 1 / (ra[m] U[c] + rb[m] V[c]) (z-axis DST pass, MN-major only)
    const float* lam_ra;
    const float* lam_rb;
    const float* lam_U;
    const float* lam_V;
    // optional fused inner product (OUT_F32 only): *dot_out += sum out[i] dot_vec[i]
    const float* dot_vec;
    double* dot_out;
    // optional, with lam_ra (z-axis DST pass): *dot_out += sum t[i] (t / Lambda)[i],
    // t the pass's output before the Lambda^{-1} scale: <r, S Lambda^{-1} S r>
    int dot_lam;
    const double* xp_num;   // OUT_XPAY: beta = *xp_num / *xp_den
    const double* xp_den;
    const float* xp_old;    // OUT_XPAY: the old p (null: out_f32 itself, updated in place)
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

// The dot_vec elements matching cnt (0..4) consecutive outputs at idx, zero
// beyond cnt; read through the non-coherent path so that the loads can be
// issued ahead of the chunk's stores.
__device__ __forceinline__ float4 dot_load(const float* __restrict__ w, long long idx, int cnt) {
    if (cnt == 4) return __ldg(reinterpret_cast<const float4*>(w + idx));
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    if (cnt > 0) r.x = __ldg(w + idx);
    if (cnt > 1) r.y = __ldg(w + idx + 1);
    if (cnt > 2) r.z = __ldg(w + idx + 2);
    return r;
}

// The old values of cnt (0..4) consecutive in/out elements at idx (zero
// beyond cnt), by plain loads: this kernel overwrites them afterwards.
__device__ __forceinline__ float4 old_load(const float* w, long long idx, int cnt) {
    if (cnt == 4) return *reinterpret_cast<const float4*>(w + idx);
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    if (cnt > 0) r.x = w[idx];
    if (cnt > 1) r.y = w[idx + 1];
    if (cnt > 2) r.z = w[idx + 2];
    return r;
}

// Four consecutive outputs (already scaled) to global memory at element index idx.
template <int OM>
__device__ __forceinline__ void store4(const Params& p, long long idx, float v0, float v1, float v2, float v3) {
    if constexpr (OM == OUT_F32) {
        *reinterpret_cast<float4*>(p.out_f32 + idx) = make_float4(v0, v1, v2, v3);
    } else if constexpr (OM == OUT_HI) {
        const __nv_bfloat162 h01 = __floats2bfloat162_rn(v0, v1);
        const __nv_bfloat162 h23 = __floats2bfloat162_rn(v2, v3);
        uint2 hv;
        hv.x = *reinterpret_cast<const uint32_t*>(&h01);
        hv.y = *reinterpret_cast<const uint32_t*>(&h23);
        *reinterpret_cast<uint2*>(p.out_hi + idx) = hv;
    } else {
        if constexpr (OM == OUT_XPAY) *reinterpret_cast<float4*>(p.out_f32 + idx) = make_float4(v0, v1, v2, v3);
        const __nv_bfloat162 h01 = __floats2bfloat162_rn(v0, v1);
        const __nv_bfloat162 h23 = __floats2bfloat162_rn(v2, v3);
        const float2 f01 = __bfloat1622float2(h01);
        const float2 f23 = __bfloat1622float2(h23);
        const __nv_bfloat162 l01 = __floats2bfloat162_rn(v0 - f01.x, v1 - f01.y);
        const __nv_bfloat162 l23 = __floats2bfloat162_rn(v2 - f23.x, v3 - f23.y);
        uint2 hv, lv;
        hv.x = *reinterpret_cast<const uint32_t*>(&h01);
        hv.y = *reinterpret_cast<const uint32_t*>(&h23);
        lv.x = *reinterpret_cast<const uint32_t*>(&l01);
        lv.y = *reinterpret_cast<const uint32_t*>(&l23);
        *reinterpret_cast<uint2*>(p.out_hi + idx) = hv;
        *reinterpret_cast<uint2*>(p.out_lo + idx) = lv;
    }
}
template <int OM>
__device__ __forceinline__ void store1(const Params& p, long long idx, float v) {
    if constexpr (OM == OUT_F32) {
        p.out_f32[idx] = v;
    } else if constexpr (OM == OUT_HI) {
        p.out_hi[idx] = __float2bfloat16_rn(v);
    } else {
        if constexpr (OM == OUT_XPAY) p.out_f32[idx] = v;
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        p.out_hi[idx] = hi;
        p.out_lo[idx] = __float2bfloat16_rn(v - __bfloat162float(hi));
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
// (err) and ntiles = gstart[ngroups], mhalves = 1.  KM (= Params::b_kmajor)
// and OM (= Params::out_mode) are compile-time so that each instance carries
// one straight-line epilogue.
template <bool GROUPED, int KM, int OM>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    axis_gemm_kernel(const __grid_constant__ Params p0, const Params* __restrict__ groups,
                     const long long* __restrict__ gstart, int ngroups, const int* __restrict__ gactive) {
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

    const long long total = p0.ntiles * p0.mhalves;
    int* const err = p0.err;
    constexpr int b_kmajor = KM;

    if (warp < PRODUCERS) {
        if (lane == 0) {
            // ------------------------------------------------ TMA producers
            const int pw = warp;
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
                    for (int kb = 0; kb < S.nkb; ++kb) {
                        if (!mbar_wait(&empty[s], ph ^ 1u, err)) { ok = false; break; }
                        uint8_t* st = stages + s * STAGE_BYTES;
                        // boxes of this stage in a fixed order; box i belongs to issuer i % PRODUCERS
                        // merged boxes: one copy for all A terms and one for both B planes
                        const int na_box = S.amap2 >= 0 ? 1 : S.na;
                        const uint32_t abytes = S.amap2 >= 0 ? (uint32_t)(S.na * A_TILE_BYTES) : (uint32_t)A_TILE_BYTES;
                        const int bbox = S.bmap2 >= 0 ? 1 : (b_kmajor ? 1 : BN / 64);
                        const int nb_box = S.bmap2 >= 0 ? 1 : S.nb * bbox;
                        const uint32_t bbytes = S.bmap2 >= 0 ? (uint32_t)(S.nb * B_TILE_BYTES)
                                                             : (b_kmajor ? (uint32_t)B_TILE_BYTES : (uint32_t)(64 * BK * 2));
                        uint32_t mine = 0;
                        for (int i = pw; i < na_box + nb_box; i += PRODUCERS) mine += i < na_box ? abytes : bbytes;
                        mbar_expect_tx(&full[s], mine);
                        for (int i = pw; i < na_box + nb_box; i += PRODUCERS) {
                            if (i < na_box) {
                                if (S.amap2 >= 0)
                                    tma_load_3d(st, &p.amaps[S.amap2], &full[s], kb * BK, mh * BM, 0);
                                else
                                    tma_load_2d(st + i * A_TILE_BYTES, &p.amaps[S.amap[i]], &full[s], kb * BK, mh * BM);
                                continue;
                            }
                            if (S.bmap2 >= 0) {
                                uint8_t* dstb = st + MAXA * A_TILE_BYTES;
                                if (p.b_rank == 3) {
                                    tma_load_3d(dstb, &p.bmaps[S.bmap2], &full[s], kb * BK, (int)(tile * BN), 0);
                                } else {
                                    const long long gb = tile * (BN / 64);
                                    tma_load_5d(dstb, &p.bmaps[S.bmap2], &full[s], 0, kb * BK, (int)(gb % p.nbc),
                                                (int)(gb / p.nbc), 0);
                                }
                                continue;
                            }
                            const int jb = i - na_box;   // B box index in the per-plane enumeration
                            const int b = jb / bbox, blk = jb % bbox;
                            uint8_t* dst = st + MAXA * A_TILE_BYTES + b * B_TILE_BYTES;
                            if (b_kmajor) {
                                tma_load_2d(dst, &p.bmaps[S.bmap[b]], &full[s], kb * BK, (int)(tile * BN));
                            } else {
                                const long long gb = tile * (BN / 64) + blk;
                                const int pl = (int)(gb / p.nbc);
                                const int c0 = (int)(gb % p.nbc) * 64;
                                tma_load_3d(dst + blk * (64 * BK * 2), &p.bmaps[S.bmap[b]], &full[s], c0, kb * BK, pl);
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
                if (filled & (1u << i)) mbar_wait(&full[i], (last_ph >> i) & 1u, err, false);
        }
    } else if (warp == MMA_WARP) {
        if (lane == 0) {
            // ------------------------------------------------ MMA issuer
            const uint32_t idesc = instr_desc(BM, BN, b_kmajor ? 0 : 1);
            // descriptor templates at stage 0; in-smem offsets are added to the
            // start-address field (address >> 4, no carry below 256 KB)
            const uint64_t a_desc0 = smem_desc(smem_u32(stages), 16, 512, 4);
            const uint64_t b_desc0 = b_kmajor ? smem_desc(smem_u32(stages + MAXA * A_TILE_BYTES), 16, 512, 4)
                                                : smem_desc(smem_u32(stages + MAXA * A_TILE_BYTES), 64 * BK * 2, 1024, 2);
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
                        const uint64_t ad_s = a_desc0 + (uint64_t)((s * STAGE_BYTES) >> 4);
                        const uint64_t bd_s = b_desc0 + (uint64_t)((s * STAGE_BYTES) >> 4);
                        for (int pr = 0; pr < S.npair; ++pr) {
                            const uint64_t ad_p = ad_s + (uint64_t)((S.pa[pr] * A_TILE_BYTES) >> 4);
                            const uint64_t bd_p = bd_s + (uint64_t)((S.pb[pr] * B_TILE_BYTES) >> 4);
#pragma unroll
                            for (int k16 = 0; k16 < BK / 16; ++k16) {
                                const uint32_t acc = (sg == 0 && kb == 0 && pr == 0 && k16 == 0) ? 0u : 1u;
                                umma_bf16(d_tmem, ad_p + (uint64_t)(k16 * (32 >> 4)), bd_p + k16 * b_k16, idesc, acc);
                            }
                        }
                        umma_commit(&empty[s]);
                        if (++s == STAGES) { s = 0; ph ^= 1u; }
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
        const int q = warp & 3;               // TMEM lane quadrant this warp may access
        const int half = (warp - EPI_WARP0) >> 2;   // which 128 of the 256 columns
        float* stg = epi + (warp - EPI_WARP0) * 32 * EPI_STRIDE;
        const int rsub = lane >> 3;           // transposed phase: 4 rows / columns per instruction
        const int cq = (lane & 7) * 4;        // ... and 4 consecutive elements per lane
        long long it = 0;
        DotAcc da;                            // fused inner product (single launches only)
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
            const int mrow0 = mh * BM + 32 * q;   // first output row of this warp
            // Lambda row factors of this lane's 8 rows, once per tile (the rows
            // are the same for every column chunk below; grouped instances,
            // short of registers, load them per chunk)
            float lra[8], lrb[8];
            const bool lam = !b_kmajor && p.lam_ra != nullptr;
            if (!GROUPED && lam) {
#pragma unroll
                for (int i8 = 0; i8 < 8; ++i8) {
                    const int m = mrow0 + i8 * 4 + rsub;
                    lra[i8] = m < p.n ? __ldg(p.lam_ra + m) : 1.f;
                    lrb[i8] = m < p.n ? __ldg(p.lam_rb + m) : 0.f;
                }
            }
            for (int cc = 0; cc < BN / 2; cc += 32) {
                const int c0 = half * (BN / 2) + cc;
                // Output positions of this lane: 8 groups i8 of up to 4 consecutive
                // elements, group i8 at oidx0 + i8 * ostep, cnt0 valid ones when
                // bit i8 of vmask is set, none otherwise.
                long long oidx0, ostep;
                int cnt0;
                unsigned vmask = 0;
                if (b_kmajor) {
                    // stg[row][line]; output Y[line * n1 + m], m contiguous
                    const int m = mrow0 + cq;
                    const long long l0 = tile * BN + c0 + rsub;
                    cnt0 = m + 4 <= p.n ? 4 : (m < p.n ? p.n - m : 0);
                    oidx0 = l0 * p.n1 + m;
                    ostep = 4LL * p.n1;
#pragma unroll
                    for (int i8 = 0; i8 < 8; ++i8)
                        if (l0 + i8 * 4 < p.lines) vmask |= 1u << i8;
                } else {
                    // stg[row][c]; output Y[pl * plane + m * C + c], c contiguous
                    const long long gb = tile * (BN / 64) + c0 / 64;
                    const int pl = (int)(gb / p.nbc);
                    const int c = (int)(gb % p.nbc) * 64 + (c0 & 63) + cq;
                    const int m0 = mrow0 + rsub;
                    cnt0 = gb < p.nblocks ? (c + 4 <= p.C ? 4 : (c < p.C ? p.C - c : 0)) : 0;
                    oidx0 = (long long)pl * p.plane + (long long)m0 * p.C + c;
                    ostep = 4LL * p.C;
#pragma unroll
                    for (int i8 = 0; i8 < 8; ++i8)
                        if (m0 + i8 * 4 < p.n) vmask |= 1u << i8;
                }
                if (cnt0 == 0) vmask = 0;
                const bool dot = OM == OUT_F32 && p.dot_vec != nullptr;
                float4 w[8];   // dot_vec (fused inner product) or the old p (OUT_XPAY) at the outputs
                if (dot) {
#pragma unroll
                    for (int i8 = 0; i8 < 8; ++i8)
                        w[i8] = dot_load(p.dot_vec, oidx0 + i8 * ostep, (vmask >> i8) & 1u ? cnt0 : 0);
                }
                if constexpr (OM == OUT_XPAY) {
                    if (xp_beta != 0.f) {
#pragma unroll
                        for (int i8 = 0; i8 < 8; ++i8)
                            w[i8] = old_load(p.xp_old ? p.xp_old : p.out_f32, oidx0 + i8 * ostep,
                                             (vmask >> i8) & 1u ? cnt0 : 0);
                    }
                }
                // Lambda column factors of this lane's 4 columns, issued before
                // the accumulator read so that their latency overlaps it
                float U[4] = {0.f, 0.f, 0.f, 0.f}, V[4] = {0.f, 0.f, 0.f, 0.f};
                if (lam && (vmask & 1u)) {
                    const int c = (int)((tile * (BN / 64) + c0 / 64) % p.nbc) * 64 + (c0 & 63) + cq;
                    if (c + 4 <= p.C && ((reinterpret_cast<uintptr_t>(p.lam_U + c) |
                                          reinterpret_cast<uintptr_t>(p.lam_V + c)) & 15) == 0) {
                        const float4 u4 = __ldg(reinterpret_cast<const float4*>(p.lam_U + c));
                        const float4 v4 = __ldg(reinterpret_cast<const float4*>(p.lam_V + c));
                        U[0] = u4.x; U[1] = u4.y; U[2] = u4.z; U[3] = u4.w;
                        V[0] = v4.x; V[1] = v4.y; V[2] = v4.z; V[3] = v4.w;
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            if (c + k < p.C) {
                                U[k] = __ldg(p.lam_U + c + k);
                                V[k] = __ldg(p.lam_V + c + k);
                            }
                    }
                }
                uint32_t r[32];
                tmem_ld32(tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * BN + c0), r);
#pragma unroll
                for (int j = 0; j < 32; ++j) stg[lane * EPI_STRIDE + j] = p.alpha * __uint_as_float(r[j]);
                __syncwarp();
                // Every staged value of this lane first (32 independent shared
                // loads), then the conversions and stores: with two epilogue
                // warps per scheduler the chunk is latency-bound, so the
                // independent work is laid out for the scheduler to overlap.
                float v[8][4];
#pragma unroll
                for (int i8 = 0; i8 < 8; ++i8)
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        v[i8][k] = b_kmajor ? stg[(cq + k) * EPI_STRIDE + i8 * 4 + rsub]
                                            : stg[(i8 * 4 + rsub) * EPI_STRIDE + cq + k];
                __syncwarp();   // the staging buffer is free for the next chunk
                if (lam && (vmask & 1u)) {   // rows ascend: none valid if the first is not
#pragma unroll
                    for (int i8 = 0; i8 < 8; ++i8)
                        if ((vmask >> i8) & 1u) {
                            const int m = mrow0 + i8 * 4 + rsub;
                            const float ra = GROUPED ? __ldg(p.lam_ra + m) : lra[i8];
                            const float rb = GROUPED ? __ldg(p.lam_rb + m) : lrb[i8];
                            float tl = 0.f;
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const float t = v[i8][k];
                                v[i8][k] = __fdividef(t, ra * U[k] + rb * V[k]);
                                if (k < cnt0) tl = fmaf(t, v[i8][k], tl);
                            }
                            if (p.dot_lam) da.add(tl);
                        }
                }
                if constexpr (OM == OUT_XPAY) {
                    if (xp_beta != 0.f) {
#pragma unroll
                        for (int i8 = 0; i8 < 8; ++i8) {
                            v[i8][0] = fmaf(xp_beta, w[i8].x, v[i8][0]);
                            v[i8][1] = fmaf(xp_beta, w[i8].y, v[i8][1]);
                            v[i8][2] = fmaf(xp_beta, w[i8].z, v[i8][2]);
                            v[i8][3] = fmaf(xp_beta, w[i8].w, v[i8][3]);
                        }
                    }
                }
#pragma unroll
                for (int i8 = 0; i8 < 8; ++i8) {
                    const int cnt = cnt0;
                    if ((vmask >> i8) & 1u) {
                        const long long idx = oidx0 + i8 * ostep;
                        if (cnt == 4) {
                            store4<OM>(p, idx, v[i8][0], v[i8][1], v[i8][2], v[i8][3]);
                        } else {
#pragma unroll
                            for (int k = 0; k < 3; ++k)
                                if (k < cnt) store1<OM>(p, idx + k, v[i8][k]);
                        }
                        if (dot) {
#pragma unroll
                            for (int k = 1; k < 4; ++k)
                                if (k >= cnt) v[i8][k] = 0.f;   // outside the grid (may be 0 / 0 above)
                            const float4 wv = w[i8];
                            da.add(fmaf(v[i8][0], wv.x, fmaf(v[i8][1], wv.y, fmaf(v[i8][2], wv.z, v[i8][3] * wv.w))));
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
            ++it;
        }
        if (p0.dot_out) {
            double t = (double)da.s - (double)da.c;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) atomicAdd(p0.dot_out, t);
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == MMA_WARP) tmem_dealloc(tmem_base, TMEM_COLS);
}

#endif  // TFDE_TC_KERNEL_IMPL

}  // namespace tc
}  // namespace tfde
