// Exact-integer slice contraction on tcgen05 (an Ozaki-type splitting) for the
// FP64-accurate apply of the per-axis operators of Eq. (linear_sys):
//
//   out[m, l] = sum_seg sum_k Op_seg[m, k] x_seg[k, l]  (+ addend_sign * addend[m, l])
//
// Every operator row m (all segments together) has one power-of-two scale
// 2^{es[m]} and every line l (all input vectors together) one scale 2^{el[l]};
// below them the operators and the inputs are written in balanced base-128
// digits (digit 0 in [-128, 128], the others in [-64, 63]): exact integers in
// BF16.  For every digit pair with s + t <= D the tensor core sums exact
// products in FP32 TMEM; one accumulator per diagonal d = s + t collects all
// segments and stays an exact integer below 2^24 (n <= 455).  The epilogue
// combines the diagonals in 128-bit integers and assembles the FP64 result
// directly from the integer bits and the two scales -- no FP64 arithmetic
// (GB300 issues FP64 instructions at about 1/100 of its FP32 rate).  The
// absolute error is about 2^{-7(D+1)} times the row maximum times the line
// maximum.
//
// One CTA per SM, persistent over tiles of 128 rows x 64 lines; warps 0..3
// TMA (the boxes of a stage dealt round-robin to four issuing threads), warp 4
// TMEM allocation + MMA issue (M=128, N = 64 per input slice, K=16), warps
// 5..20 epilogue (four per TMEM lane quadrant, 16 columns each).  Above four
// slices the diagonals of one tile fill TMEM, so the epilogue first reads
// them all into integer registers and hands TMEM back; its integer-ALU work
// (FP64 assembly, addend, stores) then overlaps the next tile's MMAs.
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
constexpr int MAXSEG = 2;
constexpr int STAGES = 3;         // ring slots; a launch uses as many of them as fit (see stage_count)
constexpr int A_TILE_BYTES = BM * BK * 2;                        // 8 KB
constexpr int B_TILE_BYTES = BN * BK * 2;                        // 4 KB
constexpr int STAGE_BYTES = MAXS * (A_TILE_BYTES + B_TILE_BYTES);  // 84 KB: largest stage (7 slices)
// The ring holds three 72 KB stages (6 slices) or two 84 KB ones (7 slices): a
// stage holds S operator tiles then S input tiles, S = the launch's slices.
constexpr int RING_BYTES = 3 * 6 * (A_TILE_BYTES + B_TILE_BYTES);    // 216 KB
constexpr int EPI_WARPS = 16;
constexpr int EPI_COLS = BN / (EPI_WARPS / 4);   // columns of a tile per epilogue warp
constexpr int CH = 4;                             // columns per epilogue chunk
constexpr int PRODUCERS = 4;                                     // TMA issuing warps (boxes dealt round-robin)
constexpr int MMA_WARP = PRODUCERS;
constexpr int EPI_WARP0 = PRODUCERS + 1;
constexpr int NUM_THREADS = 32 * (PRODUCERS + 1 + EPI_WARPS);     // 416
constexpr int NUM_BARS = 2 * STAGES + 5;
constexpr int SMEM_BYTES = 1024 + RING_BYTES + NUM_BARS * 8 + 16;
static_assert(2 * STAGE_BYTES <= RING_BYTES, "two stages of the largest slice count fit the ring");
// stages of S slices in one ring (at most STAGES)
__host__ __device__ constexpr int stage_count(int S) {
    return RING_BYTES / (S * (A_TILE_BYTES + B_TILE_BYTES)) < STAGES ? RING_BYTES / (S * (A_TILE_BYTES + B_TILE_BYTES))
                                                                      : STAGES;
}
constexpr uint32_t TMEM_COLS = 512;                              // (D + 1) x 64 <= 448 columns used
static_assert(SMEM_BYTES <= 232448, "shared memory budget of one CTA");

struct Segment {
    int na;                    // operator digit slices (leading ones; the rest are zero)
    int nb;                    // input digit slices (= D + 1)
    CUtensorMap amaps[MAXS];   // operator slices: BF16 [n][n], K-major, box {32, 128}, 64B swizzle
    CUtensorMap bmaps[MAXS];   // input slices: x axis box {32, 64} (64B swizzle); y/z {64, 32, 1} (128B)
    CUtensorMap amapm;         // all na operator slices in one box {32, 128, na} (slices stored contiguously)
    CUtensorMap bmapm;         // all nb input slices in one box: x {32, 64, nb}; y/z {64, 32, 1, nb}
    int merged;                // 1: amapm / bmapm are valid, one copy each per stage
};

struct Params {
    Segment seg[MAXSEG];
    int nseg;
    int nslices;               // D + 1
    int b_kmajor;
    int bm_rank;               // rank of the merged input map on y / z (4: y, 3: z)
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
    int value_sign;            // out = value_sign * value + addend_sign * addend
    double addend_sign;
    const double* addend;      // may be null
    double* out;
    double* norm2;             // optional: += sum over outputs of (out 2^norm_shift)^2 (FP32 terms)
    int norm_shift;
    const int* norm_shift_dev; // when set, the shift is *norm_shift_dev (set per call on the device)
    int* err;
};

#ifdef TFDE_OZ_KERNEL_IMPL
}  // namespace oz
}  // namespace tfde
#include "tfde_tc_ptx.cuh"
namespace tfde {
namespace oz {

using namespace tfde::tc;

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// The double nearest to I * 2^s for a signed 64-bit I (|I| < 2^62), rounded
// to nearest even from the integer bits, without branches: normalise the
// magnitude to bit 63, keep 53 bits, round on the guard bit with the sticky
// bits and the last kept bit, and add the (possibly carried) mantissa onto the
// exponent field.  Zero and results below the normal range give 0.
__device__ __forceinline__ double i64_ldexp(long long I, int s) {
    const unsigned long long sign = (unsigned long long)I & 0x8000000000000000ull;
    const unsigned long long mag = (unsigned long long)(I < 0 ? -I : I);
    const int lz = __clzll((long long)mag);                          // 64 for mag == 0
    const unsigned long long nrm = mag << (lz & 63);                  // leading one at bit 63
    const unsigned long long kept = nrm >> 11;                        // 53 bits, hidden bit at 52
    const unsigned long long guard = (nrm >> 10) & 1ull;
    const unsigned long long sticky = (nrm & 0x3FFull) != 0ull ? 1ull : 0ull;
    const unsigned long long m = kept + (guard & (sticky | (kept & 1ull)));   // may carry to 2^53
    const int be = 63 - lz + s + 1023;                                // biased exponent of the leading one
    const unsigned long long bits = ((unsigned long long)(long long)(be - 1) << 52) + m;
    return (mag == 0ull || be <= 0) ? 0.0 : __longlong_as_double((long long)(sign | bits));
}

// FP32 value of v * 2^shift from the FP64 bits (mantissa truncated to 24
// bits; 0 below and +-inf above the FP32 range): the terms of a norm.
__device__ __forceinline__ float scaled_f32(double v, int shift) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7FF);
    const int fe = e - 1023 + 127 + shift;
    const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
    const unsigned int mant = (unsigned int)((b >> 29) & 0x7FFFFFu);
    const unsigned int bits = fe >= 255 ? (sign | 0x7F800000u) : (sign | ((unsigned int)fe << 23) | mant);
    return (e == 0 || fe <= 0) ? 0.f : __uint_as_float(bits);
}

// Group of work item t in a grouped launch: gstart[g] <= t < gstart[g + 1].
__device__ __forceinline__ int oz_find_group(const long long* __restrict__ gstart, int ngroups, long long t) {
    int lo = 0, hi = ngroups - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(gstart + mid) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// GROUPED = false: one contraction described by p0.  GROUPED = true: a work
// list over `ngroups` contractions of the same axis and slice count (one per
// problem of a batch) whose descriptors sit in global memory; work item t
// (a row half of a line tile) belongs to group g with gstart[g] <= t <
// gstart[g + 1], groups with gactive[g] == 0 are skipped by all three roles
// alike, and p0 carries only the common fields (nslices, err) and ntiles =
// gstart[ngroups], mhalves = 1.
template <bool GROUPED>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    oz_gemm_kernel(const __grid_constant__ Params p0, const Params* __restrict__ groups,
                   const long long* __restrict__ gstart, int ngroups, const int* __restrict__ gactive) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* stages = smem;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + RING_BYTES);
    uint64_t* full = bars;
    uint64_t* empty = bars + STAGES;
    uint64_t* tfull = bars + 2 * STAGES;        // [2]
    uint64_t* tempty = bars + 2 * STAGES + 2;   // [2]
    uint64_t* mma_done = bars + 2 * STAGES + 4;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + NUM_BARS);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int S = p0.nslices;
    const int D = S - 1;
    const int nst = stage_count(S);                              // ring stages in use
    // TMEM buffers: two when the S diagonals of a tile fit in half of TMEM
    // (S <= 4), so that the epilogue of one tile overlaps the next tile's MMAs
    const int nbuf = S * BN * 2 <= (int)TMEM_COLS ? 2 : 1;
    const int stage_bytes = S * (A_TILE_BYTES + B_TILE_BYTES);   // 1024-byte multiple
    const int b_off = S * A_TILE_BYTES;                          // input tiles within a stage

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
    const long long total = p0.ntiles * p0.mhalves;
    int* const err = p0.err;
    // the descriptor and local work item of work item t (nullptr: a skipped group)
    auto item = [&](long long t, long long& lt) -> const Params* {
        lt = t;
        if (!GROUPED) return &p0;
        const int g = oz_find_group(gstart, ngroups, t);
        if (gactive && !__ldg(gactive + g)) return nullptr;
        lt = t - __ldg(gstart + g);
        return groups + g;
    };

    if (warp < PRODUCERS) {
        if (lane == 0) {
            const int pw = warp;
            int s = 0;
            uint32_t ph = 0, filled = 0, last_ph = 0;
            bool ok = true;
            for (long long t = blockIdx.x; t < total && ok; t += gridDim.x) {
                long long lt;
                const Params* pp = item(t, lt);
                if (!pp) continue;
                const Params& p = *pp;
                const int nkb = (p.n + BK - 1) / BK;
                const long long tile = lt / p.mhalves;
                const int mh = (int)(lt % p.mhalves);
                for (int sg = 0; sg < p.nseg && ok; ++sg) {
                    const Segment& G = p.seg[sg];
                    for (int kb = 0; kb < nkb; ++kb) {
                        if (!mbar_wait(&empty[s], ph ^ 1u, err)) { ok = false; break; }
                        uint8_t* st = stages + s * stage_bytes;
                        // box i of this stage (operator slices, then input slices) belongs to issuer i % PRODUCERS
                        uint32_t mine = 0;
                        if (G.merged) {
                            // two copies per stage: all operator slices, all input slices
                            if (pw == 0) mine = (uint32_t)(G.na * A_TILE_BYTES);
                            if (pw == 1 % PRODUCERS) mine += (uint32_t)(G.nb * B_TILE_BYTES);
                            mbar_expect_tx(&full[s], mine);
                            if (pw == 0) tma_load_3d(st, &G.amapm, &full[s], kb * BK, mh * BM, 0);
                            if (pw == 1 % PRODUCERS) {
                                uint8_t* dst = st + b_off;
                                if (p.b_kmajor) {
                                    tma_load_3d(dst, &G.bmapm, &full[s], kb * BK, (int)(tile * BN), 0);
                                } else if (p.bm_rank == 4) {
                                    const int pl = (int)(tile / p.nbc);
                                    const int c0 = (int)(tile % p.nbc) * 64;
                                    tma_load_4d(dst, &G.bmapm, &full[s], c0, kb * BK, pl, 0);
                                } else {
                                    tma_load_3d(dst, &G.bmapm, &full[s], (int)(tile % p.nbc) * 64, kb * BK, 0);
                                }
                            }
                            filled |= 1u << s;
                            if (ph) last_ph |= 1u << s; else last_ph &= ~(1u << s);
                            if (++s == nst) { s = 0; ph ^= 1u; }
                            continue;
                        }
                        for (int i = pw; i < G.na + G.nb; i += PRODUCERS)
                            mine += i < G.na ? (uint32_t)A_TILE_BYTES : (uint32_t)B_TILE_BYTES;
                        mbar_expect_tx(&full[s], mine);
                        for (int i = pw; i < G.na + G.nb; i += PRODUCERS) {
                            if (i < G.na) {
                                tma_load_2d(st + i * A_TILE_BYTES, &G.amaps[i], &full[s], kb * BK, mh * BM);
                                continue;
                            }
                            const int b = i - G.na;
                            uint8_t* dst = st + b_off + b * B_TILE_BYTES;
                            if (p.b_kmajor) {
                                tma_load_2d(dst, &G.bmaps[b], &full[s], kb * BK, (int)(tile * BN));
                            } else {
                                const int pl = (int)(tile / p.nbc);
                                const int c0 = (int)(tile % p.nbc) * 64;
                                tma_load_3d(dst, &G.bmaps[b], &full[s], c0, kb * BK, pl);
                            }
                        }
                        filled |= 1u << s;
                        if (ph) last_ph |= 1u << s; else last_ph &= ~(1u << s);
                        if (++s == nst) { s = 0; ph ^= 1u; }
                    }
                }
            }
            for (int i = 0; i < nst; ++i)
                if (filled & (1u << i)) mbar_wait(&full[i], (last_ph >> i) & 1u, err, false);
        }
    } else if (warp == MMA_WARP) {
        if (lane == 0) {
            // One MMA multiplies operator slice sa by up to four input slices at
            // once: the input slices sit at a uniform stride in a stage (the next
            // 64 rows on x, the next 64-column atom on y / z), so tb0..tb0+nn-1
            // form one B operand with N = 64 nn, and their products land in the
            // adjacent accumulators of diagonals sa+tb0 .. sa+tb0+nn-1.  A slice
            // is read once per 256 columns instead of once per 64.
            uint32_t idesc[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) idesc[c] = instr_desc(BM, BN * (c + 1), p0.b_kmajor ? 0 : 1);
            // descriptor templates at stage 0, tile 0; the start-address field
            // (bits 0..13, address >> 4) absorbs every in-smem offset without carry
            const uint64_t a_desc0 = smem_desc(smem_u32(stages), 16, 512, 4);
            const uint64_t b_desc0 = p0.b_kmajor ? smem_desc(smem_u32(stages + b_off), 16, 512, 4)
                                                 : smem_desc(smem_u32(stages + b_off), 4096, 1024, 2);
            const uint32_t b_k16 = p0.b_kmajor ? (32u >> 4) : (2048u >> 4);
            int s = 0;
            uint32_t ph = 0;
            bool ok = true;
            long long it = 0;   // work items this CTA has processed (skipped groups not counted)
            for (long long t = blockIdx.x; t < total && ok; t += gridDim.x) {
                long long lt;
                const Params* pp = item(t, lt);
                if (!pp) continue;
                const Params& p = *pp;
                const int nkb = (p.n + BK - 1) / BK;
                const int buf = (int)(it % nbuf);
                const uint32_t use = (uint32_t)(it / nbuf);
                ++it;
                const uint32_t dbase = tmem_base + (uint32_t)(buf * (TMEM_COLS / 2));
                if (!mbar_wait(&tempty[buf], (use & 1u) ^ 1u, err)) { ok = false; break; }
                tc_fence_after();
                for (int sg = 0; sg < p.nseg && ok; ++sg) {
                    const int na = p.seg[sg].na;
                    for (int kb = 0; kb < nkb; ++kb) {
                        if (!mbar_wait(&full[s], ph, err)) { ok = false; break; }
                        tc_fence_after();
                        const uint64_t ad_s = a_desc0 + (uint64_t)((s * stage_bytes) >> 4);
                        const uint64_t bd_s = b_desc0 + (uint64_t)((s * stage_bytes) >> 4);
                        const bool first = (sg == 0 && kb == 0);
#pragma unroll
                        for (int sa = 0; sa < MAXS; ++sa) {
                            if (sa >= na) break;
#pragma unroll
                            for (int tb0 = 0; tb0 < MAXS; tb0 += 4) {
                                if (sa + tb0 > D) break;
                                const int nn = min(4, D - sa - tb0 + 1);   // input slices in this MMA
#pragma unroll
                                for (int k16 = 0; k16 < BK / 16; ++k16) {
                                    const uint64_t ad = ad_s + (uint64_t)((sa * A_TILE_BYTES + k16 * 32) >> 4);
                                    const uint64_t bd = bd_s + (uint64_t)((tb0 * B_TILE_BYTES) >> 4) + k16 * b_k16;
                                    // the first products into the diagonals of a tile (segment 0,
                                    // k-block 0, digit 0 of the operator, first K step) overwrite them
                                    const uint32_t acc = (first && sa == 0 && k16 == 0) ? 0u : 1u;
                                    umma_bf16(dbase + (uint32_t)((sa + tb0) * BN), ad, bd, idesc[nn - 1], acc);
                                }
                            }
                        }
                        umma_commit(&empty[s]);
                        if (++s == nst) { s = 0; ph ^= 1u; }
                    }
                }
                if (ok) umma_commit(&tfull[buf]);
            }
            umma_commit(mma_done);
            mbar_wait(mma_done, 0, err, false);
        }
    } else {
        const int q = warp & 3;                 // TMEM lane quadrant
        const int part = (warp - EPI_WARP0) >> 2;   // columns [EPI_COLS part, EPI_COLS (part + 1))
        long long it = 0;
        float nacc = 0.f;                       // this thread's share of the output norm
        // destination of nacc: each group of a grouped launch has its own, and
        // the groups come in increasing order, so a warp flushes its share when
        // the next group's first tile arrives
        double* ndst = GROUPED ? nullptr : p0.norm2;
        auto flush_norm = [&]() {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) nacc += __shfl_xor_sync(0xffffffffu, nacc, o);
            if (lane == 0 && ndst) atomicAdd(ndst, (double)nacc);
            nacc = 0.f;
        };
        for (long long t = blockIdx.x; t < total; t += gridDim.x) {
            long long lt;
            const Params* pp = item(t, lt);
            if (!pp) continue;
            const Params& p = *pp;
            if (GROUPED && p.norm2 != ndst) {   // warp-uniform
                if (ndst) flush_norm();
                ndst = p.norm2;
            }
            const int nsh = p.norm_shift_dev ? __ldg(p.norm_shift_dev) : p.norm_shift;
            const int buf = (int)(it % nbuf);
            const uint32_t use = (uint32_t)(it / nbuf);
            ++it;
            const uint32_t dbase = tmem_base + (uint32_t)(buf * (TMEM_COLS / 2));
            int ok = 1;
            if (lane == 0) ok = mbar_wait(&tfull[buf], use & 1u, err) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            __syncwarp();
            tc_fence_after();
            const long long tile = lt / p.mhalves;
            const int mh = (int)(lt % p.mhalves);
            const int m = mh * BM + 32 * q + lane;
            const bool mvalid = m < p.n;
            const int es = mvalid ? __ldg(p.row_exp + m) : 0;
            // Up to six slices the accumulators of this thread's row and EPI_COLS
            // columns are read diagonal by diagonal (8 columns per TMEM load) and
            // folded into integers at once (I = sum_d a_d 2^{7(D-d)}, |a_d| < 2^24
            // exact in FP32), and TMEM goes back to the MMA warp before any output
            // work: the next tile's products overlap this tile's FP64 assembly,
            // addend reads and stores.  Seven slices need two integers per column
            // (the register file of 21 warps allows 80 per thread), so they are
            // read chunk by chunk and TMEM is handed back at the last chunk.
            static_assert(EPI_COLS % 8 == 0, "8-column TMEM loads");
            const uint32_t trow = dbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(part * EPI_COLS);
            // Output of the CH columns c0.. of row m: value(j, el) is the FP64 value of
            // column j (el its line exponent); plus the addend, the store and the norm.
            auto emit = [&](int cc, auto value) {
                const int c0 = part * EPI_COLS + cc;
                long long lbase, base;
                int cbase = 0;
                if (p.b_kmajor) {
                    lbase = tile * BN + c0;             // line of column c0; column j at line lbase + j
                    base = lbase * p.n1 + m;            // column j at + j * n1
                } else {
                    const int pl = (int)(tile / p.nbc);
                    cbase = (int)(tile % p.nbc) * 64 + c0;
                    lbase = (long long)pl * p.C + cbase;
                    base = (long long)pl * p.plane + (long long)m * p.C + cbase;   // column j at + j
                }
                // every CH-column chunk is either wholly valid or wholly outside: the
                // line count (x axis) and the plane width C (y, z axes) are multiples of 8
                const bool cvalid = p.b_kmajor ? (lbase < p.lines) : (tile < p.nblocks && cbase < p.C);
                if (!(mvalid && cvalid)) return;
                // line exponents of the CH columns: consecutive lines, 16-byte aligned
                const int4 e0 = __ldg(reinterpret_cast<const int4*>(p.line_exp + lbase));
                const int el[CH] = {e0.x, e0.y, e0.z, e0.w};
                double o[CH];
#pragma unroll
                for (int j = 0; j < CH; ++j) o[j] = value(j, el[j]);
                if (p.b_kmajor) {
                    // lanes are consecutive rows m: each store is one coalesced 256-byte row
#pragma unroll
                    for (int j = 0; j < CH; ++j) {
                        const long long idx = base + (long long)j * p.n1;
                        double v = o[j];
                        if (p.addend) v = fma(p.addend_sign, p.addend[idx], v);
                        p.out[idx] = v;
                        if (p.norm2) {
                            const float f = scaled_f32(v, nsh);
                            nacc = fmaf(f, f, nacc);
                        }
                    }
                } else {
                    // the CH columns are 8 CH contiguous, 8 CH-byte aligned bytes of row m
                    double2* dst = reinterpret_cast<double2*>(p.out + base);
                    if (p.addend) {
                        const double2* ad = reinterpret_cast<const double2*>(p.addend + base);
#pragma unroll
                        for (int v = 0; v < CH / 2; ++v) {
                            const double2 a2 = ad[v];
                            o[2 * v] = fma(p.addend_sign, a2.x, o[2 * v]);
                            o[2 * v + 1] = fma(p.addend_sign, a2.y, o[2 * v + 1]);
                        }
                    }
#pragma unroll
                    for (int v = 0; v < CH / 2; ++v) dst[v] = make_double2(o[2 * v], o[2 * v + 1]);
                    if (p.norm2) {
#pragma unroll
                        for (int j = 0; j < CH; ++j) {
                            const float f = scaled_f32(o[j], nsh);
                            nacc = fmaf(f, f, nacc);
                        }
                    }
                }
            };
            const int sh = es - 7 * (D + 2);
            if (S <= 6) {
                long long I[EPI_COLS];   // |I| < 2^{24 + 35}: int64
#pragma unroll
                for (int j = 0; j < EPI_COLS; ++j) I[j] = 0;
#pragma unroll
                for (int h8 = 0; h8 < EPI_COLS; h8 += 8) {
                    for (int d = 0; d < S; ++d) {
                        uint32_t r[8];
                        tmem_ld8(trow + (uint32_t)(d * BN + h8), r);
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            I[h8 + j] = I[h8 + j] * 128 + (long long)__float2int_rn(__uint_as_float(r[j]));
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[buf]);
#pragma unroll
                for (int cc = 0; cc < EPI_COLS; cc += CH) {
                    emit(cc, [&](int j, int el) {
                        const long long v = I[cc + j];
                        return i64_ldexp(p.value_sign < 0 ? -v : v, sh + el);
                    });
                    __syncwarp();
                }
            } else {
#pragma unroll
                for (int cc = 0; cc < EPI_COLS; cc += CH) {
                    uint32_t r[7][CH];
#pragma unroll
                    for (int d = 0; d < 7; ++d) tmem_ld4(trow + (uint32_t)(d * BN + cc), r[d]);
                    tmem_wait_ld();
                    if (cc == EPI_COLS - CH) {
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&tempty[buf]);
                    }
                    // I = h 2^21 + l needs up to 67 bits.  Below 2^62 it is formed exactly
                    // in int64; above, floor(I / 2^8) keeps at least 54 significant bits,
                    // so the rounded double moves by at most one ulp
                    emit(cc, [&](int j, int el) {
                        long long av[7];
#pragma unroll
                        for (int d = 0; d < 7; ++d) av[d] = __float2int_rn(__uint_as_float(r[d][j]));
                        const long long h = ((av[0] * 128 + av[1]) * 128 + av[2]) * 128 + av[3];
                        const long long l = (av[4] * 128 + av[5]) * 128 + av[6];
                        const bool big = h >= (1LL << 40) || h <= -(1LL << 40);
                        const long long v = big ? h * (1LL << 13) + (l >> 8) : h * (1LL << 21) + l;
                        return i64_ldexp(p.value_sign < 0 ? -v : v, sh + el + (big ? 8 : 0));
                    });
                    __syncwarp();
                }
            }
        }
        if (ndst) flush_norm();
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == MMA_WARP) tmem_dealloc(tmem_base, TMEM_COLS);
}

#endif  // TFDE_OZ_KERNEL_IMPL

}  // namespace oz
}  // namespace tfde
