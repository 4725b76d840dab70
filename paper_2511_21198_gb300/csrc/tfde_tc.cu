// Host side of the tcgen05 per-axis contraction: TMA tensor maps and launches.
#include <cudaTypedefs.h>

#include <cstring>
#include <string>

#define TFDE_TC_KERNEL_IMPL
#include "tfde_internal.h"
#include "tfde_tc.h"
#include "tfde_stats.h"

namespace tfde {
namespace tc {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }
    return fn;
}

int encode(CUtensorMap* m, const void* base, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
           const cuuint32_t* box, CUtensorMapSwizzle sw,
           CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16) {
    auto fn = encode_fn();
    if (!fn) return set_error(TFDE_ECUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint32_t es[5] = {1, 1, 1, 1, 1};   // element strides, one per dimension (rank <= 5)
    CUresult r = fn(m, dt, (cuuint32_t)rank, const_cast<void*>(base), dims, strides,
                    box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(TFDE_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return TFDE_OK;
}

int g_num_sms = 0;

}  // namespace

int encode_map(CUtensorMap* m, const void* base, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
               const cuuint32_t* box, CUtensorMapSwizzle sw) {
    return encode(m, base, rank, dims, strides, box, sw);
}

int num_sms() {
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

// Operator matrix [rows = n][cols = n] row-major BF16 -> A operand of the
// split contraction: boxes {SK, BM}, K-major, 128B swizzle.
int make_split_map_A(CUtensorMap* m, const __nv_bfloat16* base, int n) {
    if (n % 8) return set_error(TFDE_EUNSUPPORTED, "tensor-core path needs n multiple of 8");
    const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)n * 2};
    const cuuint32_t box[2] = {(cuuint32_t)SK, (cuuint32_t)BM};
    return encode(m, base, 2, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B);
}

// Operator matrix -> A operand of the exact-slice contraction: boxes {BK, BM}, K-major, 64B swizzle.
int make_map_A(CUtensorMap* m, const __nv_bfloat16* base, int n) {
    if (n % 8) return set_error(TFDE_EUNSUPPORTED, "tensor-core path needs n multiple of 8");
    const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)n * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
    return encode(m, base, 2, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_64B);
}

// Vector plane viewed along `axis` -> B operand of the split contraction
// (k-blocks of SK, 128B swizzle): x axis K-major box {SK, BN}; y / z axes
// MN-major box {64 lines, SK, 1}.
int make_map_B(CUtensorMap* m, const __nv_bfloat16* base, const int n[3], int axis) {
    const cuuint64_t n1 = n[0], n2 = n[1], n3 = n[2];
    if (n[0] % 8) return set_error(TFDE_EUNSUPPORTED, "tensor-core path needs n1 multiple of 8");
    if (axis == 0) {
        const cuuint64_t dims[2] = {n1, n2 * n3};
        const cuuint64_t strides[1] = {n1 * 2};
        const cuuint32_t box[2] = {(cuuint32_t)SK, (cuuint32_t)BN};
        return encode(m, base, 2, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B);
    }
    cuuint64_t C, K, P;
    if (axis == 1) { C = n1; K = n2; P = n3; }
    else { C = n1 * n2; K = n3; P = 1; }
    const cuuint64_t dims[3] = {C, K, P};
    const cuuint64_t strides[2] = {C * 2, C * K * 2};
    const cuuint32_t box[3] = {64, (cuuint32_t)SK, 1};
    return encode(m, base, 3, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B);
}

// Vector plane along the x axis with a custom line box for the exact-slice
// contraction (K-major, k-blocks of BK, 64B swizzle).
int make_map_B_box(CUtensorMap* m, const __nv_bfloat16* base, const int n[3], int axis, int box_lines) {
    if (axis != 0) return set_error(TFDE_EINVAL, "make_map_B_box: x axis only");
    if (n[0] % 8) return set_error(TFDE_EUNSUPPORTED, "tensor-core path needs n1 multiple of 8");
    const cuuint64_t dims[2] = {(cuuint64_t)n[0], (cuuint64_t)n[1] * (cuuint64_t)n[2]};
    const cuuint64_t strides[1] = {(cuuint64_t)n[0] * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_lines};
    return encode(m, base, 2, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_64B);
}

// Both planes of a split pair (hi at base, lo at base + N) along `axis` as one
// tensor: x axis 3-D (k, line, plane) with box {SK, BN, planes}; y / z axes,
// when the contiguous line extent C is a multiple of BN, 5-D (line in block,
// k, block, outer plane, hi/lo) with box {64, SK, BN / 64, 1, planes}, so that
// a single copy fills the whole B stage in the layout of the per-plane boxes.
// Returns the rank, or 0 when no merged map applies.
int make_map_B_pair(CUtensorMap* m, const __nv_bfloat16* base, const int n[3], int axis, int planes) {
    const cuuint64_t n1 = n[0], n2 = n[1], n3 = n[2], N = n1 * n2 * n3;
    if (axis == 0) {
        const cuuint64_t dims[3] = {n1, n2 * n3, 2};
        const cuuint64_t strides[2] = {n1 * 2, N * 2};
        const cuuint32_t box[3] = {(cuuint32_t)SK, (cuuint32_t)BN, (cuuint32_t)planes};
        return encode(m, base, 3, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B) == TFDE_OK ? 3 : 0;
    }
    cuuint64_t C, K, P;
    if (axis == 1) { C = n1; K = n2; P = n3; }
    else { C = n1 * n2; K = n3; P = 1; }
    if (C % BN != 0) return 0;
    const cuuint64_t dims[5] = {64, K, C / 64, P, 2};
    const cuuint64_t strides[4] = {C * 2, 128, C * K * 2, N * 2};
    const cuuint32_t box[5] = {64, (cuuint32_t)SK, (cuuint32_t)(BN / 64), 1, (cuuint32_t)planes};
    if (encode(m, base, 5, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B) != TFDE_OK) {
        set_error(TFDE_OK, "");
        return 0;
    }
    return 5;
}

// Output of the split contraction along `axis` (FP32 vector or one BF16
// plane) for the epilogue's tensor stores, box 32 x 32: x axis {n1, lines}
// (element (m, line) at line * n1 + m), no swizzle; y / z axes {C, n, P}
// (element (c, m, plane)), swizzled 128B (FP32) / 64B (BF16) as the
// epilogue lays out its slots.
int make_out_map(CUtensorMap* m, const void* base, const int n[3], int axis, bool f32) {
    const cuuint64_t n1 = n[0], n2 = n[1], n3 = n[2];
    const cuuint64_t es = f32 ? 4 : 2;
    const CUtensorMapDataType dt = f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    if (axis == 0) {
        const cuuint64_t dims[2] = {n1, n2 * n3};
        const cuuint64_t strides[1] = {n1 * es};
        const cuuint32_t box[2] = {32, 32};
        return encode(m, base, 2, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_NONE, dt);
    }
    cuuint64_t C, K, P;
    if (axis == 1) { C = n1; K = n2; P = n3; }
    else { C = n1 * n2; K = n3; P = 1; }
    const cuuint64_t dims[3] = {C, K, P};
    const cuuint64_t strides[2] = {C * es, C * K * es};
    const cuuint32_t box[3] = {32, 32, 1};
    return encode(m, base, 3, dims, strides, box, f32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, dt);
}

// The hi plane at base and the lo plane N elements after it as one tensor
// with a last dimension of 2: one tensor store writes a chunk of both.
int make_out_map_pair(CUtensorMap* m, const void* base, const int n[3], int axis) {
    const cuuint64_t n1 = n[0], n2 = n[1], n3 = n[2];
    const cuuint64_t N = n1 * n2 * n3;
    const CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    if (axis == 0) {
        const cuuint64_t dims[3] = {n1, n2 * n3, 2};
        const cuuint64_t strides[2] = {n1 * 2, N * 2};
        const cuuint32_t box[3] = {32, 32, 2};
        return encode(m, base, 3, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_NONE, dt);
    }
    cuuint64_t C, K, P;
    if (axis == 1) { C = n1; K = n2; P = n3; }
    else { C = n1 * n2; K = n3; P = 1; }
    const cuuint64_t dims[4] = {C, K, P, 2};
    const cuuint64_t strides[3] = {C * 2, C * K * 2, N * 2};
    const cuuint32_t box[4] = {32, 32, 1, 2};
    return encode(m, base, 4, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_64B, dt);
}

// Ring geometry of a launch from its segments: A terms at the start of a
// stage, B planes after the largest A region, as many stages as fit.
void set_ring(Params& P) {
    int na = 1, nb = 1;
    for (int g = 0; g < P.nseg; ++g) {
        if (P.seg[g].na > na) na = P.seg[g].na;
        if (P.seg[g].nb > nb) nb = P.seg[g].nb;
    }
    P.stage_b_off = na * A_TILE_BYTES;
    P.stage_bytes = P.stage_b_off + nb * B_TILE_BYTES;
    const int ns = RING_BYTES / P.stage_bytes;
    P.nstages = ns < MAX_STAGES ? ns : MAX_STAGES;
}

// Fill the geometry fields of Params for a contraction along `axis`.
void set_geometry(Params& P, const int n[3], int axis) {
    const long long n1 = n[0], n2 = n[1], n3 = n[2];
    P.n = n[axis];
    P.mhalves = (n[axis] + BM - 1) / BM;
    P.n1 = n[0];
    if (axis == 0) {
        P.b_kmajor = 1;
        P.lines = n2 * n3;
        P.ntiles = (P.lines + BN - 1) / BN;
        P.C = 0; P.nbc = 1; P.P = 1; P.nblocks = 0; P.plane = 0;
    } else {
        P.b_kmajor = 0;
        if (axis == 1) { P.C = (int)n1; P.P = (int)n3; }
        else { P.C = (int)(n1 * n2); P.P = 1; }
        P.nbc = (P.C + 63) / 64;
        P.nblocks = (long long)P.nbc * P.P;
        P.ntiles = (P.nblocks + (BN / 64) - 1) / (BN / 64);
        P.lines = (long long)P.C * P.P;
        P.plane = (long long)P.C * n[axis];
    }
}

bool attr_done = false;

template <bool G, int KM, int OM>
bool set_attr_one() {
    return cudaFuncSetAttribute(axis_gemm_kernel<G, KM, OM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                SMEM_BYTES) == cudaSuccess;
}

int set_attrs() {
    if (!attr_done) {
        const bool ok = set_attr_one<false, 0, OUT_F32>() && set_attr_one<false, 0, OUT_HILO>() &&
                        set_attr_one<false, 1, OUT_F32>() && set_attr_one<false, 1, OUT_HILO>() &&
                        set_attr_one<true, 0, OUT_F32>() && set_attr_one<true, 0, OUT_HILO>() &&
                        set_attr_one<true, 1, OUT_F32>() && set_attr_one<true, 1, OUT_HILO>() &&
                        set_attr_one<false, 0, OUT_XPAY>() && set_attr_one<false, 1, OUT_XPAY>() &&
                        set_attr_one<false, 0, OUT_HI>() && set_attr_one<false, 1, OUT_HI>() &&
                        set_attr_one<false, 0, OUT_SUM>() && set_attr_one<false, 1, OUT_SUM>() &&
                        set_attr_one<true, 0, OUT_SUM>() && set_attr_one<true, 1, OUT_SUM>();
        if (!ok) return set_error(TFDE_ECUDA, "cudaFuncSetAttribute(smem) failed");
        attr_done = true;
    }
    return TFDE_OK;
}

// Launch with programmatic stream serialisation: the kernel's set-up (barrier
// initialisation, TMEM allocation) may start while the previous kernel on the
// stream drains; the kernel waits for that kernel's completion
// (griddepcontrol.wait) before its first global memory access.
template <bool G, int KM, int OM>
void launch_one(unsigned grid, cudaStream_t s, const Params& p0, const Params* groups, const long long* gstart,
                int ngroups, const int* gactive) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(NUM_THREADS);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, axis_gemm_kernel<G, KM, OM>, p0, groups, gstart, ngroups, gactive);
}

// The kernel instance for (layout, output mode).
template <bool G>
void launch_instance(int kmajor, int out_mode, unsigned grid, cudaStream_t s, const Params& p0, const Params* groups,
                     const long long* gstart, int ngroups, const int* gactive) {
    if (out_mode == OUT_SUM) {   // the eigenbasis passes: single and grouped (the batched solver)
        if (kmajor) launch_one<G, 1, OUT_SUM>(grid, s, p0, groups, gstart, ngroups, gactive);
        else launch_one<G, 0, OUT_SUM>(grid, s, p0, groups, gstart, ngroups, gactive);
        return;
    }
    if constexpr (!G) {   // the fused direction update exists for single launches only
        if (out_mode == OUT_XPAY) {
            if (kmajor) launch_one<G, 1, OUT_XPAY>(grid, s, p0, groups, gstart, ngroups, gactive);
            else launch_one<G, 0, OUT_XPAY>(grid, s, p0, groups, gstart, ngroups, gactive);
            return;
        }
        if (out_mode == OUT_HI) {
            if (kmajor) launch_one<G, 1, OUT_HI>(grid, s, p0, groups, gstart, ngroups, gactive);
            else launch_one<G, 0, OUT_HI>(grid, s, p0, groups, gstart, ngroups, gactive);
            return;
        }
    }
    if (kmajor) {
        if (out_mode == OUT_F32) launch_one<G, 1, OUT_F32>(grid, s, p0, groups, gstart, ngroups, gactive);
        else launch_one<G, 1, OUT_HILO>(grid, s, p0, groups, gstart, ngroups, gactive);
    } else {
        if (out_mode == OUT_F32) launch_one<G, 0, OUT_F32>(grid, s, p0, groups, gstart, ngroups, gactive);
        else launch_one<G, 0, OUT_HILO>(grid, s, p0, groups, gstart, ngroups, gactive);
    }
}

namespace {
std::vector<std::pair<TuneKey, TuneVal>> g_tune;
int g_force_grid = 0, g_force_stages = 0;
unsigned g_tune_gen = 1;

// a launch kept by the recorder
struct Rec {
    TuneKey key;
    Params p0;                  // after set_ring (single) / the grouped template
    const Params* groups;
    const long long* gstart;
    int ngroups;
    long long total;
    const int* gactive;
};
bool g_recording = false;
std::vector<Rec> g_rec;

bool same(const TuneKey& a, const TuneKey& b) {
    return a.grouped == b.grouped && a.kmajor == b.kmajor && a.out_mode == b.out_mode &&
           a.stage_bytes == b.stage_bytes && a.n == b.n && a.tiles == b.tiles;
}

// grid and stages of a launch: the tuner's trial, else the table, else the defaults
void choose(const TuneKey& k, long long total, int cap, long long* grid, int* stages) {
    *grid = total < num_sms() ? total : num_sms();
    *stages = cap;
    if (g_force_grid > 0) {
        *grid = g_force_grid;
        *stages = g_force_stages;
    } else {
        for (const auto& e : g_tune)
            if (same(e.first, k)) {
                *grid = e.second.grid;
                *stages = e.second.stages;
                break;
            }
    }
    if (*grid > total) *grid = total;
    if (*grid < 1) *grid = 1;
    if (*stages > cap) *stages = cap;
    if (*stages < 2) *stages = cap < 2 ? cap : 2;
}
}  // namespace

void tune_force(int grid, int stages) {
    g_force_grid = grid;
    g_force_stages = stages;
}

int stage_capacity(int stage_bytes) {
    const int ns = RING_BYTES / stage_bytes;
    return ns < MAX_STAGES ? ns : MAX_STAGES;
}

TuneKey tune_key_single(const Params& P) {
    return TuneKey{0, P.b_kmajor, P.out_mode, P.stage_bytes, P.n, P.ntiles * P.mhalves};
}

TuneKey tune_key_grouped(int b_kmajor, int out_mode, long long total) {
    return TuneKey{1, b_kmajor, out_mode, MAXA * A_TILE_BYTES + MAXB * B_TILE_BYTES, 0, total};
}

void tune_put(const TuneKey& k, const TuneVal& v) {
    ++g_tune_gen;
    for (auto& e : g_tune)
        if (same(e.first, k)) {
            e.second = v;
            return;
        }
    g_tune.emplace_back(k, v);
}

int tune_count() { return (int)g_tune.size(); }

bool tune_entry(int i, TuneKey* k, TuneVal* v) {
    if (i < 0 || i >= (int)g_tune.size()) return false;
    *k = g_tune[i].first;
    *v = g_tune[i].second;
    return true;
}

void tune_clear() {
    g_tune.clear();
    ++g_tune_gen;
}

unsigned tune_generation() { return g_tune_gen; }

void tune_record(bool on) {
    g_recording = on;
    if (on) g_rec.clear();
}

std::vector<std::pair<int, int>> tune_candidates(long long total, int stage_bytes) {
    const long long sms = num_sms();
    std::vector<long long> grids;
    auto add = [&](long long g) {
        if (g > total) g = total;
        if (g < 1) g = 1;
        for (long long x : grids)
            if (x == g) return;
        grids.push_back(g);
    };
    add(sms);
    const long long waves = (total + sms - 1) / sms;
    add((total + waves - 1) / waves);   // the same number of waves, tiles dealt evenly
    add(sms - sms / 8);
    add(sms * 3 / 4);
    std::vector<std::pair<int, int>> c;
    const int cap = stage_capacity(stage_bytes);
    for (long long g : grids)
        for (int st = 2; st <= cap; ++st) c.emplace_back((int)g, st);
    if (cap < 2)
        for (long long g : grids) c.emplace_back((int)g, cap);
    return c;
}

int launch(const Params& P0, cudaStream_t s, double bytes, double flops) {
    if (int st = set_attrs()) return st;
    Params P = P0;
    set_ring(P);
    const long long total = P.ntiles * P.mhalves;
    long long grid;
    choose(tune_key_single(P), total, stage_capacity(P.stage_bytes), &grid, &P.nstages);
    if (g_recording) g_rec.push_back(Rec{tune_key_single(P), P, nullptr, nullptr, 0, total, nullptr});
    void* tok = stats_tc_begin(s, TFDE_KIND_SPLIT);
    launch_instance<false>(P.b_kmajor, P.out_mode, (unsigned)grid, s, P, nullptr, nullptr, 0, nullptr);
    cudaError_t e = cudaGetLastError();
    stats_tc_end(tok, s, TFDE_KIND_SPLIT, bytes, flops);
    if (e != cudaSuccess) return set_error(TFDE_ECUDA, std::string("axis_gemm_kernel launch: ") + cudaGetErrorString(e));
    return TFDE_OK;
}

int launch_grouped(const Params* groups, const long long* gstart, int ngroups, long long total, int b_kmajor,
                   int out_mode, const int* gactive, int* err, cudaStream_t s, double bytes, double flops,
                   const int* skip) {
    if (int st = set_attrs()) return st;
    if (out_mode == OUT_HI || out_mode == OUT_XPAY)
        return set_error(TFDE_EUNSUPPORTED, "grouped axis_gemm_kernel: split, FP32 or eigenbasis output only");   // no such instances
    if (total <= 0 || ngroups <= 0) return TFDE_OK;
    Params p0;
    std::memset(&p0, 0, sizeof(p0));
    p0.ntiles = total;
    p0.mhalves = 1;
    // the largest stage any group may need: two operator terms, two planes
    p0.stage_b_off = MAXA * A_TILE_BYTES;
    p0.stage_bytes = p0.stage_b_off + MAXB * B_TILE_BYTES;
    p0.b_kmajor = b_kmajor;
    p0.out_mode = out_mode;
    p0.err = err;
    p0.skip = skip;
    long long grid;
    choose(tune_key_grouped(b_kmajor, out_mode, total), total, stage_capacity(p0.stage_bytes), &grid, &p0.nstages);
    if (g_recording)
        g_rec.push_back(Rec{tune_key_grouped(b_kmajor, out_mode, total), p0, groups, gstart, ngroups, total, gactive});
    void* tok = stats_tc_begin(s, TFDE_KIND_SPLIT);
    launch_instance<true>(b_kmajor, out_mode, (unsigned)grid, s, p0, groups, gstart, ngroups, gactive);
    cudaError_t e = cudaGetLastError();
    stats_tc_end(tok, s, TFDE_KIND_SPLIT, bytes, flops);
    if (e != cudaSuccess)
        return set_error(TFDE_ECUDA, std::string("grouped axis_gemm_kernel launch: ") + cudaGetErrorString(e));
    return TFDE_OK;
}

int tune_export(tfde_tune_entry* out, int cap, int* count) {
    int k = 0;
    for (const auto& e : g_tune) {
        if (k >= cap) break;
        tfde_tune_entry& t = out[k++];
        t.grouped = e.first.grouped;
        t.kmajor = e.first.kmajor;
        t.out_mode = e.first.out_mode;
        t.stage_bytes = e.first.stage_bytes;
        t.n = e.first.n;
        t.tiles = e.first.tiles;
        t.grid = e.second.grid;
        t.stages = e.second.stages;
        t.us = e.second.us;
        t.us_default = e.second.us_default;
    }
    if (count) *count = k;
    return TFDE_OK;
}

int tune_import(const tfde_tune_entry* in, int count) {
    for (int i = 0; i < count; ++i) {
        const tfde_tune_entry& t = in[i];
        if (t.grid < 1 || t.stages < 1 || t.stages > MAX_STAGES || t.stage_bytes < 1 || t.tiles < 1 ||
            t.stage_bytes * t.stages > RING_BYTES || t.out_mode < OUT_F32 || t.out_mode > OUT_SUM)
            return set_error(TFDE_EINVAL, "tfde_tune_set: entry " + std::to_string(i) + " out of range");
    }
    for (int i = 0; i < count; ++i) {
        const tfde_tune_entry& t = in[i];
        tune_put(TuneKey{t.grouped, t.kmajor, t.out_mode, t.stage_bytes, t.n, t.tiles},
                 TuneVal{t.grid, t.stages, t.us, t.us_default});
    }
    return TFDE_OK;
}

int tune_recorded(int reps, cudaStream_t s) {
    if (reps < 1) return set_error(TFDE_EINVAL, "reps must be >= 1");
    std::vector<Rec> recs;
    for (const Rec& r : g_rec) {   // one trial set per launch class
        bool seen = false;
        for (const Rec& q : recs) seen = seen || same(q.key, r.key);
        if (!seen) recs.push_back(r);
    }
    g_rec.clear();
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return set_error(TFDE_ECUDA, "event creation failed");
    int st = TFDE_OK;
    for (const Rec& r : recs) {
        const int cap = stage_capacity(r.p0.stage_bytes);
        const long long dgrid = r.total < num_sms() ? r.total : num_sms();
        std::vector<std::pair<int, int>> cand = tune_candidates(r.total, r.p0.stage_bytes);
        TuneVal best{(int)dgrid, cap, 1e30f, 0.f};
        for (size_t c = 0; c < cand.size() && !st; ++c) {
            Params P = r.p0;
            const int grid = cand[c].first;
            P.nstages = cand[c].second;
            auto go = [&]() {
                if (r.key.grouped)
                    launch_instance<true>(r.key.kmajor, r.key.out_mode, (unsigned)grid, s, P, r.groups, r.gstart,
                                          r.ngroups, r.gactive);
                else
                    launch_instance<false>(P.b_kmajor, P.out_mode, (unsigned)grid, s, P, nullptr, nullptr, 0, nullptr);
            };
            go();
            cudaEventRecord(e0, s);
            for (int i = 0; i < reps; ++i) go();
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
                cudaGetLastError() != cudaSuccess) {
                st = set_error(TFDE_ECUDA, "autotuner trial launch failed");
                break;
            }
            const float us = 1e3f * ms / reps;
            if (grid == dgrid && P.nstages == cap) best.us_default = us;
            if (us < best.us) {
                best.us = us;
                best.grid = grid;
                best.stages = P.nstages;
            }
        }
        if (st) break;
        tune_put(r.key, best);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

// Self-test of the bounded-wait path shared by the tensor-core kernels: one
// CTA allocates TMEM, waits on an mbarrier that nothing ever arrives on, gives
// up after limit_ns (raising *err exactly as the contraction kernels do),
// releases its TMEM and returns.  No copy or MMA is in flight at any point.
// report[0] = 2 when the wait gave up (1 if it completed), report[1] = 1
// once TMEM has been released.
__global__ void __launch_bounds__(64, 1) wait_selftest_kernel(unsigned long long limit_ns, int* err, int* report) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t slot;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    if (warp == 0) tmem_alloc(&slot, 32);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 32) report[0] = mbar_wait(&bar, 0, err, false, limit_ns) ? 1 : 2;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(slot, 32);
    __syncthreads();
    if (threadIdx.x == 0) report[1] = 1;
}

int wait_selftest(long long limit_ns, int* tmem_freed, cudaStream_t s) {
    if (limit_ns < 1000 || limit_ns > (long long)WAIT_LIMIT_NS)
        return set_error(TFDE_EINVAL, "wait limit must lie in [1 us, 2 s]");
    int* d = nullptr;
    int h[3] = {0, 0, 0};
    if (cudaMalloc((void**)&d, 3 * sizeof(int)) != cudaSuccess) return set_error(TFDE_ENOMEM, "cudaMalloc failed");
    cudaError_t e = cudaMemsetAsync(d, 0, 3 * sizeof(int), s);
    if (e == cudaSuccess) {
        stats_count_launch();
        wait_selftest_kernel<<<1, 64, 0, s>>>((unsigned long long)limit_ns, d, d + 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, 3 * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return set_error(TFDE_ECUDA, std::string("wait self-test: ") + cudaGetErrorString(e));
    if (tmem_freed) *tmem_freed = h[2];
    if (h[0] != 0 && h[1] == 2) return set_error(TFDE_ETIMEOUT, "bounded wait ran out (self-test, as designed)");
    return set_error(TFDE_ECUDA, "wait self-test: the wait did not run out");
}

}  // namespace tc
}  // namespace tfde
