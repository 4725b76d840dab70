// Host interface of the tcgen05 per-axis contraction (tfde_tc.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include <utility>
#include <vector>

#include "tfde_tc_kernel.cuh"

namespace tfde {
namespace tc {

int num_sms();
// Set the shared-memory attributes of every kernel instance (once).
int set_attrs();
// BF16 tiled tensor map (rank <= 5): dims / box innermost first, strides in
// bytes for dimensions 1.. (rank - 1 entries).
int encode_map(CUtensorMap* m, const void* base, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
               const cuuint32_t* box, CUtensorMapSwizzle sw);
int make_map_A(CUtensorMap* m, const __nv_bfloat16* base, int n);
int make_split_map_A(CUtensorMap* m, const __nv_bfloat16* base, int n);
int make_out_map(CUtensorMap* m, const void* base, const int n[3], int axis, bool f32);
// the split-plane pair (hi at base, lo N elements after it) as one output tensor
int make_out_map_pair(CUtensorMap* m, const void* base, const int n[3], int axis);
void set_ring(Params& P);
int make_map_B(CUtensorMap* m, const __nv_bfloat16* base, const int n[3], int axis);
int make_map_B_box(CUtensorMap* m, const __nv_bfloat16* base, const int n[3], int axis, int box_lines);
// planes: 2 (hi and lo in one box) or 1 (the hi plane alone)
int make_map_B_pair(CUtensorMap* m, const __nv_bfloat16* base, const int n[3], int axis, int planes = 2);
void set_geometry(Params& P, const int n[3], int axis);
int launch(const Params& P, cudaStream_t s, double bytes, double flops);
// One persistent launch over the tiles of `ngroups` contractions along the same
// axis (descriptors and tile offsets gstart[0..ngroups] in device memory,
// total = gstart[ngroups]); groups with gactive[g] == 0 are skipped.  All
// groups share the layout b_kmajor and the output mode out_mode.
// Bounded-wait self-test (tfde_selftest_wait).
int wait_selftest(long long limit_ns, int* tmem_freed, cudaStream_t s);
int launch_grouped(const Params* groups, const long long* gstart, int ngroups, long long total, int b_kmajor,
                   int out_mode, const int* gactive, int* err, cudaStream_t s, double bytes, double flops,
                   const int* skip = nullptr);

// Launch parameters chosen by the autotuner (tfde_tune, tfde_batch_tune):
// the number of persistent CTAs and of ring stages, per launch class.  A
// class is the kernel instance (grouped, operand layout, output mode), the
// stage size, the rows n of the contraction (0 for grouped launches) and the
// number of 128 x 256 tiles of the launch.
struct TuneKey {
    int grouped, kmajor, out_mode, stage_bytes, n;
    long long tiles;
};
struct TuneVal {
    int grid, stages;
    float us, us_default;
};
// While set (grid > 0), every launch uses these values (the tuner's trials).
void tune_force(int grid, int stages);
// The class of a single launch with descriptor P (after set_ring) / of a grouped launch.
TuneKey tune_key_single(const Params& P);
TuneKey tune_key_grouped(int b_kmajor, int out_mode, long long total);
int stage_capacity(int stage_bytes);
void tune_put(const TuneKey& k, const TuneVal& v);
int tune_count();
// entries in insertion order
bool tune_entry(int i, TuneKey* k, TuneVal* v);
void tune_clear();
// Candidate (grid, stages) pairs of a launch class: the persistent grid at
// the SM count, the grid that deals the tiles evenly, and two smaller ones;
// 2 .. capacity ring stages.
std::vector<std::pair<int, int>> tune_candidates(long long total, int stage_bytes);
// Changes whenever the table changes (graphs captured before hold stale
// launch parameters and are rebuilt).
unsigned tune_generation();
// While recording, launch() and launch_grouped() also keep their arguments;
// tune_recorded then times every candidate of each recorded class (reps
// launches between CUDA events on s, after one warm-up launch) and keeps the
// fastest in the table.
void tune_record(bool on);
int tune_recorded(int reps, cudaStream_t s);

}  // namespace tc
}  // namespace tfde
