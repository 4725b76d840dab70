// Host interface of the tcgen05 per-axis contraction (tfde_tc.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

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

}  // namespace tc
}  // namespace tfde
