// Counters of the library's GPU work (see tfde_stats in include/tfde.h).
#pragma once
#include <cuda_runtime.h>

namespace tfde {
void stats_count_launch(unsigned n = 1);
void* stats_tc_begin(cudaStream_t s, int kind);
void stats_tc_end(void* tok, cudaStream_t s, int kind, double bytes, double flops);
int stats_reset(int time_tc);
int stats_get(tfde_stats* out);
// per-launch CUDA-event timing is on (tfde_stats_reset(1)); graph-captured
// paths stay off then, so that every launch is timed on its own
bool stats_timing();
// while set, launches are not counted (they are being captured into a graph,
// whose executions are counted instead)
void stats_set_capturing(bool on);
}  // namespace tfde
