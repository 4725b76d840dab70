// Counters of the library's GPU work (see tfde_stats in include/tfde.h).
#pragma once
#include <cuda_runtime.h>

namespace tfde {
void stats_count_launch(unsigned n = 1);
void* stats_tc_begin(cudaStream_t s, int kind);
void stats_tc_end(void* tok, cudaStream_t s, int kind, double bytes, double flops);
int stats_reset(int time_tc);
int stats_get(tfde_stats* out);
}  // namespace tfde
