// Process-wide counters of the library's GPU work (tfde_stats_* in tfde.h).
#include <vector>

#include "tfde_internal.h"
#include "tfde_stats.h"

namespace tfde {

namespace {
struct EvPair {
    cudaEvent_t a, b;
    int kind;
};
tfde_stats g_stats{};
bool g_time_tc = false;
std::vector<EvPair> g_pending, g_pool;

void harvest(bool all) {
    size_t keep = all ? 0 : g_pending.size() / 2;
    size_t done = g_pending.size() - keep;
    for (size_t i = 0; i < done; ++i) {
        float ms = 0.f;
        cudaEventSynchronize(g_pending[i].b);
        if (cudaEventElapsedTime(&ms, g_pending[i].a, g_pending[i].b) == cudaSuccess) {
            g_stats.kind[g_pending[i].kind].ms += ms;
            g_stats.kind[g_pending[i].kind].timed++;
        }
        g_pool.push_back(g_pending[i]);
    }
    g_pending.erase(g_pending.begin(), g_pending.begin() + done);
}
}  // namespace

bool g_capturing = false;

void stats_count_launch(unsigned n) {
    if (!g_capturing) g_stats.kernel_launches += n;
}

bool stats_timing() { return g_time_tc; }
void stats_set_capturing(bool on) { g_capturing = on; }

void* stats_tc_begin(cudaStream_t s, int kind) {
    if (g_capturing) return nullptr;
    g_stats.kernel_launches++;
    g_stats.kind[kind].launches++;
    if (!g_time_tc) return nullptr;
    if (g_pending.size() > 4096) harvest(false);
    EvPair e;
    if (!g_pool.empty()) {
        e = g_pool.back();
        g_pool.pop_back();
    } else {
        cudaEventCreate(&e.a);
        cudaEventCreate(&e.b);
    }
    e.kind = kind;
    cudaEventRecord(e.a, s);
    g_pending.push_back(e);
    return reinterpret_cast<void*>(1);
}

void stats_tc_end(void* tok, cudaStream_t s, int kind, double bytes, double flops) {
    if (g_capturing) return;
    g_stats.kind[kind].bytes += bytes;
    g_stats.kind[kind].flops += flops;
    if (tok) cudaEventRecord(g_pending.back().b, s);
}

int stats_reset(int time_tc) {
    harvest(true);
    g_stats = tfde_stats{};
    g_time_tc = time_tc != 0;
    return TFDE_OK;
}

int stats_get(tfde_stats* out) {
    cudaDeviceSynchronize();
    harvest(true);
    *out = g_stats;
    return TFDE_OK;
}

}  // namespace tfde
