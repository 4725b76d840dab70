// Mass operator A_N x = (A_{n3} (x) A_{n2} (x) A_{n1}) x for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need this
// operator: code running inside a pre-planned memory budget (an embedded
// solver step whose memory was fixed at start-up), hosts that forbid the
// allocator's implicit device synchronisation in a latency-critical loop, or
// plug-ins that only receive ready-made device buffers from their host
// application.  tfde_mass_apply_noalloc serves them: the two intermediate
// grid functions of the three tridiagonal sweeps live in a fixed array
// compiled into this library, so a call allocates nothing.
#include <mutex>
#include <string>

#include "tfde_internal.h"
#include "tfde_stats.h"

namespace tfde {
namespace {

// Largest grid (n1 * n2 * n3 points) the fixed scratch can hold: 2^18, e.g. 64^3.
constexpr long long kNoAllocMaxPoints = 1LL << 18;

// Two grid functions of kNoAllocMaxPoints doubles (4 MiB).  Every GPU that
// loads this library keeps this array until the process exits.  All calls
// share it and it keeps the previous call's contents.
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxPoints];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
double* g_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device.  In host code the
// array's name is only a stand-in, so the address is looked up once per device
// with cudaGetSymbolAddress (with that device current) and cached.
int scratch_on_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(TFDE_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_error(TFDE_EUNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return set_error(TFDE_ECUDA, std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") +
                                             cudaGetErrorString(e));
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return TFDE_OK;
}

int check_device_pointer(const void* p, const char* name) {
    if (!p) return set_error(TFDE_EINVAL, std::string(name) + " is NULL");
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return set_error(TFDE_EINVAL, std::string(name) + " is not a CUDA pointer");
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return set_error(TFDE_EINVAL, std::string(name) + " is not device memory");
    return TFDE_OK;
}

}  // namespace
}  // namespace tfde

using namespace tfde;

extern "C" int tfde_mass_apply_noalloc(const int n[3], const double* x, double* y, void* stream) {
    if (!n) return set_error(TFDE_EINVAL, "n is NULL");
    for (int a = 0; a < 3; ++a)
        if (n[a] < 1) return set_error(TFDE_EINVAL, "n must be >= 1 on every axis");
    const long long N = (long long)n[0] * n[1] * n[2];
    if (N > kNoAllocMaxPoints)
        return set_error(TFDE_EINVAL, "tfde_mass_apply_noalloc: the grid has " + std::to_string(N) +
                                          " points; the fixed scratch holds at most " +
                                          std::to_string(kNoAllocMaxPoints));
    int st;
    if ((st = check_device_pointer(x, "x")) || (st = check_device_pointer(y, "y"))) return st;
    double* scratch = nullptr;
    if ((st = scratch_on_current_device(&scratch))) return st;
    double* t1 = scratch;
    double* t2 = scratch + kNoAllocMaxPoints;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // y = A_{n3} (A_{n2} (A_{n1} x)): one tridiagonal (1,6,1)/8 sweep per axis;
    // every scratch element read is written earlier in the same call.
    launch_axis_stencil_f64(x, t1, axis_view(n, 0), 1.0, nullptr, 0.0, s);
    launch_axis_stencil_f64(t1, t2, axis_view(n, 1), 1.0, nullptr, 0.0, s);
    launch_axis_stencil_f64(t2, y, axis_view(n, 2), 1.0, nullptr, 0.0, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(TFDE_ECUDA, std::string("tfde_mass_apply_noalloc: ") + cudaGetErrorString(e));
    return TFDE_OK;
}
