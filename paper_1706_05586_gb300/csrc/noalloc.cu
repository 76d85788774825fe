// Allocation-free restriction and misfit: S = V^T C^T U, R_s = S - P, f = ||R_s||^2.
//
// Some callers cannot let a library allocate device memory: a latency-critical loop
// that must not stall (cudaMalloc and cudaFree can synchronize the whole device),
// or a host process whose device memory is entirely owned by another allocator
// (for example a framework's caching allocator that must account for every byte).
// This entry point serves them.  Its only scratch, the n_d x l_s intermediate
// T = C^T U, lives in the fixed array below, which every GPU that loads this
// library holds until the process exits; the caller passes all inputs and outputs.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "dot.h"
#include "dot_internal.h"

namespace {

// Scratch for T = C^T U: at most DOT_NOALLOC_MAX_T complex entries (1 MiB).
static __device__ __align__(256) double2 g_noalloc_T[DOT_NOALLOC_MAX_T];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch[kMaxDevices] = {};

int noalloc_fail(int code, const std::string& msg) { return dotk::record_error(code, msg); }

// Device address of the scratch array on the current device.  The name
// g_noalloc_T is only a host-side stand-in, so the address is looked up once per
// device (with that device current) and cached for the life of the process: a
// cudaDeviceReset (or another teardown of the device's primary context) would leave
// the cached address stale, which is why the entry point is documented as not usable
// on a device after such a reset.
int scratch_address(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(DOT_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(DOT_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_T);
        if (e != cudaSuccess || !p)
            return noalloc_fail(DOT_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch[dev] = p;
    }
    *out = g_scratch[dev];
    return DOT_OK;
}

}  // namespace

extern "C" {

int dot_restrict_misfit_noalloc(const double* X, int64_t n, int kp, int ls, int ld, const int64_t* colptrC,
                                const int32_t* rowsC, const double* valsC, int nd, const double* V, const double* P,
                                int is_complex, double* S, double* Rs, double* f, void* stream) {
    if (!X || !colptrC || !rowsC || !valsC || !V || !S || !Rs || !f)
        return noalloc_fail(DOT_EINVAL, "null pointer argument");
    if (n < 1 || ls < 1 || ld < 1 || nd < 1 || kp < ls)
        return noalloc_fail(DOT_EINVAL, "sizes must be positive and kp >= ls");
    if ((int64_t)nd * ls > DOT_NOALLOC_MAX_T)
        return noalloc_fail(DOT_EINVAL, "nd * ls = " + std::to_string((int64_t)nd * ls) + " exceeds the scratch limit " +
                                            std::to_string((int64_t)DOT_NOALLOC_MAX_T));
    void* T = nullptr;
    int rc = scratch_address(&T);
    if (rc != DOT_OK) return rc;
    // every entry of T, S, R_s and f is overwritten, so nothing needs clearing first
    cudaError_t e = dotk::restriction_misfit(is_complex != 0, X, kp, ls, colptrC, rowsC, valsC, nd, V, ld, P,
                                             P != nullptr, static_cast<double*>(T), S, Rs, f,
                                             static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return noalloc_fail(DOT_ECUDA, std::string("restriction launch: ") + cudaGetErrorString(e));
    return DOT_OK;
}

}  // extern "C"
