// Global attribution that allocates nothing.
//
// wdf_global_attribution obtains its FP64 partial-sum buffer from the stream-ordered
// allocator on every call.  Some callers cannot allocate device memory at the moment
// they want the reduction: a framework whose caching allocator already holds the
// device's memory (so a raw allocation outside it can fail), or a latency-critical
// loop in which an allocation or free may block the host or synchronise the device.
// This file gives them the same reduction (same kernels, same summation order, same
// result) with the partial sums in a fixed array in device memory that is part of the
// library image: every GPU that loads the library holds kNoAllocScratchDoubles doubles
// (2 MiB) until the process exits.
//
// All calls on a device share that one array, and it keeps whatever the last call left
// in it.  Two calls whose work overlaps on the GPU (different streams, or different host
// threads, without ordering between them) race on it and may return wrong sums; order
// such calls on one stream.  The first call on each device looks up the array's device
// address (cudaGetSymbolAddress, with that device current) and caches it; make that
// first call before any stream capture starts.
#include <mutex>
#include <string>

#include "launch.h"
#include "wdf_internal.h"
#include "woodelf.h"

namespace {

constexpr size_t kNoAllocScratchDoubles = (size_t)1 << 18;  // 2 MiB of FP64 partial sums
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

// Device address of g_noalloc_scratch per device, looked up once with that device
// current (in host code the array's name is only a host-side stand-in).
std::mutex g_mutex;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

wdf_status fail(wdf_status s, const std::string &msg) {
    wdf::set_last_error(msg);
    return s;
}

}  // namespace

extern "C" wdf_status wdf_global_attribution_noalloc(int32_t device, const float *phi, int64_t n, int64_t ldphi,
                                                     int32_t n_features, double *mean_abs, double *mean,
                                                     void *stream) {
    if (!mean_abs || !mean || (n > 0 && !phi)) return fail(WDF_EINVAL, "null argument");
    if (n < 0 || n_features < 1 || ldphi < n_features)
        return fail(WDF_EINVAL, "bad sizes: need n >= 0, n_features >= 1, ldphi >= n_features");
    if (device < 0 || device >= kMaxDevices) return fail(WDF_EINVAL, "device index out of range");
    // in 64-bit arithmetic before any narrowing, so that no size wraps past the check
    const int64_t need = wdf::global_attr_partial_doubles(n, n_features);
    if (need > (int64_t)kNoAllocScratchDoubles)
        return fail(WDF_EINVAL, "n * n_features too large for the fixed scratch: needs " + std::to_string(need) +
                                    " doubles of partial sums, the library holds " +
                                    std::to_string(kNoAllocScratchDoubles) +
                                    " (ceil(n / 4096) * n_features * 2 must not exceed it)");
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return fail(WDF_ECUDA, "cudaGetDevice failed");
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return fail(WDF_ECUDA, "cudaSetDevice failed");
    double *scratch = nullptr;
    cudaError_t e = cudaSuccess;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_ptr[device]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e == cudaSuccess) g_scratch_ptr[device] = static_cast<double *>(p);
        }
        scratch = g_scratch_ptr[device];
    }
    if (e == cudaSuccess) {
        // Every partial entry the final pass reads is written by the first pass of the
        // same call, so nothing has to be cleared first.
        e = wdf::launch_global_attr(phi, n, ldphi, n_features, scratch, mean_abs, mean, (cudaStream_t)stream);
    }
    if (prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess) return fail(WDF_ECUDA, std::string("wdf_global_attribution_noalloc: ") + cudaGetErrorString(e));
    return WDF_OK;
}
