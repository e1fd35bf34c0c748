// Sliced Rgemm without any allocation by the library or the caller.
//
// Who needs this: callers that use the plain MPBLAS Rgemm argument list (no
// workspace argument) inside a program that does not let a library allocate
// device memory -- for example an application that reserves all device
// memory for its own pool at start-up and accounts for every byte, or a
// latency-critical loop where a cudaMalloc (which may synchronise the
// device) must never happen.  Such callers cannot size and pass the
// workspace mp_dd_Rgemm_sliced needs, so this entry point takes its scratch
// from a fixed array compiled into the library instead.
//
// The array is a file-scope __device__ variable of kNoAllocScratchBytes
// (32 MiB): every device on which the library's device code is loaded holds
// it from then until the process exits.  Host code cannot use the array's
// name as a device address; every call made outside stream capture looks the
// address up with cudaGetSymbolAddress (with the call's device current) and
// caches it for calls made during a capture, so the first call on a device
// should be made before any stream capture begins.  The
// sliced Rgemm kernels then run on that memory exactly as they run on a
// caller's workspace, header included: mp_dd_noalloc_report reads the status
// word and the certificate of the last call.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace mpdd {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDev = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDev] = {};

// Device address of the scratch array on the current device.  Outside
// stream capture it is looked up on every call (cudaGetSymbolAddress, with
// that device current), so an address that changed -- the library's device
// code is loaded again after a device reset -- is never used stale; during
// capture the address cached by the last uncaptured call is used.
int scratch_address(cudaStream_t stream, void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDev) return fail(MP_DD_ERR_NO_DEVICE, "device index %d", dev);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(stream, &cs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
    std::lock_guard<std::mutex> lock(g_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_scratch_ptr[dev] = p;
    } else if (g_scratch_ptr[dev] == nullptr) {
        return fail(MP_DD_ERR_NO_DEVICE,
                    "Rgemm_sliced_noalloc: first call on a device made during stream capture");
    }
    *out = g_scratch_ptr[dev];
    return 0;
}

}  // namespace

size_t noalloc_scratch_bytes() { return kNoAllocScratchBytes; }

int run_sliced_noalloc(const GemmArgs &p, int slices, cudaStream_t stream) {
    const size_t need = sliced_workspace_bytes(p.m, p.n, p.k, slices);
    if (need > kNoAllocScratchBytes)
        return fail(MP_DD_ERR_TOO_LARGE,
                    "Rgemm_sliced_noalloc: m=%lld n=%lld k=%lld with %d slices needs %zu bytes "
                    "of scratch; the built-in scratch array holds %zu",
                    (long long)p.m, (long long)p.n, (long long)p.k, slices, need,
                    kNoAllocScratchBytes);
    void *scratch = nullptr;
    int rc = scratch_address(stream, &scratch);
    if (rc) return rc;
    // run_sliced zeroes the parts that must start at zero (status word and
    // scaling maxima) and overwrites everything else it reads.
    return run_sliced(p, slices, scratch, kNoAllocScratchBytes, stream);
}

int noalloc_report(mp_dd_split_info *info) {
    void *scratch = nullptr;
    int rc = scratch_address(tls().stream, &scratch);
    if (rc) return rc;
    return split_report(scratch, info);
}

}  // namespace mpdd
