// Shared host/device utilities of libmpdd: per-thread stream and error state,
// CUDA error mapping, BLAS-style flag parsing, launch helpers.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>

#include "mpdd.h"

namespace mpdd {

// Per-thread library state: the stream calls are issued on and the text of
// the last error (mp_dd_set_stream / mp_dd_last_error).
struct ThreadState {
    cudaStream_t stream = nullptr;
    char msg[512] = {0};
};

ThreadState &tls();

// Record a formatted message for mp_dd_last_error and return `code`.
int fail(int code, const char *fmt, ...);

// Map a CUDA runtime error to MP_DD_ERR_CUDA_BASE + e, recording `what`.
int cuda_fail(cudaError_t e, const char *what);

// Check for a launch error right after a kernel launch.
inline int check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 0 : cuda_fail(e, what);
}

// Clear the per-thread error text at the start of a call.
inline void clear_error() { tls().msg[0] = 0; }

// Case-insensitive comparison of the first character of a BLAS flag.
inline bool flag_is(const char *f, char c) {
    if (f == nullptr) return false;
    char x = f[0];
    if (x >= 'a' && x <= 'z') x = (char)(x - 'a' + 'A');
    return x == c;
}

// 'N' -> 0, 'T' or 'C' -> 1, anything else -> -1.
inline int trans_flag(const char *f) {
    if (flag_is(f, 'N')) return 0;
    if (flag_is(f, 'T') || flag_is(f, 'C')) return 1;
    return -1;
}

// 'U' -> 1, 'L' -> 2, anything else -> -1.
inline int uplo_flag(const char *f) {
    if (flag_is(f, 'U')) return 1;
    if (flag_is(f, 'L')) return 2;
    return -1;
}

inline int64_t imax(int64_t a, int64_t b) { return a > b ? a : b; }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

inline bool dd_is_zero(mp_dd x) { return x.hi == 0.0 && x.lo == 0.0; }
inline bool dd_is_one(mp_dd x) { return x.hi == 1.0 && x.lo == 0.0; }

// Verify once per process that a device of compute capability 10.3 is
// current; returns 0 or MP_DD_ERR_NO_DEVICE.
int require_device();

// Number of SMs of the current device (cached).
int sm_count();
// Stream-ordered allocation from the library's own pool (freed memory stays
// mapped for later calls); free with cudaFreeAsync.
cudaError_t pool_alloc(void **ptr, size_t bytes, cudaStream_t st);

}  // namespace mpdd
