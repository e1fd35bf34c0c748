// C ABI of libmpdd (declared in include/mpdd.h): argument checking with the
// BLAS numbering of illegal arguments, BLAS quick returns, per-thread stream
// and error state, and dispatch to the kernels.
#include <atomic>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace mpdd {

ThreadState &tls() {
    static thread_local ThreadState s;
    return s;
}

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(tls().msg, sizeof(tls().msg), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(MP_DD_ERR_CUDA_BASE + (int)e, "%s: %s (%s)", what, cudaGetErrorName(e),
                cudaGetErrorString(e));
}

namespace {
constexpr int kMaxDevices = 64;
std::atomic<int> g_dev_ok[kMaxDevices];   // 0 unknown, 1 ok, 2 unsuitable
std::atomic<int> g_sms[kMaxDevices];
}  // namespace

int require_device() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(MP_DD_ERR_NO_DEVICE, "device index %d", dev);
    int st = g_dev_ok[dev].load();
    if (st == 1) return 0;
    if (st == 0) {
        int major = 0, minor = 0, sms = 0;
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        g_sms[dev].store(sms);
        st = (major == 10 && minor == 3) ? 1 : 2;
        g_dev_ok[dev].store(st);
        if (st == 1) return 0;
        return fail(MP_DD_ERR_NO_DEVICE,
                    "libmpdd is built for sm_103a only; device %d is sm_%d%d", dev, major,
                    minor);
    }
    return fail(MP_DD_ERR_NO_DEVICE, "libmpdd is built for sm_103a only");
}

// The library's own stream-ordered memory pool on each device, for the
// scratch buffers of the host-buffer forms and the LU panels.  Its release
// threshold keeps freed memory mapped for the next call (the device's
// default pool would hand it back to the driver at every synchronisation,
// and mapping a gigabyte again costs tens of milliseconds).
cudaError_t pool_alloc(void **ptr, size_t bytes, cudaStream_t st) {
    static std::mutex mu;
    static cudaMemPool_t pools[kMaxDevices] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= kMaxDevices) return cudaMallocAsync(ptr, bytes, st);
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (pools[dev] == nullptr) {
            cudaMemPoolProps props{};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaError_t e = cudaMemPoolCreate(&pools[dev], &props);
            if (e != cudaSuccess) {
                pools[dev] = nullptr;
                return e;
            }
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        }
        pool = pools[dev];
    }
    return cudaMallocFromPoolAsync(ptr, bytes, pool, st);
}

int sm_count() {
    int dev = 0;
    cudaGetDevice(&dev);
    int s = (dev >= 0 && dev < kMaxDevices) ? g_sms[dev].load() : 0;
    if (s <= 0) {
        cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
        if (dev >= 0 && dev < kMaxDevices) g_sms[dev].store(s);
    }
    return s;
}

namespace {

// DGEMM argument checks; returns 0 or -i.
int check_gemm(const char *transa, const char *transb, int64_t m, int64_t n, int64_t k,
               mp_dd alpha, mp_dd_cmat A, int64_t lda, mp_dd_cmat B, int64_t ldb, mp_dd beta,
               mp_dd_mat C, int64_t ldc, GemmArgs &p) {
    int ta = trans_flag(transa), tb = trans_flag(transb);
    if (ta < 0) return fail(-1, "Rgemm: illegal transa");
    if (tb < 0) return fail(-2, "Rgemm: illegal transb");
    if (m < 0) return fail(-3, "Rgemm: m < 0");
    if (n < 0) return fail(-4, "Rgemm: n < 0");
    if (k < 0) return fail(-5, "Rgemm: k < 0");
    int64_t nrowa = ta ? k : m, nrowb = tb ? n : k;
    if (lda < imax(1, nrowa)) return fail(-8, "Rgemm: lda < max(1, %lld)", (long long)nrowa);
    if (ldb < imax(1, nrowb)) return fail(-10, "Rgemm: ldb < max(1, %lld)", (long long)nrowb);
    if (ldc < imax(1, m)) return fail(-13, "Rgemm: ldc < max(1, m)");
    bool need_ab = m > 0 && n > 0 && k > 0 && !dd_is_zero(alpha);
    if (need_ab && (A.hi == nullptr || A.lo == nullptr)) return fail(-7, "Rgemm: A is NULL");
    if (need_ab && (B.hi == nullptr || B.lo == nullptr)) return fail(-9, "Rgemm: B is NULL");
    if (m > 0 && n > 0 && (C.hi == nullptr || C.lo == nullptr))
        return fail(-12, "Rgemm: C is NULL");
    p = GemmArgs{};
    p.m = m; p.n = n; p.k = k;
    p.alpha = alpha; p.beta = beta;
    p.ah = A.hi; p.al = A.lo; p.lda = lda;
    p.bh = B.hi; p.bl = B.lo; p.ldb = ldb;
    p.ch = C.hi; p.cl = C.lo; p.ldc = ldc;
    p.ta = ta; p.tb = tb; p.tri = 0;
    p.alpha_zero = dd_is_zero(alpha) || k == 0;
    p.alpha_one = dd_is_one(alpha);
    p.beta_zero = dd_is_zero(beta);
    return 0;
}

// DSYRK argument checks; returns 0 or -i.  Fills p as the equivalent Rgemm
// (N, T) or (T, N) on A, A restricted to one triangle.
int check_syrk(const char *uplo, const char *trans, int64_t n, int64_t k, mp_dd alpha,
               mp_dd_cmat A, int64_t lda, mp_dd beta, mp_dd_mat C, int64_t ldc, GemmArgs &p) {
    int ul = uplo_flag(uplo), t = trans_flag(trans);
    if (ul < 0) return fail(-1, "Rsyrk: illegal uplo");
    if (t < 0) return fail(-2, "Rsyrk: illegal trans");
    if (n < 0) return fail(-3, "Rsyrk: n < 0");
    if (k < 0) return fail(-4, "Rsyrk: k < 0");
    int64_t nrowa = t ? k : n;
    if (lda < imax(1, nrowa)) return fail(-7, "Rsyrk: lda < max(1, %lld)", (long long)nrowa);
    if (ldc < imax(1, n)) return fail(-10, "Rsyrk: ldc < max(1, n)");
    bool need_a = n > 0 && k > 0 && !dd_is_zero(alpha);
    if (need_a && (A.hi == nullptr || A.lo == nullptr)) return fail(-6, "Rsyrk: A is NULL");
    if (n > 0 && (C.hi == nullptr || C.lo == nullptr)) return fail(-9, "Rsyrk: C is NULL");
    p = GemmArgs{};
    p.m = n; p.n = n; p.k = k;
    p.alpha = alpha; p.beta = beta;
    p.ah = A.hi; p.al = A.lo; p.lda = lda;
    p.bh = A.hi; p.bl = A.lo; p.ldb = lda;
    p.ch = C.hi; p.cl = C.lo; p.ldc = ldc;
    p.ta = t; p.tb = 1 - t; p.tri = ul;
    p.alpha_zero = dd_is_zero(alpha) || k == 0;
    p.alpha_one = dd_is_one(alpha);
    p.beta_zero = dd_is_zero(beta);
    return 0;
}

// BLAS quick return: nothing to compute.
bool quick_return(const GemmArgs &p) {
    if (p.m == 0 || p.n == 0) return true;
    return p.alpha_zero && dd_is_one(p.beta);
}

// Copy a rows x cols column-major plane between host and device with pitches.
int copy_plane(void *dst, int64_t dld, const void *src, int64_t sld, int64_t rows,
               int64_t cols, cudaMemcpyKind kind, cudaStream_t st) {
    if (rows == 0 || cols == 0) return 0;
    cudaError_t e;
    if (dld == rows && sld == rows)   // both tight: one contiguous copy
        e = cudaMemcpyAsync(dst, src, (size_t)rows * cols * 8, kind, st);
    else
        e = cudaMemcpy2DAsync(dst, (size_t)dld * 8, src, (size_t)sld * 8, (size_t)rows * 8,
                              (size_t)cols, kind, st);
    return e == cudaSuccess ? 0 : cuda_fail(e, "host-device copy");
}

// Run a validated problem whose A, B, C planes are host memory: stage them
// in device buffers (tight leading dimensions), compute, copy C back.
int run_host(GemmArgs p, int64_t arows, int64_t acols, int64_t brows, int64_t bcols,
             bool same_ab) {
    cudaStream_t st = tls().stream;
    const int64_t m = p.m, n = p.n;
    double *dA = nullptr, *dB = nullptr, *dC = nullptr;
    int64_t asz = arows * acols, bsz = same_ab ? 0 : brows * bcols, csz = m * n;
    int rc = 0;
    cudaError_t e;
    bool read_ab = !p.alpha_zero;
    if (read_ab && asz > 0) {
        e = pool_alloc(reinterpret_cast<void **>(&dA), sizeof(double) * 2 * asz, st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(A)");
    }
    if (read_ab && bsz > 0) {
        e = pool_alloc(reinterpret_cast<void **>(&dB), sizeof(double) * 2 * bsz, st);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMallocAsync(B)"); goto done; }
    }
    e = pool_alloc(reinterpret_cast<void **>(&dC), sizeof(double) * 2 * csz, st);
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMallocAsync(C)"); goto done; }
    if (read_ab && asz > 0) {
        if ((rc = copy_plane(dA, arows, p.ah, p.lda, arows, acols, cudaMemcpyHostToDevice, st)))
            goto done;
        if ((rc = copy_plane(dA + asz, arows, p.al, p.lda, arows, acols,
                             cudaMemcpyHostToDevice, st)))
            goto done;
    }
    if (read_ab && bsz > 0) {
        if ((rc = copy_plane(dB, brows, p.bh, p.ldb, brows, bcols, cudaMemcpyHostToDevice, st)))
            goto done;
        if ((rc = copy_plane(dB + bsz, brows, p.bl, p.ldb, brows, bcols,
                             cudaMemcpyHostToDevice, st)))
            goto done;
    }
    {
        double *hch = p.ch, *hcl = p.cl;
        int64_t hldc = p.ldc;
        if (!p.beta_zero) {
            if ((rc = copy_plane(dC, m, hch, hldc, m, n, cudaMemcpyHostToDevice, st))) goto done;
            if ((rc = copy_plane(dC + csz, m, hcl, hldc, m, n, cudaMemcpyHostToDevice, st)))
                goto done;
        } else if (p.tri != 0) {
            // the untouched triangle must come back unchanged
            if ((rc = copy_plane(dC, m, hch, hldc, m, n, cudaMemcpyHostToDevice, st))) goto done;
            if ((rc = copy_plane(dC + csz, m, hcl, hldc, m, n, cudaMemcpyHostToDevice, st)))
                goto done;
        }
        GemmArgs q = p;
        q.ah = dA; q.al = dA ? dA + asz : nullptr; q.lda = imax(1, arows);
        if (same_ab) { q.bh = q.ah; q.bl = q.al; q.ldb = q.lda; }
        else { q.bh = dB; q.bl = dB ? dB + bsz : nullptr; q.ldb = imax(1, brows); }
        q.ch = dC; q.cl = dC + csz; q.ldc = imax(1, m);
        if ((rc = launch_gemm_plain(q, st))) goto done;
        if ((rc = copy_plane(hch, hldc, dC, m, m, n, cudaMemcpyDeviceToHost, st))) goto done;
        if ((rc = copy_plane(hcl, hldc, dC + csz, m, m, n, cudaMemcpyDeviceToHost, st)))
            goto done;
    }
done:
    if (dA) cudaFreeAsync(dA, st);
    if (dB) cudaFreeAsync(dB, st);
    if (dC) cudaFreeAsync(dC, st);
    e = cudaStreamSynchronize(st);
    if (rc == 0 && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
    return rc;
}

}  // namespace
}  // namespace mpdd

using namespace mpdd;

extern "C" {

int mp_dd_set_stream(void *stream) {
    tls().stream = (cudaStream_t)stream;
    return 0;
}

void *mp_dd_get_stream(void) { return (void *)tls().stream; }

const char *mp_dd_last_error(void) { return tls().msg; }

int mp_dd_version(void) { return 1; }

int mp_dd_Rgemm(const char *transa, const char *transb, int64_t m, int64_t n, int64_t k,
                mp_dd alpha, mp_dd_cmat A, int64_t lda, mp_dd_cmat B, int64_t ldb, mp_dd beta,
                mp_dd_mat C, int64_t ldc) {
    clear_error();
    GemmArgs p;
    int rc = check_gemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, p);
    if (rc) return rc;
    if (quick_return(p)) return 0;
    if ((rc = require_device())) return rc;
    return launch_gemm_plain(p, tls().stream);
}

int mp_dd_Rsyrk(const char *uplo, const char *trans, int64_t n, int64_t k, mp_dd alpha,
                mp_dd_cmat A, int64_t lda, mp_dd beta, mp_dd_mat C, int64_t ldc) {
    clear_error();
    GemmArgs p;
    int rc = check_syrk(uplo, trans, n, k, alpha, A, lda, beta, C, ldc, p);
    if (rc) return rc;
    if (quick_return(p)) return 0;
    if ((rc = require_device())) return rc;
    return launch_gemm_plain(p, tls().stream);
}

int mp_qd_Rgemm(const char *transa, const char *transb, int64_t m, int64_t n, int64_t k,
                mp_qd alpha, mp_qd_cmat A, int64_t lda, mp_qd_cmat B, int64_t ldb, mp_qd beta,
                mp_qd_mat C, int64_t ldc) {
    clear_error();
    const int ta = trans_flag(transa), tb = trans_flag(transb);
    if (ta < 0) return fail(-1, "qd Rgemm: illegal transa");
    if (tb < 0) return fail(-2, "qd Rgemm: illegal transb");
    if (m < 0) return fail(-3, "qd Rgemm: m < 0");
    if (n < 0) return fail(-4, "qd Rgemm: n < 0");
    if (k < 0) return fail(-5, "qd Rgemm: k < 0");
    const int64_t nrowa = ta ? k : m, nrowb = tb ? n : k;
    if (lda < imax(1, nrowa)) return fail(-8, "qd Rgemm: lda < max(1, %lld)", (long long)nrowa);
    if (ldb < imax(1, nrowb)) return fail(-10, "qd Rgemm: ldb < max(1, %lld)", (long long)nrowb);
    if (ldc < imax(1, m)) return fail(-13, "qd Rgemm: ldc < max(1, m)");
    const bool alpha_zero = alpha.x[0] == 0.0 && alpha.x[1] == 0.0 && alpha.x[2] == 0.0 &&
                            alpha.x[3] == 0.0;
    const bool need_ab = m > 0 && n > 0 && k > 0 && !alpha_zero;
    for (int v = 0; v < 4; ++v) {
        if (need_ab && A.x[v] == nullptr) return fail(-7, "qd Rgemm: a plane of A is NULL");
        if (need_ab && B.x[v] == nullptr) return fail(-9, "qd Rgemm: a plane of B is NULL");
        if (m > 0 && n > 0 && C.x[v] == nullptr)
            return fail(-12, "qd Rgemm: a plane of C is NULL");
    }
    const bool beta_one = beta.x[0] == 1.0 && beta.x[1] == 0.0 && beta.x[2] == 0.0 &&
                          beta.x[3] == 0.0;
    if (m == 0 || n == 0 || ((alpha_zero || k == 0) && beta_one)) return 0;
    int rc = require_device();
    if (rc) return rc;
    return run_qd_gemm(ta, tb, m, n, k, alpha.x, A.x, lda, B.x, ldb, beta.x, C.x, ldc,
                       tls().stream);
}

int mp_dd_Rsyr2k(const char *uplo, const char *trans, int64_t n, int64_t k, mp_dd alpha,
                 mp_dd_cmat A, int64_t lda, mp_dd_cmat B, int64_t ldb, mp_dd beta,
                 mp_dd_mat C, int64_t ldc) {
    clear_error();
    const int ul = uplo_flag(uplo), t = trans_flag(trans);
    if (ul < 0) return fail(-1, "Rsyr2k: illegal uplo");
    if (t < 0) return fail(-2, "Rsyr2k: illegal trans");
    if (n < 0) return fail(-3, "Rsyr2k: n < 0");
    if (k < 0) return fail(-4, "Rsyr2k: k < 0");
    const int64_t nrow = t ? k : n;
    const bool need_ab = n > 0 && k > 0 && !dd_is_zero(alpha);
    if (need_ab && (A.hi == nullptr || A.lo == nullptr)) return fail(-6, "Rsyr2k: A is NULL");
    if (lda < imax(1, nrow)) return fail(-7, "Rsyr2k: lda < max(1, %lld)", (long long)nrow);
    if (need_ab && (B.hi == nullptr || B.lo == nullptr)) return fail(-8, "Rsyr2k: B is NULL");
    if (ldb < imax(1, nrow)) return fail(-9, "Rsyr2k: ldb < max(1, %lld)", (long long)nrow);
    if (n > 0 && (C.hi == nullptr || C.lo == nullptr)) return fail(-11, "Rsyr2k: C is NULL");
    if (ldc < imax(1, n)) return fail(-12, "Rsyr2k: ldc < max(1, n)");
    GemmArgs p{};
    p.m = n; p.n = n; p.k = k;
    p.alpha = alpha; p.beta = beta;
    // entry (i, j): row i of op(A) times row j of op(B), then B with A
    p.ah = A.hi; p.al = A.lo; p.lda = lda;
    p.bh = B.hi; p.bl = B.lo; p.ldb = ldb;
    p.a2h = B.hi; p.a2l = B.lo; p.lda2 = ldb;
    p.b2h = A.hi; p.b2l = A.lo; p.ldb2 = lda;
    p.ch = C.hi; p.cl = C.lo; p.ldc = ldc;
    p.ta = t; p.tb = 1 - t; p.tri = ul;
    p.alpha_zero = dd_is_zero(alpha) || k == 0;
    p.alpha_one = dd_is_one(alpha);
    p.beta_zero = dd_is_zero(beta);
    if (quick_return(p)) return 0;
    int rc = require_device();
    if (rc) return rc;
    return launch_gemm_plain(p, tls().stream);
}

int mp_dd_Rsymm(const char *side, const char *uplo, int64_t m, int64_t n, mp_dd alpha,
                mp_dd_cmat A, int64_t lda, mp_dd_cmat B, int64_t ldb, mp_dd beta, mp_dd_mat C,
                int64_t ldc) {
    clear_error();
    const int right = flag_is(side, 'R') ? 1 : flag_is(side, 'L') ? 0 : -1;
    if (right < 0) return fail(-1, "Rsymm: illegal side");
    const int ul = uplo_flag(uplo);
    if (ul < 0) return fail(-2, "Rsymm: illegal uplo");
    if (m < 0) return fail(-3, "Rsymm: m < 0");
    if (n < 0) return fail(-4, "Rsymm: n < 0");
    const int64_t order = right ? n : m;
    const bool need_ab = m > 0 && n > 0 && !dd_is_zero(alpha);
    if (need_ab && (A.hi == nullptr || A.lo == nullptr)) return fail(-6, "Rsymm: A is NULL");
    if (lda < imax(1, order)) return fail(-7, "Rsymm: lda < max(1, order of A)");
    if (need_ab && (B.hi == nullptr || B.lo == nullptr)) return fail(-8, "Rsymm: B is NULL");
    if (ldb < imax(1, m)) return fail(-9, "Rsymm: ldb < max(1, m)");
    if (m > 0 && n > 0 && (C.hi == nullptr || C.lo == nullptr))
        return fail(-11, "Rsymm: C is NULL");
    if (ldc < imax(1, m)) return fail(-12, "Rsymm: ldc < max(1, m)");
    GemmArgs p{};
    p.m = m; p.n = n; p.k = order;
    p.alpha = alpha; p.beta = beta;
    if (!right) {
        p.ah = A.hi; p.al = A.lo; p.lda = lda; p.sym_a = ul;
        p.bh = B.hi; p.bl = B.lo; p.ldb = ldb;
    } else {
        p.ah = B.hi; p.al = B.lo; p.lda = ldb;
        p.bh = A.hi; p.bl = A.lo; p.ldb = lda; p.sym_b = ul;
    }
    p.ch = C.hi; p.cl = C.lo; p.ldc = ldc;
    p.ta = 0; p.tb = 0; p.tri = 0;
    p.alpha_zero = dd_is_zero(alpha) || order == 0;
    p.alpha_one = dd_is_one(alpha);
    p.beta_zero = dd_is_zero(beta);
    if (quick_return(p)) return 0;
    int rc = require_device();
    if (rc) return rc;
    return launch_gemm_plain(p, tls().stream);
}

int mp_dd_Rgemm_host(const char *transa, const char *transb, int64_t m, int64_t n, int64_t k,
                     mp_dd alpha, mp_dd_cmat A, int64_t lda, mp_dd_cmat B, int64_t ldb,
                     mp_dd beta, mp_dd_mat C, int64_t ldc) {
    clear_error();
    GemmArgs p;
    int rc = check_gemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, p);
    if (rc) return rc;
    if (quick_return(p)) return 0;
    if ((rc = require_device())) return rc;
    int64_t ar = p.ta ? k : m, ac = p.ta ? m : k;
    int64_t br = p.tb ? n : k, bc = p.tb ? k : n;
    return run_host(p, ar, ac, br, bc, false);
}

int mp_dd_Rsyrk_host(const char *uplo, const char *trans, int64_t n, int64_t k, mp_dd alpha,
                     mp_dd_cmat A, int64_t lda, mp_dd beta, mp_dd_mat C, int64_t ldc) {
    clear_error();
    GemmArgs p;
    int rc = check_syrk(uplo, trans, n, k, alpha, A, lda, beta, C, ldc, p);
    if (rc) return rc;
    if (quick_return(p)) return 0;
    if ((rc = require_device())) return rc;
    int64_t ar = p.ta ? k : n, ac = p.ta ? n : k;
    return run_host(p, ar, ac, 0, 0, true);
}

size_t mp_dd_Rgemm_sliced_workspace(int64_t m, int64_t n, int64_t k, int slices) {
    if (m < 0 || n < 0 || k < 0 || slices < 0 || slices > kMaxSlices) return 0;
    return sliced_workspace_bytes(m, n, k, slices);
}

int mp_dd_Rgemm_sliced(const char *transa, const char *transb, int64_t m, int64_t n,
                       int64_t k, mp_dd alpha, mp_dd_cmat A, int64_t lda, mp_dd_cmat B,
                       int64_t ldb, mp_dd beta, mp_dd_mat C, int64_t ldc, int slices,
                       void *workspace, size_t workspace_bytes) {
    clear_error();
    GemmArgs p;
    int rc = check_gemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, p);
    if (rc) return rc;
    if (slices != 0 && (slices < 2 || slices > kMaxSlices))
        return fail(-14, "Rgemm_sliced: slices = %d outside [2, %d]", slices, kMaxSlices);
    if (quick_return(p)) return 0;
    if (workspace == nullptr) return fail(-15, "Rgemm_sliced: workspace is NULL");
    if ((rc = require_device())) return rc;
    return run_sliced(p, slices, workspace, workspace_bytes, tls().stream);
}

int mp_dd_Rgemm_sliced_noalloc(const char *transa, const char *transb, int64_t m, int64_t n,
                               int64_t k, mp_dd alpha, mp_dd_cmat A, int64_t lda, mp_dd_cmat B,
                               int64_t ldb, mp_dd beta, mp_dd_mat C, int64_t ldc, int slices) {
    clear_error();
    GemmArgs p;
    int rc = check_gemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, p);
    if (rc) return rc;
    if (slices != 0 && (slices < 2 || slices > kMaxSlices))
        return fail(-14, "Rgemm_sliced_noalloc: slices = %d outside [2, %d]", slices,
                    kMaxSlices);
    if (quick_return(p)) return 0;
    if ((rc = require_device())) return rc;
    return run_sliced_noalloc(p, slices, tls().stream);
}

size_t mp_dd_Rgemm_crt_workspace(int64_t m, int64_t n, int64_t k) {
    if (m < 0 || n < 0 || k < 0) return 0;
    return crt_workspace_bytes(m, n, k);
}

int mp_dd_Rgemm_crt(const char *transa, const char *transb, int64_t m, int64_t n, int64_t k,
                    mp_dd alpha, mp_dd_cmat A, int64_t lda, mp_dd_cmat B, int64_t ldb,
                    mp_dd beta, mp_dd_mat C, int64_t ldc, void *workspace,
                    size_t workspace_bytes) {
    clear_error();
    GemmArgs p;
    int rc = check_gemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, p);
    if (rc) return rc;
    if (quick_return(p)) return 0;
    if (workspace == nullptr) return fail(-14, "Rgemm_crt: workspace is NULL");
    if ((rc = require_device())) return rc;
    return run_crt(p, workspace, workspace_bytes, tls().stream);
}

size_t mp_dd_Rsyrk_crt_workspace(int64_t n, int64_t k) {
    if (n < 0 || k < 0) return 0;
    return crt_workspace_bytes(n, n, k, true);
}

int mp_dd_Rsyrk_crt(const char *uplo, const char *trans, int64_t n, int64_t k, mp_dd alpha,
                    mp_dd_cmat A, int64_t lda, mp_dd beta, mp_dd_mat C, int64_t ldc,
                    void *workspace, size_t workspace_bytes) {
    clear_error();
    GemmArgs p;
    int rc = check_syrk(uplo, trans, n, k, alpha, A, lda, beta, C, ldc, p);
    if (rc) return rc;
    if (quick_return(p)) return 0;
    if (workspace == nullptr) return fail(-12, "Rsyrk_crt: workspace is NULL");
    if ((rc = require_device())) return rc;
    return run_crt(p, workspace, workspace_bytes, tls().stream);
}

int mp_dd_crt_layout(int64_t m, int64_t n, int64_t k, size_t offsets[48], int *moduli) {
    clear_error();
    if (offsets == nullptr || moduli == nullptr) return fail(-4, "crt_layout: NULL output");
    if (m < 0 || n < 0 || k < 0) return fail(-1, "crt_layout: negative size");
    return crt_layout_query(m, n, k, offsets, moduli);
}

int mp_dd_sliced_layout(int64_t m, int64_t n, int64_t k, int slices, size_t offsets[8]) {
    clear_error();
    if (offsets == nullptr) return fail(-5, "sliced_layout: offsets is NULL");
    if (slices < 0 || slices > kMaxSlices) return fail(-4, "sliced_layout: slices");
    return sliced_layout(m, n, k, slices, offsets);
}

int mp_dd_workspace_status(const void *workspace, int *status) {
    clear_error();
    if (workspace == nullptr) return fail(-1, "workspace_status: workspace is NULL");
    if (status == nullptr) return fail(-2, "workspace_status: status is NULL");
    return read_status(workspace, status);
}

int mp_dd_split_report(const void *workspace, mp_dd_split_info *info) {
    clear_error();
    if (workspace == nullptr) return fail(-1, "split_report: workspace is NULL");
    if (info == nullptr) return fail(-2, "split_report: info is NULL");
    return split_report(workspace, info);
}

int mp_dd_noalloc_report(mp_dd_split_info *info) {
    clear_error();
    if (info == nullptr) return fail(-1, "noalloc_report: info is NULL");
    int rc = require_device();
    if (rc) return rc;
    return noalloc_report(info);
}

int mp_dd_magnitude_layout(int form, int64_t m, int64_t n, int64_t k, int slices,
                           size_t offsets[2]) {
    clear_error();
    if (offsets == nullptr) return fail(-6, "magnitude_layout: offsets is NULL");
    if (m < 0 || n < 0 || k < 0) return fail(-2, "magnitude_layout: negative size");
    switch (form) {
        case 1:
            if (slices < 0 || slices > kMaxSlices) return fail(-5, "magnitude_layout: slices");
            return sliced_magnitude_offsets(m, n, k, slices, offsets);
        case 2: return crt_magnitude_offsets(m, n, k, false, offsets);
        case 3: return crt_magnitude_offsets(n, n, k, true, offsets);
        default: return fail(-1, "magnitude_layout: form must be 1, 2 or 3");
    }
}

int mp_dd_Rpotrf(const char *uplo, int64_t n, mp_dd_mat A, int64_t lda, int64_t *info) {
    clear_error();
    int ul = uplo_flag(uplo);
    if (ul < 0) return fail(-1, "Rpotrf: illegal uplo");
    if (n < 0) return fail(-2, "Rpotrf: n < 0");
    if (n > 0 && (A.hi == nullptr || A.lo == nullptr)) return fail(-3, "Rpotrf: A is NULL");
    if (lda < imax(1, n)) return fail(-4, "Rpotrf: lda < max(1, n)");
    if (info == nullptr) return fail(-5, "Rpotrf: info is NULL");
    int rc = require_device();
    if (rc) return rc;
    if (n == 0) {
        cudaError_t e = cudaMemsetAsync(info, 0, sizeof(int64_t), tls().stream);
        return e == cudaSuccess ? 0 : cuda_fail(e, "info reset");
    }
    return run_potrf(ul == 2, n, A.hi, A.lo, lda, info, tls().stream);
}

size_t mp_dd_Rpotrf_crt_workspace(int64_t n) {
    if (n < 0) return 0;
    return potrf_crt_workspace_bytes(n);
}

int mp_dd_Rpotrf_crt(const char *uplo, int64_t n, mp_dd_mat A, int64_t lda, int64_t *info,
                     void *workspace, size_t workspace_bytes) {
    clear_error();
    int ul = uplo_flag(uplo);
    if (ul < 0) return fail(-1, "Rpotrf_crt: illegal uplo");
    if (n < 0) return fail(-2, "Rpotrf_crt: n < 0");
    if (n > 0 && (A.hi == nullptr || A.lo == nullptr)) return fail(-3, "Rpotrf_crt: A is NULL");
    if (lda < imax(1, n)) return fail(-4, "Rpotrf_crt: lda < max(1, n)");
    if (info == nullptr) return fail(-5, "Rpotrf_crt: info is NULL");
    const size_t need = potrf_crt_workspace_bytes(n);
    if (need > 0 && (workspace == nullptr || workspace_bytes < need))
        return fail(MP_DD_ERR_WORKSPACE, "Rpotrf_crt needs %zu workspace bytes, got %zu", need,
                    workspace_bytes);
    int rc = require_device();
    if (rc) return rc;
    if (n == 0) {
        cudaError_t e = cudaMemsetAsync(info, 0, sizeof(int64_t), tls().stream);
        return e == cudaSuccess ? 0 : cuda_fail(e, "info reset");
    }
    return run_potrf(ul == 2, n, A.hi, A.lo, lda, info, tls().stream,
                     need > 0 ? workspace : nullptr, workspace_bytes);
}

int mp_dd_Rpotrs(const char *uplo, int64_t n, int64_t nrhs, mp_dd_cmat A, int64_t lda,
                 mp_dd_mat B, int64_t ldb, const int64_t *factor_info) {
    clear_error();
    int ul = uplo_flag(uplo);
    if (ul < 0) return fail(-1, "Rpotrs: illegal uplo");
    if (n < 0) return fail(-2, "Rpotrs: n < 0");
    if (nrhs < 0) return fail(-3, "Rpotrs: nrhs < 0");
    if (n > 0 && (A.hi == nullptr || A.lo == nullptr)) return fail(-4, "Rpotrs: A is NULL");
    if (lda < imax(1, n)) return fail(-5, "Rpotrs: lda < max(1, n)");
    if (n > 0 && nrhs > 0 && (B.hi == nullptr || B.lo == nullptr))
        return fail(-6, "Rpotrs: B is NULL");
    if (ldb < imax(1, n)) return fail(-7, "Rpotrs: ldb < max(1, n)");
    if (n == 0 || nrhs == 0) return 0;
    int rc = require_device();
    if (rc) return rc;
    return run_potrs(ul == 2, n, nrhs, A.hi, A.lo, lda, B.hi, B.lo, ldb, factor_info,
                     tls().stream);
}

int mp_dd_Rtrsm(const char *side, const char *uplo, const char *transa, const char *diag,
                int64_t m, int64_t n, mp_dd alpha, mp_dd_cmat A, int64_t lda, mp_dd_mat B,
                int64_t ldb) {
    clear_error();
    const int right = flag_is(side, 'R') ? 1 : flag_is(side, 'L') ? 0 : -1;
    if (right < 0) return fail(-1, "Rtrsm: illegal side");
    const int ul = uplo_flag(uplo);
    if (ul < 0) return fail(-2, "Rtrsm: illegal uplo");
    const int ta = trans_flag(transa);
    if (ta < 0) return fail(-3, "Rtrsm: illegal transa");
    const int unit = flag_is(diag, 'U') ? 1 : flag_is(diag, 'N') ? 0 : -1;
    if (unit < 0) return fail(-4, "Rtrsm: illegal diag");
    if (m < 0) return fail(-5, "Rtrsm: m < 0");
    if (n < 0) return fail(-6, "Rtrsm: n < 0");
    const int64_t order = right ? n : m;
    const bool work = m > 0 && n > 0;
    if (work && !dd_is_zero(alpha) && (A.hi == nullptr || A.lo == nullptr))
        return fail(-8, "Rtrsm: A is NULL");
    if (lda < imax(1, order)) return fail(-9, "Rtrsm: lda < max(1, order of A)");
    if (work && (B.hi == nullptr || B.lo == nullptr)) return fail(-10, "Rtrsm: B is NULL");
    if (ldb < imax(1, m)) return fail(-11, "Rtrsm: ldb < max(1, m)");
    if (!work) return 0;
    int rc = require_device();
    if (rc) return rc;
    cudaStream_t st = tls().stream;
    if (dd_is_zero(alpha)) {
        for (double *plane : {B.hi, B.lo}) {
            cudaError_t e = cudaMemset2DAsync(plane, (size_t)ldb * sizeof(double), 0,
                                              (size_t)m * sizeof(double), (size_t)n, st);
            if (e != cudaSuccess) return cuda_fail(e, "Rtrsm: zero B");
        }
        return 0;
    }
    return run_trsm(right, ul == 2, ta, unit, m, n, alpha, A.hi, A.lo, lda, B.hi, B.lo, ldb,
                    st);
}

int mp_dd_Rgetrf(int64_t m, int64_t n, mp_dd_mat A, int64_t lda, int64_t *ipiv,
                 int64_t *info) {
    clear_error();
    if (m < 0) return fail(-1, "Rgetrf: m < 0");
    if (n < 0) return fail(-2, "Rgetrf: n < 0");
    if (m > 0 && n > 0 && (A.hi == nullptr || A.lo == nullptr))
        return fail(-3, "Rgetrf: A is NULL");
    if (lda < imax(1, m)) return fail(-4, "Rgetrf: lda < max(1, m)");
    if (m > 0 && n > 0 && ipiv == nullptr) return fail(-5, "Rgetrf: ipiv is NULL");
    if (info == nullptr) return fail(-6, "Rgetrf: info is NULL");
    int rc = require_device();
    if (rc) return rc;
    cudaStream_t st = tls().stream;
    if (m == 0 || n == 0) {
        cudaError_t e = cudaMemsetAsync(info, 0, sizeof(int64_t), st);
        return e == cudaSuccess ? 0 : cuda_fail(e, "info reset");
    }
    return run_getrf(m, n, A.hi, A.lo, lda, ipiv, info, st);
}

int mp_dd_Rgetrs(const char *trans, int64_t n, int64_t nrhs, mp_dd_cmat A, int64_t lda,
                 const int64_t *ipiv, mp_dd_mat B, int64_t ldb) {
    clear_error();
    const int t = trans_flag(trans);
    if (t < 0) return fail(-1, "Rgetrs: illegal trans");
    if (n < 0) return fail(-2, "Rgetrs: n < 0");
    if (nrhs < 0) return fail(-3, "Rgetrs: nrhs < 0");
    const bool work = n > 0 && nrhs > 0;
    if (work && (A.hi == nullptr || A.lo == nullptr)) return fail(-4, "Rgetrs: A is NULL");
    if (lda < imax(1, n)) return fail(-5, "Rgetrs: lda < max(1, n)");
    if (work && ipiv == nullptr) return fail(-6, "Rgetrs: ipiv is NULL");
    if (work && (B.hi == nullptr || B.lo == nullptr)) return fail(-7, "Rgetrs: B is NULL");
    if (ldb < imax(1, n)) return fail(-8, "Rgetrs: ldb < max(1, n)");
    if (!work) return 0;
    int rc = require_device();
    if (rc) return rc;
    return run_getrs(t, n, nrhs, A.hi, A.lo, lda, ipiv, B.hi, B.lo, ldb, tls().stream);
}

int mp_dd_potrf_diag_batch(int64_t count, const mp_dd_potrf_diag_desc *descs) {
    clear_error();
    if (count < 0) return fail(-1, "potrf_diag_batch: count < 0");
    if (count > 0 && descs == nullptr) return fail(-2, "potrf_diag_batch: descs is NULL");
    int rc = require_device();
    if (rc) return rc;
    return launch_potrf_diag_batch(count, descs, tls().stream);
}

int mp_dd_trsm_batch(int64_t count, const mp_dd_trsm_desc *descs, int64_t max_nrhs) {
    clear_error();
    if (count < 0) return fail(-1, "trsm_batch: count < 0");
    if (count > 0 && descs == nullptr) return fail(-2, "trsm_batch: descs is NULL");
    if (max_nrhs < 0) return fail(-3, "trsm_batch: max_nrhs < 0");
    int rc = require_device();
    if (rc) return rc;
    return launch_trsm_batch(count, descs, max_nrhs, tls().stream);
}

size_t mp_dd_Rgemm_grouped_workspace(int64_t count, const mp_dd_gemm_desc *descs) {
    if (count < 0 || (count > 0 && descs == nullptr)) return 0;
    return grouped_workspace_bytes(count, descs);
}

int mp_dd_Rgemm_grouped_prepare(int64_t count, const mp_dd_gemm_desc *descs, void *workspace,
                                size_t workspace_bytes) {
    clear_error();
    if (count < 0) return fail(-1, "grouped_prepare: count < 0");
    if (count > 0 && descs == nullptr) return fail(-2, "grouped_prepare: descs is NULL");
    if (workspace == nullptr) return fail(-3, "grouped_prepare: workspace is NULL");
    int rc = require_device();
    if (rc) return rc;
    return grouped_prepare(count, descs, workspace, workspace_bytes, tls().stream);
}

int mp_dd_Rgemm_grouped_run(void *workspace) {
    clear_error();
    if (workspace == nullptr) return fail(-1, "grouped_run: workspace is NULL");
    int rc = require_device();
    if (rc) return rc;
    return grouped_run(workspace, tls().stream);
}

int mp_dd_sliced_timing(int enable) {
    clear_error();
    sliced_timing_enable(enable);
    return 0;
}

int mp_dd_sliced_phase_log(float *ms, int max_calls, int *calls) {
    clear_error();
    if (max_calls < 0) return fail(-2, "sliced_phase_log: max_calls < 0");
    if (ms == nullptr && max_calls > 0) return fail(-1, "sliced_phase_log: ms is NULL");
    if (calls == nullptr) return fail(-3, "sliced_phase_log: calls is NULL");
    return sliced_timing_log(ms, max_calls, calls);
}

int mp_dd_sliced_phase_ms(float ms[3]) {
    clear_error();
    if (ms == nullptr) return fail(-1, "sliced_phase_ms: ms is NULL");
    return sliced_timing_read(ms);
}

int mp_dd_elementwise(const char *op, int64_t n, mp_dd_cmat x, mp_dd_cmat y, mp_dd_mat z) {
    clear_error();
    static const char *names[] = {"add", "mul", "div", "divr", "sqrt", "rcp"};
    int code = -1;
    for (int i = 0; i < 6 && op != nullptr; ++i)
        if (strcmp(op, names[i]) == 0) code = i;
    if (code < 0) return fail(-1, "elementwise: unknown op");
    if (n < 0) return fail(-2, "elementwise: n < 0");
    if (n == 0) return 0;
    if (x.hi == nullptr || x.lo == nullptr) return fail(-3, "elementwise: x is NULL");
    if (code < 4 && (y.hi == nullptr || y.lo == nullptr)) return fail(-4, "elementwise: y is NULL");
    if (z.hi == nullptr || z.lo == nullptr) return fail(-5, "elementwise: z is NULL");
    int rc = require_device();
    if (rc) return rc;
    return run_dd_elementwise(code, n, x.hi, x.lo, y.hi, y.lo, z.hi, z.lo, tls().stream);
}

int mp_dd_set_plain_staging(int mode) {
    clear_error();
    if (mode < 0 || mode > 2) return fail(-1, "set_plain_staging: mode must be 0, 1 or 2");
    set_plain_staging(mode);
    return 0;
}

int mp_dd_set_band_pairs(int mode) {
    clear_error();
    if (mode < 0 || mode > 2) return fail(-1, "set_band_pairs: mode must be 0, 1 or 2");
    set_band_pairs(mode);
    return 0;
}

int mp_dd_peak_fp64(double *rate) {
    clear_error();
    if (rate == nullptr) return fail(-1, "peak_fp64: rate is NULL");
    int rc = require_device();
    if (rc) return rc;
    return run_peak_fp64(tls().stream, rate);
}

int mp_dd_peak_imma(double *rate) {
    clear_error();
    if (rate == nullptr) return fail(-1, "peak_imma: rate is NULL");
    int rc = require_device();
    if (rc) return rc;
    return run_peak_imma(tls().stream, rate);
}

int mp_dd_peak_ddmac(double *rate) {
    clear_error();
    if (rate == nullptr) return fail(-1, "peak_ddmac: rate is NULL");
    int rc = require_device();
    if (rc) return rc;
    return run_peak_ddmac(tls().stream, rate);
}

}  // extern "C"
