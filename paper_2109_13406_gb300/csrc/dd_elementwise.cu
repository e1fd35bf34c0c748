// Elementwise dd arithmetic on device arrays: the scalar operations of the
// dd format (the manual's Sec. 5: hi + lo binary64 pairs) exactly as the
// kernels of this library use them, so that each can be checked on its own
// against exact rational arithmetic.
#include "common.cuh"
#include "dd_arith.cuh"
#include "kernels.cuh"

namespace mpdd {
namespace {

__global__ void dd_elementwise_kernel(int op, int64_t n, const double *__restrict__ xh,
                                      const double *__restrict__ xl,
                                      const double *__restrict__ yh,
                                      const double *__restrict__ yl, double *zh, double *zl) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const dd x{xh[i], xl[i]};
    dd z{0.0, 0.0};
    switch (op) {
        case 0: z = add(x, dd{yh[i], yl[i]}); break;
        case 1: z = mul(x, dd{yh[i], yl[i]}); break;
        case 2: z = div(x, dd{yh[i], yl[i]}); break;
        case 3: z = div_rcp(x, dd{yh[i], yl[i]}, __drcp_rn(yh[i])); break;
        case 4: {
            double r;
            z = sqrt_dd(x, r);
            break;
        }
        case 5: z = rcp_dd(x); break;
        default: break;
    }
    zh[i] = z.hi;
    zl[i] = z.lo;
}

}  // namespace

int run_dd_elementwise(int op, int64_t n, const double *xh, const double *xl, const double *yh,
                       const double *yl, double *zh, double *zl, cudaStream_t st) {
    if (n == 0) return 0;
    const int64_t blocks = ceil_div(n, (int64_t)256);
    if (blocks > 0x7fffffffLL) return fail(MP_DD_ERR_TOO_LARGE, "elementwise: n too large");
    dd_elementwise_kernel<<<(unsigned)blocks, 256, 0, st>>>(op, n, xh, xl, yh, yl, zh, zl);
    return check_launch("dd_elementwise_kernel");
}

}  // namespace mpdd
