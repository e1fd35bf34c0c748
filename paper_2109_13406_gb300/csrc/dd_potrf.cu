// dd Cholesky factorisation and solve (Rpotrf / Rpotrs, MPLAPACK routine
// table of the manual's Sec. 6; the Rpotrf benchmark of Sec. 10.5), built as
// the LAPACK blocked right-looking algorithm on three kernels (and, with a
// workspace, in outer steps of 256 columns whose updates are residue-form
// products on the tensor cores), the triangular solve Rtrsm (MPBLAS,
// Sec. 6) on the same two of them, and, further below, the LU
// factorisation Rgetrf / Rgetrs:
//
//  * diag:  unblocked Cholesky of one nb x nb diagonal block (nb <= 64), in
//           registers, on a cluster of up to 8 CTAs per block;
//  * trsm:  triangular solve with one nb x nb factor block for 4 to 32
//           right-hand-side columns per CTA (forward with U^T, backward
//           with U), optionally scaling the right-hand sides by alpha and
//           taking the diagonal as unit;
//  * the trailing updates are the dd Rsyrk / Rgemm kernels.
//
// Storage follows LAPACK: uplo 'U' factors A = U^T U in the upper triangle,
// 'L' factors A = L L^T in the lower one.  Both are handled by one code path
// through an accessor: U(i, j) = A[i + j lda] for 'U' and A[j + i lda] (= L(j,
// i)) for 'L'; right-hand-side panels are accessed the same way.
//
// info (device int64, LAPACK convention): 0, or j > 0 when the leading minor
// of order j is not positive definite.  The first failing pivot is
// recorded; the launches that follow see info != 0 and leave their matrices
// untouched.
#include <cooperative_groups.h>

#include "common.cuh"
#include "dd_arith.cuh"
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace mpdd {
namespace {

constexpr int NB = 64;        // largest diagonal block
constexpr int NT = 256;

__host__ __device__ __forceinline__ int64_t uidx(int lower, int64_t i, int64_t j, int64_t ld) {
    return lower ? (j + i * ld) : (i + j * ld);
}

// Unblocked Cholesky of one nb x nb block (nb <= 64), right-looking, with
// the block's upper triangle in registers, on a cluster of CL CTAs.  The
// triangle's 2080 entries are numbered row by row (row r holds columns
// r..63) and thread g of the cluster (g = rank * 256 + tid) holds the
// entries g + 256 CL s as dd accumulators; the rows that are done form a
// prefix of that numbering, so a warp whose entries are all done issues
// nothing.  Step j: the holder of (j, j) takes the square root of its
// accumulator, with an approximate reciprocal of it, and writes both into
// every CTA's shared memory; after a cluster barrier the holders of row j
// divide by it (one binary64 division each, div_rcp) and write the row into
// every CTA (two buffers by the parity of j); after a second barrier every
// entry (r, c) with j < r <= c subtracts U(j, r) U(j, c), with the GEMM
// kernels' deferred renormalisation (every entry has taken exactly j + 1
// updates after step j, so all renormalise at the same steps).
//
// Every FP64 instruction costs a warp ~64 cycles on GB300 (2 FP64 lanes per
// clock per SM), so the square root / division chain is kept short and the
// update, which is FP64-throughput work, is spread over the CL SMs.
constexpr int kTri = NB * (NB + 1) / 2;

struct DiagSmem {
    double rh[2][NB], rl[2][NB];   // the pivot row U(j, :)
    double uh, ul, uz;             // U(j, j) and an approximate 1 / U(j, j)
    int fail;                      // a pivot failed (or info was set on entry)
};

__device__ __forceinline__ int tri_start(int r) { return r * NB - (r * (r - 1)) / 2; }

// acc[s] with a run-time s, without local memory
template <int S>
__device__ __forceinline__ dd pick(const dd (&acc)[S], int s) {
    dd v = acc[0];
#pragma unroll
    for (int q = 1; q < S; ++q)
        if (q == s) v = acc[q];
    return v;
}

template <int S>
__device__ __forceinline__ void put(dd (&acc)[S], int s, dd v) {
#pragma unroll
    for (int q = 0; q < S; ++q)
        if (q == s) acc[q] = v;
}

template <int CL>
struct DiagCluster {
    DiagSmem *peer[CL];   // every CTA's shared block (peer[rank] is our own)
    int rank;
    __device__ DiagCluster(DiagSmem &s) {
        if constexpr (CL > 1) {
            cg::cluster_group cl = cg::this_cluster();
            rank = (int)cl.block_rank();
#pragma unroll
            for (int r = 0; r < CL; ++r) peer[r] = cl.map_shared_rank(&s, (unsigned)r);
        } else {
            rank = 0;
            peer[0] = &s;
        }
    }
    __device__ void sync() const {
        if constexpr (CL > 1)
            cg::this_cluster().sync();
        else
            __syncthreads();
    }
};

template <int CL>
__device__ void potrf_diag_one(const mp_dd_potrf_diag_desc &d, DiagSmem &s) {
    constexpr int G = CL * NT;                       // threads of the cluster
    constexpr int kSl = (kTri + G - 1) / G;          // entries per thread
    const int nbe = d.n < NB ? (int)d.n : NB;        // (n > 64 is taken as 64)
    DiagCluster<CL> cl(s);
    const int g = cl.rank * NT + (int)threadIdx.x;
    // one decision for the whole cluster: an earlier block failed
    cl.sync();                                       // every CTA has started
    if (g == 0) {
        const int stop = d.info != nullptr && *d.info != 0;
#pragma unroll
        for (int r = 0; r < CL; ++r) cl.peer[r]->fail = stop;
    }
    cl.sync();
    if (s.fail) return;
    // the (row, column) of each entry this thread holds; c = NB marks none
    int er[kSl], ec[kSl];
    {
        int r = 0;
#pragma unroll
        for (int q = 0; q < kSl; ++q) {
            const int e = g + G * q;
            while (r < NB - 1 && tri_start(r + 1) <= e) ++r;
            const bool ok = e < kTri && r + (e - tri_start(r)) < nbe;
            er[q] = ok ? r : NB;
            ec[q] = ok ? r + (e - tri_start(r)) : NB;
        }
    }
    dd acc[kSl];
#pragma unroll
    for (int q = 0; q < kSl; ++q) {
        acc[q] = dd{0.0, 0.0};
        if (ec[q] < NB) {
            const int64_t o = uidx(d.lower, er[q], ec[q], d.lda);
            acc[q] = dd{d.a_hi[o], d.a_lo[o]};
        }
    }
    int jdone = nbe;
    for (int j = 0; j < nbe; ++j) {
        const int e0 = tri_start(j);                 // (j, j)
        if (g == e0 % G) {
            const int q = e0 / G;
            dd p = pick(acc, q);
            if (!(p.hi > 0.0)) {
                renorm(p);
                put(acc, q, p);
                if (d.info != nullptr)
                    atomicCAS(reinterpret_cast<unsigned long long *>(d.info), 0ull,
                              (unsigned long long)(d.offset + j + 1));
#pragma unroll
                for (int r = 0; r < CL; ++r) cl.peer[r]->fail = 1;
            } else {
                double z;
                const dd u = sqrt_dd(p, z);
                put(acc, q, u);
#pragma unroll
                for (int r = 0; r < CL; ++r) {
                    cl.peer[r]->uh = u.hi;
                    cl.peer[r]->ul = u.lo;
                    cl.peer[r]->uz = z;
                }
            }
        }
        cl.sync();
        if (s.fail) {                                // the same in every CTA
            jdone = j;
            break;
        }
        // row j: the entries e0 + 1 .. e0 + nbe - j - 1, at most one per thread
        {
            const int first = e0 + 1, count = nbe - j - 1;
            const int e = first + (g - first % G + G) % G;
            if (e < first + count) {
                const int q = e / G;
                const dd v = div_rcp(pick(acc, q), dd{s.uh, s.ul}, s.uz);
                put(acc, q, v);
                const int c = j + 1 + (e - first);
#pragma unroll
                for (int r = 0; r < CL; ++r) {
                    cl.peer[r]->rh[j & 1][c] = v.hi;
                    cl.peer[r]->rl[j & 1][c] = v.lo;
                }
            }
        }
        cl.sync();
        const bool renorm_now = (j & (kRenormEvery - 1)) == kRenormEvery - 1;
#pragma unroll
        for (int q = 0; q < kSl; ++q) {
            if (er[q] > j && ec[q] < NB) {
                const dd ur{-s.rh[j & 1][er[q]], -s.rl[j & 1][er[q]]};
                const dd uc{s.rh[j & 1][ec[q]], s.rl[j & 1][ec[q]]};
                mac_deferred(acc[q], ur, uc);
                if (renorm_now) renorm(acc[q]);
            }
        }
    }
    // rows r < jdone hold their final values; a failing pivot leaves the
    // rest partially updated (LAPACK leaves the trailing block unspecified)
#pragma unroll
    for (int q = 0; q < kSl; ++q) {
        if (ec[q] < NB) {
            dd v = acc[q];
            if (er[q] >= jdone) renorm(v);
            const int64_t o = uidx(d.lower, er[q], ec[q], d.lda);
            d.a_hi[o] = v.hi;
            d.a_lo[o] = v.lo;
        }
    }
    cl.sync();   // no CTA leaves while another may still address its shared memory
}

template <int CL>
__global__ void __launch_bounds__(NT) potrf_diag_batch_kernel(const mp_dd_potrf_diag_desc *ds) {
    extern __shared__ double smem_d[];
    potrf_diag_one<CL>(ds[blockIdx.x / CL], *reinterpret_cast<DiagSmem *>(smem_d));
}

template <int CL>
__global__ void __launch_bounds__(NT) potrf_diag_single_kernel(const mp_dd_potrf_diag_desc d) {
    extern __shared__ double smem_d[];
    potrf_diag_one<CL>(d, *reinterpret_cast<DiagSmem *>(smem_d));
}

// Cluster size for count diagonal blocks: the largest of 8, 4, 2 that keeps
// every cluster on its own SMs, else 1.
int diag_cluster(int64_t count) {
    const int64_t sms = sm_count() > 0 ? sm_count() : 152;
    for (int cl = 8; cl >= 2; cl /= 2)
        if (count * cl <= sms) return cl;
    return 1;
}

template <int CL>
int launch_diag_cl(const mp_dd_potrf_diag_desc *ds, int64_t count,
                   const mp_dd_potrf_diag_desc &d, cudaStream_t st) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)((ds != nullptr ? count : 1) * CL));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = sizeof(DiagSmem);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = ds != nullptr ? cudaLaunchKernelEx(&cfg, potrf_diag_batch_kernel<CL>, ds)
                                  : cudaLaunchKernelEx(&cfg, potrf_diag_single_kernel<CL>, d);
    if (e != cudaSuccess) return cuda_fail(e, "potrf diagonal-block launch");
    return check_launch("potrf_diag_kernel");
}

// One launch over count diagonal blocks (ds on the device) or of the single
// block d.
int launch_diag(const mp_dd_potrf_diag_desc *ds, int64_t count, const mp_dd_potrf_diag_desc &d,
                cudaStream_t st) {
    switch (diag_cluster(ds != nullptr ? count : 1)) {
        case 8: return launch_diag_cl<8>(ds, count, d, st);
        case 4: return launch_diag_cl<4>(ds, count, d, st);
        case 2: return launch_diag_cl<2>(ds, count, d, st);
        default: return launch_diag_cl<1>(ds, count, d, st);
    }
}

// ------------------------------------------------------------------ trsm

// B := alpha B before the solve when scale != 0.
struct TrsmScale {
    dd alpha;
    int scale;
};

__device__ __forceinline__ int col_start(int c) { return (c * (c + 1)) / 2; }

// Shared memory of one solve CTA with RG row groups: U's triangle packed
// (hi, lo) and the solved rows x_i of its NT / RG columns.
__host__ __device__ constexpr size_t trsm_smem_bytes(int rg) {
    return sizeof(double) * (2 * (size_t)kTri + 2 * (size_t)NB * (NT / rg) + NB);
}

// Solve U^T X = B (trans = 1) or U X = B (trans = 0) for the columns
// [c0, c0 + NT / RG) of B, in place.  U is the n x n upper factor block;
// with d.unit_diag its diagonal is taken as one and never read.
//
// Thread t owns column t % (NT / RG) and the rows t / (NT / RG) + RG q (q <
// 64 / RG) as dd accumulators in registers.  Step i: the owner of row i
// finishes x_i (its accumulator, divided by U(i, i)) and publishes it in
// shared memory; after one barrier every thread subtracts U-entry x_i from
// its rows still to be solved, with the deferred renormalisation of the GEMM
// kernels (TwoSum on the leading parts, a FastTwoSum every 4 steps).  U's
// triangle sits in shared memory packed in the order the steps read it: by
// rows for U^T (step i reads U(i, i+1:)), by columns for U (step i reads
// U(:i-1, i)).  Every row takes the same operations in the same order
// whatever RG is, so the result does not depend on it: RG only trades
// columns per CTA (32, 16, 8, 4) against the number of CTAs.
template <int TRANS, int RG>
__device__ void trsm_one(const mp_dd_trsm_desc &d, int64_t c0, double *sm, TrsmScale sc) {
    constexpr int COLS = NT / RG, RPT = NB / RG;
    double *uh = sm, *ul = sm + kTri, *xh = sm + 2 * kTri, *xl = xh + NB * COLS;
    double *rcp = xl + NB * COLS;   // 1 / U(i, i).hi
    const int n = d.n < NB ? (int)d.n : NB;   // (n > 64 is taken as 64)
    const int tid = threadIdx.x;
    if (d.info != nullptr && *d.info != 0) return;
    const int64_t ncol = d.nrhs - c0 < COLS ? d.nrhs - c0 : COLS;
    if (ncol <= 0) return;
    const int unit = d.unit_diag != 0;
    const int col = tid % COLS, rg = tid / COLS;
    const bool col_ok = col < ncol;
    for (int e = tid; e < n * n; e += NT) {
        const int r = e % n, c = e / n;
        if (r < c || (r == c && !unit)) {
            const int64_t o = uidx(d.lower_u, r, c, d.ldu);
            const int k = TRANS ? tri_start(r) + (c - r) : col_start(c) + r;
            uh[k] = d.u_hi[o];
            ul[k] = d.u_lo[o];
            if (r == c) rcp[r] = __drcp_rn(d.u_hi[o]);
        }
    }
    dd acc[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int r = rg + RG * q;
        acc[q] = dd{0.0, 0.0};
        if (r < n && col_ok) {
            const int64_t o = uidx(d.lower_b, r, c0 + col, d.ldb);
            acc[q] = dd{d.b_hi[o], d.b_lo[o]};
            if (sc.scale) acc[q] = mul(sc.alpha, acc[q]);
        }
    }
    __syncthreads();
    // rows in solve order: i = RG qq + ri, qq unrolled so that the owner's
    // accumulator acc[qq] has a compile-time index
    int step = 0;
#pragma unroll
    for (int qs = 0; qs < RPT; ++qs) {
        const int qq = TRANS ? qs : RPT - 1 - qs;
#pragma unroll 1
        for (int k = 0; k < RG; ++k) {
            const int ri = TRANS ? k : RG - 1 - k;
            const int i = RG * qq + ri;
            if (i >= n) continue;
            if (rg == ri && col_ok) {
                if (!unit) {
                    const int kd = TRANS ? tri_start(i) : col_start(i) + i;
                    acc[qq] = div_rcp(acc[qq], dd{uh[kd], ul[kd]}, rcp[i]);
                } else {
                    renorm(acc[qq]);
                }
                xh[i * COLS + col] = acc[qq].hi;
                xl[i * COLS + col] = acc[qq].lo;
            }
            __syncthreads();
            if (col_ok) {
                // eliminate x_i: U^T: rows r > i use U(i, r); U: rows r < i use U(r, i)
                const dd x{xh[i * COLS + col], xl[i * COLS + col]};
                const int base = TRANS ? tri_start(i) - i : col_start(i);
#pragma unroll
                for (int q = 0; q < RPT; ++q) {
                    const int r = rg + RG * q;
                    if (r < n && (TRANS ? r > i : r < i))
                        mac_deferred(acc[q], dd{-uh[base + r], -ul[base + r]}, x);
                }
                if ((step & (kRenormEvery - 1)) == kRenormEvery - 1) {
                    // rows still to be solved only: a solved row holds its
                    // normalised result, on which renorm changes nothing
#pragma unroll
                    for (int q = 0; q < RPT; ++q) {
                        const int r = rg + RG * q;
                        if (TRANS ? r > i : r < i) renorm(acc[q]);
                    }
                }
            }
            ++step;
        }
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int r = rg + RG * q;
        if (r < n && col_ok) {
            renorm(acc[q]);
            const int64_t o = uidx(d.lower_b, r, c0 + col, d.ldb);
            d.b_hi[o] = acc[q].hi;
            d.b_lo[o] = acc[q].lo;
        }
    }
}

template <int RG>
__device__ __forceinline__ void trsm_any(const mp_dd_trsm_desc &d, int64_t c0, double *sm,
                                         TrsmScale sc) {
    if (d.trans)
        trsm_one<1, RG>(d, c0, sm, sc);
    else
        trsm_one<0, RG>(d, c0, sm, sc);
}

template <int RG>
__global__ void __launch_bounds__(NT, 2) trsm_batch_kernel(const mp_dd_trsm_desc *ds) {
    extern __shared__ double smem_t[];
    trsm_any<RG>(ds[blockIdx.x], (int64_t)blockIdx.y * (NT / RG), smem_t,
                 TrsmScale{dd{1.0, 0.0}, 0});
}

template <int RG>
__global__ void __launch_bounds__(NT, 2) trsm_single_kernel(const mp_dd_trsm_desc d,
                                                         TrsmScale sc) {
    extern __shared__ double smem_t[];
    trsm_any<RG>(d, (int64_t)blockIdx.y * (NT / RG), smem_t, sc);
}

constexpr TrsmScale kNoScale{dd{1.0, 0.0}, 0};

// Row groups for count solves of nrhs columns.  Measured on GB300 (one
// 64-row solve of many columns; microseconds for an SM holding k resident
// CTAs of each width): a wide CTA (32 columns) makes the best use of the
// FP64 pipe once every SM has two of them, narrow ones win while the
// columns are too few to fill the SMs.  The cost of a choice is the busiest
// SM's: ceil(CTAs / SMs) CTAs in waves of the kernel's occupancy.  The
// cheapest is taken, or a wider one within 5 % of it.
constexpr int kRgCount = 4;                 // rg = 8, 16, 32, 64
constexpr float kSolveUs[kRgCount][5] = {
    {318.f, 552.f, 552.f, 552.f, 552.f},    // 32 columns per CTA (2 resident)
    {199.f, 311.f, 442.f, 442.f, 442.f},    // 16 (3 resident)
    {133.f, 186.f, 253.f, 330.f, 330.f},    //  8 (4 resident)
    {109.f, 147.f, 195.f, 244.f, 300.f},    //  4 (5 resident)
};
int g_trsm_occ[kRgCount] = {0, 0, 0, 0};    // resident CTAs per SM (0: not queried)

float trsm_cost(int idx, int64_t per_sm) {
    int occ = g_trsm_occ[idx];
    if (occ < 1) occ = 1;
    if (occ > 5) occ = 5;
    const int64_t full = per_sm / occ, rem = per_sm % occ;
    return (float)full * kSolveUs[idx][occ - 1] + (rem ? kSolveUs[idx][rem - 1] : 0.f);
}

int trsm_row_groups(int64_t count, int64_t nrhs) {
    const int64_t sms = sm_count() > 0 ? sm_count() : 152;
    float cost[kRgCount];
    int cheapest = 0;
    for (int idx = 0; idx < kRgCount; ++idx) {
        const int64_t cols = NT / (8 << idx);
        cost[idx] = trsm_cost(idx, ceil_div(count * ceil_div(nrhs, cols), sms));
        if (cost[idx] < cost[cheapest]) cheapest = idx;
    }
    for (int idx = 0; idx < cheapest; ++idx)      // wider, nearly as cheap
        if (cost[idx] <= 1.05f * cost[cheapest]) return 8 << idx;
    return 8 << cheapest;
}

// One launch of count solves (ds on the device) or of the single solve d.
int launch_trsm(const mp_dd_trsm_desc *ds, int64_t count, const mp_dd_trsm_desc &d,
                TrsmScale sc, int64_t nrhs, cudaStream_t st) {
    const int rg = trsm_row_groups(ds != nullptr ? count : 1, nrhs);
    const int64_t gy = ceil_div(nrhs, NT / rg);
    if (gy > 65535) return fail(MP_DD_ERR_TOO_LARGE, "too many right-hand sides");
    const dim3 grid(ds != nullptr ? (unsigned)count : 1u, (unsigned)gy);
    const size_t sm = trsm_smem_bytes(rg);
    switch (rg) {
#define MPDD_TRSM_CASE(RG)                                                  \
    case RG:                                                                \
        if (ds != nullptr)                                                  \
            trsm_batch_kernel<RG><<<grid, NT, sm, st>>>(ds);                \
        else                                                                \
            trsm_single_kernel<RG><<<grid, NT, sm, st>>>(d, sc);            \
        break;
        MPDD_TRSM_CASE(8) MPDD_TRSM_CASE(16) MPDD_TRSM_CASE(32) MPDD_TRSM_CASE(64)
#undef MPDD_TRSM_CASE
    }
    return check_launch(ds != nullptr ? "trsm_batch_kernel" : "trsm_single_kernel");
}

int launch_trsm_single(const mp_dd_trsm_desc &d, TrsmScale sc, cudaStream_t st) {
    return launch_trsm(nullptr, 1, d, sc, d.nrhs, st);
}

bool g_attr_done = false;

template <int RG>
cudaError_t trsm_attrs() {
    cudaError_t e = cudaFuncSetAttribute(trsm_batch_kernel<RG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)trsm_smem_bytes(RG));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(trsm_single_kernel<RG>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)trsm_smem_bytes(RG));
    return e;
}

int set_attrs() {
    if (g_attr_done) return 0;
    cudaError_t e = trsm_attrs<8>();
    if (e == cudaSuccess) e = trsm_attrs<16>();
    if (e == cudaSuccess) e = trsm_attrs<32>();
    if (e == cudaSuccess) e = trsm_attrs<64>();
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(potrf kernels)");
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_trsm_occ[0], trsm_batch_kernel<8>, NT,
                                                  trsm_smem_bytes(8));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_trsm_occ[1], trsm_batch_kernel<16>, NT,
                                                  trsm_smem_bytes(16));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_trsm_occ[2], trsm_batch_kernel<32>, NT,
                                                  trsm_smem_bytes(32));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_trsm_occ[3], trsm_batch_kernel<64>, NT,
                                                  trsm_smem_bytes(64));
    g_attr_done = true;
    return 0;
}

}  // namespace

int launch_potrf_diag_batch(int64_t count, const mp_dd_potrf_diag_desc *ds, cudaStream_t st) {
    if (count == 0) return 0;
    int rc = set_attrs();
    if (rc) return rc;
    if (count > 0x7fffffffLL) return fail(MP_DD_ERR_TOO_LARGE, "too many blocks");
    return launch_diag(ds, count, mp_dd_potrf_diag_desc{}, st);
}

int launch_trsm_batch(int64_t count, const mp_dd_trsm_desc *ds, int64_t max_rhs,
                      cudaStream_t st) {
    if (count == 0 || max_rhs == 0) return 0;
    int rc = set_attrs();
    if (rc) return rc;
    if (count > 0x7fffffffLL) return fail(MP_DD_ERR_TOO_LARGE, "too many solves");
    return launch_trsm(ds, count, mp_dd_trsm_desc{}, kNoScale, max_rhs, st);
}

// The blocked right-looking Cholesky (LAPACK dpotrf order) of the n x n
// block at (ah, al): 64-column steps of diagonal factor, panel solve and a
// plain dd Rsyrk trailing update.  off is the block's position in the whole
// matrix (for info).
int potrf_blocked(int lower, int64_t n, double *ah, double *al, int64_t lda, int64_t *info,
                  int64_t off, cudaStream_t st) {
    int rc = 0;
    for (int64_t j = 0; j < n; j += NB) {
        const int64_t nb = n - j < NB ? n - j : NB;
        mp_dd_potrf_diag_desc dg{};
        int64_t o = uidx(lower, j, j, lda);
        dg.a_hi = ah + o; dg.a_lo = al + o; dg.lda = lda; dg.n = nb; dg.offset = off + j;
        dg.info = info; dg.lower = lower;
        if ((rc = launch_diag(nullptr, 1, dg, st))) return rc;
        const int64_t rest = n - j - nb;
        if (rest <= 0) break;
        // panel: U(J, J+1:) := U_JJ^-T A(J, J+1:)
        mp_dd_trsm_desc tr{};
        tr.u_hi = ah + o; tr.u_lo = al + o; tr.ldu = lda;
        int64_t ob = uidx(lower, j, j + nb, lda);
        tr.b_hi = ah + ob; tr.b_lo = al + ob; tr.ldb = lda;
        tr.n = nb; tr.nrhs = rest; tr.trans = 1; tr.lower_u = lower; tr.lower_b = lower;
        tr.info = info;
        if ((rc = launch_trsm_single(tr, kNoScale, st))) return rc;
        // trailing: A(J+1:, J+1:) -= U(J, J+1:)^T U(J, J+1:) on the stored triangle
        GemmArgs p{};
        p.m = rest; p.n = rest; p.k = nb;
        p.alpha = mp_dd{-1.0, 0.0}; p.beta = mp_dd{1.0, 0.0};
        p.ah = ah + ob; p.al = al + ob; p.lda = lda;
        p.bh = ah + ob; p.bl = al + ob; p.ldb = lda;
        int64_t oc = uidx(lower, j + nb, j + nb, lda);
        p.ch = ah + oc; p.cl = al + oc; p.ldc = lda;
        // upper: C -= P^T P with P = U(J, J+1:) (nb x rest, column-major): (T, N)
        // lower: C -= P P^T with P = L(J+1:, J) (rest x nb): (N, T)
        p.ta = lower ? 0 : 1; p.tb = lower ? 1 : 0; p.tri = lower ? 2 : 1;
        p.alpha_zero = 0; p.alpha_one = 0; p.beta_zero = 0;
        p.info = info;
        if ((rc = launch_gemm_plain(p, st))) return rc;
    }
    return 0;
}

// The tensor-core form: outer steps of kOuter columns.  Each factors its
// diagonal block with potrf_blocked, solves its panel P = U(J, J+1:) by
// 64-row blocks, left-looking (block i first subtracts U_JJ(:i, i)^T
// P(:i, :), a residue-form Rgemm with k = 64 i, then takes the 64-row
// solve), and updates the trailing matrix with one residue-form Rsyrk of
// k = kOuter.  Against 64-column steps this reconstructs about a quarter as
// many entries (n^3 / (6 kOuter) instead of n^3 / 384) and runs the tensor
// products with four times the depth; updates of fewer than kCrtMinRest
// columns stay on the FP64 pipe.
constexpr int64_t kCrtMinRest = 512;
constexpr int64_t kOuter = 256;

size_t potrf_crt_workspace_bytes(int64_t n) {
    const int64_t rest = n - kOuter;
    if (rest < kCrtMinRest) return 0;
    size_t w = crt_workspace_bytes(rest, rest, kOuter, true);
    const size_t g1 = crt_workspace_bytes(NB, rest, kOuter - NB, false);
    const size_t g2 = crt_workspace_bytes(rest, NB, kOuter - NB, false);
    if (g1 > w) w = g1;
    if (g2 > w) w = g2;
    return w;
}

int potrf_crt(int lower, int64_t n, double *ah, double *al, int64_t lda, int64_t *info,
              cudaStream_t st, void *ws, size_t ws_bytes) {
    int rc = 0;
    for (int64_t J = 0; J < n; J += kOuter) {
        const int64_t nbo = n - J < kOuter ? n - J : kOuter;
        const int64_t oJ = uidx(lower, J, J, lda);
        if ((rc = potrf_blocked(lower, nbo, ah + oJ, al + oJ, lda, info, J, st))) return rc;
        const int64_t rest = n - J - nbo;
        if (rest <= 0) break;
        const bool crt = rest >= kCrtMinRest;
        const int64_t oP = uidx(lower, J, J + nbo, lda);      // the panel
        for (int64_t i = 0; i < nbo; i += NB) {
            const int64_t nb = nbo - i < NB ? nbo - i : NB;
            if (i > 0) {
                GemmArgs p{};
                p.k = i;
                p.alpha = mp_dd{-1.0, 0.0}; p.beta = mp_dd{1.0, 0.0};
                p.alpha_zero = 0; p.alpha_one = 0; p.beta_zero = 0; p.tri = 0;
                p.info = info;
                const int64_t oC = uidx(lower, J + i, J + nbo, lda);
                const int64_t oU = uidx(lower, J, J + i, lda);  // U_JJ(:i, i:i+nb)
                p.ch = ah + oC; p.cl = al + oC; p.ldc = lda;
                if (!lower) {
                    // U(J+i, J+nbo:) (nb x rest) -= U_JJ(:i, i:)^T (nb x i) P(:i, :) (i x rest)
                    p.m = nb; p.n = rest; p.ta = 1; p.tb = 0;
                    p.ah = ah + oU; p.al = al + oU; p.lda = lda;
                    p.bh = ah + oP; p.bl = al + oP; p.ldb = lda;
                } else {
                    // L(J+nbo:, J+i) (rest x nb) -= P(:, :i) (rest x i) L_JJ(i:, :i)^T (i x nb)
                    p.m = rest; p.n = nb; p.ta = 0; p.tb = 1;
                    p.ah = ah + oP; p.al = al + oP; p.lda = lda;
                    p.bh = ah + oU; p.bl = al + oU; p.ldb = lda;
                }
                rc = crt ? run_crt(p, ws, ws_bytes, st) : launch_gemm_plain(p, st);
                if (rc) return rc;
            }
            mp_dd_trsm_desc tr{};
            const int64_t od = uidx(lower, J + i, J + i, lda);
            const int64_t ob = uidx(lower, J + i, J + nbo, lda);
            tr.u_hi = ah + od; tr.u_lo = al + od; tr.ldu = lda;
            tr.b_hi = ah + ob; tr.b_lo = al + ob; tr.ldb = lda;
            tr.n = nb; tr.nrhs = rest; tr.trans = 1; tr.lower_u = lower; tr.lower_b = lower;
            tr.info = info;
            if ((rc = launch_trsm_single(tr, kNoScale, st))) return rc;
        }
        // trailing: A(J+1:, J+1:) -= P^T P (upper) / P P^T (lower), k = nbo
        GemmArgs p{};
        p.m = rest; p.n = rest; p.k = nbo;
        p.alpha = mp_dd{-1.0, 0.0}; p.beta = mp_dd{1.0, 0.0};
        p.ah = ah + oP; p.al = al + oP; p.lda = lda;
        p.bh = ah + oP; p.bl = al + oP; p.ldb = lda;
        const int64_t oC = uidx(lower, J + nbo, J + nbo, lda);
        p.ch = ah + oC; p.cl = al + oC; p.ldc = lda;
        p.ta = lower ? 0 : 1; p.tb = lower ? 1 : 0; p.tri = lower ? 2 : 1;
        p.alpha_zero = 0; p.alpha_one = 0; p.beta_zero = 0;
        p.info = info;
        rc = crt ? run_crt(p, ws, ws_bytes, st) : launch_gemm_plain(p, st);
        if (rc) return rc;
    }
    return 0;
}

// Cholesky of one matrix; with a workspace (ws != nullptr) the tensor-core
// form above.
int run_potrf(int lower, int64_t n, double *ah, double *al, int64_t lda, int64_t *info,
              cudaStream_t st, void *ws, size_t ws_bytes) {
    int rc = set_attrs();
    if (rc) return rc;
    if (info != nullptr) {
        cudaError_t e = cudaMemsetAsync(info, 0, sizeof(int64_t), st);
        if (e != cudaSuccess) return cuda_fail(e, "info reset");
    }
    if (ws != nullptr) return potrf_crt(lower, n, ah, al, lda, info, st, ws, ws_bytes);
    return potrf_blocked(lower, n, ah, al, lda, info, 0, st);
}

// Solve A X = B with the factor of run_potrf (blocked forward and backward
// substitution; updates through the plain dd Rgemm kernel).
int run_potrs(int lower, int64_t n, int64_t nrhs, const double *ah, const double *al,
              int64_t lda, double *bh, double *bl, int64_t ldb, const int64_t *info,
              cudaStream_t st) {
    int rc = set_attrs();
    if (rc) return rc;
    const int64_t nblk = ceil_div(n, NB);
    auto solve_block = [&](int64_t j, int trans) -> int {
        const int64_t nb = n - j < NB ? n - j : NB;
        mp_dd_trsm_desc tr{};
        int64_t o = uidx(lower, j, j, lda);
        tr.u_hi = ah + o; tr.u_lo = al + o; tr.ldu = lda;
        tr.b_hi = bh + j; tr.b_lo = bl + j; tr.ldb = ldb;
        // B is a plain n x nrhs matrix (column-major whatever uplo is); U is
        // read through the factor accessor
        tr.n = nb; tr.nrhs = nrhs; tr.trans = trans; tr.lower_u = lower; tr.lower_b = 0;
        tr.info = info;
        return launch_trsm_single(tr, kNoScale, st);
    };
    auto update = [&](int64_t j, int forward) -> int {
        const int64_t nb = n - j < NB ? n - j : NB;
        GemmArgs p{};
        p.alpha = mp_dd{-1.0, 0.0}; p.beta = mp_dd{1.0, 0.0};
        p.alpha_zero = 0; p.alpha_one = 0; p.beta_zero = 0; p.tri = 0; p.info = info;
        if (forward) {
            // B(J+1:) -= U(J, J+1:)^T B(J)
            const int64_t rest = n - j - nb;
            if (rest <= 0) return 0;
            int64_t ou = uidx(lower, j, j + nb, lda);
            p.m = rest; p.n = nrhs; p.k = nb;
            p.ah = ah + ou; p.al = al + ou; p.lda = lda;
            p.ta = lower ? 0 : 1;   // upper: U(J, J+1:) is nb x rest -> transpose
            p.bh = bh + j; p.bl = bl + j; p.ldb = ldb; p.tb = 0;
            p.ch = bh + j + nb; p.cl = bl + j + nb; p.ldc = ldb;
        } else {
            // B(0:J) -= U(0:J, J) B(J)
            if (j == 0) return 0;
            int64_t ou = uidx(lower, 0, j, lda);
            p.m = j; p.n = nrhs; p.k = nb;
            p.ah = ah + ou; p.al = al + ou; p.lda = lda;
            p.ta = lower ? 1 : 0;   // upper: U(0:J, J) is j x nb as stored
            p.bh = bh + j; p.bl = bl + j; p.ldb = ldb; p.tb = 0;
            p.ch = bh; p.cl = bl; p.ldc = ldb;
        }
        return launch_gemm_plain(p, st);
    };
    for (int64_t b = 0; b < nblk; ++b) {
        if ((rc = solve_block(b * NB, 1))) return rc;
        if ((rc = update(b * NB, 1))) return rc;
    }
    for (int64_t b = nblk - 1; b >= 0; --b) {
        if ((rc = solve_block(b * NB, 0))) return rc;
        if ((rc = update(b * NB, 0))) return rc;
    }
    return 0;
}

// ------------------------------------------------------------------ Rtrsm
//
// Every DTRSM variant is one triangular system T Y = B' with several
// right-hand sides: for side 'L' T = op(A) and B' = B; for side 'R'
// X op(A) = B is op(A)^T X^T = B^T, so T = op(A)^T and B' = B^T (read
// through the transposed accessor).  T is then either U^T (lower: forward
// substitution) or U (upper: backward substitution) for the upper-stored
// view U(r, c) = A[uidx(lower_a, r, c)] of A's triangle.  The solve splits
// T recursively into halves (at multiples of 64): solve the first half,
// update the second half's right-hand sides with one dd Rgemm of the whole
// off-diagonal block, solve the second half.  The leaves are 64 x 64
// diagonal blocks in shared memory.  alpha is applied where each row block
// of B' is first touched: by the leaf kernel (the first block) or as the
// beta of its first Rgemm update.

namespace {

struct TrsmPlan {
    int lower_a;   // A's triangle is 'L' (read through the transposed accessor)
    int forward;   // T is lower: forward substitution
    int right;     // B' = B^T
    int unit;
    const double *ah, *al;
    int64_t lda;
    double *bh, *bl;
    int64_t ldb;
    int64_t nrhs;  // columns of B'
    mp_dd alpha;
    int alpha_one;
    cudaStream_t st;
};

int trsm_leaf(const TrsmPlan &P, int64_t j0, int64_t nt, bool first) {
    mp_dd_trsm_desc tr{};
    const int64_t o = uidx(P.lower_a, j0, j0, P.lda);
    tr.u_hi = P.ah + o; tr.u_lo = P.al + o; tr.ldu = P.lda;
    const int64_t ob = uidx(P.right, j0, 0, P.ldb);
    tr.b_hi = P.bh + ob; tr.b_lo = P.bl + ob; tr.ldb = P.ldb;
    tr.n = nt; tr.nrhs = P.nrhs; tr.trans = P.forward; tr.lower_u = P.lower_a;
    tr.lower_b = P.right; tr.unit_diag = P.unit; tr.info = nullptr;
    const TrsmScale sc{dd{P.alpha.hi, P.alpha.lo}, first && !P.alpha_one};
    return launch_trsm_single(tr, sc, P.st);
}

// B'(rows r0 .. r0+mr) -= T(rows, cols c0 .. c0+kc) B'(cols), with beta = alpha
// when these rows are touched for the first time.
int trsm_update(const TrsmPlan &P, int64_t r0, int64_t mr, int64_t c0, int64_t kc,
                bool first) {
    // T(r, c) off the diagonal is A[uidx(tl, r, c)]: as stored (tl = 0) or
    // transposed (tl = 1); the block starts at uidx(tl, r0, c0)
    const int tl = P.lower_a ^ P.forward;
    const int64_t ot = uidx(tl, r0, c0, P.lda);
    GemmArgs p{};
    p.alpha = mp_dd{-1.0, 0.0};
    p.beta = first ? P.alpha : mp_dd{1.0, 0.0};
    p.alpha_zero = 0; p.alpha_one = 0; p.beta_zero = 0; p.tri = 0; p.info = nullptr;
    if (!P.right) {
        // B(r0:, :) -= T_sub B(c0:, :)
        p.m = mr; p.n = P.nrhs; p.k = kc;
        p.ah = P.ah + ot; p.al = P.al + ot; p.lda = P.lda; p.ta = tl;
        p.bh = P.bh + c0; p.bl = P.bl + c0; p.ldb = P.ldb; p.tb = 0;
        p.ch = P.bh + r0; p.cl = P.bl + r0; p.ldc = P.ldb;
    } else {
        // B(:, r0:) -= B(:, c0:) T_sub^T
        p.m = P.nrhs; p.n = mr; p.k = kc;
        p.ah = P.bh + c0 * P.ldb; p.al = P.bl + c0 * P.ldb; p.lda = P.ldb; p.ta = 0;
        p.bh = P.ah + ot; p.bl = P.al + ot; p.ldb = P.lda; p.tb = !tl;
        p.ch = P.bh + r0 * P.ldb; p.cl = P.bl + r0 * P.ldb; p.ldc = P.ldb;
    }
    return launch_gemm_plain(p, P.st);
}

int trsm_rec(const TrsmPlan &P, int64_t j0, int64_t nt, bool first) {
    if (nt <= NB) return trsm_leaf(P, j0, nt, first);
    const int64_t h = ceil_div(nt / 2, (int64_t)NB) * NB;   // 64 <= h < nt
    int rc;
    if (P.forward) {
        if ((rc = trsm_rec(P, j0, h, first))) return rc;
        if ((rc = trsm_update(P, j0 + h, nt - h, j0, h, first))) return rc;
        return trsm_rec(P, j0 + h, nt - h, false);
    }
    if ((rc = trsm_rec(P, j0 + h, nt - h, first))) return rc;
    if ((rc = trsm_update(P, j0, h, j0 + h, nt - h, first))) return rc;
    return trsm_rec(P, j0, h, false);
}

}  // namespace

int run_trsm(int right, int lower, int trans, int unit, int64_t m, int64_t n, mp_dd alpha,
             const double *ah, const double *al, int64_t lda, double *bh, double *bl,
             int64_t ldb, cudaStream_t st) {
    int rc = set_attrs();
    if (rc) return rc;
    TrsmPlan P{};
    P.lower_a = lower;
    P.forward = lower ^ trans ^ right;
    P.right = right;
    P.unit = unit;
    P.ah = ah; P.al = al; P.lda = lda;
    P.bh = bh; P.bl = bl; P.ldb = ldb;
    P.nrhs = right ? m : n;
    P.alpha = alpha;
    P.alpha_one = alpha.hi == 1.0 && alpha.lo == 0.0;
    P.st = st;
    return trsm_rec(P, 0, right ? n : m, true);
}

// ------------------------------------------------------------------ Rgetrf
//
// LU factorisation with partial pivoting, P A = L U (DGETRF semantics), by
// the recursive column splitting of LAPACK's dgetrf2: factor the left half
// of the columns (recursively), solve L11 U12 = A12 (the Rtrsm above, unit
// lower), update A22 -= L21 U12 (the plain dd Rgemm kernel, or a
// one-thread-per-entry kernel when k or n is small), factor A22
// (recursively).  The leaves are panels of at most 32 columns, each one
// cooperative launch (getrf_panel_kernel below) followed by one launch that
// applies its interchanges to the other columns; where that kernel cannot
// run (no cooperative launch, or more than 1024 rows per CTA) a single
// column is the leaf: one CTA finds the pivot (the first row of largest
// |A(i, j)|, compared as dd values) and records it, then a second launch
// interchanges the two rows across the whole matrix and forms the
// multipliers.  dgetrf2 applies each half's interchanges to the other half
// as a block afterwards; applying them to all other columns at the leaf
// gives the same matrix, because nothing reads or writes the other half in
// between.  The top-level updates are large products; the leaves and the
// thin updates near them are latency-bound.

namespace {

constexpr int LT = 256;   // threads of the pivot-column kernel

// Pivot candidates: |x| of a normalised dd x orders by |hi| first (compared
// as the integer bit pattern, off the FP64 pipe), then by lo taken with the
// sign of hi; ties go to the lower row (the first maximum, as idamax).
struct PivotKey {
    uint64_t mag;   // |hi| bits
    double lo;      // lo * sign(hi)
    int64_t row;    // -1: none
};

__device__ __forceinline__ PivotKey pivot_key(double hi, double lo, int64_t row) {
    const uint64_t b = (uint64_t)__double_as_longlong(hi);
    return PivotKey{b & 0x7fffffffffffffffull, (b >> 63) ? -lo : lo, row};
}

// b is the better pivot than a
__device__ __forceinline__ bool better(const PivotKey &b, const PivotKey &a) {
    if (b.row < 0) return false;
    if (a.row < 0) return true;
    if (b.mag != a.mag) return b.mag > a.mag;
    if (b.lo != a.lo) return b.lo > a.lo;
    return b.row < a.row;
}

// Column j (global) of A, rows [j, m), in two launches.
//
// getrf_pivot_kernel (one CTA): the pivot row p, ipiv[j] = p + 1, and the
// interchange of the two entries of column j; a zero pivot records info and
// changes nothing (LAPACK: no interchange, no scaling).
__global__ void __launch_bounds__(LT) getrf_pivot_kernel(double *ah, double *al, int64_t lda,
                                                         int64_t m, int64_t j, int64_t *ipiv,
                                                         int64_t *info) {
    __shared__ PivotKey wk[LT / 32];
    double *ch = ah + j * lda, *cl = al + j * lda;
    PivotKey best{0, 0.0, -1};
    for (int64_t i = j + threadIdx.x; i < m; i += LT) {
        const PivotKey c = pivot_key(ch[i], cl[i], i);
        if (better(c, best)) best = c;
    }
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
    for (int off = 16; off > 0; off /= 2) {
        PivotKey o{__shfl_down_sync(0xffffffffu, best.mag, off),
                   __shfl_down_sync(0xffffffffu, best.lo, off),
                   __shfl_down_sync(0xffffffffu, best.row, off)};
        if (better(o, best)) best = o;
    }
    if (lane == 0) wk[warp] = best;
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int w = 1; w < LT / 32; ++w)
        if (better(wk[w], best)) best = wk[w];
    const int64_t p = best.row;
    ipiv[j] = p + 1;
    const double ph = ch[p], pl = cl[p];
    if (ph == 0.0 && pl == 0.0) {
        atomicCAS(reinterpret_cast<unsigned long long *>(info), 0ull, (unsigned long long)(j + 1));
        return;
    }
    if (p != j) {
        ch[p] = ch[j]; cl[p] = cl[j];
        ch[j] = ph; cl[j] = pl;
    }
}

// getrf_apply_kernel: with the pivot in place at A(j, j), CTAs [0, col_ctas)
// interchange rows j and p in every other column of A (one column per
// thread), the rest form the multipliers of column j below the diagonal, as
// LAPACK's dgetf2 does: one dd reciprocal of the pivot per CTA, then a product
// per entry (a division per entry when the pivot is below 2^-1021, where the
// reciprocal could overflow).  Column j's entries are read and written by
// one thread each, so the two roles never touch the same entry.
__global__ void __launch_bounds__(LT) getrf_apply_kernel(double *ah, double *al, int64_t lda,
                                                         int64_t m, int64_t n, int64_t j,
                                                         const int64_t *ipiv, int col_ctas) {
    __shared__ double rh, rl;
    const double ph = ah[j + j * lda], pl = al[j + j * lda];
    if (ph == 0.0 && pl == 0.0) return;   // zero pivot: nothing to apply
    const int64_t p = ipiv[j] - 1;
    if ((int)blockIdx.x < col_ctas) {
        const int64_t c = (int64_t)blockIdx.x * LT + threadIdx.x;
        if (p == j || c >= n || c == j) return;
        const int64_t oj = j + c * lda, op = p + c * lda;
        const double th = ah[oj], tl = al[oj];
        ah[oj] = ah[op]; al[oj] = al[op];
        ah[op] = th; al[op] = tl;
        return;
    }
    const bool recip = fabs(ph) >= 0x1p-1021;
    if (threadIdx.x == 0 && recip) {
        const dd r = div(dd{1.0, 0.0}, dd{ph, pl});
        rh = r.hi;
        rl = r.lo;
    }
    __syncthreads();
    const int64_t i = j + 1 + (int64_t)(blockIdx.x - col_ctas) * LT + threadIdx.x;
    if (i >= m) return;
    double *wh = ah + j * lda, *wl = al + j * lda;
    const dd v = recip ? mul(dd{wh[i], wl[i]}, dd{rh, rl}) : div(dd{wh[i], wl[i]}, dd{ph, pl});
    wh[i] = v.hi;
    wl[i] = v.lo;
}

// Row interchanges ipiv[k0 .. k1) (one-based global rows, applied in order)
// on columns [c0, c1) of A: one thread per column.
__global__ void laswp_kernel(double *ah, double *al, int64_t lda, int64_t c0, int64_t c1,
                             const int64_t *ipiv, int64_t k0, int64_t k1, int reverse) {
    const int64_t c = c0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= c1) return;
    double *ch = ah + c * lda, *cl = al + c * lda;
    for (int64_t t = 0; t < k1 - k0; ++t) {
        const int64_t k = reverse ? k1 - 1 - t : k0 + t;
        const int64_t p = ipiv[k] - 1;
        if (p != k) {
            double th = ch[k], tl = cl[k];
            ch[k] = ch[p]; cl[k] = cl[p];
            ch[p] = th; cl[p] = tl;
        }
    }
}

// The interchanges ipiv[k0 .. k1) (k1 - k0 <= 32, one-based, applied in
// order) on the columns [0, c_skip) and [c_skip + n_skip, n_all) of A.  The
// rows they touch (at most 64) and where each one's final content comes
// from are worked out once per CTA; then each thread moves one (row,
// column) entry: all loads, a barrier, all stores, instead of a chain of
// dependent swaps per column.
__global__ void __launch_bounds__(256) laswp_perm_kernel(double *ah, double *al, int64_t lda,
                                                         int64_t c_skip, int64_t n_skip,
                                                         int64_t n_all, const int64_t *ipiv,
                                                         int64_t k0, int64_t k1) {
    __shared__ int64_t S[64], src[64];
    __shared__ int ns;
    if (threadIdx.x == 0) {
        const int nk = (int)(k1 - k0);
        int cnt = nk;
        for (int t = 0; t < nk; ++t) S[t] = src[t] = k0 + t;
        for (int t = 0; t < nk; ++t) {
            const int64_t p = ipiv[k0 + t] - 1;
            int ip = -1;
            if (p >= k0 && p < k1) {
                ip = (int)(p - k0);
            } else {
                for (int q = nk; q < cnt; ++q)
                    if (S[q] == p) ip = q;
                if (ip < 0) {
                    ip = cnt++;
                    S[ip] = src[ip] = p;
                }
            }
            const int64_t tmp = src[t];
            src[t] = src[ip];
            src[ip] = tmp;
        }
        ns = cnt;
    }
    __syncthreads();
    const int i = (int)(threadIdx.x % 64);
    const int64_t q = (int64_t)blockIdx.x * 4 + threadIdx.x / 64;
    const int64_t c = q < c_skip ? q : q + n_skip;
    const bool act = i < ns && c < n_all && src[i] != S[i];
    double vh = 0.0, vl = 0.0;
    if (act) {
        vh = ah[src[i] + c * lda];
        vl = al[src[i] + c * lda];
    }
    __syncthreads();
    if (act) {
        ah[S[i] + c * lda] = vh;
        al[S[i] + c * lda] = vl;
    }
}

// C(m x n) -= A(m x k) B(k x n), all column-major, for small k or n: one
// thread per entry of C, multiply-adds l = 0 .. k-1 straight into C's value.
// (The 64 x 64 tiles of the Rgemm kernel would compute zero-padded products
// worth up to 16 / k and 64 / n times the useful ones.)
__global__ void __launch_bounds__(256) small_update_kernel(
    int64_t m, int64_t n, int64_t k, const double *__restrict__ ah,
    const double *__restrict__ al, int64_t lda, const double *__restrict__ bh,
    const double *__restrict__ bl, int64_t ldb, double *ch, double *cl, int64_t ldc) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * n) return;
    const int64_t i = e % m, j = e / m;
    dd acc{ch[i + j * ldc], cl[i + j * ldc]};
    for (int64_t l = 0; l < k; ++l)
        mac(acc, dd{-ah[i + l * lda], -al[i + l * lda]}, dd{bh[l + j * ldb], bl[l + j * ldb]});
    ch[i + j * ldc] = acc.hi;
    cl[i + j * ldc] = acc.lo;
}

constexpr int64_t kSmallUpdate = 16;   // k or n at or below this: small_update_kernel

// ---- panel of up to 32 columns in one cooperative launch
//
// getrf_panel_kernel factors the columns [j0, j0 + w) over the rows
// [j0, m) (dgetf2 on the panel: pivot, interchange within the panel,
// multipliers by the reciprocal of the pivot, rank-1 update) with every CTA
// of the grid co-resident.  CTA c owns the rows [j0 + c R, j0 + (c + 1) R).
// Per column j one grid barrier: before it, every CTA publishes its best
// candidate (key, the whole panel row, the candidate's dd reciprocal) and
// the owner of row j publishes row j; after it, every CTA picks the same
// pivot from the published keys and updates its own rows, the owner of row
// j taking the pivot row and the owner of row p taking row j's.  The
// published buffers alternate by the parity of j: a CTA overwrites a
// buffer only after the next barrier, which every reader of its previous
// contents has passed.  Interchanges outside the panel follow as one
// laswp.  Each barrier wait is bounded (~2 s): a CTA that gives up raises
// an abort flag that ends every CTA's loop, and info is set to -1.
constexpr int kPanelW = 32;
constexpr int kPanelMaxG = 256;
constexpr int kPanelThreads = 256;

struct PanelCand {
    uint64_t mag;
    double lo;
    int64_t row;                 // -1: no candidate in this CTA
    double rh, rl;               // dd reciprocal of the candidate
    double vh[kPanelW], vl[kPanelW];
};

struct PanelWs {
    unsigned int count;          // grid-barrier arrivals (zeroed before the launch)
    unsigned int abort;          // a wait gave up
    double rjh[2][kPanelW], rjl[2][kPanelW];
    PanelCand cand[2][kPanelMaxG];
};

// Thread 0 of each CTA: arrive, then wait for all G arrivals of barrier b
// (b = 1, 2, ...).  false: the wait gave up or another CTA did.
__device__ bool panel_grid_sync(PanelWs *ws, int G, unsigned int b) {
    __threadfence();
    atomicAdd(&ws->count, 1u);
    const unsigned int target = b * (unsigned int)G;
    const long long t0 = clock64();
    volatile unsigned int *cnt = &ws->count, *ab = &ws->abort;
    while (*cnt < target) {
        if (*ab) return false;
        if (clock64() - t0 > 4000000000LL) {
            atomicExch(&ws->abort, 1u);
            return false;
        }
        __nanosleep(64);
    }
    __threadfence();
    return true;
}

// The best pivot key over a warp's lanes, with the slot it came from:
// every lane ends with the same winner (keys of distinct rows are totally
// ordered by better()).
__device__ __forceinline__ void warp_best(PivotKey &k, int &slot) {
    for (int off = 16; off > 0; off /= 2) {
        const PivotKey o{__shfl_xor_sync(0xffffffffu, k.mag, off),
                         __shfl_xor_sync(0xffffffffu, k.lo, off),
                         __shfl_xor_sync(0xffffffffu, k.row, off)};
        const int os = __shfl_xor_sync(0xffffffffu, slot, off);
        if (better(o, k) || (!better(k, o) && o.row == k.row && os < slot)) {
            k = o;
            slot = os;
        }
    }
}

__global__ void __launch_bounds__(kPanelThreads) getrf_panel_kernel(
    double *ah, double *al, int64_t lda, int64_t m, int64_t j0, int w, int64_t R,
    int64_t *ipiv, int64_t *info, PanelWs *ws) {
    __shared__ double lh[1024], ll[1024];      // the multipliers of this CTA's rows (R <= 1024)
    __shared__ int s_stop;
    __shared__ int64_t s_p;
    __shared__ double s_rh, s_rl;
    __shared__ double pvh[kPanelW], pvl[kPanelW];   // the pivot row
    __shared__ double jvh[kPanelW], jvl[kPanelW];   // row j before the interchange
    const int G = (int)gridDim.x, c = (int)blockIdx.x, tid = (int)threadIdx.x;
    const int lane = tid % 32, warp = tid / 32;
    const int64_t rs = j0 + (int64_t)c * R;
    const int64_t re = rs + R < m ? rs + R : m;
    const int mn = (int)((m - j0) < w ? (m - j0) : w);   // columns that take a pivot
    double *Ah = ah + j0 * lda, *Al = al + j0 * lda;   // column jj of the panel: + jj * lda
    for (int jj = 0; jj < mn; ++jj) {
        const int64_t j = j0 + jj;
        const int par = jj & 1;
        // 1. warp 0: this CTA's best candidate in column j (rows max(j, rs) ..
        //    re) and its publication (key, panel row, dd reciprocal); warp 1:
        //    row j, by its owner.  The published buffers are written and
        //    read at L2, past L1: other CTAs write them between our reads.
        if (warp == 0) {
            PivotKey best{0, 0.0, -1};
            int dummy = 0;
            for (int64_t i = (j > rs ? j : rs) + lane; i < re; i += 32) {
                const PivotKey k = pivot_key(Ah[i + jj * lda], Al[i + jj * lda], i);
                if (better(k, best)) best = k;
            }
            warp_best(best, dummy);
            PanelCand &pc = ws->cand[par][c];
            if (best.row >= 0 && lane < w) {
                __stcg(&pc.vh[lane], Ah[best.row + lane * lda]);
                __stcg(&pc.vl[lane], Al[best.row + lane * lda]);
            }
            if (lane == 0) {
                double rh = 0.0, rl = 0.0;
                if (best.row >= 0) {
                    const double ph = Ah[best.row + jj * lda], pl = Al[best.row + jj * lda];
                    if (fabs(ph) >= 0x1p-1021) {
                        const dd r = rcp_dd(dd{ph, pl});
                        rh = r.hi;
                        rl = r.lo;
                    }
                }
                __stcg(&pc.rh, rh);
                __stcg(&pc.rl, rl);
                __stcg(reinterpret_cast<unsigned long long *>(&pc.mag),
                       (unsigned long long)best.mag);
                __stcg(&pc.lo, best.lo);
                __stcg(reinterpret_cast<long long *>(&pc.row), (long long)best.row);
            }
            __threadfence();
        } else if (warp == 1) {
            if (j >= rs && j < re && lane < w) {
                __stcg(&ws->rjh[par][lane], Ah[j + lane * lda]);
                __stcg(&ws->rjl[par][lane], Al[j + lane * lda]);
            }
            __threadfence();
        }
        __syncthreads();
        if (tid == 0) s_stop = panel_grid_sync(ws, G, (unsigned int)(jj + 1)) ? 0 : 1;
        __syncthreads();
        if (s_stop) {
            if (c == 0 && tid == 0) *info = -1;
            return;
        }
        // 2. warp 0: the pivot, the best published key (the same in every
        //    CTA), and the pivot row into shared memory; warp 1: row j
        if (warp == 0) {
            PivotKey pk{0, 0.0, -1};
            int win = 0;
            for (int q = lane; q < G; q += 32) {
                const PanelCand &o = ws->cand[par][q];
                const PivotKey k{
                    (uint64_t)__ldcg(reinterpret_cast<const unsigned long long *>(&o.mag)),
                    __ldcg(&o.lo), (int64_t)__ldcg(reinterpret_cast<const long long *>(&o.row))};
                if (better(k, pk)) {
                    pk = k;
                    win = q;
                }
            }
            warp_best(pk, win);
            const PanelCand &wc = ws->cand[par][win];
            if (lane < w) {
                pvh[lane] = __ldcg(&wc.vh[lane]);
                pvl[lane] = __ldcg(&wc.vl[lane]);
            }
            if (lane == 0) {
                s_p = pk.row;
                s_rh = __ldcg(&wc.rh);
                s_rl = __ldcg(&wc.rl);
            }
        } else if (warp == 1 && lane < w) {
            jvh[lane] = __ldcg(&ws->rjh[par][lane]);
            jvl[lane] = __ldcg(&ws->rjl[par][lane]);
        }
        __syncthreads();
        const int64_t p = s_p;               // >= j: every column has rows j .. m-1
        const double ph = pvh[jj], pl = pvl[jj];
        if (c == 0 && tid == 0) {
            ipiv[j] = p + 1;
            if (ph == 0.0 && pl == 0.0)
                atomicCAS(reinterpret_cast<unsigned long long *>(info), 0ull,
                          (unsigned long long)(j + 1));
        }
        if (ph == 0.0 && pl == 0.0) continue;   // zero pivot: no interchange, no update
        const bool recip = fabs(ph) >= 0x1p-1021;
        const dd rcp{s_rh, s_rl};
        // 3a. the interchange within the panel and the multipliers of the rows
        // r > j this CTA owns; row p takes row j's entries
        const int64_t r0 = (j + 1 > rs ? j + 1 : rs);
        for (int64_t r = r0 + tid; r < re; r += kPanelThreads) {
            const bool isp = r == p && p != j;
            const dd a = isp ? dd{jvh[jj], jvl[jj]} : dd{Ah[r + jj * lda], Al[r + jj * lda]};
            const dd l = recip ? mul(a, rcp) : div(a, dd{ph, pl});
            lh[r - rs] = l.hi;
            ll[r - rs] = l.lo;
        }
        if (j >= rs && j < re && p != j && tid < w) {   // row j := the pivot row
            Ah[j + tid * lda] = pvh[tid];
            Al[j + tid * lda] = pvl[tid];
        }
        if (p != j && p >= rs && p < re && tid < jj) {  // row p's earlier columns := row j's
            Ah[p + tid * lda] = jvh[tid];
            Al[p + tid * lda] = jvl[tid];
        }
        __syncthreads();
        // 3b. A(r, j) = l_r; A(r, jj+1 ..) -= l_r * pivot row
        const int ncol = w - jj;                      // column jj and the ones after it
        const int64_t nr = re - r0;
        for (int64_t e = tid; e < nr * ncol; e += kPanelThreads) {
            const int64_t r = r0 + e / ncol;
            const int cc = jj + (int)(e % ncol);
            const dd l{lh[r - rs], ll[r - rs]};
            const int64_t o = r + cc * lda;
            if (cc == jj) {
                Ah[o] = l.hi;
                Al[o] = l.lo;
            } else {
                const bool isp = r == p && p != j;
                dd a = isp ? dd{jvh[cc], jvl[cc]} : dd{Ah[o], Al[o]};
                mac(a, dd{-l.hi, -l.lo}, dd{pvh[cc], pvl[cc]});
                Ah[o] = a.hi;
                Al[o] = a.lo;
            }
        }
        __syncthreads();
    }
    // columns past the last pivot (a panel wider than its rows): nothing left
}


struct LuPlan {
    double *ah, *al;
    int64_t lda, m, n;     // the whole matrix
    int64_t *ipiv, *info;
    cudaStream_t st;
    PanelWs *panel_ws = nullptr;   // the panel kernel's buffers (null: column leaves)
    int64_t panel_ctas = 0;        // co-resident CTAs of the panel kernel
};

int laswp(const LuPlan &P, double *bh, double *bl, int64_t ldb, int64_t c0, int64_t c1,
          int64_t k0, int64_t k1, int reverse) {
    if (c1 <= c0 || k1 <= k0) return 0;
    const int64_t cols = c1 - c0;
    laswp_kernel<<<(unsigned)ceil_div(cols, 128), 128, 0, P.st>>>(bh, bl, ldb, c0, c1, P.ipiv,
                                                                  k0, k1, reverse);
    return check_launch("laswp_kernel");
}

// Factor the block of rows [j0, m) and columns [j0, j0 + n) (the rows above
// j0 are already final).
int getrf_rec(const LuPlan &P, int64_t j0, int64_t n) {
    const int64_t rows = P.m - j0;
    if (n <= 0 || rows <= 0) return 0;
    int rc;
    // the panel kernel: rows spread over at most panel_ctas CTAs, at least 16
    // and at most 1024 rows each (its multipliers sit in shared memory)
    int64_t G = ceil_div(rows, (int64_t)16);
    if (G > P.panel_ctas) G = P.panel_ctas;
    if (G < 1) G = 1;
    int64_t R = ceil_div(rows, G);
    G = ceil_div(rows, R);
    if (P.panel_ws != nullptr && n <= kPanelW && R <= 1024) {
        const int w = (int)n;
        cudaError_t e = cudaMemsetAsync(P.panel_ws, 0, 2 * sizeof(unsigned int), P.st);
        if (e != cudaSuccess) return cuda_fail(e, "panel barrier reset");
        double *ah = P.ah, *al = P.al;
        int64_t lda = P.lda, m = P.m, jj0 = j0;
        int ww = w;
        int64_t *ipiv = P.ipiv, *info = P.info;
        PanelWs *ws = P.panel_ws;
        void *args[] = {&ah, &al, &lda, &m, &jj0, &ww, &R, &ipiv, &info, &ws};
        e = cudaLaunchCooperativeKernel((const void *)getrf_panel_kernel, dim3((unsigned)G),
                                        dim3(kPanelThreads), args, 0, P.st);
        if (e != cudaSuccess) return cuda_fail(e, "getrf_panel_kernel launch");
        if ((rc = check_launch("getrf_panel_kernel"))) return rc;
        // the panel's interchanges on the columns left and right of it
        const int64_t k1 = j0 + (rows < n ? rows : n);
        const int64_t other = P.n - n;
        if (other <= 0) return 0;
        laswp_perm_kernel<<<(unsigned)ceil_div(other, (int64_t)4), 256, 0, P.st>>>(
            P.ah, P.al, P.lda, j0, n, P.n, P.ipiv, j0, k1);
        return check_launch("laswp_perm_kernel");
    }
    if (n == 1) {
        getrf_pivot_kernel<<<1, LT, 0, P.st>>>(P.ah, P.al, P.lda, P.m, j0, P.ipiv, P.info);
        if ((rc = check_launch("getrf_pivot_kernel"))) return rc;
        const int col_ctas = (int)ceil_div(P.n, LT);
        const int row_ctas = (int)ceil_div(P.m - j0 - 1, LT);
        if (col_ctas + row_ctas == 0) return 0;
        getrf_apply_kernel<<<col_ctas + row_ctas, LT, 0, P.st>>>(P.ah, P.al, P.lda, P.m, P.n, j0,
                                                                 P.ipiv, col_ctas);
        return check_launch("getrf_apply_kernel");
    }
    const int64_t mn = rows < n ? rows : n;
    const int64_t n1 = mn / 2 > 0 ? mn / 2 : 1, n2 = n - n1;
    if ((rc = getrf_rec(P, j0, n1))) return rc;
    // A12 := L11^-1 A12 (n1 x n2), A22 -= A21 A12
    const int64_t o11 = j0 + j0 * P.lda, o12 = j0 + (j0 + n1) * P.lda;
    if (n1 > 1 &&   // a unit 1 x 1 L11 leaves A12 as it is
        (rc = run_trsm(0, 1, 0, 1, n1, n2, mp_dd{1.0, 0.0}, P.ah + o11, P.al + o11, P.lda,
                       P.ah + o12, P.al + o12, P.lda, P.st)))
        return rc;
    const int64_t m2 = rows - n1;
    if (m2 > 0 && (n1 <= kSmallUpdate || n2 <= kSmallUpdate)) {
        const int64_t o21 = (j0 + n1) + j0 * P.lda, o22 = (j0 + n1) + (j0 + n1) * P.lda;
        const int64_t count = m2 * n2;
        small_update_kernel<<<(unsigned)ceil_div(count, 256), 256, 0, P.st>>>(
            m2, n2, n1, P.ah + o21, P.al + o21, P.lda, P.ah + o12, P.al + o12, P.lda,
            P.ah + o22, P.al + o22, P.lda);
        if ((rc = check_launch("small_update_kernel"))) return rc;
        if ((rc = getrf_rec(P, j0 + n1, n2))) return rc;
    } else if (m2 > 0) {
        GemmArgs g{};
        g.m = m2; g.n = n2; g.k = n1;
        g.alpha = mp_dd{-1.0, 0.0}; g.beta = mp_dd{1.0, 0.0};
        const int64_t o21 = (j0 + n1) + j0 * P.lda, o22 = (j0 + n1) + (j0 + n1) * P.lda;
        g.ah = P.ah + o21; g.al = P.al + o21; g.lda = P.lda;
        g.bh = P.ah + o12; g.bl = P.al + o12; g.ldb = P.lda;
        g.ch = P.ah + o22; g.cl = P.al + o22; g.ldc = P.lda;
        g.ta = 0; g.tb = 0; g.tri = 0;
        g.alpha_zero = 0; g.alpha_one = 0; g.beta_zero = 0;
        if ((rc = launch_gemm_plain(g, P.st))) return rc;
        if ((rc = getrf_rec(P, j0 + n1, n2))) return rc;
    }
    return 0;
}

}  // namespace

int run_getrf(int64_t m, int64_t n, double *ah, double *al, int64_t lda, int64_t *ipiv,
              int64_t *info, cudaStream_t st) {
    int rc = set_attrs();
    if (rc) return rc;
    cudaError_t e = cudaMemsetAsync(info, 0, sizeof(int64_t), st);
    if (e != cudaSuccess) return cuda_fail(e, "info reset");
    LuPlan P{ah, al, lda, m, n, ipiv, info, st};
    // the panel kernel needs every CTA resident at once
    int dev = 0, coop = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, getrf_panel_kernel, kPanelThreads, 0);
    const int64_t ctas = (int64_t)per_sm * (sm_count() > 0 ? sm_count() : 0);
    if (coop && ctas > 0) {
        e = pool_alloc(reinterpret_cast<void **>(&P.panel_ws), sizeof(PanelWs), st);
        if (e != cudaSuccess) return cuda_fail(e, "panel workspace");
        P.panel_ctas = ctas < kPanelMaxG ? ctas : kPanelMaxG;
        if (P.panel_ctas > (sm_count() > 0 ? sm_count() : 1)) P.panel_ctas = sm_count();
    }
    rc = getrf_rec(P, 0, n);
    if (P.panel_ws != nullptr) {
        e = cudaFreeAsync(P.panel_ws, st);
        if (rc == 0 && e != cudaSuccess) return cuda_fail(e, "panel workspace");
    }
    return rc;
}

int run_getrs(int trans, int64_t n, int64_t nrhs, const double *ah, const double *al,
              int64_t lda, const int64_t *ipiv, double *bh, double *bl, int64_t ldb,
              cudaStream_t st) {
    LuPlan P{const_cast<double *>(ah), const_cast<double *>(al), lda, n, n,
             const_cast<int64_t *>(ipiv), nullptr, st};
    int rc;
    const mp_dd one{1.0, 0.0};
    if (!trans) {
        if ((rc = laswp(P, bh, bl, ldb, 0, nrhs, 0, n, 0))) return rc;
        if ((rc = run_trsm(0, 1, 0, 1, n, nrhs, one, ah, al, lda, bh, bl, ldb, st))) return rc;
        return run_trsm(0, 0, 0, 0, n, nrhs, one, ah, al, lda, bh, bl, ldb, st);
    }
    if ((rc = run_trsm(0, 0, 1, 0, n, nrhs, one, ah, al, lda, bh, bl, ldb, st))) return rc;
    if ((rc = run_trsm(0, 1, 1, 1, n, nrhs, one, ah, al, lda, bh, bl, ldb, st))) return rc;
    return laswp(P, bh, bl, ldb, 0, nrhs, 0, n, 1);
}

}  // namespace mpdd
