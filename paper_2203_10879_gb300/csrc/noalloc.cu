// Residual certification without any device allocation.
//
// schur_refine_residuals needs a handle, and creating a handle allocates its
// workspace with cudaMalloc. Some callers cannot do that: applications whose
// GPU memory is owned by their own pool allocator (a framework's caching
// allocator that has reserved the device), services that forbid device
// allocation after start-up so that their footprint stays fixed, and code
// paths that must not trigger the implicit device synchronization a
// cudaMalloc/cudaFree can cause. For them, schur_refine_residuals_noalloc
// computes the same two measures with its scratch in a fixed array that is
// part of this library's device image.
//
// The scratch is g_residual_scratch below: 2 * 512 * 512 doubles for A Q in
// double-double (hi and lo planes), 1024 partial sums (one per 16 x 16 tile at
// n = 512) and 8 result slots -- about 4 MiB, held on every GPU that loads the
// library until the process exits. Orders above 512 are rejected.
//
// Every call on a device shares that one array and leaves its contents behind
// for the next call; the result slots are cleared at the start of each call,
// everything else is overwritten before it is read. Calls whose work overlaps
// on the GPU (other streams, other host threads) race on the array, so callers
// must order them.
//
// Host code must not pass the array's name to a kernel: on the host it is
// only a stand-in symbol, not a device address. Every call looks up the
// array's device address on the current device with cudaGetSymbolAddress
// before it launches anything: the lookup is cheap, and an address cached
// across calls would go stale when the context is torn down and created again
// (cudaDeviceReset, or a released primary context), after which the module is
// loaded again, possibly at another address.
//
// Under CUDA's default lazy module loading, the array's device memory is
// committed when the first call on a device loads this file's module. A
// caller whose pool allocator reserves the whole device should therefore make
// one call on each device before the pool takes its memory (or run with
// CUDA_MODULE_LOADING=EAGER), or that first call can fail for lack of memory.
#include <math.h>

#include "common.cuh"
#include "kernels_misc.cuh"

namespace {

constexpr int kMaxN = 512;
constexpr size_t kNN = (size_t)kMaxN * (size_t)kMaxN;
constexpr int kTiles = ((kMaxN + 15) / 16) * ((kMaxN + 15) / 16);
constexpr size_t kScratchDoubles = 2 * kNN + kTiles + 8;

}  // namespace

static __device__ __align__(256) double g_residual_scratch[kScratchDoubles];

// out[0] = sum of partial[0..count), fixed order
static __global__ void __launch_bounds__(256) noalloc_sum_kernel(const double *__restrict__ partial, int count,
                                                                double *__restrict__ out)
{
    double s = 0.0;
    for (int e = threadIdx.x; e < count; e += 256) s += partial[e];
    s = sr_block_sum<256>(s);
    if (threadIdx.x == 0) *out = s;
}

// Device address of the scratch array on the current device, looked up anew
// on every call (see the header comment for why it is not cached).
static cudaError_t scratch_address(double **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_residual_scratch);
    if (e != cudaSuccess) return e;
    *out = (double *)p;
    return cudaSuccess;
}

extern "C" sr_status schur_refine_residuals_noalloc(int n, const void *dA, int lda, const void *dQ, int ldq,
                                                    double *stril_rel, double *orth, void *cuda_stream)
{
    if (!dA || !dQ || !stril_rel || !orth || n < 1 || lda < n || ldq < n) return SR_ERR_INVALID_ARG;
    if (n > kMaxN) return SR_ERR_INVALID_ARG;   // larger than the fixed scratch array
    cudaStream_t st = (cudaStream_t)cuda_stream;
    double *s = nullptr;
    SR_CUDA_TRY(scratch_address(&s));
    double *hi = s, *lo = s + kNN, *part = s + 2 * kNN, *res = part + kTiles;
    const double *A = (const double *)dA, *Q = (const double *)dQ;
    const int tiles = ((n + 15) / 16) * ((n + 15) / 16);
    dim3 grid((n + 15) / 16, (n + 15) / 16);

    SR_CUDA_TRY(cudaMemsetAsync(res, 0, 8 * sizeof(double), st));
    // A Q in double-double, packed with leading dimension n
    sr::gemm_dd_kernel<0><<<grid, 256, 0, st>>>(n, 0, A, lda, Q, nullptr, ldq, hi, lo, n, nullptr);
    SR_CUDA_TRY(cudaGetLastError());
    // ||stril(Q^T (A Q))||^2
    sr::gemm_dd_kernel<1><<<grid, 256, 0, st>>>(n, 1, Q, ldq, hi, lo, n, nullptr, nullptr, 0, part);
    SR_CUDA_TRY(cudaGetLastError());
    noalloc_sum_kernel<<<1, 256, 0, st>>>(part, tiles, res + 0);
    SR_CUDA_TRY(cudaGetLastError());
    // ||Q^T Q - I||^2
    sr::gemm_dd_kernel<2><<<grid, 256, 0, st>>>(n, 1, Q, ldq, Q, nullptr, ldq, nullptr, nullptr, 0, part);
    SR_CUDA_TRY(cudaGetLastError());
    noalloc_sum_kernel<<<1, 256, 0, st>>>(part, tiles, res + 1);
    SR_CUDA_TRY(cudaGetLastError());
    // ||A||^2
    sr::sumsq_kernel<double><<<kTiles, 256, 0, st>>>(n, A, lda, 0, part);
    SR_CUDA_TRY(cudaGetLastError());
    noalloc_sum_kernel<<<1, 256, 0, st>>>(part, kTiles, res + 2);
    SR_CUDA_TRY(cudaGetLastError());

    double h[3] = {0.0, 0.0, 0.0};
    SR_CUDA_TRY(cudaMemcpyAsync(h, res, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    SR_CUDA_TRY(cudaStreamSynchronize(st));
    // A = 0 has Q^T A Q = 0: its relative residual is 0, not 0/0
    *stril_rel = h[2] > 0.0 ? sqrt(h[0]) / sqrt(h[2]) : 0.0;
    *orth = sqrt(h[1]);
    return SR_OK;
}
