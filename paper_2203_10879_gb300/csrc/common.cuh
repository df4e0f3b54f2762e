// Shared device helpers of the Schur-refinement library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "schur_refine.h"

#define SR_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t err__ = (expr);                         \
        if (err__ != cudaSuccess) {                         \
            sr_set_last_cuda_error(err__);                  \
            return SR_ERR_CUDA;                             \
        }                                                   \
    } while (0)

#define SR_TRY(expr)                                        \
    do {                                                    \
        sr_status st__ = (expr);                            \
        if (st__ != SR_OK) return st__;                     \
    } while (0)

void sr_set_last_cuda_error(cudaError_t e);

// Phase timing (defined by the engine): every kernel launch of the library is
// wrapped in sr_prof_begin/sr_prof_end with its phase kind (SR_PROF_*), its
// algorithmic flops and bytes and its number of launches. CUDA events are
// recorded only when the handle was created with profile = 1.
struct schur_refine_ctx;
void sr_prof_begin(schur_refine_ctx *h, int kind, long long flops, long long bytes, long long launches);
void sr_prof_end(schur_refine_ctx *h, int kind);

struct SrPhase {
    schur_refine_ctx *h;
    int kind;
    SrPhase(schur_refine_ctx *h_, int kind_, long long flops, long long bytes, long long launches)
        : h(h_), kind(kind_)
    {
        sr_prof_begin(h, kind, flops, bytes, launches);
    }
    ~SrPhase() { sr_prof_end(h, kind); }
};

// device-side error bits (read back by the host after a solve)
enum : int { SR_FLAG_NONDISTINCT = 1, SR_FLAG_NONFINITE = 2, SR_FLAG_TIMEOUT = 4 };

__host__ __device__ inline size_t sr_idx(int i, int j, int ld) { return (size_t)i + (size_t)j * (size_t)ld; }

template <typename T> struct sr_is_double { static constexpr bool value = false; };
template <> struct sr_is_double<double> { static constexpr bool value = true; };

__device__ inline bool sr_finite(float x) { return isfinite(x); }
__device__ inline bool sr_finite(double x) { return isfinite(x); }

// Block-wide sum of one double per thread; result valid in thread 0.
template <int NT>
__device__ inline double sr_block_sum(double v)
{
    __shared__ double red[NT / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (l < NT / 32) ? red[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    return v;
}
