// FP64 products emulated on the bf16 tensor cores (Ozaki-style splitting).
//
// The paper computes its high-precision products with the Ozaki scheme
// (Sec. 3: the `acc` toolbox, Ozaki, Ogita, Oishi and Rump 2012). On GB300 the
// FP64 pipe delivers ~1.2 TFLOP/s and tcgen05 has no integer MMA for sm_103a,
// so the split here targets bf16 operands with FP32 accumulation:
//
//  * every row i of op(A) and column j of B gets a power-of-two scale 2^e with
//    |entries| < 2^e; the scaled entries x in (-1, 1) are written in fixed
//    point with F = 7 + 8(s-1) fraction bits and cut into s signed digits
//    sigma_p in [-128, 128], x ~ sum_p sigma_p 2^(-7-8p) (p = 0..s-1). The
//    digits are exact in bf16. The cut is integer arithmetic only.
//  * digit matrices are multiplied pairwise on tcgen05 (kind::f16, FP32
//    accumulation in TMEM) in K-chunks of 256: every partial sum is an
//    integer below 2^22 in magnitude, hence exact. Chunk results are drained
//    from TMEM and summed exactly in 32-bit integers per level l = p + q.
//    Levels l = 0..s-1 are kept (the pairs with p + q <= s - 1).
//  * a combine kernel rebuilds C(i,j) = 2^(e_i + f_j) sum_l I_l 2^(-14-8l) in
//    FP64 and hands it to the same fused epilogues as the native FP64 path.
#pragma once
#include <climits>

#include "common.cuh"

namespace sr {

constexpr int kOzakiMaxSlices = 7;   // 7 + 8*6 = 55 fraction bits fit a 64-bit integer
constexpr int kOzakiDefaultSlices = 7;
constexpr bool kOzakiBuilt = true;
constexpr int kOzakiTile = 128;
constexpr int kOzakiKChunk = 256;
constexpr int kOzakiMaxK = 16384;     // keeps every level sum below 2^31
constexpr int kOzakiExpNonfinite = INT_MIN;

struct OzakiWork {
    int nmax = 0, smax = 0, Pmax = 0, Kmax = 0;
    void *Asl = nullptr, *Bsl = nullptr;   // bf16 digits: [s][Pmax][Kmax]
    int32_t *planes = nullptr;             // [s][Pmax cols][Pmax rows], column-major per level
    int *ea = nullptr, *fb = nullptr;      // scale exponents of op(A) rows and B columns
    alignas(64) unsigned char tmA[128];    // CUtensorMap of the op(A) digits
    alignas(64) unsigned char tmB[128];    // CUtensorMap of the B digits
};

cudaError_t ozaki_alloc(OzakiWork &w, int nmax, int slices);
void ozaki_free(OzakiWork &w);

// Splits op(A) and B and runs the slice products into w.planes. Returns
// SR_ERR_UNSUPPORTED for k > kOzakiMaxK.
sr_status ozaki_products(schur_refine_ctx *h, cudaStream_t st, OzakiWork &w, bool transA, int m, int n, int k,
                         const double *A, int lda, const double *B, int ldb, int s, int *flags);

// 2^e as a product of two normal doubles (e within +-2044)
__device__ inline double oz_pow2_scale(double v, int e)
{
    const int e1 = e / 2, e2 = e - e / 2;
    const double p1 = __longlong_as_double((long long)(1023 + e1) << 52);
    const double p2 = __longlong_as_double((long long)(1023 + e2) << 52);
    return (v * p1) * p2;
}

// C(i,j) from the level planes; ep as in gemm_simt.cuh.
template <class EP>
__global__ void __launch_bounds__(256)
ozaki_combine_kernel(int m, int n, int s, const int32_t *__restrict__ planes, int ldp, size_t pstride,
                     const int *__restrict__ ea, const int *__restrict__ fb, EP ep, double *partial)
{
    const int i = blockIdx.x * 32 + (threadIdx.x & 31);
    const int jb = blockIdx.y * 32 + (threadIdx.x >> 5);
    const int nh = s < 4 ? s : 4;
    const double sh = __longlong_as_double((long long)(1023 - 14 - 8 * (nh - 1)) << 52);
    const double sl = __longlong_as_double((long long)(1023 - 14 - 8 * (s - 1)) << 52);
    double part = 0.0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const int j = jb + 8 * w;
        if (i < m && j < n) {
            const size_t off = (size_t)i + (size_t)j * (size_t)ldp;
            long long H = 0, Lo = 0;
            for (int l = 0; l < nh; ++l) H = H * 256 + (long long)planes[off + (size_t)l * pstride];
            for (int l = nh; l < s; ++l) Lo = Lo * 256 + (long long)planes[off + (size_t)l * pstride];
            double v = fma((double)Lo, sl, (double)H * sh);
            const int e1 = ea[i], e2 = fb[j];
            if (e1 == kOzakiExpNonfinite || e2 == kOzakiExpNonfinite)
                v = __longlong_as_double(0x7ff8000000000000LL);
            else
                v = oz_pow2_scale(v, e1 + e2);
            part += ep(i, j, v);
        }
    }
    if (partial) {
        part = sr_block_sum<256>(part);
        if (threadIdx.x == 0) partial[blockIdx.x + (size_t)gridDim.x * blockIdx.y] = part;
    }
}

inline int ozaki_blocks(int m, int n) { return ((m + 31) / 32) * ((n + 31) / 32); }

template <class EP>
sr_status ozaki_gemm(schur_refine_ctx *h, cudaStream_t st, OzakiWork &w, bool transA, int m, int n, int k,
                     const double *A, int lda, const double *B, int ldb, EP ep, double *partial, int *blocks,
                     int slices, int *flags)
{
    const int s = slices > 0 ? slices : kOzakiDefaultSlices;
    if (s > w.smax || m > w.nmax || n > w.nmax || k > w.nmax) return SR_ERR_INVALID_ARG;
    SR_TRY(ozaki_products(h, st, w, transA, m, n, k, A, lda, B, ldb, s, flags));
    {
        SrPhase ph(h, SR_PROF_OZ_COMBINE, 8LL * s * m * n, (long long)m * n * (4LL * s + 16), 1);
        dim3 grid((m + 31) / 32, (n + 31) / 32);
        ozaki_combine_kernel<EP><<<grid, 256, 0, st>>>(m, n, s, w.planes, w.Pmax, (size_t)w.Pmax * w.Pmax,
                                                        w.ea, w.fb, ep, partial);
        SR_CUDA_TRY(cudaGetLastError());
    }
    *blocks = ozaki_blocks(m, n);
    return SR_OK;
}

}  // namespace sr
