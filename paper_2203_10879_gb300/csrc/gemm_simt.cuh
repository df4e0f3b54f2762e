// Register-tiled SIMT GEMM with operand loaders and fused epilogues.
//
// C(i, j) = sum_k opA(i, k) * opB(k, j), accumulated in the type T of the
// operands (double for the native FP64 high-precision products of Alg. 4,
// float for the FP32 low-precision products YW, W^2, W^3). Operands are read
// through loader functors, so the skew matrix W = L - L^H is formed on the fly
// from L, and high-precision Y is rounded to the low precision as it is read.
// The epilogue functor receives every finished entry and returns a value whose
// block sum is written to partial[block] (used for Frobenius norms).
#pragma once
#include "common.cuh"

namespace sr {

// ---- loaders: value of op(M)(r, c) ----------------------------------------
template <typename Tout, typename Tin>
struct LoadN {                       // M itself, column-major
    const Tin *p; int ld;
    static constexpr bool kRowFast = true;   // consecutive r are contiguous
    __device__ Tout operator()(int r, int c) const { return (Tout)p[sr_idx(r, c, ld)]; }
};
template <typename Tout, typename Tin>
struct LoadT {                       // M^T, column-major M
    const Tin *p; int ld;
    static constexpr bool kRowFast = false;
    __device__ Tout operator()(int r, int c) const { return (Tout)p[sr_idx(c, r, ld)]; }
};
// W = L - L^T from the strictly lower triangle of a column-major L.
template <typename Tout, typename Tin>
struct LoadSkew {
    const Tin *p; int ld;
    static constexpr bool kRowFast = true;
    __device__ Tout operator()(int r, int c) const
    {
        if (r > c) return (Tout)p[sr_idx(r, c, ld)];
        if (r < c) return -(Tout)p[sr_idx(c, r, ld)];
        return (Tout)0;
    }
};

// ---- the kernel --------------------------------------------------------------
template <typename T, int BM, int BN, int BK, int TM, int TN>
struct SimtTile {
    static constexpr int NTX = BM / TM, NTY = BN / TN, NT = NTX * NTY;
    static constexpr int LA = BM * BK / NT, LB = BK * BN / NT;   // elements loaded per thread
    static_assert(BM * BK % NT == 0 && BK * BN % NT == 0, "tile/thread mismatch");
};

template <typename T, int BM, int BN, int BK, int TM, int TN, class LA, class LB, class EP>
__global__ void __launch_bounds__(SimtTile<T, BM, BN, BK, TM, TN>::NT)
gemm_simt_kernel(int m, int n, int k, LA la, LB lb, EP ep, double *partial)
{
    using Tl = SimtTile<T, BM, BN, BK, TM, TN>;
    constexpr int NT = Tl::NT, NTX = Tl::NTX, NTY = Tl::NTY;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid % NTX, ty = tid / NTX;
    const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;

    T acc[TM][TN];
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c] = (T)0;

    T ra[Tl::LA], rb[Tl::LB];
    auto load = [&](int k0) {
#pragma unroll
        for (int q = 0; q < Tl::LA; ++q) {
            const int e = tid + q * NT;
            int r, c;
            if (LA::kRowFast) { r = e % BM; c = e / BM; } else { c = e % BK; r = e / BK; }
            const int gi = i0 + r, gk = k0 + c;
            ra[q] = (gi < m && gk < k) ? la(gi, gk) : (T)0;
        }
#pragma unroll
        for (int q = 0; q < Tl::LB; ++q) {
            const int e = tid + q * NT;
            int r, c;   // r along k, c along n
            if (LB::kRowFast) { r = e % BK; c = e / BK; } else { c = e % BN; r = e / BN; }
            const int gk = k0 + r, gj = j0 + c;
            rb[q] = (gk < k && gj < n) ? lb(gk, gj) : (T)0;
        }
    };
    auto store = [&]() {
#pragma unroll
        for (int q = 0; q < Tl::LA; ++q) {
            const int e = tid + q * NT;
            int r, c;
            if (LA::kRowFast) { r = e % BM; c = e / BM; } else { c = e % BK; r = e / BK; }
            As[c][r] = ra[q];
        }
#pragma unroll
        for (int q = 0; q < Tl::LB; ++q) {
            const int e = tid + q * NT;
            int r, c;
            if (LB::kRowFast) { r = e % BK; c = e / BK; } else { c = e % BN; r = e / BN; }
            Bs[r][c] = rb[q];
        }
    };

    load(0);
    for (int k0 = 0; k0 < k; k0 += BK) {
        store();
        __syncthreads();
        if (k0 + BK < k) load(k0 + BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TN];
#pragma unroll
            for (int r = 0; r < TM; ++r) a[r] = As[kk][tx + r * NTX];
#pragma unroll
            for (int c = 0; c < TN; ++c) b[c] = Bs[kk][ty + c * NTY];
#pragma unroll
            for (int r = 0; r < TM; ++r)
#pragma unroll
                for (int c = 0; c < TN; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }

    double part = 0.0;
#pragma unroll
    for (int c = 0; c < TN; ++c)
#pragma unroll
        for (int r = 0; r < TM; ++r) {
            const int gi = i0 + tx + r * NTX, gj = j0 + ty + c * NTY;
            if (gi < m && gj < n) part += ep(gi, gj, acc[r][c]);
        }
    if (partial) {
        part = sr_block_sum<NT>(part);
        if (tid == 0) partial[blockIdx.x + (size_t)gridDim.x * blockIdx.y] = part;
    }
}

// tile shapes
struct TileF64 { static constexpr int BM = 64, BN = 64, BK = 8, TM = 4, TN = 4; };
struct TileF64Small { static constexpr int BM = 32, BN = 32, BK = 8, TM = 2, TN = 2; };
struct TileF32 { static constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8; };

template <typename T> struct TileFor;
template <> struct TileFor<double> { using type = TileF64; };
template <> struct TileFor<float> { using type = TileF32; };

// FP64 products whose 64 x 64 grid would fill less than half of the GPU's 152
// SMs (small orders: latency-bound) use 32 x 32 tiles, 4x the blocks.
template <typename T>
inline bool simt_small(int m, int n)
{
    return sr_is_double<T>::value && ((m + 63) / 64) * ((n + 63) / 64) < 76;
}

// Number of blocks (= partial sums) a launch of an m x n product writes.
template <typename T>
inline int simt_blocks(int m, int n)
{
    if (simt_small<T>(m, n)) return ((m + 31) / 32) * ((n + 31) / 32);
    using Tl = typename TileFor<T>::type;
    return ((m + Tl::BM - 1) / Tl::BM) * ((n + Tl::BN - 1) / Tl::BN);
}

template <typename T, class Tl, class LA, class LB, class EP>
inline cudaError_t gemm_simt_tile(cudaStream_t st, int m, int n, int k, LA la, LB lb, EP ep, double *partial)
{
    dim3 grid((m + Tl::BM - 1) / Tl::BM, (n + Tl::BN - 1) / Tl::BN);
    constexpr int NT = (Tl::BM / Tl::TM) * (Tl::BN / Tl::TN);
    gemm_simt_kernel<T, Tl::BM, Tl::BN, Tl::BK, Tl::TM, Tl::TN><<<grid, NT, 0, st>>>(m, n, k, la, lb, ep,
                                                                                     partial);
    return cudaGetLastError();
}

template <typename T, class LA, class LB, class EP>
inline cudaError_t gemm_simt(cudaStream_t st, int m, int n, int k, LA la, LB lb, EP ep, double *partial)
{
    if constexpr (sr_is_double<T>::value) {
        if (simt_small<T>(m, n)) return gemm_simt_tile<T, TileF64Small>(st, m, n, k, la, lb, ep, partial);
    }
    return gemm_simt_tile<T, typename TileFor<T>::type>(st, m, n, k, la, lb, ep, partial);
}

}  // namespace sr
