// Double-double working precision (the FP64 -> double-double form of Alg. 4).
//
// A double-double matrix is two column-major planes, hi and lo, that stand
// for the unevaluated sum hi + lo. The high-precision steps of Alg. 4 (the
// products forming T^, Y and the update, the sum Sigma) run in this
// arithmetic; the low precision is FP64 (the solve and the products YW, W^2,
// W^3).
//
// This header holds the epilogues that receive a finished double-double entry
// (shared by both engines: the emulated products of ozaki.cu and the SIMT
// kernel below), the SIMT double-double product built from FP64 error-free
// transformations (TwoProd by fused multiply-add, TwoSum), and the residual
// kernel of the double-double target.
#pragma once
#include "common.cuh"

namespace sr {

// ---- epilogues (v = double-double value of entry (i, j)); kDD marks them ----------

struct EpStoreDD {
    static constexpr bool kDD = true;
    double *hi, *lo; int ld;
    __device__ double operator()(int i, int j, ddv v) const
    {
        const size_t p = sr_idx(i, j, ld);
        hi[p] = v.hi;
        lo[p] = v.lo;
        return 0.0;
    }
};

// T^ = Q^T (A Q): T^ rounded to FP64 into TE (upper = T, strictly lower = E),
// the diagonal kept in double-double (divisors of the solve), T^ itself when
// requested; returns e_ij^2 for ||E||_F.
struct EpSplitDD {
    static constexpr bool kDD = true;
    double *TE; int ldte; double *dhi, *dlo; double *thi, *tlo; int ldt;
    __device__ double operator()(int i, int j, ddv v) const
    {
        const double x = v.hi + v.lo;
        TE[sr_idx(i, j, ldte)] = x;
        if (thi) {
            thi[sr_idx(i, j, ldt)] = v.hi;
            tlo[sr_idx(i, j, ldt)] = v.lo;
        }
        if (i == j) {
            dhi[i] = v.hi;
            dlo[i] = v.lo;
        }
        return i > j ? x * x : 0.0;
    }
};

// Y = Q^T Q - I in double-double; returns y_ij^2 for ||Y||_F.
struct EpMinusIDD {
    static constexpr bool kDD = true;
    double *hi, *lo; int ld;
    __device__ double operator()(int i, int j, ddv v) const
    {
        if (i == j) v = dd_plus_d(v, -1.0);
        const size_t p = sr_idx(i, j, ld);
        hi[p] = v.hi;
        lo[p] = v.lo;
        const double y = v.hi + v.lo;
        return y * y;
    }
};

// Q_new = Q + alpha * (product) in double-double; alpha = 1/2 (update with
// Q Delta) or -1/2 (Newton-Schulz step with Q Y0), a power of two. The
// correction is small against Q, so the low parts are added in FP64 (dd_acc).
struct EpUpdateDD {
    static constexpr bool kDD = true;
    const double *qhi, *qlo; int ldq; double *nhi, *nlo; int ldn; double alpha;
    __device__ double operator()(int i, int j, ddv v) const
    {
        const size_t p = sr_idx(i, j, ldq);
        const ddv r = dd_acc(ddv{qhi[p], qlo[p]}, ddv{alpha * v.hi, alpha * v.lo});
        const size_t q = sr_idx(i, j, ldn);
        nhi[q] = r.hi;
        nlo[q] = r.lo;
        return 0.0;
    }
};

// Delta = Sigma - 2I = 2W - Y - YW + W^2 + W^3 (+ W^2 Y + W^2 Y W) summed in
// double-double (Alg. 4: Sigma in hp): Y is double-double, the other terms are
// FP64; v is the FP64 entry of W^3. W2Y, W2YW may be null.
struct EpDeltaDD {
    const double *W, *YW, *W2, *W2Y, *W2YW; int ld;
    const double *yhi, *ylo; int ldy;
    double *dhi, *dlo; int ldd;
    template <typename V>
    __device__ double operator()(int i, int j, V v) const
    {
        const size_t p = sr_idx(i, j, ld), py = sr_idx(i, j, ldy);
        ddv d = {-yhi[py], -ylo[py]};
        d = dd_plus_d(d, 2.0 * W[p]);
        d = dd_plus_d(d, -YW[p]);
        d = dd_plus_d(d, W2[p]);
        d = dd_plus_d(d, (double)v);
        if (W2Y) {
            d = dd_plus_d(d, W2Y[p]);
            d = dd_plus_d(d, W2YW[p]);
        }
        const size_t q = sr_idx(i, j, ldd);
        dhi[q] = d.hi;
        dlo[q] = d.lo;
        return 0.0;
    }
};

// ---- loaders of double-double operands ----------------------------------------------
struct LoadNDD {                  // M itself
    const double *hi, *lo; int ld;
    static constexpr bool kRowFast = true;
    __device__ ddv operator()(int r, int c) const { const size_t p = sr_idx(r, c, ld); return {hi[p], lo[p]}; }
};
struct LoadTDD {                  // M^T
    const double *hi, *lo; int ld;
    static constexpr bool kRowFast = false;
    __device__ ddv operator()(int r, int c) const { const size_t p = sr_idx(c, r, ld); return {hi[p], lo[p]}; }
};

// ---- SIMT double-double product ----------------------------------------------------
// C(i, j) = sum_k op(A)(i, k) op(B)(k, j) with double-double operands: every
// term is the exact product of the high parts (TwoProd through a fused
// multiply-add) plus the cross terms, accumulated by TwoSum with the low
// parts added in FP64 (dd_acc). 64 x 64 tiles, 256 threads with 4 x 4 entries
// each, K-blocks of 8 staged in shared memory as hi and lo planes.
constexpr int kDdBM = 64, kDdBN = 64, kDdBK = 8, kDdTM = 4, kDdTN = 4, kDdNT = 256;

template <class LA, class LB, class EP>
__global__ void __launch_bounds__(kDdNT)
gemm_ddk_kernel(int m, int n, int k, LA la, LB lb, EP ep, double *partial)
{
    constexpr int BM = kDdBM, BN = kDdBN, BK = kDdBK, TM = kDdTM, TN = kDdTN, NT = kDdNT;
    constexpr int NTX = BM / TM, NTY = BN / TN;
    constexpr int LA_N = BM * BK / NT, LB_N = BK * BN / NT;
    __shared__ double Ah[BK][BM + 1], Al[BK][BM + 1], Bh[BK][BN + 1], Bl[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid % NTX, ty = tid / NTX;
    const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
    ddv acc[TM][TN];
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c] = {0.0, 0.0};

    for (int k0 = 0; k0 < k; k0 += BK) {
#pragma unroll
        for (int q = 0; q < LA_N; ++q) {
            const int e = tid + q * NT;
            int r, c;
            if (LA::kRowFast) { r = e % BM; c = e / BM; } else { c = e % BK; r = e / BK; }
            const int gi = i0 + r, gk = k0 + c;
            const ddv v = (gi < m && gk < k) ? la(gi, gk) : ddv{0.0, 0.0};
            Ah[c][r] = v.hi;
            Al[c][r] = v.lo;
        }
#pragma unroll
        for (int q = 0; q < LB_N; ++q) {
            const int e = tid + q * NT;
            int r, c;
            if (LB::kRowFast) { r = e % BK; c = e / BK; } else { c = e % BN; r = e / BN; }
            const int gk = k0 + r, gj = j0 + c;
            const ddv v = (gk < k && gj < n) ? lb(gk, gj) : ddv{0.0, 0.0};
            Bh[r][c] = v.hi;
            Bl[r][c] = v.lo;
        }
        __syncthreads();
#pragma unroll 2
        for (int kk = 0; kk < BK; ++kk) {
            ddv a[TM], b[TN];
#pragma unroll
            for (int r = 0; r < TM; ++r) a[r] = {Ah[kk][tx + r * NTX], Al[kk][tx + r * NTX]};
#pragma unroll
            for (int c = 0; c < TN; ++c) b[c] = {Bh[kk][ty + c * NTY], Bl[kk][ty + c * NTY]};
#pragma unroll
            for (int r = 0; r < TM; ++r)
#pragma unroll
                for (int c = 0; c < TN; ++c) {
                    const double p = a[r].hi * b[c].hi;
                    double e = fma(a[r].hi, b[c].hi, -p);
                    e = fma(a[r].hi, b[c].lo, e);
                    e = fma(a[r].lo, b[c].hi, e);
                    acc[r][c] = dd_acc(acc[r][c], ddv{p, e});
                }
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

inline int ddk_blocks(int m, int n) { return ((m + kDdBM - 1) / kDdBM) * ((n + kDdBN - 1) / kDdBN); }

template <class LA, class LB, class EP>
inline cudaError_t gemm_ddk(cudaStream_t st, int m, int n, int k, LA la, LB lb, EP ep, double *partial)
{
    dim3 grid((m + kDdBM - 1) / kDdBM, (n + kDdBN - 1) / kDdBN);
    gemm_ddk_kernel<LA, LB, EP><<<grid, kDdNT, 0, st>>>(m, n, k, la, lb, ep, partial);
    return cudaGetLastError();
}

// ---- residuals of a double-double decomposition ------------------------------------
// C = op(A) B with double-double A and B, each entry accumulated in
// double-double (dd_plus), 16 x 16 tiles, one entry per thread.
// mode 0: store C (hi, lo). mode 1: partial += sum over i > j of (hi + lo)^2.
// mode 2: partial += sum over all (i, j) of (C - I)^2 (upper tiles only,
// off-diagonal entries counted twice; C symmetric).
template <int MODE>
__global__ void __launch_bounds__(256)
gemm_ddq_kernel(int n, int transA, const double *__restrict__ Ahi, const double *__restrict__ Alo, int lda,
                const double *__restrict__ Bhi, const double *__restrict__ Blo, int ldb, double *__restrict__ Chi,
                double *__restrict__ Clo, int ldc, double *__restrict__ partial)
{
    constexpr int T = 16;
    __shared__ double Ash[T][T + 1], Asl[T][T + 1], Bsh[T][T + 1], Bsl[T][T + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.x * T, j0 = blockIdx.y * T;
    const size_t bid = blockIdx.x + (size_t)gridDim.x * blockIdx.y;
    if ((MODE == 1 && i0 + T - 1 <= j0) || (MODE == 2 && i0 > j0 + T - 1)) {
        if (threadIdx.x == 0) partial[bid] = 0.0;
        return;
    }
    const int i = i0 + tx, j = j0 + ty;
    ddv acc = {0.0, 0.0};
    for (int k0 = 0; k0 < n; k0 += T) {
        {
            const int ii = transA ? ty : tx, kk = transA ? tx : ty;
            const int gi = i0 + ii, gk = k0 + kk;
            double vh = 0.0, vl = 0.0;
            if (gi < n && gk < n) {
                const size_t p = transA ? sr_idx(gk, gi, lda) : sr_idx(gi, gk, lda);
                vh = Ahi[p];
                vl = Alo[p];
            }
            Ash[kk][ii] = vh;
            Asl[kk][ii] = vl;
        }
        {
            const int gk = k0 + tx, gj = j0 + ty;
            const bool in = gk < n && gj < n;
            Bsh[tx][ty] = in ? Bhi[sr_idx(gk, gj, ldb)] : 0.0;
            Bsl[tx][ty] = in ? Blo[sr_idx(gk, gj, ldb)] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < T; ++kk)
            acc = dd_plus(acc, dd_mul(ddv{Ash[kk][tx], Asl[kk][tx]}, ddv{Bsh[kk][ty], Bsl[kk][ty]}));
        __syncthreads();
    }
    double part = 0.0;
    if (i < n && j < n) {
        if (MODE == 0) {
            Chi[sr_idx(i, j, ldc)] = acc.hi;
            Clo[sr_idx(i, j, ldc)] = acc.lo;
        } else if (MODE == 1) {
            if (i > j) {
                const double v = acc.hi + acc.lo;
                part = v * v;
            }
        } else {
            if (i <= j) {
                if (i == j) acc = dd_plus_d(acc, -1.0);
                const double v = acc.hi + acc.lo;
                part = (i == j ? 1.0 : 2.0) * v * v;
            }
        }
    }
    if (MODE != 0) {
        part = sr_block_sum<256>(part);
        if (threadIdx.x == 0) partial[bid] = part;
    }
}

// (hi, lo) <- (src, 0): a double-precision start in double-double form
__global__ void to_dd_kernel(int n, const double *__restrict__ src, int lds, double *__restrict__ hi,
                             double *__restrict__ lo, int ld)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i < n) {
        hi[sr_idx(i, j, ld)] = src[sr_idx(i, j, lds)];
        lo[sr_idx(i, j, ld)] = 0.0;
    }
}

}  // namespace sr
