// Epilogues of the products of Alg. 4, small elementwise kernels and the
// double-double residual kernel.
#pragma once
#include "common.cuh"

namespace sr {

// ---- epilogues (value v of the finished product entry (i, j)) ---------------

// plain store of a high-precision product (A Q)
struct EpStore {
    double *C; int ld;
    template <typename V>
    __device__ double operator()(int i, int j, V v) const { C[sr_idx(i, j, ld)] = (double)v; return 0.0; }
};

// plain store in low precision (W^2, YW, ...)
template <typename Tl>
struct EpStoreLp {
    Tl *C; int ld;
    template <typename V>
    __device__ double operator()(int i, int j, V v) const { C[sr_idx(i, j, ld)] = (Tl)v; return 0.0; }
};

// T^ = Q^H (A Q): the whole T^ goes to the low-precision buffer TE (upper
// triangle = T, strictly lower = E, Alg. 4 "set E, T and convert to lp"),
// its diagonal to `diag` in high precision (divisors of the solve), T^ to
// `That` in high precision when requested; returns e_ij^2 for ||E||_F.
template <typename Tl>
struct EpSplit {
    Tl *TE; int ldte; double *diag; double *That; int ldt;
    // real quasi-triangular form: T^(k+1, k) to sub[k], T^(k, k+1) to sup[k], and
    // the subdiagonal left out of ||E||^2 (the entries that are not couplings of
    // 2 x 2 blocks are added back once the blocks are known: subtracting the
    // couplings' squares afterwards would cancel ||E||^2 away)
    double *sub = nullptr, *sup = nullptr;
    template <typename V>
    __device__ double operator()(int i, int j, V v) const
    {
        const double x = (double)v;
        TE[sr_idx(i, j, ldte)] = (Tl)x;
        if (That) That[sr_idx(i, j, ldt)] = x;
        if (i == j) diag[i] = x;
        if (sub) {
            if (i == j + 1) sub[j] = x;
            if (j == i + 1) sup[i] = x;
        }
        return (i > j && !(sub && i == j + 1)) ? x * x : 0.0;
    }
};

// Y = Q^H Q - I; returns y_ij^2 for ||Y||_F.
struct EpMinusI {
    double *Y; int ld;
    template <typename V>
    __device__ double operator()(int i, int j, V v) const
    {
        const double y = (i == j) ? (double)v - 1.0 : (double)v;
        Y[sr_idx(i, j, ld)] = y;
        return y * y;
    }
};

// Q_new = Q + alpha * (product):  alpha = 1/2 with product Q Delta gives
// 1/2 Q Sigma (Alg. 4, last step); alpha = -1/2 with Q Y0 gives the initial
// Newton-Schulz step 1/2 Q (3I - Q^H Q) (eq. NS).
struct EpUpdate {
    const double *Q; int ldq; double *Qn; int ldn; double alpha;
    template <typename V>
    __device__ double operator()(int i, int j, V v) const
    {
        Qn[sr_idx(i, j, ldn)] = Q[sr_idx(i, j, ldq)] + alpha * (double)v;
        return 0.0;
    }
};

// Delta = Sigma - 2I = 2W - Y - YW + W^2 + W^3 (+ W^2 Y + W^2 Y W), summed in
// high precision (Alg. 4: "compute Sigma ... in hp"); v is the entry of W^3.
template <typename Tl>
struct EpDelta {
    const Tl *L; int ldl;       // W = L - L^H from the strictly lower part
    const double *Y; int ldy;
    const Tl *YW, *W2, *W2Y, *W2YW; int ldp;   // W2Y, W2YW may be null
    double *Delta; int ldd;
    template <typename V>
    __device__ double operator()(int i, int j, V v) const
    {
        double w = 0.0;
        if (i > j) w = (double)L[sr_idx(i, j, ldl)];
        else if (i < j) w = -(double)L[sr_idx(j, i, ldl)];
        const size_t p = sr_idx(i, j, ldp);
        double d = 2.0 * w - Y[sr_idx(i, j, ldy)] - (double)YW[p] + (double)W2[p] + (double)v;
        if (W2Y) d += (double)W2Y[p] + (double)W2YW[p];
        Delta[sr_idx(i, j, ldd)] = d;
        return 0.0;
    }
};

// Delta as above with every term already in FP64 (the emulated-product pass):
// v is the entry of W^3; W2Y, W2YW may be null.
struct EpDeltaD {
    const double *W, *Y, *YW, *W2, *W2Y, *W2YW; int ld;
    double *Delta; int ldd;
    template <typename V>
    __device__ double operator()(int i, int j, V v) const
    {
        const size_t p = sr_idx(i, j, ld);
        double d = 2.0 * W[p] - Y[p] - YW[p] + W2[p] + (double)v;
        if (W2Y) d += W2Y[p] + W2YW[p];
        Delta[sr_idx(i, j, ldd)] = d;
        return 0.0;
    }
};

// ---- complex epilogues (v = complex128 value of the entry) ------------------------
// The same operations on complex data; kComplex marks them for the emulated
// products' combine step.

struct EpStoreC {
    static constexpr bool kComplex = true;
    cd *C; int ld;
    __device__ double operator()(int i, int j, cd v) const { C[sr_idx(i, j, ld)] = v; return 0.0; }
};

struct EpSplitC {
    static constexpr bool kComplex = true;
    cf *TE; int ldte; cd *diag; cd *That; int ldt;
    __device__ double operator()(int i, int j, cd v) const
    {
        TE[sr_idx(i, j, ldte)] = cf{(float)v.x, (float)v.y};
        if (That) That[sr_idx(i, j, ldt)] = v;
        if (i == j) diag[i] = v;
        return i > j ? v.x * v.x + v.y * v.y : 0.0;
    }
};

struct EpMinusIC {
    static constexpr bool kComplex = true;
    cd *Y; int ld;
    __device__ double operator()(int i, int j, cd v) const
    {
        if (i == j) v.x -= 1.0;
        Y[sr_idx(i, j, ld)] = v;
        return v.x * v.x + v.y * v.y;
    }
};

struct EpUpdateC {
    static constexpr bool kComplex = true;
    const cd *Q; int ldq; cd *Qn; int ldn; double alpha;
    __device__ double operator()(int i, int j, cd v) const
    {
        const cd q = Q[sr_idx(i, j, ldq)];
        Qn[sr_idx(i, j, ldn)] = cd{fma(alpha, v.x, q.x), fma(alpha, v.y, q.y)};
        return 0.0;
    }
};

struct EpDeltaDC {
    static constexpr bool kComplex = true;
    const cd *W, *Y, *YW, *W2, *W2Y, *W2YW; int ld;
    cd *Delta; int ldd;
    __device__ double operator()(int i, int j, cd v) const
    {
        const size_t p = sr_idx(i, j, ld);
        cd d = 2.0 * W[p] - Y[p] - YW[p] + W2[p] + v;
        if (W2Y) d = d + W2Y[p] + W2YW[p];
        Delta[sr_idx(i, j, ldd)] = d;
        return 0.0;
    }
};

// ---- small kernels -----------------------------------------------------------

// W = L - L^H in high precision (FP64 or complex128) from the strictly lower
// triangle of L (32 x 32 tiles, both the tile and its transpose staged in
// shared memory).
template <typename Tl>
__global__ void __launch_bounds__(256) form_skew_kernel(int n, const Tl *__restrict__ L, int ldl,
                                                        typename SrNum<Tl>::hp *__restrict__ W, int ldw)
{
    using H = typename SrNum<Tl>::hp;
    __shared__ H a[32][33], b[32][33];
    const H z = SrNum<H>::zero();
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int q = ty; q < 32; q += 8) {
        const int i = i0 + tx, j = j0 + q;          // tile (I, J), rows i
        a[tx][q] = (i < n && j < n) ? sr_to_hp(L[sr_idx(i, j, ldl)]) : z;
        const int i2 = j0 + tx, j2 = i0 + q;        // tile (J, I)
        b[tx][q] = (i2 < n && j2 < n) ? sr_to_hp(L[sr_idx(i2, j2, ldl)]) : z;
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {
        const int i = i0 + tx, j = j0 + q;
        if (i < n && j < n) W[sr_idx(i, j, ldw)] = (i > j) ? a[tx][q] : ((i < j) ? -sr_conj(b[q][tx]) : z);
    }
}


template <typename Tin>
__global__ void convert_to_hp_kernel(int n, const Tin *__restrict__ src, int lds,
                                     typename SrNum<Tin>::hp *__restrict__ dst, int ldd)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i < n) dst[sr_idx(i, j, ldd)] = sr_to_hp(src[sr_idx(i, j, lds)]);
}

// partial[block] = sum of squares of the selected part of an n x n matrix
// (part 0: all, 1: strictly lower).
template <typename T>
__global__ void __launch_bounds__(256) sumsq_kernel(int n, const T *__restrict__ M, int ld, int part,
                                                    double *__restrict__ partial)
{
    double s = 0.0;
    const size_t total = (size_t)n * (size_t)n;
    for (size_t e = (size_t)blockIdx.x * 256 + threadIdx.x; e < total; e += (size_t)gridDim.x * 256) {
        const int i = (int)(e % n), j = (int)(e / n);
        if (part == 1 && i <= j) continue;
        s += sr_abs2(M[sr_idx(i, j, ld)]);
    }
    s = sr_block_sum<256>(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// out[0] = sum of partial[0..count) in a fixed order (deterministic).
static __global__ void __launch_bounds__(256) reduce_partials_kernel(const double *__restrict__ partial, int count,
                                                             double *__restrict__ out)
{
    double s = 0.0;
    for (int e = threadIdx.x; e < count; e += 256) s += partial[e];
    s = sr_block_sum<256>(s);
    if (threadIdx.x == 0) *out = s;
}

// ---- double-double residual products -------------------------------------------

// C = op(A) * (Bhi + Blo) in double-double, 16 x 16 tiles, one entry per thread.
// mode 0: store C (hi, lo).  mode 1: partial += sum over i > j of (hi + lo)^2.
// mode 2: partial += sum over all (i, j) of (C - I)^2 (upper tiles only,
// off-diagonal entries counted twice; C symmetric).
// MODE 3 (the quasi-triangular form): as MODE 1 but every subdiagonal entry
// (j+1, j) is left out of the sum, and the band of C is written to
// band[0..n) (subdiagonal C(k+1, k)), band[n..2n) (superdiagonal C(k, k+1)) and
// band[2n..3n) (diagonal), each entry's double-double value rounded once.
template <int MODE>
__global__ void __launch_bounds__(256)
gemm_dd_kernel(int n, int transA, const double *__restrict__ A, int lda, const double *__restrict__ Bhi,
               const double *__restrict__ Blo, int ldb, double *__restrict__ Chi, double *__restrict__ Clo,
               int ldc, double *__restrict__ partial, double *__restrict__ band = nullptr)
{
    constexpr int T = 16;
    __shared__ double As[T][T + 1];
    __shared__ double Bh[T][T + 1];
    __shared__ double Bl[T][T + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.x * T, j0 = blockIdx.y * T;
    const size_t bid = blockIdx.x + (size_t)gridDim.x * blockIdx.y;
    // tiles that contribute nothing in modes 1 and 2 (mode 3 keeps the tiles
    // that hold superdiagonal entries)
    if ((MODE == 1 && i0 + T - 1 <= j0) || (MODE == 3 && i0 + T < j0) || (MODE == 2 && i0 > j0 + T - 1)) {
        if (threadIdx.x == 0) partial[bid] = 0.0;
        return;
    }
    const int i = i0 + tx, j = j0 + ty;
    ddv acc = {0.0, 0.0};
    for (int k0 = 0; k0 < n; k0 += T) {
        // As[kk][ii] = op(A)(i0+ii, k0+kk)
        {
            const int ii = transA ? ty : tx, kk = transA ? tx : ty;
            const int gi = i0 + ii, gk = k0 + kk;
            double v = 0.0;
            if (gi < n && gk < n) v = transA ? A[sr_idx(gk, gi, lda)] : A[sr_idx(gi, gk, lda)];
            As[kk][ii] = v;
        }
        {
            const int gk = k0 + tx, gj = j0 + ty;
            const bool in = gk < n && gj < n;
            Bh[tx][ty] = in ? Bhi[sr_idx(gk, gj, ldb)] : 0.0;
            Bl[tx][ty] = (in && Blo) ? Blo[sr_idx(gk, gj, ldb)] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < T; ++kk) acc = dd_plus(acc, dd_times(As[kk][tx], Bh[kk][ty], Bl[kk][ty]));
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
        } else if (MODE == 3) {
            const double v = acc.hi + acc.lo;
            if (i == j + 1) band[j] = v;
            else if (i > j) part = v * v;
            if (j == i + 1) band[n + i] = v;
            if (i == j) band[2 * n + i] = v;
        } else {
            if (i <= j) {
                if (i == j) acc = dd_plus(acc, {-1.0, 0.0});
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

// Complex form of gemm_dd_kernel (complex128 data; op(A) = A^H when transA):
// real and imaginary parts each accumulated in double-double.
template <int MODE>
__global__ void __launch_bounds__(256)
gemm_dd_c_kernel(int n, int transA, const cd *__restrict__ A, int lda, const cd *__restrict__ Bhi,
                 const cd *__restrict__ Blo, int ldb, cd *__restrict__ Chi, cd *__restrict__ Clo, int ldc,
                 double *__restrict__ partial)
{
    constexpr int T = 16;
    __shared__ cd As[T][T + 1];
    __shared__ cd Bh[T][T + 1];
    __shared__ cd Bl[T][T + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.x * T, j0 = blockIdx.y * T;
    const size_t bid = blockIdx.x + (size_t)gridDim.x * blockIdx.y;
    if ((MODE == 1 && i0 + T - 1 <= j0) || (MODE == 2 && i0 > j0 + T - 1)) {
        if (threadIdx.x == 0) partial[bid] = 0.0;
        return;
    }
    const int i = i0 + tx, j = j0 + ty;
    const cd z = {0.0, 0.0};
    ddv re = {0.0, 0.0}, im = {0.0, 0.0};
    for (int k0 = 0; k0 < n; k0 += T) {
        {
            const int ii = transA ? ty : tx, kk = transA ? tx : ty;
            const int gi = i0 + ii, gk = k0 + kk;
            cd v = z;
            if (gi < n && gk < n) v = transA ? conj(A[sr_idx(gk, gi, lda)]) : A[sr_idx(gi, gk, lda)];
            As[kk][ii] = v;
        }
        {
            const int gk = k0 + tx, gj = j0 + ty;
            const bool in = gk < n && gj < n;
            Bh[tx][ty] = in ? Bhi[sr_idx(gk, gj, ldb)] : z;
            Bl[tx][ty] = (in && Blo) ? Blo[sr_idx(gk, gj, ldb)] : z;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < T; ++kk) {
            const cd a = As[kk][tx], bh = Bh[kk][ty], bl = Bl[kk][ty];
            // (a.x + i a.y)(b.x + i b.y): four exact products with the low parts folded in
            re = dd_plus(re, dd_times(a.x, bh.x, bl.x));
            re = dd_plus(re, dd_times(-a.y, bh.y, bl.y));
            im = dd_plus(im, dd_times(a.x, bh.y, bl.y));
            im = dd_plus(im, dd_times(a.y, bh.x, bl.x));
        }
        __syncthreads();
    }
    double part = 0.0;
    if (i < n && j < n) {
        if (MODE == 0) {
            Chi[sr_idx(i, j, ldc)] = cd{re.hi, im.hi};
            Clo[sr_idx(i, j, ldc)] = cd{re.lo, im.lo};
        } else if (MODE == 1) {
            if (i > j) {
                const double vr = re.hi + re.lo, vi = im.hi + im.lo;
                part = vr * vr + vi * vi;
            }
        } else {
            if (i <= j) {
                if (i == j) re = dd_plus(re, {-1.0, 0.0});
                const double vr = re.hi + re.lo, vi = im.hi + im.lo;
                part = (i == j ? 1.0 : 2.0) * (vr * vr + vi * vi);
            }
        }
    }
    if (MODE != 0) {
        part = sr_block_sum<256>(part);
        if (threadIdx.x == 0) partial[bid] = part;
    }
}

}  // namespace sr
