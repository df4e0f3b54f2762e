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

// ---- complex numbers (interleaved re, im; the layout of complex64/complex128) ----
struct __align__(8) cf { float x, y; };
struct __align__(16) cd { double x, y; };

__host__ __device__ inline cf operator+(cf a, cf b) { return {a.x + b.x, a.y + b.y}; }
__host__ __device__ inline cf operator-(cf a, cf b) { return {a.x - b.x, a.y - b.y}; }
__host__ __device__ inline cf operator-(cf a) { return {-a.x, -a.y}; }
__host__ __device__ inline cf operator*(cf a, cf b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__host__ __device__ inline cd operator+(cd a, cd b) { return {a.x + b.x, a.y + b.y}; }
__host__ __device__ inline cd operator-(cd a, cd b) { return {a.x - b.x, a.y - b.y}; }
__host__ __device__ inline cd operator-(cd a) { return {-a.x, -a.y}; }
__host__ __device__ inline cd operator*(cd a, cd b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__host__ __device__ inline cd operator*(double s, cd a) { return {s * a.x, s * a.y}; }
__host__ __device__ inline bool operator==(cf a, cf b) { return a.x == b.x && a.y == b.y; }
__host__ __device__ inline bool operator==(cd a, cd b) { return a.x == b.x && a.y == b.y; }
__host__ __device__ inline cd conj(cd a) { return {a.x, -a.y}; }
__host__ __device__ inline cf conj(cf a) { return {a.x, -a.y}; }
__device__ inline bool sr_finite(cf a) { return isfinite(a.x) && isfinite(a.y); }
__device__ inline bool sr_finite(cd a) { return isfinite(a.x) && isfinite(a.y); }

// c + a * b in the working type (one fused operation per real multiply)
__device__ inline float sr_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ inline double sr_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ inline cf sr_fma(cf a, cf b, cf c)
{
    return {fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y))};
}
__device__ inline cd sr_fma(cd a, cd b, cd c)
{
    return {fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y))};
}
__device__ inline float sr_shfl(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ inline double sr_shfl(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ inline cf sr_shfl(cf v, int src) { return {__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src)}; }
__device__ inline cd sr_shfl(cd v, int src) { return {__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src)}; }
// |x| > cap (|x|^2 > cap^2 for complex x, products and sum rounded
// separately), in the working precision: the entry threshold of Example 4
__device__ inline bool sr_over_cap(float x, double cap) { return fabsf(x) > (float)cap; }
__device__ inline bool sr_over_cap(double x, double cap) { return fabs(x) > cap; }
__device__ inline bool sr_over_cap(cf x, double cap)
{
    const float c = (float)cap;
    return __fadd_rn(__fmul_rn(x.x, x.x), __fmul_rn(x.y, x.y)) > __fmul_rn(c, c);
}
__device__ inline bool sr_over_cap(cd x, double cap)
{
    return __dadd_rn(__dmul_rn(x.x, x.x), __dmul_rn(x.y, x.y)) > __dmul_rn(cap, cap);
}
// 1 / z by Smith's scaling (avoids overflow in |z|^2)
__device__ inline float sr_recip(float z) { return 1.0f / z; }
__device__ inline double sr_recip(double z) { return 1.0 / z; }
__device__ inline cf sr_recip(cf z)
{
    if (fabsf(z.x) >= fabsf(z.y)) {
        const float r = z.y / z.x, d = z.x + z.y * r;
        return {1.0f / d, -r / d};
    }
    const float r = z.x / z.y, d = z.x * r + z.y;
    return {r / d, -1.0f / d};
}
__device__ inline cd sr_recip(cd z)
{
    if (fabs(z.x) >= fabs(z.y)) {
        const double r = z.y / z.x, d = z.x + z.y * r;
        return {1.0 / d, -r / d};
    }
    const double r = z.x / z.y, d = z.x * r + z.y;
    return {r / d, -1.0 / d};
}

// types of the high-precision counterpart (diagonals) and zero; kind tells
// the four number types apart (float, double, complex64, complex128)
template <typename T> struct SrNum;
template <> struct SrNum<float> {
    using hp = double;
    static constexpr int kind = 0;
    __host__ __device__ static float zero() { return 0.0f; }
    __host__ __device__ static float one() { return 1.0f; }
    __device__ static float from_hp(double v) { return (float)v; }
};
template <> struct SrNum<double> {
    using hp = double;
    static constexpr int kind = 1;
    __host__ __device__ static double zero() { return 0.0; }
    __host__ __device__ static double one() { return 1.0; }
    __device__ static double from_hp(double v) { return v; }
};
template <> struct SrNum<cf> {
    using hp = cd;
    static constexpr int kind = 2;
    __host__ __device__ static cf zero() { return {0.0f, 0.0f}; }
    __host__ __device__ static cf one() { return {1.0f, 0.0f}; }
    __device__ static cf from_hp(cd v) { return {(float)v.x, (float)v.y}; }
};
template <> struct SrNum<cd> {
    using hp = cd;
    static constexpr int kind = 3;
    __host__ __device__ static cd zero() { return {0.0, 0.0}; }
    __host__ __device__ static cd one() { return {1.0, 0.0}; }
    __device__ static cd from_hp(cd v) { return v; }
};

// widening to the high-precision type, |x|^2 in FP64, conjugate (identity for reals)
__device__ inline double sr_to_hp(float x) { return (double)x; }
__device__ inline double sr_to_hp(double x) { return x; }
__device__ inline cd sr_to_hp(cf x) { return {(double)x.x, (double)x.y}; }
__device__ inline cd sr_to_hp(cd x) { return x; }
__device__ inline double sr_abs2(float x) { return (double)x * (double)x; }
__device__ inline double sr_abs2(double x) { return x * x; }
__device__ inline double sr_abs2(cf x) { return (double)x.x * (double)x.x + (double)x.y * (double)x.y; }
__device__ inline double sr_abs2(cd x) { return x.x * x.x + x.y * x.y; }
__device__ inline float sr_conj(float x) { return x; }
__device__ inline double sr_conj(double x) { return x; }
__device__ inline cf sr_conj(cf x) { return conj(x); }
__device__ inline cd sr_conj(cd x) { return conj(x); }

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

// ---- double-double arithmetic (hi + lo, |lo| <= ulp(hi)/2 after renormalisation) ----
// Knuth's TwoSum, the fast renormalisation of Dekker, and products through
// fused multiply-adds (exact a*b = p + fma(a, b, -p)).
struct ddv { double hi, lo; };

__device__ inline ddv dd_two_sum(double a, double b)
{
    const double s = a + b;
    const double z = s - a;
    return {s, (a - (s - z)) + (b - z)};
}
__device__ inline ddv dd_renorm(double a, double b)
{
    const double s = a + b;
    return {s, b - (s - a)};
}
__device__ inline ddv dd_plus(ddv a, ddv b)
{
    ddv s = dd_two_sum(a.hi, b.hi);
    const ddv t = dd_two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = dd_renorm(s.hi, s.lo);
    s.lo += t.lo;
    return dd_renorm(s.hi, s.lo);
}
// exact product a*b as hi + lo, plus a*c folded into the low part
__device__ inline ddv dd_times(double a, double b, double c)
{
    const double p = a * b;
    double e = fma(a, b, -p);
    e = fma(a, c, e);
    return {p, e};
}

// a + b for a double b
__device__ inline ddv dd_plus_d(ddv a, double b)
{
    ddv s = dd_two_sum(a.hi, b);
    s.lo += a.lo;
    return dd_renorm(s.hi, s.lo);
}
// (ah + al)(bh + bl): the exact product of the high parts plus the two cross
// terms (al*bl is below the double-double rounding and dropped)
__device__ inline ddv dd_mul(ddv a, ddv b)
{
    const double p = a.hi * b.hi;
    double e = fma(a.hi, b.hi, -p);
    e = fma(a.hi, b.lo, e);
    e = fma(a.lo, b.hi, e);
    return dd_renorm(p, e);
}
// a + b with the low parts added in double (the accumulation of products:
// the error stays below a few units of 2^-104 times |a| + |b|)
__device__ inline ddv dd_acc(ddv a, ddv b)
{
    ddv s = dd_two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return dd_renorm(s.hi, s.lo);
}
