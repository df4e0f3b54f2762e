// Six-double numbers: the working precision of the SR_TARGET_D6 form (Sec. 3
// refines to 100 digits holding each number as 6 doubles). x = x0 + ... + x5,
// each word the double nearest to what the words before it leave: about 318
// bits (96 digits).
//
// As for the triple-double form, every stored value is one rounding of an
// exact integer: a product rebuilt from the residues of its operands' halves
// (the two-level split of the six-double products), or an exact sum of a few
// doubles in a 512-bit fixed-point window. The rounding takes six steps of
// round-to-nearest-even, each subtracting the word it took.
#pragma once
#include <climits>
#include <cstdint>
#include <type_traits>

#include "common.cuh"
#include "td.cuh"

namespace sr {

constexpr int kD6Words = 6;

struct d6v {
    double x[kD6Words];
};

// ---- NW-word little-endian unsigned integers (select chains keep them in registers)
template <int NW>
__device__ __forceinline__ u64 mw_word(const u64 (&W)[NW], int q)
{
    u64 v = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k)
        if (k == q) v = W[k];
    return v;
}

template <int NW>
__device__ __forceinline__ u64 mw_bits64(const u64 (&W)[NW], int s)
{
    const int q = s >> 6, r = s & 63;
    const u64 lo = mw_word<NW>(W, q), hi = mw_word<NW>(W, q + 1);
    return r ? (lo >> r) | (hi << (64 - r)) : lo;
}

template <int NW>
__device__ __forceinline__ int mw_lead(const u64 (&W)[NW])
{
    int p = -1;
#pragma unroll
    for (int k = NW - 1; k >= 0; --k)
        if (p < 0 && W[k] != 0) p = 64 * k + 63 - __clzll((long long)W[k]);
    return p;
}

template <int NW>
__device__ __forceinline__ void mw_keep_low(u64 (&W)[NW], int s)
{
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        const int b = s - 64 * k;
        if (b <= 0) W[k] = 0;
        else if (b < 64) W[k] &= (1ull << b) - 1ull;
    }
}

template <int NW>
__device__ __forceinline__ bool mw_any_below(const u64 (&W)[NW], int s)
{
    bool any = false;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        const int b = s - 64 * k;
        if (b >= 64) any |= W[k] != 0;
        else if (b > 0) any |= (W[k] & ((1ull << b) - 1ull)) != 0;
    }
    return any;
}

template <int NW>
__device__ __forceinline__ void mw_neg(u64 (&W)[NW])
{
    u64 c = 1;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        const u64 v = ~W[k] + c;
        c = (c && v == 0) ? 1ull : 0ull;
        W[k] = v;
    }
}

// acc += v (two's complement, NW words)
template <int NW>
__device__ __forceinline__ void mw_add(u64 (&acc)[NW], const u64 (&v)[NW])
{
    u64 c = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        const u64 s1 = acc[k] + v[k];
        const u64 c1 = s1 < acc[k] ? 1ull : 0ull;
        const u64 s2 = s1 + c;
        const u64 c2 = s2 < s1 ? 1ull : 0ull;
        acc[k] = s2;
        c = c1 | c2;
    }
}

// (-1)^neg W 2^xe rounded to K words (W is consumed)
template <int K, int NW>
__device__ __forceinline__ void mw_round(u64 (&W)[NW], bool neg, int xe, double (&out)[K])
{
#pragma unroll
    for (int wd = 0; wd < K; ++wd) {
        const int p = mw_lead<NW>(W);
        if (p < 0) {
            out[wd] = 0.0;
        } else if (p <= 52) {
            out[wd] = td_make(W[0], xe, neg);   // exact: at most 53 bits
            W[0] = 0;
        } else {
            const int s = p - 52;
            const u64 m = mw_bits64<NW>(W, s) & ((1ull << 53) - 1ull);
            const bool half = (mw_bits64<NW>(W, s - 1) & 1ull) != 0;
            const bool rest = mw_any_below<NW>(W, s - 1);
            const bool up = half && (rest || (m & 1ull));
            out[wd] = td_make(m + (up ? 1ull : 0ull), s + xe, neg);   // m + 1 <= 2^53: exact
            mw_keep_low<NW>(W, s);
            if (up) {
                mw_neg<NW>(W);
                mw_keep_low<NW>(W, s);
                neg = !neg;
            }
        }
    }
}

// The exact sum of C doubles rounded to six words: the terms on the grid
// 2^lsb, lsb = (largest exponent) - 400, in a 512-bit two's complement window
// (the sum stays below C 2^401 units); bits of a term below the grid are
// dropped, an error below C 2^-400 of the largest term.
template <int C>
__device__ __forceinline__ d6v d6_sum(const double (&t)[C])
{
    constexpr int NW = 8;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    d6v r;
    int emax = INT_MIN;
    bool fin = true;
#pragma unroll
    for (int i = 0; i < C; ++i) {
        u64 mt;
        int ex;
        bool ng;
        fin &= td_unpack(t[i], mt, ex, ng);
        if (mt != 0) emax = max(emax, ex + 52);
    }
    if (!fin || emax == INT_MIN) {
#pragma unroll
        for (int k = 0; k < kD6Words; ++k) r.x[k] = fin ? 0.0 : nan;
        return r;
    }
    const int lsb = emax - 400;
    u64 acc[NW];
#pragma unroll
    for (int k = 0; k < NW; ++k) acc[k] = 0;
#pragma unroll
    for (int i = 0; i < C; ++i) {
        u64 mt;
        int ex;
        bool ng;
        td_unpack(t[i], mt, ex, ng);
        if (mt == 0) continue;
        const int sh = ex - lsb;   // <= 348
        u64 v[NW];
#pragma unroll
        for (int k = 0; k < NW; ++k) v[k] = 0;
        if (sh >= 0) {
            const int q = sh >> 6, rr = sh & 63;
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                if (k == q) v[k] = mt << rr;
                if (k == q + 1 && rr) v[k] = mt >> (64 - rr);
            }
        } else if (sh > -64) {
            v[0] = mt >> (-sh);
        }
        if (ng) mw_neg<NW>(v);
        mw_add<NW>(acc, v);
    }
    const bool neg = (acc[NW - 1] >> 63) != 0;
    if (neg) mw_neg<NW>(acc);
    mw_round<kD6Words, NW>(acc, neg, lsb, r.x);
    return r;
}

// ---- epilogues of the six-double products (value v: the rounded product) ----------
// marked with kD6; planes are `pl` elements apart (the caller's ld * columns,
// or the workspace's n_max^2)

struct EpStoreD6 {
    static constexpr bool kD6 = true;
    double *C; int ld; size_t pl;
    __device__ double operator()(int i, int j, const d6v &v) const
    {
        const size_t p = sr_idx(i, j, ld);
#pragma unroll
        for (int k = 0; k < kD6Words; ++k) C[p + k * pl] = v.x[k];
        return 0.0;
    }
};

// S2: T^ into TE (leading word), the diagonal's two leading words, T^ itself
// when asked; returns the square of the leading word below the diagonal
struct EpSplitD6 {
    static constexpr bool kD6 = true;
    double *TE; int ldte; double *diag, *diag_lo;
    double *T; int ldt; size_t pl;
    __device__ double operator()(int i, int j, const d6v &v) const
    {
        TE[sr_idx(i, j, ldte)] = v.x[0];
        if (i == j) {
            diag[i] = v.x[0];
            diag_lo[i] = v.x[1];
        }
        if (T) {
            const size_t p = sr_idx(i, j, ldt);
#pragma unroll
            for (int k = 0; k < kD6Words; ++k) T[p + k * pl] = v.x[k];
        }
        return i > j ? v.x[0] * v.x[0] : 0.0;
    }
};

// Y = Q^T Q - I; returns y_ij^2 (leading word)
struct EpMinusID6 {
    static constexpr bool kD6 = true;
    double *Y; int ld; size_t pl;
    __device__ double operator()(int i, int j, const d6v &v) const
    {
        d6v y = v;
        if (i == j) {
            double t[kD6Words + 1];
#pragma unroll
            for (int k = 0; k < kD6Words; ++k) t[k] = v.x[k];
            t[kD6Words] = -1.0;
            y = d6_sum<kD6Words + 1>(t);
        }
        const size_t p = sr_idx(i, j, ld);
#pragma unroll
        for (int k = 0; k < kD6Words; ++k) Y[p + k * pl] = y.x[k];
        return y.x[0] * y.x[0];
    }
};

// Q_new = Q + alpha v, alpha a power of two
struct EpUpdateD6 {
    static constexpr bool kD6 = true;
    const double *Q; int ldq; size_t plq;
    double *N; int ldn; size_t pln;
    double alpha;
    __device__ double operator()(int i, int j, const d6v &v) const
    {
        const size_t q = sr_idx(i, j, ldq);
        double t[2 * kD6Words];
#pragma unroll
        for (int k = 0; k < kD6Words; ++k) {
            t[k] = Q[q + k * plq];
            t[kD6Words + k] = alpha * v.x[k];
        }
        const d6v r = d6_sum<2 * kD6Words>(t);
        const size_t p = sr_idx(i, j, ldn);
#pragma unroll
        for (int k = 0; k < kD6Words; ++k) N[p + k * pln] = r.x[k];
        return 0.0;
    }
};

// Delta = 2W - Y - YW + W^2 + W^3 (+ W^2 Y + W^2 Y W) summed exactly, Y six-double,
// the others FP64 (v: the entry of W^3); W = L - L^T from the strictly lower L
struct EpDeltaD6 {
    const double *L; int ldl;
    const double *YW, *W2, *W2Y, *W2YW; int ldp;
    const double *Y; int ldy; size_t ply;
    double *D; int ldd; size_t pld;
    __device__ double operator()(int i, int j, double v) const
    {
        double w = 0.0;
        if (i > j) w = L[sr_idx(i, j, ldl)];
        else if (i < j) w = -L[sr_idx(j, i, ldl)];
        const size_t p = sr_idx(i, j, ldp), y = sr_idx(i, j, ldy);
        double t[kD6Words + 6];
        t[0] = 2.0 * w;
#pragma unroll
        for (int k = 0; k < kD6Words; ++k) t[1 + k] = -Y[y + k * ply];
        t[kD6Words + 1] = -YW[p];
        t[kD6Words + 2] = W2[p];
        t[kD6Words + 3] = v;
        t[kD6Words + 4] = W2Y ? W2Y[p] : 0.0;
        t[kD6Words + 5] = W2YW ? W2YW[p] : 0.0;
        const d6v r = d6_sum<kD6Words + 6>(t);
        const size_t d = sr_idx(i, j, ldd);
#pragma unroll
        for (int k = 0; k < kD6Words; ++k) D[d + k * pld] = r.x[k];
        return 0.0;
    }
};

template <class EP, class = void> struct ep_is_d6 : std::false_type {};
template <class EP> struct ep_is_d6<EP, std::void_t<decltype(EP::kD6)>> : std::true_type {};

}  // namespace sr
