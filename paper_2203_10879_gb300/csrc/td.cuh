// Triple-double numbers: the working precision of the SR_TARGET_TD form (Sec. 3
// refines to precisions above double-double by holding each high-precision
// number as several doubles). x = x0 + x1 + x2, where x0 is the double nearest
// to x, x1 the double nearest to x - x0 and x2 the double nearest to
// x - x0 - x1: a non-overlapping expansion with |x1| <= ulp(x0)/2 and
// |x2| <= ulp(x1)/2, about 159 significant bits.
//
// Every value the form stores is made by one rounding of an exact integer:
// either a product rebuilt from its residues, or an exact sum of a few doubles
// formed in a 256-bit fixed-point window. The rounding takes three steps of
// round-to-nearest-even on the integer, each subtracting the word it took.
#pragma once
#include <climits>
#include <cstdint>
#include <type_traits>

#include "common.cuh"

namespace sr {

struct tdv {
    double x0, x1, x2;
};

using u64 = unsigned long long;

// word q of a 256-bit little-endian integer (0 outside [0, 4)); a select chain
// keeps W in registers for a run-time q
__device__ __forceinline__ u64 u256_word(const u64 (&W)[4], int q)
{
    u64 v = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (k == q) v = W[k];
    return v;
}

// bits [s, s + 64) of W
__device__ __forceinline__ u64 u256_bits64(const u64 (&W)[4], int s)
{
    const int q = s >> 6, r = s & 63;
    const u64 lo = u256_word(W, q), hi = u256_word(W, q + 1);
    return r ? (lo >> r) | (hi << (64 - r)) : lo;
}

// index of the leading set bit of W, -1 for W = 0
__device__ __forceinline__ int u256_lead(const u64 (&W)[4])
{
    int p = -1;
#pragma unroll
    for (int k = 3; k >= 0; --k)
        if (p < 0 && W[k] != 0) p = 64 * k + 63 - __clzll((long long)W[k]);
    return p;
}

// W = W mod 2^s
__device__ __forceinline__ void u256_keep_low(u64 (&W)[4], int s)
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int b = s - 64 * k;   // bits of word k that stay
        if (b <= 0) W[k] = 0;
        else if (b < 64) W[k] &= (1ull << b) - 1ull;
    }
}

// is any of the bits [0, s) of W set
__device__ __forceinline__ bool u256_any_below(const u64 (&W)[4], int s)
{
    bool any = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int b = s - 64 * k;
        if (b >= 64) any |= W[k] != 0;
        else if (b > 0) any |= (W[k] & ((1ull << b) - 1ull)) != 0;
    }
    return any;
}

// two's complement negation of a 256-bit integer
__device__ __forceinline__ void u256_neg(u64 (&W)[4])
{
    u64 c = 1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const u64 v = ~W[k] + c;
        c = (c && v == 0) ? 1ull : 0ull;
        W[k] = v;
    }
}

// (-1)^neg M 2^e as a double, M nonzero with at most 53 significant bits (the
// value is exact). A normal result is assembled from its fields with integer
// instructions (GB300's FP64 pipe is slow); one near either end of the
// exponent range goes through scalbn.
__device__ __forceinline__ double td_make(u64 M, int e, bool neg)
{
    const int top = 63 - __clzll((long long)M);   // M in [2^top, 2^(top + 1))
    const int E = e + top + 1023;                  // biased exponent
    if (E >= 1 && E <= 2046) {
        const u64 mant = top >= 52 ? M >> (top - 52) : M << (52 - top);   // drops only zero bits
        return __longlong_as_double(
            (long long)(((u64)neg << 63) | ((u64)E << 52) | (mant & ((1ull << 52) - 1ull))));
    }
    const double v = scalbn((double)M, e);
    return neg ? -v : v;
}

// (-1)^neg W 2^xe rounded to a triple-double (W is consumed)
__device__ __forceinline__ tdv td_round_u256(u64 (&W)[4], bool neg, int xe)
{
    double out[3];
#pragma unroll
    for (int wd = 0; wd < 3; ++wd) {
        const int p = u256_lead(W);
        if (p < 0) {
            out[wd] = 0.0;
        } else if (p <= 52) {
            out[wd] = td_make(W[0], xe, neg);   // exact: at most 53 bits
            W[0] = 0;
        } else {
            const int s = p - 52;
            const u64 m = u256_bits64(W, s) & ((1ull << 53) - 1ull);
            const bool half = (u256_bits64(W, s - 1) & 1ull) != 0;   // bit s - 1
            const bool rest = u256_any_below(W, s - 1);
            const bool up = half && (rest || (m & 1ull));
            out[wd] = td_make(m + (up ? 1ull : 0ull), s + xe, neg);   // m + 1 <= 2^53: exact
            u256_keep_low(W, s);
            if (up) {
                // what is left, 2^s - W, has the other sign
                u256_neg(W);
                u256_keep_low(W, s);
                neg = !neg;
            }
        }
    }
    return {out[0], out[1], out[2]};
}

// a finite double as mant 2^ex (mant < 2^53); false for NaN and infinities
__device__ __forceinline__ bool td_unpack(double x, u64 &mant, int &ex, bool &neg)
{
    const u64 bits = (u64)__double_as_longlong(x);
    const int eb = (int)((bits >> 52) & 0x7ff);
    neg = (bits >> 63) != 0;
    mant = bits & 0xfffffffffffffull;
    ex = 0;
    if (eb == 0x7ff) return false;
    if (eb == 0) ex = -1074; else { mant |= 1ull << 52; ex = eb - 1075; }
    return true;
}

// The exact sum of C doubles, rounded to a triple-double. The terms are
// placed on the grid 2^lsb, lsb = (largest exponent) - 200, in a 256-bit two's
// complement window (the sum is below C 2^201 units); the bits of a term
// below the grid are dropped, an error below C 2^-200 of the largest term.
template <int C>
__device__ __forceinline__ tdv td_sum(const double (&t)[C])
{
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
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
    if (!fin) return {nan, nan, nan};
    if (emax == INT_MIN) return {0.0, 0.0, 0.0};
    const int lsb = emax - 200;
    u64 acc[4] = {0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < C; ++i) {
        u64 mt;
        int ex;
        bool ng;
        td_unpack(t[i], mt, ex, ng);
        if (mt == 0) continue;
        const int sh = ex - lsb;   // <= 148
        u64 v[4] = {0, 0, 0, 0};
        if (sh >= 0) {
            const int q = sh >> 6, r = sh & 63;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (k == q) v[k] = mt << r;
                if (k == q + 1 && r) v[k] = mt >> (64 - r);
            }
        } else if (sh > -64) {
            v[0] = mt >> (-sh);
        }
        if (ng) u256_neg(v);
        u64 c = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const u64 s1 = acc[k] + v[k];
            const u64 c1 = s1 < acc[k] ? 1ull : 0ull;
            const u64 s2 = s1 + c;
            const u64 c2 = s2 < s1 ? 1ull : 0ull;
            acc[k] = s2;
            c = c1 | c2;
        }
    }
    const bool neg = (acc[3] >> 63) != 0;
    if (neg) u256_neg(acc);
    return td_round_u256(acc, neg, lsb);
}

// ---- epilogues of the triple-double products (value v: the rounded product) --------
// They mark themselves with kTD; the return value is the entry's share of a
// sum of squares (as the other epilogues).

// C = v (three planes)
struct EpStoreTD {
    static constexpr bool kTD = true;
    double *C0, *C1, *C2; int ld;
    __device__ double operator()(int i, int j, const tdv &v) const
    {
        const size_t p = sr_idx(i, j, ld);
        C0[p] = v.x0; C1[p] = v.x1; C2[p] = v.x2;
        return 0.0;
    }
};

// S2: T^ into TE (its leading word: the FP64 low precision), the diagonal's
// two leading words (the divisors' double-double form), T^ itself when asked;
// returns the square of the leading word below the diagonal (||E||^2)
struct EpSplitTD {
    static constexpr bool kTD = true;
    double *TE; int ldte; double *diag, *diag_lo;
    double *T0, *T1, *T2; int ldt;
    __device__ double operator()(int i, int j, const tdv &v) const
    {
        TE[sr_idx(i, j, ldte)] = v.x0;
        if (i == j) {
            diag[i] = v.x0;
            diag_lo[i] = v.x1;
        }
        if (T0) {
            const size_t p = sr_idx(i, j, ldt);
            T0[p] = v.x0; T1[p] = v.x1; T2[p] = v.x2;
        }
        return i > j ? v.x0 * v.x0 : 0.0;
    }
};

// Y = Q^T Q - I; returns y_ij^2 (leading word)
struct EpMinusITD {
    static constexpr bool kTD = true;
    double *Y0, *Y1, *Y2; int ld;
    __device__ double operator()(int i, int j, const tdv &v) const
    {
        tdv y = v;
        if (i == j) {
            const double t[4] = {v.x0, v.x1, v.x2, -1.0};
            y = td_sum<4>(t);
        }
        const size_t p = sr_idx(i, j, ld);
        Y0[p] = y.x0; Y1[p] = y.x1; Y2[p] = y.x2;
        return y.x0 * y.x0;
    }
};

// Q_new = Q + alpha v (alpha = 1/2 for Q Delta, -1/2 for the Newton-Schulz step
// with Q Y0: a power of two, so alpha v is exact)
struct EpUpdateTD {
    static constexpr bool kTD = true;
    const double *Q0, *Q1, *Q2; int ldq;
    double *N0, *N1, *N2; int ldn;
    double alpha;
    __device__ double operator()(int i, int j, const tdv &v) const
    {
        const size_t q = sr_idx(i, j, ldq);
        const double t[6] = {Q0[q], Q1[q], Q2[q], alpha * v.x0, alpha * v.x1, alpha * v.x2};
        const tdv r = td_sum<6>(t);
        const size_t p = sr_idx(i, j, ldn);
        N0[p] = r.x0; N1[p] = r.x1; N2[p] = r.x2;
        return 0.0;
    }
};

// Delta = Sigma - 2I = 2W - Y - YW + W^2 + W^3 (+ W^2 Y + W^2 Y W), summed
// exactly and rounded once; YW, W^2 (W^2 Y, W^2 Y W) in the FP64 low
// precision, Y triple-double, v the FP64 entry of W^3; W = L - L^T from the
// strictly lower part of L.
struct EpDeltaTD {
    const double *L; int ldl;
    const double *YW, *W2, *W2Y, *W2YW; int ldp;   // W2Y, W2YW may be null
    const double *Y0, *Y1, *Y2; int ldy;
    double *D0, *D1, *D2; int ldd;
    __device__ double operator()(int i, int j, double v) const
    {
        double w = 0.0;
        if (i > j) w = L[sr_idx(i, j, ldl)];
        else if (i < j) w = -L[sr_idx(j, i, ldl)];
        const size_t p = sr_idx(i, j, ldp), y = sr_idx(i, j, ldy);
        const double e1 = W2Y ? W2Y[p] : 0.0, e2 = W2YW ? W2YW[p] : 0.0;
        const double t[9] = {2.0 * w, -Y0[y], -Y1[y], -Y2[y], -YW[p], W2[p], v, e1, e2};
        const tdv r = td_sum<9>(t);
        const size_t d = sr_idx(i, j, ldd);
        D0[d] = r.x0; D1[d] = r.x1; D2[d] = r.x2;
        return 0.0;
    }
};

template <class EP, class = void> struct ep_is_td : std::false_type {};
template <class EP> struct ep_is_td<EP, std::void_t<decltype(EP::kTD)>> : std::true_type {};

}  // namespace sr
