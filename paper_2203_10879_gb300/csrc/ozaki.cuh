// FP64 products emulated on the bf16 tensor cores (Ozaki-style splitting).
//
// The paper computes its high-precision products with the Ozaki scheme
// (Sec. 3: the `acc` toolbox, Ozaki, Ogita, Oishi and Rump 2012). On GB300 the
// FP64 pipe delivers ~1.2 TFLOP/s and tcgen05 has no integer MMA for sm_103a,
// so the split here targets bf16 operands with FP32 accumulation:
//
//  * every vector (a row of op(A) or a column of B) gets a power-of-two scale
//    2^e with |entries| < 2^e; the scaled entries x in (-1, 1) are written in
//    fixed point with F = 7 + 8(s-1) fraction bits and cut into s signed digits
//    sigma_p in [-128, 128], x ~ sum_p sigma_p 2^(-7-8p) (p = 0..s-1). The
//    digits are exact in bf16. The cut is integer arithmetic only.
//  * digit matrices are multiplied pairwise on tcgen05 (kind::f16, FP32
//    accumulation in TMEM) in K-chunks of 256: every partial sum is an
//    integer below 2^22 in magnitude, hence exact. Chunk results are drained
//    from TMEM and summed exactly in 32-bit integers per level l = p + q.
//    Levels l = 0..s-1 are kept (the pairs with p + q <= s - 1).
//  * a combine kernel rebuilds C(i,j) = 2^(e_i + f_j) sum_l I_l 2^(-14-8l) in
//    FP64 and hands it to the same fused epilogues as the native FP64 path.
//
// Digits live in "slots" so that one split serves several products: the
// columns of Q feed A Q, Q^T (A Q) and Q^T Q in the same pass.
//
// Complex operands (a work area made with cplx = true): a vector x = xr + i xi
// is stored as the real vector [xr; xi] of length 2 Kh (each half padded to
// Kh, a multiple of the K-chunk) with one scale for both parts. With r_i the
// stacked row-side vector and c_j the stacked column-side vector, one output
// entry needs two real dot products over 2 Kh:
//     re = r1.c1 - g r2.c2,   im = r1.c2 + g r2.c1,
// g = -1 when the row-side slot holds columns (op = conjugate transpose, the
// only use of column digits on the row side) and g = +1 when it holds rows.
// The slice-product kernel forms them as two output columns per j (the real
// parts in plane columns [0, Pmax), the imaginary ones in [Pmax, 2 Pmax)):
// for the imaginary half the column-side K-chunks are read with the halves
// swapped, and the chunks that carry a minus sign are issued with the
// instruction descriptor's negate-A bit. Every partial sum stays an exact
// integer, as in the real case.
//
// Residue form (the Chinese-remainder variant of the scheme, selected per
// slot): instead of cutting x into digits, every vector's entries become one
// integer X = round(x 2^(t - e)) with |X| <= 2^t, and X is stored as its
// residues modulo N pairwise coprime moduli m_1..N <= 256 (symmetric residues
// in [-128, 128], exact in bf16). The integer product C = A_int B_int is then
// formed exactly modulo each m_l by ONE tcgen05 product of the residue
// matrices (FP32 sums exact as above, drained into an exact int32 sum and
// reduced modulo m_l into a byte plane), and rebuilt from its N residues by
// the Chinese remainder theorem: C = sum_l R_l w_l mod M, w_l = M_l (M_l^-1
// mod m_l), M = prod m_l, M_l = M / m_l, taken in (-M/2, M/2]. The rebuild is
// exact when K 2^(2t) < M / 2, which fixes t from N and the inner length K:
// N = 16 gives t = 56 at K <= 4096 (16 products where 7 digits take 28 digit
// pairs), N = 32 gives t = 113 at K <= 8192 for double-double operands.
#pragma once
#include <climits>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "td.cuh"
#include "d6.cuh"

namespace sr {

constexpr int kOzakiMaxSlices = 7;   // 7 + 8*6 = 55 fraction bits fit a 64-bit integer
constexpr int kOzakiDefaultSlices = 7;
// double-double operands: 7 + 8*13 = 111 fraction bits in a 128-bit integer
constexpr int kOzakiMaxSlicesDD = 14;
constexpr int kOzakiDefaultSlicesDD = 14;
constexpr int kOzakiLpSlices = 3;    // 23 fraction bits: the FP32-class products YW, W^2, W^3
constexpr bool kOzakiBuilt = true;
constexpr int kOzakiTileI = 256;      // rows of C per slice-product tile (MMA N)
constexpr int kOzakiTileJ = 128;      // columns of C per slice-product tile (MMA M, TMEM lanes)
constexpr int kOzakiKChunk = 256;
constexpr int kOzakiMaxK = 16384;     // keeps every level sum below 2^31
constexpr int kOzakiExpNonfinite = INT_MIN;
constexpr int kOzakiSlots = 12;
// residue form
constexpr int kCrtMaxModuli = 49;         // every pairwise coprime integer <= 256 the greedy rule takes
constexpr int kCrtDefaultModuli = 16;     // FP64 operands: t = 56 bits at K <= 4096
constexpr int kCrtDefaultModuliDD = 32;   // double-double operands: t = 113 bits at K <= 8192
constexpr int kCrtMaxModuliDD = 34;       // the most whose product stays below 2^256 (8 limbs)
constexpr int kCrtDefaultModuliTD = 48;   // triple-double operands: t = 162 bits at K <= 4096
constexpr int kCrtMaxLimbs = 12;          // 32-bit limbs of M (4 for N <= 16, 8 for N <= 34, 12 for N <= 49)

// The moduli in order: the largest pairwise coprime integers <= 256 taken
// greedily from 256 down (the host table builder computes the same list).
// A function of literals, so that in fully unrolled device loops every
// constant derived from a modulus folds into an immediate.
__host__ __device__ constexpr int crt_mod(int l)
{
    constexpr int kList[kCrtMaxModuli] = {256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211,
                                          199, 197, 193, 191, 181, 179, 173, 167, 163, 157, 151, 149, 139,
                                          137, 131, 127, 113, 109, 107, 103, 101, 97,  89,  83,  79,  73,
                                          71,  67,  61,  59,  53,  47,  43,  41,  37,  29};
    return l >= 0 && l < kCrtMaxModuli ? kList[l] : 1;
}
// 2^(16 k) mod m_l
__host__ __device__ constexpr uint32_t crt_pw16(int k, int l)
{
    unsigned long long p = 1;
    for (int i = 0; i < k; ++i) p = (p * 65536ull) % (unsigned long long)crt_mod(l);
    return (uint32_t)(p % (unsigned long long)crt_mod(l));
}
// ceil(2^38 / m_l): for 0 <= v < 2^28, floor(v / m) = (v * inv38) >> 38 (the
// rounding up adds less than v / 2^38 < 2^-10 < 1/m, and v / m is at least
// 1/m below the next integer); it fits 32 bits for every m >= 65
__host__ __device__ constexpr uint32_t crt_inv38(int l)
{
    return (uint32_t)(((1ull << 38) + (unsigned long long)crt_mod(l) - 1) / (unsigned long long)crt_mod(l));
}
// a multiple of m_l that is at least 2^27
__host__ __device__ constexpr uint32_t crt_off27(int l)
{
    return (uint32_t)crt_mod(l) * (((1u << 27) + (uint32_t)crt_mod(l) - 1) / (uint32_t)crt_mod(l));
}

// Moduli, CRT weights and the constants of the residue kernels (host-built,
// one copy per work area in device memory).
struct CrtTable {
    int N = 0;                                   // moduli in use
    int L = 0;                                   // 32-bit limbs holding M (M < 2^(32 L))
    double log2M = 0.0;
    int sigma = 0;                               // M and the weights are stored times 2^sigma
    float invMtop = 0.f;                         // 2^(32 (L - 1)) / (M 2^sigma)
    int m[kCrtMaxModuli];                        // the moduli, pairwise coprime, <= 256
    unsigned long long inv40[kCrtMaxModuli];     // ceil(2^40 / m): v / m = (v inv40) >> 40 for v < 2^31
    unsigned off28[kCrtMaxModuli];               // m ceil(2^28 / m): makes |v| < 2^28 non-negative mod m
    unsigned pw16[12][kCrtMaxModuli];            // 2^(16 k) mod m
    unsigned w[kCrtMaxModuli][kCrtMaxLimbs];     // CRT weights w_l < M, times 2^sigma, little-endian limbs
    unsigned M[kCrtMaxLimbs];                    // M 2^sigma (top bit at 32 L - 1)
    unsigned halfM[kCrtMaxLimbs];                // M 2^(sigma - 1)
};

// Builds the table for the first N moduli of the fixed list (the largest
// pairwise coprime integers <= 256, greedily), with M held in L = 4 limbs
// (FP64 results), 8 (double-double results) or 12 (triple-double results).
// Returns false for N outside [1, kCrtMaxModuli] or M >= 2^(32 L).
bool crt_build_table(int N, int L, CrtTable &t);
// Bits t of the integer operands for N moduli and inner length K: the
// largest t with K 2^(2t) < M / 2 (every rebuilt C is then exact).
int crt_bits(const CrtTable &t, long long K);

// vectors of a split: columns (contiguous in a column-major matrix) or rows
enum { OZ_COLS = 0, OZ_ROWS = 1 };

struct OzakiSlot {
    int cap = 0;                           // digits (residues) this slot can hold
    int crt = 0;                           // 1: residue form (see the header), 0: digits
    int t = 0;                             // residue form: bits of the integers of the last split
    int layout = OZ_COLS;                  // vectors of the last split (OZ_COLS or OZ_ROWS)
    void *dig = nullptr;                   // bf16 digits [cap][Pmax][Kmax]
    int *exps = nullptr;                   // [Pmax]
    alignas(64) unsigned char map_i[128];  // CUtensorMap over the digits, boxes of kOzakiTileI rows
    alignas(64) unsigned char map_j[128];  // the same with boxes of kOzakiTileJ rows
};

struct OzakiWork {
    int nmax = 0, Pmax = 0, Kmax = 0;
    bool cplx = false;                     // complex128 operands, stacked [re; im] digit vectors
    OzakiSlot slot[kOzakiSlots];
    int levels = 0;                        // level planes held (the largest slot capacity, at least 7)
    long long pstride_group = 0;           // grouped work area: elements per level plane
    // autotuner of the slice products' work split: the level-group count chosen
    // for each product shape (active tiles, digits, K-chunks, parts) by timing
    // the candidates on its first launch
    struct Tuned { long long key; int groups; };
    std::vector<Tuned> tuned;
    bool autotune = false;
    cudaEvent_t tev[2] = {nullptr, nullptr};
    int32_t *planes = nullptr;             // [levels][Pmax (2 Pmax if cplx) cols][Pmax rows]; the
                                           // residue form keeps byte planes [N][...] in the same buffer
    CrtTable crt;                          // residue form: host copy of the table
    CrtTable *crt_dev = nullptr;           // and its device copy (null when no slot uses residues)
    unsigned long long *vmax = nullptr;    // per-vector largest |x| (bit pattern) during a split
};

// caps[i] = digits of slot i (0 = unused); cplx: complex128 operands;
// crt_moduli > 0: slots with crt_mask bit i set hold residues modulo that
// many moduli instead of digits, rebuilt into FP64 (crt_limbs = 4),
// double-double (8) or triple- and six-double (12) results; crt_sets plane
// sets of byte planes are kept (4 for the six-double products)
cudaError_t ozaki_alloc(OzakiWork &w, int nmax, const int *caps, bool cplx, int crt_moduli = 0,
                        unsigned crt_mask = 0, int crt_limbs = 4, int crt_sets = 1);

// ---- groups of independent products (many matrices in one launch) -------------------
// A work area for a group holds the vectors of every matrix one after another
// in each digit slot: matrix b's vectors are slot rows [row0_b, row0_b + R_b),
// row0_b a multiple of 32; `rows` is the total (the slot's row stride Pmax).
// Level planes are per-matrix regions at plane offsets chosen by the caller.
// crt_moduli > 0: the slots in crt_mask hold residues (FP64 results, 4 limbs),
// whose byte planes share the level planes' buffer (plane stride plane_elems bytes)
cudaError_t ozaki_alloc_group(OzakiWork &w, int rows, int kmax, const int *caps, long long plane_elems,
                              int crt_moduli = 0, unsigned crt_mask = 0);

// one matrix of a grouped split: vectors r < R of length K (layout as in
// ozaki_split) go to slot rows row0 + r
struct SplitMat {
    const double *X;
    int ld, R, K, row0;
    int t = 0;   // residue form: fixed-point bits of the vectors
};

// one output tile of a slice product (a work item of the grouped launch)
struct MmaItem {
    int ra, rb;         // slot rows of the tile's first output row (row side) and column (column side)
    int nch;            // K-chunks of 256
    int kbl;            // K-blocks of 64 in the last chunk (1..4): K past the order is skipped
    int lb, le;         // levels [lb, le)
    int ldp;            // plane leading dimension
    int rlim, clim;     // rows / columns of the plane region from the tile's origin (writes beyond are dropped)
    long long poff;     // plane element of the tile's origin
};

// one matrix of a grouped combine: C (m x n) from the plane region at poff
// (leading dimension ldp); exponents of slot rows ra + i and rb + j
struct CombMat {
    long long poff;
    int ldp, m, n, ra, rb;
    int tsum = 0;   // residue form: t of the row side plus t of the column side
};

// The flat grids of a grouped split (device arrays): matrix a of the launch
// owns blocks [start[a], start[a + 1]) of each kernel's grid.
struct GroupSplit {
    const SplitMat *mats;
    const int *start_max;   // absmax blocks: ceil(R/32) x ceil(K/256) per matrix
    const int *start_dig;   // digit blocks: ceil(R/32) x ceil(K/64) per matrix
    int m, total_max, total_dig, maxK;
};

// matrix of flat block x: the largest a with start[a] <= x (start[m] = total)
__device__ __forceinline__ int group_find(const int *__restrict__ start, int m, int x)
{
    int lo = 0, hi = m;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (start[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

sr_status ozaki_split_group(schur_refine_ctx *h, cudaStream_t st, OzakiWork &w, int slot, const GroupSplit &g,
                            int layout, int s, long long bytes);
sr_status ozaki_product_items(schur_refine_ctx *h, cudaStream_t st, OzakiWork &w, int rows, int cols,
                              const MmaItem *items, int nitems, int s, long long flops, int *flags);
void ozaki_free(OzakiWork &w);

// longest inner dimension a work area of order nmax takes
inline int ozaki_k_limit(bool cplx) { return cplx ? kOzakiMaxK / 2 : kOzakiMaxK; }

// Splits the R vectors of length K of X (double, or complex128 when w.cplx;
// column-major with leading dimension ld; vectors = columns or rows) into s
// digits in `slot`.
sr_status ozaki_split(schur_refine_ctx *h, cudaStream_t st, OzakiWork &w, int slot, int R, int K, const void *X,
                      int ld, int layout, int s);

// The same for double-double vectors X = Xhi + Xlo (real): the fixed-point
// value of each entry is formed exactly in a 128-bit integer before the cut,
// so up to kOzakiMaxSlicesDD digits carry the low part.
sr_status ozaki_split_dd(schur_refine_ctx *h, cudaStream_t st, OzakiWork &w, int slot, int R, int K,
                         const double *Xhi, const double *Xlo, int ld, int layout, int s);
// Triple-double operands (three planes): residues modulo the 48 moduli of the
// triple-double form (t = 162 bits at K <= 4096)
sr_status ozaki_split_td(schur_refine_ctx *h, cudaStream_t st, OzakiWork &w, int slot, int R, int K,
                         const double *X0, const double *X1, const double *X2, int ld, int layout, int s);
// Six-double operands (6 planes, plane k at X + k * pl): the fixed-point value of
// T = 2t - 2 bits cut into halves X_hi 2^t + X_lo, their residues into the
// slots slot_hi and slot_lo (48 moduli each, t = 162 bits at K <= 4096)
sr_status ozaki_split_d6(schur_refine_ctx *h, cudaStream_t st, OzakiWork &w, int slot_hi, int slot_lo, int R, int K,
                         const double *X, size_t pl, int ld, int layout);

// Level planes of the product of the vectors in slot `rows` (output rows i)
// with those in slot `cols` (output columns j), inner length k. With
// symmetric = true only tiles with i-tile <= j-tile are formed. Complex: the
// row side is conjugated when slot `rows` holds columns (op = ^H).
sr_status ozaki_product(schur_refine_ctx *h, cudaStream_t st, OzakiWork &w, int rows, int cols, int m, int n, int k,
                        int s, bool symmetric, int *flags, int32_t *planes = nullptr);

// v * 2^e as a product of two normal doubles (e within +-2044)
__device__ inline double oz_pow2_scale(double v, int e)
{
    const int e1 = e / 2, e2 = e - e / 2;
    const double p1 = __longlong_as_double((long long)(1023 + e1) << 52);
    const double p2 = __longlong_as_double((long long)(1023 + e2) << 52);
    return (v * p1) * p2;
}

// v * 2^e by adding to the exponent field when v and the result are normal
// (integer work only), else through oz_pow2_scale.
__device__ inline double oz_scale(double v, int e)
{
    const long long b = __double_as_longlong(v);
    const int eb = (int)((b >> 52) & 0x7ff);
    if (eb > 0 && eb + e > 0 && eb + e < 2047) return __longlong_as_double(b + ((long long)e << 52));
    if (v == 0.0) return v;
    return oz_pow2_scale(v, e);
}

// m * 2^x as a double for 2^52 <= m < 2^53 (the leading bit at 52), built
// from its fields when the result is normal, else by two exact scalings
__device__ __forceinline__ double oz_make_double(unsigned long long m, int x, bool neg)
{
    const int E = x + 52 + 1023;
    if (E >= 1 && E <= 2046) {
        const unsigned long long b = ((unsigned long long)E << 52) | (m & 0xfffffffffffffull);
        return __longlong_as_double((long long)(neg ? (b | 0x8000000000000000ull) : b));
    }
    const double v = oz_pow2_scale((double)m, x);
    return neg ? -v : v;
}

// bit index of the leading one of M > 0
__device__ __forceinline__ int oz_msb(unsigned __int128 M)
{
    const unsigned long long hw = (unsigned long long)(M >> 64), lw = (unsigned long long)M;
    return hw ? 127 - __clzll((long long)hw) : 63 - __clzll((long long)lw);
}

// V * 2^x rounded once to the nearest double (ties away from zero): integer
// work only, the fields of the result built directly
__device__ __forceinline__ double oz_i128_to_double(__int128 V, int x)
{
    if (V == 0) return 0.0;
    const bool neg = V < 0;
    unsigned __int128 M = neg ? (unsigned __int128)(-V) : (unsigned __int128)V;
    int sh = oz_msb(M) - 52;
    unsigned long long m;
    if (sh <= 0) {
        m = (unsigned long long)M << (-sh);
    } else {
        M += (unsigned __int128)1 << (sh - 1);        // half a unit of the last kept bit
        if ((M >> (sh + 53)) != 0) ++sh;              // the rounding carried into a new leading bit
        m = (unsigned long long)(M >> sh);
    }
    return oz_make_double(m, sh + x, neg);
}

// One rebuilt entry: (-1)^neg 2^e sum_l I_l 2^(-14-8l). The s <= 7 level sums
// are added exactly in a 128-bit integer, V = sum_l I_l 256^(s-1-l) (|V| < 2^80
// for level sums below 2^31), and V 2^(e - 14 - 8(s-1)) is rounded once to a
// double without FP64 instructions (the combine is otherwise bound by the FP64
// pipe, the scarcest unit of this GPU).
__device__ __forceinline__ double oz_rebuild(const int32_t *__restrict__ planes, size_t off, size_t pstride, int s,
                                             bool neg, int e)
{
    // all level loads first (predicated), so that they are in flight together
    int32_t v[kOzakiMaxSlices];
#pragma unroll
    for (int l = 0; l < kOzakiMaxSlices; ++l) v[l] = l < s ? planes[off + (size_t)l * pstride] : 0;
    __int128 V = 0;
#pragma unroll
    for (int l = 0; l < kOzakiMaxSlices; ++l)
        if (l < s) V = V * 256 + (__int128)v[l];
    return oz_i128_to_double(neg ? -V : V, e - 14 - 8 * (s - 1));
}

// C(i,j) = sign * (rebuilt product); ep as in gemm_simt.cuh (a complex value
// cd when CPLX). With mirror, the entries below the diagonal are read from the
// transposed position (conjugated when CPLX: the product is Hermitian). A block
// wholly below the diagonal reads its mirrored block with lanes along the
// planes' contiguous index and turns it in shared memory, so that both the
// plane reads and the epilogue's accesses are coalesced.
template <class EP, bool CPLX>
__global__ void __launch_bounds__(256)
ozaki_combine_kernel(int m, int n, int s, const int32_t *__restrict__ planes, int ldp, size_t pstride, size_t imoff,
                     const int *__restrict__ ea, const int *__restrict__ fb, double sign, int mirror, EP ep,
                     double *partial)
{
    using VT = std::conditional_t<CPLX, cd, double>;
    const int i = blockIdx.x * 32 + (threadIdx.x & 31);
    const int jb = blockIdx.y * 32 + (threadIdx.x >> 5);
    const bool neg = sign < 0;
    double part = 0.0;
    if (mirror && blockIdx.x > blockIdx.y) {
        __shared__ VT turned[32][33];
        const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
        const int lj = threadIdx.x & 31, wi = threadIdx.x >> 5;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int li = wi + 8 * w, ii = i0 + li, jj = j0 + lj;
            if (ii < m && jj < n) {
                const size_t off = (size_t)jj + (size_t)ii * (size_t)ldp;   // entry (jj, ii) of the planes
                const int e1 = ea[ii], e2 = fb[jj];
                const bool bad = e1 == kOzakiExpNonfinite || e2 == kOzakiExpNonfinite;
                const double nan = __longlong_as_double(0x7ff8000000000000LL);
                const double re = bad ? nan : oz_rebuild(planes, off, pstride, s, neg, e1 + e2);
                if constexpr (CPLX) {
                    const double im = bad ? nan : oz_rebuild(planes, off + imoff, pstride, s, neg, e1 + e2);
                    turned[li][lj] = cd{re, -im};
                } else {
                    turned[li][lj] = re;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int j = jb + 8 * w;
            if (i < m && j < n) part += ep(i, j, turned[i - i0][j - j0]);
        }
        if (partial) {
            part = sr_block_sum<256>(part);
            if (threadIdx.x == 0) partial[blockIdx.x + (size_t)gridDim.x * blockIdx.y] = part;
        }
        return;
    }
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const int j = jb + 8 * w;
        if (i < m && j < n) {
            const bool mir = mirror && i > j;
            const size_t off = mir ? (size_t)j + (size_t)i * (size_t)ldp : (size_t)i + (size_t)j * (size_t)ldp;
            const int e1 = ea[i], e2 = fb[j];
            const bool bad = e1 == kOzakiExpNonfinite || e2 == kOzakiExpNonfinite;
            const double nan = __longlong_as_double(0x7ff8000000000000LL);
            const double re = bad ? nan : oz_rebuild(planes, off, pstride, s, neg, e1 + e2);
            if constexpr (CPLX) {
                double im = bad ? nan : oz_rebuild(planes, off + imoff, pstride, s, neg, e1 + e2);
                if (mir) im = -im;
                part += ep(i, j, cd{re, im});
            } else {
                part += ep(i, j, re);
            }
        }
    }
    if (partial) {
        part = sr_block_sum<256>(part);
        if (threadIdx.x == 0) partial[blockIdx.x + (size_t)gridDim.x * blockIdx.y] = part;
    }
}

inline int ozaki_blocks(int m, int n) { return ((m + 31) / 32) * ((n + 31) / 32); }


// the leading 53 bits of M > 0 as m * 2^sh (m in [2^52, 2^53); sh may be
// negative) and the remainder M - m 2^sh (zero when sh <= 0)
__device__ __forceinline__ unsigned long long oz_top53(unsigned __int128 M, int &sh, unsigned __int128 &rem)
{
    const unsigned long long hw = (unsigned long long)(M >> 64), lw = (unsigned long long)M;
    const int msb = hw ? 127 - __clzll((long long)hw) : 63 - __clzll((long long)lw);
    sh = msb - 52;
    if (sh <= 0) {
        rem = 0;
        return lw << (-sh);
    }
    const unsigned long long m = (unsigned long long)(M >> sh);
    rem = M - ((unsigned __int128)m << sh);
    return m;
}

// V * 2^x as a double-double: the leading 53 bits of |V| (truncated) and the
// leading 53 bits of the remainder, one renormalisation. Relative error below
// 2^-105; integer work apart from the final fast TwoSum.
__device__ __forceinline__ ddv oz_i128_to_dd(__int128 V, int x)
{
    if (V == 0) return {0.0, 0.0};
    const bool neg = V < 0;
    const unsigned __int128 M = neg ? (unsigned __int128)(-V) : (unsigned __int128)V;
    int sh, sh2;
    unsigned __int128 rem, rem2;
    const unsigned long long m = oz_top53(M, sh, rem);
    const double hi = oz_make_double(m, sh + x, neg);
    if (rem == 0) return {hi, 0.0};
    const unsigned long long m2 = oz_top53(rem, sh2, rem2);
    return dd_renorm(hi, oz_make_double(m2, sh2 + x, neg));
}

// One rebuilt entry in double-double: sign * 2^e * sum_l I_l 2^(-14-8l). The
// levels are summed exactly in a 128-bit integer with the last level rounded
// to whole units of the level before it, V = sum_{l <= s-2} I_l 256^(s-2-l) +
// round(I_{s-1} / 256), so that |V| < 2^123 for level sums below 2^31 and
// 14 levels; the entry is V 2^(e - 14 - 8(s-2)).
__device__ __forceinline__ ddv oz_rebuild_dd(const int32_t *__restrict__ planes, size_t off, size_t pstride, int s,
                                             double sign, int e)
{
    __int128 V = 0;
    int x;
    if (s == 1) {
        V = planes[off];
        x = e - 14;
    } else {
        for (int l = 0; l <= s - 2; ++l) V = V * 256 + (__int128)planes[off + (size_t)l * pstride];
        const int last = planes[off + (size_t)(s - 1) * pstride];
        V += (__int128)((last + 128) >> 8);
        x = e - 14 - 8 * (s - 2);
    }
    if (sign < 0) V = -V;
    return oz_i128_to_dd(V, x);
}

template <class EP>
__global__ void __launch_bounds__(256)
ozaki_combine_dd_kernel(int m, int n, int s, const int32_t *__restrict__ planes, int ldp, size_t pstride,
                        const int *__restrict__ ea, const int *__restrict__ fb, double sign, int mirror, EP ep,
                        double *partial)
{
    const int i = blockIdx.x * 32 + (threadIdx.x & 31);
    const int jb = blockIdx.y * 32 + (threadIdx.x >> 5);
    double part = 0.0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const int j = jb + 8 * w;
        if (i < m && j < n) {
            const bool mir = mirror && i > j;
            const size_t off = mir ? (size_t)j + (size_t)i * (size_t)ldp : (size_t)i + (size_t)j * (size_t)ldp;
            const int e1 = ea[i], e2 = fb[j];
            const double nan = __longlong_as_double(0x7ff8000000000000LL);
            const bool bad = e1 == kOzakiExpNonfinite || e2 == kOzakiExpNonfinite;
            const ddv v = bad ? ddv{nan, nan} : oz_rebuild_dd(planes, off, pstride, s, sign, e1 + e2);
            part += ep(i, j, v);
        }
    }
    if (partial) {
        part = sr_block_sum<256>(part);
        if (threadIdx.x == 0) partial[blockIdx.x + (size_t)gridDim.x * blockIdx.y] = part;
    }
}

// ---- residue form: rebuild by the Chinese remainder theorem -------------------------
// The table's part the rebuild needs, staged in shared memory by every block.
struct __align__(16) CrtRebuildSm {
    unsigned w[kCrtMaxModuli][kCrtMaxLimbs];
    unsigned M[kCrtMaxLimbs], halfM[kCrtMaxLimbs];
    float invMtop;
    int N, sigma;
};

__device__ __forceinline__ void crt_stage(CrtRebuildSm &sm, const CrtTable *__restrict__ tab, int L)
{
    for (int x = threadIdx.x; x < tab->N * L; x += blockDim.x) sm.w[x / L][x % L] = tab->w[x / L][x % L];
    if (threadIdx.x < L) {
        sm.M[threadIdx.x] = tab->M[threadIdx.x];
        sm.halfM[threadIdx.x] = tab->halfM[threadIdx.x];
    }
    if (threadIdx.x == 0) {
        sm.invMtop = tab->invMtop;
        sm.N = tab->N;
        sm.sigma = tab->sigma;
    }
}

// S' = sum_l R_l w'_l is given as per-limb column sums acc[k] (no carries yet;
// each below 2^45). Returns the sign of r = S' mod M' taken in (-M'/2, M'/2]
// and writes |r| to mag (r = C 2^sigma for the rebuilt integer C). The value
// is carried as 64-bit limbs with 128-bit temporaries for the carries.
template <int L>
__device__ __forceinline__ bool crt_reduce(const unsigned long long (&acc)[L], const CrtRebuildSm &T,
                                           uint32_t (&mag)[L])
{
    constexpr int H = L / 2;
    using u128 = unsigned __int128;
    unsigned long long S[H];
    unsigned long long c = 0;
    uint32_t lo32 = 0;
#pragma unroll
    for (int k = 0; k < L; ++k) {
        const unsigned long long v = acc[k] + c;
        c = v >> 32;
        if (k & 1) S[k >> 1] = ((unsigned long long)(uint32_t)v << 32) | lo32; else lo32 = (uint32_t)v;
    }
    uint32_t top = (uint32_t)c;                       // S' = top 2^(32 L) + S
    const unsigned long long *Mw = reinterpret_cast<const unsigned long long *>(T.M);
    const unsigned long long *Hw = reinterpret_cast<const unsigned long long *>(T.halfM);
    // q = floor(S'/M') < 2^13 from the top 64 bits (M' has its top bit at 32 L - 1),
    // lowered by one: the estimate is within 0.01 of S'/M', so 0 <= S' - q M' < 3 M'
    const float est = ((float)top * 4294967296.0f + (float)(uint32_t)(S[H - 1] >> 32)) * T.invMtop;
    const int qi = (int)est - 1;
    const unsigned long long q = (unsigned long long)(qi < 0 ? 0 : qi);
    unsigned long long cm = 0, br = 0;
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const u128 p = (u128)q * Mw[h] + cm;
        cm = (unsigned long long)(p >> 64);
        const u128 d = (u128)S[h] - (unsigned long long)p - br;
        S[h] = (unsigned long long)d;
        br = (unsigned long long)(d >> 64) & 1ull;
    }
    top = top - (uint32_t)cm - (uint32_t)br;
    // at most two subtractions of M' bring S' into [0, M')
#pragma unroll
    for (int rep = 0; rep < 2; ++rep) {
        unsigned long long d[H];
        unsigned long long b = 0;
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const u128 x = (u128)S[h] - Mw[h] - b;
            d[h] = (unsigned long long)x;
            b = (unsigned long long)(x >> 64) & 1ull;
        }
        if ((int)top - (int)b >= 0) {
            top -= (uint32_t)b;
#pragma unroll
            for (int h = 0; h < H; ++h) S[h] = d[h];
        }
    }
    // symmetric range: r > M'/2 stands for r - M'
    bool gt = false, decided = false;
#pragma unroll
    for (int h = H - 1; h >= 0; --h)
        if (!decided && S[h] != Hw[h]) {
            gt = S[h] > Hw[h];
            decided = true;
        }
    if (gt) {
        unsigned long long b = 0;
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const u128 x = (u128)Mw[h] - S[h] - b;
            S[h] = (unsigned long long)x;
            b = (unsigned long long)(x >> 64) & 1ull;
        }
    }
#pragma unroll
    for (int h = 0; h < H; ++h) {
        mag[2 * h] = (uint32_t)S[h];
        mag[2 * h + 1] = (uint32_t)(S[h] >> 32);
    }
    return gt;
}

// (-1)^neg |r| 2^x as a double, rounded once (|r| < 2^127 for L = 4)
__device__ __forceinline__ double crt_to_double(const uint32_t (&mag)[4], bool neg, int x)
{
    const unsigned __int128 V = ((unsigned __int128)mag[3] << 96) | ((unsigned __int128)mag[2] << 64) |
                                ((unsigned __int128)mag[1] << 32) | (unsigned __int128)mag[0];
    return oz_i128_to_double(neg ? -(__int128)V : (__int128)V, x);
}

// the same as a double-double (L = 8): the 127 leading bits of |r| are taken
// (the bits below them are beyond the double-double's 106) and converted as in
// oz_i128_to_dd
__device__ __forceinline__ ddv crt_to_dd(const uint32_t (&mag)[8], bool neg, int x)
{
    int k = 3;
#pragma unroll
    for (int a = 7; a >= 4; --a)
        if (k == 3 && mag[a] != 0) k = a;
    uint32_t w3 = 0, w2 = 0, w1 = 0, w0 = 0, wm = 0;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        if (a == k) w3 = mag[a];
        if (a == k - 1) w2 = mag[a];
        if (a == k - 2) w1 = mag[a];
        if (a == k - 3) w0 = mag[a];
        if (a == k - 4) wm = mag[a];
    }
    unsigned __int128 W = ((unsigned __int128)w3 << 96) | ((unsigned __int128)w2 << 64) |
                          ((unsigned __int128)w1 << 32) | (unsigned __int128)w0;
    int xe = x + 32 * (k - 3);
    if (w3 != 0) {
        const int lz = __clz((int)w3) - 1;   // leading bit to position 126
        if (lz > 0) {
            W = (W << lz) | (unsigned __int128)(wm >> (32 - lz));
            xe -= lz;
        } else if (lz < 0) {
            W >>= 1;
            xe += 1;
        }
    }
    return oz_i128_to_dd(neg ? -(__int128)W : (__int128)W, xe);
}

// One rebuilt plane entry at off: sign * C 2^(e1 + e2 - tsum), C from its residues
template <int L>
__device__ __forceinline__ std::conditional_t<L == 8, ddv, double>
crt_value(const uint8_t *__restrict__ planes, size_t off, size_t pstride, const CrtRebuildSm &T, int e1, int e2,
          int tsum, bool negs)
{
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    if (e1 == kOzakiExpNonfinite || e2 == kOzakiExpNonfinite) {
        if constexpr (L == 8) return ddv{nan, nan}; else return nan;
    }
    unsigned long long acc[L];
#pragma unroll
    for (int k = 0; k < L; ++k) acc[k] = 0ull;
    for (int l = 0; l < T.N; ++l) {
        const uint32_t R = planes[off + (size_t)l * pstride];
#pragma unroll
        for (int k = 0; k < L; ++k) acc[k] += (unsigned long long)R * T.w[l][k];
    }
    uint32_t mag[L];
    const bool ng = crt_reduce<L>(acc, T, mag) != negs;
    if constexpr (L == 8) return crt_to_dd(mag, ng, e1 + e2 - tsum - T.sigma);
    else return crt_to_double(mag, ng, e1 + e2 - tsum - T.sigma);
}

// ---- the column sums of a rebuild on the tensor cores ---------------------------
// acc[k] = sum_l R_l w_l[k] (R_l the residue bytes of one entry, w_l[k] the
// L 32-bit limbs of the rebuild weights) is, byte by byte, a product of the
// entries' residues (an entries x moduli matrix) with the weights' bytes (a
// moduli x 4 L matrix): every factor is an integer below 256, exact in bf16,
// and every column sum is below 64 * 255^2 < 2^22 for up to 64 moduli, exact
// in the FP32 accumulation of mma.sync. A warp forms the sums of 32
// consecutive plane rows as two m16n8k16 groups over NM / 16 steps of K and
// L / 2 tiles of 8 byte positions. The C fragment of tile j holds byte
// positions 8 j + 2 tig (+ 1) of rows g and g + 8 (g = lane / 4, tig =
// lane % 4): byte position p is byte p % 4 of limb p / 4, so a lane and
// lane ^ 1 hold the two halves of limb 2 j + tig / 2, and lane ^ 2 the limb of
// the other parity. After the exchanges, lane (g, tig) holds the L sums of row
// crt_tc_entry(lane).
__device__ __forceinline__ void sr_mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// the bf16 bits of an integer below 256 (exact: at most 8 significant bits)
__device__ __forceinline__ uint32_t bf16_of_byte(uint32_t x) { return __float_as_uint((float)x) >> 16; }
__device__ __forceinline__ uint32_t bf16_pair(uint32_t lo, uint32_t hi)
{
    return bf16_of_byte(lo) | (bf16_of_byte(hi) << 16);
}
__device__ __forceinline__ int crt_tc_entry(int lane)
{
    const int tig = lane & 3;
    return 16 * (tig & 1) + (lane >> 2) + 8 * (tig >> 1);
}
// B fragments: the weight bytes, rows k = 16 s + 2 tig (+1, +8, +9), column 8 j + g
template <int NM, int L = 12>
__device__ __forceinline__ void crt_weight_frags(const CrtRebuildSm &T, int lane,
                                                 uint32_t (&bw)[NM / 16][L / 2][2])
{
    const int g = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int s = 0; s < NM / 16; ++s)
#pragma unroll
        for (int j = 0; j < L / 2; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = 16 * s + 2 * tig + 8 * h, pos = 8 * j + g;
                const uint32_t b0 = (T.w[k][pos >> 2] >> (8 * (pos & 3))) & 255u;
                const uint32_t b1 = (T.w[k + 1][pos >> 2] >> (8 * (pos & 3))) & 255u;
                bw[s][j][h] = bf16_pair(b0, b1);
            }
}
template <int NM, int L = 12>
__device__ __forceinline__ void crt_sums_tc(const uint8_t *__restrict__ planes, size_t off, size_t pstride,
                                            const uint32_t (&bw)[NM / 16][L / 2][2], int lane, u64 (&acc)[L])
{
    constexpr int NJ = L / 2;   // tiles of 8 byte positions (2 limbs each)
    const int g = lane >> 2, tig = lane & 3;
    float c[2][NJ][4];
#pragma unroll
    for (int G = 0; G < 2; ++G)
#pragma unroll
        for (int j = 0; j < NJ; ++j)
#pragma unroll
            for (int x = 0; x < 4; ++x) c[G][j][x] = 0.f;
#pragma unroll
    for (int s = 0; s < NM / 16; ++s) {
        const size_t k0 = (size_t)(16 * s + 2 * tig);
#pragma unroll
        for (int G = 0; G < 2; ++G) {
            const uint8_t *p = planes + off + (size_t)(16 * G + g);   // row 16 G + g, modulus 0
            uint32_t a[4];
            a[0] = bf16_pair(p[k0 * pstride], p[(k0 + 1) * pstride]);
            a[1] = bf16_pair(p[8 + k0 * pstride], p[8 + (k0 + 1) * pstride]);
            a[2] = bf16_pair(p[(k0 + 8) * pstride], p[(k0 + 9) * pstride]);
            a[3] = bf16_pair(p[8 + (k0 + 8) * pstride], p[8 + (k0 + 9) * pstride]);
#pragma unroll
            for (int j = 0; j < NJ; ++j) sr_mma_bf16(c[G][j], a, bw[s][j][0], bw[s][j][1]);
        }
    }
    const bool bh = (tig & 1) != 0;   // this lane holds bytes 2, 3 (else 0, 1) of its limbs
    const bool gm = bh, hm = (tig >> 1) != 0, odd = hm;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        u64 v[2][2];   // [group][row half]: limb 2 j + tig / 2
#pragma unroll
        for (int G = 0; G < 2; ++G)
#pragma unroll
            for (int hr = 0; hr < 2; ++hr) {
                // two byte positions in 32 bits (below 2^22 + 2^30), the partner's two above them
                const uint32_t own = __float2uint_rn(c[G][j][2 * hr]) + (__float2uint_rn(c[G][j][2 * hr + 1]) << 8);
                const uint32_t oth = __shfl_xor_sync(0xffffffffu, own, 1);
                const uint32_t lo = bh ? oth : own, hi = bh ? own : oth;
                v[G][hr] = (u64)lo + ((u64)hi << 16);
            }
        // this lane's row (gm, hm): its limb of this parity is v[gm][hm]; lane ^ 2
        // holds the other parity and sends it for row (gm, hm), as this lane sends
        // v[gm][!hm] for the row of lane ^ 2
        const u64 mine = gm ? (hm ? v[1][1] : v[1][0]) : (hm ? v[0][1] : v[0][0]);
        const u64 send = gm ? (hm ? v[1][0] : v[1][1]) : (hm ? v[0][0] : v[0][1]);
        const u64 got = __shfl_xor_sync(0xffffffffu, send, 2);
        acc[2 * j] = odd ? got : mine;
        acc[2 * j + 1] = odd ? mine : got;
    }
}

template <bool CPLX, int L>
using CrtCombineValue = std::conditional_t<CPLX, cd, std::conditional_t<L == 8, ddv, double>>;

// C(i, j) = sign * (rebuilt product) with the epilogue ep, FP64 results
// (L = 4) or double-double results (L = 8): the 32 x 32 output block (bx, by)
// of one product (planes: its region's origin); returns the thread's sum of
// the epilogue's values. T is staged and turned is the block's shared turning
// buffer. Real products: each warp rebuilds 32 consecutive plane rows of four
// columns with the column sums on the tensor cores; a block wholly below the
// diagonal of a mirrored product rebuilds the block above it and turns it in
// shared memory, and entries below the diagonal of a diagonal block are read
// in place (the product tile holding a diagonal 32 x 32 block is always
// formed). Complex products: each thread takes 4 consecutive rows of one
// column (one 32-bit load per residue plane) with scalar sums; entries below
// the diagonal of a diagonal block read the mirrored position.
template <class EP, bool CPLX, int L, int NM>
__device__ __forceinline__ double crt_combine_block(int bx, int by, int m, int n, const uint8_t *__restrict__ planes,
                                                    int ldp, size_t pstride, size_t imoff, const int *__restrict__ ea,
                                                    const int *__restrict__ fb, int tsum, double sign, int mirror,
                                                    const EP &ep, const CrtRebuildSm &T,
                                                    CrtCombineValue<CPLX, L> (&turned)[32][33])
{
    static_assert(!(CPLX && L == 8), "complex products rebuild FP64 parts");
    using RV = std::conditional_t<L == 8, ddv, double>;
    using VT = CrtCombineValue<CPLX, L>;
    if constexpr (!CPLX && NM > 0 && NM % 16 == 0) {
        // real products: the column sums on the tensor cores, a warp per 32 plane
        // rows of a column (as ozaki_crt_combine_td_kernel; the rebuilt values are
        // those of the scalar sums bit for bit)
        const bool negs = sign < 0;
        const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5, a = crt_tc_entry(lane);
        uint32_t bw[NM / 16][L / 2][2];
        crt_weight_frags<NM, L>(T, lane, bw);
        const bool below = mirror && bx > by;
        const int rb = (below ? by : bx) * 32, cb = (below ? bx : by) * 32;
        const int rlim = below ? n : m, clim = below ? m : n;
        const int r = rb + a;
        const int e1 = r < rlim ? ea[r] : 0;
        const double nan = __longlong_as_double(0x7ff8000000000000LL);
        double part = 0.0;
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
            const int c = cb + wv + 8 * q;
            if (c >= clim) break;   // uniform over the warp
            const int e2 = fb[c];
            u64 acc[L];
            crt_sums_tc<NM, L>(planes, (size_t)rb + (size_t)c * ldp, pstride, bw, lane, acc);
            uint32_t mag[L];
            const bool ng = crt_reduce<L>(acc, T, mag) != negs;
            RV v;
            if constexpr (L == 8) v = crt_to_dd(mag, ng, e1 + e2 - tsum - T.sigma);
            else v = crt_to_double(mag, ng, e1 + e2 - tsum - T.sigma);
            if (e1 == kOzakiExpNonfinite || e2 == kOzakiExpNonfinite) {
                if constexpr (L == 8) v = ddv{nan, nan}; else v = nan;
            }
            if (r < rlim) {
                if (below) turned[wv + 8 * q][a] = v;
                else part += ep(r, c, v);
            }
        }
        if (below) {
            __syncthreads();
            const int i0 = bx * 32, j0 = by * 32, al = threadIdx.x & 31;
#pragma unroll 1
            for (int q = 0; q < 4; ++q) {
                const int i = i0 + al, j = j0 + wv + 8 * q;
                if (i < m && j < n) part += ep(i, j, turned[al][wv + 8 * q]);
            }
        }
        return part;
    } else {
    const int N = T.N;
    const bool negs = sign < 0;
    const int ig = threadIdx.x & 7, jl = threadIdx.x >> 3;
    const bool below = mirror && bx > by;
    // rebuilt entries (ra + 4 ig + u, ca + jl) of the planes, u = 0..3
    const int ra = (below ? by : bx) * 32 + 4 * ig;
    const int ca = (below ? bx : by) * 32 + jl;
    const int rlim = below ? n : m, clim = below ? m : n;
    VT val[4];
    auto rebuild = [&](size_t base, int e2, RV (&out)[4]) {
        unsigned long long acc[4][L];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < L; ++k) acc[u][k] = 0ull;
        if constexpr (NM > 0) {
            // the modulus count is fixed: every plane's word is loaded before the sums
            uint32_t r4[NM];
#pragma unroll
            for (int l = 0; l < NM; ++l) r4[l] = *reinterpret_cast<const uint32_t *>(planes + base + (size_t)l * pstride);
#pragma unroll
            for (int l = 0; l < NM; ++l) {
                uint32_t wl[L];
#pragma unroll
                for (int k = 0; k < L; k += 4) {
                    const uint4 w4 = *reinterpret_cast<const uint4 *>(&T.w[l][k]);
                    wl[k] = w4.x; wl[k + 1] = w4.y; wl[k + 2] = w4.z; wl[k + 3] = w4.w;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t R = (r4[l] >> (8 * u)) & 255u;
#pragma unroll
                    for (int k = 0; k < L; ++k) acc[u][k] += (unsigned long long)R * wl[k];
                }
            }
        } else {
            for (int l = 0; l < N; ++l) {
                const uint32_t r4 = *reinterpret_cast<const uint32_t *>(planes + base + (size_t)l * pstride);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t R = (r4 >> (8 * u)) & 255u;
#pragma unroll
                    for (int k = 0; k < L; ++k) acc[u][k] += (unsigned long long)R * T.w[l][k];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            uint32_t mag[L];
            const bool ng = crt_reduce<L>(acc[u], T, mag) != negs;
            const int e1 = ea[min(ra + u, rlim - 1)];
            const int x = e1 + e2 - tsum - T.sigma;
            const bool bad = e1 == kOzakiExpNonfinite || e2 == kOzakiExpNonfinite;
            const double nan = __longlong_as_double(0x7ff8000000000000LL);
            if constexpr (L == 8) {
                out[u] = bad ? ddv{nan, nan} : crt_to_dd(mag, ng, x);
            } else {
                out[u] = bad ? nan : crt_to_double(mag, ng, x);
            }
        }
    };
    const bool active = ra < rlim && ca < clim;
    if (active) {
        const size_t base = (size_t)ra + (size_t)ca * (size_t)ldp;
        const int e2 = fb[ca];
        RV re[4];
        rebuild(base, e2, re);
        if constexpr (CPLX) {
            RV im[4];
            rebuild(base + imoff, e2, im);
#pragma unroll
            for (int u = 0; u < 4; ++u) val[u] = cd{re[u], below ? -im[u] : im[u]};
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) val[u] = re[u];
        }
    }
    double part = 0.0;
    if (below) {
        // turn the mirrored block: entry (ca, ra + u) of the output
        if (active)
#pragma unroll
            for (int u = 0; u < 4; ++u) turned[jl][4 * ig + u] = val[u];
        __syncthreads();
        const int i0 = bx * 32, j0 = by * 32;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + 4 * ig + u, j = j0 + jl;
            if (i < m && j < n) part += ep(i, j, turned[4 * ig + u][jl]);
        }
    } else if (active) {
        const int j = ca;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = ra + u;
            if (i >= m) break;
            VT v = val[u];
            if (mirror && i > j) {
                // below the diagonal inside a diagonal block: the mirrored entry
                // (conjugated when complex: the product is Hermitian)
                const size_t off = (size_t)j + (size_t)i * (size_t)ldp;
                if constexpr (CPLX) {
                    v = cd{crt_value<L>(planes, off, pstride, T, ea[j], fb[i], tsum, negs),
                           -crt_value<L>(planes, off + imoff, pstride, T, ea[j], fb[i], tsum, negs)};
                } else {
                    v = crt_value<L>(planes, off, pstride, T, ea[j], fb[i], tsum, negs);
                }
            }
            part += ep(i, j, v);
        }
    }
    return part;
    }
}

template <class EP, bool CPLX, int L, int NM>
__global__ void __launch_bounds__(256)
ozaki_crt_combine_kernel(int m, int n, const uint8_t *__restrict__ planes, int ldp, size_t pstride, size_t imoff,
                         const int *__restrict__ ea, const int *__restrict__ fb, int tsum, double sign, int mirror,
                         EP ep, double *partial, const CrtTable *__restrict__ tab)
{
    __shared__ CrtRebuildSm T;
    __shared__ CrtCombineValue<CPLX, L> turned[32][33];
    crt_stage(T, tab, L);
    __syncthreads();
    double part = crt_combine_block<EP, CPLX, L, NM>(blockIdx.x, blockIdx.y, m, n, planes, ldp, pstride, imoff, ea,
                                                     fb, tsum, sign, mirror, ep, T, turned);
    if (partial) {
        part = sr_block_sum<256>(part);
        if (threadIdx.x == 0) partial[blockIdx.x + (size_t)gridDim.x * blockIdx.y] = part;
    }
}

// Grouped residue-form combine (FP64 results, NM moduli): one flat grid of
// 32 x 32 output blocks over all matrices as ozaki_combine_group_kernel, each
// matrix's planes a byte region at its poff (leading dimension ldp, a
// multiple of 32) and its own tsum.
template <class EP, int NM>
__global__ void __launch_bounds__(256)
ozaki_crt_combine_group_kernel(const uint8_t *__restrict__ planes, size_t pstride, const CombMat *__restrict__ mats,
                               const EP *__restrict__ eps, const int *__restrict__ start, int cnt,
                               const int *__restrict__ ea, const int *__restrict__ fb, double sign, int mirror,
                               double *partial, const CrtTable *__restrict__ tab)
{
    __shared__ CrtRebuildSm T;
    __shared__ CrtCombineValue<false, 4> turned[32][33];
    crt_stage(T, tab, 4);
    __syncthreads();
    const int a = group_find(start, cnt, blockIdx.x);
    const CombMat cm = mats[a];
    const int local = blockIdx.x - start[a], gx = (cm.m + 31) / 32;
    double part = crt_combine_block<EP, false, 4, NM>(local % gx, local / gx, cm.m, cm.n, planes + cm.poff, cm.ldp,
                                                      pstride, 0, ea + cm.ra, fb + cm.rb, cm.tsum, sign, mirror,
                                                      eps[a], T, turned);
    if (partial) {
        part = sr_block_sum<256>(part);
        if (threadIdx.x == 0) partial[blockIdx.x] = part;
    }
}


// Triple-double results (L = 12 limbs, the 48 moduli of the triple-double
// operands): the twelve column sums of an entry come from the warp's
// tensor-core product (crt_sums_tc); a block covers 32 x 32 entries. The
// rebuilt integer is rounded to a triple-double from its 256 leading bits (the
// bits below them lie far beyond the 159 kept).
__device__ __forceinline__ tdv crt_to_td(const uint32_t (&mag)[12], bool neg, int x)
{
    int k = 7;   // leading limb of the 256-bit window (limbs k-7 .. k)
#pragma unroll
    for (int a = 11; a >= 8; --a)
        if (k == 7 && mag[a] != 0) k = a;
    u64 W[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t lo = 0, hi = 0;
#pragma unroll
        for (int a = 0; a < 12; ++a) {
            if (a == k - 7 + 2 * q) lo = mag[a];
            if (a == k - 6 + 2 * q) hi = mag[a];
        }
        W[q] = ((u64)hi << 32) | lo;
    }
    return td_round_u256(W, neg, x + 32 * (k - 7));
}

// this lane's entry of the warp's 32 plane rows at off (every lane of the warp
// calls it together)
template <int NM>
__device__ __forceinline__ tdv crt_value_td_tc(const uint8_t *__restrict__ planes, size_t off, size_t pstride,
                                               const CrtRebuildSm &T, const uint32_t (&bw)[NM / 16][6][2],
                                               int lane, int e1, int e2, int tsum, bool negs)
{
    constexpr int L = 12;
    u64 acc[L];
    crt_sums_tc<NM>(planes, off, pstride, bw, lane, acc);
    uint32_t mag[L];
    const bool ng = crt_reduce<L>(acc, T, mag) != negs;
    const tdv v = crt_to_td(mag, ng, e1 + e2 - tsum - T.sigma);
    if (e1 == kOzakiExpNonfinite || e2 == kOzakiExpNonfinite) {
        const double nan = __longlong_as_double(0x7ff8000000000000LL);
        return {nan, nan, nan};
    }
    return v;
}

// Warp w rebuilds, for q = 0..3, 32 consecutive plane rows of column w + 8 q
// of its block (lane: row crt_tc_entry(lane)); every branch around the warp's
// tensor-core product is uniform over the warp. A mirrored block below the
// diagonal rebuilds the block above it and turns it in shared memory; entries
// below the diagonal of a diagonal block are read where they are: the product
// tile holding a diagonal 32 x 32 block is always formed.
template <class EP, int NM>
__global__ void __launch_bounds__(256)
ozaki_crt_combine_td_kernel(int m, int n, const uint8_t *__restrict__ planes, int ldp, size_t pstride,
                            const int *__restrict__ ea, const int *__restrict__ fb, int tsum, double sign, int mirror,
                            EP ep, double *partial, const CrtTable *__restrict__ tab)
{
    static_assert(NM % 16 == 0, "moduli in steps of 16");
    __shared__ CrtRebuildSm T;
    __shared__ tdv turned[32][33];
    crt_stage(T, tab, 12);
    __syncthreads();
    const bool negs = sign < 0;
    const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5, a = crt_tc_entry(lane);
    uint32_t bw[NM / 16][6][2];
    crt_weight_frags<NM>(T, lane, bw);
    const bool below = mirror && blockIdx.x > blockIdx.y;
    const int rb = (below ? blockIdx.y : blockIdx.x) * 32, cb = (below ? blockIdx.x : blockIdx.y) * 32;
    const int rlim = below ? n : m, clim = below ? m : n;
    const int r = rb + a;
    const int e1 = r < rlim ? ea[r] : 0;
    double part = 0.0;
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
        const int c = cb + wv + 8 * q;
        if (c >= clim) break;   // uniform over the warp
        const tdv v = crt_value_td_tc<NM>(planes, (size_t)rb + (size_t)c * ldp, pstride, T, bw, lane, e1, fb[c],
                                          tsum, negs);
        if (r < rlim) {
            if (below) turned[wv + 8 * q][a] = v;
            else part += ep(r, c, v);
        }
    }
    if (below) {
        __syncthreads();
        const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32, al = threadIdx.x & 31;
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + al, j = j0 + wv + 8 * q;
            if (i < m && j < n) part += ep(i, j, turned[al][wv + 8 * q]);
        }
    }
    if (partial) {
        part = sr_block_sum<256>(part);
        if (threadIdx.x == 0) partial[blockIdx.x + (size_t)gridDim.x * blockIdx.y] = part;
    }
}

// v = the 6 words mw shifted up by Q words and rr < 64 bits, in 12 words
template <int Q>
__device__ __forceinline__ void d6_place(const u64 (&mw)[6], int rr, u64 (&v)[12])
{
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const u64 lo = (k - Q >= 0 && k - Q < 6) ? mw[k - Q >= 0 && k - Q < 6 ? k - Q : 0] : 0ull;
        const u64 hi = (k - Q - 1 >= 0 && k - Q - 1 < 6) ? mw[k - Q - 1 >= 0 && k - Q - 1 < 6 ? k - Q - 1 : 0] : 0ull;
        v[k] = rr ? (lo << rr) | (hi >> (64 - rr)) : lo;
    }
}

// Six-double results: the product of operands held as two residue halves,
// X = X_hi 2^t + X_lo for each vector, is HH 2^(2t) + (HL + LH) 2^t + LL. The
// four integer products are the four plane sets (48 byte planes each) of one
// entry; each is rebuilt into 12 limbs (column sums on the tensor cores, by a
// whole warp for its 32 rows), the four are summed exactly in a 768-bit two's
// complement integer, and its 512 leading bits are rounded once to six words.
// No mirrored form: the Gram products are formed whole.
template <int NM>
__device__ __forceinline__ d6v crt_value_d6_tc(const uint8_t *__restrict__ planes, size_t off, size_t pstride,
                                               size_t setstride, const CrtRebuildSm &T,
                                               const uint32_t (&bw)[NM / 16][6][2], int lane, int e1, int e2,
                                               int t, bool negs)
{
    constexpr int L = 12, NS = 12;   // limbs of one rebuild; 64-bit words of the sum
    d6v r;
    u64 S[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) S[k] = 0;
#pragma unroll 1
    for (int set = 0; set < 4; ++set) {
        u64 acc[L];
        crt_sums_tc<NM>(planes + (size_t)set * setstride, off, pstride, bw, lane, acc);
        uint32_t mag[L];
        const bool ng = crt_reduce<L>(acc, T, mag) != negs;
        // mag (6 words) shifted by 2t (HH), t (HL, LH) or 0 (LL) into the sum; for
        // t in [160, 174] these are 5, 2 and 0 whole words and a bit shift rr
        u64 mw[L / 2];
#pragma unroll
        for (int j = 0; j < L / 2; ++j) mw[j] = ((u64)mag[2 * j + 1] << 32) | mag[2 * j];
        u64 v[NS];
        if (set == 0) d6_place<5>(mw, (2 * t) & 63, v);
        else if (set == 3) d6_place<0>(mw, 0, v);
        else d6_place<2>(mw, t & 63, v);
        if (ng) mw_neg<NS>(v);
        mw_add<NS>(S, v);
    }
    const bool neg = (S[NS - 1] >> 63) != 0;
    if (neg) mw_neg<NS>(S);
    int top = 7;   // the 512-bit window: words top - 7 .. top
#pragma unroll
    for (int k = NS - 1; k >= 8; --k)
        if (top == 7 && S[k] != 0) top = k;
    u64 W[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) W[j] = mw_word<NS>(S, top - 7 + j);
    const int T2 = 2 * (2 * t - 2);   // the operands hold T = 2t - 2 bits each
    mw_round<kD6Words, 8>(W, neg, e1 + e2 - T2 - T.sigma + 64 * (top - 7), r.x);
    if (e1 == kOzakiExpNonfinite || e2 == kOzakiExpNonfinite) {
        const double nan = __longlong_as_double(0x7ff8000000000000LL);
#pragma unroll
        for (int k = 0; k < kD6Words; ++k) r.x[k] = nan;
    }
    return r;
}

// 32 x 32 entries per block; warp w rebuilds rows blockIdx.x 32 .. + 31 of
// columns w, w + 8, w + 16, w + 24 (lane: row crt_tc_entry(lane)); every
// branch around the warp's tensor-core product is uniform over the warp.
template <class EP, int NM>
__global__ void __launch_bounds__(256)
ozaki_crt_combine_d6_kernel(int m, int n, const uint8_t *__restrict__ planes, int ldp, size_t pstride,
                            size_t setstride, const int *__restrict__ ea, const int *__restrict__ fb, int t,
                            double sign, EP ep, double *partial, const CrtTable *__restrict__ tab)
{
    static_assert(NM % 16 == 0, "moduli in steps of 16");
    __shared__ CrtRebuildSm T;
    crt_stage(T, tab, 12);
    __syncthreads();
    const bool negs = sign < 0;
    const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5;
    uint32_t bw[NM / 16][6][2];
    crt_weight_frags<NM>(T, lane, bw);
    const int i0 = blockIdx.x * 32, i = i0 + crt_tc_entry(lane);
    const int e1 = i < m ? ea[i] : 0;
    double part = 0.0;
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
        const int j = blockIdx.y * 32 + wv + 8 * q;
        if (j >= n) break;   // uniform over the warp
        const d6v v = crt_value_d6_tc<NM>(planes, (size_t)i0 + (size_t)j * ldp, pstride, setstride, T, bw, lane, e1,
                                          fb[j], t, negs);
        if (i < m) part += ep(i, j, v);
    }
    if (partial) {
        part = sr_block_sum<256>(part);
        if (threadIdx.x == 0) partial[blockIdx.x + (size_t)gridDim.x * blockIdx.y] = part;
    }
}

// The six-double product C = sign (rows) (cols) from the four products already
// formed into the plane sets 0..3 of w.planes (HH, HL, LH, LL; rows and cols
// are the high-half slots), with the epilogue ep.
template <class EP>
sr_status ozaki_combine_d6(schur_refine_ctx *h, cudaStream_t st, OzakiWork &w, int rows, int cols, int m, int n,
                           double sign, EP ep, double *partial, int *blocks)
{
    static_assert(ep_is_d6<EP>::value, "six-double epilogue");
    // the rebuild places the partial products 5 and 2 words up: t in [160, 174]
    if (w.cplx || w.crt.L != 12 || w.crt.N != kCrtDefaultModuliTD || !w.slot[rows].crt || !w.slot[cols].crt ||
        w.slot[rows].t != w.slot[cols].t || w.slot[rows].t < 160 || w.slot[rows].t > 174)
        return SR_ERR_INVALID_ARG;
    const int s = w.crt.N;
    const dim3 grid((m + 31) / 32, (n + 31) / 32);
    const size_t pstride = (size_t)w.Pmax * w.Pmax;
    SrPhase ph(h, SR_PROF_OZ_COMBINE, 4LL * 24 * 12 * s * m * n, (long long)m * n * (4LL * s + 48), 1);
    ozaki_crt_combine_d6_kernel<EP, kCrtDefaultModuliTD><<<grid, 256, 0, st>>>(
        m, n, reinterpret_cast<const uint8_t *>(w.planes), w.Pmax, pstride, (size_t)s * pstride, w.slot[rows].exps,
        w.slot[cols].exps, w.slot[rows].t, sign, ep, partial, w.crt_dev);
    SR_CUDA_TRY(cudaGetLastError());
    if (blocks) *blocks = ozaki_blocks(m, n);
    return SR_OK;
}

inline int ozaki_crt_limbs(const OzakiWork &w) { return w.crt.L; }

// epilogues of complex products carry `static constexpr bool kComplex`
template <class EP, class = void> struct ep_is_complex : std::false_type {};
template <class EP> struct ep_is_complex<EP, std::void_t<decltype(EP::kComplex)>> : std::true_type {};

// epilogues that take a double-double value carry `static constexpr bool kDD`
template <class EP, class = void> struct ep_is_dd : std::false_type {};
template <class EP> struct ep_is_dd<EP, std::void_t<decltype(EP::kDD)>> : std::true_type {};

template <class EP>
sr_status ozaki_combine(schur_refine_ctx *h, cudaStream_t st, OzakiWork &w, int rows, int cols, int m, int n, int s,
                        double sign, bool mirror, EP ep, double *partial, int *blocks)
{
    if (w.slot[rows].crt || w.slot[cols].crt) {
        // residue form: rebuild by the Chinese remainder theorem
        if (!(w.slot[rows].crt && w.slot[cols].crt) || s != w.crt.N) return SR_ERR_INVALID_ARG;
        const int tsum = w.slot[rows].t + w.slot[cols].t;
        const dim3 grid((m + 31) / 32, (n + 31) / 32);
        const uint8_t *pl = reinterpret_cast<const uint8_t *>(w.planes);
        if constexpr (ep_is_td<EP>::value) {
            if (w.cplx || w.crt.L != 12 || s != kCrtDefaultModuliTD) return SR_ERR_INVALID_ARG;
            SrPhase ph(h, SR_PROF_OZ_COMBINE, 24LL * 12 * s * m * n, (long long)m * n * (1LL * s + 48), 1);
            ozaki_crt_combine_td_kernel<EP, kCrtDefaultModuliTD><<<grid, 256, 0, st>>>(
                m, n, pl, w.Pmax, (size_t)w.Pmax * w.Pmax, w.slot[rows].exps, w.slot[cols].exps, tsum, sign,
                mirror ? 1 : 0, ep, partial, w.crt_dev);
        } else if constexpr (ep_is_dd<EP>::value) {
            if (w.cplx || w.crt.L != 8) return SR_ERR_INVALID_ARG;
            SrPhase ph(h, SR_PROF_OZ_COMBINE, 16LL * 8 * s * m * n, (long long)m * n * (1LL * s + 32), 1);
            if (s == kCrtDefaultModuliDD)
                ozaki_crt_combine_kernel<EP, false, 8, kCrtDefaultModuliDD><<<grid, 256, 0, st>>>(
                    m, n, pl, w.Pmax, (size_t)w.Pmax * w.Pmax, 0, w.slot[rows].exps, w.slot[cols].exps, tsum, sign,
                    mirror ? 1 : 0, ep, partial, w.crt_dev);
            else
                ozaki_crt_combine_kernel<EP, false, 8, 0><<<grid, 256, 0, st>>>(
                    m, n, pl, w.Pmax, (size_t)w.Pmax * w.Pmax, 0, w.slot[rows].exps, w.slot[cols].exps, tsum, sign,
                    mirror ? 1 : 0, ep, partial, w.crt_dev);
        } else {
            constexpr bool CPLX = ep_is_complex<EP>::value;
            const int c = CPLX ? 2 : 1;
            if (CPLX != w.cplx || w.crt.L != 4) return SR_ERR_INVALID_ARG;
            SrPhase ph(h, SR_PROF_OZ_COMBINE, 8LL * c * s * m * n, (long long)m * n * (1LL * c * s + 16 * c), 1);
            if (s == kCrtDefaultModuli)
                ozaki_crt_combine_kernel<EP, CPLX, 4, kCrtDefaultModuli><<<grid, 256, 0, st>>>(
                    m, n, pl, w.Pmax, (size_t)c * w.Pmax * w.Pmax, (size_t)w.Pmax * w.Pmax, w.slot[rows].exps,
                    w.slot[cols].exps, tsum, sign, mirror ? 1 : 0, ep, partial, w.crt_dev);
            else
                ozaki_crt_combine_kernel<EP, CPLX, 4, 0><<<grid, 256, 0, st>>>(
                    m, n, pl, w.Pmax, (size_t)c * w.Pmax * w.Pmax, (size_t)w.Pmax * w.Pmax, w.slot[rows].exps,
                    w.slot[cols].exps, tsum, sign, mirror ? 1 : 0, ep, partial, w.crt_dev);
        }
        SR_CUDA_TRY(cudaGetLastError());
        if (blocks) *blocks = ozaki_blocks(m, n);
        return SR_OK;
    }
    if constexpr (ep_is_td<EP>::value) {
        return SR_ERR_INVALID_ARG;   // triple-double products exist in the residue form only
    } else if constexpr (ep_is_dd<EP>::value) {
        if (w.cplx || s > w.levels) return SR_ERR_INVALID_ARG;
        SrPhase ph(h, SR_PROF_OZ_COMBINE, 24LL * s * m * n, (long long)m * n * (4LL * s + 32), 1);
        dim3 grid((m + 31) / 32, (n + 31) / 32);
        const size_t pstride = (size_t)w.Pmax * w.Pmax;
        ozaki_combine_dd_kernel<EP><<<grid, 256, 0, st>>>(m, n, s, w.planes, w.Pmax, pstride, w.slot[rows].exps,
                                                          w.slot[cols].exps, sign, mirror ? 1 : 0, ep, partial);
        SR_CUDA_TRY(cudaGetLastError());
        if (blocks) *blocks = ozaki_blocks(m, n);
        return SR_OK;
    } else {
        constexpr bool CPLX = ep_is_complex<EP>::value;
        if (CPLX != w.cplx) return SR_ERR_INVALID_ARG;
        const int c = CPLX ? 2 : 1;
        SrPhase ph(h, SR_PROF_OZ_COMBINE, 8LL * c * s * m * n, (long long)m * n * (4LL * c * s + 16 * c), 1);
        dim3 grid((m + 31) / 32, (n + 31) / 32);
        const size_t pstride = (size_t)c * w.Pmax * w.Pmax, imoff = (size_t)w.Pmax * w.Pmax;
        ozaki_combine_kernel<EP, CPLX><<<grid, 256, 0, st>>>(m, n, s, w.planes, w.Pmax, pstride, imoff,
                                                             w.slot[rows].exps, w.slot[cols].exps, sign, mirror ? 1 : 0,
                                                             ep, partial);
        SR_CUDA_TRY(cudaGetLastError());
        if (blocks) *blocks = ozaki_blocks(m, n);
        return SR_OK;
    }
}

// Grouped combine: one flat grid of 32 x 32 output blocks over all matrices
// (matrix a owns blocks [start[a], start[a + 1]), row-major over its
// ceil(m/32) x ceil(n/32) blocks); eps[a] its epilogue (FP64 results);
// partial[block] receives the block sums when partial is given.
template <class EP>
__global__ void __launch_bounds__(256)
ozaki_combine_group_kernel(int s, const int32_t *__restrict__ planes, size_t pstride, const CombMat *__restrict__ mats,
                           const EP *__restrict__ eps, const int *__restrict__ start, int cnt,
                           const int *__restrict__ ea, const int *__restrict__ fb, double sign, int mirror,
                           double *partial)
{
    const int a = group_find(start, cnt, blockIdx.x);
    const CombMat cm = mats[a];
    const int local = blockIdx.x - start[a], gx = (cm.m + 31) / 32;
    const int bx = local % gx, by = local / gx;
    const int i = bx * 32 + (threadIdx.x & 31);
    const int jb = by * 32 + (threadIdx.x >> 5);
    const EP ep = eps[a];
    const bool neg = sign < 0;
    double part = 0.0;
    if (mirror && bx > by) {
        // wholly below the diagonal: coalesced reads of the mirrored block,
        // turned in shared memory (as in ozaki_combine_kernel)
        __shared__ double turned[32][33];
        const int i0 = bx * 32, j0 = by * 32;
        const int lj = threadIdx.x & 31, wi = threadIdx.x >> 5;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int li = wi + 8 * w, ii = i0 + li, jj = j0 + lj;
            if (ii < cm.m && jj < cm.n) {
                const size_t off = (size_t)cm.poff + (size_t)jj + (size_t)ii * (size_t)cm.ldp;
                const int e1 = ea[cm.ra + ii], e2 = fb[cm.rb + jj];
                const bool bad = e1 == kOzakiExpNonfinite || e2 == kOzakiExpNonfinite;
                const double nan = __longlong_as_double(0x7ff8000000000000LL);
                turned[li][lj] = bad ? nan : oz_rebuild(planes, off, pstride, s, neg, e1 + e2);
            }
        }
        __syncthreads();
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int j = jb + 8 * w;
            if (i < cm.m && j < cm.n) part += ep(i, j, turned[i - i0][j - j0]);
        }
        if (partial) {
            part = sr_block_sum<256>(part);
            if (threadIdx.x == 0) partial[blockIdx.x] = part;
        }
        return;
    }
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const int j = jb + 8 * w;
        if (i < cm.m && j < cm.n) {
            const bool mir = mirror && i > j;
            const size_t off = (size_t)cm.poff + (mir ? (size_t)j + (size_t)i * (size_t)cm.ldp
                                                      : (size_t)i + (size_t)j * (size_t)cm.ldp);
            const int e1 = ea[cm.ra + i], e2 = fb[cm.rb + j];
            const bool bad = e1 == kOzakiExpNonfinite || e2 == kOzakiExpNonfinite;
            const double nan = __longlong_as_double(0x7ff8000000000000LL);
            part += ep(i, j, bad ? nan : oz_rebuild(planes, off, pstride, s, neg, e1 + e2));
        }
    }
    if (partial) {
        part = sr_block_sum<256>(part);
        if (threadIdx.x == 0) partial[blockIdx.x] = part;
    }
}

template <class EP>
sr_status ozaki_combine_group(schur_refine_ctx *h, cudaStream_t st, OzakiWork &w, int rows, int cols,
                              const CombMat *mats, const EP *eps, const int *start, int cnt, int total, int s,
                              double sign, bool mirror, double *partial, long long flops, long long bytes)
{
    if (cnt <= 0 || total <= 0) return SR_OK;
    SrPhase ph(h, SR_PROF_OZ_COMBINE, flops, bytes, 1);
    if (w.slot[rows].crt || w.slot[cols].crt) {
        // residue form: byte planes, 16 moduli (FP64 results)
        if (!w.slot[rows].crt || !w.slot[cols].crt || s != w.crt.N || w.crt.N != kCrtDefaultModuli ||
            w.crt.L != 4)
            return SR_ERR_INVALID_ARG;
        ozaki_crt_combine_group_kernel<EP, kCrtDefaultModuli><<<total, 256, 0, st>>>(
            reinterpret_cast<const uint8_t *>(w.planes), (size_t)w.pstride_group, mats, eps, start, cnt,
            w.slot[rows].exps, w.slot[cols].exps, sign, mirror ? 1 : 0, partial, w.crt_dev);
        SR_CUDA_TRY(cudaGetLastError());
        return SR_OK;
    }
    ozaki_combine_group_kernel<EP><<<total, 256, 0, st>>>(s, w.planes, (size_t)w.pstride_group, mats, eps, start,
                                                          cnt, w.slot[rows].exps, w.slot[cols].exps, sign,
                                                          mirror ? 1 : 0, partial);
    SR_CUDA_TRY(cudaGetLastError());
    return SR_OK;
}

// slots used by the engine
enum {
    OZS_ROWS = 0,   // generic product: op(A) rows; refinement: rows of A (split once per call)
    OZS_COLS = 1,   // generic product: B columns; refinement: columns of Q
    OZS_X = 2,      // columns of A Q, then of Delta
    OZS_QROWS = 3,  // rows of Q (update product)
    OZS_W = 4,      // columns of W (low-precision digits)
    OZS_Y = 5,      // columns of Y (low-precision digits)
    OZS_W2 = 6,     // columns of W^2 (low-precision digits)
    // six-double products: the low halves of the residue operands (the high
    // halves are in OZS_ROWS .. OZS_QROWS)
    OZS_ROWS_LO = 8,
    OZS_COLS_LO = 9,
    OZS_X_LO = 10,
    OZS_QROWS_LO = 11
};

// One emulated product C = op(A) B with the generic slots, epilogue ep
// (op(A) = A^H, the conjugate transpose, when transA and w.cplx).
template <class EP>
sr_status ozaki_gemm(schur_refine_ctx *h, cudaStream_t st, OzakiWork &w, bool transA, int m, int n, int k,
                     const void *A, int lda, const void *B, int ldb, EP ep, double *partial, int *blocks,
                     int slices, int *flags)
{
    const int s = slices > 0 ? slices : kOzakiDefaultSlices;
    if (s > w.slot[OZS_ROWS].cap || m > w.nmax || n > w.nmax || k > w.nmax) return SR_ERR_INVALID_ARG;
    SR_TRY(ozaki_split(h, st, w, OZS_ROWS, m, k, A, lda, transA ? OZ_COLS : OZ_ROWS, s));
    SR_TRY(ozaki_split(h, st, w, OZS_COLS, n, k, B, ldb, OZ_COLS, s));
    SR_TRY(ozaki_product(h, st, w, OZS_ROWS, OZS_COLS, m, n, k, s, false, flags));
    return ozaki_combine(h, st, w, OZS_ROWS, OZS_COLS, m, n, s, 1.0, false, ep, partial, blocks);
}

}  // namespace sr
