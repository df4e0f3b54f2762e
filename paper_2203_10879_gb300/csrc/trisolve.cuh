// Solver of the triangular matrix equation stril(T L - L T) = -E (Sec. 2.1).
//
// Entry (i, j), i > j, of the equation reads (eq. "lij", with the index of the
// first sum taken as t_ik l_kj, the reading consistent with Alg. 2)
//     l_ij (t_ii - t_jj) = -e_ij - sum_{k>i} t_ik l_kj + sum_{k<j} l_ik t_kj,
// so l_ij needs the entries below it in its column and left of it in its row.
// Every entry on subdiagonal d = i - j therefore depends only on subdiagonals
// d' > d, an admissible order in the sense of eq. "ordercondition" (the
// "parallel wavefront" ordering the paper mentions next to Alg. 3).
//
// The matrix is cut into B x B tiles (B = 32). Tile (I, J), I >= J, needs
// C = E_IJ + sum_{K>I} T_IK L_KJ - sum_{K<J} L_IK T_KJ (the block form of
// Alg. 3's two update products) and then solves the tile equation
// T_II X - X T_JJ = -C (eq. "l21", a triangular Sylvester equation) -- or its
// stril form when I = J -- by a wavefront over the tile's own subdiagonals
// a - b = B-1, ..., -(B-1).
//
// Tiles on block subdiagonal D = I - J depend only on tiles with D' > D, and a
// finished subdiagonal d contributes exactly two products to each tile with
// D < d: T(I, J+d) L(J+d, J) and -L(I, I-d) T(I-d, J). Step t (t = NB-1 down to
// 0) therefore runs two independent kernels:
//   trisolve_leaf_kernel    one CTA of 1024 threads per tile of subdiagonal t:
//                           applies subdiagonal t+1's two products, then solves;
//   trisolve_update_kernel  one CTA of 128 threads per tile with D < t that
//                           receives a product of subdiagonal t+1, accumulated
//                           in place in E.
// The engine captures the 2 NB launches once per order in a CUDA graph with the
// two kernels of a step side by side and a full dependency between steps.
// Divisors t_ii - t_jj are formed in FP64 from the high-precision diagonal and
// then rounded to the working type (the paper is silent here).
#pragma once
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace sr {

constexpr int kSolveTile = 32;

// Tile of the stepwise form: 16 for FP64, 32 otherwise. A leaf tile's wavefront
// runs on one SM and lies on the critical path; GB300's FP64 pipe retires about
// 2 FMA per SM per cycle, so a 32 x 32 FP64 tile (about 4000 FP64 warp
// instructions) takes ~60-100 us per block step, a 16 x 16 one about 8 times
// less for twice the steps. The update kernels' FP64 work is the same n^3/3
// FMAs for either size and runs beside the leaves. (FP32 keeps 32: at n = 4096
// its 16 x 16 form measured slower, 41.4 against 35.5 ms per refinement, the
// update launches and step gaps outweighing the shorter leaves.)
template <typename T> struct StepTile {
    static constexpr int B = SrNum<T>::kind == 1 ? 16 : kSolveTile;
};

// divisor t_ii - t_jj formed in high precision and rounded to the working type
template <typename T>
__device__ inline T sr_div_round(typename SrNum<T>::hp di, typename SrNum<T>::hp dj)
{
    return SrNum<T>::from_hp(di - dj);
}

// t_ii - t_jj from a double-double diagonal (hi, lo): TwoSum of the high
// parts, the low parts added, rounded once to FP64
__device__ inline double sr_div_round_dd(double hi_i, double lo_i, double hi_j, double lo_j)
{
    const double s = hi_i - hi_j;
    const double z = s - hi_i;
    double e = (hi_i - (s - z)) + (-hi_j - z);
    e += lo_i - lo_j;
    return s + e;
}

// Launch plan: for step t, the tiles (I << 16 | J) of subdiagonal t (solved)
// followed by the tiles with D < t that receive a product of subdiagonal t+1.
void trisolve_plan(int n, std::vector<uint32_t> &tiles, std::vector<long long> &offsets, int B = kSolveTile);

// Task list of the dataflow solve of one matrix (trisolve_flow_kernel): for
// s = NB-1 down to 0, the solve tasks of block subdiagonal s, then the helper
// tasks that subdiagonal s+1 is the last input of. A tile (I, J), D = I - J,
// whose products reach the subdiagonals d >= max(D + kFlowNear, kFlowFarNum
// NB / 16) leaves those (up to top = max(NB-1-J, I)) to helpers, kFlowChunk
// subdiagonals each, the highest first.
//   solve:  bit 63 = 0, J (bits 0-15), I (16-31), helper count (32-47),
//           the owner's highest subdiagonal (48-59)
//   helper: bit 63 = 1, J, I, lowest d (32-43), highest d (44-55), index (56-62)
constexpr int kFlowNear = 8;
constexpr int kFlowChunk = 16;
constexpr int kFlowFarNum = 8;   // helpers only for d >= kFlowFarNum NB / 16
constexpr int kFlowLag = 3;      // helpers completed by subdiagonal t follow the solves of t - kFlowLag
void trisolve_flow_plan(int n, std::vector<unsigned long long> &tasks);
void trisolve_flow_plan(int n, std::vector<unsigned long long> &tasks, int near, int chunk, int far_num, int lag);

// A group of independent solves in the same launches (schur_refine_batched):
// matrix b of the group, and its tiles in the plan as (b << 32 | I << 16 | J).
struct SolveMat {
    void *TE;
    int ld, n;
    const void *dhp;
    long long fbase;       // dataflow solve: first published word of this matrix
    void *acc = nullptr;   // stepwise solve: far products' sums apart from E (ld as TE), or none
};

// Group plan: for every step t (from the largest order's last subdiagonal
// down), the leaf tiles of all matrices with more than t block rows, then
// their update tiles; leaf[t] and upd[t] give the counts.
void trisolve_plan_group(const std::vector<int> &orders, std::vector<unsigned long long> &tiles,
                         std::vector<long long> &offsets, std::vector<long long> &nleaf, int B = kSolveTile);

// ---- contributions of subdiagonal t+1 to tiles with D < t --------------------
// Thread (tx, ty) owns the 4 x TN block rows 4tx.., columns TN*ty.., read with
// vector loads from shared memory: TN = 4 (64 threads for a 32 x 32 tile, 4
// vector loads per 32 FMAs; shared-memory bandwidth bounds the FP32 update)
// except for FP64, whose update is bound by the FP64 pipe and keeps TN = 2
// (128 threads for a 32 x 32 tile, 32 for a 16 x 16 one).
template <typename T, int B = kSolveTile> struct UpdShape {
    static constexpr int TN = SrNum<T>::kind == 1 ? 2 : 4;
    static constexpr int TX = B / 4;   // row groups of 4
    static constexpr int NT = TX * (B / TN);
};
template <typename T> struct SolveVec;
template <> struct SolveVec<float> {
    __device__ static void ld4(const float *p, float (&v)[4])
    {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    __device__ static void ld2(const float *p, float (&v)[2])
    {
        const float2 q = *reinterpret_cast<const float2 *>(p);
        v[0] = q.x; v[1] = q.y;
    }
};
template <> struct SolveVec<double> {
    __device__ static void ld4(const double *p, double (&v)[4])
    {
        const double2 q0 = *reinterpret_cast<const double2 *>(p);
        const double2 q1 = *reinterpret_cast<const double2 *>(p + 2);
        v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
    }
    __device__ static void ld2(const double *p, double (&v)[2])
    {
        const double2 q = *reinterpret_cast<const double2 *>(p);
        v[0] = q.x; v[1] = q.y;
    }
};
template <> struct SolveVec<cf> {
    __device__ static void ld4(const cf *p, cf (&v)[4])
    {
        const float4 q0 = *reinterpret_cast<const float4 *>(p);
        const float4 q1 = *reinterpret_cast<const float4 *>(p + 2);
        v[0] = {q0.x, q0.y}; v[1] = {q0.z, q0.w}; v[2] = {q1.x, q1.y}; v[3] = {q1.z, q1.w};
    }
    __device__ static void ld2(const cf *p, cf (&v)[2])
    {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = {q.x, q.y}; v[1] = {q.z, q.w};
    }
};
template <> struct SolveVec<cd> {
    __device__ static void ld4(const cd *p, cd (&v)[4])
    {
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = p[i];
    }
    __device__ static void ld2(const cd *p, cd (&v)[2])
    {
        v[0] = p[0];
        v[1] = p[1];
    }
};

// acc += Ta[0] Tb[0] - Ta[1] Tb[1] over the buffers' KB values of k for one thread's
// 4 x TN block (rows 4tx.., columns TN ty..); a product whose tiles do not
// exist (hasP / hasM false: beyond the matrix) is skipped, not multiplied by
// zeros. hasP and hasM are uniform over the threads that share the buffers.
template <typename T, int TN, int SA, int KB = kSolveTile>
__device__ __forceinline__ void tile_pair_products(const T (*Ta)[KB][SA], const T (*Tb)[KB][SA], int tx, int ty,
                                                   bool hasP, bool hasM, T (&acc)[4][TN])
{
    constexpr int B = KB;
    auto ldb = [&](const T *p, T (&v)[TN]) {
        if constexpr (TN == 4) {
            SolveVec<T>::ld4(p, v);
        } else {
            SolveVec<T>::ld2(p, v);
        }
    };
    if (hasP && hasM) {
#pragma unroll 4
        for (int k = 0; k < B; ++k) {
            T a[4], b[TN], m[4], c[TN];
            SolveVec<T>::ld4(&Ta[0][k][4 * tx], a);
            SolveVec<T>::ld4(&Ta[1][k][4 * tx], m);
            ldb(&Tb[0][k][TN * ty], b);
            ldb(&Tb[1][k][TN * ty], c);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    acc[i][j] = sr_fma(a[i], b[j], acc[i][j]);
                    acc[i][j] = sr_fma(-m[i], c[j], acc[i][j]);
                }
        }
    } else if (hasP || hasM) {
        const int u = hasP ? 0 : 1;
        const T sg = hasP ? SrNum<T>::one() : -SrNum<T>::one();
#pragma unroll 4
        for (int k = 0; k < B; ++k) {
            T a[4], b[TN];
            SolveVec<T>::ld4(&Ta[u][k][4 * tx], a);
            ldb(&Tb[u][k][TN * ty], b);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const T as = a[i] * sg;
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = sr_fma(as, b[j], acc[i][j]);
            }
        }
    }
}

template <typename T, bool GROUP = false, int B = kSolveTile>
__global__ void __launch_bounds__(UpdShape<T, B>::NT)
trisolve_update_kernel(int n, T *__restrict__ TE, int ld, int t, const uint32_t *__restrict__ plan,
                       const SolveMat *__restrict__ mats = nullptr,
                       const unsigned long long *__restrict__ gplan = nullptr, T *__restrict__ accb = nullptr,
                       int ldacc = 0)
{
    constexpr int SA = B + 4, SB = B + 4;
    uint32_t tile;
    if constexpr (GROUP) {
        const unsigned long long g = gplan[blockIdx.x];
        const SolveMat m = mats[g >> 32];
        TE = (T *)m.TE;
        ld = m.ld;
        n = m.n;
        accb = (T *)m.acc;
        ldacc = m.ld;
        tile = (uint32_t)g;
    } else {
        tile = plan[blockIdx.x];
    }
    const int NB = (n + B - 1) / B;
    const int I = (int)(tile >> 16), J = (int)(tile & 0xffffu);
    const int D = I - J;
    const int r0 = I * B, c0 = J * B;
    const int nr = min(B, n - r0), nc = min(B, n - c0);
    const int d = t + 1;
    __shared__ __align__(16) T Ta[2][B][SA];   // left operands, transposed: Ta[u][k][row]
    __shared__ __align__(16) T Tb[2][B][SB];   // right operands: Tb[u][k][col]
    constexpr int TN = UpdShape<T, B>::TN, NT = UpdShape<T, B>::NT, TX = UpdShape<T, B>::TX;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;   // block rows 4tx.., columns TN ty..
    const T Z = SrNum<T>::zero();
    const bool hasP = J + d < NB, hasM = I - d >= 0;
    const int kP = (J + d) * B, kM = (I - d) * B;
#pragma unroll
    for (int q = 0; q < B * B / NT; ++q) {
        const int e = tid + NT * q, lx = e % B, y = e / B;   // element (lx, y) of each tile
        Ta[0][y][lx] = (hasP && r0 + lx < n && kP + y < n) ? TE[sr_idx(r0 + lx, kP + y, ld)] : Z;
        Tb[0][lx][y] = (hasP && kP + lx < n && c0 + y < n) ? TE[sr_idx(kP + lx, c0 + y, ld)] : Z;
        Ta[1][y][lx] = (hasM && r0 + lx < n && kM + y < n) ? TE[sr_idx(r0 + lx, kM + y, ld)] : Z;
        Tb[1][lx][y] = (hasM && kM + lx < n && c0 + y < n) ? TE[sr_idx(kM + lx, c0 + y, ld)] : Z;
    }
    T acc[4][TN];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int x = 4 * tx + i, y = TN * ty + j;
            // with an accumulator the products sum apart from E, else into E in place
            acc[i][j] = (x < nr && y < nc && (D > 0 || x > y))
                            ? (accb ? accb[sr_idx(r0 + x, c0 + y, ldacc)] : TE[sr_idx(r0 + x, c0 + y, ld)])
                            : Z;
        }
    __syncthreads();
    tile_pair_products<T, TN, SA, B>(Ta, Tb, tx, ty, hasP, hasM, acc);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int x = 4 * tx + i, y = TN * ty + j;
            if (x < nr && y < nc && (D > 0 || x > y)) {
                if (accb) accb[sr_idx(r0 + x, c0 + y, ldacc)] = acc[i][j];
                else TE[sr_idx(r0 + x, c0 + y, ld)] = acc[i][j];
            }
        }
}

// ---- solve of the tiles of subdiagonal t ---------------------------------------
// B x B threads; thread a + B b owns entry (a, b) of the tile.
template <typename T, bool GROUP = false, int B = kSolveTile>
__global__ void __launch_bounds__(B * B)
trisolve_leaf_kernel(int n, T *__restrict__ TE, int ld, const typename SrNum<T>::hp *__restrict__ dhp,
                     const double *__restrict__ dlo, int t, const uint32_t *__restrict__ plan, int *__restrict__ flags,
                     double cap,
                     const SolveMat *__restrict__ mats = nullptr,
                     const unsigned long long *__restrict__ gplan = nullptr, T *__restrict__ accb = nullptr,
                     int ldacc = 0)
{
    using Hp = typename SrNum<T>::hp;
    constexpr int S = B + 1;
    const T Z = SrNum<T>::zero();
    uint32_t tile;
    if constexpr (GROUP) {
        // a group: each matrix has its own flag word
        const unsigned long long g = gplan[blockIdx.x];
        const SolveMat m = mats[g >> 32];
        TE = (T *)m.TE;
        ld = m.ld;
        n = m.n;
        accb = (T *)m.acc;
        ldacc = m.ld;
        dhp = (const Hp *)m.dhp;
        flags += (g >> 32);
        tile = (uint32_t)g;
    } else {
        tile = plan[blockIdx.x];
    }
    const int NB = (n + B - 1) / B;
    const int I = (int)(tile >> 16), J = (int)(tile & 0xffffu);
    const int D = I - J;
    const int r0 = I * B, c0 = J * B;
    const int nr = min(B, n - r0), nc = min(B, n - c0);
    const int d = t + 1;
    // phase 1: Ta[u][k][row], Tb[u][k][col]; phase 2: X, Ti = T_II, Tj = T_JJ
    __shared__ T sm[4][B][S];
    T (*Ta)[B][S] = sm;
    T (*Tb)[B][S] = sm + 2;
    T (*X)[S] = sm[0];
    T (*Ti)[S] = sm[1];
    T (*Tj)[S] = sm[2];
    __shared__ Hp dI[B], dJ[B];
    __shared__ double dIl[B], dJl[B];   // low parts of a double-double diagonal (dlo given)
    const int a = threadIdx.x % B, b = threadIdx.x / B;
    const bool own = a < nr && b < nc && (D > 0 || a > b);

    // 1. E plus the two products of subdiagonal t+1
    const bool hasP = d < NB && J + d < NB, hasM = d < NB && I - d >= 0;
    const int kP = (J + d) * B, kM = (I - d) * B;
    Ta[0][b][a] = (hasP && r0 + a < n && kP + b < n) ? TE[sr_idx(r0 + a, kP + b, ld)] : Z;
    Tb[0][a][b] = (hasP && kP + a < n && c0 + b < n) ? TE[sr_idx(kP + a, c0 + b, ld)] : Z;
    Ta[1][b][a] = (hasM && r0 + a < n && kM + b < n) ? TE[sr_idx(r0 + a, kM + b, ld)] : Z;
    Tb[1][a][b] = (hasM && kM + a < n && c0 + b < n) ? TE[sr_idx(kM + a, c0 + b, ld)] : Z;
    // E; with an accumulator, the far subdiagonals' products summed apart from it
    T acc = own ? TE[sr_idx(r0 + a, c0 + b, ld)] : Z;
    const T far = (own && accb) ? accb[sr_idx(r0 + a, c0 + b, ldacc)] : Z;
    const Hp hz = SrNum<Hp>::zero();
    if (threadIdx.x < B) {
        dI[threadIdx.x] = (threadIdx.x < nr) ? dhp[r0 + threadIdx.x] : hz;
        dIl[threadIdx.x] = (dlo && threadIdx.x < nr) ? dlo[r0 + threadIdx.x] : 0.0;
    } else if (threadIdx.x < 2 * B) {
        dJ[threadIdx.x - B] = (threadIdx.x - B < nc) ? dhp[c0 + threadIdx.x - B] : hz;
        dJl[threadIdx.x - B] = (dlo && threadIdx.x - B < nc) ? dlo[c0 + threadIdx.x - B] : 0.0;
    }
    __syncthreads();
    if (accb) {
        // the near products join the far ones, and E is added to their sum once
        T pn = far;
        if (hasP || hasM) {
#pragma unroll 8
            for (int k = 0; k < B; ++k) {
                pn = sr_fma(Ta[0][k][a], Tb[0][k][b], pn);
                pn = sr_fma(-Ta[1][k][a], Tb[1][k][b], pn);
            }
        }
        acc = acc + pn;
    } else if (hasP || hasM) {
#pragma unroll 8
        for (int k = 0; k < B; ++k) {
            acc = sr_fma(Ta[0][k][a], Tb[0][k][b], acc);
            acc = sr_fma(-Ta[1][k][a], Tb[1][k][b], acc);
        }
    }
    // divisor t_aa - t_bb formed in FP64 and rounded; its reciprocal (one IEEE
    // division, off the wavefront's critical path) turns each solve into a product
    T den = own ? sr_div_round<T>(dI[a], dJ[b]) : Z;
    if constexpr (SrNum<T>::kind == 1) {
        if (own && dlo) den = sr_div_round_dd(dI[a], dIl[a], dJ[b], dJl[b]);
    }
    const T rcp = (own && !(den == Z)) ? sr_recip(den) : Z;
    __syncthreads();

    // 2. wavefront over the tile's subdiagonals. When subdiagonal w is final, a
    // pending entry (a, b) adds T_II(a, b+w) X(b+w, b) (from the lane of its own
    // warp that owns (b+w, b)) and -X(a, a-w) T_JJ(a-w, b) (from shared memory).
    Ti[a][b] = (a <= b && a < nr && b < nr) ? TE[sr_idx(r0 + a, r0 + b, ld)] : Z;
    Tj[a][b] = (a <= b && a < nc && b < nc) ? TE[sr_idx(c0 + a, c0 + b, ld)] : Z;
    X[a][b] = Z;
    __syncthreads();
    const int wlo = (D > 0) ? -(B - 1) : 1;
    T xv = Z;
    int bad = 0;
    for (int w = B - 1; w >= wlo; --w) {
        if (own && a - b == w) {
            if (den == Z) {
                bad |= SR_FLAG_NONDISTINCT;
            } else {
                xv = -(acc * rcp);
                if (cap > 0.0 && sr_over_cap(xv, cap)) xv = Z;   // Example 4's trick, before any use
                if (!sr_finite(xv)) bad |= SR_FLAG_NONFINITE;
            }
            X[a][b] = xv;
        }
        __syncthreads();
        const int c = b + w;                         // (c, b): lane (c + B b) mod 32 of this warp
        const T xcol = sr_shfl(xv, (c + B * b) & 31);
        if (own && a - b < w) {
            if (c < nr) acc = sr_fma(Ti[a][c], xcol, acc);
            const int c2 = a - w;                    // (a, c2), c2 < b
            if (c2 >= 0) acc = sr_fma(-X[a][c2], Tj[c2][b], acc);
        }
    }
    if (bad) atomicOr(flags, bad);
    if (own) TE[sr_idx(r0 + a, c0 + b, ld)] = xv;
}

// The launch sequence on two streams: leaf kernels on `st`, update kernels on
// `aux`, with a full dependency between consecutive steps (events ev0, ev1).
// plan: device copy of trisolve_plan's tiles for the tile StepTile<T>::B;
// offsets: its host offsets.
template <typename T>
inline cudaError_t trisolve_launches(cudaStream_t st, cudaStream_t aux, cudaEvent_t ev0, cudaEvent_t ev1, int n,
                                     T *TE, int ld, const typename SrNum<T>::hp *dhp, const double *dlo,
                                     int *flags, const uint32_t *plan, const std::vector<long long> &offsets,
                                     double cap = 0.0, T *accb = nullptr, int ldacc = 0)
{
    constexpr int B = StepTile<T>::B;   // the plan is built for this tile
    const int NB = (n + B - 1) / B;
    // accb (optional): the far products' sums, apart from E; cleared first
    cudaError_t e = accb ? cudaMemset2DAsync(accb, (size_t)ldacc * sizeof(T), 0, (size_t)n * sizeof(T), n, st)
                         : cudaSuccess;
    if (e == cudaSuccess) e = cudaEventRecord(ev0, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev0, 0);
    for (int t = NB - 1; t >= 0 && e == cudaSuccess; --t) {
        const int l = NB - 1 - t;
        const long long nleaf = NB - t;
        const long long nupd = offsets[l + 1] - offsets[l] - nleaf;
        trisolve_leaf_kernel<T, false, B><<<(unsigned)nleaf, B * B, 0, st>>>(
            n, TE, ld, dhp, dlo, t, plan + offsets[l], flags, cap, nullptr, nullptr, accb, ldacc);
        if (nupd > 0)
            trisolve_update_kernel<T, false, B><<<(unsigned)nupd, UpdShape<T, B>::NT, 0, aux>>>(
                n, TE, ld, t, plan + offsets[l] + nleaf, nullptr, nullptr, accb, ldacc);
        e = cudaGetLastError();
        // both kernels of this step finish before either of the next starts
        if (e == cudaSuccess) e = cudaEventRecord(ev0, st);
        if (e == cudaSuccess) e = cudaEventRecord(ev1, aux);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev1, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev0, 0);
    }
    return e;
}

// The launches of a group plan (no double-double divisors; the plan built for
// the tile B): the same two-stream sequence as trisolve_launches, steps
// t = nsteps-1 .. 0.
template <typename T, int B = kSolveTile>
inline cudaError_t trisolve_launches_group(cudaStream_t st, cudaStream_t aux, cudaEvent_t ev0, cudaEvent_t ev1,
                                           const SolveMat *mats, int *flags, const unsigned long long *plan,
                                           const std::vector<long long> &offsets, const std::vector<long long> &nleaf,
                                           double cap = 0.0)
{
    const int nsteps = (int)nleaf.size();
    cudaError_t e = cudaEventRecord(ev0, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev0, 0);
    for (int l = 0; l < nsteps && e == cudaSuccess; ++l) {
        const int t = nsteps - 1 - l;
        const long long nl = nleaf[l];
        const long long nupd = offsets[l + 1] - offsets[l] - nl;
        if (nl > 0)
            trisolve_leaf_kernel<T, true, B><<<(unsigned)nl, B * B, 0, st>>>(0, nullptr, 0, nullptr, nullptr, t,
                                                                            nullptr, flags, cap, mats, plan + offsets[l]);
        if (nupd > 0)
            trisolve_update_kernel<T, true, B><<<(unsigned)nupd, UpdShape<T, B>::NT, 0, aux>>>(
                0, nullptr, 0, t, nullptr, mats, plan + offsets[l] + nl);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(ev0, st);
        if (e == cudaSuccess) e = cudaEventRecord(ev1, aux);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev1, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev0, 0);
    }
    return e;
}

// ---- symmetric A (Sec. 2.5): T diagonal, the solve elementwise ---------------
// l_ij = -e_ij / (t_ii - t_jj) for i > j (eq. "lij" with t_ik = 0 for k != i),
// the divisor formed in high precision and rounded to the working type, then
// one IEEE division: the same operations as Alg. 2 with a diagonal T. Thread
// (lane, warp) of a 256-thread block takes rows of a 32 x 32 block, four
// columns each.
template <typename T>
__global__ void __launch_bounds__(256)
diag_solve_kernel(int n, T *__restrict__ TE, int ld, const typename SrNum<T>::hp *__restrict__ dhp,
                  int *__restrict__ flags, double cap)
{
    const int i = blockIdx.x * 32 + (threadIdx.x & 31);
    const int jb = blockIdx.y * 32 + (threadIdx.x >> 5);
    int bad = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const int j = jb + 8 * w;
        if (i < n && j < i) {
            T x = SrNum<T>::zero();
            if constexpr (SrNum<T>::kind >= 2) {
                // Hermitian A: the Schur form is real diagonal, so the divisor is
                // formed from the real parts of the hp diagonal, rounded once to the
                // low precision, and divides both parts of e_ij (two IEEE divisions)
                using R = decltype(x.x);
                const R den = (R)(dhp[i].x - dhp[j].x);
                if (den == (R)0) {
                    bad |= SR_FLAG_NONDISTINCT;
                } else {
                    const T e = TE[sr_idx(i, j, ld)];
                    x = T{-(e.x / den), -(e.y / den)};
                    if (cap > 0.0 && sr_over_cap(x, cap)) x = SrNum<T>::zero();   // Example 4's trick
                    if (!sr_finite(x)) bad |= SR_FLAG_NONFINITE;
                }
            } else {
                const T den = sr_div_round<T>(dhp[i], dhp[j]);
                if (den == SrNum<T>::zero()) {
                    bad |= SR_FLAG_NONDISTINCT;
                } else {
                    x = -(TE[sr_idx(i, j, ld)] / den);
                    if (cap > 0.0 && sr_over_cap(x, cap)) x = SrNum<T>::zero();   // Example 4's trick
                    if (!sr_finite(x)) bad |= SR_FLAG_NONFINITE;
                }
            }
            TE[sr_idx(i, j, ld)] = x;
        }
    }
    if (bad) atomicOr(flags, bad);
}

// ---- block entries of the real Schur form (2 x 2 diagonal blocks) ----------
// rounded operations without contraction: the elimination below takes the
// oracle's steps one by one, so a zero pivot is found exactly where it finds one
__device__ __forceinline__ float q_mul(float x, float y) { return __fmul_rn(x, y); }
__device__ __forceinline__ double q_mul(double x, double y) { return __dmul_rn(x, y); }
__device__ __forceinline__ float q_sub(float x, float y) { return __fsub_rn(x, y); }
__device__ __forceinline__ double q_sub(double x, double y) { return __dsub_rn(x, y); }
__device__ __forceinline__ float q_div(float x, float y) { return __fdiv_rn(x, y); }
__device__ __forceinline__ double q_div(double x, double y) { return __ddiv_rn(x, y); }

// Row u of the inverse of a Kronecker matrix of order m <= 4 (padded to 4 x 4
// with the identity): Gaussian elimination with partial pivoting (the first
// largest pivot; the padding rows are never chosen while a real row has a
// nonzero in the column), applied to the identity alongside, then back
// substitution. Fully unrolled, in registers. Returns false on a zero pivot
// (a shared eigenvalue).
template <typename T>
__device__ __forceinline__ bool kron_inverse_row(T (&M)[4][4], int u, T (&row)[4])
{
    const T Z = (T)0, One = (T)1;
    T R[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) R[r][c] = r == c ? One : Z;
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int p = k;
        T best = fabs(M[k][k]);
#pragma unroll
        for (int r = k + 1; r < 4; ++r)
            if (fabs(M[r][k]) > best) {
                best = fabs(M[r][k]);
                p = r;
            }
#pragma unroll
        for (int r = k + 1; r < 4; ++r) {
            if (p == r) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const T t0 = M[k][c]; M[k][c] = M[r][c]; M[r][c] = t0;
                    const T t1 = R[k][c]; R[k][c] = R[r][c]; R[r][c] = t1;
                }
            }
        }
        if (M[k][k] == Z) { ok = false; M[k][k] = One; }
#pragma unroll
        for (int r = k + 1; r < 4; ++r) {
            const T f = q_div(M[r][k], M[k][k]);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (c >= k) M[r][c] = q_sub(M[r][c], q_mul(f, M[k][c]));
                R[r][c] = q_sub(R[r][c], q_mul(f, R[k][c]));
            }
        }
    }
    T Xc[4][4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int r = 3; r >= 0; --r) {
            T acc = R[r][c];
#pragma unroll
            for (int v = r + 1; v < 4; ++v) acc = q_sub(acc, q_mul(M[r][v], Xc[v][c]));
            Xc[r][c] = q_div(acc, M[r][r]);
        }
#pragma unroll
    for (int r = 0; r < 4; ++r)
        if (r == u)
#pragma unroll
            for (int c = 0; c < 4; ++c) row[c] = Xc[r][c];
    return ok;
}

// ---- the whole solve in one launch: a dataflow over the tiles --------------
// The same tile equations as above, solved by one persistent launch whose
// CTAs claim tasks through a ticket counter, in the order of a task list
// (trisolve_flow_plan; for a group of matrices, the tiles of the group plan).
// A solve task for tile (I, J), D = I - J, applies the two products of each
// of its subdiagonals d (the block form of Alg. 3's update products)
//     T(I, J+d) L(J+d, J)   and   -L(I, I-d) T(I-d, J)
// as soon as the two L tiles of subdiagonal d are published, adds E and the
// helpers' sum, solves the tile equation by the wavefront of
// trisolve_leaf_kernel and publishes X. Helper tasks (one matrix) take the
// products of the far subdiagonals d >= max(D + kFlowNear, kFlowFarNum NB/16)
// of a tile, kFlowChunk subdiagonals each, as soon as those are published, and
// add them into the tile's accumulator in a fixed order (helper h waits until
// h helpers are done), so the result does not depend on timing. Without them
// the products of the tiles near the main diagonal, which have the most, pile
// up at the end of the wavefront, when its subdiagonals hold the most tiles.
//
// The CTA has 512 threads, two entries of the tile each in the solve (the
// wavefront's steps are barrier-bound: few entries per thread keep them
// short), and two CTAs share an SM, so one CTA's products run while the
// other waits at its wavefront's barriers. The products of a task are split
// over NPP pair lanes (subdiagonals d = hi-l, hi-l-NPP, ... for lane l) of
// two groups each, one per half of K; every group has its own operand
// buffers and named barrier, so it waits only on its own inputs; the partial
// sums meet in shared memory.
//
// Forward progress does not need the CTAs to be co-resident: every input of
// a task (tiles of higher subdiagonals, the tile's earlier helpers, a solve
// task's helpers) holds a smaller ticket, and a ticket is taken only by a
// running CTA, so the smallest unfinished ticket always finds its inputs
// done. Every wait is bounded (kFlowSpin polls); one that runs out sets
// SR_FLAG_TIMEOUT and an abort word that ends all other waits, and the launch
// runs to its end without further waiting.
//
// work[0]: ticket counter; work[1]: abort word; work[2 + I NB + J]: tile
// (I, J) published; work[2 + NB^2 + I NB + J]: helpers of tile (I, J) done.
// The launcher clears them before the kernel.
template <typename T> struct FlowShape {
    using Hp = typename SrNum<T>::hp;
    static constexpr int B = kSolveTile;
    static constexpr int NT = 512;                  // threads of the CTA (two CTAs per SM)
    static constexpr int EPT = B * B / NT;          // entries of the tile per thread in the solve
    static constexpr int WS = NT / 32;              // warps: thread (a, w) owns columns w + WS q
    // products: rows 4tx.., columns TN ty.. per thread (TN = 4: 64 threads a
    // group; TN = 2: 128); every thread is in a group, and the two groups of a
    // pair lane take the two halves (KH) of the subdiagonal's K = 32
    static constexpr int TN = SrNum<T>::kind == 0 ? 4 : 2;
    static constexpr int NTG = 8 * (B / TN);
    static constexpr int NG = NT / NTG;             // groups
    static constexpr int NPP = NG / 2;              // pair lanes: subdiagonals in flight
    static constexpr int KH = B / 2;
    static constexpr int SA = B + 4;                // row stride of the operand buffers
    static constexpr int SX = B + 1;                // row stride of the solve's tiles
    static constexpr size_t kSlot = 4 * KH * SA;    // elements of one group's operands
    static constexpr size_t smem = (NG * kSlot + 3 * B * SX) * sizeof(T) + 2 * B * (sizeof(Hp) + sizeof(double))
                                   + 16 + 2 * B * sizeof(int);
    static_assert(NG * NTG == NT && NG % 2 == 0, "pairs of groups fill the CTA");
    static_assert(EPT * NT == B * B, "one or more whole entries per thread");
    static_assert(kSlot >= (size_t)B * SX, "a group's buffers hold its partial sums");
};
constexpr int kFlowSpin = 1 << 22;   // polls of one wait (a few hundred ns apart)

__device__ inline int flow_ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ inline void flow_st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Wait, by a whole warp, until the word *f reaches `target` (a published
// flag: 1; a helper count: the number of helpers done); false after an abort
// or a timeout. Lane 0 loads (acquire) and broadcasts, so every branch is
// uniform over the warp and the warp stays converged for the barrier that
// follows.
__device__ inline bool flow_wait(const int *f, int *abort_w, int *flags, int target = 1)
{
    const unsigned lane = threadIdx.x & 31u;
    for (int it = 0; it < kFlowSpin; ++it) {
        int v = 0, ab = 0;
        if (lane == 0) {
            v = flow_ld_acquire(f) >= target;
            if (!v) ab = *(volatile int *)abort_w;
        }
        v = __shfl_sync(0xffffffffu, v, 0);
        ab = __shfl_sync(0xffffffffu, ab, 0);
        if (v) return true;
        if (ab) return false;
        __nanosleep(it < 32 ? 32 : 256);
    }
    if (lane == 0) {
        atomicOr(flags, SR_FLAG_TIMEOUT);
        atomicExch(abort_w, 1);
    }
    __syncwarp();
    return false;
}
// named barrier of nthreads threads (whole warps); the warp reconverges
// first, as bar.sync requires of every warp that executes it
__device__ inline void flow_bar(int id, int nthreads)
{
    __syncwarp();
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
// loads of published tiles go to L2, never to a stale L1 line
__device__ inline float flow_ldcg(const float *p) { return __ldcg(p); }
__device__ inline double flow_ldcg(const double *p) { return __ldcg(p); }
__device__ inline cf flow_ldcg(const cf *p)
{
    const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    return {v.x, v.y};
}
// The wavefront of one tile of the real Schur form in the dataflow solve, and
// the store of its unknowns: over block entries, as in
// trisolve_quasi_leaf_kernel. The pending sums of a block entry meet in Cs,
// each thread forms its unknown from its row of the inverse of the block
// entry's Kronecker matrix, and entries still pending take the products with
// the block entries just finished (the row block starting at s in their
// column, the column block ending at e in their row). A call of its own:
// the block structure is read from rbq, cbq here. Returns the error flags.
template <typename T, int EPT, int WS, int SX>
__device__ __noinline__ int flow_quasi_tile(T *__restrict__ TE, int ld, int r0, int c0, int nr, int nc, int D,
                                            int a, int wq, const bool *own, T *acc, const T *kinv, T (*Ti)[SX],
                                            T (*Tj)[SX], T (*X)[SX], T (*Cs)[SX], const int *rbq, const int *cbq,
                                            double cap)
{
    constexpr int B = kSolveTile;
    const T Z = (T)0;
    const int ra = rbq[a] == 0 ? a - 1 : a;
    const int pq = rbq[ra] == 2 ? 2 : 1;
    int fsq[EPT], csq[EPT], clq[EPT], mq[EPT];
    T xv[EPT];
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
        const int b = wq + WS * q;
        csq[q] = cbq[b] == 0 ? b - 1 : b;
        clq[q] = cbq[b] == 2 ? b + 1 : b;
        mq[q] = pq * (cbq[csq[q]] == 2 ? 2 : 1);
        fsq[q] = ra - clq[q];
        xv[q] = Z;
    }
    const int wlo = (D > 0) ? -(B - 1) : 1;
    __syncthreads();
    for (int w = B - 1; w >= wlo; --w) {
#pragma unroll
        for (int q = 0; q < EPT; ++q)
            if (own[q] && fsq[q] == w) Cs[a][wq + WS * q] = acc[q];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < EPT; ++q)
            if (own[q] && fsq[q] == w) {
                T x = Z;
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    if (v < mq[q]) x = sr_fma(kinv[4 * q + v], -Cs[ra + v % pq][csq[q] + v / pq], x);
                if (cap > 0.0 && sr_over_cap(x, cap)) x = Z;   // Example 4's trick, before any use
                X[a][wq + WS * q] = x;
                xv[q] = x;
            }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int b = wq + WS * q;
            if (own[q] && fsq[q] < w) {
                const int sr0 = w + clq[q];
                if (sr0 >= 0 && sr0 < nr && rbq[sr0] != 0) {
                    acc[q] = sr_fma(Ti[a][sr0], X[sr0][b], acc[q]);
                    if (rbq[sr0] == 2) acc[q] = sr_fma(Ti[a][sr0 + 1], X[sr0 + 1][b], acc[q]);
                }
                const int e = ra - w;
                if (e >= 0 && e < nc && cbq[e] != 2) {
                    if (cbq[e] == 0) acc[q] = sr_fma(-X[a][e - 1], Tj[e - 1][b], acc[q]);
                    acc[q] = sr_fma(-X[a][e], Tj[e][b], acc[q]);
                }
            }
        }
    }
    int bad = 0;
#pragma unroll
    for (int q = 0; q < EPT; ++q)
        if (own[q]) {
            if (!sr_finite(xv[q])) bad |= SR_FLAG_NONFINITE;
            TE[sr_idx(r0 + a, c0 + wq + WS * q, ld)] = xv[q];
        }
    return bad;
}

template <typename T, bool GROUP = false, bool QUASI = false>
__global__ void __launch_bounds__(FlowShape<T>::NT, 2)
trisolve_flow_kernel(int n0, T *__restrict__ TE0, int ld0, const typename SrNum<T>::hp *__restrict__ dhp0,
                     const double *__restrict__ dlo, int *__restrict__ flags0, int *__restrict__ work,
                     const unsigned long long *__restrict__ plan, int ntasks, T *__restrict__ accb, int ldacc,
                     double cap, const SolveMat *__restrict__ mats = nullptr, const int *__restrict__ qblk = nullptr)
{
    using S = FlowShape<T>;
    using Hp = typename SrNum<T>::hp;
    constexpr int B = S::B, SA = S::SA, SX = S::SX, NTG = S::NTG, NG = S::NG, TN = S::TN, EPT = S::EPT,
                  WS = S::WS, NPP = S::NPP, KH = S::KH;
    extern __shared__ __align__(16) unsigned char flow_smem[];
    T *ops = reinterpret_cast<T *>(flow_smem);
    T (*Ti)[SX] = reinterpret_cast<T (*)[SX]>(ops + NG * S::kSlot);
    T (*Tj)[SX] = Ti + B;
    T (*X)[SX] = Tj + B;
    Hp *dI = reinterpret_cast<Hp *>(X + B);
    Hp *dJ = dI + B;
    double *dIl = reinterpret_cast<double *>(dJ + B);
    double *dJl = dIl + B;
    int *s_ticket = reinterpret_cast<int *>(dJl + B);
    int *rbq = s_ticket + 4, *cbq = rbq + B;   // real Schur form: block arrays of the tile's rows, columns

    const int tid = threadIdx.x;
    int *abort_w = work + 1;
    const int g = tid / NTG, gt = tid % NTG;   // product group
    const int pl = g >> 1, kh = g & 1;         // its pair lane and half of K
    T *slot = ops + g * S::kSlot;
    T (*Ta)[KH][SA] = reinterpret_cast<T (*)[KH][SA]>(slot);               // Ta[u][k][row]
    T (*Tb)[KH][SA] = reinterpret_cast<T (*)[KH][SA]>(slot + 2 * KH * SA);   // Tb[u][k][col]
    const int tx = gt & 7, ty = gt >> 3;    // products: rows 4tx.., columns TN ty..
    const int a = tid & 31, wq = tid >> 5;  // solve: entries (a, wq + WS q), q < EPT
    const T Z = SrNum<T>::zero();
    const Hp hz = SrNum<Hp>::zero();

    for (;;) {
        if (tid == 0) *s_ticket = atomicAdd(work, 1);
        __syncthreads();
        const int k = *s_ticket;
        if (k >= ntasks) break;
        // the task, its tile and matrix (a group: matrix b of the plan entry
        // b << 32 | I << 16 | J, with its own error word and published words;
        // one matrix: solve and helper tasks)
        const unsigned long long task = plan[k];
        int n = n0, ld = ld0;
        T *TE = TE0;
        const Hp *dhp = dhp0;
        int *flags = flags0, *pub = work + 2;
        const int I = (int)((task >> 16) & 0xffffu), J = (int)(task & 0xffffu);
        bool helper = false;
        int nhelp = 0, dlow = 0, dhigh = 0, hidx = 0;
        if constexpr (GROUP) {
            const SolveMat m = mats[task >> 32];
            TE = (T *)m.TE;
            ld = m.ld;
            n = m.n;
            dhp = (const Hp *)m.dhp;
            flags += (task >> 32);
            pub += m.fbase;
        } else {
            helper = (task >> 63) != 0;
            if (helper) {
                dlow = (int)((task >> 32) & 0xfffu);
                dhigh = (int)((task >> 44) & 0xfffu);
                hidx = (int)((task >> 56) & 0x7fu);
            } else {
                nhelp = (int)((task >> 32) & 0xffffu);
                dhigh = (int)((task >> 48) & 0xfffu);
            }
        }
        const int NB = (n + B - 1) / B;
        int *cnt = pub + NB * NB;   // helpers done per tile (one matrix only)
        const int D = I - J, r0 = I * B, c0 = J * B;
        const int nr = min(B, n - r0), nc = min(B, n - c0);

        // the pair products of subdiagonals d = dh - pl, dh - pl - NPP, ... >= dl,
        // each over this group's half of K, into pacc
        T pacc[4][TN];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) pacc[i][j] = Z;
        auto pair_products = [&](int dh, int dl) {
            for (int d = dh - pl; d >= dl; d -= NPP) {
                const bool hasP = J + d < NB, hasM = I - d >= 0;
                if (gt < 32) {   // the group's first warp waits for both inputs
                    bool ok = true;
                    if (hasP) ok = flow_wait(pub + (J + d) * NB + J, abort_w, flags);
                    if (ok && hasM) flow_wait(pub + I * NB + (I - d), abort_w, flags);
                }
                flow_bar(1 + g, NTG);
                const int kP = (J + d) * B + kh * KH, kM = (I - d) * B + kh * KH;
                // left operands: 32 rows x KH, rows along the lanes
#pragma unroll
                for (int e = gt; e < B * KH; e += NTG) {
                    const int row = e & 31, kk = e >> 5;
                    Ta[0][kk][row] = (hasP && r0 + row < n && kP + kk < n) ? TE[sr_idx(r0 + row, kP + kk, ld)] : Z;
                    Ta[1][kk][row] =
                        (hasM && r0 + row < n && kM + kk < n) ? flow_ldcg(&TE[sr_idx(r0 + row, kM + kk, ld)]) : Z;
                }
                // right operands: KH x 32 columns, k along the lanes
#pragma unroll
                for (int e = gt; e < KH * B; e += NTG) {
                    const int kk = e % KH, col = e / KH;
                    Tb[0][kk][col] =
                        (hasP && kP + kk < n && c0 + col < n) ? flow_ldcg(&TE[sr_idx(kP + kk, c0 + col, ld)]) : Z;
                    Tb[1][kk][col] = (hasM && kM + kk < n && c0 + col < n) ? TE[sr_idx(kM + kk, c0 + col, ld)] : Z;
                }
                flow_bar(1 + g, NTG);
                tile_pair_products<T, TN, SA, KH>(Ta, Tb, tx, ty, hasP, hasM, pacc);
                flow_bar(1 + g, NTG);   // the next operands overwrite this group's buffers
            }
        };
        // the groups' partial sums, each into its own operand buffer (after a
        // barrier: every group is done with its operands)
        auto store_partials = [&]() {
            T (*P)[SX] = reinterpret_cast<T (*)[SX]>(slot);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) P[4 * tx + i][TN * ty + j] = pacc[i][j];
        };
        auto partial_sum = [&](int b) {
            T v = Z;
#pragma unroll
            for (int gg = 0; gg < NG; ++gg) v = v + reinterpret_cast<const T (*)[SX]>(ops + gg * S::kSlot)[a][b];
            return v;
        };

        if (helper) {
            // helper: subdiagonals dhigh .. dlow of tile (I, J) into its
            // accumulator, after the helper before it (a fixed order of sums)
            pair_products(dhigh, dlow);
            __syncthreads();
            store_partials();
            if (tid < 32) flow_wait(cnt + I * NB + J, abort_w, flags, hidx);
            __syncthreads();
#pragma unroll
            for (int q = 0; q < EPT; ++q) {
                const int b = wq + WS * q;
                if (a < nr && b < nc) {
                    T *pa = &accb[sr_idx(r0 + a, c0 + b, ldacc)];
                    const T prev = hidx ? flow_ldcg(pa) : Z;
                    *pa = prev + partial_sum(b);
                }
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) flow_st_release(cnt + I * NB + J, hidx + 1);
            continue;
        }

        // inputs that no tile writes: T_II, T_JJ, the diagonals and E_IJ (the
        // real Schur form: with the couplings of the 2 x 2 blocks in T_II, T_JJ)
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int b = wq + WS * q;
            bool ci = false, cj = false;
            if constexpr (QUASI) {
                ci = a == b + 1 && b < nr && qblk[r0 + b] == 2;
                cj = a == b + 1 && b < nc && qblk[c0 + b] == 2;
            }
            Ti[a][b] = ((a <= b && b < nr) || ci) ? TE[sr_idx(r0 + a, r0 + b, ld)] : Z;
            Tj[a][b] = ((a <= b && b < nc) || cj) ? TE[sr_idx(c0 + a, c0 + b, ld)] : Z;
        }
        if (tid < B) {
            dI[tid] = (tid < nr) ? dhp[r0 + tid] : hz;
            dIl[tid] = (dlo && tid < nr) ? dlo[r0 + tid] : 0.0;
            if constexpr (QUASI) rbq[tid] = tid < nr ? qblk[r0 + tid] : 1;
        } else if (tid < 2 * B) {
            dJ[tid - B] = (tid - B < nc) ? dhp[c0 + tid - B] : hz;
            dJl[tid - B] = (dlo && tid - B < nc) ? dlo[c0 + tid - B] : 0.0;
            if constexpr (QUASI) cbq[tid - B] = tid - B < nc ? qblk[c0 + tid - B] : 1;
        }
        bool own[EPT];
        T acc[EPT];
        if constexpr (!QUASI) {
#pragma unroll
            for (int q = 0; q < EPT; ++q) {
                const int b = wq + WS * q;
                own[q] = a < nr && b < nc && (D > 0 || a > b);
                acc[q] = own[q] ? TE[sr_idx(r0 + a, c0 + b, ld)] : Z;
            }
        }
        __syncthreads();
        T rcp[EPT];
        int bad = 0;
        // real Schur form: each entry's block entry (first row ra of its row
        // block, columns cs..cl) and its row of the inverse of the block entry's
        // Kronecker matrix (as the leaf kernel of the padded stepwise form); the
        // block structure is read again from rbq, cbq where it is used
        T kinv[EPT][4];
        if constexpr (QUASI) {
            const int ra = rbq[a] == 0 ? a - 1 : a;
            const int p = rbq[ra] == 2 ? 2 : 1;
#pragma unroll
            for (int q = 0; q < EPT; ++q) {
                const int b = wq + WS * q;
                const int cs = cbq[b] == 0 ? b - 1 : b;
                const int m = p * (cbq[cs] == 2 ? 2 : 1);
                own[q] = a < nr && b < nc && (D > 0 || ra > cs);
                acc[q] = own[q] ? TE[sr_idx(r0 + a, c0 + b, ld)] : Z;
#pragma unroll
                for (int v = 0; v < 4; ++v) kinv[q][v] = Z;
                if (own[q]) {
                    T K[4][4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int ur = u % p, uc = u / p;
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const int vr = v % p, vc = v / p;
                            T kv = (u == v) ? (T)1 : Z;
                            if (u < m && v < m) {
                                if (u == v) kv = (T)(dI[ra + ur] - dJ[cs + uc]);
                                else if (uc == vc) kv = Ti[ra + ur][ra + vr];
                                else if (ur == vr) kv = -Tj[cs + vc][cs + uc];
                                else kv = Z;
                            }
                            K[u][v] = kv;
                        }
                    }
                    if (!kron_inverse_row(K, (a - ra) + (b - cs) * p, kinv[q])) bad |= SR_FLAG_NONDISTINCT;
                }
            }
        } else {
            // divisors t_aa - t_bb formed in high precision, rounded, inverted once
            // (before the waits: they need only the diagonals)
#pragma unroll
            for (int q = 0; q < EPT; ++q) {
                const int b = wq + WS * q;
                T den = own[q] ? sr_div_round<T>(dI[a], dJ[b]) : Z;
                if constexpr (SrNum<T>::kind == 1) {
                    if (own[q] && dlo) den = sr_div_round_dd(dI[a], dIl[a], dJ[b], dJl[b]);
                }
                if (own[q] && den == Z) bad |= SR_FLAG_NONDISTINCT;
                rcp[q] = (own[q] && !(den == Z)) ? sr_recip(den) : Z;
            }
        }

        // the owner's products: the subdiagonals its helpers leave (all of
        // them without helpers)
        const int top = max(NB - 1 - J, I);
        pair_products(GROUP ? top : dhigh, D + 1);
        __syncthreads();
        store_partials();
        if (nhelp && tid < 32) flow_wait(cnt + I * NB + J, abort_w, flags, nhelp);
        __syncthreads();
        // E, then the helpers' sum, then the groups' partial sums
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int b = wq + WS * q;
            if (nhelp && own[q]) acc[q] = acc[q] + flow_ldcg(&accb[sr_idx(r0 + a, c0 + b, ldacc)]);
            acc[q] = acc[q] + partial_sum(b);
        }

        // wavefront over the tile's subdiagonals w (see trisolve_leaf_kernel);
        // an entry with a zero divisor is set to zero and flagged
        const int wlo = (D > 0) ? -(B - 1) : 1;
        T xv[EPT];
#pragma unroll
        for (int q = 0; q < EPT; ++q) xv[q] = Z;
        if constexpr (QUASI) {
            // the block-entry wavefront and the store (flow_quasi_tile); Cs is the
            // first group's product buffers, free once every partial sum is read
            bad |= flow_quasi_tile<T, EPT, WS, SX>(TE, ld, r0, c0, nr, nc, D, a, wq, own, acc, &kinv[0][0], Ti, Tj,
                                                   X, reinterpret_cast<T (*)[SX]>(ops), rbq, cbq, cap);
        } else
        for (int w = B - 1; w >= wlo; --w) {
#pragma unroll
            for (int q = 0; q < EPT; ++q)
                if (own[q] && a - (wq + WS * q) == w) {
                    xv[q] = -(acc[q] * rcp[q]);
                    if (cap > 0.0 && sr_over_cap(xv[q], cap)) xv[q] = Z;   // Example 4's trick, before any use
                    X[a][wq + WS * q] = xv[q];
                }
            __syncthreads();
            const int c2 = a - w;                    // (a, c2): row a's entry of subdiagonal w
#pragma unroll
            for (int q = 0; q < EPT; ++q) {
                const int b = wq + WS * q;
                const int c = b + w;                 // (c, b): lane c of this warp, same q
                const T xcol = sr_shfl(xv[q], c & 31);
                if (own[q] && a - b < w) {
                    if (c < nr) acc[q] = sr_fma(Ti[a][c], xcol, acc[q]);
                    if (c2 >= 0) acc[q] = sr_fma(-X[a][c2], Tj[c2][b], acc[q]);
                }
            }
        }
        if constexpr (!QUASI) {
#pragma unroll
            for (int q = 0; q < EPT; ++q)
                if (own[q]) {
                    if (!sr_finite(xv[q])) bad |= SR_FLAG_NONFINITE;
                    TE[sr_idx(r0 + a, c0 + wq + WS * q, ld)] = xv[q];
                }
        }
        if (bad) atomicOr(flags, bad);
        __threadfence();
        __syncthreads();
        if (tid == 0) flow_st_release(pub + I * NB + J, 1);
    }
}

// The dataflow solve of a group (no double-double divisors, no helpers):
// plan = the tiles (b << 32 | I << 16 | J) in an order that lists every tile
// after its inputs; mats[b].fbase = start of matrix b's NB_b^2 published
// words in work + 2; nwords = 2 + their total.
template <typename T>
inline cudaError_t trisolve_flow_launch_group(cudaStream_t st, const SolveMat *mats, int *flags, int *work,
                                              size_t nwords, const unsigned long long *plan, int ntiles, int ctas,
                                              double cap = 0.0)
{
    cudaError_t e = cudaMemsetAsync(work, 0, nwords * sizeof(int), st);
    if (e != cudaSuccess || ntiles < 1) return e;
    trisolve_flow_kernel<T, true><<<(unsigned)std::max(1, std::min(ctas, ntiles)), FlowShape<T>::NT,
                                    FlowShape<T>::smem, st>>>(0, nullptr, 0, nullptr, nullptr, flags, work, plan,
                                                              ntiles, nullptr, 0, cap, mats);
    return cudaGetLastError();
}

// Clears the flow state and launches the dataflow solve of one matrix on st
// with at most `ctas` CTAs (one ticket loop each): plan = trisolve_flow_plan's
// tasks (device), accb = the helpers' accumulators (n x n, leading dimension
// ldacc), work = 2 + 2 NB^2 ints (ticket, abort, published words, helper
// counts).
template <typename T>
inline cudaError_t trisolve_flow_launch(cudaStream_t st, int n, T *TE, int ld, const typename SrNum<T>::hp *dhp,
                                        const double *dlo, int *flags, int *work, const unsigned long long *plan,
                                        int ntasks, T *accb, int ldacc, int ctas, double cap = 0.0,
                                        const int *qblk = nullptr)
{
    const int NB = (n + kSolveTile - 1) / kSolveTile;
    cudaError_t e = cudaMemsetAsync(work, 0, (2 + 2 * (size_t)NB * NB) * sizeof(int), st);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)std::max(1, std::min(ctas, ntasks));
    if (qblk) {
        // the real Schur form (padded order, block array qblk)
        if constexpr (SrNum<T>::kind <= 1)
            trisolve_flow_kernel<T, false, true><<<grid, FlowShape<T>::NT, FlowShape<T>::smem, st>>>(
                n, TE, ld, dhp, dlo, flags, work, plan, ntasks, accb, ldacc, cap, nullptr, qblk);
        else
            return cudaErrorInvalidValue;
    } else {
        trisolve_flow_kernel<T><<<grid, FlowShape<T>::NT, FlowShape<T>::smem, st>>>(n, TE, ld, dhp, dlo, flags, work,
                                                                                  plan, ntasks, accb, ldacc, cap);
    }
    return cudaGetLastError();
}

// Opts the kernel into its shared memory and returns the CTAs that fit the
// device at once (the launch's grid); 0 on error.
template <typename T>
inline int trisolve_flow_setup(int dev)
{
    if (cudaFuncSetAttribute(trisolve_flow_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)FlowShape<T>::smem) != cudaSuccess)
        return 0;
    if constexpr (SrNum<T>::kind <= 1) {
        if (cudaFuncSetAttribute(trisolve_flow_kernel<T, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)FlowShape<T>::smem) != cudaSuccess)
            return 0;
    }

    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, trisolve_flow_kernel<T>, FlowShape<T>::NT,
                                                      FlowShape<T>::smem) != cudaSuccess)
        return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return std::max(1, per_sm) * sms;
}

}  // namespace sr
