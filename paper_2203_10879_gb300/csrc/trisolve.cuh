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
#include <vector>

#include "common.cuh"

namespace sr {

constexpr int kSolveTile = 32;

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
void trisolve_plan(int n, std::vector<uint32_t> &tiles, std::vector<long long> &offsets);

// A group of independent solves in the same launches (schur_refine_batched):
// matrix b of the group, and its tiles in the plan as (b << 32 | I << 16 | J).
struct SolveMat {
    void *TE;
    int ld, n;
    const void *dhp;
};

// Group plan: for every step t (from the largest order's last subdiagonal
// down), the leaf tiles of all matrices with more than t block rows, then
// their update tiles; leaf[t] and upd[t] give the counts.
void trisolve_plan_group(const std::vector<int> &orders, std::vector<unsigned long long> &tiles,
                         std::vector<long long> &offsets, std::vector<long long> &nleaf);

// ---- contributions of subdiagonal t+1 to tiles with D < t --------------------
// Thread (tx, ty) owns the 4 x TN block rows 4tx.., columns TN*ty.., read with
// vector loads from shared memory: TN = 4 (64 threads, 4 vector loads per 32
// FMAs; shared-memory bandwidth bounds the FP32 update) except for FP64, whose
// update is bound by the FP64 pipe and keeps TN = 2 with 128 threads for more
// warps in flight.
template <typename T> struct UpdShape {
    static constexpr int TN = SrNum<T>::kind == 1 ? 2 : 4;
    static constexpr int NT = 8 * (32 / TN);
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

template <typename T, bool GROUP = false>
__global__ void __launch_bounds__(UpdShape<T>::NT)
trisolve_update_kernel(int n, T *__restrict__ TE, int ld, int t, const uint32_t *__restrict__ plan,
                       const SolveMat *__restrict__ mats = nullptr,
                       const unsigned long long *__restrict__ gplan = nullptr)
{
    constexpr int B = kSolveTile, SA = B + 4, SB = B + 4;
    uint32_t tile;
    if constexpr (GROUP) {
        const unsigned long long g = gplan[blockIdx.x];
        const SolveMat m = mats[g >> 32];
        TE = (T *)m.TE;
        ld = m.ld;
        n = m.n;
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
    constexpr int TN = UpdShape<T>::TN, NT = UpdShape<T>::NT, LR = NT / 32;
    const int tid = threadIdx.x;
    const int lx = tid & 31, ly = tid >> 5;   // load mapping: element (lx, ly + LR q)
    const int tx = tid & 7, ty = tid >> 3;    // block rows 4tx.., columns TN ty..
    const T Z = SrNum<T>::zero();
    const bool hasP = J + d < NB, hasM = I - d >= 0;
    const int kP = (J + d) * B, kM = (I - d) * B;
#pragma unroll
    for (int q = 0; q < 32 / LR; ++q) {
        const int y = ly + LR * q;
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
            acc[i][j] = (x < nr && y < nc && (D > 0 || x > y)) ? TE[sr_idx(r0 + x, c0 + y, ld)] : Z;
        }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < B; ++k) {
        T a[4], b[TN], m[4], c[TN];
        SolveVec<T>::ld4(&Ta[0][k][4 * tx], a);
        SolveVec<T>::ld4(&Ta[1][k][4 * tx], m);
        if constexpr (TN == 4) {
            SolveVec<T>::ld4(&Tb[0][k][4 * ty], b);
            SolveVec<T>::ld4(&Tb[1][k][4 * ty], c);
        } else {
            SolveVec<T>::ld2(&Tb[0][k][2 * ty], b);
            SolveVec<T>::ld2(&Tb[1][k][2 * ty], c);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                acc[i][j] = sr_fma(a[i], b[j], acc[i][j]);
                acc[i][j] = sr_fma(-m[i], c[j], acc[i][j]);
            }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int x = 4 * tx + i, y = TN * ty + j;
            if (x < nr && y < nc && (D > 0 || x > y)) TE[sr_idx(r0 + x, c0 + y, ld)] = acc[i][j];
        }
}

// ---- solve of the tiles of subdiagonal t ---------------------------------------
// 1024 threads; thread (lane a, warp b) owns entry (a, b) of the tile.
template <typename T, bool GROUP = false>
__global__ void __launch_bounds__(1024)
trisolve_leaf_kernel(int n, T *__restrict__ TE, int ld, const typename SrNum<T>::hp *__restrict__ dhp,
                     const double *__restrict__ dlo, int t, const uint32_t *__restrict__ plan, int *__restrict__ flags,
                     const SolveMat *__restrict__ mats = nullptr,
                     const unsigned long long *__restrict__ gplan = nullptr)
{
    using Hp = typename SrNum<T>::hp;
    constexpr int B = kSolveTile, S = B + 1;
    const T Z = SrNum<T>::zero();
    uint32_t tile;
    if constexpr (GROUP) {
        // a group: each matrix has its own flag word
        const unsigned long long g = gplan[blockIdx.x];
        const SolveMat m = mats[g >> 32];
        TE = (T *)m.TE;
        ld = m.ld;
        n = m.n;
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
    const int a = threadIdx.x & 31, b = threadIdx.x >> 5;
    const bool own = a < nr && b < nc && (D > 0 || a > b);

    // 1. E plus the two products of subdiagonal t+1
    const bool hasP = d < NB && J + d < NB, hasM = d < NB && I - d >= 0;
    const int kP = (J + d) * B, kM = (I - d) * B;
    Ta[0][b][a] = (hasP && r0 + a < n && kP + b < n) ? TE[sr_idx(r0 + a, kP + b, ld)] : Z;
    Tb[0][a][b] = (hasP && kP + a < n && c0 + b < n) ? TE[sr_idx(kP + a, c0 + b, ld)] : Z;
    Ta[1][b][a] = (hasM && r0 + a < n && kM + b < n) ? TE[sr_idx(r0 + a, kM + b, ld)] : Z;
    Tb[1][a][b] = (hasM && kM + a < n && c0 + b < n) ? TE[sr_idx(kM + a, c0 + b, ld)] : Z;
    T acc = own ? TE[sr_idx(r0 + a, c0 + b, ld)] : Z;
    const Hp hz = SrNum<Hp>::zero();
    if (threadIdx.x < B) {
        dI[threadIdx.x] = (threadIdx.x < nr) ? dhp[r0 + threadIdx.x] : hz;
        dIl[threadIdx.x] = (dlo && threadIdx.x < nr) ? dlo[r0 + threadIdx.x] : 0.0;
    } else if (threadIdx.x < 2 * B) {
        dJ[threadIdx.x - B] = (threadIdx.x - B < nc) ? dhp[c0 + threadIdx.x - B] : hz;
        dJl[threadIdx.x - B] = (dlo && threadIdx.x - B < nc) ? dlo[c0 + threadIdx.x - B] : 0.0;
    }
    __syncthreads();
    if (hasP || hasM) {
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
    // pending entry (a, b) adds T_II(a, b+w) X(b+w, b) (from lane b+w of its
    // own warp) and -X(a, a-w) T_JJ(a-w, b) (from shared memory).
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
                if (!sr_finite(xv)) bad |= SR_FLAG_NONFINITE;
            }
            X[a][b] = xv;
        }
        __syncthreads();
        const int c = b + w;                         // (c, b): lane c of this warp
        const T xcol = sr_shfl(xv, c & 31);
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
// plan: device copy of trisolve_plan's tiles; offsets: its host offsets.
template <typename T>
inline cudaError_t trisolve_launches(cudaStream_t st, cudaStream_t aux, cudaEvent_t ev0, cudaEvent_t ev1, int n,
                                     T *TE, int ld, const typename SrNum<T>::hp *dhp, const double *dlo,
                                     int *flags, const uint32_t *plan, const std::vector<long long> &offsets)
{
    const int NB = (n + kSolveTile - 1) / kSolveTile;
    cudaError_t e = cudaEventRecord(ev0, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev0, 0);
    for (int t = NB - 1; t >= 0 && e == cudaSuccess; --t) {
        const int l = NB - 1 - t;
        const long long nleaf = NB - t;
        const long long nupd = offsets[l + 1] - offsets[l] - nleaf;
        trisolve_leaf_kernel<T><<<(unsigned)nleaf, 1024, 0, st>>>(n, TE, ld, dhp, dlo, t, plan + offsets[l], flags);
        if (nupd > 0)
            trisolve_update_kernel<T><<<(unsigned)nupd, UpdShape<T>::NT, 0, aux>>>(n, TE, ld, t, plan + offsets[l] + nleaf);
        e = cudaGetLastError();
        // both kernels of this step finish before either of the next starts
        if (e == cudaSuccess) e = cudaEventRecord(ev0, st);
        if (e == cudaSuccess) e = cudaEventRecord(ev1, aux);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev1, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev0, 0);
    }
    return e;
}

// The launches of a group plan (no double-double divisors): the same two-stream
// sequence as trisolve_launches, steps t = nsteps-1 .. 0.
template <typename T>
inline cudaError_t trisolve_launches_group(cudaStream_t st, cudaStream_t aux, cudaEvent_t ev0, cudaEvent_t ev1,
                                           const SolveMat *mats, int *flags, const unsigned long long *plan,
                                           const std::vector<long long> &offsets, const std::vector<long long> &nleaf)
{
    const int nsteps = (int)nleaf.size();
    cudaError_t e = cudaEventRecord(ev0, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev0, 0);
    for (int l = 0; l < nsteps && e == cudaSuccess; ++l) {
        const int t = nsteps - 1 - l;
        const long long nl = nleaf[l];
        const long long nupd = offsets[l + 1] - offsets[l] - nl;
        if (nl > 0)
            trisolve_leaf_kernel<T, true><<<(unsigned)nl, 1024, 0, st>>>(0, nullptr, 0, nullptr, nullptr, t, nullptr,
                                                                        flags, mats, plan + offsets[l]);
        if (nupd > 0)
            trisolve_update_kernel<T, true><<<(unsigned)nupd, UpdShape<T>::NT, 0, aux>>>(0, nullptr, 0, t, nullptr, mats,
                                                                                    plan + offsets[l] + nl);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(ev0, st);
        if (e == cudaSuccess) e = cudaEventRecord(ev1, aux);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev1, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev0, 0);
    }
    return e;
}

}  // namespace sr
