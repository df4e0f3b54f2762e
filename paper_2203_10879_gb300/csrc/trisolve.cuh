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
//   trisolve_update_kernel  one CTA of 256 threads per tile with D < t that
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

template <typename T>
__device__ inline T sr_div_round(double di, double dj) { return (T)(di - dj); }

// Launch plan: for step t, the tiles (I << 16 | J) of subdiagonal t (solved)
// followed by the tiles with D < t that receive a product of subdiagonal t+1.
void trisolve_plan(int n, std::vector<uint32_t> &tiles, std::vector<long long> &offsets);

// ---- contributions of subdiagonal t+1 to tiles with D < t --------------------
// 2 x 2 register blocks: thread (tx, ty) owns rows 2tx, 2tx+1 and columns 2ty, 2ty+1.
template <typename T>
__global__ void __launch_bounds__(256)
trisolve_update_kernel(int n, T *__restrict__ TE, int ld, int t, const uint32_t *__restrict__ plan)
{
    constexpr int B = kSolveTile, S = B + 2;
    const int NB = (n + B - 1) / B;
    const uint32_t tile = plan[blockIdx.x];
    const int I = (int)(tile >> 16), J = (int)(tile & 0xffffu);
    const int D = I - J;
    const int r0 = I * B, c0 = J * B;
    const int nr = min(B, n - r0), nc = min(B, n - c0);
    const int d = t + 1;
    __shared__ __align__(16) T Ta[2][B][S];   // left operands, transposed: Ta[u][k][row]
    __shared__ __align__(16) T Tb[2][B][S];   // right operands: Tb[u][k][col]
    const int tid = threadIdx.x;
    const int lx = tid & 31, ly = tid >> 5;   // load mapping: element (lx, ly + 8q)
    const int tx = tid & 15, ty = tid >> 4;
    const bool hasP = J + d < NB, hasM = I - d >= 0;
    const int kP = (J + d) * B, kM = (I - d) * B;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int y = ly + 8 * q;
        Ta[0][y][lx] = (hasP && r0 + lx < n && kP + y < n) ? TE[sr_idx(r0 + lx, kP + y, ld)] : (T)0;
        Tb[0][lx][y] = (hasP && kP + lx < n && c0 + y < n) ? TE[sr_idx(kP + lx, c0 + y, ld)] : (T)0;
        Ta[1][y][lx] = (hasM && r0 + lx < n && kM + y < n) ? TE[sr_idx(r0 + lx, kM + y, ld)] : (T)0;
        Tb[1][lx][y] = (hasM && kM + lx < n && c0 + y < n) ? TE[sr_idx(kM + lx, c0 + y, ld)] : (T)0;
    }
    T acc[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int x = 2 * tx + i, y = 2 * ty + j;
            acc[i][j] = (x < nr && y < nc && (D > 0 || x > y)) ? TE[sr_idx(r0 + x, c0 + y, ld)] : (T)0;
        }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < B; ++k) {
        const T a0 = Ta[0][k][2 * tx], a1 = Ta[0][k][2 * tx + 1];
        const T b0 = Tb[0][k][2 * ty], b1 = Tb[0][k][2 * ty + 1];
        const T m0 = Ta[1][k][2 * tx], m1 = Ta[1][k][2 * tx + 1];
        const T n0 = Tb[1][k][2 * ty], n1 = Tb[1][k][2 * ty + 1];
        acc[0][0] = fma(a0, b0, acc[0][0]);
        acc[0][1] = fma(a0, b1, acc[0][1]);
        acc[1][0] = fma(a1, b0, acc[1][0]);
        acc[1][1] = fma(a1, b1, acc[1][1]);
        acc[0][0] = fma(-m0, n0, acc[0][0]);
        acc[0][1] = fma(-m0, n1, acc[0][1]);
        acc[1][0] = fma(-m1, n0, acc[1][0]);
        acc[1][1] = fma(-m1, n1, acc[1][1]);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int x = 2 * tx + i, y = 2 * ty + j;
            if (x < nr && y < nc && (D > 0 || x > y)) TE[sr_idx(r0 + x, c0 + y, ld)] = acc[i][j];
        }
}

// ---- solve of the tiles of subdiagonal t ---------------------------------------
// 1024 threads; thread (lane a, warp b) owns entry (a, b) of the tile.
template <typename T>
__global__ void __launch_bounds__(1024)
trisolve_leaf_kernel(int n, T *__restrict__ TE, int ld, const double *__restrict__ dhp, int t,
                     const uint32_t *__restrict__ plan, int *__restrict__ flags)
{
    constexpr int B = kSolveTile, S = B + 1;
    const int NB = (n + B - 1) / B;
    const uint32_t tile = plan[blockIdx.x];
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
    __shared__ double dI[B], dJ[B];
    const int a = threadIdx.x & 31, b = threadIdx.x >> 5;
    const bool own = a < nr && b < nc && (D > 0 || a > b);

    // 1. E plus the two products of subdiagonal t+1
    const bool hasP = d < NB && J + d < NB, hasM = d < NB && I - d >= 0;
    const int kP = (J + d) * B, kM = (I - d) * B;
    Ta[0][b][a] = (hasP && r0 + a < n && kP + b < n) ? TE[sr_idx(r0 + a, kP + b, ld)] : (T)0;
    Tb[0][a][b] = (hasP && kP + a < n && c0 + b < n) ? TE[sr_idx(kP + a, c0 + b, ld)] : (T)0;
    Ta[1][b][a] = (hasM && r0 + a < n && kM + b < n) ? TE[sr_idx(r0 + a, kM + b, ld)] : (T)0;
    Tb[1][a][b] = (hasM && kM + a < n && c0 + b < n) ? TE[sr_idx(kM + a, c0 + b, ld)] : (T)0;
    T acc = own ? TE[sr_idx(r0 + a, c0 + b, ld)] : (T)0;
    if (threadIdx.x < B) dI[threadIdx.x] = (threadIdx.x < nr) ? dhp[r0 + threadIdx.x] : 0.0;
    else if (threadIdx.x < 2 * B) dJ[threadIdx.x - B] = (threadIdx.x - B < nc) ? dhp[c0 + threadIdx.x - B] : 0.0;
    __syncthreads();
    if (hasP || hasM) {
#pragma unroll 8
        for (int k = 0; k < B; ++k) {
            acc = fma(Ta[0][k][a], Tb[0][k][b], acc);
            acc = fma(-Ta[1][k][a], Tb[1][k][b], acc);
        }
    }
    const T den = own ? sr_div_round<T>(dI[a], dJ[b]) : (T)1;
    __syncthreads();

    // 2. wavefront over the tile's subdiagonals. When subdiagonal w is final, a
    // pending entry (a, b) adds T_II(a, b+w) X(b+w, b) (from lane b+w of its
    // own warp) and -X(a, a-w) T_JJ(a-w, b) (from shared memory).
    Ti[a][b] = (a <= b && a < nr && b < nr) ? TE[sr_idx(r0 + a, r0 + b, ld)] : (T)0;
    Tj[a][b] = (a <= b && a < nc && b < nc) ? TE[sr_idx(c0 + a, c0 + b, ld)] : (T)0;
    X[a][b] = (T)0;
    __syncthreads();
    const int wlo = (D > 0) ? -(B - 1) : 1;
    T xv = (T)0;
    int bad = 0;
    for (int w = B - 1; w >= wlo; --w) {
        if (own && a - b == w) {
            if (den == (T)0) {
                bad |= SR_FLAG_NONDISTINCT;
            } else {
                xv = -acc / den;
                if (!sr_finite(xv)) bad |= SR_FLAG_NONFINITE;
            }
            X[a][b] = xv;
        }
        __syncthreads();
        const int c = b + w;                         // (c, b): lane c of this warp
        const T xcol = __shfl_sync(0xffffffffu, xv, c & 31);
        if (own && a - b < w) {
            if (c < nr) acc = fma(Ti[a][c], xcol, acc);
            const int c2 = a - w;                    // (a, c2), c2 < b
            if (c2 >= 0) acc = fma(-X[a][c2], Tj[c2][b], acc);
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
                                     T *TE, int ld, const double *dhp, int *flags, const uint32_t *plan,
                                     const std::vector<long long> &offsets)
{
    const int NB = (n + kSolveTile - 1) / kSolveTile;
    cudaError_t e = cudaEventRecord(ev0, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev0, 0);
    for (int t = NB - 1; t >= 0 && e == cudaSuccess; --t) {
        const int l = NB - 1 - t;
        const long long nleaf = NB - t;
        const long long nupd = offsets[l + 1] - offsets[l] - nleaf;
        trisolve_leaf_kernel<T><<<(unsigned)nleaf, 1024, 0, st>>>(n, TE, ld, dhp, t, plan + offsets[l], flags);
        if (nupd > 0)
            trisolve_update_kernel<T><<<(unsigned)nupd, 256, 0, aux>>>(n, TE, ld, t, plan + offsets[l] + nleaf);
        e = cudaGetLastError();
        // both kernels of this step finish before either of the next starts
        if (e == cudaSuccess) e = cudaEventRecord(ev0, st);
        if (e == cudaSuccess) e = cudaEventRecord(ev1, aux);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev1, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev0, 0);
    }
    return e;
}

}  // namespace sr
