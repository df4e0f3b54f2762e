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
// The matrix is cut into B x B tiles. Tile (I, J), I >= J, depends on tiles
// (K, J), K > I, and (I, K), K < J, so tiles on block subdiagonal D = I - J are
// independent of each other given all tiles with D' > D. One launch handles one
// block subdiagonal, from the bottom-left corner (D = NB - 1) to the diagonal
// (D = 0). Inside a launch each CTA owns one tile and
//   1. accumulates C = E_IJ + sum_{K>I} T_IK L_KJ - sum_{K<J} L_IK T_KJ
//      (the block form of Alg. 3's two update products, applied left-looking),
//   2. solves the tile equation T_II X - X T_JJ = -C (eq. "l21", a triangular
//      Sylvester equation) -- or its stril form when I = J -- by a wavefront
//      over the tile's own subdiagonals a - b = B-1, ..., -(B-1).
// Divisors t_ii - t_jj are formed in FP64 from the high-precision diagonal and
// then rounded to the working type (the paper is silent here).
#pragma once
#include "common.cuh"

namespace sr {

constexpr int kSolveTile = 32;
constexpr int kSolveThreads = 256;

template <typename T>
__device__ inline T sr_div_round(double di, double dj) { return (T)(di - dj); }

template <typename T>
__global__ void __launch_bounds__(kSolveThreads)
trisolve_wavefront_kernel(int n, T *__restrict__ TE, int ld, const double *__restrict__ dhp, int D,
                          int *__restrict__ flags)
{
    constexpr int B = kSolveTile;
    const int NB = (n + B - 1) / B;
    const int I = D + blockIdx.x;
    const int J = I - D;
    const int r0 = I * B, c0 = J * B;
    const int nr = min(B, n - r0), nc = min(B, n - c0);

    __shared__ T C[B][B + 1];
    __shared__ T Ta[B][B + 1];
    __shared__ T Tb[B][B + 1];

    const int tid = threadIdx.x;
    const int x = tid & 31, y0 = tid >> 5;   // element (x, y0 + 8q), q = 0..3

    T acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int y = y0 + 8 * q;
        const bool in = x < nr && y < nc && (D > 0 || x > y);
        acc[q] = in ? TE[sr_idx(r0 + x, c0 + y, ld)] : (T)0;
    }

    // --- 1. left-looking accumulation over the finished tiles ------------------
    // Phase 0: K = I+1..NB-1, acc += T(I,K) L(K,J).   Phase 1: K = 0..J-1, acc -= L(I,K) T(K,J).
    const int n0 = NB - 1 - I, n1 = J;
    const int ntot = n0 + n1;
    T ra[4], rb[4];
    auto fetch = [&](int s) {
        const int K = (s < n0) ? (I + 1 + s) : (s - n0);
        const int k0 = K * B;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int y = y0 + 8 * q;
            // left operand tile rows r0.., cols k0..; right operand rows k0.., cols c0..
            ra[q] = (r0 + x < n && k0 + y < n) ? TE[sr_idx(r0 + x, k0 + y, ld)] : (T)0;
            rb[q] = (k0 + x < n && c0 + y < n) ? TE[sr_idx(k0 + x, c0 + y, ld)] : (T)0;
        }
    };
    if (ntot > 0) fetch(0);
    for (int s = 0; s < ntot; ++s) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            Ta[x][y0 + 8 * q] = ra[q];
            Tb[x][y0 + 8 * q] = rb[q];
        }
        __syncthreads();
        if (s + 1 < ntot) fetch(s + 1);
        T part[4] = {(T)0, (T)0, (T)0, (T)0};
#pragma unroll 8
        for (int c = 0; c < B; ++c) {
            const T a = Ta[x][c];
#pragma unroll
            for (int q = 0; q < 4; ++q) part[q] = fma(a, Tb[c][y0 + 8 * q], part[q]);
        }
        if (s < n0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += part[q];
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] -= part[q];
        }
        __syncthreads();
    }

    // --- 2. tile solve ----------------------------------------------------------
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int y = y0 + 8 * q;
        C[x][y] = (x < nr && y < nc && (D > 0 || x > y)) ? acc[q] : (T)0;
        // Ta = T_II, Tb = T_JJ (upper triangles with diagonal)
        Ta[x][y] = (x <= y && x < nr && y < nr) ? TE[sr_idx(r0 + x, r0 + y, ld)] : (T)0;
        Tb[x][y] = (x <= y && x < nc && y < nc) ? TE[sr_idx(c0 + x, c0 + y, ld)] : (T)0;
    }
    __syncthreads();

    const int g = tid >> 3, lane = tid & 7;   // 32 groups of 8 lanes, one entry per group
    const int wlo = (D > 0) ? -(B - 1) : 1;
    int bad = 0;
    for (int w = B - 1; w >= wlo; --w) {
        const int a = g + (w > 0 ? w : 0);
        const int b = a - w;
        const bool active = a < nr && b >= 0 && b < nc && a < B;
        T s = (T)0;
        if (active) {
            for (int c = a + 1 + lane; c < nr; c += 8) s = fma(Ta[a][c], C[c][b], s);
            for (int c = lane; c < b; c += 8) s = fma(-C[a][c], Tb[c][b], s);
        }
        s += __shfl_xor_sync(0xffffffffu, s, 4);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        if (active && lane == 0) {
            const T den = sr_div_round<T>(dhp[r0 + a], dhp[c0 + b]);
            const T v = C[a][b] + s;
            if (den == (T)0) {
                bad |= SR_FLAG_NONDISTINCT;
                C[a][b] = (T)0;
            } else {
                const T l = -v / den;
                if (!sr_finite(l)) bad |= SR_FLAG_NONFINITE;
                C[a][b] = l;
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(flags, bad);

#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int y = y0 + 8 * q;
        if (x < nr && y < nc && (D > 0 || x > y)) TE[sr_idx(r0 + x, c0 + y, ld)] = C[x][y];
    }
}

template <typename T>
inline cudaError_t trisolve_wavefront(cudaStream_t st, int n, T *TE, int ld, const double *dhp, int *flags)
{
    const int NB = (n + kSolveTile - 1) / kSolveTile;
    for (int D = NB - 1; D >= 0; --D) {
        trisolve_wavefront_kernel<T><<<NB - D, kSolveThreads, 0, st>>>(n, TE, ld, dhp, D, flags);
    }
    return cudaGetLastError();
}

}  // namespace sr
