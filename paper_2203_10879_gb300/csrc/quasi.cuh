// The real quasi-triangular Schur form (Sec. 3: real Schur decompositions,
// whose 2 x 2 diagonal blocks hold complex-conjugate pairs of eigenvalues).
//
// Blocks. Rows are taken from the top; rows k, k+1 form a 2 x 2 block when the
// 2 x 2 diagonal block of T^ there has non-real eigenvalues,
// (t_kk - t_k+1,k+1)^2 + 4 t_k,k+1 t_k+1,k < 0 (in FP64). blk[k] = 2 at a
// block's first row, 0 at its second, 1 for a 1 x 1 block. In a run of
// consecutive candidate rows s, s+1, ... the blocks start at s, s+2, ...
// (taken from the top), so a block start is a candidate at an even distance
// from the start of its run: one max-scan over the rows finds every run start.
//
// Equation. E is the part of T^ below the diagonal blocks and L the strictly
// block-lower solution of sbl(T L - L T) = -E. Each block entry (I, J) solves
// T_II X - X T_JJ = -C_IJ (sizes p x q, p, q <= 2) through its Kronecker
// matrix I (x) T_II - T_JJ^T (x) I (vec(X) column-major), whose diagonal
// entries t_rr - t_cc are formed from the FP64 diagonal and rounded once. The
// matrix is inverted by Gauss-Jordan elimination with partial pivoting in the
// working precision (a zero pivot is a shared eigenvalue) before the
// wavefront reaches the entry, and the inverse applied to -C_IJ when it does.
//
// Tiles. The tiled solver needs every block inside one 32 x 32 tile, so the
// problem is solved in a padded order n': where a 2 x 2 block would start on
// the last row of a tile, a dummy 1 x 1 row is inserted (its T row and
// column zero, E zero, a diagonal of 1e30 or more, distinct for each padding
// row), which decouples exactly: its L row and column come out zero. The host builds the padded layout from the block
// array (read back at the pass's synchronization). Inside a tile the
// wavefront finishes whole block entries: block entry (I, J) is final at step
// w = (first row of I) - (last column of J), the step of its last scalar
// entry, and its entries' pending sums take only contributions of block
// entries finished at earlier steps (an entry is never pending while a
// member of its own block finishes, so the couplings inside a block never
// enter a sum: they are in the Kronecker matrix).
#pragma once
#include <vector>

#include "trisolve.cuh"

namespace sr {

// Diagonal of padding row pi: kQuasiDummy (pi + 1), apart from every real
// diagonal entry and from each other (two padding rows with one diagonal would
// make their 1 x 1 block entry singular).
constexpr double kQuasiDummy = 1e30;

// One CTA of 1024 threads. sub[k] = T^(k+1, k), sup[k] = T^(k, k+1), d the
// diagonal (FP64). Writes blk[0..n). When norm is given, the squares of the
// subdiagonal entries that are not couplings of 2 x 2 blocks are added to
// *norm (a sum of squares below the subdiagonal).
__global__ void __launch_bounds__(1024, 1)
quasi_blocks_kernel(int n, const double *__restrict__ d, const double *__restrict__ sub,
                    const double *__restrict__ sup, int *__restrict__ blk, double *norm)
{
    __shared__ int smax[1024];
    __shared__ double ssum[32];
    const int per = (n + 1023) / 1024;
    const int k0 = threadIdx.x * per, k1 = min(n, k0 + per);
    auto cand = [&](int k) -> bool {
        if (k + 1 >= n) return false;
        const double a = d[k], b = sup[k], c = sub[k], e = d[k + 1];
        return (a - e) * (a - e) + 4.0 * b * c < 0.0;
    };
    // inclusive max-scan of (cand(k) ? 0 : k + 1): the first row of k's run of candidates
    int m = 0;
    for (int k = k0; k < k1; ++k)
        if (!cand(k)) m = k + 1;
    smax[threadIdx.x] = m;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int v = threadIdx.x >= off ? smax[threadIdx.x - off] : 0;
        __syncthreads();
        smax[threadIdx.x] = max(smax[threadIdx.x], v);
        __syncthreads();
    }
    int run = threadIdx.x > 0 ? smax[threadIdx.x - 1] : 0;
    double corr = 0.0;
    for (int k = k0; k < k1; ++k) {
        const bool ck = cand(k);
        if (!ck) run = k + 1;
        const bool start = ck && ((k - run) & 1) == 0;
        blk[k] = start ? 2 : 1;
        if (!start && k + 1 < n) corr += sub[k] * sub[k];
    }
    __syncthreads();
    // second rows: set after every start is written (a start's next row may
    // belong to another thread)
    for (int k = k0; k < k1; ++k)
        if (k > 0 && blk[k - 1] == 2) blk[k] = 0;
    if (norm) {
        for (int o = 16; o > 0; o >>= 1) corr += __shfl_down_sync(0xffffffffu, corr, o);
        if ((threadIdx.x & 31) == 0) ssum[threadIdx.x >> 5] = corr;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < 32; ++w) s += ssum[w];
            *norm += s;
        }
    }
}

// The band of T (sub- and superdiagonal) of a low-precision T, widened to FP64
template <typename T>
__global__ void quasi_band_kernel(int n, const T *__restrict__ TE, int ld, double *__restrict__ sub,
                                  double *__restrict__ sup)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k + 1 < n) {
        sub[k] = (double)TE[sr_idx(k + 1, k, ld)];
        sup[k] = (double)TE[sr_idx(k, k + 1, ld)];
    } else if (k < n) {
        sub[k] = sup[k] = 0.0;
    }
}

// Padded copy: entry (pi, pj) of the order-n' problem from original (inv[pi],
// inv[pj]), dummy rows and columns zero with the diagonal kQuasiDummy; the FP64
// diagonal likewise. The coupling t_k+1,k of each 2 x 2 block goes to cq[pk]
// (pk its first padded row) as well: the shared update kernel accumulates its
// products into every strictly lower entry of a diagonal tile, couplings
// included, so the leaf reads the couplings from cq.
template <typename T>
__global__ void quasi_pad_kernel(int np, const int *__restrict__ inv, const int *__restrict__ blkq,
                                 const T *__restrict__ TE, int ld, const double *__restrict__ d,
                                 T *__restrict__ TEq, int ldq, double *__restrict__ dq, T *__restrict__ cq)
{
    const int pi = blockIdx.x * 32 + (threadIdx.x & 31);
    const int pj0 = blockIdx.y * 32 + (threadIdx.x >> 5);
    if (pi >= np) return;
    const int i = inv[pi];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const int pj = pj0 + 8 * w;
        if (pj >= np) continue;
        const int j = inv[pj];
        T v = (T)0;
        if (i >= 0 && j >= 0) v = TE[sr_idx(i, j, ld)];
        else if (pi == pj) v = (T)(kQuasiDummy * (double)(pi + 1));
        TEq[sr_idx(pi, pj, ldq)] = v;
    }
    if (blockIdx.y == 0 && threadIdx.x < 32) {
        dq[pi] = i >= 0 ? d[i] : kQuasiDummy * (double)(pi + 1);
        cq[pi] = blkq[pi] == 2 ? TE[sr_idx(i + 1, i, ld)] : (T)0;   // a block's first row is never padding
    }
}

// Back from the padded order: below the diagonal, L at the block-lower entries
// and zero at the couplings of the 2 x 2 blocks (not unknowns); the upper
// triangle is left as it is.
template <typename T>
__global__ void quasi_unpad_kernel(int n, const int *__restrict__ pos, const int *__restrict__ blk,
                                   const T *__restrict__ TEq, int ldq, T *__restrict__ TE, int ld)
{
    const int i = blockIdx.x * 32 + (threadIdx.x & 31);
    const int j0 = blockIdx.y * 32 + (threadIdx.x >> 5);
    if (i >= n) return;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const int j = j0 + 8 * w;
        if (j >= n || j >= i) continue;
        const bool coupling = i == j + 1 && blk[j] == 2;
        TE[sr_idx(i, j, ld)] = coupling ? (T)0 : TEq[sr_idx(pos[i], pos[j], ldq)];
    }
}

// Solve of the tiles of subdiagonal t in the padded order (the stepwise form):
// 1024 threads, thread (lane a, warp b) owns entry (a, b) of the tile. Phase 1
// adds E and the two products of subdiagonal t + 1 (as trisolve_leaf_kernel).
// Phase 2 is the wavefront over block entries described at the top of this
// file. Each block entry's Kronecker matrix depends on T alone, so every
// thread of the entry inverts it before the wavefront and keeps its own row
// of the inverse; when the entry is final, each thread reads the entry's
// pending sums and forms its own unknown (a product of the row with -C).
template <typename T>
__global__ void __launch_bounds__(1024, 1)
trisolve_quasi_leaf_kernel(int n, T *__restrict__ TE, int ld, const double *__restrict__ dhp,
                           const int *__restrict__ blk, const T *__restrict__ cq, int t,
                           const uint32_t *__restrict__ plan, int *__restrict__ flags, double cap)
{
    constexpr int B = kSolveTile, S = B + 1;
    const T Z = (T)0;
    const uint32_t tile = plan[blockIdx.x];
    const int NB = (n + B - 1) / B;
    const int I = (int)(tile >> 16), J = (int)(tile & 0xffffu);
    const int D = I - J;
    const int r0 = I * B, c0 = J * B;
    const int nr = min(B, n - r0), nc = min(B, n - c0);
    const int d = t + 1;
    __shared__ T sm[4][B][S];
    T (*Ta)[B][S] = sm;
    T (*Tb)[B][S] = sm + 2;
    T (*X)[S] = sm[0];
    T (*Ti)[S] = sm[1];
    T (*Tj)[S] = sm[2];
    T (*Cs)[S] = sm[3];
    __shared__ double dI[B], dJ[B];
    __shared__ int rb[B], cb[B];
    const int a = threadIdx.x & 31, b = threadIdx.x >> 5;
    if (threadIdx.x < B) {
        rb[a] = a < nr ? blk[r0 + a] : 1;
        dI[a] = a < nr ? dhp[r0 + a] : 0.0;
    } else if (threadIdx.x < 2 * B) {
        const int c = threadIdx.x - B;
        cb[c] = c < nc ? blk[c0 + c] : 1;
        dJ[c] = c < nc ? dhp[c0 + c] : 0.0;
    }
    // 1. E plus the two products of subdiagonal t+1
    const bool hasP = d < NB && J + d < NB, hasM = d < NB && I - d >= 0;
    const int kP = (J + d) * B, kM = (I - d) * B;
    Ta[0][b][a] = (hasP && r0 + a < n && kP + b < n) ? TE[sr_idx(r0 + a, kP + b, ld)] : Z;
    Tb[0][a][b] = (hasP && kP + a < n && c0 + b < n) ? TE[sr_idx(kP + a, c0 + b, ld)] : Z;
    Ta[1][b][a] = (hasM && r0 + a < n && kM + b < n) ? TE[sr_idx(r0 + a, kM + b, ld)] : Z;
    Tb[1][a][b] = (hasM && kM + a < n && c0 + b < n) ? TE[sr_idx(kM + a, c0 + b, ld)] : Z;
    __syncthreads();
    const int ra = rb[a] == 0 ? a - 1 : a;          // first row of a's block
    const int cs = cb[b] == 0 ? b - 1 : b;          // first column of b's block
    const int cl = cb[b] == 2 ? b + 1 : b;          // last column of b's block
    const bool own = a < nr && b < nc && (D > 0 || ra > cs);
    T acc = own ? TE[sr_idx(r0 + a, c0 + b, ld)] : Z;
    if (hasP || hasM) {
#pragma unroll 8
        for (int k = 0; k < B; ++k) {
            acc = sr_fma(Ta[0][k][a], Tb[0][k][b], acc);
            acc = sr_fma(-Ta[1][k][a], Tb[1][k][b], acc);
        }
    }
    __syncthreads();
    // 2. the diagonal blocks' rows of T, with the couplings of 2 x 2 blocks from cq
    Ti[a][b] = (a < nr && b < nr) ? (a <= b ? TE[sr_idx(r0 + a, r0 + b, ld)]
                                            : (a == b + 1 && rb[b] == 2 ? cq[r0 + b] : Z)) : Z;
    Tj[a][b] = (a < nc && b < nc) ? (a <= b ? TE[sr_idx(c0 + a, c0 + b, ld)]
                                            : (a == b + 1 && cb[b] == 2 ? cq[c0 + b] : Z)) : Z;
    X[a][b] = Z;
    Cs[a][b] = Z;
    __syncthreads();
    const int fs = ra - cl;                          // step at which a's and b's block entry is final
    const int p = rb[ra] == 2 ? 2 : 1, q = cb[cs] == 2 ? 2 : 1, m = p * q;
    const int ru = a - ra, cu = b - cs, me = ru + cu * p;   // this entry's index in vec(X)
    int bad = 0;
    // T_II X - X T_JJ = -C through the Kronecker matrix, vec index r + c p; the
    // diagonal t_rr - t_cc formed in FP64 and rounded once
    T kinv[4] = {Z, Z, Z, Z};
    if (own) {
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
        if (!kron_inverse_row(K, me, kinv)) bad |= SR_FLAG_NONDISTINCT;
    }
    const int wlo = (D > 0) ? -(B - 1) : 1;
    T xv = Z;
    for (int w = B - 1; w >= wlo; --w) {
        const bool fin = own && fs == w;
        if (fin) Cs[a][b] = acc;
        __syncthreads();
        if (fin) {
            T x = Z;
#pragma unroll
            for (int v = 0; v < 4; ++v)
                if (v < m) x = sr_fma(kinv[v], -Cs[ra + v % p][cs + v / p], x);
            if (cap > 0.0 && fabs((double)x) > (double)(T)cap) x = Z;   // Example 4's trick
            if (!sr_finite(x)) bad |= SR_FLAG_NONFINITE;
            X[a][b] = x;
            xv = x;
        }
        __syncthreads();
        if (own && fs < w) {
            // the row block finished in column b starts at row s; the column
            // block finished in row a ends at column e
            const int s = w + cl;
            if (s >= 0 && s < nr && rb[s] != 0) {
                acc = sr_fma(Ti[a][s], X[s][b], acc);
                if (rb[s] == 2) acc = sr_fma(Ti[a][s + 1], X[s + 1][b], acc);
            }
            const int e = ra - w;
            if (e >= 0 && e < nc && cb[e] != 2) {
                if (cb[e] == 0) acc = sr_fma(-X[a][e - 1], Tj[e - 1][b], acc);
                acc = sr_fma(-X[a][e], Tj[e][b], acc);
            }
        }
    }
    if (bad) atomicOr(flags, bad);
    if (own) TE[sr_idx(r0 + a, c0 + b, ld)] = xv;
}

// The stepwise launch sequence for the padded problem (as trisolve_launches,
// with the quasi leaf kernel; the update kernel is shared: no block crosses a
// tile, so the products between tiles are the triangular form's).
template <typename T>
inline cudaError_t trisolve_quasi_launches(cudaStream_t st, cudaStream_t aux, cudaEvent_t ev0, cudaEvent_t ev1,
                                           int n, T *TE, int ld, const double *dhp, const int *blk, const T *cq,
                                           int *flags, const uint32_t *plan, const std::vector<long long> &offsets,
                                           double cap)
{
    const int NB = (n + kSolveTile - 1) / kSolveTile;
    cudaError_t e = cudaEventRecord(ev0, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev0, 0);
    for (int t = NB - 1; t >= 0 && e == cudaSuccess; --t) {
        const int l = NB - 1 - t;
        const long long nleaf = NB - t;
        const long long nupd = offsets[l + 1] - offsets[l] - nleaf;
        trisolve_quasi_leaf_kernel<T><<<(unsigned)nleaf, 1024, 0, st>>>(n, TE, ld, dhp, blk, cq, t,
                                                                       plan + offsets[l], flags, cap);
        if (nupd > 0)
            trisolve_update_kernel<T><<<(unsigned)nupd, UpdShape<T>::NT, 0, aux>>>(n, TE, ld, t, plan + offsets[l] + nleaf);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(ev0, st);
        if (e == cudaSuccess) e = cudaEventRecord(ev1, aux);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev1, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev0, 0);
    }
    return e;
}

// Host: the padded layout of a block array. pos[k]: padded index of row k;
// inv[pi]: original row of padded row pi, -1 for a padding row; blkq: the
// padded block array. Returns the padded order.
inline int quasi_pad_layout(int n, const int *blk, std::vector<int> &pos, std::vector<int> &inv, std::vector<int> &blkq)
{
    pos.assign(n, 0);
    inv.clear();
    blkq.clear();
    for (int k = 0; k < n;) {
        if (blk[k] == 2 && k + 1 < n) {
            if ((int)inv.size() % kSolveTile == kSolveTile - 1) {   // the block would straddle a tile
                inv.push_back(-1);
                blkq.push_back(1);
            }
            pos[k] = (int)inv.size();
            inv.push_back(k);
            blkq.push_back(2);
            pos[k + 1] = (int)inv.size();
            inv.push_back(k + 1);
            blkq.push_back(0);
            k += 2;
        } else {
            pos[k] = (int)inv.size();
            inv.push_back(k);
            blkq.push_back(1);
            k += 1;
        }
    }
    return (int)inv.size();
}

}  // namespace sr
