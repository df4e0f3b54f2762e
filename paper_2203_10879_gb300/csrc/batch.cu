// schur_refine_batched with grouped launches: the independent refinements of
// a group of matrices (orders up to the handle's maximum) advance pass by pass
// together, and every stage of a pass -- each split, slice product, combine,
// the solve's steps, the elementwise kernels -- is one launch for all matrices
// that are still iterating. A pass costs about as many launches as the pass of
// one matrix, whatever the group's size.
//
// Layout: matrix b's FP64/FP32 buffers are compact (leading dimension n_b) at
// element offset o_b = sum_{b' < b} n_b'^2 of each workspace array; its
// vectors are rows [row0_b, row0_b + n_b) of every digit slot, row0_b a
// multiple of 32; its level planes are a region of round32(n_b)^2 elements.
// Work-item lists, split and combine descriptors and the per-matrix epilogues
// are rebuilt on the host for the matrices still active at the start of each
// pass and uploaded in one copy.
//
// Built for the mixed form with emulated products (real data, FP64 target,
// FP32 low precision): see sr_batch_supported.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ctx.cuh"
#include "kernels_misc.cuh"
#include "ozaki.cuh"
#include "trisolve.cuh"

namespace {

constexpr int kHp = sr::kOzakiDefaultSlices;   // digits of the FP64 products
constexpr int kLp = sr::kOzakiLpSlices;        // digits of the FP32-class products
constexpr int kNorms = 4;                      // per matrix: ||E||^2, ||Y||^2, ||A||^2, spare

inline int r32(int n) { return (n + 31) / 32 * 32; }

// ---- grouped elementwise kernels (blockIdx.z = matrix) -------------------------------

struct GMat {          // one matrix of a group: compact buffers at offset off
    long long off;
    int n;
    int ld_in;         // leading dimension of the caller's matrices
    const void *in0;   // caller input (A or Qhat)
    void *out0;        // caller output (Q)
};

// The elementwise kernels below run on one flat grid of 32 x 32 tiles over
// all matrices of a launch: matrix a owns blocks [start[a], start[a + 1]),
// row-major over its ceil(n/32) x ceil(n/32) tiles; thread (tx, ty) covers
// rows bx*32 + tx, columns by*32 + ty + 8w (w < 4).
struct Tile32 {
    int a, i, j0;
};
__device__ __forceinline__ Tile32 tile32(const int *__restrict__ start, int m, const GMat *__restrict__ mats)
{
    const int a = sr::group_find(start, m, blockIdx.x);
    const int local = blockIdx.x - start[a], g = (mats[a].n + 31) / 32;
    return {a, (local % g) * 32 + (int)(threadIdx.x & 31), (local / g) * 32 + (int)(threadIdx.x >> 5)};
}

// Q (FP64, workspace) <- Qhat (FP32, caller)
__global__ void __launch_bounds__(256) group_convert_kernel(const GMat *__restrict__ mats, const int *__restrict__ start,
                                                           int cnt, double *__restrict__ Q)
{
    const Tile32 t = tile32(start, cnt, mats);
    const GMat m = mats[t.a];
    for (int w = 0; w < 4; ++w) {
        const int j = t.j0 + 8 * w;
        if (t.i < m.n && j < m.n)
            Q[m.off + sr_idx(t.i, j, m.n)] = (double)((const float *)m.in0)[sr_idx(t.i, j, m.ld_in)];
    }
}

// caller Q (out0, ld_in) <- workspace Q (in0, compact)
__global__ void __launch_bounds__(256) group_copy_out_kernel(const GMat *__restrict__ mats,
                                                            const int *__restrict__ start, int cnt)
{
    const Tile32 t = tile32(start, cnt, mats);
    const GMat m = mats[t.a];
    for (int w = 0; w < 4; ++w) {
        const int j = t.j0 + 8 * w;
        if (t.i < m.n && j < m.n)
            ((double *)m.out0)[sr_idx(t.i, j, m.ld_in)] = ((const double *)m.in0)[sr_idx(t.i, j, m.n)];
    }
}

// W = L - L^T (FP64) from the strictly lower triangle of TE (FP32)
__global__ void __launch_bounds__(256) group_skew_kernel(const GMat *__restrict__ mats, const int *__restrict__ start,
                                                        int cnt, const float *__restrict__ TE, double *__restrict__ W)
{
    const Tile32 t = tile32(start, cnt, mats);
    const GMat m = mats[t.a];
    const float *L = TE + m.off;
    for (int w = 0; w < 4; ++w) {
        const int i = t.i, j = t.j0 + 8 * w;
        if (i < m.n && j < m.n) {
            const double v = i > j ? (double)L[sr_idx(i, j, m.n)] : (i < j ? -(double)L[sr_idx(j, i, m.n)] : 0.0);
            W[m.off + sr_idx(i, j, m.n)] = v;
        }
    }
}

// partial[block] = sum of squares of the block's tile of the caller's A
__global__ void __launch_bounds__(256) group_sumsq_kernel(const GMat *__restrict__ mats, const int *__restrict__ start,
                                                         int cnt, double *__restrict__ partial)
{
    const Tile32 t = tile32(start, cnt, mats);
    const GMat m = mats[t.a];
    double s = 0.0;
    for (int w = 0; w < 4; ++w) {
        const int j = t.j0 + 8 * w;
        if (t.i < m.n && j < m.n) {
            const double v = ((const double *)m.in0)[sr_idx(t.i, j, m.ld_in)];
            s += v * v;
        }
    }
    s = sr_block_sum<256>(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// out[map[a] * stride + slot] = sum of partial[start[a] .. start[a + 1]) in a
// fixed order; a = position in the launch, map[a] = matrix of the group
__global__ void __launch_bounds__(256) group_reduce_kernel(const double *__restrict__ partial,
                                                          const int *__restrict__ start, const int *__restrict__ map,
                                                          double *__restrict__ out, int stride, int slot)
{
    double s = 0.0;
    for (int e = start[blockIdx.x] + threadIdx.x; e < start[blockIdx.x + 1]; e += 256) s += partial[e];
    s = sr_block_sum<256>(s);
    if (threadIdx.x == 0) out[(size_t)map[blockIdx.x] * stride + slot] = s;
}

}  // namespace

struct BatchWork {
    long long cap_elems = 0;   // capacity of the compact buffers (elements)
    int cap_rows = 0, cap_count = 0, cap_k = 0;
    long long cap_planes = 0;
    double *Q0 = nullptr, *Q1 = nullptr, *AQ = nullptr, *Y = nullptr, *Delta = nullptr, *W = nullptr,
           *W2 = nullptr, *YW = nullptr, *diag = nullptr;
    float *TE = nullptr;
    float *acc = nullptr;      // stepwise group solve: far products' sums, apart from E (as TE)
    double *partial = nullptr;
    size_t npartial = 0;
    double *norms = nullptr;   // [count][kNorms]
    int *flags = nullptr;      // [count]
    sr::OzakiWork oz{};
    // descriptors: one pinned host buffer and its device copy
    unsigned char *hdesc = nullptr, *ddesc = nullptr;
    size_t desc_cap = 0;
    double *hnorms = nullptr;  // pinned mirror of norms + flags
    size_t hnorms_cap = 0;
    cudaStream_t aux = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // dataflow solve of the group: ticket, abort and published words; its grid
    int *flow = nullptr;
    size_t flow_cap = 0;
    int flow_ctas = 0;
    int crt = -1;              // the high-precision slots hold residues (1) or digits (0)
};

void sr_batch_free(BatchWork *bw)
{
    if (!bw) return;
    double *bufs[] = {bw->Q0, bw->Q1, bw->AQ, bw->Y, bw->Delta, bw->W, bw->W2, bw->YW, bw->diag, bw->partial,
                      bw->norms};
    for (double *p : bufs) cudaFree(p);
    cudaFree(bw->TE);
    cudaFree(bw->acc);
    cudaFree(bw->flags);
    cudaFree(bw->flow);
    cudaFree(bw->ddesc);
    if (bw->hdesc) cudaFreeHost(bw->hdesc);
    if (bw->hnorms) cudaFreeHost(bw->hnorms);
    sr::ozaki_free(bw->oz);
    if (bw->aux) cudaStreamDestroy(bw->aux);
    if (bw->ev0) cudaEventDestroy(bw->ev0);
    if (bw->ev1) cudaEventDestroy(bw->ev1);
    delete bw;
}

bool sr_batch_supported(const sr_options &o)
{
    const bool crt = o.hp_gemm == SR_HP_OZAKI_CRT;
    return o.dtype == SR_REAL && o.target == SR_TARGET_FP64 && (o.hp_gemm == SR_HP_OZAKI_BF16 || crt) &&
           o.lp == SR_LP_FP32 && o.qhat_type == SR_QHAT_FP32 && !o.full_sigma && sr::kOzakiBuilt &&
           (o.ozaki_slices <= 0 || o.ozaki_slices == (crt ? sr::kCrtDefaultModuli : kHp)) &&
           (o.lp_slices <= 0 || o.lp_slices == kLp) && !o.symmetric;
}

namespace {

// Serialises descriptor arrays into one host buffer; offsets are valid in
// the device copy after upload().
struct DescPack {
    std::vector<unsigned char> buf;
    template <class T>
    size_t add(const std::vector<T> &v)
    {
        const size_t off = (buf.size() + 255) / 256 * 256;
        buf.resize(off + v.size() * sizeof(T));
        if (!v.empty()) memcpy(buf.data() + off, v.data(), v.size() * sizeof(T));
        return off;
    }
};

sr_status ensure_capacity(BatchWork *bw, long long elems, int rows, int count, long long planes, int kmax,
                          size_t npartial, size_t flow_words, int dev, bool crt)
{
    cudaError_t e = cudaSuccess;
    if (flow_words > bw->flow_cap) {
        cudaFree(bw->flow);
        e = cudaMalloc((void **)&bw->flow, flow_words * sizeof(int));
        if (e != cudaSuccess) { bw->flow = nullptr; bw->flow_cap = 0; sr_set_last_cuda_error(e); return SR_ERR_OOM; }
        bw->flow_cap = flow_words;
    }
    if (!bw->flow_ctas) {
        // the group form of the dataflow solve is launched from this file
        using K = void (*)(int, float *, int, const double *, const double *, int *, int *,
                           const unsigned long long *, int, float *, int, double, const sr::SolveMat *,
                           const int *);
        const K kern = sr::trisolve_flow_kernel<float, true>;
        const size_t sm = sr::FlowShape<float>::smem;
        int per_sm = 0, sms = 0;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, sr::FlowShape<float>::NT, sm);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) { sr_set_last_cuda_error(e); return SR_ERR_CUDA; }
        bw->flow_ctas = std::max(1, per_sm) * sms;
    }
    if (elems > bw->cap_elems || rows > bw->cap_rows || planes > bw->cap_planes || count > bw->cap_count ||
        kmax > bw->cap_k || bw->crt != (crt ? 1 : 0)) {
        // grow everything together (the group's buffers are replaced wholesale)
        double **bufs[] = {&bw->Q0, &bw->Q1, &bw->AQ, &bw->Y, &bw->Delta, &bw->W, &bw->W2, &bw->YW};
        for (double **p : bufs) { cudaFree(*p); *p = nullptr; }
        cudaFree(bw->TE); bw->TE = nullptr;
        cudaFree(bw->acc); bw->acc = nullptr;
        cudaFree(bw->diag); bw->diag = nullptr;
        cudaFree(bw->norms); bw->norms = nullptr;
        cudaFree(bw->flags); bw->flags = nullptr;
        sr::ozaki_free(bw->oz);
        bw->oz = sr::OzakiWork{};
        const long long E = std::max(elems, bw->cap_elems), P = std::max(planes, bw->cap_planes);
        const int R = std::max(rows, bw->cap_rows), C = std::max(count, bw->cap_count);
        const int Kx = std::max(kmax, bw->cap_k);
        for (double **p : bufs)
            if (e == cudaSuccess) e = cudaMalloc((void **)p, (size_t)E * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc((void **)&bw->TE, (size_t)E * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void **)&bw->acc, (size_t)E * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void **)&bw->diag, (size_t)R * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc((void **)&bw->norms, (size_t)C * kNorms * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc((void **)&bw->flags, (size_t)C * sizeof(int));
        // slots: rows of A, columns of Q, columns of A Q / Delta, rows of Q (FP64
        // class: digits, or residues modulo 16 moduli); columns of W, Y, W^2 (FP32 class)
        int caps[sr::kOzakiSlots] = {kHp, kHp, kHp, kHp, kLp, kLp, kLp, 0};
        const unsigned hp_mask = (1u << sr::OZS_ROWS) | (1u << sr::OZS_COLS) | (1u << sr::OZS_X) |
                                 (1u << sr::OZS_QROWS);
        if (e == cudaSuccess)
            e = sr::ozaki_alloc_group(bw->oz, R + sr::kOzakiTileI, Kx, caps, P, crt ? sr::kCrtDefaultModuli : 0,
                                      crt ? hp_mask : 0u);
        if (e != cudaSuccess) {
            sr_set_last_cuda_error(e);
            cudaGetLastError();
            bw->cap_elems = bw->cap_rows = bw->cap_count = bw->cap_k = 0;
            bw->cap_planes = 0;
            bw->crt = -1;
            return e == cudaErrorMemoryAllocation ? SR_ERR_OOM : SR_ERR_CUDA;
        }
        bw->crt = crt ? 1 : 0;
        bw->cap_elems = E;
        bw->cap_rows = R;
        bw->cap_count = C;
        bw->cap_planes = P;
        bw->cap_k = Kx;
    }
    if (npartial > bw->npartial) {
        cudaFree(bw->partial);
        e = cudaMalloc((void **)&bw->partial, npartial * sizeof(double));
        if (e != cudaSuccess) { bw->npartial = 0; sr_set_last_cuda_error(e); return SR_ERR_OOM; }
        bw->npartial = npartial;
    }
    const size_t hn = (size_t)count * (kNorms + 1);
    if (hn > bw->hnorms_cap) {
        if (bw->hnorms) cudaFreeHost(bw->hnorms);
        e = cudaMallocHost((void **)&bw->hnorms, hn * sizeof(double));
        if (e != cudaSuccess) { bw->hnorms = nullptr; bw->hnorms_cap = 0; sr_set_last_cuda_error(e); return SR_ERR_OOM; }
        bw->hnorms_cap = hn;
    }
    if (!bw->aux) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bw->aux, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bw->ev0, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bw->ev1, cudaEventDisableTiming);
        if (e != cudaSuccess) { sr_set_last_cuda_error(e); return SR_ERR_CUDA; }
    }
    return SR_OK;
}

// Work items of a slice product for the listed matrices: tiles of 256 rows x
// 128 columns over each n_b x n_b output, all levels of s digits in one item
// (symmetric: the tiles on and above the diagonal only).
void make_items(std::vector<sr::MmaItem> &items, const std::vector<int> &act, const std::vector<int> &n,
                const std::vector<int> &row0, const std::vector<long long> &poff, int s, bool symmetric)
{
    items.clear();
    for (int b : act) {
        const int nb = n[b], ld = r32(nb);
        for (int j0 = 0; j0 < nb; j0 += sr::kOzakiTileJ)
            for (int i0 = 0; i0 < nb; i0 += sr::kOzakiTileI) {
                if (symmetric && i0 > j0 + sr::kOzakiTileJ - 1) continue;
                sr::MmaItem it{};
                it.ra = row0[b] + i0;
                it.rb = row0[b] + j0;
                it.nch = (nb + sr::kOzakiKChunk - 1) / sr::kOzakiKChunk;
                it.kbl = (nb - (it.nch - 1) * sr::kOzakiKChunk + 63) / 64;
                it.lb = 0;
                it.le = s;
                it.ldp = ld;
                it.rlim = ld - i0;
                it.clim = ld - j0;
                it.poff = poff[b] + (long long)j0 * ld + i0;
                items.push_back(it);
            }
    }
}

// Flat-grid prefix sums of the matrices of one launch, in launch order
struct Grids {
    size_t o32 = 0, omax = 0, odig = 0;
    int m = 0, t32 = 0, tmax = 0, tdig = 0;
};

Grids add_grids(DescPack &pk, const std::vector<int> &order, const std::vector<int> &n)
{
    const int m = (int)order.size();
    std::vector<int> s32(m + 1, 0), smax(m + 1, 0), sdig(m + 1, 0);
    for (int a = 0; a < m; ++a) {
        const int nb = n[order[a]], g = (nb + 31) / 32;
        s32[a + 1] = s32[a] + g * g;
        smax[a + 1] = smax[a] + g * ((nb + 255) / 256);   // absmax blocks cover 256 of K
        sdig[a + 1] = sdig[a] + g * ((nb + 63) / 64);     // digit blocks cover 64 of K (up to the order)
    }
    Grids G;
    G.o32 = pk.add(s32);
    G.omax = pk.add(smax);
    G.odig = pk.add(sdig);
    G.m = m;
    G.t32 = s32[m];
    G.tmax = smax[m];
    G.tdig = sdig[m];
    return G;
}

// bf16 flops of a slice product: s (s + 1) / 2 digit pairs, or s residue products
long long item_flops(const std::vector<sr::MmaItem> &items, int s, bool crt)
{
    long long f = 0;
    for (const auto &it : items)
        f += (crt ? (long long)s : (long long)s * (s + 1) / 2) * 2LL * sr::kOzakiTileI * sr::kOzakiTileJ *
             ((it.nch - 1) * sr::kOzakiKChunk + it.kbl * 64);
    return f;
}

}  // namespace

sr_status sr_batch_refine(schur_refine_ctx *h, int batch, const int *nv, const void *const *dA, void *const *dQ,
                          const void *const *dQhat, int *iters_out, int *status_out)
{
    using namespace sr;
    if (!h->bw) h->bw = new BatchWork();
    BatchWork *bw = h->bw;
    cudaStream_t st = h->st;
    const int max_iter = h->opt.max_iter > 0 ? h->opt.max_iter : 10;

    std::vector<int> n(nv, nv + batch), row0(batch), st_b(batch, (int)SR_ERR_NOT_CONVERGED), it_b(batch, 0);
    std::vector<long long> off(batch), poff(batch);
    long long elems = 0, planes = 0;
    int rows = 0, nmx = 0;
    for (int b = 0; b < batch; ++b) {
        off[b] = elems;
        elems += (long long)n[b] * n[b];
        row0[b] = rows;
        rows += r32(n[b]);
        poff[b] = planes;
        planes += (long long)r32(n[b]) * r32(n[b]);
        nmx = std::max(nmx, n[b]);
    }
    // partial sums: one per 32 x 32 block of every matrix (flat grids)
    long long t32_all = 0;
    for (int b = 0; b < batch; ++b) t32_all += (long long)((n[b] + 31) / 32) * ((n[b] + 31) / 32);
    // published words of the dataflow solve: NB_b^2 per matrix
    size_t flow_words = 2;
    for (int b = 0; b < batch; ++b) flow_words += (size_t)((n[b] + 31) / 32) * (size_t)((n[b] + 31) / 32);
    const bool crt = h->opt.hp_gemm == SR_HP_OZAKI_CRT;
    SR_TRY(ensure_capacity(bw, elems, rows, batch, planes, std::max(512, nmx), (size_t)t32_all, flow_words, h->dev,
                           crt));
    // FP64-class products: digits, or residues modulo 16 moduli with each matrix's
    // fixed-point bits t from its order (as schur_refine_step on that matrix alone)
    const int shp = crt ? kCrtDefaultModuli : kHp;
    const long long pb = crt ? shp : 4LL * shp;   // plane bytes per entry
    std::vector<int> tb(batch, 0);
    if (crt)
        for (int b = 0; b < batch; ++b) {
            tb[b] = crt_bits(bw->oz.crt, n[b]);
            if (tb[b] < 1 || tb[b] > 62) return SR_ERR_UNSUPPORTED;
        }

    std::vector<int> cur(batch, 0);   // buffer holding the current Q: 0 = Q0, 1 = Q1
    std::vector<double> y_last(batch, NAN), prev(batch, INFINITY), anorm(batch, 1.0);
    double *Qbuf[2] = {bw->Q0, bw->Q1};

    auto upload = [&](DescPack &pk) -> sr_status {
        // the stream is idle here (every upload follows a synchronization), so
        // the descriptor buffers may be replaced
        if (pk.buf.size() > bw->desc_cap) {
            SR_CUDA_TRY(cudaStreamSynchronize(st));
            cudaFree(bw->ddesc);
            if (bw->hdesc) cudaFreeHost(bw->hdesc);
            bw->ddesc = nullptr;
            bw->hdesc = nullptr;
            bw->desc_cap = 0;
            const size_t cap = pk.buf.size() + pk.buf.size() / 2;
            cudaError_t e = cudaMalloc((void **)&bw->ddesc, cap);
            if (e == cudaSuccess) e = cudaMallocHost((void **)&bw->hdesc, cap);
            if (e != cudaSuccess) { sr_set_last_cuda_error(e); cudaGetLastError(); return SR_ERR_OOM; }
            bw->desc_cap = cap;
        }
        memcpy(bw->hdesc, pk.buf.data(), pk.buf.size());
        SR_CUDA_TRY(cudaMemcpyAsync(bw->ddesc, bw->hdesc, pk.buf.size(), cudaMemcpyHostToDevice, st));
        return SR_OK;
    };
    auto P = [&](size_t o) { return (void *)(bw->ddesc + o); };
    const dim3 blk(256);
    auto reduce = [&](const Grids &g, size_t o_map, int slot) -> sr_status {
        SrPhase ph(h, SR_PROF_OTHER, 0, (long long)g.t32 * 8, 1);
        group_reduce_kernel<<<g.m, 256, 0, st>>>(bw->partial, (const int *)P(g.o32), (const int *)P(o_map),
                                                 bw->norms, kNorms, slot);
        SR_CUDA_TRY(cudaGetLastError());
        return SR_OK;
    };
    // norms and flags of every matrix, plus the handle's flag word
    auto sync_read = [&]() -> sr_status {
        SR_CUDA_TRY(cudaMemcpyAsync(bw->hnorms, bw->norms, (size_t)batch * kNorms * sizeof(double),
                                    cudaMemcpyDeviceToHost, st));
        SR_CUDA_TRY(cudaMemcpyAsync(bw->hnorms + (size_t)batch * kNorms, bw->flags, (size_t)batch * sizeof(int),
                                    cudaMemcpyDeviceToHost, st));
        SR_CUDA_TRY(cudaMemcpyAsync(h->hbuf + 8, h->dflags, sizeof(int), cudaMemcpyDeviceToHost, st));
        SR_CUDA_TRY(cudaStreamSynchronize(st));
        return SR_OK;
    };
    auto norm = [&](int b, int slot) { return bw->hnorms[(size_t)b * kNorms + slot]; };
    auto flag = [&](int b) {
        int f;
        memcpy(&f, (const char *)(bw->hnorms + (size_t)batch * kNorms) + sizeof(int) * b, sizeof(int));
        return f;
    };
    auto timed_out = [&]() {
        int f;
        memcpy(&f, h->hbuf + 8, sizeof(int));
        if (f & SR_FLAG_TIMEOUT) return true;
        for (int b = 0; b < batch; ++b)
            if (flag(b) & SR_FLAG_TIMEOUT) return true;   // a wait of the dataflow solve
        return false;
    };
    auto split = [&](int slot, size_t o, const Grids &g, int layout, int s, long long el) {
        const GroupSplit gs{(const SplitMat *)P(o), (const int *)P(g.omax), (const int *)P(g.odig), g.m, g.tmax,
                            g.tdig, nmx};
        return ozaki_split_group(h, st, bw->oz, slot, gs, layout, s, 16 * el);
    };
    auto combine = [&](int rs, int cs, size_t o_cm, const auto *eps, const Grids &g, int s, double sign, bool mirror,
                       double *partial, long long el, long long bytes_per) {
        return ozaki_combine_group(h, st, bw->oz, rs, cs, (const CombMat *)P(o_cm), eps, (const int *)P(g.o32), g.m,
                                   g.t32, s, sign, mirror, partial, 8LL * s * el, bytes_per * el);
    };
    auto product = [&](int rs, int cs, size_t o, const std::vector<MmaItem> &it, int s) {
        return ozaki_product_items(h, st, bw->oz, rs, cs, (const MmaItem *)P(o), (int)it.size(), s,
                                   item_flops(it, s, bw->oz.slot[rs].crt != 0), h->dflags);
    };

    SR_CUDA_TRY(cudaMemsetAsync(bw->flags, 0, (size_t)batch * sizeof(int), st));
    SR_CUDA_TRY(cudaMemsetAsync(h->dflags, 0, sizeof(int), st));

    // ---- start: ||A||^2, rows of A, Q = fl64(Qhat), one Newton-Schulz step ----------
    std::vector<int> act(batch);
    for (int b = 0; b < batch; ++b) act[b] = b;
    {
        DescPack pk;
        std::vector<GMat> ga(batch), gq(batch);
        std::vector<SplitMat> arows(batch), qcols(batch), qrows(batch), ycols(batch);
        std::vector<CombMat> cm(batch);
        std::vector<EpMinusI> epy(batch);
        std::vector<EpUpdate> epu(batch);
        for (int b = 0; b < batch; ++b) {
            const int nb = n[b];
            const long long o = off[b];
            ga[b] = GMat{o, nb, nb, dA[b], nullptr};
            gq[b] = GMat{o, nb, nb, dQhat[b], nullptr};
            arows[b] = SplitMat{(const double *)dA[b], nb, nb, nb, row0[b], tb[b]};
            qcols[b] = SplitMat{bw->Q0 + o, nb, nb, nb, row0[b], tb[b]};
            qrows[b] = SplitMat{bw->Q0 + o, nb, nb, nb, row0[b], tb[b]};
            ycols[b] = SplitMat{bw->Y + o, nb, nb, nb, row0[b], tb[b]};
            cm[b] = CombMat{poff[b], r32(nb), nb, nb, row0[b], row0[b], 2 * tb[b]};
            epy[b] = EpMinusI{bw->Y + o, nb};
            epu[b] = EpUpdate{bw->Q0 + o, nb, bw->Q1 + o, nb, -0.5};
        }
        std::vector<MmaItem> sym, full;
        make_items(sym, act, n, row0, poff, shp, true);
        make_items(full, act, n, row0, poff, shp, false);
        const size_t o_ga = pk.add(ga), o_gq = pk.add(gq), o_ar = pk.add(arows), o_qc = pk.add(qcols),
                     o_qr = pk.add(qrows), o_yc = pk.add(ycols), o_cm = pk.add(cm), o_epy = pk.add(epy),
                     o_epu = pk.add(epu), o_sym = pk.add(sym), o_full = pk.add(full), o_map = pk.add(act);
        const Grids g = add_grids(pk, act, n);
        SR_TRY(upload(pk));
        {
            SrPhase ph(h, SR_PROF_OTHER, 2 * elems, 8 * elems, 1);
            group_sumsq_kernel<<<g.t32, blk, 0, st>>>((const GMat *)P(o_ga), (const int *)P(g.o32), g.m, bw->partial);
            SR_CUDA_TRY(cudaGetLastError());
        }
        SR_TRY(reduce(g, o_map, 2));
        SR_TRY(split(OZS_ROWS, o_ar, g, OZ_ROWS, shp, elems));
        {
            SrPhase ph(h, SR_PROF_OTHER, 0, 12 * elems, 1);
            group_convert_kernel<<<g.t32, blk, 0, st>>>((const GMat *)P(o_gq), (const int *)P(g.o32), g.m, bw->Q0);
            SR_CUDA_TRY(cudaGetLastError());
        }
        SR_TRY(split(OZS_COLS, o_qc, g, OZ_COLS, shp, elems));
        SR_TRY(product(OZS_COLS, OZS_COLS, o_sym, sym, shp));
        SR_TRY(combine(OZS_COLS, OZS_COLS, o_cm, (const EpMinusI *)P(o_epy), g, shp, 1.0, true, bw->partial, elems,
                       pb + 8));
        SR_TRY(reduce(g, o_map, 1));
        SR_TRY(split(OZS_QROWS, o_qr, g, OZ_ROWS, shp, elems));
        SR_TRY(split(OZS_X, o_yc, g, OZ_COLS, shp, elems));
        SR_TRY(product(OZS_QROWS, OZS_X, o_full, full, shp));
        SR_TRY(combine(OZS_QROWS, OZS_X, o_cm, (const EpUpdate *)P(o_epu), g, shp, 1.0, false, nullptr, elems,
                       pb + 24));
        SR_TRY(sync_read());
        if (timed_out()) return SR_ERR_TIMEOUT;
        for (int b = 0; b < batch; ++b) {
            cur[b] = 1;
            y_last[b] = sqrt(norm(b, 1));
            anorm[b] = sqrt(norm(b, 2) > 0 ? norm(b, 2) : 1.0);
        }
    }

    // ---- REPEAT ... UNTIL, every live matrix in the same launches ------------------------
    for (int k = 1; k <= max_iter && !act.empty(); ++k) {
        const int m = (int)act.size();
        long long el = 0;
        for (int b : act) el += (long long)n[b] * n[b];
        // S1 + S2: A Q, T^ = Q^T (A Q) split into TE and the diagonal, ||E||^2
        {
            DescPack pk;
            std::vector<SplitMat> qcols(m), aqcols(m);
            std::vector<CombMat> cm(m);
            std::vector<EpStore> e_aq(m);
            std::vector<EpSplit<float>> e_sp(m);
            for (int a = 0; a < m; ++a) {
                const int b = act[a], nb = n[b];
                const long long o = off[b];
                qcols[a] = SplitMat{Qbuf[cur[b]] + o, nb, nb, nb, row0[b], tb[b]};
                aqcols[a] = SplitMat{bw->AQ + o, nb, nb, nb, row0[b], tb[b]};
                cm[a] = CombMat{poff[b], r32(nb), nb, nb, row0[b], row0[b], 2 * tb[b]};
                e_aq[a] = EpStore{bw->AQ + o, nb};
                e_sp[a] = EpSplit<float>{bw->TE + o, nb, bw->diag + row0[b], nullptr, nb};
            }
            std::vector<MmaItem> full;
            make_items(full, act, n, row0, poff, shp, false);
            const size_t o_qc = pk.add(qcols), o_aqc = pk.add(aqcols), o_cm = pk.add(cm), o_eaq = pk.add(e_aq),
                         o_esp = pk.add(e_sp), o_full = pk.add(full), o_map = pk.add(act);
            const Grids g = add_grids(pk, act, n);
            SR_TRY(upload(pk));
            SR_TRY(split(OZS_COLS, o_qc, g, OZ_COLS, shp, el));
            SR_TRY(product(OZS_ROWS, OZS_COLS, o_full, full, shp));
            SR_TRY(combine(OZS_ROWS, OZS_COLS, o_cm, (const EpStore *)P(o_eaq), g, shp, 1.0, false, nullptr, el,
                           pb + 8));
            SR_TRY(split(OZS_X, o_aqc, g, OZ_COLS, shp, el));
            SR_TRY(product(OZS_COLS, OZS_X, o_full, full, shp));
            SR_TRY(combine(OZS_COLS, OZS_X, o_cm, (const EpSplit<float> *)P(o_esp), g, shp, 1.0, false, bw->partial,
                           el, pb + 4));
            SR_TRY(reduce(g, o_map, 0));
            SR_TRY(sync_read());
            if (timed_out()) {
                for (int b : act) st_b[b] = SR_ERR_TIMEOUT;
                act.clear();
                break;
            }
        }
        // the stop test of schur_refine_step, per matrix
        std::vector<int> next;
        for (int b : act) {
            it_b[b] = k;
            const double tol = h->opt.tol > 0 ? h->opt.tol : 1e-14 * sqrt((double)n[b]);
            const double rT = sqrt(norm(b, 0)) / anorm[b];
            if (!isfinite(rT)) { st_b[b] = SR_ERR_NONFINITE; continue; }
            if (rT <= tol && !(y_last[b] > sqrt(tol))) { st_b[b] = SR_OK; continue; }
            if (k >= 3 && rT > 10.0 * prev[b]) { st_b[b] = SR_ERR_NOT_CONVERGED; continue; }
            prev[b] = rT;
            next.push_back(b);
        }
        act.swap(next);
        if (act.empty()) break;
        // S4 - S8 for the matrices that go on
        const int m2 = (int)act.size();
        el = 0;
        for (int b : act) el += (long long)n[b] * n[b];
        {
            DescPack pk;
            std::vector<SolveMat> sm(batch, SolveMat{nullptr, 0, 0, nullptr, 0});
            long long fwords = 2;   // dataflow solve: published words of the matrices going on
            std::vector<int> orders(batch, 0);
            std::vector<GMat> ga(m2);
            std::vector<SplitMat> wcols(m2), ycols(m2), w2cols(m2), qrows(m2), dcols(m2);
            std::vector<CombMat> cm(m2);
            std::vector<EpMinusI> e_y(m2);
            std::vector<EpStore> e_w2(m2), e_yw(m2);
            std::vector<EpDeltaD> e_d(m2);
            std::vector<EpUpdate> e_u(m2);
            for (int a = 0; a < m2; ++a) {
                const int b = act[a], nb = n[b];
                const long long o = off[b];
                double *Qc = Qbuf[cur[b]] + o, *Qo = Qbuf[cur[b] ^ 1] + o;
                sm[b] = SolveMat{bw->TE + o, nb, nb, bw->diag + row0[b], fwords - 2, bw->acc + o};
                fwords += (long long)((nb + 31) / 32) * ((nb + 31) / 32);
                orders[b] = nb;
                ga[a] = GMat{o, nb, nb, nullptr, nullptr};
                wcols[a] = SplitMat{bw->W + o, nb, nb, nb, row0[b], tb[b]};
                ycols[a] = SplitMat{bw->Y + o, nb, nb, nb, row0[b], tb[b]};
                w2cols[a] = SplitMat{bw->W2 + o, nb, nb, nb, row0[b], tb[b]};
                qrows[a] = SplitMat{Qc, nb, nb, nb, row0[b], tb[b]};
                dcols[a] = SplitMat{bw->Delta + o, nb, nb, nb, row0[b], tb[b]};
                cm[a] = CombMat{poff[b], r32(nb), nb, nb, row0[b], row0[b], 2 * tb[b]};
                e_y[a] = EpMinusI{bw->Y + o, nb};
                e_w2[a] = EpStore{bw->W2 + o, nb};
                e_yw[a] = EpStore{bw->YW + o, nb};
                e_d[a] = EpDeltaD{bw->W + o, bw->Y + o, bw->YW + o, bw->W2 + o, nullptr, nullptr, nb, bw->Delta + o, nb};
                e_u[a] = EpUpdate{Qc, nb, Qo, nb, 0.5};
            }
            std::vector<unsigned long long> plan;
            std::vector<long long> poffs, nleaf;
            trisolve_plan_group(orders, plan, poffs, nleaf, kSolveTile);   // the dataflow form's tiles too
            // the dataflow solve's tickets: the plan's solved tiles, step by step
            // (every tile after the tiles it reads)
            const bool flow = h->opt.solve_mode == 1;   // the stepwise form unless asked
            std::vector<unsigned long long> fplan;
            if (flow)
                for (size_t l = 0; l < nleaf.size(); ++l)
                    fplan.insert(fplan.end(), plan.begin() + poffs[l], plan.begin() + poffs[l] + nleaf[l]);
            std::vector<MmaItem> full_hp, sym_hp, full_lp, sym_lp;
            make_items(full_hp, act, n, row0, poff, shp, false);
            make_items(sym_hp, act, n, row0, poff, shp, true);
            make_items(full_lp, act, n, row0, poff, kLp, false);
            make_items(sym_lp, act, n, row0, poff, kLp, true);
            const size_t o_sm = pk.add(sm), o_pl = pk.add(plan), o_ga = pk.add(ga), o_wc = pk.add(wcols),
                         o_yc = pk.add(ycols), o_w2c = pk.add(w2cols), o_qr = pk.add(qrows), o_dc = pk.add(dcols),
                         o_cm = pk.add(cm), o_ey = pk.add(e_y), o_ew2 = pk.add(e_w2), o_eyw = pk.add(e_yw),
                         o_ed = pk.add(e_d), o_eu = pk.add(e_u), o_fh = pk.add(full_hp), o_sh = pk.add(sym_hp),
                         o_fl = pk.add(full_lp), o_sl = pk.add(sym_lp), o_map = pk.add(act),
                         o_fp = pk.add(fplan);
            const Grids g = add_grids(pk, act, n);
            SR_TRY(upload(pk));
            // S4: the group's solves: one dataflow launch, or step by step
            {
                long long fl = 0;
                for (int b : act) fl += 2LL * n[b] * n[b] * n[b] / 3;
                SrPhase ph(h, SR_PROF_SOLVE, fl, 4 * el, flow ? 1 : 2LL * (long long)nleaf.size());
                if (flow)
                    SR_CUDA_TRY(trisolve_flow_launch_group<float>(st, (const SolveMat *)P(o_sm), bw->flags, bw->flow,
                                                                  (size_t)fwords,
                                                                  (const unsigned long long *)P(o_fp),
                                                                  (int)fplan.size(), bw->flow_ctas, h->opt.l_cap));
                else {
                    // the matrices' accumulators start at zero (offsets below the capacity)
                    SR_CUDA_TRY(cudaMemsetAsync(bw->acc, 0, (size_t)bw->cap_elems * sizeof(float), st));
                    SR_CUDA_TRY(trisolve_launches_group<float>(st, bw->aux, bw->ev0, bw->ev1,
                                                               (const SolveMat *)P(o_sm), bw->flags,
                                                               (const unsigned long long *)P(o_pl), poffs, nleaf,
                                                               h->opt.l_cap));
                }
            }
            // S5: Y = Q^T Q - I from Q's column digits (still in slot OZS_COLS), W = L - L^T
            SR_TRY(product(OZS_COLS, OZS_COLS, o_sh, sym_hp, shp));
            SR_TRY(combine(OZS_COLS, OZS_COLS, o_cm, (const EpMinusI *)P(o_ey), g, shp, 1.0, true, bw->partial, el,
                           pb + 8));
            SR_TRY(reduce(g, o_map, 1));
            {
                SrPhase ph(h, SR_PROF_OTHER, 0, 12 * el, 1);
                group_skew_kernel<<<g.t32, blk, 0, st>>>((const GMat *)P(o_ga), (const int *)P(g.o32), g.m, bw->TE,
                                                         bw->W);
                SR_CUDA_TRY(cudaGetLastError());
            }
            // S6: W^2 = -W^T W, YW = Y^T W, W^3 = -W^T W^2 (FP32 class); S7 in the last epilogue
            SR_TRY(split(OZS_W, o_wc, g, OZ_COLS, kLp, el));
            SR_TRY(split(OZS_Y, o_yc, g, OZ_COLS, kLp, el));
            SR_TRY(product(OZS_W, OZS_W, o_sl, sym_lp, kLp));
            SR_TRY(combine(OZS_W, OZS_W, o_cm, (const EpStore *)P(o_ew2), g, kLp, -1.0, true, nullptr, el,
                           4LL * kLp + 8));
            SR_TRY(product(OZS_Y, OZS_W, o_fl, full_lp, kLp));
            SR_TRY(combine(OZS_Y, OZS_W, o_cm, (const EpStore *)P(o_eyw), g, kLp, 1.0, false, nullptr, el,
                           4LL * kLp + 8));
            SR_TRY(split(OZS_W2, o_w2c, g, OZ_COLS, kLp, el));
            SR_TRY(product(OZS_W, OZS_W2, o_fl, full_lp, kLp));
            SR_TRY(combine(OZS_W, OZS_W2, o_cm, (const EpDeltaD *)P(o_ed), g, kLp, -1.0, false, nullptr, el,
                           4LL * kLp + 40));
            // S8: Q_new = Q + 1/2 Q Delta
            SR_TRY(split(OZS_QROWS, o_qr, g, OZ_ROWS, shp, el));
            SR_TRY(split(OZS_X, o_dc, g, OZ_COLS, shp, el));
            SR_TRY(product(OZS_QROWS, OZS_X, o_fh, full_hp, shp));
            SR_TRY(combine(OZS_QROWS, OZS_X, o_cm, (const EpUpdate *)P(o_eu), g, shp, 1.0, false, nullptr, el,
                           pb + 24));
            SR_TRY(sync_read());
        }
        if (timed_out()) {
            for (int b : act) st_b[b] = SR_ERR_TIMEOUT;
            act.clear();
            break;
        }
        // a failed solve keeps the factor from before the update (as schur_refine_step)
        next.clear();
        for (int b : act) {
            const int f = flag(b);
            if (f & SR_FLAG_NONDISTINCT) { st_b[b] = SR_ERR_NONDISTINCT; continue; }
            if (f & SR_FLAG_NONFINITE) { st_b[b] = SR_ERR_NONFINITE; continue; }
            cur[b] ^= 1;
            y_last[b] = sqrt(norm(b, 1));
            next.push_back(b);
        }
        act.swap(next);
    }
    for (int b : act) st_b[b] = SR_ERR_NOT_CONVERGED;

    // the refined factors to the caller's buffers
    {
        DescPack pk;
        std::vector<GMat> go(batch);
        for (int b = 0; b < batch; ++b) go[b] = GMat{off[b], n[b], n[b], Qbuf[cur[b]] + off[b], dQ[b]};
        const size_t o_go = pk.add(go);
        std::vector<int> all(batch);
        for (int b = 0; b < batch; ++b) all[b] = b;
        const Grids g = add_grids(pk, all, n);
        SR_TRY(upload(pk));
        SrPhase ph(h, SR_PROF_OTHER, 0, 16 * elems, 1);
        group_copy_out_kernel<<<g.t32, blk, 0, st>>>((const GMat *)P(o_go), (const int *)P(g.o32), g.m);
        SR_CUDA_TRY(cudaGetLastError());
        SR_CUDA_TRY(cudaStreamSynchronize(st));
    }
    sr_status first = SR_OK;
    for (int b = 0; b < batch; ++b) {
        if (iters_out) iters_out[b] = it_b[b];
        if (status_out) status_out[b] = st_b[b];
        if (st_b[b] != SR_OK && first == SR_OK) first = (sr_status)st_b[b];
    }
    return first;
}

// schur_refine_selftest_wait_timeout: the group form of the dataflow solve on
// one 64 x 64 FP32 matrix with a plan that omits tile (1, 0), which tile
// (0, 0) reads; the kernel's wait for it runs out, SR_FLAG_TIMEOUT is set in
// the matrix's error word and the launch ends. Every access stays inside the
// buffers allocated here.
sr_status sr_flow_selftest(schur_refine_ctx *h)
{
    using namespace sr;
    constexpr int n = 64, NB = 2;
    cudaStream_t st = h->st;
    float *TE = nullptr;
    double *diag = nullptr;
    SolveMat *mat = nullptr;
    unsigned long long *plan = nullptr;
    int *flags = nullptr, *work = nullptr;
    auto release = [&]() {
        cudaFree(TE);
        cudaFree(diag);
        cudaFree(mat);
        cudaFree(plan);
        cudaFree(flags);
        cudaFree(work);
    };
    const size_t nwords = 2 + (size_t)NB * NB;
    cudaError_t e = cudaMalloc((void **)&TE, (size_t)n * n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&diag, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&mat, sizeof(SolveMat));
    if (e == cudaSuccess) e = cudaMalloc((void **)&plan, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void **)&flags, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&work, nwords * sizeof(int));
    if (e != cudaSuccess) {
        sr_set_last_cuda_error(e);
        cudaGetLastError();
        release();
        return e == cudaErrorMemoryAllocation ? SR_ERR_OOM : SR_ERR_CUDA;
    }
    // T = diag(1, 2, ..., 64), E = 0: a well-posed problem, were the plan complete
    std::vector<float> hT((size_t)n * n, 0.0f);
    std::vector<double> hd(n);
    for (int i = 0; i < n; ++i) {
        hT[(size_t)i + (size_t)i * n] = (float)(i + 1);
        hd[i] = i + 1.0;
    }
    const SolveMat hm{TE, n, n, diag, 0};
    const unsigned long long hp = 0ull;   // matrix 0, tile (0, 0) only
    e = cudaMemcpyAsync(TE, hT.data(), hT.size() * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(diag, hd.data(), n * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mat, &hm, sizeof(hm), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(plan, &hp, sizeof(hp), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(trisolve_flow_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)FlowShape<float>::smem);
    if (e == cudaSuccess) e = trisolve_flow_launch_group<float>(st, mat, flags, work, nwords, plan, 1, 1);
    int hf = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    release();
    if (e != cudaSuccess) {
        sr_set_last_cuda_error(e);
        return SR_ERR_CUDA;
    }
    return (hf & SR_FLAG_TIMEOUT) ? SR_ERR_TIMEOUT : SR_OK;
}
