// Host engine and C ABI of the Schur-refinement library: the control flow of
// Alg. 4 (Sec. 2.4) over the kernels of gemm_simt.cuh, trisolve.cuh,
// kernels_misc.cuh and the tensor-core products of ozaki.cu.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "common.cuh"
#include "ctx.cuh"
#include "dd.cuh"
#include "gemm_simt.cuh"
#include "kernels_misc.cuh"
#include "ozaki.cuh"
#include "trisolve.cuh"
#include "quasi.cuh"

void sr::trisolve_plan(int n, std::vector<uint32_t> &tiles, std::vector<long long> &offsets, int B)
{
    const int NB = (n + B - 1) / B;
    tiles.clear();
    offsets.assign(1, 0);
    for (int t = NB - 1; t >= 0; --t) {
        const int d = t + 1;
        for (int J = 0; J + t < NB; ++J) tiles.push_back((uint32_t)((J + t) << 16 | J));   // D = t: solve
        for (int D = t - 1; D >= 0; --D)
            for (int J = 0; J + D < NB; ++J) {
                const int I = J + D;
                if (J + d < NB || I - d >= 0) tiles.push_back((uint32_t)(I << 16 | J));
            }
        offsets.push_back((long long)tiles.size());
    }
}

void sr::trisolve_flow_plan(int n, std::vector<unsigned long long> &tasks)
{
    trisolve_flow_plan(n, tasks, kFlowNear, kFlowChunk, kFlowFarNum, kFlowLag);
}

void sr::trisolve_flow_plan(int n, std::vector<unsigned long long> &tasks, int near, int chunk, int far_num, int lag)
{
    using ull = unsigned long long;
    const int NB = (n + kSolveTile - 1) / kSolveTile;
    const int far = (far_num * NB) / 16;   // helpers take subdiagonals d >= far only
    near = std::max(near, 1);
    chunk = std::max(chunk, 1);
    lag = std::max(0, std::min(lag, near - 1));   // a helper (lo >= D + near) precedes its owner
    std::vector<std::vector<ull>> enabled(NB);   // helpers by the subdiagonal that completes their inputs
    std::vector<int> nh((size_t)NB * NB, 0), own((size_t)NB * NB, 0);
    for (int D = 0; D < NB; ++D)
        for (int J = 0; J + D < NB; ++J) {
            const int I = J + D, top = std::max(NB - 1 - J, I), dF = std::max(D + near, far);
            own[(size_t)I * NB + J] = std::min(top, dF - 1);   // the owner's highest subdiagonal
            if (top < dF) continue;
            const int cnt = (top - dF + chunk) / chunk;
            nh[(size_t)I * NB + J] = cnt;
            for (int h = 0; h < cnt; ++h) {
                const int hi = top - h * chunk, lo = std::max(dF, hi - chunk + 1);
                enabled[lo].push_back(1ull << 63 | (ull)h << 56 | (ull)hi << 44 | (ull)lo << 32 | (ull)I << 16 |
                                      (ull)J);
            }
        }
    // the helpers that subdiagonal t completes follow the solves of t - lag:
    // the next steps' solves (the critical path) are claimed before them
    tasks.clear();
    for (int t = NB - 1; t >= 0; --t) {
        for (int J = 0; J + t < NB; ++J) {
            const size_t x = (size_t)(J + t) * NB + J;
            tasks.push_back((ull)own[x] << 48 | (ull)nh[x] << 32 | (ull)(J + t) << 16 | (ull)J);
        }
        if (t + lag < NB) tasks.insert(tasks.end(), enabled[t + lag].begin(), enabled[t + lag].end());
    }
}

void sr::trisolve_plan_group(const std::vector<int> &orders, std::vector<unsigned long long> &tiles,
                             std::vector<long long> &offsets, std::vector<long long> &nleaf, int B)
{
    int NBmax = 0;
    for (int n : orders) NBmax = std::max(NBmax, (n + B - 1) / B);
    tiles.clear();
    nleaf.clear();
    offsets.assign(1, 0);
    for (int t = NBmax - 1; t >= 0; --t) {
        const int d = t + 1;
        long long nl = 0;
        for (size_t b = 0; b < orders.size(); ++b) {
            const int NB = (orders[b] + B - 1) / B;
            for (int J = 0; J + t < NB; ++J) {
                tiles.push_back((unsigned long long)b << 32 | (unsigned long long)((J + t) << 16 | J));
                ++nl;
            }
        }
        for (size_t b = 0; b < orders.size(); ++b) {
            const int NB = (orders[b] + B - 1) / B;
            if (t >= NB) continue;
            for (int D = t - 1; D >= 0; --D)
                for (int J = 0; J + D < NB; ++J) {
                    const int I = J + D;
                    if (J + d < NB || I - d >= 0)
                        tiles.push_back((unsigned long long)b << 32 | (unsigned long long)(I << 16 | J));
                }
        }
        nleaf.push_back(nl);
        offsets.push_back((long long)tiles.size());
    }
}

static thread_local cudaError_t g_last_cuda = cudaSuccess;
void sr_set_last_cuda_error(cudaError_t e) { g_last_cuda = e; }


static cudaEvent_t take_event(schur_refine_ctx *h)
{
    if (!h->ev_pool.empty()) {
        cudaEvent_t e = h->ev_pool.back();
        h->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void sr_prof_begin(schur_refine_ctx *h, int kind, long long flops, long long bytes, long long launches)
{
    h->prof.flops[kind] += flops;
    h->prof.bytes[kind] += bytes;
    h->prof.launches[kind] += launches;
    if (!h->opt.profile || h->capturing) return;
    cudaEvent_t a = take_event(h);
    cudaEventRecord(a, h->st);
    h->open_ev.push_back(a);
}

void sr_prof_end(schur_refine_ctx *h, int kind)
{
    if (!h->opt.profile || h->capturing || h->open_ev.empty()) return;
    cudaEvent_t a = h->open_ev.back();
    h->open_ev.pop_back();
    cudaEvent_t b = take_event(h);
    cudaEventRecord(b, h->st);
    h->pending.push_back({kind, a, b});
}

// Adds the elapsed times of finished spans (the stream must be idle).
static void harvest(schur_refine_ctx *h)
{
    for (auto &sp : h->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, sp.a, sp.b) == cudaSuccess) {
            h->prof.ms[sp.kind] += ms;
            h->prof.spans[sp.kind] += 1;
        }
        h->ev_pool.push_back(sp.a);
        h->ev_pool.push_back(sp.b);
    }
    h->pending.clear();
    cudaGetLastError();
}

namespace {

bool is_cplx(const sr_options &o) { return o.dtype == SR_COMPLEX; }
size_t lp_size(const sr_options &o) { return (o.lp == SR_LP_FP32 ? sizeof(float) : sizeof(double)) * (is_cplx(o) ? 2 : 1); }
// high-precision element: FP64, complex128, a double-double pair (two planes)
// or a triple-double (three planes)
size_t hp_size(const sr_options &o)
{
    if (o.target == SR_TARGET_TD) return 3 * sizeof(double);
    if (o.target == SR_TARGET_D6) return sr::kD6Words * sizeof(double);
    return sizeof(double) * (is_cplx(o) || o.target == SR_TARGET_DD ? 2 : 1);
}

// high-precision products emulated on the tensor cores (digits or residues)
bool is_emulated(const sr_options &o) { return o.hp_gemm == SR_HP_OZAKI_BF16 || o.hp_gemm == SR_HP_OZAKI_CRT; }

// bf16 digits (7; 14 for double-double) or residues modulo 16 (32) moduli per operand
int oz_count(const sr_options &o)
{
    if (o.target == SR_TARGET_TD || o.target == SR_TARGET_D6) return sr::kCrtDefaultModuliTD;
    if (o.ozaki_slices > 0) return o.ozaki_slices;
    const bool dd = o.target == SR_TARGET_DD;
    if (o.hp_gemm == SR_HP_OZAKI_CRT) return dd ? sr::kCrtDefaultModuliDD : sr::kCrtDefaultModuli;
    return dd ? sr::kOzakiDefaultSlicesDD : sr::kOzakiDefaultSlices;
}

sr_status check_opts(const sr_options &o)
{
    if (o.dtype != SR_REAL && o.dtype != SR_COMPLEX) return SR_ERR_INVALID_ARG;
    if (o.target != SR_TARGET_FP64 && o.target != SR_TARGET_DD && o.target != SR_TARGET_TD &&
        o.target != SR_TARGET_D6)
        return SR_ERR_INVALID_ARG;
    if (o.hp_gemm != SR_HP_FP64 && o.hp_gemm != SR_HP_OZAKI_BF16 && o.hp_gemm != SR_HP_OZAKI_CRT)
        return SR_ERR_INVALID_ARG;
    if (o.lp != SR_LP_FP32 && o.lp != SR_LP_FP64) return SR_ERR_INVALID_ARG;
    if (o.qhat_type != SR_QHAT_FP32 && o.qhat_type != SR_QHAT_FP64) return SR_ERR_INVALID_ARG;
    if ((o.batch_mode != 0 && o.batch_mode != 1) || (o.tune != 0 && o.tune != 1) || (o.graph != 0 && o.graph != 1) ||
        o.solve_mode < 0 || o.solve_mode > 2 || (o.symmetric != 0 && o.symmetric != 1) || !(o.l_cap >= 0.0) ||
        std::isinf(o.l_cap) || o.lp_slices > sr::kOzakiLpSlices || (o.quasi != 0 && o.quasi != 1))
        return SR_ERR_INVALID_ARG;
    if (o.hp_gemm == SR_HP_OZAKI_CRT) {
        // FP64 results: M < 2^128 holds for at most 16 moduli; double-double
        // (M < 2^256): 34; triple-double: the 48 of its form
        const bool mw = o.target == SR_TARGET_TD || o.target == SR_TARGET_D6;
        const int mx = o.target == SR_TARGET_DD ? sr::kCrtMaxModuliDD
                       : mw                     ? sr::kCrtDefaultModuliTD
                                                : sr::kCrtDefaultModuli;
        if (o.ozaki_slices > mx || (mw && o.ozaki_slices > 0 && o.ozaki_slices != sr::kCrtDefaultModuliTD))
            return SR_ERR_INVALID_ARG;
    } else if (o.ozaki_slices > (o.target == SR_TARGET_DD ? sr::kOzakiMaxSlicesDD : sr::kOzakiMaxSlices)) {
        return SR_ERR_INVALID_ARG;
    }
    // double-double target: real data, FP64 correction path, FP64 start
    if (o.target == SR_TARGET_DD && (o.dtype != SR_REAL || o.lp != SR_LP_FP64 || o.qhat_type != SR_QHAT_FP64))
        return SR_ERR_UNSUPPORTED;
    // triple- and six-double targets: the same, with the residue-form products only
    if ((o.target == SR_TARGET_TD || o.target == SR_TARGET_D6) &&
        (o.dtype != SR_REAL || o.lp != SR_LP_FP64 || o.qhat_type != SR_QHAT_FP64 || o.hp_gemm != SR_HP_OZAKI_CRT ||
         o.graph))
        return SR_ERR_UNSUPPORTED;
    // complex data: the emulated products with the complex64 correction path
    if (o.dtype == SR_COMPLEX && (!is_emulated(o) || o.lp != SR_LP_FP32)) return SR_ERR_UNSUPPORTED;
    // Sec. 2.5 (real symmetric or complex Hermitian A); the double-double target keeps the general form
    if (o.symmetric && o.target != SR_TARGET_FP64) return SR_ERR_UNSUPPORTED;
    // the real quasi-triangular form: real data, FP64 target, host loop, general A
    if (o.quasi && (o.dtype != SR_REAL || o.target != SR_TARGET_FP64 || o.graph || o.symmetric))
        return SR_ERR_UNSUPPORTED;
    if (is_emulated(o) && !sr::kOzakiBuilt) return SR_ERR_UNSUPPORTED;
    return SR_OK;
}

double tol_of(const schur_refine_ctx *h, int n)
{
    return h->opt.tol > 0 ? h->opt.tol : 1e-14 * sqrt((double)n);
}

sr_status reduce_to(schur_refine_ctx *h, int count, int slot)
{
    SrPhase ph(h, SR_PROF_OTHER, 0, (long long)count * 8, 1);
    sr::reduce_partials_kernel<<<1, 256, 0, h->st>>>(h->partial, count, h->dnorm + slot);
    SR_CUDA_TRY(cudaGetLastError());
    return SR_OK;
}

// Frobenius norm^2 of (part of) a matrix into dnorm[slot].
template <typename T>
sr_status sumsq(schur_refine_ctx *h, int n, const T *M, int ld, int part, int slot)
{
    const int blocks = (int)std::min<size_t>(1024, h->npartial);
    {
    SrPhase ph(h, SR_PROF_OTHER, 2LL * n * n, (long long)n * n * (long long)sizeof(T), 1);
    sr::sumsq_kernel<T><<<blocks, 256, 0, h->st>>>(n, M, ld, part, h->partial);
    SR_CUDA_TRY(cudaGetLastError());
    }
    return reduce_to(h, blocks, slot);
}

// copy dnorm (and flags) to the pinned host mirror and wait
sr_status read_back(schur_refine_ctx *h)
{
    SR_CUDA_TRY(cudaMemcpyAsync(h->hbuf, h->dnorm, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    SR_CUDA_TRY(cudaMemcpyAsync(h->hbuf + 8, h->dflags, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    SR_CUDA_TRY(cudaStreamSynchronize(h->st));
    return SR_OK;
}

int host_flags(const schur_refine_ctx *h)
{
    int f;
    memcpy(&f, h->hbuf + 8, sizeof(int));
    return f;
}

// a bounded device wait ran out somewhere since the flags were cleared
bool timed_out(const schur_refine_ctx *h) { return (host_flags(h) & SR_FLAG_TIMEOUT) != 0; }

// ---- high-precision product with the handle's engine ---------------------------
// C = op(A) B (m x n, inner k) fed to epilogue ep; when slot >= 0 the epilogue's
// returned values are summed into dnorm[slot].
template <class EP>
sr_status hp_gemm(schur_refine_ctx *h, bool transA, int m, int n, int k, const double *A, int lda,
                  const double *B, int ldb, EP ep, int slot)
{
    double *part = slot >= 0 ? h->partial : nullptr;
    int blocks = 0;
    if (is_emulated(h->opt)) {
        SR_TRY(sr::ozaki_gemm(h, h->st, h->oz, transA, m, n, k, A, lda, B, ldb, ep, part, &blocks,
                              oz_count(h->opt), h->dflags));
    } else {
        SrPhase ph(h, SR_PROF_HP_GEMM, 2LL * m * n * k, 8LL * ((long long)m * k + (long long)k * n + (long long)m * n), 1);
        using sr::LoadN;
        using sr::LoadT;
        cudaError_t e;
        if (transA)
            e = sr::gemm_simt<double>(h->st, m, n, k, LoadT<double, double>{A, lda}, LoadN<double, double>{B, ldb},
                                      ep, part);
        else
            e = sr::gemm_simt<double>(h->st, m, n, k, LoadN<double, double>{A, lda}, LoadN<double, double>{B, ldb},
                                      ep, part);
        SR_CUDA_TRY(e);
        blocks = sr::simt_blocks<double>(m, n);
    }
    if (slot >= 0) SR_TRY(reduce_to(h, blocks, slot));
    return SR_OK;
}

// ---- one pass pieces -------------------------------------------------------------

// S1 + S2: AQ = A Q, T^ = Q^H (A Q) with the split epilogue, ||E||^2 -> dnorm[0]
template <typename Tl>
sr_status form_residual(schur_refine_ctx *h, int n, const double *A, int lda, const double *Q, int ldq,
                        double *That)
{
    const int ld = h->nmax;
    SR_TRY(hp_gemm(h, false, n, n, n, A, lda, Q, ldq, sr::EpStore{h->AQ, ld}, -1));
    sr::EpSplit<Tl> ep{(Tl *)h->TE, ld, h->diag, That, n};
    if (h->opt.quasi) {
        ep.sub = h->band;
        ep.sup = h->band + h->nmax;
    }
    SR_TRY(hp_gemm(h, true, n, n, n, Q, ldq, h->AQ, ld, ep, 0));
    return SR_OK;
}

// S4: solve in low precision; ||L||^2 -> dnorm[2]
void drop_graphs(schur_refine_ctx *h)
{
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
}

// the stepwise form's launch plan for order n and tile B
sr_status ensure_plan(schur_refine_ctx *h, int n, int B)
{
    if (h->plan_n == n && h->plan_b == B) return SR_OK;
    drop_graphs(h);   // graphs hold the old plan's pointer and contents
    std::vector<uint32_t> tiles;
    sr::trisolve_plan(n, tiles, h->plan_off, B);
    if (tiles.size() > h->plan_cap) {
        // the plan is built once per order; its buffer grows only when needed
        SR_CUDA_TRY(cudaStreamSynchronize(h->st));
        cudaFree(h->plan);
        h->plan = nullptr;
        h->plan_cap = 0;
        cudaError_t e = cudaMalloc((void **)&h->plan, tiles.size() * sizeof(uint32_t));
        if (e != cudaSuccess) {
            sr_set_last_cuda_error(e);
            return e == cudaErrorMemoryAllocation ? SR_ERR_OOM : SR_ERR_CUDA;
        }
        h->plan_cap = tiles.size();
    }
    SR_CUDA_TRY(cudaMemcpyAsync(h->plan, tiles.data(), tiles.size() * sizeof(uint32_t), cudaMemcpyHostToDevice,
                                h->st));
    SR_CUDA_TRY(cudaStreamSynchronize(h->st));   // tiles is a temporary
    h->plan_n = n;
    h->plan_b = B;
    return SR_OK;
}

// task list of the dataflow solve for order n (host work and a
// synchronization: built before any capture)
sr_status ensure_flow_plan(schur_refine_ctx *h, int n)
{
    if (h->flow_plan_n == n) return SR_OK;
    std::vector<unsigned long long> tasks;
    sr::trisolve_flow_plan(n, tasks);
    if (tasks.size() > h->flow_plan_cap) {
        SR_CUDA_TRY(cudaStreamSynchronize(h->st));
        cudaFree(h->flow_plan);
        h->flow_plan = nullptr;
        h->flow_plan_cap = 0;
        cudaError_t e = cudaMalloc((void **)&h->flow_plan, tasks.size() * sizeof(unsigned long long));
        if (e != cudaSuccess) {
            sr_set_last_cuda_error(e);
            return e == cudaErrorMemoryAllocation ? SR_ERR_OOM : SR_ERR_CUDA;
        }
        h->flow_plan_cap = tasks.size();
    }
    SR_CUDA_TRY(cudaMemcpyAsync(h->flow_plan, tasks.data(), tasks.size() * sizeof(unsigned long long),
                                cudaMemcpyHostToDevice, h->st));
    SR_CUDA_TRY(cudaStreamSynchronize(h->st));   // tasks is a temporary
    h->flow_plan_n = n;
    h->flow_ntasks = (int)tasks.size();
    return SR_OK;
}

// the dataflow form serves this solve (see sr_options.solve_mode)
bool use_flow(const schur_refine_ctx *h, int kind)
{
    return kind <= 2 && h->flow_acc && (h->opt.solve_mode == 1 || (h->opt.solve_mode == 0 && kind == 0));
}

template <typename Tl>
sr_status solve(schur_refine_ctx *h, int n, Tl *TE, int ld, const typename SrNum<Tl>::hp *dhp,
                const double *dlo = nullptr)
{
    constexpr int B = sr::StepTile<Tl>::B;
    const int NB = (n + B - 1) / B;
    const int kind = SrNum<Tl>::kind;
    {
        if (h->opt.symmetric) {
            // Sec. 2.5: T diagonal, one division per entry
            SrPhase ph(h, SR_PROF_SOLVE, (long long)n * (n - 1) / 2, (long long)n * n * (long long)sizeof(Tl), 1);
            const dim3 grid((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32));
            sr::diag_solve_kernel<Tl><<<grid, 256, 0, h->st>>>(n, TE, ld, dhp, h->dflags, h->opt.l_cap);
            SR_CUDA_TRY(cudaGetLastError());
            return SR_OK;
        }
    }
    if constexpr (SrNum<Tl>::kind <= 2) {
        if (use_flow(h, kind)) {
            // one launch: the dataflow over the tiles
            SR_TRY(ensure_flow_plan(h, n));
            const long long fl = 2LL * n * n * n / 3 * (kind == 2 ? 4 : 1);
            SrPhase ph(h, SR_PROF_SOLVE, fl, (long long)n * n * (long long)sizeof(Tl), 1);
            SR_CUDA_TRY(sr::trisolve_flow_launch<Tl>(h->st, n, TE, ld, dhp, dlo, h->dflags, h->flow, h->flow_plan,
                                                     h->flow_ntasks, (Tl *)h->flow_acc, h->nmax,
                                                     h->flow_ctas[kind], h->opt.l_cap));
            return SR_OK;
        }
    }
    SR_TRY(ensure_plan(h, n, B));
    cudaGraphExec_t exec = nullptr;
    if (h->capturing) {
        // inside the refinement's own graph: the launches themselves are captured
        SR_CUDA_TRY(sr::trisolve_launches<Tl>(h->st, h->aux_st, h->sev0, h->sev1, n, TE, ld, dhp, dlo, h->dflags,
                                              h->plan, h->plan_off, h->opt.l_cap, (Tl *)h->step_acc, h->nmax));
        return SR_OK;
    }
    for (auto &g : h->graphs)
        if (g.n == n && g.TE == TE && g.ld == ld && g.dhp == dhp && g.dlo == dlo && g.kind == kind) exec = g.exec;
    if (!exec) {
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t el = sr::trisolve_launches<Tl>(h->cap_st, h->aux_st, h->sev0, h->sev1, n, TE, ld, dhp, dlo,
                                                       h->dflags, h->plan, h->plan_off, h->opt.l_cap,
                                                       (Tl *)h->step_acc, h->nmax);
            e = cudaStreamEndCapture(h->cap_st, &graph);
            if (el != cudaSuccess) e = el;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e == cudaSuccess) {
            h->graphs.push_back({n, TE, ld, dhp, dlo, kind, exec});
        } else {
            // no graph (for example while the caller captures this stream): the same
            // launches, issued directly on the two streams
            cudaGetLastError();
            exec = nullptr;
        }
    }
    const long long fl = 2LL * n * n * n / 3 * (SrNum<Tl>::kind >= 2 ? 4 : 1);   // a complex FMA is 4 real ones
    SrPhase ph(h, SR_PROF_SOLVE, fl, (long long)n * n * (long long)sizeof(Tl), 2LL * NB);
    if (exec) {
        SR_CUDA_TRY(cudaGraphLaunch(exec, h->st));
    } else {
        SR_CUDA_TRY(sr::trisolve_launches<Tl>(h->st, h->aux_st, h->sev0, h->sev1, n, TE, ld, dhp, dlo, h->dflags,
                                              h->plan, h->plan_off, h->opt.l_cap, (Tl *)h->step_acc, h->nmax));
    }
    return SR_OK;
}

// S5-S8: Y = Q^H Q - I, products in lp, Delta, Q_new = Q + 1/2 Q Delta
template <typename Tl>
sr_status update(schur_refine_ctx *h, int n, const double *Q, int ldq, double *Qn, int ldn)
{
    using sr::LoadN;
    using sr::LoadSkew;
    const int ld = h->nmax;
    SR_TRY(hp_gemm(h, true, n, n, n, Q, ldq, Q, ldq, sr::EpMinusI{h->Y, ld}, 1));
    const Tl *L = (const Tl *)h->TE;
    Tl *W2 = (Tl *)h->W2, *YW = (Tl *)h->YW;
    LoadSkew<Tl, Tl> w{L, ld};
    const long long f1 = 2LL * n * n * n, b1 = 4LL * n * n * (long long)sizeof(Tl);
    {
    SrPhase ph(h, SR_PROF_LP_GEMM, f1 * (h->opt.full_sigma ? 5 : 3), b1 * (h->opt.full_sigma ? 5 : 3),
               h->opt.full_sigma ? 5 : 3);
    SR_CUDA_TRY(sr::gemm_simt<Tl>(h->st, n, n, n, w, w, sr::EpStoreLp<Tl>{W2, ld}, nullptr));
    SR_CUDA_TRY(sr::gemm_simt<Tl>(h->st, n, n, n, LoadN<Tl, double>{h->Y, ld}, w, sr::EpStoreLp<Tl>{YW, ld},
                                  nullptr));
    Tl *W2Y = nullptr, *W2YW = nullptr;
    if (h->opt.full_sigma) {
        W2Y = (Tl *)h->W2Y;
        W2YW = (Tl *)h->W2YW;
        SR_CUDA_TRY(sr::gemm_simt<Tl>(h->st, n, n, n, LoadN<Tl, Tl>{W2, ld}, LoadN<Tl, double>{h->Y, ld},
                                      sr::EpStoreLp<Tl>{W2Y, ld}, nullptr));
        SR_CUDA_TRY(sr::gemm_simt<Tl>(h->st, n, n, n, LoadN<Tl, Tl>{W2Y, ld}, w, sr::EpStoreLp<Tl>{W2YW, ld},
                                      nullptr));
    }
    sr::EpDelta<Tl> ed{L, ld, h->Y, ld, YW, W2, W2Y, W2YW, ld, h->Delta, ld};
    SR_CUDA_TRY(sr::gemm_simt<Tl>(h->st, n, n, n, w, LoadN<Tl, Tl>{W2, ld}, ed, nullptr));
    }
    SR_TRY(hp_gemm(h, false, n, n, n, Q, ldq, h->Delta, ld, sr::EpUpdate{Q, ldq, Qn, ldn, 0.5}, -1));
    return SR_OK;
}

// ---- the pass on the emulated engine ------------------------------------------------
// Digits are split once and reused: the columns of Q serve A Q, Q^H (A Q) and
// Q^H Q; the rows of A are split once per call. The low-precision products use
// kOzakiLpSlices digits (about 24 bits, FP32-class) and only column splits:
// W^2 = -W^H W, YW = Y^H W (Y Hermitian), W^3 = -W^H W^2, W^2 Y = (W^2)^H Y.
// The same code serves real (C = false) and complex (C = true) data; the
// types and epilogues come from OzT<C>.

bool oz_pass(const schur_refine_ctx *h) { return is_emulated(h->opt) && h->opt.lp == SR_LP_FP32; }
int oz_s(const schur_refine_ctx *h) { return oz_count(h->opt); }

template <bool C> struct OzT;
template <> struct OzT<false> {
    using H = double;
    using L = float;
    using Store = sr::EpStore;
    using Split = sr::EpSplit<float>;
    using MinusI = sr::EpMinusI;
    using Update = sr::EpUpdate;
    using Delta = sr::EpDeltaD;
};
template <> struct OzT<true> {
    using H = cd;
    using L = cf;
    using Store = sr::EpStoreC;
    using Split = sr::EpSplitC;
    using MinusI = sr::EpMinusIC;
    using Update = sr::EpUpdateC;
    using Delta = sr::EpDeltaDC;
};

// Y = Q^H Q - I from the column digits of Q in slot OZS_COLS; ||Y||^2 -> dnorm[1]
// (block sums in `partial`: h->partial, or h->partial2 when it runs beside the solve)
template <bool C>
sr_status oz_gram(schur_refine_ctx *h, int n, double *partial = nullptr)
{
    using H = typename OzT<C>::H;
    const int s = oz_s(h);
    if (!partial) partial = h->partial;
    int blocks = 0;
    SR_TRY(sr::ozaki_product(h, h->st, h->oz, sr::OZS_COLS, sr::OZS_COLS, n, n, n, s, true, h->dflags));
    SR_TRY(sr::ozaki_combine(h, h->st, h->oz, sr::OZS_COLS, sr::OZS_COLS, n, n, s, 1.0, true,
                             typename OzT<C>::MinusI{(H *)h->Y, h->nmax}, partial, &blocks));
    SrPhase ph(h, SR_PROF_OTHER, 0, (long long)blocks * 8, 1);
    sr::reduce_partials_kernel<<<1, 256, 0, h->st>>>(partial, blocks, h->dnorm + 1);
    SR_CUDA_TRY(cudaGetLastError());
    return SR_OK;
}

// Starts the Gram product on gram_st after the work on st so far; the solve
// then runs on st beside it (the two share no buffer). oz_gram_join orders st
// after it again.
template <bool C>
sr_status oz_gram_fork(schur_refine_ctx *h, int n)
{
    SR_CUDA_TRY(cudaEventRecord(h->gev0, h->st));
    SR_CUDA_TRY(cudaStreamWaitEvent(h->gram_st, h->gev0, 0));
    cudaStream_t saved = h->st;
    h->st = h->gram_st;   // the phases' timing events follow the work
    const sr_status r = oz_gram<C>(h, n, h->partial2);
    h->st = saved;
    SR_TRY(r);
    SR_CUDA_TRY(cudaEventRecord(h->gev1, h->gram_st));
    return SR_OK;
}

sr_status oz_gram_join(schur_refine_ctx *h)
{
    SR_CUDA_TRY(cudaStreamWaitEvent(h->st, h->gev1, 0));
    return SR_OK;
}

// Q_new = Q + alpha * Q X (rows of Q, columns of X)
template <bool C>
sr_status oz_apply(schur_refine_ctx *h, int n, const void *Q, int ldq, const void *X, int ldx, void *Qn, int ldn,
                   double alpha)
{
    using H = typename OzT<C>::H;
    const int s = oz_s(h);
    SR_TRY(sr::ozaki_split(h, h->st, h->oz, sr::OZS_QROWS, n, n, Q, ldq, sr::OZ_ROWS, s));
    SR_TRY(sr::ozaki_split(h, h->st, h->oz, sr::OZS_X, n, n, X, ldx, sr::OZ_COLS, s));
    SR_TRY(sr::ozaki_product(h, h->st, h->oz, sr::OZS_QROWS, sr::OZS_X, n, n, n, s, false, h->dflags));
    return sr::ozaki_combine(h, h->st, h->oz, sr::OZS_QROWS, sr::OZS_X, n, n, s, 1.0, false,
                             typename OzT<C>::Update{(const H *)Q, ldq, (H *)Qn, ldn, alpha}, nullptr, nullptr);
}

template <bool C>
sr_status oz_ns_init(schur_refine_ctx *h, int n, const void *Q, int ldq, void *Qn, int ldn)
{
    SR_TRY(sr::ozaki_split(h, h->st, h->oz, sr::OZS_COLS, n, n, Q, ldq, sr::OZ_COLS, oz_s(h)));
    SR_TRY(oz_gram<C>(h, n));
    return oz_apply<C>(h, n, Q, ldq, h->Y, h->nmax, Qn, ldn, -0.5);
}

template <bool C>
sr_status oz_form_residual(schur_refine_ctx *h, int n, const void *Q, int ldq, void *That)
{
    using H = typename OzT<C>::H;
    using L = typename OzT<C>::L;
    const int s = oz_s(h), ld = h->nmax;
    int blocks = 0;
    SR_TRY(sr::ozaki_split(h, h->st, h->oz, sr::OZS_COLS, n, n, Q, ldq, sr::OZ_COLS, s));
    SR_TRY(sr::ozaki_product(h, h->st, h->oz, sr::OZS_ROWS, sr::OZS_COLS, n, n, n, s, false, h->dflags));
    SR_TRY(sr::ozaki_combine(h, h->st, h->oz, sr::OZS_ROWS, sr::OZS_COLS, n, n, s, 1.0, false,
                             typename OzT<C>::Store{(H *)h->AQ, ld}, nullptr, nullptr));
    SR_TRY(sr::ozaki_split(h, h->st, h->oz, sr::OZS_X, n, n, h->AQ, ld, sr::OZ_COLS, s));
    SR_TRY(sr::ozaki_product(h, h->st, h->oz, sr::OZS_COLS, sr::OZS_X, n, n, n, s, false, h->dflags));
    typename OzT<C>::Split sp{(L *)h->TE, ld, (H *)h->diag, (H *)That, n};
    if constexpr (!C) {
        if (h->opt.quasi) {
            sp.sub = h->band;
            sp.sup = h->band + h->nmax;
        }
    }
    SR_TRY(sr::ozaki_combine(h, h->st, h->oz, sr::OZS_COLS, sr::OZS_X, n, n, s, 1.0, false, sp, h->partial,
                             &blocks));
    return reduce_to(h, blocks, 0);
}

// ---- the real quasi-triangular form (opt.quasi) -----------------------------------
// After T^ is formed: its blocks from its band, the subdiagonal entries that
// are not couplings of 2 x 2 blocks added to ||E||^2 (dnorm[0], which the split
// epilogue summed below the subdiagonal), and the block array copied to the
// host for the solve's padded layout (read after the pass's synchronization).
sr_status quasi_detect(schur_refine_ctx *h, int n, double *norm)
{
    SrPhase ph(h, SR_PROF_OTHER, 0, 4LL * n * (long long)sizeof(double), 1);
    sr::quasi_blocks_kernel<<<1, 1024, 0, h->st>>>(n, h->diag, h->band, h->band + h->nmax, h->qblk, norm);
    SR_CUDA_TRY(cudaGetLastError());
    SR_CUDA_TRY(cudaMemcpyAsync(h->hblk, h->qblk, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, h->st));
    return SR_OK;
}

// S4 in the quasi-triangular form: the padded problem solved stepwise (the
// host's block array must be current: called after a synchronization).
template <typename Tl>
sr_status solve_quasi(schur_refine_ctx *h, int n, Tl *TE, int ld, const double *dhp)
{
    if constexpr (SrNum<Tl>::kind >= 2) {
        return SR_ERR_UNSUPPORTED;
    } else {
        std::vector<int> pos, inv, blkq;
        const int np = sr::quasi_pad_layout(n, h->hblk, pos, inv, blkq);
        if (np > h->nqmax) return SR_ERR_INVALID_ARG;
        // the maps go up through the pinned staging buffer (free again: the
        // previous upload finished before the last synchronization)
        int *hp = h->hmaps;
        std::copy(pos.begin(), pos.end(), hp);
        std::copy(inv.begin(), inv.end(), hp + n);
        std::copy(blkq.begin(), blkq.end(), hp + n + np);
        SR_CUDA_TRY(cudaMemcpyAsync(h->qpos, hp, (size_t)n * sizeof(int), cudaMemcpyHostToDevice, h->st));
        SR_CUDA_TRY(cudaMemcpyAsync(h->qinv, hp + n, (size_t)np * sizeof(int), cudaMemcpyHostToDevice, h->st));
        SR_CUDA_TRY(cudaMemcpyAsync(h->qblkq, hp + n + np, (size_t)np * sizeof(int), cudaMemcpyHostToDevice, h->st));
        Tl *TEq = (Tl *)h->TEq;
        const int ldq = h->nqmax;
        {
            SrPhase ph(h, SR_PROF_OTHER, 0, 2LL * np * np * (long long)sizeof(Tl), 1);
            const dim3 g((unsigned)((np + 31) / 32), (unsigned)((np + 31) / 32));
            sr::quasi_pad_kernel<Tl><<<g, 256, 0, h->st>>>(np, h->qinv, h->qblkq, TE, ld, dhp, TEq, ldq, h->dhpq,
                                                           (Tl *)h->qcpl);
            SR_CUDA_TRY(cudaGetLastError());
        }
        if (h->flow_acc && h->opt.solve_mode == 1) {
            // one launch: the dataflow over the tiles with block entries (on
            // request: the stepwise form measured faster here, 5.3 against 6.2 ms
            // per solve at n = 4096)
            SR_TRY(ensure_flow_plan(h, np));
            const long long fl = 2LL * np * np * np / 3;
            SrPhase ph(h, SR_PROF_SOLVE, fl, (long long)np * np * (long long)sizeof(Tl), 1);
            SR_CUDA_TRY(sr::trisolve_flow_launch<Tl>(h->st, np, TEq, ldq, h->dhpq, nullptr, h->dflags, h->flow,
                                                     h->flow_plan, h->flow_ntasks, (Tl *)h->flow_acc, ldq,
                                                     h->flow_ctas[SrNum<Tl>::kind], h->opt.l_cap, h->qblkq));
        } else {
            SR_TRY(ensure_plan(h, np, sr::kSolveTile));   // the padded order's 32-row tiles
            const int NB = (np + sr::kSolveTile - 1) / sr::kSolveTile;
            const long long fl = 2LL * np * np * np / 3;
            SrPhase ph(h, SR_PROF_SOLVE, fl, (long long)np * np * (long long)sizeof(Tl), 2LL * NB);
            SR_CUDA_TRY(sr::trisolve_quasi_launches<Tl>(h->st, h->aux_st, h->sev0, h->sev1, np, TEq, ldq, h->dhpq,
                                                        h->qblkq, (const Tl *)h->qcpl, h->dflags, h->plan, h->plan_off,
                                                        h->opt.l_cap));
        }
        {
            SrPhase ph(h, SR_PROF_OTHER, 0, 2LL * n * n * (long long)sizeof(Tl), 1);
            const dim3 g((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32));
            sr::quasi_unpad_kernel<Tl><<<g, 256, 0, h->st>>>(n, h->qpos, h->qblk, TEq, ldq, TE, ld);
            SR_CUDA_TRY(cudaGetLastError());
        }
        return SR_OK;
    }
}

template <bool C>
sr_status oz_update(schur_refine_ctx *h, int n, const void *Q, int ldq, void *Qn, int ldn, bool gram_done = false)
{
    using namespace sr;
    using H = typename OzT<C>::H;
    using L = typename OzT<C>::L;
    using Store = typename OzT<C>::Store;
    const int ld = h->nmax, sl = h->opt.lp_slices > 0 ? h->opt.lp_slices : kOzakiLpSlices;
    OzakiWork &w = h->oz;
    cudaStream_t st = h->st;
    H *Wd = (H *)h->Wd, *W2d = (H *)h->W2d, *W2Yd = (H *)h->W2Yd, *W2YWd = (H *)h->W2YWd, *Y = (H *)h->Y;
    if (!gram_done) SR_TRY(oz_gram<C>(h, n));   // Q unchanged since oz_form_residual: its column digits are current
    {
        SrPhase ph(h, SR_PROF_OTHER, 0, (long long)n * n * (long long)(sizeof(L) + sizeof(H)), 1);
        dim3 grid((n + 31) / 32, (n + 31) / 32);
        form_skew_kernel<L><<<grid, 256, 0, st>>>(n, (const L *)h->TE, ld, Wd, ld);
        SR_CUDA_TRY(cudaGetLastError());
    }
    H *YW = (H *)h->AQ;   // A Q is dead after the residual
    SR_TRY(ozaki_split(h, st, w, OZS_W, n, n, Wd, ld, OZ_COLS, sl));
    SR_TRY(ozaki_split(h, st, w, OZS_Y, n, n, Y, ld, OZ_COLS, sl));
    SR_TRY(ozaki_product(h, st, w, OZS_W, OZS_W, n, n, n, sl, true, h->dflags));
    SR_TRY(ozaki_combine(h, st, w, OZS_W, OZS_W, n, n, sl, -1.0, true, Store{W2d, ld}, nullptr, nullptr));
    SR_TRY(ozaki_product(h, st, w, OZS_Y, OZS_W, n, n, n, sl, false, h->dflags));
    SR_TRY(ozaki_combine(h, st, w, OZS_Y, OZS_W, n, n, sl, 1.0, false, Store{YW, ld}, nullptr, nullptr));
    SR_TRY(ozaki_split(h, st, w, OZS_W2, n, n, W2d, ld, OZ_COLS, sl));
    if (h->opt.full_sigma) {
        SR_TRY(ozaki_product(h, st, w, OZS_W2, OZS_Y, n, n, n, sl, false, h->dflags));
        SR_TRY(ozaki_combine(h, st, w, OZS_W2, OZS_Y, n, n, sl, 1.0, false, Store{W2Yd, ld}, nullptr, nullptr));
        SR_TRY(ozaki_split(h, st, w, 7, n, n, W2Yd, ld, OZ_ROWS, sl));
        SR_TRY(ozaki_product(h, st, w, 7, OZS_W, n, n, n, sl, false, h->dflags));
        SR_TRY(ozaki_combine(h, st, w, 7, OZS_W, n, n, sl, 1.0, false, Store{W2YWd, ld}, nullptr, nullptr));
    }
    SR_TRY(ozaki_product(h, st, w, OZS_W, OZS_W2, n, n, n, sl, false, h->dflags));
    typename OzT<C>::Delta ed{Wd, Y, YW, W2d, h->opt.full_sigma ? W2Yd : nullptr,
                              h->opt.full_sigma ? W2YWd : nullptr, ld, (H *)h->Delta, ld};
    SR_TRY(ozaki_combine(h, st, w, OZS_W, OZS_W2, n, n, sl, -1.0, false, ed, nullptr, nullptr));
    return oz_apply<C>(h, n, Q, ldq, h->Delta, ld, Qn, ldn, 0.5);
}

sr_status copy_q(schur_refine_ctx *h, int n, const void *src, int lds, void *dst, int ldd)
{
    if (src == dst) return SR_OK;
    const size_t es = hp_size(h->opt);
    SrPhase ph(h, SR_PROF_OTHER, 0, 2LL * n * n * (long long)es, 1);
    SR_CUDA_TRY(cudaMemcpy2DAsync(dst, (size_t)ldd * es, src, (size_t)lds * es, (size_t)n * es, n,
                                  cudaMemcpyDeviceToDevice, h->st));
    return SR_OK;
}

// One call of Alg. 4. Tl: low-precision type of the native path (float or
// double); C: complex data (emulated products only).
template <typename Tl, bool C>
sr_status run_step(schur_refine_ctx *h, int n, const void *A, int lda, void *dQ, int ldq, const void *dQhat,
                   void *dT, sr_norms *out)
{
    using H = typename OzT<C>::H;
    const int ld = h->nmax;
    const double tol = tol_of(h, n);
    const int max_iter = h->opt.max_iter > 0 ? h->opt.max_iter : 10;
    const bool oz = oz_pass(h);
    if (C && !oz) return SR_ERR_UNSUPPORTED;
    sr_norms nr{};
    nr.stril_rel = nr.orth = nr.w_norm = NAN;
    SR_CUDA_TRY(cudaMemsetAsync(h->dflags, 0, sizeof(int), h->st));
    SR_TRY(sumsq<H>(h, n, (const H *)A, lda, 0, 3));
    if (oz)   // rows of A: split once, used by every A Q of this call
        SR_TRY(sr::ozaki_split(h, h->st, h->oz, sr::OZS_ROWS, n, n, A, lda, sr::OZ_ROWS, oz_s(h)));

    // The working factor alternates between the caller's buffer and Qw.
    H *Qc = (H *)dQ, *Qo = (H *)h->Qw;
    int ldc = ldq, ldo = ld;
    double y_last = NAN;
    if (dQhat) {
        // Alg. 4: convert Qhat to hp, then Q <- 1/2 Qhat (3I - Qhat^H Qhat)
        {
            dim3 grid((n + 255) / 256, n);
            SrPhase ph(h, SR_PROF_OTHER, 0, 12LL * n * n * (C ? 2 : 1), 1);
            using Lq = typename OzT<C>::L;
            if (h->opt.qhat_type == SR_QHAT_FP32)
                sr::convert_to_hp_kernel<Lq><<<grid, 256, 0, h->st>>>(n, (const Lq *)dQhat, ldq, (H *)dQ, ldq);
            else
                sr::convert_to_hp_kernel<H><<<grid, 256, 0, h->st>>>(n, (const H *)dQhat, ldq, (H *)dQ, ldq);
            SR_CUDA_TRY(cudaGetLastError());
        }
        if (oz) {
            SR_TRY(oz_ns_init<C>(h, n, dQ, ldq, Qo, ldo));
        } else if constexpr (!C) {
            SR_TRY(hp_gemm(h, true, n, n, n, (const double *)dQ, ldq, (const double *)dQ, ldq,
                           sr::EpMinusI{h->Y, ld}, 1));
            SR_TRY(hp_gemm(h, false, n, n, n, (const double *)dQ, ldq, h->Y, ld,
                           sr::EpUpdate{(const double *)dQ, ldq, Qo, ldo, -0.5}, -1));
        }
        std::swap(Qc, Qo);
        std::swap(ldc, ldo);
        nr.hp_gemms += 2;
        SR_TRY(read_back(h));
        y_last = sqrt(h->hbuf[1]);
        nr.orth = y_last;
    }
    const double anorm = sqrt(h->hbuf[3] > 0 ? h->hbuf[3] : 1.0);
    sr_status status = SR_ERR_NOT_CONVERGED;
    double prev = INFINITY;
    for (int k = 1; k <= max_iter; ++k) {
        if (oz)
            SR_TRY(oz_form_residual<C>(h, n, Qc, ldc, dT));
        else if constexpr (!C)
            SR_TRY(form_residual<Tl>(h, n, (const double *)A, lda, Qc, ldc, (double *)dT));
        if (h->opt.quasi) SR_TRY(quasi_detect(h, n, h->dnorm));
        nr.hp_gemms += 2;
        nr.iters = k;
        SR_TRY(read_back(h));
        if (timed_out(h)) { status = SR_ERR_TIMEOUT; break; }
        const double anorm2 = sqrt(h->hbuf[3]);
        const double rT = sqrt(h->hbuf[0]) / (anorm2 > 0 ? anorm2 : anorm);
        nr.stril_rel = rT;
        if (!isfinite(rT)) { status = SR_ERR_NONFINITE; break; }
        const bool ok_y = !(y_last > sqrt(tol));   // NaN (not measured) passes
        if (rT <= tol && ok_y) { status = SR_OK; break; }
        if (k >= 3 && rT > 10.0 * prev) { status = SR_ERR_NOT_CONVERGED; break; }
        prev = rT;
        if (oz) SR_TRY(oz_gram_fork<C>(h, n));   // Y = Q^H Q - I beside the solve
        if constexpr (C) {
            SR_TRY(solve<cf>(h, n, (cf *)h->TE, ld, (const cd *)h->diag));
            SR_TRY(sumsq<cf>(h, n, (const cf *)h->TE, ld, 1, 2));
        } else {
            if (h->opt.quasi)
                SR_TRY(solve_quasi<Tl>(h, n, (Tl *)h->TE, ld, h->diag));
            else
                SR_TRY(solve<Tl>(h, n, (Tl *)h->TE, ld, h->diag));
            SR_TRY(sumsq<Tl>(h, n, (const Tl *)h->TE, ld, 1, 2));
        }
        if (oz) SR_TRY(oz_gram_join(h));
        SR_TRY(read_back(h));
        const int f = host_flags(h);
        if (f & SR_FLAG_TIMEOUT) { status = SR_ERR_TIMEOUT; break; }
        if (f & SR_FLAG_NONDISTINCT) { status = SR_ERR_NONDISTINCT; break; }
        if (f & SR_FLAG_NONFINITE) { status = SR_ERR_NONFINITE; break; }
        nr.w_norm = sqrt(2.0 * h->hbuf[2]);
        if (oz)
            SR_TRY(oz_update<C>(h, n, Qc, ldc, Qo, ldo, true));
        else if constexpr (!C)
            SR_TRY(update<Tl>(h, n, Qc, ldc, Qo, ldo));
        nr.hp_gemms += 2;
        std::swap(Qc, Qo);
        std::swap(ldc, ldo);
        SR_TRY(read_back(h));
        y_last = sqrt(h->hbuf[1]);
        nr.orth = y_last;
        status = SR_ERR_NOT_CONVERGED;
    }
    SR_TRY(copy_q(h, n, Qc, ldc, dQ, ldq));
    SR_CUDA_TRY(cudaStreamSynchronize(h->st));
    harvest(h);
    if (out) *out = nr;
    return status;
}

// ---- graph mode: the whole call as one CUDA graph with a device-side loop ------------
// The REPEAT loop of Alg. 4 becomes a conditional WHILE node whose body holds two
// passes (Q in the caller's buffer, then in Qw: the buffers are fixed in a graph);
// the decisions of the host loop (stop test, divergence guard, solve failures,
// max_iter) are taken by one-thread control kernels that set the conditional
// values of the enclosing WHILE and of the IF nodes that guard the solve and the
// update. Results are the same as the host loop's.

struct SrCtl {
    int k, status, iters, hp_gemms, max_iter, loc;
    double prev, y_last, rT, orth, w_norm, tol;
};

__global__ void ctl_start_kernel(SrCtl *c, const double *__restrict__ dnorm, int has_qhat, double tol, int max_iter)
{
    c->k = 0;
    c->status = SR_ERR_NOT_CONVERGED;
    c->iters = 0;
    c->hp_gemms = has_qhat ? 2 : 0;
    c->max_iter = max_iter;
    c->loc = 0;
    c->prev = INFINITY;
    c->y_last = has_qhat ? sqrt(dnorm[1]) : NAN;
    c->orth = c->y_last;
    c->rT = NAN;
    c->w_norm = NAN;
    c->tol = tol;
}

// after T^: the stop test and the divergence guard of schur_refine_step
__global__ void ctl_residual_kernel(SrCtl *c, const double *__restrict__ dnorm, const int *__restrict__ flags,
                                    cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hb,
                                    cudaGraphConditionalHandle hu, int set_hb)
{
    const int k = ++c->k;
    c->iters = k;
    c->hp_gemms += 2;
    const double an = sqrt(dnorm[3]);
    const double rT = sqrt(dnorm[0]) / (an > 0 ? an : 1.0);
    c->rT = rT;
    bool stop = true;
    int st = SR_ERR_NOT_CONVERGED;
    if (*flags & SR_FLAG_TIMEOUT) st = SR_ERR_TIMEOUT;
    else if (!isfinite(rT)) st = SR_ERR_NONFINITE;
    else if (rT <= c->tol && !(c->y_last > sqrt(c->tol))) st = SR_OK;
    else if (k >= 3 && rT > 10.0 * c->prev) st = SR_ERR_NOT_CONVERGED;
    else { stop = false; c->prev = rT; }
    c->status = st;
    const unsigned go = (!stop && k < c->max_iter) ? 1u : 0u;
    cudaGraphSetConditional(hu, stop ? 0u : 1u);
    cudaGraphSetConditional(hw, go);
    if (set_hb) cudaGraphSetConditional(hb, go);
}

// after the solve: a zero divisor or a non-finite L ends the call before the update
__global__ void ctl_solve_kernel(SrCtl *c, const double *__restrict__ dnorm, const int *__restrict__ flags,
                                 cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hb,
                                 cudaGraphConditionalHandle hu, int set_hb)
{
    const int f = *flags;
    unsigned ok = 1;
    if (f & SR_FLAG_TIMEOUT) { c->status = SR_ERR_TIMEOUT; ok = 0; }
    else if (f & SR_FLAG_NONDISTINCT) { c->status = SR_ERR_NONDISTINCT; ok = 0; }
    else if (f & SR_FLAG_NONFINITE) { c->status = SR_ERR_NONFINITE; ok = 0; }
    else c->w_norm = sqrt(2.0 * dnorm[2]);
    cudaGraphSetConditional(hu, ok);
    if (!ok) {
        cudaGraphSetConditional(hw, 0u);
        if (set_hb) cudaGraphSetConditional(hb, 0u);
    }
}

__global__ void ctl_update_kernel(SrCtl *c, const double *__restrict__ dnorm, int loc)
{
    c->hp_gemms += 2;
    c->y_last = sqrt(dnorm[1]);
    c->orth = c->y_last;
    c->loc = loc;
    c->status = SR_ERR_NOT_CONVERGED;
}

// the caller's Q <- Qw when the last update left the factor in Qw
__global__ void ctl_copy_kernel(const SrCtl *c, int n, const double *__restrict__ src, int lds, double *__restrict__ dst,
                                int ldd)
{
    if (c->loc != 1) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i < n) dst[sr_idx(i, j, ldd)] = src[sr_idx(i, j, lds)];
}

// a conditional handle of the graph being captured on h->st
sr_status cond_handle(schur_refine_ctx *h, unsigned defval, cudaGraphConditionalHandle *out)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    SR_CUDA_TRY(cudaStreamGetCaptureInfo(h->st, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    if (cs != cudaStreamCaptureStatusActive) return SR_ERR_CUDA;
    SR_CUDA_TRY(cudaGraphConditionalHandleCreate(out, g, defval, cudaGraphCondAssignDefault));
    return SR_OK;
}

// Adds a conditional node (WHILE or IF on handle hd) after the work captured so
// far on h->st and captures body() into it on the capture stream of this depth.
template <class F>
sr_status cond_node(schur_refine_ctx *h, int depth, cudaGraphConditionalNodeType type, cudaGraphConditionalHandle hd,
                    F body)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    SR_CUDA_TRY(cudaStreamGetCaptureInfo(h->st, &cs, nullptr, &g, &deps, nullptr, &nd));
    if (cs != cudaStreamCaptureStatusActive) return SR_ERR_CUDA;
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = hd;
    p.conditional.type = type;
    p.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    SR_CUDA_TRY(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
    SR_CUDA_TRY(cudaStreamUpdateCaptureDependencies(h->st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    while ((int)h->cstreams.size() <= depth) {
        cudaStream_t s = nullptr;
        SR_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        h->cstreams.push_back(s);
    }
    cudaStream_t bs = h->cstreams[depth], saved = h->st;
    SR_CUDA_TRY(cudaStreamBeginCaptureToGraph(bs, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeRelaxed));
    h->st = bs;
    const sr_status r = body();
    h->st = saved;
    cudaGraph_t done = nullptr;
    const cudaError_t e = cudaStreamEndCapture(bs, &done);
    if (r != SR_OK) return r;
    SR_CUDA_TRY(e);
    return SR_OK;
}

// one pass of the REPEAT loop inside the graph: Qc -> Qo; loc = the buffer the update leaves Q in
template <typename Tl>
sr_status graph_pass(schur_refine_ctx *h, int depth, int n, const double *A, int lda, double *Qc, int ldc, double *Qo,
                     int ldo, double *dT, int loc, cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hb,
                     int set_hb)
{
    SrCtl *c = (SrCtl *)h->ctl;
    const bool oz = oz_pass(h);
    if (oz)
        SR_TRY(oz_form_residual<false>(h, n, Qc, ldc, dT));
    else
        SR_TRY(form_residual<Tl>(h, n, A, lda, Qc, ldc, dT));
    cudaGraphConditionalHandle hu = 0;
    SR_TRY(cond_handle(h, 0, &hu));
    ctl_residual_kernel<<<1, 1, 0, h->st>>>(c, h->dnorm, h->dflags, hw, hb, hu, set_hb);
    SR_CUDA_TRY(cudaGetLastError());
    return cond_node(h, depth, cudaGraphCondTypeIf, hu, [&]() -> sr_status {
        SR_TRY(solve<Tl>(h, n, (Tl *)h->TE, h->nmax, h->diag));
        SR_TRY(sumsq<Tl>(h, n, (const Tl *)h->TE, h->nmax, 1, 2));
        cudaGraphConditionalHandle hu2 = 0;
        SR_TRY(cond_handle(h, 0, &hu2));
        ctl_solve_kernel<<<1, 1, 0, h->st>>>(c, h->dnorm, h->dflags, hw, hb, hu2, set_hb);
        SR_CUDA_TRY(cudaGetLastError());
        return cond_node(h, depth + 1, cudaGraphCondTypeIf, hu2, [&]() -> sr_status {
            if (oz)
                SR_TRY(oz_update<false>(h, n, Qc, ldc, Qo, ldo));
            else
                SR_TRY(update<Tl>(h, n, Qc, ldc, Qo, ldo));
            ctl_update_kernel<<<1, 1, 0, h->st>>>(c, h->dnorm, loc);
            SR_CUDA_TRY(cudaGetLastError());
            return SR_OK;
        });
    });
}

template <typename Tl>
sr_status build_refine_graph(schur_refine_ctx *h, int n, const void *dA, int lda, void *dQ, int ldq,
                             const void *dQhat, void *dT)
{
    const int ld = h->nmax;
    const double tol = tol_of(h, n);
    const int max_iter = h->opt.max_iter > 0 ? h->opt.max_iter : 10;
    const bool oz = oz_pass(h);
    double *Q = (double *)dQ, *Qw = h->Qw;
    const double *A = (const double *)dA;
    if (!h->ctl) SR_CUDA_TRY(cudaMalloc(&h->ctl, sizeof(SrCtl)));
    SR_TRY(ensure_plan(h, n, sr::StepTile<Tl>::B));   // host work and a synchronization: not inside a capture
    SR_TRY(ensure_flow_plan(h, n));
    while (h->cstreams.empty()) {
        cudaStream_t s = nullptr;
        SR_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        h->cstreams.push_back(s);
    }
    cudaStream_t top = h->cstreams[0], saved = h->st;
    // depth 0 is the top-level capture; conditional bodies use depths 1..4
    SR_CUDA_TRY(cudaStreamBeginCapture(top, cudaStreamCaptureModeRelaxed));
    h->st = top;
    h->capturing = true;
    auto body = [&]() -> sr_status {
        SR_CUDA_TRY(cudaMemsetAsync(h->dflags, 0, sizeof(int), h->st));
        SR_TRY(sumsq<double>(h, n, A, lda, 0, 3));
        if (oz) SR_TRY(sr::ozaki_split(h, h->st, h->oz, sr::OZS_ROWS, n, n, A, lda, sr::OZ_ROWS, oz_s(h)));
        if (dQhat) {
            dim3 grid((n + 255) / 256, n);
            if (h->opt.qhat_type == SR_QHAT_FP32)
                sr::convert_to_hp_kernel<float><<<grid, 256, 0, h->st>>>(n, (const float *)dQhat, ldq, Q, ldq);
            else
                sr::convert_to_hp_kernel<double><<<grid, 256, 0, h->st>>>(n, (const double *)dQhat, ldq, Q, ldq);
            SR_CUDA_TRY(cudaGetLastError());
            if (oz) {
                SR_TRY(oz_ns_init<false>(h, n, Q, ldq, Qw, ld));
            } else {
                SR_TRY(hp_gemm(h, true, n, n, n, (const double *)Q, ldq, (const double *)Q, ldq,
                               sr::EpMinusI{h->Y, ld}, 1));
                SR_TRY(hp_gemm(h, false, n, n, n, (const double *)Q, ldq, h->Y, ld,
                               sr::EpUpdate{(const double *)Q, ldq, Qw, ld, -0.5}, -1));
            }
            SR_CUDA_TRY(cudaMemcpy2DAsync(Q, (size_t)ldq * 8, Qw, (size_t)ld * 8, (size_t)n * 8, n,
                                          cudaMemcpyDeviceToDevice, h->st));
        }
        ctl_start_kernel<<<1, 1, 0, h->st>>>((SrCtl *)h->ctl, h->dnorm, dQhat ? 1 : 0, tol, max_iter);
        SR_CUDA_TRY(cudaGetLastError());
        cudaGraphConditionalHandle hw = 0;
        SR_TRY(cond_handle(h, 1, &hw));
        SR_TRY(cond_node(h, 1, cudaGraphCondTypeWhile, hw, [&]() -> sr_status {
            cudaGraphConditionalHandle hb = 0;
            SR_TRY(cond_handle(h, 0, &hb));
            SR_TRY(graph_pass<Tl>(h, 2, n, A, lda, Q, ldq, Qw, ld, (double *)dT, 1, hw, hb, 1));
            return cond_node(h, 2, cudaGraphCondTypeIf, hb, [&]() -> sr_status {
                return graph_pass<Tl>(h, 3, n, A, lda, Qw, ld, Q, ldq, (double *)dT, 0, hw, hb, 0);
            });
        }));
        dim3 grid((n + 255) / 256, n);
        ctl_copy_kernel<<<grid, 256, 0, h->st>>>((const SrCtl *)h->ctl, n, Qw, ld, Q, ldq);
        SR_CUDA_TRY(cudaGetLastError());
        return SR_OK;
    };
    const sr_status r = body();
    h->st = saved;
    h->capturing = false;
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(top, &graph);
    if (r != SR_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (r != SR_OK) return r;
        sr_set_last_cuda_error(e);
        return SR_ERR_CUDA;
    }
    auto &rg = h->rgraph;
    if (rg.exec) cudaGraphExecDestroy(rg.exec);
    if (rg.graph) cudaGraphDestroy(rg.graph);
    rg = schur_refine_ctx::RefineGraph{};
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    if (ei != cudaSuccess) {
        cudaGraphDestroy(graph);
        sr_set_last_cuda_error(ei);
        cudaGetLastError();
        return SR_ERR_CUDA;
    }
    rg.n = n; rg.lda = lda; rg.ldq = ldq; rg.A = dA; rg.Q = dQ; rg.Qhat = dQhat; rg.T = dT;
    rg.graph = graph;
    rg.exec = exec;
    return SR_OK;
}

template <typename Tl>
sr_status run_step_graph(schur_refine_ctx *h, int n, const void *dA, int lda, void *dQ, int ldq, const void *dQhat,
                         void *dT, sr_norms *out)
{
    auto &rg = h->rgraph;
    if (!(rg.exec && rg.n == n && rg.lda == lda && rg.ldq == ldq && rg.A == dA && rg.Q == dQ && rg.Qhat == dQhat &&
          rg.T == dT))
        SR_TRY(build_refine_graph<Tl>(h, n, dA, lda, dQ, ldq, dQhat, dT));
    SR_CUDA_TRY(cudaGraphLaunch(rg.exec, h->st));
    SrCtl c{};
    SR_CUDA_TRY(cudaMemcpyAsync(h->hbuf, h->ctl, sizeof(SrCtl), cudaMemcpyDeviceToHost, h->st));
    SR_CUDA_TRY(cudaStreamSynchronize(h->st));
    memcpy(&c, h->hbuf, sizeof(SrCtl));
    if (out) {
        out->stril_rel = c.rT;
        out->orth = c.orth;
        out->w_norm = c.w_norm;
        out->iters = c.iters;
        out->hp_gemms = c.hp_gemms;
    }
    return (sr_status)c.status;
}

// ---- double-double working precision (target SR_TARGET_DD) --------------------------
// Alg. 4 with hp = double-double and lp = FP64. A double-double matrix of the
// caller is two planes, the low one ld * n elements after the high one; the
// workspace's planes are nmax * nmax elements apart.

struct DdMat {
    double *hi, *lo;
    int ld;
};
// a triple-double matrix: three planes (caller: ld * n elements apart)
struct TdMat {
    double *x0, *x1, *x2;
    int ld;
};

bool is_dd(const sr_options &o) { return o.target == SR_TARGET_DD; }
int oz_s_dd(const schur_refine_ctx *h) { return oz_count(h->opt); }

DdMat dd_caller(const void *p, int ld, int n)
{
    double *hi = (double *)p;
    return {hi, hi + (size_t)ld * (size_t)n, ld};
}
DdMat dd_work(const schur_refine_ctx *h, double *p)
{
    return {p, p + (size_t)h->nmax * (size_t)h->nmax, h->nmax};
}

// C = op(A) B with the SIMT double-double kernel; epilogue ep, norms to dnorm[slot]
template <class EP>
sr_status ddk_gemm(schur_refine_ctx *h, bool transA, int m, int n, int k, DdMat A, DdMat B, EP ep, int slot)
{
    double *part = slot >= 0 ? h->partial : nullptr;
    {
        SrPhase ph(h, SR_PROF_HP_GEMM, 2LL * m * n * k, 16LL * ((long long)m * k + (long long)k * n + (long long)m * n),
                   1);
        const sr::LoadNDD lb{B.hi, B.lo, B.ld};
        cudaError_t e;
        if (transA)
            e = sr::gemm_ddk(h->st, m, n, k, sr::LoadTDD{A.hi, A.lo, A.ld}, lb, ep, part);
        else
            e = sr::gemm_ddk(h->st, m, n, k, sr::LoadNDD{A.hi, A.lo, A.ld}, lb, ep, part);
        SR_CUDA_TRY(e);
    }
    if (slot >= 0) SR_TRY(reduce_to(h, sr::ddk_blocks(m, n), slot));
    return SR_OK;
}

// emulated: split a double-double matrix into the handle's hp digits
sr_status oz_split_dd(schur_refine_ctx *h, int slot, int n, DdMat X, int layout)
{
    return sr::ozaki_split_dd(h, h->st, h->oz, slot, n, n, X.hi, X.lo, X.ld, layout, oz_s_dd(h));
}

// Y = Q^T Q - I (double-double) and ||Y||^2 -> dnorm[1]; emulated: from the
// column digits of Q in slot OZS_COLS
template <bool OZ>
sr_status dd_gram(schur_refine_ctx *h, int n, DdMat Q)
{
    const DdMat Y = dd_work(h, h->Y);
    const sr::EpMinusIDD ep{Y.hi, Y.lo, Y.ld};
    if constexpr (OZ) {
        const int s = oz_s_dd(h);
        int blocks = 0;
        SR_TRY(sr::ozaki_product(h, h->st, h->oz, sr::OZS_COLS, sr::OZS_COLS, n, n, n, s, true, h->dflags));
        SR_TRY(sr::ozaki_combine(h, h->st, h->oz, sr::OZS_COLS, sr::OZS_COLS, n, n, s, 1.0, true, ep, h->partial,
                                 &blocks));
        return reduce_to(h, blocks, 1);
    } else {
        return ddk_gemm(h, true, n, n, n, Q, Q, ep, 1);
    }
}

// Qn = Q + alpha Q X in double-double
template <bool OZ>
sr_status dd_apply(schur_refine_ctx *h, int n, DdMat Q, DdMat X, DdMat Qn, double alpha)
{
    const sr::EpUpdateDD ep{Q.hi, Q.lo, Q.ld, Qn.hi, Qn.lo, Qn.ld, alpha};
    if constexpr (OZ) {
        const int s = oz_s_dd(h);
        SR_TRY(oz_split_dd(h, sr::OZS_QROWS, n, Q, sr::OZ_ROWS));
        SR_TRY(oz_split_dd(h, sr::OZS_X, n, X, sr::OZ_COLS));
        SR_TRY(sr::ozaki_product(h, h->st, h->oz, sr::OZS_QROWS, sr::OZS_X, n, n, n, s, false, h->dflags));
        return sr::ozaki_combine(h, h->st, h->oz, sr::OZS_QROWS, sr::OZS_X, n, n, s, 1.0, false, ep, nullptr,
                                 nullptr);
    } else {
        return ddk_gemm(h, false, n, n, n, Q, X, ep, -1);
    }
}

// S1 + S2 in double-double: A Q, T^ = Q^T (A Q) split into TE (FP64) and the
// double-double diagonal; ||E||^2 -> dnorm[0]
template <bool OZ>
sr_status dd_form_residual(schur_refine_ctx *h, int n, DdMat A, DdMat Q, DdMat That)
{
    const DdMat AQ = dd_work(h, h->AQ);
    const int ld = h->nmax;
    const sr::EpSplitDD ep{(double *)h->TE, ld, h->diag, h->diag_lo, That.hi, That.lo, That.ld};
    if constexpr (OZ) {
        const int s = oz_s_dd(h);
        int blocks = 0;
        SR_TRY(oz_split_dd(h, sr::OZS_COLS, n, Q, sr::OZ_COLS));
        SR_TRY(sr::ozaki_product(h, h->st, h->oz, sr::OZS_ROWS, sr::OZS_COLS, n, n, n, s, false, h->dflags));
        SR_TRY(sr::ozaki_combine(h, h->st, h->oz, sr::OZS_ROWS, sr::OZS_COLS, n, n, s, 1.0, false,
                                 sr::EpStoreDD{AQ.hi, AQ.lo, AQ.ld}, nullptr, nullptr));
        SR_TRY(oz_split_dd(h, sr::OZS_X, n, AQ, sr::OZ_COLS));
        SR_TRY(sr::ozaki_product(h, h->st, h->oz, sr::OZS_COLS, sr::OZS_X, n, n, n, s, false, h->dflags));
        SR_TRY(sr::ozaki_combine(h, h->st, h->oz, sr::OZS_COLS, sr::OZS_X, n, n, s, 1.0, false, ep, h->partial,
                                 &blocks));
        return reduce_to(h, blocks, 0);
    } else {
        SR_TRY(ddk_gemm(h, false, n, n, n, A, Q, sr::EpStoreDD{AQ.hi, AQ.lo, AQ.ld}, -1));
        return ddk_gemm(h, true, n, n, n, Q, AQ, ep, 0);
    }
}

// S5-S8 in double-double: Y, W = L - L^T (FP64), YW, W^2, W^3 in FP64,
// Delta = Sigma - 2I in double-double, Q_new = Q + 1/2 Q Delta
template <bool OZ>
sr_status dd_update(schur_refine_ctx *h, int n, DdMat Q, DdMat Qn)
{
    using namespace sr;
    const int ld = h->nmax;
    cudaStream_t st = h->st;
    SR_TRY(dd_gram<OZ>(h, n, Q));   // emulated: Q's column digits are those of the residual
    const DdMat Y = dd_work(h, h->Y), Dl = dd_work(h, h->Delta);
    double *Wd = h->Wd, *W2 = (double *)h->W2, *YW = (double *)h->YW;
    double *W2Y = (double *)h->W2Y, *W2YW = (double *)h->W2YW;
    {
        SrPhase ph(h, SR_PROF_OTHER, 0, 16LL * n * n, 1);
        dim3 grid((n + 31) / 32, (n + 31) / 32);
        form_skew_kernel<double><<<grid, 256, 0, st>>>(n, (const double *)h->TE, ld, Wd, ld);
        SR_CUDA_TRY(cudaGetLastError());
    }
    const bool full = h->opt.full_sigma != 0;
    EpDeltaDD ed{Wd, YW, W2, full ? W2Y : nullptr, full ? W2YW : nullptr, ld, Y.hi, Y.lo, Y.ld, Dl.hi, Dl.lo, Dl.ld};
    if constexpr (OZ) {
        // FP64-class emulated products (7 digits): W^2 = -W^T W, YW = Y^T W,
        // W^3 = -W^T W^2, with Y rounded to FP64 (its high plane)
        const int sl = kOzakiDefaultSlices;
        OzakiWork &w = h->oz;
        SR_TRY(ozaki_split(h, st, w, OZS_W, n, n, Wd, ld, OZ_COLS, sl));
        SR_TRY(ozaki_split(h, st, w, OZS_Y, n, n, Y.hi, ld, OZ_COLS, sl));
        SR_TRY(ozaki_product(h, st, w, OZS_W, OZS_W, n, n, n, sl, true, h->dflags));
        SR_TRY(ozaki_combine(h, st, w, OZS_W, OZS_W, n, n, sl, -1.0, true, EpStore{W2, ld}, nullptr, nullptr));
        SR_TRY(ozaki_product(h, st, w, OZS_Y, OZS_W, n, n, n, sl, false, h->dflags));
        SR_TRY(ozaki_combine(h, st, w, OZS_Y, OZS_W, n, n, sl, 1.0, false, EpStore{YW, ld}, nullptr, nullptr));
        SR_TRY(ozaki_split(h, st, w, OZS_W2, n, n, W2, ld, OZ_COLS, sl));
        if (full) {
            SR_TRY(ozaki_product(h, st, w, OZS_W2, OZS_Y, n, n, n, sl, false, h->dflags));
            SR_TRY(ozaki_combine(h, st, w, OZS_W2, OZS_Y, n, n, sl, 1.0, false, EpStore{W2Y, ld}, nullptr, nullptr));
            SR_TRY(ozaki_split(h, st, w, 7, n, n, W2Y, ld, OZ_ROWS, sl));
            SR_TRY(ozaki_product(h, st, w, 7, OZS_W, n, n, n, sl, false, h->dflags));
            SR_TRY(ozaki_combine(h, st, w, 7, OZS_W, n, n, sl, 1.0, false, EpStore{W2YW, ld}, nullptr, nullptr));
        }
        SR_TRY(ozaki_product(h, st, w, OZS_W, OZS_W2, n, n, n, sl, false, h->dflags));
        SR_TRY(ozaki_combine(h, st, w, OZS_W, OZS_W2, n, n, sl, -1.0, false, ed, nullptr, nullptr));
    } else {
        const long long f1 = 2LL * n * n * n, b1 = 32LL * n * n;
        SrPhase ph(h, SR_PROF_LP_GEMM, f1 * (full ? 5 : 3), b1 * (full ? 5 : 3), full ? 5 : 3);
        const LoadN<double, double> w{Wd, ld};
        SR_CUDA_TRY(gemm_simt<double>(st, n, n, n, w, w, EpStoreLp<double>{W2, ld}, nullptr));
        SR_CUDA_TRY(gemm_simt<double>(st, n, n, n, LoadN<double, double>{Y.hi, ld}, w, EpStoreLp<double>{YW, ld},
                                      nullptr));
        if (full) {
            SR_CUDA_TRY(gemm_simt<double>(st, n, n, n, LoadN<double, double>{W2, ld},
                                          LoadN<double, double>{Y.hi, ld}, EpStoreLp<double>{W2Y, ld}, nullptr));
            SR_CUDA_TRY(gemm_simt<double>(st, n, n, n, LoadN<double, double>{W2Y, ld}, w,
                                          EpStoreLp<double>{W2YW, ld}, nullptr));
        }
        SR_CUDA_TRY(gemm_simt<double>(st, n, n, n, w, LoadN<double, double>{W2, ld}, ed, nullptr));
    }
    return dd_apply<OZ>(h, n, Q, Dl, Qn, 0.5);
}

sr_status copy_dd(schur_refine_ctx *h, int n, DdMat src, DdMat dst)
{
    if (src.hi == dst.hi) return SR_OK;
    SrPhase ph(h, SR_PROF_OTHER, 0, 32LL * n * n, 2);
    SR_CUDA_TRY(cudaMemcpy2DAsync(dst.hi, (size_t)dst.ld * 8, src.hi, (size_t)src.ld * 8, (size_t)n * 8, n,
                                  cudaMemcpyDeviceToDevice, h->st));
    SR_CUDA_TRY(cudaMemcpy2DAsync(dst.lo, (size_t)dst.ld * 8, src.lo, (size_t)src.ld * 8, (size_t)n * 8, n,
                                  cudaMemcpyDeviceToDevice, h->st));
    return SR_OK;
}

// One call of Alg. 4 with the double-double target. OZ: emulated products.
template <bool OZ>
sr_status run_step_dd(schur_refine_ctx *h, int n, const void *dA, int lda, void *dQ, int ldq, const void *dQhat,
                      void *dT, sr_norms *out)
{
    const int ld = h->nmax;
    const double tol = h->opt.tol > 0 ? h->opt.tol : 1e-28 * (double)n;
    const int max_iter = h->opt.max_iter > 0 ? h->opt.max_iter : 10;
    sr_norms nr{};
    nr.stril_rel = nr.orth = nr.w_norm = NAN;
    const DdMat A = dd_caller(dA, lda, n), Qcaller = dd_caller(dQ, ldq, n);
    const DdMat That = dT ? dd_caller(dT, n, n) : DdMat{nullptr, nullptr, n};
    SR_CUDA_TRY(cudaMemsetAsync(h->dflags, 0, sizeof(int), h->st));
    SR_TRY(sumsq<double>(h, n, A.hi, lda, 0, 3));
    if constexpr (OZ) SR_TRY(oz_split_dd(h, sr::OZS_ROWS, n, A, sr::OZ_ROWS));
    DdMat Qc = Qcaller, Qo = dd_work(h, h->Qw);
    double y_last = NAN;
    if (dQhat) {
        // Alg. 4: Qhat (FP64) to double-double, then Q <- Q - 1/2 Q (Q^T Q - I) (eq. NS)
        {
            dim3 grid((n + 255) / 256, n);
            SrPhase ph(h, SR_PROF_OTHER, 0, 24LL * n * n, 1);
            sr::to_dd_kernel<<<grid, 256, 0, h->st>>>(n, (const double *)dQhat, ldq, Qc.hi, Qc.lo, Qc.ld);
            SR_CUDA_TRY(cudaGetLastError());
        }
        if constexpr (OZ) SR_TRY(oz_split_dd(h, sr::OZS_COLS, n, Qc, sr::OZ_COLS));
        SR_TRY(dd_gram<OZ>(h, n, Qc));
        SR_TRY(dd_apply<OZ>(h, n, Qc, dd_work(h, h->Y), Qo, -0.5));
        std::swap(Qc, Qo);
        nr.hp_gemms += 2;
        SR_TRY(read_back(h));
        y_last = sqrt(h->hbuf[1]);
        nr.orth = y_last;
    }
    const double anorm = sqrt(h->hbuf[3] > 0 ? h->hbuf[3] : 1.0);
    sr_status status = SR_ERR_NOT_CONVERGED;
    double prev = INFINITY;
    for (int k = 1; k <= max_iter; ++k) {
        SR_TRY(dd_form_residual<OZ>(h, n, A, Qc, That));
        nr.hp_gemms += 2;
        nr.iters = k;
        SR_TRY(read_back(h));
        if (timed_out(h)) { status = SR_ERR_TIMEOUT; break; }
        const double rT = sqrt(h->hbuf[0]) / anorm;
        nr.stril_rel = rT;
        if (!isfinite(rT)) { status = SR_ERR_NONFINITE; break; }
        const bool ok_y = !(y_last > sqrt(tol));
        if (rT <= tol && ok_y) { status = SR_OK; break; }
        if (k >= 3 && rT > 10.0 * prev) { status = SR_ERR_NOT_CONVERGED; break; }
        prev = rT;
        SR_TRY(solve<double>(h, n, (double *)h->TE, ld, h->diag, h->diag_lo));
        SR_TRY(sumsq<double>(h, n, (const double *)h->TE, ld, 1, 2));
        SR_TRY(read_back(h));
        const int f = host_flags(h);
        if (f & SR_FLAG_TIMEOUT) { status = SR_ERR_TIMEOUT; break; }
        if (f & SR_FLAG_NONDISTINCT) { status = SR_ERR_NONDISTINCT; break; }
        if (f & SR_FLAG_NONFINITE) { status = SR_ERR_NONFINITE; break; }
        nr.w_norm = sqrt(2.0 * h->hbuf[2]);
        SR_TRY(dd_update<OZ>(h, n, Qc, Qo));
        nr.hp_gemms += 2;
        std::swap(Qc, Qo);
        SR_TRY(read_back(h));
        y_last = sqrt(h->hbuf[1]);
        nr.orth = y_last;
        status = SR_ERR_NOT_CONVERGED;
    }
    SR_TRY(copy_dd(h, n, Qc, Qcaller));
    SR_CUDA_TRY(cudaStreamSynchronize(h->st));
    harvest(h);
    if (out) *out = nr;
    return status;
}

// ---- the triple-double target (SR_TARGET_TD) -----------------------------------------
// Sec. 3 refines to working precisions above double-double by holding each
// high-precision number as several doubles; here three (about 159 bits), the
// most that one set of moduli <= 256 carries: the products are the residue
// form with 48 moduli (t = 162-bit operands at K <= 4096), rebuilt into
// 12-limb integers and rounded once to triple-doubles; the sums of the
// epilogues are exact and rounded once. The low precision is FP64 (solve with
// divisors from the two leading words of the diagonal, FP64-class products YW,
// W^2, W^3 with 7 digits), as in the double-double form.
bool is_td(const sr_options &o) { return o.target == SR_TARGET_TD; }

TdMat td_caller(const void *p, int ld, int n)
{
    double *a = (double *)p;
    const size_t pl = (size_t)ld * (size_t)n;
    return {a, a + pl, a + 2 * pl, ld};
}
TdMat td_work(const schur_refine_ctx *h, double *p)
{
    const size_t pl = (size_t)h->nmax * (size_t)h->nmax;
    return {p, p + pl, p + 2 * pl, h->nmax};
}

sr_status td_split(schur_refine_ctx *h, int slot, int n, TdMat X, int layout)
{
    return sr::ozaki_split_td(h, h->st, h->oz, slot, n, n, X.x0, X.x1, X.x2, X.ld, layout, sr::kCrtDefaultModuliTD);
}

// Y = Q^T Q - I and ||Y||^2 -> dnorm[1], from the column residues of Q in OZS_COLS
sr_status td_gram(schur_refine_ctx *h, int n)
{
    const int s = sr::kCrtDefaultModuliTD;
    const TdMat Y = td_work(h, h->Y);
    int blocks = 0;
    SR_TRY(sr::ozaki_product(h, h->st, h->oz, sr::OZS_COLS, sr::OZS_COLS, n, n, n, s, true, h->dflags));
    SR_TRY(sr::ozaki_combine(h, h->st, h->oz, sr::OZS_COLS, sr::OZS_COLS, n, n, s, 1.0, true,
                             sr::EpMinusITD{Y.x0, Y.x1, Y.x2, Y.ld}, h->partial, &blocks));
    return reduce_to(h, blocks, 1);
}

// Qn = Q + alpha Q X
sr_status td_apply(schur_refine_ctx *h, int n, TdMat Q, TdMat X, TdMat Qn, double alpha)
{
    const int s = sr::kCrtDefaultModuliTD;
    SR_TRY(td_split(h, sr::OZS_QROWS, n, Q, sr::OZ_ROWS));
    SR_TRY(td_split(h, sr::OZS_X, n, X, sr::OZ_COLS));
    SR_TRY(sr::ozaki_product(h, h->st, h->oz, sr::OZS_QROWS, sr::OZS_X, n, n, n, s, false, h->dflags));
    return sr::ozaki_combine(h, h->st, h->oz, sr::OZS_QROWS, sr::OZS_X, n, n, s, 1.0, false,
                             sr::EpUpdateTD{Q.x0, Q.x1, Q.x2, Q.ld, Qn.x0, Qn.x1, Qn.x2, Qn.ld, alpha}, nullptr,
                             nullptr);
}

// S1 + S2: A Q (A's row residues in OZS_ROWS), T^ = Q^T (A Q) into TE, the
// diagonal's two leading words and That; ||E||^2 (leading words) -> dnorm[slot]
sr_status td_form_residual(schur_refine_ctx *h, int n, TdMat Q, TdMat That, int slot)
{
    const int s = sr::kCrtDefaultModuliTD;
    const TdMat AQ = td_work(h, h->AQ);
    int blocks = 0;
    SR_TRY(td_split(h, sr::OZS_COLS, n, Q, sr::OZ_COLS));
    SR_TRY(sr::ozaki_product(h, h->st, h->oz, sr::OZS_ROWS, sr::OZS_COLS, n, n, n, s, false, h->dflags));
    SR_TRY(sr::ozaki_combine(h, h->st, h->oz, sr::OZS_ROWS, sr::OZS_COLS, n, n, s, 1.0, false,
                             sr::EpStoreTD{AQ.x0, AQ.x1, AQ.x2, AQ.ld}, nullptr, nullptr));
    SR_TRY(td_split(h, sr::OZS_X, n, AQ, sr::OZ_COLS));
    SR_TRY(sr::ozaki_product(h, h->st, h->oz, sr::OZS_COLS, sr::OZS_X, n, n, n, s, false, h->dflags));
    const sr::EpSplitTD ep{(double *)h->TE, h->nmax, h->diag, h->diag_lo, That.x0, That.x1, That.x2, That.ld};
    SR_TRY(sr::ozaki_combine(h, h->st, h->oz, sr::OZS_COLS, sr::OZS_X, n, n, s, 1.0, false, ep, h->partial, &blocks));
    return reduce_to(h, blocks, slot);
}

// S5-S8: Y, W = L - L^T (FP64), YW, W^2, W^3 (FP64-class, 7 digits, Y rounded to
// its leading word), Delta = Sigma - 2I summed exactly, Q_new = Q + 1/2 Q Delta
sr_status td_update(schur_refine_ctx *h, int n, TdMat Q, TdMat Qn)
{
    using namespace sr;
    const int ld = h->nmax;
    cudaStream_t st = h->st;
    SR_TRY(td_gram(h, n));   // Q's column residues are those of the residual's product
    const TdMat Y = td_work(h, h->Y), Dl = td_work(h, h->Delta);
    double *Wd = h->Wd, *W2 = (double *)h->W2, *YW = (double *)h->YW;
    double *W2Y = (double *)h->W2Y, *W2YW = (double *)h->W2YW;
    {
        SrPhase ph(h, SR_PROF_OTHER, 0, 16LL * n * n, 1);
        dim3 grid((n + 31) / 32, (n + 31) / 32);
        form_skew_kernel<double><<<grid, 256, 0, st>>>(n, (const double *)h->TE, ld, Wd, ld);
        SR_CUDA_TRY(cudaGetLastError());
    }
    const bool full = h->opt.full_sigma != 0;
    const EpDeltaTD ed{(const double *)h->TE, ld, YW, W2, full ? W2Y : nullptr, full ? W2YW : nullptr, ld,
                       Y.x0, Y.x1, Y.x2, Y.ld, Dl.x0, Dl.x1, Dl.x2, Dl.ld};
    const int sl = kOzakiDefaultSlices;
    OzakiWork &w = h->oz;
    SR_TRY(ozaki_split(h, st, w, OZS_W, n, n, Wd, ld, OZ_COLS, sl));
    SR_TRY(ozaki_split(h, st, w, OZS_Y, n, n, Y.x0, ld, OZ_COLS, sl));
    SR_TRY(ozaki_product(h, st, w, OZS_W, OZS_W, n, n, n, sl, true, h->dflags));
    SR_TRY(ozaki_combine(h, st, w, OZS_W, OZS_W, n, n, sl, -1.0, true, EpStore{W2, ld}, nullptr, nullptr));
    SR_TRY(ozaki_product(h, st, w, OZS_Y, OZS_W, n, n, n, sl, false, h->dflags));
    SR_TRY(ozaki_combine(h, st, w, OZS_Y, OZS_W, n, n, sl, 1.0, false, EpStore{YW, ld}, nullptr, nullptr));
    SR_TRY(ozaki_split(h, st, w, OZS_W2, n, n, W2, ld, OZ_COLS, sl));
    if (full) {
        SR_TRY(ozaki_product(h, st, w, OZS_W2, OZS_Y, n, n, n, sl, false, h->dflags));
        SR_TRY(ozaki_combine(h, st, w, OZS_W2, OZS_Y, n, n, sl, 1.0, false, EpStore{W2Y, ld}, nullptr, nullptr));
        SR_TRY(ozaki_split(h, st, w, 7, n, n, W2Y, ld, OZ_ROWS, sl));
        SR_TRY(ozaki_product(h, st, w, 7, OZS_W, n, n, n, sl, false, h->dflags));
        SR_TRY(ozaki_combine(h, st, w, 7, OZS_W, n, n, sl, 1.0, false, EpStore{W2YW, ld}, nullptr, nullptr));
    }
    SR_TRY(ozaki_product(h, st, w, OZS_W, OZS_W2, n, n, n, sl, false, h->dflags));
    SR_TRY(ozaki_combine(h, st, w, OZS_W, OZS_W2, n, n, sl, -1.0, false, ed, nullptr, nullptr));
    return td_apply(h, n, Q, Dl, Qn, 0.5);
}

sr_status copy_td(schur_refine_ctx *h, int n, TdMat src, TdMat dst)
{
    if (src.x0 == dst.x0) return SR_OK;
    SrPhase ph(h, SR_PROF_OTHER, 0, 48LL * n * n, 3);
    const double *s[3] = {src.x0, src.x1, src.x2};
    double *d[3] = {dst.x0, dst.x1, dst.x2};
    for (int k = 0; k < 3; ++k)
        SR_CUDA_TRY(cudaMemcpy2DAsync(d[k], (size_t)dst.ld * 8, s[k], (size_t)src.ld * 8, (size_t)n * 8, n,
                                      cudaMemcpyDeviceToDevice, h->st));
    return SR_OK;
}

// One call of Alg. 4 with the triple-double target (residue-form products).
sr_status run_step_td(schur_refine_ctx *h, int n, const void *dA, int lda, void *dQ, int ldq, const void *dQhat,
                      void *dT, sr_norms *out)
{
    const int ld = h->nmax;
    const double tol = h->opt.tol > 0 ? h->opt.tol : 1e-45 * (double)n;
    const int max_iter = h->opt.max_iter > 0 ? h->opt.max_iter : 10;
    sr_norms nr{};
    nr.stril_rel = nr.orth = nr.w_norm = NAN;
    const TdMat A = td_caller(dA, lda, n), Qcaller = td_caller(dQ, ldq, n);
    const TdMat That = dT ? td_caller(dT, n, n) : TdMat{nullptr, nullptr, nullptr, n};
    SR_CUDA_TRY(cudaMemsetAsync(h->dflags, 0, sizeof(int), h->st));
    SR_TRY(sumsq<double>(h, n, A.x0, lda, 0, 3));
    SR_TRY(td_split(h, sr::OZS_ROWS, n, A, sr::OZ_ROWS));
    TdMat Qc = Qcaller, Qo = td_work(h, h->Qw);
    double y_last = NAN;
    if (dQhat) {
        // Alg. 4: Qhat (FP64) as a triple-double, then Q <- Q - 1/2 Q (Q^T Q - I) (eq. NS)
        {
            SrPhase ph(h, SR_PROF_OTHER, 0, 32LL * n * n, 3);
            SR_CUDA_TRY(cudaMemcpy2DAsync(Qc.x0, (size_t)Qc.ld * 8, dQhat, (size_t)ldq * 8, (size_t)n * 8, n,
                                          cudaMemcpyDeviceToDevice, h->st));
            SR_CUDA_TRY(cudaMemset2DAsync(Qc.x1, (size_t)Qc.ld * 8, 0, (size_t)n * 8, n, h->st));
            SR_CUDA_TRY(cudaMemset2DAsync(Qc.x2, (size_t)Qc.ld * 8, 0, (size_t)n * 8, n, h->st));
        }
        SR_TRY(td_split(h, sr::OZS_COLS, n, Qc, sr::OZ_COLS));
        SR_TRY(td_gram(h, n));
        SR_TRY(td_apply(h, n, Qc, td_work(h, h->Y), Qo, -0.5));
        std::swap(Qc, Qo);
        nr.hp_gemms += 2;
        SR_TRY(read_back(h));
        y_last = sqrt(h->hbuf[1]);
        nr.orth = y_last;
    }
    const double anorm = sqrt(h->hbuf[3] > 0 ? h->hbuf[3] : 1.0);
    sr_status status = SR_ERR_NOT_CONVERGED;
    double prev = INFINITY;
    for (int k = 1; k <= max_iter; ++k) {
        SR_TRY(td_form_residual(h, n, Qc, That, 0));
        nr.hp_gemms += 2;
        nr.iters = k;
        SR_TRY(read_back(h));
        if (timed_out(h)) { status = SR_ERR_TIMEOUT; break; }
        const double rT = sqrt(h->hbuf[0]) / anorm;
        nr.stril_rel = rT;
        if (!isfinite(rT)) { status = SR_ERR_NONFINITE; break; }
        const bool ok_y = !(y_last > sqrt(tol));
        if (rT <= tol && ok_y) { status = SR_OK; break; }
        if (k >= 3 && rT > 10.0 * prev) { status = SR_ERR_NOT_CONVERGED; break; }
        prev = rT;
        SR_TRY(solve<double>(h, n, (double *)h->TE, ld, h->diag, h->diag_lo));
        SR_TRY(sumsq<double>(h, n, (const double *)h->TE, ld, 1, 2));
        SR_TRY(read_back(h));
        const int f = host_flags(h);
        if (f & SR_FLAG_TIMEOUT) { status = SR_ERR_TIMEOUT; break; }
        if (f & SR_FLAG_NONDISTINCT) { status = SR_ERR_NONDISTINCT; break; }
        if (f & SR_FLAG_NONFINITE) { status = SR_ERR_NONFINITE; break; }
        nr.w_norm = sqrt(2.0 * h->hbuf[2]);
        SR_TRY(td_update(h, n, Qc, Qo));
        nr.hp_gemms += 2;
        std::swap(Qc, Qo);
        SR_TRY(read_back(h));
        y_last = sqrt(h->hbuf[1]);
        nr.orth = y_last;
        status = SR_ERR_NOT_CONVERGED;
    }
    SR_TRY(copy_td(h, n, Qc, Qcaller));
    SR_CUDA_TRY(cudaStreamSynchronize(h->st));
    harvest(h);
    if (out) *out = nr;
    return status;
}

// ---- the six-double target (SR_TARGET_D6) ---------------------------------------------
// Sec. 3's 100-digit runs hold each high-precision number as 6 doubles (about
// 318 bits). The residue form carries at most 164 bits per operand with the
// 49 pairwise coprime moduli <= 256, so each operand is held as two halves of
// t = 162 bits (the fixed-point value of T = 2t - 2 bits, X = X_hi 2^t + X_lo),
// and each product is four residue products (HH, HL, LH, LL) of 48 moduli,
// rebuilt, combined exactly and rounded once to six words. The epilogues sum
// their terms exactly; the low precision is FP64 as in the other multi-word
// forms.
bool is_d6(const sr_options &o) { return o.target == SR_TARGET_D6; }

struct D6Mat {
    double *x;   // plane k at x + k pl
    size_t pl;
    int ld;
};
D6Mat d6_caller(const void *p, int ld, int n) { return {(double *)p, (size_t)ld * (size_t)n, ld}; }
D6Mat d6_work(const schur_refine_ctx *h, double *p) { return {p, (size_t)h->nmax * (size_t)h->nmax, h->nmax}; }
D6Mat d6_none(int n) { return {nullptr, 0, n}; }

sr_status d6_split(schur_refine_ctx *h, int slot_hi, int slot_lo, int n, D6Mat X, int layout)
{
    return sr::ozaki_split_d6(h, h->st, h->oz, slot_hi, slot_lo, n, n, X.x, X.pl, X.ld, layout);
}

// the four residue products of a six-double product into the plane sets 0..3
sr_status d6_products(schur_refine_ctx *h, int rows_hi, int rows_lo, int cols_hi, int cols_lo, int n)
{
    const int s = sr::kCrtDefaultModuliTD;
    uint8_t *base = reinterpret_cast<uint8_t *>(h->oz.planes);
    const size_t set = (size_t)s * h->oz.Pmax * h->oz.Pmax;
    const int rs[4] = {rows_hi, rows_hi, rows_lo, rows_lo}, cs[4] = {cols_hi, cols_lo, cols_hi, cols_lo};
    for (int k = 0; k < 4; ++k)
        SR_TRY(sr::ozaki_product(h, h->st, h->oz, rs[k], cs[k], n, n, n, s, false, h->dflags,
                                 reinterpret_cast<int32_t *>(base + (size_t)k * set)));
    return SR_OK;
}

// Y = Q^T Q - I and ||Y||^2 -> dnorm[1], from Q's column halves in OZS_COLS, OZS_COLS_LO
sr_status d6_gram(schur_refine_ctx *h, int n)
{
    const D6Mat Y = d6_work(h, h->Y);
    int blocks = 0;
    SR_TRY(d6_products(h, sr::OZS_COLS, sr::OZS_COLS_LO, sr::OZS_COLS, sr::OZS_COLS_LO, n));
    SR_TRY(sr::ozaki_combine_d6(h, h->st, h->oz, sr::OZS_COLS, sr::OZS_COLS, n, n, 1.0,
                                sr::EpMinusID6{Y.x, Y.ld, Y.pl}, h->partial, &blocks));
    return reduce_to(h, blocks, 1);
}

// Qn = Q + alpha Q X
sr_status d6_apply(schur_refine_ctx *h, int n, D6Mat Q, D6Mat X, D6Mat Qn, double alpha)
{
    SR_TRY(d6_split(h, sr::OZS_QROWS, sr::OZS_QROWS_LO, n, Q, sr::OZ_ROWS));
    SR_TRY(d6_split(h, sr::OZS_X, sr::OZS_X_LO, n, X, sr::OZ_COLS));
    SR_TRY(d6_products(h, sr::OZS_QROWS, sr::OZS_QROWS_LO, sr::OZS_X, sr::OZS_X_LO, n));
    return sr::ozaki_combine_d6(h, h->st, h->oz, sr::OZS_QROWS, sr::OZS_X, n, n, 1.0,
                                sr::EpUpdateD6{Q.x, Q.ld, Q.pl, Qn.x, Qn.ld, Qn.pl, alpha}, nullptr, nullptr);
}

// S1 + S2: A Q (A's row halves in OZS_ROWS, OZS_ROWS_LO), T^ = Q^T (A Q); ||E||^2 -> dnorm[slot]
sr_status d6_form_residual(schur_refine_ctx *h, int n, D6Mat Q, D6Mat That, int slot)
{
    const D6Mat AQ = d6_work(h, h->AQ);
    int blocks = 0;
    SR_TRY(d6_split(h, sr::OZS_COLS, sr::OZS_COLS_LO, n, Q, sr::OZ_COLS));
    SR_TRY(d6_products(h, sr::OZS_ROWS, sr::OZS_ROWS_LO, sr::OZS_COLS, sr::OZS_COLS_LO, n));
    SR_TRY(sr::ozaki_combine_d6(h, h->st, h->oz, sr::OZS_ROWS, sr::OZS_COLS, n, n, 1.0,
                                sr::EpStoreD6{AQ.x, AQ.ld, AQ.pl}, nullptr, nullptr));
    SR_TRY(d6_split(h, sr::OZS_X, sr::OZS_X_LO, n, AQ, sr::OZ_COLS));
    SR_TRY(d6_products(h, sr::OZS_COLS, sr::OZS_COLS_LO, sr::OZS_X, sr::OZS_X_LO, n));
    const sr::EpSplitD6 ep{(double *)h->TE, h->nmax, h->diag, h->diag_lo, That.x, That.ld, That.pl};
    SR_TRY(sr::ozaki_combine_d6(h, h->st, h->oz, sr::OZS_COLS, sr::OZS_X, n, n, 1.0, ep, h->partial, &blocks));
    return reduce_to(h, blocks, slot);
}

// S5-S8 (as td_update with six words)
sr_status d6_update(schur_refine_ctx *h, int n, D6Mat Q, D6Mat Qn)
{
    using namespace sr;
    const int ld = h->nmax;
    cudaStream_t st = h->st;
    SR_TRY(d6_gram(h, n));   // Q's column halves are those of the residual's product
    const D6Mat Y = d6_work(h, h->Y), Dl = d6_work(h, h->Delta);
    double *Wd = h->Wd, *W2 = (double *)h->W2, *YW = (double *)h->YW;
    double *W2Y = (double *)h->W2Y, *W2YW = (double *)h->W2YW;
    {
        SrPhase ph(h, SR_PROF_OTHER, 0, 16LL * n * n, 1);
        dim3 grid((n + 31) / 32, (n + 31) / 32);
        form_skew_kernel<double><<<grid, 256, 0, st>>>(n, (const double *)h->TE, ld, Wd, ld);
        SR_CUDA_TRY(cudaGetLastError());
    }
    const bool full = h->opt.full_sigma != 0;
    const EpDeltaD6 ed{(const double *)h->TE, ld, YW, W2, full ? W2Y : nullptr, full ? W2YW : nullptr, ld,
                       Y.x, Y.ld, Y.pl, Dl.x, Dl.ld, Dl.pl};
    const int sl = kOzakiDefaultSlices;
    OzakiWork &w = h->oz;
    SR_TRY(ozaki_split(h, st, w, OZS_W, n, n, Wd, ld, OZ_COLS, sl));
    SR_TRY(ozaki_split(h, st, w, OZS_Y, n, n, Y.x, ld, OZ_COLS, sl));
    SR_TRY(ozaki_product(h, st, w, OZS_W, OZS_W, n, n, n, sl, true, h->dflags));
    SR_TRY(ozaki_combine(h, st, w, OZS_W, OZS_W, n, n, sl, -1.0, true, EpStore{W2, ld}, nullptr, nullptr));
    SR_TRY(ozaki_product(h, st, w, OZS_Y, OZS_W, n, n, n, sl, false, h->dflags));
    SR_TRY(ozaki_combine(h, st, w, OZS_Y, OZS_W, n, n, sl, 1.0, false, EpStore{YW, ld}, nullptr, nullptr));
    SR_TRY(ozaki_split(h, st, w, OZS_W2, n, n, W2, ld, OZ_COLS, sl));
    if (full) {
        SR_TRY(ozaki_product(h, st, w, OZS_W2, OZS_Y, n, n, n, sl, false, h->dflags));
        SR_TRY(ozaki_combine(h, st, w, OZS_W2, OZS_Y, n, n, sl, 1.0, false, EpStore{W2Y, ld}, nullptr, nullptr));
        SR_TRY(ozaki_split(h, st, w, 7, n, n, W2Y, ld, OZ_ROWS, sl));
        SR_TRY(ozaki_product(h, st, w, 7, OZS_W, n, n, n, sl, false, h->dflags));
        SR_TRY(ozaki_combine(h, st, w, 7, OZS_W, n, n, sl, 1.0, false, EpStore{W2YW, ld}, nullptr, nullptr));
    }
    SR_TRY(ozaki_product(h, st, w, OZS_W, OZS_W2, n, n, n, sl, false, h->dflags));
    SR_TRY(ozaki_combine(h, st, w, OZS_W, OZS_W2, n, n, sl, -1.0, false, ed, nullptr, nullptr));
    return d6_apply(h, n, Q, Dl, Qn, 0.5);
}

sr_status copy_d6(schur_refine_ctx *h, int n, D6Mat src, D6Mat dst)
{
    if (src.x == dst.x) return SR_OK;
    SrPhase ph(h, SR_PROF_OTHER, 0, 96LL * n * n, sr::kD6Words);
    for (int k = 0; k < sr::kD6Words; ++k)
        SR_CUDA_TRY(cudaMemcpy2DAsync(dst.x + k * dst.pl, (size_t)dst.ld * 8, src.x + k * src.pl, (size_t)src.ld * 8,
                                      (size_t)n * 8, n, cudaMemcpyDeviceToDevice, h->st));
    return SR_OK;
}

// One call of Alg. 4 with the six-double target.
sr_status run_step_d6(schur_refine_ctx *h, int n, const void *dA, int lda, void *dQ, int ldq, const void *dQhat,
                      void *dT, sr_norms *out)
{
    const int ld = h->nmax;
    const double tol = h->opt.tol > 0 ? h->opt.tol : 1e-93 * (double)n;
    const int max_iter = h->opt.max_iter > 0 ? h->opt.max_iter : 10;
    sr_norms nr{};
    nr.stril_rel = nr.orth = nr.w_norm = NAN;
    const D6Mat A = d6_caller(dA, lda, n), Qcaller = d6_caller(dQ, ldq, n);
    const D6Mat That = dT ? d6_caller(dT, n, n) : d6_none(n);
    SR_CUDA_TRY(cudaMemsetAsync(h->dflags, 0, sizeof(int), h->st));
    SR_TRY(sumsq<double>(h, n, A.x, lda, 0, 3));
    SR_TRY(d6_split(h, sr::OZS_ROWS, sr::OZS_ROWS_LO, n, A, sr::OZ_ROWS));
    D6Mat Qc = Qcaller, Qo = d6_work(h, h->Qw);
    double y_last = NAN;
    if (dQhat) {
        // Alg. 4: Qhat (FP64) as a six-double, then Q <- Q - 1/2 Q (Q^T Q - I) (eq. NS)
        {
            SrPhase ph(h, SR_PROF_OTHER, 0, 56LL * n * n, sr::kD6Words);
            SR_CUDA_TRY(cudaMemcpy2DAsync(Qc.x, (size_t)Qc.ld * 8, dQhat, (size_t)ldq * 8, (size_t)n * 8, n,
                                          cudaMemcpyDeviceToDevice, h->st));
            for (int k = 1; k < sr::kD6Words; ++k)
                SR_CUDA_TRY(cudaMemset2DAsync(Qc.x + k * Qc.pl, (size_t)Qc.ld * 8, 0, (size_t)n * 8, n, h->st));
        }
        SR_TRY(d6_split(h, sr::OZS_COLS, sr::OZS_COLS_LO, n, Qc, sr::OZ_COLS));
        SR_TRY(d6_gram(h, n));
        SR_TRY(d6_apply(h, n, Qc, d6_work(h, h->Y), Qo, -0.5));
        std::swap(Qc, Qo);
        nr.hp_gemms += 2;
        SR_TRY(read_back(h));
        y_last = sqrt(h->hbuf[1]);
        nr.orth = y_last;
    }
    const double anorm = sqrt(h->hbuf[3] > 0 ? h->hbuf[3] : 1.0);
    sr_status status = SR_ERR_NOT_CONVERGED;
    double prev = INFINITY;
    for (int k = 1; k <= max_iter; ++k) {
        SR_TRY(d6_form_residual(h, n, Qc, That, 0));
        nr.hp_gemms += 2;
        nr.iters = k;
        SR_TRY(read_back(h));
        if (timed_out(h)) { status = SR_ERR_TIMEOUT; break; }
        const double rT = sqrt(h->hbuf[0]) / anorm;
        nr.stril_rel = rT;
        if (!isfinite(rT)) { status = SR_ERR_NONFINITE; break; }
        const bool ok_y = !(y_last > sqrt(tol));
        if (rT <= tol && ok_y) { status = SR_OK; break; }
        if (k >= 3 && rT > 10.0 * prev) { status = SR_ERR_NOT_CONVERGED; break; }
        prev = rT;
        SR_TRY(solve<double>(h, n, (double *)h->TE, ld, h->diag, h->diag_lo));
        SR_TRY(sumsq<double>(h, n, (const double *)h->TE, ld, 1, 2));
        SR_TRY(read_back(h));
        const int f = host_flags(h);
        if (f & SR_FLAG_TIMEOUT) { status = SR_ERR_TIMEOUT; break; }
        if (f & SR_FLAG_NONDISTINCT) { status = SR_ERR_NONDISTINCT; break; }
        if (f & SR_FLAG_NONFINITE) { status = SR_ERR_NONFINITE; break; }
        nr.w_norm = sqrt(2.0 * h->hbuf[2]);
        SR_TRY(d6_update(h, n, Qc, Qo));
        nr.hp_gemms += 2;
        std::swap(Qc, Qo);
        SR_TRY(read_back(h));
        y_last = sqrt(h->hbuf[1]);
        nr.orth = y_last;
        status = SR_ERR_NOT_CONVERGED;
    }
    SR_TRY(copy_d6(h, n, Qc, Qcaller));
    SR_CUDA_TRY(cudaStreamSynchronize(h->st));
    harvest(h);
    if (out) *out = nr;
    return status;
}

}  // namespace

// ============================================================================
extern "C" {

void schur_refine_default_options(sr_options *opt)
{
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->dtype = SR_REAL;
    opt->target = SR_TARGET_FP64;
    opt->hp_gemm = SR_HP_FP64;
    opt->lp = SR_LP_FP32;
    opt->qhat_type = SR_QHAT_FP32;
    opt->full_sigma = 0;
    opt->max_iter = 10;
    opt->ozaki_slices = 0;
    opt->tol = 0.0;
    opt->profile = 0;
    opt->batch_streams = 0;
    opt->batch_mode = 0;
    opt->tune = 0;
    opt->graph = 0;
    opt->solve_mode = 0;
    opt->symmetric = 0;
    opt->l_cap = 0.0;
    opt->lp_slices = 0;
    opt->quasi = 0;
}

const char *schur_refine_status_string(sr_status s)
{
    switch (s) {
    case SR_OK: return "ok";
    case SR_ERR_INVALID_ARG: return "invalid argument";
    case SR_ERR_NONDISTINCT: return "diagonal entries of T not pairwise distinct";
    case SR_ERR_NONFINITE: return "non-finite value";
    case SR_ERR_NOT_CONVERGED: return "not converged";
    case SR_ERR_TIMEOUT: return "device wait timed out";
    case SR_ERR_CUDA: return "CUDA error";
    case SR_ERR_OOM: return "out of device memory";
    case SR_ERR_UNSUPPORTED: return "unsupported option combination";
    }
    return "unknown status";
}

sr_status schur_refine_get_profile(schur_refine_t h, sr_profile *out)
{
    if (!h || !out) return SR_ERR_INVALID_ARG;
    SR_CUDA_TRY(cudaStreamSynchronize(h->st));
    harvest(h);
    *out = h->prof;
    return SR_OK;
}

sr_status schur_refine_reset_profile(schur_refine_t h)
{
    if (!h) return SR_ERR_INVALID_ARG;
    SR_CUDA_TRY(cudaStreamSynchronize(h->st));
    harvest(h);
    memset(&h->prof, 0, sizeof(h->prof));
    return SR_OK;
}

void schur_refine_destroy(schur_refine_t h)
{
    if (!h) return;
    if (h->st) cudaStreamSynchronize(h->st);
    harvest(h);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    cudaFree(h->AQ);
    cudaFree(h->Qw);
    cudaFree(h->Y);
    cudaFree(h->Delta);
    cudaFree(h->diag);
    cudaFree(h->TE);
    cudaFree(h->W2);
    cudaFree(h->YW);
    cudaFree(h->W2Y);
    cudaFree(h->W2YW);
    cudaFree(h->Wd);
    cudaFree(h->W2d);
    cudaFree(h->W2Yd);
    cudaFree(h->W2YWd);
    for (auto *sub : h->subs) schur_refine_destroy(sub);
    sr_batch_free(h->bw);
    for (auto s : h->sub_streams) cudaStreamDestroy(s);
    for (auto e : h->bjoin) cudaEventDestroy(e);
    if (h->bfork) cudaEventDestroy(h->bfork);
    drop_graphs(h);
    if (h->rgraph.exec) cudaGraphExecDestroy(h->rgraph.exec);
    if (h->rgraph.graph) cudaGraphDestroy(h->rgraph.graph);
    for (auto s : h->cstreams) cudaStreamDestroy(s);
    cudaFree(h->ctl);
    if (h->cap_st) cudaStreamDestroy(h->cap_st);
    if (h->aux_st) cudaStreamDestroy(h->aux_st);
    if (h->sev0) cudaEventDestroy(h->sev0);
    if (h->sev1) cudaEventDestroy(h->sev1);
    cudaFree(h->plan);
    cudaFree(h->partial);
    cudaFree(h->partial2);
    if (h->gram_st) cudaStreamDestroy(h->gram_st);
    if (h->gev0) cudaEventDestroy(h->gev0);
    if (h->gev1) cudaEventDestroy(h->gev1);
    cudaFree(h->dnorm);
    cudaFree(h->dflags);
    cudaFree(h->flow);
    cudaFree(h->flow_acc);
    cudaFree(h->flow_plan);
    if (h->hbuf) cudaFreeHost(h->hbuf);
    cudaFree(h->band);
    cudaFree(h->qblk);
    cudaFree(h->TEq);
    cudaFree(h->dhpq);
    cudaFree(h->qpos);
    cudaFree(h->qinv);
    cudaFree(h->qblkq);
    cudaFree(h->qcpl);
    cudaFree(h->step_acc);
    if (h->hblk) cudaFreeHost(h->hblk);
    if (h->hmaps) cudaFreeHost(h->hmaps);
    sr::ozaki_free(h->oz);
    delete h;
}

sr_status schur_refine_create(schur_refine_t *hp, int n_max, const sr_options *opt, void *cuda_stream)
{
    if (!hp) return SR_ERR_INVALID_ARG;
    *hp = nullptr;
    if (n_max < 1 || n_max > 32768) return SR_ERR_INVALID_ARG;
    sr_options o;
    schur_refine_default_options(&o);
    if (opt) o = *opt;
    SR_TRY(check_opts(o));
    schur_refine_ctx *h = new schur_refine_ctx();
    h->nmax = n_max;
    h->opt = o;
    h->st = (cudaStream_t)cuda_stream;
    cudaGetDevice(&h->dev);
    const size_t nn = (size_t)n_max * (size_t)n_max;
    const size_t lps = lp_size(o), hps = hp_size(o);
    const size_t tiles16 = ((size_t)(n_max + 15) / 16) * ((size_t)(n_max + 15) / 16);
    h->npartial = std::max<size_t>(tiles16, 4096);
    cudaError_t e = cudaSuccess;
#define SR_ALLOC(ptr, bytes)                                             \
    if (e == cudaSuccess) e = cudaMalloc((void **)&(ptr), (bytes));
    SR_ALLOC(h->AQ, nn * hps);
    SR_ALLOC(h->Qw, nn * hps);
    SR_ALLOC(h->Y, nn * hps);
    SR_ALLOC(h->Delta, nn * hps);
    SR_ALLOC(h->diag, (size_t)n_max * hps);
    SR_ALLOC(h->TE, nn * lps);
    // low-precision products of the native path
    const bool native_lp = !(is_emulated(o) && o.lp == SR_LP_FP32);
    if (native_lp) {
        SR_ALLOC(h->W2, nn * lps);
        SR_ALLOC(h->YW, nn * lps);
    }
    if (o.full_sigma && native_lp) {
        SR_ALLOC(h->W2Y, nn * lps);
        SR_ALLOC(h->W2YW, nn * lps);
    }
    SR_ALLOC(h->partial, h->npartial * sizeof(double));
    SR_ALLOC(h->dnorm, 8 * sizeof(double));
    SR_ALLOC(h->dflags, sizeof(int));
    // the real Schur form solves in a padded order: at most one padding row per tile of 32 rows
    if (o.quasi) h->nqmax = n_max + (n_max + sr::kSolveTile - 2) / (sr::kSolveTile - 1) + 1;
    const size_t nsolve = (size_t)(o.quasi ? h->nqmax : n_max);
    const size_t nbmax = (nsolve + sr::kSolveTile - 1) / sr::kSolveTile;
    SR_ALLOC(h->flow, (2 + 2 * nbmax * nbmax) * sizeof(int));
    // the dataflow solve's helper accumulators (leading dimension nsolve), where that form can serve
    if ((o.dtype == SR_REAL && o.lp == SR_LP_FP32 && o.solve_mode == 0) || o.solve_mode == 1)
        SR_ALLOC(h->flow_acc, nsolve * nsolve * lps);
    // the stepwise solve's sums of far products, kept apart from E (leading dimension n_max)
    if (!o.quasi) SR_ALLOC(h->step_acc, nn * lps);
    if (o.quasi) {
        const size_t nq = (size_t)h->nqmax;
        SR_ALLOC(h->band, 3 * (size_t)n_max * sizeof(double));
        SR_ALLOC(h->qblk, (size_t)n_max * sizeof(int));
        SR_ALLOC(h->TEq, nq * nq * lps);
        SR_ALLOC(h->dhpq, nq * sizeof(double));
        SR_ALLOC(h->qpos, (size_t)n_max * sizeof(int));
        SR_ALLOC(h->qinv, nq * sizeof(int));
        SR_ALLOC(h->qblkq, nq * sizeof(int));
        SR_ALLOC(h->qcpl, nq * lps);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&h->hblk, (size_t)n_max * sizeof(int));
        if (e == cudaSuccess) e = cudaMallocHost((void **)&h->hmaps, ((size_t)n_max + 2 * nq) * sizeof(int));
    }
#undef SR_ALLOC
    if (e == cudaSuccess) {
        // grid of the dataflow solve for each low-precision kind this handle can use
        h->flow_ctas[0] = sr::trisolve_flow_setup<float>(h->dev);
        h->flow_ctas[1] = sr::trisolve_flow_setup<double>(h->dev);
        h->flow_ctas[2] = sr::trisolve_flow_setup<cf>(h->dev);
        if (!h->flow_ctas[0] || !h->flow_ctas[1] || !h->flow_ctas[2]) e = cudaGetLastError();
        if (e == cudaSuccess && (!h->flow_ctas[0] || !h->flow_ctas[1] || !h->flow_ctas[2])) e = cudaErrorInvalidValue;
    }
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->hbuf, 16 * sizeof(double));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->aux_st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->sev0, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->sev1, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemset(h->dnorm, 0, 8 * sizeof(double));
    const bool d6 = o.target == SR_TARGET_D6;
    const bool td = o.target == SR_TARGET_TD || d6;   // 12-limb rebuilds
    const bool dd = o.target == SR_TARGET_DD || td;   // FP64 low precision with a multi-word diagonal
    if (e == cudaSuccess) h->diag_lo = dd ? h->diag + n_max : nullptr;
    if (e == cudaSuccess && dd) e = cudaMalloc((void **)&h->Wd, nn * sizeof(double));
    if (e == cudaSuccess && is_emulated(o)) {
        // the double-double product keeps 14 levels below 2^31: K up to 8192
        if (n_max > (dd ? 8192 : sr::ozaki_k_limit(is_cplx(o)))) {
            schur_refine_destroy(h);
            return SR_ERR_UNSUPPORTED;
        }
        const int shp = oz_count(o);
        const bool lp_oz = o.lp == SR_LP_FP32;
        int caps[sr::kOzakiSlots] = {shp, shp, shp, shp, 0, 0, 0, 0};
        if (dd) {
            // FP64-class digits of W, Y, W^2 (and W^2 Y) for the FP64 products YW, W^2, W^3
            caps[sr::OZS_W] = caps[sr::OZS_Y] = caps[sr::OZS_W2] = sr::kOzakiDefaultSlices;
            if (o.full_sigma) caps[7] = sr::kOzakiDefaultSlices;
        }
        if (lp_oz) {
            caps[sr::OZS_W] = caps[sr::OZS_Y] = caps[sr::OZS_W2] = sr::kOzakiLpSlices;
            if (o.full_sigma) caps[7] = sr::kOzakiLpSlices;
            e = cudaMalloc((void **)&h->Wd, nn * hps);
            if (e == cudaSuccess) e = cudaMalloc((void **)&h->W2d, nn * hps);
            if (e == cudaSuccess && o.full_sigma) e = cudaMalloc((void **)&h->W2Yd, nn * hps);
            if (e == cudaSuccess && o.full_sigma) e = cudaMalloc((void **)&h->W2YWd, nn * hps);
        }
        // residue form: the four slots of the high-precision products (rows of A,
        // columns of Q, columns of A Q and of Delta, rows of Q) hold residues
        const bool crt = o.hp_gemm == SR_HP_OZAKI_CRT;
        unsigned crt_mask = crt ? ((1u << sr::OZS_ROWS) | (1u << sr::OZS_COLS) | (1u << sr::OZS_X) |
                                   (1u << sr::OZS_QROWS))
                                : 0u;
        if (d6) {
            // the low halves of the six-double operands
            crt_mask |= (1u << sr::OZS_ROWS_LO) | (1u << sr::OZS_COLS_LO) | (1u << sr::OZS_X_LO) |
                        (1u << sr::OZS_QROWS_LO);
            caps[sr::OZS_ROWS_LO] = caps[sr::OZS_COLS_LO] = caps[sr::OZS_X_LO] = caps[sr::OZS_QROWS_LO] = shp;
        }
        if (e == cudaSuccess)
            e = sr::ozaki_alloc(h->oz, n_max, caps, is_cplx(o), crt ? shp : 0, crt_mask, td ? 12 : dd ? 8 : 4,
                                d6 ? 4 : 1);
        if (e == cudaSuccess) e = cudaMalloc((void **)&h->partial2, h->npartial * sizeof(double));
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->gram_st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->gev0, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->gev1, cudaEventDisableTiming);
        h->oz.autotune = o.tune == 1;
    }
    if (e != cudaSuccess) {
        sr_set_last_cuda_error(e);
        schur_refine_destroy(h);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? SR_ERR_OOM : SR_ERR_CUDA;
    }
    memset(h->hbuf, 0, 16 * sizeof(double));
    *hp = h;
    return SR_OK;
}

sr_status schur_refine_step(schur_refine_t h, int n, const void *dA, int lda, void *dQ, int ldq, const void *dQhat,
                            void *dT, sr_norms *out)
{
    if (!h || !dA || !dQ || n < 1 || n > h->nmax || lda < n || ldq < n) return SR_ERR_INVALID_ARG;
    if (is_td(h->opt)) return run_step_td(h, n, dA, lda, dQ, ldq, dQhat, dT, out);
    if (is_d6(h->opt)) return run_step_d6(h, n, dA, lda, dQ, ldq, dQhat, dT, out);
    if (is_dd(h->opt)) {
        if (is_emulated(h->opt)) return run_step_dd<true>(h, n, dA, lda, dQ, ldq, dQhat, dT, out);
        return run_step_dd<false>(h, n, dA, lda, dQ, ldq, dQhat, dT, out);
    }
    if (is_cplx(h->opt)) return run_step<float, true>(h, n, dA, lda, dQ, ldq, dQhat, dT, out);
    if (h->opt.graph) {
        if (h->opt.lp == SR_LP_FP32) return run_step_graph<float>(h, n, dA, lda, dQ, ldq, dQhat, dT, out);
        return run_step_graph<double>(h, n, dA, lda, dQ, ldq, dQhat, dT, out);
    }
    if (h->opt.lp == SR_LP_FP32) return run_step<float, false>(h, n, dA, lda, dQ, ldq, dQhat, dT, out);
    return run_step<double, false>(h, n, dA, lda, dQ, ldq, dQhat, dT, out);
}

sr_status schur_refine_batched(schur_refine_t h, int batch, const int *n, const void *const *dA, void *const *dQ,
                               const void *const *dQhat, int *iters_out, int *status_out)
{
    if (!h || batch < 0 || (batch > 0 && (!n || !dA || !dQ))) return SR_ERR_INVALID_ARG;
    for (int b = 0; b < batch; ++b)
        if (n[b] < 1 || n[b] > h->nmax || !dA[b] || !dQ[b]) return SR_ERR_INVALID_ARG;
    if (batch == 0) return SR_OK;
    if (h->opt.batch_mode == 0 && dQhat && sr_batch_supported(h->opt)) {
        bool all_qhat = true;
        for (int b = 0; b < batch; ++b) all_qhat = all_qhat && dQhat[b] != nullptr;
        if (all_qhat) return sr_batch_refine(h, batch, n, dA, dQ, dQhat, iters_out, status_out);
    }
    const int want = h->opt.batch_streams > 0 ? h->opt.batch_streams : 8;
    const int W = std::min(want, batch);
    std::vector<int> st(batch, (int)SR_OK), it(batch, 0);
    if (W <= 1) {
        for (int b = 0; b < batch; ++b) {
            sr_norms nr{};
            st[b] = (int)schur_refine_step(h, n[b], dA[b], n[b], dQ[b], n[b], dQhat ? dQhat[b] : nullptr, nullptr,
                                           &nr);
            it[b] = nr.iters;
            if (st[b] == SR_ERR_CUDA) break;
        }
    } else {
        // worker pool: sub-handles with the same options, each on its own stream
        while ((int)h->subs.size() < W) {
            cudaStream_t s = nullptr;
            SR_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
            sr_options o = h->opt;
            o.batch_streams = 1;
            schur_refine_t sub = nullptr;
            sr_status cs = schur_refine_create(&sub, h->nmax, &o, s);
            if (cs != SR_OK) {
                cudaStreamDestroy(s);
                return cs;
            }
            cudaEvent_t ev = nullptr;
            SR_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            h->subs.push_back(sub);
            h->sub_streams.push_back(s);
            h->bjoin.push_back(ev);
        }
        if (!h->bfork) SR_CUDA_TRY(cudaEventCreateWithFlags(&h->bfork, cudaEventDisableTiming));
        // the workers start after the work already on the handle's stream
        SR_CUDA_TRY(cudaEventRecord(h->bfork, h->st));
        for (int w = 0; w < W; ++w) SR_CUDA_TRY(cudaStreamWaitEvent(h->sub_streams[w], h->bfork, 0));
        std::atomic<int> next(0);
        std::vector<std::thread> pool;
        int dev = 0;
        cudaGetDevice(&dev);
        for (int w = 0; w < W; ++w)
            pool.emplace_back([&, w]() {
                cudaSetDevice(dev);
                for (int b = next++; b < batch; b = next++) {
                    sr_norms nr{};
                    st[b] = (int)schur_refine_step(h->subs[w], n[b], dA[b], n[b], dQ[b], n[b],
                                                   dQhat ? dQhat[b] : nullptr, nullptr, &nr);
                    it[b] = nr.iters;
                }
            });
        for (auto &t : pool) t.join();
        for (int w = 0; w < W; ++w) {
            SR_CUDA_TRY(cudaEventRecord(h->bjoin[w], h->sub_streams[w]));
            SR_CUDA_TRY(cudaStreamWaitEvent(h->st, h->bjoin[w], 0));
            // the workers' launches and timings count as the handle's
            sr_profile p{};
            if (schur_refine_get_profile(h->subs[w], &p) == SR_OK) {
                for (int k = 0; k < SR_PROF_KINDS; ++k) {
                    h->prof.ms[k] += p.ms[k];
                    h->prof.flops[k] += p.flops[k];
                    h->prof.bytes[k] += p.bytes[k];
                    h->prof.launches[k] += p.launches[k];
                    h->prof.spans[k] += p.spans[k];
                }
                schur_refine_reset_profile(h->subs[w]);
            }
        }
    }
    sr_status first = SR_OK;
    for (int b = 0; b < batch; ++b) {
        if (iters_out) iters_out[b] = it[b];
        if (status_out) status_out[b] = st[b];
        if (st[b] != SR_OK && first == SR_OK) first = (sr_status)st[b];
    }
    return first;
}

sr_status schur_refine_residuals(schur_refine_t h, int n, const void *dA, int lda, const void *dQ, int ldq,
                                 double *stril_rel, double *orth)
{
    if (!h || !dA || !dQ || !stril_rel || !orth || n < 1 || n > h->nmax || lda < n || ldq < n)
        return SR_ERR_INVALID_ARG;
    const int ld = h->nmax;
    const size_t tiles = (size_t)((n + 15) / 16) * (size_t)((n + 15) / 16);
    if (tiles > h->npartial) return SR_ERR_INVALID_ARG;
    dim3 grid((n + 15) / 16, (n + 15) / 16);
    if (is_d6(h->opt)) {
        // the six-double products of the iteration, each rounded once
        const D6Mat A = d6_caller(dA, lda, n), Q = d6_caller(dQ, ldq, n);
        SR_CUDA_TRY(cudaMemsetAsync(h->dflags, 0, sizeof(int), h->st));
        SR_TRY(d6_split(h, sr::OZS_ROWS, sr::OZS_ROWS_LO, n, A, sr::OZ_ROWS));
        SR_TRY(d6_form_residual(h, n, Q, d6_none(n), 4));
        SR_TRY(d6_gram(h, n));
        SR_CUDA_TRY(cudaMemcpyAsync(h->dnorm + 5, h->dnorm + 1, sizeof(double), cudaMemcpyDeviceToDevice, h->st));
        SR_TRY(sumsq<double>(h, n, A.x, lda, 0, 6));
    } else if (is_td(h->opt)) {
        // the triple-double products of the iteration (residue form, 48 moduli),
        // each rounded once: T^'s entries below the diagonal carry errors near
        // 2^-159 ||A||, far below the target
        const TdMat A = td_caller(dA, lda, n), Q = td_caller(dQ, ldq, n);
        SR_CUDA_TRY(cudaMemsetAsync(h->dflags, 0, sizeof(int), h->st));
        SR_TRY(td_split(h, sr::OZS_ROWS, n, A, sr::OZ_ROWS));
        SR_TRY(td_form_residual(h, n, Q, TdMat{nullptr, nullptr, nullptr, n}, 4));
        SR_TRY(td_gram(h, n));
        SR_CUDA_TRY(cudaMemcpyAsync(h->dnorm + 5, h->dnorm + 1, sizeof(double), cudaMemcpyDeviceToDevice, h->st));
        SR_TRY(sumsq<double>(h, n, A.x0, lda, 0, 6));
    } else if (is_dd(h->opt)) {
        const DdMat A = dd_caller(dA, lda, n), Q = dd_caller(dQ, ldq, n), M = dd_work(h, h->AQ);
        sr::gemm_ddq_kernel<0><<<grid, 256, 0, h->st>>>(n, 0, A.hi, A.lo, lda, Q.hi, Q.lo, ldq, M.hi, M.lo, ld,
                                                        nullptr);
        SR_CUDA_TRY(cudaGetLastError());
        sr::gemm_ddq_kernel<1><<<grid, 256, 0, h->st>>>(n, 1, Q.hi, Q.lo, ldq, M.hi, M.lo, ld, nullptr, nullptr, 0,
                                                        h->partial);
        SR_CUDA_TRY(cudaGetLastError());
        SR_TRY(reduce_to(h, (int)tiles, 4));
        sr::gemm_ddq_kernel<2><<<grid, 256, 0, h->st>>>(n, 1, Q.hi, Q.lo, ldq, Q.hi, Q.lo, ldq, nullptr, nullptr, 0,
                                                        h->partial);
        SR_CUDA_TRY(cudaGetLastError());
        SR_TRY(reduce_to(h, (int)tiles, 5));
        SR_TRY(sumsq<double>(h, n, A.hi, lda, 0, 6));
    } else if (is_cplx(h->opt)) {
        const cd *A = (const cd *)dA, *Q = (const cd *)dQ;
        cd *Mhi = (cd *)h->AQ, *Mlo = (cd *)h->Delta;
        sr::gemm_dd_c_kernel<0><<<grid, 256, 0, h->st>>>(n, 0, A, lda, Q, nullptr, ldq, Mhi, Mlo, ld, nullptr);
        SR_CUDA_TRY(cudaGetLastError());
        sr::gemm_dd_c_kernel<1><<<grid, 256, 0, h->st>>>(n, 1, Q, ldq, Mhi, Mlo, ld, nullptr, nullptr, 0,
                                                         h->partial);
        SR_CUDA_TRY(cudaGetLastError());
        SR_TRY(reduce_to(h, (int)tiles, 4));
        sr::gemm_dd_c_kernel<2><<<grid, 256, 0, h->st>>>(n, 1, Q, ldq, Q, nullptr, ldq, nullptr, nullptr, 0,
                                                         h->partial);
        SR_CUDA_TRY(cudaGetLastError());
        SR_TRY(reduce_to(h, (int)tiles, 5));
        SR_TRY(sumsq<cd>(h, n, A, lda, 0, 6));
    } else {
        const double *A = (const double *)dA, *Q = (const double *)dQ;
        // M = A Q in double-double: hi in AQ, lo in Delta
        sr::gemm_dd_kernel<0><<<grid, 256, 0, h->st>>>(n, 0, A, lda, Q, nullptr, ldq, h->AQ, h->Delta, ld,
                                                       nullptr);
        SR_CUDA_TRY(cudaGetLastError());
        if (h->opt.quasi) {
            // the quasi-triangular form: the entries below the diagonal blocks, the
            // blocks read off the band of this Q^T A Q
            sr::gemm_dd_kernel<3><<<grid, 256, 0, h->st>>>(n, 1, Q, ldq, h->AQ, h->Delta, ld, nullptr, nullptr, 0,
                                                           h->partial, h->band);
            SR_CUDA_TRY(cudaGetLastError());
            SR_TRY(reduce_to(h, (int)tiles, 4));
            sr::quasi_blocks_kernel<<<1, 1024, 0, h->st>>>(n, h->band + 2 * n, h->band, h->band + n, h->qblk,
                                                           h->dnorm + 4);
            SR_CUDA_TRY(cudaGetLastError());
        } else {
            sr::gemm_dd_kernel<1><<<grid, 256, 0, h->st>>>(n, 1, Q, ldq, h->AQ, h->Delta, ld, nullptr, nullptr, 0,
                                                           h->partial);
            SR_CUDA_TRY(cudaGetLastError());
            SR_TRY(reduce_to(h, (int)tiles, 4));
        }
        sr::gemm_dd_kernel<2><<<grid, 256, 0, h->st>>>(n, 1, Q, ldq, Q, nullptr, ldq, nullptr, nullptr, 0,
                                                       h->partial);
        SR_CUDA_TRY(cudaGetLastError());
        SR_TRY(reduce_to(h, (int)tiles, 5));
        SR_TRY(sumsq<double>(h, n, A, lda, 0, 6));
    }
    SR_TRY(read_back(h));
    // A = 0 has Q^H A Q = 0: its relative residual is 0, not 0/0
    *stril_rel = h->hbuf[6] > 0.0 ? sqrt(h->hbuf[4]) / sqrt(h->hbuf[6]) : 0.0;
    *orth = sqrt(h->hbuf[5]);
    return SR_OK;
}

sr_status schur_refine_trisolve(schur_refine_t h, int n, void *dTE, int ld, const void *dDiag)
{
    if (!h || !dTE || !dDiag || n < 1 || n > h->nmax || ld < n) return SR_ERR_INVALID_ARG;
    SR_CUDA_TRY(cudaMemsetAsync(h->dflags, 0, sizeof(int), h->st));
    if (h->opt.quasi) {
        // the blocks from the band of the low-precision T in dTE and the FP64 diagonal
        const double *d = (const double *)dDiag;
        const unsigned g = (unsigned)((n + 255) / 256);
        if (h->opt.lp == SR_LP_FP32)
            sr::quasi_band_kernel<float><<<g, 256, 0, h->st>>>(n, (const float *)dTE, ld, h->band, h->band + h->nmax);
        else
            sr::quasi_band_kernel<double><<<g, 256, 0, h->st>>>(n, (const double *)dTE, ld, h->band,
                                                                 h->band + h->nmax);
        SR_CUDA_TRY(cudaGetLastError());
        sr::quasi_blocks_kernel<<<1, 1024, 0, h->st>>>(n, d, h->band, h->band + h->nmax, h->qblk, nullptr);
        SR_CUDA_TRY(cudaGetLastError());
        SR_CUDA_TRY(cudaMemcpyAsync(h->hblk, h->qblk, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, h->st));
        SR_CUDA_TRY(cudaStreamSynchronize(h->st));
        if (h->opt.lp == SR_LP_FP32)
            SR_TRY(solve_quasi<float>(h, n, (float *)dTE, ld, d));
        else
            SR_TRY(solve_quasi<double>(h, n, (double *)dTE, ld, d));
    } else if (is_dd(h->opt) || is_td(h->opt) || is_d6(h->opt))
        SR_TRY(solve<double>(h, n, (double *)dTE, ld, (const double *)dDiag, (const double *)dDiag + n));
    else if (is_cplx(h->opt))
        SR_TRY(solve<cf>(h, n, (cf *)dTE, ld, (const cd *)dDiag));
    else if (h->opt.lp == SR_LP_FP32)
        SR_TRY(solve<float>(h, n, (float *)dTE, ld, (const double *)dDiag));
    else
        SR_TRY(solve<double>(h, n, (double *)dTE, ld, (const double *)dDiag));
    SR_TRY(read_back(h));
    const int f = host_flags(h);
    if (f & SR_FLAG_TIMEOUT) return SR_ERR_TIMEOUT;
    if (f & SR_FLAG_NONDISTINCT) return SR_ERR_NONDISTINCT;
    if (f & SR_FLAG_NONFINITE) return SR_ERR_NONFINITE;
    return SR_OK;
}

sr_status schur_refine_solve_plan(int n, unsigned long long *tasks, long long cap, long long *count)
{
    if (n < 1 || n > 32768 || !count || cap < 0) return SR_ERR_INVALID_ARG;
    std::vector<unsigned long long> t;
    sr::trisolve_flow_plan(n, t);
    *count = (long long)t.size();
    if (tasks) std::copy(t.begin(), t.begin() + (size_t)std::min<long long>(cap, (long long)t.size()), tasks);
    return SR_OK;
}

sr_status schur_refine_selftest_wait_timeout(schur_refine_t h)
{
    if (!h) return SR_ERR_INVALID_ARG;
    return sr_flow_selftest(h);
}

sr_status schur_refine_gemm(schur_refine_t h, int transA, int m, int n, int k, const void *dA, int lda,
                            const void *dB, int ldb, void *dC, int ldc)
{
    if (!h || !dA || !dB || !dC || m < 1 || n < 1 || k < 1) return SR_ERR_INVALID_ARG;
    if (m > h->nmax || n > h->nmax || k > h->nmax) return SR_ERR_INVALID_ARG;
    if (lda < (transA ? k : m) || ldb < k || ldc < m) return SR_ERR_INVALID_ARG;
    SR_CUDA_TRY(cudaMemsetAsync(h->dflags, 0, sizeof(int), h->st));
    if (is_d6(h->opt)) {
        if (m != n || n != k) return SR_ERR_INVALID_ARG;   // square products only
        const D6Mat A = d6_caller(dA, lda, k), B = d6_caller(dB, ldb, n), C = d6_caller(dC, ldc, n);
        SR_TRY(sr::ozaki_split_d6(h, h->st, h->oz, sr::OZS_ROWS, sr::OZS_ROWS_LO, m, k, A.x, A.pl, A.ld,
                                  transA ? sr::OZ_COLS : sr::OZ_ROWS));
        SR_TRY(d6_split(h, sr::OZS_COLS, sr::OZS_COLS_LO, n, B, sr::OZ_COLS));
        SR_TRY(d6_products(h, sr::OZS_ROWS, sr::OZS_ROWS_LO, sr::OZS_COLS, sr::OZS_COLS_LO, n));
        SR_TRY(sr::ozaki_combine_d6(h, h->st, h->oz, sr::OZS_ROWS, sr::OZS_COLS, m, n, 1.0,
                                    sr::EpStoreD6{C.x, C.ld, C.pl}, nullptr, nullptr));
    } else if (is_td(h->opt)) {
        const TdMat A = td_caller(dA, lda, transA ? m : k), B = td_caller(dB, ldb, n), C = td_caller(dC, ldc, n);
        const int s = sr::kCrtDefaultModuliTD;
        SR_TRY(sr::ozaki_split_td(h, h->st, h->oz, sr::OZS_ROWS, m, k, A.x0, A.x1, A.x2, lda,
                                  transA ? sr::OZ_COLS : sr::OZ_ROWS, s));
        SR_TRY(sr::ozaki_split_td(h, h->st, h->oz, sr::OZS_COLS, n, k, B.x0, B.x1, B.x2, ldb, sr::OZ_COLS, s));
        SR_TRY(sr::ozaki_product(h, h->st, h->oz, sr::OZS_ROWS, sr::OZS_COLS, m, n, k, s, false, h->dflags));
        SR_TRY(sr::ozaki_combine(h, h->st, h->oz, sr::OZS_ROWS, sr::OZS_COLS, m, n, s, 1.0, false,
                                 sr::EpStoreTD{C.x0, C.x1, C.x2, C.ld}, nullptr, nullptr));
    } else if (is_dd(h->opt)) {
        const DdMat A = dd_caller(dA, lda, transA ? m : k), B = dd_caller(dB, ldb, n), C = dd_caller(dC, ldc, n);
        const sr::EpStoreDD ep{C.hi, C.lo, C.ld};
        if (is_emulated(h->opt)) {
            const int s = oz_s_dd(h);
            SR_TRY(sr::ozaki_split_dd(h, h->st, h->oz, sr::OZS_ROWS, m, k, A.hi, A.lo, lda,
                                      transA ? sr::OZ_COLS : sr::OZ_ROWS, s));
            SR_TRY(sr::ozaki_split_dd(h, h->st, h->oz, sr::OZS_COLS, n, k, B.hi, B.lo, ldb, sr::OZ_COLS, s));
            SR_TRY(sr::ozaki_product(h, h->st, h->oz, sr::OZS_ROWS, sr::OZS_COLS, m, n, k, s, false, h->dflags));
            SR_TRY(sr::ozaki_combine(h, h->st, h->oz, sr::OZS_ROWS, sr::OZS_COLS, m, n, s, 1.0, false, ep, nullptr,
                                     nullptr));
        } else {
            SR_TRY(ddk_gemm(h, transA != 0, m, n, k, A, B, ep, -1));
        }
    } else if (is_cplx(h->opt))
        SR_TRY(sr::ozaki_gemm(h, h->st, h->oz, transA != 0, m, n, k, dA, lda, dB, ldb, sr::EpStoreC{(cd *)dC, ldc},
                              nullptr, nullptr, oz_count(h->opt), h->dflags));
    else
        SR_TRY(hp_gemm(h, transA != 0, m, n, k, (const double *)dA, lda, (const double *)dB, ldb,
                       sr::EpStore{(double *)dC, ldc}, -1));
    SR_TRY(read_back(h));
    if (timed_out(h)) return SR_ERR_TIMEOUT;
    return SR_OK;
}

}  // extern "C"
