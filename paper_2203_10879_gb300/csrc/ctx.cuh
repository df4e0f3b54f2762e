// The handle of the C ABI (schur_refine_t): options, stream, workspace and
// the cached launch plans and graphs. Shared by the translation units of the
// engine (single matrices: engine.cu; groups of matrices: batch.cu).
#pragma once
#include <vector>

#include "common.cuh"
#include "ozaki.cuh"

struct BatchWork;   // grouped-launch workspace of schur_refine_batched (batch.cu)

struct schur_refine_ctx {
    int nmax = 0;
    sr_options opt{};
    cudaStream_t st = nullptr;
    int dev = 0;
    // workspace (ld = nmax)
    double *AQ = nullptr, *Qw = nullptr, *Y = nullptr, *Delta = nullptr, *diag = nullptr;
    double *diag_lo = nullptr;   // double-double target: low parts of the diagonal of T^
    void *TE = nullptr, *W2 = nullptr, *YW = nullptr, *W2Y = nullptr, *W2YW = nullptr;   // low precision
    double *Wd = nullptr, *W2d = nullptr, *W2Yd = nullptr, *W2YWd = nullptr;   // FP64, emulated-product pass
    double *partial = nullptr;   // per-block partial sums
    size_t npartial = 0;
    double *dnorm = nullptr;     // [0] ||E||^2 [1] ||Y||^2 [2] ||W||^2 [3] ||A||^2 [4..] scratch
    int *dflags = nullptr;
    double *hbuf = nullptr;      // pinned host mirror of dnorm (8) + flags
    sr::OzakiWork oz{};
    // launch plan of the stepwise triangular solve
    int plan_n = 0, plan_b = 0;   // for order plan_n and tile plan_b
    uint32_t *plan = nullptr;
    size_t plan_cap = 0;
    std::vector<long long> plan_off;
    // the solve's two streams of work are captured once per (order, buffers)
    cudaStream_t cap_st = nullptr, aux_st = nullptr;
    cudaEvent_t sev0 = nullptr, sev1 = nullptr;
    struct SolveGraph { int n; const void *TE; int ld; const void *dhp; const void *dlo; int kind; cudaGraphExec_t exec; };
    std::vector<SolveGraph> graphs;
    // dataflow solve (see opt.solve_mode): ticket, abort, published and helper
    // words, 2 + 2 NB^2 ints; grid per low-precision kind (float, double, complex64)
    int *flow = nullptr;
    int flow_ctas[3] = {0, 0, 0};
    void *flow_acc = nullptr;                   // helpers' accumulators (n_max^2, low precision)
    unsigned long long *flow_plan = nullptr;    // task list for order flow_plan_n
    size_t flow_plan_cap = 0;
    int flow_plan_n = 0, flow_ntasks = 0;
    // schur_refine_batched: grouped-launch workspace, or worker sub-handles on their own streams
    BatchWork *bw = nullptr;
    std::vector<schur_refine_ctx *> subs;
    std::vector<cudaStream_t> sub_streams;
    cudaEvent_t bfork = nullptr;
    std::vector<cudaEvent_t> bjoin;
    // emulated pass: the Gram product Y = Q^H Q - I runs on gram_st while the
    // solve runs on st (its block sums go to partial2)
    cudaStream_t gram_st = nullptr;
    cudaEvent_t gev0 = nullptr, gev1 = nullptr;
    double *partial2 = nullptr;
    // graph mode (opt.graph): the refinement captured once per (order, buffers)
    // as one graph with device-side stop tests; capturing = true while it is built
    bool capturing = false;
    struct RefineGraph {
        int n = 0, lda = 0, ldq = 0;
        const void *A = nullptr, *Q = nullptr, *Qhat = nullptr, *T = nullptr;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
    } rgraph;
    void *ctl = nullptr;                  // device state of the graph's REPEAT loop
    std::vector<cudaStream_t> cstreams;   // capture streams of nested conditional bodies
    // real quasi-triangular form (opt.quasi): band of T^ (sub, super, diagonal
    // at offsets 0, nmax, 2 nmax), block array (device and pinned host copy), the
    // padded problem (order up to nqmax) and its index maps
    double *band = nullptr;
    int *qblk = nullptr, *hblk = nullptr;
    int nqmax = 0;
    void *TEq = nullptr, *qcpl = nullptr;   // qcpl: couplings of the 2 x 2 blocks, padded order
    void *step_acc = nullptr;               // stepwise solve: far products' sums, apart from E
    double *dhpq = nullptr;
    int *qpos = nullptr, *qinv = nullptr, *qblkq = nullptr, *hmaps = nullptr;
    // profiling
    sr_profile prof{};
    std::vector<cudaEvent_t> ev_pool;
    struct Span { int kind; cudaEvent_t a, b; };
    std::vector<Span> pending;
    std::vector<cudaEvent_t> open_ev;   // begin events of open phases (stack)
};

// schur_refine_batched with grouped launches (every stage of a pass runs for all
// matrices of the group in one launch); batch.cu
sr_status sr_batch_refine(schur_refine_ctx *h, int batch, const int *n, const void *const *dA, void *const *dQ,
                          const void *const *dQhat, int *iters_out, int *status_out);
bool sr_batch_supported(const sr_options &o);
// schur_refine_selftest_wait_timeout (batch.cu: the group form of the dataflow solve)
sr_status sr_flow_selftest(schur_refine_ctx *h);
void sr_batch_free(BatchWork *bw);
