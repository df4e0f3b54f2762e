/*
 * schur_refine.h -- C ABI of the GB300 Schur-refinement library.
 *
 * Problem (Sec. 2, eq. "lowup"; Alg. 1 REQUIRE/ENSURE; Alg. 4): given a square
 * matrix A and a nearly unitary Qhat for which Qhat^H A Qhat is nearly upper
 * triangular, compute a unitary Q (to working high precision) with Q^H A Q
 * upper triangular. The library runs the Newton-like iteration of Alg. 4 on
 * one GPU: high-precision products form T^ = Q^H A Q and Y = Q^H Q - I, a
 * low-precision solve of stril(T L - L T) = -stril(T^) (eq. "linearsystem",
 * Alg. 2/3) gives L, and the merged Newton-Schulz update of eq. "NSmerged"
 * (Sec. 2.4) moves Q.
 *
 * Conventions for every entry point:
 *   - Matrices are column-major: element (i, j) of an n x n matrix M with
 *     leading dimension ld >= n lives at M[i + j*ld].
 *   - "device" pointers must address memory of the current CUDA device;
 *     "host" pointers address host memory.
 *   - The caller owns every matrix it passes. The library owns its workspace,
 *     allocated by schur_refine_create for the handle's maximum order and
 *     released by schur_refine_destroy.
 *   - Work is enqueued on the stream given at creation. Calls that return
 *     host values (norms, residuals, statuses) synchronize that stream before
 *     returning; the others return once the work is enqueued, except where
 *     stated.
 *   - No C++ exception crosses this interface. A null handle, a null required
 *     pointer, n < 1 or n above the handle's maximum, or ld < n gives
 *     SR_ERR_INVALID_ARG and changes nothing.
 *   - A handle may be used by one host thread at a time.
 */
#ifndef SCHUR_REFINE_H
#define SCHUR_REFINE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct schur_refine_ctx *schur_refine_t;

typedef enum {
    SR_OK = 0,
    SR_ERR_INVALID_ARG = 1,
    /* two diagonal entries of T coincide: the triangular equation has no
       unique solution (Theorem 1, Sec. 2.1) */
    SR_ERR_NONDISTINCT = 2,
    /* a NaN or Inf appeared (Example 3 of Sec. 3 ends this way) */
    SR_ERR_NONFINITE = 3,
    /* the stop test did not hold within max_iter passes, or the residual grew
       tenfold (Alg. 1's "until convergence" not reached) */
    SR_ERR_NOT_CONVERGED = 4,
    /* a bounded device-side wait ran out */
    SR_ERR_TIMEOUT = 5,
    SR_ERR_CUDA = 6,
    SR_ERR_OOM = 7,
    /* the option combination is not built */
    SR_ERR_UNSUPPORTED = 8
} sr_status;

/* element type of A and Q. SR_COMPLEX (complex128 data, complex64 low
   precision) is built for the emulated products (hp_gemm SR_HP_OZAKI_BF16 or
   SR_HP_OZAKI_CRT) with lp = SR_LP_FP32 and
   orders up to 8192; other combinations give SR_ERR_UNSUPPORTED at create. */
enum { SR_REAL = 0, SR_COMPLEX = 1 };
/* working high precision. SR_TARGET_DD (double-double, Sec. 3's higher
   working precisions one level above FP64) is built for real data with
   lp = SR_LP_FP64 and qhat_type = SR_QHAT_FP64. A double-double matrix is
   two column-major planes with the same leading dimension ld, hi and lo,
   standing for hi + lo; the lo plane starts ld * c elements after the hi
   plane, c = the number of columns stored.
   SR_TARGET_TD (triple-double, about 159 bits: Sec. 3's multi-double high
   precisions one level further) is built for real data with lp =
   SR_LP_FP64, qhat_type = SR_QHAT_FP64, hp_gemm = SR_HP_OZAKI_CRT (48
   moduli; ozaki_slices 0 or 48) and orders up to 8192. A triple-double
   matrix is three planes x0, x1, x2 (each ld * c elements after the one
   before), standing for x0 + x1 + x2 with x1 the double nearest to
   x - x0 and x2 the double nearest to x - x0 - x1.
   SR_TARGET_D6 (six doubles, about 318 bits: the 100-digit precision of
   Sec. 3, held as 6 doubles as the paper does) is built with the same
   options as SR_TARGET_TD; matrices are six planes x0 .. x5 in the same
   layout, each word the double nearest to what the words before it leave.
   Each high-precision product is four residue products of the operands'
   halves (48 moduli each). */
enum { SR_TARGET_FP64 = 0, SR_TARGET_DD = 1, SR_TARGET_TD = 2, SR_TARGET_D6 = 3 };
/* engine of the high-precision products (Sec. 2.4: "hp matrix-matrix
   multiplications"; the paper uses the Ozaki scheme, Sec. 3) */
enum {
    SR_HP_FP64 = 0,       /* native FP64 arithmetic */
    SR_HP_OZAKI_BF16 = 1, /* FP64 products emulated by splitting into bf16
                             slices multiplied exactly on tensor cores */
    SR_HP_OZAKI_CRT = 2   /* FP64 (double-double) products emulated by
                             residues: each operand vector is scaled to
                             integers of t bits, the integer product is formed
                             exactly modulo N pairwise coprime moduli <= 256
                             (one bf16 tensor-core product per modulus) and
                             rebuilt by the Chinese remainder theorem; N = 16
                             (32 for SR_TARGET_DD) by default */
};
/* low precision of the solve and of the products YW, W^2, W^3 (Alg. 4) */
enum { SR_LP_FP32 = 0, SR_LP_FP64 = 1 };
/* element type of the starting factor Qhat */
enum { SR_QHAT_FP32 = 0, SR_QHAT_FP64 = 1 };

typedef struct {
    int dtype;        /* SR_REAL or SR_COMPLEX */
    int target;       /* SR_TARGET_FP64, SR_TARGET_DD, SR_TARGET_TD or SR_TARGET_D6 */
    int hp_gemm;      /* SR_HP_FP64, SR_HP_OZAKI_BF16 or SR_HP_OZAKI_CRT */
    int lp;           /* SR_LP_FP32 (mixed form) or SR_LP_FP64 (all-FP64 form) */
    int qhat_type;    /* SR_QHAT_FP32 or SR_QHAT_FP64 */
    int full_sigma;   /* 1: keep W^2 Y + W^2 Y W in Sigma (eq. NSmerged);
                         0 (default): drop them, as Sec. 2.4 does */
    int max_iter;     /* passes of the REPEAT loop; <= 0 selects 10 */
    int ozaki_slices; /* bf16 slices per operand of the emulated
                         high-precision products; <= 0 selects the library
                         default (7; 14 for SR_TARGET_DD); at most 7 (14).
                         SR_HP_OZAKI_CRT: the number of moduli N (default 16;
                         32 for SR_TARGET_DD, 48 for SR_TARGET_TD and
                         SR_TARGET_D6; at most 16 (34; 48)); the operands
                         then carry t bits, the largest t with
                         K 2^(2t) < M / 2 for inner length K and M the
                         product of the moduli (t = 56 for N = 16 and
                         K <= 4096) */
    double tol;       /* stop when ||stril(T^)||_F / ||A||_F <= tol and the
                         last ||Q^H Q - I||_F <= sqrt(tol); <= 0 selects
                         1e-14 * sqrt(n) (1e-28 * n for SR_TARGET_DD, 1e-45 * n
                         for SR_TARGET_TD, 1e-93 * n for SR_TARGET_D6) */
    int profile;      /* 1: time every phase with CUDA events on the handle's
                         stream (see schur_refine_get_profile) */
    int batch_streams;/* schur_refine_batched with worker streams: matrices
                         refined concurrently, each on its own stream and
                         workspace; <= 0 selects 8, 1 refines them one after
                         another on the handle's stream */
    int batch_mode;   /* schur_refine_batched: 0 (default) = grouped launches
                         where built (real data, FP64 target, emulated
                         products with 7 digits or 16 moduli, FP32 low
                         precision and Qhat, truncated Sigma, dQhat given),
                         else worker streams; 1 = worker streams always */
    int tune;         /* work split of the emulated slice products (groups of
                         digit levels per output tile): 0 (default) = the
                         analytic makespan estimate; 1 = on the first product
                         of each shape, time the candidate splits (1 to 4
                         groups) and keep the fastest for the handle's life
                         (that first call synchronizes the stream) */
    int graph;        /* schur_refine_step for real data and the FP64 target:
                         0 (default) = the REPEAT loop runs on the host with
                         one synchronization per step of the loop; 1 = the
                         whole call is one CUDA graph (built on the first call
                         for given order and buffers, then replayed) whose
                         loop and stop test run on the device (conditional
                         WHILE / IF nodes), one synchronization per call;
                         same results; the profile (profile = 1) is not
                         recorded in this mode */
    int solve_mode;   /* triangular solve (Sec. 2.1): 0 (default) = the
                         dataflow form for a single matrix with FP32 low
                         precision, the stepwise form otherwise (FP64 and
                         complex64 solves and grouped batches are bound by
                         their arithmetic, where the stepwise form measured
                         faster); 1 = dataflow wherever built; 2 = stepwise
                         always. Dataflow: one launch in which the tiles of
                         the wavefront are claimed in subdiagonal order and
                         each waits only for the tiles it reads (bounded
                         waits; SR_ERR_TIMEOUT if one runs out). Stepwise:
                         one launch pair per block subdiagonal, replayed from
                         a CUDA graph. Same equations, sums in another order;
                         complex128 always uses the stepwise form */
    int symmetric;    /* 1: A is real symmetric or complex Hermitian
                         (Sec. 2.5): its Schur form is real diagonal, so T^
                         splits into its diagonal T and its off-diagonal part
                         E, and the solve of S4 becomes elementwise,
                         l_ij = -e_ij / (t_ii - t_jj) for i > j (the sign of
                         eq. (lij)); for complex data the divisor is formed
                         from the real parts of the diagonal. FP64 target
                         only; grouped batches fall back to worker streams.
                         0 (default): general A */
    double l_cap;     /* > 0: the trick of Example 4 (Sec. 3) for poorly
                         separated eigenvalues: while L is computed, an entry
                         with |l_ij| > l_cap (|l|^2 > l_cap^2 for complex
                         data, in the low precision) is set to zero at once,
                         before the entries computed after it use it; the
                         paper's example value is 1e-5. 0 (default): off.
                         Negative, NaN or infinite: SR_ERR_INVALID_ARG */
    int lp_slices;    /* the mixed form with emulated products (lp =
                         SR_LP_FP32): bf16 digits per operand of the
                         low-precision products YW, W^2, W^3 (Alg. 4, "can
                         all be computed in lp"): 3 (default, <= 0) carries
                         23 fraction bits, FP32-class; 2 carries 15 bits
                         (3 digit pairs instead of 6); 1 carries 7 bits, a
                         single bf16 product. More than 3: SR_ERR_INVALID_ARG */
    int quasi;        /* 1: real quasi-triangular Schur form (Sec. 3, real
                         Schur decompositions): complex-conjugate eigenvalue
                         pairs of real A stay in 2 x 2 diagonal blocks of T.
                         Each pass reads the blocks off T^ (rows k, k+1 form a
                         block where the 2 x 2 diagonal block of T^ has
                         non-real eigenvalues, taken from the top); E and the
                         residual are the entries below the diagonal blocks,
                         L is strictly block-lower, and each block equation
                         T_II X - X T_JJ = -C is solved through its Kronecker
                         matrix (at most 4 x 4). Real data, FP64 target,
                         graph = 0, symmetric = 0. The solve is the stepwise
                         form unless solve_mode = 1 selects the dataflow form
                         (both in a padded order in which no 2 x 2 block
                         crosses a 32-row tile); with every
                         block 1 x 1 the iteration is the triangular one.
                         schur_refine_residuals and schur_refine_trisolve of
                         such a handle use the blocks too. 0 (default): the
                         triangular Schur form */
} sr_options;

/* Fills *opt with the defaults: real, FP64 target, native FP64 products,
   FP32 low precision, FP32 Qhat, truncated Sigma. */
void schur_refine_default_options(sr_options *opt);

typedef struct {
    double stril_rel;  /* ||stril(Q^H A Q)||_F / ||A||_F at the last T^ formed */
    double orth;       /* ||Q^H Q - I||_F at the last Y formed (or of Qhat) */
    double w_norm;     /* ||W||_F of the last update, W = L - L^H */
    int iters;         /* passes = number of T^ formed */
    int hp_gemms;      /* high-precision products issued (4 per pass, Tables 3/4) */
} sr_norms;

/*
 * Creates a handle for orders up to n_max with the given options (NULL for
 * the defaults) and allocates its workspace on the current device. The
 * handle enqueues all work on cuda_stream (a cudaStream_t; NULL is the legacy
 * default stream). On failure *h is set to NULL.
 * Errors: SR_ERR_INVALID_ARG (h NULL, n_max < 1, bad option value),
 * SR_ERR_UNSUPPORTED (option combination not built), SR_ERR_OOM, SR_ERR_CUDA.
 */
sr_status schur_refine_create(schur_refine_t *h, int n_max, const sr_options *opt,
                              void *cuda_stream);

/*
 * Runs Alg. 4 (Sec. 2.4) on one matrix of order n <= n_max.
 *   dA        device, n x n, lda: A in FP64 (interleaved complex128 when
 *             dtype is SR_COMPLEX; two planes when target is SR_TARGET_DD,
 *             three for SR_TARGET_TD, six for SR_TARGET_D6, and likewise dQ
 *             and dT). Not modified.
 *   dQ        device, n x n, ldq, FP64 (complex128). In: the starting factor
 *             when dQhat is NULL. Out: the refined factor.
 *   dQhat     device, n x n with leading dimension ldq, element type
 *             qhat_type (complex64/complex128 when complex; FP64, one
 *             plane, for SR_TARGET_DD and SR_TARGET_TD), or NULL. When
 *             given, Q is first set to one Newton-Schulz step of Qhat
 *             converted to FP64 (Alg. 4, second line; eq. NS), and dQ's input
 *             value is ignored.
 *   dT        device, n x n, ld n, FP64 (complex128), or NULL: receives T^ = Q^H A Q of the
 *             last pass (its upper triangle is the Schur factor T).
 *   out       host, or NULL: norms and counters of the run.
 * Each pass forms T^ (2 products); if the stop test holds the run ends,
 * otherwise it solves for L, forms Y (1 product) and updates Q (1 product).
 * Returns SR_OK when the stop test held, SR_ERR_NOT_CONVERGED after max_iter
 * passes or when the residual grew tenfold after the second pass,
 * SR_ERR_NONDISTINCT / SR_ERR_NONFINITE when the solve failed (dQ then holds
 * the factor from before the failed update). Synchronizes the stream once per
 * pass to read the residual norm.
 */
sr_status schur_refine_step(schur_refine_t h, int n, const void *dA, int lda, void *dQ, int ldq,
                            const void *dQhat, void *dT, sr_norms *out);

/*
 * Refines `batch` independent matrices of orders n[b] <= n_max (host array),
 * each exactly as schur_refine_step with dQhat given (dQhat may be NULL: then
 * dQ[b] holds each starting factor).
 *   dA[b], dQ[b], dQhat[b]: host arrays of device pointers to column-major
 *   matrices with leading dimension n[b].
 *   iters_out[b], status_out[b]: host arrays (may be NULL) receiving each
 *   matrix's pass count and status.
 * Grouped launches (batch_mode 0 where built): all matrices advance pass by
 * pass together on the handle's stream, and every stage of a pass is one
 * launch for all matrices still iterating (per-matrix stop test, statuses and
 * pass counts as schur_refine_step; two synchronizations per pass). With
 * SR_HP_OZAKI_CRT each matrix's operands carry the fixed-point bits t of its
 * own order, so its factors equal schur_refine_step's on it alone bit for bit
 * (as with digits). The grouped workspace (about 60 bytes per matrix element
 * plus 10 KiB per matrix row of digits; the residue form keeps 16 planes per
 * high-precision slot against 7 digits) is allocated on first use, grown when
 * a later call needs more, and kept by the handle.
 * Worker streams (otherwise): the matrices are distributed over batch_streams
 * workers (host threads), each with its own stream and workspace (created on
 * first use and kept by the handle), so the refinements of different matrices
 * overlap on the GPU. The workers start after the work already enqueued on the
 * handle's stream, and that stream waits for all of them before the call
 * returns. Each matrix's result is the same as from schur_refine_step.
 * Returns SR_OK if every matrix converged, else the first non-OK status in
 * batch order.
 */
sr_status schur_refine_batched(schur_refine_t h, int batch, const int *n, const void *const *dA,
                               void *const *dQ, const void *const *dQhat, int *iters_out,
                               int *status_out);

/*
 * The two accuracy measures of Sec. 3 (Examples 2 and 4):
 *   *stril_rel = ||stril(Q^H A Q)||_F / ||A||_F,  *orth = ||Q^H Q - I||_F,
 * with every product accumulated in double-double arithmetic (TwoProd/TwoSum)
 * so that values near 1e-16 are resolved (for SR_TARGET_DD the double-double
 * A and Q enter with both planes; the accumulation error, about n * 1e-32
 * relative, stays far below the target 1e-28 n). dA, dQ as in
 * schur_refine_step; stril_rel, orth: host (for A = 0, *stril_rel is 0).
 * Synchronizes the stream.
 */
sr_status schur_refine_residuals(schur_refine_t h, int n, const void *dA, int lda, const void *dQ,
                                 int ldq, double *stril_rel, double *orth);

/*
 * schur_refine_residuals without a handle and without any device allocation.
 * The paper has no counterpart; this is a service for callers that cannot
 * call cudaMalloc -- for example an application whose device memory is owned
 * by its own pool allocator, or a service that forbids device allocation
 * after start-up to keep its memory footprint fixed. Creating a handle
 * allocates a workspace, so those callers use this entry point instead.
 *   n        order, 1 <= n <= 512; larger orders give SR_ERR_INVALID_ARG
 *   dA, dQ   device, as in schur_refine_residuals (FP64, real)
 *   stril_rel, orth   host, as in schur_refine_residuals
 *   cuda_stream       the cudaStream_t to run on (NULL: legacy default stream)
 * The scratch (A Q in double-double plus partial sums, about 4 MiB) is a
 * fixed array inside the library's device image; every GPU on which it has
 * been loaded keeps it until the process exits. Under CUDA's default lazy
 * module loading that memory is committed by the first call on a device:
 * a caller whose pool allocator reserves the device should make one call on
 * each device before the pool takes its memory (or set
 * CUDA_MODULE_LOADING=EAGER), or that first call can fail for lack of memory.
 * No cudaMalloc, cudaFree or other allocating routine is called. All calls on
 * a device share that array: calls whose GPU work overlaps (other streams or
 * host threads) race and must be ordered by the caller. Each call looks up
 * the array's device address on the current device before launching its
 * kernels. For A = 0, *stril_rel is 0. Synchronizes cuda_stream.
 */
sr_status schur_refine_residuals_noalloc(int n, const void *dA, int lda, const void *dQ, int ldq,
                                         double *stril_rel, double *orth, void *cuda_stream);

/*
 * The low-precision solve alone (Alg. 4, "solve ... in lp, using Alg. 3"):
 * solves stril(T L - L T) = -E for strictly lower L, order n <= n_max.
 *   dTE    device, n x n, ld: on entry its upper triangle (with diagonal)
 *          holds T and its strictly lower triangle holds E, in the handle's
 *          low precision (float for SR_LP_FP32, double for SR_LP_FP64;
 *          complex64/complex128 when complex). On exit the strictly lower
 *          triangle holds L; the upper triangle is unchanged.
 *   dDiag  device, n entries, FP64 (complex128): the diagonal of T in high
 *          precision; divisors t_ii - t_jj are formed from it and then
 *          rounded to the low precision. SR_TARGET_DD and SR_TARGET_TD: 2n
 *          entries, the high parts of the double-double diagonal (for
 *          SR_TARGET_TD the two leading words) followed by the low parts.
 * Returns SR_ERR_NONDISTINCT on a zero divisor (Theorem 1), SR_ERR_NONFINITE
 * on a non-finite entry of L. Synchronizes the stream.
 */
sr_status schur_refine_trisolve(schur_refine_t h, int n, void *dTE, int ld, const void *dDiag);

/*
 * Self-test of the dataflow solve's bounded waits (no counterpart in the
 * paper): solves a 64 x 64 FP32 problem (2 x 2 tiles) with a launch plan
 * that lists tile (0, 0) but not the tile (1, 0) it reads, so that the wait
 * for tile (1, 0) can never be satisfied. The wait gives up after its poll
 * limit (about a second), the kernel records SR_FLAG_TIMEOUT and returns,
 * and the call returns SR_ERR_TIMEOUT with the handle and its CUDA context
 * still usable. Any other result means the bounded wait did not work.
 * Allocates and frees its own small buffers; synchronizes the stream.
 */
sr_status schur_refine_selftest_wait_timeout(schur_refine_t h);

/*
 * The task list of the dataflow solve for order n (host code only; no device
 * is used): the order in which the launch's CTAs claim tasks. 64-bit entries:
 *   solve task  (bit 63 = 0): J = bits 0-15, I = bits 16-31 (tile (I, J) of
 *               32 x 32 tiles), number of helper tasks of the tile = bits
 *               32-47, highest block subdiagonal d the tile multiplies
 *               itself = bits 48-59 (it multiplies d = I-J+1 .. that one);
 *   helper task (bit 63 = 1): J, I, lowest d = bits 32-43, highest d = bits
 *               44-55, index among the tile's helpers = bits 56-62.
 * Every task follows, in the list, the tasks whose results it reads.
 *   tasks  host array of cap entries, or NULL to query the count only
 *   count  receives the number of tasks (copied: min(cap, count))
 * Returns SR_ERR_INVALID_ARG for n < 1 or n > 32768 or a NULL count.
 */
sr_status schur_refine_solve_plan(int n, unsigned long long *tasks, long long cap, long long *count);

/*
 * The constants of the residue form of the emulated products (hp_gemm =
 * SR_HP_OZAKI_CRT; the paper computes its high-precision products with the
 * Ozaki scheme, Sec. 3, and this is the Chinese-remainder variant of that
 * scheme). Host code only; no device is used.
 *   N        number of moduli, 1..49
 *   limbs    4 (FP64 results, needs M < 2^128), 8 (double-double results,
 *            M < 2^256) or 12 (triple-double results, M < 2^384)
 *   K        inner length of the product
 *   moduli   host, N entries: the moduli, the N largest pairwise coprime
 *            integers <= 256 taken greedily from 256 down
 *   weights  host, N * limbs entries: weight l is M_l (M_l^-1 mod m_l) 2^sigma
 *            (M = prod m_l, M_l = M / m_l) as little-endian 32-bit limbs
 *   M        host, limbs entries: M 2^sigma, its top bit at 32 limbs - 1
 *   sigma    host: the scaling exponent
 *   t        host: bits of the integer operands, the largest t with
 *            K 2^(2t) < M / 2
 * Returns SR_ERR_INVALID_ARG for N or limbs out of range, M >= 2^(32 limbs),
 * K < 1 or a NULL pointer.
 */
sr_status schur_refine_crt_info(int N, int limbs, long long K, int *moduli, unsigned *weights, unsigned *M,
                                int *sigma, int *t);

/*
 * One high-precision product with the handle's engine, as used for A Q and
 * Q^H (A Q): C = op(A) B with op(A) = A (transA = 0) or A^H (transA = 1).
 *   dA  device, FP64 (complex128): m x k (transA = 0) or k x m (transA = 1), lda
 *   dB  device, k x n, ldb;  dC device, m x n, ldc (overwritten).
 * SR_TARGET_DD: A, B and C are double-double (two planes each, see
 * SR_TARGET_DD), C accurate to about k * 1e-32 relative to |op(A)| |B|.
 * SR_TARGET_TD: three planes each; C is the exact product of the operands cut
 * to t = 162 bits per row of op(A) and column of B (K <= 4096), rounded once
 * to a triple-double. SR_TARGET_D6: six planes each, m = n = k; the operands
 * are cut to 2t - 2 = 322 bits, and C is rounded once to six doubles.
 * Sizes up to n_max in every dimension.
 */
sr_status schur_refine_gemm(schur_refine_t h, int transA, int m, int n, int k, const void *dA,
                            int lda, const void *dB, int ldb, void *dC, int ldc);

/* Phases of the iteration, after the split of Sec. 3, Table 2 ("matrix
   multiplication" versus "other operations"), refined per kernel family. */
enum {
    SR_PROF_HP_GEMM = 0,    /* native FP64 high-precision products */
    SR_PROF_OZ_SPLIT = 1,   /* emulated products: splitting into bf16 slices */
    SR_PROF_OZ_MMA = 2,     /* emulated products: tensor-core slice products */
    SR_PROF_OZ_COMBINE = 3, /* emulated products: FP64 recombination + epilogue */
    SR_PROF_SOLVE = 4,      /* triangular matrix equation */
    SR_PROF_LP_GEMM = 5,    /* low-precision products YW, W^2, W^3 */
    SR_PROF_OTHER = 6,      /* conversions, norms, copies */
    SR_PROF_KINDS = 8
};

typedef struct {
    double ms[SR_PROF_KINDS];        /* device time (CUDA events), 0 unless profile = 1 */
    long long flops[SR_PROF_KINDS];  /* algorithmic flops: 2mnk per product; for
                                        SR_PROF_OZ_MMA the bf16 flops issued */
    long long bytes[SR_PROF_KINDS];  /* algorithmic bytes moved to/from HBM */
    long long launches[SR_PROF_KINDS]; /* kernels launched by the library */
    long long spans[SR_PROF_KINDS];  /* timed regions */
} sr_profile;

/* Accumulated profile since creation or the last reset (synchronizes the
   stream). out: host. */
sr_status schur_refine_get_profile(schur_refine_t h, sr_profile *out);
sr_status schur_refine_reset_profile(schur_refine_t h);

/* Releases the workspace and the handle; NULL is ignored. */
void schur_refine_destroy(schur_refine_t h);

/* Human-readable name of a status code (static storage). */
const char *schur_refine_status_string(sr_status s);

#ifdef __cplusplus
}
#endif

#endif /* SCHUR_REFINE_H */
