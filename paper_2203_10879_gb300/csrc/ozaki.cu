// Split kernels and the tcgen05 slice-product kernel of the emulated FP64
// products (see ozaki.cuh for the scheme).
//
// Slice-product kernel, persistent (one CTA per SM walks the 128 x 256 output
// tiles), 10 warps:
//   warp 0      TMA producer: K-blocks of 64 bf16 (128 bytes, 128B swizzle)
//               of one B digit matrix (MMA "A", 128 rows = output columns j)
//               and one op(A) digit matrix (MMA "B", 256 rows = output rows i)
//               into a 4-stage shared-memory ring.
//   warp 1      allocates 512 TMEM columns (two 256-column FP32 accumulators)
//               and issues tcgen05.mma (M = 128, N = 256, K = 16) from one
//               thread; each 256-long K-chunk of one digit pair fills one
//               accumulator.
//   warps 2..9  drain a full accumulator with tcgen05.ld (warp w reads TMEM
//               lanes 32*(w%4).., half (w-2)/4 of the columns), convert the
//               exact FP32 integers to int32 by adding 1.5*2^23 and taking the
//               bit pattern, and accumulate them per level; at the end of a
//               level they store the level's int32 plane (column-major).
// Every wait on an mbarrier is bounded (about 2 s of clock); on expiry the CTA
// raises SR_FLAG_TIMEOUT, lets every role leave its loop, waits (bounded) for
// its own TMA loads and MMAs, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <numeric>

#include "ozaki.cuh"

namespace sr {
namespace {

constexpr int BM = kOzakiTileJ;           // MMA M: output columns j (TMEM lanes)
constexpr int BN = kOzakiTileI;           // MMA N: output rows i (TMEM columns)
constexpr int BK = 64;                    // K per stage: 64 bf16 = 128 bytes
constexpr int KB_PER_CHUNK = kOzakiKChunk / BK;
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;      // 16 KiB: column-side digits
constexpr int B_BYTES = BN * BK * 2;      // 32 KiB: row-side digits
constexpr int NUM_THREADS = 320;
constexpr uint32_t TMEM_COLS = 2 * BN;    // two accumulators of BN columns
constexpr long long WAIT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz
constexpr int SMEM_BYTES = STAGES * (A_BYTES + B_BYTES) + 1024 + 256;

// instruction descriptor, kind::f16: D f32 (bits 4-5 = 1), A and B bf16
// (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N>>3 at bit 17,
// M>>4 at bit 24.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);
constexpr uint32_t IDESC_NEG_A = 1u << 13;   // negate the A operand (complex products)

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.b32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait. Gives up when *abort is set by another role or after
// WAIT_CYCLES (then sets *abort itself).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > WAIT_CYCLES) {
            *abort = 1;
            return false;
        }
    }
    return true;
}
// Bounded wait that ignores the abort flag (used while draining).
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > WAIT_CYCLES) return;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *map, uint32_t bar, int c0, int c1)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t acc)
{
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct MmaArgs {
    int s;            // digits per operand
    int nch;          // K-chunks of 256 (complex: both halves)
    int Pmax;         // row stride of digit matrices and planes
    int tiles_i;      // row tiles (BN rows of C)
    int tiles_j;      // column tiles (BM columns of C) per part
    int ntiles;       // tiles_i * tiles_j (* 2 when complex)
    int symmetric;    // 1: skip tiles entirely below the diagonal (mirrored by the combine)
    int cplx;         // stacked [re; im] vectors; tiles of the second half form imaginary parts
    int conj;         // complex, row side conjugated (the sign g of the header)
    int32_t *planes;  // [s][pstride]
    size_t pstride;   // Pmax * Pmax (2 Pmax * Pmax when complex)
    int *flags;
    // work items: (active tile, level group); group g holds levels
    // [lvl[g], lvl[g+1]). Item x is group x / nact of active tile x % nact.
    int nact;         // tiles formed (all, or those on and above the diagonal)
    int groups;
    int nitems;       // nact * groups (or the length of items)
    int lvl[kCrtMaxModuli + 1];
    const MmaItem *items;   // explicit work items (grouped products), else null
    // residue form: level l is the single product of the residues modulo mods[l]
    // (row-side and column-side slot plane l), drained into an exact int32 sum
    // and stored reduced modulo mods[l] as a byte plane
    int crt;
    int mods[kCrtMaxModuli];
    unsigned long long inv40[kCrtMaxModuli];
    unsigned off28[kCrtMaxModuli];
};

// what one work item needs: digit rows, K-chunks, levels, where its planes go
struct ItemView {
    int ra, rb, nch, kbl, ppa, lb, le, im, ldp, rlim, clim;
    long long poff;
};

// Digit pairs per accumulator: a one-chunk item whose K is at most 128 (64)
// accumulates 2 (4) pairs of a level before the drain, still at most 256
// products in one FP32 sum (exact below 2^22, the bias trick's range).
__device__ __forceinline__ int pairs_per_acc(int nch, int kbl) { return nch == 1 ? KB_PER_CHUNK / kbl : 1; }

// number of row tiles formed in column tile bj (of one part)
__device__ __forceinline__ int active_in_column(const MmaArgs &a, int bj)
{
    if (!a.symmetric) return a.tiles_i;
    return min(a.tiles_i, (bj * BM + BM - 1) / BN + 1);
}

// item -> tile (index as in tile_coords) and its level range
__device__ __forceinline__ void item_coords(const MmaArgs &a, int item, int &i0, int &j0, int &im, int &lb, int &le)
{
    const int g = item / a.nact;
    int r = item - g * a.nact;
    lb = a.lvl[g];
    le = a.lvl[g + 1];
    int bj = 0;
    const int cols = a.tiles_j * (a.cplx ? 2 : 1);
    for (; bj < cols; ++bj) {
        const int cnt = active_in_column(a, bj % a.tiles_j);
        if (r < cnt) break;
        r -= cnt;
    }
    i0 = r * BN;
    im = bj >= a.tiles_j;
    j0 = (im ? bj - a.tiles_j : bj) * BM;
}

template <bool ITEMS>
__device__ __forceinline__ ItemView get_item(const MmaArgs &a, int item)
{
    ItemView v;
    if constexpr (ITEMS) {
        const MmaItem it = a.items[item];
        v.ra = it.ra; v.rb = it.rb; v.nch = it.nch; v.kbl = it.kbl; v.lb = it.lb; v.le = it.le; v.im = 0;
        v.ldp = it.ldp; v.rlim = it.rlim; v.clim = it.clim; v.poff = it.poff;
        v.ppa = pairs_per_acc(v.nch, v.kbl);
        return v;
    }
    int i0, j0, im, lb, le;
    item_coords(a, item, i0, j0, im, lb, le);
    v.ra = i0; v.rb = j0; v.nch = a.nch; v.kbl = KB_PER_CHUNK; v.lb = lb; v.le = le; v.im = im;
    v.ldp = a.Pmax; v.rlim = 1 << 30; v.clim = 1 << 30; v.ppa = 1;
    v.poff = (long long)(j0 + (im ? a.Pmax : 0)) * a.Pmax + i0;
    return v;
}

// column-side K-chunk read for chunk c: the halves are swapped for an imaginary part
__device__ __forceinline__ int col_chunk(const MmaArgs &a, int c, int im)
{
    if (!im) return c;
    const int hh = a.nch >> 1;
    return c < hh ? c + hh : c - hh;
}

// the chunks whose product enters with a minus sign: second half, and
// re with g = +1 (-r2.c2) or im with g = -1 (-r2.c1)
__device__ __forceinline__ uint32_t chunk_idesc(const MmaArgs &a, int c, int im)
{
    const bool neg = a.cplx && c >= (a.nch >> 1) && (im == a.conj);
    return neg ? (IDESC | IDESC_NEG_A) : IDESC;
}

// Persistent: CTA b takes tiles b, b + gridDim.x, ... Every role walks the same
// sequence of (tile, level l, pair p, chunk c, K-block kb).
template <bool ITEMS>
__global__ void __launch_bounds__(NUM_THREADS, 1)
ozaki_mma_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, MmaArgs args)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *tileA = smem;                             // [STAGES][A_BYTES]  column-side digits (rows j)
    unsigned char *tileB = smem + STAGES * A_BYTES;          // [STAGES][B_BYTES]  row-side digits (rows i)
    uint64_t *bars = (uint64_t *)(smem + STAGES * (A_BYTES + B_BYTES));
    uint64_t *full = bars, *empty = bars + STAGES, *accf = bars + 2 * STAGES, *acce = accf + 2, *done = acce + 2;
    uint32_t *tmem_slot = (uint32_t *)(done + 1);
    volatile int *abort = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int P = args.Pmax;

    if (threadIdx.x == 0) {
        for (int q = 0; q < STAGES; ++q) {
            mbar_init(smem_u32(&full[q]), 1);
            mbar_init(smem_u32(&empty[q]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&accf[b]), 1);
            mbar_init(smem_u32(&acce[b]), 8);
        }
        mbar_init(smem_u32(done), 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer ----
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
            int stage = 0;
            uint32_t phase = 0;
            int issued = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < args.nitems && ok; item += gridDim.x) {
                const ItemView v = get_item<ITEMS>(args, item);
                for (int l = v.lb; l < v.le && ok; ++l)
                    for (int p = args.crt ? l : 0; p <= l && ok; ++p) {
                        const int q = args.crt ? l : l - p;
                        for (int c = 0; c < v.nch && ok; ++c)
                            for (int kb = 0; kb < (ITEMS && c == v.nch - 1 ? v.kbl : KB_PER_CHUNK); ++kb) {
                                if (!mbar_wait(smem_u32(&empty[stage]), phase ^ 1, abort)) { ok = false; break; }
                                const uint32_t fb = smem_u32(&full[stage]);
                                mbar_expect_tx(fb, A_BYTES + B_BYTES);
                                const int kc = c * kOzakiKChunk + kb * BK;
                                const int kcj = col_chunk(args, c, v.im) * kOzakiKChunk + kb * BK;
                                tma_load_2d(smem_u32(tileA + stage * A_BYTES), &tmB, fb, kcj, q * P + v.rb);
                                tma_load_2d(smem_u32(tileB + stage * B_BYTES), &tmA, fb, kc, p * P + v.ra);
                                ++issued;
                                if (++stage == STAGES) { stage = 0; phase ^= 1; }
                            }
                    }
            }
            // wait for the loads still in flight before the CTA may exit: load number
            // x went to stage x % STAGES in phase (x / STAGES) & 1
            const int inflight = issued < STAGES ? issued : STAGES;
            for (int d = 1; d <= inflight; ++d) {
                const int x = issued - d;
                mbar_drain(smem_u32(&full[x % STAGES]), (uint32_t)((x / STAGES) & 1));
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer ----
            int stage = 0;
            uint32_t phase = 0;
            int t = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < args.nitems && ok; item += gridDim.x) {
                const ItemView v = get_item<ITEMS>(args, item);
                // one accumulator per (pair group, chunk); a group holds v.ppa pairs
                // (more than one only for one-chunk items, whose order of loads is
                // then the same pair by pair)
                const int ppa = ITEMS ? v.ppa : 1;
                for (int l = v.lb; l < v.le && ok; ++l)
                    for (int p0 = args.crt ? l : 0; p0 <= l && ok; p0 += ppa)
                        for (int c = 0; c < v.nch && ok; ++c) {
                            const uint32_t idesc = chunk_idesc(args, c, v.im);
                            const int b = t & 1;
                            const uint32_t aph = (t >> 1) & 1;
                            if (!mbar_wait(smem_u32(&acce[b]), aph ^ 1, abort)) { ok = false; break; }
                            tc_fence_after();
                            const uint32_t dt = tmem + (uint32_t)(b * BN);
                            const int p1 = min(p0 + ppa, l + 1);
                            for (int p = p0; p < p1 && ok; ++p)
                                for (int kb = 0; kb < (ITEMS && c == v.nch - 1 ? v.kbl : KB_PER_CHUNK); ++kb) {
                                    if (!mbar_wait(smem_u32(&full[stage]), phase, abort)) { ok = false; break; }
                                    tc_fence_after();
                                    const uint64_t ad = sdesc_sw128(smem_u32(tileA + stage * A_BYTES));
                                    const uint64_t bd = sdesc_sw128(smem_u32(tileB + stage * B_BYTES));
#pragma unroll
                                    for (int kk = 0; kk < BK / 16; ++kk)
                                        mma_bf16(dt, ad + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk), idesc,
                                                 (p != p0 || kb != 0 || kk != 0) ? 1u : 0u);
                                    mma_commit(smem_u32(&empty[stage]));
                                    if (++stage == STAGES) { stage = 0; phase ^= 1; }
                                }
                            if (!ok) break;
                            mma_commit(smem_u32(&accf[b]));
                            ++t;
                        }
            }
            // all issued MMAs complete before TMEM is released
            mma_commit(smem_u32(done));
            mbar_drain(smem_u32(done), 0);
        }
    } else {
        // ---- epilogue: drain accumulators, exact integer sums per level ----
        const int ew = warp - 2;
        const int lg = warp & 3;          // TMEM lane group this warp may access
        const int half = ew >> 2;         // which BN/2 columns
        uint32_t acc[BN / 2];
        int t = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < args.nitems && ok; item += gridDim.x) {
            const ItemView v = get_item<ITEMS>(args, item);
            const int jl = lg * 32 + lane;                        // plane column from the tile's origin
            for (int l = v.lb; l < v.le && ok; ++l) {
#pragma unroll
                for (int c = 0; c < BN / 2; ++c) acc[c] = 0u;
                uint32_t count = 0;
                for (int p0 = args.crt ? l : 0; p0 <= l && ok; p0 += (ITEMS ? v.ppa : 1))
                    for (int c = 0; c < v.nch; ++c) {
                        const int b = t & 1;
                        const uint32_t aph = (t >> 1) & 1;
                        // one lane polls so the whole warp leaves together on a timeout
                        int got = 0;
                        if (lane == 0) got = mbar_wait(smem_u32(&accf[b]), aph, abort) ? 1 : 0;
                        got = __shfl_sync(0xffffffffu, got, 0);
                        if (!got) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t ta = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(b * BN + half * (BN / 2));
#pragma unroll
                        for (int g = 0; g < BN / 32; ++g) {
                            uint32_t r[16];
                            tmem_ld16(ta + 16 * g, r);
#pragma unroll
                            for (int x = 0; x < 16; ++x)
                                acc[16 * g + x] += __float_as_uint(__fadd_rn(__uint_as_float(r[x]), 12582912.0f));
                        }
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(smem_u32(&acce[b]));
                        ++t;
                        ++count;
                    }
                if (!ok) break;
                const uint32_t bias = count * 0x4B400000u;
                if (args.crt && (!ITEMS || jl < v.clim)) {
                    // the exact sum (|sum| <= 64 chunks * 2^22 = 2^28) reduced modulo m into bytes
                    // (a work item's region rows come in multiples of 32: whole 16-byte stores)
                    const uint32_t m = (uint32_t)args.mods[l], off = args.off28[l];
                    const unsigned long long inv = args.inv40[l];
                    const int rmax = ITEMS ? v.rlim - half * (BN / 2) : BN;
                    uint8_t *dst8 = reinterpret_cast<uint8_t *>(args.planes) + (size_t)l * args.pstride +
                                    (size_t)v.poff + (size_t)jl * v.ldp + (size_t)(half * (BN / 2));
#pragma unroll
                    for (int c = 0; c < BN / 2; c += 16) {
                        uint32_t wd[4];
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            uint32_t pk = 0;
#pragma unroll
                            for (int x = 0; x < 4; ++x) {
                                const uint32_t u = (acc[c + 4 * b + x] - bias) + off;   // >= 0, < 2^30
                                const uint32_t qq = (uint32_t)(((unsigned long long)u * inv) >> 40);
                                pk |= (u - qq * m) << (8 * x);
                            }
                            wd[b] = pk;
                        }
                        if (c < rmax) *reinterpret_cast<uint4 *>(dst8 + c) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
                    }
                } else if (args.crt) {
                    // a column beyond the item's region: nothing to store
                } else if (!ITEMS || jl < v.clim) {
                    int32_t *dst = args.planes + (size_t)l * args.pstride + (size_t)v.poff + (size_t)jl * v.ldp +
                                   (size_t)(half * (BN / 2));
                    const int rmax = v.rlim - half * (BN / 2);   // region rows come in multiples of 4
#pragma unroll
                    for (int c = 0; c < BN / 2; c += 4) {
                        const int4 x4 = make_int4((int)(acc[c] - bias), (int)(acc[c + 1] - bias),
                                                  (int)(acc[c + 2] - bias), (int)(acc[c + 3] - bias));
                        if (!ITEMS || c < rmax) *reinterpret_cast<int4 *>(dst + c) = x4;
                    }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    if (threadIdx.x == 0 && *abort) atomicOr(args.flags, SR_FLAG_TIMEOUT);
}

// ---- split: X(r, kk) -> s bf16 digit matrices [p][r][kk] and exponents -------------
// LAYOUT OZ_COLS: X(r, kk) = X[kk + r*ld] (vector r = column r);
// LAYOUT OZ_ROWS: X(r, kk) = X[r + kk*ld] (vector r = row r).
// Complex (Tin = cd): position kk of the stacked vector is the real part of
// entry kk for kk < Kh and the imaginary part of entry kk - Kh after that.
// Two kernels, each over a 2-D grid of (32 vectors) x (a stretch of K):
//   ozaki_absmax_kernel  largest |x| per vector (bit patterns of non-negative
//                        doubles order like the values), atomicMax per vector;
//   ozaki_digits_kernel  scale exponent from that maximum, then the fixed-point
//                        digits of every entry; rows up to the next multiple of
//                        32 and K up to Kp are written as zero digits.
constexpr int SPLIT_KT = 256;   // K per absmax CTA
constexpr int DIGIT_KT = 64;    // K per digits CTA

__device__ __forceinline__ double split_part(double v, int) { return v; }
__device__ __forceinline__ double split_part(cd v, int part) { return part ? v.y : v.x; }

// entry (r, kk) of the (stacked) vectors; Kh = INT_MAX for real input
template <typename Tin, int LAYOUT>
__device__ __forceinline__ double split_entry(const Tin *__restrict__ X, int ld, int R, int K, int Kh, int r, int kk)
{
    const int part = kk >= Kh ? 1 : 0;
    const int e = kk - part * Kh;
    if (r >= R || e >= K) return 0.0;
    const Tin v = LAYOUT == OZ_COLS ? X[(size_t)e + (size_t)r * ld] : X[(size_t)r + (size_t)e * ld];
    return split_part(v, part);
}

template <typename Tin, int LAYOUT>
__device__ __forceinline__ void split_load_tile(double (&tile)[32][33], const Tin *__restrict__ X, int ld, int R,
                                                int K, int Kh, int r0, int k0)
{
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        int v, kk;
        if (LAYOUT == OZ_COLS) { kk = k0 + tx; v = ty + 8 * w; } else { v = tx; kk = k0 + ty + 8 * w; }
        tile[v][kk - k0] = split_entry<Tin, LAYOUT>(X, ld, R, K, Kh, r0 + v, kk);
    }
}

// Kv: length of the (stacked) vectors: K, or 2 Kh when complex
template <typename Tin, int LAYOUT>
__device__ __forceinline__ void absmax_body(int bx, int by, int R, int K, int Kh, int Kv, const Tin *__restrict__ X,
                                            int ld, unsigned long long *__restrict__ vmax)
{
    __shared__ double tile[32][33];
    __shared__ unsigned long long smax[32];
    const int r0 = bx * 32, kbeg = by * SPLIT_KT;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    if (threadIdx.x < 32) smax[threadIdx.x] = 0ull;
    unsigned long long m[4] = {0ull, 0ull, 0ull, 0ull};
    for (int k0 = kbeg; k0 < kbeg + SPLIT_KT && k0 < Kv; k0 += 32) {
        __syncthreads();
        split_load_tile<Tin, LAYOUT>(tile, X, ld, R, K, Kh, r0, k0);
        __syncthreads();
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const unsigned long long b =
                (unsigned long long)__double_as_longlong(tile[ty + 8 * w][tx]) & 0x7fffffffffffffffull;
            m[w] = b > m[w] ? b : m[w];
        }
    }
#pragma unroll
    for (int w = 0; w < 4; ++w) atomicMax(&smax[ty + 8 * w], m[w]);
    __syncthreads();
    if (threadIdx.x < 32 && r0 + threadIdx.x < R) atomicMax(&vmax[r0 + threadIdx.x], smax[threadIdx.x]);
}

template <typename Tin, int LAYOUT>
__global__ void __launch_bounds__(256)
ozaki_absmax_kernel(int R, int K, int Kh, int Kv, const Tin *__restrict__ X, int ld,
                    unsigned long long *__restrict__ vmax)
{
    absmax_body<Tin, LAYOUT>(blockIdx.x, blockIdx.y, R, K, Kh, Kv, X, ld, vmax);
}

__device__ __forceinline__ int split_exponent(unsigned long long b)
{
    const int eb = (int)(b >> 52);
    if (eb == 0x7ff) return kOzakiExpNonfinite;   // Inf or NaN in the vector
    if (eb == 0) return -1022;                    // zero or subnormal maximum
    return eb - 1022;                             // max < 2^e
}

// The s balanced base-256 digits of a fixed-point integer X (plane p holds
// the digit of weight 256^(s-1-p), all in [-128, 127] but the top one) are
// the bytes of Y = X + 128 (1 + 256 + ... + 256^(s-2)) less 128, and the top
// digit is Y >> 8(s-1): adding 128 to every lower digit makes each a plain
// byte, so no carries have to be propagated digit by digit.
__device__ __forceinline__ void write_digits(long long X, int s, __nv_bfloat16 *__restrict__ o, size_t pstride)
{
    const unsigned long long bias = s > 1 ? 0x8080808080808080ull >> (8 * (9 - s)) : 0ull;
    const unsigned long long Y = (unsigned long long)X + bias;
#pragma unroll
    for (int q = 0; q < kOzakiMaxSlices - 1; ++q)
        if (q < s - 1) o[(size_t)(s - 1 - q) * pstride] = __int2bfloat16_rn((int)((Y >> (8 * q)) & 255u) - 128);
    o[0] = __int2bfloat16_rn((int)((long long)Y >> (8 * (s - 1))));
}

// the same for a 128-bit X and up to kOzakiMaxSlicesDD digits
__device__ __forceinline__ void write_digits128(__int128 X, int s, __nv_bfloat16 *__restrict__ o, size_t pstride)
{
    const int nb = s - 1;
    const unsigned long long pat = 0x8080808080808080ull;
    const unsigned long long blo = nb >= 8 ? pat : (nb > 0 ? pat >> (64 - 8 * nb) : 0ull);
    const unsigned long long bhi = nb > 8 ? pat >> (64 - 8 * (nb - 8)) : 0ull;
    const unsigned __int128 Y = (unsigned __int128)X + (((unsigned __int128)bhi << 64) | blo);
    const unsigned long long ylo = (unsigned long long)Y, yhi = (unsigned long long)(Y >> 64);
#pragma unroll
    for (int q = 0; q < kOzakiMaxSlicesDD - 1; ++q)
        if (q < nb) {
            const unsigned long long w = q < 8 ? ylo >> (8 * q) : yhi >> (8 * (q - 8));
            o[(size_t)(s - 1 - q) * pstride] = __int2bfloat16_rn((int)(w & 255u) - 128);
        }
    o[0] = __int2bfloat16_rn((int)(long long)((__int128)Y >> (8 * nb)));
}

// Kp: stacked length written (K rounded up to the chunk, or 2 Kh when complex)
template <typename Tin, int LAYOUT>
__device__ __forceinline__ void digits_body(int bx, int by, int R, int K, int Kh, int Kp, const Tin *__restrict__ X,
                                            int ld, int s, int Pmax, int Kmax,
                                            const unsigned long long *__restrict__ vmax,
                                            __nv_bfloat16 *__restrict__ out, int *__restrict__ exps)
{
    __shared__ double tile[32][33];
    __shared__ int sexp[32];
    const int r0 = bx * 32, kbeg = by * DIGIT_KT;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    if (threadIdx.x < 32) {
        const int r = r0 + threadIdx.x;
        const int e = (r < R) ? split_exponent(vmax[r]) : 0;
        sexp[threadIdx.x] = e;
        if (by == 0) exps[r] = e;
    }
    const int F = 7 + 8 * (s - 1);
    const size_t pstride = (size_t)Pmax * Kmax;
    for (int k0 = kbeg; k0 < kbeg + DIGIT_KT && k0 < Kp; k0 += 32) {
        __syncthreads();
        split_load_tile<Tin, LAYOUT>(tile, X, ld, R, K, Kh, r0, k0);
        __syncthreads();
#pragma unroll 1
        for (int w = 0; w < 4; ++w) {
            const int v = ty + 8 * w;
            const int r = r0 + v;
            const int kk = k0 + tx;
            const double x = tile[v][tx];   // zero outside the matrix
            const int e = sexp[v];
            long long Xi = 0;
            if (e != kOzakiExpNonfinite && r < R) {
                const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
                const int eb = (int)((bits >> 52) & 0x7ff);
                unsigned long long mant = bits & 0xfffffffffffffull;
                int ex;
                if (eb == 0) ex = -1074; else { mant |= 1ull << 52; ex = eb - 1075; }
                const int sh = ex + F - e;                // x * 2^(F-e) = mant * 2^sh
                unsigned long long mag;
                if (mant == 0) mag = 0;
                else if (sh >= 0) mag = mant << sh;       // sh <= F - 52 here, no overflow
                else if (-sh >= 64) mag = 0;
                else mag = (mant + (1ull << (-sh - 1))) >> (-sh);
                Xi = (bits >> 63) ? -(long long)mag : (long long)mag;
            }
            // digits in [-128, 127]; the top one takes the rest
            write_digits(Xi, s, out + (size_t)r * Kmax + (size_t)kk, pstride);
        }
    }
}

template <typename Tin, int LAYOUT>
__global__ void __launch_bounds__(256, 4)
ozaki_digits_kernel(int R, int K, int Kh, int Kp, const Tin *__restrict__ X, int ld, int s, int Pmax, int Kmax,
                    const unsigned long long *__restrict__ vmax, __nv_bfloat16 *__restrict__ out,
                    int *__restrict__ exps)
{
    digits_body<Tin, LAYOUT>(blockIdx.x, blockIdx.y, R, K, Kh, Kp, X, ld, s, Pmax, Kmax, vmax, out, exps);
}

// Grouped split: the blocks of every matrix in one flat grid; block x belongs
// to matrix a with start[a] <= x < start[a + 1] (a binary search), its
// position within the matrix's grid of (32 vectors) x (K stretch) is
// x - start[a]. Each matrix's vectors go to its own slot rows.
template <int LAYOUT>
__global__ void __launch_bounds__(256)
ozaki_absmax_group_kernel(const SplitMat *__restrict__ mats, const int *__restrict__ start, int m,
                          unsigned long long *__restrict__ vmax)
{
    const int a = group_find(start, m, blockIdx.x);
    const SplitMat g = mats[a];
    const int local = blockIdx.x - start[a], gx = (g.R + 31) / 32;
    absmax_body<double, LAYOUT>(local % gx, local / gx, g.R, g.K, INT_MAX, g.K, g.X, g.ld, vmax + g.row0);
}

template <int LAYOUT>
__global__ void __launch_bounds__(256, 4)
ozaki_digits_group_kernel(const SplitMat *__restrict__ mats, const int *__restrict__ start, int m, int s, int Pmax,
                          int Kmax, const unsigned long long *__restrict__ vmax, __nv_bfloat16 *__restrict__ out,
                          int *__restrict__ exps)
{
    const int a = group_find(start, m, blockIdx.x);
    const SplitMat g = mats[a];
    // work items stop their last K-chunk at the order rounded to 64 (MmaItem::kbl):
    // digits past that are never read
    const int Kp = (g.K + 63) / 64 * 64;
    const int local = blockIdx.x - start[a], gx = (g.R + 31) / 32;
    digits_body<double, LAYOUT>(local % gx, local / gx, g.R, g.K, INT_MAX, Kp, g.X, g.ld, s, Pmax, Kmax,
                                vmax + g.row0, out + (size_t)g.row0 * Kmax, exps + g.row0);
}

// Double-double input: the fixed-point value of hi + lo with F = 7 + 8(s-1)
// fraction bits is formed exactly in a signed 128-bit integer (each part
// rounded to the nearest unit; |hi| < 2^e bounds both), then cut into s
// digits like the FP64 split. The exponent comes from the largest |hi| of the
// vector: |hi + lo| < 2^e as well, since |lo| is at most half an ulp of hi.
__device__ __forceinline__ __int128 dd_fixed_part(double x, int F, int e)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int eb = (int)((bits >> 52) & 0x7ff);
    unsigned long long mant = bits & 0xfffffffffffffull;
    int ex;
    if (eb == 0) ex = -1074; else { mant |= 1ull << 52; ex = eb - 1075; }
    const int sh = ex + F - e;                     // x * 2^(F-e) = mant * 2^sh, sh <= F - 53
    __int128 mag;
    if (mant == 0) mag = 0;
    else if (sh >= 0) mag = (__int128)mant << sh;
    else if (-sh >= 64) mag = 0;
    else mag = (__int128)((mant + (1ull << (-sh - 1))) >> (-sh));
    return (bits >> 63) ? -mag : mag;
}

template <int LAYOUT>
__global__ void __launch_bounds__(256, 2)
ozaki_digits_dd_kernel(int R, int K, int Kp, const double *__restrict__ Xh, const double *__restrict__ Xl, int ld,
                       int s, int Pmax, int Kmax, const unsigned long long *__restrict__ vmax,
                       __nv_bfloat16 *__restrict__ out, int *__restrict__ exps)
{
    __shared__ double th[32][33], tl[32][33];
    __shared__ int sexp[32];
    const int r0 = blockIdx.x * 32, kbeg = blockIdx.y * DIGIT_KT;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    if (threadIdx.x < 32) {
        const int r = r0 + threadIdx.x;
        const int e = (r < R) ? split_exponent(vmax[r]) : 0;
        sexp[threadIdx.x] = e;
        if (blockIdx.y == 0) exps[r] = e;
    }
    const int F = 7 + 8 * (s - 1);
    const size_t pstride = (size_t)Pmax * Kmax;
    for (int k0 = kbeg; k0 < kbeg + DIGIT_KT && k0 < Kp; k0 += 32) {
        __syncthreads();
        split_load_tile<double, LAYOUT>(th, Xh, ld, R, K, INT_MAX, r0, k0);
        split_load_tile<double, LAYOUT>(tl, Xl, ld, R, K, INT_MAX, r0, k0);
        __syncthreads();
#pragma unroll 1
        for (int w = 0; w < 4; ++w) {
            const int v = ty + 8 * w;
            const int r = r0 + v;
            const int kk = k0 + tx;
            const int e = sexp[v];
            __int128 Xi = 0;
            if (e != kOzakiExpNonfinite && r < R) Xi = dd_fixed_part(th[v][tx], F, e) + dd_fixed_part(tl[v][tx], F, e);
            write_digits128(Xi, s, out + (size_t)r * Kmax + (size_t)kk, pstride);
        }
    }
}

// ---- residue form: X(r, kk) -> N bf16 residue matrices [l][r][kk] -----------------
// Each entry becomes X = round(x 2^(t - e)) (|X| <= 2^t; e the vector's scale
// exponent as for the digits) and is written as its symmetric residues modulo
// the table's moduli, in [-128, 128]. |X| is cut into 16-bit pieces u_k, and
// X mod m = (sum_k u_k (2^(16 k) mod m)) mod m with a sum below 2^27, reduced
// by one multiply with ceil(2^40 / m) (exact for sums below 2^31).
struct CrtSplitSm {
    int m[kCrtMaxModuli];
    unsigned long long inv40[kCrtMaxModuli];
    unsigned off28[kCrtMaxModuli];
    unsigned pw16[12][kCrtMaxModuli];
};

__device__ __forceinline__ void crt_split_table(CrtSplitSm &sm, const CrtTable *__restrict__ tab, int N, int pieces)
{
    for (int x = threadIdx.x; x < N; x += blockDim.x) {
        sm.m[x] = tab->m[x];
        sm.inv40[x] = tab->inv40[x];
        sm.off28[x] = tab->off28[x];
        for (int k = 0; k < pieces; ++k) sm.pw16[k][x] = tab->pw16[k][x];
    }
}

// the residues of the integer with sign neg and 16-bit pieces u[0..P) into
// planes o[l * pstride]
template <int P>
__device__ __forceinline__ void write_residues(const uint32_t (&u)[P], bool neg, const CrtSplitSm &sm, int N,
                                               __nv_bfloat16 *__restrict__ o, size_t pstride)
{
#pragma unroll 4
    for (int l = 0; l < N; ++l) {
        const uint32_t m = (uint32_t)sm.m[l];
        uint32_t v = u[0];
#pragma unroll
        for (int k = 1; k < P; ++k) v += u[k] * sm.pw16[k][l];
        const uint32_t q = (uint32_t)(((unsigned long long)v * sm.inv40[l]) >> 40);
        int r = (int)(v - q * m);
        if (neg && r) r = (int)m - r;
        if (2 * r > (int)m) r -= (int)m;
        o[(size_t)l * pstride] = __int2bfloat16_rn(r);
    }
}

template <typename Tin, int LAYOUT>
__global__ void __launch_bounds__(256, 4)
ozaki_residues_kernel(int R, int K, int Kh, int Kp, const Tin *__restrict__ X, int ld, int t, int N, int Pmax,
                      int Kmax, const unsigned long long *__restrict__ vmax, __nv_bfloat16 *__restrict__ out,
                      int *__restrict__ exps, const CrtTable *__restrict__ tab)
{
    __shared__ double tile[32][33];
    __shared__ int sexp[32];
    __shared__ CrtSplitSm sm;
    const int r0 = blockIdx.x * 32, kbeg = blockIdx.y * DIGIT_KT;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    if (threadIdx.x < 32) {
        const int r = r0 + threadIdx.x;
        const int e = (r < R) ? split_exponent(vmax[r]) : 0;
        sexp[threadIdx.x] = e;
        if (blockIdx.y == 0) exps[r] = e;
    }
    crt_split_table(sm, tab, N, 4);
    const size_t pstride = (size_t)Pmax * Kmax;
    for (int k0 = kbeg; k0 < kbeg + DIGIT_KT && k0 < Kp; k0 += 32) {
        __syncthreads();
        split_load_tile<Tin, LAYOUT>(tile, X, ld, R, K, Kh, r0, k0);
        __syncthreads();
#pragma unroll 1
        for (int w = 0; w < 4; ++w) {
            const int v = ty + 8 * w;
            const int r = r0 + v;
            const int kk = k0 + tx;
            const double x = tile[v][tx];   // zero outside the matrix
            const int e = sexp[v];
            unsigned long long mag = 0;
            bool neg = false;
            if (e != kOzakiExpNonfinite && r < R) {
                const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
                const int eb = (int)((bits >> 52) & 0x7ff);
                unsigned long long mant = bits & 0xfffffffffffffull;
                int ex;
                if (eb == 0) ex = -1074; else { mant |= 1ull << 52; ex = eb - 1075; }
                const int sh = ex + t - e;                // x 2^(t-e) = mant 2^sh, sh < t - 52
                if (mant == 0) mag = 0;
                else if (sh >= 0) mag = mant << sh;
                else if (-sh >= 64) mag = 0;
                else mag = (mant + (1ull << (-sh - 1))) >> (-sh);
                neg = (bits >> 63) != 0;
            }
            const uint32_t u[4] = {(uint32_t)(mag & 0xffff), (uint32_t)((mag >> 16) & 0xffff),
                                   (uint32_t)((mag >> 32) & 0xffff), (uint32_t)(mag >> 48)};
            write_residues<4>(u, neg, sm, N, out + (size_t)r * Kmax + (size_t)kk, pstride);
        }
    }
}

template <int LAYOUT>
__global__ void __launch_bounds__(256, 2)
ozaki_residues_dd_kernel(int R, int K, int Kp, const double *__restrict__ Xh, const double *__restrict__ Xl, int ld,
                         int t, int N, int Pmax, int Kmax, const unsigned long long *__restrict__ vmax,
                         __nv_bfloat16 *__restrict__ out, int *__restrict__ exps, const CrtTable *__restrict__ tab)
{
    __shared__ double th[32][33], tl[32][33];
    __shared__ int sexp[32];
    __shared__ CrtSplitSm sm;
    const int r0 = blockIdx.x * 32, kbeg = blockIdx.y * DIGIT_KT;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    if (threadIdx.x < 32) {
        const int r = r0 + threadIdx.x;
        const int e = (r < R) ? split_exponent(vmax[r]) : 0;
        sexp[threadIdx.x] = e;
        if (blockIdx.y == 0) exps[r] = e;
    }
    crt_split_table(sm, tab, N, 8);
    const size_t pstride = (size_t)Pmax * Kmax;
    for (int k0 = kbeg; k0 < kbeg + DIGIT_KT && k0 < Kp; k0 += 32) {
        __syncthreads();
        split_load_tile<double, LAYOUT>(th, Xh, ld, R, K, INT_MAX, r0, k0);
        split_load_tile<double, LAYOUT>(tl, Xl, ld, R, K, INT_MAX, r0, k0);
        __syncthreads();
#pragma unroll 1
        for (int w = 0; w < 4; ++w) {
            const int v = ty + 8 * w;
            const int r = r0 + v;
            const int kk = k0 + tx;
            const int e = sexp[v];
            __int128 Xi = 0;
            if (e != kOzakiExpNonfinite && r < R) Xi = dd_fixed_part(th[v][tx], t, e) + dd_fixed_part(tl[v][tx], t, e);
            const bool neg = Xi < 0;
            const unsigned __int128 mag = neg ? (unsigned __int128)(-Xi) : (unsigned __int128)Xi;
            uint32_t u[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) u[k] = (uint32_t)(mag >> (16 * k)) & 0xffffu;
            write_residues<8>(u, neg, sm, N, out + (size_t)r * Kmax + (size_t)kk, pstride);
        }
    }
}

// The same with the modulus count fixed at compile time (16 for FP64 operands,
// 32 for double-double ones): the modulus loop unrolls and every constant of a
// modulus is an immediate. The integer X is cut into 16-bit pieces with a
// signed top piece (two's complement), X = sum_k u_k 2^(16 k), so that
// v = off + sum_k u_k (2^(16 k) mod m) is a non-negative integer below 2^28
// with v = X + floor(m/2) (mod m) for either sign of X (off: floor(m/2) plus
// a multiple of m above the most negative top term). Then
// s = v - floor(v / m) m - floor(m/2) is the symmetric residue of X, in
// [-floor(m/2), m - 1 - floor(m/2)], and its bf16 bits come from the FP32
// value 1.5 2^23 + s (exact) less 1.5 2^23: the top half of the float's bits,
// since |s| <= 128 has at most 8 significant bits. Each thread turns 4
// consecutive entries of one vector into residues and stores the 4 bf16
// values of a modulus at once.
constexpr int RES_KT = 256;   // K per block of the fixed-count residue kernel

template <int P>
__device__ __forceinline__ float crt_res_float(const int32_t (&u)[P], int l)
{
    const int m = crt_mod(l);
    int32_t v = (int32_t)crt_off27(l) + m / 2 + u[0];
#pragma unroll
    for (int k = 1; k < P; ++k) v += u[k] * (int32_t)crt_pw16(k, l);    // in [0, 2^28)
    const uint32_t q = __umulhi((uint32_t)v, crt_inv38(l)) >> 6;
    const int32_t bits = v + (0x4B400000 - m / 2) - (int32_t)q * m;      // 0x4B400000 + s
    return __fsub_rn(__int_as_float(bits), 12582912.0f);                // s, exactly
}

// the bf16 bits of two exact small floats, packed (a low, b high)
__device__ __forceinline__ uint32_t crt_pack_bf16(float a, float b)
{
    return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}

// x 2^(t - e) rounded to the nearest integer (|x| < 2^e), as signed 16-bit
// pieces: P = 4 for t <= 62 (64-bit integer), P = 8 for double-double input
template <int P>
__device__ __forceinline__ void crt_pieces(double xh, double xl, int t, int e, int32_t (&u)[P])
{
    if constexpr (P == 4) {
        const unsigned long long bits = (unsigned long long)__double_as_longlong(xh);
        const int eb = (int)((bits >> 52) & 0x7ff);
        unsigned long long mant = bits & 0xfffffffffffffull;
        int ex;
        if (eb == 0) ex = -1074; else { mant |= 1ull << 52; ex = eb - 1075; }
        const int sh = ex + t - e;                // x 2^(t-e) = mant 2^sh, sh < t - 52 <= 10
        unsigned long long mag;
        if (mant == 0) mag = 0;
        else if (sh >= 0) mag = mant << sh;
        else if (-sh >= 64) mag = 0;
        else mag = (mant + (1ull << (-sh - 1))) >> (-sh);
        const long long X = (bits >> 63) ? -(long long)mag : (long long)mag;
        u[0] = (int32_t)(X & 0xffff);
        u[1] = (int32_t)((X >> 16) & 0xffff);
        u[2] = (int32_t)((X >> 32) & 0xffff);
        u[3] = (int32_t)(X >> 48);                 // signed top piece
    } else {
        const __int128 X = dd_fixed_part(xh, t, e) + dd_fixed_part(xl, t, e);
#pragma unroll
        for (int k = 0; k < P - 1; ++k) u[k] = (int32_t)((unsigned long long)(X >> (16 * k)) & 0xffffull);
        u[P - 1] = (int32_t)(long long)(X >> (16 * (P - 1)));   // signed top piece
    }
}

// block (bx, by): vectors 32 bx .., K stretch [KT by, KT (by + 1))
template <typename Tin, int LAYOUT, int NM, bool DD, int KT>
__device__ __forceinline__ void residues_fast_body(int bx, int by, int R, int K, int Kh, int Kp,
                                                   const Tin *__restrict__ X, const double *__restrict__ Xl, int ld,
                                                   int t, int Pmax, int Kmax,
                                                   const unsigned long long *__restrict__ vmax,
                                                   __nv_bfloat16 *__restrict__ out, int *__restrict__ exps)
{
    constexpr int P = DD ? 8 : 4;
    __shared__ double th[32][33];
    __shared__ double tl[DD ? 32 : 1][33];
    __shared__ int sexp[32];
    const int r0 = bx * 32, kbeg = by * KT;
    if (threadIdx.x < 32) {
        const int r = r0 + threadIdx.x;
        const int e = (r < R) ? split_exponent(vmax[r]) : 0;
        sexp[threadIdx.x] = e;
        if (by == 0) exps[r] = e;
    }
    const int v = threadIdx.x >> 3, g = threadIdx.x & 7;
    const size_t pstride = (size_t)Pmax * Kmax;
    for (int k0 = kbeg; k0 < kbeg + KT && k0 < Kp; k0 += 32) {
        __syncthreads();
        split_load_tile<Tin, LAYOUT>(th, X, ld, R, K, Kh, r0, k0);
        if constexpr (DD) split_load_tile<double, LAYOUT>(tl, Xl, ld, R, K, INT_MAX, r0, k0);
        __syncthreads();
        const int r = r0 + v, kk = k0 + 4 * g;
        const int e = sexp[v];
        const bool live = e != kOzakiExpNonfinite && r < R;
        int32_t u[4][P];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            if (live) {
                crt_pieces<P>(th[v][4 * g + x], DD ? tl[v][4 * g + x] : 0.0, t, e, u[x]);
            } else {
#pragma unroll
                for (int k = 0; k < P; ++k) u[x][k] = 0;
            }
        }
        __nv_bfloat16 *o = out + (size_t)r * Kmax + (size_t)kk;
#pragma unroll
        for (int l = 0; l < NM; ++l) {
            const uint32_t w01 = crt_pack_bf16(crt_res_float<P>(u[0], l), crt_res_float<P>(u[1], l));
            const uint32_t w23 = crt_pack_bf16(crt_res_float<P>(u[2], l), crt_res_float<P>(u[3], l));
            *reinterpret_cast<uint2 *>(o + (size_t)l * pstride) = make_uint2(w01, w23);
        }
    }
}

template <typename Tin, int LAYOUT, int NM, bool DD>
__global__ void __launch_bounds__(256)
ozaki_residues_fast_kernel(int R, int K, int Kh, int Kp, const Tin *__restrict__ X, const double *__restrict__ Xl,
                           int ld, int t, int Pmax, int Kmax, const unsigned long long *__restrict__ vmax,
                           __nv_bfloat16 *__restrict__ out, int *__restrict__ exps)
{
    residues_fast_body<Tin, LAYOUT, NM, DD, RES_KT>(blockIdx.x, blockIdx.y, R, K, Kh, Kp, X, Xl, ld, t, Pmax, Kmax,
                                                    vmax, out, exps);
}

// Grouped residue split (FP64 vectors, the 16 moduli of FP64 products): the
// flat grid of the grouped digit split (blocks of 32 vectors x 64 of K), each
// matrix with its own fixed-point bits t.
template <int LAYOUT>
__global__ void __launch_bounds__(256)
ozaki_residues_group_kernel(const SplitMat *__restrict__ mats, const int *__restrict__ start, int m, int Pmax,
                            int Kmax, const unsigned long long *__restrict__ vmax, __nv_bfloat16 *__restrict__ out,
                            int *__restrict__ exps)
{
    const int a = group_find(start, m, blockIdx.x);
    const SplitMat g = mats[a];
    const int Kp = (g.K + 63) / 64 * 64;   // work items stop at the order rounded to 64
    const int local = blockIdx.x - start[a], gx = (g.R + 31) / 32;
    residues_fast_body<double, LAYOUT, kCrtDefaultModuli, false, DIGIT_KT>(
        local % gx, local / gx, g.R, g.K, INT_MAX, Kp, g.X, nullptr, g.ld, g.t, Pmax, Kmax, vmax + g.row0,
        out + (size_t)g.row0 * Kmax, exps + g.row0);
}

// Triple-double operands: x0 + x1 + x2 times 2^(t - e), each word rounded to the
// nearest unit, summed exactly in a 192-bit two's complement integer
// (|x| < 2^e, so the sum stays below 2^(t+1) < 2^175).
__device__ __forceinline__ void td_fixed_add(double x, int t, int e, u64 (&X)[3])
{
    const u64 bits = (u64)__double_as_longlong(x);
    const int eb = (int)((bits >> 52) & 0x7ff);
    u64 mant = bits & 0xfffffffffffffull;
    int ex;
    if (eb == 0) ex = -1074; else { mant |= 1ull << 52; ex = eb - 1075; }
    if (mant == 0) return;
    const int sh = ex + t - e;                     // x 2^(t-e) = mant 2^sh, sh <= t - 52 <= 122
    u64 v[3] = {0, 0, 0};
    if (sh >= 0) {
        const int q = sh >> 6, r = sh & 63;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (k == q) v[k] = mant << r;
            if (k == q + 1 && r) v[k] = mant >> (64 - r);
        }
    } else if (-sh < 64) {
        v[0] = (mant + (1ull << (-sh - 1))) >> (-sh);
    }
    if (bits >> 63) {
        u64 c = 1;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const u64 nv = ~v[k] + c;
            c = (c && nv == 0) ? 1ull : 0ull;
            v[k] = nv;
        }
    }
    u64 c = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const u64 s1 = X[k] + v[k];
        const u64 c1 = s1 < X[k] ? 1ull : 0ull;
        const u64 s2 = s1 + c;
        const u64 c2 = s2 < s1 ? 1ull : 0ull;
        X[k] = s2;
        c = c1 | c2;
    }
}

// The residues of triple-double operands modulo the NM moduli. The fixed-point
// integer is cut into 11 pieces of 16 bits, the top one signed (bits 160-175;
// t <= 174 keeps the integer inside them); for modulus m,
// v = off + sum_k u_k (2^(16 k) mod m) lies in [0, 2^31) (off = m ceil(2^28 / m)
// lifts the most negative top term; the positive pieces add below 1.8e8), and
// v - floor(v / m) m, with the quotient from ceil(2^40 / m), is the residue,
// taken in the symmetric range. The moduli, their reciprocals and the powers
// come from the table, staged in shared memory (read as broadcasts). Each
// thread turns 4 consecutive entries of one vector into residues and stores
// the 4 bf16 values of a modulus at once (the layout of
// ozaki_residues_fast_kernel).
template <int LAYOUT>
__global__ void __launch_bounds__(256)
ozaki_residues_td_kernel(int R, int K, int Kp, const double *__restrict__ X0, const double *__restrict__ X1,
                         const double *__restrict__ X2, int ld, int t, int N, int Pmax, int Kmax,
                         const unsigned long long *__restrict__ vmax, __nv_bfloat16 *__restrict__ out,
                         int *__restrict__ exps, const CrtTable *__restrict__ tab)
{
    constexpr int P = 11;
    __shared__ double tw[3][32][33];
    __shared__ int sexp[32];
    __shared__ CrtSplitSm sm;
    const int r0 = blockIdx.x * 32, kbeg = blockIdx.y * RES_KT;
    if (threadIdx.x < 32) {
        const int r = r0 + threadIdx.x;
        const int e = (r < R) ? split_exponent(vmax[r]) : 0;
        sexp[threadIdx.x] = e;
        if (blockIdx.y == 0) exps[r] = e;
    }
    crt_split_table(sm, tab, N, P);
    const int v = threadIdx.x >> 3, g = threadIdx.x & 7;
    const size_t pstride = (size_t)Pmax * Kmax;
    for (int k0 = kbeg; k0 < kbeg + RES_KT && k0 < Kp; k0 += 32) {
        __syncthreads();
        split_load_tile<double, LAYOUT>(tw[0], X0, ld, R, K, INT_MAX, r0, k0);
        split_load_tile<double, LAYOUT>(tw[1], X1, ld, R, K, INT_MAX, r0, k0);
        split_load_tile<double, LAYOUT>(tw[2], X2, ld, R, K, INT_MAX, r0, k0);
        __syncthreads();
        const int r = r0 + v, kk = k0 + 4 * g;
        const int e = sexp[v];
        const bool live = e != kOzakiExpNonfinite && r < R;
        int32_t u[4][P];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            u64 X[3] = {0, 0, 0};
            if (live) {
#pragma unroll
                for (int wd = 0; wd < 3; ++wd) td_fixed_add(tw[wd][v][4 * g + x], t, e, X);
            }
#pragma unroll
            for (int k = 0; k < P - 1; ++k) {
                const int b = 16 * k;
                u[x][k] = (int32_t)((X[b >> 6] >> (b & 63)) & 0xffffull);
            }
            u[x][P - 1] = (int32_t)(int16_t)((X[2] >> 32) & 0xffffull);   // bits 160-175, signed
        }
        __nv_bfloat16 *o = out + (size_t)r * Kmax + (size_t)kk;
#pragma unroll 2
        for (int l = 0; l < N; ++l) {
            const int m = sm.m[l];
            const unsigned long long inv = sm.inv40[l];
            int32_t pw[P];
#pragma unroll
            for (int k = 0; k < P; ++k) pw[k] = (int32_t)sm.pw16[k][l];
            float f[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                int32_t s = (int32_t)sm.off28[l];
#pragma unroll
                for (int k = 0; k < P; ++k) s += u[x][k] * pw[k];
                const uint32_t q = (uint32_t)(((unsigned long long)(uint32_t)s * inv) >> 40);
                int32_t rr = s - (int32_t)q * m;
                if (2 * rr > m) rr -= m;
                f[x] = (float)rr;
            }
            *reinterpret_cast<uint2 *>(o + (size_t)l * pstride) =
                make_uint2(crt_pack_bf16(f[0], f[1]), crt_pack_bf16(f[2], f[3]));
        }
    }
}

// Six-double operands: x0 + ... + x5 times 2^(T - e), T = 2t - 2, each word
// rounded to the nearest unit, summed exactly in a 384-bit two's complement
// integer (|x| < 2^e: the sum stays below 2^(T+1) = 2^(2t-1)).
__device__ __forceinline__ void d6_fixed_add(double x, int T, int e, u64 (&X)[6])
{
    const u64 bits = (u64)__double_as_longlong(x);
    const int eb = (int)((bits >> 52) & 0x7ff);
    u64 mant = bits & 0xfffffffffffffull;
    int ex;
    if (eb == 0) ex = -1074; else { mant |= 1ull << 52; ex = eb - 1075; }
    if (mant == 0) return;
    const int sh = ex + T - e;                     // x 2^(T-e) = mant 2^sh, sh <= T - 52 <= 270
    u64 v[6] = {0, 0, 0, 0, 0, 0};
    if (sh >= 0) {
        const int q = sh >> 6, r = sh & 63;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            if (k == q) v[k] = mant << r;
            if (k == q + 1 && r) v[k] = mant >> (64 - r);
        }
    } else if (-sh < 64) {
        v[0] = (mant + (1ull << (-sh - 1))) >> (-sh);
    }
    if (bits >> 63) mw_neg<6>(v);
    mw_add<6>(X, v);
}

// The residues of six-double operands: the fixed-point integer X of T = 2t - 2
// bits is cut into X = X_hi 2^t + X_lo (0 <= X_lo < 2^t, |X_hi| < 2^(t-1)), and
// each half is reduced modulo the N moduli as in ozaki_residues_td_kernel (11
// pieces of 16 bits, the top one signed), into the slots' planes out_hi and
// out_lo. The six planes are read one after another through one shared tile.
template <int LAYOUT>
__global__ void __launch_bounds__(256)
ozaki_residues_d6_kernel(int R, int K, int Kp, const double *__restrict__ X, size_t pl, int ld, int t, int N,
                         int Pmax, int Kmax, const unsigned long long *__restrict__ vmax,
                         __nv_bfloat16 *__restrict__ out_hi, __nv_bfloat16 *__restrict__ out_lo,
                         int *__restrict__ exps_hi, int *__restrict__ exps_lo, const CrtTable *__restrict__ tab)
{
    constexpr int P = 11;
    __shared__ double tw[32][33];
    __shared__ int sexp[32];
    __shared__ CrtSplitSm sm;
    const int r0 = blockIdx.x * 32, kbeg = blockIdx.y * RES_KT;
    if (threadIdx.x < 32) {
        const int r = r0 + threadIdx.x;
        const int e = (r < R) ? split_exponent(vmax[r]) : 0;
        sexp[threadIdx.x] = e;
        if (blockIdx.y == 0) {
            exps_hi[r] = e;
            exps_lo[r] = e;
        }
    }
    crt_split_table(sm, tab, N, P);
    const int T = 2 * t - 2;
    const int v = threadIdx.x >> 3, g = threadIdx.x & 7;
    const size_t pstride = (size_t)Pmax * Kmax;
    for (int k0 = kbeg; k0 < kbeg + RES_KT && k0 < Kp; k0 += 32) {
        const int r = r0 + v, kk = k0 + 4 * g;
        u64 Xf[4][6];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int k = 0; k < 6; ++k) Xf[x][k] = 0;
#pragma unroll 1
        for (int wd = 0; wd < 6; ++wd) {
            __syncthreads();
            split_load_tile<double, LAYOUT>(tw, X + (size_t)wd * pl, ld, R, K, INT_MAX, r0, k0);
            __syncthreads();
            const int e = sexp[v];
            if (e != kOzakiExpNonfinite && r < R) {
#pragma unroll
                for (int x = 0; x < 4; ++x) d6_fixed_add(tw[v][4 * g + x], T, e, Xf[x]);
            }
        }
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            int32_t u[4][P];
#pragma unroll
            for (int x = 0; x < 4; ++x) {
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    if (half == 0) {
                        // X_hi = X >> t (arithmetic): piece k is bits t + 16k .. t + 16k + 15
                        const u64 b = mw_bits64<6>(Xf[x], t + 16 * k) & 0xffffull;
                        u[x][k] = k == P - 1 ? (int32_t)(int16_t)b : (int32_t)b;
                    } else {
                        // X_lo = X mod 2^t: piece k is bits 16k .. 16k + 15 below bit t
                        u64 b = mw_bits64<6>(Xf[x], 16 * k) & 0xffffull;
                        const int keep = t - 16 * k;
                        if (keep <= 0) b = 0;
                        else if (keep < 16) b &= (1ull << keep) - 1ull;
                        u[x][k] = (int32_t)b;
                    }
                }
            }
            __nv_bfloat16 *o = (half == 0 ? out_hi : out_lo) + (size_t)r * Kmax + (size_t)kk;
#pragma unroll 2
            for (int l = 0; l < N; ++l) {
                const int m = sm.m[l];
                const unsigned long long inv = sm.inv40[l];
                int32_t pw[P];
#pragma unroll
                for (int k = 0; k < P; ++k) pw[k] = (int32_t)sm.pw16[k][l];
                float f[4];
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    int32_t s = (int32_t)sm.off28[l];
#pragma unroll
                    for (int k = 0; k < P; ++k) s += u[x][k] * pw[k];
                    const uint32_t q = (uint32_t)(((unsigned long long)(uint32_t)s * inv) >> 40);
                    int32_t rr = s - (int32_t)q * m;
                    if (2 * rr > m) rr -= m;
                    f[x] = (float)rr;
                }
                *reinterpret_cast<uint2 *>(o + (size_t)l * pstride) =
                    make_uint2(crt_pack_bf16(f[0], f[1]), crt_pack_bf16(f[2], f[3]));
            }
        }
    }
}

// Splits levels 0..s-1 (level l costs l + 1 digit pairs) into G contiguous
// non-empty groups minimising the largest group cost (linear partition by
// dynamic programming); returns that cost.
int split_levels(int s, int G, int *lvl)
{
    constexpr int S = kOzakiMaxSlicesDD + 1;
    int best[S][S], cut[S][S];   // best[g][l]: levels 0..l-1 in g groups
    auto cost = [](int a, int b) { return (b * (b + 1) - a * (a + 1)) / 2; };   // levels a..b-1
    for (int l = 0; l <= s; ++l) best[1][l] = cost(0, l), cut[1][l] = 0;
    for (int g = 2; g <= G; ++g)
        for (int l = g; l <= s; ++l) {
            best[g][l] = -1;
            for (int k = g - 1; k < l; ++k) {
                const int v = std::max(best[g - 1][k], cost(k, l));
                if (best[g][l] < 0 || v < best[g][l]) { best[g][l] = v; cut[g][l] = k; }
            }
        }
    lvl[G] = s;
    for (int g = G, l = s; g >= 1; --g) {
        l = cut[g][l];
        lvl[g - 1] = l;
    }
    lvl[0] = 0;
    return best[G][s];
}

// Residue products: N levels of one product each into G contiguous groups
// whose sizes differ by at most one (larger groups first); returns the largest.
int split_levels_uniform(int N, int G, int *lvl)
{
    lvl[0] = 0;
    for (int g = 0; g < G; ++g) lvl[g + 1] = lvl[g] + N / G + (g < N % G ? 1 : 0);
    return (N + G - 1) / G;
}

int level_groups_uniform(int N, int active, int sms, int *lvl)
{
    int best_g = 1;
    long long best = -1;
    int tmp[kCrtMaxModuli + 1];
    for (int G = 1; G <= std::min(N, 8); ++G) {
        const int worst = split_levels_uniform(N, G, tmp);
        const long long waves = ((long long)active * G + sms - 1) / sms;
        const long long est = waves * worst;
        if (best < 0 || est < best) { best = est; best_g = G; }
    }
    split_levels_uniform(N, best_g, lvl);
    return best_g;
}

// Work items per tile: the number of level groups G that minimises the
// persistent grid's makespan, waves(active * G) * largest group cost; the
// grid then has fewer idle SMs in its last wave (the groups write disjoint
// level planes, so no reduction is needed).
int level_groups(int s, int active, int sms, int *lvl)
{
    int best_g = 1;
    long long best = -1;
    int tmp[kOzakiMaxSlicesDD + 1];
    for (int G = 1; G <= std::min(s, 8); ++G) {
        const int worst = split_levels(s, G, tmp);
        const long long waves = ((long long)active * G + sms - 1) / sms;
        const long long est = waves * worst;
        if (best < 0 || est < best) { best = est; best_g = G; }
    }
    split_levels(s, best_g, lvl);
    return best_g;
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cudaError_t set_mma_smem()
{
    cudaError_t e = cudaFuncSetAttribute(ozaki_mma_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ozaki_mma_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    return e;
}

cudaError_t encode_digits_map(void *map, void *base, int rows, int Kmax, int box_rows)
{
    if (!g_encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)Kmax, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)Kmax * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode((CUtensorMap *)map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

namespace {

// little-endian 32-bit limbs, enough for M < 2^384 and its products by 2^64
struct Big {
    static constexpr int kW = kCrtMaxLimbs + 2;   // room for M y_l before the shift
    uint32_t v[kW] = {};
    void mul_small(uint32_t m)
    {
        unsigned long long c = 0;
        for (auto &x : v) { const unsigned long long t = (unsigned long long)x * m + c; x = (uint32_t)t; c = t >> 32; }
    }
    uint32_t div_small(uint32_t m)   // *this /= m, returns the remainder
    {
        unsigned long long r = 0;
        for (int k = kW - 1; k >= 0; --k) {
            const unsigned long long t = (r << 32) | v[k];
            v[k] = (uint32_t)(t / m);
            r = t % m;
        }
        return (uint32_t)r;
    }
    uint32_t mod_small(uint32_t m) const { Big c = *this; return c.div_small(m); }
    int bits() const
    {
        for (int k = kW - 1; k >= 0; --k)
            if (v[k]) return 32 * k + 32 - __builtin_clz(v[k]);
        return 0;
    }
    void shl(int s)
    {
        const int w = s / 32, b = s % 32;
        for (int k = kW - 1; k >= 0; --k) {
            const uint32_t hi = k - w >= 0 ? v[k - w] : 0, lo = k - w - 1 >= 0 ? v[k - w - 1] : 0;
            v[k] = b ? (hi << b) | (lo >> (32 - b)) : hi;
        }
    }
    double to_double() const
    {
        double d = 0.0;
        for (int k = kW - 1; k >= 0; --k) d = d * 4294967296.0 + (double)v[k];
        return d;
    }
};

}  // namespace

bool crt_build_table(int N, int L, CrtTable &t)
{
    if (N < 1 || N > kCrtMaxModuli || (L != 4 && L != 8 && L != 12)) return false;
    t = CrtTable{};
    t.N = N;
    // the largest integers <= 256 that are coprime to every one taken before
    // (the list crt_mod holds as literals for the device code)
    int cnt = 0;
    for (int m = 256; m >= 2 && cnt < N; --m) {
        bool ok = true;
        for (int k = 0; k < cnt && ok; ++k) ok = std::gcd(m, t.m[k]) == 1;
        if (ok) t.m[cnt++] = m;
    }
    for (int l = 0; l < N; ++l)
        if (t.m[l] != crt_mod(l)) return false;
    Big M;
    M.v[0] = 1;
    for (int l = 0; l < N; ++l) M.mul_small((uint32_t)t.m[l]);
    const int bits = M.bits();
    if (bits > 32 * L) return false;
    t.log2M = std::log2(M.to_double());
    t.L = L;
    // the weights and M are scaled by 2^sigma so that M' = M 2^sigma has its top
    // bit at 32 L - 1; rebuilt values are then exact multiples of 2^sigma
    const int sigma = 32 * t.L - bits;
    for (int l = 0; l < N; ++l) {
        const uint32_t m = (uint32_t)t.m[l];
        Big Ml = M;
        Ml.div_small(m);                        // M_l = M / m_l (exact)
        const uint32_t a = Ml.mod_small(m);     // M_l mod m_l, invertible
        uint32_t y = 1;
        while ((a * y) % m != 1) ++y;
        Ml.mul_small(y);                        // w_l = M_l y_l < M
        Ml.shl(sigma);
        for (int k = 0; k < t.L; ++k) t.w[l][k] = Ml.v[k];
        t.inv40[l] = ((1ull << 40) + m - 1) / m;
        t.off28[l] = m * (((1u << 28) + m - 1) / m);
        unsigned long long pw = 1;
        for (int k = 0; k < 12; ++k) {
            t.pw16[k][l] = (unsigned)(pw % m);
            pw = (pw % m) * 65536ull;
        }
    }
    Big Ms = M;
    Ms.shl(sigma);
    for (int k = 0; k < t.L; ++k) t.M[k] = Ms.v[k];
    Big H = Ms;
    H.div_small(2);
    for (int k = 0; k < t.L; ++k) t.halfM[k] = H.v[k];
    t.invMtop = (float)(1.0 / ((double)t.M[t.L - 1] + (double)t.M[t.L - 2] / 4294967296.0));
    t.sigma = sigma;
    return true;
}

int crt_bits(const CrtTable &t, long long K)
{
    if (K < 1) K = 1;
    return (int)std::floor((t.log2M - 1.0 - std::log2((double)K)) / 2.0 - 1e-9);
}

cudaError_t ozaki_alloc(OzakiWork &w, int nmax, const int *caps, bool cplx, int crt_moduli, unsigned crt_mask,
                        int crt_limbs, int crt_sets)
{
    static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
    w.nmax = nmax;
    w.cplx = cplx;
    w.Pmax = (nmax + kOzakiTileI - 1) / kOzakiTileI * kOzakiTileI;
    w.Kmax = (nmax + kOzakiKChunk - 1) / kOzakiKChunk * kOzakiKChunk * (cplx ? 2 : 1);
    w.levels = kOzakiMaxSlices;
    for (int i = 0; i < kOzakiSlots; ++i)
        if (!(crt_mask >> i & 1u)) w.levels = std::max(w.levels, caps[i]);
    cudaError_t e = cudaSuccess;
    if (crt_moduli > 0) {
        if (!crt_build_table(crt_moduli, crt_limbs, w.crt)) return cudaErrorInvalidValue;
        // byte planes of the residues share the int32 level planes' buffer
        w.levels = std::max(w.levels, crt_sets * ((crt_moduli + 3) / 4));
        e = cudaMalloc((void **)&w.crt_dev, sizeof(CrtTable));
        if (e == cudaSuccess) e = cudaMemcpy(w.crt_dev, &w.crt, sizeof(CrtTable), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
    }
    e = cudaMalloc((void **)&w.planes, (size_t)w.levels * (cplx ? 2 : 1) * w.Pmax * w.Pmax * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&w.vmax, (size_t)w.Pmax * sizeof(unsigned long long));
    for (int i = 0; i < kOzakiSlots && e == cudaSuccess; ++i) {
        OzakiSlot &sl = w.slot[i];
        sl.cap = caps[i];
        sl.crt = (crt_mask >> i & 1u) && crt_moduli > 0 ? 1 : 0;
        if (sl.crt) sl.cap = crt_moduli;
        if (sl.cap <= 0) continue;
        const size_t bytes = (size_t)sl.cap * w.Pmax * w.Kmax * 2;
        e = cudaMalloc(&sl.dig, bytes);
        if (e == cudaSuccess) e = cudaMalloc((void **)&sl.exps, (size_t)w.Pmax * sizeof(int));
        // digits outside the rows and K a split writes must read as zero
        if (e == cudaSuccess) e = cudaMemset(sl.dig, 0, bytes);
        if (e == cudaSuccess) e = encode_digits_map(sl.map_j, sl.dig, sl.cap * w.Pmax, w.Kmax, BM);
        if (e == cudaSuccess) e = encode_digits_map(sl.map_i, sl.dig, sl.cap * w.Pmax, w.Kmax, BN);
    }
    if (e == cudaSuccess)
        e = set_mma_smem();
    return e;
}

void ozaki_free(OzakiWork &w)
{
    for (auto &e : w.tev)
        if (e) { cudaEventDestroy(e); e = nullptr; }
    w.tuned.clear();
    cudaFree(w.planes);
    cudaFree(w.vmax);
    cudaFree(w.crt_dev);
    w.planes = nullptr;
    w.vmax = nullptr;
    w.crt_dev = nullptr;
    for (int i = 0; i < kOzakiSlots; ++i) {
        cudaFree(w.slot[i].dig);
        cudaFree(w.slot[i].exps);
        w.slot[i].dig = nullptr;
        w.slot[i].exps = nullptr;
        w.slot[i].cap = 0;
        w.slot[i].crt = 0;
    }
}

sr_status ozaki_split(schur_refine_ctx *h, cudaStream_t st, OzakiWork &w, int slot, int R, int K, const void *X,
                      int ld, int layout, int s)
{
    if (slot < 0 || slot >= kOzakiSlots || s < 1 || s > w.slot[slot].cap || R > w.Pmax ||
        K > ozaki_k_limit(w.cplx) || K > w.nmax)
        return SR_ERR_INVALID_ARG;
    const int Kc = (K + kOzakiKChunk - 1) / kOzakiKChunk * kOzakiKChunk;
    const int Kh = w.cplx ? Kc : INT_MAX;           // start of the imaginary half (none when real)
    const int Kv = w.cplx ? 2 * Kc : K;             // stacked length read
    const int Kp = w.cplx ? 2 * Kc : Kc;            // stacked length written
    const int Rp = (R + 31) / 32 * 32;
    const int esz = w.cplx ? 16 : 8;
    SrPhase ph(h, SR_PROF_OZ_SPLIT, 0, 2LL * R * K * esz + 2LL * s * Kp * Rp, 2);
    OzakiSlot &sl = w.slot[slot];
    sl.layout = layout;
    __nv_bfloat16 *out = (__nv_bfloat16 *)sl.dig;
    int *ex = sl.exps;
    if (sl.crt) {
        if (s != w.crt.N) return SR_ERR_INVALID_ARG;
        sl.t = crt_bits(w.crt, (long long)K * (w.cplx ? 2 : 1));   // complex: dot products of 2K terms
        if (sl.t < 1 || sl.t > 62) return SR_ERR_UNSUPPORTED;
    }
    SR_CUDA_TRY(cudaMemsetAsync(w.vmax, 0, (size_t)Rp * sizeof(unsigned long long), st));
    const dim3 gmax(Rp / 32, (Kv + SPLIT_KT - 1) / SPLIT_KT);
    const dim3 gdig(Rp / 32, (Kp + DIGIT_KT - 1) / DIGIT_KT);
    const dim3 gres(Rp / 32, (Kp + RES_KT - 1) / RES_KT);
#define SR_SPLIT_LAUNCH(TIN, LAY)                                                                                 \
    ozaki_absmax_kernel<TIN, LAY><<<gmax, 256, 0, st>>>(R, K, Kh, Kv, (const TIN *)X, ld, w.vmax);                \
    if (sl.crt && s == 16)                                                                                        \
        ozaki_residues_fast_kernel<TIN, LAY, 16, false><<<gres, 256, 0, st>>>(                                    \
            R, K, Kh, Kp, (const TIN *)X, nullptr, ld, sl.t, w.Pmax, w.Kmax, w.vmax, out, ex);                    \
    else if (sl.crt)                                                                                              \
        ozaki_residues_kernel<TIN, LAY><<<gdig, 256, 0, st>>>(R, K, Kh, Kp, (const TIN *)X, ld, sl.t, s, w.Pmax,  \
                                                              w.Kmax, w.vmax, out, ex, w.crt_dev);                \
    else                                                                                                          \
        ozaki_digits_kernel<TIN, LAY><<<gdig, 256, 0, st>>>(R, K, Kh, Kp, (const TIN *)X, ld, s, w.Pmax, w.Kmax,  \
                                                            w.vmax, out, ex)
    if (w.cplx) {
        if (layout == OZ_COLS) { SR_SPLIT_LAUNCH(cd, OZ_COLS); } else { SR_SPLIT_LAUNCH(cd, OZ_ROWS); }
    } else {
        if (layout == OZ_COLS) { SR_SPLIT_LAUNCH(double, OZ_COLS); } else { SR_SPLIT_LAUNCH(double, OZ_ROWS); }
    }
#undef SR_SPLIT_LAUNCH
    SR_CUDA_TRY(cudaGetLastError());
    return SR_OK;
}

sr_status ozaki_split_dd(schur_refine_ctx *h, cudaStream_t st, OzakiWork &w, int slot, int R, int K,
                         const double *Xhi, const double *Xlo, int ld, int layout, int s)
{
    OzakiSlot &sl = w.slot[slot];
    if (w.cplx || slot < 0 || slot >= kOzakiSlots || s < 1 || s > sl.cap ||
        s > (sl.crt ? kCrtMaxModuliDD : kOzakiMaxSlicesDD) || R > w.Pmax || K > ozaki_k_limit(false) || K > w.nmax)
        return SR_ERR_INVALID_ARG;
    const int Kp = (K + kOzakiKChunk - 1) / kOzakiKChunk * kOzakiKChunk;
    const int Rp = (R + 31) / 32 * 32;
    SrPhase ph(h, SR_PROF_OZ_SPLIT, 0, 2LL * R * K * 16 + 2LL * s * Kp * Rp, 2);
    sl.layout = layout;
    __nv_bfloat16 *out = (__nv_bfloat16 *)sl.dig;
    int *ex = sl.exps;
    if (sl.crt) {
        if (s != w.crt.N) return SR_ERR_INVALID_ARG;
        sl.t = crt_bits(w.crt, K);
        if (sl.t < 1 || sl.t > 120) return SR_ERR_UNSUPPORTED;
    }
    SR_CUDA_TRY(cudaMemsetAsync(w.vmax, 0, (size_t)Rp * sizeof(unsigned long long), st));
    const dim3 gmax(Rp / 32, (K + SPLIT_KT - 1) / SPLIT_KT);
    const dim3 gdig(Rp / 32, (Kp + DIGIT_KT - 1) / DIGIT_KT);
    const dim3 gres(Rp / 32, (Kp + RES_KT - 1) / RES_KT);
    if (layout == OZ_COLS) {
        ozaki_absmax_kernel<double, OZ_COLS><<<gmax, 256, 0, st>>>(R, K, INT_MAX, K, Xhi, ld, w.vmax);
        if (sl.crt && s == 32)
            ozaki_residues_fast_kernel<double, OZ_COLS, 32, true><<<gres, 256, 0, st>>>(
                R, K, INT_MAX, Kp, Xhi, Xlo, ld, sl.t, w.Pmax, w.Kmax, w.vmax, out, ex);
        else if (sl.crt)
            ozaki_residues_dd_kernel<OZ_COLS><<<gdig, 256, 0, st>>>(R, K, Kp, Xhi, Xlo, ld, sl.t, s, w.Pmax, w.Kmax,
                                                                    w.vmax, out, ex, w.crt_dev);
        else
            ozaki_digits_dd_kernel<OZ_COLS><<<gdig, 256, 0, st>>>(R, K, Kp, Xhi, Xlo, ld, s, w.Pmax, w.Kmax, w.vmax,
                                                                  out, ex);
    } else {
        ozaki_absmax_kernel<double, OZ_ROWS><<<gmax, 256, 0, st>>>(R, K, INT_MAX, K, Xhi, ld, w.vmax);
        if (sl.crt && s == 32)
            ozaki_residues_fast_kernel<double, OZ_ROWS, 32, true><<<gres, 256, 0, st>>>(
                R, K, INT_MAX, Kp, Xhi, Xlo, ld, sl.t, w.Pmax, w.Kmax, w.vmax, out, ex);
        else if (sl.crt)
            ozaki_residues_dd_kernel<OZ_ROWS><<<gdig, 256, 0, st>>>(R, K, Kp, Xhi, Xlo, ld, sl.t, s, w.Pmax, w.Kmax,
                                                                    w.vmax, out, ex, w.crt_dev);
        else
            ozaki_digits_dd_kernel<OZ_ROWS><<<gdig, 256, 0, st>>>(R, K, Kp, Xhi, Xlo, ld, s, w.Pmax, w.Kmax, w.vmax,
                                                                  out, ex);
    }
    SR_CUDA_TRY(cudaGetLastError());
    return SR_OK;
}

sr_status ozaki_split_td(schur_refine_ctx *h, cudaStream_t st, OzakiWork &w, int slot, int R, int K,
                         const double *X0, const double *X1, const double *X2, int ld, int layout, int s)
{
    if (w.cplx || slot < 0 || slot >= kOzakiSlots) return SR_ERR_INVALID_ARG;
    OzakiSlot &sl = w.slot[slot];
    if (!sl.crt || s != kCrtDefaultModuliTD || s != w.crt.N || w.crt.L != 12 || s > sl.cap || R > w.Pmax ||
        K > ozaki_k_limit(false) || K > w.nmax)
        return SR_ERR_INVALID_ARG;
    const int Kp = (K + kOzakiKChunk - 1) / kOzakiKChunk * kOzakiKChunk;
    const int Rp = (R + 31) / 32 * 32;
    SrPhase ph(h, SR_PROF_OZ_SPLIT, 0, 3LL * R * K * 8 + 2LL * s * Kp * Rp, 2);
    sl.layout = layout;
    sl.t = crt_bits(w.crt, K);
    if (sl.t < 1 || sl.t > 174) return SR_ERR_UNSUPPORTED;
    __nv_bfloat16 *out = (__nv_bfloat16 *)sl.dig;
    SR_CUDA_TRY(cudaMemsetAsync(w.vmax, 0, (size_t)Rp * sizeof(unsigned long long), st));
    const dim3 gmax(Rp / 32, (K + SPLIT_KT - 1) / SPLIT_KT);
    const dim3 gres(Rp / 32, (Kp + RES_KT - 1) / RES_KT);
    if (layout == OZ_COLS) {
        ozaki_absmax_kernel<double, OZ_COLS><<<gmax, 256, 0, st>>>(R, K, INT_MAX, K, X0, ld, w.vmax);
        ozaki_residues_td_kernel<OZ_COLS><<<gres, 256, 0, st>>>(R, K, Kp, X0, X1, X2, ld, sl.t, s, w.Pmax, w.Kmax,
                                                               w.vmax, out, sl.exps, w.crt_dev);
    } else {
        ozaki_absmax_kernel<double, OZ_ROWS><<<gmax, 256, 0, st>>>(R, K, INT_MAX, K, X0, ld, w.vmax);
        ozaki_residues_td_kernel<OZ_ROWS><<<gres, 256, 0, st>>>(R, K, Kp, X0, X1, X2, ld, sl.t, s, w.Pmax, w.Kmax,
                                                               w.vmax, out, sl.exps, w.crt_dev);
    }
    SR_CUDA_TRY(cudaGetLastError());
    return SR_OK;
}

sr_status ozaki_split_d6(schur_refine_ctx *h, cudaStream_t st, OzakiWork &w, int slot_hi, int slot_lo, int R, int K,
                         const double *X, size_t pl, int ld, int layout)
{
    if (w.cplx || slot_hi < 0 || slot_hi >= kOzakiSlots || slot_lo < 0 || slot_lo >= kOzakiSlots) return SR_ERR_INVALID_ARG;
    OzakiSlot &sh = w.slot[slot_hi], &sl = w.slot[slot_lo];
    const int s = kCrtDefaultModuliTD;
    if (!sh.crt || !sl.crt || s != w.crt.N || w.crt.L != 12 || s > sh.cap || s > sl.cap || R > w.Pmax ||
        K > ozaki_k_limit(false) || K > w.nmax)
        return SR_ERR_INVALID_ARG;
    const int Kp = (K + kOzakiKChunk - 1) / kOzakiKChunk * kOzakiKChunk;
    const int Rp = (R + 31) / 32 * 32;
    SrPhase ph(h, SR_PROF_OZ_SPLIT, 0, 6LL * R * K * 8 + 4LL * s * Kp * Rp, 2);
    const int t = crt_bits(w.crt, K);
    if (t < 160 || t > 174) return SR_ERR_UNSUPPORTED;   // 2t - 2 >= 318 bits: six doubles
    sh.layout = sl.layout = layout;
    sh.t = sl.t = t;
    SR_CUDA_TRY(cudaMemsetAsync(w.vmax, 0, (size_t)Rp * sizeof(unsigned long long), st));
    const dim3 gmax(Rp / 32, (K + SPLIT_KT - 1) / SPLIT_KT);
    const dim3 gres(Rp / 32, (Kp + RES_KT - 1) / RES_KT);
    __nv_bfloat16 *oh = (__nv_bfloat16 *)sh.dig, *ol = (__nv_bfloat16 *)sl.dig;
    if (layout == OZ_COLS) {
        ozaki_absmax_kernel<double, OZ_COLS><<<gmax, 256, 0, st>>>(R, K, INT_MAX, K, X, ld, w.vmax);
        ozaki_residues_d6_kernel<OZ_COLS><<<gres, 256, 0, st>>>(R, K, Kp, X, pl, ld, t, s, w.Pmax, w.Kmax, w.vmax, oh,
                                                                ol, sh.exps, sl.exps, w.crt_dev);
    } else {
        ozaki_absmax_kernel<double, OZ_ROWS><<<gmax, 256, 0, st>>>(R, K, INT_MAX, K, X, ld, w.vmax);
        ozaki_residues_d6_kernel<OZ_ROWS><<<gres, 256, 0, st>>>(R, K, Kp, X, pl, ld, t, s, w.Pmax, w.Kmax, w.vmax, oh,
                                                                ol, sh.exps, sl.exps, w.crt_dev);
    }
    SR_CUDA_TRY(cudaGetLastError());
    return SR_OK;
}

sr_status ozaki_product(schur_refine_ctx *h, cudaStream_t st, OzakiWork &w, int rows, int cols, int m, int n, int k,
                        int s, bool symmetric, int *flags, int32_t *planes)
{
    if (k > ozaki_k_limit(w.cplx)) return SR_ERR_UNSUPPORTED;
    const bool crt = w.slot[rows].crt != 0;
    if (crt != (w.slot[cols].crt != 0)) return SR_ERR_INVALID_ARG;
    if (s < 1 || s > w.slot[rows].cap || s > w.slot[cols].cap) return SR_ERR_INVALID_ARG;
    if (crt ? (s != w.crt.N || s > 4 * w.levels) : s > w.levels) return SR_ERR_INVALID_ARG;
    const int Kc = (k + kOzakiKChunk - 1) / kOzakiKChunk * kOzakiKChunk;
    const int Kp = w.cplx ? 2 * Kc : Kc;
    // digits: level l sums (l + 1) * chunks exact chunk results below 2^22: keep it below 2^31;
    // residues: one product per level, its sum below 2^28 (the drain's reduction modulo m)
    if (crt ? (Kp / kOzakiKChunk) > 64 : (long long)s * (Kp / kOzakiKChunk) * (1LL << 22) >= (1LL << 31))
        return SR_ERR_UNSUPPORTED;
    const int Mp = (m + BN - 1) / BN * BN;
    const int Np = (n + BM - 1) / BM * BM;
    const long long pairs = crt ? s : (long long)s * (s + 1) / 2;
    const int tiles_i = Mp / BN, tiles_j = Np / BM;
    const int parts = w.cplx ? 2 : 1;
    long long active = 0;
    for (int bj = 0; bj < tiles_j; ++bj)
        for (int bi = 0; bi < tiles_i; ++bi)
            if (!(symmetric && bi * BN > bj * BM + BM - 1)) ++active;
    active *= parts;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
    const long long tile_flops = 2LL * BN * BM * Kp;
    SrPhase ph(h, SR_PROF_OZ_MMA, pairs * active * tile_flops,
               pairs * 2LL * Kp * (Mp + parts * Np) + 4LL * s * active * BN * BM, 1);
    MmaArgs a{};
    a.s = s;
    a.nch = Kp / kOzakiKChunk;
    a.Pmax = w.Pmax;
    a.tiles_i = tiles_i;
    a.tiles_j = tiles_j;
    a.ntiles = tiles_i * tiles_j * parts;
    a.symmetric = symmetric ? 1 : 0;
    a.cplx = w.cplx ? 1 : 0;
    a.conj = (w.cplx && w.slot[rows].layout == OZ_COLS) ? 1 : 0;
    a.planes = planes ? planes : w.planes;
    a.pstride = (size_t)parts * w.Pmax * w.Pmax;
    a.flags = flags;
    a.nact = (int)active;
    a.crt = crt ? 1 : 0;
    if (crt)
        for (int l = 0; l < s; ++l) {
            a.mods[l] = w.crt.m[l];
            a.inv40[l] = w.crt.inv40[l];
            a.off28[l] = w.crt.off28[l];
        }
    // MMA "A" (TMEM lanes) = column-side digits, MMA "B" = row-side digits
    auto launch = [&](int G) {
        a.groups = G;
        if (crt) split_levels_uniform(s, G, a.lvl); else split_levels(s, G, a.lvl);
        a.nitems = a.nact * a.groups;
        const int grid = (int)std::min<long long>(a.nitems, sms);
        ozaki_mma_kernel<false><<<grid, NUM_THREADS, SMEM_BYTES, st>>>(*(const CUtensorMap *)w.slot[rows].map_i,
                                                                       *(const CUtensorMap *)w.slot[cols].map_j, a);
        return cudaGetLastError();
    };
    const long long key = active | (long long)s << 24 | (long long)a.nch << 32 | (long long)parts << 48 |
                          (long long)a.crt << 52;
    int G = -1;
    for (const auto &t : w.tuned)
        if (t.key == key) G = t.groups;
    if (G < 0) {
        int lvl[kCrtMaxModuli + 1];
        G = crt ? level_groups_uniform(s, (int)active, sms, lvl)
                : level_groups(s, (int)active, sms, lvl);   // the makespan estimate
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cs);
        if (w.autotune && cs == cudaStreamCaptureStatusNone) {
            // time every candidate split twice (each launch rewrites the same planes)
            if (!w.tev[0]) SR_CUDA_TRY(cudaEventCreate(&w.tev[0]));
            if (!w.tev[1]) SR_CUDA_TRY(cudaEventCreate(&w.tev[1]));
            float best = -1.f;
            for (int cand = 1; cand <= std::min(s, 4); ++cand)
                for (int rep = 0; rep < 2; ++rep) {
                    SR_CUDA_TRY(cudaEventRecord(w.tev[0], st));
                    SR_CUDA_TRY(launch(cand));
                    SR_CUDA_TRY(cudaEventRecord(w.tev[1], st));
                    SR_CUDA_TRY(cudaEventSynchronize(w.tev[1]));
                    float ms = 0.f;
                    SR_CUDA_TRY(cudaEventElapsedTime(&ms, w.tev[0], w.tev[1]));
                    if (rep == 1 && (best < 0.f || ms < best)) { best = ms; G = cand; }
                }
        }
        w.tuned.push_back({key, G});
    }
    SR_CUDA_TRY(launch(G));
    return SR_OK;
}

cudaError_t ozaki_alloc_group(OzakiWork &w, int rows, int kmax, const int *caps, long long plane_elems,
                              int crt_moduli, unsigned crt_mask)
{
    w.nmax = kmax;
    w.cplx = false;
    w.Pmax = (rows + kOzakiTileI - 1) / kOzakiTileI * kOzakiTileI;
    w.Kmax = (kmax + kOzakiKChunk - 1) / kOzakiKChunk * kOzakiKChunk;
    w.levels = kOzakiMaxSlices;
    for (int i = 0; i < kOzakiSlots; ++i)
        if (!(crt_mask >> i & 1u) || crt_moduli <= 0) w.levels = std::max(w.levels, caps[i]);
    w.pstride_group = plane_elems;
    cudaError_t e = cudaSuccess;
    if (crt_moduli > 0) {
        // FP64 results (4 limbs); crt_moduli byte planes fill (crt_moduli + 3) / 4 level planes
        if (!crt_build_table(crt_moduli, 4, w.crt)) return cudaErrorInvalidValue;
        w.levels = std::max(w.levels, (crt_moduli + 3) / 4);
        e = cudaMalloc((void **)&w.crt_dev, sizeof(CrtTable));
        if (e == cudaSuccess) e = cudaMemcpy(w.crt_dev, &w.crt, sizeof(CrtTable), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
    }
    e = cudaMalloc((void **)&w.planes, (size_t)w.levels * (size_t)plane_elems * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&w.vmax, (size_t)w.Pmax * sizeof(unsigned long long));
    for (int i = 0; i < kOzakiSlots && e == cudaSuccess; ++i) {
        OzakiSlot &sl = w.slot[i];
        sl.cap = caps[i];
        sl.crt = (crt_mask >> i & 1u) && crt_moduli > 0 ? 1 : 0;
        if (sl.crt) sl.cap = crt_moduli;
        if (sl.cap <= 0) continue;
        const size_t bytes = (size_t)sl.cap * w.Pmax * w.Kmax * 2;
        e = cudaMalloc(&sl.dig, bytes);
        if (e == cudaSuccess) e = cudaMalloc((void **)&sl.exps, (size_t)w.Pmax * sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(sl.dig, 0, bytes);
        if (e == cudaSuccess) e = encode_digits_map(sl.map_j, sl.dig, sl.cap * w.Pmax, w.Kmax, BM);
        if (e == cudaSuccess) e = encode_digits_map(sl.map_i, sl.dig, sl.cap * w.Pmax, w.Kmax, BN);
    }
    if (e == cudaSuccess)
        e = set_mma_smem();
    return e;
}

sr_status ozaki_split_group(schur_refine_ctx *h, cudaStream_t st, OzakiWork &w, int slot, const GroupSplit &g,
                            int layout, int s, long long bytes)
{
    if (g.m <= 0) return SR_OK;
    if (slot < 0 || slot >= kOzakiSlots || s < 1 || s > w.slot[slot].cap || g.maxK > w.Kmax)
        return SR_ERR_INVALID_ARG;
    const bool crt = w.slot[slot].crt != 0;
    if (crt ? (s != w.crt.N || s != kCrtDefaultModuli || w.crt.L != 4) : s > kOzakiMaxSlices)
        return SR_ERR_INVALID_ARG;
    SrPhase ph(h, SR_PROF_OZ_SPLIT, 0, bytes, 2);
    w.slot[slot].layout = layout;
    w.slot[slot].t = 0;   // residue form: each matrix's t travels in its SplitMat
    __nv_bfloat16 *out = (__nv_bfloat16 *)w.slot[slot].dig;
    int *ex = w.slot[slot].exps;
    SR_CUDA_TRY(cudaMemsetAsync(w.vmax, 0, (size_t)w.Pmax * sizeof(unsigned long long), st));
    if (crt) {
        if (layout == OZ_COLS) {
            ozaki_absmax_group_kernel<OZ_COLS><<<g.total_max, 256, 0, st>>>(g.mats, g.start_max, g.m, w.vmax);
            ozaki_residues_group_kernel<OZ_COLS><<<g.total_dig, 256, 0, st>>>(g.mats, g.start_dig, g.m, w.Pmax,
                                                                              w.Kmax, w.vmax, out, ex);
        } else {
            ozaki_absmax_group_kernel<OZ_ROWS><<<g.total_max, 256, 0, st>>>(g.mats, g.start_max, g.m, w.vmax);
            ozaki_residues_group_kernel<OZ_ROWS><<<g.total_dig, 256, 0, st>>>(g.mats, g.start_dig, g.m, w.Pmax,
                                                                              w.Kmax, w.vmax, out, ex);
        }
    } else if (layout == OZ_COLS) {
        ozaki_absmax_group_kernel<OZ_COLS><<<g.total_max, 256, 0, st>>>(g.mats, g.start_max, g.m, w.vmax);
        ozaki_digits_group_kernel<OZ_COLS><<<g.total_dig, 256, 0, st>>>(g.mats, g.start_dig, g.m, s, w.Pmax, w.Kmax,
                                                                        w.vmax, out, ex);
    } else {
        ozaki_absmax_group_kernel<OZ_ROWS><<<g.total_max, 256, 0, st>>>(g.mats, g.start_max, g.m, w.vmax);
        ozaki_digits_group_kernel<OZ_ROWS><<<g.total_dig, 256, 0, st>>>(g.mats, g.start_dig, g.m, s, w.Pmax, w.Kmax,
                                                                        w.vmax, out, ex);
    }
    SR_CUDA_TRY(cudaGetLastError());
    return SR_OK;
}

sr_status ozaki_product_items(schur_refine_ctx *h, cudaStream_t st, OzakiWork &w, int rows, int cols,
                              const MmaItem *items, int nitems, int s, long long flops, int *flags)
{
    if (nitems <= 0) return SR_OK;
    const bool crt = w.slot[rows].crt && w.slot[cols].crt;
    if (w.slot[rows].crt != w.slot[cols].crt || (crt && s != w.crt.N)) return SR_ERR_INVALID_ARG;
    if (s < 1 || s > w.slot[rows].cap || s > w.slot[cols].cap || (crt ? s > 4 * w.levels : s > w.levels))
        return SR_ERR_INVALID_ARG;
    // every item's K is at most w.Kmax: level sums stay below 2^31 when s * chunks * 2^22 does
    // (a residue product: one product per level, below 2^28 for 64 chunks)
    if (crt ? (w.Kmax / kOzakiKChunk) > 64 : (long long)s * (w.Kmax / kOzakiKChunk) * (1LL << 22) >= (1LL << 31))
        return SR_ERR_UNSUPPORTED;
    SrPhase ph(h, SR_PROF_OZ_MMA, flops, 0, 1);
    MmaArgs a{};
    a.s = s;
    a.crt = crt ? 1 : 0;
    if (crt)
        for (int l = 0; l < s; ++l) {
            a.mods[l] = w.crt.m[l];
            a.inv40[l] = w.crt.inv40[l];
            a.off28[l] = w.crt.off28[l];
        }
    a.nch = w.Kmax / kOzakiKChunk;
    a.Pmax = w.Pmax;
    a.planes = w.planes;
    a.pstride = (size_t)w.pstride_group;
    a.flags = flags;
    a.items = items;
    a.nitems = nitems;
    a.nact = nitems;
    a.groups = 1;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::min(nitems, sms > 0 ? sms : 1);
    ozaki_mma_kernel<true><<<grid, NUM_THREADS, SMEM_BYTES, st>>>(*(const CUtensorMap *)w.slot[rows].map_i,
                                                                  *(const CUtensorMap *)w.slot[cols].map_j, a);
    SR_CUDA_TRY(cudaGetLastError());
    return SR_OK;
}

}  // namespace sr

extern "C" sr_status schur_refine_crt_info(int N, int limbs, long long K, int *moduli, unsigned *weights,
                                           unsigned *M, int *sigma, int *t)
{
    if (!moduli || !weights || !M || !sigma || !t || K < 1) return SR_ERR_INVALID_ARG;
    sr::CrtTable tab;
    if (!sr::crt_build_table(N, limbs, tab)) return SR_ERR_INVALID_ARG;
    for (int l = 0; l < N; ++l) {
        moduli[l] = tab.m[l];
        for (int k = 0; k < limbs; ++k) weights[l * limbs + k] = tab.w[l][k];
    }
    for (int k = 0; k < limbs; ++k) M[k] = tab.M[k];
    *sigma = tab.sigma;
    *t = sr::crt_bits(tab, K);
    return SR_OK;
}
