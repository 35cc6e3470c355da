// Tensor-core block-Toeplitz far-operator apply (tcgen05 MMA, TMA staging).
//
// The operator is the block-Toeplitz one of a regular solenoid (the coaxial-
// loop inductance depends on r, r' and z - z' only):
//
//     y[t][c] = sum_d sum_c' T_d[c][c'] p[t - d][c'],   d = t_i - t_j,
//
// element e = t C + c.  For one turn offset d this is a (C x C) by
// (C x valid turns) product, so a CTA that owns a tile of 128 channels c and a
// run of (64-channel k block, offset) stages runs, on the tensor cores,
//
//     D[c][t] += A_d[c][k] B_d[t][k],   A_d = T_d tile,  B_d[t][.] = p[t - d][.],
//
// with the turn index t as the MMA's N dimension.  For offset d only turns
// max(0, d) <= t < min(NT, NT + d) have a source row; each MMA covers exactly
// those turns (from a multiple of 8, N rounded up to 16), writes its
// accumulator at TMEM column t, and reads its B operand as a window, starting
// at row t - d, of one staged copy of p (rows -8 .. NT + 15, zero outside the
// winding).  So the Toeplitz shift costs no copy and almost no padded work.
//
// Only the offsets d >= 0 are stored: T_{-d} = T_d^T (M is symmetric), so the
// tile of T_d that serves y += T_d p, read K-major, serves y += T_d^T p read
// MN-major from the same shared memory: every table byte feeds two products.
//
// Precision: entries and inputs are scaled by powers of two (2^exT brings
// max |T| over the table below 2^14, 2^x[t] the largest |p| of turn row t)
// and split v = hi + lo into two FP16 numbers.  The staged input holds the hi
// rows and the lo rows of the turns as two blocks, so per K step three MMAs
// A_hi x B_hi, A_hi x B_lo and A_lo x B_hi add the three products that keep
// about 22 significant bits (the FP32 class) into accumulator column t.  The
// tensor cores' FP32 accumulation does not round to nearest, so its error
// grows with the number of MMAs added into one accumulator; here an
// accumulator takes only one stage (one offset, one 64-channel k block: 12
// MMAs), after which the epilogue warps add its columns into FP32 registers
// (round to nearest), column t times 2^(xmin - x[t - d]): the scale of its
// source row relative to the largest-scale row, an exact power of two of at
// most 1, so the FP32 sums stay in the range of a single global scale.  The
// reduction removes 2^(xmin + exT) in FP64.  Up to four TMEM accumulators
// rotate, so the MMAs of the next stages run while one is drained.  The CTAs'
// partial tiles are summed in a fixed order: the result is deterministic.
//
// Work split: every 128-channel tile gets the same number of CTAs (one per
// SM: 144 for 960 channels).  A tile's steps (k, D), k = 0 .. n_ct - 1,
// D = 0 .. NT - 1, pair it with column tile cb = (k - tile) mod n_ct and run
// the stages (k block, +D) and, for D > 0, (k block, -D) for both k blocks of
// cb; each CTA takes a contiguous range of steps, the ranges balanced by
// stage count.  The CTA of tile cb with the same range reads the same
// 128 x 128 region of T_D (transposed) at about the same time, so the region
// comes from DRAM once and from L2 once.  One staged copy of p (the column
// tile's 128 channels) is loaded per change of cb.
//
// CTA roles (672 threads): warp 0 issues the TMA loads, warps 1-4 issue the
// MMAs of every fourth stage each (warp 1 owns the TMEM; one thread issues a
// small-N MMA far slower than the tensor cores run it), warps 5-20 drain the
// accumulators (lane quadrant warp % 4, 8-turn groups g of one residue g mod 4).
// Every wait on an mbarrier is bounded: on a timeout the CTA raises an abort
// flag, the others stop issuing, the copies and MMAs already in flight are
// waited for (again bounded), the TMEM is freed, and the coil's status word
// reports the failure to the host.
#include "toeplitz_tc.h"
#include "seg.cuh"

#include <cuda_fp16.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

namespace cq {

constexpr int kTcM = kTcTileRows;                // channels per tile (MMA M)
constexpr int kTcK = 64;                         // channels per k block (one 128-byte FP16 row)
constexpr int kTcPad = 8;                        // zero turn rows staged below the winding
constexpr int kTcPadTop = 16;                    // and above it (an MMA's N rounds up to 16 turns)
constexpr int kTcParities = 4;                   // epilogue warps per lane quadrant (turn groups g mod kTcParities)
constexpr int kTcEpiWarps = 4 * kTcParities;     // epilogue warps: 4 lane quadrants x kTcParities
constexpr int kTcIssuers = 4;                    // MMA-issuing warps, taking the stages in turn
constexpr int kTcEpi0 = 1 + kTcIssuers;          // first epilogue warp
constexpr float kTcTableEvictFirst = 1.0f;       // fraction of the table's lines loaded evict-first
constexpr int kTcNearWarps = 1;                  // FP64 near-block products beside the apply (two-fill)
constexpr int kTcNear0 = kTcEpi0 + kTcEpiWarps;   // first near warp
constexpr int kTcThreads = 32 * kTcNear0;      // producer, MMA issuers, epilogue
constexpr int kTcThreadsNear = kTcThreads + 32 * kTcNearWarps;   // the single-coil two-fill apply: + near warps
constexpr int kTcGroups = (14 + kTcParities - 1) / kTcParities;   // 8-turn groups per epilogue warp (NT <= 112)
constexpr uint32_t kTcAStage = 2u * kTcM * kTcK * 2u;   // hi + lo table tiles, 32 KB
// MN-major A (128-byte swizzle): byte offsets between the two 64-channel
// blocks along M (8 KB) and between 8-row groups along K (1 KB)
constexpr uint32_t kTcMnLbo = 8192u;
constexpr uint32_t kTcMnSbo = 1024u;
constexpr int kTcSmemLimit = 227 * 1024;         // dynamic shared memory per CTA (opt-in maximum)
constexpr long long kTcWait = 1LL << 31;         // cycles before a wait gives up (~1 s)
constexpr int kTcBStages = 1;                    // staged copies of p (a CTA meets few k blocks)
constexpr long long kTcMinSteps = 8;             // schedule steps per CTA, at least (see tc_schedule)
constexpr long long kTcMinCtas = 4;              // CTAs per channel tile the step floor keeps
__host__ __device__ constexpr int kTcBars(int stages) { return 2 * stages + 2 * kTcBStages + 9; }

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Non-blocking test of the phase of the given parity.
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// The same test, the thread suspended (issuing nothing) until the phase
// completes or about `ns` nanoseconds have passed.
__device__ __forceinline__ bool mbar_try_sleep(uint32_t bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}
constexpr uint32_t kTcSleepNs = 2000;            // longest suspension between two limit checks
// Wait for the phase of the given parity; false on abort or after `limit`
// cycles (then the abort flag is raised).  The limit is checked after every
// failed non-blocking test, before the thread suspends again, so that a short
// limit (the test hook) runs out at the first phase that is not complete.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, long long limit) {
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > limit) {
            *abort_flag = 1;
            return false;
        }
        if (mbar_try_sleep(bar, parity, kTcSleepNs)) return true;
    }
}
// Inline fast path for a phase that has already completed.
__device__ __forceinline__ bool mbar_wait_fast(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                               long long limit) {
    return mbar_try(bar, parity) || mbar_wait(bar, parity, abort_flag, limit);
}
// The same, ignoring the abort flag (used to retire work already in flight).
__device__ __noinline__ bool mbar_wait_final(uint32_t bar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (clock64() - t0 > limit) return false;
        if (mbar_try_sleep(bar, parity, kTcSleepNs)) return true;
    }
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, int w,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, int w, int v,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(v), "r"(bar)
        : "memory");
}

// The same with an L2 cache policy (createpolicy) for the copied lines.
__device__ __forceinline__ void tma_load_5d_hint(uint32_t dst, const CUtensorMap* map, int x, int y, int z, int w,
                                                 int v, uint32_t bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7], %8;" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(v), "r"(bar), "l"(pol)
        : "memory");
}

// L2 policy of the operator table's tiles: evict first.  The table (hundreds
// of MB, read once per apply by each CTA of a pair) then streams through L2
// without pushing out what the other kernels of the solve keep there (the
// vectors, partial tiles and per-wire blocks they read every iteration).
__device__ __forceinline__ uint64_t tc_table_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, %1;" : "=l"(pol) : "f"(kTcTableEvictFirst));
    return pol;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets, descriptor version 1, layout 0 (no swizzle) or 2 (128-byte swizzle).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)layout << 61);
}
// Instruction descriptor of kind::f16: FP16 A and B, FP32 D, M = 128, N = n;
// B K-major, A K-major or (a_mn) MN-major.
__device__ __forceinline__ uint32_t idesc_f16(int n, bool a_mn) {
    return (1u << 4) | ((a_mn ? 1u : 0u) << 15) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// One stage: 4 K steps x (A_hi B_hi, A_hi B_lo, A_lo B_hi) into accumulator d
// as one block of 12 MMAs, issued by the warp's elected lane with the whole
// warp executing it (converged), every descriptor formed before the first: a
// single thread then issues them back to back at about the tensor cores' pace,
// where one MMA per address computation costs it about twice as long.  The
// first MMA overwrites the accumulator unless acc0.
__device__ __forceinline__ void mma_stage_warp(uint32_t d, uint32_t idesc, uint32_t acc0, uint64_t a_hi,
                                               uint64_t a_lo, uint64_t a_step, uint64_t b_hi, uint64_t b_lo,
                                               uint64_t b_step) {
    uint64_t ah[4], al[4], bh[4], bl[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        ah[k] = a_hi + k * a_step;
        al[k] = a_lo + k * a_step;
        bh[k] = b_hi + k * b_step;
        bl[k] = b_lo + k * b_step;
    }
    asm volatile(
        "{\n\t.reg .pred p, e, t;\n\t"
        "setp.ne.b32 p, %1, 0;\n\t"
        "setp.eq.b32 t, %1, %1;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %3, %11, %2, p;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %3, %15, %2, t;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %7, %11, %2, t;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %4, %12, %2, t;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %4, %16, %2, t;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %8, %12, %2, t;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %5, %13, %2, t;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %5, %17, %2, t;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %9, %13, %2, t;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %6, %14, %2, t;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %6, %18, %2, t;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %10, %14, %2, t;\n\t}" ::"r"(d),
        "r"(acc0), "r"(idesc), "l"(ah[0]), "l"(ah[1]), "l"(ah[2]), "l"(ah[3]), "l"(al[0]), "l"(al[1]), "l"(al[2]),
        "l"(al[3]), "l"(bh[0]), "l"(bh[1]), "l"(bh[2]), "l"(bh[3]), "l"(bl[0]), "l"(bl[1]), "l"(bl[2]), "l"(bl[3])
        : "memory");
}
// tcgen05.commit by the warp's elected lane (the same lane as in mma_stage_warp:
// elect.sync picks the same lane for the same full mask, so the commit tracks
// that lane's MMAs).
__device__ __forceinline__ void mma_commit_warp(uint32_t bar) {
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(bar)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// ---------------------------------------------------------------------------
// The apply
// ---------------------------------------------------------------------------
// The two-fill apply of one coil by one CTA: work entry wk = (channel tile,
// first step, end step), partial tile `cta` of `part`.  The tensor maps may
// live in the kernel's parameters or in global memory (a batch).
// near_src / near_dst (may be null): the near warps form the near-block part
// of q for this CTA's share of the coil's wires (FP64; the apply itself uses
// no FP64, so it runs on otherwise idle units), read by k_near_seg.
__device__ __forceinline__ void tc_apply_cta(const CUtensorMap* mapA, const CUtensorMap* mapAT,
                                             const CUtensorMap* mapB, const CoilDev& c, const TcShape sh,
                                             const int4 wk, const int cta, const int* __restrict__ pexp,
                                             float* __restrict__ part, const double* __restrict__ near_src,
                                             double* __restrict__ near_dst, const bool table_ef) {
    const CUtensorMap& tmA = *mapA;
    const CUtensorMap& tmAT = *mapAT;
    const CUtensorMap& tmB = *mapB;
    if (c.sc->done) return;
    // the limit of the waits that raise the abort flag (a test hook can shorten
    // it; the waits that retire work already in flight keep kTcWait)
    const long long wlim = c.sc->tc_wait > 0 ? c.sc->tc_wait : kTcWait;
    extern __shared__ uint8_t tc_smem[];
    const uint32_t raw = su32(tc_smem);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gbase = tc_smem + (base - raw);
    const uint32_t b_stage = 512u * (uint32_t)sh.NR;             // hi + lo staged p of 128 channels, bytes
    const uint32_t b_pitch = (b_stage + 127u) & ~127u;
    const uint32_t sA = base;                                     // sh.stages x 32 KB (1024-aligned)
    const uint32_t sB = base + (uint32_t)sh.stages * kTcAStage;   // kTcBStages staged copies of p
    const uint32_t bar_off = (uint32_t)sh.stages * kTcAStage + kTcBStages * b_pitch;
    const uint32_t sBar = base + bar_off;
    const int S = sh.stages;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(gbase + bar_off + 8 * kTcBars(S));
    uint32_t* tslot = reinterpret_cast<uint32_t*>(gbase + bar_off + 8 * kTcBars(S) + 4);
    int* xmin_s = reinterpret_cast<int*>(gbase + bar_off + 8 * kTcBars(S) + 8);
    // relative inverse input scale of staged row r (p row r - 16; zero outside the
    // winding), in four copies shifted by 0..3 entries (copy k holds entry r + k at
    // r), so that any 16 consecutive entries are four aligned 16-byte loads
    const int scp = (sh.NR + 7) & ~3;                             // floats per copy
    float* inv_s = reinterpret_cast<float*>(gbase + ((bar_off + 8 * kTcBars(S) + 16 + 15) & ~15u));
    // barriers: a_full[S], a_empty[S], b_full[kTcBStages], b_empty[kTcBStages], acc_full[4],
    // acc_empty[4], mma_done
    const uint32_t a_full = sBar, a_empty = sBar + 8u * S;
    const uint32_t b_full = sBar + 16u * S, b_empty = b_full + 8u * kTcBStages;
    const uint32_t acc_full = b_empty + 8u * kTcBStages, acc_empty = acc_full + 32u;
    const uint32_t mma_done = acc_empty + 32u;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // This CTA's work: channel tile ct, steps wk.y <= sg < wk.z.  Step sg = (k, D),
    // k = sg / NT, D = sg % NT, pairs the tile with column tile cb = (k - ct) mod
    // n_ct and runs the stages (kb, +D) and, for D > 0, (kb, -D), kb = 2 cb, 2 cb + 1.
    // Column tile cb's CTA with the same step range is at step k with cb and ct
    // exchanged: it reads the same 128 x 128 region of the stored T_D, transposed,
    // at the same time, so that region comes from DRAM once and from L2 once.
    const int ct = wk.x, c0 = ct * kTcM;
    auto col_tile = [&](int sg) { return (sg / sh.NT - ct + sh.n_ct) % sh.n_ct; };
    const int n_acc = sh.n_acc;
    const uint32_t acc_cols = (uint32_t)sh.acc_cols;

    if (threadIdx.x == 0) {
        for (int b = 0; b < kTcBars(S); ++b) {
            const uint32_t bar = sBar + 8u * b;
            // acc_empty: one arrival per epilogue warp; b_empty and mma_done: one per MMA
            // issuer; the others: one arrival (+ bytes)
            const bool two = bar == b_empty || bar == mma_done;
            mbar_init(bar, (bar >= acc_empty && bar < acc_empty + 32u) ? (uint32_t)kTcEpiWarps
                                                                         : (two ? (uint32_t)kTcIssuers : 1u));
        }
        *abort_flag = 0;
        *xmin_s = 1 << 30;
        mbar_fence_init();
    }
    __syncthreads();
    if (warp == 0) {
        const int m = warp_min_exponent(pexp, sh.NT, lane);
        if (lane == 0) *xmin_s = m;
    }
    if (warp == 1) {
        __syncwarp();
        tmem_alloc(su32(tslot), (uint32_t)sh.ncols);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(tslot);
    for (int i = threadIdx.x; i < 4 * scp; i += blockDim.x) {
        const int k = i / scp, r = i - k * scp + k, t = r - kTcPad;
        inv_s[i] = (t >= 0 && t < sh.NT) ? ldexpf(1.f, *xmin_s - pexp[t]) : 0.f;
    }
    __syncthreads();

    if (warp == 0 && lane == 0) {
        // ---- producer: per k block one staged p copy, then the table tiles of every offset
        int sa = 0, sb = 0;
        uint32_t pa = 0, pb = 0;
        uint32_t a_used = 0, a_par = 0, b_used = 0, b_par = 0;   // bit s: stage s loaded / its parity
        const uint64_t pol = tc_table_policy();
        bool ok = true;
        int D = wk.y % sh.NT, cb = col_tile(wk.y);
        for (int sg = wk.y; sg < wk.z && ok; ++sg, D = (D + 1 == sh.NT ? 0 : D + 1)) {
            if (sg != wk.y && D == 0) cb = (cb + 1 == sh.n_ct ? 0 : cb + 1);
            const int nk = min(2, sh.n_kb - 2 * cb);
            if (sg == wk.y || D == 0) {                 // a new column tile: its staged copy of p
                ok = mbar_wait(b_empty + 8u * sb, pb ^ 1u, abort_flag, wlim);
                if (!ok) break;
                mbar_expect_tx(b_full + 8u * sb, b_stage);
                // turn rows -kTcPad .. NT + kTcPadTop - 1, hi and lo, of 16 chunks
                tma_load_4d(sB + (uint32_t)sb * b_pitch, &tmB, 0, -kTcPad, 0, cb * (kTcM / 8), b_full + 8u * sb);
                b_used |= 1u << sb;
                b_par = (b_par & ~(1u << sb)) | (pb << sb);
                if (++sb == kTcBStages) { sb = 0; pb ^= 1u; }
            }
            for (int sgn = 0; sgn < (D > 0 ? 2 : 1) && ok; ++sgn)
                for (int j = 0; j < nk && ok; ++j) {
                    const int kb = 2 * cb + j, d = sgn ? -D : D;
                    ok = mbar_wait_fast(a_empty + 8u * sa, pa ^ 1u, abort_flag, wlim);
                    if (!ok) break;
                    mbar_expect_tx(a_full + 8u * sa, kTcAStage);
                    // offset d >= 0: T_d tile, K-major; d < 0: T_d = T_{-d}^T, the stored tile
                    // of T_{-d} (rows c' of this k block, columns c of the channel tile)
                    const uint32_t dst = sA + (uint32_t)sa * kTcAStage;
                    if (table_ef) {
                        if (d >= 0)
                            tma_load_5d_hint(dst, &tmA, 0, c0, kb, d, 0, a_full + 8u * sa, pol);
                        else
                            tma_load_5d_hint(dst, &tmAT, 0, kb * kTcK, c0 / kTcK, -d, 0, a_full + 8u * sa, pol);
                    } else {
                        if (d >= 0)
                            tma_load_5d(dst, &tmA, 0, c0, kb, d, 0, a_full + 8u * sa);
                        else
                            tma_load_5d(dst, &tmAT, 0, kb * kTcK, c0 / kTcK, -d, 0, a_full + 8u * sa);
                    }
                    a_used |= 1u << sa;
                    a_par = (a_par & ~(1u << sa)) | (pa << sa);
                    if (++sa == S) { sa = 0; pa ^= 1u; }
                }
        }
        // retire the copies in flight (only the latest load of a stage can be)
        for (int s = 0; s < S; ++s)
            if (a_used >> s & 1u) mbar_wait_final(a_full + 8u * s, a_par >> s & 1u, kTcWait);
        for (int s = 0; s < kTcBStages; ++s)
            if (b_used >> s & 1u) mbar_wait_final(b_full + 8u * s, b_par >> s & 1u, kTcWait);
    } else if (warp >= 1 && warp < kTcEpi0) {
        // ---- MMA issuers (whole warps, the elected lane issuing): stage i of this
        // CTA (table slot i % S, TMEM accumulator i % n_acc, the latter's first MMA
        // overwriting the columns it covers) is issued by warp 1 + i % kTcIssuers,
        // so that the issuing threads' overheads and the MMA chains into different
        // accumulators overlap; each issuer frees a staged copy of p (one arrival
        // each) once it has no more stages on it.  The issuer's stages are
        // i = me, me + 4, ...: their slot, accumulator and parities advance without
        // divisions (a runtime division costs more than issuing a stage).
        const int me = warp - 1;
        int grp = 0;
        bool ok = true;
        const uint32_t bbase = sB;                      // one staged copy (kTcBStages == 1)
        int D = wk.y % sh.NT, cb = col_tile(wk.y);
        int i0 = 0;                                     // the step's first stage
        int sa_i = me % S, ai_i = me % n_acc;           // this issuer's next stage i: i % S, i % n_acc
        uint32_t pa_i = (uint32_t)(me / S) & 1u, pacc_i = (uint32_t)(me / n_acc) & 1u;
        for (int sg = wk.y; sg < wk.z && ok; ++sg, D = (D + 1 == sh.NT ? 0 : D + 1)) {
            if (sg != wk.y && D == 0) cb = (cb + 1 == sh.n_ct ? 0 : cb + 1);
            const int nk = min(2, sh.n_kb - 2 * cb);
            if (sg == wk.y || D == 0) {
                if (sg != wk.y) mma_commit_warp(b_empty);    // free once this issuer's MMAs on it finish
                ok = __all_sync(0xffffffffu, mbar_wait(b_full, (uint32_t)grp & 1u, abort_flag, wlim));
                if (!ok) break;
                ++grp;
                tc_fence_after();
            }
            // this issuer's stages of the step: positions pos = sgn nk + j with
            // (i0 + pos) % kTcIssuers == me (one per step in the common case)
            const int ns = (D > 0 ? 2 : 1) * nk;
            for (int pos = ((me - i0) % kTcIssuers + kTcIssuers) % kTcIssuers; pos < ns && ok;
                 pos += kTcIssuers) {
                const int sgn = pos >= nk ? 1 : 0, j = pos - sgn * nk;
                const int d = sgn ? -D : D;
                // staged copy: [16 chunks of 8 channels][hi, lo][NR turn rows][8];
                // k block j of the column tile = chunks 8 j .. 8 j + 7
                const uint32_t bj = bbase + (uint32_t)j * 256u * (uint32_t)sh.NR;
                // accumulator first: its release by the drain of stage i - n_acc means
                // every stage up to there has completed its MMAs, so (S >= n_acc) the
                // previous load of this stage's slot has landed and the parity wait
                // below cannot be satisfied by the phase before it (another issuer's)
                ok = __all_sync(0xffffffffu, mbar_wait_fast(acc_empty + 8u * ai_i, pacc_i ^ 1u, abort_flag, wlim));
                if (ok) ok = __all_sync(0xffffffffu, mbar_wait_fast(a_full + 8u * sa_i, pa_i, abort_flag, wlim));
                if (!ok) break;
                tc_fence_after();
                const int t_first = d > 0 ? d : 0;
                const int t_end = d < 0 ? sh.NT + d : sh.NT;
                const int ts = t_first & ~7;
                const int n = (t_end - ts + 15) & ~15;          // turns covered = accumulator columns
                const bool amn = d < 0;
                const uint32_t ah = sA + (uint32_t)sa_i * kTcAStage;
                // K-major A: rows of 64 channels c', 8-row groups 1 KB apart, K step = 32 B.
                // MN-major A: rows of 64 channels c (two 8 KB blocks along M), one row per
                // c', 8-row groups 1 KB apart, K step = 16 rows = 2 KB.  B: K step = two
                // 8-channel chunks.  The descriptors are built once per stage and advanced
                // by adding to their address field (addr >> 4, below 2^14 for any shared
                // memory address, so the additions never carry out of it).
                const uint64_t a_hi = amn ? sdesc(ah, kTcMnLbo, kTcMnSbo, 2u) : sdesc(ah, 16u, 1024u, 2u);
                const uint64_t a_lo = a_hi + (((uint64_t)kTcM * 128u) >> 4);
                const uint64_t a_step = amn ? (2048u >> 4) : (32u >> 4);
                // B: the n rows of turns ts .. ts + n - 1 (source rows ts - d ..) of the hi
                // and of the lo half; three MMAs per K step, hi*hi + hi*lo + lo*hi, into
                // accumulator column t (n <= NT + 15 < 256: one MMA covers the turns)
                const uint64_t b_step = (2u * 32u * (uint32_t)sh.NR) >> 4;
                const uint64_t b_half = (16u * (uint32_t)sh.NR) >> 4;
                const uint32_t idesc = idesc_f16(n, amn);
                const uint32_t dcol = tmem + (uint32_t)ai_i * acc_cols + (uint32_t)ts;
                const uint32_t row0 = (uint32_t)(ts - d + kTcPad);
                const uint64_t b_hi = sdesc(bj + 16u * row0, 32u * (uint32_t)sh.NR, 128u, 0u);
                static_assert(kTcK == 64, "one stage = 4 K steps of 16");
                mma_stage_warp(dcol, idesc, 0u, a_hi, a_lo, a_step, b_hi, b_hi + b_half, b_step);
                mma_commit_warp(a_empty + 8u * sa_i);
                mma_commit_warp(acc_full + 8u * ai_i);
                // this issuer's next stage: i + kTcIssuers
                sa_i += kTcIssuers;
                while (sa_i >= S) { sa_i -= S; pa_i ^= 1u; }
                ai_i += kTcIssuers;
                while (ai_i >= n_acc) { ai_i -= n_acc; pacc_i ^= 1u; }
            }
            i0 += ns;
        }
        // every MMA issued (also after an abort) completes before the TMEM is freed
        __syncwarp();
        mma_commit_warp(mma_done);
        if (!__all_sync(0xffffffffu, mbar_wait_final(mma_done, 0u, kTcWait)) && lane == 0) *abort_flag = 1;
    } else if (warp >= kTcNear0) {
        // ---- near warps: the near-block products of this CTA's share of the
        // wires, two 16-element wires (a segment each) per warp task
        if (near_dst && c.B <= kSegMax) {
            // start once the table pipeline has filled: beside its first loads
            // they slowed the apply (4 us measured best, 12 us the same, 30 us worse)
            __nanosleep(4000);
            const int n_task = (c.W + 32 / seg_width(c.B) - 1) / (32 / seg_width(c.B));
            for (int wg = cta * kTcNearWarps + (warp - kTcNear0); wg < n_task; wg += (int)gridDim.x * kTcNearWarps) {
                const Seg s = seg_of(c, wg);
                const double pv = s.ev ? near_src[s.e] : 0.0;
                const double ge = s.ev ? c.G[s.e] : 0.0;
                const double q = near_row_product(c, s, c.block_type[s.wv ? s.w : 0], pv, ge);
                if (s.ev) near_dst[s.e] = q;
            }
        }
    } else if (warp >= kTcEpi0 && warp < kTcNear0) {
        // ---- epilogue: each stage's accumulator is added into FP32 registers (lane
        // quadrant warp % 4, turn groups of parity h), then released to the MMAs
        const int q = warp & 3;
        const int h = (warp - kTcEpi0) >> 2;
        const int cc = c0 + 32 * q + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        float acc[kTcGroups][8];                       // turn group g = kTcParities gi + h: turns 8 g .. 8 g + 7
#pragma unroll
        for (int g = 0; g < kTcGroups; ++g)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[g][j] = 0.f;
        int ai = 0;
        uint32_t pf = 0;
        bool ok = true;
        int D = wk.y % sh.NT, cb = col_tile(wk.y);
        for (int sg = wk.y; sg < wk.z && ok; ++sg, D = (D + 1 == sh.NT ? 0 : D + 1)) {
            if (sg != wk.y && D == 0) cb = (cb + 1 == sh.n_ct ? 0 : cb + 1);
            const int nk = min(2, sh.n_kb - 2 * cb);
            for (int st = 0; st < (D > 0 ? 2 : 1) * nk; ++st) {
                const int d = st >= nk ? -D : D;
                ok = __all_sync(0xffffffffu, mbar_wait_fast(acc_full + 8u * ai, (pf >> ai) & 1u, abort_flag, wlim));
                if (!ok) break;
                pf ^= 1u << ai;
                tc_fence_after();
                const int t_first = d > 0 ? d : 0;
                const int t_end = d < 0 ? sh.NT + d : sh.NT;
                const int g_lo = t_first >> 3, g_hi = (t_end + 7) >> 3;
                const uint32_t src = lane_base + (uint32_t)ai * acc_cols;
#pragma unroll
                for (int gi = 0; gi < kTcGroups; ++gi) {
                    const int g = kTcParities * gi + h;
                    if (g >= g_lo && g < g_hi) {
                        float v[8];                             // columns of turns 8 g .. 8 g + 7
                        tmem_ld8(src + 8u * (uint32_t)g, v);
                        // scales of source rows 8 g + i - d (staged rows + kTcPad): copy a % 4
                        const int a = 8 * g + kTcPad - d;
                        const float4* sc4 = reinterpret_cast<const float4*>(inv_s + (a & 3) * scp + (a & ~3));
#pragma unroll
                        for (int q4 = 0; q4 < 2; ++q4) {
                            const float4 f = sc4[q4];
                            acc[gi][4 * q4 + 0] = fmaf(v[4 * q4 + 0], f.x, acc[gi][4 * q4 + 0]);
                            acc[gi][4 * q4 + 1] = fmaf(v[4 * q4 + 1], f.y, acc[gi][4 * q4 + 1]);
                            acc[gi][4 * q4 + 2] = fmaf(v[4 * q4 + 2], f.z, acc[gi][4 * q4 + 2]);
                            acc[gi][4 * q4 + 3] = fmaf(v[4 * q4 + 3], f.w, acc[gi][4 * q4 + 3]);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acc_empty + 8u * ai);
                if (++ai == n_acc) ai = 0;
            }
        }
        if (ok && !*abort_flag && cc < sh.C) {
            // partial tile of this CTA: part[cta][t][c - c0]
            float* out = part + (size_t)cta * sh.NT * kTcM + 32 * q + lane;
#pragma unroll
            for (int gi = 0; gi < kTcGroups; ++gi) {
                const int t0 = 8 * (kTcParities * gi + h);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (t0 + j < sh.NT) out[(size_t)(t0 + j) * kTcM] = acc[gi][j];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0 && *abort_flag) {
        atomicExch(&c.sc->status, (int)ST_KERNEL);
        atomicExch(&c.sc->done, 1);
    }
    if (warp == 1) {
        __syncwarp();
        tmem_dealloc(tmem, (uint32_t)sh.ncols);
    }
}

__global__ void __launch_bounds__(kTcThreadsNear, 1)
k_toeplitz_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAT,
              const __grid_constant__ CUtensorMap tmB,
              const CoilDev* __restrict__ cd, const TcShape sh, const int4* __restrict__ work,
              const int* __restrict__ pexp, float* __restrict__ part, const double* __restrict__ near_src,
              double* __restrict__ near_dst) {
    tc_apply_cta(&tmA, &tmAT, &tmB, *cd, sh, work[blockIdx.x], (int)blockIdx.x, pexp, part, near_src, near_dst,
                 true);
}

// A batch's applies in one launch: CTA b works for coil bwork[b].x as its
// CTA bwork[b].y, with that coil's maps, schedule and partial tiles.
__global__ void __launch_bounds__(kTcThreads, 1)
k_toeplitz_tc_batch(const TcCoilArgs* __restrict__ args, const int2* __restrict__ bwork) {
    const int2 bw = bwork[blockIdx.x];
    const TcCoilArgs& A = args[bw.x];
    if (threadIdx.x == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&A.tmA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&A.tmAT)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&A.tmB)) : "memory");
    }
    // a batch's tables keep the default L2 policy (evict-first measured slower there)
    tc_apply_cta(&A.tmA, &A.tmAT, &A.tmB, *A.d, A.sh, A.work[bw.y], bw.y, A.pexp, A.part, nullptr, nullptr, false);
}

// ---------------------------------------------------------------------------
// One-fill apply: every table tile serves both of its products
// ---------------------------------------------------------------------------
//
// The apply above loads each stored tile twice (once K-major by the CTA of its
// row tile, once MN-major by the CTA of the transposed block), and what bounds
// it is the rate at which TMA fills an SM's shared memory.  Here the unit of
// work is a combination (channel tile a, 64-channel k block kb); its stage D
// loads the tile A = T_D[a rows][kb columns] once and issues
//
//   (1)  y[t][a]  += A p[t - D][kb]      M = 128 (a), K = 64 (kb), K-major A
//   (2)  y[t][kb] += A^T p[t + D][a]     M = 64 (kb), K = 128 (a), MN-major A
//
// (2) only for D > 0: T_{-D} = T_D^T (M is symmetric), so over every (a, kb)
// and D the two products give all offsets -NT < d < NT, and at D = 0 the
// stored T_0 is applied whole by (1).  The staged inputs are p[kb] (64
// channels, B of (1)) and p[a] (128 channels, B of (2)), one copy each, in
// the K-major split layout of the input; the kb copy changes with every
// combination, the a copy every n_kb combinations (kb runs fastest).
//
// Accumulators: stage i takes the pair i % n_acc, (1) into 128 lanes of its
// first acc_cols columns, (2) into the next acc_cols columns, where an M = 64
// product leaves row r of D in lane 32 (r / 16) + r % 16 (lanes 0-15 of each
// lane quadrant).  The drain warps add both into FP32 registers (as above),
// (2) read with the 16x32bx2 shape so that the 16 rows of a quadrant serve
// two 8-turn groups per load, and write a partial tile per combination the
// CTA worked on: part1[segment][t][128] for y[a], part2[segment][t][64] for
// y[kb].  The reduction sums, for every element, the segments of its channel
// tile (part1) and of its k block (part2) in a fixed order.
//
// Work split: the n_ct n_kb NT stages in (a, kb, D) order are dealt to the
// CTAs as equal contiguous ranges; a range crosses at most a few combination
// boundaries, each a new segment.
constexpr uint32_t kT2ABytes = 512u;             // bytes per staged turn row of p[a] (128 channels, hi + lo)
constexpr uint32_t kT2KBytes = 256u;             // of p[kb] (64 channels)
constexpr long long kT2MinStages = 8;            // stages per CTA, at least (small coils take few SMs)
__host__ __device__ constexpr int kT2Bars(int stages, int n_acc) { return 2 * stages + 4 + 2 * n_acc + 1; }

// Instruction descriptor of kind::f16 (FP16 A and B, FP32 D) for M = m.
__device__ __forceinline__ uint32_t idesc_f16m(int n, bool a_mn, int m) {
    return (1u << 4) | ((a_mn ? 1u : 0u) << 15) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// 16 lanes x 8 columns twice: threads 0-15 read lanes 0-15 of the quadrant at
// columns taddr .. +7, threads 16-31 the same lanes at columns taddr + 8 .. +15.
__device__ __forceinline__ void tmem_ld16x2_8(uint32_t taddr, float* v) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.16x32bx2.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8], 8;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void scale_add8(const float* inv_s, int scp, int a, const float* v, float* acc) {
    // scales of staged rows a .. a + 7 (copy a % 4 holds entry r + (a % 4) at r)
    const float4* sc4 = reinterpret_cast<const float4*>(inv_s + (a & 3) * scp + (a & ~3));
#pragma unroll
    for (int q4 = 0; q4 < 2; ++q4) {
        const float4 f = sc4[q4];
        acc[4 * q4 + 0] = fmaf(v[4 * q4 + 0], f.x, acc[4 * q4 + 0]);
        acc[4 * q4 + 1] = fmaf(v[4 * q4 + 1], f.y, acc[4 * q4 + 1]);
        acc[4 * q4 + 2] = fmaf(v[4 * q4 + 2], f.z, acc[4 * q4 + 2]);
        acc[4 * q4 + 3] = fmaf(v[4 * q4 + 3], f.w, acc[4 * q4 + 3]);
    }
}

// A bounded wait of the one-fill apply that, when it runs out, records where
// (site, CTA, stage, index, parity, thread) for the host's error message.
__device__ __noinline__ bool wait2(const CoilDev& c, uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                   long long limit, int site, int s, int i) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > limit) {
            *abort_flag = 1;
            if (atomicCAS(&c.sc->tc_where[0], 0, site) == 0) {
                c.sc->tc_where[1] = blockIdx.x;
                c.sc->tc_where[2] = s;
                c.sc->tc_where[3] = i;
                c.sc->tc_where[4] = (int)parity;
                c.sc->tc_where[5] = threadIdx.x;
            }
            return false;
        }
        if (mbar_try_sleep(bar, parity, kTcSleepNs)) return true;
    }
}

__global__ void __launch_bounds__(kTcThreads, 1)
k_toeplitz_tc2(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmB64, const CoilDev* __restrict__ cd, const TcShape sh,
               const int4* __restrict__ work, const int* __restrict__ pexp, float* __restrict__ part1,
               float* __restrict__ part2, int* __restrict__ prog) {
    const CoilDev& c = *cd;
    if (c.sc->done) return;
    const long long wlim = c.sc->tc_wait > 0 ? c.sc->tc_wait : kTcWait;
    extern __shared__ uint8_t tc_smem[];
    const uint32_t raw = su32(tc_smem);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gbase = tc_smem + (base - raw);
    const int S = sh.stages, NA = sh.n_acc, NT = sh.NT, NR = sh.NR;
    const uint32_t pa_bytes = kT2ABytes * (uint32_t)NR, pk_bytes = kT2KBytes * (uint32_t)NR;
    const uint32_t pa_pitch = (pa_bytes + 1023u) & ~1023u, pk_pitch = (pk_bytes + 1023u) & ~1023u;
    const uint32_t sA = base;                                     // S x 32 KB table slots
    const uint32_t sPA = base + (uint32_t)S * kTcAStage;          // staged p[a]
    const uint32_t sPK = sPA + pa_pitch;                          // staged p[kb]
    const uint32_t bar_off = (uint32_t)S * kTcAStage + pa_pitch + pk_pitch;
    const uint32_t sBar = base + bar_off;
    const int nbar = kT2Bars(S, NA);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(gbase + bar_off + 8 * nbar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(gbase + bar_off + 8 * nbar + 4);
    int* xmin_s = reinterpret_cast<int*>(gbase + bar_off + 8 * nbar + 8);
    // stages each drain warp has finished (this CTA's count; one word per warp):
    // an accumulator pair is free for stage i once the least of them reaches
    // i - NA + 1 (a sum over the warps would let fast warps stand in for a slow one)
    volatile unsigned* dprog = reinterpret_cast<volatile unsigned*>(gbase + bar_off + 8 * nbar + 16);
    const int scp = (NR + 7) & ~3;
    float* inv_s = reinterpret_cast<float*>(gbase + ((bar_off + 8 * nbar + 16 + 4 * kTcEpiWarps + 15) & ~15u));
    // barriers: a_full[S], a_empty[S], pa_full, pa_empty, pk_full, pk_empty, acc_full[NA], acc_empty[NA]
    // (not waited on: the issuers read the drain warps' progress words instead, see below), mma_done
    const uint32_t a_full = sBar, a_empty = sBar + 8u * S;
    const uint32_t pa_full = sBar + 16u * S, pa_empty = pa_full + 8u, pk_full = pa_full + 16u, pk_empty = pa_full + 24u;
    const uint32_t acc_full = pa_full + 32u, acc_empty = acc_full + 8u * NA;
    const uint32_t mma_done = acc_empty + 8u * NA;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int4 wk = work[blockIdx.x];                 // stages [wk.x, wk.y), first segment wk.z
    const uint32_t acc_cols = (uint32_t)sh.acc_cols;

    if (threadIdx.x == 0) {
        for (int b = 0; b < nbar; ++b) {
            const uint32_t bar = sBar + 8u * b;
            uint32_t cnt = 1u;
            if (bar >= acc_empty && bar < acc_empty + 8u * NA) cnt = (uint32_t)kTcEpiWarps;
            else if (bar == pa_empty || bar == pk_empty || bar == mma_done) cnt = (uint32_t)kTcIssuers;
            mbar_init(bar, cnt);
        }
        *abort_flag = 0;
        *xmin_s = 1 << 30;
        for (int q = 0; q < kTcEpiWarps; ++q) dprog[q] = 0u;
        mbar_fence_init();
    }
    __syncthreads();
    if (warp == 0) {
        const int m = warp_min_exponent(pexp, NT, lane);
        if (lane == 0) *xmin_s = m;
    }
    if (warp == 1) {
        __syncwarp();
        tmem_alloc(su32(tslot), (uint32_t)sh.ncols);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(tslot);
    for (int i = threadIdx.x; i < 4 * scp; i += blockDim.x) {
        const int k = i / scp, r = i - k * scp + k, t = r - kTcPad;
        inv_s[i] = (t >= 0 && t < NT) ? ldexpf(1.f, *xmin_s - pexp[t]) : 0.f;
    }
    __syncthreads();

    if (warp == 0 && lane == 0) {
        // ---- producer: the staged copies when their combination changes, then the stage's tile
        int sa = 0, cur_a = -1, cur_kb = -1, na = 0, nk = 0;
        uint32_t pa = 0, a_used = 0, a_par = 0;
        const uint64_t pol = tc_table_policy();
        bool ok = true;
        for (int s = wk.x; s < wk.y && ok; ++s) {
            const int j = s / NT, D = s - j * NT, a = j / sh.n_kb, kb = j - a * sh.n_kb;
            if (a != cur_a) {
                ok = wait2(c, pa_empty, ((uint32_t)na & 1u) ^ 1u, abort_flag, wlim, 1, s, na);
                if (!ok) break;
                mbar_expect_tx(pa_full, pa_bytes);
                tma_load_4d(sPA, &tmB, 0, -kTcPad, 0, a * (kTcM / 8), pa_full);
                ++na;
                cur_a = a;
            }
            if (kb != cur_kb) {
                ok = wait2(c, pk_empty, ((uint32_t)nk & 1u) ^ 1u, abort_flag, wlim, 2, s, nk);
                if (!ok) break;
                mbar_expect_tx(pk_full, pk_bytes);
                tma_load_4d(sPK, &tmB64, 0, -kTcPad, 0, kb * (kTcK / 8), pk_full);
                ++nk;
                cur_kb = kb;
            }
            ok = wait2(c, a_empty + 8u * sa, pa ^ 1u, abort_flag, wlim, 3, s, sa);
            if (!ok) break;
            mbar_expect_tx(a_full + 8u * sa, kTcAStage);
            tma_load_5d_hint(sA + (uint32_t)sa * kTcAStage, &tmA, 0, a * kTcM, kb, D, 0, a_full + 8u * sa, pol);
            a_used |= 1u << sa;
            a_par = (a_par & ~(1u << sa)) | (pa << sa);
            if (prog) prog[blockIdx.x * 32 + 0] = s - wk.x + 1;
            if (++sa == S) { sa = 0; pa ^= 1u; }
        }
        // retire the copies in flight (only the latest load of a slot or a staged copy can be)
        for (int q = 0; q < S; ++q)
            if (a_used >> q & 1u) mbar_wait_final(a_full + 8u * q, a_par >> q & 1u, kTcWait);
        if (na > 0) mbar_wait_final(pa_full, (uint32_t)(na - 1) & 1u, kTcWait);
        if (nk > 0) mbar_wait_final(pk_full, (uint32_t)(nk - 1) & 1u, kTcWait);
    } else if (warp >= 1 && warp < kTcEpi0 && lane == 0) {
        // ---- MMA issuers: stage i (slot i % S, accumulator pair i % NA) by warp 1 + i % kTcIssuers;
        // every issuer follows every copy change (waits for the new copy, frees the old one)
        const int me = warp - 1;
        int cur_a = -1, cur_kb = -1, na = 0, nk = 0;
        bool ok = true;
        for (int s = wk.x, i = 0; s < wk.y && ok; ++s, ++i) {
            const int j = s / NT, D = s - j * NT, a = j / sh.n_kb, kb = j - a * sh.n_kb;
            if (a != cur_a) {
                if (cur_a >= 0) mma_commit(pa_empty);
                ok = wait2(c, pa_full, (uint32_t)na & 1u, abort_flag, wlim, 4, s, na);
                if (!ok) break;
                ++na;
                cur_a = a;
                tc_fence_after();
            }
            if (kb != cur_kb) {
                if (cur_kb >= 0) mma_commit(pk_empty);
                ok = wait2(c, pk_full, (uint32_t)nk & 1u, abort_flag, wlim, 5, s, nk);
                if (!ok) break;
                ++nk;
                cur_kb = kb;
                tc_fence_after();
            }
            if (i % kTcIssuers != me) continue;
            const int sa_i = i % S, ai = i % NA;
            const uint32_t pa_i = (uint32_t)(i / S) & 1u, pacc_i = (uint32_t)(i / NA) & 1u;
            // accumulator first: the drain of stage i - NA.  With fewer accumulator pairs
            // than issuers, stages that share a pair belong to different issuers, which can
            // run ahead of one another; a parity wait cannot tell a barrier two phases behind
            // from one that is done, so the issuers wait until every drain warp has finished
            // stage i - NA.  That implies every stage up to i - NA has finished its MMAs, so
            // (S >= NA) the previous load of this stage's slot has landed and its parity wait
            // is exact.
            if (i >= NA) {
                const unsigned need = (unsigned)(i - NA + 1);
                const long long t0 = clock64();
                for (;;) {
                    unsigned m = dprog[0];
#pragma unroll
                    for (int q = 1; q < kTcEpiWarps; ++q) m = min(m, (unsigned)dprog[q]);
                    if (m >= need) break;
                    __nanosleep(32);
                    if (*abort_flag) { ok = false; break; }
                    if (clock64() - t0 > wlim) {
                        *abort_flag = 1;
                        if (atomicCAS(&c.sc->tc_where[0], 0, 6) == 0) {
                            c.sc->tc_where[1] = blockIdx.x;
                            c.sc->tc_where[2] = s;
                            c.sc->tc_where[3] = i;
                            c.sc->tc_where[5] = threadIdx.x;
                        }
                        ok = false;
                        break;
                    }
                }
                __threadfence_block();
            }
            (void)pacc_i;
            if (ok) ok = wait2(c, a_full + 8u * sa_i, pa_i, abort_flag, wlim, 7, s, sa_i);
            if (!ok) break;
            tc_fence_after();
            const uint32_t ah = sA + (uint32_t)sa_i * kTcAStage;
            const uint32_t col0 = tmem + (uint32_t)ai * 2u * acc_cols;
            {
                // (1) y[a] += T_D[a][kb] p[kb](t - D), turns D <= t < NT, from a multiple of 8
                const int ts = D & ~7;
                const int n = (NT - ts + 15) & ~15;
                const uint64_t a_hi = sdesc(ah, 16u, 1024u, 2u);
                const uint64_t a_lo = a_hi + (((uint64_t)kTcM * 128u) >> 4);
                const uint32_t row0 = (uint32_t)(ts - D + kTcPad);
                const uint64_t b_hi = sdesc(sPK + 16u * row0, 32u * (uint32_t)NR, 128u, 0u);
                const uint64_t b_lo = b_hi + ((16u * (uint32_t)NR) >> 4);
                const uint64_t b_step = (2u * 32u * (uint32_t)NR) >> 4;
                const uint32_t idesc = idesc_f16m(n, false, kTcM);
                const uint32_t dcol = col0 + (uint32_t)ts;
#pragma unroll
                for (int k = 0; k < kTcK / 16; ++k) {
                    mma_f16(dcol, a_hi + k * (32u >> 4), b_hi + k * b_step, idesc, k > 0 ? 1u : 0u);
                    mma_f16(dcol, a_hi + k * (32u >> 4), b_lo + k * b_step, idesc, 1u);
                    mma_f16(dcol, a_lo + k * (32u >> 4), b_hi + k * b_step, idesc, 1u);
                }
            }
            if (D > 0) {
                // (2) y[kb] += T_D[a][kb]^T p[a](t + D), turns 0 <= t < NT - D; the tile read
                // MN-major (M = its 64 columns, K = its 128 rows, 8-row groups 1 KB apart)
                const int n = (NT - D + 7) & ~7;
                const uint64_t a_hi = sdesc(ah, kTcMnLbo, kTcMnSbo, 2u);
                const uint64_t a_lo = a_hi + (((uint64_t)kTcM * 128u) >> 4);
                const uint32_t row0 = (uint32_t)(D + kTcPad);
                const uint64_t b_hi = sdesc(sPA + 16u * row0, 32u * (uint32_t)NR, 128u, 0u);
                const uint64_t b_lo = b_hi + ((16u * (uint32_t)NR) >> 4);
                const uint64_t b_step = (2u * 32u * (uint32_t)NR) >> 4;
                const uint32_t idesc = idesc_f16m(n, true, kTcK);
                const uint32_t dcol = col0 + acc_cols;
#pragma unroll
                for (int k = 0; k < kTcM / 16; ++k) {
                    mma_f16(dcol, a_hi + k * (2048u >> 4), b_hi + k * b_step, idesc, k > 0 ? 1u : 0u);
                    mma_f16(dcol, a_hi + k * (2048u >> 4), b_lo + k * b_step, idesc, 1u);
                    mma_f16(dcol, a_lo + k * (2048u >> 4), b_hi + k * b_step, idesc, 1u);
                }
            }
            mma_commit(a_empty + 8u * sa_i);
            mma_commit(acc_full + 8u * ai);
            if (prog) prog[blockIdx.x * 32 + 1 + me] = i + 1;
        }
        mma_commit(mma_done);
        if (!mbar_wait_final(mma_done, 0u, kTcWait)) {
            *abort_flag = 1;
            if (atomicCAS(&c.sc->tc_where[0], 0, 9) == 0) c.sc->tc_where[1] = blockIdx.x;
        }
    } else if (warp >= kTcEpi0) {
        // ---- drain: both accumulators of every stage into FP32 registers, a partial tile
        // pair per combination
        const int q = warp & 3;
        const int h = (warp - kTcEpi0) >> 2;
        const int hf = lane >> 4;                       // (2): the half of the warp (group 2m + hf)
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        float acc1[kTcGroups][8];                       // group g = kTcParities gi + h
        float acc2[2][8];                               // group 2 (h + 4 k) + hf, kb channel 16 q + lane % 16
#pragma unroll
        for (int g = 0; g < kTcGroups; ++g)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc1[g][j] = 0.f;
#pragma unroll
        for (int g = 0; g < 2; ++g)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc2[g][j] = 0.f;
        auto flush = [&](int seg) {
            float* o1 = part1 + (size_t)seg * NT * kTcM + 32 * q + lane;
#pragma unroll
            for (int gi = 0; gi < kTcGroups; ++gi) {
                const int t0 = 8 * (kTcParities * gi + h);
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    if (t0 + jj < NT) o1[(size_t)(t0 + jj) * kTcM] = acc1[gi][jj];
                    acc1[gi][jj] = 0.f;
                }
            }
            float* o2 = part2 + (size_t)seg * NT * kTcK + 16 * q + (lane & 15);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int t0 = 8 * (2 * (h + 4 * k) + hf);
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    if (t0 + jj < NT) o2[(size_t)(t0 + jj) * kTcK] = acc2[k][jj];
                    acc2[k][jj] = 0.f;
                }
            }
        };
        int ai = 0, cur_j = -1, seg = wk.z - 1;
        uint32_t pf = 0;
        bool ok = true;
        for (int s = wk.x; s < wk.y && ok; ++s) {
            const int j = s / NT, D = s - j * NT;
            if (j != cur_j) {
                if (cur_j >= 0) flush(seg);
                cur_j = j;
                ++seg;
            }
            ok = __all_sync(0xffffffffu, wait2(c, acc_full + 8u * ai, (pf >> ai) & 1u, abort_flag, wlim, 8, s, ai));
            if (!ok) break;
            pf ^= 1u << ai;
            tc_fence_after();
            const uint32_t src1 = lane_base + (uint32_t)ai * 2u * acc_cols;
            const int g_lo = D >> 3, g_hi = (NT + 7) >> 3;
#pragma unroll
            for (int gi = 0; gi < kTcGroups; ++gi) {
                const int g = kTcParities * gi + h;
                if (g >= g_lo && g < g_hi) {
                    float v[8];
                    tmem_ld8(src1 + 8u * (uint32_t)g, v);
                    scale_add8(inv_s, scp, 8 * g + kTcPad - D, v, acc1[gi]);
                }
            }
            if (D > 0) {
                const uint32_t src2 = src1 + acc_cols;
                const int g_hi2 = (NT - D + 7) >> 3;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int g0 = 2 * (h + 4 * k);             // this pair's first group (warp-uniform)
                    if (g0 < g_hi2) {
                        float v[8];
                        tmem_ld16x2_8(src2 + 8u * (uint32_t)g0, v);
                        const int g = g0 + hf;
                        if (g < g_hi2) scale_add8(inv_s, scp, 8 * g + kTcPad + D, v, acc2[k]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                dprog[warp - kTcEpi0] = (unsigned)(s - wk.x + 1);
            }
            if (prog && lane == 0) prog[blockIdx.x * 32 + 8 + (warp - kTcEpi0)] = s - wk.x + 1;
            if (++ai == NA) ai = 0;
        }
        if (ok && !*abort_flag && cur_j >= 0) flush(seg);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0 && *abort_flag) {
        atomicExch(&c.sc->status, (int)ST_KERNEL);
        atomicExch(&c.sc->done, 1);
    }
    if (warp == 1) {
        __syncwarp();
        tmem_dealloc(tmem, (uint32_t)sh.ncols);
    }
}

// ---------------------------------------------------------------------------
// Input split, reduction, table
// ---------------------------------------------------------------------------
__device__ __forceinline__ float block_max_f(float v) {
    __shared__ float sm[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sm[w] = v;
    __syncthreads();
    if (w == 0) {
        v = l < (int)(blockDim.x >> 5) ? sm[l] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (l == 0) sm[0] = v;
    }
    __syncthreads();
    return sm[0];
}

// Power-of-two exponent that brings a maximum m below 2^14 (0 if m is zero,
// not finite or not a number).
__host__ __device__ inline int tc_exponent(double m) {
    if (!(m > 0.0) || !(m < 1.0e300)) return 0;
    int e = 0;
    frexp(m, &e);                  // m < 2^e
    int x = 14 - e;
    return x > 120 ? 120 : (x < -120 ? -120 : x);
}

// p -> FP16 hi/lo in [c'/8][hi, lo][t][c' % 8] order; one block per turn row t,
// scaled by 2^pexp[t] so that the row's largest |p| lies below 2^14.  dir: p is
// the PCG's next search direction, formed here first (from the second
// iteration on), d = -z + beta d (FP64 into d, FP32 into the input copy), in
// place of a separate pass.
__device__ __forceinline__ void tc_split_row(const CoilDev& c, const TcShape& sh, __half* __restrict__ p16,
                                             int* __restrict__ pexp, int dir, const int t) {
    if (c.sc->done) return;
    float* row = c.pf + (size_t)t * sh.C;
    constexpr int kReg = 8;                      // entries per thread kept in registers
    if (sh.Cp <= kReg * (int)blockDim.x) {
        // the row in registers: one pass over memory (d, then its maximum and split)
        const bool form = dir && c.sc->iter > 0;  // the first iteration's direction is k_init's
        const double beta = form ? c.sc->beta : 0.0;
        const size_t e0 = (size_t)t * sh.C;
        float v[kReg];
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < kReg; ++k) {
            const int cc = threadIdx.x + k * (int)blockDim.x;
            float f = 0.f;
            if (cc < sh.C) {
                if (form) {
                    const double d = -c.zv[e0 + cc] + beta * c.dv[e0 + cc];
                    c.dv[e0 + cc] = d;
                    f = (float)d;
                    row[cc] = f;
                } else {
                    f = row[cc];
                }
            }
            v[k] = f;
            m = fmaxf(m, fabsf(f));
        }
        const int x = tc_exponent((double)block_max_f(m));
        if (threadIdx.x == 0) pexp[t] = x;
        const float s = ldexpf(1.f, x);
#pragma unroll
        for (int k = 0; k < kReg; ++k) {
            const int cc = threadIdx.x + k * (int)blockDim.x;
            if (cc < sh.Cp) {
                const float sv = cc < sh.C ? v[k] * s : 0.f;
                const __half hi = __float2half_rn(sv);
                const int idx = (((cc >> 3) * 2) * sh.NT + t) * 8 + (cc & 7);
                p16[idx] = hi;
                p16[idx + 8 * sh.NT] = __float2half_rn(sv - __half2float(hi));
            }
        }
        return;
    }
    if (dir && c.sc->iter > 0) {                 // the first iteration's direction is k_init's
        const double beta = c.sc->beta;
        const size_t e0 = (size_t)t * sh.C;
        for (int cc = threadIdx.x; cc < sh.C; cc += blockDim.x) {
            const double d = -c.zv[e0 + cc] + beta * c.dv[e0 + cc];
            c.dv[e0 + cc] = d;
            row[cc] = (float)d;
        }
        __syncthreads();
    }
    float m = 0.f;
    for (int cc = threadIdx.x; cc < sh.C; cc += blockDim.x) m = fmaxf(m, fabsf(row[cc]));
    const int x = tc_exponent((double)block_max_f(m));
    if (threadIdx.x == 0) pexp[t] = x;
    const float s = ldexpf(1.f, x);
    for (int cc = threadIdx.x; cc < sh.Cp; cc += blockDim.x) {
        const float v = cc < sh.C ? row[cc] * s : 0.f;
        const __half hi = __float2half_rn(v);
        const int idx = (((cc >> 3) * 2) * sh.NT + t) * 8 + (cc & 7);
        p16[idx] = hi;
        p16[idx + 8 * sh.NT] = __float2half_rn(v - __half2float(hi));
    }
}

__global__ void k_tc_split(const CoilDev* __restrict__ cd, const TcShape sh, __half* __restrict__ p16,
                           int* __restrict__ pexp, int dir) {
    tc_split_row(*cd, sh, p16, pexp, dir, (int)blockIdx.x);
}

// A batch's input splits in one launch: block (t, coil).
__global__ void k_tc_split_batch(const TcCoilArgs* __restrict__ args, int dir) {
    const TcCoilArgs& A = args[blockIdx.y];
    if ((int)blockIdx.x >= A.sh.NT) return;
    tc_split_row(*A.d, A.sh, A.p16, A.pexp, dir, (int)blockIdx.x);
}

// q[e] = 2^-(exT + xmin) x the sum of the partial tiles of the CTAs that
// worked on e's channel tile (fixed order, FP64; the loads of eight tiles are
// issued before their sums).  range[ct] = (first CTA, number of CTAs).
__device__ __forceinline__ void tc_reduce_body(const CoilDev& c, const TcShape& sh, const float* __restrict__ part,
                                               const int2* __restrict__ range, const int* __restrict__ pexp,
                                               int exT) {
    if (c.sc->done) return;
    const double inv = ldexp(1.0, -(exT + warp_min_exponent(pexp, sh.NT, threadIdx.x & 31)));
    const size_t tile = (size_t)sh.NT * kTcM;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < sh.N; e += gridDim.x * blockDim.x) {
        const int t = e / sh.C, cc = e - t * sh.C;
        const int2 rg = range[cc / kTcM];
        const float* p = part + (size_t)rg.x * tile + (size_t)t * kTcM + (cc % kTcM);
        double s = 0.0;
        int k = 0;
        for (; k + 8 <= rg.y; k += 8) {
            float v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = p[(size_t)(k + i) * tile];
#pragma unroll
            for (int i = 0; i < 8; ++i) s += (double)v[i];
        }
        for (; k < rg.y; ++k) s += (double)p[(size_t)k * tile];
        c.qv[e] = s * inv;
    }
}

__global__ void k_tc_reduce(const CoilDev* __restrict__ cd, const TcShape sh, const float* __restrict__ part,
                            const int2* __restrict__ range, const int* __restrict__ pexp, int exT) {
    tc_reduce_body(*cd, sh, part, range, pexp, exT);
}

// A batch's reductions into q (coils whose near kernel does not sum the
// partial tiles itself, or all of them with need_q): grid row = coil.
__global__ void k_tc_reduce_batch(const TcCoilArgs* __restrict__ args, int need_q) {
    const TcCoilArgs& A = args[blockIdx.y];
    if (!need_q && !A.write_q) return;
    tc_reduce_body(*A.d, A.sh, A.part, A.range, A.pexp, A.exT);
}

// Mode 1: q[e] = 2^-(exT + xmin) x (the part1 segments of e's channel tile +
// the part2 segments of e's k block), fixed order, FP64.
// The one-fill apply's reduction into q: element e sums its channel tile's
// segments of the T_d products and its k block's segments of the T_d^T
// products.  A CTA takes 32 consecutive elements; its 8 warps take every 8th
// segment of both lists (lanes = elements, so every load is coalesced), and
// warp 0 adds the 8 sums in order: the result is deterministic, and an
// element's chain of dependent loads is an eighth of its segment count.
constexpr int kT2RedSplit = 8;
__global__ void __launch_bounds__(32 * kT2RedSplit)
k_tc2_reduce(const CoilDev* __restrict__ cd, const TcShape sh, const float* __restrict__ part1,
             const float* __restrict__ part2, const int2* __restrict__ l1, const int* __restrict__ segs1,
             const int2* __restrict__ l2, const int* __restrict__ segs2, const int* __restrict__ pexp, int exT) {
    const CoilDev& c = *cd;
    if (c.sc->done) return;
    __shared__ double sums[kT2RedSplit][32];
    const int lane = threadIdx.x & 31, j = threadIdx.x >> 5;
    const double inv = ldexp(1.0, -(exT + warp_min_exponent(pexp, sh.NT, lane)));
    const size_t t1 = (size_t)sh.NT * kTcM, t2 = (size_t)sh.NT * kTcK;
    for (int e0 = blockIdx.x * 32; e0 < sh.N; e0 += gridDim.x * 32) {
        const int e = e0 + lane;
        double s = 0.0;
        if (e < sh.N) {
            const int t = e / sh.C, cc = e - t * sh.C;
            const int2 r1 = l1[cc / kTcM], r2 = l2[cc / kTcK];
            const float* p1 = part1 + (size_t)t * kTcM + (cc % kTcM);
            const float* p2 = part2 + (size_t)t * kTcK + (cc % kTcK);
            for (int k = j; k < r1.y; k += kT2RedSplit) s += (double)p1[(size_t)segs1[r1.x + k] * t1];
            for (int k = j; k < r2.y; k += kT2RedSplit) s += (double)p2[(size_t)segs2[r2.x + k] * t2];
        }
        sums[j][lane] = s;
        __syncthreads();
        if (j == 0 && e < sh.N) {
            double q = 0.0;
#pragma unroll
            for (int i = 0; i < kT2RedSplit; ++i) q += sums[i][lane];
            c.qv[e] = q * inv;
        }
        __syncthreads();
    }
}

__global__ void k_tc_absmax(const double* __restrict__ tab, long long n, double* __restrict__ out) {
    double m = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmax(m, fabs(tab[i]));
    m = warp_max(m);
    __shared__ double sm[32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sm[w]);
        out[blockIdx.x] = m;
    }
}

// FP64 table [offset + NT - 1][c][c'] -> FP16 hi/lo [half][offset][k block][c][64]
// for offsets 0 .. NT - 1 only (T_{-d} = T_d^T is read transposed), c' = 64 k
// block + column, scaled by 2^exT, so that the 128 x 64 tile of one stage is a
// contiguous 16 KB per half; intra-wire entries of offset 0 are zero (applied
// from the FP64 near blocks), padding columns c' >= C zero.
__global__ void k_tc_table(const double* __restrict__ tab, const TcShape sh, int wire_div, int exT,
                           __half* __restrict__ t16) {
    const long long total = (long long)sh.NT * sh.n_kb * sh.C * kTcK;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int kk = (int)(idx % kTcK);
        const long long rest = idx / kTcK;
        const int ci = (int)(rest % sh.C);
        const long long rest2 = rest / sh.C;
        const int cj = (int)(rest2 % sh.n_kb) * kTcK + kk;
        const int dd = (int)(rest2 / sh.n_kb);
        double v = cj < sh.C ? tab[((long long)(dd + sh.NT - 1) * sh.C + ci) * sh.C + cj] : 0.0;
        if (dd == 0 && ci / wire_div == cj / wire_div) v = 0.0;
        v = ldexp(v, exT);
        const __half hi = __double2half(v);
        t16[idx] = hi;
        t16[total + idx] = __double2half(v - (double)__half2float(hi));
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
size_t tc_smem_bytes(const TcShape& sh) {
    if (sh.mode == 1) {
        const size_t pa = ((size_t)kT2ABytes * sh.NR + 1023) & ~(size_t)1023;
        const size_t pk = ((size_t)kT2KBytes * sh.NR + 1023) & ~(size_t)1023;
        return 1024 + (size_t)sh.stages * kTcAStage + pa + pk + 8 * (size_t)kT2Bars(sh.stages, sh.n_acc) + 32 +
               4 * kTcEpiWarps +
               16 * (size_t)((sh.NR + 7) & ~3);
    }
    size_t b_pitch = ((size_t)512 * sh.NR + 127) & ~(size_t)127;
    return 1024 + kTcBStages * b_pitch + (size_t)sh.stages * kTcAStage + 8 * (size_t)kTcBars(sh.stages) + 32 +
           16 * (size_t)((sh.NR + 7) & ~3);
}

bool tc_shape(int C, int NT, int n_sm, TcShape* sh) {
    if (C < 1 || NT < 1 || NT > kTcMaxTurns) return false;
    TcShape s{};
    s.C = C;
    s.Cp = (C + 7) & ~7;
    s.NT = NT;
    s.NR = NT + kTcPad + kTcPadTop;
    s.N = C * NT;
    s.n_ct = (C + kTcM - 1) / kTcM;
    s.n_kb = (s.Cp + kTcK - 1) / kTcK;
    s.n_cta = (int)tc_schedule(s, n_sm, nullptr, nullptr);
    int used = (NT + 15) & ~7;        // an MMA's columns end before NT + 15
    s.acc_cols = 32;
    while (s.acc_cols < used) s.acc_cols *= 2;
    s.n_acc = 512 / s.acc_cols > 4 ? 4 : 512 / s.acc_cols;   // 2..4 accumulators in 512 columns
    s.ncols = s.n_acc * s.acc_cols;
    const size_t limit = kTcSmemLimit;
    s.stages = 6;                      // up to 192 KB of table copies in flight per SM
    while (s.stages > 2 && tc_smem_bytes(s) > limit) --s.stages;
    if (tc_smem_bytes(s) > limit) return false;
    // the issuers' slot waits rely on stages >= accumulators (see the MMA loop)
    if (s.n_acc > s.stages) {
        s.n_acc = s.stages;
        s.ncols = 32;
        while (s.ncols < s.n_acc * s.acc_cols) s.ncols *= 2;
    }
    *sh = s;
    return true;
}

bool tc2_shape(int C, int NT, int n_sm, int n_cta, int stages, TcShape* sh) {
    if (C < 1 || NT < 1 || NT > kTcMaxTurns) return false;
    TcShape s{};
    s.mode = 1;
    s.C = C;
    s.Cp = (C + 7) & ~7;
    s.NT = NT;
    s.NR = NT + kTcPad + kTcPadTop;
    s.N = C * NT;
    s.n_ct = (C + kTcM - 1) / kTcM;
    s.n_kb = (s.Cp + kTcK - 1) / kTcK;
    s.n_combo = s.n_ct * s.n_kb;
    const long long total = (long long)s.n_combo * NT;
    long long ctas = n_cta > 0 ? n_cta : std::min<long long>(n_sm, std::max<long long>(1, total / kT2MinStages));
    s.n_cta = (int)std::max<long long>(1, std::min<long long>(ctas, total));
    int used = (NT + 15) & ~7;        // an MMA's columns end before NT + 15
    s.acc_cols = 32;
    while (s.acc_cols < used) s.acc_cols *= 2;
    s.n_acc = 512 / (2 * s.acc_cols) > 4 ? 4 : 512 / (2 * s.acc_cols);   // accumulator pairs
    if (s.n_acc < 1) return false;
    s.ncols = 32;
    while (s.ncols < 2 * s.n_acc * s.acc_cols) s.ncols *= 2;
    const size_t limit = kTcSmemLimit;
    s.stages = stages > 0 ? stages : 6;
    while (s.stages > 2 && tc_smem_bytes(s) > limit) --s.stages;
    if (tc_smem_bytes(s) > limit) return false;
    if (s.n_acc > s.stages) {          // the issuers' slot waits rely on stages >= accumulators
        s.n_acc = s.stages;
        s.ncols = 32;
        while (s.ncols < 2 * s.n_acc * s.acc_cols) s.ncols *= 2;
    }
    *sh = s;
    return true;
}

// Equal contiguous ranges of the (a, kb, D) stage order; a CTA's range gets a
// segment per combination it touches (consecutive segment numbers), and every
// segment is listed under its channel tile (l1/segs1, the products (1)) and
// its k block (l2/segs2, the transposed products (2)), in segment order.
size_t tc2_schedule(TcShape* sh, std::vector<int4>* work, std::vector<int2>* l1, std::vector<int>* segs1,
                    std::vector<int2>* l2, std::vector<int>* segs2) {
    const long long NT = sh->NT, total = (long long)sh->n_combo * NT;
    const long long n = sh->n_cta;
    std::vector<std::vector<int>> by_a(sh->n_ct), by_kb(sh->n_kb);
    work->clear();
    int seg = 0;
    for (long long i = 0; i < n; ++i) {
        const long long s0 = total * i / n, s1 = total * (i + 1) / n;
        work->push_back(make_int4((int)s0, (int)s1, seg, 0));
        if (s1 <= s0) continue;
        for (long long j = s0 / NT; j <= (s1 - 1) / NT; ++j) {
            by_a[j / sh->n_kb].push_back(seg);
            by_kb[j % sh->n_kb].push_back(seg);
            ++seg;
        }
    }
    sh->n_seg = seg;
    l1->clear();
    l2->clear();
    segs1->clear();
    segs2->clear();
    for (auto& v : by_a) {
        l1->push_back(make_int2((int)segs1->size(), (int)v.size()));
        segs1->insert(segs1->end(), v.begin(), v.end());
    }
    for (auto& v : by_kb) {
        l2->push_back(make_int2((int)segs2->size(), (int)v.size()));
        segs2->insert(segs2->end(), v.begin(), v.end());
    }
    return (size_t)n;
}

// The same number of CTAs for every channel tile (n_sm / n_ct, at least one,
// at most one per step, and beyond four at most one per eight steps).  Tile ct's j-th CTA and tile cb's j-th CTA meet the
// 128 x 128 region (ct, cb) of every stored offset block at about the same
// time, one of them reading it transposed, so the region comes from DRAM
// once.  A tile's n_ct NT steps are split into contiguous ranges of about
// equal stage counts (a step has 2 stages per k block of its column tile, 1
// for D = 0; the half-height last column tile has one k block; a stage's cost
// is mostly its issue, nearly independent of its turns); every tile has the
// same total, so partner CTAs stay within a fraction of a range of each
// other.  work[cta] = (tile, first step, end step, 0); range[tile] = (first
// CTA, CTAs).  Returns the number of CTAs.
size_t tc_schedule(const TcShape& sh, int n_sm, std::vector<int4>* work, std::vector<int2>* range) {
    const long long steps = (long long)sh.n_ct * sh.NT;
    long long per = n_sm / sh.n_ct;
    if (per < 1) per = 1;
    if (per > steps) per = steps;
    // at least kTcMinSteps steps per CTA beyond kTcMinCtas CTAs per tile: a
    // small coil's apply then takes a few SMs, not one CTA per SM with a step
    // or two each, so a batch's applies on the side streams run side by side;
    // the kTcMinCtas floor keeps each CTA's FP32 register sums short
    const long long min_steps = sh.min_steps > 0 ? sh.min_steps : kTcMinSteps;
    const long long cap = std::max(std::min(per, kTcMinCtas), steps / min_steps);
    if (per > cap) per = cap;
    if (work && range) {
        work->clear();
        range->clear();
        for (int ct = 0; ct < sh.n_ct; ++ct) {
            range->push_back(make_int2((int)work->size(), (int)per));
            std::vector<long long> cum(steps + 1, 0);
            for (long long sg = 0; sg < steps; ++sg) {
                const int D = (int)(sg % sh.NT), cb = (int)((sg / sh.NT - ct + sh.n_ct) % sh.n_ct);
                const int nk = std::min(2, sh.n_kb - 2 * cb);
                cum[sg + 1] = cum[sg] + nk * (D > 0 ? 2 : 1);
            }
            long long s0 = 0;
            for (long long i = 0; i < per; ++i) {
                long long s1 = s0;
                const long long target = cum[steps] * (i + 1) / per;
                const long long s_max = steps - (per - 1 - i);      // leave a step for every later CTA
                while (s1 < s_max && (cum[s1 + 1] <= target || s1 == s0)) ++s1;
                if (i == per - 1) s1 = steps;
                work->push_back(make_int4(ct, (int)s0, (int)s1, 0));
                s0 = s1;
            }
        }
    }
    return (size_t)(per * sh.n_ct);
}

size_t tc_table_halves(const TcShape& sh) { return 2 * (size_t)sh.NT * sh.n_kb * sh.C * kTcK; }

cudaError_t tc_build_table(TcPlan* P, const double* tab, int wire_div, double* scratch, cudaStream_t s) {
    const TcShape& sh = P->sh;
    long long n = (long long)(2 * sh.NT - 1) * sh.C * sh.C;
    const int nb = 512;
    k_tc_absmax<<<nb, 256, 0, s>>>(tab, n, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double hm[nb];
    e = cudaMemcpyAsync(hm, scratch, sizeof(hm), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    double m = 0.0;
    for (int i = 0; i < nb; ++i) m = hm[i] > m ? hm[i] : m;
    P->exT = tc_exponent(m);
    long long total = (long long)sh.NT * sh.n_kb * sh.C * kTcK;
    long long blocks = (total + 255) / 256;
    if (blocks > 148LL * 64) blocks = 148LL * 64;
    k_tc_table<<<(unsigned)blocks, 256, 0, s>>>(tab, sh, wire_div, P->exT, P->t16);
    return cudaGetLastError();
}

namespace {
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}
}  // namespace

cudaError_t tc_encode_maps(TcPlan* P, const char** why) {
    EncodeTiled enc = encoder();
    if (!enc) {
        *why = "cuTensorMapEncodeTiled is not available from the driver";
        return cudaErrorNotSupported;
    }
    const TcShape& sh = P->sh;
    const cuuint32_t ones[5] = {1, 1, 1, 1, 1};
    {
        // [half][offset >= 0][k block][c][64]: tmA's box is one stage's 128 x 64 tile
        // (rows c, columns c') of both halves; tmAT's box is the 64 x 128 tile of
        // the transposed block (rows c' of one k block, columns c of two k blocks)
        const cuuint64_t row = (cuuint64_t)kTcK * 2;
        const cuuint64_t dims[5] = {(cuuint64_t)kTcK, (cuuint64_t)sh.C, (cuuint64_t)sh.n_kb, (cuuint64_t)sh.NT, 2};
        const cuuint64_t strides[4] = {row, row * sh.C, row * sh.C * sh.n_kb, row * sh.C * sh.n_kb * sh.NT};
        const cuuint32_t box[5] = {(cuuint32_t)kTcK, (cuuint32_t)kTcM, 1, 1, 2};
        const cuuint32_t boxT[5] = {(cuuint32_t)kTcK, (cuuint32_t)kTcK, (cuuint32_t)(kTcM / kTcK), 1, 2};
        CUresult r = enc(&P->tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 5, P->t16, dims, strides, box, ones,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r == CUDA_SUCCESS)
            r = enc(&P->tmAT, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 5, P->t16, dims, strides, boxT, ones,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            *why = "encoding the table tensor map failed";
            return cudaErrorInvalidValue;
        }
    }
    {
        // [c'/8][hi, lo][NT turn rows][8]: box = the staged copy of a column tile,
        // turn rows -kTcPad .. NT + kTcPadTop - 1 (zero fill outside the winding)
        const cuuint64_t dims[4] = {8, (cuuint64_t)sh.NT, 2, (cuuint64_t)(sh.Cp / 8)};
        const cuuint64_t strides[3] = {16, (cuuint64_t)sh.NT * 16, 2 * (cuuint64_t)sh.NT * 16};
        const cuuint32_t box[4] = {8, (cuuint32_t)sh.NR, 2, (cuuint32_t)(kTcM / 8)};
        CUresult r = enc(&P->tmB, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4, P->p16, dims, strides, box, ones,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        // the one-fill apply's p[kb]: 64 channels (8 chunks) per box
        const cuuint32_t box64[4] = {8, (cuuint32_t)sh.NR, 2, (cuuint32_t)(kTcK / 8)};
        if (r == CUDA_SUCCESS)
            r = enc(&P->tmB64, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4, P->p16, dims, strides, box64, ones,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            *why = "encoding the input tensor map failed";
            return cudaErrorInvalidValue;
        }
    }
    // the attribute belongs to the kernel, not to the coil: set the largest size
    // any coil may take, so that every coil's launch fits
    cudaError_t e = cudaFuncSetAttribute(k_toeplitz_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_toeplitz_tc2, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemLimit);
    if (e != cudaSuccess) *why = "setting the shared-memory size of the tensor-core apply failed";
    return e;
}

cudaError_t launch_tc_split(const TcPlan& P, cudaStream_t s, bool dir) {
    k_tc_split<<<P.sh.NT, 256, 0, s>>>(P.d, P.sh, P.p16, P.pexp, dir ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_tc_apply(const TcPlan& P, cudaStream_t s, bool write_q, const double* near_src, double* near_dst) {
    const TcShape& sh = P.sh;
    if (sh.mode == 1) {
        k_toeplitz_tc2<<<sh.n_cta, kTcThreads, P.smem, s>>>(P.tmA, P.tmB, P.tmB64, P.d, sh, P.work, P.pexp, P.part,
                                                             P.part2, P.prog);
        if (write_q) {
            int rb = (sh.N + 31) / 32;
            if (rb > 148 * 16) rb = 148 * 16;
            k_tc2_reduce<<<rb, 32 * kT2RedSplit, 0, s>>>(P.d, sh, P.part, P.part2, P.l1, P.segs1, P.l2, P.segs2,
                                                       P.pexp, P.exT);
        }
        return cudaGetLastError();
    }
    k_toeplitz_tc<<<sh.n_cta, kTcThreadsNear, P.smem, s>>>(P.tmA, P.tmAT, P.tmB, P.d, sh, P.work, P.pexp, P.part,
                                                        near_src, near_dst);
    if (write_q) {
        int rb = (sh.N + 255) / 256;
        if (rb > 148 * 8) rb = 148 * 8;
        k_tc_reduce<<<rb, 256, 0, s>>>(P.d, sh, P.part, P.range, P.pexp, P.exT);
    }
    return cudaGetLastError();
}

cudaError_t tc_batch_build(TcBatch* B, const std::vector<const TcPlan*>& plans, cudaStream_t s) {
    tc_batch_free(B);
    std::vector<TcCoilArgs> args(plans.size());
    std::vector<int2> bwork;
    B->n = (int)plans.size();
    B->smem = 0;
    B->maxNT = B->maxN = 0;
    for (size_t i = 0; i < plans.size(); ++i) {
        const TcPlan& P = *plans[i];
        if (P.sh.mode != 0) return cudaErrorInvalidValue;     // batches run the two-fill apply
        TcCoilArgs& A = args[i];
        A.tmA = P.tmA;
        A.tmAT = P.tmAT;
        A.tmB = P.tmB;
        A.sh = P.sh;
        A.d = P.d;
        A.work = P.work;
        A.range = P.range;
        A.pexp = P.pexp;
        A.part = P.part;
        A.p16 = P.p16;
        A.exT = P.exT;
        A.write_q = P.fused ? 0 : 1;
        for (int k = 0; k < P.sh.n_cta; ++k) bwork.push_back(make_int2((int)i, k));
        B->smem = std::max(B->smem, P.smem);
        B->maxNT = std::max(B->maxNT, P.sh.NT);
        B->maxN = std::max(B->maxN, P.sh.N);
    }
    B->n_cta = (int)bwork.size();
    cudaError_t e = cudaMalloc(&B->args, args.size() * sizeof(TcCoilArgs));
    if (e == cudaSuccess) e = cudaMalloc(&B->work, bwork.size() * sizeof(int2));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->args, args.data(), args.size() * sizeof(TcCoilArgs), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->work, bwork.data(), bwork.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_toeplitz_tc_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemLimit);
    if (e != cudaSuccess) tc_batch_free(B);
    return e;
}

void tc_batch_free(TcBatch* B) {
    if (B->args) cudaFree(B->args);
    if (B->work) cudaFree(B->work);
    B->args = nullptr;
    B->work = nullptr;
    B->n = B->n_cta = 0;
}

cudaError_t launch_tc_batch(const TcBatch& B, cudaStream_t s, bool need_q, bool dir) {
    k_tc_split_batch<<<dim3((unsigned)B.maxNT, (unsigned)B.n), 256, 0, s>>>(B.args, dir ? 1 : 0);
    k_toeplitz_tc_batch<<<(unsigned)B.n_cta, kTcThreads, B.smem, s>>>(B.args, B.work);
    int rb = (B.maxN + 255) / 256;
    if (rb > 148 * 8) rb = 148 * 8;
    k_tc_reduce_batch<<<dim3((unsigned)rb, (unsigned)B.n), 256, 0, s>>>(B.args, need_q ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_toeplitz_tc(const TcPlan& P, cudaStream_t s, bool write_q, bool dir, const double* near_src,
                               double* near_dst) {
    cudaError_t e = launch_tc_split(P, s, dir);
    return e == cudaSuccess ? launch_tc_apply(P, s, write_q, near_src, near_dst) : e;
}

}  // namespace cq
