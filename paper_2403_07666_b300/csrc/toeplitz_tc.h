// Host-side plan of the tensor-core block-Toeplitz apply (one per coil).
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

#include "common.cuh"

namespace cq {

// Sizes of one coil's tensor-core apply (all fixed at setup).
struct TcShape {
    int C, Cp, NT, NR;          // channels per turn row, C rounded up to 8, turn rows, staged p rows
    int N;                      // elements (NT C)
    int n_ct, n_kb;             // 128-channel tiles, 64-channel k blocks
    int n_cta;                  // CTAs of the apply (see tc_schedule)
    int stages;                 // table tiles in flight per CTA
    int acc_cols, n_acc;        // TMEM columns per accumulator, accumulators (stages alternate)
    int ncols;                  // TMEM columns allocated per CTA (n_acc acc_cols)
    // mode 1 (one-fill apply, k_toeplitz_tc2): work units (channel tile, k block),
    // n_acc counts accumulator pairs, n_seg partial-tile segments in all
    int mode;
    int n_combo, n_seg;
    int min_steps;              // mode 0: schedule steps per CTA at least beyond a few CTAs per tile
                                // (0: the default; 1: one CTA per SM and channel tile share)
};

struct TcPlan {
    CUtensorMap tmA;            // split table: [half][offset >= 0][c'/64][c][c' % 64] FP16, 128-byte swizzle
    CUtensorMap tmAT;           // the same table, transposed-tile boxes (offsets < 0)
    CUtensorMap tmB;            // split input: [c'/8][hi, lo][t][c' % 8] FP16, no swizzle
    CUtensorMap tmB64;          // the same input, 64-channel boxes (mode 1)
    TcShape sh;
    const CoilDev* d = nullptr; // device descriptor of the coil
    __half* t16 = nullptr;      // 2 NT n_kb C 64
    __half* p16 = nullptr;      // 2 Cp NT
    float* part = nullptr;      // n_cta x NT x 128 partial tiles (mode 1: n_seg x NT x 128)
    float* part2 = nullptr;     // mode 1: n_seg x NT x 64 partial tiles of the transposed products
    int2* l1 = nullptr;         // mode 1: per channel tile (first, count) into segs1
    int2* l2 = nullptr;         // mode 1: per k block (first, count) into segs2
    int* segs1 = nullptr;
    int* segs2 = nullptr;
    int* prog = nullptr;        // mode 1: progress per CTA (32 ints: producer, issuers, drain warps),
                                // read back when a bounded wait ran out
    std::vector<void*> sched_bufs;   // device buffers of the current schedule
    size_t sched_bytes = 0;
    struct Tuned { int mode, n_cta, stages; double us; };
    std::vector<Tuned> tuned;   // the autotuner's candidates and their measured apply time
    double tuned_us = 0.0;      // the chosen schedule's apply time
    TcShape tuned_sh{};         // the autotuner's choice for this coil alone
    bool in_batch = false;      // the schedule is the batched steps' one (tuned_sh restored when stepped alone)
    int4* work = nullptr;       // n_cta (tile, first stage, end stage, 0)
    int2* range = nullptr;      // n_ct (first CTA, CTAs)
    int* pexp = nullptr;        // NT input scale exponents (one per turn row)
    int exT = 0;                // table scale 2^exT
    size_t smem = 0;            // dynamic shared memory per CTA
    bool fused = false;         // the coil's near kernel sums the partial tiles itself
};

// One coil's arguments of a batched apply (device memory; the tensor maps
// must sit on 64-byte boundaries).
struct alignas(64) TcCoilArgs {
    CUtensorMap tmA, tmAT, tmB;
    TcShape sh;
    const CoilDev* d;
    const int4* work;
    const int2* range;
    int* pexp;
    float* part;
    __half* p16;
    int exT;
    int write_q;                // the reduction into q is this coil's (its near kernel does not sum tiles)
};

// The applies of a batch of coils as one launch of each kernel (split, apply,
// reduction): every coil with its own two-fill schedule, the CTAs of all
// coils in one grid.
struct TcBatch {
    TcCoilArgs* args = nullptr;
    int2* work = nullptr;       // per CTA: (coil, the coil's CTA index)
    int n = 0, n_cta = 0, maxNT = 0, maxN = 0;
    size_t smem = 0;
};

constexpr int kTcMaxTurns = 112;   // the staged copy's 2 (NT + 16) rows fit one TMA box (<= 256)

// Fill the shape for C channels, NT turns on n_sm SMs; false if unsupported.
bool tc_shape(int C, int NT, int n_sm, TcShape* sh);
// The same for the one-fill apply (mode 1); n_cta = 0: the default CTA count.
bool tc2_shape(int C, int NT, int n_sm, int n_cta, int stages, TcShape* sh);
// Its schedule: work[cta] = (first stage, end stage, first segment, 0) and the
// reduction lists; fills sh->n_seg.  Returns the number of CTAs.
size_t tc2_schedule(TcShape* sh, std::vector<int4>* work, std::vector<int2>* l1, std::vector<int>* segs1,
                    std::vector<int2>* l2, std::vector<int>* segs2);
size_t tc_table_halves(const TcShape& sh);
// CTA schedule of the apply; fills work/range when both are non-null.
size_t tc_schedule(const TcShape& sh, int n_sm, std::vector<int4>* work, std::vector<int2>* range);
size_t tc_smem_bytes(const TcShape& sh);

// Split the FP64 table (with intra-wire entries of offset 0 zeroed) into the
// FP16 hi/lo table; `scratch` holds at least 1024 doubles.  Synchronizes s.
cudaError_t tc_build_table(TcPlan* P, const double* tab, int wire_div, double* scratch, cudaStream_t s);
// Encode the two tensor maps (after t16 and p16 are allocated).
cudaError_t tc_encode_maps(TcPlan* P, const char** why);
// M_far p for the coil of P (from pf): the split, the apply into the partial
// tiles and, with write_q, their reduction into qv (otherwise the coil's
// shared-warp near kernel sums the tiles).  near_src / near_dst (two-fill,
// wires of at most 16 elements): the apply's near warps also form the
// near-block part of q, with dt G p, from near_src into near_dst.
// dir: form the PCG direction d = -z + beta d in the input split first.
cudaError_t launch_toeplitz_tc(const TcPlan& P, cudaStream_t s, bool write_q, bool dir = false,
                               const double* near_src = nullptr, double* near_dst = nullptr);
// Its two halves: the input split (k_tc_split) and the tensor-core product
// (k_toeplitz_tc, plus the FP64 reduction into q when write_q).
cudaError_t launch_tc_split(const TcPlan& P, cudaStream_t s, bool dir);
cudaError_t launch_tc_apply(const TcPlan& P, cudaStream_t s, bool write_q, const double* near_src = nullptr,
                            double* near_dst = nullptr);
// Batches: build (uploads the coils' arguments; every plan in the two-fill
// mode), free, and launch split + apply + reductions (need_q: every coil's
// result into q; dir: form the PCG direction first).
cudaError_t tc_batch_build(TcBatch* B, const std::vector<const TcPlan*>& plans, cudaStream_t s);
void tc_batch_free(TcBatch* B);
cudaError_t launch_tc_batch(const TcBatch& B, cudaStream_t s, bool need_q, bool dir);

}  // namespace cq
