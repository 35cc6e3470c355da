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
};

struct TcPlan {
    CUtensorMap tmA;            // split table: [half][offset >= 0][c'/64][c][c' % 64] FP16, 128-byte swizzle
    CUtensorMap tmAT;           // the same table, transposed-tile boxes (offsets < 0)
    CUtensorMap tmB;            // split input: [c'/8][hi, lo][t][c' % 8] FP16, no swizzle
    TcShape sh;
    const CoilDev* d = nullptr; // device descriptor of the coil
    __half* t16 = nullptr;      // 2 NT n_kb C 64
    __half* p16 = nullptr;      // 2 Cp NT
    float* part = nullptr;      // n_cta x NT x 128 partial tiles
    int4* work = nullptr;       // n_cta (tile, first stage, end stage, 0)
    int2* range = nullptr;      // n_ct (first CTA, CTAs)
    int* pexp = nullptr;        // NT input scale exponents (one per turn row)
    int exT = 0;                // table scale 2^exT
    size_t smem = 0;            // dynamic shared memory per CTA
    bool fused = false;         // the coil's near kernel sums the partial tiles itself
};

constexpr int kTcMaxTurns = 112;   // the staged copy's 2 (NT + 16) rows fit one TMA box (<= 256)

// Fill the shape for C channels, NT turns on n_sm SMs; false if unsupported.
bool tc_shape(int C, int NT, int n_sm, TcShape* sh);
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
// shared-warp near kernel sums the tiles).
// dir: form the PCG direction d = -z + beta d in the input split first.
cudaError_t launch_toeplitz_tc(const TcPlan& P, cudaStream_t s, bool write_q, bool dir = false);
// Its two halves: the input split (k_tc_split) and the tensor-core product
// (k_toeplitz_tc, plus the FP64 reduction into q when write_q).
cudaError_t launch_tc_split(const TcPlan& P, cudaStream_t s, bool dir);
cudaError_t launch_tc_apply(const TcPlan& P, cudaStream_t s, bool write_q);

}  // namespace cq
