// CTA-parallel tridiagonal line solve shared by the forward and adjoint heat
// steps.
#pragma once

#include "common.cuh"

namespace cq {

// Tridiagonal solve of one grid line held in shared memory v[0..G) by the
// kAdiThreads threads of the CTA, from the Thomas algorithm's precomputed
// factors in recurrence form: forward y_i = a_i y_{i-1} + inv_i v_i (a_0 = 0),
// backward x_i = c_i x_{i+1} + y_i (c_{G-1} = 0).  Both are first-order linear
// recurrences, so every thread composes the affine map of its chunk of
// ceil(G / kAdiThreads) entries, the maps are combined in thread order (a scan
// inside each warp, then the warps' totals in warp order), and each thread
// re-runs its chunk from its incoming value.  The factors are staged into f
// (3 G doubles of shared memory) first, by line_stage, so the recurrences read
// no global memory; a kernel calls line_stage before it forms v, so that the
// two sets of loads overlap.  Fixed order: deterministic.  Every thread of the
// CTA calls line_solve after v is written (it opens with a barrier) and may
// read v when it returns.
__device__ inline void line_stage(double* f, int G, const double* __restrict__ a, const double* __restrict__ inv,
                                  const double* __restrict__ cc) {
    for (int i = threadIdx.x; i < G; i += kAdiThreads) {
        f[i] = a[i];
        f[G + i] = inv[i];
        f[2 * G + i] = cc[i];
    }
}

__device__ inline void line_solve(double* v, const double* f, int G) {
    constexpr int NW = kAdiThreads / 32;
    constexpr unsigned kFull = 0xffffffffu;
    __shared__ double wA[NW], wB[NW];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const double* fa = f;
    const double* fi = f + G;
    const double* fc = f + 2 * G;
    __syncthreads();
    const int m = (G + kAdiThreads - 1) / kAdiThreads;
    const int i0 = min(tid * m, G), i1 = min(i0 + m, G);
    // forward: the chunk's map y_out = A y_in + Bc
    double A = 1.0, Bc = 0.0;
    for (int i = i0; i < i1; ++i) {
        A = fa[i] * A;
        Bc = fa[i] * Bc + v[i] * fi[i];
    }
    for (int o = 1; o < 32; o <<= 1) {                  // inclusive prefix: (mine) o (lower lanes)
        const double pA = __shfl_up_sync(kFull, A, o), pB = __shfl_up_sync(kFull, Bc, o);
        if (lane >= o) {
            Bc = A * pB + Bc;
            A = A * pA;
        }
    }
    if (lane == 31) {
        wA[wid] = A;
        wB[wid] = Bc;
    }
    __syncthreads();
    double PA = 1.0, PB = 0.0;                          // the lower warps' maps, composed in order
    for (int k = 0; k < wid; ++k) {
        PB = wA[k] * PB + wB[k];
        PA = wA[k] * PA;
    }
    // y entering the chunk: the lower threads' composed map (a_0 = 0: its input is irrelevant)
    double y = __shfl_up_sync(kFull, A * PB + Bc, 1);
    if (lane == 0) y = PB;
    for (int i = i0; i < i1; ++i) {
        y = fa[i] * y + v[i] * fi[i];
        v[i] = y;
    }
    __syncthreads();
    // backward: the chunk's map x_i0 = A x_i1 + Bc
    A = 1.0;
    Bc = 0.0;
    for (int i = i1 - 1; i >= i0; --i) {
        A = fc[i] * A;
        Bc = fc[i] * Bc + v[i];
    }
    for (int o = 1; o < 32; o <<= 1) {                  // inclusive suffix: (mine) o (higher lanes)
        const double qA = __shfl_down_sync(kFull, A, o), qB = __shfl_down_sync(kFull, Bc, o);
        if (lane + o < 32) {
            Bc = A * qB + Bc;
            A = A * qA;
        }
    }
    if (lane == 0) {
        wA[wid] = A;
        wB[wid] = Bc;
    }
    __syncthreads();
    double SB = 0.0;                                    // the higher warps' maps, composed from the top
    for (int k = NW - 1; k > wid; --k) SB = wA[k] * SB + wB[k];
    double x = __shfl_down_sync(kFull, A * SB + Bc, 1); // x just above the chunk (c_{G-1} = 0)
    if (lane == 31) x = SB;
    for (int i = i1 - 1; i >= i0; --i) {
        x = fc[i] * x + v[i];
        v[i] = x;
    }
    __syncthreads();
}

}  // namespace cq
