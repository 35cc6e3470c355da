// Warp-parallel tridiagonal line solve shared by the forward and adjoint
// heat steps.
#pragma once

#include "common.cuh"

namespace cq {

// Tridiagonal solve of one line held in shared memory, with the precomputed
// factors of the Thomas algorithm: forward y_i = (v_i - lo_i y_{i-1}) inv_i,
// backward x_i = y_i - cp_i x_{i+1}.  Both are first-order linear
// recurrences, y_i = a_i y_{i-1} + b_i, so all 32 lanes take part: each lane
// composes the affine map of its chunk of ceil(G / 32) entries, a warp scan
// combines the maps in lane order (a prefix for the forward sweep, a suffix
// for the backward one), and each lane re-runs its chunk from its incoming
// value.  Fixed order: deterministic.  Every lane of the warp calls this.
__device__ inline void warp_tridiag(double* v, int G, const double* lo, const double* inv, const double* cp) {
    const int lane = threadIdx.x & 31;
    const int m = (G + 31) / 32;
    const int i0 = min(lane * m, G), i1 = min(i0 + m, G);
    // forward: a_i = -lo_i inv_i (a_0 = 0), b_i = v_i inv_i; chunk map y_out = A y_in + Bc
    double A = 1.0, Bc = 0.0;
    for (int i = i0; i < i1; ++i) {
        const double a = i > 0 ? -lo[i] * inv[i] : 0.0;
        A = a * A;
        Bc = a * Bc + v[i] * inv[i];
    }
    for (int o = 1; o < 32; o <<= 1) {                  // inclusive prefix: (mine) o (lower lanes)
        const double pA = __shfl_up_sync(0xffffffffu, A, o), pB = __shfl_up_sync(0xffffffffu, Bc, o);
        if (lane >= o) {
            Bc = A * pB + Bc;
            A = A * pA;
        }
    }
    double y = __shfl_up_sync(0xffffffffu, Bc, 1);      // y entering the chunk (lane 0: unused, a_0 = 0)
    if (lane == 0) y = 0.0;
    for (int i = i0; i < i1; ++i) {
        const double a = i > 0 ? -lo[i] * inv[i] : 0.0;
        y = a * y + v[i] * inv[i];
        v[i] = y;
    }
    // backward: x_i = c_i x_{i+1} + y_i, c_i = -cp_i (0 at the top); chunk map x_i0 = A x_i1 + Bc
    A = 1.0;
    Bc = 0.0;
    for (int i = i1 - 1; i >= i0; --i) {
        const double cc = i < G - 1 ? -cp[i] : 0.0;
        A = cc * A;
        Bc = cc * Bc + v[i];
    }
    for (int o = 1; o < 32; o <<= 1) {                  // inclusive suffix: (mine) o (higher lanes)
        const double qA = __shfl_down_sync(0xffffffffu, A, o), qB = __shfl_down_sync(0xffffffffu, Bc, o);
        if (lane + o < 32) {
            Bc = A * qB + Bc;
            A = A * qA;
        }
    }
    double x = __shfl_down_sync(0xffffffffu, Bc, 1);    // x just above the chunk (lane 31: unused)
    if (lane == 31) x = 0.0;
    for (int i = i1 - 1; i >= i0; --i) {
        const double cc = i < G - 1 ? -cp[i] : 0.0;
        x = cc * x + v[i];
        v[i] = x;
    }
    __syncwarp();
}

}  // namespace cq
