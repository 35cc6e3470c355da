// Shared-warp layout of the per-wire kernels for wires of at most kSegMax
// elements (32 / Bp wires per warp, Bp = B rounded up to a power of two), and
// the near-block product that both the PCG's near kernel and the
// tensor-core apply's near warps run, in the same order of operations.
#pragma once

#include "common.cuh"

namespace cq {

__device__ __forceinline__ int seg_width(int B) {
    int p = 1;
    while (p < B) p <<= 1;
    return p;
}

__device__ __forceinline__ double seg_sum(double v, int Bp) {
    for (int o = Bp >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct Seg {
    int B, Bp, kk, base, w, e;
    bool wv, ev;        // wire exists, element exists
};

__device__ __forceinline__ Seg seg_of(const CoilDev& c, int warp_global) {
    Seg s;
    s.B = c.B;
    s.Bp = seg_width(c.B);
    const int lane = threadIdx.x & 31;
    s.kk = lane & (s.Bp - 1);
    s.base = lane - s.kk;
    s.w = warp_global * (32 / s.Bp) + lane / s.Bp;
    s.wv = s.w < c.W;
    s.ev = s.wv && s.kk < s.B;
    s.e = s.w * s.B + s.kk;
    return s;
}

// The near-block part of q at the lane's element: row kk of the wire's FP64
// self block (block type bt) against the wire's p, held one element per lane
// of the segment, plus dt G p on the diagonal.  Every lane of the warp calls
// it (shuffles); the value is meaningful on element lanes.
__device__ __forceinline__ double near_row_product(const CoilDev& c, const Seg& s, int bt, double pv, double ge) {
    const double* nb = c.near + (size_t)bt * s.B * s.B;
    const int row = s.kk < s.B ? s.kk : 0;
    double acc = 0.0;
    if (s.B == kSegMax) {
        // 16-element wires: the row as eight 16-byte loads, all in flight at once
        double2 nr[kSegMax / 2];
#pragma unroll
        for (int q = 0; q < kSegMax / 2; ++q) nr[q] = reinterpret_cast<const double2*>(nb + row * kSegMax)[q];
#pragma unroll
        for (int q = 0; q < kSegMax / 2; ++q) {
            acc = fma(nr[q].x, __shfl_sync(0xffffffffu, pv, s.base + 2 * q), acc);
            acc = fma(nr[q].y, __shfl_sync(0xffffffffu, pv, s.base + 2 * q + 1), acc);
        }
    } else {
        for (int j = 0; j < s.B; ++j) acc = fma(nb[row * s.B + j], __shfl_sync(0xffffffffu, pv, s.base + j), acc);
    }
    if (s.ev) acc = fma(c.dt * ge, pv, acc);
    return acc;
}

}  // namespace cq
