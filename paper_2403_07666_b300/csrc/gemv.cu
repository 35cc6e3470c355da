// Dense far-operator apply q = M_far p (the field-on-wire coupling of every
// element with every other element, Numerical Algorithm section).
//
// One coil and one time step give a single right-hand side, so this is a
// matrix-vector product: 2 flops per stored entry, bound by streaming the
// operator from HBM (or, in FP64 storage on B300, by the FP64 pipe).  The
// kernel is a persistent, grid-stride row-tile loop: each warp owns R rows,
// its lanes walk the row with 16-byte streaming loads (L2 evict-first, the
// operator is read once per apply), the input vector comes through the
// read-only path and stays L1/L2 resident.  Mixed precision stores the
// operator in FP32 or BF16 and multiplies it with the FP32 copy of p in a
// pure FP32 inner loop: two FP32 lane partials are folded into a second FP32
// level every 16 unrolled iterations, and FP64 is reached only in the per-row
// warp reduction.
#include "common.cuh"

namespace cq {

constexpr int kGemvWarps = 8;

template <int R>
__global__ void __launch_bounds__(kGemvWarps * 32)
k_gemv_f64(const CoilDev* __restrict__ cds, int which) {
    const CoilDev& c = cds[blockIdx.y];
    if (c.sc->done) return;
    const double2* __restrict__ p2 = reinterpret_cast<const double2*>(which == 0 ? c.x : c.dv);
    const double* __restrict__ M = static_cast<const double*>(c.Mfar);
    const int lane = threadIdx.x & 31;
    const int nvec = (int)(c.ld / 2);
    const int N = c.N;
    for (int row0 = (blockIdx.x * kGemvWarps + (threadIdx.x >> 5)) * R; row0 < N;
         row0 += gridDim.x * kGemvWarps * R) {
        const double2* rows[R];
#pragma unroll
        for (int r = 0; r < R; ++r)
            rows[r] = reinterpret_cast<const double2*>(M + (size_t)min(row0 + r, N - 1) * c.ld);
        double a0[R], a1[R];
#pragma unroll
        for (int r = 0; r < R; ++r) { a0[r] = 0.0; a1[r] = 0.0; }
#pragma unroll 2
        for (int j = lane; j < nvec; j += 32) {
            double2 pv = __ldg(p2 + j);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                double2 m = __ldcs(rows[r] + j);
                a0[r] = fma(m.x, pv.x, a0[r]);
                a1[r] = fma(m.y, pv.y, a1[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            double s = warp_sum(a0[r] + a1[r]);
            if (lane == r && row0 + r < N) c.qv[row0 + r] = s;
        }
    }
}

// FP32 operator.  The inner loop is pure FP32: on B300 the FP64 pipe issues
// two thread-operations per SM per clock (1/64 of FP32), so even an
// occasional FP64 conversion per vector makes the kernel FP64-bound.  Lane
// partials are kept in two FP32 levels (the inner pair is folded into the
// outer one every 16 unrolled iterations) and meet FP64 only in the final
// per-row warp reduction.
template <int R, int U>
__global__ void __launch_bounds__(kGemvWarps * 32)
k_gemv_f32(const CoilDev* __restrict__ cds) {
    const CoilDev& c = cds[blockIdx.y];
    if (c.sc->done) return;
    const float4* __restrict__ p4 = reinterpret_cast<const float4*>(c.pf);
    const float* __restrict__ M = static_cast<const float*>(c.Mfar);
    const int lane = threadIdx.x & 31;
    const int nvec = (int)(c.ld / 4);
    const int N = c.N;
    for (int row0 = (blockIdx.x * kGemvWarps + (threadIdx.x >> 5)) * R; row0 < N;
         row0 += gridDim.x * kGemvWarps * R) {
        const float4* rows[R];
#pragma unroll
        for (int r = 0; r < R; ++r)
            rows[r] = reinterpret_cast<const float4*>(M + (size_t)min(row0 + r, N - 1) * c.ld);
        float f0[R], f1[R], s2[R];
#pragma unroll
        for (int r = 0; r < R; ++r) { f0[r] = 0.f; f1[r] = 0.f; s2[r] = 0.f; }
        int j = lane, cnt = 0;
        for (; j + 32 * (U - 1) < nvec; j += 32 * U) {
            float4 pv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) pv[u] = __ldg(p4 + j + 32 * u);
            float4 m[R][U];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int u = 0; u < U; ++u) m[r][u] = __ldcs(rows[r] + j + 32 * u);
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    f0[r] = fmaf(m[r][u].x, pv[u].x, f0[r]);
                    f1[r] = fmaf(m[r][u].y, pv[u].y, f1[r]);
                    f0[r] = fmaf(m[r][u].z, pv[u].z, f0[r]);
                    f1[r] = fmaf(m[r][u].w, pv[u].w, f1[r]);
                }
            if (++cnt == 16) {
                cnt = 0;
#pragma unroll
                for (int r = 0; r < R; ++r) { s2[r] += f0[r] + f1[r]; f0[r] = 0.f; f1[r] = 0.f; }
            }
        }
        for (; j < nvec; j += 32) {
            float4 pv = __ldg(p4 + j);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float4 m = __ldcs(rows[r] + j);
                f0[r] = fmaf(m.x, pv.x, f0[r]);
                f1[r] = fmaf(m.y, pv.y, f1[r]);
                f0[r] = fmaf(m.z, pv.z, f0[r]);
                f1[r] = fmaf(m.w, pv.w, f1[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            double s = warp_sum((double)s2[r] + (double)(f0[r] + f1[r]));
            if (lane == r && row0 + r < N) c.qv[row0 + r] = s;
        }
    }
}

__device__ __forceinline__ float bf16_lo(unsigned v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(unsigned v) { return __uint_as_float(v & 0xffff0000u); }

// BF16 operator, FP32 products and accumulation (same structure as FP32).
template <int R, int U>
__global__ void __launch_bounds__(kGemvWarps * 32)
k_gemv_bf16(const CoilDev* __restrict__ cds) {
    const CoilDev& c = cds[blockIdx.y];
    if (c.sc->done) return;
    const float4* __restrict__ p4 = reinterpret_cast<const float4*>(c.pf);
    const __nv_bfloat16* __restrict__ M = static_cast<const __nv_bfloat16*>(c.Mfar);
    const int lane = threadIdx.x & 31;
    const int nvec = (int)(c.ld / 8);
    const int N = c.N;
    for (int row0 = (blockIdx.x * kGemvWarps + (threadIdx.x >> 5)) * R; row0 < N;
         row0 += gridDim.x * kGemvWarps * R) {
        const uint4* rows[R];
#pragma unroll
        for (int r = 0; r < R; ++r)
            rows[r] = reinterpret_cast<const uint4*>(M + (size_t)min(row0 + r, N - 1) * c.ld);
        float f0[R], f1[R], s2[R];
#pragma unroll
        for (int r = 0; r < R; ++r) { f0[r] = 0.f; f1[r] = 0.f; s2[r] = 0.f; }
        int j = lane, cnt = 0;
        for (; j + 32 * (U - 1) < nvec; j += 32 * U) {
            float4 pa[U], pb[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                pa[u] = __ldg(p4 + 2 * (j + 32 * u));
                pb[u] = __ldg(p4 + 2 * (j + 32 * u) + 1);
            }
            uint4 m[R][U];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int u = 0; u < U; ++u) m[r][u] = __ldcs(rows[r] + j + 32 * u);
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    f0[r] = fmaf(bf16_lo(m[r][u].x), pa[u].x, f0[r]);
                    f1[r] = fmaf(bf16_hi(m[r][u].x), pa[u].y, f1[r]);
                    f0[r] = fmaf(bf16_lo(m[r][u].y), pa[u].z, f0[r]);
                    f1[r] = fmaf(bf16_hi(m[r][u].y), pa[u].w, f1[r]);
                    f0[r] = fmaf(bf16_lo(m[r][u].z), pb[u].x, f0[r]);
                    f1[r] = fmaf(bf16_hi(m[r][u].z), pb[u].y, f1[r]);
                    f0[r] = fmaf(bf16_lo(m[r][u].w), pb[u].z, f0[r]);
                    f1[r] = fmaf(bf16_hi(m[r][u].w), pb[u].w, f1[r]);
                }
            if (++cnt == 16) {
                cnt = 0;
#pragma unroll
                for (int r = 0; r < R; ++r) { s2[r] += f0[r] + f1[r]; f0[r] = 0.f; f1[r] = 0.f; }
            }
        }
        for (; j < nvec; j += 32) {
            float4 pa = __ldg(p4 + 2 * j);
            float4 pb = __ldg(p4 + 2 * j + 1);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                uint4 m = __ldcs(rows[r] + j);
                f0[r] = fmaf(bf16_lo(m.x), pa.x, f0[r]);
                f1[r] = fmaf(bf16_hi(m.x), pa.y, f1[r]);
                f0[r] = fmaf(bf16_lo(m.y), pa.z, f0[r]);
                f1[r] = fmaf(bf16_hi(m.y), pa.w, f1[r]);
                f0[r] = fmaf(bf16_lo(m.z), pb.x, f0[r]);
                f1[r] = fmaf(bf16_hi(m.z), pb.y, f1[r]);
                f0[r] = fmaf(bf16_lo(m.w), pb.z, f0[r]);
                f1[r] = fmaf(bf16_hi(m.w), pb.w, f1[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            double s = warp_sum((double)s2[r] + (double)(f0[r] + f1[r]));
            if (lane == r && row0 + r < N) c.qv[row0 + r] = s;
        }
    }
}

// which: 0 = apply to the warm start x, 1 = apply to the search direction d.
// Mixed precision reads the FP32 copy pf, which the producers of x and d keep
// in step with the FP64 vector.
cudaError_t launch_gemv(const CoilDev* cds, int n_coils, int prec, long long max_rows, int which,
                        int n_sm, cudaStream_t s) {
    constexpr int R = 4;
    long long tiles = (max_rows + kGemvWarps * R - 1) / (kGemvWarps * R);
    long long cap = (long long)n_sm * 8;
    unsigned gx = (unsigned)(tiles < cap ? tiles : cap);
    if (gx == 0) gx = 1;
    dim3 grid(gx, n_coils);
    if (prec == PREC_FP64)
        k_gemv_f64<R><<<grid, kGemvWarps * 32, 0, s>>>(cds, which);
    else if (prec == PREC_FP32)
        k_gemv_f32<R, 4><<<grid, kGemvWarps * 32, 0, s>>>(cds);
    else
        k_gemv_bf16<R, 2><<<grid, kGemvWarps * 32, 0, s>>>(cds);
    return cudaGetLastError();
}

}  // namespace cq
