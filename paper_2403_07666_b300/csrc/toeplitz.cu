// Block-Toeplitz far-operator apply for a regular solenoid.
//
// The coaxial-loop mutual inductance depends on r_i, r_j and z_i - z_j only,
// so on a regular winding the far operator between turn rows t_i and t_j is
// one C x C block T_d with d = t_i - t_j (C = n_layers n_sub^2 channels per
// turn row, element e = t C + c):
//
//     y[t][c] = sum_d sum_c' T_d[c][c'] p[t - d][c'].
//
// These are the entries of the dense operator, not an approximation; the
// table holds C^2 (2 N_T - 1) of them instead of N^2 (0.73 GB instead of
// 36.9 GB at 96,000 elements in FP32), so the apply is bound by the FP32
// pipe rather than by HBM.  Work: 2 N^2 flops per apply as for the dense form.
//
// Decomposition: a CTA owns a tile of 32 turn rows x 64 channels and a chunk
// of DC turn offsets d; it runs a register-blocked FP32 GEMM over (d, c')
// with the p rows shifted by d read through shared memory (rows outside the
// winding read as zero).  Each CTA writes its partial tile; k_toeplitz_reduce
// sums the chunks in a fixed order into the FP64 result (deterministic).
// Lane partials fold into a second FP32 level after every 32-wide k chunk.
#include "common.cuh"

namespace cq {

constexpr int kTT = 32;    // turn rows per tile
constexpr int kTC = 64;    // channels per tile
constexpr int kTK = 32;    // k (input channel) chunk
constexpr int kDC = 16;    // turn offsets per CTA

__host__ __device__ inline int toeplitz_t_tiles(int NT) { return (NT + kTT - 1) / kTT; }
__host__ __device__ inline int toeplitz_d_chunks(int NT) { return (kTT + NT - 1 + kDC - 1) / kDC; }

// p^T: pT[c][t] = p[t][c] (FP32), so that the shifted p rows load along t.
__global__ void k_toeplitz_transpose(const CoilDev* __restrict__ cds) {
    const CoilDev& c = cds[blockIdx.y];
    if (c.op_format != 1 || c.sc->done) return;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < c.N; e += gridDim.x * blockDim.x) {
        int t = e / c.C, cc = e - t * c.C;
        c.pT[(size_t)cc * c.NT + t] = c.pf[e];
    }
}

__global__ void __launch_bounds__(128)
k_toeplitz_f32(const CoilDev* __restrict__ cds) {
    const CoilDev& c = cds[blockIdx.y];
    if (c.op_format != 1 || c.sc->done) return;
    const int C = c.C, NT = c.NT;
    const int nct = (C + kTC - 1) / kTC;
    const int ntt = toeplitz_t_tiles(NT);
    const int ndc = toeplitz_d_chunks(NT);
    int blk = blockIdx.x;
    if (blk >= nct * ntt * ndc) return;
    const int ct = blk % nct;
    const int tt = (blk / nct) % ntt;
    const int dc = blk / (nct * ntt);
    const int t0 = tt * kTT, t1 = min(t0 + kTT, NT);
    const int c0 = ct * kTC;
    // valid offsets for this row tile: 0 <= t - d < NT for some t in [t0, t1)
    const int dmin = t0 - (NT - 1);
    const int d_lo = dmin + dc * kDC;
    const int d_hi = min(d_lo + kDC, t1);            // exclusive: d <= t1 - 1

    __shared__ __align__(16) float As[kTK][kTT];     // As[k][t]  = p[t0 + t - d][k0 + k]
    __shared__ __align__(16) float Bs[kTK][kTC];     // Bs[k][cc] = T_d[c0 + cc][k0 + k]
    const int tid = threadIdx.x;
    const int tx = tid & 15;                          // channels 4 tx .. 4 tx + 3
    const int ty = tid >> 4;                          // rows     4 ty .. 4 ty + 3
    float acc[4][4], acc2[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { acc[i][j] = 0.f; acc2[i][j] = 0.f; }
    const float* __restrict__ PT = c.pT;
    const size_t CC = (size_t)C * C;

    for (int d = d_lo; d < d_hi; ++d) {
        // T_d[c][c'] = T_{-d}[c'][c]: the block of offset -d read along c gives T_d^T
        const float* Tm = c.tab32 + (size_t)(NT - 1 - d) * CC;
        for (int k0 = 0; k0 < C; k0 += kTK) {
            // A tile: 32 k x 32 rows, 8 per thread, contiguous along t
#pragma unroll
            for (int q = 0; q < (kTT * kTK) / 128; ++q) {
                int idx = tid + q * 128;
                int t = idx % kTT, k = idx / kTT;
                int ts = t0 + t - d;
                float v = 0.f;
                if (t0 + t < t1 && ts >= 0 && ts < NT && k0 + k < C) v = PT[(size_t)(k0 + k) * NT + ts];
                As[k][t] = v;
            }
            // B tile: 32 k x 64 channels, 16 per thread, contiguous along c
#pragma unroll
            for (int q = 0; q < (kTC * kTK) / 128; ++q) {
                int idx = tid + q * 128;
                int cc = idx % kTC, k = idx / kTC;
                float v = 0.f;
                if (c0 + cc < C && k0 + k < C) v = __ldg(Tm + (size_t)(k0 + k) * C + c0 + cc);
                Bs[k][cc] = v;
            }
            __syncthreads();
#pragma unroll 8
            for (int k = 0; k < kTK; ++k) {
                const float4 a = *reinterpret_cast<const float4*>(&As[k][4 * ty]);
                const float4 b = *reinterpret_cast<const float4*>(&Bs[k][4 * tx]);
#define CQ_ROW(i, ai)                                  \
    acc[i][0] = fmaf(ai, b.x, acc[i][0]);              \
    acc[i][1] = fmaf(ai, b.y, acc[i][1]);              \
    acc[i][2] = fmaf(ai, b.z, acc[i][2]);              \
    acc[i][3] = fmaf(ai, b.w, acc[i][3]);
                CQ_ROW(0, a.x)
                CQ_ROW(1, a.y)
                CQ_ROW(2, a.z)
                CQ_ROW(3, a.w)
#undef CQ_ROW
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) { acc2[i][j] += acc[i][j]; acc[i][j] = 0.f; }
        }
    }
    // partial tile -> tpart[(tt * ndc + dc)][t - t0][c]
    float* out = c.tpart + (size_t)(tt * ndc + dc) * kTT * C;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int t = 4 * ty + i;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int cc = c0 + 4 * tx + j;
            if (cc < C) out[(size_t)t * C + cc] = acc2[i][j];
        }
    }
}

// q[t C + c] = sum over the d chunks of the partial tiles (fixed order, FP64).
__global__ void k_toeplitz_reduce(const CoilDev* __restrict__ cds) {
    const CoilDev& c = cds[blockIdx.y];
    if (c.op_format != 1 || c.sc->done) return;
    const int C = c.C, NT = c.NT;
    const int ndc = toeplitz_d_chunks(NT);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < c.N; e += gridDim.x * blockDim.x) {
        int t = e / C, cc = e - t * C;
        int tt = t / kTT, tr = t - tt * kTT;
        const float* base = c.tpart + (size_t)tt * ndc * kTT * C + (size_t)tr * C + cc;
        double s = 0.0;
        for (int q = 0; q < ndc; ++q) s += (double)base[(size_t)q * kTT * C];
        c.qv[e] = s;
    }
}

// FP32 Toeplitz table from the FP64 table, intra-wire entries (offset 0,
// same wire) zero: they are applied from the FP64 near blocks.
__global__ void k_toeplitz_table(const double* __restrict__ tab, int C, int NT, int wire_div,
                                 float* __restrict__ out) {
    long long total = (long long)C * C * (2 * NT - 1);
    long long CC = (long long)C * C;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        int d = (int)(idx / CC) - (NT - 1);
        int ci = (int)((idx % CC) / C), cj = (int)(idx % C);
        double v = tab[idx];
        if (d == 0 && ci / wire_div == cj / wire_div) v = 0.0;
        out[idx] = __double2float_rn(v);
    }
}

size_t toeplitz_part_floats(int C, int NT) {
    return (size_t)toeplitz_t_tiles(NT) * toeplitz_d_chunks(NT) * kTT * C;
}

cudaError_t launch_toeplitz_table(const double* tab, int C, int NT, int wire_div, float* out, cudaStream_t s) {
    long long total = (long long)C * C * (2 * NT - 1);
    long long blocks = (total + 255) / 256;
    if (blocks > 148LL * 64) blocks = 148LL * 64;
    k_toeplitz_table<<<(unsigned)blocks, 256, 0, s>>>(tab, C, NT, wire_div, out);
    return cudaGetLastError();
}

// max_C / max_NT: the largest channel count and turn count in the batch.
cudaError_t launch_toeplitz(const CoilDev* cds, int n_coils, int max_C, int max_NT, long long max_N, int n_sm,
                            cudaStream_t s) {
    int nct = (max_C + kTC - 1) / kTC;
    unsigned gx = (unsigned)(nct * toeplitz_t_tiles(max_NT) * toeplitz_d_chunks(max_NT));
    unsigned eb = (unsigned)((max_N + 255) / 256);
    if (eb > (unsigned)n_sm * 16) eb = n_sm * 16;
    k_toeplitz_transpose<<<dim3(eb, n_coils), 256, 0, s>>>(cds);
    k_toeplitz_f32<<<dim3(gx, n_coils), 128, 0, s>>>(cds);
    k_toeplitz_reduce<<<dim3(eb, n_coils), 256, 0, s>>>(cds);
    return cudaGetLastError();
}

}  // namespace cq
