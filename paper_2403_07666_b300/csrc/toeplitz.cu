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
// Decomposition: a CTA owns a tile of 32 turn rows x 128 channels and a chunk
// of DC turn offsets d; it runs a register-blocked FP32 GEMM over (d, c')
// (4 rows x 8 channels per thread) with the p rows shifted by d read through
// double-buffered shared memory, the next tile copied in with cp.async
// while the current one is used (rows outside the winding read as zero; a
// warp whose 8 rows all fall outside for an offset skips it).  Each CTA writes
// its partial tile; k_toeplitz_reduce sums the chunks in a fixed order into
// the FP64 result (deterministic).  Lane partials fold into a second FP32
// level every 128 k terms.
#include "common.cuh"

namespace cq {

constexpr int kTT = 32;    // turn rows per tile
constexpr int kTC = 128;   // channels per tile
constexpr int kTK = 32;    // k (input channel) chunk
constexpr int kDC = 4;     // turn offsets per CTA

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

// Asynchronous 4- and 16-byte global -> shared copies; a source size of 0
// fills the destination with zeros (rows outside the winding, ragged tiles).
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
    unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0));
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src, bool valid) {
    unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int Pending>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(Pending)); }

__global__ void __launch_bounds__(128, 4)
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
    const int nd = max(d_hi - d_lo, 0);
    const int nk = (C + kTK - 1) / kTK;
    const int nq = nd * nk;                           // (d, k chunk) pairs
    const bool vec = (C & 3) == 0;                    // 16-byte copies of the table rows

    __shared__ __align__(16) float As[2][kTK][kTT];  // As[k][t]  = p[t0 + t - d][k0 + k]
    __shared__ __align__(16) float Bs[2][kTK][kTC];  // Bs[k][cc] = T_d[c0 + cc][k0 + k]
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int tx = lane & 15;                         // channels 4tx..4tx+3 and 64+4tx..64+4tx+3
    const int ty = 2 * warp + (lane >> 4);            // rows 4ty..4ty+3
    const float* __restrict__ PT = c.pT;
    const size_t CC = (size_t)C * C;

    float acc[4][8], acc2[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) { acc[i][j] = 0.f; acc2[i][j] = 0.f; }

    auto issue = [&](int q, int buf) {
        int d = d_lo + q / nk, k0 = (q % nk) * kTK;
        const float* Tm = c.tab32 + (size_t)(NT - 1 - d) * CC;   // T_d^T = T_{-d}
#pragma unroll
        for (int m = 0; m < (kTT * kTK) / 128; ++m) {
            int idx = tid + m * 128;
            int t = idx % kTT, k = idx / kTT;
            int ts = t0 + t - d;
            bool ok = t0 + t < t1 && ts >= 0 && ts < NT && k0 + k < C;
            cp_async4(&As[buf][k][t], ok ? PT + (size_t)(k0 + k) * NT + ts : PT, ok);
        }
        if (vec) {
#pragma unroll
            for (int m = 0; m < (kTC * kTK) / (4 * 128); ++m) {
                int idx = tid + m * 128;
                int c4 = idx % (kTC / 4), k = idx / (kTC / 4);
                bool ok = c0 + 4 * c4 < C && k0 + k < C;
                cp_async16(&Bs[buf][k][4 * c4], ok ? Tm + (size_t)(k0 + k) * C + c0 + 4 * c4 : Tm, ok);
            }
        } else {
            for (int m = 0; m < (kTC * kTK) / 128; ++m) {
                int idx = tid + m * 128;
                int cc = idx % kTC, k = idx / kTC;
                bool ok = c0 + cc < C && k0 + k < C;
                cp_async4(&Bs[buf][k][cc], ok ? Tm + (size_t)(k0 + k) * C + c0 + cc : Tm, ok);
            }
        }
        cp_async_commit();
    };

    if (nq > 0) issue(0, 0);
    for (int q = 0; q < nq; ++q) {
        const int buf = q & 1;
        const int d = d_lo + q / nk;
        if (q + 1 < nq) {
            issue(q + 1, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        // this warp's 8 rows t0 + 8 warp .. +7: skip the chunk if none has 0 <= t - d < NT
        const int tw = t0 + 8 * warp;
        const bool live = tw < t1 && tw + 7 - d >= 0 && tw - d < NT;
        if (live) {
#pragma unroll 8
            for (int k = 0; k < kTK; ++k) {
                const float4 a = *reinterpret_cast<const float4*>(&As[buf][k][4 * ty]);
                const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][4 * tx]);
                const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + 4 * tx]);
#define CQ_ROW(i, ai)                                   \
    acc[i][0] = fmaf(ai, b0.x, acc[i][0]);              \
    acc[i][1] = fmaf(ai, b0.y, acc[i][1]);              \
    acc[i][2] = fmaf(ai, b0.z, acc[i][2]);              \
    acc[i][3] = fmaf(ai, b0.w, acc[i][3]);              \
    acc[i][4] = fmaf(ai, b1.x, acc[i][4]);              \
    acc[i][5] = fmaf(ai, b1.y, acc[i][5]);              \
    acc[i][6] = fmaf(ai, b1.z, acc[i][6]);              \
    acc[i][7] = fmaf(ai, b1.w, acc[i][7]);
                CQ_ROW(0, a.x)
                CQ_ROW(1, a.y)
                CQ_ROW(2, a.z)
                CQ_ROW(3, a.w)
#undef CQ_ROW
            }
        }
        __syncthreads();                              // the buffer is refilled by the next issue
        if ((q + 1) % 4 == 0 || q + 1 == nq) {        // every 128 k terms: fold the lane sums
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) { acc2[i][j] += acc[i][j]; acc[i][j] = 0.f; }
        }
    }
    // partial tile -> tpart[(tt * ndc + dc)][t - t0][c]
    float* out = c.tpart + (size_t)(tt * ndc + dc) * kTT * C;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int t = 4 * ty + i;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            int cc = c0 + (j < 4 ? 4 * tx + j : 64 + 4 * tx + j - 4);
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
