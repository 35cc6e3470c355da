// Assembly of the dense mutual-inductance (Green's) operator on the device.
//
// Field on each wire from the currents of all other wires (Numerical
// Algorithm section): every element is a coaxial loop; M[i][j] is the flux
// through loop i per ampere in loop j.
//   far pairs:  Maxwell's coaxial-loop formula at the element centres,
//               written with Carlson's symmetric integrals as
//               M = mu0 sqrt(r1 r2) k (2/3 R_D(0,1-m,1) - R_F(0,1-m,1)),
//               m = k^2 = 4 r1 r2 / ((r1+r2)^2 + dz^2)
//               (equal to mu0 sqrt(r1 r2)[(2/k - k)K - (2/k)E] through
//               K = R_F, E = R_F - m R_D / 3);
//   near pairs (centre distance < 3.1 element sides): the same formula
//               averaged over both squares, 4x4 Gauss-Legendre points each;
//   self:       mu0 r (ln(8 r / (0.44705 h)) - 2), the square's geometric
//               mean distance 0.44705 h.
//
// A regular solenoid is translation-invariant along z between turns, so the
// operator is block-Toeplitz in the turn index: M[(t_i,c_i),(t_j,c_j)] =
// Tab[t_i - t_j][c_i][c_j] with C = n_layers * n_sub^2 channels per turn row.
// Only C^2 (2 N_T - 1) distinct entries are evaluated (FP64), then expanded
// into the dense far operator in its storage precision; the intra-wire
// blocks go to FP64 near blocks instead.
#include "common.cuh"

namespace cq {

__constant__ double c_gl_x[4];
__constant__ double c_gl_w[4];

// Carlson's duplication for R_F(x,y,z) and R_D(x,y,z) together (Carlson,
// "Numerical computation of real or complex elliptic integrals", 1995).
__device__ void carlson_rf_rd(double x, double y, double z, double* rf, double* rd) {
    double sum = 0.0, fac = 1.0;
    for (int it = 0; it < 40; ++it) {
        double mx = fmax(x, fmax(y, z));
        double mn = fmin(x, fmin(y, z));
        if (mx - mn < 1e-3 * mx) break;
        double sx = sqrt(x), sy = sqrt(y), sz = sqrt(z);
        double lam = sx * sy + sy * sz + sz * sx;
        sum += fac / (sz * (z + lam));
        fac *= 0.25;
        x = 0.25 * (x + lam);
        y = 0.25 * (y + lam);
        z = 0.25 * (z + lam);
    }
    {   // R_F series
        double A = (x + y + z) / 3.0;
        double X = 1.0 - x / A, Y = 1.0 - y / A, Z = -(X + Y);
        double E2 = X * Y - Z * Z, E3 = X * Y * Z;
        *rf = (1.0 - E2 / 10.0 + E3 / 14.0 + E2 * E2 / 24.0 - 3.0 * E2 * E3 / 44.0) / sqrt(A);
    }
    {   // R_D series
        double A = (x + y + 3.0 * z) / 5.0;
        double X = (A - x) / A, Y = (A - y) / A, Z = -(X + Y) / 3.0;
        double XY = X * Y, Z2 = Z * Z;
        double E2 = XY - 6.0 * Z2;
        double E3 = (3.0 * XY - 8.0 * Z2) * Z;
        double E4 = 3.0 * (XY - Z2) * Z2;
        double E5 = XY * Z2 * Z;
        double ser = 1.0 - 3.0 * E2 / 14.0 + E3 / 6.0 + 9.0 * E2 * E2 / 88.0 - 3.0 * E4 / 22.0
                   - 9.0 * E2 * E3 / 52.0 + 3.0 * E5 / 26.0;
        *rd = 3.0 * sum + fac * ser / (A * sqrt(A));
    }
}

// Mutual inductance of two coaxial filament loops; bitwise symmetric in its
// two loops (every product and sum is written commutatively).
__device__ double mutual_point(double r1, double z1, double r2, double z2) {
    double dz = z1 - z2;
    double dz2 = dz * dz;
    double s = r1 + r2;
    double dr = r1 - r2;
    double den = s * s + dz2;
    double rr = r1 * r2;
    double m = 4.0 * rr / den;
    double mc = (dr * dr + dz2) / den;
    double rf, rd;
    carlson_rf_rd(0.0, mc, 1.0, &rf, &rd);
    return kMu0 * sqrt(rr) * sqrt(m) * (2.0 / 3.0 * rd - rf);
}

__device__ double mutual_near(double r1, double z1, double h1, double r2, double z2, double h2) {
    double acc = 0.0;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            double ra = r1 + 0.5 * h1 * c_gl_x[a];
            double za = z1 + 0.5 * h1 * c_gl_x[b];
            double wab = 0.25 * c_gl_w[a] * c_gl_w[b];
            double inner = 0.0;
            for (int c2 = 0; c2 < 4; ++c2)
                for (int d2 = 0; d2 < 4; ++d2) {
                    double rb = r2 + 0.5 * h2 * c_gl_x[c2];
                    double zb = z2 + 0.5 * h2 * c_gl_x[d2];
                    inner += 0.25 * c_gl_w[c2] * c_gl_w[d2] * mutual_point(ra, za, rb, zb);
                }
            acc += wab * inner;
        }
    return acc;
}

__device__ double self_term(double r, double h) {
    return kMu0 * r * (log(8.0 * r / (0.44705 * h)) - 2.0);
}

// One distinct operator entry: channel ci on turn d against channel cj on turn 0.
__device__ double table_entry(const double* rc, const double* zc, const double* hc,
                              int ci, int cj, int d, double pitch_t) {
    if (d == 0 && ci == cj) return self_term(rc[ci], hc[ci]);
    int a = ci, b = cj;
    if (d == 0 && a > b) { a = cj; b = ci; }       // canonical order: symmetric slab
    double r1 = rc[a], z1 = zc[a] + d * pitch_t;
    double r2 = rc[b], z2 = zc[b];
    double hm = fmax(hc[a], hc[b]);
    double dr = r1 - r2, dz = z1 - z2;
    if (dr * dr + dz * dz < (3.1 * hm) * (3.1 * hm))
        return mutual_near(r1, z1, hc[a], r2, z2, hc[b]);
    return mutual_point(r1, z1, r2, z2);
}

// tab[(D + NT - 1)][ci][cj] for D in (-NT, NT); this kernel evaluates D >= 0
// and mirrors it to -D (M symmetric).
__global__ void k_table(const double* __restrict__ rc, const double* __restrict__ zc,
                        const double* __restrict__ hc, int C, int NT, double pitch_t,
                        double* __restrict__ tab) {
    long long total = (long long)C * C * NT;
    long long CC = (long long)C * C;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        int cj = (int)(idx % C);
        int ci = (int)((idx / C) % C);
        int d = (int)(idx / CC);
        double v = table_entry(rc, zc, hc, ci, cj, d, pitch_t);
        tab[(long long)(d + NT - 1) * CC + (long long)ci * C + cj] = v;
        if (d > 0) tab[(long long)(NT - 1 - d) * CC + (long long)cj * C + ci] = v;
    }
}

template <typename T> __device__ __forceinline__ T from_double(double v);
template <> __device__ __forceinline__ double from_double<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_double<float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_double<__nv_bfloat16>(double v) {
    return __double2bfloat16(v);
}

// Dense far operator from the table: row i = (t_i, c_i); intra-wire entries
// (same turn row, same wire) are zero here and live in the FP64 near blocks.
template <typename T>
__global__ void k_expand(const double* __restrict__ tab, int C, int NT, int wire_div,
                         long long N, long long ld, T* __restrict__ M) {
    long long chunks = ld / 8;
    long long total = N * chunks;
    long long CC = (long long)C * C;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        long long i = idx / chunks;
        long long j0 = (idx % chunks) * 8;
        int ti = (int)(i / C), ci = (int)(i % C);
        T* out = M + i * ld + j0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            long long j = j0 + k;
            double v = 0.0;
            if (j < N) {
                int tj = (int)(j / C), cj = (int)(j % C);
                if (!(ti == tj && ci / wire_div == cj / wire_div))
                    v = tab[(long long)(ti - tj + NT - 1) * CC + (long long)ci * C + cj];
            }
            out[k] = from_double<T>(v);
        }
    }
}

// FP64 intra-wire blocks: near[type][ka][kb] from the D = 0 slab (and, where
// nearf is given, the same blocks rounded to FP32).
__global__ void k_near_blocks(const double* __restrict__ tab, int C, int NT, int B, int n_types,
                              double* __restrict__ near, float* __restrict__ nearf) {
    long long CC = (long long)C * C;
    const double* slab = tab + (long long)(NT - 1) * CC;
    int total = n_types * B * B;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        int kb = idx % B, ka = (idx / B) % B, ty = idx / (B * B);
        int base = ty * B;
        const double v = slab[(long long)(base + ka) * C + base + kb];
        near[idx] = v;
        if (nearf) nearf[idx] = __double2float_rn(v);
    }
}

}  // namespace cq

// ---- host launchers -------------------------------------------------------

namespace cq {

cudaError_t upload_gl_rule(const double* x, const double* w) {
    cudaError_t e = cudaMemcpyToSymbol(c_gl_x, x, 4 * sizeof(double));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_gl_w, w, 4 * sizeof(double));
}

cudaError_t launch_table(const double* rc, const double* zc, const double* hc, int C, int NT,
                         double pitch_t, double* tab, cudaStream_t s) {
    long long total = (long long)C * C * NT;
    int threads = 256;
    long long blocks = (total + threads - 1) / threads;
    if (blocks > 148LL * 64) blocks = 148LL * 64;
    k_table<<<(unsigned)blocks, threads, 0, s>>>(rc, zc, hc, C, NT, pitch_t, tab);
    return cudaGetLastError();
}

cudaError_t launch_expand(const double* tab, int C, int NT, int wire_div, long long N, long long ld,
                          int prec, void* M, cudaStream_t s) {
    long long total = N * (ld / 8);
    int threads = 256;
    long long blocks = (total + threads - 1) / threads;
    if (blocks > 148LL * 128) blocks = 148LL * 128;
    if (prec == PREC_FP64)
        k_expand<double><<<(unsigned)blocks, threads, 0, s>>>(tab, C, NT, wire_div, N, ld, (double*)M);
    else if (prec == PREC_FP32)
        k_expand<float><<<(unsigned)blocks, threads, 0, s>>>(tab, C, NT, wire_div, N, ld, (float*)M);
    else
        k_expand<__nv_bfloat16><<<(unsigned)blocks, threads, 0, s>>>(tab, C, NT, wire_div, N, ld,
                                                                     (__nv_bfloat16*)M);
    return cudaGetLastError();
}

cudaError_t launch_near_blocks(const double* tab, int C, int NT, int B, int n_types, double* near,
                               float* nearf, cudaStream_t s) {
    int total = n_types * B * B;
    int threads = 256;
    int blocks = (total + threads - 1) / threads;
    k_near_blocks<<<blocks, threads, 0, s>>>(tab, C, NT, B, n_types, near, nearf);
    return cudaGetLastError();
}

}  // namespace cq
