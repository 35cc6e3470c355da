// Device-side descriptor of one coil and small helpers shared by the kernels.
//
// Every per-step kernel receives an array of CoilDev descriptors and picks its
// coil from blockIdx.y, so one launch can serve a batch of coils of uneven
// size (CTAs beyond a coil's extent return at once).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace cq {

constexpr double kPi = 3.14159265358979323846;
constexpr double kMu0 = 4.0e-7 * kPi;
constexpr int kMaxBlock = 64;        // elements per wire (block) handled by one warp
constexpr int kSegMax = 16;          // blocks this small share a warp (32 / B rounded up to a power of 2)
constexpr int kMedMax = 64;          // blocks of kSegMax + 1 .. kMedMax elements (no subelements): one
                                     // row per thread of a 64-thread CTA, FP32 inverse, stored P_w
constexpr int kMedFactorThreads = 2 * kMedMax;   // the medium-wire factor: two threads per row
constexpr int kAdiThreads = 128;     // threads per grid line of the ADI solves (tridiag.cuh)
// shared memory of one ADI line solve: the line and its three factor rows
__host__ __device__ constexpr size_t adi_smem_bytes(int G) { return 4 * (size_t)G * sizeof(double); }
constexpr int kGroupMax = 16;        // subelements per turn
constexpr int kGroupMaxSeg = 6;      // subelements per turn of blocks of at most kSegMax elements
constexpr int kSegWarps = 4;         // warps per CTA of the shared-warp kernels
constexpr int kTcTileRows = 128;     // channels per tile of the tensor-core Toeplitz apply
constexpr int kStepEndCtas = 16;     // CTAs per coil of the step-end reductions
constexpr int kStepEndThreads = 256;

enum Prec { PREC_FP64 = 0, PREC_FP32 = 1, PREC_BF16 = 2 };

// ST_KERNEL: a bounded wait inside a kernel ran out (the kernel stopped early).
enum Status { ST_OK = 0, ST_NOT_CONVERGED = 4, ST_NONFINITE = 5, ST_KERNEL = 6 };

// Per-coil scalars that live on the device (written by kernels, read back by
// the host only between launches).
struct Scalars {
    double t;            // simulated time at the start of the current step
    long long step;      // completed steps
    double It1, Ba0, Ba1, dBa;
    double scale2;       // preconditioned norm^2 of the step's right-hand side
    double rz, dq, alpha, beta;
    int iter, done, status, nonpd;
    double last_resid;
    int passes;          // loop passes of a graph-launched step (a guard on its while loop)
    long long tc_wait;   // cycles before a wait of the tensor-core apply gives up (0: its default)
    int tc_where[6];     // the first wait of the apply that ran out: site, CTA, stage, index, parity, thread
};

struct CoilDev {
    // sizes
    int N, W, B, n_types;
    int has_grid, Gr, Gz;
    int thermal, jc_model, precision;
    long long ld;                 // leading dimension (elements) of the far operator
    // element data (element order)
    const double *r, *area, *jc_factor, *strain;
    const double *strain_pow;     // |strain|^p_eps per element
    // per element, rounded once at coil creation for the mixed form's FP32
    // pointwise chain: (2 pi r, 1 / (2 pi r), area, 1 / area) and |strain|^p_eps;
    // pi r^2 in FP64 (the flux-change term of R)
    const float4 *geo_f;
    const float *strain_pow_f;
    const double *pir2;
    int lorentz;                  // the hoop strain is on (inv_Y > 0)
    const int *mat;               // 1 filament, 0 Cu
    const int *elem_grid;         // i_z * Gr + i_r
    const int *grid_elem;         // inverse map
    const int *block_type;        // near-block type per block
    const int *constrained;       // 1 if the block is a transport turn
    const double *near;           // n_types x B x B, FP64 intra-wire blocks of M
    const float *nearf;           // the same in FP32 (wires of B <= kMedMax)
    const void *Mfar;             // N x ld far operator in `precision` (dense format)
    // block-Toeplitz format of a regular solenoid: far operator entries
    // tab32[(t_i - t_j + NT - 1)][c_i][c_j] (FP32, intra-wire entries zero),
    // element e = t * C + c; partial sums per (t tile, d chunk) in tpart
    int op_format;                // 0 dense, 1 Toeplitz (FP32), 2 Toeplitz (tensor cores)
    int C, NT;
    const float *tab32;
    float *tpart;
    float *pT;                    // operator input transposed to [c][t] (FP32)
    // tensor-core Toeplitz apply (format 2): per-CTA partial tiles
    // [cta][t][kTcTileRows], (first CTA, CTAs) per channel tile, input scale
    // exponent per turn row, table scale exponent
    const float *tc_part;
    const int2 *tc_range;
    const int *tc_pexp;
    int tc_exT;
    // one-fill apply (tc_mode 1): partial tiles part1 (tc_part, [segment][t][128])
    // and part2 ([segment][t][64]); the segments of each channel tile (l1 into
    // segs1) and of each 64-channel k block (l2 into segs2)
    int tc_mode;
    const float *tc_part2;
    const int2 *tc_l1, *tc_l2;
    const int *tc_segs1, *tc_segs2;
    // stencil: per grid column (resp. row) the first node and three weights
    const int *sr_j0, *sz_j0;
    const double *sr_w, *sz_w;
    const int4 *tap_r, *tap_z;    // per element: its stencil cells' elements, and its column / row
    // thermal grid: face conductances, capacity, Thomas factors of (I - dt/2 A)
    const double *Kr, *Kz;
    const int *nborder;           // border faces per grid cell
    double Ccell, inv_Ccell, helem;
    double src_k, inv_Tref, inv_h2;   // 4 / (rho_m c0), 1 / T_ref, 1 / helem^2 of the heat source
    double u_bath, inv_dt;            // T_bath^4, 1 / dt (0 for dt = 0)
    const double *thr_a, *thr_inv, *thr_c;    // line-solve factors (recurrence form, tridiag.cuh)
    const double *thz_a, *thz_inv, *thz_c;
    // material scalars
    double E0, nexp, Jc0, Tc, Bc2_0, B_reg, C_eps, p_eps, rho_n, rho_m, c0, h0, T_ref, T_bath;
    // the same rounded to FP32 once on the host (the FP32 pointwise chain of the
    // mixed form would otherwise convert them per element on the FP64 pipe)
    float f_E0, f_nexp, f_Jc0, f_Tc, f_Bc2_0, f_B_reg, f_C_eps, f_p_eps, f_rho_n, f_T_bath;
    double inv_Y;                 // 1 / Y_eff of the Lorentz hoop strain; 0 = static strain
    // drive of the current coil_step call
    double dt, ramp, Imax, Ba_rate, Ba_max;
    int Ba_wf;
    int maxit;
    double rtol2;
    // state and work vectors (element order unless noted)
    double *I, *Phi, *x, *res, *zv, *dv, *qv, *R, *G;
    double *qn;                   // near-block part of q, formed by the tensor-core apply's near warps
    float *pf;                    // FP32 copy of the operator input (ld long)
    double *uT, *qgrid;           // grid order [Gz][Gr]
    double *ustar, *src;          // column order [Gr][Gz] (the ADI z-lines read them)
    double *L, *y1, *sigma, *cw, *uw;   // per block
    float *Lf;                          // P_w in FP32, blocks of at most kMedMax elements:
                                        // [w][row][col] up to kSegMax, [w][col][row] above
    double *isigma;                     // 1 / sigma per block
    double *parts;                // 8 x W per-block partials (see step.cu)
    double *partT;                // per grid column partial of T_max
    long long *first_jump, *first_quench;
    // per-wire statistics (rows of W): Q_total, T_max, P_max, Q_at_jump,
    // Q_at_rise, Q_at_quench; first_rise; updated by the pointwise kernels of
    // forward steps while acc_on (the adjoint's recomputations turn it off)
    double *wstat;
    long long *first_rise;
    int acc_on;
    // subelements (J = J_H + J_I): n_groups > 1 groups the B element
    // positions of every turn (group[k]); Itr is the transport part J_I a of
    // the element currents (state), xI its resistive voltage 2 pi r rho J_I
    // after k_pointwise and its rate after k_factor; zgrp = Y S^-1 rows
    // (element x n_groups), ugrp the subelement loop voltages (W x n_groups),
    // gwt the subelements' element fractions (turn voltage = sum gwt v)
    int n_groups;
    const int *group;
    double *Itr, *xI, *zgrp, *ugrp;
    double gwt[kGroupMax];
    // warm start of a solve: the PCG starts from an extrapolation of the last
    // solutions (xprev holds x_{n-2}, xprev2 x_{n-3}).  extrap: 0 plain warm
    // start; 1 forward steps (2 x_{n-1} - x_{n-2} on the third step,
    // 3 x_{n-1} - 3 x_{n-2} + x_{n-3} from the fourth on); 2 record x only;
    // 3 linear extrapolation always; the adjoint's transposed solves, with
    // xprev and xprev2 pointing at their own history: 5 record x (both
    // histories shift), 6 linear (both shift), 4 quadratic
    double *xprev, *xprev2;
    int extrap;
    // the adjoint's replayed forward steps: rec_mode 1 (its forward pass)
    // records, in k_finalize, the solution x, the residual and the loop
    // voltages each step's finalisation used, at record (device step index -
    // rec_step0); rec_mode 2 (its recomputation of a segment) restores them in
    // place of the solve (k_replay_restore), so the recomputed states equal
    // the forward pass's bit for bit, and k_step_end keeps the forward pass's
    // solver diagnostics; rec_u holds the voltages the finalisation produced,
    // which a replayed step takes in place of forming them from y and sigma
    // (so that it needs no factorisation)
    double *rec_x, *rec_res, *rec_uw, *rec_u;
    long long rec_step0;
    int rec_mode;
    double *diag;                 // ring [cap][10]
    long long diag_cap;
    Scalars *sc;
    unsigned *ticket;             // arrival counters of the last-CTA reductions (near, update, step
                                  // end, factor, init)
};

// Smallest of the n exponents e[0..n) over a warp (every lane gets it).
__device__ __forceinline__ int warp_min_exponent(const int* e, int n, int lane) {
    int m = 1 << 30;
    for (int t0 = lane; t0 < n; t0 += 128) {           // four loads in flight per lane
        int v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = t0 + 32 * k < n ? e[t0 + 32 * k] : (1 << 30);
#pragma unroll
        for (int k = 0; k < 4; ++k) m = min(m, v[k]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
    return m;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// 1 / sqrt(a) for a > 0 in FP64 without the FP64 divide and square-root
// sequences (B300's FP64 pipe is narrow): the FP32 reciprocal square root as
// the seed, then two Newton-Raphson steps y <- y (3 - a y^2) / 2, each of
// which doubles the number of correct bits (24 -> 48 -> full precision).
// Inputs outside the FP32 exponent range take the plain expression.
__device__ __forceinline__ double rsqrt_nr(double a) {
    if (!(a > 1.0e-30 && a < 1.0e30)) return 1.0 / sqrt(a);
    double y = (double)rsqrtf((float)a);
    const double h = 0.5 * a;
    y = y * (1.5 - h * y * y);
    y = y * (1.5 - h * y * y);
    return y;
}

// 1 / a in FP64 without the FP64 divide sequence: the FP32 reciprocal as the
// seed, then two Newton-Raphson steps y <- y (2 - a y) (24 -> 48 -> full
// precision bits).  Inputs outside the FP32 exponent range take the plain
// expression.
__device__ __forceinline__ double rcp_nr(double a) {
    const double m = fabs(a);
    if (!(m > 1.0e-30 && m < 1.0e30)) return 1.0 / a;
    double y = (double)__frcp_rn((float)a);
    y = y * (2.0 - a * y);
    y = y * (2.0 - a * y);
    return y;
}

// Transport current and applied field of the drive at time t.
__device__ __forceinline__ double drive_current(const CoilDev& c, double t) {
    return fmin(c.ramp * t, c.Imax);
}

__device__ __forceinline__ double drive_field(const CoilDev& c, double t) {
    if (c.Ba_wf == 0 || c.Ba_rate == 0.0) return 0.0;
    if (c.Ba_wf == 1) return fmin(c.Ba_rate * t, c.Ba_max);
    double period = 4.0 * c.Ba_max / c.Ba_rate;
    double tau = t - period * floor(t / period);
    if (tau < 0.25 * period) return c.Ba_rate * tau;
    if (tau < 0.75 * period) return c.Ba_max - c.Ba_rate * (tau - 0.25 * period);
    return -c.Ba_max + c.Ba_rate * (tau - 0.75 * period);
}

}  // namespace cq
