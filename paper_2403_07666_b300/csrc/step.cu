// Per-step kernels of the coupled electromagnetic-thermal update.
//
// One step (linearly-implicit Euler of the loop circuit equations, Numerical
// Algorithm section; heat equation by ADI, Methods):
//   k_pointwise   field from the loop flux (3-point stencil), Jc(B,T,eps),
//                 E-J law, Joule source, right-hand side R, diagonal G,
//                 per-wire constraint right-hand side c_w, detectors
//   k_factor      per wire: Cholesky of A_w = M_ww + dt G_w, y_w = A_w^-1 1,
//                 warm start (extrapolated from the last two steps' Idot)
//                 made feasible, norm of the right-hand side
//   projected PCG (operator apply = dense far GEMV + k_near; k_init,
//                 k_update, k_direction, k_reduce)
//   k_finalize    loop voltages u_w, I += dt Idot, flux += dt M Idot
//   k_adi_r/z     Peaceman-Rachford half steps in u = T^4
//   k_step_end    diagnostic record, time advance
#include "common.cuh"
#include "pointwise.cuh"
#include "tridiag.cuh"
#include "seg.cuh"

namespace cq {

// Warm start of element e for this solve's PCG: the last solution, or its
// linear or (forward steps from the fourth on) quadratic extrapolation from
// the solutions before it (see CoilDev::extrap); the history shifts whenever
// extrap is set.  ext is uniform over the launch.
__device__ __forceinline__ double warm_start(const CoilDev& c, int e, bool ext) {
    const double x = c.x[e];
    if (!c.extrap) return x;
    const double xp = c.xprev[e];
    c.xprev[e] = x;
    if (c.extrap == 1 || c.extrap >= 4) {
        const double xp2 = c.xprev2[e];
        c.xprev2[e] = xp;
        if ((c.extrap == 1 && c.sc->step >= 3) || c.extrap == 4) return 3.0 * x - 3.0 * xp + xp2;
    }
    return ext ? 2.0 * x - xp : x;
}

// The same in two halves, so that its loads can be issued early: the values
// warm_start reads, then the extrapolation and the history shift.
struct WarmIn {
    double x, xp, xp2;
};
__device__ __forceinline__ WarmIn warm_load(const CoilDev& c, int e) {
    WarmIn w;
    w.x = c.x[e];
    w.xp = c.extrap ? c.xprev[e] : 0.0;
    w.xp2 = (c.extrap == 1 || c.extrap >= 4) ? c.xprev2[e] : 0.0;
    return w;
}
__device__ __forceinline__ double warm_finish(const CoilDev& c, int e, bool ext, const WarmIn& w) {
    if (!c.extrap) return w.x;
    c.xprev[e] = w.x;
    if (c.extrap == 1 || c.extrap >= 4) {
        c.xprev2[e] = w.xp;
        if ((c.extrap == 1 && c.sc->step >= 3) || c.extrap == 4) return 3.0 * w.x - 3.0 * w.xp + w.xp2;
    }
    return ext ? 2.0 * w.x - w.xp : w.x;
}

__device__ __forceinline__ bool extrapolate(const CoilDev& c) {
    return (c.extrap == 1 && c.sc->step >= 2) || c.extrap == 3 || c.extrap == 4 || c.extrap == 6;
}

// Detectors and per-wire statistics of wire w from its start-of-step state
// (Flux Jumps Propagation and Quenches Propagation sections): onsets of the
// flux-jump criterion max |J|/Jc > 1, of the rise of the resistivity (mean
// rho/rho_n > 0.05) and of the quench criterion (mean rho/rho_n > 0.95); the
// heat accumulated before the onset step is kept with each onset; then the
// running heat Q_total += dt P_w and the running maxima of T and q.  Forward
// steps only (acc_on); onsets are only ever set once.
__device__ __forceinline__ void wire_detectors(const CoilDev& c, int w, long long st, double dt, double pj,
                                               double jr, double mean_rho, double tmx, double qmx) {
    if (!c.acc_on) return;
    const size_t W = c.W;
    double* ws = c.wstat;
    const double Q = ws[w];
    if (c.first_jump[w] < 0 && jr > 1.0) { c.first_jump[w] = st; ws[3 * W + w] = Q; }
    if (c.first_rise[w] < 0 && mean_rho > 0.05) { c.first_rise[w] = st; ws[4 * W + w] = Q; }
    if (c.first_quench[w] < 0 && mean_rho > 0.95) { c.first_quench[w] = st; ws[5 * W + w] = Q; }
    ws[w] = Q + dt * pj;
    ws[W + w] = fmax(ws[W + w], tmx);
    ws[2 * W + w] = fmax(ws[2 * W + w], qmx);
}

// Rows a2 and a5 for element e from the start-of-step state: the field from
// the loop-flux stencil, T, Jc(B, T, eps), the E-J law; writes G, R, the
// Joule source on the thermal grid and (subelements) the resistive voltage
// of J_I, and returns what the per-wire reductions need.
struct ElemOut {
    double I, pj, tq, q, jrat, frac;   // tq: T
    int fil;
};

// The FP64 form's element (every operation FP64).
__device__ __forceinline__ ElemOut pointwise_element(const CoilDev& c, int e, double Ba0, double dBa) {
    ElemOut o;
    const double r = c.r[e], a = c.area[e];
    const int fil = c.mat[e];
    const double I = c.I[e];
    double Br = 0.0, Bz = 0.0, T = c.T_bath;
    if (c.has_grid) {
        field_at(c, e, Ba0, &Br, &Bz);
        T = sqrt(sqrt(c.uT[c.elem_grid[e]]));
    }
    const double Bm = sqrt(Br * Br + Bz * Bz);
    const double J = I / a;
    const double Jc = fil ? critical_current(c, Bm, T, strain_power(c, e, r, J, Bz), c.jc_factor[e]) : 0.0;
    double frac, dfac, jrat;
    ej_law(c, fil, J, Jc, &frac, &dfac, &jrat);
    const double rho = c.rho_n * frac;
    const double E = rho * J;
    const double q = E * J;
    c.G[e] = 2.0 * kPi * r * (c.rho_n * dfac) / a;
    c.R[e] = 2.0 * kPi * r * E + kPi * r * r * dBa;
    if (c.n_groups) c.xI[e] = 2.0 * kPi * r * rho * c.Itr[e] / a;   // resistive voltage of J_I
    if (c.has_grid) c.qgrid[c.elem_grid[e]] = q;
    o.tq = T;
    o.I = I;
    o.pj = q * 2.0 * kPi * r * a;
    o.q = q;
    o.jrat = jrat;
    o.frac = frac;
    o.fil = fil;
    return o;
}

// The mixed form's element, FP64 kept to the flux stencil, the loop's
// right-hand side R and the current sum: the stencil takes the loop flux alone
// and adds the applied field afterwards (the 3-point derivative reproduces
// pi r^2 B_a exactly: B_z gains B_a, B_r nothing), and E, q, G, the Joule
// power and the reductions of the wire are FP32.  Returns q and the Joule
// power in FP32, u = T^4 and I in FP64.
struct ElemOutF {
    double I, u;
    float pj, q, jrat, frac;
    int fil;
};

// Flux derivative of the 3-point stencil along one grid axis, in FP64 (the
// loop fluxes cancel across one element), from the element's precomputed tap
// elements: no FP64 compare is spent on zero weights (each FP64 instruction
// takes a B300 scheduler 64 cycles); a tap outside the grid has a zero weight
// and names the element itself, so it adds an exact zero.
__device__ __forceinline__ double stencil_taps(const CoilDev& c, const double* w3, int4 t) {
    double d = w3[0] * c.Phi[t.x];
    d = fma(w3[1], c.Phi[t.y], d);
    return fma(w3[2], c.Phi[t.z], d);
}

__device__ __forceinline__ ElemOutF pointwise_element_f(const CoilDev& c, int e, float Ba0, double dBa) {
    ElemOutF o;
    const float4 gf = c.geo_f[e];                          // 2 pi r, 1 / (2 pi r), area, 1 / area
    const float tpr = gf.x, inv2pir = gf.y, a = gf.z, ia = gf.w;
    const int fil = c.mat[e];
    const double I = c.I[e];
    float Br = 0.0f, Bz = 0.0f, T = c.f_T_bath;
    double u = c.u_bath;
    if (c.has_grid) {
        const int g = c.elem_grid[e];
        // the stencil cells' elements precomputed: two rounds of loads instead of four
        const int4 tr = c.tap_r[e], tz = c.tap_z[e];
        const double dr = stencil_taps(c, c.sr_w + 3 * tr.w, tr);
        const double dz = stencil_taps(c, c.sz_w + 3 * tz.w, tz);
        Bz = (float)dr * inv2pir + Ba0;
        Br = -(float)dz * inv2pir;
        u = c.uT[g];
        T = sqrtf(sqrtf((float)u));
    } else {
        Bz = Ba0;
    }
    const float Bm = sqrtf(Br * Br + Bz * Bz);
    const float J = (float)I * ia;
    const float Jc = fil ? critical_current_f(c, Bm, T, strain_power_f(c, e, J, Bz), (float)c.jc_factor[e])
                         : 0.0f;
    float frac, dfac, jrat;
    ej_law_f(c, fil, fabsf(J), Jc, &frac, &dfac, &jrat);
    const float rn = c.f_rho_n;
    const float rho = rn * frac;
    const float E = rho * J;
    const float q = E * J;
    c.G[e] = (double)(tpr * (rn * dfac) * ia);
    c.R[e] = fma(c.pir2[e], dBa, (double)(tpr * E));
    if (c.n_groups) c.xI[e] = (double)(tpr * rho * ia) * c.Itr[e];   // resistive voltage of J_I
    if (c.has_grid) c.qgrid[c.elem_grid[e]] = (double)q;
    o.I = I;
    o.u = u;
    o.pj = q * tpr * a;
    o.q = q;
    o.jrat = jrat;
    o.frac = frac;
    o.fil = fil;
    return o;
}

__device__ __forceinline__ float seg_sumf(float v, int Bp) {
    for (int o = Bp >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float seg_maxf(float v, int Bp) {
    for (int o = Bp >> 1; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// Maximum of non-negative doubles through their bit patterns (ordered like
// the values): no FP64 instruction.
__device__ __forceinline__ long long seg_max_bits(long long v, int Bp) {
    for (int o = Bp >> 1; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// The wire's maximum temperature from the maximum of tq (the fourth root of
// a maximum of u is the maximum of the fourth roots).
// One warp per block (wire).  Partials: P[0] Joule power, P[1] max |J|/Jc,
// P[2] mean rho/rho_n of filament elements.
__global__ void k_pointwise(const CoilDev* __restrict__ cds) {
    const CoilDev& c = cds[blockIdx.y];
    double* parts = c.parts;
    int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (w >= c.W || c.B <= kSegMax) return;
    const bool F32 = c.precision != PREC_FP64;      // the mixed form's FP32 chain
    Scalars* sc = c.sc;
    double t0 = sc->t, dt = c.dt, t1 = t0 + dt;
    double It1 = drive_current(c, t1);
    double Ba0 = drive_field(c, t0), Ba1 = drive_field(c, t1);
    double dBa = F32 ? (Ba1 - Ba0) * c.inv_dt : (Ba1 - Ba0) / dt;
    if (w == 0 && lane == 0) {
        sc->It1 = It1; sc->Ba0 = Ba0; sc->Ba1 = Ba1; sc->dBa = dBa;
        sc->nonpd = 0;                         // k_factor of this step sets it again if needed
    }
    double sumI = 0.0, pj = 0.0, jr = 0.0, rhof = 0.0, nfil = 0.0, tmx = 0.0, qmx = 0.0;
    if (F32) {
        // the mixed form's FP32 element and reductions (as in k_pointwise_seg)
        float pjf = 0.f, jrf = 0.f, rhf = 0.f, nf = 0.f, qf = 0.f;
        long long ub = 0;
        for (int k = lane; k < c.B; k += 32) {
            const ElemOutF o = pointwise_element_f(c, w * c.B + k, (float)Ba0, dBa);
            sumI += o.I;
            pjf += o.pj;
            qf = fmaxf(qf, o.q);
            ub = max(ub, __double_as_longlong(o.u));
            if (o.fil) { jrf = fmaxf(jrf, o.jrat); rhf += o.frac; nf += 1.0f; }
        }
        sumI = warp_sum(sumI);
        pj = (double)seg_sumf(pjf, 32);
        jr = (double)seg_maxf(jrf, 32);
        rhof = (double)seg_sumf(rhf, 32);
        nfil = (double)seg_sumf(nf, 32);
        qmx = (double)seg_maxf(qf, 32);
        const long long umax = seg_max_bits(ub, 32);
        if (lane == 0) tmx = (double)sqrtf(sqrtf((float)__longlong_as_double(umax)));
    } else {
        for (int k = lane; k < c.B; k += 32) {
            const ElemOut o = pointwise_element(c, w * c.B + k, Ba0, dBa);
            sumI += o.I;
            pj += o.pj;
            tmx = fmax(tmx, o.tq);
            qmx = fmax(qmx, o.q);
            if (o.fil) { jr = fmax(jr, o.jrat); rhof += o.frac; nfil += 1.0; }
        }
        sumI = warp_sum(sumI);
        pj = warp_sum(pj);
        jr = warp_max(jr);
        rhof = warp_sum(rhof);
        nfil = warp_sum(nfil);
        tmx = warp_max(tmx);
        qmx = warp_max(qmx);
    }
    if (lane == 0) {
        // the mixed form without FP64 divisions (B300's FP64 pipe): c_w through
        // 1/dt, the wire-mean rho/rho_n (FP32 sums) in FP32
        const bool f32 = c.precision != PREC_FP64;
        c.cw[w] = c.constrained[w] ? (f32 ? (It1 - sumI) * c.inv_dt : (It1 - sumI) / dt) : 0.0;
        double mean_rho = nfil > 0.0 ? (f32 ? (double)((float)rhof / (float)nfil) : rhof / nfil) : 0.0;
        parts[0 * (size_t)c.W + w] = pj;
        parts[1 * (size_t)c.W + w] = jr;
        parts[2 * (size_t)c.W + w] = mean_rho;
        wire_detectors(c, w, sc->step, dt, pj, jr, mean_rho, tmx, qmx);
    }
}

// --------------------------------------------------- per-wire block algebra

// Solve L L^T v = v in place (L lower, B x B row-major in shared memory, its
// diagonal stored as reciprocals: FP64 division is slow on B300's FP64 pipe).
// Blocks of up to 32 elements keep v in registers, one element per lane,
// and broadcast each solved entry with a shuffle.
__device__ void chol_solve_warp(const double* L, double* v, int B, int lane) {
    if (B <= 32) {
        double x = lane < B ? v[lane] : 0.0;
        for (int k = 0; k < B; ++k) {
            double xk = __shfl_sync(0xffffffffu, x, k) * L[k * B + k];
            if (lane == k) x = xk;
            else if (lane > k && lane < B) x -= L[lane * B + k] * xk;
        }
        for (int k = B - 1; k >= 0; --k) {
            double xk = __shfl_sync(0xffffffffu, x, k) * L[k * B + k];
            if (lane == k) x = xk;
            else if (lane < k) x -= L[k * B + lane] * xk;
        }
        __syncwarp();
        if (lane < B) v[lane] = x;
        __syncwarp();
        return;
    }
    for (int k = 0; k < B; ++k) {
        if (lane == 0) v[k] *= L[k * B + k];
        __syncwarp();
        double vk = v[k];
        for (int i = k + 1 + lane; i < B; i += 32) v[i] -= L[i * B + k] * vk;
        __syncwarp();
    }
    for (int k = B - 1; k >= 0; --k) {
        if (lane == 0) v[k] *= L[k * B + k];
        __syncwarp();
        double vk = v[k];
        for (int i = lane; i < k; i += 32) v[i] -= L[k * B + i] * vk;
        __syncwarp();
    }
}

__device__ double warp_block_sum(const double* v, int B, int lane) {
    double s = 0.0;
    for (int k = lane; k < B; k += 32) s += v[k];
    return warp_sum(s);
}

// Projected preconditioner of block w: v <- A_w^-1 v, then remove the
// component that would change the wire's total current (constrained wires).
__device__ void project_precond(const CoilDev& c, int w, const double* L, const double* y, double* v,
                                int lane) {
    int B = c.B;
    chol_solve_warp(L, v, B, lane);
    if (!c.constrained[w]) return;
    if (c.n_groups) {
        // subelements: remove Y S^-1 Q^T A_w^-1 r (the part that changes a
        // subelement's net current), with the stored rows Z = Y S^-1
        const int S = c.n_groups;
        double n[kGroupMax];
#pragma unroll
        for (int g = 0; g < kGroupMax; ++g) {
            double a = 0.0;
            if (g < S)
                for (int k = lane; k < B; k += 32) a += c.group[k] == g ? v[k] : 0.0;
            n[g] = g < S ? warp_sum(a) : 0.0;
        }
        for (int k = lane; k < B; k += 32) {
            const double* Z = c.zgrp + ((size_t)w * B + k) * S;
            double corr = 0.0;
            for (int g = 0; g < S; ++g) corr += Z[g] * n[g];
            v[k] -= corr;
        }
        __syncwarp();
        return;
    }
    double s = warp_block_sum(v, B, lane);
    double f = s * c.isigma[w];
    for (int k = lane; k < B; k += 32) v[k] -= y[k] * f;
    __syncwarp();
}

// Subelement part of k_factor (blocks of more than kSegMax elements), from the
// Cholesky factor L of A_w in shared memory, y = A_w^-1 1 and sigma:
//  * the transport part on the turn alone, x_I = y u - A_w^-1 R_I,
//    u = (c_w + 1^T A_w^-1 R_I) / sigma (R_I in xI on entry, x_I replaces it),
//    and its subelement nets d = Q^T x_I;
//  * Y = A_w^-1 Q (one solve per subelement), S_m = Q^T Y, S_m^-1 by
//    Gauss-Jordan with a row per lane, and the stored rows Z = Y S_m^-1;
//  * R^T P_w R + d^T S_m^-1 d (P_w = A_w^-1 - Z Y^T on constrained turns), and
//    the warm start moved onto Q^T x = d.
// ws: shared scratch of B S + S S doubles after v and y.
__device__ void factor_groups_big(const CoilDev& c, int w, const double* L, const double* y, double* v, double* ws,
                                  double sig, int lane) {
    const int B = c.B, S = c.n_groups;
    const int con = c.constrained[w];
    double* Ysm = ws;                 // [B][S]
    double* Sm = ws + B * S;          // [S][S], inverted in place
    // transport part
    for (int k = lane; k < B; k += 32) v[k] = c.xI[w * B + k];
    __syncwarp();
    chol_solve_warp(L, v, B, lane);
    const double uI = (c.cw[w] + warp_block_sum(v, B, lane)) / sig;
    double d[kGroupMax];
#pragma unroll
    for (int g = 0; g < kGroupMax; ++g) d[g] = 0.0;
    for (int k = lane; k < B; k += 32) {
        const double xI = con ? y[k] * uI - v[k] : 0.0;
        c.xI[w * B + k] = xI;
        const int gk = c.group[k];
#pragma unroll
        for (int g = 0; g < kGroupMax; ++g)
            if (g == gk) d[g] += xI;
    }
#pragma unroll
    for (int g = 0; g < kGroupMax; ++g) d[g] = g < S ? warp_sum(d[g]) : 0.0;
    __syncwarp();
    // Y = A_w^-1 Q
    for (int g = 0; g < S; ++g) {
        for (int k = lane; k < B; k += 32) v[k] = c.group[k] == g ? 1.0 : 0.0;
        __syncwarp();
        chol_solve_warp(L, v, B, lane);
        for (int k = lane; k < B; k += 32) Ysm[k * S + g] = v[k];
        __syncwarp();
    }
    // S_m = Q^T Y and its inverse
    for (int p = lane; p < S * S; p += 32) {
        const int g = p / S, h = p - g * S;
        double a = 0.0;
        for (int k = 0; k < B; ++k)
            if (c.group[k] == g) a += Ysm[k * S + h];
        Sm[p] = a;
    }
    __syncwarp();
    int bad = 0;
    for (int kp = 0; kp < S; ++kp) {
        double piv = Sm[kp * S + kp];
        if (!(piv > 0.0)) { bad = 1; piv = 1.0; }
        const double ip = 1.0 / piv;
        const double f = lane < S ? Sm[lane * S + kp] : 0.0;
        __syncwarp();
        if (lane == kp)
            for (int j = 0; j < S; ++j) Sm[kp * S + j] = j == kp ? ip : Sm[kp * S + j] * ip;
        __syncwarp();
        if (lane < S && lane != kp)
            for (int j = 0; j < S; ++j) Sm[lane * S + j] = j == kp ? -f * ip : Sm[lane * S + j] - f * Sm[kp * S + j];
        __syncwarp();
    }
    if (bad && con && lane == 0) atomicExch(&c.sc->nonpd, 1);
    // Z = Y S_m^-1
    for (int k = lane; k < B; k += 32) {
        double* Z = c.zgrp + ((size_t)w * B + k) * S;
        for (int h = 0; h < S; ++h) {
            double a = 0.0;
            for (int g = 0; g < S; ++g) a += Ysm[k * S + g] * Sm[g * S + h];
            Z[h] = a;
        }
    }
    __syncwarp();
    // R^T P_w R: v = R, A_w^-1 v, then the subelement projection
    for (int k = lane; k < B; k += 32) v[k] = c.R[w * B + k];
    __syncwarp();
    project_precond(c, w, L, y, v, lane);
    double rn = 0.0;
    for (int k = lane; k < B; k += 32) rn += c.R[w * B + k] * v[k];
    rn = warp_sum(rn);
    double dSd = 0.0;
    for (int g = 0; g < S; ++g)
        for (int h = 0; h < S; ++h) dSd += d[g] * Sm[g * S + h] * d[h];
    // warm start, then moved onto Q^T x = d
    const bool ext = extrapolate(c);
    double gap[kGroupMax];
#pragma unroll
    for (int g = 0; g < kGroupMax; ++g) gap[g] = 0.0;
    for (int k = lane; k < B; k += 32) {
        const double x0 = warm_start(c, w * B + k, ext);
        c.x[w * B + k] = x0;
        const int gk = c.group[k];
#pragma unroll
        for (int g = 0; g < kGroupMax; ++g)
            if (g == gk) gap[g] += x0;
    }
#pragma unroll
    for (int g = 0; g < kGroupMax; ++g) gap[g] = g < S ? d[g] - warp_sum(gap[g]) : 0.0;
    for (int k = lane; k < B; k += 32) {
        const int e = w * B + k;
        double xe = c.x[e];
        if (con) {
            const double* Z = c.zgrp + (size_t)e * S;
            for (int g = 0; g < S; ++g) xe += Z[g] * gap[g];
        }
        c.x[e] = xe;
        c.pf[e] = (float)xe;
    }
    if (lane == 0) c.parts[3 * (size_t)c.W + w] = rn + (con ? dSd : 0.0);
}

// One warp per CTA, one CTA per block.  Shared: A (B*B), v (B), y (B), and
// with subelements the scratch of factor_groups_big.
__global__ void k_factor(const CoilDev* __restrict__ cds) {
    const CoilDev& c = cds[blockIdx.y];
    double* parts = c.parts;
    int w = blockIdx.x;
    if (w >= c.W || c.B <= kSegMax || (c.B <= kMedMax && c.n_groups == 0)) return;
    extern __shared__ double sm[];
    int B = c.B, lane = threadIdx.x;
    double* A = sm;
    double* v = sm + B * B;
    double* y = v + B;
    const double* nb = c.near + (size_t)c.block_type[w] * B * B;
    for (int i = lane; i < B * B; i += 32) A[i] = nb[i];
    __syncwarp();
    for (int k = lane; k < B; k += 32) A[k * B + k] += c.dt * c.G[w * B + k];
    __syncwarp();
    int bad = 0;
    for (int k = 0; k < B; ++k) {
        double piv = A[k * B + k];
        if (!(piv > 0.0)) { bad = 1; piv = 1.0; }
        double rkk = rsqrt_nr(piv);                    // the factor keeps 1 / L_kk on its diagonal
        __syncwarp();
        if (lane == 0) A[k * B + k] = rkk;
        for (int i = k + 1 + lane; i < B; i += 32) A[i * B + k] *= rkk;
        __syncwarp();
        for (int i = k + 1 + lane; i < B; i += 32) {
            double lik = A[i * B + k];
            for (int j = k + 1; j <= i; ++j) A[i * B + j] -= lik * A[j * B + k];
        }
        __syncwarp();
    }
    if (bad && lane == 0) atomicExch(&c.sc->nonpd, 1);
    double* Lg = c.L + (size_t)w * B * B;
    for (int i = lane; i < B * B; i += 32) Lg[i] = A[i];
    // y = A_w^-1 1, sigma = 1^T y
    for (int k = lane; k < B; k += 32) y[k] = 1.0;
    __syncwarp();
    chol_solve_warp(A, y, B, lane);
    double sig = warp_block_sum(y, B, lane);
    for (int k = lane; k < B; k += 32) c.y1[w * B + k] = y[k];
    if (lane == 0) {
        c.sigma[w] = sig;
        c.isigma[w] = 1.0 / sig;
    }
    __syncwarp();
    if (c.n_groups) {
        factor_groups_big(c, w, A, y, v, y + B, sig, lane);
        return;
    }
    // preconditioned norm^2 of the right-hand side: R^T Pproj(R) + c_w^2 / sigma
    for (int k = lane; k < B; k += 32) v[k] = c.R[w * B + k];
    __syncwarp();
    chol_solve_warp(A, v, B, lane);
    double cw = c.cw[w];
    int con = c.constrained[w];
    if (con) {
        double s = warp_block_sum(v, B, lane);
        double f = s / sig;
        for (int k = lane; k < B; k += 32) v[k] -= y[k] * f;
        __syncwarp();
    }
    double rn = 0.0;
    for (int k = lane; k < B; k += 32) rn += c.R[w * B + k] * v[k];
    rn = warp_sum(rn);
    // warm start from the previous steps' Idot, moved onto this step's constraint
    const bool ext = extrapolate(c);
    double sx = 0.0;
    for (int k = lane; k < B; k += 32) {
        const double x0 = warm_start(c, w * B + k, ext);
        c.x[w * B + k] = x0;
        sx += x0;
    }
    sx = warp_sum(sx);
    double corr = con ? (cw - sx) / sig : 0.0;
    for (int k = lane; k < B; k += 32) {
        int e = w * B + k;
        double xe = c.x[e] + corr * y[k];
        c.x[e] = xe;
        c.pf[e] = (float)xe;
    }
    if (lane == 0) parts[3 * (size_t)c.W + w] = rn + (con ? cw * cw / sig : 0.0);
}

// q_w += (M_ww + dt G_w) p_w for every block; optional partial p^T q.
__global__ void k_near(const CoilDev* __restrict__ cds, int which) {
    const CoilDev& c = cds[blockIdx.y];
    double* parts = c.parts;
    if (c.sc->done || c.B <= kSegMax || (c.B <= kMedMax && c.n_groups == 0)) return;
    int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (w >= c.W) return;
    const double* p = which == 0 ? c.x : c.dv;
    int B = c.B;
    const double* nb = c.near + (size_t)c.block_type[w] * B * B;
    const double* pw = p + (size_t)w * B;
    double dot = 0.0;
    for (int i = lane; i < B; i += 32) {
        double acc = 0.0;
        for (int j = 0; j < B; ++j) acc += nb[i * B + j] * pw[j];
        int e = w * B + i;
        acc += c.dt * c.G[e] * pw[i];
        double qe = c.qv[e] + acc;
        c.qv[e] = qe;
        dot += pw[i] * qe;
    }
    dot = warp_sum(dot);
    if (which == 1 && lane == 0) parts[4 * (size_t)c.W + w] = dot;
}

// Residual update of a constrained block (residual held in v): remove the
// multiplier component u 1 (u = y^T r / sigma, the loop-voltage estimate) and
// accumulate it in uw[w].  The projected preconditioner ignores that
// component in exact arithmetic; removing it keeps r small so that r^T z
// does not drown in the rounding of the large loop-voltage term
// (Gould, Hribar and Nocedal's residual update for constraint preconditioners).
__device__ void project_residual(const CoilDev& c, int w, const double* y, double* v, int lane, bool first) {
    int B = c.B;
    if (c.n_groups) {
        // subelements: remove Q u, u = Z^T r the subelement voltage estimates,
        // accumulated in ugrp
        const int S = c.n_groups;
        const int con = c.constrained[w];
        double u[kGroupMax];
#pragma unroll
        for (int g = 0; g < kGroupMax; ++g) {
            double a = 0.0;
            if (g < S)
                for (int k = lane; k < B; k += 32) a += c.zgrp[((size_t)w * B + k) * S + g] * v[k];
            u[g] = g < S ? warp_sum(a) : 0.0;
        }
        if (con) {
            for (int k = lane; k < B; k += 32) {
                const int gk = c.group[k];
                double ug = 0.0;
#pragma unroll
                for (int g = 0; g < kGroupMax; ++g)
                    if (g == gk) ug = u[g];
                v[k] -= ug;
            }
        }
        __syncwarp();
        if (lane == 0) {
            for (int g = 0; g < S; ++g) {
                double* U = c.ugrp + (size_t)w * S + g;
                if (first) *U = con ? u[g] : 0.0;
                else if (con) *U += u[g];
            }
        }
        return;
    }
    if (!c.constrained[w]) return;
    double s = 0.0;
    for (int k = lane; k < B; k += 32) s += y[k] * v[k];
    s = warp_sum(s);
    double u = s * c.isigma[w];
    for (int k = lane; k < B; k += 32) v[k] -= u;
    __syncwarp();
    if (lane == 0) c.uw[w] = first ? u : c.uw[w] + u;
}

// After q = A x0: r = q + R (projected), z = Pproj(r), d = -z; partial r^T z.
__global__ void k_init(const CoilDev* __restrict__ cds) {
    const CoilDev& c = cds[blockIdx.y];
    double* parts = c.parts;
    if (c.sc->done || c.B <= kSegMax || (c.B <= kMedMax && c.n_groups == 0)) return;
    int w = blockIdx.x;
    if (w >= c.W) return;
    extern __shared__ double sm[];
    int B = c.B, lane = threadIdx.x;
    double* L = sm;
    double* v = sm + B * B;
    double* y = v + B;
    const double* Lg = c.L + (size_t)w * B * B;
    for (int i = lane; i < B * B; i += 32) L[i] = Lg[i];
    for (int k = lane; k < B; k += 32) {
        int e = w * B + k;
        v[k] = c.qv[e] + c.R[e];
        y[k] = c.y1[e];
    }
    __syncwarp();
    if (lane == 0) c.uw[w] = 0.0;
    project_residual(c, w, y, v, lane, true);
    for (int k = lane; k < B; k += 32) c.res[w * B + k] = v[k];
    __syncwarp();
    project_precond(c, w, L, y, v, lane);
    double rz = 0.0;
    for (int k = lane; k < B; k += 32) {
        int e = w * B + k;
        c.zv[e] = v[k];
        c.dv[e] = -v[k];
        c.pf[e] = (float)(-v[k]);
        rz += c.res[e] * v[k];
    }
    rz = warp_sum(rz);
    if (lane == 0) parts[4 * (size_t)c.W + w] = rz;
}

// x += alpha d, r += alpha q (projected), z = Pproj(r); partial r^T z.
__global__ void k_update(const CoilDev* __restrict__ cds) {
    const CoilDev& c = cds[blockIdx.y];
    double* parts = c.parts;
    if (c.sc->done || c.B <= kSegMax || (c.B <= kMedMax && c.n_groups == 0)) return;
    int w = blockIdx.x;
    if (w >= c.W) return;
    extern __shared__ double sm[];
    int B = c.B, lane = threadIdx.x;
    double* L = sm;
    double* v = sm + B * B;
    double* y = v + B;
    double alpha = c.sc->alpha;
    const double* Lg = c.L + (size_t)w * B * B;
    for (int i = lane; i < B * B; i += 32) L[i] = Lg[i];
    for (int k = lane; k < B; k += 32) {
        int e = w * B + k;
        c.x[e] += alpha * c.dv[e];
        v[k] = c.res[e] + alpha * c.qv[e];
        y[k] = c.y1[e];
    }
    __syncwarp();
    project_residual(c, w, y, v, lane, false);
    for (int k = lane; k < B; k += 32) c.res[w * B + k] = v[k];
    __syncwarp();
    project_precond(c, w, L, y, v, lane);
    double rz = 0.0;
    for (int k = lane; k < B; k += 32) {
        int e = w * B + k;
        c.zv[e] = v[k];
        rz += c.res[e] * v[k];
    }
    rz = warp_sum(rz);
    if (lane == 0) parts[4 * (size_t)c.W + w] = rz;
}

// ---- blocks of kSegMax + 1 .. kMedMax elements without subelements -------
// One CTA of kMedMax threads per block, thread t holding element (row) t: the
// per-wire algebra of the shared-warp kernels (FP32 Gauss-Jordan inverse of
// A_w = M_ww + dt G_w, the projected preconditioner P_w stored in FP32, the
// FP64 residual and projections) with every FP64 operation spread over the
// block's rows instead of a warp's loops over them, and no Cholesky factor.
enum ReduceMode { RED_SCALE = 0, RED_INIT = 1, RED_ALPHA = 2, RED_BETA = 3 };
__device__ bool fused_reduce(const CoilDev& c, double head_value, unsigned* ticket, int n_cta, int mode);
__device__ __forceinline__ double tc_far_sum(const CoilDev& c, int e, double inv, int2 rg);
__device__ void loop_condition(const CoilDev& c, cudaGraphConditionalHandle h);

__device__ __forceinline__ bool is_med(const CoilDev& c) {
    return c.B > kSegMax && c.B <= kMedMax && c.n_groups == 0;
}

// Sum over the CTA's NT threads in a fixed order, the result on every thread.
template <int NT = kMedMax>
__device__ __forceinline__ double med_sum(double v, double* sh) {
    v = warp_sum(v);
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
#pragma unroll
    for (int k = 0; k < NT / 32; ++k) r += sh[k];
    __syncthreads();
    return r;
}

// Factor of one medium wire with rows padded to NP >= B slots, two threads per
// row (thread 2t + h holds slots h NP/2 .. h NP/2 + NP/2 - 1 of row t).  The
// FP32 Gauss-Jordan inverse runs rotated so that every register index is
// static: at step k the pivot column sits in slot 0, each row moves one slot to
// the left and the new entry of column k enters at slot NP - 1, so after the B
// steps slot s holds column (s + B) mod NP; the columns from B on of a real row
// start and stay exactly zero.  The row that pivots next publishes itself and
// the reciprocal of its pivot through a double buffer in shared memory: one
// barrier per step.
template <int NP>
__device__ __forceinline__ void factor_med_body(const CoilDev& c, int w, float (*prow)[kMedMax + 4], float* ip_s,
                                                float* ys, float* rs, double* sh, int* bad_any, int fuse_scale) {
    constexpr int H = NP / 2;
    // the second half-row starts 16 bytes further on where NP/2 floats would put
    // it in the first half's banks
    constexpr int HO = H % 32 == 0 ? H + 4 : H;
    constexpr unsigned kFull = 0xffffffffu;
    const int B = c.B, t = threadIdx.x >> 1, h = threadIdx.x & 1, e = w * B + t;
    const bool ev = t < B;
    // the self block is symmetric entry for entry, so row t is read as column t
    const float* nb = c.nearf + (size_t)c.block_type[w] * B * B + (ev ? t : 0);
    float a[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
        const int j = h * H + i;
        a[i] = (ev && j < B) ? nb[(size_t)j * B] : 0.f;
    }
    if (ev) {
        const float g = (float)(c.dt * c.G[e]);
#pragma unroll
        for (int i = 0; i < H; ++i)
            if (h * H + i == t) a[i] += g;
    }
    auto publish = [&](int b) {                 // this row as the next pivot row
        float4* q = reinterpret_cast<float4*>(prow[b] + h * HO);
#pragma unroll
        for (int q4 = 0; q4 < H / 4; ++q4) q[q4] = make_float4(a[4 * q4], a[4 * q4 + 1], a[4 * q4 + 2], a[4 * q4 + 3]);
        if (h == 0) {
            // without pivoting: A_w is SPD, every pivot a positive Schur
            // complement; a non-positive one flags the step as the Cholesky does
            float piv = a[0];
            if (!(piv > 0.f)) {
                *bad_any = 1;
                piv = 1.f;
            }
            ip_s[b] = 1.f / piv;
        }
    };
    if (t == 0) publish(0);
    for (int k = 0; k < B; ++k) {
        __syncthreads();
        const int b = k & 1;
        const float ip = ip_s[b];
        // the partner's first slot: slot NP/2 of the row for h = 0, slot 0 for h = 1
        const float o = __shfl_xor_sync(kFull, a[0], 1);
        const float tail = h ? 0.f : o;
        if (t == k) {
#pragma unroll
            for (int i = 0; i + 1 < H; ++i) a[i] = a[i + 1] * ip;
            a[H - 1] = h ? ip : tail * ip;
        } else if (ev) {
            const float g = (h ? o : a[0]) * ip;
            const float* pr = prow[b] + h * HO;
            const float4* q = reinterpret_cast<const float4*>(pr);
            const float pend = h ? 1.f : pr[HO];         // the slot after this half (1: column k's own entry)
            float4 v = q[0];
#pragma unroll
            for (int q4 = 0; q4 < H / 4; ++q4) {
                const float4 vn = q4 + 1 < H / 4 ? q[q4 + 1] : make_float4(pend, 0.f, 0.f, 0.f);
                a[4 * q4] = fmaf(-g, v.y, a[4 * q4 + 1]);
                a[4 * q4 + 1] = fmaf(-g, v.z, a[4 * q4 + 2]);
                a[4 * q4 + 2] = fmaf(-g, v.w, a[4 * q4 + 3]);
                a[4 * q4 + 3] = fmaf(-g, vn.x, 4 * q4 + 4 < H ? a[(4 * q4 + 4) % H] : tail);
                v = vn;
            }
        }
        if (t == k + 1 && k + 1 < B) publish(b ^ 1);
    }
    __syncthreads();
    if (*bad_any && threadIdx.x == 0) {
        atomicExch(&c.sc->nonpd, 1);
        __threadfence();                       // before this CTA's arrival on a fused reduction
    }
    // y = A_w^-1 1 (row sums of the symmetric inverse), sigma = 1^T y
    float yt = 0.f;
#pragma unroll
    for (int i = 0; i < H; ++i) yt += a[i];
    yt += __shfl_xor_sync(kFull, yt, 1);
    const bool lead = ev && h == 0;
    const double y = ev ? (double)yt : 0.0;
    const double sig = med_sum<kMedFactorThreads>(lead ? y : 0.0, sh);
    const double isg = 1.0 / sig;
    const int con = c.constrained[w];
    if (lead) c.y1[e] = y;
    if (threadIdx.x == 0) {
        c.sigma[w] = sig;
        c.isigma[w] = isg;
    }
    const double x0 = lead ? warm_start(c, e, extrapolate(c)) : 0.0;   // before the constraint
    // P_w row t, stored; R^T P_w R in FP32 (it only scales the stopping test)
    const double R = ev ? c.R[e] : 0.0;
    if (h == 0) {
        rs[t] = (float)R;
        ys[t] = (float)y;
    }
    __syncthreads();
    const float yis = (float)(y * isg);
    float pr0 = 0.f, pr1 = 0.f;
    // stored column by column ([w][j][t]: row t of P_w at stride B), so that the
    // block's threads write, and later read, consecutive words
    float* Pw = c.Lf + (size_t)w * B * B + (ev ? t : 0);
#pragma unroll
    for (int i = 0; i < H; ++i) {
        const int sl = h * H + i;
        const int j = sl + B - (sl + B >= NP ? NP : 0);      // the column in slot sl
        if (j < B) {
            const float pj = con ? a[i] - yis * ys[j] : a[i];
            if (ev) Pw[(size_t)j * B] = pj;
            if (i & 1) pr1 = fmaf(pj, rs[j], pr1);
            else pr0 = fmaf(pj, rs[j], pr0);
        }
    }
    float prt = pr0 + pr1;
    prt += __shfl_xor_sync(kFull, prt, 1);
    const double rn = med_sum<kMedFactorThreads>(lead ? R * (double)prt : 0.0, sh);
    const double cw = c.cw[w];
    // warm start moved onto this step's constraint
    const double sx = med_sum<kMedFactorThreads>(x0, sh);
    const double corr = con ? (cw - sx) * isg : 0.0;
    if (lead) {
        const double xe = x0 + corr * y;
        c.x[e] = xe;
        c.pf[e] = (float)xe;
    }
    const double scale = rn + (con ? cw * cw * isg : 0.0);
    if (threadIdx.x == 0) c.parts[3 * (size_t)c.W + w] = scale;
    if (fuse_scale) fused_reduce(c, threadIdx.x == 0 ? scale : 0.0, c.ticket + 3, c.W, RED_SCALE);
}

// fuse_scale: the last CTA sums the scale partials and starts the solve's
// scalars (the k_reduce SCALE step).
__global__ void __launch_bounds__(kMedFactorThreads, 6) k_factor_med(const CoilDev* __restrict__ cds, int fuse_scale) {
    const CoilDev& c = cds[blockIdx.y];
    const int w = blockIdx.x;
    if (w >= c.W || !is_med(c)) return;
    __shared__ __align__(16) float prow[2][kMedMax + 4];
    __shared__ float ip_s[2];
    __shared__ float ys[kMedMax];
    __shared__ float rs[kMedMax];
    __shared__ double sh[kMedFactorThreads / 32];
    __shared__ int bad_any;
    if (threadIdx.x == 0) bad_any = 0;
    if (c.B <= 32) factor_med_body<32>(c, w, prow, ip_s, ys, rs, sh, &bad_any, fuse_scale);
    else if (c.B <= 48) factor_med_body<48>(c, w, prow, ip_s, ys, rs, sh, &bad_any, fuse_scale);
    else factor_med_body<kMedMax>(c, w, prow, ip_s, ys, rs, sh, &bad_any, fuse_scale);
}

// Row t of a B x B block stored column by column (entry (t, j) at col[j B])
// against the vector v in shared memory (zero from B on), for B <= NP: the
// loads unrolled over NP slots and issued ahead of their products, four
// partial sums.
template <int NP, typename T>
__device__ __forceinline__ T med_row_dot_n(const T* col, const T* v, int B) {
    constexpr int CH = sizeof(T) == 4 ? NP : 16;   // loads in flight: the FP32 row, or 16 FP64
    T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int j0 = 0; j0 < NP; j0 += CH) {
        T m[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) m[u] = j0 + u < B ? __ldg(col + (size_t)(j0 + u) * B) : T(0);
#pragma unroll
        for (int u = 0; u < CH; ++u)
            if (j0 + u < NP) acc[u & 3] = fma(m[u], v[j0 + u], acc[u & 3]);
    }
    return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}
template <typename T>
__device__ __forceinline__ T med_row_dot(const T* col, const T* v, int B) {
    if (B <= 32) return med_row_dot_n<32>(col, v, B);
    if (B <= 48) return med_row_dot_n<48>(col, v, B);
    return med_row_dot_n<kMedMax>(col, v, B);
}

// Projected residual update and preconditioner of the block (thread t holds
// element t; v the raw residual): writes res, returns z and the block's r^T z.
// con, isg: the wire's constraint flag and 1 / sigma (loaded ahead); with
// lane_rz the thread's own term of r^T z is returned in rz.
__device__ __forceinline__ double med_residual_precond(const CoilDev& c, int w, double v, double y, bool first,
                                                       double* rz, float* vf_s, double* sh, int con, double isg,
                                                       bool lane_rz) {
    const int B = c.B, t = threadIdx.x, e = w * B + t;
    const bool ev = t < B;
    // residual update: remove u 1, u = y^T r / sigma, accumulated in uw
    const double u = med_sum(ev ? y * v : 0.0, sh) * isg;
    if (con && ev) v -= u;
    if (t == 0) {
        if (first) c.uw[w] = con ? u : 0.0;
        else if (con) c.uw[w] += u;
    }
    if (ev) c.res[e] = v;
    // z = P_w r: the row of the stored FP32 P_w against r in FP32
    vf_s[t] = ev ? (float)v : 0.f;
    __syncthreads();
    // (row t of P_w at stride B, see k_factor_med)
    double z = ev ? (double)med_row_dot(c.Lf + (size_t)w * B * B + t, vf_s, B) : 0.0;
    // the FP32 rounding's component along the constrained direction, removed in FP64
    const double sz = med_sum(z, sh);
    if (con && ev) z -= y * sz * isg;
    *rz = ev ? v * z : 0.0;
    if (!lane_rz) *rz = med_sum(*rz, sh);
    return z;
}

// After q = A x0: r = q + R (projected), z = P_w r, d = -z; r^T z, reduced
// by the last CTA when fuse_init (the k_reduce INIT step).
__global__ void __launch_bounds__(kMedMax) k_init_med(const CoilDev* __restrict__ cds, int fuse_init) {
    const CoilDev& c = cds[blockIdx.y];
    const int w = blockIdx.x;
    if (c.sc->done || w >= c.W || !is_med(c)) return;    // CTA-uniform
    __shared__ float vf_s[kMedMax];
    __shared__ double sh[kMedMax / 32];
    const int t = threadIdx.x, e = w * c.B + t;
    const bool ev = t < c.B;
    const double v = ev ? c.qv[e] + c.R[e] : 0.0;
    const double y = ev ? c.y1[e] : 0.0;
    double rz;
    const double z = med_residual_precond(c, w, v, y, true, &rz, vf_s, sh, c.constrained[w], c.isigma[w],
                                          fuse_init != 0);
    if (ev) {
        c.zv[e] = z;
        c.dv[e] = -z;
        c.pf[e] = (float)(-z);
    }
    if (fuse_init) fused_reduce(c, rz, c.ticket + 4, c.W, RED_INIT);
    else if (t == 0) c.parts[4 * (size_t)c.W + w] = rz;
}

// x += alpha d, r += alpha q (projected), z = P_w r; r^T z, reduced by the
// last CTA when fuse_beta (the k_reduce BETA step; with use_cond it also sets
// the PCG loop's condition, as k_update_seg does).
__global__ void __launch_bounds__(kMedMax)
k_update_med(const CoilDev* __restrict__ cds, int fuse_beta, cudaGraphConditionalHandle cond, int use_cond) {
    const CoilDev& c = cds[blockIdx.y];
    const int w = blockIdx.x;
    if (w >= c.W || !is_med(c)) {
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) loop_condition(c, cond);
        return;
    }
    __shared__ float vf_s[kMedMax];
    __shared__ double sh[kMedMax / 32];
    const int t = threadIdx.x, e = w * c.B + t;
    const bool ev = t < c.B;
    // what does not depend on the solve's progress, loaded with its done flag
    double xv = 0.0, dv = 0.0, rv = 0.0, qv = 0.0, y = 0.0;
    if (ev) {
        xv = c.x[e];
        dv = c.dv[e];
        rv = c.res[e];
        qv = c.qv[e];
        y = c.y1[e];
    }
    const int con = c.constrained[w];
    const double isg = c.isigma[w];
    const double alpha = c.sc->alpha;
    if (c.sc->done) {                                    // CTA-uniform
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) loop_condition(c, cond);
        return;
    }
    double v = 0.0;
    if (ev) {
        c.x[e] = xv + alpha * dv;
        v = rv + alpha * qv;
    }
    double rz;
    const double z = med_residual_precond(c, w, v, y, false, &rz, vf_s, sh, con, isg, fuse_beta != 0);
    if (ev) c.zv[e] = z;
    if (!fuse_beta) {
        if (t == 0) c.parts[4 * (size_t)c.W + w] = rz;
    } else if (fused_reduce(c, rz, c.ticket + 1, c.W, RED_BETA) && use_cond && threadIdx.x == 0) {
        loop_condition(c, cond);
    }
}

// q_w += (M_ww + dt G_w) p_w (FP64, row t on thread t), the far part taken
// from the tensor-core apply's partial tiles when far_tiles; p^T q, reduced by
// the last CTA when fuse_alpha (the k_reduce ALPHA step).
__global__ void __launch_bounds__(kMedMax) k_near_med(const CoilDev* __restrict__ cds, int which, int far_tiles,
                                                      int fuse_alpha) {
    const CoilDev& c = cds[blockIdx.y];
    const int w = blockIdx.x;
    if (w >= c.W || !is_med(c)) return;                  // CTA-uniform
    __shared__ double ps[kMedMax];
    __shared__ double sh[kMedMax / 32];
    const int B = c.B, t = threadIdx.x, e = w * B + t;
    const bool ev = t < B;
    // what does not depend on the solve's progress, loaded with its done flag
    const double* p = which == 0 ? c.x : c.dv;
    const double pv = ev ? p[e] : 0.0;
    const double ge = ev ? c.G[e] : 0.0;
    const int bt = c.block_type[w];
    const int xmin = far_tiles ? warp_min_exponent(c.tc_pexp, c.NT, threadIdx.x & 31) : 0;
    const int2 rg = (far_tiles && ev && c.tc_mode != 1) ? c.tc_range[(e % c.C) / kTcTileRows] : make_int2(0, 0);
    if (c.sc->done) return;                              // CTA-uniform
    ps[t] = pv;
    __syncthreads();
    double dot = 0.0;
    if (ev) {
        // row t read as column t (the self block is symmetric entry for entry):
        // consecutive threads, consecutive words
        const double acc = med_row_dot(c.near + (size_t)bt * B * B + t, ps, B) + c.dt * ge * pv;
        const double far = far_tiles ? tc_far_sum(c, e, ldexp(1.0, -(c.tc_exT + xmin)), rg) : c.qv[e];
        const double qe = far + acc;
        c.qv[e] = qe;
        dot = pv * qe;
    }
    if (fuse_alpha) {
        fused_reduce(c, which == 1 ? dot : 0.0, c.ticket, c.W, RED_ALPHA);
    } else {
        dot = med_sum(dot, sh);
        if (which == 1 && t == 0) c.parts[4 * (size_t)c.W + w] = dot;
    }
}

__device__ double block_reduce_sum(double v, double* sh) {
    v = warp_sum(v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    v = threadIdx.x < nw ? sh[threadIdx.x] : 0.0;
    if (wid == 0) v = warp_sum(v);
    __syncthreads();
    return v;
}

__device__ double block_reduce_max(double v, double* sh) {
    v = warp_max(v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    v = threadIdx.x < nw ? sh[threadIdx.x] : -1.0e308;
    if (wid == 0) v = warp_max(v);
    __syncthreads();
    return v;
}

// Deterministic sum of a partial array a[0..W) by one CTA (any size) and the
// scalar update that follows it.
__device__ void reduce_and_update(const CoilDev& c, int mode, const double* a, int W) {
    Scalars* sc = c.sc;
    if ((mode == RED_ALPHA || mode == RED_BETA || mode == RED_INIT) && sc->done) return;
    __shared__ double sh[32];
    // the scalars the update needs, loaded while the partials are (it runs
    // on the tail of a kernel, one CTA, every round trip in sequence)
    double rz_old = 0.0, scale2 = 0.0;
    int iter = 0;
    if (threadIdx.x == 0) {
        rz_old = sc->rz;
        scale2 = sc->scale2;
        iter = sc->iter;
    }
    // eight loads in flight per thread, summed in a fixed order
    double s0 = 0.0, s1 = 0.0;
    const int st = blockDim.x;
    for (int i0 = threadIdx.x; i0 < W; i0 += 8 * st) {
        double v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = i0 + k * st < W ? __ldcg(a + i0 + k * st) : 0.0;   // from L2
        s0 += ((v[0] + v[1]) + (v[2] + v[3]));
        s1 += ((v[4] + v[5]) + (v[6] + v[7]));
    }
    double s = block_reduce_sum(s0 + s1, sh);
    if (threadIdx.x != 0) return;
    if (mode == RED_SCALE) {
        sc->scale2 = s;
        sc->done = 0;
        sc->iter = 0;
        sc->passes = 0;
        sc->status = ST_OK;
        if (sc->nonpd) { sc->status = ST_NONFINITE; sc->done = 1; }
        if (!(s == s)) { sc->status = ST_NONFINITE; sc->done = 1; }
    } else if (mode == RED_INIT) {
        // (the relative residual sqrt(rz / scale2) is formed once per step, by k_step_end)
        sc->rz = s;
        if (!(s == s)) { sc->status = ST_NONFINITE; sc->done = 1; }
        else if (s <= c.rtol2 * scale2) sc->done = 1;
    } else if (mode == RED_ALPHA) {
        sc->dq = s;
        if (!(s > 0.0)) {                      // A is SPD on the feasible subspace
            sc->status = ST_NONFINITE;
            sc->done = 1;
            return;
        }
        sc->alpha = rz_old / s;
    } else {
        double rz_new = s;
        sc->iter = iter + 1;
        sc->beta = rz_new / rz_old;
        sc->rz = rz_new;
        if (!(rz_new == rz_new)) { sc->status = ST_NONFINITE; sc->done = 1; }
        else if (rz_new <= c.rtol2 * scale2) sc->done = 1;
        else if (iter + 1 >= c.maxit) { sc->status = ST_NOT_CONVERGED; sc->done = 1; }
    }
}

// One CTA per coil; skip_seg: coils whose kernels reduce their partials
// themselves (last CTA: the shared-warp and medium-wire kernels) are left
// alone (2: of the shared-warp coils only those without subelements, whose
// factor kernel does; the subelement factor does not).
__global__ void __launch_bounds__(1024) k_reduce(const CoilDev* __restrict__ cds, int mode, int skip_seg) {
    const CoilDev& c = cds[blockIdx.x];
    if (skip_seg && (is_med(c) || (c.B <= kSegMax && (skip_seg == 1 || c.n_groups == 0)))) return;
    reduce_and_update(c, mode, c.parts + (mode == RED_SCALE ? 3 : 4) * (size_t)c.W, c.W);
}

// Condition of a graph-launched step's PCG while loop: go on while the solve
// is not done; a pass count past maxit + 2 (which the scalar updates never
// let happen) ends it as not converged, so the loop always terminates.  One
// thread, once per pass.
__device__ void loop_condition(const CoilDev& c, cudaGraphConditionalHandle h) {
    Scalars* sc = c.sc;
    const int p = ++sc->passes;
    if (!sc->done && p > c.maxit + 2) {
        sc->status = ST_NOT_CONVERGED;
        sc->done = 1;
    }
    cudaGraphSetConditional(h, sc->done ? 0u : 1u);
}

// Fused reduction of a value held by every lane (its term of a dot product):
// every thread of the coil's first n_cta CTAs calls this.  Each CTA sums its
// lanes in a fixed order (butterfly per warp, then warps in order)
// into parts row 7 at its index; the CTA that arrives last on the counter
// (which it resets for the next launch) sums those n_cta values and does the
// scalar update of `mode`; true in that CTA.  The counter's release/acquire
// orders every CTA's partial store before the last CTA's loads.
__device__ bool fused_reduce(const CoilDev& c, double head_value, unsigned* ticket, int n_cta, int mode) {
    __shared__ double wsum[32];
    __shared__ int is_last;
    const double v = warp_sum(head_value);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
    __syncthreads();
    double* ctap = c.parts + 7 * (size_t)c.W;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
        ctap[blockIdx.x] = t;
        // release: the partial is visible before the count moves; acquire (in
        // the CTA that arrives last): every other CTA's partial is visible to
        // this thread, and through the barrier below to the rest of its CTA
        unsigned prev;
        asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(prev) : "l"(ticket) : "memory");
        is_last = prev == (unsigned)n_cta - 1u;
        if (is_last) *ticket = 0u;
    }
    __syncthreads();
    if (!is_last) return false;
    reduce_and_update(c, mode, ctap, n_cta);
    return true;
}

// ------------------------------------------ blocks of at most 16 elements
//
// The same three kernels with 32 / Bp wires per warp (Bp = B rounded up to a
// power of two): lane kk of a Bp-lane segment holds element kk of the
// segment's wire, the triangular solves broadcast inside the segment, and
// sums are xor-butterflies over the segment.  Every FP64 operation on an
// element is the one of the one-wire-per-warp kernels in the same order (the
// butterflies there only added the idle lanes' zeros), but each FP64 warp
// instruction now serves 32 / Bp wires: B300's FP64 pipe is narrow.

// (seg_width, seg_sum, Seg, seg_of and near_row_product: seg.cuh)

// Far-operator value at element e of the tensor-core Toeplitz apply: the sum
// of the partial tiles of the CTAs that worked on e's channel tile, in a fixed
// order, times 2^-(exT + xmin).  The sum runs on
// the FP32 pipe with Kahan's compensated summation and returns s - comp in
// FP64: about twice FP32's precision for these few terms, at a fraction of
// the cost of FP64 additions on B300.
__device__ __forceinline__ void kahan_add(float v, float& s, float& comp) {
    const float y = v - comp;
    const float t = s + y;
    comp = (t - s) - y;
    s = t;
}
__device__ __forceinline__ double tc_far_sum(const CoilDev& c, int e, double inv, int2 rg) {
    const int t = e / c.C, cc = e - t * c.C;
    if (c.tc_mode == 1) {
        // one-fill apply: the segments of e's channel tile, then of its k block
        const int2 r1 = c.tc_l1[cc / kTcTileRows], r2 = c.tc_l2[cc / 64];
        const float* p1 = c.tc_part + (size_t)t * kTcTileRows + (cc % kTcTileRows);
        const float* p2 = c.tc_part2 + (size_t)t * 64 + (cc % 64);
        const size_t t1 = (size_t)c.NT * kTcTileRows, t2 = (size_t)c.NT * 64;
        float s = 0.f, comp = 0.f;
        int k = 0;
        for (; k + 8 <= r1.y; k += 8) {
            float v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = p1[(size_t)c.tc_segs1[r1.x + k + i] * t1];
#pragma unroll
            for (int i = 0; i < 8; ++i) kahan_add(v[i], s, comp);
        }
        for (; k < r1.y; ++k) kahan_add(p1[(size_t)c.tc_segs1[r1.x + k] * t1], s, comp);
        for (k = 0; k + 8 <= r2.y; k += 8) {
            float v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = p2[(size_t)c.tc_segs2[r2.x + k + i] * t2];
#pragma unroll
            for (int i = 0; i < 8; ++i) kahan_add(v[i], s, comp);
        }
        for (; k < r2.y; ++k) kahan_add(p2[(size_t)c.tc_segs2[r2.x + k] * t2], s, comp);
        return ((double)s - (double)comp) * inv;
    }
    const size_t tile = (size_t)c.NT * kTcTileRows;      // (rg = tc_range[cc / kTcTileRows])
    const float* p = c.tc_part + (size_t)rg.x * tile + (size_t)t * kTcTileRows + (cc % kTcTileRows);
    // the loads of up to 24 tiles issued before their sums (one round trip for
    // the usual 18 CTAs per tile), added in tile order
    float s = 0.f, comp = 0.f;
    for (int k = 0; k < rg.y; k += 24) {
        float v[24];
#pragma unroll
        for (int i = 0; i < 24; ++i) v[i] = k + i < rg.y ? p[(size_t)(k + i) * tile] : 0.f;
#pragma unroll
        for (int i = 0; i < 24; ++i)
            if (k + i < rg.y) kahan_add(v[i], s, comp);
    }
    return ((double)s - (double)comp) * inv;
}

// q_w += (M_ww + dt G_w) p_w; optional partial p^T q (as k_near).
// far_tiles: the far part comes from the tensor-core apply's partial tiles
// (its separate reduction was skipped) instead of q.  fuse_alpha: the last
// CTA sums the p^T q partials and sets alpha (the k_reduce ALPHA step).
// near_pre: the near-block part (with dt G p) was formed by the tensor-core
// apply's near warps into qn (the same operations, see near_row_product).
__global__ void k_near_seg(const CoilDev* __restrict__ cds, int which, int far_tiles, int fuse_alpha,
                           int near_pre) {
    const CoilDev& c = cds[blockIdx.y];
    const int per_cta = (int)(blockDim.x >> 5) * (32 / seg_width(c.B));   // wires per CTA
    const int n_cta = (c.W + per_cta - 1) / per_cta;
    if (c.B > kSegMax || (int)blockIdx.x >= n_cta) return;
    const int wg = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const bool warp_on = wg * (32 / seg_width(c.B)) < c.W;   // warp-uniform
    const Seg s = seg_of(c, wg);
    // what does not depend on the solve's progress is loaded together with its
    // done flag: one round trip instead of several in sequence
    const double* p = which == 0 ? c.x : c.dv;
    const double pv = s.ev ? p[s.e] : 0.0;
    const double ge = (s.ev && !near_pre) ? c.G[s.e] : 0.0;
    const double qn = (s.ev && near_pre) ? c.qn[s.e] : 0.0;
    const int bt = c.block_type[s.wv ? s.w : 0];
    const int xmin = far_tiles ? warp_min_exponent(c.tc_pexp, c.NT, threadIdx.x & 31) : 0;
    const int2 rg = (far_tiles && s.ev && c.tc_mode != 1) ? c.tc_range[(s.e % c.C) / kTcTileRows] : make_int2(0, 0);
    if (c.sc->done) return;                             // CTA-uniform
    double head = 0.0;                                  // the lane's term of p^T q (fused reduction)
    if (warp_on) {
        const double inv = far_tiles ? ldexp(1.0, -(c.tc_exT + xmin)) : 0.0;
        const double acc = near_pre ? qn : near_row_product(c, s, bt, pv, ge);
        double dot = 0.0;
        if (s.ev) {
            double qe = (far_tiles ? tc_far_sum(c, s.e, inv, rg) : c.qv[s.e]) + acc;
            c.qv[s.e] = qe;
            dot = pv * qe;
        }
        if (fuse_alpha) {
            head = which == 1 ? dot : 0.0;              // only the total is needed: no per-wire sums
        } else {
            dot = seg_sum(dot, s.Bp);
            if (which == 1 && s.kk == 0 && s.wv) c.parts[4 * (size_t)c.W + s.w] = dot;
        }
    }
    if (fuse_alpha) fused_reduce(c, head, c.ticket, n_cta, RED_ALPHA);
}

// A lane's per-wire inputs of the preconditioner, loaded ahead of the values
// they act on: the wire's constraint flag, 1 / sigma and (16-element wires)
// row kk of P_w.
struct SegRow {
    int con;
    double isg;
    float4 p[kSegMax / 4];
};
__device__ __forceinline__ SegRow seg_row_load(const CoilDev& c, const Seg& s) {
    SegRow r;
    r.con = s.wv ? c.constrained[s.w] : 0;
    r.isg = s.wv ? c.isigma[s.w] : 0.0;
    if (s.B == kSegMax) {
        const float4* P = reinterpret_cast<const float4*>(c.Lf + ((size_t)(s.wv ? s.w : 0) * s.B + s.kk) * s.B);
#pragma unroll
        for (int q = 0; q < kSegMax / 4; ++q) r.p[q] = P[q];
    }
    return r;
}

// Projected residual update and preconditioner of the segment's wire: v is
// the raw residual on entry; writes res, z and returns z (in rz the wire's
// r^T z, or with lane_rz the lane's own term of it).
__device__ __forceinline__ double seg_residual_precond(const CoilDev& c, const Seg& s, double v, double y,
                                                        bool first, double* rz, bool lane_rz, const SegRow& pre) {
    const int con = pre.con;
    if (c.n_groups) {
        // subelements: remove Q v, v = (Y S^-1)^T r the subelement voltage
        // estimates, accumulated in ugrp
        const int S = c.n_groups;
        const int gk = s.ev ? c.group[s.kk] : -1;
        const double* Z = c.zgrp + (size_t)(s.ev ? s.e : 0) * S;
        double mine = 0.0;
#pragma unroll
        for (int g = 0; g < kGroupMaxSeg; ++g) {
            if (g < S) {
                const double vg = seg_sum(s.ev ? Z[g] * v : 0.0, s.Bp);
                if (g == gk) mine = vg;
                if (s.kk == 0 && s.wv) {
                    double* U = c.ugrp + (size_t)s.w * S + g;
                    if (first) *U = con ? vg : 0.0;
                    else if (con) *U += vg;
                }
            }
        }
        if (con && s.ev) v -= mine;
    } else {
        const double isg = pre.isg;
        // residual update: remove u 1, u = y^T r / sigma, accumulated in uw
        const double u = seg_sum(y * v, s.Bp) * isg;
        if (con && s.ev) v -= u;
        if (s.kk == 0 && s.wv) {
            if (first) c.uw[s.w] = con ? u : 0.0;
            else if (con) c.uw[s.w] += u;
        }
    }
    if (s.ev) c.res[s.e] = v;
    // z = P_w r (P_w = A_w^-1 minus, on constrained wires, the component that
    // changes the wire's total current; stored by k_factor_seg in FP32): B
    // independent FP32 products per lane, two partial sums.  The preconditioner
    // needs no more (the residual stays FP64, so the solution does not depend on
    // it), but the iterates must stay feasible: the FP32 rounding's component
    // along the constrained directions is removed in FP64.
    const float* P = c.Lf + ((size_t)(s.wv ? s.w : 0) * s.B + (s.kk < s.B ? s.kk : 0)) * s.B;
    const float vf = (float)v;
    float z0 = 0.f, z1 = 0.f;
    if (s.B == kSegMax) {
        // 16-element wires: the row as four 16-byte loads (made ahead, see seg_row_load)
        const float4* pr = pre.p;
#pragma unroll
        for (int q = 0; q < kSegMax / 4; ++q) {
            z0 = fmaf(pr[q].x, __shfl_sync(0xffffffffu, vf, s.base + 4 * q), z0);
            z1 = fmaf(pr[q].y, __shfl_sync(0xffffffffu, vf, s.base + 4 * q + 1), z1);
            z0 = fmaf(pr[q].z, __shfl_sync(0xffffffffu, vf, s.base + 4 * q + 2), z0);
            z1 = fmaf(pr[q].w, __shfl_sync(0xffffffffu, vf, s.base + 4 * q + 3), z1);
        }
    } else {
        for (int j = 0; j + 1 < s.B; j += 2) {
            z0 = fmaf(P[j], __shfl_sync(0xffffffffu, vf, s.base + j), z0);
            z1 = fmaf(P[j + 1], __shfl_sync(0xffffffffu, vf, s.base + j + 1), z1);
        }
        if (s.B & 1) z0 = fmaf(P[s.B - 1], __shfl_sync(0xffffffffu, vf, s.base + s.B - 1), z0);
    }
    double z = s.ev ? (double)(z0 + z1) : 0.0;
    if (c.n_groups) {
        const int S = c.n_groups;
        const int gk = s.ev ? c.group[s.kk] : -1;
        const double* Z = c.zgrp + (size_t)(s.ev ? s.e : 0) * S;
        double corr = 0.0;
#pragma unroll
        for (int g = 0; g < kGroupMaxSeg; ++g)
            if (g < S) {
                const double ng = seg_sum(gk == g ? z : 0.0, s.Bp);
                if (s.ev) corr += Z[g] * ng;
            }
        if (con) z -= corr;
    } else {
        const double sz = seg_sum(z, s.Bp);            // all lanes: the shuffles span the warp
        if (con) z -= y * sz * pre.isg;
    }
    *rz = s.ev ? v * z : 0.0;
    if (!lane_rz) *rz = seg_sum(*rz, s.Bp);
    return z;
}

// fuse_init: the last CTA sums the r^T z partials and sets the initial
// residual and the convergence flag (the k_reduce INIT step).  fuse_near:
// q = A x0 is formed here first, as k_near_seg (which = 0) forms it with the
// same operations (far_tiles, near_pre as there), instead of read from q.
__global__ void __launch_bounds__(32 * kSegWarps)
k_init_seg(const CoilDev* __restrict__ cds, int fuse_init, int fuse_near, int far_tiles, int near_pre) {
    const CoilDev& c = cds[blockIdx.y];
    const int per_cta = kSegWarps * (32 / seg_width(c.B));   // wires per CTA
    const int n_cta = (c.W + per_cta - 1) / per_cta;
    if (c.sc->done || c.B > kSegMax || (int)blockIdx.x >= n_cta) return;
    const int warp = threadIdx.x >> 5;
    const int wg = blockIdx.x * kSegWarps + warp;
    double head = 0.0;                                  // the lane's term of r^T z (fused reduction)
    if (wg * (32 / seg_width(c.B)) < c.W) {             // warp-uniform
        const Seg s = seg_of(c, wg);
        double qx = 0.0;
        if (fuse_near) {
            const double pv = s.ev ? c.x[s.e] : 0.0;
            const double ge = (s.ev && !near_pre) ? c.G[s.e] : 0.0;
            const double qn = (s.ev && near_pre) ? c.qn[s.e] : 0.0;
            const int bt = c.block_type[s.wv ? s.w : 0];
            const int xmin = far_tiles ? warp_min_exponent(c.tc_pexp, c.NT, threadIdx.x & 31) : 0;
            const int2 rg =
                (far_tiles && s.ev && c.tc_mode != 1) ? c.tc_range[(s.e % c.C) / kTcTileRows] : make_int2(0, 0);
            const double inv = far_tiles ? ldexp(1.0, -(c.tc_exT + xmin)) : 0.0;
            const double acc = near_pre ? qn : near_row_product(c, s, bt, pv, ge);
            if (s.ev) {
                qx = (far_tiles ? tc_far_sum(c, s.e, inv, rg) : c.qv[s.e]) + acc;
                c.qv[s.e] = qx;
            }
        } else if (s.ev) {
            qx = c.qv[s.e];
        }
        const double v = s.ev ? qx + c.R[s.e] : 0.0;
        const double y = s.ev ? c.y1[s.e] : 0.0;
        double rz;
        const double z = seg_residual_precond(c, s, v, y, true, &rz, fuse_init != 0, seg_row_load(c, s));
        if (s.ev) {
            c.zv[s.e] = z;
            c.dv[s.e] = -z;
            c.pf[s.e] = (float)(-z);
        }
        if (fuse_init) head = rz;
        else if (s.kk == 0 && s.wv) c.parts[4 * (size_t)c.W + s.w] = rz;
    }
    if (fuse_init) fused_reduce(c, head, c.ticket + 4, n_cta, RED_INIT);
}

// fuse_beta: the last CTA sums the r^T z partials and sets beta and the
// convergence flags (the k_reduce BETA step).  use_cond (one coil, a
// graph-launched step): that CTA (CTA 0 when the solve was already done) also
// sets the PCG loop's condition, in place of k_loop_cond.
__global__ void __launch_bounds__(32 * kSegWarps)
k_update_seg(const CoilDev* __restrict__ cds, int fuse_beta, cudaGraphConditionalHandle cond, int use_cond) {
    const CoilDev& c = cds[blockIdx.y];
    const int per_cta = kSegWarps * (32 / seg_width(c.B));   // wires per CTA
    const int n_cta = (c.W + per_cta - 1) / per_cta;
    if (c.B > kSegMax || (int)blockIdx.x >= n_cta) {
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) loop_condition(c, cond);
        return;
    }
    const int warp = threadIdx.x >> 5;
    const int wg = blockIdx.x * kSegWarps + warp;
    const bool warp_on = wg * (32 / seg_width(c.B)) < c.W;   // warp-uniform
    const Seg s = seg_of(c, wg);
    // what does not depend on the solve's progress is loaded together with its
    // done flag and alpha: one round trip instead of several in sequence
    double xv = 0.0, dv = 0.0, rv = 0.0, qv = 0.0, y = 0.0;
    if (s.ev) {
        xv = c.x[s.e];
        dv = c.dv[s.e];
        rv = c.res[s.e];
        qv = c.qv[s.e];
        y = c.y1[s.e];
    }
    const SegRow pre = seg_row_load(c, s);
    const double alpha = c.sc->alpha;
    if (c.sc->done) {                                   // CTA-uniform
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) loop_condition(c, cond);
        return;
    }
    double head = 0.0;                                  // the lane's term of r^T z (fused reduction)
    if (warp_on) {
        double v = 0.0;
        if (s.ev) {
            c.x[s.e] = xv + alpha * dv;
            v = rv + alpha * qv;
        }
        double rz;
        const double z = seg_residual_precond(c, s, v, y, false, &rz, fuse_beta != 0, pre);
        if (s.ev) c.zv[s.e] = z;
        if (fuse_beta) head = rz;                   // the lane's term: only the total is needed
        else if (s.kk == 0 && s.wv) c.parts[4 * (size_t)c.W + s.w] = rz;
    }
    if (fuse_beta && fused_reduce(c, head, c.ticket + 1, n_cta, RED_BETA) && use_cond && threadIdx.x == 0)
        loop_condition(c, cond);
}

__device__ __forceinline__ double seg_max(double v, int Bp) {
    for (int o = Bp >> 1; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// k_pointwise for blocks of at most 16 elements (32 / Bp wires per warp).
__global__ void k_pointwise_seg(const CoilDev* __restrict__ cds) {
    const CoilDev& c = cds[blockIdx.y];
    if (c.B > kSegMax) return;
    const int wg = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wg * (32 / seg_width(c.B)) >= c.W) return;       // warp-uniform; no CTA barrier below
    const Seg s = seg_of(c, wg);
    Scalars* sc = c.sc;
    const double t0 = sc->t, dt = c.dt, t1 = t0 + dt;
    // the drive once per warp (FP64 on one lane), broadcast
    double It1 = 0.0, Ba0 = 0.0, Ba1 = 0.0, dBa = 0.0;
    if ((threadIdx.x & 31) == 0) {
        It1 = drive_current(c, t1);
        Ba0 = drive_field(c, t0);
        Ba1 = drive_field(c, t1);
        dBa = c.precision != PREC_FP64 ? (Ba1 - Ba0) * c.inv_dt : (Ba1 - Ba0) / dt;
    }
    It1 = __shfl_sync(0xffffffffu, It1, 0);
    Ba0 = __shfl_sync(0xffffffffu, Ba0, 0);
    Ba1 = __shfl_sync(0xffffffffu, Ba1, 0);
    dBa = __shfl_sync(0xffffffffu, dBa, 0);
    if (s.w == 0 && s.kk == 0) {
        sc->It1 = It1; sc->Ba0 = Ba0; sc->Ba1 = Ba1; sc->dBa = dBa;
        sc->nonpd = 0;                         // k_factor of this step sets it again if needed
    }
    double sumI = 0.0, pj = 0.0, jr = 0.0, mean_rho = 0.0, tmx = 0.0, qmx = 0.0;
    const bool f32 = c.precision != PREC_FP64;
    if (f32) {
        // the mixed form's FP32 chain; the current sum stays FP64
        float pjf = 0.f, jrf = 0.f, rhf = 0.f, nf = 0.f, qf = 0.f;
        long long ub = 0;
        if (s.ev) {
            const ElemOutF o = pointwise_element_f(c, s.e, (float)Ba0, dBa);
            sumI = o.I;
            pjf = o.pj;
            qf = o.q;
            ub = __double_as_longlong(o.u);
            if (o.fil) { jrf = o.jrat; rhf = o.frac; nf = 1.0f; }
        }
        sumI = seg_sum(sumI, s.Bp);
        pj = (double)seg_sumf(pjf, s.Bp);
        jr = (double)seg_maxf(jrf, s.Bp);
        const float rs = seg_sumf(rhf, s.Bp), ns = seg_sumf(nf, s.Bp);
        mean_rho = ns > 0.0f ? (double)(rs / ns) : 0.0;   // the wire mean, divided in FP32
        const long long umax = seg_max_bits(ub, s.Bp);
        if (s.kk == 0) tmx = (double)sqrtf(sqrtf((float)__longlong_as_double(umax)));   // the head lane's
        qmx = (double)seg_maxf(qf, s.Bp);
    } else {
        double rhof = 0.0, nfil = 0.0;
        if (s.ev) {
            const ElemOut o = pointwise_element(c, s.e, Ba0, dBa);
            sumI = o.I;
            pj = o.pj;
            tmx = o.tq;
            qmx = o.q;
            if (o.fil) { jr = o.jrat; rhof = o.frac; nfil = 1.0; }
        }
        sumI = seg_sum(sumI, s.Bp);
        pj = seg_sum(pj, s.Bp);
        jr = seg_max(jr, s.Bp);
        rhof = seg_sum(rhof, s.Bp);
        nfil = seg_sum(nfil, s.Bp);
        tmx = seg_max(tmx, s.Bp);
        qmx = seg_max(qmx, s.Bp);
        if (s.kk == 0) mean_rho = nfil > 0.0 ? rhof / nfil : 0.0;
    }
    if (s.kk == 0 && s.wv) {
        const int w = s.w;
        double* parts = c.parts;
        c.cw[w] = c.constrained[w] ? (f32 ? (It1 - sumI) * c.inv_dt : (It1 - sumI) / dt) : 0.0;
        parts[0 * (size_t)c.W + w] = pj;
        parts[1 * (size_t)c.W + w] = jr;
        parts[2 * (size_t)c.W + w] = mean_rho;
        wire_detectors(c, w, sc->step, dt, pj, jr, mean_rho, tmx, qmx);
    }
}

// Subelement part of k_factor_seg (J = J_H + J_I), from row kk of A_w^-1 in
// a, y = A_w^-1 1 and 1 / sigma:
//  * the transport part on the turn alone, x_I = y u - A_w^-1 R_I with
//    u = (c_w + 1^T A_w^-1 R_I) / sigma (R_I, the resistive voltage of J_I,
//    is in xI on entry; x_I replaces it) and its subelement nets d = Q^T x_I;
//  * Y = A_w^-1 Q, S_m = Q^T Y (Q: element-to-subelement incidence), S_m^-1
//    by Gauss-Jordan in every lane (at most kGroupMaxSeg^2 registers), the rows
//    Z = Y S_m^-1 (stored) and P_w = A_w^-1 - Z Y^T (stored, constrained turns);
//  * R^T P_w R + d^T S_m^-1 d, and the warm start moved onto Q^T x = d.
__device__ __forceinline__ void factor_groups(const CoilDev& c, const Seg& s, const double (&a)[kSegMax], double y,
                                           double isg, int con, double xe0) {
    const int B = s.B, kk = s.kk, w = s.w, e = s.e, S = c.n_groups;
    const int gk = s.ev ? c.group[kk] : -1;
    const double RI = s.ev ? c.xI[e] : 0.0;
    double t = 0.0;
#pragma unroll
    for (int j = 0; j < kSegMax; ++j)
        if (j < B) t += a[j] * __shfl_sync(0xffffffffu, RI, s.base + j);
    const double cw = s.wv ? c.cw[w] : 0.0;
    const double uI = (cw + seg_sum(s.ev ? t : 0.0, s.Bp)) * isg;
    const double xI = (con && s.ev) ? y * uI - t : 0.0;
    if (s.ev) c.xI[e] = xI;
    double Yv[kGroupMaxSeg];
#pragma unroll
    for (int g = 0; g < kGroupMaxSeg; ++g) Yv[g] = 0.0;
#pragma unroll
    for (int j = 0; j < kSegMax; ++j) {
        if (j < B) {
            const int gj = c.group[j];
#pragma unroll
            for (int g = 0; g < kGroupMaxSeg; ++g)
                if (g == gj) Yv[g] += a[j];
        }
    }
    if (!s.ev) {
#pragma unroll
        for (int g = 0; g < kGroupMaxSeg; ++g) Yv[g] = 0.0;
    }
    double Sm[kGroupMaxSeg][kGroupMaxSeg];
#pragma unroll
    for (int g = 0; g < kGroupMaxSeg; ++g) {
#pragma unroll
        for (int h = 0; h < kGroupMaxSeg; ++h) {
            if (h < g) continue;
            double v = (g == h) ? 1.0 : 0.0;             // identity on the padding
            if (g < S && h < S) v = seg_sum(gk == g ? Yv[h] : 0.0, s.Bp);
            Sm[g][h] = v;
            Sm[h][g] = v;
        }
    }
    int bad = 0;
#pragma unroll
    for (int k = 0; k < kGroupMaxSeg; ++k) {
        double piv = Sm[k][k];
        if (!(piv > 0.0)) { bad = 1; piv = 1.0; }
        const double ip = 1.0 / piv;
        Sm[k][k] = 1.0;
#pragma unroll
        for (int j = 0; j < kGroupMaxSeg; ++j) Sm[k][j] *= ip;
#pragma unroll
        for (int i = 0; i < kGroupMaxSeg; ++i) {
            if (i == k) continue;
            const double f = Sm[i][k];
            Sm[i][k] = 0.0;
#pragma unroll
            for (int j = 0; j < kGroupMaxSeg; ++j) Sm[i][j] -= f * Sm[k][j];
        }
    }
    if (bad && con && s.wv && kk == 0) atomicExch(&c.sc->nonpd, 1);
    double Zv[kGroupMaxSeg];
#pragma unroll
    for (int h = 0; h < kGroupMaxSeg; ++h) {
        double z = 0.0;
#pragma unroll
        for (int g = 0; g < kGroupMaxSeg; ++g) z += Yv[g] * Sm[g][h];
        Zv[h] = z;
    }
    if (s.ev) {
        double* Zo = c.zgrp + (size_t)e * S;
#pragma unroll
        for (int g = 0; g < kGroupMaxSeg; ++g)
            if (g < S) Zo[g] = Zv[g];
    }
    // P_w row kk, stored; R^T P_w R
    const double R = s.ev ? c.R[e] : 0.0;
    double pr = 0.0;
#pragma unroll
    for (int j = 0; j < kSegMax; ++j) {
        if (j < B) {
            double pj = a[j];
#pragma unroll
            for (int g = 0; g < kGroupMaxSeg; ++g) {
                const double Yjg = __shfl_sync(0xffffffffu, Yv[g], s.base + j);
                if (con) pj -= Zv[g] * Yjg;
            }
            const double Rj = __shfl_sync(0xffffffffu, R, s.base + j);
            if (s.ev) c.Lf[((size_t)w * B + kk) * B + j] = (float)pj;
            pr += pj * Rj;
        }
    }
    double rn = seg_sum(s.ev ? R * pr : 0.0, s.Bp);
    // subelement shares of J_I and the warm start moved onto them
    double d[kGroupMaxSeg], gap[kGroupMaxSeg];
#pragma unroll
    for (int g = 0; g < kGroupMaxSeg; ++g) {
        d[g] = g < S ? seg_sum(gk == g ? xI : 0.0, s.Bp) : 0.0;
        gap[g] = g < S ? d[g] - seg_sum(gk == g ? xe0 : 0.0, s.Bp) : 0.0;
    }
    double dSd = 0.0, corr = 0.0;
#pragma unroll
    for (int g = 0; g < kGroupMaxSeg; ++g) {
        double sd = 0.0;
#pragma unroll
        for (int h = 0; h < kGroupMaxSeg; ++h) sd += Sm[g][h] * d[h];
        dSd += d[g] * sd;
        corr += Zv[g] * gap[g];
    }
    if (s.ev) {
        const double xe = con ? xe0 + corr : xe0;
        c.x[e] = xe;
        c.pf[e] = (float)xe;
    }
    if (kk == 0 && s.wv) c.parts[3 * (size_t)c.W + w] = rn + (con ? dSd : 0.0);
}

__device__ __forceinline__ float inv_pivot(float p) { return 1.0f / p; }
__device__ __forceinline__ double inv_pivot(double p) { return rcp_nr(p); }

// Body of k_factor_seg in the precision T of the inverse.  T = float: the
// inverse only serves the preconditioner P_w (stored in FP32 anyway) and y for
// the constraint projections, which stay exact for any y because sigma is
// summed in FP64 from the y that are stored; the PCG's residual stays FP64,
// so the solution does not depend on it.  T = double: the subelement path.
template <typename T>
__device__ __forceinline__ double factor_seg(const CoilDev& c, const Seg& s) {
    const int B = s.B, kk = s.kk, w = s.w, e = s.e;
    T a[kSegMax];
    const size_t nb0 = (size_t)c.block_type[s.wv ? w : 0] * B * B;
    if constexpr (sizeof(T) == sizeof(float)) {
        // the self blocks' FP32 copy (no per-entry conversion on the FP64 pipe)
        const float* nb = c.nearf + nb0;
#pragma unroll
        for (int j = 0; j < kSegMax; ++j)
            a[j] = (s.wv && kk < B && j < B) ? nb[kk * B + j] : (j == kk ? 1.f : 0.f);
    } else {
        const double* nb = c.near + nb0;
#pragma unroll
        for (int j = 0; j < kSegMax; ++j)
            a[j] = (s.wv && kk < B && j < B) ? nb[kk * B + j] : (j == kk ? 1.0 : 0.0);
    }
    if (s.ev) {
        const T g = (T)(c.dt * c.G[e]);
#pragma unroll
        for (int j = 0; j < kSegMax; ++j)
            if (j == kk) a[j] += g;
    }
    // what the steps after the inverse read, loaded now: its latency hides
    // behind the sweep
    const WarmIn wm = s.ev ? warm_load(c, e) : WarmIn{0.0, 0.0, 0.0};
    const bool ext = extrapolate(c);
    const int con = s.wv ? c.constrained[w] : 0;
    const double R = s.ev ? c.R[e] : 0.0;
    const double cw = s.wv ? c.cw[w] : 0.0;
    int bad = 0;
#pragma unroll
    for (int k = 0; k < kSegMax; ++k) {
        if (k < B) {
            T piv = __shfl_sync(0xffffffffu, a[k], s.base + k);
            if (!(piv > (T)0)) { bad = 1; piv = (T)1; }
            const T ip = inv_pivot(piv);
            if (kk == k) {
#pragma unroll
                for (int j = 0; j < kSegMax; ++j) a[j] = (j == k) ? ip : a[j] * ip;
            }
            // eliminate with the scaled pivot row, one broadcast entry at a time
            // (no copy of the row held in registers)
            const T f = a[k];
#pragma unroll
            for (int j = 0; j < kSegMax; ++j) {
                const T rkj = __shfl_sync(0xffffffffu, a[j], s.base + k);
                if (kk != k) a[j] = (j == k) ? -f * ip : a[j] - f * rkj;
            }
        }
    }
    if (bad && s.wv && kk == 0) {
        atomicExch(&c.sc->nonpd, 1);
        __threadfence();                       // before this CTA's arrival on a fused reduction
    }
    // y = A_w^-1 1 (row sums of the symmetric inverse), sigma = 1^T y
    T yt = 0;
#pragma unroll
    for (int j = 0; j < kSegMax; ++j)
        if (j < B) yt += a[j];
    const double y = s.ev ? (double)yt : 0.0;
    const double sig = seg_sum(y, s.Bp);
    const double isg = 1.0 / sig;
    if (s.ev) c.y1[e] = y;
    if (kk == 0 && s.wv) {
        c.sigma[w] = sig;
        c.isigma[w] = isg;
    }
    const double x0 = s.ev ? warm_finish(c, e, ext, wm) : 0.0;   // before the constraint
    if constexpr (sizeof(T) == sizeof(double)) {
        if (c.n_groups) {
            factor_groups(c, s, a, y, isg, con, x0);
            return 0.0;
        }
    }
    // P_w row kk, stored (its entries are FP32 values: the subtraction runs in
    // T = float); R^T P_w R in FP32 (it only scales the stopping test)
    const float Rf = (float)R, yf = (float)y, yis = (float)(y * isg);
    float pr0 = 0.f, pr1 = 0.f;
#pragma unroll
    for (int j = 0; j < kSegMax; ++j) {
        if (j < B) {
            const float yj = __shfl_sync(0xffffffffu, yf, s.base + j);
            const float Rj = __shfl_sync(0xffffffffu, Rf, s.base + j);
            const float pj = con ? (float)(a[j] - (T)yis * (T)yj) : (float)a[j];
            if (s.ev) c.Lf[((size_t)w * B + kk) * B + j] = pj;
            if (j & 1) pr1 = fmaf(pj, Rj, pr1);
            else pr0 = fmaf(pj, Rj, pr0);
        }
    }
    const double rn = seg_sum(s.ev ? R * (double)(pr0 + pr1) : 0.0, s.Bp);
    // warm start moved onto this step's constraint
    const double sx = seg_sum(x0, s.Bp);
    const double corr = con ? (cw - sx) * isg : 0.0;
    if (s.ev) {
        double xe = x0 + corr * y;
        c.x[e] = xe;
        c.pf[e] = (float)xe;
    }
    const double scale = rn + (con ? cw * cw * isg : 0.0);
    if (kk == 0 && s.wv) c.parts[3 * (size_t)c.W + w] = scale;
    return kk == 0 && s.wv ? scale : 0.0;
}

// k_factor for blocks of at most 16 elements.  Lane kk holds row kk of
// A_w = M_ww + dt G_w in registers and the segment inverts it in place by
// Gauss-Jordan elimination without pivoting (A_w is SPD, so every pivot is a
// positive Schur complement; a non-positive one flags the step as the
// Cholesky does), broadcasting each scaled pivot row by shuffles.  From A_w^-1:
// y = A_w^-1 1, sigma = 1^T y, and the projected preconditioner
// P_w = A_w^-1 - y y^T / sigma (constrained wires; A_w^-1 otherwise), which
// is stored (in the factor array) so that every PCG application is one
// B x B product.  Also the right-hand-side norm R^T P_w R + c_w^2 / sigma and
// the projected warm start.
// GROUPS: the coils with subelements (their path needs A_w^-1 itself, the
// transport part, in FP64), launched as a kernel of its own so that its
// registers do not weigh on the plain path (the inverse only builds the
// preconditioner, which FP32 serves; see factor_seg).
// fuse_scale (coils without subelements): the last CTA sums the scale
// partials and starts the solve's scalars (the k_reduce SCALE step).
__global__ void __launch_bounds__(32 * kSegWarps) k_factor_seg(const CoilDev* __restrict__ cds, int fuse_scale) {
    const CoilDev& c = cds[blockIdx.y];
    const int per_cta = kSegWarps * (32 / seg_width(c.B));   // wires per CTA
    const int n_cta = (c.W + per_cta - 1) / per_cta;
    if (c.B > kSegMax || c.n_groups != 0 || (int)blockIdx.x >= n_cta) return;
    const int wg = blockIdx.x * kSegWarps + (threadIdx.x >> 5);
    double head = 0.0;                                  // the wire's scale term on its head lane
    if (wg * (32 / seg_width(c.B)) < c.W) head = factor_seg<float>(c, seg_of(c, wg));   // warp-uniform
    if (fuse_scale) fused_reduce(c, head, c.ticket + 3, n_cta, RED_SCALE);
}
__global__ void __launch_bounds__(32 * kSegWarps) k_factor_seg_groups(const CoilDev* __restrict__ cds) {
    const CoilDev& c = cds[blockIdx.y];
    if (c.B > kSegMax || c.n_groups == 0) return;
    const int wg = blockIdx.x * kSegWarps + (threadIdx.x >> 5);
    if (wg * (32 / seg_width(c.B)) >= c.W) return;       // warp-uniform; no CTA barrier below
    factor_seg<double>(c, seg_of(c, wg));
}

// The PCG loop's condition as a kernel of its own (coils whose update kernel
// does not set it).
__global__ void k_loop_cond(const CoilDev* __restrict__ cds, cudaGraphConditionalHandle h) {
    loop_condition(*cds, h);
}

// d = -z + beta d (and its FP32 copy for the mixed-precision operator).
__global__ void k_direction(const CoilDev* __restrict__ cds) {
    const CoilDev& c = cds[blockIdx.y];
    if (c.sc->done) return;
    double beta = c.sc->beta;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < c.N; e += gridDim.x * blockDim.x) {
        double d = -c.zv[e] + beta * c.dv[e];
        c.dv[e] = d;
        c.pf[e] = (float)d;
    }
}

// u_w, I += dt x, flux += dt M x with M x = (r + U_w) - R - dt G x (r is the
// projected residual, U_w the loop voltage removed from it); partials V
// (parts[5]) and m (parts[6]).
// One warp per wire; the coils of k_finalize_seg are left to it.
__global__ void k_finalize(const CoilDev* __restrict__ cds) {
    const CoilDev& c = cds[blockIdx.y];
    if (c.sc->status != ST_OK) return;          // a failed coil keeps its state
    if (c.B <= kSegMax && c.n_groups == 0) return;
    double* parts = c.parts;
    int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (w >= c.W) return;
    int B = c.B;
    double dt = c.dt;
    int con = c.constrained[w];
    if (c.n_groups) {
        // subelements: M x = (r + Q v) - R - dt G x; v += (Y S^-1)^T r; the
        // transport part advances with its rate x_I
        const int S = c.n_groups;
        double V[kGroupMax], inc[kGroupMax];
#pragma unroll
        for (int g = 0; g < kGroupMax; ++g) {
            V[g] = (con && g < S) ? c.ugrp[(size_t)w * S + g] : 0.0;
            inc[g] = 0.0;
        }
        double mom = 0.0;
        for (int k = lane; k < B; k += 32) {
            int e = w * B + k;
            const int gk = c.group[k];
            double Vk = 0.0;
#pragma unroll
            for (int g = 0; g < kGroupMax; ++g)
                if (g == gk) Vk = V[g];
            double xe = c.x[e], re = c.res[e];
#pragma unroll
            for (int g = 0; g < kGroupMax; ++g)
                if (g < S) inc[g] += c.zgrp[(size_t)e * S + g] * re;
            double In = c.I[e] + dt * xe;
            c.I[e] = In;
            c.Itr[e] += dt * c.xI[e];
            c.Phi[e] += dt * ((re + Vk) - c.R[e] - dt * c.G[e] * xe);
            double r = c.r[e];
            mom += kPi * r * r * In;
        }
        double u = 0.0;
#pragma unroll
        for (int g = 0; g < kGroupMax; ++g) {
            const double vg = V[g] + warp_sum(inc[g]);
            u += c.gwt[g] * vg;
            if (lane == 0 && con && g < S) c.ugrp[(size_t)w * S + g] = vg;
        }
        mom = warp_sum(mom);
        if (lane == 0) {
            u = con ? u : 0.0;
            c.uw[w] = u;
            parts[5 * (size_t)c.W + w] = u;
            parts[6 * (size_t)c.W + w] = mom;
        }
        return;
    }
    double U = con ? c.uw[w] : 0.0;
    double yr = 0.0, mom = 0.0;
    const bool rec = c.rec_mode == 1, replay = c.rec_mode == 2;
    const size_t ri = (rec || replay) ? (size_t)(c.sc->step - c.rec_step0) : 0;
    if (rec && lane == 0) c.rec_uw[ri * c.W + w] = c.uw[w];
    for (int k = lane; k < B; k += 32) {
        int e = w * B + k;
        double xe = c.x[e];
        if (rec) {
            c.rec_x[ri * c.N + e] = xe;
            c.rec_res[ri * c.N + e] = c.res[e];
        }
        if (!replay) yr += c.y1[e] * c.res[e];
        double In = c.I[e] + dt * xe;
        c.I[e] = In;
        c.Phi[e] += dt * ((c.res[e] + U) - c.R[e] - dt * c.G[e] * xe);
        double r = c.r[e];
        mom += kPi * r * r * In;
    }
    yr = warp_sum(yr);
    mom = warp_sum(mom);
    if (lane == 0) {
        double u = con ? (replay ? c.rec_u[ri * c.W + w] : U + yr * c.isigma[w]) : 0.0;
        if (rec) c.rec_u[ri * c.W + w] = u;
        c.uw[w] = u;
        parts[5 * (size_t)c.W + w] = u;
        parts[6 * (size_t)c.W + w] = mom;
    }
}

// k_finalize for wires of at most 16 elements without subelements, 32 / Bp
// wires per warp (the same operations per element; the wire sums drop only
// the idle lanes' zeros).
__global__ void k_finalize_seg(const CoilDev* __restrict__ cds) {
    const CoilDev& c = cds[blockIdx.y];
    if (c.sc->status != ST_OK || c.B > kSegMax || c.n_groups != 0) return;
    const int wg = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wg * (32 / seg_width(c.B)) >= c.W) return;       // warp-uniform
    const Seg s = seg_of(c, wg);
    const double dt = c.dt;
    const bool rec = c.rec_mode == 1, replay = c.rec_mode == 2;
    // every load first (one round trip), then the arithmetic
    const int wl = s.wv ? s.w : 0, el = s.ev ? s.e : 0;
    const int con_w = c.constrained[wl];
    const double uw0 = c.uw[wl], isg = c.isigma[wl];
    const double xe = c.x[el], re = c.res[el], ye = c.y1[el], Ie = c.I[el], Pe = c.Phi[el];
    const double Re = c.R[el], Ge = c.G[el], pr2 = c.pir2[el];
    const long long st = c.sc->step;
    const int con = s.wv ? con_w : 0;
    const double U = con ? uw0 : 0.0;
    const size_t ri = (rec || replay) ? (size_t)(st - c.rec_step0) : 0;
    if (rec && s.kk == 0 && s.wv) c.rec_uw[ri * c.W + s.w] = uw0;
    double yr = 0.0, mom = 0.0;
    if (s.ev) {
        const int e = s.e;
        if (rec) {
            c.rec_x[ri * c.N + e] = xe;
            c.rec_res[ri * c.N + e] = re;
        }
        if (!replay) yr = ye * re;
        const double In = Ie + dt * xe;
        c.I[e] = In;
        c.Phi[e] = Pe + dt * ((re + U) - Re - dt * Ge * xe);
        mom = pr2 * In;
    }
    yr = seg_sum(yr, s.Bp);
    mom = seg_sum(mom, s.Bp);
    if (s.kk == 0 && s.wv) {
        const int w = s.w;
        const double u = con ? (replay ? c.rec_u[ri * c.W + w] : U + yr * isg) : 0.0;
        if (rec) c.rec_u[ri * c.W + w] = u;
        c.uw[w] = u;
        c.parts[5 * (size_t)c.W + w] = u;
        c.parts[6 * (size_t)c.W + w] = mom;
    }
}

// A replayed step (rec_mode 2): the solution, residual and loop voltages that
// the forward pass's finalisation of this step used, in place of the solve.
__global__ void k_replay_restore(const CoilDev* __restrict__ cds) {
    const CoilDev& c = cds[blockIdx.y];
    if (c.rec_mode != 2 || c.sc->status != ST_OK) return;
    const size_t ri = (size_t)(c.sc->step - c.rec_step0);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < c.N; e += gridDim.x * blockDim.x) {
        c.x[e] = c.rec_x[ri * c.N + e];
        c.res[e] = c.rec_res[ri * c.N + e];
        if (e < c.W) c.uw[e] = c.rec_uw[ri * c.W + e];
    }
}

// ------------------------------------------------------------------ thermal

// Source s = 4/(rho_m c0) (q - border loss / h^2) of cell g with state u.
// Only border cells lose heat to the bath: the others skip the temperature
// (two FP64 square roots on B300's narrow FP64 pipe); the constant factors
// are taken as precomputed reciprocals.
__device__ __forceinline__ double thermal_source(const CoilDev& c, int g, double u) {
    const int nb = c.nborder[g];
    double loss = 0.0;
    if (nb) {
        const double T = sqrt(sqrt(u));
        const double tr = T * c.inv_Tref;
        loss = nb * c.helem * c.h0 * (tr * tr * tr) * (T - c.T_bath);
    }
    return c.src_k * (c.qgrid[g] - loss * c.inv_h2);
}

// r-lines: u* = (I - dt/2 A_r)^-1 [(I + dt/2 A_z) u + dt/2 s].  One CTA per grid row.
__global__ void k_adi_r(const CoilDev* __restrict__ cds) {
    const CoilDev& c = cds[blockIdx.y];
    if (c.sc->status != ST_OK) return;
    int j = blockIdx.x;
    if (j >= c.Gz) return;
    extern __shared__ double sm[];
    int Gr = c.Gr, Gz = c.Gz;
    double hd = 0.5 * c.dt;
    const double invC = c.inv_Ccell;
    line_stage(sm + Gr, Gr, c.thr_a, c.thr_inv, c.thr_c);
    for (int i = threadIdx.x; i < Gr; i += blockDim.x) {
        int g = j * Gr + i;
        double u = c.uT[g];
        double s = thermal_source(c, g, u);
        c.src[(size_t)i * Gz + j] = s;
        double az = 0.0;
        if (j > 0) az += c.Kz[j - 1] * (c.uT[g - Gr] - u);
        if (j < Gz - 1) az += c.Kz[j] * (c.uT[g + Gr] - u);
        sm[i] = u + hd * (az * invC) + hd * s;
    }
    line_solve(sm, sm + Gr, Gr);
    // stored column by column: the z-lines' loads are then contiguous
    for (int i = threadIdx.x; i < Gr; i += blockDim.x) c.ustar[(size_t)i * Gz + j] = sm[i];
}

// z-lines: u' = (I - dt/2 A_z)^-1 [(I + dt/2 A_r) u* + dt/2 s].  One CTA per column.
__global__ void k_adi_z(const CoilDev* __restrict__ cds) {
    const CoilDev& c = cds[blockIdx.y];
    if (c.sc->status != ST_OK) return;
    int i = blockIdx.x;
    if (i >= c.Gr) return;
    extern __shared__ double sm[];
    int Gr = c.Gr, Gz = c.Gz;
    double hd = 0.5 * c.dt;
    const double invC = c.inv_Ccell;
    line_stage(sm + Gz, Gz, c.thz_a, c.thz_inv, c.thz_c);
    const double* col = c.ustar + (size_t)i * Gz;       // column i (and i -/+ 1 at -/+ Gz)
    for (int j = threadIdx.x; j < Gz; j += blockDim.x) {
        double us = col[j];
        double ar = 0.0;
        if (i > 0) ar += c.Kr[i - 1] * (col[j - Gz] - us);
        if (i < Gr - 1) ar += c.Kr[i] * (col[j + Gz] - us);
        sm[j] = us + hd * (ar * invC) + hd * c.src[(size_t)i * Gz + j];
    }
    line_solve(sm, sm + Gz, Gz);
    double um = 0.0;
    for (int j = threadIdx.x; j < Gz; j += blockDim.x) {
        double u = sm[j];
        c.uT[j * Gr + i] = u;
        um = fmax(um, u);
    }
    um = block_reduce_max(um, sm + Gz);     // the factor rows are free once line_solve returns
    if (threadIdx.x == 0) c.partT[i] = um;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    return v;
}

// The step's diagnostic record, then t += dt.  kStepEndCtas CTAs per coil
// (grid row = coil) each reduce a slice of the per-wire values and of the
// thermal columns into partials (parts row 7, free once the solve is done);
// the CTA that arrives last on the coil's third counter (which it resets)
// combines them in a fixed order and writes the record.  On B300 one CTA's
// FP64 pipe alone took ~28 us for the 96,000-element coil, and a warp issues
// one FP64 instruction per 64 cycles: the reductions are spread over warps.

__global__ void __launch_bounds__(kStepEndThreads) k_step_end(const CoilDev* __restrict__ cds) {
    static_assert(kStepEndCtas <= 32 && kStepEndThreads >= 6 * 32, "one warp per quantity");
    constexpr int NT = kStepEndThreads;
    const CoilDev& c = cds[blockIdx.y];
    if (c.sc->status != ST_OK) return;
    // three sums (Joule power, loop voltage, moment) in FP64; three maxima of
    // non-negative values (|J|/Jc, rho/rho_n, u = T^4) as the maxima of their
    // bit patterns, exact and off the FP64 pipe; each reduced by a warp of its own
    __shared__ double ssum[3][NT];
    __shared__ unsigned long long smax[3][NT];
    __shared__ double rsum[3];
    __shared__ unsigned long long rmax[3];
    __shared__ int is_last;
    const double* parts = c.parts;
    const size_t W = c.W;
    const int nb = gridDim.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int stride = nb * blockDim.x;
    double pj = 0.0, V = 0.0, m = 0.0;
    unsigned long long jr = 0, rh = 0, um = 0;
    auto bits = [](double v) { return (unsigned long long)__double_as_longlong(v); };
    for (int w = blockIdx.x * blockDim.x + tid; w < c.W; w += stride) {
        pj += parts[0 * W + w];
        jr = max(jr, bits(parts[1 * W + w]));
        rh = max(rh, bits(parts[2 * W + w]));
        V += parts[5 * W + w];
        m += parts[6 * W + w];
    }
    if (c.has_grid) {
        if (c.thermal) {
            for (int i = blockIdx.x * blockDim.x + tid; i < c.Gr; i += stride) um = max(um, bits(c.partT[i]));
        } else {
            for (int g = blockIdx.x * blockDim.x + tid; g < c.Gr * c.Gz; g += stride) um = max(um, bits(c.uT[g]));
        }
    }
    ssum[0][tid] = pj;
    ssum[1][tid] = V;
    ssum[2][tid] = m;
    smax[0][tid] = jr;
    smax[1][tid] = rh;
    smax[2][tid] = um;
    __syncthreads();
    if (wid < 3) {
        double v = 0.0;
        for (int k = lane; k < NT; k += 32) v += ssum[wid][k];
        v = warp_sum(v);
        if (lane == 0) rsum[wid] = v;
    } else if (wid < 6) {
        unsigned long long v = 0;
        for (int k = lane; k < NT; k += 32) v = max(v, smax[wid - 3][k]);
        v = warp_max_u64(v);
        if (lane == 0) rmax[wid - 3] = v;
    }
    __syncthreads();
    double* cp = c.parts + 7 * W;                     // 6 partials per CTA
    if (tid == 0) {
        cp[6 * blockIdx.x + 0] = rsum[0];
        cp[6 * blockIdx.x + 1] = rsum[1];
        cp[6 * blockIdx.x + 2] = rsum[2];
        cp[6 * blockIdx.x + 3] = __longlong_as_double((long long)rmax[0]);
        cp[6 * blockIdx.x + 4] = __longlong_as_double((long long)rmax[1]);
        cp[6 * blockIdx.x + 5] = __longlong_as_double((long long)rmax[2]);
        unsigned prev;
        asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(prev) : "l"(c.ticket + 2) : "memory");
        is_last = prev == (unsigned)nb - 1u;
        if (is_last) c.ticket[2] = 0u;
    }
    __syncthreads();
    if (!is_last) return;
    // the last CTA: the CTAs' partials (read from L2), one quantity per warp,
    // in a fixed order
    if (wid < 3) {
        double v = lane < nb ? __ldcg(cp + 6 * lane + wid) : 0.0;
        v = warp_sum(v);
        if (lane == 0) rsum[wid] = v;
    } else if (wid < 6) {
        unsigned long long v = lane < nb ? bits(__ldcg(cp + 6 * lane + wid)) : 0ull;
        v = warp_max_u64(v);
        if (lane == 0) rmax[wid - 3] = v;
    }
    __syncthreads();
    Scalars* sc = c.sc;
    double* rec = c.diag + (size_t)(sc->step % c.diag_cap) * 10;
    if (tid == 0) {
        const double um_max = __longlong_as_double((long long)rmax[2]);
        rec[0] = sc->t + c.dt;
        rec[1] = sc->It1;
        rec[2] = rsum[1];
        rec[3] = rsum[2];
        rec[4] = rsum[0];
        rec[5] = c.has_grid ? sqrt(sqrt(um_max)) : c.T_bath;
        rec[6] = __longlong_as_double((long long)rmax[0]);
        rec[7] = __longlong_as_double((long long)rmax[1]);
    } else if (tid == 32 && c.rec_mode != 2) {        // a replayed step keeps the solve's diagnostics
        rec[8] = (double)sc->iter;
        sc->last_resid = sc->scale2 > 0.0 ? sqrt(fmax(sc->rz, 0.0) / sc->scale2) : 0.0;
        rec[9] = sc->last_resid;
    }
    __syncthreads();
    if (tid == 0) {
        sc->t = sc->t + c.dt;
        sc->step += 1;
    }
}

// J, B_r, B_z, T of the current state into element-order buffers.
__global__ void k_read(const CoilDev* __restrict__ cds, double Ba, double* J, double* Br, double* Bz,
                       double* T) {
    const CoilDev& c = cds[blockIdx.y];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < c.N; e += gridDim.x * blockDim.x) {
        if (J) J[e] = c.I[e] / c.area[e];
        double br = 0.0, bz = 0.0;
        if (c.has_grid && (Br || Bz)) field_at(c, e, Ba, &br, &bz);
        if (Br) Br[e] = br;
        if (Bz) Bz[e] = bz;
        if (T) T[e] = c.has_grid ? sqrt(sqrt(c.uT[c.elem_grid[e]])) : c.T_bath;
    }
}

// Dynamic shared memory the forward ADI kernels may take (lines of more than
// 1,536 cells need more than the default 48 KB).
cudaError_t adi_allow_smem(size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_adi_r, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_adi_z, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace cq
