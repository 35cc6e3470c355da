// Reverse (adjoint) kernels of the coupled step, for gradients of a loss on
// the moment series and the Joule-power series with respect to the
// calibration parameters: per-element
// Jc factor f, the creep exponent n and the strain coefficient C_eps (the
// paper calibrates its E-J and Jc laws against a measured magnetization loop,
// Methods).
//
// Forward step k (state I, u = T^4; the flux is M I):
//   B = S(M I + pi r^2 B_a) / (2 pi r)        stencil, linear in I
//   Jc = Jc(|B|, T; f, C_eps),  E = rho(J, Jc; n) J,  G = 2 pi r dE/dJ / a
//   [A -P; P^T 0][Idot; u] = [-R; c],  A = M + dt diag(G),  R = 2 pi r E + ...
//   c_w = (I_t - sum_w I) / dt,  I' = I + dt Idot,  u' = ADI(u, q = E J)
// Reverse, given lam_I' and lam_u':
//   lam_Idot = dt lam_I';  solve  A mu + P nu = lam_Idot, P^T mu = 0 (the same
//   projected PCG with R := -lam_Idot, c := 0, and nu = -u);  lam_R = -mu,
//   lam_c = nu, lam_G = -dt mu Idot (K depends on G);  reverse ADI gives
//   lam_q and lam_u;  then the E-J / Jc Jacobians, the stencil transpose and
//   the operator transpose (M symmetric: one more apply).
#include "common.cuh"
#include "pointwise.cuh"
#include "tridiag.cuh"

namespace cq {

struct AdjBufs {
    double* lamI;       // lam_I of the step being reversed (output), element order
    const double* lamI_next;
    double* lamU;       // lam_u (grid), output
    const double* lamU_next;
    double* a;          // reverse-ADI intermediates (grid)
    double* b;
    double* lamQ;       // lam_q (grid)
    double* lamBr;      // per element, lam_B / (2 pi r)
    double* lamBz;
    const double* xk;   // Idot of the forward step being reversed
    double* g_f;        // dL/df accumulated (element order)
    double* gparts;     // 2 x W per-block partial sums of dL/dn and dL/dC_eps
};

// a = (I - dt/2 A_z)^-1 lam_u'   (z-lines; the matrix is symmetric)
__global__ void k_adj_adi_z(const CoilDev* __restrict__ cds, AdjBufs ab) {
    const CoilDev& c = cds[0];
    int i = blockIdx.x;
    if (i >= c.Gr) return;
    extern __shared__ double sm[];
    int Gr = c.Gr, Gz = c.Gz;
    line_stage(sm + Gz, Gz, c.thz_a, c.thz_inv, c.thz_c);
    for (int j = threadIdx.x; j < Gz; j += blockDim.x) sm[j] = ab.lamU_next[j * Gr + i];
    line_solve(sm, sm + Gz, Gz);
    for (int j = threadIdx.x; j < Gz; j += blockDim.x) ab.a[j * Gr + i] = sm[j];
}

// b = (I - dt/2 A_r)^-1 (I + dt/2 A_r) a   (r-lines)
__global__ void k_adj_adi_r(const CoilDev* __restrict__ cds, AdjBufs ab) {
    const CoilDev& c = cds[0];
    int j = blockIdx.x;
    if (j >= c.Gz) return;
    extern __shared__ double sm[];
    int Gr = c.Gr;
    double hd = 0.5 * c.dt, invC = c.inv_Ccell;
    line_stage(sm + Gr, Gr, c.thr_a, c.thr_inv, c.thr_c);
    for (int i = threadIdx.x; i < Gr; i += blockDim.x) {
        int g = j * Gr + i;
        double ai = ab.a[g];
        double ar = 0.0;
        if (i > 0) ar += c.Kr[i - 1] * (ab.a[g - 1] - ai);
        if (i < Gr - 1) ar += c.Kr[i] * (ab.a[g + 1] - ai);
        sm[i] = ai + hd * (ar * invC);
    }
    line_solve(sm, sm + Gr, Gr);
    for (int i = threadIdx.x; i < Gr; i += blockDim.x) ab.b[j * Gr + i] = sm[i];
}

// lam_u = (I + dt/2 A_z) b + (ds/du) lam_s,  lam_s = dt/2 (a + b),
// lam_q = 4/(rho_m c0) lam_s  (s = 4/(rho_m c0) (q - loss(u)/h^2)).
__global__ void k_adj_adi_src(const CoilDev* __restrict__ cds, AdjBufs ab) {
    const CoilDev& c = cds[0];
    int Gr = c.Gr, Gz = c.Gz;
    double hd = 0.5 * c.dt, invC = c.inv_Ccell;
    double cs = 4.0 / (c.rho_m * c.c0);
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < Gr * Gz; g += gridDim.x * blockDim.x) {
        int j = g / Gr;
        double bg = ab.b[g];
        double az = 0.0;
        if (j > 0) az += c.Kz[j - 1] * (ab.b[g - Gr] - bg);
        if (j < Gz - 1) az += c.Kz[j] * (ab.b[g + Gr] - bg);
        double lam_s = hd * (ab.a[g] + bg);
        double u = c.uT[g];
        double T = sqrt(sqrt(u));
        double T3r = c.T_ref * c.T_ref * c.T_ref;
        // loss = nb h h0 (T^3/T_ref^3) (T - T_bath);  d loss / dT, dT/du = T / (4u)
        double dloss_dT = c.nborder[g] * c.helem * c.h0 / T3r * (4.0 * T * T * T - 3.0 * T * T * c.T_bath);
        double ds_du = -cs / (c.helem * c.helem) * dloss_dT * (T / (4.0 * u));
        ab.lamU[g] = bg + hd * (az * invC) + ds_du * lam_s;
        ab.lamQ[g] = cs * lam_s;
    }
}

// Adjoint right-hand side: R = -dt lam_I', c_w = 0 (the PCG then solves for mu).
__global__ void k_adj_setup(const CoilDev* __restrict__ cds, AdjBufs ab) {
    const CoilDev& c = cds[0];
    int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (w >= c.W) return;
    for (int k = lane; k < c.B; k += 32) {
        int e = w * c.B + k;
        c.R[e] = -c.dt * ab.lamI_next[e];
    }
    if (lane == 0) c.cw[w] = 0.0;
}

// Loop-voltage unknown of the adjoint solve (u = U + y^T r / sigma), no state update.
__global__ void k_adj_mult(const CoilDev* __restrict__ cds) {
    const CoilDev& c = cds[0];
    int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (w >= c.W) return;
    double yr = 0.0;
    for (int k = lane; k < c.B; k += 32) yr += c.y1[w * c.B + k] * c.res[w * c.B + k];
    yr = warp_sum(yr);
    if (lane == 0) c.uw[w] = c.constrained[w] ? c.uw[w] + yr * c.isigma[w] : 0.0;
}

// Jc and its partial derivatives (zero outside the superconducting region).
struct JcD { double Jc, dBm, dT, df, dCe, dep; };

// ep = |eps|^p_eps of the element; dep = dJc/d(ep).
__device__ JcD jc_with_derivatives(const CoilDev& c, double Bm, double T, double ep, double f) {
    JcD d = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (c.jc_model == 1) {
        d.Jc = f * c.Jc0;
        d.df = c.Jc0;
        return d;
    }
    double tr = T / c.Tc;
    double Bc2 = c.Bc2_0 * (1.0 - tr * tr);
    if (!(T < c.Tc && Bm < Bc2)) return d;
    double S = 1.0 - c.C_eps * ep;
    if (!(S > 0.0)) return d;
    double bfac = 1.0 - Bm / Bc2;
    double omt = 1.0 - tr;
    double core = c.Jc0 * (omt * sqrt(omt)) * (bfac * bfac) / sqrt(Bm + c.B_reg);
    d.Jc = f * core * S;
    d.df = core * S;
    d.dCe = -f * core * ep;
    d.dep = -f * core * c.C_eps;
    d.dBm = d.Jc * (-2.0 / (bfac * Bc2) - 0.5 / (Bm + c.B_reg));
    double db_dT = Bm * (2.0 * c.Bc2_0 * tr / c.Tc) / (Bc2 * Bc2);
    d.dT = d.Jc * (-1.5 / (c.Tc * (1.0 - tr)) - 2.0 / bfac * db_dT);
    return d;
}

// The same in FP32: the mixed form's forward pointwise chain (Jc, E, G in
// FP32), whose Jacobians these are.
__device__ JcD jc_with_derivatives_f(const CoilDev& c, float Bm, float T, float ep, float f) {
    JcD d = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const float Jc0 = c.f_Jc0;
    if (c.jc_model == 1) {
        d.Jc = f * Jc0;
        d.df = Jc0;
        return d;
    }
    const float Tc = c.f_Tc, Bc20 = c.f_Bc2_0, Ce = c.f_C_eps, Breg = c.f_B_reg;
    const float tr = T / Tc;
    const float Bc2 = Bc20 * (1.0f - tr * tr);
    if (!(T < Tc && Bm < Bc2)) return d;
    const float S = 1.0f - Ce * ep;
    if (!(S > 0.0f)) return d;
    const float bfac = 1.0f - Bm / Bc2;
    const float omt = 1.0f - tr;
    const float core = Jc0 * (omt * sqrtf(omt)) * (bfac * bfac) / sqrtf(Bm + Breg);
    const float Jc = f * core * S;
    d.Jc = Jc;
    d.df = core * S;
    d.dCe = -f * core * ep;
    d.dep = -f * core * Ce;
    d.dBm = Jc * (-2.0f / (bfac * Bc2) - 0.5f / (Bm + Breg));
    const float db_dT = Bm * (2.0f * Bc20 * tr / Tc) / (Bc2 * Bc2);
    d.dT = Jc * (-1.5f / (Tc * omt) - 2.0f / bfac * db_dT);
    return d;
}

// E-J law pieces: frac = rho/rho_n, dfac = (dE/dJ)/rho_n, A1 = s/(1+s)^2,
// A2 = (n + s(2-n)) s/(1+s)^3, lnx = ln(|J|/Jc), evaluated without overflow.
struct EJD { double frac, dfac, A1, A2, lnx; };

__device__ EJD ej_with_derivatives(const CoilDev& c, int fil, double J, double Jc) {
    EJD d = {1.0, 1.0, 0.0, 0.0, 0.0};
    if (!fil || Jc <= 0.0) return d;
    double aJ = fabs(J);
    if (aJ == 0.0) { d.frac = 0.0; d.dfac = 0.0; return d; }
    double n = c.nexp;
    d.lnx = log(aJ / Jc);
    double ell = log(c.E0 / (Jc * c.rho_n)) + (n - 1.0) * d.lnx;
    if (ell > 0.0) {
        double t = exp(-ell), opt = 1.0 + t;
        d.frac = 1.0 / opt;
        d.dfac = (1.0 + n * t) / (opt * opt);
        d.A1 = t / (opt * opt);
        d.A2 = (n * t * t + (2.0 - n) * t) / (opt * opt * opt);
    } else {
        double s = exp(ell), ops = 1.0 + s;
        d.frac = s / ops;
        d.dfac = s * (s + n) / (ops * ops);
        d.A1 = s / (ops * ops);
        d.A2 = (n + s * (2.0 - n)) * s / (ops * ops * ops);
    }
    return d;
}

// The same in FP32 (aJ = |J|).
__device__ EJD ej_with_derivatives_f(const CoilDev& c, int fil, float aJ, float Jc) {
    EJD d = {1.0, 1.0, 0.0, 0.0, 0.0};
    if (!fil || Jc <= 0.0f) return d;
    if (aJ == 0.0f) { d.frac = 0.0; d.dfac = 0.0; return d; }
    const float n = c.f_nexp;
    const float lnx = logf(aJ / Jc);
    d.lnx = lnx;
    const float ell = logf(c.f_E0 / (Jc * c.f_rho_n)) + (n - 1.0f) * lnx;
    if (ell > 0.0f) {
        const float t = expf(-ell), opt = 1.0f + t;
        d.frac = 1.0f / opt;
        d.dfac = (1.0f + n * t) / (opt * opt);
        d.A1 = t / (opt * opt);
        d.A2 = (n * t * t + (2.0f - n) * t) / (opt * opt * opt);
    } else {
        const float sv = expf(ell), ops = 1.0f + sv;
        d.frac = sv / ops;
        d.dfac = sv * (sv + n) / (ops * ops);
        d.A1 = sv / (ops * ops);
        d.A2 = (n + sv * (2.0f - n)) * sv / (ops * ops * ops);
    }
    return d;
}

// Per wire (one warp): reverse of the pointwise kernel and of the constraint.
// wP = dL/dP of the step's Joule power P = sum q 2 pi r a (its diagnostic
// record), which adds wP 2 pi r a to lam_q of every element.
// The mixed form's element of k_adj_pointwise: its forward chain is FP32 from
// the field on (J = I / a included), so are the Jacobian's coefficients,
// formed from the same FP32 geometry without FP64 divisions (B300's FP64 pipe
// gives a warp one instruction per 64 cycles); the adjoint variables and every
// accumulation stay FP64.
__device__ __forceinline__ void adj_element_f(const CoilDev& c, const AdjBufs& ab, int e, double Ba0, double wP,
                                              double nu_term, double& gn, double& gce) {
    const float4 gf = c.geo_f[e];                      // 2 pi r, 1 / (2 pi r), area, 1 / area
    const int fil = c.mat[e];
    const float Jf = (float)c.I[e] * gf.w;             // the forward chain's J
    float br = 0.0f, bz = 0.0f, tf = c.f_T_bath;
    double u = 0.0;
    int g = -1;
    if (c.has_grid) {
        field_at_f(c, e, Ba0, &br, &bz);
        g = c.elem_grid[e];
        u = c.uT[g];
        tf = sqrtf(sqrtf((float)u));
    }
    const float bm = sqrtf(br * br + bz * bz);
    JcD jd = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (fil) jd = jc_with_derivatives_f(c, bm, tf, strain_power_f(c, e, Jf, bz), (float)c.jc_factor[e]);
    const EJD ej = ej_with_derivatives_f(c, fil, fabsf(Jf), (float)jd.Jc);
    const float rn = c.f_rho_n, nf = c.f_nexp, jc = (float)jd.Jc;
    const float A1 = (float)ej.A1, A2 = (float)ej.A2, lnx = (float)ej.lnx;
    const float Kg = gf.x * rn * gf.w;                 // 2 pi r rho_n / a
    const bool act = fil && jc > 0.0f;
    const float cG = (act && Jf != 0.0f) ? Kg * A2 * (nf - 1.0f) / Jf : 0.0f;   // dG/dJ
    const double mu = c.x[e];
    const double lamG = -c.dt * mu * ab.xk[e];
    const double lamR = -mu;
    const double lamq = ((c.has_grid && c.thermal) ? ab.lamQ[g] : 0.0) + wP * (double)(gf.x * gf.z);
    const double lamE = (double)gf.x * lamR + lamq * (double)Jf;
    const double lamJ = lamq * (double)(rn * (float)ej.frac * Jf) + lamE * (double)(rn * (float)ej.dfac) +
                        lamG * (double)cG;
    double lamI = ab.lamI_next[e] + lamJ * (double)gf.w + nu_term;
    if (act) {
        const float ijc = 1.0f / jc;
        const double lamJc = lamE * (double)(-rn * Jf * nf * A1 * ijc) + lamG * (double)(-Kg * A2 * nf * ijc);
        gn += lamE * (double)(rn * Jf * A1 * lnx) + lamG * (double)(Kg * (A2 * lnx + A1));
        ab.g_f[e] += lamJc * jd.df;
        gce += lamJc * jd.dCe;
        const double lamBm = lamJc * jd.dBm;
        const double lamT = lamJc * jd.dT;
        if (c.has_grid && c.thermal) ab.lamU[g] += lamT * (double)(tf / (4.0f * (float)u));
        // lam_B over 2 pi r, the scale of the stencil that k_adj_stencil_t transposes
        const double sB = bm > 0.0f ? lamBm * (double)(gf.y / bm) : 0.0;
        double lbz = sB * (double)bz;
        ab.lamBr[e] = sB * (double)br;
        if (c.lorentz) {
            // Lorentz hoop strain eps = eps0 + r J B_z / Y: d|eps|^p/d eps = p |eps|^p / eps
            const double r = c.r[e], J = (double)Jf;
            const double eps = element_strain(c, e, r, J, (double)bz);
            if (eps != 0.0) {
                const double lamEps = lamJc * jd.dep * c.p_eps * pow(fabs(eps), c.p_eps) / eps;
                lamI += lamEps * r * (double)bz * c.inv_Y * (double)gf.w;
                lbz += lamEps * r * J * c.inv_Y * (double)gf.y;
            }
        }
        ab.lamBz[e] = lbz;
    } else {
        ab.lamBr[e] = 0.0;
        ab.lamBz[e] = 0.0;
    }
    ab.lamI[e] = lamI;
}

__global__ void k_adj_pointwise(const CoilDev* __restrict__ cds, AdjBufs ab, double wP) {
    const CoilDev& c = cds[0];
    int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (w >= c.W) return;
    double dt = c.dt, n = c.nexp, rho_n = c.rho_n;
    double Ba0 = c.sc->Ba0;
    // the mixed form's forward chain is FP32 from the field on: its Jacobians too
    const bool f32 = c.precision != PREC_FP64;
    // -lam_c / dt with lam_c = nu = -u
    double nu_term = c.constrained[w] ? (f32 ? c.uw[w] * c.inv_dt : c.uw[w] / dt) : 0.0;
    double gn = 0.0, gce = 0.0;
    for (int k = lane; k < c.B; k += 32) {
        int e = w * c.B + k;
        if (f32) {
            adj_element_f(c, ab, e, Ba0, wP, nu_term, gn, gce);
            continue;
        }
        double r = c.r[e], a = c.area[e];
        double Br = 0.0, Bz = 0.0, T = c.T_bath, u = 0.0;
        int g = -1;
        int fil = c.mat[e];
        JcD jd = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        double I = c.I[e];
        double J = I / a;
        double Bm;
        if (c.has_grid) {
            field_at(c, e, Ba0, &Br, &Bz);
            g = c.elem_grid[e];
            u = c.uT[g];
            T = sqrt(sqrt(u));
        }
        Bm = sqrt(Br * Br + Bz * Bz);
        if (fil) jd = jc_with_derivatives(c, Bm, T, strain_power(c, e, r, J, Bz), c.jc_factor[e]);
        const EJD ej = ej_with_derivatives(c, fil, J, jd.Jc);
        double E = rho_n * ej.frac * J;
        double Kg = 2.0 * kPi * r * rho_n / a;
        double mu = c.x[e];
        double lamG = -dt * mu * ab.xk[e];
        double lamR = -mu;
        double lamq = ((c.has_grid && c.thermal) ? ab.lamQ[g] : 0.0) + wP * 2.0 * kPi * r * a;
        double lamE = 2.0 * kPi * r * lamR + lamq * J;
        double dGdJ = (fil && jd.Jc > 0.0 && J != 0.0) ? Kg * ej.A2 * (n - 1.0) / J : 0.0;
        double lamJ = lamq * E + lamE * rho_n * ej.dfac + lamG * dGdJ;
        double lamI = ab.lamI_next[e] + lamJ / a + nu_term;
        if (fil && jd.Jc > 0.0) {
            double dEdJc = -rho_n * J * n * ej.A1 / jd.Jc;
            double dGdJc = -Kg * ej.A2 * n / jd.Jc;
            double lamJc = lamE * dEdJc + lamG * dGdJc;
            gn += lamE * rho_n * J * ej.A1 * ej.lnx + lamG * Kg * (ej.A2 * ej.lnx + ej.A1);
            ab.g_f[e] += lamJc * jd.df;
            gce += lamJc * jd.dCe;
            double lamBm = lamJc * jd.dBm;
            double lamT = lamJc * jd.dT;
            if (c.has_grid && c.thermal) ab.lamU[g] += lamT * T / (4.0 * u);
            // lam_B over 2 pi r, the scale of the stencil that k_adj_stencil_t transposes
            const double s2pr = 1.0 / (2.0 * kPi * r);
            const double sB = Bm > 0.0 ? lamBm * s2pr / Bm : 0.0;
            double lbz = sB * Bz;
            ab.lamBr[e] = sB * Br;
            // Lorentz hoop strain eps = eps0 + r J B_z / Y: d|eps|^p/d eps = p |eps|^p / eps
            const double eps = element_strain(c, e, r, J, Bz);
            if (c.inv_Y != 0.0 && eps != 0.0) {
                const double lamEps = lamJc * jd.dep * c.p_eps * pow(fabs(eps), c.p_eps) / eps;
                lamI += lamEps * r * Bz * c.inv_Y / a;
                lbz += lamEps * r * J * c.inv_Y * s2pr;
            }
            ab.lamBz[e] = lbz;
        } else {
            ab.lamBr[e] = 0.0;
            ab.lamBz[e] = 0.0;
        }
        ab.lamI[e] = lamI;
    }
    gn = warp_sum(gn);
    gce = warp_sum(gce);
    if (lane == 0) {
        ab.gparts[w] += gn;
        ab.gparts[c.W + w] += gce;
    }
}

// lam_Phi = S^T lam_B (gather over the stencils that touch each element);
// written as the operator input (d and its FP32 copy) for the transpose apply.
__global__ void k_adj_stencil_t(const CoilDev* __restrict__ cds, AdjBufs ab) {
    const CoilDev& c = cds[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) c.sc->done = 0;
    int Gr = c.Gr, Gz = c.Gz;
    for (int e2 = blockIdx.x * blockDim.x + threadIdx.x; e2 < c.N; e2 += gridDim.x * blockDim.x) {
        int g2 = c.elem_grid[e2];
        int iz2 = g2 / Gr, ir2 = g2 - iz2 * Gr;
        // the stencils of the two cells on either side along each axis: every
        // load in bounds (clamped cell, tap 0 when unused) and issued at once,
        // unused taps not added; a zero weight adds an exact zero (lam_B is finite)
        double acc = 0.0;
#pragma unroll
        for (int d = -2; d <= 2; ++d) {
            const int i = min(max(ir2 + d, 0), Gr - 1);
            const int k = ir2 - c.sr_j0[i];
            const bool use = i == ir2 + d && k >= 0 && k <= 2;
            const double wk = c.sr_w[3 * i + (use ? k : 0)];
            const double lb = ab.lamBz[c.grid_elem[iz2 * Gr + i]];   // lam_B already over 2 pi r
            if (use) acc += wk * lb;
        }
#pragma unroll
        for (int d = -2; d <= 2; ++d) {
            const int j = min(max(iz2 + d, 0), Gz - 1);
            const int k = iz2 - c.sz_j0[j];
            const bool use = j == iz2 + d && k >= 0 && k <= 2;
            const double wk = c.sz_w[3 * j + (use ? k : 0)];
            const double lb = ab.lamBr[c.grid_elem[j * Gr + ir2]];
            if (use) acc -= wk * lb;
        }
        c.dv[e2] = acc;
        c.pf[e2] = (float)acc;
    }
}

// q_w += M_ww d_w (FP64 intra-wire blocks, no dt G term).
__global__ void k_adj_near(const CoilDev* __restrict__ cds) {
    const CoilDev& c = cds[0];
    int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (w >= c.W) return;
    int B = c.B;
    const double* nb = c.near + (size_t)c.block_type[w] * B * B;
    const double* pw = c.dv + (size_t)w * B;
    for (int i = lane; i < B; i += 32) {
        double acc = 0.0;
        for (int j = 0; j < B; ++j) acc += nb[i * B + j] * pw[j];
        c.qv[w * B + i] += acc;
    }
}

// lam_I += M lam_Phi + (dL/dm_k) pi r^2.
__global__ void k_adj_accum(const CoilDev* __restrict__ cds, AdjBufs ab, double wk, int with_field) {
    const CoilDev& c = cds[0];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < c.N; e += gridDim.x * blockDim.x) {
        double r = c.r[e];
        double v = ab.lamI[e] + wk * kPi * r * r;
        if (with_field) v += c.qv[e];
        ab.lamI[e] = v;
    }
}

// lam_I = (dL/dm) pi r^2 (start of the reverse sweep).
__global__ void k_adj_seed(const CoilDev* __restrict__ cds, double* lamI, double wk) {
    const CoilDev& c = cds[0];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < c.N; e += gridDim.x * blockDim.x) {
        double r = c.r[e];
        lamI[e] = wk * kPi * r * r;
    }
}

// dL/dn, dL/dC_eps: deterministic sums of the per-block partials.
__global__ void k_adj_reduce(const CoilDev* __restrict__ cds, const double* gparts, double* out) {
    const CoilDev& c = cds[0];
    __shared__ double sh[2][32];
    double a = 0.0, b = 0.0;
    for (int w = threadIdx.x; w < c.W; w += blockDim.x) {
        a += gparts[w];
        b += gparts[c.W + w];
    }
    a = warp_sum(a);
    b = warp_sum(b);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sh[0][wid] = a; sh[1][wid] = b; }
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        a = lane < nw ? sh[0][lane] : 0.0;
        b = lane < nw ? sh[1][lane] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
        if (lane == 0) { out[0] = a; out[1] = b; }
    }
}

// ---- host launchers ------------------------------------------------------
// Small blocks (two warps): a coil of a few thousand elements then spreads its
// wires and elements over most SMs instead of a few dozen (the reverse step's
// kernels are FP64- and latency-bound, not occupancy-bound).
constexpr int kAdjThreads = 64;

inline unsigned adj_wire_blocks(const CoilDev& h) { return (unsigned)((h.W + kAdjThreads / 32 - 1) / (kAdjThreads / 32)); }
inline unsigned adj_elem_blocks(long long n) {
    long long b = (n + kAdjThreads - 1) / kAdjThreads;
    return (unsigned)(b > 148LL * 32 ? 148LL * 32 : (b < 1 ? 1 : b));
}

// Dynamic shared memory the reverse ADI kernels may take (lines of more than
// 1,536 cells need more than the default 48 KB).
cudaError_t adj_adi_allow_smem(size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_adj_adi_z, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_adj_adi_r, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

void launch_adj_thermal(const CoilDev* d, const CoilDev& h, const AdjBufs& ab, cudaStream_t s) {
    k_adj_adi_z<<<h.Gr, kAdiThreads, adi_smem_bytes(h.Gz), s>>>(d, ab);
    k_adj_adi_r<<<h.Gz, kAdiThreads, adi_smem_bytes(h.Gr), s>>>(d, ab);
    k_adj_adi_src<<<adj_elem_blocks((long long)h.Gr * h.Gz), kAdjThreads, 0, s>>>(d, ab);
}

void launch_adj_setup(const CoilDev* d, const CoilDev& h, const AdjBufs& ab, cudaStream_t s) {
    k_adj_setup<<<adj_wire_blocks(h), kAdjThreads, 0, s>>>(d, ab);
}

void launch_adj_mult_pointwise(const CoilDev* d, const CoilDev& h, const AdjBufs& ab, double wP, cudaStream_t s) {
    k_adj_mult<<<adj_wire_blocks(h), kAdjThreads, 0, s>>>(d);
    k_adj_pointwise<<<adj_wire_blocks(h), kAdjThreads, 0, s>>>(d, ab, wP);
}

void launch_adj_stencil_t(const CoilDev* d, const CoilDev& h, const AdjBufs& ab, cudaStream_t s) {
    k_adj_stencil_t<<<adj_elem_blocks(h.N), kAdjThreads, 0, s>>>(d, ab);
}

void launch_adj_near(const CoilDev* d, const CoilDev& h, cudaStream_t s) {
    k_adj_near<<<adj_wire_blocks(h), kAdjThreads, 0, s>>>(d);
}

void launch_adj_accum(const CoilDev* d, const CoilDev& h, const AdjBufs& ab, double wk, int with_field,
                      cudaStream_t s) {
    k_adj_accum<<<adj_elem_blocks(h.N), kAdjThreads, 0, s>>>(d, ab, wk, with_field);
}

void launch_adj_seed(const CoilDev* d, const CoilDev& h, double* lamI, double wk, cudaStream_t s) {
    k_adj_seed<<<adj_elem_blocks(h.N), kAdjThreads, 0, s>>>(d, lamI, wk);
}

void launch_adj_reduce(const CoilDev* d, const double* gparts, double* out, cudaStream_t s) {
    k_adj_reduce<<<1, 256, 0, s>>>(d, gparts, out);
}

}  // namespace cq
