// Pointwise pieces of the step shared by the forward and adjoint kernels:
// the field from the loop-flux stencil, Jc(B, T, eps) and the E-J law.
#pragma once

#include "common.cuh"

namespace cq {

// ---------------------------------------------------------------- pointwise

__device__ __forceinline__ double phi_total(const CoilDev& c, int g, double Ba) {
    int e = c.grid_elem[g];
    double r = c.r[e];
    return c.Phi[e] + kPi * r * r * Ba;
}

// B_r, B_z at element e from the stencil of the total loop flux.
__device__ __forceinline__ void field_at(const CoilDev& c, int e, double Ba, double* Br, double* Bz) {
    int g = c.elem_grid[e];
    int iz = g / c.Gr, ir = g - iz * c.Gr;
    double dr = 0.0, dz = 0.0;
    int j0 = c.sr_j0[ir];
    for (int k = 0; k < 3; ++k) {
        double wk = c.sr_w[3 * ir + k];
        if (wk != 0.0) dr += wk * phi_total(c, iz * c.Gr + j0 + k, Ba);
    }
    j0 = c.sz_j0[iz];
    for (int k = 0; k < 3; ++k) {
        double wk = c.sz_w[3 * iz + k];
        if (wk != 0.0) dz += wk * phi_total(c, (j0 + k) * c.Gr + ir, Ba);
    }
    double r = c.r[e];
    *Bz = dr / (2.0 * kPi * r);
    *Br = -dz / (2.0 * kPi * r);
}

// Strain of element e: the static strain, plus with the Lorentz hoop strain
// (inv_Y > 0) r J B_z / Y_eff from the start-of-step J and B_z (Flux Jumps
// Propagation section: the electromagnetic strain from the Lorentz force).
__device__ __forceinline__ double element_strain(const CoilDev& c, int e, double r, double J, double Bz) {
    return c.strain[e] + r * J * Bz * c.inv_Y;
}

// pe = |eps|^p_eps of element e: tabulated at coil creation for the static
// strain, evaluated per step with the Lorentz term.
__device__ __forceinline__ double strain_power(const CoilDev& c, int e, double r, double J, double Bz) {
    if (c.inv_Y == 0.0) return c.strain_pow[e];
    return pow(fabs(element_strain(c, e, r, J, Bz)), c.p_eps);
}

// pe = |eps|^p_eps of the element.
__device__ __forceinline__ double critical_current(const CoilDev& c, double Bm, double T, double pe, double f) {
    if (c.jc_model == 1) return f * c.Jc0;
    double tr = T / c.Tc;
    double Bc2 = c.Bc2_0 * (1.0 - tr * tr);
    if (!(T < c.Tc && Bm < Bc2)) return 0.0;
    double strain = fmax(0.0, 1.0 - c.C_eps * pe);
    double bfac = 1.0 - Bm / Bc2;
    double omt = 1.0 - tr;
    return f * c.Jc0 * (omt * sqrt(omt)) * (bfac * bfac) / sqrt(Bm + c.B_reg) * strain;
}

// rho/rho_n, (dE/dJ)/rho_n and |J|/Jc of the parallel power-law / normal law.
__device__ __forceinline__ void ej_law(const CoilDev& c, int fil, double J, double Jc, double* frac, double* dfac,
                       double* jrat) {
    if (!fil) { *frac = 1.0; *dfac = 1.0; *jrat = 0.0; return; }
    double aJ = fabs(J);
    if (Jc <= 0.0) { *frac = 1.0; *dfac = 1.0; *jrat = aJ > 0.0 ? __longlong_as_double(0x7ff0000000000000LL) : 0.0; return; }
    *jrat = aJ / Jc;
    if (aJ == 0.0) { *frac = 0.0; *dfac = 0.0; return; }
    double n = c.nexp;
    double ell = log(c.E0 / (Jc * c.rho_n)) + (n - 1.0) * log(aJ / Jc);
    if (ell > 0.0) {
        double t = exp(-ell);
        double opt = 1.0 + t;
        *frac = 1.0 / opt;
        *dfac = (1.0 + n * t) / (opt * opt);
    } else {
        double s = exp(ell);
        double ops = 1.0 + s;
        *frac = s / ops;
        *dfac = s * (s + n) / (ops * ops);
    }
}

// ------------------------------------------------- FP32 forms (mixed mode)
//
// The mixed form (far operator stored in FP32 or as FP16 hi/lo pairs) takes
// the field and the constitutive chain in FP32, as its precision plan says:
// the stencil's flux differences are summed in FP64 (they cancel across one
// element) and only then rounded, T, Jc, the E-J law's logarithm and
// exponential, rho/rho_n and its derivative are FP32; the currents, the
// products that form G, R and q, and every accumulation stay FP64.  B300's
// FP64 pipe issues two thread-operations per SM per clock, so the FP64
// logarithms, exponentials, divisions and square roots of this chain bound
// the FP64 kernel; in FP32 they run on the 128-lane pipe.  The E-J law
// amplifies a relative error of Jc by n in E, but the current that the solve
// returns moves by about the error of Jc itself (J ~ Jc (E/E0)^(1/n)).

// B_r, B_z at element e in FP32 from FP64 stencil sums.
__device__ __forceinline__ void field_at_f(const CoilDev& c, int e, double Ba, float* Br, float* Bz) {
    int g = c.elem_grid[e];
    int iz = g / c.Gr, ir = g - iz * c.Gr;
    double dr = 0.0, dz = 0.0;
    int j0 = c.sr_j0[ir];
    for (int k = 0; k < 3; ++k) {
        double wk = c.sr_w[3 * ir + k];
        if (wk != 0.0) dr += wk * phi_total(c, iz * c.Gr + j0 + k, Ba);
    }
    j0 = c.sz_j0[iz];
    for (int k = 0; k < 3; ++k) {
        double wk = c.sz_w[3 * iz + k];
        if (wk != 0.0) dz += wk * phi_total(c, (j0 + k) * c.Gr + ir, Ba);
    }
    const float inv = 1.0f / (float)(2.0 * kPi * c.r[e]);
    *Bz = (float)dr * inv;
    *Br = -(float)dz * inv;
}

template <typename TJ>
__device__ __forceinline__ float strain_power_f(const CoilDev& c, int e, TJ J, float Bz) {
    if (!c.lorentz) return c.strain_pow_f[e];
    const float eps = (float)c.strain[e] + (float)(c.r[e] * (double)J * c.inv_Y) * Bz;
    return powf(fabsf(eps), c.f_p_eps);
}

__device__ __forceinline__ float critical_current_f(const CoilDev& c, float Bm, float T, float pe, float f) {
    if (c.jc_model == 1) return f * c.f_Jc0;
    const float tr = T / c.f_Tc;
    const float Bc2 = c.f_Bc2_0 * (1.0f - tr * tr);
    if (!(T < c.f_Tc && Bm < Bc2)) return 0.0f;
    const float strain = fmaxf(0.0f, 1.0f - c.f_C_eps * pe);
    const float bfac = 1.0f - Bm / Bc2;
    const float omt = 1.0f - tr;
    return f * c.f_Jc0 * (omt * sqrtf(omt)) * (bfac * bfac) / sqrtf(Bm + c.f_B_reg) * strain;
}

__device__ __forceinline__ void ej_law_f(const CoilDev& c, int fil, float aJ, float Jc, float* frac, float* dfac,
                                         float* jrat) {
    if (!fil) { *frac = 1.0f; *dfac = 1.0f; *jrat = 0.0f; return; }
    if (Jc <= 0.0f) { *frac = 1.0f; *dfac = 1.0f; *jrat = aJ > 0.0f ? __int_as_float(0x7f800000) : 0.0f; return; }
    *jrat = aJ / Jc;
    if (aJ == 0.0f) { *frac = 0.0f; *dfac = 0.0f; return; }
    const float n = c.f_nexp;
    const float ell = logf(c.f_E0 / (Jc * c.f_rho_n)) + (n - 1.0f) * logf(aJ / Jc);
    if (ell > 0.0f) {
        const float t = expf(-ell);
        const float opt = 1.0f + t;
        *frac = 1.0f / opt;
        *dfac = (1.0f + n * t) / (opt * opt);
    } else {
        const float s = expf(ell);
        const float ops = 1.0f + s;
        *frac = s / ops;
        *dfac = s * (s + n) / (ops * ops);
    }
}

}  // namespace cq
