// Time discretisations of the modal oscillator q'' + 2 gamma q' + omega^2 q = F
// (Sec. 3.2), both written as the difference form the kernels step:
//     v^{n+1} = v^n - eps v^n - rho q^n + r F^n,   q^{n+1} = q^n + v^{n+1}.
// It equals the three-term recursion q^{n+1} = g q^n + p q^{n-1} + r F^n with
// eps = 1 + p and rho = 1 - g - p.
//
//   Stormer-Verlet (Eq. 20-23):  r = T^2/(1+gamma T), eps = 2 gamma T/(1+gamma T),
//                                rho = r omega^2.
//   Impulse invariance (Eq. 15-19, with the denominator's roots for the
//   signs and the factor T of a sampled force in b1): with
//   w~ = sqrt(omega^2 - gamma^2) and e = exp(-gamma T),
//                                g = 2 e cos(w~ T), p = -e^2, r = T e sin(w~ T)/w~,
//                                eps = -expm1(-2 gamma T),
//                                rho = expm1(-gamma T)^2 + 4 e sin^2(w~ T / 2)
//   (both written without cancellation).  The impulse-invariant form is
//   used for oscillatory modes only (omega > gamma).
//
// The gradient epilogue needs the partial derivatives of (eps, rho, r) with
// respect to (omega^2, gamma); the adjoint sweep accumulates
//   A = sum a^{n+1} q^n, V = sum a^{n+1} v^n, F = sum a^{n+1} F^n,
// so that dL/d rho = -A, dL/d eps = -V, dL/d r = F.
#pragma once

#include <math.h>

#include "../../include/mdx.h"

namespace mdx {

struct SchemeCoef {
    double eps, rho, r;
};

struct SchemeDeriv {
    double eps_w2, eps_gm, rho_w2, rho_gm, r_w2, r_gm;
};

__host__ __device__ inline SchemeCoef scheme_coef(int scheme, double w2, double gm, double T) {
    SchemeCoef c;
    if (scheme == MDX_SCHEME_TF) {
        const double wt = sqrt(w2 - gm * gm);
        const double e = exp(-gm * T);
        const double em = expm1(-gm * T);
        const double sh = sin(0.5 * wt * T);
        c.eps = -expm1(-2.0 * gm * T);
        c.rho = em * em + 4.0 * e * sh * sh;
        c.r = T * e * sin(wt * T) / wt;
    } else {
        const double den = 1.0 + gm * T;
        const double rr = T * T / den;
        c.eps = 2.0 * gm * T / den;
        c.rho = rr * w2;
        c.r = rr;
    }
    return c;
}

__host__ __device__ inline SchemeDeriv scheme_deriv(int scheme, double w2, double gm, double T) {
    SchemeDeriv d;
    if (scheme == MDX_SCHEME_TF) {
        const double wt = sqrt(w2 - gm * gm);
        const double e = exp(-gm * T);
        const double s = sin(wt * T), co = cos(wt * T);
        const double r = T * e * s / wt;
        const double g = 2.0 * e * co, p = -e * e;
        // d/dw~ of sin(w~ T)/w~
        const double ds = (T * co * wt - s) / (wt * wt);
        d.eps_w2 = 0.0;
        d.eps_gm = 2.0 * T * e * e;
        d.rho_w2 = r;                                   // -dg/domega^2
        d.rho_gm = T * g - 2.0 * gm * r + 2.0 * T * p;  // -dg/dgamma - dp/dgamma
        d.r_w2 = T * e * ds / (2.0 * wt);
        d.r_gm = -T * r - T * e * ds * gm / wt;
    } else {
        const double den = 1.0 + gm * T;
        const double den2 = den * den;
        d.eps_w2 = 0.0;
        d.eps_gm = 2.0 * T / den2;
        d.rho_w2 = T * T / den;
        d.rho_gm = -T * T * T * w2 / den2;
        d.r_w2 = 0.0;
        d.r_gm = -T * T * T / den2;
    }
    return d;
}

// FP32 coefficients of one mode as the kernels read them: eps, rho as an
// unevaluated pair rho_hi + rho_lo (rho is subtracted from the state every
// step, so its rounding error would otherwise shift the mode's frequency), r.
struct ModeF32 {
    float eps, rho_hi, rho_lo, r;
};

inline ModeF32 mode_f32(int scheme, double w2, double gm, double T) {
    const SchemeCoef k = scheme_coef(scheme, w2, gm, T);
    ModeF32 o;
    o.eps = (float)k.eps;
    o.rho_hi = (float)k.rho;
    o.rho_lo = (float)(k.rho - (double)o.rho_hi);
    o.r = (float)k.r;
    return o;
}

// dL/d omega^2 and dL/d gamma from the adjoint sums (see above).
__host__ __device__ inline void scheme_grads(int scheme, double w2, double gm, double T, double A,
                                             double V, double F, double *d_w2, double *d_gm) {
    const SchemeDeriv d = scheme_deriv(scheme, w2, gm, T);
    *d_w2 = -A * d.rho_w2 - V * d.eps_w2 + F * d.r_w2;
    *d_gm = -A * d.rho_gm - V * d.eps_gm + F * d.r_gm;
}

}  // namespace mdx
