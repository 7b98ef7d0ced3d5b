// FP64 device evaluation of the GTO radial integral (Eq. rad-int-gto-1) through the restricted 1F1 function
// G(a, b, r) = Gamma(a)/Gamma(b) exp(-c r^2) 1F1(a; b; c^2 r^2/(c + d)) of Appendix A.
//
// The power series and the large-z asymptotic series both carry exp(-c r^2) inside their first term, so no
// intermediate overflows (Appendix A notes z - c r^2 < 0). Below a per-(a, b) switch point the power series is
// used, above it the asymptotic series truncated at its smallest term. The switch points are found once per
// context by a parallel multisection (32 probes per round, 5 rounds) for the smallest z in [1, 300] from which the
// two forms agree to 1e-13 relative.
//
// FP64 runs on the GPU only here: for building the spline table and the MLP training targets.
#pragma once

#include <cuda_runtime.h>

namespace rascal {

// e[l] = e^-z i_l(z), l = 0..L (L <= 16), with i_l the modified spherical Bessel function of the first kind, for
// z >= 0. Small z: the power series z^l/(2l+1)!! (1 + z^2/(2(2l+3)) + z^4/(8(2l+3)(2l+5))). Otherwise Miller's
// downward recurrence i_{l-1} = i_{l+1} + (2l+1)/z i_l from far above L (stable downwards), rescaled on the way
// to stay in range, then normalised by e^-z i_0(z) = (1 - e^-2z)/(2z).
__device__ inline void bessel_i_scaled(int L, double z, double* e) {
    if (z < 1e-4) {
        double df = 1.0, zl = 1.0;
        const double ez = exp(-z);
        for (int l = 0; l <= L; ++l) {
            df *= (2 * l + 1);
            e[l] = ez * zl / df * (1.0 + z * z / (2.0 * (2 * l + 3)) + z * z * z * z / (8.0 * (2 * l + 3) * (2 * l + 5)));
            zl *= z;
        }
        return;
    }
    const int top = L + 40 + (int)(z + 4.0 * sqrt(z));
    double fp1 = 0.0, f = 1e-280;  // values at l + 1 and l
    for (int l = top; l >= 1; --l) {
        const double fm1 = fp1 + (2 * l + 1) / z * f;
        fp1 = f;
        f = fm1;
        if (l - 1 <= L) e[l - 1] = f;
        if (fabs(f) > 1e250) {
            f *= 1e-250;
            fp1 *= 1e-250;
            for (int k = l - 1; k <= L; ++k)
                if (k >= 0) e[k] *= 1e-250;
        }
    }
    const double s = (-expm1(-2.0 * z) / (2.0 * z)) / e[0];
    for (int l = 0; l <= L; ++l) e[l] *= s;
}

// DVR radial integrals (Eq. rad-int-dvr, with the constant 4 pi and the density factor exp(-a r^2) kept):
// I_nl(r) = 4 pi x_n sqrt(w_n) exp(-a (x_n - r)^2) e^-z i_l(z), z = 2 a x_n r, and dI_nl/dr, for l = 0..l_max.
__device__ inline void dvr_radial(int l_max, double a, double x, double w, double r, double* I, double* dI) {
    double e[18];
    const double z = 2.0 * a * x * r;
    bessel_i_scaled(l_max + 1, z, e);
    const double g = 4.0 * 3.14159265358979323846 * x * sqrt(w) * exp(-a * (x - r) * (x - r));
    for (int l = 0; l <= l_max; ++l) {
        I[l] = g * e[l];
        if (dI) {
            // d/dz [e^-z i_l] = e^-z (i_{l+1} + (l/z) i_l - i_l); (l/z) e^-z i_l tends to 1/3 (l = 1) or 0 at z = 0
            const double lz = (z > 0.0) ? l / z * e[l] : (l == 1 ? 1.0 / 3.0 : 0.0);
            dI[l] = g * (2.0 * a * (x - r) * e[l] + 2.0 * a * x * (e[l + 1] + lz - e[l]));
        }
    }
}

__device__ inline double g_series(double a, double b, double z, double log_scale) {
    double term = exp(lgamma(a) - lgamma(b) + log_scale);
    double sum = term;
    for (int s = 0; s < 20000; ++s) {
        term *= (a + s) * z / ((b + s) * (s + 1.0));
        sum += term;
        const bool shrinking = (a + s + 1.0) * z < (b + s + 1.0) * (s + 2.0);
        if (shrinking && term <= 1e-17 * sum) break;
    }
    return sum;
}

__device__ inline double g_asymptotic(double a, double b, double z, double log_scale) {
    double term = 1.0, sum = 1.0;
    for (int s = 0; s < 400; ++s) {
        const double nxt = term * (b - a + s) * (1.0 - a + s) / ((s + 1.0) * z);
        if (nxt == 0.0 || fabs(nxt) >= fabs(term)) break;
        sum += nxt;
        term = nxt;
        if (fabs(nxt) <= 1e-17 * fabs(sum)) break;
    }
    return exp(z + log_scale + (a - b) * log(z)) * sum;
}

// G(a, b, r) for one r; zs is the switch point of this (a, b)
__device__ inline double g_eval(double a, double b, double c, double d, double r, double zs) {
    const double z = c * c * r * r / (c + d);
    const double cr2 = c * r * r;
    if (z < zs) return g_series(a, b, z, -cr2);
    return g_asymptotic(a, b, z, -cr2);
}

}  // namespace rascal
