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
