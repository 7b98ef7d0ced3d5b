// Real spherical harmonics in FP32 from Cartesian recurrences (Sec. 'Spherical Harmonics'; orthonormal, no
// Condon-Shortley phase, lm = l^2 + l + m).
//
// For a unit vector (x, y, z): Y_{l,+m} = Q_l^m C_m, Y_{l,-m} = Q_l^m S_m, Y_{l,0} = Q_l^0, with
// C_m + i S_m = (x + i y)^m and Q_l^m the normalised associated-Legendre polynomial without its (1 - z^2)^{m/2}
// factor (times sqrt 2 for m > 0). Q obeys
//   Q_m^m = K_m,   K_0 = 1/sqrt(4 pi),  K_m = K_{m-1} sqrt((2m+1)/(2m)) (times sqrt 2 at m = 1)
//   Q_l^m = A_lm (z Q_{l-1}^m - B_lm Q_{l-2}^m),  A_lm = sqrt((4l^2-1)/(l^2-m^2)),  B_lm = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1))
// so no trigonometric function is evaluated. The gradient variant carries d/dx, d/dy, d/dz of the polynomial
// extension and projects it on the tangent plane.
//
// Each translation unit that includes this header owns its copy of the constant tables and must call
// upload_ylm_constants() once (done from rascal_create).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace rascal {

static __constant__ float c_ylm_A[16 * 16];
static __constant__ float c_ylm_B[16 * 16];
static __constant__ float c_ylm_K[16];

static inline cudaError_t upload_ylm_constants(cudaStream_t stream) {
    float A[256], B[256], K[16];
    for (int i = 0; i < 256; ++i) A[i] = B[i] = 0.0f;
    double k = 1.0 / sqrt(4.0 * M_PI);
    for (int m = 0; m < 16; ++m) {
        if (m > 0) k *= sqrt((2.0 * m + 1.0) / (2.0 * m)) * (m == 1 ? sqrt(2.0) : 1.0);
        K[m] = (float)k;
        for (int l = m + 1; l < 16; ++l) {
            A[l * 16 + m] = (float)sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
            const double lm1 = l - 1.0;
            B[l * 16 + m] = (l - 1 > m) ? (float)sqrt((lm1 * lm1 - (double)m * m) / (4.0 * lm1 * lm1 - 1.0)) : 0.0f;
        }
    }
    cudaError_t e = cudaMemcpyToSymbolAsync(c_ylm_A, A, sizeof(A), 0, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_ylm_B, B, sizeof(B), 0, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_ylm_K, K, sizeof(K), 0, cudaMemcpyHostToDevice, stream);
    return e;
}

// Y for l <= l_max at unit vector (x, y, z), stored at out[lp[l] + l + m]; padded slots are left untouched.
__device__ inline void ylm_padded(float x, float y, float z, int l_max, const int* __restrict__ lp,
                                  float* __restrict__ out) {
    float cm = 1.0f, sm = 0.0f;  // (x + i y)^m
    for (int m = 0; m <= l_max; ++m) {
        float q2 = 0.0f, q1 = c_ylm_K[m];
        if (m == 0) {
            out[lp[0]] = q1;
        } else {
            out[lp[m] + 2 * m] = q1 * cm;
            out[lp[m]] = q1 * sm;
        }
        for (int l = m + 1; l <= l_max; ++l) {
            const float q = c_ylm_A[l * 16 + m] * (z * q1 - c_ylm_B[l * 16 + m] * q2);
            if (m == 0) {
                out[lp[l] + l] = q;
            } else {
                out[lp[l] + l + m] = q * cm;
                out[lp[l] + l - m] = q * sm;
            }
            q2 = q1;
            q1 = q;
        }
        const float nc = cm * x - sm * y;
        const float ns = cm * y + sm * x;
        cm = nc;
        sm = ns;
    }
}

}  // namespace rascal
