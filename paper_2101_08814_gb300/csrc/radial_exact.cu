// The radial integrals evaluated per pair from their closed forms, without spline or network (radial mode EXACT).
// GTO basis: Eq. rad-int-gto-1 with the restricted 1F1 G(a, b, r) of Appendix A, followed by the o-GTO transform S^-1/2.
//
// For each pair and radial index n, four G values are evaluated directly (series below the switch point, asymptotic
// series above): the main values M_l = G(a_l, b_l) and the auxiliary values X_l = G(a_l + 1, b_l + 1) at
// l = l_max and l_max - 1 (a_l = (n+l+3)/2, b_l = l + 3/2). All lower l follow from the two-step downward recurrence
// of Eq. 1f1-recurrence, which in this notation reads
//   X_l = z X_{l+2} + (b_l + 1) M_{l+2},      M_l = z (a_l - b_l)/a_l M_{l+2} + (b_l/a_l) X_l,
// with z = c^2 r^2/(c + d_n); the auxiliary values also give the derivative dG/dr = 2c^2 r/(c+d) X_l - 2 c r M_l.
// That is 4 n_max direct evaluations per pair for all (n, l), as Appendix A counts them.
//
// The work is FP64: the o-GTO transform cancels up to cond(S)^1/2 (about 2e5 at n_max = 16) between its terms,
// which FP32 inputs cannot survive. The result is rounded to FP32 per pair, in the [pair][l][n] layout the pair
// kernels read.
#include <algorithm>

#include "common.cuh"
#include "radial_fp64.cuh"

namespace rascal {

__global__ void k_exact_raw(int64_t np, const float4* __restrict__ rij, int n_max, int l_max, double c,
                            const double* __restrict__ gto, const double* __restrict__ zs, double* __restrict__ raw,
                            double* __restrict__ draw) {
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= np * n_max) return;
    const int64_t p = id / n_max;
    const int n = (int)(id % n_max);
    const int L1 = l_max + 1, L2 = l_max + 2;
    const double r = (double)rij[p].w;
    const double d = gto[n], Nn = gto[(n_max + 1) + n];
    const double z = c * c * r * r / (c + d);
    double M[kMaxLMax + 3], X[kMaxLMax + 3];
    for (int l = l_max; l >= 0 && l >= l_max - 1; --l) {
        const double a = 0.5 * (n + l + 3), b = l + 1.5;
        M[l] = g_eval(a, b, c, d, r, zs[n * L2 + l]);
        X[l] = g_eval(a + 1.0, b + 1.0, c, d, r, zs[(n + 1) * L2 + (l + 1)]);
    }
    for (int l = l_max - 2; l >= 0; --l) {
        const double a = 0.5 * (n + l + 3), b = l + 1.5;
        X[l] = z * X[l + 2] + (b + 1.0) * M[l + 2];
        M[l] = z * (a - b) / a * M[l + 2] + b / a * X[l];
    }
    const double pi15 = 5.568327996831707845;
    for (int l = 0; l <= l_max; ++l) {
        const double a = 0.5 * (n + l + 3);
        const double pref = pi15 * Nn * exp(l * log(c) - a * log(c + d));
        const double rl = (l == 0) ? 1.0 : pow(r, (double)l);
        const double drl = (l == 0) ? 0.0 : (l == 1 ? 1.0 : l * pow(r, (double)(l - 1)));
        const double dg = 2.0 * c * c * r / (c + d) * X[l] - 2.0 * c * r * M[l];
        raw[((p * n_max) + n) * L1 + l] = pref * rl * M[l];
        if (draw) draw[((p * n_max) + n) * L1 + l] = pref * (drl * M[l] + rl * dg);
    }
}

// o-GTO transform per (pair, l), FP64 -> FP32 in the [pair][l][n] layout (f = l n_max + n)
__global__ void k_exact_mix(int64_t np, int n_max, int l_max, const double* __restrict__ T, const double* __restrict__ raw,
                            const double* __restrict__ draw, float* __restrict__ out, float* __restrict__ dout) {
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int L1 = l_max + 1;
    if (id >= np * L1) return;
    const int64_t p = id / L1;
    const int l = (int)(id % L1);
    const int F = n_max * L1;
    for (int n = 0; n < n_max; ++n) {
        double acc = 0.0, dacc = 0.0;
        for (int k = 0; k < n_max; ++k) {
            acc += T[n * n_max + k] * raw[(p * n_max + k) * L1 + l];
            if (draw) dacc += T[n * n_max + k] * draw[(p * n_max + k) * L1 + l];
        }
        out[p * F + l * n_max + n] = (float)acc;
        if (dout) dout[p * F + l * n_max + n] = (float)dacc;
    }
}

// DVR integrals per (pair, n) in FP64 (Eq. rad-int-dvr; the basis is orthonormal, no transform follows), rounded to
// FP32 in the [pair][l][n] layout.
__global__ void k_exact_dvr(int64_t np, const float4* __restrict__ rij, int n_max, int l_max, double a,
                            const double* __restrict__ dvr, float* __restrict__ out, float* __restrict__ dout) {
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= np * n_max) return;
    const int64_t p = id / n_max;
    const int n = (int)(id % n_max);
    const int F = n_max * (l_max + 1);
    double I[kMaxLMax + 1], dI[kMaxLMax + 1];
    dvr_radial(l_max, a, dvr[n], dvr[n_max + n], (double)rij[p].w, I, dout ? dI : nullptr);
    for (int l = 0; l <= l_max; ++l) {
        out[p * F + l * n_max + n] = (float)I[l];
        if (dout) dout[p * F + l * n_max + n] = (float)dI[l];
    }
}

// Per-pair radial values for the EXACT and MLP radial modes, computed before the pair kernels run (the SPLINE mode
// evaluates its table inside them and leaves *pre_G = NULL). Reads the pair count from the device (one stream sync).
int radial_precompute(rascal_ctx* ctx, const rascal_system* sys, const int64_t* d_offsets, const float* d_rij, bool deriv,
                      const float** pre_G, const float** pre_D) {
    *pre_G = nullptr;
    *pre_D = nullptr;
    if (ctx->radial == RASCAL_RADIAL_SPLINE) return RASCAL_OK;
    if (ctx->radial == RASCAL_RADIAL_MLP && !ctx->mlp_params)
        return set_error(RASCAL_E_ARG, "radial mode MLP needs trained parameters (rascal_mlp_set_params / rascal_mlp_load)");
    RASCAL_CUDA(cudaMemcpyAsync(ctx->h_pinned, d_offsets + sys->n_atoms, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    RASCAL_CUDA(cudaStreamSynchronize(ctx->stream));
    const int64_t P = ctx->h_pinned[0];
    if (P <= 0) return RASCAL_OK;
    const size_t words = (size_t)P * ctx->F;
    void* base;
    int st = arena_get(ctx->scratch, carve_bytes(words * 4, deriv ? words * 4 : 4), &base);
    if (st) return st;
    Carver cv(base);
    float* G = cv.take<float>(words);
    float* D = deriv ? cv.take<float>(words) : nullptr;
    const float4* rij = reinterpret_cast<const float4*>(d_rij);
    st = ctx->radial == RASCAL_RADIAL_MLP ? mlp_infer(ctx, P, rij, nullptr, G, D) : radial_exact_pairs(ctx, P, rij, G, D);
    if (st) return st;
    *pre_G = G;
    *pre_D = D;
    return RASCAL_OK;
}

int radial_exact_pairs(rascal_ctx* ctx, int64_t n, const float4* rij, float* out, float* dout) {
    const int n_max = ctx->n_max, L1 = ctx->l_max + 1;
    const double c = 1.0 / (2.0 * ctx->sigma * ctx->sigma);
    if (ctx->basis == RASCAL_BASIS_DVR) {
        if (n == 0) return RASCAL_OK;
        k_exact_dvr<<<(unsigned)div_up(n * n_max, 128), 128, 0, ctx->stream>>>(n, rij, n_max, ctx->l_max, c, ctx->d_dvr,
                                                                            out, dout);
        RASCAL_LAUNCH_CHECK("k_exact_dvr");
        return RASCAL_OK;
    }
    const int64_t batch = std::min<int64_t>(n, 1 << 16);
    for (int64_t start = 0; start < n; start += batch) {
        const int64_t nb = std::min<int64_t>(batch, n - start);
        const size_t words = (size_t)nb * n_max * L1;
        void* base;
        int st = arena_get(ctx->scratch2, carve_bytes(words * 8, dout ? words * 8 : 8), &base);
        if (st) return st;
        Carver cv(base);
        double* raw = cv.take<double>(words);
        double* draw = dout ? cv.take<double>(words) : nullptr;
        k_exact_raw<<<(unsigned)div_up(nb * n_max, 128), 128, 0, ctx->stream>>>(nb, rij + start, n_max, ctx->l_max, c, ctx->d_gto,
                                                                              ctx->d_switch, raw, draw);
        RASCAL_LAUNCH_CHECK("k_exact_raw");
        k_exact_mix<<<(unsigned)div_up(nb * L1, 128), 128, 0, ctx->stream>>>(nb, n_max, ctx->l_max, ctx->d_T, raw, draw,
                                                                           out + start * (int64_t)ctx->F,
                                                                           dout ? dout + start * (int64_t)ctx->F : nullptr);
        RASCAL_LAUNCH_CHECK("k_exact_mix");
    }
    return RASCAL_OK;
}

}  // namespace rascal
