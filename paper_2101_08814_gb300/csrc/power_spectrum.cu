// Power spectrum (Eq. nu2-basis-coupled) from stored coefficients: one CTA per centre, the centre's block
// c[q][lm] is read once (coalesced), transposed into shared memory as CT[lm][q] and contracted per l by the FP32
// register-tiled Gram of ps_fp32.cuh.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "ps_fp32.cuh"

namespace rascal {

constexpr int kPsThreads = 256;

__global__ void __launch_bounds__(kPsThreads) k_power_spectrum_fp32(const float* __restrict__ coeffs, int Q, int Qp,
                                                                     int n_lm, int l_max, int ps_norm,
                                                                     const int* __restrict__ tasks, int n_tasks,
                                                                     int layout, int64_t ps_stride, float* __restrict__ ps) {
    extern __shared__ __align__(16) float CT[];  // [n_lm][Qp]
    const int64_t i = blockIdx.x;
    const float* c = coeffs + i * (int64_t)Q * n_lm;
    const int total = Q * n_lm;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int q = e / n_lm, lm = e - q * n_lm;
        CT[lm * Qp + q] = c[e];
    }
    for (int e = threadIdx.x; e < n_lm * (Qp - Q); e += blockDim.x) {
        const int lm = e / (Qp - Q), q = Q + e % (Qp - Q);
        CT[lm * Qp + q] = 0.0f;
    }
    __syncthreads();
    ps_gram_fp32(CT, Qp, Q, l_max, ps_norm, tasks, n_tasks, layout, ps + i * ps_stride);
}

int power_spectrum_setup(rascal_ctx* ctx) {
    const int Q4 = (ctx->Q + 3) / 4;
    std::vector<int> tasks;
    for (int l = ctx->l_max; l >= 0; --l)
        for (int t1 = 0; t1 < Q4; ++t1)
            for (int t2 = t1; t2 < Q4; ++t2) tasks.push_back(l | (t1 << 8) | (t2 << 16));
    ctx->n_pstasks = (int)tasks.size();
    RASCAL_CUDA(cudaMalloc(&ctx->d_pstasks, sizeof(int) * tasks.size()));
    RASCAL_CUDA(cudaMemcpyAsync(ctx->d_pstasks, tasks.data(), sizeof(int) * tasks.size(), cudaMemcpyHostToDevice, ctx->stream));
    RASCAL_CUDA(cudaFuncSetAttribute(k_power_spectrum_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    RASCAL_CUDA(cudaStreamSynchronize(ctx->stream));
    return RASCAL_OK;
}

}  // namespace rascal

using namespace rascal;

extern "C" int rascal_power_spectrum(rascal_ctx* ctx, int64_t n_centres, const float* d_coeffs, int precision,
                                     int layout, float* d_ps) {
    clear_error();
    if (!ctx) return set_error(RASCAL_E_ARG, "NULL context");
    if (n_centres < 0) return set_error(RASCAL_E_ARG, "negative n_centres");
    if (layout != RASCAL_LAYOUT_PACKED && layout != RASCAL_LAYOUT_FULL) return set_error(RASCAL_E_ARG, "unknown layout");
    if (precision != RASCAL_PS_FP32 && precision != RASCAL_PS_BF16) return set_error(RASCAL_E_ARG, "unknown precision");
    if (n_centres == 0) return RASCAL_OK;
    if (!d_coeffs || !d_ps) return set_error(RASCAL_E_ARG, "NULL device pointer");
    if (n_centres > 0x7fffffffLL) return set_error(RASCAL_E_UNSUPPORTED, "more than 2^31-1 centres in one call");
    const int Q = ctx->Q, Qp = (Q + 3) / 4 * 4;
    const int64_t stride = (int64_t)(ctx->l_max + 1) * (layout == RASCAL_LAYOUT_PACKED ? (int64_t)Q * (Q + 1) / 2 : (int64_t)Q * Q);
    if (precision == RASCAL_PS_BF16) return set_error(RASCAL_E_UNSUPPORTED, "BF16 power spectrum not built yet");
    const size_t smem = sizeof(float) * ctx->n_lm * Qp;
    k_power_spectrum_fp32<<<(unsigned)n_centres, kPsThreads, smem, ctx->stream>>>(d_coeffs, Q, Qp, ctx->n_lm, ctx->l_max,
                                                                                ctx->ps_norm, ctx->d_pstasks, ctx->n_pstasks,
                                                                                layout, stride, d_ps);
    RASCAL_LAUNCH_CHECK("k_power_spectrum_fp32");
    return RASCAL_OK;
}
