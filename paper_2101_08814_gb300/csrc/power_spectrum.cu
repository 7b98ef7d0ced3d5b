// Power spectrum (Eq. nu2-basis-coupled) from stored coefficients. FP32: one CTA per centre, the centre's block
// c[q][lm] is read once (coalesced), transposed into shared memory as CT[lm][q] and contracted per l by the FP32
// register-tiled Gram of ps_fp32.cuh. BF16 and TF32x3: the tensor-core Gram of the fused kernel (expansion.cu) run
// on the given coefficients.
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

// ---------------------------------------------------------------------------------------------------------
// Tensor-core Gram (tcgen05, cta_group::1, M = 128): for each l, D_l = C_l C_l^T with C_l = c[q][l, m] as a
// (rows q) x (K = 2l+1, zero-padded) operand in shared memory used as both A and B (K-major, no swizzle). Only
// rows q < Q of each operand are stored; the M = 128 / N = round16(Q) reads past them touch the next tile or the
// slack at the end of the region and only produce accumulator rows/columns >= Q, which are never read.
//   BF16 mode:  one kind::f16 MMA per 16-wide K step, inputs rounded to bfloat16, FP32 accumulation.
//   FP32 mode:  kind::tf32 with a hi/lo split of every input (hi = top 19 bits, lo = remainder), three MMAs per
//               8-wide K step (hi hi^T + hi lo^T + lo hi^T): the dropped lo lo^T term is below 2^-22 relative.
// Persistent CTAs of 4 warps; TMEM holds the accumulators of a group of l values (<= 256 columns); after the MMAs
// of a group complete (mbarrier), each warp reads its 32 rows with tcgen05.ld, scales by (2l+1)^-1/2, stages the
// packed (or full) block in shared memory and the CTA writes it to global memory with coalesced stores.
// ---------------------------------------------------------------------------------------------------------
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
    if (precision < RASCAL_PS_FP32 || precision > RASCAL_PS_TF32X3) return set_error(RASCAL_E_ARG, "unknown precision");
    if (n_centres == 0) return RASCAL_OK;
    if (!d_coeffs || !d_ps) return set_error(RASCAL_E_ARG, "NULL device pointer");
    if (n_centres > 0x7fffffffLL) return set_error(RASCAL_E_UNSUPPORTED, "more than 2^31-1 centres in one call");
    const int Q = ctx->Q, Qp = (Q + 3) / 4 * 4;
    const int64_t stride = (int64_t)(ctx->l_max + 1) * (layout == RASCAL_LAYOUT_PACKED ? (int64_t)Q * (Q + 1) / 2 : (int64_t)Q * Q);
    if (precision != RASCAL_PS_FP32) return power_spectrum_tc(ctx, n_centres, d_coeffs, precision, layout, d_ps);
    const size_t smem = sizeof(float) * ctx->n_lm * Qp;
    k_power_spectrum_fp32<<<(unsigned)n_centres, kPsThreads, smem, ctx->stream>>>(d_coeffs, Q, Qp, ctx->n_lm, ctx->l_max,
                                                                                ctx->ps_norm, ctx->d_pstasks, ctx->n_pstasks,
                                                                                layout, stride, d_ps);
    RASCAL_LAUNCH_CHECK("k_power_spectrum_fp32");
    return RASCAL_OK;
}
