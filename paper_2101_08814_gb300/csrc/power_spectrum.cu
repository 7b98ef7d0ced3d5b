// Power spectrum (Eq. nu2-basis-coupled) from stored coefficients: one CTA per centre, the centre's block
// c[q][lm] is read once (coalesced), transposed into shared memory as CT[lm][q] and contracted per l by the FP32
// register-tiled Gram of ps_fp32.cuh.
#include <algorithm>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"
#include "ps_fp32.cuh"
#include "tcgen05.cuh"

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
struct PsTcArgs {
    const float* coeffs;
    float* ps;
    unsigned* flags;
    int64_t n_centres, ps_stride;
    int Q, n_lm, l_max, ps_norm, layout, N, groups;
    int tile_off[kMaxLMax + 1];  // byte offsets of the per-l operand tiles (hi); lo tiles at + lo_off
    int sbo[kMaxLMax + 1];       // bytes between 8-row groups of tile l
    int nk[kMaxLMax + 1];        // MMA K steps of tile l
    int gl[kMaxLMax + 2];        // l ranges of the TMEM groups
    int lo_off, tiles_bytes, stage_floats;
};

constexpr uint32_t kPsTmemCols = 256;

template <bool TF32>
__global__ void __launch_bounds__(128) k_power_spectrum_tc(const PsTcArgs A) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint64_t s_bar;
    __shared__ uint32_t s_tmem;
    unsigned char* tiles = smem_raw;
    float* stage = reinterpret_cast<float*>(smem_raw + A.tiles_bytes);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int esz = TF32 ? 4 : 2;
    constexpr int e16 = 16 / esz;  // elements per 16-byte core-matrix row
    for (int b = tid; b < A.tiles_bytes / 16; b += blockDim.x) reinterpret_cast<uint4*>(tiles)[b] = make_uint4(0, 0, 0, 0);
    if (warp == 0) {
        tmem_alloc(&s_tmem, kPsTmemCols);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&s_bar, 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = s_tmem;
    const uint32_t tiles_s = smem_u32(tiles);
    const uint32_t idesc = instr_desc(TF32 ? 2u : 1u, 128u, (uint32_t)A.N);
    const int Qpk = A.Q * (A.Q + 1) / 2;
    const int per_l = A.layout == RASCAL_LAYOUT_PACKED ? Qpk : A.Q * A.Q;
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t i = blockIdx.x; i < A.n_centres && ok; i += gridDim.x) {
        const float* c = A.coeffs + i * (int64_t)A.Q * A.n_lm;
        for (int e = tid; e < A.Q * A.n_lm; e += blockDim.x) {
            const int q = e / A.n_lm, lm = e - q * A.n_lm;
            int l = (int)sqrtf((float)lm + 0.5f);
            if (l * l > lm) --l;
            if ((l + 1) * (l + 1) <= lm) ++l;
            const int s = lm - l * l;
            const int off = A.tile_off[l] + (q >> 3) * A.sbo[l] + (s / e16) * 128 + (q & 7) * 16 + (s % e16) * esz;
            const float v = __ldg(&c[e]);
            if (TF32) {
                const float hi = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
                *reinterpret_cast<float*>(tiles + off) = hi;
                *reinterpret_cast<float*>(tiles + A.lo_off + off) = v - hi;
            } else {
                *reinterpret_cast<__nv_bfloat16*>(tiles + off) = __float2bfloat16_rn(v);
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        for (int g = 0; g < A.groups && ok; ++g) {
            const int l0 = A.gl[g], l1 = A.gl[g + 1];
            if (tid == 0) {
                tc_fence_after();
                for (int l = l0; l < l1; ++l) {
                    const uint32_t d = taddr + (uint32_t)((l - l0) * A.N);
                    for (int kk = 0; kk < A.nk[l]; ++kk) {
                        const uint32_t a_addr = tiles_s + A.tile_off[l] + kk * 256;
                        const uint64_t da = smem_desc(a_addr, 128, A.sbo[l]);
                        if (TF32) {
                            const uint64_t dl = smem_desc(a_addr + A.lo_off, 128, A.sbo[l]);
                            mma_tf32_ss(d, da, da, idesc, kk > 0);
                            mma_tf32_ss(d, da, dl, idesc, 1);
                            mma_tf32_ss(d, dl, da, idesc, 1);
                        } else {
                            mma_bf16_ss(d, da, da, idesc, kk > 0);
                        }
                    }
                }
                mma_commit(&s_bar);
            }
            const bool done = mbar_wait_bounded(&s_bar, phase);
            ok = __syncthreads_and(done) != 0;  // uniform across the CTA: tcgen05.ld below is warp-collective
            if (!ok) {
                if (tid == 0) atomicOr(A.flags, kFlagTimeout);
                mbar_wait_bounded(&s_bar, phase);  // give in-flight MMAs a second bounded chance before TMEM is freed
            }
            phase ^= 1u;
            tc_fence_after();
            const int q = 32 * warp + lane;
            for (int l = l0; l < l1 && ok; ++l) {
                const float kl = A.ps_norm ? rsqrtf((float)(2 * l + 1)) : 1.0f;
                float* st = stage + (size_t)(l - l0) * per_l;
                for (int j = 0; j < A.N / 16; ++j) {
                    float v[16];
                    tmem_ld16(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)((l - l0) * A.N + 16 * j), v);
                    if (q < A.Q) {
#pragma unroll
                        for (int t = 0; t < 16; ++t) {
                            const int q2 = 16 * j + t;
                            if (q2 < A.Q) {
                                if (A.layout == RASCAL_LAYOUT_PACKED) {
                                    if (q2 >= q) st[packed_index(q, q2, A.Q)] = kl * v[t];
                                } else {
                                    st[q * A.Q + q2] = kl * v[t];
                                }
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            __syncthreads();
            if (ok) {
                float* dst = A.ps + i * A.ps_stride + (int64_t)l0 * per_l;
                const int count = (l1 - l0) * per_l;
                for (int t = tid; t < count; t += blockDim.x) dst[t] = stage[t];
            }
            __syncthreads();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(taddr, kPsTmemCols);
    }
}

static int make_tc_args(rascal_ctx* ctx, bool tf32, int layout, PsTcArgs& A, size_t& smem) {
    const int Q = ctx->Q;
    if (Q > 128) return set_error(RASCAL_E_UNSUPPORTED, "tensor-core power spectrum needs n_species*n_max <= 128");
    const int esz = tf32 ? 4 : 2, kstep = tf32 ? 8 : 16, e16 = 16 / esz;
    A.Q = Q;
    A.n_lm = ctx->n_lm;
    A.l_max = ctx->l_max;
    A.ps_norm = ctx->ps_norm;
    A.layout = layout;
    A.N = (Q + 15) / 16 * 16;
    const int Qr = (Q + 7) / 8 * 8;
    int off = 0, need = 0;
    for (int l = 0; l <= ctx->l_max; ++l) {
        const int kpad = (2 * l + 1 + kstep - 1) / kstep * kstep;
        A.nk[l] = kpad / kstep;
        A.sbo[l] = (kpad / e16) * 128;
        A.tile_off[l] = off;
        need = std::max(need, off + 16 * A.sbo[l]);  // M = 128 rows read from this tile's start
        off += (Qr / 8) * A.sbo[l];
    }
    int hi_bytes = (std::max(off, need) + 1023) / 1024 * 1024;
    A.lo_off = tf32 ? hi_bytes : 0;
    A.tiles_bytes = tf32 ? 2 * hi_bytes : hi_bytes;
    const int Qpk = Q * (Q + 1) / 2;
    const int per_l = layout == RASCAL_LAYOUT_PACKED ? Qpk : Q * Q;
    const int max_stage_floats = 96 * 1024 / 4;
    const int per_group_cols = (int)kPsTmemCols / A.N;
    int g = 0;
    A.gl[0] = 0;
    for (int l = 0; l <= ctx->l_max;) {
        int n = 0;
        while (l + n <= ctx->l_max && n < per_group_cols && (n + 1) * per_l <= max_stage_floats) ++n;
        if (n == 0) return set_error(RASCAL_E_UNSUPPORTED, "power-spectrum block too large for the staging buffer");
        l += n;
        A.gl[++g] = l;
    }
    A.groups = g;
    int stage = 0;
    for (int k = 0; k < g; ++k) stage = std::max(stage, (A.gl[k + 1] - A.gl[k]) * per_l);
    A.stage_floats = stage;
    smem = (size_t)A.tiles_bytes + sizeof(float) * stage;
    if (smem > 200 * 1024) return set_error(RASCAL_E_UNSUPPORTED, "tensor-core power spectrum needs %zu bytes of shared memory", smem);
    return RASCAL_OK;
}

static int launch_ps_tc(rascal_ctx* ctx, int64_t n_centres, const float* d_coeffs, bool tf32, int layout, float* d_ps,
                        int64_t stride) {
    PsTcArgs A;
    size_t smem;
    int st = make_tc_args(ctx, tf32, layout, A, smem);
    if (st) return st;
    A.coeffs = d_coeffs;
    A.ps = d_ps;
    A.flags = ctx->d_flags;
    A.n_centres = n_centres;
    A.ps_stride = stride;
    int per_sm = 1;
    if (tf32) {
        RASCAL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_power_spectrum_tc<true>, 128, smem));
    } else {
        RASCAL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_power_spectrum_tc<false>, 128, smem));
    }
    per_sm = std::max(1, std::min(per_sm, (int)(512 / kPsTmemCols)));  // TMEM: 512 columns per SM
    const int64_t grid = std::min<int64_t>(n_centres, (int64_t)ctx->n_sm * per_sm);
    if (tf32) {
        k_power_spectrum_tc<true><<<(unsigned)grid, 128, smem, ctx->stream>>>(A);
    } else {
        k_power_spectrum_tc<false><<<(unsigned)grid, 128, smem, ctx->stream>>>(A);
    }
    RASCAL_LAUNCH_CHECK("k_power_spectrum_tc");
    return RASCAL_OK;
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
    RASCAL_CUDA(cudaFuncSetAttribute(k_power_spectrum_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    RASCAL_CUDA(cudaFuncSetAttribute(k_power_spectrum_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
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
    if (precision != RASCAL_PS_FP32) return launch_ps_tc(ctx, n_centres, d_coeffs, precision == RASCAL_PS_TF32X3, layout, d_ps, stride);
    const size_t smem = sizeof(float) * ctx->n_lm * Qp;
    k_power_spectrum_fp32<<<(unsigned)n_centres, kPsThreads, smem, ctx->stream>>>(d_coeffs, Q, Qp, ctx->n_lm, ctx->l_max,
                                                                                ctx->ps_norm, ctx->d_pstasks, ctx->n_pstasks,
                                                                                layout, stride, d_ps);
    RASCAL_LAUNCH_CHECK("k_power_spectrum_fp32");
    return RASCAL_OK;
}
