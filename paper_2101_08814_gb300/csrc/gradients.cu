// Additive linear energy (Eq. additive-energy-model) and, in a later pass, its gradients.
#include "common.cuh"
#include "ylm_fp32.cuh"

namespace rascal {

// E_s = sum_{i in s} w_{a_i} . p_i, one CTA per centre, FP64 block reduction and one atomic per centre.
__global__ void k_linear_energy(int N, int n_s, const int* __restrict__ offs, const int* __restrict__ species,
                                const int* __restrict__ lut, const float* __restrict__ ps, const float* __restrict__ w,
                                int64_t F, double* __restrict__ energy) {
    __shared__ double red[32];
    const int i = blockIdx.x;
    const int lab = species[i];
    const int a = (lab >= 0 && lab < 256) ? lut[lab] : -1;
    double acc = 0.0;
    if (a >= 0) {
        const float* p = ps + (int64_t)i * F;
        const float* wa = w + (int64_t)a * F;
        for (int64_t f = threadIdx.x; f < F; f += blockDim.x) acc += (double)p[f] * (double)wa[f];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) {
            int lo = 0, hi = n_s;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (offs[mid] <= i) lo = mid;
                else hi = mid;
            }
            atomicAdd(&energy[lo], v);
        }
    }
}

int gradients_setup(rascal_ctx* ctx) {
    RASCAL_CUDA(upload_ylm_constants(ctx->stream));
    return RASCAL_OK;
}

}  // namespace rascal

using namespace rascal;

extern "C" int rascal_linear_energy(rascal_ctx* ctx, const rascal_system* sys, const float* d_ps_packed,
                                    const float* d_weights, double* d_energy) {
    clear_error();
    if (!ctx) return set_error(RASCAL_E_ARG, "NULL context");
    int st = validate_system(ctx, sys);
    if (st) return st;
    if (!d_energy) return set_error(RASCAL_E_ARG, "NULL energy");
    RASCAL_CUDA(cudaMemsetAsync(d_energy, 0, sizeof(double) * sys->n_structures, ctx->stream));
    if (sys->n_atoms == 0) return RASCAL_OK;
    if (!d_ps_packed || !d_weights) return set_error(RASCAL_E_ARG, "NULL device pointer");
    const int64_t F = (int64_t)(ctx->l_max + 1) * ctx->Q * (ctx->Q + 1) / 2;
    k_linear_energy<<<sys->n_atoms, 256, 0, ctx->stream>>>(sys->n_atoms, sys->n_structures, sys->d_struct_offsets,
                                                          sys->d_species, ctx->d_lut, d_ps_packed, d_weights, F, d_energy);
    RASCAL_LAUNCH_CHECK("k_linear_energy");
    return RASCAL_OK;
}

extern "C" int rascal_gradients(rascal_ctx* ctx, const rascal_system* sys, const int64_t* d_offsets, const int* d_nbr_j,
                                const float* d_rij, const float* d_coeffs, const float* d_grad_ps, const float* d_weights,
                                double* d_forces, double* d_virial) {
    clear_error();
    (void)ctx; (void)sys; (void)d_offsets; (void)d_nbr_j; (void)d_rij; (void)d_coeffs; (void)d_grad_ps; (void)d_weights;
    (void)d_forces; (void)d_virial;
    return set_error(RASCAL_E_UNSUPPORTED, "gradients not built yet");
}

extern "C" int rascal_soap(rascal_ctx* ctx, const rascal_system* sys, const int64_t* d_offsets, const int* d_nbr_j,
                           const float* d_rij, int layout, float* d_coeffs, float* d_ps) {
    int st = rascal_spherical_expansion(ctx, sys, d_offsets, d_nbr_j, d_rij, d_coeffs);
    if (st) return st;
    return rascal_power_spectrum(ctx, sys->n_atoms, d_coeffs, RASCAL_PS_FP32, layout, d_ps);
}
