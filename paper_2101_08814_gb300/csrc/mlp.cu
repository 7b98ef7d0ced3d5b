// Learned radial surrogate: a 1 -> H -> H -> F multilayer perceptron with SiLU activations that maps a pair
// distance to the F = n_max (l_max+1) o-GTO radial integrals I^o_nl(r) (Eq. rad-int-gto-1 after S^-1/2). The paper
// has no such network; its nearest hook is the closing remark of Sec. 'Spline optimization' that the radial basis
// invites numerical optimisation. Conventions (shared with the oracle's mlp.py):
//   t = r / r_cut;  z1 = W1 t + b1;  h1 = silu(z1);  z2 = W2 h1 + b2;  h2 = silu(z2);  y = W3 h2 + b3;
//   I^o_f(r) ~ scale_f y_f, with scale_f = max over r of |I^o_f| so every output is O(1);
//   loss L = mean over batch and outputs of (y - target/scale)^2.
// Parameters are one FP32 vector [W1 (H) | b1 (H) | W2 (H x H, row = output) | b2 (H) | W3 (F x H) | b3 (F)].
//
// Training (FP32, CUDA cores): k_mlp_forward keeps the pre-activations, k_mlp_backward_hidden back-propagates
// through the two hidden layers per sample, k_mlp_wgrad reduces the weight gradients over the batch and k_mlp_adam
// applies one bias-corrected Adam step. Targets are the exact FP64 integrals (rascal_mlp_targets).
//
// Inference (k_mlp_infer): tiles of 128 distances on the tcgen05 tensor cores with BF16 weights and activations and
// FP32 accumulators in TMEM: layer 1 (rank one) on the CUDA cores, layers 2 and 3 as M = 128 MMAs against the
// weights held in shared memory, SiLU epilogues between them, and the input tangent (d/dr) carried as a second
// set of MMAs when derivatives are requested.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "radial_fp64.cuh"
#include "tcgen05.cuh"

namespace rascal {

__device__ inline float sigmoidf_(float z) { return 1.0f / (1.0f + __expf(-z)); }
__device__ inline float silu_(float z) { return z * sigmoidf_(z); }
__device__ inline float silu_grad_(float z) {
    const float s = sigmoidf_(z);
    return s * (1.0f + z * (1.0f - s));
}

struct MlpLayout {
    int H, F;
    int oW1, ob1, oW2, ob2, oW3, ob3, n;
};

static MlpLayout mlp_layout(int H, int F) {
    MlpLayout L;
    L.H = H;
    L.F = F;
    L.oW1 = 0;
    L.ob1 = H;
    L.oW2 = 2 * H;
    L.ob2 = 2 * H + H * H;
    L.oW3 = 3 * H + H * H;
    L.ob3 = 3 * H + H * H + F * H;
    L.n = 3 * H + H * H + F * H + F;
    return L;
}

// ------------------------------------------------------------------------------------------------ training
// one CTA of H threads per sample: activations to global (z1, z2 [B][H], h1, h2 [B][H]), output residual to dy
__global__ void k_mlp_forward(int B, int H, int F, const float* __restrict__ P, MlpLayout L, const float* __restrict__ t,
                              const float* __restrict__ target, float* __restrict__ z1, float* __restrict__ z2,
                              float* __restrict__ h1g, float* __restrict__ h2g, float* __restrict__ dy,
                              float* __restrict__ loss) {
    extern __shared__ float sh[];
    float* h1 = sh;      // [H]
    float* h2 = sh + H;  // [H]
    __shared__ float red[32];
    const int b = blockIdx.x, k = threadIdx.x;
    const float tb = t[b];
    const float a1 = fmaf(P[L.oW1 + k], tb, P[L.ob1 + k]);
    z1[(int64_t)b * H + k] = a1;
    h1[k] = silu_(a1);
    h1g[(int64_t)b * H + k] = h1[k];
    __syncthreads();
    float a2 = P[L.ob2 + k];
    const float* w2 = P + L.oW2 + (int64_t)k * H;
    for (int j = 0; j < H; ++j) a2 = fmaf(w2[j], h1[j], a2);
    z2[(int64_t)b * H + k] = a2;
    h2[k] = silu_(a2);
    h2g[(int64_t)b * H + k] = h2[k];
    __syncthreads();
    float part = 0.0f;
    const float inv = 2.0f / ((float)B * (float)F);
    for (int f = k; f < F; f += blockDim.x) {
        float y = P[L.ob3 + f];
        const float* w3 = P + L.oW3 + (int64_t)f * H;
        for (int j = 0; j < H; ++j) y = fmaf(w3[j], h2[j], y);
        const float d = y - target[(int64_t)b * F + f];
        dy[(int64_t)b * F + f] = inv * d;
        part += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((k & 31) == 0) red[k >> 5] = part;
    __syncthreads();
    if (k == 0) {
        float s = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(loss, s / ((float)B * (float)F));
    }
}

// per sample: dz2 = (dy W3) * silu'(z2), dz1 = (dz2 W2) * silu'(z1)
__global__ void k_mlp_backward_hidden(int B, int H, int F, const float* __restrict__ P, MlpLayout L,
                                      const float* __restrict__ z1, const float* __restrict__ z2, const float* __restrict__ dy,
                                      float* __restrict__ dz1, float* __restrict__ dz2) {
    extern __shared__ float sh[];
    float* s_dy = sh;       // [F]
    float* s_dz2 = sh + F;  // [H]
    const int b = blockIdx.x, k = threadIdx.x;
    for (int f = k; f < F; f += blockDim.x) s_dy[f] = dy[(int64_t)b * F + f];
    __syncthreads();
    float g = 0.0f;
    for (int f = 0; f < F; ++f) g = fmaf(s_dy[f], P[L.oW3 + (int64_t)f * H + k], g);
    const float d2 = g * silu_grad_(z2[(int64_t)b * H + k]);
    dz2[(int64_t)b * H + k] = d2;
    s_dz2[k] = d2;
    __syncthreads();
    float g1 = 0.0f;
    for (int h = 0; h < H; ++h) g1 = fmaf(s_dz2[h], P[L.oW2 + (int64_t)h * H + k], g1);
    dz1[(int64_t)b * H + k] = g1 * silu_grad_(z1[(int64_t)b * H + k]);
}

// one thread per parameter: sum over the batch of the outer products (FP32, batch-ordered, deterministic)
__global__ void k_mlp_wgrad(int B, int H, int F, MlpLayout L, const float* __restrict__ t, const float* __restrict__ h1,
                            const float* __restrict__ h2, const float* __restrict__ dy, const float* __restrict__ dz1,
                            const float* __restrict__ dz2, float* __restrict__ G) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= L.n) return;
    float acc = 0.0f;
    if (idx < L.ob1) {  // W1[k]
        const int k = idx;
        for (int b = 0; b < B; ++b) acc = fmaf(dz1[(int64_t)b * H + k], t[b], acc);
    } else if (idx < L.oW2) {  // b1[k]
        const int k = idx - L.ob1;
        for (int b = 0; b < B; ++b) acc += dz1[(int64_t)b * H + k];
    } else if (idx < L.ob2) {  // W2[h][k]
        const int h = (idx - L.oW2) / H, k = (idx - L.oW2) % H;
        for (int b = 0; b < B; ++b) acc = fmaf(dz2[(int64_t)b * H + h], h1[(int64_t)b * H + k], acc);
    } else if (idx < L.oW3) {  // b2[h]
        const int h = idx - L.ob2;
        for (int b = 0; b < B; ++b) acc += dz2[(int64_t)b * H + h];
    } else if (idx < L.ob3) {  // W3[f][k]
        const int f = (idx - L.oW3) / H, k = (idx - L.oW3) % H;
        for (int b = 0; b < B; ++b) acc = fmaf(dy[(int64_t)b * F + f], h2[(int64_t)b * H + k], acc);
    } else {  // b3[f]
        const int f = idx - L.ob3;
        for (int b = 0; b < B; ++b) acc += dy[(int64_t)b * F + f];
    }
    G[idx] = acc;
}

__global__ void k_mlp_adam(int n, float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m,
                           float* __restrict__ v, float lr, float beta1, float beta2, float eps, float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = G[i];
    const float mi = beta1 * m[i] + (1.0f - beta1) * g;
    const float vi = beta2 * v[i] + (1.0f - beta2) * g * g;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// minibatch gather through a host-drawn permutation of the sample indices
__global__ void k_mlp_gather(int B, int F, const int64_t* __restrict__ order, const float* __restrict__ t_all,
                             const float* __restrict__ y_all, float* __restrict__ tb, float* __restrict__ yb) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx < B) tb[idx] = t_all[order[idx]];
    if (idx < (int64_t)B * F) {
        const int64_t b = idx / F, f = idx % F;
        yb[idx] = y_all[order[b] * F + f];
    }
}

// forward, backward through the hidden layers and weight gradients of one minibatch into ctx->mlp_grad
static int mlp_step_kernels(rascal_ctx* ctx, const MlpLayout& L, int B, const float* t, const float* tgt, float* z1,
                            float* z2, float* h1, float* h2, float* dy, float* dz1, float* dz2, float* loss) {
    const int H = L.H, F = L.F;
    k_mlp_forward<<<B, H, sizeof(float) * 2 * H, ctx->stream>>>(B, H, F, ctx->mlp_params, L, t, tgt, z1, z2, h1, h2, dy, loss);
    RASCAL_LAUNCH_CHECK("k_mlp_forward");
    k_mlp_backward_hidden<<<B, H, sizeof(float) * (F + H), ctx->stream>>>(B, H, F, ctx->mlp_params, L, z1, z2, dy, dz1, dz2);
    RASCAL_LAUNCH_CHECK("k_mlp_backward_hidden");
    k_mlp_wgrad<<<div_up(L.n, 128), 128, 0, ctx->stream>>>(B, H, F, L, t, h1, h2, dy, dz1, dz2, ctx->mlp_grad);
    RASCAL_LAUNCH_CHECK("k_mlp_wgrad");
    return RASCAL_OK;
}

// ------------------------------------------------------------------------------------------------ targets
// FP64 targets at arbitrary r from a dense FP64 clamped spline of the exact integrals (see rascal_mlp_targets)
__global__ void k_spline64_eval(int64_t n, const double* __restrict__ r, int M, double delta, int F,
                                const double* __restrict__ y, const double* __restrict__ y2, int n_max, int L1,
                                const double* __restrict__ inv_scale, float* __restrict__ out) {
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= n * F) return;
    const int64_t p = id / F;
    const int f = (int)(id % F);  // f = l n_max + n
    const int l = f / n_max, nn = f % n_max;
    const double rr = r[p];
    int k = (int)floor(rr / delta);
    k = k < 0 ? 0 : (k > M - 1 ? M - 1 : k);
    const double A = ((k + 1) * delta - rr) / delta, B = 1.0 - A;
    const double yk = y[((int64_t)k * n_max + nn) * L1 + l], yk1 = y[((int64_t)(k + 1) * n_max + nn) * L1 + l];
    const double s0 = y2[(int64_t)f * (M + 1) + k], s1 = y2[(int64_t)f * (M + 1) + k + 1];
    const double v = A * yk + B * yk1 + ((A * A * A - A) * s0 + (B * B * B - B) * s1) * delta * delta / 6.0;
    out[p * F + f] = (float)(v * inv_scale[f]);
}

// ------------------------------------------------------------------------------------------------ inference
struct MlpInferArgs {
    const float4* rij;      // pair vectors (w = r), or NULL when r is given
    const float* r_in;      // distances, or NULL
    int64_t n;
    float* out;             // [n][F] radial values scale_f y_f (f = l n_max + n)
    float* dout;            // [n][F] d/dr, or NULL
    const float* P;         // FP32 parameters (layer 1 and biases are read from here)
    const __nv_bfloat16* W2t;  // W2 as a K-major operand tile (N = H rows, K = H)
    const __nv_bfloat16* W3t;  // W3 as a K-major operand tile (N = F_pad rows, K = H)
    const float* scale;     // [F]
    MlpLayout L;
    int F_pad;              // F rounded up to 16
    float inv_rscale;       // 1 / r_cut
    unsigned* flags;
};

constexpr int kMlpH = 64;
constexpr int kMlpTile = 128;
// TMEM: values in columns 0..255, forward tangents (d/dr) in 256..511; without tangents two CTAs share an SM


// offset of element (row, k) in a K-major no-swizzle bf16 tile with K = 64 (8 chunks of 16 bytes per 8-row group)
__device__ __host__ inline int kmajor64_off(int row, int k) {
    return (row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__global__ void __launch_bounds__(128, 2) k_mlp_infer(const MlpInferArgs A) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t s_bar;
    __shared__ uint32_t s_tmem;
    const int H = kMlpH, F = A.L.F;
    unsigned char* w2 = smem;                              // 64 x 64 bf16 = 8 KB
    unsigned char* w3 = w2 + 8192;                         // F_pad x 64 bf16
    unsigned char* a1 = w3 + (size_t)A.F_pad * 128;        // 128 x 64 bf16 (h1), 16 KB
    const bool deriv = A.dout != nullptr;
    const uint32_t tm_cols = deriv ? 512u : 256u;
    unsigned char* a1d = a1 + 16384;                       // tangent of h1 (only with derivatives)
    unsigned char* a2 = a1d + (deriv ? 16384 : 0);         // h2
    unsigned char* a2d = a2 + 16384;                       // tangent of h2 (only with derivatives)
    float* s_par = reinterpret_cast<float*>(a2d + (deriv ? 16384 : 0));  // W1, b1, b2 [H each], b3, scale [F each]
    // per-warp 32 x 16 output slabs (value and derivative, pitch 17): rows leave with coalesced stores
    float* s_slab = s_par + ((3 * H + 2 * F + 3) & ~3) + (threadIdx.x >> 5) * 2 * 32 * 17;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // weights into shared memory (already laid out as operand tiles on the host side)
    for (int b = tid; b < 8192 / 16; b += blockDim.x) reinterpret_cast<uint4*>(w2)[b] = reinterpret_cast<const uint4*>(A.W2t)[b];
    for (int b = tid; b < A.F_pad * 128 / 16; b += blockDim.x)
        reinterpret_cast<uint4*>(w3)[b] = reinterpret_cast<const uint4*>(A.W3t)[b];
    for (int k = tid; k < H; k += blockDim.x) {
        s_par[k] = A.P[A.L.oW1 + k];
        s_par[H + k] = A.P[A.L.ob1 + k];
        s_par[2 * H + k] = A.P[A.L.ob2 + k];
    }
    for (int f = tid; f < F; f += blockDim.x) {
        s_par[3 * H + f] = A.P[A.L.ob3 + f];
        s_par[3 * H + F + f] = A.scale[f];
    }
    if (warp == 0) {
        tmem_alloc(&s_tmem, tm_cols);
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
    const uint32_t id2 = instr_desc(1u, 128u, (uint32_t)H);
    const uint32_t id3 = instr_desc(1u, 128u, (uint32_t)A.F_pad);
    const uint32_t s_w2 = smem_u32(w2), s_w3 = smem_u32(w3), s_a1 = smem_u32(a1), s_a1d = smem_u32(a1d),
                   s_a2 = smem_u32(a2), s_a2d = smem_u32(a2d);
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    uint32_t phase = 0;
    bool ok = true;
    const int64_t n_tiles = (A.n + kMlpTile - 1) / kMlpTile;
    for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        const int64_t p = tile * kMlpTile + tid;
        const bool valid = p < A.n;
        float r = 0.0f;
        if (valid) r = A.rij ? A.rij[p].w : A.r_in[p];
        const float tt = r * A.inv_rscale;
        // layer 1 on the CUDA cores: row = this thread's distance
        for (int k = 0; k < H; ++k) {
            const float z = fmaf(s_par[k], tt, s_par[H + k]);
            *reinterpret_cast<__nv_bfloat16*>(a1 + kmajor64_off(tid, k)) = __float2bfloat16_rn(silu_(z));
            if (deriv)
                *reinterpret_cast<__nv_bfloat16*>(a1d + kmajor64_off(tid, k)) =
                    __float2bfloat16_rn(silu_grad_(z) * s_par[k] * A.inv_rscale);
        }
        fence_proxy_async_smem();
        __syncthreads();
        // layer 2: D2 = h1 W2^T (TMEM cols 0..63), tangent in cols 256..319
        if (tid == 0) {
            tc_fence_after();
            for (int kk = 0; kk < H / 16; ++kk) {
                const uint64_t db = smem_desc(s_w2 + kk * 256, 128, 1024);
                mma_bf16_ss(taddr, smem_desc(s_a1 + kk * 256, 128, 1024), db, id2, kk > 0);
                if (deriv) mma_bf16_ss(taddr + 256, smem_desc(s_a1d + kk * 256, 128, 1024), db, id2, kk > 0);
            }
            mma_commit(&s_bar);
        }
        bool done = mbar_wait_bounded(&s_bar, phase);
        ok = __syncthreads_and(done) != 0;
        phase ^= 1u;
        if (!ok) break;
        tc_fence_after();
        for (int c0 = 0; c0 < H; c0 += 16) {
            float z[16], dz[16];
            tmem_ld16(taddr + lane_base + (uint32_t)c0, z);
            if (deriv) tmem_ld16(taddr + lane_base + 256u + (uint32_t)c0, dz);
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int k = c0 + u;
                const float zz = z[u] + s_par[2 * H + k];
                *reinterpret_cast<__nv_bfloat16*>(a2 + kmajor64_off(tid, k)) = __float2bfloat16_rn(silu_(zz));
                if (deriv)
                    *reinterpret_cast<__nv_bfloat16*>(a2d + kmajor64_off(tid, k)) = __float2bfloat16_rn(silu_grad_(zz) * dz[u]);
            }
        }
        tc_fence_before();
        fence_proxy_async_smem();
        __syncthreads();
        // layer 3: D3 = h2 W3^T (cols 0..F_pad-1), tangent at 256..
        if (tid == 0) {
            tc_fence_after();
            for (int kk = 0; kk < H / 16; ++kk) {
                const uint64_t db = smem_desc(s_w3 + kk * 256, 128, 1024);
                mma_bf16_ss(taddr, smem_desc(s_a2 + kk * 256, 128, 1024), db, id3, kk > 0);
                if (deriv) mma_bf16_ss(taddr + 256, smem_desc(s_a2d + kk * 256, 128, 1024), db, id3, kk > 0);
            }
            mma_commit(&s_bar);
        }
        done = mbar_wait_bounded(&s_bar, phase);
        ok = __syncthreads_and(done) != 0;
        phase ^= 1u;
        if (!ok) break;
        tc_fence_after();
        const int64_t row0 = tile * kMlpTile + 32 * warp;  // this warp's 32 rows (pairs)
        for (int c0 = 0; c0 < A.F_pad; c0 += 16) {
            float y[16], dy[16];
            tmem_ld16(taddr + lane_base + (uint32_t)c0, y);
            if (deriv) tmem_ld16(taddr + lane_base + 256u + (uint32_t)c0, dy);
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int f = min(c0 + u, F - 1);
                const float sc = s_par[3 * H + F + f];
                s_slab[lane * 17 + u] = sc * (y[u] + s_par[3 * H + f]);
                if (deriv) s_slab[32 * 17 + lane * 17 + u] = sc * dy[u];
            }
            __syncwarp();
            // two rows per store instruction: lanes 0..15 row 2k, lanes 16..31 row 2k+1, 16 consecutive columns
            const int cc = lane & 15, f = c0 + cc;
#pragma unroll 4
            for (int k = 0; k < 16; ++k) {
                const int rr = 2 * k + (lane >> 4);
                const int64_t pr = row0 + rr;
                if (pr < A.n && f < F) {
                    A.out[pr * F + f] = s_slab[rr * 17 + cc];
                    if (deriv) A.dout[pr * F + f] = s_slab[32 * 17 + rr * 17 + cc];
                }
            }
            __syncwarp();
        }
        tc_fence_before();
        __syncthreads();
    }
    if (!ok && tid == 0) atomicOr(A.flags, kFlagTimeout);
    if (!ok) mbar_wait_bounded(&s_bar, phase);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(taddr, tm_cols);
    }
    (void)lane;
}

}  // namespace rascal

using namespace rascal;

// ---------------------------------------------------------------------------------------------------------- API
namespace rascal {

static int mlp_check(rascal_ctx* ctx) {
    if (!ctx) return set_error(RASCAL_E_ARG, "NULL context");
    if (!ctx->mlp_params) return set_error(RASCAL_E_ARG, "no MLP in this context: call rascal_mlp_set_params first");
    return RASCAL_OK;
}

// bf16 operand tiles of W2 (H x H) and W3 (F_pad x H) from the FP32 parameters
__global__ void k_mlp_pack(int H, int F, int F_pad, const float* __restrict__ P, MlpLayout L, __nv_bfloat16* W2t,
                           __nv_bfloat16* W3t) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < H * H) {
        const int row = idx / H, k = idx % H;
        W2t[kmajor64_off(row, k) / 2] = __float2bfloat16_rn(P[L.oW2 + idx]);
    }
    if (idx < F_pad * H) {
        const int row = idx / H, k = idx % H;
        const float v = row < F ? P[L.oW3 + (int64_t)row * H + k] : 0.0f;
        W3t[kmajor64_off(row, k) / 2] = __float2bfloat16_rn(v);
    }
}

int mlp_pack(rascal_ctx* ctx) {
    const MlpLayout L = mlp_layout(ctx->mlp_hidden, ctx->F);
    const int F_pad = (ctx->F + 15) / 16 * 16;
    const int n = std::max(ctx->mlp_hidden * ctx->mlp_hidden, F_pad * ctx->mlp_hidden);
    k_mlp_pack<<<div_up(n, 256), 256, 0, ctx->stream>>>(ctx->mlp_hidden, ctx->F, F_pad, ctx->mlp_params, L,
                                                       reinterpret_cast<__nv_bfloat16*>(ctx->mlp_w2t),
                                                       reinterpret_cast<__nv_bfloat16*>(ctx->mlp_w3t));
    RASCAL_LAUNCH_CHECK("k_mlp_pack");
    return RASCAL_OK;
}

int mlp_infer(rascal_ctx* ctx, int64_t n, const float4* rij, const float* r, float* out, float* dout) {
    if (n == 0) return RASCAL_OK;
    const int F_pad = (ctx->F + 15) / 16 * 16;
    if (F_pad > 256) return set_error(RASCAL_E_UNSUPPORTED, "MLP inference needs n_max*(l_max+1) <= 256");
    MlpInferArgs A;
    A.rij = rij;
    A.r_in = r;
    A.n = n;
    A.out = out;
    A.dout = dout;
    A.P = ctx->mlp_params;
    A.W2t = reinterpret_cast<const __nv_bfloat16*>(ctx->mlp_w2t);
    A.W3t = reinterpret_cast<const __nv_bfloat16*>(ctx->mlp_w3t);
    A.scale = ctx->mlp_scale;
    A.L = mlp_layout(ctx->mlp_hidden, ctx->F);
    A.F_pad = F_pad;
    A.inv_rscale = (float)(1.0 / ctx->r_cut);
    A.flags = ctx->d_flags;
    const size_t smem = 8192 + (size_t)F_pad * 128 + (dout ? 4 : 2) * 16384 +
                        sizeof(float) * ((3 * kMlpH + 2 * ctx->F + 3) / 4 * 4 + 4 * 2 * 32 * 17) + 64;
    const int64_t tiles = (n + kMlpTile - 1) / kMlpTile;
    // one CTA per SM with tangents (all 512 TMEM columns), two without
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, (int64_t)ctx->n_sm * (dout ? 1 : 2));
    k_mlp_infer<<<grid, 128, smem, ctx->stream>>>(A);
    RASCAL_LAUNCH_CHECK("k_mlp_infer");
    return RASCAL_OK;
}

int mlp_setup(rascal_ctx* ctx) {
    RASCAL_CUDA(cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    return RASCAL_OK;
}

}  // namespace rascal

extern "C" int rascal_mlp_num_params(const rascal_ctx* ctx, int hidden) {
    if (!ctx || hidden != kMlpH) return -1;
    return mlp_layout(hidden, ctx->F).n;
}

extern "C" int rascal_mlp_set_params(rascal_ctx* ctx, int hidden, const float* h_params, const float* h_scale) {
    clear_error();
    if (!ctx || !h_params || !h_scale) return set_error(RASCAL_E_ARG, "NULL argument");
    if (hidden != kMlpH) return set_error(RASCAL_E_UNSUPPORTED, "the MLP kernels use %d hidden units", kMlpH);
    const MlpLayout L = mlp_layout(hidden, ctx->F);
    const int F_pad = (ctx->F + 15) / 16 * 16;
    if (!ctx->mlp_params) {
        RASCAL_CUDA(cudaMalloc(&ctx->mlp_params, sizeof(float) * L.n));
        RASCAL_CUDA(cudaMalloc(&ctx->mlp_m, sizeof(float) * L.n));
        RASCAL_CUDA(cudaMalloc(&ctx->mlp_v, sizeof(float) * L.n));
        RASCAL_CUDA(cudaMalloc(&ctx->mlp_grad, sizeof(float) * L.n));
        RASCAL_CUDA(cudaMalloc(&ctx->mlp_scale, sizeof(float) * ctx->F));
        RASCAL_CUDA(cudaMalloc(&ctx->mlp_w2t, sizeof(__nv_bfloat16) * hidden * hidden));
        RASCAL_CUDA(cudaMalloc(&ctx->mlp_w3t, sizeof(__nv_bfloat16) * F_pad * hidden));
    }
    ctx->mlp_hidden = hidden;
    ctx->mlp_step = 0;
    RASCAL_CUDA(cudaMemcpyAsync(ctx->mlp_params, h_params, sizeof(float) * L.n, cudaMemcpyHostToDevice, ctx->stream));
    RASCAL_CUDA(cudaMemcpyAsync(ctx->mlp_scale, h_scale, sizeof(float) * ctx->F, cudaMemcpyHostToDevice, ctx->stream));
    RASCAL_CUDA(cudaMemsetAsync(ctx->mlp_m, 0, sizeof(float) * L.n, ctx->stream));
    RASCAL_CUDA(cudaMemsetAsync(ctx->mlp_v, 0, sizeof(float) * L.n, ctx->stream));
    int st = mlp_pack(ctx);
    if (st) return st;
    RASCAL_CUDA(cudaStreamSynchronize(ctx->stream));
    return RASCAL_OK;
}

extern "C" int rascal_mlp_get_params(rascal_ctx* ctx, float* h_params, float* h_scale) {
    clear_error();
    int st = mlp_check(ctx);
    if (st) return st;
    const MlpLayout L = mlp_layout(ctx->mlp_hidden, ctx->F);
    if (h_params) RASCAL_CUDA(cudaMemcpyAsync(h_params, ctx->mlp_params, sizeof(float) * L.n, cudaMemcpyDeviceToHost, ctx->stream));
    if (h_scale) RASCAL_CUDA(cudaMemcpyAsync(h_scale, ctx->mlp_scale, sizeof(float) * ctx->F, cudaMemcpyDeviceToHost, ctx->stream));
    RASCAL_CUDA(cudaStreamSynchronize(ctx->stream));
    return RASCAL_OK;
}

extern "C" int rascal_mlp_targets(rascal_ctx* ctx, int64_t n, const double* d_r, int dense_intervals, float* d_targets,
                                  float* h_scale_out) {
    clear_error();
    if (!ctx || n < 0 || (n > 0 && (!d_r || !d_targets))) return set_error(RASCAL_E_ARG, "bad argument");
    const int M = dense_intervals > 0 ? dense_intervals : 8192;
    const int n_max = ctx->n_max, L1 = ctx->l_max + 1, F = ctx->F;
    const double delta = ctx->r_cut / M;
    const size_t bytes = carve_bytes((M + 1) * 8, 2 * 8, (size_t)(M + 1) * F * 8, (size_t)2 * F * 8, (size_t)2 * F * 8,
                                     (size_t)F * (M + 1) * 8, (size_t)F * (M + 1) * 8, (size_t)F * 8, (size_t)F * 8);
    void* base;
    int st = arena_get(ctx->scratch, bytes, &base);
    if (st) return st;
    Carver cv(base);
    double* grid = cv.take<double>(M + 1);
    double* ends = cv.take<double>(2);
    double* y = cv.take<double>((size_t)(M + 1) * F);
    double* yend = cv.take<double>((size_t)2 * F);
    double* dyend = cv.take<double>((size_t)2 * F);
    double* cp = cv.take<double>((size_t)F * (M + 1));
    double* y2 = cv.take<double>((size_t)F * (M + 1));
    double* inv_scale = cv.take<double>(F);
    (void)cv.take<double>(F);
    // exact FP64 integrals on the dense grid, clamped spline through them (error ~ 1e-14 at 8192 intervals)
    if ((st = radial_grid_fp64(ctx, M, grid, ends, y, yend, dyend, cp, y2))) return st;
    // per-output scale = max |I| on the grid
    std::vector<double> hy((size_t)(M + 1) * F);
    RASCAL_CUDA(cudaMemcpyAsync(hy.data(), y, sizeof(double) * hy.size(), cudaMemcpyDeviceToHost, ctx->stream));
    RASCAL_CUDA(cudaStreamSynchronize(ctx->stream));
    std::vector<double> inv(F), sc(F);
    for (int f = 0; f < F; ++f) {
        const int l = f / n_max, nn = f % n_max;
        double m = 0.0;
        for (int k = 0; k <= M; ++k) m = std::max(m, std::fabs(hy[((size_t)k * n_max + nn) * L1 + l]));
        sc[f] = m > 0.0 ? m : 1.0;
        inv[f] = 1.0 / sc[f];
        if (h_scale_out) h_scale_out[f] = (float)sc[f];
    }
    RASCAL_CUDA(cudaMemcpyAsync(inv_scale, inv.data(), sizeof(double) * F, cudaMemcpyHostToDevice, ctx->stream));
    if (n > 0) {
        k_spline64_eval<<<(unsigned)div_up(n * F, 256), 256, 0, ctx->stream>>>(n, d_r, M, delta, F, y, y2, n_max, L1,
                                                                             inv_scale, d_targets);
        RASCAL_LAUNCH_CHECK("k_spline64_eval");
    }
    RASCAL_CUDA(cudaStreamSynchronize(ctx->stream));
    return RASCAL_OK;
}

extern "C" int rascal_mlp_train(rascal_ctx* ctx, int64_t n_samples, const float* d_t, const float* d_targets,
                                const int64_t* d_order, int batch, int steps, float lr_max, float lr_min, int total_steps,
                                float* d_loss) {
    clear_error();
    int st = mlp_check(ctx);
    if (st) return st;
    if (batch <= 0 || steps < 0 || n_samples < batch || !d_t || !d_targets || !d_order)
        return set_error(RASCAL_E_ARG, "bad training arguments");
    const int H = ctx->mlp_hidden, F = ctx->F;
    const MlpLayout L = mlp_layout(H, F);
    const size_t bytes = carve_bytes(sizeof(float) * batch, sizeof(float) * (size_t)batch * F, sizeof(float) * (size_t)batch * H * 6,
                                     sizeof(float) * (size_t)batch * F, sizeof(float) * 4);
    void* base;
    if ((st = arena_get(ctx->scratch, bytes, &base))) return st;
    Carver cv(base);
    float* tb = cv.take<float>(batch);
    float* tgt = cv.take<float>((size_t)batch * F);
    float* act = cv.take<float>((size_t)batch * H * 6);
    float* dy = cv.take<float>((size_t)batch * F);
    float* loss_sink = cv.take<float>(4);
    float *z1 = act, *z2 = act + (size_t)batch * H, *h1 = z2 + (size_t)batch * H, *h2 = h1 + (size_t)batch * H,
          *dz1 = h2 + (size_t)batch * H, *dz2 = dz1 + (size_t)batch * H;
    const double b1 = 0.9, b2 = 0.999;
    for (int s = 0; s < steps; ++s) {
        const int64_t start = ((int64_t)ctx->mlp_step * batch) % (n_samples - batch + 1);
        k_mlp_gather<<<div_up((int64_t)batch * (F + 1), 256), 256, 0, ctx->stream>>>(batch, F, d_order + start, d_t, d_targets,
                                                                                     tb, tgt);
        RASCAL_LAUNCH_CHECK("k_mlp_gather");
        float* loss = d_loss ? d_loss + s : loss_sink;
        RASCAL_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), ctx->stream));
        if ((st = mlp_step_kernels(ctx, L, batch, tb, tgt, z1, z2, h1, h2, dy, dz1, dz2, loss))) return st;
        ++ctx->mlp_step;
        const int T = total_steps > 0 ? total_steps : steps;
        const double prog = std::min(1.0, (double)(ctx->mlp_step - 1) / std::max(1, T - 1));
        const float lr = (float)(lr_min + 0.5 * (lr_max - lr_min) * (1.0 + std::cos(3.14159265358979 * prog)));
        const float bc1 = (float)(1.0 - std::pow(b1, ctx->mlp_step)), bc2 = (float)(1.0 - std::pow(b2, ctx->mlp_step));
        k_mlp_adam<<<div_up(L.n, 256), 256, 0, ctx->stream>>>(L.n, ctx->mlp_params, ctx->mlp_grad, ctx->mlp_m, ctx->mlp_v, lr,
                                                              (float)b1, (float)b2, 1e-8f, bc1, bc2);
        RASCAL_LAUNCH_CHECK("k_mlp_adam");
    }
    return mlp_pack(ctx);
}

extern "C" int rascal_mlp_gradients(rascal_ctx* ctx, int batch, const float* d_t, const float* d_targets, float* d_grad,
                                    float* d_loss) {
    clear_error();
    int st = mlp_check(ctx);
    if (st) return st;
    if (batch <= 0 || !d_t || !d_targets || !d_grad || !d_loss) return set_error(RASCAL_E_ARG, "bad argument");
    const int H = ctx->mlp_hidden, F = ctx->F;
    const MlpLayout L = mlp_layout(H, F);
    const size_t bytes = carve_bytes(sizeof(float) * (size_t)batch * H * 6, sizeof(float) * (size_t)batch * F);
    void* base;
    if ((st = arena_get(ctx->scratch, bytes, &base))) return st;
    Carver cv(base);
    float* act = cv.take<float>((size_t)batch * H * 6);
    float* dy = cv.take<float>((size_t)batch * F);
    float *z1 = act, *z2 = act + (size_t)batch * H, *h1 = z2 + (size_t)batch * H, *h2 = h1 + (size_t)batch * H,
          *dz1 = h2 + (size_t)batch * H, *dz2 = dz1 + (size_t)batch * H;
    RASCAL_CUDA(cudaMemsetAsync(d_loss, 0, sizeof(float), ctx->stream));
    if ((st = mlp_step_kernels(ctx, L, batch, d_t, d_targets, z1, z2, h1, h2, dy, dz1, dz2, d_loss))) return st;
    RASCAL_CUDA(cudaMemcpyAsync(d_grad, ctx->mlp_grad, sizeof(float) * L.n, cudaMemcpyDeviceToDevice, ctx->stream));
    return RASCAL_OK;
}

extern "C" int rascal_mlp_eval(rascal_ctx* ctx, int64_t n, const float* d_r, float* d_out, float* d_dout) {
    clear_error();
    int st = mlp_check(ctx);
    if (st) return st;
    if (n < 0 || (n > 0 && (!d_r || !d_out))) return set_error(RASCAL_E_ARG, "bad argument");
    return mlp_infer(ctx, n, nullptr, d_r, d_out, d_dout);
}

extern "C" int rascal_mlp_save(rascal_ctx* ctx, const char* path) {
    clear_error();
    int st = mlp_check(ctx);
    if (st) return st;
    if (!path) return set_error(RASCAL_E_ARG, "NULL path");
    const MlpLayout L = mlp_layout(ctx->mlp_hidden, ctx->F);
    std::vector<float> p(L.n), m(L.n), v(L.n), s(ctx->F);
    RASCAL_CUDA(cudaMemcpyAsync(p.data(), ctx->mlp_params, sizeof(float) * L.n, cudaMemcpyDeviceToHost, ctx->stream));
    RASCAL_CUDA(cudaMemcpyAsync(m.data(), ctx->mlp_m, sizeof(float) * L.n, cudaMemcpyDeviceToHost, ctx->stream));
    RASCAL_CUDA(cudaMemcpyAsync(v.data(), ctx->mlp_v, sizeof(float) * L.n, cudaMemcpyDeviceToHost, ctx->stream));
    RASCAL_CUDA(cudaMemcpyAsync(s.data(), ctx->mlp_scale, sizeof(float) * ctx->F, cudaMemcpyDeviceToHost, ctx->stream));
    RASCAL_CUDA(cudaStreamSynchronize(ctx->stream));
    FILE* fh = std::fopen(path, "wb");
    if (!fh) return set_error(RASCAL_E_ARG, "cannot open %s for writing", path);
    const int32_t hdr[8] = {0x52534d4c /* 'RSML' */, 1, ctx->mlp_hidden, ctx->F, ctx->n_max, ctx->l_max, L.n, ctx->mlp_step};
    const double hyp[2] = {ctx->r_cut, ctx->sigma};
    bool okw = std::fwrite(hdr, sizeof(hdr), 1, fh) == 1 && std::fwrite(hyp, sizeof(hyp), 1, fh) == 1 &&
               std::fwrite(p.data(), sizeof(float), L.n, fh) == (size_t)L.n && std::fwrite(m.data(), sizeof(float), L.n, fh) == (size_t)L.n &&
               std::fwrite(v.data(), sizeof(float), L.n, fh) == (size_t)L.n && std::fwrite(s.data(), sizeof(float), ctx->F, fh) == (size_t)ctx->F;
    std::fclose(fh);
    if (!okw) return set_error(RASCAL_E_ARG, "short write to %s", path);
    return RASCAL_OK;
}

extern "C" int rascal_mlp_load(rascal_ctx* ctx, const char* path) {
    clear_error();
    if (!ctx || !path) return set_error(RASCAL_E_ARG, "NULL argument");
    FILE* fh = std::fopen(path, "rb");
    if (!fh) return set_error(RASCAL_E_ARG, "cannot open %s", path);
    int32_t hdr[8];
    double hyp[2];
    bool okr = std::fread(hdr, sizeof(hdr), 1, fh) == 1 && std::fread(hyp, sizeof(hyp), 1, fh) == 1;
    if (!okr || hdr[0] != 0x52534d4c || hdr[1] != 1 || hdr[3] != ctx->F || hdr[4] != ctx->n_max || hdr[5] != ctx->l_max ||
        hyp[0] != ctx->r_cut || hyp[1] != ctx->sigma) {
        std::fclose(fh);
        return set_error(RASCAL_E_ARG, "%s holds an MLP for other hypers or is not an MLP checkpoint", path);
    }
    const MlpLayout L = mlp_layout(hdr[2], ctx->F);
    if (L.n != hdr[6]) {
        std::fclose(fh);
        return set_error(RASCAL_E_ARG, "%s: parameter count mismatch", path);
    }
    std::vector<float> p(L.n), m(L.n), v(L.n), s(ctx->F);
    okr = std::fread(p.data(), sizeof(float), L.n, fh) == (size_t)L.n && std::fread(m.data(), sizeof(float), L.n, fh) == (size_t)L.n &&
          std::fread(v.data(), sizeof(float), L.n, fh) == (size_t)L.n && std::fread(s.data(), sizeof(float), ctx->F, fh) == (size_t)ctx->F;
    std::fclose(fh);
    if (!okr) return set_error(RASCAL_E_ARG, "%s is truncated", path);
    int st = rascal_mlp_set_params(ctx, hdr[2], p.data(), s.data());
    if (st) return st;
    RASCAL_CUDA(cudaMemcpyAsync(ctx->mlp_m, m.data(), sizeof(float) * L.n, cudaMemcpyHostToDevice, ctx->stream));
    RASCAL_CUDA(cudaMemcpyAsync(ctx->mlp_v, v.data(), sizeof(float) * L.n, cudaMemcpyHostToDevice, ctx->stream));
    RASCAL_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->mlp_step = hdr[7];
    return RASCAL_OK;
}
