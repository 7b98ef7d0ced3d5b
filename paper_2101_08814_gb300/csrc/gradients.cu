// Additive linear energy (Eq. additive-energy-model) and the analytic backward pass (Appendix B).
//
// For E = sum_i G_i . p_i (PACKED p), the pair gradient is
//   dE/dr_ji = sum_{n l m} chat^i_{a_j n l m} grad_r [ f_cut(r) I^o_nl(r) Y_lm(r^) ],
//   chat^i_l = k_l (W_l + W_l^T) C^i_l,   k_l = (2l+1)^-1/2,
// where W_l is G_i's l-block in packed upper-triangular form (zeros below the diagonal). The weights are
// contracted with the coefficients first (the adjoint chat, per centre) and only then with the per-pair feature
// gradients, the order of Eq. gpr-force-order; dc/dr is never stored: each pair's radial values, their
// r-derivatives, Y_lm and its Cartesian gradient are recomputed.
//
// With u = r/|r|, s = sum_lm Y_lm sum_n chat_{n lm} (f I_nl)' and w = sum_lm (sum_n chat_{n lm} f I_nl) dY_lm/du
// (the gradient of the polynomial extension of Y in the unit-vector components),
//   dE/dr_ji = s u + (w - (w.u) u)/|r|.
// Forces: F_j -= dE/dr_ji, F_i += dE/dr_ji (skipped when j is an image of i: the two cancel, Appendix B);
// virial V[a][b] += dE/dr_ji[a] r_ji[b] (images of i included).
#include <vector>

#include "common.cuh"
#include "ps_fp32.cuh"
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

struct GradArgs {
    const int64_t* offsets;
    const int* nbr_j;
    const float4* rij;
    const int* species;
    const int* lut;
    const int* offs;        // structure offsets
    const float4* table;
    const float* pre_G;  // per-pair radial values and r-derivatives (EXACT / MLP modes) or NULL
    const float* pre_D;
    const int* fmap;
    const float* coeffs;
    const float* grad_ps;   // [N][Fp] or NULL
    const float* weights;   // [S][Fp] or NULL
    double* forces;
    double* virial;
    unsigned* flags;
    int N, n_s, n_max, l_max, S, Q, n_lm, F, F_pad, n_pad, Lp, M, chunk, ps_norm;
    int64_t Fp;
    float inv_delta, r_cut, width;
    int lp[kMaxLMax + 2];
};

__device__ inline void cutoff_and_slope(float r, float r_cut, float w, float& f, float& df) {
    if (r <= r_cut - w) {
        f = 1.0f;
        df = 0.0f;
    } else if (r >= r_cut) {
        f = 0.0f;
        df = 0.0f;
    } else {
        const float t = (r - r_cut + w) / w;
        f = 0.5f * (1.0f + cospif(t));
        df = -0.5f * 3.14159265358979f / w * sinpif(t);
    }
}

constexpr int kGradThreads = 256;

__global__ void __launch_bounds__(kGradThreads) k_gradients(const GradArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int chunk = A.chunk;
    const size_t qn4 = ((size_t)A.Q * A.n_lm + 3) / 4 * 4;  // keeps the float4 arrays 16-byte aligned
    float* s_C = reinterpret_cast<float*>(smem_raw);         // [Q][n_lm]
    float* s_H = s_C + qn4;                                   // chat [Q][n_lm]
    float4* s_vec = reinterpret_cast<float4*>(s_H + qn4);
    float* s_G = reinterpret_cast<float*>(s_vec + chunk);    // [chunk][F_pad]   f I
    float* s_D = s_G + (size_t)chunk * A.F_pad;               // [chunk][F_pad]   (f I)'
    float* s_Y = s_D + (size_t)chunk * A.F_pad;               // [chunk][4][Lp]   Y, dY/dux, dY/duy, dY/duz
    float* s_acc = s_Y + (size_t)chunk * 4 * A.Lp;            // [chunk][4]       s, wx, wy, wz
    float* s_fc = s_acc + (size_t)chunk * 4;
    float* s_dfc = s_fc + chunk;
    int* s_spc = reinterpret_cast<int*>(s_dfc + chunk);
    int* s_j = s_spc + chunk;
    int* s_lp = s_j + chunk;
    int* s_fmap = s_lp + (kMaxLMax + 2);
    __shared__ double red[kGradThreads / 32][12];

    const int i = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int L1 = A.l_max + 1;
    if (tid < kMaxLMax + 2) s_lp[tid] = A.lp[tid];
    for (int t = tid; t < A.F_pad; t += blockDim.x) s_fmap[t] = A.fmap[t];
    const int lab_i = A.species[i];
    const int a_i = (lab_i >= 0 && lab_i < 256) ? A.lut[lab_i] : -1;
    const float* Gp = A.grad_ps ? A.grad_ps + (int64_t)i * A.Fp : (a_i >= 0 ? A.weights + (int64_t)a_i * A.Fp : nullptr);
    const float* c = A.coeffs + (int64_t)i * A.Q * A.n_lm;
    for (int e = tid; e < A.Q * A.n_lm; e += blockDim.x) s_C[e] = c[e];
    __syncthreads();
    // adjoint chat[q][lm] = k_l sum_q' (W + W^T)[q][q'] C[q'][lm]
    const int Qpk = A.Q * (A.Q + 1) / 2;
    for (int e = tid; e < A.Q * A.n_lm; e += blockDim.x) {
        const int q = e / A.n_lm, lm = e - q * A.n_lm;
        int l = 0;
        while ((l + 1) * (l + 1) <= lm) ++l;
        float acc = 0.0f;
        if (Gp) {
            const float* W = Gp + (int64_t)l * Qpk;
            for (int q2 = 0; q2 < A.Q; ++q2) {
                const int lo = min(q, q2), hi = max(q, q2);
                float wv = __ldg(&W[packed_index(lo, hi, A.Q)]);
                if (q == q2) wv *= 2.0f;
                acc = fmaf(wv, s_C[q2 * A.n_lm + lm], acc);
            }
        }
        s_H[e] = (A.ps_norm ? rsqrtf((float)(2 * l + 1)) : 1.0f) * acc;
    }
    double fi[3] = {0.0, 0.0, 0.0};
    double vir[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const int64_t seg_beg = A.offsets[i], seg_end = A.offsets[i + 1];
    for (int64_t pos = seg_beg; pos < seg_end; pos += chunk) {
        const int nc = (int)((seg_end - pos) < (int64_t)chunk ? (seg_end - pos) : (int64_t)chunk);
        __syncthreads();
        for (int t = tid; t < nc; t += blockDim.x) {
            const float4 v = A.rij[pos + t];
            const int j = A.nbr_j[pos + t];
            const int lab = A.species[j];
            int a = (lab >= 0 && lab < 256) ? A.lut[lab] : -1;
            if (!(v.w > 1e-6f)) a = -1;
            s_vec[t] = v;
            s_spc[t] = a;
            s_j[t] = j;
            float f, df;
            cutoff_and_slope(v.w, A.r_cut, A.width, f, df);
            s_fc[t] = f;
            s_dfc[t] = df;
            s_acc[4 * t] = s_acc[4 * t + 1] = s_acc[4 * t + 2] = s_acc[4 * t + 3] = 0.0f;
        }
        __syncthreads();
        // radial values and slopes: one warp per pair
        for (int p = warp; p < nc; p += nwarps) {
            const float r = s_vec[p].w, f = s_fc[p], df = s_dfc[p];
            const float x = r * A.inv_delta;
            int k = (int)x;
            k = min(max(k, 0), A.M - 1);
            const float u = x - (float)k;
            const float4* trow = A.table + (int64_t)k * A.F;
            for (int fp = lane; fp < A.F_pad; fp += 32) {
                const int col = s_fmap[fp];
                float g = 0.0f, dg = 0.0f;
                if (col >= 0) {
                    if (A.pre_G) {
                        g = __ldg(&A.pre_G[(pos + p) * A.F + col]);
                        dg = __ldg(&A.pre_D[(pos + p) * A.F + col]);
                    } else {
                        const float4 cf = __ldg(&trow[col]);
                        g = fmaf(u, fmaf(u, fmaf(u, cf.w, cf.z), cf.y), cf.x);
                        dg = fmaf(u, fmaf(u, 3.0f * cf.w, 2.0f * cf.z), cf.y) * A.inv_delta;
                    }
                }
                s_G[(size_t)p * A.F_pad + fp] = f * g;
                s_D[(size_t)p * A.F_pad + fp] = df * g + f * dg;
            }
        }
        // Y and dY/du: one thread per (pair, m) chain, forward-mode through the recurrence
        for (int idx = tid; idx < nc * L1; idx += blockDim.x) {
            const int p = idx / L1, m = idx - p * L1;
            const float4 v = s_vec[p];
            const float inv_r = v.w > 1e-6f ? 1.0f / v.w : 0.0f;
            const float x = v.x * inv_r, y = v.y * inv_r, z = v.z * inv_r;
            float cm = 1.0f, sm = 0.0f, cm1 = 0.0f, sm1 = 0.0f;  // (x+iy)^m and (x+iy)^(m-1)
            for (int t = 0; t < m; ++t) {
                cm1 = cm;
                sm1 = sm;
                const float nc2 = cm * x - sm * y;
                sm = cm * y + sm * x;
                cm = nc2;
            }
            float* Y = s_Y + (size_t)p * 4 * A.Lp;
            float* Yx = Y + A.Lp;
            float* Yy = Yx + A.Lp;
            float* Yz = Yy + A.Lp;
            float q2 = 0.0f, q1 = c_ylm_K[m], d2 = 0.0f, d1 = 0.0f;
            const float fm = (float)m;
            for (int l = m; l <= A.l_max; ++l) {
                float q, dq;
                if (l == m) {
                    q = q1;
                    dq = 0.0f;
                } else {
                    const float Al = c_ylm_A[l * 16 + m], Bl = c_ylm_B[l * 16 + m];
                    q = Al * (z * q1 - Bl * q2);
                    dq = Al * (q1 + z * d1 - Bl * d2);
                    q2 = q1;
                    d2 = d1;
                    q1 = q;
                    d1 = dq;
                }
                if (m == 0) {
                    const int s0 = s_lp[l] + l;
                    Y[s0] = q;
                    Yx[s0] = 0.0f;
                    Yy[s0] = 0.0f;
                    Yz[s0] = dq;
                } else {
                    const int sp = s_lp[l] + l + m, sn = s_lp[l] + l - m;
                    Y[sp] = q * cm;
                    Yx[sp] = q * fm * cm1;
                    Yy[sp] = -q * fm * sm1;
                    Yz[sp] = dq * cm;
                    Y[sn] = q * sm;
                    Yx[sn] = q * fm * sm1;
                    Yy[sn] = q * fm * cm1;
                    Yz[sn] = dq * sm;
                }
            }
        }
        __syncthreads();
        // contraction with chat: one thread per (pair, l)
        for (int idx = tid; idx < nc * L1; idx += blockDim.x) {
            const int p = idx / L1, l = idx - p * L1;
            const int a = s_spc[p];
            if (a < 0) continue;
            const float* H = s_H + (size_t)a * A.n_max * A.n_lm;
            const float* G = s_G + (size_t)p * A.F_pad + l * A.n_pad;
            const float* D = s_D + (size_t)p * A.F_pad + l * A.n_pad;
            const float* Y = s_Y + (size_t)p * 4 * A.Lp + s_lp[l];
            float S = 0.0f, Wx = 0.0f, Wy = 0.0f, Wz = 0.0f;
            for (int s = 0; s <= 2 * l; ++s) {
                const int lm = l * l + s;
                float uu = 0.0f, vv = 0.0f;
                for (int n = 0; n < A.n_max; ++n) {
                    const float h = H[n * A.n_lm + lm];
                    uu = fmaf(h, D[n], uu);
                    vv = fmaf(h, G[n], vv);
                }
                S = fmaf(uu, Y[s], S);
                Wx = fmaf(vv, Y[A.Lp + s], Wx);
                Wy = fmaf(vv, Y[2 * A.Lp + s], Wy);
                Wz = fmaf(vv, Y[3 * A.Lp + s], Wz);
            }
            atomicAdd(&s_acc[4 * p + 0], S);
            atomicAdd(&s_acc[4 * p + 1], Wx);
            atomicAdd(&s_acc[4 * p + 2], Wy);
            atomicAdd(&s_acc[4 * p + 3], Wz);
        }
        __syncthreads();
        // per pair: dE/dr_ji, force scatter, virial
        for (int p = tid; p < nc; p += blockDim.x) {
            if (s_spc[p] < 0) continue;
            const float4 v = s_vec[p];
            const float inv_r = 1.0f / v.w;
            const float ux = v.x * inv_r, uy = v.y * inv_r, uz = v.z * inv_r;
            const float S = s_acc[4 * p], Wx = s_acc[4 * p + 1], Wy = s_acc[4 * p + 2], Wz = s_acc[4 * p + 3];
            const float wu = Wx * ux + Wy * uy + Wz * uz;
            const float g[3] = {S * ux + (Wx - wu * ux) * inv_r, S * uy + (Wy - wu * uy) * inv_r,
                                S * uz + (Wz - wu * uz) * inv_r};
            const float rv[3] = {v.x, v.y, v.z};
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) vir[3 * a + b] += (double)g[a] * (double)rv[b];
            const int j = s_j[p];
            if (j != i) {
                for (int a = 0; a < 3; ++a) {
                    atomicAdd(&A.forces[3 * (int64_t)j + a], -(double)g[a]);
                    fi[a] += (double)g[a];
                }
            }
        }
    }
    // block reduction of F_i and the virial
    double vals[12] = {fi[0], fi[1], fi[2], vir[0], vir[1], vir[2], vir[3], vir[4], vir[5], vir[6], vir[7], vir[8]};
#pragma unroll
    for (int k = 0; k < 12; ++k)
        for (int o = 16; o > 0; o >>= 1) vals[k] += __shfl_xor_sync(0xffffffffu, vals[k], o);
    if (lane == 0)
        for (int k = 0; k < 12; ++k) red[warp][k] = vals[k];
    __syncthreads();
    if (tid < 12) {
        double s = 0.0;
        for (int w = 0; w < nwarps; ++w) s += red[w][tid];
        if (tid < 3) {
            if (s != 0.0) atomicAdd(&A.forces[3 * (int64_t)i + tid], s);
        } else {
            int lo = 0, hi = A.n_s;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (A.offs[mid] <= i) lo = mid;
                else hi = mid;
            }
            atomicAdd(&A.virial[9 * (int64_t)lo + (tid - 3)], s);
        }
    }
}

static size_t grad_smem(const rascal_ctx* ctx, int chunk) {
    const ExpPlan& P = ctx->plan;
    return sizeof(float) * 2 * (((size_t)ctx->Q * ctx->n_lm + 3) / 4 * 4) + sizeof(float4) * chunk + sizeof(float) * chunk * (2 * P.F_pad + 4 * P.Lp + 4 + 2) +
           sizeof(int) * (2 * chunk + kMaxLMax + 2 + P.F_pad) + 64;
}

int gradients_setup(rascal_ctx* ctx) {
    RASCAL_CUDA(upload_ylm_constants(ctx->stream));
    RASCAL_CUDA(cudaFuncSetAttribute(k_gradients, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
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
    if (!ctx) return set_error(RASCAL_E_ARG, "NULL context");
    int st = validate_system(ctx, sys);
    if (st) return st;
    if (!d_forces || !d_virial) return set_error(RASCAL_E_ARG, "NULL forces or virial");
    if ((d_grad_ps == nullptr) == (d_weights == nullptr))
        return set_error(RASCAL_E_ARG, "exactly one of grad_ps and weights must be given");
    RASCAL_CUDA(cudaMemsetAsync(d_forces, 0, sizeof(double) * 3 * sys->n_atoms, ctx->stream));
    RASCAL_CUDA(cudaMemsetAsync(d_virial, 0, sizeof(double) * 9 * sys->n_structures, ctx->stream));
    if (sys->n_atoms == 0) return RASCAL_OK;
    if (!d_offsets || !d_nbr_j || !d_rij || !d_coeffs) return set_error(RASCAL_E_ARG, "NULL device pointer");
    const ExpPlan& P = ctx->plan;
    GradArgs A;
    A.offsets = d_offsets;
    A.nbr_j = d_nbr_j;
    A.rij = reinterpret_cast<const float4*>(d_rij);
    A.species = sys->d_species;
    A.lut = ctx->d_lut;
    A.offs = sys->d_struct_offsets;
    A.table = ctx->d_table;
    A.fmap = ctx->d_fmap;
    A.coeffs = d_coeffs;
    A.grad_ps = d_grad_ps;
    A.weights = d_weights;
    A.forces = d_forces;
    A.virial = d_virial;
    A.flags = ctx->d_flags;
    A.N = sys->n_atoms;
    A.n_s = sys->n_structures;
    A.n_max = ctx->n_max;
    A.l_max = ctx->l_max;
    A.S = ctx->n_species;
    A.Q = ctx->Q;
    A.n_lm = ctx->n_lm;
    A.F = ctx->F;
    A.F_pad = P.F_pad;
    A.n_pad = P.n_pad;
    A.Lp = P.Lp;
    A.M = ctx->M;
    A.ps_norm = ctx->ps_norm;
    A.Fp = (int64_t)(ctx->l_max + 1) * ctx->Q * (ctx->Q + 1) / 2;
    A.inv_delta = ctx->inv_delta;
    A.r_cut = (float)ctx->r_cut;
    A.width = (float)ctx->smooth_width;
    for (int l = 0; l < kMaxLMax + 2; ++l) A.lp[l] = P.lp[l];
    int chunk = 32;
    while (chunk > 8 && grad_smem(ctx, chunk) > 200 * 1024) chunk /= 2;
    A.chunk = chunk;
    const size_t smem = grad_smem(ctx, chunk);
    if (smem > 220 * 1024) return set_error(RASCAL_E_UNSUPPORTED, "hypers too large for the gradient kernel");
    if ((st = radial_precompute(ctx, sys, d_offsets, d_rij, true, &A.pre_G, &A.pre_D))) return st;
    k_gradients<<<sys->n_atoms, kGradThreads, smem, ctx->stream>>>(A);
    RASCAL_LAUNCH_CHECK("k_gradients");
    return RASCAL_OK;
}
