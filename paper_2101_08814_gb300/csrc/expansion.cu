// Fused pair kernel for the density coefficients (Eq. spherical_expansion_coefficients_gaussians):
//   c^i_{a n l m} = sum_{j in A_i, a_j = a} f_cut(r_ji) I^o_nl(r_ji) Y_lm(r^_ji)
//
// One CTA per centre i. The centre's CSR segment of pairs is processed in chunks staged in shared memory:
//   1. stage r_ji (float4 x, y, z, r), the neighbour's species and f_cut(r) for the chunk;
//   2. list the chunk's pairs by species (warp ballots, so the order is deterministic);
//   3. per listed pair: Y_lm by the Cartesian recurrence (one thread per (pair, m) chain) and the radial values
//      G_nl = f_cut(r) I^o_nl(r) from the FP32 cubic spline table (one warp per pair, lanes over (l, n));
//   4. accumulate: each thread owns a 4(n) x 4(m) register tile of one l and one species and adds the outer
//      product G_{l, n-tile} x Y_{l, m-tile} for every pair of its species (16 FMAs per two float4 loads).
// The segment reduction happens in registers; no atomics, no intermediate written to global memory.
// Output stores go to the centre's contiguous block [n_species][n_max][(l_max+1)^2].
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "ylm_fp32.cuh"

namespace rascal {

struct ExpArgs {
    const int64_t* offsets;
    const int* nbr_j;
    const float4* rij;
    const int* species;
    const int* lut;
    const float4* table;
    const int* tasks;
    const int* fmap;
    float* coeffs;
    unsigned* flags;
    int N, n_max, l_max, S, n_lm, F, F_pad, n_pad, Lp, M, T_s, W_s, S_c, rounds, chunk, include_center;
    float inv_delta, r_cut, width;
    int lp[kMaxLMax + 2];
};

__device__ inline float cutoff_fp32(float r, float r_cut, float w) {
    if (r <= r_cut - w) return 1.0f;
    if (r >= r_cut) return 0.0f;
    return 0.5f * (1.0f + cospif((r - r_cut + w) / w));
}

__device__ inline float spline_eval(const float4* __restrict__ table, int F, int M, float inv_delta, float r, int col) {
    const float x = r * inv_delta;
    int k = (int)x;
    k = min(max(k, 0), M - 1);
    const float u = x - (float)k;
    const float4 c = __ldg(&table[(int64_t)k * F + col]);
    return fmaf(u, fmaf(u, fmaf(u, c.w, c.z), c.y), c.x);
}

__global__ void __launch_bounds__(1024) k_expansion(const ExpArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int chunk = A.chunk;
    float4* s_vec = reinterpret_cast<float4*>(smem_raw);
    float* s_G = reinterpret_cast<float*>(s_vec + chunk);            // [chunk][F_pad]
    float* s_Y = s_G + (size_t)chunk * A.F_pad;                       // [chunk][Lp]
    float* s_fc = s_Y + (size_t)chunk * A.Lp;
    int* s_spc = reinterpret_cast<int*>(s_fc + chunk);
    int* s_list = s_spc + chunk;
    int* s_start = s_list + chunk;                                    // [kMaxSpecies + 1]
    int* s_lp = s_start + (kMaxSpecies + 1);                          // [kMaxLMax + 2]
    int* s_fmap = s_lp + (kMaxLMax + 2);                              // [F_pad]

    const int i = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    if (tid < kMaxLMax + 2) s_lp[tid] = A.lp[tid];
    for (int t = tid; t < A.F_pad; t += blockDim.x) s_fmap[t] = A.fmap[t];
    const int64_t seg_beg = A.offsets[i], seg_end = A.offsets[i + 1];
    const int L1 = A.l_max + 1;

    int my_l = 0, my_nt = 0, my_mt = 0;
    const int group_threads = 32 * A.W_s;
    const int g = tid / group_threads;
    const int task = tid - g * group_threads;
    if (task < A.T_s) {
        const int packed = A.tasks[task];
        my_l = packed & 0xff;
        my_nt = (packed >> 8) & 0xff;
        my_mt = (packed >> 16) & 0xff;
    }
    __syncthreads();
    const int g_off = my_l * A.n_pad + 4 * my_nt;   // offset inside a G row
    const int y_off = s_lp[my_l] + 4 * my_mt;       // offset inside a Y row

    for (int round = 0; round < A.rounds; ++round) {
        const int a0 = round * A.S_c;
        const int na = min(A.S_c, A.S - a0);
        const bool active = (g < na) && (task < A.T_s);
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;

        for (int64_t pos = seg_beg; pos < seg_end; pos += chunk) {
            const int nc = (int)((seg_end - pos) < (int64_t)chunk ? (seg_end - pos) : (int64_t)chunk);
            for (int t = tid; t < nc; t += blockDim.x) {
                const float4 v = A.rij[pos + t];
                const int j = A.nbr_j[pos + t];
                const int lab = A.species[j];
                int a = (lab >= 0 && lab < 256) ? A.lut[lab] : -1;
                if (a < 0) atomicOr(A.flags, kFlagSpecies);
                if (!(v.w > 1e-6f)) a = -1;  // coincident atoms are flagged by the neighbour search
                s_vec[t] = v;
                s_spc[t] = a;
                s_fc[t] = cutoff_fp32(v.w, A.r_cut, A.width);
            }
            __syncthreads();
            if (warp == 0) {
                int base = 0;
                for (int ga = 0; ga < na; ++ga) {
                    const int a = a0 + ga;
                    if (lane == 0) s_start[ga] = base;
                    for (int p0 = 0; p0 < nc; p0 += 32) {
                        const int p = p0 + lane;
                        const bool mine = (p < nc) && (s_spc[p] == a);
                        const unsigned m = __ballot_sync(0xffffffffu, mine);
                        if (mine) s_list[base + __popc(m & ((1u << lane) - 1u))] = p;
                        base += __popc(m);
                    }
                }
                if (lane == 0) s_start[na] = base;
            }
            __syncthreads();
            const int n_list = s_start[na];
            // Y_lm: one thread per (listed pair, m) chain
            for (int idx = tid; idx < n_list * L1; idx += blockDim.x) {
                const int q = idx / L1;
                const int m = idx - q * L1;
                const float4 v = s_vec[s_list[q]];
                const float inv_r = 1.0f / v.w;
                const float x = v.x * inv_r, y = v.y * inv_r, z = v.z * inv_r;
                float cm = 1.0f, sm = 0.0f;
                for (int t = 0; t < m; ++t) {
                    const float nc2 = cm * x - sm * y;
                    sm = cm * y + sm * x;
                    cm = nc2;
                }
                float* yrow = s_Y + (size_t)q * A.Lp;
                float q2 = 0.0f, q1 = c_ylm_K[m];
                if (m == 0) {
                    yrow[s_lp[0]] = q1;
                } else {
                    yrow[s_lp[m] + 2 * m] = q1 * cm;
                    yrow[s_lp[m]] = q1 * sm;
                }
                for (int l = m + 1; l <= A.l_max; ++l) {
                    const float qq = c_ylm_A[l * 16 + m] * (z * q1 - c_ylm_B[l * 16 + m] * q2);
                    if (m == 0) {
                        yrow[s_lp[l] + l] = qq;
                    } else {
                        yrow[s_lp[l] + l + m] = qq * cm;
                        yrow[s_lp[l] + l - m] = qq * sm;
                    }
                    q2 = q1;
                    q1 = qq;
                }
            }
            // radial values G = f_cut I^o_nl from the spline: one warp per listed pair, lanes over padded (l, n)
            for (int q = warp; q < n_list; q += nwarps) {
                const int p = s_list[q];
                const float r = s_vec[p].w;
                const float fc = s_fc[p];
                const float x = r * A.inv_delta;
                int k = (int)x;
                k = min(max(k, 0), A.M - 1);
                const float u = x - (float)k;
                const float4* trow = A.table + (int64_t)k * A.F;
                float* grow = s_G + (size_t)q * A.F_pad;
                for (int fp = lane; fp < A.F_pad; fp += 32) {
                    const int col = s_fmap[fp];
                    float val = 0.0f;
                    if (col >= 0) {
                        const float4 c = __ldg(&trow[col]);
                        val = fc * fmaf(u, fmaf(u, fmaf(u, c.w, c.z), c.y), c.x);
                    }
                    grow[fp] = val;
                }
            }
            __syncthreads();
            if (active) {
                const int beg = s_start[g], end = s_start[g + 1];
                for (int q = beg; q < end; ++q) {
                    const float4 gv = *reinterpret_cast<const float4*>(s_G + (size_t)q * A.F_pad + g_off);
                    const float4 yv = *reinterpret_cast<const float4*>(s_Y + (size_t)q * A.Lp + y_off);
                    const float gg[4] = {gv.x, gv.y, gv.z, gv.w};
                    const float yy[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(gg[u], yy[v], acc[u][v]);
                }
            }
            __syncthreads();
        }
        if (active) {
            const int a = a0 + g;
            if (A.include_center && my_l == 0 && my_mt == 0) {
                const int lab = A.species[i];
                const int ai = (lab >= 0 && lab < 256) ? A.lut[lab] : -1;
                if (ai == a) {
                    const float fc0 = cutoff_fp32(0.0f, A.r_cut, A.width);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int n = 4 * my_nt + u;
                        if (n < A.n_max) acc[u][0] += fc0 * A.table[n].x * c_ylm_K[0];
                    }
                }
            }
            float* out = A.coeffs + ((int64_t)i * A.S + a) * A.n_max * A.n_lm + my_l * my_l;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int n = 4 * my_nt + u;
                if (n >= A.n_max) continue;
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int s = 4 * my_mt + v;
                    if (s <= 2 * my_l) out[(int64_t)n * A.n_lm + s] = acc[u][v];
                }
            }
        }
    }
}

static void make_plan(rascal_ctx* ctx) {
    ExpPlan& P = ctx->plan;
    const int L1 = ctx->l_max + 1;
    P.n_pad = (ctx->n_max + 3) / 4 * 4;
    P.F_pad = L1 * P.n_pad;
    int acc = 0;
    for (int l = 0; l <= ctx->l_max; ++l) {
        P.lp[l] = acc;
        acc += (2 * l + 1 + 3) / 4 * 4;
    }
    for (int l = ctx->l_max + 1; l < kMaxLMax + 2; ++l) P.lp[l] = acc;
    P.Lp = acc;
    int mt_total = 0;
    for (int l = 0; l <= ctx->l_max; ++l) mt_total += (2 * l + 1 + 3) / 4;
    P.T_s = (P.n_pad / 4) * mt_total;
    P.W_s = (P.T_s + 31) / 32;
    const int max_warps = 16;
    P.S_c = std::max(1, std::min(ctx->n_species, max_warps / P.W_s));
    if (P.W_s > max_warps) P.S_c = 1;
    P.rounds = (ctx->n_species + P.S_c - 1) / P.S_c;
    P.threads = 32 * P.W_s * P.S_c;
    auto smem_for = [&](int chunk) {
        return (size_t)chunk * sizeof(float4) + (size_t)chunk * (P.F_pad + P.Lp) * sizeof(float) +
               (size_t)chunk * (sizeof(float) + 2 * sizeof(int)) + (kMaxSpecies + 1 + kMaxLMax + 2 + P.F_pad) * sizeof(int) + 64;
    };
    P.chunk = 64;
    while (P.chunk > 16 && smem_for(P.chunk) > 110 * 1024) P.chunk /= 2;
    P.smem = smem_for(P.chunk);
    P.smem_ps = 0;
}

int expansion_setup(rascal_ctx* ctx) {
    make_plan(ctx);
    const ExpPlan& P = ctx->plan;
    std::vector<int> tasks;
    for (int l = 0; l <= ctx->l_max; ++l)
        for (int mt = 0; mt < (2 * l + 1 + 3) / 4; ++mt)
            for (int nt = 0; nt < P.n_pad / 4; ++nt) tasks.push_back(l | (nt << 8) | (mt << 16));
    std::vector<int> fmap(P.F_pad);
    for (int l = 0; l <= ctx->l_max; ++l)
        for (int n = 0; n < P.n_pad; ++n) fmap[l * P.n_pad + n] = (n < ctx->n_max) ? l * ctx->n_max + n : -1;
    RASCAL_CUDA(cudaMalloc(&ctx->d_tasks, sizeof(int) * tasks.size()));
    RASCAL_CUDA(cudaMalloc(&ctx->d_fmap, sizeof(int) * fmap.size()));
    RASCAL_CUDA(cudaMemcpyAsync(ctx->d_tasks, tasks.data(), sizeof(int) * tasks.size(), cudaMemcpyHostToDevice, ctx->stream));
    RASCAL_CUDA(cudaMemcpyAsync(ctx->d_fmap, fmap.data(), sizeof(int) * fmap.size(), cudaMemcpyHostToDevice, ctx->stream));
    RASCAL_CUDA(upload_ylm_constants(ctx->stream));
    RASCAL_CUDA(cudaFuncSetAttribute(k_expansion, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    RASCAL_CUDA(cudaStreamSynchronize(ctx->stream));
    return RASCAL_OK;
}

static ExpArgs make_args(rascal_ctx* ctx, const rascal_system* sys, const int64_t* d_offsets, const int* d_nbr_j,
                         const float* d_rij, float* d_coeffs) {
    const ExpPlan& P = ctx->plan;
    ExpArgs A;
    A.offsets = d_offsets;
    A.nbr_j = d_nbr_j;
    A.rij = reinterpret_cast<const float4*>(d_rij);
    A.species = sys->d_species;
    A.lut = ctx->d_lut;
    A.table = ctx->d_table;
    A.tasks = ctx->d_tasks;
    A.fmap = ctx->d_fmap;
    A.coeffs = d_coeffs;
    A.flags = ctx->d_flags;
    A.N = sys->n_atoms;
    A.n_max = ctx->n_max;
    A.l_max = ctx->l_max;
    A.S = ctx->n_species;
    A.n_lm = ctx->n_lm;
    A.F = ctx->F;
    A.F_pad = P.F_pad;
    A.n_pad = P.n_pad;
    A.Lp = P.Lp;
    A.M = ctx->M;
    A.T_s = P.T_s;
    A.W_s = P.W_s;
    A.S_c = P.S_c;
    A.rounds = P.rounds;
    A.chunk = P.chunk;
    A.include_center = ctx->include_center;
    A.inv_delta = ctx->inv_delta;
    A.r_cut = (float)ctx->r_cut;
    A.width = (float)ctx->smooth_width;
    for (int l = 0; l < kMaxLMax + 2; ++l) A.lp[l] = P.lp[l];
    return A;
}

}  // namespace rascal

using namespace rascal;

extern "C" int rascal_spherical_expansion(rascal_ctx* ctx, const rascal_system* sys, const int64_t* d_offsets,
                                          const int* d_nbr_j, const float* d_rij, float* d_coeffs) {
    clear_error();
    if (!ctx) return set_error(RASCAL_E_ARG, "NULL context");
    int st = validate_system(ctx, sys);
    if (st) return st;
    if (sys->n_atoms == 0) return RASCAL_OK;
    if (!d_offsets || !d_nbr_j || !d_rij || !d_coeffs) return set_error(RASCAL_E_ARG, "NULL device pointer");
    const ExpArgs A = make_args(ctx, sys, d_offsets, d_nbr_j, d_rij, d_coeffs);
    k_expansion<<<sys->n_atoms, ctx->plan.threads, ctx->plan.smem, ctx->stream>>>(A);
    RASCAL_LAUNCH_CHECK("k_expansion");
    return RASCAL_OK;
}
