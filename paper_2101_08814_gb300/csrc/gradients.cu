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
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "ps_fp32.cuh"
#include "tcgen05.cuh"
#include "ylm_fp32.cuh"

namespace rascal {

// Structure of atom i: the largest s < n_s with offs[s] <= i (offsets non-decreasing, offs[n_s] = the atom count),
// found by one warp in rounds of 32 probes (two rounds for up to 1024 structures); every lane returns it.
__device__ inline int warp_find_structure(const int* __restrict__ offs, int n_s, int i, int lane) {
    int lo = 0, hi = n_s;  // offs[lo] <= i < offs[hi]
    while (hi - lo > 1) {
        const int step = (hi - lo + 31) >> 5;
        const int idx = lo + lane * step;
        const unsigned m = __ballot_sync(0xffffffffu, idx < hi && offs[idx] <= i);  // a prefix of the lanes
        lo += (31 - __clz(m)) * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

// E_s = sum_{i in s} w_{a_i} . p_i, one CTA per centre, FP32 partial sums, FP64 across warps and one atomic per centre.
__global__ void k_linear_energy(int N, int n_s, const int* __restrict__ offs, const int* __restrict__ species,
                                const int* __restrict__ lut, const float* __restrict__ ps, const float* __restrict__ w,
                                int64_t F, double* __restrict__ energy) {
    __shared__ double red[32];
    const int i = blockIdx.x;
    int sid = 0;
    if (threadIdx.x < 32) sid = warp_find_structure(offs, n_s, i, threadIdx.x);  // read by thread 0 at the end
    const int lab = species[i];
    const int a = (lab >= 0 && lab < 256) ? lut[lab] : -1;
    // FP32 partial sums per thread and warp (GB300's FP64 rate is a small fraction of its FP32 rate), FP64 across
    // the warps and the structures
    float acc = 0.0f;
    if (a >= 0) {
        const float* p = ps + (int64_t)i * F;
        const float* wa = w + (int64_t)a * F;
        for (int64_t f = threadIdx.x; f < F; f += blockDim.x) acc = fmaf(p[f], wa[f], acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v += red[k];
        atomicAdd(&energy[sid], v);
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
    const float* wsym;      // weights only: k_l (W_l + W_l^T) per species and l, dense [S][L1][Q][Qw] (Qw = ceil4(Q))
    int Qw, Lp_adj, n_adj_tasks;
    int w_tiled;            // per-centre dE/dp: tiled adjoint with one dense l block staged in shared memory
    int w_off;              // bytes from the pair area to that block
    int aux_off;            // bytes from the pair area to the small tables (past both the pair area and C)
    int adj_pref[kMaxLMax + 2];  // prefix counts of the adjoint tile tasks per l
    float* forces;          // FP32 accumulation, converted to the FP64 output afterwards
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
        const float ch = cospif(0.5f * t);  // (1 + cos(pi t)) / 2 = cos^2(pi t / 2), no cancellation near r_cut
        f = ch * ch;
        df = -0.5f * 3.14159265358979f / w * sinpif(t);
    }
}

constexpr int kGradThreads = 256;

// Dense symmetric adjoint weights: Ws[a][l][k][q] = k_l (W_l + W_l^T)[k][q] from the packed upper-triangular
// weight rows (entry (q1 <= q2) at q1 (2Q - q1 - 1) / 2 + q2), zero in the padding columns q >= Q.
__global__ void k_wsym(int S, int L1, int Q, int Qw, int ps_norm, const float* __restrict__ w, int64_t Fp,
                       float* __restrict__ ws) {
    const int64_t total = (int64_t)S * L1 * Q * Qw;
    const int Qpk = Q * (Q + 1) / 2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(e % Qw);
        const int64_t r = e / Qw;
        const int k = (int)(r % Q);
        const int al = (int)(r / Q);
        const int l = al % L1, a = al / L1;
        float v = 0.0f;
        if (q < Q) {
            const int lo = min(q, k), hi = max(q, k);
            v = w[(int64_t)a * Fp + (int64_t)l * Qpk + (lo * (2 * Q - lo - 1)) / 2 + hi];
            if (q == k) v *= 2.0f;
            if (ps_norm) v *= rsqrtf((float)(2 * l + 1));
        }
        ws[e] = v;
    }
}

// One CTA per centre i:
//   1. chat = k_l (W + W^T) C from the centre's coefficients (shared memory) and its weight block (global, L1);
//   2. per chunk of the centre's pairs (two CTA barriers per chunk):
//      radial values (f I, (f I)') per pair (one warp per pair, lanes over (l, n));
//      Y and dY/du per pair (warp w runs the m = w chains for all pairs, lanes over pairs);
//      the last warp stages the next chunk's records (r_ji, the neighbour's species, j, f_cut, f_cut') into the
//      other of two buffers;
//      contraction s = sum_lm Y sum_n chat (f I)', w = sum_lm dY/du sum_n chat f I, then dE/dr_ji, the force
//      scatter and the virial (one warp per pair, lanes over lm, warp-shuffle reduction; F_i and the virial summed
//      per lane, FP64 across the warps at the end).
template <int SHAPE = 0>
__global__ void __launch_bounds__(kGradThreads, 5) k_gradients(const GradArgs A) {
    // hyper shape: compile-time constants for the instantiated shapes (kExpShapes), the launch arguments otherwise
    constexpr ExpShape Cs = kExpShapes[SHAPE];
    const int kNmax = SHAPE ? Cs.n_max : A.n_max, kLmax = SHAPE ? Cs.l_max : A.l_max;
    const int kQ = SHAPE ? Cs.n_max * Cs.S : A.Q, kNlm = SHAPE ? (Cs.l_max + 1) * (Cs.l_max + 1) : A.n_lm;
    const int kNpad = SHAPE ? exp_npad(Cs.n_max) : A.n_pad, kFpad = SHAPE ? (Cs.l_max + 1) * exp_npad(Cs.n_max) : A.F_pad;
    // with n_max a multiple of 4 the padded radial slot f = l n_pad + n is the table column l n_max + n itself
    constexpr bool kFmapId = SHAPE != 0 && Cs.n_max % 4 == 0;
    const int kF = SHAPE ? (Cs.l_max + 1) * Cs.n_max : A.F, kQw = SHAPE ? (Cs.n_max * Cs.S + 3) / 4 * 4 : A.Qw;
    const int kLpAdj = SHAPE ? exp_lp(Cs.l_max + 1) : A.Lp_adj;
    const int kAdjTasks = SHAPE ? (Cs.n_max * Cs.S + 3) / 4 * (exp_lp(Cs.l_max + 1) / 4) : A.n_adj_tasks;
    // prefix counts of the adjoint tile tasks per l: ceil(Q / 4) ceil((2l' + 1) / 4) summed over l' < l
    auto adj_pref = [&](int l) { return SHAPE ? (kQ + 3) / 4 * (exp_lp(l) / 4) : A.adj_pref[l]; };
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int chunk = A.chunk;
    const int QN = kQ * kNlm;
    const int QN4 = (QN + 3) & ~3;                            // keeps the float4 arrays 16-byte aligned
    const int Yp = kNlm | 1;                                // odd pitch: conflict-free float4 rows
    float* s_H = reinterpret_cast<float*>(smem_raw);          // chat [Q][n_lm]
    // per-pair records (r_ji, f_cut, f_cut', species index, j): two buffers that alternate between chunks, so that
    // the next chunk is staged while the current one is processed; they come first in the pair area, so that the
    // first chunk can be staged while the adjoint still reads the coefficients
    float4* s_vec = reinterpret_cast<float4*>(s_H + QN4);     // [2][chunk]
    float* s_fc = reinterpret_cast<float*>(s_vec + 2 * chunk);  // [2][chunk]
    float* s_dfc = s_fc + 2 * chunk;                          // [2][chunk]
    int* s_spc = reinterpret_cast<int*>(s_dfc + 2 * chunk);   // [2][chunk]
    int* s_j = s_spc + 2 * chunk;                             // [2][chunk]
    // the coefficients are needed only by the adjoint, before the pair loop: they share the area of Y and G
    float* s_C = reinterpret_cast<float*>(s_j + 2 * chunk);   // [Q][n_lm], or [Q][Lp_adj] padded per l (tiled adjoint)
    float4* s_Yv = reinterpret_cast<float4*>(s_C);            // [chunk][Yp]  (Y, dY/dux, dY/duy, dY/duz)
    float2* s_GD = reinterpret_cast<float2*>(s_Yv + (size_t)chunk * Yp);  // [chunk][F_pad]  (f I, (f I)')
    int* s_lofm = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(s_vec) + A.aux_off);  // [n_lm] l of lm
    int* s_fmap = s_lofm + kNlm;                            // [F_pad]
    __shared__ double red[kGradThreads / 32][12];
    __shared__ int s_sid;

    const int i = blockIdx.x;
    if ((threadIdx.x >> 5) == (blockDim.x >> 5) - 1) {  // the last warp: the centre's structure, for the virial
        const int sid = warp_find_structure(A.offs, A.n_s, i, threadIdx.x & 31);
        if ((threadIdx.x & 31) == 0) s_sid = sid;
    }
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int L1 = kLmax + 1;
    for (int lm = tid; lm < kNlm; lm += blockDim.x) s_lofm[lm] = (int)sqrtf((float)lm);  // l with l^2 <= lm
    if (!kFmapId)
        for (int t = tid; t < kFpad; t += blockDim.x) s_fmap[t] = A.fmap[t];
    const int lab_i = A.species[i];
    const int a_i = (lab_i >= 0 && lab_i < 256) ? A.lut[lab_i] : -1;
    const float* Gp = A.grad_ps ? A.grad_ps + (int64_t)i * A.Fp : (a_i >= 0 ? A.weights + (int64_t)a_i * A.Fp : nullptr);
    const float* c = A.coeffs + (int64_t)i * QN;
    const int Q = kQ, n_lm = kNlm, Qpk = Q * (Q + 1) / 2;
    // one 4 x 4 register tile of chat_l = Ws_l C_l (rows 4 qt.., columns 4 st.. of the l block), Ws_l dense and
    // symmetric with row pitch Qw (in global memory for the linear model, in shared memory for a per-centre dE/dp)
    auto adjoint_tile = [&](const float* Wl, const float* Cl, int Lq, int l, int qt, int st, bool w_global) {
        // paired FMAs (fma.rn.f32x2): each product rounded exactly as fmaf rounds it
        uint64_t ap[4][2];
#pragma unroll
        for (int u = 0; u < 4; ++u) ap[u][0] = ap[u][1] = 0ull;
        for (int k = 0; k < kQ; ++k) {
            const float4 w4 = w_global ? __ldg(reinterpret_cast<const float4*>(Wl + k * kQw))
                                       : *reinterpret_cast<const float4*>(Wl + k * kQw);
            const float4 c4 = *reinterpret_cast<const float4*>(Cl + k * Lq);
            const float ww[4] = {w4.x, w4.y, w4.z, w4.w};
            const uint64_t c01 = f2_pack(c4.x, c4.y), c23 = f2_pack(c4.z, c4.w);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint64_t wu = f2_pack(ww[u], ww[u]);
                ap[u][0] = f2_fma(wu, c01, ap[u][0]);
                ap[u][1] = f2_fma(wu, c23, ap[u][1]);
            }
        }
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            f2_unpack(ap[u][0], acc[u][0], acc[u][1]);
            f2_unpack(ap[u][1], acc[u][2], acc[u][3]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = 4 * qt + u;
            if (q >= kQ) break;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int sx = 4 * st + v;
                if (sx <= 2 * l) s_H[q * kNlm + l * l + sx] = acc[u][v];
            }
        }
    };
    if (A.wsym || A.w_tiled) {
        // adjoint as 4 x 4 register tiles of chat_l = Ws_l C_l: C staged with every l block padded to a multiple of
        // 4 columns (zeros), so that tiles load float4 rows of C and of the dense symmetric weights
        const int Lq = kLpAdj;
        // the padding columns of the l blocks (ceil4(2l + 1) - (2l + 1) of them: three for even l, one for odd l)
        // read as zero; they are disjoint from the copied columns, so the barrier after the copies covers both
        const int n_padc = 4 * (L1 >> 1) + 3 * (L1 & 1);
        for (int e = tid; e < Q * n_padc; e += blockDim.x) {
            const int q = e / n_padc, r = e - q * n_padc;
            const bool odd = (r & 3) == 3;
            const int l = 2 * (r >> 2) + (odd ? 1 : 0);
            s_C[q * Lq + exp_lp(l) + 2 * l + 1 + (odd ? 0 : (r & 3))] = 0.0f;
        }
        // lanes over lm, warps over rows; no barrier separates these copies from the prologue, so l is computed
        // here (once per lm) rather than read from s_lofm, which other warps are still writing
        for (int lm = lane; lm < n_lm; lm += 32) {
            const int l = (int)sqrtf((float)lm);  // l with l^2 <= lm < (l + 1)^2
            const int col = exp_lp(l) + (lm - l * l);
            for (int q = warp; q < Q; q += nwarps) cp_async4(s_C + q * Lq + col, c + q * n_lm + lm);
        }
        cp_async_wait_all();
        __syncthreads();
        const int QT = (Q + 3) >> 2;
        if (A.wsym) {  // linear model: the species' dense blocks, shared by all centres, from global memory (L2)
            const float* Wsa = A.wsym + (int64_t)(a_i < 0 ? 0 : a_i) * L1 * Q * kQw;
            for (int t = tid; t < kAdjTasks && a_i >= 0; t += blockDim.x) {
                int l = 0;
                while (adj_pref(l + 1) <= t) ++l;
                const int r = t - adj_pref(l);
                const int st = r / QT, qt = r - st * QT;
                adjoint_tile(Wsa + (int64_t)l * Q * kQw + 4 * qt, s_C + exp_lp(l) + 4 * st, Lq, l, qt, st, true);
            }
            if (a_i < 0)
                for (int e = tid; e < QN; e += blockDim.x) s_H[e] = 0.0f;
        } else {  // this centre's dE/dp: one l block at a time, expanded to k_l (W_l + W_l^T) in shared memory
            float* s_W = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(s_vec) + A.w_off);  // [Q][Qw]
            for (int l = 0; l < L1; ++l) {
                const float kl = A.ps_norm ? rsqrtf((float)(2 * l + 1)) : 1.0f;
                const float* Wp = Gp + (int64_t)l * Qpk;
                for (int e = tid; e < Q * kQw; e += blockDim.x) {
                    const int k = e / kQw, q = e - k * kQw;
                    float v = 0.0f;
                    if (q < Q) {  // the packed entry (lo <= hi) sits at lo (2Q - lo - 1) / 2 + hi
                        const int lo = min(q, k), hi = max(q, k);
                        v = __ldg(Wp + (lo * (2 * Q - lo - 1)) / 2 + hi);
                        if (q == k) v *= 2.0f;
                        v *= kl;
                    }
                    s_W[e] = v;
                }
                __syncthreads();
                const int ntl = QT * ((2 * l + 1 + 3) / 4);
                for (int t = tid; t < ntl; t += blockDim.x) {
                    const int st = t / QT, qt = t - st * QT;
                    adjoint_tile(s_W + 4 * qt, s_C + exp_lp(l) + 4 * st, Lq, l, qt, st, false);
                }
                __syncthreads();
            }
        }
    } else {
    for (int e = tid; e < QN; e += blockDim.x) cp_async4(s_C + e, c + e);
    cp_async_wait_all();
    __syncthreads();
    // adjoint chat[q][lm] = k_l sum_k (W + W^T)[q][k] C[k][lm]; the packed entry (q1 <= q2) sits at
    // q1 (2Q - q1 - 1) / 2 + q2, and (W + W^T) doubles the diagonal
    for (int e = tid; e < QN; e += blockDim.x) {
        const int q = e / n_lm, lm = e - q * n_lm;
        const int l = s_lofm[lm];
        float acc = 0.0f;
        if (Gp) {
            const float* W = Gp + (int64_t)l * Qpk;
            const float* Cc = s_C + lm;
            int idx = q;  // entry (k, q), k < q
            for (int k = 0; k < q; ++k) {
                acc = fmaf(__ldg(W + idx), Cc[k * n_lm], acc);
                idx += Q - k - 1;
            }
            const int ro = (q * (2 * Q - q - 1)) / 2;  // entries (q, k), k >= q
            acc = fmaf(2.0f * __ldg(W + ro + q), Cc[q * n_lm], acc);
            for (int k = q + 1; k < Q; ++k) acc = fmaf(__ldg(W + ro + k), Cc[k * n_lm], acc);
        }
        s_H[e] = (A.ps_norm ? rsqrtf((float)(2 * l + 1)) : 1.0f) * acc;
    }
    }
    // per-lane sums of F_i (lanes 0..2) and of the virial (lanes 3..11, row-major): FP32 within a warp, FP64 across
    // the warps (GB300's FP64 rate is a small fraction of its FP32 rate)
    float racc = 0.0f;
    const int64_t seg_beg = A.offsets[i], seg_end = A.offsets[i + 1];
    // the last warp stages the pairs (chunk <= 32: one pair per lane), with the next chunk's r_ji and j loaded into
    // registers one chunk ahead
    const bool stager = warp == nwarps - 1;
    float4 nv = make_float4(0.0f, 0.0f, 0.0f, 1.0f);
    int nj = 0;
    if (stager && lane < chunk && seg_beg + lane < seg_end) {
        nv = A.rij[seg_beg + lane];
        nj = A.nbr_j[seg_beg + lane];
    }
    auto stage = [&](int64_t pos, int b) {  // the chunk at pos into record buffer b
        const int t = lane;
        if (t < chunk && pos + t < seg_end) {
            const float4 v = nv;
            const int j = nj;
            if (pos + chunk + t < seg_end) {
                nv = A.rij[pos + chunk + t];
                nj = A.nbr_j[pos + chunk + t];
            }
            const int lab = A.species[j];
            int a = (lab >= 0 && lab < 256) ? A.lut[lab] : -1;
            if (!(v.w > 1e-6f)) a = -1;
            const int o = b * chunk + t;
            s_vec[o] = v;
            s_spc[o] = a;
            s_j[o] = j;
            float f, df;
            cutoff_and_slope(v.w, A.r_cut, A.width, f, df);
            s_fc[o] = f;
            s_dfc[o] = df;
        }
    };
    // the first chunk's records do not overlap the coefficients; the first barrier of the loop also ends the adjoint
    // before Y and G overwrite the coefficients
    if (stager) stage(seg_beg, 0);
    int b = 0;
    for (int64_t pos = seg_beg; pos < seg_end; pos += chunk, b ^= 1) {
        const int nc = (int)((seg_end - pos) < (int64_t)chunk ? (seg_end - pos) : (int64_t)chunk);
        // the chunk's records are staged, and the previous chunk's contraction is done with s_GD and s_Yv
        __syncthreads();
        const int bo = b * chunk;  // this chunk's records: s_vec[bo + p], ...
        // radial values and slopes: one warp per pair, lanes over padded (l, n); the warps without a Y chain first
        for (int p = nwarps - 1 - warp; p < nc; p += nwarps) {
            const float f = s_fc[bo + p], df = s_dfc[bo + p];
            float2* gd = s_GD + p * kFpad;
            if (A.pre_G) {
                const float* pg = A.pre_G + (pos + p) * kF;
                const float* pd = A.pre_D + (pos + p) * kF;
                #pragma unroll
                for (int fp = lane; fp < kFpad; fp += 32) {
                    const int col = kFmapId ? fp : s_fmap[fp];
                    const float g = col >= 0 ? __ldg(pg + col) : 0.0f, dg = col >= 0 ? __ldg(pd + col) : 0.0f;
                    gd[fp] = make_float2(f * g, df * g + f * dg);
                }
            } else {
                const float x = s_vec[bo + p].w * A.inv_delta;
                const int k = min(max((int)x, 0), A.M - 1);
                const float u = x - (float)k;
                const float4* trow = A.table + k * kF;
                #pragma unroll
                for (int fp = lane; fp < kFpad; fp += 32) {
                    const int col = kFmapId ? fp : s_fmap[fp];
                    const float4 cf = col >= 0 ? __ldg(trow + col) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    const float g = fmaf(u, fmaf(u, fmaf(u, cf.w, cf.z), cf.y), cf.x);
                    const float dg = fmaf(u, fmaf(u, 3.0f * cf.w, 2.0f * cf.z), cf.y) * A.inv_delta;
                    gd[fp] = make_float2(f * g, df * g + f * dg);
                }
            }
        }
        // Y and dY/du (gradient of the polynomial extension), forward mode through the recurrence: lanes over the
        // chunk's pairs, one chain of m per lane; a chunk of at most 8 (16) pairs gives each warp four (two) values
        // of m on 8 (16) lanes each, a larger one gives warp w the m = w, w + nwarps, ... chains on all 32 lanes
        const int lpm = nc <= 8 ? 8 : (nc <= 16 ? 16 : 32), mpw = 32 / lpm;
        for (int m = warp * mpw + lane / lpm; m < L1; m += nwarps * mpw) {
            const float km = c_ylm_K[m], fm = (float)m;
#pragma unroll 1
            for (int p = lane % lpm; p < nc; p += lpm) {
                const float4 v = s_vec[bo + p];
                const float inv_r = v.w > 1e-6f ? 1.0f / v.w : 0.0f;
                const float x = v.x * inv_r, y = v.y * inv_r, z = v.z * inv_r;
                float cm = 1.0f, sm = 0.0f, cm1 = 0.0f, sm1 = 0.0f;  // (x+iy)^m and (x+iy)^(m-1)
#pragma unroll 1
                for (int t = 0; t < m; ++t) {
                    cm1 = cm;
                    sm1 = sm;
                    const float nc2 = cm * x - sm * y;
                    sm = cm * y + sm * x;
                    cm = nc2;
                }
                float4* Yrow = s_Yv + p * Yp;
                float q2 = 0.0f, q1 = km, d2 = 0.0f, d1 = 0.0f;
#pragma unroll 1
                for (int l = m; l < L1; ++l) {
                    float q = q1, dq = d1;
                    if (l > m) {
                        const float Al = c_ylm_A[l * 16 + m], Bl = c_ylm_B[l * 16 + m];
                        q = Al * (z * q1 - Bl * q2);
                        dq = Al * (q1 + z * d1 - Bl * d2);
                        q2 = q1;
                        d2 = d1;
                        q1 = q;
                        d1 = dq;
                    }
                    const int l0 = l * l + l;
                    if (m == 0) {
                        Yrow[l0] = make_float4(q, 0.0f, 0.0f, dq);
                    } else {
                        Yrow[l0 + m] = make_float4(q * cm, q * fm * cm1, -q * fm * sm1, dq * cm);
                        Yrow[l0 - m] = make_float4(q * sm, q * fm * sm1, q * fm * cm1, dq * sm);
                    }
                }
            }
        }
        // the next chunk's records go to the other buffer, whose last readers finished before this chunk's barrier
        if (stager && pos + chunk < seg_end) stage(pos + chunk, b ^ 1);
        __syncthreads();
        // contraction with chat, then dE/dr_ji, the force scatter and the virial: one warp per pair, lanes over lm
        for (int p = warp; p < nc; p += nwarps) {
            const int a = s_spc[bo + p];
            if (a < 0) continue;  // warp-uniform
            const float* H = s_H + a * kNmax * n_lm;
            const float2* gd = s_GD + p * kFpad;
            const float4* Yrow = s_Yv + p * Yp;
            float S = 0.0f, Wx = 0.0f, Wy = 0.0f, Wz = 0.0f;
            for (int lm = lane; lm < n_lm; lm += 32) {
                const float2* g = gd + s_lofm[lm] * kNpad;
                const float* h = H + lm;
                float uu = 0.0f, vv = 0.0f;
                for (int n = 0; n < kNmax; ++n) {
                    const float hv = h[n * n_lm];
                    const float2 x = g[n];
                    vv = fmaf(hv, x.x, vv);
                    uu = fmaf(hv, x.y, uu);
                }
                const float4 y = Yrow[lm];
                S = fmaf(uu, y.x, S);
                Wx = fmaf(vv, y.y, Wx);
                Wy = fmaf(vv, y.z, Wy);
                Wz = fmaf(vv, y.w, Wz);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                S += __shfl_xor_sync(0xffffffffu, S, o);
                Wx += __shfl_xor_sync(0xffffffffu, Wx, o);
                Wy += __shfl_xor_sync(0xffffffffu, Wy, o);
                Wz += __shfl_xor_sync(0xffffffffu, Wz, o);
            }
            const float4 v = s_vec[bo + p];
            const float inv_r = 1.0f / v.w;
            const float ux = v.x * inv_r, uy = v.y * inv_r, uz = v.z * inv_r;
            const float wu = Wx * ux + Wy * uy + Wz * uz;
            const float g0 = S * ux + (Wx - wu * ux) * inv_r, g1 = S * uy + (Wy - wu * uy) * inv_r,
                        g2 = S * uz + (Wz - wu * uz) * inv_r;
            const int ra = lane < 3 ? lane : (lane - 3) / 3;  // lane 3 + 3 ra + rb: virial entry (ra, rb)
            const float ga = ra == 0 ? g0 : (ra == 1 ? g1 : g2);
            if (lane < 3) {
                const int j = s_j[bo + p];
                if (j != i) {
                    atomicAdd(&A.forces[3 * (int64_t)j + lane], -ga);
                    racc += ga;
                }
            } else if (lane < 12) {
                const int rb = (lane - 3) - 3 * ra;
                racc = fmaf(ga, rb == 0 ? v.x : (rb == 1 ? v.y : v.z), racc);
            }
        }
    }
    // block reduction of F_i and the virial
    if (lane < 12) red[warp][lane] = (double)racc;
    __syncthreads();
    if (tid < 12) {
        double s = 0.0;
        for (int w = 0; w < nwarps; ++w) s += red[w][tid];
        if (tid < 3) {
            if (s != 0.0) atomicAdd(&A.forces[3 * (int64_t)i + tid], (float)s);
        } else {
            atomicAdd(&A.virial[9 * (int64_t)s_sid + (tid - 3)], s);
        }
    }
}

__global__ void k_forces_f64(int64_t n, const float* __restrict__ f32, double* __restrict__ f64) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        f64[e] = (double)f32[e];
}

// bytes from the pair area to the small tables: the pair records, then the larger of Y and G and the staged
// coefficients
static size_t grad_aux_off(const rascal_ctx* ctx, int chunk, bool tiled) {
    const ExpPlan& P = ctx->plan;
    const size_t QN4 = ((size_t)ctx->Q * ctx->n_lm + 3) / 4 * 4;
    const size_t QL4 = tiled ? ((size_t)ctx->Q * P.Lp + 3) / 4 * 4 : QN4;
    const size_t Yp = (size_t)(ctx->n_lm | 1);
    const size_t records = 2 * (sizeof(float4) + sizeof(float) * 2 + sizeof(int) * 2) * chunk;  // two buffers
    const size_t yg = sizeof(float4) * chunk * Yp + sizeof(float2) * chunk * P.F_pad;  // Y and G, or the coefficients
    return align_up(records + std::max(yg, sizeof(float) * QL4), 16);
}

// bytes from the pair area to the dense weight block of the per-centre tiled adjoint (behind the small tables)
static size_t grad_w_off(const rascal_ctx* ctx, int chunk) {
    return align_up(grad_aux_off(ctx, chunk, true) + sizeof(int) * (ctx->n_lm + ctx->plan.F_pad), 16);
}

static size_t grad_smem(const rascal_ctx* ctx, int chunk, bool tiled, bool w_block = false) {
    const ExpPlan& P = ctx->plan;
    const size_t QN4 = ((size_t)ctx->Q * ctx->n_lm + 3) / 4 * 4;
    if (w_block)
        return sizeof(float) * QN4 + grad_w_off(ctx, chunk) + sizeof(float) * ctx->Q * ((ctx->Q + 3) / 4 * 4) + 64;
    return sizeof(float) * QN4 + grad_aux_off(ctx, chunk, tiled) + sizeof(int) * (ctx->n_lm + P.F_pad) + 64;
}

int gradients_setup(rascal_ctx* ctx) {
    RASCAL_CUDA(upload_ylm_constants(ctx->stream));
    RASCAL_CUDA(cudaFuncSetAttribute(k_gradients<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    RASCAL_CUDA(cudaFuncSetAttribute(k_gradients<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    RASCAL_CUDA(cudaFuncSetAttribute(k_gradients<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    RASCAL_CUDA(cudaFuncSetAttribute(k_gradients<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    RASCAL_CUDA(cudaFuncSetAttribute(k_gradients<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
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
    const int L1 = ctx->l_max + 1;
    const int Qw = (ctx->Q + 3) / 4 * 4;
    const size_t n_ws = d_weights ? (size_t)ctx->n_species * L1 * ctx->Q * Qw : 0;
    void* wbase;
    if ((st = arena_get(ctx->scratch_w, carve_bytes(sizeof(float) * 3 * (size_t)sys->n_atoms, sizeof(float) * n_ws),
                        &wbase)))
        return st;
    Carver wcv(wbase);
    float* f32 = wcv.take<float>(3 * (size_t)sys->n_atoms);
    float* ws = wcv.take<float>(n_ws);
    RASCAL_CUDA(cudaMemsetAsync(f32, 0, sizeof(float) * 3 * sys->n_atoms, ctx->stream));
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
    A.forces = f32;
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
    A.wsym = nullptr;
    if (d_weights) {  // dense symmetric adjoint weights per species and l, for the tiled adjoint
        A.Qw = Qw;
        A.Lp_adj = P.Lp;
        const int blocks = (int)std::min<size_t>((n_ws + 255) / 256, 4096);
        k_wsym<<<blocks, 256, 0, ctx->stream>>>(ctx->n_species, L1, ctx->Q, A.Qw, ctx->ps_norm, d_weights, A.Fp, ws);
        RASCAL_LAUNCH_CHECK("k_wsym");
        A.wsym = ws;
        const int QT = (ctx->Q + 3) / 4;
        A.adj_pref[0] = 0;
        for (int l = 0; l < L1; ++l) A.adj_pref[l + 1] = A.adj_pref[l] + QT * ((2 * l + 1 + 3) / 4);
        for (int l = L1; l < kMaxLMax + 1; ++l) A.adj_pref[l + 1] = A.adj_pref[l];
        A.n_adj_tasks = A.adj_pref[L1];
    }
    // the largest chunk (<= 32: one warp stages a chunk, a pair per lane) that keeps five CTAs per SM (48 registers); a
    // per-centre dE/dp takes the tiled adjoint with one dense l block in shared memory when four CTAs per SM keep a
    // chunk of at least 8 pairs, else the per-element adjoint
    int chunk = 32;
    bool w_tiled = false;
    if (!d_weights) {
        while (chunk > 8 && grad_smem(ctx, chunk, true, true) > 54 * 1024) --chunk;
        w_tiled = grad_smem(ctx, chunk, true, true) <= 54 * 1024;
        if (!w_tiled) chunk = 32;
    }
    const bool tiled = A.wsym != nullptr || w_tiled;
    if (!w_tiled)
        while (chunk > 1 && grad_smem(ctx, chunk, tiled) > 44 * 1024) --chunk;
    // the radial and contraction phases deal the chunk's pairs to the 8 warps: a chunk one or two pairs past a
    // multiple of 8 is rounded down, so that no nearly empty last round remains (rounding down only shrinks the
    // shared memory below)
    constexpr int kW = kGradThreads / 32;
    if (chunk > kW && chunk % kW <= 2) chunk -= chunk % kW;
    // every shared-memory offset and the size come from this final chunk
    A.chunk = chunk;
    A.w_tiled = w_tiled ? 1 : 0;
    A.w_off = 0;
    if (w_tiled) {
        A.Qw = Qw;
        A.Lp_adj = P.Lp;
        A.w_off = (int)grad_w_off(ctx, chunk);
    }
    A.aux_off = (int)grad_aux_off(ctx, chunk, tiled);
    const size_t smem = grad_smem(ctx, chunk, tiled, w_tiled);
    if (smem > 220 * 1024) return set_error(RASCAL_E_UNSUPPORTED, "hypers too large for the gradient kernel");
    if ((st = radial_precompute(ctx, sys, d_offsets, d_rij, true, &A.pre_G, &A.pre_D))) return st;
    // a compiled instance for the hyper shape when the plan's sizes match it (kExpShapes), else the generic kernel
    int shape = 0;
    for (int k = 1; k < kNumExpShapes && !shape; ++k) {
        const ExpShape& c = kExpShapes[k];
        if (ctx->n_max == c.n_max && ctx->l_max == c.l_max && ctx->n_species == c.S && P.n_pad == exp_npad(c.n_max) &&
            P.F_pad == (c.l_max + 1) * exp_npad(c.n_max) && P.Lp == exp_lp(c.l_max + 1) && ctx->Q == c.n_max * c.S &&
            ctx->n_lm == (c.l_max + 1) * (c.l_max + 1) && ctx->F == (c.l_max + 1) * c.n_max && (!A.wsym || A.Qw == (ctx->Q + 3) / 4 * 4))
            shape = k;
    }
    static_assert(kNumExpShapes == 5, "one launch case per shaped instance");
    switch (shape) {
        case 1: k_gradients<1><<<sys->n_atoms, kGradThreads, smem, ctx->stream>>>(A); break;
        case 2: k_gradients<2><<<sys->n_atoms, kGradThreads, smem, ctx->stream>>>(A); break;
        case 3: k_gradients<3><<<sys->n_atoms, kGradThreads, smem, ctx->stream>>>(A); break;
        case 4: k_gradients<4><<<sys->n_atoms, kGradThreads, smem, ctx->stream>>>(A); break;
        default: k_gradients<0><<<sys->n_atoms, kGradThreads, smem, ctx->stream>>>(A); break;
    }
    RASCAL_LAUNCH_CHECK("k_gradients");
    const int64_t n3 = 3 * (int64_t)sys->n_atoms;
    k_forces_f64<<<(unsigned)std::min<int64_t>((n3 + 255) / 256, 8192), 256, 0, ctx->stream>>>(n3, f32, d_forces);
    RASCAL_LAUNCH_CHECK("k_forces_f64");
    return RASCAL_OK;
}

namespace rascal {

// Per-pair feature gradient, explicitly (a test hook for small cases): for pair p with vector r = r_ji,
//   d[p][x][n][lm] = d/dr_x [ f_cut(r) I^o_nl(r) Y_lm(r^) ] = (f I)'(r) Y_lm u_x + f I (dY/du - (dY/du . u) u)_x / r,
// the derivative of the pair's term in c^i_{a_j n l m} (Eq. spherical_expansion_coefficients_gaussians, Appendix B).
// One CTA per pair: thread m < l_max + 1 runs the m chain of Y and of its polynomial-extension gradient, then the
// threads cover (n, lm).
__global__ void k_debug_pair_grad(int64_t P, const float4* __restrict__ rij, const float4* __restrict__ table,
                                  const float* __restrict__ pre_G, const float* __restrict__ pre_D, int n_max, int l_max,
                                  int F, int M, float inv_delta, float r_cut, float width, float* __restrict__ out) {
    extern __shared__ float sdbg[];
    const int n_lm = (l_max + 1) * (l_max + 1);
    float4* sY = reinterpret_cast<float4*>(sdbg);  // [n_lm] (Y, dY/dux, dY/duy, dY/duz)
    float2* sR = reinterpret_cast<float2*>(sY + n_lm);  // [F] (f I, (f I)')
    const int64_t p = blockIdx.x;
    const float4 v = rij[p];
    const float inv_r = v.w > 1e-6f ? 1.0f / v.w : 0.0f;
    const float x = v.x * inv_r, y = v.y * inv_r, z = v.z * inv_r;
    const int L1 = l_max + 1;
    for (int m = threadIdx.x; m < L1; m += blockDim.x) {
        float cm = 1.0f, sm = 0.0f, cm1 = 0.0f, sm1 = 0.0f;
        for (int t = 0; t < m; ++t) {
            cm1 = cm;
            sm1 = sm;
            const float nc = cm * x - sm * y;
            sm = cm * y + sm * x;
            cm = nc;
        }
        const float fm = (float)m;
        float q2 = 0.0f, q1 = c_ylm_K[m], d2 = 0.0f, d1 = 0.0f;
        for (int l = m; l < L1; ++l) {
            float q = q1, dq = d1;
            if (l > m) {
                const float Al = c_ylm_A[l * 16 + m], Bl = c_ylm_B[l * 16 + m];
                q = Al * (z * q1 - Bl * q2);
                dq = Al * (q1 + z * d1 - Bl * d2);
                q2 = q1;
                d2 = d1;
                q1 = q;
                d1 = dq;
            }
            const int l0 = l * l + l;
            if (m == 0) {
                sY[l0] = make_float4(q, 0.0f, 0.0f, dq);
            } else {
                sY[l0 + m] = make_float4(q * cm, q * fm * cm1, -q * fm * sm1, dq * cm);
                sY[l0 - m] = make_float4(q * sm, q * fm * sm1, q * fm * cm1, dq * sm);
            }
        }
    }
    float f, df;
    cutoff_and_slope(v.w, r_cut, width, f, df);
    for (int c = threadIdx.x; c < F; c += blockDim.x) {  // column l n_max + n
        float g, dg;
        if (pre_G) {
            g = pre_G[p * F + c];
            dg = pre_D[p * F + c];
        } else {
            const float xk = v.w * inv_delta;
            const int k = min(max((int)xk, 0), M - 1);
            const float u = xk - (float)k;
            const float4 cf = table[(int64_t)k * F + c];
            g = fmaf(u, fmaf(u, fmaf(u, cf.w, cf.z), cf.y), cf.x);
            dg = fmaf(u, fmaf(u, 3.0f * cf.w, 2.0f * cf.z), cf.y) * inv_delta;
        }
        sR[c] = make_float2(f * g, df * g + f * dg);
    }
    __syncthreads();
    const int per = n_max * n_lm;
    float* o = out + p * 3 * per;
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
        const int n = e / n_lm, lm = e - n * n_lm;
        const int l = (int)sqrtf((float)lm);
        const float2 R = sR[l * n_max + n];
        const float4 Yv = sY[lm];
        const float wu = Yv.y * x + Yv.z * y + Yv.w * z;
        o[e] = R.y * Yv.x * x + R.x * (Yv.y - wu * x) * inv_r;
        o[per + e] = R.y * Yv.x * y + R.x * (Yv.z - wu * y) * inv_r;
        o[2 * per + e] = R.y * Yv.x * z + R.x * (Yv.w - wu * z) * inv_r;
    }
}

}  // namespace rascal

extern "C" int rascal_debug_pair_gradients(rascal_ctx* ctx, int64_t n_pairs, const float* d_rij, float* d_dc) {
    clear_error();
    if (!ctx) return set_error(RASCAL_E_ARG, "NULL context");
    if (n_pairs < 0 || n_pairs > (1 << 20)) return set_error(RASCAL_E_ARG, "n_pairs must be in [0, 2^20] (a test hook)");
    if (n_pairs == 0) return RASCAL_OK;
    if (!d_rij || !d_dc) return set_error(RASCAL_E_ARG, "NULL device pointer");
    const float* G = nullptr;
    const float* D = nullptr;
    if (ctx->radial != RASCAL_RADIAL_SPLINE) {
        if (ctx->radial == RASCAL_RADIAL_MLP && !ctx->mlp_params)
            return set_error(RASCAL_E_ARG, "radial mode MLP needs trained parameters");
        const size_t words = (size_t)n_pairs * ctx->F;
        void* base;
        int st = arena_get(ctx->scratch, carve_bytes(words * 4, words * 4), &base);
        if (st) return st;
        Carver cv(base);
        float* g = cv.take<float>(words);
        float* d = cv.take<float>(words);
        const float4* rij = reinterpret_cast<const float4*>(d_rij);
        st = ctx->radial == RASCAL_RADIAL_MLP ? mlp_infer(ctx, n_pairs, rij, nullptr, g, d)
                                              : radial_exact_pairs(ctx, n_pairs, rij, g, d);
        if (st) return st;
        G = g;
        D = d;
    }
    const size_t smem = sizeof(float4) * ctx->n_lm + sizeof(float2) * ctx->F;
    k_debug_pair_grad<<<(unsigned)n_pairs, 128, smem, ctx->stream>>>(
        n_pairs, reinterpret_cast<const float4*>(d_rij), ctx->d_table, G, D, ctx->n_max, ctx->l_max, ctx->F, ctx->M,
        ctx->inv_delta, (float)ctx->r_cut, (float)ctx->smooth_width, d_dc);
    RASCAL_LAUNCH_CHECK("k_debug_pair_grad");
    return RASCAL_OK;
}
