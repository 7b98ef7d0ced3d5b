// Fused pair kernel for the density coefficients (Eq. spherical_expansion_coefficients_gaussians), optionally
// followed in the same CTA by the power spectrum (Eq. nu2-basis-coupled):
//   c^i_{a n l m} = sum_{j in A_i, a_j = a} f_cut(r_ji) I^o_nl(r_ji) Y_lm(r^_ji)
//   p^i_{q1 q2 l} = (2l+1)^-1/2 sum_m c^i_{q1 l m} c^i_{q2 l m}
//
// One CTA per centre i. The centre's CSR segment of pairs is processed in chunks staged in shared memory:
//   1. stage r_ji (float4 x, y, z, r), the neighbour's species and f_cut(r) for the chunk;
//   2. list the chunk's pairs by species (warp ballots, so the order is deterministic);
//   3. per pair: Y_lm by the Cartesian recurrence (one thread per (pair, m) chain) and the radial values
//      G_nl = f_cut(r) I^o_nl(r) from the FP32 cubic spline table (one warp per pair, lanes over (l, n)). With one
//      species round (the SIMT Gram forms) steps 2 and 3 run side by side, the rows of Y and G indexed by pair
//      position; otherwise step 3 follows step 2 and covers only the round's listed pairs;
//   4. accumulate: each thread owns a 4(n) x 4(m) register tile of one l and one species and adds the outer
//      product G_{l, n-tile} x Y_{l, m-tile} for every listed pair of its species (16 FMAs per two float4 loads).
// The segment reduction happens in registers; no atomics. The tiles are stored to the centre's block of c in global
// memory and, when the power spectrum is fused, also into shared memory, where the Gram runs without c ever being
// read back from HBM:
//   kGramSimt    FP32 register-tiled Gram on the CUDA cores from CT[lm][q] (ps_fp32.cuh);
//   kGramBf16    tcgen05 MMA, BF16 operands, FP32 accumulators in TMEM (tcgen05.cuh);
//   kGramTf32x3  tcgen05 MMA, TF32 hi/lo split, three MMAs per K step (FP32-grade).
// The Gram output is staged per group of l values in the (then free) pair-staging buffers and written to global
// memory by bulk copies.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "ps_fp32.cuh"
#include "tcgen05.cuh"
#include "ylm_fp32.cuh"

namespace rascal {

// kGramSel: the FP32 form restricted to listed features (its own instantiation, so that the full Gram's register
// allocation is not affected by the selection branch)
// kGramRTf32 / kGramRBf16: the tensor-core Gram in rounds of one l (operands staged per round in the pair rows,
// M = 64 MMAs into two 64-column TMEM slots, epilogue by every warp storing p straight to global memory)
enum GramMode : int { kGramNone = 0, kGramSimt = 1, kGramBf16 = 2, kGramTf32x3 = 3, kGramSel = 4, kGramRTf32 = 5,
                      kGramRBf16 = 6 };
constexpr int kRtcLbo = 144;  // bytes between core matrices adjacent along K (bank groups advance by one per step)
constexpr int kMaxGroups = kMaxLMax + 2;

struct ExpArgs {
    const int64_t* offsets;
    const int* nbr_j;
    const float4* rij;
    const int* species;
    const int* lut;
    const float4* table;
    const float* pre_G;  // per-pair radial values [P][F] (EXACT / MLP modes) or NULL (spline table)
    const float* c_in;   // tensor-core power spectrum of given coefficients [N][Q][n_lm]: no pair phase, or NULL
    const int* sel;      // selected features (FP32 form): packed (l | q1 << 8 | q2 << 16) per output column, or NULL
    int n_sel;
    const int* tasks;
    const int* fmap;
    float* coeffs;
    unsigned* flags;
    int N, n_max, l_max, S, n_lm, F, F_pad, n_pad, Lp, Ly, M, T_s, W_s, S_c, rounds, chunk, include_center;
    float inv_delta, r_cut, width;
    int lp[kMaxLMax + 2];
    // fused power spectrum
    float* ps;
    int64_t ps_stride;
    int layout, ps_norm, Q, per_l;
    int gram_off;                   // bytes: CT (SIMT, behind the pair area) or operand tiles (tensor cores, at 0)
    int pair_off;                   // bytes: start of the pair staging area (behind the tiles in tensor-core mode)
    int stage_floats;               // capacity of the staging area (aliases the pair buffers)
    int p_half;                     // SIMT: the first staging half holds p_half floats, the second the rest
    int n_groups;
    int g_lo[kMaxGroups], g_hi[kMaxGroups];      // l range [g_lo, g_hi) of each output group
    const int* ps_tasks;            // SIMT tasks, l descending
    int g_tbeg[kMaxGroups], g_tend[kMaxGroups];  // SIMT task ranges of the groups
    int Qp;                         // SIMT CT row pitch
    int N_mma, tm_cols, slot_cols, lo_off, tiles_bytes;
    int tile_off[kMaxLMax + 1], sbo[kMaxLMax + 1], nk[kMaxLMax + 1];
    // rounds of one l (kGramRTf32 / kGramRBf16)
    int rtc_half, rtc_lo, rtc_c_bytes;            // bytes per operand half, offset of the lo tile, staged c bytes
    int rtc_kq[kMaxLMax + 1];                     // units of four K elements per row (kpad / 4)
    float rtc_sc[kMaxLMax + 1];                  // operand scale s_l, s_l^2 = k_l
    uint32_t stall_polls;                        // test hook: > 0 makes the first completion wait run out
};

__device__ inline float cutoff_fp32(float r, float r_cut, float w) {
    if (r <= r_cut - w) return 1.0f;
    if (r >= r_cut) return 0.0f;
    // (1 + cos(pi t)) / 2 written as cos^2(pi t / 2): no cancellation where f is small, near r_cut
    const float c = cospif(0.5f * ((r - r_cut + w) / w));
    return c * c;
}

// Position (in floats, 0..3) at which a staged block must start in a 16-byte aligned buffer so that the staged and
// the global addresses agree modulo 16 bytes.
__device__ inline int stage_shift(const float* dst) { return (int)((reinterpret_cast<uintptr_t>(dst) >> 2) & 3); }

// Writes count floats staged at st (st and dst congruent mod 16 bytes) to dst: thread 0 issues one bulk copy for
// the aligned body, threads 0..6 store the ragged head and tail. Call after the fence and barrier that publish st.
__device__ inline void store_staged(float* dst, const float* st, int count) {
    if (threadIdx.x >= 32) return;  // warp 0 does all of it: the other warps skip the address arithmetic
    const int head = min((4 - stage_shift(dst)) & 3, count);
    const int body = (count - head) & ~3;
    const int tail = count - head - body;
    const int t = threadIdx.x;
    if (t == 0) {  // one bulk group per call, possibly empty, so that waits can count calls
        if (body > 0) bulk_store(dst + head, st + head, (uint32_t)body * 4u);
        bulk_commit();
    }
    if (t < head) dst[t] = st[t];
    if (t >= 4 && t < 4 + tail) dst[head + body + t - 4] = st[head + body + t - 4];
}

// element (q, s) of C_l into the K-major operand tile of l (BF16, or TF32 hi/lo for the three-MMA split)
template <int GRAM>
__device__ inline void put_operand(unsigned char* tiles, const ExpArgs& A, int l, int q, int s, float cv) {
    constexpr int esz = (GRAM == kGramTf32x3) ? 4 : 2, e16 = 16 / esz;
    const int off = A.tile_off[l] + (q >> 3) * A.sbo[l] + (s / e16) * 128 + (q & 7) * 16 + (s % e16) * esz;
    if (GRAM == kGramTf32x3) {
        const float hi = __uint_as_float(__float_as_uint(cv) & 0xFFFFE000u);
        *reinterpret_cast<float*>(tiles + off) = hi;
        *reinterpret_cast<float*>(tiles + A.lo_off + off) = cv - hi;
    } else {
        *reinterpret_cast<__nv_bfloat16*>(tiles + off) = __float2bfloat16_rn(cv);
    }
}

template <int GRAM, int SHAPE = 0>
__global__ void __launch_bounds__(512, 3) k_expansion(const ExpArgs A) {
    // hyper shape: compile-time constants for the instantiated shapes (the index arithmetic folds, loops of known
    // length unroll), the launch arguments otherwise
    constexpr ExpShape C = kExpShapes[SHAPE];
    const int kNmax = SHAPE ? C.n_max : A.n_max, kLmax = SHAPE ? C.l_max : A.l_max, kS = SHAPE ? C.S : A.S;
    const int kQ = SHAPE ? C.n_max * C.S : A.Q, kNlm = SHAPE ? (C.l_max + 1) * (C.l_max + 1) : A.n_lm;
    const int kNpad = SHAPE ? exp_npad(C.n_max) : A.n_pad, kFpad = SHAPE ? (C.l_max + 1) * exp_npad(C.n_max) : A.F_pad;
    // with n_max a multiple of 4 the padded radial slot f = l n_pad + n is the table column l n_max + n itself
    constexpr bool kFmapId = SHAPE != 0 && C.n_max % 4 == 0;
    const int kF = SHAPE ? (C.l_max + 1) * C.n_max : A.F, kLy = SHAPE ? exp_ly(C.l_max) : A.Ly;
    const int kQp = SHAPE ? exp_qp(C.n_max * C.S) : A.Qp, kTs = SHAPE ? exp_ts(C.n_max, C.l_max) : A.T_s;
    const int kWs = SHAPE ? (exp_ts(C.n_max, C.l_max) + 31) / 32 : A.W_s;
    const int kSc = SHAPE ? exp_sc(C.n_max, C.l_max, C.S) : A.S_c;
    const int kRounds = SHAPE ? (C.S + exp_sc(C.n_max, C.l_max, C.S) - 1) / exp_sc(C.n_max, C.l_max, C.S) : A.rounds;
    const int kChunk = SHAPE ? exp_chunk(C.n_max, C.l_max) : A.chunk;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint64_t s_bar[4];  // two MMA slots, a drain barrier and one that nothing arrives at (test hook)
    __shared__ uint32_t s_tmem;
    constexpr bool TC = (GRAM == kGramBf16 || GRAM == kGramTf32x3);
    constexpr bool RTC = (GRAM == kGramRTf32 || GRAM == kGramRBf16);
    const int chunk = kChunk;
    float4* s_vec = reinterpret_cast<float4*>(smem_raw + A.pair_off);
    float* s_G = reinterpret_cast<float*>(s_vec + chunk);            // [chunk][F_pad]
    float* s_Y = s_G + (size_t)chunk * kFpad;                       // [chunk][Ly]
    float* s_fc = s_Y + (size_t)chunk * kLy;
    int* s_spc = reinterpret_cast<int*>(s_fc + chunk);
    int* s_list = s_spc + chunk;
    int* s_start = s_list + chunk;                                    // [kMaxSpecies + 1]
    int* s_fmap = s_start + (kMaxSpecies + 1) + (kMaxLMax + 2);        // [F_pad]
    unsigned char* gram = smem_raw + A.gram_off;                      // CT or tiles
    float* stage = s_G;                                               // reused once the pairs are done

    const int i = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    if (!kFmapId) {
        #pragma unroll 1
        for (int t = tid; t < kFpad; t += blockDim.x) s_fmap[t] = A.fmap[t];
    }
    constexpr bool kCT = (GRAM == kGramSimt || GRAM == kGramSel);  // c held transposed in shared memory
    if (kCT) {  // columns Q..ceil4(Q)-1 of CT are read by the edge tiles and must be zero
        float* CT = reinterpret_cast<float*>(gram);
        const int q_end = (kQ + 3) & ~3;
        if (q_end > kQ)
            for (int lm = tid; lm < kNlm; lm += blockDim.x)
                #pragma unroll 1
                for (int c = kQ; c < q_end; ++c) CT[lm * kQp + c] = 0.0f;
    }
    if (TC || RTC) {
        if (TC)  // K padding and rows >= Q of the operand tiles must read as zero
            for (int b = tid; b < A.tiles_bytes / 16; b += blockDim.x)
                reinterpret_cast<uint4*>(gram)[b] = make_uint4(0, 0, 0, 0);
        if (warp == 0) {
            tmem_alloc(&s_tmem, (uint32_t)A.tm_cols);
            tmem_relinquish();
        }
        if (tid == 0) {
            mbar_init(&s_bar[0], 1);
            mbar_init(&s_bar[1], 1);
            mbar_init(&s_bar[2], 1);
            mbar_init(&s_bar[3], 1);
            fence_mbar_init();
        }
        tc_fence_before();
    }
    const bool given_c = TC && A.c_in != nullptr;  // power spectrum of given coefficients: no pairs
    const int64_t seg_beg = given_c ? 0 : A.offsets[i];
    const int seg_len = given_c ? 0 : (int)(A.offsets[i + 1] - seg_beg);
    const float4* seg_rij = A.rij + seg_beg;
    const int* seg_j = A.nbr_j + seg_beg;
    const float* seg_G = A.pre_G ? A.pre_G + seg_beg * kF : nullptr;
    const int L1 = kLmax + 1;

    int my_l = 0, my_nt = 0, my_mt = 0;
    const int group_threads = 32 * kWs;
    const int g = tid / group_threads;
    const int task = tid - g * group_threads;
    if (task < kTs) {
        const int packed = A.tasks[task];
        my_l = packed & 0xff;
        my_nt = (packed >> 8) & 0xff;
        my_mt = (packed >> 16) & 0xff;
    }
    // the SIMT Gram modes read what the prologue wrote (fmap, CT padding) only after the barriers of the pair phase
    // or of the CT hand-off; the tensor-core modes need it here (tile zeroing before given operands, TMEM address)
    if (!kCT) __syncthreads();
    const int g_off = my_l * kNpad + 4 * my_nt;   // offset inside a G row
    const int y_off = exp_lp(my_l) + 4 * my_mt;       // offset inside a Y row

    float* cdst_r = A.coeffs + (int64_t)i * kQ * kNlm;
    float* cst_r = stage + stage_shift(cdst_r);
    for (int round = 0; round < (given_c ? 0 : kRounds); ++round) {
        const int a0 = round * kSc;
        const int na = min(kSc, kS - a0);
        const bool active = (g < na) && (task < kTs);
        uint64_t ap[4][2];  // the thread's 4 x 4 tile as (v, v+1) pairs of FP32 sums
#pragma unroll
        for (int u = 0; u < 4; ++u) ap[u][0] = ap[u][1] = 0ull;

        for (int pos = 0; pos < seg_len; pos += chunk) {  // pair offsets relative to the centre's segment
            const int nc = min(chunk, seg_len - pos);
            // staging: r_ji and f_cut per pair. With one species round (SIMT Gram forms) the rows of Y and G are
            // indexed by pair position, and warp 0 lists the chunk's pairs by species (s_list, s_start) during the
            // radial and Y phases, which then do not wait for the neighbours' species; with several rounds the list
            // comes first and only the round's pairs get rows (so too in the tensor-core forms, where the two
            // values warp 0 would hold through the phase cost more than the wait: 2.98 against 2.91 ms in BF16)
            const bool early = kCT && kRounds == 1;
            int lab = -1;  // chunk <= 32: the neighbour's species label, held by lane p of warp 0
            float vw = 0.0f;
            auto list_pairs = [&]() {  // warp 0
                int a = -2;  // lanes without a pair match no species
                if (chunk <= 32 && lane < nc) {
                    a = (lab >= 0 && lab < 256) ? A.lut[lab] : -1;
                    if (a < 0) atomicOr(A.flags, kFlagSpecies);
                    if (!(vw > 1e-6f)) a = -1;  // coincident atoms are flagged by the neighbour search
                }
                int base = 0;
                #pragma unroll 1
                for (int ga = 0; ga < na; ++ga) {
                    if (lane == 0) s_start[ga] = base;
                    #pragma unroll 1
                    for (int p0 = 0; p0 < nc; p0 += 32) {
                        const int p = p0 + lane;
                        const bool mine = chunk <= 32 ? (a == a0 + ga) : (p < nc && s_spc[p] == a0 + ga);
                        const unsigned m = __ballot_sync(0xffffffffu, mine);
                        if (mine) s_list[base + __popc(m & ((1u << lane) - 1u))] = p;
                        base += __popc(m);
                    }
                }
                if (lane == 0) s_start[na] = base;
            };
            if (chunk <= 32) {
                if (warp == 0) {
                    if (lane < nc) {
                        const float4 v = seg_rij[pos + lane];
                        const int j = seg_j[pos + lane];
                        s_vec[lane] = v;
                        s_fc[lane] = cutoff_fp32(v.w, A.r_cut, A.width);
                        vw = v.w;
                        lab = A.species[j];
                    }
                    if (!early) list_pairs();
                }
            } else {
            #pragma unroll 1
            for (int t = tid; t < nc; t += blockDim.x) {
                const float4 v = seg_rij[pos + t];
                const int j = seg_j[pos + t];
                const int lb = A.species[j];
                int a = (lb >= 0 && lb < 256) ? A.lut[lb] : -1;
                if (a < 0) atomicOr(A.flags, kFlagSpecies);
                if (!(v.w > 1e-6f)) a = -1;  // coincident atoms are flagged by the neighbour search
                s_vec[t] = v;
                s_spc[t] = a;
                s_fc[t] = cutoff_fp32(v.w, A.r_cut, A.width);
            }
            if (!early) {
                __syncthreads();
                if (warp == 0) list_pairs();
            }
            }
            __syncthreads();
            const int n_rows = early ? nc : s_start[na];
            // Y_lm: warp w runs the chains of m = w, w + nwarps, ... with the lanes over the rows, so the recurrence
            // coefficients and the loop bounds are uniform across the warp
            #pragma unroll 1
            for (int m = warp; m < L1; m += nwarps) {
                const float km = c_ylm_K[m];
                #pragma unroll 1
                for (int q = lane; q < n_rows; q += 32) {
                    const float4 v = s_vec[early ? q : s_list[q]];
                    const float inv_r = 1.0f / v.w;
                    const float x = v.x * inv_r, y = v.y * inv_r, z = v.z * inv_r;
                    float cm = 1.0f, sm = 0.0f;
                    #pragma unroll 1
                    for (int t = 0; t < m; ++t) {
                        const float nc2 = cm * x - sm * y;
                        sm = cm * y + sm * x;
                        cm = nc2;
                    }
                    float* yrow = s_Y + q * kLy;
                    float q2 = 0.0f, q1 = km;
                    if (m == 0) {
                        yrow[exp_lp(0)] = q1;
                        #pragma unroll 1
                        for (int l = 1; l < L1; ++l) {
                            const float qq = c_ylm_A[l * 16] * (z * q1 - c_ylm_B[l * 16] * q2);
                            yrow[exp_lp(l) + l] = qq;
                            q2 = q1;
                            q1 = qq;
                        }
                    } else {
                        yrow[exp_lp(m) + 2 * m] = q1 * cm;
                        yrow[exp_lp(m)] = q1 * sm;
                        #pragma unroll 1
                        for (int l = m + 1; l < L1; ++l) {
                            const float qq = c_ylm_A[l * 16 + m] * (z * q1 - c_ylm_B[l * 16 + m] * q2);
                            float* yl = yrow + exp_lp(l) + l;
                            yl[m] = qq * cm;
                            yl[-m] = qq * sm;
                            q2 = q1;
                            q1 = qq;
                        }
                    }
                }
            }
            // radial values G = f_cut I^o_nl: one warp per row, lanes over padded (l, n); the warps without a Y chain
            // take the first rows
            for (int q = nwarps - 1 - warp; q < n_rows; q += nwarps) {
                const int p = early ? q : s_list[q];
                const float fc = s_fc[p];
                float* grow = s_G + q * kFpad;
                if (A.pre_G) {  // per-pair values (EXACT / MLP radial modes)
                    const float* prow = seg_G + (pos + p) * kF;
                    #pragma unroll
                    for (int fp = lane; fp < kFpad; fp += 32) {
                        const int col = kFmapId ? fp : s_fmap[fp];
                        grow[fp] = col >= 0 ? fc * __ldg(prow + col) : 0.0f;
                    }
                } else {        // cubic spline: interval k, local coordinate u in [0, 1)
                    const float x = s_vec[p].w * A.inv_delta;
                    const int k = min(max((int)x, 0), A.M - 1);
                    const float u = x - (float)k;
                    const float4* trow = A.table + k * kF;
                    #pragma unroll
                    for (int fp = lane; fp < kFpad; fp += 32) {
                        const int col = kFmapId ? fp : s_fmap[fp];
                        const float4 c = col >= 0 ? __ldg(trow + col) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        grow[fp] = fc * fmaf(u, fmaf(u, fmaf(u, c.w, c.z), c.y), c.x);
                    }
                }
            }
            if (early && warp == 0) list_pairs();
            __syncthreads();
            if (active) {
                const int beg = s_start[g], end = s_start[g + 1];
                for (int q = beg; q < end; ++q) {
                    const int row = early ? s_list[q] : q;
                    const float4 gv = *reinterpret_cast<const float4*>(s_G + row * kFpad + g_off);
                    const float4 yv = *reinterpret_cast<const float4*>(s_Y + row * kLy + y_off);
                    const uint64_t y01 = f2_pack(yv.x, yv.y), y23 = f2_pack(yv.z, yv.w);
                    const float gg[4] = {gv.x, gv.y, gv.z, gv.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const uint64_t gu = f2_pack(gg[u], gg[u]);
                        ap[u][0] = f2_fma(gu, y01, ap[u][0]);
                        ap[u][1] = f2_fma(gu, y23, ap[u][1]);
                    }
                }
            }
            // the next chunk or round restages the pair buffers; after the last one the SIMT Gram modes write only
            // CT, and the barrier that hands CT over comes before anything reuses the pair buffers
            if (!kCT || pos + chunk < seg_len || round + 1 < kRounds) __syncthreads();
        }
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            f2_unpack(ap[u][0], acc[u][0], acc[u][1]);
            f2_unpack(ap[u][1], acc[u][2], acc[u][3]);
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
                        if (n < kNmax) acc[u][0] += fc0 * A.table[n].x * c_ylm_K[0];
                    }
                }
            }
            if (RTC) {  // c[q][lm] staged in the (free) pair rows; the operand rounds read it from there
                const int s_end = 2 * my_l + 1 - 4 * my_mt;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (4 * my_nt + u >= kNmax) continue;
                    float* crow = cst_r + (a * kNmax + 4 * my_nt + u) * kNlm + my_l * my_l + 4 * my_mt;
                    if (s_end >= 4 && (reinterpret_cast<uintptr_t>(crow) & 15) == 0) {
                        *reinterpret_cast<float4*>(crow) = make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
                    } else {
#pragma unroll
                        for (int v = 0; v < 4; ++v)
                            if (v < s_end) crow[v] = acc[u][v];
                    }
                }
                continue;
            }
            if (kCT) {  // tile -> CT[l^2 + s][a n_max + n]; c reaches HBM from CT afterwards
                float* ct = reinterpret_cast<float*>(gram) + (my_l * my_l + 4 * my_mt) * kQp + a * kNmax + 4 * my_nt;
                const int v_end = 2 * my_l + 1 - 4 * my_mt, u_end = kNmax - 4 * my_nt;
                const bool vec = u_end >= 4 && (kNmax & 3) == 0;
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    if (v >= v_end) break;
                    float* row = ct + v * kQp;
                    if (vec) {
                        *reinterpret_cast<float4*>(row) = make_float4(acc[0][v], acc[1][v], acc[2][v], acc[3][v]);
                    } else {
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (u < u_end) row[u] = acc[u][v];
                    }
                }
                continue;
            }
            float* out = A.coeffs + ((int64_t)i * kS + a) * kNmax * kNlm + my_l * my_l;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int n = 4 * my_nt + u;
                if (n >= kNmax) continue;
                const int q = a * kNmax + n;
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int s = 4 * my_mt + v;
                    if (s > 2 * my_l) continue;
                    const float cv = acc[u][v];
                    out[n * kNlm + s] = cv;
                    if (TC) put_operand<GRAM>(gram, A, my_l, q, s, cv);
                }
            }
        }
    }
    if (GRAM == kGramNone) return;
    if (RTC) {
        // ---------------------------------------------------------------- tensor-core Gram in rounds of one l
        fence_proxy_async_smem();
        __syncthreads();
        store_staged(cdst_r, cst_r, kQ * kNlm);  // c leaves by one bulk copy (the staged c stays for the operands)
        const int Q = kQ, L1n = kLmax + 1;
        const bool packed = A.layout == RASCAL_LAYOUT_PACKED;
        unsigned char* halves = reinterpret_cast<unsigned char*>(stage) + A.rtc_c_bytes;  // behind the staged c
        const uint32_t halves_s = smem_u32(halves);
        const uint32_t taddr = s_tmem;
        const uint32_t idesc = instr_desc(GRAM == kGramRTf32 ? 2u : 1u, 64u, (uint32_t)A.N_mma);
        float* pout = A.ps + (int64_t)i * A.ps_stride;
        // operands of l into half h from the staged c: 16-byte units of four K elements (s_l c, zero beyond 2l),
        // TF32 hi and lo tiles or BF16; every thread takes some of the Q x kpad / 4 units
        auto write_ops = [&](int l, int h) {
            unsigned char* base = halves + h * A.rtc_half;
            const float sl = A.rtc_sc[l];
            const int n4 = A.rtc_kq[l];
            const float* cl = cst_r + l * l;
            for (int e = tid; e < Q * n4; e += blockDim.x) {
                const int q = e / n4, k4 = e - q * n4;
                const float* src = cl + q * kNlm + 4 * k4;
                const int s0 = 4 * k4;
                const float x0 = s0 <= 2 * l ? sl * src[0] : 0.0f;
                const float x1 = s0 + 1 <= 2 * l ? sl * src[1] : 0.0f;
                const float x2 = s0 + 2 <= 2 * l ? sl * src[2] : 0.0f;
                const float x3 = s0 + 3 <= 2 * l ? sl * src[3] : 0.0f;
                const int row = (q >> 3) * A.sbo[l] + (q & 7) * 16;
                if (GRAM == kGramRTf32) {
                    const float h0 = __uint_as_float(__float_as_uint(x0) & 0xFFFFE000u);
                    const float h1 = __uint_as_float(__float_as_uint(x1) & 0xFFFFE000u);
                    const float h2 = __uint_as_float(__float_as_uint(x2) & 0xFFFFE000u);
                    const float h3 = __uint_as_float(__float_as_uint(x3) & 0xFFFFE000u);
                    const int off = row + k4 * kRtcLbo;
                    *reinterpret_cast<float4*>(base + off) = make_float4(h0, h1, h2, h3);
                    *reinterpret_cast<float4*>(base + A.rtc_lo + off) = make_float4(x0 - h0, x1 - h1, x2 - h2, x3 - h3);
                } else {
                    const int off = row + (k4 >> 1) * kRtcLbo + (k4 & 1) * 8;
                    const __nv_bfloat162 b01 = __floats2bfloat162_rn(x0, x1), b23 = __floats2bfloat162_rn(x2, x3);
                    uint2 w;
                    w.x = *reinterpret_cast<const uint32_t*>(&b01);
                    w.y = *reinterpret_cast<const uint32_t*>(&b23);
                    *reinterpret_cast<uint2*>(base + off) = w;
                }
            }
        };
        auto issue = [&](int l, int sl) {
            const uint32_t d = taddr + (uint32_t)(sl * A.slot_cols);
            const uint32_t a0 = halves_s + (uint32_t)(sl * A.rtc_half);
            for (int kk = 0; kk < A.nk[l]; ++kk) {
                const uint32_t a_addr = a0 + (uint32_t)(kk * 2 * kRtcLbo);
                const uint64_t da = smem_desc(a_addr, kRtcLbo, (uint32_t)A.sbo[l]);
                if (GRAM == kGramRTf32) {
                    const uint64_t dl = smem_desc(a_addr + (uint32_t)A.rtc_lo, kRtcLbo, (uint32_t)A.sbo[l]);
                    mma_tf32_ss(d, da, da, idesc, kk > 0);
                    mma_tf32_ss(d, da, dl, idesc, 1);
                    mma_tf32_ss(d, dl, da, idesc, 1);
                } else {
                    mma_bf16_ss(d, da, da, idesc, kk > 0);
                }
            }
            mma_commit(&s_bar[sl]);
        };
        // rows of this warp (M = 64: TMEM lanes 32 quad + 0..15 hold rows 16 quad + 0..15); the warps of a quadrant
        // share its 16-column chunks
        const int quad = warp & 3, wq = warp >> 2, nwq = (nwarps - quad + 3) >> 2;
        const int r = 16 * quad + lane;
        const bool row_ok = lane < 16 && r < Q;
        const int cend = packed ? min(Q - 1, 16 * quad + 15) + 1 : Q;
        __shared__ int s_fail;
        if (tid == 0) s_fail = 0;
        // round k handles l = l_max - k in slot / operand half k & 1; the MMAs of round k + 1 are issued before
        // the epilogue of round k
        write_ops(kLmax, 0);
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) issue(kLmax, 0);
        for (int k = 0; k < L1n; ++k) {
            const int l = kLmax - k, sl = k & 1;
            if (k + 1 < L1n) write_ops(l - 1, sl ^ 1);  // its half was read by round k - 1's MMAs, waited for below
            fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();  // operands of round k + 1 written; round k - 1's epilogue done with slot sl ^ 1
            tc_fence_after();
            const bool go = s_fail == 0;
            if (tid == 0 && k + 1 < L1n && go) issue(l - 1, sl ^ 1);
            // the test hook points the first wait at a barrier that no MMA signals, bounded by stall_polls polls
            const bool stall = A.stall_polls != 0 && k == 0;
            const bool done = go && __all_sync(0xffffffffu, mbar_wait_bounded(stall ? &s_bar[3] : &s_bar[sl],
                                                                              (uint32_t)((k >> 1) & 1),
                                                                              stall ? A.stall_polls : (1u << 22)));
            if (!done) {
                if (lane == 0) s_fail = 1;
                continue;
            }
            tc_fence_after();
            if (16 * quad < Q) {
                const uint32_t tl = taddr + ((uint32_t)(32 * quad) << 16) + (uint32_t)(sl * A.slot_cols);
                float* out = pout + (int64_t)l * A.per_l;
                for (int c0 = 16 * wq; c0 < cend; c0 += 16 * nwq) {
                    float v[16];
                    tmem_ld16(tl + (uint32_t)c0, v);
                    // packed (q1, q2) = (column c, row r), c <= r, at c (2Q - c - 1) / 2 + r; FULL: at c Q + r
                    int o = packed ? c0 * (2 * Q - c0 - 1) / 2 + r : c0 * Q + r;
                    const int dd = row_ok ? (packed ? r - c0 : Q - 1 - c0) : -1;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        if (j <= dd) out[o] = v[j];
                        o += packed ? Q - 1 - (c0 + j) : Q;
                    }
                }
            }
        }
        if (tid == 0) {  // every MMA issued above has completed before the tensor memory is freed
            if (s_fail) atomicOr(A.flags, kFlagTimeout);
            mma_commit(&s_bar[2]);
            if (!mbar_wait_bounded(&s_bar[2], 0u)) atomicOr(A.flags, kFlagTimeout);
        }
        if (tid == 0) bulk_wait_all();
        tc_fence_before();
        __syncthreads();
        if (warp == 0) {
            tc_fence_after();
            tmem_dealloc(s_tmem, (uint32_t)A.tm_cols);
        }
        return;
    }
    if (given_c) {  // operand tiles from the given coefficients of this centre
        const float* cc = A.c_in + (int64_t)i * kQ * kNlm;
        for (int e = tid; e < kQ * kNlm; e += blockDim.x) {
            const int q = e / kNlm, lm = e - q * kNlm;
            const int l = (int)sqrtf((float)lm);
            put_operand<GRAM>(gram, A, l, q, lm - l * l, __ldg(cc + e));
        }
    }

    // ------------------------------------------------------------------------------------ fused power spectrum
    float* pout = A.ps + (int64_t)i * A.ps_stride;
    if (kCT) {
        fence_proxy_async_smem();
        __syncthreads();
        const float* CT = reinterpret_cast<const float*>(gram);
        {   // c[q][lm] = CT[lm][q]: lanes over lm (coalesced stores), float4 reads along q
            float* cdst = A.coeffs + (int64_t)i * kQ * kNlm;
            const int n_lm = kNlm, Qp = kQp;
            for (int q = 4 * warp; q < kQ; q += 4 * nwarps) {
                const int nq = kQ - q;
                float* d = cdst + q * n_lm + lane;
                const float* src = CT + lane * Qp + q;
#pragma unroll 1
                for (int lm = lane; lm < n_lm; lm += 32, d += 32, src += 32 * Qp) {
                    const float4 v = *reinterpret_cast<const float4*>(src);
                    d[0] = v.x;
                    if (nq > 1) d[n_lm] = v.y;
                    if (nq > 2) d[2 * n_lm] = v.z;
                    if (nq > 3) d[3 * n_lm] = v.w;
                }
            }
        }
        if (GRAM == kGramSel) {  // selected features only: one dot product of length 2l+1 per output, coalesced stores
            float* po = A.ps + (int64_t)i * A.n_sel;
            for (int k = tid; k < A.n_sel; k += blockDim.x) {
                const int packed = __ldg(A.sel + k);
                const int l = packed & 0xff, q1 = (packed >> 8) & 0xff, q2 = (packed >> 16) & 0xff;
                float acc = 0.0f;
                if (l <= kLmax) {
                    const float* r = CT + l * l * kQp;
                    for (int m = 0; m <= 2 * l; ++m, r += kQp) acc = fmaf(r[q1], r[q2], acc);
                    if (A.ps_norm) acc *= rsqrtf((float)(2 * l + 1));
                }
                po[k] = acc;
            }
            return;
        }
        // groups of l alternate between two staging halves; each half is written again only after the bulk store
        // issued from it two groups earlier has finished reading it. Thread 0, which issues the stores, waits for
        // the previous group's store to have read its half before the barrier that ends a group, so that one
        // barrier per group serves both hand-offs.
        for (int gi = 0; gi < A.n_groups; ++gi) {
            // tasks are sorted by decreasing cost (l); alternate rounds are dealt in reverse thread order so that
            // the threads with the longest first tile get the shortest second one. Only the threads that stage
            // tiles work out the staging address and fence their writes for the bulk copy.
            const int T = blockDim.x, tbeg = A.g_tbeg[gi], tend = A.g_tend[gi];
            bool wrote = false;
            for (int r = 0; tbeg + r * T < tend; ++r) {
                const int t = tbeg + r * T + ((r & 1) ? T - 1 - tid : tid);
                if (t >= tend) continue;
                const int lo = A.g_lo[gi];
                float* st = stage + (gi & 1) * A.p_half + stage_shift(pout + (int64_t)lo * A.per_l);
                const int packed = __ldg(&A.ps_tasks[t]);
                const int l = packed & 0xff, t1 = (packed >> 8) & 0xff, t2 = (packed >> 16) & 0xff;
                float acc[4][4];
                gram_tile_fp32(CT, kQp, l, t1, t2, acc);
                store_tile_fp32(st + (l - lo) * A.per_l, kQ, A.layout, t1, t2,
                                A.ps_norm ? rsqrtf((float)(2 * l + 1)) : 1.0f, acc);
                wrote = true;
            }
            if (wrote) fence_proxy_async_smem();
            if (tid == 0 && gi >= 1) bulk_wait_read<0>();  // the store of gi - 1 is done with the half of gi + 1
            __syncthreads();
            if (warp == 0) {
                const int lo = A.g_lo[gi];
                float* dst = pout + (int64_t)lo * A.per_l;
                store_staged(dst, stage + (gi & 1) * A.p_half + stage_shift(dst), (A.g_hi[gi] - lo) * A.per_l);
            }
        }
        if (tid == 0) bulk_wait_all();
        return;
    }
    if (TC) {
        // One MMA batch per l, D_l = C_l C_l^T (rows 0..Q-1 of a 128-row MMA; rows >= Q read whatever follows the
        // operand tile and are never used) into one of two TMEM slots: the batch for l + 2 is issued as soon as
        // the epilogue of l has read its slot, so MMA and epilogue overlap. The epilogue runs on the warps whose
        // TMEM lane quadrant holds rows < Q, one 16-column chunk per warp, into staging halves that leave by bulk
        // copies, alternating between groups of l.
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        const uint32_t taddr = s_tmem;
        const uint32_t tiles_s = smem_u32(gram);
        const uint32_t idesc = instr_desc(GRAM == kGramTf32x3 ? 2u : 1u, 128u, (uint32_t)A.N_mma);
        const int L1n = kLmax + 1;
        auto issue = [&](int l) {
            const uint32_t d = taddr + (uint32_t)((l & 1) * A.slot_cols);
            for (int kk = 0; kk < A.nk[l]; ++kk) {
                const uint32_t a_addr = tiles_s + A.tile_off[l] + kk * 256;
                const uint64_t da = smem_desc(a_addr, 128, A.sbo[l]);
                if (GRAM == kGramTf32x3) {
                    const uint64_t dl = smem_desc(a_addr + A.lo_off, 128, A.sbo[l]);
                    mma_tf32_ss(d, da, da, idesc, kk > 0);
                    mma_tf32_ss(d, da, dl, idesc, 1);
                    mma_tf32_ss(d, dl, da, idesc, 1);
                } else {
                    mma_bf16_ss(d, da, da, idesc, kk > 0);
                }
            }
            mma_commit(&s_bar[l & 1]);
        };
        if (tid == 0) {
            issue(0);
            if (L1n > 1) issue(1);
        }
        const int quad = warp & 3, q1 = 32 * quad + lane;
        const int n_chunks = A.N_mma / 16;
        const bool packed = A.layout == RASCAL_LAYOUT_PACKED;
        // offset of row q1 inside an l block: packed rows hold q2 >= q1 at q1 (2Q - q1 - 1) / 2 + q2
        const int row_off = packed ? (q1 * (2 * kQ - q1 - 1)) / 2 : q1 * kQ;
        bool ok = true;
        int gi = 0;
        for (int l = 0; l < L1n; ++l) {
            const int lo = A.g_lo[gi];
            float* dst = pout + (int64_t)lo * A.per_l;
            float* st = stage + (gi & 1) * A.p_half + stage_shift(dst);
            // warp-uniform, since tcgen05.ld is issued by whole warps; the test hook points the first wait at a
            // barrier that no MMA signals
            const bool stall = A.stall_polls != 0 && l == 0;
            const bool done = __all_sync(0xffffffffu, mbar_wait_bounded(stall ? &s_bar[3] : &s_bar[l & 1],
                                                                        (uint32_t)((l >> 1) & 1),
                                                                        stall ? A.stall_polls : (1u << 22)));
            tc_fence_after();
            if (done && 32 * quad < kQ) {
                const float kl = A.ps_norm ? rsqrtf((float)(2 * l + 1)) : 1.0f;
                float* row = st + (l - lo) * A.per_l + row_off;
                const uint32_t tl = taddr + ((uint32_t)(32 * quad) << 16) + (uint32_t)((l & 1) * A.slot_cols);
                for (int jb = warp >> 2; jb < n_chunks; jb += nwarps >> 2) {
                    if (packed && 16 * jb + 15 < 32 * quad) continue;  // chunk entirely below the diagonal
                    float v[16];
                    tmem_ld16(tl + 16 * jb, v);
                    if (q1 < kQ) {
#pragma unroll
                        for (int t = 0; t < 16; ++t) {
                            const int q2 = 16 * jb + t;
                            if (q2 < kQ && (!packed || q2 >= q1)) row[q2] = kl * v[t];
                        }
                    }
                }
            }
            const bool group_end = l + 1 == A.g_hi[gi];
            if (group_end) fence_proxy_async_smem();
            tc_fence_before();
            ok = __syncthreads_and(done) != 0;
            if (!ok) break;
            tc_fence_after();
            if (tid == 0 && l + 2 < L1n) issue(l + 2);
            if (group_end) {
                store_staged(dst, st, (A.g_hi[gi] - lo) * A.per_l);
                ++gi;
                if (gi >= 2 && gi < A.n_groups) {  // the half of group gi was last read by the store of gi - 2
                    if (tid == 0) bulk_wait_read<1>();
                    __syncthreads();
                }
            }
        }
        if (!ok && tid == 0) {  // a wait ran out: flag it, then wait (bounded) for every MMA this thread issued
            atomicOr(A.flags, kFlagTimeout);
            mma_commit(&s_bar[2]);
            if (!mbar_wait_bounded(&s_bar[2], 0u)) atomicOr(A.flags, kFlagTimeout);
        }
        if (tid == 0) bulk_wait_all();
        tc_fence_before();
        __syncthreads();
        if (warp == 0) {
            tc_fence_after();
            tmem_dealloc(s_tmem, (uint32_t)A.tm_cols);
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
    P.Ly = (acc / 4 | 1) * 4;
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
        return (size_t)chunk * sizeof(float4) + (size_t)chunk * (P.F_pad + P.Ly) * sizeof(float) +
               (size_t)chunk * (sizeof(float) + 2 * sizeof(int)) + (kMaxSpecies + 1 + kMaxLMax + 2 + P.F_pad) * sizeof(int) + 64;
    };
    P.chunk = 32;  // about 30 KB for n_max 12, l_max 9: four CTAs per SM
    while (P.chunk > 8 && smem_for(P.chunk) > 56 * 1024) P.chunk /= 2;
    P.smem = smem_for(P.chunk);
    P.smem_ps = 0;
}

template <int GRAM, int SHAPE = 0>
static int set_attr() {
    RASCAL_CUDA(cudaFuncSetAttribute(k_expansion<GRAM, SHAPE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    return RASCAL_OK;
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
    int st;
    if ((st = set_attr<kGramNone>()) || (st = set_attr<kGramSimt>()) || (st = set_attr<kGramSel>()) ||
        (st = set_attr<kGramBf16>()) ||
        (st = set_attr<kGramTf32x3>()) || (st = set_attr<kGramRTf32>()) || (st = set_attr<kGramRBf16>()) ||
        (st = set_attr<kGramSimt, 1>()) || (st = set_attr<kGramSimt, 2>()) || (st = set_attr<kGramSimt, 3>()) ||
        (st = set_attr<kGramNone, 1>()) || (st = set_attr<kGramNone, 2>()) || (st = set_attr<kGramNone, 3>()) ||
        (st = set_attr<kGramBf16, 1>()) || (st = set_attr<kGramBf16, 2>()) || (st = set_attr<kGramBf16, 3>()) ||
        (st = set_attr<kGramRTf32, 1>()) || (st = set_attr<kGramRTf32, 2>()) || (st = set_attr<kGramRTf32, 3>()) ||
        (st = set_attr<kGramSel, 1>()) || (st = set_attr<kGramSel, 2>()) || (st = set_attr<kGramSel, 3>()) ||
        (st = set_attr<kGramSimt, 4>()) || (st = set_attr<kGramNone, 4>()) || (st = set_attr<kGramBf16, 4>()) ||
        (st = set_attr<kGramRTf32, 4>()) || (st = set_attr<kGramSel, 4>()))
        return st;
    RASCAL_CUDA(cudaStreamSynchronize(ctx->stream));
    return RASCAL_OK;
}

static ExpArgs make_args(rascal_ctx* ctx, const rascal_system* sys, const int64_t* d_offsets, const int* d_nbr_j,
                         const float* d_rij, float* d_coeffs) {
    const ExpPlan& P = ctx->plan;
    ExpArgs A;
    std::memset(&A, 0, sizeof(A));
    A.offsets = d_offsets;
    A.nbr_j = d_nbr_j;
    A.rij = reinterpret_cast<const float4*>(d_rij);
    A.species = sys ? sys->d_species : nullptr;
    A.lut = ctx->d_lut;
    A.table = ctx->d_table;
    A.tasks = ctx->d_tasks;
    A.fmap = ctx->d_fmap;
    A.coeffs = d_coeffs;
    A.flags = ctx->d_flags;
    A.N = sys ? sys->n_atoms : 0;
    A.n_max = ctx->n_max;
    A.l_max = ctx->l_max;
    A.S = ctx->n_species;
    A.n_lm = ctx->n_lm;
    A.F = ctx->F;
    A.F_pad = P.F_pad;
    A.n_pad = P.n_pad;
    A.Lp = P.Lp;
    A.Ly = P.Ly;
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
    A.gram_off = (int)align_up(P.smem, 1024);
    return A;
}

// Sets the fused power-spectrum part of the arguments; returns the total dynamic shared memory in *smem.
static int make_gram(rascal_ctx* ctx, int mode, int layout, float* d_ps, ExpArgs& A, size_t* smem, int* threads) {
    const ExpPlan& P = ctx->plan;
    const int Q = ctx->Q;
    A.ps = d_ps;
    A.layout = layout;
    A.ps_norm = ctx->ps_norm;
    A.stall_polls = ctx->stall_polls;
    A.Q = Q;
    A.per_l = layout == RASCAL_LAYOUT_PACKED ? Q * (Q + 1) / 2 : Q * Q;
    A.ps_stride = (int64_t)(ctx->l_max + 1) * A.per_l;
    const size_t pair_region = (size_t)P.chunk * (P.F_pad + P.Ly);  // floats available for staging
    const int L1 = ctx->l_max + 1;
    *threads = P.threads;
    size_t gram_bytes = 0;
    size_t stage_need = 0;
    size_t tail_end = 0;  // tensor cores: end of the bytes the last MMA reads
    if (mode == kGramRTf32 || mode == kGramRBf16) {
        // one species round, M = 64 rows, N <= 64 columns per TMEM slot; one l per round
        if (P.rounds != 1 || Q > 64) return RASCAL_E_UNSUPPORTED;
        const bool tf32 = mode == kGramRTf32;
        const int esz = tf32 ? 4 : 2, kstep = tf32 ? 8 : 16, e16 = 16 / esz;
        A.N_mma = std::max(8, (Q + 7) / 8 * 8);
        int sbo_max = 0;
        for (int l = 0; l < L1; ++l) {
            const int kpad = (2 * l + 1 + kstep - 1) / kstep * kstep;
            A.nk[l] = kpad / kstep;
            A.rtc_kq[l] = kpad / 4;
            A.sbo[l] = (kpad / e16) * kRtcLbo;
            sbo_max = std::max(sbo_max, A.sbo[l]);
            A.rtc_sc[l] = ctx->ps_norm ? (float)std::pow(2.0 * l + 1.0, -0.25) : 1.0f;
        }
        A.rtc_lo = 8 * sbo_max;  // an M = 64 MMA reads 8 groups of 8 rows
        A.rtc_half = tf32 ? 2 * A.rtc_lo : A.rtc_lo;
        A.slot_cols = 64;
        A.tm_cols = 128;
        A.pair_off = 0;
        A.rtc_c_bytes = (int)align_up(sizeof(float) * ((size_t)Q * ctx->n_lm + 3), 16);
        const size_t need = (size_t)A.rtc_c_bytes + 2 * (size_t)A.rtc_half;
        size_t exp_bytes = P.smem;
        if (need > pair_region * sizeof(float)) exp_bytes += need - pair_region * sizeof(float);
        A.gram_off = (int)align_up(exp_bytes, 1024);
        *smem = exp_bytes;
        *threads = std::max(P.threads, 128);
        return *smem > 200 * 1024 ? RASCAL_E_UNSUPPORTED : RASCAL_OK;
    }
    if (mode == kGramSimt) {
        // row pitch: a multiple of 4 floats with Qp / 4 odd, so float4 reads down a column of CT are conflict-free
        A.Qp = ((Q + 3) / 4 | 1) * 4;
        gram_bytes = sizeof(float) * (size_t)ctx->n_lm * A.Qp;
        A.ps_tasks = ctx->d_pstasks;
        // staging: two halves that alternate between groups of consecutive l (descending, the task order), so that
        // the bulk store of one group overlaps the tiles of the next; a staged block may start up to 3 floats late
        // (alignment with its target in global memory). The halves may differ in size: of the splits of the pair
        // region, the one that needs the fewest groups (fewest barriers and bulk stores) is taken, the more even one
        // on a tie. (Staging the whole centre at once needs three CTAs per SM and measured slower.)
        const size_t blk = (size_t)A.per_l;
        auto half_for = [&](int n) { return ((size_t)n * blk + 3 + 3) / 4 * 4; };  // >= n blocks + 3 floats
        auto groups_for = [&](int n0, int n1) {
            int g = 0;
            for (int left = L1; left > 0; ++g) left -= (g & 1) ? n1 : n0;
            return g;
        };
        int n0 = 1, n1 = 1, n_g = groups_for(1, 1);  // one block per half (the region grows if that does not fit)
        for (int a = 1; a <= L1; ++a) {
            const size_t ha = half_for(a);
            if (ha > pair_region) break;
            const size_t rest = (pair_region - ha) / 4 * 4;
            const int b = rest > 3 ? (int)std::min<size_t>((rest - 3) / blk, (size_t)L1) : 0;
            if (a < L1 && b < 1) continue;
            const int ng = groups_for(a, a < L1 ? b : 0);
            if (ng < n_g || (ng == n_g && std::max(a, b) < std::max(n0, n1))) {
                n0 = a;
                n1 = a < L1 ? b : 0;
                n_g = ng;
            }
        }
        const size_t half = half_for(n0);
        A.p_half = (int)half;
        const int Q4 = (Q + 3) / 4;
        const int per_tile_l = Q4 * (Q4 + 1) / 2;
        int g = 0, t = 0, l = ctx->l_max;
        while (l >= 0) {
            const int n = std::min((g & 1) ? n1 : n0, l + 1);
            A.g_hi[g] = l + 1;
            A.g_lo[g] = l - n + 1;
            A.g_tbeg[g] = t;
            t += n * per_tile_l;
            A.g_tend[g] = t;
            l -= n;
            ++g;
        }
        A.n_groups = g;
        stage_need = half + (n1 > 0 ? (size_t)n1 * blk + 3 : 0);
    } else {
        if (Q > 128) return set_error(RASCAL_E_UNSUPPORTED, "tensor-core power spectrum needs n_species*n_max <= 128");
        const bool tf32 = mode == kGramTf32x3;
        const int esz = tf32 ? 4 : 2, kstep = tf32 ? 8 : 16, e16 = 16 / esz;
        A.N_mma = (Q + 15) / 16 * 16;
        const int Qr = (Q + 7) / 8 * 8;
        int off = 0, read_end = 0;
        for (int l = 0; l <= ctx->l_max; ++l) {
            const int kpad = (2 * l + 1 + kstep - 1) / kstep * kstep;
            A.nk[l] = kpad / kstep;
            A.sbo[l] = (kpad / e16) * 128;
            A.tile_off[l] = off;
            read_end = std::max(read_end, off + 16 * A.sbo[l]);  // an M = 128 MMA reads 16 row groups
            off += (Qr / 8) * A.sbo[l];
        }
        const int hi_bytes = (off + 1023) / 1024 * 1024;
        A.lo_off = tf32 ? hi_bytes : 0;
        A.tiles_bytes = tf32 ? 2 * hi_bytes : hi_bytes;
        // the tiles sit at the start of shared memory and the pair area follows them, so the rows >= Q that the
        // MMA reads past the last tile stay inside the allocation
        A.gram_off = 0;
        A.pair_off = A.tiles_bytes;
        tail_end = (size_t)A.lo_off + read_end;
        A.slot_cols = A.N_mma <= 64 ? 64 : 128;
        A.tm_cols = 2 * A.slot_cols;
        size_t half = std::max((pair_region / 2) / 4 * 4, ((size_t)A.per_l + 3 + 3) / 4 * 4);
        A.p_half = (int)half;
        const size_t cap = half - 3;
        int g = 0;
        for (int l = 0; l < L1;) {
            int n = 0;
            while (l + n < L1 && (size_t)(n + 1) * A.per_l <= cap) ++n;
            A.g_lo[g] = l;
            A.g_hi[g] = l + n;
            l += n;
            ++g;
        }
        A.n_groups = g;
        stage_need = 2 * half;
        *threads = std::max(*threads, 128);  // the epilogue needs all four TMEM lane quadrants
    }
    // the staging area aliases the pair buffers; grow the pair region if one group needs more
    size_t exp_bytes = P.smem;
    const size_t stage_bytes_avail = pair_region * sizeof(float);
    if (stage_need * sizeof(float) > stage_bytes_avail) exp_bytes += stage_need * sizeof(float) - stage_bytes_avail;
    A.stage_floats = (int)std::max(stage_need, pair_region);
    // the staging may run over the (then unused) small arrays behind the pair buffers, up to the gram region
    if (mode == kGramSimt) {
        A.pair_off = 0;
        A.gram_off = (int)align_up(exp_bytes, 1024);
        *smem = (size_t)A.gram_off + gram_bytes;
    } else {
        *smem = std::max((size_t)A.pair_off + exp_bytes, tail_end);
    }
    if (*smem > 220 * 1024) return set_error(RASCAL_E_UNSUPPORTED, "fused power spectrum needs %zu bytes of shared memory", *smem);
    return RASCAL_OK;
}

static_assert(kNumExpShapes == 5, "one dispatch case per shaped instance");

// index of the compiled shape whose derived sizes all equal this launch's, else 0 (the runtime-shaped kernel); the
// CT row pitch Qp is set (and checked) only for the forms that hold c transposed in shared memory
static int exp_shape_of(const rascal_ctx* ctx, const ExpArgs& A, bool with_qp) {
    for (int k = 1; k < kNumExpShapes; ++k) {
        const ExpShape& c = kExpShapes[k];
        if (ctx->n_max != c.n_max || ctx->l_max != c.l_max || ctx->n_species != c.S) continue;
        const bool same = A.n_max == c.n_max && A.l_max == c.l_max && A.S == c.S && A.Q == c.n_max * c.S &&
                          A.n_lm == (c.l_max + 1) * (c.l_max + 1) && A.n_pad == exp_npad(c.n_max) &&
                          A.F_pad == (c.l_max + 1) * exp_npad(c.n_max) && A.F == (c.l_max + 1) * c.n_max &&
                          A.Ly == exp_ly(c.l_max) && (!with_qp || A.Qp == exp_qp(c.n_max * c.S)) &&
                          A.T_s == exp_ts(c.n_max, c.l_max) && A.W_s == (exp_ts(c.n_max, c.l_max) + 31) / 32 &&
                          A.S_c == exp_sc(c.n_max, c.l_max, c.S) &&
                          A.rounds == (c.S + A.S_c - 1) / A.S_c && A.chunk == exp_chunk(c.n_max, c.l_max);
        bool lp_same = true;
        for (int l = 0; l <= c.l_max; ++l) lp_same = lp_same && A.lp[l] == exp_lp(l);
        if (same && lp_same) return k;
    }
    return 0;
}

template <int GRAM, int SHAPE = 0>
static int launch_expansion(rascal_ctx* ctx, const ExpArgs& A, int n_atoms, int threads, size_t smem) {
    k_expansion<GRAM, SHAPE><<<n_atoms, threads, smem, ctx->stream>>>(A);
    RASCAL_LAUNCH_CHECK("k_expansion");
    return RASCAL_OK;
}

// the compiled instance for the launch's hyper shape, else the runtime-shaped kernel
template <int GRAM>
static int launch_shaped(rascal_ctx* ctx, const ExpArgs& A, int n_atoms, int threads, size_t smem) {
    switch (exp_shape_of(ctx, A, GRAM == kGramSimt || GRAM == kGramSel)) {
        case 1: return launch_expansion<GRAM, 1>(ctx, A, n_atoms, threads, smem);
        case 2: return launch_expansion<GRAM, 2>(ctx, A, n_atoms, threads, smem);
        case 3: return launch_expansion<GRAM, 3>(ctx, A, n_atoms, threads, smem);
        case 4: return launch_expansion<GRAM, 4>(ctx, A, n_atoms, threads, smem);
        default: return launch_expansion<GRAM>(ctx, A, n_atoms, threads, smem);
    }
}

int power_spectrum_tc(rascal_ctx* ctx, int64_t n_centres, const float* d_coeffs, int precision, int layout, float* d_ps) {
    ExpArgs A = make_args(ctx, nullptr, nullptr, nullptr, nullptr, nullptr);
    A.N = (int)n_centres;
    A.c_in = d_coeffs;
    const int mode = precision == RASCAL_PS_TF32X3 ? kGramTf32x3 : kGramBf16;
    size_t smem;
    int threads;
    int st = make_gram(ctx, mode, layout, d_ps, A, &smem, &threads);
    if (st) return st;
    return mode == kGramTf32x3 ? launch_expansion<kGramTf32x3>(ctx, A, (int)n_centres, threads, smem)
                               : launch_expansion<kGramBf16>(ctx, A, (int)n_centres, threads, smem);
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
    ExpArgs A = make_args(ctx, sys, d_offsets, d_nbr_j, d_rij, d_coeffs);
    const float* pre_D;
    if ((st = radial_precompute(ctx, sys, d_offsets, d_rij, false, &A.pre_G, &pre_D))) return st;
    return launch_shaped<kGramNone>(ctx, A, sys->n_atoms, ctx->plan.threads, ctx->plan.smem);
}

// PACKED feature index -> (l | q1 << 8 | q2 << 16); out-of-range indices flag an error and decode to l = 255 (zero)
__global__ void k_decode_sel(int64_t n_sel, const int* __restrict__ sel, int Q, int l_max, int* __restrict__ out,
                             unsigned* flags) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n_sel) return;
    const int per_l = Q * (Q + 1) / 2;
    const int f = sel[k];
    if (f < 0 || f >= (l_max + 1) * per_l) {
        atomicOr(flags, kFlagSelection);
        out[k] = 255;
        return;
    }
    const int l = f / per_l, r = f - l * per_l;
    int q1 = 0;  // row q1 starts at q1 (2Q - q1 + 1) / 2 (its diagonal entry)
    while (q1 + 1 < Q && ((q1 + 1) * (2 * Q - q1)) / 2 <= r) ++q1;
    const int q2 = r - (q1 * (2 * Q - q1 - 1)) / 2;
    out[k] = l | (q1 << 8) | (q2 << 16);
}

extern "C" int rascal_soap_selected(rascal_ctx* ctx, const rascal_system* sys, const int64_t* d_offsets,
                                    const int* d_nbr_j, const float* d_rij, int64_t n_sel, const int* d_sel,
                                    float* d_coeffs, float* d_ps) {
    clear_error();
    if (!ctx) return set_error(RASCAL_E_ARG, "NULL context");
    int st = validate_system(ctx, sys);
    if (st) return st;
    if (n_sel < 1 || n_sel > 0x7fffffff) return set_error(RASCAL_E_ARG, "n_sel must be in [1, 2^31)");
    if (sys->n_atoms == 0) return RASCAL_OK;
    if (!d_offsets || !d_nbr_j || !d_rij || !d_sel || !d_coeffs || !d_ps) return set_error(RASCAL_E_ARG, "NULL device pointer");
    if (ctx->Q > 255) return set_error(RASCAL_E_UNSUPPORTED, "feature selection needs n_species*n_max <= 255");
    void* dec;
    if ((st = arena_get(ctx->scratch_sel, sizeof(int) * (size_t)n_sel, &dec))) return st;
    k_decode_sel<<<(unsigned)div_up(n_sel, 256), 256, 0, ctx->stream>>>(n_sel, d_sel, ctx->Q, ctx->l_max,
                                                                       static_cast<int*>(dec), ctx->d_flags);
    RASCAL_LAUNCH_CHECK("k_decode_sel");
    ExpArgs A = make_args(ctx, sys, d_offsets, d_nbr_j, d_rij, d_coeffs);
    const float* pre_D;
    if ((st = radial_precompute(ctx, sys, d_offsets, d_rij, false, &A.pre_G, &pre_D))) return st;
    size_t smem;
    int threads;
    if ((st = make_gram(ctx, kGramSimt, RASCAL_LAYOUT_PACKED, d_ps, A, &smem, &threads))) return st;
    A.sel = static_cast<const int*>(dec);
    A.n_sel = (int)n_sel;
    return launch_shaped<kGramSel>(ctx, A, sys->n_atoms, threads, smem);
}

extern "C" int rascal_soap(rascal_ctx* ctx, const rascal_system* sys, const int64_t* d_offsets, const int* d_nbr_j,
                           const float* d_rij, int precision, int layout, float* d_coeffs, float* d_ps) {
    clear_error();
    if (!ctx) return set_error(RASCAL_E_ARG, "NULL context");
    int st = validate_system(ctx, sys);
    if (st) return st;
    if (layout != RASCAL_LAYOUT_PACKED && layout != RASCAL_LAYOUT_FULL) return set_error(RASCAL_E_ARG, "unknown layout");
    if (precision < RASCAL_PS_FP32 || precision > RASCAL_PS_TF32X3) return set_error(RASCAL_E_ARG, "unknown precision");
    if (sys->n_atoms == 0) return RASCAL_OK;
    if (!d_offsets || !d_nbr_j || !d_rij || !d_coeffs || !d_ps) return set_error(RASCAL_E_ARG, "NULL device pointer");
    ExpArgs A = make_args(ctx, sys, d_offsets, d_nbr_j, d_rij, d_coeffs);
    const float* pre_D;
    if ((st = radial_precompute(ctx, sys, d_offsets, d_rij, false, &A.pre_G, &pre_D))) return st;
    if (precision == RASCAL_PS_TF32X3) {  // TF32x3: the tensor-core Gram in rounds of one l where the hypers fit it
        ExpArgs R = A;
        size_t smem_r;
        int threads_r;
        st = make_gram(ctx, kGramRTf32, layout, d_ps, R, &smem_r, &threads_r);
        if (st == RASCAL_OK) return launch_shaped<kGramRTf32>(ctx, R, sys->n_atoms, threads_r, smem_r);
        if (st != RASCAL_E_UNSUPPORTED) return st;
        clear_error();
    }
    const int mode = precision == RASCAL_PS_FP32 ? kGramSimt : (precision == RASCAL_PS_BF16 ? kGramBf16 : kGramTf32x3);
    size_t smem;
    int threads;
    if ((st = make_gram(ctx, mode, layout, d_ps, A, &smem, &threads))) return st;
    if (mode == kGramSimt) return launch_shaped<kGramSimt>(ctx, A, sys->n_atoms, threads, smem);
    if (mode == kGramBf16) return launch_shaped<kGramBf16>(ctx, A, sys->n_atoms, threads, smem);
    return launch_expansion<kGramTf32x3>(ctx, A, sys->n_atoms, threads, smem);
}
