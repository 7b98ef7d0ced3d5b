// Persistent, warp-specialised fused kernel: density coefficients (Eq. spherical_expansion_coefficients_gaussians)
// and the power spectrum (Eq. nu2-basis-coupled) with the per-l Gram C_l C_l^T on the tcgen05 tensor cores.
//
//   c^i_{a n l m} = sum_{j in A_i, a_j = a} f_cut(r_ji) I^o_nl(r_ji) Y_lm(r^_ji)
//   p^i_{q1 q2 l} = k_l sum_m c^i_{q1 l m} c^i_{q2 l m},   k_l = (2l+1)^-1/2
//
// One CTA per SM walks the centres i = blockIdx.x + it * gridDim.x. Its warps have fixed roles:
//   warps 0-3  epilogue: warp w reads TMEM lane quadrant w (its rows of D_l = k_l C_l C_l^T) and stores the packed
//              p block of each l straight to global memory: for column q1 of its rows q2 >= q1 the lanes write
//              consecutive addresses (D is symmetric), so every store instruction is one coalesced run;
//   warp 4     lane 0 issues the MMAs: per l and K step, D_l += A B^T with A = B = s_l C_l (s_l = k_l^1/2) in the
//              K-major core-matrix layout; TF32 hi/lo split (three MMAs, FP32-grade) or BF16 (one MMA), FP32 in TMEM;
//              M = 64 when Q <= 64 (rows 16k..16k+15 of D in TMEM lanes 32k..32k+15), else M = 128 (row i in lane i);
//   warps 5..  two producer groups of nw warps; group g handles the centres with it % 2 == g. Per chunk of up to
//              32 pairs: one warp loads and lists them by species; Y_lm by Cartesian recurrences (lanes over pairs,
//              warps over m, f_cut folded into the chain's start value) and the radial values I^o_nl (lanes over
//              (l, n), warps over pairs, FP32 cubic spline of a padded table); each thread then adds the outer
//              product G x Y over its species' pairs into a 4(n) x 4(m) register tile of one l (paired FMAs,
//              diagonal operand pairing). At the end of the centre the tiles go to the operand buffer (for the MMAs)
//              and to a c staging block, which leaves by one bulk copy.
// Hand-offs use mbarriers: op_full/op_empty (one operand buffer per producer group), tmem_full/tmem_empty
// (two TMEM slots of 256 columns, one per group of l of a centre). Every wait is bounded; a wait that runs out sets
// the timeout flag and an abort word that makes every role leave its loop at its next wait.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "f32x2.cuh"
#include "tcgen05.cuh"
#include "ylm_fp32.cuh"

namespace rascal {

constexpr int kTcChunk = 32;           // pairs listed per chunk (one lane each)
constexpr int kTcEpiWarps = 4;         // warps 0..3, TMEM lane quadrant = warp index
constexpr int kTcMmaWarp = 4;
constexpr int kTcProd0 = 5;            // first producer warp
constexpr int kTcMaxGroupWarps = 13;   // 5 + 2 * 13 = 31 warps <= 1024 threads
constexpr int kTcSlotCols = 256;       // TMEM columns per slot; two slots
constexpr int kTcMaxRounds = 16;
constexpr int kTcMaxCmds = 64;          // (l, K step) MMA batches per centre
constexpr uint32_t kTcWaitLimit = 1u << 22;
// Operand tiles are K-major core matrices (8 rows x 16 bytes, rows 16 bytes apart) without swizzling. Core matrices
// adjacent along K sit kTcLbo = 144 bytes apart (not 128) and each l's tile starts at a chosen 16-byte phase: a
// thread's 16-byte store for (l, m tile, row) then lands in bank group (lp(l)/4 + m tile + row) mod 8, so the warps'
// stores from consecutive (l, m tile) tasks spread over all 32 banks.
constexpr int kTcLbo = 144;
enum : int { kTcTf32x3 = 0, kTcBf16 = 1 };

struct TcArgs {
    const int64_t* offsets;
    const int* nbr_j;
    const float4* rij;
    const int* species;
    const int* lut;
    const float4* table;  // [M][F_pad] cubic coefficients, column l n_pad + n, zero for n >= n_max
    const float* pre_G;   // per-pair radial values [P][F] (EXACT / MLP radial modes) or NULL
    const int* fmap;      // [F_pad] -> column l n_max + n of pre_G, or -1
    float* coeffs;
    float* ps;
    unsigned* flags;
    int N, n_max, n_pad, l_max, S, Q, n_lm, F, F_pad, Ly, M, include_center, layout;
    float inv_delta, r_cut, width;
    int64_t ps_stride;
    int per_l;
    // producer groups
    int nw, nyw, ws, n_tasks, n_lmt;
    unsigned ymask[kTcMaxGroupWarps];
    int lp[kMaxLMax + 2];  // start of the padded m slots of l in a Y row
    // operand tiles
    int lo_off, Qr, N_mma, M_mma, ops_bytes;
    int tile_off[kMaxLMax + 1], sbo[kMaxLMax + 1], nk[kMaxLMax + 1];
    float sc[kMaxLMax + 1];  // operand scale s_l: s_l^2 = k_l
    // groups of l that share a TMEM slot (one round each)
    int n_rounds;
    int r_lo[kTcMaxRounds], r_hi[kTcMaxRounds];  // l in [r_lo, r_hi]
    int col_off[kMaxLMax + 1];                   // TMEM column of D_l inside its slot
    int r_cmd[kTcMaxRounds + 1];                 // commands [r_cmd[rd], r_cmd[rd + 1]) form round rd
    // shared-memory layout (bytes from the 1024-aligned base)
    int c_off, c_slot_floats, pair_off, pair_bytes, smem_bytes;
    uint32_t wait_limit;
};

// ------------------------------------------------------------------------------------------------ helpers
__device__ __forceinline__ void named_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ float tc_cutoff(float r, float r_cut, float w) {
    if (r <= r_cut - w) return 1.0f;
    if (r >= r_cut) return 0.0f;
    // (1 + cos(pi t)) / 2 written as cos^2(pi t / 2): no cancellation where f is small, near r_cut
    const float c = cospif(0.5f * ((r - r_cut + w) / w));
    return c * c;
}

// Bounded wait on an mbarrier phase that also gives up once another role has aborted.
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, uint32_t limit, volatile int* abort,
                                        unsigned* flags) {
    for (uint32_t it = 0; it < limit; ++it) {
        if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
        if (*abort) return false;
    }
    atomicOr(flags, kFlagTimeout);
    *abort = 1;
    return false;
}

// count floats staged at st (congruent with dst modulo 16 bytes) to dst: thread t == 0 issues one bulk copy of the
// aligned body and commits one bulk group (possibly empty); threads t < 7 store the ragged head and tail.
__device__ __forceinline__ void tc_store_out(float* dst, const float* st, int count, int t) {
    const int head = min((4 - (int)((reinterpret_cast<uintptr_t>(dst) >> 2) & 3)) & 3, count);
    const int body = (count - head) & ~3;
    const int tail = count - head - body;
    if (t == 0) {
        if (body > 0) bulk_store(dst + head, st + head, (uint32_t)body * 4u);
        bulk_commit();
    }
    if (t < head) dst[t] = st[t];
    if (t >= 4 && t < 4 + tail) dst[head + body + t - 4] = st[head + body + t - 4];
}

__device__ __forceinline__ int tc_shift(const float* dst) { return (int)((reinterpret_cast<uintptr_t>(dst) >> 2) & 3); }

// padded m-slot start of l: sum over l' < l of 4 ceil((2l'+1)/4)
__host__ __device__ constexpr int tc_lp(int l) {
    int a = 0;
    for (int k = 0; k < l; ++k) a += (2 * k + 1 + 3) / 4 * 4;
    return a;
}

// One Y_lm chain (fixed m = MM) up to l = L for one pair: q_m^m = start (K_m f_cut), then
// q_l = A_lm (z q_{l-1} - B_lm q_{l-2}); Y_{l,m} = q_l C_m, Y_{l,-m} = q_l S_m (m > 0), Y_{l,0} = q_l.
// Written at slot lp(l) + l + m of the pair's Y row; every index is a compile-time constant.
template <int L, int MM>
__device__ __forceinline__ void tc_ychain(float z, float start, float cm, float sm, float* __restrict__ yrow) {
    float q2 = 0.0f, q1 = start;
    if constexpr (MM == 0) {
        yrow[tc_lp(0)] = q1;
    } else {
        yrow[tc_lp(MM) + 2 * MM] = q1 * cm;
        yrow[tc_lp(MM)] = q1 * sm;
    }
#pragma unroll
    for (int l = MM + 1; l <= L; ++l) {
        const float q = c_ylm_A[l * 16 + MM] * (z * q1 - c_ylm_B[l * 16 + MM] * q2);
        if constexpr (MM == 0) {
            yrow[tc_lp(l) + l] = q;
        } else {
            yrow[tc_lp(l) + l + MM] = q * cm;
            yrow[tc_lp(l) + l - MM] = q * sm;
        }
        q2 = q1;
        q1 = q;
    }
}

template <int L, int MM = 0>
__device__ __forceinline__ void tc_ychain_m(int m, float z, float start, float cm, float sm, float* yrow) {
    if constexpr (MM <= L) {
        if (m == MM) {
            tc_ychain<L, MM>(z, start, cm, sm, yrow);
            return;
        }
        tc_ychain_m<L, MM + 1>(m, z, start, cm, sm, yrow);
    }
}

// the same chain with a run-time l_max (any l_max without a compiled specialisation)
__device__ __forceinline__ void tc_ychain_rt(int l_max, int m, const int* lp, float z, float start, float cm, float sm,
                                             float* __restrict__ yrow) {
    float q2 = 0.0f, q1 = start;
    if (m == 0) {
        yrow[lp[0]] = q1;
    } else {
        yrow[lp[m] + 2 * m] = q1 * cm;
        yrow[lp[m]] = q1 * sm;
    }
#pragma unroll 1
    for (int l = m + 1; l <= l_max; ++l) {
        const float q = c_ylm_A[l * 16 + m] * (z * q1 - c_ylm_B[l * 16 + m] * q2);
        if (m == 0) {
            yrow[lp[l] + l] = q;
        } else {
            yrow[lp[l] + l + m] = q * cm;
            yrow[lp[l] + l - m] = q * sm;
        }
        q2 = q1;
        q1 = q;
    }
}

}  // namespace rascal

namespace rascal {

// L: compile-time l_max of the Y chains (0 = run-time l_max); MODE: kTcTf32x3 or kTcBf16
template <int L, int MODE>
__global__ void __launch_bounds__(1024, 1) k_soap_tc(const TcArgs A) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t s_bar[9];  // op_full[2], op_empty[2], tmem_full[2], tmem_empty[2], drain
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ int s_go[3];        // per role (epilogue, group 0, group 1): continue after a leader's wait
    __shared__ int s_lut[256];
    __shared__ int s_lp[kMaxLMax + 2];
    __shared__ int s_fmap[kMaxLMax * kMaxNMax + 64];
    __shared__ uint32_t s_cmd[3 * kTcMaxCmds];  // per (l, K step), in round order: operand offset, SBO, TMEM column
    uint64_t* op_full = s_bar;
    uint64_t* op_empty = s_bar + 2;
    uint64_t* tm_full = s_bar + 4;
    uint64_t* tm_empty = s_bar + 6;
    uint64_t* drain = s_bar + 8;
    volatile int* abort = &s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* ops = smem;
    float* c_stage = reinterpret_cast<float*>(smem + A.c_off);

    // ---------------------------------------------------------------- set-up
    for (int b = tid; b < 2 * A.ops_bytes / 16; b += blockDim.x) reinterpret_cast<uint4*>(ops)[b] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {  // MMA command table: one entry per (l, K step) of each round
        int k = 0;
        for (int rd = 0; rd < A.n_rounds; ++rd)
            for (int l = A.r_lo[rd]; l <= A.r_hi[rd]; ++l)
                for (int kk = 0; kk < A.nk[l]; ++kk, ++k) {
                    s_cmd[3 * k] = (uint32_t)(A.tile_off[l] + kk * 2 * kTcLbo);
                    s_cmd[3 * k + 1] = (uint32_t)A.sbo[l] | (kk > 0 ? 0x80000000u : 0u);  // top bit: accumulate
                    s_cmd[3 * k + 2] = (uint32_t)A.col_off[l];
                }
    }
    for (int g = 0; g < 2; ++g) {  // padded m slots of the Y rows are read as zeros and never written
        float* sY = reinterpret_cast<float*>(smem + A.pair_off + g * A.pair_bytes + 1024) + kTcChunk * A.F_pad;
        for (int e = tid; e < kTcChunk * A.Ly; e += blockDim.x) sY[e] = 0.0f;
    }
    for (int t = tid; t < 256; t += blockDim.x) s_lut[t] = A.lut[t];
    if (tid < kMaxLMax + 2) s_lp[tid] = A.lp[tid];
    if (A.pre_G)
        for (int t = tid; t < A.F_pad; t += blockDim.x) s_fmap[t] = A.fmap[t];
    if (tid == 0) {
        for (int k = 0; k < 9; ++k) mbar_init(&s_bar[k], (k == 6 || k == 7) ? kTcEpiWarps : 1);
        s_abort = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&s_tmem, 2 * kTcSlotCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = s_tmem;
    const int n_it = (A.N > (int)blockIdx.x) ? (A.N - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (warp < kTcEpiWarps) {
        // ------------------------------------------------------------ epilogue: TMEM -> p in global memory
        // rows of this warp: M = 64: lanes 0..15 hold rows 16 qd + lane; M = 128: lane holds row 32 qd + lane
        const int qd = warp;
        const bool m64 = A.M_mma == 64;
        const int rows0 = m64 ? 16 * qd : 32 * qd;
        const int r = rows0 + lane;
        const int Q = A.Q;
        const bool row_ok = r < Q && (!m64 || lane < 16);
        const int cmax = min(Q - 1, rows0 + (m64 ? 15 : 31));  // packed: columns c <= r only
        const bool packed = A.layout == RASCAL_LAYOUT_PACKED;
        const int cend = packed ? cmax + 1 : Q;
        int R = 0;
        bool run = true;
        for (int it = 0; it < n_it && run; ++it) {
            const int i = (int)blockIdx.x + it * (int)gridDim.x;
            float* pc = A.ps + (int64_t)i * A.ps_stride;
            for (int rd = 0; rd < A.n_rounds; ++rd, ++R) {
                const int s = R & 1;
                const bool ok = tc_wait(&tm_full[s], (uint32_t)((R >> 1) & 1), A.wait_limit, abort, A.flags);
                if (!__all_sync(0xffffffffu, ok)) {
                    run = false;
                    break;
                }
                tc_fence_after();
                if (rows0 < Q) {
                    for (int l = A.r_lo[rd]; l <= A.r_hi[rd]; ++l) {
                        const uint32_t tl = taddr + ((uint32_t)(32 * qd) << 16) + (uint32_t)(s * kTcSlotCols + A.col_off[l]);
                        float* out = pc + (int64_t)l * A.per_l;
                        // packed (q1, q2) = (column c, row r), c <= r, at c (2Q - c - 1) / 2 + r; FULL: at c Q + r
                        int c0 = 0;
                        for (; c0 + 31 < cend; c0 += 32) {
                            float v[32];
                            tmem_ld32(tl + (uint32_t)c0, v);
                            int o = packed ? c0 * (2 * Q - c0 - 1) / 2 + r : c0 * Q + r;
                            const int d = row_ok ? (packed ? r - c0 : 31) : -1;  // column c0 + j is stored when j <= d
#pragma unroll
                            for (int j = 0; j < 32; ++j) {
                                if (j <= d) out[o] = v[j];
                                o += packed ? Q - 1 - (c0 + j) : Q;
                            }
                        }
                        for (; c0 < cend; c0 += 16) {
                            float v[16];
                            tmem_ld16(tl + (uint32_t)c0, v);
                            int o = packed ? c0 * (2 * Q - c0 - 1) / 2 + r : c0 * Q + r;
                            const int d = row_ok ? (packed ? r - c0 : Q - 1 - c0) : -1;
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                if (j <= d) out[o] = v[j];
                                o += packed ? Q - 1 - (c0 + j) : Q;
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tm_empty[s]);  // one arrival per epilogue warp
            }
        }
    } else if (warp == kTcMmaWarp) {
        // ------------------------------------------------------------ MMA issue (one thread)
        if (lane == 0) {
            const uint32_t ops_s = smem_u32(ops);
            const uint32_t idesc = instr_desc(MODE == kTcTf32x3 ? 2u : 1u, (uint32_t)A.M_mma, (uint32_t)A.N_mma);
            int R = 0;
            for (int it = 0; it < n_it; ++it) {
                const int g = it & 1;
                if (!tc_wait(&op_full[g], (uint32_t)((it >> 1) & 1), A.wait_limit, abort, A.flags)) break;
                tc_fence_after();
                const uint32_t base = ops_s + (uint32_t)(g * A.ops_bytes);
                bool ok = true;
                for (int rd = 0; rd < A.n_rounds; ++rd, ++R) {
                    const int s = R & 1;
                    if (R >= 2 && !tc_wait(&tm_empty[s], (uint32_t)(((R >> 1) - 1) & 1), A.wait_limit, abort, A.flags)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dslot = taddr + (uint32_t)(s * kTcSlotCols);
                    for (int k = A.r_cmd[rd]; k < A.r_cmd[rd + 1]; ++k) {
                        const uint32_t a_addr = base + s_cmd[3 * k], w = s_cmd[3 * k + 1];
                        const uint32_t d = dslot + s_cmd[3 * k + 2], accum = w >> 31, sbo = w & 0x7FFFFFFFu;
                        const uint64_t da = smem_desc(a_addr, kTcLbo, sbo);
                        if (MODE == kTcTf32x3) {
                            const uint64_t dl = smem_desc(a_addr + (uint32_t)A.lo_off, kTcLbo, sbo);
                            mma_tf32_ss(d, da, da, idesc, accum);
                            mma_tf32_ss(d, da, dl, idesc, 1);
                            mma_tf32_ss(d, dl, da, idesc, 1);
                        } else {
                            mma_bf16_ss(d, da, da, idesc, accum);
                        }
                    }
                    mma_commit(&tm_full[s]);
                }
                if (!ok) break;
                mma_commit(&op_empty[g]);  // this group's operand buffer may be rewritten once these MMAs are done
            }
            mma_commit(drain);  // every MMA issued above has completed before the TMEM is freed
            if (!mbar_wait_bounded(drain, 0u, kTcWaitLimit)) atomicOr(A.flags, kFlagTimeout);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ producers
        const int pw = warp - kTcProd0, g = pw / A.nw, lw = pw - g * A.nw, lt = lw * 32 + lane;
        const int bar_id = 2 + g, bar_n = 32 * A.nw;
        unsigned char* pair = smem + A.pair_off + g * A.pair_bytes;
        float4* s_unit = reinterpret_cast<float4*>(pair);        // unit vector r^_ji and f_cut, by list position
        float2* s_ku = reinterpret_cast<float2*>(pair + 512);    // spline interval (int bits) and local coordinate
        int* s_pidx = reinterpret_cast<int*>(pair + 768);        // pair offset inside the chunk
        int* s_start = reinterpret_cast<int*>(pair + 896);       // list start of each species, [S + 1]
        float* sG = reinterpret_cast<float*>(pair + 1024);       // [chunk][F_pad] radial values
        float* sY = sG + kTcChunk * A.F_pad;                       // [chunk][Ly] f_cut Y_lm
        float* cst0 = c_stage + g * A.c_slot_floats;
        unsigned char* opsg = ops + g * A.ops_bytes;  // this group's operand buffer
        // this thread's accumulation task: species a, l, n tile nt, m tile mt
        const int a_mine = lt / (32 * A.ws), tk = lt - a_mine * 32 * A.ws;
        const bool has_task = a_mine < A.S && tk < A.n_tasks;
        int l_t = 0, nt = 0, mt = 0;
        if (has_task) {
            nt = tk / A.n_lmt;
            int lmt = tk - nt * A.n_lmt;
            while (lmt >= (2 * l_t + 1 + 3) / 4) {
                lmt -= (2 * l_t + 1 + 3) / 4;
                ++l_t;
            }
            mt = lmt;
        }
        const int goff = l_t * A.n_pad + 4 * nt, yoff = s_lp[l_t] + 4 * mt;
        for (int it = g; it < n_it; it += 2) {
            const int i = (int)blockIdx.x + it * (int)gridDim.x;
            const int64_t seg = A.offsets[i];
            const int seg_len = (int)(A.offsets[i + 1] - seg);
            uint64_t P[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) P[k] = 0ull;
            for (int pos = 0; pos < seg_len; pos += kTcChunk) {
                const int nc = min(kTcChunk, seg_len - pos);
                if (lw == 0) {  // load the chunk, list its pairs by species (ballots: deterministic order)
                    int a = -1;
                    float4 v = make_float4(0.0f, 0.0f, 0.0f, 1.0f);
                    if (lane < nc) {
                        v = __ldg(A.rij + seg + pos + lane);
                        const int lab = __ldg(A.species + __ldg(A.nbr_j + seg + pos + lane));
                        a = (lab >= 0 && lab < 256) ? s_lut[lab] : -1;
                        if (a < 0) atomicOr(A.flags, kFlagSpecies);
                        if (!(v.w > 1e-6f)) a = -1;  // coincident atoms are flagged by the neighbour search
                    }
                    int base = 0, rank = -1;
                    for (int ga = 0; ga < A.S; ++ga) {
                        const unsigned b = __ballot_sync(0xffffffffu, a == ga);
                        if (a == ga) rank = base + __popc(b & ((1u << lane) - 1u));
                        if (lane == 0) s_start[ga] = base;
                        base += __popc(b);
                    }
                    if (lane == 0) s_start[A.S] = base;
                    if (rank >= 0) {
                        const float inv = 1.0f / v.w;
                        s_unit[rank] = make_float4(v.x * inv, v.y * inv, v.z * inv, tc_cutoff(v.w, A.r_cut, A.width));
                        const float xk = v.w * A.inv_delta;
                        const int k = min(max((int)xk, 0), A.M - 1);
                        s_ku[rank] = make_float2(__int_as_float(k), xk - (float)k);
                        s_pidx[rank] = lane;
                    }
                }
                named_sync(bar_id, bar_n);
                const int n_list = s_start[A.S];
                if (lw < A.nyw) {  // Y: lanes over listed pairs, this warp's m chains
                    if (lane < n_list) {
                        const float4 uv = s_unit[lane];
                        float* yrow = sY + lane * A.Ly;
                        unsigned mask = A.ymask[lw];
                        float cm = 1.0f, sm = 0.0f;
                        int mc = 0;
                        while (mask) {
                            const int m = __ffs(mask) - 1;
                            mask &= mask - 1u;
                            for (; mc < m; ++mc) {  // (x + i y)^m
                                const float t = cm * uv.x - sm * uv.y;
                                sm = cm * uv.y + sm * uv.x;
                                cm = t;
                            }
                            const float start = c_ylm_K[m] * uv.w;
                            if constexpr (L > 0) tc_ychain_m<L>(m, uv.z, start, cm, sm, yrow);
                            else tc_ychain_rt(A.l_max, m, s_lp, uv.z, start, cm, sm, yrow);
                        }
                    }
                } else {  // radial values: warps over listed pairs, lanes over four (l, n) slots each
                    const int nr = A.nw - A.nyw;
                    if (!A.pre_G) {  // two pairs per pass, so that eight 16-byte loads per lane are in flight
                        for (int q = lw - A.nyw; q < n_list; q += 2 * nr) {
                            const int q2 = q + nr < n_list ? q + nr : q;
                            const float2 ka = s_ku[q], kb = s_ku[q2];
                            const float4* ta = A.table + (size_t)__float_as_int(ka.x) * A.F_pad;
                            const float4* tb = A.table + (size_t)__float_as_int(kb.x) * A.F_pad;
                            for (int f4 = lane; 4 * f4 < A.F_pad; f4 += 32) {
                                float4 a[4], b[4];
#pragma unroll
                                for (int k = 0; k < 4; ++k) {
                                    a[k] = __ldg(ta + 4 * f4 + k);
                                    b[k] = __ldg(tb + 4 * f4 + k);
                                }
                                float4 oa, ob;
                                float* pa = &oa.x;
                                float* pb = &ob.x;
#pragma unroll
                                for (int k = 0; k < 4; ++k) {
                                    pa[k] = fmaf(ka.y, fmaf(ka.y, fmaf(ka.y, a[k].w, a[k].z), a[k].y), a[k].x);
                                    pb[k] = fmaf(kb.y, fmaf(kb.y, fmaf(kb.y, b[k].w, b[k].z), b[k].y), b[k].x);
                                }
                                *reinterpret_cast<float4*>(sG + q * A.F_pad + 4 * f4) = oa;
                                *reinterpret_cast<float4*>(sG + q2 * A.F_pad + 4 * f4) = ob;
                            }
                        }
                    }
                    for (int q = lw - A.nyw; q < n_list && A.pre_G; q += nr) {
                        float* grow = sG + q * A.F_pad;
                        {
                            const float* prow = A.pre_G + (seg + pos + s_pidx[q]) * A.F;
                            for (int fp = lane; fp < A.F_pad; fp += 32) {
                                const int col = s_fmap[fp];
                                grow[fp] = col >= 0 ? __ldg(prow + col) : 0.0f;
                            }
                        }
                    }
                }
                named_sync(bar_id, bar_n);
                if (has_task) {  // c tile += G x Y over this species' pairs; diagonal pairing of the FP32 pairs
                    const int beg = s_start[a_mine], end = s_start[a_mine + 1];
                    const float* gp = sG + beg * A.F_pad + goff;
                    const float* yp = sY + beg * A.Ly + yoff;
                    for (int q = beg; q < end; ++q, gp += A.F_pad, yp += A.Ly) {
                        const float4 gv = *reinterpret_cast<const float4*>(gp);
                        const float4 yv = *reinterpret_cast<const float4*>(yp);
                        const uint64_t g01 = f2_pack(gv.x, gv.y), g23 = f2_pack(gv.z, gv.w);
                        const uint64_t y01 = f2_pack(yv.x, yv.y), y10 = f2_pack(yv.y, yv.x);
                        const uint64_t y23 = f2_pack(yv.z, yv.w), y32 = f2_pack(yv.w, yv.z);
                        P[0] = f2_fma(g01, y01, P[0]);
                        P[1] = f2_fma(g01, y10, P[1]);
                        P[2] = f2_fma(g01, y23, P[2]);
                        P[3] = f2_fma(g01, y32, P[3]);
                        P[4] = f2_fma(g23, y01, P[4]);
                        P[5] = f2_fma(g23, y10, P[5]);
                        P[6] = f2_fma(g23, y23, P[6]);
                        P[7] = f2_fma(g23, y32, P[7]);
                    }
                }
                if (pos + kTcChunk < seg_len) named_sync(bar_id, bar_n);  // before the next chunk is listed
            }
            // ------------------------------------------------ end of the centre: operands and c staging
            float* cdst = A.coeffs + (int64_t)i * A.Q * A.n_lm;
            float* cst = cst0 + tc_shift(cdst);
            if (lt == 0) {
                bool ok = true;
                if (it >= 2)  // the MMAs of this group's previous centre have finished reading its operand buffer
                    ok = tc_wait(&op_empty[g], (uint32_t)(((it >> 1) - 1) & 1), A.wait_limit, abort, A.flags);
                bulk_wait_read<0>();  // this group's previous c copy has left the staging block
                s_go[1 + g] = ok ? 1 : 0;
            }
            named_sync(bar_id, bar_n);
            if (!s_go[1 + g]) break;
            if (has_task) {
                float acc[4][4];
                f2_unpack(P[0], acc[0][0], acc[1][1]);
                f2_unpack(P[1], acc[0][1], acc[1][0]);
                f2_unpack(P[2], acc[0][2], acc[1][3]);
                f2_unpack(P[3], acc[0][3], acc[1][2]);
                f2_unpack(P[4], acc[2][0], acc[3][1]);
                f2_unpack(P[5], acc[2][1], acc[3][0]);
                f2_unpack(P[6], acc[2][2], acc[3][3]);
                f2_unpack(P[7], acc[2][3], acc[3][2]);
                if (A.include_center && l_t == 0 && mt == 0) {
                    const int lab = A.species[i];
                    const int ai = (lab >= 0 && lab < 256) ? s_lut[lab] : -1;
                    if (ai == a_mine) {
                        const float f0 = tc_cutoff(0.0f, A.r_cut, A.width) * c_ylm_K[0];
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (4 * nt + u < A.n_max) acc[u][0] += f0 * __ldg(A.table + 4 * nt + u).x;
                    }
                }
                const float sl = A.sc[l_t];
                const int s_end = 2 * l_t + 1 - 4 * mt;  // valid m slots of the tile
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (4 * nt + u >= A.n_max) continue;
                    const int q = a_mine * A.n_max + 4 * nt + u;
                    float* crow = cst + q * A.n_lm + l_t * l_t + 4 * mt;
                    if (s_end >= 4 && (reinterpret_cast<uintptr_t>(crow) & 15) == 0) {
                        *reinterpret_cast<float4*>(crow) = make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
                    } else {
#pragma unroll
                        for (int v = 0; v < 4; ++v)
                            if (v < s_end) crow[v] = acc[u][v];
                    }
                    const float x0 = sl * acc[u][0], x1 = sl * acc[u][1], x2 = sl * acc[u][2], x3 = sl * acc[u][3];
                    if (MODE == kTcTf32x3) {
                        const int off = A.tile_off[l_t] + (q >> 3) * A.sbo[l_t] + mt * kTcLbo + (q & 7) * 16;
                        const float h0 = __uint_as_float(__float_as_uint(x0) & 0xFFFFE000u);
                        const float h1 = __uint_as_float(__float_as_uint(x1) & 0xFFFFE000u);
                        const float h2 = __uint_as_float(__float_as_uint(x2) & 0xFFFFE000u);
                        const float h3 = __uint_as_float(__float_as_uint(x3) & 0xFFFFE000u);
                        *reinterpret_cast<float4*>(opsg + off) = make_float4(h0, h1, h2, h3);
                        *reinterpret_cast<float4*>(opsg + A.lo_off + off) = make_float4(x0 - h0, x1 - h1, x2 - h2, x3 - h3);
                    } else {
                        const int off = A.tile_off[l_t] + (q >> 3) * A.sbo[l_t] + (mt >> 1) * kTcLbo + (q & 7) * 16 + (mt & 1) * 8;
                        const __nv_bfloat162 b01 = __floats2bfloat162_rn(x0, x1), b23 = __floats2bfloat162_rn(x2, x3);
                        uint2 w;
                        w.x = *reinterpret_cast<const uint32_t*>(&b01);
                        w.y = *reinterpret_cast<const uint32_t*>(&b23);
                        *reinterpret_cast<uint2*>(opsg + off) = w;
                    }
                }
            }
            fence_proxy_async_smem();
            named_sync(bar_id, bar_n);
            if (lt == 0) mbar_arrive(&op_full[g]);
            tc_store_out(cdst, cst, A.Q * A.n_lm, lt);
        }
        if (lt == 0) bulk_wait_all();
    }
    // ---------------------------------------------------------------- teardown
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(taddr, 2 * kTcSlotCols);
    }
}

}  // namespace rascal

namespace rascal {

// padded copy of the radial table: [M][L1 n_pad] with column l n_pad + n, zeros for n >= n_max
__global__ void k_table_pad(int M, int n_max, int n_pad, int L1, const float4* __restrict__ src, float4* __restrict__ dst) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int F_pad = L1 * n_pad;
    if (e >= (int64_t)M * F_pad) return;
    const int k = (int)(e / F_pad), f = (int)(e - (int64_t)k * F_pad);
    const int l = f / n_pad, n = f - l * n_pad;
    dst[e] = n < n_max ? src[(int64_t)k * L1 * n_max + l * n_max + n] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

template <int L>
static int tc_attr() {
    RASCAL_CUDA(cudaFuncSetAttribute(k_soap_tc<L, kTcTf32x3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    RASCAL_CUDA(cudaFuncSetAttribute(k_soap_tc<L, kTcBf16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    return RASCAL_OK;
}

int soap_tc_setup(rascal_ctx* ctx) {
    const int L1 = ctx->l_max + 1, n_pad = (ctx->n_max + 3) / 4 * 4;
    const int64_t n = (int64_t)ctx->M * L1 * n_pad;
    RASCAL_CUDA(cudaMalloc(&ctx->d_table_pad, sizeof(float4) * n));
    k_table_pad<<<(unsigned)div_up(n, 256), 256, 0, ctx->stream>>>(ctx->M, ctx->n_max, n_pad, L1, ctx->d_table,
                                                                  ctx->d_table_pad);
    RASCAL_LAUNCH_CHECK("k_table_pad");
    RASCAL_CUDA(upload_ylm_constants(ctx->stream));
    int st;
    if ((st = tc_attr<0>()) || (st = tc_attr<6>()) || (st = tc_attr<8>()) || (st = tc_attr<9>())) return st;
    return RASCAL_OK;
}

// Launch plan of k_soap_tc for the context's hypers; RASCAL_E_UNSUPPORTED when they do not fit (the caller then
// uses the per-centre kernel).
static int tc_plan(rascal_ctx* ctx, int mode, int layout, TcArgs& A, size_t* smem, int* threads) {
    std::memset(&A, 0, sizeof(A));
    const int L1 = ctx->l_max + 1, Q = ctx->Q;
    if (Q > 128) return RASCAL_E_UNSUPPORTED;
    A.n_max = ctx->n_max;
    A.n_pad = (ctx->n_max + 3) / 4 * 4;
    A.l_max = ctx->l_max;
    A.S = ctx->n_species;
    A.Q = Q;
    A.n_lm = ctx->n_lm;
    A.F = ctx->F;
    A.F_pad = L1 * A.n_pad;
    for (int l = 0; l < kMaxLMax + 2; ++l) A.lp[l] = tc_lp(std::min(l, L1));
    const int Lp = tc_lp(L1);
    A.Ly = ((Lp / 4) & 1) ? Lp : Lp + 4;  // odd number of float4 per row: fewer bank conflicts on the Y stores
    A.M = ctx->M;
    A.include_center = ctx->include_center;
    A.layout = layout;
    A.inv_delta = ctx->inv_delta;
    A.r_cut = (float)ctx->r_cut;
    A.width = (float)ctx->smooth_width;
    A.per_l = layout == RASCAL_LAYOUT_PACKED ? Q * (Q + 1) / 2 : Q * Q;
    A.ps_stride = (int64_t)L1 * A.per_l;
    A.wait_limit = ctx->wait_limit ? ctx->wait_limit : kTcWaitLimit;
    // accumulation tasks: (l, n tile, m tile) per species, ws warps per species, all species at once
    A.n_lmt = 0;
    for (int l = 0; l < L1; ++l) A.n_lmt += (2 * l + 1 + 3) / 4;
    A.n_tasks = (A.n_pad / 4) * A.n_lmt;
    A.ws = (A.n_tasks + 31) / 32;
    if (A.S * A.ws > kTcMaxGroupWarps) return RASCAL_E_UNSUPPORTED;
    A.nw = std::min(kTcMaxGroupWarps, std::max(A.S * A.ws, 8));
    // warps for the Y chains and for the radial values, by a rough instruction count of each per chunk
    const double yc = 4.0 * ctx->n_lm, rc = 25.0 * (16.0 + 8.0 * ((A.F_pad + 127) / 128));
    A.nyw = std::max(1, std::min(A.nw - 1, (int)(A.nw * yc / (yc + rc) + 0.5)));
    std::vector<double> load(A.nyw, 0.0);
    std::vector<int> ms(L1);
    for (int m = 0; m < L1; ++m) ms[m] = m;
    auto cost = [&](int m) { return m == 0 ? 4.0 * L1 : 7.0 * (L1 - m) + 4.0; };
    std::sort(ms.begin(), ms.end(), [&](int x, int y) { return cost(x) > cost(y); });
    for (int m : ms) {
        const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[w] += cost(m);
        A.ymask[w] |= 1u << m;
    }
    // operand tiles (K-major core matrices; rows Q..Qr-1 and the K padding stay zero)
    const bool tf32 = mode == kTcTf32x3;
    const int esz = tf32 ? 4 : 2, kstep = tf32 ? 8 : 16, e16 = 16 / esz;
    A.Qr = (Q + 7) / 8 * 8;
    // M = 64 when the rows fit (half the operand rows read per MMA); N a multiple of 8 (M = 64) or 16 (M = 128)
    A.M_mma = Q <= 64 ? 64 : 128;
    A.N_mma = A.M_mma == 64 ? std::max(8, (Q + 7) / 8 * 8) : std::max(16, (Q + 15) / 16 * 16);
    int off = 0, read_end = 0;
    for (int l = 0; l < L1; ++l) {
        const int kpad = (2 * l + 1 + kstep - 1) / kstep * kstep;
        A.nk[l] = kpad / kstep;
        A.sbo[l] = (kpad / e16) * kTcLbo;
        const int phase = (tc_lp(l) / 4) & 7;  // 16-byte phase of the tile start modulo 128 bytes
        off += ((phase - off / 16) % 8 + 8) % 8 * 16;
        A.tile_off[l] = off;
        read_end = std::max(read_end, off + (A.M_mma / 8) * A.sbo[l]);  // the MMA reads M / 8 groups of 8 rows
        off += (A.Qr / 8) * A.sbo[l];
        A.sc[l] = ctx->ps_norm ? (float)std::pow(2.0 * l + 1.0, -0.25) : 1.0f;
    }
    const int hi_bytes = (off + 1023) / 1024 * 1024;
    A.lo_off = tf32 ? hi_bytes : 0;
    A.ops_bytes = tf32 ? 2 * hi_bytes : hi_bytes;
    read_end += A.lo_off;
    // rounds: consecutive l whose accumulators fit one 256-column TMEM slot
    A.n_rounds = 0;
    int n_cmd = 0;
    for (int l = 0; l < L1;) {
        if (A.n_rounds >= kTcMaxRounds) return RASCAL_E_UNSUPPORTED;
        int cols = 0, h = l;
        const int stride = (A.N_mma + 15) / 16 * 16;  // the epilogue reads 16-column chunks
        while (h < L1 && cols + stride <= kTcSlotCols) {
            A.col_off[h] = cols;
            cols += stride;
            ++h;
        }
        A.r_cmd[A.n_rounds] = n_cmd;
        for (int x = l; x < h; ++x) n_cmd += A.nk[x];
        A.r_lo[A.n_rounds] = l;
        A.r_hi[A.n_rounds] = h - 1;
        ++A.n_rounds;
        l = h;
    }
    A.r_cmd[A.n_rounds] = n_cmd;
    if (n_cmd > kTcMaxCmds) return RASCAL_E_UNSUPPORTED;
    A.c_slot_floats = (Q * ctx->n_lm + 3 + 3) / 4 * 4;
    A.pair_bytes = (int)align_up(1024 + sizeof(float) * kTcChunk * (size_t)(A.F_pad + A.Ly), 128);
    A.c_off = 2 * A.ops_bytes;
    A.pair_off = (int)align_up((size_t)A.c_off + 2 * 4 * (size_t)A.c_slot_floats, 128);
    A.smem_bytes = A.pair_off + 2 * A.pair_bytes;
    A.smem_bytes = std::max(A.smem_bytes, A.ops_bytes + read_end);  // buffer 1's MMAs read up to here
    if (A.smem_bytes > 220 * 1024) return RASCAL_E_UNSUPPORTED;  // plus about 4 KB of static shared memory
    *smem = (size_t)A.smem_bytes;
    *threads = 32 * (kTcProd0 + 2 * A.nw);
    return RASCAL_OK;
}

template <int L>
static int tc_launch(rascal_ctx* ctx, int mode, const TcArgs& A, int grid, int threads, size_t smem) {
    if (mode == kTcTf32x3) k_soap_tc<L, kTcTf32x3><<<grid, threads, smem, ctx->stream>>>(A);
    else k_soap_tc<L, kTcBf16><<<grid, threads, smem, ctx->stream>>>(A);
    RASCAL_LAUNCH_CHECK("k_soap_tc");
    return RASCAL_OK;
}

// Fused expansion + tensor-core power spectrum; returns RASCAL_E_UNSUPPORTED (without touching the error message)
// when the hypers do not fit this kernel.
int soap_tc(rascal_ctx* ctx, const rascal_system* sys, const int64_t* d_offsets, const int* d_nbr_j, const float* d_rij,
            const float* pre_G, int precision, int layout, float* d_coeffs, float* d_ps) {
    const int mode = precision == RASCAL_PS_BF16 ? kTcBf16 : kTcTf32x3;
    TcArgs A;
    size_t smem;
    int threads;
    int st = tc_plan(ctx, mode, layout, A, &smem, &threads);
    if (st) return st;
    A.offsets = d_offsets;
    A.nbr_j = d_nbr_j;
    A.rij = reinterpret_cast<const float4*>(d_rij);
    A.species = sys->d_species;
    A.lut = ctx->d_lut;
    A.table = ctx->d_table_pad;
    A.pre_G = pre_G;
    A.fmap = ctx->d_fmap;
    A.coeffs = d_coeffs;
    A.ps = d_ps;
    A.flags = ctx->d_flags;
    A.N = sys->n_atoms;
    const int grid = std::min(sys->n_atoms, ctx->n_sm);
    switch (ctx->l_max) {
        case 6: return tc_launch<6>(ctx, mode, A, grid, threads, smem);
        case 8: return tc_launch<8>(ctx, mode, A, grid, threads, smem);
        case 9: return tc_launch<9>(ctx, mode, A, grid, threads, smem);
        default: return tc_launch<0>(ctx, mode, A, grid, threads, smem);
    }
}

}  // namespace rascal
