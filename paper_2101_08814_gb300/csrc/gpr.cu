// Sparse GPR energy model with the polynomial kernel on the tcgen05 tensor cores (TF32 operands, FP32 accumulation):
//
//   E_i = sum_{I in M, a_I = a_i} x_I k_I(p_i),   k_I(p_i) = (p^_i . M^_I)^zeta              (Eq. sparse-gp)
//   dE_i/dp_i = (G_i - zeta E_i p^_i) / |p_i|,    G_i = sum_I x_I zeta k_(zeta-1) M^_I   (Eq. gpr-force-order)
//
// with p^ = p/|p| and M^ = M/|M| when the model normalises (else p^ = p, M^ = M and |p| = 1). The active set is
// summed first, as the paper orders the force contraction: G_i is one GEMM over the active set, and G_i . p^_i =
// zeta E_i needs no second pass over the features.
//
// Both contractions are dense GEMMs between the centres of one species and that species' sparse points, so the
// centres are first bucketed by species (k_gpr_count, k_gpr_scatter: a stable counting sort on the device).
//   k_gpr_kernel: D[128 centres][<= 512 sparse points] = p_rows . M^T over the features, A rows gathered from the
//     feature matrix by cp.async (16-byte copies, zero-filled past the end), B = M^ rows (TF32-rounded at model
//     creation); 5-stage shared-memory pipeline (kGprStages), one thread issues the MMAs, completion per stage on mbarriers.
//     Epilogue (TMEM -> registers): the row norms (accumulated from the staged A tiles), k^zeta, E partials and the
//     per-(centre, point) factor W = x zeta k^(zeta-1), stored for the gradient GEMM.
//   k_gpr_finish: per structure, E_i summed over the passes, FP64 structure energies, zeta E_i / |p_i|^2 (the
//     normalisation's share of the chain rule; 0 without normalisation).
//   k_gpr_grad: D[128 centres][256 features] = W . M^ over the active set, epilogue dE/dp = D / |p| - zeta E p / |p|^2.
// Operand tiles in shared memory are K-major with 64 bytes of K per row and stage, in the 64-byte swizzled layout
// (8-row atoms of 512 bytes): TMA writes it for the dense operands (the sparse points, W), the gathered feature
// rows are copied into it by cp.async.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "tcgen05.cuh"

struct rascal_gpr {
    int S;                                  // species of the context the model was built for
    int64_t F, Fk, Fn;                      // features; rounded up to 16 (K of the kernel GEMM, N of the gradient)
    int zeta, normalize;
    int n_sp[rascal::kMaxSpecies];          // sparse points per species
    int n_pad[rascal::kMaxSpecies];         // rounded up to 16
    int64_t row_off[rascal::kMaxSpecies];   // first row of a species in M and x
    int64_t t_off[rascal::kMaxSpecies];     // first element of a species' block [Fn][n_pad] in MT
    int n_pad_max, passes_max;
    int64_t rows;
    float* d_M;   // [rows][Fk]   M^ rows, TF32-rounded, zero-padded
    float* d_MT;  // per species [Fn][n_pad]: M^ transposed (K-major operand of the gradient GEMM)
    float* d_x;   // [rows] x_I (0 in the padding)
    CUtensorMap tmM;                          // TMA maps of d_M and of each species' block of d_MT
    CUtensorMap tmMT[rascal::kMaxSpecies];
};

namespace rascal {

constexpr int kGprThreads = 256;
constexpr int kGprStages = 5;               // kernel GEMM pipeline depth (40 KB per stage)
constexpr int kGprStages2 = 4;              // gradient GEMM (24 KB per stage, two CTAs per SM)
constexpr int kGprKB = 16;                   // K elements (TF32) per stage: 64 bytes per operand row
constexpr int kGprATile = 128 * 64;          // bytes of one A stage
constexpr int kGprB1 = 512 * 64;             // B stage of the kernel GEMM (up to 512 sparse points)
constexpr int kGprB2 = 256 * 64;             // B stage of the gradient GEMM (256 features)

struct GprArgs {
    int N, S;
    int64_t F, Fk, Fn;
    int zeta, normalize, vec16;
    const float* p;       // [N][F] features, atom order
    const int* perm;      // [N] atoms sorted by species (stable)
    const int* off;       // [S + 1] species offsets into perm
    const float* M;
    const float* MT;
    const float* x;
    int n_pad[kMaxSpecies];
    int64_t row_off[kMaxSpecies];
    int64_t t_off[kMaxSpecies];
    int n_pad_max, passes_max;
    float* e_part;        // [passes_max][N] energy partials per 512-point pass
    float* inv;           // [N] 1/|p_i| (1 without normalisation or for p_i = 0)
    float* W;             // [N sorted][n_pad_max] x zeta k^(zeta-1) (NULL: energies only)
    const float* c2;      // [N] zeta E_i / |p_i|^2
    float* grad;          // [N][F]
    unsigned* flags;
    CUtensorMap tmM;                   // M^ rows [rows][Fk], boxes 16 B x 64 rows
    CUtensorMap tmW;                   // W [N sorted][n_pad_max]
    CUtensorMap tmMT[kMaxSpecies];     // per species M^T [Fn][n_pad]
};


__device__ inline float ipow(float k, int e) {
    float r = 1.0f;
    for (int i = 0; i < e; ++i) r *= k;
    return r;
}

// tile t -> (species, first sorted row, index within the species' tiles); false when t is past the last tile
__device__ inline bool gpr_tile(const int* s_off, int S, const int* per_mtile, int64_t t, int& s, int& row0, int& sub) {
    for (s = 0; s < S; ++s) {
        const int rows = s_off[s + 1] - s_off[s];
        const int64_t n = (int64_t)((rows + 127) / 128) * per_mtile[s];
        if (t < n) {
            row0 = s_off[s] + (int)(t / per_mtile[s]) * 128;
            sub = (int)(t % per_mtile[s]);
            return true;
        }
        t -= n;
    }
    return false;
}

// Bounded-wait failure: flag it, let the tensor core and the copies finish, and stop.
__device__ inline void gpr_fail(const GprArgs& A, uint64_t* done, uint32_t phase) {
    if (threadIdx.x == 0) atomicOr(A.flags, kFlagTimeout);
    mbar_wait_bounded(done, phase);
    cp_async_wait_all();
}

// thread 0: TMA loads still in flight after a failure (k-blocks [from, to) of this CTA) are waited for
__device__ inline void gpr_drain_tma(uint64_t* full, int stages, int64_t from, int64_t to) {
    for (int64_t i = from; i < to; ++i) mbar_wait_bounded(&full[i % stages], (uint32_t)((i / stages) & 1));
}

// ------------------------------------------------------------------------------------------ kernel GEMM
// Warp-specialised pipeline: warps 0-3 gather A (feature rows of the tile's centres) by cp.async into the 64-byte
// swizzled layout and, once their own copies of a stage have landed, arrive on its `full` barrier; warp 4 loads B (the
// species' sparse points) by TMA onto the same barrier and issues the MMAs, which release the stage through `empty`.
// The row norms are accumulated by the A threads from their own chunks and reduced per tile.
constexpr int kGprProducers = 128;  // A-copy threads (warps 0-3)
constexpr int kGprLag = 3;          // k-blocks a producer keeps in flight before it waits for its oldest

template <bool VEC16>
__global__ void __launch_bounds__(kGprThreads, 1) k_gpr_kernel(const __grid_constant__ GprArgs A) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;                                        // [stages][8 KB]
    unsigned char* sB = sA + kGprStages * kGprATile;                 // [stages][32 KB]
    float* s_x = reinterpret_cast<float*>(sB + kGprStages * kGprB1);  // [512]
    float* s_inv = s_x + 512;                                        // [128]
    float* s_E = s_inv + 128;                                        // [2][128]; [4][128] norm partials before
    int* s_atom = reinterpret_cast<int*>(s_E + 512);                 // [128]
    int* s_off = s_atom + 128;                                       // [S + 1]
    int* s_per = s_off + kMaxSpecies + 1;                            // [S] passes per species
    uint64_t* bars = reinterpret_cast<uint64_t*>(s_per + kMaxSpecies + 1);  // [stages] empty, [stages] full, done
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 2 * kGprStages + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint64_t* empty = bars;
    uint64_t* full = bars + kGprStages;
    uint64_t* done = bars + 2 * kGprStages;

    for (int s = tid; s <= A.S; s += blockDim.x) s_off[s] = A.off[s];
    for (int s = tid; s < A.S; s += blockDim.x) s_per[s] = (A.n_pad[s] + 511) / 512;
    if (warp == 0) {
        tmem_alloc(s_tmem, 512);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < kGprStages; ++i) {
            mbar_init(&empty[i], 1);
            mbar_init(&full[i], kGprProducers + 1);
        }
        mbar_init(done, 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *s_tmem;
    const uint32_t a_base = smem_u32(sA), b_base = smem_u32(sB);
    int64_t g = 0;          // k-blocks of this CTA so far (stage = g % stages, use = g / stages)
    int64_t g_tma = 0;      // warp 4: k-blocks whose B load was issued
    int64_t g_full = 0;     // warp 4: k-blocks whose stage it has seen full
    uint32_t done_phase = 0;
    bool ok = true;

    for (int64_t t = blockIdx.x;; t += gridDim.x) {
        int s, row0, pass;
        if (!gpr_tile(s_off, A.S, s_per, t, s, row0, pass)) break;
        const int n_rows = min(128, s_off[s + 1] - row0);
        const int col0 = pass * 512;
        const int ncols = min(512, A.n_pad[s] - col0);
        const int nk = (int)(A.Fk / kGprKB);
        if (tid < 128) s_atom[tid] = tid < n_rows ? A.perm[row0 + tid] : -1;
        for (int c = tid; c < 512; c += blockDim.x) s_x[c] = c < ncols ? A.x[A.row_off[s] + col0 + c] : 0.0f;
        __syncthreads();

        if (warp < 4) {
            // ---- A producers: rows r0 + 32 j (j < 4), 16-byte chunk c
            const int r0 = tid >> 2, c = tid & 3;
            const uint32_t d0 = sw64_off(r0, c);  // row r0 + 32 j lands 2048 j bytes further
            const float* pa[4];
            int64_t lim[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int atom = s_atom[r0 + 32 * j];
                pa[j] = atom >= 0 ? A.p + (int64_t)atom * A.F : A.p;
                lim[j] = atom >= 0 ? A.F : 0;
            }
            float nrm[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            auto land = [&](int kb) {  // this thread's chunks of k-block kb are in shared memory: norms, arrive
                const unsigned char* a = sA + (int)((g + kb) % kGprStages) * kGprATile + d0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float4 v = *reinterpret_cast<const float4*>(a + 2048 * j);
                    nrm[j] = fmaf(v.x, v.x, nrm[j]);
                    nrm[j] = fmaf(v.y, v.y, nrm[j]);
                    nrm[j] = fmaf(v.z, v.z, nrm[j]);
                    nrm[j] = fmaf(v.w, v.w, nrm[j]);
                }
                mbar_arrive(&full[(g + kb) % kGprStages]);
            };
            int landed = 0;
            for (int kb = 0; kb < nk && ok; ++kb) {
                const int64_t gi = g + kb;
                const int stage = (int)(gi % kGprStages);
                if (gi >= kGprStages &&
                    !mbar_wait_bounded(&empty[stage], (uint32_t)(((gi - kGprStages) / kGprStages) & 1))) {
                    ok = false;
                    break;
                }
                const int64_t k0 = (int64_t)kb * kGprKB;
                unsigned char* a = sA + stage * kGprATile + d0;
                if (VEC16) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const bool in = k0 + 4 * c < lim[j];
                        cp_async16_zfill(a + 2048 * j, in ? pa[j] + k0 + 4 * c : A.p, in ? 16u : 0u);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const bool in = k0 + 4 * c + e < lim[j];
                            cp_async4_zfill(a + 2048 * j + 4 * e, in ? pa[j] + k0 + 4 * c + e : A.p, in ? 4u : 0u);
                        }
                }
                cp_async_commit();
                if (kb >= kGprLag) {
                    cp_async_wait_group<kGprLag>();
                    fence_proxy_async_smem();
                    land(landed++);
                }
            }
            cp_async_wait_group<0>();
            fence_proxy_async_smem();
            while (ok && landed < nk) land(landed++);
#pragma unroll
            for (int j = 0; j < 4; ++j) s_E[c * 128 + r0 + 32 * j] = nrm[j];  // partials [chunk][row]
        } else if (warp == 4) {
          if (lane == 0) {
            // ---- B loads and MMAs
            const int n0 = min(256, ncols), n1 = ncols - n0;
            const int nq = (ncols + 63) / 64;
            const int brow = (int)(A.row_off[s] + col0);
            const uint32_t id0 = instr_desc(2u, 128u, (uint32_t)n0);
            const uint32_t id1 = instr_desc(2u, 128u, (uint32_t)max(n1, 16));
            auto load_b = [&](int kb) {
                const int stage = (int)((g + kb) % kGprStages);
                unsigned char* b = sB + stage * kGprB1;
                mbar_expect_tx(&full[stage], (uint32_t)(nq * 4096));
                for (int qq = 0; qq < nq; ++qq)
                    tma_load_2d(b + qq * 4096, &A.tmM, kb * kGprKB, brow + 64 * qq, &full[stage]);
                ++g_tma;
            };
            for (int i = 0; i < kGprStages - 1 && i < nk; ++i) load_b(i);
            for (int kb = 0; kb < nk; ++kb) {
                const int64_t gi = g + kb;
                const int stage = (int)(gi % kGprStages);
                if (!mbar_wait_bounded(&full[stage], (uint32_t)((gi / kGprStages) & 1))) {
                    ok = false;
                    break;
                }
                ++g_full;
                tc_fence_after();
                const uint32_t a0 = a_base + stage * kGprATile, b0 = b_base + stage * kGprB1;
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                    const uint64_t da = smem_desc_sw64(a0 + kk * 32, 512);
                    mma_tf32_ss(taddr, da, smem_desc_sw64(b0 + kk * 32, 512), id0, (kb | kk) != 0);
                    if (n1 > 0) mma_tf32_ss(taddr + 256, da, smem_desc_sw64(b0 + 16384 + kk * 32, 512), id1, (kb | kk) != 0);
                }
                mma_commit(&empty[stage]);
                const int nxt = kb + kGprStages - 1;
                if (nxt < nk) {
                    if (gi >= 1 && !mbar_wait_bounded(&empty[(gi - 1) % kGprStages], (uint32_t)(((gi - 1) / kGprStages) & 1))) {
                        ok = false;
                        break;
                    }
                    load_b(nxt);
                }
            }
            mma_commit(done);
          }
          __syncwarp();  // the other lanes of the MMA warp wait here, not in a spin beside lane 0
        }
        g += nk;
        const bool fin = mbar_wait_bounded(done, done_phase);
        done_phase ^= 1u;
        ok = __syncthreads_and(ok && fin) != 0;
        if (!ok) {
            if (warp == 4 && lane == 0) gpr_drain_tma(full, kGprStages, g_full, g_tma);
            gpr_fail(A, done, done_phase ^ 1u);
            break;
        }
        if (tid < 128) {
            const float nn = s_E[tid] + s_E[128 + tid] + s_E[256 + tid] + s_E[384 + tid];
            const float iv = (A.normalize && nn > 0.0f) ? 1.0f / sqrtf(nn) : 1.0f;
            s_inv[tid] = iv;
            if (pass == 0 && s_atom[tid] >= 0) A.inv[s_atom[tid]] = iv;
        }
        __syncthreads();
        tc_fence_after();
        // epilogue: warp -> lane quadrant (rows) and column half
        const int q = warp & 3, h = warp >> 2, row = 32 * q + lane;
        const float iv = s_inv[row];
        float e = 0.0f;
        const int c_end = min(ncols, 256 * h + 256);
        float* wrow = A.W ? A.W + (int64_t)(row0 + row) * A.n_pad_max + col0 : nullptr;
        const bool valid = row < n_rows;
        for (int cc = 256 * h; cc < c_end; cc += 16) {
            float v[16];
            tmem_ld16(taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)cc, v);
            float w[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const float k = v[u] * iv;
                const float kz1 = ipow(k, A.zeta - 1);
                const float xv = s_x[cc + u];
                e = fmaf(xv * kz1, k, e);
                w[u] = xv * (float)A.zeta * kz1;
            }
            if (wrow && valid) {
#pragma unroll
                for (int u = 0; u < 16; u += 4)
                    *reinterpret_cast<float4*>(wrow + cc + u) = make_float4(w[u], w[u + 1], w[u + 2], w[u + 3]);
            }
        }
        __syncthreads();  // the norm partials in s_E are read; the energies may reuse it
        s_E[h * 128 + row] = e;
        tc_fence_before();
        __syncthreads();
        if (tid < 128 && s_atom[tid] >= 0) A.e_part[(int64_t)pass * A.N + s_atom[tid]] = s_E[tid] + s_E[128 + tid];
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(taddr, 512);
    }
}

// ---------------------------------------------------------------------------------------- gradient GEMM
// Both operands by TMA: A = W rows [chunk][128 rows][16 B], B = the species' M^T rows [chunk][256 rows][16 B]; one
// thread runs the whole main loop (loads, MMAs, stage recycling); all warps share the epilogue.
__global__ void __launch_bounds__(kGprThreads, 2) k_gpr_grad(const __grid_constant__ GprArgs A) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;                                          // [stages][8 KB]
    unsigned char* sB = sA + kGprStages2 * kGprATile;                  // [stages][16 KB]
    int* s_atom = reinterpret_cast<int*>(sB + kGprStages2 * kGprB2);  // [128]
    int* s_off = s_atom + 128;
    int* s_per = s_off + kMaxSpecies + 1;                              // feature chunks per species
    uint64_t* bars = reinterpret_cast<uint64_t*>(s_per + kMaxSpecies + 1);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 2 * kGprStages2 + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint64_t* empty = bars;
    uint64_t* full = bars + kGprStages2;
    uint64_t* done = bars + 2 * kGprStages2;
    const int n_fc = (int)((A.Fn + 255) / 256);

    for (int s = tid; s <= A.S; s += blockDim.x) s_off[s] = A.off[s];
    for (int s = tid; s < A.S; s += blockDim.x) s_per[s] = n_fc;
    if (warp == 0) {
        tmem_alloc(s_tmem, 256);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i <= 2 * kGprStages2; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *s_tmem;
    const uint32_t a_base = smem_u32(sA), b_base = smem_u32(sB);
    int64_t g = 0;
    uint32_t done_phase = 0;
    bool ok = true;

    for (int64_t t = blockIdx.x;; t += gridDim.x) {
        int s, row0, fc;
        if (!gpr_tile(s_off, A.S, s_per, t, s, row0, fc)) break;
        const int n_rows = min(128, s_off[s + 1] - row0);
        const int f0 = fc * 256;
        const int ncols = (int)(A.Fn - f0 < 256 ? A.Fn - f0 : 256);
        const int nk = A.n_pad[s] / kGprKB;
        const int nq = (ncols + 63) / 64;
        if (tid < 128) s_atom[tid] = tid < n_rows ? A.perm[row0 + tid] : -1;
        if (nk > 0) {
            if (tid == 0) {
                const CUtensorMap* tb = &A.tmMT[s];
                auto load = [&](int kb, int stage) {
                    const int k0 = kb * kGprKB;
                    unsigned char* a = sA + stage * kGprATile;
                    unsigned char* b = sB + stage * kGprB2;
                    mbar_expect_tx(&full[stage], (uint32_t)(2 * 4096 + nq * 4096));
                    for (int qq = 0; qq < 2; ++qq) tma_load_2d(a + qq * 4096, &A.tmW, k0, row0 + 64 * qq, &full[stage]);
                    for (int qq = 0; qq < nq; ++qq) tma_load_2d(b + qq * 4096, tb, k0, f0 + 64 * qq, &full[stage]);
                };
                const uint32_t id = instr_desc(2u, 128u, (uint32_t)ncols);
                int issued = 0;
                for (int i = 0; i < kGprStages2 - 1 && i < nk; ++i, ++issued) load(i, (int)((g + i) % kGprStages2));
                int kb = 0;
                for (; kb < nk; ++kb) {
                    const int64_t gi = g + kb;
                    const int stage = (int)(gi % kGprStages2);
                    if (!mbar_wait_bounded(&full[stage], (uint32_t)((gi / kGprStages2) & 1))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = a_base + stage * kGprATile, b0 = b_base + stage * kGprB2;
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk)
                        mma_tf32_ss(taddr, smem_desc_sw64(a0 + kk * 32, 512), smem_desc_sw64(b0 + kk * 32, 512), id,
                                    (kb | kk) != 0);
                    mma_commit(&empty[stage]);
                    const int nxt = kb + kGprStages2 - 1;
                    if (nxt < nk) {
                        const int64_t prev = gi - 1;
                        if (prev >= 0 &&
                            !mbar_wait_bounded(&empty[prev % kGprStages2], (uint32_t)((prev / kGprStages2) & 1))) {
                            ok = false;
                            ++kb;
                            break;
                        }
                        load(nxt, (int)((g + nxt) % kGprStages2));
                        ++issued;
                    }
                }
                mma_commit(done);
                if (!ok) gpr_drain_tma(full, kGprStages2, g + kb, g + issued);
            }
            if (warp == 0) __syncwarp();
            g += nk;
            const bool fin = mbar_wait_bounded(done, done_phase);
            done_phase ^= 1u;
            ok = __syncthreads_and(ok && fin) != 0;
            if (!ok) {
                gpr_fail(A, done, done_phase ^ 1u);
                break;
            }
            tc_fence_after();
        } else {
            __syncthreads();
        }
        // epilogue: dE/dp = inv * G - c2 * p for this warp's rows and half of the columns
        const int q = warp & 3, h = warp >> 2, row = 32 * q + lane;
        const int atom = s_atom[row];
        const float iv = atom >= 0 && nk > 0 ? A.inv[atom] : 0.0f;
        const float cc = atom >= 0 && nk > 0 ? A.c2[atom] : 0.0f;
        const int c_end = min(ncols, 128 * h + 128);
        // the feature values of the next 16 columns are requested before this group's are used (latency overlap)
        const float* pbase = atom >= 0 ? A.p + (int64_t)atom * A.F : A.p;
        auto fetch = [&](int c, float4 (&pv)[4]) {
            const int64_t f = f0 + c;
            if (atom >= 0 && A.vec16 && f + 16 <= A.F) {
#pragma unroll
                for (int u = 0; u < 4; ++u) pv[u] = __ldg(reinterpret_cast<const float4*>(pbase + f) + u);
            }
        };
        float4 pn[4];
        if (128 * h < c_end) fetch(128 * h, pn);
        for (int c = 128 * h; c < c_end; c += 16) {
            float4 pc[4] = {pn[0], pn[1], pn[2], pn[3]};
            if (c + 16 < c_end) fetch(c + 16, pn);
            float v[16];
            if (nk > 0) {
                tmem_ld16(taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)c, v);
            } else {
#pragma unroll
                for (int u = 0; u < 16; ++u) v[u] = 0.0f;
            }
            if (atom < 0) continue;
            const int64_t f = f0 + c;
            const float* prow = A.p + (int64_t)atom * A.F + f;
            float* grow = A.grad + (int64_t)atom * A.F + f;
            if (A.vec16 && f + 16 <= A.F) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    float4 o;
                    o.x = fmaf(iv, v[4 * u], -cc * pc[u].x);
                    o.y = fmaf(iv, v[4 * u + 1], -cc * pc[u].y);
                    o.z = fmaf(iv, v[4 * u + 2], -cc * pc[u].z);
                    o.w = fmaf(iv, v[4 * u + 3], -cc * pc[u].w);
                    __stcs(reinterpret_cast<float4*>(grow) + u, o);
                }
            } else {
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    if (f + u < A.F) grow[u] = fmaf(iv, v[u], -cc * prow[u]);
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(taddr, 256);
    }
}

// --------------------------------------------------------------------------------------- species buckets
constexpr int kSortBlock = 1024;

__global__ void k_gpr_count(int N, int S, const int* __restrict__ species, const int* __restrict__ lut, int* cnt) {
    __shared__ int c[kMaxSpecies];
    if (threadIdx.x < S) c[threadIdx.x] = 0;
    __syncthreads();
    const int i = blockIdx.x * kSortBlock + threadIdx.x;
    if (i < N) {
        const int lab = species[i];
        const int a = (lab >= 0 && lab < 256) ? lut[lab] : -1;
        if (a >= 0) atomicAdd(&c[a], 1);
    }
    __syncthreads();
    if (threadIdx.x < S) cnt[blockIdx.x * S + threadIdx.x] = c[threadIdx.x];
}

// stable scatter of the atoms into per-species buckets; block 0 also writes the species offsets
__global__ void k_gpr_scatter(int N, int S, const int* __restrict__ species, const int* __restrict__ lut,
                              const int* __restrict__ cnt, int* perm, int* off) {
    __shared__ int base[kMaxSpecies];
    __shared__ int wc[kSortBlock / 32][kMaxSpecies];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nb = gridDim.x;
    if (tid < S) {
        int before = 0, total_lower = 0;
        for (int b = 0; b < nb; ++b) {
            const int* row = cnt + b * S;
            if (b < (int)blockIdx.x) before += row[tid];
            for (int s2 = 0; s2 < tid; ++s2) total_lower += row[s2];
        }
        base[tid] = total_lower + before;
        if (blockIdx.x == 0) {
            off[tid] = total_lower;
            if (tid == S - 1) {
                int tot = 0;
                for (int b = 0; b < nb; ++b)
                    for (int s2 = 0; s2 < S; ++s2) tot += cnt[b * S + s2];
                off[S] = tot;
            }
        }
    }
    for (int s2 = lane; s2 < kMaxSpecies; s2 += 32) wc[warp][s2] = 0;
    __syncthreads();
    const int i = blockIdx.x * kSortBlock + tid;
    int a = -1;
    if (i < N) {
        const int lab = species[i];
        a = (lab >= 0 && lab < 256) ? lut[lab] : -1;
    }
    const unsigned same = __match_any_sync(0xffffffffu, a);
    const int rank = __popc(same & ((1u << lane) - 1u));
    if (a >= 0 && rank == 0) wc[warp][a] = __popc(same);
    __syncthreads();
    if (a >= 0) {
        int pos = base[a] + rank;
        for (int w = 0; w < warp; ++w) pos += wc[w][a];
        perm[pos] = i;
    }
}

// per structure: E_i over the passes, zeta E_i / |p_i|^2, and the FP64 structure sum
__global__ void k_gpr_finish(int N, int S, int passes_max, const int* __restrict__ struct_off,
                             const int* __restrict__ species, const int* __restrict__ lut, const int* __restrict__ npass,
                             const float* __restrict__ e_part, const float* __restrict__ inv, int zeta, int normalize,
                             float* atomic, float* c2, double* energy) {
    __shared__ double red[32];
    const int st = blockIdx.x;
    const int i0 = struct_off[st], i1 = struct_off[st + 1];
    double acc = 0.0;
    for (int i = i0 + (int)threadIdx.x; i < i1; i += blockDim.x) {
        const int lab = species[i];
        const int a = (lab >= 0 && lab < 256) ? lut[lab] : -1;
        const int np = a >= 0 ? npass[a] : 0;
        float e = 0.0f;
        for (int k = 0; k < np; ++k) e += e_part[(int64_t)k * N + i];
        if (atomic) atomic[i] = e;
        if (c2) c2[i] = (np > 0 && normalize) ? (float)zeta * e * inv[i] * inv[i] : 0.0f;
        acc += (double)e;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0 && energy) energy[st] = v;
    }
    (void)S;
    (void)passes_max;
}

static size_t gpr_smem1() {
    return (size_t)kGprStages * (kGprATile + kGprB1) + sizeof(float) * (512 + 128 + 512) + sizeof(int) * 128 +
           sizeof(int) * 2 * (kMaxSpecies + 1) + sizeof(uint64_t) * (2 * kGprStages + 1) + 16;
}
static size_t gpr_smem2() {
    return (size_t)kGprStages2 * (kGprATile + kGprB2) + sizeof(int) * 128 + sizeof(int) * 2 * (kMaxSpecies + 1) +
           sizeof(uint64_t) * (2 * kGprStages2 + 1) + 16;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// TMA map of a row-major FP32 matrix [rows][pitch] (cols used), boxes of 16 elements (64 bytes) x 64 rows written
// with 64-byte swizzling (the operand layout of smem_desc_sw64); reads past the last row fill zeros
static int tmap_2d(CUtensorMap* m, const float* base, uint64_t cols, uint64_t rows, uint64_t pitch) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return set_error(RASCAL_E_CUDA, "cuTensorMapEncodeTiled is not available from the CUDA driver library");
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {pitch * sizeof(float)};
    cuuint32_t box[2] = {16, 64};
    cuuint32_t es[2] = {1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(RASCAL_E_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return RASCAL_OK;
}

// round to the nearest TF32 value (10 explicit mantissa bits), ties to even
static float tf32_round(float v) {
    uint32_t u;
    std::memcpy(&u, &v, 4);
    if ((u & 0x7F800000u) != 0x7F800000u) {
        u += 0xFFFu + ((u >> 13) & 1u);
        u &= ~0x1FFFu;
    }
    std::memcpy(&v, &u, 4);
    return v;
}

}  // namespace rascal

using namespace rascal;

extern "C" int rascal_gpr_create(rascal_ctx* ctx, int64_t n_sparse, int64_t n_features, const double* h_sparse,
                                 const int* h_sparse_species, const double* h_weights, int zeta, int normalize,
                                 rascal_gpr** out) {
    clear_error();
    if (!ctx || !out) return set_error(RASCAL_E_ARG, "NULL context or output pointer");
    *out = nullptr;
    if (n_sparse < 0 || n_features < 1) return set_error(RASCAL_E_ARG, "n_sparse must be >= 0 and n_features >= 1");
    if (n_sparse > 0 && (!h_sparse || !h_sparse_species || !h_weights)) return set_error(RASCAL_E_ARG, "NULL host pointer");
    if (zeta < 1 || zeta > 16) return set_error(RASCAL_E_ARG, "zeta must be in [1, 16]");
    const int S = ctx->n_species;
    std::vector<std::vector<int64_t>> rows(S);
    for (int64_t I = 0; I < n_sparse; ++I) {
        int a = -1;
        for (int s = 0; s < S; ++s)
            if (ctx->species[s] == h_sparse_species[I]) a = s;
        if (a < 0) return set_error(RASCAL_E_ARG, "sparse point %lld has species %d, not one of the context's",
                                    (long long)I, h_sparse_species[I]);
        rows[a].push_back(I);
    }
    rascal_gpr* m = new rascal_gpr();
    std::memset(m, 0, sizeof(*m));
    m->S = S;
    m->F = n_features;
    m->Fk = (n_features + 15) / 16 * 16;
    m->Fn = m->Fk;
    m->zeta = zeta;
    m->normalize = normalize ? 1 : 0;
    int64_t r = 0, t = 0;
    for (int s = 0; s < S; ++s) {
        m->n_sp[s] = (int)rows[s].size();
        m->n_pad[s] = (m->n_sp[s] + 15) / 16 * 16;
        m->row_off[s] = r;
        m->t_off[s] = t;
        r += m->n_pad[s];
        t += m->Fn * m->n_pad[s];
        m->n_pad_max = std::max(m->n_pad_max, m->n_pad[s]);
        m->passes_max = std::max(m->passes_max, (m->n_pad[s] + 511) / 512);
    }
    m->rows = r;
    std::vector<float> hM((size_t)std::max<int64_t>(r, 1) * m->Fk, 0.0f), hMT((size_t)std::max<int64_t>(t, 1), 0.0f),
        hx((size_t)std::max<int64_t>(r, 1), 0.0f);
    for (int s = 0; s < S; ++s) {
        for (int k = 0; k < m->n_sp[s]; ++k) {
            const int64_t I = rows[s][k];
            const double* src = h_sparse + I * n_features;
            double nn = 0.0;
            for (int64_t f = 0; f < n_features; ++f) nn += src[f] * src[f];
            const double sc = (m->normalize && nn > 0.0) ? 1.0 / std::sqrt(nn) : 1.0;
            const int64_t row = m->row_off[s] + k;
            for (int64_t f = 0; f < n_features; ++f) {
                const float v = tf32_round((float)(src[f] * sc));
                hM[(size_t)(row * m->Fk + f)] = v;
                hMT[(size_t)(m->t_off[s] + f * m->n_pad[s] + k)] = v;
            }
            hx[(size_t)row] = (float)h_weights[I];
        }
    }
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&m->d_M, sizeof(float) * hM.size());
    if (e == cudaSuccess) e = cudaMalloc(&m->d_MT, sizeof(float) * hMT.size());
    if (e == cudaSuccess) e = cudaMalloc(&m->d_x, sizeof(float) * hx.size());
    if (e == cudaSuccess) e = cudaMemcpy(m->d_M, hM.data(), sizeof(float) * hM.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_MT, hMT.data(), sizeof(float) * hMT.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_x, hx.data(), sizeof(float) * hx.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gpr_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gpr_smem1());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gpr_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gpr_smem1());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gpr_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gpr_smem2());
    if (e != cudaSuccess) {
        cudaFree(m->d_M);
        cudaFree(m->d_MT);
        cudaFree(m->d_x);
        delete m;
        return set_error(RASCAL_E_CUDA, "GPR model upload: %s", cudaGetErrorString(e));
    }
    int st = RASCAL_OK;
    if (m->rows > 0) st = tmap_2d(&m->tmM, m->d_M, (uint64_t)m->Fk, (uint64_t)m->rows, (uint64_t)m->Fk);
    for (int s = 0; s < S && !st; ++s)
        if (m->n_pad[s] > 0)
            st = tmap_2d(&m->tmMT[s], m->d_MT + m->t_off[s], (uint64_t)m->n_pad[s], (uint64_t)m->Fn, (uint64_t)m->n_pad[s]);
    if (st) {
        rascal_gpr_destroy(m);
        return st;
    }
    *out = m;
    return RASCAL_OK;
}

extern "C" void rascal_gpr_destroy(rascal_gpr* m) {
    if (!m) return;
    cudaFree(m->d_M);
    cudaFree(m->d_MT);
    cudaFree(m->d_x);
    delete m;
}

extern "C" int rascal_gpr_predict(rascal_ctx* ctx, const rascal_gpr* m, const rascal_system* sys, const float* d_features,
                                  float* d_atomic, double* d_energy, float* d_grad) {
    clear_error();
    if (!ctx || !m) return set_error(RASCAL_E_ARG, "NULL context or model");
    if (m->S != ctx->n_species) return set_error(RASCAL_E_ARG, "model built for another species list");
    int st = validate_system(ctx, sys);
    if (st) return st;
    const int N = sys->n_atoms;
    if (d_energy) RASCAL_CUDA(cudaMemsetAsync(d_energy, 0, sizeof(double) * sys->n_structures, ctx->stream));
    if (N == 0) return RASCAL_OK;
    if (!d_features) return set_error(RASCAL_E_ARG, "NULL features");
    const int S = m->S;
    const int nb = (int)div_up(N, kSortBlock);
    const bool grad = d_grad != nullptr;
    const int P = std::max(1, m->passes_max);
    void* base;
    st = arena_get(ctx->scratch, carve_bytes(sizeof(int) * N, sizeof(int) * nb * S, sizeof(int) * (S + 1),
                                             sizeof(int) * S, sizeof(float) * N, sizeof(float) * (size_t)P * N,
                                             sizeof(float) * N, sizeof(float) * N,
                                             grad ? sizeof(float) * (size_t)N * std::max(16, m->n_pad_max) : 16),
                   &base);
    if (st) return st;
    Carver cv(base);
    int* perm = cv.take<int>(N);
    int* cnt = cv.take<int>((size_t)nb * S);
    int* off = cv.take<int>(S + 1);
    int* npass = cv.take<int>(S);
    float* inv = cv.take<float>(N);
    float* e_part = cv.take<float>((size_t)P * N);
    float* atomic = d_atomic ? d_atomic : cv.take<float>(N);
    if (d_atomic) cv.take<float>(N);
    float* c2 = cv.take<float>(N);
    float* W = grad ? cv.take<float>((size_t)N * std::max(16, m->n_pad_max)) : nullptr;

    int hp[kMaxSpecies];
    for (int s = 0; s < S; ++s) hp[s] = (m->n_pad[s] + 511) / 512;
    RASCAL_CUDA(cudaMemcpyAsync(npass, hp, sizeof(int) * S, cudaMemcpyHostToDevice, ctx->stream));
    k_gpr_count<<<nb, kSortBlock, 0, ctx->stream>>>(N, S, sys->d_species, ctx->d_lut, cnt);
    RASCAL_LAUNCH_CHECK("k_gpr_count");
    k_gpr_scatter<<<nb, kSortBlock, 0, ctx->stream>>>(N, S, sys->d_species, ctx->d_lut, cnt, perm, off);
    RASCAL_LAUNCH_CHECK("k_gpr_scatter");

    GprArgs A;
    std::memset(&A, 0, sizeof(A));
    A.N = N;
    A.S = S;
    A.F = m->F;
    A.Fk = m->Fk;
    A.Fn = m->Fn;
    A.zeta = m->zeta;
    A.normalize = m->normalize;
    A.vec16 = (m->F % 4 == 0) && ((reinterpret_cast<uintptr_t>(d_features) & 15) == 0) &&
              (!grad || (reinterpret_cast<uintptr_t>(d_grad) & 15) == 0);
    A.p = d_features;
    A.perm = perm;
    A.off = off;
    A.M = m->d_M;
    A.MT = m->d_MT;
    A.x = m->d_x;
    for (int s = 0; s < S; ++s) {
        A.n_pad[s] = m->n_pad[s];
        A.row_off[s] = m->row_off[s];
        A.t_off[s] = m->t_off[s];
    }
    A.n_pad_max = std::max(16, m->n_pad_max);
    A.passes_max = P;
    A.e_part = e_part;
    A.inv = inv;
    A.W = W;
    A.c2 = c2;
    A.grad = d_grad;
    A.flags = ctx->d_flags;
    A.tmM = m->tmM;
    for (int s = 0; s < S; ++s) A.tmMT[s] = m->tmMT[s];
    if (grad && (st = tmap_2d(&A.tmW, W, (uint64_t)A.n_pad_max, (uint64_t)N, (uint64_t)A.n_pad_max))) return st;
    if (m->rows > 0) {
        if (A.vec16)
            k_gpr_kernel<true><<<ctx->n_sm, kGprThreads, gpr_smem1(), ctx->stream>>>(A);
        else
            k_gpr_kernel<false><<<ctx->n_sm, kGprThreads, gpr_smem1(), ctx->stream>>>(A);
        RASCAL_LAUNCH_CHECK("k_gpr_kernel");
    }
    k_gpr_finish<<<sys->n_structures, 256, 0, ctx->stream>>>(N, S, P, sys->d_struct_offsets, sys->d_species, ctx->d_lut,
                                                             npass, e_part, inv, m->zeta, m->normalize, atomic,
                                                             grad ? c2 : nullptr,
                                                             d_energy);
    RASCAL_LAUNCH_CHECK("k_gpr_finish");
    if (grad) {
        k_gpr_grad<<<2 * ctx->n_sm, kGprThreads, gpr_smem2(), ctx->stream>>>(A);
        RASCAL_LAUNCH_CHECK("k_gpr_grad");
    }
    return RASCAL_OK;
}
