// FP32 per-l Gram of the power spectrum (Eq. nu2-basis-coupled in the real basis):
//   p_{q1 q2 l} = k_l sum_m C[q1][l m] C[q2][l m],   k_l = (2l+1)^-1/2 (or 1 without ps_norm)
// from one centre's coefficients held transposed in shared memory, CT[lm][q] with q = a n_max + n contiguous and
// rows padded to Qp (a multiple of 4; columns Q..Qp-1 are zero). A task is a 4 x 4 output tile (l, t1 <= t2);
// tasks are ordered by decreasing l and dealt round-robin to the CTA's threads.
#pragma once

#include "common.cuh"
#include "f32x2.cuh"

namespace rascal {

__device__ __host__ inline int64_t packed_index(int q1, int q2, int Q) {  // q1 <= q2
    return (int64_t)q1 * Q - (int64_t)q1 * (q1 - 1) / 2 + (q2 - q1);
}

// accumulates the tile with paired FMAs (fma.rn.f32x2): each product is rounded exactly as fmaf rounds it
__device__ inline void gram_tile_fp32(const float* __restrict__ CT, int Qp, int l, int t1, int t2, float (&acc)[4][4]) {
    const float* row = CT + l * l * Qp;
    uint64_t ap[4][2];
#pragma unroll
    for (int u = 0; u < 4; ++u) ap[u][0] = ap[u][1] = 0ull;
#pragma unroll 2
    for (int s = 0; s <= 2 * l; ++s, row += Qp) {
        const float4 a = *reinterpret_cast<const float4*>(row + 4 * t1);
        const float4 b = *reinterpret_cast<const float4*>(row + 4 * t2);
        const uint64_t b01 = f2_pack(b.x, b.y), b23 = f2_pack(b.z, b.w);
        const float aa[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t au = f2_pack(aa[u], aa[u]);
            ap[u][0] = f2_fma(au, b01, ap[u][0]);
            ap[u][1] = f2_fma(au, b23, ap[u][1]);
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        f2_unpack(ap[u][0], acc[u][0], acc[u][1]);
        f2_unpack(ap[u][1], acc[u][2], acc[u][3]);
    }
}

// writes k * tile into the l-block o (PACKED: q1 <= q2 only; FULL: both triangles)
__device__ inline void store_tile_fp32(float* __restrict__ o, int Q, int layout, int t1, int t2, float k,
                                       const float (&acc)[4][4]) {
    if (layout == RASCAL_LAYOUT_PACKED) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q1 = 4 * t1 + u;
            // entry (q1, q2) of the packed block sits at q1 (2Q - q1 - 1) / 2 + q2
            float* row = o + (q1 * (2 * Q - q1 - 1)) / 2 + 4 * t2;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int q2 = 4 * t2 + v;
                if (q1 <= q2 && q2 < Q) row[v] = k * acc[u][v];
            }
        }
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q1 = 4 * t1 + u;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int q2 = 4 * t2 + v;
                if (q1 < Q && q2 < Q) {
                    o[(int64_t)q1 * Q + q2] = k * acc[u][v];
                    if (t1 != t2) o[(int64_t)q2 * Q + q1] = k * acc[u][v];
                }
            }
        }
    }
}

// tasks: packed (l | t1 << 8 | t2 << 16); out points at this centre's p block
__device__ inline void ps_gram_fp32(const float* __restrict__ CT, int Qp, int Q, int l_max, int ps_norm,
                                    const int* __restrict__ tasks, int n_tasks, int layout, float* __restrict__ out) {
    const int64_t per_l = layout == RASCAL_LAYOUT_PACKED ? (int64_t)Q * (Q + 1) / 2 : (int64_t)Q * Q;
    for (int t = threadIdx.x; t < n_tasks; t += blockDim.x) {
        const int packed = __ldg(&tasks[t]);
        const int l = packed & 0xff, t1 = (packed >> 8) & 0xff, t2 = (packed >> 16) & 0xff;
        float acc[4][4];
        gram_tile_fp32(CT, Qp, l, t1, t2, acc);
        const float k = ps_norm ? rsqrtf((float)(2 * l + 1)) : 1.0f;
        store_tile_fp32(out + l * per_l, Q, layout, t1, t2, k, acc);
    }
    (void)l_max;
}

}  // namespace rascal
