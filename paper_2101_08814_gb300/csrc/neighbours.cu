// Periodic cell-list neighbour search (Appendix B: every j, including periodic replicas, with r_ji < r_cut).
//
// Pipeline (all on the context stream):
//   k_struct_setup      per structure: inverse cell, perpendicular widths, bins >= r_cut(1+1e-6) wide per axis
//   k_atom_bin          per atom: fractional coordinates, wrap count w, bin, wrapped position p = r - w H split
//                       into FP32 hi + lo parts, counting-sort rank within the bin
//   k_atom_scatter      bin-sorted FP32 positions (float4: x, y, z, atom index)
//   k_struct_thresholds per structure: FP32 classification radii r_cut -+ delta from a rounding-error bound
//   k_pairs<count>      one warp per centre walks the stencil of bins; counts accepted pairs
//   scan                CSR offsets
//   k_pairs<fill>       same walk; accepted (j, n) keys and r_ji vectors staged in shared memory, rank-sorted by
//                       (j, n1, n2, n3) and written to the centre's CSR segment
//
// Bit-exactness with the FP64 definition: a candidate is classified in FP32 from the hi parts. The FP32 error of
// the displacement is bounded by 3.6e-7 (|p_i|_1 + |p_j|_1 + sum_k |t_k| |h_k|_1); with a 5x margin this gives
// delta, and only candidates with |d| within delta of r_cut (a few per million) are re-tested with the FP64
// formula d = (r_j - r_i) + ((n1 h1 + n2 h2) + n3 h3), d.d = (dx dx + dy dy) + dz dz < r_cut r_cut, each
// operation rounded on its own (__dadd_rn / __dmul_rn, no contraction). The output vector r_ji is computed in
// double-single arithmetic (error-free FP32 transforms) and rounded once to FP32.
#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace rascal {

struct StructInfo {
    double H[9];     // rows h1, h2, h3
    double Hinv[9];  // s = r Hinv (row vectors)
    float hhi[9], hlo[9];
    int nb[3], reach[3], pbc[3];
    int atom_begin, atom_end;
    float thr_lo2, thr_hi2, thr_tiny2;
    unsigned amax_bits;  // max over atoms of |p_hi|_1, as float bits
};

constexpr int kPairWarps = 4;     // warps per block in k_pairs
constexpr int kPairCap = 128;     // pairs a warp sorts in shared memory; larger segments use global scratch
constexpr int kNoallocCap = 256;  // the same for rascal_neighbours_noalloc, which has no overflow scratch

__device__ inline int floordiv(int a, int b) {
    const int q = a / b;
    return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

__global__ void k_struct_setup(int n_s, int n_atoms, const int* __restrict__ offs, const double* __restrict__ cells,
                               const int* __restrict__ pbc, double r_cut, StructInfo* info, int* nbins_out,
                               unsigned* flags) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_s) return;
    StructInfo& S = info[s];
    for (int k = 0; k < 9; ++k) {
        S.H[k] = cells[9 * s + k];
        S.hhi[k] = (float)S.H[k];
        S.hlo[k] = (float)(S.H[k] - (double)S.hhi[k]);
    }
    const int a = offs[s], b = offs[s + 1];
    const bool bad_offsets = (a < 0 || b < a || b > n_atoms);
    if (bad_offsets) atomicOr(flags, kFlagBadOffsets);
    S.atom_begin = a;
    S.atom_end = b;
    S.amax_bits = 0u;
    const double* h0 = S.H;
    const double* h1 = S.H + 3;
    const double* h2 = S.H + 6;
    double cr[3][3];  // cr[k] = h_{k+1} x h_{k+2}
    const double* hs[3] = {h0, h1, h2};
    for (int k = 0; k < 3; ++k) {
        const double* u = hs[(k + 1) % 3];
        const double* v = hs[(k + 2) % 3];
        cr[k][0] = u[1] * v[2] - u[2] * v[1];
        cr[k][1] = u[2] * v[0] - u[0] * v[2];
        cr[k][2] = u[0] * v[1] - u[1] * v[0];
    }
    const double det = h0[0] * cr[0][0] + h0[1] * cr[0][1] + h0[2] * cr[0][2];
    const double scale = norm3d(h0[0], h0[1], h0[2]) * norm3d(h1[0], h1[1], h1[2]) * norm3d(h2[0], h2[1], h2[2]);
    bool bad = !(fabs(det) > 1e-12 * scale);
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) S.Hinv[3 * i + k] = bad ? 0.0 : cr[k][i] / det;
    int nbins = 1;
    for (int k = 0; k < 3; ++k) {
        S.pbc[k] = pbc ? (pbc[3 * s + k] != 0) : 1;
        const double cn = norm3d(cr[k][0], cr[k][1], cr[k][2]);
        const double w = bad ? 0.0 : fabs(det) / cn;
        const double rc = r_cut * (1.0 + 1e-6);
        int nb = 1, reach = 1;
        if (bad || !(w > 0.0)) {
            nb = 1;
            reach = 1;
        } else {
            nb = (int)fmin(floor(w / rc), 1 << 20);
            if (nb < 1) nb = 1;
            if (S.pbc[k]) {
                if (w < r_cut / 64.0) {
                    atomicOr(flags, kFlagThinCell);
                    reach = 1;
                } else {
                    reach = (int)ceil(rc * nb / w);
                    if (reach < 1) reach = 1;
                }
            }
        }
        S.nb[k] = nb;
        S.reach[k] = reach;
    }
    if (bad) atomicOr(flags, kFlagGeometry);
    // cap the bin count at 2 N_s + 8 by halving the finest axis (bins only get wider, reach stays valid)
    const long cap = bad_offsets ? 1L : 2L * (b - a) + 8;
    for (;;) {
        const long prod = (long)S.nb[0] * S.nb[1] * S.nb[2];
        if (prod <= cap) break;
        int kk = 0;
        if (S.nb[1] > S.nb[kk]) kk = 1;
        if (S.nb[2] > S.nb[kk]) kk = 2;
        S.nb[kk] = S.nb[kk] / 2 > 0 ? S.nb[kk] / 2 : 1;
    }
    nbins = S.nb[0] * S.nb[1] * S.nb[2];
    nbins_out[s] = nbins;
}

__device__ inline int find_structure(const int* __restrict__ offs, int n_s, int i) {
    int lo = 0, hi = n_s;  // last s with offs[s] <= i
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (offs[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void k_atom_bin(int n_atoms, int n_s, int64_t nbins_cap, const int* __restrict__ offs, const double* __restrict__ pos,
                           const int* __restrict__ species, const int* __restrict__ lut, StructInfo* info,
                           const int64_t* __restrict__ binbase, int* __restrict__ bin_count, int* __restrict__ atom_bin,
                           int* __restrict__ atom_rank, int* __restrict__ atom_struct, int4* __restrict__ atom_cell,
                           int4* __restrict__ atom_wrap, float4* __restrict__ atom_hi, float4* __restrict__ atom_lo,
                           unsigned* flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_atoms) return;
    const int s = find_structure(offs, n_s, i);
    StructInfo& S = info[s];
    const double r[3] = {pos[3 * (int64_t)i], pos[3 * (int64_t)i + 1], pos[3 * (int64_t)i + 2]};
    // a non-finite position is reported; the clamps below keep its bin and wrap count in range, and its FP32
    // thresholds become NaN, so no pair of its structure is accepted before the call returns the error
    if (!(isfinite(r[0]) && isfinite(r[1]) && isfinite(r[2]))) atomicOr(flags, kFlagNonFinite);
    const int lab = species[i];
    int a = (lab >= 0 && lab < 256) ? lut[lab] : -1;
    if (a < 0) {
        atomicOr(flags, kFlagSpecies);
        a = 0;
    }
    int w[3], bc[3];
    for (int k = 0; k < 3; ++k) {
        const double sk = r[0] * S.Hinv[k] + r[1] * S.Hinv[3 + k] + r[2] * S.Hinv[6 + k];
        double f = sk;
        w[k] = 0;
        if (S.pbc[k]) {
            const double fl = floor(sk);
            w[k] = (int)fmax(fmin(fl, 1e9), -1e9);
            f = sk - fl;
        }
        double x = floor(f * S.nb[k]);
        x = fmin(fmax(x, 0.0), (double)(S.nb[k] - 1));
        bc[k] = (int)x;
    }
    double p[3];
    for (int c = 0; c < 3; ++c)
        p[c] = r[c] - (w[0] * S.H[c] + w[1] * S.H[3 + c] + w[2] * S.H[6 + c]);
    float hi[3], lo[3];
    for (int c = 0; c < 3; ++c) {
        hi[c] = (float)p[c];
        lo[c] = (float)(p[c] - (double)hi[c]);
    }
    const float A = fabsf(hi[0]) + fabsf(hi[1]) + fabsf(hi[2]);
    atomicMax(&S.amax_bits, __float_as_uint(A));
    const int local = (bc[0] * S.nb[1] + bc[1]) * S.nb[2] + bc[2];
    const int64_t gb64 = binbase[s] + local;
    if (gb64 < 0 || gb64 >= nbins_cap) {  // only reachable with inconsistent structure offsets
        atomicOr(flags, kFlagBadOffsets);
        atom_bin[i] = -1;
        atom_rank[i] = 0;
    } else {
        atom_bin[i] = (int)gb64;
        atom_rank[i] = atomicAdd(&bin_count[gb64], 1);
    }
    atom_struct[i] = s;
    atom_cell[i] = make_int4(bc[0], bc[1], bc[2], a);
    atom_wrap[i] = make_int4(w[0], w[1], w[2], 0);
    atom_hi[i] = make_float4(hi[0], hi[1], hi[2], A);
    atom_lo[i] = make_float4(lo[0], lo[1], lo[2], 0.0f);
}

__global__ void k_atom_scatter(int n_atoms, const int* __restrict__ atom_bin, const int* __restrict__ atom_rank,
                               const int64_t* __restrict__ bin_start, const float4* __restrict__ atom_hi,
                               float4* __restrict__ sorted_hi) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_atoms || atom_bin[i] < 0) return;
    const int64_t slot = bin_start[atom_bin[i]] + atom_rank[i];
    const float4 h = atom_hi[i];
    sorted_hi[slot] = make_float4(h.x, h.y, h.z, __int_as_float(i));
}

__global__ void k_struct_thresholds(int n_s, double r_cut, StructInfo* info) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_s) return;
    StructInfo& S = info[s];
    const double amax = (double)__uint_as_float(S.amax_bits);
    double tmax = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double hk = fabs((double)S.hhi[3 * k]) + fabs((double)S.hhi[3 * k + 1]) + fabs((double)S.hhi[3 * k + 2]);
        tmax += (S.reach[k] + 1) * hk;
    }
    const double delta = 2e-6 * (2.0 * amax + tmax) + 1e-6 * r_cut;
    const double lo = fmax(r_cut - delta, 0.0), hi = r_cut + delta;
    S.thr_lo2 = (float)(lo * lo);
    S.thr_hi2 = (float)(hi * hi);
    const double tiny = 1e-3 + delta;
    S.thr_tiny2 = (float)(tiny * tiny);
}

__device__ inline void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ inline void two_prod(float a, float b, float& p, float& e) {
    p = a * b;
    e = fmaf(a, b, -p);
}

// exact FP64 inclusion test and squared distance, same operation order as the definition
__device__ inline double exact_d2(const double* __restrict__ pos, int i, int j, const double* H, const int n[3]) {
    double d[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double rel = __dsub_rn(pos[3 * (int64_t)j + c], pos[3 * (int64_t)i + c]);
        const double sv = __dadd_rn(__dadd_rn(__dmul_rn((double)n[0], H[c]), __dmul_rn((double)n[1], H[3 + c])),
                                    __dmul_rn((double)n[2], H[6 + c]));
        d[c] = __dadd_rn(rel, sv);
    }
    return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

__device__ inline uint64_t pair_key(int j, const int n[3]) {
    return ((uint64_t)(uint32_t)j << 30) | ((uint64_t)(n[0] + 512) << 20) | ((uint64_t)(n[1] + 512) << 10) |
           (uint64_t)(n[2] + 512);
}

// CAP: pairs a warp sorts in shared memory (8 blocks of 4 warps per SM at CAP = 128)
template <bool FILL, int CAP = kPairCap>
__global__ void __launch_bounds__(kPairWarps * 32, CAP <= 128 ? 8 : 0) k_pairs(
    int n_atoms, const double* __restrict__ pos, const StructInfo* __restrict__ info, const int64_t* __restrict__ binbase,
    const int64_t* __restrict__ bin_start, const float4* __restrict__ sorted_hi, const int* __restrict__ atom_struct,
    const int4* __restrict__ atom_cell, const int4* __restrict__ atom_wrap, const float4* __restrict__ atom_hi,
    const float4* __restrict__ atom_lo, double rc2, int64_t nbins_cap, int64_t* __restrict__ counts_or_offsets, int* __restrict__ max_count,
    int* __restrict__ out_j, int* __restrict__ out_shift, float4* __restrict__ out_rij, uint64_t* __restrict__ ovf_keys,
    float4* __restrict__ ovf_vec, unsigned* flags) {
    constexpr int kPairEPL = CAP / 32;
    __shared__ uint64_t s_keys[FILL ? kPairWarps * CAP : 1];
    __shared__ float4 s_vec[FILL ? kPairWarps * CAP : 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kPairWarps + warp;
    if (i >= n_atoms) return;
    const int s = atom_struct[i];
    const StructInfo& S = info[s];
    const int4 cell = atom_cell[i];
    const int4 wi = atom_wrap[i];
    const float4 phi = atom_hi[i];
    const float4 plo = atom_lo[i];
    const float thr_lo2 = S.thr_lo2, thr_hi2 = S.thr_hi2, thr_tiny2 = S.thr_tiny2;
    const int bci[3] = {cell.x, cell.y, cell.z};
    int64_t seg_beg = 0, seg_cnt = 0;
    uint64_t* keys = s_keys + warp * CAP;
    float4* vecs = s_vec + warp * CAP;
    bool use_global = false;
    if (FILL) {
        seg_beg = counts_or_offsets[i];
        seg_cnt = counts_or_offsets[i + 1] - seg_beg;
        if (seg_cnt > CAP) {
            use_global = true;
            keys = ovf_keys + seg_beg;
            vecs = ovf_vec + seg_beg;
        }
    }
    int count = 0;
    unsigned local_flags = 0;
    // Flattened walk over the stencil: up to 32 stencil bins at a time, one per lane, their candidate counts
    // prefix-summed across the warp, then 32 candidates per iteration with each lane locating its bin by a
    // binary search over the prefix (all loop bounds warp-uniform).
    __shared__ int64_t s_beg[kPairWarps][32];
    __shared__ int4 s_t[kPairWarps][32];
    __shared__ float4 s_T[kPairWarps][32];
    __shared__ float4 s_Th[kPairWarps][FILL ? 32 : 1];
    __shared__ float4 s_Tl[kPairWarps][FILL ? 32 : 1];
    const int w0 = 2 * S.reach[0] + 1, w1 = 2 * S.reach[1] + 1, w2 = 2 * S.reach[2] + 1;
    const int n_st = w0 * w1 * w2;
    for (int g0 = 0; g0 < n_st; g0 += 32) {
        const int e = g0 + lane;
        int cnt = 0;
        if (e < n_st) {
            const int dd[3] = {e / (w1 * w2) - S.reach[0], (e / w2) % w1 - S.reach[1], e % w2 - S.reach[2]};
            int tb[3], t[3];
            bool valid = true;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int x = bci[k] + dd[k];
                if (S.pbc[k]) {
                    t[k] = floordiv(x, S.nb[k]);
                    tb[k] = x - t[k] * S.nb[k];
                } else {
                    t[k] = 0;
                    tb[k] = x;
                    if (x < 0 || x >= S.nb[k]) valid = false;
                }
            }
            const int64_t bin = binbase[s] + (tb[0] * S.nb[1] + tb[1]) * S.nb[2] + tb[2];
            if (bin < 0 || bin >= nbins_cap) valid = false;  // inconsistent offsets, already flagged
            if (valid) {
                const int64_t beg = bin_start[bin];
                cnt = (int)(bin_start[bin + 1] - beg);
                s_beg[warp][lane] = beg;
                s_t[warp][lane] = make_int4(t[0], t[1], t[2], (t[0] == 0 && t[1] == 0 && t[2] == 0) ? 1 : 0);
                float Tf[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    // explicit roundings: the count and fill passes must take identical decisions
                    Tf[c] = __fadd_rn(__fadd_rn(__fmul_rn((float)t[0], S.hhi[c]), __fmul_rn((float)t[1], S.hhi[3 + c])),
                                      __fmul_rn((float)t[2], S.hhi[6 + c]));
                }
                s_T[warp][lane] = make_float4(Tf[0], Tf[1], Tf[2], 0.0f);
                if (FILL) {
                    float Th[3], Tl[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        float sh = 0.0f, sl = 0.0f;
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            float pp, pe, s2, e2;
                            two_prod((float)t[k], S.hhi[3 * k + c], pp, pe);
                            pe += (float)t[k] * S.hlo[3 * k + c];
                            two_sum(sh, pp, s2, e2);
                            sh = s2;
                            sl += pe + e2;
                        }
                        Th[c] = sh;
                        Tl[c] = sl;
                    }
                    s_Th[warp][FILL ? lane : 0] = make_float4(Th[0], Th[1], Th[2], 0.0f);
                    s_Tl[warp][FILL ? lane : 0] = make_float4(Tl[0], Tl[1], Tl[2], 0.0f);
                }
            }
        }
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        __syncwarp();
        for (int base = 0; base < total; base += 32) {
            const int cidx = base + lane;
            // entry k of this candidate: number of entries whose inclusive prefix is <= cidx
            int k = 0;
#pragma unroll
            for (int st = 16; st >= 1; st >>= 1) {
                const int v = __shfl_sync(0xffffffffu, incl, k + st - 1);
                if (v <= cidx) k += st;
            }
            const int excl_k = __shfl_sync(0xffffffffu, incl, k) - __shfl_sync(0xffffffffu, cnt, k);
            bool accept = false;
            int j = -1;
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
            int4 tt = make_int4(0, 0, 0, 0);
            if (cidx < total) {
                tt = s_t[warp][k];
                const float4 Tf = s_T[warp][k];
                q = sorted_hi[s_beg[warp][k] + (cidx - excl_k)];
                j = __float_as_int(q.w);
                const float dx = __fsub_rn(__fadd_rn(q.x, Tf.x), phi.x);
                const float dy = __fsub_rn(__fadd_rn(q.y, Tf.y), phi.y);
                const float dz = __fsub_rn(__fadd_rn(q.z, Tf.z), phi.z);
                const float dsq = fmaf(dz, dz, fmaf(dy, dy, __fmul_rn(dx, dx)));
                if (!(j == i && tt.w)) {
                    if (dsq < thr_lo2) {
                        accept = true;
                    } else if (dsq <= thr_hi2) {
                        const int4 wj = atom_wrap[j];
                        const int n[3] = {tt.x - wj.x + wi.x, tt.y - wj.y + wi.y, tt.z - wj.z + wi.z};
                        accept = exact_d2(pos, i, j, S.H, n) < rc2;
                    }
                    if (accept && dsq < thr_tiny2) {
                        const int4 wj = atom_wrap[j];
                        const int n[3] = {tt.x - wj.x + wi.x, tt.y - wj.y + wi.y, tt.z - wj.z + wi.z};
                        if (exact_d2(pos, i, j, S.H, n) < 1e-12) local_flags |= kFlagGeometry;
                    }
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, accept);
            if (accept) {
                const int4 wj = atom_wrap[j];
                const int n[3] = {tt.x - wj.x + wi.x, tt.y - wj.y + wi.y, tt.z - wj.z + wi.z};
                if (n[0] < -kMaxShift || n[0] > kMaxShift || n[1] < -kMaxShift || n[1] > kMaxShift || n[2] < -kMaxShift ||
                    n[2] > kMaxShift)
                    local_flags |= kFlagShiftRange;
                if (FILL) {
                    const int slot = count + __popc(m & ((1u << lane) - 1u));
                    if (slot < seg_cnt) {
                        const float4 qlo = atom_lo[j];
                        const float4 Th4 = s_Th[warp][FILL ? k : 0], Tl4 = s_Tl[warp][FILL ? k : 0];
                        const float Th[3] = {Th4.x, Th4.y, Th4.z}, Tl[3] = {Tl4.x, Tl4.y, Tl4.z};
                        const float pj[3] = {q.x, q.y, q.z}, pjl[3] = {qlo.x, qlo.y, qlo.z};
                        const float pi_[3] = {phi.x, phi.y, phi.z}, pil[3] = {plo.x, plo.y, plo.z};
                        float v[3];
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc) {
                            float s1, e1, s2, e2;
                            two_sum(pj[cc], Th[cc], s1, e1);
                            e1 += pjl[cc] + Tl[cc];
                            two_sum(s1, -pi_[cc], s2, e2);
                            e2 += e1 - pil[cc];
                            v[cc] = s2 + e2;
                        }
                        const float rr = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                        const int nc[3] = {min(max(n[0], -kMaxShift), kMaxShift), min(max(n[1], -kMaxShift), kMaxShift),
                                           min(max(n[2], -kMaxShift), kMaxShift)};
                        keys[slot] = pair_key(j, nc);
                        vecs[slot] = make_float4(v[0], v[1], v[2], rr);
                    }
                }
            }
            count += __popc(m);
        }
        __syncwarp();
    }
    if (local_flags) atomicOr(flags, local_flags);
    if (!FILL) {
        if (lane == 0) {
            counts_or_offsets[i] = count;
            atomicMax(max_count, count);
        }
        return;
    }
    // rank sort of the segment by (j, n1, n2, n3) and write-out
    __syncwarp();
    const int k = (int)(seg_cnt < (int64_t)count ? seg_cnt : (int64_t)count);
    if (!use_global) {
        uint64_t mykey[kPairEPL];
        int myrank[kPairEPL];
#pragma unroll
        for (int qd = 0; qd < kPairEPL; ++qd) {
            const int e = lane + 32 * qd;
            mykey[qd] = (e < k) ? keys[e] : ~0ull;
            myrank[qd] = 0;
        }
        const int nq = (k + 31) / 32;
        for (int f = 0; f < k; ++f) {
            const uint64_t kf = keys[f];
#pragma unroll
            for (int qd = 0; qd < kPairEPL; ++qd)
                if (qd < nq) myrank[qd] += (kf < mykey[qd]);
        }
#pragma unroll
        for (int qd = 0; qd < kPairEPL; ++qd) {
            const int e = lane + 32 * qd;
            if (e < k) {
                const int64_t o = seg_beg + myrank[qd];
                const uint64_t key = mykey[qd];
                out_j[o] = (int)(key >> 30);
                out_shift[3 * o + 0] = (int)((key >> 20) & 1023) - 512;
                out_shift[3 * o + 1] = (int)((key >> 10) & 1023) - 512;
                out_shift[3 * o + 2] = (int)(key & 1023) - 512;
                out_rij[o] = vecs[e];
            }
        }
    } else {
        __threadfence_block();
        for (int e = lane; e < k; e += 32) {
            const uint64_t key = keys[e];
            int rank = 0;
            for (int f = 0; f < k; ++f) rank += (keys[f] < key);
            const int64_t o = seg_beg + rank;
            out_j[o] = (int)(key >> 30);
            out_shift[3 * o + 0] = (int)((key >> 20) & 1023) - 512;
            out_shift[3 * o + 1] = (int)((key >> 10) & 1023) - 512;
            out_shift[3 * o + 2] = (int)(key & 1023) - 512;
            out_rij[o] = vecs[e];
        }
    }
}

}  // namespace rascal

using namespace rascal;

extern "C" int rascal_neighbours(rascal_ctx* ctx, const rascal_system* sys, int64_t capacity, int64_t* d_offsets,
                                 int* d_nbr_j, int* d_shift, float* d_rij, int64_t* n_pairs) {
    clear_error();
    if (!ctx) return set_error(RASCAL_E_ARG, "NULL context");
    int st = validate_system(ctx, sys);
    if (st) return st;
    if (!d_offsets || !n_pairs || capacity < 0) return set_error(RASCAL_E_ARG, "NULL offsets / n_pairs or negative capacity");
    const int N = sys->n_atoms, n_s = sys->n_structures;
    cudaStream_t stream = ctx->stream;
    *n_pairs = 0;
    if (N == 0) {
        RASCAL_CUDA(cudaMemsetAsync(d_offsets, 0, sizeof(int64_t), stream));
        return RASCAL_OK;
    }
    const int64_t nbins_cap = 2LL * N + 8LL * n_s;
    const size_t bytes = carve_bytes(sizeof(StructInfo) * n_s, sizeof(int) * (n_s + 1), sizeof(int64_t) * (n_s + 1),
                                     sizeof(int) * nbins_cap, sizeof(int64_t) * (nbins_cap + 1), sizeof(int) * N,
                                     sizeof(int) * N, sizeof(int) * N, sizeof(int4) * N, sizeof(int4) * N,
                                     sizeof(float4) * N, sizeof(float4) * N, sizeof(float4) * N, sizeof(int) * 4);
    void* base;
    if ((st = arena_get(ctx->scratch, bytes, &base))) return st;
    Carver cv(base);
    StructInfo* info = cv.take<StructInfo>(n_s);
    int* nbins = cv.take<int>(n_s + 1);
    int64_t* binbase = cv.take<int64_t>(n_s + 1);
    int* bin_count = cv.take<int>(nbins_cap);
    int64_t* bin_start = cv.take<int64_t>(nbins_cap + 1);
    int* atom_bin = cv.take<int>(N);
    int* atom_rank = cv.take<int>(N);
    int* atom_struct = cv.take<int>(N);
    int4* atom_cell = cv.take<int4>(N);
    int4* atom_wrap = cv.take<int4>(N);
    float4* atom_hi = cv.take<float4>(N);
    float4* atom_lo = cv.take<float4>(N);
    float4* sorted_hi = cv.take<float4>(N);
    int* max_count = cv.take<int>(4);

    RASCAL_CUDA(cudaMemsetAsync(bin_count, 0, sizeof(int) * nbins_cap, stream));
    RASCAL_CUDA(cudaMemsetAsync(max_count, 0, sizeof(int), stream));
    k_struct_setup<<<(unsigned)div_up(n_s, 128), 128, 0, stream>>>(n_s, N, sys->d_struct_offsets, sys->d_cells, sys->d_pbc,
                                                                 ctx->r_cut, info, nbins, ctx->d_flags);
    RASCAL_LAUNCH_CHECK("k_struct_setup");
    if ((st = scan_exclusive(nbins, binbase, n_s, stream, ctx->scratch2))) return st;
    k_atom_bin<<<(unsigned)div_up(N, 256), 256, 0, stream>>>(N, n_s, nbins_cap, sys->d_struct_offsets, sys->d_positions, sys->d_species,
                                                           ctx->d_lut, info, binbase, bin_count, atom_bin, atom_rank,
                                                           atom_struct, atom_cell, atom_wrap, atom_hi, atom_lo, ctx->d_flags);
    RASCAL_LAUNCH_CHECK("k_atom_bin");
    if ((st = scan_exclusive(bin_count, bin_start, nbins_cap, stream, ctx->scratch2))) return st;
    k_atom_scatter<<<(unsigned)div_up(N, 256), 256, 0, stream>>>(N, atom_bin, atom_rank, bin_start, atom_hi, sorted_hi);
    RASCAL_LAUNCH_CHECK("k_atom_scatter");
    k_struct_thresholds<<<(unsigned)div_up(n_s, 128), 128, 0, stream>>>(n_s, ctx->r_cut, info);
    RASCAL_LAUNCH_CHECK("k_struct_thresholds");
    const double rc2 = ctx->r_cut * ctx->r_cut;
    const unsigned pair_blocks = (unsigned)div_up(N, kPairWarps);
    k_pairs<false><<<pair_blocks, kPairWarps * 32, 0, stream>>>(N, sys->d_positions, info, binbase, bin_start, sorted_hi,
                                                                atom_struct, atom_cell, atom_wrap, atom_hi, atom_lo, rc2,
                                                                nbins_cap, d_offsets, max_count, nullptr, nullptr, nullptr, nullptr,
                                                                nullptr, ctx->d_flags);
    RASCAL_LAUNCH_CHECK("k_pairs<count>");
    if ((st = scan_exclusive(d_offsets, d_offsets, N, stream, ctx->scratch2))) return st;
    RASCAL_CUDA(cudaMemcpyAsync(ctx->h_pinned, d_offsets + N, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
    RASCAL_CUDA(cudaMemcpyAsync(ctx->h_pinned + 1, max_count, sizeof(int), cudaMemcpyDeviceToHost, stream));
    if ((st = check_flags(ctx))) return st;  // synchronises the stream
    const int64_t P = ctx->h_pinned[0];
    const int maxc = *reinterpret_cast<int*>(ctx->h_pinned + 1);
    *n_pairs = P;
    if (P > capacity) return set_error(RASCAL_E_CAPACITY, "pair capacity %lld < required %lld", (long long)capacity, (long long)P);
    if (P == 0) return RASCAL_OK;
    if (!d_nbr_j || !d_shift || !d_rij) return set_error(RASCAL_E_ARG, "NULL pair output arrays");
    uint64_t* ovf_keys = nullptr;
    float4* ovf_vec = nullptr;
    if (maxc > kPairCap) {
        void* ob;
        if ((st = arena_get(ctx->scratch2, carve_bytes(sizeof(uint64_t) * P, sizeof(float4) * P), &ob))) return st;
        Carver oc(ob);
        ovf_keys = oc.take<uint64_t>(P);
        ovf_vec = oc.take<float4>(P);
    }
    k_pairs<true><<<pair_blocks, kPairWarps * 32, 0, stream>>>(N, sys->d_positions, info, binbase, bin_start, sorted_hi,
                                                               atom_struct, atom_cell, atom_wrap, atom_hi, atom_lo, rc2,
                                                               nbins_cap, d_offsets, nullptr, d_nbr_j, d_shift,
                                                               reinterpret_cast<float4*>(d_rij), ovf_keys, ovf_vec,
                                                               ctx->d_flags);
    RASCAL_LAUNCH_CHECK("k_pairs<fill>");
    return RASCAL_OK;
}

// ---------------------------------------------------------------------------------------------------------
// Neighbour search that allocates nothing: the same kernels as rascal_neighbours, with all scratch carved out of
// one file-scope device array. The array is a module global, so every GPU that loads the library holds it until
// the process exits. Its device address is looked up per device (cudaGetSymbolAddress with that device current)
// when a context is created on it, and cached; all calls on a device share the array.
// ---------------------------------------------------------------------------------------------------------
namespace rascal {

constexpr size_t kStaticNbrScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_nbr_scratch[kStaticNbrScratchBytes];
constexpr int kMaxDevices = 64;
static void* g_nbr_scratch_addr[kMaxDevices];
static std::mutex g_nbr_scratch_mu;

// Caches the device address of the array for ctx->device, which must be the current device. Called by
// rascal_create, so the lookup (which may load the module and reserve the array) happens before any step loop.
int nbr_static_prepare(rascal_ctx* ctx) {
    const int dev = ctx->device;
    if (dev < 0 || dev >= kMaxDevices) return set_error(RASCAL_E_UNSUPPORTED, "device ordinal %d above %d", dev, kMaxDevices - 1);
    std::lock_guard<std::mutex> lock(g_nbr_scratch_mu);
    if (!g_nbr_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_nbr_scratch);
        if (e != cudaSuccess || !p)
            return set_error(RASCAL_E_CUDA, "cudaGetSymbolAddress of the static neighbour scratch: %s", cudaGetErrorString(e));
        g_nbr_scratch_addr[dev] = p;
    }
    return RASCAL_OK;
}

// The cached address for the context's device. The kernels run on ctx->stream, which belongs to ctx->device, so a
// call made while another device is current is refused rather than handed another GPU's copy of the array.
static int static_nbr_scratch(const rascal_ctx* ctx, void** out) {
    int cur = -1;
    const cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return set_error(RASCAL_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (cur != ctx->device)
        return set_error(RASCAL_E_ARG, "the current device (%d) is not the context's device (%d)", cur, ctx->device);
    std::lock_guard<std::mutex> lock(g_nbr_scratch_mu);
    *out = g_nbr_scratch_addr[ctx->device];
    if (!*out) return set_error(RASCAL_E_CUDA, "the static neighbour scratch of device %d was not prepared", ctx->device);
    return RASCAL_OK;
}

}  // namespace rascal

extern "C" size_t rascal_neighbours_static_limit(void) { return rascal::kStaticNbrScratchBytes; }

extern "C" int rascal_neighbours_noalloc(rascal_ctx* ctx, const rascal_system* sys, int64_t capacity, int64_t* d_offsets,
                                         int* d_nbr_j, int* d_shift, float* d_rij, int64_t* n_pairs) {
    clear_error();
    if (!ctx) return set_error(RASCAL_E_ARG, "NULL context");
    int st = validate_system(ctx, sys);
    if (st) return st;
    if (!d_offsets || !n_pairs || capacity < 0) return set_error(RASCAL_E_ARG, "NULL offsets / n_pairs or negative capacity");
    const int N = sys->n_atoms, n_s = sys->n_structures;
    cudaStream_t stream = ctx->stream;
    *n_pairs = 0;
    if (N == 0) {
        RASCAL_CUDA(cudaMemsetAsync(d_offsets, 0, sizeof(int64_t), stream));
        return RASCAL_OK;
    }
    const int64_t nbins_cap = 2LL * N + 8LL * n_s;
    const int64_t sums_len = std::max(scan_tile_sums_len(n_s), std::max(scan_tile_sums_len(nbins_cap), scan_tile_sums_len(N)));
    const size_t bytes = carve_bytes(sizeof(StructInfo) * n_s, sizeof(int) * (n_s + 1), sizeof(int64_t) * (n_s + 1),
                                     sizeof(int) * nbins_cap, sizeof(int64_t) * (nbins_cap + 1), sizeof(int) * N,
                                     sizeof(int) * N, sizeof(int) * N, sizeof(int4) * N, sizeof(int4) * N,
                                     sizeof(float4) * N, sizeof(float4) * N, sizeof(float4) * N, sizeof(int) * 4,
                                     sizeof(int64_t) * sums_len);
    if (bytes > kStaticNbrScratchBytes)
        return set_error(RASCAL_E_UNSUPPORTED,
                         "this system needs %zu bytes of neighbour scratch; the no-allocation entry point holds %zu "
                         "(about 116 bytes per atom and 360 per structure): use rascal_neighbours",
                         bytes, kStaticNbrScratchBytes);
    void* base = nullptr;
    if ((st = static_nbr_scratch(ctx, &base))) return st;
    Carver cv(base);
    StructInfo* info = cv.take<StructInfo>(n_s);
    int* nbins = cv.take<int>(n_s + 1);
    int64_t* binbase = cv.take<int64_t>(n_s + 1);
    int* bin_count = cv.take<int>(nbins_cap);
    int64_t* bin_start = cv.take<int64_t>(nbins_cap + 1);
    int* atom_bin = cv.take<int>(N);
    int* atom_rank = cv.take<int>(N);
    int* atom_struct = cv.take<int>(N);
    int4* atom_cell = cv.take<int4>(N);
    int4* atom_wrap = cv.take<int4>(N);
    float4* atom_hi = cv.take<float4>(N);
    float4* atom_lo = cv.take<float4>(N);
    float4* sorted_hi = cv.take<float4>(N);
    int* max_count = cv.take<int>(4);
    int64_t* sums = cv.take<int64_t>(sums_len);

    // the array keeps the previous call's contents: the bin counters and the maximum must start at zero
    RASCAL_CUDA(cudaMemsetAsync(bin_count, 0, sizeof(int) * nbins_cap, stream));
    RASCAL_CUDA(cudaMemsetAsync(max_count, 0, sizeof(int), stream));
    k_struct_setup<<<(unsigned)div_up(n_s, 128), 128, 0, stream>>>(n_s, N, sys->d_struct_offsets, sys->d_cells, sys->d_pbc,
                                                                 ctx->r_cut, info, nbins, ctx->d_flags);
    RASCAL_LAUNCH_CHECK("k_struct_setup");
    if ((st = scan_exclusive_into(nbins, binbase, n_s, stream, sums))) return st;
    k_atom_bin<<<(unsigned)div_up(N, 256), 256, 0, stream>>>(N, n_s, nbins_cap, sys->d_struct_offsets, sys->d_positions,
                                                           sys->d_species, ctx->d_lut, info, binbase, bin_count, atom_bin,
                                                           atom_rank, atom_struct, atom_cell, atom_wrap, atom_hi, atom_lo,
                                                           ctx->d_flags);
    RASCAL_LAUNCH_CHECK("k_atom_bin");
    if ((st = scan_exclusive_into(bin_count, bin_start, nbins_cap, stream, sums))) return st;
    k_atom_scatter<<<(unsigned)div_up(N, 256), 256, 0, stream>>>(N, atom_bin, atom_rank, bin_start, atom_hi, sorted_hi);
    RASCAL_LAUNCH_CHECK("k_atom_scatter");
    k_struct_thresholds<<<(unsigned)div_up(n_s, 128), 128, 0, stream>>>(n_s, ctx->r_cut, info);
    RASCAL_LAUNCH_CHECK("k_struct_thresholds");
    const double rc2 = ctx->r_cut * ctx->r_cut;
    const unsigned pair_blocks = (unsigned)div_up(N, kPairWarps);
    k_pairs<false, kNoallocCap><<<pair_blocks, kPairWarps * 32, 0, stream>>>(N, sys->d_positions, info, binbase, bin_start, sorted_hi,
                                                                atom_struct, atom_cell, atom_wrap, atom_hi, atom_lo, rc2,
                                                                nbins_cap, d_offsets, max_count, nullptr, nullptr, nullptr,
                                                                nullptr, nullptr, ctx->d_flags);
    RASCAL_LAUNCH_CHECK("k_pairs<count>");
    if ((st = scan_exclusive_into(d_offsets, d_offsets, N, stream, sums))) return st;
    RASCAL_CUDA(cudaMemcpyAsync(ctx->h_pinned, d_offsets + N, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
    RASCAL_CUDA(cudaMemcpyAsync(ctx->h_pinned + 1, max_count, sizeof(int), cudaMemcpyDeviceToHost, stream));
    if ((st = check_flags(ctx))) return st;  // synchronises the stream
    const int64_t P = ctx->h_pinned[0];
    const int maxc = *reinterpret_cast<int*>(ctx->h_pinned + 1);
    *n_pairs = P;
    // checked before the capacity, so that a caller who resizes after RASCAL_E_CAPACITY is not refused afterwards
    if (maxc > kNoallocCap)
        return set_error(RASCAL_E_UNSUPPORTED, "a centre has %d neighbours; the no-allocation entry point sorts at most %d "
                         "per centre (rascal_neighbours has no such limit)", maxc, kNoallocCap);
    if (P > capacity) return set_error(RASCAL_E_CAPACITY, "pair capacity %lld < required %lld", (long long)capacity, (long long)P);
    if (P == 0) return RASCAL_OK;
    if (!d_nbr_j || !d_shift || !d_rij) return set_error(RASCAL_E_ARG, "NULL pair output arrays");
    k_pairs<true, kNoallocCap><<<pair_blocks, kPairWarps * 32, 0, stream>>>(N, sys->d_positions, info, binbase, bin_start, sorted_hi,
                                                               atom_struct, atom_cell, atom_wrap, atom_hi, atom_lo, rc2,
                                                               nbins_cap, d_offsets, nullptr, d_nbr_j, d_shift,
                                                               reinterpret_cast<float4*>(d_rij), nullptr, nullptr,
                                                               ctx->d_flags);
    RASCAL_LAUNCH_CHECK("k_pairs<fill>");
    return RASCAL_OK;
}
