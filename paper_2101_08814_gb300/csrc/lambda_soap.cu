// nu = 2 equivariants (lambda-SOAP, Sec. "Experimental features"): the symmetrised correlation of Eq. body-order-x at
// nu = 2 coupled to rank lambda instead of contracted to an invariant,
//   T^{lambda mu}_{(q1 l1)(q2 l2)} = sum_{m1 m2} R^{l1 l2 lambda}[m1][m2][mu] c_{q1 l1 m1} c_{q2 l2 m2},
// with R the Clebsch-Gordan coefficients <l1 m1; l2 m2 | lambda M> (Condon-Shortley) carried into the basis of the
// real harmonics the coefficients use (no Condon-Shortley phase): R = U_lambda . CG . conj(U_l1) . conj(U_l2), real
// for l1 + l2 + lambda even. Only those proper tensors are formed (the improper-rotation average of Eq. body-order-x
// removes the others), and only l1 <= l2: T(l2, l1) is the transpose of T(l1, l2).
//
// Host: Racah's closed form for the CG coefficients in FP64, the unitary U per l, the real tables per (l1, l2), kept
// as their (at most two) non-zero m1 terms per (mu, m2), cached per lambda in the context. Device: one CTA per centre; per pair the two coefficient blocks are staged in
// shared memory, then per chunk of mu the half-contractions X[q1][m2] = sum_m1 R c_{q1 l1 m1} and the output tiles
// T[q1][q2] = sum_m2 X[q1][m2] c_{q2 l2 m2}, written with streaming 16-byte stores. Bound: HBM (the output).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace rascal {

struct LsoapTable {
    int lambda = -1;
    int n_pairs = 0;
    int4* d_hdr = nullptr;   // per pair: l1, l2, offset of its entries in d_R, 0
    float4* d_R = nullptr;   // per pair [2 lambda + 1][2 l2 + 1]: the (at most two) non-zero m1 terms of R[mu][.][m2]
                             // as {value0, value1, m1_0 * Q, m1_1 * Q} (offsets as integer bits; value 0 pads)
};

static double fact(int n) {
    double f = 1.0;
    for (int k = 2; k <= n; ++k) f *= k;
    return f;
}

// <l1 m1; l2 m2 | L M>, Racah's closed form
static double cg(int l1, int m1, int l2, int m2, int L, int M) {
    if (m1 + m2 != M || L < std::abs(l1 - l2) || L > l1 + l2 || std::abs(m1) > l1 || std::abs(m2) > l2 || std::abs(M) > L)
        return 0.0;
    const double pref = std::sqrt((2.0 * L + 1.0) * fact(L + l1 - l2) * fact(L - l1 + l2) * fact(l1 + l2 - L) /
                                  fact(l1 + l2 + L + 1) * fact(L + M) * fact(L - M) * fact(l1 - m1) * fact(l1 + m1) *
                                  fact(l2 - m2) * fact(l2 + m2));
    double s = 0.0;
    for (int k = 0; k <= l1 + l2; ++k) {
        const int a[6] = {k, l1 + l2 - L - k, l1 - m1 - k, l2 + m2 - k, L - l2 + m1 + k, L - l1 - m2 + k};
        bool neg = false;
        for (int v : a) neg |= v < 0;
        if (neg) continue;
        double den = 1.0;
        for (int v : a) den *= fact(v);
        s += ((k & 1) ? -1.0 : 1.0) / den;
    }
    return pref * s;
}

// U[(m' + l)(2l+1) + (m + l)]: Y^real_{l m'} = sum_m U Y^CS_{l m}. With Z^m = N P^|m| e^{i m phi}, Y^CS_m = (-1)^m Z^m
// (m > 0) and Z^m (m <= 0); the real harmonics are Z^0, (Z^m + Z^-m)/sqrt 2 and (Z^m - Z^-m)/(i sqrt 2) (index -m).
static std::vector<std::complex<double>> u_matrix(int l) {
    const int d = 2 * l + 1;
    std::vector<std::complex<double>> U((size_t)d * d, 0.0);
    const double r = 1.0 / std::sqrt(2.0);
    const std::complex<double> I(0.0, 1.0);
    U[(size_t)l * d + l] = 1.0;
    for (int m = 1; m <= l; ++m) {
        const double sg = (m & 1) ? -1.0 : 1.0;
        U[(size_t)(l + m) * d + (l + m)] = sg * r;
        U[(size_t)(l + m) * d + (l - m)] = r;
        U[(size_t)(l - m) * d + (l + m)] = sg * r / I;
        U[(size_t)(l - m) * d + (l - m)] = -r / I;
    }
    return U;
}

// real coupling table [mu][m1'][m2'] for (l1, l2) -> L; false if it is not real (never for l1 + l2 + L even)
static bool real_table(int l1, int l2, int L, std::vector<float>& out) {
    const int d1 = 2 * l1 + 1, d2 = 2 * l2 + 1, dL = 2 * L + 1;
    const auto U1 = u_matrix(l1), U2 = u_matrix(l2), UL = u_matrix(L);
    out.assign((size_t)dL * d1 * d2, 0.0f);
    for (int u = 0; u < dL; ++u)
        for (int x = 0; x < d1; ++x)
            for (int y = 0; y < d2; ++y) {
                std::complex<double> acc = 0.0;
                for (int a = 0; a < d1; ++a) {
                    const std::complex<double> ua = std::conj(U1[(size_t)x * d1 + a]);
                    if (ua == 0.0) continue;
                    for (int b = 0; b < d2; ++b) {
                        const int M = (a - l1) + (b - l2);
                        if (std::abs(M) > L) continue;
                        const std::complex<double> ub = std::conj(U2[(size_t)y * d2 + b]);
                        if (ub == 0.0) continue;
                        acc += UL[(size_t)u * dL + (M + L)] * cg(l1, a - l1, l2, b - l2, L, M) * ua * ub;
                    }
                }
                if (std::abs(acc.imag()) > 1e-10) return false;
                out[((size_t)u * d1 + x) * d2 + y] = (float)acc.real();
            }
    return true;
}

static void lsoap_pairs(int l_max, int lam, std::vector<int2>& p) {
    p.clear();
    for (int l1 = 0; l1 <= l_max; ++l1)
        for (int l2 = l1; l2 <= l_max; ++l2)
            if (std::abs(l1 - l2) <= lam && lam <= l1 + l2 && ((l1 + l2 + lam) & 1) == 0) p.push_back(make_int2(l1, l2));
}

// One CTA per centre. The centre's coefficients are staged once, transposed to cT[lm][q]; per pair and chunk of mu
// values the half-contractions X[u][q1][m2] = sum_m1 R c_{q1 l1 m1} go to one of two buffers, one block barrier,
// then 2 x 4 output tiles per thread (one 16-byte load of cT serves four outputs), stored with streaming 16-byte
// writes. The alternating X buffers let the next chunk's X start while other threads still store this one.
constexpr int kLsoapXFloats = 6144;  // shared-memory budget of one X buffer (24 KB)

__global__ void __launch_bounds__(256) k_lambda_soap(int64_t n, const float* __restrict__ c, int Q, int n_lm, int kmax,
                                                     int lam, int mchunk, int n_pairs, const int4* __restrict__ hdr,
                                                     const float4* __restrict__ R, float* __restrict__ out) {
    extern __shared__ __align__(16) float sm[];
    const int i = blockIdx.x;
    if (i >= n) return;
    float* cT = sm;                              // [n_lm][Q]
    float* const sX0 = cT + (size_t)n_lm * Q;
    float* const sX1 = sX0 + (size_t)mchunk * Q * kmax;
    const float* ci = c + (int64_t)i * Q * n_lm;
    const int M = 2 * lam + 1;
    const int64_t QQ = (int64_t)Q * Q;
    const bool vec = (Q & 3) == 0;
    {
        const int lm = threadIdx.x % n_lm, r0 = threadIdx.x / n_lm, rs = blockDim.x / n_lm;
        if (threadIdx.x < n_lm * rs)
            for (int q = r0; q < Q; q += rs) cT[lm * Q + q] = ci[q * n_lm + lm];
    }
    // output tiling (fixed for the kernel): each thread owns one 4-column group and a stride of row pairs
    const int nq2 = Q >> 2, nq1 = Q >> 1;
    const int t_q2 = vec ? threadIdx.x % nq2 : 0, t_r = vec ? threadIdx.x / nq2 : 0;
    const int r_step = vec ? blockDim.x / nq2 : 1;
    const bool t_on = vec && threadIdx.x < nq2 * r_step;
    int buf = 0;
    __syncthreads();
    for (int p = 0; p < n_pairs; ++p) {
        const int4 h = hdr[p];
        const int l1 = h.x, l2 = h.y, d2 = 2 * l2 + 1;
        const float4* Rp = R + h.z;
        const float* A = cT + l1 * l1 * Q;  // A[m1][q]
        const float* B = cT + l2 * l2 * Q;  // B[m2][q]
        const int b_c = threadIdx.x % d2, b_r = threadIdx.x / d2, b_s = blockDim.x / d2;
        const bool b_on = threadIdx.x < d2 * b_s;
        for (int mu0 = 0; mu0 < M; mu0 += mchunk, buf ^= 1) {
            const int mc = min(mchunk, M - mu0);
            float* sX = buf ? sX1 : sX0;
            if (b_on) {
                // rows rr = u Q + q1 of X over the whole chunk, so that all mc * Q rows share the threads evenly
                int u = 0, q1 = b_r;
                while (q1 >= Q) {
                    q1 -= Q;
                    ++u;
                }
                for (int rr = b_r; rr < mc * Q; rr += b_s) {
                    const float4 e = __ldg(Rp + (size_t)(mu0 + u) * d2 + b_c);  // the two non-zero m1 of this (mu, m2)
                    const float x = fmaf(e.x, A[__float_as_int(e.z) + q1], e.y * A[__float_as_int(e.w) + q1]);
                    sX[(size_t)rr * d2 + b_c] = x;
                    q1 += b_s;
                    while (q1 >= Q) {
                        q1 -= Q;
                        ++u;
                    }
                }
            }
            __syncthreads();
            float* o = out + (((int64_t)i * n_pairs + p) * M + mu0) * QQ;
            if (vec) {
                if (t_on) {
                    // row pairs over the whole chunk: row 2 rp of [mc Q][..] is (u, q1) = (2 rp / Q, 2 rp % Q), and both
                    // X and the output of consecutive mu are contiguous, so no division is needed
                    for (int rp = t_r; rp < mc * nq1; rp += r_step) {
                        {
                            const int q2 = 4 * t_q2;
                            const float* x0 = sX + (size_t)(2 * rp) * d2;
                            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
                            for (int m2 = 0; m2 < d2; ++m2) {
                                const float4 bv = *reinterpret_cast<const float4*>(B + m2 * Q + q2);
                                const float xa = x0[m2], xb = x0[d2 + m2];
                                a.x = fmaf(xa, bv.x, a.x);
                                a.y = fmaf(xa, bv.y, a.y);
                                a.z = fmaf(xa, bv.z, a.z);
                                a.w = fmaf(xa, bv.w, a.w);
                                b.x = fmaf(xb, bv.x, b.x);
                                b.y = fmaf(xb, bv.y, b.y);
                                b.z = fmaf(xb, bv.z, b.z);
                                b.w = fmaf(xb, bv.w, b.w);
                            }
                            float* ou = o + (int64_t)(2 * rp) * Q + q2;
                            __stcs(reinterpret_cast<float4*>(ou), a);
                            __stcs(reinterpret_cast<float4*>(ou + Q), b);
                        }
                    }
                }
            } else {
                for (int e = threadIdx.x; e < mc * Q * Q; e += blockDim.x) {
                    const int u = e / (Q * Q), r = e % (Q * Q), q1 = r / Q, q2 = r % Q;
                    float t = 0.0f;
                    for (int m2 = 0; m2 < d2; ++m2) t = fmaf(sX[((size_t)u * Q + q1) * d2 + m2], B[m2 * Q + q2], t);
                    o[u * QQ + r] = t;
                }
            }
        }
    }
}

int lsoap_table(rascal_ctx* ctx, int lam, int* n_pairs, const int4** hdr, const float4** R) {
    if (lam < 0 || lam > 2 * ctx->l_max) return set_error(RASCAL_E_ARG, "lambda must be in [0, 2 l_max] = [0, %d]", 2 * ctx->l_max);
    LsoapTable*& tab = ctx->lsoap[lam];
    if (!tab) {
        std::vector<int2> P;
        lsoap_pairs(ctx->l_max, lam, P);
        std::vector<int4> h(P.size());
        std::vector<float4> all;
        std::vector<float> one;
        const int Q = ctx->Q;
        for (size_t k = 0; k < P.size(); ++k) {
            const int l1 = P[k].x, l2 = P[k].y, d1 = 2 * l1 + 1, d2 = 2 * l2 + 1;
            if (!real_table(l1, l2, lam, one))
                return set_error(RASCAL_E_UNSUPPORTED, "coupling (%d, %d) -> %d is not real", l1, l2, lam);
            h[k] = make_int4(l1, l2, (int)all.size(), 0);
            for (int u = 0; u < 2 * lam + 1; ++u)
                for (int m2 = 0; m2 < d2; ++m2) {
                    float v[2] = {0.0f, 0.0f};
                    int o[2] = {0, 0}, nz = 0;
                    for (int m1 = 0; m1 < d1; ++m1) {
                        const float r = one[((size_t)u * d1 + m1) * d2 + m2];
                        if (std::fabs(r) < 1e-7f) continue;  // exact zeros up to the rounding of the FP64 sums
                        if (nz == 2)
                            return set_error(RASCAL_E_UNSUPPORTED, "coupling (%d, %d) -> %d has more than two terms",
                                             l1, l2, lam);
                        v[nz] = r;
                        o[nz++] = m1 * Q;
                    }
                    float f[2];
                    std::memcpy(f, o, sizeof(f));  // offsets travel as integer bits
                    all.push_back(make_float4(v[0], v[1], f[0], f[1]));
                }
        }
        LsoapTable* t = new LsoapTable();
        t->lambda = lam;
        t->n_pairs = (int)P.size();
        cudaError_t e = cudaMalloc(&t->d_hdr, sizeof(int4) * std::max<size_t>(1, h.size()));
        if (e == cudaSuccess) e = cudaMalloc(&t->d_R, sizeof(float4) * std::max<size_t>(1, all.size()));
        if (e == cudaSuccess && !h.empty())
            e = cudaMemcpy(t->d_hdr, h.data(), sizeof(int4) * h.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !all.empty())
            e = cudaMemcpy(t->d_R, all.data(), sizeof(float4) * all.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(t->d_hdr);
            cudaFree(t->d_R);
            delete t;
            return set_error(RASCAL_E_CUDA, "lambda-SOAP tables: %s", cudaGetErrorString(e));
        }
        tab = t;
    }
    *n_pairs = tab->n_pairs;
    *hdr = tab->d_hdr;
    *R = tab->d_R;
    return RASCAL_OK;
}

void lsoap_free(rascal_ctx* ctx) {
    for (auto& t : ctx->lsoap) {
        if (!t) continue;
        cudaFree(t->d_hdr);
        cudaFree(t->d_R);
        delete t;
        t = nullptr;
    }
}

}  // namespace rascal

using namespace rascal;

extern "C" int rascal_lambda_soap_size(const rascal_ctx* ctx, int lambda, int* n_pairs, int64_t* features_per_centre) {
    clear_error();
    if (!ctx) return set_error(RASCAL_E_ARG, "NULL context");
    if (lambda < 0 || lambda > 2 * ctx->l_max)
        return set_error(RASCAL_E_ARG, "lambda must be in [0, 2 l_max] = [0, %d]", 2 * ctx->l_max);
    std::vector<int2> P;
    lsoap_pairs(ctx->l_max, lambda, P);
    if (n_pairs) *n_pairs = (int)P.size();
    if (features_per_centre) *features_per_centre = (int64_t)P.size() * (2 * lambda + 1) * ctx->Q * ctx->Q;
    return RASCAL_OK;
}

extern "C" int rascal_debug_real_coupling(int l1, int l2, int lambda, float* R) {
    clear_error();
    if (l1 < 0 || l2 < 0 || l1 > kMaxLMax || l2 > kMaxLMax || lambda < std::abs(l1 - l2) || lambda > l1 + l2 ||
        ((l1 + l2 + lambda) & 1) || !R)
        return set_error(RASCAL_E_ARG, "l1, l2 <= %d, |l1 - l2| <= lambda <= l1 + l2, l1 + l2 + lambda even", kMaxLMax);
    std::vector<float> t;
    if (!real_table(l1, l2, lambda, t)) return set_error(RASCAL_E_UNSUPPORTED, "coupling is not real");
    std::memcpy(R, t.data(), t.size() * sizeof(float));
    return RASCAL_OK;
}

extern "C" int rascal_lambda_soap(rascal_ctx* ctx, int64_t n_centres, const float* d_coeffs, int lambda, float* d_out) {
    clear_error();
    if (!ctx) return set_error(RASCAL_E_ARG, "NULL context");
    if (n_centres < 0) return set_error(RASCAL_E_ARG, "negative n_centres");
    int np;
    const int4* hdr;
    const float4* R;
    int st = lsoap_table(ctx, lambda, &np, &hdr, &R);
    if (st) return st;
    if (n_centres == 0 || np == 0) return RASCAL_OK;
    if (!d_coeffs || !d_out) return set_error(RASCAL_E_ARG, "NULL device pointer");
    if ((reinterpret_cast<uintptr_t>(d_out) & 15) != 0) return set_error(RASCAL_E_ARG, "d_out must be 16-byte aligned");
    if (n_centres > 0x7fffffffLL) return set_error(RASCAL_E_ARG, "too many centres for one launch");
    const int kmax = 2 * ctx->l_max + 1;
    const int mchunk = std::max(1, std::min(2 * lambda + 1, kLsoapXFloats / (ctx->Q * kmax)));
    const size_t smem = sizeof(float) * ((size_t)ctx->n_lm * ctx->Q + (size_t)2 * mchunk * ctx->Q * kmax);
    static bool attr = false;
    if (!attr) {
        RASCAL_CUDA(cudaFuncSetAttribute(k_lambda_soap, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr = true;
    }
    if (smem > 227 * 1024)
        return set_error(RASCAL_E_UNSUPPORTED, "n_species * n_max * (l_max + 1)^2 too large for the equivariant kernel");
    k_lambda_soap<<<(unsigned)n_centres, 256, smem, ctx->stream>>>(n_centres, d_coeffs, ctx->Q, ctx->n_lm, kmax, lambda,
                                                                    mchunk, np, hdr, R, d_out);
    RASCAL_LAUNCH_CHECK("k_lambda_soap");
    return RASCAL_OK;
}
