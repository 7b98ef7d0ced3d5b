// Context creation: hypers validation, GTO constants, overlap matrix and S^-1/2 (Sec. 'GTO radial basis'),
// the FP64 exact radial integrals (Eq. rad-int-gto-1 with the 1F1 of Appendix A) and the clamped cubic spline
// table (Sec. 'Spline optimization'), plus status handling and the scratch arena.
#include <math.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "radial_fp64.cuh"

namespace rascal {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int set_error(int code, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

void clear_error() { g_last_error.clear(); }

int arena_get(Arena& a, size_t bytes, void** out) {
    if (bytes == 0) bytes = 256;
    if (a.bytes < bytes) {
        if (a.ptr) cudaFree(a.ptr);
        a.ptr = nullptr;
        a.bytes = 0;
        size_t want = bytes + bytes / 8;
        cudaError_t e = cudaMalloc(&a.ptr, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            a.ptr = nullptr;
            return set_error(RASCAL_E_NOMEM, "scratch allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
        }
        a.bytes = want;
    }
    *out = a.ptr;
    return RASCAL_OK;
}

int check_flags(rascal_ctx* ctx) {
    RASCAL_CUDA(cudaMemcpyAsync(ctx->h_flags, ctx->d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    RASCAL_CUDA(cudaStreamSynchronize(ctx->stream));
    const unsigned f = *ctx->h_flags;
    if (f == 0) return RASCAL_OK;
    RASCAL_CUDA(cudaMemsetAsync(ctx->d_flags, 0, sizeof(unsigned), ctx->stream));
    if (f & kFlagSpecies) return set_error(RASCAL_E_ARG, "an atom's species label is not in the hypers' species list");
    if (f & kFlagBadOffsets) return set_error(RASCAL_E_ARG, "structure offsets are not non-decreasing within [0, n_atoms]");
    if (f & kFlagNonFinite) return set_error(RASCAL_E_ARG, "an atom position is not finite");
    if (f & kFlagGeometry) return set_error(RASCAL_E_GEOMETRY, "singular cell or coincident atoms (r < 1e-6 A)");
    if (f & kFlagThinCell) return set_error(RASCAL_E_UNSUPPORTED, "a cell is thinner than r_cut/64 along some axis");
    if (f & kFlagShiftRange) return set_error(RASCAL_E_UNSUPPORTED, "a periodic shift exceeds |n| <= 511");
    if (f & kFlagTimeout) return set_error(RASCAL_E_TIMEOUT, "a bounded wait for tensor-core completion timed out");
    if (f & kFlagSelection) return set_error(RASCAL_E_ARG, "a selected feature index is outside [0, features_packed)");
    return set_error(RASCAL_E_CUDA, "unknown device flag 0x%x", f);
}

int validate_system(const rascal_ctx* ctx, const rascal_system* sys) {
    (void)ctx;
    if (!sys) return set_error(RASCAL_E_ARG, "system is NULL");
    if (sys->n_structures < 0 || sys->n_atoms < 0) return set_error(RASCAL_E_ARG, "negative sizes in system");
    if (sys->n_atoms > 0 && (!sys->d_positions || !sys->d_species || !sys->d_struct_offsets || !sys->d_cells))
        return set_error(RASCAL_E_ARG, "system has a NULL device pointer");
    if (sys->n_atoms > 0 && sys->n_structures == 0) return set_error(RASCAL_E_ARG, "atoms without structures");
    return RASCAL_OK;
}

// ---------------------------------------------------------------------------------------------------------
// GTO constants, overlap matrix S and its symmetric inverse square root (cyclic Jacobi, FP64, one thread).
// d_n = 1/(2 sigma_n^2), sigma_n = r_cut max(sqrt n, 1)/n_max, N_n^2 = 2/(sigma_n^(2n+3) Gamma(n+3/2))   (Eq. GTO)
// S_nn' = N_n N_n' Gamma((n+n'+3)/2) / (2 (d_n + d_n')^((n+n'+3)/2))
// ---------------------------------------------------------------------------------------------------------
__global__ void k_gto_constants(int n_max, double r_cut, int orthonormal, double* gto, double* T, double* work) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double* dn = gto;
    double* Nn = gto + (n_max + 1);
    for (int n = 0; n <= n_max; ++n) {
        const double sig = r_cut * fmax(sqrt((double)n), 1.0) / n_max;
        dn[n] = 1.0 / (2.0 * sig * sig);
        Nn[n] = sqrt(2.0 / (pow(sig, 2.0 * n + 3.0) * tgamma(n + 1.5)));
    }
    const int n = n_max;
    double* A = work;          // [n][n]
    double* V = work + n * n;  // [n][n]
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            const double p = 0.5 * (i + j + 3);
            A[i * n + j] = Nn[i] * Nn[j] * 0.5 * exp(lgamma(p) - p * log(dn[i] + dn[j]));
            V[i * n + j] = (i == j) ? 1.0 : 0.0;
        }
    if (!orthonormal) {
        for (int i = 0; i < n * n; ++i) T[i] = V[i];
        return;
    }
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < n; ++i) {
            diag += A[i * n + i] * A[i * n + i];
            for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
        }
        if (off <= 1e-34 * diag) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[p * n + q];
                if (apq == 0.0) continue;
                const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    const double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    const double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += V[i * n + k] * V[j * n + k] / sqrt(A[k * n + k]);
            T[i * n + j] = acc;
        }
}

// Switch point of G(a, b) for a = (n+l+3)/2, b = l+3/2, n in [0, n_max], l in [0, l_max+1]: one warp per (n, l),
// 5 rounds of 32 probes narrowing [lo, hi] to the first probe from which every larger probe agrees to 1e-13.
__global__ void k_switch_points(int n_max, int l_max, double* zs_out) {
    const int id = blockIdx.x;
    const int L2 = l_max + 2;
    const int n = id / L2, l = id % L2;
    if (n > n_max) return;
    const double a = 0.5 * (n + l + 3), b = l + 1.5;
    const int lane = threadIdx.x;
    auto ok = [&](double z) {
        const double ser = g_series(a, b, z, -z);
        const double asy = g_asymptotic(a, b, z, -z);
        return fabs(asy - ser) <= 1e-13 * fabs(ser);
    };
    double lo = 1.0, hi = 300.0;
    const bool ok_hi = ok(hi);
    if (!ok_hi) {
        if (lane == 0) zs_out[id] = INFINITY;
        return;
    }
    if (ok(lo)) {
        if (lane == 0) zs_out[id] = lo;
        return;
    }
    for (int round = 0; round < 5; ++round) {
        const double z = lo + (hi - lo) * (lane + 1) / 33.0;
        const unsigned bad = __ballot_sync(0xffffffffu, !ok(z));
        // first probe index from which all larger probes pass
        const int k = bad ? (32 - __clz(bad)) : 0;  // one past the highest failing lane
        const double new_lo = (k == 0) ? lo : lo + (hi - lo) * k / 33.0;
        const double new_hi = (k == 32) ? hi : lo + (hi - lo) * (k + 1) / 33.0;
        lo = new_lo;
        hi = new_hi;
    }
    if (lane == 0) zs_out[id] = hi;
}

// Exact FP64 o-GTO integrals I^o_nl(r) and dI^o_nl/dr at n_pts distances: one thread per (point, l).
// I_nl(r) = pi^1.5 N_n c^l r^l (c + d_n)^-a G(a, b, r);  dG/dr = 2c^2 r/(c+d) G(a+1, b+1) - 2 c r G(a, b).
__global__ void k_radial_fp64(int64_t n_pts, const double* __restrict__ r_in, int n_max, int l_max, double c,
                              const double* __restrict__ gto, const double* __restrict__ T,
                              const double* __restrict__ zs, double* __restrict__ out, double* __restrict__ dout) {
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int L1 = l_max + 1;
    if (id >= n_pts * L1) return;
    const int64_t pt = id / L1;
    const int l = (int)(id % L1);
    const double r = r_in[pt];
    const double* dn = gto;
    const double* Nn = gto + (n_max + 1);
    double raw[kMaxNMax], draw[kMaxNMax];
    const double pi15 = 5.568327996831707845;  // pi^1.5
    for (int n = 0; n < n_max; ++n) {
        const double a = 0.5 * (n + l + 3), b = l + 1.5;
        const double d = dn[n];
        const double pref = pi15 * Nn[n] * exp(l * log(c) - a * log(c + d));
        const double g = g_eval(a, b, c, d, r, zs[n * (l_max + 2) + l]);
        const double rl = (l == 0) ? 1.0 : pow(r, (double)l);
        raw[n] = pref * rl * g;
        if (dout) {
            const double g1 = g_eval(a + 1.0, b + 1.0, c, d, r, zs[(n + 1) * (l_max + 2) + (l + 1)]);
            const double dg = 2.0 * c * c * r / (c + d) * g1 - 2.0 * c * r * g;
            const double drl = (l == 0) ? 0.0 : (l == 1 ? 1.0 : l * pow(r, (double)(l - 1)));
            draw[n] = pref * (drl * g + rl * dg);
        }
    }
    for (int n = 0; n < n_max; ++n) {
        double acc = 0.0, dacc = 0.0;
        for (int k = 0; k < n_max; ++k) {
            acc += T[n * n_max + k] * raw[k];
            if (dout) dacc += T[n * n_max + k] * draw[k];
        }
        out[(pt * n_max + n) * L1 + l] = acc;
        if (dout) dout[(pt * n_max + n) * L1 + l] = dacc;
    }
}

// Clamped cubic spline through y_k = I(r_k), r_k = k delta, with y'(0), y'(r_cut) exact: Thomas algorithm per
// function f = (l, n). y: [M+1][n_max][L1] (exact table), dy: [2][n_max][L1] end slopes, y2 out: [F][M+1].
__global__ void k_spline_solve(int M, int n_max, int L1, double delta, const double* __restrict__ y,
                               const double* __restrict__ dy, double* __restrict__ cp, double* __restrict__ y2) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    const int F = n_max * L1;
    if (f >= F) return;
    const int l = f / n_max, n = f % n_max;
    auto Y = [&](int k) { return y[((int64_t)k * n_max + n) * L1 + l]; };
    double* c = cp + (int64_t)f * (M + 1);
    double* x = y2 + (int64_t)f * (M + 1);
    const double sub = delta / 6.0;
    // row 0
    double b = delta / 3.0;
    double rhs = (Y(1) - Y(0)) / delta - dy[(0 * n_max + n) * L1 + l];
    c[0] = sub / b;
    x[0] = rhs / b;
    for (int k = 1; k <= M; ++k) {
        const double bk = (k == M) ? delta / 3.0 : 2.0 * delta / 3.0;
        const double rk = (k == M) ? dy[(1 * n_max + n) * L1 + l] - (Y(M) - Y(M - 1)) / delta
                                   : (Y(k + 1) - Y(k)) / delta - (Y(k) - Y(k - 1)) / delta;
        const double den = bk - sub * c[k - 1];
        c[k] = (k == M) ? 0.0 : sub / den;
        x[k] = (rk - sub * x[k - 1]) / den;
    }
    for (int k = M - 1; k >= 0; --k) x[k] = x[k] - c[k] * x[k + 1];
}

// Per-interval FP32 polynomial coefficients in u = r/delta - k in [0, 1]:
// y = c0 + u c1 + u^2 c2 + u^3 c3 with c0 = y_k, c1 = (y_{k+1} - y_k) - delta^2 (2 y''_k + y''_{k+1})/6,
// c2 = delta^2 y''_k / 2, c3 = delta^2 (y''_{k+1} - y''_k)/6 (the Numerical Recipes form expanded in u).
__global__ void k_spline_coeffs(int M, int n_max, int L1, double delta, const double* __restrict__ y,
                                const double* __restrict__ y2, float4* __restrict__ table) {
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int F = n_max * L1;
    if (id >= (int64_t)M * F) return;
    const int k = (int)(id / F), f = (int)(id % F);
    const int l = f / n_max, n = f % n_max;
    const double yk = y[((int64_t)k * n_max + n) * L1 + l], yk1 = y[((int64_t)(k + 1) * n_max + n) * L1 + l];
    const double s0 = y2[(int64_t)f * (M + 1) + k], s1 = y2[(int64_t)f * (M + 1) + k + 1];
    const double d2 = delta * delta;
    table[id] = make_float4((float)yk, (float)((yk1 - yk) - d2 * (2.0 * s0 + s1) / 6.0), (float)(d2 * s0 / 2.0),
                            (float)(d2 * (s1 - s0) / 6.0));
}

__device__ inline void atomic_max_pos_double(double* addr, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// Max |spline - exact| at interval midpoints, for the FP64 spline and for the FP32 coefficients.
__global__ void k_spline_error(int M, int n_max, int L1, const double* __restrict__ y, const double* __restrict__ y2,
                               double delta, const float4* __restrict__ table, const double* __restrict__ exact_mid,
                               double* err) {
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int F = n_max * L1;
    if (id >= (int64_t)M * F) return;
    const int k = (int)(id / F), f = (int)(id % F);
    const int l = f / n_max, n = f % n_max;
    const double yk = y[((int64_t)k * n_max + n) * L1 + l], yk1 = y[((int64_t)(k + 1) * n_max + n) * L1 + l];
    const double s0 = y2[(int64_t)f * (M + 1) + k], s1 = y2[(int64_t)f * (M + 1) + k + 1];
    const double A = 0.5, B = 0.5;
    const double v64 = A * yk + B * yk1 + ((A * A * A - A) * s0 + (B * B * B - B) * s1) * delta * delta / 6.0;
    const float4 t = table[id];
    const float u = 0.5f;
    const float v32 = t.x + u * (t.y + u * (t.z + u * t.w));
    const double ex = exact_mid[((int64_t)k * n_max + n) * L1 + l];
    atomic_max_pos_double(err, fabs(v64 - ex));
    atomic_max_pos_double(err + 1, fabs((double)v32 - ex));
}

__global__ void k_fill_grid(int64_t n, double step, double offset, double* r) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) r[i] = offset + step * i;
}

// Exact FP64 DVR integrals and r-derivatives at n_pts distances: one thread per (point, n); layout as k_radial_fp64.
__global__ void k_radial_dvr_fp64(int64_t n_pts, const double* __restrict__ r_in, int n_max, int l_max, double a,
                                  const double* __restrict__ dvr, double* __restrict__ out, double* __restrict__ dout) {
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= n_pts * n_max) return;
    const int64_t pt = id / n_max;
    const int n = (int)(id % n_max);
    const int L1 = l_max + 1;
    double I[kMaxLMax + 1], dI[kMaxLMax + 1];
    dvr_radial(l_max, a, dvr[n], dvr[n_max + n], r_in[pt], I, dout ? dI : nullptr);
    for (int l = 0; l < L1; ++l) {
        out[(pt * n_max + n) * L1 + l] = I[l];
        if (dout) dout[(pt * n_max + n) * L1 + l] = dI[l];
    }
}

// Gauss-Legendre points and weights on [0, X] (host, FP64): Newton iterations on the Legendre polynomial P_n,
// evaluated by its three-term recurrence, from the cosine estimates of the roots.
static void gauss_legendre(int n, double X, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double t = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;  // P_0, P_1
            for (int k = 1; k < n; ++k) {
                const double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            const double pn = (n == 0) ? 1.0 : p1, pm = (n == 1) ? 1.0 : p0;  // P_n, P_{n-1}
            dp = n * (t * pn - pm) / (t * t - 1.0);
            const double dt = pn / dp;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        // recompute P_n'(t) at the converged root for the weight
        double p0 = 1.0, p1 = t;
        for (int k = 1; k < n; ++k) {
            const double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
            p0 = p1;
            p1 = p2;
        }
        dp = n * (t * p1 - (n == 1 ? 1.0 : p0)) / (t * t - 1.0);
        x[n - 1 - i] = 0.5 * X * (t + 1.0);  // ascending
        w[n - 1 - i] = 0.5 * X * 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

static int launch_radial_fp64(rascal_ctx* ctx, int64_t n_pts, const double* d_r, double* out, double* dout) {
    const int L1 = ctx->l_max + 1;
    const int64_t threads = n_pts * L1;
    if (threads == 0) return RASCAL_OK;
    const double c = 1.0 / (2.0 * ctx->sigma * ctx->sigma);
    if (ctx->basis == RASCAL_BASIS_DVR) {
        const int64_t nt = n_pts * ctx->n_max;
        k_radial_dvr_fp64<<<(unsigned)div_up(nt, 128), 128, 0, ctx->stream>>>(n_pts, d_r, ctx->n_max, ctx->l_max, c,
                                                                             ctx->d_dvr, out, dout);
        RASCAL_LAUNCH_CHECK("k_radial_dvr_fp64");
        return RASCAL_OK;
    }
    k_radial_fp64<<<(unsigned)div_up(threads, 128), 128, 0, ctx->stream>>>(n_pts, d_r, ctx->n_max, ctx->l_max, c, ctx->d_gto,
                                                                          ctx->d_T, ctx->d_switch, out, dout);
    RASCAL_LAUNCH_CHECK("k_radial_fp64");
    return RASCAL_OK;
}

// Exact FP64 integrals on the uniform grid r_k = k r_cut/M (y [(M+1)][n_max][L1]), end slopes, and the clamped
// spline second derivatives (y2 [F][M+1]); used for the MLP training targets.
int radial_grid_fp64(rascal_ctx* ctx, int M, double* grid, double* ends, double* y, double* yend, double* dyend,
                     double* cp, double* y2) {
    const int n_max = ctx->n_max, L1 = ctx->l_max + 1, F = ctx->F;
    const double delta = ctx->r_cut / M;
    int st;
    k_fill_grid<<<div_up(M + 1, 256), 256, 0, ctx->stream>>>(M + 1, delta, 0.0, grid);
    RASCAL_LAUNCH_CHECK("k_fill_grid");
    k_fill_grid<<<1, 32, 0, ctx->stream>>>(2, ctx->r_cut, 0.0, ends);
    RASCAL_LAUNCH_CHECK("k_fill_grid");
    if ((st = launch_radial_fp64(ctx, M + 1, grid, y, nullptr))) return st;
    if ((st = launch_radial_fp64(ctx, 2, ends, yend, dyend))) return st;
    k_spline_solve<<<div_up(F, 64), 64, 0, ctx->stream>>>(M, n_max, L1, delta, y, dyend, cp, y2);
    RASCAL_LAUNCH_CHECK("k_spline_solve");
    return RASCAL_OK;
}

static int build_table(rascal_ctx* ctx, int M, double* errs_host) {
    const int n_max = ctx->n_max, L1 = ctx->l_max + 1, F = ctx->F;
    const double delta = ctx->r_cut / M;
    // device buffers: grid r [M+1], mids [M], ends [2]; exact y [(M+1) F], mid [M F], dy ends [2 F]; cp, y2 [F (M+1)]
    const size_t bytes = carve_bytes((M + 1) * 8, M * 8, 2 * 8, (size_t)(M + 1) * F * 8, (size_t)M * F * 8,
                                     (size_t)2 * F * 8, (size_t)2 * F * 8, (size_t)F * (M + 1) * 8, (size_t)F * (M + 1) * 8, 2 * 8);
    void* base;
    int st = arena_get(ctx->scratch, bytes, &base);
    if (st) return st;
    Carver cv(base);
    double* grid = cv.take<double>(M + 1);
    double* mids = cv.take<double>(M);
    double* ends = cv.take<double>(2);
    double* y = cv.take<double>((size_t)(M + 1) * F);
    double* ymid = cv.take<double>((size_t)M * F);
    double* yend = cv.take<double>((size_t)2 * F);
    double* dyend = cv.take<double>((size_t)2 * F);
    double* cp = cv.take<double>((size_t)F * (M + 1));
    double* y2 = cv.take<double>((size_t)F * (M + 1));
    double* err = cv.take<double>(2);
    k_fill_grid<<<div_up(M + 1, 256), 256, 0, ctx->stream>>>(M + 1, delta, 0.0, grid);
    RASCAL_LAUNCH_CHECK("k_fill_grid");
    k_fill_grid<<<div_up(M, 256), 256, 0, ctx->stream>>>(M, delta, 0.5 * delta, mids);
    RASCAL_LAUNCH_CHECK("k_fill_grid");
    k_fill_grid<<<1, 32, 0, ctx->stream>>>(2, ctx->r_cut, 0.0, ends);
    RASCAL_LAUNCH_CHECK("k_fill_grid");
    if ((st = launch_radial_fp64(ctx, M + 1, grid, y, nullptr))) return st;
    if ((st = launch_radial_fp64(ctx, M, mids, ymid, nullptr))) return st;
    if ((st = launch_radial_fp64(ctx, 2, ends, yend, dyend))) return st;
    k_spline_solve<<<div_up(F, 64), 64, 0, ctx->stream>>>(M, n_max, L1, delta, y, dyend, cp, y2);
    RASCAL_LAUNCH_CHECK("k_spline_solve");
    if (ctx->d_table) cudaFree(ctx->d_table);
    ctx->d_table = nullptr;
    RASCAL_CUDA(cudaMalloc(&ctx->d_table, sizeof(float4) * (size_t)M * F));
    k_spline_coeffs<<<(unsigned)div_up((int64_t)M * F, 256), 256, 0, ctx->stream>>>(M, n_max, L1, delta, y, y2, ctx->d_table);
    RASCAL_LAUNCH_CHECK("k_spline_coeffs");
    RASCAL_CUDA(cudaMemsetAsync(err, 0, 2 * sizeof(double), ctx->stream));
    k_spline_error<<<(unsigned)div_up((int64_t)M * F, 256), 256, 0, ctx->stream>>>(M, n_max, L1, y, y2, delta, ctx->d_table,
                                                                                   ymid, err);
    RASCAL_LAUNCH_CHECK("k_spline_error");
    RASCAL_CUDA(cudaMemcpyAsync(errs_host, err, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    RASCAL_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->M = M;
    ctx->inv_delta = (float)(M / ctx->r_cut);
    return RASCAL_OK;
}

}  // namespace rascal

using namespace rascal;

extern "C" const char* rascal_last_error(void) { return g_last_error.c_str(); }

extern "C" long long rascal_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" int rascal_debug_gauss_legendre(int n, double X, double* x, double* w) {
    clear_error();
    if (n < 1 || n > 64 || !(X > 0.0) || !x || !w) return set_error(RASCAL_E_ARG, "n in [1, 64], X > 0, non-NULL outputs");
    gauss_legendre(n, X, x, w);
    return RASCAL_OK;
}

extern "C" void rascal_destroy(rascal_ctx* ctx) {
    if (!ctx) return;
    cudaFree(ctx->d_table);
    cudaFree(ctx->d_T);
    cudaFree(ctx->d_gto);
    cudaFree(ctx->d_switch);
    cudaFree(ctx->d_lut);
    cudaFree(ctx->d_flags);
    cudaFree(ctx->d_tasks);
    cudaFree(ctx->d_fmap);
    cudaFree(ctx->d_pstasks);
    cudaFree(ctx->mlp_params);
    cudaFree(ctx->mlp_m);
    cudaFree(ctx->mlp_v);
    cudaFree(ctx->mlp_grad);
    cudaFree(ctx->mlp_scale);
    cudaFree(ctx->mlp_w2t);
    cudaFree(ctx->mlp_w3t);
    cudaFreeHost(ctx->h_flags);
    cudaFreeHost(ctx->h_pinned);
    cudaFree(ctx->scratch.ptr);
    cudaFree(ctx->scratch_w.ptr);
    cudaFree(ctx->d_dvr);
    lsoap_free(ctx);
    cudaFree(ctx->scratch_sel.ptr);
    cudaFree(ctx->scratch2.ptr);
    delete ctx;
}

static int create_impl(const rascal_hypers* h, void* stream, rascal_ctx** out) {
    if (!h || !out) return set_error(RASCAL_E_ARG, "NULL hypers or output pointer");
    *out = nullptr;
    if (!(h->r_cut > 0.0) || !(h->sigma > 0.0)) return set_error(RASCAL_E_ARG, "r_cut and sigma must be positive");
    if (!(h->smooth_width > 0.0) || h->smooth_width > h->r_cut)
        return set_error(RASCAL_E_ARG, "smooth_width must be in (0, r_cut]");
    if (h->n_max < 1 || h->n_max > kMaxNMax) return set_error(RASCAL_E_ARG, "n_max must be in [1, %d]", kMaxNMax);
    if (h->l_max < 0 || h->l_max > kMaxLMax) return set_error(RASCAL_E_ARG, "l_max must be in [0, %d]", kMaxLMax);
    if (h->n_species < 1 || h->n_species > kMaxSpecies || !h->species)
        return set_error(RASCAL_E_ARG, "n_species must be in [1, %d] with a species list", kMaxSpecies);
    if (h->n_species * h->n_max > kMaxQ) return set_error(RASCAL_E_ARG, "n_species*n_max must be <= %d", kMaxQ);
    if (h->radial < 0 || h->radial > 2) return set_error(RASCAL_E_ARG, "unknown radial mode %d", h->radial);
    if (h->radial_basis != RASCAL_BASIS_GTO && h->radial_basis != RASCAL_BASIS_DVR)
        return set_error(RASCAL_E_ARG, "unknown radial basis %d", h->radial_basis);
    std::vector<int> sp(h->species, h->species + h->n_species);
    std::sort(sp.begin(), sp.end());
    for (int i = 0; i < h->n_species; ++i) {
        if (sp[i] < 0 || sp[i] > 255) return set_error(RASCAL_E_ARG, "species labels must be in [0, 255]");
        if (i && sp[i] == sp[i - 1]) return set_error(RASCAL_E_ARG, "duplicate species label %d", sp[i]);
    }
    int M0 = h->spline_intervals;
    if (M0 < 0 || M0 > 65536) return set_error(RASCAL_E_ARG, "spline_intervals must be in [0, 65536]");
    if (M0 > 0 && M0 < 2) return set_error(RASCAL_E_ARG, "spline_intervals must be >= 2");
    const double acc = h->spline_accuracy > 0 ? h->spline_accuracy : 1e-8;

    rascal_ctx* ctx = new rascal_ctx();
    std::memset(ctx, 0, sizeof(*ctx));
    ctx->r_cut = h->r_cut;
    ctx->smooth_width = h->smooth_width;
    ctx->sigma = h->sigma;
    ctx->n_max = h->n_max;
    ctx->l_max = h->l_max;
    ctx->n_species = h->n_species;
    ctx->radial = h->radial;
    ctx->orthonormal = h->orthonormal ? 1 : 0;
    ctx->basis = h->radial_basis;
    ctx->include_center = h->include_center ? 1 : 0;
    ctx->ps_norm = h->ps_norm ? 1 : 0;
    for (int i = 0; i < h->n_species; ++i) ctx->species[i] = sp[i];
    ctx->stream = static_cast<cudaStream_t>(stream);
    ctx->n_lm = (h->l_max + 1) * (h->l_max + 1);
    ctx->F = h->n_max * (h->l_max + 1);
    ctx->Q = h->n_species * h->n_max;
    *out = ctx;  // destroyed by the caller path on failure

    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e != cudaSuccess) return set_error(RASCAL_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    RASCAL_CUDA(cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, ctx->device));
    const int n_max = h->n_max, L2 = h->l_max + 2;
    RASCAL_CUDA(cudaMalloc(&ctx->d_gto, sizeof(double) * 3 * (n_max + 1)));
    RASCAL_CUDA(cudaMalloc(&ctx->d_T, sizeof(double) * n_max * n_max));
    RASCAL_CUDA(cudaMalloc(&ctx->d_switch, sizeof(double) * (n_max + 1) * L2));
    if (ctx->basis == RASCAL_BASIS_DVR) {
        std::vector<double> xw(2 * n_max);
        gauss_legendre(n_max, h->r_cut + 3.0 * h->sigma, xw.data(), xw.data() + n_max);
        RASCAL_CUDA(cudaMalloc(&ctx->d_dvr, sizeof(double) * 2 * n_max));
        RASCAL_CUDA(cudaMemcpy(ctx->d_dvr, xw.data(), sizeof(double) * 2 * n_max, cudaMemcpyHostToDevice));
    }
    RASCAL_CUDA(cudaMalloc(&ctx->d_lut, sizeof(int) * 256));
    RASCAL_CUDA(cudaMalloc(&ctx->d_flags, sizeof(unsigned)));
    RASCAL_CUDA(cudaMallocHost(&ctx->h_flags, sizeof(unsigned)));
    RASCAL_CUDA(cudaMallocHost(&ctx->h_pinned, sizeof(int64_t) * 8));
    RASCAL_CUDA(cudaMemsetAsync(ctx->d_flags, 0, sizeof(unsigned), ctx->stream));
    int lut[256];
    for (int i = 0; i < 256; ++i) lut[i] = -1;
    for (int i = 0; i < h->n_species; ++i) lut[sp[i]] = i;
    RASCAL_CUDA(cudaMemcpyAsync(ctx->d_lut, lut, sizeof(lut), cudaMemcpyHostToDevice, ctx->stream));

    void* work;
    int st = arena_get(ctx->scratch2, sizeof(double) * 2 * n_max * n_max, &work);
    if (st) return st;
    k_gto_constants<<<1, 32, 0, ctx->stream>>>(n_max, h->r_cut, ctx->orthonormal, ctx->d_gto, ctx->d_T,
                                               static_cast<double*>(work));
    RASCAL_LAUNCH_CHECK("k_gto_constants");
    k_switch_points<<<(n_max + 1) * L2, 32, 0, ctx->stream>>>(n_max, h->l_max, ctx->d_switch);
    RASCAL_LAUNCH_CHECK("k_switch_points");

    double errs[2];
    int M = M0 > 0 ? M0 : 64;
    for (;;) {
        if ((st = build_table(ctx, M, errs))) return st;
        if (M0 > 0 || errs[0] <= acc || M >= 8192) break;
        M *= 2;
    }
    ctx->spline_error = errs[0];
    ctx->spline_error_fp32 = errs[1];
    if ((st = expansion_setup(ctx))) return st;
    if ((st = power_spectrum_setup(ctx))) return st;
    if ((st = gradients_setup(ctx))) return st;
    if ((st = mlp_setup(ctx))) return st;
    if ((st = nbr_static_prepare(ctx))) return st;
    RASCAL_CUDA(cudaStreamSynchronize(ctx->stream));
    return RASCAL_OK;
}

extern "C" int rascal_create(const rascal_hypers* h, void* stream, rascal_ctx** out) {
    clear_error();
    int st = create_impl(h, stream, out);
    if (st != RASCAL_OK && out && *out) {
        rascal_destroy(*out);
        *out = nullptr;
    }
    return st;
}

extern "C" int rascal_set_radial(rascal_ctx* ctx, int radial) {
    clear_error();
    if (!ctx) return set_error(RASCAL_E_ARG, "NULL context");
    if (radial < RASCAL_RADIAL_SPLINE || radial > RASCAL_RADIAL_MLP) return set_error(RASCAL_E_ARG, "unknown radial mode %d", radial);
    ctx->radial = radial;
    return RASCAL_OK;
}

extern "C" int rascal_set_stream(rascal_ctx* ctx, void* stream) {
    if (!ctx) return set_error(RASCAL_E_ARG, "NULL context");
    ctx->stream = static_cast<cudaStream_t>(stream);
    return RASCAL_OK;
}

extern "C" int rascal_info(const rascal_ctx* ctx, rascal_info_t* o) {
    if (!ctx || !o) return set_error(RASCAL_E_ARG, "NULL argument");
    o->n_species = ctx->n_species;
    o->n_max = ctx->n_max;
    o->l_max = ctx->l_max;
    o->n_lm = ctx->n_lm;
    o->coeffs_per_centre = (int64_t)ctx->Q * ctx->n_lm;
    o->features_packed = (int64_t)(ctx->l_max + 1) * ctx->Q * (ctx->Q + 1) / 2;
    o->features_full = (int64_t)(ctx->l_max + 1) * ctx->Q * ctx->Q;
    o->spline_intervals = ctx->M;
    o->spline_error = ctx->spline_error;
    o->spline_error_fp32 = ctx->spline_error_fp32;
    o->scratch_bytes = (int64_t)(ctx->scratch.bytes + ctx->scratch2.bytes + ctx->scratch_w.bytes + ctx->scratch_sel.bytes);
    return RASCAL_OK;
}

extern "C" int rascal_radial_exact_fp64(rascal_ctx* ctx, int64_t n_points, const double* d_r, double* d_out,
                                        double* d_dout) {
    clear_error();
    if (!ctx || n_points < 0 || (n_points > 0 && (!d_r || !d_out))) return set_error(RASCAL_E_ARG, "bad argument");
    return launch_radial_fp64(ctx, n_points, d_r, d_out, d_dout);
}

extern "C" int rascal_debug_wait_timeout(rascal_ctx* ctx, unsigned polls) {
    clear_error();
    if (!ctx) return set_error(RASCAL_E_ARG, "NULL context");
    ctx->stall_polls = polls;
    return RASCAL_OK;
}

extern "C" int rascal_sync(rascal_ctx* ctx) {
    clear_error();
    if (!ctx) return set_error(RASCAL_E_ARG, "NULL context");
    return check_flags(ctx);
}
