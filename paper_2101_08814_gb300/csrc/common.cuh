// Internal helpers shared by the library's translation units: status handling, the context, scratch arena and
// small device utilities. Nothing here is part of the public ABI (include/rascal.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>

#include "rascal.h"

namespace rascal {

// -------------------------------------------------------------------------------------------- limits
constexpr int kMaxNMax = 32;
constexpr int kMaxLMax = 15;
constexpr int kMaxSpecies = 16;
constexpr int kMaxQ = 256;
constexpr int kMaxShift = 511;  // |n_k| that fits the 10-bit fields of the pair sort key

// device-side error flags (bitwise OR into ctx->d_flags)
enum : unsigned {
    kFlagSpecies = 1u << 0,     // an atom's label is not in the hypers' species list
    kFlagGeometry = 1u << 1,    // singular cell or coincident atoms
    kFlagThinCell = 1u << 2,    // perpendicular cell width below r_cut / 64
    kFlagShiftRange = 1u << 3,  // |n_k| above kMaxShift
    kFlagBadOffsets = 1u << 4,  // structure offsets not increasing / out of range
    kFlagTimeout = 1u << 5,     // a bounded wait on a tensor-core completion barrier ran out
    kFlagSelection = 1u << 6,   // a selected feature index is outside the packed feature vector
    kFlagNonFinite = 1u << 7,   // an atom position is NaN or infinite
};

// -------------------------------------------------------------------------------------------- status
int set_error(int code, const char* fmt, ...);
void clear_error();
#define RASCAL_CUDA(call)                                                                               \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return ::rascal::set_error(RASCAL_E_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                             \
    } while (0)
// Every kernel launch is followed by exactly one RASCAL_LAUNCH_CHECK: it counts the launch (see
// rascal_launch_count) and turns a launch error into RASCAL_E_CUDA.
void count_launch();
#define RASCAL_LAUNCH_CHECK(what)                                                                       \
    do {                                                                                                \
        ::rascal::count_launch();                                                                       \
        cudaError_t e_ = cudaGetLastError();                                                            \
        if (e_ != cudaSuccess)                                                                          \
            return ::rascal::set_error(RASCAL_E_CUDA, "launch of %s failed: %s", what, cudaGetErrorString(e_)); \
    } while (0)

// -------------------------------------------------------------------------------------------- context
struct Arena {
    void* ptr = nullptr;
    size_t bytes = 0;
};

// Launch plan of the pair/expansion kernels, derived from the hypers once per context.
//   padded radial index: n in [0, n_pad), n_pad = n_max rounded up to 4
//   padded angular index: per l a block of mp(l) = 4*ceil((2l+1)/4) slots, slot s <-> m = s - l (s <= 2l valid),
//   block start lp(l); Lp = sum_l mp(l)
//   a task is (l, n-tile of 4, m-tile of 4) of one species: T_s tasks per species, W_s warps per species,
//   S_c species accumulated concurrently, rounds = ceil(n_species / S_c)
struct LsoapTable;  // lambda-SOAP coupling tables (lambda_soap.cu)

// Hyper shapes with their own compiled instances of the fused FP32 kernel (expansion.cu) and the gradient kernel
// (gradients.cu): the batch, large, diff and MLP workloads' n_max, l_max and species count. Index 0 stands for the
// runtime-shaped kernels, which serve every other shape. The derived sizes below mirror the host plan (make_plan,
// make_gram); the host launches a shaped instance only when every one of them equals the plan's value.
struct ExpShape {
    int n_max, l_max, S;
};
constexpr ExpShape kExpShapes[] = {{0, 0, 0}, {12, 9, 4}, {10, 8, 3}, {8, 6, 2}, {16, 12, 8}};
constexpr int kNumExpShapes = sizeof(kExpShapes) / sizeof(kExpShapes[0]);
constexpr int exp_npad(int n_max) { return (n_max + 3) / 4 * 4; }
// Y row offset of l: sum over l' < l of ceil4(2l' + 1), i.e. 4 k (k + 1) for l = 2k and 4 (k + 1)^2 for l = 2k + 1
constexpr int exp_lp(int l) { return (l & 1) ? 4 * ((l >> 1) + 1) * ((l >> 1) + 1) : 4 * (l >> 1) * ((l >> 1) + 1); }
constexpr int exp_ly(int l_max) { return (exp_lp(l_max + 1) / 4 | 1) * 4; }
constexpr int exp_qp(int Q) { return ((Q + 3) / 4 | 1) * 4; }
constexpr int exp_ts(int n_max, int l_max) { return exp_npad(n_max) / 4 * (exp_lp(l_max + 1) / 4); }
constexpr int exp_sc(int n_max, int l_max, int S) {
    const int w = (exp_ts(n_max, l_max) + 31) / 32;
    return w > 16 ? 1 : (16 / w < S ? (16 / w < 1 ? 1 : 16 / w) : S);
}
constexpr size_t exp_pair_smem(int n_max, int l_max, int chunk) {
    const int fpad = (l_max + 1) * exp_npad(n_max);
    return (size_t)chunk * 16 + (size_t)chunk * (fpad + exp_ly(l_max)) * 4 + (size_t)chunk * 12 +
           (size_t)(kMaxSpecies + 1 + kMaxLMax + 2 + fpad) * 4 + 64;
}
constexpr int exp_chunk(int n_max, int l_max) {
    int chunk = 32;  // about 30 KB for n_max 12, l_max 9: four CTAs per SM
    while (chunk > 8 && exp_pair_smem(n_max, l_max, chunk) > 56 * 1024) chunk /= 2;
    return chunk;
}

struct ExpPlan {
    int n_pad, F_pad, Lp;
    int Ly;           // Y row pitch in the expansion kernel: Lp rounded up so that Ly / 4 is odd (conflict-free rows)
    int lp[kMaxLMax + 2];
    int T_s, W_s, S_c, rounds, threads;
    int chunk;        // pairs staged per chunk
    size_t smem;      // dynamic shared memory of the expansion kernel
    size_t smem_ps;   // extra dynamic shared memory when the power spectrum is fused
};

}  // namespace rascal

struct rascal_ctx {
    // hypers (copied)
    double r_cut, smooth_width, sigma;
    int n_max, l_max, n_species, radial, orthonormal, include_center, ps_norm;
    int species[rascal::kMaxSpecies];  // sorted labels
    cudaStream_t stream;
    int device;
    int n_sm;

    // derived
    int n_lm;        // (l_max+1)^2
    int F;           // n_max * (l_max+1) radial functions, index f = l*n_max + n
    int Q;           // n_species * n_max

    // radial table: FP32 cubic coefficients per interval, [M][F] float4 (c0 + u c1 + u^2 c2 + u^3 c3, u in [0,1])
    float4* d_table;
    int M;
    float inv_delta;  // M / r_cut
    double spline_error, spline_error_fp32;

    // FP64 constants on the device
    double* d_T;        // [n_max][n_max] S^-1/2 (identity when orthonormal == 0)
    double* d_gto;      // [3][n_max+1]: d_n, N_n, (unused) for n = 0..n_max
    double* d_switch;   // [(n_max+1)][(l_max+2)] series/asymptotic switch points of G(a,b)
    int basis;          // RASCAL_BASIS_GTO or RASCAL_BASIS_DVR
    double* d_dvr;      // [2][n_max]: Gauss-Legendre points x_n and weights w_n on [0, r_cut + 3 sigma] (DVR basis)
    int* d_lut;         // [256] label -> species index or -1

    unsigned* d_flags;  // device error flags (see kFlag*)
    unsigned stall_polls;  // test hook: > 0 makes the fused tensor-core Gram's first completion wait run out
    unsigned* h_flags;  // pinned host mirror

    rascal::Arena scratch;  // grown on demand, reused across calls
    rascal::Arena scratch2;
    rascal::Arena scratch_w;  // dense symmetric weight blocks of the gradient kernel
    rascal::Arena scratch_sel;  // decoded feature selection of rascal_soap_selected
    int64_t* h_pinned;      // pinned host words for small read-backs

    rascal::ExpPlan plan;
    int* d_tasks;   // [T_s] packed (l, n-tile, m-tile) of the accumulation tasks
    int* d_fmap;    // [F_pad] table column (l*n_max + n) of a padded radial slot, -1 for padding
    int* d_pstasks; // power-spectrum tasks, see power_spectrum.cu
    int n_pstasks;

    // MLP surrogate of the radial integrals (mlp.cu); mlp_params == NULL until parameters are set
    float* mlp_params;   // FP32 master parameters
    float* mlp_m;        // Adam moments
    float* mlp_v;
    float* mlp_grad;
    float* mlp_scale;    // [F] output scales
    void* mlp_w2t;       // BF16 operand tiles for the tensor-core inference
    void* mlp_w3t;
    int mlp_hidden, mlp_step;

    // real Clebsch-Gordan tables of the nu = 2 equivariants, built on first use per lambda (lambda_soap.cu)
    rascal::LsoapTable* lsoap[2 * rascal::kMaxLMax + 1];
};

namespace rascal {

// Returns a device buffer of at least `bytes` from the arena (grows it, never shrinks). Not thread-safe per ctx.
int arena_get(Arena& a, size_t bytes, void** out);
// Turns device flags into a status (after the stream has been synchronised), then clears them.
int check_flags(rascal_ctx* ctx);

// round up
__host__ __device__ inline int64_t div_up(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline size_t align_up(size_t a, size_t b) { return (a + b - 1) / b * b; }

// Carves consecutive, 256-byte aligned sub-buffers out of one scratch allocation.
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base(static_cast<char*>(b)) {}
    template <typename T>
    T* take(size_t count) {
        T* p = reinterpret_cast<T*>(base + off);
        off = align_up(off + count * sizeof(T), 256);
        return p;
    }
};
template <typename... Ts>
inline size_t carve_bytes(Ts... sizes) {
    size_t s = 0;
    for (size_t x : {static_cast<size_t>(sizes)...}) s += align_up(x, 256);
    return s;
}

// device-wide exclusive scan: out[0..n] with out[n] = total; in and out may alias. Input int32 or int64.
int scan_exclusive(const int* in, int64_t* out, int64_t n, cudaStream_t stream, Arena& scratch);
int scan_exclusive(const int64_t* in, int64_t* out, int64_t n, cudaStream_t stream, Arena& scratch);
// the same with a caller-provided tile-sum buffer of scan_tile_sums_len(n) words (no allocation)
int64_t scan_tile_sums_len(int64_t n);
int scan_exclusive_into(const int* in, int64_t* out, int64_t n, cudaStream_t stream, int64_t* sums);
int scan_exclusive_into(const int64_t* in, int64_t* out, int64_t n, cudaStream_t stream, int64_t* sums);

int validate_system(const rascal_ctx* ctx, const rascal_system* sys);

int radial_grid_fp64(rascal_ctx* ctx, int M, double* grid, double* ends, double* y, double* yend, double* dyend,
                     double* cp, double* y2);
// MLP surrogate (mlp.cu): batched inference on the tensor cores; per-pair radial values of the EXACT mode
int mlp_infer(rascal_ctx* ctx, int64_t n, const float4* rij, const float* r, float* out, float* dout);
int radial_exact_pairs(rascal_ctx* ctx, int64_t n, const float4* rij, float* out, float* dout);
int radial_precompute(rascal_ctx* ctx, const rascal_system* sys, const int64_t* d_offsets, const float* d_rij, bool deriv,
                      const float** pre_G, const float** pre_D);

// per-translation-unit setup called from rascal_create
int mlp_setup(rascal_ctx* ctx);
int expansion_setup(rascal_ctx* ctx);
int power_spectrum_setup(rascal_ctx* ctx);
// BF16 / TF32x3 power spectrum of given coefficients [n][Q][n_lm] by the fused kernel's tensor-core Gram
int power_spectrum_tc(rascal_ctx* ctx, int64_t n_centres, const float* d_coeffs, int precision, int layout, float* d_ps);
int gradients_setup(rascal_ctx* ctx);
// caches the device address of the no-allocation neighbour scratch for ctx->device (neighbours.cu)
int nbr_static_prepare(rascal_ctx* ctx);
void lsoap_free(rascal_ctx* ctx);

}  // namespace rascal
