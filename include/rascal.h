/*
 * rascal.h - C ABI of the GB300 (sm_103a) SOAP density-expansion library.
 *
 * What it computes (arXiv:2101.08814):
 *   neighbours      every (i, j, n) with |r_j - r_i + n1 h1 + n2 h2 + n3 h3| < r_cut, periodic images included
 *                   (Appendix B: "r_ji < r_cut", j over periodic replicas)
 *   expansion       c^i_{a n l m} = sum_{j in A_i, a_j = a} f_cut(r_ji) I^o_nl(r_ji) Y_lm(r^_ji)
 *                   (Eq. spherical_expansion_coefficients_gaussians; I^o is the o-GTO radial integral of
 *                   Eq. rad-int-gto-1 orthogonalised with S^-1/2, Sec. 'GTO radial basis'; Y_lm real spherical
 *                   harmonics, Sec. 'Spherical Harmonics'; radial values from a cubic spline, Sec. 'Spline optimization')
 *   power spectrum  p^i_{(a1 n1)(a2 n2) l} = (2l+1)^-1/2 sum_m c^i_{a1 n1 l m} c^i_{a2 n2 l m}  (Eq. nu2-basis-coupled)
 *   gradients       forces -dE/dr_k and virial sum_ij dE/dr_ji (x) r_ji of E = sum_i G_i . p_i
 *                   (Eqs. energy-derivative and energy-virial, Appendix B)
 *
 * Conventions shared by every call:
 *   - Lengths are in Angstrom. Positions are [N][3] float64 and are used as given (not wrapped).
 *   - Cells are [n_structures][3][3] float64, row k is the cell vector h_{k+1}.
 *   - Species are integer labels (e.g. atomic numbers, 0..255). rascal_hypers.species lists the labels in use;
 *     the species index a of a label is its rank in the sorted list. Combined radial/species index q = a*n_max + n.
 *   - c is float32 [n_centres][n_species][n_max][(l_max+1)^2] with lm = l*l + l + m, m = -l..l.
 *   - p PACKED is float32 [n_centres][l_max+1][Q(Q+1)/2], Q = n_species*n_max, pairs q1 <= q2 row-major;
 *     p FULL is float32 [n_centres][l_max+1][Q][Q].
 *   - Every device pointer argument ("d_") is caller-owned device memory; the library only borrows it for the
 *     duration of the call. The context owns the radial table, its scratch arena and the MLP weights.
 *   - All work is enqueued on the context's CUDA stream. Calls that must read a count from the device
 *     (rascal_neighbours) synchronise that stream; the others return as soon as the work is enqueued.
 *   - Every call returns RASCAL_OK (0) or a negative RASCAL_E_* status; rascal_last_error() then holds a
 *     message for the calling thread. No call aborts the process.
 */
#ifndef RASCAL_H
#define RASCAL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RASCAL_OK 0
#define RASCAL_E_ARG (-1)         /* invalid argument (null pointer, out-of-range hyper, unknown species,
                                     non-finite position) */
#define RASCAL_E_CAPACITY (-2)    /* output buffer too small; the required size is reported */
#define RASCAL_E_CUDA (-3)        /* a CUDA runtime call failed */
#define RASCAL_E_UNSUPPORTED (-4) /* valid input outside what the kernels support (e.g. |shift| > 511) */
#define RASCAL_E_GEOMETRY (-5)    /* degenerate geometry: singular cell, coincident atoms (r < 1e-6 A) */
#define RASCAL_E_TIMEOUT (-6)     /* a bounded device-side wait ran out (reported by rascal_sync / the next check) */
#define RASCAL_E_NOMEM (-7)       /* device allocation of context scratch failed */

/* radial integral source */
#define RASCAL_RADIAL_SPLINE 0 /* FP32 cubic spline of the FP64 o-GTO integrals (default) */
#define RASCAL_RADIAL_EXACT 1  /* per-pair 1F1 series/asymptotic + recurrence, FP32 */
#define RASCAL_RADIAL_MLP 2    /* the trained MLP surrogate held by the context */

/* power-spectrum arithmetic */
#define RASCAL_PS_FP32 0   /* FP32 inputs and accumulation (CUDA cores) */
#define RASCAL_PS_BF16 1   /* BF16 inputs, FP32 accumulation (tcgen05 tensor cores) */
#define RASCAL_PS_TF32X3 2 /* FP32 inputs split into TF32 hi + lo, three tcgen05 MMAs, FP32 accumulation:
                              about 2^-21 relative per product, FP32-grade results on tensor cores */

/* radial basis */
#define RASCAL_BASIS_GTO 0 /* Gaussian-type orbitals, Eq. rad-int-gto-1 (orthonormalised unless orthonormal = 0) */
#define RASCAL_BASIS_DVR 1 /* discrete variable representation on Gauss-Legendre points, Eq. rad-int-dvr */

/* power-spectrum layout */
#define RASCAL_LAYOUT_PACKED 0
#define RASCAL_LAYOUT_FULL 1

/* Expansion parameters (paper notation). Limits: 1 <= n_max <= 32, 0 <= l_max <= 15, 1 <= n_species <= 16,
 * n_species*n_max <= 256, 0 < smooth_width <= r_cut, sigma > 0. */
typedef struct {
    double r_cut;            /* cutoff radius r_cut, Angstrom */
    double smooth_width;     /* width w of the cosine cutoff f_cut: 1 below r_cut - w, 0 at r_cut */
    double sigma;            /* Gaussian width sigma of the atom density; c = 1/(2 sigma^2) */
    int n_max;               /* radial functions n = 0..n_max-1 */
    int l_max;               /* angular channels l = 0..l_max */
    int n_species;           /* number of species labels in `species` */
    const int* species;      /* HOST pointer, n_species distinct labels in 0..255, any order */
    int radial;              /* RASCAL_RADIAL_* */
    int orthonormal;         /* 1: o-GTO basis (S^-1/2 applied in FP64), 0: raw GTO */
    int include_center;      /* 1: the centre adds its own r = 0 term to its species block */
    int ps_norm;             /* 1: keep the (2l+1)^-1/2 factor of Eq. nu2-basis-coupled */
    double spline_accuracy;  /* target max |spline - exact| at interval midpoints (FP64 build); <= 0: 1e-8 */
    int spline_intervals;    /* > 0: force this many intervals M; 0: double M from 64 until the accuracy holds */
    int radial_basis;        /* RASCAL_BASIS_GTO or RASCAL_BASIS_DVR. DVR: I_nl(r) = 4 pi x_n sqrt(w_n)
                              * exp(-a (x_n^2 + r^2)) i_l(2 a x_n r), a = 1/(2 sigma^2), on the n_max Gauss-Legendre
                              * points x_n (weights w_n) of [0, r_cut + 3 sigma]; the printed Eq. rad-int-dvr leaves
                              * out the constant 4 pi and the density factor exp(-a r^2), both kept here */
} rascal_hypers;

/* Structures in device memory. Atoms of structure s are struct_offsets[s] .. struct_offsets[s+1]-1. */
typedef struct {
    int n_structures;
    int n_atoms;
    const int* d_struct_offsets; /* [n_structures+1] int32 */
    const double* d_positions;   /* [n_atoms][3] float64 */
    const double* d_cells;       /* [n_structures][3][3] float64, rows h1, h2, h3 */
    const int* d_pbc;            /* [n_structures][3] int32, 1 = periodic along h_k; NULL = all periodic */
    const int* d_species;        /* [n_atoms] int32 labels */
} rascal_system;

typedef struct rascal_ctx rascal_ctx;

/* Sizes derived from the hypers (filled by rascal_info). */
typedef struct {
    int n_species, n_max, l_max;
    int n_lm;                    /* (l_max+1)^2 */
    int64_t coeffs_per_centre;   /* n_species*n_max*n_lm */
    int64_t features_packed;     /* (l_max+1)*Q(Q+1)/2 */
    int64_t features_full;       /* (l_max+1)*Q*Q */
    int spline_intervals;        /* M chosen for the radial table */
    double spline_error;         /* max |FP64 spline - exact| at interval midpoints, over all (n, l) */
    double spline_error_fp32;    /* the same for the FP32 coefficients the kernels read */
    int64_t scratch_bytes;       /* device bytes held by the context's scratch arenas now (they grow on demand) */
} rascal_info_t;

/* Thread-local message of the last failed call on this thread ("" if none). Never NULL. */
const char* rascal_last_error(void);

/* Diagnostics: number of CUDA kernels this library has launched in the process so far (all contexts). */
long long rascal_launch_count(void);

/* Build a context: validates the hypers, computes the GTO constants and the FP64 overlap matrix with its
 * inverse square root (Sec. 'GTO radial basis'), tabulates the o-GTO radial integrals in FP64 on the GPU with
 * the series/asymptotic 1F1 of Appendix A, solves the clamped cubic spline and stores FP32 per-interval
 * coefficients. `cuda_stream` is a cudaStream_t (NULL = legacy default stream). Synchronises the stream. */
int rascal_create(const rascal_hypers* hypers, void* cuda_stream, rascal_ctx** out);
void rascal_destroy(rascal_ctx* ctx);
int rascal_set_stream(rascal_ctx* ctx, void* cuda_stream);
int rascal_info(const rascal_ctx* ctx, rascal_info_t* out);

/* Synchronises the context stream and turns device-side error flags raised by earlier calls (unknown species
 * label, degenerate geometry, ...) into a status. */
int rascal_sync(rascal_ctx* ctx);

/* Test hook for the failure path of the fused tensor-core Gram (no counterpart in the paper). With polls > 0, the
 * first MMA-completion wait of every CTA of rascal_soap (precision BF16 or TF32X3) and of the tensor-core forms of
 * rascal_power_spectrum is made on an mbarrier that nothing arrives at, and gives up after `polls` polls (about
 * 20 ns apart). The kernel then raises the timeout flag, skips the remaining epilogues, waits (with the built-in
 * bound of 2^22 polls) for every MMA it issued and frees its tensor memory; the next synchronising call returns
 * RASCAL_E_TIMEOUT. The outputs of that call are incomplete. polls = 0 switches the hook off; the context stays
 * usable throughout. Returns RASCAL_E_ARG for a NULL context. */
int rascal_debug_wait_timeout(rascal_ctx* ctx, unsigned polls);

/* Test hooks for tables the library builds on the host (no context and no GPU needed; no counterpart in the paper).
 * rascal_debug_gauss_legendre: the n Gauss-Legendre points x[n] (ascending) and weights w[n] on [0, X] on which
 *   the DVR radial basis (Eq. rad-int-dvr) places its functions, in FP64; n in [1, 64] and X > 0, else
 *   RASCAL_E_ARG.
 * rascal_debug_real_coupling: the table R[mu][m1][m2], (2 lambda + 1) (2 l1 + 1) (2 l2 + 1) float32 values, that
 *   couples the real-harmonic coefficients of ranks l1 and l2 (the basis of rascal_spherical_expansion, index
 *   m + l) to the real rank-lambda equivariant of rascal_lambda_soap (Eq. body-order-x at nu = 2: Clebsch-Gordan
 *   coefficients carried into the real basis in FP64 and rounded once). Needs l1, l2 <= 15,
 *   |l1 - l2| <= lambda <= l1 + l2 and l1 + l2 + lambda even, else RASCAL_E_ARG. The caller owns the outputs. */
int rascal_debug_gauss_legendre(int n, double X, double* x, double* w);
int rascal_debug_real_coupling(int l1, int l2, int lambda, float* R);

/* Periodic neighbour list (Appendix B). For every atom i (all structures, in atom order) the pairs (j, n) with
 * |r_j - r_i + n H| < r_cut, (j, n) != (i, 0), sorted by (j, n1, n2, n3). The inclusion test is bit-exact with
 * the FP64 definition d = (r_j - r_i) + ((n1 h1 + n2 h2) + n3 h3), d.d = (dx dx + dy dy) + dz dz < r_cut^2.
 *   d_offsets [n_atoms+1] int64: CSR offsets (written whenever the call gets as far as counting)
 *   d_nbr_j   [capacity] int32: neighbour atom index (global numbering)
 *   d_shift   [capacity][3] int32: n
 *   d_rij     [capacity][4] float32: (x, y, z, |r_ji|) of r_ji = r_j - r_i + n H, accurate to FP32 rounding
 *   n_pairs   host out: the number of pairs P
 * If P > capacity the call returns RASCAL_E_CAPACITY with *n_pairs = P and leaves the pair arrays unwritten.
 * Synchronises the stream once (to read P). Cells with a perpendicular width below r_cut/64 return
 * RASCAL_E_UNSUPPORTED. */
int rascal_neighbours(rascal_ctx* ctx, const rascal_system* sys, int64_t capacity, int64_t* d_offsets,
                      int* d_nbr_j, int* d_shift, float* d_rij, int64_t* n_pairs);

/* rascal_neighbours for callers that cannot allocate device memory while they run (no counterpart in the paper,
 * which describes a serial CPU library). Some callers cannot call cudaMalloc: an MD engine that has reserved the
 * device memory through its own pool allocator, or a time-stepping loop that must not hit cudaMalloc / cudaFree
 * because they synchronise the whole device. This entry point takes the same arguments, launches the same kernels
 * and produces the same output, but carves every scratch buffer out of one file-scope device array of
 * rascal_neighbours_static_limit() bytes (32 MiB) instead of the context's scratch arena; it calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *   - The array is part of the library's device image: every GPU that loads the library holds it until exit.
 *   - rascal_create looks up the array's device address for the context's device (cudaGetSymbolAddress, with
 *     that device current) and caches it, so the calls themselves do no lookup. Make the call with the context's
 *     device current; otherwise it returns RASCAL_E_ARG.
 *   - All calls share the one array and it keeps the last call's contents (what must start at zero is cleared
 *     on every call). Calls that overlap on the GPU (other streams, other contexts, other host threads) race on
 *     it: serialise them.
 *   - Limits: a system needing more scratch than the array (about 116 bytes per atom plus 360 per structure:
 *     some 280k atoms in one cell) is refused with RASCAL_E_UNSUPPORTED before anything runs. A centre with more
 *     than 256 neighbours (rascal_neighbours sorts those in an allocated overflow buffer) is also refused with
 *     RASCAL_E_UNSUPPORTED, but only once the counting pass has run: d_offsets and *n_pairs are then already
 *     written, and this check comes before the capacity check.
 * Synchronises the stream once, like rascal_neighbours. */
int rascal_neighbours_noalloc(rascal_ctx* ctx, const rascal_system* sys, int64_t capacity, int64_t* d_offsets,
                              int* d_nbr_j, int* d_shift, float* d_rij, int64_t* n_pairs);
/* Size in bytes of the device array that rascal_neighbours_noalloc uses for scratch. */
size_t rascal_neighbours_static_limit(void);

/* Spherical expansion coefficients (Eq. spherical_expansion_coefficients_gaussians) of every centre from a pair
 * list made by rascal_neighbours for the same system. d_coeffs: [n_atoms][n_species][n_max][(l_max+1)^2]. */
int rascal_spherical_expansion(rascal_ctx* ctx, const rascal_system* sys, const int64_t* d_offsets,
                               const int* d_nbr_j, const float* d_rij, float* d_coeffs);

/* Test hook for small cases: the per-pair feature gradient written out (Appendix B, Eq. energy-derivative, and
 * Eq. spherical_expansion_coefficients_gaussians). For pair p with r = r_ji = d_rij[p] (the (x, y, z, |r|) rows of a
 * pair list made by rascal_neighbours) it writes
 *   d_dc [n_pairs][3][n_max][(l_max+1)^2] float32:  d/dr_x [ f_cut(r) I^o_nl(r) Y_lm(r^) ],
 * the derivative of that pair's term in c^i_{a_j n l m} with respect to the x-th component of r_ji (its species
 * block is a_j; the other blocks do not depend on this pair). Radial values come from the context's radial mode.
 * rascal_gradients never forms this tensor (it recomputes it per pair inside the contraction); this call exists to
 * check it. n_pairs <= 2^20, else RASCAL_E_ARG. */
int rascal_debug_pair_gradients(rascal_ctx* ctx, int64_t n_pairs, const float* d_rij, float* d_dc);

/* Power spectrum (Eq. nu2-basis-coupled) of n_centres coefficient blocks. precision: RASCAL_PS_FP32 or
 * RASCAL_PS_BF16 (tensor cores, inputs rounded to bfloat16, FP32 accumulation). layout: RASCAL_LAYOUT_*. */
int rascal_power_spectrum(rascal_ctx* ctx, int64_t n_centres, const float* d_coeffs, int precision, int layout,
                          float* d_ps);

/* Expansion and power spectrum in one kernel: each centre's c is written to d_coeffs and kept in shared memory,
 * where its Gram is formed (precision as in rascal_power_spectrum; RASCAL_PS_FP32 uses the CUDA cores, the
 * others tcgen05), so c is never read back from global memory. */
int rascal_soap(rascal_ctx* ctx, const rascal_system* sys, const int64_t* d_offsets, const int* d_nbr_j,
                const float* d_rij, int precision, int layout, float* d_coeffs, float* d_ps);

/* Selected power-spectrum features (sparse feature selection, Sec. "Feature dimensionality reduction"): only the
 * listed PACKED features are computed (FP32, in the fused kernel, from c held in shared memory) and written densely,
 * so the output bytes, which bound the full power spectrum, shrink with the selection.
 *   n_sel >= 1; d_sel [n_sel] int32: indices f = l Q(Q+1)/2 + q1 (2Q - q1 - 1)/2 + q2 (q1 <= q2) into the PACKED
 *     feature vector of rascal_power_spectrum, any order, repeats allowed
 *   d_coeffs [n_atoms][n_species][n_max][(l_max+1)^2] float32: written as by rascal_soap
 *   d_ps [n_atoms][n_sel] float32: d_ps[i][k] = p^i at feature d_sel[k]
 * An index outside [0, features_packed) is reported as RASCAL_E_ARG at the next synchronising call (its output is
 * left zero). */
int rascal_soap_selected(rascal_ctx* ctx, const rascal_system* sys, const int64_t* d_offsets, const int* d_nbr_j,
                         const float* d_rij, int64_t n_sel, const int* d_sel, float* d_coeffs, float* d_ps);

/* Per-structure energy of the additive linear model E = sum_i w_{a_i} . p_i (Eq. additive-energy-model) from
 * PACKED p: d_weights [n_species][features_packed] float32, d_energy [n_structures] float64 (overwritten). */
int rascal_linear_energy(rascal_ctx* ctx, const rascal_system* sys, const float* d_ps_packed,
                         const float* d_weights, double* d_energy);

/* Gradients of E = sum_i G_i . p_i (PACKED p) with respect to the positions and the cell (Appendix B).
 * Exactly one of d_grad_ps ([n_atoms][features_packed], G_i per centre) or d_weights ([n_species]
 * [features_packed], G_i = w_{a_i}, the linear model) must be non-NULL. The pair terms are recomputed per pair
 * from the spline and Y_lm; dc/dr is never stored. Pair terms are summed in FP32 (per-atom force sums in a
 * scratch FP32 array, per-centre virial sums in FP32) and written out as float64; structure sums are FP64.
 * Calls with d_weights build dense symmetric per-species weight blocks in the context's scratch first.
 *   d_forces [n_atoms][3] float64: overwritten with F_k = -dE/dr_k (images of the centre add nothing)
 *   d_virial [n_structures][9] float64: overwritten with V[a][b] = sum_pairs dE/dr_ji[a] r_ji[b] */
int rascal_gradients(rascal_ctx* ctx, const rascal_system* sys, const int64_t* d_offsets, const int* d_nbr_j,
                     const float* d_rij, const float* d_coeffs, const float* d_grad_ps, const float* d_weights,
                     double* d_forces, double* d_virial);

/* Sparse GPR energy model (Eq. sparse-gp) with the polynomial kernel k(M_I, A_i) = (M^_I . p^_i)^zeta, one model
 * per centre species: E_i = sum over the sparse points I of the centre's species of x_I k(M_I, A_i). With
 * normalize = 1 both vectors are unit-normalised (p^ = p/|p|; a centre with p = 0 keeps p^ = 0), else used as given.
 * The contractions run on the tensor cores with TF32 operands (the sparse points are rounded to the nearest TF32
 * value at creation; the features are read as FP32 and truncated to TF32 by the tensor core) and FP32 accumulation:
 * |E_i - exact| <= 2 zeta (2^-10 + 2^-11) sum_I |x_I| for unit vectors, plus FP32 summation.
 *   h_sparse [n_sparse][n_features] float64, h_sparse_species [n_sparse] int32 labels (each one of the context's),
 *   h_weights [n_sparse] float64 (x_I); all host memory, copied. n_features: length of the feature rows the
 *   predictions take (the PACKED power spectrum or a selection of it). zeta in [1, 16].
 * The model lives on the current device; it may be used with any context of the same species list. */
typedef struct rascal_gpr rascal_gpr;
int rascal_gpr_create(rascal_ctx* ctx, int64_t n_sparse, int64_t n_features, const double* h_sparse,
                      const int* h_sparse_species, const double* h_weights, int zeta, int normalize, rascal_gpr** out);
void rascal_gpr_destroy(rascal_gpr* model);

/* Energies of the model for every atom of the system as a centre (Eq. sparse-gp), and optionally their gradients
 * with respect to the features, summed over the sparse points first (Eq. gpr-force-order):
 *   dE_i/dp_i = (G_i - zeta E_i p^_i) / |p_i|,  G_i = sum_I x_I zeta k_(zeta-1) M^_I   (|p_i| = 1 without normalisation)
 * which rascal_gradients turns into forces and virial (its d_grad_ps argument).
 *   d_features [n_atoms][n_features] float32, one row per centre in atom order (rows 16-byte aligned is fastest)
 *   d_atomic [n_atoms] float32 E_i (may be NULL); d_energy [n_structures] float64 sum of E_i per structure, FP64
 *   summation (may be NULL); d_grad [n_atoms][n_features] float32 (may be NULL: energies only)
 * Asynchronous on the context stream; uses the context's scratch. */
int rascal_gpr_predict(rascal_ctx* ctx, const rascal_gpr* model, const rascal_system* sys, const float* d_features,
                       float* d_atomic, double* d_energy, float* d_grad);

/* nu = 2 equivariants (lambda-SOAP) of rank lambda from the density coefficients (Sec. 'Experimental features': the
 * correlation of Eq. body-order-x at nu = 2 coupled to rank lambda):
 *   T^{lambda mu}_{(q1 l1)(q2 l2)} = sum_{m1 m2} <l1 m1; l2 m2 | lambda mu>_real c_{q1 l1 m1} c_{q2 l2 m2}
 * with the Clebsch-Gordan coefficients carried into the real harmonic basis of the coefficients. Only proper tensors
 * (l1 + l2 + lambda even) and pairs l1 <= l2 are formed (T(l2, l1) is the transpose of T(l1, l2)), ordered by l1 then
 * l2. lambda = 0 gives (-1)^l times the power spectrum. FP32 arithmetic.
 *   d_coeffs [n_centres][n_species][n_max][(l_max+1)^2] float32 (the rascal_spherical_expansion layout)
 *   d_out [n_centres][n_pairs][2 lambda + 1][Q][Q] float32, Q = n_species n_max, 16-byte aligned
 * 0 <= lambda <= 2 l_max, else RASCAL_E_ARG. The coupling tables are built on the host on the first call per lambda
 * (a synchronous upload) and kept in the context. */
int rascal_lambda_soap_size(const rascal_ctx* ctx, int lambda, int* n_pairs, int64_t* features_per_centre);
int rascal_lambda_soap(rascal_ctx* ctx, int64_t n_centres, const float* d_coeffs, int lambda, float* d_out);

/* Exact FP64 o-GTO radial integrals I^o_nl(r) and their r-derivatives at n_points distances (Eq. rad-int-gto-1
 * with the 1F1 of Appendix A, then S^-1/2): d_r [n] float64, d_out and d_dout [n][n_max][l_max+1] float64
 * (d_dout may be NULL). Used to build the spline and the MLP training targets. */
int rascal_radial_exact_fp64(rascal_ctx* ctx, int64_t n_points, const double* d_r, double* d_out, double* d_dout);

/* Switches the radial source of an existing context between RASCAL_RADIAL_SPLINE (table), RASCAL_RADIAL_EXACT
 * (per pair, 1F1 closed form with the downward recurrence of Appendix A, FP64, then S^-1/2) and RASCAL_RADIAL_MLP
 * (the context's network). EXACT and MLP compute the per-pair values in a pass before the pair kernels and read
 * the pair count from the device (one stream synchronisation). */
int rascal_set_radial(rascal_ctx* ctx, int radial);

/* ---------------- learned radial surrogate: r -> {I^o_nl(r)}, a 1 -> H -> H -> F SiLU network ----------------
 * Not in the paper (its nearest hook is the remark that the radial basis invites numerical optimisation, end of
 * Sec. 'Spline optimization'). t = r / r_cut; z1 = W1 t + b1; h1 = silu(z1); z2 = W2 h1 + b2; h2 = silu(z2);
 * y = W3 h2 + b3; I^o_f(r) ~ scale_f y_f with f = l*n_max + n. Parameters: one FP32 vector
 * [W1 (H) | b1 (H) | W2 (H x H, row = output) | b2 (H) | W3 (F x H) | b3 (F)]; H must be 64.
 * Training runs FP32 on the CUDA cores (forward, backward, Adam); inference runs on tcgen05 with BF16 weights and
 * activations and FP32 accumulation. */
int rascal_mlp_num_params(const rascal_ctx* ctx, int hidden); /* -1 if hidden is not supported */
/* Copies host parameters and output scales [F] in, resets the Adam state and packs the BF16 tensor-core tiles. */
int rascal_mlp_set_params(rascal_ctx* ctx, int hidden, const float* h_params, const float* h_scale);
int rascal_mlp_get_params(rascal_ctx* ctx, float* h_params, float* h_scale);
/* Training targets I^o_f(r)/scale_f at n distances d_r (float64, device) into d_targets [n][F] (float32): the exact
 * FP64 integrals (Eq. rad-int-gto-1, Appendix A) are computed on a grid of dense_intervals (0: 8192) and
 * interpolated by their clamped FP64 spline (error ~1e-14 at 8192 intervals); h_scale_out [F] (host) receives
 * scale_f = max over the grid of |I^o_f|. */
int rascal_mlp_targets(rascal_ctx* ctx, int64_t n, const double* d_r, int dense_intervals, float* d_targets,
                       float* h_scale_out);
/* `steps` Adam steps (beta 0.9/0.999, eps 1e-8, cosine learning rate from lr_max to lr_min over total_steps) on
 * minibatches of `batch` samples taken in the order d_order (int64 indices into the n_samples inputs, drawn by
 * the caller); d_loss [steps] (optional) receives each step's loss. Repacks the inference tiles at the end. */
int rascal_mlp_train(rascal_ctx* ctx, int64_t n_samples, const float* d_t, const float* d_targets,
                     const int64_t* d_order, int batch, int steps, float lr_max, float lr_min, int total_steps,
                     float* d_loss);
/* Loss and parameter gradient of one batch (no update): d_grad [n_params], d_loss [1]. */
int rascal_mlp_gradients(rascal_ctx* ctx, int batch, const float* d_t, const float* d_targets, float* d_grad,
                         float* d_loss);
/* Tensor-core inference at n distances d_r (float32): d_out [n][F] = scale_f y_f, d_dout (optional) its r-derivative. */
int rascal_mlp_eval(rascal_ctx* ctx, int64_t n, const float* d_r, float* d_out, float* d_dout);
/* Checkpoint: parameters, Adam moments, step count and the hypers they belong to, in a small binary file. */
int rascal_mlp_save(rascal_ctx* ctx, const char* path);
int rascal_mlp_load(rascal_ctx* ctx, const char* path);

#ifdef __cplusplus
}
#endif

#endif /* RASCAL_H */
