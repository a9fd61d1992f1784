/*
 * sap.h -- C ABI of libsap, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of the Secant-Avoidance Projection (SAP) algorithm:
 * Kvinge, Farnell, Kirby, Peterson, "A GPU-Oriented Algorithm Design for
 * Secant-Based Dimensionality Reduction", arXiv:1807.03425.
 *
 * Problem (Sec. IV): for a point set X = {x_1..x_N} in R^n and an orthonormal
 * n x k basis U, every pair i<j of distinct points has the unit secant
 * s_ij = (x_i - x_j)/||x_i - x_j|| and the ratio r_ij = ||U^T s_ij||.  One SAP
 * iteration (Algorithm 1) finds the pair with the smallest ratio and rotates U
 * towards its secant with step alpha.  Dimension estimation (Sec. VI-A) runs
 * SAP for k = 1..k_max; the noisy-data variant (Sec. VII) discards secants
 * shorter than a threshold before normalising.
 *
 * Conventions shared by every call:
 *  - X is N x n row-major.  A basis U is n x k column-major FP64, i.e. k
 *    consecutive length-n vectors u_1..u_k.
 *  - Pairs are reported as (i, j) with 0 <= i < j < N.  Ties in the argmin go
 *    to the smallest pair index p(i,j) = i*N - i(i+1)/2 + (j-i-1); ties in the
 *    pivot choice go to the smallest column.
 *  - The library copies every input: the caller may free or reuse X and U as
 *    soon as the call returns.  Outputs are written only into caller-owned
 *    buffers.  Device memory the library needs is allocated at sap_create
 *    (and grown by sap_run for longer histories) and freed by sap_destroy.
 *  - A pointer argument is a host pointer unless the matching *_is_device
 *    flag is non-zero, in which case it is a device pointer on the handle's
 *    device.
 *  - Work is enqueued on the handle's stream (default: a stream the library
 *    creates; see sap_set_stream).  Calls that return values to the host
 *    synchronise that stream before returning.
 *  - Every call returns a status; nothing aborts, throws or traps.  A CUDA
 *    error is sticky: after SAP_E_CUDA only sap_destroy is valid.  A handle is
 *    not thread-safe.
 *  - Precision: the argmin pair and the min ratio returned are decided by an
 *    FP64 evaluation on the device from explicit differences; faster
 *    low-precision tiers only select candidates, under certified error
 *    bounds, so both paths return the same pair as an FP64 evaluation of all
 *    pairs (up to FP64 rounding on exact ties).  The pivot, Gram-Schmidt and
 *    rotation of the update run in the data's precision (FP32 or FP64); the
 *    re-orthonormalisation that follows is FP64.
 */
#ifndef SAP_H
#define SAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sap_ctx *sap_handle; /* opaque; one per dataset or batch */

typedef enum {
    SAP_OK = 0,
    SAP_E_ARG = 1,             /* an argument is out of range or NULL */
    SAP_E_STATE = 2,           /* call not valid now (e.g. no basis set yet) */
    SAP_E_NOT_ORTHONORMAL = 3, /* max |U^T U - I| > 1e-10 at sap_set_basis */
    SAP_E_NO_SECANT = 4,       /* every pair is excluded (N < 2, duplicates, eps) */
    SAP_E_OOM = 5,             /* device or host allocation failed */
    SAP_E_CUDA = 6,            /* CUDA runtime error (sticky for the handle) */
    SAP_E_TIMEOUT = 7,         /* a device-side bounded wait gave up */
    SAP_E_NO_DEVICE = 8,       /* no usable CUDA device */
    SAP_E_UNSUPPORTED = 9,     /* valid request the library does not cover */
    SAP_E_BOUNDS = 10          /* debug build (SAP_DEBUG_BOUNDS) only: a kernel met a data-dependent
                                  index out of range and skipped the access */
} sap_status;

typedef enum { SAP_F32 = 0, SAP_BF16 = 1, SAP_F64 = 2 } sap_dtype;

/* Which all-pairs form evaluates the ratios (both return the same pair):
 *  SAP_PLAIN        -- secants formed on the fly from tiles of X, projected
 *                      with U (Sec. IV; the secant set is never stored).
 *  SAP_RESTRUCTURED -- Y = X U once per iteration on tensor cores, then
 *                      r_ij = ||y_i - y_j|| / ||x_i - x_j|| over all pairs
 *                      with the lengths computed once (U^T(x_i - x_j) =
 *                      y_i - y_j). */
typedef enum { SAP_PLAIN = 0, SAP_RESTRUCTURED = 1 } sap_path;

/* Reading of the rotation step (Sec. IV): LITERAL uses the printed direction
 * (1-alpha) P P^T s + alpha (s - P P^T s); ANGLE blends the two unit vectors
 * (1-alpha) v/|v| + alpha e/|e|. */
typedef enum { SAP_UPDATE_LITERAL = 0, SAP_UPDATE_ANGLE = 1 } sap_update_mode;

/* Operand split of the tensor-core Y = X U: two-term FP16 (hi + lo, three
 * products) or two-term BF16, both with FP32 accumulation. */
typedef enum { SAP_SPLIT_FP16 = 0, SAP_SPLIT_BF16 = 1 } sap_split;

/* Statistics of the handle (read by sap_get_stats). */
typedef struct {
    int64_t n_points;        /* N */
    int32_t n_dim;           /* n */
    int32_t k;               /* target dimension of the current basis (0 if none) */
    int64_t n_pairs;         /* N(N-1)/2 */
    int64_t n_excluded;      /* duplicates plus pairs shorter than eps */
    int64_t n_near;          /* pairs evaluated from explicit differences every
                                iteration of the restructured form */
    int64_t last_tier1;      /* candidates from the all-pairs pass, last iteration */
    int64_t last_tier2;      /* candidates rechecked in FP64, last iteration */
    int64_t kernel_launches; /* kernels launched since create (graph nodes count) */
    double cert_bound;       /* absolute ratio bound of the restructured pass */
    double y_error_unit;     /* bound on |y~ - y| per unit ||x - mean|| */
    double ydf_error_unit;   /* bound on |(yh + yl) - y| per unit ||x|| (sap_project_df) */
} sap_stats;

/* Library version string. */
const char *sap_version(void);

/* Human-readable name of a status code. */
const char *sap_status_str(sap_status s);

/* Message of the last failed call on this handle ("" if none). */
const char *sap_last_error(sap_handle h);

/*
 * Create a handle for one dataset of N points in R^n (Sec. IV: "data set of k
 * points" -- N here).  X is N x n row-major in dtype dt (FP32, BF16 as
 * uint16 bits, or FP64); it is copied to the device.  The one-time length
 * preparation (explicit-difference secant lengths, exclusions, the near-pair
 * list of the restructured form) runs here.  FP64 data supports SAP_PLAIN
 * only.  N >= 2, 1 <= n <= 16384, N <= 92681 (pair indices fit in 32 bits).
 */
sap_status sap_create(const void *X, int64_t N, int32_t n, sap_dtype dt,
                      int x_is_device, sap_handle *out);

/* Release every resource of the handle.  NULL is accepted. */
sap_status sap_destroy(sap_handle h);

/* Enqueue all later work on this cudaStream_t (NULL = the library's own
 * stream).  The stream must belong to the handle's device. */
sap_status sap_set_stream(sap_handle h, void *cuda_stream);

/* Select the all-pairs form (default SAP_RESTRUCTURED for FP32/BF16 data,
 * SAP_PLAIN for FP64 data). */
sap_status sap_set_path(sap_handle h, sap_path p);

/* Select the reading of the rotation step (default SAP_UPDATE_LITERAL). */
sap_status sap_set_update_mode(sap_handle h, sap_update_mode m);

/* Select the operand split of the tensor-core product (default FP16). */
sap_status sap_set_split(sap_handle h, sap_split s);

/*
 * Noisy-data variant (Sec. VII): discard every secant whose length is less
 * than eps before normalising (d == eps is kept; decided in FP64 as
 * d^2 < eps^2).  eps = 0 restores the plain algorithm.  Re-runs the length
 * preparation.  eps < 0 or not finite -> SAP_E_ARG.
 */
sap_status sap_set_min_secant_length(sap_handle h, double eps);

/*
 * Set the current basis P^(i) (Sec. IV): U is n x k column-major FP64 with
 * orthonormal columns, 1 <= k <= min(n, 32).  Rejects max |U^T U - I| > 1e-10
 * with SAP_E_NOT_ORTHONORMAL.  Resets the iteration counter.
 */
sap_status sap_set_basis(sap_handle h, const double *U, int32_t k,
                         int u_is_device);

/*
 * The PCA start of Algorithm 1 (Sec. IV): set the basis to the top k left
 * singular vectors of the n x p matrix S of unit secants of the kept pairs
 * (distinct points, Sec. II; d >= eps after sap_set_min_secant_length,
 * Sec. VII), i.e. the eigenvectors of S S^T = sum_{i<j} s s^T with the k
 * largest eigenvalues, each signed so that its entry of largest magnitude is
 * positive.  S S^T is formed in FP64 on the device as Xc^T L X (L the
 * 1/d^2-weighted graph Laplacian of the pairs, lengths from explicit FP64
 * differences), never storing S; the n x n symmetric eigenproblem is solved
 * on the device by the cyclic Jacobi method in FP64 (round-robin parallel
 * ordering, sweeps until the off-diagonal norm is below 4 n 2^-53 of the
 * whole; SAP_E_CUDA if 40 sweeps do not get there).  U_out (nullable, host, n x k
 * column-major) receives the basis, sigma_out (nullable, k) the singular
 * values sqrt(lambda) in descending order.  1 <= k <= min(n, 32).  Resets
 * the iteration counter, like sap_set_basis.  Work memory: 8 B per pair
 * (the FP64 lengths) plus 8 N n + 8 n^2 bytes, freed before returning.
 * Synchronises.
 */
sap_status sap_secant_pca(sap_handle h, int32_t k, double *U_out, double *sigma_out);

/* Copy the current basis (n x k column-major FP64) into U_out. */
sap_status sap_get_basis(sap_handle h, double *U_out, int out_is_device);

/*
 * Algorithm 1, argmin step, under the current basis: the pair whose unit
 * secant has the smallest projected length, and that length.  Any output
 * pointer may be NULL.  Synchronises.  SAP_E_NO_SECANT if every pair is
 * excluded.
 */
sap_status sap_min_secant(sap_handle h, int64_t *i, int64_t *j, double *ratio);

/*
 * One SAP iteration (Algorithm 1): evaluate every secant, take the argmin,
 * then pivot, modified Gram-Schmidt, rotate the first column by alpha and
 * re-orthonormalise in FP64.  alpha in [0, 1].  The evaluated pair and ratio
 * (of the basis before the update) are returned through the optional
 * outputs; with all three NULL the call does not synchronise.
 */
sap_status sap_step(sap_handle h, double alpha, int64_t *i, int64_t *j,
                    double *ratio);

/*
 * iters SAP iterations followed by one more evaluation, as a captured CUDA
 * graph (Algorithm 1 loop).  hist (nullable, iters+1 entries) receives the
 * min ratio of U_0..U_iters and argmins (nullable, 2*(iters+1) entries) the
 * pairs; with both NULL the call does not synchronise and the results stay
 * on the device (sap_get_history).  The basis afterwards is U_iters.
 */
sap_status sap_run(sap_handle h, double alpha, int32_t iters, double *hist,
                   int64_t *argmins);

/* Copy the history of the last sap_run (iters+1 entries each; argmins as
 * (i, j) pairs).  Synchronises.  Either pointer may be NULL. */
sap_status sap_get_history(sap_handle h, double *hist, int64_t *argmins,
                           int32_t capacity);

/*
 * Dimension estimation (Sec. VI-A): run SAP for every k = 1..k_max from the
 * first k columns of U0 (n x k_max column-major FP64, orthonormal), iters
 * iterations each with step alpha; ratios_out[k-1] (nullable) receives the
 * min ratio of the final basis for k, and k_out (nullable) the smallest k
 * whose ratio exceeds threshold (strictly), or -1.  FP32 or BF16 data;
 * k_max <= 20 (the padded widths of all bases fill one 256-wide
 * tensor-core product).  All bases advance together: each iteration is one
 * product for all bases, then every basis's pass, recheck and update on
 * concurrent branches of one CUDA graph.  Leaves the handle's own basis
 * unchanged (its watch list restarts).  Synchronises.
 */
sap_status sap_estimate_dim(sap_handle h, const double *U0, int32_t k_max,
                            int32_t iters, double alpha, double threshold,
                            int32_t *k_out, double *ratios_out);

/* History of basis k (1 <= k <= k_max) in the last sap_estimate_dim: the min
 * ratio of U_0..U_iters and the argmin pairs, as for sap_get_history. */
sap_status sap_get_sweep_history(sap_handle h, int32_t k, double *hist,
                                 int64_t *argmins, int32_t capacity);

/* Final basis of k (1 <= k <= k_max) in the last sap_estimate_dim: n x k
 * column-major FP64 into U_out (host, or device when out_is_device). */
sap_status sap_get_sweep_basis(sap_handle h, int32_t k, double *U_out, int out_is_device);

/*
 * The projected data under the current basis (Sec. V shows such projections):
 * Y_out[i*k + c] = <x_i - mean(X), u_c>, N x k row-major FP32, computed by
 * the tensor-core product of the restructured form (split 16-bit operands,
 * FP32 accumulation).  Rows are translated by -mean(X) U, so differences of
 * rows are the projected secants U^T (x_i - x_j); each entry is within
 * sap_stats.y_error_unit * ||x_i - mean(X)|| of the exact value.
 * FP32/BF16 datasets only.  Synchronises.
 */
sap_status sap_project(sap_handle h, float *Y_out, int out_is_device);

/*
 * The projected data in extended precision: Yh_out[i*k + c] + Yl_out[i*k + c]
 * (two FP32 numbers per entry, N x k row-major each) = <x_i, u_c> for the
 * points as given (not centred), within sap_stats.ydf_error_unit * ||x_i||
 * (about 1.25 (9n + 60) 2^-48: error-free products and renormalised sums
 * of the FP32 points and the FP64 basis).  This is the Y the double-float
 * second tier of the restructured form evaluates pairs from.  FP32/BF16
 * datasets only.  Synchronises.
 */
sap_status sap_project_df(sap_handle h, float *Yh_out, float *Yl_out, int out_is_device);

/*
 * The argmin step without any device allocation, for callers that cannot
 * allocate GPU memory: code whose device memory belongs to another
 * allocator's pool, or loops that cannot afford an allocation's implicit
 * synchronisation or its failure.  The paper has no counterpart; it is a
 * deployment variant of sap_min_secant in the plain form, and returns the
 * same pair and ratio.
 *
 * X: device pointer, N x n row-major FP32; U: device pointer, n x k
 * column-major FP64 with orthonormal columns (not checked); eps: pairs with
 * ||x_i - x_j|| < eps are excluded (0: none); cuda_stream: the stream to run
 * on (NULL: the legacy default stream); i, j, ratio: host outputs
 * (nullable).  Copies the result to the host and synchronises the stream
 * before returning.  SAP_E_NO_SECANT if every pair is excluded,
 * SAP_E_TIMEOUT if a device-side bounded wait gave up.  Limits:
 * 2 <= N <= 1024, 1 <= n <= 1024, 1 <= k <= min(n, 8); anything larger
 * returns SAP_E_ARG.
 *
 * Working memory is one fixed file-scope device array of about 4.2 MB that
 * every GPU loading the library holds until exit.  The first call on a
 * device looks up its address and must come before any stream capture.
 * All calls share the array and reset it on entry; calls that overlap on the
 * GPU race, so the caller must serialise them.
 */
sap_status sap_min_secant_noalloc(const float *X, int64_t N, int32_t n, const double *U, int32_t k,
                                  double eps, void *cuda_stream, int64_t *i, int64_t *j,
                                  double *ratio);

/*
 * Soft-min objective: a smooth surrogate of the min ratio that Algorithm 1
 * maximises, for gradient-based training of the basis.  The paper has no
 * counterpart; its max-min problem (Sec. IV, the objective of Algorithm 1)
 * is the tau -> 0 limit:
 *     L(U) = -tau log sum_{i<j kept} exp(-r_ij / tau),
 * over the pairs the handle keeps (distinct points, and d_ij >= eps after
 * sap_set_min_secant_length).  min r - tau log P <= L <= min r, P = number of
 * kept pairs.  The gradient is
 *     dL/dU = sum_{i<j} p_ij (x_i - x_j)(y_i - y_j)^T / (d_ij^2 r_ij),
 *     p_ij = exp((L - r_ij)/tau),  y = U^T x,
 * an n x k matrix laid out like U (column-major FP64); pairs with
 * r_ij < 1.1e-19 count in L but not in the gradient.  L depends only on the
 * span of U, so U^T dL/dU is symmetric.
 *
 * Requirements: FP32 or BF16 data, a basis set with 1 <= k <= 8, n <= 512,
 * tau > 0; otherwise SAP_E_UNSUPPORTED / SAP_E_ARG / SAP_E_STATE.  Both
 * passes run every pair on the GPU from the stored FP32 lengths and an
 * extended-precision (FP32 hi + lo) Y = X U; the error is stated with the
 * tests and grows like 1/tau.  Results are reproducible bit for bit.
 *
 * sap_softmin_forward: L at the current basis (host output).  Synchronises.
 * sap_softmin_backward: G_out = dL/dU at the current basis, given L, the
 *   value sap_softmin_forward returned for this basis and tau (the weights
 *   p_ij are formed with it).  G_out is n x k column-major FP64, host or
 *   device (out_is_device).  Synchronises.
 * sap_softmin_ascent: `steps` Riemannian gradient-ascent steps on the
 *   Grassmannian, all on the device (one CUDA graph per step):
 *   G_R = G - U (U^T G), U <- Q factor of U + eta G_R / ||G_R||_F (FP64
 *   Cholesky QR, positive diagonal of R).  A step with G_R = 0 leaves U
 *   unchanged.  hist (nullable, host, steps + 1 doubles) receives L before
 *   each step and at the final basis.  The handle's basis is the final one
 *   (read it with sap_get_basis; sap_min_secant then judges it).
 */
sap_status sap_softmin_forward(sap_handle h, double tau, double *L_out);
sap_status sap_softmin_backward(sap_handle h, double tau, double L, double *G_out, int out_is_device);
sap_status sap_softmin_ascent(sap_handle h, double tau, double eta, int32_t steps, double *hist);

/*
 * Uneven batch: B independent datasets (Sec. VII's noisy-data setting is the
 * intended use: many small hyperspectral scenes), each X_b an N_b x n
 * row-major array of the same n and dtype (2 <= N_b <= 92681, B <= 4096),
 * run together.  The batch handle owns one dataset handle per X_b.
 * sap_set_min_secant_length, sap_set_split, sap_set_update_mode, sap_set_path
 * and sap_set_basis apply to every dataset; sap_get_stats sums over them;
 * calls on one basis (sap_step, sap_run, sap_min_secant, sap_get_basis, the
 * sweep and the soft-min calls) return SAP_E_STATE on a batch handle.
 *
 * sap_run_batch: iters SAP iterations of every dataset followed by one
 * evaluation, as one captured CUDA graph per chunk of iterations that
 * forks to every dataset's stream and joins (the datasets never wait on
 * each other inside a chunk).  hist (nullable) receives B x (iters + 1)
 * min ratios and argmins (nullable) B x (iters + 1) pairs, dataset-major.
 * Every dataset needs a basis.  Synchronises.
 */
sap_status sap_create_batch(const void *const *Xs, const int64_t *Ns, int32_t B, int32_t n,
                            sap_dtype dt, int x_is_device, sap_handle *out);
sap_status sap_batch_count(sap_handle h, int32_t *B);   /* 1 for an ordinary handle */
sap_status sap_set_basis_b(sap_handle h, int32_t b, const double *U, int32_t k, int u_is_device);
sap_status sap_get_basis_b(sap_handle h, int32_t b, double *U_out, int out_is_device);
sap_status sap_min_secant_b(sap_handle h, int32_t b, int64_t *i, int64_t *j, double *ratio);
sap_status sap_run_batch(sap_handle h, double alpha, int32_t iters, double *hist, int64_t *argmins);

/*
 * Cap of the per-pair error bound of the restructured pass (restructured
 * form of Sec. IV's argmin step, FP32/BF16 data).  The tensor-core Y gives
 * each pair's ratio a certified error b_ij = sqrt(k) eps_Y (|x_i - xbar| +
 * |x_j - xbar|) / d_ij; pairs with b_ij above the cap are skipped by the
 * pass and re-evaluated every iteration by the second tier (the near list),
 * the others are filtered in the pass with their own b_ij.  A larger cap gives a shorter
 * near list and a wider coarse filter; results do not depend on it.
 * Default 5e-4; 1e-6 <= b_cap <= 0.25, else SAP_E_ARG.  sap_autotune may
 * change it.  On a batch handle, every dataset.
 */
sap_status sap_set_pass_bound(sap_handle h, double b_cap);

/*
 * Launch parameters of one iteration.  None of them changes a result (every
 * choice selects certified candidate sets and takes the same FP64
 * decisions); they only move time.
 */
typedef struct {
    double pass_bound;              /* cap of the restructured pass's per-pair bound (sap_set_pass_bound) */
    int32_t pass_stages;            /* TMA ring depth of the restructured pass: 2..5; 0 = as many as fit */
    int32_t explicit_blocks_per_sm; /* second-tier grid (candidates and near pairs), 1..8 blocks per SM */
    int32_t update_blocks;          /* FP64 recheck + update grid, 0 (one per SM) .. 304 */
    int32_t plain_blocks_per_sm;    /* plain pass grid, 1..8 blocks per SM (FP64 data: twice) */
    int32_t programmatic_launch;    /* 1: the kernels of an iteration are chained by programmatic
                                       dependent launch (each starts early and waits where it
                                       needs its predecessor's output); 0: ordinary launches */
    int32_t refine_tier;            /* second tier of the restructured form: 1 double-float Y
                                       (O(k) per pair), 0 explicit differences (O(n k) per pair),
                                       2 explicit differences fused into the FP64 recheck (one
                                       launch fewer; n <= 256, else as 0), 3 explicit differences
                                       in extended precision (hi + lo FP32, error-free products)
                                       fused into the FP64 recheck (one launch fewer; k <= 8, else
                                       as 0), 4 explicit differences in extended precision whose
                                       list carries each pair's ratio, so the FP64 recheck takes
                                       only the pairs within the final bound, 5 explicit
                                       differences in extended precision inside the all-pairs
                                       pass: each emitted pair, and each near pair, is rechecked
                                       at once by the warp that found it, and evaluated in FP64
                                       there if it can still be the argmin; one block then takes
                                       the argmin and updates (two launches fewer, no lists;
                                       k <= 16, else as 0), -1 chosen by n and k (double-float
                                       above n = 256, else 5 for k <= 16, else 0) */
    double us_per_iteration;        /* measured by sap_autotune; 0 when set by hand */
} sap_tuning;

/*
 * Autotuner (the paper has no counterpart; its Sec. V gives no launch
 * shapes).  Times candidate parameter sets on the handle's current basis,
 * one parameter at a time from the current set, each as `iters` SAP
 * iterations with step alpha replayed from captured graphs (best of two
 * runs, CUDA events on the handle's stream), and keeps the fastest.  The
 * basis is restored afterwards and the iteration counter restarts, as after
 * sap_set_basis.  The choice is cached for the process under the problem's
 * shape (N, n, k, dtype, path, split, eps) and applied automatically by
 * sap_set_basis, sap_set_path, sap_set_split and sap_set_min_secant_length
 * when their handle reaches a new shape that has a cached choice
 * (parameters set by hand stay until the shape changes); if the environment
 * variable SAP_TUNE_CACHE names a file, choices are appended to it and read back by
 * later processes.  1 <= iters <= 4096.  On a batch handle one set is chosen
 * for all datasets together by timing whole batch iterations (the datasets
 * run concurrently), and it is not cached.  out (nullable) receives the
 * chosen set.  Synchronises.
 */
sap_status sap_autotune(sap_handle h, double alpha, int32_t iters, sap_tuning *out);

/* The handle's current launch parameters (a batch handle: its first
 * dataset's). */
sap_status sap_get_tuning(sap_handle h, sap_tuning *out);

/* Set the launch parameters by hand (ranges as in sap_tuning, else
 * SAP_E_ARG).  On a batch handle, every dataset. */
sap_status sap_set_tuning(sap_handle h, const sap_tuning *in);

/*
 * Repeated point subsampling (Sec. VI-C: SAP on many random subsets of a
 * large point set, e.g. 10 subsets of 512 of 21,025 pixels, and the
 * dimension-estimation curves compared across subsets).  Creates a batch
 * handle of R datasets, dataset b holding the rows idx[b*m + 0 .. m-1] of X
 * (N x n row-major in dtype dt, host or device as x_is_device; idx is a
 * host array of R*m indices in [0, N), drawn by the caller; a repeated
 * index yields a duplicate point, whose pairs are excluded as usual).
 * 1 <= R <= 4096, 2 <= m <= min(N, 92681).  The handle behaves as one from
 * sap_create_batch; sap_estimate_dim_b runs the dimension sweep of one
 * dataset (as sap_estimate_dim does on an ordinary handle).
 */
sap_status sap_create_subsamples(const void *X, int64_t N, int32_t n, sap_dtype dt, int x_is_device,
                                 const int64_t *idx, int32_t R, int32_t m, sap_handle *out);
sap_status sap_estimate_dim_b(sap_handle h, int32_t b, const double *U0, int32_t k_max, int32_t iters,
                              double alpha, double threshold, int32_t *k_out, double *ratios_out);

/*
 * Multi-GPU split of the argmin step (Algorithm 1, Sec. IV: the minimum over
 * all pairs is the minimum of the minima over disjoint sets of pairs), one
 * process per GPU.  The upper triangle of 128 x 128 pair tiles (I <= J), in
 * row-major order over the tile grid, is cut into `world` contiguous ranges
 * of nearly equal pair count; rank r owns range r.  Each rank holds the
 * points and the basis in full and the lengths of its own tiles only.  One
 * iteration:
 *   1. sap_shard_min on every rank: its shard's exact minimum as a record;
 *   2. an all-gather of the 16-byte records (the caller's collective, e.g.
 *      NCCL through torch.distributed);
 *   3. sap_shard_step on every rank with all records: the winning pair is
 *      re-evaluated in FP64 and every rank takes the same update, so the
 *      bases stay identical with no further exchange.
 * A record is the FP64 squared ratio q = r^2 of the shard's best pair and
 * the pair (i < j), or i = j = -1 when the shard has no candidate.
 */
typedef struct {
    double q;
    int32_t i, j;
} sap_record;

/* Tile range [t0, t1) and pair count of rank `rank` among `world` for N
 * points (host only; 1 <= world <= 4096, 0 <= rank < world).  A range may be
 * empty when world exceeds the number of tiles. */
sap_status sap_shard_range(int64_t N, int32_t world, int32_t rank, int64_t *t0, int64_t *t1,
                           int64_t *pairs);

/* The lexicographic minimum (q, then i, then j) of `count` records into out
 * (host only); records with i < 0 are skipped.  SAP_E_NO_SECANT if none. */
sap_status sap_merge_records(const sap_record *recs, int32_t count, sap_record *out);

/* Create a handle for rank `rank` of `world` on dataset X (as sap_create;
 * FP32 or BF16 data, restructured form only).  The length preparation and
 * the all-pairs pass cover only the rank's tiles.  SAP_E_ARG if the rank's
 * range is empty.  On such a handle sap_step, sap_run, sap_min_secant,
 * sap_estimate_dim, sap_autotune, sap_secant_pca, the soft-min calls and
 * the plain path return SAP_E_STATE / SAP_E_UNSUPPORTED. */
sap_status sap_create_shard(const void *X, int64_t N, int32_t n, sap_dtype dt, int x_is_device, int32_t world,
                            int32_t rank, sap_handle *out);

/* Step 1 of a sharded iteration: the exact minimum over the rank's pairs
 * under the current basis, written as one record to rec_out (host, or
 * device when out_is_device; then the call does not synchronise). */
sap_status sap_shard_min(sap_handle h, sap_record *rec_out, int out_is_device);

/* Step 3: the update toward the unit secant of the best of `count` records
 * (all ranks' records, host or device as recs_is_device), with step alpha,
 * recorded in the handle's history (sap_get_history).  The winning pair's
 * ratio is re-evaluated in FP64 under the current basis, so every rank
 * decides identically.  SAP_E_NO_SECANT if no record holds a pair (reported
 * when the call synchronises: with a host `out` pair, or at the next call
 * that reads the device status). */
sap_status sap_shard_step(sap_handle h, double alpha, const sap_record *recs, int32_t count,
                          int recs_is_device);

/*
 * Test hooks of the failure paths (no counterpart in the paper).
 * sap_inject_fault: the next CUDA call this handle checks reports an error
 * as if the runtime had returned it -- kind 1 an allocation failure
 * (SAP_E_OOM; the handle stays usable), kind 2 a CUDA error (SAP_E_CUDA,
 * sticky: every later call but sap_destroy returns SAP_E_CUDA).  Nothing is
 * sent to the device.  NULL handle or another kind -> SAP_E_ARG.
 * sap_selftest_wait: one kernel waits on an mbarrier that nothing arrives
 * on, with the bounded wait every kernel of the library uses, for
 * budget_cycles SM clocks (0 .. 4e9), then records that it gave up;
 * returns SAP_E_TIMEOUT, and the context stays usable.  No copy is in
 * flight during the wait.  Synchronises cuda_stream (NULL: the legacy
 * default stream).
 */
sap_status sap_inject_fault(sap_handle h, int32_t kind);
sap_status sap_selftest_wait(void *cuda_stream, int64_t budget_cycles);

/* Read the handle's statistics. */
sap_status sap_get_stats(sap_handle h, sap_stats *out);

/*
 * Kernel timing for measurement: while enabled, sap_step and sap_run launch
 * kernels one by one (no graph) with CUDA events around each launch on the
 * handle's stream; sap_get_kernel_time returns the accumulated device time
 * (ms) and launch count of one kernel class.  Classes: 0 Y = XU product
 * (tensor cores), 1 restructured all-pairs pass, 2 plain all-pairs pass,
 * 3 second tier (explicit differences or the double-float refine),
 * 4 double-float Y = XU, 5 FP64 recheck fused with the update, 6 soft-min
 * forward pass, 7 soft-min backward pass, 8 soft-min near pairs, 9 soft-min
 * other kernels (Y, gradient sums, ascent step).  Enabling resets the
 * accumulators.
 */
sap_status sap_set_profiling(sap_handle h, int enable);
sap_status sap_get_kernel_time(sap_handle h, int32_t kernel_class,
                               double *total_ms, int64_t *launches);

#ifdef __cplusplus
}
#endif

#endif /* SAP_H */
