/*
 * sqrtm_mp.h -- C ABI of a GB300 (sm_103a) library for the principal matrix
 * square root by the mixed-precision method of Gao, Kressner and Shao,
 * "A mixed precision algorithm for the matrix square root" (arXiv 2607.12430).
 *
 * The principal square root X of A (no eigenvalue on the closed negative real
 * axis) is the unique X with X^2 = A and every eigenvalue of X in the open
 * right half plane (Sec. 1).
 *
 * Conventions shared by every entry point:
 *   - Matrices are real, FP64, column-major: element (i, j) of a matrix with
 *     leading dimension ld sits at p[i + j*ld]; ld >= max(1, n).
 *   - Matrix pointers are DEVICE pointers into caller-owned memory unless an
 *     argument says otherwise.  The library never frees or keeps caller
 *     buffers beyond the call.  Input and output buffers must not overlap.
 *   - Work is enqueued on the handle's stream.  A call returns after its work
 *     is complete on that stream (the convergence test of the refinement
 *     loop reads one scalar back to the host each step), so outputs and the
 *     info struct are valid on return.
 *   - All scratch memory (workspace, saved factors) belongs to the handle and
 *     grows on demand with cudaMalloc; sqrtm_destroy releases it.
 *   - One handle serves one host thread at a time.
 *
 * Return values (LAPACK-style INFO):
 *    0  success
 *   -i  argument i is invalid (1-based position in the call)
 *    1  the refinement loop did not reach the tolerance within maxit steps;
 *       X holds the last iterate
 *    2  an eigenvalue lies on or next to the closed negative real axis, or a
 *       Sylvester denominator s_ii + s_jj vanished (Sec. 1, Sec. 2.1)
 *    3  the Schur QR iteration (or the eigensolver) hit its iteration cap
 *    4  the refinement diverged (the residual grew twice in a row)
 *    5  the input holds NaN or Inf
 *    6  a device-side bounded wait gave up
 *    7  CUDA error or allocation failure
 *    8  no factors saved on the handle (sqrtm_backward before a forward call)
 */
#ifndef SQRTM_MP_H
#define SQRTM_MP_H

#include <stdint.h>

/* Exported symbols: the library is built with hidden default visibility. */
#if defined(__GNUC__)
#define SQRTM_API __attribute__((visibility("default")))
#else
#define SQRTM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sqrtm_handle_s *sqrtm_handle_t;

/* Matrix kind: AUTO takes the symmetric positive definite path (Algorithm 3)
 * when A is bitwise symmetric, the general path (Algorithm 2) otherwise. */
enum { SQRTM_KIND_AUTO = 0, SQRTM_KIND_GENERAL = 1, SQRTM_KIND_SPD = 2, SQRTM_KIND_REAL = 3 };
/* SQRTM_KIND_REAL (never chosen by AUTO): Algorithm 2 in real arithmetic
 * (Remark 2.1) -- real Schur form A = Q T Q^T with T quasi-triangular (2x2
 * blocks for complex conjugate pairs, never cut), the quasi-triangular
 * square root, and corrections from quasi-triangular Sylvester solves with
 * real transforms.  Its Schur stage is a single-CTA double-shift iteration
 * (n <= 2048; larger n return -3, argument n out of range, as
 * sqrtm_step_real_schur returns -4 for its n), much slower than the complex
 * multi-bulge stage of SQRTM_KIND_GENERAL for large n. */

/* Precision options (bit flags).
 * Low-precision dense products (transforms of Algorithm 2/3 steps 3, 8 and
 * 10 and the GEMM updates inside the Sylvester and triangular square root
 * solvers): FP32 (0) is IEEE single on the CUDA cores; TF32X3 is a
 * three-term split-TF32 product on the tensor cores with FP32 accumulation
 * (error comparable to FP32).
 * FP64 residual of the symmetric positive definite path (Algorithm 3,
 * step 5): by default, for 256 <= n <= 46340, X X is formed from exact
 * products of 5- to 8-bit digit slices of X on the BF16 tensor cores and
 * summed in FP64 (error-free splitting; the terms left out are below
 * n 2^(rho_i + rho_j - 56), 2^rho_i bounding row i of X, i.e. within the
 * FP64 product's own error bound).  The general path's residual (Algorithm
 * 2, step 4) of a real iterate of the FP32 method does the same from
 * n = 512 on, with the digit slices of the rows of X against those of its
 * columns.  RESID_FP64 forces the FP64 product on the CUDA cores in both. */
enum {
    SQRTM_PREC_AUTO = -1,
    SQRTM_PREC_FP32 = 0,
    SQRTM_PREC_TF32X3 = 1,
    SQRTM_PREC_RESID_FP64 = 2,
    SQRTM_PREC_TF32X3_GENERAL = 4
};
/* SQRTM_PREC_TF32X3_GENERAL: the dense products of the general path
 * (Algorithm 2 steps 3, 8 and 10 for real A and even n >= 128: X_0 = Q S Q^H,
 * R~ = Q^H Rhat Q, X += Re(Q Y Q^H)) as split-TF32 products on the tensor
 * cores, each complex product computed as one real product over the
 * interleaved (re, im) operands; otherwise the FP32 CUDA-core products. */

typedef struct {
    double tol;      /* stop when ||A - X^2||_F <= tol ||A||_F (Algorithm 2,
                        step 6); default 1e-12 (Sec. 5) */
    int maxit;       /* refinement loop runs k = 0..maxit (Algorithm 2, step
                        4); default 10 */
    int blks;        /* block size of the Sylvester and triangular square
                        root solvers (Algorithm 1), 1..32; 0 (default): the
                        handle's tuning table, else 32 (Sec. 5) */
    int kind;        /* SQRTM_KIND_* */
    int precision;   /* SQRTM_PREC_* flags; SQRTM_PREC_AUTO (default): the
                        handle's tuning table, else SQRTM_PREC_FP32 */
    int steps;       /* >= 0: apply exactly this many corrections with the
                        stopping test nullified (the accuracy-run protocol of
                        Sec. 5.1); -1 (default): use tol / maxit */
} sqrtm_opts;

#define SQRTM_MAX_HISTORY 64

typedef struct {
    int status;          /* same code as the return value */
    int kind_used;       /* SQRTM_KIND_GENERAL or SQRTM_KIND_SPD */
    int iterations;      /* corrections applied */
    int scale_exponent;  /* e with A_s = 4^-e A, X = 2^e sqrt(A_s) */
    double norm_a;       /* ||A||_F */
    /* relative residual ||A - X_k^2||_F / ||A||_F before correction k
       (entry k), and after the last correction when it was evaluated */
    int history_len;
    double history[SQRTM_MAX_HISTORY];
    /* wall time of the phases in milliseconds, from CUDA events on the
       handle's stream: Schur / spectral decomposition, triangular square root
       plus X0, refinement loop */
    double ms_schur, ms_trisqrt, ms_refine;
    /* of ms_schur: the Hessenberg (or tridiagonal) reduction alone */
    double ms_reduction;
    /* QR sweeps and Givens rotations of the Schur iteration (general path) */
    int schur_sweeps;
    int64_t schur_rotations;
    /* general path: summed duration of the QR chase kernel's launches (ms)
     * and its in-block work, sum over sweeps of rotations x active-block
     * size (each such unit is one rotated pair of complex entries) */
    double ms_qr_chase;
    int64_t schur_work;
} sqrtm_info;

/* Tuning table of a handle, written by the project's autotuner
 * (paper_2607_12430_gb300.autotune) from timings on the GPU at hand.  Entry
 * i applies to sizes n <= n_max (entries in ascending n_max; larger n use
 * the last entry).  Fields:
 *   blks          block size of the triangular square root and Sylvester
 *                 solvers, 1..32 (used when opts->blks == 0);
 *   qr_helpers    helper CTAs of the cooperative QR chase: 0 (chase CTA
 *                 alone), 1..24, or -1 (built-in rule: 8, 16 from n = 1024);
 *   batched       sqrtm_mixed_batched: 1 sends matrices of these sizes
 *                 through the batched general path, 0 through per-matrix
 *                 calls on worker streams;
 *   spd_precision SQRTM_PREC_* flags used when opts->precision ==
 *                 SQRTM_PREC_AUTO (the TF32X3 and RESID_FP64 bits act on
 *                 Algorithm 3, TF32X3_GENERAL on Algorithm 2);
 *   trisqrt_cutoff 0: the blocked triangular square root (Sec. 2.2.1);
 *                 >= 64: the recursive splitting of Sec. 2.2.1 (S_11, S_22
 *                 recursively, S_12 from a Sylvester solve) down to blocks
 *                 of at most this size, which take the blocked method;
 *   batched_spd   sqrtm_mixed_batched with SQRTM_KIND_AUTO: 1 sends the
 *                 bitwise symmetric matrices of these sizes (n <= 256) that
 *                 take the batched path through its spectral stage
 *                 (Algorithm 3: FP32 Jacobi decomposition), 0 through the
 *                 complex Schur stage of Algorithm 2 with the other members.
 * Without a table the built-in values apply: blks 32, helpers -1, batched
 * for n <= 256, SQRTM_PREC_FP32, cutoff 0, batched_spd 1. */
typedef struct {
    int64_t n_max;
    int blks;
    int qr_helpers;
    int batched;
    int spd_precision;
    int trisqrt_cutoff;
    int batched_spd;
} sqrtm_tune_entry;

#define SQRTM_MAX_TUNE 32

/* Create a handle bound to a CUDA stream (cudaStream_t passed as void*;
 * NULL = legacy default stream).  Returns 0 or 7. */
SQRTM_API int sqrtm_create(sqrtm_handle_t *handle, void *stream);

/* Release the handle and all device memory it owns.  Returns 0. */
SQRTM_API int sqrtm_destroy(sqrtm_handle_t handle);

/* Rebind the handle to another stream. */
SQRTM_API int sqrtm_set_stream(sqrtm_handle_t handle, void *stream);

/* Limit, in nanoseconds, of each bounded device-side wait between the CTAs
 * of the cooperative QR chase (the Schur stage of the general path,
 * n >= 256): the chase CTA waiting for its helper CTAs' progress and the
 * helpers waiting for the next posted window.  A wait that runs out makes
 * every CTA of the chase leave and the call return 6; the handle stays
 * usable and its next call starts afresh.  0 (default) means 2 s.  The
 * tensor-core kernels' mbarrier waits keep their own limit.  Returns 0,
 * -1 (handle NULL) or -2 (ns < 0). */
SQRTM_API int sqrtm_set_wait_limit(sqrtm_handle_t handle, int64_t ns);

/* Fill opts with the defaults listed above. */
SQRTM_API void sqrtm_default_opts(sqrtm_opts *opts);

/* Install (count <= SQRTM_MAX_TUNE entries, validated and copied; count 0
 * clears) or read (returns the number of entries, copying at most cap) the
 * handle's tuning table.  set returns 0, -2 (table NULL with count > 0),
 * -3 (count out of range) or -4 (an entry out of range or n_max not
 * ascending). */
SQRTM_API int sqrtm_set_tuning(sqrtm_handle_t handle, const sqrtm_tune_entry *table, int count);
SQRTM_API int sqrtm_get_tuning(sqrtm_handle_t handle, sqrtm_tune_entry *table, int cap);

/* Mixed-precision principal square root, Algorithm 2 (general A) or
 * Algorithm 3 (symmetric positive definite A):
 *   Schur / spectral decomposition A = Q T Q^H in FP32, S = T^{1/2} in FP32
 *   (blocked, Sec. 2.2.1), X_0 = Q S Q^H rounded to FP32, then refinement
 *   X_{k+1} = X_k + Q Y Q^H with S Y + Y S = Q^H (A - X_k^2) Q, residual and
 *   update in FP64, transforms and Sylvester solve in low precision.
 * dA: n x n input (lda); dX: n x n output (ldx).  tol overrides opts->tol when
 * opts is NULL (defaults otherwise).  opts and info may be NULL.  The Schur
 * factors are kept on the handle for a following sqrtm_backward. */
SQRTM_API int sqrtm_mixed(sqrtm_handle_t handle, const double *dA, int64_t n, int64_t lda, double tol,
                double *dX, int64_t ldx, const sqrtm_opts *opts, sqrtm_info *info);

/* Plain FP64 Schur method (Sec. 1): A = Q T Q^H, S = T^{1/2}, X = Q S Q^H,
 * all in FP64 on the GPU, no refinement.  tol is accepted for a uniform
 * signature and ignored.  The same kernels as sqrtm_mixed, instantiated in
 * FP64. */
SQRTM_API int sqrtm_schur_fp64(sqrtm_handle_t handle, const double *dA, int64_t n, int64_t lda,
                     double tol, double *dX, int64_t ldx, const sqrtm_opts *opts,
                     sqrtm_info *info);

/* Complex input (the method is stated for A in C^{n x n}, Sec. 1): the
 * same general path (Algorithm 2) with complex iterates.  dA, dX: n x n
 * complex FP64 matrices stored as interleaved (re, im) pairs
 * (cuDoubleComplex / std::complex<double> layout), column-major, lda and
 * ldx counted in complex elements.  The residual A - X_k^2 and the update
 * are complex FP64; X_0 = Q S Q^H and the corrections Q Y Q^H are complex
 * (no real part taken).  opts->kind is ignored (Hermitian input takes the
 * Schur form too); no factors are kept for sqrtm_backward.  Other arguments
 * and return codes as for sqrtm_mixed. */
SQRTM_API int sqrtm_mixed_complex(sqrtm_handle_t handle, const void *dA, int64_t n, int64_t lda, double tol,
                                  void *dX, int64_t ldx, const sqrtm_opts *opts, sqrtm_info *info);

/* Plain FP64 Schur method for complex input: X = Q T^{1/2} Q^H in FP64,
 * no refinement; layout as for sqrtm_mixed_complex. */
SQRTM_API int sqrtm_schur_fp64_complex(sqrtm_handle_t handle, const void *dA, int64_t n, int64_t lda, double tol,
                                       void *dX, int64_t ldx, const sqrtm_opts *opts, sqrtm_info *info);

/* Mixed-precision principal cube root (Sec. 4, p = 3): the X with X^3 = A
 * whose eigenvalues have arguments in (-pi/3, pi/3], for A with no
 * eigenvalue on the closed negative real axis.  The steps of Algorithm 2
 * with the order raised: A_s = 8^-e A, FP32 Schur form, the triangular cube
 * root S = T^{1/3} with V = S^2 (blocked recurrence from S^3 = T), X_0 =
 * 2^e Q S Q^H rounded to FP32, then X_{k+1} = X_k + 2^e Q Y Q^H with
 * S^2 Y + S Y S + Y S^2 = Q^H (A - X_k^3) Q 8^-e (Eq. (3rd-order)), the
 * residual (X_k X_k in FP64, then A - X_k (X_k X_k)) and the update in FP64.
 * Arguments, opts, info and return codes as for sqrtm_mixed; opts->kind is
 * ignored (every input takes the Schur form); no factors are kept for
 * sqrtm_backward. */
SQRTM_API int sqrtm_cbrtm_mixed(sqrtm_handle_t handle, const double *dA, int64_t n, int64_t lda, double tol,
                                double *dX, int64_t ldx, const sqrtm_opts *opts, sqrtm_info *info);

/* Plain FP64 Schur method for the principal cube root (Sec. 4, p = 3):
 * X = 2^e Q S Q^H with S = T^{1/3}, all in FP64, no refinement.  Arguments
 * as for sqrtm_schur_fp64. */
SQRTM_API int sqrtm_cbrtm_schur_fp64(sqrtm_handle_t handle, const double *dA, int64_t n, int64_t lda,
                                     double tol, double *dX, int64_t ldx, const sqrtm_opts *opts,
                                     sqrtm_info *info);

/* Adjoint of the square root at the last sqrtm_mixed call on this handle:
 * given a cotangent Gbar (n x n, ldg), returns the gradient of <Gbar, X> with
 * respect to A, i.e. the solution Y (ldy) of X^T Y + Y X^T = Gbar.  Uses the
 * saved low-precision factors (X = Q S Q^H) for the correction solves
 * (Eq. (triangsylv) with the transposed operator) and refines with FP64
 * residuals Gbar - X^T Y - Y X^T until the relative residual is <= tol.
 * Returns 8 when no forward factors are stored. */
SQRTM_API int sqrtm_backward(sqrtm_handle_t handle, const double *dGbar, int64_t n, int64_t ldg,
                   double tol, double *dY, int64_t ldy, sqrtm_info *info);

/* Factors of one forward call, owned by the caller.  sqrtm_backward always
 * uses the factors of the handle's LAST forward call, so a program that
 * differentiates through several square roots (several sqrtm_mixed calls
 * before their backward passes) must keep each call's factors apart:
 *
 *   sqrtm_factors_take moves the factors that the last sqrtm_mixed call on
 *   the handle saved (general: Q, S in complex FP32; SPD: V, s = sqrt(lam)
 *   in FP32; both: the FP64 X returned, the scale exponent e) into a new
 *   factor object, without a copy.  The handle keeps no factors afterwards
 *   (sqrtm_backward then returns 8) and its next forward call allocates new
 *   factor storage.  Returns 0, -1 (handle NULL), -2 (out NULL), 8 (no
 *   factors saved: no forward call yet, or the last one was a method that
 *   keeps none -- the FP64 Schur method, the cube root, complex input, the
 *   real variant, or a call that failed), 7 (host allocation failure).
 *
 *   sqrtm_backward_factors is sqrtm_backward with the factors of f in place
 *   of the handle's: the adjoint solve X^T Y + Y X^T = Gbar (Eq.
 *   (triangsylv) with the transposed operator, refined with FP64 residuals)
 *   for the X of the call that produced f.  The work runs on the handle's
 *   stream; f's memory was written on the stream of the handle that
 *   produced it, so a caller on another stream orders the two itself.
 *   Arguments: 1 handle, 2 f, 3 dGbar, 4 n (must equal f's size, else 8),
 *   5 ldg, 6 tol, 7 dY, 8 ldy, 9 info; return codes as sqrtm_backward.
 *   f is not consumed: it may serve several backward passes.
 *
 *   sqrtm_factors_n returns f's matrix size (-1 for NULL).
 *   sqrtm_factors_destroy frees f and its device memory (cudaFree, which
 *   waits for the device); NULL is accepted.  Returns 0. */
typedef struct sqrtm_factors_s *sqrtm_factors_t;
SQRTM_API int sqrtm_factors_take(sqrtm_handle_t handle, sqrtm_factors_t *f);
SQRTM_API int sqrtm_backward_factors(sqrtm_handle_t handle, sqrtm_factors_t f, const double *dGbar, int64_t n,
                                     int64_t ldg, double tol, double *dY, int64_t ldy, sqrtm_info *info);
SQRTM_API int64_t sqrtm_factors_n(sqrtm_factors_t f);
SQRTM_API int sqrtm_factors_destroy(sqrtm_factors_t f);

/* Batched mixed-precision square roots of independent matrices of varying
 * sizes.  dA, dX: HOST arrays of `batch` device pointers; n, lda, ldx: HOST
 * arrays of sizes.  status: HOST array of `batch` ints receiving each
 * matrix's code.  opts may be NULL.  Returns the first nonzero code, else 0.
 * When the call stops before any matrix is solved (an invalid argument --
 * for a member, the code sqrtm_mixed would return for it -- or a failure
 * to set up worker streams), every status[i] receives the returned code.
 * Matrices of the sizes the tuning table marks `batched` (without a table:
 * n <= 256; the environment variable SQRTM_BATCH_MAXN, if set, is the size
 * limit instead) go through one batched general path: every stage of
 * Algorithm 2 is one launch over all of them, the convergence test runs per
 * matrix on the device and each refinement step is replayed from a CUDA
 * graph until no matrix is active (a symmetric matrix takes Algorithm 2 there
 * too).  The others, and every matrix when opts->kind is SQRTM_KIND_SPD, are
 * solved by per-matrix calls on up to 12 worker streams, concurrently with
 * the batched path. */
SQRTM_API int sqrtm_mixed_batched(sqrtm_handle_t handle, int batch, const double *const *dA,
                        const int64_t *n, const int64_t *lda, double tol,
                        double *const *dX, const int64_t *ldx, const sqrtm_opts *opts,
                        int *status);

/* Phase times of the last batched-path graph on this handle (diagnostic,
 * device clock, ms): [0] norms, scaling and Hessenberg reductions, [1] QR
 * rounds of the general members, [2] Jacobi decompositions of the
 * symmetric members, [3] triangular square roots and X_0, [4] refinement
 * loop.  Copies min(cap, 5) values into ms (HOST), the number of matrices
 * the batched path took into *count and how many of them took Algorithm 2
 * into *general (either may be NULL).  Returns 5, or -1 / -2 (NULL handle /
 * ms). */
SQRTM_API int sqrtm_batched_phases(sqrtm_handle_t handle, double *ms, int cap, int *count, int *general);

/* Split a batch of independent matrices over `parts` GPUs (one process per
 * GPU, each calling sqrtm_mixed_batched on its share; no data crosses GPUs,
 * so no collective is needed on the data path).  Longest-processing-time
 * rule with the cost n^3 of the O(n^3) stages (Schur decomposition,
 * transforms, Sylvester solves): matrices in decreasing cost (ties: lower
 * index first), each to the part with the smallest total so far (ties:
 * lowest part), which bounds the largest part by 4/3 of the optimum.
 * Deterministic, so every process computes the same partition.
 *   n: HOST array of `batch` sizes; owner: HOST array receiving each
 *   matrix's part (0 .. parts-1); load: optional HOST array of `parts`
 *   doubles receiving each part's total cost.
 * Host-only (no CUDA call).  Returns 0, -1 (batch < 0), -2 (n NULL or a
 * negative size), -3 (parts < 1), -4 (owner NULL). */
SQRTM_API int sqrtm_batch_partition(int batch, const int64_t *n, int parts, int *owner, double *load);

/* Number of CUDA kernel launches this library has issued in the process so
 * far (all handles, all threads).  Diagnostic; never resets. */
SQRTM_API int64_t sqrtm_kernel_launches(void);

/* Text describing the first CUDA failure (status 7) recorded on the handle
 * since it was created: the CUDA error name and where it happened; "" if
 * none.  Owned by the handle. */
SQRTM_API const char *sqrtm_last_error(sqrtm_handle_t handle);

/* Human-readable text for a status code (static storage). */
SQRTM_API const char *sqrtm_status_string(int code);

#ifdef __cplusplus
}
#endif

#endif /* SQRTM_MP_H */
