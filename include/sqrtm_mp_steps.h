/*
 * sqrtm_mp_steps.h -- the individual steps of the mixed-precision matrix
 * square root (arXiv 2607.12430, Algorithms 1-3), each exposed on raw device
 * pointers so that it can be checked and timed on its own.  sqrtm_mixed
 * (sqrtm_mp.h) chains exactly these kernels.
 *
 * Layouts: column-major.  "c64" arrays are interleaved complex FP32
 * (re, im) pairs, "c128" interleaved complex FP64; real arrays are float or
 * double as named.  Square low-precision work arrays use leading dimension
 * n.  `fp64` selects the FP64 instantiation of a step (complex128 / double
 * storage) instead of the low-precision one (complex64 / float).
 * All pointers are device pointers unless named *_host.  Work runs on the
 * handle's stream; calls that return a scalar synchronise the stream.
 * Return values use the codes of sqrtm_mp.h.
 */
#ifndef SQRTM_MP_STEPS_H
#define SQRTM_MP_STEPS_H

#include <stdint.h>
#include "sqrtm_mp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Scaling before the cast to low precision (Sec. 5 asks for an overflow-safe
 * scaling without fixing one): e with ||A||_F / sqrt(n) = m 2^p, m in
 * [1/2, 1), e = ceil(p/2); A_s = 4^-e A, stored as complex (imaginary part
 * 0) in dAs (n x n, ld n; c64, or c128 when fp64).  *e_host receives e,
 * *norm_host ||A||_F. */
SQRTM_API int sqrtm_step_scale(sqrtm_handle_t h, const double *dA, int64_t n, int64_t lda, void *dAs,
                     int fp64, int *e_host, double *norm_host);

/* Householder reduction of a REAL matrix to upper Hessenberg form, the
 * first stage of the Schur decomposition (Algorithm 2, step 1) as the
 * general path runs it beyond the sizes its one-cluster kernel holds:
 * A = Q H Q^T with Q = P_0 ... P_{n-3}, P_k = I - beta_k v_k v_k^T acting
 * on rows / columns k+1 .. n-1, v_k = x + sign(x_0) ||x|| e_1 for
 * x = H(k+1:n, k) (the sign convention of the complex reduction with the
 * phase of x_0).  The reduction runs in real arithmetic in the storage
 * precision (fp64 ? FP64 : FP32), three launches per column over the whole
 * GPU; Q is formed from the stored reflectors by the blocked compact-WY
 * back-transform.  dA: real FP64 n x n (lda), rounded to the storage
 * precision first; dH, dQ: complex (complex64 or complex128 by fp64) n x n
 * outputs, ld n, imaginary parts zero, H zero below the subdiagonal.
 * Returns -2/-5/-6 for a NULL dA/dH/dQ, -3 (n < 0 or n > 46340), -4
 * (lda < n), 7 on a CUDA error. */
SQRTM_API int sqrtm_step_hessenberg(sqrtm_handle_t h, const double *dA, int64_t n, int64_t lda, void *dH, void *dQ,
                                    int fp64);

/* Complex Schur decomposition (Algorithm 2, step 1): dT (in: A_s, out: T
 * upper triangular) and dQ (out: unitary) with A_s = Q T Q^H: Householder
 * Hessenberg reduction, then single-shift QR sweeps.  Returns 0 or 3. */
SQRTM_API int sqrtm_step_schur(sqrtm_handle_t h, void *dT, void *dQ, int64_t n, int fp64);

/* Symmetric eigendecomposition (Algorithm 3, step 1) of the real symmetric
 * A_s held in the real part of dAs: dV (out, real n x n, float or double)
 * and dlam (out, n).  Returns 0 or 3. */
SQRTM_API int sqrtm_step_syevd(sqrtm_handle_t h, const void *dAs, void *dV, void *dlam, int64_t n,
                     int fp64);

/* Triangular square root S = T^{1/2} (Algorithm 2, step 2; blocked method of
 * Sec. 2.2.1 with Eq. (subst) inside diagonal blocks).  dT, dS: upper
 * triangular n x n.  Returns 0 or 2. */
SQRTM_API int sqrtm_step_trisqrt(sqrtm_handle_t h, const void *dT, void *dS, int64_t n, int blks,
                       int fp64);

/* Triangular cube root (Sec. 4, p = 3): S = T^{1/3} with every diagonal
 * entry the principal cube root (argument in (-pi/3, pi/3]) and V = S^2, by
 * the blocked recurrence from S^3 = T (b x b blocks, b = min(blks, 32);
 * inside a block the point recurrence s_ij (s_ii^2 + s_ii s_jj + s_jj^2) =
 * t_ij - s_ii p_ij - sum_{i<k<j} s_ik v_kj with p_ij = sum_{i<k<j} s_ik s_kj).
 * dT, dS, dV: upper triangular n x n (ld n), complex of the precision fp64
 * selects (c64 or c128); the strict lower triangles of dS and dV are
 * written with zeros.  Returns 0, or 2 for an eigenvalue on or next to the
 * closed negative real axis. */
SQRTM_API int sqrtm_step_tricbrt(sqrtm_handle_t h, const void *dT, void *dS, void *dV, int64_t n, int blks,
                                 int fp64);

/* The same triangular square root by the recursive splitting of Sec. 2.2.1
 * (the Deadman-Higham-Ralha recursion): T split at m (n/2 rounded up to a
 * multiple of 32), S_11 and S_22 recursively, S_12 from S_11 S_12 + S_12
 * S_22 = T_12 by the blocked Sylvester solver; blocks of at most cutoff
 * (>= 64; smaller values are raised to 64) take the blocked method.
 * Returns 0 or 2. */
SQRTM_API int sqrtm_step_trisqrt_rec(sqrtm_handle_t h, const void *dT, void *dS, int64_t n, int blks, int cutoff,
                                     int fp64);

/* Real Schur form (Remark 2.1) in one CTA: dT (in: real n x n matrix, out:
 * quasi-upper-triangular T, 2x2 diagonal blocks only for complex conjugate
 * pairs) and dQ (out: orthogonal Q, A = Q T Q^T), float or double (fp64),
 * ld n, n <= 2048 (else -4); Householder reduction, then double-shift sweeps.
 * Returns 0 or 3 (iteration cap). */
SQRTM_API int sqrtm_step_real_schur(sqrtm_handle_t h, void *dT, void *dQ, int64_t n, int fp64);

/* Real quasi-triangular square root (Remark 2.1): S = T^{1/2} for real
 * quasi-upper-triangular T (1x1 diagonal blocks for real eigenvalues, 2x2
 * blocks for complex conjugate pairs, a 2x2 block marked by a nonzero
 * subdiagonal entry).  A 1x1 block gives sqrt(t); a 2x2 block with
 * eigenvalues theta +- i mu gives alpha I + (T_ii - theta I) / (2 alpha),
 * alpha = Re sqrt(theta + i mu); block (i, j) then solves S_ii S_ij +
 * S_ij S_jj = T_ij - sum_k S_ik S_kj, one block diagonal per launch.  dT,
 * dS: real n x n (ld n), float (fp64 = 0) or double.  Returns 0, or 2 for a
 * real eigenvalue <= 0 or a singular block equation. */
SQRTM_API int sqrtm_step_qtrisqrt(sqrtm_handle_t h, const void *dT, void *dS, int64_t n, int fp64);

/* S Y + Y St = C for real quasi-upper-triangular S (m x m, ld m) and St
 * (nn x nn, ld nn), never cutting a 2x2 block: block anti-diagonals of the
 * block grid in order, each block from its p x q Sylvester equation
 * (p, q <= 2).  dC (m x nn, ld m) is overwritten by Y.  Returns 0 or 2. */
SQRTM_API int sqrtm_step_qrtrsyl(sqrtm_handle_t h, const void *dS, int64_t m, const void *dSt, int64_t nn, void *dC,
                                 int fp64);

/* X_0 = Re(Q S Q^H) (Algorithm 2, step 3), computed in the storage
 * precision of Q and S, rounded to that precision and written widened to
 * FP64 into dX (ldx), times 2^e (undoing the scaling). */
SQRTM_API int sqrtm_step_form_x0(sqrtm_handle_t h, const void *dQ, const void *dS, int64_t n, int e,
                       double *dX, int64_t ldx, int fp64);

/* Residual (Algorithm 2, step 5) on the scaled problem: R = 4^-e A - X_s X_s
 * with X_s = 2^-e X, in FP64; writes fl32(R) into dRhat (float n x n) and
 * ||R||_F into *norm_host. */
SQRTM_API int sqrtm_step_residual(sqrtm_handle_t h, const double *dA, int64_t lda, const double *dX,
                        int64_t ldx, int64_t n, int e, float *dRhat, double *norm_host);

/* Transform (Algorithm 2, step 8): dRt = Q^H Rhat Q in low precision (Q c64,
 * Rhat float, Rt c64). */
SQRTM_API int sqrtm_step_transform_in(sqrtm_handle_t h, const void *dQ, const float *dRhat, void *dRt,
                            int64_t n);

/* Triangular Sylvester solve S Y + Y St = C (Algorithm 2, step 9;
 * Algorithm 1 computes the same Y): S m x m and St nn x nn upper triangular
 * (c64, ld m and nn), dC (c64, m x nn, ld m) overwritten by Y.  With
 * blks = 32, m a multiple of 16 and more than one block, one launch ordered
 * by block dependencies; otherwise one launch per block wavefront (the same
 * block equations and sums either way).  Returns 0, 2, or 6 if a bounded
 * wait between blocks gave up. */
SQRTM_API int sqrtm_step_rtrsyl(sqrtm_handle_t h, const void *dS, int64_t m, const void *dSt,
                      int64_t nn, void *dC, int blks);

/* Correction equation of the cube root's refinement (Eq. (3rd-order)):
 * S^2 Y + S Y S + Y S^2 = C for upper triangular S with V = S^2 (from
 * sqrtm_step_tricbrt), by b x b block anti-diagonal wavefronts that keep
 * Z = Y S alongside Y.  dS, dV, dC: n x n (ld n), complex of the precision
 * fp64 selects; dC is overwritten by Y.  Returns 0, or 2 for a vanishing
 * denominator s_ii^2 + s_ii s_jj + s_jj^2. */
SQRTM_API int sqrtm_step_rtrsyl3(sqrtm_handle_t h, const void *dS, const void *dV, void *dC, int64_t n, int blks,
                                 int fp64);

/* Back-transform and update (Algorithm 2, steps 10-11): dX += 2^e Re(Q Y
 * Q^H), product in low precision, addition in FP64.  Q, Y c64. */
SQRTM_API int sqrtm_step_transform_out_update(sqrtm_handle_t h, const void *dQ, const void *dY,
                                    int64_t n, int e, double *dX, int64_t ldx);

/* SPD transform with the diagonal Sylvester solve fused (Algorithm 3, steps
 * 8-9): dY = (V^T Rhat V) ./ (s_i + s_j), s_i = sqrt(lam_i).  V, Y float. */
SQRTM_API int sqrtm_step_transform_in_spd(sqrtm_handle_t h, const float *dV, const float *dlam,
                                const float *dRhat, float *dY, int64_t n);

/* SPD back-transform and update (Algorithm 3, steps 10-11):
 * dX += 2^e V Y V^T, symmetrised; V, Y float. */
SQRTM_API int sqrtm_step_transform_out_update_spd(sqrtm_handle_t h, const float *dV, const float *dY,
                                        int64_t n, int e, double *dX, int64_t ldx);

/* Low-precision dense product on the tensor cores (the transforms of
 * Algorithm 3, steps 8 and 10, in split-TF32): C = A B in FP32 with
 * A(i, k) = dA[k + i*lda] (M x K, rows contiguous) and B(k, j) = dB[k + j*ldb]
 * (K x N, columns contiguous); dC column-major (ldc).  Each operand is split
 * into two TF32 terms and C = A_hi B_hi + A_hi B_lo + A_lo B_hi is accumulated
 * in FP32 (tcgen05, sm_103a).  lda and ldb must be multiples of 4 and the
 * bases 16-byte aligned (TMA rules); returns -4 otherwise, 6 if a device-side
 * bounded wait gave up. */
SQRTM_API int sqrtm_step_gemm_tf32x3(sqrtm_handle_t h, int64_t M, int64_t N, int64_t K,
                                     const float *dA, int64_t lda, const float *dB, int64_t ldb,
                                     float *dC, int64_t ldc);

/* Complex low-precision product on the tensor cores (the transforms of
 * Algorithm 2, steps 3, 8 and 10, in split-TF32): C = op(A) op(Y), complex
 * FP32 interleaved (re, im), with row i of A stored contiguously,
 * A(i, l) = dA[l + i*lda] (M x K), op(A) = conj(A) when conj_a; Y (K x N)
 * column-major, Y(l, j) = dY[l + j*ldy], op(Y) = conj(Y) when conj_y; C
 * (M x N) column-major (ldc); all leading dimensions in complex elements.
 * Y is re-laid into a real 2K x 2N matrix (in the handle's workspace) so
 * that one real split-TF32 product over the interleaved operands gives the
 * real and imaginary parts side by side.  Returns -2 (a negative size), -5
 * (a NULL pointer), -6 (a leading dimension too small, or lda odd / a base
 * not 16-byte aligned: the TMA rules), 6 if a device-side bounded wait gave
 * up. */
SQRTM_API int sqrtm_step_cgemm_tf32x3(sqrtm_handle_t h, int64_t M, int64_t N, int64_t K, const void *dA,
                                      int64_t lda, int conj_a, const void *dY, int64_t ldy, int conj_y, void *dC,
                                      int64_t ldc);

/* Residual of the symmetric positive definite path (Algorithm 3, step 5)
 * for symmetric X: R = 4^-e A - X_s X_s with X_s = 2^-e X, FP64 accuracy;
 * writes fl32(R) (mirrored) into dRhat (float n x n) and ||R||_F into
 * *norm_host.  split = 0: X X by FP64 products on the CUDA cores;
 * split = 1: X X from exact BF16 tensor-core products of digit slices of X
 * summed in FP64 (error-free splitting; terms left out below
 * n 2^(rho_i + rho_j - 56), 2^rho_i bounding row i of X); returns -10 when
 * the splitting does not apply to n.  Status 6: a bounded wait inside a
 * tensor-core kernel gave up. */
SQRTM_API int sqrtm_step_residual_sym(sqrtm_handle_t h, const double *dA, int64_t lda, const double *dX,
                                      int64_t ldx, int64_t n, int e, float *dRhat, double *norm_host,
                                      int split);

/* Residual of the general path (Algorithm 2, step 4: R = A - X^2 in
 * double precision) with X^2 from exact BF16 tensor-core products of digit
 * slices: the rows of X (from a transposed copy) against its columns, every
 * output tile, products summed in FP64 (error-free splitting as in
 * sqrtm_step_residual_sym; terms left out below n 2^(rho_i + gamma_j - 56),
 * 2^rho_i bounding row i and 2^gamma_j column j of X).  Same scaling and
 * outputs as sqrtm_step_residual: fl32(4^-e A - (2^-e X)^2) into dRhat
 * (float n x n, ld n), ||R||_F into *norm_host.  Memory: dA, dX n x n FP64
 * column-major (lda, ldx), device, owned by the caller; the digit slices,
 * X^T and the FP64 tile accumulator live in the handle's workspace.  Errors:
 * -1 no handle, -3 lda < n, -5 ldx < n, -6 n < 0 or n > 46340, -10 the
 * splitting does not apply to n (n 2^(2b) > 2^24 for every digit width b),
 * 6 a bounded wait inside the tensor-core kernel gave up, 7 a CUDA error. */
SQRTM_API int sqrtm_step_residual_split(sqrtm_handle_t h, const double *dA, int64_t lda, const double *dX,
                                        int64_t ldx, int64_t n, int e, float *dRhat, double *norm_host);

/* The residual above for callers that cannot allocate device memory.  The
 * paper has no counterpart: this is a library service.  It takes no handle
 * (a handle allocates its workspace on first use); its scratch -- the norm's
 * per-block partial sums -- is a fixed array inside this library, held on
 * every GPU that loads the library until the process exits.
 *   dA, dX: n x n FP64 (lda, ldx); dRhat: n x n FP32 output (ld n) receiving
 *   fl32((4^-e A - (2^-e X)^2)); norm_host: optional host pointer receiving
 *   ||R||_F (when given the call waits for the GPU); stream: cudaStream_t.
 * Argument positions for the error codes: 1 dA, 2 lda, 3 dX, 4 ldx, 5 n,
 * 6 e, 7 dRhat, 8 norm_host, 9 stream; a NULL dA, dX or dRhat returns -1,
 * -3 or -7.
 * Limits: n <= 4096, otherwise -5 (checked before anything is launched).
 * Calls no cudaMalloc or cudaFree and no allocating library routine.  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * While a stream is being captured, pass norm_host = NULL: reading the norm
 * back waits for the stream, which a capture does not allow; the norm is
 * then computed but stays in the library's array, out of the caller's
 * reach, and only dRhat is the call's result.  All calls share the one
 * array: calls that overlap on the GPU race on it.  Nothing in it needs to
 * start at zero: each call writes every partial it later reads. */
SQRTM_API int sqrtm_step_residual_noalloc(const double *dA, int64_t lda, const double *dX,
                                          int64_t ldx, int64_t n, int e, float *dRhat,
                                          double *norm_host, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SQRTM_MP_STEPS_H */
