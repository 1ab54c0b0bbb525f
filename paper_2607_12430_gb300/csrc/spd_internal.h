// spd_internal.h -- launchers of the symmetric positive definite path
// (Algorithm 3): real products, tridiagonalisation and the tridiagonal
// eigensolver.
#pragma once

#include "internal.h"

namespace sqm {

enum { RG_STORE = 0, RG_DIAG_SOLVE = 1, RG_SYM_TO_F64 = 2, RG_SYM_ADD_F64 = 3, RG_ADD_F64 = 4, RG_SUB = 5 };

// C = op(A) op(B), op 0 = N, 1 = T; see rgemm.cu for the epilogues.
template <class R>
cudaError_t launch_rgemm(int opA, int opB, int m, int n, int k, const R *A, int lda, const R *B,
                         int ldb, int epi, R *C, int ldc, const R *s, double *X, int64_t ldx,
                         double scale, cudaStream_t st);

// R = (A - X X) 4^-e for symmetric X; upper tiles, mirrored.
cudaError_t launch_residual_sym_f64(const double *A, int64_t lda, const double *X, int64_t ldx,
                                    int n, int e, float *Rhat, int ldr, double *partials,
                                    int *nparts, cudaStream_t s);

// The same residual with X X from exact BF16 tensor-core products of digit
// slices of X, summed in FP64 (tc_split.cu).  Racc: n x n doubles (ld n)
// of scratch; digits: split_digit_elems(n) BF16 values; rho: n ints; err
// receives 6 if a bounded wait gives up.
bool split_residual_supported(int n);
size_t split_digit_elems(int n);
cudaError_t launch_residual_sym_split(const double *A, int64_t lda, const double *X, int64_t ldx, int n, int e,
                                      float *Rhat, int ldr, double *Racc, void *digits, int *rho,
                                      double *partials, int *nparts, int *err, cudaStream_t s);
// R = (A - X X) 4^-e for a general X by the same splitting: the rows of X
// (from XT = X^T, n x n doubles of scratch) against its columns, every
// output tile.  digitsA, digitsB: split_digit_elems(n) BF16 values each;
// rhoA, rhoB: n ints each; partials: residual_gen_split_parts(n) doubles.
int residual_gen_split_parts(int n);
cudaError_t launch_residual_gen_split(const double *A, int64_t lda, const double *X, int64_t ldx, int n, int e,
                                      float *Rhat, int ldr, double *Racc, double *XT, void *digitsA, void *digitsB,
                                      int *rhoA, int *rhoB, double *partials, int *nparts, int *err, cudaStream_t s);

// Householder tridiagonalisation A = Q Tri Q^T (A overwritten: the
// tridiagonal on its diagonal and first subdiagonal).  Reflector k,
// H_k = I - beta_k y_k y_k^T, is stored as column k of Y (y_k(i) = 0 for
// i <= k; Y must be zero on entry) and beta_k in betas[k]; Q = H_0 H_1 ...
// H_{n-3}.  ws: >= 4 n + 16 elements of R.
template <class R>
cudaError_t launch_tridiag(R *A, int n, int ld, R *Y, int ldy, R *betas, R *ws, cudaStream_t s);

// Z <- Q Z for Q = H_0 ... H_{n-3} from launch_tridiag, applied in blocks of
// kBackNb reflectors in compact WY form (Q_b = I - Y_b T_b Y_b^T, T_b upper
// triangular), last block first.  FP32: two launches (every T_b at once,
// then one CTA per panel of 32 columns of Z applying all blocks to it);
// FP64: three products per block.  Y must be zero outside the reflectors'
// supports.  scratch: >= kBackNb * (kBackNb + 2 n) + kBackNb^2 elements of R.
constexpr int kBackNb = 64;
template <class R>
cudaError_t launch_back_transform(const R *Y, int ldy, const R *betas, R *Z, int n, int ldz, R *scratch,
                                  cudaStream_t s);

// Eigen-decomposition of the symmetric tridiagonal matrix held on the
// diagonal / first subdiagonal of A (FP64 arithmetic): lam (ascending) and
// ZT (row j = unit eigenvector j, n x n, ld n); eigenvectors of eigenvalue
// clusters (closer than the eigenvalues' accuracy) are recomputed by
// projection against all the others.  scratch: 2 n * chunk doubles plus
// 11 n + 24 plus ((n + 6) / 8 + 2) * chunk.
template <class R>
cudaError_t launch_tridiag_eig(const R *A, int n, int ld, double *lam, double *ZT,
                               double *scratch, int chunk, cudaStream_t s);

}  // namespace sqm
