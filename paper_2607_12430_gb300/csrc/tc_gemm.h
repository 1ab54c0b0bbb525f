// tc_gemm.h -- split-TF32 tcgen05 GEMM (see tc_gemm.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sqm {

enum {
    TC_EPI_STORE = 0,
    TC_EPI_DIAG_SOLVE = 1,
    TC_EPI_SYM_ADD_F64 = 2,
    // complex results: accumulator columns 2j, 2j+1 are Re, Im of column j
    TC_EPI_CSTORE = 3,     // C complex (interleaved), column-major: C(i, j) at C[2 (i + j ldc)]
    TC_EPI_CSTORE_T = 4,   // the same entry stored transposed: at C[2 (j + i ldc)]
    // real parts only (accumulator column j is Re of column j), FP64 output
    TC_EPI_RE_F64_STORE = 5,  // X(i, j) = scale acc(i, j)
    TC_EPI_RE_F64_ADD = 6,    // X(i, j) += scale acc(i, j)
};

struct TcEpilogue {
    float *C;          // TC_EPI_STORE / TC_EPI_DIAG_SOLVE: FP32 output, column-major;
                       // TC_EPI_CSTORE(_T): interleaved complex output, ldc in complex elements
    int64_t ldc;
    const float *s;    // TC_EPI_DIAG_SOLVE: C_ij = (AB)_ij / (s_i + s_j)
    double *X;         // TC_EPI_SYM_ADD_F64: X_ij = X_ji = X_ij + scale (AB)_ij (i <= j)
    int64_t ldx;
    double scale;
};

// true when the operands meet the TMA rules (16-byte aligned base and
// leading dimension) and the driver exposes the tensor-map encoder
bool tc_gemm_supported(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb, const void *A,
                       const void *B);

// C = A B, A(i,k) = A[k + i lda], B(k,j) = B[k + j ldb]; err receives 6 if a
// bounded wait inside the kernel gives up
cudaError_t launch_tc3_gemm(int M, int N, int K, const float *A, int lda, const float *B, int ldb,
                            int epi, const TcEpilogue &ep, int *err, cudaStream_t s);

// Complex products on the same kernel.  The left operand's row i is a
// complex vector stored contiguously as interleaved (re, im) FP32 pairs,
// a(i, l) at A[2 (l + i lda)] (lda in complex elements), and is read as a
// real vector of length 2k; the right operand Y (k x n complex) is first
// re-laid into a real 2k x 2n matrix B (tc_relayout_*), column 2j holding
// (Re y_lj, -s_a s_y Im y_lj)_l and column 2j+1 (s_y Im y_lj, s_a Re y_lj)_l
// interleaved, so that one real product gives Re (AY)_ij in accumulator
// column 2j and Im (AY)_ij in column 2j+1; s_a = -1 conjugates the stored
// left rows, s_y = -1 conjugates Y.  With re_only, B has only the n
// columns 2j (the real part).  Bld: leading dimension of B in floats
// (a multiple of 4, >= 2k).
cudaError_t launch_tc_relayout_cplx(const void *Y, int64_t ldy, int k, int n, float sa, float sy, bool re_only,
                                    float *B, int64_t ldb, cudaStream_t s);
// the same for a real Y (k x n FP32, ldy): imaginary parts zero
cudaError_t launch_tc_relayout_real(const float *Y, int64_t ldy, int k, int n, float sa, float *B, int64_t ldb,
                                    cudaStream_t s);
// Q^T of a complex n x n matrix (ld n), no conjugation
cudaError_t launch_ctranspose(const void *Q, void *Qt, int n, cudaStream_t s);
// C = A Y with A (M x K complex rows, see above) and B the re-laid Y:
// epi TC_EPI_CSTORE / TC_EPI_CSTORE_T (N complex columns) or
// TC_EPI_RE_F64_STORE / TC_EPI_RE_F64_ADD (N real columns, re_only B)
cudaError_t launch_tc_cgemm(int M, int N, int K, const void *A, int lda_c, const float *B, int ldb, int epi,
                            const TcEpilogue &ep, int *err, cudaStream_t s);
// whether the complex path applies: TMA alignment of the operands (2 lda_c
// and ldb floats multiples of 4, 16-byte aligned bases)
bool tc_cgemm_supported(int64_t lda_c, int64_t ldb, const void *A, const void *B);

}  // namespace sqm
