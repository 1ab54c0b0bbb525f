// tc_gemm.h -- split-TF32 tcgen05 GEMM (see tc_gemm.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sqm {

enum { TC_EPI_STORE = 0, TC_EPI_DIAG_SOLVE = 1, TC_EPI_SYM_ADD_F64 = 2 };

struct TcEpilogue {
    float *C;          // TC_EPI_STORE / TC_EPI_DIAG_SOLVE: FP32 output, column-major
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

}  // namespace sqm
