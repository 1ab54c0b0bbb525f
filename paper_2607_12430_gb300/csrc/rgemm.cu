// rgemm.cu -- real dense products of the symmetric positive definite path
// (Algorithm 3) on the CUDA cores, storage precision R:
//   C = op(A) op(B), op in {N, T}, 64x64x16 shared-memory tiles, 4x4 outputs
//   per thread, with epilogues
//     RG_STORE       C = result
//     RG_DIAG_SOLVE  C_ij = result_ij / (s_i + s_j)    (Algorithm 3, step 9)
//     RG_SYM_TO_F64  X_ij = X_ji = double(R(result_ij)) * scale   (X_0)
//     RG_SYM_ADD_F64 X_ij = X_ji = X_ij + double(result_ij) * scale (update)
//     RG_ADD_F64     X_ij += double(result_ij) * scale (no mirroring)
//     RG_SUB         C = C - result
//   The two symmetric epilogues evaluate only tiles on or above the block
//   diagonal and mirror each value, so the FP64 iterate stays exactly
//   symmetric and half of the product is skipped.
// Also the symmetric FP64 residual R = (A - X X) 4^-e for symmetric X,
// upper tiles only, mirrored, with the FP32 cast and the |R|^2 partials
// fused.
#include "internal.h"
#include "spd_internal.h"

namespace sqm {

static constexpr int RB_M = 64, RB_N = 64, RB_K = 16, R_THREADS = 256;

template <class R, int OPA, int OPB, int EPI>
__global__ void __launch_bounds__(R_THREADS)
rgemm_kernel(int m, int n, int k, const R *__restrict__ A, int lda, const R *__restrict__ B,
             int ldb, R *__restrict__ C, int ldc, const R *__restrict__ s, double *__restrict__ X,
             int64_t ldx, double scale)
{
    if ((EPI == RG_SYM_TO_F64 || EPI == RG_SYM_ADD_F64) && blockIdx.x > blockIdx.y) return;
    __shared__ R As[RB_K][RB_M + 4];
    __shared__ R Bs[RB_K][RB_N + 4];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.x * RB_M, n0 = blockIdx.y * RB_N;
    R acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = R(0);
    for (int k0 = 0; k0 < k; k0 += RB_K) {
        if (OPA == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int i = tid % RB_M, kk = tid / RB_M + 4 * q;
                int gi = m0 + i, gk = k0 + kk;
                As[kk][i] = (gi < m && gk < k) ? A[gi + (int64_t)gk * lda] : R(0);
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int kk = tid % RB_K, i = tid / RB_K + 16 * q;
                int gi = m0 + i, gk = k0 + kk;
                As[kk][i] = (gi < m && gk < k) ? A[gk + (int64_t)gi * lda] : R(0);
            }
        }
        if (OPB == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int kk = tid % RB_K, j = tid / RB_K + 16 * q;
                int gk = k0 + kk, gj = n0 + j;
                Bs[kk][j] = (gk < k && gj < n) ? B[gk + (int64_t)gj * ldb] : R(0);
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int j = tid % RB_N, kk = tid / RB_N + 4 * q;
                int gk = k0 + kk, gj = n0 + j;
                Bs[kk][j] = (gk < k && gj < n) ? B[gj + (int64_t)gk * ldb] : R(0);
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < RB_K; ++kk) {
            R a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gi = m0 + ty * 4 + i;
        if (gi >= m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gj = n0 + tx * 4 + j;
            if (gj >= n) continue;
            const R v = acc[i][j];
            if (EPI == RG_STORE) {
                C[gi + (int64_t)gj * ldc] = v;
            } else if (EPI == RG_DIAG_SOLVE) {
                C[gi + (int64_t)gj * ldc] = v / (s[gi] + s[gj]);
            } else if (EPI == RG_SYM_TO_F64) {
                if (gi <= gj) {
                    double x = (double)v * scale;
                    X[gi + gj * ldx] = x;
                    X[gj + gi * ldx] = x;
                }
            } else if (EPI == RG_ADD_F64) {
                X[gi + gj * ldx] += (double)v * scale;
            } else if (EPI == RG_SUB) {
                C[gi + (int64_t)gj * ldc] -= v;
            } else {
                if (gi <= gj) {
                    double x = X[gi + gj * ldx] + (double)v * scale;
                    X[gi + gj * ldx] = x;
                    X[gj + gi * ldx] = x;
                }
            }
        }
    }
}

template <class R, int OPA, int OPB>
static cudaError_t rg_epi(int epi, dim3 g, cudaStream_t st, int m, int n, int k, const R *A,
                          int lda, const R *B, int ldb, R *C, int ldc, const R *s, double *X,
                          int64_t ldx, double scale)
{
    switch (epi) {
    case RG_STORE: rgemm_kernel<R, OPA, OPB, RG_STORE><<<g, R_THREADS, 0, st>>>(m, n, k, A, lda, B, ldb, C, ldc, s, X, ldx, scale); count_launch(); break;
    case RG_DIAG_SOLVE: rgemm_kernel<R, OPA, OPB, RG_DIAG_SOLVE><<<g, R_THREADS, 0, st>>>(m, n, k, A, lda, B, ldb, C, ldc, s, X, ldx, scale); count_launch(); break;
    case RG_SYM_TO_F64: rgemm_kernel<R, OPA, OPB, RG_SYM_TO_F64><<<g, R_THREADS, 0, st>>>(m, n, k, A, lda, B, ldb, C, ldc, s, X, ldx, scale); count_launch(); break;
    case RG_SYM_ADD_F64: rgemm_kernel<R, OPA, OPB, RG_SYM_ADD_F64><<<g, R_THREADS, 0, st>>>(m, n, k, A, lda, B, ldb, C, ldc, s, X, ldx, scale); count_launch(); break;
    case RG_SUB: rgemm_kernel<R, OPA, OPB, RG_SUB><<<g, R_THREADS, 0, st>>>(m, n, k, A, lda, B, ldb, C, ldc, s, X, ldx, scale); count_launch(); break;
    default: rgemm_kernel<R, OPA, OPB, RG_ADD_F64><<<g, R_THREADS, 0, st>>>(m, n, k, A, lda, B, ldb, C, ldc, s, X, ldx, scale); count_launch();
    }
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_rgemm(int opA, int opB, int m, int n, int k, const R *A, int lda, const R *B,
                         int ldb, int epi, R *C, int ldc, const R *s, double *X, int64_t ldx,
                         double scale, cudaStream_t st)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    dim3 g((unsigned)cdiv_i(m, RB_M), (unsigned)cdiv_i(n, RB_N));
    if (opA == 0 && opB == 0) return rg_epi<R, 0, 0>(epi, g, st, m, n, k, A, lda, B, ldb, C, ldc, s, X, ldx, scale);
    if (opA == 0 && opB == 1) return rg_epi<R, 0, 1>(epi, g, st, m, n, k, A, lda, B, ldb, C, ldc, s, X, ldx, scale);
    if (opA == 1 && opB == 0) return rg_epi<R, 1, 0>(epi, g, st, m, n, k, A, lda, B, ldb, C, ldc, s, X, ldx, scale);
    return rg_epi<R, 1, 1>(epi, g, st, m, n, k, A, lda, B, ldb, C, ldc, s, X, ldx, scale);
}

template cudaError_t launch_rgemm<float>(int, int, int, int, int, const float *, int, const float *, int, int, float *, int, const float *, double *, int64_t, double, cudaStream_t);
template cudaError_t launch_rgemm<double>(int, int, int, int, int, const double *, int, const double *, int, int, double *, int, const double *, double *, int64_t, double, cudaStream_t);

// ---------------------------------------------------------------------------
// symmetric FP64 residual
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(R_THREADS)
residual_sym_f64_kernel(const double *__restrict__ A, int64_t lda, const double *__restrict__ X,
                        int64_t ldx, int n, double sc, float *__restrict__ Rhat, int ldr,
                        double *__restrict__ partials)
{
    __shared__ double As[RB_K][RB_M + 1];
    __shared__ double Bs[RB_K][RB_N + 1];
    __shared__ double red[R_THREADS / 32];
    const int tid = threadIdx.x;
    const int pidx = blockIdx.x + blockIdx.y * gridDim.x;
    if (blockIdx.x > blockIdx.y) {
        if (tid == 0) partials[pidx] = 0.0;
        return;
    }
    const int tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.x * RB_M, n0 = blockIdx.y * RB_N;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < n; k0 += RB_K) {
        // (X X)(i, j) = sum_k X(i, k) X(k, j); X symmetric, so X(i, k) = X(k, i)
        // is read along columns for both operands (coalesced)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int kk = tid % RB_K, i = tid / RB_K + 16 * q;
            int gi = m0 + i, gk = k0 + kk;
            As[kk][i] = (gi < n && gk < n) ? X[gk + (int64_t)gi * ldx] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int kk = tid % RB_K, j = tid / RB_K + 16 * q;
            int gk = k0 + kk, gj = n0 + j;
            Bs[kk][j] = (gk < n && gj < n) ? X[gk + (int64_t)gj * ldx] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < RB_K; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    double ss = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int gi = m0 + ty * 4 + i;
        if (gi >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gj = n0 + tx * 4 + j;
            if (gj >= n || gi > gj) continue;
            double r = (A[gi + gj * lda] - acc[i][j]) * sc;
            float rf = (float)r;
            Rhat[gi + (int64_t)gj * ldr] = rf;
            Rhat[gj + (int64_t)gi * ldr] = rf;
            ss = fma(r, r, ss);
            if (gi != gj) ss = fma(r, r, ss);  // mirrored entry
        }
    }
    ss = warp_sum(ss);
    if ((tid & 31) == 0) red[tid >> 5] = ss;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < R_THREADS / 32; ++w) t += red[w];
        partials[pidx] = t;
    }
}

cudaError_t launch_residual_sym_f64(const double *A, int64_t lda, const double *X, int64_t ldx,
                                    int n, int e, float *Rhat, int ldr, double *partials,
                                    int *nparts, cudaStream_t s)
{
    dim3 g((unsigned)cdiv_i(n, RB_M), (unsigned)cdiv_i(n, RB_N));
    *nparts = (int)(g.x * g.y);
    if (n <= 0) return cudaSuccess;
    residual_sym_f64_kernel<<<g, R_THREADS, 0, s>>>(A, lda, X, ldx, n, ldexp(1.0, -2 * e), Rhat, ldr, partials); count_launch();
    return cudaGetLastError();
}

}  // namespace sqm
