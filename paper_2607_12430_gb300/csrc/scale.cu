// scale.cu -- Frobenius norm, power-of-4 scaling and the cast of A to low
// precision (the overflow-safe scaling that Sec. 5 asks for before data is
// converted to the lower precision).
//
// e is fixed from ||A||_F / sqrt(n) = m 2^p, m in [1/2, 1): e = ceil(p/2).
// A_s = 4^-e A is exact in binary floating point, and sqrt(A) = 2^e sqrt(A_s)
// exactly, so the scaling never adds rounding error.
#include "internal.h"

namespace sqm {

static constexpr int kNormThreads = 256;

// Per-CTA partial sum of squares over columns assigned round-robin; the
// partials are summed in a fixed order by finalize, so the norm (and the
// exponent derived from it) is bit-reproducible.
__global__ void norm_partials_kernel(const double *__restrict__ A, int64_t rows, int64_t cols, int64_t lda,
                                     double *__restrict__ partials)
{
    __shared__ double red[kNormThreads / 32];
    double acc = 0.0;
    for (int64_t j = blockIdx.x; j < cols; j += gridDim.x) {
        const double *col = A + j * lda;
        for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) {
            double v = col[i];
            acc = fma(v, v, acc);
        }
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        partials[blockIdx.x] = t;
    }
}

__global__ void norm_finalize_kernel(const double *__restrict__ partials, int np, int64_t n,
                                     double *d_norm, int *d_e, int root)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < np; ++i) s += partials[i];
    double nrm = sqrt(s);
    *d_norm = nrm;
    int e = 0;
    if (n > 0 && nrm > 0.0 && isfinite(nrm)) {
        double r = sqrt(s / (double)n);
        int p;
        frexp(r, &p);
        e = (p >= 0) ? (p + root - 1) / root : -((-p) / root);  // ceil(p / root)
    }
    *d_e = e;
}

cudaError_t launch_norm_scale(const double *A, int64_t n, int64_t lda, double *partials,
                              int nblk, double *d_norm, int *d_e, cudaStream_t s, int root)
{
    if (nblk < 1) nblk = 1;
    norm_partials_kernel<<<nblk, kNormThreads, 0, s>>>(A, n, n, lda, partials); count_launch();
    norm_finalize_kernel<<<1, 32, 0, s>>>(partials, nblk, n, d_norm, d_e, root); count_launch();
    return cudaGetLastError();
}

// complex A (interleaved FP64 pairs, lda in complex elements): the same
// norm over its 2n x n real view
cudaError_t launch_norm_scale_z(const double *A, int64_t n, int64_t lda, double *partials, int nblk, double *d_norm,
                                int *d_e, cudaStream_t s)
{
    if (nblk < 1) nblk = 1;
    norm_partials_kernel<<<nblk, kNormThreads, 0, s>>>(A, 2 * n, n, 2 * lda, partials); count_launch();
    norm_finalize_kernel<<<1, 32, 0, s>>>(partials, nblk, n, d_norm, d_e, 2); count_launch();
    return cudaGetLastError();
}

template <class R>
__global__ void cast_scaled_z_kernel(const double *__restrict__ A, int64_t n, int64_t lda,
                                     const int *__restrict__ d_e, cplx<R> *__restrict__ As, int64_t ldas)
{
    const double sc = ldexp(1.0, -2 * (*d_e));
    const int64_t total = n * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t % n, j = t / n;
        const double *a = A + 2 * (i + j * lda);
        As[i + j * ldas] = cplx<R>{(R)(a[0] * sc), (R)(a[1] * sc)};
    }
}

template <class R>
__global__ void cast_scaled_kernel(const double *__restrict__ A, int64_t n, int64_t lda,
                                   const int *__restrict__ d_e, cplx<R> *__restrict__ As,
                                   int64_t ldas, int root)
{
    double sc = ldexp(1.0, -root * (*d_e));
    int64_t total = n * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = t % n, j = t / n;
        As[i + j * ldas] = cplx<R>{(R)(A[i + j * lda] * sc), R(0)};
    }
}

template <class R>
__global__ void cast_scaled_real_kernel(const double *__restrict__ A, int64_t n, int64_t lda,
                                        const int *__restrict__ d_e, R *__restrict__ As,
                                        int64_t ldas)
{
    double sc = ldexp(1.0, -2 * (*d_e));
    int64_t total = n * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = t % n, j = t / n;
        As[i + j * ldas] = (R)(A[i + j * lda] * sc);
    }
}

static int grid_for(int64_t total)
{
    int64_t g = cdiv_i(total, 256);
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
}

template <class R>
cudaError_t launch_cast_scaled(const double *A, int64_t n, int64_t lda, const int *d_e,
                               cplx<R> *As, int64_t ldas, cudaStream_t s, int root)
{
    cast_scaled_kernel<R><<<grid_for(n * n), 256, 0, s>>>(A, n, lda, d_e, As, ldas, root); count_launch();
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_cast_scaled_z(const double *A, int64_t n, int64_t lda, const int *d_e, cplx<R> *As, int64_t ldas,
                                 cudaStream_t s)
{
    cast_scaled_z_kernel<R><<<grid_for(n * n), 256, 0, s>>>(A, n, lda, d_e, As, ldas); count_launch();
    return cudaGetLastError();
}

template cudaError_t launch_cast_scaled_z<float>(const double *, int64_t, int64_t, const int *, cplx<float> *, int64_t,
                                                 cudaStream_t);
template cudaError_t launch_cast_scaled_z<double>(const double *, int64_t, int64_t, const int *, cplx<double> *,
                                                  int64_t, cudaStream_t);

template <class R>
cudaError_t launch_cast_scaled_real(const double *A, int64_t n, int64_t lda, const int *d_e,
                                    R *As, int64_t ldas, cudaStream_t s)
{
    cast_scaled_real_kernel<R><<<grid_for(n * n), 256, 0, s>>>(A, n, lda, d_e, As, ldas); count_launch();
    return cudaGetLastError();
}

template cudaError_t launch_cast_scaled<float>(const double *, int64_t, int64_t, const int *,
                                                cplx<float> *, int64_t, cudaStream_t, int);
template cudaError_t launch_cast_scaled<double>(const double *, int64_t, int64_t, const int *,
                                                cplx<double> *, int64_t, cudaStream_t, int);
template cudaError_t launch_cast_scaled_real<float>(const double *, int64_t, int64_t,
                                                    const int *, float *, int64_t, cudaStream_t);
template cudaError_t launch_cast_scaled_real<double>(const double *, int64_t, int64_t,
                                                     const int *, double *, int64_t,
                                                     cudaStream_t);

}  // namespace sqm
