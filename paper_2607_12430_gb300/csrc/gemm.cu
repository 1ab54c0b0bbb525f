// gemm.cu -- dense products of the refinement loop on the CUDA cores:
//   * cgemm: C = op(A) op(B) for complex (or real-times-complex) operands in
//     the storage precision R, 64x64x16 shared-memory tiles, 4x4 outputs per
//     thread, with epilogues that write Re(C) widened to FP64 (X_0) or add it
//     into the FP64 iterate (X_{k+1} = X_k + dX, Algorithm 2 steps 10-11);
//   * residual_f64: R = (A - X X) 4^-e in FP64 (Algorithm 2 step 5) with the
//     cast of R to FP32 and per-CTA partial sums of |R|^2 fused in the
//     epilogue; partials are summed in a fixed order (bit-reproducible norm).
#include "internal.h"

namespace sqm {

static constexpr int GB_M = 64, GB_N = 64, GB_K = 16, G_THREADS = 256;

// BM x 64 output tiles (BM = 64, or 32 where 64-row tiles would leave SMs
// idle); thread (tx, ty) owns rows ty RM .. ty RM + RM - 1 and columns
// 4 tx .. 4 tx + 3.  Every output is accumulated over k in the same order
// whatever BM, so both tile shapes give identical results.
template <class R, int OPA, int OPB, bool AREAL, int EPI, int BM = GB_M>
__global__ void __launch_bounds__(G_THREADS)
cgemm_kernel(int m, int n, int k, const void *__restrict__ Av, int lda,
             const cplx<R> *__restrict__ B, int ldb, cplx<R> *__restrict__ C, int ldc,
             double *__restrict__ X, int64_t ldx, double scale, const GemmJob<R> *__restrict__ jobs)
{
    static_assert(BM == 64 || BM == 32, "tile rows");
    constexpr int RM = BM / 16;  // rows per thread; also A-tile elements per thread
    __shared__ cplx<R> As[GB_K][BM + 1];
    __shared__ cplx<R> Bs[GB_K][GB_N + 1];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * GB_N;
    if (jobs) {  // batched: the n x n product of matrix blockIdx.z, scale 2^e
        const GemmJob<R> jb = jobs[blockIdx.z];
        if (!*jb.active) return;
        m = n = k = lda = ldb = ldc = jb.n;
        if (m0 >= m || n0 >= n) return;
        Av = jb.A; B = jb.B; C = jb.C; X = jb.X; ldx = jb.ldx;
        scale = ldexp(1.0, *jb.e);
    }
    cplx<R> acc[RM][4];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cplx<R>{0, 0};

    const cplx<R> *A = reinterpret_cast<const cplx<R> *>(Av);
    const R *Ar = reinterpret_cast<const R *>(Av);

    for (int k0 = 0; k0 < k; k0 += GB_K) {
        // A tile: op(A)(m0 + i, k0 + kk)
        if (OPA == OP_N) {
#pragma unroll
            for (int q = 0; q < RM; ++q) {
                int i = tid % BM, kk = tid / BM + (G_THREADS / BM) * q;
                int gi = m0 + i, gk = k0 + kk;
                cplx<R> v{0, 0};
                if (gi < m && gk < k) {
                    if (AREAL) v = cplx<R>{Ar[gi + (int64_t)gk * lda], R(0)};
                    else v = A[gi + (int64_t)gk * lda];
                }
                As[kk][i] = v;
            }
        } else {
#pragma unroll
            for (int q = 0; q < RM; ++q) {
                int kk = tid % GB_K, i = tid / GB_K + 16 * q;
                int gi = m0 + i, gk = k0 + kk;
                cplx<R> v{0, 0};
                if (gi < m && gk < k) {
                    if (AREAL) v = cplx<R>{Ar[gk + (int64_t)gi * lda], R(0)};
                    else v = conj(A[gk + (int64_t)gi * lda]);
                }
                As[kk][i] = v;
            }
        }
        // B tile: op(B)(k0 + kk, n0 + j)
        if (OPB == OP_N) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int kk = tid % GB_K, j = tid / GB_K + 16 * q;
                int gk = k0 + kk, gj = n0 + j;
                Bs[kk][j] = (gk < k && gj < n) ? B[gk + (int64_t)gj * ldb] : cplx<R>{0, 0};
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int j = tid % GB_N, kk = tid / GB_N + 4 * q;
                int gk = k0 + kk, gj = n0 + j;
                Bs[kk][j] = (gk < k && gj < n) ? conj(B[gj + (int64_t)gk * ldb]) : cplx<R>{0, 0};
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GB_K; ++kk) {
            cplx<R> a[RM], b[4];
#pragma unroll
            for (int i = 0; i < RM; ++i) a[i] = As[kk][ty * RM + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < RM; ++i) {
        int gi = m0 + ty * RM + i;
        if (gi >= m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gj = n0 + tx * 4 + j;
            if (gj >= n) continue;
            if (EPI == EPI_STORE) C[gi + (int64_t)gj * ldc] = acc[i][j];
            else if (EPI == EPI_REAL_TO_F64) X[gi + gj * ldx] = (double)((R)acc[i][j].x) * scale;
            else if (EPI == EPI_REAL_ADD_F64) X[gi + gj * ldx] += (double)acc[i][j].x * scale;
            else if (EPI == EPI_CPLX_TO_F64) {
                double *x = X + 2 * (gi + gj * ldx);
                x[0] = (double)((R)acc[i][j].x) * scale;
                x[1] = (double)((R)acc[i][j].y) * scale;
            } else if (EPI == EPI_CPLX_ADD_F64) {
                double *x = X + 2 * (gi + gj * ldx);
                x[0] += (double)acc[i][j].x * scale;
                x[1] += (double)acc[i][j].y * scale;
            } else X[gj + gi * ldx] += (double)acc[i][j].x * scale;
        }
    }
}

template <class R, int OPA, int OPB, bool AREAL, int BM = GB_M>
static cudaError_t dispatch_epi(int epi, dim3 g, cudaStream_t s, int m, int n, int k,
                                const void *A, int lda, const cplx<R> *B, int ldb, cplx<R> *C,
                                int ldc, double *X, int64_t ldx, double scale, const GemmJob<R> *jobs = nullptr)
{
    switch (epi) {
    case EPI_STORE:
        cgemm_kernel<R, OPA, OPB, AREAL, EPI_STORE, BM><<<g, G_THREADS, 0, s>>>(m, n, k, A, lda, B, ldb, C, ldc, X, ldx, scale, jobs); count_launch();
        break;
    case EPI_REAL_TO_F64:
        cgemm_kernel<R, OPA, OPB, AREAL, EPI_REAL_TO_F64, BM><<<g, G_THREADS, 0, s>>>(m, n, k, A, lda, B, ldb, C, ldc, X, ldx, scale, jobs); count_launch();
        break;
    case EPI_REAL_ADD_F64:
        cgemm_kernel<R, OPA, OPB, AREAL, EPI_REAL_ADD_F64, BM><<<g, G_THREADS, 0, s>>>(m, n, k, A, lda, B, ldb, C, ldc, X, ldx, scale, jobs); count_launch();
        break;
    case EPI_CPLX_TO_F64:
        if (AREAL) return cudaErrorInvalidValue;
        cgemm_kernel<R, OPA, OPB, AREAL, EPI_CPLX_TO_F64, BM><<<g, G_THREADS, 0, s>>>(m, n, k, A, lda, B, ldb, C, ldc, X, ldx, scale, jobs); count_launch();
        break;
    case EPI_CPLX_ADD_F64:
        if (AREAL) return cudaErrorInvalidValue;
        cgemm_kernel<R, OPA, OPB, AREAL, EPI_CPLX_ADD_F64, BM><<<g, G_THREADS, 0, s>>>(m, n, k, A, lda, B, ldb, C, ldc, X, ldx, scale, jobs); count_launch();
        break;
    default:
        cgemm_kernel<R, OPA, OPB, AREAL, EPI_REAL_ADD_F64_T, BM><<<g, G_THREADS, 0, s>>>(m, n, k, A, lda, B, ldb, C, ldc, X, ldx, scale, jobs); count_launch();
    }
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_cgemm(int opA, int opB, int m, int n, int k, const void *A, int lda,
                         bool a_real, const cplx<R> *B, int ldb, int epi, cplx<R> *C, int ldc,
                         double *X, int64_t ldx, double scale, cudaStream_t s)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    // FP32: 32-row tiles where 64-row ones would not give every SM a tile
    if constexpr (sizeof(R) == 4) {
        static const int sms = [] {
            int dev = 0, v = 0;
            if (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                v = 0;
            return v;
        }();
        if (sms > 0 && cdiv_i(m, GB_M) * cdiv_i(n, GB_N) < sms) {
            dim3 g((unsigned)cdiv_i(m, 32), (unsigned)cdiv_i(n, GB_N));
#define SQM_D(OA, OB, AR) return dispatch_epi<R, OA, OB, AR, 32>(epi, g, s, m, n, k, A, lda, B, ldb, C, ldc, X, ldx, scale)
            if (a_real) {
                if (opA == OP_N && opB == OP_N) SQM_D(OP_N, OP_N, true);
                if (opA == OP_N && opB == OP_H) SQM_D(OP_N, OP_H, true);
                if (opA == OP_H && opB == OP_N) SQM_D(OP_H, OP_N, true);
                return cudaErrorInvalidValue;
            }
            if (opA == OP_N && opB == OP_N) SQM_D(OP_N, OP_N, false);
            if (opA == OP_N && opB == OP_H) SQM_D(OP_N, OP_H, false);
            if (opA == OP_H && opB == OP_N) SQM_D(OP_H, OP_N, false);
            SQM_D(OP_H, OP_H, false);
#undef SQM_D
        }
    }
    dim3 g((unsigned)cdiv_i(m, GB_M), (unsigned)cdiv_i(n, GB_N));
#define SQM_D(OA, OB, AR) return dispatch_epi<R, OA, OB, AR>(epi, g, s, m, n, k, A, lda, B, ldb, C, ldc, X, ldx, scale)
    if (a_real) {
        if (opA == OP_N && opB == OP_N) SQM_D(OP_N, OP_N, true);
        if (opA == OP_N && opB == OP_H) SQM_D(OP_N, OP_H, true);
        if (opA == OP_H && opB == OP_N) SQM_D(OP_H, OP_N, true);
        return cudaErrorInvalidValue;
    }
    if (opA == OP_N && opB == OP_N) SQM_D(OP_N, OP_N, false);
    if (opA == OP_N && opB == OP_H) SQM_D(OP_N, OP_H, false);
    if (opA == OP_H && opB == OP_N) SQM_D(OP_H, OP_N, false);
    SQM_D(OP_H, OP_H, false);
#undef SQM_D
}

template <class R>
cudaError_t launch_cgemm_batched(int opA, int opB, bool a_real, int epi, const GemmJob<R> *jobs, int batch, int nmax,
                                 cudaStream_t s)
{
    if (nmax <= 0 || batch <= 0) return cudaSuccess;
    dim3 g((unsigned)cdiv_i(nmax, GB_M), (unsigned)cdiv_i(nmax, GB_N), (unsigned)batch);
#define SQM_D(OA, OB, AR) return dispatch_epi<R, OA, OB, AR>(epi, g, s, 0, 0, 0, nullptr, 0, nullptr, 0, nullptr, 0, nullptr, 0, 0.0, jobs)
    if (a_real) {
        if (opA == OP_N && opB == OP_N) SQM_D(OP_N, OP_N, true);
        return cudaErrorInvalidValue;
    }
    if (opA == OP_N && opB == OP_N) SQM_D(OP_N, OP_N, false);
    if (opA == OP_N && opB == OP_H) SQM_D(OP_N, OP_H, false);
    if (opA == OP_H && opB == OP_N) SQM_D(OP_H, OP_N, false);
    return cudaErrorInvalidValue;
#undef SQM_D
}

template cudaError_t launch_cgemm_batched<float>(int, int, bool, int, const GemmJob<float> *, int, int, cudaStream_t);
template cudaError_t launch_cgemm_batched<double>(int, int, bool, int, const GemmJob<double> *, int, int, cudaStream_t);
template cudaError_t launch_cgemm<float>(int, int, int, int, int, const void *, int, bool, const cplx<float> *, int, int, cplx<float> *, int, double *, int64_t, double, cudaStream_t);
template cudaError_t launch_cgemm<double>(int, int, int, int, int, const void *, int, bool, const cplx<double> *, int, int, cplx<double> *, int, double *, int64_t, double, cudaStream_t);

// ---------------------------------------------------------------------------
// FP64 residual
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(G_THREADS)
residual_f64_kernel(const double *__restrict__ A, int64_t lda, const double *__restrict__ X,
                    int64_t ldx, const double *__restrict__ B, int64_t ldb, int n, double sc,
                    float *__restrict__ Rhat, int ldr, double *__restrict__ partials,
                    const ResJob *__restrict__ jobs)
{
    __shared__ double As[GB_K][GB_M + 1];
    __shared__ double Bs[GB_K][GB_N + 1];
    __shared__ double red[G_THREADS / 32];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.x * GB_M, n0 = blockIdx.y * GB_N;
    int part = blockIdx.x + blockIdx.y * gridDim.x;
    if (jobs) {  // batched: R = (A - X X) 4^-e of matrix blockIdx.z
        const ResJob jb = jobs[blockIdx.z];
        if (!*jb.active) return;
        n = ldr = jb.n;
        if (m0 >= n || n0 >= n) return;
        A = jb.A; lda = jb.lda; X = B = jb.X; ldx = ldb = jb.ldx; Rhat = jb.Rhat; partials = jb.partials;
        sc = ldexp(1.0, -2 * *jb.e);
        part = blockIdx.x + blockIdx.y * cdiv_i(n, GB_M);
    }
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < n; k0 += GB_K) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int i = tid % GB_M, kk = tid / GB_M + 4 * q;
            int gi = m0 + i, gk = k0 + kk;
            As[kk][i] = (gi < n && gk < n) ? X[gi + gk * ldx] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int kk = tid % GB_K, j = tid / GB_K + 16 * q;
            int gk = k0 + kk, gj = n0 + j;
            Bs[kk][j] = (gk < n && gj < n) ? B[gk + gj * ldb] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GB_K; ++kk) {
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
            if (gj >= n) continue;
            double r = (A[gi + gj * lda] - acc[i][j]) * sc;
            Rhat[gi + (int64_t)gj * ldr] = (float)r;
            ss = fma(r, r, ss);
        }
    }
    ss = warp_sum(ss);
    if ((tid & 31) == 0) red[tid >> 5] = ss;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < G_THREADS / 32; ++w) t += red[w];
        partials[part] = t;
    }
}

int residual_f64_parts(int n)
{
    return n <= 0 ? 0 : (int)(cdiv_i(n, GB_M) * cdiv_i(n, GB_N));
}

cudaError_t launch_residual_f64(const double *A, int64_t lda, const double *X, int64_t ldx,
                                int n, int e, float *Rhat, int ldr, double *partials,
                                int *nparts, cudaStream_t s)
{
    dim3 g((unsigned)cdiv_i(n, GB_M), (unsigned)cdiv_i(n, GB_N));
    *nparts = (int)(g.x * g.y);
    if (n <= 0) return cudaSuccess;
    residual_f64_kernel<<<g, G_THREADS, 0, s>>>(A, lda, X, ldx, X, ldx, n, ldexp(1.0, -2 * e), Rhat, ldr, partials,
                                                nullptr);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 residual of a complex iterate: R = (A - X X) 4^-e, complex
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(G_THREADS)
zresidual_f64_kernel(const double *__restrict__ A, int64_t lda, const double *__restrict__ X, int64_t ldx, int n,
                     double sc, cplx<float> *__restrict__ Rhat, int ldr, double *__restrict__ partials)
{
    __shared__ cplx<double> As[GB_K][GB_M + 1];
    __shared__ cplx<double> Bs[GB_K][GB_N + 1];
    __shared__ double red[G_THREADS / 32];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.x * GB_M, n0 = blockIdx.y * GB_N;
    const cplx<double> *Xc = reinterpret_cast<const cplx<double> *>(X);
    const cplx<double> *Ac = reinterpret_cast<const cplx<double> *>(A);
    cplx<double> acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cplx<double>{0.0, 0.0};
    for (int k0 = 0; k0 < n; k0 += GB_K) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int i = tid % GB_M, kk = tid / GB_M + 4 * q;
            int gi = m0 + i, gk = k0 + kk;
            As[kk][i] = (gi < n && gk < n) ? Xc[gi + gk * ldx] : cplx<double>{0.0, 0.0};
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int kk = tid % GB_K, j = tid / GB_K + 16 * q;
            int gk = k0 + kk, gj = n0 + j;
            Bs[kk][j] = (gk < n && gj < n) ? Xc[gk + gj * ldx] : cplx<double>{0.0, 0.0};
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GB_K; ++kk) {
            cplx<double> a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
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
            if (gj >= n) continue;
            const cplx<double> a = Ac[gi + gj * lda];
            const double rx = (a.x - acc[i][j].x) * sc, ry = (a.y - acc[i][j].y) * sc;
            Rhat[gi + (int64_t)gj * ldr] = cplx<float>{(float)rx, (float)ry};
            ss = fma(rx, rx, fma(ry, ry, ss));
        }
    }
    ss = warp_sum(ss);
    if ((tid & 31) == 0) red[tid >> 5] = ss;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < G_THREADS / 32; ++w) t += red[w];
        partials[blockIdx.x + blockIdx.y * gridDim.x] = t;
    }
}

cudaError_t launch_zresidual_f64(const double *A, int64_t lda, const double *X, int64_t ldx, int n, int e,
                                 cplx<float> *Rhat, int ldr, double *partials, int *nparts, cudaStream_t s)
{
    dim3 g((unsigned)cdiv_i(n, GB_M), (unsigned)cdiv_i(n, GB_N));
    *nparts = (int)(g.x * g.y);
    if (n <= 0) return cudaSuccess;
    zresidual_f64_kernel<<<g, G_THREADS, 0, s>>>(A, lda, X, ldx, n, ldexp(1.0, -2 * e), Rhat, ldr, partials);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_residual_batched(const ResJob *jobs, int batch, int nmax, cudaStream_t s)
{
    if (nmax <= 0 || batch <= 0) return cudaSuccess;
    dim3 g((unsigned)cdiv_i(nmax, GB_M), (unsigned)cdiv_i(nmax, GB_N), (unsigned)batch);
    residual_f64_kernel<<<g, G_THREADS, 0, s>>>(nullptr, 0, nullptr, 0, nullptr, 0, 0, 0.0, nullptr, 0, nullptr, jobs);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_residual_f64_ab(const double *A, int64_t lda, const double *X, int64_t ldx,
                                   const double *B, int64_t ldb, int n, int shift, float *Rhat, int ldr,
                                   double *partials, int *nparts, cudaStream_t s)
{
    dim3 g((unsigned)cdiv_i(n, GB_M), (unsigned)cdiv_i(n, GB_N));
    *nparts = (int)(g.x * g.y);
    if (n <= 0) return cudaSuccess;
    residual_f64_kernel<<<g, G_THREADS, 0, s>>>(A, lda, X, ldx, B, ldb, n, ldexp(1.0, -shift), Rhat, ldr, partials,
                                                nullptr);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 adjoint residual G - (X^T Y + Y X^T)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(G_THREADS)
adjoint_residual_f64_kernel(const double *__restrict__ G, int64_t ldg, const double *__restrict__ X,
                            int64_t ldx, const double *__restrict__ Y, int64_t ldy, int n,
                            float *__restrict__ Rhat, int ldr, double *__restrict__ partials)
{
    __shared__ double A1[GB_K][GB_M + 1];   // X^T(i, k) = X(k, i)
    __shared__ double B1[GB_K][GB_N + 1];   // Y(k, j)
    __shared__ double A2[GB_K][GB_M + 1];   // Y(i, k)
    __shared__ double B2[GB_K][GB_N + 1];   // X^T(k, j) = X(j, k)
    __shared__ double red[G_THREADS / 32];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.x * GB_M, n0 = blockIdx.y * GB_N;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < n; k0 += GB_K) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int kk = tid % GB_K, i = tid / GB_K + 16 * q;
            int gi = m0 + i, gk = k0 + kk, gj = n0 + i;
            A1[kk][i] = (gi < n && gk < n) ? X[gk + gi * ldx] : 0.0;
            B1[kk][i] = (gj < n && gk < n) ? Y[gk + gj * ldy] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int i = tid % GB_M, kk = tid / GB_M + 4 * q;
            int gi = m0 + i, gk = k0 + kk, gj = n0 + i;
            A2[kk][i] = (gi < n && gk < n) ? Y[gi + gk * ldy] : 0.0;
            B2[kk][i] = (gj < n && gk < n) ? X[gj + gk * ldx] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GB_K; ++kk) {
            double a[4], b[4], c[4], d[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { a[i] = A1[kk][ty * 4 + i]; c[i] = A2[kk][ty * 4 + i]; }
#pragma unroll
            for (int j = 0; j < 4; ++j) { b[j] = B1[kk][tx * 4 + j]; d[j] = B2[kk][tx * 4 + j]; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], fma(c[i], d[j], acc[i][j]));
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
            if (gj >= n) continue;
            double r = G[gi + gj * ldg] - acc[i][j];
            Rhat[gi + (int64_t)gj * ldr] = (float)r;
            ss = fma(r, r, ss);
        }
    }
    ss = warp_sum(ss);
    if ((tid & 31) == 0) red[tid >> 5] = ss;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < G_THREADS / 32; ++w) t += red[w];
        partials[blockIdx.x + blockIdx.y * gridDim.x] = t;
    }
}

cudaError_t launch_adjoint_residual_f64(const double *G, int64_t ldg, const double *X, int64_t ldx,
                                        const double *Y, int64_t ldy, int n, float *Rhat, int ldr,
                                        double *partials, int *nparts, cudaStream_t s)
{
    dim3 g((unsigned)cdiv_i(n, GB_M), (unsigned)cdiv_i(n, GB_N));
    *nparts = (int)(g.x * g.y);
    if (n <= 0) return cudaSuccess;
    adjoint_residual_f64_kernel<<<g, G_THREADS, 0, s>>>(G, ldg, X, ldx, Y, ldy, n, Rhat, ldr, partials); count_launch();
    return cudaGetLastError();
}

__global__ void sum_partials_kernel(const double *__restrict__ p, int np, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < np; ++i) s += p[i];
        *out = sqrt(s);
    }
}

cudaError_t launch_sum_partials(const double *partials, int np, double *d_out, cudaStream_t s)
{
    sum_partials_kernel<<<1, 32, 0, s>>>(partials, np, d_out); count_launch();
    return cudaGetLastError();
}

}  // namespace sqm
