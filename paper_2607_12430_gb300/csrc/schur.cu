// schur.cu -- complex Schur decomposition A_s = Q T Q^H in the storage
// precision R (FP32 for the mixed-precision method, FP64 for the plain Schur
// method): Householder reduction to Hessenberg form, then single-shift
// (Wilkinson) implicit QR sweeps (Sec. 1 and Algorithm 2, step 1).
//
// Hessenberg: two launches per column k.  hess_left applies the reflector
// P = I - beta v v^H from the left (one warp per column: dot + rank-1),
// hess_right from the right to H and accumulates Q <- Q P (one row per lane,
// split over 8 column segments).  Every CTA of hess_left recomputes the
// reflector from column k, which no CTA writes during that launch.
//
// The QR sweeps that follow the reduction are in qr.cu.
#include "internal.h"

namespace sqm {

static constexpr int kHessThreads = 256;

// ---------------------------------------------------------------------------
// Householder reflector for x = H(k+1:n, k): v = x + phase(x0) ||x|| e1,
// beta = 2 / ||v||^2; P x = -phase ||x|| e1.  beta = 0 when the tail of x is
// already zero (no reflection needed).
// ---------------------------------------------------------------------------
template <class R>
__device__ void block_reflector(const cplx<R> *__restrict__ col, int m, cplx<R> *vsh,
                                R *s_scal /* [beta, xnorm, ph.x, ph.y] */)
{
    __shared__ R red[2][kHessThreads / 32];
    R t_all = 0, t_tail = 0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        cplx<R> x = col[i];
        vsh[i] = x;
        R a = abs2(x);
        t_all += a;
        if (i > 0) t_tail += a;
    }
    t_all = warp_sum(t_all);
    t_tail = warp_sum(t_tail);
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { red[0][w] = t_all; red[1][w] = t_tail; }
    __syncthreads();
    if (threadIdx.x == 0) {
        R xn2 = 0, tail2 = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { xn2 += red[0][q]; tail2 += red[1][q]; }
        if (tail2 == R(0) || m <= 0) {
            s_scal[0] = 0; s_scal[1] = 0; s_scal[2] = 1; s_scal[3] = 0;
        } else {
            R xn = sqrt(xn2);
            cplx<R> x0 = vsh[0];
            R ax0 = hypot(x0.x, x0.y);
            cplx<R> ph = (ax0 == R(0)) ? cplx<R>{R(1), R(0)} : cplx<R>{x0.x / ax0, x0.y / ax0};
            // |v0|^2 = (|x0| + ||x||)^2
            R v0abs = ax0 + xn;
            R vn2 = v0abs * v0abs + tail2;
            vsh[0] = cplx<R>{ph.x * v0abs, ph.y * v0abs};
            s_scal[0] = R(2) / vn2;
            s_scal[1] = xn;
            s_scal[2] = ph.x;
            s_scal[3] = ph.y;
        }
    }
    __syncthreads();
}

template <class R>
__global__ void __launch_bounds__(kHessThreads)
hess_left_kernel(const SchurDesc<R> *__restrict__ descs, int k)
{
    extern __shared__ unsigned char smraw[];
    cplx<R> *vsh = reinterpret_cast<cplx<R> *>(smraw);
    __shared__ R s_scal[4];
    const SchurDesc<R> d = descs[blockIdx.y];
    const int n = d.n, ld = d.ld;
    if (k + 2 >= n) return;
    const int m = n - k - 1;
    cplx<R> *H = d.T;
    block_reflector<R>(H + (k + 1) + (int64_t)k * ld, m, vsh, s_scal);
    const R beta = s_scal[0];
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < m; i += blockDim.x) d.v[i] = vsh[i];
        if (threadIdx.x < 4) d.beta[threadIdx.x] = s_scal[threadIdx.x];
    }
    if (beta == R(0)) return;
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int j = k + 1 + gw; j < n; j += nw) {
        cplx<R> *c = H + (k + 1) + (int64_t)j * ld;
        cplx<R> acc{0, 0};
#pragma unroll 8
        for (int i = lane; i < m; i += 32) cfma(acc, conj(vsh[i]), c[i]);
        acc = warp_sum(acc);
        cplx<R> w = beta * acc;
#pragma unroll 8
        for (int i = lane; i < m; i += 32) cfms(c[i], vsh[i], w);
    }
}

// Rows of H (t < n) and of Q (t >= n); blockDim = (HR_ROWS, HR_SEGS): x = row
// in the tile, y = column segment (partial dot products reduced in shared
// memory).
static constexpr int HR_ROWS = 16, HR_SEGS = 16;

template <class R>
__global__ void __launch_bounds__(kHessThreads)
hess_right_kernel(const SchurDesc<R> *__restrict__ descs, int k)
{
    extern __shared__ unsigned char smraw[];
    cplx<R> *vsh = reinterpret_cast<cplx<R> *>(smraw);
    __shared__ cplx<R> part[HR_SEGS][HR_ROWS + 1];
    const SchurDesc<R> d = descs[blockIdx.y];
    const int n = d.n, ld = d.ld;
    if (k + 2 >= n) return;
    const int m = n - k - 1;
    const R beta = d.beta[0];
    const int tid = threadIdx.y * HR_ROWS + threadIdx.x;
    for (int i = tid; i < m; i += HR_ROWS * HR_SEGS) vsh[i] = d.v[i];
    if (blockIdx.x == 0 && beta != R(0)) {
        // column k of H becomes [.., -phase ||x||, 0, ..., 0]
        cplx<R> *col = d.T + (k + 1) + (int64_t)k * ld;
        const R xn = d.beta[1];
        for (int i = tid; i < m; i += HR_ROWS * HR_SEGS)
            col[i] = (i == 0) ? cplx<R>{-d.beta[2] * xn, -d.beta[3] * xn} : cplx<R>{0, 0};
    }
    __syncthreads();
    if (beta == R(0)) return;
    const int row0 = blockIdx.x * HR_ROWS;
    if (row0 >= 2 * n) return;
    const int t = row0 + threadIdx.x;
    const bool valid = t < 2 * n;
    cplx<R> *M = (t < n) ? d.T : d.Q;
    const int i = (t < n) ? t : t - n;
    cplx<R> acc{0, 0}, acc2{0, 0};
    if (valid) {
        const cplx<R> *base = M + i + (int64_t)(k + 1) * ld;
        int l = threadIdx.y;
#pragma unroll 4
        for (; l + HR_SEGS < m; l += 2 * HR_SEGS) {
            cfma(acc, base[(int64_t)l * ld], vsh[l]);
            cfma(acc2, base[(int64_t)(l + HR_SEGS) * ld], vsh[l + HR_SEGS]);
        }
        if (l < m) cfma(acc, base[(int64_t)l * ld], vsh[l]);
        acc += acc2;
    }
    part[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    cplx<R> u{0, 0};
#pragma unroll
    for (int q = 0; q < HR_SEGS; ++q) u += part[q][threadIdx.x];
    u = beta * u;
    if (valid) {
#pragma unroll 8
        for (int l = threadIdx.y; l < m; l += HR_SEGS) {
            cplx<R> &e = M[i + (int64_t)(k + 1 + l) * ld];
            cfms(e, u, conj(vsh[l]));
        }
    }
}

template <class R>
__global__ void eye_kernel(const SchurDesc<R> *__restrict__ descs)
{
    const SchurDesc<R> d = descs[blockIdx.y];
    const int n = d.n, ld = d.ld;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)n * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(t % n), j = (int)(t / n);
        d.Q[i + (int64_t)j * ld] = cplx<R>{(R)(i == j), R(0)};
    }
}

template <class R>
cudaError_t launch_hessenberg(const SchurDesc<R> *d_desc, int batch, int nmax,
                              int ctas_per_matrix, cudaStream_t s)
{
    size_t smem = (size_t)(nmax > 0 ? nmax : 1) * sizeof(cplx<R>);
    cudaError_t err;
    if (smem > 48 * 1024) {
        if ((err = allow_max_smem((const void *)hess_left_kernel<R>)))
            return err;
        if ((err = allow_max_smem((const void *)hess_right_kernel<R>)))
            return err;
    }
    eye_kernel<R><<<dim3(64, batch), 256, 0, s>>>(d_desc); count_launch();
    for (int k = 0; k + 2 < nmax; ++k) {
        int m = nmax - k - 1;
        int left_ctas = (int)cdiv_i(m, kHessThreads / 32);
        if (left_ctas > ctas_per_matrix) left_ctas = ctas_per_matrix;
        hess_left_kernel<R><<<dim3(left_ctas, batch), kHessThreads, smem, s>>>(d_desc, k); count_launch();
        int right_ctas = (int)cdiv_i(2 * nmax, HR_ROWS);
        hess_right_kernel<R><<<dim3(right_ctas, batch), dim3(HR_ROWS, HR_SEGS), smem, s>>>(d_desc, k); count_launch();
    }
    return cudaGetLastError();
}

template cudaError_t launch_hessenberg<float>(const SchurDesc<float> *, int, int, int, cudaStream_t);
template cudaError_t launch_hessenberg<double>(const SchurDesc<double> *, int, int, int, cudaStream_t);

}  // namespace sqm
