// quasi.cu -- real arithmetic for real A (Remark 2.1): the square root of a
// real quasi-upper-triangular T (1x1 diagonal blocks for real eigenvalues,
// 2x2 blocks for complex conjugate pairs) and the Sylvester solve
// S Y + Y St = C with quasi-triangular S, St, in the storage precision R
// (float or double), never cutting a 2x2 block.
//
// Both go one block diagonal (square root) or one block anti-diagonal
// (Sylvester) per launch: every block of it is independent, one warp per
// block forms its right-hand side by warp-parallel dot products and lane 0
// solves the block's p x q Sylvester equation (p, q <= 2) through its
// Kronecker form, a system of at most 4 unknowns.
#include "internal.h"

namespace sqm {

static constexpr int kQWarps = 4;  // blocks per CTA (one warp each)

// block starts of quasi-triangular T: blk[0 .. nb] (blk[nb] = n), *nb_out
template <class R>
__global__ void qblocks_kernel(const R *__restrict__ T, int ld, int n, int *__restrict__ blk, int *__restrict__ nb_out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int nb = 0, i = 0;
    while (i < n) {
        blk[nb++] = i;
        i += (i + 1 < n && T[(i + 1) + (int64_t)i * ld] != R(0)) ? 2 : 1;
    }
    blk[nb] = n;
    *nb_out = nb;
}

// A Y + Y B = C for p x q blocks (p, q <= 2); A (lda), B (ldb) small upper
// quasi-triangular blocks, C in y[r + c p]; returns false if singular
template <class R>
__device__ bool small_sylvester(int p, int q, const R *A, int64_t lda, const R *B, int64_t ldb, R y[4])
{
    const int m = p * q;
    R K[4][5];
    for (int c = 0; c < q; ++c)
        for (int r = 0; r < p; ++r) {
            const int row = r + c * p;
            for (int cc = 0; cc < q; ++cc)
                for (int rr = 0; rr < p; ++rr)
                    K[row][rr + cc * p] = (cc == c ? A[r + rr * lda] : R(0)) + (rr == r ? B[cc + c * ldb] : R(0));
            K[row][m] = y[row];
        }
    for (int col = 0; col < m; ++col) {
        int piv = col;
        for (int r = col + 1; r < m; ++r)
            if (fabs(K[r][col]) > fabs(K[piv][col])) piv = r;
        if (K[piv][col] == R(0)) return false;
        if (piv != col)
            for (int e = 0; e <= m; ++e) {
                const R t = K[col][e];
                K[col][e] = K[piv][e];
                K[piv][e] = t;
            }
        for (int r = col + 1; r < m; ++r) {
            const R f = K[r][col] / K[col][col];
            for (int e = col; e <= m; ++e) K[r][e] -= f * K[col][e];
        }
    }
    for (int r = m - 1; r >= 0; --r) {
        R acc = K[r][m];
        for (int e = r + 1; e < m; ++e) acc -= K[r][e] * y[e];
        y[r] = acc / K[r][r];
    }
    return true;
}

// diagonal blocks of S = T^{1/2}: sqrt(t) for 1x1 (t > 0), and for a 2x2
// block with eigenvalues theta +- i mu, alpha I + (T_ii - theta I) / (2 alpha)
// with alpha = Re sqrt(theta + i mu) (the principal root of the pair)
template <class R>
__global__ void qsqrt_diag_kernel(const R *__restrict__ T, int ldt, R *__restrict__ S, int lds,
                                  const int *__restrict__ blk, const int *__restrict__ nbp, int *status)
{
    const int nb = *nbp;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int i0 = blk[b], p = blk[b + 1] - i0;
    const R a = T[i0 + (int64_t)i0 * ldt];
    if (p == 1) {
        if (!(a > R(0))) { atomicExch(status, 2); return; }
        S[i0 + (int64_t)i0 * lds] = sqrt(a);
        return;
    }
    const R bb = T[i0 + (int64_t)(i0 + 1) * ldt], c = T[(i0 + 1) + (int64_t)i0 * ldt];
    const R d = T[(i0 + 1) + (int64_t)(i0 + 1) * ldt];
    const R theta = R(0.5) * (a + d);
    const R mu2 = -(R(0.25) * (a - d) * (a - d) + bb * c);
    if (!(mu2 > R(0))) { atomicExch(status, 2); return; }
    const R mu = sqrt(mu2);
    // Re sqrt(theta + i mu) without cancellation: t = sqrt((|theta| + |z|) / 2)
    // is the real part for theta >= 0, mu / (2 t) otherwise
    const R t = sqrt(R(0.5) * (fabs(theta) + hypot(theta, mu)));
    const R alpha = theta >= R(0) ? t : mu / (R(2) * t);
    const R inv = R(1) / (R(2) * alpha);
    S[i0 + (int64_t)i0 * lds] = alpha + (a - theta) * inv;
    S[i0 + (int64_t)(i0 + 1) * lds] = bb * inv;
    S[(i0 + 1) + (int64_t)i0 * lds] = c * inv;
    S[(i0 + 1) + (int64_t)(i0 + 1) * lds] = alpha + (d - theta) * inv;
}

// block superdiagonal `dist` of S: S_ii S_ij + S_ij S_jj = T_ij - sum S_ik S_kj
template <class R>
__global__ void __launch_bounds__(32 * kQWarps)
qsqrt_off_kernel(const R *__restrict__ T, int ldt, R *S, int lds, const int *__restrict__ blk,
                 const int *__restrict__ nbp, int dist, int *status)
{
    const int nb = *nbp;
    const int lane = threadIdx.x & 31;
    const int bi = blockIdx.x * kQWarps + (threadIdx.x >> 5), bj = bi + dist;
    if (bj >= nb) return;  // whole warp
    const int i0 = blk[bi], p = blk[bi + 1] - i0, j0 = blk[bj], q = blk[bj + 1] - j0;
    const int k0 = blk[bi + 1];
    R y[4];
    for (int c = 0; c < q; ++c)
        for (int r = 0; r < p; ++r) {
            R acc = R(0);
            for (int k = k0 + lane; k < j0; k += 32) acc = fma(S[(i0 + r) + (int64_t)k * lds], S[k + (int64_t)(j0 + c) * lds], acc);
            acc = warp_sum(acc);
            y[r + c * p] = T[(i0 + r) + (int64_t)(j0 + c) * ldt] - acc;
        }
    if (lane != 0) return;
    if (!small_sylvester<R>(p, q, S + i0 + (int64_t)i0 * lds, lds, S + j0 + (int64_t)j0 * lds, lds, y)) {
        atomicExch(status, 2);
        return;
    }
    for (int c = 0; c < q; ++c)
        for (int r = 0; r < p; ++r) S[(i0 + r) + (int64_t)(j0 + c) * lds] = y[r + c * p];
}

// block anti-diagonal w of S Y + Y St = C (block rows of S bottom-up, block
// columns of St left to right): block (I, J) with (nbm - 1 - I) + J = w
template <class R>
__global__ void __launch_bounds__(32 * kQWarps)
qrtrsyl_wave_kernel(const R *__restrict__ S, int lds, const int *__restrict__ bm, const int *__restrict__ nbmp, int m,
                    const R *__restrict__ St, int ldst, const int *__restrict__ bn, const int *__restrict__ nbnp,
                    R *C, int ldc, int w, int *status)
{
    const int nbm = *nbmp, nbn = *nbnp;
    const int lane = threadIdx.x & 31;
    const int g = blockIdx.x * kQWarps + (threadIdx.x >> 5);
    const int I = max(0, (nbm - 1) - w) + g;
    const int J = w - (nbm - 1 - I);
    if (I >= nbm || J < 0 || J >= nbn) return;  // whole warp
    const int i0 = bm[I], p = bm[I + 1] - i0, j0 = bn[J], q = bn[J + 1] - j0;
    const int k0 = bm[I + 1];
    R y[4];
    for (int c = 0; c < q; ++c)
        for (int r = 0; r < p; ++r) {
            R acc = R(0);
            for (int k = k0 + lane; k < m; k += 32) acc = fma(S[(i0 + r) + (int64_t)k * lds], C[k + (int64_t)(j0 + c) * ldc], acc);
            for (int l = lane; l < j0; l += 32) acc = fma(C[(i0 + r) + (int64_t)l * ldc], St[l + (int64_t)(j0 + c) * ldst], acc);
            acc = warp_sum(acc);
            y[r + c * p] = C[(i0 + r) + (int64_t)(j0 + c) * ldc] - acc;
        }
    if (lane != 0) return;
    if (!small_sylvester<R>(p, q, S + i0 + (int64_t)i0 * lds, lds, St + j0 + (int64_t)j0 * ldst, ldst, y)) {
        atomicExch(status, 2);
        return;
    }
    for (int c = 0; c < q; ++c)
        for (int r = 0; r < p; ++r) C[(i0 + r) + (int64_t)(j0 + c) * ldc] = y[r + c * p];
}

// scratch: blk (n + 1 ints) and nb (1 int) on the device; h_nb: pinned or
// pageable host int (the launch count needs nb on the host)
template <class R>
cudaError_t launch_qtrisqrt(const R *T, int ldt, R *S, int lds, int n, int *d_blk, int *d_nb, int *d_status,
                            cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    cudaError_t err;
    qblocks_kernel<R><<<1, 32, 0, s>>>(T, ldt, n, d_blk, d_nb); count_launch();
    int nb = 0;
    if ((err = cudaMemcpyAsync(&nb, d_nb, sizeof(int), cudaMemcpyDeviceToHost, s))) return err;
    if ((err = cudaStreamSynchronize(s))) return err;
    if ((err = cudaMemset2DAsync(S, (size_t)lds * sizeof(R), 0, (size_t)n * sizeof(R), (size_t)n, s))) return err;
    qsqrt_diag_kernel<R><<<cdiv_i(nb, 128), 128, 0, s>>>(T, ldt, S, lds, d_blk, d_nb, d_status); count_launch();
    for (int dist = 1; dist < nb; ++dist) {
        qsqrt_off_kernel<R><<<cdiv_i(nb - dist, kQWarps), 32 * kQWarps, 0, s>>>(T, ldt, S, lds, d_blk, d_nb, dist,
                                                                                d_status);
        count_launch();
    }
    return cudaGetLastError();
}

// scratch: bm (m + 1), bn (nn + 1), nbs (2 ints)
template <class R>
cudaError_t launch_qrtrsyl(const R *S, int lds, int m, const R *St, int ldst, int nn, R *C, int ldc, int *d_bm,
                           int *d_bn, int *d_nbs, int *d_status, cudaStream_t s)
{
    if (m <= 0 || nn <= 0) return cudaSuccess;
    cudaError_t err;
    qblocks_kernel<R><<<1, 32, 0, s>>>(S, lds, m, d_bm, d_nbs); count_launch();
    qblocks_kernel<R><<<1, 32, 0, s>>>(St, ldst, nn, d_bn, d_nbs + 1); count_launch();
    int nbs[2] = {0, 0};
    if ((err = cudaMemcpyAsync(nbs, d_nbs, 2 * sizeof(int), cudaMemcpyDeviceToHost, s))) return err;
    if ((err = cudaStreamSynchronize(s))) return err;
    const int nbm = nbs[0], nbn = nbs[1];
    for (int w = 0; w <= nbm + nbn - 2; ++w) {
        const int cnt = min(w, nbm + nbn - 2 - w) + 1;  // blocks on the anti-diagonal, at most
        qrtrsyl_wave_kernel<R><<<cdiv_i(cnt, kQWarps), 32 * kQWarps, 0, s>>>(S, lds, d_bm, d_nbs, m, St, ldst, d_bn,
                                                                             d_nbs + 1, C, ldc, w, d_status);
        count_launch();
    }
    return cudaGetLastError();
}

template cudaError_t launch_qtrisqrt<float>(const float *, int, float *, int, int, int *, int *, int *, cudaStream_t);
template cudaError_t launch_qtrisqrt<double>(const double *, int, double *, int, int, int *, int *, int *,
                                             cudaStream_t);
template cudaError_t launch_qrtrsyl<float>(const float *, int, int, const float *, int, int, float *, int, int *, int *,
                                           int *, int *, cudaStream_t);
template cudaError_t launch_qrtrsyl<double>(const double *, int, int, const double *, int, int, double *, int, int *,
                                            int *, int *, int *, cudaStream_t);

}  // namespace sqm
