// trisolve.cu -- blocked triangular square root and triangular Sylvester
// solver, in the storage precision R.
//
// Both solvers partition their matrices into b x b blocks (b = blks <= 32)
// and solve one block equation per CTA:
//   trisqrt (Sec. 2.2.1, block method):  S_II S_IJ + S_IJ S_JJ =
//       T_IJ - sum_{I<K<J} S_IK S_KJ, diagonal blocks by Eq. (subst);
//   Sylvester (Sec. 2.2.2, the block equations of Eq. (partition) down to
//   b x b leaves):  S_II Y_IJ + Y_IJ St_JJ =
//       C_IJ - sum_{K>I} S_IK Y_KJ - sum_{K<J} Y_IK St_KJ.
// Block (I, J) needs only blocks on earlier wavefronts (J - I smaller for
// trisqrt; larger I or smaller J for the Sylvester solve), so each wavefront
// is one launch whose CTAs are independent.  Inside a CTA the sums are tile
// products in shared memory, dealt round-robin to groups of 128 threads
// (partial sums added in group order), and the leaf equation is solved by
// point Bartels-Stewart substitution along anti-diagonals (4 threads per
// entry).
// The recursion of Algorithm 1 computes the same block equations; only the
// grouping of the update sums differs.
#include "internal.h"

namespace sqm {

static constexpr int TB = 32;       // maximum block edge
static constexpr int TLD = TB + 1;  // padded leading dimension in shared memory
static constexpr int kTriThreads = 128;
// Sylvester: the update terms of a block split over groups of 128 threads
// (4 for complex FP32, 2 for complex FP64: 4 tiles of shared memory each)
template <class R> struct SylCfg { static constexpr int G = sizeof(R) == 4 ? 4 : 2, THREADS = kTriThreads * G; };

template <class R>
__device__ void load_tile(cplx<R> *dst, const cplx<R> *__restrict__ src, int ld, int rows,
                          int cols)
{
    for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
        int i = e % TB, j = e / TB;
        dst[i + j * TLD] = (i < rows && j < cols) ? src[i + (int64_t)j * ld] : cplx<R>{0, 0};
    }
}

// Same tile with cp.async for the in-range part (zero padding written
// directly), by one 128-thread group (lt = thread index within the group);
// complete with cp_async_wait_all() and the group's barrier.
template <class R>
__device__ void load_tile_async_g(cplx<R> *dst, const cplx<R> *__restrict__ src, int ld, int rows, int cols, int lt)
{
    for (int e = lt; e < TB * TB; e += kTriThreads) {
        int i = e % TB, j = e / TB;
        if (i < rows && j < cols) cp_async_elem<R>(&dst[i + j * TLD], &src[i + (int64_t)j * ld]);
        else dst[i + j * TLD] = cplx<R>{0, 0};
    }
}

// barrier of one 128-thread group (named barrier 1 + g)
__device__ __forceinline__ void group_bar(int g)
{
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kTriThreads) : "memory");
}

// acc(r, c_q) -= sum_k A(r, k) B(k, c_q) for the 8 outputs a thread owns
// (row r = lt % 32, columns c_q = lt / 32 + 4 q; lt = thread index within
// its 128-thread group).
template <class R>
__device__ __forceinline__ void tile_mms(cplx<R> (&acc)[8], const cplx<R> *A, const cplx<R> *B,
                                         int kk, int lt)
{
    const int r = lt & 31, c0 = lt >> 5;
    for (int k = 0; k < kk; ++k) {
        cplx<R> a = A[r + k * TLD];
#pragma unroll
        for (int q = 0; q < 8; ++q) cfms(acc[q], a, B[k + (c0 + 4 * q) * TLD]);
    }
}

// Point Bartels-Stewart on a leaf: A (ma x ma) and B (nb x nb) upper
// triangular, C (ma x nb) overwritten by Y with A Y + Y B = C.  Anti-diagonal
// w holds the entries with j - i = w - (ma - 1); each entry depends on
// entries below it in its column and left of it in its row, all on earlier
// anti-diagonals.
template <class R>
__device__ void leaf_sylvester(const cplx<R> *A, const cplx<R> *B, cplx<R> *C, int ma, int nb,
                               int *bad)
{
    const int e = threadIdx.x >> 2, p = threadIdx.x & 3;
    for (int w = 0; w <= ma + nb - 2; ++w) {
        const int ioff = ma - 1 - w;  // j = i - ioff
        const int ilo = max(0, ioff), ihi = min(ma - 1, ioff + nb - 1);
        const int i = ilo + e;
        const bool act = i <= ihi;
        cplx<R> acc{0, 0};
        int j = i - ioff;
        if (act) {
            const int la = ma - 1 - i;  // terms A(i, k) C(k, j), k = i+1 .. ma-1
            const int L = la + j;       // plus C(i, k) B(k, j), k = 0 .. j-1
            for (int t = p; t < L; t += 4) {
                if (t < la) cfma(acc, A[i + (i + 1 + t) * TLD], C[(i + 1 + t) + j * TLD]);
                else { int k = t - la; cfma(acc, C[i + k * TLD], B[k + j * TLD]); }
            }
        }
        acc += shfl_xor(acc, 1);
        acc += shfl_xor(acc, 2);
        if (act && p == 0) {
            cplx<R> den = A[i + i * TLD] + B[j + j * TLD];
            if (den.x == R(0) && den.y == R(0)) { *bad = 1; den = cplx<R>{R(1), R(0)}; }
            C[i + j * TLD] = cdiv(C[i + j * TLD] - acc, den);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Sylvester wavefront: blocks (I, J) with J - I = w - (Mb - 1).  The update
// terms of a block are dealt round-robin to SylCfg<R>::G groups of 128 threads
// (each with its own double-buffered tiles and named barrier); the partial
// sums are added in group order, then the leaf is solved.
// ---------------------------------------------------------------------------
template <class R>
__global__ void __launch_bounds__(SylCfg<R>::THREADS)
rtrsyl_wave_kernel(const cplx<R> *__restrict__ S, int lds, int m, const cplx<R> *__restrict__ St,
                   int ldst, int nn, cplx<R> *C, int ldc, int b, int w, int *status)
{
    extern __shared__ unsigned char smraw[];
    constexpr int TT = TB * TLD, kSylGroups = SylCfg<R>::G;
    cplx<R> *tc = reinterpret_cast<cplx<R> *>(smraw);
    __shared__ int bad;
    const int Mb = (m + b - 1) / b, Nb = (nn + b - 1) / b;
    const int I = max(0, (Mb - 1) - w) + blockIdx.x;
    const int J = I + w - (Mb - 1);
    if (I >= Mb || J >= Nb || J < 0) return;
    const int g = threadIdx.x / kTriThreads, lt = threadIdx.x % kTriThreads;
    cplx<R> *ta = tc + TT * (1 + 4 * g), *tb = ta + TT, *ta2 = tb + TT, *tb2 = ta2 + TT;
    if (threadIdx.x == 0) bad = 0;
    const int i0 = I * b, j0 = J * b;
    const int bm = min(b, m - i0), bn = min(b, nn - j0);
    load_tile(tc, C + i0 + (int64_t)j0 * ldc, ldc, bm, bn);
    __syncthreads();
    cplx<R> acc[8];
    const int r = lt & 31, c0 = lt >> 5;
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = g == 0 ? tc[r + (c0 + 4 * q) * TLD] : cplx<R>{0, 0};
    // update terms: K = I+1..Mb-1 (S_IK Y_KJ), then K = 0..J-1 (Y_IK St_KJ);
    // group g takes terms g, g + G, ...; its tiles of the next term are
    // fetched asynchronously while the current one is multiplied
    const int nterm = (Mb - 1 - I) + J;
    auto issue = [&](int t, cplx<R> *da, cplx<R> *db) {
        if (t < Mb - 1 - I) {
            const int k0 = (I + 1 + t) * b, bk = min(b, m - k0);
            load_tile_async_g(da, S + i0 + (int64_t)k0 * lds, lds, bm, bk, lt);
            load_tile_async_g(db, C + k0 + (int64_t)j0 * ldc, ldc, bk, bn, lt);
        } else {
            const int k0 = (t - (Mb - 1 - I)) * b, bk = min(b, nn - k0);
            load_tile_async_g(da, C + i0 + (int64_t)k0 * ldc, ldc, bm, bk, lt);
            load_tile_async_g(db, St + k0 + (int64_t)j0 * ldst, ldst, bk, bn, lt);
        }
    };
    auto kdim = [&](int t) {
        return (t < Mb - 1 - I) ? min(b, m - (I + 1 + t) * b) : min(b, nn - (t - (Mb - 1 - I)) * b);
    };
    if (g < nterm) issue(g, ta, tb);
    for (int t = g, it = 0; t < nterm; t += kSylGroups, ++it) {
        cplx<R> *ca = (it & 1) ? ta2 : ta, *cb = (it & 1) ? tb2 : tb;
        cp_async_wait_all();
        group_bar(g);
        if (t + kSylGroups < nterm) issue(t + kSylGroups, (it & 1) ? ta : ta2, (it & 1) ? tb : tb2);
        tile_mms(acc, ca, cb, kdim(t), lt);
    }
    __syncthreads();
    // partial sums of groups 1.. into their first tile, added to group 0's in order
    if (g > 0) {
#pragma unroll
        for (int q = 0; q < 8; ++q) ta[r + (c0 + 4 * q) * TLD] = acc[q];
    }
    __syncthreads();
    if (g == 0) {
        for (int h = 1; h < kSylGroups; ++h) {
            const cplx<R> *ph = tc + TT * (1 + 4 * h);
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] += ph[r + (c0 + 4 * q) * TLD];
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) tc[r + (c0 + 4 * q) * TLD] = acc[q];
    }
    __syncthreads();
    cplx<R> *la = tc + TT, *lb = la + TT;  // group 0's tiles, free now
    load_tile(la, S + i0 + (int64_t)i0 * lds, lds, bm, bm);
    load_tile(lb, St + j0 + (int64_t)j0 * ldst, ldst, bn, bn);
    __syncthreads();
    leaf_sylvester(la, lb, tc, bm, bn, &bad);
    for (int e = threadIdx.x; e < bm * bn; e += blockDim.x) {
        int i = e % bm, j = e / bm;
        C[(i0 + i) + (int64_t)(j0 + j) * ldc] = tc[i + j * TLD];
    }
    if (threadIdx.x == 0 && bad) atomicExch(status, 2);
}

// ---------------------------------------------------------------------------
// Triangular square root, block superdiagonal d
// ---------------------------------------------------------------------------
template <class R>
__global__ void __launch_bounds__(kTriThreads)
trisqrt_diag_kernel(const cplx<R> *__restrict__ T, int ldt, cplx<R> *S, int lds, int n, int b,
                    int *status)
{
    extern __shared__ unsigned char smraw[];
    cplx<R> *ts = reinterpret_cast<cplx<R> *>(smraw);  // T block, overwritten by S
    __shared__ int bad;
    const int I = blockIdx.x;
    const int i0 = I * b, bm = min(b, n - i0);
    if (threadIdx.x == 0) bad = 0;
    load_tile(ts, T + i0 + (int64_t)i0 * ldt, ldt, bm, bm);
    __syncthreads();
    const R eps = num<R>::eps;
    if (threadIdx.x < bm) {
        int i = threadIdx.x;
        cplx<R> t = ts[i + i * TLD];
        R at = hypot(t.x, t.y);
        // eigenvalue on (or within rounding of) the closed negative real axis:
        // a real eigenvalue of the real input comes out of the complex Schur
        // form with an imaginary part of about u ||A_s|| (not u |t|), and the
        // scaled matrix has ||A_s||_F / sqrt(n) in [1/4, 1), so "within
        // rounding" is |Im t| <= max(10 u |t|, n u)
        if (t.x <= R(0) && fabs(t.y) <= fmax(R(10) * eps * at, (R)n * eps)) bad = 1;
        ts[i + i * TLD] = csqrt_(t);
    }
    __syncthreads();
    // Eq. (subst) by superdiagonals: s_ij, j - i = dd, from entries with
    // smaller j - i; 4 threads per entry share the inner sum
    const int e = threadIdx.x >> 2, p = threadIdx.x & 3;
    for (int dd = 1; dd < bm; ++dd) {
        const int i = e, j = e + dd;
        const bool act = j < bm;
        cplx<R> acc{0, 0};
        if (act)
            for (int k = i + 1 + p; k < j; k += 4) cfma(acc, ts[i + k * TLD], ts[k + j * TLD]);
        acc += shfl_xor(acc, 1);
        acc += shfl_xor(acc, 2);
        if (act && p == 0) {
            cplx<R> den = ts[i + i * TLD] + ts[j + j * TLD];
            if (den.x == R(0) && den.y == R(0)) { bad = 1; den = cplx<R>{R(1), R(0)}; }
            ts[i + j * TLD] = cdiv(ts[i + j * TLD] - acc, den);
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < bm * bm; q += blockDim.x) {
        int i = q % bm, j = q / bm;
        S[(i0 + i) + (int64_t)(i0 + j) * lds] = (i <= j) ? ts[i + j * TLD] : cplx<R>{0, 0};
    }
    if (threadIdx.x == 0 && bad) atomicExch(status, 2);
}

template <class R>
__global__ void __launch_bounds__(SylCfg<R>::THREADS)
trisqrt_off_kernel(const cplx<R> *__restrict__ T, int ldt, cplx<R> *S, int lds, int n, int b,
                   int dblk, int *status)
{
    extern __shared__ unsigned char smraw[];
    constexpr int TT = TB * TLD, G = SylCfg<R>::G;
    cplx<R> *tc = reinterpret_cast<cplx<R> *>(smraw);
    __shared__ int bad;
    const int Nb = (n + b - 1) / b;
    const int I = blockIdx.x, J = I + dblk;
    if (J >= Nb) return;
    const int g = threadIdx.x / kTriThreads, lt = threadIdx.x % kTriThreads;
    cplx<R> *ta = tc + TT * (1 + 4 * g), *tb = ta + TT, *ta2 = tb + TT, *tb2 = ta2 + TT;
    if (threadIdx.x == 0) bad = 0;
    const int i0 = I * b, j0 = J * b;
    const int bm = min(b, n - i0), bn = min(b, n - j0);
    load_tile(tc, T + i0 + (int64_t)j0 * ldt, ldt, bm, bn);
    __syncthreads();
    cplx<R> acc[8];
    const int r = lt & 31, c0 = lt >> 5;
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = g == 0 ? tc[r + (c0 + 4 * q) * TLD] : cplx<R>{0, 0};
    // K = I+1 .. J-1, dealt round-robin to the G groups of 128 threads
    const int nterm = J - I - 1;
    auto issue = [&](int t, cplx<R> *da, cplx<R> *db) {
        const int k0 = (I + 1 + t) * b, bk = min(b, n - k0);
        load_tile_async_g(da, S + i0 + (int64_t)k0 * lds, lds, bm, bk, lt);
        load_tile_async_g(db, S + k0 + (int64_t)j0 * lds, lds, bk, bn, lt);
    };
    if (g < nterm) issue(g, ta, tb);
    for (int t = g, it = 0; t < nterm; t += G, ++it) {
        cplx<R> *ca = (it & 1) ? ta2 : ta, *cb = (it & 1) ? tb2 : tb;
        cp_async_wait_all();
        group_bar(g);
        if (t + G < nterm) issue(t + G, (it & 1) ? ta : ta2, (it & 1) ? tb : tb2);
        tile_mms(acc, ca, cb, min(b, n - (I + 1 + t) * b), lt);
    }
    __syncthreads();
    if (g > 0) {
#pragma unroll
        for (int q = 0; q < 8; ++q) ta[r + (c0 + 4 * q) * TLD] = acc[q];
    }
    __syncthreads();
    if (g == 0) {
        for (int h = 1; h < G; ++h) {
            const cplx<R> *ph = tc + TT * (1 + 4 * h);
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] += ph[r + (c0 + 4 * q) * TLD];
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) tc[r + (c0 + 4 * q) * TLD] = acc[q];
    }
    __syncthreads();
    cplx<R> *la = tc + TT, *lb = la + TT;
    load_tile(la, S + i0 + (int64_t)i0 * lds, lds, bm, bm);
    load_tile(lb, S + j0 + (int64_t)j0 * lds, lds, bn, bn);
    __syncthreads();
    leaf_sylvester(la, lb, tc, bm, bn, &bad);
    for (int q = threadIdx.x; q < bm * bn; q += blockDim.x) {
        int i = q % bm, j = q / bm;
        S[(i0 + i) + (int64_t)(j0 + j) * lds] = tc[i + j * TLD];
    }
    // the mirrored block below the diagonal is zero
    for (int q = threadIdx.x; q < bn * bm; q += blockDim.x) {
        int i = q % bn, j = q / bn;
        S[(j0 + i) + (int64_t)(i0 + j) * lds] = cplx<R>{0, 0};
    }
    if (threadIdx.x == 0 && bad) atomicExch(status, 2);
}

template <class R>
static cudaError_t set_smem(const void *fn, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return allow_max_smem(fn);
}

template <class R>
cudaError_t launch_trisqrt(const cplx<R> *T, int ldt, cplx<R> *S, int lds, int n, int blks,
                           int *d_status, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int b = blks < 1 ? 1 : (blks > TB ? TB : blks);
    int Nb = (n + b - 1) / b;
    size_t sm1 = TB * TLD * sizeof(cplx<R>), sm3 = (1 + 4 * SylCfg<R>::G) * sm1;
    cudaError_t err;
    if ((err = set_smem<R>((const void *)trisqrt_off_kernel<R>, sm3))) return err;
    trisqrt_diag_kernel<R><<<Nb, kTriThreads, sm1, s>>>(T, ldt, S, lds, n, b, d_status); count_launch();
    for (int dblk = 1; dblk < Nb; ++dblk)
        trisqrt_off_kernel<R><<<Nb - dblk, SylCfg<R>::THREADS, sm3, s>>>(T, ldt, S, lds, n, b, dblk, d_status); count_launch();
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_rtrsyl(const cplx<R> *S, int lds, int m, const cplx<R> *St, int ldst, int nn,
                          cplx<R> *C, int ldc, int blks, int *d_status, cudaStream_t s)
{
    if (m <= 0 || nn <= 0) return cudaSuccess;
    int b = blks < 1 ? 1 : (blks > TB ? TB : blks);
    int Mb = (m + b - 1) / b, Nb = (nn + b - 1) / b;
    size_t sm3 = (1 + 4 * SylCfg<R>::G) * TB * TLD * sizeof(cplx<R>);
    cudaError_t err;
    if ((err = set_smem<R>((const void *)rtrsyl_wave_kernel<R>, sm3))) return err;
    for (int w = 0; w <= Mb + Nb - 2; ++w) {
        int ilo = max(0, (Mb - 1) - w);
        int ihi = min(Mb - 1, (Mb - 1) - w + (Nb - 1));
        int cnt = ihi - ilo + 1;
        if (cnt <= 0) continue;
        rtrsyl_wave_kernel<R><<<cnt, SylCfg<R>::THREADS, sm3, s>>>(S, lds, m, St, ldst, nn, C, ldc, b, w, d_status); count_launch();
    }
    return cudaGetLastError();
}

template cudaError_t launch_trisqrt<float>(const cplx<float> *, int, cplx<float> *, int, int, int, int *, cudaStream_t);
template cudaError_t launch_trisqrt<double>(const cplx<double> *, int, cplx<double> *, int, int, int, int *, cudaStream_t);
template cudaError_t launch_rtrsyl<float>(const cplx<float> *, int, int, const cplx<float> *, int, int, cplx<float> *, int, int, int *, cudaStream_t);
template cudaError_t launch_rtrsyl<double>(const cplx<double> *, int, int, const cplx<double> *, int, int, cplx<double> *, int, int, int *, cudaStream_t);

}  // namespace sqm
