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

// ---------------------------------------------------------------------------
// Real Schur form A = Q T Q^T of a real matrix in one CTA (Remark 2.1):
// Householder Hessenberg reduction, then implicit double-shift (Francis)
// sweeps with 3x3 reflectors, the shift pair being the eigenvalues of the
// trailing 2x2 block of the active block (an exceptional pair every 10
// sweeps without deflation); a deflated 2x2 block with real eigenvalues is
// split by a rotation through an eigenvector.  Thread 0 takes the scalar
// decisions, all threads apply each reflector (rows: one thread per column;
// columns and Q: one thread per row).  Bounded: 60 sweeps per deflation,
// then status 3.  T (in: A_s, out: quasi-triangular) and Q (out) are n x n
// with ld n in global memory (the matrix of one call stays in L2).
// ---------------------------------------------------------------------------
static constexpr int kRsThreads = 1024;

template <class R>
__device__ __forceinline__ R block_sum_rs(R v, R *red)
{
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    R t = R(0);
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;  // valid in thread 0
}

// Householder vector of a 3- (or 2-) vector: P = I - beta v v^T, v0 = 1,
// P x = (||x||, 0, 0)
template <class R>
__device__ void house3_dev(int len, R x, R y, R z, R v[3], R &beta)
{
    const R sig = y * y + (len == 3 ? z * z : R(0));
    v[0] = R(1); v[1] = y; v[2] = len == 3 ? z : R(0);
    if (sig == R(0)) { beta = R(0); return; }
    const R mu = sqrt(x * x + sig);
    const R v0 = x <= R(0) ? x - mu : -sig / (x + mu);
    beta = R(2) * v0 * v0 / (sig + v0 * v0);
    v[1] = y / v0;
    v[2] = len == 3 ? z / v0 : R(0);
}

template <class R>
__global__ void __launch_bounds__(kRsThreads, 1)
real_schur_kernel(R *__restrict__ T, R *__restrict__ Q, int n, int *status, int *counters)
{
    extern __shared__ unsigned char smraw[];
    R *vb = reinterpret_cast<R *>(smraw);  // n: Householder vector of the reduction
    __shared__ R red[kRsThreads / 32];
    __shared__ R s_v[3], s_beta, s_cs, s_sn;
    __shared__ int s_act, s_k, s_lo, s_hi, s_len, s_c0, s_r1;
    const int tid = threadIdx.x, nt = blockDim.x;
    const R eps = num<R>::eps;
    for (int e = tid; e < n * n; e += nt) Q[e] = (e % n == e / n) ? R(1) : R(0);
    __syncthreads();
    // ---- Hessenberg reduction: column k, reflector on rows k+1 .. n-1 ----
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        R part = R(0);
        for (int i = tid; i < m; i += nt) {
            const R x = T[(k + 1 + i) + (int64_t)k * n];
            vb[i] = x;
            if (i > 0) part += x * x;
        }
        const R sig = block_sum_rs(part, red);
        if (tid == 0) {
            const R x0 = vb[0];
            R beta = R(0), v0 = R(1), r = x0;
            if (sig != R(0)) {
                const R mu = sqrt(x0 * x0 + sig);
                v0 = x0 <= R(0) ? x0 - mu : -sig / (x0 + mu);
                beta = R(2) * v0 * v0 / (sig + v0 * v0);
                r = mu;
            }
            s_beta = beta;
            s_v[0] = v0;
            s_v[1] = r;
        }
        __syncthreads();
        const R beta = s_beta, v0 = s_v[0];
        if (beta != R(0)) {
            for (int i = tid; i < m; i += nt) vb[i] = i == 0 ? R(1) : vb[i] / v0;
            __syncthreads();
            // left: columns k+1 .. n-1 (one warp per column), column k set exactly
            const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
            for (int j = k + 1 + warp; j < n; j += nw) {
                R d = R(0);
                for (int i = lane; i < m; i += 32) d += vb[i] * T[(k + 1 + i) + (int64_t)j * n];
                d = warp_sum(d) * beta;
                for (int i = lane; i < m; i += 32) T[(k + 1 + i) + (int64_t)j * n] -= d * vb[i];
            }
            for (int i = tid; i < m; i += nt) T[(k + 1 + i) + (int64_t)k * n] = i == 0 ? s_v[1] : R(0);
            __syncthreads();
            // right: rows 0 .. n-1 of T and Q, columns k+1 .. n-1
            for (int i = tid; i < n; i += nt) {
                R u = R(0), w = R(0);
                for (int l = 0; l < m; ++l) {
                    u += T[i + (int64_t)(k + 1 + l) * n] * vb[l];
                    w += Q[i + (int64_t)(k + 1 + l) * n] * vb[l];
                }
                u *= beta;
                w *= beta;
                for (int l = 0; l < m; ++l) {
                    T[i + (int64_t)(k + 1 + l) * n] -= u * vb[l];
                    Q[i + (int64_t)(k + 1 + l) * n] -= w * vb[l];
                }
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < n * n; e += nt)
        if (e % n > e / n + 1) T[e] = R(0);
    __syncthreads();
    // ---- double-shift sweeps ----
    int hi = n - 1, iter = 0, total = 0, sweeps = 0;  // thread 0's copies
    for (;;) {
        // thread 0: deflate, then choose: 0 sweep, 1 split at s_k, 2 done, 3 failed
        if (tid == 0) {
            s_act = 2;
            while (hi >= 0) {
                int lo = hi;
                while (lo > 0) {
                    const R sub = fabs(T[lo + (int64_t)(lo - 1) * n]);
                    const R dsum = fabs(T[lo + (int64_t)lo * n]) + fabs(T[(lo - 1) + (int64_t)(lo - 1) * n]);
                    if (sub <= eps * dsum || sub == R(0)) {
                        T[lo + (int64_t)(lo - 1) * n] = R(0);
                        break;
                    }
                    --lo;
                }
                if (lo == hi) { --hi; iter = 0; continue; }
                if (lo == hi - 1) {
                    const int k = hi - 1;
                    const R a = T[k + (int64_t)k * n], b = T[k + (int64_t)(k + 1) * n];
                    const R c = T[(k + 1) + (int64_t)k * n], d = T[(k + 1) + (int64_t)(k + 1) * n];
                    const R p = R(0.5) * (a - d), disc = p * p + b * c;
                    hi -= 2;
                    iter = 0;
                    if (disc < R(0)) continue;  // a conjugate pair: a 2x2 block stays
                    const R lam = R(0.5) * (a + d) + (p >= R(0) ? sqrt(disc) : -sqrt(disc));
                    const R e0 = lam - d, nr = hypot(e0, c);
                    s_cs = e0 / nr;
                    s_sn = c / nr;
                    s_k = k;
                    s_act = 1;
                    break;
                }
                if (++iter > 60 || ++total > 60 * n + 60) { s_act = 3; break; }
                ++sweeps;
                R sft, tft;
                const R h11 = T[(hi - 1) + (int64_t)(hi - 1) * n], h12 = T[(hi - 1) + (int64_t)hi * n];
                const R h21 = T[hi + (int64_t)(hi - 1) * n], h22 = T[hi + (int64_t)hi * n];
                if (iter % 10 == 0) {
                    const R w = fabs(h21) + fabs(T[(hi - 1) + (int64_t)(hi - 2) * n]);
                    sft = R(1.5) * w + h22;
                    tft = w * w;
                } else {
                    sft = h11 + h22;
                    tft = h11 * h22 - h12 * h21;
                }
                const R a00 = T[lo + (int64_t)lo * n], a01 = T[lo + (int64_t)(lo + 1) * n];
                const R a10 = T[(lo + 1) + (int64_t)lo * n], a11 = T[(lo + 1) + (int64_t)(lo + 1) * n];
                s_v[0] = a00 * a00 + a01 * a10 - sft * a00 + tft;  // first column of (H - s1)(H - s2)
                s_v[1] = a10 * (a00 + a11 - sft);
                s_v[2] = a10 * T[(lo + 2) + (int64_t)(lo + 1) * n];
                s_lo = lo;
                s_hi = hi;
                s_act = 0;
                break;
            }
        }
        __syncthreads();
        const int act = s_act;
        if (act >= 2) {
            if (act == 3 && tid == 0) atomicExch(status, 3);
            break;
        }
        if (act == 1) {  // rotation G = [cs -sn; sn cs] on rows / columns k, k+1
            const int k = s_k;
            const R cs = s_cs, sn = s_sn;
            for (int j = k + tid; j < n; j += nt) {
                const R x = T[k + (int64_t)j * n], y = T[(k + 1) + (int64_t)j * n];
                T[k + (int64_t)j * n] = cs * x + sn * y;
                T[(k + 1) + (int64_t)j * n] = -sn * x + cs * y;
            }
            __syncthreads();
            for (int i = tid; i < n; i += nt) {
                if (i <= k + 1) {
                    const R x = T[i + (int64_t)k * n], y = T[i + (int64_t)(k + 1) * n];
                    T[i + (int64_t)k * n] = cs * x + sn * y;
                    T[i + (int64_t)(k + 1) * n] = -sn * x + cs * y;
                }
                const R x = Q[i + (int64_t)k * n], y = Q[i + (int64_t)(k + 1) * n];
                Q[i + (int64_t)k * n] = cs * x + sn * y;
                Q[i + (int64_t)(k + 1) * n] = -sn * x + cs * y;
            }
            __syncthreads();
            if (tid == 0) T[(k + 1) + (int64_t)k * n] = R(0);
            continue;
        }
        // a sweep over [lo, hi]: steps k = lo .. hi-2 with 3x3 reflectors, then a 2x2 one
        const int lo = s_lo, hs = s_hi;
        for (int k = lo; k <= hs - 1; ++k) {
            if (tid == 0) {
                R x, y, z;
                if (k == lo) {
                    x = s_v[0]; y = s_v[1]; z = s_v[2];
                } else {
                    x = T[k + (int64_t)(k - 1) * n];
                    y = T[(k + 1) + (int64_t)(k - 1) * n];
                    z = k + 2 <= hs ? T[(k + 2) + (int64_t)(k - 1) * n] : R(0);
                }
                const int len = k + 2 <= hs ? 3 : 2;
                R v[3], beta;
                house3_dev<R>(len, x, y, z, v, beta);
                s_v[0] = v[0]; s_v[1] = v[1]; s_v[2] = v[2];
                s_beta = beta;
                s_len = len;
                s_c0 = k > lo ? k - 1 : lo;
                s_r1 = min(k + len + 1, hs + 1);  // rows 0 .. r1-1 of the right application
            }
            __syncthreads();
            const R beta = s_beta, v0 = s_v[0], v1 = s_v[1], v2 = s_v[2];
            const int len = s_len, c0 = s_c0, r1 = s_r1;
            if (beta != R(0)) {
                for (int j = c0 + tid; j < n; j += nt) {
                    const R t0 = T[k + (int64_t)j * n], t1 = T[(k + 1) + (int64_t)j * n];
                    const R t2 = len == 3 ? T[(k + 2) + (int64_t)j * n] : R(0);
                    const R d = beta * (v0 * t0 + v1 * t1 + v2 * t2);
                    T[k + (int64_t)j * n] = t0 - d * v0;
                    T[(k + 1) + (int64_t)j * n] = t1 - d * v1;
                    if (len == 3) T[(k + 2) + (int64_t)j * n] = t2 - d * v2;
                }
                __syncthreads();
                for (int i = tid; i < n; i += nt) {
                    if (i < r1) {
                        const R t0 = T[i + (int64_t)k * n], t1 = T[i + (int64_t)(k + 1) * n];
                        const R t2 = len == 3 ? T[i + (int64_t)(k + 2) * n] : R(0);
                        const R d = beta * (t0 * v0 + t1 * v1 + t2 * v2);
                        T[i + (int64_t)k * n] = t0 - d * v0;
                        T[i + (int64_t)(k + 1) * n] = t1 - d * v1;
                        if (len == 3) T[i + (int64_t)(k + 2) * n] = t2 - d * v2;
                    }
                    const R q0 = Q[i + (int64_t)k * n], q1 = Q[i + (int64_t)(k + 1) * n];
                    const R q2 = len == 3 ? Q[i + (int64_t)(k + 2) * n] : R(0);
                    const R d = beta * (q0 * v0 + q1 * v1 + q2 * v2);
                    Q[i + (int64_t)k * n] = q0 - d * v0;
                    Q[i + (int64_t)(k + 1) * n] = q1 - d * v1;
                    if (len == 3) Q[i + (int64_t)(k + 2) * n] = q2 - d * v2;
                }
            }
            __syncthreads();
            if (tid == 0 && k > lo) {  // the bulge below the subdiagonal is gone
                T[(k + 1) + (int64_t)(k - 1) * n] = R(0);
                if (len == 3) T[(k + 2) + (int64_t)(k - 1) * n] = R(0);
            }
            __syncthreads();
        }
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += nt)
        if (e % n > e / n + 1) T[e] = R(0);
    if (tid == 0 && counters) counters[0] = sweeps;
}

template <class R>
cudaError_t launch_real_schur(R *T, R *Q, int n, int *d_status, int *d_counters, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const size_t smem = (size_t)(n + 8) * sizeof(R);
    cudaError_t err;
    if (smem > 48 * 1024 && (err = allow_max_smem((const void *)real_schur_kernel<R>))) return err;
    real_schur_kernel<R><<<1, kRsThreads, smem, s>>>(T, Q, n, d_status, d_counters); count_launch();
    return cudaGetLastError();
}

template cudaError_t launch_real_schur<float>(float *, float *, int, int *, int *, cudaStream_t);
template cudaError_t launch_real_schur<double>(double *, double *, int, int *, int *, cudaStream_t);

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
