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
// QR: one CTA per matrix.  Each sweep chases the bulge down the active block
// [lo, hi] in windows of W rotations: the (W+3)^2 block around the diagonal
// is chased in shared memory by one warp; the window's rotations are then
// applied by the whole CTA to the rows to the right of the window, the
// columns above it and the Schur vectors.  Deflation when
// |h(k,k-1)| <= eps (|h(k,k)| + |h(k-1,k-1)|); an exceptional shift every
// 10 sweeps without deflation; at most kItMax sweeps per eigenvalue, then
// status 3.
#include "internal.h"

namespace sqm {

static constexpr int kHessThreads = 256;
static constexpr int kItMax = 60;

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
        for (int i = lane; i < m; i += 32) cfma(acc, conj(vsh[i]), c[i]);
        acc = warp_sum(acc);
        cplx<R> w = beta * acc;
        for (int i = lane; i < m; i += 32) cfms(c[i], vsh[i], w);
    }
}

// Rows of H (t < n) and of Q (t >= n); blockDim = (32, 8): x = row in tile,
// y = column segment.
template <class R>
__global__ void __launch_bounds__(kHessThreads)
hess_right_kernel(const SchurDesc<R> *__restrict__ descs, int k)
{
    extern __shared__ unsigned char smraw[];
    cplx<R> *vsh = reinterpret_cast<cplx<R> *>(smraw);
    __shared__ cplx<R> part[8][33];
    const SchurDesc<R> d = descs[blockIdx.y];
    const int n = d.n, ld = d.ld;
    if (k + 2 >= n) return;
    const int m = n - k - 1;
    const R beta = d.beta[0];
    const int tid = threadIdx.y * 32 + threadIdx.x;
    for (int i = tid; i < m; i += 256) vsh[i] = d.v[i];
    if (blockIdx.x == 0 && beta != R(0)) {
        // column k of H becomes [.., -phase ||x||, 0, ..., 0]
        cplx<R> *col = d.T + (k + 1) + (int64_t)k * ld;
        const R xn = d.beta[1];
        for (int i = tid; i < m; i += 256)
            col[i] = (i == 0) ? cplx<R>{-d.beta[2] * xn, -d.beta[3] * xn} : cplx<R>{0, 0};
    }
    __syncthreads();
    if (beta == R(0)) return;
    const int row0 = blockIdx.x * 32;
    if (row0 >= 2 * n) return;
    const int t = row0 + threadIdx.x;
    const bool valid = t < 2 * n;
    cplx<R> *M = (t < n) ? d.T : d.Q;
    const int i = (t < n) ? t : t - n;
    cplx<R> acc{0, 0};
    if (valid) {
        for (int l = threadIdx.y; l < m; l += 8) cfma(acc, M[i + (int64_t)(k + 1 + l) * ld], vsh[l]);
    }
    part[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    cplx<R> u{0, 0};
#pragma unroll
    for (int q = 0; q < 8; ++q) u += part[q][threadIdx.x];
    u = beta * u;
    if (valid) {
        for (int l = threadIdx.y; l < m; l += 8) {
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
        if ((err = cudaFuncSetAttribute(hess_left_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
            return err;
        if ((err = cudaFuncSetAttribute(hess_right_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
            return err;
    }
    eye_kernel<R><<<dim3(64, batch), 256, 0, s>>>(d_desc);
    for (int k = 0; k + 2 < nmax; ++k) {
        int m = nmax - k - 1;
        int left_ctas = (int)cdiv_i(m, kHessThreads / 32);
        if (left_ctas > ctas_per_matrix) left_ctas = ctas_per_matrix;
        hess_left_kernel<R><<<dim3(left_ctas, batch), kHessThreads, smem, s>>>(d_desc, k);
        int right_ctas = (int)cdiv_i(2 * nmax, 32);
        hess_right_kernel<R><<<dim3(right_ctas, batch), dim3(32, 8), smem, s>>>(d_desc, k);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// QR sweeps
// ---------------------------------------------------------------------------
static constexpr int kQrThreads = 256;
// rotations per window: 32 in FP32; 16 in FP64 so the per-thread rotation
// buffer (kW + 1 complex values) stays in registers
template <class R> struct QrWin { static constexpr int W = 32; };
template <> struct QrWin<double> { static constexpr int W = 16; };

// Complex Givens G = [c s; -conj(s) c] with c real and G [x; y] = [r; 0].
template <class R>
__device__ __forceinline__ void givens(cplx<R> x, cplx<R> y, R &c, cplx<R> &s, cplx<R> &r)
{
    R ax = hypot(x.x, x.y), ay = hypot(y.x, y.y);
    if (ay == R(0)) { c = 1; s = {0, 0}; r = x; return; }
    if (ax == R(0)) { c = 0; s = {y.x / ay, -y.y / ay}; r = {ay, 0}; return; }
    R nrm = hypot(ax, ay);
    cplx<R> ph{x.x / ax, x.y / ax};
    c = ax / nrm;
    cplx<R> cy = conj(y);
    s = cplx<R>{(ph.x * cy.x - ph.y * cy.y) / nrm, (ph.x * cy.y + ph.y * cy.x) / nrm};
    r = cplx<R>{ph.x * nrm, ph.y * nrm};
}

// Eigenvalue of [a b; c d] closer to d, written without cancellation:
// d + h -/+ disc = d - bc / (h +/- disc), h = (a - d)/2, disc = sqrt(h^2 + bc).
template <class R>
__device__ cplx<R> wilkinson(cplx<R> a, cplx<R> b, cplx<R> c, cplx<R> d)
{
    cplx<R> h = R(0.5) * (a - d);
    cplx<R> bc = b * c;
    cplx<R> disc = csqrt_(h * h + bc);
    cplx<R> p1 = h + disc, p2 = h - disc;
    bool ok1 = abs2(p1) > R(0), ok2 = abs2(p2) > R(0);
    cplx<R> m1 = ok1 ? d - cdiv(bc, p1) : d;
    cplx<R> m2 = ok2 ? d - cdiv(bc, p2) : d;
    ok1 = ok1 && isfinite(m1.x) && isfinite(m1.y);
    ok2 = ok2 && isfinite(m2.x) && isfinite(m2.y);
    if (ok1 && (!ok2 || abs2(m1 - d) <= abs2(m2 - d))) return m1;
    if (ok2) return m2;
    return d;
}

template <class R>
__global__ void __launch_bounds__(kQrThreads)
qr_sweeps_kernel(const SchurDesc<R> *__restrict__ descs)
{
    constexpr int kW = QrWin<R>::W;    // rotations per window
    constexpr int kBW = kW + 3;        // window block edge
    __shared__ cplx<R> blk[kBW * kBW];
    __shared__ R rc[kW];
    __shared__ cplx<R> rs[kW];
    __shared__ int s_lo, s_hi, s_iter, s_status, s_sweeps;
    __shared__ long long s_rots;
    __shared__ cplx<R> s_mu;

    const SchurDesc<R> d = descs[blockIdx.x];
    const int n = d.n, ld = d.ld;
    cplx<R> *T = d.T;
    cplx<R> *Z = d.Q;
    const int tid = threadIdx.x;
    const int nt = blockDim.x;
    const R eps = num<R>::eps;

    if (tid == 0) { s_hi = n - 1; s_iter = 0; s_status = 0; s_sweeps = 0; s_rots = 0; }
    __syncthreads();

    while (true) {
        const int hi = s_hi;
        if (hi <= 0) break;
        if (tid == 0) s_lo = 0;
        __syncthreads();
        // deflation scan: largest k in [1, hi] with a negligible subdiagonal
        for (int k = 1 + tid; k <= hi; k += nt) {
            cplx<R> sub = T[k + (int64_t)(k - 1) * ld];
            R as = hypot(sub.x, sub.y);
            cplx<R> a = T[k + (int64_t)k * ld], b = T[(k - 1) + (int64_t)(k - 1) * ld];
            R dsum = hypot(a.x, a.y) + hypot(b.x, b.y);
            if (as == R(0) || as <= eps * dsum) atomicMax(&s_lo, k);
        }
        __syncthreads();
        const int lo = s_lo;
        if (lo == hi) {
            if (tid == 0) {
                T[hi + (int64_t)(hi - 1) * ld] = cplx<R>{0, 0};
                s_hi = hi - 1;
                s_iter = 0;
            }
            __syncthreads();
            continue;
        }
        if (tid == 0) {
            if (lo > 0) T[lo + (int64_t)(lo - 1) * ld] = cplx<R>{0, 0};
            int it = ++s_iter;
            ++s_sweeps;
            s_rots += hi - lo;
            if (it > kItMax) s_status = 3;
            cplx<R> mu;
            if (it % 10 == 0) {
                cplx<R> sub = T[hi + (int64_t)(hi - 1) * ld];
                mu = T[hi + (int64_t)hi * ld];
                mu.x += R(0.75) * hypot(sub.x, sub.y);
            } else {
                mu = wilkinson(T[(hi - 1) + (int64_t)(hi - 1) * ld], T[(hi - 1) + (int64_t)hi * ld],
                               T[hi + (int64_t)(hi - 1) * ld], T[hi + (int64_t)hi * ld]);
            }
            s_mu = mu;
        }
        __syncthreads();
        if (s_status) break;
        const cplx<R> mu = s_mu;

        for (int k0 = lo; k0 < hi; k0 += kW) {
            const int k1 = min(k0 + kW, hi);   // rotations k0 .. k1-1
            const int nrot = k1 - k0;
            const int r0 = max(k0 - 1, lo);
            const int r1 = min(k1 + 1, hi);
            const int bw = r1 - r0 + 1;
            for (int e = tid; e < bw * bw; e += nt) {
                int a = e % bw, b = e / bw;
                blk[a + b * kBW] = T[(r0 + a) + (int64_t)(r0 + b) * ld];
            }
            __syncthreads();
            if (tid < 32) {
                const int lane = tid;
                for (int k = k0; k < k1; ++k) {
                    const int kk = k - r0;
                    cplx<R> x, y;
                    if (k == lo) {
                        x = blk[kk + kk * kBW] - mu;
                        y = blk[(kk + 1) + kk * kBW];
                    } else {
                        x = blk[kk + (kk - 1) * kBW];
                        y = blk[(kk + 1) + (kk - 1) * kBW];
                    }
                    R c; cplx<R> s, r;
                    givens(x, y, c, s, r);
                    __syncwarp();
                    // rows kk, kk+1 over block columns >= (k == lo ? kk : kk-1)
                    const int cstart = (k == lo) ? kk : kk - 1;
                    for (int b = cstart + lane; b < bw; b += 32) {
                        cplx<R> p = blk[kk + b * kBW], q = blk[(kk + 1) + b * kBW];
                        blk[kk + b * kBW] = c * p + s * q;
                        blk[(kk + 1) + b * kBW] = c * q - conj(s) * p;
                    }
                    __syncwarp();
                    if (lane == 0 && k > lo) {
                        blk[kk + (kk - 1) * kBW] = r;
                        blk[(kk + 1) + (kk - 1) * kBW] = cplx<R>{0, 0};
                    }
                    __syncwarp();
                    // columns kk, kk+1 over block rows 0 .. min(kk+2, bw-1)
                    const int rend = min(kk + 2, bw - 1);
                    for (int a = lane; a <= rend; a += 32) {
                        cplx<R> p = blk[a + kk * kBW], q = blk[a + (kk + 1) * kBW];
                        blk[a + kk * kBW] = c * p + conj(s) * q;
                        blk[a + (kk + 1) * kBW] = c * q - s * p;
                    }
                    if (lane == 0) { rc[k - k0] = c; rs[k - k0] = s; }
                    __syncwarp();
                }
            }
            __syncthreads();
            for (int e = tid; e < bw * bw; e += nt) {
                int a = e % bw, b = e / bw;
                T[(r0 + a) + (int64_t)(r0 + b) * ld] = blk[a + b * kBW];
            }
            // delayed updates: (a) rows k0..k1, columns r1+1 .. n-1;
            // (b) columns k0..k1, rows 0 .. r0-1; (c) Schur vectors, all rows
            const int na = n - (r1 + 1);
            const int nb = r0;
            const int total = (na > 0 ? na : 0) + nb + n;
            for (int t = tid; t < total; t += nt) {
                cplx<R> v[kW + 1];
                if (t < na) {
                    cplx<R> *col = T + k0 + (int64_t)(r1 + 1 + t) * ld;
#pragma unroll
                    for (int q = 0; q <= kW; ++q) if (q <= nrot) v[q] = col[q];
#pragma unroll
                    for (int q = 0; q < kW; ++q) {
                        if (q < nrot) {
                            R c = rc[q]; cplx<R> s = rs[q];
                            cplx<R> p = v[q], w = v[q + 1];
                            v[q] = c * p + s * w;
                            v[q + 1] = c * w - conj(s) * p;
                        }
                    }
#pragma unroll
                    for (int q = 0; q <= kW; ++q) if (q <= nrot) col[q] = v[q];
                } else {
                    int u = t - (na > 0 ? na : 0);
                    cplx<R> *base;
                    if (u < nb) base = T + u + (int64_t)k0 * ld;
                    else base = Z + (u - nb) + (int64_t)k0 * ld;
#pragma unroll
                    for (int q = 0; q <= kW; ++q) if (q <= nrot) v[q] = base[(int64_t)q * ld];
#pragma unroll
                    for (int q = 0; q < kW; ++q) {
                        if (q < nrot) {
                            R c = rc[q]; cplx<R> s = rs[q];
                            cplx<R> p = v[q], w = v[q + 1];
                            v[q] = c * p + conj(s) * w;
                            v[q + 1] = c * w - s * p;
                        }
                    }
#pragma unroll
                    for (int q = 0; q <= kW; ++q) if (q <= nrot) base[(int64_t)q * ld] = v[q];
                }
            }
            __syncthreads();
        }
    }
    __syncthreads();
    // the strictly lower triangle is zero in exact arithmetic
    for (int64_t t = tid; t < (int64_t)n * n; t += nt) {
        int i = (int)(t % n), j = (int)(t / n);
        if (i > j) T[i + (int64_t)j * ld] = cplx<R>{0, 0};
    }
    if (tid == 0) {
        *d.status = s_status;
        if (d.counters) {
            d.counters[0] = s_sweeps;
            d.counters[1] = (int)(s_rots & 0x7fffffff);
            d.counters[2] = (int)(s_rots >> 31);
        }
    }
}

template <class R>
cudaError_t launch_qr_sweeps(const SchurDesc<R> *d_desc, int batch, cudaStream_t s)
{
    qr_sweeps_kernel<R><<<batch, kQrThreads, 0, s>>>(d_desc);
    return cudaGetLastError();
}

template cudaError_t launch_hessenberg<float>(const SchurDesc<float> *, int, int, int, cudaStream_t);
template cudaError_t launch_hessenberg<double>(const SchurDesc<double> *, int, int, int, cudaStream_t);
template cudaError_t launch_qr_sweeps<float>(const SchurDesc<float> *, int, cudaStream_t);
template cudaError_t launch_qr_sweeps<double>(const SchurDesc<double> *, int, cudaStream_t);

}  // namespace sqm
