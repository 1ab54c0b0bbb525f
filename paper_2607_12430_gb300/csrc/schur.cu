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
// Real input (every matrix the library factors) of moderate size instead
// takes hess_cluster_kernel: the whole reduction and the accumulation of Q
// in one launch of a thread-block cluster that keeps the matrix in its
// shared memory.
//
// The QR sweeps that follow the reduction are in qr.cu.
#include <cooperative_groups.h>

#include <atomic>

#include "internal.h"
#include "spd_internal.h"

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

// ---------------------------------------------------------------------------
// Real Householder Hessenberg reduction held in the shared memory of one
// thread-block cluster of CL <= 8 CTAs; CTA c keeps the columns j = c (mod
// CL) (the active columns stay spread evenly as k grows).  For column k the
// owning CTA forms P_k = I - beta v v^T from x = H(k+1:n, k) with
// v = x + sign(x_0) ||x|| e_1, beta = 2 / ||v||^2 (beta = 0 when the tail of
// x is zero) and stores v in column k of V.  P_k H changes each column on
// its own, so every CTA applies it to its columns; H P_k needs
// u = H(:, k+1:n) v, whose per-CTA parts are summed through distributed
// shared memory.  Two cluster barriers per column.  Then Q = P_0 P_1 ...
// P_{n-3} by backward accumulation (Q <- P_k Q for k = n-3 .. 0, which
// changes only columns > k), again column by column in the same shared
// memory.  H and Q are written back as complex matrices with zero
// imaginary parts.  No CTA waits on anything but the cluster's hardware
// barriers, which every CTA reaches the same number of times.
// ---------------------------------------------------------------------------
namespace cg = cooperative_groups;

static constexpr int kHessClThreads = 512;
static constexpr int kHessClMax = 8;

template <class R>
__global__ void __launch_bounds__(kHessClThreads, 1)
hess_cluster_kernel(cplx<R> *__restrict__ T, cplx<R> *__restrict__ Q, int n, int ld, R *__restrict__ Vg,
                    R *__restrict__ betas)
{
    cg::cluster_group cl = cg::this_cluster();
    const int CL = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nt = kHessClThreads, nw = kHessClThreads / 32;
    const int ncmax = (n + CL - 1) / CL;
    const int ncl = rank < n ? (n - rank + CL - 1) / CL : 0;  // columns rank, rank + CL, ...
    extern __shared__ __align__(16) unsigned char smraw[];
    R *Hs = reinterpret_cast<R *>(smraw);  // Hs[i + jl n] = column rank + jl CL
    R *vbuf = Hs + (size_t)n * ncmax;      // reflector of a column this CTA owns
    R *pbuf = vbuf + n;                    // this CTA's part of u
    R *vloc = pbuf + n;                    // the current reflector
    __shared__ R s_scal[2];                // beta, new subdiagonal entry
    __shared__ R s_red[2][nw];
    auto first_col = [&](int k) {  // first local column with global index > k
        const int d0 = k + 1 - rank;
        return d0 > 0 ? (d0 + CL - 1) / CL : 0;
    };
    auto gcol = [&](int jl) { return rank + jl * CL; };

    for (int e = tid; e < n * ncl; e += nt) {
        const int i = e % n, jl = e / n;
        Hs[i + (size_t)jl * n] = T[i + (int64_t)gcol(jl) * ld].x;
    }
    __syncthreads();
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1, o = k % CL;
        if (rank == o) {
            R *col = Hs + (size_t)(k / CL) * n + (k + 1);
            R a = 0, t = 0;
            for (int i = tid; i < m; i += nt) {
                const R x = col[i];
                a = fma(x, x, a);
                if (i > 0) t = fma(x, x, t);
            }
            a = warp_sum(a);
            t = warp_sum(t);
            if (lane == 0) { s_red[0][warp] = a; s_red[1][warp] = t; }
            __syncthreads();
            if (tid == 0) {
                R xn2 = 0, tail2 = 0;
                for (int q = 0; q < nw; ++q) { xn2 += s_red[0][q]; tail2 += s_red[1][q]; }
                const R x0 = col[0];
                if (tail2 == R(0)) {
                    s_scal[0] = 0;
                    s_scal[1] = x0;
                } else {
                    const R xn = sqrt(xn2), sg = x0 < R(0) ? R(-1) : R(1);
                    const R v0 = x0 + sg * xn;
                    s_scal[0] = R(2) / (v0 * v0 + tail2);
                    s_scal[1] = -sg * xn;
                    vbuf[0] = v0;
                }
            }
            for (int i = 1 + tid; i < m; i += nt) vbuf[i] = col[i];
            __syncthreads();
            const R beta = s_scal[0];
            if (tid == 0) betas[k] = beta;
            for (int i = tid; i < m; i += nt) Vg[(k + 1 + i) + (int64_t)k * n] = beta != R(0) ? vbuf[i] : R(0);
            if (beta != R(0))
                for (int i = tid; i < m; i += nt) col[i] = (i == 0) ? s_scal[1] : R(0);
        }
        cl.sync();
        const R beta = *cl.map_shared_rank(&s_scal[0], o);  // the same in every CTA
        const int jl0 = first_col(k);
        if (beta != R(0)) {
            const R *rv = cl.map_shared_rank(vbuf, o);
            for (int i = tid; i < m; i += nt) vloc[i] = rv[i];
            __syncthreads();
            // P_k H on this CTA's columns > k (rows k+1 .. n-1)
            for (int jl = jl0 + warp; jl < ncl; jl += nw) {
                R *c = Hs + (size_t)jl * n + (k + 1);
                R acc = 0;
                for (int i = lane; i < m; i += 32) acc = fma(vloc[i], c[i], acc);
                acc = warp_sum(acc) * beta;
                for (int i = lane; i < m; i += 32) c[i] = fma(-acc, vloc[i], c[i]);
            }
            __syncthreads();
            // this CTA's part of u = H(:, k+1:n) v
            for (int i = tid; i < n; i += nt) {
                R acc0 = 0, acc1 = 0;
                int jl = jl0;
                for (; jl + 1 < ncl; jl += 2) {
                    acc0 = fma(Hs[i + (size_t)jl * n], vloc[gcol(jl) - k - 1], acc0);
                    acc1 = fma(Hs[i + (size_t)(jl + 1) * n], vloc[gcol(jl + 1) - k - 1], acc1);
                }
                if (jl < ncl) acc0 = fma(Hs[i + (size_t)jl * n], vloc[gcol(jl) - k - 1], acc0);
                pbuf[i] = acc0 + acc1;
            }
        }
        cl.sync();
        if (beta != R(0)) {
            // H P_k: every CTA sums the parts in the same order
            for (int i = tid; i < n; i += nt) {
                R u = 0;
                for (int c = 0; c < CL; ++c) u += cl.map_shared_rank(pbuf, c)[i];
                u *= beta;
                for (int jl = jl0; jl < ncl; ++jl)
                    Hs[i + (size_t)jl * n] = fma(-u, vloc[gcol(jl) - k - 1], Hs[i + (size_t)jl * n]);
            }
        }
        __syncthreads();
    }
    __threadfence();  // V and beta (global) before the other CTAs read them for Q
    cl.sync();        // and no CTA reads another's shared memory after this point
    for (int e = tid; e < n * ncl; e += nt) {
        const int i = e % n, jl = e / n;
        T[i + (int64_t)gcol(jl) * ld] = cplx<R>{Hs[i + (size_t)jl * n], R(0)};
    }
    __syncthreads();
    for (int e = tid; e < n * ncl; e += nt) {
        const int i = e % n, jl = e / n;
        Hs[i + (size_t)jl * n] = (R)(i == gcol(jl));
    }
    __syncthreads();
    for (int k = n - 3; k >= 0; --k) {
        const R beta = __ldcg(betas + k);
        if (beta == R(0)) continue;
        const int m = n - k - 1, jl0 = first_col(k);
        for (int i = tid; i < m; i += nt) vloc[i] = __ldcg(Vg + (k + 1 + i) + (int64_t)k * n);
        __syncthreads();
        for (int jl = jl0 + warp; jl < ncl; jl += nw) {
            R *c = Hs + (size_t)jl * n + (k + 1);
            R acc = 0;
            for (int i = lane; i < m; i += 32) acc = fma(vloc[i], c[i], acc);
            acc = warp_sum(acc) * beta;
            for (int i = lane; i < m; i += 32) c[i] = fma(-acc, vloc[i], c[i]);
        }
        __syncthreads();
    }
    for (int e = tid; e < n * ncl; e += nt) {
        const int i = e % n, jl = e / n;
        Q[i + (int64_t)gcol(jl) * ld] = cplx<R>{Hs[i + (size_t)jl * n], R(0)};
    }
}

// The same reduction with the CTA's columns in registers (n <= 32 RPL <= 512,
// at most 64 columns per CTA): lane l of warp w holds rows l + 32 q
// (q < RPL) of the local columns w + 16 c (c < 4).  The owner of column k is
// one warp, which forms the reflector with shuffles alone; the left
// reflection is a warp dot product per column; the right one needs the
// partial sums over the CTA's columns, reduced across the 16 warps in shared
// memory and across the cluster through distributed shared memory.  Two
// cluster barriers per column, as above, and the backward accumulation of Q
// in the same registers.
template <class R, int RPL>
__global__ void __launch_bounds__(kHessClThreads, 1)
hess_cluster_reg_kernel(cplx<R> *__restrict__ T, cplx<R> *__restrict__ Q, int n, int ld, R *__restrict__ Vg,
                        R *__restrict__ betas, const HessJob<R> *__restrict__ jobs)
{
    constexpr int NW = kHessClThreads / 32, CPW = 4, PLD = 32 * RPL + 1;
    cg::cluster_group cl = cg::this_cluster();
    const int CL = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    if (jobs) {  // batched: cluster c of the grid reduces matrix c
        const HessJob<R> jb = jobs[blockIdx.x / CL];
        T = jb.T; Q = jb.Q; Vg = jb.V; betas = jb.betas;
        n = ld = jb.n;
    }
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ncl = rank < n ? (n - rank + CL - 1) / CL : 0;
    extern __shared__ __align__(16) unsigned char smraw[];
    R *vbuf = reinterpret_cast<R *>(smraw);  // reflector of a column this CTA owns (32 RPL)
    R *pbuf = vbuf + 32 * RPL;               // this CTA's part of u
    R *ubuf = pbuf + 32 * RPL;               // u
    R *vloc = ubuf + 32 * RPL;               // the current reflector
    R *part = vloc + 32 * RPL;               // per-warp partial sums, NW x PLD
    __shared__ R s_scal[2];
    auto gcol = [&](int jl) { return rank + jl * CL; };
    R h[CPW][RPL];
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
        const int jl = warp + NW * c;
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int i = lane + 32 * q;
            h[c][q] = (jl < ncl && i < n) ? T[i + (int64_t)gcol(jl) * ld].x : R(0);
        }
    }
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1, o = k % CL, jlk = k / CL;
        if (rank == o && warp == jlk % NW) {
            const int ck = jlk / NW;  // which of this warp's columns
            auto colk = [&](int q) {  // row lane + 32 q of column k
                R v = h[0][q];
#pragma unroll
                for (int c = 1; c < CPW; ++c) v = (ck == c) ? h[c][q] : v;
                return v;
            };
            R a = 0, t = 0, x0 = 0;
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                const int i = lane + 32 * q;
                const R xq = colk(q);
                if (i >= k + 1) a = fma(xq, xq, a);
                if (i >= k + 2) t = fma(xq, xq, t);
                if (i == k + 1) x0 = xq;
            }
            a = warp_sum(a);
            t = warp_sum(t);
            x0 = __shfl_sync(0xffffffffu, x0, (k + 1) & 31);
            R beta = 0, diag = x0, v0 = 0;
            if (t != R(0)) {
                const R xn = sqrt(a), sg = x0 < R(0) ? R(-1) : R(1);
                v0 = x0 + sg * xn;
                beta = R(2) / (v0 * v0 + t);
                diag = -sg * xn;
            }
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                const int i = lane + 32 * q;
                if (i >= k + 1 && i < n) {
                    const R vi = (i == k + 1) ? v0 : colk(q);
                    vbuf[i - k - 1] = vi;
                    Vg[i + (int64_t)k * n] = beta != R(0) ? vi : R(0);
                    if (beta != R(0)) {
                        const R nv = (i == k + 1) ? diag : R(0);
#pragma unroll
                        for (int c = 0; c < CPW; ++c)
                            if (ck == c) h[c][q] = nv;
                    }
                }
            }
            if (lane == 0) {
                s_scal[0] = beta;
                betas[k] = beta;
            }
        }
        cl.sync();
        const R beta = *cl.map_shared_rank(&s_scal[0], o);  // the same in every CTA
        R vc[CPW];
        if (beta != R(0)) {
            const R *rv = cl.map_shared_rank(vbuf, o);
            for (int i = tid; i < m; i += kHessClThreads) vloc[i] = rv[i];
            __syncthreads();
            R vr[RPL];
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                const int i = lane + 32 * q;
                vr[q] = (i >= k + 1 && i < n) ? vloc[i - k - 1] : R(0);
            }
#pragma unroll
            for (int c = 0; c < CPW; ++c) {
                const int jl = warp + NW * c;
                const bool act = jl < ncl && gcol(jl) > k;  // uniform per warp
                vc[c] = act ? vloc[gcol(jl) - k - 1] : R(0);
                if (act) {
                    // P_k H: w = beta v^T h, h -= w v
                    R d = 0;
#pragma unroll
                    for (int q = 0; q < RPL; ++q) d = fma(vr[q], h[c][q], d);
                    d = warp_sum(d) * beta;
#pragma unroll
                    for (int q = 0; q < RPL; ++q) h[c][q] = fma(-d, vr[q], h[c][q]);
                }
            }
            // this warp's part of u = H(:, k+1:n) v over its columns
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                R pq = 0;
#pragma unroll
                for (int c = 0; c < CPW; ++c) pq = fma(h[c][q], vc[c], pq);
                part[warp * PLD + lane + 32 * q] = pq;
            }
            __syncthreads();
            for (int i = tid; i < n; i += kHessClThreads) {
                R sum = 0;
#pragma unroll
                for (int w2 = 0; w2 < NW; ++w2) sum += part[w2 * PLD + i];
                pbuf[i] = sum;
            }
        }
        cl.sync();
        if (beta != R(0)) {
            // H P_k: every CTA sums the parts in the same order
            for (int i = tid; i < n; i += kHessClThreads) {
                R u = 0;
                for (int c = 0; c < CL; ++c) u += cl.map_shared_rank(pbuf, c)[i];
                ubuf[i] = u * beta;
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                const int i = lane + 32 * q;
                const R uq = i < n ? ubuf[i] : R(0);
#pragma unroll
                for (int c = 0; c < CPW; ++c) h[c][q] = fma(-uq, vc[c], h[c][q]);
            }
        }
        __syncthreads();
    }
    __threadfence();  // V and beta (global) before the other CTAs read them for Q
    cl.sync();        // and no CTA reads another's shared memory after this point
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
        const int jl = warp + NW * c;
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int i = lane + 32 * q;
            if (jl < ncl && i < n) T[i + (int64_t)gcol(jl) * ld] = cplx<R>{h[c][q], R(0)};
            h[c][q] = (R)(i == gcol(jl));
        }
    }
    // Q = P_0 ... P_{n-3}: Q <- P_k Q for k = n-3 .. 0
    for (int k = n - 3; k >= 0; --k) {
        const R beta = __ldcg(betas + k);
        if (beta == R(0)) continue;
        const int m = n - k - 1;
        for (int i = tid; i < m; i += kHessClThreads) vloc[i] = __ldcg(Vg + (k + 1 + i) + (int64_t)k * n);
        __syncthreads();
        R vr[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int i = lane + 32 * q;
            vr[q] = (i >= k + 1 && i < n) ? vloc[i - k - 1] : R(0);
        }
#pragma unroll
        for (int c = 0; c < CPW; ++c) {
            const int jl = warp + NW * c;
            if (jl < ncl && gcol(jl) > k) {
                R d = 0;
#pragma unroll
                for (int q = 0; q < RPL; ++q) d = fma(vr[q], h[c][q], d);
                d = warp_sum(d) * beta;
#pragma unroll
                for (int q = 0; q < RPL; ++q) h[c][q] = fma(-d, vr[q], h[c][q]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
        const int jl = warp + NW * c;
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int i = lane + 32 * q;
            if (jl < ncl && i < n) Q[i + (int64_t)gcol(jl) * ld] = cplx<R>{h[c][q], R(0)};
        }
    }
}

template <class R, int RPL>
static constexpr size_t hess_reg_smem()
{
    return ((size_t)4 * 32 * RPL + (size_t)(kHessClThreads / 32) * (32 * RPL + 1)) * sizeof(R);
}

static constexpr size_t kHessClSmemMax = 232448 - 1024;  // 227 KB opt-in per CTA, less the static arrays

template <class R>
static size_t hess_cluster_smem(int n, int CL)
{
    const size_t ncmax = (size_t)((n + CL - 1) / CL);
    return ((size_t)n * ncmax + 3 * (size_t)n) * sizeof(R);
}

// can a cluster of CL CTAs of `kernel` with `smem` bytes each be resident?
static bool cluster_resident(const void *kernel, int CL, size_t smem)
{
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(kHessClThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    const bool ok = cudaOccupancyMaxActiveClusters(&nclusters, kernel, &cfg) == cudaSuccess && nclusters > 0;
    cudaGetLastError();
    return ok;
}

// rows per lane of the register-resident kernel for n (0: not used; FP64
// keeps at most 4 rows per lane in registers)
template <class R>
static int hess_reg_rpl(int n)
{
    const int r = n <= 64 ? 2 : n <= 128 ? 4 : n <= 256 ? 8 : n <= 512 ? 16 : 0;
    return (sizeof(R) == sizeof(double) && r > 4) ? 0 : r;
}

template <class R>
static const void *hess_reg_fn(int rpl)
{
    switch (rpl) {
    case 2: return (const void *)hess_cluster_reg_kernel<R, 2>;
    case 4: return (const void *)hess_cluster_reg_kernel<R, 4>;
    case 8: return (const void *)hess_cluster_reg_kernel<R, sizeof(R) == sizeof(double) ? 4 : 8>;
    default: return (const void *)hess_cluster_reg_kernel<R, sizeof(R) == sizeof(double) ? 4 : 16>;
    }
}

// cluster size for an n x n matrix: the smallest that leaves at most 64
// columns per CTA (register-resident kernel up to n = 512), else the largest
// shared-memory layout that fits; 0 = too large (or no such cluster can be
// resident), use launch_hessenberg
template <class R>
int hess_cluster_size(int n)
{
    if (n < 3) return 0;
    // per kernel kind (0 = registers, 1 = shared memory) and CL: 0 unknown, 1 yes, -1 no
    static std::atomic<int> resident[2][kHessClMax + 1];
    const int rpl = hess_reg_rpl<R>(n);
    int pick = 0, kind = 0;
    if (rpl) {
        for (int CL = 1; CL <= kHessClMax; CL *= 2)
            if ((n + CL - 1) / CL <= 64) { pick = CL; break; }
    } else {
        kind = 1;
        for (int CL = 1; CL <= kHessClMax; CL *= 2) {
            if (hess_cluster_smem<R>(n, CL) > kHessClSmemMax) continue;
            pick = CL;
            if ((n + CL - 1) / CL <= 64) break;
        }
    }
    if (!pick) return 0;
    if (resident[kind][pick].load() == 0) {
        const bool ok = kind == 0 ? cluster_resident(hess_reg_fn<R>(rpl), pick, hess_reg_smem<R, 16>())
                                  : cluster_resident((const void *)hess_cluster_kernel<R>, pick, kHessClSmemMax);
        resident[kind][pick].store(ok ? 1 : -1);
    }
    return resident[kind][pick].load() > 0 ? pick : 0;
}

template <class R, int RPL>
static cudaError_t launch_hess_reg(cplx<R> *T, cplx<R> *Q, int n, int ld, R *V, R *betas, int CL, cudaStream_t s)
{
    constexpr size_t smem = hess_reg_smem<R, RPL>();
    cudaError_t err = cudaFuncSetAttribute((const void *)hess_cluster_reg_kernel<R, RPL>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err) return err;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(kHessClThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    err = cudaLaunchKernelEx(&cfg, hess_cluster_reg_kernel<R, RPL>, T, Q, n, ld, V, betas,
                             (const HessJob<R> *)nullptr);
    count_launch();
    return err;
}

template <class R, int RPL>
static cudaError_t launch_hess_reg_batched(const HessJob<R> *jobs, int count, int CL, cudaStream_t s)
{
    constexpr size_t smem = hess_reg_smem<R, RPL>();
    cudaError_t err = cudaFuncSetAttribute((const void *)hess_cluster_reg_kernel<R, RPL>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err) return err;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(CL * count);
    cfg.blockDim = dim3(kHessClThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    err = cudaLaunchKernelEx(&cfg, hess_cluster_reg_kernel<R, RPL>, (cplx<R> *)nullptr, (cplx<R> *)nullptr, 0, 0,
                             (R *)nullptr, (R *)nullptr, jobs);
    count_launch();
    return err;
}

template <class R>
cudaError_t launch_hessenberg_cluster_batched(const HessJob<R> *jobs, int count, int nmax, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    const int rpl = hess_reg_rpl<R>(std::max(nmax, 3));
    if (!rpl || hess_cluster_size<R>(std::max(nmax, 3)) == 0) return cudaErrorNotSupported;
    int CL = 1;
    while ((std::max(nmax, 3) + CL - 1) / CL > 64) CL *= 2;
    switch (rpl) {
    case 2: return launch_hess_reg_batched<R, 2>(jobs, count, CL, s);
    case 4: return launch_hess_reg_batched<R, 4>(jobs, count, CL, s);
    case 8: return launch_hess_reg_batched<R, sizeof(R) == sizeof(double) ? 4 : 8>(jobs, count, CL, s);
    default: return launch_hess_reg_batched<R, sizeof(R) == sizeof(double) ? 4 : 16>(jobs, count, CL, s);
    }
}

template cudaError_t launch_hessenberg_cluster_batched<float>(const HessJob<float> *, int, int, cudaStream_t);
template cudaError_t launch_hessenberg_cluster_batched<double>(const HessJob<double> *, int, int, cudaStream_t);

template <class R>
cudaError_t launch_hessenberg_cluster(cplx<R> *T, cplx<R> *Q, int n, int ld, R *V, R *betas, cudaStream_t s)
{
    const int CL = hess_cluster_size<R>(n);
    if (!CL) return cudaErrorNotSupported;
    switch (hess_reg_rpl<R>(n)) {
    case 2: return launch_hess_reg<R, 2>(T, Q, n, ld, V, betas, CL, s);
    case 4: return launch_hess_reg<R, 4>(T, Q, n, ld, V, betas, CL, s);
    case 8: return launch_hess_reg<R, sizeof(R) == sizeof(double) ? 4 : 8>(T, Q, n, ld, V, betas, CL, s);
    case 16: return launch_hess_reg<R, sizeof(R) == sizeof(double) ? 4 : 16>(T, Q, n, ld, V, betas, CL, s);
    default: break;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(kHessClThreads);
    cfg.dynamicSmemBytes = hess_cluster_smem<R>(n, CL);
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t err = cudaLaunchKernelEx(&cfg, hess_cluster_kernel<R>, T, Q, n, ld, V, betas);
    count_launch();
    return err;
}

template int hess_cluster_size<float>(int);
template int hess_cluster_size<double>(int);
template cudaError_t launch_hessenberg_cluster<float>(cplx<float> *, cplx<float> *, int, int, float *, float *,
                                                      cudaStream_t);
template cudaError_t launch_hessenberg_cluster<double>(cplx<double> *, cplx<double> *, int, int, double *, double *,
                                                       cudaStream_t);

// ---------------------------------------------------------------------------
// Real Householder Hessenberg reduction of a real matrix beyond the cluster
// kernel's sizes: H (n x n, ld, real) <- Q^T H Q with Q = P_0 ... P_{n-3},
// P_k = I - beta_k v_k v_k^T acting on rows / columns k+1 .. n-1.  Three
// launches per column, each spread over the whole GPU:
//   hessr_left:  every CTA forms v_k from column k (which no launch of this
//                column writes), CTA 0 stores v_k into column k of Y (rows
//                k+1..) and beta_k; each warp applies P_k to one column
//                j > k of the trailing rows (w_j = beta v^T H(k+1:, j),
//                H(k+1:, j) -= v w_j);
//   hessr_rpart: partial products u_s = H(:, seg_s) v over S column segments
//                (a thread per row);
//   hessr_rupd:  u = beta sum_s u_s in segment order, H(:, seg_s) -= u v^T,
//                and column k becomes (.., -sign(x_0) ||x||, 0, ..).
// Q is not updated column by column: it is formed at the end from the
// stored reflectors by the blocked compact-WY back-transform (GEMMs).
// ---------------------------------------------------------------------------
static constexpr int kHrThreads = 256;

template <class R>
__device__ void real_reflector(const R *__restrict__ col, int m, R *vsh, R *s_scal /* [beta, alpha] */)
{
    __shared__ R red[2][kHrThreads / 32];
    R t_all = 0, t_tail = 0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const R x = col[i];
        vsh[i] = x;
        t_all += x * x;
        if (i > 0) t_tail += x * x;
    }
    t_all = warp_sum(t_all);
    t_tail = warp_sum(t_tail);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { red[0][w] = t_all; red[1][w] = t_tail; }
    __syncthreads();
    if (threadIdx.x == 0) {
        R xn2 = 0, tail2 = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { xn2 += red[0][q]; tail2 += red[1][q]; }
        if (tail2 == R(0) || m <= 0) {
            s_scal[0] = 0;                      // no reflection
            s_scal[1] = m > 0 ? vsh[0] : R(0);  // the subdiagonal entry stays
        } else {
            const R xn = sqrt(xn2), x0 = vsh[0];
            const R sg = x0 >= R(0) ? R(1) : R(-1);
            const R v0 = x0 + sg * xn;          // no cancellation
            vsh[0] = v0;
            s_scal[0] = R(2) / (v0 * v0 + tail2);
            s_scal[1] = -sg * xn;
        }
    }
    __syncthreads();
}

template <class R>
__global__ void __launch_bounds__(kHrThreads) hessr_left_kernel(R *__restrict__ H, int n, int ld, R *__restrict__ Y,
                                                                R *__restrict__ scal, int k)
{
    extern __shared__ unsigned char smraw[];
    R *vsh = reinterpret_cast<R *>(smraw);
    __shared__ R s_scal[2];
    const int m = n - k - 1;
    real_reflector<R>(H + (k + 1) + (int64_t)k * ld, m, vsh, s_scal);
    const R beta = s_scal[0];
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < m; i += blockDim.x) Y[(k + 1) + i + (int64_t)k * ld] = beta == R(0) ? R(0) : vsh[i];
        if (threadIdx.x == 0) {
            scal[2 * k] = beta;
            scal[2 * k + 1] = s_scal[1];
        }
    }
    if (beta == R(0)) return;
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int j = k + 1 + gw; j < n; j += nw) {
        R *c = H + (k + 1) + (int64_t)j * ld;
        R acc = 0;
#pragma unroll 8
        for (int i = lane; i < m; i += 32) acc = fma(vsh[i], c[i], acc);
        const R wj = beta * warp_sum(acc);
#pragma unroll 8
        for (int i = lane; i < m; i += 32) c[i] = fma(-vsh[i], wj, c[i]);
    }
}

// grid (row tiles of kHrThreads rows, S column segments of width seg)
template <class R>
__global__ void __launch_bounds__(kHrThreads) hessr_rpart_kernel(const R *__restrict__ H, int n, int ld,
                                                                 const R *__restrict__ Y, const R *__restrict__ scal,
                                                                 R *__restrict__ part, int k, int seg)
{
    __shared__ R vs[1024];
    const int m = n - k - 1;
    if (scal[2 * k] == R(0)) return;
    const int j0 = k + 1 + blockIdx.y * seg, j1 = min(n, j0 + seg);
    const int i = blockIdx.x * kHrThreads + threadIdx.x;
    R acc = 0;
    for (int c0 = j0; c0 < j1; c0 += 1024) {
        const int c1 = min(j1, c0 + 1024);
        __syncthreads();
        for (int j = c0 + threadIdx.x; j < c1; j += blockDim.x) vs[j - c0] = Y[j + (int64_t)k * ld];
        __syncthreads();
        if (i < n) {
            const R *row = H + i;
#pragma unroll 4
            for (int j = c0; j < c1; ++j) acc = fma(row[(int64_t)j * ld], vs[j - c0], acc);
        }
    }
    (void)m;
    if (i < n) part[(int64_t)blockIdx.y * n + i] = acc;
}

template <class R>
__global__ void __launch_bounds__(kHrThreads) hessr_rupd_kernel(R *__restrict__ H, int n, int ld,
                                                                const R *__restrict__ Y, const R *__restrict__ scal,
                                                                const R *__restrict__ part, int S, int k, int seg)
{
    __shared__ R vs[1024];
    const R beta = scal[2 * k];
    const int m = n - k - 1;
    if (blockIdx.x == 0 && blockIdx.y == 0) {
        // column k: the reflected subdiagonal entry, zeros below it
        for (int i = threadIdx.x; i < m; i += blockDim.x)
            H[(k + 1) + i + (int64_t)k * ld] = i == 0 ? scal[2 * k + 1] : (beta == R(0) ? H[(k + 1) + i + (int64_t)k * ld] : R(0));
    }
    if (beta == R(0)) return;
    const int j0 = k + 1 + blockIdx.y * seg, j1 = min(n, j0 + seg);
    const int i = blockIdx.x * kHrThreads + threadIdx.x;
    R u = 0;
    if (i < n) {
        for (int q = 0; q < S; ++q) u += part[(int64_t)q * n + i];
        u *= beta;
    }
    for (int c0 = j0; c0 < j1; c0 += 1024) {
        const int c1 = min(j1, c0 + 1024);
        __syncthreads();
        for (int j = c0 + threadIdx.x; j < c1; j += blockDim.x) vs[j - c0] = Y[j + (int64_t)k * ld];
        __syncthreads();
        if (i < n) {
            R *row = H + i;
#pragma unroll 4
            for (int j = c0; j < c1; ++j) row[(int64_t)j * ld] = fma(-u, vs[j - c0], row[(int64_t)j * ld]);
        }
    }
}

// complex A_s (real parts) -> real H; Y <- 0; Qr <- I
template <class R>
__global__ void hessr_prologue_kernel(const cplx<R> *__restrict__ T, R *__restrict__ H, R *__restrict__ Y,
                                      R *__restrict__ Qr, int n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)n * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t % n), j = (int)(t / n);
        H[t] = T[t].x;
        Y[t] = R(0);
        Qr[t] = (i == j) ? R(1) : R(0);
    }
}

// real H (zero below the subdiagonal), real Q -> complex T, Q
template <class R>
__global__ void hessr_epilogue_kernel(const R *__restrict__ H, const R *__restrict__ Qr, cplx<R> *__restrict__ T,
                                      cplx<R> *__restrict__ Q, int n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)n * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t % n), j = (int)(t / n);
        T[t] = cplx<R>{i > j + 1 ? R(0) : H[t], R(0)};
        Q[t] = cplx<R>{Qr[t], R(0)};
    }
}

template <class R>
__global__ void hessr_betas_kernel(const R *__restrict__ scal, R *__restrict__ betas, int n)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        betas[k] = k + 2 < n ? scal[2 * k] : R(0);
}

template <class R>
size_t hessenberg_real_scratch(int n)
{
    // [beta_k, alpha_k] pairs, the betas gathered, 64 partial vectors, and
    // the back-transform's scratch
    return (size_t)2 * n + 64 + (size_t)n + 64 + (size_t)64 * n + (size_t)kBackNb * (kBackNb + 2 * (size_t)n) +
           (size_t)kBackNb * kBackNb + 64;
}

template <class R>
cudaError_t enqueue_hessenberg_real(const cplx<R> *T, R *H, R *Y, R *Qr, R *scratch, int n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t vbytes = (size_t)n * sizeof(R);
    cudaError_t err;
    if (vbytes > 48 * 1024 && (err = allow_max_smem((const void *)hessr_left_kernel<R>))) return err;
    R *scal = scratch, *betas = scal + 2 * (size_t)n + 64, *part = betas + n + 64, *bt = part + (size_t)64 * n;
    const int tiles = (int)cdiv_i(n, kHrThreads);
    const int S = std::max(1, std::min(64, (2 * sms + tiles - 1) / tiles));
    hessr_prologue_kernel<R><<<2 * sms, 256, 0, s>>>(T, H, Y, Qr, n); count_launch();
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        const int seg = (int)cdiv_i(m, S);
        const int lctas = (int)std::max<int64_t>(1, std::min<int64_t>(2 * sms, cdiv_i(m, kHrThreads / 32)));
        hessr_left_kernel<R><<<lctas, kHrThreads, vbytes, s>>>(H, n, n, Y, scal, k); count_launch();
        hessr_rpart_kernel<R><<<dim3(tiles, S), kHrThreads, 0, s>>>(H, n, n, Y, scal, part, k, seg); count_launch();
        hessr_rupd_kernel<R><<<dim3(tiles, S), kHrThreads, 0, s>>>(H, n, n, Y, scal, part, S, k, seg); count_launch();
    }
    // Q = P_0 P_1 ... P_{n-3} applied to I by the blocked compact-WY
    // back-transform (the reflectors' betas gathered contiguously first)
    hessr_betas_kernel<R><<<cdiv_i(n, 256), 256, 0, s>>>(scal, betas, n); count_launch();
    if ((err = launch_back_transform<R>(Y, n, betas, Qr, n, n, bt, s))) return err;
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_hessenberg_real_finish(const R *H, const R *Qr, cplx<R> *T, cplx<R> *Q, int n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    hessr_epilogue_kernel<R><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(1024, cdiv_i((int64_t)n * n, 256))), 256,
                               0, s>>>(H, Qr, T, Q, n);
    count_launch();
    return cudaGetLastError();
}

template size_t hessenberg_real_scratch<float>(int);
template size_t hessenberg_real_scratch<double>(int);
template cudaError_t enqueue_hessenberg_real<float>(const cplx<float> *, float *, float *, float *, float *, int,
                                                    cudaStream_t);
template cudaError_t enqueue_hessenberg_real<double>(const cplx<double> *, double *, double *, double *, double *,
                                                     int, cudaStream_t);
template cudaError_t launch_hessenberg_real_finish<float>(const float *, const float *, cplx<float> *, cplx<float> *,
                                                          int, cudaStream_t);
template cudaError_t launch_hessenberg_real_finish<double>(const double *, const double *, cplx<double> *,
                                                           cplx<double> *, int, cudaStream_t);

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
