// spd.cu -- symmetric positive definite path (Algorithm 3).
//
// Spectral decomposition A_s = V diag(lam) V^T (Algorithm 3, step 1):
//   1. Householder tridiagonalisation in the storage precision R (FP32 for
//      the mixed method): one launch per column that applies the symmetric
//      rank-2 update A -= v w^T + w v^T of step k (w = p - (beta/2)(v.p) v,
//      p = beta A v) and in the same pass forms the reflector and p of step
//      k+1 (one warp per column of the trailing block).  The reflectors are
//      kept (one column each) for step 4;
//   2. eigenvalues of the tridiagonal matrix: FP32 multisection (one warp
//      per eigenvalue, 32 Sturm counts per round) to a bracket of FP32
//      width, checked and finished by FP64 multisection (a few lanes per
//      eigenvalue) whose Sturm counts run the division-free recurrence of
//      the leading principal minors;
//   3. eigenvectors of the tridiagonal matrix from twisted factorisations
//      T - lam I = L D+ L^T = U D- U^T (FP64; the pivots from the leading
//      and trailing principal minors, computed without division): with
//      r = argmin |D+_r + D-_r - (d_r - lam)|, z_r = 1,
//      z_i = -(e_i / D+_i) z_{i+1} above r, z_{i+1} = -(e_i / D-_{i+1}) z_i
//      below r, normalised; members of eigenvalue clusters (closer than the
//      eigenvalues' accuracy) are recomputed as the part of a pseudo-random
//      vector orthogonal to every other eigenvector;
//   4. V = Q Z: the reflectors applied to Z in blocks of 64 in compact WY
//      form (three products per block).
// Steps 2-3 are O(n^2) work; the O(n^3) steps 1 and 4 run in R.
//
// Refinement (Algorithm 3, steps 4-12): FP64 symmetric residual, then
// Y = (V^T Rhat V) ./ (s_i + s_j) with the division fused into the second
// product, X += 2^e V Y V^T with a mirrored FP64 epilogue (X stays exactly
// symmetric).
#include <limits.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "handle.h"
#include "spd_internal.h"
#include "tc_gemm.h"

namespace sqm {

// CTA of the tridiagonalisation steps: every CTA reads the step's v, p and
// next column (3 m values) from L2 before its columns, so few wide CTAs (one
// per SM) keep that redundant traffic small; a warp takes one column
static constexpr int kTriThreads2 = 1024;
static constexpr int kTriMaxFit = 2048 / kTriThreads2 < 4 ? 2048 / kTriThreads2 : 4;
static constexpr int kTriBatch = 8;  // rows in flight per lane in tri_step_kernel

// reflector for x = A(k+1:n, k) (real): v = x + sign(x0) ||x|| e1,
// beta = 2 / ||v||^2, P x = -sign(x0) ||x|| e1
template <class R>
__device__ void real_reflector(const R *__restrict__ col, int m, R *vsh, R *scal /* beta, xn, sign */)
{
    __shared__ R red[2][kTriThreads2 / 32];
    R t_all = 0, t_tail = 0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        R x = col[i];
        vsh[i] = x;
        t_all = fma(x, x, t_all);
        if (i > 0) t_tail = fma(x, x, t_tail);
    }
    t_all = warp_sum(t_all);
    t_tail = warp_sum(t_tail);
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = t_all; red[1][threadIdx.x >> 5] = t_tail; }
    __syncthreads();
    if (threadIdx.x == 0) {
        R xn2 = 0, tail2 = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { xn2 += red[0][q]; tail2 += red[1][q]; }
        if (tail2 == R(0) || m <= 0) {
            scal[0] = 0; scal[1] = 0; scal[2] = 1;
        } else {
            R xn = sqrt(xn2);
            R x0 = vsh[0];
            R sg = (x0 >= R(0)) ? R(1) : R(-1);
            R v0 = x0 + sg * xn;
            vsh[0] = v0;
            scal[0] = R(2) / (v0 * v0 + tail2);
            scal[1] = xn;
            scal[2] = sg;
        }
    }
    __syncthreads();
}

template <class R>
__global__ void __launch_bounds__(kTriThreads2)
tri_symv_kernel(const R *__restrict__ A, int n, int ld, int k, R *__restrict__ wsv,
                R *__restrict__ wsp, R *__restrict__ wss, R *__restrict__ Y, int ldy,
                R *__restrict__ betas)
{
    extern __shared__ unsigned char smraw[];
    R *vsh = reinterpret_cast<R *>(smraw);
    __shared__ R scal[3];
    const int m = n - k - 1;
    real_reflector<R>(A + (k + 1) + (int64_t)k * ld, m, vsh, scal);
    const R beta = scal[0];
    if (blockIdx.x == 0) {
        R *yk = Y + (k + 1) + (int64_t)k * ldy;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            wsv[i] = vsh[i];
            yk[i] = vsh[i];
        }
        if (threadIdx.x < 3) wss[threadIdx.x] = scal[threadIdx.x];
        if (threadIdx.x == 0) betas[k] = beta;
    }
    if (beta == R(0)) return;
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nw = gridDim.x * (blockDim.x >> 5);
    // p_j = beta * sum_i A(k+1+i, k+1+j) v_i  (column j of the symmetric block)
    for (int j = gw; j < m; j += nw) {
        const R *c = A + (k + 1) + (int64_t)(k + 1 + j) * ld;
        R acc = 0;
#pragma unroll 8
        for (int i = lane; i < m; i += 32) acc = fma(c[i], vsh[i], acc);
        acc = warp_sum(acc);
        if (lane == 0) wsp[j] = beta * acc;
    }
}

// One step s of the tridiagonalisation in one launch: the rank-2 update of
// step s on the trailing block A(s+1:n, s+1:n) <- A - v w^T - w v^T, with
// w = p - (beta/2)(v.p) v from v, beta and p = beta A v of the previous
// launch, and in the same pass the quantities of step s+1: every CTA updates
// column s+1 of the block itself and forms its reflector (redundantly; the
// column is read, never written, in this launch), and each warp, right after
// updating a column of A(s+2:n, s+2:n), takes its product with the new
// reflector, which gives p for step s+1.  One read and one write of the
// trailing block per step instead of three passes.  Row s+1 of the block
// (above the diagonal of columns > s+1) is not kept up to date: nothing
// reads it again.  Column s receives its final entries (subdiagonal
// -sign ||x||, zeros below) and its diagonal from the previous launch; the
// values of the last column pair go to ns[4..5] (tri_finish_kernel).
// cv, cp, cs: v, p and [beta, ||x||, sign, diagonal of column s] of step s;
// nv, np, ns: the same for step s+1.
template <class R>
__global__ void __launch_bounds__(kTriThreads2)
tri_step_kernel(R *__restrict__ A, int n, int ld, int s, const R *__restrict__ cv, const R *__restrict__ cp,
                const R *__restrict__ cs, R *__restrict__ nv, R *__restrict__ np, R *__restrict__ ns,
                R *__restrict__ Y, int ldy, R *__restrict__ betas)
{
    extern __shared__ unsigned char smraw[];
    const int m = n - s - 1;  // block rows / columns s+1 .. n-1
    R *vs = reinterpret_cast<R *>(smraw), *wsm = vs + m, *cn = wsm + m, *vn = cn + m;
    __shared__ R red[kTriThreads2 / 32];
    __shared__ R s_K, s_scal[3];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const R beta = cs[0];
    const R *c1 = A + (s + 1) + (int64_t)(s + 1) * ld;  // column s+1 of the block
    R acc = 0;
    // all global reads of the prologue, kTriPro rows per thread in flight at
    // once (a step's prologue is a chain of L2 round trips otherwise); the
    // products v.p are summed in the same order either way
    constexpr int kTriPro = 8;
    for (int b0 = tid; b0 < m; b0 += kTriThreads2 * kTriPro) {
        R v[kTriPro], pq[kTriPro], c[kTriPro];
#pragma unroll
        for (int u = 0; u < kTriPro; ++u) {
            const int i = b0 + u * kTriThreads2;
            v[u] = i < m ? cv[i] : R(0);
            pq[u] = (i < m && beta != R(0)) ? cp[i] : R(0);
            c[u] = i < m ? c1[i] : R(0);
        }
#pragma unroll
        for (int u = 0; u < kTriPro; ++u) {
            const int i = b0 + u * kTriThreads2;
            if (i < m) {
                vs[i] = v[u];
                wsm[i] = pq[u];
                cn[i] = c[u];
                acc = fma(v[u], pq[u], acc);
            }
        }
    }
    acc = warp_sum(acc);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (tid == 0) {
        R t = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        s_K = R(0.5) * beta * t;
    }
    __syncthreads();
    const R K = s_K;
    for (int i = tid; i < m; i += blockDim.x) wsm[i] = beta != R(0) ? fma(-K, vs[i], wsm[i]) : R(0);
    __syncthreads();
    {
        const R v0 = vs[0], w0 = wsm[0];
        for (int i = tid; i < m; i += blockDim.x) cn[i] = fma(-vs[i], w0, fma(-wsm[i], v0, cn[i]));
    }
    __syncthreads();
    const bool more = s + 4 <= n;  // column s+1 has a reflector
    R bn = 0;
    if (more) {
        real_reflector<R>(cn + 1, m - 1, vn, s_scal);
        bn = s_scal[0];
    }
    // the step's outputs, split over all CTAs (each holds vn and the
    // scalars): column s's final entries, the reflector of step s+1 (into Y
    // and nv), its scalars
    {
        const int gt = blockIdx.x * blockDim.x + tid, gs = gridDim.x * blockDim.x;
        const bool lead = blockIdx.x == 0 && tid == 0;
        if (beta != R(0))
            for (int i = gt; i < m; i += gs) A[(s + 1 + i) + (int64_t)s * ld] = (i == 0) ? -cs[2] * cs[1] : R(0);
        if (s >= 1 && lead) A[s + (int64_t)s * ld] = cs[3];
        if (more) {
            R *yk = Y + (s + 2) + (int64_t)(s + 1) * ldy;
            for (int i = gt; i < m - 1; i += gs) {
                nv[i] = vn[i];
                yk[i] = vn[i];
            }
            if (lead) {
                ns[0] = s_scal[0]; ns[1] = s_scal[1]; ns[2] = s_scal[2]; ns[3] = cn[0];
                betas[s + 1] = bn;
            }
        } else if (lead) {
            ns[4] = cn[0];
            ns[5] = cn[1];
        }
    }
    // columns interleaved over the CTAs (column 1 + CTA + grid * warp), so
    // that every SM holds columns while there are as many as SMs
    const int gw = warp * gridDim.x + blockIdx.x;
    const int nwt = gridDim.x * (blockDim.x >> 5);
    // columns of the block: the loads of a batch of kTriBatch rows per lane
    // are issued before any is used
    for (int j = 1 + gw; j < m; j += nwt) {
        R *c = A + (s + 1) + (int64_t)(s + 1 + j) * ld;
        const R vj = vs[j], wj = wsm[j];
        R dot = 0;
        for (int i0 = 1 + lane; i0 < m; i0 += 32 * kTriBatch) {
            R x[kTriBatch];
#pragma unroll
            for (int u = 0; u < kTriBatch; ++u) {
                const int i = i0 + 32 * u;
                x[u] = i < m ? c[i] : R(0);
            }
#pragma unroll
            for (int u = 0; u < kTriBatch; ++u) {
                const int i = i0 + 32 * u;
                if (i < m) {
                    const R cc = fma(-vs[i], wj, fma(-wsm[i], vj, x[u]));
                    c[i] = cc;
                    if (more) dot = fma(cc, vn[i - 1], dot);
                }
            }
        }
        if (more) {
            dot = warp_sum(dot);
            if (lane == 0) np[j - 1] = bn * dot;
        }
    }
}

// the last two columns: diagonal and subdiagonal of column n-2 (n >= 3)
template <class R>
__global__ void tri_finish_kernel(R *__restrict__ A, int n, int ld, const R *__restrict__ ns)
{
    if (threadIdx.x == 0) {
        A[(n - 2) + (int64_t)(n - 2) * ld] = ns[4];
        A[(n - 1) + (int64_t)(n - 2) * ld] = ns[5];
    }
}

template <class R>
cudaError_t launch_tridiag(R *A, int n, int ld, R *Y, int ldy, R *betas, R *ws, cudaStream_t s)
{
    if (n < 3) return cudaSuccess;
    // two sets of (v, p, scalars), alternating between steps
    R *set[2] = {ws, ws + 2 * n + 8};
    size_t sm1 = (size_t)n * sizeof(R);
    size_t sm4 = 4 * sm1;
    cudaError_t err;
    if (sm1 > 48 * 1024 && (err = allow_max_smem((const void *)tri_symv_kernel<R>))) return err;
    if (sm4 > 48 * 1024 && (err = allow_max_smem((const void *)tri_step_kernel<R>))) return err;
    {
        const int m = n - 1;
        const int ctas = (int)std::min<int64_t>(cdiv_i(m, kTriThreads2 / 32), 304);
        tri_symv_kernel<R><<<ctas, kTriThreads2, sm1, s>>>(A, n, ld, 0, set[0], set[0] + n, set[0] + 2 * n, Y, ldy,
                                                            betas);
        count_launch();
    }
    // as many CTAs as fit at once, never a second wave (the four shared
    // vectors of m entries limit residency for large m)
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int fit = 0;  // resident CTAs per SM at the current m (grows as m shrinks)
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        if (fit < kTriMaxFit) {
            int nb = 0;
            if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tri_step_kernel<R>, kTriThreads2,
                                                                      (size_t)4 * m * sizeof(R))))
                return err;
            fit = std::max(1, std::min(kTriMaxFit, nb));
        }
        const int64_t tri_ctas = (int64_t)fit * sms;
        const int ctas = (int)std::min<int64_t>(std::max<int64_t>(1, m - 1), tri_ctas);
        R *c = set[k & 1], *x = set[(k + 1) & 1];
        tri_step_kernel<R><<<ctas, kTriThreads2, (size_t)4 * m * sizeof(R), s>>>(A, n, ld, k, c, c + n, c + 2 * n, x,
                                                                                  x + n, x + 2 * n, Y, ldy, betas);
        count_launch();
    }
    tri_finish_kernel<R><<<1, 32, 0, s>>>(A, n, ld, set[(n - 2) & 1] + 2 * n);
    count_launch();
    return cudaGetLastError();
}

template cudaError_t launch_tridiag<float>(float *, int, int, float *, int, float *, float *, cudaStream_t);
template cudaError_t launch_tridiag<double>(double *, int, int, double *, int, double *, double *, cudaStream_t);

// T of the compact WY form of one block of nb reflectors: Q_b = H_0 ... H_{nb-1}
// = I - Y T Y^T with T upper triangular, T(i,i) = beta_i and
// T(0:i, i) = -beta_i T(0:i, 0:i) G(0:i, i), G = Y^T Y (one CTA; column by
// column since column i needs the columns before it).
template <class R>
__global__ void larft_kernel(const R *__restrict__ G, int ldg, const R *__restrict__ beta, int nb,
                             R *__restrict__ Tm, int ldt)
{
    __shared__ R g[kBackNb];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) Tm[(e % nb) + (int64_t)(e / nb) * ldt] = R(0);
    __syncthreads();
    for (int i = 0; i < nb; ++i) {
        const R bi = beta[i];
        for (int c = threadIdx.x; c < i; c += blockDim.x) g[c] = G[c + (int64_t)i * ldg];
        __syncthreads();
        for (int r = threadIdx.x; r < i; r += blockDim.x) {
            R acc = 0;
            for (int c = r; c < i; ++c) acc = fma(Tm[r + (int64_t)c * ldt], g[c], acc);
            Tm[r + (int64_t)i * ldt] = -bi * acc;
        }
        if (threadIdx.x == 0) Tm[i + (int64_t)i * ldt] = bi;
        __syncthreads();
    }
}

template <class R>
static cudaError_t back_transform_products(const R *Y, int ldy, const R *betas, R *Z, int n, int ldz, R *scratch,
                                  cudaStream_t s)
{
    const int nref = std::max(0, n - 2);
    R *G = scratch, *Tm = G + kBackNb * kBackNb, *W = Tm + kBackNb * kBackNb, *W2 = W + (size_t)kBackNb * n;
    const int nblk = (int)cdiv_i(nref, kBackNb);
    for (int b = nblk - 1; b >= 0; --b) {
        const int k0 = b * kBackNb, nb = std::min(kBackNb, nref - k0);
        const int r0 = k0 + 1, mb = n - r0;
        const R *Yb = Y + r0 + (int64_t)k0 * ldy;
        cudaError_t err;
        if ((err = launch_rgemm<R>(1, 0, nb, nb, mb, Yb, ldy, Yb, ldy, RG_STORE, G, nb, nullptr, nullptr, 0, 0.0, s))) return err;
        larft_kernel<R><<<1, 64, 0, s>>>(G, nb, betas + k0, nb, Tm, nb); count_launch();
        if ((err = launch_rgemm<R>(1, 0, nb, n, mb, Yb, ldy, Z + r0, ldz, RG_STORE, W, nb, nullptr, nullptr, 0, 0.0, s))) return err;
        if ((err = launch_rgemm<R>(0, 0, nb, n, nb, Tm, nb, W, nb, RG_STORE, W2, nb, nullptr, nullptr, 0, 0.0, s))) return err;
        if ((err = launch_rgemm<R>(0, 0, mb, n, nb, Yb, ldy, W2, nb, RG_SUB, Z + r0, ldz, nullptr, nullptr, 0, 0.0, s))) return err;
    }
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// FP32 back-transform in one pass per column panel.  Z <- Q Z with
// Q = Q_0 Q_1 ... Q_{nblk-1} and Q_b = I - Y_b T_b Y_b^T acts on each column
// of Z on its own, so a CTA that owns a panel of kBtCols columns applies
// every block to it, last block first, with no synchronisation between CTAs:
//   W = Y_b^T Z_p (64 x kBtCols), W <- T_b W, Z_p -= Y_b W.
// Y_b and Z_p stream through shared memory in cp.async stages; the T_b of
// all blocks come from one earlier launch (bt_prep_kernel, a CTA per block:
// G_b = Y_b^T Y_b, then T_b column by column, T(i,i) = beta_i,
// T(0:i, i) = -beta_i T(0:i, 0:i) G(0:i, i)).  Products on 4 x 4 register
// tiles; per block and panel 2 * 64 * kBtCols FMAs per row of Y_b.
// ---------------------------------------------------------------------------
static constexpr int kBtCols = 32, kBtThreads = 256, kBtStages = 3;
static constexpr int kBtKa = 32;   // rows of Y_b, Z_p per stage of W = Y_b^T Z_p
static constexpr int kBtKc = 128;  // rows of Y_b per stage of Z_p -= Y_b W
static constexpr int kBtStA = kBtKa * (kBackNb + kBtCols), kBtStC = kBackNb * kBtKc;
static constexpr int kBtStg = kBtStages * (kBtStA > kBtStC ? kBtStA : kBtStC);
static constexpr size_t kBtApplySmem = (size_t)(kBtStg + 64 * 65 + 2 * 64 * 36) * sizeof(float);
static constexpr size_t kBtPrepSmem = (size_t)(kBtStages * kBtKa * kBackNb + 2 * 64 * 65) * sizeof(float);

__device__ __forceinline__ void bt_cp4(float *dst, const float *src, bool valid)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void bt_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void bt_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Row-major stage rows (k = row of Y_b / Z_p, i = column): the group of four
// columns holding i is XOR-ed with bits 2..4 of k, so that the copies (four
// consecutive rows of a column per thread) and the float4 reads of the
// products are free of bank conflicts.
__device__ __forceinline__ int bt_swz(int k, int i) { return (((i >> 2) ^ ((k >> 2) & 7)) << 2) | (i & 3); }

// cp.async copies of rows [r, r + kBtKa) of the leading nc (<= WIDTH)
// columns of the mb-row block P (ld ldp) into the swizzled stage st (rows of
// WIDTH floats), a thread taking four consecutive rows of one column; rows
// at or past mb and columns at or past nc are zero-filled
template <int WIDTH>
__device__ __forceinline__ void bt_stage_rows(float *st, const float *P, int ldp, int r, int mb, int nc, int tid)
{
    for (int u = tid; u < 8 * WIDTH; u += kBtThreads) {
        const int kq = u & 7, i = u >> 3;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = 4 * kq + q;
            const bool v = r + k < mb && i < nc;
            bt_cp4(st + k * WIDTH + bt_swz(k, i), v ? P + (r + k) + (int64_t)i * ldp : P, v);
        }
    }
}

__global__ void __launch_bounds__(kBtThreads) bt_prep_kernel(const float *__restrict__ Y, int ldy,
                                                             const float *__restrict__ betas, int n, int nref,
                                                             float *__restrict__ Tall)
{
    extern __shared__ __align__(16) float btsm[];
    float *ys = btsm, *gs = ys + kBtStages * kBtKa * kBackNb, *ts = gs + 64 * 65;
    const int b = blockIdx.x, tid = threadIdx.x;
    const int k0 = b * kBackNb, nb = min(kBackNb, nref - k0), r0 = k0 + 1, mb = n - r0;
    const float *Yb = Y + r0 + (int64_t)k0 * ldy;
    const int nch = (mb + kBtKa - 1) / kBtKa;
    auto issue = [&](int c) {
        if (c < nch) bt_stage_rows<kBackNb>(ys + (c % kBtStages) * kBtKa * kBackNb, Yb, ldy, c * kBtKa, mb, nb, tid);
        bt_commit();
    };
    // G = Y_b^T Y_b, thread tile G(4ty.., 4tx..)
    const int tx = tid & 15, ty = tid >> 4;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int c = 0; c < kBtStages - 1; ++c) issue(c);
    for (int c = 0; c < nch; ++c) {
        bt_wait<kBtStages - 2>();
        __syncthreads();
        issue(c + kBtStages - 1);
        const float *st = ys + (c % kBtStages) * kBtKa * kBackNb;
#pragma unroll 8
        for (int k = 0; k < kBtKa; ++k) {
            const int sw = (k >> 2) & 7;
            const float4 a = *reinterpret_cast<const float4 *>(st + k * kBackNb + ((ty ^ sw) << 2));
            const float4 g = *reinterpret_cast<const float4 *>(st + k * kBackNb + ((tx ^ sw) << 2));
            const float av[4] = {a.x, a.y, a.z, a.w}, gv[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], gv[j], acc[i][j]);
        }
    }
    bt_wait<0>();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) gs[(4 * ty + i) * 65 + 4 * tx + j] = acc[i][j];
    for (int e = tid; e < 64 * 65; e += kBtThreads) ts[e] = 0.f;
    __syncthreads();
    // T column by column (column i needs the columns before it)
    for (int i = 0; i < nb; ++i) {
        const float bi = betas[k0 + i];
        if (tid < i) {
            float t = 0.f;
            for (int c = tid; c < i; ++c) t = fmaf(ts[tid * 65 + c], gs[c * 65 + i], t);
            ts[tid * 65 + i] = -bi * t;
        } else if (tid == i) {
            ts[i * 65 + i] = bi;
        }
        __syncthreads();
    }
    float *Tb = Tall + (size_t)b * kBackNb * kBackNb;  // column-major, zero outside the leading nb x nb
    for (int e = tid; e < kBackNb * kBackNb; e += kBtThreads) Tb[e] = ts[(e & 63) * 65 + (e >> 6)];
}

__global__ void __launch_bounds__(kBtThreads) bt_apply_kernel(const float *__restrict__ Y, int ldy,
                                                              const float *__restrict__ Tall, int n, int nref,
                                                              float *__restrict__ Z, int ldz)
{
    extern __shared__ __align__(16) float btsm[];
    float *stg = btsm, *ts = stg + kBtStg, *wb = ts + 64 * 65, *w2 = wb + 64 * 36;
    const int tid = threadIdx.x;
    const int c0 = blockIdx.x * kBtCols, nc = min(kBtCols, n - c0);
    const int nblk = (nref + kBackNb - 1) / kBackNb;
    for (int b = nblk - 1; b >= 0; --b) {
        const int k0 = b * kBackNb, nb = min(kBackNb, nref - k0), r0 = k0 + 1, mb = n - r0;
        const float *Yb = Y + r0 + (int64_t)k0 * ldy;
        float *Zp = Z + r0 + (int64_t)c0 * ldz;
        {
            const float *Tb = Tall + (size_t)b * kBackNb * kBackNb;
            for (int e = tid; e < kBackNb * kBackNb; e += kBtThreads) ts[(e & 63) * 65 + (e >> 6)] = Tb[e];
        }
        // W = Y_b^T Z_p: two groups of 128 threads take the two halves of
        // each stage's rows; thread tile W(4ty.., 4tx..)
        {
            const int nch = (mb + kBtKa - 1) / kBtKa;
            auto issue = [&](int c) {
                if (c < nch) {
                    float *ya = stg + (c % kBtStages) * kBtStA, *za = ya + kBtKa * kBackNb;
                    bt_stage_rows<kBackNb>(ya, Yb, ldy, c * kBtKa, mb, nb, tid);
                    bt_stage_rows<kBtCols>(za, Zp, ldz, c * kBtKa, mb, nc, tid);
                }
                bt_commit();
            };
            const int g = tid >> 7, t = tid & 127, tx = t & 7, ty = t >> 3;
            float acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
            for (int c = 0; c < kBtStages - 1; ++c) issue(c);
            for (int c = 0; c < nch; ++c) {
                bt_wait<kBtStages - 2>();
                __syncthreads();
                issue(c + kBtStages - 1);
                const float *ya = stg + (c % kBtStages) * kBtStA, *za = ya + kBtKa * kBackNb;
#pragma unroll 8
                for (int kk = 0; kk < kBtKa / 2; ++kk) {
                    const int k = g * (kBtKa / 2) + kk, sw = (k >> 2) & 7;
                    const float4 a = *reinterpret_cast<const float4 *>(ya + k * kBackNb + ((ty ^ sw) << 2));
                    const float4 z = *reinterpret_cast<const float4 *>(za + k * kBtCols + ((tx ^ sw) << 2));
                    const float av[4] = {a.x, a.y, a.z, a.w}, zv[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], zv[j], acc[i][j]);
                }
            }
            bt_wait<0>();
            __syncthreads();
            if (g == 1) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) wb[(4 * ty + i) * 36 + 4 * tx + j] = acc[i][j];
            }
            __syncthreads();
            if (g == 0) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) wb[(4 * ty + i) * 36 + 4 * tx + j] += acc[i][j];
            }
            __syncthreads();
        }
        // W <- T_b W (T_b upper triangular, zero below its diagonal)
        {
            const int i = tid >> 2, cc = (tid & 3) * 8;
            float a[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) a[j] = 0.f;
#pragma unroll 4
            for (int l = 0; l < kBackNb; ++l) {
                const float tl = ts[i * 65 + l];
                const float4 w0 = *reinterpret_cast<const float4 *>(wb + l * 36 + cc);
                const float4 w1 = *reinterpret_cast<const float4 *>(wb + l * 36 + cc + 4);
                a[0] = fmaf(tl, w0.x, a[0]); a[1] = fmaf(tl, w0.y, a[1]);
                a[2] = fmaf(tl, w0.z, a[2]); a[3] = fmaf(tl, w0.w, a[3]);
                a[4] = fmaf(tl, w1.x, a[4]); a[5] = fmaf(tl, w1.y, a[5]);
                a[6] = fmaf(tl, w1.z, a[6]); a[7] = fmaf(tl, w1.w, a[7]);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) w2[i * 36 + cc + j] = a[j];
        }
        __syncthreads();
        // Z_p -= Y_b W: stages of kBtKc rows of Y_b (column-major, as stored);
        // thread tile Z_p(4ty.., 4tx..) of each stage, its Z values loaded
        // before the wait
        {
            const int nch = (mb + kBtKc - 1) / kBtKc;
            auto issue = [&](int c) {
                if (c < nch) {
                    float *yc = stg + (c % kBtStages) * kBtStC;
                    const int r = c * kBtKc;
                    for (int e = tid; e < kBackNb * kBtKc; e += kBtThreads) {
                        const int rr = e % kBtKc, l = e / kBtKc;
                        const bool v = r + rr < mb && l < nb;
                        bt_cp4(yc + l * kBtKc + rr, v ? Yb + (r + rr) + (int64_t)l * ldy : Yb, v);
                    }
                }
                bt_commit();
            };
            const int tx = tid & 7, ty = tid >> 3;
            for (int c = 0; c < kBtStages - 1; ++c) issue(c);
            for (int c = 0; c < nch; ++c) {
                const int r = c * kBtKc;
                float z[4][4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int row = r + 4 * ty + q, col = 4 * tx + e;
                        z[q][e] = (row < mb && col < nc) ? Zp[row + (int64_t)col * ldz] : 0.f;
                    }
                bt_wait<kBtStages - 2>();
                __syncthreads();
                issue(c + kBtStages - 1);
                const float *yc = stg + (c % kBtStages) * kBtStC;
                float acc[4][4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[q][e] = 0.f;
#pragma unroll 8
                for (int l = 0; l < kBackNb; ++l) {
                    const float4 y = *reinterpret_cast<const float4 *>(yc + l * kBtKc + 4 * ty);
                    const float4 w = *reinterpret_cast<const float4 *>(w2 + l * 36 + 4 * tx);
                    const float yv[4] = {y.x, y.y, y.z, y.w}, wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q)
#pragma unroll
                        for (int e = 0; e < 4; ++e) acc[q][e] = fmaf(yv[q], wv[e], acc[q][e]);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int row = r + 4 * ty + q, col = 4 * tx + e;
                        if (row < mb && col < nc) Zp[row + (int64_t)col * ldz] = z[q][e] - acc[q][e];
                    }
            }
            bt_wait<0>();
            __syncthreads();
        }
    }
}

template <class R>
cudaError_t launch_back_transform(const R *Y, int ldy, const R *betas, R *Z, int n, int ldz, R *scratch,
                                  cudaStream_t s)
{
    if constexpr (std::is_same<R, float>::value) {
        const int nref = std::max(0, n - 2);
        if (nref == 0) return cudaSuccess;
        const int nblk = (int)cdiv_i(nref, kBackNb);
        cudaError_t err;
        if ((err = allow_max_smem((const void *)bt_prep_kernel)) || (err = allow_max_smem((const void *)bt_apply_kernel)))
            return err;
        bt_prep_kernel<<<nblk, kBtThreads, kBtPrepSmem, s>>>(Y, ldy, betas, n, nref, scratch);
        count_launch();
        bt_apply_kernel<<<(unsigned)cdiv_i(n, kBtCols), kBtThreads, kBtApplySmem, s>>>(Y, ldy, scratch, n, nref, Z, ldz);
        count_launch();
        return cudaGetLastError();
    } else {
        return back_transform_products<R>(Y, ldy, betas, Z, n, ldz, scratch, s);
    }
}

template cudaError_t launch_back_transform<float>(const float *, int, const float *, float *, int, int, float *, cudaStream_t);
template cudaError_t launch_back_transform<double>(const double *, int, const double *, double *, int, int, double *, cudaStream_t);

// ---------------------------------------------------------------------------
// tridiagonal eigensolver in FP64
// ---------------------------------------------------------------------------
// d, e, e^2, Gershgorin interval [gl, gu] and the pivot floor
template <class R>
__global__ void tri_extract_kernel(const R *__restrict__ A, int n, int ld, double *d, double *e,
                                   double *e2, double *bounds, float *df, float *e2f)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        d[i] = (double)A[i + (int64_t)i * ld];
        double ei = (i + 1 < n) ? (double)A[(i + 1) + (int64_t)i * ld] : 0.0;
        e[i] = ei;
        e2[i] = ei * ei;
        df[i] = (float)d[i];
        e2f[i] = (float)e2[i];
    }
    __syncthreads();
    // Gershgorin interval and the largest e^2: a block reduction (min, max
    // and max are exact, so the order does not matter)
    __shared__ double s_gl[32], s_gu[32], s_em[32];
    double gl = INFINITY, gu = -INFINITY, emax2 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double r = fabs(e[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0);
        gl = fmin(gl, d[i] - r);
        gu = fmax(gu, d[i] + r);
        emax2 = fmax(emax2, e2[i]);
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
        gl = fmin(gl, __shfl_xor_sync(0xffffffffu, gl, m));
        gu = fmax(gu, __shfl_xor_sync(0xffffffffu, gu, m));
        emax2 = fmax(emax2, __shfl_xor_sync(0xffffffffu, emax2, m));
    }
    if ((threadIdx.x & 31) == 0) { s_gl[threadIdx.x >> 5] = gl; s_gu[threadIdx.x >> 5] = gu; s_em[threadIdx.x >> 5] = emax2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
            gl = fmin(gl, s_gl[q]);
            gu = fmax(gu, s_gu[q]);
            emax2 = fmax(emax2, s_em[q]);
        }
        double w = fmax(fabs(gl), fabs(gu));
        bounds[0] = gl - 4.0 * 1.1102230246251565e-16 * w * n - 1e-300;
        bounds[1] = gu + 4.0 * 1.1102230246251565e-16 * w * n + 1e-300;
        bounds[2] = 2.2250738585072014e-308 * fmax(1.0, emax2);
        bounds[3] = 1.1754943508222875e-38 * fmax(1.0, emax2);  // FP32 pivot floor
    }
}

// Number of eigenvalues of the symmetric tridiagonal T below x, from the
// leading principal minors p_i = det((T - x I)(0:i, 0:i)):
//   p_{-1} = 1,  p_0 = d_0 - x,  p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2}.
// The pivots q_i = p_i / p_{i-1} of T - x I = L D L^T are negative exactly
// where consecutive minors change sign, and by Sylvester's law of inertia
// their number of negatives is the number of eigenvalues below x (the Sturm
// sequence property of the minors).  A zero minor becomes -2^-500 p_{i-1},
// a tiny pivot of the sign opposite to its predecessor (counted negative,
// as the ratio form counts a zero pivot).  Unlike the ratio form q_i =
// (d_i - x) - e_{i-1}^2 / q_{i-1}, the recurrence needs no division: one
// FMA per step on the dependency chain, which is what bounds a count on a
// part whose FP64 operations have long latency.  Every 8 steps the pair
// (p_i, p_{i-1}) is rescaled by a power of two (exact) to stay in range;
// the next block's d_i - x and e_{i-1}^2 are formed while the current one
// runs, and the signs are read from the bits.
__device__ __forceinline__ double minor_fix(double p, double pm)
{
    // -2^-500 |pm| sign(pm) from the bits (no FP64 instruction: on this
    // part every FP64 instruction of a warp costs tens of cycles): the sign
    // flipped, the exponent lowered by 500 (floored at the smallest normal)
    const long long pb = __double_as_longlong(p);
    if ((pb << 1) != 0) return p;
    const long long mb = __double_as_longlong(pm);
    const long long ex = (mb >> 52) & 0x7FF;
    const long long nx = ex > 501 ? ex - 500 : 1;
    return __longlong_as_double(((mb ^ (long long)0x8000000000000000ull) & (long long)0x800FFFFFFFFFFFFFull) | (nx << 52));
}

__device__ __forceinline__ int sign_flip(double a, double b)
{
    return (int)((unsigned long long)(__double_as_longlong(a) ^ __double_as_longlong(b)) >> 63);
}

__device__ __forceinline__ int minor_rescale(double &p, double &pm)
{
    const unsigned long long a = (unsigned long long)__double_as_longlong(p) & 0x7FFFFFFFFFFFFFFFull;
    const unsigned long long b = (unsigned long long)__double_as_longlong(pm) & 0x7FFFFFFFFFFFFFFFull;
    const int E = max(-1000, min(1000, (int)((a > b ? a : b) >> 52) - 1023));
    const double sc = __longlong_as_double((long long)(1023 - E) << 52);  // 2^-E
    p *= sc;
    pm *= sc;
    return E;
}

// (with fm, fe: also det(T - x I) = fm 2^fe, the last minor and the sum of
// the rescaling exponents)
__device__ __forceinline__ int sturm_count(const double *__restrict__ d, const double *__restrict__ e2, int n, double x,
                                           double *fm = nullptr, int *fe = nullptr)
{
    constexpr int B = 8;
    int ex = 0;
    double pm = 1.0, p = minor_fix(d[0] - x, 1.0);
    int c = sign_flip(p, 1.0);
    int i = 1;
    double dm[B], ee[B];
    if (i + B <= n) {
#pragma unroll
        for (int u = 0; u < B; ++u) {
            dm[u] = d[i + u] - x;
            ee[u] = e2[i + u - 1];
        }
    }
    for (; i + B <= n; i += B) {
        const bool more = i + 2 * B <= n;
        double dn[B], en[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
            dn[u] = more ? d[i + B + u] - x : 0.0;
            en[u] = more ? e2[i + B + u - 1] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const double pn = minor_fix(fma(dm[u], p, -ee[u] * pm), p);
            c += sign_flip(pn, p);
            pm = p;
            p = pn;
        }
        ex += minor_rescale(p, pm);
#pragma unroll
        for (int u = 0; u < B; ++u) {
            dm[u] = dn[u];
            ee[u] = en[u];
        }
    }
    for (; i < n; ++i) {
        const double pn = minor_fix(fma(d[i] - x, p, -e2[i - 1] * pm), p);
        c += sign_flip(pn, p);
        pm = p;
        p = pn;
    }
    if (fm) { *fm = p; *fe = ex; }
    return c;
}

__device__ __forceinline__ int sturm_count_f32(const float *__restrict__ d, const float *__restrict__ e2, int n,
                                               float x, float pivmin)
{
    float q = d[0] - x;
    if (fabsf(q) < pivmin) q = -pivmin;
    int c = q < 0.0f;
    for (int i = 1; i < n; ++i) {
        q = (d[i] - x) - __fdividef(e2[i - 1], q);
        if (fabsf(q) < pivmin) q = -pivmin;
        c += q < 0.0f;
    }
    return c;
}

// FP32 multisection, one warp per eigenvalue j: each round the 32 lanes
// count at 32 equally spaced points of the bracket and the bracket shrinks
// to the subinterval where the count passes j (five rounds: 2^-25 of the
// Gershgorin width).  The FP32 counts are those of a matrix within a few
// FP32 units of T, so the bracket is widened before the FP64 stage checks it.
__global__ void __launch_bounds__(256) multisect_f32_kernel(const float *__restrict__ d, const float *__restrict__ e2,
                                                            int n, const double *__restrict__ bounds,
                                                            double *__restrict__ blo, double *__restrict__ bhi)
{
    const int lane = threadIdx.x & 31;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= n) return;  // whole warps leave together
    float lo = (float)bounds[0], hi = (float)bounds[1];
    const float pivmin = (float)bounds[3];
    for (int round = 0; round < 5; ++round) {
        const float h = (hi - lo) * (1.0f / 32.0f);
        const float x = (lane == 31) ? hi : lo + h * (float)(lane + 1);
        const int c = sturm_count_f32(d, e2, n, x, pivmin);
        const unsigned above = __ballot_sync(0xffffffffu, c > j);
        const int first = above ? __ffs(above) - 1 : 31;
        const float xf = __shfl_sync(0xffffffffu, x, first);
        const float xp = __shfl_sync(0xffffffffu, x, first > 0 ? first - 1 : 0);
        const float nlo = first > 0 ? xp : lo, nhi = xf;
        if (!(nlo < nhi)) break;
        lo = nlo;
        hi = nhi;
    }
    if (lane == 0) {
        blo[j] = lo;
        bhi[j] = hi;
    }
}

// FP64 multisection of eigenvalue j from the FP32 bracket, widened by a
// few FP32 units of the spectrum's scale; if the FP64 counts at its ends do
// not enclose j, from the Gershgorin interval instead.  K lanes per
// eigenvalue (K divides 32): each round they count at the K interior points
// that cut the bracket into K + 1 equal parts, and the bracket shrinks to the
// part where the count passes j (K = 1 is bisection).  Stops at a bracket of
// width reltol |lam| + 2u ||T|| (plus the pivot floor).  A count costs
// three FP64 instructions a step; the launcher picks the K that fills the
// FP64 units of every SM sub-partition with the fewest rounds.  Once the
// bracket holds eigenvalue j alone, the points of a round go around the
// regula falsi estimate from the determinants at the bracket's ends (a
// by-product of the counts) instead of cutting it into equal parts.
static constexpr int kBisectThreads = 64;  // two warps per CTA: the warps spread over every SM

template <int K>
__global__ void __launch_bounds__(kBisectThreads) bisect_f64_kernel(const double *__restrict__ d, const double *__restrict__ e2,
                                                         int n, const double *__restrict__ bounds,
                                                         const double *__restrict__ blo,
                                                         const double *__restrict__ bhi, double reltol,
                                                         double *__restrict__ lam)
{
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = gt / K, l = gt % K;
    const int base = (threadIdx.x & 31) & ~(K - 1);  // first lane of this eigenvalue's group
    const bool valid = j < n;                         // the rest of the last warp still shuffles
    const double gl = bounds[0], gu = bounds[1], pivmin = bounds[2];
    const double widen = 16.0 * 5.9604644775390625e-08 * fmax(fabs(gl), fabs(gu)) + pivmin;
    double lo = gl, hi = gu;
    if (valid) {
        lo = fmax(gl, blo[j] - widen);
        hi = fmin(gu, bhi[j] + widen);
    }
    // counts and determinants at both ends (two lanes at once where K >= 2)
    int c0 = 0, c1 = 0, e0 = 0, e1 = 0;
    double m0 = 1.0, m1 = 1.0;
    if (valid && (lo < hi)) {
        if (K == 1) {
            c0 = sturm_count(d, e2, n, lo, &m0, &e0);
            c1 = sturm_count(d, e2, n, hi, &m1, &e1);
        } else if (l < 2) {
            c0 = sturm_count(d, e2, n, l == 0 ? lo : hi, &m0, &e0);
        }
    }
    if (K > 1) {
        const int a = __shfl_sync(0xffffffffu, c0, base), ae = __shfl_sync(0xffffffffu, e0, base);
        const double am = __shfl_sync(0xffffffffu, m0, base);
        c1 = __shfl_sync(0xffffffffu, c0, base + 1);
        e1 = __shfl_sync(0xffffffffu, e0, base + 1);
        m1 = __shfl_sync(0xffffffffu, m0, base + 1);
        c0 = a; e0 = ae; m0 = am;
    }
    // bracket [lo, hi] with count(lo) = clo <= j < chi = count(hi) and, where
    // known (hlo, hhi), det(T - x I) at its ends as mantissa and exponent
    int clo = c0, chi = c1, flx = e0, fhx = e1;
    double flm = m0, fhm = m1;
    bool hlo = true, hhi = true;
    if (!(lo < hi) || c0 > j || c1 <= j) {
        lo = gl;
        hi = gu;
        clo = 0;
        chi = n;
        hlo = hhi = false;
    }
    const double atol = 2.0 * 1.1102230246251565e-16 * fmax(fabs(gl), fabs(gu)) + pivmin;
    const double step = 1.0 / (double)(K + 1);
    double xs_prev = 0.0;
    bool have_prev = false, plain_next = false;
    for (int it = 0; it < 160; ++it) {
        const double h = (hi - lo) * step;
        const bool conv = !valid || !(lo + h > lo && lo + h * (double)K < hi) ||
                          hi - lo <= reltol * fmax(fabs(lo), fabs(hi)) + atol;
        if (__all_sync(0xffffffffu, conv)) break;
        // points: K equal parts of the bracket, or -- once the bracket holds
        // eigenvalue j alone and its ends' determinants are known -- points at
        // +-delta/2, +-2 delta, +-8 delta, ... around the regula falsi estimate
        // x* (the root of the line through the two determinants), delta the
        // change of x* since the last round (a secant-type step converges
        // superlinearly); a round that fails to halve the bracket is followed
        // by a plain one.  The counts decide the new bracket either way.
        const bool sec = K >= 2 && hlo && hhi && clo == j && chi == j + 1 && !plain_next;
        double x = lo + h * (double)(l + 1);
        double xs = 0.0;
        if (sec) {
            const int dx = max(-1000, min(1000, fhx - flx));
            const double q = (fhm / flm) * __longlong_as_double((long long)(dx + 1023) << 52);  // f(hi) / f(lo)
            double t = 1.0 / (1.0 - q);
            if (!(t > 0.0 && t < 1.0)) t = 0.5;
            xs = lo + (hi - lo) * t;
            double delta = (hi - lo) * 0.0625;
            if (have_prev) delta = fmin(delta, fmax(fabs(xs - xs_prev), 0.25 * (reltol * fabs(xs) + atol)));
            const int half = K / 2, k = l < half ? half - 1 - l : l - half;
            const double off = delta * 0.5 * (double)(1u << (2 * k));  // delta 2^(2k-1)
            x = fmin(hi, fmax(lo, l < half ? xs - off : xs + off));
        }
        double fm = 1.0;
        int fe = 0;
        const int c = conv ? 0 : sturm_count(d, e2, n, x, &fm, &fe);
        unsigned above = __ballot_sync(0xffffffffu, c > j);
        above = (K == 32) ? above : (above >> base) & ((1u << K) - 1u);
        const int first = above ? __ffs(above) - 1 : K;  // part (x_{first-1}, x_first]
        const int sl = base + max(first - 1, 0), sh = base + min(first, K - 1);
        const double xl = __shfl_sync(0xffffffffu, x, sl), xh = __shfl_sync(0xffffffffu, x, sh);
        const int cl = __shfl_sync(0xffffffffu, c, sl), ch = __shfl_sync(0xffffffffu, c, sh);
        const double ml = __shfl_sync(0xffffffffu, fm, sl), mh = __shfl_sync(0xffffffffu, fm, sh);
        const int el = __shfl_sync(0xffffffffu, fe, sl), eh = __shfl_sync(0xffffffffu, fe, sh);
        if (!conv) {
            const double w0 = hi - lo;
            if (first > 0) { lo = xl; clo = cl; flm = ml; flx = el; hlo = true; }
            if (first < K) { hi = xh; chi = ch; fhm = mh; fhx = eh; hhi = true; }
            if (sec) {
                plain_next = hi - lo > 0.5 * w0;
                xs_prev = xs;
                have_prev = true;
            } else {
                plain_next = false;
            }
        }
    }
    if (valid && l == 0) lam[j] = 0.5 * (lo + hi);
}

// lanes per eigenvalue for bisect_f64_kernel.  Each FP64 instruction of a
// warp occupies its SM sub-partition's FP64 unit for tens of cycles (GB300
// has few FP64 units), so a round of counts costs about the number of warps
// a sub-partition holds, ceil(n K / 32 / (4 SMs)), and shrinks the bracket
// by K + 1: K minimises that over log2(K + 1).
static int bisect_lanes(int n)
{
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int best = 1;
    double best_cost = 1e300;
    for (int K = 1; K <= 32; K *= 2) {
        const double per_part = std::ceil(std::ceil((double)n * K / 32.0) / (4.0 * sms));
        const double cost = per_part / std::log2((double)K + 1.0);
        if (cost < best_cost * 0.999) { best_cost = cost; best = K; }
    }
    return best;
}

// Twisted factorisation eigenvectors for eigenvalues [j0, j0 + cnt) from the
// minors of T - lam I, P_i = det((T - lam I)(0:i, 0:i)) (P_{-1} = 1) and
// Q_i = det((T - lam I)(i:n, i:n)) (Q_n = 1), both by the division-free
// recurrence of sturm_count and stored rescaled, with one power-of-two
// exponent per 8 entries.  The pivots of T - lam I = L D+ L^T = U D- U^T are
// D+_i = P_i / P_{i-1} and D-_i = Q_i / Q_{i+1}, and
//   gamma_i = D+_i + D-_i - (d_i - lam) = det(T - lam I) / (P_{i-1} Q_{i+1})
// (the reciprocal of the i-th diagonal entry of (T - lam I)^-1), so the
// twist index r, where |gamma| is smallest, is where |P_{i-1} Q_{i+1}| is
// largest (compared by binary exponent and leading bits; the first such i).
// The vector z_r = 1, z_i = -(e_i / D+_i) z_{i+1} above r, z_{i+1} =
// -(e_i / D-_{i+1}) z_i below r telescopes to
//   z_i = P_{i-1} prod_{k=i}^{r-1} (-e_k) / P_{r-1}  (i < r),
//   z_i = Q_{i+1} prod_{k=r}^{i-1} (-e_k) / Q_{r+1}  (i > r),
// formed from the prefix products F_i = prod_{k<i} (-e_k) and G_i = 1 / F_i
// (tw_prefix_kernel; both restart after a zero e, and a component in
// another block of T than r is zero), so every component is two
// multiplications and an exponent shift, independent of the others --
// instead of a division chain along the vector.  A CTA of 128 threads takes
// 32 eigenvalues: warps 0 and 1 the forward and backward minors, then all
// four warps a quarter of the rows each for the twist and the vector.
// P, Q: [i * cnt + (j - j0)]; SP, SQ: [k * cnt + (j - j0)], the exponent of
// entries 8k-7 .. 8k (k >= 1; entry 0 in k = 0) of P, and of Q counted from
// the bottom (entry n-1-i); ZT row j (ld n) receives eigenvector j.
static constexpr int kTwBlk = 8;
static constexpr int kTwThreads = 128;

static int tw_scale_rows(int n) { return (n + kTwBlk - 2) / kTwBlk + 2; }

// v with |v| in [1, 2) and x += its binary exponent (v finite, nonzero)
__device__ __forceinline__ void mant_norm(double &v, int &x)
{
    const long long b = __double_as_longlong(v);
    x += (int)((b >> 52) & 0x7FF) - 1023;
    v = __longlong_as_double((b & (long long)0x800FFFFFFFFFFFFFull) | (1023ll << 52));
}

// v 2^k by the exponent field (integer operations); 0 below the normal range
__device__ __forceinline__ double shift_exp(double v, int k)
{
    const long long b = __double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7FF);
    if (ex == 0) return v;
    const int ne = ex + k;
    if (ne <= 0) return __longlong_as_double(b & (long long)0x8000000000000000ull);
    return __longlong_as_double((b & (long long)0x800FFFFFFFFFFFFFull) | ((long long)min(ne, 2046) << 52));
}

// F_i = prod_{k = blk_i}^{i-1} (-e_k) and G_i = 1 / F_i as (mantissa in
// [1, 2), exponent), blk_i the first row of i's block of T (after the last
// zero e above i).  One CTA: a thread's rows, a segmented scan of the
// threads' products, then the rows again from the thread's prefix.
static constexpr int kPfxThreads = 1024;
__global__ void __launch_bounds__(kPfxThreads) tw_prefix_kernel(const double *__restrict__ e, int n,
                                                                double *__restrict__ Fm, int *__restrict__ Fx,
                                                                double *__restrict__ Gm, int *__restrict__ Gx,
                                                                int *__restrict__ blk)
{
    __shared__ double sm[kPfxThreads];
    __shared__ int sx[kPfxThreads], sr[kPfxThreads], sb[kPfxThreads];
    const int t = threadIdx.x, L = (n + kPfxThreads - 1) / kPfxThreads;
    const int i0 = min(n, t * L), i1 = min(n, i0 + L);
    double m = 1.0;
    int x = 0, rs = 0, b = 0;
    for (int i = i0; i < i1; ++i) {
        if (i == 0 || e[i - 1] == 0.0) { m = 1.0; x = 0; rs = 1; b = i; }
        else { m *= -e[i - 1]; mant_norm(m, x); }
    }
    sm[t] = m; sx[t] = x; sr[t] = rs; sb[t] = b;
    __syncthreads();
    for (int off = 1; off < kPfxThreads; off <<= 1) {
        const bool has = t >= off;
        const double am = has ? sm[t - off] : 1.0;
        const int ax = has ? sx[t - off] : 0, ar = has ? sr[t - off] : 0, ab = has ? sb[t - off] : 0;
        double bm = sm[t];
        int bx = sx[t], br = sr[t], bb = sb[t];
        __syncthreads();
        if (has && !br) { bm *= am; bx += ax; mant_norm(bm, bx); br = ar; bb = ab; }
        sm[t] = bm; sx[t] = bx; sr[t] = br; sb[t] = bb;
        __syncthreads();
    }
    // the rows again from the product of the threads before this one
    m = t > 0 ? sm[t - 1] : 1.0;
    x = t > 0 ? sx[t - 1] : 0;
    b = t > 0 ? sb[t - 1] : 0;
    for (int i = i0; i < i1; ++i) {
        if (i == 0 || e[i - 1] == 0.0) { m = 1.0; x = 0; b = i; }
        else { m *= -e[i - 1]; mant_norm(m, x); }
        Fm[i] = m; Fx[i] = x; blk[i] = b;
        double g = 1.0 / m;
        int gx = -x;
        mant_norm(g, gx);
        Gm[i] = g; Gx[i] = gx;
    }
}

// one minors sweep, entry m = 0 .. n-1 from (dd(m), ee(m)) = (d - lam, e^2
// coupling m to m-1), stored by put(m, value) with the running exponent in
// sc(k) for the entries of block k
template <class DF, class EF, class PF, class SF>
__device__ __forceinline__ void minors_sweep(int n, DF dd, EF ee, PF put, SF sc)
{
    double pm = 1.0, p = minor_fix(dd(0), 1.0);
    int ex = 0;
    put(0, p);
    sc(0, 0);
    if (n > 1) sc(1, 0);
    for (int m = 1; m < n; m += kTwBlk) {
        const int hi = min(n, m + kTwBlk);
        double dv[kTwBlk], ev[kTwBlk];
#pragma unroll
        for (int u = 0; u < kTwBlk; ++u) {
            dv[u] = m + u < hi ? dd(m + u) : 0.0;
            ev[u] = m + u < hi ? ee(m + u) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kTwBlk; ++u) {
            if (m + u < hi) {
                const double pn = minor_fix(fma(dv[u], p, -ev[u] * pm), p);
                pm = p;
                p = pn;
                put(m + u, p);
            }
        }
        if (hi < n) {
            const unsigned long long a = (unsigned long long)__double_as_longlong(p) & 0x7FFFFFFFFFFFFFFFull;
            const unsigned long long b = (unsigned long long)__double_as_longlong(pm) & 0x7FFFFFFFFFFFFFFFull;
            const int E = max(-1000, min(1000, (int)((a > b ? a : b) >> 52) - 1023));
            const double s2 = __longlong_as_double((long long)(1023 - E) << 52);
            p *= s2;
            pm *= s2;
            ex += E;
            sc((hi + kTwBlk - 1) / kTwBlk, ex);
        }
    }
}

// binary exponent and leading bits of |v| (v finite, nonzero): |v| in
// [2^x, 2^(x+1)), f = |v| / 2^x in [1, 2)
__device__ __forceinline__ void split_exp(double v, int &x, float &f)
{
    const long long b = __double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFll;
    x = (int)(b >> 52) - 1023;
    f = __int_as_float(0x3F800000 | (int)((b >> 29) & 0x7FFFFF));  // leading 23 bits, integer ops only
}

__global__ void __launch_bounds__(kTwThreads) twisted_kernel(const double *__restrict__ d, const double *__restrict__ e2,
                                                             int n, const double *__restrict__ lam, int j0, int cnt,
                                                             double *__restrict__ P, double *__restrict__ Q,
                                                             int *__restrict__ SP, int *__restrict__ SQ,
                                                             const double *__restrict__ Fm, const int *__restrict__ Fx,
                                                             const double *__restrict__ Gm, const int *__restrict__ Gx,
                                                             const int *__restrict__ blk, double *__restrict__ ZT)
{
    constexpr int W = kTwThreads / 32;
    __shared__ int s_r[W][32], s_x[W][32];
    __shared__ float s_f[W][32];
    __shared__ double s_nrm[W][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int t = blockIdx.x * 32 + lane;
    const bool valid = t < cnt;
    const int j = j0 + t;
    const double x = valid ? lam[j] : 0.0;
    const size_t ld = (size_t)cnt;
    // minors: warp 0 forward (entry m = row m), warp 1 backward (entry m = row n-1-m)
    if (valid && w == 0) {
        minors_sweep(n, [&](int m) { return d[m] - x; }, [&](int m) { return e2[m - 1]; },
                     [&](int m, double v) { P[(size_t)m * ld + t] = v; },
                     [&](int k, int v) { SP[(size_t)k * ld + t] = v; });
    } else if (valid && w == 1) {
        minors_sweep(n, [&](int m) { return d[n - 1 - m] - x; }, [&](int m) { return e2[n - 1 - m]; },
                     [&](int m, double v) { Q[(size_t)(n - 1 - m) * ld + t] = v; },
                     [&](int k, int v) { SQ[(size_t)k * ld + t] = v; });
    }
    __syncthreads();
    // the stored minor of row i with its exponent: P (i = -1: 1) and Q (i = n: 1)
    auto getP = [&](int i, double &v, int &ex) {
        if (i < 0) { v = 1.0; ex = 0; return; }
        v = P[(size_t)i * ld + t];
        ex = SP[(size_t)((i + kTwBlk - 1) / kTwBlk) * ld + t];
    };
    auto getQ = [&](int i, double &v, int &ex) {
        if (i >= n) { v = 1.0; ex = 0; return; }
        v = Q[(size_t)i * ld + t];
        ex = SQ[(size_t)((n - 1 - i + kTwBlk - 1) / kTwBlk) * ld + t];
    };
    // twist index: the first i with the largest |P_{i-1} Q_{i+1}|, each warp
    // over a quarter of the rows
    const int q0 = (int)((int64_t)n * w / W), q1 = (int)((int64_t)n * (w + 1) / W);
    {
        int r = -1, bx = 0;
        float bf = 0.f;
        if (valid) {
            for (int i = q0; i < q1; ++i) {
                double pv, qv;
                int pe, qe, xp = 0, xq = 0;
                float fp = 1.f, fq = 1.f;
                getP(i - 1, pv, pe);
                getQ(i + 1, qv, qe);
                split_exp(pv, xp, fp);
                split_exp(qv, xq, fq);
                int xe = xp + pe + xq + qe;
                float f = fp * fq;
                if (f >= 2.f) { f *= 0.5f; ++xe; }
                if (r < 0 || xe > bx || (xe == bx && f > bf)) { r = i; bx = xe; bf = f; }
            }
        }
        s_r[w][lane] = r;
        s_x[w][lane] = bx;
        s_f[w][lane] = bf;
        __syncthreads();
    }
    int r = -1;
    {
        int bx = 0;
        float bf = 0.f;
        for (int q = 0; q < W; ++q) {
            const int rq = s_r[q][lane];
            if (rq >= 0 && (r < 0 || s_x[q][lane] > bx || (s_x[q][lane] == bx && s_f[q][lane] > bf))) {
                r = rq; bx = s_x[q][lane]; bf = s_f[q][lane];
            }
        }
    }
    // z_i = P_{i-1} G_i F_r / P_{r-1} above r, Q_{i+1} F_i G_r / Q_{r+1} below
    double nrm2 = 0.0;
    if (valid && r >= 0) {
        double pr, qr;
        int per, qer;
        getP(r - 1, pr, per);
        getQ(r + 1, qr, qer);
        const double cu = Fm[r] / pr, cd = Gm[r] / qr;
        const int xu = Fx[r] - per, xd = Gx[r] - qer;
        const int br = blk[r];
        for (int i = q0; i < q1; ++i) {
            double z = 1.0;
            if (i < r) {
                double pv;
                int pe;
                getP(i - 1, pv, pe);
                z = blk[i] == br ? shift_exp(pv * Gm[i] * cu, pe + Gx[i] + xu) : 0.0;
            } else if (i > r) {
                double qv;
                int qe;
                getQ(i + 1, qv, qe);
                z = blk[i] == br ? shift_exp(qv * Fm[i] * cd, qe + Fx[i] + xd) : 0.0;
            }
            ZT[j + (size_t)i * n] = z;
            nrm2 = fma(z, z, nrm2);
        }
    }
    s_nrm[w][lane] = nrm2;
    __syncthreads();
    if (valid && r >= 0) {
        double tot = 0.0;
        for (int q = 0; q < W; ++q) tot += s_nrm[q][lane];
        const double inv = 1.0 / sqrt(tot);
        for (int i = q0; i < q1; ++i) ZT[j + (size_t)i * n] *= inv;
    }
}

// ---------------------------------------------------------------------------
// Eigenvalue clusters.  Twisted factorisations of eigenvalues that lie closer
// together than the eigenvalues' own accuracy give (nearly) the same vector.
// Eigenvalue j is a cluster member when
//   lam_j - lam_{j-1} <= rtol max(|lam_j|, |lam_{j-1}|) + atol ||T||;
// the members of one cluster are consecutive, and a member's vector is
// recomputed as the part of a pseudo-random vector orthogonal to every
// eigenvector outside its cluster and to the members of its cluster done
// before it, by classical Gram-Schmidt in two passes, then normalised: for a
// symmetric T the cluster's invariant subspace is the orthogonal complement
// of the other eigenvectors (other clusters' vectors count with their
// twisted approximations).  ZT row k = eigenvector k (ZT[k + i n]); mask[k]
// = 0 for the members of the cluster in hand not yet done.
// ---------------------------------------------------------------------------
static constexpr int kClP = 8;  // row chunks of the projection products

// clusters as member ranges [first[c], last[c]]; mask = 1 everywhere
static constexpr int kClScan = 1024;
__global__ void __launch_bounds__(kClScan) cluster_scan_kernel(const double *__restrict__ lam, int n, double rtol,
                                                              double atol_rel, const double *__restrict__ bounds,
                                                              int *__restrict__ first, int *__restrict__ last,
                                                              int *__restrict__ ncl, int *__restrict__ mask)
{
    // one CTA: each thread a chunk of j; member j (j >= 1) when it lies
    // within the tolerance of j - 1; the starts are numbered by a block scan
    __shared__ int s_cnt[kClScan];
    const double atol = atol_rel * fmax(fabs(bounds[0]), fabs(bounds[1]));
    auto member = [&](int j) {
        return j >= 1 && j < n && lam[j] - lam[j - 1] <= rtol * fmax(fabs(lam[j]), fabs(lam[j - 1])) + atol;
    };
    const int t = threadIdx.x, L = (n + kClScan - 1) / kClScan, j0 = min(n, t * L), j1 = min(n, j0 + L);
    int cnt = 0;
    for (int j = j0; j < j1; ++j) {
        mask[j] = 1;
        cnt += member(j) && !member(j - 1);
    }
    s_cnt[t] = cnt;
    __syncthreads();
    for (int off = 1; off < kClScan; off <<= 1) {
        const int v = t >= off ? s_cnt[t - off] : 0;
        __syncthreads();
        s_cnt[t] += v;
        __syncthreads();
    }
    int c = s_cnt[t] - cnt;  // clusters started before this chunk
    for (int j = j0; j < j1; ++j) {
        if (!member(j)) continue;
        if (!member(j - 1)) first[c++] = j;
        if (!member(j + 1)) last[c - 1] = j;
    }
    if (t == kClScan - 1) *ncl = s_cnt[t];
}

// x_i uniform in [-1, 1): a counter-based hash (SplitMix64 finaliser) of (j, i)
__global__ void cluster_start_kernel(double *__restrict__ x, int n, int j)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t z = ((uint64_t)(uint32_t)j << 32 | (uint32_t)i) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// part[p n + k] = sum over the p-th chunk of i of ZT[k + i n] x_i
__global__ void __launch_bounds__(256) cluster_dots_kernel(const double *__restrict__ ZT, const double *__restrict__ x,
                                                           int n, double *__restrict__ part)
{
    __shared__ double xs[256];
    const int k = blockIdx.x * 256 + threadIdx.x;
    const int ilen = (n + kClP - 1) / kClP, i0 = blockIdx.y * ilen, i1 = min(n, i0 + ilen);
    double acc = 0.0;
    for (int t0 = i0; t0 < i1; t0 += 256) {
        __syncthreads();
        if (t0 + threadIdx.x < i1) xs[threadIdx.x] = x[t0 + threadIdx.x];
        __syncthreads();
        const int tn = min(256, i1 - t0);
        if (k < n)
            for (int t = 0; t < tn; ++t) acc = fma(ZT[k + (int64_t)(t0 + t) * n], xs[t], acc);
    }
    if (k < n) part[(int64_t)blockIdx.y * n + k] = acc;
}

// c_k = mask_k sum_p part[p n + k]
__global__ void cluster_csum_kernel(const double *__restrict__ part, const int *__restrict__ mask, int n,
                                    double *__restrict__ c)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double acc = 0.0;
    for (int p = 0; p < kClP; ++p) acc += part[(int64_t)p * n + k];
    c[k] = mask[k] ? acc : 0.0;
}

// x_i -= sum_k c_k ZT[k + i n], one warp per i
__global__ void __launch_bounds__(256) cluster_sub_kernel(const double *__restrict__ ZT, const double *__restrict__ c,
                                                          int n, double *__restrict__ x)
{
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;  // whole warps
    double acc = 0.0;
    for (int k = lane; k < n; k += 32) acc = fma(c[k], ZT[k + (int64_t)i * n], acc);
    acc = warp_sum(acc);
    if (lane == 0) x[i] -= acc;
}

// ZT row j = x / ||x||, mask[j] = 1 (one CTA)
__global__ void __launch_bounds__(256) cluster_store_kernel(double *__restrict__ ZT, int *__restrict__ mask,
                                                            const double *__restrict__ x, int n, int j)
{
    __shared__ double red[8];
    double a = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) a = fma(x[i], x[i], a);
    a = warp_sum(a);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += red[q];
    const double inv = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
    for (int i = threadIdx.x; i < n; i += 256) ZT[j + (int64_t)i * n] = x[i] * inv;
    if (threadIdx.x == 0) mask[j] = 1;
}

// the members' vectors (clusters of size >= 2); scratch: >= (kClP + 2) n doubles
// + 3 n + 1 ints
static cudaError_t fix_clusters(const double *lam, const double *bounds, int n, double rtol, double atol_rel,
                                double *ZT, double *scratch, cudaStream_t s)
{
    double *part = scratch, *x = part + (size_t)kClP * n, *c = x + n;
    int *first = (int *)(c + n), *last = first + n, *mask = last + n, *ncl = mask + n;
    cluster_scan_kernel<<<1, kClScan, 0, s>>>(lam, n, rtol, atol_rel, bounds, first, last, ncl, mask); count_launch();
    int m = 0;
    cudaError_t err = cudaMemcpyAsync(&m, ncl, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (!err) err = cudaStreamSynchronize(s);
    if (err || m == 0) return err;
    std::vector<int> f(m), l(m);
    if ((err = cudaMemcpyAsync(f.data(), first, sizeof(int) * m, cudaMemcpyDeviceToHost, s)) ||
        (err = cudaMemcpyAsync(l.data(), last, sizeof(int) * m, cudaMemcpyDeviceToHost, s)))
        return err;
    if ((err = cudaStreamSynchronize(s))) return err;
    const int g1 = (int)cdiv_i(n, 256);
    for (int q = 0; q < m; ++q) {
        if ((err = cudaMemsetAsync(mask + f[q], 0, sizeof(int) * (size_t)(l[q] - f[q] + 1), s))) return err;
        for (int j = f[q]; j <= l[q]; ++j) {
            cluster_start_kernel<<<g1, 256, 0, s>>>(x, n, j); count_launch();
            for (int pass = 0; pass < 2; ++pass) {
                cluster_dots_kernel<<<dim3(g1, kClP), 256, 0, s>>>(ZT, x, n, part); count_launch();
                cluster_csum_kernel<<<g1, 256, 0, s>>>(part, mask, n, c); count_launch();
                cluster_sub_kernel<<<(int)cdiv_i((int64_t)n * 32, 256), 256, 0, s>>>(ZT, c, n, x); count_launch();
            }
            cluster_store_kernel<<<1, 256, 0, s>>>(ZT, mask, x, n, j); count_launch();
        }
    }
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_tridiag_eig(const R *A, int n, int ld, double *lam, double *ZT,
                               double *scratch, int chunk, cudaStream_t s)
{
    double *d = scratch, *e = d + n, *e2 = e + n, *bounds = e2 + n;
    double *Dp = bounds + 8;
    double *Dm = Dp + (size_t)n * chunk;
    // the bisection stage's scratch lives in Dp (free until the vectors)
    double *blo = Dp, *bhi = Dp + n;
    float *df = (float *)(Dp + 2 * (size_t)n), *e2f = df + n;
    tri_extract_kernel<R><<<1, 256, 0, s>>>(A, n, ld, d, e, e2, bounds, df, e2f); count_launch();
    multisect_f32_kernel<<<(int)cdiv_i((int64_t)n * 32, 256), 256, 0, s>>>(df, e2f, n, bounds, blo, bhi); count_launch();
    // The FP32 factorisation needs eigenvectors orthogonal to FP32 working
    // precision only: |dlam| / gap well below 2^-24 takes eigenvalues to
    // about 1e-10 relative for any gap above 1e-3 |lam|.  The FP64 method
    // takes them to FP64 precision.
    const double reltol = sizeof(R) == sizeof(float) ? 1e-10 : 2.0 * 1.1102230246251565e-16;
    {
        const int K = bisect_lanes(n);
        const int grid = (int)cdiv_i((int64_t)n * K, kBisectThreads);
        switch (K) {
        case 1: bisect_f64_kernel<1><<<grid, kBisectThreads, 0, s>>>(d, e2, n, bounds, blo, bhi, reltol, lam); break;
        case 2: bisect_f64_kernel<2><<<grid, kBisectThreads, 0, s>>>(d, e2, n, bounds, blo, bhi, reltol, lam); break;
        case 4: bisect_f64_kernel<4><<<grid, kBisectThreads, 0, s>>>(d, e2, n, bounds, blo, bhi, reltol, lam); break;
        case 8: bisect_f64_kernel<8><<<grid, kBisectThreads, 0, s>>>(d, e2, n, bounds, blo, bhi, reltol, lam); break;
        case 16: bisect_f64_kernel<16><<<grid, kBisectThreads, 0, s>>>(d, e2, n, bounds, blo, bhi, reltol, lam); break;
        default: bisect_f64_kernel<32><<<grid, kBisectThreads, 0, s>>>(d, e2, n, bounds, blo, bhi, reltol, lam); break;
        }
        count_launch();
    }
    {
        // past the region fix_clusters may spill into: the minors' exponents,
        // then the prefix products of the off-diagonal
        const int rows = tw_scale_rows(n);
        int *SP = (int *)(Dm + (size_t)n * chunk + 4 * (size_t)n + 8);
        int *SQ = SP + (size_t)rows * chunk;
        // SP is 8-byte aligned and SP + 2 rows chunk ints is too: the doubles
        // follow directly
        double *Fm = (double *)(SQ + (size_t)rows * chunk), *Gm = Fm + n;
        int *Fx = (int *)(Gm + n), *Gx = Fx + n, *blkv = Gx + n;
        tw_prefix_kernel<<<1, kPfxThreads, 0, s>>>(e, n, Fm, Fx, Gm, Gx, blkv); count_launch();
        for (int j0 = 0; j0 < n; j0 += chunk) {
            int cnt = std::min(chunk, n - j0);
            twisted_kernel<<<(int)cdiv_i(cnt, 32), kTwThreads, 0, s>>>(d, e2, n, lam, j0, cnt, Dp, Dm, SP, SQ, Fm, Fx,
                                                                        Gm, Gx, blkv, ZT);
            count_launch();
        }
    }
    // clusters: eigenvalues closer than their accuracy allows (FP32 method:
    // 1e-10 relative, vectors needed to ~1e-5; FP64 method: 2u, to ~1e-8,
    // which the Newton-Schulz step then squares)
    {
        const bool f32 = sizeof(R) == sizeof(float);
        cudaError_t err = fix_clusters(lam, bounds, n, f32 ? 1e-5 : 1e-8, f32 ? 4.4e-11 : 2.2e-13, ZT, Dp, s);
        if (err) return err;
    }
    return cudaGetLastError();
}

template cudaError_t launch_tridiag_eig<float>(const float *, int, int, double *, double *, double *, int, cudaStream_t);
template cudaError_t launch_tridiag_eig<double>(const double *, int, int, double *, double *, double *, int, cudaStream_t);

// B = A^T for a square n x n matrix (32 x 32 tiles through shared memory)
template <class R>
__global__ void transpose_kernel(const R *__restrict__ A, R *__restrict__ B, int n)
{
    __shared__ R t[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int r = bx + threadIdx.x, c = by + j;
        if (r < n && c < n) t[j][threadIdx.x] = A[r + (int64_t)c * n];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int r = by + threadIdx.x, c = bx + j;
        if (r < n && c < n) B[r + (int64_t)c * n] = t[threadIdx.x][j];
    }
}

// small elementwise helpers
// ZT <- 1.5 ZT - 0.5 P  (one Newton-Schulz step towards orthogonality:
// Z <- Z (3 I - Z^T Z) / 2, written for Z^T)
__global__ void newton_schulz_combine_kernel(double *__restrict__ ZT, const double *__restrict__ P, int64_t count)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
        ZT[t] = fma(-0.5, P[t], 1.5 * ZT[t]);
}

// Z(i, j) = R(ZT(j, i)): ZT holds Z^T (row j = eigenvector j), n x n, ld n
template <class R>
__global__ void cast_transpose_kernel(const double *__restrict__ ZT, R *__restrict__ Z, int n)
{
    __shared__ double t[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int r = bx + threadIdx.x, c = by + j;
        if (r < n && c < n) t[j][threadIdx.x] = ZT[r + (int64_t)c * n];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int r = by + threadIdx.x, c = bx + j;
        if (r < n && c < n) Z[r + (int64_t)c * n] = (R)t[threadIdx.x][j];
    }
}

// s_i = sqrt(lam_i) (lam rounded to R first); status 2 for lam_i <= 0
template <class R>
__global__ void sqrt_eig_kernel(const double *__restrict__ lam, R *__restrict__ lamr, R *__restrict__ s,
                                int n, int *status)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        R l = (R)lam[i];
        lamr[i] = l;
        if (!(l > R(0))) { atomicExch(status, 2); s[i] = R(1); }
        else s[i] = sqrt(l);
    }
}

// W(:, j) = V(:, j) * s_j
template <class R>
__global__ void scale_cols_kernel(const R *__restrict__ V, const R *__restrict__ s, R *__restrict__ W, int n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)n * n; t += (int64_t)gridDim.x * blockDim.x)
        W[t] = V[t] * s[t / n];
}

static int grid1(int64_t count)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv_i(count, 256), 152 * 8));
}

}  // namespace sqm

using namespace sqm;

// ---------------------------------------------------------------------------
// spectral decomposition driver: As (real R, n x n) -> V (R), lam (R), s (R)
// ---------------------------------------------------------------------------
namespace {

template <class R>
struct SpdWork {
    R *As, *V, *lamr, *s, *W, *Y, *Qh, *vecws, *betas, *btws;
    void *digits;    // BF16 digit slices of X for the split residual (FP32 method)
    int *rho;        // their row exponents
    double *lam, *ZT, *eigscratch;
    float *Rhat;
    double *xsave;   // FP64 copy of X for the adjoint
    double *dscal;   // [0] norm, [1] rnorm, [2..] partials
    int *iscal;      // [0] e, [1] status
    int chunk;
};

template <class R>
size_t spd_bytes(int64_t n, int chunk)
{
    size_t nn = (size_t)n * n;
    int64_t nb = (n + 63) / 64;
    size_t np = (size_t)std::max<int64_t>(nb * nb, 2048) + 8;
    return Carve::round(np * sizeof(double)) + 256 + 3 * Carve::round(nn * sizeof(R)) +
           Carve::round(nn * sizeof(float)) + Carve::round(nn * sizeof(double)) +
           Carve::round((2 * (size_t)n * chunk + 3 * n + 8 + (size_t)tw_scale_rows((int)n) * chunk + 4 * (size_t)n + 8) *
                        sizeof(double)) +
           Carve::round(n * sizeof(double)) + 2 * Carve::round(n * sizeof(R)) +
           Carve::round((4 * n + 16) * sizeof(R)) + Carve::round((n + 8) * sizeof(R)) +
           Carve::round(((size_t)2 * kBackNb * kBackNb + (size_t)2 * kBackNb * n) * sizeof(R)) +
           Carve::round((size_t)(4 * n + 8) * sizeof(double)) +
           (sizeof(R) == sizeof(float) ? Carve::round(split_digit_elems((int)n) * 2) + Carve::round(n * sizeof(int)) : 0) +
           8192;
}

template <class R>
int spd_carve(sqrtm_handle_t h, int64_t n, SpdWork<R> *w)
{
    int chunk = (int)std::min<int64_t>(n, 4096);  // eigenvectors per twisted_kernel launch
    size_t nn = (size_t)n * n;
    // factors V, lamr, s persist for the adjoint / reuse
    size_t fbytes = Carve::round(nn * sizeof(R)) + 2 * Carve::round(n * sizeof(R)) +
                    Carve::round(nn * sizeof(double)) + 1024;
    if (ensure(h->fact, fbytes, h) || ensure(h->ws, spd_bytes<R>(n, chunk), h)) return 7;
    Carve cf(h->fact.p);
    w->V = cf.take<R>(nn);
    w->lamr = cf.take<R>(n);
    w->s = cf.take<R>(n);
    w->xsave = cf.take<double>(nn);
    Carve c(h->ws.p);
    int64_t nb = (n + 63) / 64;
    size_t np = (size_t)std::max<int64_t>(nb * nb, 2048) + 8;
    w->dscal = c.take<double>(np);
    w->iscal = c.take<int>(8);
    w->As = c.take<R>(nn);
    w->W = c.take<R>(nn);
    w->Qh = c.take<R>(nn);
    w->Y = w->As;  // As is dead after the tridiagonalisation
    w->Rhat = c.take<float>(nn);
    w->ZT = c.take<double>(nn);
    w->eigscratch = c.take<double>(2 * (size_t)n * chunk + 3 * n + 8 + (4 * n + 8) +
                                   (size_t)tw_scale_rows((int)n) * chunk + (4 * n + 8));
    w->lam = c.take<double>(n);
    w->vecws = c.take<R>(4 * n + 16);
    w->betas = c.take<R>(n + 8);
    w->btws = c.take<R>((size_t)2 * kBackNb * kBackNb + (size_t)2 * kBackNb * n);
    w->digits = nullptr;
    w->rho = nullptr;
    if (sizeof(R) == sizeof(float)) {
        w->digits = c.take<uint16_t>(split_digit_elems((int)n));
        w->rho = c.take<int>(n);
    }
    w->chunk = chunk;
    return 0;
}

// A_s (already in w->As) -> V, lamr, s; returns status
template <class R>
int spd_decompose(sqrtm_handle_t h, int64_t n, SpdWork<R> &w, sqrtm_info *info = nullptr)
{
    cudaStream_t s = h->stream;
    const int ni = (int)n;
    // reflectors go to Qh (zero outside their support)
    if (cudaMemsetAsync(w.Qh, 0, (size_t)n * n * sizeof(R), s)) return 7;
    {
        struct Ctx { R *A, *Y, *betas, *ws; int n; } ctx{w.As, w.Qh, w.betas, w.vecws, ni};
        auto enq = [](void *p, cudaStream_t st) -> cudaError_t {
            Ctx *c = (Ctx *)p;
            return launch_tridiag<R>(c->A, c->n, c->n, c->Y, c->n, c->betas, c->ws, st);
        };
        if (run_graph(h, 200 + (int)sizeof(R), w.As, n, 1, enq, &ctx)) return 7;
    }
    cudaEvent_t ev_red = nullptr;
    if (info) {
        if (cudaEventCreate(&ev_red)) return 7;
        if (cudaEventRecord(ev_red, s)) return 7;
    }
    if (launch_tridiag_eig<R>(w.As, ni, ni, w.lam, w.ZT, w.eigscratch, w.chunk, s)) return 7;
    if (sizeof(R) == sizeof(double)) {
        // Eigenvectors of close eigenvalues from independent twisted
        // factorisations are orthogonal only to O(u ||T|| / gap); one
        // Newton-Schulz step restores orthogonality to working precision in
        // the FP64 method (in the FP32 method the rounding to FP32 dominates).
        // (R is double here, so W and As hold n x n doubles; As is free once
        // launch_tridiag_eig has read the tridiagonal entries.)
        double *M = (double *)w.W, *P = (double *)w.As;
        if (launch_rgemm<double>(0, 1, ni, ni, ni, w.ZT, ni, w.ZT, ni, RG_STORE, M, ni, nullptr, nullptr, 0, 0.0, s)) return 7;
        if (launch_rgemm<double>(0, 0, ni, ni, ni, M, ni, w.ZT, ni, RG_STORE, P, ni, nullptr, nullptr, 0, 0.0, s)) return 7;
        newton_schulz_combine_kernel<<<grid1((int64_t)n * n), 256, 0, s>>>(w.ZT, P, (int64_t)n * n); count_launch();
    }
    // V = Q Z: Z (rounded to R) into V, then the reflectors applied to it
    cast_transpose_kernel<R><<<dim3((unsigned)cdiv_i(n, 32), (unsigned)cdiv_i(n, 32)), dim3(32, 8), 0, s>>>(w.ZT, w.V, ni);
    count_launch();
    if (launch_back_transform<R>(w.Qh, ni, w.betas, w.V, ni, ni, w.btws, s)) return 7;
    sqrt_eig_kernel<R><<<grid1(n), 256, 0, s>>>(w.lam, w.lamr, w.s, ni, w.iscal + 1); count_launch();
    if (info && ev_red) {
        float ms = 0;
        if (cudaEventSynchronize(ev_red) == cudaSuccess && cudaEventElapsedTime(&ms, h->ev[0], ev_red) == cudaSuccess)
            info->ms_reduction = ms;
        cudaEventDestroy(ev_red);
    }
    return cudaGetLastError() ? 7 : 0;
}

template <class R>
int fetch_scalar(sqrtm_handle_t h, void *dst, const void *src, size_t bytes)
{
    if (cudaMemcpyAsync(h->staging.p, src, bytes, cudaMemcpyDeviceToHost, h->stream)) return 7;
    if (cudaStreamSynchronize(h->stream)) return 7;
    memcpy(dst, h->staging.p, bytes);
    return 0;
}

template <class R>
int spd_common(sqrtm_handle_t h, const double *dA, int64_t n, int64_t lda, double tol, double *dX,
               int64_t ldx, const sqrtm_opts &o, sqrtm_info *info, bool refine)
{
    cudaStream_t s = h->stream;
    const int ni = (int)n;
    SpdWork<R> w;
    if (int rc = spd_carve<R>(h, n, &w)) return rc;
    h->fact_n = -1;
    if (cudaMemsetAsync(w.iscal, 0, 8 * sizeof(int), s)) return 7;
    if (cudaEventRecord(h->ev[0], s)) return 7;
    if (launch_norm_scale(dA, n, lda, w.dscal + 2, (int)std::min<int64_t>(n, 1024), w.dscal, w.iscal, s)) return 7;
    if (launch_cast_scaled_real<R>(dA, n, lda, w.iscal, w.As, n, s)) return 7;
    double norm_a = 0.0;
    int e = 0;
    if (fetch_scalar<R>(h, &norm_a, w.dscal, sizeof(double)) || fetch_scalar<R>(h, &e, w.iscal, sizeof(int))) return 7;
    if (info) { info->norm_a = norm_a; info->scale_exponent = e; info->kind_used = SQRTM_KIND_SPD; }
    if (!isfinite(norm_a)) return 5;
    if (norm_a == 0.0) return 2;
    if (int rc = spd_decompose<R>(h, n, w, info)) return rc;
    if (cudaEventRecord(h->ev[1], s)) return 7;
    // X_0 = V diag(s) V^T, rounded to R, times 2^e (mirrored)
    scale_cols_kernel<R><<<grid1((int64_t)n * n), 256, 0, s>>>(w.V, w.s, w.W, ni); count_launch();
    if (launch_rgemm<R>(0, 1, ni, ni, ni, w.W, ni, w.V, ni, RG_SYM_TO_F64, nullptr, 0, nullptr, dX, ldx, ldexp(1.0, e), s)) return 7;
    if (cudaEventRecord(h->ev[2], s)) return 7;
    int st = 0;
    if (fetch_scalar<R>(h, &st, w.iscal + 1, sizeof(int))) return 7;
    if (info) {
        float ms = 0;
        cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]); info->ms_schur = ms;
        cudaEventElapsedTime(&ms, h->ev[1], h->ev[2]); info->ms_trisqrt = ms;
    }
    if (st) return st;
    if (!refine) return 0;
    const double norm_as = ldexp(norm_a, -2 * e);
    // split-TF32 tensor-core transforms when asked for and the TMA rules hold
    const bool use_tc = sizeof(R) == sizeof(float) && (o.precision & SQRTM_PREC_TF32X3) &&
                        tc_gemm_supported(n, n, n, n, n, w.V, w.Rhat);
    // FP64 residual from BF16 digit products (the FP64 accumulator reuses
    // ZT, free once V is formed)
    const bool use_split = sizeof(R) == sizeof(float) && !(o.precision & SQRTM_PREC_RESID_FP64) && n >= 256 &&
                           split_residual_supported(ni);
    if (use_tc) {
        // V^T into the (now free) Householder-vector buffer
        transpose_kernel<R><<<dim3((unsigned)cdiv_i(n, 32), (unsigned)cdiv_i(n, 32)), dim3(32, 8), 0, s>>>(w.V, w.Qh, ni); count_launch();
    }
    const bool fixed = o.steps >= 0;
    const int max_corr = fixed ? o.steps : o.maxit + 1;
    int status = 0, applied = 0, grew = 0;
    double prev = INFINITY;
    for (int k = 0;; ++k) {
        if (fixed && k >= max_corr) break;
        int np = 0;
        if (use_split) {
            if (launch_residual_sym_split(dA, lda, dX, ldx, ni, e, w.Rhat, ni, w.ZT, w.digits, w.rho, w.dscal + 2,
                                          &np, w.iscal + 2, s)) return 7;
        } else if (launch_residual_sym_f64(dA, lda, dX, ldx, ni, e, w.Rhat, ni, w.dscal + 2, &np, s)) {
            return 7;
        }
        if (launch_sum_partials(w.dscal + 2, np, w.dscal + 1, s)) return 7;
        if (!fixed) {
            double rn = 0.0;
            if (fetch_scalar<R>(h, &rn, w.dscal + 1, sizeof(double))) return 7;
            double rel = rn / norm_as;
            if (info && info->history_len < SQRTM_MAX_HISTORY) info->history[info->history_len++] = rel;
            if (!isfinite(rel)) { status = 4; break; }
            if (rel <= tol) { status = 0; break; }
            if (k >= max_corr) { status = 1; break; }
            grew = (rn > prev) ? grew + 1 : 0;
            if (grew >= 2) { status = 4; break; }
            prev = rn;
        }
        // Y = (V^T Rhat V) ./ (s_i + s_j);  X += 2^e V Y V^T
        if (use_tc) {
            // tensor cores, split TF32; every operand K-contiguous:
            //   W1 = Rhat^T V (= Rhat V, Rhat exactly symmetric),
            //   Y = (V^T W1) ./ (s_i + s_j), W2^T = Y^T V^T, X += W2 V^T
            float *Vf = (float *)w.V, *VT = (float *)w.Qh, *Wf = (float *)w.W, *Yf = (float *)w.Y;
            TcEpilogue ep{};
            ep.C = Wf; ep.ldc = ni;
            if (launch_tc3_gemm(ni, ni, ni, w.Rhat, ni, Vf, ni, TC_EPI_STORE, ep, w.iscal + 2, s)) return 7;
            ep.C = Yf; ep.s = (const float *)w.s;
            if (launch_tc3_gemm(ni, ni, ni, Vf, ni, Wf, ni, TC_EPI_DIAG_SOLVE, ep, w.iscal + 2, s)) return 7;
            ep.C = Wf; ep.s = nullptr;
            if (launch_tc3_gemm(ni, ni, ni, Yf, ni, VT, ni, TC_EPI_STORE, ep, w.iscal + 2, s)) return 7;
            TcEpilogue ex{};
            ex.X = dX; ex.ldx = ldx; ex.scale = ldexp(1.0, e);
            if (launch_tc3_gemm(ni, ni, ni, Wf, ni, VT, ni, TC_EPI_SYM_ADD_F64, ex, w.iscal + 2, s)) return 7;
        } else {
            if (launch_rgemm<float>(0, 0, ni, ni, ni, w.Rhat, ni, (const float *)w.V, ni, RG_STORE, (float *)w.W, ni, nullptr, nullptr, 0, 0.0, s)) return 7;
            if (launch_rgemm<float>(1, 0, ni, ni, ni, (const float *)w.V, ni, (const float *)w.W, ni, RG_DIAG_SOLVE, (float *)w.Y, ni, (const float *)w.s, nullptr, 0, 0.0, s)) return 7;
            if (launch_rgemm<float>(0, 0, ni, ni, ni, (const float *)w.V, ni, (const float *)w.Y, ni, RG_STORE, (float *)w.W, ni, nullptr, nullptr, 0, 0.0, s)) return 7;
            if (launch_rgemm<float>(0, 1, ni, ni, ni, (const float *)w.W, ni, (const float *)w.V, ni, RG_SYM_ADD_F64, nullptr, 0, nullptr, dX, ldx, ldexp(1.0, e), s)) return 7;
        }
        ++applied;
    }
    if (cudaEventRecord(h->ev[3], s)) return 7;
    if (use_tc || use_split) {
        int tcst = 0;
        if (fetch_scalar<R>(h, &tcst, w.iscal + 2, sizeof(int))) return 7;
        if (tcst) return tcst;
    }
    if (status == 0 || status == 1) {
        if (cudaMemcpy2DAsync(w.xsave, n * sizeof(double), dX, ldx * sizeof(double), n * sizeof(double), n,
                              cudaMemcpyDeviceToDevice, s)) return 7;
        h->fact_n = n; h->fact_kind = SQRTM_KIND_SPD; h->fact_e = e; h->fact_norm = norm_a;
        h->fact_q = w.V; h->fact_s = w.s; h->fact_x = w.xsave;
    }
    if (cudaStreamSynchronize(s)) return 7;
    if (info) {
        info->iterations = applied;
        float ms = 0;
        cudaEventElapsedTime(&ms, h->ev[2], h->ev[3]); info->ms_refine = ms;
    }
    return status;
}

}  // namespace

int spd_path(sqrtm_handle_t h, const double *dA, int64_t n, int64_t lda, double tol, double *dX,
             int64_t ldx, const sqrtm_opts &o, sqrtm_info *info)
{
    return spd_common<float>(h, dA, n, lda, tol, dX, ldx, o, info, true);
}

int spd_schur_fp64(sqrtm_handle_t h, const double *dA, int64_t n, int64_t lda, double *dX,
                   int64_t ldx, const sqrtm_opts &o, sqrtm_info *info)
{
    return spd_common<double>(h, dA, n, lda, 0.0, dX, ldx, o, info, false);
}

// ---------------------------------------------------------------------------
// step-level entry points of Algorithm 3
// ---------------------------------------------------------------------------
extern "C" int sqrtm_step_syevd(sqrtm_handle_t h, const void *dAs, void *dV, void *dlam, int64_t n,
                                int fp64)
{
    if (!h) return -1;
    if (n < 0) return -5;
    if (n == 0) return 0;
    if (n > 46340) return -5;
    auto run = [&](auto tag) -> int {
        using R = decltype(tag);
        SpdWork<R> w;
        if (int rc = spd_carve<R>(h, n, &w)) return rc;
        if (cudaMemsetAsync(w.iscal, 0, 8 * sizeof(int), h->stream)) return 7;
        if (cudaMemcpyAsync(w.As, dAs, (size_t)n * n * sizeof(R), cudaMemcpyDeviceToDevice, h->stream)) return 7;
        if (int rc = spd_decompose<R>(h, n, w)) return rc;
        if (cudaMemcpyAsync(dV, w.V, (size_t)n * n * sizeof(R), cudaMemcpyDeviceToDevice, h->stream)) return 7;
        if (cudaMemcpyAsync(dlam, w.lamr, (size_t)n * sizeof(R), cudaMemcpyDeviceToDevice, h->stream)) return 7;
        h->fact_n = -1;
        int st = 0;
        if (fetch_scalar<R>(h, &st, w.iscal + 1, sizeof(int))) return 7;
        return st == 2 ? 0 : st;  // a non-positive eigenvalue is a valid decomposition here
    };
    return fp64 ? run(double(0)) : run(float(0));
}

namespace sqm {
__global__ void sqrt_vec_kernel(const float *__restrict__ lam, float *__restrict__ s, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        s[i] = sqrtf(lam[i]);
}
}  // namespace sqm

extern "C" int sqrtm_step_transform_in_spd(sqrtm_handle_t h, const float *dV, const float *dlam,
                                           const float *dRhat, float *dY, int64_t n)
{
    if (!h) return -1;
    if (n < 0) return -6;
    if (n == 0) return 0;
    const size_t nn = (size_t)n * n;
    if (ensure(h->ws, Carve::round(nn * sizeof(float)) + Carve::round(n * sizeof(float)) + 1024, h)) return 7;
    Carve c(h->ws.p);
    float *W = c.take<float>(nn);
    float *sv = c.take<float>(n);
    const int ni = (int)n;
    cudaStream_t st = h->stream;
    sqrt_vec_kernel<<<grid1(n), 256, 0, st>>>(dlam, sv, ni); count_launch();
    if (launch_rgemm<float>(0, 0, ni, ni, ni, dRhat, ni, dV, ni, RG_STORE, W, ni, nullptr, nullptr, 0, 0.0, st)) return 7;
    if (launch_rgemm<float>(1, 0, ni, ni, ni, dV, ni, W, ni, RG_DIAG_SOLVE, dY, ni, sv, nullptr, 0, 0.0, st)) return 7;
    return cudaStreamSynchronize(st) ? 7 : 0;
}

extern "C" int sqrtm_step_transform_out_update_spd(sqrtm_handle_t h, const float *dV,
                                                   const float *dY, int64_t n, int e, double *dX,
                                                   int64_t ldx)
{
    if (!h) return -1;
    if (n < 0) return -4;
    if (ldx < std::max<int64_t>(1, n)) return -7;
    if (n == 0) return 0;
    const size_t nn = (size_t)n * n;
    if (ensure(h->ws, Carve::round(nn * sizeof(float)) + 1024, h)) return 7;
    Carve c(h->ws.p);
    float *W = c.take<float>(nn);
    const int ni = (int)n;
    cudaStream_t st = h->stream;
    if (launch_rgemm<float>(0, 0, ni, ni, ni, dV, ni, dY, ni, RG_STORE, W, ni, nullptr, nullptr, 0, 0.0, st)) return 7;
    if (launch_rgemm<float>(0, 1, ni, ni, ni, W, ni, dV, ni, RG_SYM_ADD_F64, nullptr, 0, nullptr, dX, ldx, ldexp(1.0, e), st)) return 7;
    return cudaStreamSynchronize(st) ? 7 : 0;
}
