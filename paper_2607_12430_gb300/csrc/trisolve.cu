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
#include "tc_common.cuh"

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
// anti-diagonals.  An anti-diagonal has at most 32 entries, so each gets
// blockDim.x / 32 consecutive threads (4, 8 or 16) for its dot product.
template <class R>
__device__ void leaf_sylvester(const cplx<R> *A, const cplx<R> *B, cplx<R> *C, int ma, int nb,
                               int *bad)
{
    const int tpe = (int)(blockDim.x >> 5);
    const int e = threadIdx.x / tpe, p = threadIdx.x % tpe;
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
            for (int t = p; t < L; t += tpe) {
                if (t < la) cfma(acc, A[i + (i + 1 + t) * TLD], C[(i + 1 + t) + j * TLD]);
                else { int k = t - la; cfma(acc, C[i + k * TLD], B[k + j * TLD]); }
            }
        }
        for (int o = 1; o < tpe; o <<= 1) acc += shfl_xor(acc, o);
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
// One block equation of the Sylvester solve: S_II Y_IJ + Y_IJ St_JJ =
// C_IJ - sum_{K>I} S_IK Y_KJ - sum_{K<J} Y_IK St_KJ, written over C_IJ.
// The update terms are dealt round-robin to G groups of 128 threads (each
// with its own double-buffered tiles and named barrier); the partial sums
// are added in group order, then the leaf is solved.  tc: the CTA's
// dynamic shared memory; bad: a shared flag.
template <class R, int G>
__device__ void syl_block(const cplx<R> *__restrict__ S, int lds, int m, const cplx<R> *__restrict__ St, int ldst,
                          int nn, cplx<R> *C, int ldc, int b, int I, int J, int *status, cplx<R> *tc, int *bad)
{
    constexpr int TT = TB * TLD, kSylGroups = G;
    const int Mb = (m + b - 1) / b;
    const int g = threadIdx.x / kTriThreads, lt = threadIdx.x % kTriThreads;
    cplx<R> *ta = tc + TT * (1 + 4 * g), *tb = ta + TT, *ta2 = tb + TT, *tb2 = ta2 + TT;
    if (threadIdx.x == 0) *bad = 0;
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
    leaf_sylvester(la, lb, tc, bm, bn, bad);
    for (int e = threadIdx.x; e < bm * bn; e += blockDim.x) {
        int i = e % bm, j = e / bm;
        C[(i0 + i) + (int64_t)(j0 + j) * ldc] = tc[i + j * TLD];
    }
    if (threadIdx.x == 0 && *bad) atomicExch(status, 2);
}

// The same block equation for the dependency-ordered solve: each update term
// waits for its own producer's done flag (block (K, J) for S_IK Y_KJ, block
// (I, K) for Y_IK St_KJ) right before its tiles are loaded, and the terms go
// in the order their producers finish (by anti-diagonal), so a block has
// accumulated all but its last one or two terms when its neighbours finish:
// only those and the leaf lie on the critical path.  kSylMaxTerms bounds the
// term list (Mb + Nb); on a wait that gives up the block is abandoned (*fail).
static constexpr int kSylMaxTerms = 512;
template <class R, int G>
__device__ void syl_block_flow(const cplx<R> *__restrict__ S, int lds, int m, const cplx<R> *__restrict__ St,
                               int ldst, int nn, cplx<R> *C, int ldc, int b, int I, int J, int *status, cplx<R> *tc,
                               int *bad, volatile int *flags, volatile int *giveup, unsigned long long wait_ns,
                               int *fail, int *terms)
{
    constexpr int TT = TB * TLD, kSylGroups = G;
    const int Mb = (m + b - 1) / b;
    const int g = threadIdx.x / kTriThreads, lt = threadIdx.x % kTriThreads;
    cplx<R> *ta = tc + TT * (1 + 4 * g), *tb = ta + TT;
    const int i0 = I * b, j0 = J * b;
    const int bm = min(b, m - i0), bn = min(b, nn - j0);
    // terms by the anti-diagonal of their producer: S-term K (producer (K, J))
    // on level J - K + Mb - 1, Y-term K (producer (I, K)) on K - I + Mb - 1;
    // encoded K (S) or -1 - K (Y)
    const int w = J - I + Mb - 1;
    if (threadIdx.x == 0) {
        *bad = 0;
        *fail = 0;
        int c = 0;
        for (int L = 0; L < w; ++L) {
            const int ks = J - L + Mb - 1;  // S-term on this level
            if (ks > I && ks < Mb) terms[c++] = ks;
            const int ky = L - (Mb - 1) + I;  // Y-term on this level
            if (ky >= 0 && ky < J) terms[c++] = -1 - ky;
        }
    }
    load_tile(tc, C + i0 + (int64_t)j0 * ldc, ldc, bm, bn);
    __syncthreads();
    cplx<R> acc[8];
    const int r = lt & 31, c0 = lt >> 5;
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = g == 0 ? tc[r + (c0 + 4 * q) * TLD] : cplx<R>{0, 0};
    const int nterm = (Mb - 1 - I) + J;
    __shared__ int s_gok[8];
    for (int t = g; t < nterm; t += kSylGroups) {
        const int code = terms[t];
        if (lt == 0) {
            const int pf = code >= 0 ? code + J * Mb : I + (-1 - code) * Mb;
            int ok = 1;
            if (!flags[pf]) {
                const uint64_t t0 = globaltimer_ns();
                while (!flags[pf]) {
                    if (*giveup || globaltimer_ns() - t0 > wait_ns) { ok = 0; break; }
                    __nanosleep(64);
                }
            }
            __threadfence();
            s_gok[g] = ok;
        }
        group_bar(g);
        if (!s_gok[g]) {
            if (lt == 0) *fail = 1;
            break;
        }
        int bk;
        if (code >= 0) {
            const int k0 = code * b;
            bk = min(b, m - k0);
            load_tile_async_g(ta, S + i0 + (int64_t)k0 * lds, lds, bm, bk, lt);
            load_tile_async_g(tb, C + k0 + (int64_t)j0 * ldc, ldc, bk, bn, lt);
        } else {
            const int k0 = (-1 - code) * b;
            bk = min(b, nn - k0);
            load_tile_async_g(ta, C + i0 + (int64_t)k0 * ldc, ldc, bm, bk, lt);
            load_tile_async_g(tb, St + k0 + (int64_t)j0 * ldst, ldst, bk, bn, lt);
        }
        cp_async_wait_all();
        group_bar(g);
        tile_mms(acc, ta, tb, bk, lt);
        group_bar(g);  // the tiles are reloaded by the group's next term
    }
    __syncthreads();
    if (*fail) return;
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
    leaf_sylvester(la, lb, tc, bm, bn, bad);
    for (int e = threadIdx.x; e < bm * bn; e += blockDim.x) {
        int i = e % bm, j = e / bm;
        C[(i0 + i) + (int64_t)(j0 + j) * ldc] = tc[i + j * TLD];
    }
    if (threadIdx.x == 0 && *bad) atomicExch(status, 2);
}

// ---------------------------------------------------------------------------
// Sylvester wavefront: blocks (I, J) with J - I = w - (Mb - 1), one per CTA.
// ---------------------------------------------------------------------------
template <class R, int G = SylCfg<R>::G>
__global__ void __launch_bounds__(kTriThreads * G)
rtrsyl_wave_kernel(const cplx<R> *__restrict__ S, int lds, int m, const cplx<R> *__restrict__ St,
                   int ldst, int nn, cplx<R> *C, int ldc, int b, int w, int *status,
                   const TriJob<R> *__restrict__ jobs)
{
    extern __shared__ unsigned char smraw[];
    cplx<R> *tc = reinterpret_cast<cplx<R> *>(smraw);
    __shared__ int bad;
    if (jobs) {  // batched: matrix blockIdx.y solves S Y + Y S = C
        const TriJob<R> jb = jobs[blockIdx.y];
        if (!*jb.active) return;
        S = jb.S; St = jb.S; C = jb.C; status = jb.status;
        m = nn = lds = ldst = ldc = jb.n;
    }
    const int Mb = (m + b - 1) / b, Nb = (nn + b - 1) / b;
    const int I = max(0, (Mb - 1) - w) + blockIdx.x;
    const int J = I + w - (Mb - 1);
    if (I >= Mb || J >= Nb || J < 0) return;
    syl_block<R, G>(S, lds, m, St, ldst, nn, C, ldc, b, I, J, status, tc, &bad);
}

// ---------------------------------------------------------------------------
// Sylvester solve in one launch, by dependencies instead of wavefronts: the
// CTAs (all co-resident) take blocks from a ticket counter in wavefront
// order and start a block as soon as (I+1, J) and (I, J-1) are done (every
// other block it needs is done before one of these two).  A finished block
// is published by a flag after a device-scope fence.  Only for 32-row
// blocks and a leading dimension of C that is a multiple of 16 entries, so
// that no 128-byte line holds entries of two blocks: a block is then read
// by other CTAs only after it is final, and the L1 of the SM that wrote it
// holds its own stores.  sync: [0] ticket, [1] give-up flag, [2 + I + J Mb]
// done flags, all zero on entry.  Each wait is bounded (status 6).
// ---------------------------------------------------------------------------
template <class R, int G = SylCfg<R>::G>
__global__ void __launch_bounds__(kTriThreads * G)
rtrsyl_flow_kernel(const cplx<R> *__restrict__ S, int lds, int m, const cplx<R> *__restrict__ St, int ldst, int nn,
                   cplx<R> *C, int ldc, int b, int *status, int *sync, unsigned long long wait_ns)
{
    extern __shared__ unsigned char smraw[];
    cplx<R> *tc = reinterpret_cast<cplx<R> *>(smraw);
    __shared__ int bad, s_t, s_fail;
    __shared__ int s_terms[kSylMaxTerms];
    const int Mb = (m + b - 1) / b, Nb = (nn + b - 1) / b, nblk = Mb * Nb;
    volatile int *flags = sync + 2;
    for (;;) {
        if (threadIdx.x == 0) s_t = atomicAdd(&sync[0], 1);
        __syncthreads();
        int t = s_t;
        if (t >= nblk) break;
        // ticket -> (I, J): wavefront w holds I = ilo(w) .. ihi(w), J = I + w - (Mb - 1)
        int w = 0, I = 0;
        for (;; ++w) {
            const int ilo = max(0, (Mb - 1) - w), ihi = min(Mb - 1, (Mb - 1) - w + (Nb - 1));
            const int cnt = ihi - ilo + 1;
            if (cnt > 0 && t < cnt) { I = ilo + t; break; }
            if (cnt > 0) t -= cnt;
        }
        const int J = I + w - (Mb - 1);
        syl_block_flow<R, G>(S, lds, m, St, ldst, nn, C, ldc, b, I, J, status, tc, &bad, flags, sync + 1, wait_ns,
                             &s_fail, s_terms);
        __syncthreads();
        if (s_fail) {
            if (threadIdx.x == 0) {
                atomicExch(status, 6);
                atomicExch(&sync[1], 1);
            }
            break;
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicExch(&sync[2 + I + J * Mb], 1);
    }
}

// ---------------------------------------------------------------------------
// Triangular square root, block superdiagonal d
// ---------------------------------------------------------------------------
template <class R>
__global__ void __launch_bounds__(kTriThreads)
trisqrt_diag_kernel(const cplx<R> *__restrict__ T, int ldt, cplx<R> *S, int lds, int n, int b,
                    int *status, const TriJob<R> *__restrict__ jobs)
{
    extern __shared__ unsigned char smraw[];
    cplx<R> *ts = reinterpret_cast<cplx<R> *>(smraw);  // T block, overwritten by S
    __shared__ int bad;
    if (jobs) {  // batched: matrix blockIdx.y
        const TriJob<R> jb = jobs[blockIdx.y];
        if (!*jb.active) return;
        T = jb.T; S = jb.S; status = jb.status;
        n = ldt = lds = jb.n;
    }
    const int I = blockIdx.x;
    const int i0 = I * b, bm = min(b, n - i0);
    if (bm <= 0) return;
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

template <class R, int G_ = SylCfg<R>::G>
__global__ void __launch_bounds__(kTriThreads * G_)
trisqrt_off_kernel(const cplx<R> *__restrict__ T, int ldt, cplx<R> *S, int lds, int n, int b,
                   int dblk, int *status, const TriJob<R> *__restrict__ jobs)
{
    extern __shared__ unsigned char smraw[];
    constexpr int TT = TB * TLD, G = G_;
    cplx<R> *tc = reinterpret_cast<cplx<R> *>(smraw);
    __shared__ int bad;
    if (jobs) {  // batched: matrix blockIdx.y
        const TriJob<R> jb = jobs[blockIdx.y];
        if (!*jb.active) return;
        T = jb.T; S = jb.S; status = jb.status;
        n = ldt = lds = jb.n;
    }
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

// ---------------------------------------------------------------------------
// Principal cube root (Sec. 4, p = 3): S = T^(1/3) of upper triangular T with
// V = S^2 alongside, and the refinement's generalized triangular Sylvester
// equation S^2 Y + S Y S + Y S^2 = C (Eq. (3rd-order)), both by b x b block
// wavefronts whose leaves solve A^2 Y + A Y B + Y B^2 = C point by point.
// Block equations (I < J): the cube root's off-diagonal blocks satisfy
//   S_II^2 S_IJ + S_II S_IJ S_JJ + S_IJ S_JJ^2
//       = T_IJ - S_II P_IJ - sum_{I<K<J} S_IK V_KJ,  P_IJ = sum_{I<K<J} S_IK S_KJ,
//   V_IJ = S_II S_IJ + S_IJ S_JJ + P_IJ;
// the Sylvester blocks, with Z = Y S kept alongside,
//   S_II^2 Y_IJ + S_II Y_IJ S_JJ + Y_IJ S_JJ^2 = C_IJ - sum_{K>I} (V_IK Y_KJ
//       + S_IK Z_KJ) - sum_{L<J} Y_IL V_LJ - S_II Z'_IJ,
//   Z'_IJ = sum_{L<J} Y_IL S_LJ,  Z_IJ = Z'_IJ + Y_IJ S_JJ.
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ cplx<R> ccbrt_(cplx<R> z)
{
    const R r = hypot(z.x, z.y);
    if (r == R(0)) return cplx<R>{0, 0};
    const R th = atan2(z.y, z.x) / R(3);  // argument in (-pi/3, pi/3]: the principal root
    const R m = cbrt(r);
    return cplx<R>{m * cos(th), m * sin(th)};
}

// acc(r, c_q) += sum_k A(r, k) B(k, c_q) (the outputs of tile_mms)
template <class R>
__device__ __forceinline__ void tile_mma(cplx<R> (&acc)[8], const cplx<R> *A, const cplx<R> *B, int kk, int lt)
{
    const int r = lt & 31, c0 = lt >> 5;
    for (int k = 0; k < kk; ++k) {
        const cplx<R> a = A[r + k * TLD];
#pragma unroll
        for (int q = 0; q < 8; ++q) cfma(acc[q], a, B[k + (c0 + 4 * q) * TLD]);
    }
}

template <class R>
__device__ __forceinline__ void tile_store(cplx<R> *D, const cplx<R> (&acc)[8])
{
    const int r = threadIdx.x & 31, c0 = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 8; ++q) D[r + (c0 + 4 * q) * TLD] = acc[q];
}

// Point solve of A2 Y + A Y B + Y B2 = C on a leaf (A, A2 = A^2: ma x ma; B,
// B2 = B^2: nb x nb; upper triangular); C is overwritten by Y and Wt
// receives W = Y B.  Anti-diagonal by anti-diagonal (entry (i, j) needs the
// entries below it in column j and left of it in row i), 4 threads per entry:
//   y_ij (a2_ii + a_ii b_jj + b2_jj) = c_ij - sum_{k>i} (a2_ik y_kj + a_ik w_kj)
//       - sum_{l<j} y_il b2_lj - a_ii w'_ij,  w'_ij = sum_{l<j} y_il b_lj,
//   w_ij = w'_ij + y_ij b_jj.
template <class R>
__device__ void leaf_p3(const cplx<R> *A, const cplx<R> *A2, const cplx<R> *B, const cplx<R> *B2, cplx<R> *C,
                        cplx<R> *Wt, int ma, int nb, int *bad)
{
    const int e = threadIdx.x >> 2, p = threadIdx.x & 3;
    for (int w = 0; w <= ma + nb - 2; ++w) {
        const int ioff = ma - 1 - w;  // j = i - ioff
        const int ilo = max(0, ioff), ihi = min(ma - 1, ioff + nb - 1);
        const int i = ilo + e;
        const bool act = i <= ihi;
        const int j = i - ioff;
        cplx<R> acc{0, 0}, wp{0, 0};
        if (act) {
            for (int t = p; t < ma - 1 - i; t += 4) {
                const int k = i + 1 + t;
                cfma(acc, A2[i + k * TLD], C[k + j * TLD]);
                cfma(acc, A[i + k * TLD], Wt[k + j * TLD]);
            }
            for (int l = p; l < j; l += 4) {
                const cplx<R> y = C[i + l * TLD];
                cfma(acc, y, B2[l + j * TLD]);
                cfma(wp, y, B[l + j * TLD]);
            }
        }
        acc += shfl_xor(acc, 1);
        acc += shfl_xor(acc, 2);
        wp += shfl_xor(wp, 1);
        wp += shfl_xor(wp, 2);
        if (act && p == 0) {
            const cplx<R> aii = A[i + i * TLD], bjj = B[j + j * TLD];
            cfma(acc, aii, wp);
            cplx<R> den = A2[i + i * TLD] + aii * bjj + B2[j + j * TLD];
            if (den.x == R(0) && den.y == R(0)) { *bad = 1; den = cplx<R>{R(1), R(0)}; }
            const cplx<R> y = cdiv(C[i + j * TLD] - acc, den);
            C[i + j * TLD] = y;
            Wt[i + j * TLD] = wp + y * bjj;
        }
        __syncthreads();
    }
}

// diagonal blocks: the point recurrence of the triangular cube root
template <class R>
__global__ void __launch_bounds__(kTriThreads)
tricbrt_diag_kernel(const cplx<R> *__restrict__ T, int ldt, cplx<R> *S, int lds, cplx<R> *V, int ldv, int n, int b,
                    int *status)
{
    extern __shared__ unsigned char smraw[];
    cplx<R> *ts = reinterpret_cast<cplx<R> *>(smraw), *tv = ts + TB * TLD;
    __shared__ int bad;
    const int I = blockIdx.x;
    const int i0 = I * b, bm = min(b, n - i0);
    if (threadIdx.x == 0) bad = 0;
    load_tile(ts, T + i0 + (int64_t)i0 * ldt, ldt, bm, bm);
    for (int e = threadIdx.x; e < TB * TLD; e += blockDim.x) tv[e] = cplx<R>{0, 0};
    __syncthreads();
    const R eps = num<R>::eps;
    if (threadIdx.x < bm) {
        const int i = threadIdx.x;
        const cplx<R> t = ts[i + i * TLD];
        // on or near the closed negative real axis (the rule of trisqrt_diag_kernel)
        if (t.x <= R(0) && fabs(t.y) <= fmax(R(10) * eps * hypot(t.x, t.y), (R)n * eps)) bad = 1;
        const cplx<R> sv = ccbrt_(t);
        ts[i + i * TLD] = sv;
        tv[i + i * TLD] = sv * sv;
    }
    __syncthreads();
    const int e = threadIdx.x >> 2, p = threadIdx.x & 3;
    for (int dd = 1; dd < bm; ++dd) {
        const int i = e, j = e + dd;
        const bool act = j < bm;
        cplx<R> sv{0, 0}, st{0, 0};
        if (act)
            for (int k = i + 1 + p; k < j; k += 4) {
                cfma(sv, ts[i + k * TLD], ts[k + j * TLD]);
                cfma(st, ts[i + k * TLD], tv[k + j * TLD]);
            }
        sv += shfl_xor(sv, 1);
        sv += shfl_xor(sv, 2);
        st += shfl_xor(st, 1);
        st += shfl_xor(st, 2);
        if (act && p == 0) {
            const cplx<R> si = ts[i + i * TLD], sj = ts[j + j * TLD];
            cplx<R> den = si * si + si * sj + sj * sj;
            if (den.x == R(0) && den.y == R(0)) { bad = 1; den = cplx<R>{R(1), R(0)}; }
            const cplx<R> sij = cdiv(ts[i + j * TLD] - si * sv - st, den);
            ts[i + j * TLD] = sij;
            tv[i + j * TLD] = sij * (si + sj) + sv;
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < bm * bm; q += blockDim.x) {
        const int i = q % bm, j = q / bm;
        S[(i0 + i) + (int64_t)(i0 + j) * lds] = (i <= j) ? ts[i + j * TLD] : cplx<R>{0, 0};
        V[(i0 + i) + (int64_t)(i0 + j) * ldv] = (i <= j) ? tv[i + j * TLD] : cplx<R>{0, 0};
    }
    if (threadIdx.x == 0 && bad) atomicExch(status, 2);
}

// block superdiagonal dblk >= 1 of the cube root
template <class R>
__global__ void __launch_bounds__(kTriThreads)
tricbrt_off_kernel(const cplx<R> *__restrict__ T, int ldt, cplx<R> *S, int lds, cplx<R> *V, int ldv, int n, int b,
                   int dblk, int *status)
{
    extern __shared__ unsigned char smraw[];
    constexpr int TT = TB * TLD;
    cplx<R> *t0 = reinterpret_cast<cplx<R> *>(smraw), *t1 = t0 + TT, *t2 = t1 + TT, *t3 = t2 + TT,
            *t4 = t3 + TT, *t5 = t4 + TT, *t6 = t5 + TT;
    __shared__ int bad;
    const int Nb = (n + b - 1) / b;
    const int I = blockIdx.x, J = I + dblk;
    if (J >= Nb) return;
    if (threadIdx.x == 0) bad = 0;
    const int i0 = I * b, j0 = J * b;
    const int bm = min(b, n - i0), bn = min(b, n - j0);
    const int lt = threadIdx.x;
    cplx<R> pacc[8], qacc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) pacc[q] = qacc[q] = cplx<R>{0, 0};
    for (int K = I + 1; K < J; ++K) {
        const int k0 = K * b, bk = min(b, n - k0);
        load_tile(t0, S + i0 + (int64_t)k0 * lds, lds, bm, bk);
        load_tile(t1, S + k0 + (int64_t)j0 * lds, lds, bk, bn);
        load_tile(t2, V + k0 + (int64_t)j0 * ldv, ldv, bk, bn);
        __syncthreads();
        tile_mma(pacc, t0, t1, bk, lt);  // P += S_IK S_KJ
        tile_mma(qacc, t0, t2, bk, lt);  // sum S_IK V_KJ
        __syncthreads();
    }
    // right-hand side T_IJ - S_II P - sum S_IK V_KJ
    tile_store(t3, pacc);
    load_tile(t0, S + i0 + (int64_t)i0 * lds, lds, bm, bm);
    load_tile(t4, T + i0 + (int64_t)j0 * ldt, ldt, bm, bn);
    __syncthreads();
    {
        cplx<R> racc[8];
        const int r = lt & 31, c0 = lt >> 5;
#pragma unroll
        for (int q = 0; q < 8; ++q) racc[q] = t4[r + (c0 + 4 * q) * TLD] - qacc[q];
        tile_mms(racc, t0, t3, bm, lt);
        __syncthreads();
        tile_store(t4, racc);
    }
    load_tile(t1, V + i0 + (int64_t)i0 * ldv, ldv, bm, bm);
    load_tile(t2, S + j0 + (int64_t)j0 * lds, lds, bn, bn);
    load_tile(t5, V + j0 + (int64_t)j0 * ldv, ldv, bn, bn);
    for (int e = threadIdx.x; e < TT; e += blockDim.x) t6[e] = cplx<R>{0, 0};
    __syncthreads();
    leaf_p3(t0, t1, t2, t5, t4, t6, bm, bn, &bad);  // t4 = S_IJ
    // V_IJ = S_II S_IJ + S_IJ S_JJ + P
    tile_mma(pacc, t0, t4, bm, lt);
    tile_mma(pacc, t4, t2, bn, lt);
    {
        const int r = lt & 31, c0 = lt >> 5;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int c = c0 + 4 * q;
            if (r < bm && c < bn) {
                S[(i0 + r) + (int64_t)(j0 + c) * lds] = t4[r + c * TLD];
                V[(i0 + r) + (int64_t)(j0 + c) * ldv] = pacc[q];
            }
        }
    }
    // the mirrored blocks below the diagonal are zero
    for (int q = threadIdx.x; q < bn * bm; q += blockDim.x) {
        const int i = q % bn, j = q / bn;
        S[(j0 + i) + (int64_t)(i0 + j) * lds] = cplx<R>{0, 0};
        V[(j0 + i) + (int64_t)(i0 + j) * ldv] = cplx<R>{0, 0};
    }
    if (threadIdx.x == 0 && bad) atomicExch(status, 2);
}

// one anti-diagonal wavefront of S^2 Y + S Y S + Y S^2 = C (C becomes Y; Z = Y S)
template <class R>
__global__ void __launch_bounds__(kTriThreads)
rtrsyl3_wave_kernel(const cplx<R> *__restrict__ S, int lds, const cplx<R> *__restrict__ V, int ldv, int n,
                    cplx<R> *C, int ldc, cplx<R> *Z, int ldz, int b, int w, int *status)
{
    extern __shared__ unsigned char smraw[];
    constexpr int TT = TB * TLD;
    cplx<R> *t0 = reinterpret_cast<cplx<R> *>(smraw), *t1 = t0 + TT, *t2 = t1 + TT, *t3 = t2 + TT,
            *t4 = t3 + TT, *t5 = t4 + TT, *t6 = t5 + TT;
    __shared__ int bad;
    const int Nb = (n + b - 1) / b;
    const int I = max(0, (Nb - 1) - w) + blockIdx.x;
    const int J = I + w - (Nb - 1);
    if (I >= Nb || J >= Nb || J < 0) return;
    if (threadIdx.x == 0) bad = 0;
    const int i0 = I * b, j0 = J * b;
    const int bm = min(b, n - i0), bn = min(b, n - j0);
    const int lt = threadIdx.x, r = lt & 31, c0 = lt >> 5;
    cplx<R> acc[8], zp[8];
    load_tile(t5, C + i0 + (int64_t)j0 * ldc, ldc, bm, bn);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        acc[q] = t5[r + (c0 + 4 * q) * TLD];
        zp[q] = cplx<R>{0, 0};
    }
    __syncthreads();
    for (int K = I + 1; K < Nb; ++K) {  // - V_IK Y_KJ - S_IK Z_KJ
        const int k0 = K * b, bk = min(b, n - k0);
        load_tile(t0, V + i0 + (int64_t)k0 * ldv, ldv, bm, bk);
        load_tile(t1, C + k0 + (int64_t)j0 * ldc, ldc, bk, bn);
        load_tile(t2, S + i0 + (int64_t)k0 * lds, lds, bm, bk);
        load_tile(t3, Z + k0 + (int64_t)j0 * ldz, ldz, bk, bn);
        __syncthreads();
        tile_mms(acc, t0, t1, bk, lt);
        tile_mms(acc, t2, t3, bk, lt);
        __syncthreads();
    }
    for (int L = 0; L < J; ++L) {  // - Y_IL V_LJ; Z' += Y_IL S_LJ
        const int l0 = L * b, bl = min(b, n - l0);
        load_tile(t0, C + i0 + (int64_t)l0 * ldc, ldc, bm, bl);
        load_tile(t1, V + l0 + (int64_t)j0 * ldv, ldv, bl, bn);
        load_tile(t2, S + l0 + (int64_t)j0 * lds, lds, bl, bn);
        __syncthreads();
        tile_mms(acc, t0, t1, bl, lt);
        tile_mma(zp, t0, t2, bl, lt);
        __syncthreads();
    }
    tile_store(t4, zp);
    load_tile(t0, S + i0 + (int64_t)i0 * lds, lds, bm, bm);
    __syncthreads();
    tile_mms(acc, t0, t4, bm, lt);  // - S_II Z'
    tile_store(t5, acc);
    load_tile(t1, V + i0 + (int64_t)i0 * ldv, ldv, bm, bm);
    load_tile(t2, S + j0 + (int64_t)j0 * lds, lds, bn, bn);
    load_tile(t3, V + j0 + (int64_t)j0 * ldv, ldv, bn, bn);
    for (int e = threadIdx.x; e < TT; e += blockDim.x) t6[e] = cplx<R>{0, 0};
    __syncthreads();
    leaf_p3(t0, t1, t2, t3, t5, t6, bm, bn, &bad);  // t5 = Y_IJ
    tile_mma(zp, t5, t2, bn, lt);                   // Z_IJ = Z' + Y_IJ S_JJ
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int c = c0 + 4 * q;
        if (r < bm && c < bn) {
            C[(i0 + r) + (int64_t)(j0 + c) * ldc] = t5[r + c * TLD];
            Z[(i0 + r) + (int64_t)(j0 + c) * ldz] = zp[q];
        }
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
    trisqrt_diag_kernel<R><<<Nb, kTriThreads, sm1, s>>>(T, ldt, S, lds, n, b, d_status, nullptr); count_launch();
    for (int dblk = 1; dblk < Nb; ++dblk) {
        trisqrt_off_kernel<R><<<Nb - dblk, SylCfg<R>::THREADS, sm3, s>>>(T, ldt, S, lds, n, b, dblk, d_status, nullptr);
        count_launch();
    }
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_trisqrt_batched(const TriJob<R> *jobs, int batch, int nmax, int blks, cudaStream_t s)
{
    if (nmax <= 0 || batch <= 0) return cudaSuccess;
    const int b = blks < 1 ? 1 : (blks > TB ? TB : blks);
    const int Nb = (nmax + b - 1) / b;
    // one group of 128 threads per block: a batch of small matrices has few
    // update terms per block and many blocks, so the smaller footprint (5
    // tiles) lets several blocks share an SM
    const size_t sm1 = TB * TLD * sizeof(cplx<R>), sm3 = 5 * sm1;
    cudaError_t err;
    if ((err = set_smem<R>((const void *)trisqrt_off_kernel<R, 1>, sm3))) return err;
    trisqrt_diag_kernel<R><<<dim3(Nb, batch), kTriThreads, sm1, s>>>(nullptr, 0, nullptr, 0, 0, b, nullptr, jobs);
    count_launch();
    for (int dblk = 1; dblk < Nb; ++dblk) {
        trisqrt_off_kernel<R, 1><<<dim3(Nb - dblk, batch), kTriThreads, sm3, s>>>(nullptr, 0, nullptr, 0, 0, b, dblk,
                                                                                nullptr, jobs);
        count_launch();
    }
    return cudaGetLastError();
}

size_t rtrsyl_flow_ints(int m, int n)
{
    return (size_t)((m + TB - 1) / TB) * ((n + TB - 1) / TB) + 2;
}

template <class R>
cudaError_t launch_rtrsyl(const cplx<R> *S, int lds, int m, const cplx<R> *St, int ldst, int nn,
                          cplx<R> *C, int ldc, int blks, int *d_status, cudaStream_t s, int *flow, int64_t flow_cap)
{
    if (m <= 0 || nn <= 0) return cudaSuccess;
    int b = blks < 1 ? 1 : (blks > TB ? TB : blks);
    int Mb = (m + b - 1) / b, Nb = (nn + b - 1) / b;
    size_t sm3 = (1 + 4 * SylCfg<R>::G) * TB * TLD * sizeof(cplx<R>);
    cudaError_t err;
    if (flow && b == TB && ldc % 16 == 0 && ((uintptr_t)C % 128) == 0 && (int64_t)Mb * Nb + 2 <= flow_cap &&
        Mb + Nb > 2 && Mb + Nb <= kSylMaxTerms) {
        // one launch, ordered by dependencies (rtrsyl_flow_kernel)
        if ((err = set_smem<R>((const void *)rtrsyl_flow_kernel<R>, sm3))) return err;
        int dev = 0, sms = 0, per = 0;
        if ((err = cudaGetDevice(&dev)) || (err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
            return err;
        if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, rtrsyl_flow_kernel<R>, SylCfg<R>::THREADS, sm3)))
            return err;
        const int grid = (int)std::min<int64_t>((int64_t)Mb * Nb, (int64_t)std::max(1, per) * sms);
        if ((err = cudaMemsetAsync(flow, 0, ((size_t)Mb * Nb + 2) * sizeof(int), s))) return err;
        rtrsyl_flow_kernel<R><<<grid, SylCfg<R>::THREADS, sm3, s>>>(S, lds, m, St, ldst, nn, C, ldc, b, d_status, flow,
                                                                    2000000000ull);
        count_launch();
        return cudaGetLastError();
    }
    if ((err = set_smem<R>((const void *)rtrsyl_wave_kernel<R>, sm3))) return err;
    for (int w = 0; w <= Mb + Nb - 2; ++w) {
        int ilo = max(0, (Mb - 1) - w);
        int ihi = min(Mb - 1, (Mb - 1) - w + (Nb - 1));
        int cnt = ihi - ilo + 1;
        if (cnt <= 0) continue;
        rtrsyl_wave_kernel<R><<<cnt, SylCfg<R>::THREADS, sm3, s>>>(S, lds, m, St, ldst, nn, C, ldc, b, w, d_status, nullptr); count_launch();
    }
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_rtrsyl_batched(const TriJob<R> *jobs, int batch, int nmax, int blks, cudaStream_t s)
{
    if (nmax <= 0 || batch <= 0) return cudaSuccess;
    const int b = blks < 1 ? 1 : (blks > TB ? TB : blks);
    const int Nb = (nmax + b - 1) / b;
    const size_t sm3 = 5 * TB * TLD * sizeof(cplx<R>);  // one group of 128 threads per block
    cudaError_t err;
    if ((err = set_smem<R>((const void *)rtrsyl_wave_kernel<R, 1>, sm3))) return err;
    // wavefront w of every matrix at once (a matrix with fewer blocks is done
    // after its own 2 Nb_i - 1 wavefronts; its blocks of later ones return)
    for (int w = 0; w <= 2 * Nb - 2; ++w) {
        const int cnt = min(w, 2 * Nb - 2 - w) + 1;
        rtrsyl_wave_kernel<R, 1><<<dim3(cnt, batch), kTriThreads, sm3, s>>>(nullptr, 0, 0, nullptr, 0, 0, nullptr, 0, b,
                                                                             w, nullptr, jobs);
        count_launch();
    }
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_tricbrt(const cplx<R> *T, int ldt, cplx<R> *S, int lds, cplx<R> *V, int ldv, int n, int blks,
                           int *d_status, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int b = blks < 1 ? 1 : (blks > TB ? TB : blks);
    const int Nb = (n + b - 1) / b;
    const size_t sm1 = TB * TLD * sizeof(cplx<R>);
    cudaError_t err;
    if ((err = set_smem<R>((const void *)tricbrt_diag_kernel<R>, 2 * sm1))) return err;
    if ((err = set_smem<R>((const void *)tricbrt_off_kernel<R>, 7 * sm1))) return err;
    tricbrt_diag_kernel<R><<<Nb, kTriThreads, 2 * sm1, s>>>(T, ldt, S, lds, V, ldv, n, b, d_status); count_launch();
    for (int dblk = 1; dblk < Nb; ++dblk) {
        tricbrt_off_kernel<R><<<Nb - dblk, kTriThreads, 7 * sm1, s>>>(T, ldt, S, lds, V, ldv, n, b, dblk, d_status);
        count_launch();
    }
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_rtrsyl3(const cplx<R> *S, int lds, const cplx<R> *V, int ldv, cplx<R> *C, int ldc, cplx<R> *Z,
                           int ldz, int n, int blks, int *d_status, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int b = blks < 1 ? 1 : (blks > TB ? TB : blks);
    const int Nb = (n + b - 1) / b;
    const size_t sm7 = 7 * TB * TLD * sizeof(cplx<R>);
    cudaError_t err;
    if ((err = set_smem<R>((const void *)rtrsyl3_wave_kernel<R>, sm7))) return err;
    for (int w = 0; w <= 2 * Nb - 2; ++w) {
        const int ilo = max(0, (Nb - 1) - w), ihi = min(Nb - 1, (Nb - 1) - w + (Nb - 1));
        const int cnt = ihi - ilo + 1;
        if (cnt <= 0) continue;
        rtrsyl3_wave_kernel<R><<<cnt, kTriThreads, sm7, s>>>(S, lds, V, ldv, n, C, ldc, Z, ldz, b, w, d_status);
        count_launch();
    }
    return cudaGetLastError();
}

template cudaError_t launch_tricbrt<float>(const cplx<float> *, int, cplx<float> *, int, cplx<float> *, int, int, int,
                                           int *, cudaStream_t);
template cudaError_t launch_tricbrt<double>(const cplx<double> *, int, cplx<double> *, int, cplx<double> *, int, int,
                                            int, int *, cudaStream_t);
// Recursive (Deadman-Higham-Ralha) triangular square root: split T at m,
// S_11 = T_11^{1/2} and S_22 = T_22^{1/2} recursively, then S_12 from the
// Sylvester equation S_11 S_12 + S_12 S_22 = T_12 (Sec. 2.2.1), down to
// blocks of at most `cutoff`, which take the blocked method.  The split is
// rounded to a multiple of 32 so that the Sylvester solves keep whole tiles.
template <class R>
cudaError_t launch_trisqrt_rec(const cplx<R> *T, int ldt, cplx<R> *S, int lds, int n, int blks, int cutoff,
                               int *d_status, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    if (cutoff < 64) cutoff = 64;
    if (n <= cutoff) return launch_trisqrt<R>(T, ldt, S, lds, n, blks, d_status, s);
    int m = ((n / 2 + 31) / 32) * 32;
    if (m >= n) m = n / 2;
    cudaError_t err;
    if ((err = launch_trisqrt_rec<R>(T, ldt, S, lds, m, blks, cutoff, d_status, s))) return err;
    if ((err = launch_trisqrt_rec<R>(T + m + (int64_t)m * ldt, ldt, S + m + (int64_t)m * lds, lds, n - m, blks, cutoff,
                                     d_status, s)))
        return err;
    cplx<R> *S12 = S + (int64_t)m * lds;
    if ((err = cudaMemcpy2DAsync(S12, (size_t)lds * sizeof(cplx<R>), T + (int64_t)m * ldt,
                                 (size_t)ldt * sizeof(cplx<R>), (size_t)m * sizeof(cplx<R>), (size_t)(n - m),
                                 cudaMemcpyDeviceToDevice, s)))
        return err;
    if ((err = cudaMemset2DAsync(S + m, (size_t)lds * sizeof(cplx<R>), 0, (size_t)(n - m) * sizeof(cplx<R>),
                                 (size_t)m, s)))
        return err;
    return launch_rtrsyl<R>(S, lds, m, S + m + (int64_t)m * lds, lds, n - m, S12, lds, blks, d_status, s);
}

template cudaError_t launch_trisqrt_rec<float>(const cplx<float> *, int, cplx<float> *, int, int, int, int, int *,
                                               cudaStream_t);
template cudaError_t launch_trisqrt_rec<double>(const cplx<double> *, int, cplx<double> *, int, int, int, int, int *,
                                                cudaStream_t);
template cudaError_t launch_trisqrt_batched<float>(const TriJob<float> *, int, int, int, cudaStream_t);
template cudaError_t launch_trisqrt_batched<double>(const TriJob<double> *, int, int, int, cudaStream_t);
template cudaError_t launch_rtrsyl_batched<float>(const TriJob<float> *, int, int, int, cudaStream_t);
template cudaError_t launch_rtrsyl_batched<double>(const TriJob<double> *, int, int, int, cudaStream_t);
template cudaError_t launch_rtrsyl3<float>(const cplx<float> *, int, const cplx<float> *, int, cplx<float> *, int,
                                           cplx<float> *, int, int, int, int *, cudaStream_t);
template cudaError_t launch_rtrsyl3<double>(const cplx<double> *, int, const cplx<double> *, int, cplx<double> *, int,
                                            cplx<double> *, int, int, int, int *, cudaStream_t);
template cudaError_t launch_trisqrt<float>(const cplx<float> *, int, cplx<float> *, int, int, int, int *, cudaStream_t);
template cudaError_t launch_trisqrt<double>(const cplx<double> *, int, cplx<double> *, int, int, int, int *, cudaStream_t);
template cudaError_t launch_rtrsyl<float>(const cplx<float> *, int, int, const cplx<float> *, int, int, cplx<float> *, int, int, int *, cudaStream_t, int *, int64_t);
template cudaError_t launch_rtrsyl<double>(const cplx<double> *, int, int, const cplx<double> *, int, int, cplx<double> *, int, int, int *, cudaStream_t, int *, int64_t);

}  // namespace sqm
