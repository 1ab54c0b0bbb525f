// qr.cu -- shifted QR sweeps that reduce the Hessenberg matrix H to the
// upper triangular Schur factor T (Algorithm 2, step 1), accumulating the
// Givens rotations into the Schur vectors Z.
//
// Organisation (one CTA per matrix for the chase, many CTAs for the rest):
//
//  * Each sweep applies nb single shifts at once (nb = NB when the active
//    block [lo, hi] is large, the eigenvalues of its trailing nb x nb block;
//    nb = 1 with the Wilkinson shift otherwise).  Bulge g starts 3 positions
//    behind bulge g-1 and all bulges advance one position per step, so the
//    rotations of one step act on disjoint row pairs (left) and disjoint
//    column pairs (right) and are applied by different warps at once.  The
//    result equals nb consecutive single-shift sweeps.
//  * The chase runs in windows of W steps on the (W + 3 nb + 3)^2 block
//    around the bulges in shared memory.  After a window its rotations are
//    applied at once to the rest of the ACTIVE block only (rows to the right
//    of the window, columns above it) and appended to a rotation log.
//  * Entries outside the active block are never read again by the iteration,
//    so their updates (columns right of hi, rows above lo) and all updates of
//    Z are deferred and applied from the log afterwards: first a pass over
//    rows (right rotations), then a pass over columns (left rotations).  For
//    any entry every deferred right rotation precedes every deferred left one
//    (the active block only shrinks from below or moves up), so that order
//    is exact.
//  * When the log is full the chase kernel stops at a sweep boundary, the
//    passes drain the log, and the chase resumes from the saved state.
//  * Deflation: |h(k,k-1)| <= eps (|h(k,k)| + |h(k-1,k-1)|); an exceptional
//    shift after every 10 sweeps without deflation; at most kItMax sweeps
//    per eigenvalue (status 3).
#include <algorithm>

#include "internal.h"

namespace sqm {

static constexpr int kQrThreads = 256;
static constexpr int kItMax = 60;

template <class R> struct QrCfg;
template <> struct QrCfg<float> { static constexpr int W = 32, NB = 4, CH = 256; };
template <> struct QrCfg<double> { static constexpr int W = 16, NB = 4, CH = 128; };

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

// Eigenvalues of a small upper Hessenberg matrix M (nb x nb, column-major,
// ld NBMAX) by single-shift QR without vectors; one thread.  M is destroyed.
template <class R, int NBMAX>
__device__ void small_eigvals(cplx<R> *M, int nb, cplx<R> *out)
{
    const R eps = num<R>::eps;
    int hi = nb - 1, it = 0;
    while (hi > 0) {
        int lo = hi;
        while (lo > 0) {
            cplx<R> sub = M[lo + (lo - 1) * NBMAX];
            R as = hypot(sub.x, sub.y);
            cplx<R> a = M[lo + lo * NBMAX], b = M[(lo - 1) + (lo - 1) * NBMAX];
            if (as == R(0) || as <= eps * (hypot(a.x, a.y) + hypot(b.x, b.y))) break;
            --lo;
        }
        if (lo == hi) { out[hi] = M[hi + hi * NBMAX]; --hi; it = 0; continue; }
        if (++it > 40) {  // give up: use the diagonal of the unreduced block
            for (int i = lo; i <= hi; ++i) out[i] = M[i + i * NBMAX];
            hi = lo - 1;
            it = 0;
            continue;
        }
        cplx<R> mu = wilkinson(M[(hi - 1) + (hi - 1) * NBMAX], M[(hi - 1) + hi * NBMAX],
                               M[hi + (hi - 1) * NBMAX], M[hi + hi * NBMAX]);
        R c; cplx<R> s, r;
        for (int k = lo; k < hi; ++k) {
            if (k == lo) givens(M[lo + lo * NBMAX] - mu, M[(lo + 1) + lo * NBMAX], c, s, r);
            else givens(M[k + (k - 1) * NBMAX], M[(k + 1) + (k - 1) * NBMAX], c, s, r);
            for (int j = (k == lo ? k : k - 1); j < nb; ++j) {
                cplx<R> p = M[k + j * NBMAX], q = M[(k + 1) + j * NBMAX];
                M[k + j * NBMAX] = c * p + s * q;
                M[(k + 1) + j * NBMAX] = c * q - conj(s) * p;
            }
            if (k > lo) M[(k + 1) + (k - 1) * NBMAX] = cplx<R>{0, 0};
            for (int i = 0; i <= min(k + 2, hi); ++i) {
                cplx<R> p = M[i + k * NBMAX], q = M[i + (k + 1) * NBMAX];
                M[i + k * NBMAX] = c * p + conj(s) * q;
                M[i + (k + 1) * NBMAX] = c * q - s * p;
            }
        }
    }
    if (hi == 0) out[0] = M[0];
}

template <class R>
__global__ void __launch_bounds__(kQrThreads)
qr_chase_kernel(const SchurDesc<R> *__restrict__ descs)
{
    constexpr int W = QrCfg<R>::W, NB = QrCfg<R>::NB, CH = QrCfg<R>::CH;
    constexpr int BWMAX = W + 3 * NB + 3;
    constexpr int RRMAX = W + 3 * NB;  // rows touched by a window's rotations
    extern __shared__ unsigned char smraw[];
    cplx<R> *tile = reinterpret_cast<cplx<R> *>(smraw);  // (a')/(b') staging
    __shared__ cplx<R> blk[BWMAX * BWMAX];
    __shared__ int wk[NB][W];          // rotation positions of the window (-1: none)
    __shared__ R wc[NB][W];
    __shared__ cplx<R> ws[NB][W];
    __shared__ cplx<R> s_r[NB];
    __shared__ cplx<R> s_mu[NB];
    __shared__ int s_lo, s_hi, s_iter, s_status, s_done, s_nb, s_nlog, s_sweeps, s_stop, s_nwin;
    __shared__ long long s_uoff;
    __shared__ long long s_rots;
    __shared__ int s_off[NB + 1];
    __shared__ int s_goff[W];
    __shared__ int s_first[NB], s_cnt[NB];

    const SchurDesc<R> d = descs[blockIdx.x];
    const int n = d.n, ld = d.ld;
    cplx<R> *T = d.T;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nt = blockDim.x;
    const R eps = num<R>::eps;
    int *st = d.state;
    if (st[2]) {  // already finished: nothing new in the log
        if (tid == 0) { st[3] = 0; st[7] = 0; }
        return;
    }
    if (tid == 0) {
        s_hi = (st[0] < -1) ? n - 1 : st[0];
        s_iter = st[1];
        s_status = 0;
        s_done = 0;
        s_nlog = 0;
        s_nwin = 0;
        s_uoff = 0;
        s_sweeps = st[4];
        s_rots = (long long)st[5] + ((long long)st[6] << 31);
        s_stop = 0;
    }
    __syncthreads();

    while (true) {
        const int hi = s_hi;
        if (hi <= 0) { if (tid == 0) s_done = 1; break; }
        if (tid == 0) s_lo = 0;
        __syncthreads();
        for (int k = 1 + tid; k <= hi; k += nt) {
            cplx<R> sub = T[k + (int64_t)(k - 1) * ld];
            R as = hypot(sub.x, sub.y);
            cplx<R> a = T[k + (int64_t)k * ld], b = T[(k - 1) + (int64_t)(k - 1) * ld];
            if (as == R(0) || as <= eps * (hypot(a.x, a.y) + hypot(b.x, b.y))) atomicMax(&s_lo, k);
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
            const int m = hi - lo + 1;
            int nb = (m >= 4 * NB + 2) ? NB : 1;
            const long long nwin_sweep = ((hi - lo) + 3 * (nb - 1) + W - 1) / W;
            if (s_nlog + (long long)(hi - lo) * nb > d.log_cap || s_nwin + nwin_sweep > d.win_cap ||
                s_uoff + nwin_sweep * (long long)(RRMAX * RRMAX) > d.u_cap) {
                s_stop = 1;  // drain the log first
            } else {
                if (lo > 0) T[lo + (int64_t)(lo - 1) * ld] = cplx<R>{0, 0};
                int it = ++s_iter;
                ++s_sweeps;
                if (it > kItMax) s_status = 3;
                if (it % 10 == 0) {
                    nb = 1;
                    cplx<R> sub = T[hi + (int64_t)(hi - 1) * ld];
                    cplx<R> mu = T[hi + (int64_t)hi * ld];
                    mu.x += R(0.75) * hypot(sub.x, sub.y);
                    s_mu[0] = mu;
                } else if (nb == 1) {
                    s_mu[0] = wilkinson(T[(hi - 1) + (int64_t)(hi - 1) * ld], T[(hi - 1) + (int64_t)hi * ld],
                                        T[hi + (int64_t)(hi - 1) * ld], T[hi + (int64_t)hi * ld]);
                } else {
                    cplx<R> M[NB * NB];
                    const int b0 = hi - nb + 1;
                    for (int j = 0; j < nb; ++j)
                        for (int i = 0; i < nb; ++i)
                            M[i + j * NB] = (i <= j + 1) ? T[(b0 + i) + (int64_t)(b0 + j) * ld] : cplx<R>{0, 0};
                    cplx<R> ev[NB];
                    small_eigvals<R, NB>(M, nb, ev);
                    for (int g = 0; g < nb; ++g) s_mu[g] = ev[g];
                }
                s_nb = nb;
                s_rots += (long long)(hi - lo) * nb;
            }
        }
        __syncthreads();
        if (s_stop || s_status) break;
        const int nb = s_nb;
        const int nsteps = (hi - lo) + 3 * (nb - 1);

        for (int t0 = 0; t0 < nsteps; t0 += W) {
            const int t1 = min(t0 + W, nsteps);
            const int kmin = max(lo, lo + t0 - 3 * (nb - 1));
            const int kmax = min(hi - 1, lo + t1 - 1);
            const int r0 = max(lo, kmin - 1);
            const int r1 = min(hi, kmax + 2);
            const int bw = r1 - r0 + 1;
            for (int e = tid; e < bw * bw; e += nt) {
                int a = e % bw, b = e / bw;
                cp_async_elem<R>(&blk[a + b * BWMAX], &T[(r0 + a) + (int64_t)(r0 + b) * ld]);
            }
            if (tid < NB * W) wk[tid / W][tid % W] = -1;
            cp_async_wait_all();
            __syncthreads();
            // the chase: warp g moves bulge g; only the NB chase warps take part
            // (named barrier 1, NB * 32 threads).  Each warp's rotation depends
            // only on entries its own previous step wrote, so all its lanes
            // compute it redundantly; left rotations of one step touch disjoint
            // rows and right rotations disjoint columns, so one barrier after
            // each phase orders the warps.
            if (warp < NB) {
                for (int t = t0; t < t1; ++t) {
                    const int g = warp, k = lo + t - 3 * g;
                    const bool act = warp < nb && k >= lo && k < hi;
                    const int kk = k - r0;
                    R c = R(1);
                    cplx<R> s{0, 0}, r{0, 0};
                    if (act) {
                        cplx<R> x, y;
                        if (k == lo) {
                            x = blk[kk + kk * BWMAX] - s_mu[g];
                            y = blk[(kk + 1) + kk * BWMAX];
                        } else {
                            x = blk[kk + (kk - 1) * BWMAX];
                            y = blk[(kk + 1) + (kk - 1) * BWMAX];
                        }
                        givens(x, y, c, s, r);
                        if (lane == 0) {
                            wk[g][t - t0] = k;
                            wc[g][t - t0] = c;
                            ws[g][t - t0] = s;
                        }
                        __syncwarp();
                        // left rotation: rows kk, kk+1 of the block
                        const int cstart = (k == lo) ? kk : kk - 1;
                        for (int b = cstart + lane; b < bw; b += 32) {
                            cplx<R> p = blk[kk + b * BWMAX], q = blk[(kk + 1) + b * BWMAX];
                            blk[kk + b * BWMAX] = c * p + s * q;
                            blk[(kk + 1) + b * BWMAX] = c * q - conj(s) * p;
                        }
                        __syncwarp();
                        if (lane == 0 && k > lo) {
                            blk[kk + (kk - 1) * BWMAX] = r;
                            blk[(kk + 1) + (kk - 1) * BWMAX] = cplx<R>{0, 0};
                        }
                    }
                    asm volatile("bar.sync 1, %0;" ::"r"(NB * 32) : "memory");
                    if (act) {
                        // right rotation: columns kk, kk+1, block rows up to kk+2
                        const int rend = min(kk + 2, bw - 1);
                        for (int a = lane; a <= rend; a += 32) {
                            cplx<R> p = blk[a + kk * BWMAX], q = blk[a + (kk + 1) * BWMAX];
                            blk[a + kk * BWMAX] = c * p + conj(s) * q;
                            blk[a + (kk + 1) * BWMAX] = c * q - s * p;
                        }
                    }
                    asm volatile("bar.sync 1, %0;" ::"r"(NB * 32) : "memory");
                }
            }
            __syncthreads();
            for (int e = tid; e < bw * bw; e += nt) {
                int a = e % bw, b = e / bw;
                T[(r0 + a) + (int64_t)(r0 + b) * ld] = blk[a + b * BWMAX];
            }
            // log the window's rotations step by step: the (up to nb) rotations of
            // one step act on disjoint index pairs and form one group; the first
            // entry of a group carries the group size (pad), the others 0
            if (tid == 0) {
                int off = s_nlog;
                for (int q = 0; q < t1 - t0; ++q) {
                    s_goff[q] = off;
                    for (int g = 0; g < nb; ++g) off += (wk[g][q] >= 0);
                }
                s_off[NB] = off;
                for (int g = 0; g < NB; ++g) {
                    int first = -1, cnt = 0;
                    if (g < nb)
                        for (int q = 0; q < t1 - t0; ++q)
                            if (wk[g][q] >= 0) {
                                if (first < 0) first = q;
                                ++cnt;
                            }
                    s_first[g] = first;
                    s_cnt[g] = cnt;
                }
            }
            __syncthreads();
            for (int e = tid; e < NB * W; e += nt) {
                const int q = e / NB, g = e % NB;
                if (g < nb && q < t1 - t0 && wk[g][q] >= 0) {
                    int pos = s_goff[q], gsz = 0;
                    for (int u = 0; u < nb; ++u) {
                        if (wk[u][q] >= 0) {
                            if (u < g) ++pos;
                            ++gsz;
                        }
                    }
                    RotLog<R> L;
                    L.k = wk[g][q]; L.lo = lo; L.hi = hi;
                    L.pad = (pos == s_goff[q]) ? gsz : 0;
                    L.c = wc[g][q]; L.pad2 = R(0); L.s = ws[g][q];
                    d.log[pos] = L;
                }
            }
            // (a') columns r1+1 .. hi, rows kmin .. kmax+1: left rotations
            const int rr = kmax + 2 - kmin;
            for (int c0 = r1 + 1; c0 <= hi; c0 += CH) {
                const int cn = min(CH, hi - c0 + 1);
                for (int e = tid; e < rr * cn; e += nt) {
                    int a = e % rr, b = e / rr;
                    cp_async_elem<R>(&tile[a + b * (RRMAX + 1)], &T[(kmin + a) + (int64_t)(c0 + b) * ld]);
                }
                cp_async_wait_all();
                __syncthreads();
                if (tid < cn) {
                    // each bulge's rotations in this window are consecutive
                    // positions k0, k0+1, ...: carry the running element in
                    // registers and load the next one ahead of the update
                    cplx<R> *col = tile + tid * (RRMAX + 1) - kmin;
                    for (int g = 0; g < nb; ++g) {
                        const int q0 = s_first[g], cnt = s_cnt[g];
                        if (cnt <= 0) continue;
                        const int k0 = wk[g][q0];
                        cplx<R> carry = col[k0];
                        cplx<R> nxt = col[k0 + 1];
                        for (int i = 0; i < cnt; ++i) {
                            const R c = wc[g][q0 + i];
                            const cplx<R> s = ws[g][q0 + i];
                            const cplx<R> after = (i + 1 < cnt) ? col[k0 + i + 2] : cplx<R>{0, 0};
                            col[k0 + i] = c * carry + s * nxt;
                            carry = c * nxt - conj(s) * carry;
                            nxt = after;
                        }
                        col[k0 + cnt] = carry;
                    }
                }
                __syncthreads();
                for (int e = tid; e < rr * cn; e += nt) {
                    int a = e % rr, b = e / rr;
                    T[(kmin + a) + (int64_t)(c0 + b) * ld] = tile[a + b * (RRMAX + 1)];
                }
                __syncthreads();
            }
            // (b') rows lo .. r0-1, columns kmin .. kmax+1: right rotations
            for (int i0 = lo; i0 < r0; i0 += CH) {
                const int rn = min(CH, r0 - i0);
                for (int e = tid; e < rn * rr; e += nt) {
                    int a = e % rn, b = e / rn;
                    cp_async_elem<R>(&tile[a + b * (CH + 1)], &T[(i0 + a) + (int64_t)(kmin + b) * ld]);
                }
                cp_async_wait_all();
                __syncthreads();
                if (tid < rn) {
                    cplx<R> *row = tile + tid;
                    for (int g = 0; g < nb; ++g) {
                        const int q0 = s_first[g], cnt = s_cnt[g];
                        if (cnt <= 0) continue;
                        const int k0 = wk[g][q0] - kmin;
                        cplx<R> carry = row[k0 * (CH + 1)];
                        cplx<R> nxt = row[(k0 + 1) * (CH + 1)];
                        for (int i = 0; i < cnt; ++i) {
                            const R c = wc[g][q0 + i];
                            const cplx<R> s = ws[g][q0 + i];
                            const cplx<R> after = (i + 1 < cnt) ? row[(k0 + i + 2) * (CH + 1)] : cplx<R>{0, 0};
                            row[(k0 + i) * (CH + 1)] = c * carry + conj(s) * nxt;
                            carry = c * nxt - s * carry;
                            nxt = after;
                        }
                        row[(k0 + cnt) * (CH + 1)] = carry;
                    }
                }
                __syncthreads();
                for (int e = tid; e < rn * rr; e += nt) {
                    int a = e % rn, b = e / rn;
                    T[(i0 + a) + (int64_t)(kmin + b) * ld] = tile[a + b * (CH + 1)];
                }
                __syncthreads();
            }
            if (tid == 0) {
                WinRec wr;
                wr.start = s_nlog;
                wr.count = s_off[NB] - s_nlog;
                wr.kmin = kmin;
                wr.rr = rr;
                wr.lo = lo;
                wr.hi = hi;
                wr.uoff = s_uoff;
                d.win[s_nwin] = wr;
                s_nwin += 1;
                s_uoff += (long long)rr * rr;
                s_nlog = s_off[NB];
            }
            __syncthreads();
        }
    }
    __syncthreads();
    if (tid == 0) {
        st[0] = s_hi;
        st[1] = s_iter;
        st[2] = (s_done || s_status) ? 1 : 0;
        st[3] = s_nlog;
        st[7] = s_nwin;
        st[4] = s_sweeps;
        st[5] = (int)(s_rots & 0x7fffffff);
        st[6] = (int)(s_rots >> 31);
        if (s_status) *d.status = s_status;
        if (d.counters) {
            d.counters[0] = s_sweeps;
            d.counters[1] = st[5];
            d.counters[2] = st[6];
        }
    }
}

// Accumulated product of one window's rotations: U = I G_1^H G_2^H ... (the
// right rotations in log order applied to the rows of I).  Then a row
// segment x (indices kmin .. kmin+rr-1) receiving the window's right
// rotations becomes x U, and a column segment y receiving its left rotations
// becomes U^H y.  One CTA per window, thread r owns row r of U.
template <class R>
__global__ void qr_build_u_kernel(const SchurDesc<R> *__restrict__ descs)
{
    constexpr int RRMAX = QrCfg<R>::W + 3 * QrCfg<R>::NB;
    __shared__ cplx<R> u[RRMAX * (RRMAX + 1)];
    __shared__ RotLog<R> lg[64];
    const SchurDesc<R> d = descs[blockIdx.y];
    const int nwin = d.state[7];
    if ((int)blockIdx.x >= nwin) return;
    const WinRec w = d.win[blockIdx.x];
    const int rr = w.rr, r = threadIdx.x;
    const int ld = RRMAX + 1;
    if (r < rr)
        for (int c = 0; c < rr; ++c) u[r * ld + c] = cplx<R>{(R)(r == c), R(0)};
    for (int e0 = 0; e0 < w.count; e0 += 64) {
        const int en = min(64, w.count - e0);
        __syncthreads();
        if (threadIdx.x < en) lg[threadIdx.x] = d.log[w.start + e0 + threadIdx.x];
        __syncthreads();
        if (r < rr) {
            cplx<R> *row = u + r * ld;
            for (int e = 0; e < en; ++e) {
                const int a = lg[e].k - w.kmin;
                if ((unsigned)a > (unsigned)(rr - 2)) { atomicExch(d.status, 7); continue; }
                const R c = lg[e].c;
                const cplx<R> s = lg[e].s;
                cplx<R> p = row[a], q = row[a + 1];
                row[a] = c * p + conj(s) * q;
                row[a + 1] = c * q - s * p;
            }
        }
    }
    __syncthreads();
    cplx<R> *U = d.ubuf + w.uoff;
    for (int e = threadIdx.x; e < rr * rr; e += blockDim.x) {
        const int q = e % rr, c = e / rr;  // U(q, c), column-major
        U[e] = u[q * ld + c];
    }
}

// Deferred right rotations on rows (Schur vectors Z: every window; rows of T
// above the window's active block: i < lo): x <- x U_w for each window in
// order.  A CTA holds rpc rows in shared memory.
template <class R>
__global__ void __launch_bounds__(256)
qr_apply_rows_kernel(const SchurDesc<R> *__restrict__ descs, int rpc, int ctas_t)
{
    constexpr int RRMAX = QrCfg<R>::W + 3 * QrCfg<R>::NB;
    extern __shared__ unsigned char smraw[];
    const SchurDesc<R> d = descs[blockIdx.y];
    const int n = d.n, ld = d.ld;
    const int nwin = d.state[7];
    if (nwin == 0) return;
    const bool isT = blockIdx.x < ctas_t;
    const int cb = isT ? blockIdx.x : blockIdx.x - ctas_t;
    const int i0 = cb * rpc;
    if (i0 >= n) return;
    const int rn = min(rpc, n - i0);
    cplx<R> *M = isT ? d.T : d.Q;
    cplx<R> *buf = reinterpret_cast<cplx<R> *>(smraw);          // rpc x n, buf[r + c rpc]
    cplx<R> *ub[2] = {buf + (size_t)rpc * n, buf + (size_t)rpc * n + RRMAX * RRMAX};
    for (int e = threadIdx.x; e < rn * n; e += blockDim.x) {
        const int a = e % rn, b = e / rn;
        cp_async_elem<R>(&buf[a + b * rpc], &M[(i0 + a) + (int64_t)b * ld]);
    }
    // windows that touch this CTA's rows, in order; U of the next one is
    // fetched while the current one is applied
    auto next_win = [&](int wi) {
        while (wi < nwin && isT && i0 >= d.win[wi].lo) ++wi;
        return wi;
    };
    auto fetch_u = [&](int wi, cplx<R> *dst) {
        const WinRec w = d.win[wi];
        for (int e = threadIdx.x; e < w.rr * w.rr; e += blockDim.x) cp_async_elem<R>(&dst[e], &d.ubuf[w.uoff + e]);
    };
    constexpr int MAXO = (32 * RRMAX + 255) / 256;
    int wi = next_win(0), par = 0;
    if (wi < nwin) fetch_u(wi, ub[0]);
    while (wi < nwin) {
        const WinRec w = d.win[wi];
        const int rr = w.rr;
        cp_async_wait_all();
        __syncthreads();
        const int wn = next_win(wi + 1);
        if (wn < nwin) fetch_u(wn, ub[par ^ 1]);
        const cplx<R> *us = ub[par];
        cplx<R> out[MAXO];
        const int no = rn * rr;
#pragma unroll
        for (int j = 0; j < MAXO; ++j) {
            const int o = threadIdx.x + j * 256;
            out[j] = cplx<R>{0, 0};
            if (o < no) {
                const int r = o % rn, c = o / rn;
                const cplx<R> *x = buf + r + (size_t)w.kmin * rpc;
                const cplx<R> *uc = us + (size_t)c * rr;
                cplx<R> acc{0, 0};
                for (int q = 0; q < rr; ++q) cfma(acc, x[(size_t)q * rpc], uc[q]);
                out[j] = acc;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < MAXO; ++j) {
            const int o = threadIdx.x + j * 256;
            if (o < no) {
                const int r = o % rn, c = o / rn;
                if (!isT || i0 + r < w.lo) buf[r + (size_t)(w.kmin + c) * rpc] = out[j];
            }
        }
        wi = wn;
        par ^= 1;
    }
    cp_async_wait_all();
    __syncthreads();
    for (int e = threadIdx.x; e < rn * n; e += blockDim.x) {
        const int a = e % rn, b = e / rn;
        M[(i0 + a) + (int64_t)b * ld] = buf[a + b * rpc];
    }
}

// Deferred left rotations on columns of T right of the window's active block
// (j > hi): y <- U_w^H y for each window in order.  Runs after the rows pass.
template <class R>
__global__ void __launch_bounds__(256)
qr_apply_cols_kernel(const SchurDesc<R> *__restrict__ descs, int cpc)
{
    constexpr int RRMAX = QrCfg<R>::W + 3 * QrCfg<R>::NB;
    extern __shared__ unsigned char smraw[];
    const SchurDesc<R> d = descs[blockIdx.y];
    const int n = d.n, ld = d.ld;
    const int nwin = d.state[7];
    if (nwin == 0) return;
    const int j0 = blockIdx.x * cpc;
    if (j0 >= n) return;
    const int cn = min(cpc, n - j0);
    const int cs = n + 1;
    cplx<R> *buf = reinterpret_cast<cplx<R> *>(smraw);           // column jl at buf + jl cs
    cplx<R> *ub[2] = {buf + (size_t)cs * cpc, buf + (size_t)cs * cpc + RRMAX * RRMAX};
    for (int e = threadIdx.x; e < cn * n; e += blockDim.x) {
        const int a = e % n, b = e / n;
        cp_async_elem<R>(&buf[a + (size_t)b * cs], &d.T[a + (int64_t)(j0 + b) * ld]);
    }
    auto next_win = [&](int wi) {
        while (wi < nwin && j0 + cn - 1 <= d.win[wi].hi) ++wi;
        return wi;
    };
    auto fetch_u = [&](int wi, cplx<R> *dst) {
        const WinRec w = d.win[wi];
        for (int e = threadIdx.x; e < w.rr * w.rr; e += blockDim.x) cp_async_elem<R>(&dst[e], &d.ubuf[w.uoff + e]);
    };
    constexpr int MAXO = (32 * RRMAX + 255) / 256;
    int wi = next_win(0), par = 0;
    if (wi < nwin) fetch_u(wi, ub[0]);
    while (wi < nwin) {
        const WinRec w = d.win[wi];
        const int rr = w.rr;
        cp_async_wait_all();
        __syncthreads();
        const int wn = next_win(wi + 1);
        if (wn < nwin) fetch_u(wn, ub[par ^ 1]);
        const cplx<R> *us = ub[par];
        cplx<R> out[MAXO];
        const int no = cn * rr;
#pragma unroll
        for (int j = 0; j < MAXO; ++j) {
            const int o = threadIdx.x + j * 256;
            out[j] = cplx<R>{0, 0};
            if (o < no) {
                const int jl = o % cn, c = o / cn;
                const cplx<R> *y = buf + (size_t)jl * cs + w.kmin;
                const cplx<R> *uc = us + (size_t)c * rr;
                cplx<R> acc{0, 0};
                for (int q = 0; q < rr; ++q) cfma(acc, conj(uc[q]), y[q]);
                out[j] = acc;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < MAXO; ++j) {
            const int o = threadIdx.x + j * 256;
            if (o < no) {
                const int jl = o % cn, c = o / cn;
                if (j0 + jl > w.hi) buf[(size_t)jl * cs + w.kmin + c] = out[j];
            }
        }
        wi = wn;
        par ^= 1;
    }
    cp_async_wait_all();
    __syncthreads();
    for (int e = threadIdx.x; e < cn * n; e += blockDim.x) {
        const int a = e % n, b = e / n;
        d.T[a + (int64_t)(j0 + b) * ld] = buf[a + (size_t)b * cs];
    }
}

template <class R>
__global__ void qr_finish_kernel(const SchurDesc<R> *__restrict__ descs)
{
    const SchurDesc<R> d = descs[blockIdx.y];
    const int n = d.n, ld = d.ld;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)n * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(t % n), j = (int)(t / n);
        if (i > j) d.T[i + (int64_t)j * ld] = cplx<R>{0, 0};
    }
}

template <class R>
__global__ void qr_state_init_kernel(const SchurDesc<R> *__restrict__ descs, int batch)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < batch; b += gridDim.x * blockDim.x) {
        int *st = descs[b].state;
        st[0] = -2;  // fresh: start from hi = n - 1
        for (int q = 1; q < 8; ++q) st[q] = 0;
    }
}

template <class R>
int qr_rows_per_cta(int nmax)
{
    constexpr int RRMAX = QrCfg<R>::W + 3 * QrCfg<R>::NB;
    size_t per = (size_t)(std::max(nmax, 1) + 1) * sizeof(cplx<R>);
    size_t avail = 200 * 1024 - 2 * (size_t)RRMAX * RRMAX * sizeof(cplx<R>);
    size_t r = avail / per;
    return (int)std::max<size_t>(1, std::min<size_t>(32, r));
}

template <class R>
cudaError_t launch_qr_sweeps(const SchurDesc<R> *d_desc, int batch, int nmax, int *h_state,
                             const int *d_state_all, cudaStream_t s)
{
    constexpr int RRMAX = QrCfg<R>::W + 3 * QrCfg<R>::NB, CH = QrCfg<R>::CH;
    const size_t tile_bytes = std::max((size_t)(RRMAX + 1) * CH, (size_t)(CH + 1) * RRMAX) * sizeof(cplx<R>);
    const int rpc = qr_rows_per_cta<R>(nmax);
    const size_t ubytes = 2 * (size_t)RRMAX * RRMAX * sizeof(cplx<R>);
    const size_t rows_bytes = (size_t)rpc * nmax * sizeof(cplx<R>) + ubytes;
    const size_t cols_bytes = (size_t)rpc * (nmax + 1) * sizeof(cplx<R>) + ubytes;
    cudaError_t err;
    if ((err = allow_max_smem((const void *)qr_chase_kernel<R>))) return err;
    if ((err = allow_max_smem((const void *)qr_apply_rows_kernel<R>))) return err;
    if ((err = allow_max_smem((const void *)qr_apply_cols_kernel<R>))) return err;
    qr_state_init_kernel<R><<<1, 256, 0, s>>>(d_desc, batch); count_launch();
    const int ctas = (int)cdiv_i(nmax, rpc);
    bool all = false;
    for (int round = 0; round < 256 && !all; ++round) {
        qr_chase_kernel<R><<<batch, kQrThreads, tile_bytes, s>>>(d_desc); count_launch();
        if ((err = cudaMemcpyAsync(h_state, d_state_all, sizeof(int) * 8 * batch, cudaMemcpyDeviceToHost, s))) return err;
        if ((err = cudaStreamSynchronize(s))) return err;
        int maxwin = 0;
        all = true;
        for (int b = 0; b < batch; ++b) {
            all = all && h_state[8 * b + 2];
            maxwin = std::max(maxwin, h_state[8 * b + 7]);
        }
        if (maxwin > 0) {
            qr_build_u_kernel<R><<<dim3(maxwin, batch), 64, 0, s>>>(d_desc); count_launch();
            qr_apply_rows_kernel<R><<<dim3(2 * ctas, batch), 256, rows_bytes, s>>>(d_desc, rpc, ctas); count_launch();
            qr_apply_cols_kernel<R><<<dim3(ctas, batch), 256, cols_bytes, s>>>(d_desc, rpc); count_launch();
        }
    }
    qr_finish_kernel<R><<<dim3(64, batch), 256, 0, s>>>(d_desc); count_launch();
    return cudaGetLastError();
}

template cudaError_t launch_qr_sweeps<float>(const SchurDesc<float> *, int, int, int *, const int *, cudaStream_t);
template cudaError_t launch_qr_sweeps<double>(const SchurDesc<double> *, int, int, int *, const int *, cudaStream_t);

}  // namespace sqm
