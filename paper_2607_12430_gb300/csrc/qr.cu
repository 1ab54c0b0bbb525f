// qr.cu -- shifted QR sweeps that reduce the Hessenberg matrix H to the
// upper triangular Schur factor T (Algorithm 2, step 1), accumulating the
// Givens rotations into the Schur vectors Z.
//
// Organisation (one CTA of 512 threads per matrix for the chase, many CTAs
// for the rest):
//
//  * Each sweep applies nb single shifts at once: nb = min(NB, (m - 2) / 4)
//    for an active block [lo, hi] of size m, the shifts being the eigenvalues
//    of its trailing nb x nb block (the whole CTA refines them by the
//    Ehrlich-Aberth iteration, started from the previous sweep's shifts; one
//    warp's single-shift QR in shared memory if that does not converge);
//    nb = 1 uses the Wilkinson shift.  Bulge g starts 3
//    positions behind bulge g-1 and all bulges advance one position per step,
//    so the rotations of one step act on disjoint row pairs (left) and
//    disjoint column pairs (right); warp g moves bulge g.  The result equals
//    nb consecutive single-shift sweeps.
//  * The chase runs in windows of W steps on the (W + 3 NB)^2 block around
//    the bulges in shared memory.  A window's rotations form a dense W x NB
//    table (step-major, inactive entries marked), which is the rotation log.
//    After a window its rotations are applied to the rest of the ACTIVE block
//    (rows to the right of the window, columns above it) by all threads:
//    each row or column segment is shared by 4 threads, which take the
//    bulges g = sub, sub + 4, ... of every step in lock-step (a rotation of
//    bulge g at step q needs bulge g-1's rotation of step q-2 only).
//  * Entries outside the active block are never read again by the iteration,
//    so their updates (columns right of hi, rows above lo) and all updates of
//    Z are deferred: each window's rotations are multiplied into a small
//    unitary U_w (one CTA per window), then a pass over rows applies
//    x <- x U_w and a pass over columns y <- U_w^H y, window by window.  For
//    any entry every deferred right rotation precedes every deferred left one
//    (the active block only shrinks from below or moves up), so that order
//    is exact.
//  * When the log is full the chase kernel stops at a sweep boundary, the
//    passes drain the log, and the chase resumes from the saved state.
//  * Deflation: |h(k,k-1)| <= eps (|h(k,k)| + |h(k-1,k-1)|); an exceptional
//    shift after every 10 sweeps without deflation; at most kItMax sweeps
//    per eigenvalue (status 3).
//  * An active block of at most kQrTiny rows gets its whole Schur form from
//    one warp, recorded as a window with a dense U.  The chase only records
//    such a block and goes on with the blocks above it; after the launch,
//    qr_tiny_kernel solves every recorded block (one warp each; for one
//    matrix concurrently with the next round's chase) before the deferred
//    passes.
#include <algorithm>

#include "internal.h"
#include "tc_common.cuh"

namespace sqm {

static constexpr int kItMax = 60;
static constexpr int kQrCoopMinN = 256;  // smallest n for the cooperative chase
static constexpr int kQrPostMin = 64;    // fewer out-of-window rows + columns: the chase CTA does them
static constexpr int kQrTiny = 24;       // active blocks up to this size: one warp, dense U
static constexpr int kAberthIt = 24;     // iteration limit of the simultaneous shift refinement
static constexpr int kQrTinyLd = 33;     // leading dimension of its shared-memory block and U
static constexpr int kQrThreads = 512;           // chase CTA
static constexpr int kQrTpc = 4;                 // threads per row/column segment in the updates
static constexpr int kQrCh = kQrThreads / kQrTpc;  // segments per update chunk

template <class R> struct QrCfg;
template <> struct QrCfg<float> { static constexpr int W = 32, NB = 16; };
template <> struct QrCfg<double> { static constexpr int W = 16, NB = 8; };

// Shared-memory geometry of the chase kernel.
template <class R>
struct QrDims {
    static constexpr int W = QrCfg<R>::W, NB = QrCfg<R>::NB;
    static constexpr int BW = W + 3 * NB;       // largest window block
    static constexpr int BLD = BW + 1;          // its leading dimension (odd: no bank conflicts)
    static constexpr int RR = W + 3 * NB - 2;   // largest index range of a window's rotations
    static constexpr int RLD = RR + 1;          // column tile leading dimension
    static constexpr int CLD = kQrCh + 1;       // row tile leading dimension
    static constexpr int TILE = (kQrCh * RLD > RR * CLD) ? kQrCh * RLD : RR * CLD;
    static constexpr size_t chase_smem =
        (size_t)(BW * BLD + TILE) * sizeof(cplx<R>) + (size_t)W * NB * sizeof(RotLog<R>);
    static constexpr size_t build_smem = (size_t)RR * (RR + 1) * sizeof(cplx<R>) + (size_t)W * NB * sizeof(RotLog<R>);
    static_assert(NB % kQrTpc == 0, "bulges per thread");
    static_assert(NB * 16 <= kQrThreads && NB % 2 == 0, "one half-warp per bulge");
};

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

// The same rotation for FP32 from |x|^2 and |y|^2 and two reciprocal square
// roots, each refined by one Newton step written with fused multiply-adds:
// e = 1 - v y0^2 (one rounding), y1 = y0 + (y0 / 2) e (one rounding).  The
// refinement squares away the systematic part of the hardware reciprocal
// square root's error, which would otherwise accumulate over the thousands
// of rotations applied to each Schur vector (an unrefined form measured ten
// times worse orthogonality); the remaining error is rounding of either
// sign, as with correctly rounded square roots and divisions, at a fraction
// of their latency on the chase's critical path.  Tiny or huge arguments
// take the scaled path.
__device__ __forceinline__ float rsqrt_refined(float v)
{
    const float y0 = rsqrtf(v);
    const float e = fmaf(-(v * y0), y0, 1.0f);
    return fmaf(0.5f * y0, e, y0);
}
template <class R>
__device__ __forceinline__ void givens_fast(cplx<R> x, cplx<R> y, R &c, cplx<R> &s, cplx<R> &r)
{
    givens(x, y, c, s, r);
}
template <>
__device__ __forceinline__ void givens_fast<float>(cplx<float> x, cplx<float> y, float &c, cplx<float> &s,
                                                   cplx<float> &r)
{
    const float ax2 = fmaf(x.x, x.x, x.y * x.y), ay2 = fmaf(y.x, y.x, y.y * y.y);
    const float nrm2 = ax2 + ay2;
    if (!(ax2 >= 1e-30f) || !(nrm2 <= 1e30f)) {
        givens(x, y, c, s, r);
        return;
    }
    const float inv = rsqrt_refined(nrm2), invx = rsqrt_refined(ax2);
    const float f = invx * inv;  // 1 / (|x| ||(x, y)||)
    c = ax2 * f;
    s = cplx<float>{(x.x * y.x + x.y * y.y) * f, (x.y * y.x - x.x * y.y) * f};  // x conj(y) f
    const float gsc = nrm2 * f;                                                // ||(x, y)|| / |x|
    r = cplx<float>{x.x * gsc, x.y * gsc};
}

// Cheaper rotation for the shift computation only (eigenvalue estimates,
// never applied to T or Z): reciprocal square roots instead of correctly
// rounded square roots and divisions.
template <class R>
__device__ __forceinline__ void givens_approx(cplx<R> x, cplx<R> y, R &c, cplx<R> &s, cplx<R> &r)
{
    givens(x, y, c, s, r);
}
template <>
__device__ __forceinline__ void givens_approx<float>(cplx<float> x, cplx<float> y, float &c, cplx<float> &s,
                                                     cplx<float> &r)
{
    const float ax2 = fmaf(x.x, x.x, x.y * x.y), ay2 = fmaf(y.x, y.x, y.y * y.y);
    const float nrm2 = ax2 + ay2;
    if (!(ax2 >= 1e-30f) || !(nrm2 <= 1e30f)) {
        givens(x, y, c, s, r);
        return;
    }
    const float inv = rsqrtf(nrm2), invx = rsqrtf(ax2);
    const float f = invx * inv;
    c = ax2 * f;
    s = cplx<float>{(x.x * y.x + x.y * y.y) * f, (x.y * y.x - x.x * y.y) * f};
    const float gsc = nrm2 * f;
    r = cplx<float>{x.x * gsc, x.y * gsc};
}

// Eigenvalues of a small upper Hessenberg matrix M (nb x nb, nb <= 32,
// column-major, leading dimension LDM) by single-shift QR without vectors,
// one warp: lane j updates column j of a row rotation and row j of a column
// rotation.  Only the active block is updated.  M is destroyed; out[0..nb-1]
// receives the eigenvalues.
template <class R>
__device__ __forceinline__ cplx<R> shfl_c(cplx<R> v, int src)
{
    return cplx<R>{__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src)};
}

// One implicit single-shift sweep on rows / columns lo .. hi of the small
// Hessenberg matrix M (ld LDM, one warp, lane j = column j in the row half
// and row j in the column half of each rotation), optionally accumulating
// the rotations into U (U <- U G^H).  The shared-memory copy is kept up to
// date, but the entries the next step needs -- its rotation's x and y, the
// 2 x 2 block where the row and column halves overlap, the next pair of rows
// -- travel between lanes by shuffles from the lanes that computed them, so
// a rotation costs no shared-memory round trip on the critical path.  The
// arithmetic (and hence every value) is that of the plain two-phase sweep.
template <class R, int LDM, bool ACC, bool APPROX>
__device__ __forceinline__ void warp_sweep(cplx<R> *M, cplx<R> *U, int m, int lo, int hi, cplx<R> mu, int *nrot)
{
    const int lane = threadIdx.x & 31;
    const int ccols = ACC ? m : hi + 1;  // the row half runs to this column (exclusive)
    // row half of rotation k: lane j >= js holds p = M(k, j), q = M(k+1, j)
    cplx<R> p{0, 0}, q{0, 0};
    if (lane >= lo && lane < ccols) {
        p = M[lo + lane * LDM];
        q = M[(lo + 1) + lane * LDM];
    }
    cplx<R> x = shfl_c(p, lo), y = shfl_c(q, lo);
    x = x - mu;
    for (int k = lo; k < hi; ++k) {
        const int js = (k == lo) ? k : k - 1;
        // row k+2 of the columns right of k+1 is untouched until rotation k+1
        cplx<R> nxt{0, 0};
        if (k + 2 <= hi && lane >= k + 2 && lane < ccols) nxt = M[(k + 2) + lane * LDM];
        const cplx<R> sub2 = (k + 2 <= hi) ? M[(k + 2) + (k + 1) * LDM] : cplx<R>{0, 0};
        R c;
        cplx<R> s, r;
        if (APPROX) givens_approx(x, y, c, s, r);
        else givens_fast(x, y, c, s, r);
        const bool lj = lane >= js && lane < ccols;
        cplx<R> np = c * p + s * q, nq = c * q - conj(s) * p;
        if (lane == js && k > lo) {
            np = r;
            nq = cplx<R>{0, 0};
        }
        if (lj) {
            M[k + lane * LDM] = np;
            M[(k + 1) + lane * LDM] = nq;
        }
        // column half: rows lo .. min(k+2, hi) of columns k, k+1
        const cplx<R> np_k1 = shfl_c(np, k + 1), nq_k = shfl_c(nq, k);
        const int rmax = min(k + 2, hi);
        cplx<R> pp{0, 0}, qq{0, 0};
        if (lane == k) {
            pp = np;
            qq = np_k1;
        } else if (lane == k + 1) {
            pp = nq_k;
            qq = nq;
        } else if (lane == k + 2) {
            pp = cplx<R>{0, 0};
            qq = sub2;
        } else if (lane >= (ACC ? 0 : lo) && lane < k) {
            pp = M[lane + k * LDM];
            qq = M[lane + (k + 1) * LDM];
        }
        const cplx<R> npp = c * pp + conj(s) * qq, nqq = c * qq - s * pp;
        __syncwarp();  // the row half's stores land before the column half's
        if (lane >= (ACC ? 0 : lo) && lane <= rmax) {
            M[lane + k * LDM] = npp;
            M[lane + (k + 1) * LDM] = nqq;
        }
        if (ACC && lane < m) {
            const cplx<R> up = U[lane + k * LDM], uq = U[lane + (k + 1) * LDM];
            U[lane + k * LDM] = c * up + conj(s) * uq;
            U[lane + (k + 1) * LDM] = c * uq - s * up;
        }
        // the next rotation: x = M(k+1, k), y = M(k+2, k) as the column half
        // left them; rows k+1, k+2 of columns k, k+1 from the column half
        const cplx<R> a1 = shfl_c(npp, k + 1), b1 = shfl_c(nqq, k + 1);
        const cplx<R> a2 = shfl_c(npp, k + 2), b2 = shfl_c(nqq, k + 2);
        x = a1;
        y = (k + 2 <= hi) ? a2 : cplx<R>{0, 0};
        if (lane == k) {
            p = a1;
            q = a2;
        } else if (lane == k + 1) {
            p = b1;
            q = b2;
        } else {
            p = nq;
            q = nxt;
        }
        __syncwarp();
        if (nrot) ++*nrot;
    }
}

// Eigenvalues of a small upper Hessenberg matrix M (nb x nb, nb <= 32,
// column-major, leading dimension LDM) by single-shift QR without vectors,
// one warp (warp_sweep).  Only the active block is updated.  M is
// destroyed; out[0..nb-1] receives the eigenvalues.
template <class R, int LDM>
__device__ void warp_small_eigvals(cplx<R> *M, int nb, cplx<R> *out)
{
    const int lane = threadIdx.x & 31;
    const R eps = num<R>::eps;
    int hi = nb - 1, it = 0;
    while (hi > 0) {
        bool small = false;
        if (lane >= 1 && lane <= hi) {
            const cplx<R> sub = M[lane + (lane - 1) * LDM];
            const R as = hypot(sub.x, sub.y);
            const cplx<R> a = M[lane + lane * LDM], b = M[(lane - 1) + (lane - 1) * LDM];
            small = as == R(0) || as <= eps * (hypot(a.x, a.y) + hypot(b.x, b.y));
        }
        const unsigned bal = __ballot_sync(0xffffffffu, small);
        const int lo = bal ? 31 - __clz(bal) : 0;
        if (lo == hi) {
            if (lane == 0) out[hi] = M[hi + hi * LDM];
            --hi;
            it = 0;
            __syncwarp();
            continue;
        }
        if (++it > 40) {  // give up: the diagonal of the unreduced block
            for (int i = lo + lane; i <= hi; i += 32) out[i] = M[i + i * LDM];
            hi = lo - 1;
            it = 0;
            __syncwarp();
            continue;
        }
        const cplx<R> mu = wilkinson(M[(hi - 1) + (hi - 1) * LDM], M[(hi - 1) + hi * LDM],
                                     M[hi + (hi - 1) * LDM], M[hi + hi * LDM]);
        __syncwarp();
        warp_sweep<R, LDM, false, true>(M, nullptr, nb, lo, hi, mu, nullptr);
    }
    if (hi == 0 && lane == 0) out[0] = M[0];
    __syncwarp();
}

// Shifts by simultaneous refinement of all nb eigenvalue estimates of the
// small unreduced Hessenberg block M (nb x nb, nb <= 32, leading dimension
// LDM): the Ehrlich-Aberth iteration (O. Aberth, Math. Comp. 27 (1973)),
//   z_j <- z_j - N_j / (1 - N_j sum_{k != j} 1 / (z_j - z_k)),
// with every estimate updated at once, where N_j = p(z_j) / p'(z_j) and
// p(z) = det(M - z I).  The Newton ratio comes from Hyman's recurrence
// (Wilkinson, The Algebraic Eigenvalue Problem, 1965, Ch. 7): with
// x_{nb-1} = 1, row i of (M - z I) x = 0 fixes x_{i-1} through the
// subdiagonal entry M(i, i-1), for i = nb-1 down to 1; the residual of row 0
// is then p(z) times a product of subdiagonal entries that does not depend
// on z, so differentiating the recurrence gives the same multiple of p'(z)
// and the ratio of the two is N.  A segment of lanes per estimate (16 while
// nb <= 16, so a warp takes two): lane r keeps the running sums of row r for
// the residual and its derivative, and each new x_i (formed by lane i) is
// broadcast and added into the rows above it.  x, its derivative and the
// sums are rescaled together by powers of two to stay in range, which
// leaves the ratio unchanged.  No CTA-wide state other than z changes; M is
// not modified.  On entry z (shared memory) holds nb distinct starting
// estimates; true means every correction of the last
// iteration was at most tol (|z_j| + 1e-3 max|M_ij|) and z holds the
// shifts; false (no convergence within kmax iterations, or a non-finite
// value) leaves z unusable.  Every thread of the CTA calls it.
template <class R> __device__ __forceinline__ R aberth_tol();
template <> __device__ __forceinline__ float aberth_tol<float>() { return 1e-6f; }
template <> __device__ __forceinline__ double aberth_tol<double>() { return 1e-11; }

template <class R, int LDM>
__device__ bool cta_aberth_shifts(const cplx<R> *M, int nb, cplx<R> *z, R mnrm, int kmax)
{
    __shared__ cplx<R> s_inv[32], s_w[32];
    __shared__ int s_bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = (int)(blockDim.x >> 5);
    // seg lanes per estimate (a half-warp while nb <= 16, so a warp takes two)
    const int seg = nb <= 16 ? 16 : 32, per = 32 / seg, r = lane % seg, half = lane / seg;
    const R tol = aberth_tol<R>();
    const R floor_sub = mnrm * R(1e-20);
    if (tid < nb) {  // 1 / M(i, i-1) for i = tid >= 1; a vanishing entry is raised to floor_sub
        cplx<R> sb = tid ? M[tid + (tid - 1) * LDM] : cplx<R>{R(1), R(0)};
        if (!(fmax(fabs(sb.x), fabs(sb.y)) > floor_sub)) sb = cplx<R>{floor_sub, R(0)};
        s_inv[tid] = cdiv(cplx<R>{R(1), R(0)}, sb);
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int it = 0; it < kmax; ++it) {
        // every lane of a warp runs the same trip counts (the shuffles span the
        // warp); a segment past nb computes on a copy of estimate nb - 1 and
        // stores nothing
        for (int j0 = warp * per; j0 < nb; j0 += nw * per) {
            const int j = j0 + half;
            const cplx<R> mu = z[min(j, nb - 1)];
            cplx<R> s{0, 0}, ds{0, 0}, x{R(1), R(0)}, dx{0, 0};
#pragma unroll 2
            for (int i = nb - 1;; --i) {
                if (r <= i) {  // column i of (M - mu I) into rows 0 .. i
                    cplx<R> a = M[r + i * LDM];
                    if (r == i) a = a - mu;
                    cfma(ds, a, dx);
                    if (r == i) ds = ds - x;
                    cfma(s, a, x);
                }
                if (i == 0) break;
                const cplx<R> iv = s_inv[i];
                const cplx<R> xn = -(s * iv), dxn = -(ds * iv);  // meaningful on lane i of the segment
                x = cplx<R>{__shfl_sync(0xffffffffu, xn.x, i, seg), __shfl_sync(0xffffffffu, xn.y, i, seg)};
                dx = cplx<R>{__shfl_sync(0xffffffffu, dxn.x, i, seg), __shfl_sync(0xffffffffu, dxn.y, i, seg)};
                const R mag = fmax(fmax(fabs(x.x), fabs(x.y)), fmax(fabs(dx.x), fabs(dx.y)));
                const R f = mag > R(1099511627776.0) ? R(1.0 / 1099511627776.0)  // 2^40
                            : (mag > R(0) && mag < R(1.0 / 1099511627776.0)) ? R(1099511627776.0) : R(1);
                x = f * x; dx = f * dx; s = f * s; ds = f * ds;
            }
            const cplx<R> q = cdiv(s, ds);  // row 0 (lane 0 of the segment): p / p'
            const cplx<R> N{__shfl_sync(0xffffffffu, q.x, 0, seg), __shfl_sync(0xffffffffu, q.y, 0, seg)};
            cplx<R> part{0, 0};
            if (r < nb && r != j) part = cdiv(cplx<R>{R(1), R(0)}, mu - z[r]);
            for (int o = seg >> 1; o > 0; o >>= 1) {
                part.x += __shfl_xor_sync(0xffffffffu, part.x, o);
                part.y += __shfl_xor_sync(0xffffffffu, part.y, o);
            }
            const cplx<R> w = cdiv(N, cplx<R>{R(1), R(0)} - N * part);
            if (r == 0 && j < nb) s_w[j] = w;
        }
        __syncthreads();
        bool done = true;
        if (tid < nb) {
            const cplx<R> w = s_w[tid];
            const cplx<R> zn = z[tid] - w;
            if (!(isfinite(zn.x) && isfinite(zn.y))) s_bad = 1;
            done = hypot(w.x, w.y) <= tol * (hypot(zn.x, zn.y) + R(1e-3) * mnrm);
            z[tid] = zn;
        }
        const int all = __syncthreads_and(done);
        if (s_bad) return false;
        if (all) return true;
    }
    return false;
}

// Starting estimates for cta_aberth_shifts (one warp; lane q holds the
// q-th previous shift).  Warm start: the np shifts of the previous
// multishift sweep, whose trailing block ended dh rows lower (0 <= dh < nb);
// for each of the dh eigenvalues deflated since (defl) the nearest previous
// shift is dropped, then while more than nb remain the one farthest from
// every diagonal entry of M; the remaining places take diagonal entries of
// M moved apart by multiples of 1e-4 mnrm.  Cold start (np = 0): the
// diagonal of M moved by 1e-3 mnrm along the nb-th roots of unity.
template <class R>
__device__ __forceinline__ void warp_argbest(R &d, int &l, bool want_min)
{
    for (int o = 16; o > 0; o >>= 1) {
        const R od = __shfl_xor_sync(0xffffffffu, d, o);
        const int ol = __shfl_xor_sync(0xffffffffu, l, o);
        if ((want_min ? od < d : od > d) || (od == d && ol < l)) { d = od; l = ol; }
    }
}
template <class R, int LDM>
__device__ void warp_aberth_start(const cplx<R> *M, int nb, R mnrm, const cplx<R> *prev, int np, const cplx<R> *defl,
                                  int dh, cplx<R> *z)
{
    const int lane = threadIdx.x & 31;
    const cplx<R> c = lane < np ? prev[lane] : cplx<R>{0, 0};
    bool alive = lane < np;
    for (int q = 0; q < dh; ++q) {
        R d = alive ? abs2(c - defl[q]) : R(INFINITY);
        int l = lane;
        warp_argbest(d, l, true);
        if (d < R(INFINITY) && lane == l) alive = false;
    }
    int cnt = __popc(__ballot_sync(0xffffffffu, alive));
    while (cnt > nb) {
        R d = R(-1);
        if (alive) {
            d = abs2(c - M[0]);
            for (int i = 1; i < nb; ++i) d = fmin(d, abs2(c - M[i + i * LDM]));
        }
        int l = lane;
        warp_argbest(d, l, false);
        if (lane == l) alive = false;
        --cnt;
    }
    const unsigned am = __ballot_sync(0xffffffffu, alive);
    if (alive) z[__popc(am & ((1u << lane) - 1u))] = c;
    const int q = lane - cnt;  // places cnt .. nb-1
    if (q >= 0 && lane < nb) {
        const cplx<R> d = M[q + q * LDM];
        if (np > 0) {
            z[lane] = cplx<R>{d.x + R(q + 1) * R(1e-4) * mnrm, d.y};
        } else {
            R sn, cs;
            sincospi(R(2 * q) / R(nb), &sn, &cs);
            z[lane] = cplx<R>{d.x + R(1e-3) * mnrm * cs, d.y + R(1e-3) * mnrm * sn};
        }
    }
    __syncwarp();
}

// Complete Schur form of a small active block (m <= 32), one warp: single-
// shift QR with Wilkinson shifts (an exceptional shift every 10 sweeps
// without deflation) on the m x m block M in shared memory (leading
// dimension LDM), every rotation applied to the whole block (rows k, k+1
// from column k-1 on; columns k, k+1 down to row k+2) and accumulated into
// U (U <- U G^H, U = I on entry), until every subdiagonal entry is
// negligible (set to zero).  Then the rest of T needs only x <- x U (rows
// above the block, Schur vectors) and y <- U^H y (columns right of it).
// Returns false if some eigenvalue took more than kItMax sweeps.
template <class R, int LDM>
__device__ bool warp_tiny_schur(cplx<R> *M, cplx<R> *U, int m, int *sweeps, int *rots, const cplx<R> *cand = nullptr,
                                int ncand = 0)
{
    const int lane = threadIdx.x & 31;
    const R eps = num<R>::eps;
    int hi = m - 1, it = 0, nsw = 0, nrot = 0;
    bool ok = true;
    while (hi > 0) {
        bool small = false;
        if (lane >= 1 && lane <= hi) {
            const cplx<R> sub = M[lane + (lane - 1) * LDM];
            const R as = hypot(sub.x, sub.y);
            const cplx<R> a = M[lane + lane * LDM], b = M[(lane - 1) + (lane - 1) * LDM];
            small = as == R(0) || as <= eps * (hypot(a.x, a.y) + hypot(b.x, b.y));
        }
        const unsigned bal = __ballot_sync(0xffffffffu, small);
        const int lo = bal ? 31 - __clz(bal) : 0;
        __syncwarp();
        if (lo == hi) {
            if (lane == 0) M[hi + (hi - 1) * LDM] = cplx<R>{0, 0};
            --hi;
            it = 0;
            __syncwarp();
            continue;
        }
        if (lo > 0 && lane == 0) M[lo + (lo - 1) * LDM] = cplx<R>{0, 0};
        if (++it > kItMax) { ok = false; break; }
        ++nsw;
        cplx<R> mu;
        if (it % 10 == 0) {
            const cplx<R> sb = M[hi + (hi - 1) * LDM];
            mu = M[hi + hi * LDM];
            mu.x += R(0.75) * hypot(sb.x, sb.y);
        } else {
            mu = wilkinson(M[(hi - 1) + (hi - 1) * LDM], M[(hi - 1) + hi * LDM], M[hi + (hi - 1) * LDM],
                           M[hi + hi * LDM]);
            if (it == 1 && ncand > 0) {
                // first sweep on this bottom entry: the nearest of the given
                // estimates (shifts of the sweep that split this block off,
                // eigenvalue estimates of the whole matrix) replaces the
                // Wilkinson shift when both point at the same eigenvalue
                R db = R(INFINITY);
                cplx<R> zb = mu;
                for (int q = 0; q < ncand; ++q) {
                    const R dq = abs2(cand[q] - mu);
                    if (dq < db) { db = dq; zb = cand[q]; }
                }
                if (db <= R(1e-4) * abs2(mu)) mu = zb;
            }
        }
        __syncwarp();
        warp_sweep<R, LDM, true, false>(M, U, m, lo, hi, mu, &nrot);
    }
    *sweeps = nsw;
    *rots = nrot;
    return ok;
}

// Barrier among the NTH threads of the chase warps.
template <int NTH>
__device__ __forceinline__ void chase_bar()
{
    if constexpr (NTH == kQrThreads) __syncthreads();
    else asm volatile("bar.sync 1, %0;" ::"n"(NTH) : "memory");
}

// Slot of bulge g in one step's row of the rotation table: the bulges are
// split into kQrTpc runs of NB / kQrTpc consecutive bulges (one run per
// updating thread), and the table stores run position j = g mod run length
// major, so the kQrTpc threads of a segment read adjacent entries.
template <int NB>
__host__ __device__ __forceinline__ int rt_slot(int g)
{
    constexpr int NG = NB / kQrTpc;
    return (g % NG) * kQrTpc + g / NG;
}

// Apply one window's rotations (table rt, steps 0..ns-1) to a segment of
// indices kmin .. kmin + rr - 1 held at vec[i * STRIDE]; the rotation of
// step q, bulge g acts on i = off + q + 3 (NB - 1 - g) and i + 1, with
// off = kbase - kmin.  Bulge g moves in the steps q with
// t0 + q in [3 g, span - 1 + 3 g] (and g < nb).  LEFT: rows of a column
// (G [p; q]); otherwise columns of a row ([p q] G^H).
//
// The kQrTpc threads of a segment are consecutive lanes; thread sub takes
// the NG = NB / kQrTpc consecutive bulges g = sub NG + j.  At step q they
// span the L = 3 NG - 1 indices A(q) .. A(q) + L - 1, A(q) = A0 + q, which
// the thread keeps in a register ring (index i at ring[(i - A0) mod L]; the
// step loop is unrolled, so every ring index is a constant).  Each step the
// thread loads the one new index A(q) + L - 1 -- written by the thread with
// the bulges ahead at step q - 2 -- and stores A(q), which it no longer
// touches and the thread behind reads at step q + 2; one __syncwarp per
// step orders them.  All threads of the warp call this (on = false: no
// segment).  Returns false if a bulge's index range leaves [0, rr) (a
// malformed window: nothing is applied for that bulge).
template <class R, int NB, int STRIDE, bool LEFT, int TPC = kQrTpc>
__device__ __noinline__ bool apply_window(cplx<R> *vec, bool on, const RotLog<R> *rt, int ns, int off, int rr,
                                          int sub, int t0, int span, int nb)
{
    static_assert(NB % TPC == 0 && 32 % TPC == 0, "a segment's threads share a warp");
    constexpr int NG = NB / TPC, L = 3 * NG - 1 > 1 ? 3 * NG - 1 : 2, W = QrCfg<R>::W;
    const int A0 = off + 3 * (NB - NG * (sub + 1));
    int qa[NG], len[NG], slot[NG];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < NG; ++j) {
        const int g = sub * NG + j;
        slot[j] = rt_slot<NB>(g);  // the table is written in the kQrTpc layout
        const int a0 = max(0, 3 * g - t0), a1 = min(ns - 1, span - 1 + 3 * g - t0);
        qa[j] = a0;
        len[j] = (g < nb && a1 >= a0) ? a1 - a0 + 1 : 0;
        if (len[j]) {
            const int ia = off + a0 + 3 * (NB - 1 - g), ib = off + a1 + 3 * (NB - 1 - g);
            if (ia < 0 || ib > rr - 2) {
                len[j] = 0;
                ok = false;
            }
        }
    }
    cplx<R> ring[L];
#pragma unroll
    for (int i = 0; i < L - 1; ++i) {
        const int r = A0 + i;
        ring[i] = (on && r >= 0 && r < rr) ? vec[r * STRIDE] : cplx<R>{0, 0};
    }
#pragma unroll 32
    for (int q = 0; q < W; ++q) {
        if (q < ns) {
            if (on) {
                {  // the new bottom index A(q) + L - 1
                    const int r = A0 + q + L - 1;
                    ring[(q + L - 1) % L] = (r >= 0 && r < rr) ? vec[r * STRIDE] : cplx<R>{0, 0};
                }
#pragma unroll
                for (int j = 0; j < NG; ++j) {
                    if ((unsigned)(q - qa[j]) < (unsigned)len[j]) {
                        const RotLog<R> e = rt[q * NB + slot[j]];
                        const cplx<R> sv{e.sx, e.sy};
                        cplx<R> &p = ring[(q + 3 * (NG - 1 - j)) % L];
                        cplx<R> &w = ring[(q + 3 * (NG - 1 - j) + 1) % L];
                        const cplx<R> p0 = p, w0 = w;
                        if (LEFT) {
                            p = e.c * p0 + sv * w0;
                            w = e.c * w0 - conj(sv) * p0;
                        } else {
                            p = e.c * p0 + conj(sv) * w0;
                            w = e.c * w0 - sv * p0;
                        }
                    }
                }
                {  // A(q) is final for this thread
                    const int r = A0 + q;
                    if (r >= 0 && r < rr) vec[r * STRIDE] = ring[q % L];
                }
                if (q == ns - 1) {  // last step: the rest of the ring
#pragma unroll
                    for (int i = 1; i < L; ++i) {
                        const int r = A0 + q + i;
                        if (r >= 0 && r < rr) vec[r * STRIDE] = ring[(q + i) % L];
                    }
                }
            }
            __syncwarp();
        }
    }
    return ok;
}

// Loads through L2 only (ld.global.cg): in the cooperative chase, T, the
// rotation tables and the window records are written by other CTAs of the
// same grid, and L1 is not coherent across SMs.
template <class R> __device__ __forceinline__ cplx<R> ldcg_c(const cplx<R> *p);
template <> __device__ __forceinline__ cplx<float> ldcg_c<float>(const cplx<float> *p)
{
    const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    return cplx<float>{v.x, v.y};
}
template <> __device__ __forceinline__ cplx<double> ldcg_c<double>(const cplx<double> *p)
{
    const double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
    return cplx<double>{v.x, v.y};
}
template <class R> __device__ __forceinline__ RotLog<R> ldcg_rot(const RotLog<R> *p);
template <> __device__ __forceinline__ RotLog<float> ldcg_rot<float>(const RotLog<float> *p)
{
    const float4 v = __ldcg(reinterpret_cast<const float4 *>(p));
    return RotLog<float>{v.x, v.y, v.z, v.w};
}
template <> __device__ __forceinline__ RotLog<double> ldcg_rot<double>(const RotLog<double> *p)
{
    const double2 a = __ldcg(reinterpret_cast<const double2 *>(p)), b = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
    return RotLog<double>{a.x, a.y, b.x, b.y};
}
// T element into shared memory: asynchronous copy through L1 in the
// single-CTA chase, L2-coherent load in the cooperative one
template <class R, bool HELP>
__device__ __forceinline__ void load_t(cplx<R> *dst, const cplx<R> *src)
{
    if (HELP) *dst = ldcg_c<R>(src);
    else cp_async_elem<R>(dst, src);
}

static constexpr uint64_t kQrWaitNs = 2000000000ull;  // bounded inter-CTA waits (~2 s) unless the descriptor sets one

template <class R>
__device__ __forceinline__ uint64_t wait_limit(const SchurDesc<R> &d)
{
    return d.wait_ns ? (uint64_t)d.wait_ns : kQrWaitNs;
}

// Cooperative chase: one warp waits until each of the H <= 32 helpers has
// finished `target` windows, lane h watching helper h (one round trip to L2
// per poll instead of H in a row); false (warp-uniform) if a helper failed or
// the wait gave up.
template <class R>
__device__ bool warp_poll_helpers(const SchurDesc<R> &d, int H, int target)
{
    const int lane = threadIdx.x & 31;
    bool ok = true;
    if (lane < H) {
        volatile int *sy = d.sync;
        const uint64_t t0 = globaltimer_ns(), lim = wait_limit(d);
        while (sy[4 + lane] < target) {
            if (sy[2] || globaltimer_ns() - t0 > lim) { ok = false; break; }
            __nanosleep(128);  // keep the polls off the helpers' L2 lines
        }
    }
    ok = __all_sync(0xffffffffu, ok);
    __threadfence();
    return ok;
}

// Every thread of the calling CTA waits until each helper has finished
// `target` windows (warp 0 polls); false if a helper failed or the wait gave
// up.
template <class R>
__device__ bool wait_helpers(const SchurDesc<R> &d, int H, int target)
{
    __shared__ int s_ok;
    if (threadIdx.x < 32) {
        const bool ok = warp_poll_helpers(d, H, target);
        if (threadIdx.x == 0) s_ok = ok;
    }
    __syncthreads();
    const bool ok = s_ok != 0;
    __threadfence();
    __syncthreads();
    return ok;
}

// Helper CTA h of the cooperative chase: for every window the chase CTA
// posts (in order), the left rotations on the columns right of the next
// window's block and the right rotations on the rows above the window,
// restricted to the index groups it owns (groups of 8 consecutive indices,
// group g owned by helper g mod H; no other CTA writes them, so the windows
// need no ordering between helpers).  Then it publishes its count.
template <class R>
__device__ void qr_helper(const SchurDesc<R> &d, int H, int h, cplx<R> *tile, RotLog<R> *rt)
{
    using D = QrDims<R>;
    constexpr int W = D::W, NB = D::NB, RLD = D::RLD, CLD = D::CLD;
    constexpr int nt = kQrThreads;
    __shared__ int s_go, s_cnt, s_g, s_idx[kQrCh];
    __shared__ int s_win[12];
    const int tid = threadIdx.x, sub = tid % kQrTpc, seg = tid / kQrTpc;
    cplx<R> *T = d.T;
    const int ld = d.ld;
    for (int w = 0;; ++w) {
        if (tid == 0) {
            volatile int *sy = d.sync;
            const uint64_t t0 = globaltimer_ns(), lim = wait_limit(d);
            int go = 0;
            while (true) {
                if (sy[0] > w) { go = 1; break; }
                if (sy[1]) { go = 2; break; }
                if (sy[2] || globaltimer_ns() - t0 > lim) { go = 3; break; }
            }
            __threadfence();
            s_go = go;
        }
        __syncthreads();
        const int go = s_go;
        if (go != 1) {
            if (go == 3 && tid == 0) atomicExch(&d.sync[2], 1);
            return;
        }
        __threadfence();
        if (tid < 12) s_win[tid] = __ldcg(reinterpret_cast<const int *>(&d.win[__ldcg(d.postlist + w)]) + tid);
        __syncthreads();
        const int start = s_win[0], kbase = s_win[1], ns = s_win[2], kmin = s_win[3], rr = s_win[4];
        const int lo = s_win[5], hi = s_win[6], t0w = s_win[7], nb = s_win[8], r0 = s_win[9], rnext = s_win[10];
        for (int e = tid; e < W * NB; e += nt) rt[e] = ldcg_rot<R>(d.log + start + e);
        const int off = kbase - kmin;
        bool bad = false;
        // two passes: left rotations on columns (rnext, hi], right rotations
        // on rows [lo, r0); the owned indices are gathered 128 at a time
        for (int pass = 0; pass < 2; ++pass) {
            const int ilo = pass == 0 ? rnext + 1 : lo, ihi = pass == 0 ? hi : r0 - 1;
            if (ihi < ilo) continue;
            int g = ilo >> 3;
            g += ((h - g % H) % H + H) % H;
            while (g <= (ihi >> 3)) {
                __syncthreads();
                if (tid == 0) {
                    int cnt = 0, gg = g;
                    while (gg <= (ihi >> 3) && cnt + 8 <= kQrCh) {
                        for (int c = max(ilo, 8 * gg); c <= min(ihi, 8 * gg + 7); ++c) s_idx[cnt++] = c;
                        gg += H;
                    }
                    s_cnt = cnt;
                    s_g = gg;
                }
                __syncthreads();
                const int cn = s_cnt;
                g = s_g;
                if (pass == 0) {
                    for (int e = tid; e < rr * cn; e += nt) {
                        const int v = e % rr, j = e / rr;
                        tile[v + j * RLD] = ldcg_c<R>(&T[(kmin + v) + (int64_t)s_idx[j] * ld]);
                    }
                    __syncthreads();
                    if (!apply_window<R, NB, 1, true>(tile + seg * RLD, seg < cn, rt, ns, off, rr, sub, t0w, hi - lo, nb))
                        bad = true;
                    __syncthreads();
                    for (int e = tid; e < rr * cn; e += nt) {
                        const int v = e % rr, j = e / rr;
                        T[(kmin + v) + (int64_t)s_idx[j] * ld] = tile[v + j * RLD];
                    }
                } else {
                    for (int e = tid; e < cn * rr; e += nt) {
                        const int a = e % cn, v = e / cn;
                        tile[a + v * CLD] = ldcg_c<R>(&T[s_idx[a] + (int64_t)(kmin + v) * ld]);
                    }
                    __syncthreads();
                    if (!apply_window<R, NB, CLD, false>(tile + seg, seg < cn, rt, ns, off, rr, sub, t0w, hi - lo, nb))
                        bad = true;
                    __syncthreads();
                    for (int e = tid; e < cn * rr; e += nt) {
                        const int a = e % cn, v = e / cn;
                        T[s_idx[a] + (int64_t)(kmin + v) * ld] = tile[a + v * CLD];
                    }
                }
            }
        }
        if (bad) atomicExch(d.status, 7);
        __threadfence();
        __syncthreads();
        if (tid == 0) atomicExch(&d.sync[4 + h], w + 1);
    }
}

template <class R, bool HELP>
__global__ void __launch_bounds__(kQrThreads, 1)
qr_chase_kernel(const SchurDesc<R> *__restrict__ descs, int H)
{
    using D = QrDims<R>;
    constexpr int W = D::W, NB = D::NB, BLD = D::BLD, RLD = D::RLD, CLD = D::CLD;
    extern __shared__ __align__(16) unsigned char smraw[];
    cplx<R> *blk = reinterpret_cast<cplx<R> *>(smraw);   // window block, blk[a + b BLD]
    cplx<R> *tile = blk + D::BW * BLD;                     // (a')/(b') staging
    RotLog<R> *rt = reinterpret_cast<RotLog<R> *>(tile + D::TILE);  // rt[q NB + g]
    __shared__ cplx<R> s_mu[NB];
    __shared__ cplx<R> s_m[NB * (NB + 1)];
    __shared__ cplx<R> s_prev[NB], s_defl[NB];  // the last multishift sweep's shifts; eigenvalues deflated since
    __shared__ R s_mnrm;
    __shared__ int s_prevn, s_prevhi, s_prefail;
    __shared__ int s_lo, s_hi, s_iter, s_status, s_done, s_nb, s_sweeps, s_stop, s_nwin, s_nlog, s_small, s_bad, s_npost,
        s_tiny;
    __shared__ long long s_uoff, s_rots, s_work;

    const SchurDesc<R> d = descs[HELP ? 0 : blockIdx.x];
    if (HELP && blockIdx.x > 0) {
        qr_helper<R>(d, H, (int)blockIdx.x - 1, tile, rt);
        return;
    }
    const int n = d.n, ld = d.ld;
    cplx<R> *T = d.T;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nt = kQrThreads;
    const int sub = tid % kQrTpc, seg = tid / kQrTpc;
    const R eps = num<R>::eps;
    int *st = d.state;
    auto ldT = [&](int64_t idx) { return HELP ? ldcg_c<R>(T + idx) : T[idx]; };
    if (st[2]) {  // already finished: nothing new in the log
        if (tid == 0) {
            st[3] = 0; st[7] = 0; d.rstate[0] = 0;
            if (HELP) atomicExch(&d.sync[1], 1);
        }
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
        s_work = (long long)st[8] + ((long long)st[9] << 31);
        s_stop = 0;
        s_bad = 0;
        s_npost = 0;
        s_prevn = 0;
        s_prevhi = 0;
    }
    __syncthreads();

    while (true) {
        const int hi = s_hi;
        if (hi <= 0) { if (tid == 0) s_done = 1; break; }
        if (tid == 0) s_lo = 0;
        __syncthreads();
        for (int k = 1 + tid; k <= hi; k += nt) {
            cplx<R> sub_ = ldT(k + (int64_t)(k - 1) * ld);
            R as = hypot(sub_.x, sub_.y);
            cplx<R> a = ldT(k + (int64_t)k * ld), b = ldT((k - 1) + (int64_t)(k - 1) * ld);
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
            int nb = min(NB, max(1, (m - 2) / 4));
            s_tiny = m <= kQrTiny;
            const long long nwin_sweep = s_tiny ? 1 : ((hi - lo) + 3 * (nb - 1) + W - 1) / W;
            const bool fits = s_nlog + nwin_sweep * (W * NB) <= d.log_cap && s_nwin + nwin_sweep <= d.win_cap &&
                              s_uoff + nwin_sweep * (long long)(D::RR * D::RR) <= d.u_cap;
            s_small = 0;
            if (!fits) {
                s_stop = 1;  // drain the log first
                if (s_nlog == 0 && s_nwin == 0 && s_uoff == 0) s_status = 7;  // can never fit
            } else {
                if (lo > 0) T[lo + (int64_t)(lo - 1) * ld] = cplx<R>{0, 0};
            }
            if (fits && !s_tiny) {
                int it = ++s_iter;
                ++s_sweeps;
                if (it > kItMax) s_status = 3;
                if (it % 10 == 0) {
                    nb = 1;
                    cplx<R> sb = ldT(hi + (int64_t)(hi - 1) * ld);
                    cplx<R> mu = ldT(hi + (int64_t)hi * ld);
                    mu.x += R(0.75) * hypot(sb.x, sb.y);
                    s_mu[0] = mu;
                } else if (nb == 1) {
                    s_mu[0] = wilkinson(ldT((hi - 1) + (int64_t)(hi - 1) * ld), ldT((hi - 1) + (int64_t)hi * ld),
                                        ldT(hi + (int64_t)(hi - 1) * ld), ldT(hi + (int64_t)hi * ld));
                } else {
                    s_small = 1;
                }
                s_nb = nb;
                s_rots += (long long)(hi - lo) * nb;
                // in-block work: each rotation of the sweep updates two rows and
                // two columns of the active block, about m element pairs
                s_work += (long long)(hi - lo) * nb * (long long)m;
            }
        }
        __syncthreads();
        if (s_stop || s_status) break;
        if (s_tiny) {
            // a small active block: only recorded here, as one window with a
            // dense U (pad = 1; nb = number of shift estimates, the last
            // sweep's shifts, stored at the window's log entries);
            // qr_tiny_kernel gives it its whole Schur form after this launch,
            // before the deferred passes, while the chase goes on with the
            // blocks above (in the cooperative chase the helpers are done with
            // every window that touched it: they were waited for at the end of
            // the sweep that split it off)
            const int m = hi - lo + 1;
            const int nc = s_prevn;
            if (tid < nc) d.log[s_nlog + tid] = RotLog<R>{R(0), s_prev[tid].x, s_prev[tid].y, R(0)};
            if (tid == 0) {
                WinRec wr;
                wr.start = s_nlog; wr.kbase = lo; wr.nsteps = -1; wr.kmin = lo; wr.rr = m;
                wr.lo = lo; wr.hi = hi; wr.t0 = 0; wr.nb = nc; wr.r0 = lo; wr.rnext = hi; wr.pad = 1;
                wr.uoff = s_uoff;
                d.win[s_nwin] = wr;
                s_nwin += 1;
                s_uoff += (long long)m * m;
                s_nlog += NB;
                s_hi = lo - 1;
                s_iter = 0;
            }
            __syncthreads();
            continue;
        }
        const int nb = s_nb;
        if (s_small) {  // shifts: eigenvalues of the trailing nb x nb block
            // the block is fetched by the whole CTA (one round trip to L2
            // instead of a warp's nb*nb/32 dependent ones).  Its eigenvalues
            // come from the Ehrlich-Aberth iteration, started from the
            // previous sweep's shifts when its trailing block ended less
            // than nb rows lower; if that fails, one warp computes them by
            // single-shift QR.
            const int b0 = hi - nb + 1;
            if (tid == 0) s_mnrm = R(0);
            for (int e = tid; e < nb * nb; e += nt) {
                const int i = e % nb, j = e / nb;
                s_m[i + j * (NB + 1)] = (i <= j + 1) ? ldT((b0 + i) + (int64_t)(b0 + j) * ld) : cplx<R>{0, 0};
            }
            const int dh = s_prevhi - hi;
            const bool warm = s_prevn > 0 && dh >= 0 && dh < nb;
            if (warm && tid < dh) s_defl[tid] = ldT((hi + 1 + tid) + (int64_t)(hi + 1 + tid) * ld);
            __syncthreads();
            if (warp == 0) {
                R mx = R(0);
                for (int e = lane; e < nb * nb; e += 32) {
                    const cplx<R> v = s_m[(e % nb) + (e / nb) * (NB + 1)];
                    mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
                }
                for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                if (lane == 0) s_mnrm = mx;
            }
            __syncthreads();
            if (warp == 0) warp_aberth_start<R, NB + 1>(s_m, nb, s_mnrm, s_prev, warm ? s_prevn : 0, s_defl, warm ? dh : 0, s_mu);
            __syncthreads();
            if (!cta_aberth_shifts<R, NB + 1>(s_m, nb, s_mu, s_mnrm, kAberthIt)) {
                if (warp == 0) warp_small_eigvals<R, NB + 1>(s_m, nb, s_mu);
                __syncthreads();
            }
            if (tid < nb) s_prev[tid] = s_mu[tid];
            if (tid == 0) {
                s_prevn = nb;
                s_prevhi = hi;
            }
            __syncthreads();
        }
        const int nsteps = (hi - lo) + 3 * (nb - 1);

        for (int t0 = 0; t0 < nsteps; t0 += W) {
            const int t1 = min(t0 + W, nsteps), ns = t1 - t0;
            const int kmin = max(lo, lo + t0 - 3 * (nb - 1));
            const int kmax = min(hi - 1, lo + t1 - 1);
            const int r0 = max(lo, kmin - 1);
            const int r1 = min(hi, kmax + 2);
            const int bw = r1 - r0 + 1, rr = kmax + 2 - kmin;
            const int kbase = lo + t0 - 3 * (NB - 1);
            if (bw > D::BW || rr > D::RR) {  // cannot happen; guards the shared-memory bounds
                if (tid == 0) s_status = 7;
                __syncthreads();
                break;
            }
            // only the band a <= b + 2 (Hessenberg part and bulge entries):
            // the chase never reads or writes the block below it
            for (int b = warp; b < bw; b += nt / 32)
                for (int a = lane; a <= min(b + 2, bw - 1); a += 32)
                    load_t<R, HELP>(&blk[a + b * BLD], &T[(r0 + a) + (int64_t)(r0 + b) * ld]);
            for (int e = tid; e < W * NB; e += nt) rt[e] = RotLog<R>{R(1), R(0), R(0), R(0)};
            // last column of the next window's block (hi after the last window)
            const int rnext = (t1 < nsteps) ? min(hi, min(hi - 1, lo + min(t1 + W, nsteps) - 1) + 2) : hi;
            // cooperative chase: windows with more than kQrPostMin rows and
            // columns outside the next block go to the helpers (the chase CTA
            // then updates only the next block's new columns (r1, rnext]);
            // smaller ones are done here after the helpers have finished every
            // posted window, so each entry still sees the windows in order
            const bool post = HELP && (hi - rnext) + (r0 - lo) > kQrPostMin;
            // a posted window's new columns (at most W) are read during the
            // chase by the warps that do not chase, once the helpers are done
            // with every window posted before this one
            const int pre_cn = post ? rnext - r1 : 0;
            if (tid == 0) s_prefail = 0;
            cp_async_wait_all();
            __syncthreads();
            // the chase: half-warp h of warp w moves bulge g = 2 w + h.  Each
            // bulge's rotation depends only on entries its own previous step
            // wrote, so all 16 lanes compute it redundantly; left rotations of
            // one step touch disjoint rows and right rotations disjoint
            // columns, so one barrier after each phase orders the bulges.
            if (warp < NB / 2) {
                constexpr int NI = (D::BW + 15) / 16;
                const int hl = lane & 15;
                const int g = 2 * warp + (lane >> 4);
                for (int t = t0; t < t1; ++t) {
                    const int k = lo + t - 3 * g;
                    const bool act = g < nb && k >= lo && k < hi;  // uniform per half-warp
                    const int kk = k - r0;
                    // left rotation of rows kk, kk+1 from column cstart on; x and y
                    // (their entries in column cstart) are read by every lane of the
                    // half at once, off the critical path of the row loads
                    const int cstart = (k == lo) ? kk : kk - 1;
                    const int ni = act ? (bw - cstart + 15) >> 4 : 0;
                    cplx<R> x{1, 0}, y{0, 0};
                    if (act) {
                        x = blk[kk + cstart * BLD];
                        y = blk[(kk + 1) + cstart * BLD];
                    }
                    cplx<R> p[NI], q[NI];
#pragma unroll
                    for (int i = 0; i < NI; ++i) {
                        const int b = cstart + hl + 16 * i;
                        if (i < ni && b < bw) {
                            p[i] = blk[kk + b * BLD];
                            q[i] = blk[(kk + 1) + b * BLD];
                        } else {
                            p[i] = cplx<R>{1, 0};
                            q[i] = cplx<R>{0, 0};
                        }
                    }
                    if (act && k == lo) x = x - s_mu[g];
                    R c = R(1);
                    cplx<R> s{0, 0}, r{0, 0};
                    if (act) givens_fast(x, y, c, s, r);
#pragma unroll
                    for (int i = 0; i < NI; ++i) {
                        const int b = cstart + hl + 16 * i;
                        if (i < ni && b < bw) {
                            cplx<R> np = c * p[i] + s * q[i], nq = c * q[i] - conj(s) * p[i];
                            if (i == 0 && hl == 0 && k > lo) {  // the annihilated bulge entry
                                np = r;
                                nq = cplx<R>{0, 0};
                            }
                            blk[kk + b * BLD] = np;
                            blk[(kk + 1) + b * BLD] = nq;
                        }
                    }
                    if (act && hl == 0) rt[(t - t0) * NB + rt_slot<NB>(g)] = RotLog<R>{c, s.x, s.y, R(1)};
                    chase_bar<NB * 16>();
                    // right rotation: columns kk, kk+1, block rows up to kk+2
                    const int rend = min(kk + 2, bw - 1);
                    const int nr = act ? (rend + 16) >> 4 : 0;
#pragma unroll
                    for (int i = 0; i < NI; ++i) {
                        const int a = hl + 16 * i;
                        if (i < nr && a <= rend) {
                            p[i] = blk[a + kk * BLD];
                            q[i] = blk[a + (kk + 1) * BLD];
                        }
                    }
#pragma unroll
                    for (int i = 0; i < NI; ++i) {
                        const int a = hl + 16 * i;
                        if (i < nr && a <= rend) {
                            blk[a + kk * BLD] = c * p[i] + conj(s) * q[i];
                            blk[a + (kk + 1) * BLD] = c * q[i] - s * p[i];
                        }
                    }
                    chase_bar<NB * 16>();
                }
                if (pre_cn > 0) {
                    // a posted window: the chasing warps store the block band and
                    // the rotation table and post the window at once, while the
                    // other warps may still wait for the helpers
                    constexpr int NCH = NB * 16;
                    for (int b = warp; b < bw; b += NCH / 32)
                        for (int a = lane; a <= min(b + 2, bw - 1); a += 32)
                            T[(r0 + a) + (int64_t)(r0 + b) * ld] = blk[a + b * BLD];
                    RotLog<R> *dst = d.log + s_nlog;
                    for (int e = tid; e < W * NB; e += NCH) dst[e] = rt[e];
                    if (tid == 0) {
                        WinRec wr;
                        wr.start = s_nlog; wr.kbase = kbase; wr.nsteps = ns; wr.kmin = kmin; wr.rr = rr;
                        wr.lo = lo; wr.hi = hi; wr.t0 = t0; wr.nb = nb; wr.r0 = r0; wr.rnext = rnext; wr.pad = 0;
                        wr.uoff = s_uoff;
                        d.win[s_nwin] = wr;
                        d.postlist[s_npost] = s_nwin;
                    }
                    __threadfence();
                    chase_bar<NCH>();
                    if (tid == 0) atomicExch(&d.sync[0], s_npost + 1);
                }
            } else if (pre_cn > 0) {
                constexpr int NPRE = kQrThreads - NB * 16;  // threads of the warps that do not chase
                static_assert(NPRE >= 32, "the prefetch needs a warp");
                if (warp == NB / 2 && !warp_poll_helpers(d, H, s_npost) && lane == 0) s_prefail = 1;
                asm volatile("bar.sync 2, %0;" ::"n"(NPRE) : "memory");
                if (!s_prefail) {
                    const int pt = tid - NB * 16;
                    for (int e = pt; e < rr * pre_cn; e += NPRE) {
                        const int v = e % rr, j = e / rr;
                        tile[v + j * RLD] = ldcg_c<R>(&T[(kmin + v) + (int64_t)(r1 + 1 + j) * ld]);
                    }
                }
            }
            __syncthreads();
            if (s_prefail) {
                if (tid == 0) s_status = 6;
                __syncthreads();
                break;
            }
            const int off = kbase - kmin;
            if (pre_cn == 0) {  // (a prefetched window is stored and posted already)
                for (int b = warp; b < bw; b += nt / 32)
                    for (int a = lane; a <= min(b + 2, bw - 1); a += 32)
                        T[(r0 + a) + (int64_t)(r0 + b) * ld] = blk[a + b * BLD];
                RotLog<R> *dst = d.log + s_nlog;
                for (int e = tid; e < W * NB; e += nt) dst[e] = rt[e];
            }
            if (HELP && pre_cn == 0) {
                if (post && tid == 0) {
                    WinRec wr;
                    wr.start = s_nlog; wr.kbase = kbase; wr.nsteps = ns; wr.kmin = kmin; wr.rr = rr;
                    wr.lo = lo; wr.hi = hi; wr.t0 = t0; wr.nb = nb; wr.r0 = r0; wr.rnext = rnext; wr.pad = 0;
                    wr.uoff = s_uoff;
                    d.win[s_nwin] = wr;
                    d.postlist[s_npost] = s_nwin;
                }
                __threadfence();
                __syncthreads();
                if (post && tid == 0) atomicExch(&d.sync[0], s_npost + 1);
                // helpers done with every window posted before this one (all of
                // them if this one is done here; for a posted one the warps that
                // prefetched its new columns have waited for that already)
                if (!wait_helpers(d, H, s_npost)) {
                    if (tid == 0) s_status = 6;
                    __syncthreads();
                    break;
                }
            }
            // (a') columns r1+1 .. hi (cooperative, posted: .. rnext), rows kmin .. kmin+rr-1: left rotations
            const int aend = post ? rnext : hi;
            for (int c0 = r1 + 1; c0 <= aend; c0 += kQrCh) {
                const int cn = min(kQrCh, aend - c0 + 1);
                if (pre_cn == 0)  // else the tile holds them already (one chunk: cn = pre_cn)
                    for (int e = tid; e < rr * cn; e += nt) {
                        const int v = e % rr, j = e / rr;
                        load_t<R, HELP>(&tile[v + j * RLD], &T[(kmin + v) + (int64_t)(c0 + j) * ld]);
                    }
                cp_async_wait_all();
                __syncthreads();
                if (post) {
                    // at most W new columns: up to 16 threads (one bulge each) per column
                    constexpr int HT = NB < 16 ? NB : 16;
                    if (!apply_window<R, NB, 1, true, HT>(tile + (tid / HT) * RLD, (tid / HT) < cn, rt, ns, off, rr,
                                                          tid % HT, t0, hi - lo, nb))
                        s_bad = 1;
                } else if (!apply_window<R, NB, 1, true>(tile + seg * RLD, seg < cn, rt, ns, off, rr, sub, t0, hi - lo,
                                                         nb)) {
                    s_bad = 1;
                }
                __syncthreads();
                for (int e = tid; e < rr * cn; e += nt) {
                    const int v = e % rr, j = e / rr;
                    T[(kmin + v) + (int64_t)(c0 + j) * ld] = tile[v + j * RLD];
                }
                __syncthreads();
            }
            // (b') rows lo .. r0-1, columns kmin .. kmin+rr-1: right rotations
            // (the helpers' part for a posted window)
            for (int i0 = lo; i0 < (post ? lo : r0); i0 += kQrCh) {
                const int rn = min(kQrCh, r0 - i0);
                for (int e = tid; e < rn * rr; e += nt) {
                    const int a = e % rn, v = e / rn;
                    load_t<R, HELP>(&tile[a + v * CLD], &T[(i0 + a) + (int64_t)(kmin + v) * ld]);
                }
                cp_async_wait_all();
                __syncthreads();
                if (!apply_window<R, NB, CLD, false>(tile + seg, seg < rn, rt, ns, off, rr, sub, t0, hi - lo, nb))
                    s_bad = 1;
                __syncthreads();
                for (int e = tid; e < rn * rr; e += nt) {
                    const int a = e % rn, v = e / rn;
                    T[(i0 + a) + (int64_t)(kmin + v) * ld] = tile[a + v * CLD];
                }
                __syncthreads();
            }
            if (tid == 0) {
                if (post) ++s_npost;
                if (!post) {
                    WinRec wr;
                    wr.start = s_nlog; wr.kbase = kbase; wr.nsteps = ns; wr.kmin = kmin; wr.rr = rr;
                    wr.lo = lo; wr.hi = hi; wr.t0 = t0; wr.nb = nb; wr.r0 = r0; wr.rnext = rnext; wr.pad = 0;
                    wr.uoff = s_uoff;
                    d.win[s_nwin] = wr;
                }
                s_nwin += 1;
                s_uoff += (long long)rr * rr;
                s_nlog += W * NB;
                if (s_bad) s_status = 7;
            }
            if (HELP) __threadfence();  // the block and head columns, before the next block is read back
            __syncthreads();
        }
        __syncthreads();
        // cooperative chase: the whole sweep's out-of-window updates are done
        // before the next sweep reads T
        if (HELP && !s_status && !wait_helpers(d, H, s_npost)) {
            if (tid == 0) s_status = 6;
            __syncthreads();
        }
        if (s_status) break;
    }
    __syncthreads();
    if (tid == 0) {
        st[0] = s_hi;
        st[1] = s_iter;
        st[2] = (s_done || s_status) ? 1 : 0;
        st[3] = s_nlog;
        st[7] = s_nwin;
        d.rstate[0] = s_nwin;
        st[4] = s_sweeps;
        st[5] = (int)(s_rots & 0x7fffffff);
        st[6] = (int)(s_rots >> 31);
        st[8] = (int)(s_work & 0x7fffffff);
        st[9] = (int)(s_work >> 31);
        if (s_status) *d.status = s_status;
        if (HELP) {
            __threadfence();
            atomicExch(&d.sync[1], 1);  // helpers leave once every posted window is done
        }
        if (d.counters) {
            d.counters[0] = s_sweeps;
            d.counters[1] = st[5];
            d.counters[2] = st[6];
            d.counters[3] = st[8];
            d.counters[4] = st[9];
        }
    }
}

// The small active blocks that the chase recorded without solving them
// (window records with nsteps < 0 and pad = 1): the complete Schur form of
// each by one warp, written back into T, with its accumulated rotations as
// the window's dense U.  Launched after the chase launch that recorded them
// and before the deferred passes that apply those U.  A recorded block
// [lo, hi] is final when it is recorded, and nothing the chase does
// afterwards reaches inside it: the later active blocks lie above it, their
// in-window and helper updates stay within them, and their out-of-block
// updates are the deferred passes, which touch T only in rows above lo or
// columns right of a window's hi; rows above lo in columns lo..hi receive
// both this block's right rotations and the later windows' left rotations,
// which commute.  CTAs of one warp, each taking the window records
// blockIdx.x, blockIdx.x + gridDim.x, ... of the round.
template <class R>
__global__ void __launch_bounds__(32) qr_tiny_kernel(const SchurDesc<R> *__restrict__ descs)
{
    constexpr int NB = QrCfg<R>::NB;
    __shared__ cplx<R> M[kQrTiny * kQrTinyLd], U[kQrTiny * kQrTinyLd], cand[NB];
    const SchurDesc<R> d = descs[blockIdx.y];
    const int nwin = d.rstate[0], ld = d.ld, lane = threadIdx.x;
    for (int wi = blockIdx.x; wi < nwin; wi += gridDim.x) {
        const WinRec w = d.win[wi];
        if (w.nsteps >= 0 || w.pad != 1) continue;
        const int m = w.rr, lo = w.lo;
        if (m < 1 || m > kQrTiny || lo < 0 || lo + m > d.n) {
            if (lane == 0) atomicExch(d.status, 7);
            continue;
        }
        __syncwarp();  // the previous block's shared-memory reads are done
        for (int e = lane; e < m * m; e += 32) {
            const int a = e % m, b = e / m;
            M[a + b * kQrTinyLd] = d.T[(lo + a) + (int64_t)(lo + b) * ld];
            U[a + b * kQrTinyLd] = cplx<R>{(R)(a == b), R(0)};
        }
        const int nc = min(max(w.nb, 0), NB);
        if (lane < nc) {
            const RotLog<R> e = d.log[w.start + lane];
            cand[lane] = cplx<R>{e.sx, e.sy};
        }
        __syncwarp();
        int nsw = 0, nrot = 0;
        const bool ok = warp_tiny_schur<R, kQrTinyLd>(M, U, m, &nsw, &nrot, cand, nc);
        __syncwarp();
        cplx<R> *Ug = d.ubuf + w.uoff;
        for (int e = lane; e < m * m; e += 32) {
            const int a = e % m, b = e / m;
            d.T[(lo + a) + (int64_t)(lo + b) * ld] = M[a + b * kQrTinyLd];
            Ug[a + b * m] = U[a + b * kQrTinyLd];
        }
        if (lane == 0) {
            if (!ok) atomicExch(d.status, 3);
            if (d.counters) {
                atomicAdd(&d.counters[5], nsw);
                atomicAdd(&d.counters[6], nrot);
            }
        }
    }
}

// Accumulated product of one window's rotations: U = I G_1^H G_2^H ... (the
// right rotations in log order applied to the rows of I).  Then a row
// segment x (indices kmin .. kmin+rr-1) receiving the window's right
// rotations becomes x U, and a column segment y receiving its left rotations
// becomes U^H y.  CTA x takes the windows x, x + gridDim.x, ... (one each
// when the grid covers the round's windows); thread r owns row r of U.
template <class R>
__global__ void __launch_bounds__(128) qr_build_u_kernel(const SchurDesc<R> *__restrict__ descs)
{
    using D = QrDims<R>;
    constexpr int W = D::W, NB = D::NB, ULD = D::RR + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    RotLog<R> *lg = reinterpret_cast<RotLog<R> *>(smraw);
    cplx<R> *u = reinterpret_cast<cplx<R> *>(lg + W * NB);
    const SchurDesc<R> d = descs[blockIdx.y];
    const int nwin = d.rstate[0];
    for (int wi = blockIdx.x; wi < nwin; wi += gridDim.x) {
    __syncthreads();  // the previous window's shared-memory reads are done
    const WinRec w = d.win[wi];
    if (w.nsteps < 0) continue;  // a small block: U written by qr_tiny_kernel
    const int rr = w.rr, r = threadIdx.x;
    if (rr > D::RR || rr < 2) {
        if (r == 0) atomicExch(d.status, 7);
        continue;
    }
    for (int e = threadIdx.x; e < W * NB; e += blockDim.x) lg[e] = d.log[w.start + e];
    if (r < rr)
        for (int c = 0; c < rr; ++c) u[r * ULD + c] = cplx<R>{(R)(r == c), R(0)};
    __syncthreads();
    if (r < rr) {
        cplx<R> *row = u + r * ULD;
        const int off = w.kbase - w.kmin;
        bool bad = false;
        for (int q = 0; q < w.nsteps; ++q) {
#pragma unroll
            for (int g = 0; g < NB; ++g) {
                const RotLog<R> e = lg[q * NB + rt_slot<NB>(g)];
                if (e.act == R(0)) continue;
                const int a = off + q + 3 * (NB - 1 - g);
                if ((unsigned)a > (unsigned)(rr - 2)) { bad = true; continue; }
                const cplx<R> sv{e.sx, e.sy};
                const cplx<R> p = row[a], qv = row[a + 1];
                row[a] = e.c * p + conj(sv) * qv;
                row[a + 1] = e.c * qv - sv * p;
            }
        }
        if (bad) atomicExch(d.status, 7);
    }
    __syncthreads();
    cplx<R> *U = d.ubuf + w.uoff;
    for (int e = threadIdx.x; e < rr * rr; e += blockDim.x) {
        const int q = e % rr, c = e / rr;  // U(q, c), column-major
        U[e] = u[q * ULD + c];
    }
    }
}

// Deferred right rotations on rows (Schur vectors Z: every window; rows of T
// above the window's active block: i < lo): x <- x U_w for each window in
// order.  A CTA holds rpc rows in shared memory.
template <class R>
__global__ void __launch_bounds__(256)
qr_apply_rows_kernel(const SchurDesc<R> *__restrict__ descs, int rpc, int ctas_t)
{
    constexpr int RRMAX = QrDims<R>::RR;
    extern __shared__ unsigned char smraw[];
    const SchurDesc<R> d = descs[blockIdx.y];
    const int n = d.n, ld = d.ld;
    const int nwin = d.rstate[0];
    if (nwin == 0) return;
    const bool isT = blockIdx.x < ctas_t;
    const int cb = isT ? blockIdx.x : blockIdx.x - ctas_t;
    const int i0 = cb * rpc;
    if (i0 >= n) return;
    const int rn = min(rpc, n - i0);
    cplx<R> *M = isT ? d.T : d.Q;
    cplx<R> *buf = reinterpret_cast<cplx<R> *>(smraw);          // rpc x n, buf[r + c rpc]
    cplx<R> *ub[2] = {buf + (size_t)rpc * n, buf + (size_t)rpc * n + RRMAX * RRMAX};
    // T rows: column c was changed in rows i < lmax[c] (the windows' lo);
    // only those entries are written back (the rest may belong to a later
    // active block that the chase is updating meanwhile)
    int *lmax = reinterpret_cast<int *>(ub[1] + RRMAX * RRMAX);
    for (int c = threadIdx.x; c < n; c += blockDim.x) lmax[c] = 0;
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
                if (r == 0) lmax[w.kmin + c] = max(lmax[w.kmin + c], w.lo);
            }
        }
        wi = wn;
        par ^= 1;
    }
    cp_async_wait_all();
    __syncthreads();
    for (int e = threadIdx.x; e < rn * n; e += blockDim.x) {
        const int a = e % rn, b = e / rn;
        if (!isT || i0 + a < lmax[b]) M[(i0 + a) + (int64_t)b * ld] = buf[a + b * rpc];
    }
}

// Deferred left rotations on columns of T right of the window's active block
// (j > hi): y <- U_w^H y for each window in order.  Runs after the rows pass.
template <class R>
__global__ void __launch_bounds__(256)
qr_apply_cols_kernel(const SchurDesc<R> *__restrict__ descs, int cpc)
{
    constexpr int RRMAX = QrDims<R>::RR;
    extern __shared__ unsigned char smraw[];
    const SchurDesc<R> d = descs[blockIdx.y];
    const int n = d.n, ld = d.ld;
    const int nwin = d.rstate[0];
    if (nwin == 0) return;
    const int j0 = blockIdx.x * cpc;
    if (j0 >= n) return;
    const int cn = min(cpc, n - j0);
    const int cs = n + 1;
    cplx<R> *buf = reinterpret_cast<cplx<R> *>(smraw);           // column jl at buf + jl cs
    cplx<R> *ub[2] = {buf + (size_t)cs * cpc, buf + (size_t)cs * cpc + RRMAX * RRMAX};
    // row i was changed in columns j > hmin[i] (the windows' hi); only those
    // entries are written back
    int *hmin = reinterpret_cast<int *>(ub[1] + RRMAX * RRMAX);
    for (int i = threadIdx.x; i < n; i += blockDim.x) hmin[i] = n;
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
                if (jl == 0) hmin[w.kmin + c] = min(hmin[w.kmin + c], w.hi);
            }
        }
        wi = wn;
        par ^= 1;
    }
    cp_async_wait_all();
    __syncthreads();
    for (int e = threadIdx.x; e < cn * n; e += blockDim.x) {
        const int a = e % n, b = e / n;
        if (j0 + b > hmin[a]) d.T[a + (int64_t)(j0 + b) * ld] = buf[a + (size_t)b * cs];
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
        for (int q = 1; q < kQrStateInts; ++q) st[q] = 0;
        // the small-block counts that qr_tiny_kernel adds up
        if (int *c = descs[b].counters) c[5] = c[6] = 0;
    }
}

// A matrix whose iteration did not finish within the round limit gets the
// iteration-cap status.
template <class R>
__global__ void qr_mark_unfinished_kernel(const SchurDesc<R> *__restrict__ descs, int batch)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < batch; b += gridDim.x * blockDim.x)
        if (!descs[b].state[2]) atomicExch(descs[b].status, 3);
}

template <class R>
int qr_rows_per_cta(int nmax, int batch)
{
    constexpr int RRMAX = QrDims<R>::RR;
    size_t per = (size_t)(std::max(nmax, 1) + 1) * sizeof(cplx<R>);
    size_t avail = 200 * 1024 - 2 * (size_t)RRMAX * RRMAX * sizeof(cplx<R>) - (size_t)std::max(nmax, 1) * sizeof(int);
    size_t r = avail / per;
    // one matrix: about 128 row blocks, as the passes of the last round are
    // not overlapped with a chase and should spread over many SMs; a batch:
    // about 8 CTAs per SM over all matrices, since every CTA reads each
    // window's rotation product once, whatever its number of rows
    const size_t want = batch > 1 ? (size_t)cdiv_i((int64_t)std::max(nmax, 1) * batch, 152 * 8)
                                  : (size_t)cdiv_i(std::max(nmax, 1), 128);
    return (int)std::max<size_t>(1, std::min<size_t>(std::min<size_t>(32, r), want));
}

template <class R>
cudaError_t launch_qr_sweeps(const SchurDesc<R> *d_desc, int batch, int nmax, int *h_state,
                             const int *d_state_all, cudaStream_t s, float *ms_chase,
                             const SchurDesc<R> *d_desc_alt, cudaStream_t side, const cudaEvent_t *qev,
                             int *d_sync, int helpers)
{
    constexpr int RRMAX = QrDims<R>::RR;
    const int rpc = qr_rows_per_cta<R>(nmax, batch);
    const size_t ubytes = 2 * (size_t)RRMAX * RRMAX * sizeof(cplx<R>);
    const size_t mbytes = (size_t)std::max(nmax, 1) * sizeof(int);  // write-back masks
    const size_t rows_bytes = (size_t)rpc * nmax * sizeof(cplx<R>) + ubytes + mbytes;
    const size_t cols_bytes = (size_t)rpc * (nmax + 1) * sizeof(cplx<R>) + ubytes + mbytes;
    cudaError_t err;
    if ((err = allow_max_smem((const void *)qr_chase_kernel<R, false>))) return err;
    if ((err = allow_max_smem((const void *)qr_chase_kernel<R, true>))) return err;
    // cooperative chase (one chase CTA + H helper CTAs) for one large matrix
    const bool coop = d_sync != nullptr && batch == 1 && nmax >= kQrCoopMinN && helpers != 0;
    int H = helpers > 0 ? std::min(helpers, 24) : nmax >= 1024 ? 16 : 8;  // d_sync holds 4 + H counters
    if ((err = allow_max_smem((const void *)qr_build_u_kernel<R>))) return err;
    if ((err = allow_max_smem((const void *)qr_apply_rows_kernel<R>))) return err;
    if ((err = allow_max_smem((const void *)qr_apply_cols_kernel<R>))) return err;
    qr_state_init_kernel<R><<<1, 256, 0, s>>>(d_desc, batch); count_launch();
    const int ctas = (int)cdiv_i(nmax, rpc);
    bool all = false;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (ms_chase) {
        *ms_chase = 0.0f;
        if ((err = cudaEventCreate(&ev[0])) || (err = cudaEventCreate(&ev[1]))) return err;
    }
    const bool overlap = d_desc_alt && side && qev;
    bool used[2] = {false, false};
    for (int round = 0; round < 256 && !all; ++round) {
        const int par = overlap ? (round & 1) : 0;
        const SchurDesc<R> *dd = par ? d_desc_alt : d_desc;
        // this buffer set's deferred passes from two rounds ago must be done
        if (used[par] && (err = cudaStreamWaitEvent(s, qev[2 + par], 0))) break;
        if (ms_chase && (err = cudaEventRecord(ev[0], s))) break;
        if (coop) {
            if ((err = cudaMemsetAsync(d_sync, 0, (4 + H) * sizeof(int), s))) break;
            const SchurDesc<R> *arg0 = dd;
            void *args[2] = {(void *)&arg0, (void *)&H};
            if ((err = cudaLaunchCooperativeKernel((const void *)qr_chase_kernel<R, true>, dim3(1 + H), dim3(kQrThreads),
                                                   args, QrDims<R>::chase_smem, s))) break;
        } else {
            qr_chase_kernel<R, false><<<batch, kQrThreads, QrDims<R>::chase_smem, s>>>(dd, 0);
        }
        count_launch();
        if (ms_chase && (err = cudaEventRecord(ev[1], s))) break;
        if ((err = cudaMemcpyAsync(h_state, d_state_all, sizeof(int) * kQrStateInts * batch, cudaMemcpyDeviceToHost, s))) break;
        if ((err = cudaStreamSynchronize(s))) break;
        if (ms_chase) {
            float ms = 0.0f;
            if ((err = cudaEventElapsedTime(&ms, ev[0], ev[1]))) break;
            *ms_chase += ms;
        }
        int maxwin = 0;
        all = true;
        for (int b = 0; b < batch; ++b) {
            all = all && h_state[kQrStateInts * b + 2];
            maxwin = std::max(maxwin, h_state[kQrStateInts * b + 7]);
        }
        if (maxwin > 0) {
            cudaStream_t ds = s;
            if (overlap) {
                if ((err = cudaEventRecord(qev[par], s)) || (err = cudaStreamWaitEvent(side, qev[par], 0))) break;
                ds = side;
            }
            qr_tiny_kernel<R><<<dim3(maxwin, batch), 32, 0, ds>>>(dd); count_launch();
            qr_build_u_kernel<R><<<dim3(maxwin, batch), 128, QrDims<R>::build_smem, ds>>>(dd); count_launch();
            qr_apply_rows_kernel<R><<<dim3(2 * ctas, batch), 256, rows_bytes, ds>>>(dd, rpc, ctas); count_launch();
            qr_apply_cols_kernel<R><<<dim3(ctas, batch), 256, cols_bytes, ds>>>(dd, rpc); count_launch();
            if (overlap) {
                if ((err = cudaEventRecord(qev[2 + par], side))) break;
                used[par] = true;
            }
        }
    }
    // every deferred pass finishes before T is read again
    for (int q = 0; q < 2; ++q)
        if (used[q]) {
            cudaError_t e2 = cudaStreamWaitEvent(s, qev[2 + q], 0);
            if (!err) err = e2;
        }
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    if (err) return err;
    if (!all) { qr_mark_unfinished_kernel<R><<<1, 256, 0, s>>>(d_desc, batch); count_launch(); }
    qr_finish_kernel<R><<<dim3(64, batch), 256, 0, s>>>(d_desc); count_launch();
    return cudaGetLastError();
}

// Device-driven rounds for a batch (every launch one CTA per matrix, no
// cooperative chase): after each round a single thread reads every
// matrix's done flag and sets the WHILE condition of the enclosing graph;
// after max_rounds rounds the unfinished matrices get status 3.
template <class R>
__global__ void qr_round_decide_kernel(const SchurDesc<R> *__restrict__ descs, int batch, int *round,
                                       cudaGraphConditionalHandle cond, int max_rounds)
{
    __shared__ int s_open;
    if (threadIdx.x == 0) s_open = 0;
    __syncthreads();
    for (int b = threadIdx.x; b < batch; b += blockDim.x)
        if (!descs[b].state[2]) atomicOr(&s_open, 1);
    __syncthreads();
    const int r = *round + 1;
    const bool more = s_open && r < max_rounds;
    if (s_open && !more)
        for (int b = threadIdx.x; b < batch; b += blockDim.x)
            if (!descs[b].state[2]) atomicExch(descs[b].status, 3);
    __syncthreads();
    if (threadIdx.x == 0) {
        *round = r;
        cudaGraphSetConditional(cond, more ? 1u : 0u);
    }
}

namespace {
template <class R>
struct RoundCtx {
    const SchurDesc<R> *desc;
    int batch, nmax, *round;
};

template <class R>
cudaError_t enqueue_round(void *p, cudaStream_t s, cudaGraphConditionalHandle cond)
{
    const RoundCtx<R> *c = (const RoundCtx<R> *)p;
    constexpr int RRMAX = QrDims<R>::RR;
    const int rpc = qr_rows_per_cta<R>(c->nmax, c->batch);
    const size_t ubytes = 2 * (size_t)RRMAX * RRMAX * sizeof(cplx<R>);
    const size_t mbytes = (size_t)std::max(c->nmax, 1) * sizeof(int);
    const size_t rows_bytes = (size_t)rpc * c->nmax * sizeof(cplx<R>) + ubytes + mbytes;
    const size_t cols_bytes = (size_t)rpc * (c->nmax + 1) * sizeof(cplx<R>) + ubytes + mbytes;
    const int ctas = (int)cdiv_i(c->nmax, rpc);
    // windows of a round: at most the window capacity of the largest matrix
    const int ubx = (int)std::min<int64_t>(qr_win_capacity(c->nmax), 64);
    qr_chase_kernel<R, false><<<c->batch, kQrThreads, QrDims<R>::chase_smem, s>>>(c->desc, 0); count_launch();
    // (a few small blocks per matrix and round: 8 CTAs per matrix stride over its windows)
    qr_tiny_kernel<R><<<dim3(std::min(ubx, 8), c->batch), 32, 0, s>>>(c->desc); count_launch();
    qr_build_u_kernel<R><<<dim3(ubx, c->batch), 128, QrDims<R>::build_smem, s>>>(c->desc); count_launch();
    qr_apply_rows_kernel<R><<<dim3(2 * ctas, c->batch), 256, rows_bytes, s>>>(c->desc, rpc, ctas); count_launch();
    qr_apply_cols_kernel<R><<<dim3(ctas, c->batch), 256, cols_bytes, s>>>(c->desc, rpc); count_launch();
    qr_round_decide_kernel<R><<<1, 256, 0, s>>>(c->desc, c->batch, c->round, cond, 256); count_launch();
    return cudaGetLastError();
}
}  // namespace

template <class R>
cudaError_t enqueue_qr_sweeps_device(const SchurDesc<R> *d_desc, int batch, int nmax, int *d_round, cudaStream_t s,
                                     cudaStream_t body_stream)
{
    if (batch <= 0) return cudaSuccess;
    cudaError_t err;
    if ((err = allow_max_smem((const void *)qr_chase_kernel<R, false>))) return err;
    if ((err = allow_max_smem((const void *)qr_build_u_kernel<R>))) return err;
    if ((err = allow_max_smem((const void *)qr_apply_rows_kernel<R>))) return err;
    if ((err = allow_max_smem((const void *)qr_apply_cols_kernel<R>))) return err;
    qr_state_init_kernel<R><<<1, 256, 0, s>>>(d_desc, batch); count_launch();
    if ((err = cudaMemsetAsync(d_round, 0, sizeof(int), s))) return err;
    RoundCtx<R> ctx{d_desc, batch, nmax, d_round};
    if ((err = capture_while(s, body_stream, 1u, enqueue_round<R>, &ctx))) return err;
    qr_finish_kernel<R><<<dim3(64, batch), 256, 0, s>>>(d_desc); count_launch();
    return cudaGetLastError();
}

template cudaError_t enqueue_qr_sweeps_device<float>(const SchurDesc<float> *, int, int, int *, cudaStream_t, cudaStream_t);

template cudaError_t launch_qr_sweeps<float>(const SchurDesc<float> *, int, int, int *, const int *, cudaStream_t, float *,
                                             const SchurDesc<float> *, cudaStream_t, const cudaEvent_t *, int *, int);
template cudaError_t launch_qr_sweeps<double>(const SchurDesc<double> *, int, int, int *, const int *, cudaStream_t, float *,
                                              const SchurDesc<double> *, cudaStream_t, const cudaEvent_t *, int *, int);

}  // namespace sqm
