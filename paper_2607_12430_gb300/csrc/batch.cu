// batch.cu -- the batched path: many independent small matrices through
// Algorithm 2 (general members) and Algorithm 3 (symmetric members) in ONE
// CUDA graph launch per call.  Every stage is one launch (or one short
// sequence) over all matrices, each kernel indexing its matrix by blockIdx.
// The two loops of the method run on the device as conditional WHILE nodes
// of the graph: the rounds of the QR iteration (a one-thread kernel tests
// every matrix's done flag after each round) and the refinement steps (the
// convergence test runs per matrix on the device, and a one-thread kernel
// ends the loop when no matrix takes another correction).  The host reads
// the statuses once, after the graph.
//
// Per matrix i of the batch: A_i (FP64, lda_i) -> X_i (FP64, ldx_i), with the
// same scaling (A_s = 4^-e A, e = ceil(p / 2) for ||A||_F / sqrt(n) = m 2^p) as
// the single-matrix paths.  General members: FP32 complex Schur form and
// triangular square root.  Symmetric members (bitwise symmetric under
// SQRTM_KIND_AUTO, or every member under SQRTM_KIND_SPD): the FP32 spectral
// decomposition A_s = V diag(lam) V^T by cyclic Jacobi (Algorithm 3, step 1),
// handed to the shared stages as Q = V and T = diag(lam), so that the
// triangular square root gives s_i = sqrt(lam_i) (step 2) and the Sylvester
// solve with the diagonal S is y_ij = r_ij / (s_i + s_j) (step 9).  Then
// X_0 = Re(Q S Q^H) and the refinement with FP64 residual and update.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "handle.h"
#include "tc_common.cuh"

namespace sqm {

// per-matrix state of the batched path (device)
struct BState {
    const double *partials;  // residual partial sums of the current step
    double norm_a;           // ||A||_F
    double norm_as;          // ||A_s||_F = 4^-e ||A||_F
    double prev;             // previous ||R||_F (growth test)
    int np;                  // number of partials
    int e;                   // scaling exponent
    int active;              // 1 while the matrix still takes corrections
    int applied;             // corrections applied
    int grew;                // consecutive residual growths
    int status;              // final status (0 .. 7)
    int st_schur;            // Schur stage status
    int st_solve;            // triangular square root / Sylvester status
    int hist_len;
    int k;                   // convergence tests done (the step index)
    double hist[SQRTM_MAX_HISTORY];
};

struct BInput {
    const double *A;
    int64_t lda;
    int n;
};

struct BParams {
    double tol;
    int fixed;     // 1: apply exactly `steps` corrections, no test
    int max_corr;  // adaptive: at most this many corrections
    int nactive;   // matrices still taking corrections after the last test
    int iters;     // refinement steps at most (graph loop bound)
    int iter;      // refinement steps done (device loop counter)
    int round;     // QR rounds done (device loop counter)
};

// the refinement loop's condition: before the loop (any step at all?) and
// after each step (did some matrix go on, and is a step left?)
__global__ void brefine_init_kernel(BParams *prm, cudaGraphConditionalHandle cond)
{
    prm->iter = 0;
    prm->nactive = 0;
    cudaGraphSetConditional(cond, prm->iters > 0 ? 1u : 0u);
}

__global__ void brefine_next_kernel(BParams *prm, cudaGraphConditionalHandle cond)
{
    const bool go = prm->nactive > 0 && ++prm->iter < prm->iters;
    prm->nactive = 0;
    cudaGraphSetConditional(cond, go ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// symmetric members: FP32 spectral decomposition by cyclic Jacobi
// ---------------------------------------------------------------------------
// A symmetric A_s = V diag(lam) V^T (Algorithm 3, step 1) by two-sided
// Jacobi rotations in the parallel (round-robin) order: the n indices (plus
// one padding slot when n is odd) form n/2 disjoint pairs per step, each
// pair (p, q) zeroes a_pq by J = [c s; -s c] with t = tan from
// theta = (a_qq - a_pp) / (2 a_pq), t = sign(theta) / (|theta| +
// sqrt(1 + theta^2)), c = 1 / sqrt(1 + t^2), s = t c; the N - 1 steps of a
// sweep meet every pair once.  A pair is skipped (identity) when |a_pq| <=
// 2^-23 sqrt(|a_pp a_qq|) or |a_pq| <= 2^-24 ||A||_F (FP32 rounding level);
// the iteration stops after a sweep with no rotation (at most 30 sweeps,
// then status 3).  One step updates A <- J^T A J as 2 x 2 blocks
// J_k^T A({p_k, q_k}, {p_l, q_l}) J_l over the pairs k >= l -- every block
// is a disjoint set of entries -- on the packed lower triangle of A in
// shared memory (exactly symmetric), and V <- V J column pair by column pair.
struct JacJob {
    cplx<float> *T;   // in: A_s in the real parts; out: diag(lam)
    cplx<float> *Q;   // out: V (imaginary parts zero)
    float *Vw;        // scratch n x n: V when it is not kept in shared memory
    int *status;      // receives 3 (no convergence) or 7 (n out of range)
    int n;
};

static constexpr int kJacThreads = 1024;
static constexpr int kJacMaxN = 256;       // packed A: n(n+1)/2 floats in shared memory
static constexpr int kJacVsmemMaxN = 190;  // V in shared memory as well up to this size
static constexpr int kJacSweeps = 30;

__device__ __forceinline__ int jac_idx(int i, int j, int n)  // (i, j) of the lower triangle, i >= j
{
    return i + j * (2 * n - j - 1) / 2;
}

inline size_t jac_smem_bytes(int n, bool vsmem)
{
    const size_t np = ((size_t)n * (n + 1) / 2 + 3) & ~(size_t)3;
    return (np + (vsmem ? (size_t)n * n : 0)) * sizeof(float);
}

template <bool VSMEM>
__global__ void __launch_bounds__(kJacThreads) bjacobi_kernel(const JacJob *__restrict__ jobs)
{
    extern __shared__ __align__(16) float jsm[];
    __shared__ float s_c[kJacMaxN / 2], s_s[kJacMaxN / 2];
    __shared__ int s_p[kJacMaxN / 2], s_q[kJacMaxN / 2];
    __shared__ int s_col[kJacMaxN + 1];  // packed offset of column j: P(i, j) = P[i + s_col[j]], i >= j
    __shared__ float red[kJacThreads / 32];
    __shared__ float s_floor;
    __shared__ int s_rot;
    const JacJob J = jobs[blockIdx.x];
    const int n = J.n, tid = threadIdx.x;
    constexpr int nt = kJacThreads;
    if (n <= 0) return;
    if (n > kJacMaxN || (VSMEM && n > kJacVsmemMaxN)) {
        if (tid == 0) atomicExch(J.status, 7);
        return;
    }
    float *P = jsm;
    const int np = n * (n + 1) / 2;
    float *V = VSMEM ? jsm + ((np + 3) & ~3) : J.Vw;
    for (int j = tid; j <= n; j += nt) s_col[j] = j * (2 * n - j - 1) / 2;
    __syncthreads();
    float ss = 0.0f;
    for (int e = tid; e < n * n; e += nt) {
        const int i = e % n, j = e / n;
        const float a = J.T[e].x;
        if (i >= j) P[i + s_col[j]] = a;
        ss = fmaf(a, a, ss);
        V[e] = (i == j) ? 1.0f : 0.0f;
    }
    ss = warp_sum(ss);
    if ((tid & 31) == 0) red[tid >> 5] = ss;
    __syncthreads();
    if (tid == 0) {
        float t = 0.0f;
        for (int w = 0; w < nt / 32; ++w) t += red[w];
        s_floor = ldexpf(sqrtf(t), -24);
    }
    __syncthreads();
    const int N = n + (n & 1), H = N / 2;
    const int ntri = H * (H + 1) / 2;  // blocks (k, l), l <= k
    const float eps = 1.1920929e-7f;   // 2^-23
    // this thread's first block: (k0, l0) with k0 (k0 + 1) / 2 + l0 = tid
    int k0 = 0, l0 = tid;
    while (l0 > k0) { l0 -= k0 + 1; ++k0; }
    bool conv = false;
    for (int sw = 0; sw < kJacSweeps && !conv; ++sw) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int r = 0; r < N - 1; ++r) {
            if (tid < H) {
                const int a = tid == 0 ? r : (r + tid) % (N - 1);
                const int b = tid == 0 ? N - 1 : (r - tid + N - 1) % (N - 1);
                const int p = min(a, b);
                int q = max(a, b);
                float c = 1.0f, sn = 0.0f;
                if (q < n) {
                    const float app = P[p + s_col[p]], aqq = P[q + s_col[q]], apq = P[q + s_col[p]];
                    const float aa = fabsf(apq);
                    if (apq != 0.0f && aa > eps * sqrtf(fabsf(app * aqq)) && aa > s_floor) {
                        // t = tan of the angle that zeroes a_pq: with d = a_qq - a_pp and
                        // e = 2 a_pq, t = sign(d) e / (|d| + sqrt(d^2 + e^2)) (the root of
                        // t^2 + 2 t d / e - 1 = 0 of modulus <= 1); c = 1 / sqrt(1 + t^2)
                        const float d = aqq - app, e2 = 2.0f * apq;
                        const float h2 = fmaf(d, d, e2 * e2);
                        const float t = copysignf(1.0f, d) * e2 / (fabsf(d) + sqrtf(h2));
                        // 1 / sqrt(v) refined by one Newton step with fused multiply-adds,
                        // so that c^2 + s^2 = 1 to rounding (every rotation is orthogonal)
                        const float v = fmaf(t, t, 1.0f), y0 = rsqrtf(v);
                        c = fmaf(0.5f * y0, fmaf(-(v * y0), y0, 1.0f), y0);
                        sn = t * c;
                        s_rot = 1;
                    }
                } else {
                    q = -1;  // partner is the padding slot: a group of one, no rotation
                }
                s_p[tid] = p;
                s_q[tid] = q;
                s_c[tid] = c;
                s_s[tid] = sn;
            }
            __syncthreads();
            // A <- J^T A J as 2 x 2 blocks over the pairs k >= l (triangular
            // enumeration, each thread advancing nt blocks at a time)
            for (int k = k0, l = l0, e = tid; e < ntri;) {
                const float sk = s_s[k], sl = s_s[l];
                if (sk != 0.0f || sl != 0.0f) {
                    const float ck = s_c[k], cl = s_c[l];
                    const int pk = s_p[k], qk = s_q[k], pl = s_p[l], ql = s_q[l];
                    // entry (i, j) of the block lives at the packed (max, min)
                    const int i00 = pk >= pl ? pk + s_col[pl] : pl + s_col[pk];
                    const int i01 = ql < 0 ? -1 : (pk >= ql ? pk + s_col[ql] : ql + s_col[pk]);
                    const int i10 = qk < 0 ? -1 : (qk >= pl ? qk + s_col[pl] : pl + s_col[qk]);
                    const int i11 = (qk < 0 || ql < 0) ? -1 : (qk >= ql ? qk + s_col[ql] : ql + s_col[qk]);
                    const float b00 = P[i00];
                    const float b01 = i01 >= 0 ? P[i01] : 0.0f;
                    const float b10 = i10 >= 0 ? P[i10] : 0.0f;
                    const float b11 = i11 >= 0 ? P[i11] : 0.0f;
                    const float r00 = ck * b00 - sk * b10, r01 = ck * b01 - sk * b11;
                    const float r10 = sk * b00 + ck * b10, r11 = sk * b01 + ck * b11;
                    const float c00 = cl * r00 - sl * r01, c01 = sl * r00 + cl * r01;
                    const float c10 = cl * r10 - sl * r11, c11 = sl * r10 + cl * r11;
                    P[i00] = c00;
                    if (k == l) {
                        if (i10 >= 0) {  // diagonal block: (q, p) and (q, q); (p, q) is the same entry as (q, p)
                            P[i10] = c10;
                            P[i11] = c11;
                        }
                    } else {
                        if (i01 >= 0) P[i01] = c01;
                        if (i10 >= 0) P[i10] = c10;
                        if (i11 >= 0) P[i11] = c11;
                    }
                }
                e += nt;
                l += nt;
                while (l > k) { l -= k + 1; ++k; }
            }
            for (int e = tid; e < H * n; e += nt) {
                const int k = e / n, i = e - k * n;
                const float sk = s_s[k];
                if (sk == 0.0f) continue;
                const float ck = s_c[k];
                const int p = s_p[k], q = s_q[k];
                const float vp = V[i + p * n], vq = V[i + q * n];
                V[i + p * n] = ck * vp - sk * vq;
                V[i + q * n] = sk * vp + ck * vq;
            }
            __syncthreads();
        }
        conv = s_rot == 0;
        __syncthreads();
    }
    if (!conv && tid == 0) atomicExch(J.status, 3);
    for (int e = tid; e < n * n; e += nt) {
        const int i = e % n, j = e / n;
        J.Q[e] = cplx<float>{V[e], 0.0f};
        J.T[e] = cplx<float>{i == j ? P[i + s_col[i]] : 0.0f, 0.0f};
    }
}

// phase boundary of a batched call: the device clock at this point of the
// graph (one thread)
__global__ void bstamp_kernel(unsigned long long *stamps, int i)
{
    stamps[i] = globaltimer_ns();
}

// flag[b] = 1 when matrix b is not bitwise symmetric
__global__ void bsym_kernel(const BInput *__restrict__ in, int *__restrict__ nonsym)
{
    const BInput a = in[blockIdx.y];
    const int64_t nn = (int64_t)a.n * a.n;
    bool bad = false;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nn; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t % a.n, j = t / a.n;
        if (i > j && __double_as_longlong(a.A[i + j * a.lda]) != __double_as_longlong(a.A[j + i * a.lda]))
            bad = true;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) nonsym[blockIdx.y] = 1;
}

static constexpr int kBNormThreads = 256;

// ||A||_F (fixed summation order: thread-strided column-major sums, then the
// warps in order), the exponent e = ceil(p / 2) of ||A||_F / sqrt(n) = m 2^p,
// and the initial state; non-finite input gives status 5, a zero matrix 2
__global__ void __launch_bounds__(kBNormThreads)
bnorm_kernel(const BInput *__restrict__ in, BState *__restrict__ st)
{
    __shared__ double red[kBNormThreads / 32];
    const BInput a = in[blockIdx.x];
    const int64_t nn = (int64_t)a.n * a.n;
    double acc = 0.0;
    for (int64_t t = threadIdx.x; t < nn; t += blockDim.x) {
        const double v = a.A[(t % a.n) + (t / a.n) * a.lda];
        acc = fma(v, v, acc);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int w = 0; w < kBNormThreads / 32; ++w) s += red[w];
    const double nrm = sqrt(s);
    BState &q = st[blockIdx.x];
    int e = 0, status = 0;
    if (!isfinite(nrm)) status = 5;
    else if (nrm == 0.0) status = 2;  // the zero matrix has the eigenvalue 0
    else {
        int p;
        frexp(sqrt(s / (double)a.n), &p);
        e = (p >= 0) ? (p + 1) / 2 : -((-p) / 2);
    }
    q.norm_a = nrm;
    q.norm_as = ldexp(nrm, -2 * e);
    q.prev = INFINITY;
    q.e = e;
    q.active = status == 0;
    q.applied = q.grew = q.hist_len = q.k = 0;
    q.status = status;
    q.st_schur = q.st_solve = 0;
}

// T_i = fl(A_i 4^-e) as complex, or 0 for a matrix already failed (its
// Schur stage then deflates at once)
template <class R>
__global__ void bcast_kernel(const BInput *__restrict__ in, const BState *__restrict__ st,
                             const SchurDesc<R> *__restrict__ desc)
{
    const BInput a = in[blockIdx.y];
    const BState &q = st[blockIdx.y];
    cplx<R> *T = desc[blockIdx.y].T;
    const double sc = ldexp(1.0, -2 * q.e);
    const bool ok = q.active != 0;
    const int64_t nn = (int64_t)a.n * a.n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nn; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t % a.n, j = t / a.n;
        T[t] = ok ? cplx<R>{(R)(a.A[i + j * a.lda] * sc), R(0)} : cplx<R>{0, 0};
    }
}

// fold the stage statuses into the final one and stop the matrix
__global__ void bfold_kernel(BState *__restrict__ st, int batch)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    BState &q = st[b];
    const int s = q.st_schur ? q.st_schur : q.st_solve;
    if (s) {
        if (!q.status || q.active) q.status = s;
        q.active = 0;
    }
}

// the convergence test of step k (Algorithm 2, steps 5-7) for every active
// matrix, on the device: ||R||_F from the residual's partial sums (fixed
// order), then stop on the tolerance, the step limit (status 1), a non-finite
// residual or two growths in a row (status 4)
__global__ void bdecide_kernel(BState *__restrict__ st, int batch, BParams *__restrict__ prm)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    BState &q = st[b];
    if (!q.active) return;
    if (q.st_solve) {
        q.status = q.st_solve;
        q.active = 0;
        return;
    }
    const int k = q.k++;
    double s = 0.0;
    for (int i = 0; i < q.np; ++i) s += q.partials[i];
    const double rn = sqrt(s), rel = rn / q.norm_as;
    if (q.hist_len < SQRTM_MAX_HISTORY) q.hist[q.hist_len++] = rel;
    if (prm->fixed) {
        ++q.applied;
        atomicAdd(&prm->nactive, 1);
        return;
    }
    int stop = -1;
    if (!isfinite(rel)) stop = 4;
    else if (rel <= prm->tol) stop = 0;
    else if (k >= prm->max_corr) stop = 1;
    else {
        q.grew = rn > q.prev ? q.grew + 1 : 0;
        if (q.grew >= 2) stop = 4;
    }
    if (stop >= 0) {
        q.status = stop;
        q.active = 0;
        return;
    }
    q.prev = rn;
    ++q.applied;
    atomicAdd(&prm->nactive, 1);
}

namespace {

// device-side layout of one batched call; the header part (descriptor and
// job arrays) comes first so that its addresses depend on the batch size
// only, which keeps the cached graphs valid across calls
template <class R>
struct BLayout {
    SchurDesc<R> *desc;  // general members first (entries 0 .. Bg-1)
    HessJob<R> *hj;
    JacJob *jj;          // symmetric members (entries Bg .. B-1)
    TriJob<R> *tri;
    GemmJob<R> *gj;  // 6 sets of `batch` products
    ResJob *rj;
    BState *st;
    BInput *in;
    BParams *prm;
    int *qstate;
    unsigned long long *stamps;  // kBatchPhases + 1 phase boundaries (device clock, ns)
    size_t hdr_bytes;
};

template <class R>
BLayout<R> carve_header(Carve &c, int batch)
{
    BLayout<R> L;
    L.desc = c.take<SchurDesc<R>>(batch);
    L.hj = c.take<HessJob<R>>(batch);
    L.jj = c.take<JacJob>(batch);
    L.tri = c.take<TriJob<R>>(batch);
    L.gj = c.take<GemmJob<R>>(6 * (size_t)batch);
    L.rj = c.take<ResJob>(batch);
    L.st = c.take<BState>(batch);
    L.in = c.take<BInput>(batch);
    L.prm = c.take<BParams>(1);
    L.qstate = c.take<int>(kQrStateInts * (size_t)batch);
    L.stamps = c.take<unsigned long long>(kBatchPhases + 1);
    L.hdr_bytes = Carve::round(c.off);
    return L;
}

template <class R>
size_t matrix_bytes(int64_t n)
{
    const size_t nn = (size_t)n * n, cb = sizeof(cplx<R>);
    const int64_t nt = (n + 63) / 64;
    return 5 * Carve::round(nn * cb) + Carve::round(nn * sizeof(float)) + Carve::round(nt * nt * sizeof(double)) +
           Carve::round(qr_log_capacity(n) * sizeof(RotLog<R>)) + Carve::round(qr_win_capacity(n) * sizeof(WinRec)) +
           Carve::round(qr_u_capacity(n) * cb) + Carve::round((n + 8) * cb) + Carve::round(8 * sizeof(R)) +
           Carve::round(4 * sizeof(int)) + Carve::round(32 * sizeof(int)) + Carve::round(qr_win_capacity(n) * sizeof(int)) +
           Carve::round(8 * sizeof(int)) + 256;
}

// what the captured launches depend on beyond the layout's addresses: the
// sizes (size classes, grids) and kinds in batch order, the block size
struct Pipe {
    BLayout<float> L;
    const int *nord;  // sizes in batch order (host)
    int B, Bg, nmax, blks;
    cudaStream_t body_stream;
};

cudaError_t enqueue_refine_body(void *p, cudaStream_t s, cudaGraphConditionalHandle cond)
{
    using R = float;
    const Pipe *c = (const Pipe *)p;
    const BLayout<R> &L = c->L;
    const int B = c->B, nm = c->nmax;
    cudaError_t err;
    // R = (A - X X) 4^-e and ||R||_F, the per-matrix test (counting the
    // matrices that go on), R~ = Q^H Rhat Q, S Y + Y S = R~, X += 2^e Re(Q Y Q^H)
    if ((err = launch_residual_batched(L.rj, B, nm, s))) return err;
    bdecide_kernel<<<cdiv_i(B, 128), 128, 0, s>>>(L.st, B, L.prm); count_launch();
    if ((err = launch_cgemm_batched<R>(OP_N, OP_N, true, EPI_STORE, L.gj + 2 * B, B, nm, s))) return err;
    if ((err = launch_cgemm_batched<R>(OP_H, OP_N, false, EPI_STORE, L.gj + 3 * B, B, nm, s))) return err;
    if ((err = launch_rtrsyl_batched<R>(L.tri, B, nm, c->blks, s))) return err;
    if ((err = launch_cgemm_batched<R>(OP_N, OP_N, false, EPI_STORE, L.gj + 4 * B, B, nm, s))) return err;
    if ((err = launch_cgemm_batched<R>(OP_N, OP_H, false, EPI_REAL_ADD_F64, L.gj + 5 * B, B, nm, s))) return err;
    brefine_next_kernel<<<1, 1, 0, s>>>(L.prm, cond); count_launch();
    return cudaGetLastError();
}

cudaError_t enqueue_refine_init(void *p, cudaStream_t s, cudaGraphConditionalHandle cond)
{
    const Pipe *c = (const Pipe *)p;
    brefine_init_kernel<<<1, 1, 0, s>>>(c->L.prm, cond); count_launch();
    return cudaGetLastError();
}

// the whole batched call, for capture into one graph
cudaError_t enqueue_pipeline(void *p, cudaStream_t s)
{
    using R = float;
    const Pipe *c = (const Pipe *)p;
    const BLayout<R> &L = c->L;
    const int B = c->B, Bg = c->Bg, nmax = c->nmax;
    cudaError_t err;
    bstamp_kernel<<<1, 1, 0, s>>>(L.stamps, 0); count_launch();
    bnorm_kernel<<<B, kBNormThreads, 0, s>>>(L.in, L.st); count_launch();
    bcast_kernel<R><<<dim3(std::max(1, std::min(64, nmax * nmax / 1024)), B), 256, 0, s>>>(L.in, L.st, L.desc);
    count_launch();
    // general members: Hessenberg reduction (one cluster per matrix, one
    // launch per size class; the per-column kernels beyond the cluster
    // kernel's sizes), then the QR rounds on the device
    for (int i0 = 0; i0 < Bg;) {
        const int nc = c->nord[i0];
        const int cap = nc <= 64 ? 0 : nc <= 128 ? 64 : nc <= 256 ? 128 : nc <= 512 ? 256 : 512;
        int i1 = i0;
        while (i1 < Bg && c->nord[i1] > cap) ++i1;
        err = launch_hessenberg_cluster_batched<R>(L.hj + i0, i1 - i0, nc, s);
        if (err == cudaErrorNotSupported) {  // refused before any launch
            cudaGetLastError();
            err = launch_hessenberg<R>(L.desc + i0, i1 - i0, nc, std::max(1, nc / 32), s);
        }
        if (err) return err;
        i0 = i1;
    }
    bstamp_kernel<<<1, 1, 0, s>>>(L.stamps, 1); count_launch();
    if (Bg > 0 && (err = enqueue_qr_sweeps_device<R>(L.desc, Bg, c->nord[0], &L.prm->round, s, c->body_stream)))
        return err;
    bstamp_kernel<<<1, 1, 0, s>>>(L.stamps, 2); count_launch();
    // symmetric members: Jacobi, V in global memory above kJacVsmemMaxN
    for (int i0 = Bg; i0 < B;) {
        const bool vs = c->nord[i0] <= kJacVsmemMaxN;
        int i1 = i0;
        while (i1 < B && (c->nord[i1] <= kJacVsmemMaxN) == vs) ++i1;
        const size_t smem = jac_smem_bytes(c->nord[i0], vs);
        if (vs) bjacobi_kernel<true><<<i1 - i0, kJacThreads, smem, s>>>(L.jj + i0);
        else bjacobi_kernel<false><<<i1 - i0, kJacThreads, smem, s>>>(L.jj + i0);
        count_launch();
        if ((err = cudaGetLastError())) return err;
        i0 = i1;
    }
    bstamp_kernel<<<1, 1, 0, s>>>(L.stamps, 3); count_launch();
    if ((err = launch_trisqrt_batched<R>(L.tri, B, nmax, c->blks, s))) return err;
    bfold_kernel<<<cdiv_i(B, 128), 128, 0, s>>>(L.st, B); count_launch();
    // X_0 = 2^e Re(Q S Q^H), rounded to FP32
    if ((err = launch_cgemm_batched<R>(OP_N, OP_N, false, EPI_STORE, L.gj, B, nmax, s))) return err;
    if ((err = launch_cgemm_batched<R>(OP_N, OP_H, false, EPI_REAL_TO_F64, L.gj + B, B, nmax, s))) return err;
    bstamp_kernel<<<1, 1, 0, s>>>(L.stamps, 4); count_launch();
    // the refinement loop
    if ((err = capture_while(s, c->body_stream, 0u, enqueue_refine_body, (void *)c, enqueue_refine_init))) return err;
    bfold_kernel<<<cdiv_i(B, 128), 128, 0, s>>>(L.st, B); count_launch();
    bstamp_kernel<<<1, 1, 0, s>>>(L.stamps, 5); count_launch();
    return cudaGetLastError();
}

uint64_t fnv(uint64_t h, uint64_t v)
{
    for (int b = 0; b < 8; ++b) {
        h ^= (v >> (8 * b)) & 0xff;
        h *= 1099511628211ull;
    }
    return h;
}

}  // namespace
}  // namespace sqm

using namespace sqm;

// The batched path for the matrices idx[0 .. count) of a batched call;
// writes their statuses into st_out[idx[i]].
int batched_general(sqrtm_handle_t h, const int *idx, int count, const double *const *dA, const int64_t *n,
                    const int64_t *lda, double *const *dX, const int64_t *ldx, const sqrtm_opts &o, int *st_out)
{
    using R = float;
    if (count <= 0) return 0;
    cudaStream_t s = h->stream;
    const int B = count;
    const size_t pin_need = sizeof(BState) * (size_t)B + sizeof(int) * (size_t)B +
                            sizeof(unsigned long long) * (kBatchPhases + 1) + 4096;
    if (h->bpin_bytes < pin_need) {
        if (h->bpin) cudaFreeHost(h->bpin);
        h->bpin = nullptr;
        h->bpin_bytes = 0;
        if (cudaHostAlloc(&h->bpin, pin_need, cudaHostAllocDefault) != cudaSuccess) return 7;
        h->bpin_bytes = pin_need;
    }
    // which members take Algorithm 3: every one under SQRTM_KIND_SPD, none
    // under SQRTM_KIND_GENERAL, the bitwise symmetric ones under AUTO (one
    // check over all matrices, read back once)
    std::vector<int> sym(B, o.kind == SQRTM_KIND_SPD ? 1 : 0);
    if (o.kind == SQRTM_KIND_AUTO) {
        const size_t need = Carve::round(sizeof(BInput) * (size_t)B) + Carve::round(sizeof(int) * (size_t)B) + 512;
        if (ensure(h->ws, need, h)) return 7;
        Carve cw(h->ws.p);
        BInput *din = cw.take<BInput>(B);
        int *dflag = cw.take<int>(B);
        std::vector<BInput> hin(B);
        int64_t nmx = 1;
        for (int i = 0; i < B; ++i) {
            hin[i] = BInput{dA[idx[i]], lda[idx[i]], (int)n[idx[i]]};
            nmx = std::max(nmx, n[idx[i]]);
        }
        SQM_CU(cudaMemcpyAsync(din, hin.data(), sizeof(BInput) * (size_t)B, cudaMemcpyHostToDevice, s));
        SQM_CU(cudaMemsetAsync(dflag, 0, sizeof(int) * (size_t)B, s));
        bsym_kernel<<<dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(16, nmx * nmx / 4096)), B), 256, 0, s>>>(
            din, dflag);
        count_launch();
        int *hflag = (int *)((char *)h->bpin + sizeof(BState) * (size_t)B);
        SQM_CU(cudaMemcpyAsync(hflag, dflag, sizeof(int) * (size_t)B, cudaMemcpyDeviceToHost, s));
        SQM_CU(cudaStreamSynchronize(s));
        for (int i = 0; i < B; ++i) {
            const sqrtm_tune_entry *t = tune_for(h, n[idx[i]]);
            const bool spectral = t ? t->batched_spd == 1 : true;  // the tuning table's choice, else Algorithm 3
            sym[i] = (hflag[i] == 0 && n[idx[i]] <= kJacMaxN && spectral) ? 1 : 0;
        }
    } else if (o.kind == SQRTM_KIND_SPD) {
        for (int i = 0; i < B; ++i) sym[i] = n[idx[i]] <= kJacMaxN ? 1 : 0;
    }
    // batch order: general members by decreasing size, then symmetric ones
    // (the Schur stage's CTAs are scheduled in matrix order)
    std::vector<int> pos(B);
    std::iota(pos.begin(), pos.end(), 0);
    std::stable_sort(pos.begin(), pos.end(), [&](int a, int b) {
        if (sym[a] != sym[b]) return sym[a] < sym[b];
        return n[idx[a]] > n[idx[b]];
    });
    std::vector<int> ord(B), nord(B);
    int Bg = 0;
    for (int i = 0; i < B; ++i) {
        ord[i] = idx[pos[i]];
        nord[i] = (int)n[ord[i]];
        if (!sym[pos[i]]) ++Bg;
    }
    int nmax = 1;
    for (int i = 0; i < B; ++i) nmax = std::max(nmax, nord[i]);
    size_t bytes;
    {
        Carve c(nullptr);
        BLayout<R> L = carve_header<R>(c, B);
        bytes = L.hdr_bytes;
        for (int i = 0; i < B; ++i) bytes += matrix_bytes<R>(nord[i]);
        bytes += 4096;
    }
    if (ensure(h->bws, bytes, h)) return 7;
    // the header, built on the host with the device offsets, then one copy
    std::vector<char> hdr;
    Carve cd(h->bws.p);
    BLayout<R> L = carve_header<R>(cd, B);
    hdr.assign(L.hdr_bytes, 0);
    auto host = [&](const void *dev) { return hdr.data() + ((const char *)dev - (const char *)h->bws.p); };
    SchurDesc<R> *hdesc = (SchurDesc<R> *)host(L.desc);
    HessJob<R> *hhj = (HessJob<R> *)host(L.hj);
    JacJob *hjj = (JacJob *)host(L.jj);
    TriJob<R> *htri = (TriJob<R> *)host(L.tri);
    GemmJob<R> *hgj = (GemmJob<R> *)host(L.gj);
    ResJob *hrj = (ResJob *)host(L.rj);
    BInput *hin = (BInput *)host(L.in);
    BParams *hprm = (BParams *)host(L.prm);
    const bool fixed = o.steps >= 0;
    hprm->tol = o.tol;
    hprm->fixed = fixed;
    hprm->max_corr = fixed ? o.steps : o.maxit + 1;
    hprm->iters = fixed ? o.steps : o.maxit + 2;
    for (int i = 0; i < B; ++i) {
        const int m = ord[i];
        const int64_t nm = nord[i];
        const size_t nn = (size_t)nm * nm;
        cplx<R> *T = cd.take<cplx<R>>(nn), *Q = cd.take<cplx<R>>(nn), *S = cd.take<cplx<R>>(nn);
        cplx<R> *W = cd.take<cplx<R>>(nn), *Rt = cd.take<cplx<R>>(nn);
        float *Rhat = cd.take<float>(nn);
        const int64_t nt = (nm + 63) / 64;
        double *partials = cd.take<double>(nt * nt);
        SchurDesc<R> &d = hdesc[i];
        d.log = cd.take<RotLog<R>>(qr_log_capacity(nm));
        d.win = cd.take<WinRec>(qr_win_capacity(nm));
        d.u_cap = qr_u_capacity(nm);
        d.ubuf = cd.take<cplx<R>>(d.u_cap);
        d.v = cd.take<cplx<R>>(nm + 8);
        d.beta = cd.take<R>(8);
        d.rstate = cd.take<int>(4);
        d.sync = cd.take<int>(32);
        d.postlist = cd.take<int>(qr_win_capacity(nm));
        d.counters = cd.take<int>(8);
        d.state = L.qstate + kQrStateInts * (size_t)i;
        d.log_cap = (int)std::min<int64_t>(qr_log_capacity(nm), INT32_MAX);
        d.win_cap = (int)std::min<int64_t>(qr_win_capacity(nm), INT32_MAX);
        d.T = T; d.Q = Q; d.n = (int)nm; d.ld = (int)nm;
        BState *q = L.st + i;
        d.status = &q->st_schur;
        htri[i] = TriJob<R>{T, S, Rt, &q->st_solve, &q->active, (int)nm};
        hhj[i] = HessJob<R>{T, Q, (R *)W, (R *)Rt, (int)nm};  // W, Rt: free until the Schur form is done
        hjj[i] = JacJob{T, Q, (float *)W, &q->st_schur, (int)nm};  // W: free until X_0 is formed
        hin[i] = BInput{dA[m], lda[m], (int)nm};
        // products: 0 W = Q S, 1 X = 2^e Re(W Q^H), 2 W = Rhat Q, 3 Rt = Q^H W,
        // 4 W = Q Rt, 5 X += 2^e Re(W Q^H)
        hgj[0 * B + i] = GemmJob<R>{Q, S, W, nullptr, 0, &q->e, &q->active, (int)nm};
        hgj[1 * B + i] = GemmJob<R>{W, Q, nullptr, dX[m], ldx[m], &q->e, &q->active, (int)nm};
        hgj[2 * B + i] = GemmJob<R>{Rhat, Q, W, nullptr, 0, &q->e, &q->active, (int)nm};
        hgj[3 * B + i] = GemmJob<R>{Q, W, Rt, nullptr, 0, &q->e, &q->active, (int)nm};
        hgj[4 * B + i] = GemmJob<R>{Q, Rt, W, nullptr, 0, &q->e, &q->active, (int)nm};
        hgj[5 * B + i] = GemmJob<R>{W, Q, nullptr, dX[m], ldx[m], &q->e, &q->active, (int)nm};
        hrj[i] = ResJob{dA[m], lda[m], dX[m], ldx[m], Rhat, partials, &q->e, &q->active, (int)nm};
        BState *hq = (BState *)host(q);
        hq->partials = partials;
        hq->np = (int)(nt * nt);
    }
    SQM_CU(cudaMemcpyAsync(h->bws.p, hdr.data(), L.hdr_bytes, cudaMemcpyHostToDevice, s));
    if (!h->body_stream) SQM_CU(cudaStreamCreateWithFlags(&h->body_stream, cudaStreamNonBlocking));
    SQM_CU(allow_max_smem((const void *)bjacobi_kernel<true>));
    SQM_CU(allow_max_smem((const void *)bjacobi_kernel<false>));
    // one graph for the whole call, keyed by the sizes and kinds in batch
    // order and the block size (its launches take every pointer from the
    // header just copied)
    Pipe pipe{L, nord.data(), B, Bg, nmax, o.blks, h->body_stream};
    uint64_t sig = 1469598103934665603ull;
    sig = fnv(sig, (uint64_t)Bg);
    sig = fnv(sig, (uint64_t)o.blks);
    for (int i = 0; i < B; ++i) sig = fnv(sig, (uint64_t)nord[i]);
    if (run_graph(h, 400, L.desc, nmax, B, enqueue_pipeline, &pipe, sig)) return 7;
    BState *hst = (BState *)h->bpin;
    unsigned long long *hstamp = (unsigned long long *)((char *)h->bpin + sizeof(BState) * (size_t)B);
    SQM_CU(cudaMemcpyAsync(hst, L.st, sizeof(BState) * (size_t)B, cudaMemcpyDeviceToHost, s));
    SQM_CU(cudaMemcpyAsync(hstamp, L.stamps, sizeof(unsigned long long) * (kBatchPhases + 1), cudaMemcpyDeviceToHost, s));
    SQM_CU(cudaStreamSynchronize(s));
    for (int i = 0; i < B; ++i) st_out[ord[i]] = hst[i].status;
    for (int q = 0; q < kBatchPhases; ++q) h->bphase_ms[q] = 1e-6 * (double)(hstamp[q + 1] - hstamp[q]);
    h->bphase_count = B;
    h->bphase_general = Bg;
    return 0;
}
