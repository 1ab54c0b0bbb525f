// batch.cu -- the batched general path: many independent small matrices
// through Algorithm 2 in one set of launches.  Every stage is one launch (or
// one short sequence) over all matrices, each kernel indexing its matrix by
// blockIdx; the Hessenberg reduction and the whole refinement loop (residual,
// convergence test, transforms, Sylvester solve, update, for every step) are
// replayed from CUDA graphs, and the convergence test runs on the device, so
// the loop needs no host round trip.  Only the rounds of the QR iteration
// return to the host (to learn whether every matrix has converged).
//
// Per matrix i of the batch: A_i (FP64, lda_i) -> X_i (FP64, ldx_i), with the
// same scaling (A_s = 4^-e A, e = ceil(p / 2) for ||A||_F / sqrt(n) = m 2^p), FP32 complex
// Schur form, FP32 triangular square root, X_0 = Re(Q S Q^H) and the
// refinement with FP64 residual and update as sqrtm_mixed's general path.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "handle.h"

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
};

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
    SchurDesc<R> *desc;
    HessJob<R> *hj;
    TriJob<R> *tri;
    GemmJob<R> *gj;  // 6 sets of `batch` products
    ResJob *rj;
    BState *st;
    BInput *in;
    BParams *prm;
    int *qstate;
    size_t hdr_bytes;
};

template <class R>
BLayout<R> carve_header(Carve &c, int batch)
{
    BLayout<R> L;
    L.desc = c.take<SchurDesc<R>>(batch);
    L.hj = c.take<HessJob<R>>(batch);
    L.tri = c.take<TriJob<R>>(batch);
    L.gj = c.take<GemmJob<R>>(6 * (size_t)batch);
    L.rj = c.take<ResJob>(batch);
    L.st = c.take<BState>(batch);
    L.in = c.take<BInput>(batch);
    L.prm = c.take<BParams>(1);
    L.qstate = c.take<int>(kQrStateInts * (size_t)batch);
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

struct LoopCtx {
    const void *tri, *gj, *rj;
    BState *st;
    BParams *prm;
    int batch, nmax, blks;
};

// one step of the refinement for every matrix still active: R = (A - X X)
// 4^-e and ||R||_F, the test (which also counts the matrices that go on),
// then R~ = Q^H Rhat Q, S Y + Y S = R~, X += 2^e Re(Q Y Q^H)
template <class R>
cudaError_t enqueue_refine_step(void *p, cudaStream_t s)
{
    const LoopCtx *c = (const LoopCtx *)p;
    const TriJob<R> *tri = (const TriJob<R> *)c->tri;
    const GemmJob<R> *gj = (const GemmJob<R> *)c->gj;
    const ResJob *rj = (const ResJob *)c->rj;
    const int B = c->batch, nm = c->nmax;
    cudaError_t err;
    if ((err = cudaMemsetAsync(&c->prm->nactive, 0, sizeof(int), s))) return err;
    if ((err = launch_residual_batched(rj, B, nm, s))) return err;
    bdecide_kernel<<<cdiv_i(B, 128), 128, 0, s>>>(c->st, B, c->prm); count_launch();
    if ((err = launch_cgemm_batched<R>(OP_N, OP_N, true, EPI_STORE, gj + 2 * B, B, nm, s))) return err;
    if ((err = launch_cgemm_batched<R>(OP_H, OP_N, false, EPI_STORE, gj + 3 * B, B, nm, s))) return err;
    if ((err = launch_rtrsyl_batched<R>(tri, B, nm, c->blks, s))) return err;
    if ((err = launch_cgemm_batched<R>(OP_N, OP_N, false, EPI_STORE, gj + 4 * B, B, nm, s))) return err;
    if ((err = launch_cgemm_batched<R>(OP_N, OP_H, false, EPI_REAL_ADD_F64, gj + 5 * B, B, nm, s))) return err;
    return cudaGetLastError();
}

struct HessCtx {
    const void *desc;
    int batch, nmax;
};

template <class R>
cudaError_t enqueue_hess(void *p, cudaStream_t s)
{
    const HessCtx *c = (const HessCtx *)p;
    return launch_hessenberg<R>((const SchurDesc<R> *)c->desc, c->batch, c->nmax, std::max(1, c->nmax / 32), s);
}

}  // namespace
}  // namespace sqm

using namespace sqm;

// The batched general path for the matrices idx[0 .. count) of a batched
// call; writes their statuses into st_out[idx[i]].
int batched_general(sqrtm_handle_t h, const int *idx, int count, const double *const *dA, const int64_t *n,
                    const int64_t *lda, double *const *dX, const int64_t *ldx, const sqrtm_opts &o, int *st_out)
{
    using R = float;
    if (count <= 0) return 0;
    cudaStream_t s = h->stream;
    // largest first: the Schur stage's CTAs are scheduled in matrix order
    std::vector<int> ord(idx, idx + count);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return n[a] > n[b]; });
    const int B = count;
    const int nmax = (int)n[ord[0]];
    size_t bytes;
    {
        Carve c(nullptr);
        BLayout<R> L = carve_header<R>(c, B);
        bytes = L.hdr_bytes;
        for (int i = 0; i < B; ++i) bytes += matrix_bytes<R>(n[ord[i]]);
        bytes += 4096;
    }
    if (ensure(h->bws, bytes, h)) return 7;
    const size_t pin_need = sizeof(int) * kQrStateInts * (size_t)B + sizeof(BState) * (size_t)B + 4096;
    if (h->bpin_bytes < pin_need) {
        if (h->bpin) cudaFreeHost(h->bpin);
        h->bpin = nullptr;
        h->bpin_bytes = 0;
        if (cudaHostAlloc(&h->bpin, pin_need, cudaHostAllocDefault) != cudaSuccess) return 7;
        h->bpin_bytes = pin_need;
    }
    // the header, built on the host with the device offsets, then one copy
    std::vector<char> hdr;
    Carve cd(h->bws.p);
    BLayout<R> L = carve_header<R>(cd, B);
    hdr.assign(L.hdr_bytes, 0);
    auto host = [&](const void *dev) { return hdr.data() + ((const char *)dev - (const char *)h->bws.p); };
    SchurDesc<R> *hdesc = (SchurDesc<R> *)host(L.desc);
    HessJob<R> *hhj = (HessJob<R> *)host(L.hj);
    TriJob<R> *htri = (TriJob<R> *)host(L.tri);
    GemmJob<R> *hgj = (GemmJob<R> *)host(L.gj);
    ResJob *hrj = (ResJob *)host(L.rj);
    BInput *hin = (BInput *)host(L.in);
    BParams *hprm = (BParams *)host(L.prm);
    const bool fixed = o.steps >= 0;
    hprm->tol = o.tol;
    hprm->fixed = fixed;
    hprm->max_corr = fixed ? o.steps : o.maxit + 1;
    const int iters = fixed ? o.steps : o.maxit + 2;
    for (int i = 0; i < B; ++i) {
        const int m = ord[i];
        const int64_t nm = n[m];
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
    bnorm_kernel<<<B, kBNormThreads, 0, s>>>(L.in, L.st); count_launch();
    bcast_kernel<R><<<dim3(std::max(1, std::min(64, nmax * nmax / 1024)), B), 256, 0, s>>>(L.in, L.st, L.desc);
    count_launch();
    SQM_CU(cudaGetLastError());
    // Hessenberg reduction: one cluster per matrix, one launch per size
    // class (the sizes are sorted, so each class is a contiguous range);
    // the per-column kernels for sizes beyond the cluster kernel's
    for (int i0 = 0; i0 < B;) {
        const int nc = (int)n[ord[i0]];
        const int cap = nc <= 64 ? 0 : nc <= 128 ? 64 : nc <= 256 ? 128 : nc <= 512 ? 256 : 512;
        int i1 = i0;
        while (i1 < B && (int)n[ord[i1]] > cap) ++i1;
        cudaError_t err = launch_hessenberg_cluster_batched<R>(L.hj + i0, i1 - i0, nc, s);
        if (err == cudaErrorNotSupported) {
            cudaGetLastError();
            HessCtx hc{L.desc + i0, i1 - i0, nc};
            if (run_graph(h, 300, L.desc + i0, nc, i1 - i0, enqueue_hess<R>, &hc)) return 7;
        } else {
            SQM_CU(err);
        }
        i0 = i1;
    }
    SQM_CU(launch_qr_sweeps<R>(L.desc, B, nmax, (int *)h->bpin, L.qstate, s));
    SQM_CU(launch_trisqrt_batched<R>(L.tri, B, nmax, o.blks, s));
    bfold_kernel<<<cdiv_i(B, 128), 128, 0, s>>>(L.st, B); count_launch();
    // X_0 = 2^e Re(Q S Q^H), rounded to FP32
    SQM_CU(launch_cgemm_batched<R>(OP_N, OP_N, false, EPI_STORE, L.gj, B, nmax, s));
    SQM_CU(launch_cgemm_batched<R>(OP_N, OP_H, false, EPI_REAL_TO_F64, L.gj + B, B, nmax, s));
    // the refinement, one replayed graph per step; after each step the host
    // reads how many matrices go on and stops when none does
    int *h_nact = (int *)((char *)h->bpin + sizeof(int) * kQrStateInts * (size_t)B + sizeof(BState) * (size_t)B);
    for (int k = 0; k < iters; ++k) {
        LoopCtx lc{L.tri, L.gj, L.rj, L.st, L.prm, B, nmax, o.blks};
        if (run_graph(h, 100000 + o.blks, L.desc, nmax, B, enqueue_refine_step<R>, &lc)) return 7;
        SQM_CU(cudaMemcpyAsync(h_nact, &L.prm->nactive, sizeof(int), cudaMemcpyDeviceToHost, s));
        SQM_CU(cudaStreamSynchronize(s));
        if (*h_nact == 0) break;
    }
    bfold_kernel<<<cdiv_i(B, 128), 128, 0, s>>>(L.st, B); count_launch();
    BState *hst = (BState *)((char *)h->bpin + sizeof(int) * kQrStateInts * (size_t)B);
    SQM_CU(cudaMemcpyAsync(hst, L.st, sizeof(BState) * (size_t)B, cudaMemcpyDeviceToHost, s));
    SQM_CU(cudaStreamSynchronize(s));
    for (int i = 0; i < B; ++i) st_out[ord[i]] = hst[i].status;
    return 0;
}
