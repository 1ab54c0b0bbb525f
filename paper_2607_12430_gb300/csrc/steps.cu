// steps.cu -- step-level C entry points (sqrtm_mp_steps.h): each runs one
// stage of the method on caller-provided device buffers, with the same
// kernels the drivers chain.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "handle.h"
#include "spd_internal.h"
#include "tc_gemm.h"

using namespace sqm;

namespace {

struct StepScratch {
    double *dscal;   // [0] norm, [1] rnorm, [2..] partials
    int *iscal;      // [0] e, [1] status
};

int step_scratch(sqrtm_handle_t h, int64_t n, size_t extra, StepScratch *ss, void **extra_p)
{
    int64_t nb = (n + 63) / 64;
    size_t np = (size_t)std::max<int64_t>(nb * nb, 2048) + 8;
    size_t need = Carve::round(np * sizeof(double)) + 256 + Carve::round(extra) + 1024;
    if (ensure(h->ws, need, h)) return 7;
    Carve c(h->ws.p);
    ss->dscal = c.take<double>(np);
    ss->iscal = c.take<int>(8);
    *extra_p = extra ? c.take<char>(extra) : nullptr;
    if (cudaMemsetAsync(ss->iscal, 0, 8 * sizeof(int), h->stream) != cudaSuccess) return 7;
    return 0;
}

int fetch(sqrtm_handle_t h, void *dst, const void *src, size_t bytes)
{
    if (cudaMemcpyAsync(h->staging.p, src, bytes, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) return 7;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return 7;
    memcpy(dst, h->staging.p, bytes);
    return 0;
}

}  // namespace

extern "C" int sqrtm_step_scale(sqrtm_handle_t h, const double *dA, int64_t n, int64_t lda,
                                void *dAs, int fp64, int *e_host, double *norm_host)
{
    if (!h) return -1;
    if (n < 0) return -3;
    if (lda < std::max<int64_t>(1, n)) return -4;
    if (n == 0) { if (e_host) *e_host = 0; if (norm_host) *norm_host = 0; return 0; }
    StepScratch ss; void *ex;
    if (int rc = step_scratch(h, n, 0, &ss, &ex)) return rc;
    if (launch_norm_scale(dA, n, lda, ss.dscal + 2, (int)std::min<int64_t>(n, 1024), ss.dscal, ss.iscal, h->stream)) return 7;
    cudaError_t err = fp64 ? launch_cast_scaled<double>(dA, n, lda, ss.iscal, (cplx<double> *)dAs, n, h->stream)
                           : launch_cast_scaled<float>(dA, n, lda, ss.iscal, (cplx<float> *)dAs, n, h->stream);
    if (err) return 7;
    double nrm; int e;
    if (fetch(h, &nrm, ss.dscal, sizeof(double)) || fetch(h, &e, ss.iscal, sizeof(int))) return 7;
    if (e_host) *e_host = e;
    if (norm_host) *norm_host = nrm;
    return 0;
}

template <class R>
static int schur_step(sqrtm_handle_t h, cplx<R> *T, cplx<R> *Q, int64_t n)
{
    StepScratch ss; void *ex;
    size_t extra = Carve::round((n + 8) * sizeof(cplx<R>)) + Carve::round(8 * sizeof(R)) + Carve::round(sizeof(SchurDesc<R>)) +
                   Carve::round(qr_log_capacity(n) * sizeof(RotLog<R>)) + Carve::round(kQrStateInts * sizeof(int)) +
                   Carve::round(4 * sizeof(int)) +
                   Carve::round(qr_win_capacity(n) * sizeof(WinRec)) + Carve::round(qr_u_capacity(n) * sizeof(cplx<R>));
    if (int rc = step_scratch(h, n, extra, &ss, &ex)) return rc;
    Carve c(ex);
    cplx<R> *v = c.take<cplx<R>>(n + 8);
    R *beta = c.take<R>(8);
    SchurDesc<R> *dd = c.take<SchurDesc<R>>(1);
    RotLog<R> *rlog = c.take<RotLog<R>>(qr_log_capacity(n));
    int *qstate = c.take<int>(kQrStateInts);
    WinRec *wrec = c.take<WinRec>(qr_win_capacity(n));
    cplx<R> *ubuf = c.take<cplx<R>>(qr_u_capacity(n));
    int *rstate = c.take<int>(4);
    SchurDesc<R> hd;
    hd.rstate = rstate;
    hd.sync = nullptr;
    hd.postlist = nullptr;
    hd.T = T; hd.Q = Q; hd.v = v; hd.beta = beta; hd.status = ss.iscal + 1; hd.n = (int)n; hd.ld = (int)n;
    hd.counters = nullptr;
    hd.log = rlog; hd.state = qstate; hd.log_cap = (int)std::min<int64_t>(qr_log_capacity(n), INT32_MAX);
    hd.win = wrec; hd.win_cap = (int)std::min<int64_t>(qr_win_capacity(n), INT32_MAX);
    hd.ubuf = ubuf; hd.u_cap = qr_u_capacity(n);
    memcpy(h->staging.p, &hd, sizeof(hd));
    if (cudaMemcpyAsync(dd, h->staging.p, sizeof(hd), cudaMemcpyHostToDevice, h->stream)) return 7;
    if (cudaStreamSynchronize(h->stream)) return 7;
    if (launch_hessenberg<R>(dd, 1, (int)n, 64, h->stream)) return 7;
    if (launch_qr_sweeps<R>(dd, 1, (int)n, (int *)h->staging.p + 512, qstate, h->stream)) return 7;
    int st = 0;
    if (fetch(h, &st, ss.iscal + 1, sizeof(int))) return 7;
    return st;
}

// complex T = fl_R(A) (imaginary parts zero)
template <class R>
__global__ void cast_real_to_cplx_kernel(const double *__restrict__ A, int64_t lda, int n, cplx<R> *__restrict__ T)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)n * n;
         t += (int64_t)gridDim.x * blockDim.x)
        T[t] = cplx<R>{(R)A[(t % n) + (t / n) * lda], R(0)};
}

template <class R>
static int hess_step(sqrtm_handle_t h, const double *dA, int64_t n, int64_t lda, cplx<R> *H, cplx<R> *Q)
{
    const size_t nn = (size_t)n * n;
    StepScratch ss; void *ex;
    const size_t extra = 3 * Carve::round(nn * sizeof(R)) + Carve::round(hessenberg_real_scratch<R>((int)n) * sizeof(R));
    if (int rc = step_scratch(h, n, extra, &ss, &ex)) return rc;
    Carve c(ex);
    R *Hr = c.take<R>(nn), *Y = c.take<R>(nn), *Qr = c.take<R>(nn);
    R *scr = c.take<R>(hessenberg_real_scratch<R>((int)n));
    cast_real_to_cplx_kernel<R><<<256, 256, 0, h->stream>>>(dA, lda, (int)n, H); count_launch();
    if (enqueue_hessenberg_real<R>(H, Hr, Y, Qr, scr, (int)n, h->stream)) return 7;
    if (launch_hessenberg_real_finish<R>(Hr, Qr, H, Q, (int)n, h->stream)) return 7;
    if (cudaStreamSynchronize(h->stream)) return 7;
    return 0;
}

extern "C" int sqrtm_step_hessenberg(sqrtm_handle_t h, const double *dA, int64_t n, int64_t lda, void *dH, void *dQ,
                                     int fp64)
{
    if (!h) return -1;
    if (n < 0) return -3;
    if (lda < std::max<int64_t>(1, n)) return -4;
    if (n == 0) return 0;
    if (!dA) return -2;
    if (!dH) return -5;
    if (!dQ) return -6;
    if (n > 46340) return -3;
    return fp64 ? hess_step<double>(h, dA, n, lda, (cplx<double> *)dH, (cplx<double> *)dQ)
                : hess_step<float>(h, dA, n, lda, (cplx<float> *)dH, (cplx<float> *)dQ);
}

extern "C" int sqrtm_step_schur(sqrtm_handle_t h, void *dT, void *dQ, int64_t n, int fp64)
{
    if (!h) return -1;
    if (n < 0) return -4;
    if (n == 0) return 0;
    return fp64 ? schur_step<double>(h, (cplx<double> *)dT, (cplx<double> *)dQ, n)
                : schur_step<float>(h, (cplx<float> *)dT, (cplx<float> *)dQ, n);
}

extern "C" int sqrtm_step_trisqrt(sqrtm_handle_t h, const void *dT, void *dS, int64_t n, int blks,
                                  int fp64)
{
    if (!h) return -1;
    if (n < 0) return -4;
    if (blks < 1) return -5;
    if (n == 0) return 0;
    StepScratch ss; void *ex;
    if (int rc = step_scratch(h, n, 0, &ss, &ex)) return rc;
    cudaError_t err = fp64 ? launch_trisqrt<double>((const cplx<double> *)dT, (int)n, (cplx<double> *)dS, (int)n, (int)n, blks, ss.iscal + 1, h->stream)
                           : launch_trisqrt<float>((const cplx<float> *)dT, (int)n, (cplx<float> *)dS, (int)n, (int)n, blks, ss.iscal + 1, h->stream);
    if (err) return 7;
    int st = 0;
    if (fetch(h, &st, ss.iscal + 1, sizeof(int))) return 7;
    return st;
}

extern "C" int sqrtm_step_tricbrt(sqrtm_handle_t h, const void *dT, void *dS, void *dV, int64_t n, int blks,
                                  int fp64)
{
    if (!h) return -1;
    if (n < 0) return -5;
    if (blks < 1) return -6;
    if (n == 0) return 0;
    StepScratch ss; void *ex;
    if (int rc = step_scratch(h, n, 0, &ss, &ex)) return rc;
    cudaError_t err = fp64 ? launch_tricbrt<double>((const cplx<double> *)dT, (int)n, (cplx<double> *)dS, (int)n,
                                                    (cplx<double> *)dV, (int)n, (int)n, blks, ss.iscal + 1, h->stream)
                           : launch_tricbrt<float>((const cplx<float> *)dT, (int)n, (cplx<float> *)dS, (int)n,
                                                   (cplx<float> *)dV, (int)n, (int)n, blks, ss.iscal + 1, h->stream);
    if (err) return 7;
    int st = 0;
    if (fetch(h, &st, ss.iscal + 1, sizeof(int))) return 7;
    return st;
}

extern "C" int sqrtm_step_trisqrt_rec(sqrtm_handle_t h, const void *dT, void *dS, int64_t n, int blks, int cutoff,
                                      int fp64)
{
    if (!h) return -1;
    if (n < 0) return -4;
    if (blks < 1) return -5;
    if (n == 0) return 0;
    StepScratch ss; void *ex;
    if (int rc = step_scratch(h, n, 0, &ss, &ex)) return rc;
    cudaError_t err = fp64 ? launch_trisqrt_rec<double>((const cplx<double> *)dT, (int)n, (cplx<double> *)dS, (int)n,
                                                        (int)n, blks, cutoff, ss.iscal + 1, h->stream)
                           : launch_trisqrt_rec<float>((const cplx<float> *)dT, (int)n, (cplx<float> *)dS, (int)n,
                                                       (int)n, blks, cutoff, ss.iscal + 1, h->stream);
    if (err) return 7;
    int st = 0;
    if (fetch(h, &st, ss.iscal + 1, sizeof(int))) return 7;
    return st;
}

extern "C" int sqrtm_step_real_schur(sqrtm_handle_t h, void *dT, void *dQ, int64_t n, int fp64)
{
    if (!h) return -1;
    if (n < 0 || n > 2048) return -4;
    if (n == 0) return 0;
    StepScratch ss; void *ex;
    if (int rc = step_scratch(h, n, 0, &ss, &ex)) return rc;
    cudaError_t err = fp64 ? launch_real_schur<double>((double *)dT, (double *)dQ, (int)n, ss.iscal + 1, nullptr, h->stream)
                           : launch_real_schur<float>((float *)dT, (float *)dQ, (int)n, ss.iscal + 1, nullptr, h->stream);
    if (err) return 7;
    int st = 0;
    if (fetch(h, &st, ss.iscal + 1, sizeof(int))) return 7;
    return st;
}

extern "C" int sqrtm_step_qtrisqrt(sqrtm_handle_t h, const void *dT, void *dS, int64_t n, int fp64)
{
    if (!h) return -1;
    if (n < 0) return -4;
    if (n == 0) return 0;
    StepScratch ss; void *ex;
    if (int rc = step_scratch(h, n, (size_t)(n + 8) * sizeof(int), &ss, &ex)) return rc;
    int *blk = (int *)ex;
    cudaError_t err = fp64 ? launch_qtrisqrt<double>((const double *)dT, (int)n, (double *)dS, (int)n, (int)n, blk,
                                                     ss.iscal + 2, ss.iscal + 1, h->stream)
                           : launch_qtrisqrt<float>((const float *)dT, (int)n, (float *)dS, (int)n, (int)n, blk,
                                                    ss.iscal + 2, ss.iscal + 1, h->stream);
    if (err) return 7;
    int st = 0;
    if (fetch(h, &st, ss.iscal + 1, sizeof(int))) return 7;
    return st;
}

extern "C" int sqrtm_step_qrtrsyl(sqrtm_handle_t h, const void *dS, int64_t m, const void *dSt, int64_t nn, void *dC,
                                  int fp64)
{
    if (!h) return -1;
    if (m < 0) return -3;
    if (nn < 0) return -5;
    if (m == 0 || nn == 0) return 0;
    StepScratch ss; void *ex;
    if (int rc = step_scratch(h, std::max(m, nn), (size_t)(m + nn + 16) * sizeof(int), &ss, &ex)) return rc;
    int *bm = (int *)ex, *bn = bm + m + 8;
    cudaError_t err = fp64 ? launch_qrtrsyl<double>((const double *)dS, (int)m, (int)m, (const double *)dSt, (int)nn,
                                                    (int)nn, (double *)dC, (int)m, bm, bn, ss.iscal + 2, ss.iscal + 1,
                                                    h->stream)
                           : launch_qrtrsyl<float>((const float *)dS, (int)m, (int)m, (const float *)dSt, (int)nn,
                                                   (int)nn, (float *)dC, (int)m, bm, bn, ss.iscal + 2, ss.iscal + 1,
                                                   h->stream);
    if (err) return 7;
    int st = 0;
    if (fetch(h, &st, ss.iscal + 1, sizeof(int))) return 7;
    return st;
}

template <class R>
static int form_x0(sqrtm_handle_t h, const cplx<R> *Q, const cplx<R> *S, int64_t n, int e,
                   double *dX, int64_t ldx)
{
    StepScratch ss; void *ex;
    if (int rc = step_scratch(h, n, (size_t)n * n * sizeof(cplx<R>), &ss, &ex)) return rc;
    cplx<R> *W = (cplx<R> *)ex;
    if (launch_cgemm<R>(OP_N, OP_N, (int)n, (int)n, (int)n, Q, (int)n, false, S, (int)n, EPI_STORE, W, (int)n, nullptr, 0, 0.0, h->stream)) return 7;
    if (launch_cgemm<R>(OP_N, OP_H, (int)n, (int)n, (int)n, W, (int)n, false, Q, (int)n, EPI_REAL_TO_F64, nullptr, 0, dX, ldx, ldexp(1.0, e), h->stream)) return 7;
    return cudaStreamSynchronize(h->stream) ? 7 : 0;
}

extern "C" int sqrtm_step_form_x0(sqrtm_handle_t h, const void *dQ, const void *dS, int64_t n,
                                  int e, double *dX, int64_t ldx, int fp64)
{
    if (!h) return -1;
    if (n < 0) return -4;
    if (ldx < std::max<int64_t>(1, n)) return -7;
    if (n == 0) return 0;
    if (fp64) return form_x0<double>(h, (const cplx<double> *)dQ, (const cplx<double> *)dS, n, e, dX, ldx);
    return form_x0<float>(h, (const cplx<float> *)dQ, (const cplx<float> *)dS, n, e, dX, ldx);
}

extern "C" int sqrtm_step_residual(sqrtm_handle_t h, const double *dA, int64_t lda,
                                   const double *dX, int64_t ldx, int64_t n, int e, float *dRhat,
                                   double *norm_host)
{
    if (!h) return -1;
    if (n < 0) return -6;
    if (lda < std::max<int64_t>(1, n)) return -3;
    if (ldx < std::max<int64_t>(1, n)) return -5;
    if (n == 0) { if (norm_host) *norm_host = 0; return 0; }
    StepScratch ss; void *ex;
    if (int rc = step_scratch(h, n, 0, &ss, &ex)) return rc;
    int np = 0;
    if (launch_residual_f64(dA, lda, dX, ldx, (int)n, e, dRhat, (int)n, ss.dscal + 2, &np, h->stream)) return 7;
    if (launch_sum_partials(ss.dscal + 2, np, ss.dscal + 1, h->stream)) return 7;
    double rn;
    if (fetch(h, &rn, ss.dscal + 1, sizeof(double))) return 7;
    if (norm_host) *norm_host = rn;
    return 0;
}

extern "C" int sqrtm_step_residual_split(sqrtm_handle_t h, const double *dA, int64_t lda, const double *dX,
                                         int64_t ldx, int64_t n, int e, float *dRhat, double *norm_host)
{
    if (!h) return -1;
    if (n < 0) return -6;
    if (lda < std::max<int64_t>(1, n)) return -3;
    if (ldx < std::max<int64_t>(1, n)) return -5;
    if (n > 46340) return -6;
    if (!split_residual_supported((int)n)) return -10;
    if (n == 0) { if (norm_host) *norm_host = 0; return 0; }
    const size_t nn = (size_t)n * n;
    const size_t extra = 2 * Carve::round(nn * sizeof(double)) + 2 * Carve::round(split_digit_elems((int)n) * 2) +
                         2 * Carve::round(n * sizeof(int));
    StepScratch ss; void *ex;
    if (int rc = step_scratch(h, n, extra, &ss, &ex)) return rc;
    Carve c(ex);
    double *Racc = c.take<double>(nn);
    double *XT = c.take<double>(nn);
    void *da = c.take<uint16_t>(split_digit_elems((int)n));
    void *db = c.take<uint16_t>(split_digit_elems((int)n));
    int *rhoA = c.take<int>(n);
    int *rhoB = c.take<int>(n);
    int np = 0;
    if (launch_residual_gen_split(dA, lda, dX, ldx, (int)n, e, dRhat, (int)n, Racc, XT, da, db, rhoA, rhoB,
                                  ss.dscal + 2, &np, ss.iscal + 1, h->stream)) return 7;
    if (launch_sum_partials(ss.dscal + 2, np, ss.dscal + 1, h->stream)) return 7;
    double rn;
    int st = 0;
    if (fetch(h, &rn, ss.dscal + 1, sizeof(double)) || fetch(h, &st, ss.iscal + 1, sizeof(int))) return 7;
    if (norm_host) *norm_host = rn;
    return st;
}

extern "C" int sqrtm_step_residual_sym(sqrtm_handle_t h, const double *dA, int64_t lda, const double *dX,
                                       int64_t ldx, int64_t n, int e, float *dRhat, double *norm_host,
                                       int split)
{
    if (!h) return -1;
    if (n < 0) return -6;
    if (lda < std::max<int64_t>(1, n)) return -3;
    if (ldx < std::max<int64_t>(1, n)) return -5;
    if (n > 46340) return -6;
    if (split && !split_residual_supported((int)n)) return -10;
    if (n == 0) { if (norm_host) *norm_host = 0; return 0; }
    const size_t nn = (size_t)n * n;
    const size_t extra = split ? Carve::round(nn * sizeof(double)) + Carve::round(split_digit_elems((int)n) * 2) +
                                     Carve::round(n * sizeof(int))
                               : 0;
    StepScratch ss; void *ex;
    if (int rc = step_scratch(h, n, extra, &ss, &ex)) return rc;
    int np = 0;
    if (split) {
        Carve c(ex);
        double *Racc = c.take<double>(nn);
        void *digits = c.take<uint16_t>(split_digit_elems((int)n));
        int *rho = c.take<int>(n);
        if (launch_residual_sym_split(dA, lda, dX, ldx, (int)n, e, dRhat, (int)n, Racc, digits, rho, ss.dscal + 2,
                                      &np, ss.iscal + 1, h->stream)) return 7;
    } else if (launch_residual_sym_f64(dA, lda, dX, ldx, (int)n, e, dRhat, (int)n, ss.dscal + 2, &np, h->stream)) {
        return 7;
    }
    if (launch_sum_partials(ss.dscal + 2, np, ss.dscal + 1, h->stream)) return 7;
    double rn;
    int st = 0;
    if (fetch(h, &rn, ss.dscal + 1, sizeof(double)) || fetch(h, &st, ss.iscal + 1, sizeof(int))) return 7;
    if (norm_host) *norm_host = rn;
    return st;
}

extern "C" int sqrtm_step_transform_in(sqrtm_handle_t h, const void *dQ, const float *dRhat,
                                       void *dRt, int64_t n)
{
    if (!h) return -1;
    if (n < 0) return -5;
    if (n == 0) return 0;
    StepScratch ss; void *ex;
    if (int rc = step_scratch(h, n, (size_t)n * n * sizeof(cplx<float>), &ss, &ex)) return rc;
    cplx<float> *W = (cplx<float> *)ex;
    const cplx<float> *Q = (const cplx<float> *)dQ;
    if (launch_cgemm<float>(OP_N, OP_N, (int)n, (int)n, (int)n, dRhat, (int)n, true, Q, (int)n, EPI_STORE, W, (int)n, nullptr, 0, 0.0, h->stream)) return 7;
    if (launch_cgemm<float>(OP_H, OP_N, (int)n, (int)n, (int)n, Q, (int)n, false, W, (int)n, EPI_STORE, (cplx<float> *)dRt, (int)n, nullptr, 0, 0.0, h->stream)) return 7;
    return cudaStreamSynchronize(h->stream) ? 7 : 0;
}

extern "C" int sqrtm_step_rtrsyl(sqrtm_handle_t h, const void *dS, int64_t m, const void *dSt,
                                 int64_t nn, void *dC, int blks)
{
    if (!h) return -1;
    if (m < 0) return -3;
    if (nn < 0) return -5;
    if (blks < 1) return -7;
    if (m == 0 || nn == 0) return 0;
    StepScratch ss; void *ex;
    const size_t fi = rtrsyl_flow_ints((int)m, (int)nn);
    if (int rc = step_scratch(h, std::max(m, nn), fi * sizeof(int), &ss, &ex)) return rc;
    if (launch_rtrsyl<float>((const cplx<float> *)dS, (int)m, (int)m, (const cplx<float> *)dSt, (int)nn, (int)nn,
                             (cplx<float> *)dC, (int)m, blks, ss.iscal + 1, h->stream, (int *)ex, (int64_t)fi)) return 7;
    int st = 0;
    if (fetch(h, &st, ss.iscal + 1, sizeof(int))) return 7;
    return st;
}

extern "C" int sqrtm_step_rtrsyl3(sqrtm_handle_t h, const void *dS, const void *dV, void *dC, int64_t n, int blks,
                                  int fp64)
{
    if (!h) return -1;
    if (n < 0) return -5;
    if (blks < 1) return -6;
    if (n == 0) return 0;
    StepScratch ss; void *ex;
    const size_t zb = (size_t)n * n * (fp64 ? sizeof(cplx<double>) : sizeof(cplx<float>));
    if (int rc = step_scratch(h, n, zb, &ss, &ex)) return rc;
    cudaError_t err = fp64 ? launch_rtrsyl3<double>((const cplx<double> *)dS, (int)n, (const cplx<double> *)dV, (int)n,
                                                    (cplx<double> *)dC, (int)n, (cplx<double> *)ex, (int)n, (int)n,
                                                    blks, ss.iscal + 1, h->stream)
                           : launch_rtrsyl3<float>((const cplx<float> *)dS, (int)n, (const cplx<float> *)dV, (int)n,
                                                   (cplx<float> *)dC, (int)n, (cplx<float> *)ex, (int)n, (int)n, blks,
                                                   ss.iscal + 1, h->stream);
    if (err) return 7;
    int st = 0;
    if (fetch(h, &st, ss.iscal + 1, sizeof(int))) return 7;
    return st;
}

extern "C" int sqrtm_step_transform_out_update(sqrtm_handle_t h, const void *dQ, const void *dY,
                                               int64_t n, int e, double *dX, int64_t ldx)
{
    if (!h) return -1;
    if (n < 0) return -4;
    if (ldx < std::max<int64_t>(1, n)) return -7;
    if (n == 0) return 0;
    StepScratch ss; void *ex;
    if (int rc = step_scratch(h, n, (size_t)n * n * sizeof(cplx<float>), &ss, &ex)) return rc;
    cplx<float> *W = (cplx<float> *)ex;
    const cplx<float> *Q = (const cplx<float> *)dQ;
    if (launch_cgemm<float>(OP_N, OP_N, (int)n, (int)n, (int)n, Q, (int)n, false, (const cplx<float> *)dY, (int)n, EPI_STORE, W, (int)n, nullptr, 0, 0.0, h->stream)) return 7;
    if (launch_cgemm<float>(OP_N, OP_H, (int)n, (int)n, (int)n, W, (int)n, false, Q, (int)n, EPI_REAL_ADD_F64, nullptr, 0, dX, ldx, ldexp(1.0, e), h->stream)) return 7;
    return cudaStreamSynchronize(h->stream) ? 7 : 0;
}

extern "C" int sqrtm_step_gemm_tf32x3(sqrtm_handle_t h, int64_t M, int64_t N, int64_t K,
                                      const float *dA, int64_t lda, const float *dB, int64_t ldb,
                                      float *dC, int64_t ldc)
{
    if (!h) return -1;
    if (M < 0 || N < 0 || K < 0) return -2;
    if (M == 0 || N == 0) return 0;
    if (K == 0 || !tc_gemm_supported(M, N, K, lda, ldb, dA, dB) || ldc < M) return -4;
    StepScratch ss; void *ex;
    if (int rc = step_scratch(h, 1, 0, &ss, &ex)) return rc;
    TcEpilogue ep{};
    ep.C = dC; ep.ldc = ldc;
    if (launch_tc3_gemm((int)M, (int)N, (int)K, dA, (int)lda, dB, (int)ldb, TC_EPI_STORE, ep, ss.iscal + 1, h->stream)) return 7;
    int st = 0;
    if (fetch(h, &st, ss.iscal + 1, sizeof(int))) return 7;
    return st;
}

extern "C" int sqrtm_step_cgemm_tf32x3(sqrtm_handle_t h, int64_t M, int64_t N, int64_t K, const void *dA,
                                       int64_t lda, int conj_a, const void *dY, int64_t ldy, int conj_y, void *dC,
                                       int64_t ldc)
{
    if (!h) return -1;
    if (M < 0 || N < 0 || K < 0) return -2;
    if (M == 0 || N == 0) return 0;
    if (!dA || !dY || !dC) return -5;
    if (K == 0 || lda < K || ldy < K || ldc < M) return -6;
    const int64_t ldb = (2 * K + 3) / 4 * 4;  // re-laid Y: 2K floats per column, TMA-aligned
    if (!tc_cgemm_supported(lda, ldb, dA, dA)) return -6;
    StepScratch ss; void *ex;
    if (int rc = step_scratch(h, 1, (size_t)ldb * 2 * N * sizeof(float), &ss, &ex)) return rc;
    float *B = (float *)ex;
    if (launch_tc_relayout_cplx(dY, ldy, (int)K, (int)N, conj_a ? -1.0f : 1.0f, conj_y ? -1.0f : 1.0f, false, B, ldb,
                                h->stream))
        return 7;
    TcEpilogue ep{};
    ep.C = (float *)dC; ep.ldc = ldc;
    if (launch_tc_cgemm((int)M, (int)N, (int)K, dA, (int)lda, B, (int)ldb, TC_EPI_CSTORE, ep, ss.iscal + 1, h->stream))
        return 7;
    int st = 0;
    if (fetch(h, &st, ss.iscal + 1, sizeof(int))) return 7;
    return st;
}
