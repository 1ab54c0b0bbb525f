// adjoint.cu -- sqrtm_backward: gradient of <Gbar, sqrt(A)> with respect to A.
//
// The derivative of X = sqrt(A) in direction E is the F with X F + F X = E
// (the operator of the correction equation, Eq. (correction)), so the
// gradient is the solution Y of the adjoint equation X^T Y + Y X^T = Gbar.
// It is computed with the same frozen low-precision factors as the forward
// refinement (X_s = 2^-e X ~ Q S Q^H, Eq. (triangsylv)):
//   general: transposing, W = Y^T solves X W + W X = Gbar^T, so
//            Y ~ 2^-e Re(Q V Q^H)^T with S V + V S = Q^H Rhat^T Q
//            (the Sylvester solver of Algorithm 1's equation);
//   SPD:     X is symmetric, Y ~ 2^-e V [(V^T Rhat V) ./ (s_i + s_j)] V^T.
// FP64 refinement with the adjoint residual Res = Gbar - (X^T Y + Y X^T)
// (the approximate-Newton pattern of Algorithm 2 applied to a linear
// equation) runs until ||Res||_F <= tol ||Gbar||_F or maxit corrections.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "handle.h"
#include "spd_internal.h"

using namespace sqm;

namespace {

// The factors one backward pass uses: those the handle keeps from its last
// forward call, or those of a detached factor object.
struct FactView {
    int64_t n;
    int kind, e;
    const void *q, *s;
    const double *x;
};

// The adjoint solve and its refinement on the handle's stream and workspace
// with the factors f (f.n == n, already checked).
int backward_impl(sqrtm_handle_t h, const FactView &f, const double *dG, int64_t n, int64_t ldg, double tol,
                  double *dY, int64_t ldy, sqrtm_info *info)
{
    cudaStream_t s = h->stream;
    const int ni = (int)n;
    const size_t nn = (size_t)n * n;
    const bool spd = f.kind == SQRTM_KIND_SPD;
    const int e = f.e;
    const double scale = ldexp(1.0, -e);
    int64_t nb = (n + 63) / 64;
    size_t np_cap = (size_t)std::max<int64_t>(nb * nb, 2048) + 8;
    size_t need = Carve::round(np_cap * sizeof(double)) + 256 + Carve::round(nn * sizeof(float)) +
                  2 * Carve::round(nn * sizeof(cplx<float>)) + 4096;
    if (ensure(h->ws, need, h)) return 7;
    Carve c(h->ws.p);
    double *dscal = c.take<double>(np_cap);
    int *iscal = c.take<int>(8);
    float *Rhat = c.take<float>(nn);
    cplx<float> *W = c.take<cplx<float>>(nn);
    cplx<float> *Rt = c.take<cplx<float>>(nn);
    if (cudaMemsetAsync(iscal, 0, 8 * sizeof(int), s)) return 7;
    if (cudaMemset2DAsync(dY, ldy * sizeof(double), 0, n * sizeof(double), n, s)) return 7;
    if (cudaEventRecord(h->ev[0], s)) return 7;

    const int maxit = 10;
    int status = 1, applied = 0, grew = 0;
    double gnorm = -1.0, prev = INFINITY;
    for (int k = 0; k <= maxit + 1; ++k) {
        int np = 0;
        if (launch_adjoint_residual_f64(dG, ldg, f.x, n, dY, ldy, ni, Rhat, ni, dscal + 2, &np, s)) return 7;
        if (launch_sum_partials(dscal + 2, np, dscal + 1, s)) return 7;
        if (cudaMemcpyAsync(h->staging.p, dscal + 1, sizeof(double), cudaMemcpyDeviceToHost, s)) return 7;
        if (cudaStreamSynchronize(s)) return 7;
        double rn;
        memcpy(&rn, h->staging.p, sizeof(double));
        if (k == 0) {
            gnorm = rn;  // Y = 0: the residual is Gbar itself
            if (info) info->norm_a = gnorm;
            if (gnorm == 0.0) { status = 0; break; }
            if (!isfinite(gnorm)) { status = 5; break; }
        }
        double rel = rn / gnorm;
        if (info && info->history_len < SQRTM_MAX_HISTORY) info->history[info->history_len++] = rel;
        if (!isfinite(rel)) { status = 4; break; }
        if (k > 0 && rel <= tol) { status = 0; break; }
        if (k > maxit) { status = 1; break; }
        grew = (rn > prev) ? grew + 1 : 0;
        if (grew >= 2) { status = 4; break; }
        prev = rn;
        if (spd) {
            const float *V = (const float *)f.q, *sv = (const float *)f.s;
            float *Wf = (float *)W, *Yf = (float *)Rt;
            if (launch_rgemm<float>(0, 0, ni, ni, ni, Rhat, ni, V, ni, RG_STORE, Wf, ni, nullptr, nullptr, 0, 0.0, s)) return 7;
            if (launch_rgemm<float>(1, 0, ni, ni, ni, V, ni, Wf, ni, RG_DIAG_SOLVE, Yf, ni, sv, nullptr, 0, 0.0, s)) return 7;
            if (launch_rgemm<float>(0, 0, ni, ni, ni, V, ni, Yf, ni, RG_STORE, Wf, ni, nullptr, nullptr, 0, 0.0, s)) return 7;
            if (launch_rgemm<float>(0, 1, ni, ni, ni, Wf, ni, V, ni, RG_ADD_F64, nullptr, 0, nullptr, dY, ldy, scale, s)) return 7;
        } else {
            const cplx<float> *Q = (const cplx<float> *)f.q, *S = (const cplx<float> *)f.s;
            // Rt = Q^H Rhat^T Q; S V + V S = Rt; Y += 2^-e Re(Q V Q^H)^T
            if (launch_cgemm<float>(OP_H, OP_N, ni, ni, ni, Rhat, ni, true, Q, ni, EPI_STORE, W, ni, nullptr, 0, 0.0, s)) return 7;
            if (launch_cgemm<float>(OP_H, OP_N, ni, ni, ni, Q, ni, false, W, ni, EPI_STORE, Rt, ni, nullptr, 0, 0.0, s)) return 7;
            if (launch_rtrsyl<float>(S, ni, ni, S, ni, ni, Rt, ni, 32, iscal + 1, s)) return 7;
            if (launch_cgemm<float>(OP_N, OP_N, ni, ni, ni, Q, ni, false, Rt, ni, EPI_STORE, W, ni, nullptr, 0, 0.0, s)) return 7;
            if (launch_cgemm<float>(OP_N, OP_H, ni, ni, ni, W, ni, false, Q, ni, EPI_REAL_ADD_F64_T, nullptr, 0, dY, ldy, scale, s)) return 7;
        }
        ++applied;
    }
    if (cudaEventRecord(h->ev[1], s)) return 7;
    int st = 0;
    if (cudaMemcpyAsync(h->staging.p, iscal + 1, sizeof(int), cudaMemcpyDeviceToHost, s)) return 7;
    if (cudaStreamSynchronize(s)) return 7;
    memcpy(&st, h->staging.p, sizeof(int));
    if (info) {
        info->iterations = applied;
        info->kind_used = f.kind;
        info->scale_exponent = e;
        float ms = 0;
        cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]);
        info->ms_refine = ms;
        info->status = st ? st : status;
    }
    return st ? st : status;
}

}  // namespace

extern "C" int sqrtm_backward(sqrtm_handle_t h, const double *dG, int64_t n, int64_t ldg,
                              double tol, double *dY, int64_t ldy, sqrtm_info *info)
{
    if (info) memset(info, 0, sizeof(*info));
    if (!h) return -1;
    if (n < 0) return -3;
    if (n > 0 && !dG) return -2;
    if (ldg < std::max<int64_t>(1, n)) return -4;
    if (n > 0 && !dY) return -6;
    if (ldy < std::max<int64_t>(1, n)) return -7;
    if (n == 0) return 0;
    if (h->fact_n != n || !h->fact_x) return 8;
    const FactView f{h->fact_n, h->fact_kind, h->fact_e, h->fact_q, h->fact_s, h->fact_x};
    return backward_impl(h, f, dG, n, ldg, tol, dY, ldy, info);
}

extern "C" int sqrtm_backward_factors(sqrtm_handle_t h, sqrtm_factors_t fo, const double *dG, int64_t n,
                                      int64_t ldg, double tol, double *dY, int64_t ldy, sqrtm_info *info)
{
    if (info) memset(info, 0, sizeof(*info));
    if (!h) return -1;
    if (!fo) return -2;
    if (n < 0) return -4;
    if (n > 0 && !dG) return -3;
    if (ldg < std::max<int64_t>(1, n)) return -5;
    if (n > 0 && !dY) return -7;
    if (ldy < std::max<int64_t>(1, n)) return -8;
    if (n == 0) return 0;
    if (fo->n != n || !fo->x) return 8;
    const FactView f{fo->n, fo->kind, fo->e, fo->q, fo->s, fo->x};
    return backward_impl(h, f, dG, n, ldg, tol, dY, ldy, info);
}

extern "C" int sqrtm_factors_take(sqrtm_handle_t h, sqrtm_factors_t *out)
{
    if (!h) return -1;
    if (!out) return -2;
    *out = nullptr;
    if (h->fact_n < 0 || !h->fact_x) return 8;
    sqrtm_factors_s *f = new (std::nothrow) sqrtm_factors_s();
    if (!f) return 7;
    // the buffer changes owner; no cached graph takes its address as a key
    // or bakes it into a launch (the kernels read factor pointers from
    // descriptors rewritten by every call), so nothing is dropped here
    f->mem = h->fact;
    f->n = h->fact_n;
    f->kind = h->fact_kind;
    f->e = h->fact_e;
    f->norm = h->fact_norm;
    f->q = h->fact_q;
    f->s = h->fact_s;
    f->x = h->fact_x;
    h->fact = Buf{};
    h->fact_n = -1;
    h->fact_q = h->fact_s = nullptr;
    h->fact_x = nullptr;
    *out = f;
    return 0;
}

extern "C" int64_t sqrtm_factors_n(sqrtm_factors_t f) { return f ? f->n : -1; }

extern "C" int sqrtm_factors_destroy(sqrtm_factors_t f)
{
    if (!f) return 0;
    if (f->mem.p) cudaFree(f->mem.p);
    delete f;
    return 0;
}
