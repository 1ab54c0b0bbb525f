// api.cu -- C ABI of the library: handle and workspace management, the
// drivers of Algorithm 2 (general A), Algorithm 3 (SPD A), the plain FP64
// Schur method, the adjoint solve and the step-level entry points.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "handle.h"
#include "spd_internal.h"
#include "tc_gemm.h"

using namespace sqm;

#include <atomic>
static std::atomic<long long> g_launches{0};
void sqm::count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

extern "C" int64_t sqrtm_kernel_launches(void) { return (int64_t)g_launches.load(); }

cudaError_t sqm::allow_max_smem(const void *kernel)
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kernel)) != cudaSuccess) return e;
    // the dynamic part may use what the kernel's static shared memory leaves
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

// ---------------------------------------------------------------------------
// captured launch sequences
// ---------------------------------------------------------------------------
int run_graph(sqrtm_handle_t h, int tag, const void *key, int64_t n, int batch,
              cudaError_t (*enqueue)(void *ctx, cudaStream_t s), void *ctx, uint64_t sig)
{
    for (auto &g : h->graphs) {
        if (g.tag == tag && g.key == key && g.n == n && g.batch == batch && g.sig == sig) {
            if (cudaGraphLaunch(g.exec, h->stream) != cudaSuccess) return 7;
            g_launches.fetch_add(g.launches, std::memory_order_relaxed);
            return 0;
        }
    }
    if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return 7;
    long long before = g_launches.load();
    cudaGraph_t graph = nullptr;
    cudaError_t e0 = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed);
    if (e0 != cudaSuccess) { note_error(h, cudaGetErrorName(e0), __LINE__, 7); return 7; }
    cudaError_t err = enqueue(ctx, h->cap_stream);
    cudaError_t err2 = cudaStreamEndCapture(h->cap_stream, &graph);
    if (err != cudaSuccess || err2 != cudaSuccess || !graph) {
        note_error(h, cudaGetErrorName(err != cudaSuccess ? err : err2), __LINE__, 7);
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return 7;
    }
    long long nl = g_launches.load() - before;
    g_launches.fetch_sub(nl, std::memory_order_relaxed);  // counted when the graph runs
    cudaGraphExec_t exec = nullptr;
    err = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (err != cudaSuccess) { note_error(h, cudaGetErrorName(err), __LINE__, 7); return 7; }
    h->graphs.push_back({tag, key, n, batch, sig, exec, nl});
    if (cudaGraphLaunch(exec, h->stream) != cudaSuccess) return 7;
    g_launches.fetch_add(nl, std::memory_order_relaxed);
    return 0;
}

cudaError_t sqm::capture_while(cudaStream_t s, cudaStream_t body_stream, unsigned init, CondFn body, void *ctx,
                               CondFn pre)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edges = nullptr;
    size_t nd = 0;
    cudaError_t err = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &nd);
    if (err) return err;
    if (cs != cudaStreamCaptureStatusActive || !g) return cudaErrorStreamCaptureUnmatched;
    cudaGraphConditionalHandle cond;
    if ((err = cudaGraphConditionalHandleCreate(&cond, g, init, cudaGraphCondAssignDefault))) return err;
    if (pre) {
        if ((err = pre(ctx, s, cond))) return err;
        // the node goes after what pre added
        if ((err = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &nd))) return err;
    }
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = cond;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if ((err = cudaGraphAddNode(&node, g, deps, edges, nd, &p))) return err;
    cudaGraph_t body_graph = p.conditional.phGraph_out[0];
    if ((err = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies))) return err;
    if ((err = cudaStreamBeginCaptureToGraph(body_stream, body_graph, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeRelaxed)))
        return err;
    cudaError_t e1 = body(ctx, body_stream, cond);
    cudaGraph_t out = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(body_stream, &out);
    return e1 ? e1 : e2;
}

void note_error(sqrtm_handle_t h, const char *what, int line, int code)
{
    if (!h || h->last_error[0]) return;
    snprintf(h->last_error, sizeof(h->last_error), "status %d: %s (api.cu/qr/spd line %d)", code, what, line);
}

extern "C" const char *sqrtm_last_error(sqrtm_handle_t h)
{
    if (!h) return "";
    return h->last_error;
}

void drop_graphs(sqrtm_handle_t h, const void *lo, const void *hi)
{
    for (size_t i = 0; i < h->graphs.size();) {
        const char *k = (const char *)h->graphs[i].key;
        if (k >= (const char *)lo && k < (const char *)hi) {
            cudaGraphExecDestroy(h->graphs[i].exec);
            h->graphs.erase(h->graphs.begin() + i);
        } else {
            ++i;
        }
    }
}

extern "C" int sqrtm_create(sqrtm_handle_t *handle, void *stream)
{
    if (!handle) return -1;
    sqrtm_handle_s *h = new sqrtm_handle_s();
    h->stream = (cudaStream_t)stream;
    for (auto &e : h->ev)
        if (cudaEventCreate(&e) != cudaSuccess) { delete h; return 7; }
    for (auto &e : h->qev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) { delete h; return 7; }
    if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess) { delete h; return 7; }
    if (cudaMallocHost(&h->staging.p, 4096) != cudaSuccess) { delete h; return 7; }
    h->staging.bytes = 4096;
    *handle = h;
    return 0;
}

extern "C" int sqrtm_destroy(sqrtm_handle_t h)
{
    if (!h) return 0;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    for (size_t w = 0; w < h->workers.size(); ++w) {
        sqrtm_destroy(h->workers[w]);
        cudaStreamDestroy(h->worker_streams[w]);
    }
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->body_stream) cudaStreamDestroy(h->body_stream);
    if (h->side) {
        cudaStreamSynchronize(h->side);
        cudaStreamDestroy(h->side);
    }
    for (auto &e : h->qev)
        if (e) cudaEventDestroy(e);
    if (h->ws.p) cudaFree(h->ws.p);
    if (h->bws.p) cudaFree(h->bws.p);
    if (h->bpin) cudaFreeHost(h->bpin);
    if (h->fact.p) cudaFree(h->fact.p);
    if (h->staging.p) cudaFreeHost(h->staging.p);
    for (auto &e : h->ev)
        if (e) cudaEventDestroy(e);
    delete h;
    return 0;
}

extern "C" int sqrtm_set_stream(sqrtm_handle_t h, void *stream)
{
    if (!h) return -1;
    h->stream = (cudaStream_t)stream;
    return 0;
}

extern "C" int sqrtm_set_wait_limit(sqrtm_handle_t h, int64_t ns)
{
    if (!h) return -1;
    if (ns < 0) return -2;
    h->wait_ns = (unsigned long long)ns;
    for (auto *w : h->workers) w->wait_ns = h->wait_ns;
    return 0;
}

extern "C" void sqrtm_default_opts(sqrtm_opts *o)
{
    if (!o) return;
    o->tol = 1e-12;
    o->maxit = 10;
    o->blks = 0;
    o->kind = SQRTM_KIND_AUTO;
    o->precision = SQRTM_PREC_AUTO;
    o->steps = -1;
}

extern "C" int sqrtm_set_tuning(sqrtm_handle_t h, const sqrtm_tune_entry *table, int count)
{
    if (!h) return -1;
    if (count < 0 || count > SQRTM_MAX_TUNE) return -3;
    if (count > 0 && !table) return -2;
    for (int i = 0; i < count; ++i) {
        const sqrtm_tune_entry &t = table[i];
        if (t.n_max < 1 || (i > 0 && t.n_max <= table[i - 1].n_max)) return -4;
        if (t.blks < 1 || t.blks > 32 || t.qr_helpers < -1 || t.qr_helpers > 24) return -4;
        if ((t.batched != 0 && t.batched != 1) || t.spd_precision < 0 || t.spd_precision > 7) return -4;
        if (t.trisqrt_cutoff < 0 || (t.batched_spd != 0 && t.batched_spd != 1)) return -4;
    }
    h->tuning.assign(table, table + count);
    for (auto *w : h->workers) w->tuning = h->tuning;
    return 0;
}

extern "C" int sqrtm_get_tuning(sqrtm_handle_t h, sqrtm_tune_entry *table, int cap)
{
    if (!h) return -1;
    const int cnt = (int)h->tuning.size();
    for (int i = 0; i < cnt && i < cap && table; ++i) table[i] = h->tuning[i];
    return cnt;
}

const sqrtm_tune_entry *tune_for(sqrtm_handle_t h, int64_t n)
{
    if (!h || h->tuning.empty()) return nullptr;
    for (const auto &t : h->tuning)
        if (n <= t.n_max) return &t;
    return &h->tuning.back();
}

void apply_tuning(sqrtm_handle_t h, int64_t n, sqrtm_opts *o)
{
    const sqrtm_tune_entry *t = tune_for(h, n);
    if (o->blks == 0) o->blks = t ? t->blks : 32;
    if (o->precision == SQRTM_PREC_AUTO) o->precision = t ? t->spd_precision : SQRTM_PREC_FP32;
}

extern "C" const char *sqrtm_status_string(int code)
{
    switch (code) {
    case 0: return "success";
    case 1: return "refinement did not reach the tolerance within maxit steps";
    case 2: return "eigenvalue on or next to the closed negative real axis";
    case 3: return "Schur/eigensolver iteration cap reached";
    case 4: return "refinement diverged";
    case 5: return "input contains NaN or Inf";
    case 6: return "device-side wait gave up";
    case 7: return "CUDA error or allocation failure";
    case 8: return "no factors saved on the handle";
    default: return code < 0 ? "invalid argument" : "unknown status";
    }
}

static void info_reset(sqrtm_info *info)
{
    if (!info) return;
    memset(info, 0, sizeof(*info));
}

// scalars in device workspace: [0] norm, [1] residual norm, [2..] partials;
// ints: e, status(schur), status(trisqrt/solve)
struct Scalars {
    double *norm, *rnorm, *partials;
    int *e, *st_schur, *st_solve;
    int npart_cap;
};

static size_t scalars_bytes(int64_t n)
{
    int64_t nb = (n + 63) / 64;
    int64_t np = std::max<int64_t>(nb * nb, 2048);
    return Carve::round((np + 8) * sizeof(double)) + 256;
}

static Scalars carve_scalars(Carve &c, int64_t n)
{
    Scalars s;
    int64_t nb = (n + 63) / 64;
    s.npart_cap = (int)std::max<int64_t>(nb * nb, 2048);
    s.norm = c.take<double>(s.npart_cap + 8);
    s.rnorm = s.norm + 1;
    s.partials = s.norm + 2;
    int *iv = c.take<int>(16);
    s.e = iv;
    s.st_schur = iv + 1;
    s.st_solve = iv + 2;
    return s;
}

static int check_args(const void *A, int64_t n, int64_t lda, const void *X, int64_t ldx)
{
    if (n < 0) return -3;
    if (n > 0 && !A) return -2;
    if (lda < std::max<int64_t>(1, n)) return -4;
    if (n > 0 && !X) return -6;
    if (ldx < std::max<int64_t>(1, n)) return -7;
    if (n > 46340) return -3;  // n*n must fit the int indexing of the tiles
    return 0;
}

// host read of device scalars through pinned staging
static int read_scalars(sqrtm_handle_t h, const Scalars &s, double *norm, double *rnorm, int *e,
                        int *st_schur, int *st_solve)
{
    char *st = (char *)h->staging.p;
    SQM_CU(cudaMemcpyAsync(st, s.norm, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    SQM_CU(cudaMemcpyAsync(st + 16, s.e, 3 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    SQM_CU(cudaStreamSynchronize(h->stream));
    double *dv = (double *)st;
    int *iv = (int *)(st + 16);
    if (norm) *norm = dv[0];
    if (rnorm) *rnorm = dv[1];
    if (e) *e = iv[0];
    if (st_schur) *st_schur = iv[1];
    if (st_solve) *st_solve = iv[2];
    return 0;
}

static bool is_bitwise_symmetric(sqrtm_handle_t h, const double *dA, int64_t n, int64_t lda,
                                 int *flag_dev, int *rc);

// smallest n whose general-path residual uses the split-BF16 tensor-core
// products (below it the FP64 CUDA-core product is as fast)
static constexpr int64_t kGenSplitMinN = 512;

// ---------------------------------------------------------------------------
// general path (Algorithm 2) in storage precision R; refine = false gives the
// plain Schur method.  root = 3 gives the principal cube root (Sec. 4, p = 3)
// by the same steps: the triangular cube root S with V = S^2 in place of the
// triangular square root, the residual A - X (X X), and the correction
// equation S^2 Y + S Y S + Y S^2 = Q^H R Q (Eq. (3rd-order)).  cin: A and
// X are complex (interleaved FP64 pairs, lda / ldx in complex elements); the
// steps are the same with complex iterates (no real part taken).
// ---------------------------------------------------------------------------
template <class R>
static int general_path(sqrtm_handle_t h, const double *dA, int64_t n, int64_t lda, double tol,
                        double *dX, int64_t ldx, const sqrtm_opts &o, sqrtm_info *info,
                        bool refine, int root = 2, bool cin = false)
{
    cudaStream_t s = h->stream;
    const size_t nn = (size_t)n * (size_t)n;
    const size_t cb = sizeof(cplx<R>);
    // factors: Q, S persist for the adjoint
    size_t fbytes = 2 * Carve::round(nn * cb) + Carve::round(nn * sizeof(double)) + 1024;
    size_t wbytes = scalars_bytes(n) + 3 * Carve::round(nn * cb) + Carve::round(nn * sizeof(float) * (cin ? 2 : 1)) +
                    Carve::round((n + 8) * cb) + Carve::round(8 * sizeof(R)) +
                    Carve::round(2 * sizeof(SchurDesc<R>)) +
                    2 * (Carve::round(qr_log_capacity(n) * sizeof(RotLog<R>)) +
                         Carve::round(qr_win_capacity(n) * sizeof(WinRec)) + Carve::round(qr_u_capacity(n) * cb)) +
                    Carve::round(kQrStateInts * sizeof(int)) + Carve::round(4 * sizeof(int)) + Carve::round(32 * sizeof(int)) + Carve::round(qr_win_capacity(n) * sizeof(int)) + 4096 +
                    (root == 3 ? Carve::round(nn * cb) : 0) + Carve::round(rtrsyl_flow_ints((int)n, (int)n) * sizeof(int));
    // split-TF32 tensor-core transforms (X_0 = Q S Q^H, R~ = Q^H Rhat Q,
    // X += Re(Q Y Q^H)) for the FP32 square root of a real matrix of even
    // size: each complex product is one real product over interleaved
    // operands (tc_gemm.h), with Q^T and two re-laid copies of Q formed once
    // per factorisation; the re-laid right operands need 2n-float columns
    const bool use_tc = sizeof(R) == sizeof(float) && root == 2 && !cin && refine && (n % 2) == 0 && n >= 128 &&
                        (o.precision & SQRTM_PREC_TF32X3_GENERAL) != 0;
    const size_t tcf = 4 * nn;  // floats of one full re-laid n x n complex operand (2n x 2n)
    if (use_tc)
        wbytes += Carve::round(nn * cb) + 3 * Carve::round(tcf * sizeof(float)) + Carve::round(2 * nn * sizeof(float));
    // FP64 residual of a real iterate (the FP32 square root) from exact
    // split-BF16 tensor-core products (rows of X against its columns) from
    // kGenSplitMinN on, unless SQRTM_PREC_RESID_FP64 asks for FP64 products
    const int64_t npart_cap = std::max<int64_t>(((n + 63) / 64) * ((n + 63) / 64), 2048);
    const bool use_gsplit = sizeof(R) == sizeof(float) && root == 2 && !cin && refine && n >= kGenSplitMinN &&
                            n <= 46340 && !(o.precision & SQRTM_PREC_RESID_FP64) && split_residual_supported((int)n) &&
                            residual_gen_split_parts((int)n) <= npart_cap;
    if (use_gsplit)
        wbytes += 2 * Carve::round(nn * sizeof(double)) + 2 * Carve::round(split_digit_elems((int)n) * 2) +
                  2 * Carve::round(n * sizeof(int));
    if (ensure(h->fact, fbytes, h) || ensure(h->ws, wbytes, h)) return 7;
    Carve cf(h->fact.p);
    cplx<R> *Q = cf.take<cplx<R>>(nn);
    cplx<R> *S = cf.take<cplx<R>>(nn);
    double *Xsave = cf.take<double>(nn);
    Carve cw(h->ws.p);
    Scalars sc = carve_scalars(cw, n);
    cplx<R> *T = cw.take<cplx<R>>(nn);
    cplx<R> *W = cw.take<cplx<R>>(nn);
    cplx<R> *Rt = cw.take<cplx<R>>(nn);
    float *Rhat = cw.take<float>(cin ? 2 * nn : nn);  // complex input: fl32 of a complex residual
    cplx<R> *v = cw.take<cplx<R>>(n + 8);
    R *beta = cw.take<R>(8);
    // two descriptors of the same matrix with separate log / window / U
    // buffers: chase rounds alternate between them while the deferred passes
    // of the previous round run on the side stream
    SchurDesc<R> *ddesc = cw.take<SchurDesc<R>>(2);
    RotLog<R> *rlog[2];
    WinRec *wrec[2];
    cplx<R> *ubuf[2];
    for (int q = 0; q < 2; ++q) {
        rlog[q] = cw.take<RotLog<R>>(qr_log_capacity(n));
        wrec[q] = cw.take<WinRec>(qr_win_capacity(n));
        ubuf[q] = cw.take<cplx<R>>(qr_u_capacity(n));
    }
    int *qstate = cw.take<int>(kQrStateInts);
    int *rstate = cw.take<int>(4);
    int *qsync = cw.take<int>(32);
    int *qpost = cw.take<int>(qr_win_capacity(n));
    // cube root: V = S^2 beside S; X X in FP64 shares Rt's bytes (it is read
    // by the residual before Rt is next written)
    cplx<R> *V = root == 3 ? cw.take<cplx<R>>(nn) : nullptr;
    double *XX = (double *)Rt;
    // dependency flags of the one-launch Sylvester solve
    const int64_t flow_cap = (int64_t)rtrsyl_flow_ints((int)n, (int)n);
    int *flow = cw.take<int>((size_t)flow_cap);
    // tensor-core operands: Q^T; Q re-laid (for M Q); Q^H re-laid, real
    // part only (for Re(W Q^H)); the per-step re-laid Rhat and Y
    cplx<R> *Qt = use_tc ? cw.take<cplx<R>>(nn) : nullptr;
    float *QB = use_tc ? cw.take<float>(tcf) : nullptr;
    float *RB = use_tc ? cw.take<float>(tcf) : nullptr;
    float *YB = use_tc ? cw.take<float>(tcf) : nullptr;
    float *QhB = use_tc ? cw.take<float>(2 * nn) : nullptr;
    const int ld2 = 2 * (int)n;  // leading dimension of the re-laid operands (floats)
    double *gRacc = use_gsplit ? cw.take<double>(nn) : nullptr;  // split residual: FP64 tile sums,
    double *gXT = use_gsplit ? cw.take<double>(nn) : nullptr;    // X^T, the two digit sets
    void *gDa = use_gsplit ? (void *)cw.take<uint16_t>(split_digit_elems((int)n)) : nullptr;
    void *gDb = use_gsplit ? (void *)cw.take<uint16_t>(split_digit_elems((int)n)) : nullptr;
    int *gRhoA = use_gsplit ? cw.take<int>(n) : nullptr;
    int *gRhoB = use_gsplit ? cw.take<int>(n) : nullptr;
    h->fact_n = -1;

    SQM_CU(cudaMemsetAsync(sc.e, 0, 16 * sizeof(int), s));
    SQM_CU(cudaEventRecord(h->ev[0], s));
    if (cin) {
        SQM_CU(launch_norm_scale_z(dA, n, lda, sc.partials, (int)std::min<int64_t>(n, 1024), sc.norm, sc.e, s));
        SQM_CU(launch_cast_scaled_z<R>(dA, n, lda, sc.e, T, n, s));
    } else {
        SQM_CU(launch_norm_scale(dA, n, lda, sc.partials, (int)std::min<int64_t>(n, 1024), sc.norm, sc.e, s, root));
        SQM_CU(launch_cast_scaled<R>(dA, n, lda, sc.e, T, n, s, root));
    }
    double norm_a = 0.0;
    int e = 0;
    if (int rc = read_scalars(h, sc, &norm_a, nullptr, &e, nullptr, nullptr)) return rc;
    if (info) { info->norm_a = norm_a; info->scale_exponent = e; info->kind_used = SQRTM_KIND_GENERAL; }
    if (!isfinite(norm_a)) return 5;
    if (norm_a == 0.0) return 2;  // the zero matrix has the eigenvalue 0

    SchurDesc<R> hd;
    hd.T = T; hd.Q = Q; hd.v = v; hd.beta = beta; hd.status = sc.st_schur; hd.n = (int)n; hd.ld = (int)n;
    hd.counters = sc.st_schur + 3;
    hd.state = qstate; hd.log_cap = (int)std::min<int64_t>(qr_log_capacity(n), INT32_MAX);
    // rounds of at most max(64, n/2) windows, so that several rounds overlap
    // their deferred passes with the chase
    hd.win_cap = (int)std::min<int64_t>(qr_win_capacity(n), std::max<int64_t>(64, n / 2));
    hd.u_cap = qr_u_capacity(n);
    hd.wait_ns = h->wait_ns;
    SchurDesc<R> hd2[2] = {hd, hd};
    for (int q = 0; q < 2; ++q) {
        hd2[q].log = rlog[q];
        hd2[q].win = wrec[q];
        hd2[q].ubuf = ubuf[q];
        hd2[q].rstate = rstate + 2 * q;
        hd2[q].sync = qsync;
        hd2[q].postlist = qpost;
    }
    memcpy(h->staging.p, hd2, sizeof(hd2));
    SQM_CU(cudaMemcpyAsync(ddesc, h->staging.p, sizeof(hd2), cudaMemcpyHostToDevice, s));
    SQM_CU(cudaStreamSynchronize(s));
    if (!cin && hess_cluster_size<R>((int)n) > 0) {
        // A is real: the cluster-resident real reduction (W and Rt are free
        // until the Schur form is done)
        SQM_CU(launch_hessenberg_cluster<R>(T, Q, (int)n, (int)n, (R *)W, (R *)Rt, s));
    } else if (!cin && hessenberg_real_scratch<R>((int)n) <= nn) {
        // A is real, beyond the cluster's sizes: the real per-column
        // reduction over the whole GPU and Q from the stored reflectors, one
        // captured graph (W holds H and the reflectors, Rt the real Q and the
        // scratch; both are free until the Schur form is done); the complex
        // T and Q are written outside the graph
        struct Ctx { const cplx<R> *T; R *H, *Y, *Qr, *scr; int n; } ctx{T, (R *)W, (R *)W + nn, (R *)Rt, (R *)Rt + nn, (int)n};
        auto enq = [](void *p, cudaStream_t st) -> cudaError_t {
            Ctx *c = (Ctx *)p;
            return enqueue_hessenberg_real<R>(c->T, c->H, c->Y, c->Qr, c->scr, c->n, st);
        };
        if (run_graph(h, 120 + (int)sizeof(R), W, n, 1, enq, &ctx)) return 7;
        SQM_CU(launch_hessenberg_real_finish<R>((R *)W, (R *)Rt, T, Q, (int)n, s));
    } else {
        struct Ctx { SchurDesc<R> *d; int n; } ctx{ddesc, (int)n};
        auto enq = [](void *p, cudaStream_t st) -> cudaError_t {
            Ctx *c = (Ctx *)p;
            return launch_hessenberg<R>(c->d, 1, c->n, 64, st);
        };
        if (run_graph(h, 100 + (int)sizeof(R), ddesc, n, 1, enq, &ctx)) return 7;
    }
    cudaEvent_t ev_red;
    SQM_CU(cudaEventCreate(&ev_red));
    SQM_CU(cudaEventRecord(ev_red, s));
    float ms_chase = 0.0f;
    const sqrtm_tune_entry *tune = tune_for(h, n);
    SQM_CU(launch_qr_sweeps<R>(ddesc, 1, (int)n, (int *)h->staging.p + 512, qstate, s, &ms_chase, ddesc + 1, h->side,
                               h->qev, qsync, tune ? tune->qr_helpers : -1));
    SQM_CU(cudaEventRecord(h->ev[1], s));
    if (root == 3) SQM_CU(launch_tricbrt<R>(T, (int)n, S, (int)n, V, (int)n, (int)n, o.blks, sc.st_solve, s));
    else if (tune && tune->trisqrt_cutoff > 0 && n > tune->trisqrt_cutoff)
        SQM_CU(launch_trisqrt_rec<R>(T, (int)n, S, (int)n, (int)n, o.blks, tune->trisqrt_cutoff, sc.st_solve, s));
    else SQM_CU(launch_trisqrt<R>(T, (int)n, S, (int)n, (int)n, o.blks, sc.st_solve, s));
    // X_0 = Re(Q S Q^H), rounded to R, times 2^e
    const int ni = (int)n;
    if (use_tc) {
        // W <- (Q S)^T from Q^T's columns (the rows of Q); then
        // X_0 = 2^e Re(W Q^H) from W^T's columns, the FP32 accumulator
        // widened to FP64 (the rounding to FP32 of reading c10)
        TcEpilogue ep{};
        SQM_CU(launch_ctranspose(Q, Qt, ni, s));
        SQM_CU(launch_tc_relayout_cplx(Q, n, ni, ni, 1.0f, 1.0f, false, QB, ld2, s));
        SQM_CU(launch_tc_relayout_cplx(Qt, n, ni, ni, 1.0f, -1.0f, true, QhB, ld2, s));
        SQM_CU(launch_tc_relayout_cplx(S, n, ni, ni, 1.0f, 1.0f, false, YB, ld2, s));
        ep.C = (float *)W; ep.ldc = n;
        SQM_CU(launch_tc_cgemm(ni, ni, ni, Qt, ni, YB, ld2, TC_EPI_CSTORE_T, ep, sc.st_solve, s));
        ep = TcEpilogue{}; ep.X = dX; ep.ldx = ldx; ep.scale = ldexp(1.0, e);
        SQM_CU(launch_tc_cgemm(ni, ni, ni, W, ni, QhB, ld2, TC_EPI_RE_F64_STORE, ep, sc.st_solve, s));
    } else {
    SQM_CU(launch_cgemm<R>(OP_N, OP_N, (int)n, (int)n, (int)n, Q, (int)n, false, S, (int)n, EPI_STORE, W, (int)n, nullptr, 0, 0.0, s));
    SQM_CU(launch_cgemm<R>(OP_N, OP_H, (int)n, (int)n, (int)n, W, (int)n, false, Q, (int)n,
                           cin ? EPI_CPLX_TO_F64 : EPI_REAL_TO_F64, nullptr, 0, dX, ldx, ldexp(1.0, e), s));
    }
    SQM_CU(cudaEventRecord(h->ev[2], s));
    int st_schur = 0, st_solve = 0;
    if (int rc = read_scalars(h, sc, nullptr, nullptr, nullptr, &st_schur, &st_solve)) return rc;
    if (info) {
        float ms = 0;
        cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]); info->ms_schur = ms;
        cudaEventElapsedTime(&ms, h->ev[1], h->ev[2]); info->ms_trisqrt = ms;
        cudaEventElapsedTime(&ms, h->ev[0], ev_red); info->ms_reduction = ms;
        int cnt[7];  // [5..6]: the small blocks solved by qr_tiny_kernel
        SQM_CU(cudaMemcpy(cnt, sc.st_schur + 3, sizeof(cnt), cudaMemcpyDeviceToHost));
        info->schur_sweeps = cnt[0] + cnt[5];
        info->schur_rotations = (int64_t)cnt[1] + ((int64_t)cnt[2] << 31) + cnt[6];
        info->schur_work = (int64_t)cnt[3] + ((int64_t)cnt[4] << 31);  // the chase kernel's own
        info->ms_qr_chase = ms_chase;
    }
    cudaEventDestroy(ev_red);
    if (st_schur == 7) note_error(h, "malformed QR rotation log entry", __LINE__, 7);
    if (st_schur) return st_schur;
    if (st_solve) return st_solve;
    if (!refine) return 0;

    const double norm_as = ldexp(norm_a, -root * e);
    const bool fixed = o.steps >= 0;
    const int max_corr = fixed ? o.steps : o.maxit + 1;
    int status = 0, applied = 0, grew = 0;
    double prev = INFINITY;
    for (int k = 0;; ++k) {
        bool need_res = !fixed || k < max_corr;
        if (k >= max_corr && fixed) break;
        if (need_res) {
            int np = 0;
            if (root == 3) {
                SQM_CU(launch_rgemm<double>(0, 0, (int)n, (int)n, (int)n, dX, (int)ldx, dX, (int)ldx, RG_STORE, XX,
                                            (int)n, nullptr, nullptr, 0, 0.0, s));
                SQM_CU(launch_residual_f64_ab(dA, lda, dX, ldx, XX, n, (int)n, 3 * e, Rhat, (int)n, sc.partials,
                                              &np, s));
            } else if (cin) {
                SQM_CU(launch_zresidual_f64(dA, lda, dX, ldx, (int)n, e, (cplx<float> *)Rhat, (int)n, sc.partials, &np,
                                            s));
            } else if (use_gsplit) {
                SQM_CU(launch_residual_gen_split(dA, lda, dX, ldx, (int)n, e, Rhat, (int)n, gRacc, gXT, gDa, gDb, gRhoA,
                                                 gRhoB, sc.partials, &np, sc.st_solve, s));
            } else {
                SQM_CU(launch_residual_f64(dA, lda, dX, ldx, (int)n, e, Rhat, (int)n, sc.partials, &np, s));
            }
            SQM_CU(launch_sum_partials(sc.partials, np, sc.rnorm, s));
            double rn = 0.0;
            if (!fixed) {
                if (int rc = read_scalars(h, sc, nullptr, &rn, nullptr, nullptr, nullptr)) return rc;
                double rel = rn / norm_as;
                if (info && info->history_len < SQRTM_MAX_HISTORY) info->history[info->history_len++] = rel;
                if (!isfinite(rel)) { status = 4; break; }
                if (rel <= tol) { status = 0; break; }
                if (k >= max_corr) { status = 1; break; }
                grew = (rn > prev) ? grew + 1 : 0;
                if (grew >= 2) { status = 4; break; }
                prev = rn;
            }
        }
        if (use_tc) {
            // (Q^H Rhat)^T into W from Q's columns (conjugated rows of Q^H);
            // R~ = (Q^H Rhat) Q; S Y + Y S = R~; W <- (Q Y)^T;
            // X += 2^e Re(W Q^H) in the FP64 epilogue
            TcEpilogue ep{};
            SQM_CU(launch_tc_relayout_real(Rhat, n, ni, ni, -1.0f, RB, ld2, s));
            ep.C = (float *)W; ep.ldc = n;
            SQM_CU(launch_tc_cgemm(ni, ni, ni, Q, ni, RB, ld2, TC_EPI_CSTORE_T, ep, sc.st_solve, s));
            ep.C = (float *)Rt;
            SQM_CU(launch_tc_cgemm(ni, ni, ni, W, ni, QB, ld2, TC_EPI_CSTORE, ep, sc.st_solve, s));
            SQM_CU(launch_rtrsyl<R>(S, ni, ni, S, ni, ni, Rt, ni, o.blks, sc.st_solve, s, flow, flow_cap));
            SQM_CU(launch_tc_relayout_cplx(Rt, n, ni, ni, 1.0f, 1.0f, false, YB, ld2, s));
            ep.C = (float *)W;
            SQM_CU(launch_tc_cgemm(ni, ni, ni, Qt, ni, YB, ld2, TC_EPI_CSTORE_T, ep, sc.st_solve, s));
            ep = TcEpilogue{}; ep.X = dX; ep.ldx = ldx; ep.scale = ldexp(1.0, e);
            SQM_CU(launch_tc_cgemm(ni, ni, ni, W, ni, QhB, ld2, TC_EPI_RE_F64_ADD, ep, sc.st_solve, s));
            ++applied;
            continue;
        }
        // R~ = Q^H Rhat Q; Y solves S Y + Y S = R~; X += 2^e Re(Q Y Q^H)
        SQM_CU(launch_cgemm<R>(OP_N, OP_N, (int)n, (int)n, (int)n, Rhat, (int)n, !cin, Q, (int)n, EPI_STORE, W, (int)n, nullptr, 0, 0.0, s));
        SQM_CU(launch_cgemm<R>(OP_H, OP_N, (int)n, (int)n, (int)n, Q, (int)n, false, W, (int)n, EPI_STORE, Rt, (int)n, nullptr, 0, 0.0, s));
        if (root == 3)  // W is free between the transforms: it holds Z = Y S
            SQM_CU(launch_rtrsyl3<R>(S, (int)n, V, (int)n, Rt, (int)n, W, (int)n, (int)n, o.blks, sc.st_solve, s));
        else
            SQM_CU(launch_rtrsyl<R>(S, (int)n, (int)n, S, (int)n, (int)n, Rt, (int)n, o.blks, sc.st_solve, s, flow,
                                    flow_cap));
        SQM_CU(launch_cgemm<R>(OP_N, OP_N, (int)n, (int)n, (int)n, Q, (int)n, false, Rt, (int)n, EPI_STORE, W, (int)n, nullptr, 0, 0.0, s));
        SQM_CU(launch_cgemm<R>(OP_N, OP_H, (int)n, (int)n, (int)n, W, (int)n, false, Q, (int)n,
                               cin ? EPI_CPLX_ADD_F64 : EPI_REAL_ADD_F64, nullptr, 0, dX, ldx, ldexp(1.0, e), s));
        ++applied;
    }
    SQM_CU(cudaEventRecord(h->ev[3], s));
    if (int rc = read_scalars(h, sc, nullptr, nullptr, nullptr, nullptr, &st_solve)) return rc;
    if (!st_solve && (status == 0 || status == 1) && root == 2 && !cin) {
        // keep the factors and X for sqrtm_backward
        SQM_CU(cudaMemcpy2DAsync(Xsave, n * sizeof(double), dX, ldx * sizeof(double), n * sizeof(double), n,
                                 cudaMemcpyDeviceToDevice, s));
        h->fact_n = n; h->fact_kind = SQRTM_KIND_GENERAL; h->fact_e = e; h->fact_norm = norm_a;
        h->fact_q = Q; h->fact_s = S; h->fact_x = Xsave;
    }
    if (info) {
        info->iterations = applied;
        float ms = 0;
        cudaEventElapsedTime(&ms, h->ev[2], h->ev[3]); info->ms_refine = ms;
    }
    if (st_solve) return st_solve;
    return status;
}

// ---------------------------------------------------------------------------
// the real variant of Algorithm 2 (Remark 2.1) in storage precision R: real
// Schur form, quasi-triangular square root and Sylvester solves, real
// transforms; refine = false gives the plain real Schur method
// ---------------------------------------------------------------------------
template <class R>
static int real_path(sqrtm_handle_t h, const double *dA, int64_t n, int64_t lda, double tol, double *dX,
                     int64_t ldx, const sqrtm_opts &o, sqrtm_info *info, bool refine)
{
    if (n > 2048) return -3;  // size limit of the single-CTA Schur stage: argument 3 (n) out of range
    cudaStream_t s = h->stream;
    const size_t nn = (size_t)n * (size_t)n;
    size_t wbytes = scalars_bytes(n) + 5 * Carve::round(nn * sizeof(R)) + Carve::round(nn * sizeof(float)) +
                    Carve::round((size_t)(2 * n + 64) * sizeof(int)) + 4096;
    if (ensure(h->ws, wbytes, h)) return 7;
    Carve cw(h->ws.p);
    Scalars sc = carve_scalars(cw, n);
    R *T = cw.take<R>(nn);
    R *Q = cw.take<R>(nn);
    R *S = cw.take<R>(nn);
    R *W = cw.take<R>(nn);
    R *Rt = cw.take<R>(nn);
    float *Rhat = cw.take<float>(nn);
    int *bscr = cw.take<int>(2 * n + 64);  // block starts of S (n + 1), of the second operand (n + 1), counts (2)
    h->fact_n = -1;
    SQM_CU(cudaMemsetAsync(sc.e, 0, 16 * sizeof(int), s));
    SQM_CU(cudaEventRecord(h->ev[0], s));
    SQM_CU(launch_norm_scale(dA, n, lda, sc.partials, (int)std::min<int64_t>(n, 1024), sc.norm, sc.e, s));
    SQM_CU(launch_cast_scaled_real<R>(dA, n, lda, sc.e, T, n, s));
    double norm_a = 0.0;
    int e = 0;
    if (int rc = read_scalars(h, sc, &norm_a, nullptr, &e, nullptr, nullptr)) return rc;
    if (info) { info->norm_a = norm_a; info->scale_exponent = e; info->kind_used = SQRTM_KIND_REAL; }
    if (!isfinite(norm_a)) return 5;
    if (norm_a == 0.0) return 2;
    SQM_CU(launch_real_schur<R>(T, Q, (int)n, sc.st_schur, sc.st_schur + 3, s));
    SQM_CU(cudaEventRecord(h->ev[1], s));
    SQM_CU(launch_qtrisqrt<R>(T, (int)n, S, (int)n, (int)n, bscr, bscr + 2 * n + 8, sc.st_solve, s));
    // X_0 = 2^e Q S Q^T, the product rounded to R
    SQM_CU(launch_rgemm<R>(0, 0, (int)n, (int)n, (int)n, Q, (int)n, S, (int)n, RG_STORE, W, (int)n, nullptr, nullptr, 0,
                           0.0, s));
    SQM_CU(cudaMemset2DAsync(dX, (size_t)ldx * sizeof(double), 0, (size_t)n * sizeof(double), (size_t)n, s));
    SQM_CU(launch_rgemm<R>(0, 1, (int)n, (int)n, (int)n, W, (int)n, Q, (int)n, RG_ADD_F64, nullptr, 0, nullptr, dX, ldx,
                           ldexp(1.0, e), s));
    SQM_CU(cudaEventRecord(h->ev[2], s));
    int st_schur = 0, st_solve = 0;
    if (int rc = read_scalars(h, sc, nullptr, nullptr, nullptr, &st_schur, &st_solve)) return rc;
    if (info) {
        float ms = 0;
        cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]); info->ms_schur = ms;
        cudaEventElapsedTime(&ms, h->ev[1], h->ev[2]); info->ms_trisqrt = ms;
        int cnt = 0;
        SQM_CU(cudaMemcpy(&cnt, sc.st_schur + 3, sizeof(int), cudaMemcpyDeviceToHost));
        info->schur_sweeps = cnt;
    }
    if (st_schur) return st_schur;
    if (st_solve) return st_solve;
    if (!refine) return 0;
    if (sizeof(R) != sizeof(float)) return 7;  // the corrections take the FP32 residual

    const double norm_as = ldexp(norm_a, -2 * e);
    const bool fixed = o.steps >= 0;
    const int max_corr = fixed ? o.steps : o.maxit + 1;
    int status = 0, applied = 0, grew = 0;
    double prev = INFINITY;
    for (int k = 0;; ++k) {
        if (k >= max_corr && fixed) break;
        int np = 0;
        SQM_CU(launch_residual_f64(dA, lda, dX, ldx, (int)n, e, Rhat, (int)n, sc.partials, &np, s));
        SQM_CU(launch_sum_partials(sc.partials, np, sc.rnorm, s));
        if (!fixed) {
            double rn = 0.0;
            if (int rc = read_scalars(h, sc, nullptr, &rn, nullptr, nullptr, nullptr)) return rc;
            const double rel = rn / norm_as;
            if (info && info->history_len < SQRTM_MAX_HISTORY) info->history[info->history_len++] = rel;
            if (!isfinite(rel)) { status = 4; break; }
            if (rel <= tol) { status = 0; break; }
            if (k >= max_corr) { status = 1; break; }
            grew = (rn > prev) ? grew + 1 : 0;
            if (grew >= 2) { status = 4; break; }
            prev = rn;
        }
        // R~ = Q^T Rhat Q; S Y + Y S = R~ (quasi-triangular); X += 2^e Q Y Q^T
        const float *Rh = Rhat;
        SQM_CU(launch_rgemm<R>(0, 0, (int)n, (int)n, (int)n, (const R *)Rh, (int)n, Q, (int)n, RG_STORE, W, (int)n,
                               nullptr, nullptr, 0, 0.0, s));
        SQM_CU(launch_rgemm<R>(1, 0, (int)n, (int)n, (int)n, Q, (int)n, W, (int)n, RG_STORE, Rt, (int)n, nullptr,
                               nullptr, 0, 0.0, s));
        SQM_CU(launch_qrtrsyl<R>(S, (int)n, (int)n, S, (int)n, (int)n, Rt, (int)n, bscr, bscr + n + 4,
                                 bscr + 2 * n + 8, sc.st_solve, s));
        SQM_CU(launch_rgemm<R>(0, 0, (int)n, (int)n, (int)n, Q, (int)n, Rt, (int)n, RG_STORE, W, (int)n, nullptr,
                               nullptr, 0, 0.0, s));
        SQM_CU(launch_rgemm<R>(0, 1, (int)n, (int)n, (int)n, W, (int)n, Q, (int)n, RG_ADD_F64, nullptr, 0, nullptr, dX,
                               ldx, ldexp(1.0, e), s));
        ++applied;
    }
    SQM_CU(cudaEventRecord(h->ev[3], s));
    if (int rc = read_scalars(h, sc, nullptr, nullptr, nullptr, nullptr, &st_solve)) return rc;
    if (info) {
        info->iterations = applied;
        float ms = 0;
        cudaEventElapsedTime(&ms, h->ev[2], h->ev[3]); info->ms_refine = ms;
    }
    if (st_solve) return st_solve;
    return status;
}

static int resolve_opts(const sqrtm_opts *opts, double tol, sqrtm_opts *o)
{
    sqrtm_default_opts(o);
    if (opts) *o = *opts;
    else o->tol = tol;
    if (o->blks < 0 || o->blks > 4096) return -8;
    if (o->precision < SQRTM_PREC_AUTO) return -8;
    if (o->maxit < 0 || o->maxit > SQRTM_MAX_HISTORY - 2) return -8;
    return 0;
}

extern "C" int sqrtm_mixed(sqrtm_handle_t h, const double *dA, int64_t n, int64_t lda,
                           double tol, double *dX, int64_t ldx, const sqrtm_opts *opts,
                           sqrtm_info *info)
{
    info_reset(info);
    if (!h) return -1;
    if (int rc = check_args(dA, n, lda, dX, ldx)) return rc;
    sqrtm_opts o;
    if (int rc = resolve_opts(opts, tol, &o)) return rc;
    if (n == 0) return 0;
    apply_tuning(h, n, &o);
    int kind = o.kind;
    if (kind == SQRTM_KIND_AUTO) {
        int rc = 0;
        if (ensure(h->ws, 4096, h)) return 7;
        bool sym = is_bitwise_symmetric(h, dA, n, lda, (int *)h->ws.p, &rc);
        if (rc) return rc;
        kind = sym ? SQRTM_KIND_SPD : SQRTM_KIND_GENERAL;
    }
    int rc;
    if (kind == SQRTM_KIND_SPD && spd_enabled()) rc = spd_path(h, dA, n, lda, o.tol, dX, ldx, o, info);
    else if (kind == SQRTM_KIND_REAL) rc = real_path<float>(h, dA, n, lda, o.tol, dX, ldx, o, info, true);
    else rc = general_path<float>(h, dA, n, lda, o.tol, dX, ldx, o, info, true);
    if (info) info->status = rc;
    return rc;
}

extern "C" int sqrtm_schur_fp64(sqrtm_handle_t h, const double *dA, int64_t n, int64_t lda,
                                double tol, double *dX, int64_t ldx, const sqrtm_opts *opts,
                                sqrtm_info *info)
{
    (void)tol;
    info_reset(info);
    if (!h) return -1;
    if (int rc = check_args(dA, n, lda, dX, ldx)) return rc;
    sqrtm_opts o;
    if (int rc = resolve_opts(opts, tol, &o)) return rc;
    if (n == 0) return 0;
    apply_tuning(h, n, &o);
    int kind = o.kind;
    if (kind == SQRTM_KIND_AUTO) {
        int rc = 0;
        if (ensure(h->ws, 4096, h)) return 7;
        bool sym = is_bitwise_symmetric(h, dA, n, lda, (int *)h->ws.p, &rc);
        if (rc) return rc;
        kind = sym ? SQRTM_KIND_SPD : SQRTM_KIND_GENERAL;
    }
    int rc;
    if (kind == SQRTM_KIND_SPD && spd_enabled()) rc = spd_schur_fp64(h, dA, n, lda, dX, ldx, o, info);
    else if (kind == SQRTM_KIND_REAL) rc = real_path<double>(h, dA, n, lda, 0.0, dX, ldx, o, info, false);
    else rc = general_path<double>(h, dA, n, lda, 0.0, dX, ldx, o, info, false);
    h->fact_n = -1;  // the FP64 method keeps no low-precision factors
    if (info) info->status = rc;
    return rc;
}

extern "C" int sqrtm_mixed_complex(sqrtm_handle_t h, const void *dA, int64_t n, int64_t lda, double tol, void *dX,
                                   int64_t ldx, const sqrtm_opts *opts, sqrtm_info *info)
{
    info_reset(info);
    if (!h) return -1;
    if (int rc = check_args(dA, n, lda, dX, ldx)) return rc;
    sqrtm_opts o;
    if (int rc = resolve_opts(opts, tol, &o)) return rc;
    if (n == 0) return 0;
    apply_tuning(h, n, &o);
    int rc = general_path<float>(h, (const double *)dA, n, lda, o.tol, (double *)dX, ldx, o, info, true, 2, true);
    if (info) info->status = rc;
    return rc;
}

extern "C" int sqrtm_schur_fp64_complex(sqrtm_handle_t h, const void *dA, int64_t n, int64_t lda, double tol,
                                        void *dX, int64_t ldx, const sqrtm_opts *opts, sqrtm_info *info)
{
    info_reset(info);
    if (!h) return -1;
    if (int rc = check_args(dA, n, lda, dX, ldx)) return rc;
    sqrtm_opts o;
    if (int rc = resolve_opts(opts, tol, &o)) return rc;
    if (n == 0) return 0;
    apply_tuning(h, n, &o);
    int rc = general_path<double>(h, (const double *)dA, n, lda, 0.0, (double *)dX, ldx, o, info, false, 2, true);
    h->fact_n = -1;
    if (info) info->status = rc;
    return rc;
}

extern "C" int sqrtm_cbrtm_mixed(sqrtm_handle_t h, const double *dA, int64_t n, int64_t lda, double tol,
                                 double *dX, int64_t ldx, const sqrtm_opts *opts, sqrtm_info *info)
{
    info_reset(info);
    if (!h) return -1;
    if (int rc = check_args(dA, n, lda, dX, ldx)) return rc;
    sqrtm_opts o;
    if (int rc = resolve_opts(opts, tol, &o)) return rc;
    if (n == 0) return 0;
    apply_tuning(h, n, &o);
    int rc = general_path<float>(h, dA, n, lda, o.tol, dX, ldx, o, info, true, 3);
    if (info) info->status = rc;
    return rc;
}

extern "C" int sqrtm_cbrtm_schur_fp64(sqrtm_handle_t h, const double *dA, int64_t n, int64_t lda, double tol,
                                      double *dX, int64_t ldx, const sqrtm_opts *opts, sqrtm_info *info)
{
    info_reset(info);
    if (!h) return -1;
    if (int rc = check_args(dA, n, lda, dX, ldx)) return rc;
    sqrtm_opts o;
    if (int rc = resolve_opts(opts, tol, &o)) return rc;
    if (n == 0) return 0;
    apply_tuning(h, n, &o);
    int rc = general_path<double>(h, dA, n, lda, 0.0, dX, ldx, o, info, false, 3);
    h->fact_n = -1;
    if (info) info->status = rc;
    return rc;
}

// ---------------------------------------------------------------------------
// bitwise symmetry test (selects Algorithm 3 under SQRTM_KIND_AUTO)
// ---------------------------------------------------------------------------
__global__ void symmetric_kernel(const double *__restrict__ A, int64_t n, int64_t lda, int *flag)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = t % n, j = t / n;
        if (i < j) {
            double a = A[i + j * lda], b = A[j + i * lda];
            if (__double_as_longlong(a) != __double_as_longlong(b)) atomicExch(flag, 0);
        }
    }
}

static bool is_bitwise_symmetric(sqrtm_handle_t h, const double *dA, int64_t n, int64_t lda,
                                 int *flag_dev, int *rc)
{
    *rc = 0;
    int one = 1;
    if (cudaMemcpyAsync(flag_dev, &one, sizeof(int), cudaMemcpyHostToDevice, h->stream) != cudaSuccess) { *rc = 7; return false; }
    int grid = (int)std::min<int64_t>(std::max<int64_t>(1, (n * n + 255) / 256), 152 * 8);
    symmetric_kernel<<<grid, 256, 0, h->stream>>>(dA, n, lda, flag_dev); count_launch();
    int flag = 0;
    if (cudaMemcpyAsync(&flag, flag_dev, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) { *rc = 7; return false; }
    return flag != 0;
}

// ---------------------------------------------------------------------------
// batched entry point: a host-side scheduler.  Matrices are sorted by size
// (largest first) and handed out dynamically to worker threads; each worker
// owns a handle on its own non-blocking stream, so the kernels of different
// matrices overlap on the GPU.  The caller's stream is fenced on entry (the
// workers wait for work already queued on it) and on exit (it waits for all
// workers).
// ---------------------------------------------------------------------------
static int ensure_workers(sqrtm_handle_t h, int count)
{
    while ((int)h->workers.size() < count) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return 7;
        sqrtm_handle_t w = nullptr;
        if (int rc = sqrtm_create(&w, (void *)st)) { cudaStreamDestroy(st); return rc; }
        w->tuning = h->tuning;
        w->wait_ns = h->wait_ns;
        h->workers.push_back(w);
        h->worker_streams.push_back(st);
    }
    return 0;
}

// Longest-processing-time partition of a batch over `parts` workers (GPUs):
// matrices by decreasing cost n^3 (ties: lower index first), each to the
// part with the smallest load so far (ties: lowest part index).
extern "C" int sqrtm_batched_phases(sqrtm_handle_t h, double *ms, int cap, int *count, int *general)
{
    if (!h) return -1;
    if (cap > 0 && !ms) return -2;
    for (int q = 0; q < cap && q < kBatchPhases; ++q) ms[q] = h->bphase_ms[q];
    if (count) *count = h->bphase_count;
    if (general) *general = h->bphase_general;
    return kBatchPhases;
}

extern "C" int sqrtm_batch_partition(int batch, const int64_t *n, int parts, int *owner, double *load)
{
    if (batch < 0) return -1;
    if (batch > 0 && !n) return -2;
    if (parts < 1) return -3;
    if (batch > 0 && !owner) return -4;
    std::vector<double> ld((size_t)parts, 0.0);
    std::vector<int> ord((size_t)batch);
    for (int i = 0; i < batch; ++i) {
        if (n[i] < 0) return -2;
        ord[i] = i;
    }
    auto cost = [&](int i) { return (double)n[i] * (double)n[i] * (double)n[i]; };
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return cost(a) > cost(b); });
    for (int i : ord) {
        int best = 0;
        for (int p = 1; p < parts; ++p)
            if (ld[p] < ld[best]) best = p;
        owner[i] = best;
        ld[best] += cost(i);
    }
    if (load)
        for (int p = 0; p < parts; ++p) load[p] = ld[p];
    return 0;
}

extern "C" int sqrtm_mixed_batched(sqrtm_handle_t h, int batch, const double *const *dA,
                                   const int64_t *n, const int64_t *lda, double tol,
                                   double *const *dX, const int64_t *ldx, const sqrtm_opts *opts,
                                   int *status)
{
    if (batch < 0) return -2;
    if (batch == 0) return 0;
    // an early exit leaves every matrix's status at the returned code, so
    // a caller reading status[] never takes an untouched output for success
    auto fail_all = [&](int rc) {
        if (status)
            for (int i = 0; i < batch; ++i) status[i] = rc;
        return rc;
    };
    if (!h) return fail_all(-1);
    if (!dA || !n || !lda || !dX || !ldx) return fail_all(-3);
    for (int i = 0; i < batch; ++i)
        if (int rc = check_args(dA[i], n[i], lda[i], dX[i], ldx[i])) return fail_all(rc);
    sqrtm_opts o;
    if (int rc = resolve_opts(opts, tol, &o)) return fail_all(rc);
    std::vector<int> st(batch, 0);
    // matrices up to the batched size limit go through the batched general
    // path (one set of launches for all of them); larger ones, and every
    // matrix when the SPD algorithm is forced, through per-matrix calls on
    // worker threads with their own handles and streams, largest first
    // which sizes take the batched path: SQRTM_BATCH_MAXN (a size limit) if
    // set, else the tuning table, else n <= 256
    const char *env = getenv("SQRTM_BATCH_MAXN");
    const int nbmax = env ? atoi(env) : 256;
    std::vector<int> small, large;
    int64_t nsmall = 0;
    for (int i = 0; i < batch; ++i) {
        if (n[i] == 0) continue;
        const sqrtm_tune_entry *t = env ? nullptr : tune_for(h, n[i]);
        const bool b = t ? t->batched == 1 : n[i] <= nbmax;
        // the batched path's spectral (Algorithm 3) stage takes n <= 256;
        // larger matrices of a forced SPD call go to per-matrix calls
        const bool ok = o.kind != SQRTM_KIND_SPD || n[i] <= 256;
        if (b && ok) { small.push_back(i); nsmall = std::max(nsmall, n[i]); }
        else large.push_back(i);
    }
    sqrtm_opts ob = o;  // the batched path's block size: that of its largest matrix
    apply_tuning(h, std::max<int64_t>(nsmall, 1), &ob);
    const int nw = std::min<int>((int)large.size(), 12);
    if (nw > 0) {
        if (int rc = ensure_workers(h, nw)) return fail_all(rc);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail_all(7);
    // fence: workers start after the work already on the caller's stream
    cudaEvent_t start;
    if (cudaEventCreateWithFlags(&start, cudaEventDisableTiming) != cudaSuccess) return fail_all(7);
    cudaEventRecord(start, h->stream);
    for (int w = 0; w < nw; ++w) cudaStreamWaitEvent(h->worker_streams[w], start, 0);
    std::stable_sort(large.begin(), large.end(), [&](int a, int b) { return n[a] > n[b]; });
    std::atomic<int> next{0};
    auto work = [&](int w) {
        cudaSetDevice(dev);
        for (;;) {
            int q = next.fetch_add(1);
            if (q >= (int)large.size()) break;
            int i = large[q];
            st[i] = sqrtm_mixed(h->workers[w], dA[i], n[i], lda[i], tol, dX[i], ldx[i], opts, nullptr);
        }
    };
    std::vector<std::thread> threads;
    for (int w = 0; w < nw; ++w) threads.emplace_back(work, w);
    int rc_small = batched_general(h, small.data(), (int)small.size(), dA, n, lda, dX, ldx, ob, st.data());
    for (auto &t : threads) t.join();
    // fence: the caller's stream waits for every worker
    for (int w = 0; w < nw; ++w) {
        cudaEventRecord(start, h->worker_streams[w]);
        cudaStreamWaitEvent(h->stream, start, 0);
    }
    cudaEventDestroy(start);
    if (rc_small)
        for (int i : small) st[i] = rc_small;
    int first = 0;
    for (int i = 0; i < batch; ++i) {
        if (status) status[i] = st[i];
        if (st[i] && !first) first = st[i];
    }
    for (int w = 0; w < nw && !h->last_error[0]; ++w)
        if (h->workers[w]->last_error[0]) {
            snprintf(h->last_error, sizeof(h->last_error), "worker %d: %s", w, h->workers[w]->last_error);
            h->workers[w]->last_error[0] = 0;
        }
    return first;
}
