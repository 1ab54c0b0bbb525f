// internal.h -- launchers shared between the translation units of the
// library.  Host-side declarations only; every launcher enqueues work on the
// given stream and returns a cudaError_t from the launch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"

namespace sqm {

// Process-wide count of kernel launches issued by this library (diagnostic;
// reported by sqrtm_kernel_launches).
void count_launch();

// Allow a kernel the device's full opt-in dynamic shared memory.  The
// attribute is process-wide per kernel, so every caller sets the same value
// (a per-call size would race between threads launching the same kernel with
// different sizes).
cudaError_t allow_max_smem(const void *kernel);

// One entry of a chase window's rotation table: G = [c s; -conj(s) c] with
// s = sx + i sy; act = 0 marks a step in which the bulge did not move.
template <class R>
struct alignas(16) RotLog {
    R c, sx, sy, act;
};

// One chase window of the QR iteration: its rotation table is log entries
// [start, start + W NB) (step q, bulge g at start + q NB + g; that rotation
// acts on indices kbase + q + 3 (NB - 1 - g) and the next one), nsteps steps
// are used, all rotations act on indices kmin .. kmin + rr - 1, the sweep's
// active block is [lo, hi], and the window's accumulated rotation product U
// (rr x rr) is stored at ubuf + uoff.  A small active block [lo, hi] recorded
// for qr_tiny_kernel has nsteps = -1, kmin = lo, rr = hi - lo + 1, pad = 1
// and nb shift estimates (sx, sy) at log entries start .. start + nb - 1.
struct WinRec {
    int start, kbase, nsteps, kmin, rr, lo, hi;
    int t0, nb;      // first step of the window within its sweep; bulges of the sweep
    int r0, rnext;   // first row of the window block; last column of the next window's block
    int pad;         // 1: a small block for qr_tiny_kernel
    long long uoff;
};

// One matrix of a (possibly batched) Schur stage.  All arrays are device
// memory, column-major with leading dimension ld.
template <class R>
struct SchurDesc {
    RotLog<R> *log;  // scratch: rotation log (log_cap entries)
    WinRec *win;     // scratch: window records (win_cap entries)
    cplx<R> *ubuf;   // scratch: accumulated window rotations (u_cap elements)
    long long u_cap;
    int *state;      // scratch: kQrStateInts ints of QR iteration state
    int *rstate;     // scratch: [0] windows in this descriptor's buffers after its last chase round
    int *sync;       // scratch (cooperative chase): [0] windows posted, [1] quit, [2] failed, [4 + h] windows done by helper h
    int *postlist;   // scratch (cooperative chase): window record index of each posted window (win_cap entries)
    int log_cap;
    int win_cap;
    cplx<R> *T;      // in: A_s, out: upper triangular T (n x n)
    cplx<R> *Q;      // out: unitary Schur vectors (n x n)
    cplx<R> *v;      // scratch: Householder vector (>= n entries)
    R *beta;         // scratch: reflector scalars [beta, |x|, phase.x, phase.y]
    int *status;     // out: 0 / 3 (iteration cap)
    int *counters;   // out (7 ints): [0] sweeps, [1..2] rotations, [3..4] the chase kernel's in-block
                     // rotation work (int64s split lo/hi); cooperative chase: [5] sweeps and [6]
                     // rotations of the small blocks qr_tiny_kernel solves
    int n;
    int ld;
    // limit of each bounded wait between the CTAs of the cooperative chase,
    // in ns; 0 = the built-in 2 s
    unsigned long long wait_ns = 0;
};

// ---- batched general path: one entry per matrix (device arrays) ----
// Every batched launch covers all matrices (grid y or z = matrix index);
// an entry whose *active is 0 returns at once, as do the tiles beyond its n.
// All matrices are n x n with leading dimension n unless stated.
template <class R>
struct TriJob {
    const cplx<R> *T;   // triangular square root: T in, S out
    cplx<R> *S;
    cplx<R> *C;         // Sylvester solve S Y + Y S = C: C in, Y out
    int *status;        // receives 2 (see launch_trisqrt)
    const int *active;
    int n;
};
template <class R>
struct GemmJob {
    const void *A;      // R (a_real) or cplx<R>
    const cplx<R> *B;
    cplx<R> *C;         // EPI_STORE output
    double *X;          // FP64 epilogues: X (ldx), scaled by 2^(*e)
    int64_t ldx;
    const int *e;
    const int *active;
    int n;
};
struct ResJob {
    const double *A;    // R = (A - X X) 4^-e into Rhat (FP32, ld n) and the
    int64_t lda;        // per-tile partial sums of |R|^2 into partials
    const double *X;    // (tile (i, j) at i + j cdiv(n, 64))
    int64_t ldx;
    float *Rhat;
    double *partials;
    const int *e;
    const int *active;
    int n;
};
template <class R>
cudaError_t launch_trisqrt_batched(const TriJob<R> *jobs, int batch, int nmax, int blks, cudaStream_t s);
template <class R>
cudaError_t launch_rtrsyl_batched(const TriJob<R> *jobs, int batch, int nmax, int blks, cudaStream_t s);
// op pairs: (N, N), (N, H), (H, N); a_real only with (N, N)
template <class R>
cudaError_t launch_cgemm_batched(int opA, int opB, bool a_real, int epi, const GemmJob<R> *jobs, int batch, int nmax,
                                 cudaStream_t s);
cudaError_t launch_residual_batched(const ResJob *jobs, int batch, int nmax, cudaStream_t s);

// ---- scaling / norms (scale.cu) ----
// Deterministic ||A||_F: partials[nblk] then finalize; writes norm and e, the
// scaling exponent for a root of order `root`: A_s = 2^(-root e) A has
// ||A_s||_F / sqrt(n) in [2^-root, 1), and A^(1/root) = 2^e A_s^(1/root).
cudaError_t launch_norm_scale(const double *A, int64_t n, int64_t lda, double *partials,
                              int nblk, double *d_norm, int *d_e, cudaStream_t s, int root = 2);
template <class R>
cudaError_t launch_cast_scaled(const double *A, int64_t n, int64_t lda, const int *d_e,
                               cplx<R> *As, int64_t ldas, cudaStream_t s, int root = 2);
// complex input A (interleaved FP64 pairs, lda in complex elements): the
// same norm, exponent (root 2) and scaled cast
cudaError_t launch_norm_scale_z(const double *A, int64_t n, int64_t lda, double *partials, int nblk, double *d_norm,
                                int *d_e, cudaStream_t s);
template <class R>
cudaError_t launch_cast_scaled_z(const double *A, int64_t n, int64_t lda, const int *d_e, cplx<R> *As, int64_t ldas,
                                 cudaStream_t s);
template <class R>
cudaError_t launch_cast_scaled_real(const double *A, int64_t n, int64_t lda, const int *d_e,
                                    R *As, int64_t ldas, cudaStream_t s);

// ---- Schur stage (schur.cu) ----
template <class R>
cudaError_t launch_hessenberg(const SchurDesc<R> *d_desc, int batch, int nmax,
                              int ctas_per_matrix, cudaStream_t s);
// Hessenberg reduction of a REAL matrix (T holds it with zero imaginary
// parts) and Q, both written as complex n x n (ld) matrices, in one launch
// of a thread-block cluster.  V: n x n scratch of R (ld n), betas: n of R.
// hess_cluster_size returns the cluster size used for n, 0 if n is too large
// for it (then launch_hessenberg_cluster returns cudaErrorNotSupported).
template <class R>
int hess_cluster_size(int n);
template <class R>
cudaError_t launch_hessenberg_cluster(cplx<R> *T, cplx<R> *Q, int n, int ld, R *V, R *betas, cudaStream_t s);
// The register-resident cluster reduction for count matrices of sizes
// n_i <= nmax (nmax <= 512; FP64: <= 128), one cluster per matrix in one
// launch.  V: n_i x n_i of R scratch, betas: n_i of R, per job.
// cudaErrorNotSupported when nmax is too large for the kernel.
template <class R>
struct HessJob {
    cplx<R> *T;
    cplx<R> *Q;
    R *V;
    R *betas;
    int n;
};
template <class R>
cudaError_t launch_hessenberg_cluster_batched(const HessJob<R> *jobs, int count, int nmax, cudaStream_t s);
// d_state_all: the kQrStateInts-int state blocks of all matrices, contiguous
// (descs[b].state == d_state_all + kQrStateInts b); h_state: pinned host
// buffer of kQrStateInts * batch ints.  ms_chase (may be null) receives the
// summed duration of the chase kernel's launches (CUDA events on s).
// d_desc_alt (may be null): the same matrices with a second set of log,
// window and U buffers; then the chase rounds alternate between the two
// sets and each round's deferred passes run on `side` (ordered by the four
// events qev) while the next round's chase runs on s.  The deferred passes
// touch only T entries outside every later active block and Z, which the
// chase never reads.  d_sync (may be null; >= 32 ints, the descriptors'
// `sync`): with batch == 1 and a large enough n the chase runs as one
// cooperative grid of a chase CTA and helper CTAs that take the
// out-of-window updates of the active block.  helpers: number of helper
// CTAs (0: no cooperative grid; -1: 8, 16 from n = 1024).
constexpr int kQrStateInts = 16;
template <class R>
cudaError_t launch_qr_sweeps(const SchurDesc<R> *d_desc, int batch, int nmax, int *h_state,
                             const int *d_state_all, cudaStream_t s, float *ms_chase = nullptr,
                             const SchurDesc<R> *d_desc_alt = nullptr, cudaStream_t side = nullptr,
                             const cudaEvent_t *qev = nullptr, int *d_sync = nullptr, int helpers = -1);
// Real Householder Hessenberg reduction of a real matrix of any size
// (schur.cu): from the real parts of the complex A_s in T, H (real, ld n)
// becomes upper Hessenberg and Qr = P_0 ... P_{n-3} (real, ld n); Y
// receives the reflectors (n x n, ld n); scratch holds
// hessenberg_real_scratch<R>(n) elements.  Three launches per column plus
// the blocked back-transform, all capturable.  Then
// launch_hessenberg_real_finish writes T = H and Q = Qr as complex.
template <class R>
size_t hessenberg_real_scratch(int n);
template <class R>
cudaError_t enqueue_hessenberg_real(const cplx<R> *T, R *H, R *Y, R *Qr, R *scratch, int n, cudaStream_t s);
template <class R>
cudaError_t launch_hessenberg_real_finish(const R *H, const R *Qr, cplx<R> *T, cplx<R> *Q, int n, cudaStream_t s);

// Inside a stream capture on s: appends a conditional WHILE node whose
// condition is `init` at every launch of the graph and whose body is
// captured from body(ctx, body_stream, cond) (a kernel in the body sets the
// condition with cudaGraphSetConditional); pre(ctx, s, cond), if given, is
// captured on s just before the node (a kernel there may set the first
// value).  The capture on s continues after the node.
typedef cudaError_t (*CondFn)(void *ctx, cudaStream_t st, cudaGraphConditionalHandle cond);
cudaError_t capture_while(cudaStream_t s, cudaStream_t body_stream, unsigned init, CondFn body, void *ctx,
                          CondFn pre = nullptr);
// The QR rounds of a batch for capture into a graph: state initialisation,
// a WHILE node whose body is one round (chase with one CTA per matrix,
// window products, deferred passes, and a one-thread test of every
// matrix's done flag; at most 256 rounds, then status 3), and the final
// clean-up of T.  d_round: one device int of scratch.
template <class R>
cudaError_t enqueue_qr_sweeps_device(const SchurDesc<R> *d_desc, int batch, int nmax, int *d_round, cudaStream_t s,
                                     cudaStream_t body_stream);
// scratch sizes per matrix of size n: rotation log entries, window records,
// elements of accumulated window products (one round of the QR iteration
// stops at a sweep boundary before any of them would overflow)
inline int64_t qr_log_capacity(int64_t n) { return n <= 1 ? 64 : std::max<int64_t>(std::max<int64_t>(4 * n * n, 256 * n), 8192); }
inline int64_t qr_win_capacity(int64_t n) { return std::max<int64_t>(n * n / 2, 1024); }
inline int64_t qr_u_capacity(int64_t n) { return std::max<int64_t>(24 * n * n, 64 * 64 * 64); }

// ---- triangular solvers (trisolve.cu) ----
// S = T^{1/2}, blocked; status receives 2 on a zero denominator or an
// eigenvalue on the closed negative real axis.
template <class R>
cudaError_t launch_trisqrt(const cplx<R> *T, int ldt, cplx<R> *S, int lds, int n, int blks,
                           int *d_status, cudaStream_t s);
// The same by the recursive (Deadman-Higham-Ralha) splitting, with blocks of
// at most cutoff (>= 64) done by launch_trisqrt.
template <class R>
cudaError_t launch_trisqrt_rec(const cplx<R> *T, int ldt, cplx<R> *S, int lds, int n, int blks, int cutoff,
                               int *d_status, cudaStream_t s);
// Principal cube root (Sec. 4, p = 3) of upper triangular T: S = T^(1/3) and
// V = S^2 (both n x n, upper triangular); status 2 for an eigenvalue on or
// near the closed negative real axis or a zero leaf denominator.
template <class R>
cudaError_t launch_tricbrt(const cplx<R> *T, int ldt, cplx<R> *S, int lds, cplx<R> *V, int ldv, int n, int blks,
                           int *d_status, cudaStream_t s);
// S^2 Y + S Y S + Y S^2 = C (Eq. (3rd-order)) for upper triangular S with
// V = S^2: C (n x n) is overwritten by Y; Z (n x n) is scratch (Y S).
template <class R>
cudaError_t launch_rtrsyl3(const cplx<R> *S, int lds, const cplx<R> *V, int ldv, cplx<R> *C, int ldc, cplx<R> *Z,
                           int ldz, int n, int blks, int *d_status, cudaStream_t s);
// S Y + Y St = C (C overwritten by Y), blocked: one launch per block
// wavefront, or, given `flow` (device ints, flow_cap >= Mb Nb + 2 for
// Mb x Nb blocks), one launch ordered by block dependencies when the blocks
// are 32 rows and ldc is a multiple of 16 (else the wavefronts).
size_t rtrsyl_flow_ints(int m, int n);
template <class R>
cudaError_t launch_rtrsyl(const cplx<R> *S, int lds, int m, const cplx<R> *St, int ldst, int nn,
                          cplx<R> *C, int ldc, int blks, int *d_status, cudaStream_t s, int *flow = nullptr,
                          int64_t flow_cap = 0);

// ---- real quasi-triangular factors (quasi.cu; Remark 2.1) ----
// S = T^{1/2} for real quasi-upper-triangular T (n x n, ld): d_blk n + 1
// ints and d_nb 1 int of device scratch; synchronizes s once (the number of
// diagonal blocks sets the launch count).  status 2: a real eigenvalue <= 0
// or a singular block equation.
template <class R>
cudaError_t launch_qtrisqrt(const R *T, int ldt, R *S, int lds, int n, int *d_blk, int *d_nb, int *d_status,
                            cudaStream_t s);
// Real Schur form A = Q T Q^T in one CTA (T: in A, out quasi-triangular;
// Q out; both n x n, ld n, n <= 2048): status 3 when an eigenvalue needs more
// than 60 double-shift sweeps; counters[0] receives the sweeps.
template <class R>
cudaError_t launch_real_schur(R *T, R *Q, int n, int *d_status, int *d_counters, cudaStream_t s);
// S Y + Y St = C (C overwritten by Y) for real quasi-upper-triangular S
// (m x m) and St (nn x nn): scratch d_bm m + 1, d_bn nn + 1, d_nbs 2 ints.
template <class R>
cudaError_t launch_qrtrsyl(const R *S, int lds, int m, const R *St, int ldst, int nn, R *C, int ldc, int *d_bm,
                           int *d_bn, int *d_nbs, int *d_status, cudaStream_t s);

// ---- dense products (gemm.cu) ----
enum OpT { OP_N = 0, OP_H = 1 };
enum Epi { EPI_STORE = 0, EPI_REAL_TO_F64 = 1, EPI_REAL_ADD_F64 = 2, EPI_REAL_ADD_F64_T = 3, EPI_CPLX_TO_F64 = 4,
           EPI_CPLX_ADD_F64 = 5 };
// C = op(A) op(B) (m x n, inner k).  A complex or (a_real) real R.
// EPI_STORE:        C (complex) = result
// EPI_REAL_TO_F64:  X[i,j] = double(R(Re(result))) * scale
// EPI_REAL_ADD_F64: X[i,j] += double(Re(result)) * scale
// EPI_REAL_ADD_F64_T: X[j,i] += double(Re(result)) * scale (transposed)
// EPI_CPLX_TO_F64:  X (complex, interleaved FP64 pairs, ldx in complex
//                   elements)[i,j] = widened R-rounded result * scale
// EPI_CPLX_ADD_F64: X[i,j] += widened result * scale (complex)
template <class R>
cudaError_t launch_cgemm(int opA, int opB, int m, int n, int k, const void *A, int lda,
                         bool a_real, const cplx<R> *B, int ldb, int epi, cplx<R> *C, int ldc,
                         double *X, int64_t ldx, double scale, cudaStream_t s);
// R = (A - X X) * 4^-e in FP64; Rhat = fl32(R); partial sums of squares per
// CTA into partials (count returned through *nparts).
cudaError_t launch_residual_f64(const double *A, int64_t lda, const double *X, int64_t ldx,
                                int n, int e, float *Rhat, int ldr, double *partials,
                                int *nparts, cudaStream_t s);
// the number of partial sums launch_residual_f64 writes for size n
int residual_f64_parts(int n);
// The same with a second factor: R = (A - X B) * 2^-shift (the cube root's
// residual A - X (X X) with B = X X and shift = 3 e).
cudaError_t launch_residual_f64_ab(const double *A, int64_t lda, const double *X, int64_t ldx,
                                   const double *B, int64_t ldb, int n, int shift, float *Rhat, int ldr,
                                   double *partials, int *nparts, cudaStream_t s);
// Complex residual R = (A - X X) 4^-e in FP64 (A, X interleaved FP64 pairs,
// lda / ldx in complex elements); Rhat = fl32(R) (complex, ld ldr) and
// per-CTA partial sums of |R|^2.
cudaError_t launch_zresidual_f64(const double *A, int64_t lda, const double *X, int64_t ldx, int n, int e,
                                 cplx<float> *Rhat, int ldr, double *partials, int *nparts, cudaStream_t s);
// Adjoint residual Res = G - (X^T Y + Y X^T) in FP64; Rhat = fl32(Res) and
// per-CTA partial sums of |Res|^2.
cudaError_t launch_adjoint_residual_f64(const double *G, int64_t ldg, const double *X, int64_t ldx,
                                        const double *Y, int64_t ldy, int n, float *Rhat, int ldr,
                                        double *partials, int *nparts, cudaStream_t s);
// norm = sqrt(sum(partials[0:np])) in a fixed order
cudaError_t launch_sum_partials(const double *partials, int np, double *d_out, cudaStream_t s);

}  // namespace sqm
