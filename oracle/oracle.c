/*
 * oracle.c -- plain, slow, single-threaded FP64 reference for the matrix
 * square root of Gao, Kressner and Shao, "A mixed precision algorithm for the
 * matrix square root" (arXiv 2607.12430).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  The GPU library never links
 * or calls it, and it shares no source, header, table or helper with the GPU
 * code.
 *
 * Every routine follows a definition stated in the paper, written out with
 * no blocking or reordering beyond what that definition states:
 *
 *   orc_hessenberg     complex Householder reduction A = Q H Q^H (first stage
 *                      of the Schur method, Sec. 1 / Sec. 2.1).
 *   orc_schur_qr       complex single-shift (Wilkinson) implicit QR sweeps on
 *                      the Hessenberg form, H = Z T Z^H with T upper
 *                      triangular (Schur decomposition, Sec. 1 / Sec. 2.1).
 *   orc_csqrt          principal complex square root of a scalar (the
 *                      diagonal step of Sec. 2.2.1, principal branch as in the
 *                      definition of Sec. 1).
 *   orc_trisqrt        point back-substitution for T^{1/2} (Sec. 2.2.1,
 *                      Eq. (subst)).
 *   orc_sqrtm_schur    the FP64 Schur method X = Q T^{1/2} Q^H (Sec. 1); for
 *                      real A the real part is returned.
 *   orc_jacobi_eig     cyclic two-sided Jacobi for symmetric A = V diag(l) V^T
 *                      (spectral decomposition of Algorithm 3, step 1).
 *   orc_bs_solve       point Bartels-Stewart substitution for S Y + Y St = C
 *                      with S, St upper triangular (base case of Algorithm 1).
 *   orc_rtrsyl         the block recursion of Algorithm 1 (Sec. 2.2.2).
 *
 * Storage: column-major, element (i,j) of an m-by-n array with leading
 * dimension ld at a[i + j*ld].  Complex values use C99 double complex.
 *
 * Threads: when compiled with OpenMP, the loops over independent columns
 * (or rows) of the Householder updates and of the plain products run in
 * parallel; each column's arithmetic is the same sequence of operations as
 * in the serial loop, so the results are bitwise the same for any thread
 * count.  The QR sweep (a chain of dependent rotations) and the triangular
 * recurrence run serially.  orc_threads sets / reports the thread count.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex zc;

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

static const double ORC_EPS = 1.1102230246251565e-16; /* 2^-53 */

/* Thread count of the parallel loops: nthreads > 0 sets it; returns the
 * count in use (1 without OpenMP). */
int orc_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Householder reduction to upper Hessenberg form.                          */
/* For column k the reflector P = I - 2 v v^H / (v^H v), v = x + phase(x0)  */
/* ||x|| e1, maps x = H(k+1:n, k) to a multiple of e1.  P is Hermitian and  */
/* unitary, so H <- P H P and Q <- Q P keep A = Q H Q^H at every step.      */
/* H (in/out, n x n, ld = ldh) starts as A; Q (out, n x n, ld = ldq).       */
/* ------------------------------------------------------------------------ */
void orc_hessenberg(int n, zc *H, int ldh, zc *Q, int ldq)
{
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) Q[IDX(i, j, ldq)] = (i == j) ? 1.0 : 0.0;
    zc *v = (zc *)malloc(sizeof(zc) * (size_t)(n > 0 ? n : 1));
    for (int k = 0; k + 2 < n; ++k) {
        int m = n - k - 1; /* reflector acts on rows/cols k+1 .. n-1 */
        double xnorm2 = 0.0;
        for (int i = 0; i < m; ++i) {
            zc x = H[IDX(k + 1 + i, k, ldh)];
            xnorm2 += creal(x) * creal(x) + cimag(x) * cimag(x);
        }
        double tail2 = 0.0;
        for (int i = 1; i < m; ++i) {
            zc x = H[IDX(k + 1 + i, k, ldh)];
            tail2 += creal(x) * creal(x) + cimag(x) * cimag(x);
        }
        if (tail2 == 0.0) continue; /* column already a multiple of e1 */
        double xnorm = sqrt(xnorm2);
        zc x0 = H[IDX(k + 1, k, ldh)];
        double ax0 = cabs(x0);
        zc phase = (ax0 == 0.0) ? 1.0 : x0 / ax0;
        for (int i = 0; i < m; ++i) v[i] = H[IDX(k + 1 + i, k, ldh)];
        v[0] += phase * xnorm;
        double vnorm2 = 0.0;
        for (int i = 0; i < m; ++i) vnorm2 += creal(v[i]) * creal(v[i]) + cimag(v[i]) * cimag(v[i]);
        double beta = 2.0 / vnorm2;
        /* left: H(k+1:n, :) <- H - beta v (v^H H) */
#pragma omp parallel for schedule(static) if (n >= 128)
        for (int j = 0; j < n; ++j) {
            zc w = 0.0;
            for (int i = 0; i < m; ++i) w += conj(v[i]) * H[IDX(k + 1 + i, j, ldh)];
            w *= beta;
            for (int i = 0; i < m; ++i) H[IDX(k + 1 + i, j, ldh)] -= v[i] * w;
        }
        /* right: H(:, k+1:n) <- H - beta (H v) v^H */
#pragma omp parallel for schedule(static) if (n >= 128)
        for (int i = 0; i < n; ++i) {
            zc w = 0.0;
            for (int l = 0; l < m; ++l) w += H[IDX(i, k + 1 + l, ldh)] * v[l];
            w *= beta;
            for (int l = 0; l < m; ++l) H[IDX(i, k + 1 + l, ldh)] -= w * conj(v[l]);
        }
        /* accumulate: Q(:, k+1:n) <- Q - beta (Q v) v^H */
#pragma omp parallel for schedule(static) if (n >= 128)
        for (int i = 0; i < n; ++i) {
            zc w = 0.0;
            for (int l = 0; l < m; ++l) w += Q[IDX(i, k + 1 + l, ldq)] * v[l];
            w *= beta;
            for (int l = 0; l < m; ++l) Q[IDX(i, k + 1 + l, ldq)] -= w * conj(v[l]);
        }
        /* the annihilated entries are exactly zero by construction */
        H[IDX(k + 1, k, ldh)] = -phase * xnorm;
        for (int i = k + 2; i < n; ++i) H[IDX(i, k, ldh)] = 0.0;
    }
    free(v);
}

/* Complex Givens rotation G = [c s; -conj(s) c], c real, with
 * G [x; y] = [r; 0]. */
static void orc_givens(zc x, zc y, double *c, zc *s, zc *r)
{
    double ax = cabs(x), ay = cabs(y);
    if (ay == 0.0) { *c = 1.0; *s = 0.0; *r = x; return; }
    if (ax == 0.0) { *c = 0.0; *s = conj(y) / ay; *r = ay; return; }
    double nrm = hypot(ax, ay);
    zc ph = x / ax;
    *c = ax / nrm;
    *s = ph * conj(y) / nrm;
    *r = ph * nrm;
}

/* rows (p, p+1) <- G rows, columns [j0, j1) */
static void orc_rot_rows(zc *H, int ld, int p, int j0, int j1, double c, zc s)
{
    for (int j = j0; j < j1; ++j) {
        zc a = H[IDX(p, j, ld)], b = H[IDX(p + 1, j, ld)];
        H[IDX(p, j, ld)] = c * a + s * b;
        H[IDX(p + 1, j, ld)] = -conj(s) * a + c * b;
    }
}

/* columns (p, p+1) <- columns G^H, rows [i0, i1) */
static void orc_rot_cols(zc *H, int ld, int p, int i0, int i1, double c, zc s)
{
    for (int i = i0; i < i1; ++i) {
        zc a = H[IDX(i, p, ld)], b = H[IDX(i, p + 1, ld)];
        H[IDX(i, p, ld)] = c * a + conj(s) * b;
        H[IDX(i, p + 1, ld)] = -s * a + c * b;
    }
}

/* Eigenvalue of the 2x2 block [a b; c d] closer to d (Wilkinson shift). */
static zc orc_wilkinson(zc a, zc b, zc c, zc d)
{
    zc half = 0.5 * (a - d);
    zc disc = csqrt(half * half + b * c);
    zc m1 = d - b * c / (half + disc);
    zc m2 = d - b * c / (half - disc);
    /* m1, m2 are d + half -/+ disc written without cancellation; pick the
       finite one closer to d */
    int ok1 = isfinite(creal(m1)) && isfinite(cimag(m1));
    int ok2 = isfinite(creal(m2)) && isfinite(cimag(m2));
    if (ok1 && (!ok2 || cabs(m1 - d) <= cabs(m2 - d))) return m1;
    if (ok2) return m2;
    return d;
}

/* ------------------------------------------------------------------------ */
/* Complex Schur form by single-shift implicit QR sweeps on the Hessenberg  */
/* matrix H (in: Hessenberg, out: upper triangular T).  Z (in/out) is       */
/* right-multiplied by every rotation, so if A = Z H Z^H on entry then      */
/* A = Z T Z^H on exit.  A subdiagonal entry is set to zero when            */
/* |h(k,k-1)| <= eps (|h(k,k)| + |h(k-1,k-1)|).  Returns 0, or 3 when       */
/* an eigenvalue needs more than 60 sweeps.                                 */
/* ------------------------------------------------------------------------ */
int orc_schur_qr(int n, zc *H, int ldh, zc *Z, int ldz)
{
    int hi = n - 1;
    int iter = 0;
    while (hi > 0) {
        /* find the active block [lo, hi] */
        int lo = hi;
        while (lo > 0) {
            double sub = cabs(H[IDX(lo, lo - 1, ldh)]);
            double dsum = cabs(H[IDX(lo, lo, ldh)]) + cabs(H[IDX(lo - 1, lo - 1, ldh)]);
            if (sub <= ORC_EPS * dsum || sub == 0.0) {
                H[IDX(lo, lo - 1, ldh)] = 0.0;
                break;
            }
            --lo;
        }
        if (lo == hi) { /* 1x1 block deflated */
            --hi;
            iter = 0;
            continue;
        }
        if (++iter > 60) return 3;
        zc mu;
        if (iter % 10 == 0) {
            /* exceptional shift after a run of sweeps without deflation */
            mu = H[IDX(hi, hi, ldh)] + 0.75 * cabs(H[IDX(hi, hi - 1, ldh)]);
        } else {
            mu = orc_wilkinson(H[IDX(hi - 1, hi - 1, ldh)], H[IDX(hi - 1, hi, ldh)],
                               H[IDX(hi, hi - 1, ldh)], H[IDX(hi, hi, ldh)]);
        }
        /* first rotation from the shifted first column */
        double c; zc s, r;
        orc_givens(H[IDX(lo, lo, ldh)] - mu, H[IDX(lo + 1, lo, ldh)], &c, &s, &r);
        for (int k = lo; k < hi; ++k) {
            if (k > lo) {
                orc_givens(H[IDX(k, k - 1, ldh)], H[IDX(k + 1, k - 1, ldh)], &c, &s, &r);
            }
            int j0 = (k > lo) ? k - 1 : k;
            orc_rot_rows(H, ldh, k, j0, n, c, s);
            if (k > lo) H[IDX(k + 1, k - 1, ldh)] = 0.0; /* bulge annihilated */
            int i1 = (k + 2 < hi) ? k + 2 : hi;
            orc_rot_cols(H, ldh, k, 0, i1 + 1, c, s);
            orc_rot_cols(Z, ldz, k, 0, n, c, s);
        }
    }
    /* strictly lower part is zero in exact arithmetic; make it explicit */
    for (int j = 0; j < n; ++j)
        for (int i = j + 1; i < n; ++i) H[IDX(i, j, ldh)] = 0.0;
    return 0;
}

/* Principal square root of z (real part > 0 unless z is on the branch cut),
 * from sqrt(z) = t + i y/(2t), t = sqrt((|x| + |z|)/2) when x >= 0, and the
 * mirrored form |y|/(2t) + i sign(y) t when x < 0 (no cancellation). */
zc orc_csqrt(zc z)
{
    double x = creal(z), y = cimag(z);
    if (x == 0.0 && y == 0.0) return 0.0;
    double t = sqrt(0.5 * (fabs(x) + cabs(z)));
    if (x >= 0.0) return t + I * (y / (2.0 * t));
    return fabs(y) / (2.0 * t) + I * copysign(t, y);
}

/* ------------------------------------------------------------------------ */
/* S = T^{1/2} for upper triangular T (Sec. 2.2.1, Eq. (subst)):            */
/*   s_jj = sqrt(t_jj);                                                      */
/*   for j = 2..n, i = j-1 down to 1:                                        */
/*     s_ij = (t_ij - sum_{k=i+1}^{j-1} s_ik s_kj) / (s_ii + s_jj).          */
/* Returns 0, or 2 when some s_ii + s_jj is exactly zero.                    */
/* ------------------------------------------------------------------------ */
int orc_trisqrt(int n, const zc *T, int ldt, zc *S, int lds)
{
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) S[IDX(i, j, lds)] = 0.0;
    for (int j = 0; j < n; ++j) S[IDX(j, j, lds)] = orc_csqrt(T[IDX(j, j, ldt)]);
    for (int j = 1; j < n; ++j) {
        for (int i = j - 1; i >= 0; --i) {
            zc acc = T[IDX(i, j, ldt)];
            for (int k = i + 1; k < j; ++k) acc -= S[IDX(i, k, lds)] * S[IDX(k, j, lds)];
            zc den = S[IDX(i, i, lds)] + S[IDX(j, j, lds)];
            if (den == 0.0) return 2;
            S[IDX(i, j, lds)] = acc / den;
        }
    }
    return 0;
}

/* C = alpha * op(A) * op(B) + beta * C, all n x n complex; op = 'N', 'C'
 * (conjugate transpose).  Plain triple loop; C must not overlap A or B
 * (columns of C are formed independently). */
static void orc_zgemm(char ta, char tb, int n, zc alpha, const zc *A, int lda, const zc *B,
                      int ldb, zc beta, zc *C, int ldc)
{
#pragma omp parallel if (n >= 128)
    {
        zc *col = (zc *)malloc(sizeof(zc) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(static)
        for (int j = 0; j < n; ++j) {
            for (int i = 0; i < n; ++i) {
                zc acc = 0.0;
                for (int k = 0; k < n; ++k) {
                    zc a = (ta == 'N') ? A[IDX(i, k, lda)] : conj(A[IDX(k, i, lda)]);
                    zc b = (tb == 'N') ? B[IDX(k, j, ldb)] : conj(B[IDX(j, k, ldb)]);
                    acc += a * b;
                }
                col[i] = acc;
            }
            for (int i = 0; i < n; ++i)
                C[IDX(i, j, ldc)] = alpha * col[i] + (beta == 0.0 ? 0.0 : beta * C[IDX(i, j, ldc)]);
        }
        free(col);
    }
}

/* ------------------------------------------------------------------------ */
/* Complex Schur decomposition of a real matrix, A = Q T Q^H (Sec. 1):      */
/* Householder Hessenberg reduction followed by single-shift QR sweeps.    */
/* A real n x n (lda); Q, T complex n x n with ld = n.  Returns 0 or 3.     */
/* ------------------------------------------------------------------------ */
int orc_schur(int n, const double *A, int lda, zc *Q, zc *T)
{
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) T[IDX(i, j, n)] = A[IDX(i, j, lda)];
    orc_hessenberg(n, T, n, Q, n);
    return orc_schur_qr(n, T, n, Q, n);
}

/* ------------------------------------------------------------------------ */
/* The FP64 Schur method for the principal square root (Sec. 1):            */
/*   A = Q T Q^H, S = T^{1/2} by Eq. (subst), X = Q S Q^H.                  */
/* A: real n x n (lda), X: real part of the result (ldx).  Optional outputs  */
/* (may be NULL): Qout, Tout, Sout complex n x n with ld = n.                */
/* Returns 0, 2 (an eigenvalue on the closed negative real axis, or         */
/* s_ii + s_jj = 0) or 3 (QR iteration cap).                                 */
/* ------------------------------------------------------------------------ */
int orc_sqrtm_schur(int n, const double *A, int lda, double *X, int ldx, zc *Qout, zc *Tout,
                    zc *Sout)
{
    size_t nn = (size_t)n * (size_t)n;
    if (nn == 0) nn = 1;
    zc *T = (zc *)calloc(nn, sizeof(zc));
    zc *Q = (zc *)calloc(nn, sizeof(zc));
    zc *S = (zc *)calloc(nn, sizeof(zc));
    zc *W = (zc *)calloc(nn, sizeof(zc));
    zc *P = (zc *)calloc(nn, sizeof(zc));
    int st = orc_schur(n, A, lda, Q, T);
    if (st == 0) {
        for (int i = 0; i < n; ++i) {
            zc t = T[IDX(i, i, n)];
            if (creal(t) <= 0.0 && cimag(t) == 0.0) st = 2;
        }
    }
    if (st == 0) st = orc_trisqrt(n, T, n, S, n);
    if (st == 0) {
        orc_zgemm('N', 'N', n, 1.0, Q, n, S, n, 0.0, W, n);
        orc_zgemm('N', 'C', n, 1.0, W, n, Q, n, 0.0, P, n); /* P = Q S Q^H */
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) X[IDX(i, j, ldx)] = creal(P[IDX(i, j, n)]);
    }
    if (Qout) memcpy(Qout, Q, sizeof(zc) * (size_t)n * (size_t)n);
    if (Tout) memcpy(Tout, T, sizeof(zc) * (size_t)n * (size_t)n);
    if (Sout) memcpy(Sout, S, sizeof(zc) * (size_t)n * (size_t)n);
    free(T); free(Q); free(S); free(W); free(P);
    return st;
}

/* ------------------------------------------------------------------------ */
/* The same Schur method for a COMPLEX matrix (the method is stated for     */
/* A in C^{n x n}; Sec. 1): A = Q T Q^H by the complex Householder          */
/* Hessenberg reduction and single-shift QR, S = T^{1/2} by Eq. (subst),    */
/* X = Q S Q^H, all complex.  A complex n x n (lda); X complex (ldx);        */
/* Qout, Tout, Sout as above (may be NULL).  Returns 0, 2 or 3.             */
/* ------------------------------------------------------------------------ */
int orc_zsqrtm_schur(int n, const zc *A, int lda, zc *X, int ldx, zc *Qout, zc *Tout, zc *Sout)
{
    size_t nn = (size_t)n * (size_t)n;
    if (nn == 0) nn = 1;
    zc *T = (zc *)calloc(nn, sizeof(zc));
    zc *Q = (zc *)calloc(nn, sizeof(zc));
    zc *S = (zc *)calloc(nn, sizeof(zc));
    zc *W = (zc *)calloc(nn, sizeof(zc));
    zc *P = (zc *)calloc(nn, sizeof(zc));
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) T[IDX(i, j, n)] = A[IDX(i, j, lda)];
    orc_hessenberg(n, T, n, Q, n);
    int st = orc_schur_qr(n, T, n, Q, n);
    if (st == 0) {
        for (int i = 0; i < n; ++i) {
            zc t = T[IDX(i, i, n)];
            if (creal(t) <= 0.0 && cimag(t) == 0.0) st = 2;
        }
    }
    if (st == 0) st = orc_trisqrt(n, T, n, S, n);
    if (st == 0) {
        orc_zgemm('N', 'N', n, 1.0, Q, n, S, n, 0.0, W, n);
        orc_zgemm('N', 'C', n, 1.0, W, n, Q, n, 0.0, P, n); /* P = Q S Q^H */
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) X[IDX(i, j, ldx)] = P[IDX(i, j, n)];
    }
    if (Qout) memcpy(Qout, Q, sizeof(zc) * (size_t)n * (size_t)n);
    if (Tout) memcpy(Tout, T, sizeof(zc) * (size_t)n * (size_t)n);
    if (Sout) memcpy(Sout, S, sizeof(zc) * (size_t)n * (size_t)n);
    free(T); free(Q); free(S); free(W); free(P);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Cyclic two-sided Jacobi for real symmetric A = V diag(lam) V^T.          */
/* A (in, destroyed), V (out, orthogonal), lam (out, unsorted).             */
/* Each rotation zeroes a_pq with t = sign(tau)/(|tau| + sqrt(1 + tau^2)),  */
/* tau = (a_qq - a_pp) / (2 a_pq).  Stops when the off-diagonal Frobenius   */
/* norm is <= eps * ||A||_F.  Returns 0, or 3 after 100 sweeps.             */
/* ------------------------------------------------------------------------ */
int orc_jacobi_eig(int n, double *A, int lda, double *V, int ldv, double *lam)
{
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) V[IDX(i, j, ldv)] = (i == j) ? 1.0 : 0.0;
    double fro2 = 0.0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) fro2 += A[IDX(i, j, lda)] * A[IDX(i, j, lda)];
    int st = 3;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off2 = 0.0;
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i)
                if (i != j) off2 += A[IDX(i, j, lda)] * A[IDX(i, j, lda)];
        if (off2 <= ORC_EPS * ORC_EPS * fro2) { st = 0; break; }
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = A[IDX(p, q, lda)];
                if (apq == 0.0) continue;
                double tau = (A[IDX(q, q, lda)] - A[IDX(p, p, lda)]) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                /* A <- J^T A J with J = [c s; -s c] acting on (p, q) */
                for (int k = 0; k < n; ++k) {
                    double akp = A[IDX(k, p, lda)], akq = A[IDX(k, q, lda)];
                    A[IDX(k, p, lda)] = c * akp - s * akq;
                    A[IDX(k, q, lda)] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[IDX(p, k, lda)], aqk = A[IDX(q, k, lda)];
                    A[IDX(p, k, lda)] = c * apk - s * aqk;
                    A[IDX(q, k, lda)] = s * apk + c * aqk;
                }
                A[IDX(p, q, lda)] = 0.0;
                A[IDX(q, p, lda)] = 0.0;
                for (int k = 0; k < n; ++k) {
                    double vkp = V[IDX(k, p, ldv)], vkq = V[IDX(k, q, ldv)];
                    V[IDX(k, p, ldv)] = c * vkp - s * vkq;
                    V[IDX(k, q, ldv)] = s * vkp + c * vkq;
                }
            }
        }
    }
    for (int i = 0; i < n; ++i) lam[i] = A[IDX(i, i, lda)];
    return st;
}

/* ------------------------------------------------------------------------ */
/* Point Bartels-Stewart substitution for S Y + Y St = C, with S (m x m)    */
/* and St (n x n) upper triangular (base case of Algorithm 1):               */
/*   y_ij = (c_ij - sum_{k>i} s_ik y_kj - sum_{k<j} y_ik st_kj)              */
/*          / (s_ii + st_jj),                                                */
/* columns left to right, rows bottom to top.  C is overwritten by Y.       */
/* Returns 0, or 2 when a denominator is exactly zero.                      */
/* ------------------------------------------------------------------------ */
int orc_bs_solve(int m, int n, const zc *S, int lds, const zc *St, int ldst, zc *C, int ldc)
{
    for (int j = 0; j < n; ++j) {
        for (int i = m - 1; i >= 0; --i) {
            zc acc = C[IDX(i, j, ldc)];
            for (int k = i + 1; k < m; ++k) acc -= S[IDX(i, k, lds)] * C[IDX(k, j, ldc)];
            for (int k = 0; k < j; ++k) acc -= C[IDX(i, k, ldc)] * St[IDX(k, j, ldst)];
            zc den = S[IDX(i, i, lds)] + St[IDX(j, j, ldst)];
            if (den == 0.0) return 2;
            C[IDX(i, j, ldc)] = acc / den;
        }
    }
    return 0;
}

/* C(m x n) -= A(m x k) * B(k x n), plain loops */
static void orc_gemm_sub(int m, int n, int k, const zc *A, int lda, const zc *B, int ldb, zc *C,
                         int ldc)
{
#pragma omp parallel for schedule(static) if ((long)m * n * k >= 262144L)
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < m; ++i) {
            zc acc = 0.0;
            for (int l = 0; l < k; ++l) acc += A[IDX(i, l, lda)] * B[IDX(l, j, ldb)];
            C[IDX(i, j, ldc)] -= acc;
        }
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1, Y = rtrsyl(S, St, C, blks): recursive blocked solve of      */
/* S Y + Y St = C with S (m x m) and St (n x n) upper triangular.  The      */
/* right-hand side (written C in the algorithm's body, R in its header) is  */
/* overwritten with Y.  Split point: first block of size ceil(size/2).      */
/* Returns 0 or 2.                                                           */
/* ------------------------------------------------------------------------ */
int orc_rtrsyl(int m, int n, const zc *S, int lds, const zc *St, int ldst, zc *C, int ldc,
               int blks)
{
    if (m <= 0 || n <= 0) return 0;
    if (m <= blks && n <= blks) return orc_bs_solve(m, n, S, lds, St, ldst, C, ldc);
    int st;
    if (n <= m / 2) {
        /* split rows only: S = [S11 S12; 0 S22], C = [C1; C2] */
        int m1 = (m + 1) / 2, m2 = m - m1;
        const zc *S12 = S + IDX(0, m1, lds), *S22 = S + IDX(m1, m1, lds);
        zc *C1 = C, *C2 = C + IDX(m1, 0, ldc);
        if ((st = orc_rtrsyl(m2, n, S22, lds, St, ldst, C2, ldc, blks))) return st;
        orc_gemm_sub(m1, n, m2, S12, lds, C2, ldc, C1, ldc);
        return orc_rtrsyl(m1, n, S, lds, St, ldst, C1, ldc, blks);
    }
    if (m <= n / 2) {
        /* split columns only: St = [St11 St12; 0 St22], C = [C1 C2] */
        int n1 = (n + 1) / 2, n2 = n - n1;
        const zc *St12 = St + IDX(0, n1, ldst), *St22 = St + IDX(n1, n1, ldst);
        zc *C1 = C, *C2 = C + IDX(0, n1, ldc);
        if ((st = orc_rtrsyl(m, n1, S, lds, St, ldst, C1, ldc, blks))) return st;
        orc_gemm_sub(m, n2, n1, C1, ldc, St12, ldst, C2, ldc);
        return orc_rtrsyl(m, n2, S, lds, St22, ldst, C2, ldc, blks);
    }
    /* four-way split */
    int m1 = (m + 1) / 2, m2 = m - m1, n1 = (n + 1) / 2, n2 = n - n1;
    const zc *S12 = S + IDX(0, m1, lds), *S22 = S + IDX(m1, m1, lds);
    const zc *St12 = St + IDX(0, n1, ldst), *St22 = St + IDX(n1, n1, ldst);
    zc *C11 = C, *C21 = C + IDX(m1, 0, ldc), *C12 = C + IDX(0, n1, ldc),
       *C22 = C + IDX(m1, n1, ldc);
    if ((st = orc_rtrsyl(m2, n1, S22, lds, St, ldst, C21, ldc, blks))) return st;
    orc_gemm_sub(m1, n1, m2, S12, lds, C21, ldc, C11, ldc);
    orc_gemm_sub(m2, n2, n1, C21, ldc, St12, ldst, C22, ldc);
    if ((st = orc_rtrsyl(m1, n1, S, lds, St, ldst, C11, ldc, blks))) return st;
    if ((st = orc_rtrsyl(m2, n2, S22, lds, St22, ldst, C22, ldc, blks))) return st;
    orc_gemm_sub(m1, n2, m2, S12, lds, C22, ldc, C12, ldc);
    orc_gemm_sub(m1, n2, n1, C11, ldc, St12, ldst, C12, ldc);
    return orc_rtrsyl(m1, n2, S, lds, St22, ldst, C12, ldc, blks);
}

/* ---------------------------------------------------------------------------
 * Principal cube root (Sec. 4, p = 3).
 *
 * orc_ccbrt: z^(1/3) = |z|^(1/3) e^(i arg(z) / 3) with arg in (-pi, pi], the
 * root whose argument lies in (-pi/3, pi/3] (the sector of the principal
 * root).
 *
 * orc_tricbrt: S = T^(1/3) of upper triangular T (the Schur method for p-th
 * roots, Sec. 4), with V = S^2 kept alongside: from T = S V and V = S S,
 * for i < j (superdiagonal by superdiagonal)
 *   s_ij (s_ii^2 + s_ii s_jj + s_jj^2)
 *       = t_ij - s_ii sum_{i<k<j} s_ik s_kj - sum_{i<k<j} s_ik v_kj,
 *   v_ij = s_ij (s_ii + s_jj) + sum_{i<k<j} s_ik s_kj.
 *
 * orc_rtrsyl3: S^2 Y + S Y St + Y St^2 = C (Eq. (3rd-order)), S (m x m) and
 * St (n x n) upper triangular with V = S^2, Vt = St^2 given, point by point
 * in the order of Bartels-Stewart (column j left to right, row i bottom to
 * top), with W = Y St kept alongside:
 *   y_ij (v_ii + s_ii st_jj + vt_jj) = c_ij - sum_{k>i} v_ik y_kj
 *       - sum_{l<j} y_il vt_lj - s_ii w'_ij - sum_{k>i} s_ik w_kj,
 *   w'_ij = sum_{l<j} y_il st_lj,  w_ij = w'_ij + y_ij st_jj.
 * ------------------------------------------------------------------------- */
zc orc_ccbrt(zc z)
{
    double r = cabs(z);
    if (r == 0.0) return 0.0;
    double th = carg(z) / 3.0;
    double m = cbrt(r);
    return m * cos(th) + I * (m * sin(th));
}

int orc_tricbrt(int n, const zc *T, int ldt, zc *S, int lds, zc *V, int ldv)
{
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) { S[IDX(i, j, lds)] = 0.0; V[IDX(i, j, ldv)] = 0.0; }
    for (int j = 0; j < n; ++j) {
        zc s = orc_ccbrt(T[IDX(j, j, ldt)]);
        S[IDX(j, j, lds)] = s;
        V[IDX(j, j, ldv)] = s * s;
    }
    for (int d = 1; d < n; ++d) {
        for (int i = 0; i + d < n; ++i) {
            int j = i + d;
            zc sv = 0.0, st = 0.0;
            for (int k = i + 1; k < j; ++k) {
                sv += S[IDX(i, k, lds)] * S[IDX(k, j, lds)];
                st += S[IDX(i, k, lds)] * V[IDX(k, j, ldv)];
            }
            zc si = S[IDX(i, i, lds)], sj = S[IDX(j, j, lds)];
            zc den = si * si + si * sj + sj * sj;
            if (den == 0.0) return 2;
            zc sij = (T[IDX(i, j, ldt)] - si * sv - st) / den;
            S[IDX(i, j, lds)] = sij;
            V[IDX(i, j, ldv)] = sij * (si + sj) + sv;
        }
    }
    return 0;
}

int orc_rtrsyl3(int m, int n, const zc *S, int lds, const zc *V, int ldv, const zc *St, int ldst,
                const zc *Vt, int ldvt, zc *C, int ldc)
{
    zc *W = (zc *)calloc((size_t)(m > 0 ? m : 1) * (size_t)(n > 0 ? n : 1), sizeof(zc));
    if (!W) return 7;
    for (int j = 0; j < n; ++j) {
        for (int i = m - 1; i >= 0; --i) {
            zc acc = C[IDX(i, j, ldc)];
            zc wp = 0.0;
            for (int l = 0; l < j; ++l) wp += C[IDX(i, l, ldc)] * St[IDX(l, j, ldst)];
            for (int k = i + 1; k < m; ++k)
                acc -= V[IDX(i, k, ldv)] * C[IDX(k, j, ldc)] + S[IDX(i, k, lds)] * W[IDX(k, j, m)];
            for (int l = 0; l < j; ++l) acc -= C[IDX(i, l, ldc)] * Vt[IDX(l, j, ldvt)];
            acc -= S[IDX(i, i, lds)] * wp;
            zc den = V[IDX(i, i, ldv)] + S[IDX(i, i, lds)] * St[IDX(j, j, ldst)] + Vt[IDX(j, j, ldvt)];
            if (den == 0.0) { free(W); return 2; }
            zc y = acc / den;
            C[IDX(i, j, ldc)] = y;
            W[IDX(i, j, m)] = wp + y * St[IDX(j, j, ldst)];
        }
    }
    free(W);
    return 0;
}

/* X = Q T^(1/3) Q^H (real part), the FP64 Schur method for the cube root */
int orc_cbrtm_schur(int n, const double *A, int lda, double *X, int ldx, zc *Qout, zc *Tout, zc *Sout,
                    zc *Vout)
{
    size_t nn = (size_t)n * (size_t)n;
    if (nn == 0) nn = 1;
    zc *T = (zc *)calloc(nn, sizeof(zc));
    zc *Q = (zc *)calloc(nn, sizeof(zc));
    zc *S = (zc *)calloc(nn, sizeof(zc));
    zc *V = (zc *)calloc(nn, sizeof(zc));
    zc *W = (zc *)calloc(nn, sizeof(zc));
    zc *P = (zc *)calloc(nn, sizeof(zc));
    int st = orc_schur(n, A, lda, Q, T);
    if (st == 0) {
        for (int i = 0; i < n; ++i) {
            zc t = T[IDX(i, i, n)];
            if (creal(t) <= 0.0 && cimag(t) == 0.0) st = 2;
        }
    }
    if (st == 0) st = orc_tricbrt(n, T, n, S, n, V, n);
    if (st == 0) {
        orc_zgemm('N', 'N', n, 1.0, Q, n, S, n, 0.0, W, n);
        orc_zgemm('N', 'C', n, 1.0, W, n, Q, n, 0.0, P, n); /* P = Q S Q^H */
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) X[IDX(i, j, ldx)] = creal(P[IDX(i, j, n)]);
    }
    if (Qout) memcpy(Qout, Q, sizeof(zc) * (size_t)n * (size_t)n);
    if (Tout) memcpy(Tout, T, sizeof(zc) * (size_t)n * (size_t)n);
    if (Sout) memcpy(Sout, S, sizeof(zc) * (size_t)n * (size_t)n);
    if (Vout) memcpy(Vout, V, sizeof(zc) * (size_t)n * (size_t)n);
    free(T); free(Q); free(S); free(V); free(W); free(P);
    return st;
}

/* ======================================================================== */
/* Real arithmetic for real A (Remark 2.1): A = Q T Q^T with Q orthogonal    */
/* and T quasi-upper-triangular (1x1 blocks for real eigenvalues, 2x2       */
/* blocks for complex conjugate pairs); the square root and the Sylvester   */
/* solves in the same block structure, never cutting a 2x2 block.           */
/* ======================================================================== */

/* Householder reflector of a real 3-vector (or 2-vector, z unused when     */
/* len == 2): P = I - beta v v^T with v(0) = 1 and P x = (r, 0, 0).         */
static void orc_house3(int len, double x, double y, double z, double v[3], double *beta)
{
    double sig = y * y + (len == 3 ? z * z : 0.0);
    v[0] = 1.0; v[1] = y; v[2] = len == 3 ? z : 0.0;
    if (sig == 0.0) { *beta = 0.0; return; }
    double mu = sqrt(x * x + sig);
    double v0 = x <= 0.0 ? x - mu : -sig / (x + mu);
    *beta = 2.0 * v0 * v0 / (sig + v0 * v0);
    v[1] = y / v0;
    v[2] = len == 3 ? z / v0 : 0.0;
}

/* rows r0 .. r0+len-1 of M, columns c0 .. c1-1: M <- P M */
static void orc_house_rows(double *M, int ld, int r0, int len, int c0, int c1, const double v[3], double beta)
{
    if (beta == 0.0) return;
    for (int j = c0; j < c1; ++j) {
        double s = 0.0;
        for (int l = 0; l < len; ++l) s += v[l] * M[IDX(r0 + l, j, ld)];
        s *= beta;
        for (int l = 0; l < len; ++l) M[IDX(r0 + l, j, ld)] -= s * v[l];
    }
}

/* columns c0 .. c0+len-1 of M, rows r0 .. r1-1: M <- M P */
static void orc_house_cols(double *M, int ld, int c0, int len, int r0, int r1, const double v[3], double beta)
{
    if (beta == 0.0) return;
    for (int i = r0; i < r1; ++i) {
        double s = 0.0;
        for (int l = 0; l < len; ++l) s += M[IDX(i, c0 + l, ld)] * v[l];
        s *= beta;
        for (int l = 0; l < len; ++l) M[IDX(i, c0 + l, ld)] -= s * v[l];
    }
}

/* A 2x2 block at (k, k) with real eigenvalues is split by a rotation that  */
/* maps an eigenvector onto e_1 (applied to T and Q); one with complex      */
/* eigenvalues is left as it is.                                             */
static void orc_split_2x2(int n, double *H, int ldh, double *Z, int ldz, int k)
{
    double a = H[IDX(k, k, ldh)], b = H[IDX(k, k + 1, ldh)];
    double c = H[IDX(k + 1, k, ldh)], d = H[IDX(k + 1, k + 1, ldh)];
    if (c == 0.0) return;
    double p = 0.5 * (a - d), disc = p * p + b * c;
    if (disc < 0.0) return; /* complex pair: a genuine 2x2 block */
    double lam = 0.5 * (a + d) + (p >= 0.0 ? sqrt(disc) : -sqrt(disc));
    /* eigenvector for lam: (lam - d, c) (c != 0) */
    double e0 = lam - d, e1 = c, nr = hypot(e0, e1);
    double cs = e0 / nr, sn = e1 / nr;
    /* G = [cs -sn; sn cs], first column the eigenvector: H <- G^T H G */
    for (int j = k; j < n; ++j) {
        double x = H[IDX(k, j, ldh)], y = H[IDX(k + 1, j, ldh)];
        H[IDX(k, j, ldh)] = cs * x + sn * y;
        H[IDX(k + 1, j, ldh)] = -sn * x + cs * y;
    }
    for (int i = 0; i <= k + 1; ++i) {
        double x = H[IDX(i, k, ldh)], y = H[IDX(i, k + 1, ldh)];
        H[IDX(i, k, ldh)] = cs * x + sn * y;
        H[IDX(i, k + 1, ldh)] = -sn * x + cs * y;
    }
    for (int i = 0; i < n; ++i) {
        double x = Z[IDX(i, k, ldz)], y = Z[IDX(i, k + 1, ldz)];
        Z[IDX(i, k, ldz)] = cs * x + sn * y;
        Z[IDX(i, k + 1, ldz)] = -sn * x + cs * y;
    }
    H[IDX(k + 1, k, ldh)] = 0.0;
}

/* ------------------------------------------------------------------------ */
/* Real Schur form of a real upper Hessenberg H by implicit double-shift    */
/* (Francis) QR sweeps: each sweep uses the two eigenvalues of the trailing */
/* 2x2 block as a conjugate (or real) shift pair, starts from the first     */
/* column of (H - s1 I)(H - s2 I) and restores the Hessenberg form with     */
/* 3x3 Householder reflectors.  Deflation as in orc_schur_qr.  Z (in/out)   */
/* is right-multiplied by every reflector.  Returns 0 or 3.                 */
/* ------------------------------------------------------------------------ */
int orc_real_schur_qr(int n, double *H, int ldh, double *Z, int ldz)
{
    int hi = n - 1, iter = 0;
    while (hi >= 0) {
        int lo = hi;
        while (lo > 0) {
            double sub = fabs(H[IDX(lo, lo - 1, ldh)]);
            double dsum = fabs(H[IDX(lo, lo, ldh)]) + fabs(H[IDX(lo - 1, lo - 1, ldh)]);
            if (sub <= ORC_EPS * dsum || sub == 0.0) {
                H[IDX(lo, lo - 1, ldh)] = 0.0;
                break;
            }
            --lo;
        }
        if (lo == hi) { --hi; iter = 0; continue; }
        if (lo == hi - 1) {
            orc_split_2x2(n, H, ldh, Z, ldz, hi - 1);
            hi -= 2;
            iter = 0;
            continue;
        }
        if (++iter > 60) return 3;
        double s, t;
        const double h11 = H[IDX(hi - 1, hi - 1, ldh)], h12 = H[IDX(hi - 1, hi, ldh)];
        const double h21 = H[IDX(hi, hi - 1, ldh)], h22 = H[IDX(hi, hi, ldh)];
        if (iter % 10 == 0) {
            /* exceptional shift pair after a run of sweeps without deflation */
            double w = fabs(h21) + fabs(H[IDX(hi - 1, hi - 2, ldh)]);
            s = 1.5 * w + h22;
            t = w * w;
        } else {
            s = h11 + h22;             /* s1 + s2 */
            t = h11 * h22 - h12 * h21; /* s1 s2 */
        }
        const double a00 = H[IDX(lo, lo, ldh)], a01 = H[IDX(lo, lo + 1, ldh)];
        const double a10 = H[IDX(lo + 1, lo, ldh)], a11 = H[IDX(lo + 1, lo + 1, ldh)];
        double x = a00 * a00 + a01 * a10 - s * a00 + t;
        double y = a10 * (a00 + a11 - s);
        double z = a10 * H[IDX(lo + 2, lo + 1, ldh)];
        for (int k = lo; k <= hi - 2; ++k) {
            double v[3], beta;
            orc_house3(3, x, y, z, v, &beta);
            const int c0 = k > lo ? k - 1 : lo;
            orc_house_rows(H, ldh, k, 3, c0, n, v, beta);
            const int r1 = (k + 4 < hi + 1) ? k + 4 : hi + 1;
            orc_house_cols(H, ldh, k, 3, 0, r1, v, beta);
            orc_house_cols(Z, ldz, k, 3, 0, n, v, beta);
            if (k > lo) H[IDX(k + 1, k - 1, ldh)] = H[IDX(k + 2, k - 1, ldh)] = 0.0;
            x = H[IDX(k + 1, k, ldh)];
            y = H[IDX(k + 2, k, ldh)];
            if (k < hi - 2) z = H[IDX(k + 3, k, ldh)];
        }
        /* last step: a 2-vector reflector on rows / columns hi-1, hi */
        double v[3], beta;
        orc_house3(2, x, y, 0.0, v, &beta);
        orc_house_rows(H, ldh, hi - 1, 2, hi - 2, n, v, beta);
        orc_house_cols(H, ldh, hi - 1, 2, 0, hi + 1, v, beta);
        orc_house_cols(Z, ldz, hi - 1, 2, 0, n, v, beta);
        H[IDX(hi, hi - 2, ldh)] = 0.0;
    }
    /* below the first subdiagonal, and the subdiagonal outside 2x2 blocks,
     * is zero in exact arithmetic */
    for (int j = 0; j < n; ++j)
        for (int i = j + 2; i < n; ++i) H[IDX(i, j, ldh)] = 0.0;
    return 0;
}

/* Real Schur decomposition A = Q T Q^T of a real matrix: the Householder   */
/* Hessenberg reduction (real reflectors: the complex routine on a real     */
/* matrix keeps every quantity real) and the double-shift sweeps.           */
int orc_real_schur(int n, const double *A, int lda, double *Q, double *T)
{
    size_t nn = (size_t)n * (size_t)n;
    if (nn == 0) return 0;
    zc *H = (zc *)calloc(nn, sizeof(zc));
    zc *Qc = (zc *)calloc(nn, sizeof(zc));
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) H[IDX(i, j, n)] = A[IDX(i, j, lda)];
    orc_hessenberg(n, H, n, Qc, n);
    for (size_t e = 0; e < nn; ++e) { T[e] = creal(H[e]); Q[e] = creal(Qc[e]); }
    for (int j = 0; j < n; ++j)
        for (int i = j + 2; i < n; ++i) T[IDX(i, j, n)] = 0.0;
    free(H); free(Qc);
    return orc_real_schur_qr(n, T, n, Q, n);
}

/* start of each diagonal block of quasi-triangular T (blk[b] .. blk[b+1]-1) */
static int orc_blocks(int n, const double *T, int ldt, int *blk)
{
    int nb = 0, i = 0;
    while (i < n) {
        blk[nb++] = i;
        i += (i + 1 < n && T[IDX(i + 1, i, ldt)] != 0.0) ? 2 : 1;
    }
    blk[nb] = n;
    return nb;
}

/* solve the p x q Sylvester equation A Y + Y B = C (p, q <= 2) through its  */
/* Kronecker form (I (x) A + B^T (x) I) vec(Y) = vec(C), Gaussian           */
/* elimination with partial pivoting; A (lda), B (ldb), C -> Y (ldc).        */
static int orc_small_sylv(int p, int q, const double *A, int lda, const double *B, int ldb, double *C, int ldc)
{
    const int m = p * q;
    double K[4][5];
    for (int c = 0; c < q; ++c)
        for (int r = 0; r < p; ++r) {
            const int row = r + c * p;
            for (int cc = 0; cc < q; ++cc)
                for (int rr = 0; rr < p; ++rr) {
                    double v = 0.0;
                    if (cc == c) v += A[IDX(r, rr, lda)];
                    if (rr == r) v += B[IDX(cc, c, ldb)];
                    K[row][rr + cc * p] = v;
                }
            K[row][m] = C[IDX(r, c, ldc)];
        }
    for (int col = 0; col < m; ++col) {
        int piv = col;
        for (int r = col + 1; r < m; ++r)
            if (fabs(K[r][col]) > fabs(K[piv][col])) piv = r;
        if (K[piv][col] == 0.0) return 2;
        if (piv != col)
            for (int e = 0; e <= m; ++e) { double tmp = K[col][e]; K[col][e] = K[piv][e]; K[piv][e] = tmp; }
        for (int r = col + 1; r < m; ++r) {
            const double f = K[r][col] / K[col][col];
            for (int e = col; e <= m; ++e) K[r][e] -= f * K[col][e];
        }
    }
    double y[4];
    for (int r = m - 1; r >= 0; --r) {
        double acc = K[r][m];
        for (int e = r + 1; e < m; ++e) acc -= K[r][e] * y[e];
        y[r] = acc / K[r][r];
    }
    for (int c = 0; c < q; ++c)
        for (int r = 0; r < p; ++r) C[IDX(r, c, ldc)] = y[r + c * p];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* S = T^{1/2} for real quasi-triangular T (Remark 2.1; the recurrence of   */
/* Eq. (subst) over the diagonal blocks): a 1x1 block t > 0 gives sqrt(t);  */
/* a 2x2 block with eigenvalues theta +- i mu gives                          */
/*   S_ii = alpha I + (T_ii - theta I) / (2 alpha),                          */
/* alpha = Re sqrt(theta + i mu) (the principal root of the pair); block    */
/* (i, j) then solves S_ii S_ij + S_ij S_jj = T_ij - sum_{i<k<j} S_ik S_kj. */
/* Returns 0, or 2 for a real eigenvalue <= 0 or a singular block system.   */
/* ------------------------------------------------------------------------ */
int orc_qtrisqrt(int n, const double *T, int ldt, double *S, int lds)
{
    int *blk = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    const int nb = orc_blocks(n, T, ldt, blk);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) S[IDX(i, j, lds)] = 0.0;
    int st = 0;
    for (int b = 0; b < nb && !st; ++b) {
        const int i0 = blk[b], p = blk[b + 1] - blk[b];
        if (p == 1) {
            const double t = T[IDX(i0, i0, ldt)];
            if (t <= 0.0) st = 2;
            else S[IDX(i0, i0, lds)] = sqrt(t);
        } else {
            const double a = T[IDX(i0, i0, ldt)], bb = T[IDX(i0, i0 + 1, ldt)];
            const double c = T[IDX(i0 + 1, i0, ldt)], d = T[IDX(i0 + 1, i0 + 1, ldt)];
            const double theta = 0.5 * (a + d);
            const double mu2 = -(0.25 * (a - d) * (a - d) + bb * c);
            if (mu2 <= 0.0) { st = 2; break; }
            const double alpha = creal(orc_csqrt(theta + I * sqrt(mu2)));
            S[IDX(i0, i0, lds)] = alpha + (a - theta) / (2.0 * alpha);
            S[IDX(i0, i0 + 1, lds)] = bb / (2.0 * alpha);
            S[IDX(i0 + 1, i0, lds)] = c / (2.0 * alpha);
            S[IDX(i0 + 1, i0 + 1, lds)] = alpha + (d - theta) / (2.0 * alpha);
        }
    }
    for (int dist = 1; dist < nb && !st; ++dist)
        for (int bi = 0; bi + dist < nb && !st; ++bi) {
            const int bj = bi + dist;
            const int i0 = blk[bi], p = blk[bi + 1] - i0, j0 = blk[bj], q = blk[bj + 1] - j0;
            double C[4];
            for (int c = 0; c < q; ++c)
                for (int r = 0; r < p; ++r) {
                    double acc = T[IDX(i0 + r, j0 + c, ldt)];
                    for (int k = blk[bi + 1]; k < j0; ++k) acc -= S[IDX(i0 + r, k, lds)] * S[IDX(k, j0 + c, lds)];
                    C[r + c * p] = acc;
                }
            st = orc_small_sylv(p, q, &S[IDX(i0, i0, lds)], lds, &S[IDX(j0, j0, lds)], lds, C, p);
            for (int c = 0; c < q; ++c)
                for (int r = 0; r < p; ++r) S[IDX(i0 + r, j0 + c, lds)] = C[r + c * p];
        }
    free(blk);
    return st;
}

/* ------------------------------------------------------------------------ */
/* S Y + Y St = C for real quasi-triangular S (m x m) and St (n x n): block */
/* Bartels-Stewart over their diagonal blocks, block rows bottom-up and     */
/* block columns left to right,                                              */
/*   S_II Y_IJ + Y_IJ St_JJ = C_IJ - sum_{K>I} S_IK Y_KJ - sum_{L<J} Y_IL St_LJ. */
/* C (ldc) is overwritten by Y.  Returns 0 or 2 (singular block system).     */
/* ------------------------------------------------------------------------ */
int orc_qrtrsyl(int m, int n, const double *S, int lds, const double *St, int ldst, double *C, int ldc)
{
    int *bm = (int *)malloc(sizeof(int) * (size_t)(m + 1));
    int *bn = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    const int nbm = orc_blocks(m, S, lds, bm), nbn = orc_blocks(n, St, ldst, bn);
    int st = 0;
    for (int J = 0; J < nbn && !st; ++J)
        for (int Ib = nbm - 1; Ib >= 0 && !st; --Ib) {
            const int i0 = bm[Ib], p = bm[Ib + 1] - i0, j0 = bn[J], q = bn[J + 1] - j0;
            double R[4];
            for (int c = 0; c < q; ++c)
                for (int r = 0; r < p; ++r) {
                    double acc = C[IDX(i0 + r, j0 + c, ldc)];
                    for (int k = bm[Ib + 1]; k < m; ++k) acc -= S[IDX(i0 + r, k, lds)] * C[IDX(k, j0 + c, ldc)];
                    for (int l = 0; l < j0; ++l) acc -= C[IDX(i0 + r, l, ldc)] * St[IDX(l, j0 + c, ldst)];
                    R[r + c * p] = acc;
                }
            st = orc_small_sylv(p, q, &S[IDX(i0, i0, lds)], lds, &St[IDX(j0, j0, ldst)], ldst, R, p);
            for (int c = 0; c < q; ++c)
                for (int r = 0; r < p; ++r) C[IDX(i0 + r, j0 + c, ldc)] = R[r + c * p];
        }
    free(bm); free(bn);
    return st;
}
