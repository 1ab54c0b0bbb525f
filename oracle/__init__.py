"""FP64 CPU oracle for the mixed-precision matrix square root (arXiv 2607.12430).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  The GPU library never
imports, links or calls anything here, and nothing here imports the GPU library.

Two layers:

* ``oracle.c`` (loaded with ctypes): the FP64 Schur method of Sec. 1 with its
  own Householder Hessenberg reduction and single-shift complex QR, the point
  recurrence of Eq. (subst) for ``T^{1/2}``, a cyclic Jacobi eigensolver, the
  point Bartels-Stewart solve and the block recursion of Algorithm 1.
* the numpy functions below: the definitions of each refinement step of
  Algorithms 2 and 3 (residual, transform, Sylvester solve, back-transform,
  update), written in FP64 with plain matrix products as the only library
  primitive, plus Kronecker-form solves (Eq. (vec)) used as independent checks.
* the principal cube root (Sec. 4, p = 3): the triangular cube root by its
  point recurrence, the point solve of Eq. (3rd-order) and the FP64 Schur
  method (C), with the refinement steps of Sec. 4 in numpy.

Readings of the paper that the oracle fixes (the paper is silent on them):

* scaling before rounding to low precision (Sec. 5 asks for "appropriate
  scaling" without saying which): ``A_s = 4^-e A`` with ``e`` from the binary
  exponent of ``||A||_F / sqrt(n)``; then ``sqrt(A) = 2^e sqrt(A_s)`` exactly;
* real ``A`` uses the complex Schur form and the real part of every complex
  product that lands in ``X``;
* parity unpinned: none -- every function here is pinned by a test in
  ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None


def load(path):
    """Open a compiled oracle library and declare its C signatures."""
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i = ctypes.c_int
    L.orc_hessenberg.argtypes = [i, P, i, P, i]
    L.orc_hessenberg.restype = None
    L.orc_schur_qr.argtypes = [i, P, i, P, i]
    L.orc_schur_qr.restype = i
    L.orc_schur.argtypes = [i, P, i, P, P]
    L.orc_schur.restype = i
    L.orc_trisqrt.argtypes = [i, P, i, P, i]
    L.orc_trisqrt.restype = i
    L.orc_sqrtm_schur.argtypes = [i, P, i, P, i, P, P, P]
    L.orc_sqrtm_schur.restype = i
    L.orc_zsqrtm_schur.argtypes = [i, P, i, P, i, P, P, P]
    L.orc_zsqrtm_schur.restype = i
    L.orc_real_schur_qr.argtypes = [i, P, i, P, i]
    L.orc_real_schur_qr.restype = i
    L.orc_real_schur.argtypes = [i, P, i, P, P]
    L.orc_real_schur.restype = i
    L.orc_qtrisqrt.argtypes = [i, P, i, P, i]
    L.orc_qtrisqrt.restype = i
    L.orc_qrtrsyl.argtypes = [i, i, P, i, P, i, P, i]
    L.orc_qrtrsyl.restype = i
    L.orc_jacobi_eig.argtypes = [i, P, i, P, i, P]
    L.orc_jacobi_eig.restype = i
    L.orc_bs_solve.argtypes = [i, i, P, i, P, i, P, i]
    L.orc_bs_solve.restype = i
    L.orc_rtrsyl.argtypes = [i, i, P, i, P, i, P, i, i]
    L.orc_rtrsyl.restype = i
    L.orc_tricbrt.argtypes = [i, P, i, P, i, P, i]
    L.orc_tricbrt.restype = i
    L.orc_rtrsyl3.argtypes = [i, i, P, i, P, i, P, i, P, i, P, i]
    L.orc_rtrsyl3.restype = i
    L.orc_cbrtm_schur.argtypes = [i, P, i, P, i, P, P, P, P]
    L.orc_cbrtm_schur.restype = i
    L.orc_threads.argtypes = [i]
    L.orc_threads.restype = i
    return L


def threads(count=0):
    """Thread count of the oracle's parallel loops (independent columns of the
    Householder updates and plain products; bitwise the same results for any
    count): count > 0 sets it; returns the count in use."""
    return int(lib().orc_threads(int(count)))


def lib():
    """Load (building first if needed) the compiled C oracle."""
    global _lib
    if _lib is None:
        _lib = load(_build.build())
    return _lib


def _f(a, dtype):
    """Fortran-ordered contiguous copy (column-major, ld = rows)."""
    return np.array(a, dtype=dtype, order="F", copy=True)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: status {code}")
        self.code = code


# ---------------------------------------------------------------------------
# Schur method (Sec. 1; Sec. 2.1 first paragraph)
# ---------------------------------------------------------------------------
def hessenberg(A):
    """Householder reduction ``A = Q H Q^H`` (complex).  Returns (H, Q)."""
    n = A.shape[0]
    H = _f(A, np.complex128)
    Q = np.zeros((n, n), dtype=np.complex128, order="F")
    lib().orc_hessenberg(n, _p(H), max(n, 1), _p(Q), max(n, 1))
    return H, Q


def schur_qr(H, Z):
    """Single-shift complex QR on Hessenberg ``H``; returns (T, Z) with the
    rotations accumulated into ``Z``."""
    n = H.shape[0]
    T = _f(H, np.complex128)
    Zc = _f(Z, np.complex128)
    st = lib().orc_schur_qr(n, _p(T), max(n, 1), _p(Zc), max(n, 1))
    if st:
        raise OracleError(st, "schur_qr")
    return T, Zc


def schur(A):
    """Complex Schur decomposition of real ``A``: ``A = Q T Q^H``."""
    n = A.shape[0]
    Af = _f(A, np.float64)
    Q = np.zeros((n, n), dtype=np.complex128, order="F")
    T = np.zeros((n, n), dtype=np.complex128, order="F")
    st = lib().orc_schur(n, _p(Af), max(n, 1), _p(Q), _p(T))
    if st:
        raise OracleError(st, "schur")
    return Q, T


def csqrt(z):
    """Principal square root of a complex scalar: the C routine, reached
    through the 1-by-1 case of ``trisqrt`` (whose diagonal step it is)."""
    return trisqrt(np.array([[complex(z)]]))[0, 0]


def trisqrt(T):
    """``S = T^{1/2}`` of upper triangular ``T`` by Eq. (subst)."""
    n = T.shape[0]
    Tf = _f(T, np.complex128)
    S = np.zeros((n, n), dtype=np.complex128, order="F")
    st = lib().orc_trisqrt(n, _p(Tf), max(n, 1), _p(S), max(n, 1))
    if st:
        raise OracleError(st, "trisqrt")
    return S


def sqrtm_schur(A, return_factors=False):
    """The FP64 Schur method (Sec. 1): ``X = Q T^{1/2} Q^H``, real part for
    real ``A``.  This is the ground truth the paper's accuracy plots use
    (Sec. 5.1)."""
    n = A.shape[0]
    Af = _f(A, np.float64)
    X = np.zeros((n, n), dtype=np.float64, order="F")
    Q = np.zeros((n, n), dtype=np.complex128, order="F")
    T = np.zeros((n, n), dtype=np.complex128, order="F")
    S = np.zeros((n, n), dtype=np.complex128, order="F")
    st = lib().orc_sqrtm_schur(n, _p(Af), max(n, 1), _p(X), max(n, 1), _p(Q), _p(T), _p(S))
    if st:
        raise OracleError(st, "sqrtm_schur")
    if return_factors:
        return X, Q, T, S
    return X


def sqrtm_schur_complex(A, return_factors=False):
    """The FP64 Schur method for a complex matrix (the method is stated for
    A in C^{n x n}, Sec. 1): ``X = Q T^{1/2} Q^H``, all complex."""
    n = A.shape[0]
    Af = _f(A, np.complex128)
    X = np.zeros((n, n), dtype=np.complex128, order="F")
    Q = np.zeros((n, n), dtype=np.complex128, order="F")
    T = np.zeros((n, n), dtype=np.complex128, order="F")
    S = np.zeros((n, n), dtype=np.complex128, order="F")
    st = lib().orc_zsqrtm_schur(n, _p(Af), max(n, 1), _p(X), max(n, 1), _p(Q), _p(T), _p(S))
    if st:
        raise OracleError(st, "zsqrtm_schur")
    if return_factors:
        return X, Q, T, S
    return X


def refine_complex(A, Q, S, X0, steps, blks=32):
    """Algorithm 2 steps 5-11 for complex A with frozen factors and the
    stopping test nullified, in FP64: ``R = A - X X``, ``Y`` from
    ``S Y + Y S = Q^H R Q`` (Algorithm 1), ``X += Q Y Q^H`` (no real part
    taken: X is complex).  Returns the iterates ``[X0, ..., X_steps]``."""
    X = np.asarray(X0, dtype=np.complex128).copy()
    Q = np.asarray(Q, dtype=np.complex128)
    out = [X.copy()]
    for _ in range(steps):
        R = np.asarray(A, dtype=np.complex128) - X @ X
        Y = rtrsyl(S, S, Q.conj().T @ R @ Q, blks)
        X = X + Q @ Y @ Q.conj().T
        out.append(X.copy())
    return out


# ---------------------------------------------------------------------------
# real arithmetic for real A (Remark 2.1): quasi-triangular Schur form
# ---------------------------------------------------------------------------
def real_schur(A):
    """Real Schur decomposition ``A = Q T Q^T``: Q orthogonal, T
    quasi-upper-triangular (2x2 diagonal blocks only for complex conjugate
    eigenvalue pairs).  Returns (Q, T)."""
    n = A.shape[0]
    Af = _f(A, np.float64)
    Q = np.zeros((n, n), dtype=np.float64, order="F")
    T = np.zeros((n, n), dtype=np.float64, order="F")
    st = lib().orc_real_schur(n, _p(Af), max(n, 1), _p(Q), _p(T))
    if st:
        raise OracleError(st, "real_schur")
    return Q, T


def qtrisqrt(T):
    """``S = T^{1/2}`` of real quasi-upper-triangular ``T`` (real
    arithmetic, 2x2 blocks kept whole)."""
    n = T.shape[0]
    Tf = _f(T, np.float64)
    S = np.zeros((n, n), dtype=np.float64, order="F")
    st = lib().orc_qtrisqrt(n, _p(Tf), max(n, 1), _p(S), max(n, 1))
    if st:
        raise OracleError(st, "qtrisqrt")
    return S


def qrtrsyl(S, St, C):
    """``S Y + Y St = C`` for real quasi-upper-triangular S and St."""
    m, n = C.shape
    Sf, Stf, Y = _f(S, np.float64), _f(St, np.float64), _f(C, np.float64)
    st = lib().orc_qrtrsyl(m, n, _p(Sf), max(m, 1), _p(Stf), max(n, 1), _p(Y), max(m, 1))
    if st:
        raise OracleError(st, "qrtrsyl")
    return Y


def sqrtm_real_schur(A, return_factors=False):
    """The FP64 Schur method in real arithmetic (Remark 2.1):
    ``X = Q T^{1/2} Q^T`` with the real Schur form."""
    Q, T = real_schur(A)
    S = qtrisqrt(T)
    X = Q @ S @ Q.T
    if return_factors:
        return X, Q, T, S
    return X


def refine_real(A, Q, S, X0, steps):
    """Algorithm 2 steps 5-11 with real factors (Remark 2.1), stopping test
    nullified, in FP64: ``R = A - X X``; ``S Y + Y S = Q^T R Q``
    (quasi-triangular); ``X += Q Y Q^T``.  Returns ``[X0, ..., X_steps]``."""
    X = np.asarray(X0, dtype=np.float64).copy()
    out = [X.copy()]
    for _ in range(steps):
        R = np.asarray(A, dtype=np.float64) - X @ X
        Y = qrtrsyl(S, S, Q.T @ R @ Q)
        X = X + Q @ Y @ Q.T
        out.append(X.copy())
    return out


# ---------------------------------------------------------------------------
# Symmetric positive definite case (Algorithm 3)
# ---------------------------------------------------------------------------
def jacobi_eig(A):
    """Cyclic Jacobi ``A = V diag(lam) V^T`` for symmetric ``A``."""
    n = A.shape[0]
    W = _f(A, np.float64)
    V = np.zeros((n, n), dtype=np.float64, order="F")
    lam = np.zeros(n, dtype=np.float64)
    st = lib().orc_jacobi_eig(n, _p(W), max(n, 1), _p(V), max(n, 1), _p(lam))
    if st:
        raise OracleError(st, "jacobi_eig")
    return V, lam


def sqrtm_from_eig(V, lam):
    """``X = V diag(sqrt(lam)) V^T`` -- Algorithm 3 steps 2-3 applied to a
    given spectral decomposition (the SPD square root in closed form)."""
    lam = np.asarray(lam, dtype=np.float64)
    if np.any(lam <= 0):
        raise OracleError(2, "sqrtm_from_eig: non-positive eigenvalue")
    s = np.sqrt(lam)
    return (V * s[None, :]) @ V.T


def sqrtm_spd(A):
    """FP64 square root of a symmetric positive definite matrix through the
    oracle's own Jacobi spectral decomposition."""
    V, lam = jacobi_eig(A)
    return sqrtm_from_eig(V, lam)


# ---------------------------------------------------------------------------
# Triangular Sylvester equations (Sec. 2.2.2, Algorithm 1)
# ---------------------------------------------------------------------------
def bs_solve(S, St, C):
    """Point Bartels-Stewart solve of ``S Y + Y St = C`` (upper triangular)."""
    m, n = C.shape
    Sf, Stf = _f(S, np.complex128), _f(St, np.complex128)
    Y = _f(C, np.complex128)
    st = lib().orc_bs_solve(m, n, _p(Sf), max(m, 1), _p(Stf), max(n, 1), _p(Y), max(m, 1))
    if st:
        raise OracleError(st, "bs_solve")
    return Y


def rtrsyl(S, St, C, blks=32):
    """Algorithm 1: ``Y = rtrsyl(S, St, C, blks)``."""
    m, n = C.shape
    Sf, Stf = _f(S, np.complex128), _f(St, np.complex128)
    Y = _f(C, np.complex128)
    st = lib().orc_rtrsyl(m, n, _p(Sf), max(m, 1), _p(Stf), max(n, 1), _p(Y), max(m, 1),
                          int(blks))
    if st:
        raise OracleError(st, "rtrsyl")
    return Y


def sylvester_kron(S, St, C):
    """Dense solve of ``S Y + Y St = C`` in Kronecker form
    ``(I (x) S + St^T (x) I) vec(Y) = vec(C)`` (Eq. (vec)); tiny sizes only."""
    m, n = C.shape
    K = np.kron(np.eye(n), S) + np.kron(St.T, np.eye(m))
    y = np.linalg.solve(K, C.reshape(-1, order="F"))
    return y.reshape((m, n), order="F")


def adjoint_kron(X, G):
    """Gradient of ``<G, sqrtm(A)>`` with respect to real ``A``: the solution
    ``Y`` of ``X^T Y + Y X^T = G`` (adjoint of the Frechet derivative, whose
    operator is ``E -> F`` with ``X F + F X = E``, Eq. (correction)), by a
    dense Kronecker solve.  Tiny sizes only."""
    n = X.shape[0]
    K = np.kron(np.eye(n), X.T) + np.kron(X, np.eye(n))
    y = np.linalg.solve(K, np.asarray(G, dtype=np.float64).reshape(-1, order="F"))
    return y.reshape((n, n), order="F")


def adjoint_schur(Q, S, G, blks=32):
    """Same gradient through the FP64 Schur factors ``X = Q S Q^H``:
    ``X W + W X = G^T`` with ``W = Y^T``; in the Schur basis
    ``S V + V S = Q^H G^T Q`` (Algorithm 1), ``W = Q V Q^H``."""
    Gt = np.asarray(G, dtype=np.float64).T
    V = rtrsyl(S, S, Q.conj().T @ Gt @ Q, blks)
    W = Q @ V @ Q.conj().T
    return np.real(W).T.copy()


# ---------------------------------------------------------------------------
# Refinement steps of Algorithms 2 and 3, each written out in FP64
# ---------------------------------------------------------------------------
def scale_exponent(A):
    """Power-of-4 scaling before rounding ``A`` to low precision: ``e`` such
    that ``A_s = 4^-e A`` has ``||A_s||_F / sqrt(n)`` in ``[1/4, 1)``.  With
    ``r = ||A||_F / sqrt(n) = m 2^p``, ``m`` in ``[1/2, 1)``: ``e = ceil(p/2)``
    gives ``r 4^-e = m 2^(p - 2e)`` with ``p - 2e`` in ``{0, -1}``."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    if n == 0:
        return 0
    r = math.sqrt(float(np.sum(A * A)) / n)
    if r == 0.0 or not math.isfinite(r):
        return 0
    _, p = math.frexp(r)
    return -((-p) // 2)


def residual(A, X):
    """Algorithm 2/3 step 5: ``R = A - X^2`` in working precision and
    ``||R||_F``."""
    A = np.asarray(A, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    R = A - X @ X
    return R, float(np.linalg.norm(R))


def transform_in(Q, R):
    """Algorithm 2/3 step 8: ``R~ = Q^H R Q`` (in FP64 here)."""
    Q = np.asarray(Q)
    return Q.conj().T @ np.asarray(R) @ Q


def diag_solve(s, Rt):
    """Algorithm 3 step 9: ``y_ij = r_ij / (s_i + s_j)``."""
    s = np.asarray(s)
    return np.asarray(Rt) / (s[:, None] + s[None, :])


def transform_out(Q, Y):
    """Algorithm 2/3 step 10: ``dX = Q Y Q^H``; real part for real ``A``."""
    Q = np.asarray(Q)
    return np.real(Q @ np.asarray(Y) @ Q.conj().T)


def refine(A, Q, S, X0, steps, blks=32, spd=False):
    """Algorithms 2 / 3 steps 4-12 with the stopping test nullified (as in
    the accuracy runs of Sec. 5.1): ``steps`` corrections from ``X0`` with
    frozen factors ``Q``, ``S``; all arithmetic in FP64.  Returns the list of
    iterates ``[X0, X1, ..., X_steps]``."""
    X = np.asarray(X0, dtype=np.float64).copy()
    out = [X.copy()]
    for _ in range(steps):
        R, _ = residual(A, X)
        Rt = transform_in(Q, R)
        if spd:
            Y = diag_solve(np.diag(S), Rt)
        else:
            Y = rtrsyl(S, S, Rt, blks)
        X = X + transform_out(Q, Y)
        out.append(X.copy())
    return out


def rel_err(X, Xref):
    """``||X - Xref||_F / ||Xref||_F`` (the error measure of Sec. 5.1)."""
    return float(np.linalg.norm(np.asarray(X) - np.asarray(Xref)) / np.linalg.norm(Xref))


def rel_residual(X, A):
    """``||X^2 - A||_F / ||A||_F`` (the residual measure of Sec. 5.1)."""
    X = np.asarray(X, dtype=np.float64)
    A = np.asarray(A, dtype=np.float64)
    return float(np.linalg.norm(X @ X - A) / np.linalg.norm(A))


# ---------------------------------------------------------------------------
# Principal cube root (Sec. 4, p = 3)
# ---------------------------------------------------------------------------
def tricbrt(T):
    """``S = T^{1/3}`` of upper triangular ``T`` and ``V = S^2`` by the point
    recurrence of the Schur method for p-th roots (Sec. 4): for i < j,
    ``s_ij (s_ii^2 + s_ii s_jj + s_jj^2) = t_ij - s_ii sum s_ik s_kj -
    sum s_ik v_kj`` (k strictly between i and j), ``v_ij = s_ij (s_ii + s_jj)
    + sum s_ik s_kj``; ``s_ii`` the principal cube root (argument in
    (-pi/3, pi/3]).  Returns (S, V)."""
    n = T.shape[0]
    Tf = _f(T, np.complex128)
    S = np.zeros((n, n), dtype=np.complex128, order="F")
    V = np.zeros((n, n), dtype=np.complex128, order="F")
    st = lib().orc_tricbrt(n, _p(Tf), max(n, 1), _p(S), max(n, 1), _p(V), max(n, 1))
    if st:
        raise OracleError(st, "tricbrt")
    return S, V


def ccbrt(z):
    """Principal cube root of a complex scalar (the 1-by-1 case of
    ``tricbrt``, whose diagonal step it is)."""
    return tricbrt(np.array([[complex(z)]]))[0][0, 0]


def rtrsyl3(S, V, St, Vt, C):
    """Point solve of ``S^2 Y + S Y St + Y St^2 = C`` (Eq. (3rd-order)),
    ``V = S^2``, ``Vt = St^2``, upper triangular."""
    m, n = C.shape
    Y = _f(C, np.complex128)
    args = []
    for M in (S, V, St, Vt):
        Mf = _f(M, np.complex128)
        args.append(Mf)
    st = lib().orc_rtrsyl3(m, n, _p(args[0]), max(m, 1), _p(args[1]), max(m, 1), _p(args[2]), max(n, 1),
                           _p(args[3]), max(n, 1), _p(Y), max(m, 1))
    if st:
        raise OracleError(st, "rtrsyl3")
    return Y


def sylvester3_kron(S, St, C):
    """Kronecker-form solve of Eq. (3rd-order):
    ``(I (x) S^2 + St^T (x) S + (St^2)^T (x) I) vec(Y) = vec(C)``."""
    m, n = C.shape
    S = np.asarray(S, dtype=np.complex128)
    St = np.asarray(St, dtype=np.complex128)
    K = np.kron(np.eye(n), S @ S) + np.kron(St.T, S) + np.kron((St @ St).T, np.eye(m))
    y = np.linalg.solve(K, np.asarray(C, dtype=np.complex128).reshape(-1, order="F"))
    return y.reshape((m, n), order="F")


def cbrtm_schur(A, return_factors=False):
    """The FP64 Schur method for the principal cube root (Sec. 4):
    ``X = Q T^{1/3} Q^H``, real part for real ``A``."""
    n = A.shape[0]
    Af = _f(A, np.float64)
    X = np.zeros((n, n), dtype=np.float64, order="F")
    Q, T, S, V = (np.zeros((n, n), dtype=np.complex128, order="F") for _ in range(4))
    st = lib().orc_cbrtm_schur(n, _p(Af), max(n, 1), _p(X), max(n, 1), _p(Q), _p(T), _p(S), _p(V))
    if st:
        raise OracleError(st, "cbrtm_schur")
    if return_factors:
        return X, Q, T, S, V
    return X


def scale_exponent3(A):
    """Power-of-8 scaling for the cube root: ``e`` such that
    ``A_s = 8^-e A`` has ``||A_s||_F / sqrt(n)`` in ``[1/8, 1)``; then
    ``A^{1/3} = 2^e A_s^{1/3}`` exactly.  With ``r = m 2^p``, ``m`` in
    ``[1/2, 1)``: ``e = ceil(p / 3)``."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    if n == 0:
        return 0
    r = math.sqrt(float(np.sum(A * A)) / n)
    if r == 0.0 or not math.isfinite(r):
        return 0
    _, p = math.frexp(r)
    return -((-p) // 3)


def residual3(A, X):
    """Sec. 4 step 2 (p = 3): ``R = A - X^3`` in working precision."""
    X = np.asarray(X, dtype=np.float64)
    R = np.asarray(A, dtype=np.float64) - X @ (X @ X)
    return R, float(np.linalg.norm(R))


def refine3(A, Q, S, V, X0, steps):
    """Sec. 4 steps 2-4 (p = 3) with frozen factors and the stopping test
    nullified: ``R = A - X^3``; ``Y`` solves Eq. (3rd-order) with ``St = S``
    for ``Q^H R Q``; ``X += Re(Q Y Q^H)``; all in FP64.  Returns the iterates
    ``[X0, ..., X_steps]``."""
    X = np.asarray(X0, dtype=np.float64).copy()
    out = [X.copy()]
    for _ in range(steps):
        R, _ = residual3(A, X)
        Y = rtrsyl3(S, V, S, V, transform_in(Q, R))
        X = X + transform_out(Q, Y)
        out.append(X.copy())
    return out


def rel_residual3(X, A):
    """``||X^3 - A||_F / ||A||_F``."""
    X = np.asarray(X, dtype=np.float64)
    A = np.asarray(A, dtype=np.float64)
    return float(np.linalg.norm(X @ (X @ X) - A) / np.linalg.norm(A))
