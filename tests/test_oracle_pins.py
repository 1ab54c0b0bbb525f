"""Pins for the FP64 oracle: each check ties an oracle routine to something
other than itself -- a closed form the paper states, exact arithmetic, an
invariant of the principal square root, a textbook library routine, or an
independent high-precision computation -- so that a dropped term, a sign or
index error or a transposed operand fails at least one of them.

All tests here run on the CPU (no GPU marker)."""
import cmath
import math
import os

import numpy as np
import pytest

import synth

U = 2.0 ** -53
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# principal scalar square root (diagonal step of Sec. 2.2.1; branch of Sec. 1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("z,expect", [
    (4.0, 2.0), (-4.0, 2.0j), (3 + 4j, 2 + 1j), (-3 + 4j, 1 + 2j), (-3 - 4j, 1 - 2j),
    (1j, (1 + 1j) / math.sqrt(2.0)), (0.0, 0.0), (2.25, 1.5), (-1e-300 + 1e-300j, None),
])
def test_csqrt_principal_branch(orc, z, expect):
    s = orc.csqrt(z)
    if expect is not None:
        assert abs(s - expect) <= 4 * U * abs(expect)
    # agrees with the C library's principal sqrt and lies in the closed RHP
    ref = cmath.sqrt(complex(z))
    assert abs(s - ref) <= 4 * U * max(abs(ref), 1e-300)
    assert s.real >= 0.0


def test_csqrt_squares_back(orc):
    g = np.random.default_rng(1)
    for _ in range(200):
        z = complex(*(g.standard_normal(2) * 10.0 ** g.uniform(-5, 5)))
        s = orc.csqrt(z)
        assert s.real > 0
        assert abs(s * s - z) <= 8 * U * abs(z)


# --------------------------------------------------------------------------
# triangular square root, Eq. (subst)
# --------------------------------------------------------------------------
def _golden_2x2():
    rows = []
    with open(os.path.join(GOLDEN, "trisqrt_2x2.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [float(x) for x in line.split()]
            T = np.array([[complex(v[0], v[1]), complex(v[2], v[3])], [0, complex(v[4], v[5])]])
            S = np.array([[complex(v[6], v[7]), complex(v[8], v[9])], [0, complex(v[10], v[11])]])
            rows.append((T, S))
    return rows


@pytest.mark.parametrize("case", range(5))
def test_trisqrt_2x2_closed_form(orc, case):
    T, S = _golden_2x2()[case]
    Sc = orc.trisqrt(T)
    assert np.allclose(Sc, S, rtol=4 * U, atol=0)


def test_trisqrt_diagonal_exact(orc):
    d = np.array([4.0, 9.0, 0.25, 16.0, 2.25 + 0j])
    S = orc.trisqrt(np.diag(d))
    assert np.array_equal(S, np.diag(np.sqrt(d)))


@pytest.mark.parametrize("n", [3, 7, 33, 64])
def test_trisqrt_recovers_principal_root(orc, n):
    # S0 upper triangular with RHP diagonal is the principal root of S0^2
    S0 = synth.random_upper_rhp(n, seed=100 + n)
    T = np.triu(S0 @ S0)
    S = orc.trisqrt(T)
    assert np.linalg.norm(S - S0) <= 1e3 * n * U * np.linalg.norm(S0)
    assert np.linalg.norm(S @ S - T) <= 10 * n * U * np.linalg.norm(S) ** 2
    assert np.all(np.diag(S).real > 0)
    assert np.all(np.tril(S, -1) == 0)


# --------------------------------------------------------------------------
# Schur decomposition: Hessenberg + QR
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 5, 16, 47])
def test_hessenberg_similarity(orc, n):
    A = synth.gaussian((n, n), seed=200 + n)
    H, Q = orc.hessenberg(A)
    assert np.all(np.tril(H, -2) == 0)
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(n)) <= 10 * n * U
    assert np.linalg.norm(Q @ H @ Q.conj().T - A) <= 10 * n * U * max(np.linalg.norm(A), 1)


@pytest.mark.parametrize("n", [1, 2, 3, 9, 40, 97])
def test_schur_invariants(orc, n):
    A = synth.shifted_gaussian(n, 3.0, seed=300 + n)
    Q, T = orc.schur(A)
    assert np.all(np.tril(T, -1) == 0)
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(n)) <= 20 * n * U
    assert np.linalg.norm(Q @ T @ Q.conj().T - A) <= 20 * n * U * np.linalg.norm(A)


def _match_spectra(got, expect):
    """Largest distance after greedily pairing each expected eigenvalue with
    the nearest unused computed one."""
    got = list(got)
    worst = 0.0
    for z in expect:
        k = int(np.argmin([abs(w - z) for w in got]))
        worst = max(worst, abs(got.pop(k) - z))
    return worst


def test_schur_2x2_eigenvalues_closed_form(orc):
    # [[a, b], [c, d]] has eigenvalues (a+d)/2 +- sqrt(((a-d)/2)^2 + bc)
    a, b, c, d = 1.0, -5.0, 2.0, 3.0
    Q, T = orc.schur(np.array([[a, b], [c, d]]))
    disc = cmath.sqrt(((a - d) / 2) ** 2 + b * c)
    expect = sorted([(a + d) / 2 + disc, (a + d) / 2 - disc], key=lambda z: (z.imag, z.real))
    got = sorted(np.diag(T), key=lambda z: (z.imag, z.real))
    assert np.allclose(got, expect, rtol=0, atol=10 * U * 5)


def test_schur_known_spectrum(orc):
    # A = P D P^{-1} with a known real block-diagonal D
    g = np.random.default_rng(7)
    n = 12
    P = np.eye(n) + 0.3 * g.standard_normal((n, n))
    eig = []
    D = np.zeros((n, n))
    for k in range(0, n, 2):
        a, b = 2.0 + k, 0.5 + 0.1 * k
        D[k:k + 2, k:k + 2] = [[a, -b], [b, a]]
        eig += [a + 1j * b, a - 1j * b]
    A = P @ D @ np.linalg.inv(P)
    Q, T = orc.schur(A)
    assert _match_spectra(np.diag(T), np.array(eig)) <= 1e4 * U * np.linalg.norm(A)


# --------------------------------------------------------------------------
# the whole FP64 Schur method (definition of Sec. 1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 4, 31, 64, 130])
def test_sqrtm_schur_invariants(orc, n):
    A = synth.shifted_gaussian(n, 3.0, seed=400 + n)
    X = orc.sqrtm_schur(A)
    assert X.dtype == np.float64
    # X^2 = A (relative residual <= 5 n u), XA = AX, spectrum in the RHP
    assert orc.rel_residual(X, A) <= 5 * n * U
    assert np.linalg.norm(X @ A - A @ X) <= 20 * n * U * np.linalg.norm(A) * np.linalg.norm(X)
    assert np.all(np.linalg.eigvals(X).real > 0)


def test_sqrtm_schur_power_of_four_scaling_is_exact(orc):
    # sqrt(4^k A) = 2^k sqrt(A): every step is invariant under an exact
    # power-of-two scaling, so the results agree bit for bit
    A = synth.shifted_gaussian(24, 3.0, seed=5)
    X = orc.sqrtm_schur(A)
    for k in (-3, 1, 5):
        Xk = orc.sqrtm_schur(A * 4.0 ** k)
        assert np.array_equal(Xk, X * 2.0 ** k)


def test_sqrtm_schur_similarity_closed_form(orc):
    # A = P blockdiag([[a,-b],[b,a]]) P^-1; sqrt of a I + b J is p I + q J with
    # p + i q = sqrt(a + i b)
    g = np.random.default_rng(11)
    n = 16
    P = np.eye(n) + 0.25 * g.standard_normal((n, n))
    D = np.zeros((n, n))
    R = np.zeros((n, n))
    for k in range(0, n, 2):
        a, b = 1.0 + 0.5 * k, (-1) ** k * (0.3 + 0.2 * k)
        r = cmath.sqrt(complex(a, b))
        D[k:k + 2, k:k + 2] = [[a, -b], [b, a]]
        R[k:k + 2, k:k + 2] = [[r.real, -r.imag], [r.imag, r.real]]
    Pi = np.linalg.inv(P)
    A = P @ D @ Pi
    Xtrue = P @ R @ Pi
    X = orc.sqrtm_schur(A)
    kap = np.linalg.cond(P)
    assert orc.rel_err(X, Xtrue) <= 50 * n * kap * U


@pytest.mark.parametrize("n", [3, 6])
def test_sqrtm_schur_vs_mpmath(orc, n):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    A = synth.shifted_gaussian(n, 2.0, seed=500 + n)
    X = orc.sqrtm_schur(A)
    Xm = mp.sqrtm(mp.matrix(A.tolist()))
    Xh = np.array([[float(mp.re(Xm[i, j])) for j in range(n)] for i in range(n)])
    assert orc.rel_err(X, Xh) <= 100 * n * U


def test_sqrtm_schur_vs_scipy(orc):
    sl = pytest.importorskip("scipy.linalg")
    A = synth.shifted_gaussian(96, 3.0, seed=600)
    X = orc.sqrtm_schur(A)
    Xs = np.real(sl.sqrtm(A))
    assert orc.rel_err(X, Xs) <= 100 * 96 * U


def test_sqrtm_schur_negative_eigenvalue_status(orc):
    with pytest.raises(orc.OracleError) as e:
        orc.sqrtm_schur(np.diag([1.0, -2.0, 3.0]))
    assert e.value.code == 2


# --------------------------------------------------------------------------
# SPD case (Algorithm 3): Jacobi spectral decomposition and closed form
# --------------------------------------------------------------------------
def test_jacobi_and_closed_form(orc):
    A, V, lam = synth.config_spd64()
    Vj, lj = orc.jacobi_eig(A)
    n = A.shape[0]
    assert np.linalg.norm(Vj.T @ Vj - np.eye(n)) <= 100 * n * U  # rotations accumulate
    assert np.allclose(np.sort(lj), np.sort(lam), rtol=0, atol=100 * n * U * lam.max())
    Xg = orc.sqrtm_from_eig(V, lam)          # generator's decomposition
    Xj = orc.sqrtm_spd(A)                    # oracle's own Jacobi
    Xs = orc.sqrtm_schur(A)                  # oracle's general Schur route
    cond = lam.max() / lam.min()
    assert orc.rel_err(Xj, Xg) <= 10 * n * math.sqrt(cond) * U
    assert orc.rel_err(Xs, Xg) <= 10 * n * math.sqrt(cond) * U
    assert np.all(np.isfinite(Xs))


def test_sqrtm_from_eig_diagonal_exact(orc):
    X = orc.sqrtm_from_eig(np.eye(3), np.array([4.0, 9.0, 16.0]))
    assert np.array_equal(X, np.diag([2.0, 3.0, 4.0]))


# --------------------------------------------------------------------------
# triangular Sylvester solves (Sec. 2.2.2, Algorithm 1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m,n,blks", [(1, 1, 32), (5, 3, 32), (9, 9, 2), (40, 7, 4),
                                      (7, 40, 4), (33, 31, 8), (64, 64, 32), (65, 33, 16)])
def test_rtrsyl_vs_kronecker(orc, m, n, blks):
    S = synth.random_upper_rhp(m, seed=700 + m)
    St = synth.random_upper_rhp(n, seed=800 + n)
    g = np.random.default_rng(m * 1000 + n)
    C = g.standard_normal((m, n)) + 1j * g.standard_normal((m, n))
    Yk = orc.sylvester_kron(S, St, C)
    Yb = orc.bs_solve(S, St, C)
    Yr = orc.rtrsyl(S, St, C, blks)
    scale = np.linalg.norm(Yk)
    assert np.linalg.norm(Yb - Yk) <= 1e3 * (m + n) * U * scale
    assert np.linalg.norm(Yr - Yk) <= 1e3 * (m + n) * U * scale
    # the equation holds, hence each block equation of Eq. (partition)
    assert np.linalg.norm(S @ Yr + Yr @ St - C) <= 100 * (m + n) * U * np.linalg.norm(C)


def test_rtrsyl_diagonal_closed_form(orc):
    # diagonal S, St: y_ij = c_ij / (s_ii + st_jj) (Algorithm 3, step 9)
    s = np.array([1.0, 2.0, 4.0, 0.5])
    t = np.array([0.5, 1.5, 3.5])
    C = np.arange(12, dtype=float).reshape(4, 3) + 1
    Y = orc.rtrsyl(np.diag(s).astype(complex), np.diag(t).astype(complex), C, blks=1)
    assert np.array_equal(Y, C / (s[:, None] + t[None, :]))


def test_rtrsyl_upper_coupling_direction(orc):
    # exact small-integer case that distinguishes S Y + Y St from S^T Y + Y St
    # and from transposed right-hand sides
    S = np.array([[1.0, 2.0], [0.0, 1.0]], dtype=complex)
    St = np.array([[1.0, 4.0], [0.0, 3.0]], dtype=complex)
    Ytrue = np.array([[1.0, 2.0], [3.0, 4.0]])
    C = S @ Ytrue + Ytrue @ St
    for blks in (1, 32):
        assert np.array_equal(orc.rtrsyl(S, St, C, blks), Ytrue)


# --------------------------------------------------------------------------
# gradient / adjoint: X^T Y + Y X^T = G
# --------------------------------------------------------------------------
def test_adjoint_routes_and_finite_differences(orc):
    n = 8
    A = synth.shifted_gaussian(n, 3.0, seed=900)
    G = synth.gaussian((n, n), seed=901)
    X, Q, T, S = orc.sqrtm_schur(A, return_factors=True)
    Yk = orc.adjoint_kron(X, G)
    Ys = orc.adjoint_schur(Q, S, G, blks=2)
    assert orc.rel_err(Ys, Yk) <= 1e3 * n * U
    # central differences of <G, sqrtm(A)> along random directions
    h = 1e-6
    for s in range(3):
        E = synth.gaussian((n, n), seed=910 + s)
        fd = (np.sum(G * orc.sqrtm_schur(A + h * E)) - np.sum(G * orc.sqrtm_schur(A - h * E))) / (2 * h)
        an = np.sum(Yk * E)
        assert abs(fd - an) <= 1e-7 * max(abs(an), 1.0)


# --------------------------------------------------------------------------
# refinement steps (Algorithms 2 and 3)
# --------------------------------------------------------------------------
def test_scale_exponent_range(orc):
    g = np.random.default_rng(3)
    for k in range(30):
        n = int(g.integers(1, 40))
        A = g.standard_normal((n, n)) * 10.0 ** g.uniform(-30, 30)
        e = orc.scale_exponent(A)
        r = math.sqrt(float(np.sum((A * 4.0 ** -e) ** 2)) / n)
        assert 0.25 <= r < 1.0 + 1e-15


def test_residual_exact_integers(orc):
    # integer X, D: X@X and A = X^2 + D are exact, so R must equal D exactly;
    # X is nonsymmetric so X^2 != X X^T, X^T X
    g = np.random.default_rng(4)
    X = g.integers(-9, 10, (7, 7)).astype(float)
    D = g.integers(-3, 4, (7, 7)).astype(float)
    R, nr = orc.residual(X @ X + D, X)
    assert np.array_equal(R, D)
    assert nr == pytest.approx(np.sqrt(np.sum(D * D)), rel=1e-15)


def test_transforms_exact_phase_permutation(orc):
    # Q = permutation times phases in {1, i, -1, -i}: all products exact
    n = 6
    perm = [3, 0, 5, 1, 4, 2]
    ph = [1, 1j, -1, -1j, 1j, -1]
    Q = np.zeros((n, n), dtype=complex)
    for j, (p, f) in enumerate(zip(perm, ph)):
        Q[p, j] = f
    R = np.arange(n * n, dtype=float).reshape(n, n)
    Rt = orc.transform_in(Q, R)
    # (Q^H R Q)_{jk} = conj(ph_j) R[perm_j, perm_k] ph_k
    expect = np.array([[np.conj(ph[j]) * R[perm[j], perm[k]] * ph[k] for k in range(n)] for j in range(n)])
    assert np.array_equal(Rt, expect)
    assert np.array_equal(orc.transform_out(Q, Rt), R)


def test_refinement_linear_rate_theorem31(orc):
    # Theorem 3.1: with frozen Z = X0 (exact factors of X0), ||E_{k+1}|| <=
    # rho0 ||E_k||, rho0 = ||B_Z^{-1}|| (2 ||E_Z|| + ||E_0||); FP64 steps.
    n = 10
    A = synth.shifted_gaussian(n, 3.0, seed=1000)
    X = orc.sqrtm_schur(A)
    E = 1e-4 * synth.gaussian((n, n), seed=1001)
    X0 = X + E
    Q0, T0 = orc.schur(X0)          # X0 = Q0 T0 Q0^H; T0 is X0's "S"
    B = np.kron(np.eye(n), X0) + np.kron(X0.T, np.eye(n))
    binv = 1.0 / np.linalg.svd(B, compute_uv=False).min()
    rho0 = binv * (2 * np.linalg.norm(E) + np.linalg.norm(E))
    assert rho0 < 1
    its = orc.refine(A, Q0, T0, X0, steps=4, blks=4)
    errs = [np.linalg.norm(Xi - X) for Xi in its]
    for k in range(len(errs) - 1):
        if errs[k] < 1e3 * U * np.linalg.norm(X):
            break  # reached the rounding floor
        assert errs[k + 1] <= rho0 * errs[k] * (1 + 1e-6)
    assert orc.rel_err(its[-1], X) <= 100 * n * U


def test_refinement_spd_diag_solve(orc):
    # Algorithm 3 in FP64 from a perturbed spectral decomposition converges
    A, V, lam = synth.spd_case(20, -1.0, 1.0, seed=1100)
    Xtrue = orc.sqrtm_from_eig(V, lam)
    g = np.random.default_rng(5)
    Vp, _ = np.linalg.qr(V + 1e-5 * g.standard_normal(V.shape))
    lp = lam * (1 + 1e-5 * g.standard_normal(lam.shape))
    S = np.diag(np.sqrt(lp))
    X0 = (Vp * np.sqrt(lp)[None, :]) @ Vp.T
    its = orc.refine(A, Vp, S, X0, steps=5, spd=True)
    e = [orc.rel_err(Xi, Xtrue) for Xi in its]
    assert e[0] > 1e-7
    assert e[-1] <= 1e-13


# ---------------------------------------------------------------------------
# principal cube root (Sec. 4, p = 3)
# ---------------------------------------------------------------------------
def test_tricbrt_exact_integer_case(orc):
    # S = [[2, 1], [0, 3]]: T = S^3 = [[8, 19], [0, 27]] has this exact root
    T = np.array([[8.0, 19.0], [0.0, 27.0]], dtype=np.complex128)
    S, V = orc.tricbrt(T)
    # (the C library's cbrt need not be correctly rounded: a few ulps)
    assert np.abs(S - np.array([[2.0, 1.0], [0.0, 3.0]])).max() <= 8 * U * 3.0
    assert np.abs(V - np.array([[4.0, 5.0], [0.0, 9.0]])).max() <= 16 * U * 9.0


def test_ccbrt_principal_branch(orc):
    # the root with argument in (-pi/3, pi/3]; -8 sits on the branch cut
    # (argument pi), whose root is 2 e^{i pi/3}
    for z, w in ((27.0, 3.0), (-8.0, 1 + 3 ** 0.5 * 1j), (8j, 3 ** 0.5 + 1j), (-8j, 3 ** 0.5 - 1j)):
        assert abs(orc.ccbrt(z) - w) <= 4 * U * abs(w)


@pytest.mark.parametrize("n", [1, 5, 16, 40])
def test_tricbrt_cubes_back(orc, n):
    S0 = synth.random_upper_rhp(n, seed=300 + n, re_lo=1.0)
    T = np.triu(S0 @ S0 @ S0)
    S, V = orc.tricbrt(T)
    assert np.linalg.norm(S - S0) <= 1e3 * n * U * np.linalg.norm(S0)
    assert np.linalg.norm(V - S @ S) <= 100 * n * U * np.linalg.norm(V)


@pytest.mark.parametrize("m,n", [(1, 1), (6, 6), (9, 4), (4, 9)])
def test_rtrsyl3_matches_kronecker_solve(orc, m, n):
    S = synth.random_upper_rhp(m, seed=310 + m, re_lo=1.0)
    St = synth.random_upper_rhp(n, seed=320 + n, re_lo=1.0)
    C = synth.gaussian((m, n), seed=330 + m * n) + 1j * synth.gaussian((m, n), seed=331 + m * n)
    Yk = orc.sylvester3_kron(S, St, C)
    Y = orc.rtrsyl3(S, S @ S, St, St @ St, C)
    assert np.linalg.norm(Y - Yk) <= 1e3 * U * np.linalg.norm(Yk)
    # the equation itself
    assert np.linalg.norm(S @ S @ Y + S @ Y @ St + Y @ St @ St - C) <= 1e3 * U * np.linalg.norm(C)


@pytest.mark.parametrize("n", [3, 30, 80])
def test_cbrtm_schur_against_scipy_and_residual(orc, n):
    A = synth.shifted_gaussian(n, 3.0, seed=340 + n)
    X = orc.cbrtm_schur(A)
    assert orc.rel_residual3(X, A) <= 10 * n * U
    scipy_linalg = pytest.importorskip("scipy.linalg")
    Xs = scipy_linalg.fractional_matrix_power(A, 1.0 / 3.0)
    assert np.linalg.norm(Xs.imag) <= 1e-12 * np.linalg.norm(Xs)
    assert orc.rel_err(X, Xs.real) <= 1e-12
    ev = np.linalg.eigvals(X)
    assert np.all(np.abs(np.angle(ev)) < np.pi / 3)


def test_cbrtm_schur_known_similarity(orc):
    # A = P diag(d^3) P^-1 has the principal cube root P diag(d) P^-1 (d real > 0)
    g = np.random.default_rng(350)
    n = 12
    P = np.eye(n) + 0.3 * g.standard_normal((n, n))
    d = g.uniform(0.5, 2.0, n)
    A = P @ np.diag(d ** 3) @ np.linalg.inv(P)
    X = orc.cbrtm_schur(A)
    Xk = P @ np.diag(d) @ np.linalg.inv(P)
    assert orc.rel_err(X, Xk) <= 1e-12


def test_cbrtm_scaling_exponent(orc):
    for r in (1e-9, 0.3, 1.0, 7.0, 1e12):
        A = np.full((4, 4), r)
        e = orc.scale_exponent3(A)
        rs = np.linalg.norm(A * 8.0 ** -e) / 2.0
        assert 1 / 8 <= rs < 1


def test_refine3_contracts(orc):
    # Sec. 4 steps 2-4 with the exact factors from a perturbed start: the
    # correction is Newton's with a frozen derivative, so each step gains
    # several digits until rounding
    n = 20
    A = synth.shifted_gaussian(n, 3.0, seed=360)
    X, Q, T, S, V = orc.cbrtm_schur(A, return_factors=True)
    X0 = X + 1e-6 * synth.gaussian((n, n), seed=361)
    its = orc.refine3(A, Q, S, V, X0, 3)
    errs = [orc.rel_err(Xk, X) for Xk in its]
    assert errs[1] <= 1e-3 * errs[0]
    assert errs[2] <= 1e-13


# --------------------------------------------------------------------------
# complex input (the method is stated for A in C^{n x n}, Sec. 1)
# --------------------------------------------------------------------------
def _crandom(n, seed, shift=3.0):
    g = np.random.default_rng(seed)
    return shift * np.eye(n) + (g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))) / np.sqrt(2 * n)


@pytest.mark.parametrize("n", [1, 2, 5, 30, 90])
def test_zsqrtm_schur_invariants(orc, n):
    A = _crandom(n, 700 + n)
    X = orc.sqrtm_schur_complex(A)
    assert np.linalg.norm(X @ X - A) <= 20 * n * U * np.linalg.norm(A)
    assert np.all(np.linalg.eigvals(X).real > 0)


def test_zsqrtm_schur_known_similarity(orc):
    # A = P diag(d^2) P^-1 with complex d in the open right half plane has
    # the principal square root P diag(d) P^-1
    g = np.random.default_rng(710)
    n = 14
    P = np.eye(n) + 0.25 * (g.standard_normal((n, n)) + 1j * g.standard_normal((n, n)))
    d = g.uniform(0.5, 2.0, n) + 1j * g.uniform(-1.5, 1.5, n)
    Pi = np.linalg.inv(P)
    X = orc.sqrtm_schur_complex(P @ np.diag(d * d) @ Pi)
    assert orc.rel_err(X, P @ np.diag(d) @ Pi) <= 1e-12


def test_zsqrtm_schur_hermitian_closed_form(orc):
    # Hermitian positive definite A = U diag(lam) U^H: X = U diag(sqrt(lam)) U^H
    g = np.random.default_rng(720)
    n = 25
    U_, _ = np.linalg.qr(g.standard_normal((n, n)) + 1j * g.standard_normal((n, n)))
    lam = 10.0 ** g.uniform(-2.0, 2.0, n)
    X = orc.sqrtm_schur_complex((U_ * lam) @ U_.conj().T)
    assert orc.rel_err(X, (U_ * np.sqrt(lam)) @ U_.conj().T) <= 1e-12


def test_zsqrtm_schur_real_input_matches_real_method(orc):
    A = synth.shifted_gaussian(40, 3.0, seed=730)
    Xc = orc.sqrtm_schur_complex(A.astype(np.complex128))
    assert np.linalg.norm(Xc.imag) <= 1e-13 * np.linalg.norm(Xc)
    assert orc.rel_err(Xc.real, orc.sqrtm_schur(A)) <= 1e-13


def test_zsqrtm_schur_vs_scipy(orc):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    A = _crandom(50, 740)
    assert orc.rel_err(orc.sqrtm_schur_complex(A), scipy_linalg.sqrtm(A)) <= 1e-12


def test_zsqrtm_negative_real_eigenvalue_status(orc):
    T = np.diag([2.0 + 1j, -3.0 + 0j, 1.0])
    with pytest.raises(orc.OracleError) as e:
        orc.sqrtm_schur_complex(T)
    assert e.value.code == 2


def test_refine_complex_contracts(orc):
    n = 24
    A = _crandom(n, 750)
    X, Q, T, S = orc.sqrtm_schur_complex(A, return_factors=True)
    X0 = X + 1e-6 * (np.random.default_rng(751).standard_normal((n, n)) + 0j)
    its = orc.refine_complex(A, Q, S, X0, 3)
    errs = [orc.rel_err(Xk, X) for Xk in its]
    assert errs[1] <= 1e-3 * errs[0] and errs[3] <= 1e-14


# --------------------------------------------------------------------------
# real arithmetic for real A (Remark 2.1): real Schur form, quasi-triangular
# square root and Sylvester solve
# --------------------------------------------------------------------------
def _blocks(T):
    n = T.shape[0]
    out, i = [], 0
    while i < n:
        p = 2 if i + 1 < n and T[i + 1, i] != 0.0 else 1
        out.append((i, p))
        i += p
    return out


@pytest.mark.parametrize("n,shift", [(1, 0.0), (2, 0.0), (3, 0.5), (9, 0.0), (40, 0.5), (120, 0.3)])
def test_real_schur_invariants(orc, n, shift):
    A = synth.shifted_gaussian(n, shift, seed=900 + n)
    Q, T = orc.real_schur(A)
    assert np.linalg.norm(Q @ T @ Q.T - A) <= 200 * n * U * np.linalg.norm(A)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 200 * n * U
    assert np.all(np.tril(T, -2) == 0)
    for i, p in _blocks(T):
        if p == 2:  # a 2x2 block holds a complex conjugate pair
            a, b, c, d = T[i, i], T[i, i + 1], T[i + 1, i], T[i + 1, i + 1]
            assert 0.25 * (a - d) ** 2 + b * c < 0
    ev = np.sort_complex(np.linalg.eigvals(T))
    assert np.allclose(ev, np.sort_complex(np.linalg.eigvals(A)), atol=1e-10 * np.linalg.norm(A))


def test_qtrisqrt_2x2_closed_form(orc):
    # [[t, m], [-m, t]] has eigenvalues t +- i m; its principal square root is
    # [[a, m/(2a)], [-m/(2a), a]] with a = Re sqrt(t + i m)
    for t, m in [(1.0, 1.0), (0.3, 2.0), (-0.5, 1.0), (4.0, 0.01)]:
        a = cmath.sqrt(complex(t, m)).real
        S = orc.qtrisqrt(np.array([[t, m], [-m, t]]))
        assert np.allclose(S, [[a, m / (2 * a)], [-m / (2 * a), a]], rtol=4 * U, atol=4 * U)


@pytest.mark.parametrize("n", [1, 2, 7, 30, 90])
def test_qtrisqrt_squares_back_and_principal(orc, n):
    T = synth.random_quasi_upper(n, seed=910 + n)
    S = orc.qtrisqrt(T)
    assert np.linalg.norm(S @ S - T) <= 50 * n * U * np.linalg.norm(T)
    assert np.all(np.linalg.eigvals(S).real > 0)
    # same block structure
    assert np.all(np.tril(S, -2) == 0)
    assert np.all((np.diag(S, -1) != 0) == (np.diag(T, -1) != 0))


def test_real_method_matches_complex_method(orc):
    A = synth.shifted_gaussian(60, 3.0, seed=920)
    assert orc.rel_err(orc.sqrtm_real_schur(A), orc.sqrtm_schur(A)) <= 1e-13


@pytest.mark.parametrize("m,n", [(1, 1), (4, 3), (9, 12), (25, 20)])
def test_qrtrsyl_matches_kronecker(orc, m, n):
    S = synth.random_quasi_upper(m, seed=930 + m)
    St = synth.random_quasi_upper(n, seed=940 + n)
    C = synth.gaussian((m, n), seed=950 + m * n)
    Y = orc.qrtrsyl(S, St, C)
    K = np.kron(np.eye(n), S) + np.kron(St.T, np.eye(m))
    Yk = np.linalg.solve(K, C.reshape(-1, order="F")).reshape((m, n), order="F")
    assert np.linalg.norm(Y - Yk) <= 1e3 * U * np.linalg.norm(Yk)


def test_qtrisqrt_negative_real_eigenvalue_status(orc):
    T = np.array([[1.0, 2.0, 0.5], [0.0, -4.0, 1.0], [0.0, 0.0, 9.0]])
    with pytest.raises(orc.OracleError) as e:
        orc.qtrisqrt(T)
    assert e.value.code == 2


def test_refine_real_contracts(orc):
    n = 30
    A = synth.shifted_gaussian(n, 3.0, seed=960)
    X, Q, T, S = orc.sqrtm_real_schur(A, return_factors=True)
    X0 = X + 1e-6 * synth.gaussian((n, n), seed=961)
    errs = [orc.rel_err(Xk, X) for Xk in orc.refine_real(A, Q, S, X0, 3)]
    assert errs[1] <= 1e-3 * errs[0] and errs[3] <= 1e-14


def test_threads_do_not_change_results(orc):
    # the parallel loops run each column's arithmetic unchanged: the FP64
    # Schur method gives bitwise the same X on 1 thread and on all of them
    A = synth.shifted_gaussian(160, 3.0, seed=4242)
    old = orc.threads()
    try:
        orc.threads(1)
        X1, Q1, T1, S1 = orc.sqrtm_schur(A, return_factors=True)
        orc.threads(max(2, os.cpu_count() or 2))
        Xp, Qp, Tp, Sp = orc.sqrtm_schur(A, return_factors=True)
    finally:
        orc.threads(old)
    assert np.array_equal(X1, Xp) and np.array_equal(Q1, Qp) and np.array_equal(T1, Tp)
