"""Plant plausible mistakes in a copy of the C oracle (on the CPU) and check
that the pins catch every one: each mutant must fail at least one of the
invariant checks below.  The real oracle passes all of them."""
import os
import subprocess

import numpy as np
import pytest

import synth

U = 2.0 ** -53
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

# (name, original text, mutated text)
MUTATIONS = [
    ("trisqrt_sum_drops_last_term", "for (int k = i + 1; k < j; ++k) acc -= S[IDX(i, k, lds)] * S[IDX(k, j, lds)];",
     "for (int k = i + 1; k < j - 1; ++k) acc -= S[IDX(i, k, lds)] * S[IDX(k, j, lds)];"),
    ("trisqrt_denominator_sign", "zc den = S[IDX(i, i, lds)] + S[IDX(j, j, lds)];",
     "zc den = S[IDX(i, i, lds)] - S[IDX(j, j, lds)];"),
    ("trisqrt_transposed_product", "acc -= S[IDX(i, k, lds)] * S[IDX(k, j, lds)];",
     "acc -= S[IDX(k, i, lds)] * S[IDX(j, k, lds)];"),
    ("csqrt_branch", "if (x >= 0.0) return t + I * (y / (2.0 * t));",
     "if (x >= 0.0) return t - I * (y / (2.0 * t));"),
    ("householder_right_conj", "H[IDX(i, k + 1 + l, ldh)] -= w * conj(v[l]);",
     "H[IDX(i, k + 1 + l, ldh)] -= w * v[l];"),
    ("householder_no_accumulate", "for (int l = 0; l < m; ++l) Q[IDX(i, k + 1 + l, ldq)] -= w * conj(v[l]);",
     ";"),
    ("qr_rot_cols_conj", "H[IDX(i, p, ld)] = c * a + conj(s) * b;",
     "H[IDX(i, p, ld)] = c * a + s * b;"),
    ("qr_short_column_range", "orc_rot_cols(H, ldh, k, 0, i1 + 1, c, s);",
     "orc_rot_cols(H, ldh, k, 0, i1, c, s);"),
    ("qr_skip_z", "orc_rot_cols(Z, ldz, k, 0, n, c, s);", ";"),
    ("bs_wrong_coupling", "for (int k = 0; k < j; ++k) acc -= C[IDX(i, k, ldc)] * St[IDX(k, j, ldst)];",
     "for (int k = 0; k < j; ++k) acc -= C[IDX(i, k, ldc)] * St[IDX(j, k, ldst)];"),
    ("rtrsyl_drop_c22_update", "orc_gemm_sub(m2, n2, n1, C21, ldc, St12, ldst, C22, ldc);", ";"),
    ("rtrsyl_drop_c12_s12y22", "orc_gemm_sub(m1, n2, m2, S12, lds, C22, ldc, C12, ldc);", ";"),
    ("rtrsyl_row_split_order", "if ((st = orc_rtrsyl(m2, n, S22, lds, St, ldst, C2, ldc, blks))) return st;\n        orc_gemm_sub(m1, n, m2, S12, lds, C2, ldc, C1, ldc);",
     "orc_gemm_sub(m1, n, m2, S12, lds, C2, ldc, C1, ldc);\n        if ((st = orc_rtrsyl(m2, n, S22, lds, St, ldst, C2, ldc, blks))) return st;"),
    ("jacobi_angle_sign", "double tau = (A[IDX(q, q, lda)] - A[IDX(p, p, lda)]) / (2.0 * apq);",
     "double tau = (A[IDX(p, p, lda)] - A[IDX(q, q, lda)]) / (2.0 * apq);"),
    ("schur_final_product_no_conj", "orc_zgemm('N', 'C', n, 1.0, W, n, Q, n, 0.0, P, n);",
     "orc_zgemm('N', 'N', n, 1.0, W, n, Q, n, 0.0, P, n);"),
    ("tricbrt_drops_cross_term", "zc den = si * si + si * sj + sj * sj;", "zc den = si * si + sj * sj;"),
    ("tricbrt_v_update_drops_sum", "V[IDX(i, j, ldv)] = sij * (si + sj) + sv;", "V[IDX(i, j, ldv)] = sij * (si + sj);"),
    ("ccbrt_other_branch", "double th = carg(z) / 3.0;", "double th = (carg(z) + 6.283185307179586) / 3.0;"),
    ("rtrsyl3_w_without_new_entry", "W[IDX(i, j, m)] = wp + y * St[IDX(j, j, ldst)];", "W[IDX(i, j, m)] = wp;"),
    ("zsqrtm_conjugated_result", "X[IDX(i, j, ldx)] = P[IDX(i, j, n)];", "X[IDX(i, j, ldx)] = conj(P[IDX(i, j, n)]);"),
    ("qtrisqrt_2x2_sign", "S[IDX(i0, i0, lds)] = alpha + (a - theta) / (2.0 * alpha);",
     "S[IDX(i0, i0, lds)] = alpha - (a - theta) / (2.0 * alpha);"),
    ("qrtrsyl_drop_right_coupling", "for (int l = 0; l < j0; ++l) acc -= C[IDX(i0 + r, l, ldc)] * St[IDX(l, j0 + c, ldst)];", ";"),
    ("real_schur_skip_z", "orc_house_cols(Z, ldz, k, 3, 0, n, v, beta);", ";"),
    ("rtrsyl3_transposed_vt", "for (int l = 0; l < j; ++l) acc -= C[IDX(i, l, ldc)] * Vt[IDX(l, j, ldvt)];",
     "for (int l = 0; l < j; ++l) acc -= C[IDX(i, l, ldc)] * Vt[IDX(j, l, ldvt)];"),
]


def _checks(orc):
    """Invariant checks; returns the list of names that failed."""
    failed = []

    def run(name, fn):
        try:
            ok = fn()
        except Exception:
            ok = False
        if not ok:
            failed.append(name)

    A = synth.shifted_gaussian(20, 3.0, seed=42)

    def sqrtm_residual():
        X = orc.sqrtm_schur(A)
        return orc.rel_residual(X, A) <= 5 * 20 * U and np.all(np.linalg.eigvals(X).real > 0)
    run("sqrtm_residual", sqrtm_residual)

    def zsqrtm_residual():
        g = np.random.default_rng(43)
        Ac = 3.0 * np.eye(16) + (g.standard_normal((16, 16)) + 1j * g.standard_normal((16, 16))) / 6.0
        X = orc.sqrtm_schur_complex(Ac)
        return (np.linalg.norm(X @ X - Ac) <= 20 * 16 * U * np.linalg.norm(Ac)
                and np.all(np.linalg.eigvals(X).real > 0))
    run("zsqrtm_residual", zsqrtm_residual)

    def real_schur_route():
        Ar = synth.shifted_gaussian(18, 0.5, seed=44)
        Q, T = orc.real_schur(Ar)
        ok = np.linalg.norm(Q @ T @ Q.T - Ar) <= 2000 * U * np.linalg.norm(Ar)
        Ap = synth.shifted_gaussian(18, 3.0, seed=45)
        ok = ok and orc.rel_err(orc.sqrtm_real_schur(Ap), orc.sqrtm_schur(Ap)) <= 1e-12
        Tq = synth.random_quasi_upper(9, seed=46)
        C = synth.gaussian((9, 9), seed=47)
        Y = orc.qrtrsyl(Tq, Tq, C)
        return ok and np.linalg.norm(Tq @ Y + Y @ Tq - C) <= 1e3 * U * np.linalg.norm(C)
    run("real_schur_route", real_schur_route)

    def schur_similarity():
        Q, T = orc.schur(A)
        return (np.linalg.norm(Q @ T @ Q.conj().T - A) <= 200 * U * np.linalg.norm(A)
                and np.linalg.norm(Q.conj().T @ Q - np.eye(20)) <= 200 * U)
    run("schur_similarity", schur_similarity)

    def hessenberg_complex():
        g = np.random.default_rng(8)
        Ac = g.standard_normal((10, 10)) + 1j * g.standard_normal((10, 10))
        H, Q = orc.hessenberg(Ac)
        return (np.linalg.norm(Q @ H @ Q.conj().T - Ac) <= 200 * U * np.linalg.norm(Ac)
                and np.all(np.tril(H, -2) == 0))
    run("hessenberg_complex", hessenberg_complex)

    def trisqrt_root():
        S0 = synth.random_upper_rhp(9, seed=3)
        S = orc.trisqrt(np.triu(S0 @ S0))
        return np.linalg.norm(S - S0) <= 1e4 * U * np.linalg.norm(S0)
    run("trisqrt_root", trisqrt_root)

    def csqrt_values():
        return abs(orc.csqrt(3 + 4j) - (2 + 1j)) < 1e-15 and abs(orc.csqrt(-3 - 4j) - (1 - 2j)) < 1e-15
    run("csqrt_values", csqrt_values)

    def rtrsyl_kron():
        ok = True
        for m, n, b in ((9, 9, 2), (12, 3, 2), (3, 12, 2), (1, 1, 1)):
            S = synth.random_upper_rhp(m, seed=m)
            St = synth.random_upper_rhp(n, seed=50 + n)
            C = synth.gaussian((m, n), seed=m * n) + 0j
            Yk = orc.sylvester_kron(S, St, C)
            ok &= np.linalg.norm(orc.rtrsyl(S, St, C, b) - Yk) <= 1e4 * U * np.linalg.norm(Yk)
            ok &= np.linalg.norm(orc.bs_solve(S, St, C) - Yk) <= 1e4 * U * np.linalg.norm(Yk)
        return ok
    run("rtrsyl_kron", rtrsyl_kron)

    def cbrtm_residual():
        X = orc.cbrtm_schur(A)
        ev = np.linalg.eigvals(X)
        return orc.rel_residual3(X, A) <= 10 * 20 * U and np.all(np.abs(np.angle(ev)) < np.pi / 3)
    run("cbrtm_residual", cbrtm_residual)

    def tricbrt_cube():
        S0 = synth.random_upper_rhp(9, seed=4, re_lo=1.0)  # diagonal within |arg| < pi/4
        S, V = orc.tricbrt(np.triu(S0 @ S0 @ S0))
        return (np.linalg.norm(S - S0) <= 1e4 * U * np.linalg.norm(S0)
                and np.linalg.norm(V - S0 @ S0) <= 1e4 * U * np.linalg.norm(S0 @ S0))
    run("tricbrt_cube", tricbrt_cube)

    def ccbrt_values():
        return abs(orc.ccbrt(-8.0) - (1 + 3 ** 0.5 * 1j)) < 1e-14 and abs(orc.ccbrt(8j) - (3 ** 0.5 + 1j)) < 1e-14
    run("ccbrt_values", ccbrt_values)

    def rtrsyl3_kron():
        ok = True
        for m, n in ((9, 9), (7, 3), (3, 7), (1, 1)):
            S = synth.random_upper_rhp(m, seed=m + 1, re_lo=1.0)
            St = synth.random_upper_rhp(n, seed=60 + n, re_lo=1.0)
            C = synth.gaussian((m, n), seed=m * n + 1) + 0j
            Yk = orc.sylvester3_kron(S, St, C)
            Y = orc.rtrsyl3(S, S @ S, St, St @ St, C)
            ok &= np.linalg.norm(Y - Yk) <= 1e4 * U * np.linalg.norm(Yk)
        return ok
    run("rtrsyl3_kron", rtrsyl3_kron)

    def jacobi():
        As, V, lam = synth.spd_case(12, -1, 1, seed=9)
        Vj, lj = orc.jacobi_eig(As)
        return (np.allclose(np.sort(lj), np.sort(lam), atol=1e-12)
                and np.linalg.norm(Vj @ np.diag(lj) @ Vj.T - As) <= 1e-12)
    run("jacobi", jacobi)
    return failed


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation {name}: pattern not found"
    mut = src.replace(old, new, 1)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(mut)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(c), "-lm"],
                   check=True, capture_output=True)
    return str(so)


def test_real_oracle_passes_all_checks(orc):
    assert _checks(orc) == []


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_mutant_is_caught(orc, tmp_path, name, old, new):
    so = _build_mutant(tmp_path, name, old, new)
    saved = orc._lib
    try:
        orc._lib = orc.load(so)
        failed = _checks(orc)
    finally:
        orc._lib = saved
    assert failed, f"mutant {name} passed every check"
