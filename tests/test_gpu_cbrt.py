"""GPU parity tests for the principal cube root (Sec. 4, p = 3) against the
FP64 oracle.

The two new step kernels (the blocked triangular cube root and the blocked
solve of Eq. (3rd-order)) are compared element by element with the oracle's
point recurrences on the same inputs; the whole mixed-precision path and
the FP64 Schur method are compared with the oracle's FP64 Schur cube root,
and at sizes the oracle does not reach in seconds with the residual
||X^3 - A|| / ||A||, which fixes the cube root for well-conditioned A."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import U32, U64, dev_cm, host_cm

pytestmark = pytest.mark.gpu

mp = pytest.importorskip("paper_2607_12430_gb300")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    mp.lib()


def _c64(M):
    return np.asarray(M).astype(np.complex64)


# --------------------------------------------------------------------------
# triangular cube root S = T^(1/3), V = S^2
# --------------------------------------------------------------------------
@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("n,blks", [(1, 32), (2, 32), (7, 32), (32, 32), (33, 32), (100, 32), (100, 8),
                                    (70, 5), (130, 32)])
def test_tricbrt(n, blks, fp64):
    S0 = synth.random_upper_rhp(n, seed=400 + n, re_lo=1.0)
    T = np.triu(S0 @ S0 @ S0)
    dt = torch.complex128 if fp64 else torch.complex64
    u = U64 if fp64 else U32
    Tin = T if fp64 else _c64(T)
    Sd, Vd = mp.step_tricbrt(dev_cm(Tin, dt), n, blks=blks, fp64=fp64)
    S = host_cm(Sd, n).astype(np.complex128)
    V = host_cm(Vd, n).astype(np.complex128)
    So, Vo = oracle.tricbrt(Tin.astype(np.complex128))
    assert np.all(np.tril(S, -1) == 0) and np.all(np.tril(V, -1) == 0)
    assert np.linalg.norm(S - So) <= 100 * n * u * np.linalg.norm(So)
    assert np.linalg.norm(V - Vo) <= 100 * n * u * np.linalg.norm(Vo)


def test_tricbrt_principal_branch_diagonal():
    # diagonal T: each s_ii is the principal cube root of t_ii
    t = np.array([8.0, 1j, -1j, 27 * np.exp(0.9j * np.pi), 0.001 + 0.5j, 64 * np.exp(-0.99j * np.pi)])
    T = np.diag(t)
    S, _ = mp.step_tricbrt(dev_cm(T, torch.complex128), len(t), fp64=True)
    s = np.diag(host_cm(S, len(t)))
    so = np.array([oracle.ccbrt(z) for z in t])
    assert np.abs(s - so).max() <= 8 * U64 * np.abs(so).max()
    assert np.all(np.abs(np.angle(s)) <= np.pi / 3 + 1e-15)


def test_tricbrt_negative_real_eigenvalue_status():
    T = np.diag([1.0, -8.0, 27.0]).astype(np.complex64)
    with pytest.raises(mp.SqrtmError) as e:
        mp.step_tricbrt(dev_cm(T, torch.complex64), 3)
    assert e.value.code == 2


# --------------------------------------------------------------------------
# S^2 Y + S Y S + Y S^2 = C (Eq. (3rd-order))
# --------------------------------------------------------------------------
@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("n,blks", [(1, 32), (5, 32), (32, 32), (33, 32), (96, 7), (100, 16), (130, 32)])
def test_rtrsyl3(n, blks, fp64):
    S = synth.random_upper_rhp(n, seed=410 + n, re_lo=1.0)
    g = np.random.default_rng(420 + n)
    C = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    dt = torch.complex128 if fp64 else torch.complex64
    u = U64 if fp64 else U32
    if not fp64:
        S, C = _c64(S), _c64(C)
    Sd = S.astype(np.complex128)
    V = np.triu(Sd @ Sd)
    Vin = V if fp64 else _c64(V)
    Cd = dev_cm(C, dt)
    mp.step_rtrsyl3(dev_cm(S, dt), dev_cm(Vin, dt), Cd, n, blks=blks, fp64=fp64)
    Y = host_cm(Cd, n).astype(np.complex128)
    Vd = Vin.astype(np.complex128)
    Yo = oracle.rtrsyl3(Sd, Vd, Sd, Vd, C.astype(np.complex128))
    assert np.linalg.norm(Y - Yo) <= 100 * n * u * np.linalg.norm(Yo)


# --------------------------------------------------------------------------
# whole path
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 16, 65, 200])
def test_cbrtm_mixed_general(n):
    A = synth.shifted_gaussian(n, 3.0, seed=430 + n)
    X, info = mp.cbrtm_mixed(torch.from_numpy(A).cuda())
    X = X.cpu().numpy()
    Xo = oracle.cbrtm_schur(A)
    assert info["status"] == 0
    assert 1 <= info["iterations"] <= 4
    assert oracle.rel_err(X, Xo) <= 1e-12
    # the tol = 1e-12 stopping test can exit above the rounding floor; one
    # more correction reaches it
    X2, _ = mp.cbrtm_mixed(torch.from_numpy(A).cuda(), steps=info["iterations"] + 1)
    assert oracle.rel_residual3(X2.cpu().numpy(), A) <= 10 * n * U64


@pytest.mark.parametrize("n", [16, 120])
def test_cbrtm_schur_fp64(n):
    A = synth.shifted_gaussian(n, 3.0, seed=440 + n)
    X, info = mp.cbrtm_schur_fp64(torch.from_numpy(A).cuda())
    assert info["status"] == 0
    assert oracle.rel_err(X.cpu().numpy(), oracle.cbrtm_schur(A)) <= 1e-12


@pytest.mark.parametrize("mag", [1e-30, 1e25])
def test_cbrtm_scaling(mag):
    # A = 8^-e-scaled problems keep their cube roots exact up to 2^e
    n = 40
    A = synth.shifted_gaussian(n, 3.0, seed=450) * mag
    X, info = mp.cbrtm_mixed(torch.from_numpy(A).cuda())
    assert info["status"] == 0
    assert info["scale_exponent"] == oracle.scale_exponent3(A)
    assert oracle.rel_err(X.cpu().numpy(), oracle.cbrtm_schur(A)) <= 1e-12


def test_cbrtm_known_similarity():
    # A = P diag(d^3) P^-1 (d > 0) has the principal cube root P diag(d) P^-1
    g = np.random.default_rng(460)
    n = 48
    P = np.eye(n) + 0.2 * g.standard_normal((n, n)) / np.sqrt(n)
    d = g.uniform(0.5, 2.0, n)
    A = P @ np.diag(d ** 3) @ np.linalg.inv(P)
    X, info = mp.cbrtm_mixed(torch.from_numpy(A).cuda())
    assert info["status"] == 0
    assert oracle.rel_err(X.cpu().numpy(), P @ np.diag(d) @ np.linalg.inv(P)) <= 1e-12


def test_cbrtm_fixed_steps_contract():
    # the FP32 start is about u32 away; each correction gains several digits
    n = 150
    A = synth.shifted_gaussian(n, 3.0, seed=470)
    Xo = oracle.cbrtm_schur(A)
    errs = []
    for k in range(3):
        X, info = mp.cbrtm_mixed(torch.from_numpy(A).cuda(), steps=k)
        errs.append(oracle.rel_err(X.cpu().numpy(), Xo))
    assert errs[0] <= 1e-5
    assert errs[1] <= 1e-3 * errs[0]
    assert errs[2] <= 1e-13


def test_cbrtm_negative_real_eigenvalue_status():
    g = np.random.default_rng(480)
    n = 20
    P = np.linalg.qr(g.standard_normal((n, n)))[0]
    d = np.linspace(1.0, 3.0, n)
    d[7] = -2.0
    A = P @ np.diag(d) @ P.T
    _, info = mp.cbrtm_mixed(torch.from_numpy(A).cuda(), raise_on_error=False)
    assert info["status"] == 2


@pytest.mark.parametrize("n", [512, 1024])
def test_cbrtm_mixed_large_residual(n):
    # at sizes beyond the oracle's seconds: the cube root residual at the
    # FP64 rounding level, and the eigenvalues in the principal sector
    A = synth.shifted_gaussian(n, 3.0, seed=490 + n)
    X, info = mp.cbrtm_mixed(torch.from_numpy(A).cuda())
    assert info["status"] == 0
    assert info["iterations"] <= 4
    X, _ = mp.cbrtm_mixed(torch.from_numpy(A).cuda(), steps=info["iterations"] + 1)
    X = X.cpu().numpy()
    assert oracle.rel_residual3(X, A) <= 10 * n * U64
    ev = np.linalg.eigvals(X)
    assert np.all(np.abs(np.angle(ev)) < np.pi / 3)
