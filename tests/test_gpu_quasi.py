"""GPU parity tests for the real quasi-triangular kernels (Remark 2.1): the
square root of a real quasi-upper-triangular T and the quasi-triangular
Sylvester solve, element by element against the oracle's real routines on
the same (storage-precision-rounded) inputs, and on real Schur factors the
oracle computes."""
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


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("n", [1, 2, 3, 7, 33, 100, 257])
def test_qtrisqrt(n, fp64):
    T = synth.random_quasi_upper(n, seed=1000 + n)
    dt, u = (torch.float64, U64) if fp64 else (torch.float32, U32)
    Tin = T if fp64 else T.astype(np.float32)
    S = host_cm(mp.step_qtrisqrt(dev_cm(Tin, dt), n, fp64=fp64), n).astype(np.float64)
    So = oracle.qtrisqrt(Tin.astype(np.float64))
    assert np.all(np.tril(S, -2) == 0)
    assert np.linalg.norm(S - So) <= 100 * n * u * np.linalg.norm(So)


def test_qtrisqrt_of_real_schur_factor():
    # the real Schur factor of a real matrix (oracle) as input: X = Q S Q^T
    # is the principal square root
    n = 80
    A = synth.shifted_gaussian(n, 3.0, seed=1010)
    Q, T = oracle.real_schur(A)
    S = host_cm(mp.step_qtrisqrt(dev_cm(T, torch.float64), n, fp64=True), n)
    assert oracle.rel_err(Q @ S @ Q.T, oracle.sqrtm_schur(A)) <= 1e-12


def test_qtrisqrt_negative_real_eigenvalue_status():
    T = np.array([[1.0, 2.0, 0.5], [0.0, -4.0, 1.0], [0.0, 0.0, 9.0]], dtype=np.float32)
    with pytest.raises(mp.SqrtmError) as e:
        mp.step_qtrisqrt(dev_cm(T, torch.float32), 3)
    assert e.value.code == 2


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("m,nn", [(1, 1), (2, 3), (9, 12), (40, 31), (130, 129)])
def test_qrtrsyl(m, nn, fp64):
    S = synth.random_quasi_upper(m, seed=1020 + m)
    St = synth.random_quasi_upper(nn, seed=1030 + nn)
    C = synth.gaussian((m, nn), seed=1040 + m * nn)
    dt, u = (torch.float64, U64) if fp64 else (torch.float32, U32)
    if not fp64:
        S, St, C = S.astype(np.float32), St.astype(np.float32), C.astype(np.float32)
    Cd = dev_cm(C, dt)
    mp.step_qrtrsyl(dev_cm(S, dt), m, dev_cm(St, dt), nn, Cd, fp64=fp64)
    Y = host_cm(Cd, m, nn).astype(np.float64)
    Yo = oracle.qrtrsyl(S.astype(np.float64), St.astype(np.float64), C.astype(np.float64))
    assert np.linalg.norm(Y - Yo) <= 100 * (m + nn) * u * np.linalg.norm(Yo)


# --------------------------------------------------------------------------
# real Schur stage and the whole real variant (SQRTM_KIND_REAL)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("n", [1, 2, 3, 8, 41, 130])
def test_real_schur(n, fp64):
    A = synth.shifted_gaussian(n, 0.7, seed=1100 + n)
    dt, u = (torch.float64, U64) if fp64 else (torch.float32, U32)
    Ain = A if fp64 else A.astype(np.float32)
    Td = dev_cm(Ain, dt)
    Qd = mp.step_real_schur(Td, n, fp64=fp64)
    T = host_cm(Td, n).astype(np.float64)
    Q = host_cm(Qd, n).astype(np.float64)
    A64 = Ain.astype(np.float64)
    assert np.linalg.norm(Q @ T @ Q.T - A64) <= 50 * n * u * np.linalg.norm(A64)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 50 * n * u
    assert np.all(np.tril(T, -2) == 0)
    sub = np.diag(T, -1)
    assert not np.any((sub[1:] != 0) & (sub[:-1] != 0))  # 2x2 blocks do not overlap
    for i in np.nonzero(sub)[0]:
        a, b, c, d = T[i, i], T[i, i + 1], T[i + 1, i], T[i + 1, i + 1]
        assert 0.25 * (a - d) ** 2 + b * c < 0  # a complex conjugate pair
    ev = np.sort_complex(np.linalg.eigvals(T))
    evo = np.sort_complex(np.linalg.eigvals(oracle.real_schur(A64)[1]))
    assert np.abs(ev - evo).max() <= 200 * n * u * np.linalg.norm(A64)


@pytest.mark.parametrize("n", [1, 2, 5, 16, 65, 150])
def test_sqrtm_mixed_real_kind(n):
    A = synth.shifted_gaussian(n, 1.5, seed=1200 + n)
    X, info = mp.sqrtm_mixed(torch.from_numpy(A).cuda(), kind=mp.KIND_REAL)
    assert info["status"] == 0 and info["kind_used"] == mp.KIND_REAL
    assert 1 <= info["iterations"] <= 4
    Xo = oracle.sqrtm_real_schur(A)
    assert oracle.rel_err(X.cpu().numpy(), Xo) <= 1e-12
    assert oracle.rel_err(Xo, oracle.sqrtm_schur(A)) <= 1e-12


def test_real_kind_fp64_method_and_steps():
    n = 90
    A = synth.shifted_gaussian(n, 1.5, seed=1300)
    Xo = oracle.sqrtm_real_schur(A)
    X64, i64 = mp.sqrtm_schur_fp64(torch.from_numpy(A).cuda(), kind=mp.KIND_REAL)
    assert i64["status"] == 0 and oracle.rel_err(X64.cpu().numpy(), Xo) <= 1e-12
    errs = []
    for k in range(3):
        X, info = mp.sqrtm_mixed(torch.from_numpy(A).cuda(), kind=mp.KIND_REAL, steps=k)
        assert info["status"] == 0
        errs.append(oracle.rel_err(X.cpu().numpy(), Xo))
    assert errs[0] <= 1e-5 and errs[1] <= 1e-3 * errs[0] and errs[2] <= 1e-13


def test_real_kind_negative_eigenvalue_status():
    g = np.random.default_rng(1400)
    n = 12
    P = np.linalg.qr(g.standard_normal((n, n)))[0]
    d = np.linspace(1.0, 2.0, n)
    d[5] = -1.0
    _, info = mp.sqrtm_mixed(torch.from_numpy(P @ np.diag(d) @ P.T).cuda(), kind=mp.KIND_REAL,
                             raise_on_error=False)
    assert info["status"] == 2
