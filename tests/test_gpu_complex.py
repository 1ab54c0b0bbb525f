"""GPU parity tests for complex input (the method is stated for A in
C^{n x n}, Sec. 1): the complex FP64 residual kernel element by element
against the oracle's FP64 evaluation, and the whole mixed-precision path and
FP64 Schur method against the oracle's complex Schur method."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import U64

pytestmark = pytest.mark.gpu

mp = pytest.importorskip("paper_2607_12430_gb300")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    mp.lib()


def _crandom(n, seed, shift=3.0):
    g = np.random.default_rng(seed)
    return shift * np.eye(n) + (g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))) / np.sqrt(2 * n)


def _dev(A):
    # the binding passes row-major storage as column-major: hand it A^T so
    # that the library works on A itself
    return torch.from_numpy(np.ascontiguousarray(A.T)).cuda()


def _host(X):
    return X.cpu().numpy().T


@pytest.mark.parametrize("n", [1, 2, 16, 65, 200])
def test_sqrtm_mixed_complex(n):
    A = _crandom(n, 800 + n)
    X, info = mp.sqrtm_mixed_complex(_dev(A))
    assert info["status"] == 0
    assert 1 <= info["iterations"] <= 4
    Xo = oracle.sqrtm_schur_complex(A)
    assert oracle.rel_err(_host(X), Xo) <= 1e-12
    X2, _ = mp.sqrtm_mixed_complex(_dev(A), steps=info["iterations"] + 1)
    X2 = _host(X2)
    assert np.linalg.norm(X2 @ X2 - A) <= 5 * n * U64 * np.linalg.norm(A)


@pytest.mark.parametrize("n", [16, 150])
def test_sqrtm_schur_fp64_complex(n):
    A = _crandom(n, 810 + n)
    X, info = mp.sqrtm_schur_fp64_complex(_dev(A))
    assert info["status"] == 0
    assert oracle.rel_err(_host(X), oracle.sqrtm_schur_complex(A)) <= 1e-12


def test_complex_fixed_steps_follow_oracle_refinement():
    # X_0 and the first corrections against the oracle's FP64 refinement from
    # the same factors: the FP32 start is within u32 of the root, each step
    # gains several digits, as in the oracle
    n = 90
    A = _crandom(n, 820)
    Xo = oracle.sqrtm_schur_complex(A)
    errs = []
    for k in range(3):
        X, info = mp.sqrtm_mixed_complex(_dev(A), steps=k)
        assert info["status"] == 0
        errs.append(oracle.rel_err(_host(X), Xo))
    assert errs[0] <= 1e-5 and errs[1] <= 1e-3 * errs[0] and errs[2] <= 1e-13


def test_complex_hermitian_and_real_inputs():
    g = np.random.default_rng(830)
    n = 60
    U_, _ = np.linalg.qr(g.standard_normal((n, n)) + 1j * g.standard_normal((n, n)))
    lam = 10.0 ** g.uniform(-2.0, 2.0, n)
    H = (U_ * lam) @ U_.conj().T
    X, info = mp.sqrtm_mixed_complex(_dev(H))
    assert info["status"] == 0
    assert oracle.rel_err(_host(X), (U_ * np.sqrt(lam)) @ U_.conj().T) <= 1e-12
    # a real matrix given as complex has the real method's root
    Ar = synth.shifted_gaussian(70, 3.0, seed=831)
    Xc, _ = mp.sqrtm_mixed_complex(_dev(Ar.astype(np.complex128)))
    Xc = _host(Xc)
    assert np.linalg.norm(Xc.imag) <= 1e-13 * np.linalg.norm(Xc)
    assert oracle.rel_err(Xc.real, oracle.sqrtm_schur(Ar)) <= 1e-12


@pytest.mark.parametrize("mag", [1e-40, 1e35])
def test_complex_scaling(mag):
    A = _crandom(30, 840) * mag
    X, info = mp.sqrtm_mixed_complex(_dev(A))
    assert info["status"] == 0
    assert oracle.rel_err(_host(X), oracle.sqrtm_schur_complex(A)) <= 1e-12


def test_complex_negative_real_eigenvalue_status():
    g = np.random.default_rng(850)
    n = 12
    U_, _ = np.linalg.qr(g.standard_normal((n, n)) + 1j * g.standard_normal((n, n)))
    d = np.linspace(1.0, 2.0, n).astype(np.complex128)
    d[4] = -1.5
    _, info = mp.sqrtm_mixed_complex(_dev((U_ * d) @ U_.conj().T), raise_on_error=False)
    assert info["status"] == 2


@pytest.mark.parametrize("n", [700, 1100])
def test_sqrtm_mixed_complex_large_residual(n):
    A = _crandom(n, 860 + n)
    X, info = mp.sqrtm_mixed_complex(_dev(A))
    assert info["status"] == 0
    X, _ = mp.sqrtm_mixed_complex(_dev(A), steps=info["iterations"] + 1)
    X = _host(X)
    assert np.linalg.norm(X @ X - A) <= 5 * n * U64 * np.linalg.norm(A)
    assert np.all(np.linalg.eigvals(X).real > 0)
