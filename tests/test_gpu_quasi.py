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
