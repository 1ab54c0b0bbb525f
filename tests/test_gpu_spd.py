"""GPU parity tests for the symmetric positive definite path (Algorithm 3)
against the FP64 oracle: the spectral decomposition, the fused transform +
diagonal Sylvester solve, the mirrored update, and the whole square root at
reduced and full size."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import U32, U64, check_kstar, dev_cm, host_cm

pytestmark = pytest.mark.gpu

mp = pytest.importorskip("paper_2607_12430_gb300")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    mp.lib()


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("n", [1, 2, 17, 25, 41, 64, 200, 513, 1100, 2100])
def test_syevd(n, fp64):
    # the sizes span the lane counts of the FP64 multisection and ragged
    # warps; n = 25 and 41 make the eigenvector kernel's exponent table an
    # odd number of ints (the doubles after it must stay 8-byte aligned)
    A, V0, lam0 = synth.spd_case(n, -2.0, 2.0, seed=200 + n)
    e = oracle.scale_exponent(A)
    As = A * 4.0 ** -e
    dt = torch.float64 if fp64 else torch.float32
    u = U64 if fp64 else U32
    Asr = As if fp64 else As.astype(np.float32)
    V, lam = mp.step_syevd(dev_cm(Asr, dt), n, fp64=fp64)
    V = host_cm(V, n).astype(np.float64)
    lam = lam.cpu().numpy().astype(np.float64)
    nrm2 = np.linalg.norm(As, 2)
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= 100 * n * u
    assert np.linalg.norm((V * lam[None, :]) @ V.T - As) <= 100 * n * u * np.linalg.norm(As)
    assert np.abs(np.sort(lam) - np.sort(lam0 * 4.0 ** -e)).max() <= 100 * n * u * nrm2


def test_syevd_every_small_size():
    # every n from 3 to 72: odd and even sizes, ragged warps and every parity
    # of the scratch tables the eigensolver carves per size
    for n in range(3, 73):
        A, _, lam0 = synth.spd_case(n, -2.0, 2.0, seed=900 + n)
        e = oracle.scale_exponent(A)
        As = A * 4.0 ** -e
        V, lam = mp.step_syevd(dev_cm(As.astype(np.float32), torch.float32), n, fp64=False)
        V = host_cm(V, n).astype(np.float64)
        lam = lam.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(V.T @ V - np.eye(n)) <= 100 * n * U32, n
        assert np.linalg.norm((V * lam[None, :]) @ V.T - As) <= 100 * n * U32 * np.linalg.norm(As), n
        assert np.abs(np.sort(lam) - np.sort(lam0 * 4.0 ** -e)).max() <= 100 * n * U32 * np.linalg.norm(As, 2), n


@pytest.mark.parametrize("n", [1, 33, 128, 300])
def test_transform_in_spd(n):
    V = synth.haar_orthogonal(n, synth.rng(300 + n)).astype(np.float32)
    lam = (10.0 ** synth.rng(301 + n).uniform(-2, 2, n)).astype(np.float32)
    R = synth.gaussian((n, n), seed=302 + n)
    R = (R + R.T).astype(np.float32)
    Y = host_cm(mp.step_transform_in_spd(dev_cm(V, torch.float32), dev_cm(lam, torch.float32),
                                         dev_cm(R, torch.float32), n), n)
    s = np.sqrt(lam.astype(np.float64))
    Yo = oracle.diag_solve(s, oracle.transform_in(V.astype(np.float64), R.astype(np.float64)))
    smin = s.min()
    assert np.linalg.norm(Y - Yo) <= 20 * n * U32 * np.linalg.norm(R) / (2 * smin)


@pytest.mark.parametrize("n,e", [(1, 0), (70, 0), (130, 2)])
def test_transform_out_update_spd(n, e):
    V = synth.haar_orthogonal(n, synth.rng(310 + n)).astype(np.float32)
    Y = synth.gaussian((n, n), seed=311 + n)
    Y = (Y + Y.T).astype(np.float32)
    X0 = synth.gaussian((n, n), seed=312 + n)
    X0 = X0 + X0.T
    Xd = dev_cm(X0, torch.float64)
    mp.step_transform_out_update_spd(dev_cm(V, torch.float32), dev_cm(Y, torch.float32), n, Xd, e=e)
    X = host_cm(Xd, n)
    Xo = X0 + oracle.transform_out(V.astype(np.float64), Y.astype(np.float64)) * 2.0 ** e
    assert np.array_equal(X, X.T)  # mirrored epilogue keeps X exactly symmetric
    assert np.linalg.norm(X - Xo) <= 10 * n * U32 * np.linalg.norm(Y) * 2.0 ** e


@pytest.mark.parametrize("n,lo,hi", [(1, 0.0, 0.0), (2, -1.0, 1.0), (64, -2.0, 2.0), (257, -3.0, 3.0),
                                     (600, -3.0, 3.0)])
def test_sqrtm_mixed_spd(n, lo, hi):
    A, V, lam = synth.spd_case(n, lo, hi, seed=320 + n, force_ends=(n > 2))
    Xo = oracle.sqrtm_from_eig(V, lam)
    Xg = oracle.refine(A, V, np.diag(np.sqrt(lam)), Xo, steps=1, spd=True)[-1]
    X, info = mp.sqrtm_mixed(torch.from_numpy(A).cuda())
    assert info["status"] == 0
    assert info["kind_used"] == mp.KIND_SPD
    # the paper's residual test (tol = 1e-12) certifies a forward error of
    # about kappa-weighted 1e-12 only; the forward-error target is checked on
    # the stopping-test-nullified iterates (Sec. 5.1 protocol)
    errs = []
    for k in range(1, 9):
        Xk, _ = mp.sqrtm_mixed(torch.from_numpy(A).cuda(), steps=k)
        Xk = Xk.cpu().numpy()
        assert np.array_equal(Xk, Xk.T)
        errs.append(oracle.rel_err(Xk, Xg))
    check_kstar(errs, 1e-13)
    assert oracle.rel_residual(Xk, A) <= 5 * n * U64


def test_sqrtm_schur_fp64_spd64():
    """The n = 64 SPD workload, plain FP64 method only."""
    A, V, lam = synth.config_spd64()
    X, info = mp.sqrtm_schur_fp64(torch.from_numpy(A).cuda())
    assert info["kind_used"] == mp.KIND_SPD
    Xo = oracle.sqrtm_from_eig(V, lam)
    assert oracle.rel_err(X.cpu().numpy(), Xo) <= 1e-13
    # the oracle's own Jacobi route agrees as well
    assert oracle.rel_err(X.cpu().numpy(), oracle.sqrtm_spd(A)) <= 1e-13


@pytest.mark.parametrize("n,mult", [(64, 2), (256, 4), (256, 32), (512, 300), (1024, 1000)])
def test_repeated_eigenvalue(n, mult):
    # a repeated eigenvalue: the twisted factorisations of its copies would
    # all return the same vector; both methods must still find an orthonormal
    # basis of its eigenspace
    g = np.random.default_rng(n + mult)
    V = synth.haar_orthogonal(n, g)
    lam = 10.0 ** g.uniform(-2, 2, n)
    lam[:mult] = 0.5
    A = (V * lam[None, :]) @ V.T
    A = (A + A.T) / 2
    Xo = oracle.sqrtm_from_eig(V, lam)
    X, info = mp.sqrtm_schur_fp64(torch.from_numpy(A).cuda())
    assert info["kind_used"] == mp.KIND_SPD
    assert oracle.rel_err(X.cpu().numpy(), Xo) <= 1e-13
    errs = []
    for k in (1, 2, 3, 4, 5):
        X, info = mp.sqrtm_mixed(torch.from_numpy(A).cuda(), steps=k)
        errs.append(oracle.rel_err(X.cpu().numpy(), Xo))
    check_kstar(errs, 1e-13)


def test_spd_indefinite_status():
    A = np.diag([1.0, -1.0, 2.0, 3.0])
    _, info = mp.sqrtm_mixed(torch.from_numpy(A).cuda(), raise_on_error=False)
    assert info["status"] == 2


@pytest.mark.slow
def test_spd4096_full_size_parity():
    """The n = 4096, kappa = 1e6 SPD workload at full size; reference: the
    closed form V diag(sqrt(lam)) V^T of the generator's decomposition,
    polished by one FP64 refinement step with those exact factors."""
    A, V, lam = synth.config_spd4096()
    Xcf = oracle.sqrtm_from_eig(V, lam)
    Xg = oracle.refine(A, V, np.diag(np.sqrt(lam)), Xcf, steps=1, spd=True)[-1]
    errs = []
    for k in (2, 3, 4, 5, 6, 7):
        X, info = mp.sqrtm_mixed(torch.from_numpy(A).cuda(), steps=k)
        X = X.cpu().numpy()
        errs.append(oracle.rel_err(X, Xg))
        assert np.array_equal(X, X.T)
    check_kstar(errs, 1e-13)
