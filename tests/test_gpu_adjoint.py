"""GPU tests of the adjoint (sqrtm_backward): the gradient of <G, sqrt(A)>
is the solution Y of X^T Y + Y X^T = G.  Checked against the dense FP64
Kronecker solve at n = 16, against the oracle's FP64 Schur-factor solve and
central finite differences (h = 1e-6) at n = 256, and through
torch.autograd."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

mp = pytest.importorskip("paper_2607_12430_gb300")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    mp.lib()


@pytest.mark.parametrize("kind", ["general", "spd"])
@pytest.mark.parametrize("seed", range(4))
def test_adjoint_kronecker_n16(kind, seed):
    n = 16
    if kind == "general":
        A = synth.shifted_gaussian(n, 3.0, seed=400 + seed)
    else:
        A, _, _ = synth.spd_case(n, -1.0, 1.0, seed=400 + seed)
    G = synth.gaussian((n, n), seed=410 + seed)
    # Y inherits the forward iterate's error times the condition of
    # Y -> X^T Y + Y X^T, so the forward solve is converged to the FP64 floor
    X, info = mp.sqrtm_mixed(torch.from_numpy(A).cuda(), tol=1e-15, steps=6)
    Y, binfo = mp.sqrtm_backward(torch.from_numpy(G).cuda(), tol=1e-14)
    Xo = oracle.sqrtm_schur(A)
    Yo = oracle.adjoint_kron(Xo, G)
    assert binfo["status"] == 0
    assert oracle.rel_err(Y.cpu().numpy(), Yo) <= 1e-12


def test_adjoint_n256_schur_oracle_and_fd():
    """Differentiation workload shape: n = 256, A = 3I + G/sqrt(n),
    cotangent N(0,1)."""
    As, Gs = synth.config_adjoint(count=2)
    for A, G in zip(As, Gs):
        X, info = mp.sqrtm_mixed(torch.from_numpy(A).cuda())
        Y, binfo = mp.sqrtm_backward(torch.from_numpy(G).cuda(), tol=1e-13)
        Y = Y.cpu().numpy()
        Xo, Q, T, S = oracle.sqrtm_schur(A, return_factors=True)
        Yo = oracle.adjoint_schur(Q, S, G)
        assert binfo["status"] == 0
        assert oracle.rel_err(Y, Yo) <= 1e-11
        h = 1e-6
        for s in range(2):
            E = synth.gaussian(A.shape, seed=420 + s)
            Xp, _ = mp.sqrtm_mixed(torch.from_numpy(A + h * E).cuda(), steps=4)
            Xm, _ = mp.sqrtm_mixed(torch.from_numpy(A - h * E).cuda(), steps=4)
            fd = float(np.sum(G * (Xp.cpu().numpy() - Xm.cpu().numpy()))) / (2 * h)
            an = float(np.sum(Y * E))
            assert abs(fd - an) <= 1e-6 * abs(an) + 1e-6


def test_autograd_function():
    n = 24
    A = torch.from_numpy(synth.shifted_gaussian(n, 3.0, seed=430)).cuda().requires_grad_(True)
    G = torch.from_numpy(synth.gaussian((n, n), seed=431)).cuda()
    X = mp.sqrtm(A, tol=1e-14)
    (X * G).sum().backward()
    Xo = oracle.sqrtm_schur(A.detach().cpu().numpy())
    Yo = oracle.adjoint_kron(Xo, G.cpu().numpy())
    assert oracle.rel_err(A.grad.cpu().numpy(), Yo) <= 1e-12


def test_backward_without_factors_status():
    n = 8
    A = torch.from_numpy(synth.shifted_gaussian(n, 3.0, seed=440)).cuda()
    mp.sqrtm_schur_fp64(A)  # the FP64 method keeps no low-precision factors
    _, info = mp.sqrtm_backward(torch.ones((n, n), dtype=torch.float64, device="cuda"), raise_on_error=False)
    assert info["status"] == 8
