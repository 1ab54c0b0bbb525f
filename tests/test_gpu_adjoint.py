"""GPU tests of the adjoint (sqrtm_backward, sqrtm_backward_factors): the
gradient of <G, sqrt(A)> is the solution Y of X^T Y + Y X^T = G.  Checked
against the dense FP64 Kronecker solve at n = 16, against the oracle's FP64
Schur-factor solve at n = 256, by central finite differences (h = 1e-6) on
every matrix of the differentiation workload (64 x n = 256), and through
torch.autograd with several square roots in one graph, each of which must
be differentiated with its own factors."""
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


def _case16(kind, seed):
    n = 16
    if kind == "general":
        return synth.shifted_gaussian(n, 3.0, seed=seed)
    A, _, _ = synth.spd_case(n, -1.0, 1.0, seed=seed)
    return A


@pytest.mark.parametrize("kind", ["general", "spd"])
@pytest.mark.parametrize("seed", range(4))
def test_adjoint_kronecker_n16(kind, seed):
    n = 16
    A = _case16(kind, 400 + seed)
    G = synth.gaussian((n, n), seed=410 + seed)
    # Y inherits the forward iterate's error times the condition of
    # Y -> X^T Y + Y X^T, so the forward solve is converged to the FP64 floor
    X, info = mp.sqrtm_mixed(torch.from_numpy(A).cuda(), tol=1e-15, steps=6)
    Y, binfo = mp.sqrtm_backward(torch.from_numpy(G).cuda(), tol=1e-14)
    Xo = oracle.sqrtm_schur(A)
    Yo = oracle.adjoint_kron(Xo, G)
    assert binfo["status"] == 0
    assert oracle.rel_err(Y.cpu().numpy(), Yo) <= 1e-12


def test_adjoint_n256_schur_oracle():
    """Differentiation workload shape: n = 256, A = 3I + G/sqrt(n), cotangent
    N(0,1).  X = sqrt(A) is close to sqrt(3) I, so the adjoint operator
    Y -> X^T Y + Y X^T has condition number about 1.4: a backward solve
    refined to a relative residual of 1e-13 is within 1e-12 of the oracle's
    gradient (itself accurate to the FP64 floor)."""
    As, Gs = synth.config_adjoint(count=4)
    for A, G in zip(As, Gs):
        mp.sqrtm_mixed(torch.from_numpy(A).cuda())
        Y, binfo = mp.sqrtm_backward(torch.from_numpy(G).cuda(), tol=1e-13)
        _, Q, _, S = oracle.sqrtm_schur(A, return_factors=True)
        Yo = oracle.adjoint_schur(Q, S, G)
        assert binfo["status"] == 0
        assert oracle.rel_err(Y.cpu().numpy(), Yo) <= 1e-12


def test_adjoint_workload_autograd_and_finite_differences():
    """All 64 matrices of the differentiation workload through torch.autograd
    in ONE graph (64 forward calls on the same handle before any backward
    pass), each gradient checked by central differences (h = 1e-6) in 4
    seeded directions: the truncation error h^2 ||D^3 sqrt|| and the rounding
    error u / h put the difference quotient within about 1e-10 relative of
    the derivative, so 1e-7 relative is a safe bound that a gradient built
    from another matrix's factors (errors of order 1) cannot meet."""
    As, Gs = synth.config_adjoint()
    h = 1e-6
    leaves = [torch.from_numpy(A).cuda().requires_grad_(True) for A in As]
    loss = 0.0
    for Ad, G in zip(leaves, Gs):
        loss = loss + (mp.sqrtm(Ad, tol=1e-13) * torch.from_numpy(G).cuda()).sum()
    loss.backward()
    for i, (A, G, Ad) in enumerate(zip(As, Gs, leaves)):
        Y = Ad.grad.cpu().numpy()
        for d in range(4):
            E = synth.gaussian(A.shape, seed=5000 + 4 * i + d)
            Xp, _ = mp.sqrtm_mixed(torch.from_numpy(A + h * E).cuda(), steps=4)
            Xm, _ = mp.sqrtm_mixed(torch.from_numpy(A - h * E).cuda(), steps=4)
            fd = float(np.sum(G * (Xp.cpu().numpy() - Xm.cpu().numpy()))) / (2 * h)
            an = float(np.sum(Y * E))
            assert abs(fd - an) <= 1e-7 * abs(an), (i, d, fd, an)
    # and the first four against the oracle's FP64 Schur-factor gradient
    for i in range(4):
        _, Q, _, S = oracle.sqrtm_schur(As[i], return_factors=True)
        Yo = oracle.adjoint_schur(Q, S, Gs[i])
        assert oracle.rel_err(leaves[i].grad.cpu().numpy(), Yo) <= 1e-12


def test_autograd_function():
    n = 24
    A = torch.from_numpy(synth.shifted_gaussian(n, 3.0, seed=430)).cuda().requires_grad_(True)
    G = torch.from_numpy(synth.gaussian((n, n), seed=431)).cuda()
    X = mp.sqrtm(A, tol=1e-14)
    (X * G).sum().backward()
    Xo = oracle.sqrtm_schur(A.detach().cpu().numpy())
    Yo = oracle.adjoint_kron(Xo, G.cpu().numpy())
    assert oracle.rel_err(A.grad.cpu().numpy(), Yo) <= 1e-12


def test_autograd_interleaved_calls_keep_their_own_factors():
    """Two square roots of the same size in one graph, a plain forward call
    of that size and one of another size in between, and an SPD square root
    too: every gradient must match the Kronecker gradient of its OWN X."""
    n = 16
    A1 = _case16("general", 450)
    A2 = _case16("general", 451)
    A3 = _case16("spd", 452)
    G1, G2, G3 = (synth.gaussian((n, n), seed=460 + k) for k in range(3))
    t1, t2, t3 = (torch.from_numpy(A).cuda().requires_grad_(True) for A in (A1, A2, A3))
    X1 = mp.sqrtm(t1, tol=1e-15)
    mp.sqrtm_mixed(torch.from_numpy(_case16("general", 453)).cuda())           # same n, no autograd
    mp.sqrtm_mixed(torch.from_numpy(synth.shifted_gaussian(20, 3.0, seed=454)).cuda())  # other n
    X2 = mp.sqrtm(t2, tol=1e-15)
    X3 = mp.sqrtm(t3, tol=1e-15)
    mp.sqrtm_mixed(torch.from_numpy(_case16("general", 455)).cuda())
    loss = ((X1 * torch.from_numpy(G1).cuda()).sum() + (X2 * torch.from_numpy(G2).cuda()).sum()
            + (X3 * torch.from_numpy(G3).cuda()).sum())
    loss.backward()
    for t, A, G in ((t1, A1, G1), (t2, A2, G2), (t3, A3, G3)):
        Yo = oracle.adjoint_kron(oracle.sqrtm_schur(A), G)
        assert oracle.rel_err(t.grad.cpu().numpy(), Yo) <= 1e-12
    # a gradient taken from the wrong call's factors would be far off
    wrong = oracle.adjoint_kron(oracle.sqrtm_schur(A2), G1)
    assert oracle.rel_err(t1.grad.cpu().numpy(), wrong) > 1e-3


def test_backward_factors_entry_points():
    n = 16
    A1, A2 = _case16("general", 470), _case16("general", 471)
    G = synth.gaussian((n, n), seed=472)
    mp.sqrtm_mixed(torch.from_numpy(A1).cuda(), tol=1e-15, steps=6)
    f1 = mp.take_factors()
    assert f1.n == n
    # the handle keeps none after the move
    _, info = mp.sqrtm_backward(torch.from_numpy(G).cuda(), raise_on_error=False)
    assert info["status"] == 8
    with pytest.raises(mp.SqrtmError) as e:
        mp.take_factors()
    assert e.value.code == 8
    mp.sqrtm_mixed(torch.from_numpy(A2).cuda(), tol=1e-15, steps=6)
    Y1, i1 = mp.sqrtm_backward_factors(f1, torch.from_numpy(G).cuda(), tol=1e-14)
    Y1b, _ = mp.sqrtm_backward_factors(f1, torch.from_numpy(G).cuda(), tol=1e-14)  # not consumed
    Y2, _ = mp.sqrtm_backward(torch.from_numpy(G).cuda(), tol=1e-14)               # the handle's own
    assert i1["status"] == 0
    assert oracle.rel_err(Y1.cpu().numpy(), oracle.adjoint_kron(oracle.sqrtm_schur(A1), G)) <= 1e-12
    assert torch.equal(Y1, Y1b)
    assert oracle.rel_err(Y2.cpu().numpy(), oracle.adjoint_kron(oracle.sqrtm_schur(A2), G)) <= 1e-12
    # size mismatch: status 8
    G8 = torch.ones((8, 8), dtype=torch.float64, device="cuda")
    _, info = mp.sqrtm_backward_factors(f1, G8, raise_on_error=False)
    assert info["status"] == 8
    f1.close()


def test_backward_without_factors_status():
    n = 8
    A = torch.from_numpy(synth.shifted_gaussian(n, 3.0, seed=440)).cuda()
    mp.sqrtm_schur_fp64(A)  # the FP64 method keeps no low-precision factors
    _, info = mp.sqrtm_backward(torch.ones((n, n), dtype=torch.float64, device="cuda"), raise_on_error=False)
    assert info["status"] == 8
