"""GPU parity tests for the general path (Algorithm 2) against the FP64 oracle.

Each step kernel is called through the C ABI on seeded inputs and compared
element by element with the oracle's FP64 evaluation of the same step on the
same (FP32-rounded) inputs; the tolerances follow from the precision the
step runs in (unit roundoff u32 = 2^-24 for the low-precision steps, u64 =
2^-53 for the FP64 ones) times the size of the inner sums."""
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


def _c64(M):
    return np.asarray(M).astype(np.complex64)


# --------------------------------------------------------------------------
# a1: scaling
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,mag", [(1, 1.0), (7, 1e-20), (64, 3.0), (130, 1e30)])
def test_scale_exact(n, mag):
    A = synth.gaussian((n, n), seed=10 + n) * mag
    As, e, nrm = mp.step_scale(dev_cm(A, torch.float64), n)
    # the same integer rule on both sides (reading c1): the exponent is exact
    assert e == oracle.scale_exponent(A)
    assert nrm == pytest.approx(np.linalg.norm(A), rel=1e-14)
    expect = (A * 4.0 ** -e).astype(np.float32).astype(np.complex64)
    assert np.array_equal(host_cm(As, n), expect)


# --------------------------------------------------------------------------
# a2: complex Schur decomposition
# --------------------------------------------------------------------------
def _match(got, expect):
    got = list(got)
    worst = 0.0
    for z in expect:
        k = int(np.argmin([abs(w - z) for w in got]))
        worst = max(worst, abs(got.pop(k) - z))
    return worst


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("n", [1, 2, 5, 33, 100, 257, 512])
def test_schur(n, fp64):
    A = synth.shifted_gaussian(n, 3.0, seed=20 + n)
    u = U64 if fp64 else U32
    As, e, _ = mp.step_scale(dev_cm(A, torch.float64), n, fp64=fp64)
    Q = mp.step_schur(As, n, fp64=fp64)
    T = host_cm(As, n).astype(np.complex128)
    Qh = host_cm(Q, n).astype(np.complex128)
    Asn = A * 4.0 ** -e
    assert np.all(np.tril(T, -1) == 0)
    assert np.linalg.norm(Qh.conj().T @ Qh - np.eye(n)) <= 50 * n * u
    assert np.linalg.norm(Qh @ T @ Qh.conj().T - Asn) <= 50 * n * u * np.linalg.norm(Asn)
    Qo, To = oracle.schur(Asn)
    assert _match(np.diag(T), np.diag(To)) <= 200 * n * u * np.linalg.norm(Asn)


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 64, 130, 700])
def test_hessenberg_real(n, fp64):
    """The real per-column reduction (the general path beyond the cluster
    kernel's sizes) against the oracle's Householder reduction, which takes
    the same reflector signs: H agrees to rounding, Q is orthogonal and
    Q H Q^T reproduces A."""
    A = synth.shifted_gaussian(n, 3.0, seed=25 + n)
    u = U64 if fp64 else U32
    Ar = A if fp64 else A.astype(np.float32).astype(np.float64)
    H, Q = mp.step_hessenberg(dev_cm(A, torch.float64), n, fp64=fp64)
    H = host_cm(H, n).astype(np.complex128)
    Q = host_cm(Q, n).astype(np.complex128)
    assert np.all(np.imag(H) == 0) and np.all(np.imag(Q) == 0)
    H, Q = np.real(H), np.real(Q)
    assert np.all(np.tril(H, -2) == 0)
    nA = np.linalg.norm(Ar)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 20 * n * u
    assert np.linalg.norm(Q @ H @ Q.T - Ar) <= 20 * n * u * nA
    Ho, Qo = oracle.hessenberg(Ar)
    assert np.linalg.norm(H - np.real(Ho)) <= 50 * n * u * nA
    assert np.linalg.norm(Q - np.real(Qo)) <= 50 * n * u * np.sqrt(n)


# --------------------------------------------------------------------------
# a3: triangular square root
# --------------------------------------------------------------------------
@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("n,blks", [(1, 32), (7, 32), (32, 32), (33, 32), (100, 32), (100, 8), (70, 5)])
def test_trisqrt(n, blks, fp64):
    S0 = synth.random_upper_rhp(n, seed=30 + n)
    T = np.triu(S0 @ S0)
    dt = torch.complex128 if fp64 else torch.complex64
    u = U64 if fp64 else U32
    Tin = T if fp64 else _c64(T)
    S = host_cm(mp.step_trisqrt(dev_cm(Tin, dt), n, blks=blks, fp64=fp64), n).astype(np.complex128)
    So = oracle.trisqrt(Tin.astype(np.complex128))
    assert np.all(np.tril(S, -1) == 0)
    assert np.linalg.norm(S - So) <= 100 * n * u * np.linalg.norm(So)


def test_trisqrt_negative_real_eigenvalue_status():
    T = np.diag([1.0, -4.0, 9.0]).astype(np.complex64)
    with pytest.raises(mp.SqrtmError) as e:
        mp.step_trisqrt(dev_cm(T, torch.complex64), 3)
    assert e.value.code == 2


# --------------------------------------------------------------------------
# a4: X0 = Re(Q S Q^H)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,e", [(1, 0), (65, 0), (130, 3)])
def test_form_x0(n, e):
    Q = _c64(synth.random_unitary(n, seed=40 + n))
    S = _c64(synth.random_upper_rhp(n, seed=41 + n))
    X = host_cm(mp.step_form_x0(dev_cm(Q, torch.complex64), dev_cm(S, torch.complex64), n, e=e), n)
    Qd, Sd = Q.astype(np.complex128), S.astype(np.complex128)
    Xo = np.real(Qd @ Sd @ Qd.conj().T) * 2.0 ** e
    assert np.abs(X - Xo).max() <= 10 * n * U32 * np.abs(Sd).max() * n * 2.0 ** e
    # X0 is the FP32 rounding of the product, widened to FP64
    assert np.array_equal(X, (X / 2.0 ** e).astype(np.float32).astype(np.float64) * 2.0 ** e)


# --------------------------------------------------------------------------
# a5: FP64 residual
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,e", [(1, 0), (63, 0), (64, 0), (200, 2), (129, -1)])
def test_residual(n, e):
    X = synth.gaussian((n, n), seed=50 + n)
    A = X @ X + 1e-6 * synth.gaussian((n, n), seed=51 + n)
    Rhat, rn = mp.step_residual(dev_cm(A, torch.float64), dev_cm(X, torch.float64), n, e=e)
    R, rno = oracle.residual(A, X)
    R *= 4.0 ** -e
    rno *= 4.0 ** -e
    err = np.abs(host_cm(Rhat, n).astype(np.float64) - R)
    bound = np.abs(R) * U32 + 4 * n * U64 * (np.abs(X) @ np.abs(X)) * 4.0 ** -e
    assert np.all(err <= bound)
    assert rn == pytest.approx(rno, rel=1e-6)


def test_residual_exact_integers():
    g = np.random.default_rng(3)
    n = 40
    X = g.integers(-9, 10, (n, n)).astype(float)
    D = g.integers(-3, 4, (n, n)).astype(float)
    Rhat, rn = mp.step_residual(dev_cm(X @ X + D, torch.float64), dev_cm(X, torch.float64), n)
    assert np.array_equal(host_cm(Rhat, n), D.astype(np.float32))
    assert rn == np.sqrt(np.sum(D * D))


# --------------------------------------------------------------------------
# a6: transform R~ = Q^H R Q
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 17, 64, 150])
def test_transform_in(n):
    Q = _c64(synth.random_unitary(n, seed=60 + n))
    R = synth.gaussian((n, n), seed=61 + n).astype(np.float32)
    Rt = host_cm(mp.step_transform_in(dev_cm(Q, torch.complex64), dev_cm(R, torch.float32), n), n)
    Ro = oracle.transform_in(Q.astype(np.complex128), R.astype(np.float64))
    assert np.linalg.norm(Rt - Ro) <= 10 * n * U32 * np.linalg.norm(R)


# --------------------------------------------------------------------------
# a7: triangular Sylvester solve
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m,nn,blks", [(1, 1, 32), (5, 3, 32), (32, 32, 32), (33, 31, 32), (64, 100, 32),
                                       (100, 64, 16), (96, 96, 7), (130, 129, 32),
                                       # blks 32 and m a multiple of 16: the one-launch dependency-ordered solve
                                       (96, 160, 32), (256, 256, 32), (512, 512, 32), (48, 512, 32)])
def test_rtrsyl(m, nn, blks):
    S = _c64(synth.random_upper_rhp(m, seed=70 + m))
    St = _c64(synth.random_upper_rhp(nn, seed=71 + nn))
    g = np.random.default_rng(m * 1000 + nn)
    C = _c64(g.standard_normal((m, nn)) + 1j * g.standard_normal((m, nn)))
    Cd = dev_cm(C, torch.complex64)
    mp.step_rtrsyl(dev_cm(S, torch.complex64), m, dev_cm(St, torch.complex64), nn, Cd, blks=blks)
    Y = host_cm(Cd, m, nn)
    Yo = oracle.rtrsyl(S.astype(np.complex128), St.astype(np.complex128), C.astype(np.complex128), blks)
    assert np.linalg.norm(Y - Yo) <= 100 * (m + nn) * U32 * np.linalg.norm(Yo)


# --------------------------------------------------------------------------
# a8 + a9: back-transform and FP64 update
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,e", [(1, 0), (77, 0), (128, -2)])
def test_transform_out_update(n, e):
    Q = _c64(synth.random_unitary(n, seed=80 + n))
    g = np.random.default_rng(n)
    Y = _c64(g.standard_normal((n, n)) + 1j * g.standard_normal((n, n)))
    X0 = synth.gaussian((n, n), seed=81 + n)
    Xd = dev_cm(X0, torch.float64)
    mp.step_transform_out_update(dev_cm(Q, torch.complex64), dev_cm(Y, torch.complex64), n, Xd, e=e)
    X = host_cm(Xd, n)
    Xo = X0 + oracle.transform_out(Q.astype(np.complex128), Y.astype(np.complex128)) * 2.0 ** e
    assert np.linalg.norm(X - Xo) <= 10 * n * U32 * np.linalg.norm(Y) * 2.0 ** e


# --------------------------------------------------------------------------
# whole path: sqrtm_mixed and sqrtm_schur_fp64 against the FP64 Schur oracle
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 16, 65, 200])
def test_sqrtm_mixed_general(n):
    A = synth.shifted_gaussian(n, 3.0, seed=90 + n)
    X, info = mp.sqrtm_mixed(torch.from_numpy(A).cuda(), kind=mp.KIND_GENERAL)
    X = X.cpu().numpy()
    Xo = oracle.sqrtm_schur(A)
    assert info["status"] == 0
    assert oracle.rel_err(X, Xo) <= 1e-12
    assert 1 <= info["iterations"] <= 4
    # the tol = 1e-12 stopping test can exit above the rounding floor; one
    # more correction reaches the relative residual bound 5 n u
    X2, _ = mp.sqrtm_mixed(torch.from_numpy(A).cuda(), kind=mp.KIND_GENERAL, steps=info["iterations"] + 1)
    assert oracle.rel_residual(X2.cpu().numpy(), A) <= 5 * n * U64


@pytest.mark.parametrize("n", [600, 700, 1024])
def test_sqrtm_mixed_general_large(n):
    # n = 600: the shared-memory layout of the cluster Hessenberg reduction
    # (above 512); n = 1024: the two-launch-per-column reduction and the
    # cooperative chase with 16 helper CTAs over several rounds
    A = synth.shifted_gaussian(n, 3.0, seed=97 + n)
    Xo = oracle.sqrtm_schur(A)
    errs = []
    for k in (1, 2, 3, 4):
        X, info = mp.sqrtm_mixed(torch.from_numpy(A).cuda(), kind=mp.KIND_GENERAL, steps=k)
        assert info["status"] == 0
        errs.append(oracle.rel_err(X.cpu().numpy(), Xo))
    # k* corrections reach 1e-12 and later ones stay there
    assert check_kstar(errs, 1e-12) + 1 <= 3, errs
    assert oracle.rel_residual(X.cpu().numpy(), A) <= 5 * n * U64


@pytest.mark.parametrize("n", [1, 3, 64, 201, 512])
def test_sqrtm_schur_fp64(n):
    A = synth.shifted_gaussian(n, 3.0, seed=95 + n)
    X, info = mp.sqrtm_schur_fp64(torch.from_numpy(A).cuda(), kind=mp.KIND_GENERAL)
    Xo = oracle.sqrtm_schur(A)
    assert oracle.rel_err(X.cpu().numpy(), Xo) <= 1e-12


def test_general512_full_size_parity():
    """The n = 512 workload (A = 3I + G/sqrt(n)) at full size, in the same
    launch configuration the benchmark times."""
    A = synth.config_general512()
    X, info = mp.sqrtm_mixed(torch.from_numpy(A).cuda(), kind=mp.KIND_GENERAL)
    Xo = oracle.sqrtm_schur(A)
    X = X.cpu().numpy()
    assert info["status"] == 0
    assert oracle.rel_err(X, Xo) <= 1e-12
    assert oracle.rel_residual(X, A) <= 1e-12
    assert 2 <= info["iterations"] <= 4
    # per-step errors decrease (stopping test nullified, Sec. 5.1)
    errs = []
    for k in range(0, 5):
        Xk, _ = mp.sqrtm_mixed(torch.from_numpy(A).cuda(), kind=mp.KIND_GENERAL, steps=k)
        errs.append(oracle.rel_err(Xk.cpu().numpy(), Xo))
    assert errs[0] > 1e-8
    # 2 to 4 corrections reach 1e-12 (the workload's statement), falling
    # strictly until then, and later corrections keep it there
    assert 2 <= check_kstar(errs, 1e-12) <= 4, errs
    X4, _ = mp.sqrtm_mixed(torch.from_numpy(A).cuda(), kind=mp.KIND_GENERAL, steps=4)
    assert oracle.rel_residual(X4.cpu().numpy(), A) <= 5 * 512 * U64


def test_status_codes():
    # eigenvalue on the negative real axis
    A = np.diag([1.0, -2.0, 3.0]) + 0.0
    A[0, 2] = 1e-3
    _, info = mp.sqrtm_mixed(torch.from_numpy(A).cuda(), raise_on_error=False, kind=mp.KIND_GENERAL)
    assert info["status"] == 2
    # NaN input
    B = synth.shifted_gaussian(8, 3.0, seed=1)
    B[2, 3] = np.nan
    _, info = mp.sqrtm_mixed(torch.from_numpy(B).cuda(), raise_on_error=False)
    assert info["status"] == 5
    # empty input
    X, info = mp.sqrtm_mixed(torch.zeros((0, 0), dtype=torch.float64, device="cuda"))
    assert info["status"] == 0 and X.shape == (0, 0)


# --------------------------------------------------------------------------
# a3 by the recursive splitting (Deadman-Higham-Ralha) against the oracle
# --------------------------------------------------------------------------
@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("n,cutoff", [(100, 64), (130, 64), (300, 64), (300, 128), (700, 256)])
def test_trisqrt_recursive(n, cutoff, fp64):
    S0 = synth.random_upper_rhp(n, seed=35 + n)
    T = np.triu(S0 @ S0)
    dt = torch.complex128 if fp64 else torch.complex64
    u = U64 if fp64 else U32
    Tin = T if fp64 else _c64(T)
    S = host_cm(mp.step_trisqrt_rec(dev_cm(Tin, dt), n, cutoff=cutoff, fp64=fp64), n).astype(np.complex128)
    So = oracle.trisqrt(Tin.astype(np.complex128))
    assert np.all(np.tril(S, -1) == 0)
    assert np.linalg.norm(S - So) <= 100 * n * u * np.linalg.norm(So)


def test_sqrtm_mixed_recursive_trisqrt_from_tuning():
    n = 600
    A = torch.from_numpy(synth.shifted_gaussian(n, 3.0, seed=36)).cuda()
    saved = mp.get_tuning()
    try:
        mp.set_tuning([{"n_max": 1 << 20, "blks": 32, "qr_helpers": -1, "batched": 1, "spd_precision": 0,
                        "trisqrt_cutoff": 256}])
        X, info = mp.sqrtm_mixed(A, kind=mp.KIND_GENERAL, steps=3)
    finally:
        mp.set_tuning(saved)
    assert info["status"] == 0
    assert oracle.rel_residual(X.cpu().numpy(), A.cpu().numpy()) <= 5 * n * U64


# --------------------------------------------------------------------------
# status 6: a bounded device wait that runs out (no fault, no hang)
# --------------------------------------------------------------------------
def test_bounded_wait_gives_up_then_handle_recovers():
    """The cooperative chase (n >= 256) waits on its helper CTAs and they on
    it, each wait bounded.  With a 1 ns limit the first wait that has to
    wait at all gives up: every CTA leaves and the call returns 6.  The same
    handle then runs a normal call whose result matches the oracle."""
    n = 512
    A = synth.config_general512()
    Ad = torch.from_numpy(A).cuda()
    saved = mp.get_tuning()
    try:
        # the cooperative chase with 8 helper CTAs, whatever the shipped table says
        mp.set_tuning([{"n_max": 1 << 20, "blks": 32, "qr_helpers": 8, "batched": 1, "spd_precision": 0}])
        mp.set_wait_limit(1)
        _, info = mp.sqrtm_mixed(Ad, kind=mp.KIND_GENERAL, raise_on_error=False)
    finally:
        mp.set_wait_limit(0)
        mp.set_tuning(saved)
    assert info["status"] == 6
    X, info = mp.sqrtm_mixed(Ad, kind=mp.KIND_GENERAL)
    assert info["status"] == 0
    assert oracle.rel_err(X.cpu().numpy(), oracle.sqrtm_schur(A)) <= 1e-12
    with pytest.raises(mp.SqrtmError) as e:
        mp.set_wait_limit(-1)
    assert e.value.code == -2
