"""The FP64 residual of the SPD path (Algorithm 3, step 5) with X X from exact
BF16 tensor-core products of digit slices (error-free splitting), against
plain FP64 arithmetic on the host: bit-exact where the product is exactly
representable, within the FP64 product's error bound otherwise, and the
whole SPD square root with it against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import U64, check_kstar, dev_cm, host_cm

pytestmark = pytest.mark.gpu

mp = pytest.importorskip("paper_2607_12430_gb300")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    mp.lib()


def _dyadic_sym(n, bits, seed, row_exp=None):
    """Symmetric X = D M D / 2^bits with integer M, |M| < 2^bits, D = diag(2^k)."""
    g = np.random.default_rng(seed)
    M = g.integers(-(2 ** bits) + 1, 2 ** bits, size=(n, n)).astype(np.float64)
    M = np.triu(M) + np.triu(M, 1).T
    X = M / 2.0 ** bits
    if row_exp is not None:
        d = 2.0 ** row_exp
        X = d[:, None] * X * d[None, :]
    return X


@pytest.mark.parametrize("n,bits", [(300, 10), (1000, 12), (513, 10), (2200, 12)])
def test_split_residual_bit_exact_on_dyadic_inputs(n, bits):
    # every product and partial sum of X X is exact in FP64, and two digits
    # (7 bits up to n = 1024, 6 above) hold every entry of X relative to its
    # row's power of two (rows scaled by 1 or 2 exercise the per-row
    # exponents), so no digit pair is left out: both GPU residuals must
    # equal the host's exactly.  n = 2200 has more 128 x 128 output tiles
    # than the GPU has SMs, so CTAs take several tiles each
    g = np.random.default_rng(n)
    X = _dyadic_sym(n, bits, seed=n, row_exp=g.integers(0, 2, size=n))
    A = X @ X + _dyadic_sym(n, 8, seed=n + 1) / 2.0 ** 12
    R = A - X @ X  # exact
    for split in (False, True):
        Rhat, nrm = mp.step_residual_sym(dev_cm(A, torch.float64), dev_cm(X, torch.float64), n, e=0, split=split)
        Rh = host_cm(Rhat, n)
        assert np.array_equal(Rh, R.astype(np.float32)), f"split={split}"
        assert nrm == pytest.approx(np.linalg.norm(R), rel=1e-14)


@pytest.mark.parametrize("n", [256, 1000, 2048])
def test_split_residual_within_fp64_bound(n):
    # cancellation regime of the refinement: A = X X + E with E ~ 1e-13
    g = np.random.default_rng(7 + n)
    X = g.standard_normal((n, n)) / np.sqrt(n)
    X = (X + X.T) / 2 + 2.0 * np.eye(n)
    E = g.standard_normal((n, n)) * 1e-13
    E = (E + E.T) / 2
    A = X @ X + E
    e = 1
    R_host = (A - X @ X) * 4.0 ** -e
    absXX = np.abs(X) @ np.abs(X) * 4.0 ** -e
    Xd, Ad = dev_cm(X, torch.float64), dev_cm(A, torch.float64)
    Rs, ns = mp.step_residual_sym(Ad, Xd, n, e=e, split=True)
    Rf, nf = mp.step_residual_sym(Ad, Xd, n, e=e, split=False)
    Rs, Rf = host_cm(Rs, n).astype(np.float64), host_cm(Rf, n).astype(np.float64)
    # each of the three differs from the exact residual by at most about
    # n u (|X| |X|)_ij (FP64 product) plus the FP32 rounding of Rhat
    bound = 2 * n * U64 * absXX + 2.0 ** -24 * np.abs(R_host)
    assert np.all(np.abs(Rs - R_host) <= 2 * bound)
    assert np.all(np.abs(Rs - Rf) <= 2 * bound)
    assert ns == pytest.approx(nf, rel=1e-3)
    assert np.array_equal(Rs, Rs.T)


def test_split_residual_rejects_unsupported_size():
    n = 46341
    A = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(mp.SqrtmError):
        mp.step_residual_sym(A, A, n, split=True)


@pytest.mark.parametrize("resid", ["split", "fp64"])
def test_spd_sqrtm_with_split_residual(resid):
    # kappa = 1e6 SPD at n = 1024, fixed corrections: the split residual must
    # drive the same convergence as the FP64 product (Algorithm 3, <= 1e-13)
    n = 1024
    A, V, lam = synth.config_spd4096(n=n)
    Xo = (V * np.sqrt(lam)[None, :]) @ V.T
    prec = mp.PREC_FP32 if resid == "split" else mp.PREC_RESID_FP64
    errs = []
    for k in range(1, 7):
        X, info = mp.sqrtm_mixed(torch.from_numpy(np.ascontiguousarray(A)).cuda(), steps=k, precision=prec)
        errs.append(oracle.rel_err(X.cpu().numpy(), Xo))
    check_kstar(errs, 1e-13)


# ---------------------------------------------------------------------------
# general X (Algorithm 2, step 4): rows of X against its columns
# ---------------------------------------------------------------------------
def _dyadic_gen(n, bits, seed, row_exp=None, col_exp=None):
    """General X = D_r M D_c / 2^bits with integer M, |M| < 2^bits."""
    g = np.random.default_rng(seed)
    X = g.integers(-(2 ** bits) + 1, 2 ** bits, size=(n, n)).astype(np.float64) / 2.0 ** bits
    if row_exp is not None:
        X = (2.0 ** row_exp)[:, None] * X
    if col_exp is not None:
        X = X * (2.0 ** col_exp)[None, :]
    return X


@pytest.mark.parametrize("n,bits", [(300, 10), (513, 10), (1000, 12), (2200, 12)])
def test_gen_split_residual_bit_exact_on_dyadic_inputs(n, bits):
    # every product and partial sum of X X is exact in FP64 and the digit
    # slices hold every entry of a row (scaled by its row power of two; the
    # column scalings 1 or 2 add one bit) and of a column exactly, so no
    # digit pair is left out: the split residual equals the exact one, as
    # does the FP64 CUDA-core product.  n = 2200 has more 256 x 128 output
    # tiles than SMs
    g = np.random.default_rng(n + 5)
    X = _dyadic_gen(n, bits, seed=n, row_exp=g.integers(0, 2, size=n), col_exp=g.integers(0, 2, size=n))
    A = X @ X + _dyadic_gen(n, 8, seed=n + 1) / 2.0 ** 12
    R = A - X @ X  # exact
    Ad, Xd = dev_cm(A, torch.float64), dev_cm(X, torch.float64)
    Rs, ns = mp.step_residual_split(Ad, Xd, n, e=0)
    assert np.array_equal(host_cm(Rs, n), R.astype(np.float32))
    assert ns == pytest.approx(np.linalg.norm(R), rel=1e-14)
    Rf, nf = mp.step_residual(Ad, Xd, n, e=0)
    assert np.array_equal(host_cm(Rf, n), R.astype(np.float32))


@pytest.mark.parametrize("n", [256, 777, 2048])
def test_gen_split_residual_within_fp64_bound(n):
    # the refinement's cancellation regime for a nonsymmetric iterate:
    # A = X X + E, E ~ 1e-13, against the oracle's FP64 residual
    g = np.random.default_rng(11 + n)
    X = g.standard_normal((n, n)) / np.sqrt(n) + 2.0 * np.eye(n)
    A = X @ X + g.standard_normal((n, n)) * 1e-13
    e = 1
    R_ref = oracle.residual(A, X)[0] * 4.0 ** -e
    absXX = np.abs(X) @ np.abs(X) * 4.0 ** -e
    Ad, Xd = dev_cm(A, torch.float64), dev_cm(X, torch.float64)
    Rs, ns = mp.step_residual_split(Ad, Xd, n, e=e)
    Rs = host_cm(Rs, n).astype(np.float64)
    # the split residual and the oracle's each differ from the exact one by
    # at most about n u (|X| |X|)_ij, plus the FP32 rounding of Rhat
    bound = 2 * n * U64 * absXX + 2.0 ** -24 * np.abs(R_ref)
    assert np.all(np.abs(Rs - R_ref) <= 2 * bound)
    assert ns == pytest.approx(np.linalg.norm(R_ref), rel=1e-3)


def test_gen_split_residual_rejects_bad_arguments():
    Ad = dev_cm(np.eye(8), torch.float64)
    Rh = torch.empty(64, dtype=torch.float32, device="cuda")
    # lda < n is argument 3, ldx < n argument 5, n < 0 argument 6
    assert mp.lib().sqrtm_step_residual_split(mp.handle(), mp._ptr(Ad), 4, mp._ptr(Ad), 8, 8, 0, mp._ptr(Rh), None) == -3
    assert mp.lib().sqrtm_step_residual_split(mp.handle(), mp._ptr(Ad), 8, mp._ptr(Ad), 4, 8, 0, mp._ptr(Rh), None) == -5
    assert mp.lib().sqrtm_step_residual_split(mp.handle(), mp._ptr(Ad), 8, mp._ptr(Ad), 8, -1, 0, mp._ptr(Rh), None) == -6


def test_general_path_split_and_fp64_residuals_agree():
    # the general square root at n = 512 with the split residual (the
    # default from n = 512) and with FP64 products: both within the 1e-12
    # target of the oracle, and within rounding of each other
    A = synth.config_general512()
    At = torch.from_numpy(A).cuda()
    X1, i1 = mp.sqrtm_mixed(At, kind=mp.KIND_GENERAL, steps=2)
    X2, i2 = mp.sqrtm_mixed(At, kind=mp.KIND_GENERAL, steps=2, precision=mp.PREC_RESID_FP64)
    assert i1["status"] == 0 and i2["status"] == 0
    Xo = oracle.sqrtm_schur(A)
    X1, X2 = X1.cpu().numpy(), X2.cpu().numpy()
    assert oracle.rel_err(X1, Xo) <= 1e-12 and oracle.rel_err(X2, Xo) <= 1e-12
    assert oracle.rel_err(X1, X2) <= 1e-13
