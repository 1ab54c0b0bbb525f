"""GPU tests of the split-TF32 tcgen05 products used for the low-precision
transforms (Algorithm 3, steps 8 and 10; Algorithm 2, steps 3, 8 and 10 in
complex arithmetic), against the FP64 product of the same FP32 inputs, and of
both refinements with their transforms on the tensor cores against the
oracle."""
import numpy as np
import pytest
import torch

import synth
from gpu_util import check_kstar

pytestmark = pytest.mark.gpu

mp = pytest.importorskip("paper_2607_12430_gb300")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    mp.lib()


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (128, 128, 96), (256, 384, 512), (200, 136, 100),
                                   (1024, 1024, 1024)])
def test_gemm_tf32x3(M, N, K):
    g = np.random.default_rng(M * 7 + N * 3 + K)
    A = g.standard_normal((M, K)).astype(np.float32)
    B = g.standard_normal((K, N)).astype(np.float32)
    a_rows = torch.from_numpy(np.ascontiguousarray(A)).cuda().reshape(-1)      # row i contiguous
    b_cols = torch.from_numpy(np.ascontiguousarray(B.T)).cuda().reshape(-1)    # column j contiguous
    C = mp.step_gemm_tf32x3(a_rows, b_cols, M, N, K).cpu().numpy().reshape((M, N), order="F")
    Cref = A.astype(np.float64) @ B.astype(np.float64)
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64)
    err = np.abs(C - Cref)
    # split-TF32 with FP32 accumulation: a few 2^-22 relative per term plus
    # the FP32 sum over K
    assert np.all(err <= (8 * 2.0 ** -22 + K * 2.0 ** -24) * scale)
    # and clearly better than a single TF32 product would be (2^-11)
    assert np.max(err / scale) < 2.0 ** -16


def test_spd_refinement_tf32x3_matches_oracle():
    """The SPD refinement with its transforms on the tensor cores reaches the
    same accuracy as the FP32 CUDA-core transforms."""
    import oracle
    n = 512
    A, V, lam = synth.spd_case(n, -3.0, 3.0, seed=900, force_ends=True)
    Xo = oracle.sqrtm_from_eig(V, lam)
    Xg = oracle.refine(A, V, np.diag(np.sqrt(lam)), Xo, steps=1, spd=True)[-1]
    errs = []
    for k in range(1, 8):
        X, info = mp.sqrtm_mixed(torch.from_numpy(A).cuda(), steps=k, precision=mp.PREC_TF32X3)
        X = X.cpu().numpy()
        assert np.array_equal(X, X.T)
        errs.append(oracle.rel_err(X, Xg))
    check_kstar(errs, 1e-13)


@pytest.mark.parametrize("M,N,K,ca,cy", [(128, 128, 64, False, False), (128, 200, 128, True, False),
                                          (200, 136, 100, False, True), (130, 130, 130, True, True),
                                          (512, 512, 512, True, False)])
def test_cgemm_tf32x3(M, N, K, ca, cy):
    """The complex product as one real split-TF32 product over interleaved
    operands (Algorithm 2's transforms): every entry within the split-TF32
    error of the FP64 product of the same FP32 inputs."""
    g = np.random.default_rng(M * 11 + N * 5 + K + 2 * ca + cy)
    A = (g.standard_normal((M, K)) + 1j * g.standard_normal((M, K))).astype(np.complex64)
    Y = (g.standard_normal((K, N)) + 1j * g.standard_normal((K, N))).astype(np.complex64)
    a_rows = torch.from_numpy(np.ascontiguousarray(A)).cuda().reshape(-1)
    y_cm = torch.from_numpy(np.ascontiguousarray(Y.T)).cuda().reshape(-1)
    C = mp.step_cgemm_tf32x3(a_rows, y_cm, M, N, K, conj_a=ca, conj_y=cy).cpu().numpy().reshape((M, N), order="F")
    Ad = A.astype(np.complex128)
    Yd = Y.astype(np.complex128)
    Cref = (Ad.conj() if ca else Ad) @ (Yd.conj() if cy else Yd)
    # each of Re, Im sums 2K real products of moduli at most |a| |y|
    scale = 2.0 * (np.abs(Ad) @ np.abs(Yd))
    err = np.abs(C - Cref)
    assert np.all(err <= (8 * 2.0 ** -22 + 2 * K * 2.0 ** -24) * scale)
    assert np.max(err / scale) < 2.0 ** -16


@pytest.mark.parametrize("n", [128, 130, 512, 1024])
def test_general_refinement_tf32x3_matches_oracle(n):
    """Algorithm 2 with X_0 and the transforms as split-TF32 tensor-core
    products: 1e-12 against the FP64 oracle within 3 corrections (the
    workload's 2 to 4), no growth after."""
    import oracle
    A = synth.shifted_gaussian(n, 3.0, seed=910 + n) if n != 512 else synth.config_general512()
    Xo = oracle.sqrtm_schur(A)
    errs = []
    for k in range(0, 5):
        X, info = mp.sqrtm_mixed(torch.from_numpy(A).cuda(), kind=mp.KIND_GENERAL, steps=k,
                                 precision=mp.PREC_TF32X3_GENERAL)
        assert info["status"] == 0
        errs.append(oracle.rel_err(X.cpu().numpy(), Xo))
    assert errs[0] <= 1e-4  # X_0: FP32 Schur factors, product accumulated in FP32
    assert check_kstar(errs, 1e-12) <= 3, errs


def test_general_tf32x3_odd_size_falls_back():
    """Odd n breaks the operands' 16-byte row alignment: the CUDA-core
    products are used instead, with the same result accuracy."""
    import oracle
    n = 129
    A = synth.shifted_gaussian(n, 3.0, seed=920)
    X, info = mp.sqrtm_mixed(torch.from_numpy(A).cuda(), kind=mp.KIND_GENERAL, steps=3,
                             precision=mp.PREC_TF32X3_GENERAL)
    assert info["status"] == 0
    assert oracle.rel_err(X.cpu().numpy(), oracle.sqrtm_schur(A)) <= 1e-12
