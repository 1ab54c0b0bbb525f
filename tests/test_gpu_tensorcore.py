"""GPU tests of the split-TF32 tcgen05 product used for the low-precision
transforms (Algorithm 3, steps 8 and 10), against the FP64 product of the same
FP32 inputs."""
import numpy as np
import pytest
import torch

import synth

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
    for k in range(3, 8):
        X, info = mp.sqrtm_mixed(torch.from_numpy(A).cuda(), steps=k, precision=mp.PREC_TF32X3)
        X = X.cpu().numpy()
        assert np.array_equal(X, X.T)
        errs.append(oracle.rel_err(X, Xg))
    assert min(errs) <= 1e-13, errs
