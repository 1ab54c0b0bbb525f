"""The allocation-free residual entry point (for callers that cannot allocate
device memory, e.g. while a stream is being captured or inside another
library's fixed memory budget) must return what the regular residual entry
point returns.  Two calls in a row share the library's fixed scratch array, so
the second call also checks that nothing left over from the first leaks into
its result.  Collected last (file name) so that a failure here cannot hide
other tests when pytest stops at the first failure."""
import ctypes

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


def _case(n, seed):
    X = synth.gaussian((n, n), seed=seed)
    A = X @ X + 1e-6 * synth.gaussian((n, n), seed=seed + 1)
    return dev_cm(A, torch.float64), dev_cm(X, torch.float64)


def test_residual_noalloc_matches_regular_entry_point_twice():
    # two different problems back to back: the second must not see the first's scratch
    for n, e, seed in [(300, 1, 11), (129, 0, 12)]:
        A, X = _case(n, seed)
        R_ref, nrm_ref = mp.step_residual(A, X, n, e=e)
        out = torch.empty(n * n, dtype=torch.float32, device="cuda")
        R, nrm = mp.step_residual_noalloc(A, X, n, e=e, out=out)
        torch.cuda.synchronize()
        # same kernels, same inputs: identical FP32 output, norm within the
        # FP64 rounding of a different summation order at most
        assert torch.equal(R, R_ref)
        assert nrm == pytest.approx(nrm_ref, rel=1e-12)
        # and the oracle's FP64 residual A - X^2, element by element: each
        # entry within the FP32 rounding of R plus the FP64 error of the
        # n-term products
        Ah, Xh = host_cm(A, n), host_cm(X, n)
        Ro, nrm_o = oracle.residual(Ah, Xh)
        Ro *= 4.0 ** -e
        err = np.abs(host_cm(R, n).astype(np.float64) - Ro)
        bound = np.abs(Ro) * U32 + 4 * n * U64 * (np.abs(Xh) @ np.abs(Xh)) * 4.0 ** -e
        assert np.all(err <= bound)
        assert nrm == pytest.approx(nrm_o * 4.0 ** -e, rel=1e-6)


def test_residual_noalloc_rejects_too_large():
    n = 4097
    A = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(mp.SqrtmError) as e:
        mp.step_residual_noalloc(A, A, n, out=torch.zeros(1, dtype=torch.float32, device="cuda"))
    assert e.value.code == -5


def test_residual_noalloc_null_arguments():
    # a NULL matrix pointer reports its own argument position (dA 1, dX 3,
    # dRhat 7); nothing is launched
    L = mp.lib()
    n = 8
    buf = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    out = torch.zeros(n * n, dtype=torch.float32, device="cuda")
    null = ctypes.c_void_p(0)
    p = ctypes.c_void_p(buf.data_ptr())
    q = ctypes.c_void_p(out.data_ptr())
    st = mp._stream_ptr()
    assert L.sqrtm_step_residual_noalloc(null, n, p, n, n, 0, q, None, st) == -1
    assert L.sqrtm_step_residual_noalloc(p, n, null, n, n, 0, q, None, st) == -3
    assert L.sqrtm_step_residual_noalloc(p, n, p, n, n, 0, null, None, st) == -7
