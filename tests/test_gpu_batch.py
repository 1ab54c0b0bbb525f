"""GPU tests of the batched entry point on the batch workload's distribution
(sizes uniform in [16, 256], half SPD with lambda in [1e-2, 1e2], half
2I + G/sqrt(n)), against the FP64 oracle on every matrix of a sample."""
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


def _reference(item):
    kind, A, V, lam = item
    if kind == "spd":
        return oracle.sqrtm_from_eig(V, lam)
    return oracle.sqrtm_schur(A)


def test_batched_matches_oracle():
    items = synth.batch_case(count=24, seed=synth.BASE_SEED + 3)
    As = [torch.from_numpy(it[1]).cuda() for it in items]
    Xs, st = mp.sqrtm_mixed_batched(As, steps=4)
    assert st == [0] * len(items), (st, mp.last_error())
    for it, X in zip(items, Xs):
        Xo = _reference(it)
        tol = 1e-13 if it[0] == "spd" else 1e-12
        assert oracle.rel_err(X.cpu().numpy(), Xo) <= tol, (it[0], it[1].shape)


def test_batched_default_tolerance_and_status():
    items = synth.batch_case(count=8, seed=77)
    As = [torch.from_numpy(it[1]).cuda() for it in items]
    bad = torch.from_numpy(np.diag([1.0, -1.0, 2.0])).cuda()  # eigenvalue -1
    Xs, st = mp.sqrtm_mixed_batched(As + [bad])
    assert st[:-1] == [0] * len(items)
    assert st[-1] == 2
    for it, X in zip(items, Xs):
        assert oracle.rel_residual(X.cpu().numpy(), it[1]) <= 1e-12
