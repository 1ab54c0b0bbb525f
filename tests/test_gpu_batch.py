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


def test_batched_mixed_sizes_and_failures():
    # matrices above the batched size limit go through per-matrix calls, the
    # rest through the batched path; failures stay per matrix
    import os
    g = np.random.default_rng(5)
    items = synth.batch_case(count=10, seed=91)
    As = [it[1] for it in items]
    As += [synth.shifted_gaussian(300, 3.0, seed=92), synth.shifted_gaussian(1, 3.0, seed=93),
           synth.shifted_gaussian(2, 3.0, seed=94)]
    nan = synth.shifted_gaussian(20, 3.0, seed=95)
    nan[3, 4] = np.nan
    zero = np.zeros((7, 7))
    tens = [torch.from_numpy(np.ascontiguousarray(A)).cuda() for A in As]
    tens += [torch.from_numpy(nan).cuda(), torch.from_numpy(zero).cuda()]
    Xs, st = mp.sqrtm_mixed_batched(tens)
    assert st[:len(As)] == [0] * len(As), st
    assert st[len(As):] == [5, 2]
    for A, X in zip(As, Xs):
        assert oracle.rel_err(X.cpu().numpy(), oracle.sqrtm_schur(A)) <= 1e-12


@pytest.mark.parametrize("steps", [0, 1, 3])
def test_batched_fixed_steps_match_single(steps):
    # the batched path applies the same corrections as sqrtm_mixed's general
    # path: after k corrections both are within FP32 rounding differences of
    # each other (k = 0) or at the same FP64 accuracy (k >= 3)
    items = synth.batch_case(count=6, seed=96)
    As = [torch.from_numpy(it[1]).cuda() for it in items]
    Xs, st = mp.sqrtm_mixed_batched(As, steps=steps)
    assert st == [0] * len(As)
    for it, A, X in zip(items, As, Xs):
        X1, _ = mp.sqrtm_mixed(A, kind=mp.KIND_GENERAL, steps=steps)
        Xo = _reference(it)
        e_b = oracle.rel_err(X.cpu().numpy(), Xo)
        e_1 = oracle.rel_err(X1.cpu().numpy(), Xo)
        if steps == 0:
            assert e_b <= 1e-5 and e_1 <= 1e-5
        elif steps == 1:
            assert e_b <= 1e-9 and e_1 <= 1e-9
        else:
            assert e_b <= 1e-13 and e_1 <= 1e-13


def test_batched_iteration_limit_status():
    # maxit = 0 allows one correction: the FP32 start plus one step stays
    # above tol = 1e-15, so every matrix returns status 1
    items = synth.batch_case(count=4, seed=97)
    As = [torch.from_numpy(it[1]).cuda() for it in items]
    _, st = mp.sqrtm_mixed_batched(As, tol=1e-15, maxit=0)
    assert st == [1] * len(As)


def test_sharded_batch_single_rank_matches_batched_call(tmp_path):
    """The multi-GPU batch call with one rank (a gloo process group on a file
    store): the LPT share is the whole batch, solved by sqrtm_mixed_batched
    on this GPU, and the statuses come back in input order."""
    import torch.distributed as dist
    items = synth.batch_case(count=12, seed=synth.BASE_SEED + 31)
    host = [torch.from_numpy(np.ascontiguousarray(it[1])) for it in items]
    dist.init_process_group("gloo", init_method="file://" + str(tmp_path / "pg"), rank=0, world_size=1)
    try:
        out, st = mp.sqrtm_mixed_batched_sharded(host, steps=4)
    finally:
        dist.destroy_process_group()
    assert st == [0] * len(items)
    assert sorted(out) == list(range(len(items)))
    for i, it in enumerate(items):
        tol = 1e-13 if it[0] == "spd" else 1e-12
        assert oracle.rel_err(out[i].cpu().numpy(), _reference(it)) <= tol
