"""GPU tests of the batched entry point on the batch workload's distribution
(sizes uniform in [16, 256], half SPD with lambda in [1e-2, 1e2], half
2I + G/sqrt(n)), against the FP64 oracle on every matrix of a sample."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import check_kstar

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


class _Table:
    """A tuning table for the duration of a test: batched_spd = 1 sends the
    symmetric members through the spectral stage (Algorithm 3), 0 through
    the complex Schur stage (Algorithm 2)."""

    def __init__(self, spectral):
        self.spectral = spectral

    def __enter__(self):
        self.saved = mp.get_tuning()
        mp.set_tuning([{"n_max": 1 << 20, "blks": 32, "qr_helpers": -1, "batched": 1, "spd_precision": 0,
                        "batched_spd": int(self.spectral)}])

    def __exit__(self, *a):
        mp.set_tuning(self.saved)


@pytest.mark.parametrize("spectral", [True, False])
def test_batched_matches_oracle(spectral):
    """Every member of a 64-matrix sample of the batch workload (one graph
    launch: the symmetric half through the Jacobi spectral stage of
    Algorithm 3 or through Algorithm 2, the rest through Algorithm 2),
    against the oracle: the closed form V diag(sqrt(lam)) V^T for the
    symmetric members (<= 1e-13, kappa <= 1e4), the FP64 Schur method for
    the others (<= 1e-12)."""
    items = synth.batch_case(count=64, seed=synth.BASE_SEED + 3)
    As = [torch.from_numpy(it[1]).cuda() for it in items]
    with _Table(spectral):
        Xs, st = mp.sqrtm_mixed_batched(As, steps=5)
        ph = mp.batched_phases()
    assert st == [0] * len(items), (st, mp.last_error())
    nsym = sum(1 for it in items if it[0] == "spd")
    assert ph["matrices"] == len(items)
    assert ph["general"] == (len(items) - nsym if spectral else len(items))
    for it, X in zip(items, Xs):
        Xo = _reference(it)
        tol = 1e-13 if it[0] == "spd" else 1e-12
        assert oracle.rel_err(X.cpu().numpy(), Xo) <= tol, (it[0], it[1].shape)


def test_batched_symmetric_members_forced_and_indefinite():
    """SQRTM_KIND_SPD sends every member through the spectral stage; a
    symmetric matrix with a negative eigenvalue has no real principal square
    root there either (status 2), and its neighbours are unaffected."""
    items = [it for it in synth.batch_case(count=12, seed=98) if it[0] == "spd"]
    As = [torch.from_numpy(np.ascontiguousarray(it[1])).cuda() for it in items]
    bad = synth.spd_case(40, -1.0, 1.0, seed=99)[0]
    bad = bad - 2.0 * np.eye(40) * np.linalg.eigvalsh(bad)[0]  # lowest eigenvalue now negative
    bad = 0.5 * (bad + bad.T)
    Xs, st = mp.sqrtm_mixed_batched(As + [torch.from_numpy(bad).cuda()], steps=5, kind=mp.KIND_SPD)
    assert st == [0] * len(As) + [2]
    for it, X in zip(items, Xs):
        assert oracle.rel_err(X.cpu().numpy(), _reference(it)) <= 1e-13


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
        X = X.cpu().numpy()
        Xo = oracle.sqrtm_schur(A)
        # the default stopping test is the paper's relative residual test
        # (tol = 1e-12), and it certifies the forward error only through the
        # condition of the square root: to first order ||dX|| <= ||L|| ||dA||
        # with the Frechet derivative L(E) solving X L + L X = E, so the
        # relative forward error is at most cond_rel * 1e-12 with
        # cond_rel = ||A|| / (||X|| sep(X, -X)); for symmetric A,
        # sep = 2 sqrt(lam_min) (kappa up to 1e4 here), for the shifted
        # Gaussians sep ~ 2 sqrt(2) and cond_rel ~ 1
        assert oracle.rel_residual(X, A) <= 1e-12
        if np.array_equal(A, A.T):
            cond = np.linalg.norm(A, 2) / (2 * np.sqrt(np.linalg.eigvalsh(A)[0]) * np.linalg.norm(Xo, 2))
        else:
            cond = 1.0
        assert oracle.rel_err(X, Xo) <= max(1.0, 2.0 * cond) * 1e-12


@pytest.mark.parametrize("steps", [0, 1, 3])
def test_batched_fixed_steps_match_single(steps):
    # for its general members the batched path applies the same corrections
    # as sqrtm_mixed's general path: after k corrections both are within
    # FP32 rounding differences of each other (k = 0) or at the same FP64
    # accuracy (k >= 3)
    items = synth.batch_case(count=6, seed=96)
    As = [torch.from_numpy(it[1]).cuda() for it in items]
    Xs, st = mp.sqrtm_mixed_batched(As, steps=steps)
    assert st == [0] * len(As)
    for it, A, X in zip(items, As, Xs):
        if it[0] == "spd":
            continue
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


def test_batched_symmetric_members_contract_each_step():
    """Symmetric members take the FP32 Jacobi factors (Algorithm 3): each
    correction with these frozen factors multiplies the forward error by
    about their backward error (FP32 rotations: a few 1e-4 at n ~ 250), so
    the error falls by at least 100x per step until the FP64 floor, reaching
    1e-13 within 5 corrections and staying there."""
    items = [it for it in synth.batch_case(count=16, seed=96) if it[0] == "spd"]
    As = [torch.from_numpy(np.ascontiguousarray(it[1])).cuda() for it in items]
    errs = []
    with _Table(True):
        for k in range(0, 7):
            Xs, st = mp.sqrtm_mixed_batched(As, steps=k)
            assert st == [0] * len(As)
            assert mp.batched_phases()["general"] == 0
            errs.append([oracle.rel_err(X.cpu().numpy(), _reference(it)) for it, X in zip(items, Xs)])
    for j in range(len(items)):
        e = [errs[k][j] for k in range(len(errs))]
        kstar = check_kstar(e, 1e-13)
        assert kstar <= 5, e
        assert all(e[k + 1] <= max(1e-2 * e[k], 1e-14) for k in range(kstar)), e  # 1e-14: the FP64 floor


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
