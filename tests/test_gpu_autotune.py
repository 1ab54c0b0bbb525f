"""GPU tests of the tuning table and the autotuner: validation of the table,
that a tuned choice acts like the same explicit option, and a short
autotuning run whose installed table leaves every result accurate."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

mp = pytest.importorskip("paper_2607_12430_gb300")


@pytest.fixture(autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    mp.lib()
    saved = mp.get_tuning()
    yield
    mp.set_tuning(saved)


def _entry(n_max, blks=32, helpers=-1, batched=1, prec=0, cutoff=0, batched_spd=1):
    return {"n_max": n_max, "blks": blks, "qr_helpers": helpers, "batched": batched, "spd_precision": prec,
            "trisqrt_cutoff": cutoff, "batched_spd": batched_spd}


@pytest.mark.parametrize("bad,code", [
    ([_entry(256), _entry(128)], -4),          # n_max not ascending
    ([_entry(256, blks=0)], -4),               # block size out of range
    ([_entry(256, helpers=25)], -4),
    ([_entry(256, batched=2)], -4),
    ([_entry(256, cutoff=-1)], -4),
    ([_entry(256, batched_spd=2)], -4),
    ([_entry(i + 1) for i in range(33)], -3),  # too many entries
])
def test_set_tuning_rejects(bad, code):
    with pytest.raises(mp.SqrtmError) as e:
        mp.set_tuning(bad)
    assert e.value.code == code


def test_tuning_round_trip():
    t = [_entry(128, blks=8), _entry(1024, blks=16, helpers=0, batched=0, prec=1, cutoff=256, batched_spd=0)]
    mp.set_tuning(t)
    assert mp.get_tuning() == t
    mp.set_tuning([])
    assert mp.get_tuning() == []


@pytest.mark.parametrize("n,blks,helpers", [(100, 8, -1), (300, 16, 0), (300, 32, 16)])
def test_tuned_choice_equals_explicit_option(n, blks, helpers):
    A = torch.from_numpy(synth.shifted_gaussian(n, 3.0, seed=600 + n)).cuda()
    mp.set_tuning([_entry(1 << 20, blks=blks, helpers=helpers)])
    Xt, it = mp.sqrtm_mixed(A, kind=mp.KIND_GENERAL, steps=2)
    Xe, ie = mp.sqrtm_mixed(A, kind=mp.KIND_GENERAL, steps=2, blks=blks)
    assert it["status"] == 0 and ie["status"] == 0
    assert ((Xt - Xe).norm() / Xe.norm()).item() <= 1e-15
    Xo = oracle.sqrtm_schur(A.cpu().numpy())
    assert oracle.rel_err(Xt.cpu().numpy(), Xo) <= 1e-12


def test_autotune_short_run_installs_accurate_table():
    from paper_2607_12430_gb300 import autotune
    res = autotune.autotune(sizes=(64, 256), reps=1, batch_count=4)
    t = mp.get_tuning()
    assert t == res["table"] and [e["n_max"] for e in t] == [64, 256]
    items = synth.batch_case(count=6, seed=601)
    As = [torch.from_numpy(it[1]).cuda() for it in items]
    Xs, st = mp.sqrtm_mixed_batched(As)
    assert st == [0] * len(As)
    for it, X in zip(items, Xs):
        assert oracle.rel_residual(X.cpu().numpy(), it[1]) <= 1e-12
    A = torch.from_numpy(synth.shifted_gaussian(200, 3.0, seed=602)).cuda()
    X, info = mp.sqrtm_mixed(A)
    assert info["status"] == 0
    assert oracle.rel_err(X.cpu().numpy(), oracle.sqrtm_schur(A.cpu().numpy())) <= 1e-12
