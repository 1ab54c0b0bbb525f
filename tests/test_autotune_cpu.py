"""The autotuner's choice logic (pure functions: measurements in, tuning
table out), without a GPU."""
import math

from paper_2607_12430_gb300 import autotune as at


def test_pick_fastest_and_ties():
    assert at.pick_fastest({8: 3.0, 16: 2.0, 32: 2.5}) == 16
    # within 1 %: the first listed wins
    assert at.pick_fastest({32: 1.000, 16: 0.995}) == 32
    assert at.pick_fastest({32: 1.0, 16: 0.95}) == 16


def test_pick_precision_respects_accuracy_gate():
    times = {0: 2.0, 1: 1.0}
    assert at.pick_precision(times, {0: 1e-15, 1: 1e-14}) == 1
    assert at.pick_precision(times, {0: 1e-15, 1: 1e-12}) == 0
    assert at.pick_precision(times, {0: math.inf, 1: math.inf}) == 0
    # neither reaches the target: the faster plan if no worse than 1.5x FP32's
    assert at.pick_precision(times, {0: 7.4e-13, 1: 7.3e-13}) == 1
    assert at.pick_precision(times, {0: 7.4e-13, 1: 2e-12}) == 0


def test_build_table_orders_buckets_and_fills_builtins():
    measured = [
        {"n": 512, "blks": {8: 3.0, 16: 2.0, 32: 2.1}, "helpers": {0: 5.0, 8: 3.0, 16: 3.5},
         "cutoff": {0: 2.0, 256: 1.5},
         "spd": {0: 1.0, 1: 0.8}, "spd_err": {0: 1e-15, 1: 2e-15}, "batched": 0.5, "per_matrix": 0.4},
        {"n": 64, "blks": {8: 1.0, 16: 1.0, 32: 1.0}, "helpers": {}, "spd": {}, "spd_err": {},
         "batched": 0.1, "per_matrix": 0.9, "batched_spectral": 0.3, "batched_schur": 0.2},
        {"n": 4096, "blks": {}, "helpers": {}, "spd": {}, "spd_err": {}},
    ]
    t = at.build_table(measured)
    assert [e["n_max"] for e in t] == [64, 512, 4096]
    assert t[0] == {"n_max": 64, "blks": 8, "qr_helpers": -1, "spd_precision": 0, "batched": 1, "trisqrt_cutoff": 0,
                    "batched_spd": 0}
    assert t[1] == {"n_max": 512, "blks": 16, "qr_helpers": 8, "spd_precision": 1, "batched": 0,
                    "trisqrt_cutoff": 256, "batched_spd": 1}
    assert t[2] == {"n_max": 4096, "blks": 32, "qr_helpers": -1, "spd_precision": 0, "batched": 0,
                    "trisqrt_cutoff": 0, "batched_spd": 1}


def test_shipped_tables_are_valid():
    import json
    import os
    d = os.path.join(os.path.dirname(at.__file__), "tuning")
    if not os.path.isdir(d):
        return
    for f in os.listdir(d):
        if not f.endswith(".json"):
            continue
        res = json.load(open(os.path.join(d, f)))
        t = res["table"]
        assert isinstance(res["device"], str) and 0 < len(t) <= 32
        assert all(a["n_max"] < b["n_max"] for a, b in zip(t, t[1:]))
        for e in t:
            assert 1 <= e["blks"] <= 32 and -1 <= e["qr_helpers"] <= 24
            assert e["batched"] in (0, 1) and 0 <= e["spd_precision"] <= 3
            assert e.get("trisqrt_cutoff", 0) == 0 or e["trisqrt_cutoff"] >= 64
