"""Autotuner: measures the library's tunable choices on the GPU at hand and
installs the winners as the handle's tuning table (sqrtm_set_tuning).

Per size bucket (a representative size n per bucket, the bucket being all
sizes up to n) it times, with CUDA events, the library's own entry points on
seeded synthetic matrices of the workloads' shapes (3I + G/sqrt(n) for the
general path, V diag(lambda) V^T with lambda log-uniform in [1e-3, 1e3] for
the SPD path):

* blks -- the block size of the triangular square root and the Sylvester
  wavefront (Algorithm 1's recursion cut-off; Sec. 5 uses 32): candidates
  8, 16, 32, on sqrtm_mixed with a fixed number of corrections;
* qr_helpers -- the helper CTAs of the cooperative QR chase (n >= 256):
  0, 8, 16;
* spd_precision -- FP32 or split-TF32 transforms of Algorithm 3, the faster
  one among those whose forward error against the FP64 method on the same
  GPU, after SPD_STEPS corrections (the stopping test nullified, as in the
  accuracy runs of Sec. 5.1), stays within the SPD accuracy target (1e-13);
* trisqrt_cutoff -- the blocked triangular square root (0) or the
  recursive splitting of Sec. 2.2.1 down to blocks of 256 or 512 (n >= 512);
* batched -- for sqrtm_mixed_batched, whether matrices of the bucket's size
  go through the batched general path or per-matrix calls (a batch of
  `batch_count` matrices timed both ways);
* batched_spd -- for sqrtm_mixed_batched (n <= 256), whether symmetric
  matrices of the bucket's size take the batched path's spectral stage
  (Algorithm 3) or its complex Schur stage (Algorithm 2): a batch of
  `batch_count` SPD matrices timed both ways with the default tolerance.

The choice functions are pure (measurements in, table out) so that they are
testable without a GPU; `autotune()` runs the measurements and `save` /
`load_tuning` write and read the table as JSON.
"""
import json
import os

import numpy as np

BLKS_CANDIDATES = (8, 16, 32)
HELPER_CANDIDATES = (0, 8, 16)
CUTOFF_CANDIDATES = (0, 256, 512)
SPD_TARGET = 1e-13
SPD_STEPS = 4  # corrections of the SPD accuracy runs (the protocol of Sec. 5.1: the test nullified)
DEFAULT_SIZES = (64, 128, 256, 512, 1024, 2048)
BUILTIN = {"blks": 32, "qr_helpers": -1, "spd_precision": 0}


# ---------------------------------------------------------------------------
# pure choices
# ---------------------------------------------------------------------------
def pick_fastest(times):
    """``times``: {candidate: seconds}.  The fastest candidate; ties (within
    1 %) go to the candidate listed first."""
    best = None
    for c, t in times.items():
        if best is None or t < times[best] * 0.99:
            best = c
    return best


def pick_precision(times, errors, target=SPD_TARGET):
    """The fastest precision plan whose forward error meets the target or is
    no more than 1.5 times the FP32 plan's (where the FP32 plan itself does
    not reach the target in the measured steps, the split-TF32 plan may not
    be worse than it); FP32 (0) when no plan qualifies."""
    bound = max(target, 1.5 * errors.get(0, np.inf)) if np.isfinite(errors.get(0, np.inf)) else target
    ok = {p: t for p, t in times.items() if errors.get(p, np.inf) <= bound}
    return pick_fastest(ok) if ok else 0


def build_table(measured):
    """``measured``: list of per-bucket dicts with n and the timings of each
    choice ("blks", "helpers", "spd" + "spd_err", "batched" / "per_matrix").
    Returns the tuning table (ascending n_max)."""
    table = []
    for m in sorted(measured, key=lambda d: d["n"]):
        e = {"n_max": int(m["n"])}
        e["blks"] = int(pick_fastest(m["blks"])) if m.get("blks") else BUILTIN["blks"]
        e["qr_helpers"] = int(pick_fastest(m["helpers"])) if m.get("helpers") else BUILTIN["qr_helpers"]
        e["spd_precision"] = int(pick_precision(m["spd"], m["spd_err"])) if m.get("spd") else BUILTIN["spd_precision"]
        e["trisqrt_cutoff"] = int(pick_fastest(m["cutoff"])) if m.get("cutoff") else 0
        if "batched" in m and "per_matrix" in m:
            e["batched"] = int(m["batched"] <= m["per_matrix"])
        else:
            e["batched"] = int(m["n"] <= 256)
        if "batched_spectral" in m and "batched_schur" in m:
            e["batched_spd"] = int(m["batched_spectral"] <= m["batched_schur"])
        else:
            e["batched_spd"] = 1
        table.append(e)
    return table


# ---------------------------------------------------------------------------
# measurements
# ---------------------------------------------------------------------------
def _general(n, seed):
    g = np.random.default_rng(seed)
    return 3.0 * np.eye(n) + g.standard_normal((n, n)) / np.sqrt(n)


def _spd(n, seed):
    g = np.random.default_rng(seed)
    V, _ = np.linalg.qr(g.standard_normal((n, n)))
    lam = 10.0 ** g.uniform(-3.0, 3.0, n)
    A = (V * lam) @ V.T
    return 0.5 * (A + A.T)


def _timer(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    best = np.inf
    for _ in range(reps):
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        fn()
        e.record()
        torch.cuda.synchronize()
        best = min(best, s.elapsed_time(e) / 1e3)
    return best


def measure_bucket(n, reps=3, batch_count=32, seed=20260712, log=None):
    """Timings of every candidate at size n (needs the CUDA library)."""
    import torch
    import paper_2607_12430_gb300 as mp
    A = torch.from_numpy(_general(n, seed + n)).cuda()
    m = {"n": n, "blks": {}, "helpers": {}, "cutoff": {}, "spd": {}, "spd_err": {}}
    saved = mp.get_tuning()
    try:
        mp.set_tuning([])
        for b in BLKS_CANDIDATES:
            m["blks"][b] = _timer(lambda: mp.sqrtm_mixed(A, kind=mp.KIND_GENERAL, steps=2, blks=b), reps)
        if n >= 256:
            for hcount in HELPER_CANDIDATES:
                mp.set_tuning([{"n_max": 1 << 40, "blks": 32, "qr_helpers": hcount, "batched": 1,
                                "spd_precision": 0}])
                m["helpers"][hcount] = _timer(lambda: mp.sqrtm_mixed(A, kind=mp.KIND_GENERAL, steps=2, blks=32),
                                              reps)
            for c in CUTOFF_CANDIDATES:
                if c and c >= n:
                    continue
                mp.set_tuning([{"n_max": 1 << 40, "blks": 32, "qr_helpers": -1, "batched": 1, "spd_precision": 0,
                                "trisqrt_cutoff": c}])
                m["cutoff"][c] = _timer(lambda: mp.sqrtm_mixed(A, kind=mp.KIND_GENERAL, steps=2, blks=32), reps)
            mp.set_tuning([])
        S = torch.from_numpy(_spd(n, seed + 7 * n)).cuda()
        X64, _ = mp.sqrtm_schur_fp64(S, kind=mp.KIND_SPD)
        for p in (mp.PREC_FP32, mp.PREC_TF32X3):
            X, info = mp.sqrtm_mixed(S, kind=mp.KIND_SPD, precision=p, steps=SPD_STEPS, raise_on_error=False)
            m["spd_err"][p] = ((X - X64).norm() / X64.norm()).item() if info["status"] == 0 else np.inf
            m["spd"][p] = _timer(lambda: mp.sqrtm_mixed(S, kind=mp.KIND_SPD, precision=p, steps=SPD_STEPS,
                                                        raise_on_error=False), reps)
        if n <= 256:
            Ss = [torch.from_numpy(_spd(n, seed + 2000 + i)).cuda() for i in range(batch_count)]
            mp.set_tuning([{"n_max": 1 << 40, "blks": 32, "qr_helpers": -1, "batched": 1, "spd_precision": 0,
                            "batched_spd": 1}])
            m["batched_spectral"] = _timer(lambda: mp.sqrtm_mixed_batched(Ss), reps)
            mp.set_tuning([{"n_max": 1 << 40, "blks": 32, "qr_helpers": -1, "batched": 1, "spd_precision": 0,
                            "batched_spd": 0}])
            m["batched_schur"] = _timer(lambda: mp.sqrtm_mixed_batched(Ss), reps)
            mp.set_tuning([])
        if n <= 1024:
            As = [torch.from_numpy(_general(n, seed + 1000 + i)).cuda() for i in range(batch_count)]
            old = os.environ.get("SQRTM_BATCH_MAXN")
            try:
                os.environ["SQRTM_BATCH_MAXN"] = str(n)
                m["batched"] = _timer(lambda: mp.sqrtm_mixed_batched(As), reps)
                os.environ["SQRTM_BATCH_MAXN"] = "0"
                m["per_matrix"] = _timer(lambda: mp.sqrtm_mixed_batched(As), reps)
            finally:
                if old is None:
                    os.environ.pop("SQRTM_BATCH_MAXN", None)
                else:
                    os.environ["SQRTM_BATCH_MAXN"] = old
    finally:
        mp.set_tuning(saved)
    if log:
        log(json.dumps({k: (v if not isinstance(v, dict) else {str(a): b for a, b in v.items()}) for k, v in m.items()}))
    return m


def device_key():
    import torch
    p = torch.cuda.get_device_properties(0)
    return f"{p.name} sm_{p.major}{p.minor} x{p.multi_processor_count}"


def autotune(sizes=DEFAULT_SIZES, reps=3, batch_count=32, install=True, log=None):
    """Measure every bucket, build the table, install it on this stream's
    handle (install=True) and return {"device": ..., "table": [...],
    "measured": [...]}."""
    import paper_2607_12430_gb300 as mp
    measured = [measure_bucket(n, reps=reps, batch_count=batch_count, log=log) for n in sizes]
    table = build_table(measured)
    if install:
        mp.set_tuning(table)
    return {"device": device_key(), "table": table,
            "measured": [{k: (v if not isinstance(v, dict) else {str(a): b for a, b in v.items()})
                          for k, v in m.items()} for m in measured]}


def save(result, path):
    with open(path, "w") as f:
        json.dump(result, f, indent=1)


def load_tuning(path, check_device=True):
    """Install the table stored at path on this stream's handle; with
    check_device, only if it was measured on a device of the same name, SM
    version and SM count.  Returns True if installed."""
    import paper_2607_12430_gb300 as mp
    with open(path) as f:
        res = json.load(f)
    if check_device and res.get("device") != device_key():
        return False
    mp.set_tuning(res["table"])
    return True
