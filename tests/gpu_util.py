"""Helpers for the GPU tests: column-major transfers between numpy and the
device (the C ABI is column-major)."""
import numpy as np
import torch


def dev_cm(M, dtype):
    """numpy matrix -> 1-D CUDA tensor holding it column-major."""
    a = np.asarray(M)
    flat = np.ascontiguousarray(a.ravel(order="F"))
    return torch.from_numpy(flat).to(dtype=dtype, device="cuda")


def host_cm(t, rows, cols=None):
    cols = rows if cols is None else cols
    return t.detach().cpu().numpy().reshape((rows, cols), order="F")


U32 = 2.0 ** -24
U64 = 2.0 ** -53


def check_kstar(errs, tol, decreasing=True):
    """errs[i]: forward error after the i-th of an increasing sequence of
    correction counts (stopping test nullified).  Returns k*, the first index
    with errs[k*] <= tol, after asserting that one exists, that the error
    falls strictly up to it (when `decreasing`), and that no later count
    takes the error back above tol (no growth once converged)."""
    ks = [i for i, e in enumerate(errs) if e <= tol]
    assert ks, f"never reached {tol}: {errs}"
    kstar = ks[0]
    if decreasing:
        assert all(errs[i + 1] < errs[i] for i in range(kstar)), errs
    assert all(e <= tol for e in errs[kstar:]), f"error grew back above {tol} after k* = {kstar}: {errs}"
    return kstar
