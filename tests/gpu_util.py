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
