"""Seeded synthetic inputs shared by the tests, the oracle checks and the
benchmark.

This module draws random numbers and assembles test matrices; it holds none
of the square-root method's arithmetic.  Every generator takes an explicit
seed (numpy PCG64 through ``default_rng``) and returns FP64 column-major
(Fortran-ordered) arrays.

Workloads (sizes and distributions of the five benchmark configurations):

* ``spd_case(n, lo, hi)``: ``A = V diag(lam) V^T`` with ``V`` Haar-orthogonal
  (QR of an N(0,1) matrix with the signs of ``diag(R)`` made positive) and
  ``lam`` log-uniform in ``[10^lo, 10^hi]``; ``force_ends`` pins the extreme
  eigenvalues so the condition number is exactly ``10^(hi-lo)``.
* ``shifted_gaussian(n, shift)``: ``A = shift I + G / sqrt(n)``, ``G`` i.i.d.
  N(0,1): spectrum in a disc of radius about 1 around ``shift``.
* ``batch_case``: sizes uniform in ``[16, 256]``, even items SPD with
  ``lam`` log-uniform in ``[1e-2, 1e2]``, odd items ``2I + G/sqrt(n)``.
* ``table1_case``: the nonsymmetric/symmetric U(0,1) / N(0,1) matrices plus a
  shift, and the shifted Hilbert matrix, of the paper's Table 1 (the shift for
  the random sets is the bulk spectral radius plus one).
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20260712


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def haar_orthogonal(n: int, g: np.random.Generator) -> np.ndarray:
    Z = g.standard_normal((n, n))
    Q, R = np.linalg.qr(Z)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return np.asfortranarray(Q * d[None, :])


def log_uniform(n: int, lo: float, hi: float, g: np.random.Generator,
                force_ends: bool = False) -> np.ndarray:
    lam = 10.0 ** g.uniform(lo, hi, size=n)
    if force_ends and n >= 2:
        lam[0] = 10.0 ** lo
        lam[1] = 10.0 ** hi
    return lam


def spd_case(n: int, lo: float, hi: float, seed: int, force_ends: bool = False):
    """Returns (A, V, lam) with A = V diag(lam) V^T, symmetrised."""
    g = rng(seed)
    V = haar_orthogonal(n, g)
    lam = log_uniform(n, lo, hi, g, force_ends)
    A = (V * lam[None, :]) @ V.T
    A = 0.5 * (A + A.T)
    return np.asfortranarray(A), V, lam


def shifted_gaussian(n: int, shift: float, seed: int) -> np.ndarray:
    g = rng(seed)
    G = g.standard_normal((n, n))
    A = G / np.sqrt(n)
    A[np.diag_indices(n)] += shift
    return np.asfortranarray(A)


def gaussian(shape, seed: int) -> np.ndarray:
    return np.asfortranarray(rng(seed).standard_normal(shape))


def batch_sizes(count: int, seed: int, lo: int = 16, hi: int = 256) -> np.ndarray:
    return rng(seed).integers(lo, hi + 1, size=count)


def batch_case(count: int = 2048, seed: int = BASE_SEED + 3, lo: int = 16, hi: int = 256):
    """Returns a list of (kind, A, V, lam) with kind 'spd' or 'general'
    (V, lam are None for 'general')."""
    sizes = batch_sizes(count, seed, lo, hi)
    out = []
    for i, n in enumerate(sizes):
        if i % 2 == 0:
            A, V, lam = spd_case(int(n), -2.0, 2.0, seed * 7919 + i)
            out.append(("spd", A, V, lam))
        else:
            out.append(("general", shifted_gaussian(int(n), 2.0, seed * 7919 + i), None, None))
    return out


def random_upper_rhp(n: int, seed: int, offdiag_scale: float = 1.0,
                     re_lo: float = 0.5, re_hi: float = 2.0) -> np.ndarray:
    """Complex upper triangular matrix with diagonal in the right half plane
    (Re in [re_lo, re_hi], Im in [-1, 1]) and N(0,1)/sqrt(n) above it: a
    stand-in for a triangular square root factor."""
    g = rng(seed)
    S = (g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))) * (offdiag_scale / np.sqrt(max(n, 1)))
    S = np.triu(S, 1)
    S[np.diag_indices(n)] = g.uniform(re_lo, re_hi, size=n) + 1j * g.uniform(-1.0, 1.0, size=n)
    return np.asfortranarray(S)


def random_quasi_upper(n: int, seed: int, pair_frac: float = 0.5) -> np.ndarray:
    """Real quasi-upper-triangular matrix (a stand-in for a real Schur factor):
    diagonal blocks 1x1 with entries in [0.5, 2], or 2x2 [[t, m r], [-m / r, t]]
    with t in [0.5, 2], m in [0.2, 1], r in [0.5, 2] (eigenvalues t +- i m, in
    the right half plane), about pair_frac of the rows in 2x2 blocks; N(0,1)/sqrt(n)
    above the blocks."""
    g = rng(seed)
    T = np.triu(g.standard_normal((n, n)) / np.sqrt(max(n, 1)), 1)
    i = 0
    while i < n:
        if i + 1 < n and g.uniform() < pair_frac:
            t, m, r = g.uniform(0.5, 2.0), g.uniform(0.2, 1.0), g.uniform(0.5, 2.0)
            T[i, i] = T[i + 1, i + 1] = t
            T[i, i + 1] = m * r
            T[i + 1, i] = -m / r
            i += 2
        else:
            T[i, i] = g.uniform(0.5, 2.0)
            i += 1
    return np.asfortranarray(T)


def random_unitary(n: int, seed: int) -> np.ndarray:
    g = rng(seed)
    Z = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    Q, R = np.linalg.qr(Z)
    d = np.diag(R)
    d = d / np.abs(d)
    return np.asfortranarray(Q * d[None, :])


def hilbert(n: int) -> np.ndarray:
    i = np.arange(n)
    return np.asfortranarray(1.0 / (i[:, None] + i[None, :] + 1.0))


def table1_case(set_id: str, n: int, seed: int, bulk_shift_only: bool = False) -> np.ndarray:
    """Table 1 generators.  The paper shifts the random sets so that their
    real eigenvalues are strictly positive and safe from 0 without stating
    the amount; here the shift is the bulk spectral radius plus one --
    nonsymmetric N(0,1): sqrt(n)+1; nonsymmetric U(0,1): sqrt(n/12)+1 (the
    rank-one mean part n/2 is a positive real eigenvalue); symmetric N(0,1):
    2 sqrt(n)+1; symmetric U(0,1): 2 sqrt(n/12)+1 -- raised, where a draw's
    edge eigenvalue falls further out, until every real eigenvalue is >= 1
    (bulk_shift_only=True keeps the bulk shift).  Set VII: H_n + 1e-6 I."""
    g = rng(seed)
    sym = set_id in ("V", "VI")
    if set_id in ("I", "III"):
        A = g.uniform(0.0, 1.0, (n, n)); shift = np.sqrt(n / 12.0) + 1.0
    elif set_id in ("II", "IV"):
        A = g.standard_normal((n, n)); shift = np.sqrt(n) + 1.0
    elif set_id == "V":
        L = np.tril(g.uniform(0.0, 1.0, (n, n))); A = L + np.tril(L, -1).T
        shift = 2.0 * np.sqrt(n / 12.0) + 1.0
    elif set_id == "VI":
        L = np.tril(g.standard_normal((n, n))); A = L + np.tril(L, -1).T
        shift = 2.0 * np.sqrt(n) + 1.0
    elif set_id == "VII":
        A = hilbert(n); A[np.diag_indices(n)] += 1e-6
        return np.asfortranarray(A)
    else:
        raise ValueError(set_id)
    if not bulk_shift_only:
        ev = np.linalg.eigvalsh(A) if sym else np.linalg.eigvals(A)
        ev = np.asarray(ev)
        real = ev.real[np.abs(ev.imag) <= 1e-8 * np.abs(ev).max()] if not sym else ev
        if real.size:
            shift = max(shift, 1.0 - real.min())
    A[np.diag_indices(n)] += shift
    return np.asfortranarray(A)


# The five benchmark configurations -----------------------------------------
def config_spd64(seed: int = BASE_SEED + 0):
    """n = 64 SPD, lam log-uniform in [1e-2, 1e2] (FP64 Schur method only)."""
    return spd_case(64, -2.0, 2.0, seed)


def config_general512(seed: int = BASE_SEED + 1, n: int = 512):
    """n = 512, A = 3I + G/sqrt(n)."""
    return shifted_gaussian(n, 3.0, seed)


def config_spd4096(seed: int = BASE_SEED + 2, n: int = 4096):
    """n = 4096 SPD, kappa = 1e6 exactly (lam in [1e-3, 1e3], ends pinned)."""
    return spd_case(n, -3.0, 3.0, seed, force_ends=True)


def config_adjoint(seed: int = BASE_SEED + 4, count: int = 64, n: int = 256):
    """count matrices A = 3I + G/sqrt(n) and cotangents Gbar ~ N(0,1)."""
    As = [shifted_gaussian(n, 3.0, seed * 31 + 2 * i) for i in range(count)]
    Gs = [gaussian((n, n), seed * 31 + 2 * i + 1) for i in range(count)]
    return As, Gs
