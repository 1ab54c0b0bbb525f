"""GB300 (sm_103a) mixed-precision matrix square root (arXiv 2607.12430).

Thin Python binding over the C ABI in ``include/sqrtm_mp.h`` and
``include/sqrtm_mp_steps.h``: every function marshals torch tensors (device
memory and the current CUDA stream) into the C call of the same name; all
computation runs in the library's CUDA kernels.  There is no CPU path: if the
compiled library is missing, every call raises.

Layout: the C ABI is column-major.  A contiguous (row-major) torch tensor is
the column-major storage of its transpose, and the principal square root
commutes with transposition (sqrt(A^T) = sqrt(A)^T), so row-major tensors are
passed through unchanged and the result comes back row-major.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build_mod

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = _build_mod.LIB

STATUS = {
    0: "success", 1: "not converged", 2: "eigenvalue on the closed negative real axis",
    3: "Schur iteration cap", 4: "diverged", 5: "NaN/Inf input", 6: "device wait gave up",
    7: "CUDA error", 8: "no saved factors",
}

KIND_AUTO, KIND_GENERAL, KIND_SPD, KIND_REAL = 0, 1, 2, 3
PREC_AUTO, PREC_FP32, PREC_TF32X3, PREC_RESID_FP64, PREC_TF32X3_GENERAL = -1, 0, 1, 2, 4
MAX_HISTORY = 64
MAX_TUNE = 32


class SqrtmError(RuntimeError):
    def __init__(self, code, what):
        msg = f"{what} failed with status {code} ({STATUS.get(code, 'invalid argument')})"
        if code == 7 and _lib is not None:
            try:
                msg += ": " + last_error()
            except Exception:
                pass
        super().__init__(msg)
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("blks", ctypes.c_int),
                ("kind", ctypes.c_int), ("precision", ctypes.c_int), ("steps", ctypes.c_int)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("n_max", ctypes.c_int64), ("blks", ctypes.c_int), ("qr_helpers", ctypes.c_int),
                ("batched", ctypes.c_int), ("spd_precision", ctypes.c_int), ("trisqrt_cutoff", ctypes.c_int),
                ("batched_spd", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("kind_used", ctypes.c_int), ("iterations", ctypes.c_int),
                ("scale_exponent", ctypes.c_int), ("norm_a", ctypes.c_double),
                ("history_len", ctypes.c_int), ("history", ctypes.c_double * MAX_HISTORY),
                ("ms_schur", ctypes.c_double), ("ms_trisqrt", ctypes.c_double),
                ("ms_refine", ctypes.c_double), ("ms_reduction", ctypes.c_double),
                ("schur_sweeps", ctypes.c_int), ("schur_rotations", ctypes.c_int64),
                ("ms_qr_chase", ctypes.c_double), ("schur_work", ctypes.c_int64)]

    def as_dict(self):
        return {"status": self.status, "kind_used": self.kind_used, "iterations": self.iterations,
                "scale_exponent": self.scale_exponent, "norm_a": self.norm_a,
                "history": [self.history[i] for i in range(self.history_len)],
                "ms_schur": self.ms_schur, "ms_trisqrt": self.ms_trisqrt, "ms_refine": self.ms_refine,
                "ms_reduction": self.ms_reduction, "schur_sweeps": self.schur_sweeps,
                "schur_rotations": self.schur_rotations, "ms_qr_chase": self.ms_qr_chase,
                "schur_work": self.schur_work}


_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_L = ctypes.c_int64
_D = ctypes.c_double

_SIGS = {
    "sqrtm_create": ([ctypes.POINTER(_P), _P], _I),
    "sqrtm_destroy": ([_P], _I),
    "sqrtm_set_stream": ([_P, _P], _I),
    "sqrtm_set_wait_limit": ([_P, _L], _I),
    "sqrtm_default_opts": ([ctypes.POINTER(Opts)], None),
    "sqrtm_set_tuning": ([_P, ctypes.POINTER(TuneEntry), _I], _I),
    "sqrtm_get_tuning": ([_P, ctypes.POINTER(TuneEntry), _I], _I),
    "sqrtm_mixed": ([_P, _P, _L, _L, _D, _P, _L, ctypes.POINTER(Opts), ctypes.POINTER(Info)], _I),
    "sqrtm_schur_fp64": ([_P, _P, _L, _L, _D, _P, _L, ctypes.POINTER(Opts), ctypes.POINTER(Info)], _I),
    "sqrtm_mixed_complex": ([_P, _P, _L, _L, _D, _P, _L, ctypes.POINTER(Opts), ctypes.POINTER(Info)], _I),
    "sqrtm_schur_fp64_complex": ([_P, _P, _L, _L, _D, _P, _L, ctypes.POINTER(Opts), ctypes.POINTER(Info)], _I),
    "sqrtm_cbrtm_mixed": ([_P, _P, _L, _L, _D, _P, _L, ctypes.POINTER(Opts), ctypes.POINTER(Info)], _I),
    "sqrtm_cbrtm_schur_fp64": ([_P, _P, _L, _L, _D, _P, _L, ctypes.POINTER(Opts), ctypes.POINTER(Info)], _I),
    "sqrtm_backward": ([_P, _P, _L, _L, _D, _P, _L, ctypes.POINTER(Info)], _I),
    "sqrtm_factors_take": ([_P, ctypes.POINTER(_P)], _I),
    "sqrtm_backward_factors": ([_P, _P, _P, _L, _L, _D, _P, _L, ctypes.POINTER(Info)], _I),
    "sqrtm_factors_n": ([_P], _L),
    "sqrtm_factors_destroy": ([_P], _I),
    "sqrtm_mixed_batched": ([_P, _I, _P, _P, _P, _D, _P, _P, ctypes.POINTER(Opts), _P], _I),
    "sqrtm_batch_partition": ([_I, _P, _I, _P, _P], _I),
    "sqrtm_batched_phases": ([_P, _P, _I, _P, _P], _I),
    "sqrtm_status_string": ([_I], ctypes.c_char_p),
    "sqrtm_kernel_launches": ([], _L),
    "sqrtm_last_error": ([_P], ctypes.c_char_p),
    "sqrtm_step_scale": ([_P, _P, _L, _L, _P, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)], _I),
    "sqrtm_step_schur": ([_P, _P, _P, _L, _I], _I),
    "sqrtm_step_hessenberg": ([_P, _P, _L, _L, _P, _P, _I], _I),
    "sqrtm_step_syevd": ([_P, _P, _P, _P, _L, _I], _I),
    "sqrtm_step_trisqrt": ([_P, _P, _P, _L, _I, _I], _I),
    "sqrtm_step_trisqrt_rec": ([_P, _P, _P, _L, _I, _I, _I], _I),
    "sqrtm_step_qtrisqrt": ([_P, _P, _P, _L, _I], _I),
    "sqrtm_step_real_schur": ([_P, _P, _P, _L, _I], _I),
    "sqrtm_step_qrtrsyl": ([_P, _P, _L, _P, _L, _P, _I], _I),
    "sqrtm_step_tricbrt": ([_P, _P, _P, _P, _L, _I, _I], _I),
    "sqrtm_step_rtrsyl3": ([_P, _P, _P, _P, _L, _I, _I], _I),
    "sqrtm_step_form_x0": ([_P, _P, _P, _L, _I, _P, _L, _I], _I),
    "sqrtm_step_residual": ([_P, _P, _L, _P, _L, _L, _I, _P, ctypes.POINTER(_D)], _I),
    "sqrtm_step_transform_in": ([_P, _P, _P, _P, _L], _I),
    "sqrtm_step_rtrsyl": ([_P, _P, _L, _P, _L, _P, _I], _I),
    "sqrtm_step_transform_out_update": ([_P, _P, _P, _L, _I, _P, _L], _I),
    "sqrtm_step_transform_in_spd": ([_P, _P, _P, _P, _P, _L], _I),
    "sqrtm_step_transform_out_update_spd": ([_P, _P, _P, _L, _I, _P, _L], _I),
    "sqrtm_step_gemm_tf32x3": ([_P, _L, _L, _L, _P, _L, _P, _L, _P, _L], _I),
    "sqrtm_step_cgemm_tf32x3": ([_P, _L, _L, _L, _P, _L, _I, _P, _L, _I, _P, _L], _I),
    "sqrtm_step_residual_sym": ([_P, _P, _L, _P, _L, _L, _I, _P, ctypes.POINTER(_D), _I], _I),
    "sqrtm_step_residual_split": ([_P, _P, _L, _P, _L, _L, _I, _P, ctypes.POINTER(_D)], _I),
    "sqrtm_step_residual_noalloc": ([_P, _L, _P, _L, _L, _I, _P, ctypes.POINTER(_D), _P], _I),
}


def lib():
    """Load the compiled library (``build()`` first).  Raises if it is missing:
    there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run build_library())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def last_error() -> str:
    """First CUDA failure recorded on this stream's handle ("" if none)."""
    return lib().sqrtm_last_error(handle()).decode()


def kernel_launches() -> int:
    """Kernel launches the library has issued in this process."""
    return int(lib().sqrtm_kernel_launches())


def build_library(force: bool = False) -> str:
    """Compile the CUDA library (no-op when it is up to date); returns its path."""
    return _build_mod.build(force=force)


# ---------------------------------------------------------------------------
# handles: one per (device, stream)
# ---------------------------------------------------------------------------
_handles: dict = {}


def _stream_ptr():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def handle():
    dev = torch.cuda.current_device()
    st = torch.cuda.current_stream().cuda_stream
    key = (dev, st)
    h = _handles.get(key)
    if h is None:
        hp = ctypes.c_void_p()
        rc = lib().sqrtm_create(ctypes.byref(hp), ctypes.c_void_p(st))
        if rc:
            raise SqrtmError(rc, "sqrtm_create")
        h = hp
        _handles[key] = h
        _install_shipped_tuning(h)
    return h


TUNING_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning")


def _install_shipped_tuning(h):
    """A new handle takes the tuning table the autotuner stored for this
    device model under tuning/ (if any); SQRTM_NO_TUNING=1 skips it."""
    if os.environ.get("SQRTM_NO_TUNING") == "1" or not os.path.isdir(TUNING_DIR):
        return
    import json
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    key = f"{p.name} sm_{p.major}{p.minor} x{p.multi_processor_count}"
    for f in sorted(os.listdir(TUNING_DIR)):
        if not f.endswith(".json"):
            continue
        with open(os.path.join(TUNING_DIR, f)) as fh:
            res = json.load(fh)
        if res.get("device") != key:
            continue
        t = res["table"]
        rc = lib().sqrtm_set_tuning(h, _tune_array(t), len(t))
        if rc:
            raise SqrtmError(rc, "sqrtm_set_tuning (" + f + ")")
        return


def _check_square(A, name="A", dtype=torch.float64):
    if not isinstance(A, torch.Tensor) or not A.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if A.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    if A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise ValueError(f"{name} must be square")
    if not A.is_contiguous():
        A = A.contiguous()
    return A


def _out_like(out, A, name="out"):
    """The caller's output buffer (must be a contiguous float64 CUDA tensor of
    A's shape) or a new one."""
    if out is None:
        return torch.empty(A.shape, dtype=A.dtype, device=A.device)
    if (not isinstance(out, torch.Tensor) or out.shape != A.shape or out.dtype != A.dtype
            or out.device != A.device or not out.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous {A.dtype} tensor of shape {tuple(A.shape)} on {A.device}")
    return out


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else ctypes.c_void_p(0)


def set_tuning(entries):
    """Install a tuning table (list of dicts with n_max, blks, qr_helpers,
    batched, spd_precision and optionally trisqrt_cutoff and batched_spd;
    ascending n_max)
    on this stream's handle; an empty list clears it."""
    rc = lib().sqrtm_set_tuning(handle(), _tune_array(entries), len(entries))
    if rc:
        raise SqrtmError(rc, "sqrtm_set_tuning")


def set_wait_limit(ns):
    """Limit (ns) of the cooperative QR chase's bounded inter-CTA waits on
    this stream's handle; 0 restores the default (2 s)."""
    _rc(lib().sqrtm_set_wait_limit(handle(), int(ns)), "sqrtm_set_wait_limit")


def get_tuning():
    """The tuning table of this stream's handle (list of dicts)."""
    arr = (TuneEntry * MAX_TUNE)()
    cnt = lib().sqrtm_get_tuning(handle(), arr, MAX_TUNE)
    return [{"n_max": arr[i].n_max, "blks": arr[i].blks, "qr_helpers": arr[i].qr_helpers,
             "batched": arr[i].batched, "spd_precision": arr[i].spd_precision,
             "trisqrt_cutoff": arr[i].trisqrt_cutoff, "batched_spd": arr[i].batched_spd} for i in range(cnt)]


def _tune_array(entries):
    arr = (TuneEntry * max(1, len(entries)))()
    for i, e in enumerate(entries):
        arr[i] = TuneEntry(int(e["n_max"]), int(e["blks"]), int(e["qr_helpers"]), int(e["batched"]),
                           int(e["spd_precision"]), int(e.get("trisqrt_cutoff", 0)), int(e.get("batched_spd", 1)))
    return arr


def make_opts(tol=1e-12, maxit=10, blks=0, kind=KIND_AUTO, precision=PREC_AUTO, steps=-1):
    o = Opts()
    lib().sqrtm_default_opts(ctypes.byref(o))
    o.tol, o.maxit, o.blks, o.kind, o.precision, o.steps = tol, maxit, blks, kind, precision, steps
    return o


# ---------------------------------------------------------------------------
# C-ABI entry points
# ---------------------------------------------------------------------------
def sqrtm_mixed(A, tol=1e-12, out=None, raise_on_error=True, **kw):
    """Mixed-precision principal square root (Algorithms 2 / 3).  Returns
    ``(X, info_dict)``."""
    A = _check_square(A)
    n = A.shape[0]
    X = _out_like(out, A)
    o = make_opts(tol=tol, **kw)
    info = Info()
    ld = max(1, n)
    rc = lib().sqrtm_mixed(handle(), _ptr(A), n, ld, tol, _ptr(X), ld, ctypes.byref(o), ctypes.byref(info))
    if rc and raise_on_error:
        raise SqrtmError(rc, "sqrtm_mixed")
    d = info.as_dict()
    d["status"] = rc
    return X, d


def sqrtm_schur_fp64(A, out=None, raise_on_error=True, **kw):
    """Plain FP64 Schur method on the GPU.  Returns ``(X, info_dict)``."""
    A = _check_square(A)
    n = A.shape[0]
    X = _out_like(out, A)
    o = make_opts(**kw)
    info = Info()
    ld = max(1, n)
    rc = lib().sqrtm_schur_fp64(handle(), _ptr(A), n, ld, 0.0, _ptr(X), ld, ctypes.byref(o), ctypes.byref(info))
    if rc and raise_on_error:
        raise SqrtmError(rc, "sqrtm_schur_fp64")
    d = info.as_dict()
    d["status"] = rc
    return X, d


def sqrtm_mixed_complex(A, tol=1e-12, out=None, raise_on_error=True, **kw):
    """Mixed-precision principal square root of a complex128 CUDA matrix
    (Algorithm 2 with complex iterates).  Returns ``(X, info_dict)``."""
    A = _check_square(A, dtype=torch.complex128)
    n = A.shape[0]
    X = _out_like(out, A)
    o = make_opts(tol=tol, **kw)
    info = Info()
    ld = max(1, n)
    rc = lib().sqrtm_mixed_complex(handle(), _ptr(A), n, ld, tol, _ptr(X), ld, ctypes.byref(o), ctypes.byref(info))
    if rc and raise_on_error:
        raise SqrtmError(rc, "sqrtm_mixed_complex")
    d = info.as_dict()
    d["status"] = rc
    return X, d


def sqrtm_schur_fp64_complex(A, out=None, raise_on_error=True, **kw):
    """Plain FP64 Schur method for a complex128 CUDA matrix."""
    A = _check_square(A, dtype=torch.complex128)
    n = A.shape[0]
    X = _out_like(out, A)
    o = make_opts(**kw)
    info = Info()
    ld = max(1, n)
    rc = lib().sqrtm_schur_fp64_complex(handle(), _ptr(A), n, ld, 0.0, _ptr(X), ld, ctypes.byref(o),
                                        ctypes.byref(info))
    if rc and raise_on_error:
        raise SqrtmError(rc, "sqrtm_schur_fp64_complex")
    d = info.as_dict()
    d["status"] = rc
    return X, d


def cbrtm_mixed(A, tol=1e-12, out=None, raise_on_error=True, **kw):
    """Mixed-precision principal cube root (Sec. 4, p = 3).  Returns
    ``(X, info_dict)``."""
    A = _check_square(A)
    n = A.shape[0]
    X = _out_like(out, A)
    o = make_opts(tol=tol, **kw)
    info = Info()
    ld = max(1, n)
    rc = lib().sqrtm_cbrtm_mixed(handle(), _ptr(A), n, ld, tol, _ptr(X), ld, ctypes.byref(o), ctypes.byref(info))
    if rc and raise_on_error:
        raise SqrtmError(rc, "sqrtm_cbrtm_mixed")
    d = info.as_dict()
    d["status"] = rc
    return X, d


def cbrtm_schur_fp64(A, out=None, raise_on_error=True, **kw):
    """Plain FP64 Schur method for the principal cube root on the GPU."""
    A = _check_square(A)
    n = A.shape[0]
    X = _out_like(out, A)
    o = make_opts(**kw)
    info = Info()
    ld = max(1, n)
    rc = lib().sqrtm_cbrtm_schur_fp64(handle(), _ptr(A), n, ld, 0.0, _ptr(X), ld, ctypes.byref(o),
                                      ctypes.byref(info))
    if rc and raise_on_error:
        raise SqrtmError(rc, "sqrtm_cbrtm_schur_fp64")
    d = info.as_dict()
    d["status"] = rc
    return X, d


def sqrtm_backward(G, tol=1e-12, out=None, raise_on_error=True):
    """Gradient of <G, sqrtm(A)> for the last sqrtm_mixed call on this
    stream's handle: Y with X^T Y + Y X^T = G."""
    G = _check_square(G, "G")
    n = G.shape[0]
    Y = _out_like(out, G)
    info = Info()
    ld = max(1, n)
    rc = lib().sqrtm_backward(handle(), _ptr(G), n, ld, tol, _ptr(Y), ld, ctypes.byref(info))
    if rc and raise_on_error:
        raise SqrtmError(rc, "sqrtm_backward")
    d = info.as_dict()
    d["status"] = rc
    return Y, d


class Factors:
    """The factors of one forward call (sqrtm_factors_take), owned by this
    object: its device memory is released when it is garbage-collected."""

    def __init__(self, ptr):
        self._p = ptr

    @property
    def n(self):
        return int(lib().sqrtm_factors_n(self._p))

    def close(self):
        if self._p:
            lib().sqrtm_factors_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def take_factors():
    """Detach the factors of the last sqrtm_mixed call on this stream's
    handle (no copy); the handle keeps none afterwards."""
    fp = ctypes.c_void_p()
    rc = lib().sqrtm_factors_take(handle(), ctypes.byref(fp))
    if rc:
        raise SqrtmError(rc, "sqrtm_factors_take")
    return Factors(fp)


def sqrtm_backward_factors(factors, G, tol=1e-12, out=None, raise_on_error=True):
    """Gradient of <G, sqrtm(A)> for the forward call whose factors are
    ``factors`` (a Factors object): Y with X^T Y + Y X^T = G."""
    G = _check_square(G, "G")
    n = G.shape[0]
    Y = _out_like(out, G)
    info = Info()
    ld = max(1, n)
    rc = lib().sqrtm_backward_factors(handle(), factors._p, _ptr(G), n, ld, tol, _ptr(Y), ld, ctypes.byref(info))
    if rc and raise_on_error:
        raise SqrtmError(rc, "sqrtm_backward_factors")
    d = info.as_dict()
    d["status"] = rc
    return Y, d


def sqrtm_mixed_batched(As, tol=1e-12, outs=None, raise_on_error=False, **kw):
    """Square roots of a list of square float64 CUDA tensors of any sizes.
    Returns ``(list_of_X, list_of_status)``.  A negative return code (an
    invalid argument: nothing was solved) always raises; raise_on_error=True
    also raises when some matrix failed."""
    As = [_check_square(A) for A in As]
    Xs = [_out_like(o, A) for o, A in zip(outs, As)] if outs is not None else [_out_like(None, A) for A in As]
    b = len(As)
    pa = (ctypes.c_void_p * b)(*[A.data_ptr() for A in As])
    px = (ctypes.c_void_p * b)(*[X.data_ptr() for X in Xs])
    ns = (ctypes.c_int64 * b)(*[A.shape[0] for A in As])
    st = (ctypes.c_int * b)()
    o = make_opts(tol=tol, **kw)
    rc = lib().sqrtm_mixed_batched(handle(), b, ctypes.cast(pa, _P), ctypes.cast(ns, _P), ctypes.cast(ns, _P),
                                   tol, ctypes.cast(px, _P), ctypes.cast(ns, _P), ctypes.byref(o),
                                   ctypes.cast(st, _P))
    if rc < 0 or (rc and raise_on_error):
        raise SqrtmError(rc, "sqrtm_mixed_batched")
    return Xs, list(st)


def batched_phases():
    """Phase times (ms, device clock) of the last batched-path graph on this
    stream's handle, with the number of matrices it took and how many of
    them were general."""
    ms = (ctypes.c_double * 5)()
    cnt, gen = ctypes.c_int(), ctypes.c_int()
    lib().sqrtm_batched_phases(handle(), ctypes.cast(ms, _P), 5, ctypes.byref(cnt), ctypes.byref(gen))
    names = ["prepare_and_hessenberg", "qr_rounds", "jacobi", "trisqrt_x0", "refinement"]
    return {"ms": dict(zip(names, list(ms))), "matrices": cnt.value, "general": gen.value}


def batch_partition(sizes, parts):
    """LPT partition of a batch over `parts` GPUs (sqrtm_batch_partition):
    returns (owner list, per-part cost list)."""
    b = len(sizes)
    ns = (ctypes.c_int64 * max(1, b))(*[int(x) for x in sizes])
    own = (ctypes.c_int * max(1, b))()
    load = (ctypes.c_double * max(1, parts))()
    _rc(lib().sqrtm_batch_partition(b, ctypes.cast(ns, _P), int(parts), ctypes.cast(own, _P),
                                    ctypes.cast(load, _P)), "sqrtm_batch_partition")
    return [own[i] for i in range(b)], [load[p] for p in range(parts)]


def sharded_run(sizes, rank, world, solve, gather):
    """The multi-GPU batch protocol, independent of how a share is solved:
    every rank computes the same LPT partition, solves its own matrices with
    ``solve(indices) -> statuses`` and the statuses are collected with
    ``gather(obj) -> list of every rank's obj`` (a host-side exchange of
    small integers; the matrices never leave their GPU).  Returns
    ``(own indices, statuses of the whole batch in input order)``."""
    owner, _ = batch_partition(sizes, world)
    mine = [i for i, o in enumerate(owner) if o == rank]
    st = solve(mine) if mine else []
    parts = gather((mine, list(st)))
    full = [None] * len(sizes)
    for idx, sts in parts:
        for i, v in zip(idx, sts):
            full[i] = int(v)
    return mine, full


def sqrtm_mixed_batched_sharded(As, tol=1e-12, group=None, **kw):
    """The batch split over the processes of torch.distributed (one GPU
    each): rank r solves the matrices the LPT partition gives it, on its own
    GPU, through sqrtm_mixed_batched; statuses are gathered on every rank.
    ``As`` is the whole batch as host (CPU) float64 tensors; each rank copies
    only its own share to its GPU.  Returns ``({index: X on this GPU},
    statuses of the whole batch)``."""
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {}

    def solve(idx):
        mats = [As[i].to(dev) for i in idx]
        Xs, st = sqrtm_mixed_batched(mats, tol=tol, **kw)
        out.update(zip(idx, Xs))
        return st

    def gather(obj):
        res = [None] * world
        dist.all_gather_object(res, obj, group=group)
        return res

    _, full = sharded_run([A.shape[0] for A in As], rank, world, solve, gather)
    return out, full


class _SqrtmFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, tol):
        X, info = sqrtm_mixed(A, tol=tol)
        ctx.tol = tol
        # this call's own factors: later forward calls on the same handle
        # (another sqrtm in the graph, a plain sqrtm_mixed) cannot replace them
        ctx.factors = take_factors() if info["kind_used"] in (KIND_GENERAL, KIND_SPD) else None
        return X

    @staticmethod
    def backward(ctx, G):
        if ctx.factors is None:
            raise SqrtmError(8, "sqrtm backward")
        Y, _ = sqrtm_backward_factors(ctx.factors, G.contiguous(), tol=ctx.tol)
        return Y, None


def sqrtm(A, tol=1e-12):
    """Differentiable principal square root (forward: sqrtm_mixed; backward:
    sqrtm_backward_factors with the factors that forward call computed)."""
    return _SqrtmFn.apply(A, tol)


# ---------------------------------------------------------------------------
# step-level entry points (sqrtm_mp_steps.h); arrays are column-major, so
# callers pass tensors whose storage is column-major (e.g. M.T.contiguous().T
# is not needed: use fortran_view below)
# ---------------------------------------------------------------------------
def col_major(t):
    """Return a tensor whose row-major storage holds ``t`` column-major (i.e.
    ``t.T.contiguous()``); use ``from_col_major`` to read results back."""
    return t.transpose(-1, -2).contiguous()


def from_col_major(t):
    return t.transpose(-1, -2)


def _rc(rc, what):
    if rc:
        raise SqrtmError(rc, what)


def step_scale(A_cm, n, fp64=False):
    """A_cm: float64 tensor holding A column-major (n*n).  Returns
    (As_cm complex, e, norm)."""
    dt = torch.complex128 if fp64 else torch.complex64
    As = torch.empty(n * n, dtype=dt, device=A_cm.device)
    e = ctypes.c_int()
    nrm = ctypes.c_double()
    _rc(lib().sqrtm_step_scale(handle(), _ptr(A_cm), n, n, _ptr(As), int(fp64), ctypes.byref(e), ctypes.byref(nrm)), "scale")
    return As, e.value, nrm.value


def step_hessenberg(A_cm, n, fp64=False):
    """Real Householder Hessenberg reduction: A_cm float64 column-major
    (n*n).  Returns (H_cm, Q_cm) complex with zero imaginary parts."""
    dt = torch.complex128 if fp64 else torch.complex64
    H = torch.empty(n * n, dtype=dt, device=A_cm.device)
    Q = torch.empty(n * n, dtype=dt, device=A_cm.device)
    _rc(lib().sqrtm_step_hessenberg(handle(), _ptr(A_cm), n, n, _ptr(H), _ptr(Q), int(fp64)), "hessenberg")
    return H, Q


def step_schur(T_cm, n, fp64=False):
    """In place: T_cm (complex, column-major A_s) becomes T; returns Q_cm."""
    Q = torch.empty_like(T_cm)
    _rc(lib().sqrtm_step_schur(handle(), _ptr(T_cm), _ptr(Q), n, int(fp64)), "schur")
    return Q


def step_syevd(As_cm, n, fp64=False):
    dt = torch.float64 if fp64 else torch.float32
    V = torch.empty(n * n, dtype=dt, device=As_cm.device)
    lam = torch.empty(n, dtype=dt, device=As_cm.device)
    _rc(lib().sqrtm_step_syevd(handle(), _ptr(As_cm), _ptr(V), _ptr(lam), n, int(fp64)), "syevd")
    return V, lam


def step_trisqrt(T_cm, n, blks=32, fp64=False):
    S = torch.empty_like(T_cm)
    _rc(lib().sqrtm_step_trisqrt(handle(), _ptr(T_cm), _ptr(S), n, blks, int(fp64)), "trisqrt")
    return S


def step_trisqrt_rec(T_cm, n, blks=32, cutoff=256, fp64=False):
    S = torch.empty_like(T_cm)
    _rc(lib().sqrtm_step_trisqrt_rec(handle(), _ptr(T_cm), _ptr(S), n, blks, cutoff, int(fp64)), "trisqrt_rec")
    return S


def step_real_schur(A_cm, n, fp64=False):
    """In place: A_cm (real, column-major) becomes the quasi-triangular T;
    returns Q_cm with A = Q T Q^T."""
    Q = torch.empty_like(A_cm)
    _rc(lib().sqrtm_step_real_schur(handle(), _ptr(A_cm), _ptr(Q), n, int(fp64)), "real_schur")
    return Q


def step_qtrisqrt(T_cm, n, fp64=False):
    """Real quasi-triangular square root: T_cm real (float32 / float64)
    column-major; returns S_cm."""
    S = torch.empty_like(T_cm)
    _rc(lib().sqrtm_step_qtrisqrt(handle(), _ptr(T_cm), _ptr(S), n, int(fp64)), "qtrisqrt")
    return S


def step_qrtrsyl(S_cm, m, St_cm, nn, C_cm, fp64=False):
    """In place: C_cm (real, m x nn column-major) becomes Y of
    S Y + Y St = C with real quasi-triangular S, St."""
    _rc(lib().sqrtm_step_qrtrsyl(handle(), _ptr(S_cm), m, _ptr(St_cm), nn, _ptr(C_cm), int(fp64)), "qrtrsyl")
    return C_cm


def step_tricbrt(T_cm, n, blks=32, fp64=False):
    """Triangular cube root: returns (S_cm, V_cm) with V = S^2."""
    S = torch.empty_like(T_cm)
    V = torch.empty_like(T_cm)
    _rc(lib().sqrtm_step_tricbrt(handle(), _ptr(T_cm), _ptr(S), _ptr(V), n, blks, int(fp64)), "tricbrt")
    return S, V


def step_rtrsyl3(S_cm, V_cm, C_cm, n, blks=32, fp64=False):
    """In place: C_cm (n x n column-major) becomes Y of S^2 Y + S Y S + Y S^2 = C."""
    _rc(lib().sqrtm_step_rtrsyl3(handle(), _ptr(S_cm), _ptr(V_cm), _ptr(C_cm), n, blks, int(fp64)), "rtrsyl3")
    return C_cm


def step_form_x0(Q_cm, S_cm, n, e=0, fp64=False):
    X = torch.empty(n * n, dtype=torch.float64, device=Q_cm.device)
    _rc(lib().sqrtm_step_form_x0(handle(), _ptr(Q_cm), _ptr(S_cm), n, e, _ptr(X), n, int(fp64)), "form_x0")
    return X


def step_residual(A_cm, X_cm, n, e=0):
    Rhat = torch.empty(n * n, dtype=torch.float32, device=A_cm.device)
    nrm = ctypes.c_double()
    _rc(lib().sqrtm_step_residual(handle(), _ptr(A_cm), n, _ptr(X_cm), n, n, e, _ptr(Rhat), ctypes.byref(nrm)), "residual")
    return Rhat, nrm.value


def step_residual_sym(A_cm, X_cm, n, e=0, split=False):
    """Symmetric FP64 residual of the SPD path; split=True forms X X from
    exact BF16 tensor-core digit products summed in FP64."""
    Rhat = torch.empty(n * n, dtype=torch.float32, device=A_cm.device)
    nrm = ctypes.c_double()
    _rc(lib().sqrtm_step_residual_sym(handle(), _ptr(A_cm), n, _ptr(X_cm), n, n, e, _ptr(Rhat),
                                      ctypes.byref(nrm), int(split)), "residual_sym")
    return Rhat, nrm.value


def step_residual_split(A_cm, X_cm, n, e=0):
    """FP64 residual of the general path with X X from exact BF16
    tensor-core digit products (rows of X against its columns) summed in
    FP64."""
    Rhat = torch.empty(n * n, dtype=torch.float32, device=A_cm.device)
    nrm = ctypes.c_double()
    _rc(lib().sqrtm_step_residual_split(handle(), _ptr(A_cm), n, _ptr(X_cm), n, n, e, _ptr(Rhat),
                                        ctypes.byref(nrm)), "residual_split")
    return Rhat, nrm.value


def step_residual_noalloc(A_cm, X_cm, n, e=0, out=None):
    """The FP64 residual without any device allocation inside the library
    (for callers that cannot allocate); ``out`` may supply the FP32 output
    buffer so that this call allocates nothing at all."""
    Rhat = out if out is not None else torch.empty(n * n, dtype=torch.float32, device=A_cm.device)
    nrm = ctypes.c_double()
    _rc(lib().sqrtm_step_residual_noalloc(_ptr(A_cm), n, _ptr(X_cm), n, n, e, _ptr(Rhat),
                                          ctypes.byref(nrm), _stream_ptr()), "residual_noalloc")
    return Rhat, nrm.value


def step_transform_in(Q_cm, Rhat_cm, n):
    Rt = torch.empty(n * n, dtype=torch.complex64, device=Q_cm.device)
    _rc(lib().sqrtm_step_transform_in(handle(), _ptr(Q_cm), _ptr(Rhat_cm), _ptr(Rt), n), "transform_in")
    return Rt


def step_rtrsyl(S_cm, m, St_cm, nn, C_cm, blks=32):
    """In place: C_cm (complex64, m x nn column-major) becomes Y."""
    _rc(lib().sqrtm_step_rtrsyl(handle(), _ptr(S_cm), m, _ptr(St_cm), nn, _ptr(C_cm), blks), "rtrsyl")
    return C_cm


def step_transform_out_update(Q_cm, Y_cm, n, X_cm, e=0):
    _rc(lib().sqrtm_step_transform_out_update(handle(), _ptr(Q_cm), _ptr(Y_cm), n, e, _ptr(X_cm), n), "transform_out_update")
    return X_cm


def step_transform_in_spd(V_cm, lam, Rhat_cm, n):
    Y = torch.empty(n * n, dtype=torch.float32, device=V_cm.device)
    _rc(lib().sqrtm_step_transform_in_spd(handle(), _ptr(V_cm), _ptr(lam), _ptr(Rhat_cm), _ptr(Y), n), "transform_in_spd")
    return Y


def step_transform_out_update_spd(V_cm, Y_cm, n, X_cm, e=0):
    _rc(lib().sqrtm_step_transform_out_update_spd(handle(), _ptr(V_cm), _ptr(Y_cm), n, e, _ptr(X_cm), n), "transform_out_update_spd")
    return X_cm


def step_gemm_tf32x3(A_rows, B_cols, M, N, K):
    """C = A B on the tensor cores (split TF32).  A_rows: float32 tensor whose
    storage holds A row by row (row i = A_rows[i*K:(i+1)*K]); B_cols: B column
    by column.  Returns C column-major (M*N)."""
    C = torch.empty(M * N, dtype=torch.float32, device=A_rows.device)
    _rc(lib().sqrtm_step_gemm_tf32x3(handle(), M, N, K, _ptr(A_rows), K, _ptr(B_cols), K, _ptr(C), M),
        "gemm_tf32x3")
    return C


def step_cgemm_tf32x3(A_rows, Y_cm, M, N, K, conj_a=False, conj_y=False):
    """C = op(A) op(Y) on the tensor cores (split TF32), complex64.  A_rows:
    complex64 tensor whose storage holds A row by row; Y_cm: Y column-major.
    Returns C column-major (M*N complex64)."""
    C = torch.empty(M * N, dtype=torch.complex64, device=A_rows.device)
    _rc(lib().sqrtm_step_cgemm_tf32x3(handle(), M, N, K, _ptr(A_rows), K, int(conj_a), _ptr(Y_cm), K,
                                      int(conj_y), _ptr(C), M), "cgemm_tf32x3")
    return C
