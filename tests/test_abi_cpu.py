"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function that include/*.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in ("sqrtm_mp.h", "sqrtm_mp_steps.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        names += re.findall(r"SQRTM_API\s+[\w\s\*]+?\b(sqrtm_\w+)\s*\(", src)
    return sorted(set(names))


def test_headers_declare_entry_points():
    names = _declared()
    for must in ("sqrtm_mixed", "sqrtm_schur_fp64", "sqrtm_backward", "sqrtm_create",
                 "sqrtm_destroy", "sqrtm_mixed_batched", "sqrtm_step_residual",
                 "sqrtm_step_rtrsyl", "sqrtm_step_schur", "sqrtm_step_trisqrt", "sqrtm_cbrtm_mixed",
                 "sqrtm_cbrtm_schur_fp64", "sqrtm_step_tricbrt", "sqrtm_step_rtrsyl3"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_2607_12430_gb300 as pkg
    path = pkg.build_library()
    L = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert missing == []


def test_binding_signatures_cover_header():
    import paper_2607_12430_gb300 as pkg
    assert sorted(pkg._SIGS) == _declared()


def test_status_strings_without_gpu():
    import paper_2607_12430_gb300 as pkg
    L = pkg.lib()
    for code in range(-3, 9):
        assert isinstance(L.sqrtm_status_string(code), bytes)


def test_no_oracle_in_product_path():
    # the product package must never import the oracle
    pkgdir = os.path.join(ROOT, "paper_2607_12430_gb300")
    for dirpath, _, files in os.walk(pkgdir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "liboracle" not in txt, f
