"""The C-ABI library loads and exports every entry point declared in
include/*.h.  Host-only calls; no CUDA work is issued here."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(sa_[a-zA-Z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2511_20432_gb300 import build
    build.build()
    from paper_2511_20432_gb300 import _binding
    return _binding


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"sa_create", "sa_create_patch", "sa_set_material", "sa_set_scan", "sa_step",
            "sa_eval_T"} <= names
    raw = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(raw, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    o = lib.options()
    assert o.precision == lib.SA_FP64 and o.pcg_tol == 1e-10 and o.half_space_factor == 2.0
    assert lib.status_name(lib.SA_ERR_NOT_CONVERGED) == "SA_ERR_NOT_CONVERGED"
    # NULL context: argument errors, no device work
    assert lib.lib.sa_set_material(None, 1.0, 1.0, 1.0, 1.0) == lib.SA_ERR_ARG
    assert lib.lib.sa_step(None, 0.5, 1e-5, 1, None) == lib.SA_ERR_ARG
    assert lib.lib.sa_last_error(None) == b"null context"
    assert lib.lib.sa_eval_T(None, None, 0, None, 0) == lib.SA_ERR_ARG
    assert lib.lib.sa_eval_flux(None, None, None, 0, None, None, 0) == lib.SA_ERR_ARG
    assert lib.lib.sa_eval_flux(None, None, None, 3, None, None, 0) == lib.SA_ERR_ARG
