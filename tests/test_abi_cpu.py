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


def _header_signatures():
    """name -> parameter kinds ('P' pointer, 'D' double, 'F' float, 'I' int or
    enum, 'LL' long long, 'ULL' unsigned long long) from include/*.h."""
    sigs = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"[\w\s\*]+?\b(sa_\w+)\s*\(([^;{}]*?)\)\s*;", src):
            name, params = m.group(1), m.group(2).strip()
            kinds = []
            if params and params != "void":
                for p in params.split(","):
                    p = " ".join(p.split())
                    if "*" in p or "[" in p:
                        kinds.append("P")
                    elif "double" in p:
                        kinds.append("D")
                    elif "float" in p:
                        kinds.append("F")
                    elif "unsigned long long" in p:
                        kinds.append("ULL")
                    elif "long long" in p:
                        kinds.append("LL")
                    else:
                        kinds.append("I")
            sigs[name] = kinds
    return sigs


def _ctypes_kind(t):
    import ctypes as C
    if t in (C.c_void_p, C.c_char_p) or (isinstance(t, type) and issubclass(t, C._Pointer)):
        return "P"
    return {C.c_double: "D", C.c_float: "F", C.c_int: "I", C.c_longlong: "LL",
            C.c_ulonglong: "ULL"}[t]


def test_binding_argument_types_match_the_header(lib):
    sigs = _header_signatures()
    assert "sa_eval_flux" in sigs and len(sigs["sa_eval_flux"]) == 7
    for name, kinds in sorted(sigs.items()):
        f = getattr(lib.lib, name)
        assert f.argtypes is not None, name          # every declared call is typed
        assert [_ctypes_kind(t) for t in f.argtypes] == kinds, name


def test_struct_layouts_match_the_header(lib):
    """sizeof and every field offset of the option, statistics and size
    structs, from a C program compiled against include/sa.h, against the
    binding's ctypes mirrors."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = {"sa_options": lib.sa_options, "sa_step_stats": lib.sa_step_stats,
               "sa_sizes": lib.sa_sizes, "sa_batch_shapes": lib.sa_batch_shapes}
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "sa.h"', "int main(void) {"]
    for name, cls in structs.items():
        src.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            src.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    src.append("return 0; }")
    out_dir = os.path.join(ROOT, "paper_2511_20432_gb300", "_build")
    os.makedirs(out_dir, exist_ok=True)
    c_path = os.path.join(out_dir, "abi_layout.c")
    exe = os.path.join(out_dir, "abi_layout")
    with open(c_path, "w") as fh:
        fh.write("\n".join(src) + "\n")
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), c_path, "-o", exe],
                   check=True)
    got = dict(l.split() for l in subprocess.run([exe], check=True, capture_output=True,
                                                 text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)
