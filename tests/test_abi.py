"""The C ABI library builds, loads and exports what include/nomad.h declares.

No compute calls: these run without a GPU.
"""
import ctypes
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "nomad.h")


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"NOMAD_API\s+[\w\s\*]*?\b(nomad_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1312_0193_gb300 import nomad as nb
    return nb.load_library(), nb


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("nomad_create", "nomad_load_ratings", "nomad_epoch", "nomad_rmse",
                     "nomad_get_factors", "nomad_objective", "nomad_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    cdll, nb = lib
    out = subprocess.run(["nm", "-D", "--defined-only", nb.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(nomad_\w+)", out))
    for name in declared_functions():
        assert name in exported, name
        assert name in nb.SIGNATURES, name  # and bound in Python
    assert set(nb.SIGNATURES) <= exported


def test_struct_layouts_match_header(lib, tmp_path):
    """sizeof/offsetof of the public structs, from gcc on the header, equal
    the ctypes mirrors of the binding."""
    _, nb = lib
    fields = {"nomad_schedule": nb.nomad_schedule, "nomad_info": nb.nomad_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "nomad.h"',
             "int main(void) {"]
    for sname, cls in fields.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (sname, sname))
        for fname, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' %
                         (sname, fname, sname, fname))
    lines.append("return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)],
                   check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for sname, cls in fields.items():
        assert int(got[sname]) == ctypes.sizeof(cls), sname
        for fname, _ in cls._fields_:
            assert int(got["%s.%s" % (sname, fname)]) == getattr(cls, fname).offset, fname


def test_host_only_entry_points(lib):
    cdll, nb = lib
    s = nb.nomad_schedule_default()
    assert abs(s.alpha - 0.012) < 1e-7 and abs(s.beta - 0.05) < 1e-7
    assert s.mode == nb.NOMAD_MODE_EPOCH and s.precision == nb.NOMAD_FP32
    assert s.debug_drop_item == -1 and s.seed == 1
    for code in range(-9, 1):
        assert cdll.nomad_error_string(code)
    assert cdll.nomad_error_string(-100) == b"unknown error"
    h = ctypes.c_void_p()
    # bad arguments are rejected before any device work
    assert cdll.nomad_create(0, 10, 4, 0.1, ctypes.byref(s), ctypes.byref(h)) == \
        nb.NOMAD_ERR_INVALID_ARG
    assert cdll.nomad_create(10, 10, 513, 0.1, ctypes.byref(s), ctypes.byref(h)) == \
        nb.NOMAD_ERR_INVALID_ARG
    assert cdll.nomad_create(10, 10, 4, -1.0, ctypes.byref(s), ctypes.byref(h)) == \
        nb.NOMAD_ERR_INVALID_ARG
    assert not h.value
    assert cdll.nomad_epoch(None, 1, None) == nb.NOMAD_ERR_INVALID_ARG
    # several problems: no array, no handles, a NULL handle
    assert cdll.nomad_epoch_many(None, 1, 1, None) == nb.NOMAD_ERR_INVALID_ARG
    arr = (ctypes.c_void_p * 2)(None, None)
    assert cdll.nomad_epoch_many(arr, 0, 1, None) == nb.NOMAD_ERR_INVALID_ARG
    assert cdll.nomad_epoch_many(arr, 2, 1, None) == nb.NOMAD_ERR_INVALID_ARG
    ns = ctypes.c_int64(-1)
    assert cdll.nomad_last_epoch_span_ns(None, ctypes.byref(ns), None) == \
        nb.NOMAD_ERR_INVALID_ARG
    assert ns.value == -1
    cdll.nomad_destroy(None)


def test_no_gpu_fails_loudly(lib):
    """Without a GPU the library refuses to run: there is no CPU fallback."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    _, nb = lib
    with pytest.raises(nb.NomadError) as e:
        nb.Nomad(10, 10, 4, 0.1)
    assert e.value.code == nb.NOMAD_ERR_CUDA


def test_binding_constants_match_header():
    """Every NOMAD_* integer constant of the header has the same value in
    the binding (precision, modes, error codes, ...)."""
    from paper_1312_0193_gb300 import nomad as nb
    with open(HEADER) as f:
        src = f.read()
    defs = dict(re.findall(r"#define\s+(NOMAD_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", src))
    assert "NOMAD_FP8" in defs
    for name, val in defs.items():
        if name in ("NOMAD_H_", "NOMAD_NOALLOC_MAX_TILES"):
            continue
        assert getattr(nb, name) == int(val), name
