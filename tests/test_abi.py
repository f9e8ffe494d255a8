"""CPU-side checks of the C ABI: the library loads, exports every entry
point include/elm.h declares, and rejects bad arguments before launching."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import __graft_entry__

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    from paper_2011_02436_gb300 import _lib
    return _lib.load()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(elm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"elm_hidden", "elm_pinv_rank", "elm_train", "elm_predict"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_2011_02436_gb300 import _lib
    assert sorted(n for n, _, _ in _lib.SIGNATURES) == declared_functions()


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """ctypes mirrors of the structs have the sizes and offsets gcc gives."""
    import subprocess
    from paper_2011_02436_gb300 import _lib
    src = tmp_path / "layout.c"
    fields = {"elm_problem": [f for f, _ in _lib.elm_problem._fields_],
              "elm_train_opts": [f for f, _ in _lib.elm_train_opts._fields_],
              "elm_result": [f for f, _ in _lib.elm_result._fields_]}
    body = ['#include <stdio.h>', '#include <stddef.h>', '#include "elm.h"', "int main(void){"]
    for st, fs in fields.items():
        body.append('printf("%%zu\\n", sizeof(%s));' % st)
        for f in fs:
            body.append('printf("%%zu\\n", offsetof(%s, %s));' % (st, f))
    body.append("return 0;}")
    src.write_text("\n".join(body))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)],
                   check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    expect = []
    for st in fields:
        cls = getattr(_lib, st)
        expect.append(C.sizeof(cls))
        expect += [getattr(cls, f).offset for f in fields[st]]
    assert out == expect


def test_status_strings(lib):
    assert lib.elm_status_string(0) == b"ok"
    assert lib.elm_status_string(1) == b"invalid argument"
    assert lib.elm_status_string(99) == b"unknown status"


def test_null_context_is_rejected(lib):
    from paper_2011_02436_gb300 import _lib
    assert lib.elm_train(None, None, 0, None, None) == 1
    assert lib.elm_hidden(None, None, 0, 1, 1, 1, None, 1, None, None, 1, 0, 0, None, 1) == 1
    assert lib.elm_pinv_rank(None, None, 1, 1, 1, 0.0, None, None, None, 0) == 1
    assert lib.elm_predict(None, None, 0, 1, 1, 1, None, 1, None, None, 1, 0, None, 1, 1,
                           None, 1) == 1
    assert lib.elm_create(None, 0, None) == 1
    assert lib.elm_destroy(None) == 0


def test_package_fails_loudly_without_library(monkeypatch):
    from paper_2011_02436_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", "/nonexistent/libelm.so")
    with pytest.raises(ImportError):
        _lib.load()
