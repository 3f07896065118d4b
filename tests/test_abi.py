"""The C-ABI library builds, loads and exports every entry point include/*.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(cht_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    from paper_1601_04017_gb300 import _build

    return _build.build()


def test_header_declares_the_boundary():
    names = set(declared_functions())
    for want in ["cht_create", "cht_insert", "cht_build", "cht_merge", "cht_find", "cht_insert_or_update", "cht_erase",
                 "cht_migrate", "cht_destroy", "cht_size", "cht_export", "cht_status_string"]:
        assert want in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_without_gpu(lib_path):
    lib = ctypes.CDLL(lib_path)
    for n in declared_functions():
        assert hasattr(lib, n)
    lib.cht_status_string.restype = ctypes.c_char_p
    assert lib.cht_status_string(4) == b"table full"
    assert lib.cht_version() >= 100


def test_binding_rejects_bad_arrays():
    import numpy as np

    from paper_1601_04017_gb300 import cht

    with pytest.raises(TypeError):
        cht._ptr(np.zeros(4, np.int32), 8)
    with pytest.raises(ValueError):
        cht._ptr(np.zeros(4, np.int64), 8, n=5)
    p, n, cuda = cht._ptr(np.zeros(4, np.uint64), 8, n=4)
    assert n == 4 and not cuda and p
