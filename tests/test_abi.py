"""The C-ABI library loads on a machine without a GPU and exports every symbol that
include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(mppic_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2211_15605_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mppic_create", "mppic_bin", "mppic_deposit", "mppic_interp", "mppic_step",
                     "mppic_destroy", "mppic_last_error", "mppic_check"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_argument_errors_without_gpu(lib):
    """Invalid configurations are rejected on the host before any device call."""
    from paper_2211_15605_gb300 import mppic, synth
    L = mppic.load()
    p = synth.make_params(4, 4, 4)
    for bad in (dict(dt=0.0), dict(dx=-1.0), dict(nx=0)):
        q = dict(p)
        q.update(bad)
        c = mppic.make_config(q, 32, 1)
        h = ctypes.c_void_p()
        st = L.mppic_create(ctypes.byref(c), 1, None, None, None, ctypes.byref(h))
        assert st == mppic.ERR_INVALID
        assert L.mppic_last_error(None)
    c = mppic.make_config(p, 16, 1)
    h = ctypes.c_void_p()
    assert L.mppic_create(ctypes.byref(c), 1, None, None, None, ctypes.byref(h)) == mppic.ERR_INVALID
    c = mppic.make_config(p, 32, 1)
    assert L.mppic_create(ctypes.byref(c), 2, None, None, None, ctypes.byref(h)) == mppic.ERR_INVALID


def test_product_path_does_not_import_the_oracle():
    """The package and the library sources never refer to the oracle."""
    pkg = os.path.join(ROOT, "paper_2211_15605_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h")):
            txt = open(path).read()
            assert "import oracle" not in txt and "mppic_oracle" not in txt, path


def test_every_declaration_cites_the_paper():
    """Each entry point's comment in include/*.h names the passage of the paper it follows (a
    section or an equation) or says that the paper has no counterpart."""
    missing, commented = [], set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        for m in re.finditer(r"/\*((?:(?!\*/).)*)\*/\s*\n((?:[^;/]|/(?!\*))*?\b(mppic_[a-z0-9_]+)\s*\()",
                             src, flags=re.S):
            comment, name = m.group(1), m.group(3)
            commented.add(name)
            if not re.search(r"Sec\.\s*\d|Eq\.\s*\d|no\s+(?:\*\s*)?counterpart", comment, flags=re.I):
                missing.append(name)
    assert not missing, missing
    assert commented == set(declared_functions())
