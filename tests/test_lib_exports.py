"""The C-ABI library builds, loads without a GPU, and exports every entry
point declared in include/img.h (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "img.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(img_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("img_create", "img_set_covariance", "img_dirty", "img_mvdr_bound",
              "img_solve", "img_destroy", "img_status_str"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1505_01348_gb300 import build as b
    path = b.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_1505_01348_gb300 import _lib
    assert sorted(_lib.EXPORTS) == sorted(n for n in _declared() if n in _lib.EXPORTS)
    assert set(_lib.EXPORTS) <= set(_declared())


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1505_01348_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.findall(r"import\s+(\w+)", text)
                assert "from oracle" not in text and "import oracle" not in text


def test_status_strings_without_gpu():
    from paper_1505_01348_gb300 import _lib
    lib = _lib.load(build_if_missing=True)
    assert lib.img_status_str(0) == b"ok"
    assert b"positive definite" in lib.img_status_str(3)
