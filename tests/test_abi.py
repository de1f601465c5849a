"""The C-ABI library loads and exports every entry point its headers declare
(no compute call: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2606_16765_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DECL = re.compile(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b((?:lbm|fno|ffno|unet)_\w+)\s*\(", re.M)


def declared(header):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return sorted(set(DECL.findall(text)))


@pytest.fixture(scope="module")
def libs():
    return _build.build()


def test_headers_declare_entry_points():
    names = declared(os.path.join(ROOT, "include", "lbm.h"))
    for must in ("lbm_create", "lbm_step", "lbm_read_mean", "lbm_read_snapshot", "lbm_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(libs):
    for header in glob.glob(os.path.join(ROOT, "include", "*.h")):
        names = declared(header)
        assert names, header
        found = False
        for path in libs.values():
            L = ctypes.CDLL(path)
            missing = [n for n in names if not hasattr(L, n)]
            if len(missing) < len(names):
                found = True
                assert not missing, (header, path, missing)
        assert found, f"no library exports the entry points of {header}"


def test_product_binding_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2606_16765_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True) + \
            glob.glob(os.path.join(pkg, "csrc", "*")):
        text = open(path, errors="ignore").read()
        assert "import oracle" not in text and "from oracle" not in text, path
        assert "lbm_oracle" not in text, path
