"""The C-ABI library builds, loads and exports every entry point of
include/mqs.h (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

from paper_2507_19246_gb300 import build as B
from paper_2507_19246_gb300 import mqs

HEADER = os.path.join(B.ROOT, "include", "mqs.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(mqs_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ctypes.CDLL(B.LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("mqs_create", "mqs_upload_mesh", "mqs_set_samples", "mqs_propagate",
                 "mqs_read_qoi", "mqs_mlmc_readout"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    assert sorted(mqs.exported_symbols()) == _declared()
    for name in _declared():
        assert callable(getattr(mqs, name)), name


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(mqs, "_lib", None)
    monkeypatch.setattr(mqs, "lib_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        mqs.load()
