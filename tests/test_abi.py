"""The C ABI library builds, loads without a GPU and exports every entry point that
include/trals.h declares (no compute calls). CPU only."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "trals.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:tr_status|void|int|const char\*)\s+(tr_\w+)\s*\(", text,
                                 flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2010_08581_gb300 import build, trals
    if not os.path.exists(trals.LIB_PATH):
        build.build()
    return trals.LIB_PATH


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("tr_create", "tr_destroy", "tr_leverage", "tr_sample", "tr_subchain",
                     "tr_gather", "tr_solve", "tr_als_sampled", "tr_rel_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_2010_08581_gb300 import trals
    assert sorted(trals.SIGNATURES) == _declared()
    trals.load()


def test_binding_refuses_to_run_without_library(tmp_path, monkeypatch):
    from paper_2010_08581_gb300 import trals
    monkeypatch.setattr(trals, "_lib", None)
    monkeypatch.setattr(trals, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        trals.load()


def test_create_without_gpu_reports_an_error(lib_path):
    """With no visible GPU, tr_create returns a status instead of aborting."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    from paper_2010_08581_gb300 import trals
    lib = trals.load()
    h = ctypes.c_void_p()
    st = lib.tr_create(ctypes.byref(h), 0, 0)
    assert st != trals.TR_OK
    assert not h.value
    lib.tr_destroy(None)
