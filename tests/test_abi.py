"""CPU-side checks of the C ABI: the library builds for sm_103a, loads without
a GPU, and exports every entry point that include/fock.h declares.  No compute
call is made here."""
import ctypes
import os
import re

import pytest

from paper_2005_13679_gb300 import _build, fock

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fock.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fock_[A-Za-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_binding_names():
    assert declared_functions() == sorted(fock.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_strerror_and_version_without_gpu(lib):
    fock.load()
    assert fock.fock_strerror(0) == "ok"
    assert fock.fock_strerror(fock.FOCK_ERR_ALIAS) == "input and output buffers overlap"
    assert "unknown" in fock.fock_strerror(-999)
    assert fock.fock_version() >= 100


def test_library_targets_sm103a():
    objs = [f for f in os.listdir(_build.OUT) if f.endswith(".o")]
    assert objs, "no object files"
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(fock, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        fock.load(str(tmp_path / "libfock.so"))


def test_binding_constants_match_the_header():
    """Every FOCK_* constant the header defines has the same value in the binding."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    defs = dict(re.findall(r"#define\s+(FOCK_[A-Z0-9_]+)\s+(-?\d+)\b", text))
    assert "FOCK_ERR_NOT_CONSERVING" in defs and "FOCK_PATH_LIST" in defs
    for name, value in defs.items():
        assert hasattr(fock, name), name
        assert getattr(fock, name) == int(value), name


def test_every_status_has_its_own_message(lib):
    fock.load()
    codes = sorted(v for k, v in vars(fock).items() if k.startswith("FOCK_ERR_"))
    msgs = [fock.fock_strerror(c) for c in codes]
    assert all("unknown" not in m for m in msgs)
    assert len(set(msgs)) == len(msgs)
