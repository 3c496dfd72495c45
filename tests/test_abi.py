"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point declared in include/pdq.h (no compute calls)."""
import ctypes
import re

from paper_2408_17063_gb300 import build


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    from paper_2408_17063_gb300 import pdq
    declared = pdq.header_symbols()
    assert len(declared) >= 25
    missing = [s for s in declared if not hasattr(lib, s)]
    assert missing == []
    # the binding covers every declared entry point and nothing else
    assert sorted(pdq._SIGS) == declared


def test_header_documents_every_entry_point():
    text = open(build.os.path.join(build.INCLUDE, "pdq.h")).read()
    for name in re.findall(r"\b(pdq_[a-z0-9_]+)\s*\(", text):
        assert f"{name}(" in text


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2408_17063_gb300 import pdq
    monkeypatch.setattr(pdq, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pdq, "_lib", None)
    import pytest
    with pytest.raises(ImportError):
        pdq.load()
