"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/grover_mps.h declares (no compute calls: no GPU here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "grover_mps.h")).read()
    return sorted(set(re.findall(r"\b(grover_mps_\w+)\s*\(", src)))


def test_header_and_binding_agree():
    from paper_2601_03832_gb300 import binding
    assert sorted(binding.EXPORTS) == _declared()


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_03832_gb300 import binding
    lib = ctypes.CDLL(binding.LIB_PATH)
    missing = [s for s in _declared() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2601_03832_gb300 import binding
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "missing.so"))
    try:
        binding.load()
    except RuntimeError as e:
        assert "not built" in str(e)
    else:
        raise AssertionError("load() must raise when the CUDA library is missing")
