"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/grover_mps.h declares (no compute calls: no GPU here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header="grover_mps.h", prefix="grover_mps_"):
    src = open(os.path.join(ROOT, "include", header)).read()
    return sorted(set(re.findall(r"\b(" + prefix + r"\w+)\s*\(", src)))


def test_header_and_binding_agree():
    from paper_2601_03832_gb300 import binding
    assert sorted(binding.EXPORTS) == _declared()
    assert sorted(binding.SV_EXPORTS) == _declared("grover_sv.h", "grover_sv_")


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_03832_gb300 import binding
    lib = ctypes.CDLL(binding.LIB_PATH)
    declared = _declared() + _declared("grover_sv.h", "grover_sv_")
    missing = [s for s in declared if not hasattr(lib, s)]
    assert not missing, missing
    from paper_2601_03832_gb300 import peaks
    plib = ctypes.CDLL(peaks.LIB_PATH)
    assert all(hasattr(plib, s) for s in _declared("gmps_peaks.h", "gmps_peak_"))


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


def test_config_validation_needs_no_gpu():
    """grover_mps_create_ex checks its configuration on the host before any
    CUDA call: each invalid field is refused with its status and a message."""
    import pytest
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_03832_gb300 import binding as B
    cases = [
        (dict(n=0, marked=[0]), 1, "n must be"),
        (dict(n=65, marked=[0]), 1, "n must be"),
        (dict(n=5, marked=[]), 1, "M must be >= 1"),
        (dict(n=2, marked=[0, 1, 2, 3]), 1, "M must be < 2^n"),
        (dict(n=20, marked=list(range(65))), 9, "built maximum"),
        (dict(n=5, marked=[3, 3]), 1, "duplicate"),
        (dict(n=5, marked=[40]), 1, "bits >= n"),
        (dict(n=5, marked=[3], chi_max=0), 1, "chi_max"),
        (dict(n=5, marked=[3], tol=-1.0), 1, "tol"),
        (dict(n=5, marked=[3], tol=float("nan")), 1, "tol"),
        (dict(n=5, marked=[3], dtype=7), 1, "dtype"),
        (dict(n=5, marked=[3], apply=4), 1, "apply"),
        (dict(n=5, marked=[3], threads=48), 1, "threads"),
        (dict(n=5, marked=[3], threads=512), 1, "threads"),
        (dict(n=5, marked=[3], max_sweeps=-1), 1, "max_sweeps"),
    ]
    for kw, status, text in cases:
        n, marked = kw.pop("n"), kw.pop("marked")
        with pytest.raises(B.GMPSError) as e:
            B.GroverMPS(n, marked, **kw)
        assert e.value.status == status, (n, marked, kw)
        assert text in str(e.value), (str(e.value), text)


def test_noalloc_validation_matches_handle_path_without_gpu():
    """grover_mps_run_noalloc validates with the same routine as
    grover_mps_create_ex (same statuses and messages), before any CUDA call."""
    import pytest
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_03832_gb300 import binding as B
    cases = [
        (dict(n=0, marked=[0]), 1, "n must be"),
        (dict(n=20, marked=list(range(65))), 9, "built maximum"),
        (dict(n=5, marked=[3, 3]), 1, "duplicate"),
        (dict(n=5, marked=[40]), 1, "bits >= n"),
        (dict(n=5, marked=[3], chi_max=0), 1, "chi_max"),
        (dict(n=5, marked=[3], tol=float("nan")), 1, "tol"),
        (dict(n=5, marked=[3], apply=4), 1, "apply"),
        (dict(n=5, marked=[3], k=-1), 1, "k must be"),
    ]
    for kw, status, text in cases:
        n, marked, k = kw.pop("n"), kw.pop("marked"), kw.pop("k", 1)
        with pytest.raises(B.GMPSError) as e:
            B.run_noalloc(n, marked, k, **kw)
        assert e.value.status == status, (n, marked, kw)
        assert text in str(e.value), (str(e.value), text)


def test_statevector_validation_needs_no_gpu():
    """grover_sv_create refuses invalid arguments before any CUDA call."""
    import pytest
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_03832_gb300 import binding as B
    cases = [
        (dict(n=0, marked=[0]), "n must be"),
        (dict(n=37, marked=[0]), "n must be"),
        (dict(n=5, marked=[]), "M must be"),
        (dict(n=1, marked=[0, 1]), "M must be < 2^n"),
        (dict(n=5, marked=[3, 3]), "duplicate"),
        (dict(n=5, marked=[40]), "bits >= n"),
        (dict(n=5, marked=[3], dtype="dw"), "dtype"),
    ]
    for kw, text in cases:
        with pytest.raises(B.GMPSError) as e:
            B.GroverSV(**kw)
        assert e.value.status == 1
        assert text in str(e.value), (str(e.value), text)


def test_fault_injection_hook_needs_no_gpu():
    """grover_mps_debug_fail_allocations takes a count >= 0 and refuses a
    negative one, without any CUDA call; 0 clears it."""
    import pytest
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_03832_gb300 import binding as B
    with pytest.raises(B.GMPSError) as e:
        B.debug_fail_allocations(-1)
    assert e.value.status == 1 and "count" in str(e.value)
    B.debug_fail_allocations(3)
    B.debug_fail_allocations(0)
