"""The C ABI library builds, loads without a GPU, and exports every symbol
include/tor.h declares.  No compute calls here."""
import ctypes
import os
import re

from paper_2109_04528_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "tor.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tor_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_loads():
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in header_functions():
        assert hasattr(lib, name), f"{name} declared in tor.h but not exported"


def test_binding_covers_header():
    assert sorted(binding.EXPORTS) == header_functions()


def test_strerror_without_gpu():
    assert binding.tor_strerror(binding.TOR_ENOTPD) == "I - O is not positive definite"
    assert binding.tor_strerror(99) == "unknown status"


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(binding, "_LIB", None)
    monkeypatch.setattr(build, "library_path", lambda: str(tmp_path / "nope.so"))
    try:
        binding.load_library()
    except binding.TorError as e:
        assert "not built" in str(e)
    else:
        raise AssertionError("expected TorError")
    finally:
        monkeypatch.setattr(binding, "_LIB", None)
