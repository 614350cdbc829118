"""CPU-side checks of the C ABI boundary: the library builds, loads without a
GPU and exports every function include/sw.h declares.  No compute calls."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(sw_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2211_10769_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sw_ctx_create", "sw_ctx_destroy", "sw_strerror", "sw_encode", "sw_score",
                     "sw_align", "sw_alignment_free"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_strerror_without_gpu(lib):
    lib.sw_strerror.restype = ctypes.c_char_p
    assert lib.sw_strerror(0) == b"ok"
    assert lib.sw_strerror(-1) == b"invalid argument"


def test_null_context_arguments_without_gpu(lib):
    """Calls that only inspect their arguments reject a null context."""
    lib.sw_ctx_timing.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.sw_ctx_kernel_time.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.sw_ctx_launches.argtypes = [ctypes.c_void_p]
    lib.sw_ctx_launches.restype = ctypes.c_int64
    assert lib.sw_ctx_timing(None, 1) == -1
    assert lib.sw_ctx_kernel_time(None, 0, None, None) == -1
    assert lib.sw_ctx_launches(None) == -1


def test_binding_refuses_missing_library(tmp_path, monkeypatch):
    from paper_2211_10769_gb300 import binding
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(RuntimeError):
        binding.load()
