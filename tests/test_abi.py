"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/sv.h declares (no GPU compute is called here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "sv.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(sv_[a-z0-9_]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2411_01964_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sv_init_primes", "sv_verify_range", "sv_min_k", "sv_submit", "sv_poll", "sv_cancel",
                     "sv_create", "sv_destroy", "sv_strerror", "sv_verify_batch", "sv_sieve_bitmap"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2411_01964_gb300 import binding
    names = declared_functions()
    assert set(names) <= set(binding._SIGS), set(names) - set(binding._SIGS)
    for n in names:
        assert callable(getattr(binding, n)), n


def test_host_only_entry_points(lib):
    lib.sv_strerror.restype = ctypes.c_char_p
    assert lib.sv_strerror(0) == b"ok"
    assert b"range" in lib.sv_strerror(2)
    lib.sv_bitmap_words.restype = ctypes.c_uint64
    lib.sv_bitmap_words.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    assert lib.sv_bitmap_words(0, 0) == 0
    assert lib.sv_bitmap_words(0, 64) == 1     # odd 1..63
    assert lib.sv_bitmap_words(0, 65) == 1     # 65 itself is excluded
    assert lib.sv_bitmap_words(0, 66) == 2     # ... up to 65
    assert lib.sv_bitmap_words(64, 128) == 1


def test_null_arguments_are_rejected_without_a_device(lib):
    lib.sv_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.sv_create(None, None) == 1  # SV_EINVAL
    lib.sv_verify_range.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p]
    assert lib.sv_verify_range(None, 3, 5, None) == 1
    lib.sv_destroy.argtypes = [ctypes.c_void_p]
    lib.sv_destroy(None)


def test_no_cpu_fallback_in_the_product_path():
    """The package never imports the oracle, and the binding refuses to run
    without the compiled library."""
    pkg = os.path.join(ROOT, "paper_2411_01964_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "oracle.c" not in src, f


def test_kernel_timing_argument(monkeypatch):
    """sv_kernel_timing's binding: False is off, True every kernel (-1), a set of
    kernel names their bit mask (bit i for kernel id i)."""
    from paper_2411_01964_gb300 import binding

    seen = []

    class FakeLib:
        def sv_kernel_timing(self, ctx, arg):
            seen.append(arg)
            return 0

    monkeypatch.setattr(binding, "load", lambda *a, **k: FakeLib())
    binding.sv_kernel_timing(None, False)
    binding.sv_kernel_timing(None, True)
    binding.sv_kernel_timing(None, ["tile"])
    binding.sv_kernel_timing(None, ["init", "list_compact"])
    ids = binding.KERNEL_IDS
    assert seen == [0, -1, 1 << ids["tile"], (1 << ids["init"]) | (1 << ids["list_compact"])]
    with pytest.raises(KeyError):
        binding.sv_kernel_timing(None, ["no_such_kernel"])
