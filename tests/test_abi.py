"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/sre.h declares (no compute calls: these run without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sre.h")


def declared_symbols():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"SRE_API\s+[\w\s\*]*?\b(sre_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2512_24685_gb300 import build
    build.build()
    from paper_2512_24685_gb300 import binding
    return binding.load_library()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["sre_plan_create", "sre_plan_destroy", "sre_m2", "sre_m2_async", "sre_m2_host",
                 "sre_m2_batched", "sre_sum4_range", "sre_server_create", "sre_server_submit",
                 "sre_server_poll", "sre_server_stats", "sre_server_destroy", "sre_status_str"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_2512_24685_gb300 import binding
    out = subprocess.run(["nm", "-D", "--defined-only", binding.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (sre_\w+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    for s in declared_symbols():
        assert hasattr(lib, s)


def test_library_is_built_for_sm_103a():
    from paper_2512_24685_gb300 import binding
    out = subprocess.run(["cuobjdump", "--list-elf", binding.library_path()],
                         capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_status_strings(lib):
    for code in range(11):
        s = lib.sre_status_str(code)
        assert s and isinstance(s, bytes)
    assert lib.sre_status_str(0) == b"ok"
    assert lib.sre_version() >= 10000


def test_argument_validation_without_device(lib):
    h = ctypes.c_void_p()
    assert lib.sre_plan_create(0, 0, ctypes.byref(h)) == 1          # N out of range
    assert lib.sre_plan_create(25, 0, ctypes.byref(h)) == 1
    assert lib.sre_plan_create(10, 7, ctypes.byref(h)) == 1         # bad dtype
    assert lib.sre_plan_create(10, 0, None) == 1                    # null out
    assert lib.sre_plan_destroy(None) == 0
    assert lib.sre_m2(None, None, 10, None, None) == 1


def test_binding_fails_loudly_without_cuda():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2512_24685_gb300 import binding
    with pytest.raises(RuntimeError):
        binding.Plan(8)
