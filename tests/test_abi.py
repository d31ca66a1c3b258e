"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/hd.h declares (no compute call: no GPU needed)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "hd.h")).read()
    return sorted(set(re.findall(r"^HD_API [^;(]*?\b(hd_\w+)\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2211_16422_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("hd_ctx_create", "hd_encode", "hd_build_library", "hd_search_open", "hd_search_host",
                 "hd_status_string", "hd_last_error_message"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.hd_status_string.restype = ctypes.c_char_p
    lib.hd_version.restype = ctypes.c_uint32
    assert lib.hd_status_string(0) == b"HD_OK"
    assert lib.hd_status_string(4) == b"HD_ERR_TIMEOUT"
    assert lib.hd_version() >= 100


def test_binding_names_match_header():
    from paper_2211_16422_gb300 import hd
    assert set(_declared()) <= set(hd._SIGS)


def test_arch_flag_is_sm103a():
    from paper_2211_16422_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_oracle_not_reachable_from_product():
    pkg = os.path.join(ROOT, "paper_2211_16422_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "hd_oracle" not in src, f
