"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function include/ftp.h declares, and rejects
bad arguments before touching a device."""
import ctypes
import os
import re

import pytest

import __graft_entry__
from paper_2101_12348_gb300 import ftp

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "ftp.h")


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return ftp.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ftp_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_binding_exports():
    assert declared_functions() == sorted(ftp.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(ftp.LIB_PATH)
    for name in declared_functions():
        assert hasattr(raw, name), name


def test_status_strings(lib):
    for code in range(9):
        s = ftp.ftp_status_string(code)
        assert isinstance(s, str) and s
    assert ftp.ftp_status_string(0) == "ok"
    assert "unknown" in ftp.ftp_status_string(99)


@pytest.mark.parametrize("args,expect", [
    (dict(max_nobs=1, max_H=3, grid=(0.1, 1, 10)), 1),
    (dict(max_nobs=10, max_H=0, grid=(0.1, 1, 10)), 1),
    (dict(max_nobs=10, max_H=17, grid=(0.1, 1, 10)), 8),
    (dict(max_nobs=10, max_H=3, grid=(0.0, 1, 10)), 1),
    (dict(max_nobs=10, max_H=3, grid=(0.1, 0, 10)), 1),
    (dict(max_nobs=10, max_H=3, grid=(float("nan"), 1, 10)), 1),
    (dict(max_nobs=10, max_H=3, grid=(0.1, 1, 0)), 1),
    # the last bin k0 + nf - 1 beyond 2^30 (an FFT of more than 2^31 cells),
    # including bins whose grid arithmetic would overflow int64
    (dict(max_nobs=10, max_H=3, grid=(0.1, 2**30, 2)), 8),
    (dict(max_nobs=10, max_H=3, grid=(0.1, 1, 2**40)), 8),
    (dict(max_nobs=10, max_H=3, grid=(0.1, 2**62, 10)), 8),
    (dict(max_nobs=10, max_H=3, grid=(0.1, 2**62, 2**62)), 8),
])
def test_plan_argument_validation(lib, args, expect):
    with pytest.raises(ftp.FtpError) as e:
        ftp.ftp_plan(**args)
    assert e.value.status == expect


def test_null_plan_is_rejected(lib):
    import numpy as np
    t = np.arange(4.0)
    with pytest.raises(ftp.FtpError) as e:
        ftp.ftp_sums(None, t, t, t, 4, 1, np.zeros(4))
    assert e.value.status == 1
    ftp.ftp_destroy(None)  # no-op


def test_build_compiles_every_translation_unit():
    from paper_2101_12348_gb300 import build as b
    cus = sorted(f for f in os.listdir(b.CSRC) if f.endswith(".cu"))
    assert sorted(b.SOURCES) == cus


def test_missing_library_fails_loudly(tmp_path):
    """The binding has no CPU fallback: loading a library that is not there
    raises instead of returning something that computes elsewhere."""
    with pytest.raises(FileNotFoundError, match="no CPU fallback"):
        ftp.load(str(tmp_path / "libftp_gb300.so"))


def test_product_path_never_touches_the_oracle():
    """Neither the CUDA sources nor the Python binding import, include or
    name the oracle package: the oracle is test infrastructure only."""
    pkg = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_2101_12348_gb300")
    pattern = re.compile(r"(^\s*(import|from)\s+oracle\b)|(#include\s*[<\"][^>\"]*oracle)|"
                         r"(import_module\(\s*[\"']oracle)", re.M)
    checked = 0
    for root, _, files in os.walk(pkg):
        if "_build" in root or "__pycache__" in root:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                checked += 1
                assert not pattern.search(open(os.path.join(root, f)).read()), f
    assert checked >= 10
