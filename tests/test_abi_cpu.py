"""The C-ABI library loads and exports every entry point the header
declares; host-side behaviour that needs no GPU.  CPU only."""
import ctypes
import os
import re

import pytest

from paper_2609_05960_gb300 import _build, gtpower

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    src = open(os.path.join(ROOT, "include", "gtpower.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return re.findall(r"^\s*(?:int|void|const char\*|int64_t)\s+(gtp_\w+)\s*\(", src, re.M)


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return gtpower.load()


def test_header_declares_the_abi():
    names = header_symbols()
    assert len(names) == len(set(names))
    assert set(names) == set(gtpower.ABI_SYMBOLS)


def test_library_exports_every_header_symbol(lib):
    for name in header_symbols():
        assert hasattr(lib, name), name


def test_build_targets_sm103a_only():
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_create_without_a_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p(1)
    rc = lib.gtp_create(ctypes.byref(h), 0, None)
    assert rc == gtpower.GTP_ECUDA
    assert not h.value
    assert lib.gtp_last_error(None) == b"null context"
    assert lib.gtp_load_library(None, 0, None, 0.0, 0, None, 0, None, None, 0, None, 0) == gtpower.GTP_EINVAL
    assert lib.gtp_run_power(None, 0, 10, None, 0) == gtpower.GTP_EINVAL
