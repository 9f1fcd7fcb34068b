"""The C-ABI library loads and exports every entry point the header
declares; host-side behaviour that needs no GPU.  CPU only."""
import ctypes
import os
import re

import numpy as np
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


def _declarations():
    """(name, comment block just above it) of every entry point in the header."""
    src = open(os.path.join(ROOT, "include", "gtpower.h")).read()
    out = []
    for m in re.finditer(r"^\s*(?:int|void|const char\*|int64_t)\s+(gtp_\w+)\s*\(", src, re.M):
        before = src[:m.start()]
        i = before.rfind("*/")
        j = before.rfind("/*", 0, i)
        out.append((m.group(1), before[j:i] if i >= 0 and j >= 0 else ""))
    return out


# Handle and plumbing calls of the boundary that carry no method of the paper.
PLUMBING = {"gtp_create", "gtp_destroy", "gtp_set_stream", "gtp_last_error", "gtp_set_param", "gtp_get_param",
            "gtp_measure_reductions", "gtp_measure_replay", "gtp_pack_events"}


def test_every_method_entry_point_cites_its_source():
    """Each declaration that computes part of the method names the passage of
    the paper it follows, or says that the paper has no counterpart."""
    cite = re.compile(r"Sec\. \d|Eq\. \d|Eqs\. \d|Algorithm \d|no counterpart|has no (?:batched form|adjoint)")
    missing = [n for n, c in _declarations() if n not in PLUMBING and not cite.search(c)]
    assert not missing, missing


def _cpu_noalloc_args(G=5, E=12, n_bins=10):
    import torch
    lib_n_in = np.array([1, 2], np.int32)
    n_tab = 1 * 2 + 2 * 4
    t = dict(e_int=torch.zeros(n_tab * 49), p_leak=torch.zeros(4 + 8), cell=torch.zeros(G, dtype=torch.int32),
             load_ff=torch.zeros(G), slew_ps=torch.zeros(G, 2, 2), gate_offsets=torch.zeros(G + 1, dtype=torch.int64),
             events=torch.zeros(E, 2, dtype=torch.int32), init_state=torch.zeros(G, dtype=torch.uint8))
    out = dict(waveform=torch.zeros(n_bins, dtype=torch.float64), e_leak=torch.zeros(G, dtype=torch.float64),
               e_int_out=None, e_sw=None, final_state=torch.zeros(G, dtype=torch.uint8))
    return lib_n_in, t, out


def _validate(n_in, t, out, window_ps=100, bin_ps=10):
    return gtpower._noalloc_validate(n_in, t["e_int"], t["p_leak"], t["cell"], t["load_ff"], t["slew_ps"], window_ps,
                                     t["gate_offsets"], t["events"], t["init_state"], bin_ps, 7, 7, out,
                                     require_cuda=False)


def test_noalloc_binding_rejects_bad_lengths_before_the_call():
    """Short outputs or inputs are caught in the binding, since the C side
    cannot see device-array lengths."""
    import torch
    n_in, t, out = _cpu_noalloc_args()
    assert _validate(n_in, t, out)[:2] == (5, 2)
    bad_cases = [
        ("waveform", dict(out, waveform=torch.zeros(9, dtype=torch.float64)), t),
        ("gate_offsets", out, dict(t, gate_offsets=torch.zeros(5, dtype=torch.int64))),
        ("final_state", dict(out, final_state=torch.zeros(4, dtype=torch.uint8)), t),
        ("load_ff", out, dict(t, load_ff=torch.zeros(4))),
        ("e_int", out, dict(t, e_int=torch.zeros(10 * 49 - 1))),
        ("events", out, dict(t, events=torch.zeros(24, dtype=torch.int32))),
        ("slew stride", out, dict(t, slew_ps=torch.zeros(5, 1, 2))),
    ]
    for name, o, tt in bad_cases:
        with pytest.raises(ValueError, match=name):
            _validate(n_in, tt, o)
    with pytest.raises(ValueError):
        _validate(n_in, t, out, window_ps=105, bin_ps=10)
    with pytest.raises(TypeError):
        _validate(n_in, dict(t, cell=torch.zeros(5, dtype=torch.int64)), out)
    with pytest.raises(TypeError):
        gtpower._noalloc_validate(n_in, t["e_int"], t["p_leak"], t["cell"], t["load_ff"], t["slew_ps"], 100,
                                  t["gate_offsets"], t["events"], t["init_state"], 10, 7, 7, out, require_cuda=True)
