"""The allocation-free entry point gtp_run_power_noalloc, through the C ABI.

It is checked against gtp_run_power (the context-based entry point) and
directly against the FP64 oracle, on two calls in a row (the second call
reuses the static scratch the first one left behind), at exactly the largest
window the scratch holds, one bin past it (rejected before any work), and at
odd bin sizes with events sitting exactly on bin boundaries.  Collected last
on purpose: it must also pass after every other test has used the library in
this process."""
import numpy as np
import pytest

import oracle
import synth
from cases import small_random

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _device_inputs(lib, net, tr):
    import torch
    d = torch.device("cuda", 0)
    return dict(
        e_int=torch.from_numpy(lib.e_int).to(d), p_leak=torch.from_numpy(lib.p_leak).to(d),
        cell=torch.from_numpy(net.cell).to(d), load_ff=torch.from_numpy(net.load_ff).to(d),
        slew_ps=torch.from_numpy(np.ascontiguousarray(net.slew_ps)).to(d),
        gate_offsets=torch.from_numpy(tr.offsets).to(d),
        events=torch.from_numpy(tr.records.view(np.int32)).to(d),
        init_state=torch.from_numpy(tr.init_state).to(d))


def _call(lib, dev, window_ps, bin_ps, out=None):
    from paper_2609_05960_gb300 import gtpower
    gtpower.gtp_run_power_noalloc(lib.n_in, lib.vdd, lib.slew_axis, lib.load_axis, dev["e_int"], dev["p_leak"],
                                  dev["cell"], dev["load_ff"], dev["slew_ps"], window_ps, dev["gate_offsets"],
                                  dev["events"], dev["init_state"], bin_ps, **(out or {}))


def _noalloc(lib, tr, dev, bin_ps):
    import torch
    G = dev["cell"].numel()
    d = dev["cell"].device
    out = dict(waveform=torch.full((tr.window_ps // bin_ps,), float("nan"), dtype=torch.float64, device=d),
               e_leak=torch.full((G,), float("nan"), dtype=torch.float64, device=d),
               e_int_out=torch.full((G,), float("nan"), dtype=torch.float64, device=d),
               e_sw=torch.full((G,), float("nan"), dtype=torch.float64, device=d),
               final_state=torch.full((G,), 255, dtype=torch.uint8, device=d))
    _call(lib, dev, tr.window_ps, bin_ps, out)
    return {k: v.cpu().numpy() for k, v in out.items()}


def _existing(lib, net, tr, bin_ps):
    from paper_2609_05960_gb300 import Engine
    eng = Engine(0)
    try:
        eng.load_library(lib)
        eng.load_netlist(net)
        eng.load_events(0, tr)
        w = eng.run_power(0, bin_ps).cpu().numpy()
        ge = eng.gate_energy(0, device=False)
    finally:
        eng.close()
    return w, ge


def _reference(lib, net, tr, bin_ps):
    ref = oracle.walk(lib, net, tr, bin_ps)
    ge = {k: ref[k] for k in ("e_leak", "e_int", "e_sw", "final_state")}
    return oracle.waveform_w(ref["bins"], bin_ps), ge


def _assert_close(got, w, ge):
    rel = np.abs(got["waveform"] - w) / np.abs(w)
    assert rel.max() <= TOL, f"bin {rel.argmax()}: {got['waveform'][rel.argmax()]} vs {w[rel.argmax()]}"
    np.testing.assert_array_equal(got["final_state"], ge["final_state"])
    for k_got, k_ref in (("e_leak", "e_leak"), ("e_int_out", "e_int"), ("e_sw", "e_sw")):
        err = np.abs(got[k_got] - ge[k_ref])
        assert (err <= TOL * np.abs(ge[k_ref]) + 1e-9).all(), k_ref


def _on_boundaries(tr, bin_ps, every=3):
    """Every `every`-th gate's timestamps moved down onto the bin boundary
    below them (order within a gate is kept; ties appear, which are legal)."""
    rec = tr.records.copy()
    for g in range(0, len(tr.offsets) - 1, every):
        a, b = int(tr.offsets[g]), int(tr.offsets[g + 1])
        rec[a:b, 0] = (rec[a:b, 0] // bin_ps) * bin_ps
    return synth.Trace(tr.window_ps, tr.offsets, np.ascontiguousarray(rec), tr.init_state, 0, 0)


@pytest.fixture(scope="module")
def case():
    # several merge tiles of bins (10,000 bins of 10 ps) and a ragged last tile
    lib, net, tr = small_random(n_gates=3000, n_events=200_000, window_ps=100_000, seed=23, tie_p=0.05)
    return lib, net, tr, 10


def test_noalloc_matches_run_power_and_oracle_twice(case):
    lib, net, tr, bin_ps = case
    w, ge = _existing(lib, net, tr, bin_ps)
    w_ref, ge_ref = _reference(lib, net, tr, bin_ps)
    dev = _device_inputs(lib, net, tr)
    first = _noalloc(lib, tr, dev, bin_ps)
    _assert_close(first, w, ge)
    _assert_close(first, w_ref, ge_ref)
    second = _noalloc(lib, tr, dev, bin_ps)
    _assert_close(second, w, ge)
    _assert_close(second, w_ref, ge_ref)


@pytest.mark.parametrize("bin_ps", [7, 1000])
def test_noalloc_odd_bins_with_boundary_events(bin_ps):
    n_bins = 1000 if bin_ps == 1000 else 14_285
    lib, net, tr = small_random(n_gates=600, n_events=60_000, window_ps=n_bins * bin_ps, seed=31, tie_p=0.02)
    tr = _on_boundaries(tr, bin_ps)
    dev = _device_inputs(lib, net, tr)
    w_ref, ge_ref = _reference(lib, net, tr, bin_ps)
    w, ge = _existing(lib, net, tr, bin_ps)
    for _ in range(2):
        got = _noalloc(lib, tr, dev, bin_ps)
        _assert_close(got, w_ref, ge_ref)
        _assert_close(got, w, ge)


def test_noalloc_at_the_largest_window_and_one_bin_past_it():
    """Exactly GTP_NOALLOC_MAX_BINS bins (the merge's tile sums fill their
    region) matches the oracle; one bin more is rejected on the host."""
    from paper_2609_05960_gb300 import gtpower
    nmax = gtpower.GTP_NOALLOC_MAX_BINS
    bin_ps = 3
    lib, net, tr = small_random(n_gates=400, n_events=50_000, window_ps=nmax * bin_ps, seed=41, tie_p=0.02)
    tr = _on_boundaries(tr, bin_ps, every=5)
    dev = _device_inputs(lib, net, tr)
    w_ref, ge_ref = _reference(lib, net, tr, bin_ps)
    for _ in range(2):
        got = _noalloc(lib, tr, dev, bin_ps)
        assert got["waveform"].shape == (nmax,)
        _assert_close(got, w_ref, ge_ref)
    with pytest.raises(gtpower.GtpError) as ei:
        _call(lib, dev, (nmax + 1) * 1, 1)
    assert ei.value.code == gtpower.GTP_ERANGE


def test_noalloc_errors_then_recovers(case):
    """A window beyond the scratch is rejected on the host; a malformed trace
    is reported by the kernel; the next good call still matches (the error
    word and accumulators are cleared at every call)."""
    import torch
    from paper_2609_05960_gb300 import gtpower
    lib, net, tr, bin_ps = case
    dev = _device_inputs(lib, net, tr)
    big = 2 * gtpower.GTP_NOALLOC_MAX_BINS
    with pytest.raises(gtpower.GtpError) as ei:
        _call(lib, dev, big, 1)
    assert ei.value.code == gtpower.GTP_ERANGE
    # swap the timestamps of the first two distinct-time records of one gate
    counts = np.diff(tr.offsets)
    rec = tr.records.copy()
    g = int(np.argmax(counts))
    a = int(tr.offsets[g])
    b = a + 1 + int(np.argmax(rec[a + 1:a + counts[g], 0] != rec[a, 0]))
    rec[a, 0], rec[b, 0] = rec[b, 0], rec[a, 0]
    bad = dict(dev, events=dev["events"].clone())
    bad["events"].copy_(torch.from_numpy(rec.view(np.int32)))
    with pytest.raises(gtpower.GtpError) as ei:
        _noalloc(lib, tr, bad, bin_ps)
    assert ei.value.code == gtpower.GTP_EORDER
    w, ge = _existing(lib, net, tr, bin_ps)
    _assert_close(_noalloc(lib, tr, dev, bin_ps), w, ge)


def test_noalloc_refuses_a_capturing_stream(case):
    """The call waits for its stream, so on a stream under capture it returns
    GTP_EINVAL without enqueuing anything; the capture then ends cleanly."""
    import torch
    from paper_2609_05960_gb300 import gtpower
    lib, net, tr, bin_ps = case
    dev = _device_inputs(lib, net, tr)
    _noalloc(lib, tr, dev, bin_ps)  # the device's first call (set-up) outside capture
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            with pytest.raises(gtpower.GtpError) as ei:
                gtpower.gtp_run_power_noalloc(lib.n_in, lib.vdd, lib.slew_axis, lib.load_axis, dev["e_int"],
                                              dev["p_leak"], dev["cell"], dev["load_ff"], dev["slew_ps"],
                                              tr.window_ps, dev["gate_offsets"], dev["events"], dev["init_state"],
                                              bin_ps, stream=s.cuda_stream)
        finally:
            g.capture_end()
    assert ei.value.code == gtpower.GTP_EINVAL
