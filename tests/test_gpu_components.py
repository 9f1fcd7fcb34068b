"""Per-component waveforms (leakage, internal, switching, glitch; Sec. 2.2)
on the GPU against the FP64 oracle, through the C ABI, for every walk (one
thread per gate, the density-split walk at three segment lengths), with and
without glitch detection.

Bar: each component's bins within 1e-5 relative of the oracle's (a component
that is zero in a bin must be zero there, up to 1e-9 of that component's
largest bin), the total equal to the plain run's, and the per-gate results
as for the plain walk."""
import numpy as np
import pytest

import oracle
import synth
from cases import small_random

pytestmark = pytest.mark.gpu

TOL = 1e-5
KERNELS = [
    dict(kernel=1),
    dict(kernel=0, records_per_thread=4, dense_min=16),
    dict(kernel=0, records_per_thread=8),
    dict(kernel=0, records_per_thread=16, dense_min=64),
]
KID = ["per_gate", "seg_k4", "seg_k8", "seg_k16"]
NAMES = ("leakage", "internal", "switching", "glitch")


@pytest.fixture(scope="module")
def engine():
    from paper_2609_05960_gb300 import Engine
    e = Engine(0)
    yield e
    e.close()


def _setup(engine, lib, net, params):
    engine.load_library(lib)
    engine.load_netlist(net)
    for k in ("kernel", "records_per_thread", "dense_min", "ctas_per_sm", "tile_min", "piece_len", "group_bin_bytes"):
        engine.set_param(k, -1)
    for k, v in (params or {}).items():
        engine.set_param(k, v)


def _check_components(got, ref, bin_ps):
    want = oracle.waveform_w(ref["comp_bins"], bin_ps)
    for k, name in enumerate(NAMES):
        err = np.abs(got[k] - want[k])
        bad = err > TOL * np.abs(want[k]) + 1e-9 * max(np.abs(want[k]).max(), 1e-30)
        assert not bad.any(), f"{name}: bin {np.argmax(bad)} got {got[k][np.argmax(bad)]} want {want[k][np.argmax(bad)]}"


@pytest.mark.parametrize("params", KERNELS, ids=KID)
@pytest.mark.parametrize("clock", [0, 400])
def test_components_match_oracle(engine, params, clock):
    lib, net, tr = small_random(n_gates=300, n_events=60_000, window_ps=300_000, seed=81, tie_p=0.05, zipf_s=1.3)
    out_slew = np.random.default_rng(81).uniform(5.0, 150.0, (net.n_gates, 2)).astype(np.float32)
    _setup(engine, lib, net, params)
    engine.set_glitch(clock, out_slew if clock else None)
    engine.load_events(0, tr)
    import torch
    total = torch.empty(tr.window_ps // 50, dtype=torch.float64, device=engine.device)
    comp = engine.run_power_components(0, 50, total=total).cpu().numpy()
    ref = oracle.walk(lib, net, tr, 50, glitch=(clock, out_slew) if clock else None, components=True)
    _check_components(comp, ref, 50)
    if clock == 0:
        assert not comp[3].any()
    else:
        assert comp[3].sum() > 0
    # the total is the plain run's, and the components add up to it
    want_total = oracle.waveform_w(ref["bins"], 50)
    assert (np.abs(total.cpu().numpy() - want_total) / want_total).max() <= TOL
    np.testing.assert_allclose(comp.sum(0), total.cpu().numpy(), rtol=2e-6)
    ge = engine.gate_energy(0, device=False)
    np.testing.assert_array_equal(ge["n_events"], ref["n_events"])
    np.testing.assert_array_equal(ge["final_state"], ref["final_state"])
    engine.set_glitch(0)


def test_components_on_host_then_a_plain_run(engine):
    """Host outputs; a plain run afterwards is unaffected (graph replay
    included)."""
    import torch
    lib, net, tr = small_random(n_gates=500, n_events=80_000, window_ps=200_000, seed=82, tie_p=0.02)
    _setup(engine, lib, net, None)
    engine.load_events(2, tr)
    comp = np.empty((4, tr.window_ps // 40))
    total = np.empty(tr.window_ps // 40)
    engine.run_power_components(2, 40, out=comp, total=total)
    ref = oracle.walk(lib, net, tr, 40, components=True)
    _check_components(comp, ref, 40)
    plain = torch.empty(tr.window_ps // 40, dtype=torch.float64, device=engine.device)
    engine.run_power(2, 40, out=plain, graph=True)
    np.testing.assert_allclose(plain.cpu().numpy(), total, rtol=2e-6)
    engine.run_power(2, 40, out=plain, graph=True)
    np.testing.assert_allclose(plain.cpu().numpy(), total, rtol=2e-6)


def test_components_tiny_workload(engine):
    """The tiny workload (2,000 gates, 200k events, 10k bins) element by
    element."""
    lib, net, tr = synth.make_inputs(synth.CONFIGS["tiny"])
    _setup(engine, lib, net, None)
    engine.load_events(0, tr)
    comp = engine.run_power_components(0, 100).cpu().numpy()
    _check_components(comp, oracle.walk(lib, net, tr, 100, components=True), 100)


def test_components_reject_graph_replay_and_a_missing_output(engine):
    import torch
    from paper_2609_05960_gb300 import GtpError, gtpower
    lib, net, tr = small_random(n_gates=20, n_events=500, window_ps=5_000, seed=83)
    _setup(engine, lib, net, None)
    engine.load_events(0, tr)
    with pytest.raises(GtpError) as ei:
        gtpower.gtp_run_power_components(engine.ctx, 0, 100, None)
    assert ei.value.code == gtpower.GTP_EINVAL
    comp = torch.empty((4, 50), dtype=torch.float64, device=engine.device)
    rc = gtpower.load().gtp_run_power_components(engine.ctx, 0, 100, None, comp.data_ptr(),
                                                 gtpower.GTP_DEVICE | gtpower.GTP_GRAPH)
    assert rc == gtpower.GTP_EINVAL
