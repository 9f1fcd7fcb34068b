"""Batched windows (one persistent launch, CUDA-graph replay), the adjoint
walk against the FP64 oracle adjoint, the autograd wrapper, and the
autotuner.  All through the C ABI on the GPU."""
import numpy as np
import pytest

import oracle
import synth
from cases import small_random

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def engine():
    from paper_2609_05960_gb300 import Engine
    e = Engine(0)
    yield e
    e.close()


def _reset(engine):
    for k in ("kernel", "records_per_thread", "dense_min", "ctas_per_sm", "tile_min", "piece_len", "group_bin_bytes"):
        engine.set_param(k, -1)


def _windows(net, n_win, seed0=100, bin_ps=20):
    """Windows of uneven length and density over one netlist."""
    rng = np.random.default_rng(seed0)
    out = []
    for w in range(n_win):
        n_bins = int(rng.integers(50, 3000))
        n_ev = int(rng.integers(0, 40_000)) if w % 5 else 0
        counts = synth.zipf_counts(net.n_gates, n_ev, 1.2, None, seed0 + w) if n_ev else np.zeros(net.n_gates, np.int64)
        tr = synth.make_trace(net, counts, n_bins * bin_ps, seed0 + w, tie_p=0.02 * (w % 3))
        out.append(tr)
    return out


@pytest.mark.parametrize("group_bytes,piece", [(1, -1), (20_000, -1), (20_000, 4096), (-1, 4096)])
def test_window_groups_match_oracle(engine, group_bytes, piece):
    """Windows walked group after group (group_bin_bytes 1: each window its
    own group; 20,000 B: groups of a few windows; the default: one group),
    with and without pieces, repeated (graph replay), against the oracle."""
    lib = synth.make_library(1)
    net = synth.make_netlist(lib, 300, seed=7)
    trs = _windows(net, 11, seed0=300)
    engine.load_library(lib)
    engine.load_netlist(net)
    _reset(engine)
    engine.set_param("group_bin_bytes", group_bytes)
    engine.set_param("piece_len", piece)
    for w, tr in enumerate(trs):
        engine.load_events(w, tr)
    order = [3, 0, 7, 1, 10, 2, 9, 4, 8, 5, 6]
    for it in range(3):
        waves = engine.run_power_batched(order, 20, graph=it > 0)
        n_groups = engine.get_param("run_groups")
        if group_bytes == 1:
            assert n_groups == len(order)
        elif group_bytes < 0:
            assert n_groups == 1
        else:
            assert 1 < n_groups < len(order)
        for k, w in enumerate(order):
            ref = oracle.walk(lib, net, trs[w], 20)
            want = oracle.waveform_w(ref["bins"], 20)
            got = waves[k].cpu().numpy()
            assert (np.abs(got - want) / np.abs(want)).max() <= TOL, f"window {w}"
            ge = engine.gate_energy(w, device=False)
            np.testing.assert_array_equal(ge["final_state"], ref["final_state"])
            np.testing.assert_array_equal(ge["n_events"], ref["n_events"])
            for key in ("e_leak", "e_int", "e_sw"):
                assert np.all(np.abs(ge[key] - ref[key]) <= TOL * np.abs(ref[key]) + 1e-9), (w, key)


@pytest.mark.parametrize("rpt", [4, 8, 16])
def test_batched_windows_match_oracle(engine, rpt):
    lib = synth.make_library(1)
    net = synth.make_netlist(lib, 300, seed=7)
    trs = _windows(net, 11)
    engine.load_library(lib)
    engine.load_netlist(net)
    _reset(engine)
    engine.set_param("records_per_thread", rpt)
    for w, tr in enumerate(trs):
        engine.load_events(w, tr)
    waves = engine.run_power_batched(list(range(len(trs))), 20)
    for w, tr in enumerate(trs):
        ref = oracle.walk(lib, net, tr, 20)
        want = oracle.waveform_w(ref["bins"], 20)
        got = waves[w].cpu().numpy()
        assert (np.abs(got - want) / np.abs(want)).max() <= TOL, f"window {w}"
        ge = engine.gate_energy(w, device=False)
        np.testing.assert_array_equal(ge["final_state"], ref["final_state"])
        np.testing.assert_array_equal(ge["n_events"], ref["n_events"])
        for k in ("e_leak", "e_int", "e_sw"):
            assert np.all(np.abs(ge[k] - ref[k]) <= TOL * np.abs(ref[k]) + 1e-9), (w, k)


def test_batched_graph_replay_and_single_runs_agree(engine):
    import torch
    lib = synth.make_library(1)
    net = synth.make_netlist(lib, 500, seed=8)
    trs = _windows(net, 7, seed0=200)
    engine.load_library(lib)
    engine.load_netlist(net)
    _reset(engine)
    for w, tr in enumerate(trs):
        engine.load_events(w, tr)
    ids = [3, 0, 6, 2, 5, 1, 4]
    outs = [torch.empty(trs[w].window_ps // 20, dtype=torch.float64, device=engine.device) for w in ids]
    engine.run_power_batched(ids, 20, outs=outs, graph=True)
    first = [o.clone() for o in outs]
    for o in outs:
        o.zero_()
    engine.run_power_batched(ids, 20, outs=outs, graph=True)  # replay
    for a, b, w in zip(first, outs, ids):
        ref = oracle.waveform_w(oracle.walk(lib, net, trs[w], 20)["bins"], 20)
        for x in (a, b):
            assert (np.abs(x.cpu().numpy() - ref) / ref).max() <= TOL
        single = engine.run_power(w, 20).cpu().numpy()
        assert (np.abs(single - ref) / ref).max() <= TOL


def _grad_close(got, want, rtol=1e-4):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    scale = np.abs(want).max() if want.size else 0.0
    bad = np.abs(got - want) > rtol * np.abs(want) + 1e-5 * scale
    assert not bad.any(), f"{bad.sum()} entries off; first {np.argmax(bad)}: got {got[np.argmax(bad)]} want {want[np.argmax(bad)]}"


@pytest.mark.parametrize("rpt", [4, 8, 16])
@pytest.mark.parametrize("tie_p", [0.0, 0.3])
def test_adjoint_matches_oracle_adjoint(engine, rpt, tie_p):
    import torch
    lib, net, tr = small_random(n_gates=400, n_events=60_000, window_ps=400_000, seed=61, tie_p=tie_p)
    bin_ps = 50
    engine.load_library(lib)
    engine.load_netlist(net)
    _reset(engine)
    engine.set_param("records_per_thread", rpt)
    rng = np.random.default_rng(1)
    es = rng.uniform(0.5, 2.0, lib.n_cells).astype(np.float32)
    ls = rng.uniform(0.5, 2.0, lib.n_cells).astype(np.float32)
    engine.set_scales(es, ls)
    engine.load_events(0, tr)
    engine.run_power(0, bin_ps)
    n_bins = tr.window_ps // bin_ps
    w = rng.normal(size=n_bins).astype(np.float32) * 1e3
    dC, de, dl = engine.run_power_backward(0, bin_ps, torch.from_numpy(w).to(engine.device))
    rC, rde, rdl = oracle.adjoint(lib, net, tr, bin_ps, w.astype(np.float64), escale=es.astype(np.float64),
                                  lscale=ls.astype(np.float64))
    _grad_close(dC.cpu().numpy(), rC)
    _grad_close(de.cpu().numpy(), rde)
    _grad_close(dl.cpu().numpy(), rdl)


def test_autograd_peak_loss_matches_oracle(engine):
    import torch
    from paper_2609_05960_gb300 import peak_loss, power_waveform
    lib, net, tr = small_random(n_gates=300, n_events=50_000, window_ps=300_000, seed=62, tie_p=0.01)
    bin_ps = 100
    engine.load_library(lib)
    engine.load_netlist(net)
    _reset(engine)
    engine.load_events(0, tr)
    dev = engine.device
    C = torch.tensor(net.load_ff, dtype=torch.float32, device=dev, requires_grad=True)
    es = torch.ones(lib.n_cells, dtype=torch.float32, requires_grad=True)
    ls = torch.ones(lib.n_cells, dtype=torch.float32, requires_grad=True)
    P = power_waveform(engine, 0, bin_ps, C, es, ls)
    P.retain_grad()
    loss = peak_loss(P)
    loss.backward()
    Pr = oracle.waveform_w(oracle.walk(lib, net, tr, bin_ps)["bins"], bin_ps)
    assert (np.abs(P.detach().cpu().numpy() - Pr) / Pr).max() <= TOL
    # the loss gradient at the GPU waveform, pushed through the FP64 oracle adjoint
    dLdP = P.grad.cpu().numpy()
    rC, rde, rdl = oracle.adjoint(lib, net, tr, bin_ps, dLdP.astype(np.float32).astype(np.float64))
    _grad_close(C.grad.cpu().numpy(), rC, rtol=2e-4)
    _grad_close(es.grad.numpy(), rde, rtol=2e-4)
    _grad_close(ls.grad.numpy(), rdl, rtol=2e-4)


def test_adjoint_gate_without_events_and_window_without_events(engine):
    import torch
    lib = synth.make_library(1)
    net = synth.make_netlist(lib, 40, seed=9)
    counts = np.zeros(40, np.int64)
    counts[[2, 7]] = [30, 5]
    tr = synth.make_trace(net, counts, 20_000, seed=3)
    tr0 = synth.make_trace(net, np.zeros(40, np.int64), 20_000, seed=4)
    engine.load_library(lib)
    engine.load_netlist(net)
    _reset(engine)
    for wi, t in ((0, tr), (1, tr0)):
        engine.load_events(wi, t)
        engine.run_power(wi, 100)
        g = np.linspace(1, 2, 200).astype(np.float32)
        dC, de, dl = engine.run_power_backward(wi, 100, torch.from_numpy(g).to(engine.device))
        rC, rde, rdl = oracle.adjoint(lib, net, t, 100, g.astype(np.float64))
        _grad_close(dC.cpu().numpy(), rC)
        _grad_close(de.cpu().numpy(), rde)
        _grad_close(dl.cpu().numpy(), rdl)


def test_autotune_picks_a_valid_plan(engine):
    lib, net, tr = small_random(n_gates=2000, n_events=300_000, window_ps=1_000_000, seed=63)
    engine.load_library(lib)
    engine.load_netlist(net)
    _reset(engine)
    engine.load_events(0, tr)
    ms = engine.autotune([0], 100, iters=2)
    assert ms > 0
    assert engine.get_param("records_per_thread") in (4, 8, 16)
    assert engine.get_param("dense_min") in (64, 256, 512, 1024)
    w = engine.run_power(0, 100).cpu().numpy()
    ref = oracle.waveform_w(oracle.walk(lib, net, tr, 100)["bins"], 100)
    assert (np.abs(w - ref) / ref).max() <= TOL


def test_single_window_graph_follows_reloads_and_times_phases(engine):
    """A captured single-window run is replayed only while the launch sizes
    it holds still apply: reloading the window with another length or with no
    events gives a new graph, and every run matches the oracle.  Phase timing
    recorded inside the graph accumulates once per replay."""
    lib = synth.make_library(1)
    net = synth.make_netlist(lib, 300, seed=12)
    engine.load_library(lib)
    engine.load_netlist(net)
    _reset(engine)
    specs = [(2500, 30_000), (2500, 30_000), (7000, 50_000), (400, 0), (7000, 20_000)]
    for i, (n_bins, n_ev) in enumerate(specs):
        counts = synth.zipf_counts(net.n_gates, n_ev, 1.2, None, 300 + i) if n_ev else np.zeros(net.n_gates, np.int64)
        tr = synth.make_trace(net, counts, n_bins * 20, 300 + i, tie_p=0.05)
        engine.load_events(0, tr)
        ref = oracle.waveform_w(oracle.walk(lib, net, tr, 20)["bins"], 20)
        for _ in range(2):
            got = engine.run_power(0, 20, graph=True).cpu().numpy()
            assert got.shape == ref.shape
            assert (np.abs(got - ref) / ref).max() <= TOL, (i, n_bins, n_ev)
    engine.set_param("timing", 1)
    for _ in range(3):
        engine.run_power(0, 20, graph=True)
    assert engine.get_param("n_timed") == 3
    assert engine.get_param("t_walk_ns") > 0 and engine.get_param("t_merge_ns") > 0
    engine.set_param("timing", 1)  # and on the stream, without a graph
    got = engine.run_power(0, 20).cpu().numpy()
    assert (np.abs(got - ref) / ref).max() <= TOL
    assert engine.get_param("n_timed") == 1 and engine.get_param("t_walk_ns") > 0
    engine.set_param("timing", 0)


@pytest.mark.parametrize("staged", [0, 1])
@pytest.mark.parametrize("rpt", [4, 8, 16])
def test_adjoint_gate_table_placements_match_oracle(engine, staged, rpt):
    """Both adjoint builds (sparse threads' gate tables in place or staged in
    shared memory) against the FP64 oracle adjoint, with whole and split gates."""
    import torch
    lib, net, tr = small_random(n_gates=300, n_events=80_000, window_ps=400_000, seed=63, tie_p=0.05, zipf_s=1.4)
    bin_ps = 50
    engine.load_library(lib)
    engine.load_netlist(net)
    _reset(engine)
    engine.set_param("records_per_thread", rpt)
    engine.set_param("bwd_staged", staged)
    rng = np.random.default_rng(2)
    es = rng.uniform(0.5, 2.0, lib.n_cells).astype(np.float32)
    ls = rng.uniform(0.5, 2.0, lib.n_cells).astype(np.float32)
    engine.set_scales(es, ls)
    engine.load_events(0, tr)
    w = rng.normal(size=tr.window_ps // bin_ps).astype(np.float32) * 1e3
    rC, rde, rdl = oracle.adjoint(lib, net, tr, bin_ps, w.astype(np.float64), escale=es.astype(np.float64),
                                  lscale=ls.astype(np.float64))
    for piece_len in (-1, 4096):  # -1: no gate split; 4096: the busiest gates in pieces
        engine.set_param("piece_len", piece_len)
        dC, de, dl = engine.run_power_backward(0, bin_ps, torch.from_numpy(w).to(engine.device))
        _grad_close(dC.cpu().numpy(), rC)
        _grad_close(de.cpu().numpy(), rde)
        _grad_close(dl.cpu().numpy(), rdl)
    engine.set_param("bwd_staged", -1)
    engine.set_param("piece_len", -1)
    engine.set_scales(None, None)
