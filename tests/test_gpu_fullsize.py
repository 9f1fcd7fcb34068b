"""Full-size workloads on the GPU, in the launch configuration the benchmark
times, against the FP64 oracle on every bin and every gate.  The oracle runs
over the whole workload on every host core (oracle/fullsize.py: gate ranges
in spawned processes, each regenerating its gates' records from the seeds,
with the range-mode leakage split), so every waveform bin is compared within
1e-5 relative and every gate's count and final state bit-exactly, its
energies within 1e-5.  Invariants that hold at any size are checked too: sum
over bins = sum over gates, and merging pairs of fine bins = coarse bins.

Workloads (synthetic, seeded; see synth.CONFIGS):
  large    1M gates, 200M events, Zipf 1.2 cap 1e5, 10 us, 10 ps bins
  adjoint  500k gates, 100M events, 5 us, 10 ps bins
  batched  200k gates, 64 windows of 1k-100k bins and 1M-20M events
  stress   10M gates, 2B events (16 GB), Zipf 1.5 cap 1e7, 100 us, 10 ps bins
"""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from oracle import fullsize

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = 1e-5


@pytest.fixture(scope="module")
def opool():
    p = fullsize.Pool()
    yield p
    p.close()


def _full_check(wave, ge, ref, bin_ps, e_gl=None):
    """Every bin within TOL relative; every gate's count and final state
    exact and energies within TOL (1e-9 fJ floor)."""
    err = fullsize.bin_errors(wave.cpu().numpy() if hasattr(wave, "cpu") else wave, ref["bins"], bin_ps)
    assert err["max_rel_bin_err"] <= TOL, err
    got = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in ge.items()}
    if e_gl is not None:
        got["e_gl"] = e_gl.cpu().numpy() if hasattr(e_gl, "cpu") else e_gl
    ge_err = fullsize.gate_errors(got, ref, ("e_leak", "e_int", "e_sw") + (("e_gl",) if e_gl is not None else ()))
    assert ge_err["count_mismatches"] == 0 and ge_err["state_mismatches"] == 0, ge_err
    for k, v in ge_err.items():
        if k.startswith("max_rel"):
            assert v <= TOL, ge_err
    return err


@pytest.fixture(scope="module")
def engine():
    from paper_2609_05960_gb300 import Engine
    e = Engine(0)
    yield e
    e.close()


def _gpu_trace(engine, net, cfg, counts, seed=None):
    import torch
    tr, rec = synth.make_trace_gpu(net, counts, cfg.window_ps, cfg.seed_ev if seed is None else seed, cfg.tie_p,
                                   device=engine.device)
    off = torch.from_numpy(tr.offsets).to(engine.device)
    init = torch.from_numpy(tr.init_state).to(engine.device)
    return tr, rec, off, init


def _sample_gates(counts, n_random=1500, n_hot=16, seed=0):
    rng = np.random.default_rng(seed)
    hot = np.argsort(-counts, kind="stable")[:n_hot]
    empty = np.flatnonzero(counts == 0)[:8]
    rnd = rng.choice(len(counts), size=min(n_random, len(counts)), replace=False)
    return np.unique(np.concatenate([hot, empty, rnd]))


def _oracle_gates(lib, net, tr, gates, bin_ps):
    off, rec = synth.gate_records(net, tr, gates)
    sub_net = synth.Netlist(net.cell[gates], net.load_ff[gates], np.ascontiguousarray(net.slew_ps[gates]),
                            net.n_pins[gates], net.level[gates], net.fanin[gates])
    sub_tr = synth.Trace(tr.window_ps, off, rec, tr.init_state[gates], tr.seed, tr.tie24)
    return sub_net, sub_tr, oracle.walk(lib, sub_net, sub_tr, bin_ps, waveform=False)


def _check_gates(ge, ref, gates):
    got = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v)[gates] for k, v in ge.items()}
    np.testing.assert_array_equal(got["n_events"], ref["n_events"])
    np.testing.assert_array_equal(got["final_state"], ref["final_state"])
    for k in ("e_leak", "e_int", "e_sw"):
        err = np.abs(got[k] - ref[k])
        bad = err > TOL * np.abs(ref[k]) + 1e-9
        assert not bad.any(), f"{k}: gate {gates[np.argmax(bad)]} got {got[k][np.argmax(bad)]} want {ref[k][np.argmax(bad)]}"


def _totals_agree(wave, ge, bin_ps):
    e_bins = float((wave.double() * (bin_ps * 1e3)).sum())
    e_gates = float(ge["e_leak"].sum() + ge["e_int"].sum() + ge["e_sw"].sum())
    assert e_bins == pytest.approx(e_gates, rel=1e-6)


def _defaults(engine):
    for k in ("kernel", "records_per_thread", "dense_min", "ctas_per_sm", "tile_min", "piece_len", "group_bin_bytes"):
        engine.set_param(k, -1)


def test_large_full_size(engine, opool):
    cfg = synth.CONFIGS["large"]
    lib = synth.make_library(cfg.seed_lib)
    net = synth.make_netlist(lib, cfg.n_gates, cfg.seed_net)
    counts = synth.zipf_counts(cfg.n_gates, cfg.n_events, cfg.zipf_s, cfg.cap, cfg.seed_ev)
    engine.load_library(lib)
    engine.load_netlist(net)
    _defaults(engine)
    tr, rec, off, init = _gpu_trace(engine, net, cfg, counts)
    engine.load_events(0, window_ps=cfg.window_ps, offsets=off, records=rec, init_state=init, borrow=True)
    wave = engine.run_power(0, cfg.bin_ps, graph=False)
    ge = engine.gate_energy(0, device=True)
    assert engine.get_param("dense_min") == 512  # chosen for 200M events (1.3M an SM): the run above walks it
    # the GPU generator writes the host generator's bits
    host = synth.gate_records(net, tr, np.arange(4))[1]
    assert np.array_equal(host, rec[:len(host)].cpu().numpy().view(np.uint32))
    ref = opool.walk(fullsize.Workload.of(cfg), cfg.bin_ps)
    _full_check(wave, ge, ref, cfg.bin_ps)
    _totals_agree(wave, ge, cfg.bin_ps)
    # coarse bins = merged fine bins
    wave2 = engine.run_power(0, 2 * cfg.bin_ps)
    np.testing.assert_allclose(wave.view(-1, 2).mean(1).cpu().numpy(), wave2.cpu().numpy(), rtol=TOL)


def test_large_full_size_with_glitches(engine, opool):
    """Large with clock-cycle glitch detection at a 1 GHz clock: every bin and
    every gate (glitch energy included) against the oracle, and the totals
    over bins and gates."""
    cfg = synth.CONFIGS["large"]
    lib = synth.make_library(cfg.seed_lib)
    net = synth.make_netlist(lib, cfg.n_gates, cfg.seed_net)
    counts = synth.zipf_counts(cfg.n_gates, cfg.n_events, cfg.zipf_s, cfg.cap, cfg.seed_ev)
    wl = fullsize.Workload.of(cfg, clock_ps=1000)
    out_slew = np.random.default_rng(wl.out_slew_seed).uniform(*wl.out_slew_range, (cfg.n_gates, 2)).astype(np.float32)
    engine.load_library(lib)
    engine.load_netlist(net)
    _defaults(engine)
    engine.set_glitch(1000, out_slew)
    tr, rec, off, init = _gpu_trace(engine, net, cfg, counts)
    engine.load_events(0, window_ps=cfg.window_ps, offsets=off, records=rec, init_state=init, borrow=True)
    wave = engine.run_power(0, cfg.bin_ps)
    ge = engine.gate_energy(0, device=True)
    e_gl = engine.gate_glitch(0, device=True)
    ref = opool.walk(wl, cfg.bin_ps)
    assert ref["e_gl"].sum() > 0
    _full_check(wave, ge, ref, cfg.bin_ps, e_gl=e_gl)
    e_bins = float((wave.double() * (cfg.bin_ps * 1e3)).sum())
    e_gates = float(ge["e_leak"].sum() + ge["e_int"].sum() + ge["e_sw"].sum() + e_gl.sum())
    assert e_bins == pytest.approx(e_gates, rel=1e-6)
    engine.set_glitch(0)


def test_adjoint_full_size(engine, opool):
    import torch
    from paper_2609_05960_gb300 import peak_loss
    cfg = synth.CONFIGS["adjoint"]
    lib = synth.make_library(cfg.seed_lib)
    net = synth.make_netlist(lib, cfg.n_gates, cfg.seed_net)
    counts = synth.zipf_counts(cfg.n_gates, cfg.n_events, cfg.zipf_s, cfg.cap, cfg.seed_ev)
    engine.load_library(lib)
    engine.load_netlist(net)
    _defaults(engine)
    tr, rec, off, init = _gpu_trace(engine, net, cfg, counts)
    engine.load_events(0, window_ps=cfg.window_ps, offsets=off, records=rec, init_state=init, borrow=True)
    P = engine.run_power(0, cfg.bin_ps).clone().requires_grad_(True)
    # the forward waveform and per-gate results, in full, against the oracle
    _full_check(P.detach(), engine.gate_energy(0, device=True), opool.walk(fullsize.Workload.of(cfg), cfg.bin_ps),
                cfg.bin_ps)
    peak_loss(P).backward()
    g = P.grad.to(torch.float32)
    dC, de, dl = engine.run_power_backward(0, cfg.bin_ps, g)
    # per-gate load gradients of sampled gates against the FP64 oracle adjoint
    gates = _sample_gates(counts, n_random=600, n_hot=8)
    sub_net, sub_tr, _ = _oracle_gates(lib, net, tr, gates, cfg.bin_ps)
    rC, _, _ = oracle.adjoint(lib, sub_net, sub_tr, cfg.bin_ps, g.cpu().numpy().astype(np.float64))
    got = dC.cpu().numpy()[gates]
    scale = np.abs(rC).max()
    assert np.all(np.abs(got - rC) <= 1e-4 * np.abs(rC) + 1e-5 * scale)
    # cell-scale gradients: the waveform is linear in each scale, so for the
    # linear functional w.P with w = dL/dP, dL/ds_c = w.(P(s = e_c) - P(s = 0))
    w = g.double()
    z = np.zeros(lib.n_cells, np.float32)
    engine.set_scales(z, z)
    base = float((engine.run_power(0, cfg.bin_ps) * w).sum())
    for c in range(lib.n_cells):
        e = z.copy()
        e[c] = 1.0
        engine.set_scales(e, z)
        ge_ = float((engine.run_power(0, cfg.bin_ps) * w).sum()) - base
        engine.set_scales(z, e)
        gl_ = float((engine.run_power(0, cfg.bin_ps) * w).sum()) - base
        assert float(de[c]) == pytest.approx(ge_, rel=1e-4)
        assert float(dl[c]) == pytest.approx(gl_, rel=1e-4)
    engine.set_scales(None, None)


def test_batched_full_size(engine, opool):
    """All 64 windows of the batched workload, replayed from a CUDA graph:
    every bin and every gate of every window against the oracle."""
    import torch
    lib = synth.make_library(1)
    net = synth.make_netlist(lib, synth.BATCHED_GATES, 2)
    wins = synth.batched_windows()
    engine.load_library(lib)
    engine.load_netlist(net)
    _defaults(engine)
    keep = []
    cfgs = []
    for w, spec in enumerate(wins):
        cfg = synth.Config(f"w{w}", synth.BATCHED_GATES, spec["n_events"], 1.2, 100_000, spec["window_ps"], 10,
                           seed_ev=spec["seed"])
        counts = synth.zipf_counts(cfg.n_gates, cfg.n_events, 1.2, 100_000, cfg.seed_ev)
        tr, rec, off, init = _gpu_trace(engine, net, cfg, counts)
        engine.load_events(w, window_ps=cfg.window_ps, offsets=off, records=rec, init_state=init, borrow=True)
        keep.append((rec, off, init))
        cfgs.append(cfg)
    ids = list(range(len(wins)))
    outs = [torch.empty(s["window_ps"] // 10, dtype=torch.float64, device=engine.device) for s in wins]
    engine.run_power_batched(ids, 10, outs=outs, graph=True)
    engine.run_power_batched(ids, 10, outs=outs, graph=True)  # graph replay
    worst = 0.0
    for w in ids:
        ge = engine.gate_energy(w, device=True)
        _totals_agree(outs[w], ge, 10)
        err = _full_check(outs[w], ge, opool.walk(fullsize.Workload.of(cfgs[w]), 10), 10)
        worst = max(worst, err["max_rel_bin_err"])
    assert worst <= TOL


def test_stress_full_size(engine, opool):
    """Stress (10M gates, 2B events, 10M bins): every bin and every gate
    against the oracle in the plain form, sampled load gradients in the
    adjoint form, and every bin and gate of each window in the batched form
    (four windows of 500M events)."""
    import torch
    cfg = synth.CONFIGS["stress"]
    lib = synth.make_library(cfg.seed_lib)
    net = synth.make_netlist(lib, cfg.n_gates, cfg.seed_net)
    counts = synth.zipf_counts(cfg.n_gates, cfg.n_events, cfg.zipf_s, cfg.cap, cfg.seed_ev)
    engine.load_library(lib)
    engine.load_netlist(net)
    _defaults(engine)
    tr, rec, off, init = _gpu_trace(engine, net, cfg, counts)
    engine.load_events(0, window_ps=cfg.window_ps, offsets=off, records=rec, init_state=init, borrow=True)
    wave = engine.run_power(0, cfg.bin_ps)
    ge = engine.gate_energy(0, device=True)
    _full_check(wave, ge, opool.walk(fullsize.Workload.of(cfg), cfg.bin_ps), cfg.bin_ps)
    _totals_agree(wave, ge, cfg.bin_ps)
    # adjoint form on the same window: sampled load gradients
    g = torch.linspace(1.0, 2.0, wave.numel(), device=engine.device, dtype=torch.float32)
    dC, de, dl = engine.run_power_backward(0, cfg.bin_ps, g)
    few = _sample_gates(counts, n_random=400, n_hot=4)[:40]
    sub_net, sub_tr, _ = _oracle_gates(lib, net, tr, few, cfg.bin_ps)
    rC, _, _ = oracle.adjoint(lib, sub_net, sub_tr, cfg.bin_ps, g.cpu().numpy().astype(np.float64))
    got = dC.cpu().numpy()[few]
    assert np.all(np.abs(got - rC) <= 1e-4 * np.abs(rC) + 1e-5 * np.abs(rC).max())
    del rec, off, init, wave
    torch.cuda.empty_cache()
    # batched form: 4 windows of 500M events
    keep = []
    cfgs = []
    for w in range(4):
        c4 = dataclasses.replace(cfg, n_events=cfg.n_events // 4, seed_ev=cfg.seed_ev + 10 * (w + 1))
        cnt = synth.zipf_counts(c4.n_gates, c4.n_events, c4.zipf_s, c4.cap, c4.seed_ev)
        t4, r4, o4, i4 = _gpu_trace(engine, net, c4, cnt)
        engine.load_events(w, window_ps=c4.window_ps, offsets=o4, records=r4, init_state=i4, borrow=True)
        keep.append((r4, o4, i4))
        cfgs.append(c4)
    outs = engine.run_power_batched([0, 1, 2, 3], cfg.bin_ps)
    for w in range(4):
        ge = engine.gate_energy(w, device=True)
        _totals_agree(outs[w], ge, cfg.bin_ps)
        _full_check(outs[w], ge, opool.walk(fullsize.Workload.of(cfgs[w]), cfg.bin_ps), cfg.bin_ps)
