"""The oracle walk against the per-picosecond brute-force simulator, and the
invariants any correct walk must satisfy.  CPU only."""
import numpy as np
import pytest

import oracle
from oracle import brute
import synth
from cases import concat_netlists, permute_gates, small_random


@pytest.mark.parametrize("seed,tie_p,bin_ps", [(11, 0.0, 100), (12, 0.05, 50), (13, 0.3, 75), (14, 0.6, 1)])
def test_walk_matches_per_picosecond_brute_force(seed, tie_p, bin_ps):
    lib, net, tr = small_random(n_gates=7, n_events=250, window_ps=1500, seed=seed, tie_p=tie_p)
    rng = np.random.default_rng(seed)
    es = rng.uniform(0.5, 2.0, lib.n_cells)
    ls = rng.uniform(0.5, 2.0, lib.n_cells)
    got = oracle.walk(lib, net, tr, bin_ps, escale=es, lscale=ls)
    want = brute.simulate(lib, net, tr, bin_ps, escale=es, lscale=ls)
    np.testing.assert_allclose(got["bins"], want["bins"], rtol=1e-10, atol=1e-12)
    for k in ("e_leak", "e_int", "e_sw"):
        np.testing.assert_allclose(got[k], want[k], rtol=1e-10, atol=1e-12)
    np.testing.assert_array_equal(got["n_events"], want["n_events"])
    np.testing.assert_array_equal(got["final_state"], want["final_state"])


def test_brute_force_with_extrapolated_slews_and_loads():
    lib, net, tr = small_random(n_gates=5, n_events=120, window_ps=900, seed=21, tie_p=0.1)
    net.slew_ps[:, :, 0] = 2.0          # below the slew axis
    net.slew_ps[:, :, 1] = 500.0        # above it
    net.load_ff[::2] = 0.05             # below the load axis
    net.load_ff[1::2] = 30.0            # above it
    got = oracle.walk(lib, net, tr, 30)
    want = brute.simulate(lib, net, tr, 30)
    np.testing.assert_allclose(got["bins"], want["bins"], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(got["e_int"], want["e_int"], rtol=1e-10)


def _seeded(n_gates=300, n_events=20_000, window=200_000, seed=31, tie_p=0.01):
    return small_random(n_gates=n_gates, n_events=n_events, window_ps=window, seed=seed, tie_p=tie_p)


def test_bin_sum_equals_gate_sum():
    lib, net, tr = _seeded()
    out = oracle.walk(lib, net, tr, 100)
    total = out["e_leak"].sum() + out["e_int"].sum() + out["e_sw"].sum()
    assert out["bins"].sum() == pytest.approx(total, rel=1e-12)


def test_merging_fine_bins_gives_coarse_bins():
    lib, net, tr = _seeded()
    fine = oracle.walk(lib, net, tr, 50)["bins"]
    coarse = oracle.walk(lib, net, tr, 100)["bins"]
    np.testing.assert_allclose(fine.reshape(-1, 2).sum(1), coarse, rtol=1e-12, atol=1e-15)


def test_gate_order_permutation_invariance():
    lib, net, tr = _seeded(n_gates=120, n_events=8_000)
    perm = np.random.default_rng(3).permutation(net.n_gates)
    a = oracle.walk(lib, net, tr, 100)
    net2, tr2 = permute_gates(net, tr, perm)
    b = oracle.walk(lib, net2, tr2, 100)
    np.testing.assert_allclose(a["bins"], b["bins"], rtol=1e-12, atol=1e-15)
    for k in ("e_leak", "e_int", "e_sw", "final_state", "n_events"):
        np.testing.assert_array_equal(a[k][perm], b[k])


def test_superposition_of_netlists():
    lib = synth.make_library(1)
    _, netA, trA = small_random(n_gates=50, n_events=3000, window_ps=100_000, seed=41)
    _, netB, trB = small_random(n_gates=70, n_events=5000, window_ps=100_000, seed=42)
    net, tr = concat_netlists(lib, [(netA, trA), (netB, trB)])
    a = oracle.walk(lib, netA, trA, 100)["bins"]
    b = oracle.walk(lib, netB, trB, 100)["bins"]
    ab = oracle.walk(lib, net, tr, 100)["bins"]
    np.testing.assert_allclose(ab, a + b, rtol=1e-12, atol=1e-15)


def test_linearity_in_energy_and_leakage_scales():
    lib, net, tr = _seeded(n_gates=100, n_events=5000)
    rng = np.random.default_rng(7)
    es, ls = rng.uniform(0.5, 2, lib.n_cells), rng.uniform(0.5, 2, lib.n_cells)
    base = oracle.walk(lib, net, tr, 100, escale=es, lscale=ls)
    dbl = oracle.walk(lib, net, tr, 100, escale=2 * es, lscale=3 * ls)
    np.testing.assert_allclose(dbl["e_int"], 2 * base["e_int"], rtol=1e-14)
    np.testing.assert_allclose(dbl["e_leak"], 3 * base["e_leak"], rtol=1e-14)
    np.testing.assert_array_equal(dbl["e_sw"], base["e_sw"])
    z = np.zeros(lib.n_cells)
    parts = [oracle.walk(lib, net, tr, 100, escale=e, lscale=l)["bins"] for e, l in
             [(es, z), (z, ls), (z, z)]]
    np.testing.assert_allclose(base["bins"], parts[0] + parts[1] - parts[2], rtol=1e-12, atol=1e-14)


def test_sampled_bins_and_gate_subsets_match_full_walk():
    lib, net, tr = _seeded(n_gates=200, n_events=10_000)
    full = oracle.walk(lib, net, tr, 100)
    sample = np.array([0, 3, 17, 500, 1999])
    part = oracle.walk(lib, net, tr, 100, sample_bins=sample)
    np.testing.assert_allclose(part["bins"], full["bins"][sample], rtol=1e-13)
    gates = np.array([5, 0, 199, 42])
    sub = oracle.walk(lib, net, tr, 100, gates=gates, waveform=False)
    for k in ("e_leak", "e_int", "e_sw", "n_events", "final_state"):
        np.testing.assert_array_equal(sub[k], full[k][gates])
