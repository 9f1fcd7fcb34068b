"""Pins for the FP64 oracle adjoint: central finite differences of the
oracle forward, exact linearity in the scales, and the switching-energy
derivative.  CPU only."""
import numpy as np
import pytest

import oracle
import synth
from cases import netlist_from, single_cell_library, small_random, trace_from


def _loss_linear(w, bins, bin_ps):
    return float(np.dot(w, oracle.waveform_w(bins, bin_ps)))


def _away_from_knots(C):
    """Move loads off the load-axis knots so that a +-0.1% step stays in one segment."""
    la = np.array(synth.LOAD_AXIS_FF, np.float64)
    C = np.asarray(C, np.float64).copy()
    for k in la:
        near = np.abs(C - k) < 0.01 * k
        C[near] = k * 1.03
    return C


def test_adjoint_dC_matches_central_differences_linear_loss():
    lib, net, tr = small_random(n_gates=25, n_events=3000, window_ps=50_000, seed=51, tie_p=0.02)
    bin_ps = 100
    C = _away_from_knots(net.load_ff)
    w = np.random.default_rng(0).normal(size=tr.window_ps // bin_ps)
    dC, _, _ = oracle.adjoint(lib, net, tr, bin_ps, w, load_ff=C)
    for g in range(net.n_gates):
        h = 1e-3 * C[g]
        Cp, Cm = C.copy(), C.copy()
        Cp[g] += h
        Cm[g] -= h
        lp = _loss_linear(w, oracle.walk(lib, net, tr, bin_ps, load_ff=Cp)["bins"], bin_ps)
        lm = _loss_linear(w, oracle.walk(lib, net, tr, bin_ps, load_ff=Cm)["bins"], bin_ps)
        assert dC[g] == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-12)


def test_adjoint_dC_matches_central_differences_peak_loss():
    """Loss = sum P^2 + tau * log sum exp(P / tau), tau = 0.01 * mean(P) held fixed."""
    lib, net, tr = small_random(n_gates=12, n_events=1500, window_ps=20_000, seed=52, tie_p=0.02)
    bin_ps = 50
    C = _away_from_knots(net.load_ff)

    def loss(bins):
        P = oracle.waveform_w(bins, bin_ps) * 1e3  # mW keeps both terms O(1)
        return float(np.sum(P * P) + tau * np.log(np.sum(np.exp((P - P.max()) / tau))) + P.max())

    P0 = oracle.waveform_w(oracle.walk(lib, net, tr, bin_ps, load_ff=C)["bins"], bin_ps) * 1e3
    tau = 0.01 * P0.mean()
    soft = np.exp((P0 - P0.max()) / tau)
    soft /= soft.sum()
    dLdP = (2 * P0 + soft) * 1e3  # dL/dP in W
    dC, _, _ = oracle.adjoint(lib, net, tr, bin_ps, dLdP, load_ff=C)
    for g in range(net.n_gates):
        h = 1e-3 * C[g]
        Cp, Cm = C.copy(), C.copy()
        Cp[g] += h
        Cm[g] -= h
        fd = (loss(oracle.walk(lib, net, tr, bin_ps, load_ff=Cp)["bins"])
              - loss(oracle.walk(lib, net, tr, bin_ps, load_ff=Cm)["bins"])) / (2 * h)
        assert dC[g] == pytest.approx(fd, rel=2e-3, abs=1e-9)


def test_adjoint_scales_are_exact_by_linearity():
    lib, net, tr = small_random(n_gates=40, n_events=4000, window_ps=40_000, seed=53)
    bin_ps = 100
    w = np.random.default_rng(1).normal(size=tr.window_ps // bin_ps)
    es = np.ones(lib.n_cells)
    ls = np.ones(lib.n_cells)
    _, de, dl = oracle.adjoint(lib, net, tr, bin_ps, w, escale=es, lscale=ls)
    z = np.zeros(lib.n_cells)
    base = _loss_linear(w, oracle.walk(lib, net, tr, bin_ps, escale=z, lscale=z)["bins"], bin_ps)
    for c in range(lib.n_cells):
        e = np.zeros(lib.n_cells)
        e[c] = 1.0
        le = _loss_linear(w, oracle.walk(lib, net, tr, bin_ps, escale=e, lscale=z)["bins"], bin_ps)
        ll = _loss_linear(w, oracle.walk(lib, net, tr, bin_ps, escale=z, lscale=e)["bins"], bin_ps)
        assert de[c] == pytest.approx(le - base, rel=1e-9, abs=1e-15)
        assert dl[c] == pytest.approx(ll - base, rel=1e-9, abs=1e-15)


def test_switching_energy_derivative_is_half_vdd_squared():
    lib = single_cell_library(1, lambda *a: 0.0, lambda s: 5.0, vdd=0.8)
    net = netlist_from(lib, [0], [2.0])
    tr = trace_from([[(110, 1, 1), (290, 1, 0), (310, 1, 1)]], [0], 400)
    w = np.array([1.0, 2.0, 3.0, 4.0])
    dC, _, _ = oracle.adjoint(lib, net, tr, 100, w)
    vdd = lib.vdd
    assert dC[0] == pytest.approx((2.0 + 3.0 + 4.0) * 0.5 * vdd * vdd * 1e-3 / 100, rel=1e-14)
