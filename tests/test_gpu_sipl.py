"""A library given as Liberty-style state patterns (Sec. 4.1): expanded on
the host by gtp_sipl_expand, loaded, and walked on the GPU, against the
oracle walking the library its traversal builds.  Bar as for the plain walk."""
import numpy as np
import pytest

import oracle
import synth
from oracle import sipl

pytestmark = pytest.mark.gpu

TOL = 1e-5
NS, NL = len(synth.SLEW_AXIS_PS), len(synth.LOAD_AXIS_FF)


def _cells(rng):
    """A multiplexer (pins A, B, S, Y) with conditions on the select pin, and
    a 5-input cell with random overlapping, partly don't-care patterns."""
    tab = lambda lo, hi: rng.uniform(lo, hi, (NS, NL)).astype(np.float32)
    mux = (3, [(0, -1, 0b100, 0b000, tab(1, 2)), (0, -1, 0b100, 0b100, tab(2, 3)), (1, 1, 0b100, 0b100, tab(3, 4))],
           rng.uniform(0.5, 5.0, (3, 2, NS, NL)).astype(np.float32),
           [(0b0011, 0, 7.0), (0b1000, 0b1000, 9.0)], 1.0)
    n_in = 5
    ip = []
    for _ in range(14):
        pin = int(rng.integers(0, n_in))
        allowed = ((1 << n_in) - 1) & ~(1 << pin)
        care = int(rng.integers(0, allowed + 1)) & allowed
        ip.append((pin, int(rng.integers(-1, 2)), care, int(rng.integers(0, 1 << n_in)) & care, tab(0.5, 5.0)))
    lp = [(int(c), int(v) & int(c), float(rng.uniform(1, 50))) for c, v in rng.integers(0, 64, (20, 2))]
    wide = (n_in, ip, rng.uniform(0.5, 5.0, (n_in, 2, NS, NL)).astype(np.float32), lp, 3.0)
    return [mux, wide]


def _library(cells, expand):
    e, l = zip(*[expand(n, NS, NL, ip, d, lp, ld) for n, ip, d, lp, ld in cells])
    return synth.Library([f"C{i}" for i in range(len(cells))], np.array([c[0] for c in cells], np.int32),
                         float(np.float32(synth.VDD)), np.array(synth.SLEW_AXIS_PS, np.float32),
                         np.array(synth.LOAD_AXIS_FF, np.float32), np.concatenate(e), np.concatenate(l))


def test_pattern_library_walk_matches_oracle():
    from paper_2609_05960_gb300 import Engine, gtpower
    rng = np.random.default_rng(91)
    cells = _cells(rng)
    lib_gpu = _library(cells, gtpower.gtp_sipl_expand)
    lib_ref = _library(cells, sipl.dense_cell)
    net = synth.make_netlist(lib_gpu, 400, seed=92)
    counts = synth.zipf_counts(400, 80_000, 1.2, None, 93)
    tr = synth.make_trace(net, counts, 200_000, 93, tie_p=0.05)
    eng = Engine(0)
    try:
        eng.load_library(lib_gpu)
        eng.load_netlist(net)
        eng.load_events(0, tr)
        w = eng.run_power(0, 50).cpu().numpy()
        ref = oracle.walk(lib_ref, net, tr, 50)
        want = oracle.waveform_w(ref["bins"], 50)
        assert (np.abs(w - want) / want).max() <= TOL
        ge = eng.gate_energy(0, device=False)
        np.testing.assert_array_equal(ge["final_state"], ref["final_state"])
        for k in ("e_leak", "e_int", "e_sw"):
            bad = np.abs(ge[k] - ref[k]) > TOL * np.abs(ref[k]) + 1e-9
            assert not bad.any(), k
    finally:
        eng.close()
