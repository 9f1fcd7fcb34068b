"""Per-picosecond brute-force power simulator for hand-sized cases.

TEST INFRASTRUCTURE ONLY.  It pins the interval-based oracle walk
(``gtp_oracle.c``) by a different route: instead of integrating leakage over
inter-event intervals and splitting them at bin boundaries, it steps through
every picosecond of the window, applies the events of that picosecond (all
lookups at the state held before the picosecond's events, then the state
update, as in Algorithm 1's timestamp loop), and charges one picosecond of
leakage at the state holding during that picosecond.  Table interpolation is
delegated to ``scipy.interpolate.RegularGridInterpolator`` (linear, with
linear extrapolation outside the axes), not to the oracle's own routine.
Glitch detection, when asked for, follows the paper's counting formulation
(Sec. 2.4.1, Algorithm 1): per pin, a counter of events in the current clock
cycle, reset when a new cycle starts; an event that brings its pin's counter
above one is a glitch, scaled by Eq. (glitch scaling ratio).

Only for windows of a few thousand ps and a handful of gates.
"""
from __future__ import annotations

import numpy as np
from scipy.interpolate import RegularGridInterpolator


def _tables(lib):
    """Map (cell, pin, edge, side) -> interpolator and (cell, state) -> leakage."""
    ns, nl = len(lib.slew_axis), len(lib.load_axis)
    axes = (np.asarray(lib.slew_axis, np.float64), np.asarray(lib.load_axis, np.float64))
    tabs, leaks = {}, {}
    pos = 0
    lpos = 0
    for c, n_in in enumerate(np.asarray(lib.n_in)):
        n_in = int(n_in)
        for pin in range(n_in):
            for edge in range(2):
                for side in range(2 ** (n_in - 1)):
                    block = np.asarray(lib.e_int[pos * ns * nl:(pos + 1) * ns * nl], np.float64).reshape(ns, nl)
                    tabs[(c, pin, edge, side)] = RegularGridInterpolator(
                        axes, block, method="linear", bounds_error=False, fill_value=None)
                    pos += 1
        for state in range(2 ** (n_in + 1)):
            leaks[(c, state)] = float(lib.p_leak[lpos])
            lpos += 1
    return tabs, leaks


def simulate(lib, net, trace, bin_ps: int, escale=None, lscale=None, load_ff=None, glitch=None):
    """Returns dict(bins[fJ], comp_bins[4][n_bins] (leakage, internal,
    switching, glitch), e_leak, e_int, e_sw, e_gl, n_events, final_state).  glitch = (clock_ps, out_slew[n_gates][2] {fall, rise})."""
    clock, out_slew = glitch if glitch is not None else (0, None)
    T = int(trace.window_ps)
    n_bins = T // bin_ps
    n_gates = len(net.cell)
    n_cells = len(lib.n_in)
    escale = np.ones(n_cells) if escale is None else np.asarray(escale, np.float64)
    lscale = np.ones(n_cells) if lscale is None else np.asarray(lscale, np.float64)
    C_all = np.asarray(net.load_ff if load_ff is None else load_ff, np.float64)
    tabs, leaks = _tables(lib)
    vdd = float(lib.vdd)
    bins = np.zeros(n_bins)
    comp = np.zeros((4, n_bins))
    out = dict(e_leak=np.zeros(n_gates), e_int=np.zeros(n_gates), e_sw=np.zeros(n_gates), e_gl=np.zeros(n_gates),
               n_events=np.zeros(n_gates, np.int64), final_state=np.zeros(n_gates, np.uint8))
    for g in range(n_gates):
        c = int(net.cell[g])
        n_in = int(lib.n_in[c])
        n_pins = n_in + 1
        C = float(C_all[g])
        bits = [(int(trace.init_state[g]) >> p) & 1 for p in range(n_pins)]
        at = {}
        a, b = int(trace.offsets[g]), int(trace.offsets[g + 1])
        for k in range(a, b):
            t = int(np.int32(trace.records[k, 0]))
            meta = int(trace.records[k, 1])
            at.setdefault(t, []).append((meta & 0xF, (meta >> 4) & 1))
        count = [0] * n_pins   # events of each pin in the current clock cycle
        last = [0] * n_pins    # each pin's previous event time
        cycle = -1
        for tau in range(T):
            if clock and tau // clock != cycle:
                cycle = tau // clock
                count = [0] * n_pins
            for pin, value in at.get(tau, []):
                if pin < n_in:
                    others = [bits[p] for p in range(n_in) if p != pin]
                    side = sum(v << k for k, v in enumerate(others))
                    slew = float(net.slew_ps[g, pin, value])
                    E = escale[c] * float(tabs[(c, pin, value, side)]([[slew, C]])[0])
                    rise_fall = float(net.slew_ps[g, pin, 0]) + float(net.slew_ps[g, pin, 1])
                else:
                    E = 0.5 * C * vdd * vdd
                    rise_fall = float(out_slew[g][0]) + float(out_slew[g][1]) if clock else 0.0
                is_glitch = False
                if clock:
                    count[pin] += 1
                    if count[pin] > 1:
                        width = tau - last[pin]
                        E *= 1.0 if rise_fall <= 0 else min(1.0, (2.0 * width / rise_fall) ** 2)
                        is_glitch = True
                    last[pin] = tau
                kind = 3 if is_glitch else (1 if pin < n_in else 2)
                out[("e_leak", "e_int", "e_sw", "e_gl")[kind]][g] += E
                comp[kind, tau // bin_ps] += E
                bins[tau // bin_ps] += E
            for pin, value in at.get(tau, []):
                bits[pin] = value
            state = sum(v << p for p, v in enumerate(bits))
            e = leaks[(c, state)] * lscale[c] * 1e-6
            bins[tau // bin_ps] += e
            comp[0, tau // bin_ps] += e
            out["e_leak"][g] += e
        out["n_events"][g] = b - a
        out["final_state"][g] = sum(v << p for p, v in enumerate(bits))
    out["bins"] = bins
    out["comp_bins"] = comp
    return out


def simulate_patterns(plib, pnet, ptrace, bin_ps: int, clock: int = 0):
    """The same per-picosecond stepping for gates whose cells are given by
    state patterns (up to 32 pins; synth.patterns layout): each lookup scans
    the cell's patterns in list order (oracle/sipl.py) at the state held
    before the picosecond's events; tables are interpolated by
    RegularGridInterpolator.  Output transition times for glitch detection
    are pnet.out_slew_ps.  Returns bins (fJ) and per-gate results."""
    from . import sipl

    T = int(ptrace.window_ps)
    n_bins = T // bin_ps
    G = pnet.n_gates
    axes = (np.asarray(plib.slew_axis, np.float64), np.asarray(plib.load_axis, np.float64))
    vdd = float(plib.vdd)
    bins = np.zeros(n_bins)
    out = dict(e_leak=np.zeros(G), e_int=np.zeros(G), e_sw=np.zeros(G), e_gl=np.zeros(G),
               n_events=np.zeros(G, np.int64), final_state=np.zeros(G, np.uint32))
    for g in range(G):
        n_in, ip, dflt, lp, ld = plib.cell(int(pnet.cell[g]))
        n_pins = n_in + 1
        C = float(pnet.load_ff[g])
        bits = [(int(ptrace.init_state[g]) >> p) & 1 for p in range(n_pins)]
        at = {}
        a, b = int(ptrace.offsets[g]), int(ptrace.offsets[g + 1])
        for k in range(a, b):
            at.setdefault(int(ptrace.t_ps[k]), []).append((int(ptrace.pin[k]), int(ptrace.value[k])))
        count = [0] * n_pins
        last = [0] * n_pins
        cycle = -1
        for tau in range(T):
            if clock and tau // clock != cycle:
                cycle = tau // clock
                count = [0] * n_pins
            state = sum(v << p for p, v in enumerate(bits))
            for pin, value in at.get(tau, []):
                if pin < n_in:
                    tab = sipl.internal_item(pin, value, state & ((1 << n_in) - 1), ip, dflt)
                    f = RegularGridInterpolator(axes, np.asarray(tab, np.float64), method="linear",
                                                bounds_error=False, fill_value=None)
                    E = float(f([[float(pnet.slew_ps[g, pin, value]), C]])[0])
                    rise_fall = float(pnet.slew_ps[g, pin, 0]) + float(pnet.slew_ps[g, pin, 1])
                else:
                    E = 0.5 * C * vdd * vdd
                    rise_fall = float(pnet.out_slew_ps[g, 0]) + float(pnet.out_slew_ps[g, 1])
                kind = 1 if pin < n_in else 2
                if clock:
                    count[pin] += 1
                    if count[pin] > 1:
                        E *= 1.0 if rise_fall <= 0 else min(1.0, (2.0 * (tau - last[pin]) / rise_fall) ** 2)
                        kind = 3
                    last[pin] = tau
                out[("e_leak", "e_int", "e_sw", "e_gl")[kind]][g] += E
                bins[tau // bin_ps] += E
            for pin, value in at.get(tau, []):
                bits[pin] = value
            state = sum(v << p for p, v in enumerate(bits))
            e = sipl.leakage_item(state, lp, ld) * 1e-6
            bins[tau // bin_ps] += e
            out["e_leak"][g] += e
        out["n_events"][g] = b - a
        out["final_state"][g] = sum(v << p for p, v in enumerate(bits))
    out["bins"] = bins
    return out
