"""Seeded synthetic pattern cells, gates and traces: cells given by their
Liberty-style state patterns, up to 32 pins, for the state-pattern walk
(state-indexed arrays up to a pin threshold, pattern traversal above it).

Like the rest of ``synth`` this holds only random draws and the structure of
the inputs, none of the power arithmetic.

A cell has ``n_in`` input pins (0 .. n_in-1) and one output pin (n_in); a
state has bit q = value of pin q.
  * internal patterns ``(pin, edge, care, val, table)``: an event on input
    ``pin`` with new value ``edge`` (-1 = either) whose other input pins
    match ``(state & care) == val`` takes ``table`` (n_slew x n_load, fJ);
    care never holds the event's pin or the output pin.  The first matching
    pattern in list order wins; otherwise the cell's default table of
    (pin, edge).
  * leakage patterns ``(care, val, power)`` over all pins (nW); the first
    match wins, otherwise the cell's default leakage.

The cells stand in for the paper's wide cells and macros (SRAM macros with
dozens of pins; Sec. 4.1): a 20-pin SRAM-like macro with clock, chip and
write enables, 8 address and 8 data inputs and one output; multiplexers
whose data-pin tables depend on the select value (12 and 21 pins); and cells
of 4 to 16 pins with random overlapping patterns.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Tuple

import numpy as np

from . import LOAD_AXIS_FF, SLEW_AXIS_PS, VDD, keys, offsets_from_counts, uniform

STREAM_PAT = 30       # pattern structure
STREAM_PAT_TAB = 31   # tables and powers
STREAM_PNET = 32      # pattern netlist: cells, loads, slews
STREAM_PT_TIME = 33
STREAM_PT_PIN = 34
STREAM_PT_INIT = 35
STREAM_PT_TIE = 36

# (name, input pins, kind): kind "sram" (n_in = 19), "mux" (n_in = 2^k + k),
# "random" (any n_in)
PATTERN_CELLS = [
    ("AOI3P", 3, "random"), ("OAI4P", 4, "random"), ("CPLX5", 5, "random"), ("AOI8P", 8, "random"),
    ("MUX8P", 11, "mux"), ("SLICE15", 15, "random"), ("SRAM20", 19, "sram"), ("MUX16P", 20, "mux"),
]
# default share of gates per cell in make_pattern_netlist
PATTERN_WEIGHTS = [0.25, 0.2, 0.15, 0.1, 0.1, 0.06, 0.08, 0.06]


@dataclasses.dataclass
class PatternLibrary:
    names: List[str]
    n_in: np.ndarray          # int32[n_cells]
    vdd: float
    slew_axis: np.ndarray     # float32[n_slew], ps
    load_axis: np.ndarray     # float32[n_load], fF
    int_offsets: np.ndarray   # int32[n_cells + 1]: cell c's internal patterns
    int_pin: np.ndarray       # int32[n_int]
    int_edge: np.ndarray      # int32[n_int]: 0 fall, 1 rise, -1 either
    int_care: np.ndarray      # uint32[n_int]
    int_val: np.ndarray       # uint32[n_int]
    int_tab: np.ndarray       # float32[n_int, n_slew, n_load] fJ
    int_default: np.ndarray   # float32[sum n_in, 2, n_slew, n_load]: cell-major, per (pin, edge)
    leak_offsets: np.ndarray  # int32[n_cells + 1]
    leak_care: np.ndarray     # uint32[n_leak]
    leak_val: np.ndarray      # uint32[n_leak]
    leak_pw: np.ndarray       # float32[n_leak] nW
    leak_default: np.ndarray  # float32[n_cells] nW

    @property
    def n_cells(self) -> int:
        return len(self.n_in)

    @property
    def max_in(self) -> int:
        return int(self.n_in.max())

    def default_base(self, c: int) -> int:
        return int(self.n_in[:c].sum())

    def cell(self, c: int) -> Tuple[int, list, np.ndarray, list, float]:
        """(n_in, internal patterns, defaults [n_in, 2, ns, nl], leakage
        patterns, default leakage) of cell c, in the form oracle/sipl.py takes."""
        a, b = int(self.int_offsets[c]), int(self.int_offsets[c + 1])
        ip = [(int(self.int_pin[k]), int(self.int_edge[k]), int(self.int_care[k]), int(self.int_val[k]),
               self.int_tab[k]) for k in range(a, b)]
        n = int(self.n_in[c])
        d0 = self.default_base(c)
        dflt = self.int_default[d0:d0 + n]
        la, lb = int(self.leak_offsets[c]), int(self.leak_offsets[c + 1])
        lp = [(int(self.leak_care[k]), int(self.leak_val[k]), float(self.leak_pw[k])) for k in range(la, lb)]
        return n, ip, dflt, lp, float(self.leak_default[c])


class _Draw:
    """Sequential draws from one (seed, stream, b) counter sequence."""

    def __init__(self, seed: int, stream: int, b: int):
        self.seed, self.stream, self.b, self.i = seed, stream, b, 0

    def u(self, n: int = 1) -> np.ndarray:
        k = keys(self.seed, self.stream, n, self.b, self.i)
        self.i += n
        return (k >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def int(self, hi: int) -> int:
        return int(self.u()[0] * hi)

    def mask(self, allowed: int, p: float) -> int:
        bits = [q for q in range(32) if (allowed >> q) & 1]
        u = self.u(len(bits)) if bits else []
        m = 0
        for q, x in zip(bits, u):
            if x < p:
                m |= 1 << q
        return m


def _sram_patterns(d: _Draw, tab):
    """SRAM-like macro: CLK 0, CEN 1 (active low), WEN 2 (active low), A 3..10,
    D 11..18, output Q 19."""
    CLK, CEN, WEN = 0, 1, 2
    A = list(range(3, 11))
    D = list(range(11, 19))
    ce, we = 1 << CEN, 1 << WEN
    ip = [(CLK, 1, ce | we, 0, tab(20, 40)),        # write cycle
          (CLK, 1, ce | we, we, tab(15, 30)),       # read cycle
          (CLK, 1, ce, ce, tab(1, 2)),              # disabled
          (CLK, 0, 0, 0, tab(3, 6)),                # clock fall
          (CEN, -1, 1 << CLK, 0, tab(2, 4)),
          (WEN, -1, ce, 0, tab(2, 4))]
    for a in A:
        ip.append((a, -1, ce, 0, tab(1, 3)))
    for q in D:
        ip.append((q, -1, ce | we, 0, tab(1, 3)))
    Q = 1 << 19
    lp = [(ce | Q, ce | Q, 40.0 + 20.0 * float(d.u()[0])),   # standby, output high
          (ce, ce, 30.0 + 20.0 * float(d.u()[0])),           # standby
          (ce | we, 0, 300.0 + 100.0 * float(d.u()[0])),     # write enabled
          (ce | we, we, 250.0 + 100.0 * float(d.u()[0]))]    # read enabled
    return ip, lp


def _mux_patterns(n_in: int, d: _Draw, tab):
    """2^k data pins, then k select pins, output last: a data pin's tables
    depend on whether the select value picks it."""
    k = 1
    while (1 << k) + k < n_in:
        k += 1
    assert (1 << k) + k == n_in
    sel0 = 1 << k
    smask = ((1 << k) - 1) << sel0
    ip = []
    for i in range(1 << k):
        ip.append((i, -1, smask, i << sel0, tab(2, 4)))     # the selected input
    for j in range(k):
        p = sel0 + j
        care = d.mask(smask & ~(1 << p), 0.5)
        ip.append((p, 1, care, d.mask(care, 0.5), tab(2, 5)))
    lp = []
    out = 1 << n_in
    for v in range(min(1 << k, 8)):
        lp.append((smask | out, (v << sel0) | (out if v & 1 else 0), 10.0 + 40.0 * float(d.u()[0])))
    lp.append((out, out, 20.0 + 10.0 * float(d.u()[0])))
    return ip, lp


def _random_patterns(n_in: int, d: _Draw, tab):
    inputs = (1 << n_in) - 1
    ip = []
    for _ in range(2 * n_in):
        pin = d.int(n_in)
        edge = d.int(3) - 1
        care = d.mask(inputs & ~(1 << pin), 0.3)
        ip.append((pin, edge, care, d.mask(care, 0.5), tab(0.5, 5)))
    lp = []
    for _ in range(n_in + 2):
        care = d.mask((2 << n_in) - 1, 0.3)
        lp.append((care, d.mask(care, 0.5), 1.0 + 49.0 * float(d.u()[0])))
    return ip, lp


def make_pattern_library(seed: int = 1, cells=PATTERN_CELLS) -> PatternLibrary:
    ns, nl = len(SLEW_AXIS_PS), len(LOAD_AXIS_FF)
    n_in = np.array([k for _, k, _ in cells], np.int32)
    ipo, lpo = [0], [0]
    ipin, iedge, icare, ival, itab, dflt = [], [], [], [], [], []
    lcare, lval, lpw, ldef = [], [], [], []
    for c, (name, n, kind) in enumerate(cells):
        d = _Draw(seed, STREAM_PAT, c)
        dt = _Draw(seed, STREAM_PAT_TAB, c)

        def tab(lo, hi):
            return (lo + (hi - lo) * dt.u(ns * nl)).reshape(ns, nl).astype(np.float32)

        if kind == "sram":
            assert n == 19
            ip, lp = _sram_patterns(d, tab)
        elif kind == "mux":
            ip, lp = _mux_patterns(n, d, tab)
        else:
            ip, lp = _random_patterns(n, d, tab)
        for pin, edge, care, val, t in ip:
            ipin.append(pin)
            iedge.append(edge)
            icare.append(care)
            ival.append(val)
            itab.append(t)
        ipo.append(len(ipin))
        for _ in range(n):
            dflt.append(np.stack([tab(0.5, 3), tab(0.5, 3)]))
        for care, val, pw in lp:
            lcare.append(care)
            lval.append(val)
            lpw.append(pw)
        lpo.append(len(lcare))
        ldef.append(1.0 + 9.0 * float(d.u()[0]))
    return PatternLibrary([n for n, _, _ in cells], n_in, float(np.float32(VDD)),
                          np.array(SLEW_AXIS_PS, np.float32), np.array(LOAD_AXIS_FF, np.float32),
                          np.array(ipo, np.int32), np.array(ipin, np.int32), np.array(iedge, np.int32),
                          np.array(icare, np.uint32), np.array(ival, np.uint32),
                          np.array(itab, np.float32).reshape(-1, ns, nl),
                          np.array(dflt, np.float32).reshape(-1, 2, ns, nl),
                          np.array(lpo, np.int32), np.array(lcare, np.uint32), np.array(lval, np.uint32),
                          np.array(lpw, np.float32), np.array(ldef, np.float32))


def pattern_library_from(cells, vdd: float = VDD) -> PatternLibrary:
    """A pattern library from explicit cells: a list of (n_in, internal
    patterns, defaults [n_in, 2, ns, nl], leakage patterns, default leakage),
    the form PatternLibrary.cell returns."""
    ns, nl = len(SLEW_AXIS_PS), len(LOAD_AXIS_FF)
    ipo, lpo = [0], [0]
    ip_all, lp_all, dflt, ldef = [], [], [], []
    for n, ip, d, lp, ld in cells:
        ip_all += list(ip)
        ipo.append(len(ip_all))
        dflt.append(np.broadcast_to(np.asarray(d, np.float32), (n, 2, ns, nl)))
        lp_all += list(lp)
        lpo.append(len(lp_all))
        ldef.append(ld)
    tabs = np.array([np.broadcast_to(np.asarray(t, np.float32), (ns, nl)) for *_, t in ip_all],
                    np.float32).reshape(-1, ns, nl)
    return PatternLibrary([f"P{i}" for i in range(len(cells))], np.array([c[0] for c in cells], np.int32),
                          float(np.float32(vdd)), np.array(SLEW_AXIS_PS, np.float32),
                          np.array(LOAD_AXIS_FF, np.float32), np.array(ipo, np.int32),
                          np.array([p[0] for p in ip_all], np.int32), np.array([p[1] for p in ip_all], np.int32),
                          np.array([p[2] for p in ip_all], np.uint32), np.array([p[3] for p in ip_all], np.uint32),
                          tabs, np.concatenate(dflt).astype(np.float32), np.array(lpo, np.int32),
                          np.array([p[0] for p in lp_all], np.uint32), np.array([p[1] for p in lp_all], np.uint32),
                          np.array([p[2] for p in lp_all], np.float32), np.array(ldef, np.float32))


# --------------------------------------------------------------------------- netlist
@dataclasses.dataclass
class PatternNetlist:
    cell: np.ndarray          # int32[n]
    load_ff: np.ndarray       # float32[n]
    slew_ps: np.ndarray       # float32[n, stride, 2] input transition times (edge 0 fall, 1 rise)
    out_slew_ps: np.ndarray   # float32[n, 2] output {fall, rise} transition times
    n_pins: np.ndarray        # int32[n] = n_in(cell) + 1

    @property
    def n_gates(self) -> int:
        return len(self.cell)

    @property
    def slew_stride(self) -> int:
        return self.slew_ps.shape[1]


def make_pattern_netlist(plib: PatternLibrary, n_gates: int, seed: int = 2, weights=None,
                         load_range=(0.5, 12.0), slew_range=(10.0, 200.0)) -> PatternNetlist:
    """Cells drawn with the given weights (default PATTERN_WEIGHTS), loads
    U[0.5, 12] fF, transition times U[10, 200] ps."""
    G = int(n_gates)
    w = np.asarray(PATTERN_WEIGHTS if weights is None else weights, np.float64)
    cdf = np.cumsum(w / w.sum())
    u = uniform(seed, STREAM_PNET, G, b=0)
    cell = np.minimum(np.searchsorted(cdf, u, side="right"), plib.n_cells - 1).astype(np.int32)
    load = (load_range[0] + (load_range[1] - load_range[0]) * uniform(seed, STREAM_PNET, G, b=1)).astype(np.float32)
    stride = plib.max_in
    us = uniform(seed, STREAM_PNET, G * stride * 2, b=2).reshape(G, stride, 2)
    slew = (slew_range[0] + (slew_range[1] - slew_range[0]) * us).astype(np.float32)
    n_in = plib.n_in[cell]
    for p in range(stride):
        slew[n_in <= p, p, :] = 0.0
    uo = uniform(seed, STREAM_PNET, G * 2, b=3).reshape(G, 2)
    oslew = (slew_range[0] + (slew_range[1] - slew_range[0]) * uo).astype(np.float32)
    return PatternNetlist(cell, load, slew, oslew, (n_in + 1).astype(np.int32))


# --------------------------------------------------------------------------- traces
@dataclasses.dataclass
class PatternTrace:
    window_ps: int
    offsets: np.ndarray       # int64[n + 1]
    t_ps: np.ndarray          # int32[E], non-decreasing within a gate
    pin: np.ndarray           # uint8[E]
    value: np.ndarray         # uint8[E] new value (always a toggle)
    init_state: np.ndarray    # uint32[n]

    @property
    def n_events(self) -> int:
        return int(self.offsets[-1])


def make_pattern_trace(pnet: PatternNetlist, counts, window_ps: int, seed: int, tie_p: float = 0.0,
                       clock_pin_share: float = 0.0) -> PatternTrace:
    """Per gate: sorted uniform times in [0, window_ps), a record repeating
    the previous record's time with probability tie_p, pins uniform over the
    gate's pins (pin 0 takes clock_pin_share of the events on top, like a
    clock), and values that toggle each pin from a random initial state."""
    counts = np.asarray(counts, np.int64)
    G = pnet.n_gates
    off = offsets_from_counts(counts)
    E = int(off[-1])
    t_all = np.empty(E, np.int32)
    pin_all = np.empty(E, np.uint8)
    val_all = np.empty(E, np.uint8)
    nk = keys(seed, STREAM_PT_INIT, G)
    init = np.empty(G, np.uint32)
    for g in range(G):
        n_p = int(pnet.n_pins[g])
        full = (1 << n_p) - 1
        init[g] = np.uint32(int(nk[g]) & full)
        a, b = int(off[g]), int(off[g + 1])
        n = b - a
        if n == 0:
            continue
        t = np.sort((keys(seed, STREAM_PT_TIME, n, g) % np.uint64(window_ps)).astype(np.int64))
        if tie_p > 0:
            tie = uniform(seed, STREAM_PT_TIE, n, g) < tie_p
            tie[0] = False
            idx = np.where(tie, 0, np.arange(n))
            t = t[np.maximum.accumulate(idx)]
        u = uniform(seed, STREAM_PT_PIN, n, g)
        if clock_pin_share > 0:
            pin = np.where(u < clock_pin_share, 0,
                           np.minimum(((u - clock_pin_share) / (1 - clock_pin_share) * n_p).astype(np.int64), n_p - 1))
        else:
            pin = np.minimum((u * n_p).astype(np.int64), n_p - 1)
        order = np.argsort(pin, kind="stable")
        sp = pin[order]
        first = np.searchsorted(sp, sp, side="left")
        occ = np.empty(n, np.int64)
        occ[order] = np.arange(n) - first
        bit = (int(init[g]) >> pin) & 1
        val = (bit ^ ((occ + 1) & 1)).astype(np.uint8)
        t_all[a:b] = t
        pin_all[a:b] = pin
        val_all[a:b] = val
    return PatternTrace(int(window_ps), off, t_all, pin_all, val_all, init)
