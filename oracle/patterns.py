"""The FP64 walk of gates whose cells are given by state patterns.

TEST INFRASTRUCTURE ONLY (used by ``tests/``, ``bench.py``'s oracle checks and
the smoke check).  The GPU engine never imports it.

This is the walk of the C oracle (gtp_oracle.c) restated in plain Python for
gates of up to 32 pins, with every power item found by scanning the cell's
state patterns in list order (``oracle/sipl.py``): the fallback path of
Sec. 4.1, which the paper takes for gates with more pins than its
state-indexed threshold.  Per gate, in record order:
  * records sharing a timestamp form a group; every lookup of a group uses
    the state held before the group, and the state changes after the whole
    group [Algorithm 1, the timestamp loop];
  * leakage: the power of the state held since the previous group, over the
    time since then [Eq. 4], split over the bins the interval overlaps in
    proportion to the overlap [Sec. 2.4.2];
  * an input-pin event: the internal-power table of (pin, new value, other
    input pins of the pre-group state), interpolated bilinearly at the pin's
    transition time for that edge and the gate's load [Sec. 2.2];
  * an output-pin event: 0.5 * C * Vdd^2 [Eq. 1];
  * with a clock period: an event on a pin that already had an event earlier
    in the same clock cycle is a glitch event, its energy scaled by
    min(1, (2 * pulse width / (rise + fall transition time))^2) and counted as
    glitch energy [Sec. 2.4.1, Eq. 2];
  * dynamic energy goes to the bin holding the event's time.
Units: ps, fF, V, fJ, nW; E[fJ] = P[nW] * dt[ps] * 1e-6.

Malformed traces raise oracle.OracleError with the C oracle's codes and the
first bad record: -3 for a time outside [0, window) or a pin >= the gate's
pin count (times are checked per group, at the group's first record), -2 for
a time below the previous group's, -4 for a value equal to the pin's current
value.

``adjoint`` is the chain rule through the same walk: dL/dC per pattern gate
for a loss of the power waveform.

Parity status: the walk is pinned against the C oracle walk on cells of up
to 7 inputs (sipl.dense_cell turns the patterns into the C oracle's
state-indexed library), and on a 20-pin cell by closed forms; the adjoint
against the C oracle's adjoint on the same small cells and by central
differences of the walk on the wide cells (tests/test_oracle_patterns.py).
"""
from __future__ import annotations

import numpy as np

from . import OracleError, bilinear, bilinear_dload
from . import sipl


def _split(bins, P, a, b, bin_ps):
    """Leakage power P over [a, b) ps into the bins it overlaps (fJ)."""
    if b <= a:
        return
    k0, k1 = a // bin_ps, (b - 1) // bin_ps
    for k in range(k0, k1 + 1):
        lo, hi = max(a, k * bin_ps), min(b, (k + 1) * bin_ps)
        bins[k] += P * (hi - lo) * 1e-6


def _split_range(bins, diff, P, a, b, bin_ps):
    """_split with the bins the interval covers whole added through a
    difference array (same sums, FP64 additions reordered); `diff` has
    len(bins) + 1 entries and is turned into per-bin amounts at the end."""
    if b <= a:
        return
    k0, k1 = a // bin_ps, (b - 1) // bin_ps
    if k0 == k1:
        bins[k0] += P * (b - a) * 1e-6
        return
    bins[k0] += P * ((k0 + 1) * bin_ps - a) * 1e-6
    bins[k1] += P * (b - k1 * bin_ps) * 1e-6
    if k1 > k0 + 1:
        diff[k0 + 1] += P * bin_ps * 1e-6
        diff[k1] -= P * bin_ps * 1e-6


def walk(plib, pnet, ptrace, bin_ps: int, glitch_clock_ps: int = 0, gates=None, range_split: bool = True,
         components: bool = False) -> dict:
    """Bins (fJ) and per-gate results (e_leak, e_int, e_sw, e_gl in fJ,
    n_events, final_state as uint32) of the selected gates (default all).
    The output transition times for glitch detection are pnet.out_slew_ps.
    With ``components``, ``comp_bins`` [4][n_bins] splits the bins into
    leakage, internal, switching and glitch energy (Sec. 2.2's components)."""
    T = int(ptrace.window_ps)
    if bin_ps <= 0 or T % bin_ps:
        raise ValueError("window_ps must be a multiple of bin_ps")
    n_bins = T // bin_ps
    bins = np.zeros(n_bins, np.float64)
    diff = np.zeros(n_bins + 1, np.float64) if range_split else None
    comp = np.zeros((4, n_bins), np.float64) if components else None
    cdiff = np.zeros(n_bins + 1, np.float64) if components and range_split else None
    sel = np.arange(pnet.n_gates) if gates is None else np.asarray(gates, np.int64)
    out = {k: np.zeros(len(sel), np.float64) for k in ("e_leak", "e_int", "e_sw", "e_gl")}
    out["n_events"] = np.zeros(len(sel), np.int64)
    out["final_state"] = np.zeros(len(sel), np.uint32)
    half_v2 = 0.5 * float(plib.vdd) * float(plib.vdd)
    cells = {}
    clk = int(glitch_clock_ps)
    def split(P, a, b):
        if range_split:
            _split_range(bins, diff, P, a, b, bin_ps)
            if comp is not None:
                _split_range(comp[0], cdiff, P, a, b, bin_ps)
        else:
            _split(bins, P, a, b, bin_ps)
            if comp is not None:
                _split(comp[0], P, a, b, bin_ps)
    for i, g in enumerate(sel):
        g = int(g)
        c = int(pnet.cell[g])
        if c not in cells:
            cells[c] = plib.cell(c)
        n_in, ip, dflt, lp, ld = cells[c]
        n_pins = n_in + 1
        in_mask = (1 << n_in) - 1
        C = float(pnet.load_ff[g])
        S = int(ptrace.init_state[g])
        a, b = int(ptrace.offsets[g]), int(ptrace.offsets[g + 1])
        t_prev = 0
        El = Ei = Es = Eg = 0.0
        last = [-1] * n_pins
        r = a
        while r < b:
            t = int(ptrace.t_ps[r])
            j = r
            while j < b and int(ptrace.t_ps[j]) == t:
                j += 1
            if t < 0 or t >= T:
                raise OracleError(-3, r)
            if t < t_prev:
                raise OracleError(-2, r)
            P = sipl.leakage_item(S, lp, ld)
            El += P * (t - t_prev) * 1e-6
            split(P, t_prev, t)
            S_next = S
            for e in range(r, j):
                pin, v = int(ptrace.pin[e]), int(ptrace.value[e])
                if pin >= n_pins:
                    raise OracleError(-3, e)
                if (S_next >> pin) & 1 == v:
                    raise OracleError(-4, e)
                S_next ^= 1 << pin
                if pin < n_in:
                    tab = sipl.internal_item(pin, v, S & in_mask, ip, dflt)
                    sl = pnet.slew_ps[g, pin]
                    E = bilinear(plib.slew_axis, plib.load_axis, tab, float(sl[v]), C)
                    sum_slew = float(sl[0]) + float(sl[1])
                else:
                    E = half_v2 * C
                    sum_slew = float(pnet.out_slew_ps[g, 0]) + float(pnet.out_slew_ps[g, 1])
                if clk > 0 and last[pin] >= 0 and last[pin] // clk == t // clk:
                    if sum_slew > 0:
                        x = 2.0 * (t - last[pin]) / sum_slew
                        E *= min(1.0, x * x)
                    Eg += E
                    kind = 3
                elif pin < n_in:
                    Ei += E
                    kind = 1
                else:
                    Es += E
                    kind = 2
                if comp is not None:
                    comp[kind, t // bin_ps] += E
                last[pin] = t
                bins[t // bin_ps] += E
            S = S_next
            t_prev = t
            r = j
        P = sipl.leakage_item(S, lp, ld)
        El += P * (T - t_prev) * 1e-6
        split(P, t_prev, T)
        out["e_leak"][i], out["e_int"][i], out["e_sw"][i], out["e_gl"][i] = El, Ei, Es, Eg
        out["n_events"][i] = b - a
        out["final_state"][i] = S
    if range_split:
        bins += np.cumsum(diff[:-1])
        if comp is not None:
            comp[0] += np.cumsum(cdiff[:-1])
    out["bins"] = bins
    if comp is not None:
        out["comp_bins"] = comp
    return out


def adjoint(plib, pnet, ptrace, bin_ps: int, dLdP, glitch_clock_ps: int = 0, gates=None) -> np.ndarray:
    """dL/dC (fF^-1 units of L) of the selected pattern gates (default all),
    for a loss L of the power waveform P_b = E_b * 1e-3 / bin_ps (W) given
    dL/dP_b per bin.  Walks the gates as walk() does (same groups, states,
    checks and glitch detection); only the dynamic energies depend on a
    gate's load C:
      * an input-pin event: the slope in load of its bilinear interpolation
        on the located load segment [Sec. 2.2];
      * an output-pin event: 0.5 * Vdd^2 [Eq. 1];
      * a glitch event's derivative carries its ratio, which depends on
        times and transition times only [Sec. 2.4.1, Eq. 2];
    each times dL/dP of the event's bin and dP_b/dE_b = 1e-3 / bin_ps."""
    T = int(ptrace.window_ps)
    if bin_ps <= 0 or T % bin_ps:
        raise ValueError("window_ps must be a multiple of bin_ps")
    g_bin = np.asarray(dLdP, np.float64) * (1e-3 / bin_ps)
    sel = np.arange(pnet.n_gates) if gates is None else np.asarray(gates, np.int64)
    dC = np.zeros(len(sel), np.float64)
    half_v2 = 0.5 * float(plib.vdd) * float(plib.vdd)
    clk = int(glitch_clock_ps)
    cells = {}
    for i, g in enumerate(sel):
        g = int(g)
        c = int(pnet.cell[g])
        if c not in cells:
            cells[c] = plib.cell(c)
        n_in, ip, dflt, _, _ = cells[c]
        n_pins = n_in + 1
        in_mask = (1 << n_in) - 1
        C = float(pnet.load_ff[g])
        S = int(ptrace.init_state[g])
        a, b = int(ptrace.offsets[g]), int(ptrace.offsets[g + 1])
        t_prev = 0
        last = [-1] * n_pins
        acc = 0.0
        r = a
        while r < b:
            t = int(ptrace.t_ps[r])
            j = r
            while j < b and int(ptrace.t_ps[j]) == t:
                j += 1
            if t < 0 or t >= T:
                raise OracleError(-3, r)
            if t < t_prev:
                raise OracleError(-2, r)
            S_next = S
            for e in range(r, j):
                pin, v = int(ptrace.pin[e]), int(ptrace.value[e])
                if pin >= n_pins:
                    raise OracleError(-3, e)
                if (S_next >> pin) & 1 == v:
                    raise OracleError(-4, e)
                S_next ^= 1 << pin
                if pin < n_in:
                    tab = sipl.internal_item(pin, v, S & in_mask, ip, dflt)
                    sl = pnet.slew_ps[g, pin]
                    dE = bilinear_dload(plib.slew_axis, plib.load_axis, tab, float(sl[v]), C)
                    sum_slew = float(sl[0]) + float(sl[1])
                else:
                    dE = half_v2
                    sum_slew = float(pnet.out_slew_ps[g, 0]) + float(pnet.out_slew_ps[g, 1])
                if clk > 0 and last[pin] >= 0 and last[pin] // clk == t // clk and sum_slew > 0:
                    x = 2.0 * (t - last[pin]) / sum_slew
                    dE *= min(1.0, x * x)
                last[pin] = t
                acc += g_bin[t // bin_ps] * dE
            S = S_next
            t_prev = t
            r = j
        dC[i] = acc
    return dC
