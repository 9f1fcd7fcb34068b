"""Liberty-style state patterns resolved by traversal.

TEST INFRASTRUCTURE ONLY (imported by ``tests/``).  This is the plain
definition that state-indexed lookup replaces (Sec. 3.1, and the
fallback path of Sec. 4.1): to find the power item of a state, scan the
cell's state patterns in list order and take the first whose fixed pins
match the state; a state no pattern matches takes the default item.  A
pattern is (care, val): the pins in the bit mask ``care`` (bit q = pin q)
must hold the values in ``val``; the other pins are don't-care.

``dense_cell`` evaluates that traversal at every state to build the arrays a
state-indexed library holds (the layout of ``synth.Library``), so that the
oracle walk can run on a library given as patterns.  It shares nothing with
the engine's expansion, which enumerates each pattern's don't-care pins.
"""
from __future__ import annotations

import numpy as np


def input_state(side: int, pin: int) -> int:
    """Input-pin state with pin `pin` at 0 and the other input pins taken, in
    pin order, from the bits of `side`."""
    low = side & ((1 << pin) - 1)
    high = (side >> pin) << (pin + 1)
    return low | high


def internal_item(pin: int, edge: int, state: int, int_patterns, int_default):
    """Table of an event on `pin` with edge `edge` at input state `state`:
    int_patterns is a list of (pin, edge or -1, care, val, table)."""
    for p, e, care, val, table in int_patterns:
        if p == pin and (e < 0 or e == edge) and (state & care) == val:
            return np.asarray(table, np.float32)
    return np.asarray(int_default[pin][edge], np.float32)


def leakage_item(state: int, leak_patterns, leak_default: float) -> float:
    """Leakage (nW) at full pin state `state`: leak_patterns is a list of
    (care, val, power)."""
    for care, val, power in leak_patterns:
        if (state & care) == val:
            return float(np.float32(power))
    return float(np.float32(leak_default))


def dense_cell(n_in: int, n_slew: int, n_load: int, int_patterns, int_default, leak_patterns, leak_default):
    """(e_int, p_leak) of one cell in the state-indexed layout: e_int holds
    n_in pins x 2 edges x 2^(n_in-1) side states x (n_slew x n_load), p_leak
    2^(n_in+1) full states."""
    tabs = []
    for pin in range(n_in):
        for edge in range(2):
            for side in range(2 ** (n_in - 1)):
                t = internal_item(pin, edge, input_state(side, pin), int_patterns, int_default)
                tabs.append(np.broadcast_to(t, (n_slew, n_load)).reshape(-1))
    leak = [leakage_item(s, leak_patterns, leak_default) for s in range(2 ** (n_in + 1))]
    return np.concatenate(tabs).astype(np.float32), np.array(leak, np.float32)
