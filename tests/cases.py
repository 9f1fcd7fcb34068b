"""Hand-built and small seeded cases shared by the oracle pins and the GPU
parity tests.  Builds the same containers as the ``synth`` generator."""
from __future__ import annotations

import json
import os

import numpy as np

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def records_from(events):
    """events: list of (t, pin, value) -> uint32[n, 2]."""
    rec = np.zeros((len(events), 2), np.uint32)
    for k, (t, pin, v) in enumerate(events):
        rec[k, 0] = np.uint32(np.int32(t).view(np.uint32))
        rec[k, 1] = pin | (v << 4)
    return rec


def trace_from(per_gate_events, init, window_ps):
    counts = np.array([len(e) for e in per_gate_events], np.int64)
    off = synth.offsets_from_counts(counts)
    rec = np.concatenate([records_from(e) for e in per_gate_events]) if off[-1] else np.zeros((0, 2), np.uint32)
    return synth.Trace(int(window_ps), off, np.ascontiguousarray(rec), np.asarray(init, np.uint8), 0, 0)


def single_cell_library(n_in, table_fn, leak_fn, vdd=0.8):
    """One-cell library; table_fn(pin, edge, side) -> 7x7 array, leak_fn(state) -> nW."""
    ns, nl = len(synth.SLEW_AXIS_PS), len(synth.LOAD_AXIS_FF)
    tabs = []
    for pin in range(n_in):
        for edge in range(2):
            for side in range(2 ** (n_in - 1)):
                tabs.append(np.broadcast_to(np.asarray(table_fn(pin, edge, side), np.float32), (ns, nl)))
    leak = np.array([leak_fn(s) for s in range(2 ** (n_in + 1))], np.float32)
    return synth.Library(["CELL"], np.array([n_in], np.int32), float(np.float32(vdd)),
                         np.array(synth.SLEW_AXIS_PS, np.float32), np.array(synth.LOAD_AXIS_FF, np.float32),
                         np.concatenate([t.reshape(-1) for t in tabs]).astype(np.float32), leak)


def netlist_from(lib, cells, loads, slews=None):
    cells = np.asarray(cells, np.int32)
    G = len(cells)
    stride = lib.max_in
    if slews is None:
        slews = np.full((G, stride, 2), 40.0, np.float32)
    slews = np.asarray(slews, np.float32).reshape(G, stride, 2)
    n_pins = (lib.n_in[cells] + 1).astype(np.uint8)
    return synth.Netlist(cells, np.asarray(loads, np.float32), np.ascontiguousarray(slews), n_pins,
                         np.zeros(G, np.int32), -np.ones((G, stride), np.int64))


def and2_worked():
    with open(os.path.join(GOLDEN, "and2_worked.json")) as f:
        fx = json.load(f)
    lib = single_cell_library(2, lambda pin, edge, side: 1.0 + pin + 2.0 * edge + 4.0 * side,
                              lambda s: 10.0 + s, vdd=fx["vdd"])
    net = netlist_from(lib, [0], [fx["load_ff"]])
    tr = trace_from([fx["events"]], [fx["init_state"]], fx["window_ps"])
    return fx, lib, net, tr


def small_random(n_gates=8, n_events=300, window_ps=1500, seed=11, tie_p=0.05, zipf_s=1.1, lib_seed=1):
    """A small seeded case on the synthetic 12-cell library, with ties."""
    lib = synth.make_library(lib_seed)
    net = synth.make_netlist(lib, n_gates, seed + 1)
    counts = synth.zipf_counts(n_gates, n_events, zipf_s, None, seed)
    tr = synth.make_trace(net, counts, window_ps, seed, tie_p)
    return lib, net, tr


def concat_netlists(lib, parts):
    """Union of (net, trace) pairs over one library (same window)."""
    nets, trs = zip(*parts)
    cell = np.concatenate([n.cell for n in nets])
    load = np.concatenate([n.load_ff for n in nets])
    slew = np.concatenate([n.slew_ps for n in nets])
    net = netlist_from(lib, cell, load, slew)
    counts = np.concatenate([np.diff(t.offsets) for t in trs])
    off = synth.offsets_from_counts(counts)
    rec = np.concatenate([t.records for t in trs])
    init = np.concatenate([t.init_state for t in trs])
    return net, synth.Trace(trs[0].window_ps, off, np.ascontiguousarray(rec), init, 0, 0)


def permute_gates(net, tr, perm):
    perm = np.asarray(perm)
    lib_like_stride = net.slew_ps.shape[1]
    counts = np.diff(tr.offsets)[perm]
    off = synth.offsets_from_counts(counts)
    rec = np.concatenate([tr.records[tr.offsets[g]:tr.offsets[g + 1]] for g in perm])
    net2 = synth.Netlist(net.cell[perm], net.load_ff[perm], np.ascontiguousarray(net.slew_ps[perm]),
                         net.n_pins[perm], net.level[perm], net.fanin[perm])
    assert net2.slew_ps.shape[1] == lib_like_stride
    return net2, synth.Trace(tr.window_ps, off, np.ascontiguousarray(rec), tr.init_state[perm], 0, 0)
