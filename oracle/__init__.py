"""FP64 CPU oracle for gate-level time-based power analysis.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The GPU engine never imports,
links or calls it, and it shares no code with the engine.

``gtp_oracle.c`` holds the walk and the adjoint (plain loops, FP64); this
module marshals numpy arrays into it.  ``brute`` holds an independent
per-picosecond simulator for hand-sized cases.  Inputs are duck-typed: any
objects with the fields of ``synth.Library``, ``synth.Netlist`` and
``synth.Trace`` work.

Paper anchors: events and gate state (Sec. 2.1); power models (Sec. 2.2);
switching energy (Eq. 1, Sec. 2.4.1) and leakage energy (Eq. 4, Sec. 2.4.2); per-bin
leakage split (Sec. 2.4.2); timestamp-group semantics (Algorithm 1);
state-indexed lookup (Sec. 4.1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

OK, EINVAL, EORDER, ERANGE, ENOTOGGLE = 0, -1, -2, -3, -4


def build(force: bool = False) -> None:
    src = os.path.join(_HERE, "gtp_oracle.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-std=c11", "-ffp-contract=off",
                               "-o", _LIB_PATH + ".tmp", src])
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)


class _Lib(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int32), ("n_in", ctypes.c_void_p), ("vdd", ctypes.c_double),
                ("n_slew", ctypes.c_int32), ("slew_axis", ctypes.c_void_p),
                ("n_load", ctypes.c_int32), ("load_axis", ctypes.c_void_p),
                ("e_int", ctypes.c_void_p), ("p_leak", ctypes.c_void_p),
                ("escale", ctypes.c_void_p), ("lscale", ctypes.c_void_p)]


class _Net(ctypes.Structure):
    _fields_ = [("n_gates", ctypes.c_int64), ("cell", ctypes.c_void_p), ("load_ff", ctypes.c_void_p),
                ("slew_ps", ctypes.c_void_p), ("slew_stride", ctypes.c_int32)]


class _Glitch(ctypes.Structure):
    _fields_ = [("clock_ps", ctypes.c_int64), ("out_slew_ps", ctypes.c_void_p)]


class _Trace(ctypes.Structure):
    _fields_ = [("window_ps", ctypes.c_int64), ("offsets", ctypes.c_void_p), ("records", ctypes.c_void_p),
                ("init_state", ctypes.c_void_p)]


_clib = None


def _lib():
    global _clib
    if _clib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        lib.oracle_walk.restype = ctypes.c_int
        lib.oracle_walk.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int64, P, P, ctypes.c_int64, P,
                                    P, P, P, P, P, P, P, P, P]
        lib.oracle_walk_range.restype = ctypes.c_int
        lib.oracle_walk_range.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int64, P, P, P, P, P, P, P, P, P, P,
                                          P]
        lib.oracle_adjoint.restype = ctypes.c_int
        lib.oracle_adjoint.argtypes = [P, P, P, ctypes.c_int64, P, ctypes.c_int64, P, P, P, P, P]
        lib.oracle_bilinear.restype = ctypes.c_double
        lib.oracle_bilinear.argtypes = [ctypes.c_int32, P, ctypes.c_int32, P, P, ctypes.c_double,
                                        ctypes.c_double]
        lib.oracle_bilinear_dload.restype = ctypes.c_double
        lib.oracle_bilinear_dload.argtypes = lib.oracle_bilinear.argtypes
        _clib = lib
    return _clib


def _c(a, dtype):
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


class OracleError(RuntimeError):
    def __init__(self, code, record):
        super().__init__(f"oracle rejected the trace: code {code} at record {record}")
        self.code = code
        self.record = record


def _structs(lib, net, trace, escale, lscale, load_ff):
    keep = []

    def p(a):
        keep.append(a)
        return a.ctypes.data

    n_cells = len(lib.n_in)
    es = _c(np.ones(n_cells) if escale is None else escale, np.float64)
    ls = _c(np.ones(n_cells) if lscale is None else lscale, np.float64)
    L = _Lib(n_cells, p(_c(lib.n_in, np.int32)), float(lib.vdd), len(lib.slew_axis),
             p(_c(lib.slew_axis, np.float32)), len(lib.load_axis), p(_c(lib.load_axis, np.float32)),
             p(_c(lib.e_int, np.float32)), p(_c(lib.p_leak, np.float32)), p(es), p(ls))
    C = net.load_ff if load_ff is None else load_ff
    slew = _c(net.slew_ps, np.float32)
    N = _Net(len(net.cell), p(_c(net.cell, np.int32)), p(_c(C, np.float64)), p(slew), slew.shape[1])
    T = _Trace(int(trace.window_ps), p(_c(trace.offsets, np.int64)), p(_c(trace.records, np.uint32)),
               p(_c(trace.init_state, np.uint8)))
    return L, N, T, keep


def _glitch(glitch, keep):
    """(clock_ps, out_slew[n_gates][2] {fall, rise} ps) -> _Glitch, or None."""
    if glitch is None:
        return None
    clock_ps, out_slew = glitch
    a = _c(out_slew, np.float32)
    keep.append(a)
    return _Glitch(int(clock_ps), a.ctypes.data)


def walk(lib, net, trace, bin_ps: int, escale=None, lscale=None, load_ff=None, gates=None,
         sample_bins=None, waveform: bool = True, glitch=None, components: bool = False,
         leak_range: bool = False):
    """Run the FP64 walk.  Returns a dict with ``bins`` (fJ per bin; the
    sampled bins only if ``sample_bins`` is given), ``e_leak``, ``e_int``,
    ``e_sw``, ``e_gl`` (fJ per gate), ``n_events`` and ``final_state``.  With
    ``gates`` the per-gate outputs follow that order (and ``bins`` only
    receive those gates' contributions).  ``glitch`` = (clock_ps, out_slew
    [n_gates][2] {fall, rise} ps) turns on glitch detection; e_gl is 0
    without it.  ``components`` adds ``comp_bins`` [4][len(bins)]: the bins
    split into leakage, internal, switching and glitch energy (fJ).
    ``leak_range`` (all bins only) uses the range-mode leakage split of the
    C walk: the same bins up to FP64 addition order, in time proportional to
    events + bins rather than gates x bins (pinned against the plain split in
    tests/test_oracle_range.py)."""
    L, N, T, keep = _structs(lib, net, trace, escale, lscale, load_ff)
    GL = _glitch(glitch, keep)
    n_bins = int(trace.window_ps) // int(bin_ps) if bin_ps > 0 else 0
    if gates is not None:
        gates = _c(gates, np.int64)
        n_sel = len(gates)
    else:
        n_sel = len(net.cell)
    if sample_bins is not None:
        sample_bins = _c(sample_bins, np.int64)
        if len(sample_bins) and (np.any(np.diff(sample_bins) <= 0) or sample_bins[0] < 0
                                 or sample_bins[-1] >= n_bins):
            raise ValueError("sample_bins must be sorted, unique and in range")
        bins = np.zeros(len(sample_bins), np.float64)
    else:
        bins = np.zeros(max(n_bins, 0), np.float64)
    comp = np.zeros((4, len(bins)), np.float64) if components else None
    out = {k: np.zeros(n_sel, np.float64) for k in ("e_leak", "e_int", "e_sw", "e_gl")}
    out["n_events"] = np.zeros(n_sel, np.int64)
    out["final_state"] = np.zeros(n_sel, np.uint8)
    bad = ctypes.c_int64(-1)
    nullp = None
    if leak_range and sample_bins is None:
        rc = _lib().oracle_walk_range(
            ctypes.byref(L), ctypes.byref(N), ctypes.byref(T), int(bin_ps), n_sel,
            gates.ctypes.data if gates is not None else nullp,
            bins.ctypes.data if waveform else nullp,
            out["e_leak"].ctypes.data, out["e_int"].ctypes.data, out["e_sw"].ctypes.data,
            out["n_events"].ctypes.data, out["final_state"].ctypes.data, ctypes.byref(bad),
            ctypes.byref(GL) if GL is not None else nullp, out["e_gl"].ctypes.data,
            comp.ctypes.data if comp is not None else nullp)
        del keep
        if rc == EINVAL:
            raise ValueError("invalid bin size / window")
        if rc != OK:
            raise OracleError(rc, bad.value)
        out["bins"] = bins
        if comp is not None:
            out["comp_bins"] = comp
        return out
    rc = _lib().oracle_walk(
        ctypes.byref(L), ctypes.byref(N), ctypes.byref(T), int(bin_ps), n_sel,
        gates.ctypes.data if gates is not None else nullp,
        bins.ctypes.data if waveform else nullp,
        len(sample_bins) if sample_bins is not None else 0,
        sample_bins.ctypes.data if sample_bins is not None else nullp,
        out["e_leak"].ctypes.data, out["e_int"].ctypes.data, out["e_sw"].ctypes.data,
        out["n_events"].ctypes.data, out["final_state"].ctypes.data, ctypes.byref(bad),
        ctypes.byref(GL) if GL is not None else nullp, out["e_gl"].ctypes.data,
        comp.ctypes.data if comp is not None else nullp)
    del keep
    if rc == EINVAL:
        raise ValueError("invalid bin size / window")
    if rc != OK:
        raise OracleError(rc, bad.value)
    out["bins"] = bins
    if comp is not None:
        out["comp_bins"] = comp
    return out


def adjoint(lib, net, trace, bin_ps: int, dLdP, escale=None, lscale=None, load_ff=None, gates=None, glitch=None):
    """FP64 gradient of L(P) given dL/dP per bin (P in W); returns
    (dC, d_escale[n_cells], d_lscale[n_cells]).  With ``gates`` only those
    gates are walked (dC follows their order; the cell gradients then hold
    only their contributions).  ``glitch`` as for walk()."""
    L, N, T, keep = _structs(lib, net, trace, escale, lscale, load_ff)
    GL = _glitch(glitch, keep)
    g = _c(dLdP, np.float64)
    if gates is not None:
        gates = _c(gates, np.int64)
    n_sel = len(gates) if gates is not None else len(net.cell)
    dC = np.zeros(n_sel, np.float64)
    de = np.zeros(len(lib.n_in), np.float64)
    dl = np.zeros(len(lib.n_in), np.float64)
    rc = _lib().oracle_adjoint(ctypes.byref(L), ctypes.byref(N), ctypes.byref(T), int(bin_ps), g.ctypes.data,
                               n_sel, gates.ctypes.data if gates is not None else None,
                               dC.ctypes.data, de.ctypes.data, dl.ctypes.data,
                               ctypes.byref(GL) if GL is not None else None)
    del keep
    if rc != OK:
        raise ValueError(f"oracle_adjoint failed: {rc}")
    return dC, de, dl


def bilinear(slew_axis, load_axis, table, slew: float, load: float) -> float:
    sa, la = _c(slew_axis, np.float32), _c(load_axis, np.float32)
    tb = _c(table, np.float32)
    return _lib().oracle_bilinear(len(sa), sa.ctypes.data, len(la), la.ctypes.data, tb.ctypes.data,
                                  float(slew), float(load))


def bilinear_dload(slew_axis, load_axis, table, slew: float, load: float) -> float:
    sa, la = _c(slew_axis, np.float32), _c(load_axis, np.float32)
    tb = _c(table, np.float32)
    return _lib().oracle_bilinear_dload(len(sa), sa.ctypes.data, len(la), la.ctypes.data, tb.ctypes.data,
                                        float(slew), float(load))


def design_power(result: dict, window_ps: int, bin_ps: int) -> dict:
    """Design-level power from a walk() result (W) [Eq. 3,
    Sec. 2.4.1: a component's energy over the analysis time, here the
    window; peak power, Sec. 5: the largest bin of the waveform]."""
    to_w = 1e-3 / float(window_ps)
    p = {k: float(np.sum(result[e])) * to_w for k, e in (("p_leak", "e_leak"), ("p_int", "e_int"),
                                                          ("p_sw", "e_sw"), ("p_gl", "e_gl"))}
    p["p_total"] = p["p_leak"] + p["p_int"] + p["p_sw"] + p["p_gl"]
    w = waveform_w(result["bins"], bin_ps)
    p["peak_bin"] = int(np.argmax(w)) if len(w) else -1
    p["p_peak"] = float(w[p["peak_bin"]]) if len(w) else 0.0
    return p


def waveform_w(bins_fj: np.ndarray, bin_ps: int) -> np.ndarray:
    """Power per bin in W from energy per bin in fJ: fJ/ps = mW."""
    return np.asarray(bins_fj, np.float64) * 1e-3 / float(bin_ps)
