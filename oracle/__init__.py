"""CPU oracle of the multi-morphology HH + Hines stepper (FP64).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by
the CPU-baseline leg of ``bench.py``; never by the library.  It shares no code
with the CUDA path.  ``mm_oracle.c`` holds the arithmetic (see its header for
the step order and the readings of the paper); this module builds it with gcc
and wraps it with ctypes.  ``mlp.py`` holds the FP64 oracle of the cost-model
network.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_LIB_TWIN = os.path.join(_BUILD, "liboracle_twin.so")
_lock = threading.Lock()
_lib = None
_lib_twin = None


def build(force: bool = False, twin: bool = False) -> str:
    """Compile mm_oracle.c (gcc, -O2, no FMA contraction, OpenMP).  twin:
    the same oracle with its membrane sums in the opposite order
    (ORC_SUM_REVERSED), an equally valid FP64 evaluation that rounds
    differently."""
    os.makedirs(_BUILD, exist_ok=True)
    out = _LIB_TWIN if twin else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fno-fast-math",
               "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"] + (["-DORC_SUM_REVERSED"] if twin else [])
        subprocess.check_call(cmd)
        os.replace(tmp, out)
    return out


class Params(C.Structure):
    _fields_ = [(k, C.c_double) for k in
                ("gNa", "gK", "gL", "ENa", "EK", "EL", "Cm", "Ra", "v_init", "threshold", "tau_syn", "e_syn")]


def params_from(d: dict) -> Params:
    return Params(*[float(d[k]) for k in
                    ("gNa", "gK", "gL", "ENa", "EK", "EL", "Cm", "Ra", "v_init", "threshold", "tau_syn", "e_syn")])


_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)


def lib(twin: bool = False):
    global _lib, _lib_twin
    with _lock:
        if (_lib_twin if twin else _lib) is None:
            L = C.CDLL(build(twin=twin))
            L.orc_area_cm2.restype = C.c_double
            L.orc_area_cm2.argtypes = [C.c_double, C.c_double]
            L.orc_rhalf_Mohm.restype = C.c_double
            L.orc_rhalf_Mohm.argtypes = [C.c_double, C.c_double, C.c_double]
            L.orc_exprelr.restype = C.c_double
            L.orc_exprelr.argtypes = [C.c_double]
            L.orc_rates.restype = None
            L.orc_rates.argtypes = [C.c_double, _D]
            L.orc_gates_inf.restype = None
            L.orc_gates_inf.argtypes = [C.c_double, _D, _D, _D]
            L.orc_gate_step.restype = None
            L.orc_gate_step.argtypes = [C.c_double, C.c_double, _D, _D, _D]
            L.orc_hines_solve.restype = None
            L.orc_hines_solve.argtypes = [_D, _D, _D, _D, _I32, C.c_int32, _I64]
            L.orc_geometry.restype = None
            L.orc_geometry.argtypes = [C.c_int32, _I64, _I32, _D, _D, C.POINTER(Params), _D, _D, _D]
            L.orc_assemble.restype = None
            L.orc_assemble.argtypes = [C.c_int32, _I32, _D, _D, _D, _D, _D, _D, _D, _D, C.c_double,
                                       C.POINTER(Params), C.c_double, C.c_int, _D, _D, _D, _D]
            L.orc_simulate.restype = C.c_int
            L.orc_simulate.argtypes = [C.c_int32, _I64, _I32, _D, _D, _D,
                                       C.c_int64, _I32, _I32, _I32, _D, _D, _I32,
                                       C.POINTER(Params), C.c_double, C.c_int, C.c_int64, _D,
                                       _D, _D, _D, _D, _D, _D, _I32, _I32, _D, C.c_int64, _I64, C.c_int]
            L.orc_part_create.restype = C.c_void_p
            L.orc_part_create.argtypes = [C.c_int32, _I64, _I32, _D, _D, _D, C.c_int64, _I32, _I32, _I32, _D, _D,
                                          C.c_int32, C.POINTER(Params), C.c_double, C.c_int]
            L.orc_part_destroy.restype = None
            L.orc_part_destroy.argtypes = [C.c_void_p]
            L.orc_part_step.restype = C.c_int
            L.orc_part_step.argtypes = [C.c_void_p, C.c_int64]
            L.orc_part_fired.restype = C.c_int64
            L.orc_part_fired.argtypes = [C.c_void_p, C.c_int64, C.c_int32, _I32, _I64, C.c_int64]
            L.orc_part_inject.restype = C.c_int
            L.orc_part_inject.argtypes = [C.c_void_p, C.c_int64, _I32, _I64]
            L.orc_part_read.restype = C.c_int64
            L.orc_part_read.argtypes = [C.c_void_p, _D, _D, _D, _D, _D]
            if twin:
                _lib_twin = L
            else:
                _lib = L
    return _lib_twin if twin else _lib


def _p(a, ct):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


# ------------------------------------------------------------------ pieces

def exprelr(x: float) -> float:
    return lib().orc_exprelr(float(x))


def rates(V: float) -> np.ndarray:
    """[alpha_m, beta_m, alpha_h, beta_h, alpha_n, beta_n] at V (1/ms)."""
    r = np.zeros(6)
    lib().orc_rates(float(V), _p(r, C.c_double))
    return r


def gates_inf(V: float):
    m, h, n = C.c_double(), C.c_double(), C.c_double()
    lib().orc_gates_inf(float(V), C.byref(m), C.byref(h), C.byref(n))
    return m.value, h.value, n.value


def gate_step(V: float, dt: float, m: float, h: float, n: float):
    cm, ch, cn = C.c_double(m), C.c_double(h), C.c_double(n)
    lib().orc_gate_step(float(V), float(dt), C.byref(cm), C.byref(ch), C.byref(cn))
    return cm.value, ch.value, cn.value


def hines_solve(a, b, c, rhs, parent, count_ops: bool = False):
    """Algorithm 1 on one tree; returns the solution (and the op count)."""
    a, b, c, rhs = _f64(a).copy(), _f64(b).copy(), _f64(c).copy(), _f64(rhs).copy()
    parent = _i32(parent)
    ops = np.zeros(1, np.int64)
    lib().orc_hines_solve(_p(a, C.c_double), _p(b, C.c_double), _p(c, C.c_double),
                          _p(rhs, C.c_double), _p(parent, C.c_int32), len(rhs), _p(ops, C.c_int64))
    return (rhs, int(ops[0])) if count_ops else rhs


def geometry(comp_offset, parent, length_um, diam_um, params: dict):
    """(area_cm2, C_nF, gax_uS) per compartment."""
    off = _i64(comp_offset)
    parent = _i32(parent)
    L, d = _f64(length_um), _f64(diam_um)
    n = int(off[-1])
    area, Cn, gax = np.zeros(n), np.zeros(n), np.zeros(n)
    pr = params_from(params)
    lib().orc_geometry(len(off) - 1, _p(off, C.c_int64), _p(parent, C.c_int32), _p(L, C.c_double),
                       _p(d, C.c_double), C.byref(pr), _p(area, C.c_double), _p(Cn, C.c_double),
                       _p(gax, C.c_double))
    return area, Cn, gax


SCHEMES = {"be": 0, "cn": 1}


def assemble(parent, V, m, h, n, gsyn, area, Cn, gax, stim_nA, params: dict, dt: float, scheme: str = "be"):
    """Hines system (a, b, c, rhs) of one neuron for dV.

    scheme "be": backward Euler with the membrane conductance implicit (the
    default reading of Eq. 2); "cn": Eq. 2 as printed, half of each axial
    coupling implicit and the current explicit (Crank-Nicolson diffusion)."""
    k = len(V)
    parent = _i32(parent)
    arrs = [_f64(x) for x in (V, m, h, n, gsyn, area, Cn, gax)]
    a, b, c, rhs = np.zeros(k), np.zeros(k), np.zeros(k), np.zeros(k)
    pr = params_from(params)
    lib().orc_assemble(k, _p(parent, C.c_int32), *[_p(x, C.c_double) for x in arrs], float(stim_nA),
                       C.byref(pr), float(dt), SCHEMES[scheme], _p(a, C.c_double), _p(b, C.c_double), _p(c, C.c_double),
                       _p(rhs, C.c_double))
    return a, b, c, rhs


# --------------------------------------------------------------- simulation

class Result:
    def __init__(self, V, m, h, n, g, soma_trace, spk_neuron, spk_t, n_spikes, spk_comp=None):
        self.V, self.m, self.h, self.n, self.g = V, m, h, n, g
        self.soma_trace = soma_trace
        self.spk_neuron = spk_neuron
        self.spk_t = spk_t
        self.n_spikes = n_spikes
        self.spk_comp = np.zeros_like(spk_neuron) if spk_comp is None else spk_comp

    def spikes_sorted(self):
        """(neuron, t) ordered by (t, neuron)."""
        o = np.lexsort((self.spk_neuron, self.spk_t))
        return self.spk_neuron[o], self.spk_t[o]

    def point_spikes_sorted(self):
        """(neuron, local compartment, t) ordered by (t, neuron, compartment)."""
        o = np.lexsort((self.spk_comp, self.spk_neuron, self.spk_t))
        return self.spk_neuron[o], self.spk_comp[o], self.spk_t[o]


def simulate(net, n_steps: int, dt: float = None, params: dict = None, V_init=None,
             record_soma: bool = False, spike_cap: int = None, threads: int = 0, scheme: str = "be",
             detect: str = "soma") -> Result:
    """Run the oracle on a ``netgen.Network`` for n_steps steps (scheme as
    in ``assemble``).  detect "soma": the threshold test runs at every soma;
    "points": at every distinct (source neuron, ``syn_src_comp``) point that
    synapses leave from (all somata when the network has no source
    compartments), Sec. 2's spike computation over the synapse points."""
    if detect not in ("soma", "points"):
        raise ValueError(f"unknown detection mode {detect!r}")
    dt = net.dt if dt is None else dt
    params = net.params if params is None else params
    pr = params_from(params)
    off = _i64(net.comp_offset)
    parent = _i32(net.parent)
    L, d, stim = _f64(net.length_um), _f64(net.diam_um), _f64(net.stim_nA)
    src, dst, comp = _i32(net.syn_src), _i32(net.syn_dst), _i32(net.syn_comp)
    w, dl = _f64(net.syn_w), _f64(net.syn_delay_ms)
    scomp = None
    if detect == "points":
        sc = getattr(net, "syn_src_comp", None)
        scomp = _i32(np.zeros(len(src), np.int32) if sc is None else sc)
    N = len(off) - 1
    Cc = int(off[-1])
    V, m, h, n, g = np.zeros(Cc), np.zeros(Cc), np.zeros(Cc), np.zeros(Cc), np.zeros(Cc)
    trace = np.zeros((N, n_steps + 1)) if record_soma else None
    n_pt = N if scomp is None else len(np.unique(src.astype(np.int64) * (1 << 32) + scomp))
    cap = spike_cap if spike_cap is not None else max(1024, n_pt * (n_steps // 40 + 2))
    spn = np.zeros(cap, np.int32)
    spc = np.zeros(cap, np.int32)
    spt = np.zeros(cap, np.float64)
    nsp = np.zeros(1, np.int64)
    vi = None if V_init is None else _f64(V_init)
    rc = lib().orc_simulate(N, _p(off, C.c_int64), _p(parent, C.c_int32), _p(L, C.c_double),
                            _p(d, C.c_double), _p(stim, C.c_double), len(src), _p(src, C.c_int32),
                            _p(dst, C.c_int32), _p(comp, C.c_int32), _p(w, C.c_double), _p(dl, C.c_double),
                            _p(scomp, C.c_int32),
                            C.byref(pr), float(dt), SCHEMES[scheme], int(n_steps), _p(vi, C.c_double),
                            _p(V, C.c_double), _p(m, C.c_double), _p(h, C.c_double), _p(n, C.c_double),
                            _p(g, C.c_double), _p(trace, C.c_double), _p(spn, C.c_int32), _p(spc, C.c_int32),
                            _p(spt, C.c_double), cap,
                            _p(nsp, C.c_int64), int(threads))
    if rc == -1:
        raise ValueError("oracle: invalid network")
    if rc == -2:
        raise MemoryError("oracle: allocation failed")
    if rc == -3:
        raise OverflowError("oracle: spike capacity exceeded")
    k = int(nsp[0])
    return Result(V, m, h, n, g, trace, spn[:k].copy(), spt[:k].copy(), k, spc[:k].copy())


class Part:
    """A steppable FP64 network part (orc_part_*): ``net`` a netgen.Network
    whose synapse sources n_neurons .. n_neurons + n_ext - 1 are external
    (neurons simulated elsewhere).  The same methods as the library's network
    for a sharded run: step, read_fired, inject_spikes, read_voltages."""

    def __init__(self, net, n_ext: int = 0, scheme: str = "be", twin: bool = False):
        self._keep = dict(off=_i64(net.comp_offset), parent=_i32(net.parent), L=_f64(net.length_um),
                          d=_f64(net.diam_um), stim=_f64(net.stim_nA), src=_i32(net.syn_src), dst=_i32(net.syn_dst),
                          comp=_i32(net.syn_comp), w=_f64(net.syn_w), dl=_f64(net.syn_delay_ms))
        k = self._keep
        self._pr = params_from(net.params)
        self.n_neurons, self.n_comp = net.n_neurons, net.n_comp
        self._L = lib(twin)
        self._h = self._L.orc_part_create(net.n_neurons, _p(k["off"], C.c_int64), _p(k["parent"], C.c_int32),
                                        _p(k["L"], C.c_double), _p(k["d"], C.c_double), _p(k["stim"], C.c_double),
                                        len(k["src"]), _p(k["src"], C.c_int32), _p(k["dst"], C.c_int32),
                                        _p(k["comp"], C.c_int32), _p(k["w"], C.c_double), _p(k["dl"], C.c_double),
                                        int(n_ext), C.byref(self._pr), float(net.dt), SCHEMES[scheme])
        if not self._h:
            raise ValueError("oracle: invalid network part")

    def step(self, n: int):
        if self._L.orc_part_step(self._h, int(n)) != 0:
            raise MemoryError("oracle: allocation failed")

    def read_fired(self, step0: int, n_steps: int):
        cap = max(1, self.n_neurons * max(1, n_steps))
        nrn, st = np.empty(cap, np.int32), np.empty(cap, np.int64)
        k = self._L.orc_part_fired(self._h, int(step0), int(n_steps), _p(nrn, C.c_int32), _p(st, C.c_int64), cap)
        return nrn[:k].copy(), st[:k].copy()

    def inject_spikes(self, ext_src, step):
        src, st = _i32(ext_src), _i64(step)
        if self._L.orc_part_inject(self._h, len(src), _p(src, C.c_int32), _p(st, C.c_int64)) != 0:
            raise ValueError("oracle: a spike handed in too late or out of range")

    def read_voltages(self):
        V = np.empty(self.n_comp)
        self._L.orc_part_read(self._h, _p(V, C.c_double), None, None, None, None)
        return V

    def close(self):
        if self._h:
            self._L.orc_part_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
