"""ctypes binding of the C-ABI in include/mm.h (argument marshalling only).

Every step of the simulation runs in the CUDA library; this module converts
NumPy inputs to the C structs, hands PyTorch's caching allocator to the
library for device memory, and turns status codes into exceptions.  There is
no fallback: if the library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

MM_OK, MM_EINVAL, MM_ENOMEM, MM_ECUDA, MM_ETIMEOUT, MM_ENUMERIC, MM_EOVERFLOW, MM_ESTATE, MM_ENOTSUP = range(9)
MM_FP64, MM_FP32C = 0, 1
MM_SCHED_SIZE_SORTED, MM_SCHED_COST = 0, 1
STATE = {"V": 0, "m": 1, "h": 2, "n": 3, "gsyn": 4}
SCHEMES = {"be": 0, "cn": 1}
DETECT = {"soma": 0, "points": 1}  # MM_SCHEME_BE, MM_SCHEME_CN
PRECISION = {"fp64": MM_FP64, "fp32c": MM_FP32C}


class MMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_status_name(status)}: {message}")
        self.status = status


class Morphologies(C.Structure):
    _fields_ = [("n_neurons", C.c_int32), ("comp_offset", C.POINTER(C.c_int64)), ("parent", C.POINTER(C.c_int32)),
                ("length_um", C.POINTER(C.c_double)), ("diam_um", C.POINTER(C.c_double))]


class ChannelParams(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("gNa", "gK", "gL", "ENa", "EK", "EL", "Cm", "Ra", "v_init", "threshold_mV")]


class Synapses(C.Structure):
    _fields_ = [("n", C.c_int64), ("src_neuron", C.POINTER(C.c_int32)), ("dst_neuron", C.POINTER(C.c_int32)),
                ("dst_comp", C.POINTER(C.c_int32)), ("weight_uS", C.POINTER(C.c_double)),
                ("delay_ms", C.POINTER(C.c_double)), ("tau_ms", C.c_double), ("e_rev_mV", C.c_double),
                ("src_comp", C.POINTER(C.c_int32))]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
RELEASE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("release", RELEASE_FN), ("ctx", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("schedule", C.c_int32), ("graph_steps", C.c_int32),
                ("block_threads", C.c_int32), ("group_comps", C.c_int32), ("device", C.c_int32),
                ("time_items", C.c_int32), ("scheme", C.c_int32), ("detect", C.c_int32),
                ("deterministic_delivery", C.c_int32),
                ("dt_ms", C.c_double), ("spike_capacity", C.c_int64), ("cuda_stream", C.c_void_p),
                ("cost", C.POINTER(C.c_float)), ("allocator", Allocator), ("n_ext_sources", C.c_int32)]


class KernelTimes(C.Structure):
    _fields_ = [("step_kernel_ms", C.c_double), ("step_kernel_launches", C.c_int64),
                ("deliver_kernel_ms", C.c_double), ("deliver_kernel_launches", C.c_int64),
                ("giant_kernel_ms", C.c_double), ("giant_kernel_launches", C.c_int64),
                ("big_kernel_ms", C.c_double), ("big_kernel_launches", C.c_int64)]


class LaunchInfo(C.Structure):
    _fields_ = [(k, C.c_int32) for k in ("work_items", "blocks", "threads", "blocks_per_sm", "smem_bytes",
                                          "max_item_comps", "max_item_segments", "max_item_waves", "giant_items",
                                          "big_items", "big_blocks", "big_threads", "big_smem_bytes",
                                          "max_big_item_comps")] + [("comps", C.c_int64 * 3),
                                                                    ("sites", C.c_int64 * 3)]


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load the CUDA library (raises if it is not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise ImportError(f"CUDA library {path} is not built; run __graft_entry__.build()")
            _build.build()
        L = C.CDLL(path)
        P = C.POINTER
        net_p = C.c_void_p
        L.mm_default_options.argtypes = [P(Options)]
        L.mm_default_options.restype = None
        L.mm_create_network.argtypes = [P(Morphologies), P(ChannelParams), P(Synapses), P(C.c_double), P(Options),
                                        P(net_p)]
        L.mm_step.argtypes = [net_p, C.c_int64, C.c_double]
        L.mm_synchronize.argtypes = [net_p]
        L.mm_read_voltages.argtypes = [net_p, P(C.c_double), C.c_int64]
        L.mm_read_state.argtypes = [net_p, C.c_int32, P(C.c_double), C.c_int64]
        L.mm_read_soma_voltages.argtypes = [net_p, P(C.c_double), C.c_int64]
        L.mm_read_spikes.argtypes = [net_p, P(C.c_int32), P(C.c_double), C.c_int64, P(C.c_int64)]
        L.mm_read_spike_points.argtypes = [net_p, P(C.c_int32), P(C.c_int32), P(C.c_double), C.c_int64,
                                           P(C.c_int64)]
        L.mm_read_outputs.argtypes = [net_p, P(C.c_double), C.c_int64, P(C.c_int32), P(C.c_int32), P(C.c_double),
                                      C.c_int64, P(C.c_int64)]
        L.mm_read_outputs.restype = C.c_int
        L.mm_train_schedule.argtypes = [P(Morphologies), P(ChannelParams), P(C.c_double), P(Options), C.c_int32,
                                        C.c_int32, C.c_int32, C.c_float, C.c_uint64, P(C.c_float), C.c_int64,
                                        C.c_void_p]
        L.mm_train_schedule.restype = C.c_int
        L.mm_set_stimulus.argtypes = [net_p, P(C.c_double), C.c_int64]
        L.mm_get_step.argtypes = [net_p, P(C.c_int64)]
        L.mm_save_state.argtypes = [net_p, C.c_void_p, C.c_size_t, P(C.c_size_t)]
        L.mm_load_state.argtypes = [net_p, C.c_void_p, C.c_size_t]
        L.mm_set_kernel_timing.argtypes = [net_p, C.c_int32]
        L.mm_read_kernel_timing.argtypes = [net_p, P(KernelTimes), C.c_int32]
        L.mm_get_launch_info.argtypes = [net_p, P(LaunchInfo)]
        L.mm_autotune.argtypes = [P(Morphologies), P(ChannelParams), P(Synapses), P(C.c_double), P(Options),
                                  C.c_int64, C.c_int32, C.c_int32, P(TunePoint), C.c_int32, P(C.c_int32), P(Options)]
        L.mm_autotune.restype = C.c_int
        L.mm_read_neuron_times.argtypes = [net_p, P(C.c_double), C.c_int64]
        L.mm_read_neuron_times.restype = C.c_int
        L.mm_neuron_features.argtypes = [P(Morphologies), P(C.c_float), C.c_int64]
        L.mm_neuron_features.restype = C.c_int
        L.mm_mlp_create.argtypes = [C.c_uint64, P(C.c_void_p)]
        L.mm_mlp_set_params.argtypes = [C.c_void_p, P(C.c_float), C.c_int64]
        L.mm_mlp_get_params.argtypes = [C.c_void_p, P(C.c_float), C.c_int64]
        L.mm_mlp_set_normalisation.argtypes = [C.c_void_p, P(C.c_float), P(C.c_float), C.c_float, C.c_float]
        L.mm_mlp_loss_grad.argtypes = [C.c_void_p, P(C.c_float), P(C.c_float), C.c_int64, P(C.c_float),
                                       P(C.c_float), C.c_int64]
        L.mm_mlp_train.argtypes = [C.c_void_p, P(C.c_float), P(C.c_float), C.c_int64, C.c_int32, C.c_float,
                                   P(C.c_float)]
        L.mm_mlp_predict.argtypes = [C.c_void_p, P(C.c_float), C.c_int64, P(C.c_float)]
        L.mm_mlp_destroy.argtypes = [C.c_void_p]
        L.mm_mlp_destroy.restype = None
        for name in ("mm_mlp_create", "mm_mlp_set_params", "mm_mlp_get_params", "mm_mlp_set_normalisation",
                     "mm_mlp_loss_grad", "mm_mlp_train", "mm_mlp_predict"):
            getattr(L, name).restype = C.c_int
        L.mm_selftest_bounded_wait.argtypes = [C.c_int32, C.c_uint32]
        L.mm_selftest_bounded_wait.restype = C.c_int
        L.mm_inject_spikes.argtypes = [net_p, C.c_int64, P(C.c_int32), P(C.c_int64)]
        L.mm_inject_spikes.restype = C.c_int
        L.mm_read_fired.argtypes = [net_p, C.c_int64, C.c_int32, P(C.c_int32), P(C.c_int64), C.c_int64, P(C.c_int64)]
        L.mm_read_fired.restype = C.c_int
        L.mm_hines_solve.argtypes = [C.c_int32, C.c_int64] + [C.c_void_p] * 8
        L.mm_hines_solve.restype = C.c_int
        L.mm_hines_solve_noalloc.argtypes = [C.c_int32, C.c_int64] + [C.c_void_p] * 8
        L.mm_hines_solve_noalloc.restype = C.c_int
        L.mm_last_error.argtypes = [net_p]
        L.mm_last_error.restype = C.c_char_p
        L.mm_status_string.argtypes = [C.c_int]
        L.mm_status_string.restype = C.c_char_p
        L.mm_destroy.argtypes = [net_p]
        L.mm_destroy.restype = None
        for name in ("mm_create_network", "mm_step", "mm_synchronize", "mm_read_voltages", "mm_read_state",
                     "mm_read_soma_voltages", "mm_read_spikes", "mm_read_spike_points", "mm_set_stimulus", "mm_get_step",
                     "mm_save_state", "mm_load_state", "mm_set_kernel_timing", "mm_read_kernel_timing",
                     "mm_get_launch_info"):
            getattr(L, name).restype = C.c_int
        _lib = L
        return L


def _status_name(s: int) -> str:
    names = ["MM_OK", "MM_EINVAL", "MM_ENOMEM", "MM_ECUDA", "MM_ETIMEOUT", "MM_ENUMERIC", "MM_EOVERFLOW",
             "MM_ESTATE", "MM_ENOTSUP"]
    return names[s] if 0 <= s < len(names) else f"status {s}"


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


N_FEATURES = 16


def neuron_features(net) -> np.ndarray:
    """[n_neurons, 16] morphology features (host computation in the library)."""
    L = load()
    off = np.ascontiguousarray(net.comp_offset, np.int64)
    par = np.ascontiguousarray(net.parent, np.int32)
    Lu = np.ascontiguousarray(net.length_um, np.float64)
    Du = np.ascontiguousarray(net.diam_um, np.float64)
    morph = Morphologies(net.n_neurons, _ptr(off, C.c_int64), _ptr(par, C.c_int32), _ptr(Lu, C.c_double),
                         _ptr(Du, C.c_double))
    out = np.empty((net.n_neurons, N_FEATURES), np.float32)
    st = L.mm_neuron_features(C.byref(morph), _ptr(out, C.c_float), out.size)
    if st != MM_OK:
        raise MMError(st, "mm_neuron_features")
    return out


MLP_PARAMS = 5313


class MLP:
    """The learned cost model (16 -> 64 -> 64 -> 1, BF16 weights, FP32
    accumulation), trained and run by the library's kernels."""

    def __init__(self, seed: int = 0):
        self._L = load()
        self._h = C.c_void_p()
        st = self._L.mm_mlp_create(int(seed), C.byref(self._h))
        if st != MM_OK:
            raise MMError(st, "mm_mlp_create")

    def _ok(self, st, what):
        if st != MM_OK:
            raise MMError(st, what)

    def set_params(self, theta):
        t = np.ascontiguousarray(theta, np.float32)
        self._ok(self._L.mm_mlp_set_params(self._h, _ptr(t, C.c_float), t.size), "mm_mlp_set_params")

    def get_params(self) -> np.ndarray:
        t = np.empty(MLP_PARAMS, np.float32)
        self._ok(self._L.mm_mlp_get_params(self._h, _ptr(t, C.c_float), t.size), "mm_mlp_get_params")
        return t

    def set_normalisation(self, mu, sd, y_mu: float, y_sd: float):
        mu = np.ascontiguousarray(mu, np.float32)
        sd = np.ascontiguousarray(sd, np.float32)
        self._ok(self._L.mm_mlp_set_normalisation(self._h, _ptr(mu, C.c_float), _ptr(sd, C.c_float), y_mu, y_sd),
                 "mm_mlp_set_normalisation")

    def loss_grad(self, X, y):
        X = np.ascontiguousarray(X, np.float32)
        y = np.ascontiguousarray(y, np.float32)
        loss = C.c_float()
        g = np.empty(MLP_PARAMS, np.float32)
        self._ok(self._L.mm_mlp_loss_grad(self._h, _ptr(X, C.c_float), _ptr(y, C.c_float), y.size, C.byref(loss),
                                          _ptr(g, C.c_float), g.size), "mm_mlp_loss_grad")
        return loss.value, g

    def train(self, X, y, epochs: int, lr: float = 3e-3) -> np.ndarray:
        X = np.ascontiguousarray(X, np.float32)
        y = np.ascontiguousarray(y, np.float32)
        losses = np.empty(max(1, epochs), np.float32)
        self._ok(self._L.mm_mlp_train(self._h, _ptr(X, C.c_float), _ptr(y, C.c_float), y.size, int(epochs),
                                      float(lr), _ptr(losses, C.c_float)), "mm_mlp_train")
        return losses[:epochs]

    def predict(self, X) -> np.ndarray:
        X = np.ascontiguousarray(X, np.float32)
        out = np.empty(X.shape[0], np.float32)
        self._ok(self._L.mm_mlp_predict(self._h, _ptr(X, C.c_float), X.shape[0], _ptr(out, C.c_float)),
                 "mm_mlp_predict")
        return out

    def close(self):
        if self._h:
            self._L.mm_mlp_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def selftest_bounded_wait(device: int = 0, max_polls: int = 1000) -> int:
    """mm_selftest_bounded_wait: the status (MM_ETIMEOUT when the bounded
    wait on a barrier nothing arrives at gave up and reported it)."""
    return int(load().mm_selftest_bounded_wait(int(device), int(max_polls)))


def hines_solve(tree_offset, parent, a, b, c, rhs, stream=None):
    """Algorithm 1 on a batch of trees held in CUDA tensors (int64 offsets,
    int32 local parents, float64 a, b, c, rhs); returns x (a CUDA tensor)."""
    import torch
    L = load()
    x = torch.empty_like(rhs)
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    st = L.mm_hines_solve(int(tree_offset.numel() - 1), int(rhs.numel()), tree_offset.data_ptr(),
                          parent.data_ptr(), a.data_ptr(), b.data_ptr(), c.data_ptr(), rhs.data_ptr(),
                          x.data_ptr(), s)
    if st != MM_OK:
        raise MMError(st, "mm_hines_solve")
    return x


class TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator."""

    def __init__(self, device: int):
        import torch
        self._torch = torch
        self.device = torch.device("cuda", device)
        self.blocks = {}
        self._alloc = ALLOC_FN(self._do_alloc)
        self._release = RELEASE_FN(self._do_release)

    def _do_alloc(self, nbytes, ctx):
        try:
            t = self._torch.empty(int(nbytes), dtype=self._torch.uint8, device=self.device)
        except Exception:
            return None
        p = t.data_ptr()
        self.blocks[p] = t
        return p

    def _do_release(self, ptr, ctx):
        self.blocks.pop(ptr, None)

    def struct(self) -> Allocator:
        return Allocator(self._alloc, self._release, None)

    def bytes_held(self) -> int:
        return sum(t.numel() for t in self.blocks.values())


def _marshal(net):
    """C structs of a netgen.Network (and the arrays they point into, which
    must stay alive while the structs are used)."""
    a = dict(
        off=np.ascontiguousarray(net.comp_offset, np.int64), parent=np.ascontiguousarray(net.parent, np.int32),
        L=np.ascontiguousarray(net.length_um, np.float64), D=np.ascontiguousarray(net.diam_um, np.float64),
        src=np.ascontiguousarray(net.syn_src, np.int32), dst=np.ascontiguousarray(net.syn_dst, np.int32),
        comp=np.ascontiguousarray(net.syn_comp, np.int32), w=np.ascontiguousarray(net.syn_w, np.float64),
        dl=np.ascontiguousarray(net.syn_delay_ms, np.float64),
        stim=np.ascontiguousarray(net.stim_nA, np.float64))
    sc = getattr(net, "syn_src_comp", None)
    a["scomp"] = None if sc is None else np.ascontiguousarray(sc, np.int32)
    morph = Morphologies(net.n_neurons, _ptr(a["off"], C.c_int64), _ptr(a["parent"], C.c_int32),
                         _ptr(a["L"], C.c_double), _ptr(a["D"], C.c_double))
    p = net.params
    chan = ChannelParams(p["gNa"], p["gK"], p["gL"], p["ENa"], p["EK"], p["EL"], p["Cm"], p["Ra"], p["v_init"],
                         p["threshold"])
    syn = Synapses(len(a["src"]), _ptr(a["src"], C.c_int32), _ptr(a["dst"], C.c_int32), _ptr(a["comp"], C.c_int32),
                   _ptr(a["w"], C.c_double), _ptr(a["dl"], C.c_double), p["tau_syn"], p["e_syn"],
                   _ptr(a["scomp"], C.c_int32) if a["scomp"] is not None else None)
    return a, morph, chan, syn


class ScheduleReport(C.Structure):
    _fields_ = [("n_timed", C.c_int32), ("n_holdout", C.c_int32), ("r2_holdout", C.c_double),
                ("final_loss", C.c_double), ("mean_time_us", C.c_double), ("r2_holdout_size_only", C.c_double)]


def train_schedule(net, n_timed: int = 5000, steps: int = 40, epochs: int = 600, lr: float = 3e-3, seed: int = 0,
                   device: int = 0, stream=None) -> dict:
    """mm_train_schedule on a netgen.Network: the learned per-neuron cost
    (for Network(cost=...)) and the report."""
    L = load()
    a, morph, chan, _syn = _marshal(net)
    opt = Options()
    L.mm_default_options(C.byref(opt))
    opt.device = device
    opt.dt_ms = float(net.dt)
    if stream is not None:
        opt.cuda_stream = C.c_void_p(int(stream))
    alloc = TorchAllocator(device)
    opt.allocator = alloc.struct()
    cost = np.empty(net.n_neurons, np.float32)
    rep = ScheduleReport()
    st = L.mm_train_schedule(C.byref(morph), C.byref(chan), _ptr(a["stim"], C.c_double), C.byref(opt),
                             int(n_timed), int(steps), int(epochs), float(lr), C.c_uint64(seed),
                             _ptr(cost, C.c_float), cost.size, C.byref(rep))
    if st != MM_OK:
        raise MMError(st, "mm_train_schedule failed")
    return {"cost": cost, "n_timed": rep.n_timed, "n_holdout": rep.n_holdout, "r2_holdout": rep.r2_holdout,
            "r2_holdout_size_only": rep.r2_holdout_size_only, "final_loss": rep.final_loss,
            "mean_time_us": rep.mean_time_us}


class TunePoint(C.Structure):
    _fields_ = [("block_threads", C.c_int32), ("group_comps", C.c_int32), ("status", C.c_int32),
                ("ms_per_step", C.c_double)]


def autotune(net, precision: str = "fp32c", sample_comps: int = 2_000_000, warmup: int = 3, steps: int = 20,
             device: int = 0, stream=None, cost: Optional[np.ndarray] = None, graph_steps: int = 40,
             detect: str = "soma") -> dict:
    """mm_autotune on a netgen.Network: the fastest (block_threads,
    group_comps) measured on a stratified sample, and every candidate."""
    L = load()
    a, morph, chan, syn = _marshal(net)
    opt = Options()
    L.mm_default_options(C.byref(opt))
    opt.precision = PRECISION[precision]
    opt.graph_steps = graph_steps
    opt.device = device
    opt.dt_ms = float(net.dt)
    opt.detect = DETECT[detect]
    keep = None
    if cost is not None:
        keep = np.ascontiguousarray(cost, np.float32)
        opt.schedule = MM_SCHED_COST
        opt.cost = _ptr(keep, C.c_float)
    if stream is not None:
        opt.cuda_stream = C.c_void_p(int(stream))
    alloc = TorchAllocator(device)
    opt.allocator = alloc.struct()
    pts = (TunePoint * 16)()
    npts = C.c_int32(0)
    best = Options()
    st = L.mm_autotune(C.byref(morph), C.byref(chan), C.byref(syn), _ptr(a["stim"], C.c_double), C.byref(opt),
                       int(sample_comps), int(warmup), int(steps), pts, 16, C.byref(npts), C.byref(best))
    if st != MM_OK:
        raise MMError(st, "mm_autotune failed")
    del keep
    points = [{"block_threads": p.block_threads, "group_comps": p.group_comps, "status": _status_name(p.status),
               "ms_per_step": p.ms_per_step} for p in pts[:npts.value]]
    return {"block_threads": best.block_threads, "group_comps": best.group_comps, "points": points,
            "sample_comps": int(sample_comps)}


class Network:
    """A network living on one GPU; see include/mm.h for the semantics."""

    def __init__(self, net, precision: str = "fp64", cost: Optional[np.ndarray] = None, graph_steps: int = 40,
                 block_threads: int = 0, group_comps: int = 0, spike_capacity: int = 0, device: int = 0,
                 stream=None, torch_alloc: bool = True, time_items: bool = False, scheme: str = "be",
                 detect: str = "soma", deterministic: bool = False, n_ext_sources: int = 0):
        L = load()
        self._L = L
        self._h = C.c_void_p()
        self.n_neurons = net.n_neurons
        self.n_comp = net.n_comp
        self.dt = float(net.dt)
        # keep the NumPy inputs alive for the duration of the create call
        self._in, morph, chan, syn = _marshal(net)
        a = self._in
        opt = Options()
        L.mm_default_options(C.byref(opt))
        opt.precision = PRECISION[precision]
        opt.graph_steps = graph_steps
        opt.block_threads = block_threads
        opt.group_comps = group_comps
        opt.device = device
        opt.dt_ms = self.dt
        opt.spike_capacity = spike_capacity
        opt.time_items = 1 if time_items else 0
        opt.scheme = SCHEMES[scheme]
        opt.detect = DETECT[detect]
        opt.deterministic_delivery = 1 if deterministic else 0
        opt.n_ext_sources = int(n_ext_sources)
        # the library's automatic spike-buffer size (mm_options.spike_capacity)
        if spike_capacity > 0:
            self._spk_cap = int(spike_capacity)
        elif detect == "points":
            sc = a["scomp"] if a["scomp"] is not None else np.zeros(len(a["src"]), np.int32)
            n_pt = len(np.unique(a["src"].astype(np.int64) * (1 << 32) + sc))
            self._spk_cap = max(1 << 16, n_pt * 16)
        else:
            self._spk_cap = max(1 << 16, self.n_neurons * 64)
        self._spk_buf = None
        self._cost = None
        if cost is not None:
            self._cost = np.ascontiguousarray(cost, np.float32)
            opt.schedule = MM_SCHED_COST
            opt.cost = _ptr(self._cost, C.c_float)
        if stream is not None:
            opt.cuda_stream = C.c_void_p(int(stream))
        self._alloc = TorchAllocator(device) if torch_alloc else None
        if self._alloc is not None:
            opt.allocator = self._alloc.struct()
        st = L.mm_create_network(C.byref(morph), C.byref(chan), C.byref(syn), _ptr(a["stim"], C.c_double),
                                 C.byref(opt), C.byref(self._h))
        if st != MM_OK:
            raise MMError(st, "mm_create_network failed: " + L.mm_last_error(None).decode())
        self._in = None

    # ---------------------------------------------------------------- helpers
    def _check(self, st: int, what: str):
        if st != MM_OK:
            raise MMError(st, f"{what}: {self._L.mm_last_error(self._h).decode()}")

    def close(self):
        if self._h:
            self._L.mm_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------ calls
    def step(self, n_steps: int):
        self._check(self._L.mm_step(self._h, int(n_steps), self.dt), "mm_step")

    def synchronize(self):
        self._check(self._L.mm_synchronize(self._h), "mm_synchronize")

    @property
    def steps(self) -> int:
        s = C.c_int64()
        self._check(self._L.mm_get_step(self._h, C.byref(s)), "mm_get_step")
        return s.value

    def read_voltages(self, out: Optional[np.ndarray] = None) -> np.ndarray:
        return self.read_state("V", out)

    def read_state(self, which: str, out: Optional[np.ndarray] = None) -> np.ndarray:
        if out is None:
            out = np.empty(self.n_comp, np.float64)
        self._check(self._L.mm_read_state(self._h, STATE[which], _ptr(out, C.c_double), out.size), "mm_read_state")
        return out

    def read_soma(self, out: Optional[np.ndarray] = None) -> np.ndarray:
        if out is None:
            out = np.empty(self.n_neurons, np.float64)
        self._check(self._L.mm_read_soma_voltages(self._h, _ptr(out, C.c_double), out.size), "mm_read_soma_voltages")
        return out

    def _spike_arrays(self, cap: Optional[int]):
        # host arrays as large as the device buffer, kept between calls
        if cap is not None and cap != self._spk_cap:
            return np.empty(cap, np.int32), np.empty(cap, np.int32), np.empty(cap, np.float64), cap
        if self._spk_buf is None:
            c = self._spk_cap
            self._spk_buf = (np.empty(c, np.int32), np.empty(c, np.int32), np.empty(c, np.float64))
        return (*self._spk_buf, self._spk_cap)

    def read_spike_points(self, cap: Optional[int] = None):
        """(neuron, LOCAL compartment, t_ms) drained since the last call,
        ordered by (t, neuron, compartment)."""
        nr, cp, tt, cap = self._spike_arrays(cap)
        n = C.c_int64()
        st = self._L.mm_read_spike_points(self._h, _ptr(nr, C.c_int32), _ptr(cp, C.c_int32), _ptr(tt, C.c_double),
                                          cap, C.byref(n))
        self._check(st, "mm_read_spike_points")
        return nr[:n.value].copy(), cp[:n.value].copy(), tt[:n.value].copy()

    @property
    def spike_capacity(self) -> int:
        """Spike records the device buffer holds between two drains."""
        return self._spk_cap

    def read_outputs(self, soma: Optional[np.ndarray] = None):
        """One round trip per step: the soma voltages and the spikes drained
        since the last call, (soma, (neuron, compartment, t_ms))."""
        if soma is None:
            soma = np.empty(self.n_neurons, np.float64)
        nr, cp, tt, cap = self._spike_arrays(None)
        n = C.c_int64()
        st = self._L.mm_read_outputs(self._h, _ptr(soma, C.c_double), soma.size, _ptr(nr, C.c_int32),
                                     _ptr(cp, C.c_int32), _ptr(tt, C.c_double), cap, C.byref(n))
        self._check(st, "mm_read_outputs")
        return soma, (nr[:n.value].copy(), cp[:n.value].copy(), tt[:n.value].copy())

    def read_spikes(self, cap: Optional[int] = None, allow_overflow: bool = False):
        """(neuron, t_ms) drained since the last call, ordered by (t, neuron)."""
        nr, _, tt, cap = self._spike_arrays(cap)
        n = C.c_int64()
        st = self._L.mm_read_spikes(self._h, _ptr(nr, C.c_int32), _ptr(tt, C.c_double), cap, C.byref(n))
        if st == MM_EOVERFLOW and allow_overflow:
            k = min(cap, n.value)
            return nr[:k].copy(), tt[:k].copy()
        self._check(st, "mm_read_spikes")
        return nr[:n.value].copy(), tt[:n.value].copy()

    def inject_spikes(self, ext_src: np.ndarray, step: np.ndarray):
        """Spikes of the external sources (mm_inject_spikes): ext_src[k] fired in step[k]."""
        src = np.ascontiguousarray(ext_src, np.int32)
        stp = np.ascontiguousarray(step, np.int64)
        if src.shape != stp.shape:
            raise ValueError("ext_src and step differ in length")
        self._check(self._L.mm_inject_spikes(self._h, src.size, _ptr(src, C.c_int32), _ptr(stp, C.c_int64)),
                    "mm_inject_spikes")

    def read_fired(self, step0: int, n_steps: int):
        """(user neuron ids, steps) of this network's spikes in steps step0 .. step0 + n_steps - 1."""
        cap = max(1, self.n_neurons * max(1, n_steps))
        nrn = np.empty(cap, np.int32)
        stp = np.empty(cap, np.int64)
        n = C.c_int64(0)
        self._check(self._L.mm_read_fired(self._h, int(step0), int(n_steps), _ptr(nrn, C.c_int32),
                                          _ptr(stp, C.c_int64), cap, C.byref(n)), "mm_read_fired")
        return nrn[:n.value].copy(), stp[:n.value].copy()

    def set_stimulus(self, stim_nA: np.ndarray):
        s = np.ascontiguousarray(stim_nA, np.float64)
        self._check(self._L.mm_set_stimulus(self._h, _ptr(s, C.c_double), s.size), "mm_set_stimulus")

    def save_state(self) -> bytes:
        n = C.c_size_t()
        self._check(self._L.mm_save_state(self._h, None, 0, C.byref(n)), "mm_save_state")
        buf = C.create_string_buffer(n.value)
        self._check(self._L.mm_save_state(self._h, buf, n.value, C.byref(n)), "mm_save_state")
        return buf.raw

    def set_kernel_timing(self, enable: bool):
        self._check(self._L.mm_set_kernel_timing(self._h, 1 if enable else 0), "mm_set_kernel_timing")

    def read_kernel_timing(self, reset: bool = True) -> dict:
        t = KernelTimes()
        self._check(self._L.mm_read_kernel_timing(self._h, C.byref(t), 1 if reset else 0), "mm_read_kernel_timing")
        return {k: getattr(t, k) for k, _ in KernelTimes._fields_}

    def read_neuron_times(self) -> np.ndarray:
        out = np.empty(self.n_neurons, np.float64)
        self._check(self._L.mm_read_neuron_times(self._h, _ptr(out, C.c_double), out.size), "mm_read_neuron_times")
        return out

    def launch_info(self) -> dict:
        li = LaunchInfo()
        self._check(self._L.mm_get_launch_info(self._h, C.byref(li)), "mm_get_launch_info")
        return {k: (list(getattr(li, k)) if k in ("comps", "sites") else getattr(li, k)) for k, _ in LaunchInfo._fields_}

    def load_state(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        self._check(self._L.mm_load_state(self._h, buf, len(blob)), "mm_load_state")
