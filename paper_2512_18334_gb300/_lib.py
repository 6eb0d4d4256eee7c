"""ctypes declarations of include/vc_gb300.h.  Loads the in-tree library and
fails loudly when it is missing."""
from __future__ import annotations

import ctypes
import os
import struct
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_FILE = os.path.join(HERE, "libvc_gb300.so")

VC_OK = 0
VC_EINVAL = -1
VC_ENOMEM = -2
VC_ECAPACITY = -3
VC_ETIMEOUT = -4
VC_ECUDA = -5
VC_EBUDGET = -6

_lock = threading.Lock()
_lib = None


class VcError(RuntimeError):
    def __init__(self, status: int, msg: str, stats: dict | None = None):
        super().__init__(f"{msg} (status {status})")
        self.status = status
        self.stats = stats


class Options(ctypes.Structure):
    _fields_ = [
        ("use_components", ctypes.c_int32),
        ("team", ctypes.c_int32),
        ("dtype_bytes", ctypes.c_int32),
        ("stack_depth", ctypes.c_int32),
        ("worklist_capacity", ctypes.c_int32),
        ("registry_capacity", ctypes.c_int32),
        ("load_balance", ctypes.c_int32),
        ("idle_timeout_ms", ctypes.c_int32),
        ("node_budget", ctypes.c_int64),
        ("disable_bounds", ctypes.c_int32),
        ("disable_root_rules", ctypes.c_int32),
        ("breakdown", ctypes.c_int32),
        ("offload_below", ctypes.c_int32),
        ("disable_dyn_bounds", ctypes.c_int32),
        ("crown", ctypes.c_int32),
        ("cuda_graph", ctypes.c_int32),
        ("capacity_retries", ctypes.c_int32),
        ("label_propagation", ctypes.c_int32),
    ]


PHASES = ("pop", "reduce", "components", "branch", "complete", "idle")


class Stats(ctypes.Structure):
    _fields_ = [
        ("nodes", ctypes.c_int64),
        ("component_branches", ctypes.c_int64),
        ("leaves", ctypes.c_int64),
        ("pruned", ctypes.c_int64),
        ("offloaded", ctypes.c_int64),
        ("trivial_components", ctypes.c_int64),
        ("comp_hist", ctypes.c_int64 * 16),
        ("n", ctypes.c_int32),
        ("n_induced", ctypes.c_int32),
        ("m_induced", ctypes.c_int32),
        ("forced", ctypes.c_int32),
        ("greedy_size", ctypes.c_int32),
        ("dtype_bytes", ctypes.c_int32),
        ("team", ctypes.c_int32),
        ("workers", ctypes.c_int32),
        ("max_stack", ctypes.c_int32),
        ("err_where", ctypes.c_int32),
        ("launches", ctypes.c_int32),
        ("root_rounds", ctypes.c_int32),
        ("ms_root", ctypes.c_double),
        ("ms_search", ctypes.c_double),
        ("ms_total", ctypes.c_double),
        ("root_cycles", ctypes.c_int64 * 4),
        ("search_bytes", ctypes.c_int64),
        ("phase_cycles", ctypes.c_int64 * 6),
        ("crown_forced", ctypes.c_int32),
        ("crown_removed", ctypes.c_int32),
        ("crown_skipped", ctypes.c_int32),
        ("cuda_graph", ctypes.c_int32),
        ("retries", ctypes.c_int32),
        ("best_found", ctypes.c_int32),
    ]

    def to_dict(self) -> dict:
        # one unpack of the whole struct (a getattr per field costs more than
        # the rest of a small solve's host time)
        vals = _STATS_STRUCT.unpack_from(self)
        d = {}
        i = 0
        for name, ln in _STATS_LAYOUT:
            if ln:
                d[name] = vals[i:i + ln]
                i += ln
            else:
                d[name] = vals[i]
                i += 1
        h = d["comp_hist"]
        d["comp_hist"] = {k + 2: h[k] for k in range(16) if h[k]}
        d["root_cycles"] = list(d["root_cycles"])
        d["phase_cycles"] = dict(zip(PHASES, d["phase_cycles"]))
        return d


def _struct_of(cls):
    """A struct.Struct reading a ctypes Structure of int32 / int64 / double
    fields and arrays of them, and the (name, array length or 0) layout."""
    codes = {ctypes.c_int64: "q", ctypes.c_int32: "i", ctypes.c_double: "d"}
    fmt, layout, pos = "=", [], 0
    for name, ct in cls._fields_:
        off = getattr(cls, name).offset
        if off > pos:
            fmt += f"{off - pos}x"
        if issubclass(ct, ctypes.Array):
            fmt += codes[ct._type_] * ct._length_
            layout.append((name, ct._length_))
        else:
            fmt += codes[ct]
            layout.append((name, 0))
        pos = off + ctypes.sizeof(ct)
    if ctypes.sizeof(cls) > pos:
        fmt += f"{ctypes.sizeof(cls) - pos}x"
    return struct.Struct(fmt), layout


_STATS_STRUCT, _STATS_LAYOUT = _struct_of(Stats)


class ServerConfig(ctypes.Structure):
    _fields_ = [
        ("max_inflight", ctypes.c_int32),
        ("max_induced", ctypes.c_int32),
        ("dtype_bytes", ctypes.c_int32),
        ("team", ctypes.c_int32),
        ("stack_depth", ctypes.c_int32),
        ("worklist_capacity", ctypes.c_int32),
        ("registry_capacity", ctypes.c_int32),
        ("quantum_us", ctypes.c_int32),
        ("use_components", ctypes.c_int32),
        ("load_balance", ctypes.c_int32),
        ("idle_timeout_ms", ctypes.c_int32),
        ("max_induced_large", ctypes.c_int32),
        ("arena_bytes", ctypes.c_int64),
        ("node_budget", ctypes.c_int64),
        ("cover_buffer", ctypes.c_int64),
    ]


class ServerResult(ctypes.Structure):
    _fields_ = [
        ("tag", ctypes.c_int64),
        ("status", ctypes.c_int32),
        ("size", ctypes.c_int32),
        ("yes", ctypes.c_int32),
        ("n", ctypes.c_int32),
        ("n_induced", ctypes.c_int32),
        ("cover_len", ctypes.c_int32),
        ("cover_off", ctypes.c_int64),
        ("nodes", ctypes.c_int64),
        ("t_submit_ms", ctypes.c_double),
        ("t_admit_ms", ctypes.c_double),
        ("t_done_ms", ctypes.c_double),
    ]


class ServerStats(ctypes.Structure):
    _fields_ = [
        ("steps", ctypes.c_int64),
        ("slices", ctypes.c_int64),
        ("submitted", ctypes.c_int64),
        ("admitted", ctypes.c_int64),
        ("completed", ctypes.c_int64),
        ("nodes", ctypes.c_int64),
        ("search_bytes", ctypes.c_int64),
        ("h2d_bytes", ctypes.c_int64),
        ("d2h_bytes", ctypes.c_int64),
        ("resets", ctypes.c_int64),
        ("ms_admit", ctypes.c_double),
        ("ms_search", ctypes.c_double),
        ("ms_retire", ctypes.c_double),
        ("workers", ctypes.c_int32),
        ("team", ctypes.c_int32),
        ("dtype_bytes", ctypes.c_int32),
        ("max_induced", ctypes.c_int32),
        ("slot_bytes", ctypes.c_int32),
        ("max_stack", ctypes.c_int32),
        ("device_bytes", ctypes.c_int64),
        ("wait_polls", ctypes.c_int64),
        ("preemptions", ctypes.c_int64),
        ("max_node_ns", ctypes.c_int64),
        ("max_exit_ns", ctypes.c_int64),
    ]

    def to_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


# Every symbol the header declares, with its ctypes signature.
_P = ctypes.c_void_p
_I = ctypes.c_int32
SIGNATURES = {
    "vc_options_default": (ctypes.c_int, [_P]),
    "vc_load_csr": (ctypes.c_int, [_I, _P, _P, _P, _P]),
    "vc_load_csr_device": (ctypes.c_int, [_I, _P, _P, _P, _P]),
    "vc_solve_min": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "vc_solve_k": (ctypes.c_int, [_P, _I, _P, _P, _P, _P, _P]),
    "vc_solve_batch": (ctypes.c_int, [_I, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "vc_solve_mis": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "vc_autotune": (ctypes.c_int, [_I, _P, _P, _P, _I, _P, _P, _P, _P, _I, _P]),
    "vc_root_reduce_static": (ctypes.c_int, [_I, _I, _P, _P, _I, _P, _P, _P, _P, _P, _P]),
    "vc_free": (None, [_P]),
    "vc_trim": (ctypes.c_int, []),
    "vc_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "vc_last_cuda_error": (ctypes.c_char_p, []),
    "vc_server_config_default": (ctypes.c_int, [_P]),
    "vc_server_create": (ctypes.c_int, [_P, _P, _P]),
    "vc_server_submit": (ctypes.c_int, [_P, _I, _P, _P, _I, ctypes.c_int64]),
    "vc_server_step": (ctypes.c_int, [_P, _P]),
    "vc_server_counts": (ctypes.c_int, [_P, _P, _P, _P]),
    "vc_server_poll": (ctypes.c_int, [_P, _I, _P, _P, _P, ctypes.c_int64]),
    "vc_server_get_stats": (ctypes.c_int, [_P, _P]),
    "vc_server_free": (None, [_P]),
    "vc_measure_l2_read": (ctypes.c_int, [ctypes.c_int64, _I, _I, _P, _P]),
}


def lib_path() -> str:
    return _LIB_FILE


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_FILE):
                raise ImportError(
                    f"{_LIB_FILE} is missing: build it with "
                    "`python -m paper_2512_18334_gb300.build` (there is no fallback)")
            L = ctypes.CDLL(_LIB_FILE)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def strerror(status: int) -> str:
    return lib().vc_strerror(int(status)).decode()


def check(status: int, stats=None) -> None:
    if status != VC_OK:
        msg = strerror(status)
        if status in (VC_ECUDA, VC_ENOMEM):
            msg += ": " + lib().vc_last_cuda_error().decode()
        raise VcError(int(status), msg, stats.to_dict() if stats is not None else None)
