"""Exact vertex cover on one GB300: Python binding of libvc_gb300.so.

Argument marshalling only; every step of the solve runs in the CUDA library
(see ``include/vc_gb300.h``).  The library must be built first
(``python -m paper_2512_18334_gb300.build`` or ``__graft_entry__.build()``);
importing this package never falls back to anything else.

    import paper_2512_18334_gb300 as vc
    g = vc.Graph.from_csr(row_ptr, col)          # host numpy arrays
    size, cover, stats = vc.solve_min(g)
    yes, cover, stats = vc.solve_k(g, k)

    srv = vc.Server(max_induced=2048)                 # resident search, continuous batching
    srv.submit(row_ptr, col, tag=7)
    results = srv.drain()                             # steps until every request retired
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _lib as _L
from ._lib import (VC_OK, VC_EINVAL, VC_ENOMEM, VC_ECAPACITY, VC_ETIMEOUT, VC_ECUDA, VC_EBUDGET,
                   VcError, Options, Stats, ServerConfig, ServerResult, ServerStats, lib_path)

__all__ = [
    "Graph", "solve_min", "solve_k", "solve_mis", "solve_batch", "autotune", "trim", "options", "Server", "VcError",
    "lib_path",
    "VC_OK", "VC_EINVAL", "VC_ENOMEM", "VC_ECAPACITY", "VC_ETIMEOUT", "VC_ECUDA", "VC_EBUDGET",
]


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(int(stream.cuda_stream))   # torch.cuda.Stream


_DEFAULTS: bytes | None = None


def options(**kw) -> Options:
    """vc_options with the library defaults, overridden by keyword."""
    global _DEFAULTS
    if _DEFAULTS is None:
        o = Options()
        _L.check(_L.lib().vc_options_default(ctypes.byref(o)))
        _DEFAULTS = bytes(o)
    o = Options.from_buffer_copy(_DEFAULTS)
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


class Graph:
    """A CSR graph resident on the device (owns a vc_graph handle)."""

    def __init__(self, handle, n: int, m2: int):
        self._h = handle
        self.n = n
        self.m2 = m2

    @classmethod
    def from_csr(cls, row_ptr, col, stream=None) -> "Graph":
        """Copy host CSR arrays (int32) to the device (vc_load_csr)."""
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        c = np.ascontiguousarray(col, dtype=np.int32)
        n = int(rp.size - 1)
        h = ctypes.c_void_p()
        _L.check(_L.lib().vc_load_csr(n, rp.ctypes.data_as(ctypes.c_void_p),
                                      c.ctypes.data_as(ctypes.c_void_p) if c.size else None,
                                      _stream_handle(stream), ctypes.byref(h)))
        return cls(h, n, int(rp[-1]) if n >= 0 else 0)

    @classmethod
    def from_device(cls, row_ptr, col, stream=None) -> "Graph":
        """CSR already in HBM: torch int32 CUDA tensors (vc_load_csr_device)."""
        if row_ptr.dtype.itemsize != 4 or col.dtype.itemsize != 4:
            raise TypeError("row_ptr and col must be int32")
        if not (row_ptr.is_cuda and col.is_cuda):
            raise TypeError("from_device expects CUDA tensors")
        rp = row_ptr.contiguous()
        c = col.contiguous()
        n = int(rp.numel() - 1)
        h = ctypes.c_void_p()
        _L.check(_L.lib().vc_load_csr_device(n, ctypes.c_void_p(rp.data_ptr()),
                                             ctypes.c_void_p(c.data_ptr()) if c.numel() else None,
                                             _stream_handle(stream), ctypes.byref(h)))
        return cls(h, n, int(c.numel()))

    def close(self):
        if self._h is not None and self._h.value:
            _L.lib().vc_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def trim() -> int:
    """Free the search workspaces kept between solves (vc_trim)."""
    return int(_L.lib().vc_trim())


def measure_l2_read(bytes_: int = 32 << 20, reps: int = 50, trials: int = 5, stream=None) -> float:
    """L2 read bandwidth of the current device in GB/s (vc_measure_l2_read)."""
    out = ctypes.c_double(0.0)
    _L.check(_L.lib().vc_measure_l2_read(int(bytes_), int(reps), int(trials), _stream_handle(stream),
                                         ctypes.byref(out)))
    return float(out.value)


def _opts(opts, kw):
    if opts is None:
        return options(**kw)
    if kw:
        raise TypeError("pass either an Options object or keywords")
    return opts


def solve_min(g: Graph, opts: Options | None = None, want_cover: bool = True, **kw):
    """Minimum vertex cover: (size, cover int32 array or None, stats dict)."""
    o = _opts(opts, kw)
    size = ctypes.c_int32(-1)
    cover = np.empty(max(g.n, 1), np.int32) if want_cover else None
    clen = ctypes.c_int32(0)
    st = Stats()
    _L.check(_L.lib().vc_solve_min(g._h, ctypes.byref(o), ctypes.byref(size),
                                   cover.ctypes.data if want_cover else None,
                                   ctypes.byref(clen), ctypes.byref(st)), st)
    return size.value, (cover[:clen.value] if want_cover else None), st.to_dict()


def solve_k(g: Graph, k: int, opts: Options | None = None, want_cover: bool = True, **kw):
    """Is there a cover of size <= k?  (yes, cover or None, stats dict)."""
    o = _opts(opts, kw)
    yes = ctypes.c_int32(0)
    cover = np.zeros(max(g.n, 1), np.int32)
    clen = ctypes.c_int32(0)
    st = Stats()
    _L.check(_L.lib().vc_solve_k(g._h, int(k), ctypes.byref(o), ctypes.byref(yes),
                                 cover.ctypes.data_as(ctypes.c_void_p) if want_cover else None,
                                 ctypes.byref(clen), ctypes.byref(st)), st)
    return bool(yes.value), (cover[:clen.value].copy() if want_cover and yes.value else None), st.to_dict()


def solve_mis(g: Graph, opts: Options | None = None, want_set: bool = True, **kw):
    """Exact maximum independent set (complement of a minimum cover):
    (size, vertex int32 array or None, stats dict)."""
    o = _opts(opts, kw)
    size = ctypes.c_int32(-1)
    out = np.zeros(max(g.n, 1), np.int32)
    slen = ctypes.c_int32(0)
    st = Stats()
    _L.check(_L.lib().vc_solve_mis(g._h, ctypes.byref(o), ctypes.byref(size),
                                   out.ctypes.data_as(ctypes.c_void_p) if want_set else None,
                                   ctypes.byref(slen), ctypes.byref(st)), st)
    return size.value, (out[:slen.value].copy() if want_set else None), st.to_dict()


TUNED_FIELDS = ("team", "dtype_bytes", "offload_below", "stack_depth", "worklist_capacity")


def autotune(graphs, ks=None, opts: Options | None = None, repeats: int = 2, max_trials: int = 64, **kw):
    """vc_autotune on a batch: (best Options, best ms, [(options dict, ms), ...])."""
    o = _opts(opts, kw)
    count = len(graphs)
    arr = (ctypes.c_void_p * count)(*[gr._h for gr in graphs])
    ks_arr = None
    if ks is not None:
        ks_np = np.ascontiguousarray(ks, dtype=np.int32)
        ks_arr = ks_np.ctypes.data_as(ctypes.c_void_p)
    best = Options()
    best_ms = ctypes.c_double(0.0)
    tried = (Options * max_trials)()
    tried_ms = (ctypes.c_double * max_trials)()
    n = ctypes.c_int32(0)
    _L.check(_L.lib().vc_autotune(count, arr, ks_arr, ctypes.byref(o), int(repeats), ctypes.byref(best),
                                  ctypes.byref(best_ms), tried, tried_ms, max_trials, ctypes.byref(n)))
    table = [({f: getattr(tried[i], f) for f in TUNED_FIELDS}, tried_ms[i]) for i in range(min(n.value, max_trials))]
    return best, best_ms.value, table


def solve_batch(graphs, ks=None, opts: Options | None = None, want_covers: bool = True,
                raise_on_error: bool = True, **kw):
    """Many queries in one launch.  ks[i] < 0 (or ks None) asks for the minimum
    cover of graphs[i]; ks[i] >= 0 asks whether a cover <= ks[i] exists.
    Returns (sizes, yes, status, covers list or None, stats dict)."""
    o = _opts(opts, kw)
    count = len(graphs)
    arr = (ctypes.c_void_p * count)(*[gr._h for gr in graphs])
    ks_arr = None
    if ks is not None:
        ks_np = np.ascontiguousarray(ks, dtype=np.int32)
        ks_arr = ks_np.ctypes.data_as(ctypes.c_void_p)
    sizes = np.zeros(count, np.int32)
    yes = np.zeros(count, np.int32)
    status = np.zeros(count, np.int32)
    lens = np.zeros(count, np.int32)
    bufs = [np.zeros(max(gr.n, 1), np.int32) for gr in graphs] if want_covers else None
    cov_ptrs = (ctypes.c_void_p * count)(*[b.ctypes.data for b in bufs]) if want_covers else None
    st = Stats()
    rc = _L.lib().vc_solve_batch(count, arr, ks_arr, ctypes.byref(o),
                                 sizes.ctypes.data_as(ctypes.c_void_p), yes.ctypes.data_as(ctypes.c_void_p),
                                 status.ctypes.data_as(ctypes.c_void_p), cov_ptrs,
                                 lens.ctypes.data_as(ctypes.c_void_p), ctypes.byref(st))
    if raise_on_error:
        _L.check(rc, st)
    covers = [b[:l].copy() for b, l in zip(bufs, lens)] if want_covers else None
    return sizes, yes.astype(bool), status, covers, st.to_dict()


class Server:
    """Request server with continuous batching (vc_server_*): requests are
    admitted by device memory, root-reduced and searched in time slices
    together with the requests already in flight; the search state stays
    resident on the device between steps."""

    def __init__(self, stream=None, **cfg):
        c = ServerConfig()
        _L.check(_L.lib().vc_server_config_default(ctypes.byref(c)))
        for k, v in cfg.items():
            if not hasattr(c, k):
                raise TypeError(f"unknown server option {k}")
            setattr(c, k, v)
        self.config = c
        self._h = ctypes.c_void_p()
        _L.check(_L.lib().vc_server_create(ctypes.byref(c), _stream_handle(stream), ctypes.byref(self._h)))
        self._covers = np.zeros(1 << 20, np.int32)
        self._next_tag = 0

    def submit(self, row_ptr, col, k: int = -1, tag: int | None = None) -> int:
        """Queue one graph (host CSR arrays, copied); returns its tag."""
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        cl = np.ascontiguousarray(col, dtype=np.int32)
        if tag is None:
            tag = self._next_tag
        self._next_tag = max(self._next_tag, int(tag) + 1)
        _L.check(_L.lib().vc_server_submit(self._h, int(rp.size - 1), rp.ctypes.data_as(ctypes.c_void_p),
                                           cl.ctypes.data_as(ctypes.c_void_p) if cl.size else None,
                                           int(k), int(tag)))
        return int(tag)

    def step(self) -> int:
        """One scheduling iteration; returns the number of requests retired."""
        done = ctypes.c_int32(0)
        _L.check(_L.lib().vc_server_step(self._h, ctypes.byref(done)))
        return done.value

    def counts(self):
        """(queued, in flight, retired but not polled)."""
        q, f, r = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _L.check(_L.lib().vc_server_counts(self._h, ctypes.byref(q), ctypes.byref(f), ctypes.byref(r)))
        return q.value, f.value, r.value

    def poll(self, max_results: int = 4096) -> list:
        """Retired requests in completion order, as dicts with the cover."""
        out = []
        while True:
            res = (ServerResult * max_results)()
            cnt = ctypes.c_int32(0)
            _L.check(_L.lib().vc_server_poll(self._h, max_results, res, ctypes.byref(cnt),
                                             self._covers.ctypes.data_as(ctypes.c_void_p),
                                             int(self._covers.size)))
            for i in range(cnt.value):
                r = res[i]
                d = {name: getattr(r, name) for name, _ in ServerResult._fields_}
                off, ln = r.cover_off, r.cover_len
                d["cover"] = self._covers[off:off + ln].copy() if ln > 0 else np.zeros(0, np.int32)
                out.append(d)
            if cnt.value == 0:
                if self.counts()[2] > 0:            # the next cover is larger than the buffer
                    self._covers = np.zeros(self._covers.size * 2, np.int32)
                    continue
                return out
            if cnt.value < max_results and self.counts()[2] == 0:
                return out

    def drain(self, max_steps: int = 1 << 30) -> list:
        """Step until nothing is queued or in flight; returns every result."""
        out = []
        for _ in range(max_steps):
            q, f, _r = self.counts()
            if q == 0 and f == 0:
                break
            self.step()
            out.extend(self.poll())
        out.extend(self.poll())
        return out

    def stats(self) -> dict:
        st = ServerStats()
        _L.check(_L.lib().vc_server_get_stats(self._h, ctypes.byref(st)))
        return st.to_dict()

    def close(self):
        if self._h is not None and self._h.value:
            _L.lib().vc_server_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
