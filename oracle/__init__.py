"""CPU oracle for exact vertex cover -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA solver never calls it and
shares no code with it; the product path fails loudly when its CUDA library
is missing instead of falling back here.

The arithmetic lives in ``vc_oracle.c`` (plain sequential C, written from the
paper's definitions and Algorithm 2).  This module compiles it with gcc on
first use and wraps it with ctypes.  Every function takes CSR arrays
(``row_ptr`` int32[n+1], ``col`` int32[row_ptr[n]]).

Pinned by ``tests/test_oracle_pins.py`` against brute force, closed forms,
Koenig's theorem, additivity over disjoint unions and relabelling invariance.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_libs: dict = {}

EBUDGET = -2


class OracleBudgetExceeded(RuntimeError):
    pass


def build(mutant: int = 0) -> str:
    """Compile the oracle (optionally with a planted mistake, for the pin
    self-test) and return the path of the shared library."""
    os.makedirs(_BUILD, exist_ok=True)
    name = "liboracle.so" if mutant == 0 else f"liboracle_mut{mutant}.so"
    out = os.path.join(_BUILD, name)
    if (not os.path.exists(out)) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC]
        if mutant:
            cmd.insert(1, f"-DORC_MUTANT={mutant}")
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def _lib(mutant: int = 0):
    with _lock:
        if mutant not in _libs:
            lib = ctypes.CDLL(build(mutant))
            P = ctypes.c_void_p
            I = ctypes.c_int
            LL = ctypes.c_longlong
            lib.orc_verify_cover.argtypes = [I, P, P, P]
            lib.orc_brute_mvc.argtypes = [I, P, P, P]
            lib.orc_greedy.argtypes = [I, P, P, P]
            lib.orc_mvc.argtypes = [I, P, P, LL, I, P, P]
            lib.orc_pvc.argtypes = [I, P, P, I, LL, P, P, P]
            lib.orc_max_matching.argtypes = [I, P, P, P]
            lib.orc_rule_violation.argtypes = [I, P, P, P, LL]
            lib.orc_rule_violation.restype = LL
            _libs[mutant] = lib
        return _libs[mutant]


def _csr(row_ptr, col):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    c = np.ascontiguousarray(col, dtype=np.int32)
    if c.size == 0:
        c = np.zeros(1, dtype=np.int32)
    return rp, c


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def verify_cover(n, row_ptr, col, cover_flags, mutant: int = 0) -> bool:
    rp, c = _csr(row_ptr, col)
    f = np.ascontiguousarray(cover_flags, dtype=np.uint8)
    if f.size == 0:
        f = np.zeros(1, np.uint8)
    return bool(_lib(mutant).orc_verify_cover(n, _p(rp), _p(c), _p(f)))


def brute_mvc(n, row_ptr, col, mutant: int = 0):
    """(size, cover flags) by enumerating subsets in increasing size; n <= 30."""
    rp, c = _csr(row_ptr, col)
    out = np.zeros(max(n, 1), np.uint8)
    k = _lib(mutant).orc_brute_mvc(n, _p(rp), _p(c), _p(out))
    if k < 0:
        raise ValueError("brute force needs n <= 30")
    return k, out[:n]


def greedy(n, row_ptr, col):
    rp, c = _csr(row_ptr, col)
    out = np.zeros(max(n, 1), np.uint8)
    k = _lib().orc_greedy(n, _p(rp), _p(c), _p(out))
    return k, out[:n]


def mvc(n, row_ptr, col, node_budget: int = 0, use_components: bool = True,
        mutant: int = 0):
    """Exact MVC by Algorithm 2.  Returns (size, cover flags, stats dict)."""
    rp, c = _csr(row_ptr, col)
    out = np.zeros(max(n, 1), np.uint8)
    st = np.zeros(2, np.int64)
    k = _lib(mutant).orc_mvc(n, _p(rp), _p(c), int(node_budget), int(use_components),
                             _p(out), _p(st))
    if k == EBUDGET:
        raise OracleBudgetExceeded(f"more than {node_budget} search-tree nodes")
    if k < 0:
        raise RuntimeError(f"oracle error {k}")
    return k, out[:n], {"nodes": int(st[0]), "component_branches": int(st[1])}


def pvc(n, row_ptr, col, k: int, node_budget: int = 0, mutant: int = 0):
    """Is there a cover of size <= k?  Returns (yes, size or -1, cover flags)."""
    rp, c = _csr(row_ptr, col)
    out = np.zeros(max(n, 1), np.uint8)
    size = ctypes.c_int(-1)
    st = np.zeros(2, np.int64)
    r = _lib(mutant).orc_pvc(n, _p(rp), _p(c), int(k), int(node_budget), _p(out),
                             ctypes.byref(size), _p(st))
    if r == EBUDGET:
        raise OracleBudgetExceeded(f"more than {node_budget} search-tree nodes")
    if r < 0:
        raise RuntimeError(f"oracle error {r}")
    return bool(r), int(size.value), out[:n]


def max_matching(n, row_ptr, col):
    """Size of a maximum matching of a bipartite graph (-1 if not bipartite)."""
    rp, c = _csr(row_ptr, col)
    mate = np.zeros(max(n, 1), np.int32)
    k = _lib().orc_max_matching(n, _p(rp), _p(c), _p(mate))
    return k, mate[:n]


def rule_violation(n, row_ptr, col, removed_flags, b: int):
    """None if no Section 2.2 rule applies to G minus the removed vertices,
    else (vertex, rule) with rule in {"degree-one", "triangle", "high-degree"}."""
    rp, c = _csr(row_ptr, col)
    f = np.ascontiguousarray(removed_flags, dtype=np.uint8)
    if f.size == 0:
        f = np.zeros(1, np.uint8)
    r = _lib().orc_rule_violation(n, _p(rp), _p(c), _p(f), int(b))
    if r < 0:
        return None
    return int(r // 4), {1: "degree-one", 2: "triangle", 3: "high-degree"}[int(r % 4)]
