"""CPU oracle for the exhaustive flux-balanced pathway traversal.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_1804_02867_gb300``) and never imports it.

* ``efm_oracle.c``  -- the plain C enumerator (built into ``liboracle.so``);
* ``reference.py``  -- a pure-Python restatement for tiny inputs;
* ``bruteforce.py`` -- brute-force EFM enumeration over every support;
* ``mlp.py``        -- fp64 forward / gradient of the proposal model.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "efm_oracle.c")

TRUNCATED, CAPPED, OVERFLOW_DROPPED = 1, 2, 4
COUNTER_FIELDS = ("levels", "seeds", "expansions", "overflow", "balanced", "candidates", "results",
                  "pruned", "frontier", "frontier_max", "status", "zero_flux")


class _Limits(ctypes.Structure):
    _fields_ = [("max_len", ctypes.c_int32), ("max_secondary", ctypes.c_int32),
                ("max_results", ctypes.c_int64), ("max_frontier", ctypes.c_int64),
                ("flags", ctypes.c_int32), ("reserved", ctypes.c_int32)]


NO_PRUNE = 1  # _Limits.flags: skip the superset rule (the plain definition)
SUBTRACTIVE = 2  # _Limits.flags: Eq. 5 steps as well (states carry their flux vector)


class _Counters(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in COUNTER_FIELDS]


@dataclass
class Limits:
    max_len: int = 64
    max_secondary: int = 4
    max_results: int = 0
    max_frontier: int = 0
    prune: bool = True  # False: no superset rule, the definition alone
    subtractive: bool = False  # True: Eq. 5 steps with the zero-flux discard of Prop. 3

    def c_struct(self) -> "_Limits":
        flags = (0 if self.prune else NO_PRUNE) | (SUBTRACTIVE if self.subtractive else 0)
        return _Limits(self.max_len, self.max_secondary, self.max_results, self.max_frontier, flags, 0)


def build(force: bool = False) -> str:
    """Compile the C oracle (plain gcc, no architecture-specific flags)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-Wall", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER
        lib.oracle_enumerate.argtypes = [
            ctypes.c_int32, ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32),
            P(ctypes.c_uint8), P(ctypes.c_uint8), ctypes.c_int32, P(_Limits),
            P(P(ctypes.c_uint64)), P(ctypes.c_int64), P(ctypes.c_int32), P(_Counters)]
        lib.oracle_enumerate.restype = ctypes.c_int
        lib.oracle_rank.argtypes = [ctypes.c_int32, ctypes.c_int32, P(ctypes.c_int64), ctypes.c_int32,
                                    P(ctypes.c_int32)]
        lib.oracle_rank.restype = ctypes.c_int
        lib.oracle_column_map.argtypes = [ctypes.c_int32, P(ctypes.c_uint8), P(ctypes.c_int32),
                                          P(ctypes.c_int32)]
        lib.oracle_column_map.restype = ctypes.c_int
        lib.oracle_enumerate_from.argtypes = [
            ctypes.c_int32, ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32),
            P(ctypes.c_uint8), P(ctypes.c_uint8), P(ctypes.c_int32), ctypes.c_int32, P(_Limits),
            P(P(ctypes.c_uint64)), P(ctypes.c_int64), P(ctypes.c_int32), P(_Counters)]
        lib.oracle_enumerate_from.restype = ctypes.c_int
        lib.oracle_sample.argtypes = [
            ctypes.c_int32, ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32),
            P(ctypes.c_uint8), P(ctypes.c_uint8), ctypes.c_int32, P(_Limits), ctypes.c_uint64, ctypes.c_int64,
            P(P(ctypes.c_uint64)), P(ctypes.c_int64), P(ctypes.c_int32), P(_Counters)]
        lib.oracle_sample.restype = ctypes.c_int
        lib.oracle_splitmix_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.oracle_splitmix_at.restype = ctypes.c_uint64
        lib.oracle_free.argtypes = [ctypes.c_void_p]
        lib.oracle_free.restype = None
        _lib = lib
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def enumerate_pathways(net, target: int, limits: Limits):
    """Run the C oracle for one (network, target).  Returns
    (supports uint64[n, W] sorted by (|U|, column list), counters dict)."""
    lib = _load()
    rp = np.ascontiguousarray(net.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(net.col_idx, dtype=np.int32)
    cf = np.ascontiguousarray(net.coef, dtype=np.int32)
    rv = np.ascontiguousarray(net.reversible, dtype=np.uint8)
    ex = np.ascontiguousarray(net.external, dtype=np.uint8)
    lim = limits.c_struct()
    out = ctypes.POINTER(ctypes.c_uint64)()
    n = ctypes.c_int64(0)
    W = ctypes.c_int32(0)
    ctr = _Counters()
    rc = lib.oracle_enumerate(net.n_met, net.n_rxn, _ptr(rp, ctypes.c_int32), _ptr(ci, ctypes.c_int32),
                              _ptr(cf, ctypes.c_int32), _ptr(rv, ctypes.c_uint8), _ptr(ex, ctypes.c_uint8),
                              int(target), ctypes.byref(lim), ctypes.byref(out), ctypes.byref(n),
                              ctypes.byref(W), ctypes.byref(ctr))
    if rc != 0:
        if out:
            lib.oracle_free(out)
        raise RuntimeError(f"oracle_enumerate failed with code {rc}")
    w = W.value
    if n.value > 0:
        arr = np.ctypeslib.as_array(out, shape=(n.value * w,)).copy().reshape(n.value, w)
    else:
        arr = np.zeros((0, w), dtype=np.uint64)
    lib.oracle_free(out)
    return arr, {f: int(getattr(ctr, f)) for f in COUNTER_FIELDS}


def enumerate_from(net, columns, limits: Limits):
    """The traversal from one seed set R_in of split columns (Prop. 1):
    every column of R_in starts with flux 1.  Returns (supports, counters)
    like enumerate_pathways."""
    lib = _load()
    rp = np.ascontiguousarray(net.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(net.col_idx, dtype=np.int32)
    cf = np.ascontiguousarray(net.coef, dtype=np.int32)
    rv = np.ascontiguousarray(net.reversible, dtype=np.uint8)
    ex = np.ascontiguousarray(net.external, dtype=np.uint8)
    cols = np.ascontiguousarray(columns, dtype=np.int32)
    lim = limits.c_struct()
    out = ctypes.POINTER(ctypes.c_uint64)()
    n = ctypes.c_int64(0)
    W = ctypes.c_int32(0)
    ctr = _Counters()
    rc = lib.oracle_enumerate_from(net.n_met, net.n_rxn, _ptr(rp, ctypes.c_int32), _ptr(ci, ctypes.c_int32),
                                   _ptr(cf, ctypes.c_int32), _ptr(rv, ctypes.c_uint8), _ptr(ex, ctypes.c_uint8),
                                   _ptr(cols, ctypes.c_int32), len(cols), ctypes.byref(lim), ctypes.byref(out),
                                   ctypes.byref(n), ctypes.byref(W), ctypes.byref(ctr))
    if rc != 0:
        if out:
            lib.oracle_free(out)
        raise RuntimeError(f"oracle_enumerate_from failed with code {rc}")
    w = W.value
    arr = np.ctypeslib.as_array(out, shape=(n.value * w,)).copy().reshape(n.value, w) if n.value > 0 else \
        np.zeros((0, w), dtype=np.uint64)
    lib.oracle_free(out)
    return arr, {f: int(getattr(ctr, f)) for f in COUNTER_FIELDS}


def sample_pathways(net, target: int, limits: Limits, seed: int, n_walks: int):
    """Monte-Carlo mode: n_walks random walks (one random OR branch per
    step, SplitMix64 counters under `seed`).  Returns (distinct accepted
    supports sorted like enumerate_pathways, counters dict)."""
    lib = _load()
    rp = np.ascontiguousarray(net.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(net.col_idx, dtype=np.int32)
    cf = np.ascontiguousarray(net.coef, dtype=np.int32)
    rv = np.ascontiguousarray(net.reversible, dtype=np.uint8)
    ex = np.ascontiguousarray(net.external, dtype=np.uint8)
    lim = Limits(limits.max_len, limits.max_secondary, 0, 0).c_struct()
    out = ctypes.POINTER(ctypes.c_uint64)()
    n = ctypes.c_int64(0)
    W = ctypes.c_int32(0)
    ctr = _Counters()
    rc = lib.oracle_sample(net.n_met, net.n_rxn, _ptr(rp, ctypes.c_int32), _ptr(ci, ctypes.c_int32),
                           _ptr(cf, ctypes.c_int32), _ptr(rv, ctypes.c_uint8), _ptr(ex, ctypes.c_uint8), int(target),
                           ctypes.byref(lim), ctypes.c_uint64(seed), int(n_walks), ctypes.byref(out), ctypes.byref(n),
                           ctypes.byref(W), ctypes.byref(ctr))
    if rc != 0:
        if out:
            lib.oracle_free(out)
        raise RuntimeError(f"oracle_sample failed with code {rc}")
    w = W.value
    arr = np.ctypeslib.as_array(out, shape=(n.value * w,)).copy().reshape(n.value, w) if n.value > 0 else \
        np.zeros((0, w), dtype=np.uint64)
    lib.oracle_free(out)
    return arr, {f: int(getattr(ctr, f)) for f in COUNTER_FIELDS}


def splitmix_at(seed: int, c: int) -> int:
    """The oracle's counter-based random number (SplitMix64 first output)."""
    return int(_load().oracle_splitmix_at(ctypes.c_uint64(seed), ctypes.c_uint64(c)))


def rank(A, force_big: bool = False) -> int:
    """Exact rank over Q of an integer matrix (Bareiss; bigint fallback)."""
    lib = _load()
    A = np.ascontiguousarray(np.asarray(A, dtype=np.int64))
    if A.ndim != 2 or A.size == 0:
        return 0
    r = ctypes.c_int32(0)
    rc = lib.oracle_rank(A.shape[0], A.shape[1], _ptr(A, ctypes.c_int64), int(force_big), ctypes.byref(r))
    if rc != 0:
        raise RuntimeError(f"oracle_rank failed with code {rc}")
    return r.value


def column_map(net):
    """Split columns: (original reaction, direction) per column."""
    lib = _load()
    rv = np.ascontiguousarray(net.reversible, dtype=np.uint8)
    n = net.n_rxn + int(rv.sum())
    cr = np.zeros(n, dtype=np.int32)
    cd = np.zeros(n, dtype=np.int32)
    lib.oracle_column_map(net.n_rxn, _ptr(rv, ctypes.c_uint8), _ptr(cr, ctypes.c_int32), _ptr(cd, ctypes.c_int32))
    return cr, cd


def supports_to_lists(supports) -> list:
    """uint64[n, W] bitsets -> list of ascending column tuples."""
    out = []
    for row in np.asarray(supports, dtype=np.uint64):
        cols = []
        for w, word in enumerate(row):
            word = int(word)
            while word:
                low = word & -word
                cols.append(w * 64 + low.bit_length() - 1)
                word ^= low
        out.append(tuple(cols))
    return out


def first_k(net, target: int, k: int, max_len: int, max_secondary: int):
    """The k smallest results (by |U|, then ascending column list) of the
    traversal with no frontier budget and no cap.

    Results of popcount <= P are exactly the results of the traversal run
    with max_len = P (every state on a path to such a result has popcount
    <= P), so the definition is evaluated by deepening P until at least k
    results of popcount <= P exist (or P = max_len), then keeping the k
    smallest.  Returns (supports uint64[min(k, n), W], the P used)."""
    for P in range(1, max_len + 1):
        sup, _ = enumerate_pathways(net, target, Limits(P, max_secondary, 0, 0))
        if len(sup) >= k or P == max_len:
            return sup[:k], P
    raise AssertionError("unreachable")


def first_k_within(net, target: int, k: int, max_len: int, max_secondary: int, max_frontier: int):
    """first_k evaluated under a frontier budget, for networks whose complete
    levels do not fit in host memory.  The same deepening; a run at P whose
    every level stayed within max_frontier holds exactly the results of
    popcount <= P, so the answer is the definition's.  Returns (supports,
    the P used, certified); certified is False when the run at P overflowed
    the budget, and the supports are then not the definition's answer."""
    for P in range(1, max_len + 1):
        sup, ctr = enumerate_pathways(net, target, Limits(P, max_secondary, 0, max_frontier))
        if ctr["status"] & TRUNCATED:
            return sup[:k], P, False
        if len(sup) >= k or P == max_len:
            return sup[:k], P, True
    raise AssertionError("unreachable")
