"""Thin ctypes binding over the C-ABI in include/efmgraph.h.

Argument marshalling only: every step of the traversal runs in the CUDA
kernels of libefmgraph.so.  Importing this module on a machine without the
built library raises -- there is no CPU fallback.

The C functions are exposed under their C names (efm_load_network, ...);
`Network` and `enumerate_targets` are conveniences that call exactly those.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

EFM_TRUNCATED, EFM_CAPPED, EFM_OVERFLOW_DROPPED = 1, 2, 4
COUNTER_FIELDS = ("levels", "seeds", "expansions", "overflow", "balanced", "candidates", "results", "pruned",
                  "frontier", "frontier_max", "status", "zero_flux")
EXPORTS = ("efm_load_network", "efm_network_shape", "efm_column_map", "efm_find_pathways", "efm_fetch_results",
           "efm_job_timing", "efm_free_job", "efm_free_net", "efm_status_str", "efm_set_allocator",
           "efm_sort_supports_noalloc", "efm_find_pathways_batch", "efm_batch_tuning", "efm_batch_set_tuning",
           "efm_model_create",
           "efm_model_params", "efm_model_add_rows", "efm_model_rows", "efm_model_clear_rows", "efm_model_forward",
           "efm_model_gradient", "efm_model_train", "efm_model_trace", "efm_model_free", "efm_sample_pathways",
           "efm_flux_vectors", "efm_find_pathways_from", "efm_dependent_reactions", "efm_check_bounded_wait")
EFM_NOALLOC_MAX_ROWS = 1 << 20
EFM_MLP_FEATURES, EFM_MLP_HIDDEN = 128, 256
EFM_MLP_PARAMS = 256 * 128 + 256 + 1


class efm_batch_tune(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int32), ("largest_first", ctypes.c_int32), ("warps_per_job", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("queue_chunk", ctypes.c_int32), ("pinned", ctypes.c_int32),
                ("sample_default_ms", ctypes.c_float), ("sample_tuned_ms", ctypes.c_float)]


class efm_limits(ctypes.Structure):
    _fields_ = [("max_len", ctypes.c_int32), ("max_secondary", ctypes.c_int32), ("max_results", ctypes.c_int64),
                ("max_frontier", ctypes.c_int64), ("first_k", ctypes.c_int32), ("proposal", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class efm_counters(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in COUNTER_FIELDS]


class EfmError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {status_str(code)} ({code})")
        self.code = code


_lib = None
_P = ctypes.POINTER


def library_path() -> str:
    return _build.LIB


def load_library(path: str | None = None):
    """Load libefmgraph.so (built in-tree by build.build()).  Raises if the
    library is missing: the product path has no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} not built; run paper_1804_02867_gb300.build.build()")
    lib = ctypes.CDLL(path)
    lib.efm_load_network.argtypes = [ctypes.c_int32, ctypes.c_int32, _P(ctypes.c_int32), _P(ctypes.c_int32),
                                     _P(ctypes.c_int32), _P(ctypes.c_uint8), _P(ctypes.c_uint8), ctypes.c_size_t,
                                     _P(ctypes.c_void_p)]
    lib.efm_load_network.restype = ctypes.c_int
    lib.efm_network_shape.argtypes = [ctypes.c_void_p, _P(ctypes.c_int32), _P(ctypes.c_int32), _P(ctypes.c_int32)]
    lib.efm_network_shape.restype = ctypes.c_int
    lib.efm_column_map.argtypes = [ctypes.c_void_p, _P(ctypes.c_int32), _P(ctypes.c_int8)]
    lib.efm_column_map.restype = ctypes.c_int
    lib.efm_find_pathways.argtypes = [ctypes.c_void_p, _P(ctypes.c_int32), ctypes.c_int32, _P(efm_limits),
                                      ctypes.c_void_p, _P(ctypes.c_void_p)]
    lib.efm_find_pathways.restype = ctypes.c_int
    lib.efm_fetch_results.argtypes = [ctypes.c_void_p, ctypes.c_int32, _P(ctypes.c_uint64), ctypes.c_int64,
                                      _P(ctypes.c_int64), _P(ctypes.c_int32), _P(efm_counters)]
    lib.efm_fetch_results.restype = ctypes.c_int
    lib.efm_job_timing.argtypes = [ctypes.c_void_p, ctypes.c_int32, _P(ctypes.c_double), _P(ctypes.c_double),
                                   _P(ctypes.c_int64), _P(ctypes.c_double), _P(ctypes.c_int64)]
    lib.efm_job_timing.restype = ctypes.c_int
    lib.efm_free_job.argtypes = [ctypes.c_void_p]
    lib.efm_free_job.restype = None
    lib.efm_free_net.argtypes = [ctypes.c_void_p]
    lib.efm_free_net.restype = None
    lib.efm_status_str.argtypes = [ctypes.c_int]
    lib.efm_status_str.restype = ctypes.c_char_p
    lib.efm_set_allocator.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.efm_set_allocator.restype = ctypes.c_int
    lib.efm_sort_supports_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                              ctypes.c_size_t]
    lib.efm_sort_supports_noalloc.restype = ctypes.c_int
    lib.efm_find_pathways_batch.argtypes = [_P(ctypes.c_void_p), _P(ctypes.c_int32), ctypes.c_int32, _P(efm_limits),
                                            ctypes.c_void_p, _P(ctypes.c_void_p)]
    lib.efm_find_pathways_batch.restype = ctypes.c_int
    lib.efm_batch_tuning.argtypes = [_P(efm_batch_tune)]
    lib.efm_batch_tuning.restype = ctypes.c_int
    lib.efm_batch_set_tuning.argtypes = [_P(efm_batch_tune)]
    lib.efm_batch_set_tuning.restype = ctypes.c_int
    F = _P(ctypes.c_float)
    lib.efm_model_create.argtypes = [ctypes.c_uint64, ctypes.c_size_t, _P(ctypes.c_void_p)]
    lib.efm_model_params.argtypes = [ctypes.c_void_p, F, ctypes.c_int32]
    lib.efm_model_add_rows.argtypes = [ctypes.c_void_p, F, F, ctypes.c_int64]
    lib.efm_model_rows.argtypes = [ctypes.c_void_p, _P(ctypes.c_int64), _P(ctypes.c_int64)]
    lib.efm_model_clear_rows.argtypes = [ctypes.c_void_p]
    lib.efm_model_forward.argtypes = [ctypes.c_void_p, F, ctypes.c_int64, F]
    lib.efm_model_gradient.argtypes = [ctypes.c_void_p, ctypes.c_float, F, F]
    lib.efm_model_train.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_uint64, F]
    lib.efm_model_trace.argtypes = [ctypes.c_void_p, ctypes.c_void_p, _P(ctypes.c_int32), ctypes.c_int32,
                                    _P(efm_limits), ctypes.c_int64]
    for name in ("efm_model_create", "efm_model_params", "efm_model_add_rows", "efm_model_rows",
                 "efm_model_clear_rows", "efm_model_forward", "efm_model_gradient", "efm_model_train",
                 "efm_model_trace"):
        getattr(lib, name).restype = ctypes.c_int
    lib.efm_dependent_reactions.argtypes = [ctypes.c_void_p, ctypes.c_int32, _P(ctypes.c_uint64), _P(ctypes.c_uint64),
                                            _P(ctypes.c_int32), _P(ctypes.c_double)]
    lib.efm_dependent_reactions.restype = ctypes.c_int
    lib.efm_find_pathways_from.argtypes = [ctypes.c_void_p, _P(ctypes.c_int32), ctypes.c_int32, _P(efm_limits),
                                           _P(ctypes.c_void_p)]
    lib.efm_find_pathways_from.restype = ctypes.c_int
    lib.efm_flux_vectors.argtypes = [ctypes.c_void_p, _P(ctypes.c_uint64), ctypes.c_int64, _P(ctypes.c_int64),
                                     _P(ctypes.c_int8)]
    lib.efm_flux_vectors.restype = ctypes.c_int
    lib.efm_sample_pathways.argtypes = [ctypes.c_void_p, ctypes.c_int32, _P(efm_limits), ctypes.c_uint64,
                                        ctypes.c_int64, _P(ctypes.c_void_p)]
    lib.efm_sample_pathways.restype = ctypes.c_int
    lib.efm_check_bounded_wait.argtypes = [ctypes.c_void_p, _P(ctypes.c_int64), _P(ctypes.c_double)]
    lib.efm_check_bounded_wait.restype = ctypes.c_int
    lib.efm_model_free.argtypes = [ctypes.c_void_p]
    lib.efm_model_free.restype = None
    _lib = lib
    return lib


def status_str(code: int) -> str:
    return load_library().efm_status_str(int(code)).decode()


def _arr(a, dt, ct):
    a = np.ascontiguousarray(a, dtype=dt)
    return a, a.ctypes.data_as(_P(ct))


def _stream_handle(stream) -> int:
    if stream is None:
        import torch

        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# --- C-ABI calls under their C names ---------------------------------------

def efm_load_network(n_met, n_rxn, row_ptr, col_idx, coef, reversible, external, stream=None) -> int:
    lib = load_library()
    rp, prp = _arr(row_ptr, np.int32, ctypes.c_int32)
    ci, pci = _arr(col_idx, np.int32, ctypes.c_int32)
    cf, pcf = _arr(coef, np.int32, ctypes.c_int32)
    rv, prv = _arr(reversible, np.uint8, ctypes.c_uint8)
    ex, pex = _arr(external, np.uint8, ctypes.c_uint8)
    h = ctypes.c_void_p()
    rc = lib.efm_load_network(int(n_met), int(n_rxn), prp, pci, pcf, prv, pex, _stream_handle(stream),
                              ctypes.byref(h))
    if rc != 0:
        raise EfmError(rc, "efm_load_network")
    return h.value


def efm_network_shape(net) -> tuple:
    n, w, m = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    rc = load_library().efm_network_shape(net, ctypes.byref(n), ctypes.byref(w), ctypes.byref(m))
    if rc != 0:
        raise EfmError(rc, "efm_network_shape")
    return n.value, w.value, m.value


def efm_column_map(net):
    n, _, _ = efm_network_shape(net)
    rx = np.zeros(n, dtype=np.int32)
    d = np.zeros(n, dtype=np.int8)
    rc = load_library().efm_column_map(net, rx.ctypes.data_as(_P(ctypes.c_int32)), d.ctypes.data_as(_P(ctypes.c_int8)))
    if rc != 0:
        raise EfmError(rc, "efm_column_map")
    return rx, d


EFM_PLAIN, EFM_LEARNED = 0, 1
EFM_ADDITIVE, EFM_SUBTRACTIVE = 0, 1


def efm_find_pathways(net, targets, max_len, max_secondary, max_results=0, max_frontier=0, first_k=0,
                      proposal=EFM_PLAIN, model=None, variant=EFM_ADDITIVE):
    """Returns (job handle, warning flags).  first_k > 0 asks for exactly the
    K smallest results; proposal / model set the order of that search;
    variant EFM_SUBTRACTIVE adds the Eq. 5 steps."""
    tg, ptg = _arr(targets, np.int32, ctypes.c_int32)
    lim = efm_limits(int(max_len), int(max_secondary), int(max_results), int(max_frontier), int(first_k),
                     int(proposal), int(variant), 0)
    job = ctypes.c_void_p()
    rc = load_library().efm_find_pathways(net, ptg, len(tg), ctypes.byref(lim), model, ctypes.byref(job))
    if rc < 0:
        raise EfmError(rc, "efm_find_pathways")
    return job.value, rc


def efm_find_pathways_from(net, columns, max_len, max_secondary, max_results=0, max_frontier=0, first_k=0,
                           variant=EFM_ADDITIVE):
    """Traversal from a seed set of split columns.  Returns (job, flags)."""
    cols, pc = _arr(columns, np.int32, ctypes.c_int32)
    lim = efm_limits(int(max_len), int(max_secondary), int(max_results), int(max_frontier), int(first_k), EFM_PLAIN,
                     int(variant), 0)
    job = ctypes.c_void_p()
    rc = load_library().efm_find_pathways_from(net, pc, len(cols), ctypes.byref(lim), ctypes.byref(job))
    if rc < 0:
        raise EfmError(rc, "efm_find_pathways_from")
    return job.value, rc


def enumerate_from(network, columns, max_len, max_secondary, max_results=0, max_frontier=0, first_k=0,
                   variant=EFM_ADDITIVE):
    """efm_find_pathways_from + fetch: (supports, counters)."""
    job, _ = efm_find_pathways_from(network.handle, columns, max_len, max_secondary, max_results, max_frontier,
                                    first_k, variant)
    try:
        sup, ctr, _ = efm_fetch_results(job, 0)
        return sup, ctr
    finally:
        efm_free_job(job)


def efm_dependent_reactions(network, depth):
    """DEPTHy: (dep_out, dep_in) bool[M_int, N] flux-dependent column tags,
    r (most steps out of a metabolite), kernel ms."""
    M, W, N = network.n_internal, network.words, network.n_columns
    o = np.zeros((max(M, 1), W), dtype=np.uint64)
    i = np.zeros((max(M, 1), W), dtype=np.uint64)
    r = ctypes.c_int32()
    ms = ctypes.c_double()
    rc = load_library().efm_dependent_reactions(network.handle, int(depth), o.ctypes.data_as(_P(ctypes.c_uint64)),
                                                i.ctypes.data_as(_P(ctypes.c_uint64)), ctypes.byref(r),
                                                ctypes.byref(ms))
    if rc != 0:
        raise EfmError(rc, "efm_dependent_reactions")

    def bits(a):
        b = np.unpackbits(a[:M].view(np.uint8), axis=1, bitorder="little").astype(bool)
        return b[:, :N]
    return bits(o), bits(i), r.value, ms.value


EFM_FLUX_COLUMNS = 64


def efm_flux_vectors(net, supports):
    """Flux vectors of uint64[n, W] supports: (int64[n, 64] fluxes in
    ascending column order, int8[n] status: 1 exact, 0 overflow, -1 not a
    single positive ray)."""
    sup = np.ascontiguousarray(supports, dtype=np.uint64)
    n = sup.shape[0] if sup.ndim == 2 else 0
    flux = np.zeros((max(n, 1), EFM_FLUX_COLUMNS), dtype=np.int64)
    st = np.zeros(max(n, 1), dtype=np.int8)
    rc = load_library().efm_flux_vectors(net, sup.ctypes.data_as(_P(ctypes.c_uint64)), n,
                                         flux.ctypes.data_as(_P(ctypes.c_int64)), st.ctypes.data_as(_P(ctypes.c_int8)))
    if rc != 0:
        raise EfmError(rc, "efm_flux_vectors")
    return flux[:n], st[:n]


def efm_check_bounded_wait(net):
    """Run the library's bounded-wait failure path once (a device wait on a
    flag that nothing sets).  Returns (status, polls, waited_ms); the status
    is EFM_ETIMEOUT (-4) when the wait gave up, as it should.  Other
    errors raise EfmError."""
    polls, ms = ctypes.c_int64(), ctypes.c_double()
    rc = load_library().efm_check_bounded_wait(net, ctypes.byref(polls), ctypes.byref(ms))
    if rc < 0 and rc != -4:
        raise EfmError(rc, "efm_check_bounded_wait")
    return rc, polls.value, ms.value


def efm_sample_pathways(net, target, max_len, max_secondary, seed, n_walks):
    """Monte-Carlo walks.  Returns (job handle, warning flags)."""
    lim = efm_limits(int(max_len), int(max_secondary), 0, 0, 0, 0)
    job = ctypes.c_void_p()
    rc = load_library().efm_sample_pathways(net, int(target), ctypes.byref(lim), ctypes.c_uint64(int(seed)),
                                            int(n_walks), ctypes.byref(job))
    if rc < 0:
        raise EfmError(rc, "efm_sample_pathways")
    return job.value, rc


def sample_target(network, target, max_len, max_secondary, seed, n_walks, timing=False):
    """efm_sample_pathways + fetch: (supports, counters[, timing dict])."""
    job, _ = efm_sample_pathways(network.handle, target, max_len, max_secondary, seed, n_walks)
    try:
        sup, ctr, _ = efm_fetch_results(job, 0)
        return (sup, ctr, efm_job_timing(job, 0)) if timing else (sup, ctr)
    finally:
        efm_free_job(job)


def efm_find_pathways_batch(nets, targets, max_len, max_secondary, max_results=0, max_frontier=1 << 12):
    """One job per (net handle, target) in one persistent launch.
    Returns (job handle, OR of warning flags)."""
    hs = (ctypes.c_void_p * len(nets))(*[ctypes.c_void_p(h) for h in nets])
    tg, ptg = _arr(targets, np.int32, ctypes.c_int32)
    lim = efm_limits(int(max_len), int(max_secondary), int(max_results), int(max_frontier), 0, 0)
    job = ctypes.c_void_p()
    rc = load_library().efm_find_pathways_batch(hs, ptg, len(tg), ctypes.byref(lim), None, ctypes.byref(job))
    if rc < 0:
        raise EfmError(rc, "efm_find_pathways_batch")
    return job.value, rc


TUNE_FIELDS = ("ctas_per_sm", "largest_first", "warps_per_job", "tile", "queue_chunk", "pinned", "sample_default_ms",
               "sample_tuned_ms")


def efm_batch_tuning():
    """The configuration the last batch ran with, as a dict (None before any)."""
    t = efm_batch_tune()
    rc = load_library().efm_batch_tuning(ctypes.byref(t))
    return {f: getattr(t, f) for f in TUNE_FIELDS} if rc == 0 else None


def efm_batch_set_tuning(cfg=None, **kw):
    """Pin the batched launch configuration (ctas_per_sm, largest_first,
    warps_per_job, tile, queue_chunk), or return to the search with None."""
    if cfg is None and not kw:
        rc = load_library().efm_batch_set_tuning(None)
    else:
        t = efm_batch_tune()
        for f, v in {**(cfg or {}), **kw}.items():
            if f in TUNE_FIELDS[:5]:
                setattr(t, f, int(v))
        rc = load_library().efm_batch_set_tuning(ctypes.byref(t))
    if rc < 0:
        raise EfmError(rc, "efm_batch_set_tuning")


def efm_fetch_results(job, idx, copy=True, out=None):
    """Returns (supports uint64[n, W] or None if copy is False, counters
    dict, flags).  `out` may supply the host buffer (e.g. pinned memory)."""
    lib = load_library()
    n = ctypes.c_int64()
    w = ctypes.c_int32()
    ctr = efm_counters()
    rc = lib.efm_fetch_results(job, int(idx), None, 0, ctypes.byref(n), ctypes.byref(w), ctypes.byref(ctr))
    if rc < 0:
        raise EfmError(rc, "efm_fetch_results")
    counters = {f: int(getattr(ctr, f)) for f in COUNTER_FIELDS}
    if not copy:
        return None, counters, rc
    if out is None or out.shape[0] < n.value or out.dtype != np.uint64 or not out.flags.c_contiguous:
        out = np.zeros((n.value, w.value), dtype=np.uint64)
    else:
        out = out[:n.value]
    rc = lib.efm_fetch_results(job, int(idx), out.ctypes.data_as(_P(ctypes.c_uint64)), n.value, ctypes.byref(n),
                               None, None)
    if rc < 0:
        raise EfmError(rc, "efm_fetch_results")
    return out, counters, rc


def efm_job_timing(job, idx):
    """Returns dict(total_ms, expand_ms, expand_launches, expand_bytes, kernel_launches)."""
    t, e, n, b, k = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_int64()
    rc = load_library().efm_job_timing(job, int(idx), ctypes.byref(t), ctypes.byref(e), ctypes.byref(n),
                                       ctypes.byref(b), ctypes.byref(k))
    if rc != 0:
        raise EfmError(rc, "efm_job_timing")
    return dict(total_ms=t.value, expand_ms=e.value, expand_launches=n.value, expand_bytes=b.value,
                kernel_launches=k.value)


def efm_free_job(job):
    if job:
        load_library().efm_free_job(job)


def efm_free_net(net):
    if net:
        load_library().efm_free_net(net)


def efm_sort_supports_noalloc(supports_in_ptr, n_rows, words_per_set, supports_out_ptr, stream=None) -> int:
    """Device pointers in and out (caller-owned); returns the status code."""
    return load_library().efm_sort_supports_noalloc(int(supports_in_ptr), int(n_rows), int(words_per_set),
                                                    int(supports_out_ptr), _stream_handle(stream))


# --- PyTorch caching allocator as the library's device allocator -------------

_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_void_p)
_keep = []


def use_torch_allocator():
    """Route the library's device allocations through torch's caching
    allocator (so the library shares the PyTorch memory pool)."""
    import torch

    dev = torch.cuda.current_device()

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream))
        except Exception:
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = _ALLOC_T(_alloc), _FREE_T(_free)
    _keep[:] = [a, f]
    rc = load_library().efm_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), None)
    if rc != 0:
        raise EfmError(rc, "efm_set_allocator")


# --- learned proposal ---------------------------------------------------------

def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None:
        a = a.reshape(shape)
    return a, a.ctypes.data_as(_P(ctypes.c_float))


def efm_model_create(seed=0, stream=None) -> int:
    m = ctypes.c_void_p()
    rc = load_library().efm_model_create(int(seed), _stream_handle(stream), ctypes.byref(m))
    if rc != 0:
        raise EfmError(rc, "efm_model_create")
    return m.value


def efm_model_params(model, params=None):
    """Read the FP32 parameters (params None) or replace them."""
    if params is None:
        out = np.zeros(EFM_MLP_PARAMS, dtype=np.float32)
        rc = load_library().efm_model_params(model, out.ctypes.data_as(_P(ctypes.c_float)), 0)
        if rc != 0:
            raise EfmError(rc, "efm_model_params")
        return out
    p, pp = _f32(params, (EFM_MLP_PARAMS,))
    rc = load_library().efm_model_params(model, pp, 1)
    if rc != 0:
        raise EfmError(rc, "efm_model_params")
    return p


def efm_model_add_rows(model, x, y):
    x, px = _f32(x, (-1, EFM_MLP_FEATURES))
    y, py = _f32(y, (-1,))
    rc = load_library().efm_model_add_rows(model, px, py, len(y))
    if rc != 0:
        raise EfmError(rc, "efm_model_add_rows")


def efm_model_rows(model):
    n, pos = ctypes.c_int64(), ctypes.c_int64()
    rc = load_library().efm_model_rows(model, ctypes.byref(n), ctypes.byref(pos))
    if rc != 0:
        raise EfmError(rc, "efm_model_rows")
    return n.value, pos.value


def efm_model_clear_rows(model):
    load_library().efm_model_clear_rows(model)


def efm_model_forward(model, x):
    x, px = _f32(x, (-1, EFM_MLP_FEATURES))
    out = np.zeros(len(x), dtype=np.float32)
    rc = load_library().efm_model_forward(model, px, len(x), out.ctypes.data_as(_P(ctypes.c_float)))
    if rc != 0:
        raise EfmError(rc, "efm_model_forward")
    return out


def efm_model_gradient(model, pos_weight=1.0):
    g = np.zeros(EFM_MLP_PARAMS, dtype=np.float32)
    loss = ctypes.c_float()
    rc = load_library().efm_model_gradient(model, float(pos_weight), g.ctypes.data_as(_P(ctypes.c_float)),
                                           ctypes.byref(loss))
    if rc != 0:
        raise EfmError(rc, "efm_model_gradient")
    return g, loss.value


def efm_model_train(model, epochs, batch_tiles=8, lr=1e-3, pos_weight=1.0, seed=0):
    loss = ctypes.c_float()
    rc = load_library().efm_model_train(model, int(epochs), int(batch_tiles), float(lr), float(pos_weight), int(seed),
                                        ctypes.byref(loss))
    if rc != 0:
        raise EfmError(rc, "efm_model_train")
    return loss.value


def efm_model_trace(model, net, targets, max_len, max_secondary, first_k, max_frontier=0, rows_per_level=4096):
    tg, ptg = _arr(targets, np.int32, ctypes.c_int32)
    lim = efm_limits(int(max_len), int(max_secondary), 0, int(max_frontier), int(first_k), EFM_PLAIN)
    rc = load_library().efm_model_trace(model, net, ptg, len(tg), ctypes.byref(lim), int(rows_per_level))
    if rc != 0:
        raise EfmError(rc, "efm_model_trace")


def efm_model_free(model):
    load_library().efm_model_free(model)


def save_model(model, path):
    """Write the model's FP32 parameters (efm_model_params) to a .npy file."""
    np.save(path, efm_model_params(model))


def load_model(path, stream=None):
    """A new model with the parameters of a file written by save_model."""
    p = np.load(path)
    if p.shape != (EFM_MLP_PARAMS,) or p.dtype != np.float32:
        raise ValueError(f"{path}: not a saved proposal model")
    m = efm_model_create(0, stream)
    try:
        efm_model_params(m, p)
    except Exception:
        efm_model_free(m)
        raise
    return m


# --- conveniences ------------------------------------------------------------

class Network:
    """A loaded network (owns the C handle)."""

    def __init__(self, net, stream=None):
        self.src = net
        self.handle = efm_load_network(net.n_met, net.n_rxn, net.row_ptr, net.col_idx, net.coef, net.reversible,
                                       net.external, stream)
        self.n_columns, self.words, self.n_internal = efm_network_shape(self.handle)

    def close(self):
        efm_free_net(self.handle)
        self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def enumerate_targets(network: Network, targets, max_len, max_secondary, max_results=0, max_frontier=0,
                      timing=False, first_k=0, proposal=EFM_PLAIN, model=None, variant=EFM_ADDITIVE):
    """Run efm_find_pathways over `targets` and fetch every target's result.
    Returns a list of (supports, counters[, timing dict])."""
    job, _ = efm_find_pathways(network.handle, list(targets), max_len, max_secondary, max_results, max_frontier,
                               first_k, proposal, model, variant)
    try:
        out = []
        for i in range(len(targets)):
            sup, ctr, _ = efm_fetch_results(job, i)
            if timing:
                out.append((sup, ctr, efm_job_timing(job, i)))
            else:
                out.append((sup, ctr))
        return out
    finally:
        efm_free_job(job)
