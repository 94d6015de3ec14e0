"""Thin Python binding of the C ABI in ``include/wv.h`` (ctypes).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Functions carry the C names; device buffers are torch tensors
(int64 or uint64 storage, contiguous, on the current CUDA device) and the
stream defaults to torch's current stream.  A non-OK status raises
``WvError``.  There is no CPU fallback: if the library cannot be built or
loaded, the first call raises.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build as _build

WV_OK, WV_EINVAL, WV_ENOMEM, WV_ERANGE, WV_ECUDA, WV_ETIMEOUT, WV_ECANCELLED, WV_EBUSY = range(8)
WV_P_MAX = 1 << 37
WV_RESIDUE_INVALID = (1 << 64) - 1
WV_KIND_BERNOULLI, WV_KIND_EULER, WV_KIND_NEAR_B, WV_KIND_NEAR_E = 1, 2, 4, 8

_STATUS = {0: "WV_OK", 1: "WV_EINVAL", 2: "WV_ENOMEM", 3: "WV_ERANGE", 4: "WV_ECUDA",
           5: "WV_ETIMEOUT", 6: "WV_ECANCELLED", 7: "WV_EBUSY"}


class WvError(RuntimeError):
    def __init__(self, status: int, msg: str, count: int | None = None):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status
        self.count = count


class wv_hit(ctypes.Structure):
    _fields_ = [("p", ctypes.c_uint64), ("kind", ctypes.c_uint32), ("pad", ctypes.c_uint32)]


class wv_request(ctypes.Structure):
    _fields_ = [("d_primes", ctypes.c_void_p), ("n", ctypes.c_size_t),
                ("d_out_b", ctypes.c_void_p), ("d_out_e", ctypes.c_void_p)]


class wv_server_config(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_size_t), ("max_active", ctypes.c_uint32),
                ("epoch_terms", ctypes.c_double), ("device", ctypes.c_int),
                ("epoch_form", ctypes.c_int), ("epoch_block", ctypes.c_int),
                ("piece_log2", ctypes.c_int), ("reserved", ctypes.c_int * 4)]


class wv_query_info(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("kind", ctypes.c_int), ("state", ctypes.c_int),
                ("status", ctypes.c_int), ("n_primes", ctypes.c_uint64), ("n_hits", ctypes.c_uint64),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class wv_options(ctypes.Structure):
    _fields_ = [("cong_b", ctypes.c_int), ("cong_e", ctypes.c_int), ("block", ctypes.c_int),
                ("ilp", ctypes.c_int), ("tile_terms", ctypes.c_int), ("max_tiles", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int), ("arith", ctypes.c_int),
                ("check_primes", ctypes.c_int), ("tiling", ctypes.c_int),
                ("uform_min31", ctypes.c_int), ("uform_min64", ctypes.c_int),
                ("reserved", ctypes.c_int * 4)]


_lock = threading.Lock()
_lib = None
_u64, _sz, _vp, _i32 = ctypes.c_uint64, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_int
_pu64, _psz = ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_size_t)

_SIGS = {
    "wv_version": ([], ctypes.c_char_p),
    "wv_last_error": ([], ctypes.c_char_p),
    "wv_is_prime": ([_u64], _i32),
    "wv_sieve": ([_u64, _u64, _vp, _sz, _psz, _vp], _i32),
    "wv_sieve_count": ([_u64, _u64, _pu64, _vp], _i32),
    "wv_bernoulli_pm3": ([_vp, _sz, _vp, _vp], _i32),
    "wv_euler_pm3": ([_vp, _sz, _vp, _vp], _i32),
    "wv_residues_pm3": ([_vp, _sz, _vp, _vp, _vp], _i32),
    "wv_residues_ex": ([_vp, _sz, _vp, _vp, ctypes.POINTER(wv_options), _vp], _i32),
    "wv_residues_pm3_noalloc": ([_vp, _sz, _vp, _vp, _vp], _i32),
    "wv_search": ([_u64, _u64, _vp, _sz, _psz, _vp], _i32),
    "wv_residues_general": ([_vp, _sz, ctypes.c_uint32, ctypes.c_uint32, _vp, _vp, _vp], _i32),
    "wv_general_rows": ([_i32], _i32),
    "wv_general_row": ([_i32, _i32] + [ctypes.POINTER(ctypes.c_uint32)] * 4 +
                       [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_uint32),
                        ctypes.POINTER(ctypes.c_uint32)], _i32),
    "wv_congruence_terms": ([_i32, _i32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_uint64),
                             _i32, ctypes.POINTER(_i32)], _i32),
    "wv_congruence_default": ([_i32], _i32),
    "wv_congruence_for_range": ([_u64, _u64, ctypes.POINTER(_i32), ctypes.POINTER(_i32)], None),
    "wv_histogram": ([_u64, _u64, ctypes.c_uint32, _vp, _vp, _psz, _vp], _i32),
    "wv_search_ex": ([_u64, _u64, _u64, _vp, _sz, _psz, _vp, _vp, _vp, _sz, _psz,
                      ctypes.POINTER(wv_options), _vp], _i32),
    "wv_congruence_count": ([], _i32),
    "wv_congruence_info": ([_i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                            ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_char_p)], _i32),
    "wv_congruence_row": ([_i32, _i32, ctypes.POINTER(ctypes.c_int64)] +
                          [ctypes.POINTER(ctypes.c_uint32)] * 4, _i32),
    "wv_profile_enable": ([_i32], None),
    "wv_profile_reset": ([], None),
    "wv_profile_collect": ([], _i32),
    "wv_profile_kernels": ([], _i32),
    "wv_profile_get": ([_i32, ctypes.POINTER(ctypes.c_char_p), _pu64,
                        ctypes.POINTER(ctypes.c_double)], _i32),
    "wv_profile_launches": ([], _u64),
    "wv_count_terms": ([_pu64, _sz, _i32, _i32, _pu64, _pu64], _i32),
    "wv_batch_create": ([ctypes.c_void_p, _sz, ctypes.POINTER(wv_options), ctypes.POINTER(_vp)], _i32),
    "wv_batch_run": ([_vp, _vp], _i32),
    "wv_batch_info": ([_vp, _psz, _psz, _psz], _i32),
    "wv_batch_groups": ([_vp, _psz], _i32),
    "wv_batch_destroy": ([_vp], _i32),
    "wv_server_create": ([ctypes.POINTER(wv_server_config), ctypes.POINTER(_vp)], _i32),
    "wv_server_submit_range": ([_vp, _u64, _u64, _pu64], _i32),
    "wv_server_submit_prime": ([_vp, _u64, _pu64], _i32),
    "wv_server_wait": ([_vp, _u64, ctypes.c_double, ctypes.POINTER(wv_query_info)], _i32),
    "wv_server_query": ([_vp, _u64, ctypes.POINTER(wv_query_info)], _i32),
    "wv_server_result": ([_vp, _u64, _pu64, _pu64, _pu64, _sz, _psz], _i32),
    "wv_server_release": ([_vp, _u64], _i32),
    "wv_server_stats": ([_vp, _pu64, _pu64, _psz, ctypes.POINTER(ctypes.c_uint32)], _i32),
    "wv_server_destroy": ([_vp], _i32),
}


def lib_path() -> str:
    return _build.LIB


def load():
    """Build (if needed) and load libwv.so; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        lib = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def declared_symbols():
    return sorted(_SIGS)


def _check(st: int, count: int | None = None):
    if st != WV_OK:
        msg = load().wv_last_error().decode()
        raise WvError(st, msg, count)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    import torch
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if t.dtype not in (torch.int64, torch.uint64):
        raise TypeError("expected an int64/uint64 tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _options(opt: dict | None):
    if not opt:
        return None
    o = wv_options()
    o.cong_b = o.cong_e = -1
    for k, v in opt.items():
        setattr(o, k, int(v))
    return ctypes.byref(o)


# ------------------------------------------------------------------ entry points
def wv_version() -> str:
    return load().wv_version().decode()


def wv_last_error() -> str:
    return load().wv_last_error().decode()


def wv_is_prime(n: int) -> int:
    """1 if n is prime, 0 if not, -1 for n >= 2^37 (host only)."""
    return load().wv_is_prime(n)


def wv_sieve(lo: int, hi: int, d_out, stream=None) -> int:
    """Primes of [lo, hi) into d_out (device); returns the count."""
    n = ctypes.c_size_t(0)
    cap = 0 if d_out is None else d_out.numel()
    st = load().wv_sieve(lo, hi, _ptr(d_out) if cap else None, cap, ctypes.byref(n), _stream(stream))
    _check(st, n.value)
    return n.value


def wv_sieve_count(lo: int, hi: int, stream=None) -> int:
    c = ctypes.c_uint64(0)
    _check(load().wv_sieve_count(lo, hi, ctypes.byref(c), _stream(stream)))
    return c.value


def wv_bernoulli_pm3(d_primes, d_out, stream=None) -> None:
    _check(load().wv_bernoulli_pm3(_ptr(d_primes), d_primes.numel(), _ptr(d_out), _stream(stream)))


def wv_euler_pm3(d_primes, d_out, stream=None) -> None:
    _check(load().wv_euler_pm3(_ptr(d_primes), d_primes.numel(), _ptr(d_out), _stream(stream)))


def wv_residues_pm3(d_primes, d_out_b, d_out_e, stream=None) -> None:
    _check(load().wv_residues_pm3(_ptr(d_primes), d_primes.numel(), _ptr(d_out_b), _ptr(d_out_e),
                                  _stream(stream)))


def wv_residues_pm3_noalloc(d_primes, d_out_b, d_out_e, stream=None) -> None:
    """wv_residues_pm3 without any allocation (at most 1024 primes per call);
    for callers that cannot allocate device memory during a call."""
    _check(load().wv_residues_pm3_noalloc(_ptr(d_primes), d_primes.numel(), _ptr(d_out_b),
                                          _ptr(d_out_e), _stream(stream)))


def wv_residues_ex(d_primes, d_out_b, d_out_e, options: dict | None = None, stream=None) -> None:
    _check(load().wv_residues_ex(_ptr(d_primes), d_primes.numel(), _ptr(d_out_b), _ptr(d_out_e),
                                 _options(options), _stream(stream)))


def wv_search(lo: int, hi: int, d_hits, stream=None) -> int:
    """Hits of [lo, hi) into d_hits (an int64 tensor of shape (cap, 2) holding
    wv_hit records); returns the hit count."""
    n = ctypes.c_size_t(0)
    cap = 0 if d_hits is None else d_hits.shape[0]
    st = load().wv_search(lo, hi, _ptr(d_hits) if cap else None, cap, ctypes.byref(n), _stream(stream))
    _check(st, n.value)
    return n.value


def wv_search_ex(lo: int, hi: int, near: int, d_hits, d_primes=None, d_res_b=None, d_res_e=None,
                 options: dict | None = None, stream=None):
    """Returns (n_hits, n_primes)."""
    nh, npr = ctypes.c_size_t(0), ctypes.c_size_t(0)
    cap = 0 if d_hits is None else d_hits.shape[0]
    caps = [t.numel() for t in (d_primes, d_res_b, d_res_e) if t is not None]
    cap_p = min(caps) if caps else 0
    st = load().wv_search_ex(lo, hi, near, _ptr(d_hits) if cap else None, cap, ctypes.byref(nh),
                             _ptr(d_primes), _ptr(d_res_b), _ptr(d_res_e), cap_p,
                             ctypes.byref(npr), _options(options), _stream(stream))
    _check(st, nh.value)
    return nh.value, npr.value


def wv_residues_general(d_primes, e_b: int, e_e: int, d_out_b=None, d_out_e=None, stream=None):
    """B_{p-e_b} mod p and E_{p-1-e_e} mod p (an exponent 0 skips its kind)."""
    n = d_primes.numel()
    _check(load().wv_residues_general(_ptr(d_primes), n, e_b, e_e, _ptr(d_out_b), _ptr(d_out_e),
                                      _stream(stream)))


def wv_general_rows(kind: int) -> int:
    return load().wv_general_rows(kind)


def wv_general_row(kind: int, row: int):
    """((xn, xd, yn, yd), [(c_i, d_i)...], lhs (a, b, c)) of a general-index row."""
    v = [ctypes.c_uint32() for _ in range(4)]
    c, d, l = (ctypes.c_int32 * 3)(), (ctypes.c_uint32 * 3)(), (ctypes.c_uint32 * 3)()
    _check(load().wv_general_row(kind, row, *[ctypes.byref(x) for x in v], c, d, l))
    return tuple(x.value for x in v), [(c[i], d[i]) for i in range(3) if c[i]], tuple(l)


def wv_histogram(lo: int, hi: int, d_hist_b=None, d_hist_e=None, stream=None) -> int:
    """Adds the bin counts of <B_{p-3}>_p / p and <E_{p-3}>_p / p for the primes
    of [lo, hi) to the given int64 device tensors (bins = their length);
    returns the number of primes."""
    ts = [t for t in (d_hist_b, d_hist_e) if t is not None]
    bins = ts[0].numel() if ts else 0
    if any(t.numel() != bins for t in ts):
        raise ValueError("histogram tensors differ in length")
    npr = ctypes.c_size_t(0)
    _check(load().wv_histogram(lo, hi, bins, _ptr(d_hist_b), _ptr(d_hist_e), ctypes.byref(npr),
                               _stream(stream)))
    return npr.value


def wv_congruence_count() -> int:
    return load().wv_congruence_count()


def wv_congruence_info(cid: int):
    """(name, kind, n_rows, lhs) -- kind 0 = B_{p-3}, 1 = E_{p-3}."""
    k, n, l, nm = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_char_p()
    _check(load().wv_congruence_info(cid, ctypes.byref(k), ctypes.byref(n), ctypes.byref(l),
                                     ctypes.byref(nm)))
    return nm.value.decode(), k.value, n.value, l.value


def wv_congruence_default(kind: int) -> int:
    return load().wv_congruence_default(kind)


def wv_congruence_for_range(lo: int, hi: int):
    """(B id, E id) the range-aware calls use for primes of [lo, hi)."""
    b, e = _i32(), _i32()
    load().wv_congruence_for_range(lo, hi, ctypes.byref(b), ctypes.byref(e))
    return b.value, e.value


def wv_congruence_terms(cid: int, row: int):
    """[(c_k, d_k)]: the row's coefficient is sum_k c_k d_k^t."""
    c, d, n = (ctypes.c_int64 * 64)(), (ctypes.c_uint64 * 64)(), _i32()
    _check(load().wv_congruence_terms(cid, row, c, d, 64, ctypes.byref(n)))
    return [(c[k], d[k]) for k in range(n.value)]


def wv_congruence_row(cid: int, row: int):
    """(coef, xn, xd, yn, yd)."""
    c = ctypes.c_int64()
    v = [ctypes.c_uint32() for _ in range(4)]
    _check(load().wv_congruence_row(cid, row, ctypes.byref(c), *[ctypes.byref(x) for x in v]))
    return (c.value,) + tuple(x.value for x in v)


def wv_count_terms(primes, cong_b: int = -1, cong_e: int = -1):
    """(terms_b, terms_e) for a host list of primes; -2 skips a kind."""
    a = np.ascontiguousarray(np.asarray(primes, dtype=np.uint64))
    tb, te = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().wv_count_terms(a.ctypes.data_as(_pu64), a.size, cong_b, cong_e,
                                 ctypes.byref(tb), ctypes.byref(te)))
    return tb.value, te.value


def wv_profile_enable(on: bool = True) -> None:
    load().wv_profile_enable(1 if on else 0)


def wv_profile_reset() -> None:
    load().wv_profile_reset()


def wv_profile_collect() -> dict:
    """Fold pending events; returns {kernel: (launches, total_ms)}."""
    lib = load()
    _check(lib.wv_profile_collect())
    out = {}
    for i in range(lib.wv_profile_kernels()):
        nm, la, ms = ctypes.c_char_p(), ctypes.c_uint64(), ctypes.c_double()
        _check(lib.wv_profile_get(i, ctypes.byref(nm), ctypes.byref(la), ctypes.byref(ms)))
        out[nm.value.decode()] = (la.value, ms.value)
    return out


def wv_profile_launches() -> int:
    return int(load().wv_profile_launches())


def wv_profile_kernels() -> int:
    return int(load().wv_profile_kernels())


def wv_profile_get(idx: int):
    """(name, launches, total_ms) of profiled kernel `idx`."""
    nm, la, ms = ctypes.c_char_p(), ctypes.c_uint64(), ctypes.c_double()
    _check(load().wv_profile_get(idx, ctypes.byref(nm), ctypes.byref(la), ctypes.byref(ms)))
    return nm.value.decode(), la.value, ms.value


class Batch:
    """Handle of a captured batch; keeps the request tensors alive."""

    def __init__(self, handle, tensors):
        self.handle = handle
        self._tensors = tensors

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.wv_batch_destroy(self.handle)
            self.handle = None


def wv_batch_create(requests, options: dict | None = None) -> Batch:
    """requests: list of (d_primes, d_out_b, d_out_e) device tensors (outputs may be None)."""
    arr = (wv_request * len(requests))()
    keep = []
    for i, (dp, ob, oe) in enumerate(requests):
        arr[i].d_primes = _ptr(dp).value if dp.numel() else None
        arr[i].n = dp.numel()
        arr[i].d_out_b = _ptr(ob).value if ob is not None else None
        arr[i].d_out_e = _ptr(oe).value if oe is not None else None
        keep += [dp, ob, oe]
    h = ctypes.c_void_p()
    _check(load().wv_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(requests), _options(options),
                                  ctypes.byref(h)))
    return Batch(h, keep)


def wv_batch_run(batch: Batch, stream=None) -> None:
    _check(load().wv_batch_run(batch.handle, _stream(stream)))


def wv_batch_info(batch: Batch):
    """(requests, primes, graph nodes)."""
    a, b, c = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(load().wv_batch_info(batch.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def wv_batch_groups(batch: Batch) -> int:
    """Number of congruence groups of the batch."""
    a = ctypes.c_size_t()
    _check(load().wv_batch_groups(batch.handle, ctypes.byref(a)))
    return a.value


def wv_batch_destroy(batch: Batch) -> None:
    if batch.handle:
        _check(load().wv_batch_destroy(batch.handle))
        batch.handle = None



# ------------------------------------------------------------------ serving
def _info(i: wv_query_info) -> dict:
    return {"id": i.id, "kind": ("range", "prime")[i.kind], "state": i.state, "status": i.status,
            "n_primes": i.n_primes, "n_hits": i.n_hits, "t_submit": i.t_submit,
            "t_admit": i.t_admit, "t_done": i.t_done}


def wv_server_create(mem_budget: int = 0, max_active: int = 0, epoch_terms: float = 0.0,
                     device: int = -1, epoch_form: int = 0, epoch_block: int = 0,
                     piece_log2: int = 0):
    cfg = wv_server_config()
    cfg.mem_budget, cfg.max_active, cfg.epoch_terms, cfg.device = mem_budget, max_active, epoch_terms, device
    cfg.epoch_form, cfg.epoch_block, cfg.piece_log2 = epoch_form, epoch_block, piece_log2
    h = ctypes.c_void_p()
    _check(load().wv_server_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def wv_server_submit_range(server, lo: int, hi: int) -> int:
    i = ctypes.c_uint64()
    _check(load().wv_server_submit_range(server, lo, hi, ctypes.byref(i)))
    return i.value


def wv_server_submit_prime(server, p: int) -> int:
    i = ctypes.c_uint64()
    _check(load().wv_server_submit_prime(server, p, ctypes.byref(i)))
    return i.value


def wv_server_wait(server, qid: int, timeout_s: float = -1.0) -> dict:
    info = wv_query_info()
    _check(load().wv_server_wait(server, qid, timeout_s, ctypes.byref(info)))
    return _info(info)


def wv_server_query(server, qid: int) -> dict:
    info = wv_query_info()
    _check(load().wv_server_query(server, qid, ctypes.byref(info)))
    return _info(info)


def wv_server_result(server, qid: int):
    """(primes, B residues, E residues) of a finished query as numpy uint64 arrays."""
    n = ctypes.c_size_t()
    lib = load()
    st = lib.wv_server_result(server, qid, None, None, None, 0, ctypes.byref(n))
    if st not in (WV_OK, WV_ERANGE):
        _check(st)
    out = [np.zeros(max(n.value, 1), dtype=np.uint64) for _ in range(3)]
    ptrs = [a.ctypes.data_as(_pu64) for a in out]
    _check(lib.wv_server_result(server, qid, *ptrs, n.value, ctypes.byref(n)))
    return tuple(a[:n.value] for a in out)


def wv_server_release(server, qid: int) -> None:
    _check(load().wv_server_release(server, qid))


def wv_server_stats(server) -> dict:
    e, t, b, pk = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_size_t(), ctypes.c_uint32()
    _check(load().wv_server_stats(server, ctypes.byref(e), ctypes.byref(t), ctypes.byref(b),
                                  ctypes.byref(pk)))
    return {"epochs": e.value, "tiles": t.value, "bytes_in_use": b.value, "peak_active": pk.value}


def wv_server_destroy(server) -> None:
    _check(load().wv_server_destroy(server))
