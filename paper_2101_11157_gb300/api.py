"""Allocating convenience wrappers over the thin binding (``wv.py``).

Device buffers come from PyTorch; all computation runs in libwv.  The
``*_host`` helpers take and return host arrays: they copy the inputs from
pinned host memory to the device, run the library call, and copy the results
back, which is the end-to-end path a host caller uses.
"""
from __future__ import annotations

import numpy as np

from . import wv


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required (libwv has no CPU path)")
    return torch


def sieve(lo: int, hi: int, stream=None):
    """Device int64 tensor of the primes in [lo, hi)."""
    torch = _torch()
    n = wv.wv_sieve_count(lo, hi, stream) if hi > lo else 0
    out = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
    if n:
        wv.wv_sieve(lo, hi, out, stream)
    return out[:n]


def residues(d_primes, want_b: bool = True, want_e: bool = True, options=None, stream=None):
    """(B residues, E residues) as device int64 tensors (None for a skipped kind)."""
    torch = _torch()
    rb = torch.empty_like(d_primes) if want_b else None
    re = torch.empty_like(d_primes) if want_e else None
    if d_primes.numel():
        wv.wv_residues_ex(d_primes, rb, re, options, stream)
    return rb, re


def to_u64(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def residues_host(primes, options=None, stream=None):
    """Host primes -> host (B, E) residues (numpy uint64) through pinned buffers."""
    torch = _torch()
    a = np.ascontiguousarray(np.asarray(primes, dtype=np.uint64))
    h_in = torch.from_numpy(a.view(np.int64)).pin_memory()
    d_in = h_in.to("cuda", non_blocking=True)
    rb, re = residues(d_in, options=options, stream=stream)
    h_b = torch.empty(a.size, dtype=torch.int64, pin_memory=True)
    h_e = torch.empty(a.size, dtype=torch.int64, pin_memory=True)
    h_b.copy_(rb, non_blocking=True)
    h_e.copy_(re, non_blocking=True)
    torch.cuda.current_stream().synchronize()
    return h_b.numpy().view(np.uint64), h_e.numpy().view(np.uint64)


def search(lo: int, hi: int, near: int = 0, with_residues: bool = False, cap: int = 4096,
           options=None, stream=None):
    """Hits in [lo, hi) as a list of (p, kind); with_residues also returns the
    device tensors (primes, B residues, E residues) of every prime in range."""
    torch = _torch()
    hits = torch.empty((cap, 2), dtype=torch.int64, device="cuda")
    if with_residues:
        n = wv.wv_sieve_count(max(lo, 5), hi, stream) if hi > max(lo, 5) else 0
        pr = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
        rb, re = torch.empty_like(pr), torch.empty_like(pr)
    else:
        pr = rb = re = None
    nh, npr = wv.wv_search_ex(lo, hi, near, hits, pr, rb, re, options, stream)
    h = hits[:nh].cpu().numpy()
    out = [(int(np.uint64(r[0])), int(r[1]) & 0xFFFFFFFF) for r in h]
    if with_residues:
        return out, pr[:npr], rb[:npr], re[:npr]
    return out


def symmetric(r: int, p: int) -> int:
    """<r>_p in (-p/2, p/2]."""
    r %= p
    return r - p if r > p // 2 else r
