"""The allocation-free entry point, wv_residues_pm3_noalloc.

It exists for callers that cannot allocate device memory while they run: a
host whose device memory is all handed to its own pool allocator, or a
real-time loop that cannot pay for the device synchronisation cudaMalloc and
cudaFree bring.  It must give exactly the residues of wv_residues_pm3.  This
file is named so that pytest collects it last; it also passes on its own in a
fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2101_11157_gb300 import api, wv  # noqa: E402


def _c_call(name, d_primes, out_b, out_e):
    lib = wv.load()
    fn = getattr(lib, name)
    st = fn(ctypes.c_void_p(d_primes.data_ptr()), d_primes.numel(),
            ctypes.c_void_p(out_b.data_ptr()), ctypes.c_void_p(out_e.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == wv.WV_OK, lib.wv_last_error().decode()


def _both(d_primes):
    """(reference residues via wv_residues_pm3, no-alloc residues), as numpy."""
    rb, re = torch.empty_like(d_primes), torch.empty_like(d_primes)
    nb, ne = torch.full_like(d_primes, -7), torch.full_like(d_primes, -7)
    _c_call("wv_residues_pm3", d_primes, rb, re)
    _c_call("wv_residues_pm3_noalloc", d_primes, nb, ne)
    torch.cuda.synchronize()
    return [api.to_u64(x) for x in (rb, re, nb, ne)]


def test_noalloc_matches_the_allocating_entry_point_twice():
    # first call: primes on both arithmetic paths (below and above 2^30) and
    # the small special primes; second call: a different, shorter list, so a
    # result left over from the first call would show up as a mismatch
    first = np.concatenate([
        np.array([5, 7, 11, 13, 149, 241, 16843], dtype=np.uint64),
        api.to_u64(api.sieve(1_062_200_000, 1_062_204_000)),
        api.to_u64(api.sieve(2**30, 2**30 + 3000)),
    ])
    second = api.to_u64(api.sieve(10**7, 10**7 + 3000))
    assert first.size <= 1024 and second.size <= 1024
    for primes in (first, second):
        d = torch.from_numpy(primes.view(np.int64)).cuda()
        rb, re, nb, ne = _both(d)
        assert np.array_equal(nb, rb)
        assert np.array_equal(ne, re)
    # the known zeros among the first list
    d = torch.from_numpy(first[:7].view(np.int64)).cuda()
    rb, re, nb, ne = _both(d)
    assert nb[6] == 0 and ne[4] == 0 and ne[5] == 0


def test_noalloc_rejects_more_than_its_limit():
    d = torch.full((1025,), 1_000_003, dtype=torch.int64, device="cuda")
    out = torch.empty_like(d)
    lib = wv.load()
    st = lib.wv_residues_pm3_noalloc(ctypes.c_void_p(d.data_ptr()), d.numel(),
                                     ctypes.c_void_p(out.data_ptr()), None, None)
    assert st == wv.WV_ERANGE
    assert "1024" in lib.wv_last_error().decode()


_FRESH = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, {root!r})
from paper_2101_11157_gb300 import wv
primes = np.array({primes!r}, dtype=np.uint64)
s = torch.cuda.Stream()  # torch creates its streams with cudaStreamNonBlocking
with torch.cuda.stream(s):
    d = torch.from_numpy(primes.view(np.int64)).cuda()
    ob, oe = torch.full_like(d, -7), torch.full_like(d, -7)
    wv.wv_residues_pm3_noalloc(d, ob, oe, s) if {noalloc!r} else wv.wv_residues_pm3(d, ob, oe, s)
s.synchronize()
print(json.dumps([ob.cpu().numpy().view(np.uint64).tolist(), oe.cpu().numpy().view(np.uint64).tolist()]))
"""


@pytest.mark.parametrize("noalloc", [True, False])
def test_first_call_on_a_non_blocking_stream_in_a_fresh_process(noalloc, orc):
    # The first call of a process uploads the congruence rows; a caller's
    # non-blocking stream is not ordered after that upload by itself.  The
    # residues must still be the oracle's.
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    primes = [int(p) for p in orc.sieve(1_000_000, 1_001_000)] + [16843, 1_062_232_319, 2**30 + 3]
    code = _FRESH.format(root=root, primes=primes, noalloc=noalloc)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    gb, ge = json.loads(out.stdout.strip().splitlines()[-1])
    small = [p for p in primes if p < 10**8]
    rb, re = orc.residues(small)
    assert gb[:len(small)] == [int(x) for x in rb] and ge[:len(small)] == [int(x) for x in re]
    assert gb[small.index(16843)] == 0  # the Wolstenholme prime
    # the two large primes against residues stored by the oracle
    from conftest import read_golden
    gold = {int(p): (int(b), int(e)) for p, b, e in read_golden("serve_sample_residues.txt")}
    for i in (len(small), len(small) + 1):
        assert (gb[i], ge[i]) == gold[primes[i]], primes[i]
    assert ge[len(small)] == 0  # 1062232319, a Vandiver prime
