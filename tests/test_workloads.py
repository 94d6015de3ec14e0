"""The seeded input generators: determinism and the stated distributions."""
import numpy as np

from paper_2101_11157_gb300 import workloads as W


def test_is_prime_small():
    brute = [n for n in range(200) if n > 1 and all(n % d for d in range(2, int(n ** 0.5) + 1))]
    assert [n for n in range(200) if W.is_prime(n)] == brute
    assert W.is_prime(2**31 - 1) and not W.is_prime(2**32 + 1)
    assert W.next_prime(10**9) == 1000000007


def test_batch_requests_deterministic_and_in_range():
    a = W.batch_requests(seed=7, k=6)
    b = W.batch_requests(seed=7, k=6)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    for r in a:
        assert 1 <= r.size <= 4096
        assert np.all(np.diff(r.astype(np.int64)) > 0)
        assert r.min() >= 1e5 and r.max() < 1e10
        assert all(W.is_prime(int(v)) for v in r[:20])


def test_serving_stream_shape():
    s = W.serving_stream(seed=11, n=40)
    assert s == W.serving_stream(seed=11, n=40)
    ts = [q["t"] for q in s]
    assert all(t2 > t1 for t1, t2 in zip(ts, ts[1:]))
    for q in s:
        if q["kind"] == "range":
            assert 1e6 <= q["lo"] <= 1e10 and 1e3 <= q["hi"] - q["lo"] <= 1e6
        else:
            assert W.is_prime(q["p"])


def test_seeded_subset():
    ps = W.primes_in(1000, 2000)
    s = W.seeded_subset(ps, 8, seed=3, must_include=[1009])
    assert 1009 in s and s.size in (8, 9)
    assert np.array_equal(s, W.seeded_subset(ps, 8, seed=3, must_include=[1009]))
