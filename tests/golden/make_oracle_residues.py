"""Write stored oracle residues for the workloads the CPU oracle cannot redo
inside a test run.

Every value written here comes from ``oracle/`` alone: the primes of a window
from the oracle's plain sieve, B_{p-3} mod p by the Stafford-Vandiver
congruence at k = (p-3)/2 (Sec. 2, eqn 2.4, i.e. eqn 3.2) and E_{p-3} mod p
by Glaisher's congruence (Sec. 4, eqn 4.1, sign (-1)^k), both summed with the
plain accumulation of eqn 3.12 in 128-bit remainders.  The seeded prime
lists come from ``paper_2101_11157_gb300.workloads``, the input-generator
module that holds none of the residue arithmetic.  Nothing here touches the
CUDA library.

Targets (files under ``tests/golden/``):

* ``p1e9_window`` -> ``p1e9_window_residues.txt``: every prime of
  [1062200000, 1062300000) (4907 primes; about 12 core-seconds each);
* ``top_subset`` -> ``top_window_subset_residues.txt``: the 8 primes of
  [1e11 - 1e4, 1e11) drawn by ``default_rng(5)`` (about an hour each);
* ``batch_sample`` -> ``batch_seed7_sample_residues.txt``: of each of the 64
  seed-7 requests (p in [1e5, 1e10)), its smallest prime and one drawn by
  ``default_rng(1)``;
* ``serve_sample`` -> ``serve_sample_residues.txt``: primes of the serving
  test's queries that are too large for the oracle inside a test: six drawn
  by ``default_rng(2)`` from each range above 1e8, and the single primes.

Run (resumable: finished primes are kept in ``<file>.partial``)::

    python tests/golden/make_oracle_residues.py --target batch_sample --threads 8
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2101_11157_gb300 import workloads as W  # noqa: E402

HEADER = """# B_{p-3} mod p and E_{p-3} mod p, each the canonical residue in [0, p).
# Definitions: Sec. 1 (Bernoulli numbers from z/(e^z - 1); Euler numbers from sec z).
# Computed by the CPU oracle only: B by the Stafford-Vandiver congruence (Sec. 2, eqn 2.4
# at k = (p-3)/2, i.e. eqn 3.2), E by Glaisher's congruence (Sec. 4, eqn 4.1 with the
# sign (-1)^k), each sum accumulated as in eqn 3.12 with 128-bit remainders.
# Written by: python tests/golden/make_oracle_residues.py --target {target}
# Workload: {what}
# columns: p B E
"""

# The serving test's queries whose primes are too large for the oracle inside
# a test run (tests/test_gpu_serve.py holds the same list).
SERVE_RANGES = [(2 * 10**9, 2 * 10**9 + 30000), (999_999_000, 1_000_001_000),
                (2 * 10**9 + 30000, 2 * 10**9 + 60000)]
SERVE_PRIMES = [1062232319, 2**30 + 3]


def _primes_p1e9():
    return O.sieve(*W.P1E9_WINDOW), "every prime of [1062200000, 1062300000)"


def _primes_top():
    pr = O.sieve(*W.TOP_WINDOW)
    rng = np.random.default_rng(5)
    idx = rng.choice(pr.size, size=8, replace=False)
    return (np.sort(pr[idx]),
            "the 8 primes of [1e11 - 1e4, 1e11) at default_rng(5).choice(391, 8, replace=False)")


def _primes_batch():
    reqs = W.batch_requests(seed=7)
    rng = np.random.default_rng(1)
    out = set()
    for r in reqs:
        out.add(int(r[0]))
        out.add(int(r[int(rng.integers(r.size))]))
    return (np.array(sorted(out), dtype=np.uint64),
            "of each of the 64 requests of batch_requests(seed=7), its smallest prime and "
            "r[default_rng(1).integers(len(r))], requests in order")


def _primes_serve():
    rng = np.random.default_rng(2)
    out = set(int(p) for p in SERVE_PRIMES)
    for lo, hi in SERVE_RANGES:
        pr = O.sieve(lo, hi)
        out.update(int(v) for v in pr[rng.choice(pr.size, size=6, replace=False)])
    return (np.array(sorted(out), dtype=np.uint64),
            "six primes drawn by default_rng(2) from each of the ranges "
            + ", ".join(f"[{a}, {b})" for a, b in SERVE_RANGES)
            + "; the single primes " + ", ".join(str(p) for p in SERVE_PRIMES))


TARGETS = {
    "p1e9_window": ("p1e9_window_residues.txt", _primes_p1e9),
    "top_subset": ("top_window_subset_residues.txt", _primes_top),
    "batch_sample": ("batch_seed7_sample_residues.txt", _primes_batch),
    "serve_sample": ("serve_sample_residues.txt", _primes_serve),
}


def _read_rows(path):
    rows = {}
    if os.path.exists(path):
        with open(path) as f:
            for line in f:
                line = line.split("#", 1)[0].split()
                if len(line) == 3:
                    rows[int(line[0])] = (int(line[1]), int(line[2]))
    return rows


def run(target: str, threads: int, chunk: int) -> str:
    fname, gen = TARGETS[target]
    primes, what = gen()
    path = os.path.join(HERE, fname)
    partial = path + ".partial"
    done = _read_rows(partial)
    todo = [int(p) for p in primes if int(p) not in done]
    # largest first, so the longest primes do not form the tail
    todo.sort(reverse=True)
    print(f"{target}: {primes.size} primes, {len(done)} already done", flush=True)
    t0 = time.time()
    with open(partial, "a") as f:
        for i in range(0, len(todo), chunk):
            part = np.array(todo[i:i + chunk], dtype=np.uint64)
            b, e = O.residues(part, threads=threads)
            for p, rb, re in zip(part, b, e):
                f.write(f"{int(p)} {int(rb)} {int(re)}\n")
                done[int(p)] = (int(rb), int(re))
            f.flush()
            print(f"  {len(done)}/{primes.size} after {time.time() - t0:.0f} s", flush=True)
    with open(path + ".tmp", "w") as f:
        f.write(HEADER.replace("{target}", target).replace("{what}", what))
        for p in sorted(int(v) for v in primes):
            rb, re = done[p]
            f.write(f"{p} {rb} {re}\n")
    os.replace(path + ".tmp", path)
    os.remove(partial)
    return path


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--target", choices=sorted(TARGETS), action="append", required=True)
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--chunk", type=int, default=0, help="primes per oracle call (default 4 x threads)")
    a = ap.parse_args()
    for t in a.target:
        print(run(t, a.threads, a.chunk or 4 * a.threads), flush=True)


if __name__ == "__main__":
    main()
