"""Autotuner for the residue launch shape.

Times the accumulation kernels (CUDA events on the launching stream, through
the library's profiler) for a grid of ``wv_options`` on a given set of primes,
checks that every shape returns bit-identical residues, and records the
fastest shape per GPU and p-bucket (floor(log2 p_max)) in a JSON cache.
``tune_batch`` does the same for a whole batch (the graph-captured launch
sequence of ``wv_batch_create``) and caches its choice per GPU and workload.

    python -m paper_2101_11157_gb300.tune --lo 1062200000 --hi 1062300000 --grid arith
    python -m paper_2101_11157_gb300.tune --lo 1062200000 --hi 1062300000 --grid shape --save
    python -m paper_2101_11157_gb300.tune --grid alu --range-congruences
"""
from __future__ import annotations

import argparse
import itertools
import json
import math
import os

import numpy as np

from . import build as _build
from . import wv

CACHE = os.path.join(_build.OUT, "tune_cache.json")

GRIDS = {
    # the hot-loop formulations (wv_options.arith) at the default shape
    "arith": [{"arith": a, "ilp": i} for a, i in itertools.product((1, 2, 4, 9), (1, 2))],
    # launch shapes for the default formulation
    "shape": [{"ilp": i, "tile_terms": t, "max_tiles": m}
              for i, (t, m) in itertools.product((1, 2), ((1 << 18, 16), (1 << 20, 8), (1 << 22, 4)))],
    # the grouped 64-bit forms (2^30 <= p < 2^37): group sizes, shrink interval, register budget
    "m64": [{"arith": a} for a in (9, *range(12, 19), 21)],
    # the 64-bit default with its table additions as PTX carry chains (all, or a share in
    # three-input form on the integer ALU)
    "m64cc": [{"arith": a} for a in (9, *range(32, 37))],
    # the 64-bit default (four-step shrink of its tables) against the earlier shrink (37)
    "m64shrink": [{"arith": a} for a in (9, 37)],
    # the 64-bit default (rolled per-chain set-up) against the unrolled set-up (38)
    "m64setup": [{"arith": a} for a in (9, 38)],
    # the paper's own arithmetic (eqn 3.15, double-precision quotients) against the default
    "paper": [{"arith": 9}, {"arith": 23}],
    # the 32-bit grouped form 9 with 0 / 4 / 6 / all of its table additions ALU-only (9: 4 and 2)
    "alu": [{"arith": a, "ilp": i} for a, i in itertools.product((9, 25, 26, 27, 28), (2, 1))],
    # group sizes of the 32-bit form: 9 (2 cubes / 3 squares) against 3 cubes, 4 squares, both (31,
    # the default)
    "groups": [{"arith": a, "ilp": i} for a, i in itertools.product((9, 29, 30, 31), (2, 1))],
    # groups of 4 cubes / 5 squares (39) against the default 31
    "groups2": [{"arith": a, "ilp": 2} for a in (31, 39)],
    # resident blocks per SM (persistent grid) for the 32-bit forms 9 and 26
    "occ": [{"arith": a, "ilp": i, "blocks_per_sm": b}
            for a, i, b in itertools.product((9, 26), (2, 1), (3, 4, 5, 6))],
    "block": [{"block": b} for b in (32, 64, 128, 256)],
    "default": [{}],
}


def _time(d, rb, re, opt, reps):
    import torch
    wv.wv_residues_ex(d, rb, re, opt or None)
    torch.cuda.synchronize()
    wv.wv_profile_reset()
    wv.wv_profile_enable(True)
    for _ in range(reps):
        wv.wv_residues_ex(d, rb, re, opt or None)
    torch.cuda.synchronize()
    prof = wv.wv_profile_collect()
    wv.wv_profile_enable(False)
    ms = sum(v[1] for k, v in prof.items() if k.startswith("accumulate")) / reps
    return ms


def sweep(primes, grid, reps: int = 2):
    """Yield dicts {options, acc_ms, terms_per_clk_sm, identical} for each shape."""
    import torch
    grid = list(grid)
    d = torch.from_numpy(np.asarray(primes, dtype=np.uint64).view(np.int64)).cuda()
    rb, re = torch.empty_like(d), torch.empty_like(d)
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    cong = next(((o.get("cong_b", -1), o.get("cong_e", -1)) for o in grid), (-1, -1))
    tb, te = wv.wv_count_terms(np.asarray(primes, dtype=np.uint64), *cong)
    ref = None
    for opt in grid:
        ms = _time(d, rb, re, opt, reps)
        out = (rb.cpu().numpy().copy(), re.cpu().numpy().copy())
        if ref is None:
            ref = out
        same = bool(np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1]))
        # SM clock: the device's maximum (the bench records the clocks it saw)
        clk = props.clock_rate * 1e3 if hasattr(props, "clock_rate") else 2.07e9
        tpc = (tb + te) / (ms / 1e3) / props.multi_processor_count / clk if ms else 0.0
        yield {"options": opt, "acc_ms": round(ms, 3), "terms_per_clk_sm": round(tpc, 3),
               "identical": same}


# launch shapes tried for a batch (one graph-captured launch sequence over many requests)
BATCH_GRID = [{}, {"block": 32}, {"tile_terms": 1 << 19, "max_tiles": 32},
              {"block": 32, "tile_terms": 1 << 19, "max_tiles": 32},
              {"tile_terms": 1 << 21, "max_tiles": 8}, {"ilp": 1}]


def tune_batch(reqs, grid=None, reps: int = 1, key: str | None = None, path: str = CACHE):
    """Choose the launch shape of a batch by timing it.

    reqs: list of (d_primes, d_out_b, d_out_e) device tensors, as for
    wv.wv_batch_create.  Each option set in `grid` is captured into its own
    batch, replayed once untimed and `reps` times under CUDA events; every
    shape must give bit-identical residues.  Returns (best options, table).
    With `key`, the choice is cached per GPU under that key and reused."""
    import torch
    name = torch.cuda.get_device_name()
    if key:
        hit = load_cache(path).get(name, {}).get("batch:" + key)
        if hit is not None:
            return hit, []
    grid = BATCH_GRID if grid is None else grid
    stream = torch.cuda.current_stream()
    table, ref = [], None
    for opt in grid:
        b = wv.wv_batch_create(reqs, opt or None)
        try:
            wv.wv_batch_run(b, stream)
            torch.cuda.synchronize()
            ms = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                wv.wv_batch_run(b, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
        finally:
            wv.wv_batch_destroy(b)
        out = [(rb.clone(), re.clone()) for _, rb, re in reqs]
        if ref is None:
            ref = out
        same = all(torch.equal(a, c) and torch.equal(b_, d) for (a, b_), (c, d) in zip(out, ref))
        table.append({"options": opt, "ms": min(ms), "identical": bool(same)})
    bad = [r for r in table if not r["identical"]]
    if bad:
        raise RuntimeError(f"batch shapes disagree: {bad}")
    best = min(table, key=lambda r: r["ms"])["options"]
    if key:
        cache = load_cache(path)
        cache.setdefault(name, {})["batch:" + key] = best
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    return best, table


def bucket(p_max: int) -> int:
    return int(math.floor(math.log2(max(int(p_max), 2))))


def load_cache(path: str = CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def best_options(primes, path: str = CACHE):
    """Cached best options for this GPU and the largest prime's bucket (or None)."""
    try:
        import torch
        name = torch.cuda.get_device_name()
    except Exception:
        return None
    cache = load_cache(path)
    if len(primes) == 0:
        return None
    b = str(bucket(int(np.max(np.asarray(primes, dtype=np.uint64)))))
    return cache.get(name, {}).get(b)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--lo", type=int, default=1_062_200_000)
    ap.add_argument("--hi", type=int, default=1_062_300_000)
    ap.add_argument("--grid", default="shape", choices=sorted(GRIDS))
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--save", action="store_true", help="record the fastest shape in the cache")
    ap.add_argument("--range-congruences", action="store_true",
                    help="sum the congruences the range-aware calls pick for [lo, hi) "
                         "(default: those of the prime-list calls, BB30 and EE33)")
    args = ap.parse_args()
    import torch

    from . import api
    primes = api.to_u64(api.sieve(args.lo, args.hi))
    grid = GRIDS[args.grid]
    if args.range_congruences:
        cb, ce = wv.wv_congruence_for_range(args.lo, args.hi)
        grid = [{**o, "cong_b": cb, "cong_e": ce} for o in grid]
    rows = []
    for r in sweep(primes, grid, args.reps):
        print(json.dumps(r), flush=True)
        rows.append(r)
    bad = [r for r in rows if not r["identical"]]
    if bad:
        raise SystemExit(f"shapes disagree: {bad}")
    if args.save and rows:
        best = min(rows, key=lambda r: r["acc_ms"])
        cache = load_cache()
        cache.setdefault(torch.cuda.get_device_name(), {})[str(bucket(primes.max()))] = best["options"]
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
        print(json.dumps({"saved": best, "bucket": bucket(primes.max()), "cache": CACHE}))


if __name__ == "__main__":
    main()
