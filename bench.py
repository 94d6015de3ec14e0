#!/usr/bin/env python3
"""Benchmark: B_{p-3} and E_{p-3} mod p for every prime of the 1e5-wide window
[1062200000, 1062300000) near 1e9 (4907 primes, all < 2^30).

One step = the whole path over the window: segmented sieve on the device,
planning, the persistent accumulation of the library's default congruences
for B_{p-3} and E_{p-3} (generated from BB30, eqn 3.7, and EE33, eqn 5.6),
per-prime finalisation, and flag/compaction of the zero residues
(wv_search_ex).  The headline value is primes/s (each prime gets both
residues); modmul/s counts two modular multiplications per summed term
(eqn 3.12).

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 launch with torch.distributed.run; the N ranks search the N
consecutive 1e5-wide windows from 1062200000, split into contiguous shards of
equal estimated cost by the library's range sharding (weak scaling, no
data-path collective; NCCL only for the max-over-ranks time and the prime
count).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("primes/sec and modmul/sec at p≈1e9 (B_{p-3},E_{p-3} mod p), "
          "% IMAD peak; p99 latency")
LO, HI = 1_062_200_000, 1_062_300_000
WIDTH = HI - LO
IMAD_PER_SM_CLK = 64          # 32-bit integer multiply-add results per SM per clock
IMAD_SLOTS_PER_MODMUL = 5     # one 32-bit Montgomery product: mul.wide (2) + mul.lo (1) + mul.hi (2)
SM_MAX_MHZ_FALLBACK = 2070.0
# --workload top: the 391 primes of [1e11 - 1e4, 1e11) on the 64-bit path.  One 64-bit
# Montgomery product for p < 2^37 (R = 2^64 in two 32-bit REDC rounds) costs 17 IMAD slots:
# c g as three mul.wide and one mul.lo (7), each REDC round one mul.lo and two mul.wide (10).
TOP_LO, TOP_WIDTH = 10**11 - 10**4, 10**4
IMAD_SLOTS_PER_MODMUL64 = 17
# Per accumulation kernel, from one `ncu --set full` capture of a small case of the same
# workload (the summary named in "profile"): the IMAD-pipe busy share
# (sm__pipe_fmaheavy_cycles_active, of peak), the terms summed per SM per clock in that capture,
# and the DRAM bytes (read + write) per prime of the capture.  The roofline fraction of a bench
# run is that busy share scaled by the run's own terms per SM per clock.  Set an entry to None
# whenever its kernel changes, until it is captured again.
PIPE_PROFILE = {
    # k_accumulate<0,1,48,1> (form 48: the u form on pieces of 3072+ terms, lane chains; chain
    # set-up with folded REDC products; group loop unrolled by two): 492 primes of [1062200000,
    # 1062210000), BB2244 + EE2004, 2.3139e10 terms, 7.998 ms at 2.067 GHz; IMAD pipe 79.43 %,
    # ALU 69.54 % of elapsed.  Traffic: one launch of the full window (--metrics
    # dram__bytes_read.sum,dram__bytes_write.sum, the second launch): 1.042 GB read + 0.637 GB
    # written
    "accumulate_m31": {"imad_pct": 0.7943, "alu_pct": 0.6954, "terms_per_clk_sm": 9.209,
                       "inst_per_term": 6.8121e9 * 32 / 2.3139e10,
                       "traffic_bytes": 1041792512 + 636746752,
                       "profile": "profiles/accumulate_m31_p1e9_small.md"},
    # k_accumulate_m64cap<50,128,1> (form 50: the u form with one-round products on pieces of
    # 32768+ terms, cheaper per-chain set-up): 17 primes of [1e11 - 1e4, 1e11 - 9500), BB3802 +
    # EE4122, 6.8787e10 terms, 42.019 ms at 2.068 GHz; IMAD pipe 88.41 %, ALU 54.63 %.  Traffic:
    # one launch of the full 391-prime window (the second launch): 111.6 MB read + 53.8 MB written
    "accumulate_m64": {"imad_pct": 0.8841, "alu_pct": 0.5463, "terms_per_clk_sm": 5.2087,
                       "inst_per_term": 3.2788e10 * 32 / 6.8787e10,
                       "traffic_bytes": 111565056 + 53785600,
                       "profile": "profiles/accumulate_m64_top_window.md"},
}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        rows = []
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 10:
                continue
            if self.uuid and self.uuid not in parts[1]:
                continue
            rows.append(parts)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def gpu_uuid(torch):
    try:
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return u.replace("GPU-", "")
    except Exception:
        return None


# ---------------------------------------------------------------- CPU oracle
def oracle_sample(k: int, seed: int = 7):
    from paper_2101_11157_gb300 import workloads as W
    ps = W.primes_in(LO, LO + 20000)  # a seeded draw from the window's first 2e4
    return W.seeded_subset(ps, k, seed)


def run_oracle_step(primes, threads: int):
    """Both residues for `primes` with the oracle on `threads` host threads
    (one prime per thread at a time, B then E)."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    b, e = O.residues(primes, method_b="default", method_e="default", threads=threads)
    return time.perf_counter() - t0, {"b": b, "e": e}


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    sample = oracle_sample(cores, seed=11)
    for _ in range(args.warmup):
        run_oracle_step(sample, cores)
    times = []
    for _ in range(args.steps):
        dt, _ = run_oracle_step(sample, cores)
        times.append(dt)
    ms = 1000.0 * sum(times) / len(times)
    val = len(sample) / (ms / 1000.0)
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "primes/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int128",
        "data": "synthetic: primes of the window near 1.06e9 (no dataset)",
        "config": {"workload": f"B_{{p-3}}, E_{{p-3}} mod p for primes in [{LO}, {HI}); "
                               "reference = plain CPU oracle (Stafford-Vandiver eqn 2.4 for B, "
                               "Glaisher eqn 4.1 for E), one seeded prime per host core per step",
                   "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": val, "unit": "primes/s", "cores": cores, "kind": "oracle",
                         "value_per_core": val / cores,
                         "sample": f"{len(sample)} seeded primes of the window per step (one per host "
                                   f"core), B then E on each of {cores} threads"},
        "e2e": {"value": val, "unit": "primes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm
def gpu_arm(args):
    import numpy as np
    import torch

    from paper_2101_11157_gb300 import api, wv

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    top = args.workload == "top"
    # N ranks search N windows' worth of the range (weak scaling), split into contiguous
    # shards of equal estimated cost (sum of p) by the library's range sharding
    from paper_2101_11157_gb300 import shard
    if top:  # the ws 1e4-wide windows just below 1e11
        width = min(args.width, TOP_WIDTH)
        span = (TOP_LO - (ws - 1) * TOP_WIDTH, TOP_LO + width)
    else:
        width = args.width
        span = (LO, LO + (ws - 1) * WIDTH + width)
    lo, hi = shard.shard_of(span[0], span[1], rank, ws)
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count

    # inputs: the window's primes (for counting terms and for the e2e leg)
    d_pr_all = api.sieve(lo, hi)
    primes = api.to_u64(d_pr_all)
    n_primes = primes.size
    cong = wv.wv_congruence_for_range(lo, hi)  # the congruences the search uses on this window
    tb, te = wv.wv_count_terms(primes, *cong)
    modmuls_per_step = 2 * (tb + te)
    cap_h = 64
    hits = torch.empty((cap_h, 2), dtype=torch.int64, device="cuda")
    d_pr = torch.empty(n_primes, dtype=torch.int64, device="cuda")
    d_rb, d_re = torch.empty_like(d_pr), torch.empty_like(d_pr)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")  # > L2 (129 MB)

    def step():
        return wv.wv_search_ex(lo, hi, 0, hits, d_pr, d_rb, d_re, None, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # timed region: K steps, CUDA events per step, L2 flushed between steps
    uuid = gpu_uuid(torch)
    sampler = ClockSampler(uuid)
    sampler.start()
    time.sleep(0.3)
    wv.wv_profile_reset()
    wv.wv_profile_enable(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    t_wall = time.perf_counter()
    nh = 0
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        nh, npr = step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    wv.wv_profile_enable(False)
    prof = wv.wv_profile_collect()
    launches = wv.wv_profile_launches()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms) / len(step_ms)
    if dist:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    # e2e: host prime list in pinned memory -> device -> residues -> host, with the
    # congruences the search picks for the window (a caller who knows the range passes them)
    e2e_opt = {"cong_b": cong[0], "cong_e": cong[1]}
    h_in = torch.from_numpy(primes.view(np.int64)).pin_memory()
    h_b = torch.empty(n_primes, dtype=torch.int64, pin_memory=True)
    h_e = torch.empty(n_primes, dtype=torch.int64, pin_memory=True)
    d_in = torch.empty_like(d_pr)
    e2e_ms = []
    for i in range(max(1, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d_in.copy_(h_in, non_blocking=True)
        wv.wv_residues_ex(d_in, d_rb, d_re, e2e_opt, stream)
        h_b.copy_(d_rb, non_blocking=True)
        h_e.copy_(d_re, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1000 * (time.perf_counter() - t0))
    e2e_step = statistics.median(e2e_ms)
    if dist:
        t = torch.tensor([e2e_step], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_step = float(t.item())

    # CPU oracle baseline (rank 0, N = 1 only): one seeded prime of the window per host core,
    # all cores busy
    cpu = None
    if ws == 1 and rank == 0 and not args.no_cpu and not top:
        cores = os.cpu_count() or 1
        sample = oracle_sample(cores, seed=7)
        dt, res = run_oracle_step(sample, threads=cores)
        cpu = {"value": len(sample) / dt, "unit": "primes/s", "cores": cores, "kind": "oracle",
               "sample": f"{len(sample)} seeded primes of the window (one per host core, both residues): "
                         "B by Stafford-Vandiver (eqn 2.4), E by Glaisher (eqn 4.1), 128-bit remainders",
               "seconds": dt,
               # one prime per core, all cores at once: the rate of one core
               "value_per_core": len(sample) / dt / cores}
        # the oracle and the GPU agree on the sample
        idx = np.searchsorted(primes, sample)
        gb, ge = api.to_u64(d_rb)[idx], api.to_u64(d_re)[idx]
        cpu["agrees_with_gpu"] = bool(np.array_equal(gb, res["b"]) and np.array_equal(ge, res["e"]))

    # roofline of the dominant kernel (the p < 2^30 accumulation; the 64-bit one for top): the
    # integer multiply (IMAD) pipe.  frac = the pipe's busy share in the kernel's ncu capture,
    # scaled by this run's terms per SM per clock against the capture's.
    kname = "accumulate_m64" if top else "accumulate_m31"
    slots = IMAD_SLOTS_PER_MODMUL64 if top else IMAD_SLOTS_PER_MODMUL
    acc_launches, acc_ms = prof.get(kname, (0, 0.0))
    acc_avg_ms = acc_ms / max(1, acc_launches)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz") or SM_MAX_MHZ_FALLBACK)
    clk_mhz = float((clocks or {}).get("sm_mhz") or sm_max)
    tpcs = (tb + te) / (acc_avg_ms / 1e3) / sms / (clk_mhz * 1e6) if acc_avg_ms else 0.0
    prof_k = PIPE_PROFILE.get(kname)
    full_launch = width == (TOP_WIDTH if top else WIDTH)
    pipe_peak = sms * clk_mhz * 1e6  # IMAD-pipe cycles per second over all SMs
    if prof_k:
        frac = prof_k["imad_pct"] * tpcs / prof_k["terms_per_clk_sm"]
        roof = {"bound": "alu", "achieved": frac * pipe_peak, "peak": pipe_peak,
                "unit": "IMAD-pipe cycles/s", "frac": frac,
                "traffic": prof_k["traffic_bytes"] if full_launch else None,
                "traffic_basis": (f"ncu dram__bytes_read.sum + dram__bytes_write.sum of one full launch "
                                  f"({prof_k['profile']})" if prof_k["traffic_bytes"] else
                                  "not captured for the current kernel at this size"),
                "frac_basis": f"IMAD-pipe busy {prof_k['imad_pct']:.3f} at {prof_k['terms_per_clk_sm']:.3f} "
                              f"terms/clk/SM ({prof_k['profile']}); this run {tpcs:.3f} terms/clk/SM at "
                              f"{clk_mhz:.0f} MHz",
                "alu_pipe_busy_in_capture": prof_k.get("alu_pct"),
                # multiply-pipe lane-cycles and instructions (all pipes) per algorithmic
                # Montgomery product (two per summed term, eqn 3.12), from the capture
                "imad_slots_per_modmul": prof_k["imad_pct"] * IMAD_PER_SM_CLK
                                         / prof_k["terms_per_clk_sm"] / 2.0,
                "inst_per_modmul": prof_k["inst_per_term"] / 2.0}
    else:
        roof = {"bound": "alu", "achieved": None, "peak": pipe_peak, "unit": "IMAD-pipe cycles/s",
                "frac": None, "traffic": None,
                "frac_basis": "no ncu capture of the current kernel"}
    # the same work counted as two Montgomery products per summed term (eqn 3.12), against the
    # IMAD slots one exact product costs (profiles/int_pipe_probes.md); the grouped forms issue
    # fewer slots per term, so this can exceed the pipe fraction (and 1 on the 64-bit path)
    peak_gmodmul = sms * IMAD_PER_SM_CLK * clk_mhz * 1e6 / slots / 1e9
    achieved_gmodmul = (modmuls_per_step / (acc_avg_ms / 1000.0)) / 1e9 if acc_avg_ms else 0.0
    roof.update({"kernel": kname, "kernel_ms": acc_avg_ms, "terms_per_clk_sm": tpcs,
                 "modmul_equiv_frac": achieved_gmodmul / peak_gmodmul if peak_gmodmul else None,
                 "modmul_equiv": {"achieved": achieved_gmodmul, "peak": peak_gmodmul, "unit": "Gmodmul/s",
                                  "peak_basis": f"{sms} SMs x {IMAD_PER_SM_CLK} IMAD lanes/clk x "
                                                f"{clk_mhz:.0f} MHz / {slots} IMAD slots per "
                                                f"{'64' if top else '32'}-bit Montgomery product"}})
    total_primes, total_modmuls = n_primes, modmuls_per_step
    if dist:
        t = torch.tensor([n_primes, modmuls_per_step], device="cuda", dtype=torch.int64)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        total_primes, total_modmuls = int(t[0].item()), int(t[1].item())
    value = total_primes / (ms / 1000.0)
    cong_names = [wv.wv_congruence_info(c)[0] for c in cong]
    line = {
        "metric": METRIC, "value": value, "unit": "primes/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic: every prime of the window, sieved on the device (no dataset)",
        "config": {"workload": f"sieve + B_{{p-3}} ({cong_names[0]}) + E_{{p-3}} ({cong_names[1]}) mod p "
                               f"+ zero/near flags for all primes in [{lo}, {hi}) per GPU"
                               + (" (64-bit path, 2^31 <= p < 2^37)" if top else ""),
                   "primes_per_gpu": int(n_primes), "congruences": "+".join(cong_names),
                   "terms_per_step": int(tb + te), "parallelism": f"range-sharded x{ws}",
                   "range": list(span), "shard": [lo, hi], "primes_all_gpus": int(total_primes),
                   "l2": "flushed between steps (256 MB write)"},
        "modmul_per_s": total_modmuls / (ms / 1000.0),
        "roofline": roof,
        "e2e": {"value": total_primes / (e2e_step / 1000.0), "unit": "primes/s",
                "h2d_bytes_per_step": int(n_primes * 8), "d2h_bytes_per_step": int(n_primes * 16),
                "path": "host prime list (pinned) -> wv_residues_ex (the window's congruences) -> host residues"},
        "gpu_launches": int(launches),
        "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()},
        "wall_s": wall, "hits": int(nh),
        "clocks": clocks,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if top:
        line["cpu_baseline"] = None
        line["cpu_baseline_note"] = ("not timed: the oracle needs about an hour per prime near 1e11 "
                                     "(eqn 2.4 / eqn 4.1 single sums); its stored residues of 8 of "
                                     "these primes are checked by the GPU tests")
    # the batched and serving forms against the plain one, on the same GPU (rank 0, N = 1)
    if ws == 1 and rank == 0 and not top and not args.no_extras:
        from paper_2101_11157_gb300 import workloads as W
        try:
            r = batch_measure(W.batch_requests(seed=7), steps=2, warmup=1)
            line["batch"] = {k: r[k] for k in (
                "batched_primes_s", "per_request_primes_s", "ratio", "per_request_default_primes_s",
                "ratio_vs_default", "identical_results", "congruence_groups", "per_request_calls",
                "primes", "requests", "batched_ms", "per_request_ms")}
            line["batch"]["workload"] = ("64 requests of batch_requests(seed=7): 1..4096 primes each, "
                                         "log-uniform in [1e5, 1e10); per_request = one wv_residues_ex per "
                                         "request and congruence group (same congruences as the batch)")
        except Exception as exc:  # reported, not hidden
            line["batch"] = {"error": repr(exc)}
        try:
            sq = W.serving_stream(seed=11, n=args.serve_queries)
            r = serve_measure(sq, epoch_terms=4e10)
            line["serve"] = {k: r[k] for k in (
                "served_primes_s", "plain_primes_s", "ratio", "latency", "plain_latency",
                "identical_results", "queries", "primes", "makespan_s", "plain_makespan_s")}
            line["serve"]["workload"] = (f"the first {len(sq)} queries of serving_stream(seed=11): "
                                         "Poisson arrivals at 200/s, half ranges [10^U(6,10), +10^U(3,6)), "
                                         "half single primes; latency = completion - arrival; plain = one "
                                         "query at a time in arrival order")
        except Exception as exc:
            line["serve"] = {"error": repr(exc)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- batch / serve
def _pctl(xs, q):
    import numpy as np
    return float(np.percentile(np.asarray(xs), q)) if len(xs) else None


def _band_groups(primes):
    """Positions of `primes` grouped by the congruence pair the range-aware
    calls pick for [p, p + 1): {(cong_b, cong_e): index array}."""
    import numpy as np

    from paper_2101_11157_gb300 import wv
    groups = {}
    for i, p in enumerate(np.asarray(primes, dtype=np.uint64)):
        groups.setdefault(wv.wv_congruence_for_range(int(p), int(p) + 1), []).append(i)
    return {k: np.asarray(v, dtype=np.int64) for k, v in groups.items()}


def batch_measure(reqs_np, steps: int, warmup: int, options=None, autotune_key=None):
    """The batched form against one call per request, on the same GPU.

    batched: wv_batch (one graph; primes grouped by the congruence pair their
    size calls for).  per_request: one wv_residues_ex per request and
    congruence group, with the same pairs (the plain form, range-aware).
    per_request_default: one wv_residues_pm3 per request (BB30 + EE33)."""
    import numpy as np
    import torch

    from paper_2101_11157_gb300 import wv
    stream = torch.cuda.current_stream()
    reqs = []
    for a in reqs_np:
        d = torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()
        reqs.append((d, torch.empty_like(d), torch.empty_like(d)))
    n = sum(a.size for a in reqs_np)
    table = []
    if autotune_key:
        from paper_2101_11157_gb300 import tune
        options, table = tune.tune_batch(reqs, key=autotune_key)
    b = wv.wv_batch_create(reqs, options or None)
    _, _, nodes = wv.wv_batch_info(b)
    groups_in_batch = wv.wv_batch_groups(b)
    # the plain form: per request and congruence group, sub-tensors made outside the timing
    plain = []   # (request, positions, primes, out B, out E, options)
    terms = 0
    for r, a in enumerate(reqs_np):
        for (cb, ce), idx in _band_groups(a).items():
            sub = torch.from_numpy(np.ascontiguousarray(a[idx]).view(np.int64)).cuda()
            plain.append((r, idx, sub, torch.empty_like(sub), torch.empty_like(sub),
                          {"cong_b": cb, "cong_e": ce}))
            tb, te = wv.wv_count_terms(a[idx], cb, ce)
            terms += tb + te

    def timed(fn, k):
        ms = []
        for _ in range(k):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    run_batch = lambda: wv.wv_batch_run(b, stream)
    run_plain = lambda: [wv.wv_residues_ex(d, rb, re, o, stream) for _, _, d, rb, re, o in plain]
    run_default = lambda: [wv.wv_residues_pm3(d, rb, re, stream) for d, rb, re in reqs]
    for fn in (run_batch, run_plain, run_default):
        for _ in range(warmup):
            fn()
    torch.cuda.synchronize()
    ms_b = timed(run_batch, steps)
    out_b = [(rb.clone(), re.clone()) for _, rb, re in reqs]
    ms_p = timed(run_plain, steps)
    ms_d = timed(run_default, steps)
    same = all(torch.equal(rb, x) and torch.equal(re, y) for (_, rb, re), (x, y) in zip(reqs, out_b))
    for r, idx, _, rb, re, _ in plain:
        x, y = out_b[r]
        same = same and np.array_equal(x.cpu().numpy()[idx], rb.cpu().numpy()) \
            and np.array_equal(y.cpu().numpy()[idx], re.cpu().numpy())
    wv.wv_batch_destroy(b)
    mb, mp, md = statistics.median(ms_b), statistics.median(ms_p), statistics.median(ms_d)
    return {"batched_primes_s": n / (mb / 1e3), "per_request_primes_s": n / (mp / 1e3),
            "ratio": mp / mb, "per_request_default_primes_s": n / (md / 1e3),
            "ratio_vs_default": md / mb, "batched_ms": mb, "per_request_ms": mp,
            "per_request_default_ms": md, "modmul_per_s": 2 * terms / (mb / 1e3),
            "identical_results": bool(same), "graph_nodes": nodes,
            "congruence_groups": groups_in_batch, "per_request_calls": len(plain),
            "options": options or {}, "autotune": table, "steps": steps, "warmup": warmup,
            "requests": len(reqs_np), "primes": int(n), "terms": int(terms)}


def batch_arm(args):
    """64 seeded requests of uneven cost: one graph-captured batch vs one call per request."""
    import torch

    from paper_2101_11157_gb300 import workloads as W
    torch.cuda.set_device(0)
    reqs_np = W.batch_requests(seed=7, k=args.requests, max_len=args.max_len)
    key = None if args.no_autotune else f"requests{len(reqs_np)}-seed7-max{args.max_len}-grouped"
    r = batch_measure(reqs_np, args.steps, args.warmup, autotune_key=key)
    line = {"workload": "batch", "metric": "primes/s, 64 requests in one launch vs one launch per request",
            "value": r["batched_primes_s"], "unit": "primes/s", **r,
            "config": {"requests": len(reqs_np), "primes": r["primes"], "terms": r["terms"],
                       "lengths": "floor(2^U(0,12)) clamped to [1, %d]" % args.max_len,
                       "primes_from": "next_prime(10^U(5,10)), seed 7"}}
    print(json.dumps(line), flush=True)
    return 0


def serve_measure(stream_q, epoch_terms: float, epoch_form: int = 0, epoch_block: int = 0,
                  plain_block: int = 0, piece_log2: int = 0):
    """Serve a stream of queries (continuous batching) and, for comparison,
    run it one query at a time in arrival order; both pick congruences by the
    query's range."""
    import numpy as np
    import torch

    from paper_2101_11157_gb300 import api, wv
    srv = wv.wv_server_create(epoch_terms=epoch_terms, epoch_form=epoch_form, epoch_block=epoch_block,
                              piece_log2=piece_log2)
    t0 = time.perf_counter()
    ids = []
    for q in stream_q:
        dt = q["t"] - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        ids.append(wv.wv_server_submit_range(srv, q["lo"], q["hi"]) if q["kind"] == "range"
                   else wv.wv_server_submit_prime(srv, q["p"]))
    infos = [wv.wv_server_wait(srv, i) for i in ids]
    makespan = time.perf_counter() - t0
    st = wv.wv_server_stats(srv)
    served_res = [wv.wv_server_result(srv, i) for i in ids]
    wv.wv_server_destroy(srv)
    lat = [i["t_done"] - i["t_submit"] for i in infos]
    wait_admit = [i["t_admit"] - i["t_submit"] for i in infos]
    service = [i["t_done"] - i["t_admit"] for i in infos]
    n_primes = sum(i["n_primes"] for i in infos)
    t0 = time.perf_counter()
    lat_p = []
    same = True
    popt = {"block": plain_block} if plain_block else None
    for q, res in zip(stream_q, served_res):
        dt = q["t"] - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        if q["kind"] == "range":
            lo = max(q["lo"], 5)
            if q["hi"] > lo:
                _, pr, rb, re = api.search(lo, q["hi"], with_residues=True, options=popt)
            else:
                pr = rb = re = torch.empty(0, dtype=torch.int64, device="cuda")
        else:
            pr = torch.tensor([q["p"]], dtype=torch.int64, device="cuda")
            rb, re = api.residues(pr, options=popt)
        torch.cuda.synchronize()
        lat_p.append(time.perf_counter() - t0 - q["t"])
        same = same and np.array_equal(api.to_u64(rb), res[1]) and np.array_equal(api.to_u64(re), res[2])
    makespan_p = time.perf_counter() - t0
    kinds = [q["kind"] for q in stream_q]

    def stats(ls):
        out = {}
        for k in ("prime", "range"):
            xs = [x for x, kk in zip(ls, kinds) if kk == k]
            out[k] = {"p50_s": _pctl(xs, 50), "p99_s": _pctl(xs, 99), "n": len(xs)}
        return out
    return {"served_primes_s": n_primes / makespan, "plain_primes_s": n_primes / makespan_p,
            "ratio": makespan_p / makespan, "makespan_s": makespan, "plain_makespan_s": makespan_p,
            "latency": stats(lat), "plain_latency": stats(lat_p), "identical_results": bool(same),
            "admission_wait": stats(wait_admit), "service_time": stats(service), "server": st,
            "queries": len(stream_q), "primes": int(n_primes)}


def serve_arm(args):
    """A seeded Poisson stream of range and single-prime queries, served with
    continuous batching and, for comparison, one query at a time."""
    import torch

    from paper_2101_11157_gb300 import workloads as W
    torch.cuda.set_device(0)
    stream_q = W.serving_stream(seed=11, n=args.queries, rate=args.rate)
    if args.max_range:
        for q in stream_q:
            if q["kind"] == "range":
                q["hi"] = min(q["hi"], q["lo"] + args.max_range)
    r = serve_measure(stream_q, args.epoch_terms, args.epoch_form, args.epoch_block, args.plain_block,
                      args.piece_log2)
    line = {"workload": "serve", "metric": "primes/s and p50/p99 latency, continuous batching vs one query at a time",
            "value": r["served_primes_s"], "unit": "primes/s", **r,
            "config": {"queries": len(stream_q), "rate_per_s": args.rate, "seed": 11,
                       "range_len_cap": args.max_range or None,
                       "epoch_terms": args.epoch_terms, "primes": r["primes"],
                       "plain_block": args.plain_block or None,
                       "epoch_form": args.epoch_form,
                       "epoch_block": args.epoch_block or 32,
                       "piece_log2": args.piece_log2 or 17}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wv", choices=["wv", "reference"])
    ap.add_argument("--width", type=int, default=WIDTH, help="window width (smaller for profiling)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extras", action="store_true",
                    help="window workload only: skip the batch and serving comparisons")
    ap.add_argument("--serve-queries", type=int, default=48,
                    help="queries of the seeded stream served in the default run")
    ap.add_argument("--workload", default="window", choices=["window", "top", "batch", "serve"])
    ap.add_argument("--requests", type=int, default=64, help="batch: number of requests")
    ap.add_argument("--max-len", type=int, default=4096, help="batch: longest request")
    ap.add_argument("--no-autotune", action="store_true", help="batch: library default launch shape")
    ap.add_argument("--queries", type=int, default=256, help="serve: queries in the stream")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: mean arrivals per second")
    ap.add_argument("--max-range", type=int, default=0, help="serve: cap on range length (0: none)")
    ap.add_argument("--epoch-terms", type=float, default=4e10, help="serve: terms per epoch")
    ap.add_argument("--epoch-form", type=int, default=0,
                    help="serve: 0 default (1), 1 persistent over both paths, 2 one warp per tile, "
                         "3 persistent per path")
    ap.add_argument("--epoch-block", type=int, default=0, help="serve: epoch block size (0: 32)")
    ap.add_argument("--piece-log2", type=int, default=0,
                    help="serve: longest piece of a sum in a query's plan, 2^k terms (0: 17)")
    ap.add_argument("--plain-block", type=int, default=0,
                    help="serve: accumulation block size of the one-query-at-a-time form (0: default)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "batch":
        return batch_arm(args)
    if args.workload == "serve":
        return serve_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
