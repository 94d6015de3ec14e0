"""Congruence generator: Proposition 2.1 (Tanner and Wagstaff) as a program.

A congruence is  LHS * X = sum_j c_j(t) S_t(x_j, y_j)  (mod p)  with
S_t(x, y) = sum_{xp < s < yp} s^t, where X is B_{2k} (t = 2k - 1, odd) or
E_{p-1-2k} (t = p - 1 - 2k, even) and each coefficient c_j(t) is a formal
sum of powers, sum_d c_d d^t.  The three transformations of Prop. 2.1 act on
such expressions:

  separation   S_t(x, z) = S_t(x, y) + S_t(y, z)
  reflection   S_t(x, y) = (-1)^t S_t(1 - y, 1 - x)
  subdivision  S_t(x, y) = d^t sum_{i<d} S_t((x + i)/d, (y + i)/d)

After each subdivision the expression is simplified: every sum is moved into
[0, 1/2] by reflection (split at 1/2 first by separation), the pieces are
summed on the common refinement of their endpoints (separation), zero pieces
are dropped and neighbours with equal coefficients merged.  The cost of a
congruence is p sum_j (y_j - x_j), the approximate number of terms (Sec. 2).

Uses (Sec. 2 "Exhaustive searches", "Heuristic searches"):
  * derive the paper's congruences from Vandiver's congruence (Bernoulli)
    and from eqn 4.1 (Euler) by the subdivision sequences the paper gives,
    and check the library's transcribed tables against them;
  * exhaustive search: all sequences of at most l subdivisions with
    d <= d_i at step i, keeping the least cost for each number of sums;
  * greedy (heuristic) search: repeatedly take the cheapest congruence
    reachable with lambda subdivisions of d <= D.

    python -m paper_2101_11157_gb300.congen --derive           # all derivations + table check
    python -m paper_2101_11157_gb300.congen --greedy 40 --D 8  # cost per round
    python -m paper_2101_11157_gb300.congen --exhaustive 2,3,3
"""
from __future__ import annotations

import argparse
import itertools
from fractions import Fraction as F

HALF = F(1, 2)


class Congruence:
    """sum_j coef_j S_t(x_j, y_j) with coef_j = {d: c} meaning sum_d c d^t.

    kind 'B' (t odd: reflection sign -1) or 'E' (t even: sign +1); `lhs`
    describes the left side for display and specialisation."""

    def __init__(self, kind: str, lhs, sums, history=()):
        self.kind = kind
        self.lhs = lhs
        self.sums = sums  # list of (x, y, coef) with 0 <= x < y <= 1/2, sorted, simplified
        self.history = tuple(history)

    @property
    def sign(self) -> int:
        return -1 if self.kind == "B" else 1

    @property
    def m(self) -> int:
        return len(self.sums)

    @property
    def cost(self) -> F:
        return sum((y - x for x, y, _ in self.sums), F(0))

    def key(self):
        return tuple((x, y, tuple(sorted(c.items()))) for x, y, c in self.sums)

    def __repr__(self):
        return f"Congruence({self.kind}, m={self.m}, cost={self.cost} p)"


def _add(a: dict, b: dict, scale: int = 1) -> dict:
    out = dict(a)
    for d, c in b.items():
        v = out.get(d, 0) + scale * c
        if v:
            out[d] = v
        else:
            out.pop(d, None)
    return out


def _reflect_into_half(kind: str, raw):
    sign = -1 if kind == "B" else 1
    out = []
    for x, y, c in raw:
        parts = [(x, HALF), (HALF, y)] if x < HALF < y else [(x, y)]  # separation at 1/2
        for a, b in parts:
            if a >= HALF:
                out.append((1 - b, 1 - a, {d: sign * v for d, v in c.items()}))
            else:
                out.append((a, b, c))
    return out


def simplify(kind: str, raw) -> list:
    """Reflect into [0, 1/2], sum on the common refinement, merge equal neighbours.

    A sweep over the endpoints keeps the running coefficient of the covering
    sums, so the cost is O(n log n) dictionary updates."""
    moved = _reflect_into_half(kind, raw)
    events = {}
    for x, y, c in moved:
        events.setdefault(x, []).append((1, c))
        events.setdefault(y, []).append((-1, c))
    cuts = sorted(events)
    cur, pieces = {}, []
    for a, b in zip(cuts, cuts[1:]):
        for sgn, c in events[a]:
            cur = _add(cur, c, sgn)
        if cur:
            if pieces and pieces[-1][1] == a and pieces[-1][2] == cur:
                pieces[-1][1] = b
            else:
                pieces.append([a, b, dict(cur)])
    return [(a, b, c) for a, b, c in pieces]


def subdivide(cg: Congruence, x: F, y: F, d: int) -> Congruence:
    """Apply subdivision with d to c S_t(x, y), where [x, y] lies inside one
    sum of cg (separation splits that sum first); then simplify."""
    x, y = F(x), F(y)
    raw, done = [], False
    for a, b, c in cg.sums:
        if not done and a <= x and y <= b:
            if a < x:
                raw.append((a, x, c))
            if y < b:
                raw.append((y, b, c))
            scaled = {dd * d: v for dd, v in c.items()}
            raw += [((x + i) / d, (y + i) / d, scaled) for i in range(d)]
            done = True
        else:
            raw.append((a, b, c))
    if not done:
        raise ValueError(f"no sum contains ({x}, {y})")
    return Congruence(cg.kind, cg.lhs, simplify(cg.kind, raw), cg.history + ((x, y, d),))


# ---------------------------------------------------------------- starting relations
def vandiver() -> Congruence:
    """C_k(2,5,6) B_{2k} = S_{2k-1}(1/6, 1/5) + S_{2k-1}(1/3, 2/5) (Sec. 2, eqn 2.5)."""
    raw = [(F(1, 6), F(1, 5), {1: 1}), (F(1, 3), F(2, 5), {1: 1})]
    return Congruence("B", ("C", (2, 5, 6)), simplify("B", raw))


def stafford_vandiver() -> Congruence:
    """C_k(3,4,6) B_{2k} = S_{2k-1}(1/6, 1/4) (Sec. 2, eqn 2.4)."""
    return Congruence("B", ("C", (3, 4, 6)), [(F(1, 6), F(1, 4), {1: 1})])


def glaisher_e1() -> Congruence:
    """(-1)^k 4^{2k-1} E_t = S_t(0, 1/4), t = p - 1 - 2k (Sec. 4, eqn 4.1 with
    the (-1)^k sign)."""
    return Congruence("E", ("E1",), [(F(0), F(1, 4), {1: 1})])


# The paper's derivations (Sec. 2 and Sec. 4): (start, steps), each step the
# interval subdivided and d.  Two readings of the text:
#  * B9 "starting with Vandiver's congruence": the printed B9 follows from B2
#    (Vandiver's congruence after its own first subdivision), not from the
#    bare congruence: its sums (3^t + 6^t) S_t(1/18, ...) and -2^t S_t(11/36,
#    1/3) carry B2's factor (1 + 2^t) and term -2^t S_t(3/10, 1/3);
#  * E5 -> E9 names S_t(0, 1/128), but E5 holds S_t(0, 1/64) and E9 holds
#    32^t S_t(0, 1/128) = (16^t 2^t) S_t(0, 1/128): the step subdivides
#    S_t(0, 1/64).
DERIVATIONS = {
    "BB2": ("vandiver", [((1, 3), (2, 5), 2)]),
    "BB6": ("BB2", [((3, 10), (1, 3), 2), ((1, 3), (7, 20), 2), ((13, 40), (1, 3), 2),
                    ((1, 3), (27, 80), 2)]),
    "BB9": ("BB2", [((1, 6), (1, 5), 3), ((4, 15), (5, 18), 2), ((7, 18), (2, 5), 2),
                    ((11, 36), (1, 3), 5)]),
    "BB16": ("BB9", [((7, 36), (1, 5), 3), ((3, 10), (11, 36), 3), ((47, 180), (4, 15), 2),
                     ((47, 360), (2, 15), 2), ((83, 180), (7, 15), 2)]),
    "BB22": ("BB16", [((1, 3), (61, 180), 3), ((1, 9), (61, 540), 2), ((4, 15), (29, 108), 2),
                      ((29, 108), (97, 360), 2), ((479, 1080), (4, 9), 2)]),
    "BB30": ("BB22", [((43, 108), (2, 5), 6), ((4, 15), (173, 648), 2), ((4, 9), (241, 540), 2),
                      ((299, 1080), (5, 18), 2)]),
    "EE3": ("e1", [((0, 1), (1, 4), 2), ((0, 1), (1, 8), 2)]),
    "EE5": ("EE3", [((0, 1), (1, 16), 2), ((0, 1), (1, 32), 2)]),
    "EE9": ("EE5", [((0, 1), (1, 64), 2), ((3, 8), (7, 16), 3)]),
    "EE16": ("EE9", [((3, 16), (5, 24), 3), ((7, 16), (11, 24), 3), ((0, 1), (1, 128), 2),
                     ((1, 8), (7, 48), 2), ((11, 24), (15, 32), 2)]),
    "EE24": ("EE16", [((0, 1), (1, 256), 2), ((1, 16), (5, 72), 4), ((41, 96), (7, 16), 3),
                      ((41, 288), (7, 48), 2), ((15, 32), (137, 288), 2)]),
}


def derive(name: str, _cache={}) -> Congruence:
    if name in _cache:
        return _cache[name]
    if name == "vandiver":
        cg = vandiver()
    elif name == "e1":
        cg = glaisher_e1()
    else:
        start, steps = DERIVATIONS[name]
        cg = derive(start)
        for (xn, xd), (yn, yd), d in steps:
            cg = subdivide(cg, F(xn, xd), F(yn, yd), d)
    _cache[name] = cg
    return cg


# ---------------------------------------------------------------- specialisation
def specialise(cg: Congruence):
    """The form at the index of the search (B_{p-3}: t = p - 4; E_{p-3}: t = p - 3):
    d^t -> d^-3 (B) or d^-2 (E).  Returns (lhs, [(coef, x, y)]) as rationals."""
    e = 3 if cg.kind == "B" else 2
    if cg.lhs[0] == "C":
        a, b, c = cg.lhs[1]
        # C_k(a,b,c) with p - 2k = e and 4k = 2(p - e) = -2e (mod p)
        lhs = F(a**e + b**e - c**e - 1, -2 * e)
    else:
        lhs = F(-(4 ** (e - 1)))  # (-1)^k 4^{2k-1} at 2k = e = 2
    rows = [(sum((F(v, d**e) for d, v in c.items()), F(0)), x, y) for x, y, c in cg.sums]
    return lhs, rows


def matches_table(cg: Congruence, lhs_int: int, rows_int) -> bool:
    """Whether the library's row list (coef, x, y) with constant lhs_int is the
    specialised form of cg: the same intervals, coefficients proportional to
    the left sides."""
    lhs, rows = specialise(cg)
    if len(rows) != len(rows_int):
        return False
    mine = sorted((x, y, c / lhs) for c, x, y in rows)
    theirs = sorted((F(x), F(y), F(c, lhs_int)) for c, x, y in rows_int)
    return mine == theirs


def evaluate(cg: Congruence, p: int, t: int) -> int:
    """The right side mod p at exponent t (plain Python, for checks)."""
    total = 0
    for x, y, c in cg.sums:
        coef = sum(v * pow(d, t, p) for d, v in c.items()) % p
        lo = (x.numerator * p) // x.denominator + 1
        hi = -((-y.numerator * p) // y.denominator)
        total += coef * sum(pow(s, t, p) for s in range(lo, hi))
    return total % p


# ---------------------------------------------------------------- searches
def moves(cg: Congruence, dmax: int):
    for x, y, _ in cg.sums:
        for d in range(2, dmax + 1):
            yield x, y, d


def exhaustive(start: Congruence, ds) -> dict:
    """All congruences reachable with at most len(ds) subdivisions, the i-th
    with 2 <= d <= ds[i]; returns {m: least-cost congruence with m sums}."""
    best = {start.m: start}
    frontier = {start.key(): start}
    for dmax in ds:
        nxt = {}
        for cg in frontier.values():
            for x, y, d in moves(cg, dmax):
                c2 = subdivide(cg, x, y, d)
                k = c2.key()
                if k not in nxt:
                    nxt[k] = c2
                if c2.m not in best or c2.cost < best[c2.m].cost:
                    best[c2.m] = c2
        frontier = nxt
    return best


def _coef_at(sums, starts, v):
    import bisect
    i = bisect.bisect_right(starts, v) - 1
    if i >= 0 and sums[i][0] <= v < sums[i][1]:
        return sums[i][2]
    return {}


def cost_delta(cg: Congruence, j: int, d: int, starts=None) -> F:
    """The change of cost when sum j of cg is subdivided with d, without
    building the new congruence: the new coefficient is compared with the old
    one on every piece the change touches."""
    import bisect
    if starts is None:
        starts = [a for a, _, _ in cg.sums]
    a, b, c = cg.sums[j]
    scaled = {dd * d: v for dd, v in c.items()}
    mods = [(a, b, {dd: -v for dd, v in c.items()})]
    mods += _reflect_into_half(cg.kind, [((a + i) / d, (b + i) / d, scaled) for i in range(d)])
    cuts = set()
    for x, y, _ in mods:
        cuts.add(x)
        cuts.add(y)
        i = max(bisect.bisect_right(starts, x) - 1, 0)
        while i < len(cg.sums) and cg.sums[i][0] < y:
            for v in (cg.sums[i][0], cg.sums[i][1]):
                if x < v < y:
                    cuts.add(v)
            i += 1
    cuts = sorted(cuts)
    delta = F(0)
    for u, v in zip(cuts, cuts[1:]):
        inside = [m for m in mods if m[0] <= u and v <= m[1]]
        if not inside:
            continue
        old = _coef_at(cg.sums, starts, u)
        new = old
        for _, _, dc in inside:
            new = _add(new, dc)
        delta += (v - u) * ((1 if new else 0) - (1 if old else 0))
    return delta


def greedy_fast(start: Congruence, rounds: int, D: int = 8, min_gain: F = F(0), log=None):
    """The heuristic search with lambda = 1, choosing each round's subdivision
    by its exact cost change (cost_delta) and applying only the best one."""
    cg = start
    out = [cg]
    for r in range(rounds):
        starts = [a for a, _, _ in cg.sums]
        best = None
        for j in range(cg.m):
            for d in range(2, D + 1):
                dl = cost_delta(cg, j, d, starts)
                if best is None or dl < best[0]:
                    best = (dl, j, d)
        if best is None or best[0] >= -min_gain:
            break
        a, b, _ = cg.sums[best[1]]
        cg = subdivide(cg, a, b, best[2])
        out.append(cg)
        if log:
            log(r, cg)
    return out


def greedy(start: Congruence, rounds: int, D: int = 8, lam: int = 1):
    """The heuristic search: each round takes the cheapest congruence reachable
    with `lam` subdivisions of d <= D.  Returns the list of congruences."""
    out = [start]
    cg = start
    for _ in range(rounds):
        cands = {cg.key(): cg}
        for _ in range(lam):
            nxt = {}
            for c in cands.values():
                for x, y, d in moves(c, D):
                    c2 = subdivide(c, x, y, d)
                    nxt.setdefault(c2.key(), c2)
            cands = nxt
        cg = min(cands.values(), key=lambda c: (c.cost, c.m))
        out.append(cg)
    return out


# ---------------------------------------------------------------- generated tables
# Cheaper congruences for B_{p-3} and E_{p-3} from the greedy search (Sec. 2,
# "Heuristic searches", with lambda = 1, D = 8): (name, start, rounds).
# The Bernoulli ones start from B30 as derived here (formal coefficients,
# left side C_k(2,5,6), which is 14 at 2k = p - 3); the Euler ones from the
# library's E33 table (integer coefficients relative to its left side).
GENERATED = [("BB249", "BB30", 40), ("BB476", "BB30", 80), ("BB1115", "BB30", 200),
             ("BB2244", "BB30", 400), ("BB3802", "BB30", 680),
             ("EE200", "EE33", 40), ("EE404", "EE33", 80), ("EE967", "EE33", 200),
             ("EE2004", "EE33", 400), ("EE4122", "EE33", 800)]


def generated(which=None):
    """{name: (congruence, lhs as an integer)} for the GENERATED list."""
    starts = {}
    out = {}
    for name, start, rounds in GENERATED:
        if which and name not in which:
            continue
        if start not in starts:
            if start == "EE33":
                lhs, rows = library_table("EE33")
                cg = Congruence("E", ("table", lhs), simplify("E", [(x, y, {1: c}) for c, x, y in rows]))
            else:
                cg, lhs = derive(start), 14
            rounds_needed = max(r for n, s, r in GENERATED if s == start and (not which or n in which))
            starts[start] = (greedy_fast(cg, rounds_needed), lhs)
        traj, lhs = starts[start]
        cg = traj[min(rounds, len(traj) - 1)]
        assert f"{name[:2]}{cg.m}" == name, (name, cg.m)
        out[name] = (cg, lhs)
    return out


def emit_header(path: str):
    """Write the generated congruences as a C header for the library."""
    gens = generated()
    dist_all, rows_all, tc_all, td_all, entries = [], [], [], [], []
    for name, _, _ in GENERATED:
        cg, lhs = gens[name]
        dist = sorted({d for _, _, c in cg.sums for d in c})
        dpos = {d: i for i, d in enumerate(dist)}
        entries.append((name, 0 if cg.kind == "B" else 1, cg.m, lhs, len(rows_all), len(dist_all),
                        len(dist), cg.cost))
        for x, y, c in cg.sums:
            assert max(x.numerator, x.denominator, y.numerator, y.denominator) < 2**32
            rows_all.append((x.numerator, x.denominator, y.numerator, y.denominator, len(tc_all), len(c)))
            for d in sorted(c):
                tc_all.append(c[d])
                td_all.append(dpos[d])
        dist_all += dist
    L = ["// Generated by paper_2101_11157_gb300/congen.py (emit_header): congruences for",
         "// B_{p-3} and E_{p-3} from the greedy search of Sec. 2 (\"Heuristic searches\")",
         "// over Prop. 2.1.  Row j of a congruence is (sum_k c_k d_k^t) S_t(xn/xd, yn/yd),",
         "// t = p - 4 (B) or p - 3 (E), so d^t = d^-3 resp. d^-2; the left side is `lhs`.",
         "// Do not edit: regenerate with `python -m paper_2101_11157_gb300.congen --emit`.",
         "#pragma once", "#include <stdint.h>", "",
         "struct WvGenTable {", "  const char *name;", "  int kind;", "  int nrows;", "  int64_t lhs;",
         "  uint32_t row0, dist0, ndist;", "  double cost;  // in units of p", "};", "",
         "static const WvGenTable kWvGenTables[] = {"]
    for name, kind, m, lhs, r0, d0, nd, cost in entries:
        L.append(f'  {{"{name}", {kind}, {m}, {lhs}LL, {r0}u, {d0}u, {nd}u, {float(cost)!r}}},')
    L += ["};", "static const int kWvNumGenTables = (int)(sizeof(kWvGenTables) / sizeof(kWvGenTables[0]));",
          "", "// xn, xd, yn, yd, first term, number of terms",
          "static const uint32_t kWvGenRows[][6] = {"]
    L += ["  {%d, %d, %d, %d, %d, %d}," % r for r in rows_all]
    L += ["};", "", "static const int64_t kWvGenTermC[] = {"]
    for i in range(0, len(tc_all), 12):
        L.append("  " + " ".join(f"{v}," for v in tc_all[i:i + 12]))
    L += ["};", "", "// index of d_k in the congruence's list of distinct bases",
          "static const uint16_t kWvGenTermD[] = {"]
    for i in range(0, len(td_all), 16):
        L.append("  " + " ".join(f"{v}," for v in td_all[i:i + 16]))
    L += ["};", "", "static const uint64_t kWvGenDist[] = {"]
    for i in range(0, len(dist_all), 12):
        L.append("  " + " ".join(f"{v}ull," for v in dist_all[i:i + 12]))
    L += ["};", ""]
    with open(path, "w") as f:
        f.write("\n".join(L))
    return entries


# ---------------------------------------------------------------- library tables
def library_table(name: str):
    """(lhs, [(coef, (xn, xd), (yn, yd))]) of a transcribed congruence in the library."""
    from . import wv
    for cid in range(wv.wv_congruence_count()):
        nm, kind, n, lhs = wv.wv_congruence_info(cid)
        if nm == name:
            rows = []
            for r in range(n):
                coef, xn, xd, yn, yd = wv.wv_congruence_row(cid, r)
                rows.append((coef, F(xn, xd), F(yn, yd)))
            return lhs, rows
    raise KeyError(name)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--derive", action="store_true", help="derive the paper's congruences, check the tables")
    ap.add_argument("--greedy", type=int, default=0, help="rounds of the heuristic search")
    ap.add_argument("--D", type=int, default=8)
    ap.add_argument("--lam", type=int, default=1)
    ap.add_argument("--exhaustive", default="", help="comma-separated d_i, e.g. 3,3,2")
    ap.add_argument("--start", default="vandiver", choices=["vandiver", "sv", "e1", *DERIVATIONS])
    ap.add_argument("--emit", action="store_true", help="write csrc/wv_tables_gen.h")
    args = ap.parse_args()
    if args.emit:
        import os
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "wv_tables_gen.h")
        for name, kind, m, lhs, r0, d0, nd, cost in emit_header(path):
            print(f"{name}: m={m} cost=p/{float(1 / cost):.3f} distinct bases={nd}")
        return
    start = stafford_vandiver() if args.start == "sv" else derive(args.start)
    if args.derive:
        for name in DERIVATIONS:
            cg = derive(name)
            lhs, rows = library_table(name)
            ok = matches_table(cg, lhs, [(c, x, y) for c, x, y in rows])
            print(f"{name:5s} m={cg.m:3d} cost={cg.cost}p (p/{float(1 / cg.cost):.3f})  "
                  f"library table {'matches' if ok else 'DIFFERS'}")
    if args.exhaustive:
        ds = [int(v) for v in args.exhaustive.split(",")]
        for m, cg in sorted(exhaustive(start, ds).items()):
            print(f"m={m:3d} cost={cg.cost}p = p/{float(1 / cg.cost):.3f}  via {cg.history}")
    if args.greedy:
        for i, cg in enumerate(greedy(start, args.greedy, args.D, args.lam)):
            print(f"round {i:3d}: m={cg.m:4d} cost={cg.cost}p = p/{float(1 / cg.cost):.3f}")


if __name__ == "__main__":
    main()
