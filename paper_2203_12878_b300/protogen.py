"""Seeded synthetic memory access protocols (inputs only).

This module builds protocol *text* plus the bounds it is checked under (thread
count, array sizes, parameter values).  It serves both the product path and
the oracle, and it holds none of the checking method: it never evaluates an
index, never decides a verdict.  Where a generator knows something by
construction (for example "this protocol is race-free because every cell has
one owner thread", or "a conflicting write was planted at phase p, array l,
cell k"), it records that in ``meta`` so that tests can pin the oracle to it.

Workload families (all seeded with ``random.Random``):

* ``config1``     -- 256 threads, one array of 2048 cells, an 8-iteration
                     synchronized loop (three variants).
* ``random_small``-- tiny random protocols over the whole syntax (T <= 8,
                     loop bounds <= 4, arrays <= 16 cells): conditionals,
                     min/max, floor division, Euclidean remainder, thread-
                     dependent bounds, parameters, syncs, out-of-range indices.
* ``config2``     -- one protocol, 1024 threads, 2 arrays of 2^20 cells, loop
                     nests of depth <= 3 with trip counts in 1..64, indices
                     (a*tid + b*x + c*y + d) mod N with coefficients in
                     [-8, 8], 1..6 syncs, reads and writes 50/50, about 10^7
                     accesses.  ``mode="literal"`` draws exactly that (most
                     such protocols are racy); ``mode="constructed"`` keeps the
                     shape but makes every cell owned by one thread, then
                     plants one conflicting write in 10% of seeds.
* ``config3``     -- 65,536 threads, 4 arrays of 2^24 cells, depth <= 2,
                     trip counts 1..32, 8 phases, about 2x10^8 accesses;
                     race-free and single-planted-race variants.
* ``config4``     -- a batch of protocols with log-uniform thread counts in
                     32..1024, depth <= 2, trip counts 1..32, 1..4 phases,
                     1..3 arrays of 2^12..2^18 cells, 20% with a planted race.
* ``shifted_small``-- mid-sized protocols (hundreds to thousands of threads,
                     arrays of odd sizes up to ~40,000 cells, 1..3 phases)
                     whose indices are mostly +-tid plus a function of the
                     loop variables (with or without a remainder), mixed with
                     accesses of other tid coefficients and conditions on the
                     loop variables; races arise where such ranges overlap.
* ``strided_small``-- the same sizes with indices a * tid plus a function of
                     the loop variables, a in +-{2, 3, 5, 7, 8} (with a
                     remainder that wraps at most once over the threads, or
                     none and kept in range), mixed with +-tid, tid-free and
                     conditional accesses; quiet seeds write only cells
                     a * (tid + T * k) and are race-free by construction.
"""
from __future__ import annotations

import dataclasses
import math
import random
from typing import Optional


@dataclasses.dataclass
class Protocol:
    text: str
    nthreads: int
    cells: list
    params: list = dataclasses.field(default_factory=list)
    meta: dict = dataclasses.field(default_factory=dict)

    def bounds(self):
        return self.nthreads, list(self.cells), list(self.params)


# --------------------------------------------------------------- config 1 --

def config1(variant: str = "drf") -> Protocol:
    """256 threads, A of 2048 cells, forS x in 0..8 { wr A[tid+256x]; sync;
    rd A[((tid+1) mod 256)+256x] }.  Variants: "drf" as written, "rdwr" with
    the read turned into a write, "nosync" with the sync removed."""
    second = "wr" if variant == "rdwr" else "rd"
    sync = "" if variant == "nosync" else " sync;"
    text = ("array A;\n"
            "forS x in 0 .. 8 {\n"
            f"  wr A[tid + 256 * x];{sync}\n"
            f"  {second} A[((tid + 1) % 256) + 256 * x];\n"
            "}\n")
    return Protocol(text, 256, [2048], [], {"variant": variant, "accesses": 4096})


# ------------------------------------------------------ small random ones --

class _Scope:
    def __init__(self, params):
        self.vars = []
        self.params = list(params)
        self.n = 0

    def fresh(self):
        self.n += 1
        return f"v{self.n}"


def _small_expr(r: random.Random, sc: _Scope, depth: int) -> str:
    names = ["tid"] + sc.vars + sc.params
    if depth <= 0 or r.random() < 0.35:
        k = r.random()
        if k < 0.45:
            return r.choice(names)
        return str(r.randint(0, 6)) if r.random() < 0.8 else f"(-{r.randint(1, 6)})"
    op = r.choice(["+", "+", "-", "*", "*", "/", "%", "min", "max"])
    a = _small_expr(r, sc, depth - 1)
    b = _small_expr(r, sc, depth - 1)
    if op in ("/", "%"):
        # mostly a non-zero literal divisor; sometimes an expression (may be 0)
        if r.random() < 0.85:
            b = str(r.choice([1, 2, 3, 4, 5, -2, -3]))
            if b.startswith("-"):
                b = f"({b})"
    if op in ("min", "max"):
        return f"{op}({a}, {b})"
    return f"({a} {op} {b})"


def _small_cond(r: random.Random, sc: _Scope, depth: int) -> str:
    k = r.random()
    if depth <= 0 or k < 0.6:
        rel = r.choice(["==", "!=", "<", "<=", ">", ">="])
        return f"{_small_expr(r, sc, 1)} {rel} {_small_expr(r, sc, 1)}"
    if k < 0.7:
        return r.choice(["true", "false"])
    if k < 0.8:
        return f"!({_small_cond(r, sc, depth - 1)})"
    op = r.choice(["&&", "||"])
    return f"({_small_cond(r, sc, depth - 1)}) {op} ({_small_cond(r, sc, depth - 1)})"


def _small_index(r: random.Random, sc: _Scope, cells: int, oob_prob: float) -> str:
    e = _small_expr(r, sc, 2)
    if r.random() < oob_prob:
        return e
    return f"({e}) % {cells}"


def _small_block(r, sc, arrays, cells, synced, depth, budget, oob_prob):
    out = []
    n = r.randint(1, 3)
    for _ in range(n):
        if budget[0] <= 0:
            break
        budget[0] -= 1
        k = r.random()
        if k < 0.42:
            i = r.randrange(len(arrays))
            mode = r.choice(["rd", "wr"])
            out.append(f"{mode} {arrays[i]}[{_small_index(r, sc, cells[i], oob_prob)}];")
        elif k < 0.52 and synced:
            out.append("sync;")
        elif k < 0.57:
            out.append("skip;")
        elif k < 0.72 and depth > 0:
            c = _small_cond(r, sc, 2)
            th = _small_block(r, sc, arrays, cells, False, depth - 1, budget, oob_prob)
            el = _small_block(r, sc, arrays, cells, False, depth - 1, budget, oob_prob) if r.random() < 0.6 else None
            s = f"if ({c}) {{ {' '.join(th)} }}"
            if el is not None:
                s += f" else {{ {' '.join(el)} }}"
            out.append(s)
        elif depth > 0:
            kind = "forS" if (synced and r.random() < 0.5) else "forU"
            v = sc.fresh()
            lo = r.choice(["0", "0", "1", str(r.randint(0, 2))])
            if r.random() < 0.25:
                hi = r.choice(["tid", "tid + 1", f"min(tid, {r.randint(1, 4)})", f"{r.randint(0, 4)} - tid"])
            elif r.random() < 0.2 and sc.vars:
                hi = f"{r.choice(sc.vars)} + {r.randint(0, 2)}"
            elif r.random() < 0.2 and sc.params:
                hi = r.choice(sc.params)
            else:
                hi = str(r.randint(0, 4))
            sc.vars.append(v)
            body = _small_block(r, sc, arrays, cells, kind == "forS", depth - 1, budget, oob_prob)
            sc.vars.pop()
            out.append(f"{kind} {v} in {lo} .. {hi} {{ {' '.join(body)} }}")
    return out


def random_small(seed: int, oob_prob: float = 0.04) -> Protocol:
    """A tiny random protocol over the whole syntax (T <= 8, small bounds)."""
    r = random.Random(seed)
    narrays = r.randint(1, 2)
    arrays = ["A", "B"][:narrays]
    cells = [r.randint(1, 16) for _ in range(narrays)]
    params = ["M"] if r.random() < 0.3 else []
    pvals = [r.randint(0, 4) for _ in params]
    sc = _Scope(params)
    body = _small_block(r, sc, arrays, cells, True, 3, [10], oob_prob)
    decl = f"array {', '.join(arrays)};\n"
    if params:
        decl += f"param {', '.join(params)};\n"
    text = decl + "\n".join(body) + "\n"
    return Protocol(text, r.randint(1, 8), cells, pvals, {"seed": seed})


# -------------------------------------------------- loop-nest generators --

@dataclasses.dataclass
class _Loop:
    kind: str          # "forS" / "forU"
    var: str
    trip: int
    body: list         # of _Loop / _Acc / "sync"


@dataclasses.dataclass
class _Acc:
    mode: str
    array: int
    index: str         # filled in after the nest is fixed


def _count_accesses(items, mult=1):
    n = 0
    for it in items:
        if isinstance(it, _Loop):
            n += _count_accesses(it.body, mult * it.trip)
        elif isinstance(it, _Acc):
            n += mult
    return n


def _count_syncs(items, mult=1):
    n = 0
    for it in items:
        if isinstance(it, _Loop):
            n += _count_syncs(it.body, mult * it.trip)
        elif it == "sync":
            n += mult
    return n


def _render(items, indent=0):
    pad = "  " * indent
    lines = []
    for it in items:
        if isinstance(it, _Loop):
            lines.append(f"{pad}{it.kind} {it.var} in 0 .. {it.trip} {{")
            lines.extend(_render(it.body, indent + 1))
            lines.append(f"{pad}}}")
        elif isinstance(it, _Acc):
            lines.append(f"{pad}{it.mode} {'ABCD'[it.array]}[{it.index}];")
        else:
            lines.append(f"{pad}{it}" if it.endswith(";") or it.endswith("}") else f"{pad}{it};")
    return lines


def _gen_nest(r: random.Random, max_depth: int, trip_hi: int, narrays: int, nsyncs: int):
    """A top-level sequence of 1..3 loop nests (depth <= max_depth); sync
    statements only where the synchronized fragment allows them: at top level
    or directly inside forS bodies whose ancestors are all forS."""
    counter = [0]

    def var():
        counter[0] += 1
        return "xyzwuv"[counter[0] - 1] if counter[0] <= 6 else f"q{counter[0]}"

    def nest(depth, synced):
        kind = "forS" if synced and r.random() < 0.6 else "forU"
        lp = _Loop(kind, var(), r.randint(1, trip_hi), [])
        inner_synced = synced and kind == "forS"
        nacc = r.randint(1, 3)
        for _ in range(nacc):
            lp.body.append(_Acc(r.choice(["rd", "wr"]), r.randrange(narrays), ""))
        if depth < max_depth and r.random() < 0.75:
            lp.body.insert(r.randint(0, len(lp.body)), nest(depth + 1, inner_synced))
        return lp

    top = [nest(1, True) for _ in range(r.randint(1, 3))]
    # sync slots: (list, position) pairs in synchronized context
    slots = []

    def collect(items, synced):
        if not synced:
            return
        slots.append(items)
        for it in items:
            if isinstance(it, _Loop) and it.kind == "forS":
                collect(it.body, True)

    collect(top, True)
    for _ in range(nsyncs):
        target = r.choice(slots)
        target.insert(r.randint(0, len(target)), "sync")
    return top


def _loop_vars_of(items, acc, stack=()):
    """Names of the loops enclosing access ``acc`` (outermost first)."""
    for it in items:
        if it is acc:
            return list(stack)
        if isinstance(it, _Loop):
            got = _loop_vars_of(it.body, acc, stack + (it.var,))
            if got is not None:
                return got
    return None


def _all_accs(items):
    for it in items:
        if isinstance(it, _Loop):
            yield from _all_accs(it.body)
        elif isinstance(it, _Acc):
            yield it


def _all_loops(items):
    for it in items:
        if isinstance(it, _Loop):
            yield it
            yield from _all_loops(it.body)


def _scale_to(r: random.Random, top, nthreads, lo_target, hi_target, trip_hi):
    """Adjust trip counts (staying in 1..trip_hi) until the access count is in range."""
    for _ in range(400):
        n = nthreads * _count_accesses(top)
        if lo_target <= n <= hi_target:
            return n
        loops = list(_all_loops(top))
        if n > hi_target:
            lp = max(loops, key=lambda l: l.trip)
            if lp.trip == 1:
                break
            lp.trip = max(1, lp.trip * 3 // 4)
        else:
            cands = [l for l in loops if l.trip < trip_hi]
            if not cands:
                break
            lp = r.choice(cands)
            lp.trip = min(trip_hi, lp.trip + max(1, lp.trip // 3))
    return nthreads * _count_accesses(top)


def _fmt_coef(c: int, term: str) -> str:
    if c < 0:
        return f"({c}) * {term}"
    return f"{c} * {term}"


def _literal_index(r: random.Random, vars_, ncells: int) -> str:
    terms = [_fmt_coef(r.randint(-8, 8), "tid")]
    for v in vars_[:2] if len(vars_) <= 2 else vars_[-2:]:
        terms.append(_fmt_coef(r.randint(-8, 8), v))
    d = r.randint(-8, 8)
    terms.append(f"({d})" if d < 0 else str(d))
    return f"({' + '.join(terms)}) % {ncells}"


def _owner_index(sigma: int, offset: int, nthreads: int, group: int, vars_, r: random.Random, ncells: int) -> str:
    """Index (sigma*tid + T*g + offset) mod N with g in [0, group): the cell
    determines its writer thread, so distinct threads never share a cell."""
    if vars_ and group > 1:
        coefs = [r.randint(1, 5) for _ in vars_]
        g = " + ".join(_fmt_coef(c, v) for c, v in zip(coefs, vars_))
        gexpr = f"(({g}) % {group})"
    else:
        gexpr = "0"
    return f"({sigma} * tid + {nthreads} * {gexpr} + {offset}) % {ncells}"


def _plant(r: random.Random, top, narrays: int, cells, nthreads: int):
    """Insert `if (tid == a || tid == b) { wr L[k]; }` at a top-level position;
    returns the planted (phase, array, cell).  The phase is the number of syncs
    the top-level statements before it run (their trip counts are literals)."""
    pos = r.randint(0, len(top))
    phase = _count_syncs(top[:pos])
    loc = r.randrange(narrays)
    k = r.randrange(cells[loc])
    a = r.randrange(nthreads)
    b = r.randrange(nthreads - 1)
    if b >= a:
        b += 1
    top.insert(pos, f"if (tid == {a} || tid == {b}) {{ wr {'ABCD'[loc]}[{k}]; }}")
    return {"planted": True, "phase": phase, "loc": loc, "index": k, "threads": sorted((a, b))}


def _nest_protocol(r, top, narrays, cells, nthreads, mode, plant):
    accs = list(_all_accs(top))
    meta = {"mode": mode}
    if mode == "literal":
        for a in accs:
            a.index = _literal_index(r, _loop_vars_of(top, a), cells[a.array])
    else:
        # one owner map per array for the whole protocol; the last array is
        # read-only with literal indices (reads never race with reads)
        ro = narrays - 1 if narrays > 1 else None
        owner = [(r.choice([1, -1]), r.randrange(cells[i])) for i in range(narrays)]
        for a in accs:
            if ro is not None and a.array == ro:
                a.mode = "rd"
                a.index = _literal_index(r, _loop_vars_of(top, a), cells[a.array])
            else:
                sigma, off = owner[a.array]
                group = max(1, cells[a.array] // nthreads)
                a.index = _owner_index(sigma, off, nthreads, group, _loop_vars_of(top, a), r, cells[a.array])
        meta["race_free_by_construction"] = not plant
    if plant:
        meta.update(_plant(r, top, narrays, cells, nthreads))
    else:
        meta["planted"] = False
    decl = f"array {', '.join('ABCD'[i] for i in range(narrays))};\n"
    text = decl + "\n".join(_render(top)) + "\n"
    return text, meta


# ---------------------------------------------------------- shifted_small --

def shifted_small(seed: int) -> Protocol:
    """A protocol of the shape described in the module header
    (``shifted_small``): every index provably inside its array, the same
    sync structure for every thread."""
    r = random.Random(0x5F17 ^ (seed * 2246822519))
    nthreads = r.choice([r.randint(100, 700), r.randint(700, 4100)])
    narrays = r.randint(1, 3)
    names = "ABC"[:narrays]
    cells = [r.randint(nthreads + 1, 41000) for _ in range(narrays)]
    lines = [f"array {', '.join(names)};"]
    nphases = r.randint(1, 3)
    # quiet seeds: in each phase one array is written, only at cells
    # tid + T * (its iteration), and only the other arrays are read -- race-free
    quiet = r.random() < 0.4
    if quiet:
        cells = [max(c, nthreads * 40) for c in cells]
    for ph in range(nphases):
        if ph:
            lines.append("sync;")
        for _ in range(r.randint(1, 3)):
            depth = r.randint(1, 2)
            vs = ["x", "y"][:depth]
            trips = [r.randint(1, 6) for _ in vs]
            body = []
            for _ in range(r.randint(1, 3)):
                a = r.randrange(narrays)
                n = cells[a]
                if quiet:
                    w = ph % narrays
                    if a == w:
                        body.append(f"wr {names[a]}[tid + {nthreads} * (({' + '.join(vs)}) % 40)];")
                    elif narrays > 1:
                        body.append(f"rd {names[a]}[({r.choice(['', '-1 * '])}tid + {r.randint(0, 999)} * {vs[0]}) % {n}];")
                    continue
                mode = r.choice(["rd", "wr", "wr"])
                kind = r.random()
                if kind < 0.4:              # (+-tid + f(x, y)) mod m, m <= the array, m >= threads
                    m = r.randint(nthreads, n)
                    sgn = r.choice(["", "-1 * "])
                    f = " + ".join(f"{r.randint(0, 9000)} * {v}" for v in vs)
                    body.append(f"{mode} {names[a]}[({sgn}tid + {f} + {r.randint(-5000, 5000)}) % {m}];")
                elif kind < 0.65:           # tid + g(x, y) with no remainder, kept in range
                    span = n - nthreads
                    g = f"(({' + '.join(f'{r.randint(1, 5)} * {v}' for v in vs)}) % {max(1, span // 8)})"
                    body.append(f"{mode} {names[a]}[tid + {g} * {r.randint(0, 8)}];")
                elif kind < 0.75:           # -tid + c, no remainder
                    body.append(f"{mode} {names[a]}[{nthreads - 1} - tid + {r.randint(0, n - nthreads)}];")
                elif kind < 0.9:            # another tid coefficient (mostly read)
                    body.append(f"{r.choice(['rd', 'rd', mode])} {names[a]}[({r.choice([2, 3, -2, 0])} * tid + {vs[-1]}) % {n}];")
                else:                       # a condition on a loop variable
                    body.append(f"if ({vs[0]} < {r.randint(1, 4)}) {{ {mode} {names[a]}[(tid + 7 * {vs[0]}) % {n}]; }}")
            if not body:
                body.append("skip;")
            text = "\n".join(body)
            kws, synced = [], True        # forS only inside forS (Fig. 1)
            for _ in vs:
                kws.append("forS" if synced and r.random() < 0.3 else "forU")
                synced = kws[-1] == "forS"
            for v, t, kw in reversed(list(zip(vs, trips, kws))):
                text = f"{kw} {v} in 0 .. {t} {{\n{text}\n}}"
            lines.append(text)
    return Protocol("\n".join(lines) + "\n", nthreads, cells, [], {"seed": seed})


# --------------------------------------------------------- strided_small --

def strided_small(seed: int) -> Protocol:
    """A protocol of the shape described in the module header
    (``strided_small``): every index provably inside its array, the same
    sync structure for every thread."""
    r = random.Random(0x57D1 ^ (seed * 2654435761))
    nthreads = r.choice([r.randint(64, 600), r.randint(600, 2000)])
    narrays = r.randint(1, 3)
    names = "ABC"[:narrays]
    quiet = r.random() < 0.4
    strides = [2, 3, 5, 7, 8, -2, -3, -5, -7, -8]
    cells = [r.randint(8 * nthreads + 1, 9 * nthreads + 20000) for _ in range(narrays)]
    kq = r.choice(strides[:5])      # quiet seeds: the one stride of every write
    if quiet:
        cells = [max(c, 8 * nthreads * 6 + 1) for c in cells]
    lines = [f"array {', '.join(names)};"]
    for ph in range(r.randint(1, 3)):
        if ph:
            lines.append("sync;")
        for _ in range(r.randint(1, 3)):
            depth = r.randint(1, 2)
            vs = ["x", "y"][:depth]
            trips = [r.randint(1, 5) for _ in vs]
            body = []
            for _ in range(r.randint(1, 3)):
                a = r.randrange(narrays)
                n = cells[a]
                if quiet:
                    w = ph % narrays
                    if a == w:              # distinct cells kq * (tid + T * j), j < 6, per thread and j
                        body.append(f"wr {names[a]}[{kq} * (tid + {nthreads} * (({' + '.join(vs)}) % 6))];")
                    elif narrays > 1:
                        body.append(f"rd {names[a]}[({r.choice(strides)} * tid + {r.randint(0, 999)} * {vs[0]}) % {n}];")
                    continue
                mode = r.choice(["rd", "wr", "wr"])
                kind = r.random()
                k = r.choice(strides)
                if kind < 0.4:              # (a * tid + f) mod m, one wrap at most: (T - 1) |a| < m <= n
                    m = r.randint((nthreads - 1) * abs(k) + 1, n)
                    f = " + ".join(f"{r.randint(0, 3000)} * {v}" for v in vs)
                    body.append(f"{mode} {names[a]}[({k} * tid + {f} + {r.randint(-4000, 4000)}) % {m}];")
                elif kind < 0.65:           # a * tid + g + base, no remainder, in range
                    span = n - abs(k) * (nthreads - 1) - 1
                    gm = max(1, span // 12)
                    g = f"(({' + '.join(f'{r.randint(1, 5)} * {v}' for v in vs)}) % {gm})"
                    base = 0 if k > 0 else abs(k) * (nthreads - 1)
                    body.append(f"{mode} {names[a]}[{k} * tid + {base} + {g} * {r.randint(0, 8)}];")
                elif kind < 0.8:            # +-tid with a remainder
                    m = r.randint(nthreads, n)
                    body.append(f"{mode} {names[a]}[({r.choice(['', '-1 * '])}tid + {r.randint(0, 99)} * {vs[-1]}) % {m}];")
                elif kind < 0.9:            # the same cell for every thread
                    body.append(f"rd {names[a]}[({vs[-1]} * 13) % {n}];")
                else:                       # a condition on a loop variable
                    body.append(f"if ({vs[0]} < {r.randint(1, 4)}) {{ {mode} {names[a]}[({k} * tid + 11 * {vs[0]}) % {n}]; }}")
            if not body:
                body.append("skip;")
            text = "\n".join(body)
            kws, synced = [], True        # forS only inside forS (Fig. 1)
            for _ in vs:
                kws.append("forS" if synced and r.random() < 0.3 else "forU")
                synced = kws[-1] == "forS"
            for v, t, kw in reversed(list(zip(vs, trips, kws))):
                text = f"{kw} {v} in 0 .. {t} {{\n{text}\n}}"
            lines.append(text)
    return Protocol("\n".join(lines) + "\n", nthreads, cells, [], {"seed": seed, "quiet": quiet})


# --------------------------------------------------------------- config 2 --

def config2(seed: int, mode: str = "literal", target: float = 1e7, plant: Optional[bool] = None) -> Protocol:
    """1024 threads, 2 arrays of 2^20 cells, depth <= 3, trip counts 1..64,
    1..6 syncs, about ``target`` accesses (scaled to [0.5, 2] x target)."""
    r = random.Random(0x2C0F2 ^ (seed * 7919))
    nthreads, narrays, ncells = 1024, 2, 1 << 20
    for _ in range(64):
        top = _gen_nest(r, 3, 64, narrays, r.randint(1, 6))
        n = _scale_to(r, top, nthreads, int(0.5 * target), int(2 * target), 64)
        if 0.5 * target <= n <= 2 * target:
            break
    if plant is None:
        plant = (mode == "constructed") and r.random() < 0.10
    cells = [ncells] * narrays
    text, meta = _nest_protocol(r, top, narrays, cells, nthreads, mode, plant)
    meta.update(seed=seed, accesses=n, syncs=_count_syncs(top))
    return Protocol(text, nthreads, cells, [], meta)


# --------------------------------------------------------------- config 3 --

def config3(seed: int, racy: bool = False, target: float = 2e8) -> Protocol:
    """65,536 threads, 4 arrays of 2^24 cells, depth <= 2, trip counts 1..32,
    8 phases (7 top-level syncs between 8 loop nests), about 2x10^8 accesses."""
    r = random.Random(0x3C0F3 ^ (seed * 104729))
    nthreads, narrays, ncells = 65536, 4, 1 << 24
    per_phase = target / 8
    top = []
    for ph in range(8):
        for _ in range(64):
            nest = _gen_nest(r, 2, 32, narrays, 0)[0]
            n = _scale_to(r, [nest], nthreads, int(0.6 * per_phase), int(1.6 * per_phase), 32)
            if 0.6 * per_phase <= n <= 1.6 * per_phase:
                break
        if ph:
            top.append("sync")
        top.append(nest)
    cells = [ncells] * narrays
    text, meta = _nest_protocol(r, top, narrays, cells, nthreads, "constructed", racy)
    meta.update(seed=seed, accesses=nthreads * _count_accesses([t for t in top if isinstance(t, _Loop)]),
                syncs=7)
    return Protocol(text, nthreads, cells, [], meta)


# --------------------------------------------------------------- config 4 --

def config4_one(r: random.Random, racy: bool) -> Protocol:
    """One protocol of the batched workload."""
    nthreads = int(round(math.exp(r.uniform(math.log(32), math.log(1024)))))
    narrays = r.randint(1, 3)
    cells = [1 << r.randint(12, 18) for _ in range(narrays)]
    nphases = r.randint(1, 4)
    top = []
    for ph in range(nphases):
        if ph:
            top.append("sync")
        top.append(_gen_nest(r, 2, 32, narrays, 0)[0])
    text, meta = _nest_protocol(r, top, narrays, cells, nthreads, "constructed", racy)
    meta.update(accesses=nthreads * _count_accesses([t for t in top if isinstance(t, _Loop)]),
                syncs=nphases - 1)
    return Protocol(text, nthreads, cells, [], meta)


def config4(master_seed: int = 1, count: int = 4096, racy_frac: float = 0.2):
    """The batched workload: ``count`` protocols, 20% with a planted race."""
    r = random.Random(0x4C0F4 ^ (master_seed * 1000003))
    return [config4_one(r, r.random() < racy_frac) for _ in range(count)]


def config5_arrivals(rate: float, duration_s: float, seed: int = 1):
    """Poisson arrival times (seconds) and, per arrival, which family it is
    drawn from: 90% the batched family, 10% the one-protocol family."""
    r = random.Random(0x5C0F5 ^ seed)
    t, out = 0.0, []
    while True:
        t += r.expovariate(rate)
        if t >= duration_s:
            return out
        out.append((t, "batch" if r.random() < 0.9 else "single"))


# ------------------------------------------------------------- BabyCUDA --

def random_babycuda(seed: int, ill_typed: bool = False) -> Protocol:
    """A small random BabyCUDA program (Fig. 3 syntax): reads bind data
    variables ("let x = A[n];") that flow only into write payloads
    ("A[n] := m;"), conditionals and loops over tid / loop variables /
    parameters, forS and sync in the synchronized fragment.  With
    ill_typed=True one index depends on a data variable (not typable)."""
    r = random.Random(0xBABC ^ (seed * 2654435761))
    narrays = r.randint(1, 2)
    arrays = ["A", "B"][:narrays]
    cells = [r.randint(1, 12) for _ in range(narrays)]
    params = ["M"] if r.random() < 0.3 else []
    pvals = [r.randint(0, 3) for _ in params]
    counter = [0]
    planted = [False]

    def fresh(prefix):
        counter[0] += 1
        return f"{prefix}{counter[0]}"

    def iexpr(names, depth=2):
        if depth <= 0 or r.random() < 0.4:
            return r.choice(names) if r.random() < 0.6 else str(r.randint(0, 5))
        op = r.choice(["+", "-", "*", "+"])
        return f"({iexpr(names, depth - 1)} {op} {iexpr(names, depth - 1)})"

    def block(typable, data, synced, depth, budget):
        out = []
        for _ in range(r.randint(1, 3)):
            if budget[0] <= 0:
                break
            budget[0] -= 1
            k = r.random()
            i = r.randrange(narrays)
            if k < 0.3:
                x = fresh("x")
                ix = iexpr(typable)
                if ill_typed and not planted[0] and data:
                    ix = f"{r.choice(data)} + {ix}"          # the index depends on data
                    planted[0] = True
                out.append(f"let {x} = {arrays[i]}[({ix}) % {cells[i]}];")
                data = data + [x]
            elif k < 0.6:
                payload = iexpr(typable + data)
                ix = iexpr(typable)
                if ill_typed and not planted[0] and data:
                    ix = f"{r.choice(data)} + {ix}"          # the index depends on data
                    planted[0] = True
                out.append(f"{arrays[i]}[({ix}) % {cells[i]}] := {payload};")
            elif k < 0.68 and synced:
                out.append("sync;")
            elif k < 0.72:
                out.append("skip;")
            elif k < 0.85 and depth > 0:
                c = f"{iexpr(typable, 1)} {r.choice(['==', '!=', '<', '>=', '<='])} {iexpr(typable, 1)}"
                th = block(typable, data, False, depth - 1, budget)
                el = block(typable, data, False, depth - 1, budget)
                out.append(f"if ({c}) {{ {' '.join(th)} }} else {{ {' '.join(el)} }}")
            elif depth > 0:
                kind = "forS" if synced and r.random() < 0.5 else "for"
                v = fresh("v")
                hi = r.choice([str(r.randint(0, 3)), "tid", "tid + 1"] + ([params[0]] if params else []))
                body = block(typable + [v], data, kind == "forS", depth - 1, budget)
                out.append(f"{kind} {v} in 0 .. {hi} {{ {' '.join(body)} }}")
        return out

    typable = ["tid"] + params
    body = block(typable, [], True, 3, [10])
    if ill_typed and not planted[0]:
        body += [f"let xz = {arrays[0]}[0];", f"{arrays[0]}[xz % {cells[0]}] := 1;"]
    decl = f"array {', '.join(arrays)};\n" + (f"param {', '.join(params)};\n" if params else "")
    return Protocol(decl + "\n".join(body) + "\n", r.randint(1, 6), cells, pvals, {"seed": seed})
