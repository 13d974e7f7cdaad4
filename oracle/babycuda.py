"""BabyCUDA with array contents: the semantics of Fig. 3 executed directly.

TEST INFRASTRUCTURE ONLY (used by tests/test_theorem1.py).  Pure Python, for
small programs.  Nothing here is shared with the product library.

A program is run for every thread id (rule par).  Each thread sees its own
reads and writes of the current phase and the shared history of earlier
phases; a read looks its value up with `lastwrite` (rules lastwrite-curr /
-prev / -undef: the thread's own current writes first, then earlier phases
from the most recent one, undefined if the index was never written); a
write records index and payload (rule write).  The synchronized fragment,
which the paper omits, is read as in the checker: a per-thread phase
counter bumped by `sync`; all threads finish a phase before the next one
starts, so a read in phase p sees every write of phases < p.

When an earlier phase is racy, more than one thread may have written an
index in it and `lastwrite` is not a function; this implementation then
takes the value written by the smallest tid.  For well-typed programs the
choice cannot change which indices are accessed (values only flow into
payloads), which is what Theorem 1 is about.

Syntax: declarations as in protocol text; statements
  let NAME = A[expr];   A[expr] := expr;   if (cond) {..} else {..}
  for NAME in expr .. expr {..}   forS NAME in expr .. expr {..}   sync;   skip;
"""
from __future__ import annotations

import re

UNDEF = None


class EvalError(Exception):
    def __init__(self, kind):
        super().__init__(kind)
        self.kind = kind          # "INDEX_OOB" / "DIV_ZERO"


# ------------------------------------------------------------------ parser --

_TOK = re.compile(r"\s*(?:(#[^\n]*|//[^\n]*)|(\d+)|([A-Za-z_]\w*)|(\.\.|==|!=|<=|>=|&&|\|\||:=|[;,{}\[\]()+\-*/%<>=!]))")


def _tokens(src):
    pos, out = 0, []
    while pos < len(src):
        m = _TOK.match(src, pos)
        if not m or m.end() == pos:
            if src[pos:].strip() == "":
                break
            raise SyntaxError(f"bad character at {pos}")
        pos = m.end()
        if m.group(1):
            continue
        if m.group(2):
            out.append(("int", int(m.group(2))))
        elif m.group(3):
            out.append(("name", m.group(3)))
        elif m.group(4):
            out.append(("p", m.group(4)))
    out.append(("end", None))
    return out


class _P:
    def __init__(self, src):
        self.t = _tokens(src)
        self.i = 0

    def peek(self, k=0):
        return self.t[self.i + k]

    def take(self):
        tok = self.t[self.i]
        self.i += 1
        return tok

    def want(self, kind, val=None):
        tok = self.take()
        if tok[0] != kind or (val is not None and tok[1] != val):
            raise SyntaxError(f"expected {val or kind}, got {tok}")
        return tok[1]

    def isp(self, val):
        return self.peek() == ("p", val)

    def isw(self, val):
        return self.peek() == ("name", val)

    # expressions: (op, args...) tuples
    def atom(self):
        kind, val = self.take()
        if kind == "int":
            return ("lit", val)
        if kind == "p" and val == "(":
            e = self.expr()
            self.want("p", ")")
            return e
        if kind == "p" and val == "-":
            return ("neg", self.atom())
        if kind == "name" and val in ("min", "max"):
            self.want("p", "(")
            a = self.expr()
            self.want("p", ",")
            b = self.expr()
            self.want("p", ")")
            return (val, a, b)
        if kind == "name":
            return ("var", val)
        raise SyntaxError(f"unexpected {val}")

    def term(self):
        e = self.atom()
        while self.peek()[0] == "p" and self.peek()[1] in ("*", "/", "%"):
            op = self.take()[1]
            e = (op, e, self.atom())
        return e

    def expr(self):
        e = self.term()
        while self.peek()[0] == "p" and self.peek()[1] in ("+", "-"):
            op = self.take()[1]
            e = (op, e, self.term())
        return e

    def catom(self):
        if self.isw("true") or self.isw("false"):
            return ("bool", self.take()[1] == "true")
        if self.isp("!"):
            self.take()
            return ("not", self.catom())
        if self.isp("("):
            save = self.i
            try:
                a = self.expr()
                if self.peek()[0] == "p" and self.peek()[1] in ("==", "=", "!=", "<", "<=", ">", ">="):
                    op = self.take()[1]
                    return ("cmp", op, a, self.expr())
            except SyntaxError:
                pass
            self.i = save
            self.take()
            c = self.cond()
            self.want("p", ")")
            return c
        a = self.expr()
        op = self.take()[1]
        return ("cmp", op, a, self.expr())

    def conj(self):
        c = self.catom()
        while self.isp("&&"):
            self.take()
            c = ("and", c, self.catom())
        return c

    def cond(self):
        c = self.conj()
        while self.isp("||"):
            self.take()
            c = ("or", c, self.conj())
        return c

    def block(self):
        self.want("p", "{")
        body = self.stmts("}")
        self.want("p", "}")
        return body

    def stmts(self, end):
        out = []
        while not (self.peek()[0] == "end" or self.peek() == ("p", end)):
            out.append(self.stmt())
        return out

    def stmt(self):
        if self.isw("skip"):
            self.take(); self.want("p", ";")
            return ("skip",)
        if self.isw("sync"):
            self.take(); self.want("p", ";")
            return ("sync",)
        if self.isw("let"):
            self.take()
            name = self.want("name")
            self.want("p", "=")
            arr = self.want("name")
            self.want("p", "[")
            ix = self.expr()
            self.want("p", "]")
            self.want("p", ";")
            return ("let", name, arr, ix)
        if self.isw("if"):
            self.take()
            self.want("p", "(")
            c = self.cond()
            self.want("p", ")")
            th = self.block()
            el = []
            if self.isw("else"):
                self.take()
                el = self.block()
            return ("if", c, th, el)
        if self.isw("for") or self.isw("forS"):
            kind = self.take()[1]
            var = self.want("name")
            self.want("name", "in")
            lo = self.expr()
            self.want("p", "..")
            hi = self.expr()
            return ("for", var, lo, hi, self.block(), kind == "forS")
        arr = self.want("name")
        self.want("p", "[")
        ix = self.expr()
        self.want("p", "]")
        self.want("p", ":=")
        val = self.expr()
        self.want("p", ";")
        return ("write", arr, ix, val)

    def program(self):
        arrays, params = [], []
        while self.isw("array") or self.isw("param"):
            kind = self.take()[1]
            names = [self.want("name")]
            while self.isp(","):
                self.take()
                names.append(self.want("name"))
            self.want("p", ";")
            (arrays if kind == "array" else params).extend(names)
        body = self.stmts(None)
        if self.peek()[0] != "end":
            raise SyntaxError("trailing input")
        return arrays, params, body


# --------------------------------------------------------------- semantics --

def _floor_div(a, b):
    if b == 0:
        raise EvalError("DIV_ZERO")
    return a // b                    # Python's // is floor division


def _euclid_mod(a, b):
    if b == 0:
        raise EvalError("DIV_ZERO")
    return a % abs(b)                # in [0, |b|)


def _ev(e, env):
    op = e[0]
    if op == "lit":
        return e[1]
    if op == "var":
        return env[e[1]]
    if op == "neg":
        v = _ev(e[1], env)
        return UNDEF if v is UNDEF else -v
    a, b = _ev(e[1], env), _ev(e[2], env)
    if a is UNDEF or b is UNDEF:     # an undefined value stays undefined
        return UNDEF
    if op == "+": return a + b
    if op == "-": return a - b
    if op == "*": return a * b
    if op == "/": return _floor_div(a, b)
    if op == "%": return _euclid_mod(a, b)
    if op == "min": return min(a, b)
    if op == "max": return max(a, b)
    raise ValueError(op)


def _cv(c, env):
    op = c[0]
    if op == "bool": return c[1]
    if op == "not": return not _cv(c[1], env)
    if op == "and":
        l, r = _cv(c[1], env), _cv(c[2], env)
        return l and r
    if op == "or":
        l, r = _cv(c[1], env), _cv(c[2], env)
        return l or r
    a, b = _ev(c[2], env), _ev(c[3], env)
    rel = c[1]
    return {"==": a == b, "=": a == b, "!=": a != b, "<": a < b, "<=": a <= b, ">": a > b, ">=": a >= b}[rel]


def run(src: str, nthreads: int, cells, params=()):
    """Executes the program for every thread.  Returns a dict with
    `phases` (list of {tid: {array: (reads set, writes dict)}}), `syncs`
    (per tid), and `error` ((kind, tid) of the smallest failing tid, or None)."""
    arrays, pnames, body = _P(src).program()
    aidx = {a: i for i, a in enumerate(arrays)}
    history = []                                     # completed phases, oldest first

    def lastwrite(arr, j, own):
        if j in own[arr][1]:                         # lastwrite-curr (own current phase)
            return own[arr][1][j]
        for ph in reversed(history):                 # lastwrite-prev, most recent first
            writers = sorted(t for t, rw in ph.items() if j in rw[arr][1])
            if writers:
                return ph[writers[0]][arr][1][j]
        return UNDEF                                 # lastwrite-undef

    def thread(tid):
        env = {"tid": tid}
        env.update(zip(pnames, params))
        cur = [{a: (set(), {}) for a in range(len(arrays))}]

        def exec_list(stmts):
            saved = dict(env)
            for s in stmts:
                yield from exec_stmt(s)
            env.clear()
            env.update(saved)

        def exec_stmt(s):
            k = s[0]
            if k == "skip":
                return
            if k == "sync":
                yield "sync"                         # the scheduler closes the phase
                return
            if k in ("let", "write"):
                arr = aidx[s[1]] if k == "write" else aidx[s[2]]
                j = _ev(s[2] if k == "write" else s[3], env)
                if j is UNDEF or j < 0 or j >= cells[arr]:
                    raise EvalError("INDEX_OOB")
                if k == "write":                     # rule write
                    cur[0][arr][1][j] = _ev(s[3], env)
                else:                                # rule read
                    cur[0][arr][0].add(j)
                    env[s[1]] = lastwrite(arr, j, cur[0])
                return
            if k == "if":                            # rules if-t / if-f
                yield from exec_list(s[2] if _cv(s[1], env) else s[3])
                return
            if k == "for":                           # rules for-1 / for-2
                lo, hi = _ev(s[2], env), _ev(s[3], env)
                for x in range(lo, hi):
                    env[s[1]] = x
                    yield from exec_list(s[4])
                env.pop(s[1], None)
                return
            raise ValueError(k)

        gen = exec_list(body)
        return gen, cur

    runs = {t: thread(t) for t in range(nthreads)}
    alive = set(range(nthreads))
    syncs = {t: 0 for t in range(nthreads)}
    errors = {}
    phases = []
    while alive:
        phase = {}
        for t in sorted(alive):
            gen, cur = runs[t]
            try:
                next(gen)                            # runs until its next sync
                syncs[t] += 1
            except StopIteration:
                alive.discard(t)
            except EvalError as e:
                errors[t] = e.kind
                alive.discard(t)
            phase[t] = cur[0]
            cur[0] = {a: (set(), {}) for a in range(len(arrays))}
        phases.append(phase)
        history.append(phase)                        # rule par: merge, then the next phase
    err = None
    if errors:
        t = min(errors)
        err = (errors[t], t)
    return {"phases": phases, "syncs": syncs, "error": err, "narrays": len(arrays)}


def access_set(res):
    """{(phase, array, index, tid, mode)} of a run (mode 1 = write)."""
    out = set()
    for p, ph in enumerate(res["phases"]):
        for t, rw in ph.items():
            for a, (r, w) in rw.items():
                out.update((p, a, j, t, 0) for j in r)
                out.update((p, a, j, t, 1) for j in w)
    return out


def history_drf(res) -> bool:
    """Definition 1 on the history: no phase has i1 != i2 and j with j
    written by i1 and read or written by i2 (per array)."""
    for ph in res["phases"]:
        tids = sorted(ph)
        for a in range(res["narrays"]):
            for i1 in tids:
                w1 = set(ph[i1][a][1])
                if not w1:
                    continue
                for i2 in tids:
                    if i2 != i1 and w1 & (ph[i2][a][0] | set(ph[i2][a][1])):
                        return False
    return True
