// Interval analysis, lowering to the device program, and work
// decomposition (see prepare.h).
//
// Interval analysis: every expression node gets the range of values it can
// take over tid in [0, T), parameters at their given values and each loop
// variable over [min lo, max hi - 1] of its loop's bounds.  A node whose
// range leaves int64 makes the protocol OVERFLOW_RISK (arithmetic is on
// mathematical integers held in int64; the paper's expressions are over the
// naturals, Fig. 1, with operators left open).  If every range fits int32
// the GPU evaluates in 32-bit arithmetic.  An access whose index provably
// lies in [0, cells) and cannot divide by zero needs no evaluation in the
// count pass.  Trip counts give static upper bounds on syncs (phase-field
// width), accesses and interpreter steps per thread.
#include <algorithm>
#include <cstring>
#include <functional>
#include <stdexcept>

#include "prepare.h"

namespace drf {
namespace {

using i128 = __int128;
constexpr i128 kI64Min = INT64_MIN, kI64Max = INT64_MAX;
constexpr i128 kI32Min = INT32_MIN, kI32Max = INT32_MAX;
constexpr i128 kHuge = (i128)1 << 100;     // saturation for counts

struct Iv {
    i128 lo = 0, hi = -1;                  // empty when lo > hi
    bool empty() const { return lo > hi; }
    static Iv point(i128 v) { return Iv{v, v}; }
};

i128 sat(i128 v) { return v > kHuge ? kHuge : v; }
i128 mul_sat(i128 a, i128 b)
{
    if (a == 0 || b == 0) return 0;
    if (a > 0 && b > 0) {
        // counts: no 128-bit division on the common path
        i128 r;
        if (__builtin_mul_overflow(a, b, &r)) return kHuge;
        return sat(r);
    }
    if (a > kHuge / b) return kHuge;
    return sat(a * b);
}

// ceil(a / b) for a >= 0, b > 0, in 64-bit arithmetic when both fit.
i128 div_ceil(i128 a, i128 b)
{
    if (a < ((i128)1 << 62) && b < ((i128)1 << 62))
        return (i128)(((uint64_t)a + (uint64_t)b - 1) / (uint64_t)b);
    return (a + b - 1) / b;
}

i128 floor_div(i128 a, i128 b)
{
    i128 q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
    return q;
}

// Map from AST nodes to their analysis results: open addressing over one
// array (the analyses store a value for nearly every node, so per-entry
// allocations would dominate their cost).  References returned by at() stay
// valid until the next insertion.
template <typename K, typename V>
class NodeMap {
public:
    V &operator[](const K *k)
    {
        if ((n_ + 1) * 2 > slots_.size()) rehash(std::max<size_t>(64, slots_.size() * 2));
        Slot &x = slots_[probe(k)];
        if (!x.key) {
            x.key = k;
            x.val = V{};
            n_++;
        }
        return x.val;
    }
    const V &at(const K *k) const
    {
        if (slots_.empty() || slots_[probe(k)].key != k) throw std::out_of_range("node without an analysis result");
        return slots_[probe(k)].val;
    }
    size_t count(const K *k) const { return !slots_.empty() && slots_[probe(k)].key == k; }

private:
    struct Slot {
        const K *key = nullptr;
        V val{};
    };
    std::vector<Slot> slots_;
    size_t n_ = 0;

    size_t probe(const K *k) const
    {
        const size_t mask = slots_.size() - 1;
        size_t i = (size_t)(((uintptr_t)k >> 4) * 0x9E3779B97F4A7C15ull >> 20) & mask;
        while (slots_[i].key && slots_[i].key != k) i = (i + 1) & mask;
        return i;
    }
    void rehash(size_t cap)
    {
        std::vector<Slot> old(cap);
        old.swap(slots_);
        for (const Slot &x : old)
            if (x.key) slots_[probe(x.key)] = x;
    }
};

struct LoopInfo {
    i128 trip_max = 0;       // over all threads and outer iterations
    i128 body_steps = 0;     // steps per iteration, upper bound
    i128 body_tuples = 0;
};

struct Work {
    i128 tuples = 0, steps = 0, syncs = 0;
};

class Analyzer {
public:
    Analyzer(uint32_t T, const uint64_t *cells, const int64_t *params, uint16_t nslots)
        : T_(T), cells_(cells), params_(params), var_(nslots) {}

    bool risk = false;
    bool wide = false;
    bool maybe_div0 = false;                               // some division's divisor may be zero
    NodeMap<Stmt, LoopInfo> loops;
    NodeMap<Stmt, bool> count_eval;                      // access -> evaluate index in the count pass
    bool any_count_eval = false;                         // some access must be evaluated in the count pass
    NodeMap<Expr, Iv> ranges;

    NodeMap<Stmt, Work> work;                            // per statement, upper bounds per thread

    Work stmt(const Stmt &s, bool reachable)
    {
        Work w = stmt_inner(s, reachable);
        work[&s] = w;
        return w;
    }

    Work stmt_inner(const Stmt &s, bool reachable)
    {
        Work w;
        switch (s.op) {
        case SOp::Skip:
            return w;
        case SOp::Sync:
            w.steps = 1; w.syncs = 1;
            return w;
        case SOp::Access: {
            bool div0 = false;
            Iv ix = expr(*s.index, div0, reachable);
            bool in_range = !ix.empty() && ix.lo >= 0 && ix.hi < (i128)cells_[s.loc];
            count_eval[&s] = !(in_range && !div0);
            if (!(in_range && !div0)) any_count_eval = true;
            w.tuples = 1; w.steps = 1;
            return w;
        }
        case SOp::Seq:
            for (auto &it : s.items) {
                Work x = stmt(*it, reachable);
                w.tuples = sat(w.tuples + x.tuples);
                w.steps = sat(w.steps + x.steps);
                w.syncs = sat(w.syncs + x.syncs);
            }
            return w;
        case SOp::If: {
            cond(*s.cond, reachable);
            Work a = stmt(*s.then_s, reachable), b = stmt(*s.else_s, reachable);
            w.tuples = std::max(a.tuples, b.tuples);
            w.steps = sat(std::max(a.steps, b.steps) + 2);
            w.syncs = std::max(a.syncs, b.syncs);
            return w;
        }
        case SOp::ForU:
        case SOp::ForS: {
            bool d0 = false;
            Iv lo = expr(*s.lo, d0, reachable), hi = expr(*s.hi, d0, reachable);
            LoopInfo li;
            Iv v;
            if (!lo.empty() && !hi.empty()) { v.lo = lo.lo; v.hi = hi.hi - 1; }
            li.trip_max = v.empty() ? 0 : sat(hi.hi - lo.lo);
            var_[s.slot] = v;
            Work b = stmt(*s.body, reachable && !v.empty());
            li.body_steps = sat(b.steps + 1);
            li.body_tuples = b.tuples;
            loops[&s] = li;
            w.tuples = mul_sat(li.trip_max, b.tuples);
            w.steps = sat(1 + mul_sat(li.trip_max, li.body_steps));
            w.syncs = mul_sat(li.trip_max, b.syncs);
            return w;
        }
        }
        return w;
    }

private:
    uint32_t T_;
    const uint64_t *cells_;
    const int64_t *params_;
    std::vector<Iv> var_;

    void note(const Iv &v, bool reachable)
    {
        if (!reachable || v.empty()) return;
        if (v.lo < kI64Min || v.hi > kI64Max) risk = true;
        if (v.lo < kI32Min || v.hi > kI32Max) wide = true;
    }

    void cond(const Cond &c, bool reachable)
    {
        bool d0 = false;
        switch (c.op) {
        case COp::True: case COp::False: return;
        case COp::And: case COp::Or: cond(*c.l, reachable); cond(*c.r, reachable); return;
        case COp::Not: cond(*c.l, reachable); return;
        default: expr(*c.a, d0, reachable); expr(*c.b, d0, reachable); return;
        }
    }

    Iv expr(const Expr &e, bool &div0, bool reachable)
    {
        Iv r = expr_inner(e, div0, reachable);
        note(r, reachable);
        // once a value may leave int64 the protocol is rejected; clamping just
        // past that range keeps every later product inside 128 bits
        const i128 clamp = kI64Max + 2;
        if (!r.empty()) { r.lo = std::max(r.lo, -clamp); r.hi = std::min(r.hi, clamp); }
        ranges[&e] = r;
        return r;
    }

    Iv expr_inner(const Expr &e, bool &div0, bool reachable)
    {
        switch (e.op) {
        case EOp::Const: return Iv::point(e.value);
        case EOp::Tid: return Iv{0, (i128)T_ - 1};
        case EOp::Param: return Iv::point(params_[e.slot]);
        case EOp::Var: return var_[e.slot];
        case EOp::Neg: {
            Iv a = expr(*e.a, div0, reachable);
            if (a.empty()) return a;
            return Iv{-a.hi, -a.lo};
        }
        default: break;
        }
        Iv a = expr(*e.a, div0, reachable), b = expr(*e.b, div0, reachable);
        if (a.empty() || b.empty()) return Iv{};
        switch (e.op) {
        case EOp::Add: return Iv{a.lo + b.lo, a.hi + b.hi};
        case EOp::Sub: return Iv{a.lo - b.hi, a.hi - b.lo};
        case EOp::Mul: {
            i128 c[4] = {a.lo * b.lo, a.lo * b.hi, a.hi * b.lo, a.hi * b.hi};
            return Iv{*std::min_element(c, c + 4), *std::max_element(c, c + 4)};
        }
        case EOp::Min: return Iv{std::min(a.lo, b.lo), std::min(a.hi, b.hi)};
        case EOp::Max: return Iv{std::max(a.lo, b.lo), std::max(a.hi, b.hi)};
        case EOp::Div:
        case EOp::Mod: {
            if (b.lo <= 0 && b.hi >= 0) div0 = maybe_div0 = true;
            Iv parts[2] = {Iv{b.lo, std::min(b.hi, (i128)-1)}, Iv{std::max(b.lo, (i128)1), b.hi}};
            Iv r;
            bool any = false;
            for (const Iv &p : parts) {
                if (p.empty()) continue;
                Iv q;
                if (e.op == EOp::Div) {
                    // floor(a / b) is monotone in a, and in b on a sign-constant range
                    i128 c[4] = {floor_div(a.lo, p.lo), floor_div(a.lo, p.hi), floor_div(a.hi, p.lo),
                                 floor_div(a.hi, p.hi)};
                    q = Iv{*std::min_element(c, c + 4), *std::max_element(c, c + 4)};
                } else {
                    i128 m = std::max(p.lo < 0 ? -p.lo : p.lo, p.hi < 0 ? -p.hi : p.hi);
                    i128 mmin = std::min(p.lo < 0 ? -p.lo : p.lo, p.hi < 0 ? -p.hi : p.hi);
                    if (a.lo >= 0 && a.hi < mmin) q = a;        // already reduced
                    else q = Iv{0, m - 1};
                }
                if (!any) r = q;
                else r = Iv{std::min(r.lo, q.lo), std::max(r.hi, q.hi)};
                any = true;
            }
            return any ? r : Iv{};                        // divisor always zero
        }
        default: return Iv{};
        }
    }
};

// ------------------------------------------------------------------ lowering

struct Lowerer {
    const int64_t *params;
    const NodeMap<Expr, Iv> &ranges;
    const NodeMap<Stmt, bool> &count_eval;
    std::vector<Insn> insns;
    std::vector<uint64_t> xcode;
    std::vector<int> slot_reg;        // AST slot -> device register (nesting depth)
    int max_stack = 0;
    bool too_deep = false;

    // (register or kAffTid, coefficient) pairs of a linear form: at most one
    // per register and one for tid, kept inline (no allocation per node).
    struct Term {
        uint32_t first;               // register or kAffTid
        i128 second;                  // coefficient
    };
    struct Terms {
        uint32_t n = 0;
        Term v[kMaxVars + 1];         // the first n are set
        Terms() {}
        Terms(const Terms &o) : n(o.n) { std::copy(o.v, o.v + o.n, v); }
        Terms &operator=(const Terms &o) { n = o.n; std::copy(o.v, o.v + o.n, v); return *this; }
        Term *begin() { return v; }
        Term *end() { return v + n; }
        const Term *begin() const { return v; }
        const Term *end() const { return v + n; }
        bool empty() const { return n == 0; }
        size_t size() const { return n; }
        const Term &operator[](size_t i) const { return v[i]; }
        void push_back(const Term &t)
        {
            if (n > kMaxVars) throw std::length_error("linear form with too many terms");
            v[n++] = t;
        }
        void emplace_back(uint32_t reg, i128 c) { push_back(Term{reg, c}); }
    };

    // Folded form of an expression: a constant, or a linear combination of
    // tid / registers, or neither.
    struct Lin {
        bool ok = false;
        i128 c0 = 0;
        Terms terms;
    };

    static void add_term(Lin &l, uint32_t reg, i128 c)
    {
        for (auto &t : l.terms)
            if (t.first == reg) { t.second += c; return; }
        l.terms.emplace_back(reg, c);
    }

    Lin linear(const Expr &e)
    {
        Lin l;
        const i128 lim = (i128)1 << 62;
        switch (e.op) {
        case EOp::Const: l.ok = true; l.c0 = e.value; return l;
        case EOp::Param: l.ok = true; l.c0 = params[e.slot]; return l;
        case EOp::Tid: l.ok = true; add_term(l, kAffTid, 1); return l;
        case EOp::Var: l.ok = true; add_term(l, (uint32_t)slot_reg[e.slot], 1); return l;
        case EOp::Neg: {
            Lin a = linear(*e.a);
            if (!a.ok) return l;
            a.c0 = -a.c0;
            for (auto &t : a.terms) t.second = -t.second;
            return a;
        }
        case EOp::Add:
        case EOp::Sub: {
            Lin a = linear(*e.a), b = linear(*e.b);
            if (!a.ok || !b.ok) return l;
            i128 s = e.op == EOp::Add ? 1 : -1;
            a.c0 += s * b.c0;
            for (auto &t : b.terms) add_term(a, t.first, s * t.second);
            if (a.c0 > lim || a.c0 < -lim) return l;
            for (auto &t : a.terms) if (t.second > lim || t.second < -lim) return l;
            return a;
        }
        case EOp::Mul: {
            Lin a = linear(*e.a), b = linear(*e.b);
            if (!a.ok || !b.ok) return l;
            if (!a.terms.empty() && !b.terms.empty()) return l;       // not linear
            Lin &v = a.terms.empty() ? b : a;
            i128 k = a.terms.empty() ? a.c0 : b.c0;
            if (k > lim || k < -lim) return l;
            v.c0 *= k;
            for (auto &t : v.terms) t.second *= k;
            if (v.c0 > lim || v.c0 < -lim) return l;
            for (auto &t : v.terms) if (t.second > lim || t.second < -lim) return l;
            return v;
        }
        default: return l;
        }
    }

    void word(uint8_t op, int64_t arg = 0) { xcode.push_back((uint64_t)op | ((uint64_t)arg << 8)); }
    void lit(int64_t v) { xcode.push_back((uint64_t)v); }

    void emit_linear(const Lin &l)
    {
        Terms terms;
        for (auto &t : l.terms) if (t.second != 0) terms.push_back(t);
        if (terms.empty()) { word(X_CONST); lit((int64_t)l.c0); return; }
        if (terms.size() == 1 && terms[0].second == 1 && l.c0 == 0) {
            if (terms[0].first == kAffTid) word(X_TID);
            else word(X_VAR, terms[0].first);
            return;
        }
        word(X_AFF, (int64_t)terms.size());
        for (auto &t : terms) { lit(t.first); lit((int64_t)t.second); }
        lit((int64_t)l.c0);
    }

    // Emits code for e; depth is the stack height before it runs.
    void emit_expr(const Expr &e, int depth)
    {
        if (depth + 1 > max_stack) max_stack = depth + 1;
        Lin l = linear(e);
        if (l.ok) { emit_linear(l); return; }
        switch (e.op) {
        case EOp::Neg: emit_expr(*e.a, depth); word(X_NEG); return;
        case EOp::Div:
        case EOp::Mod: {
            Lin d = linear(*e.b);
            bool konst = d.ok && d.terms.empty() && d.c0 != 0;
            emit_expr(*e.a, depth);
            if (konst) {
                i128 m = d.c0;
                if (e.op == EOp::Mod && m > 0 && (m & (m - 1)) == 0) { word(X_MASK); lit((int64_t)(m - 1)); }
                else { word(e.op == EOp::Div ? X_DIVC : X_MODC); lit((int64_t)m); }
                return;
            }
            emit_expr(*e.b, depth + 1);
            word(e.op == EOp::Div ? X_DIV : X_MOD);
            return;
        }
        default: break;
        }
        emit_expr(*e.a, depth);
        emit_expr(*e.b, depth + 1);
        static const uint8_t code[] = {0, 0, 0, 0, X_ADD, X_SUB, X_MUL, 0, 0, X_MIN, X_MAX};
        word(code[(int)e.op]);
    }

    void emit_cond(const Cond &c, int depth)
    {
        if (depth + 1 > max_stack) max_stack = depth + 1;
        switch (c.op) {
        case COp::True: word(X_CONST); lit(1); return;
        case COp::False: word(X_CONST); lit(0); return;
        case COp::Not: emit_cond(*c.l, depth); word(X_NOT); return;
        case COp::And: case COp::Or:
            emit_cond(*c.l, depth); emit_cond(*c.r, depth + 1);
            word(c.op == COp::And ? X_AND : X_OR);
            return;
        default: break;
        }
        emit_expr(*c.a, depth);
        emit_expr(*c.b, depth + 1);
        static const uint8_t code[] = {0, 0, X_EQ, X_NE, X_LT, X_LE, X_GT, X_GE};
        word(code[(int)c.op]);
    }

    int32_t expr_code(const Expr &e)
    {
        int32_t off = (int32_t)xcode.size();
        emit_expr(e, 0);
        word(X_RET);
        return off;
    }

    int32_t cond_code(const Cond &c)
    {
        int32_t off = (int32_t)xcode.size();
        emit_cond(c, 0);
        word(X_RET);
        return off;
    }

    int32_t pc() const { return (int32_t)insns.size(); }

    int32_t emit(uint8_t op, uint8_t a = 0, uint16_t b = 0, int32_t c = 0, int32_t d = 0, int32_t e = 0)
    {
        insns.push_back(Insn{op, a, b, c, d, e});
        return pc() - 1;
    }

    NodeMap<Stmt, std::pair<int32_t, int32_t>> range;   // [begin, end) pcs
    NodeMap<Stmt, bool> fast;                           // loops lowered to I_FASTLOOP

    // An innermost loop whose body is only accesses (whose indices the count
    // pass need not evaluate) and syncs, each index linear in the variables
    // with at most a constant remainder or division on top, becomes one
    // I_FASTLOOP followed by its accesses.
    bool try_fast(const Stmt &s, int depth)
    {
        std::vector<const Stmt *> body;
        if (s.body->op == SOp::Seq) for (auto &it : s.body->items) body.push_back(it.get());
        else body.push_back(s.body.get());
        struct Acc { const Stmt *st; Lin rest; i128 coef; uint8_t post; i128 pconst; uint32_t phase_off; };
        std::vector<Acc> accs;
        uint32_t syncs = 0;
        const uint32_t reg = (uint32_t)depth;
        for (const Stmt *b : body) {
            if (b->op == SOp::Skip) continue;
            if (b->op == SOp::Sync) { if (++syncs > 255) return false; continue; }
            if (b->op != SOp::Access || count_eval.at(b)) return false;
            const Expr *e = b->index.get();
            uint8_t post = FP_NONE;
            i128 pc = 0;
            if (e->op == EOp::Mod || e->op == EOp::Div) {
                Lin d = linear(*e->b);
                if (!d.ok || !d.terms.empty() || d.c0 == 0) return false;
                if (e->op == EOp::Mod) {
                    if (d.c0 > 0 && (d.c0 & (d.c0 - 1)) == 0) { post = FP_MASK; pc = d.c0 - 1; }
                    else { post = FP_MOD; pc = d.c0; }
                } else {
                    post = FP_DIV; pc = d.c0;
                }
                e = e->a.get();
            }
            Lin l = linear(*e);
            if (!l.ok) return false;
            Acc a{b, Lin{}, 0, post, pc, syncs};
            a.rest.ok = true;
            a.rest.c0 = l.c0;
            for (auto &t : l.terms) {
                if (t.first == reg) a.coef += t.second;
                else a.rest.terms.push_back(t);
            }
            accs.push_back(a);
        }
        if (accs.empty() || accs.size() > kFastMax) return false;
        int32_t lo = expr_code(*s.lo), hi = expr_code(*s.hi);
        emit(I_FASTLOOP, (uint8_t)depth, (uint16_t)syncs, lo, hi, (int32_t)accs.size());
        for (const Acc &a : accs) {
            int32_t rest = (int32_t)xcode.size();
            if (max_stack < 1) max_stack = 1;
            emit_linear(a.rest);
            word(X_RET);
            int32_t consts = (int32_t)xcode.size();
            lit((int64_t)a.coef);
            lit((int64_t)a.pconst);
            uint8_t flags = (uint8_t)((a.st->write ? AF_WRITE : 0) | (a.post << 2));
            emit(I_FASTACC, flags, a.st->loc, rest, consts, (int32_t)a.phase_off);
        }
        fast[&s] = true;
        return true;
    }

    void stmt(const Stmt &s, int depth)
    {
        int32_t begin = pc();
        stmt_inner(s, depth);
        range[&s] = {begin, pc()};
    }

    void stmt_inner(const Stmt &s, int depth)
    {
        switch (s.op) {
        case SOp::Skip: return;
        case SOp::Sync: emit(I_SYNC); return;
        case SOp::Access: {
            uint8_t flags = (s.write ? AF_WRITE : 0) | (count_eval.at(&s) ? AF_EVAL_IN_COUNT : 0);
            emit(I_ACCESS, flags, s.loc, expr_code(*s.index));
            return;
        }
        case SOp::Seq:
            for (auto &it : s.items) stmt(*it, depth);
            return;
        case SOp::If: {
            int32_t ip = emit(I_IF, 0, 0, cond_code(*s.cond));
            stmt(*s.then_s, depth);
            bool has_else = !(s.else_s->op == SOp::Skip ||
                              (s.else_s->op == SOp::Seq && s.else_s->items.empty()));
            if (has_else) {
                int32_t jp = emit(I_JUMP);
                insns[ip].d = pc();
                stmt(*s.else_s, depth);
                insns[jp].c = pc();
            } else {
                insns[ip].d = pc();
            }
            return;
        }
        case SOp::ForU:
        case SOp::ForS: {
            if (depth >= kMaxVars) { too_deep = true; return; }
            slot_reg[s.slot] = depth;
            if (try_fast(s, depth)) return;
            int32_t lo = expr_code(*s.lo), hi = expr_code(*s.hi);
            int32_t lp = emit(I_LOOP, (uint8_t)depth, 0, lo, hi);
            int32_t body = pc();
            stmt(*s.body, depth + 1);
            int32_t ep = emit(I_ENDLOOP, (uint8_t)depth, 0, body);
            insns[lp].e = ep;
            return;
        }
        }
    }
};

// Cuts a statement list into items in program order.  A loop that deserves
// at least two items is split: into chunks of iterations when it deserves no
// more items than it has iterations, otherwise into single iterations whose
// bodies are cut recursively.  Consecutive statements that are not split form
// one "run" item.
struct Splitter {
    const Analyzer &an;
    const Lowerer &lw;
    std::vector<ItemDesc> &items;
    std::vector<uint64_t> &isteps;
    uint32_t split_pc[kMaxSplit] = {};
    uint32_t split_j[kMaxSplit] = {};
    int depth = 0;

    i128 max_item_tuples = 0;
    // With a constant sync structure (every forS bound the same for all
    // threads and iterations), the syncs a thread has executed when an item
    // starts -- the phase at the item's start -- is the same for every
    // thread: `phase` tracks it along the traversal, item_phase gets it per
    // item.  Meaningful only when the caller established that structure.
    i128 phase = 0;
    std::vector<uint64_t> item_phase;

    void push_item(uint32_t start, uint32_t stop, uint16_t chunked, uint32_t chunk, i128 steps, i128 tuples,
                   i128 at_phase)
    {
        item_phase.push_back((uint64_t)std::min<i128>(std::max<i128>(at_phase, 0), (i128)1 << 62));
        max_item_tuples = std::max(max_item_tuples, tuples);
        ItemDesc d{};
        d.start_pc = start;
        d.stop_pc = stop;
        d.nsplit = (uint16_t)depth;
        d.chunked = chunked;
        d.chunk = chunk;
        for (int l = 0; l < depth; l++) { d.split_pc[l] = split_pc[l]; d.j[l] = split_j[l]; }
        items.push_back(d);
        isteps.push_back((uint64_t)std::min<i128>(std::max<i128>(steps, 1), (i128)1 << 62));
    }

    void list(const Stmt &seq, i128 budget)
    {
        // the statements of the list (a sequence's items, else the statement itself)
        struct Stmts {
            const Stmt &s;
            struct It {
                const Stmt &s;
                size_t i;
                const Stmt *operator*() const { return s.op == SOp::Seq ? s.items[i].get() : &s; }
                It &operator++() { i++; return *this; }
                bool operator!=(const It &o) const { return i != o.i; }
            };
            It begin() const { return It{s, 0}; }
            It end() const { return It{s, s.op == SOp::Seq ? s.items.size() : 1}; }
        } xs{seq};
        i128 total = 0;
        for (const Stmt *x : xs) total = sat(total + an.work.at(x).steps);
        int32_t run_b = -1, run_e = -1;
        i128 run_steps = 0, run_tuples = 0, run_phase = 0;
        auto flush = [&] {
            if (run_b >= 0 && run_e > run_b)
                push_item((uint32_t)run_b, (uint32_t)run_e, 0, 1, run_steps, run_tuples, run_phase);
            run_b = -1; run_steps = 0; run_tuples = 0;
        };
        for (const Stmt *x : xs) {
            auto r = lw.range.at(x);
            const i128 x_phase = phase, x_syncs = an.work.at(x).syncs;
            phase = sat(phase + x_syncs);                            // the phase after x
            if (r.first == r.second) continue;                       // no code (skip)
            i128 steps = an.work.at(x).steps;
            i128 ks = total > 0 ? div_ceil(budget * steps, total) : 1;
            bool loop = x->op == SOp::ForU || x->op == SOp::ForS;
            const LoopInfo *li = loop ? &an.loops.at(x) : nullptr;
            if (!loop || ks < 2 || depth >= kMaxSplit || li->trip_max < 1 || li->trip_max > (i128)UINT32_MAX) {
                if (run_b < 0) { run_b = r.first; run_phase = x_phase; }
                run_e = r.second;
                run_steps = sat(run_steps + steps);
                run_tuples = sat(run_tuples + an.work.at(x).tuples);
                continue;
            }
            flush();
            const i128 m = li->trip_max;
            const uint32_t loop_pc = (uint32_t)r.first, end_pc = (uint32_t)r.second;   // ENDLOOP is end_pc - 1
            split_pc[depth] = loop_pc;
            const bool is_fast = lw.fast.count(x) != 0;
            const i128 body_syncs = an.work.at(x->body.get()).syncs;
            if (ks <= m || depth + 1 >= kMaxSplit || is_fast) {
                // chunks of iterations (a fast loop starts at its own instruction)
                i128 parts = std::min(ks, m);
                i128 chunk = div_ceil(m, parts);
                i128 nch = div_ceil(m, chunk);
                for (i128 c = 0; c < nch; c++) {
                    split_j[depth] = (uint32_t)c;
                    depth++;
                    push_item(is_fast ? loop_pc : loop_pc + 1, end_pc, is_fast ? 2 : 1, (uint32_t)chunk,
                              mul_sat(chunk, li->body_steps), mul_sat(chunk, li->body_tuples),
                              sat(x_phase + mul_sat(mul_sat(c, chunk), body_syncs)));
                    depth--;
                }
            } else {
                i128 sub = div_ceil(ks, m);
                const i128 after = phase;
                for (i128 j = 0; j < m; j++) {
                    split_j[depth] = (uint32_t)j;
                    depth++;
                    phase = sat(x_phase + mul_sat(j, body_syncs));
                    list(*x->body, sub);
                    depth--;
                }
                phase = after;
            }
        }
        flush();
    }
};

// Finds the accesses of a protocol with static phases that the range pass
// can apply (RangeAccess): walks the statements in program order keeping the
// phase (the syncs every thread has run), the enclosing loops and the
// enclosing conditions.
struct RangeFinder {
    const Analyzer &an;
    Lowerer &lw;
    uint32_t T;
    std::vector<RangeLoop> loops;
    std::vector<std::pair<int32_t, bool>> guards;
    std::vector<RangeAccess> out;

    static bool has_tid(const Expr &e)
    {
        if (e.op == EOp::Tid) return true;
        return (e.a && has_tid(*e.a)) || (e.b && has_tid(*e.b));
    }

    static bool cond_has_tid(const Cond &c)
    {
        if ((c.a && has_tid(*c.a)) || (c.b && has_tid(*c.b))) return true;
        return (c.l && cond_has_tid(*c.l)) || (c.r && cond_has_tid(*c.r));
    }

    // The coefficient of tid when e is tid times it plus a part without tid
    // (tid only under sums, differences, negations and products by
    // constants); false otherwise.
    bool tid_coef(const Expr &e, i128 &k)
    {
        if (!has_tid(e)) { k = 0; return true; }
        switch (e.op) {
        case EOp::Tid: k = 1; return true;
        case EOp::Neg: if (!tid_coef(*e.a, k)) return false; k = -k; return true;
        case EOp::Add: case EOp::Sub: {
            i128 a, b;
            if (!tid_coef(*e.a, a) || !tid_coef(*e.b, b)) return false;
            k = e.op == EOp::Add ? a + b : a - b;
            return k < ((i128)1 << 62) && k > -((i128)1 << 62);
        }
        case EOp::Mul: {
            const bool ta = has_tid(*e.a);
            Lowerer::Lin c = lw.linear(ta ? *e.b : *e.a);
            if (!c.ok || !c.terms.empty()) return false;
            i128 x;
            if (!tid_coef(ta ? *e.a : *e.b, x)) return false;
            k = x * c.c0;
            return k < ((i128)1 << 62) && k > -((i128)1 << 62);
        }
        default: return false;
        }
    }

    // A copy of e with tid replaced by 0.
    static ExprP at_tid_zero(const Expr &e)
    {
        auto r = std::make_unique<Expr>();
        if (e.op == EOp::Tid) { r->op = EOp::Const; r->value = 0; return r; }
        r->op = e.op;
        r->value = e.value;
        r->slot = e.slot;
        if (e.a) r->a = at_tid_zero(*e.a);
        if (e.b) r->b = at_tid_zero(*e.b);
        return r;
    }

    void access(const Stmt &s, uint32_t pc, i128 phase)
    {
        if (guards.size() > 8 || loops.size() > 8 || phase >= ((i128)1 << 31)) return;
        const Expr *e = s.index.get();
        uint64_t modn = 0;
        if (e->op == EOp::Mod) {
            Lowerer::Lin d = lw.linear(*e->b);
            if (!d.ok || !d.terms.empty() || d.c0 <= 0 || d.c0 >= ((i128)1 << 62)) return;
            modn = (uint64_t)d.c0;
            e = e->a.get();
        }
        i128 k = 0;
        if (!tid_coef(*e, k) || k > kRangeMaxSigma || k < -kRangeMaxSigma) return;
        // with a remainder, the index wraps around it at most kRangeMaxWraps
        // times over the threads (a run of consecutive tids per wrap)
        if (modn && (i128)(T ? T - 1 : 0) * (k < 0 ? -k : k) >= (i128)modn * kRangeMaxWraps) return;
        RangeAccess r;
        r.pc = pc;
        r.phase = (uint32_t)phase;
        r.loc = s.loc;
        r.write = s.write;
        r.sigma = (int32_t)k;
        r.modn = modn;
        ExprP c0 = at_tid_zero(*e);
        r.cexpr = lw.expr_code(*c0);
        r.loops = loops;
        r.guards = guards;
        i128 it = 1;
        for (const RangeLoop &l : loops) it = mul_sat(it, (i128)l.trip_max);
        r.iters = it > ((i128)1 << 62) ? (1ull << 62) : (uint64_t)it;
        out.push_back(std::move(r));
    }

    // Returns the phase after s; `ok`: s's accesses may still qualify.
    i128 walk(const Stmt &s, i128 phase, bool ok)
    {
        switch (s.op) {
        case SOp::Skip: return phase;
        case SOp::Sync: return phase + 1;
        case SOp::Access:
            if (ok) access(s, (uint32_t)lw.range.at(&s).first, phase);
            return phase;
        case SOp::Seq:
            for (auto &it : s.items) phase = walk(*it, phase, ok);
            return phase;
        case SOp::If: {
            const int32_t c = lw.insns.at((size_t)lw.range.at(&s).first).c;
            const bool gok = ok && !cond_has_tid(*s.cond);
            guards.emplace_back(c, true);
            walk(*s.then_s, phase, gok);
            guards.back().second = false;
            walk(*s.else_s, phase, gok);
            guards.pop_back();
            return phase + an.work.at(&s).syncs;    // (no sync inside an if)
        }
        case SOp::ForU:
        case SOp::ForS: {
            const i128 after = phase + an.work.at(&s).syncs;
            const bool in_one_phase = an.work.at(s.body.get()).syncs == 0;
            const bool bok = ok && in_one_phase && !has_tid(*s.lo) && !has_tid(*s.hi) && an.loops.at(&s).trip_max > 0;
            const uint32_t lpc = (uint32_t)lw.range.at(&s).first;
            const Insn &L = lw.insns.at(lpc);
            loops.push_back(RangeLoop{L.a, L.c, L.d, (uint64_t)std::min<i128>(an.loops.at(&s).trip_max, (i128)1 << 40)});
            if (lw.fast.count(&s)) {
                // a fast loop: its accesses follow its instruction in body order
                uint32_t j = 0;
                std::vector<const Stmt *> body;
                if (s.body->op == SOp::Seq) for (auto &it : s.body->items) body.push_back(it.get());
                else body.push_back(s.body.get());
                for (const Stmt *b : body)
                    if (b->op == SOp::Access) {
                        if (bok) access(*b, lpc + 1 + j, phase);
                        j++;
                    }
            } else {
                walk(*s.body, phase, bok);
            }
            loops.pop_back();
            return after;
        }
        }
        return phase;
    }
};

}  // namespace

// Evaluates expression code (devprog.h's stack machine) on the host, with
// tid and the loop variables `vars`, on mathematical integers: false on a
// division or remainder by zero, a value outside int64 or malformed code.
bool host_eval(const std::vector<uint64_t> &xc, int32_t off, int64_t tid, const int64_t *vars, int64_t &out)
{
    using i128 = __int128;
    i128 st[kMaxStack + 2];
    int d = 0;
    auto fits = [](i128 v) { return v >= (i128)INT64_MIN && v <= (i128)INT64_MAX; };
    auto fdiv = [](i128 a, i128 b) { i128 q = a / b; if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1; return q; };
    auto emod = [](i128 a, i128 b) { i128 r = a % b; if (r < 0) r += b < 0 ? -b : b; return r; };
    size_t i = (size_t)off;
    for (int guard = 0; guard < 1 << 16; guard++) {
        if (i >= xc.size()) return false;
        const uint64_t w = xc[i++];
        const uint32_t op = (uint32_t)(w & 0xff);
        if (op != X_RET && d >= kMaxStack + 1) return false;
        switch (op) {
        case X_RET:
            if (d != 1 || !fits(st[0])) return false;
            out = (int64_t)st[0];
            return true;
        case X_CONST: if (i >= xc.size()) return false; st[d++] = (int64_t)xc[i++]; break;
        case X_TID: st[d++] = tid; break;
        case X_VAR: if ((w >> 8) >= (uint64_t)kMaxVars) return false; st[d++] = vars[w >> 8]; break;
        case X_AFF: {
            const uint32_t n = (uint32_t)(w >> 8);
            i128 acc = 0;
            for (uint32_t t = 0; t < n; t++) {
                if (i + 1 >= xc.size()) return false;
                const uint32_t reg = (uint32_t)xc[i++];
                const int64_t coef = (int64_t)xc[i++];
                if (reg != kAffTid && reg >= (uint32_t)kMaxVars) return false;
                acc += (i128)coef * (reg == kAffTid ? tid : vars[reg]);
                if (!fits(acc)) return false;
            }
            if (i >= xc.size()) return false;
            acc += (int64_t)xc[i++];
            st[d++] = acc;
            break;
        }
        case X_NEG: if (d < 1) return false; st[d - 1] = -st[d - 1]; break;
        case X_NOT: if (d < 1) return false; st[d - 1] = st[d - 1] == 0; break;
        case X_DIVC: case X_MODC: case X_MASK: {
            if (d < 1 || i >= xc.size()) return false;
            const int64_t c = (int64_t)xc[i++];
            if (op == X_MASK) st[d - 1] = (i128)(int64_t)((uint64_t)(int64_t)st[d - 1] & (uint64_t)c);
            else if (c == 0) return false;
            else st[d - 1] = op == X_DIVC ? fdiv(st[d - 1], c) : emod(st[d - 1], c);
            break;
        }
        default: {
            if (d < 2) return false;
            const i128 a = st[d - 2], b = st[d - 1];
            i128 r = 0;
            switch (op) {
            case X_ADD: r = a + b; break;
            case X_SUB: r = a - b; break;
            case X_MUL: if (!fits(a) || !fits(b)) return false; r = a * b; break;
            case X_MIN: r = b < a ? b : a; break;
            case X_MAX: r = b > a ? b : a; break;
            case X_DIV: if (b == 0) return false; r = fdiv(a, b); break;
            case X_MOD: if (b == 0) return false; r = emod(a, b); break;
            case X_EQ: r = a == b; break;
            case X_NE: r = a != b; break;
            case X_LT: r = a < b; break;
            case X_LE: r = a <= b; break;
            case X_GT: r = a > b; break;
            case X_GE: r = a >= b; break;
            case X_AND: r = (a != 0) & (b != 0); break;
            case X_OR: r = (a != 0) | (b != 0); break;
            default: return false;
            }
            if (!fits(r)) return false;
            d--;
            st[d - 1] = r;
        }
        }
    }
    return false;
}

// The distinct offsets c of a range access over its loops' iterations (the
// conditions applied), and how many iterations it runs; false when an
// evaluation fails or more than `cap` iterations would be visited.
bool range_offsets(const std::vector<uint64_t> &xcode, const RangeAccess &r, uint64_t cap, std::vector<int64_t> &cs,
                   uint64_t &iters)
{
    int64_t vars[kMaxVars] = {};
    uint64_t visited = 0;
    iters = 0;
    cs.clear();
    bool ok = true;
    std::function<void(size_t)> rec = [&](size_t l) {
        if (!ok) return;
        if (l == r.loops.size()) {
            for (const auto &g : r.guards) {
                int64_t c = 0;
                if (!host_eval(xcode, g.first, 0, vars, c)) { ok = false; return; }
                if ((c != 0) != g.second) return;
            }
            int64_t c = 0;
            if (!host_eval(xcode, r.cexpr, 0, vars, c)) { ok = false; return; }
            if (r.modn) {
                c %= (int64_t)r.modn;
                if (c < 0) c += (int64_t)r.modn;
            }
            cs.push_back(c);
            iters++;
            return;
        }
        const RangeLoop &L = r.loops[l];
        int64_t lo = 0, hi = 0;
        if (L.reg >= (uint32_t)kMaxVars || !host_eval(xcode, L.lo, 0, vars, lo) || !host_eval(xcode, L.hi, 0, vars, hi)) {
            ok = false;
            return;
        }
        for (int64_t x = lo; x < hi && ok; x++) {
            if (++visited > cap) { ok = false; return; }
            vars[L.reg] = x;
            rec(l + 1);
        }
    };
    rec(0);
    if (!ok) return false;
    std::sort(cs.begin(), cs.end());
    cs.erase(std::unique(cs.begin(), cs.end()), cs.end());
    return true;
}

Error prepare(const uint8_t *bc, size_t len, uint32_t nthreads, uint32_t nlocs, const uint64_t *cells,
              uint32_t nparams, const int64_t *params, const PrepareOpts &opts, Prepared &out)
{
    Protocol p;
    Error err = decode_bytecode(bc, len, p);
    if (!err.ok()) return err;
    if (nlocs != p.narrays || nparams != p.nparams)
        return Error::make(S_INVALID_ARG, "bounds give " + std::to_string(nlocs) + " arrays and " +
                                              std::to_string(nparams) + " params; the protocol declares " +
                                              std::to_string(p.narrays) + " and " + std::to_string(p.nparams));
    if ((nlocs && !cells) || (nparams && !params)) return Error::make(S_INVALID_ARG, "null array sizes or params");
    if (nthreads > (1u << 27)) return Error::make(S_LIMIT, "more than 2^27 threads");

    out = Prepared{};
    out.nthreads = nthreads;
    out.narrays = nlocs;
    out.cells.assign(cells, cells + nlocs);

    Analyzer an(nthreads ? nthreads : 1, cells, params, p.nslots);
    Work w = an.stmt(*p.body, nthreads > 0);
    if (an.risk) return Error::make(S_OVERFLOW_RISK, "an intermediate value may leave the 64-bit range");
    if (w.syncs >= ((i128)1 << 32)) return Error::make(S_LIMIT, "more than 2^32 syncs per thread");
    if ((i128)nthreads * w.tuples > (i128)kMaxTupleBound)
        return Error::make(S_LIMIT, "the protocol may make more than 2^36 accesses");
    if ((i128)nthreads * w.steps > (i128)kMaxStepBound)
        return Error::make(S_LIMIT, "the protocol may run more than 2^42 steps");
    out.wide = an.wide;
    out.max_syncs = (uint64_t)w.syncs;
    out.max_tuples = (uint64_t)w.tuples;
    out.max_steps = (uint64_t)w.steps;

    Lowerer lw{params, an.ranges, an.count_eval};
    lw.slot_reg.assign(p.nslots, 0);

    lw.stmt(*p.body, 0);
    if (lw.too_deep) return Error::make(S_LIMIT, "loops nested more than 16 deep");
    if (lw.max_stack > kMaxStack) return Error::make(S_LIMIT, "expression needs more than 16 stack slots");
    lw.emit(I_END);
    if (lw.insns.size() > (1u << 24) || lw.xcode.size() > (1u << 26)) return Error::make(S_LIMIT, "protocol too large");

    // --- work decomposition: how many items each thread is cut into
    i128 total = std::max<i128>(1, w.steps);
    uint64_t groups = nthreads ? (nthreads + 31) / 32 : 1;
    i128 k_want = std::max<i128>(1, ((i128)opts.desired_warp_items + groups - 1) / groups);
    i128 k_work = std::max<i128>(1, total / std::max<uint64_t>(1, opts.min_item_steps));
    // a small protocol is still cut into enough items for about a sixteenth
    // of the desired warp items (one wave of warps for a lone check), even
    // when that makes its items short: its time is the chain of dependent
    // steps one lane runs, not the steps' total
    const i128 k_floor = std::min<i128>(((i128)opts.desired_warp_items / 16 + groups - 1) / groups,
                                        total / std::max<uint64_t>(1, opts.min_short_item_steps));
    i128 K = std::min<i128>(std::min(k_want, std::max(k_work, k_floor)), opts.max_items);
    if ((i128)K * nthreads > ((i128)1 << 27)) K = std::max<i128>(1, ((i128)1 << 27) / std::max<uint32_t>(1, nthreads));

    std::vector<ItemDesc> items;
    std::vector<uint64_t> isteps, iphase;
    for (int attempt = 0; attempt < 16; attempt++) {
        items.clear();
        isteps.clear();
        Splitter sp{an, lw, items, isteps};
        sp.list(*p.body, K);
        iphase = sp.item_phase;
        if (sp.max_item_tuples >= ((i128)1 << 32))
            return Error::make(S_LIMIT, "a work item may make 2^32 accesses or more");
        if (items.size() <= opts.max_items || K <= 1) break;
        K = std::max<i128>(1, K / 2);                          // too fine: coarsen
    }
    if (items.empty()) {
        ItemDesc d{};
        items.push_back(d);                                    // nothing to run
        isteps.push_back(1);
        iphase.assign(1, 0);
    }
    if ((i128)items.size() * nthreads > ((i128)1 << 28)) return Error::make(S_LIMIT, "too many work items");

    // Static phases: every forS bound is one value for all threads and
    // iterations (the analysis's range of each is a single point), so the
    // sync structure, and with it the phase at each item's start, is the
    // same for every thread; and no evaluation can fail (every index is
    // proven in range, no divisor may be zero).  Then the per-thread sync
    // counts all agree (no barrier divergence) and the count and scan passes
    // have nothing to add: the specialized kernels take the phases as
    // constants.
    bool constant_syncs = true;
    std::vector<const Stmt *> todo{p.body.get()};
    while (!todo.empty() && constant_syncs) {
        const Stmt *t = todo.back();
        todo.pop_back();
        if (t->op == SOp::ForS) {
            const Iv &lo = an.ranges.at(t->lo.get()), &hi = an.ranges.at(t->hi.get());
            if (lo.empty() || hi.empty() || lo.lo != lo.hi || hi.lo != hi.hi) constant_syncs = false;
        }
        for (auto &it : t->items) todo.push_back(it.get());
        if (t->body) todo.push_back(t->body.get());
        if (t->then_s) todo.push_back(t->then_s.get());
        if (t->else_s) todo.push_back(t->else_s.get());
    }
    bool may_fail = an.maybe_div0;
    may_fail = may_fail || an.any_count_eval;
    out.static_phases = constant_syncs && !may_fail && iphase.size() == items.size();
    for (uint64_t ph : iphase) if (ph > w.syncs) out.static_phases = false;
    if (out.static_phases) out.item_phase.assign(iphase.begin(), iphase.end());
    if (out.static_phases && nthreads > 0) {
        RangeFinder rf{an, lw, nthreads};
        rf.walk(*p.body, 0, true);
        if (lw.xcode.size() > (1u << 26)) return Error::make(S_LIMIT, "protocol too large");
        // the distinct offsets of each, by evaluating its loops (at most
        // kRangeIterCap iterations over all of them; the rest are left to
        // the table pass)
        uint64_t budget = kRangeIterCap;
        for (RangeAccess &r : rf.out) {
            uint64_t iters = 0;
            if (!range_offsets(lw.xcode, r, budget, r.offsets, iters) || iters == 0) continue;
            budget -= std::min<uint64_t>(budget, iters);
            r.run_iters = iters;
            out.range_access.push_back(std::move(r));
        }
    }

    out.insns = std::move(lw.insns);
    out.xcode = std::move(lw.xcode);
    out.items = std::move(items);
    out.item_steps = std::move(isteps);
    return Error{};
}

}  // namespace drf
