// Portable protocol bytecode ("DRFB", version 1): the wire format of the C
// ABI.  Little-endian; a 16-byte header followed by the statement tree in
// prefix order.
//
//   header : 'D' 'R' 'F' 'B' | u16 version=1 | u16 flags=0 | u16 narrays |
//            u16 nparams | u16 nslots | u16 reserved=0
//   stmt   : 0x01 skip | 0x02 sync | 0x03 u8 mode(1=wr) u16 loc expr
//          | 0x04 u32 count stmt*count | 0x05 cond stmt stmt
//          | 0x06 forU u16 slot expr(lo) expr(hi) stmt
//          | 0x07 forS u16 slot expr(lo) expr(hi) stmt
//   expr   : 0x20 i64 const | 0x21 tid | 0x22 u16 slot | 0x23 u16 param
//          | 0x24..0x2A (+ - * / % min max) expr expr | 0x2B neg expr
//   cond   : 0x40 true | 0x41 false | 0x42..0x47 (= != < <= > >=) expr expr
//          | 0x48 and cond cond | 0x49 or cond cond | 0x4A not cond
//
// The decoder re-checks every rule the text parser enforces, because a
// caller may build bytecode by other means: loop variables must be bound by
// an enclosing loop and never rebound (rules t-n, t-b, t-for of Fig. 4),
// sync / forS only in the synchronized fragment (Fig. 1), arrays and
// parameters in range, nesting within the implementation's limits, and no
// trailing or missing bytes.
#include <cstring>

#include "ast.h"

namespace drf {
namespace {

enum : uint8_t {
    B_SKIP = 0x01, B_SYNC = 0x02, B_ACCESS = 0x03, B_SEQ = 0x04, B_IF = 0x05, B_FORU = 0x06, B_FORS = 0x07,
    B_CONST = 0x20, B_TID = 0x21, B_VAR = 0x22, B_PARAM = 0x23, B_ADD = 0x24, B_SUB = 0x25, B_MUL = 0x26,
    B_DIV = 0x27, B_MOD = 0x28, B_MIN = 0x29, B_MAX = 0x2A, B_NEG = 0x2B,
    B_TRUE = 0x40, B_FALSE = 0x41, B_EQ = 0x42, B_NE = 0x43, B_LT = 0x44, B_LE = 0x45, B_GT = 0x46,
    B_GE = 0x47, B_AND = 0x48, B_OR = 0x49, B_NOT = 0x4A,
};

struct Writer {
    std::vector<uint8_t> out;
    void u8(uint8_t v) { out.push_back(v); }
    void u16(uint16_t v) { u8((uint8_t)v); u8((uint8_t)(v >> 8)); }
    void u32(uint32_t v) { for (int i = 0; i < 4; i++) u8((uint8_t)(v >> (8 * i))); }
    void i64(int64_t v) { for (int i = 0; i < 8; i++) u8((uint8_t)((uint64_t)v >> (8 * i))); }

    void expr(const Expr &e)
    {
        switch (e.op) {
        case EOp::Const: u8(B_CONST); i64(e.value); return;
        case EOp::Tid: u8(B_TID); return;
        case EOp::Var: u8(B_VAR); u16(e.slot); return;
        case EOp::Param: u8(B_PARAM); u16(e.slot); return;
        case EOp::Neg: u8(B_NEG); expr(*e.a); return;
        default: break;
        }
        static const uint8_t code[] = {0, 0, 0, 0, B_ADD, B_SUB, B_MUL, B_DIV, B_MOD, B_MIN, B_MAX};
        u8(code[(int)e.op]);
        expr(*e.a);
        expr(*e.b);
    }

    void cond(const Cond &c)
    {
        switch (c.op) {
        case COp::True: u8(B_TRUE); return;
        case COp::False: u8(B_FALSE); return;
        case COp::And: u8(B_AND); cond(*c.l); cond(*c.r); return;
        case COp::Or: u8(B_OR); cond(*c.l); cond(*c.r); return;
        case COp::Not: u8(B_NOT); cond(*c.l); return;
        default: break;
        }
        static const uint8_t code[] = {0, 0, B_EQ, B_NE, B_LT, B_LE, B_GT, B_GE};
        u8(code[(int)c.op]);
        expr(*c.a);
        expr(*c.b);
    }

    void stmt(const Stmt &s)
    {
        switch (s.op) {
        case SOp::Skip: u8(B_SKIP); return;
        case SOp::Sync: u8(B_SYNC); return;
        case SOp::Access: u8(B_ACCESS); u8(s.write ? 1 : 0); u16(s.loc); expr(*s.index); return;
        case SOp::Seq:
            u8(B_SEQ); u32((uint32_t)s.items.size());
            for (auto &it : s.items) stmt(*it);
            return;
        case SOp::If: u8(B_IF); cond(*s.cond); stmt(*s.then_s); stmt(*s.else_s); return;
        case SOp::ForU:
        case SOp::ForS:
            u8(s.op == SOp::ForU ? B_FORU : B_FORS); u16(s.slot);
            expr(*s.lo); expr(*s.hi); stmt(*s.body);
            return;
        }
    }
};

struct Reader {
    const uint8_t *p;
    size_t n, pos = 0;
    uint16_t narrays = 0, nparams = 0, nslots = 0;
    std::vector<uint8_t> bound;       // slot -> currently in scope
    std::vector<uint8_t> used;        // slot -> binder seen already
    int loops = 0, depth = 0;
    Error err;

    bool fail(int status, const char *msg)
    {
        if (err.ok()) err = Error::make(status, std::string("bytecode offset ") + std::to_string(pos) + ": " + msg);
        return false;
    }
    bool need(size_t k) { return pos + k <= n ? true : fail(S_INVALID_BYTECODE, "truncated"); }
    bool u8(uint8_t &v) { if (!need(1)) return false; v = p[pos++]; return true; }
    bool u16(uint16_t &v) { if (!need(2)) return false; v = (uint16_t)(p[pos] | (p[pos + 1] << 8)); pos += 2; return true; }
    bool u32(uint32_t &v)
    {
        if (!need(4)) return false;
        v = 0;
        for (int i = 0; i < 4; i++) v |= (uint32_t)p[pos + i] << (8 * i);
        pos += 4;
        return true;
    }
    bool i64(int64_t &v)
    {
        if (!need(8)) return false;
        uint64_t u = 0;
        for (int i = 0; i < 8; i++) u |= (uint64_t)p[pos + i] << (8 * i);
        pos += 8;
        v = (int64_t)u;
        return true;
    }

    bool expr(ExprP &out, int d)
    {
        if (d > kMaxExprDepth) return fail(S_LIMIT, "expression nested too deeply");
        uint8_t op;
        if (!u8(op)) return false;
        out.reset(new Expr);
        Expr &e = *out;
        switch (op) {
        case B_CONST: e.op = EOp::Const; return i64(e.value);
        case B_TID: e.op = EOp::Tid; return true;
        case B_VAR:
            e.op = EOp::Var;
            if (!u16(e.slot)) return false;
            if (e.slot >= nslots || !bound[e.slot]) return fail(S_UNBOUND_VAR, "variable not bound by an enclosing loop");
            return true;
        case B_PARAM:
            e.op = EOp::Param;
            if (!u16(e.slot)) return false;
            if (e.slot >= nparams) return fail(S_UNBOUND_VAR, "parameter out of range");
            return true;
        case B_NEG: e.op = EOp::Neg; return expr(e.a, d + 1);
        case B_ADD: case B_SUB: case B_MUL: case B_DIV: case B_MOD: case B_MIN: case B_MAX: {
            static const EOp m[] = {EOp::Add, EOp::Sub, EOp::Mul, EOp::Div, EOp::Mod, EOp::Min, EOp::Max};
            e.op = m[op - B_ADD];
            return expr(e.a, d + 1) && expr(e.b, d + 1);
        }
        default: return fail(S_INVALID_BYTECODE, "bad expression opcode");
        }
    }

    bool cond(CondP &out, int d)
    {
        if (d > kMaxExprDepth) return fail(S_LIMIT, "condition nested too deeply");
        uint8_t op;
        if (!u8(op)) return false;
        out.reset(new Cond);
        Cond &c = *out;
        switch (op) {
        case B_TRUE: c.op = COp::True; return true;
        case B_FALSE: c.op = COp::False; return true;
        case B_AND: c.op = COp::And; return cond(c.l, d + 1) && cond(c.r, d + 1);
        case B_OR: c.op = COp::Or; return cond(c.l, d + 1) && cond(c.r, d + 1);
        case B_NOT: c.op = COp::Not; return cond(c.l, d + 1);
        case B_EQ: case B_NE: case B_LT: case B_LE: case B_GT: case B_GE: {
            static const COp m[] = {COp::Eq, COp::Ne, COp::Lt, COp::Le, COp::Gt, COp::Ge};
            c.op = m[op - B_EQ];
            return expr(c.a, d + 1) && expr(c.b, d + 1);
        }
        default: return fail(S_INVALID_BYTECODE, "bad condition opcode");
        }
    }

    bool stmt(StmtP &out, bool synced)
    {
        if (++depth > kMaxStmtDepth) return fail(S_LIMIT, "statements nested too deeply");
        uint8_t op;
        if (!u8(op)) return false;
        out.reset(new Stmt);
        Stmt &s = *out;
        bool ok = true;
        switch (op) {
        case B_SKIP: s.op = SOp::Skip; break;
        case B_SYNC:
            s.op = SOp::Sync;
            if (!synced) return fail(S_SYNC_IN_UNSYNC, "sync inside an unsynchronized fragment");
            break;
        case B_ACCESS: {
            s.op = SOp::Access;
            uint8_t mode;
            if (!u8(mode) || !u16(s.loc)) return false;
            if (mode > 1) return fail(S_INVALID_BYTECODE, "bad access mode");
            if (s.loc >= narrays) return fail(S_UNKNOWN_ARRAY, "array out of range");
            s.write = mode == 1;
            ok = expr(s.index, 0);
            break;
        }
        case B_SEQ: {
            s.op = SOp::Seq;
            uint32_t count;
            if (!u32(count)) return false;
            if (count > n - pos) return fail(S_INVALID_BYTECODE, "sequence longer than the buffer");
            s.items.resize(count);
            for (uint32_t i = 0; i < count && ok; i++) ok = stmt(s.items[i], synced);
            break;
        }
        case B_IF:
            s.op = SOp::If;
            ok = cond(s.cond, 0) && stmt(s.then_s, false) && stmt(s.else_s, false);
            break;
        case B_FORU:
        case B_FORS: {
            s.op = op == B_FORU ? SOp::ForU : SOp::ForS;
            if (s.op == SOp::ForS && !synced) return fail(S_SYNC_IN_UNSYNC, "forS inside an unsynchronized fragment");
            if (!u16(s.slot)) return false;
            if (s.slot >= nslots) return fail(S_INVALID_BYTECODE, "loop slot out of range");
            if (used[s.slot]) return fail(S_REBIND, "loop variable slot bound twice");
            if (!expr(s.lo, 0) || !expr(s.hi, 0)) return false;
            if (++loops > kMaxLoopDepth) return fail(S_LIMIT, "loops nested too deeply");
            used[s.slot] = 1;
            bound[s.slot] = 1;
            ok = stmt(s.body, s.op == SOp::ForS);
            bound[s.slot] = 0;
            loops--;
            break;
        }
        default: return fail(S_INVALID_BYTECODE, "bad statement opcode");
        }
        depth--;
        return ok;
    }
};

}  // namespace

std::vector<uint8_t> encode_bytecode(const Protocol &p)
{
    Writer w;
    w.u8('D'); w.u8('R'); w.u8('F'); w.u8('B');
    w.u16(1); w.u16(0);
    w.u16(p.narrays); w.u16(p.nparams); w.u16(p.nslots); w.u16(0);
    w.stmt(*p.body);
    return w.out;
}

Error decode_bytecode(const uint8_t *data, size_t len, Protocol &out)
{
    if (!data || len < 16) return Error::make(S_INVALID_BYTECODE, "bytecode shorter than its header");
    if (std::memcmp(data, "DRFB", 4) != 0) return Error::make(S_INVALID_BYTECODE, "bad magic");
    Reader r{data, len};
    r.pos = 4;
    uint16_t version, flags, reserved;
    r.u16(version); r.u16(flags);
    r.u16(r.narrays); r.u16(r.nparams); r.u16(r.nslots); r.u16(reserved);
    if (version != 1 || flags != 0 || reserved != 0) return Error::make(S_INVALID_BYTECODE, "unsupported version or flags");
    r.bound.assign(r.nslots, 0);
    r.used.assign(r.nslots, 0);
    Protocol p;
    p.narrays = r.narrays; p.nparams = r.nparams; p.nslots = r.nslots;
    if (!r.stmt(p.body, true)) return r.err;
    if (r.pos != len) return Error::make(S_INVALID_BYTECODE, "trailing bytes after the protocol");
    if (p.body->op != SOp::Seq) {               // the top level is always a sequence
        StmtP seq(new Stmt);
        seq->op = SOp::Seq;
        seq->items.push_back(std::move(p.body));
        p.body = std::move(seq);
    }
    out = std::move(p);
    return Error{};
}

}  // namespace drf
