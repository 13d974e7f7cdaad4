// Protocol text -> AST.  Statements are parsed by recursive descent;
// expressions and conditions share one precedence-climbing (Pratt) parser
// whose result is then split into integer expressions and boolean
// conditions, rejecting ill-typed mixtures.  Names are resolved as soon as
// they are read (rule t-n / t-b, Fig. 4: only tid, parameters and enclosing
// loop variables may appear), and the synchronized-fragment rule of Fig. 1
// (no sync or forS inside forU / if) is enforced while parsing.
#include <cctype>
#include <cstring>
#include <string>
#include <utility>

#include "ast.h"

namespace drf {
namespace {

enum class Tk { End, Int, Name, Punct, Bad };

struct Token {
    Tk kind = Tk::End;
    std::string text;
    int64_t value = 0;
    bool too_big = false;
    int line = 1;
};

std::vector<Token> tokenize(const std::string &src)
{
    std::vector<Token> out;
    size_t i = 0;
    int line = 1;
    static const char *two[] = {"..", "==", "!=", "<=", ">=", "&&", "||"};
    while (true) {
        while (i < src.size()) {
            char c = src[i];
            if (c == '\n') { line++; i++; }
            else if (c == ' ' || c == '\t' || c == '\r') i++;
            else if (c == '#' || (c == '/' && i + 1 < src.size() && src[i + 1] == '/'))
                while (i < src.size() && src[i] != '\n') i++;
            else break;
        }
        Token t;
        t.line = line;
        if (i >= src.size()) { t.kind = Tk::End; out.push_back(t); return out; }
        char c = src[i];
        if (std::isdigit((unsigned char)c)) {
            unsigned __int128 v = 0;
            size_t j = i;
            while (j < src.size() && std::isdigit((unsigned char)src[j])) {
                v = v * 10 + (unsigned)(src[j] - '0');
                if (v > (unsigned __int128)INT64_MAX) t.too_big = true;
                j++;
            }
            t.kind = Tk::Int;
            t.value = t.too_big ? 0 : (int64_t)v;
            t.text = src.substr(i, j - i);
            i = j;
        } else if (std::isalpha((unsigned char)c) || c == '_') {
            size_t j = i;
            while (j < src.size() && (std::isalnum((unsigned char)src[j]) || src[j] == '_')) j++;
            t.kind = Tk::Name;
            t.text = src.substr(i, j - i);
            i = j;
        } else {
            t.kind = Tk::Bad;
            for (const char *p : two)
                if (src.compare(i, 2, p) == 0) { t.kind = Tk::Punct; t.text = p; i += 2; break; }
            if (t.kind == Tk::Bad) {
                if (std::strchr(";,{}[]()+-*/%<>=!:", c)) { t.kind = Tk::Punct; t.text = std::string(1, c); }
                else t.text = std::string(1, c);
                i++;
            }
        }
        out.push_back(std::move(t));
    }
}

const char *kReserved[] = {"array", "param", "skip", "sync", "rd", "wr", "if", "else", "forU",
                           "forS", "in", "tid", "min", "max", "true", "false"};

bool reserved(const std::string &s)
{
    for (const char *r : kReserved)
        if (s == r) return true;
    return false;
}

// Untyped operator tree produced by the Pratt parser.
struct PNode {
    enum Kind { Lit, Tid, Var, Param, BoolLit, Unary, Binary } kind = Lit;
    int64_t value = 0;
    uint16_t slot = 0;
    bool bval = false;
    std::string op;
    std::unique_ptr<PNode> a, b;
};
using PNodeP = std::unique_ptr<PNode>;

struct ParseFail {
    Error err;
};

class Parser {
public:
    // baby: read BabyCUDA (Fig. 3) instead of MAP text and infer its MAP by
    // the rules of Fig. 4 while parsing (see parse_babycuda_text)
    explicit Parser(const std::string &src, bool baby = false) : toks_(tokenize(src)), baby_(baby) {}

    Error run(Protocol &out)
    {
        try {
            parse_decls();
            out.body = parse_seq(true, /*until_brace=*/false);
            if (cur().kind != Tk::End) fail(S_PARSE, "unexpected token '" + cur().text + "'");
            out.narrays = (uint16_t)arrays_.size();
            out.nparams = (uint16_t)params_.size();
            out.nslots = nslots_;
        } catch (ParseFail &f) {
            return f.err;
        }
        return Error{};
    }

private:
    std::vector<Token> toks_;
    size_t pos_ = 0;
    std::vector<std::string> arrays_, params_;
    std::vector<std::pair<std::string, uint16_t>> scope_;   // enclosing loop variables
    uint16_t nslots_ = 0;
    int depth_ = 0;
    const bool baby_;
    std::vector<std::string> data_;     // BabyCUDA: names bound by a read (values, not in V)
    bool payload_ = false;              // BabyCUDA: parsing a write's payload

    const Token &cur() const { return toks_[pos_]; }
    void advance() { if (pos_ + 1 < toks_.size()) pos_++; }
    bool is_punct(const char *p) const { return cur().kind == Tk::Punct && cur().text == p; }
    bool is_word(const char *w) const { return cur().kind == Tk::Name && cur().text == w; }

    [[noreturn]] void fail(int status, const std::string &msg)
    {
        const Token &t = cur();
        if (t.kind == Tk::Bad && status == S_PARSE)
            throw ParseFail{Error::make(S_PARSE, "line " + std::to_string(t.line) + ": bad character '" + t.text + "'")};
        throw ParseFail{Error::make(status, "line " + std::to_string(t.line) + ": " + msg)};
    }

    void expect(const char *p)
    {
        if (!is_punct(p)) fail(S_PARSE, std::string("expected '") + p + "'");
        advance();
    }

    void parse_decls()
    {
        while (is_word("array") || is_word("param")) {
            bool arr = is_word("array");
            advance();
            while (true) {
                if (cur().kind != Tk::Name || reserved(cur().text)) fail(S_PARSE, "expected a name");
                for (auto &n : arrays_) if (n == cur().text) fail(S_REBIND, "'" + n + "' declared twice");
                for (auto &n : params_) if (n == cur().text) fail(S_REBIND, "'" + n + "' declared twice");
                (arr ? arrays_ : params_).push_back(cur().text);
                if (arrays_.size() > 65535 || params_.size() > 65535) fail(S_LIMIT, "too many declarations");
                advance();
                if (is_punct(",")) { advance(); continue; }
                break;
            }
            expect(";");
        }
    }

    // ------------------------------------------------ expressions (Pratt)
    static int infix_power(const Token &t)
    {
        if (t.kind != Tk::Punct) return -1;
        const std::string &s = t.text;
        if (s == "||") return 10;
        if (s == "&&") return 20;
        if (s == "==" || s == "=" || s == "!=" || s == "<" || s == "<=" || s == ">" || s == ">=") return 30;
        if (s == "+" || s == "-") return 40;
        if (s == "*" || s == "/" || s == "%") return 50;
        return -1;
    }

    PNodeP primary()
    {
        if (++depth_ > 4 * kMaxExprDepth) fail(S_LIMIT, "expression nested too deeply");
        PNodeP n(new PNode);
        const Token &t = cur();
        if (t.kind == Tk::Int) {
            if (t.too_big) fail(S_PARSE, "integer literal out of range");
            n->kind = PNode::Lit; n->value = t.value; advance();
        } else if (is_punct("(")) {
            advance();
            n = pratt(0);
            expect(")");
        } else if (is_punct("-")) {
            n->kind = PNode::Unary; n->op = "-"; advance();
            n->a = primary();                  // binds tighter than any infix operator
        } else if (is_punct("!")) {
            n->kind = PNode::Unary; n->op = "!"; advance();
            n->a = pratt(25);                  // negates a whole comparison, not an operand
        } else if (is_word("min") || is_word("max")) {
            n->kind = PNode::Binary; n->op = t.text; advance();
            expect("(");
            n->a = pratt(0);
            expect(",");
            n->b = pratt(0);
            expect(")");
        } else if (is_word("tid")) {
            n->kind = PNode::Tid; advance();
        } else if (is_word("true") || is_word("false")) {
            n->kind = PNode::BoolLit; n->bval = is_word("true"); advance();
        } else if (t.kind == Tk::Name && !reserved(t.text)) {
            bool found = false;
            for (size_t i = scope_.size(); i-- > 0;)
                if (scope_[i].first == t.text) { n->kind = PNode::Var; n->slot = scope_[i].second; found = true; break; }
            if (!found)
                for (size_t i = 0; i < params_.size(); i++)
                    if (params_[i] == t.text) { n->kind = PNode::Param; n->slot = (uint16_t)i; found = true; break; }
            if (!found && baby_)
                for (auto &d : data_)
                    if (d == t.text) {
                        // a value read from an array: allowed in a payload only (rule t-write
                        // ignores the payload; rule t-read keeps the binder out of V)
                        if (!payload_)
                            fail(S_UNBOUND_VAR, "'" + t.text + "' holds data read from an array; an index, "
                                                "condition or bound may not depend on it (rule t-read)");
                        n->kind = PNode::Lit; found = true; break;
                    }
            if (!found) fail(S_UNBOUND_VAR, "unbound variable '" + t.text + "'");
            advance();
        } else {
            fail(S_PARSE, "expected an expression");
        }
        depth_--;
        return n;
    }

    PNodeP pratt(int min_power)
    {
        PNodeP lhs = primary();
        while (true) {
            int p = infix_power(cur());
            if (p < 0 || p <= min_power) break;
            std::string op = cur().text;
            advance();
            PNodeP rhs = pratt(p == 30 ? 30 : p);   // comparisons do not chain
            PNodeP n(new PNode);
            n->kind = PNode::Binary; n->op = op; n->a = std::move(lhs); n->b = std::move(rhs);
            lhs = std::move(n);
            if (p == 30 && infix_power(cur()) == 30) fail(S_PARSE, "comparisons do not chain");
        }
        return lhs;
    }

    static bool is_bool(const PNode &n)
    {
        if (n.kind == PNode::BoolLit) return true;
        if (n.kind == PNode::Unary) return n.op == "!";
        if (n.kind == PNode::Binary) {
            const std::string &s = n.op;
            return s == "||" || s == "&&" || s == "==" || s == "=" || s == "!=" || s == "<" ||
                   s == "<=" || s == ">" || s == ">=";
        }
        return false;
    }

    ExprP to_expr(const PNode &n)
    {
        if (is_bool(n)) fail(S_PARSE, "a condition where an integer expression is expected");
        ExprP e(new Expr);
        switch (n.kind) {
        case PNode::Lit: e->op = EOp::Const; e->value = n.value; break;
        case PNode::Tid: e->op = EOp::Tid; break;
        case PNode::Var: e->op = EOp::Var; e->slot = n.slot; break;
        case PNode::Param: e->op = EOp::Param; e->slot = n.slot; break;
        case PNode::Unary: e->op = EOp::Neg; e->a = to_expr(*n.a); break;
        case PNode::Binary: {
            const std::string &s = n.op;
            e->op = s == "+" ? EOp::Add : s == "-" ? EOp::Sub : s == "*" ? EOp::Mul : s == "/" ? EOp::Div :
                    s == "%" ? EOp::Mod : s == "min" ? EOp::Min : EOp::Max;
            e->a = to_expr(*n.a);
            e->b = to_expr(*n.b);
            break;
        }
        default: fail(S_PARSE, "a condition where an integer expression is expected");
        }
        return e;
    }

    CondP to_cond(const PNode &n)
    {
        if (!is_bool(n)) fail(S_PARSE, "an integer expression where a condition is expected");
        CondP c(new Cond);
        if (n.kind == PNode::BoolLit) { c->op = n.bval ? COp::True : COp::False; return c; }
        if (n.kind == PNode::Unary) { c->op = COp::Not; c->l = to_cond(*n.a); return c; }
        const std::string &s = n.op;
        if (s == "&&" || s == "||") {
            c->op = s == "&&" ? COp::And : COp::Or;
            c->l = to_cond(*n.a);
            c->r = to_cond(*n.b);
            return c;
        }
        c->op = (s == "==" || s == "=") ? COp::Eq : s == "!=" ? COp::Ne : s == "<" ? COp::Lt :
                s == "<=" ? COp::Le : s == ">" ? COp::Gt : COp::Ge;
        c->a = to_expr(*n.a);
        c->b = to_expr(*n.b);
        return c;
    }

    ExprP parse_expr() { PNodeP n = pratt(0); return to_expr(*n); }
    CondP parse_cond() { PNodeP n = pratt(0); return to_cond(*n); }

    // ------------------------------------------------------- statements
    StmtP parse_block(bool synced)
    {
        expect("{");
        const size_t data_mark = data_.size();          // reads bind until the end of their block
        StmtP s = parse_seq(synced, true);
        data_.resize(data_mark);
        expect("}");
        return s;
    }

    bool bound_anywhere(const std::string &name) const
    {
        for (auto &v : scope_) if (v.first == name) return true;
        for (auto &p : params_) if (p == name) return true;
        for (auto &d : data_) if (d == name) return true;
        return false;
    }

    int array_index(const std::string &name)
    {
        for (size_t i = 0; i < arrays_.size(); i++) if (arrays_[i] == name) return (int)i;
        fail(S_UNKNOWN_ARRAY, "unknown array '" + name + "'");
    }

    // BabyCUDA statements: "let x = A[n];" (rule t-read: rd A[n], x stays out
    // of V for the rest of the block) and "A[n] := m;" (rule t-write: wr A[n]).
    StmtP parse_baby_access()
    {
        StmtP s(new Stmt);
        s->op = SOp::Access;
        if (is_word("let")) {
            advance();
            if (cur().kind != Tk::Name || reserved(cur().text) || cur().text == "let" || cur().text == "for")
                fail(S_PARSE, "expected a name");
            std::string name = cur().text;
            if (bound_anywhere(name)) fail(S_REBIND, "'" + name + "' is already bound");
            advance();
            expect("=");
            if (cur().kind != Tk::Name) fail(S_PARSE, "expected an array name");
            s->loc = (uint16_t)array_index(cur().text);
            advance();
            expect("[");
            s->index = parse_expr();
            expect("]");
            expect(";");
            s->write = false;
            data_.push_back(name);
            return s;
        }
        s->loc = (uint16_t)array_index(cur().text);
        advance();
        expect("[");
        s->index = parse_expr();
        expect("]");
        if (!(is_punct(":") || (cur().kind == Tk::Bad && cur().text == ":"))) fail(S_PARSE, "expected ':='");
        advance();
        expect("=");
        payload_ = true;
        parse_expr();                                    // the payload is dropped by the MAP
        payload_ = false;
        expect(";");
        s->write = true;
        return s;
    }

    StmtP parse_seq(bool synced, bool until_brace)
    {
        StmtP seq(new Stmt);
        seq->op = SOp::Seq;
        while (cur().kind != Tk::End && !(until_brace && is_punct("}")))
            seq->items.push_back(parse_stmt(synced));
        return seq;
    }

    StmtP parse_stmt(bool synced)
    {
        if (++depth_ > kMaxStmtDepth) fail(S_LIMIT, "statements nested too deeply");
        StmtP s(new Stmt);
        if (baby_ && (is_word("rd") || is_word("wr"))) fail(S_PARSE, "BabyCUDA has no rd / wr statements");
        if (baby_ && (is_word("let") ||
                      (cur().kind == Tk::Name && !reserved(cur().text) && cur().text != "for" &&
                       toks_[pos_ + 1].kind == Tk::Punct && toks_[pos_ + 1].text == "["))) {
            s = parse_baby_access();
        } else if (is_word("skip")) {
            advance(); expect(";");
            s->op = SOp::Skip;
        } else if (is_word("sync")) {
            if (!synced) fail(S_SYNC_IN_UNSYNC, "sync inside an unsynchronized fragment");
            advance(); expect(";");
            s->op = SOp::Sync;
        } else if (is_word("rd") || is_word("wr")) {
            s->op = SOp::Access;
            s->write = is_word("wr");
            advance();
            if (cur().kind != Tk::Name) fail(S_PARSE, "expected an array name");
            int loc = -1;
            for (size_t i = 0; i < arrays_.size(); i++) if (arrays_[i] == cur().text) loc = (int)i;
            if (loc < 0) fail(S_UNKNOWN_ARRAY, "unknown array '" + cur().text + "'");
            s->loc = (uint16_t)loc;
            advance();
            expect("[");
            s->index = parse_expr();
            expect("]");
            expect(";");
        } else if (is_word("if")) {
            s->op = SOp::If;
            advance();
            expect("(");
            s->cond = parse_cond();
            expect(")");
            s->then_s = parse_block(false);
            if (is_word("else")) { advance(); s->else_s = parse_block(false); }
            else { s->else_s.reset(new Stmt); s->else_s->op = SOp::Skip; }
        } else if (is_word("forU") || is_word("forS") || (baby_ && is_word("for"))) {
            bool sync_loop = is_word("forS");
            if (sync_loop && !synced) fail(S_SYNC_IN_UNSYNC, "forS inside an unsynchronized fragment");
            s->op = sync_loop ? SOp::ForS : SOp::ForU;
            advance();
            if (cur().kind != Tk::Name || reserved(cur().text)) fail(S_PARSE, "expected a loop variable");
            std::string name = cur().text;
            for (auto &v : scope_) if (v.first == name) fail(S_REBIND, "'" + name + "' is already bound");
            for (auto &p : params_) if (p == name) fail(S_REBIND, "'" + name + "' is already bound");
            advance();
            if (!is_word("in")) fail(S_PARSE, "expected 'in'");
            advance();
            s->lo = parse_expr();          // bounds live in the enclosing scope (rule t-for)
            expect("..");
            s->hi = parse_expr();
            if (nslots_ == 65535) fail(S_LIMIT, "too many loops");
            s->slot = nslots_++;
            scope_.emplace_back(name, s->slot);
            s->body = parse_block(sync_loop);
            scope_.pop_back();
        } else {
            fail(S_PARSE, "expected a statement");
        }
        depth_--;
        return s;
    }
};

}  // namespace

Error parse_text(const std::string &text, Protocol &out)
{
    Parser p(text);
    return p.run(out);
}

Error parse_babycuda_text(const std::string &text, Protocol &out)
{
    Parser p(text, true);
    return p.run(out);
}

}  // namespace drf
