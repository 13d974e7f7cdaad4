// Protocol AST -> MAP text (the syntax of include/drf.h).  Every expression
// and condition is fully parenthesised, so the text parses back to the same
// tree.
#include <string>

#include "ast.h"

namespace drf {
namespace {

void expr(const Expr &e, std::string &o)
{
    switch (e.op) {
    case EOp::Const:
        if (e.value < 0) o += "(0 - " + std::to_string((unsigned long long)(0ull - (unsigned long long)e.value)) + ")";
        else o += std::to_string(e.value);
        return;
    case EOp::Tid: o += "tid"; return;
    case EOp::Var: o += "v" + std::to_string(e.slot); return;
    case EOp::Param: o += "P" + std::to_string(e.slot); return;
    case EOp::Neg: o += "(-"; expr(*e.a, o); o += ")"; return;
    case EOp::Min: case EOp::Max:
        o += e.op == EOp::Min ? "min(" : "max(";
        expr(*e.a, o); o += ", "; expr(*e.b, o); o += ")";
        return;
    default: break;
    }
    static const char *ops[] = {"", "", "", "", " + ", " - ", " * ", " / ", " % "};
    o += "(";
    expr(*e.a, o);
    o += ops[(int)e.op];
    expr(*e.b, o);
    o += ")";
}

void cond(const Cond &c, std::string &o)
{
    switch (c.op) {
    case COp::True: o += "true"; return;
    case COp::False: o += "false"; return;
    case COp::Not: o += "!("; cond(*c.l, o); o += ")"; return;
    case COp::And: case COp::Or:
        o += "(("; cond(*c.l, o); o += c.op == COp::And ? ") && (" : ") || ("; cond(*c.r, o); o += "))";
        return;
    default: break;
    }
    static const char *rel[] = {"", "", " == ", " != ", " < ", " <= ", " > ", " >= "};
    o += "(";
    expr(*c.a, o);
    o += rel[(int)c.op];
    expr(*c.b, o);
    o += ")";
}

void stmt(const Stmt &s, int ind, std::string &o)
{
    std::string pad((size_t)ind * 2, ' ');
    switch (s.op) {
    case SOp::Skip: o += pad + "skip;\n"; return;
    case SOp::Sync: o += pad + "sync;\n"; return;
    case SOp::Access:
        o += pad + (s.write ? "wr A" : "rd A") + std::to_string(s.loc) + "[";
        expr(*s.index, o);
        o += "];\n";
        return;
    case SOp::Seq:
        for (auto &it : s.items) stmt(*it, ind, o);
        return;
    case SOp::If:
        o += pad + "if (";
        cond(*s.cond, o);
        o += ") {\n";
        stmt(*s.then_s, ind + 1, o);
        if (s.else_s->op == SOp::Skip) {          // no else branch (the parser's implicit skip)
            o += pad + "}\n";
            return;
        }
        o += pad + "} else {\n";
        stmt(*s.else_s, ind + 1, o);
        o += pad + "}\n";
        return;
    case SOp::ForU:
    case SOp::ForS:
        o += pad + (s.op == SOp::ForU ? "forU v" : "forS v") + std::to_string(s.slot) + " in ";
        expr(*s.lo, o);
        o += " .. ";
        expr(*s.hi, o);
        o += " {\n";
        stmt(*s.body, ind + 1, o);
        o += pad + "}\n";
        return;
    }
}

}  // namespace

std::string protocol_text(const Protocol &p)
{
    std::string o;
    if (p.narrays) {
        o += "array ";
        for (uint16_t i = 0; i < p.narrays; i++) o += (i ? ", A" : "A") + std::to_string(i);
        o += ";\n";
    }
    if (p.nparams) {
        o += "param ";
        for (uint16_t i = 0; i < p.nparams; i++) o += (i ? ", P" : "P") + std::to_string(i);
        o += ";\n";
    }
    stmt(*p.body, 0, o);
    return o;
}

}  // namespace drf
