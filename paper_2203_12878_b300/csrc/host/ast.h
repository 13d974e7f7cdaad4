// Protocol abstract syntax used by the host front-end (text parser, bytecode
// codec, analysis and lowering).  Mirrors Fig. 1 (syntax of MAPs) with the
// synchronized fragment admitting accesses: statements are skip, sync,
// accesses rd/wr A[n], sequences, conditionals, forU and forS loops.
#pragma once

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

namespace drf {

enum class EOp : uint8_t { Const, Tid, Var, Param, Add, Sub, Mul, Div, Mod, Min, Max, Neg };
enum class COp : uint8_t { True, False, Eq, Ne, Lt, Le, Gt, Ge, And, Or, Not };
enum class SOp : uint8_t { Skip, Sync, Access, Seq, If, ForU, ForS };

struct Expr {
    EOp op = EOp::Const;
    int64_t value = 0;       // Const
    uint16_t slot = 0;       // Var: loop-variable slot; Param: parameter index
    std::unique_ptr<Expr> a, b;
};
using ExprP = std::unique_ptr<Expr>;

struct Cond {
    COp op = COp::True;
    ExprP a, b;                    // comparisons
    std::unique_ptr<Cond> l, r;    // And / Or / Not (l only)
};
using CondP = std::unique_ptr<Cond>;

struct Stmt {
    SOp op = SOp::Skip;
    bool write = false;            // Access
    uint16_t loc = 0;              // Access
    uint16_t slot = 0;             // ForU / ForS: the loop variable's slot
    ExprP index;                   // Access
    ExprP lo, hi;                  // ForU / ForS
    CondP cond;                    // If
    std::unique_ptr<Stmt> then_s, else_s, body;
    std::vector<std::unique_ptr<Stmt>> items;   // Seq
};
using StmtP = std::unique_ptr<Stmt>;

struct Protocol {
    uint16_t narrays = 0;
    uint16_t nparams = 0;
    uint16_t nslots = 0;           // loop variables (each binder has its own slot)
    StmtP body;                    // a Seq
};

// Status codes of the C ABI (include/drf.h), repeated here for host code.
enum Status : int {
    S_OK = 0, S_INVALID_ARG = -1, S_PARSE = -2, S_INVALID_BYTECODE = -3, S_UNBOUND_VAR = -4,
    S_UNKNOWN_ARRAY = -5, S_REBIND = -6, S_SYNC_IN_UNSYNC = -7, S_OVERFLOW_RISK = -8,
    S_INDEX_OOB = -9, S_DIV_ZERO = -10, S_KEY_TOO_WIDE = -11, S_NOMEM = -12, S_CUDA = -13,
    S_TIMEOUT = -14, S_BUSY = -15, S_LIMIT = -16, S_NOT_FOUND = -17, S_INTERNAL = -18
};

struct Error {
    int status = S_OK;
    std::string message;
    bool ok() const { return status == S_OK; }
    static Error make(int s, std::string m) { Error e; e.status = s; e.message = std::move(m); return e; }
};

// Front-end entry points.
Error parse_text(const std::string &text, Protocol &out);
// BabyCUDA text (Fig. 3 syntax: "let x = A[n];", "A[n] := m;", if, for,
// forS, sync, skip) typed into its MAP by the rules of Fig. 4.
Error parse_babycuda_text(const std::string &text, Protocol &out);
// MAP text of a protocol (arrays named A0.., parameters P0.., loop
// variables v<slot>); parse_text reads it back to the same protocol.
std::string protocol_text(const Protocol &p);
std::vector<uint8_t> encode_bytecode(const Protocol &p);
Error decode_bytecode(const uint8_t *data, size_t len, Protocol &out);

// Nesting limits of this implementation.
constexpr int kMaxLoopDepth = 15;     // loops nested inside each other
constexpr int kMaxExprDepth = 48;     // expression / condition tree depth
constexpr int kMaxStmtDepth = 64;     // statement nesting (if / loops)

}  // namespace drf
