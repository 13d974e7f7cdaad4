/*
 * drf_oracle.c -- reference oracle for data-race-freedom checking of memory
 * access protocols (MAPs).  TEST INFRASTRUCTURE ONLY: it is compiled and called
 * by the test suite, by the smoke check and by the benchmark's CPU-baseline
 * leg, never by the product library.  It shares no code, header, table or
 * helper with the CUDA path: it has its own lexer, parser, validator,
 * evaluator and checker, written from the paper's definitions.
 *
 * What it computes (paper: "Provable GPU Data-Races in Static Race
 * Detection", Liew, Cogumbreiro, Lange, PLACES 2022):
 *
 *   * Protocol syntax: Fig. 1 (syntax of MAPs) -- arithmetic expressions over
 *     tid and variables, boolean conditions, accesses rd[n] / wr[n], skip,
 *     sequencing, conditionals, unsynchronized loops for^U, and the
 *     synchronized fragment (sync, for^S).  Read with the accesses allowed
 *     inside the synchronized fragment (the printed grammar omits them).
 *   * Per-thread evaluation: the big-step rules of Fig. 3 -- seq, if-t, if-f,
 *     for-1, for-2, skip, and the read / write rules with array contents
 *     dropped (a MAP keeps only mode and index, Sec. 2 and rule t-write in
 *     Fig. 4).  The synchronized fragment is omitted in the paper; it is read
 *     here as a per-thread phase counter bumped by every executed sync.
 *   * Rule par (Fig. 3): every thread id runs independently with tid
 *     substituted; their read/write sets are merged into one phase.
 *   * Definition 1 (DRF program, Sec. 3): a phase is racy iff two distinct
 *     threads i1 != i2 and an index j exist with j written by i1 and read or
 *     written by i2; a history is DRF iff every phase is.  One behavioural
 *     type per array (Sec. 3): the same index in different arrays never
 *     conflicts.
 *
 * Two checkers over the same per-thread histories:
 *   method 0 ("A") -- Definition 1 taken literally: per phase and array, every
 *     ordered pair of distinct threads, intersecting the first thread's write
 *     set with the second thread's read-and-write set.
 *   method 1 ("B") -- the same predicate per cell: all accesses grouped by
 *     (phase, array, index); per cell the two smallest distinct accessor tids
 *     and the two smallest distinct writer tids.  A cell is racy iff it has a
 *     writer and two distinct accessors.  B is validated against A by the
 *     tests; B is the one that scales to millions of accesses.
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - loop range lo..hi is x = lo, lo+1, ..., hi-1 (rules for-1 / for-2);
 *     the bounds are evaluated once, at loop entry;
 *   - arithmetic is on mathematical integers held in int64; an operation
 *     whose exact result leaves int64 is an evaluation error (OVERFLOW);
 *     '/' is floor division, '%' is the Euclidean remainder (in [0,|m|));
 *     division or remainder by 0 is an evaluation error (DIV_ZERO);
 *   - every array has a size; an index outside [0, size) is an evaluation
 *     error (INDEX_OOB); errors are reported for the smallest failing tid,
 *     with the number of accesses that thread completed before the failure;
 *   - threads that execute different numbers of syncs give the verdict
 *     BARRIER_DIVERGENCE (smallest tid whose count differs from thread 0's);
 *   - the witness of a racy protocol is the lexicographically smallest
 *     (phase, array, index, i, j) over racing pairs with i < j;
 *   - precedence: evaluation error > barrier divergence > race.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <stdarg.h>
#include <ctype.h>

/* Status codes.  The numeric values are an interface agreement with the
 * product's C header (the tests compare statuses by value). */
enum {
    OR_OK = 0,
    OR_E_INVALID_ARG = -1,
    OR_E_PARSE = -2,
    OR_E_UNBOUND_VAR = -4,
    OR_E_UNKNOWN_ARRAY = -5,
    OR_E_REBIND = -6,
    OR_E_SYNC_IN_UNSYNC = -7,
    OR_E_OVERFLOW = -8,
    OR_E_INDEX_OOB = -9,
    OR_E_DIV_ZERO = -10,
    OR_E_NOMEM = -12
};

enum { V_DRF = 0, V_RACY = 1, V_DIVERGENCE = 2 };

typedef struct {
    int32_t status;
    int32_t verdict;
    uint32_t phase, loc;
    uint64_t index;
    uint32_t tid_i, tid_j;
    uint32_t i_writes, j_writes;
    uint32_t div_tid, sync_count_0, sync_count_div;
    uint32_t phases;
    uint64_t tuples;
    uint32_t err_tid, pad0;
    uint64_t err_ordinal;
} oracle_result;

/* ------------------------------------------------------------------ AST -- */

typedef enum { EK_INT, EK_TID, EK_VAR, EK_PARAM, EK_BIN, EK_NEG } ExprKind;
typedef enum { OP_ADD, OP_SUB, OP_MUL, OP_DIV, OP_MOD, OP_MIN, OP_MAX } BinOp;
typedef struct Expr {
    ExprKind kind;
    int64_t value;          /* EK_INT */
    int slot;               /* EK_VAR: loop-variable slot, EK_PARAM: param index */
    BinOp op;
    struct Expr *a, *b;
} Expr;

typedef enum { CK_TRUE, CK_FALSE, CK_CMP, CK_AND, CK_OR, CK_NOT } CondKind;
typedef enum { R_EQ, R_NE, R_LT, R_LE, R_GT, R_GE } RelOp;
typedef struct Cond {
    CondKind kind;
    RelOp rel;
    Expr *a, *b;
    struct Cond *l, *r;
} Cond;

typedef enum { SK_SKIP, SK_SYNC, SK_ACCESS, SK_SEQ, SK_IF, SK_FOR_U, SK_FOR_S } StmtKind;
typedef struct Stmt {
    StmtKind kind;
    int write;              /* SK_ACCESS: 1 = wr, 0 = rd */
    int loc;                /* SK_ACCESS: array index */
    Expr *index;            /* SK_ACCESS */
    Cond *cond;             /* SK_IF */
    struct Stmt *then_s, *else_s;
    int slot;               /* SK_FOR_*: loop-variable slot */
    Expr *lo, *hi;          /* SK_FOR_* */
    struct Stmt *body;      /* SK_FOR_* */
    struct Stmt **items;    /* SK_SEQ */
    int nitems;
} Stmt;

/* Simple arena so that a parse can be freed in one go. */
typedef struct Arena { struct Arena *next; size_t used, cap; char data[]; } Arena;

typedef struct {
    Arena *arena;
    /* declarations */
    char **arrays; int narrays;
    char **params; int nparams;
    int nslots;             /* loop-variable slots handed out */
    Stmt *body;
} Program;

static void *arena_alloc(Program *p, size_t n)
{
    n = (n + 15) & ~(size_t)15;
    if (!p->arena || p->arena->used + n > p->arena->cap) {
        size_t cap = n > 65536 ? n : 65536;
        Arena *a = (Arena *)malloc(sizeof(Arena) + cap);
        if (!a) return NULL;
        a->next = p->arena; a->used = 0; a->cap = cap;
        p->arena = a;
    }
    void *r = p->arena->data + p->arena->used;
    p->arena->used += n;
    memset(r, 0, n);
    return r;
}

static void program_free(Program *p)
{
    Arena *a = p->arena;
    while (a) { Arena *n = a->next; free(a); a = n; }
    free(p->arrays);
    free(p->params);
    memset(p, 0, sizeof(*p));
}

/* --------------------------------------------------------------- lexer -- */

typedef enum {
    T_EOF, T_INT, T_IDENT,
    T_SEMI, T_COMMA, T_LBRACE, T_RBRACE, T_LBRACK, T_RBRACK, T_LPAREN, T_RPAREN,
    T_DOTDOT, T_PLUS, T_MINUS, T_STAR, T_SLASH, T_PERCENT,
    T_EQ, T_NE, T_LT, T_LE, T_GT, T_GE, T_ANDAND, T_OROR, T_BANG,
    T_BAD
} TokKind;

typedef struct {
    TokKind kind;
    const char *start; int len;
    int64_t value;
    int line;
    int int_overflow;
} Token;

typedef struct {
    const char *src, *pos;
    int line;
    Token tok;
    Program *prog;
    int status;
    char *msg; int msglen;
    /* loop variables in scope: names and slots */
    char *scope_names[256]; int scope_slots[256]; int nscope;
} Parser;

static void lex_next(Parser *ps)
{
    const char *s = ps->pos;
    for (;;) {
        while (*s == ' ' || *s == '\t' || *s == '\r' || *s == '\n') {
            if (*s == '\n') ps->line++;
            s++;
        }
        if (*s == '#' || (s[0] == '/' && s[1] == '/')) {
            while (*s && *s != '\n') s++;
            continue;
        }
        break;
    }
    Token t; memset(&t, 0, sizeof t);
    t.start = s; t.line = ps->line;
    if (!*s) { t.kind = T_EOF; ps->tok = t; ps->pos = s; return; }
    if (isdigit((unsigned char)*s)) {
        uint64_t v = 0; int ovf = 0;
        while (isdigit((unsigned char)*s)) {
            unsigned d = (unsigned)(*s - '0');
            if (v > (UINT64_C(9223372036854775807) - d) / 10) ovf = 1;
            else v = v * 10 + d;
            s++;
        }
        t.kind = T_INT; t.value = (int64_t)v; t.int_overflow = ovf;
    } else if (isalpha((unsigned char)*s) || *s == '_') {
        while (isalnum((unsigned char)*s) || *s == '_') s++;
        t.kind = T_IDENT;
    } else {
        char c = *s, c1 = s[1];
        s++;
        switch (c) {
        case ';': t.kind = T_SEMI; break;
        case ',': t.kind = T_COMMA; break;
        case '{': t.kind = T_LBRACE; break;
        case '}': t.kind = T_RBRACE; break;
        case '[': t.kind = T_LBRACK; break;
        case ']': t.kind = T_RBRACK; break;
        case '(': t.kind = T_LPAREN; break;
        case ')': t.kind = T_RPAREN; break;
        case '+': t.kind = T_PLUS; break;
        case '-': t.kind = T_MINUS; break;
        case '*': t.kind = T_STAR; break;
        case '/': t.kind = T_SLASH; break;
        case '%': t.kind = T_PERCENT; break;
        case '.': if (c1 == '.') { s++; t.kind = T_DOTDOT; } else t.kind = T_BAD; break;
        case '=': if (c1 == '=') s++; t.kind = T_EQ; break;
        case '!': if (c1 == '=') { s++; t.kind = T_NE; } else t.kind = T_BANG; break;
        case '<': if (c1 == '=') { s++; t.kind = T_LE; } else t.kind = T_LT; break;
        case '>': if (c1 == '=') { s++; t.kind = T_GE; } else t.kind = T_GT; break;
        case '&': if (c1 == '&') { s++; t.kind = T_ANDAND; } else t.kind = T_BAD; break;
        case '|': if (c1 == '|') { s++; t.kind = T_OROR; } else t.kind = T_BAD; break;
        default: t.kind = T_BAD; break;
        }
    }
    t.len = (int)(s - t.start);
    ps->pos = s;
    ps->tok = t;
}

static int tok_is(const Parser *ps, const char *word)
{
    return ps->tok.kind == T_IDENT && (int)strlen(word) == ps->tok.len &&
           strncmp(ps->tok.start, word, (size_t)ps->tok.len) == 0;
}

static int fail(Parser *ps, int status, const char *fmt, ...)
{
    if (ps->status == OR_OK) {
        ps->status = status;
        if (ps->msg && ps->msglen > 0) {
            int n = snprintf(ps->msg, (size_t)ps->msglen, "line %d: ", ps->tok.line);
            if (n < 0) n = 0;
            if (n < ps->msglen) {
                va_list ap; va_start(ap, fmt);
                vsnprintf(ps->msg + n, (size_t)(ps->msglen - n), fmt, ap);
                va_end(ap);
            }
        }
    }
    return 0;
}

static int expect(Parser *ps, TokKind k, const char *what)
{
    if (ps->status) return 0;
    if (ps->tok.kind != k) return fail(ps, OR_E_PARSE, "expected %s", what);
    lex_next(ps);
    return 1;
}

static const char *reserved[] = {
    "array", "param", "skip", "sync", "rd", "wr", "if", "else", "forU", "forS",
    "in", "tid", "min", "max", "true", "false", NULL
};

static int is_reserved(const Token *t)
{
    for (int i = 0; reserved[i]; i++)
        if ((int)strlen(reserved[i]) == t->len && strncmp(t->start, reserved[i], (size_t)t->len) == 0)
            return 1;
    return 0;
}

static char *tok_dup(Parser *ps)
{
    char *s = (char *)arena_alloc(ps->prog, (size_t)ps->tok.len + 1);
    if (!s) { fail(ps, OR_E_NOMEM, "out of memory"); return NULL; }
    memcpy(s, ps->tok.start, (size_t)ps->tok.len);
    s[ps->tok.len] = 0;
    return s;
}

static int name_eq(const Token *t, const char *name)
{
    return (int)strlen(name) == t->len && strncmp(t->start, name, (size_t)t->len) == 0;
}

/* -------------------------------------------------------------- parser -- */

static Expr *parse_expr(Parser *ps);

static Expr *mk_expr(Parser *ps, ExprKind k)
{
    Expr *e = (Expr *)arena_alloc(ps->prog, sizeof(Expr));
    if (!e) fail(ps, OR_E_NOMEM, "out of memory");
    else e->kind = k;
    return e;
}

static Expr *mk_bin(Parser *ps, BinOp op, Expr *a, Expr *b)
{
    Expr *e = mk_expr(ps, EK_BIN);
    if (e) { e->op = op; e->a = a; e->b = b; }
    return e;
}

static Expr *parse_atom(Parser *ps)
{
    if (ps->status) return NULL;
    if (ps->tok.kind == T_INT) {
        if (ps->tok.int_overflow) { fail(ps, OR_E_PARSE, "integer literal out of range"); return NULL; }
        Expr *e = mk_expr(ps, EK_INT);
        if (e) e->value = ps->tok.value;
        lex_next(ps);
        return e;
    }
    if (ps->tok.kind == T_LPAREN) {
        lex_next(ps);
        Expr *e = parse_expr(ps);
        expect(ps, T_RPAREN, "')'");
        return e;
    }
    if (tok_is(ps, "min") || tok_is(ps, "max")) {
        BinOp op = tok_is(ps, "min") ? OP_MIN : OP_MAX;
        lex_next(ps);
        expect(ps, T_LPAREN, "'('");
        Expr *a = parse_expr(ps);
        expect(ps, T_COMMA, "','");
        Expr *b = parse_expr(ps);
        expect(ps, T_RPAREN, "')'");
        return ps->status ? NULL : mk_bin(ps, op, a, b);
    }
    if (tok_is(ps, "tid")) {
        lex_next(ps);
        return mk_expr(ps, EK_TID);
    }
    if (ps->tok.kind == T_IDENT && !is_reserved(&ps->tok)) {
        /* innermost loop variable first, then parameters (scope check, rule t-n) */
        for (int i = ps->nscope - 1; i >= 0; i--) {
            if (name_eq(&ps->tok, ps->scope_names[i])) {
                Expr *e = mk_expr(ps, EK_VAR);
                if (e) e->slot = ps->scope_slots[i];
                lex_next(ps);
                return e;
            }
        }
        for (int i = 0; i < ps->prog->nparams; i++) {
            if (name_eq(&ps->tok, ps->prog->params[i])) {
                Expr *e = mk_expr(ps, EK_PARAM);
                if (e) e->slot = i;
                lex_next(ps);
                return e;
            }
        }
        fail(ps, OR_E_UNBOUND_VAR, "unbound variable '%.*s'", ps->tok.len, ps->tok.start);
        return NULL;
    }
    fail(ps, OR_E_PARSE, "expected an expression");
    return NULL;
}

static Expr *parse_unary(Parser *ps)
{
    if (ps->status) return NULL;
    if (ps->tok.kind == T_MINUS) {
        lex_next(ps);
        Expr *a = parse_unary(ps);
        if (ps->status) return NULL;
        Expr *e = mk_expr(ps, EK_NEG);
        if (e) e->a = a;
        return e;
    }
    return parse_atom(ps);
}

static Expr *parse_term(Parser *ps)
{
    Expr *e = parse_unary(ps);
    while (!ps->status && (ps->tok.kind == T_STAR || ps->tok.kind == T_SLASH || ps->tok.kind == T_PERCENT)) {
        BinOp op = ps->tok.kind == T_STAR ? OP_MUL : ps->tok.kind == T_SLASH ? OP_DIV : OP_MOD;
        lex_next(ps);
        Expr *b = parse_unary(ps);
        if (ps->status) return NULL;
        e = mk_bin(ps, op, e, b);
    }
    return ps->status ? NULL : e;
}

static Expr *parse_expr(Parser *ps)
{
    Expr *e = parse_term(ps);
    while (!ps->status && (ps->tok.kind == T_PLUS || ps->tok.kind == T_MINUS)) {
        BinOp op = ps->tok.kind == T_PLUS ? OP_ADD : OP_SUB;
        lex_next(ps);
        Expr *b = parse_term(ps);
        if (ps->status) return NULL;
        e = mk_bin(ps, op, e, b);
    }
    return ps->status ? NULL : e;
}

static Cond *parse_cond(Parser *ps);

static Cond *mk_cond(Parser *ps, CondKind k)
{
    Cond *c = (Cond *)arena_alloc(ps->prog, sizeof(Cond));
    if (!c) fail(ps, OR_E_NOMEM, "out of memory");
    else c->kind = k;
    return c;
}

/* The rest of a comparison whose left operand has been parsed. */
static Cond *finish_cmp(Parser *ps, Expr *a)
{
    if (ps->status) return NULL;
    if (!(ps->tok.kind >= T_EQ && ps->tok.kind <= T_GE)) {
        fail(ps, OR_E_PARSE, "expected a comparison operator");
        return NULL;
    }
    TokKind k = ps->tok.kind;
    lex_next(ps);
    Expr *b = parse_expr(ps);
    if (ps->status) return NULL;
    Cond *c = mk_cond(ps, CK_CMP);
    if (c) {
        c->a = a; c->b = b;
        c->rel = k == T_EQ ? R_EQ : k == T_NE ? R_NE : k == T_LT ? R_LT :
                 k == T_LE ? R_LE : k == T_GT ? R_GT : R_GE;
    }
    return c;
}

/* An atom of a condition: true | false | ! atom | expr relop expr | ( cond ).
 * A leading '(' may open either a parenthesised condition or an arithmetic
 * expression; the comparison is tried first and the parser backs up. */
static Cond *parse_cond_atom(Parser *ps)
{
    if (ps->status) return NULL;
    if (tok_is(ps, "true")) { lex_next(ps); return mk_cond(ps, CK_TRUE); }
    if (tok_is(ps, "false")) { lex_next(ps); return mk_cond(ps, CK_FALSE); }
    if (ps->tok.kind == T_BANG) {
        lex_next(ps);
        Cond *a = parse_cond_atom(ps);
        if (ps->status) return NULL;
        Cond *c = mk_cond(ps, CK_NOT);
        if (c) c->l = a;
        return c;
    }
    if (ps->tok.kind == T_LPAREN) {
        const char *save_pos = ps->pos; Token save_tok = ps->tok; int save_line = ps->line;
        Expr *a = parse_expr(ps);
        if (!ps->status && ps->tok.kind >= T_EQ && ps->tok.kind <= T_GE)
            return finish_cmp(ps, a);
        /* not a comparison: back up and parse a parenthesised condition */
        ps->status = OR_OK;
        if (ps->msg && ps->msglen > 0) ps->msg[0] = 0;
        ps->pos = save_pos; ps->tok = save_tok; ps->line = save_line;
        lex_next(ps);
        Cond *c = parse_cond(ps);
        expect(ps, T_RPAREN, "')'");
        return ps->status ? NULL : c;
    }
    Expr *a = parse_expr(ps);
    return finish_cmp(ps, a);
}

static Cond *parse_conj(Parser *ps)
{
    Cond *c = parse_cond_atom(ps);
    while (!ps->status && ps->tok.kind == T_ANDAND) {
        lex_next(ps);
        Cond *r = parse_cond_atom(ps);
        if (ps->status) return NULL;
        Cond *n = mk_cond(ps, CK_AND);
        if (n) { n->l = c; n->r = r; }
        c = n;
    }
    return ps->status ? NULL : c;
}

static Cond *parse_cond(Parser *ps)
{
    Cond *c = parse_conj(ps);
    while (!ps->status && ps->tok.kind == T_OROR) {
        lex_next(ps);
        Cond *r = parse_conj(ps);
        if (ps->status) return NULL;
        Cond *n = mk_cond(ps, CK_OR);
        if (n) { n->l = c; n->r = r; }
        c = n;
    }
    return ps->status ? NULL : c;
}

static Stmt *mk_stmt(Parser *ps, StmtKind k)
{
    Stmt *s = (Stmt *)arena_alloc(ps->prog, sizeof(Stmt));
    if (!s) fail(ps, OR_E_NOMEM, "out of memory");
    else s->kind = k;
    return s;
}

/* synced != 0: the statement sits in the synchronized fragment, where sync
 * and for^S are allowed; inside for^U and if bodies they are not (Fig. 1). */
static Stmt *parse_block(Parser *ps, int synced);

static Stmt *parse_stmt(Parser *ps, int synced)
{
    if (ps->status) return NULL;
    if (tok_is(ps, "skip")) {
        lex_next(ps);
        expect(ps, T_SEMI, "';'");
        return mk_stmt(ps, SK_SKIP);
    }
    if (tok_is(ps, "sync")) {
        if (!synced) { fail(ps, OR_E_SYNC_IN_UNSYNC, "sync inside an unsynchronized fragment"); return NULL; }
        lex_next(ps);
        expect(ps, T_SEMI, "';'");
        return mk_stmt(ps, SK_SYNC);
    }
    if (tok_is(ps, "rd") || tok_is(ps, "wr")) {
        int write = tok_is(ps, "wr");
        lex_next(ps);
        if (ps->tok.kind != T_IDENT) { fail(ps, OR_E_PARSE, "expected an array name"); return NULL; }
        int loc = -1;
        for (int i = 0; i < ps->prog->narrays; i++)
            if (name_eq(&ps->tok, ps->prog->arrays[i])) loc = i;
        if (loc < 0) { fail(ps, OR_E_UNKNOWN_ARRAY, "unknown array '%.*s'", ps->tok.len, ps->tok.start); return NULL; }
        lex_next(ps);
        expect(ps, T_LBRACK, "'['");
        Expr *ix = parse_expr(ps);
        expect(ps, T_RBRACK, "']'");
        expect(ps, T_SEMI, "';'");
        if (ps->status) return NULL;
        Stmt *s = mk_stmt(ps, SK_ACCESS);
        if (s) { s->write = write; s->loc = loc; s->index = ix; }
        return s;
    }
    if (tok_is(ps, "if")) {
        lex_next(ps);
        expect(ps, T_LPAREN, "'('");
        Cond *c = parse_cond(ps);
        expect(ps, T_RPAREN, "')'");
        Stmt *th = parse_block(ps, 0);
        Stmt *el = NULL;
        if (!ps->status && tok_is(ps, "else")) {
            lex_next(ps);
            el = parse_block(ps, 0);
        }
        if (ps->status) return NULL;
        if (!el) el = mk_stmt(ps, SK_SKIP);
        Stmt *s = mk_stmt(ps, SK_IF);
        if (s) { s->cond = c; s->then_s = th; s->else_s = el; }
        return s;
    }
    if (tok_is(ps, "forU") || tok_is(ps, "forS")) {
        int is_s = tok_is(ps, "forS");
        if (is_s && !synced) { fail(ps, OR_E_SYNC_IN_UNSYNC, "forS inside an unsynchronized fragment"); return NULL; }
        lex_next(ps);
        if (ps->tok.kind != T_IDENT || is_reserved(&ps->tok)) { fail(ps, OR_E_PARSE, "expected a loop variable"); return NULL; }
        /* binders are distinct from every name in scope (rule t-for: x not in V) */
        for (int i = 0; i < ps->nscope; i++)
            if (name_eq(&ps->tok, ps->scope_names[i])) { fail(ps, OR_E_REBIND, "'%.*s' is already bound", ps->tok.len, ps->tok.start); return NULL; }
        for (int i = 0; i < ps->prog->nparams; i++)
            if (name_eq(&ps->tok, ps->prog->params[i])) { fail(ps, OR_E_REBIND, "'%.*s' is already bound", ps->tok.len, ps->tok.start); return NULL; }
        char *name = tok_dup(ps);
        lex_next(ps);
        if (!tok_is(ps, "in")) { fail(ps, OR_E_PARSE, "expected 'in'"); return NULL; }
        lex_next(ps);
        /* the bounds are typed in the enclosing scope (rule t-for) */
        Expr *lo = parse_expr(ps);
        expect(ps, T_DOTDOT, "'..'");
        Expr *hi = parse_expr(ps);
        if (ps->status) return NULL;
        if (ps->nscope >= 256) { fail(ps, OR_E_PARSE, "loops nested too deeply"); return NULL; }
        int slot = ps->prog->nslots++;
        ps->scope_names[ps->nscope] = name;
        ps->scope_slots[ps->nscope] = slot;
        ps->nscope++;
        Stmt *body = parse_block(ps, is_s);
        ps->nscope--;
        if (ps->status) return NULL;
        Stmt *s = mk_stmt(ps, is_s ? SK_FOR_S : SK_FOR_U);
        if (s) { s->slot = slot; s->lo = lo; s->hi = hi; s->body = body; }
        return s;
    }
    fail(ps, OR_E_PARSE, "expected a statement");
    return NULL;
}

/* A sequence of statements up to '}' or end of input. */
static Stmt *parse_seq(Parser *ps, int synced, TokKind end)
{
    Stmt **items = NULL; int n = 0, cap = 0;
    while (!ps->status && ps->tok.kind != end && ps->tok.kind != T_EOF) {
        Stmt *s = parse_stmt(ps, synced);
        if (ps->status) break;
        if (n == cap) {
            cap = cap ? cap * 2 : 8;
            Stmt **ni = (Stmt **)realloc(items, sizeof(Stmt *) * (size_t)cap);
            if (!ni) { fail(ps, OR_E_NOMEM, "out of memory"); break; }
            items = ni;
        }
        items[n++] = s;
    }
    if (ps->status) { free(items); return NULL; }
    Stmt *seq = mk_stmt(ps, SK_SEQ);
    if (seq) {
        seq->items = (Stmt **)arena_alloc(ps->prog, sizeof(Stmt *) * (size_t)(n ? n : 1));
        if (!seq->items) { free(items); fail(ps, OR_E_NOMEM, "out of memory"); return NULL; }
        if (n) memcpy(seq->items, items, sizeof(Stmt *) * (size_t)n);
        seq->nitems = n;
    }
    free(items);
    return seq;
}

static Stmt *parse_block(Parser *ps, int synced)
{
    if (!expect(ps, T_LBRACE, "'{'")) return NULL;
    Stmt *s = parse_seq(ps, synced, T_RBRACE);
    expect(ps, T_RBRACE, "'}'");
    return ps->status ? NULL : s;
}

static int add_name(Parser *ps, char ***list, int *n)
{
    if (ps->tok.kind != T_IDENT || is_reserved(&ps->tok)) return fail(ps, OR_E_PARSE, "expected a name");
    Program *p = ps->prog;
    for (int i = 0; i < p->narrays; i++)
        if (name_eq(&ps->tok, p->arrays[i])) return fail(ps, OR_E_REBIND, "'%.*s' declared twice", ps->tok.len, ps->tok.start);
    for (int i = 0; i < p->nparams; i++)
        if (name_eq(&ps->tok, p->params[i])) return fail(ps, OR_E_REBIND, "'%.*s' declared twice", ps->tok.len, ps->tok.start);
    char *name = tok_dup(ps);
    if (!name) return 0;
    char **nl = (char **)realloc(*list, sizeof(char *) * (size_t)(*n + 1));
    if (!nl) return fail(ps, OR_E_NOMEM, "out of memory");
    nl[*n] = name; *list = nl; (*n)++;
    lex_next(ps);
    return 1;
}

static int parse_program(const char *text, Program *prog, char *msg, int msglen)
{
    Parser ps; memset(&ps, 0, sizeof ps);
    memset(prog, 0, sizeof *prog);
    ps.src = ps.pos = text; ps.line = 1; ps.prog = prog; ps.msg = msg; ps.msglen = msglen;
    if (msg && msglen > 0) msg[0] = 0;
    lex_next(&ps);
    /* declarations: "array A, B;" and "param M;" */
    while (!ps.status && (tok_is(&ps, "array") || tok_is(&ps, "param"))) {
        int is_array = tok_is(&ps, "array");
        lex_next(&ps);
        for (;;) {
            if (is_array) add_name(&ps, &prog->arrays, &prog->narrays);
            else add_name(&ps, &prog->params, &prog->nparams);
            if (ps.status) break;
            if (ps.tok.kind == T_COMMA) { lex_next(&ps); continue; }
            break;
        }
        expect(&ps, T_SEMI, "';'");
    }
    if (!ps.status) prog->body = parse_seq(&ps, 1, T_EOF);
    if (!ps.status && ps.tok.kind != T_EOF) fail(&ps, OR_E_PARSE, "unexpected token");
    if (!ps.status && ps.tok.kind == T_BAD) fail(&ps, OR_E_PARSE, "bad character");
    return ps.status;
}

/* ----------------------------------------------------------- evaluator -- */

/* One thread's evaluation state (rules of Fig. 3 with tid substituted,
 * rule par).  Accesses are appended to a growable list. */
typedef struct {
    uint32_t phase;
    uint32_t loc;
    int64_t index;
    uint32_t tid;
    uint32_t write;
} Tuple;

typedef struct {
    Tuple *v; size_t n, cap;
    int nomem;
} TupleVec;

typedef struct {
    const Program *prog;
    const uint64_t *cells;
    const int64_t *params;
    int64_t *vars;          /* loop-variable slots */
    uint32_t tid;
    uint32_t phase;         /* syncs executed so far */
    uint64_t ordinal;       /* accesses completed so far */
    int error;              /* first evaluation error of this thread */
    uint64_t err_ordinal;
    TupleVec *out;          /* NULL: count only */
} Thread;

static void push_tuple(TupleVec *tv, Tuple t)
{
    if (tv->n == tv->cap) {
        size_t cap = tv->cap ? tv->cap * 2 : 1024;
        Tuple *nv = (Tuple *)realloc(tv->v, sizeof(Tuple) * cap);
        if (!nv) { tv->nomem = 1; return; }
        tv->v = nv; tv->cap = cap;
    }
    tv->v[tv->n++] = t;
}

static void set_error(Thread *th, int code)
{
    if (!th->error) { th->error = code; th->err_ordinal = th->ordinal; }
}

/* floor(a / b) for b != 0, or an overflow error for INT64_MIN / -1 */
static int floor_div(int64_t a, int64_t b, int64_t *q)
{
    if (a == INT64_MIN && b == -1) return OR_E_OVERFLOW;
    int64_t t = a / b;               /* C truncates toward zero */
    if ((a % b != 0) && ((a < 0) != (b < 0))) t -= 1;
    *q = t;
    return OR_OK;
}

/* Euclidean remainder: the r in [0, |b|) with a = b*q + r */
static int64_t euclid_mod(int64_t a, int64_t b)
{
    if (b == -1 || b == 1) return 0;
    int64_t r = a % b;
    if (r < 0) r = (b > 0) ? r + b : r - b;
    return r;
}

static int eval_expr(Thread *th, const Expr *e, int64_t *out)
{
    int64_t a, b;
    int st;
    switch (e->kind) {
    case EK_INT: *out = e->value; return OR_OK;
    case EK_TID: *out = (int64_t)th->tid; return OR_OK;
    case EK_VAR: *out = th->vars[e->slot]; return OR_OK;
    case EK_PARAM: *out = th->params[e->slot]; return OR_OK;
    case EK_NEG:
        if ((st = eval_expr(th, e->a, &a))) return st;
        if (a == INT64_MIN) return OR_E_OVERFLOW;
        *out = -a;
        return OR_OK;
    case EK_BIN:
        if ((st = eval_expr(th, e->a, &a))) return st;
        if ((st = eval_expr(th, e->b, &b))) return st;
        switch (e->op) {
        case OP_ADD: return __builtin_add_overflow(a, b, out) ? OR_E_OVERFLOW : OR_OK;
        case OP_SUB: return __builtin_sub_overflow(a, b, out) ? OR_E_OVERFLOW : OR_OK;
        case OP_MUL: return __builtin_mul_overflow(a, b, out) ? OR_E_OVERFLOW : OR_OK;
        case OP_DIV: if (b == 0) return OR_E_DIV_ZERO; return floor_div(a, b, out);
        case OP_MOD: if (b == 0) return OR_E_DIV_ZERO; *out = euclid_mod(a, b); return OR_OK;
        case OP_MIN: *out = a < b ? a : b; return OR_OK;
        case OP_MAX: *out = a > b ? a : b; return OR_OK;
        }
    }
    return OR_E_PARSE;
}

static int eval_cond(Thread *th, const Cond *c, int *out)
{
    int64_t a, b; int l, r, st;
    switch (c->kind) {
    case CK_TRUE: *out = 1; return OR_OK;
    case CK_FALSE: *out = 0; return OR_OK;
    case CK_NOT:
        if ((st = eval_cond(th, c->l, &l))) return st;
        *out = !l; return OR_OK;
    case CK_AND:   /* both sides are evaluated: no short circuit */
        if ((st = eval_cond(th, c->l, &l))) return st;
        if ((st = eval_cond(th, c->r, &r))) return st;
        *out = l && r; return OR_OK;
    case CK_OR:
        if ((st = eval_cond(th, c->l, &l))) return st;
        if ((st = eval_cond(th, c->r, &r))) return st;
        *out = l || r; return OR_OK;
    case CK_CMP:
        if ((st = eval_expr(th, c->a, &a))) return st;
        if ((st = eval_expr(th, c->b, &b))) return st;
        switch (c->rel) {
        case R_EQ: *out = a == b; break;
        case R_NE: *out = a != b; break;
        case R_LT: *out = a < b; break;
        case R_LE: *out = a <= b; break;
        case R_GT: *out = a > b; break;
        case R_GE: *out = a >= b; break;
        }
        return OR_OK;
    }
    return OR_E_PARSE;
}

/* Runs one statement for one thread.  Returns 0 to continue, 1 once the
 * thread has hit an evaluation error (the thread stops there). */
static int run_stmt(Thread *th, const Stmt *s)
{
    int64_t v, lo, hi; int c, st;
    switch (s->kind) {
    case SK_SKIP:                                   /* rule skip */
        return 0;
    case SK_SYNC:                                   /* barrier: next phase */
        th->phase++;
        return 0;
    case SK_ACCESS:                                 /* rules read / write */
        if ((st = eval_expr(th, s->index, &v))) { set_error(th, st); return 1; }
        if (v < 0 || (uint64_t)v >= th->cells[s->loc]) { set_error(th, OR_E_INDEX_OOB); return 1; }
        if (th->out) {
            Tuple t = { th->phase, (uint32_t)s->loc, v, th->tid, (uint32_t)s->write };
            push_tuple(th->out, t);
        }
        th->ordinal++;
        return 0;
    case SK_SEQ:                                    /* rule seq */
        for (int i = 0; i < s->nitems; i++)
            if (run_stmt(th, s->items[i])) return 1;
        return 0;
    case SK_IF:                                     /* rules if-t / if-f */
        if ((st = eval_cond(th, s->cond, &c))) { set_error(th, st); return 1; }
        return run_stmt(th, c ? s->then_s : s->else_s);
    case SK_FOR_U:
    case SK_FOR_S:                                  /* rules for-1 / for-2 */
        if ((st = eval_expr(th, s->lo, &lo))) { set_error(th, st); return 1; }
        if ((st = eval_expr(th, s->hi, &hi))) { set_error(th, st); return 1; }
        for (int64_t x = lo; x < hi; x++) {
            th->vars[s->slot] = x;
            if (run_stmt(th, s->body)) return 1;
        }
        return 0;
    }
    return 0;
}

/* ------------------------------------------------------------- checkers -- */

typedef struct {
    uint32_t nthreads, nlocs, nparams;
    const uint64_t *cells;
    const int64_t *params;
} Bounds;

/* All threads' histories.  tuples: every access of every thread, in program
 * order per thread, threads in tid order.  syncs[t]: syncs thread t ran. */
typedef struct {
    TupleVec tv;
    uint32_t *syncs;
    int status;
    uint32_t err_tid;
    uint64_t err_ordinal;
    uint64_t total;        /* dynamic accesses, all threads */
} History;

static int run_all(const Program *prog, const Bounds *b, History *h, int keep_tuples)
{
    memset(h, 0, sizeof *h);
    h->syncs = (uint32_t *)calloc(b->nthreads ? b->nthreads : 1, sizeof(uint32_t));
    int64_t *vars = (int64_t *)calloc((size_t)(prog->nslots ? prog->nslots : 1), sizeof(int64_t));
    if (!h->syncs || !vars) { free(vars); return OR_E_NOMEM; }
    for (uint32_t t = 0; t < b->nthreads; t++) {            /* rule par */
        Thread th; memset(&th, 0, sizeof th);
        th.prog = prog; th.cells = b->cells; th.params = b->params; th.vars = vars;
        th.tid = t; th.out = keep_tuples ? &h->tv : NULL;
        run_stmt(&th, prog->body);
        if (h->tv.nomem) { free(vars); return OR_E_NOMEM; }
        h->syncs[t] = th.phase;
        h->total += th.ordinal;
        if (th.error && h->status == OR_OK) {               /* smallest failing tid */
            h->status = th.error; h->err_tid = t; h->err_ordinal = th.err_ordinal;
        }
    }
    free(vars);
    return OR_OK;
}

static void history_free(History *h)
{
    free(h->tv.v); free(h->syncs);
    memset(h, 0, sizeof *h);
}

/* -- method A: Definition 1 over every ordered pair of distinct threads -- */

typedef struct { uint32_t phase, loc, write; int64_t index; } Acc;

static int acc_cmp(const void *x, const void *y)
{
    const Acc *a = (const Acc *)x, *b = (const Acc *)y;
    if (a->phase != b->phase) return a->phase < b->phase ? -1 : 1;
    if (a->loc != b->loc) return a->loc < b->loc ? -1 : 1;
    if (a->write != b->write) return a->write < b->write ? -1 : 1;
    if (a->index != b->index) return a->index < b->index ? -1 : 1;
    return 0;
}

/* range [lo, hi) of thread-sorted accesses with the given (phase, loc, write) */
static void acc_range(const Acc *v, size_t n, uint32_t phase, uint32_t loc, uint32_t write, size_t *lo, size_t *hi)
{
    Acc key = { phase, loc, write, INT64_MIN };
    size_t a = 0, b = n;
    while (a < b) { size_t m = (a + b) / 2; if (acc_cmp(&v[m], &key) < 0) a = m + 1; else b = m; }
    *lo = a;
    key.index = INT64_MAX;
    b = n;
    while (a < b) { size_t m = (a + b) / 2; if (acc_cmp(&v[m], &key) <= 0) a = m + 1; else b = m; }
    *hi = a;
}

static int in_sorted(const Acc *v, size_t lo, size_t hi, int64_t x)
{
    size_t end = hi;
    while (lo < hi) { size_t m = (lo + hi) / 2; if (v[m].index < x) lo = m + 1; else hi = m; }
    return lo < end && v[lo].index == x;
}

/* Smallest j in W1 that is also in R2 or W2 (all sorted, duplicate-free);
 * returns 0 if the intersection is empty. */
static int first_common(const Acc *w1, size_t nw1, const Acc *r2, size_t nr2, const Acc *w2, size_t nw2, int64_t *j)
{
    size_t a = 0, b = 0, c = 0;
    while (a < nw1) {
        int64_t x = w1[a].index;
        while (b < nr2 && r2[b].index < x) b++;
        while (c < nw2 && w2[c].index < x) c++;
        if ((b < nr2 && r2[b].index == x) || (c < nw2 && w2[c].index == x)) { *j = x; return 1; }
        a++;
    }
    return 0;
}

static int check_pairs(const Program *prog, const Bounds *b, History *h, oracle_result *out)
{
    uint32_t T = b->nthreads;
    /* H per thread: the set of (phase, loc, mode, index) it touched */
    Acc **per = (Acc **)calloc(T ? T : 1, sizeof(Acc *));
    size_t *cnt = (size_t *)calloc(T ? T : 1, sizeof(size_t));
    if (!per || !cnt) { free(per); free(cnt); return OR_E_NOMEM; }
    size_t pos = 0;
    uint32_t maxphase = 0;
    for (uint32_t t = 0; t < T; t++) {
        size_t start = pos;
        while (pos < h->tv.n && h->tv.v[pos].tid == t) pos++;
        size_t n = pos - start;
        per[t] = (Acc *)malloc(sizeof(Acc) * (n ? n : 1));
        if (!per[t]) { for (uint32_t u = 0; u < t; u++) free(per[u]); free(per); free(cnt); return OR_E_NOMEM; }
        for (size_t i = 0; i < n; i++) {
            const Tuple *tp = &h->tv.v[start + i];
            per[t][i].phase = tp->phase; per[t][i].loc = tp->loc;
            per[t][i].write = tp->write; per[t][i].index = tp->index;
            if (tp->phase > maxphase) maxphase = tp->phase;
        }
        qsort(per[t], n, sizeof(Acc), acc_cmp);
        size_t u = 0;                         /* R and W are sets: drop repeats */
        for (size_t i = 0; i < n; i++)
            if (u == 0 || acc_cmp(&per[t][u - 1], &per[t][i]) != 0) per[t][u++] = per[t][i];
        cnt[t] = u;
    }
    (void)prog;
    int found = 0;
    for (uint32_t ph = 0; ph <= maxphase && !found; ph++) {
        for (uint32_t l = 0; l < b->nlocs && !found; l++) {
            int have = 0; int64_t bj = 0; uint32_t bi = 0, bk = 0;
            for (uint32_t i1 = 0; i1 < T; i1++) {
                size_t w1lo, w1hi;
                acc_range(per[i1], cnt[i1], ph, l, 1, &w1lo, &w1hi);
                if (w1lo == w1hi) continue;
                for (uint32_t i2 = 0; i2 < T; i2++) {
                    if (i2 == i1) continue;
                    size_t r2lo, r2hi, w2lo, w2hi;
                    acc_range(per[i2], cnt[i2], ph, l, 0, &r2lo, &r2hi);
                    acc_range(per[i2], cnt[i2], ph, l, 1, &w2lo, &w2hi);
                    int64_t j;
                    if (!first_common(per[i1] + w1lo, w1hi - w1lo, per[i2] + r2lo, r2hi - r2lo,
                                      per[i2] + w2lo, w2hi - w2lo, &j)) continue;
                    uint32_t lo = i1 < i2 ? i1 : i2, hi = i1 < i2 ? i2 : i1;
                    if (!have || j < bj || (j == bj && (lo < bi || (lo == bi && hi < bk)))) {
                        have = 1; bj = j; bi = lo; bk = hi;
                    }
                }
            }
            if (have) {
                size_t wlo, whi;
                found = 1;
                out->verdict = V_RACY;
                out->phase = ph; out->loc = l; out->index = (uint64_t)bj;
                out->tid_i = bi; out->tid_j = bk;
                acc_range(per[bi], cnt[bi], ph, l, 1, &wlo, &whi);
                out->i_writes = (uint32_t)in_sorted(per[bi], wlo, whi, bj);
                acc_range(per[bk], cnt[bk], ph, l, 1, &wlo, &whi);
                out->j_writes = (uint32_t)in_sorted(per[bk], wlo, whi, bj);
            }
        }
    }
    for (uint32_t t = 0; t < T; t++) free(per[t]);
    free(per); free(cnt);
    if (!found) out->verdict = V_DRF;
    return OR_OK;
}

/* -- method B: per-cell owner records over accesses grouped by cell -- */

static int tuple_cell_cmp(const void *x, const void *y)
{
    const Tuple *a = (const Tuple *)x, *b = (const Tuple *)y;
    if (a->phase != b->phase) return a->phase < b->phase ? -1 : 1;
    if (a->loc != b->loc) return a->loc < b->loc ? -1 : 1;
    if (a->index != b->index) return a->index < b->index ? -1 : 1;
    return 0;
}

#define NONE 0xFFFFFFFFu

/* keep the two smallest distinct values seen */
static void two_smallest(uint32_t *first, uint32_t *second, uint32_t x)
{
    if (x == *first || x == *second) return;
    if (x < *first) { *second = *first; *first = x; }
    else if (x < *second) *second = x;
}

static int check_cells(History *h, oracle_result *out)
{
    Tuple *v = h->tv.v;
    size_t n = h->tv.n;
    qsort(v, n, sizeof(Tuple), tuple_cell_cmp);
    out->verdict = V_DRF;
    size_t i = 0;
    while (i < n) {
        size_t j = i;
        uint32_t t0 = NONE, t1 = NONE, w0 = NONE, w1 = NONE;
        while (j < n && tuple_cell_cmp(&v[i], &v[j]) == 0) {
            two_smallest(&t0, &t1, v[j].tid);
            if (v[j].write) two_smallest(&w0, &w1, v[j].tid);
            j++;
        }
        /* a writer plus a second distinct accessor is a racing pair */
        if (w0 != NONE && t1 != NONE) {
            out->verdict = V_RACY;
            out->phase = v[i].phase; out->loc = v[i].loc; out->index = (uint64_t)v[i].index;
            out->tid_i = t0;
            if (w0 == t0) {           /* t0 writes: its smallest partner is t1 */
                out->tid_j = t1; out->i_writes = 1; out->j_writes = (w1 == t1);
            } else {                  /* t0 only reads: its partner must write */
                out->tid_j = w0; out->i_writes = 0; out->j_writes = 1;
            }
            return OR_OK;
        }
        i = j;
    }
    return OR_OK;
}

/* ------------------------------------------------------------ entry points */

static int check_bounds(const Program *prog, const Bounds *b, char *msg, int msglen)
{
    if ((int)b->nlocs != prog->narrays || (int)b->nparams != prog->nparams) {
        if (msg && msglen > 0)
            snprintf(msg, (size_t)msglen, "protocol declares %d arrays and %d params, bounds give %u and %u",
                     prog->narrays, prog->nparams, b->nlocs, b->nparams);
        return OR_E_INVALID_ARG;
    }
    if ((b->nlocs && !b->cells) || (b->nparams && !b->params)) return OR_E_INVALID_ARG;
    return OR_OK;
}

/* method: 0 = A (pairs, Definition 1 literally), 1 = B (per-cell records),
 * 2 = evaluation only (status, tuples, syncs; no race check). */
int oracle_check(const char *text, uint32_t nthreads, uint32_t nlocs, const uint64_t *cells,
                 uint32_t nparams, const int64_t *params, int method, oracle_result *out,
                 char *msg, int msglen)
{
    if (!text || !out) return OR_E_INVALID_ARG;
    memset(out, 0, sizeof *out);
    out->verdict = -1;
    Program prog;
    int st = parse_program(text, &prog, msg, msglen);
    if (st) { program_free(&prog); out->status = st; return st; }
    Bounds b = { nthreads, nlocs, nparams, cells, params };
    st = check_bounds(&prog, &b, msg, msglen);
    if (st) { program_free(&prog); out->status = st; return st; }
    History h;
    st = run_all(&prog, &b, &h, method != 2);
    if (st) { history_free(&h); program_free(&prog); out->status = st; return st; }
    out->tuples = h.total;
    if (h.status) {                              /* evaluation error wins */
        out->status = h.status; out->err_tid = h.err_tid; out->err_ordinal = h.err_ordinal;
        history_free(&h); program_free(&prog);
        return out->status;
    }
    out->phases = nthreads ? h.syncs[0] + 1 : 0;
    for (uint32_t t = 0; t < nthreads; t++) {    /* barrier divergence next */
        if (h.syncs[t] != h.syncs[0]) {
            out->verdict = V_DIVERGENCE;
            out->div_tid = t; out->sync_count_0 = h.syncs[0]; out->sync_count_div = h.syncs[t];
            history_free(&h); program_free(&prog);
            return OR_OK;
        }
    }
    out->sync_count_0 = nthreads ? h.syncs[0] : 0;
    if (method == 0) st = check_pairs(&prog, &b, &h, out);
    else if (method == 1) st = check_cells(&h, out);
    else out->verdict = V_DRF;
    history_free(&h); program_free(&prog);
    out->status = st;
    return st;
}

/* Every access of every thread, as rows of five u64: phase, loc, index, tid,
 * mode (1 = write).  Returns the number of accesses (rows written up to cap),
 * or a negative status. */
int64_t oracle_tuples(const char *text, uint32_t nthreads, uint32_t nlocs, const uint64_t *cells,
                      uint32_t nparams, const int64_t *params, uint64_t *rows, int64_t cap,
                      char *msg, int msglen)
{
    Program prog;
    int st = parse_program(text, &prog, msg, msglen);
    if (st) { program_free(&prog); return st; }
    Bounds b = { nthreads, nlocs, nparams, cells, params };
    st = check_bounds(&prog, &b, msg, msglen);
    if (st) { program_free(&prog); return st; }
    History h;
    st = run_all(&prog, &b, &h, 1);
    if (st || h.status) { int r = st ? st : h.status; history_free(&h); program_free(&prog); return r; }
    int64_t n = (int64_t)h.tv.n;
    for (int64_t i = 0; i < n && i < cap; i++) {
        const Tuple *t = &h.tv.v[i];
        rows[5 * i + 0] = t->phase; rows[5 * i + 1] = t->loc; rows[5 * i + 2] = (uint64_t)t->index;
        rows[5 * i + 3] = t->tid; rows[5 * i + 4] = t->write;
    }
    history_free(&h); program_free(&prog);
    return n;
}

/* Every thread's accesses to one cell (phase, loc, index), without storing
 * the others: the two smallest distinct accessor tids and the two smallest
 * distinct writer tids (0xFFFFFFFF when absent), the number of accesses to
 * the cell and the total number of accesses.  For checking a witness of a
 * protocol too large to check whole. */
typedef struct {
    uint32_t t0, t1, w0, w1;
    uint64_t cell_accesses;
    uint64_t total;
    int32_t status;
    uint32_t pad;
} oracle_cell_result;

static void cell_visit(const Tuple *t, uint32_t phase, uint32_t loc, int64_t index, oracle_cell_result *r)
{
    if (t->phase != phase || t->loc != loc || t->index != index) return;
    two_smallest(&r->t0, &r->t1, t->tid);
    if (t->write) two_smallest(&r->w0, &r->w1, t->tid);
    r->cell_accesses++;
}

int oracle_cell(const char *text, uint32_t nthreads, uint32_t nlocs, const uint64_t *cells, uint32_t nparams,
                const int64_t *params, uint32_t phase, uint32_t loc, uint64_t index, oracle_cell_result *out,
                char *msg, int msglen)
{
    memset(out, 0, sizeof *out);
    out->t0 = out->t1 = out->w0 = out->w1 = NONE;
    Program prog;
    int st = parse_program(text, &prog, msg, msglen);
    if (st) { program_free(&prog); out->status = st; return st; }
    Bounds b = { nthreads, nlocs, nparams, cells, params };
    st = check_bounds(&prog, &b, msg, msglen);
    if (st) { program_free(&prog); out->status = st; return st; }
    int64_t *vars = (int64_t *)calloc((size_t)(prog.nslots ? prog.nslots : 1), sizeof(int64_t));
    TupleVec tv; memset(&tv, 0, sizeof tv);
    if (!vars) { program_free(&prog); out->status = OR_E_NOMEM; return OR_E_NOMEM; }
    for (uint32_t t = 0; t < nthreads && !out->status; t++) {   /* one thread at a time */
        Thread th; memset(&th, 0, sizeof th);
        th.prog = &prog; th.cells = cells; th.params = params; th.vars = vars;
        th.tid = t; th.out = &tv;
        tv.n = 0;
        run_stmt(&th, prog.body);
        if (tv.nomem) { out->status = OR_E_NOMEM; break; }
        if (th.error) { out->status = th.error; break; }
        for (size_t i = 0; i < tv.n; i++) cell_visit(&tv.v[i], phase, loc, (int64_t)index, out);
        out->total += th.ordinal;
    }
    free(tv.v); free(vars); program_free(&prog);
    return out->status;
}

/* Parse and validate only: 0 or the validation status, and the declared
 * array and param counts. */
int oracle_validate(const char *text, int *narrays, int *nparams, char *msg, int msglen)
{
    Program prog;
    int st = parse_program(text, &prog, msg, msglen);
    if (narrays) *narrays = prog.narrays;
    if (nparams) *nparams = prog.nparams;
    program_free(&prog);
    return st;
}

/* ------------------------------------------- method B on several cores -- */

/* A driver that runs the same steps as oracle_check's method B on several
 * host threads, for the CPU baseline and for protocols with hundreds of
 * millions of accesses.  It changes nothing in what is computed:
 *   1. rule par: each worker runs run_stmt for a contiguous range of thread
 *      ids (the threads are independent by that rule), keeping its own
 *      accesses, sync counts and first error;
 *   2. the evaluation error of the smallest failing tid wins, then barrier
 *      divergence against thread 0, exactly as in oracle_check;
 *   3. the accesses are grouped into shards of consecutive cells in the
 *      lexicographic order (phase, array, index) -- per (phase, array), the
 *      index range cut into equal chunks -- and each shard is checked like
 *      check_cells does (sort by cell, per-cell two smallest accessors and
 *      writers).  Cells never span two shards, so every cell's verdict is
 *      the one method B gives it, and the first racy cell of the first shard
 *      that has one is the lexicographically smallest racy cell.
 * Needs POSIX threads. */
#include <pthread.h>

typedef struct {
    const Program *prog;
    const Bounds *b;
    uint32_t t_lo, t_hi;
    uint32_t *syncs;           /* shared, indexed by tid */
    TupleVec tv;
    int error;                 /* first error of the smallest failing tid of the range */
    uint32_t err_tid;
    uint64_t err_ordinal;
    uint64_t total;
    int status;                /* OR_E_NOMEM */
} EvalJob;

static void *eval_worker(void *arg)
{
    EvalJob *j = (EvalJob *)arg;
    int64_t *vars = (int64_t *)calloc((size_t)(j->prog->nslots ? j->prog->nslots : 1), sizeof(int64_t));
    if (!vars) { j->status = OR_E_NOMEM; return NULL; }
    for (uint32_t t = j->t_lo; t < j->t_hi; t++) {
        Thread th; memset(&th, 0, sizeof th);
        th.prog = j->prog; th.cells = j->b->cells; th.params = j->b->params; th.vars = vars;
        th.tid = t; th.out = &j->tv;
        run_stmt(&th, j->prog->body);
        if (j->tv.nomem) { j->status = OR_E_NOMEM; break; }
        j->syncs[t] = th.phase;
        j->total += th.ordinal;
        if (th.error && !j->error) { j->error = th.error; j->err_tid = t; j->err_ordinal = th.err_ordinal; }
    }
    free(vars);
    return NULL;
}

typedef struct {
    uint32_t nlocs;
    uint64_t chunk[64];        /* index range of one shard, per array */
    uint32_t per_loc[64];      /* shards per (phase, array) */
    uint32_t base[64];         /* first shard of an array within a phase */
    uint32_t per_phase;        /* shards per phase */
} ShardMap;

static uint32_t shard_of(const ShardMap *m, const Tuple *t)
{
    return t->phase * m->per_phase + m->base[t->loc] + (uint32_t)((uint64_t)t->index / m->chunk[t->loc]);
}

typedef struct {
    EvalJob *jobs; int njobs;
    const ShardMap *map;
    uint64_t *offs;            /* [job][shard]: where this job's tuples of the shard go */
    uint32_t nshards;
    Tuple *all;
    int w;                     /* this worker */
    /* shard checking */
    uint64_t *start;           /* [nshards + 1] */
    uint32_t *next;            /* shared shard counter */
    pthread_mutex_t *mu;
    oracle_result *shard_res;  /* one per shard; verdict -1 = not racy */
} CellJob;

static void *count_worker(void *arg)
{
    CellJob *c = (CellJob *)arg;
    const EvalJob *j = &c->jobs[c->w];
    uint64_t *cnt = c->offs + (size_t)c->w * c->nshards;
    for (size_t i = 0; i < j->tv.n; i++) cnt[shard_of(c->map, &j->tv.v[i])]++;
    return NULL;
}

static void *scatter_worker(void *arg)
{
    CellJob *c = (CellJob *)arg;
    EvalJob *j = &c->jobs[c->w];
    uint64_t *off = c->offs + (size_t)c->w * c->nshards;
    for (size_t i = 0; i < j->tv.n; i++) c->all[off[shard_of(c->map, &j->tv.v[i])]++] = j->tv.v[i];
    return NULL;
}

static void *shard_worker(void *arg)
{
    CellJob *c = (CellJob *)arg;
    for (;;) {
        pthread_mutex_lock(c->mu);
        uint32_t s = (*c->next)++;
        pthread_mutex_unlock(c->mu);
        if (s >= c->nshards) return NULL;
        History h; memset(&h, 0, sizeof h);
        h.tv.v = c->all + c->start[s];
        h.tv.n = (size_t)(c->start[s + 1] - c->start[s]);
        oracle_result r; memset(&r, 0, sizeof r);
        check_cells(&h, &r);             /* sorts the shard in place */
        if (r.verdict != V_RACY) r.verdict = -1;
        c->shard_res[s] = r;
    }
}

/* Method B on `workers` host threads (0: one).  Same result as
 * oracle_check(..., method 1, ...). */
int oracle_check_mt(const char *text, uint32_t nthreads, uint32_t nlocs, const uint64_t *cells,
                    uint32_t nparams, const int64_t *params, int workers, oracle_result *out,
                    char *msg, int msglen)
{
    if (!text || !out) return OR_E_INVALID_ARG;
    memset(out, 0, sizeof *out);
    out->verdict = -1;
    if (workers < 1) workers = 1;
    if (workers > 1024) workers = 1024;
    if ((uint32_t)workers > nthreads && nthreads) workers = (int)nthreads;
    Program prog;
    int st = parse_program(text, &prog, msg, msglen);
    if (st) { program_free(&prog); out->status = st; return st; }
    Bounds b = { nthreads, nlocs, nparams, cells, params };
    st = check_bounds(&prog, &b, msg, msglen);
    if (!st && nlocs > 64) st = OR_E_INVALID_ARG;
    if (st) { program_free(&prog); out->status = st; return st; }

    uint32_t *syncs = (uint32_t *)calloc(nthreads ? nthreads : 1, sizeof(uint32_t));
    EvalJob *jobs = (EvalJob *)calloc((size_t)workers, sizeof(EvalJob));
    pthread_t *th = (pthread_t *)calloc((size_t)workers, sizeof(pthread_t));
    if (!syncs || !jobs || !th) { free(syncs); free(jobs); free(th); program_free(&prog); return out->status = OR_E_NOMEM; }
    /* 1. rule par over contiguous tid ranges */
    for (int w = 0; w < workers; w++) {
        jobs[w].prog = &prog; jobs[w].b = &b; jobs[w].syncs = syncs;
        jobs[w].t_lo = (uint32_t)((uint64_t)nthreads * (uint64_t)w / (uint64_t)workers);
        jobs[w].t_hi = (uint32_t)((uint64_t)nthreads * (uint64_t)(w + 1) / (uint64_t)workers);
        pthread_create(&th[w], NULL, eval_worker, &jobs[w]);
    }
    for (int w = 0; w < workers; w++) pthread_join(th[w], NULL);
    uint64_t total = 0, n = 0;
    int error = 0; uint32_t err_tid = 0; uint64_t err_ord = 0;
    for (int w = 0; w < workers; w++) {
        if (jobs[w].status) st = jobs[w].status;
        total += jobs[w].total;
        n += jobs[w].tv.n;
        if (jobs[w].error && !error) { error = jobs[w].error; err_tid = jobs[w].err_tid; err_ord = jobs[w].err_ordinal; }
    }
    Tuple *all = NULL;
    uint64_t *offs = NULL, *start = NULL;
    oracle_result *shard_res = NULL;
    if (st) goto done;
    out->tuples = total;
    /* 2. evaluation error, then barrier divergence */
    if (error) {
        out->status = error; out->err_tid = err_tid; out->err_ordinal = err_ord;
        st = error;
        goto done;
    }
    out->phases = nthreads ? syncs[0] + 1 : 0;
    for (uint32_t t = 0; t < nthreads; t++) {
        if (syncs[t] != syncs[0]) {
            out->verdict = V_DIVERGENCE;
            out->div_tid = t; out->sync_count_0 = syncs[0]; out->sync_count_div = syncs[t];
            goto done;
        }
    }
    out->sync_count_0 = nthreads ? syncs[0] : 0;
    out->verdict = V_DRF;
    if (n == 0) goto done;
    {
        /* 3. shards of consecutive cells, (phase, array, index) order */
        ShardMap m; memset(&m, 0, sizeof m);
        m.nlocs = nlocs;
        uint64_t cells_total = 0;
        for (uint32_t l = 0; l < nlocs; l++) cells_total += cells[l];
        const uint32_t phases = syncs[0] + 1;
        /* every (phase, array) cut into chunks: the accesses of one phase
           may all fall into a single array, so each phase alone gets enough
           shards to keep every worker busy */
        const uint64_t per_phase_want = (uint64_t)workers * 16;
        for (uint32_t l = 0; l < nlocs; l++) {
            uint64_t k = cells_total ? (per_phase_want * cells[l] + cells_total - 1) / cells_total : 1;
            if (k < 1) k = 1;
            if (k > 4096) k = 4096;
            m.chunk[l] = (cells[l] + k - 1) / k;
            if (m.chunk[l] == 0) m.chunk[l] = 1;
            m.per_loc[l] = (uint32_t)((cells[l] + m.chunk[l] - 1) / m.chunk[l]);
            if (m.per_loc[l] == 0) m.per_loc[l] = 1;
            m.base[l] = m.per_phase;
            m.per_phase += m.per_loc[l];
        }
        const uint32_t nshards = phases * m.per_phase;
        all = (Tuple *)malloc(sizeof(Tuple) * (size_t)n);
        offs = (uint64_t *)calloc((size_t)workers * nshards, sizeof(uint64_t));
        start = (uint64_t *)calloc((size_t)nshards + 1, sizeof(uint64_t));
        shard_res = (oracle_result *)calloc(nshards, sizeof(oracle_result));
        if (!all || !offs || !start || !shard_res) { st = OR_E_NOMEM; goto done; }
        CellJob *cj = (CellJob *)calloc((size_t)workers, sizeof(CellJob));
        if (!cj) { st = OR_E_NOMEM; goto done; }
        pthread_mutex_t mu = PTHREAD_MUTEX_INITIALIZER;
        uint32_t next = 0;
        for (int w = 0; w < workers; w++) {
            cj[w] = (CellJob){ jobs, workers, &m, offs, nshards, all, w, start, &next, &mu, shard_res };
            pthread_create(&th[w], NULL, count_worker, &cj[w]);
        }
        for (int w = 0; w < workers; w++) pthread_join(th[w], NULL);
        uint64_t run = 0;
        for (uint32_t s = 0; s < nshards; s++) {
            start[s] = run;
            for (int w = 0; w < workers; w++) {
                uint64_t c = offs[(size_t)w * nshards + s];
                offs[(size_t)w * nshards + s] = run;
                run += c;
            }
        }
        start[nshards] = run;
        for (int w = 0; w < workers; w++) pthread_create(&th[w], NULL, scatter_worker, &cj[w]);
        for (int w = 0; w < workers; w++) pthread_join(th[w], NULL);
        for (int w = 0; w < workers; w++) { free(jobs[w].tv.v); jobs[w].tv.v = NULL; jobs[w].tv.n = 0; }
        for (int w = 0; w < workers; w++) pthread_create(&th[w], NULL, shard_worker, &cj[w]);
        for (int w = 0; w < workers; w++) pthread_join(th[w], NULL);
        free(cj);
        for (uint32_t s = 0; s < nshards; s++) {
            const oracle_result *r = &shard_res[s];
            if (r->verdict != V_RACY) continue;
            out->verdict = V_RACY;
            out->phase = r->phase; out->loc = r->loc; out->index = r->index;
            out->tid_i = r->tid_i; out->tid_j = r->tid_j;
            out->i_writes = r->i_writes; out->j_writes = r->j_writes;
            break;
        }
    }
done:
    if (st == OR_E_NOMEM) { out->status = st; out->verdict = -1; }
    for (int w = 0; w < workers; w++) free(jobs[w].tv.v);
    free(jobs); free(th); free(syncs); free(all); free(offs); free(start); free(shard_res);
    program_free(&prog);
    return st;
}
