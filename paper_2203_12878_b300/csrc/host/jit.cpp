// Run-time specialization (see jit.h): code generation, NVRTC, loading.
#include "jit.h"

#include <dlfcn.h>
#include <nvrtc.h>

#include <cstring>
#include <map>
#include <mutex>
#include <sstream>

#include "engine.h"
#include "jit_headers.inc"   // generated by the build: the shared headers as text

namespace drf {
namespace {

constexpr size_t kMaxShapes = 64;           // distinct item shapes one protocol may specialize
constexpr size_t kMaxSourceBytes = 4 << 20;  // generated source

std::string lit64(int64_t v)
{
    if (v == INT64_MIN) return "(-9223372036854775807LL - 1)";
    return std::to_string(v) + "LL";
}

std::string ulit(uint64_t v) { return std::to_string(v) + "ull"; }

// The text of one shared header, without its #pragma once and quoted includes
// (the generated source inlines the headers itself, in dependency order).
std::string header_text(const char *h)
{
    std::istringstream in(h);
    std::ostringstream out;
    std::string line;
    while (std::getline(in, line)) {
        if (line.rfind("#pragma once", 0) == 0 || line.rfind("#include \"", 0) == 0) continue;
        out << line << "\n";
    }
    return out.str();
}

enum Mode { GM_COUNT, GM_TABLE, GM_CELL };

struct ShapeKey {
    uint32_t start, stop, nsplit, chunked;
    uint32_t split_pc[kMaxSplit];
    bool operator<(const ShapeKey &o) const { return std::memcmp(this, &o, sizeof o) < 0; }
};

class Gen {
  public:
    Gen(const Prepared &p, const DevProto &d, const std::vector<uint64_t> &cbase)
        : p_(p), d_(d), cbase_(cbase), V_(p.wide ? "int64_t" : "int32_t"),
          U_(p.wide ? "uint64_t" : "uint32_t")
    {
    }

    std::string error;

    // One device function per (shape, mode).
    bool shape_fn(const ShapeKey &k, uint32_t id, Mode m, std::ostringstream &o)
    {
        mode_ = m;
        body_.str("");
        tmp_ = 0;
        const char *name[] = {"count", "table", "cell"};
        o << "static __device__ __forceinline__ void s" << id << "_" << name[m] << "(";
        if (m == GM_COUNT) o << "const drf::ItemDesc &it, uint32_t tid, uint32_t &count, uint32_t &syncs, uint32_t &err)";
        if (m == GM_TABLE)
            o << "const drf::BatchArgs &a, const drf::ItemDesc &it, uint32_t tid, uint32_t phase, "
                 "unsigned long long &last_bid)";
        if (m == GM_CELL) o << "const drf::ItemDesc &it, uint32_t tid, uint32_t phase, const CellTarget &tg, uint32_t &hit)";
        o << "\n{\n";
        o << "    " << V_ << " v[" << kMaxVars << "], h[" << kMaxVars << "];\n";
        o << "    (void)tid; (void)it;\n";
        // prologue: the split loops at this item's iterations
        for (uint32_t l = 0; l < k.nsplit; l++) {
            const Insn &L = p_.insns.at(k.split_pc[l]);
            if (L.op != I_LOOP && L.op != I_FASTLOOP) return fail("split level is not a loop");
            body_ << "    {\n";
            std::string lo = expr(L.c), hi = expr(L.d);
            if (!error.empty()) return false;
            body_ << "        const " << V_ << " lo = " << lo << ", hi = " << hi << ";\n";
            body_ << "        const uint64_t trip = lo < hi ? (uint64_t)(" << U_ << ")((" << U_ << ")hi - (" << U_
                  << ")lo) : 0;\n";
            const std::string va = "v[" + std::to_string(L.a) + "]", ha = "h[" + std::to_string(L.a) + "]";
            if (k.chunked && l + 1 == k.nsplit) {
                body_ << "        const uint64_t start = (uint64_t)it.j[" << l << "] * it.chunk;\n";
                body_ << "        if (trip <= start) goto done;\n";
                body_ << "        " << va << " = (" << V_ << ")((" << U_ << ")lo + (" << U_ << ")start);\n";
                body_ << "        " << ha << " = (trip - start > it.chunk) ? (" << V_ << ")((" << U_ << ")" << va
                      << " + (" << U_ << ")it.chunk) : hi;\n";
            } else {
                body_ << "        if (trip <= it.j[" << l << "]) goto done;\n";
                body_ << "        " << va << " = (" << V_ << ")((" << U_ << ")lo + (" << U_ << ")it.j[" << l << "]);\n";
            }
            body_ << "    }\n";
        }
        // the code range [start, stop); reaching stop ends the item
        for (uint32_t pc = k.start; pc < k.stop;) {
            const Insn &in = p_.insns.at(pc);
            if (in.op == I_FASTACC) return fail("stray fast access");
            body_ << "L" << pc << ":;\n";
            uint32_t next = pc + 1;
            if (!insn(k, pc, in, next)) return false;
            pc = next;
        }
        body_ << "L" << k.stop << ":;\n";
        body_ << "done:;\n";
        for (uint32_t t : targets_)
            if (t < k.start || t > k.stop || labels_skip_.count(t)) return fail("jump target outside the item");
        targets_.clear();
        labels_skip_.clear();
        o << body_.str() << "}\n\n";
        return error.empty();
    }

  private:
    const Prepared &p_;
    const DevProto &d_;
    const std::vector<uint64_t> &cbase_;
    const char *V_, *U_;
    Mode mode_ = GM_COUNT;
    std::ostringstream body_;
    int tmp_ = 0;
    std::vector<uint32_t> targets_;
    std::map<uint32_t, bool> labels_skip_;

    bool fail(const std::string &m)
    {
        if (error.empty()) error = m;
        return false;
    }

    std::string fail_div0() const { return mode_ == GM_COUNT ? "{ err = 2u; goto done; }" : "goto done;"; }

    std::string temp(const std::string &e)
    {
        std::string n = "t" + std::to_string(tmp_++);
        body_ << "        const " << V_ << " " << n << " = " << e << ";\n";
        return n;
    }

    std::string cast(const std::string &e) const { return std::string("(") + V_ + ")(" + e + ")"; }
    std::string u(const std::string &e) const { return std::string("(") + U_ + ")" + e; }

    // Statements computing the expression code at `off` (stack machine of
    // devprog.h); returns the C expression of its value.  Division or
    // remainder by a zero operand jumps to the failure exit.
    std::string expr(int32_t off)
    {
        std::vector<std::string> st;
        size_t i = (size_t)off;
        for (int guard = 0; guard < 1 << 16; guard++) {
            if (i >= p_.xcode.size()) { fail("expression code out of range"); return "0"; }
            const uint64_t w = p_.xcode[i++];
            const uint32_t op = (uint32_t)(w & 0xff);
            auto pop = [&]() {
                std::string s = st.empty() ? std::string("0") : st.back();
                if (st.empty()) fail("expression stack underflow");
                else st.pop_back();
                return s;
            };
            switch (op) {
            case X_RET: return st.empty() ? (fail("empty expression"), std::string("0")) : st.back();
            case X_CONST: st.push_back(cast(lit64((int64_t)p_.xcode.at(i++)))); break;
            case X_TID: st.push_back(cast("tid")); break;
            case X_VAR: st.push_back("v[" + std::to_string((uint32_t)(w >> 8)) + "]"); break;
            case X_AFF: {
                const uint32_t n = (uint32_t)(w >> 8);
                std::string e = "(" + u("0");
                for (uint32_t t = 0; t < n; t++) {
                    const uint32_t reg = (uint32_t)p_.xcode.at(i++);
                    const uint64_t coef = p_.xcode.at(i++);
                    const std::string v = reg == kAffTid ? u("tid") : u("v[" + std::to_string(reg) + "]");
                    e += " + " + u("(" + ulit(coef) + ")") + " * " + v;
                }
                e += " + " + u("(" + ulit(p_.xcode.at(i++)) + ")") + ")";
                st.push_back(temp(cast(e)));
                break;
            }
            case X_ADD: case X_SUB: case X_MUL: {
                std::string b = pop(), a = pop();
                const char *o = op == X_ADD ? " + " : op == X_SUB ? " - " : " * ";
                st.push_back(temp(cast(u(a) + o + u(b))));
                break;
            }
            case X_MIN: case X_MAX: {
                std::string b = pop(), a = pop();
                st.push_back(temp("(" + b + (op == X_MIN ? " < " : " > ") + a + " ? " + b + " : " + a + ")"));
                break;
            }
            case X_NEG: { std::string a = pop(); st.push_back(temp(cast(u("0") + " - " + u(a)))); break; }
            case X_DIV: case X_MOD: {
                std::string b = pop(), a = pop();
                body_ << "        if (" << b << " == 0) " << fail_div0() << "\n";
                st.push_back(temp(std::string(op == X_DIV ? "drf::floor_div<" : "drf::euclid_mod<") + V_ + ", " + U_ +
                                  ">(" + a + ", " + b + ")"));
                break;
            }
            case X_DIVC: case X_MODC: {
                std::string c = cast(lit64((int64_t)p_.xcode.at(i++)));
                std::string a = pop();
                st.push_back(temp(std::string(op == X_DIVC ? "drf::floor_div<" : "drf::euclid_mod<") + V_ + ", " + U_ +
                                  ">(" + a + ", " + c + ")"));
                break;
            }
            case X_MASK: {
                std::string m = ulit(p_.xcode.at(i++));
                std::string a = pop();
                st.push_back(temp(cast(u(a) + " & " + u("(" + m + ")"))));
                break;
            }
            case X_EQ: case X_NE: case X_LT: case X_LE: case X_GT: case X_GE: {
                static const char *rel[] = {" == ", " != ", " < ", " <= ", " > ", " >= "};
                std::string b = pop(), a = pop();
                st.push_back(temp(cast(a + rel[op - X_EQ] + b)));
                break;
            }
            case X_AND: case X_OR: {
                std::string b = pop(), a = pop();
                st.push_back(temp(cast("(" + a + " != 0)" + (op == X_AND ? " & " : " | ") + "(" + b + " != 0)")));
                break;
            }
            case X_NOT: { std::string a = pop(); st.push_back(temp(cast(a + " == 0"))); break; }
            default: fail("unknown expression op " + std::to_string(op)); return "0";
            }
            if (!error.empty()) return "0";
        }
        fail("expression too long");
        return "0";
    }

    // The access's effect in the current mode.  `ph`, `idx` are C expressions.
    void access(const std::string &ph, uint32_t loc, const std::string &idx, bool write)
    {
        if (mode_ == GM_TABLE) {
            body_ << "        if (" << ph << " < " << d_.tab_phases << "u && " << idx << " >= 0 && (uint64_t)(" << U_
                  << ")" << idx << " < " << ulit(p_.cells.at(loc)) << ") "
                  << "put(a, (unsigned long long)" << ph << " * " << ulit(d_.cells_sum) << " + "
                  << ulit(d_.tab_off + cbase_.at(loc)) << " + (unsigned long long)(" << U_ << ")" << idx << ", tid, "
                  << (write ? 1 : 0) << "u, last_bid);\n"
                  << "        else atomicOr(&a.ctrl->flags, (unsigned)drf::CF_TABLE_RANGE);\n";
        } else if (mode_ == GM_CELL) {
            body_ << "        if (" << ph << " == tg.phase && tg.loc == " << loc << "u && (unsigned long long)(" << U_
                  << ")" << idx << " == tg.idx) hit |= " << (write ? 3 : 1) << "u;\n";
        }
    }

    bool insn(const ShapeKey &k, uint32_t pc, const Insn &in, uint32_t &next)
    {
        switch (in.op) {
        case I_END:
            body_ << "    goto done;\n";
            return true;
        case I_ACCESS: {
            const bool write = (in.a & AF_WRITE) != 0;
            body_ << "    {\n";
            if (mode_ == GM_COUNT && !(in.a & AF_EVAL_IN_COUNT)) {
                body_ << "        count++;\n";
            } else {
                std::string idx = expr(in.c);
                if (!error.empty()) return false;
                body_ << "        if (" << idx << " < 0 || (uint64_t)(" << U_ << ")" << idx
                      << " >= " << ulit(p_.cells.at(in.b)) << ") " << (mode_ == GM_COUNT ? "{ err = 1u; goto done; }" : "goto done;")
                      << "\n";
                if (mode_ == GM_COUNT) body_ << "        count++;\n";
                else access("phase", in.b, idx, write);
            }
            body_ << "    }\n";
            return true;
        }
        case I_SYNC:
            if (mode_ == GM_COUNT) body_ << "    syncs++;\n";
            else body_ << "    phase++;\n";
            if (mode_ == GM_CELL) body_ << "    if (phase > tg.phase) goto done;\n";
            return true;
        case I_LOOP: {
            body_ << "    {\n";
            std::string lo = expr(in.c), hi = expr(in.d);
            if (!error.empty()) return false;
            body_ << "        if (" << lo << " < " << hi << ") { v[" << (int)in.a << "] = " << lo << "; h[" << (int)in.a
                  << "] = " << hi << "; } else goto L" << in.e + 1 << ";\n";
            body_ << "    }\n";
            targets_.push_back((uint32_t)in.e + 1);
            return true;
        }
        case I_ENDLOOP: {
            const std::string va = "v[" + std::to_string(in.a) + "]";
            body_ << "    " << va << " = (" << V_ << ")((" << U_ << ")" << va << " + 1u);\n";
            body_ << "    if (" << va << " < h[" << (int)in.a << "]) goto L" << in.c << ";\n";
            targets_.push_back((uint32_t)in.c);
            return true;
        }
        case I_IF: {
            body_ << "    {\n";
            std::string c = expr(in.c);
            if (!error.empty()) return false;
            body_ << "        if (!" << c << ") goto L" << in.d << ";\n    }\n";
            targets_.push_back((uint32_t)in.d);
            return true;
        }
        case I_JUMP:
            body_ << "    goto L" << in.c << ";\n";
            targets_.push_back((uint32_t)in.c);
            return true;
        case I_FASTLOOP: {
            const uint32_t m = (uint32_t)in.e, spi = in.b;
            if (m == 0 || m > kFastMax) return fail("bad fast loop");
            for (uint32_t j = 1; j <= m; j++) labels_skip_[pc + j] = true;
            next = pc + 1 + m;
            const std::string va = "v[" + std::to_string(in.a) + "]", ha = "h[" + std::to_string(in.a) + "]";
            body_ << "    {\n";
            std::string lo, hi;
            if (k.chunked == 2 && k.nsplit && pc == k.split_pc[k.nsplit - 1]) {
                lo = va;             // this item's chunk of the loop, set by the prologue
                hi = ha;
            } else {
                lo = expr(in.c);
                hi = expr(in.d);
                if (!error.empty()) return false;
            }
            body_ << "        const " << V_ << " flo = " << lo << ", fhi = " << hi << ";\n";
            body_ << "        if (flo < fhi) {\n";
            body_ << "        const uint64_t trip = (uint64_t)(" << U_ << ")((" << U_ << ")fhi - (" << U_ << ")flo);\n";
            if (mode_ == GM_COUNT) {
                body_ << "        count += (uint32_t)(trip * " << m << "u);\n";
                if (spi) body_ << "        syncs += (uint32_t)(trip * " << spi << "u);\n";
                body_ << "        }\n    }\n";
                return true;
            }
            std::vector<std::string> rest(m);
            for (uint32_t j = 0; j < m; j++) {
                const Insn &A = p_.insns.at(pc + 1 + j);
                if (A.op != I_FASTACC) return fail("fast loop without its accesses");
                rest[j] = expr(A.c);
                if (!error.empty()) return false;
            }
            // index of fast access j at loop value `x` (a C expression)
            auto idx_of = [&](uint32_t j, const std::string &x) {
                const Insn &A = p_.insns.at(pc + 1 + j);
                const uint64_t coef = p_.xcode.at((size_t)A.d), pcon = p_.xcode.at((size_t)A.d + 1);
                const uint32_t post = (A.a >> 2) & 3;
                std::string v = cast(u(rest[j]) + " + " + u("(" + ulit(coef) + ")") + " * " + u(x));
                if (post == FP_MASK) return cast(u(v) + " & " + u("(" + ulit(pcon) + ")"));
                if (post == FP_MOD)
                    return std::string("drf::euclid_mod<") + V_ + ", " + U_ + ">(" + v + ", " + cast(lit64((int64_t)pcon)) + ")";
                if (post == FP_DIV)
                    return std::string("drf::floor_div<") + V_ + ", " + U_ + ">(" + v + ", " + cast(lit64((int64_t)pcon)) + ")";
                return v;
            };
            std::string tail_start = "0";
            if (mode_ == GM_TABLE) {
                // unrolled by UF: all record copies of UF iterations are read
                // before any update, so the reads overlap (a copy older than an
                // update of the same cell is still a valid filter: records
                // only gain bits)
                const uint32_t UF = m == 1 ? 8 : m == 2 ? 4 : 2;
                body_ << "        const uint64_t tmain = trip - trip % " << UF << "u;\n";
                body_ << "        for (uint64_t t = 0; t < tmain; t += " << UF << "u) {\n";
                for (uint32_t q = 0; q < UF; q++) {
                    body_ << "        const " << V_ << " x" << q << " = (" << V_ << ")((" << U_ << ")flo + (" << U_
                          << ")(t + " << q << "u));\n";
                    body_ << "        const uint32_t p" << q << " = phase + (uint32_t)((t + " << q << "u) * " << spi << "u);\n";
                    for (uint32_t j = 0; j < m; j++) {
                        const Insn &A = p_.insns.at(pc + 1 + j);
                        const std::string sfx = std::to_string(q) + "_" + std::to_string(j);
                        body_ << "        const " << V_ << " i" << sfx << " = " << idx_of(j, "x" + std::to_string(q)) << ";\n";
                        body_ << "        const uint32_t h" << sfx << " = p" << q << " + " << (uint32_t)A.e << "u;\n";
                        body_ << "        const bool k" << sfx << " = h" << sfx << " < " << d_.tab_phases << "u && i" << sfx
                              << " >= 0 && (uint64_t)(" << U_ << ")i" << sfx << " < " << ulit(p_.cells.at(A.b)) << ";\n";
                        body_ << "        const unsigned long long o" << sfx << " = k" << sfx << " ? (unsigned long long)h" << sfx
                              << " * " << ulit(d_.cells_sum) << " + " << ulit(d_.tab_off + cbase_.at(A.b))
                              << " + (unsigned long long)(" << U_ << ")i" << sfx << " : 0ull;\n";
                        body_ << "        const uint32_t c" << sfx << " = k" << sfx
                              << " ? __ldca(reinterpret_cast<const uint32_t *>(a.table) + o" << sfx << ") : 0u;\n";
                    }
                }
                for (uint32_t q = 0; q < UF; q++)
                    for (uint32_t j = 0; j < m; j++) {
                        const Insn &A = p_.insns.at(pc + 1 + j);
                        const std::string sfx = std::to_string(q) + "_" + std::to_string(j);
                        body_ << "        if (k" << sfx << ") put_cur(a, o" << sfx << ", c" << sfx << ", tid, "
                              << ((A.a & AF_WRITE) ? 1 : 0) << "u, last_bid);\n"
                              << "        else atomicOr(&a.ctrl->flags, (unsigned)drf::CF_TABLE_RANGE);\n";
                    }
                body_ << "        }\n";
                tail_start = "tmain";
            }
            body_ << "        for (uint64_t t = " << tail_start << "; t < trip; t++) {\n";
            body_ << "        const " << V_ << " x = (" << V_ << ")((" << U_ << ")flo + (" << U_ << ")t);\n";
            body_ << "        const uint32_t ph0 = phase + (uint32_t)(t * " << spi << "u);\n";
            if (mode_ == GM_CELL) body_ << "        if (ph0 > tg.phase) break;\n";
            for (uint32_t j = 0; j < m; j++) {
                const Insn &A = p_.insns.at(pc + 1 + j);
                body_ << "        {\n";
                body_ << "        const " << V_ << " fi = " << idx_of(j, "x") << ";\n";
                body_ << "        const uint32_t fph = ph0 + " << (uint32_t)A.e << "u;\n";
                access("fph", A.b, "fi", (A.a & AF_WRITE) != 0);
                body_ << "        }\n";
            }
            body_ << "        }\n";
            if (spi) body_ << "        phase += (uint32_t)(trip * " << spi << "u);\n";
            body_ << "        }\n    }\n";
            if (mode_ == GM_CELL) body_ << "    if (phase > tg.phase) goto done;\n";
            return true;
        }
        default:
            return fail("unknown instruction " + std::to_string(in.op));
        }
    }
};

const char *kPrelude = R"DRF(
#define DRF_JIT 1
typedef signed char int8_t;
typedef unsigned char uint8_t;
typedef short int16_t;
typedef unsigned short uint16_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
)DRF";

const char *kHelpers = R"DRF(
struct CellTarget { uint32_t phase, loc; unsigned long long idx; };

// Apply an access to its cell's owner record given a copy `cur` of it read
// through L1 (drf::owner_put), and mark the cell's block as touched (the
// bitmap word is read through L1 first too).
static __device__ __forceinline__ void put_cur(const drf::BatchArgs &a, unsigned long long off, uint32_t cur,
                                               uint32_t tid, uint32_t w, unsigned long long &last_bid)
{
    uint32_t *cell = reinterpret_cast<uint32_t *>(a.table) + off;
    drf::owner_put(cell, cur, tid, w);
    const unsigned long long bid = off >> drf::kTabBlockLog;
    if (bid != last_bid) {
        const uint32_t bit = 1u << (uint32_t)(bid & 31);
        if (!(__ldca(&a.touch[bid >> 5]) & bit)) atomicOr(&a.touch[bid >> 5], bit);
        last_bid = bid;
    }
}

static __device__ __forceinline__ void put(const drf::BatchArgs &a, unsigned long long off, uint32_t tid, uint32_t w,
                                           unsigned long long &last_bid)
{
    put_cur(a, off, __ldca(reinterpret_cast<const uint32_t *>(a.table) + off), tid, w, last_bid);
}
)DRF";

}  // namespace

Error jit_source(const Prepared &p, const BatchHost &b, std::string &src, std::vector<uint16_t> &item_shape)
{
    if (b.protos.size() != 1) return Error::make(S_INVALID_ARG, "specialization takes a batch of one protocol");
    if (!b.table_ok) return Error::make(S_LIMIT, "the protocol has no owner table");
    const DevProto &d = b.protos[0];
    std::map<ShapeKey, uint16_t> shapes;
    std::vector<ShapeKey> keys;
    item_shape.clear();
    for (const ItemDesc &it : p.items) {
        ShapeKey k{};
        k.start = it.start_pc;
        k.stop = it.stop_pc;
        k.nsplit = it.nsplit;
        k.chunked = it.chunked;
        for (uint32_t l = 0; l < it.nsplit && l < (uint32_t)kMaxSplit; l++) k.split_pc[l] = it.split_pc[l];
        auto f = shapes.find(k);
        if (f == shapes.end()) {
            if (keys.size() >= kMaxShapes) return Error::make(S_LIMIT, "too many item shapes to specialize");
            f = shapes.emplace(k, (uint16_t)keys.size()).first;
            keys.push_back(k);
        }
        item_shape.push_back(f->second);
    }
    std::ostringstream o;
    o << kPrelude;
    o << header_text(kJitDevprogH) << header_text(kJitBatchArgsH) << header_text(kJitIntmathCuh)
      << header_text(kJitOwnerCuh);
    o << kHelpers;
    Gen g(p, d, b.cbase);
    const Mode modes[] = {GM_COUNT, GM_TABLE, GM_CELL};
    for (Mode m : modes)
        for (size_t s = 0; s < keys.size(); s++)
            if (!g.shape_fn(keys[s], (uint32_t)s, m, o))
                return Error::make(S_LIMIT, "cannot specialize: " + g.error);
    auto dispatch = [&](const char *call) {
        std::ostringstream c;
        c << "            switch (shape[P.item_off + wi.k]) {\n";
        for (size_t s = 0; s < keys.size(); s++) {
            std::string fn = call;
            fn.replace(fn.find('#'), 1, std::to_string(s));
            c << "            case " << s << ": " << fn << "; break;\n";
        }
        c << "            default: break;\n            }\n";
        return c.str();
    };
    const char *loop_head = R"DRF(    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (blockDim.x / 32);
    for (uint32_t w = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; w < a.nwitems; w += warps) {
        const drf::WarpItem wi = a.witems[w];
        const drf::DevProto P = a.protos[wi.proto];
        const drf::ItemDesc it = a.items[P.item_off + wi.k];
        const uint32_t tid = wi.g * 32 + lane;
        const bool alive = tid < P.nthreads;
        const uint64_t li = P.lane_off + (uint64_t)wi.k * P.nthreads + tid;
)DRF";
    // count pass: the interpreter's M_COUNT outputs
    o << "extern \"C\" __global__ void __launch_bounds__(256) drf_count(drf::BatchArgs a, const uint16_t *__restrict__ shape)\n{\n"
      << loop_head
      << "        uint32_t count = 0, syncs = 0, err = 0;\n"
      << "        if (alive) {\n" << dispatch("s#_count(it, tid, count, syncs, err)") << "        }\n"
      << R"DRF(        if (alive) {
            a.cnt[li] = count;
            a.syn[li] = syncs;
            if (err) {
                a.erro[li] = ((unsigned long long)count << 8) | err;
                atomicMin(&a.err_key[wi.proto], ((unsigned long long)tid << 32) | wi.k);
            }
        }
        const uint32_t total = __reduce_add_sync(0xFFFFFFFFu, count);
        if (lane == 0) {
            a.wcnt[w] = total;
            if (total) {
                atomicAdd(&a.blocksum[w / drf::kWScanPerBlock], (unsigned long long)total);
                atomicAdd(&a.ptuples[wi.proto], (unsigned long long)total);
            }
        }
    }
}
)DRF";
    // table pass: owner records, plus the barrier-divergence check
    o << "extern \"C\" __global__ void __launch_bounds__(256) drf_table(drf::BatchArgs a, const uint16_t *__restrict__ shape)\n{\n"
      << loop_head
      << R"DRF(        if (wi.k == 0 && alive && a.totsyn[P.tid_off + tid] != a.totsyn[P.tid_off])
            atomicMin(&a.div_tid[wi.proto], tid);
        if (!alive) continue;
        const uint32_t phase = a.phs[li];
        unsigned long long last_bid = ~0ull;
)DRF"
      << dispatch("s#_table(a, it, tid, phase, last_bid)") << "    }\n}\n";
    // witness pass: which threads access / write the first racy cell
    o << "extern \"C\" __global__ void __launch_bounds__(256) drf_cell(drf::BatchArgs a, const uint16_t *__restrict__ shape)\n{\n"
      << R"DRF(    const unsigned long long bp = a.best_pos[0];
    if (bp == ~0ull || a.err_key[0] != ~0ull || a.div_tid[0] != 0xFFFFFFFFu) return;
    CellTarget tg;
    {
        const drf::DevProto P0 = a.protos[0];
        const unsigned long long rel = bp - P0.tab_off;
        const unsigned long long row = rel / P0.cells_sum;
        const unsigned long long c = rel - row * P0.cells_sum;
        const uint64_t *cb = a.cbase + P0.cells_off;
        uint32_t l = 0;
        while (l + 1 < P0.nlocs && cb[l + 1] <= c) l++;
        tg.phase = (uint32_t)row;
        tg.loc = l;
        tg.idx = c - cb[l];
    }
)DRF"
      << loop_head
      << R"DRF(        if (!alive) continue;
        const uint32_t phase = a.phs[li];
        if (phase > tg.phase) continue;
        uint32_t hit = 0;
)DRF"
      << dispatch("s#_cell(it, tid, phase, tg, hit)")
      << R"DRF(        if (hit) {
            const uint64_t bb = P.tid_off + tid;
            atomicOr(&a.hit_acc[bb >> 5], 1u << (uint32_t)(bb & 31));
            if (hit & 2) atomicOr(&a.hit_wr[bb >> 5], 1u << (uint32_t)(bb & 31));
        }
    }
}
)DRF";
    src = o.str();
    if (src.size() > kMaxSourceBytes) return Error::make(S_LIMIT, "specialized source too large");
    return Error{};
}

// ------------------------------------------------------------------ NVRTC

namespace {

struct Nvrtc {
    bool ok = false;
    std::string why;
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
};

const Nvrtc &nvrtc()
{
    static Nvrtc n = [] {
        Nvrtc r;
        void *h = nullptr;
        for (const char *name : {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"})
            if ((h = dlopen(name, RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) { r.why = "NVRTC (libnvrtc.so.13) not found"; return r; }
        r.create = (decltype(r.create))dlsym(h, "nvrtcCreateProgram");
        r.compile = (decltype(r.compile))dlsym(h, "nvrtcCompileProgram");
        r.log_size = (decltype(r.log_size))dlsym(h, "nvrtcGetProgramLogSize");
        r.log = (decltype(r.log))dlsym(h, "nvrtcGetProgramLog");
        r.cubin_size = (decltype(r.cubin_size))dlsym(h, "nvrtcGetCUBINSize");
        r.cubin = (decltype(r.cubin))dlsym(h, "nvrtcGetCUBIN");
        r.destroy = (decltype(r.destroy))dlsym(h, "nvrtcDestroyProgram");
        r.ok = r.create && r.compile && r.log_size && r.log && r.cubin_size && r.cubin && r.destroy;
        if (!r.ok) r.why = "NVRTC lacks an expected entry point";
        return r;
    }();
    return n;
}

}  // namespace

Error jit_compile(const std::string &src, std::vector<char> &cubin, std::string &log)
{
    const Nvrtc &n = nvrtc();
    if (!n.ok) { log = n.why; return Error::make(S_NOT_FOUND, n.why); }
    nvrtcProgram prog = nullptr;
    if (n.create(&prog, src.c_str(), "drf_specialized.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
        return Error::make(S_INTERNAL, "nvrtcCreateProgram failed");
    const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo", "--disable-warnings"};
    const nvrtcResult r = n.compile(prog, 4, opts);
    size_t ls = 0;
    n.log_size(prog, &ls);
    log.assign(ls, '\0');
    if (ls) n.log(prog, &log[0]);
    Error e;
    if (r != NVRTC_SUCCESS) {
        e = Error::make(S_INTERNAL, "NVRTC compilation failed");
    } else {
        size_t cs = 0;
        n.cubin_size(prog, &cs);
        cubin.assign(cs, 0);
        if (!cs || n.cubin(prog, cubin.data()) != NVRTC_SUCCESS) e = Error::make(S_INTERNAL, "NVRTC produced no cubin");
    }
    n.destroy(&prog);
    return e;
}

Error jit_load(const std::vector<char> &cubin, JitModule &m)
{
    cudaError_t ce = cudaLibraryLoadData(&m.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (ce == cudaSuccess) ce = cudaLibraryGetKernel(&m.count, m.lib, "drf_count");
    if (ce == cudaSuccess) ce = cudaLibraryGetKernel(&m.table, m.lib, "drf_table");
    if (ce == cudaSuccess) ce = cudaLibraryGetKernel(&m.cell, m.lib, "drf_cell");
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return Error::make(S_CUDA, std::string("loading the specialized kernels: ") + cudaGetErrorString(ce));
    }
    return Error{};
}

JitModule::~JitModule()
{
    if (lib) cudaLibraryUnload(lib);
}

}  // namespace drf
