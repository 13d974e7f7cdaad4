// Run-time specialization (see jit.h): code generation, NVRTC, loading.
#include "jit.h"

#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <mutex>
#include <sstream>
#include <functional>
#include <algorithm>

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
          U_(p.wide ? "uint64_t" : "uint32_t"),
          narrow_(d.tab_off + (uint64_t)d.tab_phases * d.cells_sum <= (1ull << 32))
    {
    }

    // Record offsets fit 32 bits when the protocol's rows end below 2^32.
    bool narrow() const { return narrow_; }

    std::string error;

    // Accesses whose records the range pass makes (RangeAccess): the table
    // pass counts them and leaves their records alone.
    void set_range_skip(const std::set<uint32_t> &pcs) { skip_ = pcs; }

    // One device function per (shape, mode).
    bool shape_fn(const ShapeKey &k, uint32_t id, Mode m, std::ostringstream &o)
    {
        mode_ = m;
        body_.str("");
        tmp_ = 0;
        const char *name[] = {"count", "table", "cell"};
        o << "static __device__ __forceinline__ void s" << id << "_" << name[m] << "(";
        if (m == GM_COUNT) o << "const IJ &it, uint32_t tid, uint32_t &count, uint32_t &syncs, uint32_t &err)";
        if (m == GM_TABLE)
            o << "const drf::BatchArgs &a, const IJ &it, uint32_t tid, uint32_t phase, uint32_t &nacc)";
        if (m == GM_CELL) o << "const IJ &it, uint32_t tid, uint32_t phase, const CellTarget &tg, uint32_t &hit)";
        o << "\n{\n";
        o << "    " << V_ << " v[" << kMaxVars << "], h[" << kMaxVars << "];\n";
        o << "    (void)tid; (void)it;\n";
        if (m == GM_TABLE) o << "    uint32_t *const tab = reinterpret_cast<uint32_t *>(a.table);\n    (void)tab;\n";
        jump_targets_.clear();
        for (uint32_t pc = k.start; pc < k.stop && pc < p_.insns.size(); pc++) {
            const Insn &in = p_.insns[pc];
            if (in.op == I_LOOP) jump_targets_.insert((uint32_t)in.e + 1);
            if (in.op == I_ENDLOOP || in.op == I_JUMP) jump_targets_.insert((uint32_t)in.c);
            if (in.op == I_IF) jump_targets_.insert((uint32_t)in.d);
        }
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
    const bool narrow_;
    Mode mode_ = GM_COUNT;
    std::ostringstream body_;
    int tmp_ = 0;
    std::vector<uint32_t> targets_;
    std::map<uint32_t, bool> labels_skip_;
    std::set<uint32_t> jump_targets_;      // every jump target of the item being generated
    int slot_ = 0;                         // names of batched-update temporaries
    std::set<uint32_t> skip_;              // accesses the range pass applies

    // One access of a batch of owner-table updates: the access applies when
    // `k` holds; `o` is its record offset and `c` a copy of its record.
    struct Slot { std::string k, o, c; bool write, uniform; };

    // The updates of a batch whose record copies are already read
    // (owner.cuh's rule, split in three rounds so that one warp waits for at
    // most one round trip of claims): first every claim of a cell whose copy
    // is empty (compare-and-swap), then the bits the non-empty copies ask
    // for, then the outcome of the claims -- a lost claim adds the bits the
    // winner's record asks for, and the won claims of the lanes running
    // together mark their blocks as touched with one reduction per touch
    // word (touch_created).  Accesses whose index does not read tid go
    // through put_warp_cur.
    void updates(const std::vector<Slot> &S)
    {
        std::vector<std::string> n(S.size());
        for (size_t i = 0; i < S.size(); i++) {
            if (S[i].uniform) continue;
            n[i] = "n" + std::to_string(slot_++);
            body_ << "        uint32_t " << n[i] << " = 1u;\n";
            body_ << "        if (" << S[i].k << " && " << S[i].c << " == 0u) " << n[i] << " = atomicCAS(tab + " << S[i].o
                  << ", 0u, (tid + 1u)" << (S[i].write ? " | 0x80000000u" : "") << ");\n";
        }
        for (size_t i = 0; i < S.size(); i++) {
            if (S[i].uniform) continue;
            body_ << "        if (" << S[i].k << " && " << S[i].c << " != 0u) { const uint32_t nd = drf::owner_need(" << S[i].c
                  << ", tid, " << (S[i].write ? 1 : 0) << "u); if (nd) atomicOr(tab + " << S[i].o << ", nd); }\n";
        }
        for (size_t i = 0; i < S.size(); i++) {
            if (S[i].uniform) continue;
            body_ << "        if (" << S[i].k << " && " << S[i].c << " == 0u && " << n[i] << " != 0u) { const uint32_t nd = "
                  << "drf::owner_need(" << n[i] << ", tid, " << (S[i].write ? 1 : 0) << "u); if (nd) atomicOr(tab + "
                  << S[i].o << ", nd); }\n";
            body_ << "        touch_created(a.touch, " << S[i].o << ", " << S[i].k << " && " << S[i].c << " == 0u && " << n[i]
                  << " == 0u);\n";
        }
        for (size_t i = 0; i < S.size(); i++)
            if (S[i].uniform)
                body_ << "        if (" << S[i].k << ") put_warp_cur(tab, a.touch, " << S[i].o << ", " << S[i].c << ", tid, "
                      << (S[i].write ? 1 : 0) << "u);\n";
    }

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

    // Whether the expression code at `off` reads tid (directly or as an
    // affine term).  Loop variables do not count: lanes at the same point of
    // the same iteration agree on them.
    bool uses_tid(int32_t off) const
    {
        size_t i = (size_t)off;
        for (int guard = 0; guard < 1 << 16 && i < p_.xcode.size(); guard++) {
            const uint64_t w = p_.xcode[i++];
            switch ((uint32_t)(w & 0xff)) {
            case X_RET: return false;
            case X_TID: return true;
            case X_CONST: case X_DIVC: case X_MODC: case X_MASK: i++; break;
            case X_AFF: {
                const uint32_t n = (uint32_t)(w >> 8);
                for (uint32_t t = 0; t < n; t++, i += 2)
                    if ((uint32_t)p_.xcode.at(i) == kAffTid && p_.xcode.at(i + 1) != 0) return true;
                i++;
                break;
            }
            default: break;
            }
        }
        return true;
    }

    // Record offset of (phase `ph`, array `loc`, index `idx`) -- C expressions
    // known to be in range -- in the offset type of the generated source.
    std::string offset(const std::string &ph, uint32_t loc, const std::string &idx) const
    {
        if (narrow_)
            return "(toff_t)((uint32_t)" + ph + " * " + std::to_string((uint32_t)d_.cells_sum) + "u + " +
                   std::to_string((uint32_t)(d_.tab_off + cbase_.at(loc))) + "u + (uint32_t)(" + U_ + ")" + idx + ")";
        return "(toff_t)((unsigned long long)" + ph + " * " + ulit(d_.cells_sum) + " + " +
               ulit(d_.tab_off + cbase_.at(loc)) + " + (unsigned long long)(" + U_ + ")" + idx + ")";
    }

    // The access's effect in the witness pass.  `ph`, `idx` are C expressions.
    void access(const std::string &ph, uint32_t loc, const std::string &idx, bool write)
    {
        if (mode_ == GM_CELL)
            body_ << "        if (" << ph << " == tg.phase && tg.loc == " << loc << "u && (unsigned long long)(" << U_ << ")"
                  << idx << " == tg.idx) hit |= " << (write ? 3 : 1) << "u;\n";
    }

    // A run of consecutive accesses (no jump lands inside it) in the table
    // pass: every index first (an evaluation error ends the thread's item;
    // the check then reports the error and no verdict, so the run's updates
    // do not matter), then every record copy, then the batch's updates.
    bool access_run(const ShapeKey &k, uint32_t pc, uint32_t &next)
    {
        uint32_t end = pc + 1;
        while (end < k.stop && end - pc < 8 && p_.insns.at(end).op == I_ACCESS && !jump_targets_.count(end)) end++;
        next = end;
        body_ << "    {\n";
        std::vector<std::string> idx;
        for (uint32_t q = pc; q < end; q++) {
            const Insn &A = p_.insns.at(q);
            if (skip_.count(q)) { idx.emplace_back(); continue; }     // the range pass applies it
            idx.push_back(expr(A.c));
            if (!error.empty()) return false;
            body_ << "        if (" << idx.back() << " < 0 || (uint64_t)(" << U_ << ")" << idx.back() << " >= "
                  << ulit(p_.cells.at(A.b)) << ") goto done;\n";
        }
        uint32_t kept_run = 0;                 // (the range pass's tuples are counted on the host)
        for (uint32_t q = pc; q < end; q++) kept_run += skip_.count(q) ? 0u : 1u;
        if (kept_run) body_ << "        nacc += " << kept_run << "u;\n";
        body_ << "        const bool kr = phase < " << d_.tab_phases << "u;\n";
        body_ << "        if (!kr) atomicOr(&a.ctrl->flags, (unsigned)drf::CF_TABLE_RANGE);\n";
        std::vector<Slot> S;
        for (uint32_t q = pc; q < end; q++) {
            const Insn &A = p_.insns.at(q);
            if (skip_.count(q)) continue;
            const std::string sfx = std::to_string(slot_++);
            body_ << "        const toff_t o" << sfx << " = kr ? " << offset("phase", A.b, idx[q - pc]) << " : (toff_t)0;\n";
            body_ << "        const uint32_t c" << sfx << " = kr ? __ldcg(tab + o" << sfx << ") : 0u;\n";
            S.push_back(Slot{"kr", "o" + sfx, "c" + sfx, (A.a & AF_WRITE) != 0, !uses_tid(A.c)});
        }
        updates(S);
        body_ << "    }\n";
        return true;
    }

    // Whether the loop at pc holds no sync and no access but the range
    // pass's (the host's LB_RANGE_ONLY rule, on this program).
    bool range_only_loop(uint32_t pc) const
    {
        if (skip_.empty()) return false;
        const uint32_t e = (uint32_t)p_.insns.at(pc).e;
        if (e >= p_.insns.size()) return false;
        for (uint32_t q = pc + 1; q <= e; q++) {
            const Insn &x = p_.insns[q];
            if (x.op == I_SYNC || x.op == I_END) return false;
            if ((x.op == I_ACCESS || x.op == I_FASTACC) && !skip_.count(q)) return false;
            if (x.op == I_FASTLOOP && x.b != 0) return false;
        }
        return true;
    }

    bool insn(const ShapeKey &k, uint32_t pc, const Insn &in, uint32_t &next)
    {
        switch (in.op) {
        case I_END:
            body_ << "    goto done;\n";
            return true;
        case I_ACCESS: {
            if (mode_ == GM_TABLE) return access_run(k, pc, next);
            if (mode_ == GM_CELL && skip_.count(pc)) return true;     // its witnesses come from the range pass
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
            if (mode_ != GM_COUNT && range_only_loop(pc)) {
                next = (uint32_t)in.e + 1;        // the range pass has the whole loop (and its witnesses)
                return true;
            }
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
            uint32_t kept = 0;
            for (uint32_t j = 0; j < m; j++) kept += skip_.count(pc + 1 + j) ? 0 : 1;
            if (mode_ == GM_TABLE && kept == 0) {
                // every access of the loop is the range pass's (its tuples are
                // counted on the host)
                if (spi) body_ << "        phase += (uint32_t)(trip * " << spi << "u);\n";
                body_ << "        }\n    }\n";
                return true;
            }
            if (mode_ == GM_TABLE) {
                // groups of UF iterations: every record copy of a group is
                // read before any update (a copy older than an update of the
                // same cell is still a valid filter: records only gain bits)
                // one iteration per group: deeper groups read more copies
                // before their updates but hold more registers, and on this
                // pass occupancy hides the claims' round trips better (groups
                // of 2, 4, 8, 16 accesses measured 3-30% slower)
                const uint32_t UF = 1;
                body_ << "        nacc += (uint32_t)(trip * " << kept << "u);\n";
                body_ << "        for (uint64_t t = 0; t < trip; t += " << UF << "u) {\n";
                std::vector<Slot> S;
                std::vector<std::string> acts, ks;
                for (uint32_t q = 0; q < UF; q++) {
                    const std::string qs = std::to_string(q);
                    body_ << "        const bool a" << qs << " = t + " << q << "u < trip;\n";
                    body_ << "        const " << V_ << " x" << qs << " = (" << V_ << ")((" << U_ << ")flo + (" << U_
                          << ")(t + " << q << "u));\n";
                    body_ << "        const uint32_t p" << qs << " = phase + (uint32_t)((t + " << q << "u) * " << spi << "u);\n";
                    for (uint32_t j = 0; j < m; j++) {
                        const Insn &A = p_.insns.at(pc + 1 + j);
                        if (skip_.count(pc + 1 + j)) continue;        // the range pass applies it
                        const std::string sfx = qs + "_" + std::to_string(j);
                        body_ << "        const " << V_ << " i" << sfx << " = " << idx_of(j, "x" + qs) << ";\n";
                        body_ << "        const uint32_t h" << sfx << " = p" << qs << " + " << (uint32_t)A.e << "u;\n";
                        // the post-operation may already confine the index to the array
                        const uint32_t post = (A.a >> 2) & 3;
                        const int64_t pk = (int64_t)p_.xcode.at((size_t)A.d + 1);
                        const uint64_t ncell = p_.cells.at(A.b);
                        const bool in_range = (post == FP_MASK && (uint64_t)pk < ncell) ||
                                              (post == FP_MOD && pk != 0 && pk != INT64_MIN &&
                                               (uint64_t)(pk < 0 ? -pk : pk) <= ncell);
                        body_ << "        const bool k" << sfx << " = a" << qs << " && h" << sfx << " < " << d_.tab_phases << "u";
                        if (!in_range)
                            body_ << " && i" << sfx << " >= 0 && (uint64_t)(" << U_ << ")i" << sfx << " < " << ulit(ncell);
                        body_ << ";\n";
                        body_ << "        const toff_t o" << sfx << " = k" << sfx << " ? "
                              << offset("h" + sfx, A.b, "i" + sfx) << " : (toff_t)0;\n";
                        body_ << "        const uint32_t c" << sfx << " = k" << sfx << " ? __ldcg(tab + o" << sfx << ") : 0u;\n";
                        S.push_back(Slot{"k" + sfx, "o" + sfx, "c" + sfx, (A.a & AF_WRITE) != 0, !uses_tid(A.c)});
                        acts.push_back("a" + qs);
                        ks.push_back("k" + sfx);
                    }
                }
                updates(S);
                for (size_t i = 0; i < ks.size(); i++)
                    body_ << "        if (" << acts[i] << " && !" << ks[i]
                          << ") atomicOr(&a.ctrl->flags, (unsigned)drf::CF_TABLE_RANGE);\n";
                body_ << "        }\n";
                if (spi) body_ << "        phase += (uint32_t)(trip * " << spi << "u);\n";
                body_ << "        }\n    }\n";
                return true;
            }
            // witness pass: whether the thread's accesses of the loop hit the
            // witness cell.  With syncs in the body at most one iteration lies
            // in the witness phase, and it is evaluated alone.  Without, an
            // access whose index is (rest + coef * x) mod n (a mask or a
            // Euclidean remainder, n < 2^31) hits target on the loop's range
            // iff coef * x == target - rest (mod n) has a solution x there: with
            // g = gcd(coef mod n, n) that needs g | (target - rest), and the
            // solutions are x0 + i * (n / g), x0 from the inverse of coef / g
            // modulo n / g -- constants of the access, computed here.  Other
            // accesses iterate the loop.
            // (accesses the range pass applies give their witnesses there)
            std::vector<bool> solved(m, false);
            for (uint32_t j = 0; j < m; j++) solved[j] = skip_.count(pc + 1 + j) != 0;
            for (uint32_t j = 0; j < m && spi == 0; j++) {
                if (solved[j]) continue;
                const Insn &A = p_.insns.at(pc + 1 + j);
                const uint32_t post = (A.a >> 2) & 3;
                const int64_t pk = (int64_t)p_.xcode.at((size_t)A.d + 1);
                const int64_t coef = (int64_t)p_.xcode.at((size_t)A.d);
                __int128 n = 0;
                if (post == FP_MASK) n = (__int128)(uint64_t)pk + 1;
                if (post == FP_MOD && pk != 0 && pk != INT64_MIN) n = pk < 0 ? -(__int128)pk : (__int128)pk;
                if (n < 2 || n >= ((__int128)1 << 31)) continue;
                // coef as the lowered arithmetic sees it (the U word, read as V)
                const __int128 cv = p_.wide ? (__int128)coef : (__int128)(int32_t)(uint32_t)(uint64_t)coef;
                __int128 ca = cv % n;
                if (ca < 0) ca += n;
                __int128 g = ca, r2 = n;
                while (r2 != 0) { const __int128 t = g % r2; g = r2; r2 = t; }
                if (ca == 0) g = n;
                const __int128 mm = n / g;
                __int128 inv = 0;
                if (ca != 0 && mm > 1) {                   // (ca / g) * inv == 1 (mod mm), extended Euclid
                    __int128 r0 = (ca / g) % mm, r1 = mm, s0 = 1, s1 = 0;
                    while (r1 != 0) {
                        const __int128 q = r0 / r1;
                        __int128 t = r0 - q * r1; r0 = r1; r1 = t;
                        t = s0 - q * s1; s0 = s1; s1 = t;
                    }
                    inv = s0 % mm;
                    if (inv < 0) inv += mm;
                }
                const std::string N = ulit((uint64_t)n), G = ulit((uint64_t)g), M = ulit((uint64_t)mm), I = ulit((uint64_t)inv);
                const char *hitbits = (A.a & AF_WRITE) ? "3u" : "1u";
                body_ << "        if (phase + " << (uint32_t)A.e << "u == tg.phase && tg.loc == " << A.b << "u && tg.idx < " << N
                      << ") {\n";
                if (post == FP_MASK)
                    body_ << "        const unsigned long long rm = (unsigned long long)(" << U_ << ")" << rest[j] << " & "
                          << ulit((uint64_t)pk) << ";\n";
                else
                    body_ << "        const long long rq = (long long)" << rest[j] << " % (long long)" << N << ";\n"
                          << "        const unsigned long long rm = rq < 0 ? (unsigned long long)(rq + (long long)" << N
                          << ") : (unsigned long long)rq;\n";
                body_ << "        const unsigned long long cc = tg.idx >= rm ? tg.idx - rm : tg.idx + " << N << " - rm;\n";
                if (ca == 0) {
                    body_ << "        if (cc == 0) hit |= " << hitbits << ";\n";
                } else if (mm == 1) {
                    body_ << "        if (cc % " << G << " == 0) hit |= " << hitbits << ";\n";
                } else {
                    body_ << "        if (cc % " << G << " == 0) {\n"
                          << "        const unsigned long long x0 = (cc / " << G << ") * " << I << " % " << M << ";\n"
                          << "        const long long lq = (long long)flo % (long long)" << M << ";\n"
                          << "        const unsigned long long lm = lq < 0 ? (unsigned long long)(lq + (long long)" << M
                          << ") : (unsigned long long)lq;\n"
                          << "        if ((x0 >= lm ? x0 - lm : x0 + " << M << " - lm) < trip) hit |= " << hitbits << ";\n"
                          << "        }\n";
                }
                body_ << "        }\n";
                solved[j] = true;
            }
            bool all_solved = true;
            for (uint32_t j = 0; j < m; j++) all_solved = all_solved && solved[j];
            if (spi) {
                for (uint32_t j = 0; j < m; j++) {
                    if (solved[j]) continue;
                    const Insn &A = p_.insns.at(pc + 1 + j);
                    body_ << "        {\n"
                          << "        const long long dt = (long long)tg.phase - (long long)phase - " << (uint32_t)A.e << "ll;\n"
                          << "        if (dt >= 0 && dt % " << spi << "ll == 0 && (unsigned long long)(dt / " << spi
                          << "ll) < trip && tg.loc == " << A.b << "u) {\n"
                          << "        const " << V_ << " x = (" << V_ << ")((" << U_ << ")flo + (" << U_ << ")(dt / " << spi
                          << "ll));\n"
                          << "        const " << V_ << " fi = " << idx_of(j, "x") << ";\n"
                          << "        if ((unsigned long long)(" << U_ << ")fi == tg.idx) hit |= "
                          << ((A.a & AF_WRITE) ? "3u" : "1u") << ";\n"
                          << "        }\n        }\n";
                }
            } else if (!all_solved) {
                body_ << "        if (phase == tg.phase)\n";
                body_ << "        for (uint64_t t = 0; t < trip; t++) {\n";
                body_ << "        const " << V_ << " x = (" << V_ << ")((" << U_ << ")flo + (" << U_ << ")t);\n";
                for (uint32_t j = 0; j < m; j++) {
                    if (solved[j]) continue;
                    const Insn &A = p_.insns.at(pc + 1 + j);
                    body_ << "        {\n";
                    body_ << "        const " << V_ << " fi = " << idx_of(j, "x") << ";\n";
                    access("phase", A.b, "fi", (A.a & AF_WRITE) != 0);
                    body_ << "        }\n";
                }
                body_ << "        }\n";
            }
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

// The split-loop positions of one item (its ItemDesc's j and chunk), and
// with static phases the phases at the item's start and end.
struct __align__(16) IJ { uint32_t j[4]; uint32_t chunk, phase, phase_end, pad; };

// Apply an access to its cell's owner record given a copy `cur` of it read
// through L2 (drf::owner_put); the update that creates the record marks its
// block as touched.
static __device__ __forceinline__ void put_cur(uint32_t *table, uint32_t *touch, toff_t off, uint32_t cur, uint32_t tid,
                                               uint32_t w)
{
    if (drf::owner_put(table + off, cur, tid, w)) drf::owner_touch(touch, off, drf::kTabBlockLog);
}

// Keeps the two smallest distinct values seen in f < s.
static __device__ __forceinline__ void two_smallest(uint32_t &f, uint32_t &s, uint32_t x)
{
    if (x == f || x == s) return;
    if (x < f) { s = f; f = x; }
    else if (x < s) s = x;
}

// Marks the blocks of the records that the lanes running together created
// (`created`): lanes whose blocks share a touch word set their bits with one
// update -- a warp's new records usually lie in one word's blocks.
static __device__ __forceinline__ void touch_created(uint32_t *touch, toff_t off, bool created)
{
    const unsigned am = __activemask();
    if (!__any_sync(am, created)) return;
    const uint32_t bid = (uint32_t)(off >> drf::kTabBlockLog);
    const unsigned grp = __match_any_sync(am, bid >> 5);
    const uint32_t bits = __reduce_or_sync(grp, created ? 1u << (bid & 31) : 0u);
    if ((threadIdx.x & 31) == (uint32_t)(__ffs(grp) - 1) && bits) atomicOr(touch + (bid >> 5), bits);
}

// An access whose index does not read tid: the lanes running together
// usually hit one cell, and then the lowest of them updates it for all (two
// or more lanes are two or more threads).  Lanes that disagree update their
// own cells.
static __device__ __forceinline__ void put_warp_cur(uint32_t *table, uint32_t *touch, toff_t off, uint32_t cur,
                                                    uint32_t tid, uint32_t w)
{
    const unsigned am = __activemask();
    const int lead = __ffs(am) - 1;
    const toff_t off0 = __shfl_sync(am, off, lead);
    if (__all_sync(am, off == off0)) {
        if ((int)(threadIdx.x & 31) == lead) {
            const bool created = __popc(am) >= 2 ? drf::owner_put_many(table + off, cur, w)
                                                 : drf::owner_put(table + off, cur, tid, w);
            if (created) drf::owner_touch(touch, off, drf::kTabBlockLog);
        }
    } else {
        put_cur(table, touch, off, cur, tid, w);
    }
}

)DRF";

constexpr size_t kMaxConstItems = 1024;  // items whose schedule and positions are compiled in
constexpr uint64_t kMaxPhaseRanges = 1u << 16;   // phases whose item ranges are compiled in

}  // namespace

Error jit_source(const Prepared &p, const BatchHost &b, std::string &src, std::vector<uint16_t> &item_shape,
                 bool *static_phases, bool *compiled_schedule, bool *range_pass)
{
    if (static_phases) *static_phases = false;
    if (compiled_schedule) *compiled_schedule = false;
    if (range_pass) *range_pass = false;
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
    Gen g(p, d, b.cbase);
    o << "typedef " << (g.narrow() ? "uint32_t" : "unsigned long long") << " toff_t;   // owner-record offset\n";
    o << kHelpers;

    // The schedule (warp-item w -> item, thread group) compiled in: items
    // longest first, the 32-thread groups of one item consecutive, as the
    // batch's warp-item array holds it; else that array is read.
    const uint32_t K = (uint32_t)p.items.size(), G = (d.nthreads + 31) / 32;
    bool csched = K <= kMaxConstItems && K < (1u << 16) && (uint64_t)K * G == b.witems.size();
    std::vector<uint32_t> order(K);
    for (uint32_t pos = 0; csched && pos < K; pos++) {
        order[pos] = b.witems[(size_t)pos * G].k;
        for (uint32_t gg = 0; gg < G && csched; gg++) {
            const WarpItem &wi = b.witems[(size_t)pos * G + gg];
            if (wi.proto != 0 || wi.k != order[pos] || wi.g != gg || wi.k >= K) csched = false;
        }
    }
    // static phases (see Prepared): the phase of every item is compiled in,
    // and the table pass counts the tuples the count pass would have
    const bool stat = csched && p.static_phases && p.item_phase.size() == K;
    if (static_phases) *static_phases = stat;
    if (compiled_schedule) *compiled_schedule = csched;
    if (csched) {
        // read-only global data, not __constant__: warps index it by their
        // work item, and a per-item table of kilobytes outgrows the constant
        // cache while L1 keeps it after the first reads
        o << "static __device__ const uint32_t c_ord[" << K << "] = {";   // item | shape << 16, in schedule order
        for (uint32_t pos = 0; pos < K; pos++) o << (pos ? "," : "") << (order[pos] | ((uint32_t)item_shape[order[pos]] << 16)) << "u";
        o << "};\nstatic __device__ const IJ c_it[" << K << "] = {";   // per item; pad: its shape
        for (uint32_t k = 0; k < K; k++) {
            const ItemDesc &it = p.items[k];
            o << (k ? "," : "") << "{{" << it.j[0] << "u," << it.j[1] << "u," << it.j[2] << "u," << it.j[3] << "u},"
              << it.chunk << "u," << (stat ? p.item_phase[k] : 0u) << "u,"
              << (stat ? (k + 1 < K ? p.item_phase[k + 1] : (uint32_t)p.max_syncs) : 0u) << "u,"
              << item_shape[k] << "u}";
        }
        o << "};\n";
    }
    // With static phases, items in program order start (and end) in
    // non-decreasing phases, so the items that run any part of phase P are
    // one range [c_plo[P], c_phi[P]): the witness pass visits only the
    // range of the witness cell's phase.
    const uint64_t nph = (uint64_t)p.max_syncs + 1;
    const bool ranged = stat && nph <= kMaxPhaseRanges;
    if (ranged) {
        // item k runs phases [item_phase[k], end_phase(k)]
        auto end_phase = [&](uint32_t k) -> uint64_t { return k + 1 < K ? p.item_phase[k + 1] : p.max_syncs; };
        std::vector<uint32_t> plo(nph), phi(nph);
        uint32_t lo = 0, hi = 0;
        for (uint64_t ph = 0; ph < nph; ph++) {
            while (lo < K && end_phase(lo) < ph) lo++;
            if (hi < lo) hi = lo;
            while (hi < K && p.item_phase[hi] <= ph) hi++;
            plo[ph] = lo;
            phi[ph] = hi;
        }
        o << "static __device__ const uint32_t c_plo[" << nph << "] = {";
        for (uint64_t ph = 0; ph < nph; ph++) o << (ph ? "," : "") << plo[ph] << "u";
        o << "};\nstatic __device__ const uint32_t c_phi[" << nph << "] = {";
        for (uint64_t ph = 0; ph < nph; ph++) o << (ph ? "," : "") << phi[ph] << "u";
        o << "};\n";
    }
    // The range pass (pack_batch's plan_range): the table pass leaves the
    // protocol's range accesses to it and only counts them.
    const bool range = !b.rlive.empty() && !b.range_pcs.empty() && !b.range_pcs[0].empty();
    if (range_pass) *range_pass = range;
    if (range) g.set_range_skip(std::set<uint32_t>(b.range_pcs[0].begin(), b.range_pcs[0].end()));
    const Mode modes[] = {GM_COUNT, GM_TABLE, GM_CELL};
    for (Mode m : modes)
        for (size_t s = 0; s < keys.size(); s++)
            if (!g.shape_fn(keys[s], (uint32_t)s, m, o))
                return Error::make(S_LIMIT, "cannot specialize: " + g.error);
    auto dispatch = [&](const char *call) {
        std::ostringstream c;
        c << "            switch (shp) {\n";
        for (size_t s = 0; s < keys.size(); s++) {
            std::string fn = call;
            fn.replace(fn.find('#'), 1, std::to_string(s));
            c << "            case " << s << ": " << fn << "; break;\n";
        }
        c << "            default: break;\n            }\n";
        return c.str();
    };
    // the loop over warp-items: k (item), g (thread group), shp (its code
    // shape), it (its split-loop positions), tid, alive, li (its per-(item,
    // thread) slot); the protocol's descriptor fields are literals
    const std::string T = std::to_string(d.nthreads) + "u", LANE_OFF = ulit(d.lane_off), TID_OFF = ulit(d.tid_off);
    std::ostringstream lh;
    lh << "    const uint32_t lane = threadIdx.x & 31;\n"
          "    const uint32_t warps = gridDim.x * (blockDim.x / 32);\n";
    if (csched) {
        lh << "    for (uint32_t w = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; w < " << (uint64_t)K * G
           << "u; w += warps) {\n"
           << "        const uint32_t pos = w / " << G << "u;\n"
           << "        const uint32_t ord = __ldg(&c_ord[pos]);\n"
           << "        const uint32_t k = ord & 0xFFFFu, shp = ord >> 16, g = w - pos * " << G << "u;\n"
           << "        IJ it;\n"
           << "        {\n"
           << "            const uint4 w0 = __ldg(reinterpret_cast<const uint4 *>(&c_it[k]));\n"
           << "            const uint4 w1 = __ldg(reinterpret_cast<const uint4 *>(&c_it[k]) + 1);\n"
           << "            it.j[0] = w0.x; it.j[1] = w0.y; it.j[2] = w0.z; it.j[3] = w0.w;\n"
           << "            it.chunk = w1.x; it.phase = w1.y; it.phase_end = w1.z; it.pad = 0;\n"
           << "        }\n";
    } else {
        lh << "    for (uint32_t w = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; w < a.nwitems; w += warps) {\n"
           << "        const drf::WarpItem wi = a.witems[w];\n"
           << "        const uint32_t k = wi.k, g = wi.g, shp = shape[" << d.item_off << "u + k];\n"
           << "        const drf::ItemDesc &itd = a.items[" << d.item_off << "u + k];\n"
           << "        IJ it;\n"
           << "        for (int l = 0; l < 4; l++) it.j[l] = itd.j[l];\n"
           << "        it.chunk = itd.chunk;\n"
           << "        it.phase = 0;\n"
           << "        it.phase_end = 0;\n";
    }
    lh << "        const uint32_t tid = g * 32 + lane;\n"
       << "        const bool alive = tid < " << T << ";\n"
       << "        const uint64_t li = " << LANE_OFF << " + (uint64_t)k * " << T << " + tid;\n"
       << "        (void)shp; (void)li;\n";
    const std::string loop_head = lh.str();
    // every kernel lets its successor launch, then waits for its predecessor
    // (programmatic dependent launch; no-ops under a plain launch), then
    // issues a device-scope acquire fence, as the pipeline's pdl_begin does
    const char *sig = "(drf::BatchArgs a, const uint16_t *__restrict__ shape)\n{\n    (void)shape;\n"
                      "    asm volatile(\"griddepcontrol.launch_dependents;\" ::: \"memory\");\n"
                      "    asm volatile(\"griddepcontrol.wait;\" ::: \"memory\");\n"
                      "    asm volatile(\"fence.acq_rel.gpu;\" ::: \"memory\");\n";
    // count pass: the interpreter's M_COUNT outputs
    o << "extern \"C\" __global__ void __launch_bounds__(256) drf_count" << sig << loop_head
      << "        uint32_t count = 0, syncs = 0, err = 0;\n"
      << "        if (alive) {\n" << dispatch("s#_count(it, tid, count, syncs, err)") << "        }\n"
      << R"DRF(        if (alive) {
            a.cnt[li] = count;
            a.syn[li] = syncs;
            if (err) {
                a.erro[li] = ((unsigned long long)count << 8) | err;
                atomicMin(&a.err_key[0], ((unsigned long long)tid << 32) | k);
            }
        }
        const uint32_t total = __reduce_add_sync(0xFFFFFFFFu, count);
        if (lane == 0) {
            a.wcnt[w] = total;
            if (total) {
                atomicAdd(&a.blocksum[w / drf::kWScanPerBlock], (unsigned long long)total);
                atomicAdd(&a.ptuples[0], (unsigned long long)total);
            }
        }
    }
}
)DRF";
    // table pass: owner records, plus the barrier-divergence check
    o << "extern \"C\" __global__ void __launch_bounds__(256) drf_table" << sig;
    if (stat) {
        // phases compiled in; tuples counted here (one shared-memory sum per
        // block, one global add per block)
        o << "    __shared__ unsigned long long s_tuples;\n"
          << "    if (threadIdx.x == 0) s_tuples = 0;\n"
          // every thread executes the same syncs: thread 0's count, which the
          // finalize pass reports, is the protocol's static count
          << "    if (blockIdx.x == 0 && threadIdx.x == 0) a.totsyn[" << TID_OFF << "] = " << (uint32_t)p.max_syncs << "u;\n"
          << "    __syncthreads();\n"
          << loop_head
          << "        uint32_t nacc = 0;\n"
          << "        if (alive) {\n"
          << "            const uint32_t phase = it.phase;\n"
          << dispatch("s#_table(a, it, tid, phase, nacc)")
          << "        }\n"
          << "        const uint32_t tot = __reduce_add_sync(0xFFFFFFFFu, nacc);\n"
          << "        if (lane == 0 && tot) atomicAdd(&s_tuples, (unsigned long long)tot);\n"
          << "    }\n"
          << "    __syncthreads();\n"
          << "    if (threadIdx.x == 0 && s_tuples) {\n"
          << "        atomicAdd(&a.ptuples[0], s_tuples);\n"
          << "        atomicAdd(&a.ctrl->total, s_tuples);\n"
          << "    }\n}\n";
    } else {
        o << loop_head
          << "        if (k == 0 && alive && a.totsyn[" << TID_OFF << " + tid] != a.totsyn[" << TID_OFF << "])\n"
          << "            atomicMin(&a.div_tid[0], tid);\n"
          << "        if (!alive) continue;\n"
          << "        const uint32_t phase = a.phs[li];\n"
          << "        uint32_t nacc = 0;\n"
          << dispatch("s#_table(a, it, tid, phase, nacc)")
          << "    }\n}\n";
    }
    // witness pass: which threads access / write the first racy cell; with
    // static phases and no range pass its last block to finish also writes
    // the result (the finalize pass of the interpreted pipeline), so the
    // launch needs no further kernel
    o << "extern \"C\" __global__ void __launch_bounds__(256) drf_cell" << sig
      << "    const unsigned long long bp = __ldcg(&a.best_pos[0]);\n"
      << "    const bool live = !(bp == ~0ull || __ldcg(&a.err_key[0]) != ~0ull || __ldcg(&a.div_tid[0]) != 0xFFFFFFFFu);\n"
      << "    CellTarget tg{};\n"
      << "    if (live) {\n"
      << "    {\n"
      << "        const unsigned long long rel = bp - " << ulit(d.tab_off) << ";\n"
      << "        const unsigned long long row = rel / " << ulit(d.cells_sum ? d.cells_sum : 1) << ";\n"
      << "        const unsigned long long c = rel - row * " << ulit(d.cells_sum) << ";\n"
      << "        uint32_t l = 0;\n";
    for (uint32_t l = 1; l < d.nlocs; l++) o << "        if (c >= " << ulit(b.cbase.at(l)) << ") l = " << l << "u;\n";
    o << "        static const unsigned long long cb[" << std::max<uint32_t>(1, d.nlocs) << "] = {";
    for (uint32_t l = 0; l < std::max<uint32_t>(1, d.nlocs); l++) o << (l ? "," : "") << ulit(l < d.nlocs ? b.cbase.at(l) : 0);
    o << "};\n"
      << "        tg.phase = (uint32_t)row;\n        tg.loc = l;\n        tg.idx = c - cb[l];\n    }\n";
    if (ranged) {
        // the items of the witness phase only, their thread groups consecutive
        o << "    const uint32_t klo = tg.phase < " << nph << "u ? __ldg(&c_plo[tg.phase]) : 0u;\n"
          << "    const uint32_t nw = tg.phase < " << nph << "u ? (__ldg(&c_phi[tg.phase]) - klo) * " << G << "u : 0u;\n"
          << "    const uint32_t lane = threadIdx.x & 31;\n"
          << "    const uint32_t warps = gridDim.x * (blockDim.x / 32);\n"
          << "    for (uint32_t w = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; w < nw; w += warps) {\n"
          << "        const uint32_t kk = w / " << G << "u, k = klo + kk, g = w - kk * " << G << "u;\n"
          << "        IJ it;\n"
          << "        uint32_t shp;\n"
          << "        {\n"
          << "            const uint4 w0 = __ldg(reinterpret_cast<const uint4 *>(&c_it[k]));\n"
          << "            const uint4 w1 = __ldg(reinterpret_cast<const uint4 *>(&c_it[k]) + 1);\n"
          << "            it.j[0] = w0.x; it.j[1] = w0.y; it.j[2] = w0.z; it.j[3] = w0.w;\n"
          << "            it.chunk = w1.x; it.phase = w1.y; it.phase_end = w1.z; it.pad = 0;\n"
          << "            shp = w1.w;\n"
          << "        }\n"
          << "        const uint32_t tid = g * 32 + lane;\n"
          << "        if (tid >= " << T << ") continue;\n"
          << "        const uint32_t phase = it.phase;\n";
    } else {
        o << loop_head
          << (stat ? "        if (it.phase > tg.phase || it.phase_end < tg.phase || !alive) continue;\n"
                     "        const uint32_t phase = it.phase;\n"
                   : "        if (!alive) continue;\n        const uint32_t phase = a.phs[li];\n        if (phase > tg.phase) continue;\n");
    }
    o << R"DRF(        uint32_t hit = 0;
)DRF"
      << dispatch("s#_cell(it, tid, phase, tg, hit)")
      << "        const uint64_t bb = " << TID_OFF << " + tid;\n"
      << R"DRF(        // the lanes running together that share a hit word set their bits
        // with one update (a race's cell is usually hit by many threads)
        const unsigned am = __activemask();
        const unsigned grp = __match_any_sync(am, bb >> 5);
        const uint32_t bit = 1u << (uint32_t)(bb & 31);
        const uint32_t acc = __reduce_or_sync(grp, (hit & 1u) ? bit : 0u);
        const uint32_t wr = __reduce_or_sync(grp, (hit & 2u) ? bit : 0u);
        if ((threadIdx.x & 31) == (uint32_t)(__ffs(grp) - 1)) {
            if (acc) atomicOr(&a.hit_acc[bb >> 5], acc);
            if (wr) atomicOr(&a.hit_wr[bb >> 5], wr);
        }
    }
    }
)DRF";
    // (with the range pass the interpreted finalize pass runs instead: it
    // adds the witnesses the range pass holds)
    if (stat && !range) {
        // the last block: the two smallest accessors and writers of the cell
        // from the hit bits (static phases: no evaluation error or barrier
        // divergence can occur), then the protocol's result
        const uint64_t b0 = d.tid_off, b1 = d.tid_off + d.nthreads;
        o << "    __shared__ unsigned int s_last;\n"
          << "    __shared__ uint32_t s_red[4][8];\n"
          << "    __syncthreads();\n"
          << "    if (threadIdx.x == 0) {\n"
          << "        __threadfence();\n"
          << "        s_last = atomicAdd(&a.ctrl->blocks_done, 1u) == gridDim.x - 1 ? 1u : 0u;\n"
          << "    }\n"
          << "    __syncthreads();\n"
          << "    if (!s_last) return;\n"
          << "    __threadfence();\n"
          << "    if (threadIdx.x == 0 && a.nkeys != drf::kUncounted && __ldcg(&a.ctrl->total) != a.nkeys)\n"
          << "        atomicOr(&a.ctrl->flags, drf::CF_COUNT_MISMATCH);\n"
          << "    drf::DevResult r = {};\n"
          << "    r.tuples = __ldcg(&a.ptuples[0]);\n"
          << "    r.phases = " << (uint32_t)p.max_syncs << "u + 1u;\n"
          << "    r.sync_count_0 = " << (uint32_t)p.max_syncs << "u;\n"
          << "    if (!live) {\n"
          << "        r.verdict = 0;\n"
          << "        if (threadIdx.x == 0) a.results[0] = r;\n"
          << "        return;\n"
          << "    }\n"
          << "    uint32_t t0 = 0xFFFFFFFFu, t1 = 0xFFFFFFFFu, w0 = 0xFFFFFFFFu, w1 = 0xFFFFFFFFu;\n"
          // (a protocol without threads has no racy cell: the loop is for T >= 1)
          << "    for (uint64_t wd = " << ulit(b0 >> 5) << " + threadIdx.x; wd <= " << ulit(b1 > b0 ? (b1 - 1) >> 5 : 0)
          << " && " << (b1 > b0 ? "true" : "false") << "; wd += blockDim.x) {\n"
          << "        uint32_t ma = __ldcg(&a.hit_acc[wd]), mw = __ldcg(&a.hit_wr[wd]);\n"
          << "        const uint64_t lo = wd * 32;\n"
          << "        if (lo < " << ulit(b0) << ") { ma &= ~0u << (uint32_t)(" << ulit(b0) << " - lo); mw &= ~0u << (uint32_t)("
          << ulit(b0) << " - lo); }\n"
          << "        if (lo + 32 > " << ulit(b1) << ") { const uint32_t keep = (1u << (uint32_t)(" << ulit(b1)
          << " - lo)) - 1; ma &= keep; mw &= keep; }\n"
          << "        for (int q = 0; q < 2 && ma; q++) { two_smallest(t0, t1, (uint32_t)(lo + (uint32_t)(__ffs(ma) - 1) - "
          << ulit(b0) << ")); ma &= ma - 1; }\n"
          << "        for (int q = 0; q < 2 && mw; q++) { two_smallest(w0, w1, (uint32_t)(lo + (uint32_t)(__ffs(mw) - 1) - "
          << ulit(b0) << ")); mw &= mw - 1; }\n"
          << "    }\n"
          << R"DRF(    for (int o = 16; o; o >>= 1) {
        const uint32_t u0 = __shfl_xor_sync(0xFFFFFFFFu, t0, o), u1 = __shfl_xor_sync(0xFFFFFFFFu, t1, o);
        const uint32_t v0 = __shfl_xor_sync(0xFFFFFFFFu, w0, o), v1 = __shfl_xor_sync(0xFFFFFFFFu, w1, o);
        two_smallest(t0, t1, u0); two_smallest(t0, t1, u1);
        two_smallest(w0, w1, v0); two_smallest(w0, w1, v1);
    }
    const uint32_t wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s_red[0][wid] = t0; s_red[1][wid] = t1; s_red[2][wid] = w0; s_red[3][wid] = w1; }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (uint32_t q = 1; q < blockDim.x / 32; q++) {
        two_smallest(t0, t1, s_red[0][q]); two_smallest(t0, t1, s_red[1][q]);
        two_smallest(w0, w1, s_red[2][q]); two_smallest(w0, w1, s_red[3][q]);
    }
    r.verdict = 1;
    r.phase = tg.phase;
    r.loc = tg.loc;
    r.index = tg.idx;
    r.tid_i = t0;
    if (w0 == t0) { r.tid_j = t1; r.i_writes = 1; r.j_writes = (w1 == t1); }
    else { r.tid_j = w0; r.i_writes = 0; r.j_writes = 1; }
    a.results[0] = r;
)DRF";
    }
    o << "}\n";
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
