// Device pipeline: a concrete check of Definition 1 (DRF program, Sec. 3)
// for every thread id at once (rule par, Fig. 3).
//
//   init      clear the launch's control block and per-protocol reductions
//   count     interpret every (item, thread): accesses, syncs, first error
//   scan      per thread, exclusive scan of syncs over items -> phase at item
//             start; exclusive scan of per-warp access counts -> key offsets
//
// Then one of two back ends.  Sort path:
//   emit      interpret again, writing one 64-bit key per access
//             (proto | phase | array | index | tid | mode), coalesced per
//             warp; builds the digit histograms of every radix pass
//   radix     stable LSD radix sort on the key bits above tid, one pass per
//             8-bit digit (onesweep: per-tile ranking with warp ballots,
//             cross-tile digit offsets by decoupled look-back with bounded
//             waits); passes whose digit is constant are skipped
//   detect    segments of equal (proto, phase, array, index); a segment is
//             racy iff it holds a write and two distinct tids; min-reduce the
//             sorted position of the first racy segment per protocol
// Owner-table path (no sort; one record per (proto, phase, array, index)):
//   table     interpret again, updating each access's owner record (first
//             accessor, "a second thread", "written"; owner.cuh) and marking
//             the cell's block as touched
//   tscan     list the touched blocks (compaction of the touch bitmap), then
//             read them, one warp per block: a cell is racy iff written and
//             accessed by a second thread; min-reduce the first racy
//             position per protocol; clear what was read
//   witness   interpret the racy protocols once more, up to the witness
//             cell's phase, collecting which threads access / write it
// Both:
//   finalize  per protocol: first evaluation error (smallest tid, then the
//             number of accesses before it), else barrier divergence, else
//             the witness of the first racy cell: i = smallest accessor,
//             j = its smallest admissible partner
#include <cstdint>

#include "intmath.cuh"
#include "owner.cuh"
#include "pipeline.cuh"
#include "radix.cuh"

namespace drf {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr uint32_t kErrOob = 1, kErrDiv0 = 2;
constexpr unsigned long long kNone = ~0ull;

__device__ __forceinline__ Insn load_insn(const Insn *p)
{
    int4 v = __ldg(reinterpret_cast<const int4 *>(p));
    Insn r;
    r.op = (uint8_t)(v.x & 0xff);
    r.a = (uint8_t)((v.x >> 8) & 0xff);
    r.b = (uint16_t)((uint32_t)v.x >> 16);
    r.c = v.y;
    r.d = v.z;
    r.e = v.w;
    return r;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Stack machine over the expression code (see devprog.h).  Returns false on
// a division or remainder by zero.
template <typename V>
__device__ bool eval(const uint64_t *__restrict__ xc, int32_t off, uint32_t tid, const V *vars, V &out)
{
    using U = typename Unsigned<V>::T;
    // the top of the stack lives in a register and the entries below it in
    // st (st[d - 2] is the one under the top): the usual index -- one affine
    // form, then a remainder or mask -- never touches st
    V st[kMaxStack];
    V top = 0;
    int d = 0;                                   // stack depth
    auto push = [&](V x) {
        if (d) st[d - 1] = top;
        top = x;
        d++;
    };
    const uint64_t *p = xc + off;
    while (true) {
        uint64_t w = __ldg(p++);
        uint32_t op = (uint32_t)(w & 0xff);
        switch (op) {
        case X_RET: out = top; return true;
        case X_CONST: push((V)(int64_t)__ldg(p++)); break;
        case X_TID: push((V)tid); break;
        case X_VAR: push(vars[(uint32_t)(w >> 8)]); break;
        case X_AFF: {
            uint32_t n = (uint32_t)(w >> 8);
            U acc = 0;
            for (uint32_t i = 0; i < n; i++) {
                uint32_t reg = (uint32_t)__ldg(p++);
                U coef = (U)__ldg(p++);
                U v = reg == kAffTid ? (U)tid : (U)vars[reg];
                acc += coef * v;
            }
            acc += (U)__ldg(p++);
            push((V)acc);
            break;
        }
        case X_NEG: top = (V)(0 - (U)top); break;
        case X_DIVC: top = floor_div<V, U>(top, (V)(int64_t)__ldg(p++)); break;
        case X_MODC: top = euclid_mod<V, U>(top, (V)(int64_t)__ldg(p++)); break;
        case X_MASK: top = (V)((U)top & (U)__ldg(p++)); break;
        case X_NOT: top = top == 0; break;
        case X_ADD: case X_SUB: case X_MUL: case X_MIN: case X_MAX: case X_DIV: case X_MOD:
        case X_EQ: case X_NE: case X_LT: case X_LE: case X_GT: case X_GE: case X_AND: case X_OR: {
            // binary: a (under the top) op b (the top)
            const V a = st[d - 2], b = top;
            d--;
            switch (op) {
            case X_ADD: top = (V)((U)a + (U)b); break;
            case X_SUB: top = (V)((U)a - (U)b); break;
            case X_MUL: top = (V)((U)a * (U)b); break;
            case X_MIN: top = b < a ? b : a; break;
            case X_MAX: top = b > a ? b : a; break;
            case X_DIV:
                if (b == 0) return false;
                top = floor_div<V, U>(a, b);
                break;
            case X_MOD:
                if (b == 0) return false;
                top = euclid_mod<V, U>(a, b);
                break;
            case X_EQ: top = a == b; break;
            case X_NE: top = a != b; break;
            case X_LT: top = a < b; break;
            case X_LE: top = a <= b; break;
            case X_GT: top = a > b; break;
            case X_GE: top = a >= b; break;
            case X_AND: top = (a != 0) & (b != 0); break;
            case X_OR: top = (a != 0) | (b != 0); break;
            }
            break;
        }
        default: return false;   // not produced by the lowering
        }
    }
}

// Per-warp histogram cache: the emit kernel counts digits in shared memory.
struct EmitShared {
    unsigned int hist[kMaxPasses][kRadixBins];
};

// Adds one key per lane in `ok` to the shared digit histograms of every
// radix pass.  When all lanes' digits agree (the usual case for the digits
// above the index field) the lowest lane adds the whole warp's count at
// once; otherwise every lane adds its own key.
__device__ __forceinline__ void hist_add(EmitShared *sh, const KeyLayout &L, unsigned long long key, bool ok)
{
    const unsigned om = __ballot_sync(kFull, ok);
    if (om == 0) return;
    const int lead = __ffs(om) - 1;
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t q = 0; q < L.passes; q++) {
        uint32_t d = (uint32_t)(key >> (L.sort_lo + q * L.digit_bits)) & ((1u << L.digit_bits) - 1);
        uint32_t d0 = __shfl_sync(kFull, d, lead);
        if (__all_sync(kFull, !ok || d == d0)) {
            if ((int)lane == lead) atomicAdd(&sh->hist[q][d0], (unsigned)__popc(om));
        } else if (ok) {
            atomicAdd(&sh->hist[q][d], 1u);
        }
    }
}

__device__ __forceinline__ unsigned long long make_key(uint32_t p, uint32_t phase, uint32_t loc, unsigned long long idx,
                                                      unsigned long long tidpart, uint32_t wbit, const KeyLayout &L)
{
    unsigned long long key = ((unsigned long long)p << L.phase_bits) | phase;
    key = (key << L.loc_bits) | loc;
    key = (key << L.idx_bits) | idx;
    return (key << (L.tid_bits + 1)) | tidpart | wbit;
}

__device__ __forceinline__ unsigned long long key_or_zero(bool ok, uint32_t p, uint32_t phase, uint32_t loc,
                                                         unsigned long long idx, unsigned long long tidpart,
                                                         uint32_t flags, const KeyLayout &L)
{
    return ok ? make_key(p, phase, loc, idx, tidpart, flags & AF_WRITE, L) : 0ull;
}

// Post-operation of a fast-loop index on its linear value.
template <typename V, typename U>
__device__ __forceinline__ V fast_post(V v, uint32_t kind, U c)
{
    if (kind == FP_MASK) return (V)((U)v & c);
    if (kind == FP_MOD) return euclid_mod<V, U>(v, (V)c);
    if (kind == FP_DIV) return floor_div<V, U>(v, (V)c);
    return v;
}

// Interpretation modes of one item.
enum : int {
    M_COUNT = 0,   // accesses, syncs and the first error per (item, thread)
    M_EMIT = 1,    // one sort key per access
    M_TABLE = 2,   // one owner-record update per access
    M_CELL = 3,    // which threads access / write one given cell
};

// Applies each valid lane's access to its owner record (owner.cuh); the
// update that creates a record marks its block as touched.  When every valid
// lane hits one cell (an index that does not depend on tid), one lane
// updates the record for the warp.  The record is read first (through L2,
// where every SM sees the same record; nothing here relies on what an SM's
// L1 may still hold from earlier launches); the update is skipped when the
// copy already implies it.
__device__ __forceinline__ void table_put(const BatchArgs &a, bool ok, unsigned long long off, uint32_t tid,
                                          uint32_t w)
{
    const unsigned m = __ballot_sync(kFull, ok);
    if (m == 0) return;
    const int lead = __ffs(m) - 1;
    const unsigned long long off0 = __shfl_sync(kFull, off, lead);
    uint32_t *cell = reinterpret_cast<uint32_t *>(a.table) + off;
    bool created = false;
    if (__all_sync(kFull, !ok || off == off0)) {
        const unsigned wm = __ballot_sync(kFull, ok && w);
        if ((int)(threadIdx.x & 31) == lead)
            created = __popc(m) >= 2 ? owner_put_many(cell, __ldcg(cell), wm != 0)
                                     : owner_put(cell, __ldcg(cell), tid, w);
    } else if (ok) {
        created = owner_put(cell, __ldcg(cell), tid, w);
    }
    if (created) owner_touch(a.touch, off, kTabBlockLog);
}

// The cell whose accessors the M_CELL pass collects.
struct CellTarget {
    uint32_t phase, loc;
    unsigned long long idx;
};

// Interprets one item for the 32 threads of a warp (threads 32g .. 32g+31).
// All lanes fetch the instruction at the smallest pc among running lanes and
// only lanes at that pc execute it, so lanes that diverge on a thread-
// dependent condition or trip count re-converge at the join point.
template <typename V, int MODE>
__device__ void run_item(const BatchArgs &a, uint32_t p, const DevProto &P, const ItemDesc &it, uint32_t k,
                         uint32_t g, uint32_t w, EmitShared *sh, const CellTarget &tg)
{
    using U = typename Unsigned<V>::T;
    constexpr bool EMIT = MODE == M_EMIT;
    constexpr bool TAB = MODE == M_TABLE;
    constexpr bool CELL = MODE == M_CELL;
    constexpr bool PHASED = MODE != M_COUNT;      // knows the phase of every access
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t tid = g * 32 + lane;
    const bool alive = tid < P.nthreads;
    const Insn *prog = a.insns + P.insn_off;
    const uint64_t *xc = a.xcode + P.xcode_off;
    const uint64_t *cells = a.cells + P.cells_off;
    const uint64_t li = P.lane_off + (uint64_t)k * P.nthreads + tid;

    V vars[kMaxVars];
    V his[kMaxVars];
    uint32_t count = 0, syncs = 0, err = 0;
    uint32_t pc = it.start_pc;
    bool running = alive;

    // Prologue: position the split loops at this item's iteration(s).
    if (running) {
        for (uint32_t l = 0; l < it.nsplit; l++) {
            Insn L = load_insn(prog + it.split_pc[l]);
            V lo, hi;
            if (!eval<V>(xc, L.c, tid, vars, lo) || !eval<V>(xc, L.d, tid, vars, hi)) {
                err = kErrDiv0; running = false; break;
            }
            uint64_t trip = lo < hi ? (uint64_t)(U)((U)hi - (U)lo) : 0;
            if (it.chunked && l + 1 == it.nsplit) {
                uint64_t start = (uint64_t)it.j[l] * it.chunk;
                if (trip <= start) { running = false; break; }
                V x0 = (V)((U)lo + (U)start);
                vars[L.a] = x0;
                his[L.a] = (trip - start > it.chunk) ? (V)((U)x0 + (U)it.chunk) : hi;
            } else {
                if (trip <= it.j[l]) { running = false; break; }
                vars[L.a] = (V)((U)lo + (U)it.j[l]);
            }
        }
    }
    if (running && pc == it.stop_pc) running = false;

    uint32_t phase = 0;
    // count-free launches: every protocol has static phases, and the item's
    // start phase comes from the host instead of the scan
    if (PHASED && alive) phase = a.count_free ? __ldg(a.iphase + P.item_off + k) : a.phs[li];
    if (CELL && phase > tg.phase) running = false;     // phases only grow: nothing here reaches the cell
    unsigned long long cursor = 0, wend = 0;
    if (EMIT) {
        cursor = a.wbase[w];
        wend = cursor + a.wcnt[w];
    }
    const KeyLayout L = a.L;
    const unsigned long long tidpart = (((unsigned long long)tid) << 1);
    // owner-table state
    const uint64_t *cb = a.cbase + P.cells_off;
    uint32_t hit = 0;                                  // M_CELL: 1 accessed, 2 wrote

    while (true) {
        unsigned act = __ballot_sync(kFull, running);
        if (act == 0) break;
        uint32_t mpc = __reduce_min_sync(kFull, running ? pc : 0xFFFFFFFFu);
        const bool ex = running && pc == mpc;
        const Insn in = load_insn(prog + mpc);
        switch (in.op) {
        case I_ACCESS: {
            bool ok = ex;
            V idx = 0;
            // the witness pass runs only protocols none of whose accesses
            // fails, and needs the index only of accesses in the cell's phase
            // and array; neither it nor the table pass needs the index of an
            // access the range pass applies (k_finalize adds its witnesses)
            const bool rng = a.range_on && (in.a & AF_RANGE);
            // (the sort path with range keys: k_range_emit writes these keys)
            const bool rngk = a.range_keys && (in.a & AF_RANGE);
            const bool need = CELL ? (phase == tg.phase && in.b == tg.loc && !rng)
                                   : TAB ? !rng : !rngk && (PHASED || (in.a & AF_EVAL_IN_COUNT));
            if (ex && need) {
                if (!eval<V>(xc, in.c, tid, vars, idx)) { err = kErrDiv0; ok = false; }
                else if (idx < 0 || (uint64_t)(U)idx >= __ldg(cells + in.b)) { err = kErrOob; ok = false; }
            }
            if (ex && !ok) running = false;
            if (EMIT) {
                const bool ke = ok && !rngk;
                unsigned em = __ballot_sync(kFull, ke);
                if (ke) {
                    unsigned long long pos = cursor + __popc(em & lanemask_lt());
                    unsigned long long key = make_key(p, phase, in.b, (unsigned long long)(U)idx, tidpart, in.a & AF_WRITE, L);
                    if (pos < wend && pos < a.nkeys) a.keys[0][pos] = key;
                    else atomicOr(&a.ctrl->flags, CF_EMIT_OVERFLOW);
                }
                hist_add(sh, L, key_or_zero(ke, p, phase, in.b, (unsigned long long)(U)idx, tidpart, in.a, L), ke);
                cursor += __popc(em);
            } else if (TAB) {
                const bool put = ok && phase < P.tab_phases;
                if (ok && !put) atomicOr(&a.ctrl->flags, CF_TABLE_RANGE);
                const unsigned long long off =
                    put ? P.tab_off + (uint64_t)phase * P.cells_sum + __ldg(cb + in.b) + (uint64_t)(U)idx : 0ull;
                // an access the range pass applies is only counted here
                table_put(a, !rng && put && off >= a.shard_lo && off < a.shard_hi, off, tid, in.a & AF_WRITE);
            } else if (CELL) {
                if (ok && !rng && phase == tg.phase && in.b == tg.loc && (unsigned long long)(U)idx == tg.idx)
                    hit |= 1u | ((in.a & AF_WRITE) << 1);
            } else if (ok && !rngk) {
                count++;
            }
            if (TAB && ok && !(rng && a.rcount)) count++;      // (range tuples: counted on the host)
            if (ok) pc++;
            break;
        }
        case I_SYNC:
            if (ex) {
                if (PHASED) phase++; else syncs++;
                pc++;
                if (CELL && phase > tg.phase) running = false;
            }
            break;
        case I_LOOP:
            if (ex && (((TAB || CELL) && a.range_on) || (!TAB && !CELL && a.range_keys)) && (in.b & LB_RANGE_ONLY)) {
                pc = (uint32_t)in.e + 1;            // the range pass has the whole loop
                break;
            }
            if (ex) {
                V lo, hi;
                if (!eval<V>(xc, in.c, tid, vars, lo) || !eval<V>(xc, in.d, tid, vars, hi)) {
                    err = kErrDiv0; running = false;
                } else if (lo < hi) {
                    vars[in.a] = lo; his[in.a] = hi; pc++;
                } else {
                    pc = (uint32_t)in.e + 1;
                }
            }
            break;
        case I_ENDLOOP:
            if (ex) {
                V x = (V)((U)vars[in.a] + 1);
                vars[in.a] = x;
                pc = x < his[in.a] ? (uint32_t)in.c : pc + 1;
            }
            break;
        case I_IF:
            if (ex) {
                V c;
                if (!eval<V>(xc, in.c, tid, vars, c)) { err = kErrDiv0; running = false; }
                else pc = c ? pc + 1 : (uint32_t)in.d;
            }
            break;
        case I_JUMP:
            if (ex) pc = (uint32_t)in.c;
            break;
        case I_FASTLOOP: {
            V lo = 0, hi = 0;
            bool okb = ex;
            if (ex) {
                if (it.chunked == 2 && mpc == it.split_pc[it.nsplit - 1]) {
                    lo = vars[in.a]; hi = his[in.a];            // this item's chunk of the loop
                } else if (!eval<V>(xc, in.c, tid, vars, lo) || !eval<V>(xc, in.d, tid, vars, hi)) {
                    err = kErrDiv0; running = false; okb = false;
                }
            }
            const uint64_t trip = (okb && lo < hi) ? (uint64_t)(U)((U)hi - (U)lo) : 0;
            const uint32_t m = (uint32_t)in.e;
            // the table and witness passes take a loop whose accesses the
            // range pass all applies in one step: the table pass counts them
            bool skip = ((TAB || CELL) && a.range_on) || (EMIT && a.range_keys);
            for (uint32_t j = 0; j < m && skip; j++) skip = (load_insn(prog + mpc + 1 + j).a & AF_RANGE) != 0;
            if (!PHASED) {
                // (with range keys the range accesses' tuples are the pieces')
                uint32_t mc = m;
                if (a.range_keys)
                    for (uint32_t j = 0; j < m; j++) mc -= (load_insn(prog + mpc + 1 + j).a & AF_RANGE) ? 1u : 0u;
                if (okb) { count += (uint32_t)(trip * mc); syncs += (uint32_t)(trip * in.b); }
            } else if (skip) {
                if (okb) {
                    if (TAB && !a.rcount) count += (uint32_t)(trip * m);
                    phase += (uint32_t)(trip * in.b);
                }
                if (CELL && phase > tg.phase) running = false;
            } else {
                V rest[kFastMax];
                U coef[kFastMax], pcon[kFastMax];
                uint32_t meta[kFastMax];
                uint64_t lim[kFastMax];                          // owner table: array size
#pragma unroll
                for (uint32_t j = 0; j < kFastMax; j++) {
                    if (j < m) {
                        const Insn A = load_insn(prog + mpc + 1 + j);
                        rest[j] = 0;
                        if (okb) eval<V>(xc, A.c, tid, vars, rest[j]);
                        coef[j] = (U)__ldg(xc + A.d);
                        pcon[j] = (U)__ldg(xc + A.d + 1);
                        meta[j] = (uint32_t)A.a | ((uint32_t)A.b << 8);
                        meta[j] |= (uint32_t)A.e << 24;          // phase offset: at most 255 syncs per iteration
                        if (TAB) lim[j] = __ldg(cells + A.b);
                    }
                }
                const uint32_t spi = in.b;
                for (uint64_t t = 0;; t++) {
                    const uint32_t ph0 = phase + (uint32_t)(t * spi);
                    const bool act = okb && t < trip && (!CELL || ph0 <= tg.phase);
                    const unsigned am = __ballot_sync(kFull, act);
                    if (am == 0) break;
                    const V x = (V)((U)lo + (U)t);
                    const unsigned long long before = __popc(am & lanemask_lt());
#pragma unroll
                    for (uint32_t j = 0; j < kFastMax; j++) {
                        if (j < m) {
                            const uint32_t mt = meta[j];
                            const V v = (V)((U)rest[j] + coef[j] * (U)x);
                            const V idx = fast_post<V, U>(v, (mt >> 2) & 3, pcon[j]);
                            const uint32_t ph = ph0 + (mt >> 24), loc = (mt >> 8) & 0xFFFF;
                            if (EMIT && !(a.range_keys && (mt & AF_RANGE))) {
                                const unsigned long long key =
                                    act ? make_key(p, ph, loc, (unsigned long long)(U)idx, tidpart, mt & AF_WRITE, L)
                                        : 0ull;
                                if (act) {
                                    unsigned long long pos = cursor + before;
                                    if (pos < wend && pos < a.nkeys) a.keys[0][pos] = key;
                                    else atomicOr(&a.ctrl->flags, CF_EMIT_OVERFLOW);
                                }
                                hist_add(sh, L, key, act);
                                cursor += __popc(am);
                            } else if (TAB) {
                                // the lowering proved the index in range; the check keeps every
                                // table write inside this protocol's rows regardless
                                const bool put = act && ph < P.tab_phases && idx >= 0 && (uint64_t)(U)idx < lim[j];
                                if (act && !put) atomicOr(&a.ctrl->flags, CF_TABLE_RANGE);
                                const unsigned long long off =
                                    put ? P.tab_off + (uint64_t)ph * P.cells_sum + __ldg(cb + loc) + (uint64_t)(U)idx
                                        : 0ull;
                                const bool mine = !(a.range_on && (mt & AF_RANGE));
                                table_put(a, mine && put && off >= a.shard_lo && off < a.shard_hi, off, tid,
                                          mt & AF_WRITE);
                            } else if (CELL) {
                                if (act && !(a.range_on && (mt & AF_RANGE)) && ph == tg.phase && loc == tg.loc &&
                                    (unsigned long long)(U)idx == tg.idx)
                                    hit |= 1u | ((mt & AF_WRITE) << 1);
                            }
                        }
                    }
                }
                if (okb) phase += (uint32_t)(trip * spi);
                if (TAB && okb) {
                    uint32_t mc = m;                  // range accesses' tuples are counted on the host
                    if (a.rcount)
                        for (uint32_t j = 0; j < m; j++) mc -= (meta[j] & AF_RANGE) ? 1u : 0u;
                    count += (uint32_t)(trip * mc);
                }
                if (CELL && phase > tg.phase) running = false;
            }
            if (okb) pc = mpc + 1 + m;
            break;
        }
        default:
            if (ex) running = false;
            break;
        }
        if (ex && running && pc == it.stop_pc) running = false;
    }

    if (!PHASED && alive) {
        a.cnt[li] = count;
        a.syn[li] = syncs;
        if (err) {
            a.erro[li] = ((unsigned long long)count << 8) | err;
            atomicMin(&a.err_key[p], ((unsigned long long)tid << 32) | k);
        }
    }
    if (!PHASED) {
        uint32_t total = __reduce_add_sync(kFull, count);
        if (lane == 0) {
            a.wcnt[w] = total;
            if (total) {
                atomicAdd(&a.blocksum[w / kWScanPerBlock], (unsigned long long)total);
                atomicAdd(&a.ptuples[p], (unsigned long long)total);
            }
        }
    }
    if (TAB && a.count_free) {
        // no count pass ran: the table pass counts the tuples
        const uint32_t total = __reduce_add_sync(kFull, count);
        if (lane == 0 && total) {
            atomicAdd(&a.ptuples[p], (unsigned long long)total);
            atomicAdd(&a.ctrl->total, (unsigned long long)total);
        }
    }
    if (CELL) {
        // the warp's lanes that share a hit word set their bits with one
        // update (a race's cell is usually hit by many threads)
        const uint64_t b = P.tid_off + tid;
        const unsigned grp = __match_any_sync(kFull, b >> 5);
        const uint32_t bit = 1u << (uint32_t)(b & 31);
        const uint32_t acc = __reduce_or_sync(grp, (hit & 1u) ? bit : 0u);
        const uint32_t wr = __reduce_or_sync(grp, (hit & 2u) ? bit : 0u);
        if (lane == (uint32_t)(__ffs(grp) - 1)) {
            if (acc) atomicOr(&a.hit_acc[b >> 5], acc);
            if (wr) atomicOr(&a.hit_wr[b >> 5], wr);
        }
    }
}

// ------------------------------------------------------------------ kernels

// Programmatic dependent launch: the kernels after init are launched with
// programmatic stream serialization, so a kernel's blocks may start while
// the previous kernel drains.  Each first lets its own successor launch
// (every block of it is resident by then, so the successor's waiting blocks
// cannot keep any of it from running), then waits until the previous kernel
// has completed and its writes are visible.  Under a plain launch both are
// no-ops.
//
// Then a device-scope acquire fence, so that no later load of the thread is
// ordered before the writes the wait made visible.  It is a defence only:
// the kernels read data that earlier kernels of a launch write through L2
// (ld.global.cg), owner records included, and do not depend on what an SM's
// L1 may still hold.
__device__ __forceinline__ void pdl_begin()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

__global__ void k_init(BatchArgs a)
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i < a.nprotos) {
        a.err_key[i] = kNone;
        a.div_tid[i] = 0xFFFFFFFFu;
        a.best_pos[i] = kNone;
        a.ptuples[i] = a.rcount && a.rtup ? a.rtup[i] : 0ull;    // range tuples: counted on the host
    }
    if (i < (uint64_t)kMaxPasses * kRadixBins) a.hist[i] = 0;
    if (i < a.nwblocks) a.blocksum[i] = 0;
    if (i < sizeof(Control) / sizeof(unsigned int)) reinterpret_cast<unsigned int *>(a.ctrl)[i] = 0;
    if (i == 0) *a.epoch = *a.epoch + 1;
}

// The witness cell of protocol P from its first racy owner-table position.
__device__ __forceinline__ CellTarget decode_cell(const BatchArgs &a, const DevProto &P, unsigned long long pos)
{
    const unsigned long long rel = pos - P.tab_off;
    const unsigned long long row = rel / P.cells_sum;
    const unsigned long long c = rel - row * P.cells_sum;
    const uint64_t *cb = a.cbase + P.cells_off;
    uint32_t l = 0;
    while (l + 1 < P.nlocs && __ldg(cb + l + 1) <= c) l++;
    return CellTarget{(uint32_t)row, l, c - __ldg(cb + l)};
}

template <int MODE> struct InterpShared { unsigned int unused; };
template <> struct InterpShared<M_EMIT> { EmitShared e; };

// One kernel per arithmetic width (WIDE: 64-bit); each skips the warp-items
// of protocols of the other width.
template <int MODE, bool WIDE>
__global__ void __launch_bounds__(256) k_interp(BatchArgs a)
{
    pdl_begin();
    constexpr bool EMIT = MODE == M_EMIT;
    __shared__ InterpShared<MODE> shm;
    EmitShared *sh = nullptr;
    if constexpr (EMIT) {
        sh = &shm.e;
        for (int i = threadIdx.x; i < kMaxPasses * kRadixBins; i += blockDim.x) (&sh->hist[0][0])[i] = 0;
        __syncthreads();
    }
    const uint32_t warps = gridDim.x * (blockDim.x / 32);
    CellTarget tg{};
    uint32_t tg_proto = 0xFFFFFFFFu;     // M_CELL: protocol whose witness cell tg holds
    bool tg_live = false;
    for (uint32_t w = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; w < a.nwitems; w += warps) {
        const WarpItem wi = a.witems[w];
        const DevProto P = a.protos[wi.proto];
        if ((P.wide != 0) != WIDE) continue;
        if (MODE == M_CELL) {
            // only racy protocols whose verdict is not an error or a divergence
            if (wi.proto != tg_proto) {
                tg_proto = wi.proto;
                // the reductions of earlier kernels of this launch, read through L2
                const unsigned long long bp = __ldcg(a.best_pos + wi.proto);
                tg_live = bp != kNone && __ldcg(a.err_key + wi.proto) == kNone &&
                          __ldcg(a.div_tid + wi.proto) == 0xFFFFFFFFu;
                if (tg_live) tg = decode_cell(a, P, bp);
            }
            if (!tg_live) continue;
            // nothing to do for an item that starts after the witness phase,
            // or ends before it (the next item starts before it), in every lane
            const uint32_t tid = wi.g * 32 + (threadIdx.x & 31);
            const uint64_t lk = P.lane_off + (uint64_t)wi.k * P.nthreads + tid;
            bool reach;
            if (a.count_free)          // static phases: the same for every thread
                reach = tid < P.nthreads && __ldg(a.iphase + P.item_off + wi.k) <= tg.phase &&
                        (wi.k + 1 == P.nitems || __ldg(a.iphase + P.item_off + wi.k + 1) >= tg.phase);
            else
                reach = tid < P.nthreads && a.phs[lk] <= tg.phase &&
                        (wi.k + 1 == P.nitems || a.phs[lk + P.nthreads] >= tg.phase);
            if (!__any_sync(kFull, reach)) continue;
        }
        const ItemDesc it = a.items[P.item_off + wi.k];
        if (MODE != M_COUNT && MODE != M_CELL && wi.k == 0) {
            uint32_t tid = wi.g * 32 + (threadIdx.x & 31);
            if (a.count_free) {
                // static phases: no divergence is possible, and no scan
                // wrote the sync totals -- thread 0's, which the result
                // reports, is the protocol's static count
                if (tid == 0) a.totsyn[P.tid_off] = P.tab_phases - 1;
            } else if (tid < P.nthreads && a.totsyn[P.tid_off + tid] != a.totsyn[P.tid_off]) {
                // barrier divergence: every thread must run as many syncs as thread 0
                atomicMin(&a.div_tid[wi.proto], tid);
            }
        }
        if (WIDE) run_item<int64_t, MODE>(a, wi.proto, P, it, wi.k, wi.g, w, sh, tg);
        else run_item<int32_t, MODE>(a, wi.proto, P, it, wi.k, wi.g, w, sh, tg);
    }
    if constexpr (EMIT) {
        __syncthreads();
        for (int i = threadIdx.x; i < (int)(a.L.passes * kRadixBins); i += blockDim.x) {
            unsigned int v = (&sh->hist[0][0])[i];
            if (v) atomicAdd(&a.hist[i], (unsigned long long)v);
        }
    }
}

// Two roles.  Blocks [0, col_blocks): per-thread exclusive scan of syncs over
// items, 32 threads (columns) per block, each column's items split over the
// block's 8 warps.  The remaining blocks: exclusive scan of per-warp-item
// access counts (4096 per block; the block's offset is the sum of the earlier
// blocks' totals, accumulated by the count kernel).
__global__ void __launch_bounds__(kScanThreads) k_scan(BatchArgs a, uint32_t col_blocks)
{
    pdl_begin();
    if (blockIdx.x < col_blocks) {
        __shared__ uint32_t s_part[kScanThreads / 32][32];
        const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        const uint64_t c = (uint64_t)blockIdx.x * 32 + lane;
        const bool valid = c < a.ncols;
        DevProto P{};
        if (valid) {
            uint32_t lo = 0, hi = a.nprotos - 1;           // protocol owning column c
            while (lo < hi) {
                uint32_t mid = (lo + hi + 1) / 2;
                if (a.protos[mid].tid_off <= c) lo = mid; else hi = mid - 1;
            }
            P = a.protos[lo];
        }
        const uint32_t t = valid ? (uint32_t)(c - P.tid_off) : 0;
        const uint32_t K = valid ? P.nitems : 0;
        const uint32_t per = (K + kScanThreads / 32 - 1) / (kScanThreads / 32);
        const uint32_t k0 = min(K, wid * per), k1 = min(K, k0 + per);
        const uint32_t *syn = a.syn + P.lane_off + t;
        uint32_t sum = 0;
        uint32_t k = k0;
        for (; k + 8 <= k1; k += 8) {                      // eight loads in flight
            uint32_t v[8];
#pragma unroll
            for (int u = 0; u < 8; u++) v[u] = syn[(uint64_t)(k + u) * P.nthreads];
#pragma unroll
            for (int u = 0; u < 8; u++) sum += v[u];
        }
        for (; k < k1; k++) sum += syn[(uint64_t)k * P.nthreads];
        s_part[wid][lane] = sum;
        __syncthreads();
        uint32_t run = 0, total = 0;
        for (uint32_t w = 0; w < kScanThreads / 32; w++) {
            if (w < wid) run += s_part[w][lane];
            total += s_part[w][lane];
        }
        uint32_t *phs = a.phs + P.lane_off + t;
        for (k = k0; k < k1; k++) {
            uint64_t off = (uint64_t)k * P.nthreads;
            phs[off] = run;
            run += syn[off];
        }
        if (valid && wid == 0) a.totsyn[c] = total;
        return;
    }
    const uint32_t b = blockIdx.x - col_blocks;
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    __shared__ unsigned long long s_base;
    // offset of this block: the totals of all earlier blocks
    unsigned long long pre = 0;
    for (uint32_t i = threadIdx.x; i < b; i += kScanThreads) pre += a.blocksum[i];
    for (int o = 16; o; o >>= 1) pre += __shfl_xor_sync(kFull, pre, o);
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x / 32] = pre;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int i = 0; i < kScanThreads / 32; i++) s += s_warp[i];
        s_base = s;
        if (b + 1 == a.nwblocks) a.ctrl->total = s + a.blocksum[b];
    }
    __syncthreads();
    // scan 16 consecutive counts per thread
    constexpr int kPer = kWScanPerBlock / kScanThreads;
    uint64_t first = (uint64_t)b * kWScanPerBlock + threadIdx.x * kPer;
    uint32_t v[kPer];
    unsigned long long sum = 0;
#pragma unroll
    for (int i = 0; i < kPer; i++) {
        v[i] = first + i < a.nwitems ? a.wcnt[first + i] : 0;
        sum += v[i];
    }
    // block-wide exclusive scan of the per-thread sums
    const int lane = threadIdx.x & 31, wid = threadIdx.x / 32;
    unsigned long long incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    __syncthreads();
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    unsigned long long wpre = 0;
    for (int i = 0; i < wid; i++) wpre += s_warp[i];
    unsigned long long run = s_base + wpre + incl - sum;
#pragma unroll
    for (int i = 0; i < kPer; i++) {
        if (first + i < a.nwitems) a.wbase[first + i] = run;
        run += v[i];
    }
}

// ------------------------------------------------------------ radix pass

// Number of non-trivial passes (digit not constant over all keys) before
// `pass`, and whether `pass` itself is non-trivial.  Uniform over the block.
__device__ int nontrivial_before(const BatchArgs &a, uint32_t pass, bool *self)
{
    int before = 0;
    for (uint32_t q = 0; q <= pass; q++) {
        int nz = __syncthreads_count(threadIdx.x < kRadixBins && a.hist[q * kRadixBins + threadIdx.x] != 0);
        if (q < pass) before += nz > 1;
        else *self = nz > 1;
    }
    return before & 1 ? 1 : 0;
}

template <int ITEMS>
__global__ void __launch_bounds__(kRadixThreads, ITEMS >= 24 ? 2 : 3) k_radix(BatchArgs a, uint32_t pass)
{
    __shared__ radix::PassShared<kRadixThreads, ITEMS> sh;
    bool self;
    const int before = nontrivial_before(a, pass, &self);
    if (!self) return;                       // constant digit: the pass would not move any key
    radix::PassArgs A;
    A.src = a.keys[before];
    A.dst = a.keys[before ^ 1];
    A.n = a.nkeys;
    A.shift = a.L.sort_lo + pass * a.L.digit_bits;
    A.nbits = min(a.L.digit_bits, a.L.sort_bits - pass * a.L.digit_bits);
    A.hist = a.hist + pass * kRadixBins;
    A.status = a.status + (uint64_t)pass * a.ntiles * kRadixBins;
    A.tile_counter = &a.ctrl->tile_counter[pass];
    A.tag = (unsigned long long)(*a.epoch & radix::kTagMask) << radix::kTagShift;
    A.flags = &a.ctrl->flags;
    // the test hook stalls the look-back and gives each wait 64 spins
    A.spin_limit = a.stall_lookback ? 64u : radix::kSpinLimit;
    A.stall_first = a.stall_lookback;
    radix::pass<kRadixThreads, ITEMS>(A, sh);
}

// ------------------------------------------------------------- detection
// A segment (equal proto | phase | array | index) is racy iff it holds a
// write and two distinct tids (Definition 1: a writer and a second,
// different accessor).  Per contiguous piece of a segment the detector keeps
// (min tid, max tid, any write, whether the piece holds the segment's first
// key, that key's position): an associative summary, combined across keys
// by a segmented scan (segment starts are the scan's reset flags).

__device__ __forceinline__ Agg agg_empty() { return Agg{0xFFFFFFFFu, 0u, 0u, kNone}; }

__device__ __forceinline__ Agg agg_key(unsigned long long k, uint32_t tid_mask, bool head, unsigned long long pos)
{
    uint32_t t = (uint32_t)(k >> 1) & tid_mask;
    return Agg{t, t, (uint32_t)(k & 1) | (head ? 2u : 0u) | 4u, head ? pos : kNone};
}

// a is the left piece, b the right piece of the same segment
__device__ __forceinline__ Agg agg_cat(const Agg &a, const Agg &b)
{
    if (!(a.bits & 4)) return b;
    if (!(b.bits & 4)) return a;
    return Agg{min(a.mint, b.mint), max(a.maxt, b.maxt), (a.bits | (b.bits & 1)), a.start};
}

__device__ __forceinline__ bool agg_racy(const Agg &a) { return (a.bits & 1) && a.mint != a.maxt; }

struct SegVal {
    uint32_t f;                 // a segment starts inside this range
    Agg v;                      // summary of the range's last segment piece
};

__device__ __forceinline__ SegVal seg_op(const SegVal &l, const SegVal &r)
{
    return SegVal{l.f | r.f, r.f ? r.v : agg_cat(l.v, r.v)};
}

__device__ __forceinline__ SegVal seg_shfl_up(const SegVal &x, int o)
{
    SegVal y;
    y.f = __shfl_up_sync(kFull, x.f, o);
    y.v.mint = __shfl_up_sync(kFull, x.v.mint, o);
    y.v.maxt = __shfl_up_sync(kFull, x.v.maxt, o);
    y.v.bits = __shfl_up_sync(kFull, x.v.bits, o);
    y.v.start = __shfl_up_sync(kFull, x.v.start, o);
    return y;
}

// Exclusive segmented scan over the threads of a block (all threads call).
// s_warp: shared scratch of blockDim/32 entries.
__device__ SegVal block_seg_exclusive(SegVal x, SegVal *s_warp)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    SegVal inc = x;
    for (int o = 1; o < 32; o <<= 1) {
        SegVal y = seg_shfl_up(inc, o);
        if (lane >= o) inc = seg_op(y, inc);
    }
    SegVal exc = seg_shfl_up(inc, 1);
    if (lane == 0) exc = SegVal{0, agg_empty()};
    if (lane == 31) s_warp[wid] = inc;
    __syncthreads();
    SegVal pre{0, agg_empty()};
    for (int w = 0; w < wid && w < nw; w++) pre = seg_op(pre, s_warp[w]);
    __syncthreads();
    return seg_op(pre, exc);
}

// Sorted-key buffer parity: passes whose digit was constant did not move
// the keys.  Uniform over the block.
__device__ __forceinline__ int sorted_parity(const BatchArgs &a)
{
    int before = 0;
    for (uint32_t q = 0; q < a.L.passes; q++) {
        int nz = __syncthreads_count(threadIdx.x < kRadixBins && a.hist[q * kRadixBins + threadIdx.x] != 0);
        before += nz > 1;
    }
    return before & 1;
}

struct DetectShared {
    unsigned long long keys[kDetectTile + kDetectTile / 16];   // one pad word per 16 keys
    SegVal warp[kDetectThreads / 32];
    unsigned long long best;
};

__device__ __forceinline__ uint32_t pad16(uint32_t i) { return i + (i >> 4); }

// Records a complete racy segment of protocol `proto` starting at `pos`.
__device__ __forceinline__ void note_racy(const BatchArgs &a, uint32_t proto, uint32_t tile_proto,
                                          unsigned long long pos, unsigned long long &local_best)
{
    if (proto == tile_proto) local_best = min(local_best, pos);
    else if (proto < a.nprotos) atomicMin(&a.best_pos[proto], pos);
}

// One 4096-key tile per block: complete segments inside the tile are judged
// here; the pieces of segments that cross the tile's edges go to the tile
// record for k_resolve.
__global__ void __launch_bounds__(kDetectThreads) k_detect(BatchArgs a)
{
    __shared__ DetectShared sh;
    const unsigned long long *keys = a.keys[sorted_parity(a)];
    const uint64_t n = a.nkeys;
    const uint32_t lo = a.L.sort_lo;
    const uint32_t proto_shift = a.L.sort_bits - a.L.proto_bits;
    const uint32_t tid_mask = a.L.tid_bits ? (1u << a.L.tid_bits) - 1 : 0;
    const uint64_t base = (uint64_t)blockIdx.x * kDetectTile;
    const uint32_t valid = (uint32_t)min((uint64_t)kDetectTile, n - base);
    for (uint32_t i = threadIdx.x; i < valid; i += kDetectThreads) sh.keys[pad16(i)] = keys[base + i];
    if (threadIdx.x == 0) sh.best = kNone;
    __syncthreads();
    const unsigned long long prev_seg = base ? (keys[base - 1] >> lo) : ~0ull;
    const bool has_next = base + valid < n;
    const unsigned long long next_seg = has_next ? (keys[base + valid] >> lo) : ~0ull;
    const unsigned long long first_seg = sh.keys[0] >> lo;
    const uint32_t tile_proto = a.L.proto_bits ? (uint32_t)(first_seg >> proto_shift) : 0;

    // this thread's keys: [i0, i1) of the tile
    const uint32_t i0 = threadIdx.x * kDetectItems;
    const uint32_t i1 = min(valid, i0 + kDetectItems);
    // pass 1: the thread's summary for the scan
    SegVal mine{0, agg_empty()};
    unsigned long long pseg = i0 == 0 ? prev_seg : (i0 < valid ? sh.keys[pad16(i0 - 1)] >> lo : 0);
    for (uint32_t i = i0; i < i1; i++) {
        unsigned long long k = sh.keys[pad16(i)];
        unsigned long long sg = k >> lo;
        bool head = (base + i == 0) || sg != pseg;
        SegVal e{head ? 1u : 0u, agg_key(k, tid_mask, head, base + i)};
        mine = seg_op(mine, e);
        pseg = sg;
    }
    SegVal carry = block_seg_exclusive(mine, sh.warp);
    // pass 2: close every segment that ends inside the tile
    unsigned long long local_best = kNone;
    Agg run = carry.v;
    unsigned long long run_seg = i0 == 0 ? prev_seg : (i0 < valid ? sh.keys[pad16(i0 - 1)] >> lo : 0);
    TileRec *rec = a.trec + blockIdx.x;
    for (uint32_t i = i0; i < i1; i++) {
        unsigned long long k = sh.keys[pad16(i)];
        unsigned long long sg = k >> lo;
        bool head = (base + i == 0) || sg != run_seg;
        if (head) {
            if (run.bits & 4) {            // the piece before i is a whole segment or the tile's first one
                if (run.bits & 2) {
                    if (agg_racy(run))
                        note_racy(a, a.L.proto_bits ? (uint32_t)(run_seg >> proto_shift) : 0, tile_proto,
                                  run.start, local_best);
                } else {
                    rec->first = run;      // continues from the previous tile, ends here
                }
            }
            run = agg_key(k, tid_mask, true, base + i);
        } else {
            run = agg_cat(run, agg_key(k, tid_mask, false, base + i));
        }
        run_seg = sg;
    }
    if (i1 == valid && i0 < valid) {
        // the thread holding the tile's last key settles the open segment
        uint32_t flags = 0;
        if (base && prev_seg == first_seg) flags |= TR_STARTS_CONT;
        if (has_next && next_seg == run_seg) flags |= TR_ENDS_CONT;
        if (flags & TR_ENDS_CONT) {
            if (run.bits & 2) rec->last = run;
            else { rec->first = run; flags |= TR_SINGLE; }
        } else if (run.bits & 2) {
            if (agg_racy(run))
                note_racy(a, a.L.proto_bits ? (uint32_t)(run_seg >> proto_shift) : 0, tile_proto, run.start,
                          local_best);
        } else {
            rec->first = run;              // the continuing segment ends at the tile's end
        }
        rec->first_seg = first_seg;
        rec->last_seg = run_seg;
        rec->flags = flags;
    }
    if (local_best != kNone) atomicMin(&sh.best, local_best);
    __syncthreads();
    if (threadIdx.x == 0 && sh.best != kNone && tile_proto < a.nprotos) atomicMin(&a.best_pos[tile_proto], sh.best);
}

// One block settles every segment that crosses tile edges: a segment opened
// as the last piece of tile r (TR_ENDS_CONT without TR_SINGLE) runs through
// single tiles and ends in the first piece of the next tile that is not
// single.  Segmented scan over tiles, each thread a contiguous chunk.
__global__ void __launch_bounds__(1024) k_resolve(BatchArgs a)
{
    __shared__ SegVal s_warp[32];
    const uint32_t nt = a.ndtiles;
    const uint32_t per = (nt + blockDim.x - 1) / blockDim.x;
    const uint32_t r0 = min(nt, threadIdx.x * per), r1 = min(nt, r0 + per);
    const uint32_t proto_shift = a.L.sort_bits - a.L.proto_bits;
    auto element = [&](uint32_t r, const TileRec &t) {
        bool single = t.flags & TR_SINGLE;
        SegVal e;
        e.f = single ? 0u : 1u;
        e.v = single ? t.first : ((t.flags & TR_ENDS_CONT) ? t.last : agg_empty());
        return e;
    };
    SegVal mine{0, agg_empty()};
    for (uint32_t r = r0; r < r1; r++) mine = seg_op(mine, element(r, a.trec[r]));
    SegVal carry = block_seg_exclusive(mine, s_warp);
    Agg run = carry.v;
    for (uint32_t r = r0; r < r1; r++) {
        const TileRec t = a.trec[r];
        if (t.flags & TR_SINGLE) { run = agg_cat(run, t.first); continue; }
        if (t.flags & TR_STARTS_CONT) {
            Agg whole = agg_cat(run, t.first);
            if ((whole.bits & 2) && agg_racy(whole)) {
                uint32_t proto = a.L.proto_bits ? (uint32_t)(t.first_seg >> proto_shift) : 0;
                if (proto < a.nprotos) atomicMin(&a.best_pos[proto], whole.start);
            }
        }
        run = (t.flags & TR_ENDS_CONT) ? t.last : agg_empty();
    }
}

// ------------------------------------------------------------ owner table

// Protocol whose table rows hold record `pos` (the last one starting at or
// before it).
__device__ uint32_t proto_of_record(const BatchArgs &a, unsigned long long pos)
{
    uint32_t lo = 0, hi = a.nprotos - 1;
    while (lo < hi) {
        uint32_t mid = (lo + hi + 1) / 2;
        if (__ldg(&a.protos[mid].tab_off) <= pos) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Lists the touched blocks of the owner table: one thread per touch word,
// one atomicAdd per warp for its words' share of the list; clears the words
// it read and the witness hit bits for the M_CELL pass.
__global__ void __launch_bounds__(kTabScanThreads) k_tlist(BatchArgs a)
{
    pdl_begin();
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t gthreads = (uint64_t)gridDim.x * kTabScanThreads;
    for (uint64_t i = blockIdx.x * (uint64_t)kTabScanThreads + threadIdx.x; i < a.nhit; i += gthreads) {
        a.hit_acc[i] = 0;
        a.hit_wr[i] = 0;
    }
    const uint64_t nwords = touch_words(a.tab_cells);
    const uint64_t cap = table_blocks(a.tab_cells);
    const uint64_t first = (blockIdx.x * (uint64_t)kTabScanThreads) & ~31ull;
    for (uint64_t base = first + (threadIdx.x & ~31u); base < nwords; base += gthreads) {
        const uint64_t wd = base + lane;
        // through L2: the table pass's blocks may have left lines of this
        // launch's data in this SM's L1, and a dependent launch that starts
        // early gets no fresh L1 (the same holds for the scan's reads below)
        const uint32_t bits = wd < nwords ? __ldcg(a.touch + wd) : 0u;
        if (bits) a.touch[wd] = 0;
        const uint32_t cnt = (uint32_t)__popc(bits);
        uint32_t incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, o);
            if ((int)lane >= o) incl += y;
        }
        const uint32_t total = __shfl_sync(kFull, incl, 31);
        if (total == 0) continue;
        unsigned long long at = 0;
        if (lane == 31) at = atomicAdd(&a.ctrl->touched, (unsigned long long)total);
        at = __shfl_sync(kFull, at, 31) + (incl - cnt);
        for (uint32_t b = bits; b; b &= b - 1, at++) {
            if (at < cap) a.tlist[at] = (uint32_t)(wd * 32 + (uint32_t)(__ffs(b) - 1));
            else atomicOr(&a.ctrl->flags, CF_TABLE_RANGE);
        }
    }
}

// Reads every listed block of the owner table: records each protocol's first
// racy cell -- the smallest position, since rows are phase-major, then array,
// then index, the lexicographic order of the witness -- and clears every
// record it read, so that the table is all zero again for the next launch
// (k_tlist cleared the touch words).  One warp per listed block.
__global__ void __launch_bounds__(kTabScanThreads) k_tscan(BatchArgs a)
{
    pdl_begin();
    constexpr int V4 = 2;                               // uint4 loads per lane per block
    constexpr int PER = kTabBlock / 32;                 // records per lane per block
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t gthreads = (uint64_t)gridDim.x * kTabScanThreads;
    __shared__ uint32_t s_proto;
    __shared__ unsigned long long s_best;
    if (threadIdx.x == 0) { s_proto = 0xFFFFFFFFu; s_best = kNone; }
    __syncthreads();
    unsigned long long listed = __ldcg(&a.ctrl->touched);
    if (listed > table_blocks(a.tab_cells)) listed = table_blocks(a.tab_cells);
    const uint64_t warps = gthreads / 32;
    // a lane's smallest racy position, per protocol ([cand_lo, cand_hi) its records)
    unsigned long long cand = kNone, cand_lo = 0, cand_hi = 0;
    uint32_t cand_p = 0;
    auto flush = [&]() {
        if (cand != kNone && __ldcg(&a.best_pos[cand_p]) > cand) atomicMin(&a.best_pos[cand_p], cand);
        cand = kNone;
    };
    auto note = [&](unsigned long long pos) {
        if (cand != kNone && pos >= cand_lo && pos < cand_hi) {
            cand = pos < cand ? pos : cand;
            return;
        }
        flush();
        cand_p = proto_of_record(a, pos);
        const DevProto &P = a.protos[cand_p];
        cand = pos;
        cand_lo = P.tab_off;
        cand_hi = P.tab_off + (uint64_t)P.tab_phases * P.cells_sum;
    };
    for (uint64_t e = (blockIdx.x * (uint64_t)kTabScanThreads + threadIdx.x) / 32; e < listed; e += warps) {
        const uint64_t blk = __ldcg(a.tlist + e);
        const uint4 *src = reinterpret_cast<const uint4 *>(a.table) + blk * (kTabBlock / 4) + (uint64_t)lane * V4;
        uint4 v[V4];
        // through L2: this SM's L1 may hold copies of these records that the
        // table pass read before other SMs updated them -- a stale zero would
        // leave its record uncleared for the next launch
#pragma unroll
        for (int q = 0; q < V4; q++) v[q] = __ldcg(src + q);
        uint4 *dst = reinterpret_cast<uint4 *>(a.table) + blk * (kTabBlock / 4) + (uint64_t)lane * V4;
        const unsigned long long pos0 = blk * kTabBlock + (uint64_t)lane * PER;
#pragma unroll
        for (int q = 0; q < V4; q++) {
            const uint4 x = v[q];
            if ((x.x | x.y | x.z | x.w) == 0) continue;
            const uint32_t r[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (owner_racy(r[k])) note(pos0 + q * 4 + k);
            dst[q] = make_uint4(0, 0, 0, 0);
        }
    }
    // final candidates: min over the warp, then over the block, when they
    // belong to one protocol (the usual case); otherwise each lane's own
    const unsigned has = __ballot_sync(kFull, cand != kNone);
    if (has) {
        const uint32_t p0 = __shfl_sync(kFull, cand_p, __ffs(has) - 1);
        if (__all_sync(kFull, cand == kNone || cand_p == p0)) {
            unsigned long long m = cand;
            for (int o = 16; o; o >>= 1) {
                const unsigned long long y = __shfl_xor_sync(kFull, m, o);
                m = y < m ? y : m;
            }
            cand = lane == 0 ? m : kNone;
            cand_p = p0;
            if (lane == 0) {
                const uint32_t prev = atomicCAS(&s_proto, 0xFFFFFFFFu, p0);
                if (prev == 0xFFFFFFFFu || prev == p0) { atomicMin(&s_best, m); cand = kNone; }
            }
        }
    }
    flush();
    __syncthreads();
    if (threadIdx.x == 0 && s_best != kNone) {
        cand = s_best;
        cand_p = s_proto;
        flush();
    }
}

// ------------------------------------------------------------- range pass
// Accesses whose index is (sigma * tid + c) mod m or sigma * tid + c
// (sigma = +-1, c a function of the loop variables), in loops and
// conditions that do not read tid and hold no sync: at one offset c, the
// threads whose index falls into a range of cells are one interval of tids
// (two when the remainder wraps).  The host lists, per task of kRangeRecs
// consecutive owner records, the (access, offset) pairs that reach it; one
// block per listed task holds the task's records in shared memory, merges
// the table pass's records there, applies the intervals, and finds the
// task's first racy record per protocol.  The table scan that follows reads
// the table pass's records elsewhere.

struct RangeShared {
    RPiece ent[kRangeChunk];                      // the round's pieces
    uint32_t pre[kRangeChunk];                    // also the task's racy-record bitmap at its end
    uint32_t n, tot, plain, bits[kRangeRecs / 8192];
    unsigned long long updates;                   // record updates the block made
};
static_assert(kRangeChunk * 32 >= kRangeRecs, "the racy bitmap needs a bit per record");

// The records [lo, hi) a piece's span covers (every step-th of them its own).
__device__ __forceinline__ void range_span(const RPiece &x, int32_t &lo, int32_t &hi)
{
    const int32_t len = (int32_t)(x.lenf & kRLen);
    const int32_t last = x.l0 + x.step * (len - 1);
    lo = len ? min(x.l0, last) : 0;
    hi = len ? max(x.l0, last) + 1 : 0;
}

// Whether two pieces may share a record: their spans overlap, unless both
// step by the same |s| > 1 from records in different residue classes mod s.
__device__ __forceinline__ bool range_meet(const RPiece &x, const RPiece &y)
{
    int32_t a0, a1, b0, b1;
    range_span(x, a0, a1);
    range_span(y, b0, b1);
    if (!(a0 < b1 && b0 < a1)) return false;
    const int32_t s = abs(x.step);
    return !(s > 1 && s == abs(y.step) && (x.l0 - y.l0) % s != 0);
}

// Applies the round's intervals (sh.ent[0 .. sh.n)) to the task's records:
// every (interval, offset) pair spread over the block.  Within one interval
// every record has one tid; when no two intervals share a record (checked
// for rounds of up to 64), no two threads update one record and each update
// is a plain read and write of the record (owner.cuh's rule), four records
// read before any is written; otherwise the updates are atomic.  Leaves
// sh.n at 0.
__device__ void range_apply(uint32_t *rec, RangeShared &sh)
{
    const uint32_t n = sh.n;
    if (threadIdx.x < 32) {
        bool clash = n > 64;
        for (uint32_t e = threadIdx.x; e < n && !clash; e += 32) {
            const RPiece x = sh.ent[e];
            for (uint32_t f = e + 1; f < n; f++)
                if (range_meet(x, sh.ent[f])) { clash = true; break; }
        }
        clash = __any_sync(kFull, clash);
        // exclusive prefix of the lengths
        uint32_t carry = 0;
        for (uint32_t b = 0; b < n; b += 32) {
            const uint32_t e = b + threadIdx.x;
            const uint32_t v = e < n ? (sh.ent[e].lenf & kRLen) : 0u;
            uint32_t inc = v;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, inc, o);
                if ((int)threadIdx.x >= o) inc += y;
            }
            if (e < n) sh.pre[e] = carry + inc - v;
            carry += __shfl_sync(kFull, inc, 31);
        }
        if (threadIdx.x == 0) { sh.tot = carry; sh.plain = clash ? 0u : 1u; sh.updates += carry; }
    }
    __syncthreads();
    const uint32_t total = sh.tot;
    const bool plain = sh.plain != 0;
    if (total >= n * 2u * kRangeThreads) {
        // long intervals: the block takes them one by one, a record per
        // thread (no position search)
        for (uint32_t e = 0; e < n; e++) {
            const RPiece x = sh.ent[e];
            const uint32_t len = x.lenf & kRLen, w = (x.lenf & kRWrite) ? 1u : 0u;
            const int32_t step = x.step;
            uint32_t o0 = threadIdx.x;
            if (x.lenf & kRSat) {
                // records two or more threads reach: "second thread" (and
                // "written") whatever they held
                const uint32_t bits = kOwnerMulti | (w << 31);
                for (; o0 < len; o0 += kRangeThreads) {
                    uint32_t *const r = rec + (x.l0 + step * (int32_t)o0);
                    if (plain) *r |= bits;
                    else if ((*r & bits) != bits) atomicOr(r, bits);
                }
                continue;
            }
            if (plain) {
                // four records per thread and step, every one in the interval
                const uint32_t wbit = w << 31;
                const int32_t d = step * (int32_t)kRangeThreads;
                for (; o0 + 3u * kRangeThreads < len; o0 += 4u * kRangeThreads) {
                    const int32_t i0 = x.l0 + step * (int32_t)o0;
                    const uint32_t t1 = x.t0 + o0 + 1u;
                    uint32_t old[4];
#pragma unroll
                    for (int k = 0; k < 4; k++) old[k] = rec[i0 + k * d];
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        rec[i0 + k * d] = owner_merge(old[k], t1 + (uint32_t)k * kRangeThreads, wbit);
                }
                for (; o0 < len; o0 += kRangeThreads) {
                    const int32_t i = x.l0 + step * (int32_t)o0;
                    rec[i] = owner_merge(rec[i], x.t0 + o0 + 1u, wbit);
                }
                continue;
            }
            // pieces that share records: a plain read first (a record
            // another piece has already saturated needs nothing), then a
            // claim by compare-and-swap or the missing bits
            for (; o0 < len; o0 += 4u * kRangeThreads) {
                int32_t ri[4];
                uint32_t cur[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const uint32_t o = o0 + (uint32_t)k * kRangeThreads;
                    ri[k] = o < len ? x.l0 + step * (int32_t)o : -1;
                }
#pragma unroll
                for (int k = 0; k < 4; k++) cur[k] = ri[k] >= 0 ? rec[ri[k]] : 0u;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    if (ri[k] < 0) continue;
                    const uint32_t t = x.t0 + o0 + (uint32_t)k * kRangeThreads;
                    uint32_t c = cur[k];
                    if (c == 0u) {
                        c = atomicCAS(rec + ri[k], 0u, (t + 1u) | (w << 31));
                        if (c == 0u) continue;
                    }
                    if (const uint32_t need = owner_need(c, t, w)) atomicOr(rec + ri[k], need);
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) sh.n = 0;
        return;
    }
    // short intervals: positions of the round spread over the block; this
    // thread's current interval kept in registers (entry e covers positions
    // [base, nxt) of the round)
    uint32_t e = 0, base = 0, nxt = 0;
    RPiece x{};
    if (total) { x = sh.ent[0]; nxt = n > 1 ? sh.pre[1] : total; }
    // per position: its record ri (-1: none), its thread + 1 (t1; 0 for a
    // kRSat piece) and the bits it brings (wb: "written" for a writer; for
    // kRSat also "second thread")
    for (uint32_t q0 = threadIdx.x; q0 < total; q0 += 4u * kRangeThreads) {
        int32_t ri[4];
        uint32_t t1[4], wb[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const uint32_t q = q0 + (uint32_t)k * kRangeThreads;
            ri[k] = -1;
            if (q < total) {
                while (q >= nxt) {                    // positions only grow
                    e++;
                    base = nxt;
                    x = sh.ent[e];
                    nxt = e + 1 < n ? sh.pre[e + 1] : total;
                }
                const uint32_t o = q - base;
                const bool sat = (x.lenf & kRSat) != 0;
                t1[k] = sat ? 0u : x.t0 + o + 1u;
                wb[k] = ((x.lenf & kRWrite) ? kOwnerWritten : 0u) | (sat ? kOwnerMulti : 0u);
                ri[k] = x.l0 + x.step * (int32_t)o;
            }
        }
        if (plain) {
            uint32_t old[4];
#pragma unroll
            for (int k = 0; k < 4; k++) old[k] = ri[k] >= 0 ? rec[ri[k]] : 0u;
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (ri[k] >= 0) rec[ri[k]] = t1[k] ? owner_merge(old[k], t1[k], wb[k]) : old[k] | wb[k];
        } else {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (ri[k] < 0) continue;
                uint32_t *const r = rec + ri[k];
                if (!t1[k]) { atomicOr(r, wb[k]); continue; }
                const uint32_t c = atomicCAS(r, 0u, t1[k] | wb[k]);
                if (c == 0u) continue;
                if (const uint32_t need = owner_need(c, t1[k] - 1u, wb[k] >> 31)) atomicOr(r, need);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) sh.n = 0;
}

__global__ void __launch_bounds__(kRangeThreads, kRangeBlocksPerSm) k_range(BatchArgs a)
{
    pdl_begin();
    extern __shared__ uint4 r_dyn[];
    uint32_t *const rec = reinterpret_cast<uint32_t *>(r_dyn);
    uint4 *const r4 = r_dyn;
    __shared__ RangeShared sh;
    if (threadIdx.x == 0) { sh.n = 0; sh.updates = 0; }
    // the shared records are zero at the start of every task: cleared here
    // once, then by the pass that ends each task
    for (uint32_t i = threadIdx.x; i < kRangeRecs / 4; i += kRangeThreads) r4[i] = make_uint4(0u, 0u, 0u, 0u);
    uint32_t *const tab = reinterpret_cast<uint32_t *>(a.table);
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // tasks come from a launch-wide counter in rtask's order (most work
    // first); thread 0 fetches the next task and reads its record while the
    // block works on this one
    __shared__ RTask s_task[2];
    const RTask none{~0u, 0u, 0u, 0u};
    auto task_at = [&a, &none](uint32_t i) {
        if (i >= a.nrtask) return none;
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(a.rtask) + i);
        return RTask{v.x, v.y, v.z, v.w};
    };
    uint32_t nx = 0;                                      // thread 0: the index of the task after this one
    if (threadIdx.x == 0) {
        s_task[0] = task_at(atomicAdd(&a.ctrl->range_next, 1u));
        nx = atomicAdd(&a.ctrl->range_next, 1u);
    }
    __syncthreads();
    for (uint32_t it = 0;; it++) {
        const RTask tk = s_task[it & 1u];
        if (tk.task == ~0u) break;
        // thread 0: the next task's record (stored in the other slot before
        // this task's last barrier; this slot is rewritten only in the next
        // task, after every thread has read it)
        RTask nt = none;
        if (threadIdx.x == 0) {
            nt = task_at(nx);
            if (nx < a.nrtask) nx = atomicAdd(&a.ctrl->range_next, 1u);
        }
        const unsigned long long r0 = (unsigned long long)tk.task * kRangeRecs;
        const unsigned long long r1 = r0 + kRangeRecs < a.tab_cells ? r0 + kRangeRecs : a.tab_cells;
        const uint32_t nrec = (uint32_t)(r1 - r0);
        // this entry's part of the task (blocks [blo, bhi) of 256 records),
        // and within it the window this launch may record (a shard)
        const uint32_t blo = tk.win & 0xFFFFu, bhi = tk.win >> 16;
        const uint32_t rlo = blo * 256u, rhi = bhi * 256u < nrec ? bhi * 256u : nrec;
        const unsigned long long w0 = r0 + rlo > a.shard_lo ? r0 + rlo : a.shard_lo;
        const unsigned long long w1 = r0 + rhi < a.shard_hi ? r0 + rhi : a.shard_hi;
        __syncthreads();                                  // the previous task is done with rec and sh
        // the blocks of 256 records the table pass touched in the part:
        // merged into the shared copy and cleared in the table (through L2:
        // this SM's L1 may hold lines the table pass read), one warp per
        // block; their touch bits cleared (atomically: another part of the
        // task may clear other bits of the same word at the same time)
        const uint32_t nwords = (nrec + 8191u) >> 13;
        uint32_t tb = 0;
        if (threadIdx.x < nwords) {
            const uint32_t b0 = threadIdx.x * 32u;            // the word's first block in the task
            const uint32_t lo = blo > b0 ? blo - b0 : 0u, hi = bhi < b0 + 32u ? (bhi > b0 ? bhi - b0 : 0u) : 32u;
            const uint32_t mask = lo < hi ? (hi - lo == 32u ? ~0u : ((1u << (hi - lo)) - 1u) << lo) : 0u;
            tb = mask ? __ldcg(a.touch + (r0 >> 13) + threadIdx.x) & mask : 0u;
            sh.bits[threadIdx.x] = tb;
            if (tb) atomicAnd(a.touch + (r0 >> 13) + threadIdx.x, ~tb);
        }
        if (__syncthreads_or(tb != 0u)) {
            const uint32_t nblk = (rhi + 255u) >> 8;
            for (uint32_t b = blo + warp; b < nblk; b += kRangeThreads / 32) {
                if (!((sh.bits[b >> 5] >> (b & 31u)) & 1u)) continue;
                for (uint32_t i = b * 256u + lane * 4u; i < b * 256u + 256u && i < nrec; i += 128u) {
                    if (i + 4u <= nrec) {                 // 16-byte aligned: r0 and i are multiples of 4
                        uint4 *g = reinterpret_cast<uint4 *>(tab + r0 + i);
                        const uint4 v = __ldcg(g);
                        if (v.x | v.y | v.z | v.w) { r4[i >> 2] = v; *g = make_uint4(0u, 0u, 0u, 0u); }
                    } else {
                        for (uint32_t j = i; j < nrec; j++) {
                            const uint32_t v = __ldcg(tab + r0 + j);
                            if (v) { rec[j] = v; tab[r0 + j] = 0u; }
                        }
                    }
                }
            }
            __syncthreads();
        }
        // the task's pieces, a round of up to kRangeChunk at a time; a part
        // of a task, or a shard, keeps what lies inside its window
        const bool whole = w0 == r0 && w1 == r1;
        for (uint32_t p0 = tk.p0; p0 < tk.p1 && w0 < w1; p0 += kRangeChunk) {
            const uint32_t np = tk.p1 - p0 < kRangeChunk ? tk.p1 - p0 : kRangeChunk;
            if (threadIdx.x < np) {
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(a.rpiece) + p0 + threadIdx.x);
                RPiece x{v.x, v.y, (int32_t)v.z, (int32_t)v.w};
                if (!whole) {
                    long long ct0, cl0, clen;
                    range_clip(x.t0, x.l0, x.lenf & kRLen, x.step, (long long)(w0 - r0), (long long)(w1 - r0), ct0,
                               cl0, clen);
                    x = RPiece{(uint32_t)ct0, (uint32_t)clen | (x.lenf & ~kRLen), (int32_t)cl0, x.step};
                }
                sh.ent[threadIdx.x] = x;
            }
            if (threadIdx.x == 0) sh.n = np;
            __syncthreads();
            range_apply(rec, sh);
        }
        // one pass over the task's records: the racy ones into a bitmap
        // (sh.pre, free after the last round), every record cleared for the
        // next task
        uint32_t *const racy = sh.pre;
        for (uint32_t i = threadIdx.x; i < kRangeRecs / 32; i += kRangeThreads) racy[i] = 0u;
        __syncthreads();
        bool found = false;
        for (uint32_t q = (rlo >> 2) + threadIdx.x; q < (rhi + 3u) >> 2; q += kRangeThreads) {
            const uint4 v = r4[q];
            if (v.x | v.y | v.z | v.w) {
                r4[q] = make_uint4(0u, 0u, 0u, 0u);
                const uint32_t m = (owner_racy(v.x) ? 1u : 0u) | (owner_racy(v.y) ? 2u : 0u) |
                                   (owner_racy(v.z) ? 4u : 0u) | (owner_racy(v.w) ? 8u : 0u);
                if (m) { atomicOr(&racy[q >> 3], m << ((q & 7u) * 4u)); found = true; }
            }
        }
        if (threadIdx.x == 0) s_task[(it + 1u) & 1u] = nt;
        // the first racy record of each protocol whose rows meet the task
        // (rows are phase-major, then array, then index: the lexicographic
        // order of the witness), by the first warp
        if (__syncthreads_or(found) && warp == 0) {
            uint32_t p = proto_of_record(a, r0 + rlo);
            while (true) {
                const DevProto P = a.protos[p];
                const unsigned long long pe = P.tab_off + (unsigned long long)P.tab_phases * P.cells_sum;
                const unsigned long long s0 = P.tab_off > r0 + rlo ? P.tab_off : r0 + rlo;
                const unsigned long long s1 = pe < r0 + rhi ? pe : r0 + rhi;
                if (s0 < s1) {
                    const uint32_t lo = (uint32_t)(s0 - r0), hi = (uint32_t)(s1 - r0);
                    for (uint32_t wb = (lo >> 5); wb <= ((hi - 1) >> 5); wb += 32) {
                        const uint32_t wd = wb + lane;
                        uint32_t bits = wd <= ((hi - 1) >> 5) ? racy[wd] : 0u;
                        if (wd == (lo >> 5)) bits &= ~0u << (lo & 31u);
                        if (wd == ((hi - 1) >> 5) && (hi & 31u)) bits &= (1u << (hi & 31u)) - 1u;
                        const unsigned any = __ballot_sync(kFull, bits != 0u);
                        if (any) {
                            const uint32_t src = (uint32_t)__ffs(any) - 1u;
                            const uint32_t first = __shfl_sync(kFull, bits, src);
                            if (lane == 0)
                                atomicMin(&a.best_pos[p], r0 + (wb + src) * 32u + (uint32_t)(__ffs(first) - 1));
                            break;
                        }
                    }
                }
                if (p + 1 >= a.nprotos || __ldg(&a.protos[p + 1].tab_off) >= r0 + rhi) break;
                p++;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && sh.updates) atomicAdd(&a.ctrl->range_tuples, sh.updates);
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.rcount) atomicAdd(&a.ctrl->total, a.rtotal);
}

// The sort path's keys of the range accesses (BatchArgs::range_keys): one
// per (piece as cut, thread), with their digit histograms, as the
// interpreted emit pass writes the other accesses' keys.  Block b writes the
// range keys [nrkeys * b / G, nrkeys * (b + 1) / G): its warp 0 finds the
// piece holding the first of them (a 32-way search of the pieces' key
// positions), then the block stages kREmitThreads pieces at a time in
// shared memory, and each thread writes every kREmitThreads-th key of the
// staged span, k0 + o * d, coalesced with its neighbours'.
constexpr int kREmitThreads = 512;

__global__ void __launch_bounds__(kREmitThreads) k_range_emit(BatchArgs a)
{
    pdl_begin();
    __shared__ EmitShared sh;
    __shared__ unsigned long long s_pre[kREmitThreads + 1], s_k0[kREmitThreads], s_d[kREmitThreads];
    __shared__ uint32_t s_e0;
    for (int i = threadIdx.x; i < kMaxPasses * kRadixBins; i += blockDim.x) (&sh.hist[0][0])[i] = 0;
    const KeyLayout L = a.L;
    const uint32_t t = threadIdx.x, lane = t & 31;
    const unsigned long long total = a.nrkeys, base = a.nkeys - a.nrkeys;
    const unsigned long long kb0 = total * blockIdx.x / gridDim.x, kb1 = total * (blockIdx.x + 1) / gridDim.x;
    const uint32_t n = a.nwkeys;
    if (t < 32) {
        // the last piece whose first key is at or before kb0 (pieces are
        // never empty, and wkeys[0].pre is 0)
        uint32_t lo = 0, hi = n;
        while (hi - lo > 1) {
            const uint32_t step = (hi - lo + 31) / 32, q = lo + lane * step;
            const bool le = q < hi && __ldg(&a.wkeys[q].pre) <= kb0;
            const unsigned m = __ballot_sync(kFull, le);
            const uint32_t last = 31u - (uint32_t)__clz(m);
            const uint32_t nlo = lo + last * step;
            hi = nlo + step < hi ? nlo + step : hi;
            lo = nlo;
        }
        if (t == 0) s_e0 = lo;
    }
    __syncthreads();
    uint32_t e0 = s_e0;
    unsigned long long k = kb0;
    while (k < kb1) {
        {
            const uint32_t e = e0 + t;
            if (e < n) {
                const RKeys w = a.wkeys[e];
                s_pre[t] = w.pre;
                s_k0[t] = w.k0;
                s_d[t] = w.d;
            } else {
                s_pre[t] = total;
                s_k0[t] = s_d[t] = 0;
            }
            if (t == 0) s_pre[kREmitThreads] = e0 + kREmitThreads < n ? __ldg(&a.wkeys[e0 + kREmitThreads].pre) : total;
        }
        __syncthreads();
        const unsigned long long kend = s_pre[kREmitThreads] < kb1 ? s_pre[kREmitThreads] : kb1;
        uint32_t j = 0;                                    // this thread's staged piece
        for (unsigned long long k1 = k; k1 < kend; k1 += kREmitThreads) {
            const unsigned long long kk = k1 + t;
            const bool ok = kk < kend;
            unsigned long long key = 0;
            if (ok) {
                if (s_pre[j + 1] <= kk) {
                    // past the piece: the last staged piece starting at or before kk
                    uint32_t lo = j + 1, hi = kREmitThreads;
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi + 1) / 2;
                        if (s_pre[mid] <= kk) lo = mid; else hi = mid - 1;
                    }
                    j = lo;
                }
                key = s_k0[j] + (kk - s_pre[j]) * s_d[j];
                const unsigned long long pos = base + kk;
                if (pos < a.nkeys) a.keys[0][pos] = key;
                else atomicOr(&a.ctrl->flags, CF_EMIT_OVERFLOW);
            }
            hist_add(&sh, L, key, ok);
        }
        k = kend;
        e0 += kREmitThreads;
        __syncthreads();
    }
    for (int i = threadIdx.x; i < (int)(L.passes * kRadixBins); i += blockDim.x) {
        const unsigned int h = (&sh.hist[0][0])[i];
        if (h) atomicAdd(&a.hist[i], (unsigned long long)h);
    }
    // the launch's key total counts these keys too (the count pass did not)
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&a.ctrl->total, a.nrkeys);
}

__device__ __forceinline__ void two_smallest(uint32_t &f, uint32_t &s, uint32_t x)
{
    if (x == f || x == s) return;
    if (x < f) { s = f; f = x; }
    else if (x < s) s = x;
}

// One block per protocol: evaluation error, else barrier divergence, else the
// witness of the first racy cell.  Sorted keys (TABLE false): the witness
// segment is found by binary search for its end, and the block reduces its
// accesses.  Owner table (TABLE true): the cell is decoded from its table
// position, and the block reduces the per-thread hit bits of the M_CELL
// pass.  Either way the result is the two smallest distinct tids of all
// accesses to the cell and of its writes.  THREADS per block: on sorted keys
// a batch of a few protocols gets wide blocks (a race's segment can hold
// tens of thousands of keys).
template <bool TABLE, int THREADS = kFinalizeThreads>
__global__ void __launch_bounds__(THREADS) k_finalize(BatchArgs a)
{
    constexpr int kFinalizeThreads = THREADS;
    pdl_begin();
    __shared__ uint32_t s_red[4][kFinalizeThreads / 32];
    __shared__ unsigned long long s_end;
    const uint32_t p = blockIdx.x;
    const uint32_t t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int parity = TABLE ? 0 : sorted_parity(a);
    if (p == 0 && t == 0 && a.nkeys != kUncounted && a.ctrl->total != a.nkeys)
        atomicOr(&a.ctrl->flags, CF_COUNT_MISMATCH);
    const DevProto P = a.protos[p];
    const KeyLayout L = a.L;
    DevResult r = {};
    r.verdict = -1;
    // the reductions of earlier kernels of this launch, read through L2
    r.tuples = __ldcg(a.ptuples + p);
    const unsigned long long ek = __ldcg(a.err_key + p);
    const unsigned long long bp = __ldcg(a.best_pos + p);
    const uint32_t dt = __ldcg(a.div_tid + p);
    if (ek == kNone && P.nthreads && dt == 0xFFFFFFFFu && bp != kNone) {
        uint32_t t0 = 0xFFFFFFFFu, t1 = 0xFFFFFFFFu, w0 = 0xFFFFFFFFu, w1 = 0xFFFFFFFFu;
        unsigned long long seg = 0;
        if (TABLE) {
            // this protocol's bits: [tid_off, tid_off + T) of the hit arrays
            const uint64_t b0 = P.tid_off, b1 = P.tid_off + P.nthreads;
#pragma unroll 4
            for (uint64_t wd = (b0 >> 5) + t; wd <= ((b1 - 1) >> 5); wd += kFinalizeThreads) {
                uint32_t ma = __ldcg(a.hit_acc + wd), mw = __ldcg(a.hit_wr + wd);
                const uint64_t lo = wd * 32;
                if (lo < b0) { ma &= ~0u << (uint32_t)(b0 - lo); mw &= ~0u << (uint32_t)(b0 - lo); }
                if (lo + 32 > b1) {
                    const uint32_t keep = (1u << (uint32_t)(b1 - lo)) - 1;
                    ma &= keep; mw &= keep;
                }
                for (int q = 0; q < 2 && ma; q++) {
                    two_smallest(t0, t1, (uint32_t)(lo + (uint32_t)(__ffs(ma) - 1) - b0));
                    ma &= ma - 1;
                }
                for (int q = 0; q < 2 && mw; q++) {
                    two_smallest(w0, w1, (uint32_t)(lo + (uint32_t)(__ffs(mw) - 1) - b0));
                    mw &= mw - 1;
                }
            }
            if (a.range_on) {
                // the accesses the range pass applied are not in the hit bits
                // (the interpreted witness pass skips them): the threads of
                // the pieces of the racy record's task that land on it
                const unsigned long long task = bp / kRangeRecs;
                // the task's index in rlive (ascending), in two rounds of loads:
                // the slice of rlive (one per thread) that can hold it, then
                // its entries side by side
                __shared__ uint32_t s_slice, s_li;
                if (t == 0) { s_slice = 0; s_li = 0xFFFFFFFFu; }
                __syncthreads();
                const uint32_t per = (a.nlive + kFinalizeThreads - 1) / kFinalizeThreads;
                if (t * per < a.nlive && __ldg(a.rlive + t * per) <= task) atomicMax(&s_slice, t);
                __syncthreads();
                for (uint32_t q = s_slice * per + t; q < s_slice * per + per && q < a.nlive; q += kFinalizeThreads)
                    if (__ldg(a.rlive + q) == task) s_li = q;
                __syncthreads();
                const uint32_t lo = s_li;
                if (lo != 0xFFFFFFFFu) {
                    const long long x = (long long)(bp - task * kRangeRecs);
                    const uint32_t e1 = __ldg(a.rfirst + lo + 1);
                    for (uint32_t e = __ldg(a.rfirst + lo) + t; e < e1; e += kFinalizeThreads) {
                        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(a.wpiece) + e);
                        const long long d = x - (long long)(int32_t)v.z, st = (long long)(int32_t)v.w;
                        const long long len = (long long)(v.y & kRLen);
                        if (st == 0) {
                            // every thread of the piece at l0: its two smallest
                            if (d != 0 || len == 0) continue;
                            for (uint32_t q = 0; q < 2 && q < len; q++) {
                                two_smallest(t0, t1, v.x + q);
                                if (v.y & kRWrite) two_smallest(w0, w1, v.x + q);
                            }
                            continue;
                        }
                        // x = l0 + step * o for some o < len
                        if (d % st != 0) continue;
                        const long long o = d / st;
                        if (o < 0 || o >= len) continue;
                        const uint32_t tid = v.x + (uint32_t)o;          // the piece's thread at the record
                        two_smallest(t0, t1, tid);
                        if (v.y & kRWrite) two_smallest(w0, w1, tid);
                    }
                }
            }
        } else {
            const unsigned long long *keys = a.keys[parity];
            const uint32_t tid_mask = L.tid_bits ? (1u << L.tid_bits) - 1 : 0;
            seg = keys[bp] >> L.sort_lo;
            if (t == 0) {               // first position after the segment
                unsigned long long lo = bp + 1, hi = a.nkeys;
                while (lo < hi) {
                    unsigned long long mid = lo + (hi - lo) / 2;
                    if ((keys[mid] >> L.sort_lo) == seg) lo = mid + 1; else hi = mid;
                }
                s_end = lo;
            }
            __syncthreads();
            const unsigned long long end = s_end;
            for (unsigned long long j = bp + t; j < end; j += kFinalizeThreads) {
                unsigned long long x = keys[j];
                uint32_t tid = (uint32_t)(x >> 1) & tid_mask;
                two_smallest(t0, t1, tid);
                if (x & 1) two_smallest(w0, w1, tid);
            }
        }
        for (int o = 16; o; o >>= 1) {
            uint32_t u0 = __shfl_xor_sync(kFull, t0, o), u1 = __shfl_xor_sync(kFull, t1, o);
            uint32_t v0 = __shfl_xor_sync(kFull, w0, o), v1 = __shfl_xor_sync(kFull, w1, o);
            two_smallest(t0, t1, u0); two_smallest(t0, t1, u1);
            two_smallest(w0, w1, v0); two_smallest(w0, w1, v1);
        }
        if (lane == 0) { s_red[0][wid] = t0; s_red[1][wid] = t1; s_red[2][wid] = w0; s_red[3][wid] = w1; }
        __syncthreads();
        if (t == 0) {
            for (int w = 1; w < kFinalizeThreads / 32; w++) {
                two_smallest(t0, t1, s_red[0][w]); two_smallest(t0, t1, s_red[1][w]);
                two_smallest(w0, w1, s_red[2][w]); two_smallest(w0, w1, s_red[3][w]);
            }
            r.verdict = 1;
            r.phases = __ldcg(a.totsyn + P.tid_off) + 1;
            r.sync_count_0 = __ldcg(a.totsyn + P.tid_off);
            if (TABLE) {
                const CellTarget c = decode_cell(a, P, bp);
                r.phase = c.phase;
                r.loc = c.loc;
                r.index = c.idx;
            } else {
                r.index = seg & (L.idx_bits ? (~0ull >> (64 - L.idx_bits)) : 0);
                r.loc = (uint32_t)((seg >> L.idx_bits) & (L.loc_bits ? (~0ull >> (64 - L.loc_bits)) : 0));
                r.phase = (uint32_t)((seg >> (L.idx_bits + L.loc_bits)) &
                                     (L.phase_bits ? (~0ull >> (64 - L.phase_bits)) : 0));
            }
            r.tid_i = t0;
            if (w0 == t0) { r.tid_j = t1; r.i_writes = 1; r.j_writes = (w1 == t1); }
            else { r.tid_j = w0; r.i_writes = 0; r.j_writes = 1; }
            a.results[p] = r;
        }
        return;
    }
    if (t != 0) return;
    if (ek != kNone) {
        uint32_t tid = (uint32_t)(ek >> 32), k = (uint32_t)ek;
        unsigned long long e = a.erro[P.lane_off + (uint64_t)k * P.nthreads + tid];
        unsigned long long pre = 0;
        for (uint32_t q = 0; q < k; q++) pre += a.cnt[P.lane_off + (uint64_t)q * P.nthreads + tid];
        r.status = (e & 0xff) == kErrOob ? -9 : -10;
        r.err_tid = tid;
        r.err_ordinal = pre + (e >> 8);
    } else if (P.nthreads == 0) {
        r.verdict = 0;
        r.phases = 0;
    } else {
        const uint32_t s0 = __ldcg(a.totsyn + P.tid_off);
        r.phases = s0 + 1;
        r.sync_count_0 = s0;
        if (dt != 0xFFFFFFFFu) {
            r.verdict = 2;
            r.div_tid = dt;
            r.sync_count_div = __ldcg(a.totsyn + P.tid_off + dt);
        } else {
            r.verdict = 0;
        }
    }
    a.results[p] = r;
}

}  // namespace

// ---------------------------------------------------------------- launchers

static int interp_grid(uint32_t nwitems, int sms)
{
    uint32_t g = (nwitems + 7) / 8;
    uint32_t cap = (uint32_t)sms * 8;
    return (int)(g < cap ? (g ? g : 1) : cap);
}

static void mark(cudaEvent_t *ev, int *nev, cudaStream_t s)
{
    if (!ev || !nev) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    // inside a graph capture only an external record becomes a timing node
    if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(ev[(*nev)++], s, cudaEventRecordExternal);
    else cudaEventRecord(ev[(*nev)++], s);
}

// Launch configuration with programmatic stream serialization (pdl_begin).
struct PdlConfig {
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    PdlConfig(dim3 grid, dim3 block, cudaStream_t s)
    {
        cfg.gridDim = grid;
        cfg.blockDim = block;
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
};

template <typename... P>
static void launch_pdl(void (*k)(BatchArgs, P...), dim3 grid, dim3 block, cudaStream_t s, const BatchArgs &a, P... p)
{
    PdlConfig c(grid, block, s);
    cudaLaunchKernelEx(&c.cfg, k, a, p...);
}

// One launch of a specialized kernel (a cudaKernel_t) over the warp-items,
// with programmatic stream serialization (the generated kernels begin as
// pdl_begin does).
static void launch_jit(const void *k, const BatchArgs &a, const JitLaunch *j, cudaStream_t s, int sms)
{
    BatchArgs args = a;
    const uint16_t *shape = j->shape;
    void *params[] = {&args, &shape};
    PdlConfig c(dim3((unsigned)interp_grid(a.nwitems, sms)), dim3(256), s);
    cudaLaunchKernelExC(&c.cfg, k, params);
}

// The range pass: kRangeBlocksPerSm blocks per SM, each holding one task's
// records in dynamic shared memory (the kernel's attributes set once per
// device: that much dynamic shared memory, and all of the SM's unified L1 /
// shared memory as shared memory so that the blocks fit).
static void launch_range(const BatchArgs &a, cudaStream_t s, int sms)
{
    static bool ready[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !ready[dev]) {
        cudaFuncSetAttribute((const void *)k_range, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRangeSmem);
        cudaFuncSetAttribute((const void *)k_range, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        ready[dev] = true;
    }
    const uint32_t want = (uint32_t)sms * kRangeBlocksPerSm;
    PdlConfig c(dim3(a.nrtask < want ? (a.nrtask ? a.nrtask : 1) : want), dim3(kRangeThreads), s);
    c.cfg.dynamicSmemBytes = kRangeSmem;
    cudaLaunchKernelEx(&c.cfg, k_range, a);
}

// The interpreter, and specialized kernels without a compiled-in schedule,
// read the batch's warp-item array: a batch loaded without it cannot run them.
static bool schedule_missing(const BatchArgs &a, const JitLaunch *j)
{
    return a.nwitems && !a.witems && !(j && j->csched);
}

// The launch's arguments with rcount set when the table pass counts the
// tuples (an interpreted launch without count pass, or specialized kernels
// with static phases that leave the range accesses to the range pass) and
// the range pass runs: the range accesses' tuples then come from the host.
static BatchArgs with_rcount(const BatchArgs &a, const JitLaunch *j)
{
    BatchArgs b = a;
    const bool jit_counts = j && j->table && j->static_phases;
    b.rcount = (a.range_on && a.path == PATH_TABLE && a.rtup && (jit_counts ? j->range : a.count_free != 0)) ||
                       (a.range_keys && a.rtup)
                   ? 1u
                   : 0u;
    return b;
}

cudaError_t launch_front(const BatchArgs &a0, cudaStream_t s, int sms, cudaEvent_t *ev, int *nev, const JitLaunch *j)
{
    const BatchArgs a = with_rcount(a0, j);
    if (schedule_missing(a, j)) return cudaErrorInvalidValue;
    uint64_t init_n = a.nprotos;
    if (init_n < (uint64_t)kMaxPasses * kRadixBins) init_n = (uint64_t)kMaxPasses * kRadixBins;
    if (init_n < a.nwblocks) init_n = a.nwblocks;
    mark(ev, nev, s);
    k_init<<<(unsigned)((init_n + 255) / 256), 256, 0, s>>>(a);
    mark(ev, nev, s);
    // nothing to count or scan: specialized kernels with the phases compiled
    // in, or interpreted owner-table launches of a batch with static phases
    if ((j && j->static_phases) || (a.count_free && a.path == PATH_TABLE)) return cudaGetLastError();
    if (j && j->count) {
        launch_jit(j->count, a, j, s, sms);
    } else {
        if (a.has_narrow) launch_pdl(k_interp<M_COUNT, false>, dim3(interp_grid(a.nwitems, sms)), dim3(256), s, a);
        if (a.has_wide) launch_pdl(k_interp<M_COUNT, true>, dim3(interp_grid(a.nwitems, sms)), dim3(256), s, a);
    }
    mark(ev, nev, s);
    uint32_t col_blocks = (uint32_t)((a.ncols + 31) / 32);
    launch_pdl(k_scan, dim3(col_blocks + a.nwblocks), dim3(kScanThreads), s, a, col_blocks);
    mark(ev, nev, s);
    return cudaGetLastError();
}

template <int MODE>
static void launch_interp(const BatchArgs &a, cudaStream_t s, int sms)
{
    if (a.has_narrow) k_interp<MODE, false><<<interp_grid(a.nwitems, sms), 256, 0, s>>>(a);
    if (a.has_wide) k_interp<MODE, true><<<interp_grid(a.nwitems, sms), 256, 0, s>>>(a);
}

template <int MODE>
static void launch_interp_pdl(const BatchArgs &a, cudaStream_t s, int sms)
{
    if (a.has_narrow) launch_pdl(k_interp<MODE, false>, dim3(interp_grid(a.nwitems, sms)), dim3(256), s, a);
    if (a.has_wide) launch_pdl(k_interp<MODE, true>, dim3(interp_grid(a.nwitems, sms)), dim3(256), s, a);
}

static cudaError_t launch_back_table(const BatchArgs &a0, cudaStream_t s, int sms, cudaEvent_t *ev, int *nev,
                                     const JitLaunch *j)
{
    const BatchArgs a = with_rcount(a0, j);
    if (j && j->table && j->range && !a.range_on) return cudaErrorInvalidValue;   // its range accesses would be lost
    if (j && j->table) launch_jit(j->table, a, j, s, sms);
    else launch_interp_pdl<M_TABLE>(a, s, sms);
    mark(ev, nev, s);
    if (a.range_on) {
        launch_range(a, s, sms);
        mark(ev, nev, s);
    }
    const uint64_t cap = (uint64_t)sms * 8;
    uint64_t lgrid = (touch_words(a.tab_cells) + kTabScanThreads - 1) / kTabScanThreads;
    if (lgrid > cap) lgrid = cap;
    if (lgrid == 0) lgrid = 1;
    launch_pdl(k_tlist, dim3((unsigned)lgrid), dim3(kTabScanThreads), s, a);
    uint64_t grid = (table_blocks(a.tab_cells) + kTabScanThreads / 32 - 1) / (kTabScanThreads / 32);
    if (grid > cap) grid = cap;
    if (grid == 0) grid = 1;
    launch_pdl(k_tscan, dim3((unsigned)grid), dim3(kTabScanThreads), s, a);
    mark(ev, nev, s);
    if (j && j->cell) launch_jit(j->cell, a, j, s, sms);
    else launch_interp_pdl<M_CELL>(a, s, sms);
    mark(ev, nev, s);
    // specialized kernels with static phases and no range pass write the
    // result from the witness pass's last block
    if (!(j && j->cell && j->static_phases && !j->range)) {
        // a few protocols: wide blocks, so that each protocol's hit words
        // and witness search take few rounds of loads
        if (a.nprotos <= kFinalizeWideProtos)
            launch_pdl(k_finalize<true, kFinalizeWideThreads>, dim3(a.nprotos), dim3(kFinalizeWideThreads), s, a);
        else
            launch_pdl(k_finalize<true>, dim3(a.nprotos), dim3(kFinalizeThreads), s, a);
        mark(ev, nev, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_back(const BatchArgs &a, cudaStream_t s, int sms, cudaEvent_t *ev, int *nev, const JitLaunch *j)
{
    if (schedule_missing(a, j)) return cudaErrorInvalidValue;
    if (a.path == PATH_TABLE) return launch_back_table(a, s, sms, ev, nev, j);
    launch_interp<M_EMIT>(a, s, sms);
    if (a.range_keys) {
        // the range accesses' keys, from the pieces
        // blocks of at least 8 keys per thread, up to 4 per SM
        const unsigned long long need = (a.nrkeys + 8 * kREmitThreads - 1) / (8 * kREmitThreads);
        const uint32_t want = (uint32_t)sms * 4;
        k_range_emit<<<need < want ? (uint32_t)(need ? need : 1) : want, kREmitThreads, 0, s>>>(a);
    }
    mark(ev, nev, s);
    for (uint32_t q = 0; q < a.L.passes; q++) {
        if (a.ntiles) {
            const uint32_t items = radix_items_or_default(a.radix_items);
            if (items == 12) k_radix<12><<<a.ntiles, kRadixThreads, 0, s>>>(a, q);
            else if (items == 24) k_radix<24><<<a.ntiles, kRadixThreads, 0, s>>>(a, q);
            else k_radix<16><<<a.ntiles, kRadixThreads, 0, s>>>(a, q);
        }
        mark(ev, nev, s);
    }
    if (a.ndtiles) {
        k_detect<<<a.ndtiles, kDetectThreads, 0, s>>>(a);
        k_resolve<<<1, 1024, 0, s>>>(a);
    }
    mark(ev, nev, s);
    if (a.nprotos <= kFinalizeWideProtos)
        k_finalize<false, kFinalizeWideThreads><<<a.nprotos, kFinalizeWideThreads, 0, s>>>(a);
    else
        k_finalize<false><<<a.nprotos, kFinalizeThreads, 0, s>>>(a);
    mark(ev, nev, s);
    return cudaGetLastError();
}

int stage_names(const char **names, int cap, uint32_t passes, uint32_t path, bool static_phases, bool count_free,
                bool range)
{
    static const char *radix[kMaxPasses] = {"radix0", "radix1", "radix2", "radix3",
                                            "radix4", "radix5", "radix6", "radix7"};
    const char *all[kMaxStages];
    int n = 0;
    all[n++] = "init";
    if (!static_phases && !(count_free && path == PATH_TABLE)) { all[n++] = "count"; all[n++] = "scan"; }
    if (path == PATH_TABLE) {
        all[n++] = "table";
        if (range) all[n++] = "range";
        all[n++] = "tscan";
        all[n++] = static_phases && !range ? "witness+finalize" : "witness";
    } else {
        all[n++] = "emit";
        for (uint32_t q = 0; q < passes && q < (uint32_t)kMaxPasses; q++) all[n++] = radix[q];
        all[n++] = "detect";
    }
    if (!(static_phases && path == PATH_TABLE && !range)) all[n++] = "finalize";
    for (int i = 0; i < n && i < cap; i++) names[i] = all[i];
    return n;
}

}  // namespace drf
