// Batch packing, device buffers and the two-phase pipeline run.
#include "engine.h"

#include <algorithm>
#include <atomic>
#include <cstring>
#include <numeric>

namespace drf {

bool ensure(DevBuf &b, size_t bytes, size_t *in_use, uint64_t limit)
{
    if (b.cap >= bytes) return true;
    size_t want = std::max(bytes, b.cap + b.cap / 4);       // grow by at least 25%
    if (limit && *in_use - b.cap + want > limit) want = bytes;
    if (limit && *in_use - b.cap + want > limit) return false;
    release(b, in_use);
    if (cudaMalloc(&b.p, want) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return false;
    }
    b.cap = want;
    b.gen++;
    *in_use += want;
    return true;
}

void release(DevBuf &b, size_t *in_use)
{
    if (b.p) {
        cudaFree(b.p);
        *in_use -= b.cap;
        b.gen++;
    }
    b.p = nullptr;
    b.cap = 0;
}

void BatchHost::renew()
{
    static std::atomic<uint64_t> counter{0};
    version = ++counter;
}

void BatchHost::expand_witems()
{
    if (expanded()) return;
    renew();
    witems.resize(nwitems);
    WarpItem *wi = witems.data();
    for (const Run &r : runs)
        for (uint32_t g = 0; g < r.groups; g++) *wi++ = WarpItem{r.proto, r.k, g};
}

Error pack_batch(const std::vector<const Prepared *> &ps, BatchHost &out, bool expand, uint32_t digit_bits,
                 uint64_t range_min)
{
    // cleared, not reassigned: a reused image keeps its vectors' capacity
    out.insns.clear();
    out.xcode.clear();
    out.items.clear();
    out.protos.clear();
    out.cells.clear();
    out.cbase.clear();
    out.witems.clear();
    out.iphase.clear();
    out.runs.clear();
    out.nwitems = 0;
    out.ncols = out.lanes = out.tuple_bound = out.table_cells = 0;
    out.L = KeyLayout{};
    out.table_ok = false;
    out.all_static = !ps.empty();
    KeyLayout L{};
    const uint32_t n = (uint32_t)ps.size();
    L.proto_bits = n > 1 ? bits_for(n - 1) : 0;
    for (const Prepared *p : ps) {
        L.phase_bits = std::max(L.phase_bits, bits_for(p->max_syncs));
        L.loc_bits = std::max(L.loc_bits, bits_for(p->narrays ? p->narrays - 1 : 0));
        for (uint64_t c : p->cells) L.idx_bits = std::max(L.idx_bits, bits_for(c ? c - 1 : 0));
        L.tid_bits = std::max(L.tid_bits, bits_for(p->nthreads ? p->nthreads - 1 : 0));
    }
    L.sort_lo = L.tid_bits + 1;
    L.sort_bits = L.proto_bits + L.phase_bits + L.loc_bits + L.idx_bits;
    if (L.sort_lo + L.sort_bits > 64)
        return Error::make(S_KEY_TOO_WIDE, "phase, array, index and thread fields need " +
                                               std::to_string(L.sort_lo + L.sort_bits) + " bits");
    // the digit width asked for (4..8), widened when the sort key would need
    // more than kMaxPasses passes of it
    L.digit_bits = std::min<uint32_t>(kRadixBits, std::max<uint32_t>(4, digit_bits ? digit_bits : kRadixBits));
    if ((L.sort_bits + L.digit_bits - 1) / L.digit_bits > (uint32_t)kMaxPasses)
        L.digit_bits = (L.sort_bits + kMaxPasses - 1) / kMaxPasses;
    L.passes = L.sort_bits ? (L.sort_bits + L.digit_bits - 1) / L.digit_bits : 0;
    out.L = L;

    // one entry per (protocol, item); its thread groups follow it in order
    struct W { uint32_t proto, k, groups; uint64_t steps; };
    std::vector<W> ws;
    uint64_t nwitems = 0;
    bool table_fits = true;
    for (uint32_t i = 0; i < n; i++) {
        const Prepared &p = *ps[i];
        DevProto d{};
        d.insn_off = (uint32_t)out.insns.size();
        d.xcode_off = (uint32_t)out.xcode.size();
        d.item_off = (uint32_t)out.items.size();
        d.nitems = (uint32_t)p.items.size();
        d.nthreads = p.nthreads;
        d.wide = p.wide ? 1 : 0;
        d.nlocs = p.narrays;
        d.cells_off = (uint32_t)out.cells.size();
        d.lane_off = out.lanes;
        d.tid_off = out.ncols;
        // owner-table rows: one per phase the static sync bound allows
        uint64_t row = 0;
        for (uint64_t c : p.cells) {
            out.cbase.push_back(row);
            row = row + c < row ? ~0ull : row + c;
        }
        d.tab_off = out.table_cells;
        d.cells_sum = row;
        d.tab_phases = p.max_syncs < 0xFFFFFFFFull ? (uint32_t)(p.max_syncs + 1) : 0;
        const bool stat = p.static_phases && p.item_phase.size() == p.items.size() && d.tab_phases;
        d.flags = stat ? DP_STATIC : 0;
        out.all_static = out.all_static && stat;
        for (size_t k = 0; k < p.items.size(); k++) out.iphase.push_back(stat ? p.item_phase[k] : 0u);
        if (!d.tab_phases || (row && (unsigned __int128)row * d.tab_phases > kMaxTableBytes)) table_fits = false;
        else out.table_cells += row * d.tab_phases;
        if (out.table_cells > kMaxTableBytes) table_fits = false;
        out.insns.insert(out.insns.end(), p.insns.begin(), p.insns.end());
        out.xcode.insert(out.xcode.end(), p.xcode.begin(), p.xcode.end());
        out.items.insert(out.items.end(), p.items.begin(), p.items.end());
        out.cells.insert(out.cells.end(), p.cells.begin(), p.cells.end());
        out.protos.push_back(d);
        out.lanes += (uint64_t)d.nitems * p.nthreads;
        out.ncols += p.nthreads;
        out.tuple_bound += p.tuple_bound();
        uint32_t groups = (p.nthreads + 31) / 32;
        for (uint32_t k = 0; k < d.nitems; k++) ws.push_back(W{i, k, groups, p.item_steps[k]});
        nwitems += (uint64_t)d.nitems * groups;
    }
    if (out.insns.size() >= (1ull << 31) || out.xcode.size() >= (1ull << 31) || out.items.size() >= (1ull << 31) ||
        nwitems >= (1ull << 31) || out.lanes >= (1ull << 31))
        return Error::make(S_LIMIT, "batch too large");
    out.table_ok = table_fits && out.table_bytes() <= kMaxTableBytes;
    if (!out.table_ok) out.table_cells = 0;
    // longest items first, so that the grid-stride loops end together (a
    // stable order: equal items keep protocol and item order, and the
    // groups of one item stay consecutive)
    std::stable_sort(ws.begin(), ws.end(), [](const W &x, const W &y) { return x.steps > y.steps; });
    out.runs.reserve(ws.size());
    for (auto &w : ws) out.runs.push_back(BatchHost::Run{w.proto, w.k, w.groups});
    out.nwitems = nwitems;
    if (expand) out.expand_witems();
    plan_range(ps, out, range_min);                // (clears the previous pack's range work when none)
    out.renew();
    return Error{};
}


namespace {

// The threads of range access r at offset c (reduced mod the modulus when
// there is one) as runs of consecutive tids whose cells are sigma apart:
// (first tid, count, first tid's cell) -- one run without a remainder (or
// for sigma 0), else one per wrap of the index around the modulus (at most
// kRangeMaxWraps + 1).  Cells outside the array are clipped by the caller.
struct Run { int64_t t0, len, cell0; };

void range_runs(const RangeAccess &r, int64_t c, uint32_t T, std::vector<Run> &out)
{
    out.clear();
    const int64_t t = (int64_t)T, s = r.sigma;
    if (!r.modn || s == 0) {
        if (t > 0) out.push_back(Run{0, t, c});
        return;
    }
    // c in [0, N): the index sigma * tid + c lies in [q N, (q + 1) N) for one
    // q per run; the run ends where q changes
    const int64_t N = (int64_t)r.modn;
    for (int64_t a = 0; a < t;) {
        const int64_t v = s * a + c;
        const int64_t q = v >= 0 ? v / N : -((-v + N - 1) / N);
        int64_t b = s > 0 ? ((q + 1) * N - c + s - 1) / s : range_floordiv(c - q * N, -s) + 1;
        if (b > t) b = t;
        out.push_back(Run{a, b - a, v - q * N});
        a = b;
    }
}

// Whether protocol i of a packed batch takes the range pass: static phases
// and range accesses that make a quarter of its tuples or more.
bool range_candidate(const Prepared &p, const DevProto &d, unsigned __int128 &rt)
{
    rt = 0;
    if (!(d.flags & DP_STATIC) || p.range_access.empty()) return false;
    for (const RangeAccess &r : p.range_access) rt += (unsigned __int128)r.run_iters * p.nthreads;
    return rt * 4 >= (unsigned __int128)p.tuple_bound();
}

// One task's pieces as the range pass applies them.  Pieces of one step s
// whose records fall in one residue class mod |s| are compared record by
// record along that class: records that pieces of one base (record minus
// s times thread: the same thread at every record) reach keep that base's
// threads, in one piece however many accesses and offsets repeat them;
// records that two or more bases reach -- two different threads -- become
// kRSat pieces, which only set "second thread" (and "written" where some
// covering piece writes).  Pieces of different steps are left as they are;
// the kernel checks which pieces meet.
void merge_pieces(const RPiece *in, size_t n, std::vector<RPiece> &out)
{
    out.clear();
    // pieces of step 0 (every thread of the piece on one record): per
    // record, one thread stays a one-record piece, two or more saturate it
    struct Z { int32_t l0; uint32_t t0, t1; bool w; };     // threads [t0, t1)
    static thread_local std::vector<Z> zs;                  // (scratch kept between calls)
    zs.clear();
    for (size_t i = 0; i < n; i++)
        if (in[i].step == 0 && (in[i].lenf & kRLen))
            zs.push_back(Z{in[i].l0, in[i].t0, in[i].t0 + (in[i].lenf & kRLen), (in[i].lenf & kRWrite) != 0});
    std::sort(zs.begin(), zs.end(), [](const Z &x, const Z &y) { return x.l0 < y.l0; });
    for (size_t i = 0; i < zs.size();) {
        size_t j = i;
        bool w = false, many = false;
        for (; j < zs.size() && zs[j].l0 == zs[i].l0; j++) {
            w = w || zs[j].w;
            many = many || zs[j].t1 - zs[j].t0 > 1 || zs[j].t0 != zs[i].t0;
        }
        const uint32_t wf = w ? kRWrite : 0u;
        out.push_back(many ? RPiece{0u, 1u | kRSat | wf, zs[i].l0, 1} : RPiece{zs[i].t0, 1u | wf, zs[i].l0, 1});
        i = j;
    }
    struct P { int64_t s, a, r, base, u0, u1; bool w; };    // lattice coordinates u: record = r + a * u
    static thread_local std::vector<P> ps;
    ps.clear();
    for (size_t i = 0; i < n; i++) {
        const RPiece &x = in[i];
        const int64_t len = x.lenf & kRLen;
        if (!len || x.step == 0) continue;
        const int64_t s = x.step, a = s < 0 ? -s : s, l0 = x.l0;
        const int64_t r = ((l0 % a) + a) % a, ul = (l0 - r) / a;
        const int64_t u0 = s > 0 ? ul : ul - len + 1, u1 = s > 0 ? ul + len : ul + 1;
        ps.push_back(P{s, a, r, l0 - s * (int64_t)x.t0, u0, u1, (x.lenf & kRWrite) != 0});
    }
    std::sort(ps.begin(), ps.end(), [](const P &x, const P &y) {
        return x.s != y.s ? x.s < y.s : x.r != y.r ? x.r < y.r : x.u0 < y.u0;
    });
    struct Ev { int64_t u; int d; size_t k; };
    static thread_local std::vector<Ev> ev;
    // active pieces per base (count, writers): a few at a time, kept in a
    // short list
    struct Act { int64_t base; int cnt, wr; };
    static thread_local std::vector<Act> act;
    for (size_t g0 = 0; g0 < ps.size();) {
        size_t g1 = g0;
        while (g1 < ps.size() && ps[g1].s == ps[g0].s && ps[g1].r == ps[g0].r) g1++;
        const int64_t s = ps[g0].s, a = ps[g0].a, r = ps[g0].r;
        ev.clear();
        for (size_t k = g0; k < g1; k++) {
            ev.push_back(Ev{ps[k].u0, +1, k});
            ev.push_back(Ev{ps[k].u1, -1, k});
        }
        std::sort(ev.begin(), ev.end(), [](const Ev &x, const Ev &y) { return x.u < y.u; });
        act.clear();
        int writers = 0;
        // the output run being extended: kind 0 none, 1 one base, 2 saturated
        int kind = 0;
        int64_t run_u0 = 0, run_base = 0;
        bool run_w = false;
        auto close = [&](int64_t u_end) {
            if (kind == 0 || u_end <= run_u0) { kind = 0; return; }
            const int64_t len = u_end - run_u0;
            const uint32_t wf = run_w ? kRWrite : 0u;
            if (kind == 2) {
                out.push_back(RPiece{0u, (uint32_t)len | kRSat | wf, (int32_t)(r + a * run_u0), (int32_t)a});
            } else if (s > 0) {
                const int64_t l0 = r + a * run_u0;
                out.push_back(RPiece{(uint32_t)((l0 - run_base) / s), (uint32_t)len | wf, (int32_t)l0, (int32_t)s});
            } else {
                const int64_t l0 = r + a * (u_end - 1);           // threads ascend as records descend
                out.push_back(RPiece{(uint32_t)((l0 - run_base) / s), (uint32_t)len | wf, (int32_t)l0, (int32_t)s});
            }
            kind = 0;
        };
        for (size_t e = 0; e < ev.size();) {
            const int64_t u = ev[e].u;
            for (; e < ev.size() && ev[e].u == u; e++) {
                const P &p = ps[ev[e].k];
                size_t q = 0;
                while (q < act.size() && act[q].base != p.base) q++;
                if (q == act.size()) act.push_back(Act{p.base, 0, 0});
                act[q].cnt += ev[e].d;
                act[q].wr += p.w ? ev[e].d : 0;
                writers += p.w ? ev[e].d : 0;
                if (act[q].cnt == 0) { act[q] = act.back(); act.pop_back(); }
            }
            // the state from u on
            const int nk = act.empty() ? 0 : act.size() == 1 ? 1 : 2;
            const int64_t nb = nk == 1 ? act[0].base : 0;
            const bool nw = writers > 0;
            if (nk != kind || nw != run_w || (nk == 1 && nb != run_base)) {
                close(u);
                if (nk) { kind = nk; run_u0 = u; run_base = nb; run_w = nw; }
            }
        }
        close(ev.empty() ? 0 : ev.back().u);
        g0 = g1;
    }
}

// Sets (or, with set false, clears) LB_RANGE_ONLY on every loop of one
// protocol's program whose body holds no sync and only AF_RANGE accesses.
void mark_range_loops(Insn *in, size_t n, bool set)
{
    for (size_t pc = 0; pc < n; pc++) {
        if (in[pc].op != I_LOOP) continue;
        if (!set) { in[pc].b &= (uint16_t)~LB_RANGE_ONLY; continue; }
        const size_t e = (size_t)in[pc].e;
        bool only = e < n;
        for (size_t q = pc + 1; only && q <= e; q++) {
            const Insn &x = in[q];
            if (x.op == I_SYNC || x.op == I_END) only = false;
            else if ((x.op == I_ACCESS || x.op == I_FASTACC) && !(x.a & AF_RANGE)) only = false;
            else if (x.op == I_FASTLOOP && x.b != 0) only = false;
        }
        if (only) in[pc].b |= LB_RANGE_ONLY;
    }
}

void clear_range(BatchHost &out, size_t nprotos)
{
    out.rpiece.clear();
    out.wpiece.clear();
    out.rtask.clear();
    out.rlive.clear();
    out.rfirst.clear();
    out.range_pcs.assign(nprotos, {});
    out.range_tuples = 0;
    out.rtup.clear();
    out.wkeys.clear();
    out.nrkeys = 0;
}

}  // namespace

void plan_range(const std::vector<const Prepared *> &ps, BatchHost &out, uint64_t range_min)
{
    clear_range(out, ps.size());
    if (!out.table_ok) return;                     // the pieces are laid out in the owner table's records
    // a batch whose range accesses make few tuples runs faster without the
    // pass (its planning, upload and kernel would cost more than it saves)
    unsigned __int128 all = 0, rt = 0;
    for (size_t i = 0; i < ps.size(); i++)
        if (range_candidate(*ps[i], out.protos[i], rt)) all += rt;
    if (all == 0 || all < range_min) return;
    // each piece as cut, with its task and its first thread's sort key
    struct E { uint32_t task; RPiece piece; unsigned long long k0; };
    const KeyLayout &L = out.L;
    std::vector<E> ent;
    for (size_t i = 0; i < ps.size(); i++) {
        const Prepared &p = *ps[i];
        const DevProto &d = out.protos[i];
        if (!range_candidate(p, d, rt)) continue;
        const size_t e0 = ent.size();
        uint64_t tuples = 0;
        for (const RangeAccess &r : p.range_access) {
            if (r.phase >= d.tab_phases || r.loc >= d.nlocs || r.offsets.empty() || r.modn >= (1ull << 40)) continue;
            // (offsets far outside any array would only fail the check: the
            // table pass keeps such an access)
            if (std::any_of(r.offsets.begin(), r.offsets.end(),
                            [](int64_t c) { return c < -(1ll << 50) || c > (1ll << 50); }))
                continue;
            const int64_t ncells = (int64_t)p.cells[r.loc];
            const int64_t sb = (int64_t)(d.tab_off + (uint64_t)r.phase * d.cells_sum + out.cbase[d.cells_off + r.loc]);
            const uint32_t wf = r.write ? kRWrite : 0u;
            const long long s = r.sigma;
            std::vector<Run> runs;
            for (int64_t c : r.offsets) {
                range_runs(r, c, p.nthreads, runs);
                for (size_t q = 0; q < runs.size(); q++) {
                    // within the array, then cut at task boundaries
                    long long t0, l0, len;
                    range_clip(runs[q].t0, sb + runs[q].cell0, runs[q].len, s, sb, sb + ncells, t0, l0, len);
                    while (len > 0) {
                        const long long task = l0 / (long long)kRangeRecs, base = task * (long long)kRangeRecs;
                        long long ct0, cl0, clen;
                        range_clip(t0, l0, len, s, base, base + (long long)kRangeRecs, ct0, cl0, clen);
                        // the key fields of the interpreted emit pass
                        unsigned long long k0 = ((unsigned long long)i << L.phase_bits) | r.phase;
                        k0 = (k0 << L.loc_bits) | r.loc;
                        k0 = (k0 << L.idx_bits) | (unsigned long long)(cl0 - sb);
                        k0 = (k0 << L.sort_lo) | ((unsigned long long)ct0 << 1) | (r.write ? 1u : 0u);
                        ent.push_back(E{(uint32_t)task, RPiece{(uint32_t)ct0, (uint32_t)clen | wf, (int32_t)(cl0 - base),
                                                               (int32_t)s}, k0});
                        t0 += clen;
                        l0 += s * clen;
                        len -= clen;
                    }
                }
            }
            out.range_pcs[i].push_back(r.pc);
            tuples += r.run_iters * (uint64_t)p.nthreads;
        }
        if (ent.size() > kRangeMaxEntries) {           // too many: this protocol keeps the table pass
            ent.resize(e0);
            out.range_pcs[i].clear();
            continue;
        }
        for (uint32_t pc : out.range_pcs[i]) out.insns[d.insn_off + pc].a |= AF_RANGE;
        mark_range_loops(&out.insns[d.insn_off], p.insns.size(), true);
        out.range_tuples += tuples;
        if (out.rtup.empty()) out.rtup.assign(ps.size(), 0);
        out.rtup[i] = tuples;
    }
    if (out.range_tuples < range_min) {              // protocols left out: under the minimum after all
        for (size_t i = 0; i < ps.size(); i++) {
            for (uint32_t pc : out.range_pcs[i]) out.insns[out.protos[i].insn_off + pc].a &= (uint8_t)~AF_RANGE;
            if (!out.range_pcs[i].empty()) mark_range_loops(&out.insns[out.protos[i].insn_off], ps[i]->insns.size(), false);
        }
        clear_range(out, ps.size());
        return;
    }
    // the pieces grouped by task, tasks ascending, each task's pieces in the
    // order they were cut (a counting sort over the table's tasks)
    const uint64_t ntasks = (out.table_cells + kRangeRecs - 1) / kRangeRecs;
    std::vector<uint32_t> at(ntasks + 1, 0);
    for (const E &x : ent) at[x.task + 1]++;
    for (uint64_t t = 0; t < ntasks; t++) {
        if (at[t + 1]) {
            out.rlive.push_back((uint32_t)t);
            out.rfirst.push_back(at[t]);
        }
        at[t + 1] += at[t];
    }
    if (!out.rlive.empty()) out.rfirst.push_back((uint32_t)ent.size());
    out.wpiece.resize(ent.size());
    out.wkeys.resize(ent.size());
    for (const E &x : ent) {
        const uint32_t q = at[x.task]++;
        out.wpiece[q] = x.piece;
        // next thread: index field + step, thread field + 1
        out.wkeys[q] = RKeys{0, x.k0, ((unsigned long long)(long long)x.piece.step << L.sort_lo) + 2ull,
                             x.piece.lenf & kRLen};
    }
    for (RKeys &k : out.wkeys) {
        k.pre = out.nrkeys;
        out.nrkeys += k.len;
    }
    // each task's pieces merged (merge_pieces): [mfirst[i], mfirst[i + 1])
    // of rpiece, and the record updates they make
    std::vector<uint32_t> mfirst;
    std::vector<uint64_t> work;
    std::vector<RPiece> tmp;
    for (size_t i = 0; i < out.rlive.size(); i++) {
        mfirst.push_back((uint32_t)out.rpiece.size());
        merge_pieces(out.wpiece.data() + out.rfirst[i], out.rfirst[i + 1] - out.rfirst[i], tmp);
        uint64_t w = 0;
        for (const RPiece &x : tmp) w += x.lenf & kRLen;
        out.rpiece.insert(out.rpiece.end(), tmp.begin(), tmp.end());
        work.push_back(w);
    }
    mfirst.push_back((uint32_t)out.rpiece.size());
    // a task with much work is split into parts over disjoint blocks of its
    // records (a part per kRangeSplitWork record updates, assuming them
    // spread evenly), each taken by its own block; blocks take the parts
    // from a shared counter, the largest first, so that the launch does not
    // end on a few blocks still working through big ones
    struct Part { RTask t; uint64_t work; };
    std::vector<Part> parts;
    parts.reserve(out.rlive.size());
    const uint64_t nblk_all = (out.table_cells + 255) / 256;
    for (size_t i = 0; i < out.rlive.size(); i++) {
        const uint64_t first = (uint64_t)out.rlive[i] * (kRangeRecs / 256);
        const uint32_t nblk = (uint32_t)std::min<uint64_t>(kRangeRecs / 256, nblk_all - first);
        const uint32_t k = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(nblk, (work[i] + kRangeSplitWork - 1) / kRangeSplitWork));
        for (uint32_t q = 0; q < k; q++) {
            const uint32_t b0 = nblk * q / k, b1 = nblk * (q + 1) / k;
            parts.push_back(Part{RTask{out.rlive[i], mfirst[i], mfirst[i + 1], b0 | (b1 << 16)}, work[i] / k});
        }
    }
    std::stable_sort(parts.begin(), parts.end(), [](const Part &x, const Part &y) { return x.work > y.work; });
    out.rtask.reserve(parts.size());
    for (const Part &x : parts) out.rtask.push_back(x.t);
}

DeviceBatch::~DeviceBatch()
{
    DevBuf *all[] = {&image, &cnt, &syn, &phs, &erro, &totsyn, &wcnt, &wbase, &blocksum, &keys0, &keys1, &hist,
                     &status, &trec, &err_key, &div_tid, &best_pos, &ptuples, &out, &epoch, &table,
                     &touch, &tlist, &hit, &ishape};
    for (DevBuf *b : all) release(*b, &in_use);
    if (staged) cudaEventDestroy(staged);
    if (stage) cudaFreeHost(stage);
    if (out_host) cudaFreeHost(out_host);
}

cudaError_t DeviceBatch::fetch(cudaStream_t s, bool ctrl_only)
{
    const size_t bytes = ctrl_only ? sizeof(Control) : kOutResults + (size_t)args.nprotos * sizeof(DevResult);
    d2h_bytes += bytes;
    return cudaMemcpyAsync(out_host, out.p, bytes, cudaMemcpyDeviceToHost, s);
}

namespace {

// One section of the batch image: its bytes start at a 256-byte boundary.
struct Section {
    const void *src;
    size_t bytes;
    size_t off;
};

template <typename T>
Section section(const std::vector<T> &v, size_t &end)
{
    Section x{v.data(), v.size() * sizeof(T), end};
    end += (x.bytes + 255) & ~(size_t)255;
    return x;
}

}  // namespace

Error DeviceBatch::load(const BatchHost &b, cudaStream_t s, bool schedule)
{
    static const std::vector<WarpItem> no_witems;
    static const std::vector<RKeys> no_wkeys;
    // the range pieces' key templates: only for the sort path's range keys
    const bool keys = path_pref == 1 && b.nrkeys && !b.rtup.empty();
    const uint64_t np = b.protos.size();
    const uint64_t nw = b.nwitems;
    const uint32_t nwblocks = (uint32_t)std::max<uint64_t>(1, (nw + kWScanPerBlock - 1) / kWScanPerBlock);
    h2d_bytes = 0;
    d2h_bytes = 0;
    // the image: every host section packed into pinned memory, then one copy
    size_t end = 0;
    const Section sec[] = {section(b.insns, end), section(b.xcode, end), section(b.items, end),
                           section(b.protos, end), section(b.cells, end), section(b.cbase, end),
                           section(schedule ? b.witems : no_witems, end), section(b.iphase, end), section(b.rpiece, end),
                           section(b.rtask, end), section(b.rlive, end), section(b.rfirst, end),
                           section(b.wpiece, end), section(b.rtup, end), section(keys ? b.wkeys : no_wkeys, end)};
    const size_t total = std::max<size_t>(end, 256);
    bool ok = ensure(image, total, &in_use, limit);
    // the stage already holds this image (the same pack loaded again): it is
    // copied to the device as it is
    const bool restage = !(b.version && staged_version == b.version && staged_schedule == schedule &&
                           staged_keys == keys && stage && stage_cap >= total);
    // the previous copy out of the stage must be done before it is rewritten
    if (ok && staged_pending && restage) ok = cudaEventSynchronize(staged) == cudaSuccess;
    if (restage) staged_pending = false;
    if (ok && stage_cap < total) {
        const size_t want = std::max(total, stage_cap + stage_cap / 4);
        if (stage) cudaFreeHost(stage);
        stage = nullptr;
        stage_cap = 0;
        ok = cudaHostAlloc(&stage, want, cudaHostAllocDefault) == cudaSuccess;
        if (ok) stage_cap = want;
        else stage = nullptr;
    }
    if (ok && !staged) ok = cudaEventCreateWithFlags(&staged, cudaEventDisableTiming) == cudaSuccess;
    if (ok) {
        if (restage) {
            staged_version = 0;
            for (const Section &x : sec)
                if (x.bytes) std::memcpy((char *)stage + x.off, x.src, x.bytes);
            staged_version = b.version;
            staged_schedule = schedule;
            staged_keys = keys;
        }
        ok = cudaMemcpyAsync(image.p, stage, end ? end : 16, cudaMemcpyHostToDevice, s) == cudaSuccess &&
             cudaEventRecord(staged, s) == cudaSuccess;
        staged_pending = ok;
        h2d_bytes = end;
    }
    const size_t lanes = std::max<uint64_t>(b.lanes, 1);
    ok = ok && ensure(cnt, lanes * 4, &in_use, limit) && ensure(syn, lanes * 4, &in_use, limit) &&
         ensure(phs, lanes * 4, &in_use, limit) && ensure(erro, lanes * 8, &in_use, limit) &&
         ensure(totsyn, std::max<uint64_t>(b.ncols, 1) * 4, &in_use, limit) &&
         ensure(wcnt, std::max<uint64_t>(nw, 1) * 4, &in_use, limit) &&
         ensure(wbase, std::max<uint64_t>(nw, 1) * 8, &in_use, limit) &&
         ensure(blocksum, (size_t)nwblocks * 8, &in_use, limit) &&
         ensure(hist, (size_t)kMaxPasses * kRadixBins * 8, &in_use, limit) &&
         ensure(err_key, np * 8, &in_use, limit) && ensure(div_tid, np * 4, &in_use, limit) &&
         ensure(best_pos, np * 8, &in_use, limit) && ensure(ptuples, np * 8, &in_use, limit) &&
         ensure(out, kOutResults + np * sizeof(DevResult), &in_use, limit);
    if (ok && out_host_cap < kOutResults + np * sizeof(DevResult)) {
        // every reader of the mirror waits for its copy before the next load
        const size_t want = std::max(kOutResults + np * sizeof(DevResult), out_host_cap + out_host_cap / 4);
        if (out_host) cudaFreeHost(out_host);
        out_host = nullptr;
        out_host_cap = 0;
        ok = cudaHostAlloc(&out_host, want, cudaHostAllocDefault) == cudaSuccess;
        if (ok) out_host_cap = want;
        else out_host = nullptr;
    }
    if (ok && !epoch.p) {
        ok = ensure(epoch, 16, &in_use, limit) && cudaMemsetAsync(epoch.p, 0, 16, s) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        return Error::make(S_NOMEM, "device allocation failed");
    }
    BatchArgs &a = args;
    char *img = (char *)image.p;
    a.insns = (const Insn *)(img + sec[0].off);
    a.xcode = (const uint64_t *)(img + sec[1].off);
    a.items = (const ItemDesc *)(img + sec[2].off);
    a.protos = (const DevProto *)(img + sec[3].off);
    a.cells = (const uint64_t *)(img + sec[4].off);
    a.cbase = (const uint64_t *)(img + sec[5].off);
    // without its expansion, kernels that read the schedule refuse to launch
    a.witems = schedule && b.expanded() ? (const WarpItem *)(img + sec[6].off) : nullptr;
    a.iphase = (const uint32_t *)(img + sec[7].off);
    a.count_free = 0;
    a.rpiece = (const RPiece *)(img + sec[8].off);
    a.rtask = (const RTask *)(img + sec[9].off);
    a.rlive = (const uint32_t *)(img + sec[10].off);
    a.rfirst = (const uint32_t *)(img + sec[11].off);
    a.wpiece = (const RPiece *)(img + sec[12].off);
    a.rtup = b.rtup.empty() ? nullptr : (const unsigned long long *)(img + sec[13].off);
    a.rtotal = b.rtup.empty() ? 0ull : b.range_tuples;
    a.rcount = 0;
    a.wkeys = (const RKeys *)(img + sec[14].off);
    // a forced sort path emits the range accesses' keys from the pieces
    a.range_keys = keys ? 1u : 0u;
    a.nrkeys = a.range_keys ? b.nrkeys : 0ull;
    a.nwkeys = a.range_keys ? (uint32_t)b.wkeys.size() : 0u;
    a.nlive = (uint32_t)b.rlive.size();
    a.nrtask = (uint32_t)b.rtask.size();
    a.range_on = 0;
    a.nwitems = (uint32_t)nw;
    a.nprotos = (uint32_t)np;
    a.has_narrow = a.has_wide = 0;
    for (const DevProto &d : b.protos) (d.wide ? a.has_wide : a.has_narrow) = 1;
    a.ncols = b.ncols;
    a.cnt = (uint32_t *)cnt.p;
    a.syn = (uint32_t *)syn.p;
    a.phs = (uint32_t *)phs.p;
    a.erro = (unsigned long long *)erro.p;
    a.totsyn = (uint32_t *)totsyn.p;
    a.wcnt = (uint32_t *)wcnt.p;
    a.wbase = (unsigned long long *)wbase.p;
    a.blocksum = (unsigned long long *)blocksum.p;
    a.nwblocks = nwblocks;
    a.hist = (unsigned long long *)hist.p;
    a.err_key = (unsigned long long *)err_key.p;
    a.div_tid = (uint32_t *)div_tid.p;
    a.best_pos = (unsigned long long *)best_pos.p;
    a.ptuples = (unsigned long long *)ptuples.p;
    a.ctrl = (Control *)out.p;
    a.results = (DevResult *)((char *)out.p + kOutResults);
    a.epoch = (uint32_t *)epoch.p;
    a.L = b.L;
    a.radix_items = radix_items;
    a.stall_lookback = 0;
    a.shard_lo = shard_lo;
    a.shard_hi = shard_hi;
    a.nkeys = 0;
    a.ntiles = 0;
    a.keys[0] = (unsigned long long *)keys0.p;
    a.keys[1] = (unsigned long long *)keys1.p;
    a.status = (unsigned long long *)status.p;
    a.path = PATH_SORT;
    a.table = nullptr;
    a.tab_cells = 0;
    a.touch = nullptr;
    a.tlist = nullptr;
    a.hit_acc = a.hit_wr = nullptr;
    a.nhit = 0;
    return Error{};
}

Error DeviceBatch::size_table(const BatchHost &b, uint64_t n, cudaStream_t s)
{
    const uint64_t recs = table_blocks(b.table_cells) * kTabBlock;
    const size_t tb = std::max<uint64_t>(recs * 4, 16);
    const size_t wb = std::max<uint64_t>(touch_words(b.table_cells) * 4, 16);
    const uint64_t nhit = (b.ncols + 31) / 32 + 1;
    const uint64_t old_table = table.gen, old_touch = touch.gen;
    const size_t lb = std::max<uint64_t>(table_blocks(b.table_cells) * 4, 16);
    if (!ensure(table, tb, &in_use, limit) || !ensure(touch, wb, &in_use, limit) ||
        !ensure(tlist, lb, &in_use, limit) || !ensure(hit, nhit * 8, &in_use, limit)) {
        cudaGetLastError();
        // the table or its touch bits may have moved to fresh memory that was
        // not cleared: clear them when the next launch sizes them
        if (table.gen != old_table || touch.gen != old_touch) table_dirty = true;
        return Error::make(S_NOMEM, "device allocation of a " + std::to_string(tb) + "-byte owner table failed");
    }
    // the kernels keep the table and its touch bits all zero between
    // launches; fresh memory (or a failed launch) needs one clear
    if (table.gen != old_table || touch.gen != old_touch || table_dirty) {
        if (cudaMemsetAsync(table.p, 0, table.cap, s) != cudaSuccess ||
            cudaMemsetAsync(touch.p, 0, touch.cap, s) != cudaSuccess)
            return Error::make(S_CUDA, "memset failed");
        table_dirty = false;
    }
    BatchArgs &a = args;
    a.path = PATH_TABLE;
    a.range_on = a.nlive ? 1u : 0u;
    a.table = table.p;
    a.tab_cells = b.table_cells;
    a.touch = (uint32_t *)touch.p;
    a.tlist = (uint32_t *)tlist.p;
    a.hit_acc = (uint32_t *)hit.p;
    a.hit_wr = (uint32_t *)hit.p + nhit;
    a.nhit = nhit;
    a.nkeys = n;
    a.ntiles = 0;
    a.ndtiles = 0;
    return Error{};
}

uint32_t auto_path(const BatchHost &b, uint64_t n)
{
    // The table path reads only the blocks the accesses touched, so its cost
    // follows the tuples; the table's size costs memory and one clear.  Take
    // it unless the table is far larger than the accesses that fill it.
    if (!b.table_ok) return PATH_SORT;
    const uint64_t bytes = b.table_bytes();
    return bytes <= std::max<uint64_t>(256ull << 20, n * 256) ? PATH_TABLE : PATH_SORT;
}

Error DeviceBatch::choose_path(const BatchHost &b, uint64_t n, cudaStream_t s)
{
    uint32_t path = path_pref == 1 ? PATH_SORT : path_pref == 2 ? PATH_TABLE : auto_path(b, n);
    if (path == PATH_TABLE) {
        Error e = b.table_ok ? size_table(b, n, s)
                             : Error::make(S_LIMIT, "the owner table of this batch would exceed " +
                                                        std::to_string(kMaxTableBytes >> 30) + " GiB");
        if (e.ok()) return e;
        if (path_pref == 2) return e;
    }
    args.path = PATH_SORT;
    return size_keys(n, s);
}

Error DeviceBatch::size_keys(uint64_t n, cudaStream_t s)
{
    n += args.range_keys ? args.nrkeys : 0;        // the range accesses' keys follow the counted ones
    const uint32_t tiles = radix_tiles(n, args.radix_items);
    const size_t kb = std::max<uint64_t>(n, 1) * 8;
    const size_t sb = std::max<size_t>((size_t)args.L.passes * tiles * kRadixBins * 8, 16);
    const uint64_t old_status = status.gen;
    const uint32_t dtiles = detect_tiles(n);
    bool ok = ensure(keys0, kb, &in_use, limit) && ensure(keys1, kb, &in_use, limit) &&
              ensure(status, sb, &in_use, limit) &&
              ensure(trec, std::max<size_t>((size_t)dtiles * sizeof(TileRec), 16), &in_use, limit);
    if (!ok) {
        cudaGetLastError();
        return Error::make(S_NOMEM, "device allocation for " + std::to_string(n) + " access keys failed");
    }
    // fresh look-back words must not carry a stale tag; clear them when the
    // buffer is new and well before the 22-bit launch tag wraps
    if (status.gen != old_status || status_launches >= (1ull << 21)) {
        if (cudaMemsetAsync(status.p, 0, status.cap, s) != cudaSuccess) return Error::make(S_CUDA, "memset failed");
        status_launches = 0;
    }
    args.nkeys = n;
    args.range_on = 0;
    args.ntiles = tiles;
    args.ndtiles = dtiles;
    args.trec = (TileRec *)trec.p;
    args.keys[0] = (unsigned long long *)keys0.p;
    args.keys[1] = (unsigned long long *)keys1.p;
    args.status = (unsigned long long *)status.p;
    return Error{};
}

static int flags_status(unsigned flags)
{
    if (flags & CF_LOOKBACK_TIMEOUT) return S_TIMEOUT;
    if (flags) return S_INTERNAL;
    return S_OK;
}

// Copies the mirrored results into `out` and checks the control flags.
static int collect(const DeviceBatch &w, std::vector<DevResult> &out, std::string &err)
{
    out.assign(w.host_results(), w.host_results() + w.args.nprotos);
    const unsigned flags = w.host_ctrl()->flags;
    int st = flags_status(flags);
    if (st) err = "device pipeline consistency check failed (flags " + std::to_string(flags) + ")";
    return st;
}

int run_batch(DeviceBatch &w, int sms, cudaStream_t s, const BatchHost &b, std::vector<DevResult> &out,
              std::string &err)
{
    Error e = w.load(b, s);
    if (!e.ok()) { err = e.message; return e.status; }
    // When the tuple bound already selects the owner table (the automatic
    // choice made on the bound, or the table asked for), nothing the host
    // does depends on the count: front and back run in one go, one wait.
    if (b.table_ok && w.path_pref != 1 && (w.path_pref == 2 || auto_path(b, b.tuple_bound) == PATH_TABLE)) {
        e = w.size_table(b, kUncounted, s);
        if (e.ok()) {
            w.args.count_free = b.all_static ? 1u : 0u;   // nothing to count first: no count or scan pass
            w.status_launches++;
            if (launch_front(w.args, s, sms, nullptr, nullptr) != cudaSuccess ||
                launch_back(w.args, s, sms, nullptr, nullptr) != cudaSuccess || w.fetch(s, false) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                err = cudaGetErrorString(cudaGetLastError());
                w.table_dirty = true;
                return S_CUDA;
            }
            return collect(w, out, err);
        }
        if (w.path_pref == 2) { err = e.message; return e.status; }
        cudaGetLastError();                          // no room for the table: count, then choose
    }
    if (launch_front(w.args, s, sms, nullptr, nullptr) != cudaSuccess || w.fetch(s, true) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        err = cudaGetErrorString(cudaGetLastError());
        return S_CUDA;
    }
    const uint64_t n = w.host_ctrl()->total;
    w.args.count_free = 0;                           // the count pass ran
    e = w.choose_path(b, n, s);
    if (!e.ok()) { err = e.message; return e.status; }
    w.args.stall_lookback = 0;
    if (w.stall_lookback && w.args.path == PATH_SORT) {
        w.args.stall_lookback = 1;
        w.stall_lookback--;
    }
    w.status_launches++;
    if (launch_back(w.args, s, sms, nullptr, nullptr) != cudaSuccess || w.fetch(s, false) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        err = cudaGetErrorString(cudaGetLastError());
        w.table_dirty = true;
        return S_CUDA;
    }
    return collect(w, out, err);
}

JitEntry::~JitEntry()
{
    if (shape) cudaFree(shape);
}

int run_batch_jit(drf_ctx *ctx, const BatchHost &b, const JitLaunch &j, cudaStream_t s, std::vector<DevResult> &out)
{
    DeviceBatch &w = ctx->work;
    w.limit = ctx->opts.max_device_bytes;
    w.path_pref = 2;                               // specialized kernels run the owner-table back end
    Error e = w.load(b, s, !j.csched);             // a compiled-in schedule needs no warp-item array
    if (e.ok()) e = w.choose_path(b, b.tuple_bound, s);
    if (!e.ok() || w.args.path != PATH_TABLE) {
        ctx->last_error = e.message;
        return e.ok() ? S_LIMIT : e.status;
    }
    w.args.nkeys = kUncounted;                     // no sizing run: the count is known only afterwards
    w.status_launches++;
    if (launch_front(w.args, s, ctx->sms, nullptr, nullptr, &j) != cudaSuccess ||
        launch_back(w.args, s, ctx->sms, nullptr, nullptr, &j) != cudaSuccess || w.fetch(s, false) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        ctx->last_error = cudaGetErrorString(cudaGetLastError());
        w.table_dirty = true;
        return S_CUDA;
    }
    return collect(w, out, ctx->last_error);
}

std::shared_ptr<const Prepared> PrepCache::get(const uint8_t *bc, size_t len, const drf_bounds *b,
                                               const PrepareOpts &po, Error &err)
{
    err = Error{};
    if (!bc || !b) {
        err = Error::make(S_INVALID_ARG, "null bytecode or bounds");
        return nullptr;
    }
    if ((b->nlocs && !b->loc_cells) || (b->nparams && !b->params)) {
        err = Error::make(S_INVALID_ARG, "null array sizes or params");
        return nullptr;
    }
    std::string key;
    key.reserve(len + 64 + 8 * (b->nlocs + b->nparams));
    auto put = [&key](const void *x, size_t n) { key.append((const char *)x, n); };
    put(&po, sizeof po);
    put(&b->nthreads, sizeof b->nthreads);
    put(&b->nlocs, sizeof b->nlocs);
    if (b->nlocs) put(b->loc_cells, b->nlocs * sizeof(uint64_t));
    put(&b->nparams, sizeof b->nparams);
    if (b->nparams) put(b->params, b->nparams * sizeof(int64_t));
    put(&len, sizeof len);
    put(bc, len);
    {
        std::lock_guard<std::mutex> g(mu_);
        auto it = map_.find(key);
        if (it != map_.end()) return it->second;
    }
    auto p = std::make_shared<Prepared>();
    err = prepare(bc, len, b->nthreads, b->nlocs, b->loc_cells, b->nparams, b->params, po, *p);
    if (!err.ok()) return nullptr;
    std::lock_guard<std::mutex> g(mu_);
    if (map_.size() >= kCap) map_.clear();
    map_.emplace(std::move(key), p);
    return p;
}

int path_pref_of(const drf_opts &o)
{
    if (o.flags & DRF_OPT_PATH_SORT) return 1;
    if (o.flags & DRF_OPT_PATH_TABLE) return 2;
    return 0;
}

uint64_t range_min_of(const drf_opts &o) { return (o.flags & DRF_OPT_RANGE_ANY) ? 0 : kRangeMinTuples; }

uint64_t range_min_once(const drf_opts &o) { return (o.flags & DRF_OPT_RANGE_ANY) ? 0 : ~0ull; }

int run_batch(drf_ctx *ctx, const BatchHost &b, cudaStream_t s, std::vector<DevResult> &out)
{
    ctx->work.limit = ctx->opts.max_device_bytes;
    ctx->work.path_pref = path_pref_of(ctx->opts);
    return run_batch(ctx->work, ctx->sms, s, b, out, ctx->last_error);
}

void to_public(const DevResult &d, drf_result *o)
{
    std::memset(o, 0, sizeof *o);
    o->status = d.status;
    o->verdict = d.status ? -1 : d.verdict;
    o->phase = d.phase;
    o->loc = d.loc;
    o->index = d.index;
    o->tid_i = d.tid_i;
    o->tid_j = d.tid_j;
    o->i_writes = d.i_writes;
    o->j_writes = d.j_writes;
    o->div_tid = d.div_tid;
    o->sync_count_0 = d.sync_count_0;
    o->sync_count_div = d.sync_count_div;
    o->phases = d.phases;
    o->tuples = d.tuples;
    o->err_tid = d.err_tid;
    o->err_ordinal = d.err_ordinal;
}

}  // namespace drf
