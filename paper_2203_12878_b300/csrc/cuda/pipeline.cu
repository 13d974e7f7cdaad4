// Device pipeline: a concrete check of Definition 1 (DRF program, Sec. 3)
// for every thread id at once (rule par, Fig. 3).
//
//   init      clear the launch's control block and per-protocol reductions
//   count     interpret every (item, thread): accesses, syncs, first error
//   scan      per thread, exclusive scan of syncs over items -> phase at item
//             start; exclusive scan of per-warp access counts -> key offsets
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
//   finalize  per protocol: first evaluation error (smallest tid, then the
//             number of accesses before it), else barrier divergence, else
//             the witness of the first racy segment: i = smallest accessor,
//             j = its smallest admissible partner
#include <cstdint>

#include "pipeline.cuh"

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

// ------------------------------------------------------- integer semantics
// Floor division and Euclidean remainder.  The host's interval analysis
// guarantees b != 0 where no check is made and that no result overflows.
template <typename V, typename U>
__device__ __forceinline__ V floor_div(V a, V b)
{
    V q = a / b;
    V r = (V)((U)a - (U)q * (U)b);
    if (r != 0 && ((r < 0) != (b < 0))) q -= 1;
    return q;
}

template <typename V, typename U>
__device__ __forceinline__ V euclid_mod(V a, V b)
{
    V r = a % b;
    if (r < 0) r = (V)(b > 0 ? (U)r + (U)b : (U)r - (U)b);
    return r;
}

template <typename V> struct Unsigned;
template <> struct Unsigned<int32_t> { using T = uint32_t; };
template <> struct Unsigned<int64_t> { using T = uint64_t; };

// Stack machine over the expression code (see devprog.h).  Returns false on
// a division or remainder by zero.
template <typename V>
__device__ bool eval(const uint64_t *__restrict__ xc, int32_t off, uint32_t tid, const V *vars, V &out)
{
    using U = typename Unsigned<V>::T;
    V st[kMaxStack];
    int sp = 0;
    const uint64_t *p = xc + off;
    while (true) {
        uint64_t w = __ldg(p++);
        uint32_t op = (uint32_t)(w & 0xff);
        switch (op) {
        case X_RET: out = st[0]; return true;
        case X_CONST: st[sp++] = (V)(int64_t)__ldg(p++); break;
        case X_TID: st[sp++] = (V)tid; break;
        case X_VAR: st[sp++] = vars[(uint32_t)(w >> 8)]; break;
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
            st[sp++] = (V)acc;
            break;
        }
        case X_ADD: sp--; st[sp - 1] = (V)((U)st[sp - 1] + (U)st[sp]); break;
        case X_SUB: sp--; st[sp - 1] = (V)((U)st[sp - 1] - (U)st[sp]); break;
        case X_MUL: sp--; st[sp - 1] = (V)((U)st[sp - 1] * (U)st[sp]); break;
        case X_MIN: sp--; st[sp - 1] = st[sp] < st[sp - 1] ? st[sp] : st[sp - 1]; break;
        case X_MAX: sp--; st[sp - 1] = st[sp] > st[sp - 1] ? st[sp] : st[sp - 1]; break;
        case X_NEG: st[sp - 1] = (V)(0 - (U)st[sp - 1]); break;
        case X_DIV:
        case X_MOD: {
            V b = st[--sp];
            if (b == 0) return false;
            st[sp - 1] = op == X_DIV ? floor_div<V, U>(st[sp - 1], b) : euclid_mod<V, U>(st[sp - 1], b);
            break;
        }
        case X_DIVC: st[sp - 1] = floor_div<V, U>(st[sp - 1], (V)(int64_t)__ldg(p++)); break;
        case X_MODC: st[sp - 1] = euclid_mod<V, U>(st[sp - 1], (V)(int64_t)__ldg(p++)); break;
        case X_MASK: st[sp - 1] = (V)((U)st[sp - 1] & (U)__ldg(p++)); break;
        case X_EQ: sp--; st[sp - 1] = st[sp - 1] == st[sp]; break;
        case X_NE: sp--; st[sp - 1] = st[sp - 1] != st[sp]; break;
        case X_LT: sp--; st[sp - 1] = st[sp - 1] < st[sp]; break;
        case X_LE: sp--; st[sp - 1] = st[sp - 1] <= st[sp]; break;
        case X_GT: sp--; st[sp - 1] = st[sp - 1] > st[sp]; break;
        case X_GE: sp--; st[sp - 1] = st[sp - 1] >= st[sp]; break;
        case X_AND: sp--; st[sp - 1] = (st[sp - 1] != 0) & (st[sp] != 0); break;
        case X_OR: sp--; st[sp - 1] = (st[sp - 1] != 0) | (st[sp] != 0); break;
        case X_NOT: st[sp - 1] = st[sp - 1] == 0; break;
        default: return false;   // not produced by the lowering
        }
    }
}

// Per-warp histogram cache: the emit kernel counts digits in shared memory.
struct EmitShared {
    unsigned int hist[kMaxPasses][kRadixBins];
};

// Interprets one item for the 32 threads of a warp (threads 32g .. 32g+31).
// All lanes fetch the instruction at the smallest pc among running lanes and
// only lanes at that pc execute it, so lanes that diverge on a thread-
// dependent condition or trip count re-converge at the join point.
template <typename V, bool EMIT>
__device__ void run_item(const BatchArgs &a, uint32_t p, const DevProto &P, const ItemDesc &it, uint32_t k,
                         uint32_t g, uint32_t w, EmitShared *sh)
{
    using U = typename Unsigned<V>::T;
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
    unsigned long long cursor = 0, wend = 0;
    if (EMIT) {
        if (alive) phase = a.phs[li];
        cursor = a.wbase[w];
        wend = cursor + a.wcnt[w];
    }
    const KeyLayout L = a.L;
    const unsigned long long tidpart = (((unsigned long long)tid) << 1);

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
            if (ex && (EMIT || (in.a & AF_EVAL_IN_COUNT))) {
                if (!eval<V>(xc, in.c, tid, vars, idx)) { err = kErrDiv0; ok = false; }
                else if (idx < 0 || (uint64_t)(U)idx >= __ldg(cells + in.b)) { err = kErrOob; ok = false; }
            }
            if (ex && !ok) running = false;
            if (EMIT) {
                unsigned em = __ballot_sync(kFull, ok);
                if (ok) {
                    unsigned long long pos = cursor + __popc(em & lanemask_lt());
                    unsigned long long key = ((unsigned long long)p << L.phase_bits) | phase;
                    key = (key << L.loc_bits) | in.b;
                    key = (key << L.idx_bits) | (unsigned long long)(U)idx;
                    key = (key << (L.tid_bits + 1)) | tidpart | (in.a & AF_WRITE);
                    if (pos < wend && pos < a.nkeys) {
                        a.keys[0][pos] = key;
                        for (uint32_t q = 0; q < L.passes; q++)
                            atomicAdd(&sh->hist[q][(key >> (L.sort_lo + q * kRadixBits)) & (kRadixBins - 1)], 1u);
                    } else {
                        atomicOr(&a.ctrl->flags, CF_EMIT_OVERFLOW);
                    }
                }
                cursor += __popc(em);
            } else if (ok) {
                count++;
            }
            if (ok) pc++;
            break;
        }
        case I_SYNC:
            if (ex) { if (EMIT) phase++; else syncs++; pc++; }
            break;
        case I_LOOP:
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
        default:
            if (ex) running = false;
            break;
        }
        if (ex && running && pc == it.stop_pc) running = false;
    }

    if (!EMIT && alive) {
        a.cnt[li] = count;
        a.syn[li] = syncs;
        if (err) {
            a.erro[li] = ((unsigned long long)count << 8) | err;
            atomicMin(&a.err_key[p], ((unsigned long long)tid << 32) | k);
        }
    }
    if (!EMIT) {
        uint32_t total = __reduce_add_sync(kFull, count);
        if (lane == 0) {
            a.wcnt[w] = total;
            if (total) {
                atomicAdd(&a.blocksum[w / kWScanPerBlock], (unsigned long long)total);
                atomicAdd(&a.ptuples[p], (unsigned long long)total);
            }
        }
    }
}

// ------------------------------------------------------------------ kernels

__global__ void k_init(BatchArgs a)
{
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i < a.nprotos) {
        a.err_key[i] = kNone;
        a.div_tid[i] = 0xFFFFFFFFu;
        a.best_pos[i] = kNone;
        a.ptuples[i] = 0;
    }
    if (i < (uint64_t)kMaxPasses * kRadixBins) a.hist[i] = 0;
    if (i < a.nwblocks) a.blocksum[i] = 0;
    if (i < sizeof(Control) / sizeof(unsigned int)) reinterpret_cast<unsigned int *>(a.ctrl)[i] = 0;
    if (i == 0) *a.epoch = *a.epoch + 1;
}

template <bool EMIT>
__global__ void __launch_bounds__(256) k_interp(BatchArgs a)
{
    __shared__ EmitShared sh;
    if (EMIT) {
        for (int i = threadIdx.x; i < kMaxPasses * kRadixBins; i += blockDim.x) (&sh.hist[0][0])[i] = 0;
        __syncthreads();
    }
    const uint32_t warps = gridDim.x * (blockDim.x / 32);
    for (uint32_t w = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; w < a.nwitems; w += warps) {
        const WarpItem wi = a.witems[w];
        const DevProto P = a.protos[wi.proto];
        const ItemDesc it = a.items[P.item_off + wi.k];
        if (EMIT && wi.k == 0) {
            // barrier divergence: every thread must run as many syncs as thread 0
            uint32_t tid = wi.g * 32 + (threadIdx.x & 31);
            if (tid < P.nthreads && a.totsyn[P.tid_off + tid] != a.totsyn[P.tid_off])
                atomicMin(&a.div_tid[wi.proto], tid);
        }
        if (P.wide) run_item<int64_t, EMIT>(a, wi.proto, P, it, wi.k, wi.g, w, &sh);
        else run_item<int32_t, EMIT>(a, wi.proto, P, it, wi.k, wi.g, w, &sh);
    }
    if (EMIT) {
        __syncthreads();
        for (int i = threadIdx.x; i < (int)(a.L.passes * kRadixBins); i += blockDim.x) {
            unsigned int v = (&sh.hist[0][0])[i];
            if (v) atomicAdd(&a.hist[i], (unsigned long long)v);
        }
    }
}

// Two roles.  Blocks [0, col_blocks): per-thread exclusive scan of syncs over
// items.  The remaining blocks: exclusive scan of per-warp-item access counts
// (4096 per block; the block's offset is the sum of the earlier blocks'
// totals, accumulated by the count kernel).
__global__ void __launch_bounds__(kScanThreads) k_scan(BatchArgs a, uint32_t col_blocks)
{
    if (blockIdx.x < col_blocks) {
        uint64_t c = blockIdx.x * (uint64_t)kScanThreads + threadIdx.x;
        if (c >= a.ncols) return;
        uint32_t lo = 0, hi = a.nprotos - 1;               // protocol owning column c
        while (lo < hi) {
            uint32_t mid = (lo + hi + 1) / 2;
            if (a.protos[mid].tid_off <= c) lo = mid; else hi = mid - 1;
        }
        const DevProto P = a.protos[lo];
        uint32_t t = (uint32_t)(c - P.tid_off);
        uint32_t run = 0;
        for (uint32_t k = 0; k < P.nitems; k++) {
            uint64_t li = P.lane_off + (uint64_t)k * P.nthreads + t;
            a.phs[li] = run;
            run += a.syn[li];
        }
        a.totsyn[c] = run;
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
// Look-back status word: flag (bits 62..63: 1 aggregate, 2 inclusive
// prefix), launch tag (bits 40..61), count (bits 0..39).
constexpr unsigned long long kFlagAgg = 1ull << 62, kFlagPrefix = 2ull << 62;
constexpr unsigned long long kValueMask = (1ull << 40) - 1;
constexpr int kTagShift = 40;
constexpr unsigned long long kTagMask = (1ull << 22) - 1;
constexpr uint32_t kSpinLimit = 1u << 22;   // ~ a second of waiting at most

__device__ __forceinline__ unsigned long long ld_status(const unsigned long long *p)
{
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}
__device__ __forceinline__ void st_status(unsigned long long *p, unsigned long long v)
{
    *reinterpret_cast<volatile unsigned long long *>(p) = v;
}

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
    return before;
}

__global__ void __launch_bounds__(kRadixThreads) k_radix(BatchArgs a, uint32_t pass)
{
    static_assert(kRadixThreads == kRadixBins, "one thread per digit");
    __shared__ unsigned long long s_keys[kRadixTile];
    __shared__ uint32_t s_whist[kRadixThreads / 32][kRadixBins];
    __shared__ uint32_t s_tstart[kRadixBins];
    __shared__ unsigned long long s_gofs[kRadixBins];
    __shared__ unsigned long long s_scan[kRadixThreads / 32];
    __shared__ uint32_t s_tile;

    bool self;
    int before = nontrivial_before(a, pass, &self);
    if (!self) return;
    const unsigned long long *src = a.keys[before & 1];
    unsigned long long *dst = a.keys[(before + 1) & 1];
    const uint32_t t = threadIdx.x, lane = t & 31, wid = t / 32;
    const uint32_t shift = a.L.sort_lo + pass * kRadixBits;
    const uint32_t nbits = min((uint32_t)kRadixBits, a.L.sort_bits - pass * kRadixBits);
    const uint32_t dmask = (1u << nbits) - 1;
    const unsigned long long tag = (unsigned long long)(*a.epoch & kTagMask) << kTagShift;
    unsigned long long *status = a.status + (uint64_t)pass * a.ntiles * kRadixBins;

    for (int w = 0; w < kRadixThreads / 32; w++) s_whist[w][t] = 0;
    if (t == 0) s_tile = (uint32_t)atomicAdd(&a.ctrl->tile_counter[pass], 1ull);
    // global start of every digit: exclusive scan of this pass's histogram
    unsigned long long h = a.hist[pass * kRadixBins + t];
    unsigned long long incl = h;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_scan[wid] = incl;
    __syncthreads();
    unsigned long long dbase = incl - h;
    for (uint32_t i = 0; i < wid; i++) dbase += s_scan[i];
    const uint32_t tile = s_tile;
    const uint64_t base = (uint64_t)tile * kRadixTile;
    const uint64_t n = a.nkeys;

    // load: warp w owns keys [w*512, (w+1)*512) of the tile, 32 per round
    unsigned long long key[kRadixItems];
    uint32_t rank[kRadixItems];
    const uint64_t wbase = base + wid * (32 * kRadixItems);
#pragma unroll
    for (int i = 0; i < kRadixItems; i++) {
        uint64_t idx = wbase + i * 32 + lane;
        key[i] = idx < n ? src[idx] : 0;
    }
    // rank within the warp, stable in (round, lane) order
#pragma unroll
    for (int i = 0; i < kRadixItems; i++) {
        uint64_t idx = wbase + i * 32 + lane;
        bool valid = idx < n;
        uint32_t d = (uint32_t)(key[i] >> shift) & dmask;
        unsigned peers = __ballot_sync(kFull, valid);
        for (uint32_t b = 0; b < nbits; b++) {
            unsigned bal = __ballot_sync(kFull, (d >> b) & 1);
            peers &= ((d >> b) & 1) ? bal : ~bal;
        }
        uint32_t before_me = __popc(peers & lanemask_lt());
        uint32_t prior = valid ? s_whist[wid][d] : 0;
        __syncwarp();
        if (valid && before_me == 0) s_whist[wid][d] = prior + __popc(peers);
        __syncwarp();
        rank[i] = prior + before_me;
    }
    __syncthreads();
    // per digit: exclusive offsets of each warp, and the tile's count
    uint32_t cnt = 0;
    for (int w = 0; w < kRadixThreads / 32; w++) {
        uint32_t c = s_whist[w][t];
        s_whist[w][t] = cnt;
        cnt += c;
    }
    // publish this tile's aggregate for digit t, then look back
    unsigned long long *my = status + (uint64_t)tile * kRadixBins + t;
    if (tile == 0) st_status(my, kFlagPrefix | tag | cnt);
    else st_status(my, kFlagAgg | tag | cnt);
    unsigned long long excl = 0;
    if (tile > 0) {
        int64_t j = (int64_t)tile - 1;
        uint32_t spins = 0;
        bool gave_up = false;
        while (j >= 0) {
            unsigned long long s = ld_status(status + (uint64_t)j * kRadixBins + t);
            if ((s & (kTagMask << kTagShift)) != tag || (s >> 62) == 0) {
                if (++spins > kSpinLimit) { gave_up = true; break; }
                __nanosleep(spins < 64 ? 32 : 256);
                continue;
            }
            excl += s & kValueMask;
            if ((s >> 62) == 2) break;
            j--;
        }
        if (gave_up) atomicOr(&a.ctrl->flags, CF_LOOKBACK_TIMEOUT);
        st_status(my, kFlagPrefix | tag | ((excl + cnt) & kValueMask));
    }
    // tile-local start of every digit
    uint32_t tincl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, tincl, o);
        if (lane >= o) tincl += y;
    }
    __syncthreads();
    if (lane == 31) s_scan[wid] = tincl;
    __syncthreads();
    uint32_t tstart = tincl - cnt;
    for (uint32_t i = 0; i < wid; i++) tstart += (uint32_t)s_scan[i];
    s_tstart[t] = tstart;
    s_gofs[t] = dbase + excl;
    __syncthreads();
    // scatter into tile order in shared memory, then stream out per digit run
#pragma unroll
    for (int i = 0; i < kRadixItems; i++) {
        uint64_t idx = wbase + i * 32 + lane;
        if (idx < n) {
            uint32_t d = (uint32_t)(key[i] >> shift) & dmask;
            s_keys[s_tstart[d] + s_whist[wid][d] + rank[i]] = key[i];
        }
    }
    __syncthreads();
    const uint32_t valid_n = (uint32_t)min((uint64_t)kRadixTile, n - base);
    bool bad = false;
    for (uint32_t j = t; j < valid_n; j += kRadixThreads) {
        unsigned long long k = s_keys[j];
        uint32_t d = (uint32_t)(k >> shift) & dmask;
        unsigned long long pos = s_gofs[d] + (j - s_tstart[d]);
        if (pos < n) dst[pos] = k;
        else bad = true;              // histogram and keys disagree: never write past the buffer
    }
    if (bad) atomicOr(&a.ctrl->flags, CF_EMIT_OVERFLOW);
}

// ------------------------------------------------------------- detection

__device__ __forceinline__ int sorted_parity(const BatchArgs &a)
{
    int before = 0;
    for (uint32_t q = 0; q < a.L.passes; q++) {
        int nz = __syncthreads_count(threadIdx.x < kRadixBins && a.hist[q * kRadixBins + threadIdx.x] != 0);
        before += nz > 1;
    }
    return before & 1;
}

__global__ void __launch_bounds__(kDetectThreads) k_detect(BatchArgs a)
{
    __shared__ unsigned long long s_keys[kDetectTile + 1];
    const unsigned long long *keys = a.keys[sorted_parity(a)];
    const uint64_t n = a.nkeys;
    const uint32_t lo = a.L.sort_lo;
    const uint32_t proto_shift = a.L.sort_bits - a.L.proto_bits;
    const uint32_t tid_mask = a.L.tid_bits ? (1u << a.L.tid_bits) - 1 : 0;
    for (uint64_t base = (uint64_t)blockIdx.x * kDetectTile; base < n; base += (uint64_t)gridDim.x * kDetectTile) {
        const uint32_t valid = (uint32_t)min((uint64_t)kDetectTile, n - base);
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < valid; i += kDetectThreads) s_keys[i + 1] = keys[base + i];
        if (threadIdx.x == 0) s_keys[0] = base ? keys[base - 1] : 0;
        __syncthreads();
        for (uint32_t r = 0; r < kDetectItems; r++) {
            uint32_t i = threadIdx.x * kDetectItems + r;
            if (i >= valid) break;
            unsigned long long k = s_keys[i + 1];
            unsigned long long seg = k >> lo;
            if (base + i > 0 && (s_keys[i] >> lo) == seg) continue;     // not a segment start
            // walk the segment: racy iff it has a write and two distinct tids
            uint32_t first = (uint32_t)(k >> 1) & tid_mask;
            bool writes = k & 1, two = false;
            uint64_t j = base + i + 1;
            while (j < n && !(writes && two)) {
                unsigned long long x = (j - base < valid) ? s_keys[j - base + 1] : __ldg(keys + j);
                if ((x >> lo) != seg) break;
                writes |= x & 1;
                two |= (((uint32_t)(x >> 1) & tid_mask) != first);
                j++;
            }
            if (writes && two) {
                uint32_t proto = a.L.proto_bits ? (uint32_t)(seg >> proto_shift) : 0;
                if (proto < a.nprotos) atomicMin(&a.best_pos[proto], (unsigned long long)(base + i));
            }
        }
    }
}

__device__ __forceinline__ void two_smallest(uint32_t &f, uint32_t &s, uint32_t x)
{
    if (x == f || x == s) return;
    if (x < f) { s = f; f = x; }
    else if (x < s) s = x;
}

// Parity of the buffer holding the sorted keys, computed by one warp.
__device__ __forceinline__ int sorted_parity_warp(const BatchArgs &a)
{
    const uint32_t lane = threadIdx.x & 31;
    int before = 0;
    for (uint32_t q = 0; q < a.L.passes; q++) {
        int nz = 0;
        for (uint32_t d = lane; d < kRadixBins; d += 32) nz += a.hist[q * kRadixBins + d] != 0;
        nz = __reduce_add_sync(kFull, (unsigned)nz);
        before += nz > 1;
    }
    return before & 1;
}

// One warp per protocol: evaluation error, else barrier divergence, else the
// witness of the first racy segment (re-reduced here: the two smallest
// distinct tids of all accesses and of the writes).
__global__ void k_finalize(BatchArgs a)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t p = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (p == 0 && lane == 0 && a.ctrl->total != a.nkeys) atomicOr(&a.ctrl->flags, CF_COUNT_MISMATCH);
    if (p >= a.nprotos) return;
    const DevProto P = a.protos[p];
    const KeyLayout L = a.L;
    DevResult r = {};
    r.verdict = -1;
    r.tuples = a.ptuples[p];
    const unsigned long long ek = a.err_key[p];
    if (ek != kNone) {
        uint32_t tid = (uint32_t)(ek >> 32), k = (uint32_t)ek;
        unsigned long long e = a.erro[P.lane_off + (uint64_t)k * P.nthreads + tid];
        unsigned long long pre = 0;
        for (uint32_t q = lane; q < k; q += 32) pre += a.cnt[P.lane_off + (uint64_t)q * P.nthreads + tid];
        for (int o = 16; o; o >>= 1) pre += __shfl_xor_sync(kFull, pre, o);
        r.status = (e & 0xff) == kErrOob ? -9 : -10;
        r.err_tid = tid;
        r.err_ordinal = pre + (e >> 8);
    } else if (P.nthreads == 0) {
        r.verdict = 0;
        r.phases = 0;
    } else {
        const uint32_t s0 = a.totsyn[P.tid_off];
        r.phases = s0 + 1;
        r.sync_count_0 = s0;
        const uint32_t dt = a.div_tid[p];
        const unsigned long long bp = a.best_pos[p];
        if (dt != 0xFFFFFFFFu) {
            r.verdict = 2;
            r.div_tid = dt;
            r.sync_count_div = a.totsyn[P.tid_off + dt];
        } else if (bp != kNone) {
            const unsigned long long *keys = a.keys[sorted_parity_warp(a)];
            const uint32_t tid_mask = L.tid_bits ? (1u << L.tid_bits) - 1 : 0;
            const unsigned long long seg = keys[bp] >> L.sort_lo;
            uint32_t t0 = 0xFFFFFFFFu, t1 = 0xFFFFFFFFu, w0 = 0xFFFFFFFFu, w1 = 0xFFFFFFFFu;
            for (uint64_t b = bp;; b += 32) {
                uint64_t j = b + lane;
                unsigned long long x = j < a.nkeys ? keys[j] : 0;
                bool in = j < a.nkeys && (x >> L.sort_lo) == seg;
                if (in) {
                    uint32_t tid = (uint32_t)(x >> 1) & tid_mask;
                    two_smallest(t0, t1, tid);
                    if (x & 1) two_smallest(w0, w1, tid);
                }
                if (__ballot_sync(kFull, !in)) break;
            }
            for (int o = 16; o; o >>= 1) {
                uint32_t u0 = __shfl_xor_sync(kFull, t0, o), u1 = __shfl_xor_sync(kFull, t1, o);
                uint32_t v0 = __shfl_xor_sync(kFull, w0, o), v1 = __shfl_xor_sync(kFull, w1, o);
                two_smallest(t0, t1, u0); two_smallest(t0, t1, u1);
                two_smallest(w0, w1, v0); two_smallest(w0, w1, v1);
            }
            r.verdict = 1;
            r.index = seg & (L.idx_bits ? (~0ull >> (64 - L.idx_bits)) : 0);
            r.loc = (uint32_t)((seg >> L.idx_bits) & (L.loc_bits ? (~0ull >> (64 - L.loc_bits)) : 0));
            r.phase = (uint32_t)((seg >> (L.idx_bits + L.loc_bits)) & (L.phase_bits ? (~0ull >> (64 - L.phase_bits)) : 0));
            r.tid_i = t0;
            if (w0 == t0) { r.tid_j = t1; r.i_writes = 1; r.j_writes = (w1 == t1); }
            else { r.tid_j = w0; r.i_writes = 0; r.j_writes = 1; }
        } else {
            r.verdict = 0;
        }
    }
    if (lane == 0) a.results[p] = r;
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

cudaError_t launch_front(const BatchArgs &a, cudaStream_t s, int sms, cudaEvent_t *ev, int *nev)
{
    uint64_t init_n = a.nprotos;
    if (init_n < (uint64_t)kMaxPasses * kRadixBins) init_n = (uint64_t)kMaxPasses * kRadixBins;
    if (init_n < a.nwblocks) init_n = a.nwblocks;
    mark(ev, nev, s);
    k_init<<<(unsigned)((init_n + 255) / 256), 256, 0, s>>>(a);
    mark(ev, nev, s);
    k_interp<false><<<interp_grid(a.nwitems, sms), 256, 0, s>>>(a);
    mark(ev, nev, s);
    uint32_t col_blocks = (uint32_t)((a.ncols + kScanThreads - 1) / kScanThreads);
    k_scan<<<col_blocks + a.nwblocks, kScanThreads, 0, s>>>(a, col_blocks);
    mark(ev, nev, s);
    return cudaGetLastError();
}

cudaError_t launch_back(const BatchArgs &a, cudaStream_t s, int sms, cudaEvent_t *ev, int *nev)
{
    k_interp<true><<<interp_grid(a.nwitems, sms), 256, 0, s>>>(a);
    mark(ev, nev, s);
    for (uint32_t q = 0; q < a.L.passes; q++) {
        if (a.ntiles) k_radix<<<a.ntiles, kRadixThreads, 0, s>>>(a, q);
        mark(ev, nev, s);
    }
    uint64_t dt = (a.nkeys + kDetectTile - 1) / kDetectTile;
    uint64_t cap = (uint64_t)sms * 8;
    if (dt) k_detect<<<(unsigned)(dt < cap ? dt : cap), kDetectThreads, 0, s>>>(a);
    mark(ev, nev, s);
    k_finalize<<<(a.nprotos + 7) / 8, 256, 0, s>>>(a);
    mark(ev, nev, s);
    return cudaGetLastError();
}

int stage_names(const char **names, int cap, uint32_t passes)
{
    static const char *radix[kMaxPasses] = {"radix0", "radix1", "radix2", "radix3",
                                            "radix4", "radix5", "radix6", "radix7"};
    const char *all[4 + kMaxPasses + 2];
    int n = 0;
    all[n++] = "init"; all[n++] = "count"; all[n++] = "scan"; all[n++] = "emit";
    for (uint32_t q = 0; q < passes && q < (uint32_t)kMaxPasses; q++) all[n++] = radix[q];
    all[n++] = "detect"; all[n++] = "finalize";
    for (int i = 0; i < n && i < cap; i++) names[i] = all[i];
    return n;
}

}  // namespace drf
