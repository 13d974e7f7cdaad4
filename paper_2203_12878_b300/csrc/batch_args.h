// Argument block of the device pipeline and the layout constants its
// kernels share.  Plain data only: included by the host code, the CUDA
// sources and, as text, by the per-protocol kernels compiled at run time.
#pragma once

#include "devprog.h"

namespace drf {

// Summary of a contiguous piece of one segment of equal sort keys, and the
// per-tile record of the pieces that touch a detection tile's edges.
struct Agg {
    uint32_t mint, maxt;
    uint32_t bits;              // 1: any write, 2: holds the segment head, 4: non-empty
    unsigned long long start;   // sorted position of the head (valid with bit 2)
};

struct TileRec {
    unsigned long long first_seg, last_seg;   // sort keys of the tile's first and last key
    Agg first;                                // in-tile piece of the segment continuing from the previous tile
    Agg last;                                 // the tile's last segment piece, when it continues into the next tile
    uint32_t flags;                           // TR_*
    uint32_t pad;
};

enum : uint32_t {
    TR_STARTS_CONT = 1,   // the tile's first key continues a segment of the previous tile
    TR_ENDS_CONT = 2,     // the tile's last segment continues into the next tile
    TR_SINGLE = 4,        // the tile lies inside one segment that crosses both edges
};

// One piece of the range pass's work: the threads t0 .. t0 + len - 1 of
// one range access at one offset, whose records (relative to the first
// record of their task) are l0, l0 + step, l0 + 2 step, ... (step: the
// access's tid coefficient; 0 -- every thread at l0 -- only among the
// pieces as cut, never among the merged ones), and whether they write (kRWrite);
// lenf holds len and the flags.  With kRSat the piece stands for records
// that two or more different threads reach: each gets the "second thread"
// bit (and "written" with kRWrite), and t0 is unused.
struct RPiece {
    uint32_t t0, lenf;
    int32_t l0, step;
};
constexpr uint32_t kRSat = 1u << 31, kRWrite = 1u << 30, kRLen = (1u << 30) - 1;

// A task of the range pass: its index (its records start at task *
// kRangeRecs), its pieces [p0, p1), and the part of its records this entry
// covers, in blocks of 256 records: [win & 0xFFFF, win >> 16) (a task with
// much work is split into several entries over disjoint parts, each taken
// by its own block).
struct RTask {
    uint32_t task, p0, p1, win;
};

// One range piece's keys on the sort path: its o-th thread's key is
// k0 + o * d (modulo 2^64: the index field steps by the piece's step and
// the thread field by one, neither leaving its field), at key position
// pre + o of the range keys, for o < len.
struct RKeys {
    unsigned long long pre, k0, d, len;
};

#if defined(__CUDACC__)
#define DRF_HD __host__ __device__
#else
#define DRF_HD
#endif

// Floor of x / d for d > 0.
DRF_HD inline long long range_floordiv(long long x, long long d) { return x >= 0 ? x / d : -((-x + d - 1) / d); }

// The part of a piece (threads t0 + o, o < len, at records l0 + step * o;
// step 0: every thread at l0) whose records lie in [w0, w1): its first
// thread, first record and length (0 when none).
DRF_HD inline void range_clip(long long t0, long long l0, long long len, long long step, long long w0, long long w1,
                              long long &ct0, long long &cl0, long long &clen)
{
    long long olo, ohi;                           // w0 <= l0 + step * o < w1
    if (step == 0) {
        olo = 0;
        ohi = l0 >= w0 && l0 < w1 ? len : 0;
    } else if (step > 0) {
        olo = range_floordiv(w0 - l0 + step - 1, step);
        ohi = range_floordiv(w1 - l0 + step - 1, step);
    } else {
        const long long b = -step;
        olo = range_floordiv(l0 - w1, b) + 1;
        ohi = range_floordiv(l0 - w0, b) + 1;
    }
    if (olo < 0) olo = 0;
    if (ohi > len) ohi = len;
    if (olo >= ohi) { ct0 = t0; cl0 = l0; clen = 0; return; }
    ct0 = t0 + olo;
    cl0 = l0 + step * olo;
    clen = ohi - olo;
}

// Owner records per task of the range pass: a multiple of the 8,192 records
// one touch word covers, so that every task owns its touch words.
constexpr uint32_t kRangeRecs = 16384;
constexpr uint32_t kRangeThreads = 512;
constexpr uint32_t kRangeChunk = 512;                       // pieces applied per round
constexpr uint32_t kRangeSmem = kRangeRecs * 4;             // dynamic shared memory of a range block
constexpr uint32_t kRangeBlocksPerSm = 3;

// Everything the kernels of one launch touch.  Device pointers unless noted.
struct BatchArgs {
    // device programs of the batch
    const Insn *insns;
    const uint64_t *xcode;
    const ItemDesc *items;
    const DevProto *protos;
    const uint64_t *cells;
    const WarpItem *witems;
    const uint32_t *iphase;          // per item (item_off + k): its start phase when the protocol is DP_STATIC
    uint32_t nwitems;
    uint32_t nprotos;
    uint32_t has_narrow, has_wide;   // protocols with 32-bit / 64-bit arithmetic present
    uint64_t ncols;                  // sum of thread counts (per-thread arrays)
    // per (item, thread)
    uint32_t *cnt;                   // accesses
    uint32_t *syn;                   // syncs
    uint32_t *phs;                   // phase at item start (exclusive scan of syn)
    unsigned long long *erro;        // (local ordinal << 8) | error code
    // per (protocol, thread)
    uint32_t *totsyn;
    // per warp-item
    uint32_t *wcnt;
    unsigned long long *wbase;
    unsigned long long *blocksum;    // per 4096 warp-items
    uint32_t nwblocks;
    // keys
    unsigned long long *keys[2];
    uint64_t nkeys;                  // tuples this launch must produce (plan size)
    unsigned long long *hist;        // [kMaxPasses][kRadixBins]
    unsigned long long *status;      // [passes][ntiles][kRadixBins] look-back words
    uint32_t ntiles;
    uint32_t radix_items;            // keys per thread of a radix tile (12, 16 or 24; 0 = 16)
    uint32_t stall_lookback;         // test hook: radix passes leave tile 0's status out and wait briefly
    TileRec *trec;                   // [ndtiles] detection tile records
    uint32_t ndtiles;
    // per protocol
    unsigned long long *err_key;     // min (tid << 32 | item) with an evaluation error
    uint32_t *div_tid;               // min tid whose sync count differs from thread 0's
    unsigned long long *best_pos;    // min sorted position of a racy segment
    unsigned long long *ptuples;
    DevResult *results;
    Control *ctrl;
    uint32_t *epoch;                 // persists across launches
    KeyLayout L;
    // owner table (the sort-free path): one record per (protocol, phase,
    // array, index) cell, all zero between launches
    uint32_t path;                   // PATH_SORT or PATH_TABLE
    // Owner-table launches of a batch whose protocols are all DP_STATIC: no
    // count or scan pass; the interpreted passes take item phases from
    // `iphase`, the table pass counts the tuples and writes thread 0's sync
    // total, and nothing checks barrier divergence (none is possible).
    uint32_t count_free;
    // Shard of a one-protocol check (drf_check_shard): the table and range
    // passes update only the records at positions [shard_lo, shard_hi);
    // [0, ~0) otherwise.
    unsigned long long shard_lo, shard_hi;
    // The range pass (owner-table launches): tasks of kRangeRecs records
    // that range accesses reach (rlive, ascending), each with its pieces as
    // cut [rfirst[i], rfirst[i + 1]) of wpiece (what the witness search
    // reads); rtask, the same tasks (or parts of them) in the order blocks
    // take them (most record updates first), each with its merged pieces
    // [p0, p1) of rpiece (what the range pass applies).  The table pass
    // leaves accesses marked AF_RANGE alone when range_on is set.
    const RPiece *rpiece;
    const RPiece *wpiece;
    const RTask *rtask;
    const uint32_t *rlive;
    const uint32_t *rfirst;
    uint32_t nlive;
    uint32_t nrtask;                // entries of rtask (nlive or more: parts of split tasks)
    // per protocol, the access tuples of its range accesses (host-counted);
    // with rcount set the table pass counts only the other accesses and
    // these are added (k_init per protocol, k_range the launch's rtotal)
    const unsigned long long *rtup;
    unsigned long long rtotal;
    uint32_t rcount;
    // The sort path with the range pieces (range_keys): the count and emit
    // passes leave the range accesses out, and k_range_emit writes one key
    // per (piece as cut, thread) -- nrkeys keys from position
    // nkeys - nrkeys on, wkeys[0 .. nwkeys) in key order -- with their
    // digit histograms.
    const RKeys *wkeys;
    unsigned long long nrkeys;
    uint32_t nwkeys;
    uint32_t range_keys;
    uint32_t range_on;
    void *table;                     // [tab_cells] 32-bit owner records, padded to whole blocks
    uint64_t tab_cells;
    uint32_t *touch;                 // one bit per block of kTabBlock records written this launch
    uint32_t *tlist;                 // [table blocks] the touched blocks, in the order first touched
    const uint64_t *cbase;           // per (protocol, array): first record of the array in a phase row
    uint32_t *hit_acc, *hit_wr;      // per (protocol, thread) bit: accessed / wrote the witness cell
    uint64_t nhit;                   // words of each hit array
};

enum : uint32_t { PATH_SORT = 0, PATH_TABLE = 1 };

// BatchArgs::nkeys of a launch whose tuple count is not known in advance
// (no sizing run); the finalize kernel then skips its count check.
constexpr unsigned long long kUncounted = ~0ull;

constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 16;
constexpr int kRadixTile = kRadixThreads * kRadixItems;     // 4096 keys
constexpr int kDetectThreads = 256;
constexpr int kDetectItems = 16;
constexpr int kDetectTile = kDetectThreads * kDetectItems;  // 4096 keys
constexpr int kFinalizeThreads = 128;
constexpr int kFinalizeWideThreads = 1024;   // finalize blocks of a batch of at most kFinalizeWideProtos
constexpr uint32_t kFinalizeWideProtos = 16;
constexpr int kScanThreads = 256;
constexpr int kWScanPerBlock = 4096;                        // warp-items per scan block
constexpr int kTabBlockLog = 8;
constexpr int kTabBlock = 1 << kTabBlockLog;                // owner-table records per touch bit
constexpr int kTabScanThreads = 256;

// Owner-table blocks and touch-bitmap words for `cells` records.
#if defined(__CUDACC__) || defined(__CUDACC_RTC__)
#define DRF_HOST_DEVICE __host__ __device__
#else
#define DRF_HOST_DEVICE
#endif
DRF_HOST_DEVICE inline uint64_t table_blocks(uint64_t cells) { return (cells + kTabBlock - 1) / kTabBlock; }
DRF_HOST_DEVICE inline uint64_t touch_words(uint64_t cells) { return (table_blocks(cells) + 31) / 32; }

}  // namespace drf
