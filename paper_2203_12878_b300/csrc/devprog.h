// Device program: the form the host lowers a protocol into before the GPU
// interprets it.  Internal to the library (the portable wire format is the
// bytecode of bytecode.cpp); shared by the host lowering and the kernels.
//
// A protocol becomes a flat array of 16-byte instructions (structured
// control flow with explicit jump targets) plus an array of 64-bit
// expression-code words evaluated by a small stack machine.  Parameters are
// folded into constants at lowering time, so a device program is specific to
// one (bytecode, bounds) pair.
//
// Work decomposition: every thread's execution is cut into K "items" that
// run independently -- runs of consecutive statements, single iterations of
// loops (whose bodies are cut further), or chunks of a loop's iterations.
// Items are numbered in program order, so a per-thread exclusive scan of the
// syncs each item executes gives the phase every item starts in.
#pragma once

#ifndef __CUDACC_RTC__
#include <cstdint>
#endif

namespace drf {

constexpr int kMaxVars = 16;        // loop-variable registers (one per nesting depth)
constexpr int kMaxStack = 16;       // expression evaluation stack
constexpr int kMaxPasses = 8;       // radix passes (64 key bits / 8)
constexpr int kRadixBits = 8;       // the widest radix digit (a launch may use narrower ones: KeyLayout::digit_bits)
constexpr int kRadixBins = 1 << kRadixBits;

// ---------------------------------------------------------------- instructions
enum : uint8_t {
    I_END = 0,
    I_ACCESS = 1,    // a: flags (AF_*), b: array, c: index expression
    I_SYNC = 2,
    I_LOOP = 3,      // a: variable register, b: LB_* flags, c: lo expression, d: hi expression, e: pc of the ENDLOOP
    I_ENDLOOP = 4,   // a: variable register, c: first pc of the body
    I_IF = 5,        // c: condition expression, d: pc to continue at when false
    I_JUMP = 6,      // c: target pc
    // An innermost loop whose body holds only accesses and syncs, with every
    // index an affine function of the loop variable (plus a constant
    // remainder / division): a: variable register, b: syncs per iteration (< 256),
    // c: lo expression, d: hi expression, e: number m of I_FASTACC entries
    // that follow.  The count pass takes trip * m accesses in one step.
    I_FASTLOOP = 7,
    // a: AF_WRITE | post kind << 2 (FP_*), b: array, c: expression of the
    // index without its loop-variable term, d: xcode offset of the words
    // [coefficient of the loop variable, post-op constant], e: syncs before
    // this access within one iteration
    I_FASTACC = 8,
};

enum : uint8_t { FP_NONE = 0, FP_MASK = 1, FP_MOD = 2, FP_DIV = 3 };

// I_LOOP flags, set when a batch is packed: LB_RANGE_ONLY -- the loop's body
// holds no sync and no access but range accesses (AF_RANGE), so a launch
// that runs the range pass need not enter it in the table and witness
// passes (its tuples are counted on the host).
enum : uint16_t { LB_RANGE_ONLY = 1 };
constexpr uint32_t kFastMax = 4;    // accesses per fast loop body

enum : uint8_t {
    AF_WRITE = 1,         // access mode: write
    AF_EVAL_IN_COUNT = 2, // the count pass must evaluate the index (it may fail)
    AF_RANGE = 16,        // the range pass applies it (owner-table launches with BatchArgs::range_on)
};

struct Insn {
    uint8_t op;
    uint8_t a;
    uint16_t b;
    int32_t c;
    int32_t d;
    int32_t e;
};
static_assert(sizeof(Insn) == 16, "Insn is 16 bytes");

// ------------------------------------------------------------ expression code
// One 64-bit word per operation: opcode in bits 0..7, operand in bits 8..63.
// X_CONST, X_DIVC, X_MODC and X_MASK take the next word as their constant;
// X_AFF n is followed by n (register, coefficient) word pairs and a constant
// word (register 255 is tid).  Comparisons and connectives push 0 / 1.
enum : uint8_t {
    X_RET = 0, X_CONST, X_TID, X_VAR, X_ADD, X_SUB, X_MUL, X_DIV, X_MOD, X_MIN, X_MAX, X_NEG,
    X_DIVC, X_MODC, X_MASK, X_AFF,
    X_EQ, X_NE, X_LT, X_LE, X_GT, X_GE, X_AND, X_OR, X_NOT,
};
constexpr uint32_t kAffTid = 255;

// ------------------------------------------------------------------ items
// An item fixes the iteration of up to kMaxSplit enclosing loops (the split
// levels, outermost first) and runs the code [start_pc, stop_pc) inside the
// innermost one.  When `chunked` is set, the innermost level is not fixed
// but runs iterations [j*chunk, (j+1)*chunk) of its trip, and the code range
// is that loop's whole body through its ENDLOOP.
constexpr int kMaxSplit = 4;

struct ItemDesc {
    uint32_t start_pc;
    uint32_t stop_pc;
    uint16_t nsplit;
    uint16_t chunked;               // 1: chunk of an I_LOOP, 2: chunk of an I_FASTLOOP (start_pc is the loop)
    uint32_t chunk;
    uint32_t split_pc[kMaxSplit];   // pcs of the split I_LOOP instructions
    uint32_t j[kMaxSplit];          // iteration index (or chunk index, innermost chunked level)
};
static_assert(sizeof(ItemDesc) == 48, "ItemDesc is 48 bytes");

// ------------------------------------------------------------ batch layout
struct DevProto {
    uint32_t insn_off;     // into the batch instruction array
    uint32_t xcode_off;    // into the batch expression-code array
    uint32_t item_off;     // into the batch item array
    uint32_t nitems;       // K
    uint32_t nthreads;     // T
    uint32_t wide;         // 1: 64-bit arithmetic, 0: 32-bit
    uint32_t nlocs;
    uint32_t cells_off;    // into the batch array-size array
    uint64_t lane_off;     // per-(item, thread) arrays: lane_off + k * T + t
    uint64_t tid_off;      // per-thread arrays: tid_off + t
    // owner table: phase-major rows of cells_sum records, array after array
    uint64_t tab_off;      // first record of this protocol
    uint64_t cells_sum;    // records per phase row (sum of the array sizes)
    uint32_t tab_phases;   // rows: the static bound on syncs per thread, plus one
    uint32_t flags;        // DP_* below
};

enum : uint32_t {
    // every thread runs the same syncs (tab_phases - 1 of them) and no
    // evaluation can fail; the batch's item-phase array holds, per item, the
    // phase at its start
    DP_STATIC = 1,
};

struct WarpItem {
    uint32_t proto;
    uint32_t k;            // item index within the protocol
    uint32_t g;            // thread group: threads 32g .. 32g+31
};

// Access key: ((((proto | phase) | loc) | index) | tid) | mode, most
// significant field first.  The fields above tid form the sort key.
struct KeyLayout {
    uint32_t tid_bits;
    uint32_t idx_bits;
    uint32_t loc_bits;
    uint32_t phase_bits;
    uint32_t proto_bits;
    uint32_t sort_lo;      // first sort bit = tid_bits + 1
    uint32_t sort_bits;    // idx + loc + phase + proto bits
    uint32_t passes;       // ceil(sort_bits / digit_bits), at most kMaxPasses
    uint32_t digit_bits;   // radix digit width, 4..kRadixBits
};

// Per-launch control block (cleared by the init kernel).
struct Control {
    unsigned long long tile_counter[kMaxPasses];
    unsigned long long total;          // access tuples of the launch
    unsigned int detect_tiles;
    unsigned int flags;                // CF_* internal failures
    unsigned long long touched;        // owner-table blocks listed this launch
    unsigned int blocks_done;          // blocks of the witness pass that have finished
    unsigned int range_next;           // range pass: tasks handed out so far
    unsigned long long range_tuples;   // access tuples the range pass applied
};

enum : unsigned {
    CF_LOOKBACK_TIMEOUT = 1,   // a radix pass gave up waiting on a predecessor tile
    CF_EMIT_OVERFLOW = 2,      // emission disagreed with the count pass
    CF_COUNT_MISMATCH = 4,     // the launch's tuple total differs from the plan's
    CF_TABLE_RANGE = 8,        // an access fell outside its protocol's owner-table rows
};

// Device-side result of one protocol (converted to drf_result on the host).
struct DevResult {
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
};

}  // namespace drf
