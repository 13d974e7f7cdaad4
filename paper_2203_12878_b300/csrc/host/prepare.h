// Host-side preparation of one protocol for the device pipeline: decode and
// validate the bytecode, check the bounds, run interval analysis, lower to a
// device program and cut each thread's execution into items.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../devprog.h"
#include "ast.h"

namespace drf {

struct PrepareOpts {
    // scheduling: desired warp-items for the whole launch, and the least
    // interpreter steps per lane an item should carry
    uint64_t desired_warp_items = 148 * 128;
    uint64_t min_item_steps = 64;
    uint64_t min_short_item_steps = 4;   // items of a small protocol (cut for parallelism)
    uint32_t max_items = 1u << 14;
};

// An access the owner table's range pass can apply cell by cell: it runs in
// one phase (no enclosing loop holds a sync), its enclosing loops' bounds
// and conditions do not read tid, and its index is (sigma * tid + c) or
// (sigma * tid + c) mod modn with sigma an integer of magnitude at most
// kRangeMaxSigma (0: one cell for every thread) and c a function of the loop
// variables alone (with a remainder, (T - 1) * |sigma| < kRangeMaxWraps *
// modn).  The threads that reach a given range of cells in one iteration
// are then a few runs of consecutive tids (one per wrap of the index around
// the modulus), their cells sigma apart, found without visiting the others.
constexpr int32_t kRangeMaxSigma = 64;
constexpr int32_t kRangeMaxWraps = 64;
struct RangeLoop {
    uint32_t reg;                 // the loop variable's register
    int32_t lo, hi;               // expression code of the bounds
    uint64_t trip_max;            // trip count bound over all outer iterations
};
struct RangeAccess {
    uint32_t pc;                  // its I_ACCESS or I_FASTACC instruction
    uint32_t phase, loc;
    bool write;
    int32_t sigma;                // tid's coefficient, |sigma| <= kRangeMaxSigma
    uint64_t modn;                // 0: no remainder; else the index is a Euclidean remainder by modn
    int32_t cexpr;                // expression code of the index before the remainder, at tid = 0
    std::vector<RangeLoop> loops; // enclosing loops, outermost first
    std::vector<std::pair<int32_t, bool>> guards;   // enclosing conditions' code and the branch taken
    uint64_t iters;               // product of the loops' trip bounds (saturated)
    // found by evaluating the loops at preparation: the distinct offsets c
    // (reduced mod modn when there is a remainder) and the iterations run
    std::vector<int64_t> offsets;
    uint64_t run_iters = 0;
};

// Loop iterations preparation evaluates to find range accesses' offsets,
// over all of one protocol's range accesses.
constexpr uint64_t kRangeIterCap = 1ull << 22;

// Expression code (devprog.h's stack machine) evaluated on the host over
// mathematical integers; false on a division by zero, a value outside int64
// or malformed code.
bool host_eval(const std::vector<uint64_t> &xc, int32_t off, int64_t tid, const int64_t *vars, int64_t &out);
// The distinct offsets of a range access over its loops' iterations (its
// conditions applied) and the iterations it runs; false when an evaluation
// fails or more than `cap` iterations would be visited.
bool range_offsets(const std::vector<uint64_t> &xcode, const RangeAccess &r, uint64_t cap, std::vector<int64_t> &cs,
                   uint64_t &iters);

struct Prepared {
    uint32_t nthreads = 0;
    uint32_t narrays = 0;
    std::vector<uint64_t> cells;
    bool wide = false;                // needs 64-bit arithmetic
    uint64_t max_syncs = 0;           // per thread, upper bound
    uint64_t max_tuples = 0;          // per thread, upper bound
    uint64_t max_steps = 0;           // interpreter steps per thread, upper bound
    std::vector<Insn> insns;
    std::vector<uint64_t> xcode;
    std::vector<ItemDesc> items;
    std::vector<uint64_t> item_steps; // per item, upper bound of steps per lane
    // Set when every thread runs the same sync structure and no evaluation
    // can fail; item_phase then holds, per item, the phase at its start.
    bool static_phases = false;
    std::vector<uint32_t> item_phase;
    // With static phases: the accesses the range pass can take (see RangeAccess)
    std::vector<RangeAccess> range_access;

    uint64_t tuple_bound() const { return (uint64_t)nthreads * max_tuples; }
};

// bounds: thread count, array sizes and parameter values (validated here).
Error prepare(const uint8_t *bc, size_t len, uint32_t nthreads, uint32_t nlocs, const uint64_t *cells,
              uint32_t nparams, const int64_t *params, const PrepareOpts &opts, Prepared &out);

// Number of bits needed for values 0 .. x.
inline uint32_t bits_for(uint64_t x)
{
    uint32_t b = 0;
    while (b < 64 && (x >> b) != 0) b++;
    return b;
}

// Limits on the amount of work one check may ask for.
constexpr uint64_t kMaxTupleBound = 1ull << 36;    // access tuples, all threads
constexpr uint64_t kMaxStepBound = 1ull << 42;     // interpreter steps, all threads

}  // namespace drf
