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
