// Autotuning of a plan's launch configuration and its cache.
#pragma once

#include <cstdint>
#include <string>

namespace drf {

// A plan's tunable launch configuration.
struct PlanConfig {
    uint32_t granularity = 128;   // desired warp-items per SM for the whole batch (item-to-warp schedule)
    uint32_t radix_items = 16;    // keys per thread of a radix tile (12, 16 or 24)
    uint32_t path = 0;            // back end: 0 the context's choice, 1 sort, 2 owner table
    uint32_t jit = 0;             // 1: kernels specialized to the (single) protocol
    uint32_t radix_bits = 0;      // sort path: radix digit width (4..8); 0 = the context's choice
};

// Digit widths the tuner tries on the fastest sort-path configuration.
constexpr uint32_t kTuneRadixBits[] = {6, 7};

// Candidate configurations the tuner times.
constexpr uint32_t kTuneGranularity[] = {32, 128, 512};
constexpr uint32_t kTuneRadixItems[] = {12, 16, 24};
constexpr int kTuneReps = 15;                 // timed launches per candidate (median)

// Process-wide cache of tuned configurations, keyed by a workload signature;
// when DRF_TUNE_CACHE names a file the cache is loaded from it once and
// every new entry is appended to it.
bool tune_lookup(const std::string &key, PlanConfig &out);
void tune_store(const std::string &key, const PlanConfig &cfg, double ms);

}  // namespace drf
