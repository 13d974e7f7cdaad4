// Device pipeline of the checker: argument block and host-side launchers.
#pragma once

#include <cuda_runtime.h>

#include "../batch_args.h"

namespace drf {

// Keys per thread of a radix tile: a tuning choice among these (0 = 16).
inline uint32_t radix_items_or_default(uint32_t items) { return items == 12 || items == 24 ? items : 16; }
inline uint32_t radix_tiles(uint64_t n, uint32_t items = kRadixItems)
{
    const uint64_t tile = (uint64_t)kRadixThreads * radix_items_or_default(items);
    return (uint32_t)((n + tile - 1) / tile);
}
inline uint32_t detect_tiles(uint64_t n) { return (uint32_t)((n + kDetectTile - 1) / kDetectTile); }

// Kernels specialized to one protocol at run time (host/jit.h), launched in
// place of the interpreter's count, table and witness passes when set; all
// take (BatchArgs, const uint16_t *item_shape).
struct JitLaunch {
    const void *count = nullptr, *table = nullptr, *cell = nullptr;
    const uint16_t *shape = nullptr;   // device: per item, its code shape
    // The kernels take every item's phase as a constant and the table pass
    // counts the tuples: the count and scan passes are left out.
    bool static_phases = false;
    // The warp-item schedule is compiled in: the kernels do not read the
    // batch's warp-item array.
    bool csched = false;
    // The table kernel leaves the batch's range accesses to the range pass:
    // launches need BatchArgs::range_on.
    bool range = false;
};

// Stage launchers (all asynchronous on `s`).  Each returns cudaGetLastError().
// When ev is non-null, an event is recorded before the first kernel of
// launch_front and after every kernel; *nev counts the events recorded.
cudaError_t launch_front(const BatchArgs &a, cudaStream_t s, int sms, cudaEvent_t *ev, int *nev,
                         const JitLaunch *j = nullptr);   // init, count, scan
// PATH_SORT: emit, radix, detect, finalize.  PATH_TABLE: table, tscan, witness, finalize.
cudaError_t launch_back(const BatchArgs &a, cudaStream_t s, int sms, cudaEvent_t *ev, int *nev,
                        const JitLaunch *j = nullptr);

// Names of the stages whose boundaries launch_front / launch_back record.
// static_phases: the launch leaves the count and scan passes out (JitLaunch).
// count_free: an interpreted owner-table launch without them (BatchArgs::count_free).
// range: the launch runs the range pass (before the table scan).
int stage_names(const char **names, int cap, uint32_t passes, uint32_t path, bool static_phases = false,
                bool count_free = false, bool range = false);
constexpr int kMaxStages = 4 + kMaxPasses + 2;

}  // namespace drf
