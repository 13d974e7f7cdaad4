// Run-time specialization of the owner-table back end to one protocol.
//
// The interpreter kernels execute a protocol's lowered program (devprog.h)
// instruction by instruction.  For a plan over a single protocol the same
// program can be translated to straight CUDA C -- loops as loops, every
// coefficient, array size and table stride a constant, the loop variables
// in registers -- compiled for sm_103a with NVRTC and loaded as a library.
// The generated count, table and witness kernels replace the interpreter's
// for those passes and compute exactly what it computes: the translation is
// instruction by instruction over the same lowered program and the same item
// decomposition.  NVRTC is loaded on first use; without it (or when a
// protocol's program is too large to specialize) plans keep the interpreter.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../cuda/pipeline.cuh"
#include "prepare.h"

namespace drf {

struct BatchHost;

// CUDA source of the specialized kernels of protocol 0 of `b` (a batch of
// one protocol prepared as `p`); item_shape receives, per item, the index
// of the code shape its kernels dispatch on.  *static_phases (when not null)
// is set when the kernels take every item's phase as a constant
// (Prepared::static_phases): the table pass then needs neither the count
// nor the scan pass, and counts the tuples itself.  *compiled_schedule (when
// not null) is set when the warp-item schedule is compiled in: the kernels
// then read neither the batch's warp-item array nor its item descriptors.
// `b` must hold its expanded warp-item array.
// *range_pass (when not null) is set when the batch's range pass (pack_batch,
// plan_range) takes some of the protocol's accesses: the generated table
// pass only counts those, the precompiled range pass applies them.
Error jit_source(const Prepared &p, const BatchHost &b, std::string &src, std::vector<uint16_t> &item_shape,
                 bool *static_phases = nullptr, bool *compiled_schedule = nullptr, bool *range_pass = nullptr);

// Compiles `src` for sm_103a with NVRTC.  On failure, `log` holds the
// compiler's log (or why NVRTC is unavailable).
Error jit_compile(const std::string &src, std::vector<char> &cubin, std::string &log);

// The loaded kernels of one specialized protocol.
struct JitModule {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t count = nullptr, table = nullptr, cell = nullptr;
    JitModule() = default;
    JitModule(const JitModule &) = delete;
    JitModule &operator=(const JitModule &) = delete;
    ~JitModule();
};

Error jit_load(const std::vector<char> &cubin, JitModule &m);

}  // namespace drf
