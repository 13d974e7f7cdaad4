// Host engine: packs prepared protocols into a device batch, owns device
// buffers, and runs the pipeline (directly or as a captured CUDA graph).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../../include/drf.h"
#include "../cuda/pipeline.cuh"
#include "jit.h"
#include "prepare.h"
#include "tune.h"

namespace drf {

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    // bumped by every allocation and release: memory that must start out
    // zero is cleared when this changes (a new allocation can come back at
    // the address just freed, so the address says nothing)
    uint64_t gen = 0;
};

// Grow-only device allocation; returns false on failure.
bool ensure(DevBuf &b, size_t bytes, size_t *in_use, uint64_t limit);
void release(DevBuf &b, size_t *in_use);

// Host image of a batch.
struct BatchHost {
    std::vector<Insn> insns;
    std::vector<uint64_t> xcode;
    std::vector<ItemDesc> items;
    std::vector<DevProto> protos;
    std::vector<uint64_t> cells;
    std::vector<uint64_t> cbase;     // per (protocol, array): offset of the array within a table row
    // the warp-item schedule: runs of (protocol, item, its thread groups),
    // longest items first; `witems` is its expansion into one entry per
    // warp item, made only when a kernel reads it (expand_witems)
    struct Run { uint32_t proto, k, groups; };
    std::vector<Run> runs;
    uint64_t nwitems = 0;
    std::vector<WarpItem> witems;
    bool expanded() const { return witems.size() == nwitems; }
    void expand_witems();
    // a number no other image content had (process-wide), renewed whenever
    // the image changes: a device batch that staged this version need not
    // stage it again
    uint64_t version = 0;
    void renew();
    uint64_t ncols = 0;
    uint64_t lanes = 0;
    uint64_t tuple_bound = 0;
    KeyLayout L{};
    uint64_t table_cells = 0;        // owner-table records of the whole batch
    bool table_ok = false;           // the owner-table path can run this batch
    // per item (batch order): its start phase for DP_STATIC protocols, else 0
    std::vector<uint32_t> iphase;
    // every protocol is DP_STATIC: owner-table launches may leave the count
    // and scan passes out (BatchArgs::count_free)
    bool all_static = false;
    // the range pass's work (BatchArgs::rpiece ..): per task of kRangeRecs
    // owner records that range accesses reach (rlive, ascending) its pieces
    // as cut [rfirst[i], rfirst[i + 1]) of wpiece, and the tasks again (or
    // their parts) in the order blocks take them (rtask: most record updates
    // first) with their merged pieces in rpiece; the accesses' instructions
    // carry AF_RANGE in `insns`.  range_pcs: per protocol, the pcs (in its
    // own program) of its range accesses; range_tuples: the access tuples
    // they make.
    std::vector<RPiece> rpiece, wpiece;
    std::vector<RTask> rtask;
    std::vector<uint32_t> rlive, rfirst;
    std::vector<std::vector<uint32_t>> range_pcs;
    uint64_t range_tuples = 0;
    std::vector<unsigned long long> rtup;      // per protocol: the tuples of its range accesses
    // the sort path's keys of the range accesses: per piece as cut, its
    // keys' position, first key and step, and their total
    std::vector<RKeys> wkeys;
    uint64_t nrkeys = 0;
    uint64_t table_bytes() const { return table_cells * 4; }   // one 32-bit owner record per cell
};

// Largest owner table (bytes) the library sets up for one batch.
constexpr uint64_t kMaxTableBytes = 64ull << 30;

// Packs prepared protocols (all valid) into a batch; fails with
// S_KEY_TOO_WIDE when the combined key layout exceeds 64 bits.  digit_bits:
// the sort path's radix digit width (4..8; 0 = 8).
constexpr uint64_t kRangeMinTuples = 1ull << 22;   // default: a batch's range tuples below this, no range pass
Error pack_batch(const std::vector<const Prepared *> &ps, BatchHost &out, bool expand = true,
                 uint32_t digit_bits = 0, uint64_t range_min = kRangeMinTuples);

// The range pass's work of a packed batch (BatchHost::rpiece ..): the
// range accesses (Prepared::range_access) of every protocol with static
// phases whose range accesses make a quarter of its tuples or more, each
// offset's threads cut into pieces at the boundaries of the tasks of owner
// records their cells fall into, and AF_RANGE set on their instructions.
// Called by pack_batch; a batch without an owner table gets none.
void plan_range(const std::vector<const Prepared *> &ps, BatchHost &out, uint64_t range_min);
constexpr size_t kRangeMaxEntries = 1u << 24;                // pieces of a batch at most
constexpr uint64_t kRangeSplitWork = 1u << 15;               // record updates per part of a task

// Offset of the results after the control block in a batch's report.
constexpr size_t kOutResults = 128;
static_assert(sizeof(Control) <= kOutResults, "control block fits before the results");

// Device buffers of one batch (a plan owns one; a context reuses one).
struct DeviceBatch {
    // the batch's host image (program, items, protocols, array sizes, table
    // bases, warp items): one device arena, filled by one copy from `stage`
    DevBuf image;
    void *stage = nullptr;            // pinned host staging buffer of the image
    size_t stage_cap = 0;
    cudaEvent_t staged = nullptr;     // recorded after the copy out of `stage`
    bool staged_pending = false;
    uint64_t staged_version = 0;      // BatchHost::version the stage holds (0: none)
    bool staged_schedule = false;     // ... and whether with the warp-item array
    bool staged_keys = false;         // ... and whether with the range pieces' key templates
    DevBuf cnt, syn, phs, erro, totsyn, wcnt, wbase, blocksum;
    DevBuf keys0, keys1, hist, status, trec;
    DevBuf err_key, div_tid, best_pos, ptuples, epoch;
    DevBuf table, touch, tlist, hit, ishape;
    // what a launch reports: the control block, then one result per
    // protocol, read back by one copy into a pinned mirror
    DevBuf out;
    void *out_host = nullptr;
    size_t out_host_cap = 0;
    size_t in_use = 0;
    uint64_t limit = 0;
    uint64_t status_launches = 0;     // launches since the look-back words were cleared
    uint64_t h2d_bytes = 0, d2h_bytes = 0;   // copies of the last run
    uint32_t radix_items = 16;                // radix tile shape (tuning choice)
    int path_pref = 0;                        // 0: choose per batch, 1: sort path, 2: owner-table path
    bool table_dirty = false;                 // a failed launch may have left records behind
    uint32_t stall_lookback = 0;              // test hook: launches left whose radix look-back stalls
    // drf_check_shard: the owner-table positions the launches update
    unsigned long long shard_lo = 0, shard_hi = ~0ull;
    JitLaunch jit{};                          // specialized kernels (plans over one protocol)
    BatchArgs args{};

    ~DeviceBatch();
    Control *host_ctrl() const { return (Control *)out_host; }
    const DevResult *host_results() const { return (const DevResult *)((const char *)out_host + kOutResults); }
    // Queues the copy of the control block (ctrl_only) or of the control
    // block and every result into the pinned mirror.
    cudaError_t fetch(cudaStream_t s, bool ctrl_only);
    // Uploads the batch and sizes every buffer that does not depend on the
    // tuple count.
    // schedule false: the warp-item array is left out (kernels with the
    // schedule compiled in do not read it)
    Error load(const BatchHost &b, cudaStream_t s, bool schedule = true);
    // Sizes the key and look-back buffers for n tuples (sort path).
    Error size_keys(uint64_t n, cudaStream_t s);
    // Sizes the owner table, its touch bits and the witness hit bits
    // (owner-table path); a new or grown table is cleared once.
    Error size_table(const BatchHost &b, uint64_t n, cudaStream_t s);
    // Picks the back end for a batch of n tuples (after the count pass) and
    // sizes its buffers.  Falls back to the sort path when the table
    // cannot be allocated, unless the table path was asked for.
    Error choose_path(const BatchHost &b, uint64_t n, cudaStream_t s);
};

// The back end the automatic choice takes for a batch of n tuples.
uint32_t auto_path(const BatchHost &b, uint64_t n);

// Kernels specialized to one protocol under one set of bounds, kept by a
// context for its later checks of the same protocol (DRF_OPT_SPECIALIZE).
struct JitEntry {
    std::unique_ptr<JitModule> mod;   // null: the protocol could not be specialized
    JitLaunch launch{};
    void *shape = nullptr;            // device: per item, its code shape
    JitEntry() = default;
    JitEntry(const JitEntry &) = delete;
    JitEntry &operator=(const JitEntry &) = delete;
    ~JitEntry();
};

// Prepared protocols of earlier checks, keyed by the bytecode, the bounds
// and the preparation options (a check of a protocol seen before skips
// validation, interval analysis, lowering and the item cut).  Thread-safe;
// at most kCap entries, then it starts over.
class PrepCache {
public:
    std::shared_ptr<const Prepared> get(const uint8_t *bc, size_t len, const drf_bounds *b, const PrepareOpts &po,
                                        Error &err);

private:
    static constexpr size_t kCap = 4096;
    std::mutex mu_;
    std::unordered_map<std::string, std::shared_ptr<const Prepared>> map_;
};

struct Timing;

}  // namespace drf

struct drf_ctx {
    int device = 0;
    int sms = 148;
    cudaStream_t stream = nullptr;
    drf_opts opts{};
    std::string last_error;
    drf::DeviceBatch work;            // reused by drf_check / drf_check_batch
    drf::BatchHost host;              // host image of the last batch (its vectors keep their capacity)
    void *server = nullptr;           // drf::Server when running
    std::mutex mu;                    // guards `work` between the caller and the server thread
    // specialized kernels of protocols checked before, keyed by bytecode and
    // bounds (DRF_OPT_SPECIALIZE; at most kJitCacheEntries, then cleared)
    std::map<std::string, std::unique_ptr<drf::JitEntry>> jit_cache;
    drf::PrepCache prep_cache;        // prepared protocols of earlier checks and server requests
    // `host` holds the pack of this prepared protocol under this radix digit
    // width (a check of the protocol packed just before reuses it)
    std::shared_ptr<const drf::Prepared> host_of;
    uint32_t host_digit_bits = 0;
};

struct drf_plan {
    drf_ctx *ctx = nullptr;
    uint32_t n = 0;
    drf::BatchHost host;
    drf::DeviceBatch dev;
    uint64_t tuples = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t last_stream = nullptr;
    std::vector<cudaEvent_t> events;
    int nevents = 0;
    bool profiled = false;
    drf::PlanConfig cfg;
    std::unique_ptr<drf::JitModule> jit;   // specialized kernels, when the plan uses them
    std::string jit_log;                   // why specialization was not used, when asked for
};

namespace drf {

// Runs one batch on the buffers `w`: front, size, back; results into `out`
// (one per packed protocol).  Returns a batch-level status; `err` gets a
// message.
int run_batch(DeviceBatch &w, int sms, cudaStream_t s, const BatchHost &b, std::vector<DevResult> &out,
              std::string &err);
int run_batch(drf_ctx *ctx, const BatchHost &b, cudaStream_t s, std::vector<DevResult> &out);

// One protocol on the context's buffers with kernels specialized to it:
// the owner-table path, front and back in one go (one wait).  A non-zero
// return other than a CUDA failure means the caller may run the
// interpreter instead.
int run_batch_jit(drf_ctx *ctx, const BatchHost &b, const JitLaunch &j, cudaStream_t s, std::vector<DevResult> &out);

constexpr size_t kJitCacheEntries = 32;
// drf_check specializes only protocols that may make this many accesses: a
// smaller check takes well under a millisecond interpreted, far less than
// the compile (0.1 - 1 s) would cost it the first time.
constexpr uint64_t kJitMinTuples = 1ull << 21;

// Back-end preference of a context's options: 0 automatic, 1 sort, 2 owner table.
int path_pref_of(const drf_opts &o);
// Fewest range-pass tuples a batch needs to take the pass under these options.
uint64_t range_min_of(const drf_opts &o);
// The same for a batch of several protocols checked once (drf_check_batch,
// the server's rounds): none without DRF_OPT_RANGE_ANY.
uint64_t range_min_once(const drf_opts &o);

void to_public(const DevResult &d, drf_result *out);

}  // namespace drf
