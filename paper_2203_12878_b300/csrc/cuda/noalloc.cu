// drf_check_noalloc: the whole check without any device allocation.
//
// Some callers cannot call cudaMalloc at the time they need a check: code
// that runs while another component owns the device's memory budget (a
// framework whose caching allocator has reserved the free memory), code
// whose certification allows no allocation after start-up, or code on a
// path where an allocation's implicit synchronisation is not acceptable.
// For them every buffer of the pipeline is carved out of one file-scope
// device array of fixed size, reserved when the library is loaded and held
// by every GPU that loads it until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../../include/drf.h"
#include "../host/engine.h"
#include "pipeline.cuh"

namespace drf {
namespace {

constexpr size_t kNoAllocScratchBytes = DRF_NOALLOC_SCRATCH_BYTES;

// The scratch array.  In host code its name is only a host-side stand-in:
// its device address comes from cudaGetSymbolAddress, looked up on every
// call (a lookup allocates nothing), so that a device whose context was torn
// down and made again (cudaDeviceReset) gets the address of the array in its
// new context, never a stale one.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
// One lock per device (the array is per device): held for a whole call, so
// that calls on one device from several host threads run one after another;
// calls on different devices proceed in parallel.
std::mutex g_mu[kMaxDevices];

struct Carver {
    unsigned char *base;
    size_t used = 0;
    bool ok = true;
    template <typename T>
    T *take(size_t count)
    {
        size_t bytes = (std::max<size_t>(count, 1) * sizeof(T) + 255) & ~(size_t)255;
        if (used + bytes > kNoAllocScratchBytes) { ok = false; return nullptr; }
        T *p = reinterpret_cast<T *>(base + used);
        used += bytes;
        return p;
    }
};

template <typename T>
bool put(T *dst, const std::vector<T> &v, cudaStream_t s)
{
    return v.empty() || cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s) == cudaSuccess;
}

void fail_result(int status, drf_result *out)
{
    std::memset(out, 0, sizeof *out);
    out->status = status;
    out->verdict = -1;
}

}  // namespace
}  // namespace drf

using namespace drf;

extern "C" int drf_check_noalloc(const uint8_t *bytecode, size_t len, const drf_bounds *bounds, drf_result *out,
                                 void *stream)
{
    if (!out) return DRF_E_INVALID_ARG;
    if (!bytecode || !bounds) { fail_result(DRF_E_INVALID_ARG, out); return DRF_E_INVALID_ARG; }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        fail_result(DRF_E_CUDA, out);
        return DRF_E_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu[dev]);
    // the array's device address in the current context (on a device's first
    // call this also loads the library's device code there)
    unsigned char *base = nullptr;
    {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            fail_result(DRF_E_CUDA, out);
            return DRF_E_CUDA;
        }
        base = static_cast<unsigned char *>(p);
    }
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t s = (cudaStream_t)stream;

    Prepared prep;
    PrepareOpts po;
    po.desired_warp_items = (uint64_t)sms * 128;
    Error e = prepare(bytecode, len, bounds->nthreads, bounds->nlocs, bounds->loc_cells, bounds->nparams,
                      bounds->params, po, prep);
    if (!e.ok()) { fail_result(e.status, out); return e.status; }
    BatchHost bh;
    e = pack_batch({&prep}, bh);
    if (!e.ok()) { fail_result(e.status, out); return e.status; }

    // carve the fixed buffers; the launch epoch sits first so it survives calls
    Carver c{base};
    uint32_t *epoch = c.take<uint32_t>(4);
    BatchArgs a{};
    const uint64_t nw = bh.witems.size();
    const uint32_t nwblocks = (uint32_t)std::max<uint64_t>(1, (nw + kWScanPerBlock - 1) / kWScanPerBlock);
    Insn *insns = c.take<Insn>(bh.insns.size());
    uint64_t *xcode = c.take<uint64_t>(bh.xcode.size());
    ItemDesc *items = c.take<ItemDesc>(bh.items.size());
    DevProto *protos = c.take<DevProto>(bh.protos.size());
    uint64_t *cells = c.take<uint64_t>(bh.cells.size());
    WarpItem *witems = c.take<WarpItem>(nw);
    uint32_t *iphase = c.take<uint32_t>(bh.iphase.size());
    a.cnt = c.take<uint32_t>(bh.lanes);
    a.syn = c.take<uint32_t>(bh.lanes);
    a.phs = c.take<uint32_t>(bh.lanes);
    a.erro = c.take<unsigned long long>(bh.lanes);
    a.totsyn = c.take<uint32_t>(bh.ncols);
    a.wcnt = c.take<uint32_t>(nw);
    a.wbase = c.take<unsigned long long>(nw);
    a.blocksum = c.take<unsigned long long>(nwblocks);
    a.hist = c.take<unsigned long long>((size_t)kMaxPasses * kRadixBins);
    a.err_key = c.take<unsigned long long>(1);
    a.div_tid = c.take<uint32_t>(1);
    a.best_pos = c.take<unsigned long long>(1);
    a.ptuples = c.take<unsigned long long>(1);
    a.results = c.take<DevResult>(1);
    a.ctrl = c.take<Control>(1);
    if (!c.ok) { fail_result(DRF_E_LIMIT, out); return DRF_E_LIMIT; }
    a.insns = insns; a.xcode = xcode; a.items = items; a.protos = protos; a.cells = cells; a.witems = witems;
    a.iphase = iphase;
    a.count_free = 0;
    a.shard_lo = 0;
    a.shard_hi = ~0ull;
    a.rpiece = nullptr;                   // the sort path: no range pass
    a.wpiece = nullptr;
    a.rtask = nullptr;
    a.rlive = nullptr;
    a.rfirst = nullptr;
    a.nlive = 0;
    a.nrtask = 0;
    a.rtup = nullptr;
    a.rtotal = 0;
    a.rcount = 0;
    a.wkeys = nullptr;
    a.nrkeys = 0;
    a.nwkeys = 0;
    a.range_keys = 0;
    a.range_on = 0;
    a.nwitems = (uint32_t)nw;
    a.nprotos = 1;
    a.ncols = bh.ncols;
    a.nwblocks = nwblocks;
    a.epoch = epoch;
    a.L = bh.L;
    for (const DevProto &d : bh.protos) (d.wide ? a.has_wide : a.has_narrow) = 1;
    if (!put(insns, bh.insns, s) || !put(xcode, bh.xcode, s) || !put(items, bh.items, s) ||
        !put(protos, bh.protos, s) || !put(cells, bh.cells, s) || !put(witems, bh.witems, s) ||
        !put(iphase, bh.iphase, s)) {
        cudaGetLastError();
        fail_result(DRF_E_CUDA, out);
        return DRF_E_CUDA;
    }

    // count pass: the number of access keys decides the rest of the layout
    Control ctrl{};
    if (launch_front(a, s, sms, nullptr, nullptr) != cudaSuccess ||
        cudaMemcpyAsync(&ctrl, a.ctrl, sizeof ctrl, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        fail_result(DRF_E_CUDA, out);
        return DRF_E_CUDA;
    }
    const uint64_t n = ctrl.total;
    a.nkeys = n;
    a.ntiles = radix_tiles(n);
    a.ndtiles = detect_tiles(n);
    a.keys[0] = c.take<unsigned long long>(n);
    a.keys[1] = c.take<unsigned long long>(n);
    const size_t status_words = (size_t)a.L.passes * a.ntiles * kRadixBins;
    a.status = c.take<unsigned long long>(status_words);
    a.trec = c.take<TileRec>(a.ndtiles);
    if (!c.ok) { fail_result(DRF_E_LIMIT, out); return DRF_E_LIMIT; }   // more keys than the array holds
    // the look-back words may lie where an earlier call left other data
    // (all calls share the array): clear them every call
    if (cudaMemsetAsync(a.status, 0, status_words * 8, s) != cudaSuccess) {
        cudaGetLastError();
        fail_result(DRF_E_CUDA, out);
        return DRF_E_CUDA;
    }
    DevResult r{};
    if (launch_back(a, s, sms, nullptr, nullptr) != cudaSuccess ||
        cudaMemcpyAsync(&r, a.results, sizeof r, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&ctrl, a.ctrl, sizeof ctrl, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        fail_result(DRF_E_CUDA, out);
        return DRF_E_CUDA;
    }
    if (ctrl.flags) {
        int st = (ctrl.flags & CF_LOOKBACK_TIMEOUT) ? DRF_E_TIMEOUT : DRF_E_INTERNAL;
        fail_result(st, out);
        return st;
    }
    to_public(r, out);
    return out->status;
}
