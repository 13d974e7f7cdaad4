// The C ABI of include/drf.h.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>

#include "engine.h"
#include "jit.h"
#include "server.h"
#include "tune.h"

using namespace drf;

namespace {

int fail(drf_ctx *ctx, int status, const std::string &msg)
{
    if (ctx) ctx->last_error = msg;
    return status;
}

int cuda_fail(drf_ctx *ctx, cudaError_t e)
{
    cudaGetLastError();
    return fail(ctx, S_CUDA, std::string("CUDA: ") + cudaGetErrorString(e));
}

cudaStream_t pick(drf_ctx *ctx, void *stream) { return stream ? (cudaStream_t)stream : ctx->stream; }

Error prepare_one(const uint8_t *bc, size_t len, const drf_bounds *b, const PrepareOpts &po, Prepared &out)
{
    if (!bc || !b) return Error::make(S_INVALID_ARG, "null bytecode or bounds");
    return prepare(bc, len, b->nthreads, b->nlocs, b->loc_cells, b->nparams, b->params, po, out);
}

// The specialized kernels of one protocol under its bounds, from the
// context's cache, compiled and loaded on a miss (a protocol that cannot be
// specialized is remembered as such).  The key is the bytecode and the
// bounds themselves: the kernels depend on nothing else (the preparation
// options of drf_check are fixed per context).
const JitEntry *jit_entry(drf_ctx *ctx, const uint8_t *bc, size_t len, const drf_bounds *b, const Prepared &p,
                          BatchHost &bh)
{
    std::string key;
    auto put = [&key](const void *x, size_t n) { key.append((const char *)x, n); };
    put(&len, sizeof len);
    put(bc, len);
    put(&b->nthreads, sizeof b->nthreads);
    put(&b->nlocs, sizeof b->nlocs);
    if (b->nlocs) put(b->loc_cells, b->nlocs * sizeof(uint64_t));
    put(&b->nparams, sizeof b->nparams);
    if (b->nparams) put(b->params, b->nparams * sizeof(int64_t));
    auto found = ctx->jit_cache.find(key);
    if (found != ctx->jit_cache.end()) return found->second.get();
    if (ctx->jit_cache.size() >= kJitCacheEntries) ctx->jit_cache.clear();
    auto je = std::make_unique<JitEntry>();
    std::string src, log;
    std::vector<uint16_t> shapes;
    std::vector<char> cubin;
    bool stat = false, csched = false, range = false;
    auto mod = std::make_unique<JitModule>();
    bh.expand_witems();                            // the generator reads the schedule
    Error e = jit_source(p, bh, src, shapes, &stat, &csched, &range);
    if (e.ok()) e = jit_compile(src, cubin, log);
    if (e.ok()) e = jit_load(cubin, *mod);
    if (e.ok() && (cudaMalloc(&je->shape, std::max<size_t>(shapes.size() * 2, 16)) != cudaSuccess ||
                   cudaMemcpy(je->shape, shapes.data(), shapes.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess))
        e = Error::make(S_NOMEM, "device allocation failed");
    cudaGetLastError();
    if (e.ok()) {
        je->launch.count = (const void *)mod->count;
        je->launch.table = (const void *)mod->table;
        je->launch.cell = (const void *)mod->cell;
        je->launch.range = range;
        je->launch.shape = (const uint16_t *)je->shape;
        je->launch.static_phases = stat;
        je->launch.csched = csched;
        je->mod = std::move(mod);
    }
    const JitEntry *out = je.get();
    ctx->jit_cache[key] = std::move(je);
    return out;
}

void error_result(int status, drf_result *out)
{
    std::memset(out, 0, sizeof *out);
    out->status = status;
    out->verdict = -1;
}

}  // namespace

extern "C" {

int drf_version(void) { return 1; }

const char *drf_status_string(int s)
{
    switch (s) {
    case DRF_OK: return "DRF_OK";
    case DRF_E_INVALID_ARG: return "DRF_E_INVALID_ARG";
    case DRF_E_PARSE: return "DRF_E_PARSE";
    case DRF_E_INVALID_BYTECODE: return "DRF_E_INVALID_BYTECODE";
    case DRF_E_UNBOUND_VAR: return "DRF_E_UNBOUND_VAR";
    case DRF_E_UNKNOWN_ARRAY: return "DRF_E_UNKNOWN_ARRAY";
    case DRF_E_REBIND: return "DRF_E_REBIND";
    case DRF_E_SYNC_IN_UNSYNC: return "DRF_E_SYNC_IN_UNSYNC";
    case DRF_E_OVERFLOW_RISK: return "DRF_E_OVERFLOW_RISK";
    case DRF_E_INDEX_OOB: return "DRF_E_INDEX_OOB";
    case DRF_E_DIV_ZERO: return "DRF_E_DIV_ZERO";
    case DRF_E_KEY_TOO_WIDE: return "DRF_E_KEY_TOO_WIDE";
    case DRF_E_NOMEM: return "DRF_E_NOMEM";
    case DRF_E_CUDA: return "DRF_E_CUDA";
    case DRF_E_TIMEOUT: return "DRF_E_TIMEOUT";
    case DRF_E_BUSY: return "DRF_E_BUSY";
    case DRF_E_LIMIT: return "DRF_E_LIMIT";
    case DRF_E_NOT_FOUND: return "DRF_E_NOT_FOUND";
    case DRF_E_INTERNAL: return "DRF_E_INTERNAL";
    default: return "DRF_E_UNKNOWN";
    }
}

int drf_ctx_create(int device, const drf_opts *opts, drf_ctx **out)
{
    if (!out) return DRF_E_INVALID_ARG;
    *out = nullptr;
    if (opts && opts->radix_bits && (opts->radix_bits < 4 || opts->radix_bits > 8)) return DRF_E_INVALID_ARG;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) { cudaGetLastError(); return DRF_E_CUDA; }
    drf_ctx *ctx = new (std::nothrow) drf_ctx;
    if (!ctx) return DRF_E_NOMEM;
    ctx->device = device;
    if (opts) ctx->opts = *opts;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && sms > 0) ctx->sms = sms;
    if ((e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking)) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return DRF_E_CUDA;
    }
    *out = ctx;
    return DRF_OK;
}

void drf_ctx_destroy(drf_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->server) drf_server_stop(ctx);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    cudaStreamDestroy(ctx->stream);
    delete ctx;                       // frees the workspace's device buffers
}

const char *drf_last_error(const drf_ctx *ctx) { return ctx ? ctx->last_error.c_str() : ""; }

int drf_protocol_compile(const char *text, uint8_t **bytecode, size_t *len, char *err, size_t errlen)
{
    if (err && errlen) err[0] = 0;
    if (!text || !bytecode || !len) return DRF_E_INVALID_ARG;
    *bytecode = nullptr;
    *len = 0;
    Protocol p;
    Error e = parse_text(text, p);
    if (!e.ok()) {
        if (err && errlen) { std::strncpy(err, e.message.c_str(), errlen - 1); err[errlen - 1] = 0; }
        return e.status;
    }
    std::vector<uint8_t> bc = encode_bytecode(p);
    uint8_t *buf = (uint8_t *)std::malloc(bc.size());
    if (!buf) return DRF_E_NOMEM;
    std::memcpy(buf, bc.data(), bc.size());
    *bytecode = buf;
    *len = bc.size();
    return DRF_OK;
}

int drf_babycuda_infer(const char *text, uint8_t **bytecode, size_t *len, char *err, size_t errlen)
{
    if (err && errlen) err[0] = 0;
    if (!text || !bytecode || !len) return DRF_E_INVALID_ARG;
    *bytecode = nullptr;
    *len = 0;
    Protocol p;
    Error e = parse_babycuda_text(text, p);
    if (!e.ok()) {
        if (err && errlen) { std::strncpy(err, e.message.c_str(), errlen - 1); err[errlen - 1] = 0; }
        return e.status;
    }
    std::vector<uint8_t> bc = encode_bytecode(p);
    uint8_t *buf = (uint8_t *)std::malloc(bc.size());
    if (!buf) return DRF_E_NOMEM;
    std::memcpy(buf, bc.data(), bc.size());
    *bytecode = buf;
    *len = bc.size();
    return DRF_OK;
}

int drf_protocol_text(const uint8_t *bytecode, size_t len, char **text)
{
    if (!text) return DRF_E_INVALID_ARG;
    *text = nullptr;
    Protocol p;
    Error e = decode_bytecode(bytecode, len, p);
    if (!e.ok()) return e.status;
    std::string t = protocol_text(p);
    char *buf = (char *)std::malloc(t.size() + 1);
    if (!buf) return DRF_E_NOMEM;
    std::memcpy(buf, t.c_str(), t.size() + 1);
    *text = buf;
    return DRF_OK;
}

int drf_protocol_info(const uint8_t *bytecode, size_t len, uint32_t *nlocs, uint32_t *nparams)
{
    Protocol p;
    Error e = decode_bytecode(bytecode, len, p);
    if (!e.ok()) return e.status;
    if (nlocs) *nlocs = p.narrays;
    if (nparams) *nparams = p.nparams;
    return DRF_OK;
}

int drf_protocol_analyze(const uint8_t *bytecode, size_t len, const drf_bounds *bounds, drf_analysis *out)
{
    if (!out) return DRF_E_INVALID_ARG;
    std::memset(out, 0, sizeof *out);
    Prepared p;
    Error e = prepare_one(bytecode, len, bounds, PrepareOpts{}, p);
    if (!e.ok()) return e.status;
    BatchHost bh;
    e = pack_batch({&p}, bh, true, 0, 0);
    out->tuple_bound = p.tuple_bound();
    out->sync_bound = p.max_syncs;
    out->items = (uint32_t)p.items.size();
    out->wide_arithmetic = p.wide ? 1 : 0;
    out->sort_bits = bh.L.sort_bits;
    out->key_bits = bh.L.sort_lo + bh.L.sort_bits;
    out->range_tuples = bh.rlive.empty() ? 0 : bh.range_tuples;
    return e.status;
}

void drf_free(void *p) { std::free(p); }

int drf_check(drf_ctx *ctx, const uint8_t *bytecode, size_t len, const drf_bounds *bounds, drf_result *out,
              void *stream)
{
    if (!ctx || !out) return DRF_E_INVALID_ARG;
    const uint8_t *const bcs[1] = {bytecode};
    const size_t lens[1] = {len};
    int st = drf_check_batch(ctx, 1, bcs, lens, bounds, out, stream);
    return st ? st : out->status;
}

int drf_check_batch(drf_ctx *ctx, uint32_t n, const uint8_t *const *bytecodes, const size_t *lens,
                    const drf_bounds *bounds, drf_result *out, void *stream)
{
    if (!ctx || !out || (n && (!bytecodes || !lens || !bounds))) return DRF_E_INVALID_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    cudaError_t ce = cudaSetDevice(ctx->device);
    if (ce != cudaSuccess) return cuda_fail(ctx, ce);
    ctx->last_error.clear();
    PrepareOpts po;
    po.desired_warp_items = std::max<uint64_t>(1, (uint64_t)ctx->sms * 128 / std::max<uint32_t>(1, n));
    // prepared programs come from the context's cache when the same
    // protocol was checked before under the same bounds
    std::vector<std::shared_ptr<const Prepared>> preps(n);
    std::vector<const Prepared *> valid;
    std::vector<uint32_t> where;
    for (uint32_t i = 0; i < n; i++) {
        Error e;
        preps[i] = ctx->prep_cache.get(bytecodes[i], lens[i], &bounds[i], po, e);
        if (!e.ok()) {
            error_result(e.status, &out[i]);
            if (n == 1) ctx->last_error = e.message;
            continue;
        }
        valid.push_back(preps[i].get());
        where.push_back(i);
    }
    if (valid.empty()) return DRF_OK;
    cudaStream_t s = pick(ctx, stream);
    BatchHost &bh = ctx->host;
    // one protocol that may run specialized kernels: the warp-item schedule
    // is expanded only if the kernels that run read it (compiled-in
    // schedules do not)
    const bool jit_try = valid.size() == 1 && (ctx->opts.flags & DRF_OPT_SPECIALIZE) && path_pref_of(ctx->opts) != 1;
    // a check of the one protocol packed last time reuses that pack (the
    // host image; it is still uploaded with every check)
    Error e;
    const bool same_pack = valid.size() == 1 && ctx->host_of && ctx->host_of.get() == valid[0] &&
                           ctx->host_digit_bits == ctx->opts.radix_bits && (bh.expanded() || jit_try);
    if (!same_pack) {
        ctx->host_of.reset();
        e = pack_batch(valid, bh, !jit_try, ctx->opts.radix_bits,
                       valid.size() == 1 ? range_min_of(ctx->opts) : range_min_once(ctx->opts));
        if (e.ok() && valid.size() == 1) {
            ctx->host_of = preps[where[0]];
            ctx->host_digit_bits = ctx->opts.radix_bits;
        }
    }
    if (e.status == S_KEY_TOO_WIDE && valid.size() > 1) {
        // the combined key does not fit: check the protocols one by one
        for (size_t j = 0; j < valid.size(); j++) {
            Error ej = pack_batch({valid[j]}, bh, true, ctx->opts.radix_bits, range_min_once(ctx->opts));
            if (!ej.ok()) { error_result(ej.status, &out[where[j]]); continue; }
            std::vector<DevResult> r;
            int st = run_batch(ctx, bh, s, r);
            if (st) return st;
            to_public(r[0], &out[where[j]]);
        }
        return DRF_OK;
    }
    if (!e.ok()) {
        for (uint32_t i : where) error_result(e.status, &out[i]);
        if (n == 1) ctx->last_error = e.message;
        return DRF_OK;
    }
    std::vector<DevResult> r;
    // one protocol with DRF_OPT_SPECIALIZE: the kernels compiled for it (the
    // first check of a protocol under given bounds compiles them), when its
    // owner table is of a size the automatic choice would take
    if (jit_try && bh.table_ok && bh.tuple_bound >= kJitMinTuples && auto_path(bh, bh.tuple_bound) == PATH_TABLE) {
        const uint32_t i = where[0];
        const JitEntry *je = jit_entry(ctx, bytecodes[i], lens[i], &bounds[i], *valid[0], bh);
        if (je && je->mod) {
            if (!je->launch.csched) bh.expand_witems();
            int st = run_batch_jit(ctx, bh, je->launch, s, r);
            if (st == S_OK) {
                to_public(r[0], &out[i]);
                return DRF_OK;
            }
            if (st == S_CUDA) return st;
            ctx->last_error.clear();                // no room for the table: interpret
        }
    }
    bh.expand_witems();                            // the interpreter reads the schedule
    int st = run_batch(ctx, bh, s, r);
    if (st) return st;
    for (size_t j = 0; j < where.size(); j++) to_public(r[j], &out[where[j]]);
    return DRF_OK;
}

int drf_ctx_transfer_bytes(const drf_ctx *ctx, uint64_t *h2d, uint64_t *d2h)
{
    if (!ctx) return DRF_E_INVALID_ARG;
    if (h2d) *h2d = ctx->work.h2d_bytes;
    if (d2h) *d2h = ctx->work.d2h_bytes;
    return DRF_OK;
}

int drf_debug_sorted_keys(drf_ctx *ctx, uint64_t *keys, uint64_t cap, uint64_t *n, uint32_t layout[5])
{
    if (!ctx || !n) return DRF_E_INVALID_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    cudaError_t ce = cudaSetDevice(ctx->device);
    if (ce != cudaSuccess) return cuda_fail(ctx, ce);
    const BatchArgs &a = ctx->work.args;
    if (a.path == PATH_TABLE)
        return fail(ctx, DRF_E_NOT_FOUND, "the last check ran the owner-table path, which sorts no keys");
    *n = a.nkeys;
    if (layout) {
        layout[0] = a.L.tid_bits; layout[1] = a.L.idx_bits; layout[2] = a.L.loc_bits;
        layout[3] = a.L.phase_bits; layout[4] = a.L.proto_bits;
    }
    if (!keys || !cap || !a.nkeys) return DRF_OK;
    // the sorted keys sit in the buffer the last non-trivial pass wrote
    std::vector<unsigned long long> hist((size_t)kMaxPasses * kRadixBins);
    if ((ce = cudaMemcpy(hist.data(), a.hist, hist.size() * 8, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(ctx, ce);
    int passes = 0;
    for (uint32_t q = 0; q < a.L.passes; q++) {
        int nz = 0;
        for (int d = 0; d < kRadixBins; d++) nz += hist[(size_t)q * kRadixBins + d] != 0;
        passes += nz > 1;
    }
    uint64_t m = std::min<uint64_t>(cap, a.nkeys);
    if ((ce = cudaMemcpy(keys, a.keys[passes & 1], m * 8, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(ctx, ce);
    return DRF_OK;
}

}  // extern "C"

namespace {

// Owner-table positions [lo, hi) of shard k of n of a prepared protocol:
// the positions phase * (sum of array sizes) + (the array's offset) + index
// over the phases the static sync bound allows, cut into n equal parts.
Error shard_window(const Prepared &p, uint32_t shard, uint32_t nshards, uint64_t &lo, uint64_t &hi, uint64_t &total)
{
    if (nshards == 0 || shard >= nshards) return Error::make(S_INVALID_ARG, "shard index out of range");
    unsigned __int128 row = 0;
    for (uint64_t c : p.cells) row += c;
    const unsigned __int128 t = row * ((unsigned __int128)p.max_syncs + 1);
    if (t >= ((unsigned __int128)1 << 63)) return Error::make(S_LIMIT, "more than 2^63 cell positions");
    total = (uint64_t)t;
    lo = (uint64_t)(t * shard / nshards);
    hi = (uint64_t)(t * (shard + 1) / nshards);
    return Error{};
}

bool same_facts(const drf_result &a, const drf_result &b)
{
    if (a.status != b.status || a.tuples != b.tuples) return false;
    if (a.status != DRF_OK) return a.err_tid == b.err_tid && a.err_ordinal == b.err_ordinal;
    if (a.phases != b.phases || a.sync_count_0 != b.sync_count_0) return false;
    const bool ad = a.verdict == DRF_VERDICT_BARRIER_DIVERGENCE, bd = b.verdict == DRF_VERDICT_BARRIER_DIVERGENCE;
    if (ad != bd) return false;
    return !ad || (a.div_tid == b.div_tid && a.sync_count_div == b.sync_count_div);
}

}  // namespace

extern "C" {

int drf_shard_range(const uint8_t *bytecode, size_t len, const drf_bounds *bounds, uint32_t shard, uint32_t nshards,
                    uint64_t *lo, uint64_t *hi, uint64_t *positions)
{
    if (!lo || !hi) return DRF_E_INVALID_ARG;
    Prepared p;
    Error e = prepare_one(bytecode, len, bounds, PrepareOpts{}, p);
    uint64_t total = 0;
    if (e.ok()) e = shard_window(p, shard, nshards, *lo, *hi, total);
    if (e.ok() && positions) *positions = total;
    return e.status;
}

int drf_check_shard(drf_ctx *ctx, const uint8_t *bytecode, size_t len, const drf_bounds *bounds, uint32_t shard,
                    uint32_t nshards, drf_result *out, void *stream)
{
    if (!ctx || !out) return DRF_E_INVALID_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    cudaError_t ce = cudaSetDevice(ctx->device);
    if (ce != cudaSuccess) return cuda_fail(ctx, ce);
    ctx->last_error.clear();
    PrepareOpts po;
    po.desired_warp_items = (uint64_t)ctx->sms * 128;
    Prepared p;
    Error e = prepare_one(bytecode, len, bounds, po, p);
    uint64_t lo = 0, hi = 0, total = 0;
    if (e.ok()) e = shard_window(p, shard, nshards, lo, hi, total);
    ctx->host_of.reset();
    if (e.ok()) e = pack_batch({&p}, ctx->host, true, ctx->opts.radix_bits, range_min_of(ctx->opts));
    if (e.ok() && !ctx->host.table_ok) e = Error::make(S_LIMIT, "the protocol's owner table does not fit");
    if (!e.ok()) {
        error_result(e.status, out);
        return fail(ctx, e.status, e.message);
    }
    DeviceBatch &w = ctx->work;
    w.limit = ctx->opts.max_device_bytes;
    w.path_pref = 2;                          // the shard is a window of the owner table
    w.shard_lo = lo;
    w.shard_hi = hi;
    std::vector<DevResult> r;
    int st = run_batch(w, ctx->sms, pick(ctx, stream), ctx->host, r, ctx->last_error);
    w.shard_lo = 0;
    w.shard_hi = ~0ull;
    if (st) return st;
    to_public(r[0], out);
    return out->status;
}

int drf_merge_shards(const drf_result *parts, uint32_t n, drf_result *out)
{
    if (!parts || !out || n == 0) return DRF_E_INVALID_ARG;
    for (uint32_t i = 1; i < n; i++)
        if (!same_facts(parts[0], parts[i])) return DRF_E_INTERNAL;   // the shards disagree on a global fact
    *out = parts[0];
    if (out->status != DRF_OK || out->verdict == DRF_VERDICT_BARRIER_DIVERGENCE) return out->status;
    // the lexicographically smallest racy cell over the shards, with its witness
    const drf_result *best = nullptr;
    for (uint32_t i = 0; i < n; i++) {
        const drf_result &x = parts[i];
        if (x.verdict != DRF_VERDICT_RACY) continue;
        if (!best || x.phase < best->phase || (x.phase == best->phase && x.loc < best->loc) ||
            (x.phase == best->phase && x.loc == best->loc && x.index < best->index))
            best = &x;
    }
    if (best) {
        *out = *best;
    } else {
        out->verdict = DRF_VERDICT_DRF;
        out->phase = out->loc = 0;
        out->index = 0;
        out->tid_i = out->tid_j = out->i_writes = out->j_writes = 0;
    }
    return DRF_OK;
}

int drf_debug_stall_lookback(drf_ctx *ctx, uint32_t launches)
{
    if (!ctx) return DRF_E_INVALID_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    ctx->work.stall_lookback = launches;
    return DRF_OK;
}

int drf_check_param_sweep(drf_ctx *ctx, const uint8_t *bytecode, size_t len, const drf_bounds *bounds,
                          uint32_t param, int64_t lo, int64_t hi, drf_result *out, void *stream)
{
    if (!ctx || !bytecode || !bounds || !out || hi < lo) return DRF_E_INVALID_ARG;
    if (param >= bounds->nparams || !bounds->params) return DRF_E_INVALID_ARG;
    if ((uint64_t)(hi - lo) > (1u << 20)) return fail(ctx, DRF_E_LIMIT, "more than 2^20 parameter values");
    const uint32_t n = (uint32_t)(hi - lo);
    if (n == 0) return DRF_OK;
    std::vector<int64_t> values((size_t)n * bounds->nparams);
    std::vector<drf_bounds> bs(n, *bounds);
    std::vector<const uint8_t *> bcs(n, bytecode);
    std::vector<size_t> lens(n, len);
    for (uint32_t k = 0; k < n; k++) {
        int64_t *v = &values[(size_t)k * bounds->nparams];
        std::memcpy(v, bounds->params, sizeof(int64_t) * bounds->nparams);
        v[param] = lo + (int64_t)k;
        bs[k].params = v;
    }
    return drf_check_batch(ctx, n, bcs.data(), lens.data(), bs.data(), out, stream);
}

int drf_protocol_specialize(const uint8_t *bytecode, size_t len, const drf_bounds *bounds, int compile,
                            char **source, char *log, size_t loglen)
{
    if (log && loglen) log[0] = 0;
    if (!source) return DRF_E_INVALID_ARG;
    *source = nullptr;
    Prepared p;
    Error e = prepare_one(bytecode, len, bounds, PrepareOpts{}, p);
    if (!e.ok()) return e.status;
    BatchHost bh;
    e = pack_batch({&p}, bh);
    if (!e.ok()) return e.status;
    std::string src, clog;
    std::vector<uint16_t> shapes;
    e = jit_source(p, bh, src, shapes);
    if (!e.ok()) clog = e.message;
    if (e.ok()) {
        char *buf = (char *)std::malloc(src.size() + 1);
        if (!buf) return DRF_E_NOMEM;
        std::memcpy(buf, src.c_str(), src.size() + 1);
        *source = buf;
        if (compile) {
            std::vector<char> cubin;
            e = jit_compile(src, cubin, clog);
        }
    }
    if (log && loglen) { std::strncpy(log, clog.c_str(), loglen - 1); log[loglen - 1] = 0; }
    return e.status;
}

// ------------------------------------------------------------------- plans

}  // extern "C"

namespace {

// Prepares, packs and uploads a batch under one launch configuration and
// does the sizing run (count pass, then the whole pipeline once so that
// evaluation errors surface).  On failure returns the status and leaves
// *out null.
int build_plan(drf_ctx *ctx, uint32_t n, const uint8_t *const *bytecodes, const size_t *lens,
               const drf_bounds *bounds, const PlanConfig &cfg, drf_plan **out)
{
    *out = nullptr;
    PrepareOpts po;
    po.desired_warp_items = std::max<uint64_t>(1, (uint64_t)ctx->sms * cfg.granularity / n);
    std::vector<Prepared> preps(n);
    std::vector<const Prepared *> ptrs;
    for (uint32_t i = 0; i < n; i++) {
        Error e = prepare_one(bytecodes[i], lens[i], &bounds[i], po, preps[i]);
        if (!e.ok()) return fail(ctx, e.status, "protocol " + std::to_string(i) + ": " + e.message);
        ptrs.push_back(&preps[i]);
    }
    drf_plan *plan = new (std::nothrow) drf_plan;
    if (!plan) return DRF_E_NOMEM;
    plan->ctx = ctx;
    plan->n = n;
    plan->cfg = cfg;
    Error e = pack_batch(ptrs, plan->host, true, cfg.radix_bits ? cfg.radix_bits : ctx->opts.radix_bits,
                         range_min_of(ctx->opts));
    if (!e.ok()) { delete plan; return fail(ctx, e.status, e.message); }
    cudaStream_t s = ctx->stream;
    DeviceBatch &d = plan->dev;
    d.limit = ctx->opts.max_device_bytes;
    d.radix_items = cfg.radix_items;
    d.path_pref = cfg.path ? (int)cfg.path : path_pref_of(ctx->opts);
    if (cfg.jit) d.path_pref = 2;                  // specialized kernels run the owner-table back end
    e = d.load(plan->host, s);
    if (!e.ok()) { delete plan; return fail(ctx, e.status, e.message); }
    if (cfg.jit) {
        // kernels specialized to the protocol: generate, compile (NVRTC), load
        std::string src;
        std::vector<uint16_t> shapes;
        std::vector<char> cubin;
        auto mod = std::make_unique<JitModule>();
        bool stat = false, csched = false, range = false;
        e = n == 1 ? jit_source(preps[0], plan->host, src, shapes, &stat, &csched, &range)
                   : Error::make(S_INVALID_ARG, "specialization takes a plan of one protocol");
        d.jit.static_phases = stat;
        d.jit.csched = csched;
        if (e.ok()) e = jit_compile(src, cubin, plan->jit_log);
        if (e.ok()) e = jit_load(cubin, *mod);
        if (e.ok() && (!ensure(d.ishape, std::max<size_t>(shapes.size() * 2, 16), &d.in_use, d.limit) ||
                       cudaMemcpyAsync(d.ishape.p, shapes.data(), shapes.size() * 2, cudaMemcpyHostToDevice, s) !=
                           cudaSuccess))
            e = Error::make(S_NOMEM, "device allocation failed");
        if (!e.ok()) {
            cudaGetLastError();
            const std::string why = e.message + (plan->jit_log.empty() ? "" : "\n" + plan->jit_log);
            delete plan;
            return fail(ctx, e.status, "specialization: " + why);
        }
        plan->jit = std::move(mod);
        d.jit.count = (const void *)plan->jit->count;
        d.jit.table = (const void *)plan->jit->table;
        d.jit.cell = (const void *)plan->jit->cell;
        d.jit.range = range;
        d.jit.shape = (const uint16_t *)d.ishape.p;
    }
    cudaError_t ce;
    // the sizing run counts with the count and scan passes even when the
    // plan's launches leave them out
    JitLaunch sizing = d.jit;
    sizing.static_phases = false;
    sizing.range = false;
    if ((ce = launch_front(d.args, s, ctx->sms, nullptr, nullptr, &sizing)) != cudaSuccess ||
        (ce = d.fetch(s, true)) != cudaSuccess || (ce = cudaStreamSynchronize(s)) != cudaSuccess) {
        delete plan;
        return cuda_fail(ctx, ce);
    }
    // (the count pass leaves out the range accesses whose keys come from the pieces)
    const uint64_t counted = d.host_ctrl()->total;
    plan->tuples = counted + (d.args.range_keys ? plan->host.range_tuples : 0);
    e = d.choose_path(plan->host, counted, s);
    if (!e.ok()) { delete plan; return fail(ctx, e.status, e.message); }
    plan->cfg.path = d.args.path == PATH_TABLE ? 2 : 1;
    if (cfg.jit && d.args.path != PATH_TABLE) { delete plan; return fail(ctx, DRF_E_LIMIT, "specialization needs the owner table"); }
    d.status_launches++;
    std::vector<DevResult> res(n);
    if ((ce = launch_back(d.args, s, ctx->sms, nullptr, nullptr, &d.jit)) != cudaSuccess ||
        (ce = cudaMemcpyAsync(res.data(), d.args.results, n * sizeof(DevResult), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (ce = cudaStreamSynchronize(s)) != cudaSuccess) {
        delete plan;
        return cuda_fail(ctx, ce);
    }
    for (uint32_t i = 0; i < n; i++)
        if (res[i].status) { delete plan; return fail(ctx, res[i].status, "protocol " + std::to_string(i) + " fails to evaluate"); }
    // the plan's own launches: interpreted owner-table launches of a batch
    // whose protocols all have static phases need no count or scan pass
    d.args.count_free = (!cfg.jit && d.args.path == PATH_TABLE && plan->host.all_static) ? 1u : 0u;
    *out = plan;
    return DRF_OK;
}

// Best of `reps` direct launches of the whole pipeline, in milliseconds.
// Before each launch `flush` (when not null) is overwritten, outside the
// timed events, so that every launch starts with a cold L2 as a check of a
// new batch does.
// Device time of one launch of the plan's pipeline: the median of `reps`
// launches, each after a write of `flush_bytes` (a cold L2), following
// `warm` untimed launches.  The launches are queued back to back, as a
// plan's user runs them, so that the GPU stays at its working clocks (the
// first launches of freshly loaded kernels, and launches after an idle gap,
// run slower than that steady state).
double time_plan(drf_plan *plan, int reps, void *flush, size_t flush_bytes, int warm = 3)
{
    drf_ctx *ctx = plan->ctx;
    cudaStream_t s = ctx->stream;
    DeviceBatch &d = plan->dev;
    const int n = warm + reps;
    std::vector<cudaEvent_t> ev(2 * n, nullptr);
    bool ok = true;
    for (auto &e : ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
    for (int r = 0; ok && r < n; r++) {
        d.status_launches++;
        if (flush) cudaMemsetAsync(flush, r & 0xff, flush_bytes, s);
        cudaEventRecord(ev[2 * r], s);
        launch_front(d.args, s, ctx->sms, nullptr, nullptr, &d.jit);
        launch_back(d.args, s, ctx->sms, nullptr, nullptr, &d.jit);
        cudaEventRecord(ev[2 * r + 1], s);
    }
    std::vector<double> ms_all;
    if (ok && cudaStreamSynchronize(s) == cudaSuccess) {
        for (int r = warm; r < n; r++) {
            float ms = 0;
            if (cudaEventElapsedTime(&ms, ev[2 * r], ev[2 * r + 1]) == cudaSuccess) ms_all.push_back(ms);
        }
    }
    for (auto &e : ev) if (e) cudaEventDestroy(e);
    cudaGetLastError();
    if (ms_all.empty()) return 1e30;
    std::sort(ms_all.begin(), ms_all.end());
    return ms_all[ms_all.size() / 2];
}

// Records the plan's pipeline as one CUDA graph (timing events inside when
// the context profiles stages).
int capture_plan(drf_plan *plan)
{
    drf_ctx *ctx = plan->ctx;
    cudaStream_t s = ctx->stream;
    DeviceBatch &d = plan->dev;
    plan->profiled = (ctx->opts.flags & DRF_OPT_PROFILE_STAGES) != 0;
    if (plan->profiled) {
        plan->events.resize(kMaxStages + 1);
        for (auto &ev : plan->events) cudaEventCreate(&ev);
    }
    cudaEvent_t *evp = plan->profiled ? plan->events.data() : nullptr;
    int nev = 0;
    cudaError_t ce;
    if ((ce = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return cuda_fail(ctx, ce);
    cudaError_t e1 = launch_front(d.args, s, ctx->sms, evp, &nev, &d.jit);
    cudaError_t e2 = launch_back(d.args, s, ctx->sms, evp, &nev, &d.jit);
    ce = cudaStreamEndCapture(s, &plan->graph);
    plan->nevents = nev;
    if (e1 != cudaSuccess || e2 != cudaSuccess || ce != cudaSuccess ||
        (ce = cudaGraphInstantiate(&plan->exec, plan->graph, 0)) != cudaSuccess)
        return cuda_fail(ctx, ce != cudaSuccess ? ce : (e1 != cudaSuccess ? e1 : e2));
    return DRF_OK;
}

std::string signature(drf_ctx *ctx, uint32_t n, const drf_plan *p)
{
    uint32_t maxt = 0;
    for (const DevProto &d : p->host.protos) maxt = std::max(maxt, d.nthreads);
    return "sms" + std::to_string(ctx->sms) + "_n" + std::to_string(bits_for(n)) + "_t" +
           std::to_string(bits_for(p->tuples)) + "_s" + std::to_string(p->host.L.sort_bits) + "_T" +
           std::to_string(bits_for(maxt)) + "_b" + std::to_string(bits_for(p->host.table_bytes())) + "_p" +
           std::to_string(path_pref_of(ctx->opts));
}

}  // namespace

extern "C" {

int drf_plan_create(drf_ctx *ctx, uint32_t n, const uint8_t *const *bytecodes, const size_t *lens,
                    const drf_bounds *bounds, drf_plan **out)
{
    if (!ctx || !out || !n || !bytecodes || !lens || !bounds) return DRF_E_INVALID_ARG;
    *out = nullptr;
    std::lock_guard<std::mutex> lock(ctx->mu);
    cudaError_t ce = cudaSetDevice(ctx->device);
    if (ce != cudaSuccess) return cuda_fail(ctx, ce);
    drf_plan *plan = nullptr;
    PlanConfig first;
    const bool specialize = (ctx->opts.flags & DRF_OPT_SPECIALIZE) && n == 1 && path_pref_of(ctx->opts) != 1;
    std::string jit_why;
    if (specialize && !(ctx->opts.flags & DRF_OPT_AUTOTUNE)) {
        first.jit = 1;
        if (build_plan(ctx, n, bytecodes, lens, bounds, first, &plan)) {
            jit_why = ctx->last_error;        // not specializable here: keep the interpreter
            first.jit = 0;
            plan = nullptr;
        }
    }
    int st = plan ? 0 : build_plan(ctx, n, bytecodes, lens, bounds, first, &plan);
    if (st) return st;
    if (!jit_why.empty()) plan->jit_log = jit_why;
    if (ctx->opts.flags & DRF_OPT_AUTOTUNE) {
        // tune: time every candidate configuration, keep the fastest; a
        // workload signature seen before reuses its choice
        const std::string key = signature(ctx, n, plan);
        PlanConfig best_cfg;
        bool kept = false;                    // `plan` is the fastest candidate as measured
        if (!tune_lookup(key, best_cfg)) {
            // scratch larger than L2, overwritten before each timed launch
            const size_t flush_bytes = 256ull << 20;
            void *flush = nullptr;
            if (cudaMalloc(&flush, flush_bytes) != cudaSuccess) { cudaGetLastError(); flush = nullptr; }
            double best = time_plan(plan, kTuneReps, flush, flush_bytes);
            best_cfg = plan->cfg;
            // candidates: the sort path under every granularity and tile
            // shape, the owner table (no radix tiles) under every granularity
            const int pref = path_pref_of(ctx->opts);
            std::vector<PlanConfig> cands;
            for (uint32_t g : kTuneGranularity) {
                if (pref != 2)
                    for (uint32_t it : kTuneRadixItems) cands.push_back(PlanConfig{g, it, 1, 0});
                if (pref != 1 && plan->host.table_ok) cands.push_back(PlanConfig{g, 16, 2, 0});
                if (specialize && plan->host.table_ok) cands.push_back(PlanConfig{g, 16, 2, 1});
            }
            const PlanConfig timed = plan->cfg;   // the first plan's configuration, timed above
            for (const PlanConfig &c : cands) {
                if (c.granularity == timed.granularity && c.path == timed.path && c.jit == timed.jit &&
                    (c.path == 2 || c.radix_items == timed.radix_items))
                    continue;
                drf_plan *cand = nullptr;
                if (build_plan(ctx, n, bytecodes, lens, bounds, c, &cand)) continue;
                double ms = time_plan(cand, kTuneReps, flush, flush_bytes);
                // the winner is kept as built: its timing covers its own
                // buffers (the same configuration in other device memory --
                // an owner table elsewhere -- can run measurably slower)
                if (ms < best) {
                    best = ms;
                    best_cfg = c;
                    std::swap(plan, cand);
                }
                drf_plan_destroy(cand);
            }
            // the radix digit width, on the fastest sort-path configuration
            // (unless the context fixes it)
            if (best_cfg.path == 1 && ctx->opts.radix_bits == 0) {
                for (uint32_t bits : kTuneRadixBits) {
                    PlanConfig c = best_cfg;
                    c.radix_bits = bits;
                    drf_plan *cand = nullptr;
                    if (build_plan(ctx, n, bytecodes, lens, bounds, c, &cand)) continue;
                    double ms = time_plan(cand, kTuneReps, flush, flush_bytes);
                    if (ms < best) {
                        best = ms;
                        best_cfg = c;
                        std::swap(plan, cand);
                    }
                    drf_plan_destroy(cand);
                }
            }
            if (flush) cudaFree(flush);
            tune_store(key, best_cfg, best);
            kept = true;
        }
        if (!kept && (best_cfg.granularity != plan->cfg.granularity || best_cfg.radix_items != plan->cfg.radix_items ||
                      best_cfg.path != plan->cfg.path || best_cfg.jit != plan->cfg.jit ||
                      best_cfg.radix_bits != plan->cfg.radix_bits)) {
            drf_plan_destroy(plan);
            plan = nullptr;
            if ((st = build_plan(ctx, n, bytecodes, lens, bounds, best_cfg, &plan))) return st;
        }
    }
    if ((st = capture_plan(plan))) { drf_plan_destroy(plan); return st; }
    *out = plan;
    return DRF_OK;
}

int drf_plan_config(const drf_plan *plan, uint32_t *granularity, uint32_t *radix_items, uint32_t *radix_bits)
{
    if (!plan) return DRF_E_INVALID_ARG;
    if (granularity) *granularity = plan->cfg.granularity;
    if (radix_items) *radix_items = plan->cfg.radix_items;
    if (radix_bits) *radix_bits = plan->host.L.digit_bits;
    return DRF_OK;
}

int drf_plan_specialized(const drf_plan *plan, uint32_t *specialized, char *log, size_t loglen)
{
    if (!plan || !specialized) return DRF_E_INVALID_ARG;
    *specialized = plan->jit ? (plan->dev.jit.static_phases ? (plan->dev.args.range_on ? 3 : 2) : 1) : 0;
    if (log && loglen) {
        std::strncpy(log, plan->jit_log.c_str(), loglen - 1);
        log[loglen - 1] = 0;
    }
    return DRF_OK;
}

int drf_plan_path(const drf_plan *plan, uint32_t *path)
{
    if (!plan || !path) return DRF_E_INVALID_ARG;
    *path = plan->dev.args.path == PATH_TABLE ? DRF_PATH_TABLE : DRF_PATH_SORT;
    return DRF_OK;
}

int drf_plan_launch(drf_plan *plan, void *stream)
{
    if (!plan || !plan->exec) return DRF_E_INVALID_ARG;
    drf_ctx *ctx = plan->ctx;
    cudaSetDevice(ctx->device);
    cudaStream_t s = pick(ctx, stream);
    DeviceBatch &d = plan->dev;
    if (++d.status_launches >= (1ull << 21) && d.status.p) {
        if (cudaMemsetAsync(d.status.p, 0, d.status.cap, s) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError());
        d.status_launches = 0;
    }
    cudaError_t e = cudaGraphLaunch(plan->exec, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    plan->last_stream = s;
    return DRF_OK;
}

int drf_plan_results(drf_plan *plan, drf_result *out)
{
    if (!plan || !out) return DRF_E_INVALID_ARG;
    drf_ctx *ctx = plan->ctx;
    cudaSetDevice(ctx->device);
    cudaStream_t s = plan->last_stream ? plan->last_stream : ctx->stream;
    DeviceBatch &d = plan->dev;
    cudaError_t e;
    if ((e = d.fetch(s, false)) != cudaSuccess || (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(ctx, e);
    const unsigned flags = d.host_ctrl()->flags;
    if (flags & CF_LOOKBACK_TIMEOUT) return fail(ctx, DRF_E_TIMEOUT, "radix look-back gave up waiting");
    if (flags) return fail(ctx, DRF_E_INTERNAL, "device consistency flags " + std::to_string(flags));
    const DevResult *res = d.host_results();
    for (uint32_t i = 0; i < plan->n; i++) to_public(res[i], &out[i]);
    return DRF_OK;
}

int drf_plan_info(const drf_plan *plan, uint64_t *tuples, uint32_t *sort_passes, uint32_t *kernels_per_launch,
                  uint32_t *sort_bits)
{
    if (!plan) return DRF_E_INVALID_ARG;
    const bool table = plan->dev.args.path == PATH_TABLE;
    if (tuples) *tuples = plan->tuples;
    if (sort_passes) *sort_passes = table ? 0 : plan->host.L.passes;
    if (kernels_per_launch) {
        uint32_t widths = plan->dev.args.has_narrow + plan->dev.args.has_wide;
        const uint32_t range = table && plan->dev.args.range_on ? 1 : 0;      // the range pass
        // init, table, (range,) tlist, tscan, witness + finalize (with the
        // range pass the finalize pass is its own kernel)
        if (table && plan->dev.jit.static_phases) *kernels_per_launch = 5 + 2 * range;
        else if (table && plan->dev.args.count_free) *kernels_per_launch = 2 * widths + 4 + range;   // init, 2x interp, tlist, tscan, finalize
        else if (table) *kernels_per_launch = 3 * widths + 5 + range;   // init, 3x interp, scan, tlist, tscan, finalize
        else *kernels_per_launch = 2 * widths + 5 + plan->host.L.passes +   // init, 2x interp, scan, passes, detect, resolve, finalize
                                   (plan->dev.args.range_keys ? 1 : 0);     // (the range accesses' keys)
    }
    if (sort_bits) *sort_bits = plan->host.L.sort_bits;
    return DRF_OK;
}

int drf_plan_keys(const drf_plan *plan, uint64_t *keys)
{
    if (!plan || !keys) return DRF_E_INVALID_ARG;
    *keys = plan->dev.args.path == PATH_TABLE ? 0 : plan->dev.args.nkeys;
    return DRF_OK;
}

int drf_plan_stage_times(drf_plan *plan, const char **names, float *ms, int cap, int *count)
{
    if (!plan || !count) return DRF_E_INVALID_ARG;
    *count = 0;
    if (!plan->profiled) return fail(plan->ctx, DRF_E_INVALID_ARG, "context created without DRF_OPT_PROFILE_STAGES");
    cudaSetDevice(plan->ctx->device);
    cudaStream_t s = plan->last_stream ? plan->last_stream : plan->ctx->stream;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(plan->ctx, e);
    const char *all[kMaxStages];
    int nn = stage_names(all, kMaxStages, plan->host.L.passes, plan->dev.args.path, plan->dev.jit.static_phases,
                         plan->dev.args.count_free != 0, plan->dev.args.range_on != 0);
    int n = std::min(nn, plan->nevents - 1);
    for (int i = 0; i < n && i < cap; i++) {
        float t = 0;
        if ((e = cudaEventElapsedTime(&t, plan->events[i], plan->events[i + 1])) != cudaSuccess) return cuda_fail(plan->ctx, e);
        if (names) names[i] = all[i];
        if (ms) ms[i] = t;
        (*count)++;
    }
    return DRF_OK;
}

int drf_plan_range_tuples(const drf_plan *plan, uint64_t *tuples, uint64_t *updates)
{
    if (!plan || !tuples) return DRF_E_INVALID_ARG;
    *tuples = plan->dev.args.range_on ? plan->host.range_tuples : 0;
    if (updates) {
        *updates = 0;
        if (plan->dev.args.range_on) {
            drf_ctx *ctx = plan->ctx;
            cudaSetDevice(ctx->device);
            cudaStream_t s = plan->last_stream ? plan->last_stream : ctx->stream;
            DeviceBatch &d = const_cast<drf_plan *>(plan)->dev;
            cudaError_t e;
            if ((e = d.fetch(s, true)) != cudaSuccess || (e = cudaStreamSynchronize(s)) != cudaSuccess)
                return cuda_fail(ctx, e);
            *updates = d.host_ctrl()->range_tuples;
        }
    }
    return DRF_OK;
}

void drf_plan_destroy(drf_plan *plan)
{
    if (!plan) return;
    cudaSetDevice(plan->ctx->device);
    if (plan->last_stream) cudaStreamSynchronize(plan->last_stream);
    cudaStreamSynchronize(plan->ctx->stream);
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    for (auto ev : plan->events) cudaEventDestroy(ev);
    delete plan;
}

}  // extern "C"
