// Continuous-batching check server.
//
// Callers submit checks from any thread; each request is validated and
// lowered in the caller's thread (host work overlaps the GPU), then queued.
// Two worker threads, each with its own CUDA stream and device buffers, pull
// rounds from the queue: a round takes requests in arrival order while the
// sum of their access-tuple bounds (16 bytes of sort buffers per tuple) fits
// the round budget and the protocol cap.  While one round waits on the GPU
// the other worker forms and launches the next one, so requests that arrive
// mid-round are admitted as soon as a worker frees up, and two rounds'
// kernels overlap on the device.  A round is one pass of the batched
// pipeline, so every result equals what drf_check returns for the request
// alone.
#include "server.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>
#include <unordered_set>

#include "engine.h"

namespace drf {

namespace {
using Clock = std::chrono::steady_clock;
}

// A spin-wait hint to the core.
inline void cpu_relax()
{
#if defined(__x86_64__) || defined(__i386__)
    __builtin_ia32_pause();
#endif
}

class Server {
public:
    Server(drf_ctx *ctx, const drf_server_opts &o) : ctx_(ctx), opts_(o)
    {
        if (!opts_.max_round_tuples) opts_.max_round_tuples = 1ull << 26;
        if (!opts_.max_round_protocols) opts_.max_round_protocols = 4096;
        if (!opts_.max_queue) opts_.max_queue = 1u << 20;
    }

    int start()
    {
        for (int i = 0; i < kWorkers; i++) {
            std::unique_ptr<Lane> l(new Lane);
            if (cudaStreamCreateWithFlags(&l->s, cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                return S_CUDA;
            }
            l->dev.limit = ctx_->opts.max_device_bytes;
            l->dev.path_pref = path_pref_of(ctx_->opts);
            lanes_.push_back(std::move(l));
        }
        for (int i = 0; i < kWorkers; i++) workers_.emplace_back([this, i] { work(i); });
        return S_OK;
    }

    ~Server()
    {
        stop();
        cudaSetDevice(ctx_->device);
        for (auto &l : lanes_) {
            if (l->s) { cudaStreamSynchronize(l->s); cudaStreamDestroy(l->s); }
        }
    }

    void stop()
    {
        {
            std::lock_guard<std::mutex> g(mu_);
            stopping_ = true;
        }
        cv_work_.notify_all();
        for (auto &t : workers_) if (t.joinable()) t.join();
        workers_.clear();
    }

    int submit(const uint8_t *bc, size_t len, const drf_bounds *b, uint64_t *ticket)
    {
        if (!bc || !b || !ticket) return S_INVALID_ARG;
        std::unique_ptr<Request> r(new Request);
        r->t_submit = Clock::now();
        // cut a request for its share of a round: alone (no backlog) as finely
        // as a lone check, whose latency is its longest lane; behind a backlog
        // it will share its round with the requests ahead of it, and coarser
        // items keep preparation (on the caller's thread) cheap
        size_t backlog;
        {
            std::lock_guard<std::mutex> g(mu_);
            backlog = pending_.size();
        }
        // (the desired warp items are rounded down to a power of two, so that
        // a protocol seen before reuses its prepared program from the
        // context's cache at most backlog levels)
        PrepareOpts po;
        uint64_t want = std::max<uint64_t>((uint64_t)ctx_->sms * 2, (uint64_t)ctx_->sms * 128 / (1 + backlog));
        while (want & (want - 1)) want &= want - 1;
        po.desired_warp_items = want;
        Error e;
        r->prep = ctx_->prep_cache.get(bc, len, b, po, e);
        std::lock_guard<std::mutex> g(mu_);
        if (stopping_) return S_BUSY;
        if (queue_.size() >= opts_.max_queue) return S_BUSY;
        r->ticket = next_ticket_++;
        *ticket = r->ticket;
        if (!e.ok()) {                      // rejected up front: done at once
            Done d{};
            d.r.status = e.status;
            d.r.verdict = -1;
            done_[r->ticket] = d;
            cv_done_.notify_all();
            return S_OK;
        }
        pending_.insert(r->ticket);
        queue_.push_back(std::move(r));
        queued_.store(queue_.size(), std::memory_order_release);
        cv_work_.notify_one();
        return S_OK;
    }

    int poll(uint64_t ticket, drf_result *out, int64_t timeout_us, uint64_t *latency_ns)
    {
        std::unique_lock<std::mutex> g(mu_);
        auto ready = [&] { return done_.count(ticket) != 0; };
        if (!ready()) {
            if (!pending_.count(ticket)) return S_NOT_FOUND;
            if (timeout_us < 0) cv_done_.wait(g, ready);
            else if (!cv_done_.wait_for(g, std::chrono::microseconds(timeout_us), ready)) return S_TIMEOUT;
        }
        auto it = done_.find(ticket);
        *out = it->second.r;
        if (latency_ns) *latency_ns = it->second.latency_ns;
        done_.erase(it);
        return S_OK;
    }

    void stats(uint64_t *rounds, uint64_t *completed, uint32_t *max_round)
    {
        std::lock_guard<std::mutex> g(mu_);
        if (rounds) *rounds = rounds_;
        if (completed) *completed = completed_;
        if (max_round) *max_round = max_round_;
    }

private:
    static constexpr int kWorkers = 2;

    struct Request {
        uint64_t ticket = 0;
        std::shared_ptr<const Prepared> prep;
        Clock::time_point t_submit;
    };
    struct Done {
        drf_result r;
        uint64_t latency_ns;
    };
    struct Lane {
        DeviceBatch dev;
        BatchHost host;               // host image of the lane's last round (keeps its capacity)
        cudaStream_t s = nullptr;
    };

    drf_ctx *ctx_;
    drf_server_opts opts_;
    std::mutex mu_;
    std::condition_variable cv_work_, cv_done_;
    std::deque<std::unique_ptr<Request>> queue_;
    std::unordered_map<uint64_t, Done> done_;
    std::unordered_set<uint64_t> pending_;
    uint64_t next_ticket_ = 1;
    bool stopping_ = false;
    std::vector<std::thread> workers_;
    std::vector<std::unique_ptr<Lane>> lanes_;
    std::atomic<size_t> queued_{0};   // queue_.size(), for polling workers (written under mu_)
    uint64_t rounds_ = 0, completed_ = 0;
    uint32_t max_round_ = 0;

    void finish(const std::vector<std::unique_ptr<Request>> &round, const std::vector<drf_result> &res)
    {
        auto now = Clock::now();
        std::lock_guard<std::mutex> g(mu_);
        for (size_t i = 0; i < round.size(); i++) {
            Done d;
            d.r = res[i];
            d.latency_ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(now - round[i]->t_submit).count();
            done_[round[i]->ticket] = d;
            pending_.erase(round[i]->ticket);
        }
        completed_ += round.size();
        cv_done_.notify_all();
    }

    void work(int id)
    {
        cudaSetDevice(ctx_->device);
        Lane &lane = *lanes_[id];
        while (true) {
            std::vector<std::unique_ptr<Request>> round;
            {
                std::unique_lock<std::mutex> g(mu_);
                // an idle worker first polls the queue for opts_.poll_us (its
                // core stays awake: a request arriving meanwhile starts at once),
                // then sleeps until notified
                bool polled = opts_.poll_us == 0;
                while (!stopping_ && queue_.empty()) {
                    if (!polled) {
                        g.unlock();
                        const auto until = Clock::now() + std::chrono::microseconds(opts_.poll_us);
                        while (queued_.load(std::memory_order_acquire) == 0 && Clock::now() < until) cpu_relax();
                        g.lock();
                        polled = true;
                        continue;
                    }
                    cv_work_.wait(g);
                }
                if (queue_.empty()) return;                 // stopping and drained
                uint64_t budget = 0;
                while (!queue_.empty() && round.size() < opts_.max_round_protocols) {
                    uint64_t tb = queue_.front()->prep->tuple_bound();
                    if (!round.empty() && budget + tb > opts_.max_round_tuples) break;
                    budget += tb;
                    round.push_back(std::move(queue_.front()));
                    queue_.pop_front();
                    queued_.store(queue_.size(), std::memory_order_release);
                }
                rounds_++;
                if (round.size() > max_round_) max_round_ = (uint32_t)round.size();
                if (!queue_.empty()) cv_work_.notify_one();   // let the other worker take the rest
            }
            std::vector<drf_result> res(round.size());
            run_round(lane, round, res);
            finish(round, res);
        }
    }

    // A round's protocols [lo, hi) as one batch.  A batch that fails as a
    // whole for want of room -- its combined key wider than 64 bits, its
    // buffers beyond the context's device-memory cap, its owner table beyond
    // the limit -- is run again in halves, down to single protocols, so that
    // every request gets the result it would get alone, whatever it was
    // mixed with.
    void run_group(Lane &lane, const std::vector<const Prepared *> &ps, size_t lo, size_t hi,
                   std::vector<drf_result> &res)
    {
        BatchHost &bh = lane.host;
        std::string err;
        std::vector<DevResult> dr;
        std::vector<const Prepared *> part(ps.begin() + (long)lo, ps.begin() + (long)hi);
        Error e = pack_batch(part, bh, true, ctx_->opts.radix_bits, range_min_once(ctx_->opts));
        int st = e.status;
        if (e.ok()) st = run_batch(lane.dev, ctx_->sms, lane.s, bh, dr, err);
        if (st == S_OK) {
            for (size_t i = lo; i < hi; i++) to_public(dr[i - lo], &res[i]);
            return;
        }
        if (hi - lo > 1 && (st == S_KEY_TOO_WIDE || st == S_NOMEM || st == S_LIMIT)) {
            const size_t mid = lo + (hi - lo) / 2;
            run_group(lane, ps, lo, mid, res);
            run_group(lane, ps, mid, hi, res);
            return;
        }
        for (size_t i = lo; i < hi; i++) { res[i] = drf_result{}; res[i].status = st; res[i].verdict = -1; }
    }

    void run_round(Lane &lane, const std::vector<std::unique_ptr<Request>> &round, std::vector<drf_result> &res)
    {
        std::vector<const Prepared *> ps;
        for (auto &r : round) ps.push_back(r->prep.get());
        run_group(lane, ps, 0, ps.size(), res);
    }
};

}  // namespace drf

using drf::Server;

extern "C" {

int drf_server_start(drf_ctx *ctx, const drf_server_opts *opts)
{
    if (!ctx) return DRF_E_INVALID_ARG;
    if (ctx->server) return DRF_E_BUSY;
    if (cudaSetDevice(ctx->device) != cudaSuccess) { cudaGetLastError(); return DRF_E_CUDA; }
    drf_server_opts o{};
    if (opts) o = *opts;
    if (o.reserved || o.poll_us > 1000000u) return DRF_E_INVALID_ARG;   // polls of at most a second
    Server *s = new Server(ctx, o);
    int st = s->start();
    if (st) { delete s; return st; }
    ctx->server = s;
    return DRF_OK;
}

int drf_server_submit(drf_ctx *ctx, const uint8_t *bytecode, size_t len, const drf_bounds *bounds, uint64_t *ticket)
{
    if (!ctx) return DRF_E_INVALID_ARG;
    if (!ctx->server) return DRF_E_BUSY;
    return static_cast<Server *>(ctx->server)->submit(bytecode, len, bounds, ticket);
}

int drf_server_poll(drf_ctx *ctx, uint64_t ticket, drf_result *out, int64_t timeout_us, uint64_t *latency_ns)
{
    if (!ctx || !out) return DRF_E_INVALID_ARG;
    if (!ctx->server) return DRF_E_BUSY;
    return static_cast<Server *>(ctx->server)->poll(ticket, out, timeout_us, latency_ns);
}

int drf_server_stats(drf_ctx *ctx, uint64_t *rounds, uint64_t *completed, uint32_t *max_round)
{
    if (!ctx) return DRF_E_INVALID_ARG;
    if (!ctx->server) return DRF_E_BUSY;
    static_cast<Server *>(ctx->server)->stats(rounds, completed, max_round);
    return DRF_OK;
}

int drf_server_stop(drf_ctx *ctx)
{
    if (!ctx) return DRF_E_INVALID_ARG;
    if (!ctx->server) return DRF_OK;
    Server *s = static_cast<Server *>(ctx->server);
    s->stop();
    delete s;
    ctx->server = nullptr;
    return DRF_OK;
}

}  // extern "C"
