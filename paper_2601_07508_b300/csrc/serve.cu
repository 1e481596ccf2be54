// Serving loop: continuous batching of modular products as they arrive.
//
// A worker thread owns the device side.  Clients submit problems (device
// pointers to A, B, C plus p) from any thread and get a ticket.  Each turn the
// worker
//   1. retires finished batches (event query): their requests complete, their
//      workspace returns to the arena, waiters are woken;
//   2. while fewer than max_inflight batches are on the GPU, forms a batch:
//      its head is the queued request with the least word-product work
//      (within the first kScan), or the oldest one once it has waited more
//      than kAgeFactor times its estimated run time (shortest work first
//      with aging: a medium request does not wait behind several large ones,
//      and a large one cannot starve); then later queued requests (in arrival
//      order) whose work is at most kCostRatio times the head's -- all
//      requests of a batch complete together, so a small request is not held
//      back by a much larger batch-mate.  A request joins if its workspace
//      fits in the arena now (admission against the memory budget) and the
//      batch has room,
//      then builds the batch's tables, copies them to the device and launches
//      the batched kernels on the next of its streams -- so requests that
//      arrive while other batches run are admitted as memory frees up, and
//      their work overlaps with the batches already on the device;
//   3. otherwise sleeps briefly (or until a submission arrives).
// Latency of a request = completion observed by the worker - arrival time
// (the submit time, or an earlier scheduled arrival given by the client).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "mwmm_internal.h"

using mwmm::Plan;

namespace {

constexpr uint64_t kStagingBytes = 32ull << 20;  // pinned table staging per stream
constexpr int kScan = 512;                         // queued requests a batch formation looks at
constexpr double kCostRatio = 4.0;                 // batch-mates do at most this much more work than the head
constexpr double kAgeFactor = 3.0;                 // a request waiting this many times its run time goes next
constexpr double kAgeFloor = 1e-3;                 // ... plus this many seconds
constexpr int64_t kDirectItems = 32;                // requests with more work items run their own kernels
constexpr int64_t kMaxTableItems = 8192;            // table items per batch (bounds the host's table building)

uint64_t align256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

// First-fit allocator over [0, size): offsets of 256-byte-aligned regions.
class Arena {
   public:
    void init(uint64_t size) {
        size_ = size;
        free_.clear();
        if (size) free_[0] = size;
        used_ = peak_ = 0;
    }
    bool alloc(uint64_t bytes, uint64_t &off) {
        bytes = align256(bytes ? bytes : 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                off = it->first;
                const uint64_t rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[off + bytes] = rest;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t bytes) {
        bytes = align256(bytes ? bytes : 256);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {  // merge with the next region
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {  // merge with the previous region
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    uint64_t size() const { return size_; }
    uint64_t peak() const { return peak_; }

   private:
    std::map<uint64_t, uint64_t> free_;
    uint64_t size_ = 0, used_ = 0, peak_ = 0;
};

struct Request {
    mwmm_problem prob;
    Plan plan;
    double t_arrival = 0, t_done = 0;
    int state = 0;  // 0 queued, 1 on the GPU, 2 done
    mwmm_status status = MWMM_OK;
    uint64_t ws_off = 0, ws_bytes = 0;
    double flops = 0;
};

struct Inflight {
    std::vector<uint64_t> tickets;
    cudaEvent_t ev = nullptr;
    int slot = 0;
};

}  // namespace

struct mwmm_server_s {
    int form = MWMM_FORM_AUTO;  // AUTO: each request's tensor form (INT8 or CRT) from the planner's cost model
    int max_batch = 64, max_inflight = 2;
    uint8_t *arena_dev = nullptr;
    int *err = nullptr;
    Arena arena;
    std::vector<cudaStream_t> streams;
    std::vector<uint8_t *> staging;  // pinned, one per slot
    std::vector<uint8_t *> dtables;  // device table region, one per slot (part of the budget)
    std::vector<int> slot_busy;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    std::vector<Inflight> inflight;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::chrono::steady_clock::time_point t0;
    // stats
    int64_t submitted = 0, completed = 0, rejected = 0, batches = 0, peak_queue = 0, peak_inflight = 0;
    double flops_done = 0, first_arrival = -1, last_done = 0, batched_requests = 0;
    std::vector<double> latencies;
    mwmm_status worker_error = MWMM_OK;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

// Move finished batches to done (lock held).
bool retire(mwmm_server_s *S) {
    bool any = false;
    for (size_t b = 0; b < S->inflight.size();) {
        Inflight &f = S->inflight[b];
        cudaError_t q = cudaEventQuery(f.ev);
        if (q == cudaErrorNotReady) {
            ++b;
            continue;
        }
        const double t = S->now();
        for (uint64_t tk : f.tickets) {
            Request &r = *S->reqs[tk];
            r.state = 2;
            r.t_done = t;
            if (q != cudaSuccess) r.status = MWMM_ERR_CUDA;
            S->arena.release(r.ws_off, r.ws_bytes);
            S->completed += 1;
            S->flops_done += r.flops;
            S->latencies.push_back(t - r.t_arrival);
            S->last_done = t;
        }
        S->slot_busy[f.slot] = 0;
        cudaEventDestroy(f.ev);
        S->inflight.erase(S->inflight.begin() + (long)b);
        any = true;
    }
    if (any) S->cv_done.notify_all();
    return any;
}

// Form and launch one batch (lock held on entry and exit; released while the
// tables are built).  Returns true if a batch was launched.
bool launch_one(mwmm_server_s *S, std::unique_lock<std::mutex> &lock) {
    if ((int)S->inflight.size() >= S->max_inflight || S->queue.empty()) return false;
    int slot = -1;
    for (int i = 0; i < (int)S->slot_busy.size(); ++i)
        if (!S->slot_busy[i]) {
            slot = i;
            break;
        }
    if (slot < 0) return false;
    // admission: the head, then similar-sized requests in arrival order,
    // while the workspace fits the arena.  The head is the queued request
    // with the least work (among the first kScan), unless the oldest one has
    // waited more than kAgeFactor times its estimated run time: short
    // requests pass long ones, and a long one cannot starve.
    std::vector<uint64_t> tickets;
    uint64_t table_est = 0;
    int64_t table_items = 0;
    auto work = [](const Request &r) {  // word products x 2 m n k
        return (r.plan.form == MWMM_FORM_CRT8 ? (double)r.plan.crt_s : (double)r.plan.u * r.plan.v) * r.flops;
    };
    size_t head = 0;
    {
        const Request &old = *S->reqs[S->queue.front()];
        const double run_s = work(old) / 1.0e15 + 5e-5;  // ~1 PFLOP/s of word products plus launch overhead
        if (S->now() - old.t_arrival <= kAgeFactor * run_s + kAgeFloor) {
            double best = work(old);
            for (size_t qi = 1; qi < S->queue.size() && (int)qi < kScan; ++qi) {
                const double w = work(*S->reqs[S->queue[qi]]);
                if (w < best) {
                    best = w;
                    head = qi;
                }
            }
        }
    }
    if (head != 0) {  // move the head to the front; the others keep their order
        const uint64_t tk = S->queue[head];
        S->queue.erase(S->queue.begin() + (long)head);
        S->queue.push_front(tk);
    }
    const double cap = kCostRatio * work(*S->reqs[S->queue.front()]);
    for (size_t qi = 0; qi < S->queue.size() && (int)qi < kScan && (int)tickets.size() < S->max_batch;) {
        Request &r = *S->reqs[S->queue[qi]];
        if (!tickets.empty() && work(r) > cap) {  // too large for this batch: it waits for its own
            ++qi;
            continue;
        }
        const uint64_t est = 4096 + 96 * (uint64_t)(r.plan.A_rows / 64 + 1) * (r.plan.nkb + 1) * 2 +
                             128 * (uint64_t)r.plan.nsums * r.plan.nkc * (r.plan.A_rows / 128 + 1) *
                                 (r.plan.B_rows / 256 + 1);
        if (table_est + est > kStagingBytes / 2 && !tickets.empty()) break;
        const int64_t ti = mwmm::batch_items(r.plan) > kDirectItems ? 0 : mwmm::batch_items(r.plan);
        if (!tickets.empty() && table_items + ti > kMaxTableItems) {  // keeps the host's table building short
            ++qi;
            continue;
        }
        table_items += ti;
        uint64_t off = 0;
        if (!S->arena.alloc(r.plan.ws_bytes, off)) break;
        r.ws_off = off;
        r.ws_bytes = r.plan.ws_bytes;
        r.state = 1;
        tickets.push_back(S->queue[qi]);
        S->queue.erase(S->queue.begin() + (long)qi);
        table_est += est;
    }
    if (tickets.empty()) return false;
    S->slot_busy[slot] = 1;
    // Large requests (many work items) run the single-product kernels, whose
    // items are computed on the device; the others share the batch's tables,
    // which the worker builds on the host.
    std::vector<Plan> plans, direct;
    std::vector<mwmm_problem> probs, dprobs;
    std::vector<uint8_t *> wsb, dws;
    std::vector<Plan> all_plans;
    std::vector<mwmm_problem> all_probs;
    for (uint64_t tk : tickets) {
        Request &r = *S->reqs[tk];
        const bool dir = mwmm::batch_items(r.plan) > kDirectItems;
        (dir ? direct : plans).push_back(r.plan);
        (dir ? dprobs : probs).push_back(r.prob);
        (dir ? dws : wsb).push_back(S->arena_dev + r.ws_off);
        all_plans.push_back(r.plan);
        all_probs.push_back(r.prob);
    }
    lock.unlock();
    mwmm::BatchTables T;
    mwmm::build_batch_tables(plans.data(), probs.data(), wsb.data(), (int)plans.size(), S->err, T);
    uint64_t off[mwmm::kBatchTables];
    // straight into the slot's pinned staging buffer (free: the slot's previous batch has retired)
    const uint64_t tb = mwmm::pack_batch_tables_to(T, S->staging[slot], kStagingBytes, off);
    lock.lock();
    Inflight f;
    f.tickets = tickets;
    f.slot = slot;
    mwmm_status st = tb > kStagingBytes ? MWMM_ERR_BUDGET : MWMM_OK;
    if (st == MWMM_OK) {
        cudaStream_t s = S->streams[slot];
        lock.unlock();
        cudaError_t e = cudaSuccess;
        if (tb) e = cudaMemcpyAsync(S->dtables[slot], S->staging[slot], tb, cudaMemcpyHostToDevice, s);
        for (size_t i = 0; e == cudaSuccess && i < all_plans.size(); ++i)  // k = 0: C = 0
            if (all_plans[i].m > 0 && all_plans[i].n > 0 && all_plans[i].k == 0)
                e = cudaMemset2DAsync(all_probs[i].C, (size_t)all_probs[i].ldc * 8, 0, (size_t)all_plans[i].n * 8,
                                      (size_t)all_plans[i].m, s);
        for (size_t i = 0; e == cudaSuccess && i < direct.size(); ++i) {
            direct[i].err_dev = S->err;
            e = (cudaError_t)mwmm::launch_product(direct[i], dprobs[i].A, dprobs[i].lda, dprobs[i].B, dprobs[i].ldb,
                                                  dprobs[i].C, dprobs[i].ldc, dws[i], s);
        }
        if (e == cudaSuccess && tb)
            e = (cudaError_t)mwmm::launch_batch_tables(T, S->dtables[slot], off, S->form == MWMM_FORM_FP64,
                                                       mwmm::kTcMaxChunk / mwmm::kTcKB, S->err, s);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(f.ev, s);
        lock.lock();
        if (e != cudaSuccess) st = MWMM_ERR_CUDA;
    }
    if (st != MWMM_OK) {  // fail the batch's requests
        const double t = S->now();
        for (uint64_t tk : tickets) {
            Request &r = *S->reqs[tk];
            r.state = 2;
            r.status = st;
            r.t_done = t;
            S->arena.release(r.ws_off, r.ws_bytes);
        }
        if (f.ev) cudaEventDestroy(f.ev);
        S->slot_busy[slot] = 0;
        S->worker_error = st;
        S->cv_done.notify_all();
        return false;
    }
    S->inflight.push_back(f);
    S->batches += 1;
    S->batched_requests += (double)tickets.size();
    S->peak_inflight = std::max<int64_t>(S->peak_inflight, (int64_t)S->inflight.size());
    return true;
}

void worker_main(mwmm_server_s *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lock(S->mu);
    for (;;) {
        bool progress = retire(S);
        while (launch_one(S, lock)) progress = true;
        if (S->stop && S->queue.empty() && S->inflight.empty()) break;
        if (!progress) {
            if (S->inflight.empty())
                S->cv_work.wait_for(lock, std::chrono::milliseconds(2));
            else {
                lock.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lock.lock();
            }
        }
    }
}

}  // namespace

extern "C" {

mwmm_status mwmm_serve_create(mwmm_server_t *out, size_t mem_budget_bytes, int max_inflight,
                              const mwmm_serve_opts *opts) {
    if (!out) return MWMM_ERR_ARG;
    *out = nullptr;
    const int slots = max_inflight > 0 ? max_inflight : 2;
    // the per-slot table regions come out of the budget
    if (mem_budget_bytes < (uint64_t)slots * kStagingBytes + (16u << 20)) return MWMM_ERR_BUDGET;
    mwmm_server_s *S = new (std::nothrow) mwmm_server_s();
    if (!S) return MWMM_ERR_NOMEM;
    S->max_inflight = slots;
    const uint64_t arena_bytes = mem_budget_bytes - (uint64_t)slots * kStagingBytes;
    if (opts) {
        if (opts->form < MWMM_FORM_AUTO || opts->form > MWMM_FORM_CRT8) {
            delete S;
            return MWMM_ERR_ARG;
        }
        if (opts->max_batch > 0) S->max_batch = opts->max_batch;
        S->form = opts->form;
    }
    S->t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaGetDevice(&S->device);
    if (e == cudaSuccess) e = cudaMalloc(&S->arena_dev, mem_budget_bytes);  // arena, then table regions
    if (e == cudaSuccess) e = cudaMalloc(&S->err, 256);
    if (e == cudaSuccess) e = cudaMemset(S->err, 0, 256);
    if (e == cudaSuccess) e = (cudaError_t)mwmm::prepare_kernel_attributes();
    for (int i = 0; e == cudaSuccess && i < S->max_inflight; ++i) {
        cudaStream_t s;
        uint8_t *h = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) S->streams.push_back(s);
        if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&h), kStagingBytes, cudaHostAllocDefault);
        if (e == cudaSuccess) S->staging.push_back(h);
        if (e == cudaSuccess) S->dtables.push_back(S->arena_dev + arena_bytes + (uint64_t)i * kStagingBytes);
    }
    if (e != cudaSuccess) {
        for (auto s : S->streams) cudaStreamDestroy(s);
        for (auto h : S->staging) cudaFreeHost(h);
        if (S->arena_dev) cudaFree(S->arena_dev);
        if (S->err) cudaFree(S->err);
        delete S;
        return e == cudaErrorMemoryAllocation ? MWMM_ERR_NOMEM : MWMM_ERR_CUDA;
    }
    S->arena.init(arena_bytes);
    S->slot_busy.assign(S->max_inflight, 0);
    S->worker = std::thread(worker_main, S);
    *out = S;
    return MWMM_OK;
}

double mwmm_serve_now(mwmm_server_t S) { return S ? S->now() : 0.0; }

mwmm_status mwmm_serve_submit(mwmm_server_t S, const mwmm_problem *prob, double t_arrival, uint64_t *ticket) {
    if (!S || !prob || !ticket) return MWMM_ERR_ARG;
    *ticket = 0;
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) return MWMM_ERR_NOMEM;
    mwmm_plan_opts o;
    std::memset(&o, 0, sizeof(o));
    o.ksplit = 1;    // requests run as batched tiles over the whole K range
    o.tc_pair = -1;  // one-CTA tiles, also for the large requests launched
                     // directly: pair clusters wait for two free SMs beside the
                     // small batches (measured: 0.8 x load p99 4.6-5.7 ms with
                     // them against 3.5-3.6 ms, saturation level)
    o.tc_fused = 1;  // and write diagonal sums for the batched recombination
    o.tc_fill = 1;   // batches of requests share the SMs
    const int form = S->form != MWMM_FORM_AUTO ? S->form : mwmm::choose_tensor_form(prob->m, prob->n, prob->k, prob->p);
    mwmm_status st = mwmm::make_plan(&r->plan, prob->m, prob->n, prob->k, prob->p, 0, 0, form, &o);
    if (st != MWMM_OK) return st;
    const Plan &pl = r->plan;
    if (pl.m > 0 && pl.n > 0 &&
        (!prob->C || prob->ldc < pl.n || (pl.k > 0 && (!prob->A || !prob->B || prob->lda < pl.k || prob->ldb < pl.n))))
        return MWMM_ERR_ARG;
    r->prob = *prob;
    r->flops = 2.0 * pl.m * pl.n * pl.k;
    std::lock_guard<std::mutex> lock(S->mu);
    // A request whose workspace exceeds the whole arena can never run.
    if (align256(pl.ws_bytes) > S->arena.size()) {
        S->rejected += 1;
        return MWMM_ERR_BUDGET;
    }
    const double t = S->now();
    r->t_arrival = (t_arrival >= 0 && t_arrival <= t) ? t_arrival : t;
    if (S->first_arrival < 0 || r->t_arrival < S->first_arrival) S->first_arrival = r->t_arrival;
    const uint64_t tk = S->next_ticket++;
    S->reqs[tk] = std::move(r);
    S->queue.push_back(tk);
    S->submitted += 1;
    S->peak_queue = std::max<int64_t>(S->peak_queue, (int64_t)S->queue.size());
    *ticket = tk;
    S->cv_work.notify_one();
    return MWMM_OK;
}

mwmm_status mwmm_serve_poll(mwmm_server_t S, uint64_t ticket) {
    if (!S) return MWMM_ERR_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return MWMM_ERR_ARG;
    return it->second->state == 2 ? it->second->status : MWMM_ERR_BUSY;
}

mwmm_status mwmm_serve_wait(mwmm_server_t S, uint64_t ticket, int timeout_ms) {
    if (!S) return MWMM_ERR_ARG;
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return MWMM_ERR_ARG;
    Request *r = it->second.get();
    auto done = [&] { return r->state == 2; };
    if (timeout_ms < 0) S->cv_done.wait(lock, done);
    else if (!S->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), done)) return MWMM_ERR_TIMEOUT;
    return r->status;
}

mwmm_status mwmm_serve_latency(mwmm_server_t S, uint64_t ticket, double *seconds) {
    if (!S || !seconds) return MWMM_ERR_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return MWMM_ERR_ARG;
    if (it->second->state != 2) return MWMM_ERR_BUSY;
    *seconds = it->second->t_done - it->second->t_arrival;
    return MWMM_OK;
}

mwmm_status mwmm_serve_stats(mwmm_server_t S, mwmm_serve_report *o) {
    if (!S || !o) return MWMM_ERR_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    std::memset(o, 0, sizeof(*o));
    o->submitted = S->submitted;
    o->completed = S->completed;
    o->rejected = S->rejected;
    o->batches = S->batches;
    o->mean_batch = S->batches ? S->batched_requests / (double)S->batches : 0.0;
    o->peak_queue = S->peak_queue;
    o->peak_inflight = S->peak_inflight;
    o->peak_bytes = S->arena.peak();
    o->budget_bytes = S->arena.size() + (uint64_t)S->dtables.size() * kStagingBytes;
    o->flops_2mnk = S->flops_done;
    o->busy_s = S->first_arrival >= 0 ? S->last_done - S->first_arrival : 0.0;
    o->gops = o->busy_s > 0 ? S->flops_done / o->busy_s / 1e9 : 0.0;
    if (!S->latencies.empty()) {
        std::vector<double> l = S->latencies;
        std::sort(l.begin(), l.end());
        auto pct = [&](double q) {
            size_t i = (size_t)(q * (double)(l.size() - 1) + 0.5);
            return l[std::min(i, l.size() - 1)] * 1e3;
        };
        o->p50_ms = pct(0.50);
        o->p99_ms = pct(0.99);
        o->max_ms = l.back() * 1e3;
        double s = 0;
        for (double x : l) s += x;
        o->mean_ms = s / (double)l.size() * 1e3;
    }
    int flags[2] = {0, 0};
    if (cudaMemcpy(flags, S->err, sizeof(flags), cudaMemcpyDeviceToHost) == cudaSuccess && flags[0])
        return MWMM_ERR_TIMEOUT;
    return S->worker_error;
}

mwmm_status mwmm_serve_reset_stats(mwmm_server_t S) {
    if (!S) return MWMM_ERR_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    S->submitted = S->completed = S->rejected = S->batches = S->peak_queue = S->peak_inflight = 0;
    S->flops_done = 0;
    S->first_arrival = -1;
    S->last_done = 0;
    S->batched_requests = 0;
    S->latencies.clear();
    for (auto it = S->reqs.begin(); it != S->reqs.end();)  // forget finished requests
        it = it->second->state == 2 ? S->reqs.erase(it) : std::next(it);
    return MWMM_OK;
}

void mwmm_serve_destroy(mwmm_server_t S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    for (auto s : S->streams) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    for (auto h : S->staging) cudaFreeHost(h);
    if (S->arena_dev) cudaFree(S->arena_dev);
    if (S->err) cudaFree(S->err);
    delete S;
}

}  // extern "C"
