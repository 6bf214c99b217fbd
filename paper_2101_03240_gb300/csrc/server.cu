// server.cu -- the continuous-batching request loop of include/ibip.h
// (ibip_server_*): invasion jobs (Section 2.1, with the trapping of Section
// 2.2.3 and the curve of Sections 2.2.1-2.2.2) admitted by device memory.
//
// Design
//   - One device arena of the whole memory budget, allocated once.  A host
//     first-fit allocator hands each admitted job one contiguous piece of
//     ibip_job_footprint bytes; the job's scratch is carved from that piece
//     (the slot context runs in arena mode) and stays resident until the job
//     completes, when the piece is returned and merged with its free
//     neighbours.
//   - max_slots worker threads, each driving its own context and
//     non-blocking stream.  Jobs wait in arrival order; whenever a slot is
//     idle and the head job's piece can be carved, the head is admitted.  No
//     job overtakes an earlier one, and a job that fits the arena is always
//     admitted once the jobs ahead of it have run.
//   - The invasion of a job is one persistent CTA, so the jobs in flight run
//     side by side on different SMs; their EDT, rank, trapping and curve
//     kernels interleave on the other streams.  Trapping uses the per-round
//     launches of the widest-path propagation, never a cooperative grid,
//     whose residency could not be guaranteed beside other streams' kernels,
//     nor its work queue, whose resident blocks would hold the SMs.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace {

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

int64_t up256(int64_t b) { return (b + 255) & ~(int64_t)255; }

// Scratch words of the recursive scan for n inputs (mirrors scan.cu).
int64_t scan_work_bytes(int64_t n)
{
    constexpr int64_t kPerBlock = 4096;
    int64_t need = 16;
    for (int64_t m = (n + kPerBlock - 1) / kPerBlock; m > 1; m = (m + kPerBlock - 1) / kPerBlock) need += m * 2;
    return need * 4;
}

// First-fit allocator of byte ranges of [0, size), free ranges merged.
class RangeAlloc {
public:
    explicit RangeAlloc(size_t size) : size_(size)
    {
        if (size) free_[0] = size;
    }
    bool alloc(size_t n, size_t *off)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n, o2 = it->first + n;
            free_.erase(it);
            if (rest) free_[o2] = rest;
            used_ += n;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t size() const { return size_; }

private:
    size_t size_, used_ = 0;
    std::map<size_t, size_t> free_;   // offset -> length
};

struct Ticket {
    ibip_job job;
    ibip_result res;
    int done = 0;
};

}  // namespace

struct ibip_server {
    int device = 0;
    char *arena = nullptr;
    RangeAlloc alloc{0};
    std::mutex mu;
    std::condition_variable cv_slots, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Ticket> tickets;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<ibip_ctx *> ctxs;
    std::vector<std::thread> threads;
    int64_t submitted = 0, completed = 0, running = 0, peak_running = 0, peak_bytes = 0;
};

extern "C" int64_t ibip_job_footprint(ibip_dims d, int with_dt2)
{
    if (d.nx < 1 || d.ny < 1 || d.nz < 1) return -1;
    const int64_t N = nvox(d);
    int64_t b = 0;
    auto add = [&](int64_t x) { b += up256(x > 16 ? x : 16); };
    if (with_dt2) add(4 * N);   // dt2
    add(2 * N);                 // EDT pass-z distances
    add(4 * N);                 // EDT pass-y partial sums
    add((int64_t)kSmallBytes);
    // invasion set-up, with the pore count bounded by N
    const int64_t nl0 = (N + 63) / 64, nl1 = (nl0 + 63) / 64, nl2 = (nl1 + 63) / 64, nl3 = (nl2 + 63) / 64;
    add(4 * N);                                                  // rank
    add(8 * N);                                                  // (idx, dt2) by rank
    add((int64_t)d.nx * d.ny * ((d.nz + 31) / 32) * 4);          // available bit-plane
    add((int64_t)d.nx * d.ny * ((d.nz + 31) / 32) * 4);          // queued bit-plane
    add((nl0 + nl1 + nl2 + nl3) * 8);                            // frontier bitmap
    add(8 * N + 64);                                             // overflow work lists
    const int64_t maxd = (int64_t)(d.nx - 1) * (d.nx - 1) + (int64_t)(d.ny - 1) * (d.ny - 1) +
                         (int64_t)(d.nz - 1) * (d.nz - 1);
    add(4 * (maxd + 2));                                         // bucket ids by dt2
    int64_t mat = N / 4 > (1 << 20) ? N / 4 : (1 << 20);
    if (maxd + 1 > mat) mat = maxd + 1;
    add(4 * mat);                                                // (bucket, chunk) counts
    int64_t nscan = mat > maxd + 2 ? mat : maxd + 2;
    if (N + 2 > nscan) nscan = N + 2;
    for (int q = 0; q < 3; q++) add(scan_work_bytes(nscan));     // scan work, regrown at most thrice
    // trapping: widest-path field, tile lists and round counters
    add(4 * N);
    const int64_t nt = (int64_t)((d.nx + 3) / 4) * ((d.ny + 7) / 8) * ((d.nz + 31) / 32);
    add(256 + (3 * nt + 2 * ((1 << 16) + 2) + 4) * 4);
    // curve: per-step histogram (steps <= pore voxels <= N)
    add(4 * (N + 2));
    return b;
}

namespace {

void slot_main(ibip_server *S, int slot)
{
    ibip_ctx *ctx = S->ctxs[slot];
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        // admit the head job when its piece of the arena can be carved
        size_t off = 0, bytes = 0;
        uint64_t t = 0;
        S->cv_slots.wait(lk, [&] {
            if (S->queue.empty()) return S->stop;
            const Ticket &h = S->tickets[S->queue.front()];
            bytes = (size_t)ibip_job_footprint(h.job.dims, h.job.dt2 == nullptr);
            return S->alloc.alloc(bytes, &off);
        });
        if (S->queue.empty()) return;   // stopping, nothing left
        t = S->queue.front();
        S->queue.pop_front();
        Ticket &tk = S->tickets[t];
        ibip_job job = tk.job;
        tk.res.t_start_ns = now_ns();
        tk.res.slot = slot;
        tk.res.mem_reserved = (int64_t)bytes;
        S->running++;
        if (S->running > S->peak_running) S->peak_running = S->running;
        if ((int64_t)S->alloc.used() > S->peak_bytes) S->peak_bytes = (int64_t)S->alloc.used();
        // another slot may admit the next job at once
        S->cv_slots.notify_all();
        lk.unlock();

        ctx->arena = S->arena + off;
        ctx->arena_size = bytes;
        ctx->arena_used = 0;
        for (int i = 0; i < SC_NSLOTS; i++) { ctx->slot[i] = nullptr; ctx->slot_bytes[i] = 0; }
        const int st = ibip_run_job(ctx, job);
        // an early error return may leave kernels queued that still write
        // into this job's piece: drain the stream before the piece is freed
        ibip_sync(ctx, ctx->stream);
        if (st == IBIP_ERR_CUDA) cudaGetLastError();
        const int64_t t_end = now_ns();
        const int64_t used = (int64_t)ctx->arena_used;
        for (int i = 0; i < SC_NSLOTS; i++) { ctx->slot[i] = nullptr; ctx->slot_bytes[i] = 0; }

        lk.lock();
        S->alloc.release(off, bytes);
        Ticket &tk2 = S->tickets[t];
        tk2.res.status = st;
        tk2.res.n_steps = job.n_steps;
        tk2.res.t_end_ns = t_end;
        tk2.res.mem_used = used;
        tk2.done = 1;
        S->running--;
        S->completed++;
        S->cv_done.notify_all();
        S->cv_slots.notify_all();
    }
}

}  // namespace

extern "C" {

int ibip_server_create(ibip_server **out, ibip_ctx *ctx, size_t mem_budget, int max_slots)
{
    if (!out) return IBIP_ERR_ARG;
    *out = nullptr;
    if (!ctx || max_slots < 1 || max_slots > 128 || mem_budget < 4096) return IBIP_ERR_ARG;
    ibip_server *S = new (std::nothrow) ibip_server;
    if (!S) return IBIP_ERR_OOM;
    S->device = ctx->device;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    int st = IBIP_OK;
    mem_budget &= ~(size_t)255;
    if (cudaMalloc((void **)&S->arena, mem_budget) != cudaSuccess) {
        cudaGetLastError();
        S->arena = nullptr;
        st = IBIP_ERR_OOM;
    }
    S->alloc = RangeAlloc(S->arena ? mem_budget : 0);
    // every slot's wide kernels (EDT, rank sort, widest path, curve) queue
    // at the device's lowest stream priority and its one-CTA invasion at the
    // highest: when an SM frees up, a waiting invasion is placed before more
    // blocks of the other jobs' wide kernels
    int prio_low = 0, prio_high = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess) {
        cudaGetLastError();
        prio_low = prio_high = 0;
    }
    for (int i = 0; st == IBIP_OK && i < max_slots; i++) {
        ibip_ctx *c = nullptr;
        cudaStream_t s = nullptr, si = nullptr;
        cudaEvent_t ev = nullptr, evb = nullptr;
        if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, prio_low) != cudaSuccess) {
            cudaGetLastError();
            st = IBIP_ERR_CUDA;
            break;
        }
        if (cudaStreamCreateWithPriority(&si, cudaStreamNonBlocking, prio_high) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&evb, cudaEventDisableTiming | cudaEventBlockingSync) != cudaSuccess) {
            cudaGetLastError();
            if (ev) cudaEventDestroy(ev);
            if (si) cudaStreamDestroy(si);
            cudaStreamDestroy(s);
            st = IBIP_ERR_CUDA;
            break;
        }
        st = ibip_create(&c, S->device, s);
        if (st) { cudaStreamDestroy(s); cudaStreamDestroy(si); cudaEventDestroy(ev); cudaEventDestroy(evb); break; }
        c->no_coop = 1;
        c->stream_inv = si;   // owned by the context from here on
        c->ev_inv = ev;
        c->ev_block = evb;
        S->ctxs.push_back(c);
    }
    if (st == IBIP_OK) {
        try {
            for (int i = 0; i < max_slots; i++) S->threads.emplace_back(slot_main, S, i);
        } catch (...) {
            st = IBIP_ERR_CUDA;
        }
    }
    if (prev >= 0) cudaSetDevice(prev);
    if (st) {
        ibip_server_destroy(S);
        return st;
    }
    *out = S;
    return IBIP_OK;
}

int ibip_server_destroy(ibip_server *S)
{
    if (!S) return IBIP_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_slots.notify_all();
    for (auto &t : S->threads) t.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    for (ibip_ctx *c : S->ctxs) {
        cudaStream_t s = c->stream;
        c->arena = nullptr;
        for (int i = 0; i < SC_NSLOTS; i++) c->slot[i] = nullptr;
        ibip_destroy(c);
        cudaStreamDestroy(s);
    }
    if (S->arena) cudaFree(S->arena);
    if (prev >= 0) cudaSetDevice(prev);
    delete S;
    return IBIP_OK;
}

int ibip_server_submit(ibip_server *S, const ibip_job *job, uint64_t *h_ticket)
{
    if (!S || !job || !h_ticket) return IBIP_ERR_ARG;
    if (!ibip_job_valid(*job)) return IBIP_ERR_ARG;
    const int64_t need = ibip_job_footprint(job->dims, job->dt2 == nullptr);
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return IBIP_ERR_ARG;
    if (need < 0 || (size_t)need > S->alloc.size()) return IBIP_ERR_OOM;
    const uint64_t t = S->next_ticket++;
    Ticket &tk = S->tickets[t];
    tk.job = *job;
    tk.res = ibip_result{};
    tk.res.status = IBIP_OK;
    tk.res.slot = -1;
    tk.res.t_submit_ns = now_ns();
    S->queue.push_back(t);
    S->submitted++;
    *h_ticket = t;
    S->cv_slots.notify_all();
    return IBIP_OK;
}

int ibip_server_wait(ibip_server *S, uint64_t ticket, int64_t timeout_us, int *h_done, ibip_result *h_result)
{
    if (!S || !h_done) return IBIP_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return IBIP_ERR_ARG;
    auto ready = [&] { return S->tickets[ticket].done != 0; };
    if (timeout_us < 0) S->cv_done.wait(lk, ready);
    else if (timeout_us > 0) S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    const Ticket &tk = S->tickets[ticket];
    *h_done = tk.done;
    if (tk.done && h_result) *h_result = tk.res;
    return IBIP_OK;
}

int ibip_server_poll(ibip_server *S, uint64_t ticket, int *h_done, ibip_result *h_result)
{
    return ibip_server_wait(S, ticket, 0, h_done, h_result);
}

int ibip_server_stats(ibip_server *S, int64_t *h, int n)
{
    if (!S || !h || n < 0) return IBIP_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    int64_t launches = 0;
    for (const ibip_ctx *c : S->ctxs) launches += c->launches;
    const int64_t v[9] = {S->submitted, S->completed, S->running, (int64_t)S->queue.size(),
                          (int64_t)S->alloc.used(), (int64_t)S->alloc.size(), S->peak_running, S->peak_bytes,
                          launches};
    for (int i = 0; i < n && i < 9; i++) h[i] = v[i];
    return IBIP_OK;
}

}  // extern "C"
