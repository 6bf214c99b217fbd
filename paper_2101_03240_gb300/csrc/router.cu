// router.cu -- request routing over several continuous-batching servers
// (include/ibip.h, ibip_router_*): serving replicas on several GPUs.
//
// The invasion of one image is a serial chain of steps (Section 2.1: each
// step's sphere depends on the previous step's stamp), so several GPUs
// serve a request stream by taking whole requests: one ibip_server per
// replica (a device, possibly listed more than once), no collective, no
// peer memory.  Each request goes to the replica with the least
// outstanding work (voxels of the jobs submitted to it and not yet seen
// complete) among those whose arena can hold the job; ties go to the lowest
// replica index.  The caller places the job's buffers on the chosen
// replica's device (ibip_router_route, then ibip_router_submit).
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace {

struct Replica {
    int device = 0;
    ibip_ctx *ctx = nullptr;
    ibip_server *srv = nullptr;
    int64_t capacity = 0;                           // arena bytes
    int64_t load = 0;                               // outstanding voxels
    int64_t routed = 0;                             // jobs submitted so far
    std::unordered_map<uint64_t, int64_t> pending;  // server ticket -> voxels, not yet seen complete
};

}  // namespace

struct ibip_router {
    std::mutex mu;
    std::vector<Replica> reps;
    // router ticket -> (replica, server ticket)
    std::unordered_map<uint64_t, std::pair<int, uint64_t>> tickets;
    uint64_t next_ticket = 1;
};

namespace {

// drops the completed jobs from a replica's outstanding work (mu held)
void refresh(Replica &R)
{
    for (auto it = R.pending.begin(); it != R.pending.end();) {
        int done = 0;
        if (ibip_server_poll(R.srv, it->first, &done, nullptr) == IBIP_OK && done) {
            R.load -= it->second;
            it = R.pending.erase(it);
        } else {
            ++it;
        }
    }
}

}  // namespace

extern "C" {

int ibip_route_pick(int n, const int64_t *h_load, const int64_t *h_capacity, int64_t footprint)
{
    if (n < 1 || !h_load || !h_capacity || footprint < 0) return IBIP_ERR_ARG;
    int best = -1;
    for (int i = 0; i < n; i++) {
        if (h_capacity[i] < footprint) continue;
        if (best < 0 || h_load[i] < h_load[best]) best = i;
    }
    return best < 0 ? IBIP_ERR_OOM : best;
}

int ibip_router_create(ibip_router **out, int n, const int *h_devices, size_t mem_budget, int max_slots)
{
    if (!out) return IBIP_ERR_ARG;
    *out = nullptr;
    if (n < 1 || n > 64 || !h_devices) return IBIP_ERR_ARG;
    ibip_router *R = new (std::nothrow) ibip_router;
    if (!R) return IBIP_ERR_OOM;
    R->reps.resize(n);
    int st = IBIP_OK;
    for (int i = 0; i < n && st == IBIP_OK; i++) {
        Replica &P = R->reps[i];
        P.device = h_devices[i];
        st = ibip_create(&P.ctx, P.device, nullptr);
        if (st) break;
        st = ibip_server_create(&P.srv, P.ctx, mem_budget, max_slots);
        if (st == IBIP_OK) {
            int64_t s[6];
            ibip_server_stats(P.srv, s, 6);
            P.capacity = s[5];
        }
    }
    if (st) {
        ibip_router_destroy(R);
        return st;
    }
    *out = R;
    return IBIP_OK;
}

int ibip_router_destroy(ibip_router *R)
{
    if (!R) return IBIP_ERR_ARG;
    for (Replica &P : R->reps) {
        if (P.srv) ibip_server_destroy(P.srv);
        if (P.ctx) ibip_destroy(P.ctx);
    }
    delete R;
    return IBIP_OK;
}

int ibip_router_route(ibip_router *R, ibip_dims dims, int with_dt2, int *h_replica, int *h_device)
{
    if (!R || !h_replica || dims.nx < 1 || dims.ny < 1 || dims.nz < 1) return IBIP_ERR_ARG;
    const int64_t need = ibip_job_footprint(dims, with_dt2);
    std::lock_guard<std::mutex> lk(R->mu);
    const int n = (int)R->reps.size();
    std::vector<int64_t> load(n), cap(n);
    for (int i = 0; i < n; i++) {
        refresh(R->reps[i]);
        load[i] = R->reps[i].load;
        cap[i] = R->reps[i].capacity;
    }
    const int r = ibip_route_pick(n, load.data(), cap.data(), need);
    if (r < 0) return r;
    *h_replica = r;
    if (h_device) *h_device = R->reps[r].device;
    return IBIP_OK;
}

int ibip_router_submit(ibip_router *R, int replica, const ibip_job *job, uint64_t *h_ticket)
{
    if (!R || !job || !h_ticket || replica < 0 || replica >= (int)R->reps.size()) return IBIP_ERR_ARG;
    Replica &P = R->reps[replica];
    uint64_t t = 0;
    const int st = ibip_server_submit(P.srv, job, &t);
    if (st) return st;
    std::lock_guard<std::mutex> lk(R->mu);
    const int64_t vox = (int64_t)job->dims.nx * job->dims.ny * job->dims.nz;
    P.pending[t] = vox;
    P.load += vox;
    P.routed++;
    const uint64_t rt = R->next_ticket++;
    R->tickets[rt] = {replica, t};
    *h_ticket = rt;
    return IBIP_OK;
}

int ibip_router_wait(ibip_router *R, uint64_t ticket, int64_t timeout_us, int *h_done, ibip_result *h_result,
                     int *h_replica)
{
    if (!R || !h_done) return IBIP_ERR_ARG;
    std::pair<int, uint64_t> rt;
    {
        std::lock_guard<std::mutex> lk(R->mu);
        auto it = R->tickets.find(ticket);
        if (it == R->tickets.end()) return IBIP_ERR_ARG;
        rt = it->second;
    }
    Replica &P = R->reps[rt.first];
    const int st = ibip_server_wait(P.srv, rt.second, timeout_us, h_done, h_result);
    if (st) return st;
    if (h_replica) *h_replica = rt.first;
    if (*h_done) {
        std::lock_guard<std::mutex> lk(R->mu);
        auto it = P.pending.find(rt.second);
        if (it != P.pending.end()) {
            P.load -= it->second;
            P.pending.erase(it);
        }
    }
    return IBIP_OK;
}

int ibip_router_stats(ibip_router *R, int replica, int64_t *h_stats, int n)
{
    if (!R || !h_stats || n < 0 || replica < 0 || replica >= (int)R->reps.size()) return IBIP_ERR_ARG;
    std::lock_guard<std::mutex> lk(R->mu);
    Replica &P = R->reps[replica];
    refresh(P);
    int64_t v[12] = {P.device, P.routed, P.load};
    const int st = ibip_server_stats(P.srv, v + 3, 9);
    if (st) return st;
    for (int i = 0; i < n && i < 12; i++) h_stats[i] = v[i];
    return IBIP_OK;
}

}  // extern "C"
