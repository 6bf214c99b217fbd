// api.cu -- the C ABI declared in include/ibip.h: argument checks, context
// and scratch management, and the order of kernel launches for each call.
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "common.cuh"
#include <nvtx3/nvToolsExt.h>

namespace {
// An NVTX range around each compute call of the ABI (visible to nsys and to
// ncu --nvtx; the calls cost nothing when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace

int ibip_invade_run(ibip_ctx *ctx, const int32_t *dt2, ibip_dims d, int inlet, int64_t max_steps,
                    int32_t *seq, int32_t *step_r2, int32_t *step_centre, int64_t cap, int64_t *h_out,
                    const uint8_t *mask = nullptr, int resume = 0);
int ibip_pc_launch(ibip_ctx *ctx, const int32_t *seq, ibip_dims d, const int32_t *r2, int64_t K, double voxel,
                   double sigma, double cos_theta, float *S, float *Pc, float *sat);
int ibip_trap_finish(ibip_ctx *ctx, const int32_t *seq, const int32_t *M, ibip_dims d, int rerank, uint8_t *trapped,
                     int32_t *seq_out, const int32_t *r2_in = nullptr, int64_t k_in = 0, int32_t *r2_out = nullptr,
                     int64_t *h_nout = nullptr);
int ibip_size_launch(ibip_ctx *ctx, const int32_t *seq, ibip_dims d, const int32_t *r2, int64_t K, int32_t *out);
int ibip_level_init(ibip_ctx *ctx, const uint8_t *img, ibip_dims d, int32_t *level);
int ibip_level_counts(ibip_ctx *ctx, const int32_t *level, ibip_dims d, int L, int64_t *h_counts);

namespace {

constexpr int kMaxDim = 16384;
constexpr int kMaxRounds = 1 << 20;

bool dims_ok(ibip_dims d)
{
    if (d.nx < 1 || d.ny < 1 || d.nz < 1) return false;
    if (d.nx > kMaxDim || d.ny > kMaxDim || d.nz > kMaxDim) return false;
    return nvox(d) < (1ll << 31);
}

bool face_ok(int f) { return f >= 0 && f <= 5; }

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

struct ProfLog {
    struct Rec { int cls; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t open[IBIP_K_NCLASSES] = {};
    cudaEvent_t get()
    {
        cudaEvent_t e = nullptr;
        if (!pool.empty()) { e = pool.back(); pool.pop_back(); return e; }
        if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
        return e;
    }
    void clear()
    {
        for (auto &r : recs) { pool.push_back(r.a); pool.push_back(r.b); }
        recs.clear();
        for (auto &e : open) if (e) { pool.push_back(e); e = nullptr; }
    }
    ~ProfLog()
    {
        clear();
        for (auto e : pool) cudaEventDestroy(e);
    }
};

}  // namespace

void ibip_prof_begin(ibip_ctx *ctx, int cls)
{
    ProfLog *p = (ProfLog *)ctx->prof;
    if (!p || cls < 0 || cls >= IBIP_K_NCLASSES || p->open[cls] || p->recs.size() >= 65536) return;
    cudaEvent_t e = p->get();
    if (!e) return;
    cudaEventRecord(e, ctx->stream);
    p->open[cls] = e;
}

void ibip_prof_end(ibip_ctx *ctx, int cls)
{
    ProfLog *p = (ProfLog *)ctx->prof;
    if (!p || cls < 0 || cls >= IBIP_K_NCLASSES || !p->open[cls]) return;
    cudaEvent_t e = p->get();
    if (!e) return;
    cudaEventRecord(e, ctx->stream);
    p->recs.push_back({cls, p->open[cls], e});
    p->open[cls] = nullptr;
}

int ibip_cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return IBIP_OK;
    if (e == cudaErrorMemoryAllocation) return IBIP_ERR_OOM;
    return IBIP_ERR_CUDA;
}

void *ibip_scratch(ibip_ctx *ctx, int slot, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (ctx->slot_bytes[slot] >= bytes) return ctx->slot[slot];
    if (ctx->fail_alloc > 0 && --ctx->fail_alloc == 0) return nullptr;   // injected failure
    if (ctx->arena) {
        const size_t b = (bytes + 255) & ~(size_t)255;
        if (ctx->arena_used + b > ctx->arena_size) return nullptr;
        ctx->slot[slot] = ctx->arena + ctx->arena_used;
        ctx->slot_bytes[slot] = b;
        ctx->arena_used += b;
        return ctx->slot[slot];
    }
    if (ctx->slot[slot]) {
        ibip_sync(ctx, ctx->stream);
        cudaFree(ctx->slot[slot]);
        ctx->slot[slot] = nullptr;
        ctx->slot_bytes[slot] = 0;
    }
    size_t want = bytes + bytes / 8;   // headroom so small growth does not reallocate
    void *p = nullptr;
    if (cudaMalloc(&p, want) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    ctx->slot[slot] = p;
    ctx->slot_bytes[slot] = want;
    return p;
}

bool ibip_job_valid(const ibip_job &J)
{
    return J.image && J.seq && dims_ok(J.dims) && face_ok(J.inlet) && J.capacity_steps >= 0 &&
           (J.capacity_steps == 0 || J.step_r2) && (!J.trapped || face_ok(J.outlet)) &&
           ((J.sat_per_step != nullptr) == (J.pc_per_step != nullptr)) && (!J.sat_per_step || J.voxel_m > 0.0);
}

// The invasion's counters become the context's, except entries 30-32,
// which belong to the last widest-path propagation.
void keep_invade_stats(ibip_ctx *ctx, const int64_t *out)
{
    int64_t mm[3];
    memcpy(mm, ctx->inv_stats + 30, sizeof(mm));
    memcpy(ctx->inv_stats, out, kInvStats * sizeof(int64_t));
    memcpy(ctx->inv_stats + 30, mm, sizeof(mm));
}

int ibip_run_job(ibip_ctx *ctx, ibip_job &J)
{
    J.n_steps = 0;
    int32_t *d = J.dt2;
    if (!d) d = (int32_t *)ibip_scratch(ctx, SC_DT2, (size_t)nvox(J.dims) * sizeof(int32_t));
    if (!d) return IBIP_ERR_OOM;
    int st = ibip_edt_launch(ctx, J.image, J.dims, d);
    if (st) return st;
    int64_t out[kInvStats] = {0};
    st = ibip_invade_run(ctx, d, J.dims, J.inlet, nvox(J.dims), J.seq, J.step_r2, J.step_centre, J.capacity_steps,
                         out);
    if (st) return st;
    J.n_steps = out[0];
    if (out[1] != IBIP_OK) return (int)out[1];
    if (out[0] > J.capacity_steps) return IBIP_ERR_ARG;
    const int32_t *curve_seq = J.seq;
    if (J.trapped) {
        int32_t *M = (int32_t *)ibip_scratch(ctx, SC_MM, (size_t)nvox(J.dims) * sizeof(int32_t));
        if (!M) return IBIP_ERR_OOM;
        st = ibip_maximin_launch(ctx, J.seq, J.dims, J.outlet, M, kMaxRounds);
        if (!st) st = ibip_trap_finish(ctx, J.seq, M, J.dims, 0, J.trapped, J.seq_out);
        if (st) return st;
        if (J.seq_out) curve_seq = J.seq_out;
    }
    if (J.sat_per_step) {
        const double pi = 3.14159265358979323846;
        st = ibip_pc_launch(ctx, curve_seq, J.dims, J.step_r2, J.n_steps, J.voxel_m, J.sigma,
                            cos(J.theta_deg * pi / 180.0), J.sat_per_step, J.pc_per_step, nullptr);
        if (st) return st;
    }
    return ibip_cuda_status(ibip_sync(ctx, ctx->stream));
}

// Post-processing of a batched call (trapping, curves) for a group of its
// images, after their invasions are done.
struct BatchPost {
    ibip_ctx *ctx;
    ibip_job *jobs;
    IbipBatchItem *it;
    int32_t *M;
    std::vector<int64_t> M_off;
    std::vector<char> early;
    int early_err = IBIP_OK;
};

int batch_post_group(BatchPost &P, const std::vector<int> &group, bool shared_device)
{
    ibip_ctx *ctx = P.ctx;
    std::vector<IbipMaximinJob> mj;
    std::vector<int> mj_of;
    for (int j : group) {
        ibip_job &J = P.jobs[j];
        J.n_steps = P.it[j].n_steps;
        J.status = P.it[j].status;
        if (J.status == IBIP_OK && J.n_steps > J.capacity_steps) J.status = IBIP_ERR_ARG;
        if (J.status != IBIP_OK || !J.trapped) continue;
        mj.push_back(IbipMaximinJob{J.seq, J.dims, J.outlet, P.M + P.M_off[j]});
        mj_of.push_back(j);
    }
    // Beside the batch's last running invasion CTAs no cooperative grid may
    // start.  Several images run on the widest path's work queue, whose
    // blocks take the free SMs without needing all to be resident (the
    // remaining invasion CTAs are resident already, so nothing waits for
    // those SMs); a single image, which could get the cooperative rounds,
    // runs one launch per round instead.
    const int keep_nc = ctx->no_coop;
    ctx->no_coop = shared_device && mj.size() == 1 ? 1 : keep_nc;
    int st = mj.empty() ? IBIP_OK : ibip_maximin_multi(ctx, (int)mj.size(), mj.data(), kMaxRounds);
    ctx->no_coop = keep_nc;
    if (st) {
        if (st != IBIP_ERR_NOT_CONVERGED) return st;
        for (int j : mj_of) P.jobs[j].status = st;
    }
    std::vector<IbipCurveItem> ci;
    const double pi = 3.14159265358979323846;
    std::vector<const int32_t *> Mof(P.M_off.size(), nullptr);
    for (size_t q = 0; q < mj.size(); q++) Mof[mj_of[q]] = mj[q].M;
    for (int j : group) {
        ibip_job &J = P.jobs[j];
        if (J.status != IBIP_OK) continue;
        const int32_t *M = J.trapped ? Mof[j] : nullptr;
        if (!M && !J.sat_per_step) continue;
        ci.push_back(IbipCurveItem{J.seq, M, J.trapped, J.seq_out, J.step_r2, J.sat_per_step, J.pc_per_step, J.dims,
                                   J.n_steps, J.voxel_m, J.sigma, cos(J.theta_deg * pi / 180.0)});
    }
    return ibip_curve_batch_launch(ctx, (int)ci.size(), ci.data());
}

// the images done while the largest invasions still run: on the second stream
int batch_early(void *user, int n_done, const int *done)
{
    BatchPost &P = *(BatchPost *)user;
    ibip_ctx *ctx = P.ctx;
    std::vector<int> group(done, done + n_done);
    for (int j : group) P.early[j] = 1;
    cudaStream_t keep = ctx->stream;
    ctx->stream = ctx->stream2;
    const int st = batch_post_group(P, group, true);
    ctx->stream = keep;
    P.early_err = st;
    return st;
}

cudaError_t ibip_sync(ibip_ctx *ctx, cudaStream_t s)
{
    if (!ctx->ev_block) return cudaStreamSynchronize(s);
    const cudaError_t e = cudaEventRecord(ctx->ev_block, s);
    if (e != cudaSuccess) return e;
    return cudaEventSynchronize(ctx->ev_block);
}

extern "C" {

int ibip_create(ibip_ctx **out, int device, void *cuda_stream)
{
    if (!out) return IBIP_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return device < 0 || (n > 0 && device >= n) ? IBIP_ERR_ARG : IBIP_ERR_CUDA;
    }
    DeviceGuard g(device);
    ibip_ctx *c = new (std::nothrow) ibip_ctx;
    if (!c) return IBIP_ERR_OOM;
    memset(c, 0, sizeof(*c));
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    if (!cuda_stream) {
        // no stream given: the context's own, which does not serialise
        // against unrelated work on the legacy default stream
        if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return IBIP_ERR_CUDA;
        }
        c->stream = c->own_stream;
    }
    if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMallocHost(&c->h_pinned, 65536) != cudaSuccess) {
        cudaGetLastError();
        if (c->own_stream) cudaStreamDestroy(c->own_stream);
        delete c;
        return IBIP_ERR_CUDA;
    }
    void *hc = nullptr, *dc = nullptr;
    if (cudaHostAlloc(&c->h_done, (size_t)kMaxBatch * sizeof(IbipBatchDone), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(&c->d_done, c->h_done, 0) != cudaSuccess ||
        cudaHostAlloc(&hc, 64, cudaHostAllocMapped) != cudaSuccess || cudaHostGetDevicePointer(&dc, hc, 0) != cudaSuccess) {
        cudaGetLastError();
        if (hc) cudaFreeHost(hc);
        if (c->h_done) cudaFreeHost(c->h_done);
        cudaFreeHost(c->h_pinned);
        if (c->own_stream) cudaStreamDestroy(c->own_stream);
        delete c;
        return IBIP_ERR_CUDA;
    }
    c->h_cancel = (volatile int *)hc;
    c->d_cancel = (int *)dc;
    *c->h_cancel = 0;
    *out = c;
    return IBIP_OK;
}

int ibip_destroy(ibip_ctx *ctx)
{
    if (!ctx) return IBIP_ERR_ARG;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    delete (ProfLog *)ctx->prof;
    for (int i = 0; i < SC_NSLOTS; i++)
        if (ctx->slot[i] && !ctx->arena) cudaFree(ctx->slot[i]);
    if (ctx->stream2) {
        cudaStreamSynchronize(ctx->stream2);
        cudaStreamDestroy(ctx->stream2);
    }
    if (ctx->own_stream) {
        cudaStreamSynchronize(ctx->own_stream);
        cudaStreamDestroy(ctx->own_stream);
    }
    if (ctx->stream_inv) {
        cudaStreamSynchronize(ctx->stream_inv);
        cudaStreamDestroy(ctx->stream_inv);
    }
    if (ctx->ev_inv) cudaEventDestroy(ctx->ev_inv);
    if (ctx->ev_block) cudaEventDestroy(ctx->ev_block);
    if (ctx->h_done) cudaFreeHost(ctx->h_done);
    if (ctx->h_cancel) cudaFreeHost((void *)ctx->h_cancel);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    delete ctx;
    return IBIP_OK;
}

int ibip_set_stream(ibip_ctx *ctx, void *cuda_stream)
{
    if (!ctx) return IBIP_ERR_ARG;
    if (!cuda_stream && !ctx->own_stream) {
        // back to a stream of the context's own, created on first need
        DeviceGuard g(ctx->device);
        if (cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            ctx->own_stream = nullptr;
            return IBIP_ERR_CUDA;
        }
    }
    ctx->stream = cuda_stream ? (cudaStream_t)cuda_stream : ctx->own_stream;
    return IBIP_OK;
}

int ibip_get_stream(const ibip_ctx *ctx, void **h_stream)
{
    if (!ctx || !h_stream) return IBIP_ERR_ARG;
    *h_stream = (void *)ctx->stream;
    return IBIP_OK;
}

int ibip_synchronize(ibip_ctx *ctx)
{
    if (!ctx) return IBIP_ERR_ARG;
    DeviceGuard g(ctx->device);
    return ibip_cuda_status(ibip_sync(ctx, ctx->stream));
}

int64_t ibip_launch_count(const ibip_ctx *ctx) { return ctx ? ctx->launches : -1; }

int ibip_invade_stats(const ibip_ctx *ctx, int64_t *h_stats, int n)
{
    if (!ctx || !h_stats || n < 0) return IBIP_ERR_ARG;
    for (int i = 0; i < n && i < kInvStats; i++) h_stats[i] = ctx->inv_stats[i];
    return IBIP_OK;
}

int ibip_cancel(ibip_ctx *ctx, int on)
{
    if (!ctx || (on != 0 && on != 1) || !ctx->h_cancel) return IBIP_ERR_ARG;
    *ctx->h_cancel = on;
    return IBIP_OK;
}

int ibip_debug_fail_alloc(ibip_ctx *ctx, int nth)
{
    if (!ctx || nth < 0) return IBIP_ERR_ARG;
    ctx->fail_alloc = nth;
    return IBIP_OK;
}

int ibip_set_autotune(ibip_ctx *ctx, int mode, const char *cache_path)
{
    if (!ctx || (mode != 0 && mode != 1)) return IBIP_ERR_ARG;
    if (cache_path && strlen(cache_path) >= sizeof(ctx->tune_path)) return IBIP_ERR_ARG;
    ctx->autotune = mode;
    ctx->tune_path[0] = 0;
    if (cache_path) {
        strcpy(ctx->tune_path, cache_path);
        ibip_tune_load(cache_path);
    }
    return IBIP_OK;
}

int ibip_set_edt_tiles(ibip_ctx *ctx, int z_warps, int strip_warps)
{
    if (!ctx) return IBIP_ERR_ARG;
    return ibip_edt_tile_set(ctx, z_warps, strip_warps);
}

int ibip_edt_tiles(ibip_ctx *ctx, ibip_dims dims, int *h_z_warps, int *h_strip_warps)
{
    if (!ctx || !h_z_warps || !h_strip_warps || !dims_ok(dims)) return IBIP_ERR_ARG;
    ibip_edt_tile_get(ctx, dims, h_z_warps, h_strip_warps);
    return IBIP_OK;
}

int ibip_invade_trace(ibip_ctx *ctx, int32_t *d_trace, int64_t capacity_records)
{
    if (!ctx || (d_trace && (capacity_records < 0 || ((uintptr_t)d_trace & 15)))) return IBIP_ERR_ARG;
    ctx->trace = d_trace;
    ctx->trace_cap = d_trace ? capacity_records : 0;
    return IBIP_OK;
}

int ibip_profile_enable(ibip_ctx *ctx, int on)
{
    if (!ctx) return IBIP_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (on) {
        if (!ctx->prof) ctx->prof = new (std::nothrow) ProfLog;
        if (!ctx->prof) return IBIP_ERR_OOM;
        ibip_sync(ctx, ctx->stream);
        ((ProfLog *)ctx->prof)->clear();
    } else if (ctx->prof) {
        ibip_sync(ctx, ctx->stream);
        delete (ProfLog *)ctx->prof;
        ctx->prof = nullptr;
    }
    return IBIP_OK;
}

int ibip_profile_read(ibip_ctx *ctx, int cls, double *h_ms, int64_t *h_spans)
{
    if (!ctx || !h_ms || !h_spans || cls < 0 || cls >= IBIP_K_NCLASSES) return IBIP_ERR_ARG;
    DeviceGuard g(ctx->device);
    *h_ms = 0.0;
    *h_spans = 0;
    ProfLog *p = (ProfLog *)ctx->prof;
    if (!p) return IBIP_OK;
    cudaError_t e = ibip_sync(ctx, ctx->stream);
    if (e != cudaSuccess) return ibip_cuda_status(e);
    for (auto &r : p->recs) {
        if (r.cls != cls) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) { *h_ms += ms; (*h_spans)++; }
        else cudaGetLastError();
    }
    return IBIP_OK;
}

int ibip_edt(ibip_ctx *ctx, const uint8_t *image, ibip_dims dims, int32_t *dt2)
{
    NvtxRange nvtx_range("ibip_edt");
    if (!ctx || !image || !dt2 || !dims_ok(dims)) return IBIP_ERR_ARG;
    DeviceGuard g(ctx->device);
    return ibip_edt_launch(ctx, image, dims, dt2);
}

int ibip_invade(ibip_ctx *ctx, const uint8_t *image, const int32_t *dt2, ibip_dims dims, int inlet,
                int64_t max_steps, int32_t *seq, int32_t *step_r2, int32_t *step_centre, int64_t capacity_steps,
                int64_t *h_n_steps)
{
    NvtxRange nvtx_range("ibip_invade");
    if (!ctx || !image || !seq || !h_n_steps || !dims_ok(dims) || !face_ok(inlet) || max_steps < 0 ||
        capacity_steps < 0 || (capacity_steps > 0 && !step_r2))
        return IBIP_ERR_ARG;
    DeviceGuard g(ctx->device);
    *h_n_steps = 0;
    const int32_t *d = dt2;
    if (!d) {
        int32_t *t = (int32_t *)ibip_scratch(ctx, SC_DT2, (size_t)nvox(dims) * sizeof(int32_t));
        if (!t) return IBIP_ERR_OOM;
        int st = ibip_edt_launch(ctx, image, dims, t);
        if (st) return st;
        d = t;
    }
    int64_t out[kInvStats] = {0};
    int st = ibip_invade_run(ctx, d, dims, inlet, max_steps, seq, step_r2, step_centre, capacity_steps, out);
    if (st) return st;
    keep_invade_stats(ctx, out);
    *h_n_steps = out[0];
    if (out[1] != IBIP_OK) return (int)out[1];
    if (out[0] > capacity_steps) return IBIP_ERR_ARG;
    return IBIP_OK;
}

int ibip_invade_ex(ibip_ctx *ctx, const uint8_t *image, const int32_t *dt2, ibip_dims dims, int inlet,
                   const uint8_t *inlet_mask, int resume, int64_t max_steps, int32_t *seq, int32_t *step_r2,
                   int32_t *step_centre, int64_t capacity_steps, int64_t *h_n_steps)
{
    NvtxRange nvtx_range("ibip_invade_ex");
    if (!ctx || !image || !seq || !h_n_steps || !dims_ok(dims) || (!inlet_mask && !face_ok(inlet)) ||
        max_steps < 0 || capacity_steps < 0 || (capacity_steps > 0 && !step_r2) || (resume != 0 && resume != 1))
        return IBIP_ERR_ARG;
    DeviceGuard g(ctx->device);
    *h_n_steps = 0;
    const int32_t *d = dt2;
    if (!d) {
        int32_t *t = (int32_t *)ibip_scratch(ctx, SC_DT2, (size_t)nvox(dims) * sizeof(int32_t));
        if (!t) return IBIP_ERR_OOM;
        int st = ibip_edt_launch(ctx, image, dims, t);
        if (st) return st;
        d = t;
    }
    int64_t out[kInvStats] = {0};
    int st = ibip_invade_run(ctx, d, dims, inlet_mask ? 0 : inlet, max_steps, seq, step_r2, step_centre,
                             capacity_steps, out, inlet_mask, resume);
    if (st) return st;
    keep_invade_stats(ctx, out);
    *h_n_steps = out[0];
    if (out[1] != IBIP_OK) return (int)out[1];
    if (out[0] > capacity_steps) return IBIP_ERR_ARG;
    return IBIP_OK;
}

int ibip_invade_literal(ibip_ctx *ctx, const uint8_t *image, const int32_t *dt2, ibip_dims dims, int inlet,
                        int64_t max_steps, int32_t *seq, int32_t *cstep, int32_t *step_r2, int32_t *step_count,
                        int64_t capacity_steps, int64_t *h_n_steps)
{
    NvtxRange nvtx_range("ibip_invade_literal");
    if (!ctx || !image || !seq || !cstep || !h_n_steps || !dims_ok(dims) || !face_ok(inlet) || max_steps < 0 ||
        capacity_steps < 0 || (capacity_steps > 0 && (!step_r2 || !step_count)))
        return IBIP_ERR_ARG;
    DeviceGuard g(ctx->device);
    *h_n_steps = 0;
    const int32_t *d = dt2;
    if (!d) {
        int32_t *t = (int32_t *)ibip_scratch(ctx, SC_DT2, (size_t)nvox(dims) * sizeof(int32_t));
        if (!t) return IBIP_ERR_OOM;
        int st = ibip_edt_launch(ctx, image, dims, t);
        if (st) return st;
        d = t;
    }
    int64_t out[2] = {0, 0};
    int st = ibip_literal_run(ctx, d, dims, inlet, max_steps, seq, cstep, step_r2, step_count, capacity_steps, out);
    if (st) return st;
    *h_n_steps = out[0];
    if (out[1] != IBIP_OK) return (int)out[1];
    if (out[0] > capacity_steps) return IBIP_ERR_ARG;
    return IBIP_OK;
}

int ibip_invade_literal_batched(ibip_ctx *ctx, int32_t n, ibip_literal_job *jobs, int *h_cluster)
{
    NvtxRange nvtx_range("ibip_invade_literal_batched");
    if (!ctx || !jobs || n < 1 || n > kMaxBatch) return IBIP_ERR_ARG;
    int64_t need_dt2 = 0;
    for (int j = 0; j < n; j++) {
        const ibip_literal_job &J = jobs[j];
        if (!J.image || !J.seq || !J.cstep || !dims_ok(J.dims) || !face_ok(J.inlet) || J.capacity_steps < 0 ||
            (J.capacity_steps > 0 && (!J.step_r2 || !J.step_count)))
            return IBIP_ERR_ARG;
        if (!J.dt2) need_dt2 += (nvox(J.dims) + 63) & ~(int64_t)63;
    }
    DeviceGuard g(ctx->device);
    int32_t *pool = need_dt2 ? (int32_t *)ibip_scratch(ctx, SC_BDT2, (size_t)need_dt2 * sizeof(int32_t)) : nullptr;
    if (need_dt2 && !pool) return IBIP_ERR_OOM;
    std::vector<IbipLitItem> it(n);
    std::vector<const uint8_t *> ims;
    std::vector<ibip_dims> dms;
    std::vector<int32_t *> dts;
    int64_t off = 0;
    for (int j = 0; j < n; j++) {
        ibip_literal_job &J = jobs[j];
        const int32_t *d = J.dt2;
        if (!d) {
            int32_t *t = pool + off;
            off += (nvox(J.dims) + 63) & ~(int64_t)63;
            ims.push_back(J.image); dms.push_back(J.dims); dts.push_back(t);
            d = t;
        }
        it[j] = IbipLitItem{d, J.dims, J.inlet, J.max_steps < 0 ? INT64_MAX : J.max_steps, J.seq, J.cstep,
                            J.step_r2, J.step_count, J.capacity_steps, 0, 0};
    }
    if (!ims.empty()) {
        const int st = ibip_edt_batch_launch(ctx, (int)ims.size(), ims.data(), dms.data(), dts.data());
        if (st) return st;
    }
    const int st = ibip_literal_batch_run(ctx, n, it.data(), ctx->lit_cluster, h_cluster);
    if (st) return st;
    int first = IBIP_OK;
    for (int j = 0; j < n; j++) {
        jobs[j].n_steps = it[j].n_steps;
        jobs[j].status = it[j].status;
        if (jobs[j].status == IBIP_OK && jobs[j].n_steps > jobs[j].capacity_steps) jobs[j].status = IBIP_ERR_ARG;
        if (first == IBIP_OK && jobs[j].status != IBIP_OK) first = jobs[j].status;
    }
    return first;
}

int ibip_set_shared_device(ibip_ctx *ctx, int on)
{
    if (!ctx) return IBIP_ERR_ARG;
    ctx->no_coop = on ? 1 : 0;
    return IBIP_OK;
}

int ibip_set_literal_cluster(ibip_ctx *ctx, int cluster)
{
    if (!ctx || !(cluster == 0 || cluster == 1 || cluster == 2 || cluster == 4 || cluster == 8 || cluster == 16))
        return IBIP_ERR_ARG;
    ctx->lit_cluster = cluster;
    return IBIP_OK;
}

int ibip_trapping(ibip_ctx *ctx, const int32_t *seq, ibip_dims dims, int outlet, int rerank, uint8_t *trapped,
                  int32_t *seq_out)
{
    NvtxRange nvtx_range("ibip_trapping");
    if (!ctx || !seq || !trapped || !dims_ok(dims) || !face_ok(outlet)) return IBIP_ERR_ARG;
    DeviceGuard g(ctx->device);
    int32_t *M = (int32_t *)ibip_scratch(ctx, SC_MM, (size_t)nvox(dims) * sizeof(int32_t));
    if (!M) return IBIP_ERR_OOM;
    int st = ibip_maximin_launch(ctx, seq, dims, outlet, M, kMaxRounds);
    if (st) return st;
    st = ibip_trap_finish(ctx, seq, M, dims, rerank, trapped, seq_out);
    if (st) return st;
    return ibip_cuda_status(ibip_sync(ctx, ctx->stream));
}

int ibip_trapping_ex(ibip_ctx *ctx, const int32_t *seq, ibip_dims dims, int outlet, uint8_t *trapped,
                     int32_t *seq_out, const int32_t *step_r2, int64_t n_steps, int32_t *step_r2_out,
                     int64_t *h_n_steps_out)
{
    NvtxRange nvtx_range("ibip_trapping_ex");
    if (!ctx || !seq || !trapped || !seq_out || !h_n_steps_out || !dims_ok(dims) || !face_ok(outlet) ||
        n_steps < 0 || (n_steps > 0 && (!step_r2 || !step_r2_out)))
        return IBIP_ERR_ARG;
    DeviceGuard g(ctx->device);
    int32_t *M = (int32_t *)ibip_scratch(ctx, SC_MM, (size_t)nvox(dims) * sizeof(int32_t));
    if (!M) return IBIP_ERR_OOM;
    int st = ibip_maximin_launch(ctx, seq, dims, outlet, M, kMaxRounds);
    if (st) return st;
    st = ibip_trap_finish(ctx, seq, M, dims, 1, trapped, seq_out, step_r2, n_steps, step_r2_out, h_n_steps_out);
    if (st) return st;
    return ibip_cuda_status(ibip_sync(ctx, ctx->stream));
}

int ibip_size_image(ibip_ctx *ctx, const int32_t *seq, ibip_dims dims, const int32_t *step_r2, int64_t n_steps,
                    int32_t *r2_image)
{
    NvtxRange nvtx_range("ibip_size_image");
    if (!ctx || !seq || !r2_image || !dims_ok(dims) || n_steps < 0 || (n_steps > 0 && !step_r2))
        return IBIP_ERR_ARG;
    DeviceGuard g(ctx->device);
    return ibip_size_launch(ctx, seq, dims, step_r2, n_steps, r2_image);
}

int ibip_morph_drainage_ex(ibip_ctx *ctx, const uint8_t *image, const int32_t *dt2, ibip_dims dims, int inlet,
                           const int32_t *h_r2_levels, const int32_t *h_dilate_r2, int32_t n_levels, int32_t *level,
                           int64_t *h_counts)
{
    NvtxRange nvtx_range("ibip_morph_drainage");
    if (!ctx || !image || !dt2 || !level || !h_counts || !dims_ok(dims) || !face_ok(inlet) || n_levels < 0 ||
        n_levels > 8192 ||
        (n_levels > 0 && !h_r2_levels))
        return IBIP_ERR_ARG;
    const int32_t *Td = h_dilate_r2 ? h_dilate_r2 : h_r2_levels;
    for (int i = 0; i < n_levels; i++) {
        if (h_r2_levels[i] < 1 || Td[i] < 1) return IBIP_ERR_ARG;
        if (i > 0 && h_r2_levels[i] >= h_r2_levels[i - 1]) return IBIP_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    int32_t *W = (int32_t *)ibip_scratch(ctx, SC_MM, (size_t)nvox(dims) * sizeof(int32_t));
    if (!W) return IBIP_ERR_OOM;
    int st = ibip_level_init(ctx, image, dims, level);
    if (st) return st;
    if (n_levels == 0) return ibip_cuda_status(ibip_sync(ctx, ctx->stream));
    st = ibip_maximin_launch(ctx, dt2, dims, inlet, W, kMaxRounds);
    if (st) return st;
    // radii above the largest widest-path value trim to the empty set: skip
    int wmax = 0;
    st = ibip_max_launch(ctx, W, nvox(dims), &wmax);
    if (st) return st;
    int first = 0;
    while (first < n_levels && h_r2_levels[first] > wmax) first++;
    if (n_levels <= 254) {
        uint8_t *fl = (uint8_t *)ibip_scratch(ctx, SC_FL, (size_t)nvox(dims) + 256 * sizeof(int32_t) + 256);
        if (!fl) return IBIP_ERR_OOM;
        int32_t *T_dev = (int32_t *)(fl + (((size_t)nvox(dims) + 255) & ~(size_t)255));
        cudaMemcpyAsync(T_dev, h_r2_levels, (size_t)n_levels * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream);
        st = ibip_first_level_launch(ctx, W, dims, T_dev, n_levels, fl);
        if (st) return st;
        for (int i = first; i < n_levels; i++) {
            st = ibip_dilate_first_level_launch(ctx, fl, Td[i], i, dims, level);
            if (st) return st;
        }
    } else {
        for (int i = first; i < n_levels; i++) {
            st = ibip_dilate_level_launch(ctx, W, h_r2_levels[i], Td[i], i + 1, dims, level);
            if (st) return st;
        }
    }
    return ibip_level_counts(ctx, level, dims, n_levels, h_counts);
}

int ibip_morph_drainage(ibip_ctx *ctx, const uint8_t *image, const int32_t *dt2, ibip_dims dims, int inlet,
                        const int32_t *h_r2_levels, int32_t n_levels, int32_t *level, int64_t *h_counts)
{
    return ibip_morph_drainage_ex(ctx, image, dt2, dims, inlet, h_r2_levels, nullptr, n_levels, level, h_counts);
}

int ibip_invade_batched(ibip_ctx *ctx, int32_t n, ibip_job *jobs)
{
    NvtxRange nvtx_range("ibip_invade_batched");
    if (!ctx || !jobs || n < 1 || n > kMaxBatch) return IBIP_ERR_ARG;
    int64_t need_dt2 = 0;
    for (int j = 0; j < n; j++) {
        const ibip_job &J = jobs[j];
        if (!ibip_job_valid(J)) return IBIP_ERR_ARG;
        if (!J.dt2) need_dt2 += (nvox(J.dims) + 63) & ~(int64_t)63;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t s = ctx->stream;
    int32_t *pool = need_dt2 ? (int32_t *)ibip_scratch(ctx, SC_BDT2, (size_t)need_dt2 * sizeof(int32_t)) : nullptr;
    if (need_dt2 && !pool) return IBIP_ERR_OOM;
    std::vector<IbipBatchItem> it(n);
    std::vector<const uint8_t *> ims(n);
    std::vector<ibip_dims> dms(n);
    std::vector<int32_t *> dts(n);
    int64_t off = 0;
    for (int j = 0; j < n; j++) {
        ibip_job &J = jobs[j];
        int32_t *d = J.dt2;
        if (!d) { d = pool + off; off += (nvox(J.dims) + 63) & ~(int64_t)63; }
        ims[j] = J.image; dms[j] = J.dims; dts[j] = d;
        it[j] = IbipBatchItem{d, J.dims, J.inlet, nvox(J.dims), J.seq, J.step_r2, J.step_centre,
                              J.capacity_steps, 0, 0};
    }
    int st = ibip_edt_batch_launch(ctx, n, ims.data(), dms.data(), dts.data());
    if (st) return st;
    // Trapping and curves run in two groups: the images whose invasion is
    // done while the last few still run (on a second stream, overlapping
    // them), then the rest.  All scratch they use is sized first, so nothing
    // is reallocated while kernels run.
    if (!ctx->stream2 && cudaStreamCreateWithFlags(&ctx->stream2, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        ctx->stream2 = nullptr;
        return IBIP_ERR_CUDA;
    }
    BatchPost P;
    P.ctx = ctx;
    P.jobs = jobs;
    P.it = it.data();
    P.M_off.assign(n, -1);
    P.early.assign(n, 0);
    int64_t mm_total = 0, nt_total = 0, cnt_total = 0;
    for (int j = 0; j < n; j++) {
        const ibip_job &J = jobs[j];
        if (J.trapped) {
            P.M_off[j] = mm_total;
            mm_total += (nvox(J.dims) + 63) & ~(int64_t)63;
            nt_total += (int64_t)((J.dims.nx + 3) / 4) * ((J.dims.ny + 7) / 8) * ((J.dims.nz + 31) / 32);
        }
        if (J.sat_per_step) cnt_total += nvox(J.dims) + 2;
    }
    P.M = mm_total ? (int32_t *)ibip_scratch(ctx, SC_MM, (size_t)mm_total * sizeof(int32_t)) : nullptr;
    const size_t tile_bytes = ((size_t)n * 64 + 255) / 256 * 256 + ((size_t)3 * nt_total + 2 * ((1 << 16) + 2) + 4) * 4;
    if ((mm_total && !P.M) || (nt_total && !ibip_scratch(ctx, SC_TILE, tile_bytes)) ||
        !ibip_scratch(ctx, SC_HIST, ibip_curve_batch_bytes(n, cnt_total)) ||
        !ibip_scratch(ctx, SC_SCAN, ibip_scan_scratch_bytes(cnt_total + 1)) || !ibip_scratch(ctx, SC_SMALL, kSmallBytes))
        return IBIP_ERR_OOM;
    st = ibip_invade_batch_run(ctx, n, it.data(), batch_early, &P);
    cudaError_t e2 = ibip_sync(ctx, ctx->stream2);
    if (st && st != P.early_err) return st;
    if (e2 != cudaSuccess) return ibip_cuda_status(e2);
    std::vector<int> rest;
    for (int j = 0; j < n; j++)
        if (!P.early[j]) rest.push_back(j);
    st = batch_post_group(P, rest, false);
    if (st) return st;
    cudaError_t e = ibip_sync(ctx, s);
    if (e != cudaSuccess) return ibip_cuda_status(e);
    for (int j = 0; j < n; j++)
        if (jobs[j].status == IBIP_ERR_CANCELLED && ctx->h_cancel) *ctx->h_cancel = 0;   // the request is served
    if (P.early_err) return P.early_err;
    for (int j = 0; j < n; j++)
        if (jobs[j].status != IBIP_OK) return jobs[j].status;
    return IBIP_OK;
}

int ibip_equal_saturation(ibip_ctx *ctx, const int32_t *seq, const int32_t *level, ibip_dims dims,
                          int64_t n_steps, int32_t n_levels, int64_t *h_steps, int64_t *h_diff, int64_t *h_count)
{
    NvtxRange nvtx_range("ibip_equal_saturation");
    if (!ctx || !seq || !level || !h_diff || !dims_ok(dims) || n_steps < 0 || n_steps >= (1ll << 31) ||
        n_levels < 1 || n_levels > 254)
        return IBIP_ERR_ARG;
    DeviceGuard g(ctx->device);
    return ibip_eqsat_launch(ctx, seq, level, dims, n_steps, n_levels, h_steps, h_diff, h_count);
}

int ibip_pc_envelope(ibip_ctx *ctx, const int32_t *seq, ibip_dims dims, const int32_t *step_r2, int64_t n_steps,
                     const int32_t *h_r2_levels, int32_t n_levels, int64_t *h_steps, int64_t *h_count)
{
    NvtxRange nvtx_range("ibip_pc_envelope");
    if (!ctx || !seq || !dims_ok(dims) || n_steps < 0 || n_steps >= (1ll << 31) || (n_steps > 0 && !step_r2) ||
        n_levels < 1 || n_levels > 254 || !h_r2_levels || !h_steps || !h_count)
        return IBIP_ERR_ARG;
    for (int i = 0; i < n_levels; i++) {
        if (h_r2_levels[i] < 1) return IBIP_ERR_ARG;
        if (i > 0 && h_r2_levels[i] >= h_r2_levels[i - 1]) return IBIP_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    return ibip_envelope_launch(ctx, seq, dims, step_r2, n_steps, h_r2_levels, n_levels, h_steps, h_count);
}

int ibip_pc_curve(ibip_ctx *ctx, const int32_t *seq, ibip_dims dims, const int32_t *step_r2, int64_t n_steps,
                  double voxel_m, double sigma, double theta_deg, float *sat_per_step, float *pc_per_step,
                  float *sat_image)
{
    NvtxRange nvtx_range("ibip_pc_curve");
    if (!ctx || !seq || !dims_ok(dims) || n_steps < 0 || n_steps >= (1ll << 31) ||
        (n_steps > 0 && (!step_r2 || !sat_per_step || !pc_per_step)) || (sat_image && !sat_per_step) ||
        !(voxel_m > 0.0))
        return IBIP_ERR_ARG;
    DeviceGuard g(ctx->device);
    const double pi = 3.14159265358979323846;
    const double ct = cos(theta_deg * pi / 180.0);
    return ibip_pc_launch(ctx, seq, dims, step_r2, n_steps, voxel_m, sigma, ct, sat_per_step, pc_per_step,
                          sat_image);
}

const char *ibip_status_string(int s)
{
    switch (s) {
    case IBIP_OK: return "ok";
    case IBIP_ERR_ARG: return "invalid argument";
    case IBIP_ERR_CUDA: return "CUDA runtime error";
    case IBIP_ERR_OOM: return "out of device memory";
    case IBIP_ERR_STEP_LIMIT: return "step limit reached with candidates left";
    case IBIP_ERR_NOT_CONVERGED: return "propagation did not converge within its round or activation limit";
    case IBIP_ERR_CANCELLED: return "cancelled";
    case IBIP_ERR_BOUNDS: return "device index check failed";
    case IBIP_ERR_TOO_LARGE: return "image exceeds the fixed scratch of ibip_edt_noalloc (2^21 voxels)";
    default: return "unknown status";
    }
}

}  // extern "C"
