// common.cuh -- internal helpers shared by the libibip CUDA sources.
#pragma once

#include <cuda_runtime.h>
#include <string>
#include <stdint.h>

#include "../../include/ibip.h"

#define IBIP_INF32 0x7fffffff

// Scratch slots owned by a context (grown on demand, reused across calls).
enum ScratchSlot {
    SC_DT2 = 0,   // int32[N]      EDT when the caller passes none
    SC_D1,        // uint16[N]     EDT pass-1 output
    SC_G2,        // int32[N]      EDT pass-2 output
    SC_RANK,      // int32[N]      rank of each pore voxel
    SC_OKEY,      // int2[Npore]   (idx, dt2) by rank
    SC_AVAIL,     // u32 bit-plane (pore and not yet invaded)
    SC_ADDED,     // u32 bit-plane (ever queued as a candidate)
    SC_FB,        // u64 frontier bitmap levels 0..3
    SC_PRES,      // int32 presence / bucket id by dt2 value
    SC_MAT,       // int32 per-(bucket, chunk) counts
    SC_SCAN,      // scan partial sums
    SC_MM,        // int32[N]      maximin field
    SC_TILE,      // u8 tile activity flags
    SC_HIST,      // int32 histogram
    SC_SMALL,     // small device scalars
    SC_LIST,      // int32 overflow work lists of the invasion kernel
    SC_FL,        // uint8 first opening level per voxel, and the level radii
    SC_BSTAT,     // batched invasion: per-image pore statistics
    SC_BARENA,    // batched invasion: per-image ranks, bit-planes, bitmaps
    SC_BJOBS,     // batched invasion: job table
    SC_BDT2,      // batched invasion: EDTs of images given without one
    SC_LIT,       // paper-literal invasion: bucket lists, counters, bit-plane
    SC_LITB,      // batched paper-literal invasion: every image's buckets, lists, bit-planes
    SC_LITJ,      // batched paper-literal invasion: job table, statistics, outputs
    SC_BSORT,     // batched invasion: sort job table, presence pool
    SC_NSLOTS
};

// int64 counters an invasion reports (ibip_invade_stats)
constexpr int kInvStats = 48;

struct ibip_ctx {
    int device;
    cudaStream_t stream;
    // The non-blocking stream the context created for itself (ibip_create
    // with no stream), destroyed with the context; null when none.
    cudaStream_t own_stream;
    int sm_count;
    int64_t launches;
    void *slot[SC_NSLOTS];
    size_t slot_bytes[SC_NSLOTS];
    void *h_pinned;   // small pinned host buffer for scalar readback
    void *prof;       // event log when profiling is on (api.cu), else null
    int64_t inv_stats[kInvStats];   // counters of the last ibip_invade (ibip_invade_stats)
    // Per-batch timing records of later single-image invasions (device
    // array of int4, capacity in records), or null.
    void *trace;
    int64_t trace_cap;
    // Arena mode (server slots): scratch is carved from [arena, arena +
    // arena_size) and never freed; a request that does not fit fails.
    char *arena;
    size_t arena_size, arena_used;
    // Kernels share the device with other streams: no cooperative launches.
    int no_coop;
    // Server slots: the invasion kernel goes to this stream (of the
    // device's highest priority, owned by the context, with an event that
    // orders it after the work queued before it), so that its one CTA is
    // placed ahead of the waiting blocks of other jobs' wide kernels; null
    // elsewhere.
    cudaStream_t stream_inv;
    cudaEvent_t ev_inv;
    // Server slots: an event created with cudaEventBlockingSync; the
    // library's waits record it and sleep on it instead of spinning, so
    // that many slot threads on few host cores do not starve each other's
    // launches.  Null elsewhere (plain stream synchronisation).
    cudaEvent_t ev_block;
    // Batched invasion: a second stream for post-processing images whose
    // invasion is done while others still run, and host-mapped completion
    // records written by the invasion CTAs.
    cudaStream_t stream2;
    void *h_done, *d_done;
    // Tile shapes: autotune (0 off, 1 on), a forced EDT tile (index + 1,
    // 0 = automatic) and the file that keeps tuning results ("" = none).
    int autotune, edt_tile;
    // CTAs per image cluster of the batched paper-literal invasion
    // (0 = automatic).
    int lit_cluster;
    char tune_path[512];
    // Cancellation: a host-mapped flag the invasion kernels poll (host and
    // device addresses), and a test hook that fails the n-th scratch
    // allocation from now (0 = off).
    volatile int *h_cancel;
    int *d_cancel;
    int fail_alloc;
};

// Completion record of one image of a batched invasion (host-mapped).
struct IbipBatchDone {
    int64_t steps;
    int32_t status;
    int32_t done;
};
// Called once, on the host, when all but a few images of a batched invasion
// are done (their n_steps and status are filled in); the others still run.
typedef int (*IbipBatchEarly)(void *user, int n_done, const int *done_items);

// Profiling: CUDA-event pairs around each kernel class, on the context's
// stream, only while ibip_profile_enable(ctx, 1) is in effect.
// Waits for the work queued on stream s (see ibip_ctx::ev_block).
cudaError_t ibip_sync(ibip_ctx *ctx, cudaStream_t s);
void ibip_prof_begin(ibip_ctx *ctx, int cls);
void ibip_prof_end(ibip_ctx *ctx, int cls);

// Bytes of the SC_SMALL slot: int scalars at int offsets 0..15, the
// invasion kernel's int64 outputs from byte 64 (at most 64 values).
constexpr size_t kSmallBytes = 64 + 64 * sizeof(int64_t);

// Grow-only scratch.  Returns nullptr on failure.
void *ibip_scratch(ibip_ctx *ctx, int slot, size_t bytes);

#define IBIP_LAUNCH(ctx) ((ctx)->launches++)

// One image of a batched invasion (internal form of ibip_job).
struct IbipBatchItem {
    const int32_t *dt2;
    ibip_dims d;
    int inlet;
    int64_t max_steps;
    int32_t *seq, *step_r2, *step_centre;
    int64_t cap;
    int64_t n_steps;   // out
    int status;        // out
};
constexpr int kMaxBatch = 4096;   // two int64 per image fit the pinned readback buffer
int ibip_invade_batch_run(ibip_ctx *ctx, int n, IbipBatchItem *items, IbipBatchEarly early = nullptr,
                          void *user = nullptr);
// Scratch bytes the scans take for n entries.
size_t ibip_scan_scratch_bytes(int64_t n);

// Argument checks of one ibip_job, and the whole one-image path for it
// (EDT, invasion, trapping and curve as requested), synchronous on the
// context's stream; fills n_steps and returns the job's status.
bool ibip_job_valid(const ibip_job &J);
int ibip_run_job(ibip_ctx *ctx, ibip_job &J);

// Status helpers.
int ibip_cuda_status(cudaError_t e);

static inline int64_t nvox(ibip_dims d) { return (int64_t)d.nx * d.ny * d.nz; }

// ---- internal launchers (one file each) ---------------------------------
// EDT: feature = (image == 0).  Output dt2.
int ibip_edt_launch(ibip_ctx *ctx, const uint8_t *image, ibip_dims d, int32_t *dt2);
// The same for n images, one launch per pass (batched call).
int ibip_edt_batch_launch(ibip_ctx *ctx, int n, const uint8_t *const *images, const ibip_dims *dims,
                          int32_t *const *dt2);
// MIO helper: for feature = (W >= T), marks level[v] = lvl where level[v] == -1
// and the squared distance to the feature set is < Td.
int ibip_dilate_level_launch(ibip_ctx *ctx, const int32_t *W, int32_t T, int32_t Td, int32_t lvl, ibip_dims d,
                             int32_t *level);
// MIO with a per-voxel first level (uint8, L <= 254): fl[v] = first i with
// W[v] >= T[i]; then level i's trimmed set is {fl <= i}.
int ibip_first_level_launch(ibip_ctx *ctx, const int32_t *W, ibip_dims d, const int32_t *T_dev, int L, uint8_t *fl);
int ibip_dilate_first_level_launch(ibip_ctx *ctx, const uint8_t *fl, int32_t T, int32_t i, ibip_dims d,
                                   int32_t *level);
int ibip_max_launch(ibip_ctx *ctx, const int32_t *a, int64_t n, int *h_max);
// Maximin propagation from a face through voxels with val != 0 (val == -1
// counts as +inf).  Writes M (-1 where unreachable).
int ibip_maximin_launch(ibip_ctx *ctx, const int32_t *val, ibip_dims d, int face, int32_t *M,
                        int max_rounds);
// The same for several images in one cooperative launch.
struct IbipMaximinJob {
    const int32_t *val;
    ibip_dims d;
    int face;
    int32_t *M;
};
int ibip_maximin_multi(ibip_ctx *ctx, int n, const IbipMaximinJob *jobs, int max_rounds);
// Pore statistics of a dt2 image: stats[0] = largest finite value, [1] =
// pore voxels, [2] = 1 if any value is infinite (stats zeroed by the caller).
int ibip_stats_launch(ibip_ctx *ctx, const int32_t *dt2, int64_t N, int *stats);
// Paper-literal invasion (literal.cu); h_out = [steps, status].
// One image of a batched paper-literal invasion (ibip_invade_literal_batched).
struct IbipLitItem {
    const int32_t *dt2;
    ibip_dims d;
    int inlet;
    int64_t max_steps;
    int32_t *seq, *cstep, *step_r2, *step_count;
    int64_t cap;
    int64_t n_steps;   // filled
    int status;        // filled
};
// All images' setup, then one cluster per image in one launch (cluster =
// CTAs per image; 0 = automatic, tuned on the first call of a batch shape
// when ctx->autotune is on).  Writes the cluster size used to *h_cluster.
int ibip_literal_batch_run(ibip_ctx *ctx, int n, IbipLitItem *items, int cluster, int *h_cluster);
int ibip_literal_run(ibip_ctx *ctx, const int32_t *dt2, ibip_dims d, int inlet, int64_t max_steps, int32_t *seq,
                     int32_t *cstep, int32_t *step_r2, int32_t *step_count, int64_t cap, int64_t *h_out);
// Equal-saturation comparison of a sequence image with opening levels.
int ibip_eqsat_launch(ibip_ctx *ctx, const int32_t *seq, const int32_t *level, ibip_dims d, int64_t K, int L,
                      int64_t *h_steps, int64_t *h_diff, int64_t *h_count);
// Drainage envelope at opening levels (ibip_pc_envelope).
int ibip_envelope_launch(ibip_ctx *ctx, const int32_t *seq, ibip_dims d, const int32_t *step_r2, int64_t K,
                         const int32_t *h_levels, int L, int64_t *h_steps, int64_t *h_count);
// Trapped mask and saturation / Pc curve of many images in one launch per
// stage (batched call): M null = no trapping, S null = no curve.
struct IbipCurveItem {
    const int32_t *seq, *M;
    uint8_t *trapped;
    int32_t *seq_out;
    const int32_t *r2;
    float *S, *Pc;
    ibip_dims d;
    int64_t K;
    double voxel, sigma, cos_theta;
};
int ibip_curve_batch_launch(ibip_ctx *ctx, int n, const IbipCurveItem *items);
// Scratch bytes of that launch for n items with cnt_total pooled counts (sum of K + 2).
size_t ibip_curve_batch_bytes(int n, int64_t cnt_total);
// Scans.
int ibip_scan_excl_i32(ibip_ctx *ctx, const int32_t *in, int32_t *out, int64_t n);
int ibip_scan_incl_i32(ibip_ctx *ctx, const int32_t *in, int32_t *out, int64_t n);

__device__ __forceinline__ int64_t d_lin(int x, int y, int z, int ny, int nz)
{
    return ((int64_t)x * ny + y) * nz + z;
}

__device__ __forceinline__ bool d_on_face(int x, int y, int z, int nx, int ny, int nz, int face)
{
    switch (face) {
    case 0: return x == 0;
    case 1: return x == nx - 1;
    case 2: return y == 0;
    case 3: return y == ny - 1;
    case 4: return z == 0;
    default: return z == nz - 1;
    }
}

// floor(sqrt(e)) for 0 <= e < 2^31, exact.
__device__ __forceinline__ int d_isqrt(int e)
{
    int h = (int)sqrtf((float)e);
    while (h > 0 && (int64_t)h * h > e) h--;
    while ((int64_t)(h + 1) * (h + 1) <= e) h++;
    return h;
}

// largest r >= 0 with r*r < r2 (r2 >= 1): the ball's half-width along an axis
__device__ __forceinline__ int d_ball_hw(int r2) { return d_isqrt(r2 - 1); }

// Tile-shape tuning results (tune.cu): keyed by kernel, shape class and SM
// count; shared by the process, optionally persisted in a text file.
bool ibip_tune_get(const std::string &key, int *choice);
void ibip_tune_put(const std::string &key, int choice, double us, const char *path);
int ibip_tune_load(const char *path);
// EDT tile shapes (edt.cu): force one of the candidates (0, 0 = automatic),
// and the shape an EDT of these dimensions would use now.
int ibip_edt_tile_set(ibip_ctx *ctx, int z_warps, int strip_warps);
void ibip_edt_tile_get(ibip_ctx *ctx, ibip_dims d, int *z_warps, int *strip_warps);
