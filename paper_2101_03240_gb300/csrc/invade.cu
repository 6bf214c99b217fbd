// invade.cu -- volume-controlled invasion (Section 2.1, Figures 1-2).
//
// Step k picks the candidate with the largest dt2 (lowest linear index on
// ties) and stamps step k into every uninvaded voxel of the ball
// |p - c|^2 < dt2[c].  Candidates are uninvaded pore voxels 6-adjacent to an
// invaded voxel or lying on the inlet face.
//
// GPU design (one persistent CTA per image):
//  * Rank: pore voxels are ranked once by (dt2 descending, index ascending),
//    a stable counting sort over dt2 values (per-chunk bucket counts, one
//    flat scan, per-chunk stable scatter).  The priority order of the whole
//    invasion is this static rank, so the candidate set is a bitmap over
//    ranks (64-ary, four levels; the upper levels in shared memory, stale
//    summary bits cleared lazily) and "the best candidate" is its first set
//    bit.
//  * Bit-planes (one bit per voxel, rows padded to 32-bit words) hold
//    "pore and not invaded" (avail) and "ever queued as a candidate" (added).
//  * Speculative batches: each iteration takes the first M set bits of the
//    candidate bitmap (the M best candidates, in order).  Item j is skipped
//    when an earlier kept item's ball covers it (it will be invaded, not
//    chosen).  Every uninvaded, never-queued voxel u adjacent to kept ball i
//    would join the candidates after step i; if u outranks a later item it
//    would be chosen first, so the batch is cut to
//        J = min over such (i, u) of max(i + 1, #items ranked above u).
//    This bound only ever cuts too early, never too late, so the committed
//    prefix is exactly what one-step-at-a-time processing produces.  The
//    committed balls are stamped together (each voxel owned by the lowest
//    committed ball covering it), covered candidates leave the bitmap, and
//    new candidates (outside every committed ball) enter it.
#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>
#include <climits>

#include "common.cuh"

namespace {

constexpr int kM = 64;           // batch size (items per iteration)
constexpr int kNT = 768;         // threads of the persistent CTA (measured: 384, 512, 640, 768, 896, 1024 -> 1742, 1626, 1517, 1493, 1509, 1564 ms on the 512^3 blobs)
constexpr int kChunk = 4096;     // voxels per rank-sort chunk (minimum)
constexpr int kSmemL1Max = 12288;   // level-1 words of one image of a batched call (shared memory)
constexpr int kNOut = kInvStats;   // int64 outputs of the invasion kernel
static_assert(64 + kNOut * sizeof(long long) <= kSmallBytes, "output slot too small");

typedef unsigned long long u64;

__device__ __forceinline__ uint32_t ldcg32(const uint32_t *p) { return __ldcg(p); }
__device__ __forceinline__ u64 ldcg64(const u64 *p) { return __ldcg(p); }

// ------------------------------------------------------------ rank sort --

__global__ void k_stats(const int32_t *__restrict__ dt2, int64_t N, int *stats)
{
    int mx = 0, np = 0, inf = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        int d = dt2[v];
        if (d > 0) {
            np++;
            if (d == IBIP_INF32) inf = 1; else mx = max(mx, d);
        }
    }
    for (int o = 16; o; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        np += __shfl_xor_sync(0xffffffffu, np, o);
        inf |= __shfl_xor_sync(0xffffffffu, inf, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(stats + 0, mx);
        atomicAdd(stats + 1, np);
        atomicOr(stats + 2, inf);
    }
}

__global__ void k_presence(const int32_t *__restrict__ dt2, int64_t N, int32_t *pres)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        int d = dt2[v];
        if (d > 0 && d != IBIP_INF32) pres[d] = 1;
    }
}

// bucket of a pore voxel: 0 for the largest dt2 value present.  incl[d] is
// the inclusive count of present values <= d; B the number of values.
struct Bucket {
    const int32_t *incl;
    int B;
    int inf;   // image without solid: one bucket
    __device__ int operator()(int d) const
    {
        if (d <= 0) return -1;
        if (inf) return 0;
        return B - __ldg(incl + d);
    }
};

// One warp per chunk of voxels [c*S, c*S + S): counts per bucket into
// mat[b*C + c] (SMEM: counters in shared memory, B <= 1024).
template <bool SMEM>
__global__ void k_chunk_hist(const int32_t *__restrict__ dt2, int64_t N, int S, int C, Bucket bk,
                             int32_t *mat)
{
    extern __shared__ int32_t s_cnt[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = blockIdx.x * (blockDim.x >> 5) + w;
    if (c >= C) return;
    int32_t *cnt = SMEM ? s_cnt + w * bk.B : nullptr;
    for (int b = lane; b < bk.B; b += 32) {
        if (SMEM) cnt[b] = 0; else mat[(int64_t)b * C + c] = 0;
    }
    __syncwarp();
    int64_t v0 = (int64_t)c * S, v1 = min((int64_t)N, v0 + S);
    for (int64_t v = v0 + lane; v - lane < v1; v += 32) {
        int b = v < v1 ? bk(dt2[v]) : -1;
        unsigned peers = __match_any_sync(0xffffffffu, b);
        int leader = __ffs(peers) - 1;
        if (lane == leader && b >= 0) {
            if (SMEM) cnt[b] += __popc(peers);
            else mat[(int64_t)b * C + c] += __popc(peers);
        }
        __syncwarp();
    }
    if (SMEM)
        for (int b = lane; b < bk.B; b += 32) mat[(int64_t)b * C + c] = cnt[b];
}

template <bool SMEM>
__global__ void k_chunk_scatter(const int32_t *__restrict__ dt2, int64_t N, int S, int C, Bucket bk,
                                int32_t *mat, int32_t *__restrict__ rank, int2 *__restrict__ okey)
{
    extern __shared__ int32_t s_cnt[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = blockIdx.x * (blockDim.x >> 5) + w;
    if (c >= C) return;
    int32_t *cnt = SMEM ? s_cnt + w * bk.B : nullptr;
    if (SMEM) {
        for (int b = lane; b < bk.B; b += 32) cnt[b] = mat[(int64_t)b * C + c];
        __syncwarp();
    }
    int64_t v0 = (int64_t)c * S, v1 = min((int64_t)N, v0 + S);
    const unsigned lt = (1u << lane) - 1;
    for (int64_t v = v0 + lane; v - lane < v1; v += 32) {
        int d = v < v1 ? dt2[v] : 0;
        int b = v < v1 ? bk(d) : -1;
        unsigned peers = __match_any_sync(0xffffffffu, b);
        int leader = __ffs(peers) - 1;
        int base = 0;
        if (lane == leader && b >= 0) base = SMEM ? cnt[b] : mat[(int64_t)b * C + c];
        base = __shfl_sync(0xffffffffu, base, leader);
        if (b >= 0) {
            int r = base + __popc(peers & lt);
            rank[v] = r;
            okey[r] = make_int2((int)v, d);
        } else if (v < v1) {
            rank[v] = -1;
        }
        if (lane == leader && b >= 0) {
            if (SMEM) cnt[b] = base + __popc(peers);
            else mat[(int64_t)b * C + c] = base + __popc(peers);
        }
        __syncwarp();
    }
}

// out slot holding the rank of the first voxel with the smallest value (the
// single-voxel regime's dt2 = 1 bucket): every larger value ranks before it
constexpr int kFirst1Slot = 35;

__global__ void k_last_bucket_rank(const int32_t *pos, int base, int64_t *out)
{
    if (threadIdx.x == 0) *out = (int64_t)(*pos - base);
}

// ------------------------------------------- rank sort of many images --
// The same counting sort for every image of a batch at once: per-image
// arrays live at offsets in pooled buffers, one flat scan serves all images
// (each subtracts the pool's running total at its own start), and each
// kernel finds its image from its block index by binary search over the
// images' first blocks.
struct SortJob {
    const int32_t *dt2;
    int64_t N;
    int32_t *seq, *rank;
    int2 *okey;
    int64_t pres_off;   // first entry of this image's presence segment
    int maxd, hasinf;
    int pres_base;      // pool total before the segment (device-written)
    int B;              // distinct values (device-written, then read back)
    int S, C, smem;     // chunk length, chunks, counters in shared memory
    int64_t mat_off;    // first entry of this image's (bucket, chunk) matrix
    int mat_base;       // pool total before the matrix (device-written)
    int blk_vox, blk_chunk;   // first block of this image in the voxel / chunk launches
    int64_t *out;             // the invasion's output slots (the last bucket's first rank goes there)
};

__device__ __forceinline__ int find_job(const SortJob *jobs, int n, int blk, bool chunk)
{
    int lo = 0, hi = n;   // largest j whose first block is <= blk
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if ((chunk ? jobs[mid].blk_chunk : jobs[mid].blk_vox) <= blk) lo = mid; else hi = mid;
    }
    return lo;
}

constexpr int kVoxBlock = 256, kVoxPer = 8;   // voxel launches: 2048 voxels per block

// seq = -1 on pore, 0 on solid; presence of each finite value
__global__ void k_seq_pres_b(const SortJob *__restrict__ jobs, int n, int32_t *pres)
{
    const int j = find_job(jobs, n, blockIdx.x, false);
    const SortJob &J = jobs[j];
    const int64_t v0 = (int64_t)(blockIdx.x - J.blk_vox) * kVoxBlock * kVoxPer;
    for (int q = 0; q < kVoxPer; q++) {
        const int64_t v = v0 + q * kVoxBlock + threadIdx.x;
        if (v >= J.N) break;
        const int d = J.dt2[v];
        J.seq[v] = d > 0 ? -1 : 0;
        if (d > 0 && d != IBIP_INF32) pres[J.pres_off + d] = 1;
    }
}

// pore statistics of many images (as k_stats), kVoxBlock * kVoxPer voxels
// per block; a block finds its image by binary search over first blocks
struct StatJob {
    const int32_t *dt2;
    int64_t N;
    int blk;
};

__global__ void k_stats_b(const StatJob *__restrict__ jobs, int n, int *stats)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (jobs[mid].blk <= (int)blockIdx.x) lo = mid; else hi = mid;
    }
    const StatJob &J = jobs[lo];
    const int64_t v0 = (int64_t)(blockIdx.x - J.blk) * kVoxBlock * kVoxPer;
    int mx = 0, np = 0, inf = 0;
    for (int q = 0; q < kVoxPer; q++) {
        const int64_t v = v0 + q * kVoxBlock + threadIdx.x;
        if (v >= J.N) break;
        const int d = J.dt2[v];
        if (d > 0) {
            np++;
            if (d == IBIP_INF32) inf = 1; else mx = max(mx, d);
        }
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    np = __reduce_add_sync(0xffffffffu, np);
    inf = __reduce_or_sync(0xffffffffu, inf);
    if ((threadIdx.x & 31) == 0 && (np | inf)) {
        atomicMax(stats + 3 * lo, mx);
        atomicAdd(stats + 3 * lo + 1, np);
        atomicOr(stats + 3 * lo + 2, inf);
    }
}

// after the flat inclusive scan of the presence pool: each image's base and
// number of distinct values
__global__ void k_pres_base_b(SortJob *jobs, int n, const int32_t *__restrict__ incl)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    SortJob &J = jobs[j];
    const int base = J.pres_off > 0 ? incl[J.pres_off - 1] : 0;
    J.pres_base = base;
    J.B = J.hasinf ? 1 : incl[J.pres_off + J.maxd] - base;
}

__device__ __forceinline__ int bucket_b(const SortJob &J, const int32_t *__restrict__ incl, int d)
{
    if (d <= 0) return -1;
    if (J.hasinf) return 0;
    return J.B - (__ldg(incl + J.pres_off + d) - J.pres_base);
}

// k_chunk_hist for every image: one warp per chunk
__global__ void k_chunk_hist_b(const SortJob *__restrict__ jobs, int n, const int32_t *__restrict__ incl,
                               int32_t *mat)
{
    extern __shared__ int32_t s_cnt[];
    const int j = find_job(jobs, n, blockIdx.x, true);
    const SortJob &J = jobs[j];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = (blockIdx.x - J.blk_chunk) * (blockDim.x >> 5) + w;
    if (c >= J.C) return;
    int32_t *m = mat + J.mat_off;
    int32_t *cnt = J.smem ? s_cnt + w * J.B : nullptr;
    for (int b = lane; b < J.B; b += 32) {
        if (J.smem) cnt[b] = 0; else m[(int64_t)b * J.C + c] = 0;
    }
    __syncwarp();
    const int64_t v0 = (int64_t)c * J.S, v1 = min(J.N, v0 + J.S);
    for (int64_t v = v0 + lane; v - lane < v1; v += 32) {
        const int b = v < v1 ? bucket_b(J, incl, J.dt2[v]) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(peers) - 1;
        if (lane == leader && b >= 0) {
            if (J.smem) cnt[b] += __popc(peers);
            else m[(int64_t)b * J.C + c] += __popc(peers);
        }
        __syncwarp();
    }
    if (J.smem)
        for (int b = lane; b < J.B; b += 32) m[(int64_t)b * J.C + c] = cnt[b];
}

// after the flat exclusive scan of the matrix pool: each image's base
__global__ void k_mat_base_b(SortJob *jobs, int n, const int32_t *__restrict__ mat)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    SortJob &J = jobs[j];
    J.mat_base = mat[J.mat_off];
    J.out[kFirst1Slot] = (int64_t)(mat[J.mat_off + (int64_t)(J.B - 1) * J.C] - J.mat_base);
}

__global__ void k_chunk_scatter_b(const SortJob *__restrict__ jobs, int n, const int32_t *__restrict__ incl,
                                  int32_t *mat)
{
    extern __shared__ int32_t s_cnt[];
    const int j = find_job(jobs, n, blockIdx.x, true);
    const SortJob &J = jobs[j];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = (blockIdx.x - J.blk_chunk) * (blockDim.x >> 5) + w;
    if (c >= J.C) return;
    int32_t *m = mat + J.mat_off;
    int32_t *cnt = J.smem ? s_cnt + w * J.B : nullptr;
    if (J.smem) {
        for (int b = lane; b < J.B; b += 32) cnt[b] = m[(int64_t)b * J.C + c] - J.mat_base;
        __syncwarp();
    }
    const int64_t v0 = (int64_t)c * J.S, v1 = min(J.N, v0 + J.S);
    const unsigned lt = (1u << lane) - 1;
    for (int64_t v = v0 + lane; v - lane < v1; v += 32) {
        const int d = v < v1 ? J.dt2[v] : 0;
        const int b = v < v1 ? bucket_b(J, incl, d) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (lane == leader && b >= 0) base = J.smem ? cnt[b] : m[(int64_t)b * J.C + c] - J.mat_base;
        base = __shfl_sync(0xffffffffu, base, leader);
        if (b >= 0) {
            const int r = base + __popc(peers & lt);
            J.rank[v] = r;
            J.okey[r] = make_int2((int)v, d);
        } else if (v < v1) {
            J.rank[v] = -1;
        }
        if (lane == leader && b >= 0) {
            if (J.smem) cnt[b] = base + __popc(peers);
            else m[(int64_t)b * J.C + c] = base + __popc(peers) + J.mat_base;
        }
        __syncwarp();
    }
}

// ------------------------------------------------------- invasion state --

struct Inv {
    int nx, ny, nz, NW, inlet;
    int NL0, NL1, NL2, NL3;
    int64_t max_steps, cap, npore;
    int isq_n;         // entries of the shared-memory isqrt table
    const int32_t *rank;
    const int2 *okey;
    const int32_t *dt2;
    uint32_t *avail, *added;
    u64 *fb0, *fb1, *fb2, *fb3;
    int32_t *seq, *step_r2, *step_centre;
    int64_t *out;      // out[0] = steps, out[1] = status, out[2] = iterations
    const uint8_t *mask;   // inlet voxels (nonzero), or null: the inlet face
    int resume;            // seq holds an earlier run's steps 1..k0 on entry
    int64_t k0;            // steps already taken (resume), else 0
    int4 *trace;           // per-batch records (two int4 each, see trace_batch), or null
    const int *cancel;     // host-mapped cancel flag, polled every few batches, or null
    int64_t trace_cap;     // records that fit in trace
};

// Global accesses of the invasion loop.  In a checked build (IBIP_CHECKED)
// each index is compared with its array's extent first: an index outside
// it is counted in out[kErrSlot] and the access is skipped (a load gives a
// neutral value), and the call returns IBIP_ERR_BOUNDS; nothing traps.  In
// the normal build they are the plain accesses.
constexpr int kErrSlot = 34;
__device__ __forceinline__ bool in_range(const Inv &a, int64_t i, int64_t n)
{
#ifdef IBIP_CHECKED
    if (i >= 0 && i < n) return true;
    atomicAdd((unsigned long long *)(a.out + kErrSlot), 1ull);
    return false;
#else
    (void)a; (void)i; (void)n;
    return true;
#endif
}
__device__ __forceinline__ int64_t n_vox(const Inv &a) { return (int64_t)a.nx * a.ny * a.nz; }
__device__ __forceinline__ int64_t n_words(const Inv &a) { return (int64_t)a.nx * a.ny * a.NW; }
__device__ __forceinline__ void seq_put(const Inv &a, int64_t v, int32_t label)
{
    if (in_range(a, v, n_vox(a))) a.seq[v] = label;
}
__device__ __forceinline__ int rank_at(const Inv &a, int64_t v)
{
    return in_range(a, v, n_vox(a)) ? __ldg(a.rank + v) : 0;
}
__device__ __forceinline__ void fb0_set(const Inv &a, int r)
{
    if (in_range(a, r >> 6, a.NL0)) atomicOr(a.fb0 + (r >> 6), 1ull << (r & 63));
}
__device__ __forceinline__ void fb0_clear(const Inv &a, int r)
{
    if (in_range(a, r >> 6, a.NL0)) atomicAnd(a.fb0 + (r >> 6), ~(1ull << (r & 63)));
}
__device__ __forceinline__ uint32_t plane_ld(const Inv &a, const uint32_t *pl, int64_t w)
{
    return in_range(a, w, n_words(a)) ? ldcg32(pl + w) : 0u;
}
__device__ __forceinline__ void plane_and(const Inv &a, uint32_t *pl, int64_t w, uint32_t m)
{
    if (in_range(a, w, n_words(a))) atomicAnd(pl + w, m);
}
// returns the word before the OR (all ones when out of range: nothing new)
__device__ __forceinline__ uint32_t plane_or(const Inv &a, uint32_t *pl, int64_t w, uint32_t m)
{
    return in_range(a, w, n_words(a)) ? atomicOr(pl + w, m) : 0xffffffffu;
}
__device__ __forceinline__ void list_put(const Inv &a, int *g, int64_t i, int v)
{
    if (in_range(a, i, a.npore)) g[i] = v;
}

__global__ void k_seq_init(const int32_t *__restrict__ dt2, int64_t N, int32_t *seq)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
        seq[v] = dt2[v] > 0 ? -1 : 0;
}

// one thread per bit-plane word: avail bits (pore, not yet invaded) and the
// first candidates: inlet voxels (the mask, else the inlet face) and, when
// resuming, every uninvaded pore voxel next to an invaded one
__device__ void plane_word(const Inv &a, int64_t w)
{
    int64_t row = w / a.NW;
    int zw = (int)(w - row * a.NW);
    int x = (int)(row / a.ny), y = (int)(row - (int64_t)x * a.ny);
    uint32_t av = 0, ad = 0;
    for (int b = 0; b < 32; b++) {
        int z = zw * 32 + b;
        if (z >= a.nz) break;
        int64_t v = row * a.nz + z;
        if (a.dt2[v] <= 0) continue;
        if (a.resume && a.seq[v] != -1) continue;
        av |= 1u << b;
        bool cand = a.mask ? a.mask[v] != 0 : d_on_face(x, y, z, a.nx, a.ny, a.nz, a.inlet);
        if (!cand && a.resume) {
            const int nxs[6] = {x - 1, x + 1, x, x, x, x}, nys[6] = {y, y, y - 1, y + 1, y, y},
                      nzs[6] = {z, z, z, z, z - 1, z + 1};
            for (int q = 0; q < 6 && !cand; q++) {
                if (nxs[q] < 0 || nys[q] < 0 || nzs[q] < 0 || nxs[q] >= a.nx || nys[q] >= a.ny || nzs[q] >= a.nz)
                    continue;
                cand = a.seq[d_lin(nxs[q], nys[q], nzs[q], a.ny, a.nz)] >= 1;
            }
        }
        if (cand) {
            ad |= 1u << b;
            int r = a.rank[v];
            fb0_set(a, r);
            atomicOr(a.fb1 + (r >> 12), 1ull << ((r >> 6) & 63));
            atomicOr(a.fb2 + (r >> 18), 1ull << ((r >> 12) & 63));
            atomicOr(a.fb3 + (r >> 24), 1ull << ((r >> 18) & 63));
        }
    }
    a.avail[w] = av;
    a.added[w] = ad;
}

__global__ void k_plane_init(Inv a)
{
    const int64_t nw = (int64_t)a.nx * a.ny * a.NW;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x)
        plane_word(a, w);
}

// n / d for 0 <= n < 2^31 and a run-time invariant d >= 1: one multiply-high
// and two shifts (Granlund & Montgomery, "Division by invariant integers
// using multiplication", 1994; the round-up variant for unsigned n).
struct FastDiv {
    uint32_t d, m;
    int s;
};

FastDiv make_fastdiv(uint32_t d)
{
    FastDiv f{d, 0u, 0};
    if (d <= 1) return f;
    int s = 0;
    while ((1ull << s) < d) s++;
    f.s = s;
    f.m = (uint32_t)((((1ull << 32) * ((1ull << s) - d)) / d) + 1);
    return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv &f)
{
    if (f.d <= 1) return n;
    uint32_t t = __umulhi(f.m, n);
    return (t + ((n - t) >> 1)) >> (f.s - 1);
}

constexpr int kList = 2048;        // shared-memory work-list entries
constexpr int kRowBudget = 8192;   // ball rows per batch (at least one item)

// floor(sqrt(e)): table lookup below n (shared memory), exact integer
// square root above
struct Isq {
    const int *t;
    int n;
    __device__ __forceinline__ int operator()(int e) const { return e < n ? t[e] : d_isqrt(e); }
};

struct Batch {
    int idx[kM], r2[kM], x[kM], y[kM], z[kM], rank[kM], step[kM], h[kM];
    int bx0[kM], by0[kM], wy[kM];      // ball rows: clamped bounding square
    int dx0[kM], dy0[kM], dwy[kM];     // shell rows: the square grown by one
    int upre[kM + 1], dpre[kM + 1];    // prefix sums of ball rows / shell rows
    u64 ovl[kM];
    u64 keep;
    Isq isq;
    u64 big;
    int bigl[kM];      // the items of `big`, in order
    uint32_t cont32[kM][2], ovl32[kM][2];
    int m, mcap, J, stop, mtarget, tstop;
    int cur1;          // no level-1 summary word below this index is set
    int nA, nC, nD;    // work-list fill counts (shell candidates, removals, additions)
    int ovf;           // the shell-candidate list overflowed this iteration
    int64_t kk;        // step count handed back by the single-voxel loop
    // single-voxel loop: candidates queued by the last commit, the rank up
    // to which the batch holds every candidate, and the next batch's source
    int nN, novf, tmerge, Rk, nT, minN;
};

// bits [a, b] (inclusive, within word w of a row) as a mask
__device__ __forceinline__ uint32_t span_mask(int w, int a, int b)
{
    int lo = max(a - w * 32, 0), hi = min(b - w * 32, 31);
    if (lo > hi) return 0u;
    uint32_t m = 0xffffffffu >> (31 - hi);
    return m & (0xffffffffu << lo);
}

// Squared offsets fit in int32: dimensions are at most 16384, so
// dx^2 + dy^2 + dz^2 < 2^30, and r2 - 1 - dx^2 - dy^2 >= -2^29 even for
// r2 = INT32_MAX (an image without solid).
// z-interval of ball i at row (x, y): returns false if the row misses it
__device__ __forceinline__ bool ball_run(const Batch &B, int i, int x, int y, int &lo, int &hi)
{
    const int dx = x - B.x[i], dy = y - B.y[i];
    const int e = B.r2[i] - 1 - dx * dx - dy * dy;
    if (e < 0) return false;
    const int h = B.isq(e);
    lo = B.z[i] - h;
    hi = B.z[i] + h;
    return true;
}


// Half-width of ball i's run at row (x, y), -1 when the row misses the ball
// or lies outside the image.
__device__ __forceinline__ int run_hw(const Inv &a, const Batch &B, int i, int x, int y)
{
    if (x < 0 || y < 0 || x >= a.nx || y >= a.ny) return -1;
    const int dx = x - B.x[i], dy = y - B.y[i];
    const int e = B.r2[i] - 1 - dx * dx - dy * dy;
    return e < 0 ? -1 : B.isq(e);
}

// The shell of ball i in row (x, y): voxels outside the ball with a face
// neighbour inside it.  With h the row's own half-width and hl the largest
// half-width of the four lateral rows, they are hR < |z - cz| <= Hs,
// Hs = max(hl, h + 1 if the row meets the ball).  Returns false if empty;
// else the z-span [za, zb] to scan and the ball's own run [ra, rb] to mask
// out (ra > rb when the row misses the ball), clamped to the image.
__device__ __forceinline__ bool shell_row(const Inv &a, const Batch &B, int i, int x, int y, int &za, int &zb,
                                          int &ra, int &rb)
{
    const int h = run_hw(a, B, i, x, y);
    int hs = max(max(run_hw(a, B, i, x - 1, y), run_hw(a, B, i, x + 1, y)),
                 max(run_hw(a, B, i, x, y - 1), run_hw(a, B, i, x, y + 1)));
    if (h >= 0) hs = max(hs, h + 1);
    if (hs < 0) return false;
    const int cz = B.z[i];
    za = max(cz - hs, 0);
    zb = min(cz + hs, a.nz - 1);
    ra = h >= 0 ? cz - h : 1;
    rb = h >= 0 ? cz + h : 0;
    return za <= zb;
}

__device__ __forceinline__ int lower_rank(const Batch &B, int m, int r)
{
    int lo = 0, hi = m;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (B.rank[mid] < r) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int unit_item(const int *pre, int n, int u)
{
    int lo = 0, hi = n;   // largest i with pre[i] <= u
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (pre[mid] <= u) lo = mid; else hi = mid;
    }
    return lo;
}


// Thread tid's contiguous share of the row units [0, U) of items [0, n):
// f(u, i, x, y) for each unit u, i its item (pre = prefix sums of the items'
// unit counts) and (x, y) its row in the item's square (origin sx0/sy0,
// width swy).  Consecutive units of one item advance (x, y) without a
// division; f returns false to stop early.
template <class F>
__device__ __forceinline__ void for_units(const int *pre, int n, int U, const int *sx0, const int *sy0,
                                          const int *swy, int tid, F f)
{
    const int C = (U + kNT - 1) / kNT;
    int u = tid * C;
    const int u1 = min(U, u + C);
    if (u >= u1) return;
    int i = unit_item(pre, n + 1, u);
    int t = u - pre[i];
    int w = swy[i], y0 = sy0[i];
    int x = sx0[i] + t / w, y = y0 + t % w;
    int nxt = pre[i + 1];
    for (; u < u1; u++) {
        while (u >= nxt) {
            i++;
            nxt = pre[i + 1];
            w = swy[i];
            y0 = sy0[i];
            x = sx0[i];
            y = y0;
        }
        if (!f(u, i, x, y)) return;
        if (++y >= y0 + w) { y = y0; x++; }
    }
}

// position of the k-th (0-based) set bit of a 32-bit word: binary search on
// popcounts of the lower halves
__device__ __forceinline__ int nth_bit32(uint32_t w, int k)
{
    int pos = 0, c;
    c = __popc(w & 0xffffu); if (k >= c) { k -= c; w >>= 16; pos += 16; }
    c = __popc(w & 0xffu);   if (k >= c) { k -= c; w >>= 8;  pos += 8; }
    c = __popc(w & 0xfu);    if (k >= c) { k -= c; w >>= 4;  pos += 4; }
    c = __popc(w & 0x3u);    if (k >= c) { k -= c; w >>= 2;  pos += 2; }
    c = (int)(w & 1u);       if (k >= c) { pos += 1; }
    return pos;
}

// position of the k-th (0-based) set bit of w
__device__ __forceinline__ int nth_bit(u64 w, int k)
{
    uint32_t lo = (uint32_t)w;
    int pl = __popc(lo);
    if (k < pl) return nth_bit32(lo, k);
    return 32 + nth_bit32((uint32_t)(w >> 32), k - pl);
}

// The six face neighbours of voxel (x, y, z) with linear index v: for each,
// whether it is inside the image, its bit-plane word index and bit, and its
// linear index.
struct Nb6 {
    int64_t word[6];
    int v[6];
    uint32_t bit[6];
    bool ok[6];
};

__device__ __forceinline__ void nb6(const Inv &a, int x, int y, int z, int v, Nb6 &n)
{
    const int64_t row = (int64_t)x * a.ny + y;
    const int64_t nyz = (int64_t)a.ny * a.nz;
    n.ok[0] = z > 0;          n.v[0] = v - 1;              n.word[0] = row * a.NW + ((z - 1) >> 5);  n.bit[0] = 1u << ((z - 1) & 31);
    n.ok[1] = z < a.nz - 1;   n.v[1] = v + 1;              n.word[1] = row * a.NW + ((z + 1) >> 5);  n.bit[1] = 1u << ((z + 1) & 31);
    n.ok[2] = y > 0;          n.v[2] = v - a.nz;           n.word[2] = (row - 1) * a.NW + (z >> 5);   n.bit[2] = 1u << (z & 31);
    n.ok[3] = y < a.ny - 1;   n.v[3] = v + a.nz;           n.word[3] = (row + 1) * a.NW + (z >> 5);   n.bit[3] = 1u << (z & 31);
    n.ok[4] = x > 0;          n.v[4] = (int)(v - nyz);     n.word[4] = (row - a.ny) * a.NW + (z >> 5); n.bit[4] = 1u << (z & 31);
    n.ok[5] = x < a.nx - 1;   n.v[5] = (int)(v + nyz);     n.word[5] = (row + a.ny) * a.NW + (z >> 5); n.bit[5] = 1u << (z & 31);
}

// Candidate mask (bit q set = neighbour q is uninvaded and never queued),
// all twelve bit-plane loads issued together.
__device__ __forceinline__ unsigned nb6_candidates(const Inv &a, const Nb6 &n)
{
    uint32_t av[6], ad[6];
#pragma unroll
    for (int q = 0; q < 6; q++) {
        av[q] = n.ok[q] ? plane_ld(a, a.avail, n.word[q]) : 0u;
        ad[q] = n.ok[q] ? plane_ld(a, a.added, n.word[q]) : 0u;
    }
    unsigned c = 0;
#pragma unroll
    for (int q = 0; q < 6; q++)
        if ((av[q] & n.bit[q]) && !(ad[q] & n.bit[q])) c |= 1u << q;
    return c;
}

// Diagnostic counters of the invasion, kept by thread 0 in shared memory
// (slot = index in the kernel's output, see ibip_invade_stats).
enum Diag {
    D_ITERS = 2, D_SEL = 3, D_BOUND = 4, D_COMMIT = 5, D_ITEMS = 6, D_COMMITTED = 7, D_STALE = 8, D_ROWS = 9,
    D_SMALL_CYC = 10, D_SMALL_N = 11, D_GATHER = 12, D_PAIRS = 14, D_TAIL = 15, D_SMALL_SEL = 16,
    D_SMALL_BOUND = 17, D_SMALL_COMMIT = 18, D_TINY_IT = 19, D_TINY_STEPS = 20, D_TINY_CYC = 21, D_S3_CONT = 22,
    D_S3_PREFIX = 23, D_B1 = 24, D_B2 = 25, D_M1 = 26, D_M2 = 27, D_TG = 28, D_TB = 29, D_TC = 33, D_TRACE = 36,
    D_SPAN_CYC = 37, D_SPAN_NS = 38, D_SHELL_UNITS = 39, D_LISTED = 40, D_REMOVED = 41, D_SINGLE = 42,
    D_TMERGE = 43, D_TMERGE_CYC = 44, D_GROUNDS = 45, D_GATHERS = 46
};

// Warp-wide: the first (up to mt) set bits of the rank bitmap, i.e. the best
// candidates in priority order, written to rank_out[0..m); returns m (0 when
// no candidate is left).  Lane 0 walks the summary levels to the first
// flagged level-1 word; the warp loads the level-0 words of up to 32 flagged
// entries of that and the next three level-1 words, unflags the empty ones
// (stale summary bits: removals never clear summaries) and takes the
// leading set bits, each lane extracting up to two of them.
template <bool L1SMEM>
__device__ int gather_top(const Inv &a, u64 *s1, u64 *s2, u64 *s3, int *cur1, int lane, int mt, int *rank_out,
                          long long *n_stale)
{
    for (;;) {
        // first two non-empty level-1 words: scan 32 words from the cursor
        // (every level-1 word below it is empty), else walk the summaries
        const int c = *(volatile int *)cur1;
        const int q = c + lane;
        const u64 wl = q < a.NL1 ? (L1SMEM ? s1[q] : ldcg64(s1 + q)) : 0ull;
        unsigned nz = __ballot_sync(0xffffffffu, wl != 0ull);
        int i1a = -1, i1b = -1;
        u64 wa = 0, wb = 0;
        if (nz) {
            const int la = __ffs(nz) - 1;
            i1a = c + la;
            wa = __shfl_sync(0xffffffffu, wl, la);
            nz &= nz - 1;
            if (nz) {
                const int lb = __ffs(nz) - 1;
                i1b = c + lb;
                wb = __shfl_sync(0xffffffffu, wl, lb);
            }
        } else {
            if (lane == 0) {
                for (;;) {
                    int i3 = -1;
                    for (int t = 0; t < a.NL3; t++) if (s3[t]) { i3 = t; break; }
                    if (i3 < 0) break;
                    int i2 = i3 * 64 + __ffsll(s3[i3]) - 1;
                    u64 w2 = s2[i2];
                    if (!w2) { s3[i3] &= ~(1ull << (i2 & 63)); continue; }
                    int c1 = i2 * 64 + __ffsll(w2) - 1;
                    u64 w1 = L1SMEM ? s1[c1] : ldcg64(s1 + c1);
                    if (!w1) {
                        s2[i2] &= ~(1ull << (c1 & 63));
                        if (!s2[i2]) s3[i3] &= ~(1ull << (i2 & 63));
                        continue;
                    }
                    i1a = c1;
                    wa = w1;
                    break;
                }
            }
            i1a = __shfl_sync(0xffffffffu, i1a, 0);
            wa = __shfl_sync(0xffffffffu, wa, 0);
        }
        if (i1a < 0) return 0;
        if (lane == 0) *cur1 = i1a;
        // lane l takes the l-th flagged level-0 word of the two level-1 words
        const int pa = __popcll(wa);
        int c0 = -1;
        if (lane < pa) c0 = i1a * 64 + nth_bit(wa, lane);
        else if (i1b >= 0 && lane - pa < __popcll(wb)) c0 = i1b * 64 + nth_bit(wb, lane - pa);
        u64 w0 = c0 >= 0 ? ldcg64(a.fb0 + c0) : 0ull;
        const bool st = c0 >= 0 && w0 == 0ull;
        if (st) {   // unflag: bit (c0 & 63) of level-1 word c0 >> 6, as a 32-bit half
            uint32_t *p = (uint32_t *)(s1 + (c0 >> 6)) + ((c0 >> 5) & 1);
            atomicAnd(p, ~(1u << (c0 & 31)));
        }
        const unsigned stale = __ballot_sync(0xffffffffu, st);
        if (lane == 0) {
            if (stale) n_stale[0] += __popc(stale);
            n_stale[D_GROUNDS - D_STALE]++;   // rounds of the gather
        }
        const int cnt = __popcll(w0);
        int inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        const int tot = __shfl_sync(0xffffffffu, inc, 31);
        if (tot == 0) {
            __syncwarp();
            continue;
        }
        const int m = min(tot, mt);
        if (__reduce_max_sync(0xffffffffu, (unsigned)cnt) <= 4) {
            // sparse words: each lane writes the items of its own word, in
            // order, from the exclusive prefix of the counts on
            u64 w = w0;
            for (int p = inc - cnt; w && p < m; p++, w &= w - 1) rank_out[p] = c0 * 64 + __ffsll((long long)w) - 1;
        } else {
            // dense words: item p (p = lane, lane + 32) comes from the lane
            // whose inclusive count first exceeds p
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int p = lane + 32 * h;
                int lo = 0;
#pragma unroll
                for (int step = 16; step; step >>= 1) {
                    int v = __shfl_sync(0xffffffffu, inc, lo + step - 1);
                    if (v <= p) lo += step;
                }
                const int src = min(lo, 31);
                const u64 w = __shfl_sync(0xffffffffu, w0, src);
                const int ex = __shfl_sync(0xffffffffu, inc - cnt, src);
                const int cw = __shfl_sync(0xffffffffu, c0, src);
                if (p < m) rank_out[p] = cw * 64 + nth_bit(w, p - ex);
            }
        }
        __syncwarp();
        return m;
    }
}

// Warp 0: the batch items (up to mt best candidates) with their data in B:
// rank, linear index, dt2, coordinates and, with FULL, the ball's half-width,
// clamped bounding square and row count (in upre[j + 1]).  Returns m.
template <bool L1SMEM, bool FULL>
__device__ int gather_items(const Inv &a, Batch &B, u64 *s1, u64 *s2, u64 *s3, int lane, int mt,
                            const FastDiv &fd_nyz, const FastDiv &fd_nz, long long *n_stale)
{
    const int m = gather_top<L1SMEM>(a, s1, s2, s3, &B.cur1, lane, mt, B.rank, n_stale);
    if (lane == 0) n_stale[D_GATHERS - D_STALE]++;
    const uint32_t nyz = (uint32_t)a.ny * (uint32_t)a.nz;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int j = lane + 32 * h;
        if (j >= m) continue;
        const int rkj = B.rank[j];
        const int2 e = __ldg(a.okey + rkj);
        const uint32_t x = fdiv((uint32_t)e.x, fd_nyz);
        const uint32_t rem = (uint32_t)e.x - x * nyz;
        const uint32_t y = fdiv(rem, fd_nz);
        B.idx[j] = e.x;
        B.r2[j] = e.y;
        B.x[j] = (int)x; B.y[j] = (int)y; B.z[j] = (int)(rem - y * (uint32_t)a.nz);
        if (FULL) {
            const int hw = B.isq(e.y - 1);
            B.h[j] = hw;
            const int x0 = max((int)x - hw, 0), x1 = min((int)x + hw, a.nx - 1);
            const int y0 = max((int)y - hw, 0), y1 = min((int)y + hw, a.ny - 1);
            B.bx0[j] = x0; B.by0[j] = y0; B.wy[j] = y1 - y0 + 1;
            B.upre[j + 1] = (x1 - x0 + 1) * (y1 - y0 + 1);
            const int u0 = max((int)x - hw - 1, 0), u1 = min((int)x + hw + 1, a.nx - 1);
            const int v0 = max((int)y - hw - 1, 0), v1 = min((int)y + hw + 1, a.ny - 1);
            B.dx0[j] = u0; B.dy0[j] = v0; B.dwy[j] = v1 - v0 + 1;
            // single-voxel balls use one shell unit (their six neighbours)
            B.dpre[j + 1] = e.y == 1 ? 1 : (u1 - u0 + 1) * (v1 - v0 + 1);
            B.cont32[j][0] = B.cont32[j][1] = 0u;
            B.ovl32[j][0] = B.ovl32[j][1] = 0u;
        }
    }
    __syncwarp();
    return m;
}

// Flag rank r in the three summary levels (32-bit halves of the 64-bit
// words; bit index r >> 6 in level 1, r >> 12 in level 2, r >> 18 in level 3).
// While a commit runs the summaries only gain bits (the gather clears stale
// ones in its own phase) and the cursor only falls, so each is read first
// and written only when it changes: most additions touch no shared atomic.
__device__ __forceinline__ void flag_rank(u64 *s1, u64 *s2, u64 *s3, int *cur1, int r)
{
    uint32_t *p1 = (uint32_t *)s1 + (r >> 11), *p2 = (uint32_t *)s2 + (r >> 17), *p3 = (uint32_t *)s3 + (r >> 23);
    const uint32_t b1 = 1u << ((r >> 6) & 31), b2 = 1u << ((r >> 12) & 31), b3 = 1u << ((r >> 18) & 31);
    const int c = *(volatile int *)cur1;
    const uint32_t w1 = *(volatile uint32_t *)p1, w2 = *(volatile uint32_t *)p2, w3 = *(volatile uint32_t *)p3;
    if ((r >> 12) < c) atomicMin(cur1, r >> 12);
    if (!(w1 & b1)) atomicOr(p1, b1);
    if (!(w2 & b2)) atomicOr(p2, b2);
    if (!(w3 & b3)) atomicOr(p3, b3);
}

__device__ __forceinline__ void bar_sync_64() { asm volatile("bar.sync 1, 64;" ::: "memory"); }

// SM clock for the phase timers: read only in the profiling kernel (the
// reads are scheduling barriers that cost the loop about a tenth of its time)
template <bool P>
__device__ __forceinline__ long long tclk()
{
    if constexpr (P) return clock64();
    else return 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}


// One timing record per batch (thread 0): first step (0-based), steps
// committed, SM cycles from batch selection to the end of its commit, the
// loop that ran it (0 main, 1 single-voxel), then items taken, ball rows
// stamped, shell rows scanned and shell candidates listed (the last two 0
// in the single-voxel loop).  Counted past the capacity.
__device__ __forceinline__ void trace_batch(const Inv &a, long long &ntr, int64_t k, int n, long long cyc, int loop,
                                            int items, int rows, int shell, int listed)
{
    if (!a.trace) return;
    if (ntr < a.trace_cap) {
        a.trace[2 * ntr] = make_int4((int)k, n, (int)min(cyc, (long long)INT_MAX), loop);
        a.trace[2 * ntr + 1] = make_int4(items, rows, shell, listed);
    }
    ntr++;
}

// The lone item of a batch (ball larger than its centre), committed as step
// `label`: per row of its one-voxel-dilated square, the voxels of its run
// that are still uninvaded are stamped (those that were queued leave the
// rank bitmap) and the uninvaded, never-queued voxels of the shell part of
// the row are queued.  Rows are disjoint, so their words are too; nothing
// else runs meanwhile.
__device__ __forceinline__ void commit_single(const Inv &a, const Batch &B, u64 *s1, u64 *s2, u64 *s3, int tid,
                                              int32_t label)
{
    for_units(B.dpre, 1, B.dpre[1], B.dx0, B.dy0, B.dwy, tid, [&](int, int, int x, int y) -> bool {
        int za, zb, ra, rb;
        if (!shell_row(a, B, 0, x, y, za, zb, ra, rb)) return true;
        const int r0 = max(ra, 0), r1 = min(rb, a.nz - 1);   // the ball's run (empty when r0 > r1)
        const int64_t row = (int64_t)x * a.ny + y;
        const int64_t vb = row * a.nz;
        for (int w = za >> 5; w <= (zb >> 5); w++) {
            const int64_t rw = row * a.NW + w;
            const uint32_t av = plane_ld(a, a.avail, rw), ad = plane_ld(a, a.added, rw);
            const uint32_t ballm = r0 <= r1 ? span_mask(w, r0, r1) : 0u;
            const uint32_t newly = av & ballm;
            const uint32_t cand = av & ~ad & span_mask(w, za, zb) & ~ballm;
            if (newly) plane_and(a, a.avail, rw, ~newly);
            if (cand) plane_or(a, a.added, rw, cand);
            for (uint32_t n2 = newly; n2; n2 &= n2 - 1) seq_put(a, vb + w * 32 + __ffs(n2) - 1, label);
            for (uint32_t g = newly & ad; g; g &= g - 1) {
                const int r = rank_at(a, vb + w * 32 + __ffs(g) - 1);
                fb0_clear(a, r);
            }
            for (uint32_t c = cand; c; c &= c - 1) {
                const int r = rank_at(a, vb + w * 32 + __ffs(c) - 1);
                fb0_set(a, r);
                flag_rank(s1, s2, s3, (int *)&B.cur1, r);
            }
        }
        return true;
    });
}

// Single-voxel regime.  Once the best candidate has dt2 == 1 every candidate
// does, each ball is its own centre, and those centres are queued already:
// stamping a batch changes no other voxel's candidate status, so each item
// can look at its six neighbours once, before the commit, both to bound J and
// to know what it will queue.  Runs on warps 0-1 (64 threads, named barrier
// 1) until the best candidate is no longer single-voxel, the front is empty
// or the step limit is reached.
constexpr int kNewCap = 6 * kM;   // candidates one single-voxel batch can queue
constexpr int kTinyM = kM;       // batch size of the single-voxel loop
constexpr int kMinMerge = 16;     // smaller merged batches are refilled from the bitmap

template <bool L1SMEM, bool PROF>
__device__ void tiny_loop(const Inv &a, Batch &B, u64 *s1, u64 *s2, u64 *s3, const int tid, int64_t &k,
                          const FastDiv &fd_nyz, const FastDiv &fd_nz, long long *sD, int *sNr, int *sNv, int *tR,
                          int *tI)
{
    const int lane = tid & 31;
    const int first1 = (int)a.out[kFirst1Slot];   // ranks below it hold dt2 > 1
    int tpoll = 0;   // batches since the last cancel poll (thread 0)
    if (tid == 0) { B.tmerge = 0; B.nN = 0; B.novf = 0; }
    bar_sync_64();
    for (;;) {
        const long long ta = tclk<PROF>();
        // Next batch.  A committed single-voxel ball stamps only its own
        // centre, so the frontier changed only by the committed items and
        // the candidates that commit queued (ranks known): every candidate
        // ranked at or below Rk is an uncommitted item or such a new one.
        // Their sorted merge is an exact prefix of the frontier; it is used
        // when it is large enough, else the batch is gathered afresh.
        bool gather = !B.tmerge;
        if (!gather) {
            const int m0 = B.m, J0 = B.J, Rk = B.Rk, nN = B.nN;
            if (tid == 0) { B.nT = m0 - J0; B.minN = INT_MAX; }
            bar_sync_64();
            int cnt = 0, mn = INT_MAX;
            for (int e = tid; e < nN; e += 64) {
                const int r = sNr[e];
                if (r <= Rk) { cnt++; mn = min(mn, r); }
            }
            cnt = __reduce_add_sync(0xffffffffu, cnt);
            mn = __reduce_min_sync(0xffffffffu, mn);
            if (lane == 0) { atomicAdd(&B.nT, cnt); atomicMin(&B.minN, mn); }
            bar_sync_64();
            const int T = B.nT;
            if (B.minN < first1) {   // a larger ball was exposed: back to the main loop
                if (tid == 0) B.stop = 0;
                break;
            }
            if (T >= kMinMerge) {
                // position of each element = ranks below it among both sets
                for (int e = tid; e < (m0 - J0) + nN; e += 64) {
                    int key, v;
                    if (e < m0 - J0) { key = B.rank[J0 + e]; v = B.idx[J0 + e]; }
                    else {
                        key = sNr[e - (m0 - J0)]; v = sNv[e - (m0 - J0)];
                        if (key > Rk) continue;
                    }
                    int lo = J0, hi = m0;   // remaining items ranked below key
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (B.rank[mid] < key) lo = mid + 1; else hi = mid;
                    }
                    int pos = lo - J0;
                    for (int f = 0; f < nN; f++) {
                        const int r = sNr[f];
                        pos += (r <= Rk && r < key);
                    }
                    if (pos < kM) { tR[pos] = key; tI[pos] = v; }
                }
                bar_sync_64();
                const int m = min(T, kTinyM);
                if (tid < m) {
                    const uint32_t v = (uint32_t)tI[tid];
                    const uint32_t x = fdiv(v, fd_nyz), rem = v - x * (uint32_t)a.ny * (uint32_t)a.nz;
                    const uint32_t y = fdiv(rem, fd_nz);
                    B.rank[tid] = tR[tid];
                    B.idx[tid] = (int)v;
                    B.r2[tid] = 1;
                    B.x[tid] = (int)x; B.y[tid] = (int)y; B.z[tid] = (int)(rem - y * (uint32_t)a.nz);
                }
                if (tid == 0) {
                    if (T > kTinyM) B.Rk = tR[kTinyM - 1];   // the truncated tail is still in the bitmap
                    int stop = 0, mcap = m;
                    const int64_t remain = a.max_steps - k;
                    if (remain < (int64_t)m) mcap = (int)max(remain, (int64_t)0);
                    if (mcap == 0) stop = 2;
                    if (k > a.npore) stop = 3;
                    B.tstop = stop; B.m = m; B.mcap = mcap; B.J = mcap;
                }
            } else {
                gather = true;
            }
        }
        if (gather && tid < 32) {
            const int m = gather_items<L1SMEM, false>(a, B, s1, s2, s3, lane, kTinyM, fd_nyz, fd_nz, sD + D_STALE);
            if (lane == 0) {
                int stop = 0, mcap = m;
                const int64_t remain = a.max_steps - k;
                if (m == 0) stop = 1;
                else if (B.r2[0] != 1) stop = 4;
                else {
                    if (remain < (int64_t)m) mcap = (int)max(remain, (int64_t)0);
                    if (mcap == 0) stop = 2;
                }
                if (k > a.npore) stop = 3;
                B.tstop = stop; B.m = m; B.mcap = mcap; B.J = mcap;
                B.Rk = m > 0 ? B.rank[m - 1] : INT_MAX;
            }
        }
        if (tid == 0) {
            B.nN = 0;
            B.novf = 0;
            // every 64th batch: the host's cancel flag (stop before committing)
            if (a.cancel && (tpoll++ & 63) == 0 && B.tstop == 0 && *(const volatile int *)a.cancel) B.tstop = 5;
        }
        bar_sync_64();
        const long long tb = tclk<PROF>();
        if (tid == 0 && !gather) {
            sD[D_TMERGE]++;
            if (PROF) sD[D_TMERGE_CYC] += tb - ta;
        }
        if (PROF && tid == 0) sD[D_TG] += tb - ta;
        const int st = B.tstop;
        if (st) {
            if (st != 4 && tid == 0) B.stop = st;
            break;
        }
        const int m = B.m, mcap = B.mcap, j = tid;
        Nb6 nb;
        unsigned cand = 0;
        int rr[6];
        int jl = INT_MAX;
        if (j < mcap) {
            nb6(a, B.x[j], B.y[j], B.z[j], B.idx[j], nb);
            cand = nb6_candidates(a, nb);
            int best = INT_MAX;
#pragma unroll
            for (int q = 0; q < 6; q++) {
                rr[q] = ((cand >> q) & 1) ? rank_at(a, nb.v[q]) : INT_MAX;
                best = min(best, rr[q]);
            }
            if (cand) jl = max(j + 1, lower_rank(B, m, best));
        }
        jl = __reduce_min_sync(0xffffffffu, jl);
        if (lane == 0 && jl < INT_MAX) atomicMin(&B.J, jl);
        bar_sync_64();
        const long long tc = tclk<PROF>();
        if (PROF && tid == 0) sD[D_TB] += tc - tb;
        const int J = B.J;
        if (j < J) {
            const int x = B.x[j], y = B.y[j], z = B.z[j];
            plane_and(a, a.avail, ((int64_t)x * a.ny + y) * a.NW + (z >> 5), ~(1u << (z & 31)));
            seq_put(a, B.idx[j], (int32_t)(k + 1 + j));
            const int r = B.rank[j];
            fb0_clear(a, r);
            if (k + j < a.cap) {
                a.step_r2[k + j] = 1;
                if (a.step_centre) a.step_centre[k + j] = B.idx[j];
            }
            uint32_t got[6];
#pragma unroll
            for (int q = 0; q < 6; q++)
                got[q] = ((cand >> q) & 1) ? plane_or(a, a.added, nb.word[q], nb.bit[q]) : nb.bit[q];
            unsigned fr = 0;
#pragma unroll
            for (int q = 0; q < 6; q++)
                if (!(got[q] & nb.bit[q])) fr |= 1u << q;
            if (fr) {
                int slot = atomicAdd(&B.nN, __popc(fr));
#pragma unroll
                for (int q = 0; q < 6; q++) {
                    if (!((fr >> q) & 1)) continue;
                    const int rq = rr[q];
                    fb0_set(a, rq);
                    flag_rank(s1, s2, s3, &B.cur1, rq);
                    if (slot < kNewCap) { sNr[slot] = rq; sNv[slot] = nb.v[q]; }
                    else B.novf = 1;
                    slot++;
                }
            }
        }
        k += J;
        if (tid == 0) { sD[D_TINY_IT]++; sD[D_TINY_STEPS] += J; }
        bar_sync_64();
        if (tid == 0) {
            B.tmerge = !B.novf;
            if (PROF) {
                const long long te = tclk<PROF>();
                sD[D_TC] += te - tc;
                trace_batch(a, sD[D_TRACE], k - J, J, te - ta, 1, m, J, 0, 0);
            }
        }
        bar_sync_64();
    }
}

template <bool L1SMEM, bool PROF>
__device__ __forceinline__ void invade_body(const Inv &a, const FastDiv &fd_nyz, const FastDiv &fd_nz, int *gC,
                                            int *gD)
{
    extern __shared__ u64 s_fb[];
    __shared__ Batch B;
    __shared__ int sLA[kList];
    __shared__ unsigned char sLAi[kList];
    __shared__ int sLAr[kList];
    __shared__ int sLC[kList];
    __shared__ int sLD[kList];
    __shared__ int sNr[kNewCap], sNv[kNewCap], tR[kM], tI[kM];
    u64 *s1 = L1SMEM ? s_fb : a.fb1;
    u64 *s2 = s_fb + (L1SMEM ? a.NL1 : 0);
    u64 *s3 = s2 + a.NL2;
    const int tid = threadIdx.x, lane = tid & 31;
    if (L1SMEM)
        for (int i = tid; i < a.NL1; i += kNT) s1[i] = a.fb1[i];
    for (int i = tid; i < a.NL2; i += kNT) s2[i] = a.fb2[i];
    for (int i = tid; i < a.NL3; i += kNT) s3[i] = a.fb3[i];
    int *isq_t = (int *)(s3 + a.NL3);
    for (int e = tid; e < a.isq_n; e += kNT) isq_t[e] = d_isqrt(e);
    if (tid == 0) {
        a.out[kErrSlot] = 0;
        B.mtarget = kM;
        B.cur1 = 0;
        B.upre[0] = 0;
        B.dpre[0] = 0;
        B.isq.t = isq_t;
        B.isq.n = a.isq_n;
    }
    __syncthreads();

    const long long span_c0 = clock64();
    const unsigned long long span_t0 = global_ns();
    int64_t k = a.k0;
    // diagnostics (thread 0): cycles per phase, items, stale summary bits, ...
    __shared__ long long sD[kNOut];
    int poll = 0;   // batches since the last cancel poll (lane 0 of warp 0)
    if (tid == 0)
        for (int q = 0; q < kNOut; q++) sD[q] = 0;
    for (;;) {
        long long t0 = tclk<PROF>();
        // ------------------------------------------------------ select batch
        // The best candidates are the first set bits of the rank bitmap.  Lane
        // 0 walks the summary levels to the first flagged level-1 word; the
        // warp then loads the level-0 words of up to 32 flagged entries of
        // that and the next three level-1 words, drops (and unflags) empty
        // ones, and takes the leading set bits as the batch.
        // S1 (warp 0): the batch items and their data.
        if (tid < 32) {
            // every 16th batch, lane 0 reads the host's cancel flag (issued
            // before the gather, used after it)
            int cz = 0;
            if (lane == 0 && a.cancel && (poll++ & 15) == 0) cz = *(const volatile int *)a.cancel;
            const int m = gather_items<L1SMEM, true>(a, B, s1, s2, s3, lane, B.mtarget, fd_nyz, fd_nz, sD + D_STALE);
            const bool bg0 = lane < m && B.r2[lane] > 1, bg1 = lane + 32 < m && B.r2[lane + 32] > 1;
            const unsigned b0 = __ballot_sync(0xffffffffu, bg0), b1 = __ballot_sync(0xffffffffu, bg1);
            const u64 big = (u64)b0 | ((u64)b1 << 32);
            const unsigned below = (1u << lane) - 1;
            if (bg0) B.bigl[__popc(b0 & below)] = lane;
            if (bg1) B.bigl[__popc(b0) + __popc(b1 & below)] = lane + 32;
            if (lane == 0) {
                B.m = m;
                B.big = big;
                B.stop = m == 0 ? 1 : (cz ? 5 : 0);   // 5: cancelled, before this batch commits
                if (PROF) sD[D_GATHER] += tclk<PROF>() - t0;
            }
        }
        __syncthreads();
        if (B.stop) break;
        if (B.r2[0] == 1) {
            long long tt = tclk<PROF>();
            if (tid < 64) tiny_loop<L1SMEM, PROF>(a, B, s1, s2, s3, tid, k, fd_nyz, fd_nz, sD, sNr, sNv, tR, tI);
            if (tid == 0) B.kk = k;
            __syncthreads();
            k = B.kk;
            if (PROF && tid == 0) sD[D_TINY_CYC] += tclk<PROF>() - tt;
            if (B.stop) break;
            continue;
        }
        if (B.m == 1) {
            // A lone item is committed whatever its shell holds (the cut is
            // never below one), so one pass over the rows of its dilated
            // square stamps its ball and queues its shell: no pairwise
            // tests, no bound, no lists.
            const long long tf = tclk<PROF>();
            if (a.max_steps - k < 1 || k > a.npore) {   // the same for every thread
                if (tid == 0) B.stop = a.max_steps - k < 1 ? 2 : 3;
                break;
            }
            commit_single(a, B, s1, s2, s3, tid, (int32_t)(k + 1));
            if (tid == 0) {
                if (k < a.cap) {
                    a.step_r2[k] = B.r2[0];
                    if (a.step_centre) a.step_centre[k] = B.idx[0];
                }
                B.mtarget = 16;
            }
            const int rows1 = B.upre[1], shell1 = B.dpre[1];
            __syncthreads();
            k += 1;
            if (tid == 0) {
                sD[D_ITERS]++;
                sD[D_ITEMS] += 1;
                sD[D_COMMITTED] += 1;
                sD[D_ROWS] += rows1;
                sD[D_SHELL_UNITS] += shell1;
                sD[D_SINGLE]++;
                if (PROF) {
                    const long long te = tclk<PROF>();
                    sD[D_SEL] += tf - t0;
                    sD[D_COMMIT] += te - tf;
                    trace_batch(a, sD[D_TRACE], k - 1, 1, te - t0, 0, 1, rows1, shell1, 0);
                }
            }
            continue;
        }
        // S2 (all threads): pairwise tests between every item j and every item
        // b whose ball is more than its centre voxel (two distinct
        // single-voxel balls never meet).  cont: j lies in the ball of an
        // earlier b; ovl: the ball boxes of j and b, grown by one voxel, meet.
        {
            const long long tb = tclk<PROF>();
            const int m = B.m;
            const u64 big = B.big;
            // pair p: big item bigl[p >> sh] against item p & (2^sh - 1)
            const int sh = m <= 32 ? 5 : 6;
            const int npair = __popcll(big) << sh;
            for (int p = tid; p < npair; p += kNT) {
                const int j = p & ((1 << sh) - 1);
                if (j >= m) continue;
                const int b = B.bigl[p >> sh];
                if (j == b) continue;
                const int dx = B.x[j] - B.x[b], dy = B.y[j] - B.y[b], dz = B.z[j] - B.z[b];
                if (b < j && dx * dx + dy * dy + dz * dz < B.r2[b])
                    atomicOr(&B.cont32[j][b >> 5], 1u << (b & 31));
                const int lim = B.h[b] + B.h[j] + 1;
                if (abs(dx) <= lim && abs(dy) <= lim && abs(dz) <= lim) {
                    atomicOr(&B.ovl32[j][b >> 5], 1u << (b & 31));
                    atomicOr(&B.ovl32[b][j >> 5], 1u << (j & 31));
                }
            }
            __syncthreads();
            if (PROF && tid == 0) sD[D_PAIRS] += tclk<PROF>() - tb;
        }
        // S3 (warp 0): skip covered items, apply the step limit and the row
        // budget, number the steps, prefix-sum the row units.  Up to 32
        // items: one per lane, 32-bit masks.
        if (tid < 32 && B.m <= 32) {
            const long long tc = tclk<PROF>();
            const int m = B.m;
            const bool act = lane < m;
            // containers are earlier items, so all below 32
            const uint32_t cont = act ? B.cont32[lane][0] : 0u;
            if (act) B.ovl[lane] = (u64)B.ovl32[lane][0];
            const uint32_t valid = m == 32 ? 0xffffffffu : ((1u << m) - 1);
            const uint32_t has = __ballot_sync(0xffffffffu, cont != 0u);
            uint32_t keep = valid & ~has, decided = ~(has & valid);
            // an item is kept iff no kept earlier item's ball contains it
            while (~decided) {
                const bool rd = !((decided >> lane) & 1) && (cont & ~decided) == 0u;
                const bool kp = rd && (cont & keep) == 0u;
                decided |= __ballot_sync(0xffffffffu, rd);
                keep |= __ballot_sync(0xffffffffu, kp);
            }
            int mcap = m;
            const int64_t remain = a.max_steps - k;
            if ((int64_t)__popc(keep) > remain) {
                uint32_t t = keep;
                for (int64_t q = 0; q < remain; q++) t &= t - 1;
                mcap = __ffs(t) - 1;
            }
            const bool kj = act && lane < mcap && ((keep >> lane) & 1);
            const int r = kj ? B.upre[lane + 1] : 0, d = kj ? B.dpre[lane + 1] : 0;
            int inc = r, dinc = d;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, inc, o);
                const int td = __shfl_up_sync(0xffffffffu, dinc, o);
                if (lane >= o) { inc = min(inc + t, 1 << 30); dinc = min(dinc + td, 1 << 30); }
            }
            // the batch stops before the shell-row budget is exceeded
            const unsigned ob = __ballot_sync(0xffffffffu, lane > 0 && dinc > kRowBudget);
            if (ob) mcap = min(mcap, __ffs(ob) - 1);
            const int src = max(mcap - 1, 0);
            int last = __shfl_sync(0xffffffffu, inc, src), dlast = __shfl_sync(0xffffffffu, dinc, src);
            if (mcap == 0) { last = 0; dlast = 0; }
            if (act) {
                B.step[lane] = ((keep >> lane) & 1) ? __popc(keep & ((1u << lane) - 1)) : -1;
                B.upre[lane + 1] = lane < mcap ? inc : last;
                B.dpre[lane + 1] = lane < mcap ? dinc : dlast;
            }
            __syncwarp();
            if (lane == 0) {
                B.upre[0] = 0;
                B.dpre[0] = 0;
                B.mcap = mcap;
                B.J = mcap;
                B.keep = keep;
                B.stop = mcap == 0 ? 2 : 0;
                B.nA = 0; B.nC = 0; B.nD = 0; B.ovf = 0;
                if (PROF) sD[D_TAIL] += tclk<PROF>() - tc;
            }
        } else if (tid < 32) {
            const long long tc = tclk<PROF>();
            const int m = B.m;
            u64 cont[2];
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const int j = lane + 32 * q;
                cont[q] = j < m ? ((u64)B.cont32[j][0] | ((u64)B.cont32[j][1] << 32)) : 0ull;
                if (j < m) B.ovl[j] = (u64)B.ovl32[j][0] | ((u64)B.ovl32[j][1] << 32);
            }
            u64 has = (u64)__ballot_sync(0xffffffffu, cont[0] != 0) |
                      ((u64)__ballot_sync(0xffffffffu, cont[1] != 0) << 32);
            u64 valid = m == 64 ? ~0ull : ((1ull << m) - 1);
            u64 keep = valid & ~has;
            // An item is kept iff no kept earlier item's ball contains it.
            // Containers come earlier, so rounds that settle every item whose
            // containers are all settled reach the sequential answer.
            u64 decided = ~(has & valid);
            while (~decided) {
                bool rd[2], kp[2];
#pragma unroll
                for (int q = 0; q < 2; q++) {
                    const int j = lane + 32 * q;
                    rd[q] = !((decided >> j) & 1) && (cont[q] & ~decided) == 0;
                    kp[q] = rd[q] && (cont[q] & keep) == 0;
                }
                decided |= (u64)__ballot_sync(0xffffffffu, rd[0]) | ((u64)__ballot_sync(0xffffffffu, rd[1]) << 32);
                keep |= (u64)__ballot_sync(0xffffffffu, kp[0]) | ((u64)__ballot_sync(0xffffffffu, kp[1]) << 32);
            }
            const long long tc2 = tclk<PROF>();
            if (PROF && tid == 0) sD[D_S3_CONT] += tc2 - tc;
            // step limit: items past the (max_steps - k)-th kept one are dropped
            int mcap = m;
            int64_t remain = a.max_steps - k;
            if ((int64_t)__popcll(keep) > remain) {
                u64 t = keep;
                for (int64_t q = 0; q < remain; q++) t &= t - 1;
                mcap = __ffsll(t) - 1;
            }
            // row units of kept items below mcap, prefix-summed (two items per
            // lane): ball rows (stamping) and shell rows (candidates); the
            // batch stops before the shell-row budget is exceeded
            int j0 = 2 * lane, j1 = 2 * lane + 1;
            const bool k0 = j0 < mcap && ((keep >> j0) & 1), k1 = j1 < mcap && ((keep >> j1) & 1);
            int r0 = k0 ? B.upre[j0 + 1] : 0, r1 = k1 ? B.upre[j1 + 1] : 0;
            int d0 = k0 ? B.dpre[j0 + 1] : 0, d1 = k1 ? B.dpre[j1 + 1] : 0;
            int inc = r0 + r1, dinc = d0 + d1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, inc, o);
                int td = __shfl_up_sync(0xffffffffu, dinc, o);
                if (lane >= o) { inc = min(inc + t, 1 << 30); dinc = min(dinc + td, 1 << 30); }
            }
            int ex = inc - r0 - r1, dex = dinc - d0 - d1;
            const bool over0 = j0 > 0 && dex + d0 > kRowBudget;
            const bool over1 = dex + d0 + d1 > kRowBudget;
            unsigned ob0 = __ballot_sync(0xffffffffu, over0), ob1 = __ballot_sync(0xffffffffu, over1);
            int cut = 64;
            if (ob0 | ob1) {
                int l = __ffs(ob0 | ob1) - 1;
                cut = ((ob0 >> l) & 1) ? 2 * l : 2 * l + 1;
            }
            mcap = min(mcap, cut);
            if (PROF && tid == 0) sD[D_S3_PREFIX] += tclk<PROF>() - tc2;
            // prefix through item mcap - 1, carried by every later item
            const bool odd = (mcap - 1) & 1;
            int last = __shfl_sync(0xffffffffu, odd ? inc : ex + r0, max(mcap - 1, 0) >> 1);
            int dlast = __shfl_sync(0xffffffffu, odd ? dinc : dex + d0, max(mcap - 1, 0) >> 1);
            if (mcap == 0) { last = 0; dlast = 0; }
            __syncwarp();
            if (j0 < m) {
                B.step[j0] = ((keep >> j0) & 1) ? __popcll(keep & ((1ull << j0) - 1)) : -1;
                B.upre[j0 + 1] = j0 < mcap ? ex + r0 : last;
                B.dpre[j0 + 1] = j0 < mcap ? dex + d0 : dlast;
            }
            if (j1 < m) {
                B.step[j1] = ((keep >> j1) & 1) ? __popcll(keep & ((1ull << j1) - 1)) : -1;
                B.upre[j1 + 1] = j1 < mcap ? ex + r0 + r1 : last;
                B.dpre[j1 + 1] = j1 < mcap ? dex + d0 + d1 : dlast;
            }
            __syncwarp();
            if (lane == 0) {
                B.upre[0] = 0;
                B.dpre[0] = 0;
                B.mcap = mcap;
                B.J = mcap;
                B.keep = keep;
                B.stop = mcap == 0 ? 2 : 0;
                B.nA = 0; B.nC = 0; B.nD = 0; B.ovf = 0;
                if (PROF) sD[D_TAIL] += tclk<PROF>() - tc;
            }
        }
        __syncthreads();
        long long t1 = tclk<PROF>();
        if (PROF && tid == 0) sD[D_SEL] += t1 - t0;
        if (B.stop) break;
        if (k > a.npore) {   // every step invades its own centre: cannot happen
            if (tid == 0) B.stop = 3;
            break;
        }
        const int mcap = B.mcap, m = B.m;

        // ---------------------------------------- candidate bound (shell)
        // Stage 1 lists the never-queued, uninvaded neighbours u of each kept
        // ball; stage 2 looks up their ranks in parallel and lowers J to
        // max(i + 1, #items ranked above u).
        {
            const int U = B.dpre[mcap];
            for_units(B.dpre, mcap, U, B.dx0, B.dy0, B.dwy, tid, [&](int u, int i, int x, int y) -> bool {
                // units are ordered by item; items at or past the current J will
                // not be committed (the list also feeds the commit, so every
                // item below J is enumerated in full)
                if (i >= *(volatile int *)&B.J) return false;
                if (B.r2[i] == 1) {
                    // single-voxel ball: its shell is its six neighbours
                    Nb6 nb;
                    nb6(a, B.x[i], B.y[i], B.z[i], B.idx[i], nb);
                    const unsigned c = nb6_candidates(a, nb);
                    if (!c) return true;
                    // static indices keep nb in registers
                    int slot = atomicAdd(&B.nA, __popc(c));
#pragma unroll
                    for (int q = 0; q < 6; q++) {
                        if (!((c >> q) & 1)) continue;
                        if (slot < kList) {
                            sLA[slot] = nb.v[q];
                            sLAi[slot] = (unsigned char)i;
                        } else {
                            B.ovf = 1;
                            const int ru = rank_at(a, nb.v[q]);
                            atomicMin(&B.J, max(i + 1, lower_rank(B, m, ru)));
                        }
                        slot++;
                    }
                    return true;
                }
                int za, zb, ra, rbz;
                if (!shell_row(a, B, i, x, y, za, zb, ra, rbz)) return true;
                const int64_t row = (int64_t)x * a.ny + y;
                for (int w = za >> 5; w <= (zb >> 5); w++) {
                    uint32_t cand = plane_ld(a, a.avail, row * a.NW + w) & ~plane_ld(a, a.added, row * a.NW + w) &
                                    span_mask(w, za, zb) & ~span_mask(w, ra, rbz);
                    if (!cand) continue;
                    for (int slot = atomicAdd(&B.nA, __popc(cand)); cand; cand &= cand - 1, slot++) {
                        const int z = w * 32 + __ffs(cand) - 1;
                        if (slot < kList) {
                            sLA[slot] = (int)(row * a.nz + z);
                            sLAi[slot] = (unsigned char)i;
                        } else {
                            B.ovf = 1;
                            const int ru = rank_at(a, row * a.nz + z);
                            atomicMin(&B.J, max(i + 1, lower_rank(B, m, ru)));
                        }
                    }
                }
                return true;
            });
            __syncthreads();
            if (PROF && tid == 0) sD[D_B1] += tclk<PROF>() - t1;
            // entries of items at or past J are never committed; the ranks
            // of up to four entries per thread are loaded together, and each
            // warp lowers J once
            const int n = min(B.nA, kList);
            int jl = *(volatile int *)&B.J;
            for (int e0 = tid; e0 < n; e0 += 4 * kNT) {
                int ru[4], it[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int e = e0 + q * kNT;
                    it[q] = e < n ? sLAi[e] : kM;
                    ru[q] = it[q] < jl ? rank_at(a, sLA[e]) : 0;
                }
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    if (it[q] >= jl) continue;
                    sLAr[e0 + q * kNT] = ru[q];
                    if (it[q] + 1 < jl) jl = min(jl, max(it[q] + 1, lower_rank(B, m, ru[q])));
                }
            }
            jl = __reduce_min_sync(0xffffffffu, jl);
            if (lane == 0) atomicMin(&B.J, jl);
        }
        __syncthreads();
        long long t2 = tclk<PROF>();
        if (PROF && tid == 0) sD[D_BOUND] += t2 - t1;
        long long tm1 = t2;

        // --------------------------------------------------------- commit
        // Stage 1, per row of each committed ball: stamp the voxels this ball
        // owns (not covered by a lower committed ball), list the stamped ones
        // that were queued candidates (removals) and the neighbours outside
        // every committed ball that become candidates (additions; the atomic
        // on `added` makes each listed once).  Stage 2 applies both lists to
        // the rank bitmap in parallel.
        const int J = B.J;
        const u64 jmask = J >= 64 ? ~0ull : ((1ull << J) - 1);
        {
            const int64_t k1 = k + 1;
            const int U = B.upre[J];
            for_units(B.upre, J, U, B.bx0, B.by0, B.wy, tid, [&](int u, int i, int x, int y) -> bool {
                if (B.r2[i] == 1) {
                    // a kept single-voxel item is a queued candidate that no
                    // lower ball covers: it owns its voxel and its rank is known
                    const int z = B.z[i];
                    const int64_t w = ((int64_t)B.x[i] * a.ny + B.y[i]) * a.NW + (z >> 5);
                    plane_and(a, a.avail, w, ~(1u << (z & 31)));
                    seq_put(a, B.idx[i], (int32_t)(k1 + B.step[i]));
                    const int r = B.rank[i];
                    fb0_clear(a, r);
                    return true;
                }
                int lo, hi;
                if (!ball_run(B, i, x, y, lo, hi)) return true;
                const int z0 = max(lo, 0), z1 = min(hi, a.nz - 1);
                const int64_t rb = ((int64_t)x * a.ny + y) * a.NW;
                const int64_t vb = ((int64_t)x * a.ny + y) * a.nz;
                const int32_t label = (int32_t)(k1 + B.step[i]);
                const u64 lower = B.ovl[i] & B.keep & ((1ull << i) - 1);
                for (int w = z0 >> 5; w <= (z1 >> 5); w++) {
                    uint32_t own = span_mask(w, z0, z1);
                    for (u64 om = lower; om && own; om &= om - 1) {
                        int i2 = __ffsll(om) - 1, l2, h2;
                        if (ball_run(B, i2, x, y, l2, h2)) own &= ~span_mask(w, l2, h2);
                    }
                    if (!own) continue;
                    // `added` does not change during this stage: load it with `avail`
                    const uint32_t av = plane_ld(a, a.avail, rb + w), ad = plane_ld(a, a.added, rb + w);
                    const uint32_t newly = av & own;
                    if (!newly) continue;
                    plane_and(a, a.avail, rb + w, ~newly);
                    uint32_t gone = newly & ad;
                    for (uint32_t n2 = newly; n2; n2 &= n2 - 1) seq_put(a, vb + w * 32 + __ffs(n2) - 1, label);
                    if (!gone) continue;
                    for (int slot = atomicAdd(&B.nC, __popc(gone)); gone; gone &= gone - 1, slot++) {
                        const int v = (int)(vb + w * 32 + __ffs(gone) - 1);
                        if (slot < kList) sLC[slot] = v; else list_put(a, gC, slot - kList, v);
                    }
                }
                return true;
            });
            for (int j = tid; j < J; j += kNT) {
                if (B.step[j] < 0) continue;
                int64_t s = k + B.step[j];
                if (s < a.cap) {
                    a.step_r2[s] = B.r2[j];
                    if (a.step_centre) a.step_centre[s] = B.idx[j];
                }
            }
        }
        __syncthreads();
        tm1 = tclk<PROF>();
        if (PROF && tid == 0) sD[D_M1] += tm1 - t2;
        if (!B.ovf) {
            // Stage 2 from the candidate list of the bound pass (complete for
            // every committed item, ranks already loaded): a listed voxel
            // that is still uninvaded after the stamping lies outside every
            // committed ball; queue it once.  Apply the removals too.
            // Four entries per thread at a time, so that their loads and
            // returning atomics overlap.  Removed and added voxels differ
            // (one is stamped, the other not), so the order does not matter.
            const int n = min(B.nA, kList), tot = n + B.nC;
            for (int e0 = tid; e0 < tot; e0 += 4 * kNT) {
                int64_t wd[4];
                uint32_t bt[4], got[4];
                int rr[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int e = e0 + q * kNT;
                    wd[q] = -1; bt[q] = 0; got[q] = 0; rr[q] = -1;
                    if (e < n) {
                        if (sLAi[e] < J) {
                            const uint32_t v = (uint32_t)sLA[e];
                            const uint32_t row = fdiv(v, fd_nz), z = v - row * (uint32_t)a.nz;
                            wd[q] = (int64_t)row * a.NW + (z >> 5);
                            bt[q] = 1u << (z & 31);
                            rr[q] = sLAr[e];
                            got[q] = plane_ld(a, a.avail, wd[q]);
                        }
                    } else if (e < tot) {
                        const int f = e - n;
                        rr[q] = rank_at(a, (f < kList ? sLC[f] : gC[f - kList]));
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    if (wd[q] >= 0) {
                        // still uninvaded after the stamping: queue it once
                        got[q] = (got[q] & bt[q]) && !(plane_or(a, a.added, wd[q], bt[q]) & bt[q]);
                    } else if (rr[q] >= 0) {
                        fb0_clear(a, rr[q]);
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    if (wd[q] < 0 || !got[q]) continue;
                    const int r = rr[q];
                    fb0_set(a, r);
                    flag_rank(s1, s2, s3, &B.cur1, r);
                }
            }
        } else {
        // Stage 2: with every committed ball stamped, a shell voxel that is
        // still uninvaded and never queued lies outside all of them: queue it.
        {
            const int U = B.dpre[J];
            for_units(B.dpre, J, U, B.dx0, B.dy0, B.dwy, tid, [&](int u, int i, int x, int y) -> bool {
                if (B.r2[i] == 1) {
                    Nb6 nb;
                    nb6(a, B.x[i], B.y[i], B.z[i], B.idx[i], nb);
                    unsigned c = nb6_candidates(a, nb);
                    unsigned fr = 0;
#pragma unroll
                    for (int q = 0; q < 6; q++)
                        if ((c >> q) & 1)
                            if (!(plane_or(a, a.added, nb.word[q], nb.bit[q]) & nb.bit[q])) fr |= 1u << q;
                    int rr[6];
#pragma unroll
                    for (int q = 0; q < 6; q++) rr[q] = ((fr >> q) & 1) ? rank_at(a, nb.v[q]) : -1;
#pragma unroll
                    for (int q = 0; q < 6; q++) {
                        const int r = rr[q];
                        if (r < 0) continue;
                        fb0_set(a, r);
                        flag_rank(s1, s2, s3, &B.cur1, r);
                    }
                    return true;
                }
                int za, zb, ra, rbz;
                if (!shell_row(a, B, i, x, y, za, zb, ra, rbz)) return true;
                const int64_t row = (int64_t)x * a.ny + y;
                for (int w = za >> 5; w <= (zb >> 5); w++) {
                    const uint32_t cand = plane_ld(a, a.avail, row * a.NW + w) & ~plane_ld(a, a.added, row * a.NW + w) &
                                          span_mask(w, za, zb) & ~span_mask(w, ra, rbz);
                    if (!cand) continue;
                    uint32_t fresh = cand & ~plane_or(a, a.added, row * a.NW + w, cand);
                    for (; fresh; fresh &= fresh - 1) {
                        const int v = (int)(row * a.nz + w * 32 + __ffs(fresh) - 1);
                        const int slot = atomicAdd(&B.nD, 1);
                        if (slot < kList) sLD[slot] = v; else list_put(a, gD, slot - kList, v);
                    }
                }
                return true;
            });
        }
        __syncthreads();
        // Stage 3: apply removals and additions to the rank bitmap.
        {
            const int nC = B.nC, nD = B.nD;
            for (int e = tid; e < nC + nD; e += kNT) {
                if (e < nC) {
                    int v = e < kList ? sLC[e] : gC[e - kList];
                    int r = rank_at(a, v);
                    fb0_clear(a, r);
                } else {
                    int f = e - nC;
                    int v = f < kList ? sLD[f] : gD[f - kList];
                    int r = rank_at(a, v);
                    fb0_set(a, r);
                    flag_rank(s1, s2, s3, &B.cur1, r);
                }
            }
        }
        }
        const int nk = __popcll(B.keep & jmask);
        k += nk;
        int tr_rows = 0, tr_shell = 0, tr_listed = 0, tr_removed = 0;
        bool small = false;
        if (tid == 0) {
            tr_rows = B.upre[J]; tr_shell = B.dpre[mcap]; tr_listed = B.nA; tr_removed = B.nC;
            small = tr_rows == nk && B.r2[0] == 1;
            B.mtarget = min(kM, max(16, 2 * J + 8));
        }
        __syncthreads();
        const long long t3 = tclk<PROF>();
        if (tid == 0) {
            sD[D_ITERS]++;
            sD[D_ITEMS] += m;
            sD[D_COMMITTED] += J;
            sD[D_ROWS] += tr_rows;
            sD[D_SHELL_UNITS] += tr_shell;
            sD[D_LISTED] += tr_listed;
            sD[D_REMOVED] += tr_removed;
            if (PROF) {
                sD[D_COMMIT] += t3 - t2;
                sD[D_M2] += t3 - tm1;
                trace_batch(a, sD[D_TRACE], k - nk, nk, t3 - t0, 0, m, tr_rows, tr_shell, tr_listed);
            }
            if (small) {
                sD[D_SMALL_CYC] += t3 - t0;
                sD[D_SMALL_N]++;
                sD[D_SMALL_SEL] += t1 - t0;
                sD[D_SMALL_BOUND] += t2 - t1;
                sD[D_SMALL_COMMIT] += t3 - t2;
            }
        }
    }
    if (tid == 0) {
        sD[D_SPAN_CYC] = clock64() - span_c0;
        sD[D_SPAN_NS] = (long long)(global_ns() - span_t0);
        sD[D_B2] = sD[D_BOUND] - sD[D_B1];
        for (int q = 2; q < kNOut; q++)
            if (q != kFirst1Slot && q != kErrSlot) a.out[q] = sD[q];
        a.out[0] = k;
        a.out[1] = B.stop == 2 ? IBIP_ERR_STEP_LIMIT
                   : B.stop == 3 ? IBIP_ERR_BOUNDS
                   : B.stop == 5 ? IBIP_ERR_CANCELLED : IBIP_OK;
        if (*(volatile int64_t *)(a.out + kErrSlot)) a.out[1] = IBIP_ERR_BOUNDS;   // checked build only
    }
}

template <bool L1SMEM, bool PROF>
__global__ void __launch_bounds__(kNT, 1) k_invade(Inv a, FastDiv fd_nyz, FastDiv fd_nz, int *gC, int *gD)
{
    invade_body<L1SMEM, PROF>(a, fd_nyz, fd_nz, gC, gD);
}

// One image per CTA: many invasions in one launch (all with level 1 of the
// rank bitmap in shared memory).
struct InvJob {
    Inv a;
    FastDiv fd_nyz, fd_nz;
    int *gC, *gD;
    int blk_plane;   // first block of this image in the batched plane set-up
    int flag;        // this image's completion record
};

// bit-planes and first candidates of every image: one thread per word
__global__ void k_plane_init_b(const InvJob *__restrict__ jobs, int n)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (jobs[mid].blk_plane <= (int)blockIdx.x) lo = mid; else hi = mid;
    }
    const Inv &a = jobs[lo].a;
    const int64_t w = (int64_t)(blockIdx.x - jobs[lo].blk_plane) * blockDim.x + threadIdx.x;
    if (w < (int64_t)a.nx * a.ny * a.NW) plane_word(a, w);
}

// rec (host-mapped, when given): image i's steps and status, then its done
// flag, once its results are visible to later kernels on the device.
__global__ void __launch_bounds__(kNT, 1) k_invade_batch(const InvJob *__restrict__ jobs, IbipBatchDone *rec)
{
    const InvJob j = jobs[blockIdx.x];
    invade_body<true, false>(j.a, j.fd_nyz, j.fd_nz, j.gC, j.gD);
    if (!rec) return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile IbipBatchDone *r = rec + j.flag;
        r->steps = j.a.out[0];
        r->status = (int32_t)j.a.out[1];
        __threadfence_system();
        r->done = 1;
    }
}

}  // namespace

// --------------------------------------------------------------- launcher --

namespace {

// Device memory one invasion needs beyond its inputs and outputs.
struct JobMem {
    int32_t *rank;
    int2 *okey;
    uint32_t *avail, *added;
    u64 *fb;
    int *gl;
    int64_t *out;
};

struct JobSizes {
    size_t rank, okey, plane, fb, gl, out;
    size_t total() const { return rank + okey + 2 * plane + fb + gl + out; }
};

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

// Lets the kernel take all the dynamic shared memory the device allows.  The
// value is the same on every call, so threads driving different contexts can
// set it concurrently.
void allow_max_dyn_smem(const void *func)
{
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, func) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

JobSizes job_sizes(ibip_dims d, int npore)
{
    JobSizes z;
    const int64_t N = nvox(d);
    const int NL0 = (npore + 63) / 64, NL1 = (NL0 + 63) / 64, NL2 = (NL1 + 63) / 64, NL3 = (NL2 + 63) / 64;
    z.rank = up256((size_t)N * sizeof(int32_t));
    z.okey = up256((size_t)npore * sizeof(int2));
    z.plane = up256((size_t)d.nx * d.ny * ((d.nz + 31) / 32) * sizeof(uint32_t));
    z.fb = up256(((size_t)NL0 + NL1 + NL2 + NL3) * sizeof(u64));
    z.gl = up256((size_t)2 * npore * sizeof(int) + 64);
    z.out = up256(kNOut * sizeof(int64_t));
    return z;
}

JobMem carve(char *p, const JobSizes &z)
{
    JobMem m;
    m.rank = (int32_t *)p; p += z.rank;
    m.okey = (int2 *)p; p += z.okey;
    m.avail = (uint32_t *)p; p += z.plane;
    m.added = (uint32_t *)p; p += z.plane;
    m.fb = (u64 *)p; p += z.fb;
    m.gl = (int *)p; p += z.gl;
    m.out = (int64_t *)p;
    return m;
}

// The invasion kernel's view of one image, its scratch carved as in `mem`.
Inv make_inv(const int32_t *dt2, ibip_dims d, int inlet, int64_t max_steps, int32_t *seq, int32_t *step_r2,
             int32_t *step_centre, int64_t cap, int maxd, int npore, const JobMem &mem, const uint8_t *mask,
             int resume, int64_t k0)
{
    Inv a;
    a.nx = d.nx; a.ny = d.ny; a.nz = d.nz; a.NW = (d.nz + 31) / 32; a.inlet = inlet;
    a.NL0 = (npore + 63) / 64;
    a.NL1 = (a.NL0 + 63) / 64;
    a.NL2 = (a.NL1 + 63) / 64;
    a.NL3 = (a.NL2 + 63) / 64;
    a.max_steps = max_steps > INT64_MAX - k0 ? INT64_MAX : k0 + max_steps;   // a total
    a.cap = cap;
    a.mask = mask;
    a.resume = resume;
    a.k0 = k0;
    a.npore = npore;
    a.rank = mem.rank; a.okey = mem.okey; a.dt2 = dt2;
    a.avail = mem.avail; a.added = mem.added;
    a.fb0 = mem.fb; a.fb1 = mem.fb + a.NL0; a.fb2 = a.fb1 + a.NL1; a.fb3 = a.fb2 + a.NL2;
    a.seq = seq; a.step_r2 = step_r2; a.step_centre = step_centre; a.out = mem.out;
    a.isq_n = std::min(maxd + 1, 16384);
    a.trace = nullptr;
    a.trace_cap = 0;
    a.cancel = nullptr;
    return a;
}

size_t fb_words(const Inv &a) { return (size_t)a.NL0 + a.NL1 + a.NL2 + a.NL3; }

// Rank sort, sequence initialisation and bit-plane / bitmap set-up of one
// invasion whose pore statistics (largest finite dt2, pore count, whether
// dt2 is infinite) are known.  Queued on the context stream; synchronises
// once (the number of distinct dt2 values sizes the counting sort).
int invade_setup(ibip_ctx *ctx, const int32_t *dt2, ibip_dims d, int inlet, int64_t max_steps, int32_t *seq,
                 int32_t *step_r2, int32_t *step_centre, int64_t cap, int maxd, int npore, int hasinf,
                 const JobMem &mem, Inv *out_a, const uint8_t *mask = nullptr, int resume = 0, int64_t k0 = 0)
{
    cudaStream_t s = ctx->stream;
    const int64_t N = nvox(d);
    const int gs = ctx->sm_count * 8;
    int *h = (int *)ctx->h_pinned;
    if (!resume) {
        k_seq_init<<<gs, 256, 0, s>>>(dt2, N, seq);
        IBIP_LAUNCH(ctx);
    }
    // -- bucket ids by dt2 value
    int32_t *incl = (int32_t *)ibip_scratch(ctx, SC_PRES, ((size_t)maxd + 2) * sizeof(int32_t));
    if (!incl) return IBIP_ERR_OOM;
    int B = 1;
    if (!hasinf) {
        cudaMemsetAsync(incl, 0, ((size_t)maxd + 1) * sizeof(int32_t), s);
        k_presence<<<gs, 256, 0, s>>>(dt2, N, incl);
        IBIP_LAUNCH(ctx);
        int st = ibip_scan_incl_i32(ctx, incl, incl, (int64_t)maxd + 1);
        if (st) return st;
        cudaMemcpyAsync(h, incl + maxd, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (ibip_sync(ctx, s) != cudaSuccess) return IBIP_ERR_CUDA;
        B = h[0];
    }
    Bucket bk{incl, B, hasinf};
    // -- stable counting sort by bucket
    // chunks of S voxels; the (bucket, chunk) count matrix is kept to at most
    // max(N/4, 2^20) entries (one byte per voxel) by widening the chunks
    int64_t S = kChunk;
    const int64_t mat_lim = std::max(N / 4, (int64_t)1 << 20);
    while (S < N && (N + S - 1) / S * (int64_t)B > mat_lim) S *= 2;
    const int C = (int)((N + S - 1) / S);
    int32_t *mat = (int32_t *)ibip_scratch(ctx, SC_MAT, (size_t)C * B * sizeof(int32_t));
    if (!mat) return IBIP_ERR_OOM;
    const bool smem = B <= 1024;
    const int wpb = 4;
    const size_t sm = smem ? (size_t)wpb * B * sizeof(int32_t) : 0;
    const int nb = (C + wpb - 1) / wpb;
    if (smem) k_chunk_hist<true><<<nb, wpb * 32, sm, s>>>(dt2, N, (int)S, C, bk, mat);
    else k_chunk_hist<false><<<nb, wpb * 32, 0, s>>>(dt2, N, (int)S, C, bk, mat);
    IBIP_LAUNCH(ctx);
    int st = ibip_scan_excl_i32(ctx, mat, mat, (int64_t)C * B);
    if (st) return st;
    // rank of the first voxel of the last bucket (the smallest value), read
    // before the scatter advances the counters
    k_last_bucket_rank<<<1, 32, 0, s>>>(mat + (int64_t)(B - 1) * C, 0, mem.out + kFirst1Slot);
    IBIP_LAUNCH(ctx);
    if (smem) k_chunk_scatter<true><<<nb, wpb * 32, sm, s>>>(dt2, N, (int)S, C, bk, mat, mem.rank, mem.okey);
    else k_chunk_scatter<false><<<nb, wpb * 32, 0, s>>>(dt2, N, (int)S, C, bk, mat, mem.rank, mem.okey);
    IBIP_LAUNCH(ctx);
    // -- bit-planes and the candidate bitmap
    Inv a = make_inv(dt2, d, inlet, max_steps, seq, step_r2, step_centre, cap, maxd, npore, mem, mask, resume, k0);
    cudaMemsetAsync(mem.fb, 0, fb_words(a) * sizeof(u64), s);
    k_plane_init<<<gs, 256, 0, s>>>(a);
    IBIP_LAUNCH(ctx);
    *out_a = a;
    return ibip_cuda_status(cudaGetLastError());
}

size_t invade_dyn_smem(const Inv &a, bool l1smem)
{
    return ((l1smem ? a.NL1 : 0) + (size_t)a.NL2 + a.NL3) * sizeof(u64) + (size_t)a.isq_n * sizeof(int);
}

// Level 1 of the rank bitmap goes to shared memory whenever it fits beside
// the kernel's static shared memory within the device's per-block opt-in
// limit (227 KB on this GPU: about 2.3 M summary bits, i.e. up to ~150 M
// pore voxels); beyond that it stays in global memory.
bool l1_fits_smem(const Inv &a)
{
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, (const void *)k_invade<true, false>) != cudaSuccess) {
        cudaGetLastError();
        return a.NL1 <= kSmemL1Max;
    }
    cudaFuncAttributes fp;
    if (cudaFuncGetAttributes(&fp, (const void *)k_invade<true, true>) != cudaSuccess) {
        cudaGetLastError();
        return a.NL1 <= kSmemL1Max;
    }
    const size_t stat = fa.sharedSizeBytes > fp.sharedSizeBytes ? fa.sharedSizeBytes : fp.sharedSizeBytes;
    return invade_dyn_smem(a, true) + stat <= (size_t)optin;
}

}  // namespace

int ibip_invade_run(ibip_ctx *ctx, const int32_t *dt2, ibip_dims d, int inlet, int64_t max_steps,
                    int32_t *seq, int32_t *step_r2, int32_t *step_centre, int64_t cap, int64_t *h_out,
                    const uint8_t *mask, int resume)
{
    cudaStream_t s = ctx->stream;
    const int64_t N = nvox(d);
    int k0 = 0;   // steps of the run being resumed: the largest seq value
    if (resume) {
        int st = ibip_max_launch(ctx, seq, N, &k0);
        if (st) return st;
    }
    int *stats = (int *)ibip_scratch(ctx, SC_SMALL, kSmallBytes);
    if (!stats) return IBIP_ERR_OOM;
    int *h = (int *)ctx->h_pinned;
    ibip_prof_begin(ctx, IBIP_K_RANK);
    cudaMemsetAsync(stats, 0, 3 * sizeof(int), s);
    k_stats<<<ctx->sm_count * 8, 256, 0, s>>>(dt2, N, stats);
    IBIP_LAUNCH(ctx);
    cudaMemcpyAsync(h, stats, 3 * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (ibip_sync(ctx, s) != cudaSuccess) return IBIP_ERR_CUDA;
    const int maxd = h[0], npore = h[1], hasinf = h[2];
    if (npore == 0) {
        if (!resume) {
            k_seq_init<<<ctx->sm_count * 8, 256, 0, s>>>(dt2, N, seq);
            IBIP_LAUNCH(ctx);
        }
        ibip_prof_end(ctx, IBIP_K_RANK);
        for (int i = 0; i < kNOut; i++) h_out[i] = 0;
        h_out[0] = k0;
        h_out[1] = IBIP_OK;
        return ibip_cuda_status(ibip_sync(ctx, s));
    }
    const JobSizes z = job_sizes(d, npore);
    JobMem mem;
    mem.rank = (int32_t *)ibip_scratch(ctx, SC_RANK, z.rank);
    mem.okey = (int2 *)ibip_scratch(ctx, SC_OKEY, z.okey);
    mem.avail = (uint32_t *)ibip_scratch(ctx, SC_AVAIL, z.plane);
    mem.added = (uint32_t *)ibip_scratch(ctx, SC_ADDED, z.plane);
    mem.fb = (u64 *)ibip_scratch(ctx, SC_FB, z.fb);
    mem.gl = (int *)ibip_scratch(ctx, SC_LIST, z.gl);
    int64_t *small = (int64_t *)ibip_scratch(ctx, SC_SMALL, kSmallBytes);
    if (!mem.rank || !mem.okey || !mem.avail || !mem.added || !mem.fb || !mem.gl || !small) return IBIP_ERR_OOM;
    mem.out = small + 8;
    Inv a;
    int st = invade_setup(ctx, dt2, d, inlet, max_steps, seq, step_r2, step_centre, cap, maxd, npore, hasinf, mem, &a,
                          mask, resume, k0);
    if (st) return st;
    a.trace = (int4 *)ctx->trace;
    a.trace_cap = ctx->trace ? ctx->trace_cap : 0;
    a.cancel = ctx->d_cancel;
    ibip_prof_end(ctx, IBIP_K_RANK);
    const FastDiv fd_nyz = make_fastdiv((uint32_t)d.ny * (uint32_t)d.nz), fd_nz = make_fastdiv((uint32_t)d.nz);
    const bool l1smem = l1_fits_smem(a);
    const bool prof = a.trace != nullptr;   // phase timers and the trace: a separate kernel
    const size_t dyn = invade_dyn_smem(a, l1smem);
    ibip_prof_begin(ctx, IBIP_K_INVADE);
    if (ctx->stream_inv) {
        // server slot: the kernel runs on the high-priority stream, after
        // everything queued so far on the slot's own stream
        if (cudaEventRecord(ctx->ev_inv, s) != cudaSuccess ||
            cudaStreamWaitEvent(ctx->stream_inv, ctx->ev_inv, 0) != cudaSuccess)
            return ibip_cuda_status(cudaGetLastError());
        s = ctx->stream_inv;
    }
    if (l1smem) {
        if (prof) {
            allow_max_dyn_smem((const void *)k_invade<true, true>);
            k_invade<true, true><<<1, kNT, dyn, s>>>(a, fd_nyz, fd_nz, mem.gl, mem.gl + npore);
        } else {
            allow_max_dyn_smem((const void *)k_invade<true, false>);
            k_invade<true, false><<<1, kNT, dyn, s>>>(a, fd_nyz, fd_nz, mem.gl, mem.gl + npore);
        }
    } else {
        if (prof) {
            allow_max_dyn_smem((const void *)k_invade<false, true>);
            k_invade<false, true><<<1, kNT, dyn, s>>>(a, fd_nyz, fd_nz, mem.gl, mem.gl + npore);
        } else {
            allow_max_dyn_smem((const void *)k_invade<false, false>);
            k_invade<false, false><<<1, kNT, dyn, s>>>(a, fd_nyz, fd_nz, mem.gl, mem.gl + npore);
        }
    }
    IBIP_LAUNCH(ctx);
    ibip_prof_end(ctx, IBIP_K_INVADE);
    int64_t *ho = (int64_t *)ctx->h_pinned;
    cudaMemcpyAsync(ho, mem.out, kNOut * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaError_t e = ibip_sync(ctx, s);
    if (e != cudaSuccess) return ibip_cuda_status(e);
    for (int i = 0; i < kNOut; i++) h_out[i] = ho[i];
    if (h_out[1] == IBIP_ERR_CANCELLED && ctx->h_cancel) *ctx->h_cancel = 0;   // the request is served
    return IBIP_OK;
}

int ibip_stats_launch(ibip_ctx *ctx, const int32_t *dt2, int64_t N, int *stats)
{
    k_stats<<<ctx->sm_count * 8, 256, 0, ctx->stream>>>(dt2, N, stats);
    IBIP_LAUNCH(ctx);
    return IBIP_OK;
}

// ------------------------------------------------------------- batched --

int ibip_invade_batch_run(ibip_ctx *ctx, int n, IbipBatchItem *it, IbipBatchEarly early, void *user)
{
    cudaStream_t s = ctx->stream;
    if (n <= 0) return IBIP_OK;
    if (n > kMaxBatch) return IBIP_ERR_ARG;
    int *h = (int *)ctx->h_pinned;
    // pore statistics of every image, one synchronisation
    // (one launch for all images: blocks find their image in a table)
    const size_t st_bytes = ((size_t)3 * n * sizeof(int) + 255) / 256 * 256;
    char *sbuf = (char *)ibip_scratch(ctx, SC_BSTAT, st_bytes + (size_t)n * sizeof(StatJob));
    if (!sbuf) return IBIP_ERR_OOM;
    int *st3 = (int *)sbuf;
    StatJob *dsj = (StatJob *)(sbuf + st_bytes);
    std::vector<StatJob> sjobs(n);
    int blk_st = 0;
    for (int j = 0; j < n; j++) {
        sjobs[j] = StatJob{it[j].dt2, nvox(it[j].d), blk_st};
        blk_st += (int)((nvox(it[j].d) + (int64_t)kVoxBlock * kVoxPer - 1) / ((int64_t)kVoxBlock * kVoxPer));
    }
    ibip_prof_begin(ctx, IBIP_K_RANK);
    cudaMemsetAsync(st3, 0, (size_t)3 * n * sizeof(int), s);
    cudaMemcpyAsync(dsj, sjobs.data(), (size_t)n * sizeof(StatJob), cudaMemcpyHostToDevice, s);
    k_stats_b<<<blk_st, kVoxBlock, 0, s>>>(dsj, n, st3);
    IBIP_LAUNCH(ctx);
    cudaMemcpyAsync(h, st3, (size_t)3 * n * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (ibip_sync(ctx, s) != cudaSuccess) return IBIP_ERR_CUDA;
    std::vector<int> maxd(n), npore(n), hasinf(n);
    size_t total = 0;
    std::vector<JobSizes> z(n);
    for (int j = 0; j < n; j++) {
        maxd[j] = h[3 * j]; npore[j] = h[3 * j + 1]; hasinf[j] = h[3 * j + 2];
        it[j].n_steps = 0;
        it[j].status = IBIP_OK;
        if (npore[j] == 0) continue;
        z[j] = job_sizes(it[j].d, npore[j]);
        if ((npore[j] + 63) / 64 > (int64_t)kSmemL1Max * 64) return IBIP_ERR_ARG;   // too large for one-CTA batching
        total += z[j].total();
    }
    char *arena = (char *)ibip_scratch(ctx, SC_BARENA, total + 256);
    if (!arena) return IBIP_ERR_OOM;
    std::vector<InvJob> jobs;
    std::vector<int> idx;
    std::vector<int64_t *> outs(n, nullptr);
    size_t off = 0, dyn = 0;
    // images with pore: one sort job each; the others only need seq
    std::vector<SortJob> sj;
    std::vector<JobMem> mems;
    int64_t pres_total = 0, pore_total = 0;
    int blk_vox = 0;
    for (int j = 0; j < n; j++) {
        if (npore[j] == 0) {
            k_seq_init<<<ctx->sm_count * 2, 256, 0, s>>>(it[j].dt2, nvox(it[j].d), it[j].seq);
            IBIP_LAUNCH(ctx);
            continue;
        }
        pore_total += npore[j];
        if (pore_total >= (1ll << 31)) return IBIP_ERR_ARG;   // the whole batch's ranks share one int32 scan
        const JobMem mem = carve(arena + off, z[j]);
        off += z[j].total();
        SortJob q = {};
        q.dt2 = it[j].dt2; q.N = nvox(it[j].d); q.seq = it[j].seq; q.rank = mem.rank; q.okey = mem.okey;
        q.out = mem.out;
        q.maxd = hasinf[j] ? 0 : maxd[j]; q.hasinf = hasinf[j];
        q.pres_off = pres_total;
        pres_total += (int64_t)q.maxd + 1;
        q.blk_vox = blk_vox;
        blk_vox += (int)((q.N + kVoxBlock * kVoxPer - 1) / (kVoxBlock * kVoxPer));
        sj.push_back(q);
        mems.push_back(mem);
        idx.push_back(j);
    }
    const int m0 = (int)sj.size();
    if (m0 > 0) {
        // presence of every value: one scan and one read-back for all images
        const size_t tab = ((size_t)m0 * sizeof(SortJob) + 255) / 256 * 256;
        char *sw = (char *)ibip_scratch(ctx, SC_BSORT, tab + (size_t)pres_total * 4);
        if (!sw) return IBIP_ERR_OOM;
        SortJob *djobs = (SortJob *)sw;
        int32_t *pres = (int32_t *)(sw + tab);
        cudaMemcpyAsync(djobs, sj.data(), (size_t)m0 * sizeof(SortJob), cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(pres, 0, (size_t)pres_total * 4, s);
        k_seq_pres_b<<<blk_vox, kVoxBlock, 0, s>>>(djobs, m0, pres);
        IBIP_LAUNCH(ctx);
        int st = ibip_scan_incl_i32(ctx, pres, pres, pres_total);
        if (st) return st;
        k_pres_base_b<<<(m0 + 127) / 128, 128, 0, s>>>(djobs, m0, pres);
        IBIP_LAUNCH(ctx);
        cudaMemcpyAsync(sj.data(), djobs, (size_t)m0 * sizeof(SortJob), cudaMemcpyDeviceToHost, s);
        if (ibip_sync(ctx, s) != cudaSuccess) return IBIP_ERR_CUDA;
        // chunking of each image's counting sort, as in the one-image set-up
        const int wpb = 4;
        int64_t mat_total = 0;
        int blk_chunk = 0, maxBs = 1;
        for (auto &q : sj) {
            int64_t S = kChunk;
            const int64_t mat_lim = std::max(q.N / 4, (int64_t)1 << 20);
            while (S < q.N && (q.N + S - 1) / S * (int64_t)q.B > mat_lim) S *= 2;
            q.S = (int)S;
            q.C = (int)((q.N + S - 1) / S);
            q.smem = q.B <= 1024;
            if (q.smem) maxBs = std::max(maxBs, q.B);
            q.mat_off = mat_total;
            mat_total += (int64_t)q.C * q.B;
            q.blk_chunk = blk_chunk;
            blk_chunk += (q.C + wpb - 1) / wpb;
        }
        if (mat_total >= (1ll << 31)) return IBIP_ERR_ARG;
        int32_t *mat = (int32_t *)ibip_scratch(ctx, SC_MAT, (size_t)mat_total * sizeof(int32_t));
        if (!mat) return IBIP_ERR_OOM;
        cudaMemcpyAsync(djobs, sj.data(), (size_t)m0 * sizeof(SortJob), cudaMemcpyHostToDevice, s);
        const size_t sm = (size_t)wpb * maxBs * sizeof(int32_t);
        k_chunk_hist_b<<<blk_chunk, wpb * 32, sm, s>>>(djobs, m0, pres, mat);
        IBIP_LAUNCH(ctx);
        st = ibip_scan_excl_i32(ctx, mat, mat, mat_total);
        if (st) return st;
        k_mat_base_b<<<(m0 + 127) / 128, 128, 0, s>>>(djobs, m0, mat);
        IBIP_LAUNCH(ctx);
        k_chunk_scatter_b<<<blk_chunk, wpb * 32, sm, s>>>(djobs, m0, pres, mat);
        IBIP_LAUNCH(ctx);
    }
    for (int q = 0; q < m0; q++) {
        const int j = idx[q];
        const JobMem &mem = mems[q];
        InvJob J;
        J.a = make_inv(it[j].dt2, it[j].d, it[j].inlet, it[j].max_steps, it[j].seq, it[j].step_r2, it[j].step_centre,
                       it[j].cap, maxd[j], npore[j], mem, nullptr, 0, 0);
        J.a.cancel = ctx->d_cancel;
        cudaMemsetAsync(mem.fb, 0, fb_words(J.a) * sizeof(u64), s);
        J.fd_nyz = make_fastdiv((uint32_t)it[j].d.ny * (uint32_t)it[j].d.nz);
        J.fd_nz = make_fastdiv((uint32_t)it[j].d.nz);
        J.gC = mem.gl;
        J.gD = mem.gl + npore[j];
        J.blk_plane = 0;
        dyn = std::max(dyn, invade_dyn_smem(J.a, true));
        outs[j] = mem.out;
        jobs.push_back(J);
    }
    const int m = (int)jobs.size();
    if (m > 0) {
        std::vector<int> order(m);
        for (int q = 0; q < m; q++) order[q] = q;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return nvox(it[idx[a]].d) > nvox(it[idx[b]].d);
        });
        std::vector<InvJob> sorted(m);
        int blk_plane = 0;
        for (int q = 0; q < m; q++) {
            sorted[q] = jobs[order[q]];
            sorted[q].flag = order[q];
            sorted[q].blk_plane = blk_plane;
            const Inv &a = sorted[q].a;
            blk_plane += (int)(((int64_t)a.nx * a.ny * a.NW + 255) / 256);
        }
        InvJob *djobs = (InvJob *)ibip_scratch(ctx, SC_BJOBS, (size_t)m * sizeof(InvJob));
        if (!djobs) return IBIP_ERR_OOM;
        cudaMemcpyAsync(djobs, sorted.data(), (size_t)m * sizeof(InvJob), cudaMemcpyHostToDevice, s);
        k_plane_init_b<<<blk_plane, 256, 0, s>>>(djobs, m);
        IBIP_LAUNCH(ctx);
        ibip_prof_end(ctx, IBIP_K_RANK);
        ibip_prof_begin(ctx, IBIP_K_INVADE);
        allow_max_dyn_smem((const void *)k_invade_batch);
        volatile IbipBatchDone *hd = early ? (volatile IbipBatchDone *)ctx->h_done : nullptr;
        if (hd)
            for (int q = 0; q < m; q++) hd[q].done = 0;
        k_invade_batch<<<m, kNT, dyn, s>>>(djobs, hd ? (IbipBatchDone *)ctx->d_done : nullptr);
        IBIP_LAUNCH(ctx);
        ibip_prof_end(ctx, IBIP_K_INVADE);
        if (hd) {
            // records arrive as CTAs finish; once all but kTail images are
            // done, `early` post-processes those while the rest still run
            constexpr int kTail = 8;
            std::vector<char> seen(m, 0);
            std::vector<int> done;
            int nseen = 0, first_err = IBIP_OK;
            bool fired = false;
            for (;;) {
                const bool ended = cudaStreamQuery(s) != cudaErrorNotReady;
                for (int q = 0; q < m; q++) {
                    if (seen[q] || !hd[q].done) continue;
                    std::atomic_thread_fence(std::memory_order_acquire);   // the record, then its flag
                    seen[q] = 1;
                    nseen++;
                    it[idx[q]].n_steps = hd[q].steps;
                    it[idx[q]].status = hd[q].status;
                    done.push_back(idx[q]);
                }
                if (!fired && nseen > 0 && m - nseen <= kTail && nseen < m) {
                    fired = true;
                    const int st = early(user, (int)done.size(), done.data());
                    if (st) first_err = st;
                }
                if (nseen == m) break;
                if (ended) {   // the kernel ended without every record: a device error
                    cudaGetLastError();
                    return IBIP_ERR_CUDA;
                }
                std::this_thread::yield();
            }
            cudaError_t e = ibip_sync(ctx, s);
            if (e != cudaSuccess) return ibip_cuda_status(e);
            return first_err;
        }
        // steps and status of every job
        int64_t *ho = (int64_t *)ctx->h_pinned;
        for (int q = 0; q < m; q++) cudaMemcpyAsync(ho + 2 * q, outs[idx[q]], 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        cudaError_t e = ibip_sync(ctx, s);
        if (e != cudaSuccess) return ibip_cuda_status(e);
        for (int q = 0; q < m; q++) {
            it[idx[q]].n_steps = ho[2 * q];
            it[idx[q]].status = (int)ho[2 * q + 1];
        }
    } else {
        ibip_prof_end(ctx, IBIP_K_RANK);
        cudaError_t e = ibip_sync(ctx, s);
        if (e != cudaSuccess) return ibip_cuda_status(e);
    }
    return IBIP_OK;
}
