// maximin.cu -- widest-path (maximin) propagation from an image face, used
// by defending-phase trapping (Section 2.2.3) and by the trimming step of
// morphological-opening drainage (Section 2.4.1).
//
// For a value field val (0 = blocked, -1 = +infinity, else the value) and a
// face F, M[v] is the largest, over 6-paths through unblocked voxels from a
// voxel of F to v, of the smallest value on the path (v included); -1 where
// no such path exists.  M is the least fixed point of
//     M[v] = max(M[v], min(val[v], max over neighbours u of M[u]))
// started from M = val on F.  Trapping thresholds it against seq (a voxel of
// step k is trapped iff M < k); opening keeps {M >= T}.
//
// GPU: one persistent cooperative grid.  The image is cut into 16 x 16 x 32
// tiles (z contiguous); a block loads a tile's values and its field with a
// one-voxel face halo into shared memory and relaxes it to the tile's own
// fixed point by directional line walks: a thread walks one line of the
// tile along z, y or x, forwards then backwards, carrying the running
// max-min of the line, so a value crosses the whole tile in one walk; the
// three directions alternate until three walks in a row change nothing.  A
// tile whose face rose above a neighbour's value queues that neighbour on
// the next round's work list; rounds are separated by a grid-wide barrier
// and end when a list is empty (or at the round cap).  Contexts that share
// the device with other streams run the same rounds as one ordinary launch
// each instead.
#include <cooperative_groups.h>

#include <vector>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int TX = 16, TY = 16, TZ = 32;
constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
// shared-memory strides: the field has a one-voxel halo on every face and a
// z stride of 35 words, the values a z stride of 33, so that the z walks
// (one thread per (x, y) line, lanes along y) read distinct banks
constexpr int HY = TY + 2, PZ = TZ + 3, VZ = TZ + 1;
constexpr int kFieldWords = (TX + 2) * HY * PZ;
constexpr int kValWords = TX * TY * VZ;
constexpr size_t kSmemBytes = (size_t)(kFieldWords + kValWords) * sizeof(int32_t);
constexpr int kMaxWalks = 3 * 32;               // line walks per activation before it re-queues itself
constexpr int kMaxRoundsDev = 1 << 16;

__device__ __forceinline__ int as_val(int v) { return v == -1 ? IBIP_INF32 : v; }

// the walk value of a voxel: blocked (0) never carries a path, never
// invaded (-1) is +infinity
__device__ __forceinline__ int walk_val(int v) { return v == 0 ? -1 : as_val(v); }

__device__ __forceinline__ int fidx(int hx, int hy, int hz) { return (hx * HY + hy) * PZ + hz; }
__device__ __forceinline__ int vidx(int lx, int ly, int lz) { return (lx * TY + ly) * VZ + lz; }

__global__ void k_mm_init(const int32_t *__restrict__ val, int nx, int ny, int nz, int face, int32_t *M)
{
    const int64_t N = (int64_t)nx * ny * nz;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        int z = (int)(v % nz);
        int64_t r = v / nz;
        int y = (int)(r % ny), x = (int)(r / ny);
        int s = val[v];
        M[v] = (s != 0 && d_on_face(x, y, z, nx, ny, nz, face)) ? as_val(s) : -1;
    }
}

// One image of a (possibly batched) propagation; its tiles are numbered
// tile0 .. tile0 + tx*ty*tz - 1 in the global tile space.
struct MMJob {
    const int32_t *val;
    int32_t *M;
    int nx, ny, nz, tx, ty, tz, face, tile0;
};

// tiles touching each image's face start the first round's list
__global__ void k_mm_seed(const MMJob *__restrict__ jobs, int njobs, int ntot, int *list, int *count, int *mark)
{
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ntot; g += gridDim.x * blockDim.x) {
        int lo = 0, hi = njobs;   // job: largest j with tile0 <= g
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (jobs[mid].tile0 <= g) lo = mid; else hi = mid;
        }
        const MMJob &J = jobs[lo];
        const int t = g - J.tile0;
        const int bz = t % J.tz, by = (t / J.tz) % J.ty, bx = t / (J.tz * J.ty);
        bool on = false;
        switch (J.face) {
        case 0: on = bx == 0; break;
        case 1: on = bx == J.tx - 1; break;
        case 2: on = by == 0; break;
        case 3: on = by == J.ty - 1; break;
        case 4: on = bz == 0; break;
        default: on = bz == J.tz - 1; break;
        }
        if (on) {
            mark[g] = 0;
            list[atomicAdd(count, 1)] = g;
        }
    }
}

struct MMArgs {
    const MMJob *jobs;
    int njobs;
    int *list0, *list1;   // work lists of global tile ids, alternating by round
    int *count, *head;    // per-round list sizes and take counters [max_rounds + 2]
    int *mark;            // per tile: last round it was queued for
    int *status;          // [0] rounds run, [1] 1 if the round cap was hit, [2] line walks
    int max_rounds;
};

// One walk along a line of n voxels: field entries f[0], f[fs], ..., values
// v[0], v[vs], ...; the running value enters from the halo entry before the
// first voxel (f[-fs]) and leaves into nothing.  Forward then backward.
// Bit i of the result: entry i rose.
template <int n>
__device__ __forceinline__ uint32_t walk_line(int32_t *f, int fs, const int32_t *v, int vs)
{
    uint32_t ch = 0;
    int m = f[-fs];
#pragma unroll 8
    for (int i = 0; i < n; i++) {
        const int cur = f[i * fs];
        const int nm = max(cur, min(v[i * vs], m));
        if (nm != cur) { f[i * fs] = nm; ch |= 1u << i; }
        m = nm;
    }
    m = f[n * fs];
#pragma unroll 8
    for (int i = n - 1; i >= 0; i--) {
        const int cur = f[i * fs];
        const int nm = max(cur, min(v[i * vs], m));
        if (nm != cur) { f[i * fs] = nm; ch |= 1u << i; }
        m = nm;
    }
    return ch;
}

// Claims and relaxes the tiles of round r's list until the list is drained.
// A tile queues a neighbour for round r + 1 only where one of its face
// voxels rose in this activation above the neighbour's value across that
// face (as loaded): M only grows, so no other neighbour can improve.  In
// round 0 the seeded values count as risen.
__device__ void mm_round(const MMArgs &a, int r, int32_t *sM, int32_t *sV, uint32_t *sRise, int *s_tile,
                         int *s_wake)
{
    const int cnt = __ldcg(a.count + r);
    const int *list = (r & 1) ? a.list1 : a.list0;
    int *next = (r & 1) ? a.list0 : a.list1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) {
            const int q = atomicAdd(&a.head[r], 1);
            *s_tile = q < cnt ? __ldcg(list + q) : -1;
        }
        __syncthreads();
        const int g = *s_tile;
        if (g < 0) break;
        int lo = 0, hi = a.njobs;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(&a.jobs[mid].tile0) <= g) lo = mid; else hi = mid;
        }
        const MMJob J = a.jobs[lo];
        const int t = g - J.tile0;
        const int bz = t % J.tz, by = (t / J.tz) % J.ty, bx = t / (J.tz * J.ty);
        const int x0 = bx * TX, y0 = by * TY, z0 = bz * TZ;
        const int z = z0 + lane;
        const bool zin = z < J.nz;
        // rows of 32 z voxels: the tile's 256 rows (values, field and the
        // two z-end halo entries) and the 64 rows of the x / y face halos
        // (field only); a warp takes every 16th row, all loads of four rows
        // issued before their shared-memory stores
        constexpr int kRows = TX * TY + 2 * TX + 2 * TY;
#pragma unroll 1
        for (int r0 = w; r0 < kRows; r0 += 4 * kWarps) {
            int fv[4], vv[4], ez[4];
            int hx[4], hy[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int row = r0 + u * kWarps;
                fv[u] = -1; vv[u] = 0; ez[u] = -1;
                hx[u] = -1; hy[u] = -1;
                if (row >= kRows) continue;
                if (row < TX * TY) {
                    hx[u] = row / TY + 1; hy[u] = row % TY + 1;
                } else {
                    const int q = row - TX * TY;   // 0..63: x0-1, x0+16 faces (16 rows each), then y faces
                    if (q < 2 * TY) { hx[u] = q < TY ? 0 : TX + 1; hy[u] = q % TY + 1; }
                    else { const int p = q - 2 * TY; hy[u] = p < TX ? 0 : TY + 1; hx[u] = p % TX + 1; }
                }
                const int x = x0 + hx[u] - 1, y = y0 + hy[u] - 1;
                if (x < 0 || y < 0 || x >= J.nx || y >= J.ny) continue;
                const int64_t rb = d_lin(x, y, 0, J.ny, J.nz);
                if (zin) {
                    fv[u] = __ldcg(J.M + rb + z);
                    if (row < TX * TY) vv[u] = __ldg(J.val + rb + z);
                }
                if (row < TX * TY) {   // z-end halo: lane 0 the entry before, lane 31 the one after
                    if (lane == 0 && z0 > 0) ez[u] = __ldcg(J.M + rb + z0 - 1);
                    if (lane == 31 && z0 + TZ < J.nz) ez[u] = __ldcg(J.M + rb + z0 + TZ);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int row = r0 + u * kWarps;
                if (row >= kRows) continue;
                sM[fidx(hx[u], hy[u], lane + 1)] = fv[u];
                if (row < TX * TY) {
                    sV[vidx(hx[u] - 1, hy[u] - 1, lane)] = walk_val(vv[u]);
                    if (lane == 0) sM[fidx(hx[u], hy[u], 0)] = ez[u];
                    if (lane == 31) sM[fidx(hx[u], hy[u], TZ + 1)] = ez[u];
                }
            }
        }
        if (threadIdx.x < 6) s_wake[threadIdx.x] = 0;
        if (threadIdx.x < TX * TY) sRise[threadIdx.x] = 0;
        __syncthreads();
        // the tile's face values as loaded (round 0: the seeds count as
        // risen): per thread the x- and y-face voxels of one (row, z) and,
        // for threads 0..255, the z-face voxels of one (x, y) line
        const int fa = w;
        const int zx = threadIdx.x >> 4 & 15, zy = threadIdx.x & 15;
        int mold[6];
        mold[0] = r == 0 ? -1 : sM[fidx(1, fa + 1, lane + 1)];          // x = 0 face, y = fa
        mold[1] = r == 0 ? -1 : sM[fidx(TX, fa + 1, lane + 1)];         // x = 15 face
        mold[2] = r == 0 ? -1 : sM[fidx(fa + 1, 1, lane + 1)];          // y = 0 face, x = fa
        mold[3] = r == 0 ? -1 : sM[fidx(fa + 1, TY, lane + 1)];         // y = 15 face
        mold[4] = r == 0 ? -1 : sM[fidx(zx + 1, zy + 1, 1)];            // z = 0 face
        mold[5] = r == 0 ? -1 : sM[fidx(zx + 1, zy + 1, TZ)];           // z = 31 face
        // walks: z (threads 0..255, one (x, y) line each), y (warp = x,
        // lane = z), x (warp = y, lane = z), cycled until three walks in a
        // row change nothing; sRise[x * 16 + y] collects the z bits of the
        // voxels that rose (each row word has one writer per walk)
        int quiet = 0, walks = 0;
        for (int dir = 0; walks < kMaxWalks; dir = dir == 2 ? 0 : dir + 1) {
            bool ch = false;
            if (dir == 0) {
                if (threadIdx.x < TX * TY) {
                    const int lx = threadIdx.x / TY, ly = threadIdx.x % TY;
                    const uint32_t b = walk_line<TZ>(sM + fidx(lx + 1, ly + 1, 1), 1, sV + vidx(lx, ly, 0), 1);
                    if (b) { sRise[threadIdx.x] |= b; ch = true; }
                }
            } else if (dir == 1) {
                const uint32_t b = walk_line<TY>(sM + fidx(w + 1, 1, lane + 1), PZ, sV + vidx(w, 0, lane), VZ);
#pragma unroll
                for (int i = 0; i < TY; i++) {   // voxel (w, i, lane) rose: bit lane of row (w, i)
                    const uint32_t m = __ballot_sync(0xffffffffu, b >> i & 1u);
                    if (lane == 0 && m) sRise[w * TY + i] |= m;
                }
                ch = b != 0;
            } else {
                const uint32_t b = walk_line<TX>(sM + fidx(1, w + 1, lane + 1), HY * PZ, sV + vidx(0, w, lane), TY * VZ);
#pragma unroll
                for (int i = 0; i < TX; i++) {   // voxel (i, w, lane): bit lane of row (i, w)
                    const uint32_t m = __ballot_sync(0xffffffffu, b >> i & 1u);
                    if (lane == 0 && m) sRise[i * TY + w] |= m;
                }
                ch = b != 0;
            }
            walks++;
            if (__syncthreads_or(ch)) quiet = 0;
            else if (++quiet == 3) break;
        }
        const bool conv = quiet == 3;
        if (threadIdx.x == 0) atomicAdd(a.status + 2, walks);
        // wake a neighbour across a face where a face voxel rose above the
        // neighbour's value there
        if (z0 + lane < J.nz) {
            const int zz = lane + 1;
            int v;
            v = sM[fidx(1, fa + 1, zz)];
            if (v > mold[0] && v > sM[fidx(0, fa + 1, zz)]) s_wake[0] = 1;
            v = sM[fidx(TX, fa + 1, zz)];
            if (v > mold[1] && v > sM[fidx(TX + 1, fa + 1, zz)]) s_wake[1] = 1;
            v = sM[fidx(fa + 1, 1, zz)];
            if (v > mold[2] && v > sM[fidx(fa + 1, 0, zz)]) s_wake[2] = 1;
            v = sM[fidx(fa + 1, TY, zz)];
            if (v > mold[3] && v > sM[fidx(fa + 1, TY + 1, zz)]) s_wake[3] = 1;
        }
        if (threadIdx.x < TX * TY) {
            int v = sM[fidx(zx + 1, zy + 1, 1)];
            if (v > mold[4] && v > sM[fidx(zx + 1, zy + 1, 0)]) s_wake[4] = 1;
            v = sM[fidx(zx + 1, zy + 1, TZ)];
            if (v > mold[5] && v > sM[fidx(zx + 1, zy + 1, TZ + 1)]) s_wake[5] = 1;
        }
        __syncthreads();
        // store the voxels that rose (each belongs to this tile alone)
#pragma unroll 4
        for (int row = w; row < TX * TY; row += kWarps) {
            if (!(sRise[row] >> lane & 1u)) continue;
            const int lx = row / TY, ly = row % TY;
            J.M[d_lin(x0 + lx, y0 + ly, z, J.ny, J.nz)] = sM[fidx(lx + 1, ly + 1, lane + 1)];
        }
        if (threadIdx.x < 7) {   // one lane per neighbour (6) and the tile itself: the atomics overlap
            const int q = threadIdx.x, nr = r + 1;
            int nb = -1;
            switch (q) {
            case 0: if (bx > 0 && s_wake[0]) nb = g - J.tz * J.ty; break;
            case 1: if (bx < J.tx - 1 && s_wake[1]) nb = g + J.tz * J.ty; break;
            case 2: if (by > 0 && s_wake[2]) nb = g - J.tz; break;
            case 3: if (by < J.ty - 1 && s_wake[3]) nb = g + J.tz; break;
            case 4: if (bz > 0 && s_wake[4]) nb = g - 1; break;
            case 5: if (bz < J.tz - 1 && s_wake[5]) nb = g + 1; break;
            default: if (!conv) nb = g; break;
            }
            if (nb >= 0 && atomicMax(&a.mark[nb], nr) < nr) next[atomicAdd(&a.count[nr], 1)] = nb;
        }
        __syncthreads();
    }
}

// All rounds in one cooperative launch, a grid barrier between rounds.
__global__ void __launch_bounds__(kThreads, 2) k_mm_persistent(MMArgs a)
{
    cg::grid_group grid = cg::this_grid();
    extern __shared__ int32_t s_mm[];
    __shared__ uint32_t sRise[TX * TY];
    __shared__ int s_tile, s_wake[6];
    int r = 0;
    for (;; r++) {
        if (__ldcg(a.count + r) == 0 || r >= a.max_rounds) break;
        mm_round(a, r, s_mm, s_mm + kFieldWords, sRise, &s_tile, s_wake);
        __threadfence();
        grid.sync();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.status[0] = r;
        a.status[1] = (r >= a.max_rounds && __ldcg(a.count + r) != 0) ? 1 : 0;
    }
}

// One round per launch: for contexts whose kernels share the device with
// other streams (a cooperative grid could not be made resident beside them).
__global__ void __launch_bounds__(kThreads, 2) k_mm_round(MMArgs a, int r)
{
    extern __shared__ int32_t s_mm[];
    __shared__ uint32_t sRise[TX * TY];
    __shared__ int s_tile, s_wake[6];
    if (r >= a.max_rounds || __ldcg(a.count + r) == 0) return;
    mm_round(a, r, s_mm, s_mm + kFieldWords, sRise, &s_tile, s_wake);
}

}  // namespace

int ibip_maximin_multi(ibip_ctx *ctx, int n, const IbipMaximinJob *jobs, int max_rounds)
{
    cudaStream_t s = ctx->stream;
    if (n <= 0) return IBIP_OK;
    std::vector<MMJob> J(n);
    int64_t ntot = 0;
    for (int j = 0; j < n; j++) {
        const ibip_dims d = jobs[j].d;
        J[j].val = jobs[j].val; J[j].M = jobs[j].M;
        J[j].nx = d.nx; J[j].ny = d.ny; J[j].nz = d.nz;
        J[j].tx = (d.nx + TX - 1) / TX; J[j].ty = (d.ny + TY - 1) / TY; J[j].tz = (d.nz + TZ - 1) / TZ;
        J[j].face = jobs[j].face;
        J[j].tile0 = (int)ntot;
        ntot += (int64_t)J[j].tx * J[j].ty * J[j].tz;
    }
    if (ntot >= (1ll << 30)) return IBIP_ERR_ARG;
    const int nt = (int)ntot;
    const int rounds = max_rounds < kMaxRoundsDev ? max_rounds : kMaxRoundsDev;
    // layout: jobs | list0[nt] list1[nt] mark[nt] count[rounds+2] head[rounds+2] status[4]
    const size_t jb = ((size_t)n * sizeof(MMJob) + 255) & ~(size_t)255;
    const size_t ints = (size_t)3 * nt + 2 * ((size_t)rounds + 2) + 4;
    char *w0 = (char *)ibip_scratch(ctx, SC_TILE, jb + ints * sizeof(int));
    if (!w0) return IBIP_ERR_OOM;
    MMJob *djobs = (MMJob *)w0;
    int *w = (int *)(w0 + jb);
    MMArgs a;
    a.jobs = djobs; a.njobs = n;
    a.list0 = w; a.list1 = w + nt; a.mark = w + 2 * nt;
    a.count = w + 3 * nt; a.head = a.count + rounds + 2; a.status = a.head + rounds + 2;
    a.max_rounds = rounds;
    ibip_prof_begin(ctx, IBIP_K_MAXIMIN);
    cudaMemcpyAsync(djobs, J.data(), (size_t)n * sizeof(MMJob), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(a.mark, 0xff, (size_t)nt * sizeof(int), s);   // -1: never queued
    cudaMemsetAsync(a.count, 0, (2 * ((size_t)rounds + 2) + 4) * sizeof(int), s);   // counts, heads, status
    for (int j = 0; j < n; j++) {
        k_mm_init<<<ctx->sm_count * 4, 256, 0, s>>>(J[j].val, J[j].nx, J[j].ny, J[j].nz, J[j].face, J[j].M);
        IBIP_LAUNCH(ctx);
    }
    k_mm_seed<<<(nt + 255) / 256, 256, 0, s>>>(djobs, n, nt, a.list0, a.count, a.mark);
    IBIP_LAUNCH(ctx);
    int *h = (int *)ctx->h_pinned;
    if (cudaFuncSetAttribute(k_mm_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_mm_round, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) !=
            cudaSuccess) {
        cudaGetLastError();
        return IBIP_ERR_CUDA;
    }
    if (ctx->no_coop) {
        // rounds in chunks; the next round's list size is read back after
        // each chunk (an empty round's launch returns at once)
        constexpr int kChunkRounds = 16;
        const int grid = ctx->sm_count;
        int r = 0;
        for (;;) {
            for (int q = 0; q < kChunkRounds && r < rounds; q++, r++) {
                k_mm_round<<<grid, kThreads, kSmemBytes, s>>>(a, r);
                IBIP_LAUNCH(ctx);
            }
            cudaMemcpyAsync(h, a.count + r, sizeof(int), cudaMemcpyDeviceToHost, s);
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return ibip_cuda_status(e);
            if (h[0] == 0) break;
            if (r >= rounds) {
                ibip_prof_end(ctx, IBIP_K_MAXIMIN);
                return IBIP_ERR_NOT_CONVERGED;
            }
        }
        ibip_prof_end(ctx, IBIP_K_MAXIMIN);
        return IBIP_OK;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mm_persistent, kThreads, kSmemBytes) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return IBIP_ERR_CUDA;
    }
    int grid = ctx->sm_count * per_sm;
    if (grid > nt) grid = nt;
    void *args[] = {&a};
    cudaError_t e = cudaLaunchCooperativeKernel((void *)k_mm_persistent, grid, kThreads, args, kSmemBytes, s);
    IBIP_LAUNCH(ctx);
    if (e != cudaSuccess) return ibip_cuda_status(e);
    cudaMemcpyAsync(h, a.status, 3 * sizeof(int), cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
    ibip_prof_end(ctx, IBIP_K_MAXIMIN);
    if (e != cudaSuccess) return ibip_cuda_status(e);
    // diagnostics of the last propagation: rounds, tile activations, sweeps
    {
        const int nr = h[0] < rounds ? h[0] : rounds, conv_flag = h[1], sweeps = h[2];
        int *hc = (int *)ctx->h_pinned;
        int64_t act = 0;
        for (int r0 = 0; r0 < nr; r0 += 8192) {
            const int c = nr - r0 < 8192 ? nr - r0 : 8192;
            cudaMemcpyAsync(hc, a.count + r0, (size_t)c * sizeof(int), cudaMemcpyDeviceToHost, s);
            if (cudaStreamSynchronize(s) != cudaSuccess) return IBIP_ERR_CUDA;
            for (int q = 0; q < c; q++) act += hc[q];
        }
        ctx->inv_stats[30] = nr;
        ctx->inv_stats[31] = act;
        ctx->inv_stats[32] = sweeps;
        return conv_flag ? IBIP_ERR_NOT_CONVERGED : IBIP_OK;
    }
}

int ibip_maximin_launch(ibip_ctx *ctx, const int32_t *val, ibip_dims d, int face, int32_t *M, int max_rounds)
{
    IbipMaximinJob j{val, d, face, M};
    return ibip_maximin_multi(ctx, 1, &j, max_rounds);
}
