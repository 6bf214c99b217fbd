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
// GPU: the image is cut into 4 x 8 x 32 tiles (z contiguous); a block loads
// a tile with a one-voxel halo into shared memory and relaxes it until it
// stops changing, and a tile that changed wakes each neighbour across a
// face where one of its voxels rose above the neighbour's value.  Two
// schedules run the same relaxation:
//  * rounds: woken tiles form the next round's work list; rounds end when
//    a list is empty (or at the round cap).  One persistent cooperative
//    grid with a grid-wide barrier between rounds for one large image; one
//    ordinary launch per round in contexts that share the device with
//    other streams, so that their kernels' blocks get in between rounds.
//  * queue: one persistent ordinary launch over a work queue, no rounds and
//    no barrier; the propagation ends when the queue is empty and no tile
//    is being relaxed.  Used for batches and smaller images.
// Everything other blocks write (the field, the lists, the queue, the
// counters) is read with L2-coherent loads: the SM's L1 may hold a stale
// line.
#include <cooperative_groups.h>

#include <cstring>
#include <vector>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int TX = 4, TY = 8, TZ = 32;
constexpr int kThreads = 256;
constexpr int kPer = TX * TY * TZ / kThreads;   // voxels per thread
constexpr int kInner = 96;                      // relaxation sweeps per activation
// resident blocks per SM the register budget is sized for (measured on the
// 512^3 blobs' trapping: 4 -> 36.7 ms, 5 -> 39.2 ms, 6 -> 43.8 ms)
constexpr int kMinBlocks = 4;
constexpr int kMaxRoundsDev = 1 << 16;
// Single images of fewer tiles use the queue.  Measured with both schedules
// (trapping of the 200^3 sphere pack, 8,750 tiles: rounds 3.50 ms, queue
// 2.24 ms; of the 512^3 blobs, 131,072 tiles: 37.2 / 43.0 ms; the queue
// then still stored whole tiles, before its atomic write-back of risen
// voxels); the bound is the geometric midpoint of the two.
constexpr int kQueueTiles = 32768;
// a queue block that waits for work gives up, and stops the propagation
// with an error status, once the grid has made no progress for this long
constexpr unsigned long long kStallNs = 5000000000ull;
// activation cap of the queue, in activations per tile (~20 in practice)
constexpr int kQueueActsPerTile = 512;

__device__ __forceinline__ unsigned long long mm_now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int as_val(int v) { return v == -1 ? IBIP_INF32 : v; }

// M = val on the unblocked voxels of the face, -1 elsewhere; a warp per
// row (x, y), lanes along z, no per-voxel division
__global__ void k_mm_init(const int32_t *__restrict__ val, int nx, int ny, int nz, int face, int32_t *M)
{
    const int lane = threadIdx.x & 31;
    const int64_t nrows = (int64_t)nx * ny;
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < nrows; row += wstride) {
        const int x = (int)(row / ny), y = (int)(row - (int64_t)x * ny);
        const bool row_on = (face == 0 && x == 0) || (face == 1 && x == nx - 1) || (face == 2 && y == 0) ||
                            (face == 3 && y == ny - 1);
        const int64_t b = row * nz;
        for (int z = lane; z < nz; z += 32) {
            const bool on = row_on || (face == 4 && z == 0) || (face == 5 && z == nz - 1);
            int m = -1;
            if (on) {
                const int sv = val[b + z];
                if (sv != 0) m = as_val(sv);
            }
            M[b + z] = m;
        }
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
    int *status;          // [0] rounds run, [1] 1 if the round cap was hit, [2] relaxation sweeps
    int max_rounds;
};

// Claims and relaxes the tiles of round r's list until the list is drained.
// A tile queues a neighbour for round r + 1 only where one of its face
// voxels rose in this activation above the neighbour's value across that
// face (as loaded): M only grows, so no other neighbour can improve.  In
// round 0 the seeded values count as risen.
__device__ void mm_round(const MMArgs &a, int r, int32_t (*sM)[TY + 2][TZ + 2], int *s_tile, int *s_wake)
{
    const int cnt = __ldcg(a.count + r);
    const int *list = (r & 1) ? a.list1 : a.list0;
    int *next = (r & 1) ? a.list0 : a.list1;
    // thread 0 claims one tile ahead: the claim is issued when the current
    // tile starts and its list entry read after the relaxation, so neither
    // round trip lies on the path between two tiles
    int next_g = -1;
    if (threadIdx.x == 0) {
        const int q = atomicAdd(&a.head[r], 1);
        next_g = q < cnt ? __ldcg(list + q) : -1;
    }
    for (;;) {
        if (threadIdx.x == 0) *s_tile = next_g;
        __syncthreads();
        const int g = *s_tile;
        if (g < 0) break;
        int q_next = 0;
        if (threadIdx.x == 0) q_next = atomicAdd(&a.head[r], 1);
        int lo = 0, hi = a.njobs;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(&a.jobs[mid].tile0) <= g) lo = mid; else hi = mid;
        }
        const MMJob J = a.jobs[lo];
        const int t = g - J.tile0;
        const int bz = t % J.tz, by = (t / J.tz) % J.ty, bx = t / (J.tz * J.ty);
        const int x0 = bx * TX, y0 = by * TY, z0 = bz * TZ;
        // the tile's values and the field on the tile plus a one-voxel halo:
        // every load is issued before the first store to shared memory
        int sval[kPer], lx[kPer], ly[kPer], lz[kPer];
#pragma unroll
        for (int k = 0; k < kPer; k++) {
            const int i = threadIdx.x + k * kThreads;
            lz[k] = i % TZ; ly[k] = (i / TZ) % TY; lx[k] = i / (TZ * TY);
            const int x = x0 + lx[k], y = y0 + ly[k], z = z0 + lz[k];
            sval[k] = (x < J.nx && y < J.ny && z < J.nz) ? J.val[d_lin(x, y, z, J.ny, J.nz)] : 0;
        }
        constexpr int kHalo = (TX + 2) * (TY + 2) * (TZ + 2);
        constexpr int kHaloPer = (kHalo + kThreads - 1) / kThreads;
        int hv[kHaloPer];
#pragma unroll
        for (int u = 0; u < kHaloPer; u++) {
            const int i = threadIdx.x + u * kThreads;
            const int hz = i % (TZ + 2), hy = (i / (TZ + 2)) % (TY + 2), hx = i / ((TZ + 2) * (TY + 2));
            const int x = x0 + hx - 1, y = y0 + hy - 1, z = z0 + hz - 1;
            hv[u] = -1;
            if (i < kHalo && x >= 0 && y >= 0 && z >= 0 && x < J.nx && y < J.ny && z < J.nz)
                hv[u] = __ldcg(J.M + d_lin(x, y, z, J.ny, J.nz));
        }
        int32_t *sflat = &sM[0][0][0];
#pragma unroll
        for (int u = 0; u < kHaloPer; u++) {
            const int i = threadIdx.x + u * kThreads;
            if (i < kHalo) sflat[i] = hv[u];
        }
#pragma unroll
        for (int k = 0; k < kPer; k++) sval[k] = as_val(sval[k]);
        if (threadIdx.x < 6) s_wake[threadIdx.x] = 0;
        __syncthreads();
        int mold[kPer];
#pragma unroll
        for (int k = 0; k < kPer; k++) mold[k] = r == 0 ? -1 : sM[lx[k] + 1][ly[k] + 1][lz[k] + 1];
        bool any = false, conv = false;
        int sweeps = 0;
        for (int it = 0; it < kInner; it++) {
            sweeps++;
            int ch = 0;
#pragma unroll
            for (int k = 0; k < kPer; k++) {
                if (sval[k] == 0) continue;
                const int hx = lx[k] + 1, hy = ly[k] + 1, hz = lz[k] + 1;
                const int b = max(max(max(sM[hx - 1][hy][hz], sM[hx + 1][hy][hz]), max(sM[hx][hy - 1][hz], sM[hx][hy + 1][hz])),
                                  max(sM[hx][hy][hz - 1], sM[hx][hy][hz + 1]));
                const int nv = min(b, sval[k]);
                if (nv > sM[hx][hy][hz]) { sM[hx][hy][hz] = nv; ch = 1; }
            }
            if (!__syncthreads_or(ch)) { conv = true; break; }
            any = true;
        }
        if (threadIdx.x == 0) {
            atomicAdd(a.status + 2, sweeps);
            next_g = q_next < cnt ? __ldcg(list + q_next) : -1;
        }
#pragma unroll
        for (int k = 0; k < kPer; k++) {
            if (sval[k] == 0) continue;
            const int hx = lx[k] + 1, hy = ly[k] + 1, hz = lz[k] + 1;
            const int mv = sM[hx][hy][hz];
            if (mv <= mold[k]) continue;   // not risen here
            if (lx[k] == 0 && mv > sM[0][hy][hz]) s_wake[0] = 1;
            if (lx[k] == TX - 1 && mv > sM[TX + 1][hy][hz]) s_wake[1] = 1;
            if (ly[k] == 0 && mv > sM[hx][0][hz]) s_wake[2] = 1;
            if (ly[k] == TY - 1 && mv > sM[hx][TY + 1][hz]) s_wake[3] = 1;
            if (lz[k] == 0 && mv > sM[hx][hy][0]) s_wake[4] = 1;
            if (lz[k] == TZ - 1 && mv > sM[hx][hy][TZ + 1]) s_wake[5] = 1;
        }
        __syncthreads();
        if (any) {
#pragma unroll
            for (int k = 0; k < kPer; k++) {
                const int x = x0 + lx[k], y = y0 + ly[k], z = z0 + lz[k];
                if (x < J.nx && y < J.ny && z < J.nz && sval[k] != 0)
                    J.M[d_lin(x, y, z, J.ny, J.nz)] = sM[lx[k] + 1][ly[k] + 1][lz[k] + 1];
            }
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
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_mm_persistent(MMArgs a)
{
    cg::grid_group grid = cg::this_grid();
    __shared__ int32_t sM[TX + 2][TY + 2][TZ + 2];
    __shared__ int s_tile, s_wake[6];
    int r = 0;
    for (;; r++) {
        if (__ldcg(a.count + r) == 0 || r >= a.max_rounds) break;
        mm_round(a, r, sM, &s_tile, s_wake);
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
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_mm_round(MMArgs a, int r)
{
    __shared__ int32_t sM[TX + 2][TY + 2][TZ + 2];
    __shared__ int s_tile, s_wake[6];
    if (r >= a.max_rounds || __ldcg(a.count + r) == 0) return;
    mm_round(a, r, sM, &s_tile, s_wake);
}

// The work queue: a ring of entries (tile id, bit 30 = queued as a seed; -1 =
// empty slot) with monotone head and tail counters.  A block takes a
// ticket (head) before it needs the tile and waits, when it does, for the
// push that fills its slot.  A tile is pushed only when its flag goes from
// 0 to 1 and the flag is cleared when it is taken, so the ring never holds
// more than ntiles entries; its capacity adds a slot per block for the
// tickets not yet filled.
struct MMQ {
    const MMJob *jobs;
    int njobs;
    int *ring;                    // [cap]
    int *queued;                  // per tile: 1 while in the ring
    unsigned long long *head, *tail;
    int *pending;                 // tiles in the ring or being relaxed
    unsigned long long *acts;     // tile activations so far (progress)
    int *sweeps;                  // relaxation sweeps (diagnostics)
    int *stop;                    // 1: activation cap reached, 2: no progress
    long long max_acts;
    int cap;
};

constexpr int kSeedBit = 1 << 30;

// Queue tile g unless it is waiting already; a seed tile's first relaxation
// counts every voxel as risen (its face values were set before it ran).
// pending counts the tile before it can be taken, so the count never
// reaches 0 while work remains.
__device__ __forceinline__ void mmq_push(const MMQ &Q, int g, bool seed)
{
    if (atomicCAS(Q.queued + g, 0, 1) != 0) return;
    atomicAdd(Q.pending, 1);
    __threadfence();
    const unsigned long long t = atomicAdd(Q.tail, 1ull);
    *(volatile int *)(Q.ring + (int)(t % (unsigned long long)Q.cap)) = g | (seed ? kSeedBit : 0);
}

// The tile of ticket h (*seed: queued as a seed), or -1 once the
// propagation is over (nothing queued or being relaxed, so no push will
// come) or stopped.  Only the ticket's holder reads its slot.
__device__ int mmq_take(const MMQ &Q, unsigned long long h, bool *seed)
{
    volatile int *slot = Q.ring + (int)(h % (unsigned long long)Q.cap);
    unsigned long long seen = ~0ull, since = 0;
    for (;;) {
        if (*(volatile int *)Q.stop) return -1;
        const int raw = *slot;
        if (raw >= 0) {
            *slot = -1;
            const int g = raw & (kSeedBit - 1);
            *seed = (raw & kSeedBit) != 0;
            atomicAnd(Q.queued + g, 0);
            __threadfence();
            return g;
        }
        if (*(volatile int *)Q.pending == 0) return -1;
        // blocks still relaxing may queue more; give up only when the
        // whole grid has made no progress for kStallNs
        const unsigned long long a = *(volatile unsigned long long *)Q.acts;
        const unsigned long long now = mm_now_ns();
        if (a != seen) { seen = a; since = now; }
        else if (now - since > kStallNs) { atomicExch(Q.stop, 2); return -1; }
        __nanosleep(64);
    }
}

// The tile of ticket h if its slot is filled already (returns false, and
// takes nothing, otherwise).
__device__ __forceinline__ bool mmq_try_take(const MMQ &Q, unsigned long long h, int *g, bool *seed)
{
    volatile int *slot = Q.ring + (int)(h % (unsigned long long)Q.cap);
    const int raw = *slot;
    if (raw < 0) return false;
    *slot = -1;
    *g = raw & (kSeedBit - 1);
    *seed = (raw & kSeedBit) != 0;
    atomicAnd(Q.queued + *g, 0);
    __threadfence();
    return true;
}

// tiles touching each image's face are queued first (queue schedule)
__global__ void k_mm_qseed(MMQ Q, int ntot)
{
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ntot; g += gridDim.x * blockDim.x) {
        int lo = 0, hi = Q.njobs;   // job: largest j with tile0 <= g
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (Q.jobs[mid].tile0 <= g) lo = mid; else hi = mid;
        }
        const MMJob &J = Q.jobs[lo];
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
        if (on) mmq_push(Q, g, true);
    }
}

// One persistent launch: each block relaxes tiles from the queue until the
// propagation is over.  Thread 0 takes the ticket of the block's next tile
// when the current one starts, so that atomic is off the path between tiles.
// A tile queues a neighbour only where one of its face voxels rose in this
// relaxation above the neighbour's value across that face (as loaded): M
// only grows, so no other neighbour can improve.  A seed tile's first
// relaxation counts its face values as risen.
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_mm_queue(MMQ Q)
{
    __shared__ int32_t sM[TX + 2][TY + 2][TZ + 2];
    __shared__ int s_tile, s_seed, s_wake[6];
    int next_g = -1, my_acts = 0, my_sweeps = 0;
    bool next_seed = false;
    if (threadIdx.x == 0) next_g = mmq_take(Q, atomicAdd(Q.head, 1ull), &next_seed);
    for (;;) {
        if (threadIdx.x == 0) { s_tile = next_g; s_seed = next_seed ? 1 : 0; }
        __syncthreads();
        const int g = s_tile;
        const bool seed = s_seed != 0;
        if (g < 0) {
            if (threadIdx.x == 0 && my_acts) {
                atomicAdd(Q.sweeps, my_sweeps);
                atomicAdd(Q.acts, (unsigned long long)my_acts);
            }
            break;
        }
        unsigned long long ticket = 0;
        if (threadIdx.x == 0) ticket = atomicAdd(Q.head, 1ull);
        int lo = 0, hi = Q.njobs;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(&Q.jobs[mid].tile0) <= g) lo = mid; else hi = mid;
        }
        const MMJob J = Q.jobs[lo];
        const int t = g - J.tile0;
        const int bz = t % J.tz, by = (t / J.tz) % J.ty, bx = t / (J.tz * J.ty);
        const int x0 = bx * TX, y0 = by * TY, z0 = bz * TZ;
        // the tile's values and the field on the tile plus a one-voxel halo:
        // every load is issued before the first store to shared memory
        int sval[kPer], lx[kPer], ly[kPer], lz[kPer];
#pragma unroll
        for (int k = 0; k < kPer; k++) {
            const int i = threadIdx.x + k * kThreads;
            lz[k] = i % TZ; ly[k] = (i / TZ) % TY; lx[k] = i / (TZ * TY);
            const int x = x0 + lx[k], y = y0 + ly[k], z = z0 + lz[k];
            sval[k] = (x < J.nx && y < J.ny && z < J.nz) ? J.val[d_lin(x, y, z, J.ny, J.nz)] : 0;
        }
        constexpr int kHalo = (TX + 2) * (TY + 2) * (TZ + 2);
        constexpr int kHaloPer = (kHalo + kThreads - 1) / kThreads;
        int hv[kHaloPer];
#pragma unroll
        for (int u = 0; u < kHaloPer; u++) {
            const int i = threadIdx.x + u * kThreads;
            const int hz = i % (TZ + 2), hy = (i / (TZ + 2)) % (TY + 2), hx = i / ((TZ + 2) * (TY + 2));
            const int x = x0 + hx - 1, y = y0 + hy - 1, z = z0 + hz - 1;
            hv[u] = -1;
            if (i < kHalo && x >= 0 && y >= 0 && z >= 0 && x < J.nx && y < J.ny && z < J.nz)
                hv[u] = __ldcg(J.M + d_lin(x, y, z, J.ny, J.nz));
        }
        int32_t *sflat = &sM[0][0][0];
#pragma unroll
        for (int u = 0; u < kHaloPer; u++) {
            const int i = threadIdx.x + u * kThreads;
            if (i < kHalo) sflat[i] = hv[u];
        }
#pragma unroll
        for (int k = 0; k < kPer; k++) sval[k] = as_val(sval[k]);
        if (threadIdx.x < 6) s_wake[threadIdx.x] = 0;
        __syncthreads();
        int mold[kPer];
#pragma unroll
        for (int k = 0; k < kPer; k++) mold[k] = seed ? -1 : sM[lx[k] + 1][ly[k] + 1][lz[k] + 1];
        bool any = false, conv = false;
        int sweeps = 0;
        for (int it = 0; it < kInner; it++) {
            sweeps++;
            int ch = 0;
#pragma unroll
            for (int k = 0; k < kPer; k++) {
                if (sval[k] == 0) continue;
                const int hx = lx[k] + 1, hy = ly[k] + 1, hz = lz[k] + 1;
                const int b = max(max(max(sM[hx - 1][hy][hz], sM[hx + 1][hy][hz]), max(sM[hx][hy - 1][hz], sM[hx][hy + 1][hz])),
                                  max(sM[hx][hy][hz - 1], sM[hx][hy][hz + 1]));
                const int nv = min(b, sval[k]);
                if (nv > sM[hx][hy][hz]) { sM[hx][hy][hz] = nv; ch = 1; }
            }
            if (!__syncthreads_or(ch)) { conv = true; break; }
            any = true;
        }
        // the next tile, if its push has come already: taken while this
        // one's results are written
        bool got = false;
        if (threadIdx.x == 0) got = mmq_try_take(Q, ticket, &next_g, &next_seed);
#pragma unroll
        for (int k = 0; k < kPer; k++) {
            if (sval[k] == 0) continue;
            const int hx = lx[k] + 1, hy = ly[k] + 1, hz = lz[k] + 1;
            const int mv = sM[hx][hy][hz];
            if (mv <= mold[k]) continue;   // not risen here
            if (lx[k] == 0 && mv > sM[0][hy][hz]) s_wake[0] = 1;
            if (lx[k] == TX - 1 && mv > sM[TX + 1][hy][hz]) s_wake[1] = 1;
            if (ly[k] == 0 && mv > sM[hx][0][hz]) s_wake[2] = 1;
            if (ly[k] == TY - 1 && mv > sM[hx][TY + 1][hz]) s_wake[3] = 1;
            if (lz[k] == 0 && mv > sM[hx][hy][0]) s_wake[4] = 1;
            if (lz[k] == TZ - 1 && mv > sM[hx][hy][TZ + 1]) s_wake[5] = 1;
        }
        // A tile woken again while it is being relaxed can be taken by
        // another block before this one finishes, so two blocks may relax
        // it at once; the one that loaded older values must not overwrite
        // the other's.  Only risen voxels are written, by atomic maximum:
        // the field never falls.
        if (any) {
#pragma unroll
            for (int k = 0; k < kPer; k++) {
                const int x = x0 + lx[k], y = y0 + ly[k], z = z0 + lz[k];
                const int mv = sM[lx[k] + 1][ly[k] + 1][lz[k] + 1];
                if (x < J.nx && y < J.ny && z < J.nz && sval[k] != 0 && mv > mold[k])
                    atomicMax(J.M + d_lin(x, y, z, J.ny, J.nz), mv);
            }
        }
        // the field's stores are visible before any neighbour is queued
        __threadfence();
        __syncthreads();
        if (threadIdx.x < 7) {   // one lane per neighbour (6) and the tile itself: the pushes overlap
            const int q = threadIdx.x;
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
            if (nb >= 0) mmq_push(Q, nb, false);
            __threadfence();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // counters in batches of 16 tiles (the activation cap and the
            // stall watch need no finer grain)
            my_sweeps += sweeps;
            if (++my_acts == 16) {
                atomicAdd(Q.sweeps, my_sweeps);
                if ((long long)atomicAdd(Q.acts, 16ull) + 16 >= Q.max_acts) atomicExch(Q.stop, 1);
                my_acts = my_sweeps = 0;
            }
            atomicSub(Q.pending, 1);   // this tile is done; its pushes were counted first
            if (!got) next_g = mmq_take(Q, ticket, &next_seed);
        }
    }
}

}  // namespace

namespace {

// The queue schedule over the jobs' tiles (0 .. nt-1).
int mm_run_queue(ibip_ctx *ctx, int n, const std::vector<MMJob> &J, int nt, int rounds)
{
    cudaStream_t s = ctx->stream;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mm_queue, kThreads, 0) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return IBIP_ERR_CUDA;
    }
    int grid = ctx->sm_count * per_sm;
    if (grid > nt) grid = nt;
    const int cap = nt + grid + 64;
    // layout: jobs | head tail acts (u64) pending sweeps stop (int) | ring[cap] queued[nt]
    const size_t jb = ((size_t)n * sizeof(MMJob) + 255) & ~(size_t)255;
    const size_t cb = 64;
    char *w0 = (char *)ibip_scratch(ctx, SC_TILE, jb + cb + ((size_t)cap + nt) * sizeof(int));
    if (!w0) return IBIP_ERR_OOM;
    MMQ Q;
    Q.jobs = (MMJob *)w0; Q.njobs = n;
    unsigned long long *c64 = (unsigned long long *)(w0 + jb);
    Q.head = c64; Q.tail = c64 + 1; Q.acts = c64 + 2;
    int *c32 = (int *)(c64 + 3);
    Q.pending = c32; Q.sweeps = c32 + 1; Q.stop = c32 + 2;
    Q.ring = (int *)(w0 + jb + cb); Q.queued = Q.ring + cap;
    Q.cap = cap;
    Q.max_acts = (long long)(rounds < kQueueActsPerTile ? rounds : kQueueActsPerTile) * nt;
    ibip_prof_begin(ctx, IBIP_K_MAXIMIN);
    cudaMemcpyAsync((void *)Q.jobs, J.data(), (size_t)n * sizeof(MMJob), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(w0 + jb, 0, cb, s);                              // counters
    cudaMemsetAsync(Q.ring, 0xff, (size_t)cap * sizeof(int), s);     // -1: empty slots
    cudaMemsetAsync(Q.queued, 0, (size_t)nt * sizeof(int), s);
    for (int j = 0; j < n; j++) {
        k_mm_init<<<ctx->sm_count * 4, 256, 0, s>>>(J[j].val, J[j].nx, J[j].ny, J[j].nz, J[j].face, J[j].M);
        IBIP_LAUNCH(ctx);
    }
    k_mm_qseed<<<(nt + 255) / 256, 256, 0, s>>>(Q, nt);
    IBIP_LAUNCH(ctx);
    // a server slot issues it on its high-priority stream, beside the wide
    // kernels of the other jobs
    if (ctx->stream_inv) {
        if (cudaEventRecord(ctx->ev_inv, s) != cudaSuccess ||
            cudaStreamWaitEvent(ctx->stream_inv, ctx->ev_inv, 0) != cudaSuccess)
            return ibip_cuda_status(cudaGetLastError());
        s = ctx->stream_inv;
    }
    k_mm_queue<<<grid, kThreads, 0, s>>>(Q);
    IBIP_LAUNCH(ctx);
    int *h = (int *)ctx->h_pinned;
    // acts (u64), then pending, sweeps, stop (int)
    cudaMemcpyAsync(h, (const void *)Q.acts, sizeof(unsigned long long) + 3 * sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaError_t e = ibip_sync(ctx, s);
    ibip_prof_end(ctx, IBIP_K_MAXIMIN);
    if (e != cudaSuccess) return ibip_cuda_status(e);
    unsigned long long acts;
    memcpy(&acts, h, sizeof(acts));
    const int *c = h + 2;   // pending, sweeps, stop
    ctx->inv_stats[30] = 0;   // no rounds
    ctx->inv_stats[31] = (int64_t)acts;
    ctx->inv_stats[32] = c[1];
    return c[2] ? IBIP_ERR_NOT_CONVERGED : IBIP_OK;
}

// The round schedule as one ordinary launch per round, for contexts that
// share the device with other streams: short launches let the blocks of
// other streams' kernels (higher-priority ones first) in between rounds.
int mm_run_round_launches(ibip_ctx *ctx, const MMArgs &a, int rounds)
{
    cudaStream_t s = ctx->stream;
    int *h = (int *)ctx->h_pinned;
    // rounds in chunks; the next round's list size is read back after
    // each chunk (an empty round's launch returns at once).  A server
    // slot issues them on its high-priority stream: each round is a
    // short launch that would otherwise wait behind the wide kernels of
    // the other jobs.
    if (ctx->stream_inv) {
        if (cudaEventRecord(ctx->ev_inv, s) != cudaSuccess ||
            cudaStreamWaitEvent(ctx->stream_inv, ctx->ev_inv, 0) != cudaSuccess)
            return ibip_cuda_status(cudaGetLastError());
        s = ctx->stream_inv;
    }
    constexpr int kChunkRounds = 16;
    const int grid = ctx->sm_count;
    int r = 0;
    for (;;) {
        for (int q = 0; q < kChunkRounds && r < rounds; q++, r++) {
            k_mm_round<<<grid, kThreads, 0, s>>>(a, r);
            IBIP_LAUNCH(ctx);
        }
        cudaMemcpyAsync(h, a.count + r, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaError_t e = ibip_sync(ctx, s);
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

// The round schedule: one cooperative grid (one large image), or one
// launch per round in shared-device mode.
int mm_run_rounds(ibip_ctx *ctx, int n, const std::vector<MMJob> &J, int nt, int rounds)
{
    cudaStream_t s = ctx->stream;
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
    if (ctx->no_coop) return mm_run_round_launches(ctx, a, rounds);
    int *h = (int *)ctx->h_pinned;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mm_persistent, kThreads, 0) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return IBIP_ERR_CUDA;
    }
    int grid = ctx->sm_count * per_sm;
    if (grid > nt) grid = nt;
    void *args[] = {&a};
    cudaError_t e = cudaLaunchCooperativeKernel((void *)k_mm_persistent, grid, kThreads, args, 0, s);
    IBIP_LAUNCH(ctx);
    if (e != cudaSuccess) return ibip_cuda_status(e);
    cudaMemcpyAsync(h, a.status, 3 * sizeof(int), cudaMemcpyDeviceToHost, s);
    e = ibip_sync(ctx, s);
    ibip_prof_end(ctx, IBIP_K_MAXIMIN);
    if (e != cudaSuccess) return ibip_cuda_status(e);
    // diagnostics of the last propagation: rounds, tile activations, sweeps
    const int nr = h[0] < rounds ? h[0] : rounds, conv_flag = h[1], sweeps = h[2];
    int *hc = (int *)ctx->h_pinned;
    int64_t act = 0;
    for (int r0 = 0; r0 < nr; r0 += 8192) {
        const int c = nr - r0 < 8192 ? nr - r0 : 8192;
        cudaMemcpyAsync(hc, a.count + r0, (size_t)c * sizeof(int), cudaMemcpyDeviceToHost, s);
        if (ibip_sync(ctx, s) != cudaSuccess) return IBIP_ERR_CUDA;
        for (int q = 0; q < c; q++) act += hc[q];
    }
    ctx->inv_stats[30] = nr;
    ctx->inv_stats[31] = act;
    ctx->inv_stats[32] = sweeps;
    return conv_flag ? IBIP_ERR_NOT_CONVERGED : IBIP_OK;
}

}  // namespace

int ibip_maximin_multi(ibip_ctx *ctx, int n, const IbipMaximinJob *jobs, int max_rounds)
{
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
    // beside other streams' kernels (shared-device mode): rounds as short
    // launches; neither a cooperative grid, which needs every block
    // resident, nor the queue, whose resident blocks would hold the SMs
    // against other streams' kernels until the propagation ends
    if (!ctx->no_coop && (n > 1 || nt < kQueueTiles)) return mm_run_queue(ctx, n, J, nt, rounds);
    return mm_run_rounds(ctx, n, J, nt, rounds);
}

int ibip_maximin_launch(ibip_ctx *ctx, const int32_t *val, ibip_dims d, int face, int32_t *M, int max_rounds)
{
    IbipMaximinJob j{val, d, face, M};
    return ibip_maximin_multi(ctx, 1, &j, max_rounds);
}
