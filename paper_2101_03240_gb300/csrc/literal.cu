// literal.cu -- the invasion exactly as Section 2.1 prints it (the
// paper-literal rule of ibip_invade_literal):
//   candidates = the inlets plus their face neighbours; every candidate
//   holding the largest distance value is an insertion point of the step
//   (all tied maxima at once); a sphere of integer radius R = trunc(dt)
//   (footnote 1) is written, step number k, into every pore voxel within
//   distance R that no earlier step invaded; the insertion points join the
//   inlets and their value drops to zero.
//
// GPU design.  Each pore voxel is queued once, when it first becomes a
// candidate, into the list of its distance value ("bucket"; buckets are
// numbered by decreasing value and own consecutive ranges of one list array
// sized by a histogram).  A step takes the highest non-empty bucket, and
// every entry queued there before the step is an insertion point: the step
// consumes the bucket's whole pending range, stamps the spheres of all its
// points in parallel, then queues their uninvaded face neighbours (entries
// queued now are examined from the next step on, as in the definition).
// One persistent CTA of 1024 threads runs the steps, with the buckets'
// counters and a bitmap of non-empty buckets in shared memory (up to ~10k
// distinct values); spheres are written with fire-and-forget atomic minima,
// so a step never waits on a read of the sequence image.
#include <cooperative_groups.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kLT = 1024;                 // threads of the step kernel
constexpr size_t kLitSmem = 160 * 1024;   // bucket bookkeeping kept in shared memory up to this

struct Lit {
    int nx, ny, nz, inlet;
    int64_t N;
    const int32_t *dt2;
    int32_t *seq, *cstep, *step_r2, *step_count;
    int64_t cap, max_steps;
    int npore;
    uint32_t *queued;      // one bit per voxel: ever queued
    int32_t *list;         // [npore]: bucket b owns [bstart[b], bstart[b] + size of b)
    const int32_t *bstart; // [B]
    const int32_t *bval;   // [B] distance value of bucket b (decreasing in b)
    int32_t *tail;         // [B] entries queued so far
    int32_t *head;         // [B] entries consumed so far
    uint32_t *ne;          // [ceil(B / 32)] non-empty buckets
    const int32_t *incl;   // incl[v] = number of present values <= v (bucket of v = B - incl[v])
    int B, hasinf;
    int64_t *out;          // [0] steps, [1] status
};

__device__ __forceinline__ int bucket_of(const Lit &a, int v) { return a.hasinf ? 0 : a.B - __ldg(a.incl + v); }

// Bucket bookkeeping: in shared memory when the buckets fit (SMEM), else in
// the global arrays of Lit.
struct Book {
    int32_t *tail, *head;
    const int32_t *bstart, *bval;
    uint32_t *ne;
};

// queue voxel u if it is pore and was never queued
__device__ __forceinline__ void enqueue(const Lit &a, const Book &k, int64_t u)
{
    const int v = __ldg(a.dt2 + u);
    if (v == 0) return;
    const uint32_t bit = 1u << (u & 31);
    if (atomicOr(a.queued + (u >> 5), bit) & bit) return;
    const int b = bucket_of(a, v);
    const int pos = atomicAdd(k.tail + b, 1);
    a.list[k.bstart[b] + pos] = (int32_t)u;
    atomicOr(k.ne + (b >> 5), 1u << (b & 31));
}

__device__ __forceinline__ void coords(const Lit &a, uint32_t v, int &x, int &y, int &z)
{
    z = (int)(v % (uint32_t)a.nz);
    const uint32_t r = v / (uint32_t)a.nz;
    y = (int)(r % (uint32_t)a.ny);
    x = (int)(r / (uint32_t)a.ny);
}

// the inlet face and its face neighbours are the first candidates
__global__ void k_lit_seed(Lit a)
{
    const Book bk{a.tail, a.head, a.bstart, a.bval, a.ne};
    const int f = a.inlet, ax = f >> 1;
    const int n0 = ax == 0 ? a.ny : a.nx, n1 = ax == 2 ? a.ny : a.nz;   // the face's two extents
    const int fixed = (f & 1) ? (ax == 0 ? a.nx : ax == 1 ? a.ny : a.nz) - 1 : 0;
    const int64_t nf = (int64_t)n0 * n1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(i / n1), q = (int)(i % n1);
        int x, y, z;
        if (ax == 0) { x = fixed; y = p; z = q; }
        else if (ax == 1) { x = p; y = fixed; z = q; }
        else { x = p; y = q; z = fixed; }
        const int dx[7] = {0, -1, 1, 0, 0, 0, 0}, dy[7] = {0, 0, 0, -1, 1, 0, 0}, dz[7] = {0, 0, 0, 0, 0, -1, 1};
        for (int d = 0; d < 7; d++) {
            const int u0 = x + dx[d], u1 = y + dy[d], u2 = z + dz[d];
            if (u0 < 0 || u1 < 0 || u2 < 0 || u0 >= a.nx || u1 >= a.ny || u2 >= a.nz) continue;
            enqueue(a, bk, d_lin(u0, u1, u2, a.ny, a.nz));
        }
    }
}

// The steps.  During the run an uninvaded pore voxel holds INT32_MAX, so a
// sphere writes min(seq, k) with fire-and-forget atomics (steps only grow,
// so the minimum is the first step that covered the voxel); k_lit_final
// turns the remaining INT32_MAX back into -1.
template <bool SMEM>
__global__ void __launch_bounds__(kLT, 1) k_lit_steps(Lit a)
{
    extern __shared__ uint32_t s_lit[];
    __shared__ int s_b, s_h, s_n, s_stop;
    const int tid = threadIdx.x, lane = tid & 31;
    const int nw = (a.B + 31) >> 5;
    Book bk{a.tail, a.head, a.bstart, a.bval, a.ne};
    if (SMEM) {
        uint32_t *ne = s_lit;
        int32_t *t = (int32_t *)(s_lit + nw);
        for (int i = tid; i < nw; i += kLT) ne[i] = a.ne[i];
        for (int i = tid; i < a.B; i += kLT) {
            t[i] = a.tail[i];
            t[a.B + i] = a.head[i];
            t[2 * a.B + i] = a.bstart[i];
            t[3 * a.B + i] = a.bval[i];
        }
        bk = Book{t, t + a.B, t + 2 * a.B, t + 3 * a.B, ne};
        __syncthreads();
    }
    int64_t k = 0;
    for (;;) {
        if (tid < 32) {
            // highest non-empty bucket: first set bit of the bitmap
            int b = -1;
            for (int w0 = 0; w0 < nw && b < 0; w0 += 32) {
                const int w = w0 + lane;
                const uint32_t m = w < nw ? *(volatile uint32_t *)(bk.ne + w) : 0u;
                const unsigned bal = __ballot_sync(0xffffffffu, m != 0u);
                if (bal) {
                    const int l = __ffs(bal) - 1;
                    const uint32_t ml = __shfl_sync(0xffffffffu, m, l);
                    b = ((w0 + l) << 5) + __ffs(ml) - 1;
                }
            }
            if (lane == 0) {
                int stop = 0;
                if (b < 0) stop = 1;
                else if (k >= a.max_steps) stop = 2;
                else if (k >= a.npore) stop = 3;   // every step consumes a queued voxel: cannot happen
                s_stop = stop;
                if (!stop) {
                    const int h = bk.head[b], t = *(volatile int *)(bk.tail + b);
                    bk.head[b] = t;
                    // consumed: the bucket is empty until this step queues into it
                    atomicAnd(bk.ne + (b >> 5), ~(1u << (b & 31)));
                    s_b = b; s_h = h; s_n = t - h;
                }
            }
        }
        __syncthreads();
        if (s_stop) break;
        k++;
        const int b = s_b, n = s_n;
        const int32_t *pts = a.list + bk.bstart[b] + s_h;
        const int v = bk.bval[b];
        const int R = d_isqrt(v);                              // trunc(dt)
        const int64_t RR = (int64_t)R * R;
        const int Re = min(R, max(a.nx, max(a.ny, a.nz)));     // reach inside the image
        const int side = 2 * Re + 1;
        const int64_t rows = (int64_t)side * side;
        // spheres: one item per (point, row of the bounding square)
        for (int64_t it = tid; it < (int64_t)n * rows; it += kLT) {
            const int q = (int)(it / rows);
            const int r = (int)(it - (int64_t)q * rows);
            const int ddx = r / side - Re, ddy = r % side - Re;
            const int64_t rem = RR - (int64_t)ddx * ddx - (int64_t)ddy * ddy;
            if (rem < 0) continue;
            int cx, cy, cz;
            coords(a, (uint32_t)pts[q], cx, cy, cz);
            const int x = cx + ddx, y = cy + ddy;
            if (x < 0 || y < 0 || x >= a.nx || y >= a.ny) continue;
            const int hz = d_isqrt((int)min(rem, (int64_t)IBIP_INF32));
            const int z0 = max(0, cz - hz), z1 = min(a.nz - 1, cz + hz);
            int32_t *row = a.seq + d_lin(x, y, 0, a.ny, a.nz);
            for (int z = z0; z <= z1; z++) atomicMin(row + z, (int32_t)k);
        }
        // the points join the inlets: mark them, queue their neighbours
        for (int64_t it = tid; it < (int64_t)n * 6; it += kLT) {
            const int q = (int)(it / 6), d = (int)(it - (int64_t)q * 6);
            const uint32_t c = (uint32_t)pts[q];
            int x, y, z;
            coords(a, c, x, y, z);
            if (d == 0) a.cstep[c] = (int32_t)k;
            x += d == 0 ? -1 : d == 1 ? 1 : 0;
            y += d == 2 ? -1 : d == 3 ? 1 : 0;
            z += d == 4 ? -1 : d == 5 ? 1 : 0;
            if (x < 0 || y < 0 || z < 0 || x >= a.nx || y >= a.ny || z >= a.nz) continue;
            enqueue(a, bk, d_lin(x, y, z, a.ny, a.nz));
        }
        if (tid == 0 && k <= a.cap) {
            a.step_r2[k - 1] = (int32_t)RR;
            a.step_count[k - 1] = n;
        }
        __syncthreads();
    }
    if (tid == 0) {
        a.out[0] = k;
        a.out[1] = s_stop == 2 ? IBIP_ERR_STEP_LIMIT : (s_stop == 3 ? IBIP_ERR_BOUNDS : IBIP_OK);
    }
}

// The same steps on a thread-block cluster: CTA 0 keeps the bucket
// bookkeeping in its shared memory and picks each step's bucket; every CTA
// of the cluster stamps a share of the spheres and queues a share of the
// neighbours, reaching CTA 0's counters through distributed shared memory.
// Two cluster barriers per step: after the pick, and after the step's work.
// List entries written by other SMs are read with L2-coherent loads.
__device__ __forceinline__ void lit_cluster_run(const Lit &a)
{
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ uint32_t s_litc[];
    __shared__ int s_step[6];   // CTA 0: bucket, first entry, count, stop, list start, value
    __shared__ int s_loc[6];    // every CTA: its copy of CTA 0's s_step
    const unsigned rank = cl.block_rank(), ncta = cl.num_blocks();
    const int tid = threadIdx.x, lane = tid & 31;
    const int gtid = (int)rank * kLT + tid, gstride = (int)ncta * kLT;
    const int nw = (a.B + 31) >> 5;
    uint32_t *const s_lit = s_litc;
    uint32_t *ne0 = cl.map_shared_rank(s_lit, 0);
    int32_t *t0 = (int32_t *)(ne0 + nw);
    const Book bk0{t0, t0 + a.B, t0 + 2 * a.B, t0 + 3 * a.B, ne0};   // CTA 0's book, from any CTA
    const int *step0 = cl.map_shared_rank(s_step, 0);
    if (rank == 0) {
        int32_t *t = (int32_t *)(s_lit + nw);
        for (int i = tid; i < nw; i += kLT) s_lit[i] = a.ne[i];
        for (int i = tid; i < a.B; i += kLT) {
            t[i] = a.tail[i];
            t[a.B + i] = a.head[i];
            t[2 * a.B + i] = a.bstart[i];
            t[3 * a.B + i] = a.bval[i];
        }
    }
    cl.sync();
    int64_t k = 0;
    for (;;) {
        if (rank == 0 && tid < 32) {
            int b = -1;
            for (int w0 = 0; w0 < nw && b < 0; w0 += 32) {
                const int w = w0 + lane;
                const uint32_t m = w < nw ? *(volatile uint32_t *)(s_lit + w) : 0u;
                const unsigned bal = __ballot_sync(0xffffffffu, m != 0u);
                if (bal) {
                    const int l = __ffs(bal) - 1;
                    const uint32_t ml = __shfl_sync(0xffffffffu, m, l);
                    b = ((w0 + l) << 5) + __ffs(ml) - 1;
                }
            }
            if (lane == 0) {
                int stop = 0;
                if (b < 0) stop = 1;
                else if (k >= a.max_steps) stop = 2;
                else if (k >= a.npore) stop = 3;
                s_step[3] = stop;
                if (!stop) {
                    int32_t *t = (int32_t *)(s_lit + nw);
                    const int h = t[a.B + b], tl = *(volatile int *)(t + b);
                    t[a.B + b] = tl;
                    atomicAnd(s_lit + (b >> 5), ~(1u << (b & 31)));
                    s_step[0] = b; s_step[1] = h; s_step[2] = tl - h;
                    s_step[4] = t[2 * a.B + b]; s_step[5] = t[3 * a.B + b];
                }
            }
        }
        cl.sync();
        if (tid < 6) s_loc[tid] = step0[tid];
        __syncthreads();
        if (s_loc[3]) break;
        k++;
        const int n = s_loc[2];
        const int32_t *pts = a.list + s_loc[4] + s_loc[1];
        const int v = s_loc[5];
        const int R = d_isqrt(v);
        const int64_t RR = (int64_t)R * R;
        const int Re = min(R, max(a.nx, max(a.ny, a.nz)));
        const int side = 2 * Re + 1;
        const int64_t rows = (int64_t)side * side;
        for (int64_t it = gtid; it < (int64_t)n * rows; it += gstride) {
            const int q = (int)(it / rows);
            const int r = (int)(it - (int64_t)q * rows);
            const int ddx = r / side - Re, ddy = r % side - Re;
            const int64_t rem = RR - (int64_t)ddx * ddx - (int64_t)ddy * ddy;
            if (rem < 0) continue;
            int cx, cy, cz;
            coords(a, (uint32_t)__ldcg(pts + q), cx, cy, cz);
            const int x = cx + ddx, y = cy + ddy;
            if (x < 0 || y < 0 || x >= a.nx || y >= a.ny) continue;
            const int hz = d_isqrt((int)min(rem, (int64_t)IBIP_INF32));
            const int z0 = max(0, cz - hz), z1 = min(a.nz - 1, cz + hz);
            int32_t *row = a.seq + d_lin(x, y, 0, a.ny, a.nz);
            for (int z = z0; z <= z1; z++) atomicMin(row + z, (int32_t)k);
        }
        for (int64_t it = gtid; it < (int64_t)n * 6; it += gstride) {
            const int q = (int)(it / 6), d = (int)(it - (int64_t)q * 6);
            const uint32_t c = (uint32_t)__ldcg(pts + q);
            int x, y, z;
            coords(a, c, x, y, z);
            if (d == 0) a.cstep[c] = (int32_t)k;
            x += d == 0 ? -1 : d == 1 ? 1 : 0;
            y += d == 2 ? -1 : d == 3 ? 1 : 0;
            z += d == 4 ? -1 : d == 5 ? 1 : 0;
            if (x < 0 || y < 0 || z < 0 || x >= a.nx || y >= a.ny || z >= a.nz) continue;
            enqueue(a, bk0, d_lin(x, y, z, a.ny, a.nz));
        }
        if (rank == 0 && tid == 0 && k <= a.cap) {
            a.step_r2[k - 1] = (int32_t)RR;
            a.step_count[k - 1] = n;
        }
        cl.sync();
    }
    if (rank == 0 && tid == 0) {
        a.out[0] = k;
        a.out[1] = s_loc[3] == 2 ? IBIP_ERR_STEP_LIMIT : (s_loc[3] == 3 ? IBIP_ERR_BOUNDS : IBIP_OK);
    }
    cl.sync();   // CTA 0's shared memory stays alive until every CTA has read it
}

__global__ void __launch_bounds__(kLT, 1) k_lit_cluster(Lit a) { lit_cluster_run(a); }

// Many images, one cluster each: cluster c (blocks c * size .. c * size +
// size - 1) runs the steps of image jobs[c] from start to end.
__global__ void __launch_bounds__(kLT, 1) k_lit_cluster_b(const Lit *__restrict__ jobs)
{
    cg::cluster_group cl = cg::this_cluster();
    const Lit a = jobs[blockIdx.x / cl.num_blocks()];
    lit_cluster_run(a);
}

// uninvaded voxels back to -1, every image of a batch (blockIdx.x = image)
__global__ void k_lit_final_b(const Lit *__restrict__ jobs)
{
    const Lit &a = jobs[blockIdx.x];
    for (int64_t v = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; v < a.N; v += (int64_t)gridDim.y * blockDim.x)
        if (a.seq[v] == IBIP_INF32) a.seq[v] = -1;
}

__global__ void k_lit_final(int32_t *seq, int64_t N)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
        if (seq[v] == IBIP_INF32) seq[v] = -1;
}

__global__ void k_lit_init(const int32_t *__restrict__ dt2, int64_t N, int32_t *seq, int32_t *cstep)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        seq[v] = dt2[v] ? IBIP_INF32 : 0;   // uninvaded pore: see k_lit_steps
        cstep[v] = 0;
    }
}

// presence of each distance value among pore voxels
__global__ void k_lit_presence(const int32_t *__restrict__ dt2, int64_t N, int32_t *pres)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        const int d = dt2[v];
        if (d > 0 && d != IBIP_INF32 && pres[d] == 0) pres[d] = 1;
    }
}

// voxels per bucket
__global__ void k_lit_hist(const int32_t *__restrict__ dt2, int64_t N, const int32_t *incl, int B, int hasinf,
                           int32_t *cnt)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        const int d = dt2[v];
        if (d == 0) continue;
        atomicAdd(cnt + (hasinf ? 0 : B - incl[d]), 1);
    }
}

// value of each bucket
__global__ void k_lit_bval(const int32_t *incl, int maxd, int B, int hasinf, int32_t *bval)
{
    if (hasinf) {
        if (blockIdx.x == 0 && threadIdx.x == 0) bval[0] = IBIP_INF32;
        return;
    }
    for (int v = blockIdx.x * blockDim.x + threadIdx.x + 1; v <= maxd; v += gridDim.x * blockDim.x)
        if (incl[v] != incl[v - 1]) bval[B - incl[v]] = v;
}

}  // namespace

// Largest cluster (16, 8, 4 or 2 CTAs of 1024 threads with `book` bytes of
// shared memory) the device can place; 0 if none.
static int lit_cluster_size(size_t book)
{
    cudaFuncSetAttribute(k_lit_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLitSmem);
    cudaFuncSetAttribute(k_lit_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    for (int cs = 16; cs >= 2; cs /= 2) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(kLT);
        cfg.dynamicSmemBytes = book;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_lit_cluster, &cfg) == cudaSuccess && n > 0) return cs;
        cudaGetLastError();
    }
    return 0;
}

int ibip_literal_run(ibip_ctx *ctx, const int32_t *dt2, ibip_dims d, int inlet, int64_t max_steps, int32_t *seq,
                     int32_t *cstep, int32_t *step_r2, int32_t *step_count, int64_t cap, int64_t *h_out)
{
    cudaStream_t s = ctx->stream;
    const int64_t N = nvox(d);
    const int gs = ctx->sm_count * 8;
    int *stats = (int *)ibip_scratch(ctx, SC_SMALL, kSmallBytes);
    if (!stats) return IBIP_ERR_OOM;
    int *h = (int *)ctx->h_pinned;
    ibip_prof_begin(ctx, IBIP_K_RANK);
    // largest finite value, pore count, whether values are infinite
    cudaMemsetAsync(stats, 0, 3 * sizeof(int), s);
    ibip_stats_launch(ctx, dt2, N, stats);
    cudaMemcpyAsync(h, stats, 3 * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (ibip_sync(ctx, s) != cudaSuccess) return IBIP_ERR_CUDA;
    const int maxd = h[0], npore = h[1], hasinf = h[2];
    k_lit_init<<<gs, 256, 0, s>>>(dt2, N, seq, cstep);
    IBIP_LAUNCH(ctx);
    if (npore == 0) {
        ibip_prof_end(ctx, IBIP_K_RANK);
        h_out[0] = 0;
        h_out[1] = IBIP_OK;
        return ibip_cuda_status(ibip_sync(ctx, s));
    }
    // buckets: distinct values in decreasing order
    int32_t *incl = (int32_t *)ibip_scratch(ctx, SC_PRES, ((size_t)maxd + 2) * sizeof(int32_t));
    if (!incl) return IBIP_ERR_OOM;
    int B = 1;
    if (!hasinf) {
        cudaMemsetAsync(incl, 0, ((size_t)maxd + 1) * sizeof(int32_t), s);
        k_lit_presence<<<gs, 256, 0, s>>>(dt2, N, incl);
        IBIP_LAUNCH(ctx);
        int st = ibip_scan_incl_i32(ctx, incl, incl, (int64_t)maxd + 1);
        if (st) return st;
        cudaMemcpyAsync(h, incl + maxd, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (ibip_sync(ctx, s) != cudaSuccess) return IBIP_ERR_CUDA;
        B = h[0];
    }
    const int nw = (B + 31) / 32;
    // one arena: list | bstart | bval | tail | head | cnt | ne | queued | out
    const size_t planes = ((size_t)N + 31) / 32;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t o_list = 0, o_bstart = o_list + up((size_t)npore * 4), o_bval = o_bstart + up((size_t)B * 4),
                 o_tail = o_bval + up((size_t)B * 4), o_head = o_tail + up((size_t)B * 4),
                 o_cnt = o_head + up((size_t)B * 4), o_ne = o_cnt + up((size_t)B * 4),
                 o_q = o_ne + up((size_t)nw * 4), o_out = o_q + up(planes * 4), total = o_out + up(64);
    char *w = (char *)ibip_scratch(ctx, SC_LIT, total);
    if (!w) return IBIP_ERR_OOM;
    Lit a;
    a.nx = d.nx; a.ny = d.ny; a.nz = d.nz; a.inlet = inlet; a.N = N;
    a.dt2 = dt2; a.seq = seq; a.cstep = cstep; a.step_r2 = step_r2; a.step_count = step_count;
    a.cap = cap; a.max_steps = max_steps; a.npore = npore;
    a.list = (int32_t *)(w + o_list);
    a.bstart = (const int32_t *)(w + o_bstart);
    a.bval = (const int32_t *)(w + o_bval);
    a.tail = (int32_t *)(w + o_tail);
    a.head = (int32_t *)(w + o_head);
    a.ne = (uint32_t *)(w + o_ne);
    a.queued = (uint32_t *)(w + o_q);
    a.incl = incl;
    a.B = B; a.hasinf = hasinf;
    a.out = (int64_t *)(w + o_out);
    int32_t *cnt = (int32_t *)(w + o_cnt);
    // tail, head, cnt and ne are contiguous: clear them at once, and the plane
    cudaMemsetAsync(w + o_tail, 0, o_q - o_tail, s);
    cudaMemsetAsync(w + o_q, 0, planes * 4, s);
    k_lit_hist<<<gs, 256, 0, s>>>(dt2, N, incl, B, hasinf, cnt);
    IBIP_LAUNCH(ctx);
    int st = ibip_scan_excl_i32(ctx, cnt, (int32_t *)a.bstart, B);
    if (st) return st;
    k_lit_bval<<<std::max(1, std::min(gs, (maxd + 255) / 256)), 256, 0, s>>>(incl, maxd, B, hasinf,
                                                                             (int32_t *)a.bval);
    IBIP_LAUNCH(ctx);
    const int nface = (inlet >> 1) == 0 ? d.ny * d.nz : (inlet >> 1) == 1 ? d.nx * d.nz : d.nx * d.ny;
    k_lit_seed<<<std::max(1, std::min(gs, (nface + 255) / 256)), 256, 0, s>>>(a);
    IBIP_LAUNCH(ctx);
    ibip_prof_end(ctx, IBIP_K_RANK);
    ibip_prof_begin(ctx, IBIP_K_INVADE);
    const size_t book = (size_t)nw * 4 + (size_t)B * 16;
    const int cs = book <= kLitSmem ? lit_cluster_size(book) : 0;
    if (cs > 1) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(kLT);
        cfg.dynamicSmemBytes = book;
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t e = cudaLaunchKernelEx(&cfg, k_lit_cluster, a);
        if (e != cudaSuccess) return ibip_cuda_status(e);
    } else if (book <= kLitSmem) {
        cudaFuncSetAttribute(k_lit_steps<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLitSmem);
        k_lit_steps<true><<<1, kLT, book, s>>>(a);
    } else {
        k_lit_steps<false><<<1, kLT, 0, s>>>(a);
    }
    IBIP_LAUNCH(ctx);
    k_lit_final<<<gs, 256, 0, s>>>(seq, N);
    IBIP_LAUNCH(ctx);
    ibip_prof_end(ctx, IBIP_K_INVADE);
    int64_t *ho = (int64_t *)ctx->h_pinned;
    cudaMemcpyAsync(ho, a.out, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaError_t e = ibip_sync(ctx, s);
    if (e != cudaSuccess) return ibip_cuda_status(e);
    h_out[0] = ho[0];
    h_out[1] = ho[1];
    return IBIP_OK;
}

// ---------------------------------------------------------------- batched --
// Many images, each on a thread-block cluster of its own, in one launch.
// The set-up of every image (statistics, buckets, the first candidates) runs
// first, each image's lists and counters carved from one pooled buffer with
// room for its largest possible bucket count; then one launch of
// k_lit_cluster_b with one cluster per image that has pore voxels.  Each
// cluster runs exactly the steps of the one-image kernel, so results equal
// the one-image calls bit for bit.

namespace {

// Whether clusters of cs CTAs with `book` bytes of shared memory can be
// placed at all.
bool lit_cluster_fits(int cs, size_t book)
{
    cudaFuncSetAttribute(k_lit_cluster_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLitSmem);
    cudaFuncSetAttribute(k_lit_cluster_b, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(kLT);
    cfg.dynamicSmemBytes = book;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_lit_cluster_b, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n > 0;
}

struct LitBatchSizes {
    size_t incl, list, b4, ne, q, total;
};

// upper bounds of one image's pooled arrays (buckets bounded by the
// largest possible squared distance of its box)
LitBatchSizes lit_batch_sizes(ibip_dims d)
{
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const int64_t N = nvox(d);
    const int64_t maxd = (int64_t)(d.nx - 1) * (d.nx - 1) + (int64_t)(d.ny - 1) * (d.ny - 1) +
                         (int64_t)(d.nz - 1) * (d.nz - 1) + 1;
    LitBatchSizes z;
    z.incl = up((size_t)(maxd + 2) * 4);
    z.list = up((size_t)N * 4);
    z.b4 = up((size_t)(maxd + 2) * 4);
    z.ne = up((size_t)((maxd + 33) / 32) * 4);
    z.q = up((size_t)((N + 31) / 32) * 4);
    // incl | list | bstart | bval | tail | head | cnt | ne | queued
    z.total = z.incl + z.list + 5 * z.b4 + z.ne + z.q;
    return z;
}

// every image through the one-image path
int lit_each(ibip_ctx *ctx, int n, IbipLitItem *items)
{
    for (int j = 0; j < n; j++) {
        IbipLitItem &it = items[j];
        int64_t out[2] = {0, 0};
        const int st = ibip_literal_run(ctx, it.dt2, it.d, it.inlet, it.max_steps, it.seq, it.cstep, it.step_r2,
                                        it.step_count, it.cap, out);
        if (st) return st;
        it.n_steps = out[0];
        it.status = (int)out[1];
    }
    return IBIP_OK;
}

// One run of the whole batch with clusters of (at most) cs CTAs: fewer
// when the device cannot place cs with the batch's bucket bookkeeping, and
// the one-image path per image when some image's bookkeeping exceeds shared
// memory.  *cs_used gets the cluster size run (0: one image at a time).
int lit_batch_once(ibip_ctx *ctx, int n, IbipLitItem *items, int cs, int *cs_used)
{
    cudaStream_t s = ctx->stream;
    const int gs = ctx->sm_count * 8;
    *cs_used = 0;
    if (cs == 0) return lit_each(ctx, n, items);
    // job table | statistics (4 ints per image) | outputs (8 int64 per image)
    const size_t jt = ((size_t)n * sizeof(Lit) + 255) & ~(size_t)255;
    const size_t st_b = ((size_t)n * 4 * sizeof(int) + 255) & ~(size_t)255;
    char *jw = (char *)ibip_scratch(ctx, SC_LITJ, jt + st_b + (size_t)n * 8 * sizeof(int64_t));
    if (!jw) return IBIP_ERR_OOM;
    Lit *djobs = (Lit *)jw;
    int *stats = (int *)(jw + jt);
    int64_t *outs = (int64_t *)(jw + jt + st_b);
    std::vector<size_t> off(n + 1, 0);
    for (int j = 0; j < n; j++) off[j + 1] = off[j] + lit_batch_sizes(items[j].d).total;
    char *pool = (char *)ibip_scratch(ctx, SC_LITB, off[n]);
    if (!pool) return IBIP_ERR_OOM;
    ibip_prof_begin(ctx, IBIP_K_RANK);
    // statistics of every image, one read-back
    cudaMemsetAsync(stats, 0, (size_t)n * 4 * sizeof(int), s);
    cudaMemsetAsync(outs, 0, (size_t)n * 8 * sizeof(int64_t), s);
    for (int j = 0; j < n; j++) {
        ibip_stats_launch(ctx, items[j].dt2, nvox(items[j].d), stats + 4 * j);
    }
    int *h = (int *)ctx->h_pinned;   // n <= 4096: 4n ints fit the pinned buffer
    cudaMemcpyAsync(h, stats, (size_t)n * 4 * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (ibip_sync(ctx, s) != cudaSuccess) return IBIP_ERR_CUDA;
    std::vector<int> maxd(n), npore(n), hasinf(n), B(n, 1);
    for (int j = 0; j < n; j++) { maxd[j] = h[4 * j]; npore[j] = h[4 * j + 1]; hasinf[j] = h[4 * j + 2]; }
    // present distance values, scanned: the bucket count of every image
    std::vector<int32_t *> incl(n);
    for (int j = 0; j < n; j++) {
        const IbipLitItem &it = items[j];
        const int64_t N = nvox(it.d);
        incl[j] = (int32_t *)(pool + off[j]);
        k_lit_init<<<gs, 256, 0, s>>>(it.dt2, N, it.seq, it.cstep);
        IBIP_LAUNCH(ctx);
        if (npore[j] == 0 || hasinf[j]) continue;
        cudaMemsetAsync(incl[j], 0, ((size_t)maxd[j] + 1) * sizeof(int32_t), s);
        k_lit_presence<<<gs, 256, 0, s>>>(it.dt2, N, incl[j]);
        IBIP_LAUNCH(ctx);
        const int st = ibip_scan_incl_i32(ctx, incl[j], incl[j], (int64_t)maxd[j] + 1);
        if (st) return st;
        cudaMemcpyAsync(h + j, incl[j] + maxd[j], sizeof(int), cudaMemcpyDeviceToHost, s);
    }
    if (ibip_sync(ctx, s) != cudaSuccess) return IBIP_ERR_CUDA;
    size_t book = 0;
    for (int j = 0; j < n; j++) {
        if (npore[j] > 0 && !hasinf[j]) B[j] = h[j];
        if (npore[j] > 0) book = std::max(book, (size_t)((B[j] + 31) / 32) * 4 + (size_t)B[j] * 16);
    }
    if (book > kLitSmem) return lit_each(ctx, n, items);   // bookkeeping too large for shared memory
    while (cs > 1 && !lit_cluster_fits(cs, book)) cs /= 2;
    if (!lit_cluster_fits(cs, book)) return lit_each(ctx, n, items);
    *cs_used = cs;
    // buckets, first candidates and the job table
    std::vector<Lit> jobs;
    std::vector<int> which;
    for (int j = 0; j < n; j++) {
        IbipLitItem &it = items[j];
        it.n_steps = 0;
        it.status = IBIP_OK;
        if (npore[j] == 0) continue;
        const LitBatchSizes z = lit_batch_sizes(it.d);
        char *w = pool + off[j] + z.incl;
        const int64_t N = nvox(it.d);
        const int nw = (B[j] + 31) / 32;
        Lit a;
        a.nx = it.d.nx; a.ny = it.d.ny; a.nz = it.d.nz; a.inlet = it.inlet; a.N = N;
        a.dt2 = it.dt2; a.seq = it.seq; a.cstep = it.cstep; a.step_r2 = it.step_r2; a.step_count = it.step_count;
        a.cap = it.cap; a.max_steps = it.max_steps; a.npore = npore[j];
        a.list = (int32_t *)w;
        a.bstart = (const int32_t *)(w + z.list);
        a.bval = (const int32_t *)(w + z.list + z.b4);
        a.tail = (int32_t *)(w + z.list + 2 * z.b4);
        a.head = (int32_t *)(w + z.list + 3 * z.b4);
        int32_t *cnt = (int32_t *)(w + z.list + 4 * z.b4);
        a.ne = (uint32_t *)(w + z.list + 5 * z.b4);
        a.queued = (uint32_t *)(w + z.list + 5 * z.b4 + z.ne);
        a.incl = incl[j];
        a.B = B[j]; a.hasinf = hasinf[j];
        a.out = outs + 8 * jobs.size();
        // tail, head, cnt, ne and the queued plane are contiguous
        cudaMemsetAsync(a.tail, 0, 3 * z.b4 + z.ne + z.q, s);
        k_lit_hist<<<gs, 256, 0, s>>>(it.dt2, N, incl[j], B[j], hasinf[j], cnt);
        IBIP_LAUNCH(ctx);
        const int st = ibip_scan_excl_i32(ctx, cnt, (int32_t *)a.bstart, B[j]);
        if (st) return st;
        k_lit_bval<<<std::max(1, std::min(gs, (maxd[j] + 255) / 256)), 256, 0, s>>>(incl[j], maxd[j], B[j], hasinf[j],
                                                                                    (int32_t *)a.bval);
        IBIP_LAUNCH(ctx);
        const int f = it.inlet >> 1;
        const int nface = f == 0 ? it.d.ny * it.d.nz : f == 1 ? it.d.nx * it.d.nz : it.d.nx * it.d.ny;
        k_lit_seed<<<std::max(1, std::min(gs, (nface + 255) / 256)), 256, 0, s>>>(a);
        IBIP_LAUNCH(ctx);
        (void)nw;
        jobs.push_back(a);
        which.push_back(j);
    }
    ibip_prof_end(ctx, IBIP_K_RANK);
    if (jobs.empty()) return ibip_cuda_status(ibip_sync(ctx, s));
    const int nj = (int)jobs.size();
    cudaMemcpyAsync(djobs, jobs.data(), (size_t)nj * sizeof(Lit), cudaMemcpyHostToDevice, s);
    ibip_prof_begin(ctx, IBIP_K_INVADE);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(nj * cs));
    cfg.blockDim = dim3(kLT);
    cfg.dynamicSmemBytes = book;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_lit_cluster_b, (const Lit *)djobs);
    if (e != cudaSuccess) return ibip_cuda_status(e);
    IBIP_LAUNCH(ctx);
    k_lit_final_b<<<dim3((unsigned)nj, 16), 256, 0, s>>>(djobs);
    IBIP_LAUNCH(ctx);
    ibip_prof_end(ctx, IBIP_K_INVADE);
    int64_t *ho = (int64_t *)ctx->h_pinned;   // 8 int64 per job: nj <= 1024 per read-back
    for (int c0 = 0; c0 < nj; c0 += 1024) {
        const int c = std::min(1024, nj - c0);
        cudaMemcpyAsync(ho, outs + 8 * (size_t)c0, (size_t)c * 8 * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        e = ibip_sync(ctx, s);
        if (e != cudaSuccess) return ibip_cuda_status(e);
        for (int q = 0; q < c; q++) {
            IbipLitItem &it = items[which[c0 + q]];
            it.n_steps = ho[8 * q];
            it.status = (int)ho[8 * q + 1];
        }
    }
    return IBIP_OK;
}

}  // namespace

int ibip_literal_batch_run(ibip_ctx *ctx, int n, IbipLitItem *items, int cluster, int *h_cluster)
{
    static const int kCand[] = {1, 2, 4, 8, 16};
    int used = 0;
    int cs = cluster;
    if (cs <= 0) {
        int64_t vox = 0;
        for (int j = 0; j < n; j++) vox += nvox(items[j].d);
        int p2 = 0;
        while (p2 < 62 && ((int64_t)1 << p2) < vox) p2++;
        const std::string key = "lit_b:" + std::to_string(n) + ":" + std::to_string(p2) + ":" +
                                std::to_string(ctx->sm_count);
        int t = 0;
        if (ctx->autotune && ibip_tune_get(key, &t)) {
            cs = t;
        } else if (ctx->autotune) {
            // time every cluster size on this batch; the runs give identical
            // results, the last one's stay in the outputs
            double best = 1e30;
            int best_cs = 0;
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            for (int c : kCand) {
                cudaEventRecord(e0, ctx->stream);
                const int st = lit_batch_once(ctx, n, items, c, &used);
                cudaEventRecord(e1, ctx->stream);
                if (st) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return st;
                }
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (used == c && ms < best) { best = ms; best_cs = c; }
                if (used != c) break;   // larger clusters cannot be placed either
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            ibip_tune_put(key, best_cs, best * 1e3, ctx->tune_path);
            if (h_cluster) *h_cluster = best_cs;
            return IBIP_OK;
        } else {
            // enough clusters to fill the SMs: more CTAs per image when few
            cs = 1;
            while (cs < 8 && (int64_t)n * cs * 2 <= ctx->sm_count) cs *= 2;
        }
    }
    const int st = lit_batch_once(ctx, n, items, cs, &used);
    if (h_cluster) *h_cluster = used;
    return st;
}
