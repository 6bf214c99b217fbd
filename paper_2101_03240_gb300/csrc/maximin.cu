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
// GPU: tiles of 4 x 8 x 32 voxels (z contiguous) relax in shared memory until
// they stop changing; a tile that changed wakes its six neighbours for the
// next round; rounds repeat until no tile is awake.
#include "common.cuh"

namespace {

constexpr int TX = 4, TY = 8, TZ = 32;
constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
constexpr int kThreads = 256;
constexpr int kPer = TX * TY * TZ / kThreads;
constexpr int kInner = 96;

__device__ __forceinline__ int as_val(int v) { return v == -1 ? IBIP_INF32 : v; }

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

__global__ void __launch_bounds__(kThreads) k_mm_round(const int32_t *__restrict__ val, int nx, int ny, int nz,
                                                      int tx, int ty, int tz, int32_t *M, int *act, int round,
                                                      int *last)
{
    __shared__ int32_t sM[HX][HY][HZ];
    const int t = blockIdx.x;
    if (act[t] != round) return;
    const int bz = t % tz, by = (t / tz) % ty, bx = t / (tz * ty);
    const int x0 = bx * TX, y0 = by * TY, z0 = bz * TZ;
    // load tile + halo
    for (int i = threadIdx.x; i < HX * HY * HZ; i += kThreads) {
        int hz = i % HZ, hy = (i / HZ) % HY, hx = i / (HZ * HY);
        int x = x0 + hx - 1, y = y0 + hy - 1, z = z0 + hz - 1;
        int m = -1;
        if (x >= 0 && y >= 0 && z >= 0 && x < nx && y < ny && z < nz) m = M[d_lin(x, y, z, ny, nz)];
        sM[hx][hy][hz] = m;
    }
    int sval[kPer];
    int lx[kPer], ly[kPer], lz[kPer];
#pragma unroll
    for (int k = 0; k < kPer; k++) {
        int i = threadIdx.x + k * kThreads;
        lz[k] = i % TZ; ly[k] = (i / TZ) % TY; lx[k] = i / (TZ * TY);
        int x = x0 + lx[k], y = y0 + ly[k], z = z0 + lz[k];
        sval[k] = (x < nx && y < ny && z < nz) ? as_val(val[d_lin(x, y, z, ny, nz)]) : 0;
    }
    __syncthreads();
    bool any = false, conv = false;
    for (int it = 0; it < kInner; it++) {
        int ch = 0;
#pragma unroll
        for (int k = 0; k < kPer; k++) {
            if (sval[k] == 0) continue;
            int hx = lx[k] + 1, hy = ly[k] + 1, hz = lz[k] + 1;
            int b = max(max(max(sM[hx - 1][hy][hz], sM[hx + 1][hy][hz]), max(sM[hx][hy - 1][hz], sM[hx][hy + 1][hz])),
                        max(sM[hx][hy][hz - 1], sM[hx][hy][hz + 1]));
            int nv = min(b, sval[k]);
            if (nv > sM[hx][hy][hz]) { sM[hx][hy][hz] = nv; ch = 1; }
        }
        if (!__syncthreads_or(ch)) { conv = true; break; }
        any = true;
    }
    if (!any) return;
#pragma unroll
    for (int k = 0; k < kPer; k++) {
        int x = x0 + lx[k], y = y0 + ly[k], z = z0 + lz[k];
        if (x < nx && y < ny && z < nz && sval[k] != 0) M[d_lin(x, y, z, ny, nz)] = sM[lx[k] + 1][ly[k] + 1][lz[k] + 1];
    }
    if (threadIdx.x == 0) {
        const int nxt = round + 1;
        if (bx > 0) act[t - tz * ty] = nxt;
        if (bx < tx - 1) act[t + tz * ty] = nxt;
        if (by > 0) act[t - tz] = nxt;
        if (by < ty - 1) act[t + tz] = nxt;
        if (bz > 0) act[t - 1] = nxt;
        if (bz < tz - 1) act[t + 1] = nxt;
        if (!conv) act[t] = nxt;
        atomicMax(last, nxt);
    }
}

}  // namespace

int ibip_maximin_launch(ibip_ctx *ctx, const int32_t *val, ibip_dims d, int face, int32_t *M, int max_rounds)
{
    cudaStream_t s = ctx->stream;
    const int tx = (d.nx + TX - 1) / TX, ty = (d.ny + TY - 1) / TY, tz = (d.nz + TZ - 1) / TZ;
    const int nt = tx * ty * tz;
    int *act = (int *)ibip_scratch(ctx, SC_TILE, (size_t)nt * sizeof(int));
    int *small = (int *)ibip_scratch(ctx, SC_SMALL, kSmallBytes);
    if (!act || !small) return IBIP_ERR_OOM;
    int *last = small + 4;
    ibip_prof_begin(ctx, IBIP_K_MAXIMIN);
    cudaMemsetAsync(act, 0, (size_t)nt * sizeof(int), s);
    cudaMemsetAsync(last, 0, sizeof(int), s);
    k_mm_init<<<ctx->sm_count * 8, 256, 0, s>>>(val, d.nx, d.ny, d.nz, face, M);
    IBIP_LAUNCH(ctx);
    int *h = (int *)ctx->h_pinned;
    const int kBatch = 8;
    for (int r = 0; r < max_rounds; r += kBatch) {
        for (int q = r; q < r + kBatch; q++) {
            k_mm_round<<<nt, kThreads, 0, s>>>(val, d.nx, d.ny, d.nz, tx, ty, tz, M, act, q, last);
            IBIP_LAUNCH(ctx);
        }
        cudaMemcpyAsync(h, last, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return ibip_cuda_status(e);
        if (h[0] < r + kBatch) {   // no tile woken for the next round
            ibip_prof_end(ctx, IBIP_K_MAXIMIN);
            return IBIP_OK;
        }
    }
    ibip_prof_end(ctx, IBIP_K_MAXIMIN);
    return IBIP_ERR_NOT_CONVERGED;
}
