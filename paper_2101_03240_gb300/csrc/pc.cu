// pc.cu -- saturation and capillary pressure per step (Sections 2.2.1 and
// 2.2.2; Washburn relation as written in Section 2.4.1), plus the helpers
// trapping and opening need: thresholding against seq, re-ranking and
// level counts.
#include "common.cuh"

namespace {

// cnt[s] += 1 for 1 <= seq <= K (warp-aggregated: equal values in a warp
// cost one atomic); npore counts seq != 0.
__global__ void k_hist_seq(const int32_t *__restrict__ seq, int64_t N, int64_t K, int32_t *cnt, int *npore)
{
    const int lane = threadIdx.x & 31;
    int np = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < N; base += stride) {
        int64_t v = base + threadIdx.x;
        int s = v < N ? seq[v] : 0;
        np += s != 0;
        int key = (s >= 1 && s <= K) ? s : 0;
        unsigned peers = __match_any_sync(0xffffffffu, key);
        if (key && lane == __ffs(peers) - 1) atomicAdd(cnt + key, __popc(peers));
    }
    for (int o = 16; o; o >>= 1) np += __shfl_xor_sync(0xffffffffu, np, o);
    if (lane == 0 && np) atomicAdd(npore, np);
}

__global__ void k_pc(const int32_t *__restrict__ cum, const int *npore, const int32_t *__restrict__ r2, int64_t K,
                     double voxel, double num, float *S, float *Pc)
{
    const double np = (double)*npore;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K; k += (int64_t)gridDim.x * blockDim.x) {
        if (S) S[k] = (float)((double)cum[k + 1] / np);
        if (Pc) Pc[k] = (float)(num / (sqrt((double)r2[k]) * voxel));
    }
}

__global__ void k_sat(const int32_t *__restrict__ seq, int64_t N, int64_t K, const float *__restrict__ S, float *out)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        int s = seq[v];
        out[v] = (s >= 1 && s <= K) ? S[s - 1] : __int_as_float(0x7f800000);
    }
}

__global__ void k_max_seq(const int32_t *__restrict__ seq, int64_t N, int *mx)
{
    int m = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
        m = max(m, seq[v]);
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(mx, m);
}

// trapped iff invaded and the widest-path value from the outlet is below the
// voxel's own step
__global__ void k_trap_cmp(const int32_t *__restrict__ seq, const int32_t *__restrict__ M, int64_t N,
                           uint8_t *trapped, int32_t *seq_out, int32_t *mark)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        int s = seq[v];
        bool t = s >= 1 && M[v] < s;
        trapped[v] = t;
        int o = t ? -1 : s;
        if (seq_out) seq_out[v] = o;
        if (mark && o >= 1) mark[o] = 1;
    }
}

__global__ void k_remap(int32_t *seq_out, int64_t N, const int32_t *__restrict__ map)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        int s = seq_out[v];
        if (s >= 1) seq_out[v] = map[s];
    }
}

__global__ void k_level_init(const uint8_t *__restrict__ img, int64_t N, int32_t *level)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
        level[v] = img[v] ? -1 : 0;
}

// maximin value field for opening: dt2 on pore, 0 on solid (blocked)
__global__ void k_level_hist(const int32_t *__restrict__ level, int64_t N, int L, int32_t *cnt)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < N; base += stride) {
        int64_t v = base + threadIdx.x;
        int l = v < N ? level[v] : 0;
        int key = (l >= 1 && l <= L) ? l : 0;
        unsigned peers = __match_any_sync(0xffffffffu, key);
        if (key && lane == __ffs(peers) - 1) atomicAdd(cnt + key, __popc(peers));
    }
}

}  // namespace

int ibip_pc_launch(ibip_ctx *ctx, const int32_t *seq, ibip_dims d, const int32_t *r2, int64_t K, double voxel,
                   double sigma, double cos_theta, float *S, float *Pc, float *sat)
{
    cudaStream_t s = ctx->stream;
    const int64_t N = nvox(d);
    int32_t *cnt = (int32_t *)ibip_scratch(ctx, SC_HIST, ((size_t)K + 2) * sizeof(int32_t));
    int *small = (int *)ibip_scratch(ctx, SC_SMALL, kSmallBytes);
    if (!cnt || !small) return IBIP_ERR_OOM;
    int *np = small + 8;
    ibip_prof_begin(ctx, IBIP_K_PC);
    cudaMemsetAsync(cnt, 0, ((size_t)K + 2) * sizeof(int32_t), s);
    cudaMemsetAsync(np, 0, sizeof(int), s);
    const int gs = ctx->sm_count * 8;
    k_hist_seq<<<gs, 256, 0, s>>>(seq, N, K, cnt, np);
    IBIP_LAUNCH(ctx);
    int st = ibip_scan_incl_i32(ctx, cnt, cnt, K + 1);
    if (st) return st;
    const double num = -2.0 * sigma * cos_theta;
    if (K > 0) {
        k_pc<<<(unsigned)((K + 255) / 256 < gs ? (K + 255) / 256 : gs), 256, 0, s>>>(cnt, np, r2, K, voxel, num, S, Pc);
        IBIP_LAUNCH(ctx);
    }
    if (sat) {
        k_sat<<<gs, 256, 0, s>>>(seq, N, K, S, sat);
        IBIP_LAUNCH(ctx);
    }
    ibip_prof_end(ctx, IBIP_K_PC);
    return ibip_cuda_status(cudaGetLastError());
}

int ibip_trap_finish(ibip_ctx *ctx, const int32_t *seq, const int32_t *M, ibip_dims d, int rerank, uint8_t *trapped,
                     int32_t *seq_out)
{
    cudaStream_t s = ctx->stream;
    const int64_t N = nvox(d);
    const int gs = ctx->sm_count * 8;
    if (!rerank || !seq_out) {
        ibip_prof_begin(ctx, IBIP_K_TRAP);
        k_trap_cmp<<<gs, 256, 0, s>>>(seq, M, N, trapped, seq_out, nullptr);
        IBIP_LAUNCH(ctx);
        ibip_prof_end(ctx, IBIP_K_TRAP);
        return ibip_cuda_status(cudaGetLastError());
    }
    int *small = (int *)ibip_scratch(ctx, SC_SMALL, kSmallBytes);
    if (!small) return IBIP_ERR_OOM;
    int *mx = small + 12;
    ibip_prof_begin(ctx, IBIP_K_TRAP);
    cudaMemsetAsync(mx, 0, sizeof(int), s);
    k_max_seq<<<gs, 256, 0, s>>>(seq, N, mx);
    IBIP_LAUNCH(ctx);
    int *h = (int *)ctx->h_pinned;
    cudaMemcpyAsync(h, mx, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return IBIP_ERR_CUDA;
    const int K = h[0];
    int32_t *mark = (int32_t *)ibip_scratch(ctx, SC_HIST, ((size_t)K + 2) * sizeof(int32_t));
    if (!mark) return IBIP_ERR_OOM;
    cudaMemsetAsync(mark, 0, ((size_t)K + 2) * sizeof(int32_t), s);
    k_trap_cmp<<<gs, 256, 0, s>>>(seq, M, N, trapped, seq_out, mark);
    IBIP_LAUNCH(ctx);
    int st = ibip_scan_incl_i32(ctx, mark, mark, (int64_t)K + 1);
    if (st) return st;
    k_remap<<<gs, 256, 0, s>>>(seq_out, N, mark);
    IBIP_LAUNCH(ctx);
    ibip_prof_end(ctx, IBIP_K_TRAP);
    return ibip_cuda_status(cudaGetLastError());
}

int ibip_max_launch(ibip_ctx *ctx, const int32_t *a, int64_t n, int *h_max)
{
    int *small = (int *)ibip_scratch(ctx, SC_SMALL, kSmallBytes);
    if (!small) return IBIP_ERR_OOM;
    int *mx = small + 13;
    cudaStream_t s = ctx->stream;
    cudaMemsetAsync(mx, 0x80, sizeof(int), s);   // INT_MIN-ish start
    k_max_seq<<<ctx->sm_count * 8, 256, 0, s>>>(a, n, mx);
    IBIP_LAUNCH(ctx);
    cudaMemcpyAsync(ctx->h_pinned, mx, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ibip_cuda_status(e);
    *h_max = *(int *)ctx->h_pinned;
    return IBIP_OK;
}

int ibip_level_init(ibip_ctx *ctx, const uint8_t *img, ibip_dims d, int32_t *level)
{
    k_level_init<<<ctx->sm_count * 8, 256, 0, ctx->stream>>>(img, nvox(d), level);
    IBIP_LAUNCH(ctx);
    return ibip_cuda_status(cudaGetLastError());
}

int ibip_level_counts(ibip_ctx *ctx, const int32_t *level, ibip_dims d, int L, int64_t *h_counts)
{
    cudaStream_t s = ctx->stream;
    int32_t *cnt = (int32_t *)ibip_scratch(ctx, SC_HIST, ((size_t)L + 2) * sizeof(int32_t));
    if (!cnt) return IBIP_ERR_OOM;
    cudaMemsetAsync(cnt, 0, ((size_t)L + 2) * sizeof(int32_t), s);
    k_level_hist<<<ctx->sm_count * 8, 256, 0, s>>>(level, nvox(d), L, cnt);
    IBIP_LAUNCH(ctx);
    int32_t *h = (int32_t *)ctx->h_pinned;
    cudaMemcpyAsync(h, cnt, ((size_t)L + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ibip_cuda_status(e);
    int64_t run = 0;
    for (int i = 0; i < L; i++) { run += h[i + 1]; h_counts[i] = run; }
    return IBIP_OK;
}
