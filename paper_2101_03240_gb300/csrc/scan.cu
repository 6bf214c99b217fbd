// scan.cu -- device-wide prefix sums over int32 arrays (reduce, scan the
// block totals recursively, then scan each block with its offset).
#include "common.cuh"

namespace {

constexpr int kScanThreads = 512;
constexpr int kPerThread = 8;
constexpr int kPerBlock = kScanThreads * kPerThread;

__device__ __forceinline__ int warp_incl(int v, int lane)
{
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// block-wide exclusive scan of one value per thread; returns the prefix and
// writes the block total to *total
__device__ int block_excl(int v, int *total)
{
    __shared__ int s_w[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = warp_incl(v, lane);
    if (lane == 31) s_w[w] = inc;
    __syncthreads();
    if (w == 0) {
        int t = lane < kScanThreads / 32 ? s_w[lane] : 0;
        int ti = warp_incl(t, lane);
        if (lane < kScanThreads / 32) s_w[lane] = ti - t;
        if (lane == kScanThreads / 32 - 1) *total = ti;
    }
    __syncthreads();
    int r = inc - v + s_w[w];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_block_sums(const int32_t *in, int64_t n, int32_t *sums)
{
    __shared__ int s_total;
    int64_t b = (int64_t)blockIdx.x * kPerBlock + (int64_t)threadIdx.x * kPerThread;
    int acc = 0;
    for (int k = 0; k < kPerThread; k++) if (b + k < n) acc += in[b + k];
    block_excl(acc, &s_total);
    if (threadIdx.x == 0) sums[blockIdx.x] = s_total;
}

__global__ void __launch_bounds__(kScanThreads) k_block_scan(const int32_t *in, int64_t n,
                                                             const int32_t *offs, int32_t *out, int incl)
{
    __shared__ int s_total;
    int64_t b = (int64_t)blockIdx.x * kPerBlock + (int64_t)threadIdx.x * kPerThread;
    int v[kPerThread];
    int acc = 0;
    for (int k = 0; k < kPerThread; k++) {
        v[k] = b + k < n ? in[b + k] : 0;
        acc += v[k];
    }
    int run = block_excl(acc, &s_total) + (offs ? offs[blockIdx.x] : 0);
    for (int k = 0; k < kPerThread; k++) {
        if (incl) run += v[k];
        if (b + k < n) out[b + k] = run;
        if (!incl) run += v[k];
    }
}

int scan_rec(ibip_ctx *ctx, const int32_t *in, int32_t *out, int64_t n, int incl, int32_t *work)
{
    int64_t nb = (n + kPerBlock - 1) / kPerBlock;
    if (nb == 1) {
        k_block_scan<<<1, kScanThreads, 0, ctx->stream>>>(in, n, nullptr, out, incl);
        IBIP_LAUNCH(ctx);
        return IBIP_OK;
    }
    int32_t *sums = work, *offs = work + nb;
    k_block_sums<<<(unsigned)nb, kScanThreads, 0, ctx->stream>>>(in, n, sums);
    IBIP_LAUNCH(ctx);
    int st = scan_rec(ctx, sums, offs, nb, 0, work + 2 * nb);
    if (st) return st;
    k_block_scan<<<(unsigned)nb, kScanThreads, 0, ctx->stream>>>(in, n, offs, out, incl);
    IBIP_LAUNCH(ctx);
    return IBIP_OK;
}

size_t scan_words(int64_t n)
{
    size_t need = 16;
    for (int64_t m = (n + kPerBlock - 1) / kPerBlock; m > 1; m = (m + kPerBlock - 1) / kPerBlock)
        need += (size_t)m * 2;
    return need;
}

int scan_impl(ibip_ctx *ctx, const int32_t *in, int32_t *out, int64_t n, int incl)
{
    if (n <= 0) return IBIP_OK;
    const size_t need = scan_words(n);
    int32_t *work = (int32_t *)ibip_scratch(ctx, SC_SCAN, need * sizeof(int32_t));
    if (!work) return IBIP_ERR_OOM;
    int st = scan_rec(ctx, in, out, n, incl, work);
    return st ? st : ibip_cuda_status(cudaGetLastError());
}

}  // namespace

size_t ibip_scan_scratch_bytes(int64_t n) { return scan_words(n) * sizeof(int32_t); }

int ibip_scan_excl_i32(ibip_ctx *ctx, const int32_t *in, int32_t *out, int64_t n)
{
    return scan_impl(ctx, in, out, n, 0);
}

int ibip_scan_incl_i32(ibip_ctx *ctx, const int32_t *in, int32_t *out, int64_t n)
{
    return scan_impl(ctx, in, out, n, 1);
}
