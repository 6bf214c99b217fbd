// pc.cu -- saturation and capillary pressure per step (Sections 2.2.1 and
// 2.2.2; Washburn relation as written in Section 2.4.1), plus the helpers
// trapping and opening need: thresholding against seq, re-ranking and
// level counts.
#include <algorithm>
#include <vector>

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

// cnt[l] += 1 for 1 <= level <= L: a per-block histogram in shared memory
// (warp-aggregated: equal levels in a warp cost one shared atomic), added to
// the global one once per bin and block
__global__ void k_level_hist(const int32_t *__restrict__ level, int64_t N, int L, int32_t *cnt)
{
    extern __shared__ int32_t s_lh[];   // L + 1 bins
    for (int i = threadIdx.x; i <= L; i += blockDim.x) s_lh[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < N; base += stride) {
        int64_t v = base + threadIdx.x;
        int l = v < N ? level[v] : 0;
        int key = (l >= 1 && l <= L) ? l : 0;
        unsigned peers = __match_any_sync(0xffffffffu, key);
        if (key && lane == __ffs(peers) - 1) atomicAdd(s_lh + key, __popc(peers));
    }
    __syncthreads();
    for (int i = threadIdx.x + 1; i <= L; i += blockDim.x)
        if (s_lh[i]) atomicAdd(cnt + i, s_lh[i]);
}

// Equal-saturation comparison with the opening (Section 3.1.1, by integer
// counts).  k_i = the smallest step whose cumulative count cum[k] reaches
// n_i (cum[K] if none does); one thread per level.
__global__ void k_eqsat_steps(const int32_t *__restrict__ cum, int64_t K, const int32_t *__restrict__ n, int L,
                              int32_t *kq)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L) return;
    const int32_t want = n[i];
    int64_t lo = 0, hi = K;   // cum is non-decreasing; cum[0] = 0
    if (cum[K] < want) { kq[i] = (int32_t)K; return; }
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (cum[mid] >= want) hi = mid; else lo = mid + 1;
    }
    kq[i] = (int32_t)lo;
}

// A voxel is in the opening's set of level i from i = level - 1 on, and in
// the invasion's matched set from the first i with k_i >= seq on: the two
// differ on the levels between those two starts.  Difference array over
// levels, per block in shared memory.
constexpr int kMaxEqLevels = 256;
__global__ void k_eqsat(const int32_t *__restrict__ seq, const int32_t *__restrict__ level, int64_t N,
                        const int32_t *__restrict__ kq, int L, int32_t *dh)
{
    __shared__ int32_t s_k[kMaxEqLevels];
    __shared__ int32_t s_h[kMaxEqLevels + 1];
    for (int i = threadIdx.x; i < L; i += blockDim.x) s_k[i] = kq[i];
    for (int i = threadIdx.x; i <= L; i += blockDim.x) s_h[i] = 0;
    __syncthreads();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        const int lv = level[v], sq = seq[v];
        const int a = lv >= 1 ? lv - 1 : L;
        int b = L;
        if (sq >= 1) {
            int lo = 0, hi = L;   // first i with k_i >= seq (k is non-decreasing)
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s_k[mid] >= sq) hi = mid; else lo = mid + 1;
            }
            b = lo;
        }
        if (a != b) {
            atomicAdd(s_h + min(a, b), 1);
            atomicAdd(s_h + max(a, b), -1);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= L; i += blockDim.x)
        if (s_h[i]) atomicAdd(dh + i, s_h[i]);
}

// Drainage envelope at the opening's levels (Sections 2.2.2 and 3.1.1): the
// levels a step's sphere lies below are a prefix [0, p) of the strictly
// decreasing T (p = the first level with T <= r2); the first step below
// level i is the smallest step with p > i, collected as a minimum per p - 1
// and completed by a suffix minimum over the levels.
__global__ void k_env_first(const int32_t *__restrict__ r2, int64_t K, const int32_t *__restrict__ T, int L,
                            int32_t *first)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < K; base += stride) {   // block-uniform
        const int64_t j = base + threadIdx.x;
        int lo = -1;
        if (j < K) {
            const int v = r2[j];
            int hi = L;   // first level with T <= v
            lo = 0;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (T[mid] <= v) hi = mid; else lo = mid + 1;
            }
        }
        // steps of a warp are consecutive: the lowest lane of each group
        // with the same target holds the group's smallest step
        const unsigned peers = __match_any_sync(0xffffffffu, lo);
        if (lo > 0 && lane == __ffs(peers) - 1) atomicMin(first + lo - 1, (int32_t)j);
    }
}

// re-ranked trapping: the radius of every surviving step, in its new order
// (map = inclusive prefix count of surviving steps)
__global__ void k_compact_r2(const int32_t *__restrict__ map, int64_t K, const int32_t *__restrict__ r2,
                             int32_t *r2_out)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; k <= K; k += (int64_t)gridDim.x * blockDim.x)
        if (map[k] != map[k - 1]) r2_out[map[k] - 1] = r2[k - 1];
}

// the size of the sphere that invaded each voxel (Section 2.2.2, Figure 5
// right), as its squared radius; 0 on solid, -1 on uninvaded pore
__global__ void k_size_image(const int32_t *__restrict__ seq, int64_t N, const int32_t *__restrict__ r2, int64_t K,
                             int32_t *out)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        const int s = seq[v];
        out[v] = s == 0 ? 0 : (s >= 1 && s <= K ? r2[s - 1] : -1);
    }
}

// ---- the same for every image of a batch: one launch per stage, each
// block finding its image by binary search over the images' first blocks
struct CurveJob {
    const int32_t *seq;     // invasion sequence
    const int32_t *M;       // widest-path field from the outlet, or null: no trapping
    uint8_t *trapped;
    int32_t *seq_out;       // or null
    const int32_t *cseq;    // the sequence the curve counts (seq_out after trapping, else seq)
    const int32_t *r2;
    float *S, *Pc;          // null: no curve
    int64_t N, K, cnt_off;  // voxels, steps, first entry of the pooled per-step counts [K + 2]
    double voxel, num;      // voxel size and -2 sigma cos(theta)
    int blk_vox, blk_k;     // first block in the voxel and step launches
};

constexpr int kCvBlock = 256, kCvPer = 8;

__device__ __forceinline__ int find_cjob(const CurveJob *jobs, int n, int blk, bool steps)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if ((steps ? jobs[mid].blk_k : jobs[mid].blk_vox) <= blk) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_trap_cmp_b(const CurveJob *__restrict__ jobs, int n)
{
    const CurveJob &J = jobs[find_cjob(jobs, n, blockIdx.x, false)];
    if (!J.M) return;
    const int64_t v0 = (int64_t)(blockIdx.x - J.blk_vox) * kCvBlock * kCvPer;
    for (int q = 0; q < kCvPer; q++) {
        const int64_t v = v0 + q * kCvBlock + threadIdx.x;
        if (v >= J.N) break;
        const int sq = J.seq[v];
        const bool t = sq >= 1 && J.M[v] < sq;
        J.trapped[v] = t;
        if (J.seq_out) J.seq_out[v] = t ? -1 : sq;
    }
}

// per-step counts (warp-aggregated; a block holds one image) and pore counts
__global__ void k_hist_seq_b(const CurveJob *__restrict__ jobs, int n, int32_t *cnt, int *npore)
{
    const int j = find_cjob(jobs, n, blockIdx.x, false);
    const CurveJob &J = jobs[j];
    if (!J.S) return;
    const int lane = threadIdx.x & 31;
    const int64_t v0 = (int64_t)(blockIdx.x - J.blk_vox) * kCvBlock * kCvPer;
    int np = 0;
    for (int q = 0; q < kCvPer; q++) {
        const int64_t v = v0 + q * kCvBlock + threadIdx.x;
        const int sq = v < J.N ? J.cseq[v] : 0;
        np += sq != 0;
        const int key = (sq >= 1 && sq <= J.K) ? sq : 0;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        if (key && lane == __ffs(peers) - 1) atomicAdd(cnt + J.cnt_off + key, __popc(peers));
    }
    for (int o = 16; o; o >>= 1) np += __shfl_xor_sync(0xffffffffu, np, o);
    if (lane == 0 && np) atomicAdd(npore + j, np);
}

// after the flat inclusive scan of the counts: S and Pc of every step (the
// formulas of k_pc; an image's counts are relative to its segment's start)
__global__ void k_pc_b(const CurveJob *__restrict__ jobs, int n, const int32_t *__restrict__ cum,
                       const int *__restrict__ npore)
{
    const int j = find_cjob(jobs, n, blockIdx.x, true);
    const CurveJob &J = jobs[j];
    if (!J.S) return;
    const int64_t k = (int64_t)(blockIdx.x - J.blk_k) * blockDim.x + threadIdx.x;
    if (k >= J.K) return;
    const double np = (double)npore[j];
    const int32_t base = cum[J.cnt_off];   // the segment's count of step 0 is zero
    J.S[k] = (float)((double)(cum[J.cnt_off + k + 1] - base) / np);
    J.Pc[k] = (float)(J.num / (sqrt((double)J.r2[k]) * J.voxel));
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
                     int32_t *seq_out, const int32_t *r2_in, int64_t k_in, int32_t *r2_out, int64_t *h_nout)
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
    if (ibip_sync(ctx, s) != cudaSuccess) return IBIP_ERR_CUDA;
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
    if (r2_in && r2_out) {
        const int64_t Kc = K < k_in ? K : k_in;
        k_compact_r2<<<gs, 256, 0, s>>>(mark, Kc, r2_in, r2_out);
        IBIP_LAUNCH(ctx);
    }
    if (h_nout) {
        cudaMemcpyAsync(h, mark + K, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (ibip_sync(ctx, s) != cudaSuccess) return IBIP_ERR_CUDA;
        *h_nout = h[0];
    }
    ibip_prof_end(ctx, IBIP_K_TRAP);
    return ibip_cuda_status(cudaGetLastError());
}

int ibip_size_launch(ibip_ctx *ctx, const int32_t *seq, ibip_dims d, const int32_t *r2, int64_t K, int32_t *out)
{
    k_size_image<<<ctx->sm_count * 8, 256, 0, ctx->stream>>>(seq, nvox(d), r2, K, out);
    IBIP_LAUNCH(ctx);
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
    cudaError_t e = ibip_sync(ctx, s);
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
    k_level_hist<<<ctx->sm_count * 8, 256, ((size_t)L + 1) * sizeof(int32_t), s>>>(level, nvox(d), L, cnt);
    IBIP_LAUNCH(ctx);
    int32_t *h = (int32_t *)ctx->h_pinned;
    cudaMemcpyAsync(h, cnt, ((size_t)L + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaError_t e = ibip_sync(ctx, s);
    if (e != cudaSuccess) return ibip_cuda_status(e);
    int64_t run = 0;
    for (int i = 0; i < L; i++) { run += h[i + 1]; h_counts[i] = run; }
    return IBIP_OK;
}

int ibip_eqsat_launch(ibip_ctx *ctx, const int32_t *seq, const int32_t *level, ibip_dims d, int64_t K, int L,
                      int64_t *h_steps, int64_t *h_diff, int64_t *h_count)
{
    cudaStream_t s = ctx->stream;
    const int64_t N = nvox(d);
    const int gs = ctx->sm_count * 8;
    // layout: cum[K + 2] | lv[L + 2] | kq[L] | dh[L + 1] | npore
    const size_t words = (size_t)K + 2 + (L + 2) + L + (L + 1) + 1;
    int32_t *w = (int32_t *)ibip_scratch(ctx, SC_HIST, words * sizeof(int32_t));
    if (!w) return IBIP_ERR_OOM;
    int32_t *cum = w, *lv = cum + K + 2, *kq = lv + L + 2, *dh = kq + L, *np = dh + L + 1;
    cudaMemsetAsync(w, 0, words * sizeof(int32_t), s);
    k_hist_seq<<<gs, 256, 0, s>>>(seq, N, K, cum, np);
    IBIP_LAUNCH(ctx);
    int st = ibip_scan_incl_i32(ctx, cum, cum, K + 1);
    if (st) return st;
    k_level_hist<<<gs, 256, ((size_t)L + 1) * sizeof(int32_t), s>>>(level, N, L, lv);
    IBIP_LAUNCH(ctx);
    st = ibip_scan_incl_i32(ctx, lv + 1, lv + 1, L);   // lv[1 + i] = voxels with 1 <= level <= i + 1
    if (st) return st;
    k_eqsat_steps<<<(L + 127) / 128, 128, 0, s>>>(cum, K, lv + 1, L, kq);
    IBIP_LAUNCH(ctx);
    k_eqsat<<<gs, 256, 0, s>>>(seq, level, N, kq, L, dh);
    IBIP_LAUNCH(ctx);
    int32_t *h = (int32_t *)ctx->h_pinned;   // L <= 254: 3L + 1 words fit the pinned buffer
    cudaMemcpyAsync(h, lv + 1, (size_t)L * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(h + L, kq, (size_t)L * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(h + 2 * L, dh, ((size_t)L + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaError_t e = ibip_sync(ctx, s);
    if (e != cudaSuccess) return ibip_cuda_status(e);
    int64_t run = 0;
    for (int i = 0; i < L; i++) {
        run += h[2 * L + i];
        if (h_count) h_count[i] = h[i];
        if (h_steps) h_steps[i] = h[L + i];
        h_diff[i] = run;
    }
    return IBIP_OK;
}

int ibip_envelope_launch(ibip_ctx *ctx, const int32_t *seq, ibip_dims d, const int32_t *step_r2, int64_t K,
                         const int32_t *h_levels, int L, int64_t *h_steps, int64_t *h_count)
{
    cudaStream_t s = ctx->stream;
    const int64_t N = nvox(d);
    const int gs = ctx->sm_count * 8;
    // layout: cum[K + 2] | T[L] | first[L] | npore
    const size_t words = (size_t)K + 2 + 2 * (size_t)L + 1;
    int32_t *w = (int32_t *)ibip_scratch(ctx, SC_HIST, words * sizeof(int32_t));
    if (!w) return IBIP_ERR_OOM;
    int32_t *cum = w, *T = cum + K + 2, *first = T + L, *np = first + L;
    cudaMemsetAsync(cum, 0, ((size_t)K + 2) * sizeof(int32_t), s);
    cudaMemsetAsync(first, 0x7f, (size_t)L * sizeof(int32_t), s);   // 0x7f7f7f7f: no step below
    cudaMemcpyAsync(T, h_levels, (size_t)L * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    k_hist_seq<<<gs, 256, 0, s>>>(seq, N, K, cum, np);
    IBIP_LAUNCH(ctx);
    int st = ibip_scan_incl_i32(ctx, cum, cum, K + 1);   // cum[k] = voxels with 1 <= seq <= k
    if (st) return st;
    if (K > 0) {
        k_env_first<<<(int)std::min<int64_t>((K + 255) / 256, gs), 256, 0, s>>>(step_r2, K, T, L, first);
        IBIP_LAUNCH(ctx);
    }
    int32_t *h = (int32_t *)ctx->h_pinned;   // L <= 254
    cudaMemcpyAsync(h, first, (size_t)L * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaError_t e = ibip_sync(ctx, s);
    if (e != cudaSuccess) return ibip_cuda_status(e);
    int64_t run = K;
    for (int i = L - 1; i >= 0; i--) {   // suffix minimum: steps below level i+1 are below level i too
        if ((int64_t)h[i] < run) run = h[i];
        h_steps[i] = run;
    }
    // the counts at those steps
    for (int i = 0; i < L; i++) {
        cudaMemcpyAsync(h + i, cum + h_steps[i], sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    }
    e = ibip_sync(ctx, s);
    if (e != cudaSuccess) return ibip_cuda_status(e);
    for (int i = 0; i < L; i++) h_count[i] = h[i];
    return IBIP_OK;
}

int ibip_curve_batch_launch(ibip_ctx *ctx, int n, const IbipCurveItem *items)
{
    cudaStream_t s = ctx->stream;
    if (n <= 0) return IBIP_OK;
    std::vector<CurveJob> jobs;
    std::vector<int> which;
    int64_t cnt_total = 0;
    int blk_vox = 0, blk_k = 0;
    bool any_trap = false, any_curve = false;
    for (int i = 0; i < n; i++) {
        const IbipCurveItem &it = items[i];
        if (!it.M && !it.S) continue;
        CurveJob J = {};
        J.seq = it.seq; J.M = it.M; J.trapped = it.trapped; J.seq_out = it.seq_out;
        J.cseq = (it.M && it.seq_out) ? it.seq_out : it.seq;
        J.r2 = it.r2; J.S = it.S; J.Pc = it.Pc;
        J.N = nvox(it.d); J.K = it.S ? it.K : 0;
        J.cnt_off = cnt_total;
        if (it.S) cnt_total += J.K + 2;
        J.voxel = it.voxel; J.num = -2.0 * it.sigma * it.cos_theta;
        J.blk_vox = blk_vox;
        blk_vox += (int)((J.N + kCvBlock * kCvPer - 1) / (kCvBlock * kCvPer));
        J.blk_k = blk_k;
        blk_k += (int)((J.K + 255) / 256);
        any_trap |= it.M != nullptr;
        any_curve |= it.S != nullptr;
        jobs.push_back(J);
        which.push_back(i);
    }
    const int m = (int)jobs.size();
    if (m == 0) return IBIP_OK;
    if (cnt_total >= (1ll << 31)) return IBIP_ERR_ARG;
    const size_t tab = ((size_t)m * sizeof(CurveJob) + 255) / 256 * 256;
    const size_t npb = ((size_t)m * sizeof(int) + 255) / 256 * 256;
    char *w = (char *)ibip_scratch(ctx, SC_HIST, ibip_curve_batch_bytes(m, cnt_total));
    if (!w) return IBIP_ERR_OOM;
    CurveJob *dj = (CurveJob *)w;
    int *np = (int *)(w + tab);
    int32_t *cnt = (int32_t *)(w + tab + npb);
    cudaMemcpyAsync(dj, jobs.data(), (size_t)m * sizeof(CurveJob), cudaMemcpyHostToDevice, s);
    if (any_trap) {
        ibip_prof_begin(ctx, IBIP_K_TRAP);
        k_trap_cmp_b<<<blk_vox, kCvBlock, 0, s>>>(dj, m);
        IBIP_LAUNCH(ctx);
        ibip_prof_end(ctx, IBIP_K_TRAP);
    }
    if (any_curve) {
        ibip_prof_begin(ctx, IBIP_K_PC);
        cudaMemsetAsync(w + tab, 0, npb + (size_t)(cnt_total + 1) * sizeof(int32_t), s);
        k_hist_seq_b<<<blk_vox, kCvBlock, 0, s>>>(dj, m, cnt, np);
        IBIP_LAUNCH(ctx);
        int st = ibip_scan_incl_i32(ctx, cnt, cnt, cnt_total);
        if (st) return st;
        if (blk_k > 0) {
            k_pc_b<<<blk_k, 256, 0, s>>>(dj, m, cnt, np);
            IBIP_LAUNCH(ctx);
        }
        ibip_prof_end(ctx, IBIP_K_PC);
    }
    return ibip_cuda_status(cudaGetLastError());
}

size_t ibip_curve_batch_bytes(int n, int64_t cnt_total)
{
    return ((size_t)n * sizeof(CurveJob) + 255) / 256 * 256 + ((size_t)n * sizeof(int) + 255) / 256 * 256 +
           (size_t)(cnt_total + 1) * sizeof(int32_t);
}
