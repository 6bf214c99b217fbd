// edt.cu -- exact squared Euclidean distance transform (Section 2.1, the
// distance transform of the pore space, Figure 2b) and the per-level
// dilation of morphological-opening drainage (Section 2.4.1).
//
// The squared EDT is separable: dt2(x,y,z) = min over features (a,b,c) of
// (x-a)^2 + (y-b)^2 + (z-c)^2.  Three passes:
//   pass z: d1 = distance along z to the nearest feature in the row (uint16,
//           0xFFFF = none), from warp ballots over 32-voxel chunks;
//   pass y: g2(y) = min_j d1(j)^2 + (y-j)^2 over the y column;
//   pass x: dt2(x) = min_j g2(j) + (x-j)^2 over the x column.
// Passes y and x stage a column strip (32 consecutive z, all of the line) in
// shared memory so every global access is a coalesced 64/128-byte row, and
// evaluate each output by a search that widens from j = i outwards and stops
// once (i-j)^2 alone reaches the best value (or the optional cap): exact,
// integer-only, and proportional to the distance itself.
#include "common.cuh"

namespace {

constexpr int kZWarps = 8;          // rows per block in pass z
constexpr int kMaxChunks = 512;     // nz <= 16384
constexpr int kStripW = 32;         // z lanes per strip in passes y / x
constexpr int kStripWarps = 8;

struct FeatSolid {
    const uint8_t *img;
    __device__ bool operator()(int64_t v) const { return __ldg(img + v) == 0; }
};
struct FeatAtLeast {
    const int32_t *w;
    int32_t t;
    __device__ bool operator()(int64_t v) const { return __ldg(w + v) >= t; }
};
// opening: voxel v belongs to the trimmed set of level i iff its first level
// (the first radius index whose T it reaches) is <= i
struct FeatFirstLevel {
    const uint8_t *fl;
    int i;
    __device__ bool operator()(int64_t v) const { return __ldg(fl + v) <= i; }
};

// first level of every voxel: the smallest i with W >= T[i] (255 if none)
__global__ void k_first_level(const int32_t *__restrict__ W, int64_t N, const int32_t *__restrict__ T, int L,
                              uint8_t *fl)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        const int w = W[v];
        int lo = 0, hi = L;   // T is strictly decreasing: first index with T <= w
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(T + mid) <= w) hi = mid; else lo = mid + 1;
        }
        fl[v] = (uint8_t)(lo < L ? lo : 255);
    }
}

template <class Feat>
__global__ void __launch_bounds__(kZWarps * 32) k_edt_z(Feat feat, int nrows, int nz, int cap,
                                                        uint16_t *__restrict__ d1)
{
    __shared__ uint32_t s_mask[kZWarps][kMaxChunks];
    __shared__ int s_left[kZWarps][kMaxChunks];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * kZWarps + w;
    if (row >= nrows) return;
    const int64_t base = row * nz;
    const int nch = (nz + 31) >> 5;
    const int NONE = 1 << 29;
    int carry = -NONE;
    // feature tests of eight chunks are issued before their ballots so the
    // loads overlap
    for (int c0 = 0; c0 < nch; c0 += 8) {
        bool f[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const int z = ((c0 + q) << 5) + lane;
            f[q] = c0 + q < nch && z < nz && feat(base + z);
        }
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const int c = c0 + q;
            if (c >= nch) break;
            const uint32_t m = __ballot_sync(0xffffffffu, f[q]);
            if (lane == 0) { s_mask[w][c] = m; s_left[w][c] = carry; }
            if (m) carry = (c << 5) + 31 - __clz(m);
        }
    }
    __syncwarp();
    int right = NONE;
    for (int c = nch - 1; c >= 0; c--) {
        uint32_t m = s_mask[w][c];
        int z = (c << 5) + lane;
        uint32_t ml = m & (0xffffffffu >> (31 - lane));
        int left = ml ? (c << 5) + 31 - __clz(ml) : s_left[w][c];
        uint32_t mr = m & (0xffffffffu << lane);
        int rt = mr ? (c << 5) + __ffs(mr) - 1 : right;
        if (z < nz) {
            int d = min(z - left, rt - z);
            d1[base + z] = (d > cap) ? (uint16_t)0xffff : (uint16_t)d;
        }
        if (m) right = (c << 5) + __ffs(m) - 1;
    }
}

// One min-plus line search.  `g(j)` returns the squared partial distance or
// IBIP_INF32.  Values >= cap2 are reported as IBIP_INF32.
template <class G>
__device__ __forceinline__ int line_min(const G &g, int i, int n, int cap2)
{
    int best = g(i);
    int lim = best < cap2 ? best : cap2;
    for (int d = 1;; d++) {
        int64_t dd = (int64_t)d * d;
        if (dd >= lim) break;
        int j0 = i - d, j1 = i + d;
        if (j0 < 0 && j1 >= n) break;
        if (j0 >= 0) {
            int v = g(j0);
            if (v != IBIP_INF32 && v + dd < best) { best = v + (int)dd; lim = best < cap2 ? best : cap2; }
        }
        if (j1 < n) {
            int v = g(j1);
            if (v != IBIP_INF32 && v + dd < best) { best = v + (int)dd; lim = best < cap2 ? best : cap2; }
        }
    }
    return best >= cap2 ? IBIP_INF32 : best;
}

// pass y: strip = (x, all y, 32 z).  blockIdx.x = z strip, blockIdx.y = x.
template <bool SMEM>
__global__ void __launch_bounds__(kStripWarps * 32) k_edt_y(const uint16_t *__restrict__ d1, int ny,
                                                            int nz, int cap2, int32_t *__restrict__ g2)
{
    extern __shared__ uint16_t s_col[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int x = blockIdx.y, z = blockIdx.x * kStripW + lane;
    const bool ok = z < nz;
    const int64_t b = (int64_t)x * ny * nz + z;
    if (SMEM) {
#pragma unroll 8
        for (int y = w; y < ny; y += kStripWarps) s_col[y * kStripW + lane] = ok ? __ldg(d1 + b + (int64_t)y * nz) : 0xffff;
        __syncthreads();
    }
    if (!ok) return;
    auto g = [&](int j) -> int {
        uint16_t v = SMEM ? s_col[j * kStripW + lane] : __ldg(d1 + b + (int64_t)j * nz);
        return v == 0xffff ? IBIP_INF32 : (int)v * (int)v;
    };
    for (int y = w; y < ny; y += kStripWarps) g2[b + (int64_t)y * nz] = line_min(g, y, ny, cap2);
}

struct EpiStore {
    int32_t *out;
    __device__ void operator()(int64_t v, int val) const { out[v] = val; }
};
// MIO: voxels within the dilation that have no level yet get `lvl`.
struct EpiLevel {
    int32_t *level;
    int32_t T, lvl;
    __device__ void operator()(int64_t v, int val) const
    {
        if (val < T && level[v] == -1) level[v] = lvl;
    }
};

// pass x: strip = (y, all x, 32 z).  blockIdx.x = z strip, blockIdx.y = y.
template <bool SMEM, class Epi>
__global__ void __launch_bounds__(kStripWarps * 32) k_edt_x(const int32_t *__restrict__ g2, int nx,
                                                            int ny, int nz, int cap2, Epi epi)
{
    extern __shared__ int32_t s_colx[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int y = blockIdx.y, z = blockIdx.x * kStripW + lane;
    const bool ok = z < nz;
    const int64_t st = (int64_t)ny * nz;
    const int64_t b = (int64_t)y * nz + z;
    if (SMEM) {
#pragma unroll 8
        for (int x = w; x < nx; x += kStripWarps) s_colx[x * kStripW + lane] = ok ? __ldg(g2 + b + x * st) : IBIP_INF32;
        __syncthreads();
    }
    if (!ok) return;
    auto g = [&](int j) -> int { return SMEM ? s_colx[j * kStripW + lane] : __ldg(g2 + b + j * st); };
    for (int x = w; x < nx; x += kStripWarps) epi(b + x * st, line_min(g, x, nx, cap2));
}

constexpr size_t kSmemBudget = 200 * 1024;

template <class Feat, class Epi>
int edt_passes(ibip_ctx *ctx, Feat feat, ibip_dims d, int cap, int cap2, Epi epi, int cls)
{
    int64_t N = nvox(d);
    uint16_t *d1 = (uint16_t *)ibip_scratch(ctx, SC_D1, N * sizeof(uint16_t));
    int32_t *g2 = (int32_t *)ibip_scratch(ctx, SC_G2, N * sizeof(int32_t));
    if (!d1 || !g2) return IBIP_ERR_OOM;
    cudaStream_t s = ctx->stream;
    int nrows = d.nx * d.ny;
    ibip_prof_begin(ctx, cls);
    k_edt_z<Feat><<<(nrows + kZWarps - 1) / kZWarps, kZWarps * 32, 0, s>>>(feat, nrows, d.nz, cap, d1);
    IBIP_LAUNCH(ctx);
    dim3 gy((d.nz + kStripW - 1) / kStripW, d.nx);
    size_t sy = (size_t)d.ny * kStripW * sizeof(uint16_t);
    if (sy <= kSmemBudget) {
        cudaFuncSetAttribute(k_edt_y<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget);
        k_edt_y<true><<<gy, kStripWarps * 32, sy, s>>>(d1, d.ny, d.nz, cap2, g2);
    } else {
        k_edt_y<false><<<gy, kStripWarps * 32, 0, s>>>(d1, d.ny, d.nz, cap2, g2);
    }
    IBIP_LAUNCH(ctx);
    dim3 gx((d.nz + kStripW - 1) / kStripW, d.ny);
    size_t sx = (size_t)d.nx * kStripW * sizeof(int32_t);
    if (sx <= kSmemBudget) {
        cudaFuncSetAttribute(k_edt_x<true, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget);
        k_edt_x<true, Epi><<<gx, kStripWarps * 32, sx, s>>>(g2, d.nx, d.ny, d.nz, cap2, epi);
    } else {
        k_edt_x<false, Epi><<<gx, kStripWarps * 32, 0, s>>>(g2, d.nx, d.ny, d.nz, cap2, epi);
    }
    IBIP_LAUNCH(ctx);
    ibip_prof_end(ctx, cls);
    return ibip_cuda_status(cudaGetLastError());
}

}  // namespace

int ibip_edt_launch(ibip_ctx *ctx, const uint8_t *image, ibip_dims d, int32_t *dt2)
{
    return edt_passes(ctx, FeatSolid{image}, d, 0xfffe, IBIP_INF32, EpiStore{dt2}, IBIP_K_EDT);
}

int ibip_first_level_launch(ibip_ctx *ctx, const int32_t *W, ibip_dims d, const int32_t *T_dev, int L, uint8_t *fl)
{
    k_first_level<<<ctx->sm_count * 8, 256, 0, ctx->stream>>>(W, nvox(d), T_dev, L, fl);
    IBIP_LAUNCH(ctx);
    return ibip_cuda_status(cudaGetLastError());
}

int ibip_dilate_first_level_launch(ibip_ctx *ctx, const uint8_t *fl, int32_t T, int32_t i, ibip_dims d, int32_t *level)
{
    int cap = 0;
    while ((int64_t)(cap + 1) * (cap + 1) < T && cap < 0xfffe) cap++;
    return edt_passes(ctx, FeatFirstLevel{fl, i}, d, cap, T, EpiLevel{level, T, i + 1}, IBIP_K_DILATE);
}

int ibip_dilate_level_launch(ibip_ctx *ctx, const int32_t *W, int32_t T, int32_t lvl, ibip_dims d,
                             int32_t *level)
{
    // Only squared distances < T matter: a 1-D distance r with r*r >= T is
    // as good as none, and every partial sum >= T is capped.
    int cap = 0;
    while ((int64_t)(cap + 1) * (cap + 1) < T && cap < 0xfffe) cap++;
    return edt_passes(ctx, FeatAtLeast{W, T}, d, cap, T, EpiLevel{level, T, lvl}, IBIP_K_DILATE);
}

// ------------------------------------------------------------------------
// ibip_edt_noalloc: the same three EDT passes for callers that may not
// allocate device memory.  The pass-y intermediate lives in a fixed
// file-scope device array; the pass-z intermediate (uint16 per voxel) is
// written into the first half of the caller's dt2 buffer, which pass x then
// overwrites with the result.
// ------------------------------------------------------------------------

#include <mutex>

namespace {

constexpr int64_t kNoallocMaxVoxels = 1ll << 21;   // 2,097,152 voxels (e.g. 128^3): 8 MB below

// Shared by every call on a device; held by every GPU that loads the library.
static __device__ __align__(256) int32_t g_noalloc_g2[kNoallocMaxVoxels];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
int32_t *g_noalloc_ptr[kNoallocMaxDevices];   // device address of g_noalloc_g2, per device

}  // namespace

extern "C" int ibip_edt_noalloc(const uint8_t *image, ibip_dims d, int32_t *dt2, void *cuda_stream)
{
    if (!image || !dt2 || d.nx < 1 || d.ny < 1 || d.nz < 1 || d.nx > 16384 || d.ny > 16384 || d.nz > 16384)
        return IBIP_ERR_ARG;
    const int64_t N = nvox(d);
    if (N > kNoallocMaxVoxels) return IBIP_ERR_TOO_LARGE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) {
        cudaGetLastError();
        return IBIP_ERR_CUDA;
    }
    int32_t *g2 = nullptr;
    {
        // one-time set-up per device, with that device current: the host-side
        // name of the array is not a device address, so ask the runtime for it
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_g2) != cudaSuccess || !p) {
                cudaGetLastError();
                return IBIP_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = (int32_t *)p;
        }
        g2 = g_noalloc_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    uint16_t *d1 = (uint16_t *)dt2;   // 2 bytes per voxel inside the 4-byte output
    const int nrows = d.nx * d.ny;
    k_edt_z<FeatSolid><<<(nrows + kZWarps - 1) / kZWarps, kZWarps * 32, 0, s>>>(FeatSolid{image}, nrows, d.nz, 0xfffe, d1);
    dim3 gy((d.nz + kStripW - 1) / kStripW, d.nx);
    const size_t sy = (size_t)d.ny * kStripW * sizeof(uint16_t);
    if (sy <= kSmemBudget) {
        cudaFuncSetAttribute(k_edt_y<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget);
        k_edt_y<true><<<gy, kStripWarps * 32, sy, s>>>(d1, d.ny, d.nz, IBIP_INF32, g2);
    } else {
        k_edt_y<false><<<gy, kStripWarps * 32, 0, s>>>(d1, d.ny, d.nz, IBIP_INF32, g2);
    }
    dim3 gx((d.nz + kStripW - 1) / kStripW, d.ny);
    const size_t sx = (size_t)d.nx * kStripW * sizeof(int32_t);
    if (sx <= kSmemBudget) {
        cudaFuncSetAttribute(k_edt_x<true, EpiStore>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget);
        k_edt_x<true, EpiStore><<<gx, kStripWarps * 32, sx, s>>>(g2, d.nx, d.ny, d.nz, IBIP_INF32, EpiStore{dt2});
    } else {
        k_edt_x<false, EpiStore><<<gx, kStripWarps * 32, 0, s>>>(g2, d.nx, d.ny, d.nz, IBIP_INF32, EpiStore{dt2});
    }
    return ibip_cuda_status(cudaGetLastError());
}
