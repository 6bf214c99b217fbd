// edt.cu -- exact squared Euclidean distance transform (Section 2.1, the
// distance transform of the pore space, Figure 2b) and the per-level
// dilation of morphological-opening drainage (Section 2.4.1).
//
// The squared EDT is separable: dt2(x,y,z) = min over features (a,b,c) of
// (x-a)^2 + (y-b)^2 + (z-c)^2.  Three passes:
//   pass z: d1 = distance along z to the nearest feature in the row (uint16,
//           0xFFFF = none), from warp scans over 16-voxel lane segments;
//   pass y: g2(y) = min_j d1(j)^2 + (y-j)^2 over the y column;
//   pass x: dt2(x) = min_j g2(j) + (x-j)^2 over the x column.
// Passes y and x stage a column strip (32 consecutive z, all of the line) in
// shared memory so every global access is a coalesced 64/128-byte row, and
// evaluate each output by a search that widens from j = i outwards and stops
// once (i-j)^2 alone reaches the best value (or the optional cap): exact,
// integer-only, and proportional to the distance itself.
#include <algorithm>
#include <cstdio>
#include <string>
#include <vector>

#include "common.cuh"

namespace {

constexpr int kZWarps = 8;          // rows per block in pass z
constexpr int kStripW = 32;         // z lanes per strip in passes y / x
constexpr int kStripWarps = 16;

// bytes of w equal to zero (or <= a per-byte bound) as 4 bits, lowest
// address first
__device__ __forceinline__ uint32_t byte_bits(uint32_t x)
{
    return (x & 1u) | ((x >> 7) & 2u) | ((x >> 14) & 4u) | ((x >> 21) & 8u);
}

// The feature tests of a pass-z row: bits16 for the
// 16 voxels base+z0 .. base+z0+15 (bit k = voxel z0+k; none past nz).
struct FeatSolid {
    const uint8_t *img;
    __device__ uint32_t bits16(int64_t base, int z0, int nz) const
    {
        const uint8_t *p = img + base + z0;
        if (z0 + 16 <= nz && ((uintptr_t)p & 15) == 0) {
            const uint4 v = __ldg((const uint4 *)p);
            return byte_bits(__vcmpeq4(v.x, 0)) | byte_bits(__vcmpeq4(v.y, 0)) << 4 |
                   byte_bits(__vcmpeq4(v.z, 0)) << 8 | byte_bits(__vcmpeq4(v.w, 0)) << 12;
        }
        uint32_t m = 0;
        for (int k = 0; k < 16 && z0 + k < nz; k++) m |= (uint32_t)(__ldg(p + k) == 0) << k;
        return m;
    }
};
struct FeatAtLeast {
    const int32_t *w;
    int32_t t;
    __device__ uint32_t bits16(int64_t base, int z0, int nz) const
    {
        const int32_t *p = w + base + z0;
        uint32_t m = 0;
        if (z0 + 16 <= nz && ((uintptr_t)p & 15) == 0) {
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int4 v = __ldg((const int4 *)p + q);
                m |= (uint32_t)(v.x >= t) << (4 * q) | (uint32_t)(v.y >= t) << (4 * q + 1) |
                     (uint32_t)(v.z >= t) << (4 * q + 2) | (uint32_t)(v.w >= t) << (4 * q + 3);
            }
            return m;
        }
        for (int k = 0; k < 16 && z0 + k < nz; k++) m |= (uint32_t)(__ldg(p + k) >= t) << k;
        return m;
    }
};
// opening: voxel v belongs to the trimmed set of level i iff its first level
// (the first radius index whose T it reaches) is <= i
struct FeatFirstLevel {
    const uint8_t *fl;
    int i;
    __device__ uint32_t bits16(int64_t base, int z0, int nz) const
    {
        const uint8_t *p = fl + base + z0;
        if (z0 + 16 <= nz && ((uintptr_t)p & 15) == 0) {
            const uint4 v = __ldg((const uint4 *)p);
            const uint32_t b = (uint32_t)i * 0x01010101u;   // i <= 254
            return byte_bits(__vcmpleu4(v.x, b)) | byte_bits(__vcmpleu4(v.y, b)) << 4 |
                   byte_bits(__vcmpleu4(v.z, b)) << 8 | byte_bits(__vcmpleu4(v.w, b)) << 12;
        }
        uint32_t m = 0;
        for (int k = 0; k < 16 && z0 + k < nz; k++) m |= (uint32_t)(__ldg(p + k) <= i) << k;
        return m;
    }
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

// pass z: one warp per row.  A lane takes 16 consecutive voxels (one vector
// load); rows are walked in tiles of 512 voxels, left to right to find each
// lane's nearest feature on the left (warp max-scan, carried across tiles),
// then right to left for the nearest on the right (min-scan), writing the
// distances as packed 16-byte stores.
template <class Feat, int ZW = kZWarps>
__device__ __forceinline__ void edt_z_block(const Feat &feat, int blk, int nrows, int nz, int cap,
                                            uint16_t *__restrict__ d1)
{
    extern __shared__ unsigned char s_zraw[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blk * ZW + w;
    if (row >= nrows) return;   // whole warps only; no block barrier follows
    const int ntile = (nz + 511) >> 9;
    uint16_t *s_m = (uint16_t *)s_zraw + (size_t)w * ntile * 32;
    int *s_l = (int *)(s_zraw + (size_t)ZW * ntile * 64) + (size_t)w * ntile * 32;
    const int64_t base = row * nz;
    const int NONE = 1 << 29;
    int carry = -NONE;
    for (int t = 0; t < ntile; t++) {
        const int z0 = (t << 9) + (lane << 4);
        const uint32_t m = z0 < nz ? feat.bits16(base, z0, nz) : 0u;
        s_m[t * 32 + lane] = (uint16_t)m;
        int last = m ? z0 + 31 - __clz(m) : -NONE;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, last, o);
            if (lane >= o) last = max(last, v);
        }
        int before = __shfl_up_sync(0xffffffffu, last, 1);
        if (lane == 0) before = -NONE;
        s_l[t * 32 + lane] = max(carry, before);
        carry = max(carry, __shfl_sync(0xffffffffu, last, 31));
    }
    int carry_r = NONE;
    for (int t = ntile - 1; t >= 0; t--) {
        const int z0 = (t << 9) + (lane << 4);
        const uint32_t m = s_m[t * 32 + lane];
        const int lb = s_l[t * 32 + lane];
        int first = m ? z0 + __ffs(m) - 1 : NONE;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_down_sync(0xffffffffu, first, o);
            if (lane + o < 32) first = min(first, v);
        }
        int after = __shfl_down_sync(0xffffffffu, first, 1);
        if (lane == 31) after = NONE;
        const int ra = min(carry_r, after);
        carry_r = min(carry_r, __shfl_sync(0xffffffffu, first, 0));
        if (z0 >= nz) continue;
        uint32_t packed[8];
#pragma unroll
        for (int k = 0; k < 16; k++) {
            const int z = z0 + k;
            const uint32_t ml = m & (0xffffu >> (15 - k));   // features at or left of z in this lane
            const uint32_t mr = m >> k;                       // features at or right of z
            const int left = ml ? z0 + 31 - __clz(ml) : lb;
            const int right = mr ? z + __ffs(mr) - 1 : ra;
            const int d = min(z - left, right - z);
            const uint32_t v = d > cap ? 0xffffu : (uint32_t)d;
            if (k & 1) packed[k >> 1] |= v << 16;
            else packed[k >> 1] = v;
        }
        uint16_t *o = d1 + base + z0;
        if (z0 + 16 <= nz && ((uintptr_t)o & 15) == 0) {
            uint4 *o4 = (uint4 *)o;
            o4[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
            o4[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
        } else {
#pragma unroll
            for (int k = 0; k < 16; k++)   // static indices keep packed[] in registers
                if (z0 + k < nz) o[k] = (uint16_t)(packed[k >> 1] >> ((k & 1) * 16));
        }
    }
}

template <class Feat, int ZW = kZWarps>
__global__ void __launch_bounds__(ZW * 32) k_edt_z(Feat feat, int nrows, int nz, int cap, uint16_t *__restrict__ d1)
{
    edt_z_block<Feat, ZW>(feat, blockIdx.x, nrows, nz, cap, d1);
}

size_t edt_z_smem(int nz, int zw = kZWarps) { return (size_t)zw * ((nz + 511) >> 9) * 32 * 6; }

// Sentinel of the partial sums: larger than any squared distance of an image
// within the dimension limits (3 * 16383^2 < 2^30), and small enough that
// adding a squared offset (< 2^28) cannot overflow.
constexpr int kNone = 1 << 30;

// One min-plus line search: min over j of f(j) + (i - j)^2, where `g(j)`
// returns f(j) or kNone.  The search widens from j = i and stops once the
// squared offset alone reaches the best value so far (or `lim`).  Returns a
// value >= lim when nothing below lim exists.
template <class G>
__device__ __forceinline__ int line_min(const G &g, int i, int n, int lim)
{
    int best = min(g(i), lim);
    const int dmax = max(i, n - 1 - i);
    int dd = 1;
#pragma unroll 2
    for (int d = 1; d <= dmax && dd < best; d++) {
        const int vl = i - d >= 0 ? g(i - d) : kNone;
        const int vr = i + d < n ? g(i + d) : kNone;
        best = min(best, min(vl, vr) + dd);
        dd += 2 * d + 1;
    }
    return best;
}

// The same search over a staged column in shared memory (`col` points at
// entry 0 of this lane's column, entries kStripW apart): both sides while
// both are inside the line, then the remaining side alone.
__device__ __forceinline__ int line_min_smem(const int32_t *col, int i, int n, int lim)
{
    const int32_t *c = col + i * kStripW;
    int best = min(c[0], lim);
    const int both = min(i, n - 1 - i);
    int d = 1, dd = 1;
#pragma unroll 2
    for (; d <= both && dd < best; d++) {
        best = min(best, min(c[-d * kStripW], c[d * kStripW]) + dd);
        dd += 2 * d + 1;
    }
    if (dd < best) {
        const int step = i - d >= 0 ? -kStripW : kStripW;   // the side still inside
        const int end = step < 0 ? i : n - 1 - i;
        for (; d <= end && dd < best; d++) {
            best = min(best, c[d * step] + dd);
            dd += 2 * d + 1;
        }
    }
    return best;
}

// The search for output i continued from distance d (dd = d * d), each
// side while it is inside the line.
__device__ __forceinline__ int line_min_smem_from(const int32_t *col, int i, int n, int best, int d, int dd)
{
    const int32_t *c = col + i * kStripW;
    for (; dd < best && (d <= i || d <= n - 1 - i); d++) {
        const int vl = d <= i ? c[-d * kStripW] : kNone;
        const int vr = d <= n - 1 - i ? c[d * kStripW] : kNone;
        best = min(best, min(vl, vr) + dd);
        dd += 2 * d + 1;
    }
    return best;
}

// Four consecutive outputs i0 .. i0 + 3 (all inside the line) of the same
// search.  The windows of the four outputs move together: at distance d,
// output k needs f(i0 + k - d) and f(i0 + k + d), so the left ends
// (L0..L3) and right ends (R0..R3) shift by one entry per step and each
// step loads two entries for four outputs.  Past an end of the line each
// output finishes alone.
__device__ __forceinline__ void line_min4_smem(const int32_t *col, int i0, int n, int lim, int (&b)[4])
{
    const int32_t *c = col + i0 * kStripW;
    int L0 = c[0], L1 = c[kStripW], L2 = c[2 * kStripW], L3 = c[3 * kStripW];
    int R0 = L0, R1 = L1, R2 = L2, R3 = L3;
    b[0] = min(L0, lim); b[1] = min(L1, lim); b[2] = min(L2, lim); b[3] = min(L3, lim);
    const int both = min(i0, n - 4 - i0);
    int d = 1, dd = 1;
    int bmax = max(max(b[0], b[1]), max(b[2], b[3]));
    for (; d <= both && dd < bmax; d++) {
        L3 = L2; L2 = L1; L1 = L0; L0 = c[-d * kStripW];
        R0 = R1; R1 = R2; R2 = R3; R3 = c[(3 + d) * kStripW];
        b[0] = min(b[0], min(L0, R0) + dd);
        b[1] = min(b[1], min(L1, R1) + dd);
        b[2] = min(b[2], min(L2, R2) + dd);
        b[3] = min(b[3], min(L3, R3) + dd);
        dd += 2 * d + 1;
        bmax = max(max(b[0], b[1]), max(b[2], b[3]));
    }
    if (dd < bmax) {
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (dd < b[k]) b[k] = line_min_smem_from(col, i0 + k, n, b[k], d, dd);
    }
}

// 16-byte asynchronous copies global -> shared (bypassing L1): a strip's
// rows are all in flight at once, with no registers holding them
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Shared memory of a staged pass-y block: the int32 squares of the column
// strip, plus (when rows of the pass-z output start on 16-byte boundaries,
// nz % 8 == 0) the raw uint16 strip that the asynchronous copies land in.
__host__ __device__ __forceinline__ size_t edt_y_smem(int ny, int nz)
{
    return (size_t)ny * kStripW * sizeof(int32_t) + ((nz & 7) == 0 ? (size_t)ny * kStripW * sizeof(uint16_t) : 0);
}

// pass y: strip = (x, all y, 32 z).  blockIdx.x = z strip, blockIdx.y = x.
// Output: partial sums < cap2, kNone elsewhere.  The staged column holds
// the squared pass-z distances.
// the staged body of pass y for z strip `strip` of plane x
template <int SW = kStripWarps>
__device__ __forceinline__ void edt_y_block_smem(const uint16_t *__restrict__ d1, int ny, int nz, int cap2,
                                                 int32_t *__restrict__ g2, int strip, int x)
{
    extern __shared__ int32_t s_col[];
    __shared__ int s_any[kStripW];   // per z lane: the column holds a feature
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int z = strip * kStripW + lane;
    const bool ok = z < nz;
    const int64_t b = (int64_t)x * ny * nz + z;
    const int lim = min(cap2, kNone);
    if (threadIdx.x < kStripW) s_any[threadIdx.x] = 0;
    __syncthreads();
    bool any = false;
    if ((nz & 7) == 0) {
        // rows of 32 uint16 as four 16-byte pieces, copied asynchronously
        // into the raw strip (pieces past nz hold "no feature"), then
        // squared into the column; element i of the strip is z lane i % 32
        uint16_t *s_raw = (uint16_t *)(s_col + (size_t)ny * kStripW);
        const int zs = strip * kStripW;
        const int npc = min(4, (nz - zs) >> 3);
        const uint16_t *row0 = d1 + (int64_t)x * ny * nz + zs;
        for (int q = threadIdx.x; q < ny * 4; q += blockDim.x) {
            const int y = q >> 2, pc = q & 3;
            uint16_t *dst = s_raw + y * kStripW + pc * 8;
            if (pc < npc) {
                cp_async16(dst, row0 + (int64_t)y * nz + pc * 8);
            } else {
#pragma unroll
                for (int k = 0; k < 8; k++) dst[k] = 0xffff;
            }
        }
        cp_async_wait_all();
        __syncthreads();
        for (int i = threadIdx.x; i < ny * kStripW; i += blockDim.x) {   // i % 32 == lane
            const int v = s_raw[i];
            any |= v != 0xffff;
            s_col[i] = v == 0xffff ? kNone : v * v;
        }
    } else {
#pragma unroll 8
        for (int y = w; y < ny; y += SW) {
            const int v = ok ? __ldg(d1 + b + (int64_t)y * nz) : 0xffff;
            any |= v != 0xffff;
            s_col[y * kStripW + lane] = v == 0xffff ? kNone : v * v;
        }
    }
    if (any) s_any[lane] = 1;
    __syncthreads();
    if (!ok) return;
    if (!s_any[lane]) {   // no feature in the column: nothing within reach
        for (int y = w; y < ny; y += SW) g2[b + (int64_t)y * nz] = kNone;
        return;
    }
    // four consecutive outputs per warp and pass, the tail one at a time
    const int ny4 = ny & ~3;
    for (int y0 = 4 * w; y0 < ny4; y0 += 4 * SW) {
        int v[4];
        line_min4_smem(s_col + lane, y0, ny, lim, v);
#pragma unroll
        for (int k = 0; k < 4; k++) g2[b + (int64_t)(y0 + k) * nz] = v[k] >= lim ? kNone : v[k];
    }
    for (int y = ny4 + w; y < ny; y += SW) {
        const int v = line_min_smem(s_col + lane, y, ny, lim);
        g2[b + (int64_t)y * nz] = v >= lim ? kNone : v;
    }
}

template <bool SMEM, int SW = kStripWarps>
__global__ void __launch_bounds__(SW * 32) k_edt_y(const uint16_t *__restrict__ d1, int ny, int nz, int cap2,
                                                   int32_t *__restrict__ g2)
{
    if (SMEM) {
        edt_y_block_smem<SW>(d1, ny, nz, cap2, g2, blockIdx.x, blockIdx.y);
        return;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int x = blockIdx.y, z = blockIdx.x * kStripW + lane;
    const bool ok = z < nz;
    const int64_t b = (int64_t)x * ny * nz + z;
    const int lim = min(cap2, kNone);
    if (!ok) return;
    auto g = [&](int j) -> int {
        const int v = __ldg(d1 + b + (int64_t)j * nz);
        return v == 0xffff ? kNone : v * v;
    };
    for (int y = w; y < ny; y += SW) {
        const int v = line_min(g, y, ny, lim);
        g2[b + (int64_t)y * nz] = v >= lim ? kNone : v;
    }
}

// Epilogues of pass x: need(v) says whether voxel v's value is wanted at all
// (the search is skipped otherwise), operator() takes it.
struct EpiStore {
    int32_t *out;
    __device__ bool need(int64_t) const { return true; }
    __device__ void operator()(int64_t v, int val) const { out[v] = val; }
};
// MIO: voxels within the dilation that have no level yet get `lvl`; voxels
// with a level (solid, or an earlier level) keep it and need no search.
struct EpiLevel {
    int32_t *level;
    int32_t T, lvl;
    __device__ bool need(int64_t v) const { return level[v] == -1; }
    __device__ void operator()(int64_t v, int val) const
    {
        if (val < T) level[v] = lvl;
    }
};

// pass x: strip = (y, all x, 32 z).  blockIdx.x = z strip, blockIdx.y = y.
// Final values >= cap2 (or no feature at all) are reported as IBIP_INF32.
// the staged body of pass x for z strip `strip` of row y
template <class Epi, int SW = kStripWarps>
__device__ __forceinline__ void edt_x_block_smem(const int32_t *__restrict__ g2, int nx, int ny, int nz, int cap2,
                                                 const Epi &epi, int strip, int y)
{
    extern __shared__ int32_t s_colx[];
    __shared__ int s_anyx[kStripW];   // per z lane: the column holds a finite partial sum
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int z = strip * kStripW + lane;
    const bool ok = z < nz;
    const int64_t st = (int64_t)ny * nz;
    const int64_t b = (int64_t)y * nz + z;
    const int lim = min(cap2, kNone);
    if (threadIdx.x < kStripW) s_anyx[threadIdx.x] = 0;
    __syncthreads();
    bool any = false;
    if ((nz & 3) == 0) {
        // rows of 32 int32 as eight 16-byte pieces copied asynchronously
        // straight into the column (pieces past nz hold kNone)
        const int zs = strip * kStripW;
        const int npc = min(8, (nz - zs) >> 2);
        const int32_t *row0 = g2 + (int64_t)y * nz + zs;
        for (int q = threadIdx.x; q < nx * 8; q += blockDim.x) {
            const int xr = q >> 3, pc = q & 7;
            int32_t *dst = s_colx + xr * kStripW + pc * 4;
            if (pc < npc) {
                cp_async16(dst, row0 + (int64_t)xr * st + pc * 4);
            } else {
                dst[0] = kNone; dst[1] = kNone; dst[2] = kNone; dst[3] = kNone;
            }
        }
        cp_async_wait_all();
        __syncthreads();
        for (int x = w; x < nx; x += SW) any |= s_colx[x * kStripW + lane] != kNone;
    } else {
#pragma unroll 8
        for (int x = w; x < nx; x += SW) {
            const int v = ok ? __ldg(g2 + b + x * st) : kNone;
            any |= v != kNone;
            s_colx[x * kStripW + lane] = v;
        }
    }
    if (any) s_anyx[lane] = 1;
    __syncthreads();
    if (!ok) return;
    const bool none = !s_anyx[lane];   // nothing within reach: every value is IBIP_INF32
    if (none) {
        for (int x = w; x < nx; x += SW)
            if (epi.need(b + x * st)) epi(b + x * st, IBIP_INF32);
        return;
    }
    // four consecutive outputs per warp and pass (skipped when none is
    // wanted), the tail one at a time
    const int nx4 = nx & ~3;
    for (int x0 = 4 * w; x0 < nx4; x0 += 4 * SW) {
        bool nd[4];
#pragma unroll
        for (int k = 0; k < 4; k++) nd[k] = epi.need(b + (int64_t)(x0 + k) * st);
        if (!(nd[0] || nd[1] || nd[2] || nd[3])) continue;
        int v[4];
        line_min4_smem(s_colx + lane, x0, nx, lim, v);
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (nd[k]) epi(b + (int64_t)(x0 + k) * st, v[k] >= lim ? IBIP_INF32 : v[k]);
    }
    for (int x = nx4 + w; x < nx; x += SW) {
        if (!epi.need(b + x * st)) continue;
        const int v = line_min_smem(s_colx + lane, x, nx, lim);
        epi(b + x * st, v >= lim ? IBIP_INF32 : v);
    }
}

template <bool SMEM, class Epi, int SW = kStripWarps>
__global__ void __launch_bounds__(SW * 32) k_edt_x(const int32_t *__restrict__ g2, int nx, int ny, int nz, int cap2,
                                                   Epi epi)
{
    if (SMEM) {
        edt_x_block_smem<Epi, SW>(g2, nx, ny, nz, cap2, epi, blockIdx.x, blockIdx.y);
        return;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int y = blockIdx.y, z = blockIdx.x * kStripW + lane;
    const bool ok = z < nz;
    const int64_t st = (int64_t)ny * nz;
    const int64_t b = (int64_t)y * nz + z;
    const int lim = min(cap2, kNone);
    if (!ok) return;
    auto g = [&](int j) -> int { return __ldg(g2 + b + j * st); };
    for (int x = w; x < nx; x += SW) {
        if (!epi.need(b + x * st)) continue;
        const int v = line_min(g, x, nx, lim);
        epi(b + x * st, v >= lim ? IBIP_INF32 : v);
    }
}

constexpr size_t kSmemBudget = 200 * 1024;

template <class Feat, class Epi, int ZW = kZWarps, int SW = kStripWarps>
int edt_passes(ibip_ctx *ctx, Feat feat, ibip_dims d, int cap, int cap2, Epi epi, int cls)
{
    int64_t N = nvox(d);
    uint16_t *d1 = (uint16_t *)ibip_scratch(ctx, SC_D1, N * sizeof(uint16_t));
    int32_t *g2 = (int32_t *)ibip_scratch(ctx, SC_G2, N * sizeof(int32_t));
    if (!d1 || !g2) return IBIP_ERR_OOM;
    cudaStream_t s = ctx->stream;
    int nrows = d.nx * d.ny;
    ibip_prof_begin(ctx, cls);
    k_edt_z<Feat, ZW><<<(nrows + ZW - 1) / ZW, ZW * 32, edt_z_smem(d.nz, ZW), s>>>(feat, nrows, d.nz, cap, d1);
    IBIP_LAUNCH(ctx);
    dim3 gy((d.nz + kStripW - 1) / kStripW, d.nx);
    size_t sy = edt_y_smem(d.ny, d.nz);
    if (sy <= kSmemBudget) {
        cudaFuncSetAttribute(k_edt_y<true, SW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget);
        k_edt_y<true, SW><<<gy, SW * 32, sy, s>>>(d1, d.ny, d.nz, cap2, g2);
    } else {
        k_edt_y<false, SW><<<gy, SW * 32, 0, s>>>(d1, d.ny, d.nz, cap2, g2);
    }
    IBIP_LAUNCH(ctx);
    dim3 gx((d.nz + kStripW - 1) / kStripW, d.ny);
    size_t sx = (size_t)d.nx * kStripW * sizeof(int32_t);
    if (sx <= kSmemBudget) {
        cudaFuncSetAttribute(k_edt_x<true, Epi, SW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget);
        k_edt_x<true, Epi, SW><<<gx, SW * 32, sx, s>>>(g2, d.nx, d.ny, d.nz, cap2, epi);
    } else {
        k_edt_x<false, Epi, SW><<<gx, SW * 32, 0, s>>>(g2, d.nx, d.ny, d.nz, cap2, epi);
    }
    IBIP_LAUNCH(ctx);
    ibip_prof_end(ctx, cls);
    return ibip_cuda_status(cudaGetLastError());
}

// ---- the three passes for many images, one launch per pass: each block
// finds its image by binary search over the images' first blocks
struct EdtJob {
    const uint8_t *img;
    int32_t *dt2;
    uint16_t *d1;
    int32_t *g2;
    int nx, ny, nz;
    int blk_z, blk_y, blk_x;
};

__device__ __forceinline__ int find_ejob(const EdtJob *jobs, int n, int blk, int pass)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        const int f = pass == 0 ? jobs[mid].blk_z : pass == 1 ? jobs[mid].blk_y : jobs[mid].blk_x;
        if (f <= blk) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kZWarps * 32) k_edt_z_b(const EdtJob *__restrict__ jobs, int n)
{
    const EdtJob &J = jobs[find_ejob(jobs, n, blockIdx.x, 0)];
    edt_z_block(FeatSolid{J.img}, blockIdx.x - J.blk_z, J.nx * J.ny, J.nz, 0xfffe, J.d1);
}

__global__ void __launch_bounds__(kStripWarps * 32) k_edt_y_b(const EdtJob *__restrict__ jobs, int n)
{
    const EdtJob &J = jobs[find_ejob(jobs, n, blockIdx.x, 1)];
    const int lb = blockIdx.x - J.blk_y, ns = (J.nz + kStripW - 1) / kStripW;
    edt_y_block_smem(J.d1, J.ny, J.nz, IBIP_INF32, J.g2, lb % ns, lb / ns);
}

__global__ void __launch_bounds__(kStripWarps * 32) k_edt_x_b(const EdtJob *__restrict__ jobs, int n)
{
    const EdtJob &J = jobs[find_ejob(jobs, n, blockIdx.x, 2)];
    const int lb = blockIdx.x - J.blk_x, ns = (J.nz + kStripW - 1) / kStripW;
    edt_x_block_smem(J.g2, J.nx, J.ny, J.nz, IBIP_INF32, EpiStore{J.dt2}, lb % ns, lb / ns);
}

}  // namespace

// ---- tile shapes of the squared EDT: rows per block of pass z and warps
// per block of passes y and x.  Entry 0 is the built-in shape.
namespace {

struct EdtTile {
    int zw, sw;
};
constexpr EdtTile kEdtTiles[] = {{8, 16}, {4, 16}, {16, 16}, {8, 8}, {4, 8}, {16, 8}};
constexpr int kNEdtTiles = (int)(sizeof(kEdtTiles) / sizeof(kEdtTiles[0]));

int edt_run_tile(ibip_ctx *ctx, int t, const uint8_t *image, ibip_dims d, int32_t *dt2)
{
    const FeatSolid f{image};
    const EpiStore e{dt2};
    switch (t) {
    case 1: return edt_passes<FeatSolid, EpiStore, 4, 16>(ctx, f, d, 0xfffe, IBIP_INF32, e, IBIP_K_EDT);
    case 2: return edt_passes<FeatSolid, EpiStore, 16, 16>(ctx, f, d, 0xfffe, IBIP_INF32, e, IBIP_K_EDT);
    case 3: return edt_passes<FeatSolid, EpiStore, 8, 8>(ctx, f, d, 0xfffe, IBIP_INF32, e, IBIP_K_EDT);
    case 4: return edt_passes<FeatSolid, EpiStore, 4, 8>(ctx, f, d, 0xfffe, IBIP_INF32, e, IBIP_K_EDT);
    case 5: return edt_passes<FeatSolid, EpiStore, 16, 8>(ctx, f, d, 0xfffe, IBIP_INF32, e, IBIP_K_EDT);
    default: return edt_passes<FeatSolid, EpiStore, 8, 16>(ctx, f, d, 0xfffe, IBIP_INF32, e, IBIP_K_EDT);
    }
}

int ceil_log2(int v)
{
    int c = 0;
    while ((1 << c) < v) c++;
    return c;
}

// shape class: each dimension rounded up to a power of two, and the SM count
std::string edt_key(const ibip_ctx *ctx, ibip_dims d)
{
    char k[96];
    snprintf(k, sizeof(k), "edt:%d.%d.%d:sm%d", ceil_log2(d.nx), ceil_log2(d.ny), ceil_log2(d.nz), ctx->sm_count);
    return k;
}

// Time every tile shape on this call's own input (each run writes the same
// dt2) and keep the fastest: one warm-up run, then the best of three.
int edt_tune(ibip_ctx *ctx, const uint8_t *image, ibip_dims d, int32_t *dt2, int *best_out, double *us_out)
{
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return IBIP_ERR_CUDA;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return IBIP_ERR_CUDA;
    }
    int best = 0, st = IBIP_OK;
    float best_ms = 1e30f;
    for (int t = 0; t < kNEdtTiles && st == IBIP_OK; t++) {
        st = edt_run_tile(ctx, t, image, d, dt2);
        float ms_min = 1e30f;
        for (int r = 0; r < 3 && st == IBIP_OK; r++) {
            cudaEventRecord(a, ctx->stream);
            st = edt_run_tile(ctx, t, image, d, dt2);
            cudaEventRecord(b, ctx->stream);
            if (st == IBIP_OK) st = ibip_cuda_status(cudaEventSynchronize(b));
            float ms = 0.f;
            if (st == IBIP_OK && cudaEventElapsedTime(&ms, a, b) == cudaSuccess) ms_min = std::min(ms_min, ms);
        }
        if (st == IBIP_OK && ms_min < best_ms) { best_ms = ms_min; best = t; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *best_out = best;
    *us_out = best_ms * 1e3;
    return st;
}

int edt_tile_for(ibip_ctx *ctx, ibip_dims d)
{
    if (ctx->edt_tile > 0) return ctx->edt_tile - 1;
    int t = 0;
    if (ctx->autotune && ibip_tune_get(edt_key(ctx, d), &t) && t >= 0 && t < kNEdtTiles) return t;
    return 0;
}

}  // namespace

int ibip_edt_launch(ibip_ctx *ctx, const uint8_t *image, ibip_dims d, int32_t *dt2)
{
    if (ctx->edt_tile == 0 && ctx->autotune) {
        const std::string key = edt_key(ctx, d);
        int t = 0;
        if (!ibip_tune_get(key, &t)) {
            double us = 0.0;
            const int st = edt_tune(ctx, image, d, dt2, &t, &us);
            if (st) return st;
            ibip_tune_put(key, t, us, ctx->tune_path);
        }
    }
    return edt_run_tile(ctx, edt_tile_for(ctx, d), image, d, dt2);
}

int ibip_edt_tile_set(ibip_ctx *ctx, int z_warps, int strip_warps)
{
    if (z_warps == 0 && strip_warps == 0) {
        ctx->edt_tile = 0;
        return IBIP_OK;
    }
    for (int t = 0; t < kNEdtTiles; t++)
        if (kEdtTiles[t].zw == z_warps && kEdtTiles[t].sw == strip_warps) {
            ctx->edt_tile = t + 1;
            return IBIP_OK;
        }
    return IBIP_ERR_ARG;
}

void ibip_edt_tile_get(ibip_ctx *ctx, ibip_dims d, int *z_warps, int *strip_warps)
{
    const EdtTile &t = kEdtTiles[edt_tile_for(ctx, d)];
    *z_warps = t.zw;
    *strip_warps = t.sw;
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

int ibip_dilate_level_launch(ibip_ctx *ctx, const int32_t *W, int32_t T, int32_t Td, int32_t lvl, ibip_dims d,
                             int32_t *level)
{
    // Only squared distances < Td matter: a 1-D distance r with r*r >= Td
    // is as good as none, and every partial sum >= Td is capped.
    int cap = 0;
    while ((int64_t)(cap + 1) * (cap + 1) < Td && cap < 0xfffe) cap++;
    return edt_passes(ctx, FeatAtLeast{W, T}, d, cap, Td, EpiLevel{level, Td, lvl}, IBIP_K_DILATE);
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
    k_edt_z<FeatSolid><<<(nrows + kZWarps - 1) / kZWarps, kZWarps * 32, edt_z_smem(d.nz), s>>>(FeatSolid{image}, nrows,
                                                                                              d.nz, 0xfffe, d1);
    dim3 gy((d.nz + kStripW - 1) / kStripW, d.nx);
    const size_t sy = edt_y_smem(d.ny, d.nz);
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

int ibip_edt_batch_launch(ibip_ctx *ctx, int n, const uint8_t *const *images, const ibip_dims *dims,
                          int32_t *const *dt2)
{
    cudaStream_t s = ctx->stream;
    if (n <= 0) return IBIP_OK;
    std::vector<EdtJob> jobs(n);
    int64_t vox = 0;
    size_t smz = 0, smy = 0, smx = 0;
    int bz = 0, by = 0, bx = 0;
    for (int j = 0; j < n; j++) {
        const ibip_dims d = dims[j];
        EdtJob &J = jobs[j];
        J.img = images[j]; J.dt2 = dt2[j];
        J.nx = d.nx; J.ny = d.ny; J.nz = d.nz;
        const int ns = (d.nz + kStripW - 1) / kStripW;
        J.blk_z = bz; bz += (d.nx * d.ny + kZWarps - 1) / kZWarps;
        J.blk_y = by; by += ns * d.nx;
        J.blk_x = bx; bx += ns * d.ny;
        smz = std::max(smz, edt_z_smem(d.nz));
        smy = std::max(smy, edt_y_smem(d.ny, d.nz));
        smx = std::max(smx, (size_t)d.nx * kStripW * sizeof(int32_t));
        vox += (nvox(d) + 63) & ~(int64_t)63;
    }
    if (smy > kSmemBudget || smx > kSmemBudget) {
        // a column too long to stage: one image at a time
        for (int j = 0; j < n; j++) {
            const int st = ibip_edt_launch(ctx, images[j], dims[j], dt2[j]);
            if (st) return st;
        }
        return IBIP_OK;
    }
    uint16_t *d1 = (uint16_t *)ibip_scratch(ctx, SC_D1, (size_t)vox * sizeof(uint16_t));
    int32_t *g2 = (int32_t *)ibip_scratch(ctx, SC_G2, (size_t)vox * sizeof(int32_t));
    const size_t tab = (size_t)n * sizeof(EdtJob);
    EdtJob *dj = (EdtJob *)ibip_scratch(ctx, SC_BJOBS, tab);
    if (!d1 || !g2 || !dj) return IBIP_ERR_OOM;
    int64_t off = 0;
    for (int j = 0; j < n; j++) {
        jobs[j].d1 = d1 + off;
        jobs[j].g2 = g2 + off;
        off += (nvox(dims[j]) + 63) & ~(int64_t)63;
    }
    ibip_prof_begin(ctx, IBIP_K_EDT);
    cudaMemcpyAsync(dj, jobs.data(), tab, cudaMemcpyHostToDevice, s);
    cudaFuncSetAttribute(k_edt_y_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget);
    cudaFuncSetAttribute(k_edt_x_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget);
    k_edt_z_b<<<bz, kZWarps * 32, smz, s>>>(dj, n);
    IBIP_LAUNCH(ctx);
    k_edt_y_b<<<by, kStripWarps * 32, smy, s>>>(dj, n);
    IBIP_LAUNCH(ctx);
    k_edt_x_b<<<bx, kStripWarps * 32, smx, s>>>(dj, n);
    IBIP_LAUNCH(ctx);
    ibip_prof_end(ctx, IBIP_K_EDT);
    return ibip_cuda_status(cudaGetLastError());
}
