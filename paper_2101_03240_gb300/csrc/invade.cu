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
#include "common.cuh"

namespace {

constexpr int kM = 64;           // batch size (items per iteration)
constexpr int kNT = 512;         // threads of the persistent CTA
constexpr int kChunk = 4096;     // voxels per rank-sort chunk (minimum)
constexpr int kSmemL1Max = 12288;

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

// ------------------------------------------------------- invasion state --

struct Inv {
    int nx, ny, nz, NW, inlet;
    int NL0, NL1, NL2, NL3;
    int64_t max_steps, cap, npore;
    const int32_t *rank;
    const int2 *okey;
    const int32_t *dt2;
    uint32_t *avail, *added;
    u64 *fb0, *fb1, *fb2, *fb3;
    int32_t *seq, *step_r2, *step_centre;
    int64_t *out;      // out[0] = steps, out[1] = status, out[2] = iterations
};

__global__ void k_seq_init(const int32_t *__restrict__ dt2, int64_t N, int32_t *seq)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
        seq[v] = dt2[v] > 0 ? -1 : 0;
}

// one thread per bit-plane word: avail bits, inlet-face candidates
__global__ void k_plane_init(Inv a)
{
    const int64_t nw = (int64_t)a.nx * a.ny * a.NW;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
        int64_t row = w / a.NW;
        int zw = (int)(w - row * a.NW);
        int x = (int)(row / a.ny), y = (int)(row - (int64_t)x * a.ny);
        uint32_t av = 0, ad = 0;
        for (int b = 0; b < 32; b++) {
            int z = zw * 32 + b;
            if (z >= a.nz) break;
            int64_t v = row * a.nz + z;
            if (a.dt2[v] <= 0) continue;
            av |= 1u << b;
            if (d_on_face(x, y, z, a.nx, a.ny, a.nz, a.inlet)) {
                ad |= 1u << b;
                int r = a.rank[v];
                atomicOr(a.fb0 + (r >> 6), 1ull << (r & 63));
                atomicOr(a.fb1 + (r >> 12), 1ull << ((r >> 6) & 63));
                atomicOr(a.fb2 + (r >> 18), 1ull << ((r >> 12) & 63));
                atomicOr(a.fb3 + (r >> 24), 1ull << ((r >> 18) & 63));
            }
        }
        a.avail[w] = av;
        a.added[w] = ad;
    }
}

struct Batch {
    int idx[kM], r2[kM], x[kM], y[kM], z[kM], rank[kM], step[kM];
    int bx0[kM], by0[kM], wy[kM];
    int upre[kM + 1];
    u64 ovl[kM];
    u64 keep;
    int m, mcap, J, nsteps, stop;
};

// bits [a, b] (inclusive, within word w of a row) as a mask
__device__ __forceinline__ uint32_t span_mask(int w, int a, int b)
{
    int lo = max(a - w * 32, 0), hi = min(b - w * 32, 31);
    if (lo > hi) return 0u;
    uint32_t m = 0xffffffffu >> (31 - hi);
    return m & (0xffffffffu << lo);
}

// z-interval of ball i at row (x, y): returns false if the row misses it
__device__ __forceinline__ bool ball_run(const Batch &B, int i, int x, int y, int &lo, int &hi)
{
    int dx = x - B.x[i], dy = y - B.y[i];
    int64_t e = (int64_t)B.r2[i] - 1 - (int64_t)dx * dx - (int64_t)dy * dy;
    if (e < 0) return false;
    int h = d_isqrt((int)e);
    lo = B.z[i] - h;
    hi = B.z[i] + h;
    return true;
}

// Candidate intervals next to ball i's run [lo, hi] at row (x, y): the two
// z-ends and the parts of the four lateral rows outside ball i.  Calls
// f(xr, yr, a, b) per non-empty interval (clamped to the image).
template <class F>
__device__ __forceinline__ void for_each_shell(const Inv &a, const Batch &B, int i, int x, int y, int lo,
                                               int hi, F f)
{
    int z0 = max(lo, 0), z1 = min(hi, a.nz - 1);
    if (lo - 1 >= 0) f(x, y, lo - 1, lo - 1);
    if (hi + 1 <= a.nz - 1) f(x, y, hi + 1, hi + 1);
    const int DX[4] = {-1, 1, 0, 0}, DY[4] = {0, 0, -1, 1};
#pragma unroll
    for (int q = 0; q < 4; q++) {
        int xr = x + DX[q], yr = y + DY[q];
        if (xr < 0 || yr < 0 || xr >= a.nx || yr >= a.ny) continue;
        int l2, h2;
        if (!ball_run(B, i, xr, yr, l2, h2)) {
            f(xr, yr, z0, z1);
        } else {
            if (z0 <= l2 - 1) f(xr, yr, z0, min(z1, l2 - 1));
            if (h2 + 1 <= z1) f(xr, yr, max(z0, h2 + 1), z1);
        }
    }
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

__device__ __forceinline__ int unit_item(const Batch &B, int n, int u)
{
    int lo = 0, hi = n;   // largest i with upre[i] <= u
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (B.upre[mid] <= u) lo = mid; else hi = mid;
    }
    return lo;
}

template <bool L1SMEM>
__global__ void __launch_bounds__(kNT, 1) k_invade(Inv a)
{
    extern __shared__ u64 s_fb[];
    __shared__ Batch B;
    u64 *s1 = L1SMEM ? s_fb : a.fb1;
    u64 *s2 = s_fb + (L1SMEM ? a.NL1 : 0);
    u64 *s3 = s2 + a.NL2;
    const int tid = threadIdx.x, lane = tid & 31;
    if (L1SMEM)
        for (int i = tid; i < a.NL1; i += kNT) s1[i] = a.fb1[i];
    for (int i = tid; i < a.NL2; i += kNT) s2[i] = a.fb2[i];
    for (int i = tid; i < a.NL3; i += kNT) s3[i] = a.fb3[i];
    __syncthreads();

    int64_t k = 0, iters = 0;
    for (;;) {
        // ---------------------------------------------------- select batch
        if (tid < 32) {
            int i0 = -1;
            if (lane == 0) {
                for (;;) {
                    int i3 = -1;
                    for (int t = 0; t < a.NL3; t++) if (s3[t]) { i3 = t; break; }
                    if (i3 < 0) break;
                    int i2 = i3 * 64 + __ffsll(s3[i3]) - 1;
                    u64 w2 = s2[i2];
                    if (!w2) { s3[i3] &= ~(1ull << (i2 & 63)); continue; }
                    int i1 = i2 * 64 + __ffsll(w2) - 1;
                    u64 w1 = L1SMEM ? s1[i1] : ldcg64(s1 + i1);
                    if (!w1) {
                        s2[i2] &= ~(1ull << (i1 & 63));
                        if (!s2[i2]) s3[i3] &= ~(1ull << (i2 & 63));
                        continue;
                    }
                    int c0 = i1 * 64 + __ffsll(w1) - 1;
                    u64 w0 = ldcg64(a.fb0 + c0);
                    if (!w0) {
                        u64 nw1 = w1 & ~(1ull << (c0 & 63));
                        s1[i1] = nw1;
                        if (!nw1) {
                            s2[i2] &= ~(1ull << (i1 & 63));
                            if (!s2[i2]) s3[i3] &= ~(1ull << (i2 & 63));
                        }
                        continue;
                    }
                    i0 = c0;
                    break;
                }
            }
            i0 = __shfl_sync(0xffffffffu, i0, 0);
            int m = 0;
            if (i0 >= 0) {
                int wi = i0 + lane;
                u64 w = wi < a.NL0 ? ldcg64(a.fb0 + wi) : 0ull;
                int c = __popcll(w);
                int inc = c;
                for (int o = 1; o < 32; o <<= 1) {
                    int t = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += t;
                }
                int tot = __shfl_sync(0xffffffffu, inc, 31);
                m = min(tot, kM);
                int pos = inc - c;
                while (w && pos < m) {
                    B.rank[pos] = wi * 64 + __ffsll(w) - 1;
                    w &= w - 1;
                    pos++;
                }
            }
            __syncwarp();
            // item data
            const int64_t nyz = (int64_t)a.ny * a.nz;
            for (int j = lane; j < m; j += 32) {
                int2 e = __ldg(a.okey + B.rank[j]);
                B.idx[j] = e.x;
                B.r2[j] = e.y;
                int x = (int)(e.x / nyz), rem = (int)(e.x - (int64_t)x * nyz);
                int y = rem / a.nz, z = rem - y * a.nz;
                B.x[j] = x; B.y[j] = y; B.z[j] = z;
                int h = d_ball_hw(e.y);
                int x0 = max(x - h, 0), x1 = min(x + h, a.nx - 1);
                int y0 = max(y - h, 0), y1 = min(y + h, a.ny - 1);
                B.bx0[j] = x0; B.by0[j] = y0; B.wy[j] = y1 - y0 + 1;
                B.upre[j + 1] = (x1 - x0 + 1) * (y1 - y0 + 1);   // rows, fixed below
            }
            __syncwarp();
            // Pairwise tests, looping only over items whose ball is more than
            // the centre voxel (r2 > 1): two distinct r2 == 1 balls never
            // meet.  cont: item j lies in the ball of an earlier item b;
            // ovl: the ball boxes of j and b, grown by one voxel, intersect.
            int hj[2];
            u64 cont[2] = {0ull, 0ull}, ovl[2] = {0ull, 0ull};
            bool bg[2];
            for (int q = 0; q < 2; q++) {
                int j = lane + 32 * q;
                bg[q] = j < m && B.r2[j] > 1;
                hj[q] = j < m ? d_ball_hw(B.r2[j]) : 0;
            }
            u64 big = (u64)__ballot_sync(0xffffffffu, bg[0]) | ((u64)__ballot_sync(0xffffffffu, bg[1]) << 32);
            for (u64 bm = big; bm; bm &= bm - 1) {
                const int b = __ffsll(bm) - 1;
                const int bx = B.x[b], by = B.y[b], bz = B.z[b], br2 = B.r2[b];
                const int bh = d_ball_hw(br2);
                u64 hit = 0;
                for (int q = 0; q < 2; q++) {
                    int j = lane + 32 * q;
                    if (j >= m || j == b) continue;
                    int64_t dx = B.x[j] - bx, dy = B.y[j] - by, dz = B.z[j] - bz;
                    if (b < j && dx * dx + dy * dy + dz * dz < (int64_t)br2) cont[q] |= 1ull << b;
                    int64_t lim = bh + hj[q] + 1;
                    if (llabs(dx) <= lim && llabs(dy) <= lim && llabs(dz) <= lim) {
                        ovl[q] |= 1ull << b;
                        hit |= 1ull << j;
                    }
                }
                u64 hall = (u64)__ballot_sync(0xffffffffu, (hit & 0xffffffffull) != 0) |
                           ((u64)__ballot_sync(0xffffffffu, (hit >> 32) != 0) << 32);
                if ((b & 31) == lane) ovl[b >> 5] |= hall;
            }
            u64 has = (u64)__ballot_sync(0xffffffffu, cont[0] != 0) |
                      ((u64)__ballot_sync(0xffffffffu, cont[1] != 0) << 32);
            u64 valid = m == 64 ? ~0ull : ((1ull << m) - 1);
            u64 keep = valid & ~has;
            u64 pend = has & valid;
            while (pend) {
                int j = __ffsll(pend) - 1;
                pend &= pend - 1;
                u64 cj = __shfl_sync(0xffffffffu, j < 32 ? cont[0] : cont[1], j & 31);
                if (!(cj & keep)) keep |= 1ull << j;
            }
            for (int q = 0; q < 2; q++) {
                int j = lane + 32 * q;
                if (j < m) B.ovl[j] = ovl[q];
            }
            // step limit
            int mcap = m;
            int64_t remain = a.max_steps - k;
            int nkeep = __popcll(keep);
            if ((int64_t)nkeep > remain) {
                u64 t = keep;
                for (int64_t q = 0; q < remain; q++) t &= t - 1;
                mcap = __ffsll(t) - 1;   // first item beyond the limit
            }
            for (int h = 0; h < 2; h++) {
                int j = lane + 32 * h;
                if (j < m) {
                    bool kp = (keep >> j) & 1;
                    B.step[j] = kp ? __popcll(keep & ((1ull << j) - 1)) : -1;
                    if (!kp || j >= mcap) B.upre[j + 1] = 0;
                }
            }
            __syncwarp();
            if (lane == 0) {
                // row units, prefix-summed; a batch never holds more than 2^30
                // of them (keeps the unit index in an int)
                B.upre[0] = 0;
                for (int j = 0; j < m; j++) {
                    if (j > 0 && j < mcap && (int64_t)B.upre[j] + B.upre[j + 1] > (1 << 30)) mcap = j;
                    B.upre[j + 1] = j < mcap ? B.upre[j] + B.upre[j + 1] : B.upre[j];
                }
                B.m = m;
                B.mcap = mcap;
                B.J = mcap;
                B.stop = (m == 0) ? 1 : (mcap == 0 ? 2 : 0);
                B.keep = keep;
            }
        }
        __syncthreads();
        if (B.stop) break;
        if (k > a.npore) {   // every step invades its own centre: cannot happen
            if (tid == 0) B.stop = 3;
            break;
        }
        const int mcap = B.mcap, m = B.m;

        // ---------------------------------------------------- shell pass
        {
            const int U = B.upre[mcap];
            for (int u = tid; u < U; u += kNT) {
                int i = unit_item(B, mcap + 1, u);
                if (i + 1 >= *(volatile int *)&B.J) continue;   // cannot tighten J
                int t = u - B.upre[i];
                int x = B.bx0[i] + t / B.wy[i], y = B.by0[i] + t % B.wy[i];
                int lo, hi;
                if (!ball_run(B, i, x, y, lo, hi)) continue;
                for_each_shell(a, B, i, x, y, lo, hi, [&](int xr, int yr, int za, int zb) {
                    int64_t rb = ((int64_t)xr * a.ny + yr) * a.NW;
                    int64_t vb = ((int64_t)xr * a.ny + yr) * a.nz;
                    for (int w = za >> 5; w <= (zb >> 5); w++) {
                        uint32_t cand = ldcg32(a.avail + rb + w) & ~ldcg32(a.added + rb + w) & span_mask(w, za, zb);
                        while (cand) {
                            int z = w * 32 + __ffs(cand) - 1;
                            cand &= cand - 1;
                            int ru = __ldg(a.rank + vb + z);
                            int c = max(i + 1, lower_rank(B, m, ru));
                            atomicMin(&B.J, c);
                        }
                    }
                });
            }
        }
        __syncthreads();

        // --------------------------------------------------- commit pass
        {
            const int J = B.J;
            const u64 jmask = J >= 64 ? ~0ull : ((1ull << J) - 1);
            const int64_t k1 = k + 1;
            const int U = B.upre[J];
            for (int u = tid; u < U; u += kNT) {
                int i = unit_item(B, J + 1, u);
                int t = u - B.upre[i];
                int x = B.bx0[i] + t / B.wy[i], y = B.by0[i] + t % B.wy[i];
                int lo, hi;
                if (!ball_run(B, i, x, y, lo, hi)) continue;
                const int z0 = max(lo, 0), z1 = min(hi, a.nz - 1);
                const int64_t rb = ((int64_t)x * a.ny + y) * a.NW;
                const int64_t vb = ((int64_t)x * a.ny + y) * a.nz;
                const int32_t label = (int32_t)(k1 + B.step[i]);
                for (int w = z0 >> 5; w <= (z1 >> 5); w++) {
                    uint32_t own = span_mask(w, z0, z1);
                    for (u64 om = B.ovl[i] & B.keep & ((1ull << i) - 1); om && own; om &= om - 1) {
                        int i2 = __ffsll(om) - 1, l2, h2;
                        if (ball_run(B, i2, x, y, l2, h2)) own &= ~span_mask(w, l2, h2);
                    }
                    if (!own) continue;
                    uint32_t newly = ldcg32(a.avail + rb + w) & own;
                    if (!newly) continue;
                    atomicAnd(a.avail + rb + w, ~newly);
                    uint32_t gone = newly & ldcg32(a.added + rb + w);
                    uint32_t n2 = newly;
                    while (n2) {
                        int z = w * 32 + __ffs(n2) - 1;
                        n2 &= n2 - 1;
                        a.seq[vb + z] = label;
                    }
                    while (gone) {
                        int z = w * 32 + __ffs(gone) - 1;
                        gone &= gone - 1;
                        int r = __ldg(a.rank + vb + z);
                        atomicAnd(a.fb0 + (r >> 6), ~(1ull << (r & 63)));
                    }
                }
                for_each_shell(a, B, i, x, y, lo, hi, [&](int xr, int yr, int za, int zb) {
                    int64_t rb2 = ((int64_t)xr * a.ny + yr) * a.NW;
                    int64_t vb2 = ((int64_t)xr * a.ny + yr) * a.nz;
                    for (int w = za >> 5; w <= (zb >> 5); w++) {
                        uint32_t msk = span_mask(w, za, zb);
                        for (u64 om = B.ovl[i] & B.keep & jmask; om && msk; om &= om - 1) {
                            int i2 = __ffsll(om) - 1, l2, h2;
                            if (ball_run(B, i2, xr, yr, l2, h2)) msk &= ~span_mask(w, l2, h2);
                        }
                        if (!msk) continue;
                        uint32_t cand = ldcg32(a.avail + rb2 + w) & ~ldcg32(a.added + rb2 + w) & msk;
                        if (!cand) continue;
                        atomicOr(a.added + rb2 + w, cand);
                        while (cand) {
                            int z = w * 32 + __ffs(cand) - 1;
                            cand &= cand - 1;
                            int r = __ldg(a.rank + vb2 + z);
                            atomicOr(a.fb0 + (r >> 6), 1ull << (r & 63));
                            atomicOr(s1 + (r >> 12), 1ull << ((r >> 6) & 63));
                            atomicOr(s2 + (r >> 18), 1ull << ((r >> 12) & 63));
                            atomicOr(s3 + (r >> 24), 1ull << ((r >> 18) & 63));
                        }
                    }
                });
            }
            for (int j = tid; j < J; j += kNT) {
                if (B.step[j] < 0) continue;
                int64_t s = k + B.step[j];
                if (s < a.cap) {
                    a.step_r2[s] = B.r2[j];
                    if (a.step_centre) a.step_centre[s] = B.idx[j];
                }
            }
        }
        // steps committed: kept items below J
        k += __popcll(B.keep & (B.J >= 64 ? ~0ull : ((1ull << B.J) - 1)));
        iters++;
        __syncthreads();
    }
    if (tid == 0) {
        a.out[0] = k;
        a.out[1] = (B.stop == 2) ? IBIP_ERR_STEP_LIMIT : (B.stop == 3 ? IBIP_ERR_BOUNDS : IBIP_OK);
        a.out[2] = iters;
    }
}

}  // namespace

// --------------------------------------------------------------- launcher --

int ibip_invade_run(ibip_ctx *ctx, const int32_t *dt2, ibip_dims d, int inlet, int64_t max_steps,
                    int32_t *seq, int32_t *step_r2, int32_t *step_centre, int64_t cap, int64_t *h_out)
{
    cudaStream_t s = ctx->stream;
    const int64_t N = nvox(d);
    int *stats = (int *)ibip_scratch(ctx, SC_SMALL, 256);
    if (!stats) return IBIP_ERR_OOM;
    int *h = (int *)ctx->h_pinned;
    ibip_prof_begin(ctx, IBIP_K_RANK);
    cudaMemsetAsync(stats, 0, 3 * sizeof(int), s);
    int gs = ctx->sm_count * 8;
    k_stats<<<gs, 256, 0, s>>>(dt2, N, stats);
    IBIP_LAUNCH(ctx);
    cudaMemcpyAsync(h, stats, 3 * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return IBIP_ERR_CUDA;
    const int maxd = h[0], npore = h[1], hasinf = h[2];

    k_seq_init<<<gs, 256, 0, s>>>(dt2, N, seq);
    IBIP_LAUNCH(ctx);
    if (npore == 0) {
        ibip_prof_end(ctx, IBIP_K_RANK);
        h_out[0] = 0; h_out[1] = IBIP_OK; h_out[2] = 0;
        return ibip_cuda_status(cudaStreamSynchronize(s));
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
        if (cudaStreamSynchronize(s) != cudaSuccess) return IBIP_ERR_CUDA;
        B = h[0];
    }
    Bucket bk{incl, B, hasinf};

    // -- stable counting sort by bucket
    int64_t S = kChunk;
    while ((N + S - 1) / S * (int64_t)B > (1ll << 26)) S *= 2;
    const int C = (int)((N + S - 1) / S);
    int32_t *mat = (int32_t *)ibip_scratch(ctx, SC_MAT, (size_t)C * B * sizeof(int32_t));
    int32_t *rank = (int32_t *)ibip_scratch(ctx, SC_RANK, (size_t)N * sizeof(int32_t));
    int2 *okey = (int2 *)ibip_scratch(ctx, SC_OKEY, (size_t)npore * sizeof(int2));
    if (!mat || !rank || !okey) return IBIP_ERR_OOM;
    const bool smem = B <= 1024;
    const int wpb = 4;
    size_t sm = smem ? (size_t)wpb * B * sizeof(int32_t) : 0;
    int nb = (C + wpb - 1) / wpb;
    if (smem) k_chunk_hist<true><<<nb, wpb * 32, sm, s>>>(dt2, N, (int)S, C, bk, mat);
    else k_chunk_hist<false><<<nb, wpb * 32, 0, s>>>(dt2, N, (int)S, C, bk, mat);
    IBIP_LAUNCH(ctx);
    int st = ibip_scan_excl_i32(ctx, mat, mat, (int64_t)C * B);
    if (st) return st;
    if (smem) k_chunk_scatter<true><<<nb, wpb * 32, sm, s>>>(dt2, N, (int)S, C, bk, mat, rank, okey);
    else k_chunk_scatter<false><<<nb, wpb * 32, 0, s>>>(dt2, N, (int)S, C, bk, mat, rank, okey);
    IBIP_LAUNCH(ctx);

    // -- bit-planes and the candidate bitmap
    Inv a;
    a.nx = d.nx; a.ny = d.ny; a.nz = d.nz; a.NW = (d.nz + 31) / 32; a.inlet = inlet;
    a.NL0 = (npore + 63) / 64;
    a.NL1 = (a.NL0 + 63) / 64;
    a.NL2 = (a.NL1 + 63) / 64;
    a.NL3 = (a.NL2 + 63) / 64;
    a.max_steps = max_steps;
    a.cap = cap;
    a.npore = npore;
    a.rank = rank; a.okey = okey; a.dt2 = dt2;
    const int64_t nw = (int64_t)d.nx * d.ny * a.NW;
    a.avail = (uint32_t *)ibip_scratch(ctx, SC_AVAIL, nw * sizeof(uint32_t));
    a.added = (uint32_t *)ibip_scratch(ctx, SC_ADDED, nw * sizeof(uint32_t));
    size_t nfb = (size_t)a.NL0 + a.NL1 + a.NL2 + a.NL3;
    u64 *fb = (u64 *)ibip_scratch(ctx, SC_FB, nfb * sizeof(u64));
    int64_t *out = (int64_t *)ibip_scratch(ctx, SC_SMALL, 256);
    if (!a.avail || !a.added || !fb || !out) return IBIP_ERR_OOM;
    out += 8;
    a.fb0 = fb; a.fb1 = fb + a.NL0; a.fb2 = a.fb1 + a.NL1; a.fb3 = a.fb2 + a.NL2;
    a.seq = seq; a.step_r2 = step_r2; a.step_centre = step_centre; a.out = out;
    cudaMemsetAsync(fb, 0, nfb * sizeof(u64), s);
    k_plane_init<<<gs, 256, 0, s>>>(a);
    IBIP_LAUNCH(ctx);
    ibip_prof_end(ctx, IBIP_K_RANK);

    const bool l1smem = a.NL1 <= kSmemL1Max;
    size_t dyn = ((l1smem ? a.NL1 : 0) + (size_t)a.NL2 + a.NL3) * sizeof(u64);
    ibip_prof_begin(ctx, IBIP_K_INVADE);
    if (l1smem) {
        cudaFuncSetAttribute(k_invade<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn + 1024);
        k_invade<true><<<1, kNT, dyn, s>>>(a);
    } else {
        cudaFuncSetAttribute(k_invade<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn + 1024);
        k_invade<false><<<1, kNT, dyn, s>>>(a);
    }
    IBIP_LAUNCH(ctx);
    ibip_prof_end(ctx, IBIP_K_INVADE);
    int64_t *ho = (int64_t *)ctx->h_pinned;
    cudaMemcpyAsync(ho, out, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ibip_cuda_status(e);
    h_out[0] = ho[0]; h_out[1] = ho[1]; h_out[2] = ho[2];
    return IBIP_OK;
}
