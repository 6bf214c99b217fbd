/*
 * ibip_oracle.c -- plain, slow CPU oracle for image-based invasion
 * percolation (IBIP; Gostick, Yang & Boek, "Simulating volume-controlled
 * invasion of a non-wetting fluid in volumetric images using basic image
 * processing tools", arXiv 2101.03240).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference for the
 * CUDA library.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no source, header, table or helper
 * with the CUDA path, and the CUDA path never calls it.
 *
 * Conventions (the paper is silent on all of them):
 *   - image shape (nx, ny, nz), C order, idx = (x*ny + y)*nz + z;
 *   - image byte nonzero = pore (void), 0 = solid; 6-connectivity;
 *   - voxels outside the image are NOT solid;
 *   - dt2: squared Euclidean distance to the nearest solid voxel, 0 on solid,
 *     INT32_MAX on pore when the image has no solid at all;
 *   - seq: 0 solid, -1 pore never invaded, k >= 1 invaded at step k;
 *   - faces: 0=X0 (x=0) 1=X1 (x=nx-1) 2=Y0 3=Y1 4=Z0 5=Z1.
 *
 * Each function names the passage of the paper it follows.  Everything is
 * written for obviousness, not speed, except where a second, faster variant
 * is provided for large images; every fast variant is checked bit-exact
 * against its plain twin by the tests.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_INF32 INT32_MAX
#define OR_OK 0
#define OR_STEP_LIMIT (-4)
#define OR_CAPACITY (-1)

static int64_t lin(int64_t x, int64_t y, int64_t z, int64_t ny, int64_t nz)
{
    return (x * ny + y) * nz + z;
}

static void coords(int64_t v, int64_t ny, int64_t nz, int64_t *x, int64_t *y, int64_t *z)
{
    *z = v % nz;
    *y = (v / nz) % ny;
    *x = v / (nz * ny);
}

static int on_face(int64_t x, int64_t y, int64_t z, int nx, int ny, int nz, int face)
{
    switch (face) {
    case 0: return x == 0;
    case 1: return x == nx - 1;
    case 2: return y == 0;
    case 3: return y == ny - 1;
    case 4: return z == 0;
    case 5: return z == nz - 1;
    default: return 0;
    }
}

static const int NB[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};

/* largest r >= 0 with r*r < r2 (r2 >= 1), i.e. the half-width of the ball
 * d^2 < r2 along one axis */
static int64_t ball_halfwidth(int64_t r2)
{
    int64_t r = (int64_t)sqrt((double)(r2 - 1));
    while (r > 0 && r * r > r2 - 1) r--;
    while ((r + 1) * (r + 1) <= r2 - 1) r++;
    return r;
}

/* ------------------------------------------------------------------------
 * Distance transform of the pore space (Section 2.1, Figure 2b).  dt2 is
 * the squared Euclidean distance from each pore voxel to the nearest solid
 * voxel.
 * ---------------------------------------------------------------------- */

/* EDT-brute: the definition written out.  O(N * Nsolid). */
void or_edt_brute(const uint8_t *img, int nx, int ny, int nz, int32_t *dt2)
{
    int64_t N = (int64_t)nx * ny * nz, ns = 0;
    int64_t *sx = malloc(sizeof(int64_t) * (N ? N : 1) * 3);
    for (int64_t v = 0; v < N; v++)
        if (!img[v]) {
            int64_t x, y, z;
            coords(v, ny, nz, &x, &y, &z);
            sx[3 * ns] = x; sx[3 * ns + 1] = y; sx[3 * ns + 2] = z;
            ns++;
        }
    for (int64_t v = 0; v < N; v++) {
        if (!img[v]) { dt2[v] = 0; continue; }
        if (ns == 0) { dt2[v] = OR_INF32; continue; }
        int64_t x, y, z, best = INT64_MAX;
        coords(v, ny, nz, &x, &y, &z);
        for (int64_t s = 0; s < ns; s++) {
            int64_t dx = x - sx[3 * s], dy = y - sx[3 * s + 1], dz = z - sx[3 * s + 2];
            int64_t d = dx * dx + dy * dy + dz * dz;
            if (d < best) best = d;
        }
        dt2[v] = (int32_t)best;
    }
    free(sx);
}

/* One 1-D min-plus pass  g'(i) = min_j g(j) + (i-j)^2  along a line of n
 * values with stride s.  INT32_MAX marks "no feature seen on this line"
 * (every real value is below 2^30, a squared offset below 2^28, so sums
 * stay below INT32_MAX).  The search walks j outward from i and stops once
 * (i-j)^2 alone is no smaller than the best value found, or than `limit`:
 * every later term is at least that large.  Values below `limit` are
 * therefore exact; at or above it the output is only known to be >= limit
 * (INT64_MAX = no limit). */
static void minplus_line(const int32_t *g, int32_t *out, int64_t n, int64_t s, int64_t limit)
{
    for (int64_t i = 0; i < n; i++) {
        int64_t best = g[i * s];
        for (int64_t d = 1; d < n; d++) {
            if (best != INT32_MAX && d * d >= best) break;
            if (d * d >= limit) break;
            int64_t j0 = i - d, j1 = i + d;
            if (j0 < 0 && j1 >= n) break;
            if (j0 >= 0 && g[j0 * s] != INT32_MAX && g[j0 * s] + d * d < best) best = g[j0 * s] + d * d;
            if (j1 < n && g[j1 * s] != INT32_MAX && g[j1 * s] + d * d < best) best = g[j1 * s] + d * d;
        }
        out[i * s] = (int32_t)best;
    }
}

/* The same pass over m neighbouring lines at once: element i of line k is
 * g[i * s + k] (k = 0..m-1 contiguous in memory), so every step of the
 * search reads m consecutive values.  The search for output row i stops
 * once (i-j)^2 is no smaller than every line's best value, or than
 * `limit`. */
static void minplus_rows(const int32_t *g, int32_t *out, int64_t n, int64_t s, int64_t m, int64_t limit,
                         int64_t *best)
{
    for (int64_t i = 0; i < n; i++) {
        int64_t worst = 0;
        for (int64_t k = 0; k < m; k++) {
            best[k] = g[i * s + k];
            if (best[k] > worst) worst = best[k];
        }
        for (int64_t d = 1; d < n; d++) {
            if (worst != INT32_MAX && d * d >= worst) break;
            if (d * d >= limit) break;
            int64_t j0 = i - d, j1 = i + d;
            if (j0 < 0 && j1 >= n) break;
            worst = 0;
            for (int64_t k = 0; k < m; k++) {
                if (j0 >= 0 && g[j0 * s + k] != INT32_MAX && g[j0 * s + k] + d * d < best[k])
                    best[k] = g[j0 * s + k] + d * d;
                if (j1 < n && g[j1 * s + k] != INT32_MAX && g[j1 * s + k] + d * d < best[k])
                    best[k] = g[j1 * s + k] + d * d;
                if (best[k] > worst) worst = best[k];
            }
        }
        for (int64_t k = 0; k < m; k++) out[i * s + k] = (int32_t)best[k];
    }
}

/* EDT-sep: the squared EDT is separable (a sum of squared per-axis offsets),
 * so three 1-D min-plus passes give the same value as EDT-brute.  `feat`
 * marks the feature voxels the distance is taken to (solid for the pore
 * EDT).  Output INT32_MAX where no feature exists in the whole image.
 * Outputs below `limit` are exact; the others are only >= limit (a term
 * at or above the limit in one pass stays at or above it in the next, since
 * every pass adds a non-negative square).  a, b: work arrays of N int32. */
static void edt_sep_work(const uint8_t *feat, int nx, int ny, int nz, int32_t *out, int64_t limit, int32_t *a,
                         int32_t *b)
{
    int64_t N = (int64_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < N; v++) a[v] = feat[v] ? 0 : INT32_MAX;
    /* along z */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < (int64_t)nx * ny; r++) minplus_line(a + r * nz, b + r * nz, nz, 1, limit);
    /* along y: the nz lines of one x slab together */
#pragma omp parallel
    {
        int64_t *best = malloc(sizeof(int64_t) * (nz > 0 ? nz : 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t x = 0; x < nx; x++) minplus_rows(b + x * ny * nz, a + x * ny * nz, ny, nz, nz, limit, best);
        free(best);
    }
    /* along x: the nz lines of one y row together, into the output */
#pragma omp parallel
    {
        int64_t *best = malloc(sizeof(int64_t) * (nz > 0 ? nz : 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t y = 0; y < ny; y++) minplus_rows(a + y * nz, out + y * nz, nx, (int64_t)ny * nz, nz, limit, best);
        free(best);
    }
}

static void edt_sep_core(const uint8_t *feat, int nx, int ny, int nz, int32_t *out, int64_t limit)
{
    int64_t N = (int64_t)nx * ny * nz;
    int32_t *a = malloc(sizeof(int32_t) * (N ? N : 1));
    int32_t *b = malloc(sizeof(int32_t) * (N ? N : 1));
    edt_sep_work(feat, nx, ny, nz, out, limit, a, b);
    free(a);
    free(b);
}

void or_edt_sep(const uint8_t *img, int nx, int ny, int nz, int32_t *dt2)
{
    int64_t N = (int64_t)nx * ny * nz;
    uint8_t *solid = malloc(N ? N : 1);
    for (int64_t v = 0; v < N; v++) solid[v] = img[v] == 0;
    edt_sep_core(solid, nx, ny, nz, dt2, INT64_MAX);
    free(solid);
}

/* ------------------------------------------------------------------------
 * Invasion (Section 2.1, Figures 1 and 2).  Each step picks the candidate
 * voxel with the largest distance value and inserts a sphere there, writing
 * the step number only into voxels not invaded before.
 *
 * Readings used (the paper describes a variant; these fix the variant):
 *   candidates = uninvaded pore voxels that are 6-adjacent to an invaded
 *                voxel, or lie on the inlet face (the face behaves as an
 *                invaded reservoir just outside the image);
 *   one sphere per step; equal dt2 -> lowest linear index;
 *   the sphere of step k is {p : |p - c|^2 < dt2[c]}.
 * ---------------------------------------------------------------------- */

/* write step k into every uninvaded voxel of the ball; returns how many */
static int64_t stamp(int32_t *seq, int nx, int ny, int nz, int64_t c, int64_t r2, int32_t k,
                     int64_t *newlist)
{
    int64_t cx, cy, cz, n = 0;
    coords(c, ny, nz, &cx, &cy, &cz);
    int64_t r = ball_halfwidth(r2);
    int64_t x0 = cx - r < 0 ? 0 : cx - r, x1 = cx + r > nx - 1 ? nx - 1 : cx + r;
    int64_t y0 = cy - r < 0 ? 0 : cy - r, y1 = cy + r > ny - 1 ? ny - 1 : cy + r;
    int64_t z0 = cz - r < 0 ? 0 : cz - r, z1 = cz + r > nz - 1 ? nz - 1 : cz + r;
    for (int64_t x = x0; x <= x1; x++)
        for (int64_t y = y0; y <= y1; y++)
            for (int64_t z = z0; z <= z1; z++) {
                int64_t d = (x - cx) * (x - cx) + (y - cy) * (y - cy) + (z - cz) * (z - cz);
                if (d >= r2) continue;
                int64_t p = lin(x, y, z, ny, nz);
                if (seq[p] != -1) continue;
                seq[p] = k;
                if (newlist) newlist[n] = p;
                n++;
            }
    return n;
}

static int has_invaded_nb(const int32_t *seq, int nx, int ny, int nz, int64_t x, int64_t y, int64_t z)
{
    for (int d = 0; d < 6; d++) {
        int64_t a = x + NB[d][0], b = y + NB[d][1], c = z + NB[d][2];
        if (a < 0 || b < 0 || c < 0 || a >= nx || b >= ny || c >= nz) continue;
        if (seq[lin(a, b, c, ny, nz)] >= 1) return 1;
    }
    return 0;
}

/* Invade-scan: every step rescans the whole image for the candidate set,
 * exactly as the definition reads.  O(steps * N).  Returns the number of
 * steps K; *status = OR_STEP_LIMIT if max_steps stopped a non-empty front. */
/* inlet voxels: the given mask (nonzero = inlet; Section 2.1 marks the
 * inlets with a Boolean image of the image's shape), else the
 * inlet face */
static int is_inlet(const uint8_t *mask, int64_t v, int64_t x, int64_t y, int64_t z, int nx, int ny, int nz,
                    int inlet)
{
    return mask ? mask[v] != 0 : on_face(x, y, z, nx, ny, nz, inlet);
}

int64_t or_invade_scan_mask(const uint8_t *img, const int32_t *dt2, int nx, int ny, int nz, int inlet,
                            const uint8_t *mask, int64_t max_steps, int32_t *seq, int32_t *step_r2,
                            int32_t *step_centre, int64_t cap, int *status)
{
    int64_t N = (int64_t)nx * ny * nz, k = 0;
    for (int64_t v = 0; v < N; v++) seq[v] = img[v] ? -1 : 0;
    *status = OR_OK;
    for (;;) {
        int64_t best = -1, bestd = -1;
        for (int64_t v = 0; v < N; v++) {
            if (seq[v] != -1) continue;
            int64_t x, y, z;
            coords(v, ny, nz, &x, &y, &z);
            if (!is_inlet(mask, v, x, y, z, nx, ny, nz, inlet) && !has_invaded_nb(seq, nx, ny, nz, x, y, z)) continue;
            if (dt2[v] > bestd) { bestd = dt2[v]; best = v; }
        }
        if (best < 0) break;
        if (k >= max_steps) { *status = OR_STEP_LIMIT; break; }
        k++;
        stamp(seq, nx, ny, nz, best, bestd, (int32_t)k, NULL);
        if (k <= cap) {
            step_r2[k - 1] = (int32_t)bestd;
            if (step_centre) step_centre[k - 1] = (int32_t)best;
        }
    }
    return k;
}

/* max-heap of 64-bit keys; key = dt2 << 32 | (0xffffffff - idx), so the
 * largest key is the largest dt2 with the smallest index */
typedef struct { uint64_t *a; int64_t n, cap; } heap_t;

static void hpush(heap_t *h, uint64_t key)
{
    if (h->n == h->cap) {
        h->cap = h->cap ? 2 * h->cap : 1024;
        h->a = realloc(h->a, sizeof(uint64_t) * h->cap);
    }
    int64_t i = h->n++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h->a[p] >= key) break;
        h->a[i] = h->a[p];
        i = p;
    }
    h->a[i] = key;
}

static uint64_t hpop(heap_t *h)
{
    uint64_t top = h->a[0], last = h->a[--h->n];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        uint64_t mv = last;
        if (l < h->n && h->a[l] > mv) { m = l; mv = h->a[l]; }
        if (r < h->n && h->a[r] > mv) { m = r; mv = h->a[r]; }
        if (m == i) break;
        h->a[i] = h->a[m];
        i = m;
    }
    if (h->n) h->a[i] = last;
    return top;
}

static uint64_t hkey(int32_t d, int64_t idx)
{
    return ((uint64_t)(uint32_t)d << 32) | (uint64_t)(0xffffffffu - (uint32_t)idx);
}

/* Invade-heap: the same process with the candidate set kept in a priority
 * queue (the classic invasion-percolation queue of Wilkinson & Willemsen,
 * cited in Section 1).  A voxel is queued once, when it first becomes a
 * candidate; popped entries already invaded are skipped.  Same result as
 * invade-scan, far faster; used on large images and as the timed CPU
 * baseline. */
int64_t or_invade_heap_mask(const uint8_t *img, const int32_t *dt2, int nx, int ny, int nz, int inlet,
                            const uint8_t *mask, int64_t max_steps, int32_t *seq, int32_t *step_r2,
                            int32_t *step_centre, int64_t cap, int *status)
{
    int64_t N = (int64_t)nx * ny * nz, k = 0;
    uint8_t *queued = calloc(N ? N : 1, 1);
    int64_t *newlist = malloc(sizeof(int64_t) * (N ? N : 1));
    heap_t h = {0};
    for (int64_t v = 0; v < N; v++) {
        seq[v] = img[v] ? -1 : 0;
        int64_t x, y, z;
        coords(v, ny, nz, &x, &y, &z);
        if (img[v] && is_inlet(mask, v, x, y, z, nx, ny, nz, inlet)) {
            queued[v] = 1;
            hpush(&h, hkey(dt2[v], v));
        }
    }
    *status = OR_OK;
    while (h.n) {
        uint64_t key = h.a[0];
        int64_t c = (int64_t)(0xffffffffu - (uint32_t)(key & 0xffffffffu));
        if (seq[c] != -1) { hpop(&h); continue; }
        if (k >= max_steps) { *status = OR_STEP_LIMIT; break; }
        hpop(&h);
        k++;
        int64_t r2 = dt2[c];
        int64_t n = stamp(seq, nx, ny, nz, c, r2, (int32_t)k, newlist);
        if (k <= cap) {
            step_r2[k - 1] = (int32_t)r2;
            if (step_centre) step_centre[k - 1] = (int32_t)c;
        }
        for (int64_t i = 0; i < n; i++) {
            int64_t x, y, z;
            coords(newlist[i], ny, nz, &x, &y, &z);
            for (int d = 0; d < 6; d++) {
                int64_t a = x + NB[d][0], b = y + NB[d][1], cc = z + NB[d][2];
                if (a < 0 || b < 0 || cc < 0 || a >= nx || b >= ny || cc >= nz) continue;
                int64_t q = lin(a, b, cc, ny, nz);
                if (seq[q] != -1 || queued[q]) continue;
                queued[q] = 1;
                hpush(&h, hkey(dt2[q], q));
            }
        }
    }
    free(h.a);
    free(queued);
    free(newlist);
    return k;
}

/* ------------------------------------------------------------------------
 * Trapping (Section 2.2.3).  Thresholding the sequence in decreasing order,
 * a voxel invaded at step k is trapped when, just before step k, it is cut
 * off from the outlet face by invaded voxels: no 6-path through pore voxels
 * whose sequence value is >= k (never-invaded pore counts as +infinity)
 * joins it to a pore voxel on the outlet face.  Only invaded voxels can be
 * trapped; outlet-face voxels never are.
 * ---------------------------------------------------------------------- */

static int64_t seq_inf(int32_t s) { return s == -1 ? INT64_MAX : s; }

static int32_t max_seq(const int32_t *seq, int64_t N)
{
    int32_t K = 0;
    for (int64_t v = 0; v < N; v++) if (seq[v] > K) K = seq[v];
    return K;
}

/* dense rank of the step values that survive (Section 2.2.3: the sequence is
 * re-ranked to be contiguous after trapped voxels are reset) */
static void rerank(int32_t *s, int64_t N)
{
    int32_t K = max_seq(s, N);
    int32_t *map = calloc((size_t)K + 1, sizeof(int32_t));
    for (int64_t v = 0; v < N; v++) if (s[v] >= 1) map[s[v]] = 1;
    int32_t r = 0;
    for (int32_t k = 1; k <= K; k++) if (map[k]) map[k] = ++r;
    for (int64_t v = 0; v < N; v++) if (s[v] >= 1) s[v] = map[s[v]];
    free(map);
}

static void finish_trap(const int32_t *seq, int64_t N, const uint8_t *trapped, int do_rerank, int32_t *seq_out)
{
    if (!seq_out) return;
    for (int64_t v = 0; v < N; v++) seq_out[v] = trapped[v] ? -1 : seq[v];
    if (do_rerank) rerank(seq_out, N);
}

/* Trap-BFS: for every step k, flood from the outlet face through voxels with
 * seq >= k; the step-k voxels not reached are trapped.  O(K * N). */
void or_trap_bfs(const int32_t *seq, int nx, int ny, int nz, int outlet, int do_rerank,
                 uint8_t *trapped, int32_t *seq_out)
{
    int64_t N = (int64_t)nx * ny * nz;
    int32_t K = max_seq(seq, N);
    uint8_t *seen = malloc(N ? N : 1);
    int64_t *q = malloc(sizeof(int64_t) * (N ? N : 1));
    memset(trapped, 0, N);
    for (int32_t k = 1; k <= K; k++) {
        memset(seen, 0, N);
        int64_t qh = 0, qt = 0;
        for (int64_t v = 0; v < N; v++) {
            if (seq[v] == 0 || seq_inf(seq[v]) < k) continue;
            int64_t x, y, z;
            coords(v, ny, nz, &x, &y, &z);
            if (on_face(x, y, z, nx, ny, nz, outlet)) { seen[v] = 1; q[qt++] = v; }
        }
        while (qh < qt) {
            int64_t v = q[qh++], x, y, z;
            coords(v, ny, nz, &x, &y, &z);
            for (int d = 0; d < 6; d++) {
                int64_t a = x + NB[d][0], b = y + NB[d][1], c = z + NB[d][2];
                if (a < 0 || b < 0 || c < 0 || a >= nx || b >= ny || c >= nz) continue;
                int64_t u = lin(a, b, c, ny, nz);
                if (seen[u] || seq[u] == 0 || seq_inf(seq[u]) < k) continue;
                seen[u] = 1;
                q[qt++] = u;
            }
        }
        for (int64_t v = 0; v < N; v++) if (seq[v] == k && !seen[v]) trapped[v] = 1;
    }
    finish_trap(seq, N, trapped, do_rerank, seq_out);
    free(seen);
    free(q);
}

static int64_t uf_find(int64_t *p, int64_t a)
{
    while (p[a] != a) { p[a] = p[p[a]]; a = p[a]; }
    return a;
}

static void uf_union(int64_t *p, int64_t *sz, int64_t a, int64_t b)
{
    a = uf_find(p, a);
    b = uf_find(p, b);
    if (a == b) return;
    if (sz[a] < sz[b]) { int64_t t = a; a = b; b = t; }
    p[b] = a;
    sz[a] += sz[b];
}

/* voxel indices grouped by sequence value: never-invaded pore first, then
 * k = K, K-1, ..., 1 (order[start[g] .. start[g+1]) is group g) */
static void group_desc(const int32_t *seq, int64_t N, int32_t K, int64_t **order_out, int64_t **start_out)
{
    int64_t G = (int64_t)K + 1; /* group 0: seq = -1; group g >= 1: seq = K + 1 - g */
    int64_t *cnt = calloc(G + 1, sizeof(int64_t));
    int64_t *order = malloc(sizeof(int64_t) * (N ? N : 1));
    for (int64_t v = 0; v < N; v++) {
        if (seq[v] == 0) continue;
        int64_t g = seq[v] == -1 ? 0 : (int64_t)K + 1 - seq[v];
        cnt[g + 1]++;
    }
    for (int64_t g = 0; g < G; g++) cnt[g + 1] += cnt[g];
    int64_t *pos = malloc(sizeof(int64_t) * (G + 1));
    memcpy(pos, cnt, sizeof(int64_t) * (G + 1));
    for (int64_t v = 0; v < N; v++) {
        if (seq[v] == 0) continue;
        int64_t g = seq[v] == -1 ? 0 : (int64_t)K + 1 - seq[v];
        order[pos[g]++] = v;
    }
    free(pos);
    *order_out = order;
    *start_out = cnt;
}

/* Trap-UF: the reverse search of Section 2.2.3 (after Masson 2016) done once
 * with a union-find: voxels are added in decreasing sequence order, joined to
 * already-added pore neighbours and to a virtual outlet node; a step-k voxel
 * is trapped iff, after all step-k voxels are added, its set does not hold
 * the outlet node.  Same result as Trap-BFS in O(N alpha(N)). */
void or_trap_uf(const int32_t *seq, int nx, int ny, int nz, int outlet, int do_rerank,
                uint8_t *trapped, int32_t *seq_out)
{
    int64_t N = (int64_t)nx * ny * nz;
    int32_t K = max_seq(seq, N);
    int64_t *order, *start;
    group_desc(seq, N, K, &order, &start);
    int64_t *p = malloc(sizeof(int64_t) * (N + 1)), *sz = malloc(sizeof(int64_t) * (N + 1));
    uint8_t *added = calloc(N ? N : 1, 1);
    for (int64_t v = 0; v <= N; v++) { p[v] = v; sz[v] = 1; }
    memset(trapped, 0, N);
    for (int64_t g = 0; g <= K; g++) {
        for (int64_t i = start[g]; i < start[g + 1]; i++) {
            int64_t v = order[i], x, y, z;
            added[v] = 1;
            coords(v, ny, nz, &x, &y, &z);
            if (on_face(x, y, z, nx, ny, nz, outlet)) uf_union(p, sz, v, N);
            for (int d = 0; d < 6; d++) {
                int64_t a = x + NB[d][0], b = y + NB[d][1], c = z + NB[d][2];
                if (a < 0 || b < 0 || c < 0 || a >= nx || b >= ny || c >= nz) continue;
                int64_t u = lin(a, b, c, ny, nz);
                if (added[u]) uf_union(p, sz, v, u);
            }
        }
        if (g == 0) continue; /* never-invaded voxels are not "trapped" */
        for (int64_t i = start[g]; i < start[g + 1]; i++)
            if (uf_find(p, order[i]) != uf_find(p, N)) trapped[order[i]] = 1;
    }
    finish_trap(seq, N, trapped, do_rerank, seq_out);
    free(order); free(start); free(p); free(sz); free(added);
}

/* ------------------------------------------------------------------------
 * Checks used by the tests to pin the invasion (not part of the method).
 * ---------------------------------------------------------------------- */

/* Number of invaded voxels that are NOT 6-connected to the inlet face
 * through voxels with 1 <= seq <= their own step (voxels added in
 * increasing step order to a union-find with a virtual inlet node). */
int64_t or_count_unconnected(const int32_t *seq, int nx, int ny, int nz, int inlet)
{
    int64_t N = (int64_t)nx * ny * nz, bad = 0;
    int32_t K = max_seq(seq, N);
    int64_t *cnt = calloc((size_t)K + 2, sizeof(int64_t));
    int64_t *order = malloc(sizeof(int64_t) * (N ? N : 1));
    for (int64_t v = 0; v < N; v++) if (seq[v] >= 1) cnt[seq[v] + 1]++;
    for (int32_t k = 0; k <= K; k++) cnt[k + 1] += cnt[k];
    int64_t *pos = malloc(sizeof(int64_t) * ((size_t)K + 2));
    memcpy(pos, cnt, sizeof(int64_t) * ((size_t)K + 2));
    for (int64_t v = 0; v < N; v++) if (seq[v] >= 1) order[pos[seq[v]]++] = v;
    int64_t *p = malloc(sizeof(int64_t) * (N + 1)), *sz = malloc(sizeof(int64_t) * (N + 1));
    for (int64_t v = 0; v <= N; v++) { p[v] = v; sz[v] = 1; }
    for (int32_t k = 1; k <= K; k++) {
        for (int64_t i = cnt[k]; i < cnt[k + 1]; i++) {
            int64_t v = order[i], x, y, z;
            coords(v, ny, nz, &x, &y, &z);
            if (on_face(x, y, z, nx, ny, nz, inlet)) uf_union(p, sz, v, N);
            for (int d = 0; d < 6; d++) {
                int64_t a = x + NB[d][0], b = y + NB[d][1], c = z + NB[d][2];
                if (a < 0 || b < 0 || c < 0 || a >= nx || b >= ny || c >= nz) continue;
                int64_t u = lin(a, b, c, ny, nz);
                if (seq[u] >= 1 && seq[u] <= k) uf_union(p, sz, v, u);
            }
        }
        for (int64_t i = cnt[k]; i < cnt[k + 1]; i++)
            if (uf_find(p, order[i]) != uf_find(p, N)) bad++;
    }
    free(cnt); free(order); free(pos); free(p); free(sz);
    return bad;
}

/* ------------------------------------------------------------------------
 * Morphological image opening drainage, MIO (Section 1 and Section 2.4.1):
 * for decreasing sphere sizes, erode the pore space, trim what is not
 * connected to the inlet (after the erosion, before the dilation), dilate.
 * Level i uses the squared radius T[i] (strictly decreasing):
 *   E_i = {pore v : dt2[v] >= T_i}                       (erosion)
 *   trimmed E_i = members of E_i 6-connected within E_i to E_i's inlet face
 *   D_i = {p : exists c in trimmed E_i with |p - c|^2 < T_i}   (dilation)
 * level[p] = i+1 for the first level i with p in D_i; -1 pore never reached;
 * 0 solid.  counts[i] = number of voxels with 1 <= level <= i+1.
 *
 * The *_td variants take the dilation's bound separately: D_i = {p : exists
 * c in trimmed E_i with |p - c|^2 < Td_i} (Td = T gives the above).  With
 * T_i = R^2 and Td_i = R^2 + 1 for integer radii R the opening uses the ball
 * |p - c|^2 <= R^2, the structuring element of the paper-literal invasion
 * (Section 2.1, footnote 1: integer radius), so that the two can be compared
 * at equal saturation with the structuring element held fixed (Section
 * 3.1.1).
 * ---------------------------------------------------------------------- */

static void mio_trim(const uint8_t *img, const int32_t *dt2, int nx, int ny, int nz, int inlet,
                     int64_t T, uint8_t *trim, int64_t *q)
{
    int64_t N = (int64_t)nx * ny * nz, qh = 0, qt = 0;
    memset(trim, 0, N);
    for (int64_t v = 0; v < N; v++) {
        if (!img[v] || dt2[v] < T) continue;
        int64_t x, y, z;
        coords(v, ny, nz, &x, &y, &z);
        if (on_face(x, y, z, nx, ny, nz, inlet)) { trim[v] = 1; q[qt++] = v; }
    }
    while (qh < qt) {
        int64_t v = q[qh++], x, y, z;
        coords(v, ny, nz, &x, &y, &z);
        for (int d = 0; d < 6; d++) {
            int64_t a = x + NB[d][0], b = y + NB[d][1], c = z + NB[d][2];
            if (a < 0 || b < 0 || c < 0 || a >= nx || b >= ny || c >= nz) continue;
            int64_t u = lin(a, b, c, ny, nz);
            if (trim[u] || !img[u] || dt2[u] < T) continue;
            trim[u] = 1;
            q[qt++] = u;
        }
    }
}

static void mio_counts(const int32_t *level, int64_t N, int32_t L, int64_t *counts)
{
    if (!counts) return;
    for (int32_t i = 0; i < L; i++) counts[i] = 0;
    for (int64_t v = 0; v < N; v++) if (level[v] >= 1 && level[v] <= L) counts[level[v] - 1]++;
    for (int32_t i = 1; i < L; i++) counts[i] += counts[i - 1];
}

/* MIO-plain: dilation by stamping the ball around every trimmed voxel. */
void or_mio_plain_td(const uint8_t *img, const int32_t *dt2, int nx, int ny, int nz, int inlet,
                     const int32_t *T, const int32_t *Td, int32_t L, int32_t *level, int64_t *counts)
{
    int64_t N = (int64_t)nx * ny * nz;
    uint8_t *trim = malloc(N ? N : 1), *dil = malloc(N ? N : 1);
    int64_t *q = malloc(sizeof(int64_t) * (N ? N : 1));
    for (int64_t v = 0; v < N; v++) level[v] = img[v] ? -1 : 0;
    for (int32_t i = 0; i < L; i++) {
        int64_t t = T[i], td = Td[i];
        mio_trim(img, dt2, nx, ny, nz, inlet, t, trim, q);
        memset(dil, 0, N);
        int64_t r = ball_halfwidth(td);
        for (int64_t c = 0; c < N; c++) {
            if (!trim[c]) continue;
            int64_t cx, cy, cz;
            coords(c, ny, nz, &cx, &cy, &cz);
            for (int64_t x = cx - r; x <= cx + r; x++)
                for (int64_t y = cy - r; y <= cy + r; y++)
                    for (int64_t z = cz - r; z <= cz + r; z++) {
                        if (x < 0 || y < 0 || z < 0 || x >= nx || y >= ny || z >= nz) continue;
                        if ((x - cx) * (x - cx) + (y - cy) * (y - cy) + (z - cz) * (z - cz) < td)
                            dil[lin(x, y, z, ny, nz)] = 1;
                    }
        }
        for (int64_t v = 0; v < N; v++) if (dil[v] && level[v] == -1) level[v] = i + 1;
    }
    mio_counts(level, N, L, counts);
    free(trim); free(dil); free(q);
}

void or_mio_plain(const uint8_t *img, const int32_t *dt2, int nx, int ny, int nz, int inlet,
                  const int32_t *T, int32_t L, int32_t *level, int64_t *counts)
{
    or_mio_plain_td(img, dt2, nx, ny, nz, inlet, T, T, L, level, counts);
}

/* MIO-edt: identical result; the dilation of the trimmed set by the ball
 * d^2 < Td is the set where the squared distance to the trimmed set is
 * < Td, computed with EDT-sep taken to the trimmed voxels (exact below Td,
 * which is all the membership test reads). */
void or_mio_edt_td(const uint8_t *img, const int32_t *dt2, int nx, int ny, int nz, int inlet,
                   const int32_t *T, const int32_t *Td, int32_t L, int32_t *level, int64_t *counts)
{
    int64_t N = (int64_t)nx * ny * nz;
    uint8_t *trim = malloc(N ? N : 1);
    int64_t *q = malloc(sizeof(int64_t) * (N ? N : 1));
    int32_t *d = malloc(sizeof(int32_t) * (N ? N : 1));
    int32_t *wa = malloc(sizeof(int32_t) * (N ? N : 1)), *wb = malloc(sizeof(int32_t) * (N ? N : 1));
    for (int64_t v = 0; v < N; v++) level[v] = img[v] ? -1 : 0;
    for (int32_t i = 0; i < L; i++) {
        mio_trim(img, dt2, nx, ny, nz, inlet, T[i], trim, q);
        int any = 0;
        for (int64_t v = 0; v < N && !any; v++) any = trim[v];
        if (!any) continue;   /* nothing trimmed: the dilation is empty */
        edt_sep_work(trim, nx, ny, nz, d, Td[i], wa, wb);
#pragma omp parallel for schedule(static)
        for (int64_t v = 0; v < N; v++) if (d[v] < Td[i] && level[v] == -1) level[v] = i + 1;
    }
    mio_counts(level, N, L, counts);
    free(trim); free(q); free(d); free(wa); free(wb);
}

void or_mio_edt(const uint8_t *img, const int32_t *dt2, int nx, int ny, int nz, int inlet,
                const int32_t *T, int32_t L, int32_t *level, int64_t *counts)
{
    or_mio_edt_td(img, dt2, nx, ny, nz, inlet, T, T, L, level, counts);
}

/* ------------------------------------------------------------------------
 * Saturation and capillary pressure per step (Sections 2.2.1 and 2.2.2,
 * Washburn relation as written in Section 2.4.1: Pc = -2 sigma cos(theta)/R).
 *   cnt[k] = voxels with seq == k;  S_k = (sum_{j<=k} cnt[j]) / Npore,
 *   Npore = every pore voxel of the image (seq != 0);
 *   R_k = sqrt(step_r2[k]) * voxel_m  (the radius of the sphere d^2 < r2);
 *   Pc_k = (-2 sigma cos(theta)) / R_k,  cos(theta) = cos(theta_deg*pi/180).
 * All in double, one rounding to float.  sat_image[v] = S_{seq[v]} for
 * 1 <= seq[v] <= K, +infinity otherwise (never below any threshold).
 * ---------------------------------------------------------------------- */
void or_pc_curve(const int32_t *seq, int64_t N, const int32_t *step_r2, int64_t K, double voxel_m,
                 double sigma, double theta_deg, float *S, float *Pc, float *sat_image)
{
    const double pi = 3.14159265358979323846;
    int64_t *cnt = calloc((size_t)K + 1, sizeof(int64_t));
    int64_t npore = 0;
    for (int64_t v = 0; v < N; v++) {
        if (seq[v] != 0) npore++;
        if (seq[v] >= 1 && seq[v] <= K) cnt[seq[v]]++;
    }
    double ct = cos(theta_deg * pi / 180.0);
    int64_t cum = 0;
    for (int64_t k = 1; k <= K; k++) {
        cum += cnt[k];
        S[k - 1] = (float)((double)cum / (double)npore);
        Pc[k - 1] = (float)((-2.0 * sigma * ct) / (sqrt((double)step_r2[k - 1]) * voxel_m));
    }
    if (sat_image)
        for (int64_t v = 0; v < N; v++)
            sat_image[v] = (seq[v] >= 1 && seq[v] <= K) ? S[seq[v] - 1] : INFINITY;
    free(cnt);
}

/* ------------------------------------------------------------------------
 * Invasion exactly as Section 2.1 prints it (the paper-literal rule; the
 * functions above use the frontier rule instead).  The state is an inlets
 * image and a working copy of the distance values:
 *   1. the candidates are the inlets plus their face neighbours (dilation by
 *      a cross, i.e. a structuring element of radius 1);
 *   2. the largest distance value over the candidates is found, and every
 *      candidate holding it is an insertion point of this step (all tied
 *      maxima at once);
 *   3. at each insertion point c a sphere of integer radius R = trunc(dt)
 *      (footnote 1; dt = sqrt(dt2)) is inserted: every pore voxel p with
 *      |p - c|^2 <= R^2 not invaded before gets the step number;
 *   4. the insertion points join the inlets and their distance values are
 *      set to zero, so they are not chosen again.
 * The loop ends when the largest candidate value is zero.
 * Readings where the text is silent: the inlets start as every voxel of the
 * inlet face; a sphere is the set of voxels within distance R (a ball
 * structuring element of radius R), written only into pore voxels (when dt
 * is an integer the ball reaches the nearest solid voxel); steps whose
 * spheres meet no uninvaded voxel still count.
 * Outputs: seq; cstep[v] = the step at which v was an insertion point (0 if
 * never); per step the squared radius R^2 and the number of insertion
 * points.
 * ---------------------------------------------------------------------- */

/* floor(sqrt(v)) for 0 <= v < 2^31, exact */
static int64_t isqrt_floor(int64_t v)
{
    int64_t r = (int64_t)sqrt((double)v);
    while (r > 0 && r * r > v) r--;
    while ((r + 1) * (r + 1) <= v) r++;
    return r;
}

/* step k's sphere of squared radius rr at c, pore voxels only */
static void stamp_literal(const uint8_t *img, int32_t *seq, int nx, int ny, int nz, int64_t c, int64_t rr,
                          int32_t k)
{
    int64_t cx, cy, cz;
    coords(c, ny, nz, &cx, &cy, &cz);
    int64_t r = isqrt_floor(rr);
    int64_t x0 = cx - r < 0 ? 0 : cx - r, x1 = cx + r > nx - 1 ? nx - 1 : cx + r;
    int64_t y0 = cy - r < 0 ? 0 : cy - r, y1 = cy + r > ny - 1 ? ny - 1 : cy + r;
    int64_t z0 = cz - r < 0 ? 0 : cz - r, z1 = cz + r > nz - 1 ? nz - 1 : cz + r;
    for (int64_t x = x0; x <= x1; x++)
        for (int64_t y = y0; y <= y1; y++)
            for (int64_t z = z0; z <= z1; z++) {
                int64_t d = (x - cx) * (x - cx) + (y - cy) * (y - cy) + (z - cz) * (z - cz);
                if (d > rr) continue;
                int64_t p = lin(x, y, z, ny, nz);
                if (img[p] && seq[p] == -1) seq[p] = k;
            }
}

/* Literal-scan: the steps above with the candidate set rebuilt from the
 * inlets image over the whole image every step.  O(steps * N). */
int64_t or_invade_literal_scan(const uint8_t *img, const int32_t *dt2, int nx, int ny, int nz, int inlet,
                               int64_t max_steps, int32_t *seq, int32_t *cstep, int32_t *step_r2,
                               int32_t *step_count, int64_t cap, int *status)
{
    int64_t N = (int64_t)nx * ny * nz, k = 0;
    uint8_t *inl = calloc(N ? N : 1, 1), *cand = calloc(N ? N : 1, 1);
    int32_t *dt = malloc(sizeof(int32_t) * (N ? N : 1));
    for (int64_t v = 0; v < N; v++) {
        int64_t x, y, z;
        coords(v, ny, nz, &x, &y, &z);
        seq[v] = img[v] ? -1 : 0;
        cstep[v] = 0;
        dt[v] = dt2[v];
        inl[v] = (uint8_t)on_face(x, y, z, nx, ny, nz, inlet);
    }
    *status = OR_OK;
    for (;;) {
        /* 1: inlets dilated by a cross */
        for (int64_t v = 0; v < N; v++) {
            int64_t x, y, z;
            coords(v, ny, nz, &x, &y, &z);
            int c = inl[v];
            for (int d = 0; d < 6 && !c; d++) {
                int64_t a = x + NB[d][0], b = y + NB[d][1], e = z + NB[d][2];
                if (a < 0 || b < 0 || e < 0 || a >= nx || b >= ny || e >= nz) continue;
                c = inl[lin(a, b, e, ny, nz)];
            }
            cand[v] = (uint8_t)c;
        }
        /* 2: the largest value under the candidates */
        int32_t best = 0;
        for (int64_t v = 0; v < N; v++)
            if (cand[v] && dt[v] > best) best = dt[v];
        if (best == 0) break;
        if (k >= max_steps) { *status = OR_STEP_LIMIT; break; }
        k++;
        int64_t R = isqrt_floor(best), count = 0;
        /* 3: a sphere at every maximum */
        for (int64_t v = 0; v < N; v++) {
            if (!cand[v] || dt[v] != best) continue;
            stamp_literal(img, seq, nx, ny, nz, v, R * R, (int32_t)k);
            cstep[v] = (int32_t)k;
            count++;
        }
        /* 4: the insertion points join the inlets; their values drop to 0 */
        for (int64_t v = 0; v < N; v++)
            if (cstep[v] == k) { inl[v] = 1; dt[v] = 0; }
        if (k <= cap) {
            step_r2[k - 1] = (int32_t)(R * R);
            step_count[k - 1] = (int32_t)count;
        }
    }
    free(inl);
    free(cand);
    free(dt);
    return k;
}

/* Literal-queue: the same process with every voxel queued once, when it
 * first becomes a candidate, in a max-heap on its distance value.  A step
 * pops every queued voxel holding the largest value before it queues the
 * neighbours of its insertion points, so voxels that become candidates
 * during step k are first examined at step k + 1, as in the scan. */
int64_t or_invade_literal_queue(const uint8_t *img, const int32_t *dt2, int nx, int ny, int nz, int inlet,
                                int64_t max_steps, int32_t *seq, int32_t *cstep, int32_t *step_r2,
                                int32_t *step_count, int64_t cap, int *status)
{
    int64_t N = (int64_t)nx * ny * nz, k = 0;
    uint8_t *queued = calloc(N ? N : 1, 1);
    int64_t *pts = malloc(sizeof(int64_t) * (N ? N : 1));
    heap_t h = {0};
    for (int64_t v = 0; v < N; v++) {
        seq[v] = img[v] ? -1 : 0;
        cstep[v] = 0;
    }
    /* the inlet face and its face neighbours; zero values never win */
    for (int64_t v = 0; v < N; v++) {
        int64_t x, y, z;
        coords(v, ny, nz, &x, &y, &z);
        if (!on_face(x, y, z, nx, ny, nz, inlet)) continue;
        for (int d = -1; d < 6; d++) {
            int64_t a = x, b = y, e = z;
            if (d >= 0) { a += NB[d][0]; b += NB[d][1]; e += NB[d][2]; }
            if (a < 0 || b < 0 || e < 0 || a >= nx || b >= ny || e >= nz) continue;
            int64_t u = lin(a, b, e, ny, nz);
            if (queued[u] || dt2[u] == 0) continue;
            queued[u] = 1;
            hpush(&h, hkey(dt2[u], u));
        }
    }
    *status = OR_OK;
    while (h.n > 0) {
        int32_t best = (int32_t)(h.a[0] >> 32);
        if (k >= max_steps) { *status = OR_STEP_LIMIT; break; }
        k++;
        int64_t R = isqrt_floor(best), n = 0;
        while (h.n > 0 && (int32_t)(h.a[0] >> 32) == best) {
            uint64_t key = hpop(&h);
            pts[n++] = (int64_t)(0xffffffffu - (uint32_t)(key & 0xffffffffu));
        }
        for (int64_t q = 0; q < n; q++) {
            stamp_literal(img, seq, nx, ny, nz, pts[q], R * R, (int32_t)k);
            cstep[pts[q]] = (int32_t)k;
        }
        for (int64_t q = 0; q < n; q++) {
            int64_t x, y, z;
            coords(pts[q], ny, nz, &x, &y, &z);
            for (int d = 0; d < 6; d++) {
                int64_t a = x + NB[d][0], b = y + NB[d][1], e = z + NB[d][2];
                if (a < 0 || b < 0 || e < 0 || a >= nx || b >= ny || e >= nz) continue;
                int64_t u = lin(a, b, e, ny, nz);
                if (queued[u] || dt2[u] == 0) continue;
                queued[u] = 1;
                hpush(&h, hkey(dt2[u], u));
            }
        }
        if (k <= cap) {
            step_r2[k - 1] = (int32_t)(R * R);
            step_count[k - 1] = (int32_t)n;
        }
    }
    free(h.a);
    free(queued);
    free(pts);
    return k;
}

/* the inlet face as the inlets (no mask) */
int64_t or_invade_scan(const uint8_t *img, const int32_t *dt2, int nx, int ny, int nz, int inlet,
                       int64_t max_steps, int32_t *seq, int32_t *step_r2, int32_t *step_centre,
                       int64_t cap, int *status)
{
    return or_invade_scan_mask(img, dt2, nx, ny, nz, inlet, NULL, max_steps, seq, step_r2, step_centre, cap, status);
}

int64_t or_invade_heap(const uint8_t *img, const int32_t *dt2, int nx, int ny, int nz, int inlet,
                       int64_t max_steps, int32_t *seq, int32_t *step_r2, int32_t *step_centre,
                       int64_t cap, int *status)
{
    return or_invade_heap_mask(img, dt2, nx, ny, nz, inlet, NULL, max_steps, seq, step_r2, step_centre, cap, status);
}

int or_abi_version(void) { return 1; }
