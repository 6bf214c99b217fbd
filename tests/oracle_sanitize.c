/* Host sanitizer run of the oracle (test infrastructure).  Built by
 * tests/test_oracle_sanitize.py with AddressSanitizer and
 * UndefinedBehaviorSanitizer together with oracle/ibip_oracle.c; it runs
 * every oracle routine on small seeded images, including the degenerate
 * shapes, and checks that the plain definitions and their fast twins agree
 * (EDT brute force vs separable, invasion by rescan vs heap, paper-literal
 * rescan vs queue, trapping by flood fill vs union-find, opening by plain
 * dilation vs EDT).  Exit status 0 = all agree; a sanitizer report aborts. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

void or_edt_brute(const uint8_t *img, int nx, int ny, int nz, int32_t *dt2);
void or_edt_sep(const uint8_t *img, int nx, int ny, int nz, int32_t *dt2);
int64_t or_invade_scan(const uint8_t *img, const int32_t *dt2, int nx, int ny, int nz, int inlet, int64_t max_steps,
                       int32_t *seq, int32_t *step_r2, int32_t *step_centre, int64_t cap, int *status);
int64_t or_invade_heap(const uint8_t *img, const int32_t *dt2, int nx, int ny, int nz, int inlet, int64_t max_steps,
                       int32_t *seq, int32_t *step_r2, int32_t *step_centre, int64_t cap, int *status);
int64_t or_invade_literal_scan(const uint8_t *img, const int32_t *dt2, int nx, int ny, int nz, int inlet,
                               int64_t max_steps, int32_t *seq, int32_t *cstep, int32_t *step_r2,
                               int32_t *step_count, int64_t cap, int *status);
int64_t or_invade_literal_queue(const uint8_t *img, const int32_t *dt2, int nx, int ny, int nz, int inlet,
                                int64_t max_steps, int32_t *seq, int32_t *cstep, int32_t *step_r2,
                                int32_t *step_count, int64_t cap, int *status);
void or_trap_bfs(const int32_t *seq, int nx, int ny, int nz, int outlet, int do_rerank, uint8_t *trapped,
                 int32_t *seq_out);
void or_trap_uf(const int32_t *seq, int nx, int ny, int nz, int outlet, int do_rerank, uint8_t *trapped,
                int32_t *seq_out);
void or_mio_plain(const uint8_t *img, const int32_t *dt2, int nx, int ny, int nz, int inlet, const int32_t *T,
                  int32_t L, int32_t *level, int64_t *counts);
void or_mio_edt(const uint8_t *img, const int32_t *dt2, int nx, int ny, int nz, int inlet, const int32_t *T,
                int32_t L, int32_t *level, int64_t *counts);
void or_pc_curve(const int32_t *seq, int64_t N, const int32_t *step_r2, int64_t K, double voxel_m, double sigma,
                 double theta_deg, float *S, float *Pc, float *sat_image);

static uint64_t g_state = 0x9e3779b97f4a7c15ull;

static uint32_t rnd(void)   /* xorshift64*, seeded above */
{
    g_state ^= g_state >> 12;
    g_state ^= g_state << 25;
    g_state ^= g_state >> 27;
    return (uint32_t)((g_state * 0x2545f4914f6cdd1dull) >> 32);
}

static int fails = 0;

static void check(int ok, const char *what, int nx, int ny, int nz)
{
    if (!ok) {
        fprintf(stderr, "mismatch: %s on %dx%dx%d\n", what, nx, ny, nz);
        fails++;
    }
}

static void run_case(int nx, int ny, int nz, int porosity_pct)
{
    const int64_t N = (int64_t)nx * ny * nz;
    const size_t n1 = (size_t)(N ? N : 1);
    uint8_t *img = malloc(n1);
    int32_t *d1 = malloc(n1 * 4), *d2 = malloc(n1 * 4);
    for (int64_t v = 0; v < N; v++) img[v] = (int)(rnd() % 100) < porosity_pct;
    or_edt_brute(img, nx, ny, nz, d1);
    or_edt_sep(img, nx, ny, nz, d2);
    check(memcmp(d1, d2, (size_t)N * 4) == 0, "edt brute vs separable", nx, ny, nz);

    const int inlet = (int)(rnd() % 6), outlet = (int)(rnd() % 6);
    int32_t *s1 = malloc(n1 * 4), *s2 = malloc(n1 * 4);
    int32_t *r1 = malloc(n1 * 4), *r2 = malloc(n1 * 4), *c1 = malloc(n1 * 4), *c2 = malloc(n1 * 4);
    int st1 = 0, st2 = 0;
    const int64_t k1 = or_invade_scan(img, d1, nx, ny, nz, inlet, N, s1, r1, c1, N, &st1);
    const int64_t k2 = or_invade_heap(img, d1, nx, ny, nz, inlet, N, s2, r2, c2, N, &st2);
    check(k1 == k2 && st1 == st2, "invasion step counts", nx, ny, nz);
    check(memcmp(s1, s2, (size_t)N * 4) == 0, "invasion sequence, rescan vs heap", nx, ny, nz);
    check(memcmp(r1, r2, (size_t)k1 * 4) == 0 && memcmp(c1, c2, (size_t)k1 * 4) == 0, "invasion steps", nx, ny,
          nz);
    /* a step limit in the middle: the same prefix from both */
    if (k1 > 2) {
        const int64_t lim = k1 / 2;
        const int64_t q1 = or_invade_scan(img, d1, nx, ny, nz, inlet, lim, s1, r1, c1, N, &st1);
        const int64_t q2 = or_invade_heap(img, d1, nx, ny, nz, inlet, lim, s2, r2, c2, N, &st2);
        check(q1 == lim && q2 == lim && st1 == st2, "step limit", nx, ny, nz);
        check(memcmp(s1, s2, (size_t)N * 4) == 0, "limited sequence", nx, ny, nz);
        or_invade_heap(img, d1, nx, ny, nz, inlet, N, s1, r1, c1, N, &st1);   /* full run again */
    }

    int32_t *cs1 = malloc(n1 * 4), *cs2 = malloc(n1 * 4), *n1c = malloc(n1 * 4), *n2c = malloc(n1 * 4);
    const int64_t l1 = or_invade_literal_scan(img, d1, nx, ny, nz, inlet, N, s2, cs1, r2, n1c, N, &st1);
    int32_t *s3 = malloc(n1 * 4);
    const int64_t l2 = or_invade_literal_queue(img, d1, nx, ny, nz, inlet, N, s3, cs2, c2, n2c, N, &st2);
    check(l1 == l2 && st1 == st2, "literal step counts", nx, ny, nz);
    check(memcmp(s2, s3, (size_t)N * 4) == 0 && memcmp(cs1, cs2, (size_t)N * 4) == 0, "literal sequence", nx,
          ny, nz);
    check(memcmp(r2, c2, (size_t)l1 * 4) == 0 && memcmp(n1c, n2c, (size_t)l1 * 4) == 0, "literal steps", nx,
          ny, nz);

    uint8_t *t1 = malloc(n1), *t2 = malloc(n1);
    for (int rr = 0; rr < 2; rr++) {
        or_trap_bfs(s1, nx, ny, nz, outlet, rr, t1, s2);
        or_trap_uf(s1, nx, ny, nz, outlet, rr, t2, s3);
        check(memcmp(t1, t2, (size_t)N) == 0 && memcmp(s2, s3, (size_t)N * 4) == 0, "trapping bfs vs uf", nx,
              ny, nz);
    }

    int32_t mx = 0;
    for (int64_t v = 0; v < N; v++)
        if (img[v] && d1[v] != INT32_MAX && d1[v] > mx) mx = d1[v];
    int32_t T[3];
    int L = 0;
    if (mx >= 1) {
        T[L++] = mx;
        if (mx / 2 >= 1 && mx / 2 < mx) T[L++] = mx / 2;
        if (T[L - 1] > 1) T[L++] = 1;
        int32_t *lv1 = malloc(n1 * 4), *lv2 = malloc(n1 * 4);
        int64_t cn1[3], cn2[3];
        or_mio_plain(img, d1, nx, ny, nz, inlet, T, L, lv1, cn1);
        or_mio_edt(img, d1, nx, ny, nz, inlet, T, L, lv2, cn2);
        check(memcmp(lv1, lv2, (size_t)N * 4) == 0 && memcmp(cn1, cn2, (size_t)L * 8) == 0, "opening plain vs edt",
              nx, ny, nz);
        free(lv1);
        free(lv2);
    }

    float *S = malloc(n1 * 4), *P = malloc(n1 * 4), *sat = malloc(n1 * 4);
    or_pc_curve(s1, N, r1, k1, 5e-6, 0.072, 180.0, S, P, sat);
    for (int64_t k = 1; k < k1; k++) check(S[k] >= S[k - 1], "saturation rises", nx, ny, nz);

    free(img); free(d1); free(d2); free(s1); free(s2); free(s3); free(r1); free(r2); free(c1); free(c2);
    free(cs1); free(cs2); free(n1c); free(n2c); free(t1); free(t2); free(S); free(P); free(sat);
}

int main(void)
{
    static const int shapes[][3] = {{1, 1, 1}, {1, 1, 9}, {1, 7, 1}, {5, 1, 1}, {2, 3, 4}, {7, 6, 5},
                                    {9, 9, 9}, {3, 17, 11}, {12, 10, 14}, {16, 16, 16}};
    static const int por[] = {0, 30, 60, 85, 100};
    int cases = 0;
    for (size_t i = 0; i < sizeof(shapes) / sizeof(shapes[0]); i++)
        for (size_t p = 0; p < sizeof(por) / sizeof(por[0]); p++)
            for (int rep = 0; rep < 2; rep++) {
                run_case(shapes[i][0], shapes[i][1], shapes[i][2], por[p]);
                cases++;
            }
    printf("%d cases, %d mismatches\n", cases, fails);
    return fails ? 1 : 0;
}
