/*
 * Seeded synthetic inputs for the symmetric-SpMM / LOBPCG workloads.
 *
 * This module holds NO arithmetic of the eigensolver: it only draws random
 * numbers and lays them out.  Both the CPU oracle and the CUDA path read its
 * output; neither depends on the other.
 *
 * Matrix recipe (a stand-in for the nuclear CI Hamiltonians of the paper's
 * Table "tbl:dataset", whose block -> tile -> element structure is described
 * in Section 3.3, "Local sparse SpMM": dense-ish tiles near the diagonal,
 * every diagonal tile and diagonal element present):
 *   - n rows, lower triangle (incl. diagonal) stored as CSR, columns sorted.
 *   - 16x16 tile grid, R = ceil(n/16) tile-rows.
 *   - tile-row r always holds its diagonal tile (lower triangle incl. diag).
 *   - T_f = (nnz_per_row*16 - 136)/256 off-diagonal tiles per tile-row on
 *     average: floor(T_f) plus one more with probability frac(T_f), capped
 *     at the r tile columns that exist left of the diagonal.
 *   - each off-diagonal tile column c < r is "scattered" (uniform in [0,r))
 *     with probability 0.10, else "clustered" (uniform in [max(0,r-w), r),
 *     w = ceil(0.05*n/16) tile units); duplicates are redrawn.
 *   - off-diagonal tiles are fully dense (256 entries).
 *   - values: off-diagonal N(0,1)/10, diagonal U[0,200].
 *
 * Random numbers: splitmix64 (Steele, Lea, Flood 2014; constants as
 * published by Vigna), uniform doubles from the top 53 bits, normals by the
 * Box-Muller transform.  Every tile-row owns its own streams, so the result
 * does not depend on the number of threads.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define TILE 16

typedef struct { uint64_t s; } sm64;

static uint64_t sm64_next(sm64 *g) {
    uint64_t z = (g->s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Stream seeded from (seed, a, b): mixes the three words through splitmix. */
static sm64 sm64_stream(uint64_t seed, uint64_t a, uint64_t b) {
    sm64 g = { seed ^ 0x5851F42D4C957F2DULL };
    uint64_t h = sm64_next(&g);
    g.s = h ^ (a * 0xD6E8FEB86659FD93ULL);
    h = sm64_next(&g);
    g.s = h ^ (b * 0xA0761D6478BD642FULL + 0x2545F4914F6CDD1DULL);
    sm64_next(&g);
    return g;
}

static double u01(sm64 *g) {               /* [0,1) */
    return (double)(sm64_next(g) >> 11) * (1.0 / 9007199254740992.0);
}

typedef struct { sm64 g; int have; double spare; } normal_gen;

static double normal(normal_gen *ng) {
    if (ng->have) { ng->have = 0; return ng->spare; }
    double u1 = 1.0 - u01(&ng->g);          /* (0,1] */
    double u2 = u01(&ng->g);
    double rad = sqrt(-2.0 * log(u1));
    double ang = 6.283185307179586476925286766559 * u2;
    ng->spare = rad * sin(ang);
    ng->have = 1;
    return rad * cos(ang);
}

/* ------------------------------------------------------------------ plan */

typedef struct {
    int64_t n;
    int64_t R;          /* tile rows */
    int32_t tmax;       /* max off-diagonal tiles per tile-row */
    int32_t *tcnt;      /* [R] */
    int32_t *tcol;      /* [R*tmax], sorted ascending per tile-row */
    int64_t *row_ptr;   /* [n+1] */
    uint64_t seed;
} synth_plan;

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Builds the tile placement and row pointers.  Returns NULL on bad input. */
void *synth_plan_create(int64_t n, double nnz_per_row, uint64_t seed,
                        double scatter_frac, double window_frac) {
    if (n <= 0) return NULL;
    synth_plan *p = (synth_plan *)calloc(1, sizeof(synth_plan));
    if (!p) return NULL;
    p->n = n;
    p->R = (n + TILE - 1) / TILE;
    p->seed = seed;
    double tf = (nnz_per_row * TILE - 136.0) / 256.0;
    if (tf < 0) tf = 0;
    int32_t tfl = (int32_t)floor(tf);
    double tfrac = tf - tfl;
    p->tmax = tfl + 1;
    p->tcnt = (int32_t *)calloc((size_t)p->R, sizeof(int32_t));
    p->tcol = (int32_t *)calloc((size_t)p->R * p->tmax, sizeof(int32_t));
    p->row_ptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!p->tcnt || !p->tcol || !p->row_ptr) {
        free(p->tcnt); free(p->tcol); free(p->row_ptr); free(p); return NULL;
    }
    int64_t w = (int64_t)ceil(window_frac * (double)n / TILE);
    if (w < 1) w = 1;
    int64_t R = p->R;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t r = 0; r < R; r++) {
        sm64 g = sm64_stream(seed, (uint64_t)r, 1);
        int32_t want = tfl + (u01(&g) < tfrac ? 1 : 0);
        if (want > r) want = (int32_t)r;
        int32_t *cols = p->tcol + (size_t)r * p->tmax;
        int32_t got = 0;
        while (got < want) {
            int64_t c = -1;
            for (int attempt = 0; attempt < 64 && c < 0; attempt++) {
                int64_t lo = (u01(&g) < scatter_frac) ? 0 : (r - w > 0 ? r - w : 0);
                int64_t cand = lo + (int64_t)(u01(&g) * (double)(r - lo));
                if (cand >= r) cand = r - 1;
                int dup = 0;
                for (int32_t q = 0; q < got; q++) if (cols[q] == cand) { dup = 1; break; }
                if (!dup) c = cand;
            }
            if (c < 0) {                    /* deterministic fallback: smallest free */
                for (int64_t cand = 0; cand < r && c < 0; cand++) {
                    int dup = 0;
                    for (int32_t q = 0; q < got; q++) if (cols[q] == cand) { dup = 1; break; }
                    if (!dup) c = cand;
                }
            }
            cols[got++] = (int32_t)c;
        }
        qsort(cols, (size_t)got, sizeof(int32_t), cmp_i32);
        p->tcnt[r] = got;
    }
    /* row lengths: 16 per off-diagonal tile + the diagonal tile's triangle */
    p->row_ptr[0] = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t r = i / TILE;
        p->row_ptr[i + 1] = p->row_ptr[i] + (int64_t)TILE * p->tcnt[r] + (i - r * TILE + 1);
    }
    return p;
}

int64_t synth_plan_nnz(void *hp) { return ((synth_plan *)hp)->row_ptr[((synth_plan *)hp)->n]; }

void synth_plan_row_ptr(void *hp, int64_t *out) {
    synth_plan *p = (synth_plan *)hp;
    memcpy(out, p->row_ptr, sizeof(int64_t) * (size_t)(p->n + 1));
}

/* Fills col[nnz] and val[nnz] (float64 if val_fp32 == 0, float32 otherwise). */
void synth_plan_fill(void *hp, int32_t *col, void *val, int val_fp32) {
    synth_plan *p = (synth_plan *)hp;
    int64_t n = p->n, R = p->R;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < R; r++) {
        normal_gen ng = { sm64_stream(p->seed, (uint64_t)r, 2), 0, 0.0 };
        sm64 gd = sm64_stream(p->seed, (uint64_t)r, 3);
        const int32_t *tc = p->tcol + (size_t)r * p->tmax;
        int32_t nt = p->tcnt[r];
        for (int64_t i = r * TILE; i < (r + 1) * TILE && i < n; i++) {
            int64_t e = p->row_ptr[i];
            for (int32_t t = 0; t < nt; t++) {
                for (int q = 0; q < TILE; q++) {
                    double v = normal(&ng) / 10.0;
                    col[e] = (int32_t)(tc[t] * TILE + q);
                    if (val_fp32) ((float *)val)[e] = (float)v; else ((double *)val)[e] = v;
                    e++;
                }
            }
            for (int64_t j = r * TILE; j <= i; j++) {
                double v = (j == i) ? 200.0 * u01(&gd) : normal(&ng) / 10.0;
                col[e] = (int32_t)j;
                if (val_fp32) ((float *)val)[e] = (float)v; else ((double *)val)[e] = v;
                e++;
            }
        }
    }
}

void synth_plan_destroy(void *hp) {
    synth_plan *p = (synth_plan *)hp;
    if (!p) return;
    free(p->tcnt); free(p->tcol); free(p->row_ptr); free(p);
}

/* n x k row-major N(0,1) block (the initial guess X0), one stream per 1024 rows. */
void synth_normal_block(int64_t n, int32_t k, uint64_t seed, void *out, int out_fp32) {
    int64_t nb = (n + 1023) / 1024;
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nb; b++) {
        normal_gen ng = { sm64_stream(seed, (uint64_t)b, 7), 0, 0.0 };
        int64_t i1 = (b + 1) * 1024 < n ? (b + 1) * 1024 : n;
        for (int64_t e = b * 1024 * (int64_t)k; e < i1 * (int64_t)k; e++) {
            double v = normal(&ng);
            if (out_fp32) ((float *)out)[e] = (float)v; else ((double *)out)[e] = v;
        }
    }
}

/* m uniform doubles in [lo,hi) from stream (seed, tag). */
void synth_uniform(int64_t m, uint64_t seed, uint64_t tag, double lo, double hi, double *out) {
    sm64 g = sm64_stream(seed, tag, 11);
    for (int64_t i = 0; i < m; i++) out[i] = lo + (hi - lo) * u01(&g);
}

/* m standard normals from stream (seed, tag). */
void synth_normals(int64_t m, uint64_t seed, uint64_t tag, double *out) {
    normal_gen ng = { sm64_stream(seed, tag, 13), 0, 0.0 };
    for (int64_t i = 0; i < m; i++) out[i] = normal(&ng);
}

/* m uniform 64-bit words from stream (seed, tag) (for sample selection). */
void synth_u64(int64_t m, uint64_t seed, uint64_t tag, uint64_t *out) {
    sm64 g = sm64_stream(seed, tag, 17);
    for (int64_t i = 0; i < m; i++) out[i] = sm64_next(&g);
}
