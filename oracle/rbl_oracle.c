/*
 * rbl_oracle.c -- plain FP64 CPU oracle for the random-batch list (RBL) force step
 * of Liang, Xu & Zhao, "Random-batch list algorithm for short-range molecular
 * dynamics simulations" (arXiv 2105.04884).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct statement of
 * what the GPU path computes.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table or
 * constant generator with the CUDA library; every function restates the paper (or
 * a published algorithm it relies on) directly.
 *
 * Build: cc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC -fopenmp.
 * `-ffp-contract=off` is required: the pair-classification rule below is defined
 * as separately rounded IEEE single-precision operations, and an FMA contraction
 * would change which side of a cutoff a pair lands on.
 *
 * Pinned by tests/test_oracle_*.py (closed forms, brute force, invariants,
 * published known-answer vectors).  Functions without a pin say so.
 *
 * Conventions (each is a reading of the paper):
 *  - reduced LJ units, sigma = epsilon = m = k_B = 1 (Sec. 3); charges (the Ewald
 *    real-space extension) in units where two unit charges at distance r have
 *    Coulomb energy 1/r.
 *  - positions x[i*3+a] in [0, L_a), periodic, particle index == tag.
 *  - the decision "is r_ij below a cutoff" is taken on a 32-bit fixed-point image
 *    of the positions, in IEEE binary32 (the precision of the GPU kernels), see
 *    orc_pair_r2f; the force values themselves are FP64 from FP64 positions.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EOVERFLOW 3

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11, Sec. 4.2).  Round function: two 32x32->64 products of
 * counter words 0 and 2 with the published multipliers, outputs permuted and
 * xored with the other counter words and the key; the key is bumped by the
 * published Weyl constants between rounds.                                   */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)prod1;
        uint32_t n2 = (uint32_t)(prod0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)prod0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A stream of 32-bit words for one (seed, step, tag, stream id): counter =
 * (step_lo, step_hi, tag, stream<<24 | block), key = (seed_lo, seed_hi); the four
 * words of each block are consumed in order, blocks in increasing order.       */
typedef struct {
    uint32_t key[2];
    uint32_t ctr[4];
    uint32_t buf[4];
    int pos;
} word_stream;

static void ws_init(word_stream *ws, uint64_t seed, uint64_t step, uint32_t tag, uint32_t stream)
{
    ws->key[0] = (uint32_t)seed;
    ws->key[1] = (uint32_t)(seed >> 32);
    ws->ctr[0] = (uint32_t)step;
    ws->ctr[1] = (uint32_t)(step >> 32);
    ws->ctr[2] = tag;
    ws->ctr[3] = stream << 24;
    ws->pos = 4;
}

static uint32_t ws_next(word_stream *ws)
{
    if (ws->pos == 4) {
        orc_philox4x32_10(ws->ctr, ws->key, ws->buf);
        ws->ctr[3] += 1u; /* next block */
        ws->pos = 0;
    }
    return ws->buf[ws->pos++];
}

/* Uniform integer in [0, s), s >= 1: Lemire, "Fast random integer generation in
 * an interval", ACM TOMACS 2019, multiply-shift with rejection of the low words
 * below 2^32 mod s.                                                              */
static uint32_t ws_uniform_below(word_stream *ws, uint32_t s)
{
    uint64_t m = (uint64_t)ws_next(ws) * (uint64_t)s;
    uint32_t low = (uint32_t)m;
    if (low < s) {
        uint32_t threshold = (uint32_t)(0u - s) % s;
        while (low < threshold) {
            m = (uint64_t)ws_next(ws) * (uint64_t)s;
            low = (uint32_t)m;
        }
    }
    return (uint32_t)(m >> 32);
}

/* Exposed for tests: n words of the stream. */
void orc_stream_words(uint64_t seed, uint64_t step, uint32_t tag, uint32_t stream, int n, uint32_t *out)
{
    word_stream ws;
    ws_init(&ws, seed, step, tag, stream);
    for (int k = 0; k < n; ++k) out[k] = ws_next(&ws);
}

/* Exposed for tests: n bounded draws (all with the same bound s). */
void orc_stream_uniform_below(uint64_t seed, uint64_t step, uint32_t tag, uint32_t stream, uint32_t s, int n,
                              uint32_t *out)
{
    word_stream ws;
    ws_init(&ws, seed, step, tag, stream);
    for (int k = 0; k < n; ++k) out[k] = ws_uniform_below(&ws, s);
}

/* ------------------------------------------------------------------------- */
/* Random batch B(i) (Sec. 2, Eq. (4) and Algorithm 1, "randomly choose p
 * particles ... if N > p, otherwise choose all").  Sampling is without
 * replacement (the (p-1)/(N-1) factor of the second moment in Appendix A), i.e. a
 * uniform p-subset of the N_s shell positions, drawn with Floyd's algorithm
 * (Bentley & Floyd, CACM 30(9), 1987): for k = N_s-p .. N_s-1 draw t uniform in
 * [0, k]; insert t unless already chosen, in which case insert k.
 * Output: the chosen positions in ascending order; returns their number.        */
/* ------------------------------------------------------------------------- */
static int floyd_from_stream(word_stream *ws, int n_s, int p, int32_t *out)
{
    if (n_s <= p) {
        for (int k = 0; k < n_s; ++k) out[k] = k;
        return n_s;
    }
    int count = 0;
    for (int k = n_s - p; k < n_s; ++k) {
        int32_t t = (int32_t)ws_uniform_below(ws, (uint32_t)k + 1u);
        int seen = 0;
        for (int q = 0; q < count; ++q)
            if (out[q] == t) { seen = 1; break; }
        out[count++] = seen ? k : t;
    }
    /* ascending order (insertion sort; p is small) */
    for (int a = 1; a < count; ++a) {
        int32_t v = out[a];
        int b = a - 1;
        while (b >= 0 && out[b] > v) { out[b + 1] = out[b]; --b; }
        out[b + 1] = v;
    }
    return count;
}

int orc_batch_positions(uint64_t seed, uint64_t step, uint32_t tag, int n_s, int p, int32_t *out)
{
    word_stream ws;
    ws_init(&ws, seed, step, tag, 0u);
    return floyd_from_stream(&ws, n_s, p, out);
}

/* Floyd's algorithm driven by an explicit sequence of draws t_k in [0, k]
 * (tests enumerate every sequence to show each subset is equally likely).      */
int orc_floyd_from_draws(int n_s, int p, const int32_t *draws, int32_t *out)
{
    int count = 0;
    for (int k = n_s - p, d = 0; k < n_s; ++k, ++d) {
        int32_t t = draws[d];
        int seen = 0;
        for (int q = 0; q < count; ++q)
            if (out[q] == t) { seen = 1; break; }
        out[count++] = seen ? k : t;
    }
    return count;
}

/* ------------------------------------------------------------------------- */
/* Thermostat noise (Sec. 2, Eq. (2)): three standard normals per particle and
 * step from stream 1, by the Box-Muller transform of four words
 * a_k = ((w_k >> 9) + 1/2) 2^-23 (exactly representable in binary32 and FP64):
 *   xi_x = sqrt(-2 ln a0) cos(2 pi a1), xi_y = sqrt(-2 ln a0) sin(2 pi a1),
 *   xi_z = sqrt(-2 ln a2) cos(2 pi a3).                                          */
/* ------------------------------------------------------------------------- */
void orc_gaussians(uint64_t seed, uint64_t step, uint32_t tag, double out[3])
{
    word_stream ws;
    ws_init(&ws, seed, step, tag, 1u);
    double a[4];
    for (int k = 0; k < 4; ++k) a[k] = ((double)(ws_next(&ws) >> 9) + 0.5) * (1.0 / 8388608.0);
    const double two_pi = 6.283185307179586476925286766559;
    double r0 = sqrt(-2.0 * log(a[0]));
    double r1 = sqrt(-2.0 * log(a[2]));
    out[0] = r0 * cos(two_pi * a[1]);
    out[1] = r0 * sin(two_pi * a[1]);
    out[2] = r1 * cos(two_pi * a[3]);
}

/* ------------------------------------------------------------------------- */
/* Pair classification.  The paper decides core (r < r_c) / shell (r_c <= r < r_s)
 * membership on r_ij (Sec. 2, Eqs. (3)-(4)).  The decision is taken on a 32-bit
 * fixed-point image of each coordinate, u = rint(x * 2^32 / L) mod 2^32 (the exact
 * product rounded once to the nearest integer), whose
 * two's-complement difference is the minimum-image separation in units of
 * L / 2^32; the squared distance is then formed in binary32 with one rounding
 * per operation: d = (float)(int32)(u_i - u_j) * h, r2 = (dx*dx + dy*dy) + dz*dz. */
/* ------------------------------------------------------------------------- */
typedef struct {
    double L[3];
    double inv[3]; /* 2^32 / L (FP64) */
    float h[3];    /* (float)(L / 2^32) */
} fixed_frame;

static void frame_init(fixed_frame *f, const double L[3])
{
    for (int a = 0; a < 3; ++a) {
        f->L[a] = L[a];
        f->inv[a] = 4294967296.0 / L[a];
        f->h[a] = (float)(L[a] / 4294967296.0);
    }
}

/* rint(x * 2^32/L) with one rounding: the exact product is rounded to the nearest
 * integer (ties to even) by a fused multiply-add onto 1.5 * 2^52, whose ulp is 1. */
static uint32_t quantize1(double x, double inv)
{
    const double magic = 6755399441055744.0;
    return (uint32_t)(uint64_t)(int64_t)(fma(x, inv, magic) - magic);
}

void orc_quantize(int n, const double *x, const double L[3], uint32_t *u)
{
    fixed_frame f;
    frame_init(&f, L);
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) u[i * 3 + a] = quantize1(x[i * 3 + a], f.inv[a]);
}

static float pair_r2f(const uint32_t *ui, const uint32_t *uj, const float h[3])
{
    float d0 = (float)(int32_t)(ui[0] - uj[0]) * h[0];
    float d1 = (float)(int32_t)(ui[1] - uj[1]) * h[1];
    float d2 = (float)(int32_t)(ui[2] - uj[2]) * h[2];
    float s = d0 * d0;
    float t = d1 * d1;
    s = s + t;
    t = d2 * d2;
    return s + t;
}

/* Exposed for tests: r2 of pairs (i[k], j[k]) from fixed-point coordinates. */
void orc_pair_r2f(int n, const uint32_t *u, const double L[3], const int32_t *pi, const int32_t *pj, float *out)
{
    fixed_frame f;
    frame_init(&f, L);
    for (int k = 0; k < n; ++k) out[k] = pair_r2f(u + 3 * pi[k], u + 3 * pj[k], f.h);
}

/* Thresholds in binary32, each rounded once from FP64. */
typedef struct {
    float core_list;  /* (r_c + skin)^2 */
    float shell_lo;   /* max(r_c - skin, 0)^2 */
    float cut_list;   /* (r_s + skin)^2 */
    float rc2;        /* r_c^2 */
    float rs2;        /* r_s^2 */
    float disp;       /* (skin/2)^2 */
} thresholds;

static thresholds make_thresholds(double rc, double rs, double skin)
{
    thresholds t;
    double lo = rc - skin > 0.0 ? rc - skin : 0.0;
    t.core_list = (float)((rc + skin) * (rc + skin));
    t.shell_lo = (float)(lo * lo);
    t.cut_list = (float)((rs + skin) * (rs + skin));
    t.rc2 = (float)(rc * rc);
    t.rs2 = (float)(rs * rs);
    t.disp = (float)(0.25 * skin * skin);
    return t;
}

/* ------------------------------------------------------------------------- */
/* Linked cells (Sec. 2, Fig. 1): cubic-ish cells of width >= (r_s + skin)/K on a
 * per-axis grid of n_a = floor(L_a K / (r_s + skin)) cells; a particle's cell is
 * c_a = floor(u_a n_a / 2^32) (exact integer arithmetic on the fixed-point image).
 * The stencil of a cell is (2K+1)^3 cells (offsets -K..K per axis), or, on an
 * axis with fewer than 2K+1 cells, every cell of that axis once (offsets
 * 0..n_a-1), visited z-major, x-minor.  Row order of a list = (stencil slot of
 * the neighbour's cell, the neighbour's x image u_x, tag): this is the canonical
 * order in which batch positions are counted.                                   */
/* ------------------------------------------------------------------------- */
typedef struct {
    int n[3];
    int nofs[3];
    int ofs[3][16];
} cell_grid;

static void grid_init(cell_grid *g, const double L[3], double rcut, int K)
{
    for (int a = 0; a < 3; ++a) {
        int n = (int)floor(L[a] * (double)K / rcut);
        if (n < 1) n = 1;
        g->n[a] = n;
        if (n >= 2 * K + 1) {
            g->nofs[a] = 2 * K + 1;
            for (int o = 0; o < 2 * K + 1; ++o) g->ofs[a][o] = o - K;
        } else {
            g->nofs[a] = n;
            for (int o = 0; o < n; ++o) g->ofs[a][o] = o;
        }
    }
}

static void cell_of(const cell_grid *g, const uint32_t *u, int c[3])
{
    for (int a = 0; a < 3; ++a) c[a] = (int)(((uint64_t)u[a] * (uint64_t)g->n[a]) >> 32);
}

/* slot index of cell cj in the stencil of cell ci, or -1 */
static int stencil_slot(const cell_grid *g, const int ci[3], const int cj[3])
{
    int idx[3];
    for (int a = 0; a < 3; ++a) {
        idx[a] = -1;
        for (int o = 0; o < g->nofs[a]; ++o) {
            int c = ci[a] + g->ofs[a][o];
            c %= g->n[a];
            if (c < 0) c += g->n[a];
            if (c == cj[a]) { idx[a] = o; break; }
        }
        if (idx[a] < 0) return -1;
    }
    return (idx[2] * g->nofs[1] + idx[1]) * g->nofs[0] + idx[0];
}

void orc_cell_grid(const double L[3], double rs, double skin, int K, int32_t n_out[3])
{
    cell_grid g;
    grid_init(&g, L, rs + skin, K);
    for (int a = 0; a < 3; ++a) n_out[a] = g.n[a];
}

void orc_cells(int n, const uint32_t *u, const double L[3], double rs, double skin, int K, int32_t *cell_out)
{
    cell_grid g;
    grid_init(&g, L, rs + skin, K);
    for (int i = 0; i < n; ++i) {
        int c[3];
        cell_of(&g, u + 3 * i, c);
        cell_out[i] = (c[2] * g.n[1] + c[1]) * g.n[0] + c[0];
    }
}

/* ------------------------------------------------------------------------- */
/* Two-level neighbour lists with a skin (Sec. 2: core list from the nearest
 * cells, shell list from the stencil; the cell edge a little larger than the
 * cutoff so that lists survive several steps):
 *   core_i  = { j != i : r2 <  (r_c + skin)^2 }
 *   shell_i = { j != i : max(r_c - skin, 0)^2 <= r2 < (r_s + skin)^2 }
 *   full_i  = { j != i : r2 <  (r_s + skin)^2 }      (classical Verlet list)
 * Rows are written at stride cap; returns ORC_EOVERFLOW if a row does not fit.
 * orc_build_lists_brute tests all pairs; orc_build_lists_cells walks the stencil.
 * Both emit rows in the canonical (stencil slot, tag) order.                    */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t slot;
    uint32_t ux;
    int32_t tag;
} row_key;

static int cmp_row_key(const void *a, const void *b)
{
    const row_key *x = (const row_key *)a, *y = (const row_key *)b;
    if (x->slot != y->slot) return x->slot < y->slot ? -1 : 1;
    if (x->ux != y->ux) return x->ux < y->ux ? -1 : 1;
    return (x->tag > y->tag) - (x->tag < y->tag);
}

static void sort_row(int32_t *row, int len, const cell_grid *g, const int *cells3, const uint32_t *u, int i,
                     row_key *scratch)
{
    for (int k = 0; k < len; ++k) {
        scratch[k].slot = stencil_slot(g, cells3 + 3 * i, cells3 + 3 * row[k]);
        scratch[k].ux = u[3 * row[k]];
        scratch[k].tag = row[k];
    }
    qsort(scratch, (size_t)len, sizeof(row_key), cmp_row_key);
    for (int k = 0; k < len; ++k) row[k] = scratch[k].tag;
}

int orc_build_lists_brute(int n, const double *x, const double L[3], double rc, double rs, double skin, int K,
                          int cap_core, int cap_shell, int cap_full, int32_t *core, int32_t *n_core,
                          int32_t *shell, int32_t *n_shell, int32_t *full, int32_t *n_full)
{
    fixed_frame f;
    frame_init(&f, L);
    thresholds t = make_thresholds(rc, rs, skin);
    cell_grid g;
    grid_init(&g, L, rs + skin, K);
    uint32_t *u = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (size_t)n);
    int *cells3 = (int *)malloc(sizeof(int) * 3 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) u[3 * i + a] = quantize1(x[3 * i + a], f.inv[a]);
        cell_of(&g, u + 3 * i, cells3 + 3 * i);
    }
    int status = ORC_OK;
#pragma omp parallel
    {
        int maxcap = cap_core > cap_shell ? cap_core : cap_shell;
        if (cap_full > maxcap) maxcap = cap_full;
        row_key *scratch = (row_key *)malloc(sizeof(row_key) * (size_t)(maxcap + 1));
#pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i) {
            int nc = 0, ns = 0, nf = 0;
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                float r2 = pair_r2f(u + 3 * i, u + 3 * j, f.h);
                if (r2 < t.core_list) {
                    if (nc < cap_core) core[(size_t)i * cap_core + nc] = j;
                    ++nc;
                }
                if (r2 >= t.shell_lo && r2 < t.cut_list) {
                    if (ns < cap_shell) shell[(size_t)i * cap_shell + ns] = j;
                    ++ns;
                }
                if (r2 < t.cut_list && full) {
                    if (nf < cap_full) full[(size_t)i * cap_full + nf] = j;
                    ++nf;
                }
            }
            if (nc > cap_core || ns > cap_shell || (full && nf > cap_full)) {
#pragma omp atomic write
                status = ORC_EOVERFLOW;
            } else {
                sort_row(core + (size_t)i * cap_core, nc, &g, cells3, u, i, scratch);
                sort_row(shell + (size_t)i * cap_shell, ns, &g, cells3, u, i, scratch);
                if (full) sort_row(full + (size_t)i * cap_full, nf, &g, cells3, u, i, scratch);
            }
            n_core[i] = nc;
            n_shell[i] = ns;
            if (n_full) n_full[i] = nf;
        }
        free(scratch);
    }
    free(u);
    free(cells3);
    return status;
}

int orc_build_lists_cells(int n, const double *x, const double L[3], double rc, double rs, double skin, int K,
                          int cap_core, int cap_shell, int cap_full, int32_t *core, int32_t *n_core,
                          int32_t *shell, int32_t *n_shell, int32_t *full, int32_t *n_full)
{
    fixed_frame f;
    frame_init(&f, L);
    thresholds t = make_thresholds(rc, rs, skin);
    cell_grid g;
    grid_init(&g, L, rs + skin, K);
    int ncell = g.n[0] * g.n[1] * g.n[2];
    uint32_t *u = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (size_t)n);
    int *cell = (int *)malloc(sizeof(int) * (size_t)n);
    int *start = (int *)calloc((size_t)ncell + 1, sizeof(int));
    int *members = (int *)malloc(sizeof(int) * (size_t)n);
    for (int i = 0; i < n; ++i) {
        int c[3];
        for (int a = 0; a < 3; ++a) u[3 * i + a] = quantize1(x[3 * i + a], f.inv[a]);
        cell_of(&g, u + 3 * i, c);
        cell[i] = (c[2] * g.n[1] + c[1]) * g.n[0] + c[0];
        start[cell[i] + 1] += 1;
    }
    for (int c = 0; c < ncell; ++c) start[c + 1] += start[c];
    {
        int *fill = (int *)malloc(sizeof(int) * (size_t)ncell);
        memcpy(fill, start, sizeof(int) * (size_t)ncell);
        for (int i = 0; i < n; ++i) members[fill[cell[i]]++] = i; /* ascending tag within a cell */
        free(fill);
    }
    /* within a cell: ascending x image, then tag */
    {
        row_key *keys = (row_key *)malloc(sizeof(row_key) * (size_t)(n > 0 ? n : 1));
        for (int c = 0; c < ncell; ++c) {
            int m = start[c + 1] - start[c];
            for (int k = 0; k < m; ++k) {
                int j = members[start[c] + k];
                keys[k].slot = 0;
                keys[k].ux = u[3 * j];
                keys[k].tag = j;
            }
            qsort(keys, (size_t)m, sizeof(row_key), cmp_row_key);
            for (int k = 0; k < m; ++k) members[start[c] + k] = keys[k].tag;
        }
        free(keys);
    }
    int status = ORC_OK;
#pragma omp parallel for schedule(dynamic, 256)
    for (int i = 0; i < n; ++i) {
        int ci[3];
        cell_of(&g, u + 3 * i, ci);
        int nc = 0, ns = 0, nf = 0;
        for (int oz = 0; oz < g.nofs[2]; ++oz)
            for (int oy = 0; oy < g.nofs[1]; ++oy)
                for (int ox = 0; ox < g.nofs[0]; ++ox) {
                    int cz = ((ci[2] + g.ofs[2][oz]) % g.n[2] + g.n[2]) % g.n[2];
                    int cy = ((ci[1] + g.ofs[1][oy]) % g.n[1] + g.n[1]) % g.n[1];
                    int cx = ((ci[0] + g.ofs[0][ox]) % g.n[0] + g.n[0]) % g.n[0];
                    int c = (cz * g.n[1] + cy) * g.n[0] + cx;
                    for (int m = start[c]; m < start[c + 1]; ++m) {
                        int j = members[m];
                        if (j == i) continue;
                        float r2 = pair_r2f(u + 3 * i, u + 3 * j, f.h);
                        if (r2 < t.core_list) {
                            if (nc < cap_core) core[(size_t)i * cap_core + nc] = j;
                            ++nc;
                        }
                        if (r2 >= t.shell_lo && r2 < t.cut_list) {
                            if (ns < cap_shell) shell[(size_t)i * cap_shell + ns] = j;
                            ++ns;
                        }
                        if (r2 < t.cut_list && full) {
                            if (nf < cap_full) full[(size_t)i * cap_full + nf] = j;
                            ++nf;
                        }
                    }
                }
        if (nc > cap_core || ns > cap_shell || (full && nf > cap_full)) {
#pragma omp atomic write
            status = ORC_EOVERFLOW;
        }
        n_core[i] = nc;
        n_shell[i] = ns;
        if (n_full) n_full[i] = nf;
    }
    free(u);
    free(cell);
    free(start);
    free(members);
    return status;
}

/* ------------------------------------------------------------------------- */
/* LJ 12-6 pair (Sec. 2, Eq. (1)): u(r) = 4 (r^-12 - r^-6); the force on i due to
 * j is f_ij = 24 (2 r^-12 - r^-6) / r^2 * d_ij, d_ij = minimum-image x_i - x_j.  */
/* ------------------------------------------------------------------------- */
static void min_image(const double *xi, const double *xj, const double L[3], double d[3])
{
    for (int a = 0; a < 3; ++a) {
        double v = xi[a] - xj[a];
        v -= L[a] * nearbyint(v / L[a]);
        d[a] = v;
    }
}

static double lj_pair(const double d[3], double fvec[3], double *virial)
{
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double ir2 = 1.0 / r2;
    double ir6 = ir2 * ir2 * ir2;
    double coef = 24.0 * (2.0 * ir6 * ir6 - ir6) * ir2;
    for (int a = 0; a < 3; ++a) fvec[a] = coef * d[a];
    if (virial) *virial = 24.0 * (2.0 * ir6 * ir6 - ir6);
    return 4.0 * (ir6 * ir6 - ir6);
}

/* Charged pairs: the LJ 12-6 pair plus the Ewald real-space term, the short-range
 * part of the Coulomb interaction to which the RBL extends unchanged (Sec. 2,
 * closing remarks; Sec. 4):
 *   u_C(r) = q_i q_j erfc(alpha r) / r,
 *   r . f_C = q_i q_j (erfc(alpha r) / r + (2 alpha / sqrt(pi)) exp(-alpha^2 r^2)),
 * f_C = (r . f_C) / r^2 d_ij.  q == NULL: the LJ pair alone (bit for bit).       */
typedef struct {
    const double *q; /* charge of each particle, or NULL */
    double alpha;    /* Ewald splitting parameter */
} pair_pot;

static double pot_pair(const pair_pot *pp, int i, int j, const double d[3], double fvec[3], double *virial)
{
    if (!pp || !pp->q) return lj_pair(d, fvec, virial);
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double ir2 = 1.0 / r2;
    double ir6 = ir2 * ir2 * ir2;
    double w = 24.0 * (2.0 * ir6 * ir6 - ir6);
    double u = 4.0 * (ir6 * ir6 - ir6);
    double qq = pp->q[i] * pp->q[j];
    double r = sqrt(r2);
    double ec = erfc(pp->alpha * r) / r;
    u += qq * ec;
    w += qq * (ec + 2.0 * pp->alpha / sqrt(3.14159265358979323846) * exp(-pp->alpha * pp->alpha * r2));
    double coef = w * ir2;
    for (int a = 0; a < 3; ++a) fvec[a] = coef * d[a];
    if (virial) *virial = w;
    return u;
}

/* Pair energy and radial force magnitude of two charges q_i q_j = qq at distance
 * r[k] (qq = 0: the LJ pair). */
void orc_pair(int n, const double *r, double qq, double alpha, double *u_out, double *fmag_out)
{
    const double q2[2] = {1.0, qq};
    pair_pot pp = {q2, alpha};
    for (int k = 0; k < n; ++k) {
        double d[3] = {r[k], 0.0, 0.0}, fv[3];
        u_out[k] = pot_pair(&pp, 0, 1, d, fv, NULL);
        fmag_out[k] = fv[0];
    }
}

void orc_lj(int n, const double *r, double *u_out, double *fmag_out)
{
    for (int k = 0; k < n; ++k) {
        double d[3] = {r[k], 0.0, 0.0}, fv[3];
        u_out[k] = lj_pair(d, fv, NULL);
        fmag_out[k] = fv[0];
    }
}

/* ------------------------------------------------------------------------- */
/* RBL force (Sec. 2, Eqs. (3)-(4); Algorithm 1, force lines):
 *   F_i,c = sum over core_i with r2 < r_c^2 of f_ij
 *   F~_i,s = (N_s/p) sum over j in B(i) with r_c^2 <= r2 < r_s^2 of f_ij,
 * B(i) = whole shell row when N_s <= p (scale 1), else the Floyd p-subset drawn
 * from stream 0 of (seed, step, tag i).  Outputs F_i = F_i,c + F~_i,s (before the
 * net-force correction), and the RBL estimates of the energy and virial
 * (each pair term weighted like its force, halved per particle).
 * batch_out (optional, stride p): the chosen shell entries (tags), in position
 * order; batch_n: their number.                                               */
/* ------------------------------------------------------------------------- */
/* RBL force on particle i from its core row and shell row (Eqs. (3)-(4)):
 * F_i = sum over the core row of f_ij for r < r_c, plus s times the sum over the
 * batch B(i) of f_ij for r_c <= r < r_s, s = N_s/p when N_s > p (else 1); the batch
 * is the Floyd sample of row positions drawn from Philox stream 0 of (seed, step,
 * tag i).  Also returns this particle's halves of the energy and virial estimates. */
static void force_one(int i, const double *x, const uint32_t *u, const fixed_frame *f, const thresholds *t,
                      const pair_pot *pp, const double L[3], int p, uint64_t seed, uint64_t step,
                      const int32_t *crow, int nc, const int32_t *srow, int ns, int32_t *pos, double Fi[3],
                      double *e_i, double *w_i,
                      int32_t *batch_out, int32_t *batch_n)
{
    double fc[3] = {0, 0, 0}, fs[3] = {0, 0, 0};
    double ec = 0.0, es = 0.0, wc = 0.0, wsum = 0.0;
    for (int k = 0; k < nc; ++k) {
        int j = crow[k];
        float r2f = pair_r2f(u + 3 * i, u + 3 * j, f->h);
        if (!(r2f < t->rc2)) continue;
        double d[3], fv[3], vir;
        min_image(x + 3 * i, x + 3 * j, L, d);
        ec += pot_pair(pp, i, j, d, fv, &vir);
        wc += vir;
        for (int a = 0; a < 3; ++a) fc[a] += fv[a];
    }
    int nb = orc_batch_positions(seed, step, (uint32_t)i, ns, p, pos);
    double s = ns > p ? (double)ns / (double)p : 1.0;
    for (int b = 0; b < nb; ++b) {
        int j = srow[pos[b]];
        if (batch_out) batch_out[b] = j;
        float r2f = pair_r2f(u + 3 * i, u + 3 * j, f->h);
        if (!(r2f >= t->rc2 && r2f < t->rs2)) continue;
        double d[3], fv[3], vir;
        min_image(x + 3 * i, x + 3 * j, L, d);
        es += pot_pair(pp, i, j, d, fv, &vir);
        wsum += vir;
        for (int a = 0; a < 3; ++a) fs[a] += fv[a];
    }
    if (batch_n) *batch_n = nb;
    for (int a = 0; a < 3; ++a) Fi[a] = fc[a] + s * fs[a];
    *e_i = 0.5 * (ec + s * es);
    *w_i = 0.5 * (wc + s * wsum);
}

int orc_rbl_forces(int n, const double *x, const double L[3], double rc, double rs, double skin, int p,
                   uint64_t seed, uint64_t step, const int32_t *core, const int32_t *n_core, int cap_core,
                   const int32_t *shell, const int32_t *n_shell, int cap_shell, double *F, double *energy_virial,
                   int32_t *batch_out, int32_t *batch_n, const double *q, double alpha)
{
    const pair_pot pp = {q, alpha};
    fixed_frame f;
    frame_init(&f, L);
    thresholds t = make_thresholds(rc, rs, skin);
    uint32_t *u = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (size_t)n);
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) u[3 * i + a] = quantize1(x[3 * i + a], f.inv[a]);
    double e_tot = 0.0, w_tot = 0.0;
#pragma omp parallel reduction(+ : e_tot, w_tot)
    {
        int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)(p > 0 ? p : 1));
#pragma omp for schedule(static)
        for (int i = 0; i < n; ++i) {
            double e_i, w_i;
            force_one(i, x, u, &f, &t, &pp, L, p, seed, step, core + (size_t)i * cap_core, n_core[i],
                      shell + (size_t)i * cap_shell, n_shell[i], pos, F + 3 * (size_t)i, &e_i, &w_i,
                      batch_out ? batch_out + (size_t)i * p : NULL, batch_n ? batch_n + i : NULL);
            e_tot += e_i;
            w_tot += w_i;
        }
        free(pos);
    }
    if (energy_virial) {
        energy_virial[0] = e_tot;
        energy_virial[1] = w_tot;
    }
    free(u);
    return ORC_OK;
}

/* Rows, batch and force of m sampled particles idx[0..m) of a large system, each
 * computed on its own: the core and shell rows by testing every other particle
 * (the definition, as in orc_build_lists_brute) and sorting them into the
 * canonical order, the batch and the force as in orc_rbl_forces (no mean
 * subtraction: that needs every particle).  Rows at stride cap_core / cap_shell,
 * batches at stride p, forces [m][3].  For checking a large system particle by
 * particle.                                                                     */
int orc_sample(int n, const double *x, const double L[3], double rc, double rs, double skin, int K, int p,
               uint64_t seed, uint64_t step, int m, const int32_t *idx, int cap_core, int cap_shell,
               int32_t *core, int32_t *n_core, int32_t *shell, int32_t *n_shell, int32_t *batch,
               int32_t *n_batch, double *F, const double *q, double alpha)
{
    const pair_pot pp = {q, alpha};
    fixed_frame f;
    frame_init(&f, L);
    thresholds t = make_thresholds(rc, rs, skin);
    cell_grid g;
    grid_init(&g, L, rs + skin, K);
    uint32_t *u = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (size_t)n);
    int *cells3 = (int *)malloc(sizeof(int) * 3 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) u[3 * i + a] = quantize1(x[3 * i + a], f.inv[a]);
        cell_of(&g, u + 3 * i, cells3 + 3 * i);
    }
    int status = ORC_OK;
#pragma omp parallel
    {
        int maxcap = cap_core > cap_shell ? cap_core : cap_shell;
        row_key *scratch = (row_key *)malloc(sizeof(row_key) * (size_t)(maxcap + 1));
        int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)(p > 0 ? p : 1));
#pragma omp for schedule(dynamic, 1)
        for (int k = 0; k < m; ++k) {
            const int i = idx[k];
            int32_t *crow = core + (size_t)k * cap_core, *srow = shell + (size_t)k * cap_shell;
            int nc = 0, ns = 0;
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                float r2 = pair_r2f(u + 3 * i, u + 3 * j, f.h);
                if (r2 < t.core_list) {
                    if (nc < cap_core) crow[nc] = j;
                    ++nc;
                }
                if (r2 >= t.shell_lo && r2 < t.cut_list) {
                    if (ns < cap_shell) srow[ns] = j;
                    ++ns;
                }
            }
            n_core[k] = nc;
            n_shell[k] = ns;
            if (nc > cap_core || ns > cap_shell) {
#pragma omp atomic write
                status = ORC_EOVERFLOW;
                continue;
            }
            sort_row(crow, nc, &g, cells3, u, i, scratch);
            sort_row(srow, ns, &g, cells3, u, i, scratch);
            double e_i, w_i;
            force_one(i, x, u, &f, &t, &pp, L, p, seed, step, crow, nc, srow, ns, pos, F + 3 * (size_t)k, &e_i,
                      &w_i, batch + (size_t)k * p, n_batch + k);
        }
        free(pos);
        free(scratch);
    }
    free(u);
    free(cells3);
    return status;
}

/* Classical cutoff force from a full Verlet list: sum over full_i with
 * r2 < r_s^2 of f_ij; energy and virial summed over unordered pairs.           */
int orc_full_forces(int n, const double *x, const double L[3], double rs, const int32_t *full,
                    const int32_t *n_full, int cap_full, double *F, double *energy_virial, const double *q,
                    double alpha)
{
    const pair_pot pp = {q, alpha};
    fixed_frame f;
    frame_init(&f, L);
    float rs2 = (float)(rs * rs);
    uint32_t *u = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (size_t)n);
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) u[3 * i + a] = quantize1(x[3 * i + a], f.inv[a]);
    double e_tot = 0.0, w_tot = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : e_tot, w_tot)
    for (int i = 0; i < n; ++i) {
        double fi[3] = {0, 0, 0};
        const int32_t *row = full + (size_t)i * cap_full;
        for (int k = 0; k < n_full[i]; ++k) {
            int j = row[k];
            float r2f = pair_r2f(u + 3 * i, u + 3 * j, f.h);
            if (!(r2f < rs2)) continue;
            double d[3], fv[3], vir;
            min_image(x + 3 * i, x + 3 * j, L, d);
            e_tot += 0.5 * pot_pair(&pp, i, j, d, fv, &vir);
            w_tot += 0.5 * vir;
            for (int a = 0; a < 3; ++a) fi[a] += fv[a];
        }
        for (int a = 0; a < 3; ++a) F[3 * i + a] = fi[a];
    }
    if (energy_virial) {
        energy_virial[0] = e_tot;
        energy_virial[1] = w_tot;
    }
    free(u);
    return ORC_OK;
}

/* All-pairs O(N^2) cutoff force with no lists at all (the definition the lists
 * must reproduce).  Energy and virial over unordered pairs i < j.               */
void orc_brute_forces(int n, const double *x, const double L[3], double rs, double *F, double *energy_virial,
                      const double *q, double alpha)
{
    const pair_pot pp = {q, alpha};
    fixed_frame f;
    frame_init(&f, L);
    float rs2 = (float)(rs * rs);
    uint32_t *u = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (size_t)n);
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) u[3 * i + a] = quantize1(x[3 * i + a], f.inv[a]);
    double e_tot = 0.0, w_tot = 0.0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : e_tot, w_tot)
    for (int i = 0; i < n; ++i) {
        double fi[3] = {0, 0, 0};
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            float r2f = pair_r2f(u + 3 * i, u + 3 * j, f.h);
            if (!(r2f < rs2)) continue;
            double d[3], fv[3], vir;
            min_image(x + 3 * i, x + 3 * j, L, d);
            double e = pot_pair(&pp, i, j, d, fv, &vir);
            if (j > i) {
                e_tot += e;
                w_tot += vir;
            }
            for (int a = 0; a < 3; ++a) fi[a] += fv[a];
        }
        for (int a = 0; a < 3; ++a) F[3 * i + a] = fi[a];
    }
    if (energy_virial) {
        energy_virial[0] = e_tot;
        energy_virial[1] = w_tot;
    }
    free(u);
}

/* Net-force correction (Sec. 2 after Eq. (4); Appendix A, F_cor): subtract the
 * mean force so that the total force, and hence total momentum, is conserved. */
void orc_subtract_mean(int n, double *F)
{
    double m[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) m[a] += F[3 * i + a];
    for (int a = 0; a < 3; ++a) m[a] /= (double)n;
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) F[3 * i + a] -= m[a];
}

/* ------------------------------------------------------------------------- */
/* Time stepping (Algorithm 1; Sec. 2, Eq. (2); Sec. 3: velocity-Verlet for the
 * underdamped Langevin equation, gamma = 1).  The splitting is BAOAB (Leimkuhler
 * & Matthews 2013, cited by the paper with the algorithm):
 *   B: v += dt/2 F   A: x += dt/2 v   O: v = c1 v + sqrt((1 - c1^2) T) xi
 *   A: x += dt/2 v   wrap   [rebuild?]   F = F(x)   B: v += dt/2 F,
 * c1 = exp(-gamma dt).  gamma = 0 is plain velocity-Verlet: B, x += dt v, wrap,
 * [rebuild?], F, B.  Lists are rebuilt when some particle has moved by more than
 * skin/2 since the last build (distance taken like the pair rule).  Step n uses
 * batch and noise counters n; the force after step n uses counter n + 1.        */
/* ------------------------------------------------------------------------- */
typedef struct {
    double L[3];
    double rc, rs, skin;
    int p;
    int K;
    double dt, T, gamma;
    uint64_t seed;
    int subtract_mean;
    int full_list; /* 1: classical cutoff (no batch) */
    int cap_core, cap_shell, cap_full;
    const double *q; /* charges (NULL: LJ only) */
    double alpha;
} orc_params;

typedef struct {
    int n;
    double *x, *v, *F;
    int32_t *core, *n_core, *shell, *n_shell, *full, *n_full;
    uint32_t *u_build;
    uint64_t step;
    int64_t n_rebuild;
    double ev[2];
} orc_state;

static int orc_rebuild(const orc_params *pr, orc_state *s)
{
    int st;
    if (pr->full_list)
        st = orc_build_lists_cells(s->n, s->x, pr->L, pr->rc, pr->rs, pr->skin, pr->K, pr->cap_core,
                                   pr->cap_shell, pr->cap_full, s->core, s->n_core, s->shell, s->n_shell,
                                   s->full, s->n_full);
    else
        st = orc_build_lists_cells(s->n, s->x, pr->L, pr->rc, pr->rs, pr->skin, pr->K, pr->cap_core,
                                   pr->cap_shell, 0, s->core, s->n_core, s->shell, s->n_shell, NULL, NULL);
    orc_quantize(s->n, s->x, pr->L, s->u_build);
    s->n_rebuild += 1;
    return st;
}

static int orc_need_rebuild(const orc_params *pr, const orc_state *s)
{
    fixed_frame f;
    frame_init(&f, pr->L);
    thresholds t = make_thresholds(pr->rc, pr->rs, pr->skin);
    int need = 0;
    for (int i = 0; i < s->n && !need; ++i) {
        uint32_t ui[3];
        for (int a = 0; a < 3; ++a) ui[a] = quantize1(s->x[3 * i + a], f.inv[a]);
        if (pair_r2f(ui, s->u_build + 3 * i, f.h) > t.disp) need = 1;
    }
    return need;
}

static int orc_force_eval(const orc_params *pr, orc_state *s)
{
    int st;
    if (pr->full_list)
        st = orc_full_forces(s->n, s->x, pr->L, pr->rs, s->full, s->n_full, pr->cap_full, s->F, s->ev, pr->q,
                             pr->alpha);
    else
        st = orc_rbl_forces(s->n, s->x, pr->L, pr->rc, pr->rs, pr->skin, pr->p, pr->seed, s->step, s->core,
                            s->n_core, pr->cap_core, s->shell, s->n_shell, pr->cap_shell, s->F, s->ev, NULL,
                            NULL, pr->q, pr->alpha);
    if (pr->subtract_mean) orc_subtract_mean(s->n, s->F);
    return st;
}

static void wrap(double *x, const double L[3])
{
    for (int a = 0; a < 3; ++a) {
        if (x[a] < 0.0) x[a] += L[a];
        if (x[a] >= L[a]) x[a] -= L[a];
    }
}

/* Runs n_steps steps from (x, v); x, v updated in place; F_out gets the final
 * force (after the mean subtraction when enabled); stats_out = {U_est, W_est,
 * rebuilds}.  Lists are built at the start.  step0 = counter of the first force. */
int orc_run(int n, double *x, double *v, double *F_out, const double L[3], double rc, double rs, double skin,
            int p, int K, double dt, double T, double gamma, uint64_t seed, uint64_t step0, int n_steps,
            int subtract_mean, int full_list, int cap_core, int cap_shell, int cap_full, double *stats_out,
            const double *q, double alpha)
{
    orc_params pr;
    memcpy(pr.L, L, sizeof(pr.L));
    pr.rc = rc; pr.rs = rs; pr.skin = skin; pr.p = p; pr.K = K;
    pr.dt = dt; pr.T = T; pr.gamma = gamma; pr.seed = seed;
    pr.subtract_mean = subtract_mean; pr.full_list = full_list;
    pr.cap_core = cap_core; pr.cap_shell = cap_shell; pr.cap_full = cap_full;
    pr.q = q; pr.alpha = alpha;
    orc_state s;
    s.n = n; s.x = x; s.v = v; s.F = F_out; s.step = step0; s.n_rebuild = 0;
    s.core = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * cap_core);
    s.shell = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * cap_shell);
    s.full = full_list ? (int32_t *)malloc(sizeof(int32_t) * (size_t)n * cap_full) : NULL;
    s.n_core = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    s.n_shell = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    s.n_full = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    s.u_build = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (size_t)n);
    int st = orc_rebuild(&pr, &s);
    if (st == ORC_OK) st = orc_force_eval(&pr, &s);
    double c1 = exp(-gamma * dt);
    double c2 = sqrt((1.0 - c1 * c1) * T);
    for (int it = 0; it < n_steps && st == ORC_OK; ++it) {
        double half = 0.5 * dt;
        for (int i = 0; i < n; ++i) {
            double *xi = x + 3 * i, *vi = v + 3 * i, *Fi = s.F + 3 * i;
            for (int a = 0; a < 3; ++a) vi[a] += half * Fi[a];
            if (gamma > 0.0) {
                double xi_n[3];
                orc_gaussians(seed, s.step, (uint32_t)i, xi_n);
                for (int a = 0; a < 3; ++a) xi[a] += half * vi[a];
                for (int a = 0; a < 3; ++a) vi[a] = c1 * vi[a] + c2 * xi_n[a];
                for (int a = 0; a < 3; ++a) xi[a] += half * vi[a];
            } else {
                for (int a = 0; a < 3; ++a) xi[a] += dt * vi[a];
            }
            wrap(xi, L);
        }
        s.step += 1;
        if (orc_need_rebuild(&pr, &s)) st = orc_rebuild(&pr, &s);
        if (st != ORC_OK) break;
        st = orc_force_eval(&pr, &s);
        for (int i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a) v[3 * i + a] += half * s.F[3 * i + a];
    }
    if (stats_out) {
        stats_out[0] = s.ev[0];
        stats_out[1] = s.ev[1];
        stats_out[2] = (double)s.n_rebuild;
    }
    free(s.core); free(s.shell); free(s.full); free(s.n_core); free(s.n_shell); free(s.n_full); free(s.u_build);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Observables (Sec. 3).                                                         */
/* ------------------------------------------------------------------------- */
/* Tail corrections for r >= r_s of an unshifted truncated LJ fluid of density
 * rho: per-particle energy (8/3) pi rho (r_s^-9/3 - r_s^-3) and pressure
 * (16/3) pi rho^2 (2 r_s^-9/3 - r_s^-3).                                       */
void orc_tail(double rho, double rs, double out[2])
{
    const double pi = 3.14159265358979323846264338327950288;
    double i3 = 1.0 / (rs * rs * rs);
    double i9 = i3 * i3 * i3;
    out[0] = 8.0 / 3.0 * pi * rho * (i9 / 3.0 - i3);
    out[1] = 16.0 / 3.0 * pi * rho * rho * (2.0 * i9 / 3.0 - i3);
}

/* Kinetic energy sum(v^2)/2 and the instantaneous pressure
 * P = rho T_kin + W / (3V), T_kin = 2K / (3N), W = sum over pairs of r.f. */
void orc_thermo(int n, const double *v, const double L[3], double W, double out[3])
{
    double k = 0.0;
    for (int i = 0; i < 3 * n; ++i) k += v[i] * v[i];
    k *= 0.5;
    double V = L[0] * L[1] * L[2];
    double tkin = 2.0 * k / (3.0 * n);
    out[0] = k;
    out[1] = tkin;
    out[2] = (double)n / V * tkin + W / (3.0 * V);
}

/* Radial distribution function histogram (Sec. 3, g(r) definition): counts of
 * ordered pairs (i, j != i) with bin = floor(sqrt(r2) / dr) < nbins, r2 taken
 * like the pair rule and the square root in binary32.                           */
void orc_rdf_counts(int n, const double *x, const double L[3], float dr, int nbins, int64_t *hist)
{
    fixed_frame f;
    frame_init(&f, L);
    uint32_t *u = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (size_t)n);
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) u[3 * i + a] = quantize1(x[3 * i + a], f.inv[a]);
    memset(hist, 0, sizeof(int64_t) * (size_t)nbins);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            float r = sqrtf(pair_r2f(u + 3 * i, u + 3 * j, f.h));
            float q = r / dr;
            if (q < (float)nbins) hist[(int)q] += 1;
        }
    free(u);
}

/* ------------------------------------------------------------------------- */
/* Thread count of the OpenMP loops, for timing the oracle single-threaded and on
 * all host cores.  Forces, lists and trajectories do not depend on it; only the
 * order of the FP64 energy/virial reductions does.                           */
/* ------------------------------------------------------------------------- */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Density profile along one axis (Sec. 3 observables): particle counts in nbins
 * slabs of equal width; particle i goes to bin floor(u_a nbins / 2^32), u_a its
 * 32-bit fixed-point image (the rule that assigns cells).  hist accumulated.    */
/* ------------------------------------------------------------------------- */
void orc_density_profile(int n, const double *x, const double L[3], int axis, int nbins, int64_t *hist)
{
    fixed_frame f;
    frame_init(&f, L);
    for (int i = 0; i < n; ++i) {
        uint32_t u = quantize1(x[3 * i + axis], f.inv[axis]);
        hist[(int)(((uint64_t)u * (uint64_t)nbins) >> 32)] += 1;
    }
}

/* ------------------------------------------------------------------------- */
/* The paper's own sampling pool (Sec. 2, Fig. 1).  The box is cut into cells of
 * edge at least r_c + skin (n_a = floor(L_a / (r_c + skin)); the paper's "slightly
 * larger than r_c").  The pool I(i) is every particle j != i in the stencil of
 * (2m + 1)^3 cells centred on i's cell, m = floor(r_s / r_c) + 1 (fewer cells, each
 * once, on an axis with fewer than 2m + 1), in canonical order (stencil slot, u_x,
 * tag) on that grid.  The core row, j != i with r2 < (r_c + skin)^2, is sorted the
 * same way.  A batch is then drawn from the pool exactly as from a shell row and
 * scaled by N_I / p (Eq. (4) with N_I), so orc_rbl_forces applies unchanged with
 * the pool in place of the shell rows.  Brute force over all pairs.              */
/* ------------------------------------------------------------------------- */
static void grid_init_pool(cell_grid *g, const double L[3], double rc, double rs, double skin)
{
    const int m = (int)floor(rs / rc) + 1;
    for (int a = 0; a < 3; ++a) {
        int n = (int)floor(L[a] / (rc + skin));
        if (n < 1) n = 1;
        g->n[a] = n;
        if (n >= 2 * m + 1) {
            g->nofs[a] = 2 * m + 1;
            for (int o = 0; o < 2 * m + 1; ++o) g->ofs[a][o] = o - m;
        } else {
            g->nofs[a] = n;
            for (int o = 0; o < n; ++o) g->ofs[a][o] = o;
        }
    }
}

int orc_build_pool(int n, const double *x, const double L[3], double rc, double rs, double skin, int cap_core,
                   int cap_pool, int32_t *core, int32_t *n_core, int32_t *pool, int32_t *n_pool, int32_t *grid_n)
{
    fixed_frame f;
    frame_init(&f, L);
    thresholds t = make_thresholds(rc, rs, skin);
    cell_grid g;
    grid_init_pool(&g, L, rc, rs, skin);
    if (grid_n)
        for (int a = 0; a < 3; ++a) grid_n[a] = g.n[a];
    uint32_t *u = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (size_t)n);
    int *cells3 = (int *)malloc(sizeof(int) * 3 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) u[3 * i + a] = quantize1(x[3 * i + a], f.inv[a]);
        cell_of(&g, u + 3 * i, cells3 + 3 * i);
    }
    int status = ORC_OK;
#pragma omp parallel
    {
        int maxcap = cap_core > cap_pool ? cap_core : cap_pool;
        row_key *scratch = (row_key *)malloc(sizeof(row_key) * (size_t)(maxcap + 1));
#pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i) {
            int nc = 0, np = 0;
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                if (stencil_slot(&g, cells3 + 3 * i, cells3 + 3 * j) >= 0) {
                    if (np < cap_pool) pool[(size_t)i * cap_pool + np] = j;
                    ++np;
                }
                float r2 = pair_r2f(u + 3 * i, u + 3 * j, f.h);
                if (r2 < t.core_list) {
                    if (nc < cap_core) core[(size_t)i * cap_core + nc] = j;
                    ++nc;
                }
            }
            if (nc > cap_core || np > cap_pool) {
#pragma omp atomic write
                status = ORC_EOVERFLOW;
            } else {
                sort_row(core + (size_t)i * cap_core, nc, &g, cells3, u, i, scratch);
                sort_row(pool + (size_t)i * cap_pool, np, &g, cells3, u, i, scratch);
            }
            n_core[i] = nc;
            n_pool[i] = np;
        }
        free(scratch);
    }
    free(u);
    free(cells3);
    return status;
}
