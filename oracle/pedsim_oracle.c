/*
 * Plain single-threaded CPU oracle of the bi-directional pedestrian cellular
 * automaton (Least Effort Model and the pheromone-guided ACO variant) of
 * Dutta, McLeod, Friesen, "GPU accelerated Nature Inspired Methods for
 * Modelling Large Scale Bi-Directional Pedestrian Movement".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or constant table with the
 * CUDA library; both follow the same written rules independently.
 *
 * The oracle is deliberately slow and literal.  It keeps the paper's data
 * structures: the environment matrix `mat` (0 empty, 1 group A, 2 group B),
 * the index matrix (agent id per cell, 0 = empty) and a per-agent property
 * matrix with ROW, COLUMN, FUTURE ROW and FUTURE COLUMN (Sec. IV.a, Table I),
 * and it runs the paper's phases in order each step:
 *   1. initial calculation + tour construction (Sec. IV.b-c): every agent
 *      inspects its 8 neighbours and writes its FUTURE cell;
 *   2. agent movement (Sec. IV.d): evaporation (Eq. 3) first, then every
 *      empty cell gathers the agents whose FUTURE points at it and picks one
 *      (scatter-to-gather, no atomics), then the deposit (Eq. 4).
 *
 * Geometry (transposed from the paper's top/bottom groups so that "forward"
 * runs along the contiguous x axis): H rows by W columns, cell c = y*W + x.
 * Group A starts in the leftmost band_cols columns and heads +x; group B
 * starts in the rightmost band_cols columns and heads -x.  Cells outside the
 * grid are never available (Sec. III: border and corner positions).
 *
 * Readings of points the paper leaves open (each one is a choice, stated
 * where it is used):
 *   - neighbour numbering of Fig. 1 (missing figure) from Sec. IV.b: #1
 *     forward, #2/#3 forward diagonals, #4/#5 lateral, #6 back, #7/#8 back
 *     diagonals (left before right of the heading);
 *   - the constant distance table (Sec. IV.a) = Euclidean distance from the
 *     neighbour to the point two cells ahead of the agent:
 *     {1, sqrt2, sqrt2, sqrt5, sqrt5, 3, sqrt10, sqrt10}; D_min = 1 so the
 *     heuristic of Eq. 2 is eta_i = D_min/D_i = 1/D_i (Eq. 1 with n_i = 0);
 *   - the LEM normal draw (Sec. II.A, Sec. IV.c) is the classical sum of 12
 *     uniforms (here 12 independent 16-bit words) minus its mean, scaled by
 *     2^-16/sigma; negative -> 0, then rounded half up, then clamped to the
 *     last rank; equal-distance pairs are ordered by one random bit each;
 *   - ACO (Eq. 2) with integer alpha, beta; if every weight is zero the
 *     agent falls back to the LEM choice;
 *   - conflict winner = claimant[floor(r * k / 2^32)] with claimants taken in
 *     fixed row-major neighbour order (Sec. IV.d, Fig. 4);
 *   - an agent on its target edge column stays there (Sec. III: as far as
 *     possible until no further movement is possible);
 *   - crossing (Sec. VI) = first entry into the opposite placement band;
 *   - random numbers are Philox4x64-10 keyed by (seed, cell, step, stream)
 *     instead of the paper's CURAND states.
 *
 * Arithmetic is IEEE binary32, round to nearest, no FMA contraction (build
 * with -ffp-contract=off), subnormals kept.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Philox4x64-10, from its published definition (Salmon, Moraes, Dror, Shaw, */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 4.2): each     */
/* round multiplies words 0 and 2 by two fixed odd constants, swaps the      */
/* halves across the pairs and xors in the key; the key is bumped by two     */
/* Weyl constants between rounds.                                            */
/* ------------------------------------------------------------------------ */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ULL;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ULL;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ULL; /* golden ratio */
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73BULL; /* sqrt(3) - 1  */

ORC_EXPORT void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2],
                                  uint64_t out[4])
{
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        unsigned __int128 p0 = (unsigned __int128)PHILOX_M0 * x0;
        unsigned __int128 p1 = (unsigned __int128)PHILOX_M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        x0 = hi1 ^ x1 ^ k0;
        x1 = lo1;
        x2 = hi0 ^ x3 ^ k1;
        x3 = lo0;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Random streams: one counter per (cell, step, purpose). */
enum { STREAM_PROPOSE = 1, STREAM_CONFLICT = 2, STREAM_PLACE = 3 };

/* ------------------------------------------------------------------------ */
/* Parameters and state                                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint32_t model;        /* 0 = LEM (Sec. II.A), 1 = ACO (Sec. II.B)        */
    uint32_t n_per_side;   /* agents in each group                            */
    uint32_t band_cols;    /* placement band width at each edge               */
    float    rho;          /* evaporation rate of Eq. 3, 0 < rho <= 1         */
    float    tau0;         /* initial pheromone on every cell                 */
    float    deposit;      /* constant deposit per visit (deposit_mode 0)     */
    uint32_t alpha, beta;  /* exponents of Eq. 2                              */
    uint32_t deposit_mode; /* 0 = constant, 1 = 1/L_k of Eq. 5                */
    float    lem_sigma;    /* standard deviation of the LEM normal draw       */
} orc_params;

typedef struct {
    uint64_t step;
    uint32_t agents[2], crossed[2], parked[2];
    uint64_t moved, conflicts;
} orc_stats;

typedef struct {
    int W, H, mirror;
    orc_params p;
    uint64_t seed, step;
    uint32_t n_agents;          /* 2 * n_per_side                              */
    uint8_t  *mat;              /* environment matrix                          */
    uint32_t *index;            /* index matrix                                */
    /* property matrix, rows 0..n_agents (row 0 unused, Sec. IV.a) */
    uint8_t  *group;
    int32_t  *row, *col, *future_row, *future_col;
    uint32_t *arrival;          /* step at which the agent first crossed, 0 = not yet */
    float    *tour;             /* tour length L_k (Eq. 5)                     */
    float    *tau[2];           /* pheromone matrices of group A and group B  */
    uint64_t moved, conflicts;
} orc_t;

/* Agent-frame neighbour offsets for i = 0..8 (0 = the agent's own cell).
 * The absolute offset of neighbour i of an agent heading s (+1 for group A,
 * -1 for group B) is (s*FRAME_FX[i], s*FRAME_FY[i]): forward is +s in x and
 * "left of the heading" is -s in y.                                         */
static const int FRAME_FX[9] = {0, 1, 1, 1, 0, 0, -1, -1, -1};
static const int FRAME_FY[9] = {0, 0, -1, 1, -1, 1, 0, -1, 1};

/* Fixed absolute scan order of the gather step (row-major over dy, dx). */
static const int SCAN_DX[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
static const int SCAN_DY[8] = {-1, -1, -1, 0, 0, 1, 1, 1};

/* eta_i = 1/D_i with D the distance from neighbour i to the point two cells
 * ahead of the agent; the float is the correctly rounded value.              */
static float eta_table[9];
static int   eta_ready = 0;

static void init_eta(void)
{
    if (eta_ready) return;
    /* squared distances from neighbour (fx, fy) to (2, 0) in the agent frame */
    for (int i = 1; i <= 8; ++i) {
        double dx = 2.0 - FRAME_FX[i], dy = 0.0 - FRAME_FY[i];
        double d = sqrt(dx * dx + dy * dy);
        eta_table[i] = (float)(1.0 / d);
    }
    eta_table[0] = 0.0f;
    eta_ready = 1;
}

ORC_EXPORT float orc_eta(int i)
{
    init_eta();
    return (i >= 1 && i <= 8) ? eta_table[i] : 0.0f;
}

static int in_grid(const orc_t *o, int x, int y)
{
    return x >= 0 && x < o->W && y >= 0 && y < o->H;
}

/* Counter word for a cell: the cell index, or its point reflection through
 * the grid centre in the test-only mirror mode.                              */
static uint64_t cell_key(const orc_t *o, int x, int y)
{
    uint64_t c = (uint64_t)y * (uint64_t)o->W + (uint64_t)x;
    if (o->mirror) c = (uint64_t)o->W * (uint64_t)o->H - 1u - c;
    return c;
}

static void draw(const orc_t *o, int x, int y, uint64_t step, uint64_t stream,
                 uint64_t r[4])
{
    uint64_t ctr[4] = {cell_key(o, x, y), step, stream, 0};
    uint64_t key[2] = {o->seed, 0};
    orc_philox4x64_10(ctr, key, r);
}

/* ------------------------------------------------------------------------ */
/* LEM choice (Eq. 1 and Sec. II.A)                                          */
/* ------------------------------------------------------------------------ */

/* Sum of the twelve 16-bit words of r[0], r[1], r[2]. */
static int32_t twelve_uniform_sum(const uint64_t r[4])
{
    int32_t s = 0;
    for (int w = 0; w < 3; ++w)
        for (int h = 0; h < 4; ++h)
            s += (int32_t)((r[w] >> (16 * h)) & 0xFFFFu);
    return s;
}

/* Scale of the normal draw: 2^-16 is 1/sqrt(var) of the 12-word sum up to a
 * relative 2^-33, below binary32 resolution.                                */
static float lem_scale(float sigma) { return 0x1p-16f / sigma; }

/* Rank index from the 12-word sum: negative -> 0, rounded half up, clamped
 * to the highest rank m-1 (Sec. II.A).                                       */
ORC_EXPORT int orc_lem_rank(int32_t sum12, int m, float sigma)
{
    float z = (float)(sum12 - 393210) * lem_scale(sigma);  /* 12 * 32767.5 */
    float zc = fmaxf(z, 0.0f);
    int k = (int)floorf(zc + 0.5f);
    if (k > m - 1) k = m - 1;
    return k;
}

/* Test helper: rank index for every possible 12-word sum 0..786420. */
ORC_EXPORT void orc_lem_rank_table(int m, float sigma, int8_t *out)
{
    for (int32_t s = 0; s <= 12 * 65535; ++s) out[s] = (int8_t)orc_lem_rank(s, m, sigma);
}

/* Available neighbours listed by ascending distance; each equal-distance
 * pair (2,3), (4,5), (7,8) is listed left-first unless its tie bit is set.   */
static int lem_choice(const int avail[9], const uint64_t r[4], float sigma)
{
    int order[8] = {1, 2, 3, 4, 5, 6, 7, 8};
    if (r[3] & 1u) { order[1] = 3; order[2] = 2; }
    if (r[3] & 2u) { order[3] = 5; order[4] = 4; }
    if (r[3] & 4u) { order[6] = 8; order[7] = 7; }
    int list[8], m = 0;
    for (int j = 0; j < 8; ++j)
        if (avail[order[j]]) list[m++] = order[j];
    if (m == 0) return 0;
    int k = orc_lem_rank(twelve_uniform_sum(r), m, sigma);
    return list[k];
}

/* ------------------------------------------------------------------------ */
/* ACO choice (Eq. 2): roulette over tau^alpha * eta^beta                     */
/* ------------------------------------------------------------------------ */
static float int_pow(float v, uint32_t e)
{
    float p = 1.0f;
    if (e == 0) return p;
    p = v;
    for (uint32_t i = 1; i < e; ++i) p = p * v;
    return p;
}

ORC_EXPORT float orc_aco_weight(float tau, float eta, uint32_t alpha, uint32_t beta)
{
    return int_pow(tau, alpha) * int_pow(eta, beta);
}

/* Roulette pick among i = 2..8 with u24 the 24-bit uniform; w[0..8].  Returns
 * 0 when the sum is zero (caller falls back to LEM).                         */
ORC_EXPORT int orc_aco_pick(const float w[9], uint32_t u24)
{
    float S = 0.0f;
    for (int i = 2; i <= 8; ++i) S = S + w[i];
    if (!(S > 0.0f)) return 0;
    float u = (float)u24 * 0x1p-24f;
    float t = u * S;
    float cum = 0.0f;
    int last = 0;
    for (int i = 2; i <= 8; ++i) {
        cum = cum + w[i];
        if (w[i] > 0.0f) last = i;
        if (t < cum) return i;
    }
    return last;
}

/* Test helper: histogram of the roulette over every one of the 2^24 u24. */
ORC_EXPORT void orc_aco_histogram(const float w[9], uint64_t counts[9])
{
    for (int i = 0; i < 9; ++i) counts[i] = 0;
    for (uint32_t u = 0; u < (1u << 24); ++u) counts[orc_aco_pick(w, u)]++;
}

/* Conflict winner index among k claimants from a 32-bit uniform. */
ORC_EXPORT uint32_t orc_conflict_index(uint32_t r32, uint32_t k)
{
    return (uint32_t)(((uint64_t)r32 * (uint64_t)k) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Phase 1+2 of a step: one agent decides its FUTURE cell (Sec. IV.b, IV.c)  */
/* Returns the agent-frame index 0..8 (0 = stay).                            */
/* ------------------------------------------------------------------------ */
static int decide(const orc_t *o, int x, int y, int g)
{
    const int s = (g == 1) ? 1 : -1;
    /* an agent on its target edge column has arrived and stays */
    if ((g == 1 && x == o->W - 1) || (g == 2 && x == 0)) return 0;

    int avail[9];
    avail[0] = 0;
    for (int i = 1; i <= 8; ++i) {
        int nx = x + s * FRAME_FX[i], ny = y + s * FRAME_FY[i];
        avail[i] = in_grid(o, nx, ny) && o->mat[ny * o->W + nx] == 0;
    }
    /* forward-first (Sec. III): no further calculation when #1 is empty */
    if (avail[1]) return 1;

    uint64_t r[4];
    draw(o, x, y, o->step, STREAM_PROPOSE, r);

    if (o->p.model == 1) {
        const float *tau = o->tau[g - 1];
        float w[9] = {0};
        for (int i = 2; i <= 8; ++i) {
            if (!avail[i]) continue;
            int nx = x + s * FRAME_FX[i], ny = y + s * FRAME_FY[i];
            w[i] = orc_aco_weight(tau[ny * o->W + nx], eta_table[i], o->p.alpha, o->p.beta);
        }
        int pick = orc_aco_pick(w, (uint32_t)(r[3] >> 40));
        if (pick != 0) return pick;
        /* every weight zero: fall back to the least-effort rule */
    }
    return lem_choice(avail, r, o->p.lem_sigma);
}

/* Test hook: the frame index the agent at (x, y) would choose at this step. */
ORC_EXPORT int orc_decide_at(const orc_t *o, int x, int y)
{
    if (!in_grid(o, x, y)) return -1;
    int g = o->mat[y * o->W + x];
    if (g == 0) return -1;
    return decide(o, x, y, g);
}

/* ------------------------------------------------------------------------ */
/* Construction, placement (Sec. IV.a)                                        */
/* ------------------------------------------------------------------------ */
ORC_EXPORT int orc_check_params(int W, int H, const orc_params *p)
{
    if (W < 16 || H < 16 || (W % 16) != 0 || (H % 16) != 0) return -22;
    if ((int64_t)W * (int64_t)H > ((int64_t)1 << 31)) return -22;
    if (p->model > 1 || p->deposit_mode > 1) return -22;
    if (p->band_cols < 1 || 2u * p->band_cols > (uint32_t)W) return -22;
    if ((uint64_t)p->n_per_side > (uint64_t)p->band_cols * (uint64_t)H) return -22;
    if (!(p->lem_sigma > 0.0f) || !isfinite(p->lem_sigma)) return -22;
    if (p->model == 1) {
        if (!(p->rho > 0.0f && p->rho <= 1.0f)) return -22;
        if (p->alpha > 4 || p->beta > 4) return -22;
        if (!(p->tau0 >= 0.0f) || !isfinite(p->tau0)) return -22;
        if (!(p->deposit >= 0.0f) || !isfinite(p->deposit)) return -22;
    }
    return 0;
}

typedef struct { uint64_t key, tie; int32_t cell; } place_key;

static int cmp_place_key(const void *a, const void *b)
{
    const place_key *u = (const place_key *)a, *v = (const place_key *)b;
    if (u->key != v->key) return u->key < v->key ? -1 : 1;
    if (u->tie != v->tie) return u->tie < v->tie ? -1 : 1;
    return 0;
}

static int cmp_int32(const void *a, const void *b)
{
    int32_t u = *(const int32_t *)a, v = *(const int32_t *)b;
    return (u > v) - (u < v);
}

/* Uniform placement of n agents in a band of columns [x0, x1): the n band
 * cells with the smallest Philox keys (ties by counter cell word) are taken;
 * ids are handed out in increasing cell index starting at first_id.          */
static void place_group(orc_t *o, int g, int x0, int x1, uint32_t first_id)
{
    const uint32_t n = o->p.n_per_side;
    const int bw = x1 - x0;
    const size_t m = (size_t)bw * (size_t)o->H;
    place_key *keys = (place_key *)malloc(m * sizeof(place_key));
    size_t j = 0;
    for (int y = 0; y < o->H; ++y)
        for (int x = x0; x < x1; ++x) {
            uint64_t r[4];
            draw(o, x, y, 0, STREAM_PLACE, r);
            keys[j].key = r[0];
            keys[j].tie = cell_key(o, x, y);
            keys[j].cell = y * o->W + x;
            ++j;
        }
    qsort(keys, m, sizeof(place_key), cmp_place_key);
    int32_t *cells = (int32_t *)malloc((n ? n : 1) * sizeof(int32_t));
    for (uint32_t i = 0; i < n; ++i) cells[i] = keys[i].cell;
    qsort(cells, n, sizeof(int32_t), cmp_int32);
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t id = first_id + i;
        int32_t c = cells[i];
        o->mat[c] = (uint8_t)g;
        o->index[c] = id;
        o->group[id] = (uint8_t)g;
        o->row[id] = c / o->W;
        o->col[id] = c % o->W;
        o->future_row[id] = o->row[id];
        o->future_col[id] = o->col[id];
    }
    free(cells);
    free(keys);
}

ORC_EXPORT void orc_destroy(orc_t *o)
{
    if (!o) return;
    free(o->mat); free(o->index); free(o->group); free(o->row); free(o->col);
    free(o->future_row); free(o->future_col); free(o->arrival); free(o->tour);
    free(o->tau[0]); free(o->tau[1]);
    free(o);
}

static orc_t *alloc_state(int W, int H, const orc_params *p, uint64_t seed, int mirror)
{
    init_eta();
    orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
    if (!o) return NULL;
    o->W = W; o->H = H; o->mirror = mirror; o->p = *p; o->seed = seed; o->step = 0;
    o->n_agents = 2u * p->n_per_side;
    size_t cells = (size_t)W * (size_t)H, rows = (size_t)o->n_agents + 1;
    o->mat = (uint8_t *)calloc(cells, 1);
    o->index = (uint32_t *)calloc(cells, sizeof(uint32_t));
    o->group = (uint8_t *)calloc(rows, 1);
    o->row = (int32_t *)calloc(rows, sizeof(int32_t));
    o->col = (int32_t *)calloc(rows, sizeof(int32_t));
    o->future_row = (int32_t *)calloc(rows, sizeof(int32_t));
    o->future_col = (int32_t *)calloc(rows, sizeof(int32_t));
    o->arrival = (uint32_t *)calloc(rows, sizeof(uint32_t));
    o->tour = (float *)calloc(rows, sizeof(float));
    o->tau[0] = (float *)calloc(cells, sizeof(float));
    o->tau[1] = (float *)calloc(cells, sizeof(float));
    if (!o->mat || !o->index || !o->group || !o->row || !o->col || !o->future_row ||
        !o->future_col || !o->arrival || !o->tour || !o->tau[0] || !o->tau[1]) {
        orc_destroy(o);
        return NULL;
    }
    for (size_t c = 0; c < cells; ++c) { o->tau[0][c] = p->tau0; o->tau[1][c] = p->tau0; }
    return o;
}

ORC_EXPORT orc_t *orc_create(int W, int H, const orc_params *p, uint64_t seed, int mirror)
{
    if (orc_check_params(W, H, p) != 0) return NULL;
    orc_t *o = alloc_state(W, H, p, seed, mirror);
    if (!o) return NULL;
    place_group(o, 1, 0, (int)p->band_cols, 1u);
    place_group(o, 2, W - (int)p->band_cols, W, p->n_per_side + 1u);
    return o;
}

/* Test hook: start from an arbitrary state.  occ/ids describe the grid (ids
 * must be a permutation of 1..n over the occupied cells; an agent's group is
 * its occ code); tau planes may be NULL (then tau0); arrival may be NULL
 * (then zero).  n_per_side in p is ignored.                                  */
ORC_EXPORT orc_t *orc_create_from_state(int W, int H, const orc_params *p, uint64_t seed,
                                        uint64_t step, int mirror, const uint8_t *occ,
                                        const uint32_t *ids, const float *tauA,
                                        const float *tauB, const uint32_t *arrival)
{
    orc_params q = *p;
    size_t cells = (size_t)W * (size_t)H;
    uint32_t n = 0;
    for (size_t c = 0; c < cells; ++c) n += occ[c] != 0;
    q.n_per_side = (n + 1) / 2;
    orc_t *o = alloc_state(W, H, &q, seed, mirror);
    if (!o) return NULL;
    o->n_agents = n;
    o->step = step;
    for (size_t c = 0; c < cells; ++c) {
        if (!occ[c]) continue;
        uint32_t id = ids[c];
        if (id < 1 || id > n || occ[c] > 2 || o->group[id] != 0) { orc_destroy(o); return NULL; }
        o->mat[c] = occ[c];
        o->index[c] = id;
        o->group[id] = occ[c];
        o->row[id] = (int32_t)(c / (size_t)W);
        o->col[id] = (int32_t)(c % (size_t)W);
        if (arrival) o->arrival[id] = arrival[id];
    }
    if (tauA) memcpy(o->tau[0], tauA, cells * sizeof(float));
    if (tauB) memcpy(o->tau[1], tauB, cells * sizeof(float));
    return o;
}

/* ------------------------------------------------------------------------ */
/* One synchronous step t -> t+1                                             */
/* ------------------------------------------------------------------------ */
typedef struct { uint32_t agent; int32_t cell; } move_t;

static int in_opposite_band(const orc_t *o, int g, int x)
{
    return g == 1 ? x >= o->W - (int)o->p.band_cols : x < (int)o->p.band_cols;
}

static void one_step(orc_t *o)
{
    const int W = o->W, H = o->H;

    /* Initial calculation and tour construction: every agent fills FUTURE. */
    for (uint32_t a = 1; a <= o->n_agents; ++a) {
        int x = o->col[a], y = o->row[a], g = o->group[a];
        int s = (g == 1) ? 1 : -1;
        int i = decide(o, x, y, g);
        o->future_col[a] = x + s * FRAME_FX[i];
        o->future_row[a] = y + s * FRAME_FY[i];
    }

    /* Agent movement, evaporation first (Eq. 3 before Eq. 4). */
    if (o->p.model == 1) {
        const float q = 1.0f - o->p.rho;
        for (size_t c = 0; c < (size_t)W * (size_t)H; ++c) {
            o->tau[0][c] = o->tau[0][c] * q;
            o->tau[1][c] = o->tau[1][c] * q;
        }
    }

    /* Gather: each empty cell collects its claimants in the fixed order. */
    move_t *moves = (move_t *)malloc(((size_t)o->n_agents + 1) * sizeof(move_t));
    size_t n_moves = 0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            if (o->mat[y * W + x] != 0) continue;
            uint32_t claimant[8];
            uint32_t k = 0;
            for (int j = 0; j < 8; ++j) {
                int jj = o->mirror ? 7 - j : j;
                int nx = x + SCAN_DX[jj], ny = y + SCAN_DY[jj];
                if (!in_grid(o, nx, ny)) continue;
                uint32_t a = o->index[ny * W + nx];
                if (a != 0 && o->future_col[a] == x && o->future_row[a] == y)
                    claimant[k++] = a;
            }
            if (k == 0) continue;
            uint32_t pick = 0;
            if (k >= 2) {
                uint64_t r[4];
                draw(o, x, y, o->step, STREAM_CONFLICT, r);
                pick = orc_conflict_index((uint32_t)(r[0] >> 32), k);
                o->conflicts++;
            }
            moves[n_moves].agent = claimant[pick];
            moves[n_moves].cell = y * W + x;
            ++n_moves;
        }

    /* Exchange the winners with their empty target cells; deposit. */
    for (size_t m = 0; m < n_moves; ++m) {
        uint32_t a = moves[m].agent;
        int32_t to = moves[m].cell;
        int32_t from = o->row[a] * W + o->col[a];
        int g = o->group[a];
        int tx = to % W, ty = to / W;
        int diagonal = (tx != o->col[a]) && (ty != o->row[a]);
        o->mat[to] = (uint8_t)g;
        o->index[to] = a;
        o->mat[from] = 0;
        o->index[from] = 0;
        o->col[a] = tx;
        o->row[a] = ty;
        o->moved++;
        if (o->p.model == 1) {
            float dtau = o->p.deposit;
            if (o->p.deposit_mode == 1) {
                /* Eq. 5: the tour length grows by the step length first */
                o->tour[a] = o->tour[a] + (diagonal ? (float)sqrt(2.0) : 1.0f);
                dtau = 1.0f / o->tour[a];
            }
            o->tau[g - 1][to] = o->tau[g - 1][to] + dtau;
        }
        if (o->arrival[a] == 0 && in_opposite_band(o, g, tx))
            o->arrival[a] = (uint32_t)(o->step + 1);
    }
    free(moves);
    o->step++;
}

ORC_EXPORT int orc_step(orc_t *o, int n)
{
    if (!o || n < 0) return -22;
    for (int i = 0; i < n; ++i) one_step(o);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Read-back                                                                  */
/* ------------------------------------------------------------------------ */
ORC_EXPORT void orc_get_state(const orc_t *o, uint8_t *occ, uint32_t *ids, float *tauA,
                              float *tauB, uint32_t *arrival, float *tour)
{
    size_t cells = (size_t)o->W * (size_t)o->H;
    if (occ) memcpy(occ, o->mat, cells);
    if (ids) memcpy(ids, o->index, cells * sizeof(uint32_t));
    if (tauA) memcpy(tauA, o->tau[0], cells * sizeof(float));
    if (tauB) memcpy(tauB, o->tau[1], cells * sizeof(float));
    if (arrival) memcpy(arrival, o->arrival, ((size_t)o->n_agents + 1) * sizeof(uint32_t));
    if (tour) memcpy(tour, o->tour, ((size_t)o->n_agents + 1) * sizeof(float));
}

ORC_EXPORT void orc_get_stats(const orc_t *o, orc_stats *st)
{
    memset(st, 0, sizeof(*st));
    st->step = o->step;
    for (int y = 0; y < o->H; ++y)
        for (int x = 0; x < o->W; ++x) {
            int g = o->mat[y * o->W + x];
            if (!g) continue;
            st->agents[g - 1]++;
            if ((g == 1 && x == o->W - 1) || (g == 2 && x == 0)) st->parked[g - 1]++;
        }
    for (uint32_t a = 1; a <= o->n_agents; ++a)
        if (o->arrival[a]) st->crossed[o->group[a] - 1]++;
    st->moved = o->moved;
    st->conflicts = o->conflicts;
}

ORC_EXPORT uint32_t orc_n_agents(const orc_t *o) { return o->n_agents; }
ORC_EXPORT uint64_t orc_current_step(const orc_t *o) { return o->step; }
