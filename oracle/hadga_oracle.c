/*
 * hadga_oracle.c -- plain, slow, obviously correct CPU reference of the
 * genetic algorithm's per-generation population step (Balogh & Ruiz,
 * "A GPU accelerated Genetic Algorithm for the Construction of Hadamard
 * Matrices", arXiv 2208.14961).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header or constant table with
 * the CUDA library; both sides implement the same published definitions
 * (Philox4x32-10, the paper's operators) independently.
 *
 * Population layout (Sec. 3.1, Eq. (1)-(2), Sec. 3.4): P = 4N matrices of
 * order m = 4k, int8 row-major, entry (i, j) of matrix q at
 * pop[q*m*m + i*m + j]; slots [0, 2N) are parents, [2N, 4N) offspring.
 *
 * Randomness.  The paper draws from cuRAND / cupy.random and is therefore
 * not reproducible; every draw here comes from Philox4x32-10 (Salmon, Moraes,
 * Dror, Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11) with
 *   key     = (seed, pop_id)
 *   counter = (op, generation, index, (sub << 16) | block)
 * Each counter yields four 32-bit words, consumed in order; the stream
 * continues with block + 1.  A word w maps to an integer in [lo, hi] by
 * lo + floor(w * (hi - lo + 1) / 2^32) (multiply-shift, no rejection).
 *
 * Fitness values are accumulated in 64-bit integers; Gram entries in int32.
 *
 * Parity status: every function below is pinned by a test against something
 * other than itself (see the header of each function for what pins it).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_OP_INIT = 0, ORC_OP_SELECT = 1, ORC_OP_CROSS = 2, ORC_OP_MUTATE = 3, ORC_OP_CONFIG = 4,
       ORC_OP_PSELECT = 5 };
enum { ORC_FIT_SQ = 0, ORC_FIT_ABS = 1, ORC_FIT_NNZ = 2 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11, Sec. 4.2): ten rounds of two 32x32->64 multiplies, */
/* key schedule bumped by the Weyl constants between rounds.                */
/* Pinned by the published known-answer vectors.                            */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t mul_a = 0xD2511F53u, mul_b = 0xCD9E8D57u;
    const uint32_t weyl_a = 0x9E3779B9u, weyl_b = 0xBB67AE85u;
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += weyl_a;
            k1 += weyl_b;
        }
        uint64_t prod_a = (uint64_t)mul_a * (uint64_t)x0;
        uint64_t prod_b = (uint64_t)mul_b * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(prod_b >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)prod_b;
        uint32_t y2 = (uint32_t)(prod_a >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)prod_a;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* A sequential word stream over consecutive Philox blocks. */
typedef struct {
    uint32_t key[2];
    uint32_t ctr[4];
    uint32_t block;
    uint32_t sub;
    uint32_t words[4];
    int used;
} orc_stream;

static void stream_open(orc_stream *s, uint32_t seed, uint32_t pop_id, uint32_t op,
                        uint32_t gen, uint32_t index, uint32_t sub)
{
    s->key[0] = seed;
    s->key[1] = pop_id;
    s->ctr[0] = op;
    s->ctr[1] = gen;
    s->ctr[2] = index;
    s->sub = sub;
    s->block = 0;
    s->used = 4; /* forces a refill on the first draw */
}

static uint32_t stream_next(orc_stream *s)
{
    if (s->used == 4) {
        s->ctr[3] = (s->sub << 16) | s->block;
        orc_philox4x32_10(s->ctr, s->key, s->words);
        s->block += 1;
        s->used = 0;
    }
    return s->words[s->used++];
}

/* Integer in [lo, hi] from one 32-bit word (multiply-shift). */
uint32_t orc_uniform(uint32_t w, uint32_t lo, uint32_t hi)
{
    uint64_t span = (uint64_t)hi - (uint64_t)lo + 1u;
    return lo + (uint32_t)(((uint64_t)w * span) >> 32);
}

/* Exposed for tests: the first `count` words of one stream. */
void orc_stream_words(uint32_t seed, uint32_t pop_id, uint32_t op, uint32_t gen,
                      uint32_t index, uint32_t sub, int32_t count, uint32_t *out)
{
    orc_stream s;
    stream_open(&s, seed, pop_id, op, gen, index, sub);
    for (int32_t t = 0; t < count; ++t)
        out[t] = stream_next(&s);
}

/* ------------------------------------------------------------------------ */
/* a1  Initial population (Sec. 3.1; Sec. 6 listing, population set-up and */
/* the column-shuffle kernel).  Every matrix starts all +1 with the upper   */
/* half of columns 2..m set to -1; each of those columns is then shuffled   */
/* by Fisher-Yates.  Column 1 (index 0) stays all +1.                       */
/* Pinned by: column balance, column 0, chi-square uniformity at m = 4.     */
/* ------------------------------------------------------------------------ */
static void init_one(int8_t *Q, int32_t m, uint32_t seed, uint32_t pop_id, uint32_t slot)
{
    int8_t *col = (int8_t *)malloc((size_t)m);
    for (int32_t i = 0; i < m; ++i)
        Q[(size_t)i * m + 0] = 1;
    for (int32_t j = 1; j < m; ++j) {
        for (int32_t i = 0; i < m; ++i)
            col[i] = (i < m / 2) ? (int8_t)-1 : (int8_t)1;
        orc_stream s;
        stream_open(&s, seed, pop_id, ORC_OP_INIT, 0u, slot, (uint32_t)j);
        for (int32_t i1 = 0; i1 < m - 1; ++i1) {
            int32_t i2 = i1 + (int32_t)orc_uniform(stream_next(&s), 0u, (uint32_t)(m - 1 - i1));
            int8_t t = col[i1];
            col[i1] = col[i2];
            col[i2] = t;
        }
        for (int32_t i = 0; i < m; ++i)
            Q[(size_t)i * m + j] = col[i];
    }
    free(col);
}

void orc_init_population(int8_t *pop, int32_t m, int64_t P, uint32_t seed, uint32_t pop_id)
{
    int64_t q;
#pragma omp parallel for schedule(static)
    for (q = 0; q < P; ++q)
        init_one(pop + (size_t)q * m * m, m, seed, pop_id, (uint32_t)q);
}

/* The initial matrices of the listed slots only (matrix t of `out` is slot
 * slots[t]), for checking samples of populations too large to build here. */
void orc_init_slots(int8_t *out, int32_t m, const int64_t *slots, int64_t n, uint32_t seed, uint32_t pop_id)
{
    int64_t t;
#pragma omp parallel for schedule(static)
    for (t = 0; t < n; ++t)
        init_one(out + (size_t)t * m * m, m, seed, pop_id, (uint32_t)slots[t]);
}

/* ------------------------------------------------------------------------ */
/* a2  Column Gram G = Q^T Q (Sec. 3.2) by the triple loop.                 */
/* Pinned by: float64 batched matmul, Sylvester/Paley, m = 4 enumeration.   */
/* ------------------------------------------------------------------------ */
void orc_gram(const int8_t *Q, int32_t m, int32_t *G)
{
    for (int32_t i = 0; i < m; ++i)
        for (int32_t j = 0; j < m; ++j) {
            int32_t acc = 0;
            for (int32_t r = 0; r < m; ++r)
                acc += (int32_t)Q[(size_t)r * m + i] * (int32_t)Q[(size_t)r * m + j];
            G[(size_t)i * m + j] = acc;
        }
}

/* Fitness of one matrix.
 *   ORC_FIT_SQ : sum over i < j of G_ij^2 (sum of squared column inner
 *                products over the strict upper triangle)
 *   ORC_FIT_ABS: F1 = sum over all i, j of |G_ij| - m^2   (Eq. (3) / (8))
 *   ORC_FIT_NNZ: F2 = number of nonzero entries of G - m (Eq. (4) / (9))
 */
static uint64_t fitness_one(const int8_t *Q, int32_t m, int32_t kind, int32_t *G)
{
    orc_gram(Q, m, G);
    if (kind == ORC_FIT_SQ) {
        uint64_t acc = 0;
        for (int32_t i = 0; i < m; ++i)
            for (int32_t j = i + 1; j < m; ++j) {
                int64_t g = G[(size_t)i * m + j];
                acc += (uint64_t)(g * g);
            }
        return acc;
    }
    if (kind == ORC_FIT_ABS) {
        int64_t acc = 0;
        for (int32_t i = 0; i < m; ++i)
            for (int32_t j = 0; j < m; ++j) {
                int64_t g = G[(size_t)i * m + j];
                acc += g < 0 ? -g : g;
            }
        return (uint64_t)(acc - (int64_t)m * m);
    }
    /* ORC_FIT_NNZ */
    int64_t nnz = 0;
    for (int32_t i = 0; i < m; ++i)
        for (int32_t j = 0; j < m; ++j)
            nnz += G[(size_t)i * m + j] != 0;
    return (uint64_t)(nnz - m);
}

void orc_fitness(const int8_t *pop, int32_t m, int64_t first, int64_t count, int32_t kind, uint64_t *F)
{
    int64_t q;
#pragma omp parallel
    {
        int32_t *G = (int32_t *)malloc(sizeof(int32_t) * (size_t)m * m);
#pragma omp for schedule(static)
        for (q = first; q < first + count; ++q)
            F[q] = fitness_one(pop + (size_t)q * m * m, m, kind, G);
        free(G);
    }
}

/* ------------------------------------------------------------------------ */
/* a5  Column-exchange crossover (Sec. 3.4, Fig. 2, Eq. (6)).  With cut c,  */
/* O1 = P1[:, :c] | P2[:, c:]  and  O2 = P2[:, :c] | P1[:, c:].             */
/* Pinned by: the worked 4x4 example of Fig. 2; column conservation.        */
/* ------------------------------------------------------------------------ */
void orc_crossover_pair(const int8_t *P1, const int8_t *P2, int8_t *O1, int8_t *O2, int32_t m, int32_t c)
{
    for (int32_t i = 0; i < m; ++i)
        for (int32_t j = 0; j < m; ++j) {
            size_t e = (size_t)i * m + j;
            if (j < c) {
                O1[e] = P1[e];
                O2[e] = P2[e];
            } else {
                O1[e] = P2[e];
                O2[e] = P1[e];
            }
        }
}

/* Cut point of pair k at generation gen: c in [1, m-1] (the listing's draw
 * range; the prose's 1 < c < m is read as this range). */
int32_t orc_cut_point(int32_t m, uint32_t seed, uint32_t pop_id, uint32_t gen, uint32_t k)
{
    orc_stream s;
    stream_open(&s, seed, pop_id, ORC_OP_CROSS, gen, k, 0u);
    return (int32_t)orc_uniform(stream_next(&s), 1u, (uint32_t)(m - 1));
}

void orc_crossover(int8_t *pop, int32_t m, int64_t N, uint32_t seed, uint32_t pop_id, uint32_t gen)
{
    const size_t S = (size_t)m * m;
    int64_t k;
#pragma omp parallel for schedule(static)
    for (k = 0; k < N; ++k) {
        int32_t c = orc_cut_point(m, seed, pop_id, gen, (uint32_t)k);
        orc_crossover_pair(pop + (size_t)k * S, pop + (size_t)(N + k) * S,
                           pop + (size_t)(2 * N + k) * S, pop + (size_t)(3 * N + k) * S, m, c);
    }
}

/* ------------------------------------------------------------------------ */
/* a6  Balanced pair-flip mutation, method 3 (Sec. 3.5, Eq. (7), Fig. 3).   */
/* For each of NC columns (in order) and each of NR row pairs (in order):   */
/* the two entries are negated only when their signs differ, so every       */
/* column keeps its balance.  The same NR pairs serve every chosen column.  */
/* Pinned by: the four worked 8x8 examples of Fig. 3; balance invariants.   */
/* ------------------------------------------------------------------------ */
int32_t orc_mutate_explicit(int8_t *Q, int32_t m, int32_t NC, int32_t NR, const int32_t *cols,
                            const int32_t *rows1, const int32_t *rows2)
{
    int32_t flips = 0;
    for (int32_t jc = 0; jc < NC; ++jc) {
        int32_t c = cols[jc];
        for (int32_t ir = 0; ir < NR; ++ir) {
            size_t e1 = (size_t)rows1[ir] * m + c;
            size_t e2 = (size_t)rows2[ir] * m + c;
            if (Q[e1] != Q[e2]) {
                Q[e1] = (int8_t)-Q[e1];
                Q[e2] = (int8_t)-Q[e2];
                flips += 1;
            }
        }
    }
    return flips;
}

/* Draws of offspring o at generation gen: NC columns in [1, m-1], then NR
 * first rows and NR second rows in [0, m-1], from one stream. */
void orc_mutation_draws(int32_t m, int32_t NC, int32_t NR, uint32_t seed, uint32_t pop_id,
                        uint32_t gen, uint32_t o, int32_t *cols, int32_t *rows1, int32_t *rows2)
{
    orc_stream s;
    stream_open(&s, seed, pop_id, ORC_OP_MUTATE, gen, o, 0u);
    for (int32_t jc = 0; jc < NC; ++jc)
        cols[jc] = (int32_t)orc_uniform(stream_next(&s), 1u, (uint32_t)(m - 1));
    for (int32_t ir = 0; ir < NR; ++ir)
        rows1[ir] = (int32_t)orc_uniform(stream_next(&s), 0u, (uint32_t)(m - 1));
    for (int32_t ir = 0; ir < NR; ++ir)
        rows2[ir] = (int32_t)orc_uniform(stream_next(&s), 0u, (uint32_t)(m - 1));
}

/* Method 3 of Sec. 3.5 (method 2 is NC = NR = 1): offspring o draws from
 * stream index o.  Method 1 (`shared` set): the same column and row pairs
 * for every offspring of the generation, drawn once from stream index 2N
 * (a stream no single offspring uses).  In both, a pair is flipped only
 * when its two entries differ. */
void orc_mutate(int8_t *pop, int32_t m, int64_t N, int32_t NC, int32_t NR, uint32_t seed,
                uint32_t pop_id, uint32_t gen, int32_t shared)
{
    const size_t S = (size_t)m * m;
    int64_t o;
#pragma omp parallel
    {
        int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * (size_t)NC);
        int32_t *r1 = (int32_t *)malloc(sizeof(int32_t) * (size_t)NR);
        int32_t *r2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)NR);
#pragma omp for schedule(static)
        for (o = 0; o < 2 * N; ++o) {
            orc_mutation_draws(m, NC, NR, seed, pop_id, gen, shared ? (uint32_t)(2 * N) : (uint32_t)o, cols, r1,
                               r2);
            orc_mutate_explicit(pop + (size_t)(2 * N + o) * S, m, NC, NR, cols, r1, r2);
        }
        free(cols);
        free(r1);
        free(r2);
    }
}

/* ------------------------------------------------------------------------ */
/* a4  Random order of the survivors (Sec. 3.3; Sec. 6 listing, the random  */
/* permutation in the selection line).  pi is the permutation that sorts    */
/* the keys (u_d, d), d in [0, n), ascending, where u_d is word (d mod 4)   */
/* of Philox block (SELECT, gen, floor(d / 4), 0): independent uniform keys */
/* give a uniformly random order (ties of u are broken by d).               */
/* Pinned by: argsort of the raw stream words; chi-square uniformity over   */
/* all 3!, 4! and 5! orders.                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint32_t u;
    uint32_t d;
} orc_rkey;

static int rkey_cmp(const void *a, const void *b)
{
    const orc_rkey *x = (const orc_rkey *)a, *y = (const orc_rkey *)b;
    if (x->u != y->u)
        return x->u < y->u ? -1 : 1;
    if (x->d != y->d)
        return x->d < y->d ? -1 : 1;
    return 0;
}

uint32_t orc_select_key(uint32_t seed, uint32_t pop_id, uint32_t gen, uint32_t d)
{
    uint32_t ctr[4] = {ORC_OP_SELECT, gen, d / 4u, 0u};
    uint32_t key[2] = {seed, pop_id};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    return w[d % 4u];
}

void orc_perm(uint32_t n, uint32_t seed, uint32_t pop_id, uint32_t gen, uint32_t *pi)
{
    orc_rkey *k = (orc_rkey *)malloc(sizeof(orc_rkey) * (size_t)(n ? n : 1));
    for (uint32_t d = 0; d < n; ++d) {
        k[d].u = orc_select_key(seed, pop_id, gen, d);
        k[d].d = d;
    }
    qsort(k, (size_t)n, sizeof(orc_rkey), rkey_cmp);
    for (uint32_t p = 0; p < n; ++p)
        pi[p] = k[p].d;
    free(k);
}

/* ------------------------------------------------------------------------ */
/* a3 + a4  Truncation selection (Sec. 3.3; Sec. 6 listing, selection line) */
/* The 2N individuals that come first in ascending (F, slot) order survive. */
/* Listed in increasing slot order s_0 < ... < s_{2N-1}, parent slot p      */
/* receives s_{pi(p)}.  The set is the listing's argsort(F)[:2N]; taking it */
/* in slot order before the uniform permutation pi leaves the distribution  */
/* of the result unchanged.  The right-hand side is read from a copy, as in */
/* the listing.                                                             */
/* Pinned by: brute force on small populations (sort + bijection).          */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t f;
    int64_t slot;
} orc_key;

static int key_cmp(const void *a, const void *b)
{
    const orc_key *x = (const orc_key *)a, *y = (const orc_key *)b;
    if (x->f != y->f)
        return x->f < y->f ? -1 : 1;
    if (x->slot != y->slot)
        return x->slot < y->slot ? -1 : 1;
    return 0;
}

/* Survivors in slot order: writes 2N slot indices into surv. */
void orc_survivors(const uint64_t *F, int64_t N, int64_t *surv)
{
    const int64_t P = 4 * N;
    orc_key *keys = (orc_key *)malloc(sizeof(orc_key) * (size_t)P);
    unsigned char *alive = (unsigned char *)calloc((size_t)P, 1);
    for (int64_t q = 0; q < P; ++q) {
        keys[q].f = F[q];
        keys[q].slot = q;
    }
    qsort(keys, (size_t)P, sizeof(orc_key), key_cmp);
    for (int64_t r = 0; r < 2 * N; ++r)
        alive[keys[r].slot] = 1;
    int64_t d = 0;
    for (int64_t q = 0; q < P; ++q)
        if (alive[q])
            surv[d++] = q;
    free(keys);
    free(alive);
}

void orc_select(int8_t *pop, uint64_t *F, int32_t m, int64_t N, uint32_t seed, uint32_t pop_id, uint32_t gen)
{
    const size_t S = (size_t)m * m;
    const int64_t P = 4 * N;
    int64_t *surv = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * N));
    int8_t *old_pop = (int8_t *)malloc(S * (size_t)P);
    uint64_t *old_F = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)P);
    memcpy(old_pop, pop, S * (size_t)P);
    memcpy(old_F, F, sizeof(uint64_t) * (size_t)P);
    uint32_t *pi = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(2 * N));
    orc_survivors(old_F, N, surv);
    orc_perm((uint32_t)(2 * N), seed, pop_id, gen, pi);
    int64_t p;
#pragma omp parallel for schedule(static)
    for (p = 0; p < 2 * N; ++p) {
        int64_t src = surv[pi[p]];
        memcpy(pop + (size_t)p * S, old_pop + (size_t)src * S, S);
        F[p] = old_F[src];
    }
    free(pi);
    free(surv);
    free(old_pop);
    free(old_F);
}

/* ------------------------------------------------------------------------ */
/* Probabilistic selection (Sec. 3.3: selection with probabilities inverse  */
/* proportional to the fitness values, which the paper names and reports    */
/* as no better than truncation; Sec. 4.1 on stalling).  The paper gives no */
/* formula; the reading implemented here:                                   */
/*   weight      w_q = floor(2^32 / (F_q + 1))   (integer; F = 0 allowed)   */
/*   cumulative  C_q = w_0 + ... + w_q,  W = C_{P-1}  (< 2^63)             */
/*   parent slot p in [0, 2N), independently, with replacement:            */
/*     u = (word 0 << 32) | word 1 of Philox, key (seed, pop_id), counter   */
/*         (PSELECT, g, p, 0);  t = floor(u W / 2^64)  (in [0, W))          */
/*     receives the individual q with C_{q-1} <= t < C_q                   */
/* and its fitness moves with it; the right-hand side is read from a copy.  */
/* Pinned by: chi-square of the selection frequencies against w_q / W on    */
/* tiny populations, the degenerate cases (equal F: uniform; one F = 0 and  */
/* the rest huge: always that one), monotone frequency in F, and every      */
/* parent being a copy of an individual of the previous population.         */
/* ------------------------------------------------------------------------ */
uint64_t orc_psel_weight(uint64_t f)
{
    return ((uint64_t)1 << 32) / (f + 1u);
}

/* The individual drawn for parent slot p (weights from F[0, P)). */
int64_t orc_psel_pick(const uint64_t *C, int64_t P, uint32_t seed, uint32_t pop_id, uint32_t gen, uint32_t p)
{
    uint32_t ctr[4] = {ORC_OP_PSELECT, gen, p, 0u};
    uint32_t key[2] = {seed, pop_id};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    const uint64_t u = ((uint64_t)w[0] << 32) | (uint64_t)w[1];
    const uint64_t W = C[P - 1];
    const uint64_t t = (uint64_t)(((unsigned __int128)u * (unsigned __int128)W) >> 64);
    /* smallest q with C_q > t (binary search over the increasing C) */
    int64_t lo = 0, hi = P - 1;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (C[mid] > t)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

void orc_select_prob(int8_t *pop, uint64_t *F, int32_t m, int64_t N, uint32_t seed, uint32_t pop_id, uint32_t gen)
{
    const size_t S = (size_t)m * m;
    const int64_t P = 4 * N;
    int8_t *old_pop = (int8_t *)malloc(S * (size_t)P);
    uint64_t *old_F = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)P);
    uint64_t *C = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)P);
    memcpy(old_pop, pop, S * (size_t)P);
    memcpy(old_F, F, sizeof(uint64_t) * (size_t)P);
    uint64_t run = 0;
    for (int64_t q = 0; q < P; ++q) {
        run += orc_psel_weight(old_F[q]);
        C[q] = run;
    }
    int64_t p;
#pragma omp parallel for schedule(static)
    for (p = 0; p < 2 * N; ++p) {
        const int64_t src = orc_psel_pick(C, P, seed, pop_id, gen, (uint32_t)p);
        memcpy(pop + (size_t)p * S, old_pop + (size_t)src * S, S);
        F[p] = old_F[src];
    }
    free(C);
    free(old_pop);
    free(old_F);
}

/* ------------------------------------------------------------------------ */
/* a8  Best individual: least F, lowest slot on ties (Sec. 6 listing, the   */
/* minimum of F and the loop test).                                         */
/* ------------------------------------------------------------------------ */
void orc_best(const uint64_t *F, int64_t P, int64_t *slot, uint64_t *fit)
{
    int64_t best = 0;
    for (int64_t q = 1; q < P; ++q)
        if (F[q] < F[best])
            best = q;
    *slot = best;
    *fit = F[best];
}

/* ------------------------------------------------------------------------ */
/* a1..a8  The generation loop (Sec. 3 enumerated steps; Sec. 6 listing):   */
/* selection (truncation, or the probabilistic variant when selection = 1), */
/* crossover, mutation, then fitness of the 2N offspring; the               */
/* parents keep the fitness carried by the selection.  Generation numbers   */
/* run from gen0 + 1; traj receives the best after each generation.        */
/* When stop_at_zero is set the loop ends after the first generation whose  */
/* best fitness is 0.  Returns the number of generations run.              */
/* ------------------------------------------------------------------------ */
int32_t orc_run(int8_t *pop, uint64_t *F, int32_t m, int64_t N, int32_t NC, int32_t NR, int32_t kind,
                uint32_t seed, uint32_t pop_id, uint32_t gen0, int32_t generations, int32_t stop_at_zero,
                uint64_t *traj_fit, int64_t *traj_slot, int32_t shared_mutation, int32_t selection)
{
    int32_t done = 0;
    for (int32_t t = 0; t < generations; ++t) {
        uint32_t gen = gen0 + (uint32_t)t + 1u;
        if (selection == 1)
            orc_select_prob(pop, F, m, N, seed, pop_id, gen);
        else
            orc_select(pop, F, m, N, seed, pop_id, gen);
        orc_crossover(pop, m, N, seed, pop_id, gen);
        orc_mutate(pop, m, N, NC, NR, seed, pop_id, gen, shared_mutation);
        orc_fitness(pop, m, 2 * N, 2 * N, kind, F);
        int64_t bs;
        uint64_t bf;
        orc_best(F, 4 * N, &bs, &bf);
        if (traj_fit)
            traj_fit[t] = bf;
        if (traj_slot)
            traj_slot[t] = bs;
        done = t + 1;
        if (stop_at_zero && bf == 0u)
            break;
    }
    return done;
}

/* Population size of order position idx for the mixed-order workload:
 * N = 500 + U[0, 4500] from Philox (CONFIG, 0, idx, 0) word 0, key (seed, 0). */
int64_t orc_mixed_N(uint32_t seed, uint32_t idx)
{
    orc_stream s;
    stream_open(&s, seed, 0u, ORC_OP_CONFIG, 0u, idx, 0u);
    return 500 + (int64_t)orc_uniform(stream_next(&s), 0u, 4500u);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2, Table 1: batched real Gram F_b = Q_b^T Q_b of B real m x m       */
/* matrices (the NumPy vs CuPy speed comparison; not a step of the GA).     */
/* Triple loop in double precision, summing over the rows r in ascending    */
/* order: G_ij = sum_r Q_ri Q_rj, matrix b at Q[b*m*m + r*m + i].           */
/* Pinned by: Sylvester H^T H = mI, the diagonal, single-entry and rank-one */
/* closed forms, the exact rational Gram within the summation error bound,  */
/* and an orthogonal factor from a QR decomposition.                        */
/* ------------------------------------------------------------------------ */
void orc_gram_real(const double *Q, int32_t m, int64_t B, double *G)
{
    int64_t b;
#pragma omp parallel for schedule(static)
    for (b = 0; b < B; ++b) {
        const double *q = Q + (size_t)b * m * m;
        double *g = G + (size_t)b * m * m;
        for (int32_t i = 0; i < m; ++i)
            for (int32_t j = 0; j < m; ++j) {
                double acc = 0.0;
                for (int32_t r = 0; r < m; ++r)
                    acc += q[(size_t)r * m + i] * q[(size_t)r * m + j];
                g[(size_t)i * m + j] = acc;
            }
    }
}

int32_t orc_num_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int32_t n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
}
