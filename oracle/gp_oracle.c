/*
 * CPU oracle for GP fitness evaluation and subtree crossover.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file: only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg and reference arm (--impl reference) may use it.  It shares no code, header or table with the
 * CUDA library.
 *
 * What it follows (Langdon & Banzhaf, "Faster Genetic Programming GPquick via
 * multicore and Advanced Vector Extensions", 2019):
 *   - Sec. 2.2: the traditional recursive EVAL.  Each call reads the opcode at
 *     the instruction pointer and advances it; x and constants return at
 *     once; ADD, SUB, MUL, DIV call EVAL twice (first argument, then second)
 *     and combine.  Here each call returns all fitness cases at once (the
 *     single-pass variant of Sec. 2.2), computed with plain scalar loops.
 *   - Table gp.details: function set MUL ADD DIV SUB; DIV is protected,
 *     (y != 0) ? x / y : 1.0f, where x, y are DIV's first and second argument.
 *   - Table gp.details / Sec. 3.2: fitness = (1/48) sum |GP(x_i) - y_i|,
 *     accumulated by a plain for loop in case order (Sec. 2.2, last para.).
 *   - Sec. 3.2: a hit is a case with |error| within 0.01.
 *   - Sec. 3.1: one child per crossover: mum with the subtree at the mum
 *     point replaced by dad's subtree at the dad point.
 *   - Table gp.details / Sec. 3.2: generational, non-elitist; both parents
 *     of every child chosen by tournaments of size 7 on fitness (lower is
 *     better); both crossover points uniform over all nodes of the parent
 *     (Sec. 3.1), chosen in a fixed sequential order (Sec. 3.1, last para.).
 *     The random numbers are a counter-based stream (SplitMix64 of Steele,
 *     Lea & Flood 2014 indexed by a counter), bounded by Lemire's
 *     multiply-shift with rejection (ACM TOMACS 2019), so any draw can be
 *     recomputed from (seed, generation, child, purpose, index).
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math (no contraction of a*b+c,
 * IEEE binary32/binary64 round-to-nearest, subnormals kept).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2
#define OR_EMALFORMED 3
#define OR_MAX_CASES 64

enum { ADD = 0, SUB = 1, MUL = 2, DIV = 3, XVAR = 4, CONST0 = 5 };

/* ------------------------------------------------------------------ */
/* Recursive EVAL, binary32                                             */
/* ------------------------------------------------------------------ */

typedef struct {
    const uint8_t *t;
    uint64_t n;
    uint64_t pc;
    const float *x;
    const float *c;
    uint32_t nc;      /* number of constants */
    uint32_t ncases;
    float div0;
    int err;
} ctx32;

static void eval32(ctx32 *s, float *out)
{
    if (s->err) return;
    if (s->pc >= s->n) { s->err = OR_EMALFORMED; return; }
    uint8_t op = s->t[s->pc++];
    uint32_t i;
    if (op == XVAR) {
        for (i = 0; i < s->ncases; i++) out[i] = s->x[i];
        return;
    }
    if (op >= CONST0) {
        if ((uint32_t)(op - CONST0) >= s->nc) { s->err = OR_EMALFORMED; return; }
        float v = s->c[op - CONST0];
        for (i = 0; i < s->ncases; i++) out[i] = v;
        return;
    }
    float a[OR_MAX_CASES], b[OR_MAX_CASES];
    eval32(s, a);            /* first argument  */
    eval32(s, b);            /* second argument */
    if (s->err) return;
    switch (op) {
    case ADD: for (i = 0; i < s->ncases; i++) out[i] = a[i] + b[i]; break;
    case SUB: for (i = 0; i < s->ncases; i++) out[i] = a[i] - b[i]; break;
    case MUL: for (i = 0; i < s->ncases; i++) out[i] = a[i] * b[i]; break;
    default:  for (i = 0; i < s->ncases; i++) out[i] = (b[i] != 0.0f) ? a[i] / b[i] : s->div0; break;
    }
}

/* ------------------------------------------------------------------ */
/* Recursive EVAL, binary64 (tables widened from the same FP32 inputs) */
/* ------------------------------------------------------------------ */

typedef struct {
    const uint8_t *t;
    uint64_t n;
    uint64_t pc;
    const double *x;
    const double *c;
    uint32_t nc;
    uint32_t ncases;
    double div0;
    int err;
} ctx64;

static void eval64(ctx64 *s, double *out)
{
    if (s->err) return;
    if (s->pc >= s->n) { s->err = OR_EMALFORMED; return; }
    uint8_t op = s->t[s->pc++];
    uint32_t i;
    if (op == XVAR) {
        for (i = 0; i < s->ncases; i++) out[i] = s->x[i];
        return;
    }
    if (op >= CONST0) {
        if ((uint32_t)(op - CONST0) >= s->nc) { s->err = OR_EMALFORMED; return; }
        double v = s->c[op - CONST0];
        for (i = 0; i < s->ncases; i++) out[i] = v;
        return;
    }
    double a[OR_MAX_CASES], b[OR_MAX_CASES];
    eval64(s, a);
    eval64(s, b);
    if (s->err) return;
    switch (op) {
    case ADD: for (i = 0; i < s->ncases; i++) out[i] = a[i] + b[i]; break;
    case SUB: for (i = 0; i < s->ncases; i++) out[i] = a[i] - b[i]; break;
    case MUL: for (i = 0; i < s->ncases; i++) out[i] = a[i] * b[i]; break;
    default:  for (i = 0; i < s->ncases; i++) out[i] = (b[i] != 0.0) ? a[i] / b[i] : s->div0; break;
    }
}

/* ------------------------------------------------------------------ */
/* Tree structure helpers (prefix order, arity 2 for codes 0..3)        */
/* ------------------------------------------------------------------ */

/* Depth of the tree (root = 1) by an explicit walk; 0 if malformed. */
uint64_t oracle_tree_depth(const uint8_t *t, uint64_t n)
{
    /* pending[d] = children still to read at depth d */
    uint64_t cap = 1024, top = 0, best = 0, k;
    uint8_t *pending = (uint8_t *)malloc(cap);
    if (!pending) return 0;
    for (k = 0; k < n; k++) {
        if (k > 0) {
            while (top > 0 && pending[top - 1] == 0) top--;
            if (top == 0) { free(pending); return 0; }   /* extra nodes */
            pending[top - 1]--;
        }
        if (top + 1 > best) best = top + 1;
        if (t[k] < XVAR) {
            if (top == cap) {
                uint8_t *p2 = (uint8_t *)realloc(pending, cap * 2);
                if (!p2) { free(pending); return 0; }
                pending = p2; cap *= 2;
            }
            pending[top++] = 2;
        }
    }
    while (top > 0 && pending[top - 1] == 0) top--;
    free(pending);
    return top == 0 ? best : 0;
}

/* 1 if t is exactly one prefix tree over codes < 5 + n_consts, else 0. */
int oracle_check_tree(const uint8_t *t, uint64_t n, uint32_t n_consts)
{
    int64_t need = 1;            /* subtrees still to read */
    uint64_t k;
    if (n == 0) return 0;
    for (k = 0; k < n; k++) {
        if (need <= 0) return 0;
        if (t[k] >= CONST0 + n_consts) return 0;
        need += (t[k] < XVAR) ? 1 : -1;
    }
    return need == 0;
}

/* End (exclusive) of the subtree rooted at i: walk forward counting the
 * subtrees still to be read until none remain. */
int oracle_subtree_end(const uint8_t *t, uint64_t n, uint64_t i, uint64_t *end)
{
    int64_t need = 1;
    uint64_t k = i;
    if (i >= n) return OR_EINVAL;
    while (need > 0) {
        if (k >= n) return OR_EMALFORMED;
        need += (t[k] < XVAR) ? 1 : -1;
        k++;
    }
    *end = k;
    return OR_OK;
}

/* Sec. 3.1: child = mum[0,i) ++ dad[j, end_d) ++ mum[end_m, n_m). */
int oracle_crossover(const uint8_t *mum, uint64_t n_m, const uint8_t *dad, uint64_t n_d,
                     uint64_t i, uint64_t j, uint8_t *child, uint64_t cap, uint64_t *n_child)
{
    uint64_t em, ed, len;
    int st = oracle_subtree_end(mum, n_m, i, &em);
    if (st) return st;
    st = oracle_subtree_end(dad, n_d, j, &ed);
    if (st) return st;
    len = i + (ed - j) + (n_m - em);
    *n_child = len;
    if (child == NULL) return OR_OK;          /* size query */
    if (len > cap) return OR_ENOMEM;
    memcpy(child, mum, i);
    memcpy(child + i, dad + j, ed - j);
    memcpy(child + i + (ed - j), mum + em, n_m - em);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Fitness (Table gp.details): plain loop in case order                 */
/* ------------------------------------------------------------------ */

float oracle_mae_f32(const float *out, const float *y, uint32_t n_cases, uint32_t *hits)
{
    float s = 0.0f;
    uint32_t h = 0, i;
    for (i = 0; i < n_cases; i++) {
        float e = fabsf(out[i] - y[i]);
        s = s + e;
        if (e < 0.01f) h++;
    }
    if (hits) *hits = h;
    return s / (float)n_cases;
}

double oracle_mae_f64(const double *out, const double *y, uint32_t n_cases)
{
    double s = 0.0;
    uint32_t i;
    for (i = 0; i < n_cases; i++) s = s + fabs(out[i] - y[i]);
    return s / (double)n_cases;
}

/* ------------------------------------------------------------------ */
/* Evaluation entry points.  Recursion depth equals tree depth, so each */
/* evaluation runs on a thread whose stack is sized from that depth.    */
/* ------------------------------------------------------------------ */

typedef struct {
    const uint8_t *t; uint64_t n;
    const float *x; uint32_t ncases;
    const float *c; uint32_t nc; float div0;
    float *out32; double *out64;
    int st;
} job_t;

/* Generous bound on the recursion's stack use: two case arrays per frame
 * plus call overhead, doubled. */
static size_t stack_bytes_for(uint64_t depth, int wide)
{
    size_t frame = (size_t)2 * OR_MAX_CASES * (wide ? 8 : 4) + 256;
    return (size_t)(depth + 64) * frame * 2;
}

static void run_job(job_t *j)
{
    if (j->out32) {
        ctx32 s = { j->t, j->n, 0, j->x, j->c, j->nc, j->ncases, j->div0, 0 };
        eval32(&s, j->out32);
        j->st = s.err ? s.err : (s.pc == j->n ? OR_OK : OR_EMALFORMED);
    } else {
        double xd[OR_MAX_CASES];
        double *cd = (double *)malloc(sizeof(double) * (j->nc ? j->nc : 1));
        uint32_t i;
        if (!cd) { j->st = OR_ENOMEM; return; }
        for (i = 0; i < j->ncases; i++) xd[i] = (double)j->x[i];
        for (i = 0; i < j->nc; i++) cd[i] = (double)j->c[i];
        ctx64 s = { j->t, j->n, 0, xd, cd, j->nc, j->ncases, (double)j->div0, 0 };
        eval64(&s, j->out64);
        j->st = s.err ? s.err : (s.pc == j->n ? OR_OK : OR_EMALFORMED);
        free(cd);
    }
}

static void *job_thread(void *p) { run_job((job_t *)p); return NULL; }

static int run_on_big_stack(job_t *j, uint64_t depth)
{
    pthread_attr_t a;
    pthread_t th;
    size_t sz = stack_bytes_for(depth, j->out64 != NULL);
    if (sz < ((size_t)2 << 20)) { run_job(j); return j->st; }   /* fits the caller's stack */
    sz += (size_t)8 << 20;
    if (pthread_attr_init(&a)) return OR_ENOMEM;
    if (pthread_attr_setstacksize(&a, sz)) { pthread_attr_destroy(&a); return OR_ENOMEM; }
    if (pthread_create(&th, &a, job_thread, j)) { pthread_attr_destroy(&a); return OR_ENOMEM; }
    pthread_join(th, NULL);
    pthread_attr_destroy(&a);
    return j->st;
}

static int eval_tree(const uint8_t *t, uint64_t n, const float *x, uint32_t ncases,
                     const float *c, uint32_t nc, float div0, float *o32, double *o64)
{
    uint64_t depth;
    if (ncases == 0 || ncases > OR_MAX_CASES) return OR_EINVAL;
    if (!oracle_check_tree(t, n, nc)) return OR_EMALFORMED;
    depth = oracle_tree_depth(t, n);
    job_t j = { t, n, x, ncases, c, nc, div0, o32, o64, 0 };
    return run_on_big_stack(&j, depth);
}

int oracle_eval_tree_f32(const uint8_t *t, uint64_t n, const float *x, uint32_t ncases,
                         const float *c, uint32_t nc, float div0, float *out)
{
    return eval_tree(t, n, x, ncases, c, nc, div0, out, NULL);
}

int oracle_eval_tree_f64(const uint8_t *t, uint64_t n, const float *x, uint32_t ncases,
                         const float *c, uint32_t nc, float div0, double *out)
{
    return eval_tree(t, n, x, ncases, c, nc, div0, NULL, out);
}

/* ------------------------------------------------------------------ */
/* Population: trees handed out dynamically to worker threads, as the  */
/* paper's pthreads dispatcher does (Sec. 2.3); results do not depend  */
/* on which thread evaluates which tree.                                */
/* ------------------------------------------------------------------ */

typedef struct {
    const uint8_t *nodes; const uint64_t *offs; uint32_t ntrees;
    const float *x; const float *y; uint32_t ncases;
    const float *c; uint32_t nc; float div0;
    float *out; float *fit; uint32_t *hits;
    double *out64; double *fit64;
    uint32_t next; int st;
    pthread_mutex_t mu;
} pop_t;

static void *pop_worker(void *p)
{
    pop_t *P = (pop_t *)p;
    float o32[OR_MAX_CASES];
    double o64[OR_MAX_CASES], y64[OR_MAX_CASES];
    uint32_t i;
    for (i = 0; i < P->ncases; i++) y64[i] = (double)P->y[i];
    for (;;) {
        uint32_t t;
        pthread_mutex_lock(&P->mu);
        t = P->next++;
        pthread_mutex_unlock(&P->mu);
        if (t >= P->ntrees) break;
        const uint8_t *tree = P->nodes + P->offs[t];
        uint64_t n = P->offs[t + 1] - P->offs[t];
        int st;
        if (P->out || P->fit) {
            st = eval_tree(tree, n, P->x, P->ncases, P->c, P->nc, P->div0, o32, NULL);
            if (st) { pthread_mutex_lock(&P->mu); if (!P->st) P->st = st; pthread_mutex_unlock(&P->mu); continue; }
            if (P->out) memcpy(P->out + (size_t)t * P->ncases, o32, sizeof(float) * P->ncases);
            if (P->fit) P->fit[t] = oracle_mae_f32(o32, P->y, P->ncases, P->hits ? &P->hits[t] : NULL);
        }
        if (P->out64 || P->fit64) {
            st = eval_tree(tree, n, P->x, P->ncases, P->c, P->nc, P->div0, NULL, o64);
            if (st) { pthread_mutex_lock(&P->mu); if (!P->st) P->st = st; pthread_mutex_unlock(&P->mu); continue; }
            if (P->out64) memcpy(P->out64 + (size_t)t * P->ncases, o64, sizeof(double) * P->ncases);
            if (P->fit64) P->fit64[t] = oracle_mae_f64(o64, y64, P->ncases);
        }
    }
    return NULL;
}

int oracle_eval_population(const uint8_t *nodes, const uint64_t *offs, uint32_t ntrees,
                           const float *x, const float *y, uint32_t ncases,
                           const float *c, uint32_t nc, float div0,
                           float *out, float *fit, uint32_t *hits,
                           double *out64, double *fit64, int n_threads)
{
    pop_t P;
    pthread_t th[512];
    int k, started = 0;
    if (ncases == 0 || ncases > OR_MAX_CASES) return OR_EINVAL;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 512) n_threads = 512;
    memset(&P, 0, sizeof(P));
    P.nodes = nodes; P.offs = offs; P.ntrees = ntrees;
    P.x = x; P.y = y; P.ncases = ncases; P.c = c; P.nc = nc; P.div0 = div0;
    P.out = out; P.fit = fit; P.hits = hits; P.out64 = out64; P.fit64 = fit64;
    pthread_mutex_init(&P.mu, NULL);
    if (n_threads == 1) {
        pop_worker(&P);
    } else {
        for (k = 0; k < n_threads; k++)
            if (pthread_create(&th[k], NULL, pop_worker, &P) == 0) started++;
        for (k = 0; k < started; k++) pthread_join(th[k], NULL);
        if (started == 0) pop_worker(&P);
    }
    pthread_mutex_destroy(&P.mu);
    return P.st;
}

/* ---- Generation: tournament selection and crossover points ------------- */
/*
 * Output i (i = 0, 1, ...) of the SplitMix64 generator seeded with `seed`:
 * the state after i + 1 steps of the Weyl sequence, passed through the
 * generator's mixing function.
 */
uint64_t oracle_sm64_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/*
 * Counter of one draw: generation g (< 2^24), child c (< 2^28), purpose p
 * (0 mum tournament, 1 dad tournament, 2 mum point, 3 dad point), index k
 * within the purpose (< 32: tournament entrant) and attempt a (< 16).
 */
static uint64_t draw_counter(uint64_t g, uint64_t c, uint64_t p, uint64_t k, uint64_t a)
{
    return (g << 40) | (c << 12) | (p << 9) | (k << 4) | a;
}

/*
 * Uniform integer in [0, n), n >= 1: the high word of r * n for the first
 * attempt whose low word is at least 2^64 mod n (Lemire 2019); the attempts
 * use counters base, base + 1, ... (at most 16; the last one is taken if
 * all 16 were rejected, which has probability below 2^-16 even for the
 * worst n).
 */
uint64_t oracle_bounded(uint64_t seed, uint64_t base, uint64_t n)
{
    const uint64_t t = (0 - n) % n;
    unsigned __int128 m = 0;
    int a;
    for (a = 0; a < 16; a++) {
        m = (unsigned __int128)oracle_sm64_at(seed, base + (uint64_t)a) * n;
        if ((uint64_t)m >= t) break;
    }
    return (uint64_t)(m >> 64);
}

/*
 * Tournament: `size` entrants drawn uniformly with replacement from the
 * population; the one with the lowest fitness wins, NaN counting as worst
 * and ties going to the entrant drawn first.
 */
uint32_t oracle_tournament(const float *fitness, uint32_t n_pop, uint64_t seed, uint64_t g,
                           uint64_t c, uint32_t purpose, uint32_t size)
{
    uint32_t best = 0, k;
    float best_f = 0.0f;
    for (k = 0; k < size; k++) {
        const uint32_t e = (uint32_t)oracle_bounded(seed, draw_counter(g, c, purpose, k, 0), n_pop);
        const float f = isnan(fitness[e]) ? INFINITY : fitness[e];
        if (k == 0 || f < best_f) {
            best = e;
            best_f = f;
        }
    }
    return best;
}

/*
 * The crossover records of one generation: for child c = 0 .. n_children-1,
 * in order, mum and dad by tournament on the parents' fitness, then the mum
 * point and the dad point, each uniform over the chosen parent's nodes.
 */
int oracle_generation(const float *fitness, const uint64_t *sizes, uint32_t n_pop,
                      uint32_t n_children, uint64_t seed, uint64_t g, uint32_t tsize,
                      uint32_t *mum, uint32_t *dad, uint64_t *mum_point, uint64_t *dad_point)
{
    uint32_t c;
    if (n_pop == 0 || tsize == 0 || tsize > 32 || g >= (1ull << 24) || n_children > (1u << 28))
        return OR_EINVAL;
    for (c = 0; c < n_children; c++) {
        mum[c] = oracle_tournament(fitness, n_pop, seed, g, c, 0, tsize);
        dad[c] = oracle_tournament(fitness, n_pop, seed, g, c, 1, tsize);
        mum_point[c] = oracle_bounded(seed, draw_counter(g, c, 2, 0, 0), sizes[mum[c]]);
        dad_point[c] = oracle_bounded(seed, draw_counter(g, c, 3, 0, 0), sizes[dad[c]]);
    }
    return OR_OK;
}
