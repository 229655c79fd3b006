/*
 * ORACLE — test infrastructure only. Plain, slow, obviously correct CPU
 * evaluation of SPARQL basic graph patterns. Only the tests, the smoke entry
 * point and the benchmark's CPU-baseline leg may load this library; the
 * engine never does. It shares no code with the CUDA engine.
 *
 * What it computes (the plain definition the method reaches exactly):
 * the triples T are a set of (s, p, o) with vertex ids s, o and 1-based
 * predicate ids p (Sec. 6.2.1 step 2). A basic graph pattern Q is a list of
 * triple patterns (Sec. 2.2.1) whose subject / object is a constant vertex
 * or a variable and whose predicate is a constant; its meaning is the
 * conjunction of its triple patterns (Sec. 2.2.3):
 *
 *     R(Q) = { mu : Var(Q) -> V | for all (s,p,o) in Q: (mu(s), p, mu(o)) in T }
 *
 * (mu is the identity on constants; two variables may take the same vertex.)
 * Rows are emitted as int32 tuples in variable order 0..k-1 and sorted
 * lexicographically.
 *
 * Also here, for the per-step checks of the engine:
 *   - the predicate-selection vectors y = A (x) u_p (Eq. 4) and
 *     y = A^T (x) u_p (Eq. 5): y(i) = 1 when row / column i of the RDF
 *     matrix holds predicate p;
 *   - the row-sorted and column-sorted triple lists (the content of a
 *     CSR / CSC RDF matrix whose entries are predicate labels, Sec. 6.2).
 *
 * Algorithm (index nested-loop join by backtracking):
 *   1. Deduplicate T, then keep three sorted copies: by (s,p,o), by (o,p,s)
 *      and by (p,s,o).
 *   2. Join order, by this oracle's own rule: repeatedly take the remaining
 *      pattern with the most bound ends (a constant, or a variable bound by
 *      an earlier pattern), ties to the fewest triples with its predicate,
 *      then to the lowest pattern index.
 *   3. Backtrack over the order: both ends bound -> membership test; one end
 *      bound -> range of the (s,p) or (o,p) sorted copy; none bound -> range
 *      of the predicate's triples. A repeated variable must take one value.
 *   4. Emit mu after the last pattern; sort the rows; check there are no
 *      duplicates (there cannot be any under these semantics).
 * With threads > 1 the candidates of the first pattern are split among
 * OpenMP threads, each with its own output buffer.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { uint32_t a, b, c; } tri;   /* sorted lexicographically by (a, b, c) */

typedef struct {
    uint64_t n;
    uint32_t n_vertices, n_preds;
    tri* spo;          /* (s, p, o) */
    tri* ops;          /* (o, p, s) */
    tri* pso;          /* (p, s, o) */
    uint64_t* pcount;  /* triples per predicate, index 0..n_preds */
} orc_index;

static int cmp_tri(const void* x, const void* y) {
    const tri* u = (const tri*)x; const tri* v = (const tri*)y;
    if (u->a != v->a) return u->a < v->a ? -1 : 1;
    if (u->b != v->b) return u->b < v->b ? -1 : 1;
    if (u->c != v->c) return u->c < v->c ? -1 : 1;
    return 0;
}

void orc_index_free(orc_index* ix) {
    if (!ix) return;
    free(ix->spo); free(ix->ops); free(ix->pso); free(ix->pcount); free(ix);
}

/* Sort t[0..n) by (a, b, c) when its entries are already grouped by a in
 * the buckets off[0..n_keys]: each bucket is sorted on its own (in
 * parallel; buckets are independent). */
static void sort_buckets(tri* t, const uint64_t* off, uint64_t n_keys) {
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t k = 0; k < (int64_t)n_keys; ++k)
        if (off[k + 1] - off[k] > 1) qsort(t + off[k], off[k + 1] - off[k], sizeof(tri), cmp_tri);
}

/* Bucket offsets of n entries by key key(i) < n_keys (a counting pass). */
static uint64_t* bucket_offsets(uint64_t n_keys, uint64_t n, const uint32_t* key, uint64_t stride) {
    uint64_t* off = (uint64_t*)calloc(n_keys + 1, sizeof(uint64_t));
    if (!off) return NULL;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        #pragma omp atomic
        off[key[(uint64_t)i * stride] + 1]++;
    }
    for (uint64_t k = 0; k < n_keys; ++k) off[k + 1] += off[k];
    return off;
}

/* Build the index. Returns NULL on a bad triple (vertex >= n_vertices or
 * predicate not in 1..n_preds) or when memory runs out. Each sorted copy is
 * made by grouping the triples by their first field (a counting sort) and
 * sorting every group by the other two; the (p, s, o) copy is a stable
 * grouping of the (s, p, o) one by p, which keeps (s, o) order inside each
 * group. */
orc_index* orc_index_build(const uint32_t* s, const uint32_t* p, const uint32_t* o, uint64_t n,
                           uint32_t n_vertices, uint32_t n_preds) {
    for (uint64_t i = 0; i < n; ++i)
        if (s[i] >= n_vertices || o[i] >= n_vertices || p[i] < 1 || p[i] > n_preds) return NULL;
    orc_index* ix = (orc_index*)calloc(1, sizeof(orc_index));
    if (!ix) return NULL;
    ix->n_vertices = n_vertices; ix->n_preds = n_preds;
    uint64_t cap = n ? n : 1;
    ix->spo = (tri*)malloc(sizeof(tri) * cap);
    ix->pcount = (uint64_t*)calloc((size_t)n_preds + 1, sizeof(uint64_t));
    uint64_t* off = bucket_offsets(n_vertices, n, s, 1);
    const uint64_t n_cur = (n_vertices > n_preds ? n_vertices : n_preds) + 1ull;
    uint64_t* cur = (uint64_t*)malloc(sizeof(uint64_t) * n_cur);
    if (!ix->spo || !ix->pcount || !off || !cur) { free(off); free(cur); orc_index_free(ix); return NULL; }
    memcpy(cur, off, sizeof(uint64_t) * n_vertices);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        uint64_t at;
        #pragma omp atomic capture
        at = cur[s[i]]++;
        ix->spo[at].a = s[i]; ix->spo[at].b = p[i]; ix->spo[at].c = o[i];
    }
    sort_buckets(ix->spo, off, n_vertices);
    uint64_t m = 0;
    for (uint64_t i = 0; i < n; ++i)
        if (m == 0 || cmp_tri(&ix->spo[m - 1], &ix->spo[i]) != 0) ix->spo[m++] = ix->spo[i];
    ix->n = m;
    free(off);
    cap = m ? m : 1;
    ix->ops = (tri*)malloc(sizeof(tri) * cap);
    ix->pso = (tri*)malloc(sizeof(tri) * cap);
    off = bucket_offsets(n_vertices, m, &ix->spo[0].c, 3);
    if (!ix->ops || !ix->pso || !off) { free(off); free(cur); orc_index_free(ix); return NULL; }
    memcpy(cur, off, sizeof(uint64_t) * n_vertices);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)m; ++i) {
        tri t = ix->spo[i];
        uint64_t at;
        #pragma omp atomic capture
        at = cur[t.c]++;
        ix->ops[at].a = t.c; ix->ops[at].b = t.b; ix->ops[at].c = t.a;
    }
    sort_buckets(ix->ops, off, n_vertices);
    free(off);
    for (uint64_t i = 0; i < m; ++i) ix->pcount[ix->spo[i].b]++;
    uint64_t acc = 0;
    for (uint32_t q = 0; q <= n_preds; ++q) { cur[q] = acc; acc += ix->pcount[q]; }
    for (uint64_t i = 0; i < m; ++i) {   /* stable: (s, o) order stays inside each p */
        tri t = ix->spo[i];
        uint64_t at = cur[t.b]++;
        ix->pso[at].a = t.b; ix->pso[at].b = t.a; ix->pso[at].c = t.c;
    }
    free(cur);
    return ix;
}

uint64_t orc_index_size(const orc_index* ix) { return ix->n; }

/* Copy the deduplicated triples out, sorted by (s,p,o) when by_object == 0
 * (the row order of a CSR RDF matrix) or by (o,p,s) when by_object == 1
 * (the column order of a CSC one). Arrays hold orc_index_size() entries. */
void orc_index_triples(const orc_index* ix, int by_object, uint32_t* s, uint32_t* p, uint32_t* o) {
    const tri* t = by_object ? ix->ops : ix->spo;
    for (uint64_t i = 0; i < ix->n; ++i) {
        if (by_object) { o[i] = t[i].a; p[i] = t[i].b; s[i] = t[i].c; }
        else { s[i] = t[i].a; p[i] = t[i].b; o[i] = t[i].c; }
    }
}

/* Eq. 4 (dir 0) / Eq. 5 (dir 1): out[i] = 1 when row i (column i) of the
 * RDF matrix holds predicate pred, else 0. out has n_vertices bytes. */
void orc_presence(const orc_index* ix, int dir, uint32_t pred, uint8_t* out) {
    memset(out, 0, ix->n_vertices);
    for (uint64_t i = 0; i < ix->n; ++i) {
        const tri* t = &ix->spo[i];
        if (t->b == pred) out[dir ? t->c : t->a] = 1;
    }
}

/* first index in [lo, hi) whose key is >= (a, b, c) */
static uint64_t lower(const tri* t, uint64_t lo, uint64_t hi, uint32_t a, uint32_t b, uint32_t c) {
    tri key = {a, b, c};
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (cmp_tri(&t[mid], &key) < 0) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* [begin, end) of the entries whose first two fields are (a, b) */
static void range2(const tri* t, uint64_t n, uint32_t a, uint32_t b, uint64_t* begin, uint64_t* end) {
    *begin = lower(t, 0, n, a, b, 0);
    *end = (b == UINT32_MAX) ? lower(t, 0, n, a + 1, 0, 0) : lower(t, 0, n, a, b + 1, 0);
}

static void range1(const tri* t, uint64_t n, uint32_t a, uint64_t* begin, uint64_t* end) {
    *begin = lower(t, 0, n, a, 0, 0);
    *end = lower(t, 0, n, a + 1, 0, 0);
}

static int member(const orc_index* ix, uint32_t s, uint32_t p, uint32_t o) {
    uint64_t i = lower(ix->spo, 0, ix->n, s, p, o);
    return i < ix->n && ix->spo[i].a == s && ix->spo[i].b == p && ix->spo[i].c == o;
}

/* ------------------------------------------------------------------ */

#define MAXPAT 64
#define MAXVAR 64

typedef struct {
    int64_t s, p, o;   /* as given: >= 0 constant, < 0 variable -(k+1) */
} pat_t;

typedef struct {
    int32_t* rows;
    uint64_t n, cap;
    uint32_t k;
    int oom;
    int count_only;          /* count the rows, store none */
    uint64_t steps, max_steps;   /* join calls made; give up past max_steps (0: no limit) */
    int stop;
} rowbuf;

static void emit(rowbuf* rb, const int64_t* mu) {
    if (rb->count_only) { rb->n++; return; }
    if (rb->oom) return;
    if (rb->n == rb->cap) {
        uint64_t nc = rb->cap ? rb->cap * 2 : 1024;
        int32_t* r = (int32_t*)realloc(rb->rows, sizeof(int32_t) * nc * (rb->k ? rb->k : 1));
        if (!r) { rb->oom = 1; return; }
        rb->rows = r; rb->cap = nc;
    }
    for (uint32_t v = 0; v < rb->k; ++v) rb->rows[rb->n * rb->k + v] = (int32_t)mu[v];
    rb->n++;
}

typedef struct {
    const orc_index* ix;
    const pat_t* order;
    uint32_t n_pat;
} join_t;

static int var_of(int64_t x) { return x < 0 ? (int)(-x - 1) : -1; }

static void join(const join_t* J, uint32_t d, int64_t* mu, rowbuf* rb) {
    if (rb->stop) return;
    if (rb->max_steps && ++rb->steps > rb->max_steps) { rb->stop = 1; return; }
    if (d == J->n_pat) { emit(rb, mu); return; }
    const pat_t* q = &J->order[d];
    const orc_index* ix = J->ix;
    int vs = var_of(q->s), vo = var_of(q->o);
    uint32_t p = (uint32_t)q->p;
    int sb = vs < 0 || mu[vs] >= 0;
    int ob = vo < 0 || mu[vo] >= 0;
    int64_t sval = vs < 0 ? q->s : mu[vs];
    int64_t oval = vo < 0 ? q->o : mu[vo];
    uint64_t b, e;
    if (sb && ob) {
        if (member(ix, (uint32_t)sval, p, (uint32_t)oval)) join(J, d + 1, mu, rb);
    } else if (sb) {
        range2(ix->spo, ix->n, (uint32_t)sval, p, &b, &e);
        for (uint64_t i = b; i < e; ++i) { mu[vo] = ix->spo[i].c; join(J, d + 1, mu, rb); }
        mu[vo] = -1;
    } else if (ob) {
        range2(ix->ops, ix->n, (uint32_t)oval, p, &b, &e);
        for (uint64_t i = b; i < e; ++i) { mu[vs] = ix->ops[i].c; join(J, d + 1, mu, rb); }
        mu[vs] = -1;
    } else {
        range1(ix->pso, ix->n, p, &b, &e);
        for (uint64_t i = b; i < e; ++i) {
            if (vs == vo) {
                if (ix->pso[i].b != ix->pso[i].c) continue;
                mu[vs] = ix->pso[i].b;
            } else { mu[vs] = ix->pso[i].b; mu[vo] = ix->pso[i].c; }
            join(J, d + 1, mu, rb);
        }
        mu[vs] = -1; mu[vo] = -1;
    }
}

static uint32_t cmp_k;
static int cmp_row(const void* x, const void* y) {
    const int32_t* u = (const int32_t*)x; const int32_t* v = (const int32_t*)y;
    for (uint32_t i = 0; i < cmp_k; ++i) if (u[i] != v[i]) return u[i] < v[i] ? -1 : 1;
    return 0;
}

/* Checks the query and orders its patterns (step 2). Returns the number of
 * variables, or -1 for a bad query. */
static int prepare(const orc_index* ix, const int64_t* patterns, uint32_t n_pat, pat_t* order) {
    if (n_pat == 0 || n_pat > MAXPAT) return -1;
    int used[MAXVAR] = {0};
    int k = 0;
    pat_t pats[MAXPAT];
    for (uint32_t i = 0; i < n_pat; ++i) {
        pats[i].s = patterns[3 * i]; pats[i].p = patterns[3 * i + 1]; pats[i].o = patterns[3 * i + 2];
        if (pats[i].p < 1 || pats[i].p > (int64_t)ix->n_preds) return -1;
        int64_t ends[2] = {pats[i].s, pats[i].o};
        for (int j = 0; j < 2; ++j) {
            if (ends[j] >= 0) { if (ends[j] >= (int64_t)ix->n_vertices) return -1; }
            else {
                int v = var_of(ends[j]);
                if (v >= MAXVAR) return -1;
                used[v] = 1;
                if (v + 1 > k) k = v + 1;
            }
        }
    }
    if (k == 0) return -1;
    for (int v = 0; v < k; ++v) if (!used[v]) return -1;

    /* join order (step 2) */
    int taken[MAXPAT] = {0}, bound[MAXVAR] = {0};
    for (uint32_t d = 0; d < n_pat; ++d) {
        int best = -1, best_b = -1; uint64_t best_c = 0;
        for (uint32_t i = 0; i < n_pat; ++i) {
            if (taken[i]) continue;
            int vs = var_of(pats[i].s), vo = var_of(pats[i].o);
            int nb = (vs < 0 || bound[vs]) + (vo < 0 || bound[vo]);
            uint64_t c = ix->pcount[pats[i].p];
            if (nb > best_b || (nb == best_b && c < best_c)) { best = (int)i; best_b = nb; best_c = c; }
        }
        taken[best] = 1; order[d] = pats[best];
        int vs = var_of(pats[best].s), vo = var_of(pats[best].o);
        if (vs >= 0) bound[vs] = 1;
        if (vo >= 0) bound[vo] = 1;
    }
    return k;
}

/* Step 3 over the ordered patterns into one buffer per thread (the first
 * pattern's candidates split among the threads). */
static void run_join(const orc_index* ix, const pat_t* order, uint32_t n_pat, int k, int threads,
                     rowbuf* bufs) {
    join_t J = {ix, order, n_pat};

    /* split the first pattern's candidates among threads */
    const pat_t* q0 = &order[0];
    int vs0 = var_of(q0->s), vo0 = var_of(q0->o);
    const tri* base; uint64_t b = 0, e = 0; int mode;
    if (vs0 < 0 && vo0 < 0) { mode = 0; }
    else if (vs0 < 0) { mode = 1; base = ix->spo; range2(ix->spo, ix->n, (uint32_t)q0->s, (uint32_t)q0->p, &b, &e); }
    else if (vo0 < 0) { mode = 2; base = ix->ops; range2(ix->ops, ix->n, (uint32_t)q0->o, (uint32_t)q0->p, &b, &e); }
    else { mode = 3; base = ix->pso; range1(ix->pso, ix->n, (uint32_t)q0->p, &b, &e); }
    (void)base;
    if (mode == 0) {
        int64_t mu[MAXVAR];
        for (int v = 0; v < k; ++v) mu[v] = -1;
        join(&J, 0, mu, &bufs[0]);
    } else {
        #pragma omp parallel for num_threads(threads) schedule(dynamic, 64)
        for (int64_t i = (int64_t)b; i < (int64_t)e; ++i) {
#ifdef _OPENMP
            int t = omp_get_thread_num();
#else
            int t = 0;
#endif
            int64_t mu[MAXVAR];
            for (int v = 0; v < k; ++v) mu[v] = -1;
            if (mode == 1) mu[vo0] = ix->spo[i].c;
            else if (mode == 2) mu[vs0] = ix->ops[i].c;
            else {
                if (vs0 == vo0) {
                    if (ix->pso[i].b != ix->pso[i].c) continue;
                    mu[vs0] = ix->pso[i].b;
                } else { mu[vs0] = ix->pso[i].b; mu[vo0] = ix->pso[i].c; }
            }
            join(&J, 1, mu, &bufs[t]);
        }
    }
}

/* Evaluate a BGP.
 *   patterns   n_pat x 3 int64 (s, p, o): s, o >= 0 constant vertex id,
 *              < 0 variable -(k+1); p a predicate id in 1..n_preds.
 *   threads    OpenMP threads for the first pattern's candidates (>= 1).
 *   rows_out   malloc'd int32 rows (n_rows x n_vars), caller frees with orc_free.
 * Returns 0; -1 bad query (no variables, variable ids not dense, bad
 * predicate or vertex); -2 out of memory; -3 a duplicate row (a bug). */
int orc_eval(const orc_index* ix, const int64_t* patterns, uint32_t n_pat, int threads,
             int32_t** rows_out, uint64_t* n_rows, uint32_t* n_vars) {
    *rows_out = NULL; *n_rows = 0; *n_vars = 0;
    pat_t order[MAXPAT];
    const int k = prepare(ix, patterns, n_pat, order);
    if (k < 0) return -1;
    if (threads < 1) threads = 1;
    rowbuf* bufs = (rowbuf*)calloc((size_t)threads, sizeof(rowbuf));
    if (!bufs) return -2;
    for (int t = 0; t < threads; ++t) bufs[t].k = (uint32_t)k;
    run_join(ix, order, n_pat, k, threads, bufs);

    uint64_t total = 0; int oom = 0;
    for (int t = 0; t < threads; ++t) { total += bufs[t].n; oom |= bufs[t].oom; }
    int32_t* rows = oom ? NULL : (int32_t*)malloc(sizeof(int32_t) * (total ? total : 1) * (uint64_t)k);
    if (!rows) oom = 1;
    uint64_t at = 0;
    for (int t = 0; t < threads; ++t) {
        if (!oom && bufs[t].n) memcpy(rows + at * k, bufs[t].rows, sizeof(int32_t) * bufs[t].n * k);
        at += bufs[t].n;
        free(bufs[t].rows);
    }
    free(bufs);
    if (oom) { free(rows); return -2; }
    cmp_k = (uint32_t)k;
    qsort(rows, total, sizeof(int32_t) * k, cmp_row);
    for (uint64_t i = 1; i < total; ++i)
        if (cmp_row(rows + (i - 1) * k, rows + i * k) == 0) { free(rows); return -3; }
    *rows_out = rows; *n_rows = total; *n_vars = (uint32_t)k;
    return 0;
}

void orc_free(void* p) { free(p); }

/* The number of answer rows of a BGP (as orc_eval, without storing them),
 * giving up when the join makes more than max_steps calls (0: no limit) over
 * all threads: a measure of the work the query takes here.
 * Returns 0; -1 bad query; -2 out of memory; -4 the step limit was reached
 * (*n_rows is then a lower bound). *steps gets the calls made (may be NULL). */
int orc_count(const orc_index* ix, const int64_t* patterns, uint32_t n_pat, int threads,
              uint64_t max_steps, uint64_t* n_rows, uint64_t* steps) {
    *n_rows = 0;
    if (steps) *steps = 0;
    pat_t order[MAXPAT];
    const int k = prepare(ix, patterns, n_pat, order);
    if (k < 0) return -1;
    if (threads < 1) threads = 1;
    rowbuf* bufs = (rowbuf*)calloc((size_t)threads, sizeof(rowbuf));
    if (!bufs) return -2;
    for (int t = 0; t < threads; ++t) {
        bufs[t].k = (uint32_t)k;
        bufs[t].count_only = 1;
        bufs[t].max_steps = max_steps ? (max_steps + threads - 1) / threads : 0;
    }
    run_join(ix, order, n_pat, k, threads, bufs);
    int stopped = 0;
    for (int t = 0; t < threads; ++t) {
        *n_rows += bufs[t].n;
        if (steps) *steps += bufs[t].steps;
        stopped |= bufs[t].stop;
    }
    free(bufs);
    return stopped ? -4 : 0;
}
