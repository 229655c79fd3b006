/*
 * rdfgen — seeded synthetic RDF graphs and BGP queries.
 *
 * This module only produces inputs. It holds none of the evaluation method:
 * no candidate scans, no grouped evaluation, no binding trees. Both the
 * oracle and the CUDA engine consume what it writes, and neither shares any
 * other code.
 *
 * Random numbers. Every draw is a pure function of (seed, stream, counter)
 * built from the SplitMix64 output mix (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014; constants as published in
 * Vigna's splitmix64.c reference):
 *     key  = mix64(seed ^ (stream * 0xD1B54A32D192ED03))
 *     draw = mix64(key + (counter + 1) * 0x9E3779B97F4A7C15)
 *
 * Graphs. R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004) with Graph500
 * quadrant probabilities: each of `scale` levels picks a quadrant from a
 * 32-bit uniform, most significant bit first, no noise. Vertex ids are then
 * passed through a keyed bijection of [0, 2^scale) so hubs are spread over
 * the id space. Predicates are drawn independently from Zipf(s) over 1..P
 * (predicate ids are 1-based; 0 means "no entry", as in the paper's
 * encoding, Sec. 6.2.1). Exactly n_edges triples are drawn; duplicates are
 * left in (the consumers deduplicate).
 *
 * Queries. A query shape is an undirected connected multigraph over shape
 * vertices. It is embedded by a seeded random walk: shape vertex 0 is
 * mapped to an endpoint of a uniformly drawn triple, every tree edge (in
 * the order given) draws a uniform incident triple of its mapped end, and
 * every non-tree edge draws a uniform triple among those joining its two
 * mapped ends (the attempt fails if none exists). The triples found give
 * the predicates and directions, so the embedding itself is one match.
 * Shape vertices flagged constant keep their mapped id.
 *
 * Result-size bound. For rejection of queries whose answers would be too
 * large to hold, rdfgen_tree_bound() counts the matches of the query's
 * spanning tree (non-tree edges dropped), which bounds the full count from
 * above. It is input selection only.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GAMMA 0x9E3779B97F4A7C15ULL
#define STREAM_MUL 0xD1B54A32D192ED03ULL

enum { ST_RMAT = 1, ST_PERM = 2, ST_LABEL = 3, ST_QUERY = 4 };

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
    return mix64(seed ^ (stream * STREAM_MUL));
}

static inline uint64_t draw(uint64_t key, uint64_t ctr) {
    return mix64(key + (ctr + 1) * GAMMA);
}

uint64_t rdfgen_draw(uint64_t seed, uint64_t stream, uint64_t ctr) {
    return draw(stream_key(seed, stream), ctr);
}

/* Keyed bijection of [0, 2^scale): four rounds of multiply-by-odd, add-key
 * and xorshift, each a bijection modulo 2^scale. */
typedef struct { uint64_t mul[4], add[4]; uint64_t mask; int shift; } perm_t;

static void perm_init(perm_t* pm, uint64_t seed, int scale) {
    uint64_t k = stream_key(seed, ST_PERM);
    for (int r = 0; r < 4; ++r) {
        pm->mul[r] = draw(k, 2 * r) | 1ULL;
        pm->add[r] = draw(k, 2 * r + 1);
    }
    pm->mask = (scale >= 64) ? ~0ULL : ((1ULL << scale) - 1ULL);
    pm->shift = scale / 2 + 1;
}

static inline uint64_t perm_apply(const perm_t* pm, uint64_t x) {
    for (int r = 0; r < 4; ++r) {
        x = (x * pm->mul[r] + pm->add[r]) & pm->mask;
        x ^= x >> pm->shift;
    }
    return x;
}

uint64_t rdfgen_perm(uint64_t seed, int scale, uint64_t x) {
    perm_t pm; perm_init(&pm, seed, scale);
    return perm_apply(&pm, x & pm.mask);
}

/* R-MAT triples with Zipf(zipf_s) predicates in 1..n_preds.
 * abcd: the four quadrant probabilities (a, b, c, d); d is implied. */
int rdfgen_rmat(int scale, uint64_t n_edges, uint32_t n_preds, double zipf_s,
                double a, double b, double c, uint64_t seed,
                uint32_t* s_out, uint32_t* p_out, uint32_t* o_out) {
    if (scale < 1 || scale > 31 || n_preds < 1) return -1;
    const uint64_t ta = (uint64_t)(a * 4294967296.0);
    const uint64_t tb = (uint64_t)((a + b) * 4294967296.0);
    const uint64_t tc = (uint64_t)((a + b + c) * 4294967296.0);
    double* cdf = (double*)malloc(sizeof(double) * n_preds);
    if (!cdf) return -2;
    double acc = 0.0;
    for (uint32_t i = 0; i < n_preds; ++i) { acc += 1.0 / pow((double)(i + 1), zipf_s); cdf[i] = acc; }
    for (uint32_t i = 0; i < n_preds; ++i) cdf[i] /= acc;
    cdf[n_preds - 1] = 1.0;
    perm_t pm; perm_init(&pm, seed, scale);
    const uint64_t krm = stream_key(seed, ST_RMAT), klab = stream_key(seed, ST_LABEL);
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < (int64_t)n_edges; ++e) {
        uint64_t s = 0, o = 0, r = 0;
        for (int l = 0; l < scale; ++l) {
            if ((l & 1) == 0) r = draw(krm, (uint64_t)e * 16 + (uint64_t)(l >> 1));
            uint64_t u = (l & 1) ? (r >> 32) : (r & 0xFFFFFFFFULL);
            uint64_t bs, bo;
            if (u < ta) { bs = 0; bo = 0; }
            else if (u < tb) { bs = 0; bo = 1; }
            else if (u < tc) { bs = 1; bo = 0; }
            else { bs = 1; bo = 1; }
            s = (s << 1) | bs; o = (o << 1) | bo;
        }
        double u = (double)(draw(klab, (uint64_t)e) >> 11) * (1.0 / 9007199254740992.0);
        uint32_t lo = 0, hi = n_preds - 1;
        while (lo < hi) { uint32_t mid = (lo + hi) >> 1; if (cdf[mid] > u) hi = mid; else lo = mid + 1; }
        s_out[e] = (uint32_t)perm_apply(&pm, s);
        o_out[e] = (uint32_t)perm_apply(&pm, o);
        p_out[e] = lo + 1;
    }
    free(cdf);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Adjacency used for query sampling and for the tree bound.          */

typedef struct {
    uint32_t n_vertices, n_preds;
    uint64_t n;
    const uint32_t *s, *p, *o;     /* caller-owned raw triples (kept alive by caller) */
    uint64_t *out_off, *in_off;    /* per vertex: triple indices of out / in edges */
    uint64_t *out_idx, *in_idx;
    uint64_t *pred_off;            /* per predicate: triple indices */
    uint64_t *pred_idx;
} rdf_adj;

void rdfgen_adj_free(rdf_adj* g) {
    if (!g) return;
    free(g->out_off); free(g->in_off); free(g->out_idx); free(g->in_idx);
    free(g->pred_off); free(g->pred_idx); free(g);
}

/* Bucket triple indices by key (a counting sort). The scatter runs in
 * parallel; each bucket is then sorted so the result is deterministic. */
static int cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x > y) - (x < y);
}

static int bucket(uint64_t n_keys, const uint32_t* key, uint64_t n, uint64_t** off_out, uint64_t** idx_out) {
    uint64_t* off = (uint64_t*)calloc(n_keys + 1, sizeof(uint64_t));
    uint64_t* idx = (uint64_t*)malloc(sizeof(uint64_t) * (n ? n : 1));
    uint64_t* cur = (uint64_t*)malloc(sizeof(uint64_t) * (n_keys ? n_keys : 1));
    if (!off || !idx || !cur) { free(off); free(idx); free(cur); return -1; }
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        #pragma omp atomic
        off[key[i] + 1]++;
    }
    for (uint64_t k = 0; k < n_keys; ++k) off[k + 1] += off[k];
    memcpy(cur, off, sizeof(uint64_t) * n_keys);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        uint64_t slot;
        #pragma omp atomic capture
        slot = cur[key[i]]++;
        idx[slot] = (uint64_t)i;
    }
    free(cur);
    #pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t k = 0; k < (int64_t)n_keys; ++k)
        if (off[k + 1] - off[k] > 1) qsort(idx + off[k], off[k + 1] - off[k], sizeof(uint64_t), cmp_u64);
    *off_out = off; *idx_out = idx;
    return 0;
}

rdf_adj* rdfgen_adj_build(const uint32_t* s, const uint32_t* p, const uint32_t* o, uint64_t n,
                          uint32_t n_vertices, uint32_t n_preds) {
    rdf_adj* g = (rdf_adj*)calloc(1, sizeof(rdf_adj));
    if (!g) return NULL;
    g->n_vertices = n_vertices; g->n_preds = n_preds; g->n = n; g->s = s; g->p = p; g->o = o;
    if (bucket(n_vertices, s, n, &g->out_off, &g->out_idx) ||
        bucket(n_vertices, o, n, &g->in_off, &g->in_idx) ||
        bucket((uint64_t)n_preds + 1, p, n, &g->pred_off, &g->pred_idx)) {
        rdfgen_adj_free(g); return NULL;
    }
    return g;
}

/* Embed one query shape.
 *   n_sv          shape vertices; shape vertex 0 is the walk start
 *   n_se, se      shape edges as (u, w) pairs; the first n_sv-1 edges must form a
 *                 spanning tree in which the u end is already reached when the
 *                 edge is visited; the rest are non-tree edges
 *   is_const      per shape vertex: 1 = constant
 *   dir_req       per shape edge: 0 = any direction, 1 = u must be the subject,
 *                 2 = u must be the object (tree edges only)
 *   plo, phi      per shape edge: its predicate must lie in plo[e]..phi[e]
 *                 (both NULL: any predicate)
 *   patterns      out: n_se x 3 int64 (s, p, o); variables are -(k+1) with k
 *                 the rank of the shape vertex among non-constant ones
 *   mapped        out: the graph vertex of each shape vertex
 *   u_subject     out: per shape edge, 1 when its u end is the triple's subject
 * Returns 0 on success, 1 when this attempt found no embedding. */
static inline int pred_ok(const rdf_adj* g, uint64_t t, const uint32_t* plo, const uint32_t* phi,
                          uint32_t e) {
    return !plo || (g->p[t] >= plo[e] && g->p[t] <= phi[e]);
}

int rdfgen_embed(const rdf_adj* g, uint32_t n_sv, uint32_t n_se, const uint32_t* se,
                 const uint8_t* is_const, const uint8_t* dir_req, const uint32_t* plo,
                 const uint32_t* phi, uint64_t seed, uint64_t attempt,
                 int64_t* patterns, uint32_t* mapped, uint8_t* u_subject) {
    if (g->n == 0 || n_sv == 0 || n_se + 1 < n_sv) return 1;
    const uint64_t kq = stream_key(seed, ST_QUERY);
    uint64_t ctr = attempt * 4096;
    int64_t* mv = (int64_t*)malloc(sizeof(int64_t) * n_sv);
    for (uint32_t v = 0; v < n_sv; ++v) mv[v] = -1;
    uint64_t t0 = draw(kq, ctr++) % g->n;
    mv[0] = (draw(kq, ctr++) & 1) ? g->o[t0] : g->s[t0];
    int ok = 1;
    for (uint32_t e = 0; e < n_se && ok; ++e) {
        uint32_t u = se[2 * e], w = se[2 * e + 1];
        uint64_t gu, ti; int u_is_subject;
        if (e + 1 < n_sv) {                       /* tree edge: u reached, w new */
            if (mv[u] < 0 || mv[w] >= 0) { ok = 0; break; }
            gu = (uint64_t)mv[u];
            uint64_t dout = g->out_off[gu + 1] - g->out_off[gu];
            uint64_t din = g->in_off[gu + 1] - g->in_off[gu];
            if (dir_req[e] == 1) din = 0;
            if (dir_req[e] == 2) { dout = 0; }
            if (dout + din == 0) { ok = 0; break; }
            uint64_t dout_full = g->out_off[gu + 1] - g->out_off[gu];
            if (plo) {
                /* uniform among the incident triples whose predicate is in range */
                uint64_t cnt = 0;
                for (uint64_t k = 0; k < dout; ++k) cnt += pred_ok(g, g->out_idx[g->out_off[gu] + k], plo, phi, e);
                for (uint64_t k = 0; k < din; ++k) cnt += pred_ok(g, g->in_idx[g->in_off[gu] + k], plo, phi, e);
                if (cnt == 0) { ok = 0; break; }
                uint64_t pick = draw(kq, ctr++) % cnt;
                ti = 0; u_is_subject = 1;
                for (uint64_t k = 0; k < dout; ++k) {
                    uint64_t t = g->out_idx[g->out_off[gu] + k];
                    if (pred_ok(g, t, plo, phi, e)) { if (pick == 0) { ti = t; u_is_subject = 1; goto picked; } --pick; }
                }
                for (uint64_t k = 0; k < din; ++k) {
                    uint64_t t = g->in_idx[g->in_off[gu] + k];
                    if (pred_ok(g, t, plo, phi, e)) { if (pick == 0) { ti = t; u_is_subject = 0; goto picked; } --pick; }
                }
            picked:
                mv[w] = u_is_subject ? g->o[ti] : g->s[ti];
            } else {
                uint64_t r = draw(kq, ctr++) % (dout + din);
                if (dir_req[e] == 2) r += dout_full;
                if (r < dout_full) { ti = g->out_idx[g->out_off[gu] + r]; u_is_subject = 1; mv[w] = g->o[ti]; }
                else { ti = g->in_idx[g->in_off[gu] + (r - dout_full)]; u_is_subject = 0; mv[w] = g->s[ti]; }
            }
        } else {                                   /* non-tree edge: both ends mapped */
            if (mv[u] < 0 || mv[w] < 0) { ok = 0; break; }
            gu = (uint64_t)mv[u];
            uint64_t gw = (uint64_t)mv[w];
            uint64_t dout = g->out_off[gu + 1] - g->out_off[gu];
            uint64_t din = g->in_off[gu + 1] - g->in_off[gu];
            uint64_t cnt = 0;
            for (uint64_t k = 0; k < dout; ++k) {
                uint64_t t = g->out_idx[g->out_off[gu] + k];
                cnt += g->o[t] == gw && pred_ok(g, t, plo, phi, e);
            }
            for (uint64_t k = 0; k < din; ++k) {
                uint64_t t = g->in_idx[g->in_off[gu] + k];
                cnt += g->s[t] == gw && pred_ok(g, t, plo, phi, e);
            }
            if (cnt == 0) { ok = 0; break; }
            uint64_t pick = draw(kq, ctr++) % cnt;
            ti = 0; u_is_subject = 1;
            for (uint64_t k = 0; k < dout; ++k) {
                uint64_t t = g->out_idx[g->out_off[gu] + k];
                if (g->o[t] == gw && pred_ok(g, t, plo, phi, e)) { if (pick == 0) { ti = t; u_is_subject = 1; goto found; } --pick; }
            }
            for (uint64_t k = 0; k < din; ++k) {
                uint64_t t = g->in_idx[g->in_off[gu] + k];
                if (g->s[t] == gw && pred_ok(g, t, plo, phi, e)) { if (pick == 0) { ti = t; u_is_subject = 0; goto found; } --pick; }
            }
        found:;
        }
        patterns[3 * e + 1] = g->p[ti];
        u_subject[e] = (uint8_t)u_is_subject;
        patterns[3 * e + 0] = u_is_subject ? (int64_t)u : (int64_t)w;   /* shape ids for now */
        patterns[3 * e + 2] = u_is_subject ? (int64_t)w : (int64_t)u;
    }
    if (ok) {
        int64_t* var_of = (int64_t*)malloc(sizeof(int64_t) * n_sv);
        int64_t k = 0;
        for (uint32_t v = 0; v < n_sv; ++v) var_of[v] = is_const[v] ? mv[v] : -(k++ + 1);
        for (uint32_t e = 0; e < n_se; ++e) {
            patterns[3 * e + 0] = var_of[patterns[3 * e + 0]];
            patterns[3 * e + 2] = var_of[patterns[3 * e + 2]];
        }
        for (uint32_t v = 0; v < n_sv; ++v) mapped[v] = (uint32_t)mv[v];
        free(var_of);
    }
    free(mv);
    return ok ? 0 : 1;
}
/* Upper bound on the number of matches of a query: the exact match count
 * of its spanning tree (first n_sv-1 shape edges of the embedding order,
 * non-tree edges dropped), counting raw triples with multiplicity.
 *   n_sv, se    the shape used for the embedding (tree edges first)
 *   is_const, mapped, u_subject  as returned by rdfgen_embed
 *   patterns    n_se x 3, from rdfgen_embed
 * A tree DP: f_u(x) = prod over children w of sum_{y joined to x by the
 * child's edge} f_w(y). Children whose vector has a small support (their
 * subtree holds a constant) are folded first through the adjacency of that
 * support; later children are then evaluated only where the parent is
 * still non-zero. Only when both sides are dense does a fold read the
 * predicate's whole triple list. Returns the bound as a double. */

typedef struct { double* v; uint32_t* sup; uint64_t nsup; int sparse; } dvec;

static void dvec_support(dvec* d, uint32_t N, uint64_t small) {
    uint64_t nz = 0;
    for (uint32_t x = 0; x < N; ++x) nz += d->v[x] != 0.0;
    d->sparse = nz < small;
    d->nsup = 0;
    if (d->sparse) {
        d->sup = (uint32_t*)realloc(d->sup, sizeof(uint32_t) * (nz ? nz : 1));
        for (uint32_t x = 0; x < N; ++x) if (d->v[x] != 0.0) d->sup[d->nsup++] = x;
    }
}

double rdfgen_tree_bound(const rdf_adj* g, uint32_t n_sv, const uint32_t* se,
                         const uint8_t* is_const, const uint32_t* mapped, const int64_t* patterns,
                         const uint8_t* u_subject) {
    const uint32_t N = g->n_vertices;
    const uint64_t small = N / 16 + 1;
    dvec* f = (dvec*)calloc(n_sv, sizeof(dvec));
    double* tmp = (double*)malloc(sizeof(double) * N);
    /* parent edge of every shape vertex (tree edges only) */
    int64_t* pe = (int64_t*)malloc(sizeof(int64_t) * n_sv);
    for (uint32_t v = 0; v < n_sv; ++v) pe[v] = -1;
    for (uint32_t e = 0; e + 1 < n_sv; ++e) pe[se[2 * e + 1]] = e;
    /* discovery order: vertex 0, then the child of each tree edge in order */
    uint32_t* order = (uint32_t*)malloc(sizeof(uint32_t) * n_sv);
    order[0] = 0;
    for (uint32_t e = 0; e + 1 < n_sv; ++e) order[e + 1] = se[2 * e + 1];
    for (int64_t oi = (int64_t)n_sv - 1; oi >= 0; --oi) {
        uint32_t u = order[oi];
        dvec* fu = &f[u];
        fu->v = (double*)malloc(sizeof(double) * N);
        if (is_const[u]) {
            memset(fu->v, 0, sizeof(double) * N);
            fu->v[mapped[u]] = 1.0;
            fu->sup = (uint32_t*)malloc(sizeof(uint32_t));
            fu->sup[0] = mapped[u]; fu->nsup = 1; fu->sparse = 1;
        } else {
            for (uint32_t x = 0; x < N; ++x) fu->v[x] = 1.0;
            fu->sparse = 0;
        }
        /* children of u, sparse ones first */
        for (int pass = 0; pass < 2; ++pass) {
            for (uint32_t e = 0; e + 1 < n_sv; ++e) {
                if (se[2 * e] != u) continue;
                uint32_t w = se[2 * e + 1];
                dvec* fw = &f[w];
                if ((pass == 0) != (fw->sparse != 0)) continue;
                uint32_t p = (uint32_t)patterns[3 * e + 1];
                int us = u_subject[e];
                /* x is u's end, y is w's end of a triple with label p */
                const uint64_t* xoff = us ? g->out_off : g->in_off;
                const uint64_t* xix = us ? g->out_idx : g->in_idx;
                const uint64_t* yoff = us ? g->in_off : g->out_off;
                const uint64_t* yix = us ? g->in_idx : g->out_idx;
                if (fu->sparse) {
                    /* evaluate only where f_u is non-zero, through x's adjacency */
                    uint64_t keep = 0;
                    for (uint64_t k = 0; k < fu->nsup; ++k) {
                        uint32_t x = fu->sup[k];
                        double acc = 0.0;
                        for (uint64_t t = xoff[x]; t < xoff[x + 1]; ++t) {
                            uint64_t ti = xix[t];
                            if (g->p[ti] != p) continue;
                            acc += fw->v[us ? g->o[ti] : g->s[ti]];
                        }
                        fu->v[x] *= acc;
                        if (fu->v[x] != 0.0) fu->sup[keep++] = x;
                    }
                    fu->nsup = keep;
                } else if (fw->sparse) {
                    memset(tmp, 0, sizeof(double) * N);
                    for (uint64_t k = 0; k < fw->nsup; ++k) {
                        uint32_t y = fw->sup[k];
                        for (uint64_t t = yoff[y]; t < yoff[y + 1]; ++t) {
                            uint64_t ti = yix[t];
                            if (g->p[ti] != p) continue;
                            tmp[us ? g->s[ti] : g->o[ti]] += fw->v[y];
                        }
                    }
                    for (uint32_t x = 0; x < N; ++x) fu->v[x] *= tmp[x];
                    dvec_support(fu, N, small);
                } else {
                    int nt = 1;
#ifdef _OPENMP
                    nt = omp_get_max_threads();
#endif
                    double* part = (double*)calloc((size_t)nt * N, sizeof(double));
                    const uint64_t b0 = g->pred_off[p], b1 = g->pred_off[p + 1];
                    const double* wv = fw->v;
                    double* uv = fu->v;
                    #pragma omp parallel num_threads(nt)
                    {
                        int tid = 0;
#ifdef _OPENMP
                        tid = omp_get_thread_num();
#endif
                        double* mine = part + (size_t)tid * N;
                        #pragma omp for schedule(static)
                        for (int64_t t = (int64_t)b0; t < (int64_t)b1; ++t) {
                            uint64_t ti = g->pred_idx[t];
                            uint32_t x = us ? g->s[ti] : g->o[ti];
                            uint32_t y = us ? g->o[ti] : g->s[ti];
                            mine[x] += wv[y];
                        }
                        #pragma omp for schedule(static)
                        for (int64_t x = 0; x < (int64_t)N; ++x) {
                            double acc = 0.0;
                            for (int k = 0; k < nt; ++k) acc += part[(size_t)k * N + x];
                            uv[x] *= acc;
                        }
                    }
                    free(part);
                    dvec_support(fu, N, small);
                }
            }
        }
        /* children are no longer needed */
        for (uint32_t e = 0; e + 1 < n_sv; ++e) {
            if (se[2 * e] != u) continue;
            uint32_t w = se[2 * e + 1];
            free(f[w].v); free(f[w].sup); f[w].v = NULL; f[w].sup = NULL;
        }
    }
    double total = 0.0;
    if (f[0].sparse) for (uint64_t k = 0; k < f[0].nsup; ++k) total += f[0].v[f[0].sup[k]];
    else for (uint32_t x = 0; x < N; ++x) total += f[0].v[x];
    free(f[0].v); free(f[0].sup);
    free(f); free(tmp); free(pe); free(order);
    return total;
}

/* Tree bound rooted at a constant: the same spanning-tree match count as
 * rdfgen_tree_bound, computed top-down from shape vertex `root` (which must
 * be a constant) through the adjacency of the vertices actually reached,
 * with memoisation per (shape vertex, graph vertex). Returns -1 once more
 * than work_cap adjacency entries have been visited (the query is then far
 * too unselective to keep). Input selection only. */
typedef struct { uint32_t* key; double* val; uint64_t cap, n; } memo_t;

static double* memo_get(memo_t* m, uint32_t k, int* fresh) {
    if (2 * (m->n + 1) > m->cap) {
        uint64_t nc = m->cap ? 2 * m->cap : 1024;
        uint32_t* nk = (uint32_t*)malloc(sizeof(uint32_t) * nc);
        double* nv = (double*)malloc(sizeof(double) * nc);
        for (uint64_t i = 0; i < nc; ++i) nk[i] = 0xffffffffu;
        for (uint64_t i = 0; i < m->cap; ++i) {
            if (m->key[i] == 0xffffffffu) continue;
            uint64_t h = mix64(m->key[i]) & (nc - 1);
            while (nk[h] != 0xffffffffu) h = (h + 1) & (nc - 1);
            nk[h] = m->key[i]; nv[h] = m->val[i];
        }
        free(m->key); free(m->val);
        m->key = nk; m->val = nv; m->cap = nc;
    }
    uint64_t h = mix64(k) & (m->cap - 1);
    while (m->key[h] != 0xffffffffu) {
        if (m->key[h] == k) { *fresh = 0; return &m->val[h]; }
        h = (h + 1) & (m->cap - 1);
    }
    m->key[h] = k; m->n++; *fresh = 1;
    return &m->val[h];
}

typedef struct {
    const rdf_adj* g;
    uint32_t n_sv;
    const uint32_t* se;
    const uint8_t* is_const;
    const uint32_t* mapped;
    const int64_t* patterns;
    const uint8_t* u_subject;
    memo_t* memo;
    uint64_t work, cap;
} rooted_t;

/* matches of the subtree of shape vertex w (away from tree edge via) with w -> y */
static double rooted_count(rooted_t* c, uint32_t w, uint32_t y, int64_t via) {
    if (c->is_const[w] && c->mapped[w] != y) return 0.0;
    int fresh = 0;
    double* slot = memo_get(&c->memo[w], y, &fresh);
    if (!fresh) return *slot;
    *slot = 0.0;
    double prod = 1.0;
    for (uint32_t e = 0; e + 1 < c->n_sv && prod != 0.0; ++e) {
        if ((int64_t)e == via) continue;
        uint32_t a = c->se[2 * e], b = c->se[2 * e + 1], u;
        int w_subj;
        if (a == w) { u = b; w_subj = c->u_subject[e] != 0; }
        else if (b == w) { u = a; w_subj = c->u_subject[e] == 0; }
        else continue;
        const uint32_t p = (uint32_t)c->patterns[3 * e + 1];
        const uint64_t* off = w_subj ? c->g->out_off : c->g->in_off;
        const uint64_t* ix = w_subj ? c->g->out_idx : c->g->in_idx;
        double sum = 0.0;
        for (uint64_t t = off[y]; t < off[y + 1]; ++t) {
            if (++c->work > c->cap) return 0.0;
            const uint64_t ti = ix[t];
            if (c->g->p[ti] != p) continue;
            sum += rooted_count(c, u, w_subj ? c->g->o[ti] : c->g->s[ti], (int64_t)e);
            if (c->work > c->cap) return 0.0;
        }
        prod *= sum;
    }
    slot = memo_get(&c->memo[w], y, &fresh);   /* the table may have moved */
    *slot = prod;
    return prod;
}

double rdfgen_tree_bound_rooted(const rdf_adj* g, uint32_t n_sv, const uint32_t* se,
                                const uint8_t* is_const, const uint32_t* mapped,
                                const int64_t* patterns, const uint8_t* u_subject, uint32_t root,
                                uint64_t work_cap) {
    if (root >= n_sv || !is_const[root]) return -1.0;
    rooted_t c = {g, n_sv, se, is_const, mapped, patterns, u_subject, NULL, 0, work_cap};
    c.memo = (memo_t*)calloc(n_sv, sizeof(memo_t));
    double total = rooted_count(&c, root, mapped[root], -1);
    for (uint32_t v = 0; v < n_sv; ++v) { free(c.memo[v].key); free(c.memo[v].val); }
    free(c.memo);
    return c.work > work_cap ? -1.0 : total;
}
