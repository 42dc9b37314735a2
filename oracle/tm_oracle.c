/*
 * CPU oracle for exact delta-temporal motif counting.
 *
 * TEST INFRASTRUCTURE ONLY. The tests, the smoke check and the benchmark's
 * CPU-baseline leg are the only code that may load this library. It shares no
 * code, header, table or helper with the CUDA path.
 *
 * What it computes (arXiv 2204.09236):
 *   - orc_count: Algorithm 1 (FAST-Star/Pair) and Algorithm 2 (FAST-Tri), run
 *     for every centre node, in the order and notation of the paper.
 *   - orc_brute: the definitions themselves (Def. 2, Def. 3, Problem 1): every
 *     time-ordered edge triple whose span is at most delta, classified into the
 *     paper's counters Star[Type,d1,d2,d3] (Sec. IV-A), Pair[d1,d2,d3]
 *     (Sec. IV-A case (b)) and Tri[Type,di,dj,dk] (Sec. IV-B).
 *   - orc_brute_classes: the 36 motif classes of Problem 1 straight from the
 *     edge pattern of each instance (Def. 3: same direction and time order).
 *
 * Encoding: Type I=0, II=1, III=2; direction o (outward from the centre) = 0,
 * in (inward to the centre) = 1. Flat indices:
 *   Star/Tri: ((T*2 + a)*2 + b)*2 + c        Pair: (a*2 + b)*2 + c
 *
 * Readings of the paper (its text leaves these open):
 *   - Ties in time (Def. 2 only asks t1 <= t2 <= t3): edges are totally
 *     ordered by (t, edge id), edge id = array index, and each 3-edge set is
 *     counted once, in that order. Every order comparison of Algorithm 2 is
 *     taken in this total order; delta tests use raw timestamps.
 *   - Window: t3 - t1 <= delta (Def. 2; Alg. 1 break test; Alg. 2). Every
 *     window test is written as a difference of two timestamps compared with
 *     delta (t_j - delta <= t_k is tested as t_j - t_k <= delta), so no sum
 *     overflows; orc_build rejects graphs whose timestamp span does not fit
 *     in int64, which keeps every difference representable.
 *   - dir_k of a triangle is relative to v = e_i.v (Sec. IV-B definition).
 *   - Self-loops are rejected (all workloads have u != v).
 */
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O 0
#define IN 1
#define T_I 0
#define T_II 1
#define T_III 2
#define STAR(T, a, b, c) star[(((T) * 2 + (a)) * 2 + (b)) * 2 + (c)]
#define PAIR(a, b, c) pair[((a) * 2 + (b)) * 2 + (c)]
#define TRI(T, a, b, c) tri[(((T) * 2 + (a)) * 2 + (b)) * 2 + (c)]

/* ------------------------------------------------------------------ graph */

/* One entry of S_u (Table 1): e = (t, v, dir) w.r.t. centre u, plus edge id. */
typedef struct {
    int64_t t;
    int32_t id;
    int32_t v;
    int32_t dir;
} s_entry;

/* One edge of E_(v,w), stored with its true source. */
typedef struct {
    int64_t t;
    int32_t id;
    int32_t src;
} p_entry;

typedef struct {
    int64_t m;
    int32_t n;
    int64_t *off; /* n+1: S_u = S[off[u] .. off[u+1]) */
    s_entry *S;   /* 2m */
    int64_t npairs;
    int64_t *pkey; /* sorted keys lo*n + hi */
    int64_t *poff; /* npairs+1 */
    p_entry *P;    /* m, grouped by pair, sorted by (t, id) */
} orc_graph;

/* The HashMaps m_in / m_out of Algorithm 1 (direct addressing by node id,
 * with the list of touched keys for HashMap.Init()). Each thread of
 * orc_count_mt has its own. */
typedef struct {
    int64_t *map_in, *map_out;
    int32_t *touched;
} alg1_maps;

static int maps_init(alg1_maps *h, int32_t n, int64_t m) {
    h->map_in = calloc((size_t)n + 1, sizeof(int64_t));
    h->map_out = calloc((size_t)n + 1, sizeof(int64_t));
    h->touched = malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    return h->map_in && h->map_out && h->touched;
}

static void maps_free(alg1_maps *h) {
    free(h->map_in);
    free(h->map_out);
    free(h->touched);
}

/* (t, id) total order */
static int before(int64_t ta, int32_t ia, int64_t tb, int32_t ib) {
    return ta < tb || (ta == tb && ia < ib);
}

static int cmp_s(const void *a, const void *b) {
    const s_entry *x = a, *y = b;
    if (before(x->t, x->id, y->t, y->id)) return -1;
    if (before(y->t, y->id, x->t, x->id)) return 1;
    return 0;
}

typedef struct {
    int64_t key;
    p_entry e;
} keyed_p;

static int cmp_kp(const void *a, const void *b) {
    const keyed_p *x = a, *y = b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (before(x->e.t, x->e.id, y->e.t, y->e.id)) return -1;
    if (before(y->e.t, y->e.id, x->e.t, x->e.id)) return 1;
    return 0;
}

void orc_free(orc_graph *g) {
    if (!g) return;
    free(g->off);
    free(g->S);
    free(g->pkey);
    free(g->poff);
    free(g->P);
    free(g);
}

/* Returns NULL on invalid input (negative id, self-loop, m < 0, timestamp
 * span beyond int64) or OOM. */
orc_graph *orc_build(int64_t m, const int32_t *src, const int32_t *dst, const int64_t *t) {
    if (m < 0) return NULL;
    int32_t n = 0;
    int64_t tmin = 0, tmax = 0;
    for (int64_t e = 0; e < m; e++) {
        if (src[e] < 0 || dst[e] < 0 || src[e] == dst[e]) return NULL;
        if (src[e] + 1 > n) n = src[e] + 1;
        if (dst[e] + 1 > n) n = dst[e] + 1;
        if (e == 0 || t[e] < tmin) tmin = t[e];
        if (e == 0 || t[e] > tmax) tmax = t[e];
    }
    if (m > 0 && (uint64_t)tmax - (uint64_t)tmin > (uint64_t)INT64_MAX) return NULL;
    orc_graph *g = calloc(1, sizeof(orc_graph));
    if (!g) return NULL;
    g->m = m;
    g->n = n;
    g->off = calloc((size_t)n + 1, sizeof(int64_t));
    g->S = malloc(sizeof(s_entry) * (size_t)(2 * m + 1));
    if (!g->off || !g->S) {
        orc_free(g);
        return NULL;
    }
    /* S_u: every edge incident to u, as (t, other node, direction w.r.t. u) */
    for (int64_t e = 0; e < m; e++) {
        g->off[src[e] + 1]++;
        g->off[dst[e] + 1]++;
    }
    for (int32_t u = 0; u < n; u++) g->off[u + 1] += g->off[u];
    int64_t *fill = malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!fill) {
        orc_free(g);
        return NULL;
    }
    memcpy(fill, g->off, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t e = 0; e < m; e++) {
        s_entry a = {t[e], (int32_t)e, dst[e], O};
        s_entry b = {t[e], (int32_t)e, src[e], IN};
        g->S[fill[src[e]]++] = a;
        g->S[fill[dst[e]]++] = b;
    }
    free(fill);
    for (int32_t u = 0; u < n; u++)
        qsort(g->S + g->off[u], (size_t)(g->off[u + 1] - g->off[u]), sizeof(s_entry), cmp_s);

    /* E_(v,w): edges grouped by unordered node pair, each list sorted by (t, id) */
    keyed_p *kp = malloc(sizeof(keyed_p) * (size_t)(m + 1));
    g->P = malloc(sizeof(p_entry) * (size_t)(m + 1));
    g->pkey = malloc(sizeof(int64_t) * (size_t)(m + 1));
    g->poff = malloc(sizeof(int64_t) * (size_t)(m + 2));
    if (!kp || !g->P || !g->pkey || !g->poff) {
        free(kp);
        orc_free(g);
        return NULL;
    }
    for (int64_t e = 0; e < m; e++) {
        int64_t lo = src[e] < dst[e] ? src[e] : dst[e];
        int64_t hi = src[e] < dst[e] ? dst[e] : src[e];
        kp[e].key = lo * (int64_t)n + hi;
        kp[e].e.t = t[e];
        kp[e].e.id = (int32_t)e;
        kp[e].e.src = src[e];
    }
    qsort(kp, (size_t)m, sizeof(keyed_p), cmp_kp);
    g->npairs = 0;
    for (int64_t i = 0; i < m; i++) {
        if (i == 0 || kp[i].key != kp[i - 1].key) {
            g->pkey[g->npairs] = kp[i].key;
            g->poff[g->npairs] = i;
            g->npairs++;
        }
        g->P[i] = kp[i].e;
    }
    g->poff[g->npairs] = m;
    free(kp);
    return g;
}

int64_t orc_num_nodes(const orc_graph *g) { return g->n; }
int64_t orc_num_entries(const orc_graph *g) { return 2 * g->m; }

/* E_(v,w) as [*b, *e) in g->P; empty range if the pair has no edge. */
static void pair_range(const orc_graph *g, int32_t v, int32_t w, int64_t *b, int64_t *e) {
    int64_t lo = v < w ? v : w, hi = v < w ? w : v;
    int64_t key = lo * (int64_t)g->n + hi;
    int64_t l = 0, r = g->npairs;
    while (l < r) {
        int64_t mid = (l + r) / 2;
        if (g->pkey[mid] < key) l = mid + 1;
        else r = mid;
    }
    if (l < g->npairs && g->pkey[l] == key) {
        *b = g->poff[l];
        *e = g->poff[l + 1];
    } else {
        *b = *e = 0;
    }
}

/* ----------------------------------------------------------- Algorithm 1 */

/* Body of Algorithm 1 for one first edge e1 = S_u[i] (global index i in S,
 * centre segment [sb, se)). m_in / m_out count the second-edge candidates
 * strictly between e1 and the current e3, per neighbour; #e_in / #e_out count
 * them over all neighbours. */
static void alg1_first_edge(const orc_graph *g, alg1_maps *h, int64_t i, int64_t se,
                            int64_t delta, uint64_t *star, uint64_t *pair) {
    const s_entry *S = g->S;
    const s_entry e1 = S[i];
    int64_t n_in = 0, n_out = 0;
    int64_t ntouched = 0;
    for (int64_t j = i + 1; j < se; j++) {
        const s_entry e3 = S[j];
        if (e3.t - e1.t > delta) break;
        if (e3.v == e1.v) {
            PAIR(e1.dir, IN, e3.dir) += h->map_in[e1.v];
            PAIR(e1.dir, O, e3.dir) += h->map_out[e1.v];
            STAR(T_II, e1.dir, IN, e3.dir) += n_in - h->map_in[e1.v];
            STAR(T_II, e1.dir, O, e3.dir) += n_out - h->map_out[e1.v];
        } else {
            STAR(T_I, e1.dir, IN, e3.dir) += h->map_in[e3.v];
            STAR(T_I, e1.dir, O, e3.dir) += h->map_out[e3.v];
            STAR(T_III, e1.dir, IN, e3.dir) += h->map_in[e1.v];
            STAR(T_III, e1.dir, O, e3.dir) += h->map_out[e1.v];
        }
        if (h->map_in[e3.v] == 0 && h->map_out[e3.v] == 0) h->touched[ntouched++] = e3.v;
        if (e3.dir == IN) {
            h->map_in[e3.v] += 1;
            n_in += 1;
        } else {
            h->map_out[e3.v] += 1;
            n_out += 1;
        }
    }
    /* HashMap.Init() for the next e1 */
    for (int64_t k = 0; k < ntouched; k++) {
        h->map_in[h->touched[k]] = 0;
        h->map_out[h->touched[k]] = 0;
    }
}

/* ----------------------------------------------------------- Algorithm 2 */

/* Body of Algorithm 2 for one e_i = S_u[i]. For every e_j after e_i with
 * t_j <= t_i + delta and a different neighbour, scan E_(v,w) from the first
 * edge with t >= t_j - delta (Sec. IV-B's shortcut, which limits xi to the edges
 * within delta) and classify each e_k by its place in the total order. */
static void alg2_first_edge(const orc_graph *g, int64_t i, int64_t se, int64_t delta,
                            uint64_t *tri) {
    const s_entry *S = g->S;
    const s_entry ei = S[i];
    for (int64_t j = i + 1; j < se; j++) {
        const s_entry ej = S[j];
        if (ej.t - ei.t > delta) break;
        if (ej.v == ei.v) continue;
        const int32_t v = ei.v, w = ej.v;
        int64_t b, e;
        pair_range(g, v, w, &b, &e);
        /* first edge of E_(v,w) with t >= t_j - delta */
        int64_t l = b, r = e;
        while (l < r) {
            int64_t mid = (l + r) / 2;
            if (ej.t - g->P[mid].t > delta) l = mid + 1;
            else r = mid;
        }
        for (int64_t k = l; k < e; k++) {
            const p_entry ek = g->P[k];
            const int dk = ek.src == v ? O : IN; /* o: from v to w */
            if (ej.t - ek.t <= delta && before(ek.t, ek.id, ei.t, ei.id)) {
                TRI(T_I, ei.dir, ej.dir, dk)++;
            } else if (before(ei.t, ei.id, ek.t, ek.id) && before(ek.t, ek.id, ej.t, ej.id)) {
                TRI(T_II, ei.dir, ej.dir, dk)++;
            } else if (before(ej.t, ej.id, ek.t, ek.id) && ek.t - ei.t <= delta) {
                TRI(T_III, ei.dir, ej.dir, dk)++;
            } else if (ek.t - ei.t > delta) {
                break;
            }
        }
    }
}

static int32_t centre_of(const orc_graph *g, int64_t i) {
    int32_t l = 0, r = g->n; /* largest u with off[u] <= i */
    while (r - l > 1) {
        int32_t mid = l + (r - l) / 2;
        if (g->off[mid] <= i) l = mid;
        else r = mid;
    }
    return l;
}

/* All 56 cells for every centre node (Algorithm 1 and Algorithm 2). The
 * counters are accumulated, not cleared. Returns -1 on delta < 0, -2 when
 * out of memory. */
int orc_count(orc_graph *g, int64_t delta, uint64_t *star, uint64_t *pair, uint64_t *tri) {
    if (delta < 0) return -1;
    alg1_maps h;
    if (!maps_init(&h, g->n, g->m)) {
        maps_free(&h);
        return -2;
    }
    for (int32_t u = 0; u < g->n; u++) {
        const int64_t sb = g->off[u], se = g->off[u + 1];
        for (int64_t i = sb; i < se; i++) {
            alg1_first_edge(g, &h, i, se, delta, star, pair);
            alg2_first_edge(g, i, se, delta, tri);
        }
    }
    maps_free(&h);
    return 0;
}

/* Same as orc_count, restricted to the first edges S[idx[k]] (global indices
 * into the concatenated S_u lists). Used to time a bounded sample. */
int orc_count_entries(orc_graph *g, int64_t delta, const int64_t *idx, int64_t k,
                      uint64_t *star, uint64_t *pair, uint64_t *tri) {
    if (delta < 0) return -1;
    for (int64_t q = 0; q < k; q++)
        if (idx[q] < 0 || idx[q] >= 2 * g->m) return -1;
    alg1_maps h;
    if (!maps_init(&h, g->n, g->m)) {
        maps_free(&h);
        return -2;
    }
    for (int64_t q = 0; q < k; q++) {
        const int64_t i = idx[q];
        const int32_t u = centre_of(g, i);
        const int64_t se = g->off[u + 1];
        alg1_first_edge(g, &h, i, se, delta, star, pair);
        alg2_first_edge(g, i, se, delta, tri);
    }
    maps_free(&h);
    return 0;
}

/* The counters contributed by one centre node u. */
int orc_count_centre(orc_graph *g, int64_t delta, int32_t u, uint64_t *star, uint64_t *pair,
                     uint64_t *tri) {
    if (delta < 0 || u < 0 || u >= g->n) return -1;
    alg1_maps h;
    if (!maps_init(&h, g->n, g->m)) {
        maps_free(&h);
        return -2;
    }
    const int64_t sb = g->off[u], se = g->off[u + 1];
    for (int64_t i = sb; i < se; i++) {
        alg1_first_edge(g, &h, i, se, delta, star, pair);
        alg2_first_edge(g, i, se, delta, tri);
    }
    maps_free(&h);
    return 0;
}

/* ------------------------------------------- hierarchical parallel count */

/* orc_count on several host threads: the paper's hierarchical scheme
 * (Sec. IV-C) with centres shared out dynamically (inter-node) and a high-
 * degree centre's first edges split into ranges (intra-node). The 2m first
 * edges of the concatenated S_u lists are cut into chunks of `chunk`
 * consecutive positions, which may cut one S_u into several chunks; threads
 * take the next chunk from a shared counter, run the Algorithm 1 and
 * Algorithm 2 bodies for each first edge of it with their own HashMaps and
 * their own counters, and the counters are summed at the end. Every first
 * edge is processed exactly once, and the body of one first edge reads only
 * the graph, so the sum equals orc_count. */
typedef struct {
    const orc_graph *g;
    int64_t delta, chunk, nchunks;
    atomic_llong *next;
    uint64_t cells[56];
    int status;
} mt_worker;

static void *mt_run(void *arg) {
    mt_worker *w = arg;
    const orc_graph *g = w->g;
    alg1_maps h;
    if (!maps_init(&h, g->n, g->m)) {
        maps_free(&h);
        w->status = -2;
        return NULL;
    }
    uint64_t *star = w->cells, *pair = w->cells + 24, *tri = w->cells + 32;
    for (;;) {
        const int64_t c = atomic_fetch_add(w->next, 1);
        if (c >= w->nchunks) break;
        const int64_t b = c * w->chunk;
        const int64_t e = b + w->chunk < 2 * g->m ? b + w->chunk : 2 * g->m;
        int32_t u = centre_of(g, b);
        for (int64_t i = b; i < e; i++) {
            while (g->off[u + 1] <= i) u++;
            alg1_first_edge(g, &h, i, g->off[u + 1], w->delta, star, pair);
            alg2_first_edge(g, i, g->off[u + 1], w->delta, tri);
        }
    }
    maps_free(&h);
    return NULL;
}

/* Returns 0, -1 on a bad argument (delta < 0, nthreads < 1, chunk < 1), -2
 * when out of memory or a thread cannot start. Accumulates like orc_count. */
int orc_count_mt(orc_graph *g, int64_t delta, int32_t nthreads, int64_t chunk, uint64_t *star,
                 uint64_t *pair, uint64_t *tri) {
    if (delta < 0 || nthreads < 1 || chunk < 1) return -1;
    if (g->m == 0) return 0;
    mt_worker *w = calloc((size_t)nthreads, sizeof(mt_worker));
    pthread_t *th = calloc((size_t)nthreads, sizeof(pthread_t));
    int *started = calloc((size_t)nthreads, sizeof(int));
    atomic_llong next;
    atomic_init(&next, 0);
    int rc = 0;
    if (!w || !th || !started) rc = -2;
    for (int32_t k = 0; rc == 0 && k < nthreads; k++) {
        w[k].g = g;
        w[k].delta = delta;
        w[k].chunk = chunk;
        w[k].nchunks = (2 * g->m + chunk - 1) / chunk;
        w[k].next = &next;
        started[k] = pthread_create(&th[k], NULL, mt_run, &w[k]) == 0;
        if (!started[k]) rc = -2;
    }
    for (int32_t k = 0; w && th && started && k < nthreads; k++) {
        if (!started[k]) continue;
        pthread_join(th[k], NULL);
        if (w[k].status) rc = w[k].status;
    }
    for (int32_t k = 0; rc == 0 && k < nthreads; k++) {
        for (int c = 0; c < 24; c++) star[c] += w[k].cells[c];
        for (int c = 0; c < 8; c++) pair[c] += w[k].cells[24 + c];
        for (int c = 0; c < 24; c++) tri[c] += w[k].cells[32 + c];
    }
    free(w);
    free(th);
    free(started);
    return rc;
}

/* ------------------------------------------------------ the definitions */

typedef struct {
    int64_t t;
    int32_t id, s, d;
} edge;

static int cmp_edge(const void *a, const void *b) {
    const edge *x = a, *y = b;
    if (before(x->t, x->id, y->t, y->id)) return -1;
    if (before(y->t, y->id, x->t, x->id)) return 1;
    return 0;
}

static edge *sorted_edges(int64_t m, const int32_t *src, const int32_t *dst, const int64_t *t) {
    edge *E = malloc(sizeof(edge) * (size_t)(m + 1));
    if (!E) return NULL;
    for (int64_t e = 0; e < m; e++) {
        E[e].t = t[e];
        E[e].id = (int32_t)e;
        E[e].s = src[e];
        E[e].d = dst[e];
    }
    qsort(E, (size_t)m, sizeof(edge), cmp_edge);
    return E;
}

static int dir_wrt(const edge *e, int32_t u) { return e->s == u ? O : IN; }
static int touches(const edge *e, int32_t u) { return e->s == u || e->d == u; }
static int same_pair(const edge *a, const edge *b) {
    return (a->s == b->s && a->d == b->d) || (a->s == b->d && a->d == b->s);
}

/* Classify one time-ordered triple (x < y < z) into the counters. */
static void classify_triple(const edge *x, const edge *y, const edge *z, uint64_t *star,
                            uint64_t *pair, uint64_t *tri) {
    const edge *tr[3] = {x, y, z};
    int32_t nodes[6];
    int nn = 0;
    for (int k = 0; k < 3; k++) {
        int32_t ends[2] = {tr[k]->s, tr[k]->d};
        for (int q = 0; q < 2; q++) {
            int seen = 0;
            for (int r = 0; r < nn; r++) seen |= nodes[r] == ends[q];
            if (!seen) nodes[nn++] = ends[q];
        }
    }
    if (nn == 2) {
        /* pair motif: one instance seen from each of its two nodes */
        for (int q = 0; q < 2; q++) {
            const int32_t u = nodes[q];
            PAIR(dir_wrt(x, u), dir_wrt(y, u), dir_wrt(z, u))++;
        }
        return;
    }
    if (nn != 3) return; /* four or more nodes: not a 2/3-node motif */
    const int s01 = same_pair(x, y), s02 = same_pair(x, z), s12 = same_pair(y, z);
    /* three nodes: two edges on one node pair (star) or three pairs (triangle) */
    if (s01 + s02 + s12 > 0) {
        /* star: the centre is the node on all three edges; the isolated edge is
         * the one whose node pair occurs once; Type = its time position */
        int32_t c = -1;
        for (int r = 0; r < 3; r++)
            if (touches(x, nodes[r]) && touches(y, nodes[r]) && touches(z, nodes[r])) c = nodes[r];
        const int iso = s12 ? 0 : (s02 ? 1 : 2);
        STAR(iso, dir_wrt(x, c), dir_wrt(y, c), dir_wrt(z, c))++;
        return;
    }
    /* triangle: seen from each vertex u, e_i < e_j are u's two edges and e_k
     * is the opposite edge; Type by where e_k falls; dir_k relative to e_i.v */
    for (int r = 0; r < 3; r++) {
        const int32_t u = nodes[r];
        int inc[2], ni = 0, opp = -1;
        for (int k = 0; k < 3; k++) {
            if (touches(tr[k], u)) inc[ni++] = k;
            else opp = k;
        }
        const edge *ei = tr[inc[0]], *ej = tr[inc[1]], *ek = tr[opp];
        const int32_t v = ei->s == u ? ei->d : ei->s;
        const int type = opp < inc[0] ? T_I : (opp < inc[1] ? T_II : T_III);
        TRI(type, dir_wrt(ei, u), dir_wrt(ej, u), dir_wrt(ek, v))++;
    }
}

/* Every triple e1 < e2 < e3 (total order) with t3 - t1 <= delta. */
int orc_brute(int64_t m, const int32_t *src, const int32_t *dst, const int64_t *t, int64_t delta,
              uint64_t *star, uint64_t *pair, uint64_t *tri) {
    if (delta < 0 || m < 0) return -1;
    edge *E = sorted_edges(m, src, dst, t);
    if (!E) return -2;
    for (int64_t a = 0; a < m; a++)
        for (int64_t b = a + 1; b < m && E[b].t - E[a].t <= delta; b++)
            for (int64_t c = b + 1; c < m && E[c].t - E[a].t <= delta; c++)
                classify_triple(&E[a], &E[b], &E[c], star, pair, tri);
    free(E);
    return 0;
}

/* ---------------------------------------------------- the 36 classes */

/* Output layout out[i][j] = M_(i+1)(j+1). A motif is named by its edge
 * pattern: edges in time order, nodes numbered 1, 2, 3 by first appearance
 * (so the first edge is always 1->2). Labels given by the paper: M24 (Sec.
 * IV-A counter example), M63, M46, M65 (Sec. III examples), M25 (Sec. IV-B),
 * M55, M56, M65, M66 (pair isomorphisms); the remaining placements are this
 * project's convention: star rows 1-4 x cols 1-4 and rows 5-6 x cols 1-4,
 * triangles rows 1-4 x cols 5-6, pairs rows 5-6 x cols 5-6. */
static const char *LAYOUT[36] = {
    "12 13 12", "12 13 21", "12 13 13", "12 13 31", "12 13 23", "12 13 32",
    "12 31 12", "12 31 21", "12 31 13", "12 23 32", "12 31 23", "12 31 32",
    "12 31 31", "12 23 12", "12 23 21", "12 23 23", "12 23 13", "12 23 31",
    "12 32 12", "12 32 21", "12 32 23", "12 32 32", "12 32 13", "12 32 31",
    "12 12 13", "12 12 23", "12 12 32", "12 21 13", "12 12 12", "12 21 21",
    "12 21 31", "12 21 23", "12 12 31", "12 21 32", "12 21 12", "12 12 21",
};

void orc_layout(char *codes /* 36 x 16 */) {
    for (int k = 0; k < 36; k++) {
        memset(codes + 16 * k, 0, 16);
        strncpy(codes + 16 * k, LAYOUT[k], 15);
    }
}

/* Canonical code of a time-ordered triple, or -1 if it spans four nodes. */
static int class_of(const edge *x, const edge *y, const edge *z) {
    const edge *tr[3] = {x, y, z};
    int32_t nodes[3];
    int nn = 0;
    char code[16];
    int p = 0;
    for (int k = 0; k < 3; k++) {
        int32_t ends[2] = {tr[k]->s, tr[k]->d};
        for (int q = 0; q < 2; q++) {
            int lab = -1;
            for (int r = 0; r < nn; r++)
                if (nodes[r] == ends[q]) lab = r;
            if (lab < 0) {
                if (nn == 3) return -1;
                nodes[nn] = ends[q];
                lab = nn++;
            }
            code[p++] = (char)('1' + lab);
        }
        code[p++] = k < 2 ? ' ' : '\0';
    }
    for (int c = 0; c < 36; c++)
        if (strcmp(code, LAYOUT[c]) == 0) return c;
    return -2; /* unreachable for 2/3-node triples */
}

int orc_brute_classes(int64_t m, const int32_t *src, const int32_t *dst, const int64_t *t,
                      int64_t delta, uint64_t *out36) {
    if (delta < 0 || m < 0) return -1;
    edge *E = sorted_edges(m, src, dst, t);
    if (!E) return -2;
    int rc = 0;
    for (int64_t a = 0; a < m; a++)
        for (int64_t b = a + 1; b < m && E[b].t - E[a].t <= delta; b++)
            for (int64_t c = b + 1; c < m && E[c].t - E[a].t <= delta; c++) {
                const int k = class_of(&E[a], &E[b], &E[c]);
                if (k >= 0) out36[k]++;
                else if (k == -2) rc = -3;
            }
    free(E);
    return rc;
}

/* Map the 56 counter cells to the 36 classes. Which cells belong to a class
 * is derived here from the definitions, not tabulated: the class's own
 * three-edge pattern (nodes 1,2,3 -> ids 0,1,2, times 0,1,2) is classified by
 * classify_triple, and the cells it lands in are that class's cells (one Star
 * cell; two mirror Pair cells, Sec. IV-A; three Tri cells, one per type,
 * Sec. IV-B). A class count is the value of its first cell; returns the
 * number of classes whose cells disagree (0 when the paper's isomorphism
 * claims hold). */
int orc_merge(const uint64_t *star, const uint64_t *pair, const uint64_t *tri, uint64_t *out36) {
    int bad = 0;
    for (int c = 0; c < 36; c++) {
        edge tr[3];
        for (int k = 0; k < 3; k++) {
            tr[k].t = k;
            tr[k].id = k;
            tr[k].s = LAYOUT[c][3 * k] - '1';
            tr[k].d = LAYOUT[c][3 * k + 1] - '1';
        }
        uint64_t s[24] = {0}, p[8] = {0}, q[24] = {0};
        classify_triple(&tr[0], &tr[1], &tr[2], s, p, q);
        int have = 0;
        uint64_t val = 0;
        for (int k = 0; k < 24; k++)
            if (s[k]) {
                if (have && star[k] != val) bad++;
                if (!have) val = star[k];
                have = 1;
            }
        for (int k = 0; k < 8; k++)
            if (p[k]) {
                if (have && pair[k] != val) bad++;
                if (!have) val = pair[k];
                have = 1;
            }
        for (int k = 0; k < 24; k++)
            if (q[k]) {
                if (have && tri[k] != val) bad++;
                if (!have) val = tri[k];
                have = 1;
            }
        out36[c] = val;
    }
    return bad;
}

/* The cells of class c (for tests): writes 1 into each cell of the class. */
void orc_class_cells(int c, uint64_t *star, uint64_t *pair, uint64_t *tri) {
    edge tr[3];
    for (int k = 0; k < 3; k++) {
        tr[k].t = k;
        tr[k].id = k;
        tr[k].s = LAYOUT[c][3 * k] - '1';
        tr[k].d = LAYOUT[c][3 * k + 1] - '1';
    }
    classify_triple(&tr[0], &tr[1], &tr[2], star, pair, tri);
}
