/*
 * tm.h - exact delta-temporal motif counting on one GB300 (sm_103a).
 *
 * Computes, for a directed temporal multigraph and a window delta, the counts
 * of all 36 two- and three-node, three-edge delta-temporal motifs of
 * arXiv 2204.09236 (Problem 1, Sec. III; motif = Def. 2, instance = Def. 3),
 * through the paper's counters Star[Type,d1,d2,d3] and Pair[d1,d2,d3]
 * (Sec. IV-A) and Tri[Type,di,dj,dk] (Sec. IV-B).
 *
 * Conventions shared by every call:
 *   - An edge is (src[i], dst[i], t[i]); its edge id is the index i.
 *   - Edges are totally ordered by (t, edge id). Def. 2 only asks
 *     t1 <= t2 <= t3; with this order every 3-edge set is counted at most once.
 *     The window test is t3 - t1 <= delta on raw timestamps.
 *   - Direction codes: o (outward from the centre) = 0, in = 1.
 *     Types I/II/III = 0/1/2 (Sec. IV-A star types, Sec. IV-B triangle types).
 *     Flat cell index: Star/Tri ((T*2+a)*2+b)*2+c, Pair (a*2+b)*2+c.
 *   - The 56-cell raw layout is star[24] | pair[8] | tri[24].
 *   - out[36] is row-major out[i][j] = count of M_(i+1)(j+1); tm_layout gives
 *     the edge pattern of each entry.
 *   - Every call returns TM_OK (0) or a negative TM_E* code, and records a
 *     message that tm_last_error() returns (per host thread). Calls that
 *     return a pointer return NULL on error.
 *   - No call falls back to the CPU: without a CUDA device every counting
 *     call fails with TM_ECUDA.
 */
#ifndef TM_H
#define TM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    TM_OK = 0,
    TM_EINVAL = -1,   /* invalid argument or input graph */
    TM_ENOMEM = -2,   /* device allocation failed */
    TM_ECUDA = -3,    /* CUDA runtime error (message names the call) */
    TM_ETIMEOUT = -4, /* a bounded device-side wait gave up */
    TM_EBUDGET = -5   /* request exceeds a memory budget */
};

/* Opaque graph resident in device memory; owns its buffers. */
typedef struct tm_graph tm_graph;

/*
 * Builds the device-resident graph: sorts the edges by (t, edge id), builds
 * every node's incident sequence S_u (Table 1; S_u of Alg. 1 and Alg. 2) and
 * every node pair's edge list E_(v,w) (Alg. 2), with a hash from node pair to
 * list.
 *   src, dst: int32[m] node ids, >= 0, src[i] != dst[i]. n = max id + 1.
 *   t:        int64[m] timestamps; max(t) - min(t) must fit in int64.
 *   m:        number of edges, 0 <= m < 2^30. m == 0 builds an empty graph.
 * The three pointers may be host or device memory (each is classified with
 * cudaPointerGetAttributes); they are read during the call only and may be
 * NULL when m == 0. Runs on the library's own stream and returns after the
 * build has finished. Returns NULL on error (TM_EINVAL for a rejected input:
 * m out of range, NULL pointer, negative id, self-loop, timestamp span
 * overflow; TM_ENOMEM, TM_ECUDA otherwise).
 */
tm_graph *tm_build(const int32_t *src, const int32_t *dst, const int64_t *t, int64_t m);

/* Same as tm_build, enqueued on `stream` (a cudaStream_t; NULL = legacy
 * default stream). Device inputs must be ready in stream order. The call
 * waits for two small device-to-host reads (node count, timestamp range and
 * validation flags, which size the graph's buffers; the number of node pairs,
 * which sizes the hash) and returns once the build's work has finished. Part
 * of that work runs on internal side streams forked from `stream` and joined
 * back into it. */
tm_graph *tm_build_async(const int32_t *src, const int32_t *dst, const int64_t *t, int64_t m,
                         void *stream);

/* Releases the graph's device memory after the library stream has drained.
 * Work that other streams still have queued on the graph must be complete
 * (synchronise them first). NULL-safe. */
void tm_free(tm_graph *g);

/* Releases the graph's device memory in stream order on `stream`: the
 * buffers return to the pool once the work queued before this call on that
 * stream has finished. The handle is invalid on return. NULL-safe. */
void tm_free_async(tm_graph *g, void *stream);

/*
 * Counts all 36 motifs for window delta (>= 0; delta == 0 counts only triples
 * that share one timestamp). out: host uint64[36], row-major 6x6 as above.
 * Synchronous. The graph is not modified; concurrent calls on one graph from
 * several host threads are allowed.
 * Errors: TM_EINVAL (NULL graph/out, delta < 0), TM_ECUDA.
 */
int tm_count(const tm_graph *g, int64_t delta, uint64_t out[36]);

/*
 * The paper's own counters (Sec. IV-A, IV-B) for window delta: star[24] =
 * Star[T][d1][d2][d3], pair[8] = Pair[d1][d2][d3], tri[24] =
 * Tri[T][di][dj][dk], host memory. Synchronous.
 */
int tm_count_raw(const tm_graph *g, int64_t delta, uint64_t star[24], uint64_t pair[8],
                 uint64_t tri[24]);

/*
 * Enqueues the count on `stream` and writes the 56 raw cells (star|pair|tri)
 * to dev_cells, a device uint64[56] owned by the caller. Returns as soon as
 * the work is enqueued; the cells are valid once the stream reaches that
 * point. Must not overlap another count that uses the same dev_cells.
 * Like tm_count, tm_count_raw and tm_count_select, it borrows about 36 bytes
 * per edge of scratch (window starts, the list of entries with Star/Pair
 * terms, the Tri joins) from the device's stream-ordered memory pool for the
 * duration of the count; the batched calls use a slab of their own and
 * tm_count_noalloc uses none.
 */
int tm_count_async(const tm_graph *g, int64_t delta, void *stream, uint64_t *dev_cells);

/*
 * The 56 raw cells of the centres listed in `centres` only (host int32[k],
 * each in [0, n)): their Star and Pair cells (Alg. 1 run at those centres)
 * and their Tri type-II cells (the triangles whose opposite edge is in the
 * middle of the time order, Sec. IV-B). Tri types I and III are left zero.
 * Used to compare single centres against a reference at full graph size.
 */
int tm_count_centres(const tm_graph *g, int64_t delta, const int32_t *centres, int32_t k,
                     uint64_t cells[56]);

/*
 * One shard of the centres (Sec. IV-C: centres are independent, so the
 * counters are sums over centres): the Star and Pair cells and the Tri
 * type-II cells of the centres u with owner[u] == rank, counted by the same
 * kernels as tm_count (its window starts, Star/Pair list and Tri join, each
 * join counting only the triangles centred at an owned endpoint). owner:
 * int32[n] (n = tm_graph_nodes), host or device memory, read during the call.
 * Tri types I and III are left zero: summing the cells of every rank (e.g. one
 * all-reduce of the 56 cells over the ranks of a multi-GPU job, each with the
 * whole graph built) and then tm_fill_tri_types gives tm_count_raw's cells.
 * cells: host uint64[56]. Borrows pool scratch like tm_count plus 4 n bytes.
 */
int tm_count_shard(const tm_graph *g, int64_t delta, const int32_t *owner, int32_t rank,
                   uint64_t cells[56]);

/*
 * Category-selective counting (the per-category variants FAST-Pair /
 * FAST-Tri that the paper times separately, Sec. V-C, Table 3): what =
 * TM_SELECT_STAR_PAIR runs only Algorithm 1's counters (Star and Pair
 * cells), TM_SELECT_TRI only Algorithm 2's (Tri cells), both = all 56.
 * cells: host uint64[56]; the cells of the category not selected are 0.
 */
#define TM_SELECT_STAR_PAIR 1
#define TM_SELECT_TRI 2
int tm_count_select(const tm_graph *g, int64_t delta, int32_t what, uint64_t cells[56]);

/*
 * Counts one graph for k windows deltas[0..k) (any order, repeats allowed);
 * out[i*36 .. i*36+36) as in tm_count. The windows are sorted and counted in
 * sweeps of up to 8: the windows of an entry nest, so one pass finds every
 * entry's window start for all of them, one walk of each entry's
 * same-neighbour links gives every window's Star/Pair terms, and the Tri
 * joins run once per window on those starts. Borrows about 36 bytes per edge
 * and window of pool scratch (one sweep at a time); rejects a negative delta
 * and 2m * 8 >= 2^31 entries in one sweep.
 * The paper's delta sensitivity experiment (Sec. V-E, Fig. 11(a)) is this
 * call over a list of deltas.
 */
int tm_count_multi(const tm_graph *g, const int64_t *deltas, int32_t k, uint64_t *out);

/*
 * Folds 56 raw cells into the 36 classes (out[36] as above) on the host.
 * Returns the number of classes whose isomorphic cells disagree (the pair
 * mirror cells, Sec. IV-A; the three triangle cells of a class, one per
 * type, Sec. IV-B): 0 for any output of this library.
 */
int tm_merge(const uint64_t cells[56], uint64_t out[36]);

/*
 * Fills the Tri type-I and type-III cells of a 56-cell vector (host memory)
 * from its type-II cells: each triangle instance adds one to a type-I, a
 * type-II and a type-III cell of its class (Sec. IV-B counts every instance
 * once per vertex), which gives Tri[II,i,j,k] = Tri[I,!k,!j,!i] =
 * Tri[III,!i,k,j]. Used after summing type-II cells over shards of centres
 * (tm_count_centres, tm_count_shard). Star and Pair cells are not touched.
 * Returns TM_OK, or TM_EINVAL for NULL.
 */
int tm_fill_tri_types(uint64_t cells[56]);

/* Writes the edge pattern of each class, codes[i*6+j] = pattern of
 * M_(i+1)(j+1): edges in time order, nodes 1,2,3 by first appearance, e.g.
 * "12 13 21". Returns TM_OK. */
int tm_layout(char codes[36][16]);

/*
 * Batched counting. Many graphs, each with its own window, are counted
 * together by the same kernels as one graph (window starts, Star/Pair sweep,
 * Tri join), each kernel ONE persistent launch over a table of segments (a
 * segment = one graph, or one component of a tm_build_many graph, or one
 * window of tm_count_multi): its warps or blocks take units of work (entry
 * ranges, listed entries, joins) of one segment at a time from the table in
 * order, the paper's dynamic scheduling over centres (Sec. IV-C) as device
 * work units. The launch sequence (segment table upload, clears, the kernels,
 * the Tri type fill, the cell download) is captured once in a CUDA graph and
 * replayed; only the staged table changes between calls. The scratch of the
 * kernels (18 bytes per incident entry) is a device slab that the call keeps
 * for the next batch and grows (cudaMalloc) only for a batch larger than all
 * before it. Synchronous.
 */

/* Counts gs[i] with window deltas[i] for i < n; out[i*36 .. i*36+36) as in
 * tm_count (host memory). All graphs must be on the current device. */
int tm_count_batch(const tm_graph *const *gs, const int64_t *deltas, int32_t n, uint64_t *out);

/* Builds k graphs as ONE device graph of k components (graph c's node v
 * becomes node base_c + v; its edge ids keep their order), so that all k are
 * sorted and indexed by one pass of the build instead of k small ones.
 * src[c], dst[c], t[c]: arrays of graph c (host or device memory, m[c]
 * entries, same rules as tm_build). Counting the whole result with tm_count
 * gives the sum over the components; tm_count_many counts each component
 * with its own window. Returns NULL on error (as tm_build). */
tm_graph *tm_build_many(int32_t k, const int32_t *const *src, const int32_t *const *dst,
                        const int64_t *const *t, const int64_t *m);

/* Number of components (1 for a graph from tm_build; -1 for NULL). */
int32_t tm_graph_components(const tm_graph *g);

/* Counts each component c of g (tm_build_many) with window deltas[c] in one
 * batched launch; out[c*36 .. c*36+36) as in tm_count. */
int tm_count_many(const tm_graph *g, const int64_t *deltas, uint64_t *out);

/* Batching parameters: entries per warp unit of the streaming passes
 * (rounded down to a multiple of 128, at least 256; 0 keeps the current value)
 * and blocks per SM of the Tri join (0 = as many as fit). */
int tm_batch_config(int64_t item_entries, int32_t blocks_per_sm);
int tm_batch_get_config(int64_t *item_entries, int32_t *blocks_per_sm);

/* Autotuner: times tm_count_many on g with windows deltas (reps timed runs
 * per setting) over units of {256, 512, 1024, 2048} entries and Tri-join
 * blocks per SM {1, ..., max}, checks that every setting gives the same
 * cells, makes the fastest the library's setting and reports it. */
int tm_tune_batch(const tm_graph *g, const int64_t *deltas, int32_t reps,
                  int64_t *best_item_entries, int32_t *best_blocks_per_sm, double *best_ms);

/*
 * Serving loop. A server keeps built graphs resident on the device for
 * repeat queries and counts requests as they arrive: worker threads (each
 * with its own stream) repeatedly take the pending requests that can be
 * admitted now (continuous batching) - re-queries of resident graphs, and
 * new graphs whose estimated device bytes fit in the budget after evicting
 * the least recently used idle graphs - build the new graphs and count the
 * whole wave in one batched launch (tm_count_batch). A request that arrives
 * while waves are on the device joins a later wave as slots and memory free
 * up. Latency = completion minus submission (host clock).
 */
typedef struct tm_server tm_server;

typedef struct {
    int64_t key;          /* caller's key of the graph */
    const int32_t *src;   /* new graph: host arrays of m edges (copied at */
    const int32_t *dst;   /*   submission); a re-query of a resident graph */
    const int64_t *t;     /*   passes NULL and m = 0 */
    int64_t m;
    int64_t n_hint;       /* node count if known (memory estimate), else 0 */
    int64_t delta;        /* window, >= 0 */
} tm_request_desc;

typedef struct {
    int64_t submitted, completed, failed, pending;
    int64_t resident_graphs, resident_bytes, evictions, builds, waves, edges_counted;
    double p50_ms, p99_ms, max_ms; /* latency quantiles of completed requests */
} tm_server_stats_t;

/* budget_bytes: device bytes for resident graphs, builds in progress and the
 * workers' counting scratch (each worker counts its waves in runs of at most
 * budget / (192 * workers) entries, 2^14..2^24, with a slab of 18 bytes per
 * entry that it keeps; a larger graph is counted alone and charges the
 * excess while resident); workers: 1..64 worker threads (streams);
 * max_wave: most requests per wave. NULL on error (TM_EBUDGET when the
 * workers' slabs alone exceed the budget). */
tm_server *tm_server_create(int64_t budget_bytes, int32_t workers, int32_t max_wave);
/* Returns the request id (>= 0) or a negative TM_E* code. A request whose
 * key names a resident graph counts that graph (its edges, if given, are not
 * used). */
int64_t tm_server_submit(tm_server *s, const tm_request_desc *req);
/* TM_OK with out[36] (as tm_count) and the latency when done, 1 while
 * pending, or the request's negative error code (TM_EBUDGET: the graph can
 * never fit the budget; TM_EINVAL: unknown key without edges, bad input). */
int tm_server_poll(tm_server *s, int64_t id, uint64_t out[36], double *latency_ms);
/* As tm_server_poll, waiting up to timeout_s seconds; TM_ETIMEOUT if the
 * request is still pending then. */
int tm_server_wait(tm_server *s, int64_t id, uint64_t out[36], double *latency_ms,
                   double timeout_s);
int tm_server_stats(tm_server *s, tm_server_stats_t *st);
/* The server's admission estimate for a graph of m edges and n nodes: the
 * device bytes it holds while resident, and the extra bytes its build and a
 * count of it alone need at peak (a new graph is admitted when they fit in
 * the budget beside the workers' counting scratch, which the server reserves
 * at creation: about 1/8 of the budget, at most 16M entries per worker). */
int tm_estimate_bytes(int64_t m, int64_t n, int64_t *resident, int64_t *build_scratch);
/* Keys of the resident graphs (up to cap written); returns how many there are. */
int32_t tm_server_resident(tm_server *s, int64_t *keys, int32_t cap);
/* Finishes the queued requests, stops the workers, frees every graph. */
void tm_server_destroy(tm_server *s);

/*
 * Incremental counting of an edge stream. The paper motivates exact counts
 * for frequently updated dynamic systems (Sec. I); a stream keeps the counts
 * of every edge appended so far for one window delta without rebuilding the
 * whole graph. tm_stream_append adds a batch of k edges (host or device
 * arrays as in tm_build) whose timestamps are all >= the last timestamp
 * appended before; edge ids continue from the edges before the batch, so a
 * batch edge is ordered after every earlier edge of equal timestamp, and
 * inside the batch by its index. The batch adds exactly the motif instances
 * whose last edge is in it: every instance lies within delta of its last
 * edge (Def. 2), so they are counted as cells(tail + batch) - cells(tail),
 * where the tail is the appended edges within delta of the last timestamp
 * (the only edges the stream keeps on the device; each of the two graphs is
 * built and counted by the library's kernels). added (host uint64[56], may be
 * NULL) receives the batch's raw cells; the running cells and classes come
 * from tm_stream_counts. A failed append (TM_EINVAL: a timestamp below the
 * last one, bad ids, tail + batch >= 2^30 edges) leaves the stream unchanged.
 * Calls on one stream are serialised.
 */
typedef struct tm_stream tm_stream;
tm_stream *tm_stream_create(int64_t delta);
int tm_stream_append(tm_stream *st, const int32_t *src, const int32_t *dst, const int64_t *t,
                     int64_t k, uint64_t added[56]);
/* Running 56 raw cells and/or 36 classes (either may be NULL). */
int tm_stream_counts(tm_stream *st, uint64_t cells[56], uint64_t out[36]);
/* Edges appended so far / edges kept in the tail (-1 for NULL). */
int64_t tm_stream_edges(tm_stream *st);
int64_t tm_stream_tail(tm_stream *st);
void tm_stream_free(tm_stream *st);

/* Number of nodes / edges of a built graph (-1 for NULL). */
int64_t tm_graph_nodes(const tm_graph *g);
int64_t tm_graph_edges(const tm_graph *g);

/* The compute capability the library's kernels were compiled for, as the
 * CUDA runtime reports it for one of them on the current device
 * (cudaFuncGetAttributes binaryVersion, e.g. 103 for sm_103a). Needs a CUDA
 * device; returns TM_ECUDA without one. */
int tm_kernel_arch(int32_t *arch);

/* Kernels this library has launched in this process so far (all devices). */
uint64_t tm_launch_count(void);

/*
 * Phase timers (tracing). While enabled, the library records a CUDA event
 * pair on the launching stream around each phase below, so a phase's time is
 * its device time on that stream. tm_profile_read waits for the recorded
 * events, adds each phase's elapsed milliseconds into ms[TM_NPHASES] and its
 * number of timed occurrences into calls[TM_NPHASES] (both host arrays,
 * either may be NULL), and clears the record.
 */
enum {
    TM_PH_VALIDATE = 0, /* input upload and validation */
    TM_PH_TIME_SORT,    /* radix sort of the edges by (t, edge id) */
    TM_PH_INCIDENT,     /* S_u for every centre */
    TM_PH_PAIRS,        /* pair lists, pair hash, same-neighbour links */
    TM_PH_STAR_PAIR,    /* the Star/Pair counting kernel */
    TM_PH_TRI,          /* the Tri counting kernel */
    TM_NPHASES
};
void tm_profile_enable(int on);
int tm_profile_read(double ms[], uint64_t calls[]);

/*
 * tm_count_noalloc - counting for callers that cannot allocate. (The paper
 * has no counterpart: this is a deployment entry point of this library.)
 *
 * A serving thread that must stay inside a device-memory budget fixed up
 * front, a process whose allocator is sized and locked, or code that must not
 * risk the implicit synchronisation of cudaMalloc / cudaFree can call this
 * instead of tm_count. It counts the k graphs gs[i] (built earlier with
 * tm_build) for windows deltas[i] and writes out[i*36 .. i*36+36) (host
 * memory, layout as tm_count). It calls no cudaMalloc, cudaFree or other
 * allocating routine: the 56 counter cells of each graph live in a
 * file-scope device array of TM_NOALLOC_MAX_GRAPHS * 56 uint64 (112 KiB),
 * which every device that loads this library holds until the process exits.
 *   - k must be in [0, TM_NOALLOC_MAX_GRAPHS]; larger k returns TM_EINVAL.
 *   - The work is enqueued on `stream` (a cudaStream_t, NULL = legacy default
 *     stream); the call returns after the results are on the host.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture begins.
 *   - Every call uses the same array and clears the slots it uses first;
 *     calls whose work overlaps on the GPU (other host threads, other
 *     streams) race on it and must be serialised by the caller.
 */
#define TM_NOALLOC_MAX_GRAPHS 256
int tm_count_noalloc(const tm_graph *const *gs, const int64_t *deltas, int32_t k, void *stream,
                     uint64_t *out);

/* Message of the last failed call on this host thread; *code (if not NULL)
 * receives its TM_E* code. Never NULL. */
const char *tm_last_error(int *code);

#ifdef __cplusplus
}
#endif

#endif /* TM_H */
