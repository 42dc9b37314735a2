// Internal declarations of the GB300 temporal-motif library (not installed).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "tm.h"

namespace tmi {

// ---------------------------------------------------------------- errors

struct Error {
    int code;
    std::string msg;
};

[[noreturn]] void fail(int code, const std::string &msg);
[[noreturn]] void cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define TM_CUDA(call)                                                                  \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) ::tmi::cuda_fail(e_, #call, __FILE__, __LINE__);       \
    } while (0)

// Every kernel launch of the library goes through TM_LAUNCH so that launch
// errors are caught at the call site and launches are counted.
extern std::atomic<uint64_t> g_launches;
#define TM_LAUNCH(kernel, grid, block, smem, stream, ...)                              \
    do {                                                                               \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                    \
        ::tmi::g_launches.fetch_add(1, std::memory_order_relaxed);                     \
        TM_CUDA(cudaGetLastError());                                                   \
    } while (0)

// Phase timer: records a CUDA event pair around a scope on stream s while
// profiling is enabled (tm_profile_enable).
struct PhaseTimer {
    PhaseTimer(int phase, cudaStream_t s);
    ~PhaseTimer();
    int phase;
    cudaStream_t stream;
    cudaEvent_t start = nullptr;
};

// ------------------------------------------------------------- memory

// Stream-ordered device allocation from the device's default memory pool
// (its release threshold is raised once per device so freed blocks stay
// cached for the next build).
void *dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void *p, cudaStream_t s);

template <typename T>
T *dev_alloc_n(int64_t n, cudaStream_t s) {
    return static_cast<T *>(dev_alloc(sizeof(T) * (size_t)(n > 0 ? n : 1), s));
}

int num_sms();

// ------------------------------------------------------------ graph

// Hash slot: unordered node pair -> its edge list E_(v,w) in the pair list.
// A pair with a single edge keeps that edge in the slot itself:
// begin = -(rank + 1), end = 1 if its source is the smaller id, else 0.
struct PairSlot {
    uint64_t key;  // (smaller id) << 32 | larger id; EMPTY_KEY if unused
    int32_t begin;
    int32_t end;
};
constexpr uint64_t EMPTY_KEY = ~0ull;

// The incident sequences S_u (Table 1: e = (t, v, dir) w.r.t. centre u) of
// all centres, one after the other, each in (t, edge id) order; entry p of
// the whole sequence is spread over the arrays below (structure of arrays,
// 32 bytes per entry), so that every kernel reads only the fields it needs.
struct DevGraph {
    int64_t m = 0;
    int32_t n = 0;
    int64_t tmin = 0;
    int64_t *tt = nullptr;      // 2m: t - t_min
    uint2 *tn = nullptr;        // 2m: {other endpoint v | dir << 31 (0 = o, 1 = in), rank}
    int32_t *tc = nullptr;      // 2m: centre u
    int32_t *cin = nullptr;     // 2m+1: inward entries before p in the whole sequence
    int2 *lk = nullptr;         // 2m: {previous, next} entry of the same centre and
                                //     neighbour, or -1
    int32_t *off = nullptr;     // n+1: S_u = entries [off[u], off[u+1])
    int32_t *pos_src = nullptr; // m, by rank: entry of the edge at its source
    int32_t *pos_dst = nullptr; // m, by rank: entry of the edge at its destination
    // m, by rank: (source << 32) | destination, kept only for a graph whose
    // entries are concentrated on few nodes (its Tri jobs are then found in
    // rank order); null otherwise
    uint64_t *sd = nullptr;
    // pair list, m+1 entries: runs = E_(v,w) (grouped by node pair, ranks
    // ascending); .x = rank of the edge, .y = exclusive prefix over the list of
    // "source is the smaller id" (entry m holds the total).
    int2 *pl = nullptr;
    PairSlot *hash = nullptr;   // open addressing, linear probing
    uint32_t hash_mask = 0;
    // blocked Bloom filter of the node pairs (three bits in one 64-bit word
    // per pair): most join probes ask about pairs that never met, and this
    // filter (at most 32 MB, kept in L2) answers them without touching the hash
    uint64_t *bloom = nullptr;
    uint32_t bloom_mask = 0;
};

// Word index and bit mask of a pair key in the Bloom filter.
__host__ __device__ inline uint64_t bloom_bits(uint64_t key, uint32_t mask, uint32_t *word) {
    uint64_t h = key * 0x9e3779b97f4a7c15ull;
    h ^= h >> 29;
    h *= 0xbf58476d1ce4e5b9ull;
    h ^= h >> 32;
    *word = (uint32_t)h & mask;
    return (1ull << ((h >> 40) & 63)) | (1ull << ((h >> 46) & 63)) | (1ull << ((h >> 52) & 63));
}

__host__ __device__ inline uint64_t pair_key(uint32_t a, uint32_t b) {
    return a < b ? ((uint64_t)a << 32) | b : ((uint64_t)b << 32) | a;
}

__host__ __device__ inline uint32_t hash_pair(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return (uint32_t)k;
}

// ------------------------------------------------------- primitives

// Exclusive prefix sum: out[i] = sum(in[0..i)), out[n] = total (out has n+1
// elements; out == in is allowed when in also has n+1 elements); n >= 0.
void exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s);
// The same over the low bit of each element of `in`.
void exclusive_scan_low_bit(const uint32_t *in, int32_t *out, int64_t n, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of key.
// Sorts `keys`/`vals` of length n using the given scratch buffers of the same
// length; on return the sorted data is in (*keys_out, *vals_out), which is
// either the input or the scratch pair. Key buffers must be 16-byte aligned.
// (Sorts whose first pass generates its items, or whose last pass writes them
// in another form, use the kernels of radix.cuh directly.)
// Payload of an incident entry while it is sorted by centre: everything its
// S_u entry needs, so the entry is written without gathers afterwards.
struct EntryPayload {
    int64_t t;      // t - t_min
    uint32_t nbr;   // the other endpoint
    uint32_t code;  // (rank << 1) | side, side 1 = at the destination (inward)
};
// The same with a 32-bit timestamp, for graphs whose timestamp span fits 32
// bits (12 bytes instead of 16 through every pass of the sort).
struct EntryPayload32 {
    uint32_t t;
    uint32_t nbr;
    uint32_t code;
};
// Payload of an edge while the pair list is sorted: the position of its
// entry at the smaller endpoint with, in bit 31, whether the smaller endpoint
// is its source; that endpoint; the edge's rank.
struct PairPayload {
    uint32_t ps;
    uint32_t centre;
    int32_t rank;
    __host__ __device__ uint32_t pos() const { return ps & 0x7fffffffu; }
    __host__ __device__ uint32_t srcmin() const { return ps >> 31; }
};
// One pair-hash insertion: the pair key and its run (or single edge).
struct HashRecord {
    uint64_t key;
    int32_t begin;
    int32_t end;
};
void radix_sort_u32_rec(uint32_t *keys, HashRecord *vals, uint32_t *keys_tmp, HashRecord *vals_tmp,
                        int64_t n, int bits, cudaStream_t s, uint32_t **keys_out,
                        HashRecord **vals_out);
void radix_sort_u32_pair(uint32_t *keys, PairPayload *vals, uint32_t *keys_tmp,
                         PairPayload *vals_tmp, int64_t n, int bits, cudaStream_t s,
                         uint32_t **keys_out, PairPayload **vals_out);
void radix_sort_u64_v64(uint64_t *keys, uint64_t *vals, uint64_t *keys_tmp, uint64_t *vals_tmp,
                        int64_t n, int bits, cudaStream_t s, uint64_t **keys_out,
                        uint64_t **vals_out);

// --------------------------------------------------------- counting

// Number of 56 raw cells: Star[24] | Pair[8] | Tri[24].
constexpr int NCELLS = 56;

// Adds the counts of entries [begin, end) (as e3 for Star/Pair and as
// e_j for Tri type II) into dev_cells (uint64[56], device). When
// `tri_types_all` is set the Tri type-I/III cells are filled from type II by
// the triangle rotation identity after the whole graph has been counted.
void launch_count(const DevGraph &g, int64_t delta, int32_t begin, int32_t end,
                  unsigned long long *dev_cells, cudaStream_t s);
void launch_fill_tri_types(unsigned long long *dev_cells, cudaStream_t s);

// Only the Star/Pair kernel and/or only the Tri kernel (with its type fill
// unless fill is false), after the window-start pass both of them read. With
// `own` (device int32[n]), only the centres u with own[u] == own_rank are
// counted (a shard of the centres; Tri type II only, fill must be false).
void launch_count_parts(const DevGraph &g, int64_t delta, bool star_pair, bool tri,
                        unsigned long long *dev_cells, cudaStream_t s, bool fill = true,
                        const int32_t *own = nullptr, int32_t own_rank = 0);

// The whole-graph count (Star/Pair, Tri, type-I/III fill) into dev_cells with
// no phase timers and no allocation of any kind.
void launch_count_untimed(const DevGraph &g, int64_t delta, unsigned long long *dev_cells,
                          cudaStream_t s);

// ------------------------------------------------- segmented counting

// One counting segment: the entries [begin, end) of graph g (whole edges:
// both entries of each of its edges lie inside), counted with window delta
// into the 56 device cells at `cells`. Its scratch is indexed from xbase (an
// even number: the sum of the lengths of the segments before it).
struct Segment {
    DevGraph g;
    int64_t delta;
    unsigned long long *cells;
    int32_t begin, end;
    int64_t xbase;
};

// Scratch of a segmented count: window starts (4 B per entry), lists of
// back-active entries (4 B per entry), Tri joins (20 B per edge) and the
// per-segment counters and unit prefixes, carved from one device block.
struct CountScratch {
    int32_t *wl = nullptr;
    int32_t *act = nullptr;
    void *jobs = nullptr;
    int32_t *counts = nullptr;
    int32_t k_cap = 0;
};
size_t count_scratch_bytes(int64_t entries, int32_t k);
void count_scratch_carve(void *base, int64_t entries, int32_t k, CountScratch &sc);

// Entries per warp unit of the streaming count passes on the one-graph path.
constexpr int32_t COUNT_ECHUNK = 512;

// The fast count (window starts, Star/Pair list sweep, Tri jobs and join,
// type-I/III fill) of one segment (`one`, host) or of a device table of
// segments (d_segs; d_meta = {k, prefix over the segments of their units of
// echunk entries, k + 1 values}; k_cap bounds k and sizes the counters).
// Scratch must cover the total entries of the segments. join_blocks_per_sm
// limits the Tri join's occupancy (0: as many as fit); echunk (a multiple of
// 128) is the entries per warp unit of the streaming passes. With a table,
// every launch reads its sizes from device memory, so the sequence can be
// captured in a CUDA graph once and replayed for any table within the
// capacities.
void launch_count_segments(const Segment *one, const Segment *d_segs, const int32_t *d_meta,
                           int32_t k_cap, bool star_pair, bool tri, bool fill,
                           const CountScratch &sc, cudaStream_t s, int join_blocks_per_sm,
                           int32_t echunk, const int32_t *own = nullptr, int32_t own_rank = 0,
                           bool windows_ready = false);

// The counts of one graph for k <= 8 windows deltas[0..k) (ascending) in one
// sweep: one pass finds every entry's k window starts, one walk per listed
// entry gives every window's Star/Pair terms, and the Tri joins run one
// segment per window; window i's 56 cells (Tri types filled) are added into
// dev_cells + 56 i.
void launch_count_multi_delta(const DevGraph &g, const int64_t *deltas, int32_t k,
                              unsigned long long *dev_cells, cudaStream_t s);
int count_join_blocks_per_sm();
// binaryVersion of a library kernel on the current device (e.g. 103).
int kernel_binary_version();

// Read access to a built graph, and error recording, for entry points that
// live outside api.cu.
bool graph_view(const tm_graph *h, const DevGraph **g, int *device);
void record_error(int code, const std::string &msg);
int current_device_id();

}  // namespace tmi

// The opaque handle of include/tm.h. A graph built from several component
// graphs (tm_build_many) keeps where each component's entries start.
struct tm_graph {
    tmi::DevGraph g;
    int device = 0;
    std::vector<int32_t> comp_toff;  // k+1 entry offsets; empty: one component
};
