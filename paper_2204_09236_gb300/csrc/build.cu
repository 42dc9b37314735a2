// tm_build: the device-resident graph.
//
// Steps (on the caller's stream; the entry offsets, in-prefix, link
// initialisation and position scatter of step 4 run on a side stream beside
// the pair sort of step 5, and the hash table is cleared beside the
// insertion records):
//   1. validate ids / self-loops, find n, min t, max t          (k_validate)
//   2. stable radix sort of the edges by t - t_min -> rank order  (ties keep
//      the edge-id order: the (t, edge id) total order); skipped when the
//      input is already in time order
//   3. incident entries of every centre, stable radix sort by centre: S_u in
//      (t, id) order for every u (Table 1; "get S_u" in Alg. 1 and Alg. 2)
//   4. in-count prefix over the entries (cin), entry positions of each edge
//   5. stable radix sort of the edges by node pair: every E_(v,w) (Alg. 2) is
//      a run of the pair list in rank order; a hash maps a pair to its run
//   6. links between consecutive same-neighbour entries of a centre
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "radix.cuh"

namespace tmi {

namespace {

struct Validation {
    int32_t max_id;
    int32_t bad_neg;
    int32_t bad_loop;
    int32_t unsorted;  // some t[e] < t[e-1]: the input is not in time order
    long long tmin;
    long long tmax;
};

__global__ void k_validate(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                           const int64_t *__restrict__ t, int64_t m, Validation *v) {
    int32_t mx = -1, neg = 0, loop = 0, uns = 0;
    long long tmn = LLONG_MAX, tmx = LLONG_MIN;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = src[e], b = dst[e];
        neg |= (a < 0) | (b < 0);
        loop |= a == b;
        mx = max(mx, max(a, b));
        long long x = t[e];
        tmn = min(tmn, x);
        tmx = max(tmx, x);
        if (e > 0) uns |= x < t[e - 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        neg |= __shfl_xor_sync(0xffffffffu, neg, o);
        loop |= __shfl_xor_sync(0xffffffffu, loop, o);
        uns |= __shfl_xor_sync(0xffffffffu, uns, o);
        tmn = min(tmn, __shfl_xor_sync(0xffffffffu, tmn, o));
        tmx = max(tmx, __shfl_xor_sync(0xffffffffu, tmx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&v->max_id, mx);
        if (neg) atomicOr(&v->bad_neg, 1);
        if (loop) atomicOr(&v->bad_loop, 1);
        if (uns) atomicOr(&v->unsorted, 1);
        atomicMin(&v->tmin, tmn);
        atomicMax(&v->tmax, tmx);
    }
}

__global__ void k_validation_init(Validation *v) {
    v->max_id = -1;
    v->bad_neg = 0;
    v->bad_loop = 0;
    v->unsorted = 0;
    v->tmin = LLONG_MAX;
    v->tmax = LLONG_MIN;
}

template <typename K>
__global__ void k_time_keys(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                            const int64_t *__restrict__ t, int64_t m, long long tmin,
                            K *__restrict__ keys, uint64_t *__restrict__ vals) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        keys[e] = (K)((unsigned long long)t[e] - (unsigned long long)tmin);
        vals[e] = ((uint64_t)(uint32_t)src[e] << 32) | (uint32_t)dst[e];
    }
}

// The first pass of the time sort forms its items from the edges in id
// order: key t - t_min, value (src << 32) | dst.
template <typename K>
struct TimeGen {
    static constexpr bool VEC_KEYS = false;
    const int32_t *__restrict__ src;
    const int32_t *__restrict__ dst;
    const int64_t *__restrict__ t;
    long long tmin;
    __device__ __forceinline__ bool valid(int64_t) const { return true; }
    __device__ __forceinline__ K key(int64_t e) const {
        return (K)((unsigned long long)t[e] - (unsigned long long)tmin);
    }
    __device__ __forceinline__ uint64_t val(int64_t e) const {
        return ((uint64_t)(uint32_t)src[e] << 32) | (uint32_t)dst[e];
    }
};

// The incident entries, generated from the edges in rank order as the first
// pass of their sort by centre reads them: entry i = 2 * rank + side of the
// edge of that rank sits at its source (side 0, direction o) or destination
// (side 1, direction in), keyed by that centre and carrying its timestamp, its
// neighbour and (rank << 1) | side.
template <typename TK, typename V>
struct EntryGen {
    static constexpr bool VEC_KEYS = false;
    const TK *__restrict__ tkey;      // t - t_min in rank order
    const uint64_t *__restrict__ sd;  // (src << 32) | dst in rank order
    __device__ __forceinline__ bool valid(int64_t) const { return true; }
    __device__ __forceinline__ uint32_t key(int64_t i) const {
        const uint64_t v = sd[i >> 1];
        return (i & 1) ? (uint32_t)v : (uint32_t)(v >> 32);
    }
    __device__ __forceinline__ V val(int64_t i) const {
        const uint64_t v = sd[i >> 1];
        const uint32_t other = (i & 1) ? (uint32_t)(v >> 32) : (uint32_t)v;
        return V{static_cast<decltype(V::t)>(tkey[i >> 1]), other, (uint32_t)i};
    }
};

// The last pass of the centre sort writes every entry in its final form: the
// entry arrays and its code (rank << 1 | side) for the position scatter and
// the in-prefix.
template <typename V>
struct EntryStore {
    int64_t *__restrict__ tt;
    uint2 *__restrict__ tn;
    int32_t *__restrict__ tc;
    uint32_t *__restrict__ codes;
    __device__ __forceinline__ void store(int64_t p, uint32_t c, const V &q) const {
        tt[p] = (int64_t)q.t;
        tn[p] = make_uint2(q.nbr | ((q.code & 1u) << 31), q.code >> 1);
        tc[p] = (int32_t)c;
        codes[p] = q.code;
    }
};

// The first pass of the pair sort reads the entries and keeps those at the
// smaller endpoint of their edge (one per edge), keyed by the larger one. The
// entries are in (centre, rank) order, so the stable sort yields every node
// pair's edges as one run in rank order.
struct PairGen {
    static constexpr bool VEC_KEYS = false;
    const uint2 *__restrict__ tn;
    const int32_t *__restrict__ tc;
    __device__ __forceinline__ bool valid(int64_t p) const {
        return (uint32_t)tc[p] < (tn[p].x & 0x7fffffffu);
    }
    __device__ __forceinline__ uint32_t key(int64_t p) const { return tn[p].x & 0x7fffffffu; }
    __device__ __forceinline__ PairPayload val(int64_t p) const {
        const uint2 e = tn[p];
        // o at the smaller endpoint: it is the source
        const uint32_t srcmin = (e.x >> 31) ? 0u : 1u;
        return PairPayload{(uint32_t)p | (srcmin << 31), (uint32_t)tc[p], (int32_t)e.y};
    }
};

// off[u] = first position of centre u in the centre-sorted entries.
__global__ void k_offsets(const uint32_t *__restrict__ centre, int64_t n2, int64_t n,
                          int32_t *__restrict__ off) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p <= n2;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lo = p == 0 ? 0 : (int64_t)centre[p - 1] + 1;
        const int64_t hi = p == n2 ? n : (int64_t)centre[p];
        for (int64_t u = lo; u <= hi; u++) off[u] = (int32_t)p;
    }
}

// Entries at the centres of degree >= dmin, summed into *sum (few centres
// pass, so few atomics).
__global__ void k_heavy_entries(const int32_t *__restrict__ off, int64_t n, int64_t dmin,
                                unsigned long long *__restrict__ sum) {
    unsigned long long local = 0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = (int64_t)off[u + 1] - off[u];
        if (d >= dmin) local += (unsigned long long)d;
    }
    if (local) atomicAdd(sum, local);
}

// pos_src / pos_dst[rank] = position of the edge's entry at its source /
// destination, for the ranks in [rlo, rhi) only. The build runs this once per
// rank range whose part of the two arrays fits in L2, so the random 4-byte
// stores merge in L2 instead of each costing a DRAM read-modify-write. The
// codes stream in 128-bit loads, two per thread at a time, so that enough of
// them are in flight to keep DRAM busy.
__device__ __forceinline__ void pos_store(uint32_t c, int64_t p, uint32_t rlo, uint32_t rhi,
                                          int32_t *__restrict__ pos_src,
                                          int32_t *__restrict__ pos_dst) {
    const uint32_t r = c >> 1;
    if (r >= rlo && r < rhi) {
        if (c & 1u) pos_dst[r] = (int32_t)p;
        else pos_src[r] = (int32_t)p;
    }
}

__global__ void k_pos_scatter(const uint32_t *__restrict__ codes, int64_t n2, uint32_t rlo,
                              uint32_t rhi, int32_t *__restrict__ pos_src,
                              int32_t *__restrict__ pos_dst) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    // whole uint4 groups of codes (none if the array is not 16-byte aligned)
    const int64_t nv = (reinterpret_cast<uintptr_t>(codes) & 15) ? 0 : n2 / 4;
    const uint4 *cv = reinterpret_cast<const uint4 *>(codes);
    for (int64_t v = tid; v < nv; v += 2 * nthreads) {
        // streamed: evict first, keep L2 for the stores
        const uint4 a = __ldcs(cv + v);
        const bool two = v + nthreads < nv;
        const uint4 b = two ? __ldcs(cv + v + nthreads) : make_uint4(0, 0, 0, 0);
        const int64_t pa = 4 * v, pb = 4 * (v + nthreads);
        pos_store(a.x, pa, rlo, rhi, pos_src, pos_dst);
        pos_store(a.y, pa + 1, rlo, rhi, pos_src, pos_dst);
        pos_store(a.z, pa + 2, rlo, rhi, pos_src, pos_dst);
        pos_store(a.w, pa + 3, rlo, rhi, pos_src, pos_dst);
        if (two) {
            pos_store(b.x, pb, rlo, rhi, pos_src, pos_dst);
            pos_store(b.y, pb + 1, rlo, rhi, pos_src, pos_dst);
            pos_store(b.z, pb + 2, rlo, rhi, pos_src, pos_dst);
            pos_store(b.w, pb + 3, rlo, rhi, pos_src, pos_dst);
        }
    }
    for (int64_t p = 4 * nv + tid; p < n2; p += nthreads)
        pos_store(__ldcs(codes + p), p, rlo, rhi, pos_src, pos_dst);
}

// Pair list element k (one edge of the node pair (centre, pkey[k]), in rank
// order): its rank into pl, whether its source is the smaller id, whether it
// starts a new node pair, and the same-neighbour links of its two entries.
// Consecutive edges of one node pair are consecutive same-neighbour entries at
// both of its nodes. Entries whose pair has one edge keep the links of the
// memset (-1, -1); the others get their whole (prev, next) from their own
// element. A warp takes LINK_U groups of 32 consecutive elements at a time
// (the random position reads of all groups in flight together) and passes the
// neighbouring elements' keys and entry positions along with shuffles, across
// group borders too; only the elements just outside its 32 * LINK_U are read
// again.
constexpr int LINK_U = 4;

__device__ __forceinline__ int32_t big_pos(const PairPayload &q, const int32_t *__restrict__ pos_src,
                                           const int32_t *__restrict__ pos_dst) {
    // entry position at the larger endpoint
    return q.srcmin() ? pos_dst[q.rank] : pos_src[q.rank];
}

__global__ void k_pair_links(const uint32_t *__restrict__ pkey, const PairPayload *__restrict__ pp,
                             const int32_t *__restrict__ pos_src,
                             const int32_t *__restrict__ pos_dst, int64_t m, int2 *__restrict__ pl,
                             int32_t *__restrict__ srcmin, int32_t *__restrict__ head,
                             int2 *__restrict__ lk) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    constexpr unsigned FULL = 0xffffffffu;
    for (int64_t base = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * (32 * LINK_U);
         base < m; base += nwarps * (32 * LINK_U)) {
        PairPayload q[LINK_U];
        uint32_t key[LINK_U];
#pragma unroll
        for (int u = 0; u < LINK_U; u++) {
            const int64_t k = base + 32 * u + lane;
            q[u] = PairPayload{};
            key[u] = 0xffffffffu;
            if (k < m) {
                q[u] = pp[k];
                key[u] = pkey[k];
            }
        }
        // the elements just before and after the warp's range
        PairPayload qp{}, qn{};
        uint32_t kp = 0xffffffffu, kn = 0xffffffffu;
        if (lane == 0 && base > 0 && base - 1 < m) {
            qp = pp[base - 1];
            kp = pkey[base - 1];
        }
        const int64_t after = base + 32 * LINK_U;
        if (lane == 31 && after < m) {
            qn = pp[after];
            kn = pkey[after];
        }
        bool same_p[LINK_U], same_n[LINK_U];
        int32_t big[LINK_U];
#pragma unroll
        for (int u = 0; u < LINK_U; u++) {
            const int64_t k = base + 32 * u + lane;
            uint32_t key_p = __shfl_up_sync(FULL, key[u], 1);
            uint32_t cen_p = __shfl_up_sync(FULL, q[u].centre, 1);
            uint32_t key_n = __shfl_down_sync(FULL, key[u], 1);
            uint32_t cen_n = __shfl_down_sync(FULL, q[u].centre, 1);
            // across the group borders: lane 31 of the group before, lane 0 of the one after
            const uint32_t kb = __shfl_sync(FULL, key[u > 0 ? u - 1 : 0], 31);
            const uint32_t cb = __shfl_sync(FULL, q[u > 0 ? u - 1 : 0].centre, 31);
            const uint32_t ka = __shfl_sync(FULL, key[u + 1 < LINK_U ? u + 1 : u], 0);
            const uint32_t ca = __shfl_sync(FULL, q[u + 1 < LINK_U ? u + 1 : u].centre, 0);
            if (lane == 0) {
                key_p = u > 0 ? kb : kp;
                cen_p = u > 0 ? cb : qp.centre;
            }
            if (lane == 31) {
                key_n = u + 1 < LINK_U ? ka : kn;
                cen_n = u + 1 < LINK_U ? ca : qn.centre;
            }
            const bool in = k < m;
            same_p[u] = in && k > 0 && key_p == key[u] && cen_p == q[u].centre;
            same_n[u] = in && k + 1 < m && key_n == key[u] && cen_n == q[u].centre;
            big[u] = (same_p[u] || same_n[u]) ? big_pos(q[u], pos_src, pos_dst) : -1;
        }
        int32_t big_before = -1, big_after = -1;
        if (lane == 0 && same_p[0]) big_before = big_pos(qp, pos_src, pos_dst);
        if (lane == 31 && same_n[LINK_U - 1]) big_after = big_pos(qn, pos_src, pos_dst);
#pragma unroll
        for (int u = 0; u < LINK_U; u++) {
            const int64_t k = base + 32 * u + lane;
            int32_t pos_p = __shfl_up_sync(FULL, (int32_t)q[u].pos(), 1);
            int32_t big_p = __shfl_up_sync(FULL, big[u], 1);
            int32_t pos_n = __shfl_down_sync(FULL, (int32_t)q[u].pos(), 1);
            int32_t big_n = __shfl_down_sync(FULL, big[u], 1);
            const int32_t pb = __shfl_sync(FULL, (int32_t)q[u > 0 ? u - 1 : 0].pos(), 31);
            const int32_t bb = __shfl_sync(FULL, big[u > 0 ? u - 1 : 0], 31);
            const int32_t pa = __shfl_sync(FULL, (int32_t)q[u + 1 < LINK_U ? u + 1 : u].pos(), 0);
            const int32_t ba = __shfl_sync(FULL, big[u + 1 < LINK_U ? u + 1 : u], 0);
            if (lane == 0) {
                pos_p = u > 0 ? pb : (int32_t)qp.pos();
                big_p = u > 0 ? bb : big_before;
            }
            if (lane == 31) {
                pos_n = u + 1 < LINK_U ? pa : (int32_t)qn.pos();
                big_n = u + 1 < LINK_U ? ba : big_after;
            }
            if (k >= m) continue;
            pl[k].x = q[u].rank;
            srcmin[k] = (int32_t)q[u].srcmin();
            head[k] = same_p[u] ? 0 : 1;
            if (same_p[u] || same_n[u]) {
                lk[q[u].pos()] = make_int2(same_p[u] ? pos_p : -1, same_n[u] ? pos_n : -1);
                lk[big[u]] = make_int2(same_p[u] ? big_p : -1, same_n[u] ? big_n : -1);
            }
        }
    }
}

__global__ void k_pair_cum(const int32_t *__restrict__ cum, int64_t m, int2 *__restrict__ pl) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= m;
         k += (int64_t)gridDim.x * blockDim.x) {
        pl[k].y = cum[k];
        if (k == m) pl[k].x = INT_MAX;
    }
}

__global__ void k_run_begins(const int32_t *__restrict__ head, const int32_t *__restrict__ run_id,
                             int64_t m, int32_t *__restrict__ run_begin) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (head[k]) run_begin[run_id[k]] = (int32_t)k;
    }
}

// One insertion record per node pair (a single-edge pair keeps its edge:
// begin = -(rank + 1), end = source-is-min), keyed by the slot region it
// hashes to; also sets the pair's bits in the Bloom filter.
__global__ void k_hash_records(const int32_t *__restrict__ run_begin, int64_t nruns, int64_t m,
                               const uint32_t *__restrict__ pkey,
                               const PairPayload *__restrict__ pp, uint32_t mask, int region_shift,
                               uint32_t *__restrict__ region, HashRecord *__restrict__ rec,
                               unsigned long long *__restrict__ bloom, uint32_t bloom_mask) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nruns;
         j += (int64_t)gridDim.x * blockDim.x) {
        int32_t b = run_begin[j];
        int32_t e = j + 1 < nruns ? run_begin[j + 1] : (int32_t)m;
        const PairPayload q = pp[b];
        const uint64_t key = pair_key(q.centre, pkey[b]);
        uint32_t word;
        const uint64_t bits = bloom_bits(key, bloom_mask, &word);
        atomicOr(&bloom[word], (unsigned long long)bits);
        if (e - b == 1) {
            b = -(q.rank + 1);
            e = (int32_t)q.srcmin();
        }
        region[j] = (hash_pair(key) & mask) >> region_shift;
        rec[j] = HashRecord{key, b, e};
    }
}

// Inserts the records of one slot region ([start[r], start[r+1]) of the
// region-sorted records): the region's part of the table stays in L2 while
// its random compare-and-swaps run.
__global__ void k_hash_insert(const HashRecord *__restrict__ rec, const int32_t *__restrict__ start,
                              int r, PairSlot *__restrict__ H, uint32_t mask) {
    const int32_t lo = start[r], hi = start[r + 1];
    for (int64_t j = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < hi;
         j += (int64_t)gridDim.x * blockDim.x) {
        const HashRecord q = rec[j];
        uint32_t h = hash_pair(q.key) & mask;
        for (uint32_t probe = 0; probe <= mask; probe++) {
            unsigned long long prev =
                atomicCAS((unsigned long long *)&H[h].key, (unsigned long long)EMPTY_KEY,
                          (unsigned long long)q.key);
            if (prev == EMPTY_KEY) {
                H[h].begin = q.begin;
                H[h].end = q.end;
                break;
            }
            h = (h + 1) & mask;
        }
    }
}

int bits_for(uint64_t maxval) {
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) b++;
    return b;
}

unsigned grid_for(int64_t n, int threads = 256) {
    int64_t blocks = (n + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms() * 16;
    if (blocks > cap) blocks = cap;
    return (unsigned)(blocks > 0 ? blocks : 1);
}

// Host-to-device copies of n pieces (destination, source, bytes) spread over
// s and three upload streams of the current device; s waits for all of them.
// The destinations were allocated in s's order, so the upload streams first
// wait for s.
template <typename D, typename H, typename B>
void upload(size_t n, D dst_of, H src_of, B bytes_of, cudaStream_t s) {
    static std::mutex mu;
    static cudaStream_t aux[64][3] = {};
    const int dev = current_device_id();
    cudaStream_t up[3] = {nullptr, nullptr, nullptr};
    if (dev >= 0 && dev < 64) {
        std::lock_guard<std::mutex> lk(mu);
        for (int k = 0; k < 3; k++) {
            if (!aux[dev][k]) TM_CUDA(cudaStreamCreateWithFlags(&aux[dev][k], cudaStreamNonBlocking));
            up[k] = aux[dev][k];
        }
    }
    cudaEvent_t fork, join[3];
    TM_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    for (int k = 0; k < 3; k++) TM_CUDA(cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming));
    TM_CUDA(cudaEventRecord(fork, s));
    bool used[3] = {false, false, false};
    for (size_t i = 0; i < n; i++) {
        const int k = (int)(i % 4) - 1;  // piece 0 on s, the others on the upload streams
        cudaStream_t st = (k < 0 || !up[k]) ? s : up[k];
        if (st != s && !used[k]) {
            TM_CUDA(cudaStreamWaitEvent(st, fork, 0));
            used[k] = true;
        }
        TM_CUDA(cudaMemcpyAsync(dst_of(i), src_of(i), bytes_of(i), cudaMemcpyHostToDevice, st));
    }
    for (int k = 0; k < 3; k++)
        if (used[k]) {
            TM_CUDA(cudaEventRecord(join[k], up[k]));
            TM_CUDA(cudaStreamWaitEvent(s, join[k], 0));
        }
    cudaEventDestroy(fork);
    for (int k = 0; k < 3; k++) cudaEventDestroy(join[k]);
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Streams of the current device for build work that runs beside s: a pool
// of four per device, taken in turn, created on first use.
cudaStream_t side_stream() {
    static std::mutex mu;
    static cudaStream_t pool[64][4] = {};
    static std::atomic<unsigned> turn{0};
    const int dev = current_device_id();
    if (dev < 0 || dev >= 64) return nullptr;
    const unsigned k = turn.fetch_add(1) & 3u;
    std::lock_guard<std::mutex> lk(mu);
    if (!pool[dev][k]) TM_CUDA(cudaStreamCreateWithFlags(&pool[dev][k], cudaStreamNonBlocking));
    return pool[dev][k];
}

// Build work beside s on a side stream st: fork() lets st run after s's work
// so far, join() makes s wait for st's work so far. The destructor joins as
// well, so that on the way out of a failing build nothing that s frees is
// still in use on st.
struct Side {
    cudaStream_t s, st;
    cudaEvent_t ev = nullptr;
    explicit Side(cudaStream_t s_) : s(s_) {
        const cudaStream_t x = side_stream();
        st = x ? x : s;
        TM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    void fork() {
        TM_CUDA(cudaEventRecord(ev, s));
        TM_CUDA(cudaStreamWaitEvent(st, ev, 0));
    }
    void join() {
        TM_CUDA(cudaEventRecord(ev, st));
        TM_CUDA(cudaStreamWaitEvent(s, ev, 0));
    }
    // join() without error checks, for the way out of a failing build
    void join_quiet() {
        cudaEventRecord(ev, st);
        cudaStreamWaitEvent(s, ev, 0);
    }
    ~Side() {
        join_quiet();
        cudaEventDestroy(ev);
    }
    Side(const Side &) = delete;
    Side &operator=(const Side &) = delete;
};

void build_pairs(DevGraph &g, int nb, Side &side, cudaStream_t s) {
    const int64_t m = g.m, n2 = 2 * m;
    uint32_t *k1 = dev_alloc_n<uint32_t>(m, s), *k2 = dev_alloc_n<uint32_t>(m, s);
    PairPayload *v1 = dev_alloc_n<PairPayload>(m, s), *v2 = dev_alloc_n<PairPayload>(m, s);
    // the last pass writes the pair not read by it (see radix::sort)
    const int passes = nb > 8 ? (nb + 7) / 8 : 1;
    uint32_t *sk = passes & 1 ? k1 : k2;
    PairPayload *sv = passes & 1 ? v1 : v2;
    radix::sort<uint32_t, PairPayload>(PairGen{g.tn, g.tc},
                                       radix::ArrayOut<uint32_t, PairPayload>{sk, sv}, k1, v1, k2,
                                       v2, n2, m, nb, s);

    int32_t *srcmin = dev_alloc_n<int32_t>(m, s);
    int32_t *head = dev_alloc_n<int32_t>(m, s);
    int32_t *run_id = dev_alloc_n<int32_t>(m + 1, s);
    int32_t *cum = dev_alloc_n<int32_t>(m + 1, s);
    side.join();  // off, cin, the links' initial value and the positions
    TM_LAUNCH(k_pair_links, grid_for(m), 256, 0, s, sk, sv, g.pos_src, g.pos_dst, m, g.pl, srcmin,
              head, g.lk);
    // the source-is-min prefix of the pair list beside the run ids
    side.fork();
    exclusive_scan_i32(srcmin, cum, m, side.st);
    TM_LAUNCH(k_pair_cum, grid_for(m + 1), 256, 0, side.st, cum, m, g.pl);
    dev_free(cum, side.st);
    dev_free(srcmin, side.st);
    exclusive_scan_i32(head, run_id, m, s);
    int32_t nruns = 0;
    TM_CUDA(cudaMemcpyAsync(&nruns, run_id + m, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    TM_CUDA(cudaStreamSynchronize(s));
    uint64_t cap = 16;
    while (cap < 2ull * (uint64_t)nruns) cap <<= 1;
    g.hash = dev_alloc_n<PairSlot>((int64_t)cap, s);
    g.hash_mask = (uint32_t)(cap - 1);
    // the table is cleared beside the insertion records
    side.fork();
    TM_CUDA(cudaMemsetAsync(g.hash, 0xff, sizeof(PairSlot) * cap, side.st));
    // about 8 filter bits per pair, at most 2^22 words (32 MB)
    uint64_t words = 128;
    while (words < (uint64_t)nruns / 8 && words < (1ull << 22)) words <<= 1;
    g.bloom = dev_alloc_n<uint64_t>((int64_t)words, s);
    g.bloom_mask = (uint32_t)(words - 1);
    TM_CUDA(cudaMemsetAsync(g.bloom, 0, sizeof(uint64_t) * words, s));
    int32_t *run_begin = dev_alloc_n<int32_t>(nruns + 1, s);
    TM_LAUNCH(k_run_begins, grid_for(m), 256, 0, s, head, run_id, m, run_begin);
    // regions of 2^22 slots (64 MB of table): insertion records are grouped
    // by region with one radix pass, then inserted one region at a time
    int cap_bits = 0;
    while ((1ull << cap_bits) < cap) cap_bits++;
    const int region_shift = cap_bits > 22 ? 22 : cap_bits;
    const int nregions = 1 << (cap_bits - region_shift);
    uint32_t *rk1 = dev_alloc_n<uint32_t>(nruns, s), *rk2 = dev_alloc_n<uint32_t>(nruns, s);
    HashRecord *rv1 = dev_alloc_n<HashRecord>(nruns, s), *rv2 = dev_alloc_n<HashRecord>(nruns, s);
    int32_t *rstart = dev_alloc_n<int32_t>(nregions + 1, s);
    TM_LAUNCH(k_hash_records, grid_for(nruns), 256, 0, s, run_begin, (int64_t)nruns, m, sk, sv,
              g.hash_mask, region_shift, rk1, rv1, (unsigned long long *)g.bloom, g.bloom_mask);
    uint32_t *rks;
    HashRecord *rvs;
    radix_sort_u32_rec(rk1, rv1, rk2, rv2, nruns, bits_for((uint64_t)(nregions - 1)), s, &rks, &rvs);
    TM_LAUNCH(k_offsets, grid_for((int64_t)nruns + 1), 256, 0, s, rks, (int64_t)nruns,
              (int64_t)nregions, rstart);
    side.join();
    for (int r = 0; r < nregions; r++)
        TM_LAUNCH(k_hash_insert, grid_for((int64_t)nruns / nregions + 1), 256, 0, s, rvs, rstart, r,
                  g.hash, g.hash_mask);
    dev_free(rk1, s);
    dev_free(rk2, s);
    dev_free(rv1, s);
    dev_free(rv2, s);
    dev_free(rstart, s);
    dev_free(run_begin, s);
    dev_free(run_id, s);
    dev_free(head, s);
    dev_free(k1, s);
    dev_free(k2, s);
    dev_free(v1, s);
    dev_free(v2, s);
}

// Sorts the edges by t - t_min (stable: ties keep the edge-id order), then
// sorts their 2m incident entries by centre (stable: each S_u stays in rank
// order): the first pass of the second sort generates the entries from the
// rank-ordered edges, its last pass writes the entry arrays of g, the entry
// codes. Then off, cin and the position arrays. Scratch buffers
// (and, through release_inputs, the edge arrays) are released as soon as the
// kernels after them no longer read them.
// Input already in time order (t non-decreasing along the edge ids, as
// temporal-graph files usually come): its order is the (t, edge id) order, so
// the time sort is skipped.
template <typename K, typename Release>
void sort_edges_and_entries(const int32_t *src, const int32_t *dst, const int64_t *t, DevGraph &g,
                            int keybits, int nbits, bool time_ordered, Release release_inputs,
                            Side &side, uint64_t **rank_sd, unsigned long long *heavy,
                            cudaStream_t s) {
    const int64_t m = g.m, n2 = 2 * m, n = g.n;
    K *sk;
    uint64_t *sv;
    K *k1 = dev_alloc_n<K>(m, s);
    uint64_t *v1 = dev_alloc_n<uint64_t>(m, s);
    {
        PhaseTimer pt(TM_PH_TIME_SORT, s);
        if (time_ordered) {
            TM_LAUNCH(k_time_keys<K>, grid_for(m), 256, 0, s, src, dst, t, m, (long long)g.tmin,
                      k1, v1);
            sk = k1;
            sv = v1;
        } else {
            // the first pass reads the edge arrays themselves; the last writes
            // the pair it does not read (see radix::sort)
            K *k2 = dev_alloc_n<K>(m, s);
            uint64_t *v2 = dev_alloc_n<uint64_t>(m, s);
            const int passes = keybits > 8 ? (keybits + 7) / 8 : 1;
            sk = passes & 1 ? k1 : k2;
            sv = passes & 1 ? v1 : v2;
            radix::sort<K, uint64_t>(TimeGen<K>{src, dst, t, (long long)g.tmin},
                                     radix::ArrayOut<K, uint64_t>{sk, sv}, k1, v1, k2, v2, m, m,
                                     keybits, s);
            // the pair not holding the result is free now
            dev_free(sk == k1 ? k2 : k1, s);
            dev_free(sv == v1 ? v2 : v1, s);
        }
        release_inputs();
    }
    *rank_sd = sv;  // the rank-ordered (src, dst) words: the caller keeps or frees them
    PhaseTimer pt(TM_PH_INCIDENT, s);
    uint32_t *codes = dev_alloc_n<uint32_t>(n2, s);
    // a 32-bit time key travels as a 32-bit timestamp
    using V = std::conditional_t<sizeof(K) == 4, EntryPayload32, EntryPayload>;
    using radix::ArrayIn;
    using radix::ArrayOut;
    const EntryGen<K, V> gen{sk, sv};
    const EntryStore<V> out{g.tt, g.tn, g.tc, codes};
    const int passes = nbits > 8 ? (nbits + 7) / 8 : 1;
    const int64_t ntiles = (n2 + radix::Cfg<uint32_t, V>::TILE - 1) / radix::Cfg<uint32_t, V>::TILE;
    int32_t *hist = dev_alloc_n<int32_t>(radix::RADIX * ntiles + 1, s);
    if (passes == 1) {
        radix::pass<uint32_t, V>(gen, out, n2, 0, hist, s);
        dev_free(sk, s);
    } else {
        uint32_t *ka = dev_alloc_n<uint32_t>(n2, s);
        V *va = dev_alloc_n<V>(n2, s);
        radix::pass<uint32_t, V>(gen, ArrayOut<uint32_t, V>{ka, va}, n2, 0, hist, s);
        dev_free(sk, s);
        for (int p = 1; p + 1 < passes; p++) {
            uint32_t *kb = dev_alloc_n<uint32_t>(n2, s);
            V *vb = dev_alloc_n<V>(n2, s);
            radix::pass<uint32_t, V>(ArrayIn<uint32_t, V>{ka, va}, ArrayOut<uint32_t, V>{kb, vb}, n2,
                                     8 * p, hist, s);
            dev_free(ka, s);
            dev_free(va, s);
            ka = kb;
            va = vb;
        }
        radix::pass<uint32_t, V>(ArrayIn<uint32_t, V>{ka, va}, out, n2, 8 * (passes - 1), hist, s);
        dev_free(ka, s);
        dev_free(va, s);
    }
    dev_free(hist, s);
    // the rest runs beside the pair sort, which reads only tn and tc
    side.fork();
    const cudaStream_t ss = side.st;
    TM_LAUNCH(k_offsets, grid_for(n2 + 1), 256, 0, ss, reinterpret_cast<const uint32_t *>(g.tc),
              n2, n, g.off);
    // how concentrated the entries are: those at centres holding 1/64 of them or more
    TM_LAUNCH(k_heavy_entries, grid_for(n), 256, 0, ss, g.off, n, std::max<int64_t>(1, n2 / 64),
              heavy);
    exclusive_scan_low_bit(codes, g.cin, n2, ss);
    TM_CUDA(cudaMemsetAsync(g.lk, 0xff, sizeof(int2) * n2, ss));
    // both position arrays take 8 bytes per rank: at most 64 MB of them per pass
    const int64_t ranks_per_pass = (int64_t)8 << 20;
    for (int64_t rlo = 0; rlo < m; rlo += ranks_per_pass)
        TM_LAUNCH(k_pos_scatter, grid_for(n2), 256, 0, ss, codes, n2, (uint32_t)rlo,
                  (uint32_t)std::min<int64_t>(m, rlo + ranks_per_pass), g.pos_src, g.pos_dst);
    dev_free(codes, ss);
}

}  // namespace

void free_graph(DevGraph &g, cudaStream_t s) {
    dev_free(g.tt, s);
    dev_free(g.tn, s);
    dev_free(g.tc, s);
    dev_free(g.cin, s);
    dev_free(g.lk, s);
    dev_free(g.off, s);
    dev_free(g.pos_src, s);
    dev_free(g.pos_dst, s);
    dev_free(g.sd, s);
    dev_free(g.pl, s);
    dev_free(g.hash, s);
    dev_free(g.bloom, s);
    g = DevGraph();
}

// Builds g from host or device arrays on stream s. Throws Error.
void build_graph(const int32_t *src_in, const int32_t *dst_in, const int64_t *t_in, int64_t m,
                 cudaStream_t s, DevGraph &g) {
    if (m < 0 || m >= (int64_t(1) << 30)) fail(TM_EINVAL, "tm_build: m must be in [0, 2^30)");
    if (m > 0 && (!src_in || !dst_in || !t_in))
        fail(TM_EINVAL, "tm_build: NULL edge array with m > 0");
    g = DevGraph();
    g.m = m;
    const int32_t *src = src_in, *dst = dst_in;
    const int64_t *t = t_in;
    int32_t *h_src = nullptr, *h_dst = nullptr;
    int64_t *h_t = nullptr;
    if (m > 0) {
        // host arrays are copied in (device arrays are read in place): the
        // pieces go out on s and the three upload streams at once, so several
        // copy engines share the upload, and s waits for all of them
        struct Piece {
            void *d;
            const void *h;
            size_t bytes;
        };
        std::vector<Piece> pieces;
        if (!is_device_ptr(src_in)) {
            h_src = dev_alloc_n<int32_t>(m, s);
            pieces.push_back({h_src, src_in, sizeof(int32_t) * m});
            src = h_src;
        }
        if (!is_device_ptr(dst_in)) {
            h_dst = dev_alloc_n<int32_t>(m, s);
            pieces.push_back({h_dst, dst_in, sizeof(int32_t) * m});
            dst = h_dst;
        }
        if (!is_device_ptr(t_in)) {
            h_t = dev_alloc_n<int64_t>(m, s);
            const size_t half = sizeof(int64_t) * (m / 2);
            pieces.push_back({h_t, t_in, half});
            pieces.push_back({reinterpret_cast<char *>(h_t) + half,
                              reinterpret_cast<const char *>(t_in) + half,
                              sizeof(int64_t) * m - half});
        }
        upload(pieces.size(), [&](size_t i) { return pieces[i].d; },
               [&](size_t i) { return pieces[i].h; }, [&](size_t i) { return pieces[i].bytes; },
               s);
        if (h_t) t = h_t;
    }
    auto release_inputs = [&]() {
        if (h_src) dev_free(h_src, s);
        if (h_dst) dev_free(h_dst, s);
        if (h_t) dev_free(h_t, s);
        h_src = h_dst = nullptr;
        h_t = nullptr;
    };

    Validation hv;
    {
        PhaseTimer pt(TM_PH_VALIDATE, s);
        Validation *dv = dev_alloc_n<Validation>(1, s);
        TM_LAUNCH(k_validation_init, 1, 1, 0, s, dv);
        if (m > 0) TM_LAUNCH(k_validate, grid_for(m), 256, 0, s, src, dst, t, m, dv);
        TM_CUDA(cudaMemcpyAsync(&hv, dv, sizeof(hv), cudaMemcpyDeviceToHost, s));
        TM_CUDA(cudaStreamSynchronize(s));
        dev_free(dv, s);
    }
    if (hv.bad_neg || hv.bad_loop) {
        release_inputs();
        fail(TM_EINVAL, hv.bad_neg ? "tm_build: negative node id" : "tm_build: self-loop (src == dst)");
    }
    const int64_t n = (int64_t)hv.max_id + 1;
    g.n = (int32_t)n;
    uint64_t span = 0;
    if (m > 0) {
        span = (uint64_t)hv.tmax - (uint64_t)hv.tmin;
        if (span > (uint64_t)INT64_MAX) {
            release_inputs();
            fail(TM_EINVAL, "tm_build: max(t) - min(t) does not fit in int64");
        }
        g.tmin = hv.tmin;
    }

    g.off = dev_alloc_n<int32_t>(n + 1, s);
    g.tt = dev_alloc_n<int64_t>(2 * m, s);
    g.tn = dev_alloc_n<uint2>(2 * m, s);
    g.tc = dev_alloc_n<int32_t>(2 * m, s);
    g.cin = dev_alloc_n<int32_t>(2 * m + 1, s);
    g.lk = dev_alloc_n<int2>(2 * m, s);
    g.pos_src = dev_alloc_n<int32_t>(m, s);
    g.pos_dst = dev_alloc_n<int32_t>(m, s);
    g.pl = dev_alloc_n<int2>(m + 1, s);
    if (m == 0) {
        TM_CUDA(cudaMemsetAsync(g.off, 0, sizeof(int32_t) * (n + 1), s));
        TM_CUDA(cudaMemsetAsync(g.cin, 0, sizeof(int32_t), s));
        TM_CUDA(cudaMemsetAsync(g.pl, 0, sizeof(int2), s));
        g.hash = dev_alloc_n<PairSlot>(16, s);
        g.hash_mask = 15;
        TM_CUDA(cudaMemsetAsync(g.hash, 0xff, sizeof(PairSlot) * 16, s));
        g.bloom = dev_alloc_n<uint64_t>(128, s);
        g.bloom_mask = 127;
        TM_CUDA(cudaMemsetAsync(g.bloom, 0, sizeof(uint64_t) * 128, s));
        TM_CUDA(cudaStreamSynchronize(s));
        return;
    }

    // 2-4. rank order, then S_u for every centre
    const int keybits = bits_for(span);
    const int nbits = bits_for((uint64_t)(n - 1));
    const bool time_ordered = hv.unsorted == 0;
    Side side(s);
    uint64_t *rank_sd = nullptr;
    unsigned long long *heavy = dev_alloc_n<unsigned long long>(1, s);
    TM_CUDA(cudaMemsetAsync(heavy, 0, sizeof(unsigned long long), s));
    try {
        if (keybits <= 32)
            sort_edges_and_entries<uint32_t>(src, dst, t, g, keybits, nbits, time_ordered,
                                             release_inputs, side, &rank_sd, heavy, s);
        else
            sort_edges_and_entries<uint64_t>(src, dst, t, g, keybits, nbits, time_ordered,
                                             release_inputs, side, &rank_sd, heavy, s);

        // 5-6. pair list, same-neighbour links, hash
        {
            PhaseTimer pt(TM_PH_PAIRS, s);
            build_pairs(g, nbits, side, s);
        }
    } catch (...) {
        side.join_quiet();
        dev_free(rank_sd, s);
        dev_free(heavy, s);
        throw;
    }
    side.join();
    unsigned long long hh = 0;
    TM_CUDA(cudaMemcpyAsync(&hh, heavy, sizeof hh, cudaMemcpyDeviceToHost, s));
    dev_free(heavy, s);
    TM_CUDA(cudaStreamSynchronize(s));
    // a graph with 15 % or more of its entries at such centres keeps its
    // rank-ordered endpoints, and its Tri jobs are found in rank order
    if (20 * hh >= 3 * (unsigned long long)(2 * m)) g.sd = rank_sd;
    else dev_free(rank_sd, s);
}

}  // namespace tmi
