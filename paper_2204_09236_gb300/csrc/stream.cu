// Incremental counting of an edge stream: batches of edges are appended in
// time order, and each batch adds exactly the motif instances whose last edge
// it contains.
//
// An instance's edges all lie within delta of its last edge (Def. 2), and
// counts are sums over instances, so with T = the appended edges whose
// timestamp is within delta of the batch's first timestamp (the "tail") and
// B = the batch, the instances with their last edge in B are
//   cells(T + B) - cells(T),
// both counted by the library's build and count kernels. Only the edges
// within delta of the last appended timestamp can take part in a later
// instance, so the stream keeps only those on the device.
#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>
#include <vector>

#include "tm_internal.cuh"

namespace tmi {

void build_graph(const int32_t *src, const int32_t *dst, const int64_t *t, int64_t m,
                 cudaStream_t s, DevGraph &g);
void free_graph(DevGraph &g, cudaStream_t s);

namespace {

struct MinMax {
    long long tmin, tmax;
};

__global__ void k_minmax_init(MinMax *r) {
    r->tmin = LLONG_MAX;
    r->tmax = LLONG_MIN;
}

__global__ void k_minmax(const int64_t *__restrict__ t, int64_t k, MinMax *r) {
    long long mn = LLONG_MAX, mx = LLONG_MIN;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k;
         i += (int64_t)gridDim.x * blockDim.x) {
        mn = min(mn, (long long)t[i]);
        mx = max(mx, (long long)t[i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&r->tmin, mn);
        atomicMax(&r->tmax, mx);
    }
}

// Sort keys (t - tmin) and values (batch index) of the batch.
__global__ void k_batch_keys(const int64_t *__restrict__ t, int64_t k, long long tmin,
                             uint64_t *__restrict__ keys, uint64_t *__restrict__ idx) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k;
         i += (int64_t)gridDim.x * blockDim.x) {
        keys[i] = (uint64_t)t[i] - (uint64_t)tmin;
        idx[i] = (uint64_t)i;
    }
}

// out[i] = in[perm[i]] for the three edge arrays.
__global__ void k_gather_edges(const int32_t *__restrict__ s_in, const int32_t *__restrict__ d_in,
                               const int64_t *__restrict__ t_in, const uint64_t *__restrict__ perm,
                               int64_t k, int32_t *__restrict__ s_out, int32_t *__restrict__ d_out,
                               int64_t *__restrict__ t_out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = (int64_t)perm[i];
        s_out[i] = s_in[j];
        d_out[i] = d_in[j];
        t_out[i] = t_in[j];
    }
}

// First index i of the time-ordered t[0, n) with last - t[i] <= delta.
__global__ void k_tail_cut(const int64_t *__restrict__ t, int64_t n, long long last,
                           long long delta, int64_t *cut) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if ((unsigned long long)last - (unsigned long long)t[mid] > (unsigned long long)delta)
            lo = mid + 1;
        else
            hi = mid;
    }
    *cut = lo;
}

int bits_of(uint64_t v) {
    int b = 0;
    while (b < 64 && (v >> b) != 0) b++;
    return b;
}

unsigned grid_of(int64_t n) {
    int64_t b = (n + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 8;
    return (unsigned)std::max<int64_t>(1, std::min(b, cap));
}

template <typename F>
int guard(F &&f) {
    try {
        f();
        return TM_OK;
    } catch (const Error &e) {
        record_error(e.code, e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        record_error(TM_ENOMEM, "host allocation failed");
        return TM_ENOMEM;
    } catch (...) {
        record_error(TM_ECUDA, "unexpected internal error");
        return TM_ECUDA;
    }
}

}  // namespace
}  // namespace tmi

struct tm_stream {
    std::mutex mu;
    int device = 0;
    int64_t delta = 0;
    cudaStream_t s = nullptr;
    // the tail: appended edges with last_t - t <= delta, in (t, edge id) order,
    // at [off, off + len) of the three arrays (one allocation each)
    int32_t *src = nullptr, *dst = nullptr;
    int64_t *t = nullptr;
    int64_t off = 0, len = 0;
    int64_t edges = 0;
    bool any = false;
    int64_t last_t = 0;
    uint64_t cells[56] = {};
};

namespace tmi {
namespace {

// The 56 cells (Tri types I/III filled) of the n edges (device arrays), with
// a graph built and released on stream s.
void count_edges(const int32_t *src, const int32_t *dst, const int64_t *t, int64_t n,
                 int64_t delta, cudaStream_t s, uint64_t out[NCELLS]) {
    std::memset(out, 0, sizeof(uint64_t) * NCELLS);
    if (n == 0) return;
    DevGraph g;
    unsigned long long *dc = nullptr;
    try {
        build_graph(src, dst, t, n, s, g);
        dc = dev_alloc_n<unsigned long long>(NCELLS, s);
        TM_CUDA(cudaMemsetAsync(dc, 0, sizeof(unsigned long long) * NCELLS, s));
        launch_count_parts(g, delta, true, true, dc, s, true);
        TM_CUDA(cudaMemcpyAsync(out, dc, sizeof(uint64_t) * NCELLS, cudaMemcpyDeviceToHost, s));
        TM_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        dev_free(dc, s);
        free_graph(g, s);
        throw;
    }
    dev_free(dc, s);
    free_graph(g, s);
}

void append(tm_stream *st, const int32_t *src, const int32_t *dst, const int64_t *t, int64_t k,
            uint64_t add[NCELLS]) {
    std::memset(add, 0, sizeof(uint64_t) * NCELLS);
    if (k == 0) return;
    const int64_t len = st->len, n = len + k;
    if (n >= (int64_t(1) << 30)) fail(TM_EINVAL, "tm_stream_append: tail + batch must be < 2^30 edges");
    cudaStream_t s = st->s;
    std::vector<void *> scratch;  // released at the end, also on failure
    auto alloc = [&](size_t bytes) {
        void *p = dev_alloc(bytes, s);
        scratch.push_back(p);
        return p;
    };
    int32_t *cs = nullptr, *cd = nullptr;
    int64_t *ct = nullptr;
    try {
        int32_t *bs = static_cast<int32_t *>(alloc(sizeof(int32_t) * k));
        int32_t *bd = static_cast<int32_t *>(alloc(sizeof(int32_t) * k));
        int64_t *bt = static_cast<int64_t *>(alloc(sizeof(int64_t) * k));
        TM_CUDA(cudaMemcpyAsync(bs, src, sizeof(int32_t) * k, cudaMemcpyDefault, s));
        TM_CUDA(cudaMemcpyAsync(bd, dst, sizeof(int32_t) * k, cudaMemcpyDefault, s));
        TM_CUDA(cudaMemcpyAsync(bt, t, sizeof(int64_t) * k, cudaMemcpyDefault, s));
        MinMax *dmm = static_cast<MinMax *>(alloc(sizeof(MinMax)));
        TM_LAUNCH(k_minmax_init, 1, 1, 0, s, dmm);
        TM_LAUNCH(k_minmax, grid_of(k), 256, 0, s, bt, k, dmm);
        MinMax mm;
        TM_CUDA(cudaMemcpyAsync(&mm, dmm, sizeof mm, cudaMemcpyDeviceToHost, s));
        TM_CUDA(cudaStreamSynchronize(s));
        if (st->any && mm.tmin < st->last_t)
            fail(TM_EINVAL, "tm_stream_append: a timestamp is below the last appended timestamp");
        const uint64_t span = (uint64_t)mm.tmax - (uint64_t)mm.tmin;
        if (span > (uint64_t)INT64_MAX) fail(TM_EINVAL, "tm_stream_append: timestamp span overflows");
        // the batch in (t, edge id) order after the tail
        uint64_t *k1 = static_cast<uint64_t *>(alloc(sizeof(uint64_t) * k));
        uint64_t *v1 = static_cast<uint64_t *>(alloc(sizeof(uint64_t) * k));
        uint64_t *k2 = static_cast<uint64_t *>(alloc(sizeof(uint64_t) * k));
        uint64_t *v2 = static_cast<uint64_t *>(alloc(sizeof(uint64_t) * k));
        TM_LAUNCH(k_batch_keys, grid_of(k), 256, 0, s, bt, k, mm.tmin, k1, v1);
        uint64_t *ks, *perm;
        radix_sort_u64_v64(k1, v1, k2, v2, k, std::max(1, bits_of(span)), s, &ks, &perm);
        cs = dev_alloc_n<int32_t>(n, s);
        cd = dev_alloc_n<int32_t>(n, s);
        ct = dev_alloc_n<int64_t>(n, s);
        if (len > 0) {
            TM_CUDA(cudaMemcpyAsync(cs, st->src + st->off, sizeof(int32_t) * len,
                                    cudaMemcpyDeviceToDevice, s));
            TM_CUDA(cudaMemcpyAsync(cd, st->dst + st->off, sizeof(int32_t) * len,
                                    cudaMemcpyDeviceToDevice, s));
            TM_CUDA(cudaMemcpyAsync(ct, st->t + st->off, sizeof(int64_t) * len,
                                    cudaMemcpyDeviceToDevice, s));
        }
        TM_LAUNCH(k_gather_edges, grid_of(k), 256, 0, s, bs, bd, bt, perm, k, cs + len, cd + len,
                  ct + len);
        // the new instances: cells(tail + batch) - cells(tail)
        uint64_t c1[NCELLS], c0[NCELLS];
        count_edges(cs, cd, ct, n, st->delta, s, c1);
        count_edges(cs, cd, ct, len, st->delta, s, c0);
        for (int c = 0; c < NCELLS; c++) add[c] = c1[c] - c0[c];
        // the new tail: the edges within delta of the new last timestamp
        int64_t *dcut = static_cast<int64_t *>(alloc(sizeof(int64_t)));
        TM_LAUNCH(k_tail_cut, 1, 1, 0, s, ct, n, mm.tmax, st->delta, dcut);
        int64_t cut = 0;
        TM_CUDA(cudaMemcpyAsync(&cut, dcut, sizeof cut, cudaMemcpyDeviceToHost, s));
        TM_CUDA(cudaStreamSynchronize(s));
        dev_free(st->src, s);
        dev_free(st->dst, s);
        dev_free(st->t, s);
        st->src = cs;
        st->dst = cd;
        st->t = ct;
        st->off = cut;
        st->len = n - cut;
        st->edges += k;
        st->last_t = mm.tmax;
        st->any = true;
        for (int c = 0; c < NCELLS; c++) st->cells[c] += add[c];
    } catch (...) {
        for (void *p : scratch) dev_free(p, s);
        dev_free(cs, s);
        dev_free(cd, s);
        dev_free(ct, s);
        throw;
    }
    for (void *p : scratch) dev_free(p, s);
}

}  // namespace
}  // namespace tmi

using namespace tmi;

extern "C" {

tm_stream *tm_stream_create(int64_t delta) {
    tm_stream *st = nullptr;
    const int rc = guard([&] {
        if (delta < 0) fail(TM_EINVAL, "tm_stream_create: delta must be >= 0");
        st = new tm_stream();
        st->delta = delta;
        st->device = current_device_id();
        num_sms();  // per-device set-up
        if (cudaStreamCreateWithFlags(&st->s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete st;
            st = nullptr;
            fail(TM_ECUDA, "tm_stream_create: cudaStreamCreateWithFlags failed");
        }
    });
    return rc == TM_OK ? st : nullptr;
}

int tm_stream_append(tm_stream *st, const int32_t *src, const int32_t *dst, const int64_t *t,
                     int64_t k, uint64_t added[56]) {
    return guard([&] {
        if (!st) fail(TM_EINVAL, "NULL stream");
        if (k < 0 || (k > 0 && (!src || !dst || !t))) fail(TM_EINVAL, "tm_stream_append: bad batch");
        std::lock_guard<std::mutex> lk(st->mu);
        if (current_device_id() != st->device) fail(TM_EINVAL, "stream was created on another device");
        uint64_t add[NCELLS];
        append(st, src, dst, t, k, add);
        if (added) std::memcpy(added, add, sizeof add);
    });
}

int tm_stream_counts(tm_stream *st, uint64_t cells[56], uint64_t out[36]) {
    return guard([&] {
        if (!st) fail(TM_EINVAL, "NULL stream");
        std::lock_guard<std::mutex> lk(st->mu);
        if (cells) std::memcpy(cells, st->cells, sizeof st->cells);
        if (out) tm_merge(st->cells, out);
    });
}

int64_t tm_stream_edges(tm_stream *st) {
    if (!st) return -1;
    std::lock_guard<std::mutex> lk(st->mu);
    return st->edges;
}

int64_t tm_stream_tail(tm_stream *st) {
    if (!st) return -1;
    std::lock_guard<std::mutex> lk(st->mu);
    return st->len;
}

void tm_stream_free(tm_stream *st) {
    if (!st) return;
    guard([&] {
        dev_free(st->src, st->s);
        dev_free(st->dst, st->s);
        dev_free(st->t, st->s);
        TM_CUDA(cudaStreamSynchronize(st->s));
    });
    cudaStreamDestroy(st->s);
    delete st;
}

}  // extern "C"
