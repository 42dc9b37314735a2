// C-ABI of the library (include/tm.h): argument checks, error codes, the
// library stream and memory pool, and the 56-cell -> 36-class fold.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "tm_internal.cuh"

namespace tmi {

std::atomic<uint64_t> g_launches{0};

namespace {
thread_local int t_err_code = TM_OK;
thread_local std::string t_err_msg = "no error";

void set_error(int code, const std::string &msg) {
    t_err_code = code;
    t_err_msg = msg;
}
}  // namespace

void fail(int code, const std::string &msg) { throw Error{code, msg}; }

void cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    char buf[512];
    std::snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    throw Error{e == cudaErrorMemoryAllocation ? TM_ENOMEM : TM_ECUDA, buf};
}

namespace {
std::mutex g_dev_mu;
bool g_pool_ready[64] = {};
int g_sms[64] = {};

int current_device() {
    int d = 0;
    TM_CUDA(cudaGetDevice(&d));
    return d;
}

void ensure_device_setup(int d) {
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (d < 0 || d >= 64 || g_pool_ready[d]) return;
    cudaMemPool_t pool;
    TM_CUDA(cudaDeviceGetDefaultMemPool(&pool, d));
    uint64_t thr = UINT64_MAX;  // keep freed blocks cached for the next build
    TM_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    TM_CUDA(cudaDeviceGetAttribute(&g_sms[d], cudaDevAttrMultiProcessorCount, d));
    g_pool_ready[d] = true;
}
}  // namespace

namespace {
std::atomic<int> g_profile{0};
std::mutex g_prof_mu;
struct PhaseRec {
    int phase;
    cudaEvent_t a, b;
};
std::vector<PhaseRec> g_prof_recs;
}  // namespace

PhaseTimer::PhaseTimer(int ph, cudaStream_t s) : phase(ph), stream(s) {
    if (!g_profile.load(std::memory_order_relaxed)) return;
    if (cudaEventCreate(&start) != cudaSuccess || cudaEventRecord(start, s) != cudaSuccess) {
        cudaGetLastError();
        start = nullptr;
    }
}

PhaseTimer::~PhaseTimer() {
    if (!start) return;
    cudaEvent_t stop;
    if (cudaEventCreate(&stop) != cudaSuccess || cudaEventRecord(stop, stream) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_recs.push_back({phase, start, stop});
}

int num_sms() {
    int d = current_device();
    ensure_device_setup(d);
    return g_sms[d] > 0 ? g_sms[d] : 1;
}

void *dev_alloc(size_t bytes, cudaStream_t s) {
    ensure_device_setup(current_device());
    void *p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char buf[128];
        std::snprintf(buf, sizeof buf, "device allocation of %zu bytes failed: %s", bytes,
                      cudaGetErrorString(e));
        throw Error{TM_ENOMEM, buf};
    }
    return p;
}

void dev_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

void build_graph(const int32_t *src, const int32_t *dst, const int64_t *t, int64_t m,
                 cudaStream_t s, DevGraph &g);
void free_graph(DevGraph &g, cudaStream_t s);

// Class table of the GPU side: for each class M_ij (row-major), the raw cells
// (Star 0..23 | Pair 24..31 | Tri 32..55) it occupies; the first is the one
// reported. Star classes own one cell, pair classes the two mirror cells
// (Sec. IV-A), triangle classes one cell per type (Sec. IV-B) with the type-II
// cell first.
static const int8_t CLASS_CELLS[36][3] = {
    {8, -1, -1},  {9, -1, -1},  {0, -1, -1},  {1, -1, -1},  {44, 48, 38}, {46, 49, 36},
    {10, -1, -1}, {11, -1, -1}, {2, -1, -1},  {5, -1, -1},  {45, 50, 34}, {47, 51, 32},
    {3, -1, -1},  {13, -1, -1}, {12, -1, -1}, {4, -1, -1},  {40, 52, 39}, {42, 53, 37},
    {15, -1, -1}, {14, -1, -1}, {6, -1, -1},  {7, -1, -1},  {41, 54, 35}, {43, 55, 33},
    {16, -1, -1}, {22, -1, -1}, {23, -1, -1}, {18, -1, -1}, {24, 31, -1}, {27, 28, -1},
    {19, -1, -1}, {20, -1, -1}, {17, -1, -1}, {21, -1, -1}, {26, 29, -1}, {25, 30, -1},
};

// Edge pattern of each class: edges in time order, nodes 1, 2, 3 by first
// appearance. M24, M25, M46, M55, M56, M63, M65, M66 follow the paper's own
// examples; the other placements are this library's convention (star
// classes in rows 1-4 and 5-6 x cols 1-4, triangles rows 1-4 x cols 5-6,
// pairs rows 5-6 x cols 5-6).
static const char *CLASS_CODE[36] = {
    "12 13 12", "12 13 21", "12 13 13", "12 13 31", "12 13 23", "12 13 32",
    "12 31 12", "12 31 21", "12 31 13", "12 23 32", "12 31 23", "12 31 32",
    "12 31 31", "12 23 12", "12 23 21", "12 23 23", "12 23 13", "12 23 31",
    "12 32 12", "12 32 21", "12 32 23", "12 32 32", "12 32 13", "12 32 31",
    "12 12 13", "12 12 23", "12 12 32", "12 21 13", "12 12 12", "12 21 21",
    "12 21 31", "12 21 23", "12 12 31", "12 21 32", "12 21 12", "12 12 21",
};

namespace {

// One non-blocking stream per device for the synchronous calls.
cudaStream_t lib_stream() {
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    int d = current_device();
    std::lock_guard<std::mutex> lk(mu);
    if (!streams[d]) TM_CUDA(cudaStreamCreateWithFlags(&streams[d], cudaStreamNonBlocking));
    return streams[d];
}

template <typename F>
int guarded(F &&f) {
    try {
        f();
        return TM_OK;
    } catch (const Error &e) {
        set_error(e.code, e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        set_error(TM_ENOMEM, "host allocation failed");
        return TM_ENOMEM;
    } catch (...) {
        set_error(TM_ECUDA, "unexpected internal error");
        return TM_ECUDA;
    }
}

}  // namespace
}  // namespace tmi

using namespace tmi;

bool tmi::graph_view(const tm_graph *h, const DevGraph **g, int *device) {
    if (!h) return false;
    *g = &h->g;
    *device = h->device;
    return true;
}

void tmi::record_error(int code, const std::string &msg) { set_error(code, msg); }

int tmi::current_device_id() { return current_device(); }

namespace {

tm_graph *build_on(const int32_t *src, const int32_t *dst, const int64_t *t, int64_t m,
                   cudaStream_t s) {
    tm_graph *h = nullptr;
    int rc = guarded([&] {
        h = new tm_graph();
        h->device = current_device();
        try {
            build_graph(src, dst, t, m, s, h->g);
        } catch (...) {
            free_graph(h->g, s);
            delete h;
            h = nullptr;
            throw;
        }
    });
    return rc == TM_OK ? h : nullptr;
}

void count_cells(const tm_graph *g, int64_t delta, cudaStream_t s, unsigned long long *dcells) {
    TM_CUDA(cudaMemsetAsync(dcells, 0, sizeof(unsigned long long) * NCELLS, s));
    launch_count(g->g, delta, 0, (int32_t)(2 * g->g.m), dcells, s);
    launch_fill_tri_types(dcells, s);
}

void check_count_args(const tm_graph *g, int64_t delta) {
    if (!g) fail(TM_EINVAL, "NULL graph");
    if (delta < 0) fail(TM_EINVAL, "delta must be >= 0");
    int d = current_device();
    if (d != g->device) fail(TM_EINVAL, "graph was built on another device");
}

void sync_count(const tm_graph *g, int64_t delta, uint64_t *cells56) {
    check_count_args(g, delta);
    cudaStream_t s = lib_stream();
    unsigned long long *d = dev_alloc_n<unsigned long long>(NCELLS, s);
    count_cells(g, delta, s, d);
    TM_CUDA(cudaMemcpyAsync(cells56, d, sizeof(uint64_t) * NCELLS, cudaMemcpyDeviceToHost, s));
    dev_free(d, s);
    TM_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

extern "C" {

tm_graph *tm_build(const int32_t *src, const int32_t *dst, const int64_t *t, int64_t m) {
    cudaStream_t s = nullptr;
    if (guarded([&] { s = lib_stream(); }) != TM_OK) return nullptr;
    return build_on(src, dst, t, m, s);
}

tm_graph *tm_build_async(const int32_t *src, const int32_t *dst, const int64_t *t, int64_t m,
                         void *stream) {
    return build_on(src, dst, t, m, (cudaStream_t)stream);
}

void tm_free(tm_graph *g) {
    if (!g) return;
    guarded([&] {
        cudaStream_t s = lib_stream();
        free_graph(g->g, s);
        TM_CUDA(cudaStreamSynchronize(s));
    });
    delete g;
}

void tm_free_async(tm_graph *g, void *stream) {
    if (!g) return;
    guarded([&] { free_graph(g->g, (cudaStream_t)stream); });
    delete g;
}

int tm_count(const tm_graph *g, int64_t delta, uint64_t out[36]) {
    return guarded([&] {
        if (!out) fail(TM_EINVAL, "NULL out");
        uint64_t cells[NCELLS];
        sync_count(g, delta, cells);
        tm_merge(cells, out);
    });
}

int tm_count_raw(const tm_graph *g, int64_t delta, uint64_t star[24], uint64_t pair[8],
                 uint64_t tri[24]) {
    return guarded([&] {
        if (!star || !pair || !tri) fail(TM_EINVAL, "NULL counter array");
        uint64_t cells[NCELLS];
        sync_count(g, delta, cells);
        std::memcpy(star, cells, sizeof(uint64_t) * 24);
        std::memcpy(pair, cells + 24, sizeof(uint64_t) * 8);
        std::memcpy(tri, cells + 32, sizeof(uint64_t) * 24);
    });
}

int tm_count_async(const tm_graph *g, int64_t delta, void *stream, uint64_t *dev_cells) {
    return guarded([&] {
        check_count_args(g, delta);
        if (!dev_cells) fail(TM_EINVAL, "NULL dev_cells");
        count_cells(g, delta, (cudaStream_t)stream, (unsigned long long *)dev_cells);
    });
}

int tm_count_centres(const tm_graph *g, int64_t delta, const int32_t *centres, int32_t k,
                     uint64_t cells[56]) {
    return guarded([&] {
        check_count_args(g, delta);
        if (k < 0 || (k > 0 && !centres) || !cells) fail(TM_EINVAL, "bad centre list");
        std::vector<int32_t> off(2);
        cudaStream_t s = lib_stream();
        unsigned long long *d = dev_alloc_n<unsigned long long>(NCELLS, s);
        TM_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned long long) * NCELLS, s));
        for (int32_t i = 0; i < k; i++) {
            if (centres[i] < 0 || centres[i] >= g->g.n) {
                dev_free(d, s);
                fail(TM_EINVAL, "centre id out of range");
            }
            TM_CUDA(cudaMemcpyAsync(off.data(), g->g.off + centres[i], sizeof(int32_t) * 2,
                                    cudaMemcpyDeviceToHost, s));
            TM_CUDA(cudaStreamSynchronize(s));
            launch_count(g->g, delta, off[0], off[1], d, s);
        }
        TM_CUDA(cudaMemcpyAsync(cells, d, sizeof(uint64_t) * NCELLS, cudaMemcpyDeviceToHost, s));
        dev_free(d, s);
        TM_CUDA(cudaStreamSynchronize(s));
    });
}

int tm_count_shard(const tm_graph *g, int64_t delta, const int32_t *owner, int32_t rank,
                   uint64_t cells[56]) {
    return guarded([&] {
        check_count_args(g, delta);
        if (!owner || !cells || rank < 0) fail(TM_EINVAL, "bad shard arguments");
        cudaStream_t s = lib_stream();
        const int64_t n = g->g.n;
        int32_t *own = dev_alloc_n<int32_t>(n, s);
        unsigned long long *d = dev_alloc_n<unsigned long long>(NCELLS, s);
        try {
            if (n > 0)
                TM_CUDA(cudaMemcpyAsync(own, owner, sizeof(int32_t) * n, cudaMemcpyDefault, s));
            TM_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned long long) * NCELLS, s));
            launch_count_parts(g->g, delta, true, true, d, s, false, own, rank);
            TM_CUDA(cudaMemcpyAsync(cells, d, sizeof(uint64_t) * NCELLS, cudaMemcpyDeviceToHost, s));
            TM_CUDA(cudaStreamSynchronize(s));
        } catch (...) {
            dev_free(own, s);
            dev_free(d, s);
            throw;
        }
        dev_free(own, s);
        dev_free(d, s);
    });
}

int tm_count_select(const tm_graph *g, int64_t delta, int32_t what, uint64_t cells[56]) {
    return guarded([&] {
        check_count_args(g, delta);
        if (!cells || what < 1 || what > 3) fail(TM_EINVAL, "bad selection");
        cudaStream_t s = lib_stream();
        unsigned long long *d = dev_alloc_n<unsigned long long>(NCELLS, s);
        TM_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned long long) * NCELLS, s));
        launch_count_parts(g->g, delta, (what & TM_SELECT_STAR_PAIR) != 0,
                           (what & TM_SELECT_TRI) != 0, d, s);
        TM_CUDA(cudaMemcpyAsync(cells, d, sizeof(uint64_t) * NCELLS, cudaMemcpyDeviceToHost, s));
        dev_free(d, s);
        TM_CUDA(cudaStreamSynchronize(s));
    });
}

int tm_merge(const uint64_t cells[56], uint64_t out[36]) {
    if (!cells || !out) {
        set_error(TM_EINVAL, "NULL argument");
        return TM_EINVAL;
    }
    int bad = 0;
    for (int c = 0; c < 36; c++) {
        const uint64_t v = cells[CLASS_CELLS[c][0]];
        bool same = true;
        for (int k = 1; k < 3; k++)
            if (CLASS_CELLS[c][k] >= 0 && cells[CLASS_CELLS[c][k]] != v) same = false;
        bad += same ? 0 : 1;
        out[c] = v;
    }
    return bad;
}

int tm_fill_tri_types(uint64_t cells[56]) {
    if (!cells) {
        set_error(TM_EINVAL, "NULL cells");
        return TM_EINVAL;
    }
    uint64_t *tri = cells + 32;
    for (int di = 0; di < 2; di++)
        for (int dj = 0; dj < 2; dj++)
            for (int dk = 0; dk < 2; dk++) {
                const uint64_t v = tri[8 + (di * 2 + dj) * 2 + dk];
                tri[((1 - dk) * 2 + (1 - dj)) * 2 + (1 - di)] = v;     // type I
                tri[16 + ((1 - di) * 2 + dk) * 2 + dj] = v;            // type III
            }
    return TM_OK;
}

int tm_kernel_arch(int32_t *arch) {
    return guarded([&] {
        if (!arch) fail(TM_EINVAL, "NULL arch");
        *arch = kernel_binary_version();
    });
}

int tm_layout(char codes[36][16]) {
    if (!codes) return TM_EINVAL;
    for (int c = 0; c < 36; c++) {
        std::memset(codes[c], 0, 16);
        std::strncpy(codes[c], CLASS_CODE[c], 15);
    }
    return TM_OK;
}

int64_t tm_graph_nodes(const tm_graph *g) { return g ? g->g.n : -1; }
int64_t tm_graph_edges(const tm_graph *g) { return g ? g->g.m : -1; }

uint64_t tm_launch_count(void) { return g_launches.load(); }

void tm_profile_enable(int on) { g_profile.store(on ? 1 : 0); }

int tm_profile_read(double ms[], uint64_t calls[]) {
    return guarded([&] {
        std::vector<PhaseRec> recs;
        {
            std::lock_guard<std::mutex> lk(g_prof_mu);
            recs.swap(g_prof_recs);
        }
        for (auto &r : recs) {
            float x = 0.f;
            TM_CUDA(cudaEventSynchronize(r.b));
            TM_CUDA(cudaEventElapsedTime(&x, r.a, r.b));
            if (r.phase >= 0 && r.phase < TM_NPHASES) {
                if (ms) ms[r.phase] += x;
                if (calls) calls[r.phase] += 1;
            }
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
    });
}

const char *tm_last_error(int *code) {
    if (code) *code = t_err_code;
    return t_err_msg.c_str();
}

}  // extern "C"
