// Batched counting: many graphs (or the components of one multi-component
// graph, or one graph for several windows), each with its own delta, counted
// together as a table of segments by the fast count kernels: every kernel of
// the sequence is one persistent launch over all segments, whose warps or
// blocks take units of work (entry ranges, listed entries, joins) of one
// segment at a time in order. The launch sequence (uploads of the segment
// table, clears, the kernels, the type-I/III fill, the download of the cells)
// is captured once in a CUDA graph and replayed; the table is data, so a new
// batch only rewrites the pinned staging buffers.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "tm_internal.cuh"

namespace tmi {

void build_graph(const int32_t *src, const int32_t *dst, const int64_t *t, int64_t m,
                 cudaStream_t s, DevGraph &g);
void free_graph(DevGraph &g, cudaStream_t s);

namespace {

// Process-wide batching parameters (set by tm_batch_config / tm_tune_batch):
// entries per warp unit of the streaming passes and the Tri join's blocks
// per SM (0: as many as fit).
std::mutex g_cfg_mu;
int64_t g_item_entries = COUNT_ECHUNK;
int32_t g_blocks_per_sm = 0;

struct JobSpec {
    const DevGraph *g;
    int64_t delta;
    int32_t tbegin, tend;  // the job's entries in g
};

// Reusable device + pinned buffers and the captured launch sequence: the
// segment table and its unit prefix are staged in pinned memory, and one
// CUDA graph uploads them, clears the cells, runs the segmented count
// (window starts, Star/Pair list, Tri jobs and join, type fill) and
// downloads the cells. The scratch is one device block sized for the
// plan's entry capacity, so a call allocates nothing unless the batch is
// larger than every batch before it.
class BatchPlan {
   public:
    ~BatchPlan() { release(); }

    // Counts the jobs; cells_out receives 56 cells per job.
    void run(const std::vector<JobSpec> &jobs, int64_t item_entries, int blocks_per_sm,
             cudaStream_t s, std::vector<uint64_t> &cells_out) {
        const int32_t nj = (int32_t)jobs.size();
        const int32_t echunk = (int32_t)std::max<int64_t>(128, item_entries / 128 * 128);
        int64_t total = 0;
        for (const JobSpec &j : jobs) total += (int64_t)j.tend - j.tbegin;
        ensure(nj, total, blocks_per_sm, echunk, s);
        int64_t xbase = 0;
        h_meta_[0] = nj;
        h_meta_[1] = 0;
        for (int32_t j = 0; j < nj; j++) {
            Segment &sg = h_segs_[j];
            sg.g = *jobs[j].g;
            sg.delta = jobs[j].delta;
            sg.cells = d_cells_ + (size_t)NCELLS * j;
            sg.begin = jobs[j].tbegin;
            sg.end = jobs[j].tend;
            sg.xbase = xbase;
            const int64_t len = (int64_t)jobs[j].tend - jobs[j].tbegin;
            xbase += len;
            h_meta_[2 + j] = h_meta_[1 + j] + (int32_t)((len + echunk - 1) / echunk);
        }
        TM_CUDA(cudaGraphLaunch(exec_, s));
        g_launches.fetch_add(launches_per_run_, std::memory_order_relaxed);
        TM_CUDA(cudaStreamSynchronize(s));
        cells_out.assign(h_cells_, h_cells_ + (size_t)NCELLS * nj);
    }

   private:
    void ensure(int32_t nj, int64_t entries, int bps, int32_t echunk, cudaStream_t s) {
        if (exec_ && nj <= cap_jobs_ && entries <= cap_entries_ && bps == bps_ &&
            echunk == echunk_ && s == stream_)
            return;
        const int32_t want_jobs = std::max(nj, cap_jobs_);
        const int64_t want_entries = std::max(entries, cap_entries_);
        release();
        cap_jobs_ = 64;
        while (cap_jobs_ < want_jobs) cap_jobs_ <<= 1;
        cap_entries_ = 1 << 16;
        while (cap_entries_ < want_entries) cap_entries_ <<= 1;
        bps_ = bps;
        echunk_ = echunk;
        stream_ = s;
        TM_CUDA(cudaMalloc(&d_segs_, sizeof(Segment) * cap_jobs_));
        TM_CUDA(cudaMalloc(&d_meta_, sizeof(int32_t) * (cap_jobs_ + 2)));
        TM_CUDA(cudaMalloc(&d_cells_, sizeof(unsigned long long) * NCELLS * cap_jobs_));
        TM_CUDA(cudaMalloc(&d_scratch_, count_scratch_bytes(cap_entries_, cap_jobs_)));
        TM_CUDA(cudaMallocHost(&h_segs_, sizeof(Segment) * cap_jobs_));
        TM_CUDA(cudaMallocHost(&h_meta_, sizeof(int32_t) * (cap_jobs_ + 2)));
        TM_CUDA(cudaMallocHost(&h_cells_, sizeof(unsigned long long) * NCELLS * cap_jobs_));
        std::memset(h_segs_, 0, sizeof(Segment) * cap_jobs_);
        std::memset(h_meta_, 0, sizeof(int32_t) * (cap_jobs_ + 2));
        count_scratch_carve(d_scratch_, cap_entries_, cap_jobs_, scratch_);
        cudaGraph_t graph;
        const uint64_t l0 = g_launches.load();
        TM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        try {
            TM_CUDA(cudaMemcpyAsync(d_segs_, h_segs_, sizeof(Segment) * cap_jobs_,
                                    cudaMemcpyHostToDevice, s));
            TM_CUDA(cudaMemcpyAsync(d_meta_, h_meta_, sizeof(int32_t) * (cap_jobs_ + 2),
                                    cudaMemcpyHostToDevice, s));
            TM_CUDA(cudaMemsetAsync(d_cells_, 0, sizeof(unsigned long long) * NCELLS * cap_jobs_, s));
            launch_count_segments(nullptr, d_segs_, d_meta_, cap_jobs_, true, true, true, scratch_,
                                  s, bps_, echunk_);
            TM_CUDA(cudaMemcpyAsync(h_cells_, d_cells_, sizeof(unsigned long long) * NCELLS * cap_jobs_,
                                    cudaMemcpyDeviceToHost, s));
        } catch (...) {
            cudaGraph_t dead;
            cudaStreamEndCapture(s, &dead);
            if (dead) cudaGraphDestroy(dead);
            throw;
        }
        TM_CUDA(cudaStreamEndCapture(s, &graph));
        // the captured launches were counted once; every replay counts them again
        launches_per_run_ = g_launches.load() - l0;
        g_launches.fetch_sub(launches_per_run_);
        cudaError_t e = cudaGraphInstantiate(&exec_, graph, 0);
        cudaGraphDestroy(graph);
        TM_CUDA(e);
    }

    void release() {
        if (exec_) cudaGraphExecDestroy(exec_);
        exec_ = nullptr;
        cudaFree(d_segs_);
        cudaFree(d_meta_);
        cudaFree(d_cells_);
        cudaFree(d_scratch_);
        cudaFreeHost(h_segs_);
        cudaFreeHost(h_meta_);
        cudaFreeHost(h_cells_);
        d_segs_ = nullptr;
        d_meta_ = nullptr;
        d_cells_ = nullptr;
        d_scratch_ = nullptr;
        h_segs_ = nullptr;
        h_meta_ = nullptr;
        h_cells_ = nullptr;
        cap_jobs_ = 0;
        cap_entries_ = 0;
    }

    int32_t cap_jobs_ = 0;
    int64_t cap_entries_ = 0;
    int bps_ = -1;
    int32_t echunk_ = 0;
    uint64_t launches_per_run_ = 0;
    cudaStream_t stream_ = nullptr;
    cudaGraphExec_t exec_ = nullptr;
    Segment *d_segs_ = nullptr, *h_segs_ = nullptr;
    int32_t *d_meta_ = nullptr, *h_meta_ = nullptr;  // k, unit prefix (k + 1)
    unsigned long long *d_cells_ = nullptr, *h_cells_ = nullptr;
    void *d_scratch_ = nullptr;
    CountScratch scratch_;
};

// One plan and one stream per device for the synchronous batched calls.
struct DevicePlan {
    std::mutex mu;
    BatchPlan plan;
    cudaStream_t stream = nullptr;
};
DevicePlan g_plans[64];

DevicePlan &plan_for(int dev) {
    if (dev < 0 || dev >= 64) fail(TM_EINVAL, "device index out of range");
    return g_plans[dev];
}

void run_jobs(const std::vector<JobSpec> &jobs, std::vector<uint64_t> &cells, int64_t item_entries,
              int32_t bps) {
    DevicePlan &dp = plan_for(current_device_id());
    std::lock_guard<std::mutex> lk(dp.mu);
    if (!dp.stream) TM_CUDA(cudaStreamCreateWithFlags(&dp.stream, cudaStreamNonBlocking));
    dp.plan.run(jobs, item_entries, bps, dp.stream, cells);
}

void current_config(int64_t &ie, int32_t &bps) {
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    ie = g_item_entries;
    bps = g_blocks_per_sm;
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

void check_graph(const tm_graph *g) {
    if (!g) fail(TM_EINVAL, "NULL graph");
    if (g->device != current_device_id()) fail(TM_EINVAL, "graph was built on another device");
}

std::vector<JobSpec> component_jobs(const tm_graph *g, const int64_t *deltas) {
    std::vector<JobSpec> jobs;
    const int32_t k = g->comp_toff.empty() ? 1 : (int32_t)g->comp_toff.size() - 1;
    for (int32_t c = 0; c < k; c++) {
        if (deltas[c] < 0) fail(TM_EINVAL, "delta must be >= 0");
        const int32_t b = g->comp_toff.empty() ? 0 : g->comp_toff[c];
        const int32_t e = g->comp_toff.empty() ? (int32_t)(2 * g->g.m) : g->comp_toff[c + 1];
        jobs.push_back(JobSpec{&g->g, deltas[c], b, e});
    }
    return jobs;
}

// --------------------------------------------------- multi-component build

struct CompCheck {
    int32_t bad_neg;
    int32_t bad_loop;
};

__device__ __forceinline__ int32_t comp_of(const int64_t *eoff, int32_t k, int64_t e) {
    int32_t lo = 0, hi = k;  // largest c with eoff[c] <= e
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (eoff[mid] <= e) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void k_comp_max(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                           const int64_t *__restrict__ eoff, int32_t k, int64_t M,
                           int32_t *__restrict__ maxid, CompCheck *chk) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < M;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = src[e], b = dst[e];
        if (a < 0 || b < 0) chk->bad_neg = 1;
        if (a == b) chk->bad_loop = 1;
        const int32_t c = comp_of(eoff, k, e);
        int32_t v = max(a, b);
        // a warp inside one component combines first: a large component would
        // otherwise send all its edges to one atomic
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, c);
        if (peers == 0xffffffffu) {
            for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
            if ((threadIdx.x & 31) == 0) atomicMax(&maxid[c], v);
        } else {
            atomicMax(&maxid[c], v);
        }
    }
}

__global__ void k_comp_offset(int32_t *__restrict__ src, int32_t *__restrict__ dst,
                              const int64_t *__restrict__ eoff, const int32_t *__restrict__ nbase,
                              int32_t k, int64_t M) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < M;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t base = nbase[comp_of(eoff, k, e)];
        src[e] += base;
        dst[e] += base;
    }
}

__global__ void k_comp_toff(const int32_t *__restrict__ off, const int32_t *__restrict__ nbase,
                            int32_t k, int32_t *__restrict__ toff) {
    const int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c <= k) toff[c] = off[nbase[c]];
}

}  // namespace

void *new_batch_plan() { return new BatchPlan(); }
void delete_batch_plan(void *plan) { delete static_cast<BatchPlan *>(plan); }

// Counts whole graphs with their windows on stream s with a caller-owned
// plan, in runs of at most max_entries entries (a larger graph runs alone).
void run_batch_on(const std::vector<const DevGraph *> &graphs, const std::vector<int64_t> &deltas,
                  void *plan, cudaStream_t s, int64_t max_entries, std::vector<uint64_t> &cells) {
    int64_t ie;
    int32_t bps;
    current_config(ie, bps);
    cells.clear();
    std::vector<JobSpec> run;
    std::vector<uint64_t> part;
    int64_t total = 0;
    auto flush = [&] {
        if (run.empty()) return;
        static_cast<BatchPlan *>(plan)->run(run, ie, bps, s, part);
        cells.insert(cells.end(), part.begin(), part.end());
        run.clear();
        total = 0;
    };
    for (size_t i = 0; i < graphs.size(); i++) {
        const int64_t len = 2 * graphs[i]->m;
        if (!run.empty() && (total + len > max_entries || (int32_t)run.size() >= 64)) flush();
        run.push_back(JobSpec{graphs[i], deltas[i], 0, (int32_t)len});
        total += len;
    }
    flush();
}

}  // namespace tmi

using namespace tmi;

extern "C" {

int tm_count_batch(const tm_graph *const *gs, const int64_t *deltas, int32_t n, uint64_t *out) {
    return guard([&] {
        if (n < 0 || (n > 0 && (!gs || !deltas || !out))) fail(TM_EINVAL, "bad batch arguments");
        if (n == 0) return;
        std::vector<JobSpec> jobs;
        for (int32_t i = 0; i < n; i++) {
            check_graph(gs[i]);
            if (deltas[i] < 0) fail(TM_EINVAL, "delta must be >= 0");
            jobs.push_back(JobSpec{&gs[i]->g, deltas[i], 0, (int32_t)(2 * gs[i]->g.m)});
        }
        int64_t ie;
        int32_t bps;
        current_config(ie, bps);
        std::vector<uint64_t> cells;
        run_jobs(jobs, cells, ie, bps);
        for (int32_t i = 0; i < n; i++) tm_merge(cells.data() + (size_t)NCELLS * i, out + 36 * (size_t)i);
    });
}

tm_graph *tm_build_many(int32_t k, const int32_t *const *src, const int32_t *const *dst,
                        const int64_t *const *t, const int64_t *m) {
    tm_graph *h = nullptr;
    int rc = guard([&] {
        if (k <= 0 || !src || !dst || !t || !m) fail(TM_EINVAL, "tm_build_many: bad arguments");
        std::vector<int64_t> eoff(k + 1, 0);
        for (int32_t c = 0; c < k; c++) {
            if (m[c] < 0) fail(TM_EINVAL, "tm_build_many: negative edge count");
            if (m[c] > 0 && (!src[c] || !dst[c] || !t[c]))
                fail(TM_EINVAL, "tm_build_many: NULL edge array");
            eoff[c + 1] = eoff[c] + m[c];
        }
        const int64_t M = eoff[k];
        if (M >= (int64_t(1) << 30)) fail(TM_EINVAL, "tm_build_many: total edges must be < 2^30");
        DevicePlan &dp = plan_for(current_device_id());
        cudaStream_t s;
        {
            std::lock_guard<std::mutex> lk(dp.mu);
            if (!dp.stream) TM_CUDA(cudaStreamCreateWithFlags(&dp.stream, cudaStreamNonBlocking));
            s = dp.stream;
        }
        int32_t *a = dev_alloc_n<int32_t>(M, s), *b = dev_alloc_n<int32_t>(M, s);
        int64_t *tt = dev_alloc_n<int64_t>(M, s);
        int64_t *d_eoff = dev_alloc_n<int64_t>(k + 1, s);
        int32_t *d_max = dev_alloc_n<int32_t>(k + 1, s);
        CompCheck *d_chk = dev_alloc_n<CompCheck>(1, s);
        auto cleanup = [&] {
            dev_free(a, s);
            dev_free(b, s);
            dev_free(tt, s);
            dev_free(d_eoff, s);
            dev_free(d_max, s);
            dev_free(d_chk, s);
        };
        try {
            for (int32_t c = 0; c < k; c++) {
                if (!m[c]) continue;
                TM_CUDA(cudaMemcpyAsync(a + eoff[c], src[c], sizeof(int32_t) * m[c], cudaMemcpyDefault, s));
                TM_CUDA(cudaMemcpyAsync(b + eoff[c], dst[c], sizeof(int32_t) * m[c], cudaMemcpyDefault, s));
                TM_CUDA(cudaMemcpyAsync(tt + eoff[c], t[c], sizeof(int64_t) * m[c], cudaMemcpyDefault, s));
            }
            TM_CUDA(cudaMemcpyAsync(d_eoff, eoff.data(), sizeof(int64_t) * (k + 1),
                                    cudaMemcpyHostToDevice, s));
            TM_CUDA(cudaMemsetAsync(d_max, 0xff, sizeof(int32_t) * (k + 1), s));
            TM_CUDA(cudaMemsetAsync(d_chk, 0, sizeof(CompCheck), s));
            if (M > 0)
                TM_LAUNCH(k_comp_max, (unsigned)std::min<int64_t>((M + 255) / 256, num_sms() * 16), 256,
                          0, s, a, b, d_eoff, k, M, d_max, d_chk);
            std::vector<int32_t> maxid(k + 1);
            CompCheck chk;
            TM_CUDA(cudaMemcpyAsync(maxid.data(), d_max, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, s));
            TM_CUDA(cudaMemcpyAsync(&chk, d_chk, sizeof chk, cudaMemcpyDeviceToHost, s));
            TM_CUDA(cudaStreamSynchronize(s));
            if (chk.bad_neg) fail(TM_EINVAL, "tm_build_many: negative node id");
            if (chk.bad_loop) fail(TM_EINVAL, "tm_build_many: self-loop (src == dst)");
            std::vector<int32_t> nbase(k + 1, 0);
            for (int32_t c = 0; c < k; c++) {
                const int64_t nb = (int64_t)nbase[c] + maxid[c] + 1;
                if (nb >= (int64_t(1) << 31)) fail(TM_EINVAL, "tm_build_many: too many nodes in total");
                nbase[c + 1] = (int32_t)nb;
            }
            TM_CUDA(cudaMemcpyAsync(d_max, nbase.data(), sizeof(int32_t) * (k + 1),
                                    cudaMemcpyHostToDevice, s));
            if (M > 0)
                TM_LAUNCH(k_comp_offset, (unsigned)std::min<int64_t>((M + 255) / 256, num_sms() * 16),
                          256, 0, s, a, b, d_eoff, d_max, k, M);
            h = new tm_graph();
            h->device = current_device_id();
            try {
                build_graph(a, b, tt, M, s, h->g);
                // components without edges and ids above the last edge: the union's
                // node count can be below nbase[k]; clamp into [0, n]
                std::vector<int32_t> nb2(nbase);
                for (auto &x : nb2) x = std::min(x, h->g.n);
                TM_CUDA(cudaMemcpyAsync(d_max, nb2.data(), sizeof(int32_t) * (k + 1),
                                        cudaMemcpyHostToDevice, s));
                int32_t *d_toff = reinterpret_cast<int32_t *>(d_eoff);
                TM_LAUNCH(k_comp_toff, (unsigned)((k + 1 + 127) / 128), 128, 0, s, h->g.off, d_max, k,
                          d_toff);
                h->comp_toff.resize(k + 1);
                TM_CUDA(cudaMemcpyAsync(h->comp_toff.data(), d_toff, sizeof(int32_t) * (k + 1),
                                        cudaMemcpyDeviceToHost, s));
                TM_CUDA(cudaStreamSynchronize(s));
            } catch (...) {
                free_graph(h->g, s);
                delete h;
                h = nullptr;
                throw;
            }
        } catch (...) {
            cleanup();
            throw;
        }
        cleanup();
        TM_CUDA(cudaStreamSynchronize(s));
    });
    return rc == TM_OK ? h : nullptr;
}

int tm_count_multi(const tm_graph *g, const int64_t *deltas, int32_t k, uint64_t *out) {
    return guard([&] {
        check_graph(g);
        if (k < 0 || (k > 0 && (!deltas || !out))) fail(TM_EINVAL, "bad multi-delta arguments");
        if (k == 0) return;
        std::vector<int32_t> order(k);
        for (int32_t i = 0; i < k; i++) {
            if (deltas[i] < 0) fail(TM_EINVAL, "delta must be >= 0");
            order[i] = i;
        }
        // one sweep per run of up to 8 windows in ascending order
        std::stable_sort(order.begin(), order.end(),
                         [&](int32_t a, int32_t b) { return deltas[a] < deltas[b]; });
        DevicePlan &dp = plan_for(current_device_id());
        std::lock_guard<std::mutex> lk(dp.mu);
        if (!dp.stream) TM_CUDA(cudaStreamCreateWithFlags(&dp.stream, cudaStreamNonBlocking));
        cudaStream_t s = dp.stream;
        unsigned long long *d = static_cast<unsigned long long *>(
            dev_alloc(sizeof(unsigned long long) * NCELLS * k, s));
        std::vector<uint64_t> cells((size_t)NCELLS * k);
        try {
            TM_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned long long) * NCELLS * k, s));
            std::vector<int64_t> sorted(k);
            for (int32_t i = 0; i < k; i++) sorted[i] = deltas[order[i]];
            for (int32_t i = 0; i < k; i += 8) {
                const int32_t c = std::min<int32_t>(8, k - i);
                launch_count_multi_delta(g->g, sorted.data() + i, c, d + (size_t)NCELLS * i, s);
            }
            TM_CUDA(cudaMemcpyAsync(cells.data(), d, sizeof(uint64_t) * NCELLS * k,
                                    cudaMemcpyDeviceToHost, s));
            TM_CUDA(cudaStreamSynchronize(s));
        } catch (...) {
            dev_free(d, s);
            throw;
        }
        dev_free(d, s);
        for (int32_t i = 0; i < k; i++)
            tm_merge(cells.data() + (size_t)NCELLS * i, out + 36 * (size_t)order[i]);
    });
}

int32_t tm_graph_components(const tm_graph *g) {
    if (!g) return -1;
    return g->comp_toff.empty() ? 1 : (int32_t)g->comp_toff.size() - 1;
}

int tm_count_many(const tm_graph *g, const int64_t *deltas, uint64_t *out) {
    return guard([&] {
        check_graph(g);
        if (!deltas || !out) fail(TM_EINVAL, "NULL argument");
        std::vector<JobSpec> jobs = component_jobs(g, deltas);
        int64_t ie;
        int32_t bps;
        current_config(ie, bps);
        std::vector<uint64_t> cells;
        run_jobs(jobs, cells, ie, bps);
        for (size_t i = 0; i < jobs.size(); i++) tm_merge(cells.data() + NCELLS * i, out + 36 * i);
    });
}

int tm_batch_config(int64_t item_entries, int32_t blocks_per_sm) {
    return guard([&] {
        if (item_entries < 0 || blocks_per_sm < 0) fail(TM_EINVAL, "negative batch parameter");
        std::lock_guard<std::mutex> lk(g_cfg_mu);
        if (item_entries > 0) g_item_entries = std::max<int64_t>(256, item_entries);
        if (blocks_per_sm >= 0) g_blocks_per_sm = blocks_per_sm;
    });
}

int tm_batch_get_config(int64_t *item_entries, int32_t *blocks_per_sm) {
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    if (item_entries) *item_entries = g_item_entries;
    if (blocks_per_sm) *blocks_per_sm = g_blocks_per_sm;
    return TM_OK;
}

int tm_tune_batch(const tm_graph *g, const int64_t *deltas, int32_t reps, int64_t *best_item_entries,
                  int32_t *best_blocks_per_sm, double *best_ms) {
    return guard([&] {
        check_graph(g);
        if (!deltas || reps <= 0) fail(TM_EINVAL, "bad tuning arguments");
        std::vector<JobSpec> jobs = component_jobs(g, deltas);
        const int64_t ies[] = {256, 512, 1024, 2048};
        const int maxb = count_join_blocks_per_sm();
        std::vector<int32_t> bpss;
        for (int b = 1; b <= maxb; b++) bpss.push_back(b);
        double best = 1e300;
        int64_t bi = g_item_entries;
        int32_t bb = g_blocks_per_sm;
        std::vector<uint64_t> cells, ref;
        for (int64_t ie : ies)
            for (int32_t bps : bpss) {
                run_jobs(jobs, cells, ie, bps);  // warm-up (and capture)
                if (ref.empty()) ref = cells;
                if (cells != ref) fail(TM_ECUDA, "tm_tune_batch: configurations disagree");
                double total = 0;
                for (int r = 0; r < reps; r++) {
                    auto t0 = std::chrono::steady_clock::now();
                    run_jobs(jobs, cells, ie, bps);
                    total += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
                }
                const double ms = total / reps;
                if (ms < best) {
                    best = ms;
                    bi = ie;
                    bb = bps;
                }
            }
        {
            std::lock_guard<std::mutex> lk(g_cfg_mu);
            g_item_entries = bi;
            g_blocks_per_sm = bb;
        }
        if (best_item_entries) *best_item_entries = bi;
        if (best_blocks_per_sm) *best_blocks_per_sm = bb;
        if (best_ms) *best_ms = best;
    });
}

}  // extern "C"
