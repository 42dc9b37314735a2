// Batched counting: many graphs (or the components of one multi-component
// graph), each with its own delta, counted by one persistent launch fed by a
// device work queue. The launch sequence (uploads of the job table and the
// queue, clears, the persistent kernel, the type-I/III fill, the download of
// the cells) is captured once in a CUDA graph and replayed; the queue is
// data, so a new batch only rewrites the pinned staging buffers.
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

// Process-wide batching parameters (set by tm_batch_config / tm_tune_batch).
// Defaults: what tm_tune_batch picked on the 512-graph batch workload; small
// items keep a window-heavy range from becoming the last block standing.
std::mutex g_cfg_mu;
int64_t g_item_entries = 4096;
int32_t g_blocks_per_sm = 2;  // 0: as many as fit

struct JobSpec {
    const DevGraph *g;
    int64_t delta;
    int32_t tbegin, tend;  // the job's entries in g->T
};

// Reusable device + pinned buffers and the captured launch sequence.
class BatchPlan {
   public:
    ~BatchPlan() { release(); }

    // Counts the jobs; cells_out receives 56 cells per job.
    void run(const std::vector<JobSpec> &jobs, int64_t item_entries, int blocks_per_sm,
             cudaStream_t s, std::vector<uint64_t> &cells_out) {
        const int32_t nj = (int32_t)jobs.size();
        items_.clear();
        for (int32_t j = 0; j < nj; j++) {
            const int64_t len = (int64_t)jobs[j].tend - jobs[j].tbegin;
            for (int kind = 0; kind < 2; kind++)
                for (int64_t b = jobs[j].tbegin; b < jobs[j].tend; b += item_entries) {
                    const int64_t e = std::min<int64_t>(b + item_entries, jobs[j].tend);
                    items_.push_back(WorkItem{j, kind, (int32_t)b, (int32_t)e});
                }
            (void)len;
        }
        // largest items first (the last items to finish are the short ones)
        std::stable_sort(items_.begin(), items_.end(), [](const WorkItem &a, const WorkItem &b) {
            return (a.end - a.begin) > (b.end - b.begin);
        });
        const int32_t ni = (int32_t)items_.size();
        int sms = num_sms();
        int bps = blocks_per_sm > 0 ? std::min(blocks_per_sm, batch_blocks_per_sm())
                                    : batch_blocks_per_sm();
        const int grid = std::max(1, sms * bps);
        ensure(nj, ni, grid, s);
        for (int32_t j = 0; j < nj; j++) {
            h_jobs_[j].g = *jobs[j].g;
            h_jobs_[j].delta = jobs[j].delta;
            h_jobs_[j].cells = d_cells_ + (size_t)NCELLS * j;
        }
        if (ni) std::memcpy(h_items_, items_.data(), sizeof(WorkItem) * ni);
        h_counts_[0] = ni;
        h_counts_[1] = nj;
        TM_CUDA(cudaGraphLaunch(exec_, s));
        g_launches.fetch_add(2, std::memory_order_relaxed);
        TM_CUDA(cudaStreamSynchronize(s));
        cells_out.assign(h_cells_, h_cells_ + (size_t)NCELLS * nj);
    }

   private:
    void ensure(int32_t nj, int32_t ni, int grid, cudaStream_t s) {
        if (exec_ && nj <= cap_jobs_ && ni <= cap_items_ && grid == grid_ && s == stream_) return;
        release();
        cap_jobs_ = 64;
        while (cap_jobs_ < nj) cap_jobs_ <<= 1;
        cap_items_ = 1024;
        while (cap_items_ < ni) cap_items_ <<= 1;
        grid_ = grid;
        stream_ = s;
        TM_CUDA(cudaMalloc(&d_jobs_, sizeof(BatchJob) * cap_jobs_));
        TM_CUDA(cudaMalloc(&d_items_, sizeof(WorkItem) * cap_items_));
        TM_CUDA(cudaMalloc(&d_counts_, sizeof(int32_t) * 4));
        TM_CUDA(cudaMalloc(&d_cells_, sizeof(unsigned long long) * NCELLS * cap_jobs_));
        TM_CUDA(cudaMallocHost(&h_jobs_, sizeof(BatchJob) * cap_jobs_));
        TM_CUDA(cudaMallocHost(&h_items_, sizeof(WorkItem) * cap_items_));
        TM_CUDA(cudaMallocHost(&h_counts_, sizeof(int32_t) * 4));
        TM_CUDA(cudaMallocHost(&h_cells_, sizeof(unsigned long long) * NCELLS * cap_jobs_));
        std::memset(h_jobs_, 0, sizeof(BatchJob) * cap_jobs_);
        std::memset(h_items_, 0, sizeof(WorkItem) * cap_items_);
        cudaGraph_t graph;
        TM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        try {
            TM_CUDA(cudaMemcpyAsync(d_jobs_, h_jobs_, sizeof(BatchJob) * cap_jobs_,
                                    cudaMemcpyHostToDevice, s));
            TM_CUDA(cudaMemcpyAsync(d_items_, h_items_, sizeof(WorkItem) * cap_items_,
                                    cudaMemcpyHostToDevice, s));
            TM_CUDA(cudaMemcpyAsync(d_counts_, h_counts_, sizeof(int32_t) * 2,
                                    cudaMemcpyHostToDevice, s));
            TM_CUDA(cudaMemsetAsync(d_counts_ + 2, 0, sizeof(int32_t), s));
            TM_CUDA(cudaMemsetAsync(d_cells_, 0, sizeof(unsigned long long) * NCELLS * cap_jobs_, s));
            launch_batch(d_jobs_, d_items_, d_counts_, d_counts_ + 2, grid, s);
            launch_fill_tri_types_batch(d_cells_, d_counts_ + 1, cap_jobs_, s);
            TM_CUDA(cudaMemcpyAsync(h_cells_, d_cells_, sizeof(unsigned long long) * NCELLS * cap_jobs_,
                                    cudaMemcpyDeviceToHost, s));
        } catch (...) {
            cudaGraph_t dead;
            cudaStreamEndCapture(s, &dead);
            if (dead) cudaGraphDestroy(dead);
            throw;
        }
        TM_CUDA(cudaStreamEndCapture(s, &graph));
        cudaError_t e = cudaGraphInstantiate(&exec_, graph, 0);
        cudaGraphDestroy(graph);
        TM_CUDA(e);
    }

    void release() {
        if (exec_) cudaGraphExecDestroy(exec_);
        exec_ = nullptr;
        cudaFree(d_jobs_);
        cudaFree(d_items_);
        cudaFree(d_counts_);
        cudaFree(d_cells_);
        cudaFreeHost(h_jobs_);
        cudaFreeHost(h_items_);
        cudaFreeHost(h_counts_);
        cudaFreeHost(h_cells_);
        d_jobs_ = nullptr;
        d_items_ = nullptr;
        d_counts_ = nullptr;
        d_cells_ = nullptr;
        h_jobs_ = nullptr;
        h_items_ = nullptr;
        h_counts_ = nullptr;
        h_cells_ = nullptr;
        cap_jobs_ = cap_items_ = 0;
    }

    std::vector<WorkItem> items_;
    int32_t cap_jobs_ = 0, cap_items_ = 0;
    int grid_ = 0;
    cudaStream_t stream_ = nullptr;
    cudaGraphExec_t exec_ = nullptr;
    BatchJob *d_jobs_ = nullptr, *h_jobs_ = nullptr;
    WorkItem *d_items_ = nullptr, *h_items_ = nullptr;
    int32_t *d_counts_ = nullptr, *h_counts_ = nullptr;  // nitems, njobs, head
    unsigned long long *d_cells_ = nullptr, *h_cells_ = nullptr;
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

// Counts whole graphs with their windows on stream s with a caller-owned plan.
void run_batch_on(const std::vector<const DevGraph *> &graphs, const std::vector<int64_t> &deltas,
                  void *plan, cudaStream_t s, std::vector<uint64_t> &cells) {
    std::vector<JobSpec> jobs;
    for (size_t i = 0; i < graphs.size(); i++)
        jobs.push_back(JobSpec{graphs[i], deltas[i], 0, (int32_t)(2 * graphs[i]->m)});
    int64_t ie;
    int32_t bps;
    current_config(ie, bps);
    static_cast<BatchPlan *>(plan)->run(jobs, ie, bps, s, cells);
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
        std::vector<JobSpec> jobs;
        for (int32_t i = 0; i < k; i++) {
            if (deltas[i] < 0) fail(TM_EINVAL, "delta must be >= 0");
            jobs.push_back(JobSpec{&g->g, deltas[i], 0, (int32_t)(2 * g->g.m)});
        }
        int64_t ie;
        int32_t bps;
        current_config(ie, bps);
        std::vector<uint64_t> cells;
        run_jobs(jobs, cells, ie, bps);
        for (int32_t i = 0; i < k; i++) tm_merge(cells.data() + (size_t)NCELLS * i, out + 36 * (size_t)i);
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
        const int64_t ies[] = {4096, 16384, 65536, 262144};
        const int maxb = batch_blocks_per_sm();
        std::vector<int32_t> bpss;
        for (int b = 1; b <= maxb; b *= 2) bpss.push_back(b);
        if (bpss.back() != maxb) bpss.push_back(maxb);
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
