// Serving loop: count requests of different sizes arrive over time; worker
// threads turn the pending ones into waves (continuous batching), admit new
// graphs against a device-memory budget, keep built graphs resident for
// repeat-delta queries (least recently used graphs are evicted first), build
// the wave's new graphs on the worker's own stream and count the whole wave
// with one batched persistent launch. Waves of different workers overlap on
// the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tm_internal.cuh"

namespace tmi {

void build_graph(const int32_t *src, const int32_t *dst, const int64_t *t, int64_t m,
                 cudaStream_t s, DevGraph &g);
void free_graph(DevGraph &g, cudaStream_t s);
void run_batch_on(const std::vector<const DevGraph *> &graphs, const std::vector<int64_t> &deltas,
                  void *plan, cudaStream_t s, int64_t max_entries, std::vector<uint64_t> &cells);
void *new_batch_plan();
void delete_batch_plan(void *plan);

namespace {

using Clock = std::chrono::steady_clock;

// Device bytes a resident graph holds (the entry arrays tt, tn, tc, cin, lk, off,
// positions, rank-ordered endpoints when kept, pair list, hash, Bloom filter)
// and the extra scratch its build needs at peak.
int64_t resident_bytes(int64_t m, int64_t n) {
    int64_t hash = 16;
    while (hash < 2 * m) hash <<= 1;
    return 64 * m + 4 + 8 * m + 8 * m + 8 * (m + 1) + 16 * hash + 4 * (n + 1) + m + (1 << 20);
}
int64_t build_scratch_bytes(int64_t m) { return 104 * m + (1 << 20); }

// Each worker counts its waves in runs of at most count_cap entries with a
// scratch slab of count_scratch_bytes(count_cap, WAVE_JOBS) bytes that it
// keeps; the server reserves the workers' slabs in its budget. A graph with
// more entries than that is counted alone with a larger slab, and the excess
// is charged to the graph while it is resident.
constexpr int32_t WAVE_JOBS = 64;
int64_t count_cap_entries(int64_t budget, int32_t workers) {
    int64_t cap = budget / (8 * (int64_t)workers * 24);
    if (cap > (int64_t(1) << 24)) cap = int64_t(1) << 24;
    if (cap < (int64_t(1) << 14)) cap = int64_t(1) << 14;
    return cap;
}
int64_t count_excess_bytes(int64_t m, int64_t cap) {
    if (2 * m <= cap) return 0;
    return (int64_t)count_scratch_bytes(2 * m, WAVE_JOBS) - (int64_t)count_scratch_bytes(cap, WAVE_JOBS);
}

struct Request {
    int64_t id;
    int64_t key;
    int64_t delta;
    bool has_edges;
    std::vector<int32_t> src, dst;
    std::vector<int64_t> t;
    int64_t n_hint = 0;
    Clock::time_point submitted;
    // results
    int status = 1;  // 1 pending, TM_OK done, < 0 failed
    std::string error;
    uint64_t out[36] = {};
    double latency_ms = 0;
};

struct Resident {
    tm_graph *g = nullptr;
    int64_t bytes = 0;
    int refs = 0;        // waves currently using it
    bool building = false;
    std::list<int64_t>::iterator lru;
};

}  // namespace
}  // namespace tmi

struct tm_server {
    int64_t budget = 0;
    int32_t max_wave = 64;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stopping = false;
    std::deque<tmi::Request *> pending;
    std::unordered_map<int64_t, tmi::Request *> all;  // by id
    std::unordered_map<int64_t, tmi::Resident> cache;  // by graph key
    std::list<int64_t> lru;                            // front = least recently used
    int64_t used = 0;                                  // resident + reserved bytes
    int64_t count_cap = 0;                             // entries per counting run
    int64_t reserved = 0;                              // the workers' counting slabs
    int32_t busy = 0;                                  // workers with a wave in flight
    int64_t next_id = 0;
    // statistics
    int64_t completed = 0, failed = 0, evictions = 0, builds = 0, waves = 0, edges_counted = 0;
    std::vector<double> latencies;
    std::vector<std::thread> workers;
};

namespace tmi {
namespace {

void finish(tm_server *S, Request *r, int status, const std::string &err) {
    r->status = status;
    r->error = err;
    r->latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - r->submitted).count();
    if (status == TM_OK) {
        S->completed++;
        S->latencies.push_back(r->latency_ms);
    } else {
        S->failed++;
    }
    r->src.clear();
    r->src.shrink_to_fit();
    r->dst.clear();
    r->dst.shrink_to_fit();
    r->t.clear();
    r->t.shrink_to_fit();
}

// Frees least-recently-used idle graphs until `need` more bytes fit.
bool make_room(tm_server *S, int64_t need, cudaStream_t s) {
    auto it = S->lru.begin();
    while (S->used + need > S->budget && it != S->lru.end()) {
        auto c = S->cache.find(*it);
        if (c != S->cache.end() && c->second.refs == 0 && !c->second.building) {
            tm_graph *g = c->second.g;
            S->used -= c->second.bytes;
            S->cache.erase(c);
            it = S->lru.erase(it);
            free_graph(g->g, s);
            delete g;
            S->evictions++;
        } else {
            ++it;
        }
    }
    return S->used + need <= S->budget;
}

void touch(tm_server *S, Resident &res, int64_t key) {
    S->lru.erase(res.lru);
    res.lru = S->lru.insert(S->lru.end(), key);
}

struct WaveEntry {
    Request *r;
    bool builds;  // this wave builds the graph
    int64_t scratch;
};

void worker_loop(tm_server *S) {
    cudaSetDevice(S->device);
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return;
    void *plan = new_batch_plan();
    std::vector<WaveEntry> wave;
    while (true) {
        wave.clear();
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stopping || !S->pending.empty(); });
            if (S->stopping && S->pending.empty()) break;
            // take up to max_wave admissible requests in arrival order
            for (auto it = S->pending.begin(); it != S->pending.end() && (int)wave.size() < S->max_wave;) {
                Request *r = *it;
                auto c = S->cache.find(r->key);
                if (c != S->cache.end()) {
                    if (c->second.building) {  // its build is in another wave
                        ++it;
                        continue;
                    }
                    c->second.refs++;
                    touch(S, c->second, r->key);
                    wave.push_back({r, false, 0});
                    it = S->pending.erase(it);
                    continue;
                }
                if (!r->has_edges) {
                    finish(S, r, TM_EINVAL, "no resident graph with this key and no edges given");
                    it = S->pending.erase(it);
                    S->cv_done.notify_all();
                    continue;
                }
                const int64_t m = (int64_t)r->src.size();
                const int64_t need = resident_bytes(m, r->n_hint) + build_scratch_bytes(m) +
                                     count_excess_bytes(m, S->count_cap);
                if (need > S->budget - S->reserved) {
                    finish(S, r, TM_EBUDGET, "graph does not fit in the server's memory budget");
                    it = S->pending.erase(it);
                    S->cv_done.notify_all();
                    continue;
                }
                if (!make_room(S, need, s)) {  // wait until in-flight waves free memory
                    ++it;
                    continue;
                }
                S->used += need;
                Resident res;
                res.building = true;
                res.refs = 1;
                res.bytes = need;
                res.lru = S->lru.insert(S->lru.end(), r->key);
                S->cache[r->key] = res;
                wave.push_back({r, true, build_scratch_bytes(m)});
                it = S->pending.erase(it);
            }
            if (wave.empty()) {
                if (S->busy == 0) {
                    // no wave in flight and every idle graph evicted: what is still
                    // pending can never be admitted
                    for (Request *r : S->pending)
                        finish(S, r, TM_EBUDGET,
                               "graph does not fit beside the server's reserved scratch");
                    S->pending.clear();
                    S->cv_done.notify_all();
                    continue;
                }
                // nothing admissible now: wait for a wave to finish or new work
                S->cv_work.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
            S->waves++;
            S->busy++;
        }
        // build the new graphs of the wave on this worker's stream
        std::vector<int> ok(wave.size(), 1);
        for (size_t i = 0; i < wave.size(); i++) {
            if (!wave[i].builds) continue;
            Request *r = wave[i].r;
            tm_graph *g = new tm_graph();
            g->device = S->device;
            try {
                build_graph(r->src.data(), r->dst.data(), r->t.data(), (int64_t)r->src.size(), s,
                            g->g);
            } catch (const Error &e) {
                free_graph(g->g, s);
                delete g;
                std::lock_guard<std::mutex> lk(S->mu);
                auto c = S->cache.find(r->key);
                S->used -= c->second.bytes;
                S->lru.erase(c->second.lru);
                S->cache.erase(c);
                finish(S, r, e.code, e.msg);
                ok[i] = 0;
                continue;
            }
            std::lock_guard<std::mutex> lk(S->mu);
            auto &res = S->cache[r->key];
            res.g = g;
            res.building = false;
            // the build scratch is back in the pool: keep only the resident bytes
            const int64_t keep =
                resident_bytes(g->g.m, g->g.n) + count_excess_bytes(g->g.m, S->count_cap);
            S->used -= res.bytes - keep;
            res.bytes = keep;
            S->builds++;
        }
        // one batched launch for every request of the wave
        std::vector<const DevGraph *> gs;
        std::vector<int64_t> deltas;
        std::vector<size_t> idx;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (size_t i = 0; i < wave.size(); i++) {
                if (!ok[i]) continue;
                gs.push_back(&S->cache[wave[i].r->key].g->g);
                deltas.push_back(wave[i].r->delta);
                idx.push_back(i);
            }
        }
        std::vector<uint64_t> cells;
        int status = TM_OK;
        std::string err;
        try {
            if (!gs.empty()) run_batch_on(gs, deltas, plan, s, S->count_cap, cells);
        } catch (const Error &e) {
            status = e.code;
            err = e.msg;
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (size_t q = 0; q < idx.size(); q++) {
                Request *r = wave[idx[q]].r;
                if (status == TM_OK) {
                    tm_merge(cells.data() + (size_t)NCELLS * q, r->out);
                    S->edges_counted += gs[q]->m;
                }
                finish(S, r, status, err);
            }
            for (auto &we : wave) {
                auto c = S->cache.find(we.r->key);
                if (c != S->cache.end()) c->second.refs--;
            }
            S->busy--;
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
    delete_batch_plan(plan);
    cudaStreamDestroy(s);
}

}  // namespace
}  // namespace tmi

using namespace tmi;

extern "C" {

tm_server *tm_server_create(int64_t budget_bytes, int32_t workers, int32_t max_wave) {
    if (budget_bytes <= 0 || workers <= 0 || workers > 64 || max_wave <= 0) {
        record_error(TM_EINVAL, "tm_server_create: budget, workers (1..64) and max_wave must be > 0");
        return nullptr;
    }
    tm_server *S = new tm_server();
    S->budget = budget_bytes;
    S->max_wave = max_wave;
    S->count_cap = count_cap_entries(budget_bytes, workers);
    // the workers' counting slabs are held for the server's lifetime
    S->reserved = (int64_t)workers * (int64_t)count_scratch_bytes(S->count_cap, WAVE_JOBS);
    S->used = S->reserved;
    if (S->used >= budget_bytes) {
        record_error(TM_EBUDGET, "tm_server_create: budget below the workers' counting scratch");
        delete S;
        return nullptr;
    }
    try {
        S->device = current_device_id();
        num_sms();  // per-device set-up before the workers start
    } catch (const Error &e) {
        record_error(e.code, e.msg);
        delete S;
        return nullptr;
    }
    for (int i = 0; i < workers; i++) S->workers.emplace_back(worker_loop, S);
    return S;
}

int64_t tm_server_submit(tm_server *S, const tm_request_desc *d) {
    if (!S || !d) {
        record_error(TM_EINVAL, "tm_server_submit: NULL argument");
        return TM_EINVAL;
    }
    if (d->delta < 0 || d->m < 0 || (d->m > 0 && (!d->src || !d->dst || !d->t))) {
        record_error(TM_EINVAL, "tm_server_submit: bad request");
        return TM_EINVAL;
    }
    Request *r = new Request();
    r->key = d->key;
    r->delta = d->delta;
    r->has_edges = d->src != nullptr || d->m > 0;
    r->n_hint = d->n_hint;
    if (d->m > 0) {
        r->src.assign(d->src, d->src + d->m);
        r->dst.assign(d->dst, d->dst + d->m);
        r->t.assign(d->t, d->t + d->m);
    }
    r->submitted = Clock::now();
    int64_t id;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        id = r->id = S->next_id++;
        S->all[id] = r;
        S->pending.push_back(r);
    }
    S->cv_work.notify_one();
    return id;
}

static int copy_result(tm_server *S, Request *r, uint64_t out[36], double *latency_ms) {
    (void)S;
    if (r->status == 1) return 1;
    if (latency_ms) *latency_ms = r->latency_ms;
    if (r->status != TM_OK) {
        record_error(r->status, r->error);
        return r->status;
    }
    if (out) std::memcpy(out, r->out, sizeof(uint64_t) * 36);
    return TM_OK;
}

int tm_server_poll(tm_server *S, int64_t id, uint64_t out[36], double *latency_ms) {
    if (!S) return TM_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) {
        record_error(TM_EINVAL, "unknown request id");
        return TM_EINVAL;
    }
    return copy_result(S, it->second, out, latency_ms);
}

int tm_server_wait(tm_server *S, int64_t id, uint64_t out[36], double *latency_ms, double timeout_s) {
    if (!S) return TM_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) {
        record_error(TM_EINVAL, "unknown request id");
        return TM_EINVAL;
    }
    Request *r = it->second;
    const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                          std::chrono::duration<double>(timeout_s));
    if (!S->cv_done.wait_until(lk, until, [&] { return r->status != 1; })) {
        record_error(TM_ETIMEOUT, "tm_server_wait: request still pending");
        return TM_ETIMEOUT;
    }
    return copy_result(S, r, out, latency_ms);
}

int tm_server_stats(tm_server *S, tm_server_stats_t *st) {
    if (!S || !st) return TM_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(st, 0, sizeof *st);
    st->submitted = S->next_id;
    st->completed = S->completed;
    st->failed = S->failed;
    st->pending = (int64_t)S->pending.size();
    st->resident_graphs = (int64_t)S->cache.size();
    st->resident_bytes = S->used;
    st->evictions = S->evictions;
    st->builds = S->builds;
    st->waves = S->waves;
    st->edges_counted = S->edges_counted;
    if (!S->latencies.empty()) {
        std::vector<double> l(S->latencies);
        std::sort(l.begin(), l.end());
        auto q = [&](double p) { return l[std::min(l.size() - 1, (size_t)(p * (l.size() - 1) + 0.5))]; };
        st->p50_ms = q(0.50);
        st->p99_ms = q(0.99);
        st->max_ms = l.back();
    }
    return TM_OK;
}

int tm_estimate_bytes(int64_t m, int64_t n, int64_t *resident, int64_t *build_scratch) {
    if (m < 0 || n < 0) return TM_EINVAL;
    if (resident) *resident = resident_bytes(m, n);
    if (build_scratch)
        *build_scratch = build_scratch_bytes(m) + (int64_t)count_scratch_bytes(2 * m, 1);
    return TM_OK;
}

int32_t tm_server_resident(tm_server *S, int64_t *keys, int32_t cap) {
    if (!S) return TM_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    int32_t k = 0;
    for (auto &kv : S->cache) {
        if (kv.second.building) continue;
        if (keys && k < cap) keys[k] = kv.first;
        k++;
    }
    return k;
}

void tm_server_destroy(tm_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
    }
    S->cv_work.notify_all();
    for (auto &w : S->workers) w.join();
    cudaSetDevice(S->device);
    for (auto &kv : S->cache) {
        if (kv.second.g) {
            free_graph(kv.second.g->g, nullptr);
            delete kv.second.g;
        }
    }
    cudaDeviceSynchronize();
    for (auto &kv : S->all) delete kv.second;
    delete S;
}

}  // extern "C"
