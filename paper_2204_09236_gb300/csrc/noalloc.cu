// tm_count_noalloc: counting that allocates no memory at all.
//
// Some callers cannot allocate device memory while they count: a serving
// thread that runs under a fixed device-memory budget handed out up front, a
// process whose allocator has been sized and locked, or code that must not
// trigger the implicit synchronisation a cudaMalloc / cudaFree can cause.
// This entry point counts already-built graphs for such callers. The only
// device memory it uses besides the graphs and the caller's host output is
// the file-scope array below, which the CUDA runtime places on every device
// that loads this library and keeps there until the process exits.
#include <cstring>
#include <mutex>
#include <string>

#include "tm_internal.cuh"

namespace tmi {
namespace {

// 56 uint64 counter cells per graph, for at most TM_NOALLOC_MAX_GRAPHS graphs
// per call: 256 * 56 * 8 bytes = 112 KiB on each device.
static __device__ __align__(256) unsigned long long g_noalloc_cells[TM_NOALLOC_MAX_GRAPHS * NCELLS];

// Device address of g_noalloc_cells, looked up once per device. In host code
// the symbol name is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress with that device current.
std::mutex g_mu;
unsigned long long *g_cells_ptr[64] = {};

unsigned long long *cells_on_device(int dev) {
    if (dev < 0 || dev >= 64) fail(TM_EINVAL, "tm_count_noalloc: device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_cells_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_cells);
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail(TM_ECUDA, std::string("tm_count_noalloc: cudaGetSymbolAddress failed: ") +
                               cudaGetErrorString(e));
        }
        g_cells_ptr[dev] = static_cast<unsigned long long *>(p);
    }
    return g_cells_ptr[dev];
}

}  // namespace
}  // namespace tmi

using namespace tmi;

extern "C" int tm_count_noalloc(const tm_graph *const *gs, const int64_t *deltas, int32_t k,
                                void *stream, uint64_t *out) {
    try {
        if (k < 0 || k > TM_NOALLOC_MAX_GRAPHS)
            fail(TM_EINVAL, "tm_count_noalloc: k = " + std::to_string(k) +
                                " is outside [0, TM_NOALLOC_MAX_GRAPHS = " +
                                std::to_string(TM_NOALLOC_MAX_GRAPHS) + "]");
        if (k == 0) return TM_OK;
        if (!gs || !deltas || !out) fail(TM_EINVAL, "tm_count_noalloc: NULL argument");
        const int dev = current_device_id();
        const DevGraph *views[TM_NOALLOC_MAX_GRAPHS];
        for (int32_t i = 0; i < k; i++) {
            int gdev = -1;
            if (!graph_view(gs[i], &views[i], &gdev)) fail(TM_EINVAL, "tm_count_noalloc: NULL graph");
            if (gdev != dev) fail(TM_EINVAL, "tm_count_noalloc: graph built on another device");
            if (deltas[i] < 0) fail(TM_EINVAL, "tm_count_noalloc: delta must be >= 0");
        }
        unsigned long long *cells = cells_on_device(dev);
        cudaStream_t s = (cudaStream_t)stream;
        // the array keeps the previous call's contents: clear the slots in use
        TM_CUDA(cudaMemsetAsync(cells, 0, sizeof(unsigned long long) * NCELLS * (size_t)k, s));
        for (int32_t i = 0; i < k; i++) launch_count_untimed(*views[i], deltas[i], cells + NCELLS * i, s);
        // all k graphs' cells in one copy and one wait, into this thread's
        // fixed host array (no host allocation either)
        static thread_local uint64_t raw[TM_NOALLOC_MAX_GRAPHS * NCELLS];
        TM_CUDA(cudaMemcpyAsync(raw, cells, sizeof(uint64_t) * NCELLS * (size_t)k,
                                cudaMemcpyDeviceToHost, s));
        TM_CUDA(cudaStreamSynchronize(s));
        for (int32_t i = 0; i < k; i++) tm_merge(raw + NCELLS * (size_t)i, out + 36 * (size_t)i);
        return TM_OK;
    } catch (const Error &e) {
        record_error(e.code, e.msg);
        return e.code;
    } catch (...) {
        record_error(TM_ECUDA, "tm_count_noalloc: unexpected internal error");
        return TM_ECUDA;
    }
}
