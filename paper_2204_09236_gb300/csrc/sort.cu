// Device prefix sums and the array-to-array radix sorts.
//
// The radix sort orders the edges by (t, edge id) (stability keeps the id
// order of equal timestamps), the incident entries by centre, and the edges
// by node pair; its kernels are in radix.cuh.
#include "radix.cuh"

namespace tmi {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;  // 4096

using radix::block_excl_scan;

// The value a scan adds for one input element.
struct Identity {
    __device__ __forceinline__ int operator()(int32_t v) const { return v; }
};
struct LowBit {
    __device__ __forceinline__ int operator()(uint32_t v) const { return (int)(v & 1u); }
};

template <typename T, typename F>
__global__ void k_tile_sums(const T *__restrict__ in, int64_t n, int32_t *__restrict__ sums, F f) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int acc = 0;
#pragma unroll
    for (int r = 0; r < SCAN_ITEMS; r++) {
        int64_t i = base + r * SCAN_THREADS + threadIdx.x;
        if (i < n) acc += f(in[i]);
    }
    __shared__ int total;
    block_excl_scan<SCAN_THREADS>(acc, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// One block scans `sums` (exclusive) in place.
__global__ void k_scan_sums(int32_t *sums, int64_t n) {
    __shared__ int total;
    int carry = 0;
    for (int64_t base = 0; base < n; base += SCAN_THREADS) {
        int64_t i = base + threadIdx.x;
        int v = i < n ? sums[i] : 0;
        int ex = block_excl_scan<SCAN_THREADS>(v, &total);
        if (i < n) sums[i] = carry + ex;
        carry += total;
        __syncthreads();
    }
}

// Shared-memory index of tile element i, padded by one word per 32 so that
// both the coalesced phase (thread t touches t + 256 r) and the per-thread
// phase (thread t touches 16 t + k) are free of bank conflicts.
__device__ __forceinline__ int scan_pad(int i) { return i + (i >> 5); }

template <typename T, typename F>
__global__ void k_tile_apply(const T *in, int32_t *out, int64_t n, const int32_t *__restrict__ sums,
                             F f) {
    __shared__ int32_t tile[SCAN_TILE + SCAN_TILE / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
#pragma unroll
    for (int r = 0; r < SCAN_ITEMS; r++) {
        int64_t i = base + r * SCAN_THREADS + threadIdx.x;
        tile[scan_pad(r * SCAN_THREADS + threadIdx.x)] = i < n ? f(in[i]) : 0;
    }
    __syncthreads();
    int loc[SCAN_ITEMS];
    int acc = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        loc[k] = acc;
        acc += tile[scan_pad(threadIdx.x * SCAN_ITEMS + k)];
    }
    __shared__ int total;
    int ex = block_excl_scan<SCAN_THREADS>(acc, &total) + sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) tile[scan_pad(threadIdx.x * SCAN_ITEMS + k)] = ex + loc[k];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < SCAN_ITEMS; r++) {
        int64_t i = base + r * SCAN_THREADS + threadIdx.x;
        if (i < n) out[i] = tile[scan_pad(r * SCAN_THREADS + threadIdx.x)];
    }
    if (base + SCAN_TILE >= n && threadIdx.x == 0) {
        // the last tile also writes the grand total
        out[n] = sums[blockIdx.x] + total;
    }
}

template <typename T, typename F>
void scan_impl(const T *in, int32_t *out, int64_t n, cudaStream_t s, F f) {
    if (n == 0) {
        TM_CUDA(cudaMemsetAsync(out, 0, sizeof(int32_t), s));
        return;
    }
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    int32_t *sums = dev_alloc_n<int32_t>(tiles, s);
    TM_LAUNCH((k_tile_sums<T, F>), (unsigned)tiles, SCAN_THREADS, 0, s, in, n, sums, f);
    TM_LAUNCH(k_scan_sums, 1, SCAN_THREADS, 0, s, sums, tiles);
    TM_LAUNCH((k_tile_apply<T, F>), (unsigned)tiles, SCAN_THREADS, 0, s, in, out, n, sums, f);
    dev_free(sums, s);
}

}  // namespace

void exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s) {
    scan_impl(in, out, n, s, Identity{});
}

void exclusive_scan_low_bit(const uint32_t *in, int32_t *out, int64_t n, cudaStream_t s) {
    scan_impl(in, out, n, s, LowBit{});
}

// ------------------------------------------------------------ radix sort

namespace {

// Array-to-array sort: the passes ping-pong between the input and the
// scratch pair, and the result lands in the scratch pair after an odd number
// of passes, in the input pair after an even number.
template <typename K, typename V>
void radix_sort_impl(K *keys, V *vals, K *keys_tmp, V *vals_tmp, int64_t n, int bits,
                     cudaStream_t s, K **keys_out, V **vals_out) {
    *keys_out = keys;
    *vals_out = vals;
    if (n <= 0) return;
    const int passes = bits > 8 ? (bits + 7) / 8 : 1;
    K *kf = passes & 1 ? keys_tmp : keys;
    V *vf = passes & 1 ? vals_tmp : vals;
    radix::sort<K, V>(radix::ArrayIn<K, V>{keys, vals}, radix::ArrayOut<K, V>{kf, vf}, keys_tmp,
                      vals_tmp, keys, vals, n, n, bits, s);
    *keys_out = kf;
    *vals_out = vf;
}

}  // namespace

void radix_sort_u32_rec(uint32_t *keys, HashRecord *vals, uint32_t *keys_tmp, HashRecord *vals_tmp,
                        int64_t n, int bits, cudaStream_t s, uint32_t **keys_out,
                        HashRecord **vals_out) {
    radix_sort_impl<uint32_t, HashRecord>(keys, vals, keys_tmp, vals_tmp, n, bits, s, keys_out,
                                          vals_out);
}

void radix_sort_u32_pair(uint32_t *keys, PairPayload *vals, uint32_t *keys_tmp,
                         PairPayload *vals_tmp, int64_t n, int bits, cudaStream_t s,
                         uint32_t **keys_out, PairPayload **vals_out) {
    radix_sort_impl<uint32_t, PairPayload>(keys, vals, keys_tmp, vals_tmp, n, bits, s, keys_out,
                                           vals_out);
}

void radix_sort_u64_v64(uint64_t *keys, uint64_t *vals, uint64_t *keys_tmp, uint64_t *vals_tmp,
                        int64_t n, int bits, cudaStream_t s, uint64_t **keys_out,
                        uint64_t **vals_out) {
    radix_sort_impl<uint64_t, uint64_t>(keys, vals, keys_tmp, vals_tmp, n, bits, s, keys_out,
                                        vals_out);
}

}  // namespace tmi
