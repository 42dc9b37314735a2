// Device prefix sums and a stable LSD radix sort (8-bit digits).
//
// The radix sort orders the edges by (t, edge id) (stability keeps the id
// order of equal timestamps), the incident entries by centre, and the edges
// by node pair. Each pass: per-tile digit histograms, one exclusive scan over
// (digit, tile), and a stable scatter that ranks a tile in shared memory and
// writes every digit's run with consecutive addresses.
#include "tm_internal.cuh"

namespace tmi {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;  // 4096

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += o;
    }
    return v;
}

// Exclusive scan of one value per thread over the block; returns the
// exclusive prefix and writes the block total to *total.
template <int NT>
__device__ __forceinline__ int block_excl_scan(int v, int *total) {
    __shared__ int warp_sums[NT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = warp_incl_scan(v);
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = lane < NT / 32 ? warp_sums[lane] : 0;
        int wi = warp_incl_scan(w);
        if (lane < NT / 32) warp_sums[lane] = wi - w;
        if (lane == NT / 32 - 1) *total = wi;
    }
    __syncthreads();
    int r = inc - v + warp_sums[warp];
    __syncthreads();
    return r;
}

__global__ void k_tile_sums(const int32_t *__restrict__ in, int64_t n, int32_t *__restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int acc = 0;
#pragma unroll
    for (int r = 0; r < SCAN_ITEMS; r++) {
        int64_t i = base + r * SCAN_THREADS + threadIdx.x;
        if (i < n) acc += in[i];
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

__global__ void k_tile_apply(const int32_t *__restrict__ in, int32_t *__restrict__ out, int64_t n,
                             const int32_t *__restrict__ sums) {
    __shared__ int32_t tile[SCAN_TILE];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
#pragma unroll
    for (int r = 0; r < SCAN_ITEMS; r++) {
        int64_t i = base + r * SCAN_THREADS + threadIdx.x;
        tile[r * SCAN_THREADS + threadIdx.x] = i < n ? in[i] : 0;
    }
    __syncthreads();
    int loc[SCAN_ITEMS];
    int acc = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        loc[k] = acc;
        acc += tile[threadIdx.x * SCAN_ITEMS + k];
    }
    __shared__ int total;
    int ex = block_excl_scan<SCAN_THREADS>(acc, &total) + sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) tile[threadIdx.x * SCAN_ITEMS + k] = ex + loc[k];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < SCAN_ITEMS; r++) {
        int64_t i = base + r * SCAN_THREADS + threadIdx.x;
        if (i < n) out[i] = tile[r * SCAN_THREADS + threadIdx.x];
    }
    if (base + SCAN_TILE >= n && threadIdx.x == 0) {
        // the last tile also writes the grand total
        out[n] = sums[blockIdx.x] + total;
    }
}

}  // namespace

void exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s) {
    if (n == 0) {
        TM_CUDA(cudaMemsetAsync(out, 0, sizeof(int32_t), s));
        return;
    }
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    int32_t *sums = dev_alloc_n<int32_t>(tiles, s);
    TM_LAUNCH(k_tile_sums, (unsigned)tiles, SCAN_THREADS, 0, s, in, n, sums);
    TM_LAUNCH(k_scan_sums, 1, SCAN_THREADS, 0, s, sums, tiles);
    TM_LAUNCH(k_tile_apply, (unsigned)tiles, SCAN_THREADS, 0, s, in, out, n, sums);
    dev_free(sums, s);
}

// ------------------------------------------------------------ radix sort

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RADIX = 256;

// Items per thread: a tile (keys + values staged in shared memory) stays
// under the 48 KB static shared-memory limit.
template <typename K>
struct RsTile {
    static constexpr int ITEMS = sizeof(K) == 4 ? 16 : 8;
    static constexpr int TILE = RS_THREADS * ITEMS;
};

template <typename K>
__global__ void k_radix_hist(const K *__restrict__ keys, int64_t n, int shift,
                             int32_t *__restrict__ hist, int64_t ntiles) {
    constexpr int RS_ITEMS = RsTile<K>::ITEMS, RS_TILE = RsTile<K>::TILE;
    __shared__ int h[RADIX];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int r = 0; r < RS_ITEMS; r++) {
        int64_t i = base + r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & (RADIX - 1)], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

template <typename K>
__global__ void __launch_bounds__(RS_THREADS)
    k_radix_scatter(const K *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                    K *__restrict__ keys_out, uint32_t *__restrict__ vals_out, int64_t n,
                    int shift, const int32_t *__restrict__ base_off, int64_t ntiles) {
    constexpr int RS_ITEMS = RsTile<K>::ITEMS, RS_TILE = RsTile<K>::TILE;
    __shared__ K sk[RS_TILE];
    __shared__ uint32_t sv[RS_TILE];
    __shared__ int digit_start[RADIX];  // tile-local exclusive start of each digit
    __shared__ int running[RADIX];      // items of each digit placed so far
    __shared__ int warp_cnt[RS_WARPS][RADIX];
    __shared__ int gbase[RADIX];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    const int tile_n = (int)(n - base < RS_TILE ? n - base : RS_TILE);

    // tile histogram -> digit_start
    running[tid] = 0;
    for (int w = 0; w < RS_WARPS; w++) warp_cnt[w][tid] = 0;
    __syncthreads();
    for (int r = 0; r < RS_ITEMS; r++) {
        int li = r * RS_THREADS + tid;
        if (li < tile_n) atomicAdd(&running[(unsigned)(keys_in[base + li] >> shift) & (RADIX - 1)], 1);
    }
    __syncthreads();
    {
        __shared__ int total;
        int c = running[tid];
        int ex = block_excl_scan<RS_THREADS>(c, &total);
        digit_start[tid] = ex;
        running[tid] = 0;
        gbase[tid] = base_off[(int64_t)tid * ntiles + blockIdx.x];
    }
    __syncthreads();

    const unsigned lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < RS_ITEMS; r++) {
        int li = r * RS_THREADS + tid;
        bool valid = li < tile_n;
        K key = valid ? keys_in[base + li] : K(0);
        uint32_t val = valid ? vals_in[base + li] : 0u;
        int d = valid ? (int)((unsigned)(key >> shift) & (RADIX - 1)) : RADIX;  // RADIX: no digit
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int lrank = __popc(peers & lt_mask);
        int leader = __ffs(peers) - 1;
        if (valid && lane == leader) warp_cnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            // digit tid: prefix over the warps of this round
            int run = running[tid];
            for (int w = 0; w < RS_WARPS; w++) {
                int c = warp_cnt[w][tid];
                warp_cnt[w][tid] = run;
                run += c;
            }
            running[tid] = run;
        }
        __syncthreads();
        if (valid) {
            int pos = digit_start[d] + warp_cnt[warp][d] + lrank;
            sk[pos] = key;
            sv[pos] = val;
        }
        __syncthreads();
        for (int w = 0; w < RS_WARPS; w++) warp_cnt[w][tid] = 0;
        __syncthreads();
    }
    // write out: consecutive smem positions of one digit go to consecutive
    // global positions
    for (int r = 0; r < RS_ITEMS; r++) {
        int li = r * RS_THREADS + tid;
        if (li < tile_n) {
            K key = sk[li];
            int d = (int)((unsigned)(key >> shift) & (RADIX - 1));
            int64_t g = (int64_t)gbase[d] + (li - digit_start[d]);
            keys_out[g] = key;
            vals_out[g] = sv[li];
        }
    }
}

template <typename K>
void radix_sort_impl(K *keys, uint32_t *vals, K *keys_tmp, uint32_t *vals_tmp, int64_t n,
                     int bits, cudaStream_t s, K **keys_out, uint32_t **vals_out) {
    K *kin = keys, *kout = keys_tmp;
    uint32_t *vin = vals, *vout = vals_tmp;
    if (n > 1 && bits > 0) {
        constexpr int RS_TILE = RsTile<K>::TILE;
        const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
        int32_t *hist = dev_alloc_n<int32_t>(RADIX * ntiles + 1, s);
        for (int shift = 0; shift < bits; shift += 8) {
            TM_LAUNCH(k_radix_hist<K>, (unsigned)ntiles, RS_THREADS, 0, s, kin, n, shift, hist,
                      ntiles);
            exclusive_scan_i32(hist, hist, RADIX * ntiles, s);
            TM_LAUNCH(k_radix_scatter<K>, (unsigned)ntiles, RS_THREADS, 0, s, kin, vin, kout,
                      vout, n, shift, hist, ntiles);
            K *tk = kin;
            kin = kout;
            kout = tk;
            uint32_t *tv = vin;
            vin = vout;
            vout = tv;
        }
        dev_free(hist, s);
    }
    *keys_out = kin;
    *vals_out = vin;
}

}  // namespace

void radix_sort_u32(uint32_t *keys, uint32_t *vals, uint32_t *keys_tmp, uint32_t *vals_tmp,
                    int64_t n, int bits, cudaStream_t s, uint32_t **keys_out,
                    uint32_t **vals_out) {
    radix_sort_impl<uint32_t>(keys, vals, keys_tmp, vals_tmp, n, bits, s, keys_out, vals_out);
}

void radix_sort_u64(uint64_t *keys, uint32_t *vals, uint64_t *keys_tmp, uint32_t *vals_tmp,
                    int64_t n, int bits, cudaStream_t s, uint64_t **keys_out,
                    uint32_t **vals_out) {
    radix_sort_impl<uint64_t>(keys, vals, keys_tmp, vals_tmp, n, bits, s, keys_out, vals_out);
}

}  // namespace tmi
