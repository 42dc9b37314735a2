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
constexpr int RADIX = 256;  // 8-bit digits; one thread per digit in the tile scan

// Items per lane: a warp ranks 32 * ITEMS consecutive items. Wide key/value
// pairs use half the items to keep registers (one block of 256 threads needs
// them for the keys, values and ranks of its tile) and shared memory down.
template <typename K, typename V>
struct RsCfg {
    static constexpr int ITEMS = sizeof(K) + sizeof(V) <= 8 ? 16 : 8;
    static constexpr int TILE = RS_THREADS * ITEMS;
};

template <typename K>
__device__ __forceinline__ int digit_of(K k, int shift) {
    return (int)((unsigned)(k >> shift) & (RADIX - 1));
}

// Lanes of the warp holding the same value d (9 bits: digits 0..255 and the
// "no item" marker 256), from nine ballots: a lane keeps the lanes that agree
// with it on every bit.
__device__ __forceinline__ unsigned warp_peers9(int d) {
    unsigned peers = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < 9; b++) {
        const bool bit = (d >> b) & 1;
        const unsigned bal = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bal : ~bal;
    }
    return peers;
}

// Per-tile digit histogram: 128-bit loads, warp-private shared counters
// (plain shared atomics; a skewed digit only contends inside one warp).
template <typename K, int RS_ITEMS>
__global__ void __launch_bounds__(RS_THREADS)
    k_radix_hist(const K *__restrict__ keys, int64_t n, int shift, int32_t *__restrict__ hist,
                 int64_t ntiles) {
    constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
    constexpr int PER_VEC = 16 / sizeof(K);
    __shared__ int h[RS_WARPS][RADIX];
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * RADIX; i += RS_THREADS) (&h[0][0])[i] = 0;
    __syncthreads();
    const int64_t tbase = (int64_t)blockIdx.x * RS_TILE;
    const int tile_n = (int)(n - tbase < RS_TILE ? n - tbase : RS_TILE);
    if (tile_n == RS_TILE) {
        const uint4 *v = reinterpret_cast<const uint4 *>(keys + tbase);
#pragma unroll
        for (int r = 0; r < RS_ITEMS / PER_VEC; r++) {
            const uint4 q = v[r * RS_THREADS + threadIdx.x];
            const K *kk = reinterpret_cast<const K *>(&q);
#pragma unroll
            for (int c = 0; c < PER_VEC; c++) atomicAdd(&h[warp][digit_of(kk[c], shift)], 1);
        }
    } else {
        for (int li = threadIdx.x; li < tile_n; li += RS_THREADS)
            atomicAdd(&h[warp][digit_of(keys[tbase + li], shift)], 1);
    }
    __syncthreads();
    int c = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; w++) c += h[w][threadIdx.x];
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = c;
}

// Stable scatter of one tile. Warp w ranks its 512 consecutive items in
// order with warp-private digit counters; one block-wide scan turns the
// counters into tile offsets; the tile is reordered in shared memory and
// written out so that each digit's run goes to consecutive addresses.
template <typename K, typename V>
__global__ void __launch_bounds__(RS_THREADS, 4)
    k_radix_scatter(const K *__restrict__ keys_in, const V *__restrict__ vals_in,
                    K *__restrict__ keys_out, V *__restrict__ vals_out, int64_t n, int shift,
                    const int32_t *__restrict__ base_off, int64_t ntiles) {
    constexpr int RS_ITEMS = RsCfg<K, V>::ITEMS, RS_TILE = RsCfg<K, V>::TILE;
    extern __shared__ __align__(16) unsigned char smem[];
    int *cnt = reinterpret_cast<int *>(smem);                       // [RS_WARPS][RADIX]
    K *sk = reinterpret_cast<K *>(cnt + RS_WARPS * RADIX);          // [RS_TILE]
    V *sv = reinterpret_cast<V *>(sk + RS_TILE);                    // [RS_TILE]
    __shared__ int digit_off[RADIX];
    __shared__ int gbase[RADIX];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t tbase = (int64_t)blockIdx.x * RS_TILE;
    const int tile_n = (int)(n - tbase < RS_TILE ? n - tbase : RS_TILE);
    for (int i = tid; i < RS_WARPS * RADIX; i += RS_THREADS) cnt[i] = 0;
    __syncthreads();

    K key[RS_ITEMS];
    V val[RS_ITEMS];
    int rnk[RS_ITEMS];
    const unsigned lt_mask = (1u << lane) - 1u;
    const int wofs = warp * 32 * RS_ITEMS;
#pragma unroll
    for (int r = 0; r < RS_ITEMS; r++) {
        const int li = wofs + r * 32 + lane;
        const bool valid = li < tile_n;
        key[r] = valid ? keys_in[tbase + li] : K(0);
        val[r] = valid ? vals_in[tbase + li] : V{};
        const int d = valid ? digit_of(key[r], shift) : RADIX;
        const unsigned peers = warp_peers9(d);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (d < RADIX && lane == leader) base = atomicAdd(&cnt[warp * RADIX + d], __popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        rnk[r] = base + __popc(peers & lt_mask);
    }
    __syncthreads();
    {
        // digit `tid`: exclusive prefix over the warps, then over the digits
        int tot = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) {
            const int c = cnt[w * RADIX + tid];
            cnt[w * RADIX + tid] = tot;
            tot += c;
        }
        __shared__ int total;
        const int ex = block_excl_scan<RS_THREADS>(tot, &total);
        digit_off[tid] = ex;
        gbase[tid] = base_off[(int64_t)tid * ntiles + blockIdx.x];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ITEMS; r++) {
        const int li = wofs + r * 32 + lane;
        if (li < tile_n) {
            const int d = digit_of(key[r], shift);
            const int pos = digit_off[d] + cnt[warp * RADIX + d] + rnk[r];
            sk[pos] = key[r];
            sv[pos] = val[r];
        }
    }
    __syncthreads();
    for (int li = tid; li < tile_n; li += RS_THREADS) {
        const K k = sk[li];
        const int d = digit_of(k, shift);
        const int64_t g = (int64_t)gbase[d] + (li - digit_off[d]);
        keys_out[g] = k;
        vals_out[g] = sv[li];
    }
}

template <typename K, typename V>
void radix_sort_impl(K *keys, V *vals, K *keys_tmp, V *vals_tmp, int64_t n, int bits,
                     cudaStream_t s, K **keys_out, V **vals_out) {
    K *kin = keys, *kout = keys_tmp;
    V *vin = vals, *vout = vals_tmp;
    if ((reinterpret_cast<uintptr_t>(keys) | reinterpret_cast<uintptr_t>(keys_tmp)) & 15)
        fail(TM_EINVAL, "radix sort: key buffers must be 16-byte aligned");
    if (n > 1 && bits > 0) {
        constexpr int RS_TILE = RsCfg<K, V>::TILE;
        const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
        const size_t smem = sizeof(int) * RS_WARPS * RADIX + (sizeof(K) + sizeof(V)) * RS_TILE;
        static bool attr_set = false;
        if (!attr_set) {
            TM_CUDA(cudaFuncSetAttribute(k_radix_scatter<K, V>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr_set = true;
        }
        int32_t *hist = dev_alloc_n<int32_t>(RADIX * ntiles + 1, s);
        for (int shift = 0; shift < bits; shift += 8) {
            TM_LAUNCH((k_radix_hist<K, RsCfg<K, V>::ITEMS>), (unsigned)ntiles, RS_THREADS, 0, s, kin, n, shift, hist,
                      ntiles);
            exclusive_scan_i32(hist, hist, RADIX * ntiles, s);
            TM_LAUNCH((k_radix_scatter<K, V>), (unsigned)ntiles, RS_THREADS, smem, s, kin, vin,
                      kout, vout, n, shift, hist, ntiles);
            K *tk = kin;
            kin = kout;
            kout = tk;
            V *tv = vin;
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
    radix_sort_impl<uint32_t, uint32_t>(keys, vals, keys_tmp, vals_tmp, n, bits, s, keys_out,
                                        vals_out);
}

void radix_sort_u64(uint64_t *keys, uint32_t *vals, uint64_t *keys_tmp, uint32_t *vals_tmp,
                    int64_t n, int bits, cudaStream_t s, uint64_t **keys_out,
                    uint32_t **vals_out) {
    radix_sort_impl<uint64_t, uint32_t>(keys, vals, keys_tmp, vals_tmp, n, bits, s, keys_out,
                                        vals_out);
}

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

void radix_sort_u32_ent(uint32_t *keys, EntryPayload *vals, uint32_t *keys_tmp,
                        EntryPayload *vals_tmp, int64_t n, int bits, cudaStream_t s,
                        uint32_t **keys_out, EntryPayload **vals_out) {
    radix_sort_impl<uint32_t, EntryPayload>(keys, vals, keys_tmp, vals_tmp, n, bits, s, keys_out,
                                            vals_out);
}

void radix_sort_u32_v64(uint32_t *keys, uint64_t *vals, uint32_t *keys_tmp, uint64_t *vals_tmp,
                        int64_t n, int bits, cudaStream_t s, uint32_t **keys_out,
                        uint64_t **vals_out) {
    radix_sort_impl<uint32_t, uint64_t>(keys, vals, keys_tmp, vals_tmp, n, bits, s, keys_out,
                                        vals_out);
}

void radix_sort_u64_v64(uint64_t *keys, uint64_t *vals, uint64_t *keys_tmp, uint64_t *vals_tmp,
                        int64_t n, int bits, cudaStream_t s, uint64_t **keys_out,
                        uint64_t **vals_out) {
    radix_sort_impl<uint64_t, uint64_t>(keys, vals, keys_tmp, vals_tmp, n, bits, s, keys_out,
                                        vals_out);
}

}  // namespace tmi
