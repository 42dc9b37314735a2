// Stable LSD radix sort kernels (8-bit digits), templated on where a pass
// reads its items (In) and where it writes them (Out), so that the first pass
// of a sort can generate its items from another array and the last pass can
// write them in their final form, without a separate kernel on either side.
//
// Each pass: per-tile digit histograms, one exclusive scan over (digit, tile),
// and a stable scatter that ranks a tile in shared memory and writes every
// digit's run with consecutive addresses.
//
// In:  valid(i) (whether item i takes part: a first pass may drop items),
//      key(i) -> K, val(i) -> V; VEC_KEYS and keys (128-bit key loads, only
//      for inputs whose items are all valid)
// Out: store(g, K, const V&), g in [0, number of valid items)
#pragma once

#include <atomic>

#include "tm_internal.cuh"

namespace tmi {
namespace {  // each translation unit instantiates its own kernels
namespace radix {

constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;
constexpr int RADIX = 256;  // 8-bit digits; one thread per digit in the tile scan

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

// Items per lane: a warp ranks 32 * ITEMS consecutive items. Wide key/value
// pairs use half the items to keep registers (one block of 256 threads needs
// them for the keys, values and ranks of its tile) and shared memory down.
template <typename K, typename V>
struct Cfg {
    static constexpr int ITEMS = sizeof(K) + sizeof(V) <= 8 ? 16 : 8;
    static constexpr int TILE = THREADS * ITEMS;
};

template <typename K>
__device__ __forceinline__ int digit_of(K k, int shift) {
    return (int)((unsigned)(k >> shift) & (RADIX - 1));
}

// Plain arrays on either side of a pass.
template <typename K, typename V>
struct ArrayIn {
    static constexpr bool VEC_KEYS = true;
    const K *__restrict__ keys;
    const V *__restrict__ vals;
    __device__ __forceinline__ bool valid(int64_t) const { return true; }
    __device__ __forceinline__ K key(int64_t i) const { return keys[i]; }
    __device__ __forceinline__ V val(int64_t i) const { return vals[i]; }
};

template <typename K, typename V>
struct ArrayOut {
    K *__restrict__ keys;
    V *__restrict__ vals;
    __device__ __forceinline__ void store(int64_t g, K k, const V &v) const {
        keys[g] = k;
        vals[g] = v;
    }
};

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

// Per-tile digit histogram (warp-private shared counters; a skewed digit
// only contends inside one warp), 128-bit key loads where the keys are an
// array.
template <typename K, int ITEMS, typename In>
__global__ void __launch_bounds__(THREADS)
    k_radix_hist(In in, int64_t n, int shift, int32_t *__restrict__ hist, int64_t ntiles) {
    constexpr int TILE = THREADS * ITEMS;
    __shared__ int h[WARPS][RADIX];
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < WARPS * RADIX; i += THREADS) (&h[0][0])[i] = 0;
    __syncthreads();
    const int64_t tbase = (int64_t)blockIdx.x * TILE;
    const int tile_n = (int)(n - tbase < TILE ? n - tbase : TILE);
    if constexpr (In::VEC_KEYS) {
        constexpr int PER_VEC = 16 / sizeof(K);
        if (tile_n == TILE) {
            const uint4 *v = reinterpret_cast<const uint4 *>(in.keys + tbase);
#pragma unroll
            for (int r = 0; r < ITEMS / PER_VEC; r++) {
                const uint4 q = v[r * THREADS + threadIdx.x];
                const K *kk = reinterpret_cast<const K *>(&q);
#pragma unroll
                for (int c = 0; c < PER_VEC; c++) atomicAdd(&h[warp][digit_of(kk[c], shift)], 1);
            }
        } else {
            for (int li = threadIdx.x; li < tile_n; li += THREADS)
                atomicAdd(&h[warp][digit_of(in.key(tbase + li), shift)], 1);
        }
    } else {
        for (int li = threadIdx.x; li < tile_n; li += THREADS)
            if (in.valid(tbase + li)) atomicAdd(&h[warp][digit_of(in.key(tbase + li), shift)], 1);
    }
    __syncthreads();
    int c = 0;
#pragma unroll
    for (int w = 0; w < WARPS; w++) c += h[w][threadIdx.x];
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = c;
}

// Stable scatter of one tile. The tile's keys are loaded first (all loads in
// flight together), then warp w ranks its 32 * ITEMS consecutive items in
// order with warp-private digit counters; the values are loaded while one
// block-wide scan turns the counters into tile offsets; the tile is reordered
// in shared memory and written out so that each digit's run goes to
// consecutive addresses.
template <typename K, typename V, typename In, typename Out>
__global__ void __launch_bounds__(THREADS, 4)
    k_radix_scatter(In in, Out out, int64_t n, int shift, const int32_t *__restrict__ base_off,
                    int64_t ntiles) {
    constexpr int ITEMS = Cfg<K, V>::ITEMS, TILE = Cfg<K, V>::TILE;
    extern __shared__ __align__(16) unsigned char smem[];
    int *cnt = reinterpret_cast<int *>(smem);               // [WARPS][RADIX]
    K *sk = reinterpret_cast<K *>(cnt + WARPS * RADIX);     // [TILE]
    V *sv = reinterpret_cast<V *>(sk + TILE);               // [TILE]
    __shared__ int digit_off[RADIX];
    __shared__ int gbase[RADIX];
    __shared__ int tile_valid;  // items of the tile that take part

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t tbase = (int64_t)blockIdx.x * TILE;
    const int tile_n = (int)(n - tbase < TILE ? n - tbase : TILE);
    for (int i = tid; i < WARPS * RADIX; i += THREADS) cnt[i] = 0;

    K key[ITEMS];
    V val[ITEMS];
    int rnk[ITEMS];
    unsigned ok = 0;  // bit r: item r of this lane takes part
    const unsigned lt_mask = (1u << lane) - 1u;
    const int wofs = warp * 32 * ITEMS;
#pragma unroll
    for (int r = 0; r < ITEMS; r++) {
        const int li = wofs + r * 32 + lane;
        const bool v = li < tile_n && in.valid(tbase + li);
        ok |= (unsigned)v << r;
        key[r] = v ? in.key(tbase + li) : K(0);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < ITEMS; r++) {
        const int d = (ok >> r) & 1u ? digit_of(key[r], shift) : RADIX;
        const unsigned peers = warp_peers9(d);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (d < RADIX && lane == leader) base = atomicAdd(&cnt[warp * RADIX + d], __popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        rnk[r] = base + __popc(peers & lt_mask);
    }
#pragma unroll
    for (int r = 0; r < ITEMS; r++)
        val[r] = (ok >> r) & 1u ? in.val(tbase + wofs + r * 32 + lane) : V{};
    __syncthreads();
    {
        // digit `tid`: exclusive prefix over the warps, then over the digits
        int tot = 0;
#pragma unroll
        for (int w = 0; w < WARPS; w++) {
            const int c = cnt[w * RADIX + tid];
            cnt[w * RADIX + tid] = tot;
            tot += c;
        }
        const int ex = block_excl_scan<THREADS>(tot, &tile_valid);
        digit_off[tid] = ex;
        gbase[tid] = base_off[(int64_t)tid * ntiles + blockIdx.x];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < ITEMS; r++) {
        if ((ok >> r) & 1u) {
            const int d = digit_of(key[r], shift);
            const int pos = digit_off[d] + cnt[warp * RADIX + d] + rnk[r];
            sk[pos] = key[r];
            sv[pos] = val[r];
        }
    }
    __syncthreads();
    for (int li = tid; li < tile_valid; li += THREADS) {
        const K k = sk[li];
        const int d = digit_of(k, shift);
        out.store((int64_t)gbase[d] + (li - digit_off[d]), k, sv[li]);
    }
}

template <typename K, typename V>
constexpr size_t scatter_smem() {
    return sizeof(int) * WARPS * RADIX + (sizeof(K) + sizeof(V)) * Cfg<K, V>::TILE;
}

// One pass from the n items of `in` (valid or not) to `out` on digit `shift`;
// hist holds RADIX * ntiles + 1 counters.
template <typename K, typename V, typename In, typename Out>
void pass(In in, Out out, int64_t n, int shift, int32_t *hist, cudaStream_t s) {
    constexpr int TILE = Cfg<K, V>::TILE;
    const int64_t ntiles = (n + TILE - 1) / TILE;
    constexpr size_t smem = scatter_smem<K, V>();
    static std::atomic<unsigned long long> attr_devices{0};  // devices whose attribute is set
    const int dev = current_device_id();
    if (dev >= 64 || !((attr_devices.load() >> dev) & 1ull)) {
        TM_CUDA(cudaFuncSetAttribute(k_radix_scatter<K, V, In, Out>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (dev < 64) attr_devices.fetch_or(1ull << dev);
    }
    TM_LAUNCH((k_radix_hist<K, Cfg<K, V>::ITEMS, In>), (unsigned)ntiles, THREADS, 0, s, in, n,
              shift, hist, ntiles);
    exclusive_scan_i32(hist, hist, RADIX * ntiles, s);
    TM_LAUNCH((k_radix_scatter<K, V, In, Out>), (unsigned)ntiles, THREADS, smem, s, in, out, n,
              shift, hist, ntiles);
}

// Sorts the n valid items of the n_in items of `in` on the low `bits` bits of
// their keys (at least one pass, so that `out` is always written): the first
// pass reads `in`, the last writes `out`, the passes between ping-pong through
// (ka, va) and (kb, vb), which hold n items each. `out` must not be the buffer
// pair the last pass reads: (kb, vb) after an odd number of passes above one,
// (ka, va) after an even number.
template <typename K, typename V, typename In, typename Out>
void sort(In in, Out out, K *ka, V *va, K *kb, V *vb, int64_t n_in, int64_t n, int bits,
          cudaStream_t s) {
    if (n_in <= 0) return;
    if ((reinterpret_cast<uintptr_t>(ka) | reinterpret_cast<uintptr_t>(kb)) & 15)
        fail(TM_EINVAL, "radix sort: key buffers must be 16-byte aligned");
    const int passes = bits > 8 ? (bits + 7) / 8 : 1;
    const int64_t nmax = n_in > n ? n_in : n;
    const int64_t ntiles = (nmax + Cfg<K, V>::TILE - 1) / Cfg<K, V>::TILE;
    int32_t *hist = dev_alloc_n<int32_t>(RADIX * ntiles + 1, s);
    if (passes == 1) {
        pass<K, V>(in, out, n_in, 0, hist, s);
    } else {
        pass<K, V>(in, ArrayOut<K, V>{ka, va}, n_in, 0, hist, s);
        K *kc = ka, *kn = kb;
        V *vc = va, *vn = vb;
        for (int p = 1; p + 1 < passes; p++) {
            pass<K, V>(ArrayIn<K, V>{kc, vc}, ArrayOut<K, V>{kn, vn}, n, 8 * p, hist, s);
            K *tk = kc;
            kc = kn;
            kn = tk;
            V *tv = vc;
            vc = vn;
            vn = tv;
        }
        pass<K, V>(ArrayIn<K, V>{kc, vc}, out, n, 8 * (passes - 1), hist, s);
    }
    dev_free(hist, s);
}

}  // namespace radix
}  // namespace
}  // namespace tmi
