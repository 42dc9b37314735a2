// Counting kernels: FAST-Star/Pair (Alg. 1) and FAST-Tri (Alg. 2) restated
// for a data-parallel GPU sweep. Both produce exactly the paper's counters;
// the restatements are derived in the comments below.
//
// Notation for one centre u: S = S_u in (t, edge id) order, positions are
// global indices into g.T; C_in(p) = inward entries before position p
// (TEnt::cin, a global prefix, so only differences inside one centre are
// used) and C_o(p) = p - C_in(p). For an entry r: W(r) = [lo(r), r), the
// earlier entries with t_r - t_p <= delta; F(r) = (r, hi(r)], the later
// entries with t_q - t_r <= delta.
//
// Star/Pair (Alg. 1 counts, per third edge r with node w and dir d3):
//   Pair[d1,d2,d3]     += pairs (a < b) in W(r) with node w, dirs (d1, d2)
//   Star-II[d1,d2,d3]  += sum over a in W(r), node w, dir d1, of the d2
//                         entries strictly between a and r, minus the Pair term
//   Star-I[d1,d2,d3]   += sum over b in W(r), node w, dir d2, of the d1
//                         entries in [lo(r), b), minus the Pair term
//   Star-III[d1,d2,d3] += (same-node pairs in W(r), any node) - Pair term.
// The "same-node pairs in W(r)" total is not local to w; summed over all r of
// one direction d3 it equals
//   sum_q n_q[d1] * #(d3 entries after q)  -  sum_p f_p[d2] * #(d3 entries after hi(p))
// with d2 = dir(q) in the first sum and d1 = dir(p) in the second, where
// n_q[d] counts same-node entries of direction d in W(q) and f_p[d] those in
// F(p). (Pairs enter the window when their later entry arrives and leave when
// the earlier one drops out, which happens exactly for the r after hi(p).)
// Every term is local to one entry and its same-neighbour entries, which are
// reached through the prev/next links: no per-centre hash table is needed.
//
// Tri (Alg. 2): only type II is computed. Each triangle instance adds exactly
// one count to a type-I, a type-II and a type-III cell of the same class
// (Sec. IV-B, "counted three times"), so the type-I and type-III cells are
// filled from type II by the rotation identity
//   Tri[II,di,dj,dk] = Tri[I,!dk,!dj,!di] = Tri[III,!di,dk,dj].
// Type II at centre u for the later u-edge e_j = r (node w): the pairs
// (e_i in W(r) with node x != w, e_k in E_(x,w)) with e_i < e_k < e_j. The
// kernel enumerates the smaller of W_u(r) and W_w(twin of r) and counts the
// matching edges of the pair list by binary search on rank.
#include "tm_internal.cuh"

namespace tmi {

namespace {

constexpr int THREADS = 256;

__device__ __forceinline__ int dir_of(uint32_t nbr) { return (int)(nbr >> 31); }
__device__ __forceinline__ uint32_t node_of(uint32_t nbr) { return nbr & 0x7fffffffu; }

// First position p in [b, r] with T[p].t >= bound; T[r].t >= bound holds.
__device__ __forceinline__ int32_t gallop_lo(const TEnt *__restrict__ T, int32_t b, int32_t r,
                                             int64_t bound) {
    int32_t hi = r, lo = b - 1, step = 1;
    while (true) {
        int32_t p = hi - step;
        if (p < b) break;
        if (T[p].t < bound) {
            lo = p;
            break;
        }
        hi = p;
        step <<= 1;
    }
    while (hi - lo > 1) {
        int32_t mid = lo + ((hi - lo) >> 1);
        if (T[mid].t >= bound) hi = mid;
        else lo = mid;
    }
    return hi;
}

// Last position q in [r, e) with T[q].t - tr <= delta.
__device__ __forceinline__ int32_t gallop_hi(const TEnt *__restrict__ T, int32_t r, int32_t e,
                                             int64_t tr, int64_t delta) {
    int32_t lo = r, hi = e, step = 1;
    while (true) {
        int32_t q = lo + step;
        if (q >= e) break;
        if (T[q].t - tr > delta) {
            hi = q;
            break;
        }
        lo = q;
        step <<= 1;
    }
    while (hi - lo > 1) {
        int32_t mid = lo + ((hi - lo) >> 1);
        if (T[mid].t - tr <= delta) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Cells are flat: Star ((T*2+a)*2+b)*2+c at 0..23, Pair (a*2+b)*2+c at
// 24..31, Tri ((T*2+a)*2+b)*2+c at 32..55.
template <int NC>
__device__ void block_flush(const unsigned long long (&acc)[NC], int cell0,
                            unsigned long long *__restrict__ cells) {
    __shared__ unsigned long long red[NC];
    if (threadIdx.x < NC) red[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NC; c++) {
        unsigned long long v = acc[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&red[c], v);
    }
    __syncthreads();
    if (threadIdx.x < NC && red[threadIdx.x]) atomicAdd(&cells[cell0 + threadIdx.x], red[threadIdx.x]);
}

// Accumulator index helpers (local arrays with compile-time indices).
//   acc[0..7]   Pair[d1][d2][d3]
//   acc[8..15]  Star-I[d1][d2][d3]
//   acc[16..23] Star-II
//   acc[24..31] Star-III
#define IX(a, b, c) ((((a) * 2) + (b)) * 2 + (c))

template <int D3>
__device__ __forceinline__ void star_pair_entry(const TEnt *__restrict__ T,
                                                const int32_t *__restrict__ off, int64_t m2,
                                                int64_t m, int64_t delta, int32_t r,
                                                const TEnt &e, unsigned long long (&acc)[32]) {
    const int64_t tr = e.t;
    // backward walk over same-neighbour entries inside W(r)
    uint64_t n[2] = {0, 0}, c2s[2][2] = {{0, 0}, {0, 0}};
    uint64_t X[2][2] = {{0, 0}, {0, 0}};   // X[d1][d2]: d2 entries strictly between a and r
    uint64_t Yp[2][2] = {{0, 0}, {0, 0}};  // Yp[d2][d1]: d1 entries in [S_u begin, b)
    const int32_t cin_r = e.cin;
    int32_t a = e.prev, cur = r;
    bool any = false;
    while (a >= 0 && a < cur) {  // links strictly decrease: the walk always ends
        const TEnt ea = T[a];
        if (tr - ea.t > delta) break;
        any = true;
        const int da = dir_of(ea.nbr);
        // pairs (a, later same-node entries in the window)
        c2s[da][0] += n[0];
        c2s[da][1] += n[1];
        n[da] += 1;
        const int64_t between_in = (int64_t)cin_r - (ea.cin + da);
        const int64_t between_o = (int64_t)(r - a - 1) - between_in;
        X[da][0] += (uint64_t)between_o;
        X[da][1] += (uint64_t)between_in;
        Yp[da][0] += (uint64_t)(a - ea.cin);  // C_o(a)
        Yp[da][1] += (uint64_t)ea.cin;        // C_in(a)
        cur = a;
        a = ea.prev;
    }
    const int32_t u = e.centre;
    const int32_t seg_end = off[u + 1];
    const int64_t cin_end = seg_end < m2 ? (int64_t)T[seg_end].cin : m;
    if (any) {
        const int32_t lo = gallop_lo(T, off[u], r, tr - delta);
        const int64_t cin_lo = T[lo].cin;
        const int64_t co_lo = (int64_t)lo - cin_lo;
#pragma unroll
        for (int d1 = 0; d1 < 2; d1++)
#pragma unroll
            for (int d2 = 0; d2 < 2; d2++) {
                const uint64_t s = c2s[d1][d2];
                acc[IX(d1, d2, D3)] += s;                                         // Pair
                acc[16 + IX(d1, d2, D3)] += X[d1][d2] - s;                        // Star-II
                const uint64_t base = d1 ? (uint64_t)cin_lo : (uint64_t)co_lo;   // C_d1(lo)
                acc[8 + IX(d1, d2, D3)] += Yp[d2][d1] - n[d2] * base - s;         // Star-I
                acc[24 + IX(d1, d2, D3)] -= s;                                    // Star-III
            }
        // Star-III, pairs entering: n_r[d1] x #(d3' entries after r)
        const int64_t after_in = cin_end - (cin_r + D3);
        const int64_t after_o = (int64_t)(seg_end - r - 1) - after_in;
#pragma unroll
        for (int d1 = 0; d1 < 2; d1++) {
            acc[24 + IX(d1, D3, 0)] += n[d1] * (uint64_t)after_o;
            acc[24 + IX(d1, D3, 1)] += n[d1] * (uint64_t)after_in;
        }
    }
    // forward walk: same-neighbour entries inside F(r) (pairs leaving)
    int32_t b = e.next;
    uint64_t f[2] = {0, 0};
    cur = r;
    while (b > cur && b < m2) {  // links strictly increase: the walk always ends
        const TEnt eb = T[b];
        if (eb.t - tr > delta) break;
        f[dir_of(eb.nbr)] += 1;
        cur = b;
        b = eb.next;
    }
    if (f[0] + f[1]) {
        const int32_t hi = gallop_hi(T, r, seg_end, tr, delta);
        const TEnt eh = T[hi];
        const int64_t cin_h1 = (int64_t)eh.cin + dir_of(eh.nbr);  // C_in(hi+1)
        const int64_t after_in = cin_end - cin_h1;
        const int64_t after_o = (int64_t)(seg_end - hi - 1) - after_in;
#pragma unroll
        for (int d2 = 0; d2 < 2; d2++) {
            acc[24 + IX(D3, d2, 0)] -= f[d2] * (uint64_t)after_o;
            acc[24 + IX(D3, d2, 1)] -= f[d2] * (uint64_t)after_in;
        }
    }
}

__global__ void __launch_bounds__(THREADS)
    k_star_pair(const TEnt *__restrict__ T, const int32_t *__restrict__ off, int64_t m, int64_t delta,
                int32_t begin, int32_t end, unsigned long long *__restrict__ cells) {
    unsigned long long acc[32];
#pragma unroll
    for (int c = 0; c < 32; c++) acc[c] = 0;
    const int64_t m2 = 2 * m;
    for (int64_t i = begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < end;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = (int32_t)i;
        const TEnt e = T[r];
        if (dir_of(e.nbr)) star_pair_entry<1>(T, off, m2, m, delta, r, e, acc);
        else star_pair_entry<0>(T, off, m2, m, delta, r, e, acc);
    }
    // acc order: Pair, Star-I, Star-II, Star-III -> cells Star[T] at 0.., Pair at 24..
    unsigned long long star[24], pair[8];
#pragma unroll
    for (int c = 0; c < 8; c++) {
        pair[c] = acc[c];
        star[c] = acc[8 + c];
        star[8 + c] = acc[16 + c];
        star[16 + c] = acc[24 + c];
    }
    block_flush<24>(star, 0, cells);
    block_flush<8>(pair, 24, cells);
}

__device__ __forceinline__ int2 find_pair(const PairSlot *__restrict__ H, uint32_t mask,
                                          uint64_t key) {
    uint32_t h = hash_pair(key) & mask;
    for (uint32_t probe = 0; probe <= mask; probe++) {
        const PairSlot s = H[h];
        if (s.key == key) return make_int2(s.begin, s.end);
        if (s.key == EMPTY_KEY) break;
        h = (h + 1) & mask;
    }
    return make_int2(0, 0);
}

// First index in [b, e) with pl_rank >= x.
__device__ __forceinline__ int32_t lower_rank(const int32_t *__restrict__ pl, int32_t b, int32_t e,
                                              int32_t x) {
    while (b < e) {
        int32_t mid = b + ((e - b) >> 1);
        if (pl[mid] < x) b = mid + 1;
        else e = mid;
    }
    return b;
}

template <int DJ>
__device__ __forceinline__ void tri_entry(const DevGraph &g, int64_t delta, int32_t r,
                                          const TEnt &e, unsigned long long (&acc)[8]) {
    const TEnt *__restrict__ T = g.T;
    const int64_t tj = e.t;
    const uint32_t u = (uint32_t)e.centre, w = node_of(e.nbr);
    const int32_t lo_u = gallop_lo(T, g.off[u], r, tj - delta);
    const int32_t wu = r - lo_u;
    if (wu == 0) return;
    const int32_t twin = DJ == 0 ? g.pos_dst[e.rank] : g.pos_src[e.rank];
    const int32_t lo_w = gallop_lo(T, g.off[w], twin, tj - delta);
    const int32_t ww = twin - lo_w;
    if (ww == 0) return;
    if (wu <= ww) {
        // e_i in W_u(r), e_k in E_(x, w) with rank_i < rank_k < rank_j
        for (int32_t a = lo_u; a < r; a++) {
            const TEnt ea = T[a];
            const uint32_t x = node_of(ea.nbr);
            if (x == w) continue;
            const int2 run = find_pair(g.hash, g.hash_mask, pair_key(x, w));
            if (run.x == run.y) continue;
            const int32_t k0 = lower_rank(g.pl_rank, run.x, run.y, ea.rank + 1);
            const int32_t k1 = lower_rank(g.pl_rank, k0, run.y, e.rank);
            const int32_t cnt = k1 - k0;
            if (cnt == 0) continue;
            const int32_t fmin = g.pl_cum[k1] - g.pl_cum[k0];  // edges whose source is min(x, w)
            const int32_t from_x = x < w ? fmin : cnt - fmin;   // e_k = x -> w: o w.r.t. x
            const int di = dir_of(ea.nbr);
            if (di) {
                acc[IX(1, DJ, 0)] += (unsigned long long)from_x;
                acc[IX(1, DJ, 1)] += (unsigned long long)(cnt - from_x);
            } else {
                acc[IX(0, DJ, 0)] += (unsigned long long)from_x;
                acc[IX(0, DJ, 1)] += (unsigned long long)(cnt - from_x);
            }
        }
    } else {
        // e_k in W_w(twin) with node x != u; e_i in E_(u, x) at positions >= lo_u
        // of S_u, i.e. rank >= rank(T[lo_u]), and rank_i < rank_k
        const int32_t rank_lo = T[lo_u].rank;
        for (int32_t k = lo_w; k < twin; k++) {
            const TEnt ek = T[k];
            const uint32_t x = node_of(ek.nbr);
            if (x == u) continue;
            const int2 run = find_pair(g.hash, g.hash_mask, pair_key(u, x));
            if (run.x == run.y) continue;
            const int32_t k0 = lower_rank(g.pl_rank, run.x, run.y, rank_lo);
            const int32_t k1 = lower_rank(g.pl_rank, k0, run.y, ek.rank);
            const int32_t cnt = k1 - k0;
            if (cnt == 0) continue;
            const int32_t fmin = g.pl_cum[k1] - g.pl_cum[k0];
            const int32_t from_u = u < x ? fmin : cnt - fmin;  // e_i = u -> x: o w.r.t. u
            const int dk = 1 - dir_of(ek.nbr);                  // e_k w.r.t. x
            if (dk) {
                acc[IX(0, DJ, 1)] += (unsigned long long)from_u;
                acc[IX(1, DJ, 1)] += (unsigned long long)(cnt - from_u);
            } else {
                acc[IX(0, DJ, 0)] += (unsigned long long)from_u;
                acc[IX(1, DJ, 0)] += (unsigned long long)(cnt - from_u);
            }
        }
    }
}

__global__ void __launch_bounds__(THREADS)
    k_tri(const DevGraph g, int64_t delta, int32_t begin, int32_t end,
          unsigned long long *__restrict__ cells) {
    unsigned long long acc[8];
#pragma unroll
    for (int c = 0; c < 8; c++) acc[c] = 0;
    for (int64_t i = begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < end;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = (int32_t)i;
        const TEnt e = g.T[r];
        if (dir_of(e.nbr)) tri_entry<1>(g, delta, r, e, acc);
        else tri_entry<0>(g, delta, r, e, acc);
    }
    // type II lives at Tri cells 8..15 (T = 1)
    block_flush<8>(acc, 32 + 8, cells);
}

__global__ void k_fill_tri_types(unsigned long long *cells) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long *tri = cells + 32;
    for (int di = 0; di < 2; di++)
        for (int dj = 0; dj < 2; dj++)
            for (int dk = 0; dk < 2; dk++) {
                const unsigned long long v = tri[8 + IX(di, dj, dk)];
                tri[IX(1 - dk, 1 - dj, 1 - di)] = v;       // type I
                tri[16 + IX(1 - di, dk, dj)] = v;          // type III
            }
}

}  // namespace

void launch_count(const DevGraph &g, int64_t delta, int32_t begin, int32_t end,
                  unsigned long long *dev_cells, cudaStream_t s) {
    if (end <= begin) return;
    const int64_t n = end - begin;
    int64_t blocks = (n + THREADS - 1) / THREADS;
    const int64_t cap = (int64_t)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    {
        PhaseTimer pt(TM_PH_STAR_PAIR, s);
        TM_LAUNCH(k_star_pair, (unsigned)blocks, THREADS, 0, s, g.T, g.off, g.m, delta, begin, end,
                  dev_cells);
    }
    {
        PhaseTimer pt(TM_PH_TRI, s);
        TM_LAUNCH(k_tri, (unsigned)blocks, THREADS, 0, s, g, delta, begin, end, dev_cells);
    }
}

void launch_fill_tri_types(unsigned long long *dev_cells, cudaStream_t s) {
    TM_LAUNCH(k_fill_tri_types, 1, 32, 0, s, dev_cells);
}

}  // namespace tmi
