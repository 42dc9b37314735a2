// Counting kernels: FAST-Star/Pair (Alg. 1) and FAST-Tri (Alg. 2) restated
// for a data-parallel GPU sweep. Both produce exactly the paper's counters;
// the restatements are derived in the comments below.
//
// Notation for one centre u: S = S_u in (t, edge id) order, positions are
// global entry indices; C_in(p) = inward entries before position p (g.cin, a
// global prefix, so only differences inside one centre are used) and
// C_o(p) = p - C_in(p). For an entry r: W(r) = [lo(r), r), the
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
// (Sec. IV-B counts each instance three times), so the type-I and type-III
// cells are filled from type II by the rotation identity
//   Tri[II,di,dj,dk] = Tri[I,!dk,!dj,!di] = Tri[III,!di,dk,dj].
// Type II at centre u with later u-edge e_j = (u, w): pairs e_i < e_k < e_j
// with e_i = (u, x) in W_u(e_j) and e_k = (x, w), which then lies in
// W_w(e_j). So for each edge e_j the type-II triangles at BOTH of its
// endpoints are the same-neighbour matches between the two endpoint windows
// W_u(e_j) and W_w(e_j): a match (a in W_u, k in W_w) with a < k is centred at
// u, one with k < a at w. Each edge is joined once, at its source entry: the
// smaller window is enumerated and the matches are found in the bigger one
// through the pair list (hash lookup of E_(big, x), binary search on rank).
// k_tri_jobs lists the edges whose two windows are both non-empty and
// k_tri_join runs their joins; k_tri does both in one kernel without scratch.
//
// Star/Pair work lists: an entry has W(r) terms only if its previous
// same-neighbour entry p lies in W(r) (it is "back-active"), and F(p) holds a
// same-neighbour entry exactly when p's next one, r, is back-active with p.
// So k_window_lo lists the back-active entries while it finds every lo(r),
// and k_star_pair_list makes each of them produce its own W terms and its
// predecessor's F term; k_star_pair does the same per entry without scratch.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstring>
#include <vector>

#include "tm_internal.cuh"

namespace tmi {

namespace {

constexpr int THREADS = 256;
constexpr int WARPS_PER_BLOCK = THREADS / 32;

__device__ __forceinline__ int dir_of(uint32_t nbr) { return (int)(nbr >> 31); }

__device__ __forceinline__ int32_t warp_incl_scan_i32(int32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += o;
    }
    return v;
}
__device__ __forceinline__ uint32_t node_of(uint32_t nbr) { return nbr & 0x7fffffffu; }

// First position p in [b, r] with tt[p] >= bound; tt[r] >= bound holds.
__device__ __forceinline__ int32_t gallop_lo(const int64_t *__restrict__ tt, int32_t b, int32_t r,
                                             int64_t bound) {
    int32_t hi = r, lo = b - 1, step = 1;
    while (true) {
        int32_t p = hi - step;
        if (p < b) break;
        if (tt[p] < bound) {
            lo = p;
            break;
        }
        hi = p;
        step <<= 1;
    }
    while (hi - lo > 1) {
        int32_t mid = lo + ((hi - lo) >> 1);
        if (tt[mid] >= bound) hi = mid;
        else lo = mid;
    }
    return hi;
}

// Last position q in [r, e) with tt[q] - tr <= delta.
__device__ __forceinline__ int32_t gallop_hi(const int64_t *__restrict__ tt, int32_t r, int32_t e,
                                             int64_t tr, int64_t delta) {
    int32_t lo = r, hi = e, step = 1;
    while (true) {
        int32_t q = lo + step;
        if (q >= e) break;
        if (tt[q] - tr > delta) {
            hi = q;
            break;
        }
        lo = q;
        step <<= 1;
    }
    while (hi - lo > 1) {
        int32_t mid = lo + ((hi - lo) >> 1);
        if (tt[mid] - tr <= delta) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Cells are flat: Star ((T*2+a)*2+b)*2+c at 0..23, Pair (a*2+b)*2+c at
// 24..31, Tri ((T*2+a)*2+b)*2+c at 32..55.
// Adds acc[SRC + c] (c < NC) of every thread of the block into
// cells[cell0 + c]: warp shuffles, shared atomics, one global atomic per cell.
template <int NC, int SRC, int NA>
__device__ void block_flush(const unsigned long long (&acc)[NA], int cell0,
                            unsigned long long *__restrict__ cells) {
    __shared__ unsigned long long red[NC];
    __syncthreads();
    if (threadIdx.x < NC) red[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NC; c++) {
        unsigned long long v = acc[SRC + c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&red[c], v);
    }
    __syncthreads();
    if (threadIdx.x < NC && red[threadIdx.x]) atomicAdd(&cells[cell0 + threadIdx.x], red[threadIdx.x]);
}

// Star/Pair accumulator layout (shared memory, one set per block):
//   sacc[0..7]   Pair[d1][d2][d3]
//   sacc[8..15]  Star-I[d1][d2][d3]
//   sacc[16..23] Star-II
//   sacc[24..31] Star-III
// Most entries contribute nothing (no same-neighbour entry in their window),
// so contributions go straight to shared memory with atomics instead of
// living in 32 registers per thread.
#define IX(a, b, c) ((((a) * 2) + (b)) * 2 + (c))

__device__ __forceinline__ void add_cell(unsigned long long *sacc, int i, uint64_t v) {
    if (v) atomicAdd(&sacc[i], (unsigned long long)v);
}

// Block total of sacc[32] into the global cells (Star 0..23, Pair 24..31).
__device__ __forceinline__ void flush_star_pair(const unsigned long long *sacc,
                                                unsigned long long *__restrict__ cells) {
    if (threadIdx.x < 32) {
        const int i = threadIdx.x;
        const unsigned long long v = sacc[i];
        if (v) atomicAdd(&cells[i < 8 ? 24 + i : i - 8], v);
    }
}

// The contributions of entry r (direction D3), its window bounds searched
// here.
template <int D3>
__device__ __forceinline__ void star_pair_entry(const DevGraph &g, int64_t delta, int32_t r,
                                                int64_t tr, int32_t u, int2 lr,
                                                unsigned long long *sacc) {
    const int64_t *__restrict__ tt = g.tt;
    const int32_t seg_b = g.off[u], seg_end = g.off[u + 1];
    // W(r) and F(r) bounds from the neighbouring entries of S_u (local reads);
    // the same-neighbour links are followed only when they land inside.
    const bool wnd_back = lr.x >= 0 && r > seg_b && tr - tt[r - 1] <= delta;
    // the next same-neighbour entry lies in F(r) exactly when it is within delta
    const bool wnd_fwd = lr.y >= 0 && tt[lr.y] - tr <= delta;
    if (!wnd_back && !wnd_fwd) return;
    const int64_t cin_end = g.cin[seg_end];
    const int64_t cin_r = g.cin[r];
    if (wnd_back) {
        const int32_t lo = gallop_lo(tt, seg_b, r, tr - delta);
        if (lr.x >= lo) {
            // per direction d of the run entries: n_d (count), c2s_{d,d'} (pairs),
            // X_{d,d'} (d' entries strictly between a and r), Y_{d,d'} (d' entries
            // before b, as a prefix); kept in scalars so they stay in registers
            uint64_t n0 = 0, n1 = 0, c00 = 0, c01 = 0, c10 = 0, c11 = 0;
            uint64_t X00 = 0, X01 = 0, X10 = 0, X11 = 0, Y00 = 0, Y01 = 0, Y10 = 0, Y11 = 0;
            int32_t a = lr.x, cur = r;
            while (a >= lo && a < cur) {  // links strictly decrease: the walk always ends
                const int da = dir_of(g.tn[a].x);
                const int64_t cin_a = g.cin[a];
                const uint64_t between_in = (uint64_t)(cin_r - (cin_a + da));
                const uint64_t between_o = (uint64_t)(r - a - 1) - between_in;
                const uint64_t co_a = (uint64_t)(a - cin_a), ci_a = (uint64_t)cin_a;
                if (da) {  // pairs (a, later same-node entries in the window)
                    c10 += n0;
                    c11 += n1;
                    n1 += 1;
                    X10 += between_o;
                    X11 += between_in;
                    Y10 += co_a;
                    Y11 += ci_a;
                } else {
                    c00 += n0;
                    c01 += n1;
                    n0 += 1;
                    X00 += between_o;
                    X01 += between_in;
                    Y00 += co_a;
                    Y01 += ci_a;
                }
                cur = a;
                a = g.lk[a].x;
            }
            const uint64_t n[2] = {n0, n1};
            const uint64_t c2s[2][2] = {{c00, c01}, {c10, c11}};
            const uint64_t X[2][2] = {{X00, X01}, {X10, X11}};
            const uint64_t Yp[2][2] = {{Y00, Y01}, {Y10, Y11}};
            const int64_t cin_lo = g.cin[lo];
            const int64_t co_lo = (int64_t)lo - cin_lo;
#pragma unroll
            for (int d1 = 0; d1 < 2; d1++)
#pragma unroll
                for (int d2 = 0; d2 < 2; d2++) {
                    const uint64_t sp = c2s[d1][d2];
                    add_cell(sacc, IX(d1, d2, D3), sp);                                // Pair
                    add_cell(sacc, 16 + IX(d1, d2, D3), X[d1][d2] - sp);               // Star-II
                    const uint64_t base = d1 ? (uint64_t)cin_lo : (uint64_t)co_lo;    // C_d1(lo)
                    add_cell(sacc, 8 + IX(d1, d2, D3), Yp[d2][d1] - n[d2] * base - sp); // Star-I
                    add_cell(sacc, 24 + IX(d1, d2, D3), 0 - sp);                       // Star-III
                }
            // Star-III, pairs entering: n_r[d1] x #(d3' entries after r)
            const int64_t after_in = cin_end - (cin_r + D3);
            const int64_t after_o = (int64_t)(seg_end - r - 1) - after_in;
#pragma unroll
            for (int d1 = 0; d1 < 2; d1++) {
                add_cell(sacc, 24 + IX(d1, D3, 0), n[d1] * (uint64_t)after_o);
                add_cell(sacc, 24 + IX(d1, D3, 1), n[d1] * (uint64_t)after_in);
            }
        }
    }
    if (wnd_fwd) {
        const int32_t hi = gallop_hi(tt, lr.y, seg_end, tr, delta);  // hi >= lr.y
        {
            // same-neighbour entries inside F(r): pairs leaving after hi(r)
            uint64_t f0 = 0, f1 = 0;
            int32_t b = lr.y, cur = r;
            while (b > cur && b <= hi) {  // links strictly increase: the walk always ends
                if (dir_of(g.tn[b].x)) f1 += 1;
                else f0 += 1;
                cur = b;
                b = g.lk[b].y;
            }
            const uint64_t f[2] = {f0, f1};
            const int64_t cin_h1 = (int64_t)g.cin[hi] + dir_of(g.tn[hi].x);  // C_in(hi+1)
            const int64_t after_in = cin_end - cin_h1;
            const int64_t after_o = (int64_t)(seg_end - hi - 1) - after_in;
#pragma unroll
            for (int d2 = 0; d2 < 2; d2++) {
                add_cell(sacc, 24 + IX(D3, d2, 0), 0 - f[d2] * (uint64_t)after_o);
                add_cell(sacc, 24 + IX(D3, d2, 1), 0 - f[d2] * (uint64_t)after_in);
            }
        }
    }
}

// The contributions of a back-active entry r (its previous same-neighbour
// entry p = lk[r].x lies in W(r), lo(r) = lo_r) with the window starts known:
// r's own W(r) terms, and the F(p) term of p. p's next same-neighbour entry is
// r, so F(p) holds a same-neighbour entry exactly when r is back-active with
// p: the F terms of all entries are produced here, by the entries that
// follow them, and an entry whose predecessor is outside its window does
// nothing at all.
// Its counts go to the calling lane's copy of the 32 cells: cell i at
// lane_cells[i * SP_COPIES] (see k_star_pair_list).
constexpr int SP_COPIES = 33;  // 32 lane copies per cell, padded against bank conflicts

__device__ __forceinline__ void lane_add(unsigned long long *lane_cells, int i, uint64_t v) {
    if (v) atomicAdd(&lane_cells[i * SP_COPIES], (unsigned long long)v);
}

__device__ __forceinline__ void star_pair_back_active(const DevGraph &g, int64_t delta, int32_t r,
                                                      int2 lr, int32_t lo,
                                                      unsigned long long *sacc) {
    const int64_t *__restrict__ tt = g.tt;
    const int32_t u = g.tc[r];
    const int32_t seg_end = g.off[u + 1];
    const int64_t tr = tt[r];
    const int D3 = dir_of(g.tn[r].x);
    const int64_t cin_end = g.cin[seg_end];
    const int64_t cin_r = g.cin[r];
    {
        // W(r): as in star_pair_entry
        uint64_t n0 = 0, n1 = 0, c00 = 0, c01 = 0, c10 = 0, c11 = 0;
        uint64_t X00 = 0, X01 = 0, X10 = 0, X11 = 0, Y00 = 0, Y01 = 0, Y10 = 0, Y11 = 0;
        int32_t a = lr.x, cur = r;
        while (a >= lo && a < cur) {  // links strictly decrease: the walk always ends
            const int da = dir_of(g.tn[a].x);
            const int64_t cin_a = g.cin[a];
            const uint64_t between_in = (uint64_t)(cin_r - (cin_a + da));
            const uint64_t between_o = (uint64_t)(r - a - 1) - between_in;
            const uint64_t co_a = (uint64_t)(a - cin_a), ci_a = (uint64_t)cin_a;
            if (da) {
                c10 += n0;
                c11 += n1;
                n1 += 1;
                X10 += between_o;
                X11 += between_in;
                Y10 += co_a;
                Y11 += ci_a;
            } else {
                c00 += n0;
                c01 += n1;
                n0 += 1;
                X00 += between_o;
                X01 += between_in;
                Y00 += co_a;
                Y01 += ci_a;
            }
            cur = a;
            a = g.lk[a].x;
        }
        const uint64_t n[2] = {n0, n1};
        const uint64_t c2s[2][2] = {{c00, c01}, {c10, c11}};
        const uint64_t X[2][2] = {{X00, X01}, {X10, X11}};
        const uint64_t Yp[2][2] = {{Y00, Y01}, {Y10, Y11}};
        const int64_t cin_lo = g.cin[lo];
        const int64_t co_lo = (int64_t)lo - cin_lo;
#pragma unroll
        for (int d1 = 0; d1 < 2; d1++)
#pragma unroll
            for (int d2 = 0; d2 < 2; d2++) {
                const uint64_t sp = c2s[d1][d2];
                lane_add(sacc, IX(d1, d2, D3), sp);                                 // Pair
                lane_add(sacc, 16 + IX(d1, d2, D3), X[d1][d2] - sp);                // Star-II
                const uint64_t base = d1 ? (uint64_t)cin_lo : (uint64_t)co_lo;     // C_d1(lo)
                lane_add(sacc, 8 + IX(d1, d2, D3), Yp[d2][d1] - n[d2] * base - sp);  // Star-I
                lane_add(sacc, 24 + IX(d1, d2, D3), 0 - sp);                        // Star-III
            }
        const int64_t after_in = cin_end - (cin_r + D3);
        const int64_t after_o = (int64_t)(seg_end - r - 1) - after_in;
#pragma unroll
        for (int d1 = 0; d1 < 2; d1++) {
            lane_add(sacc, 24 + IX(d1, D3, 0), n[d1] * (uint64_t)after_o);
            lane_add(sacc, 24 + IX(d1, D3, 1), n[d1] * (uint64_t)after_in);
        }
    }
    {
        // F(p) of the predecessor p: its same-neighbour entries from r on
        const int32_t p = lr.x;
        const int64_t tp = tt[p];
        const int Dp = dir_of(g.tn[p].x);
        const int32_t hi = gallop_hi(tt, r, seg_end, tp, delta);  // t_r - t_p <= delta
        uint64_t f0 = 0, f1 = 0;
        int32_t b = r, cur = p;
        while (b > cur && b <= hi) {  // links strictly increase: the walk always ends
            if (dir_of(g.tn[b].x)) f1 += 1;
            else f0 += 1;
            cur = b;
            b = g.lk[b].y;
        }
        const uint64_t f[2] = {f0, f1};
        const int64_t cin_h1 = (int64_t)g.cin[hi] + dir_of(g.tn[hi].x);  // C_in(hi+1)
        const int64_t after_in = cin_end - cin_h1;
        const int64_t after_o = (int64_t)(seg_end - hi - 1) - after_in;
#pragma unroll
        for (int d2 = 0; d2 < 2; d2++) {
            lane_add(sacc, 24 + IX(Dp, d2, 0), 0 - f[d2] * (uint64_t)after_o);
            lane_add(sacc, 24 + IX(Dp, d2, 1), 0 - f[d2] * (uint64_t)after_in);
        }
    }
}

// Star/Pair contributions of the entries [begin, end), visited by threads
// tid, tid + nthreads, ..., each finding its own window bounds.
__device__ __forceinline__ void star_pair_range(const DevGraph &g, int64_t delta, int64_t begin,
                                                int64_t end, int64_t tid, int64_t nthreads,
                                                unsigned long long *sacc) {
    for (int64_t i = begin + tid; i < end; i += nthreads) {
        const int32_t r = (int32_t)i;
        const int64_t tr = g.tt[r];
        const uint32_t nbr = g.tn[r].x;
        const int32_t u = g.tc[r];
        const int2 lr = g.lk[r];
        if (dir_of(nbr)) star_pair_entry<1>(g, delta, r, tr, u, lr, sacc);
        else star_pair_entry<0>(g, delta, r, tr, u, lr, sacc);
    }
}

// First position p in [a, r] with tt[p] >= bound, searching forward from a
// with first step `step` (a guess of the distance); tt[r] >= bound holds.
__device__ __forceinline__ int32_t gallop_fwd(const int64_t *__restrict__ tt, int32_t a, int32_t r,
                                              int64_t bound, int32_t step) {
    if (tt[a] >= bound) return a;
    int32_t lo = a, hi = r;  // tt[lo] < bound <= tt[hi]
    while (true) {
        const int32_t p = lo + step;
        if (p >= r) break;
        if (tt[p] >= bound) {
            hi = p;
            break;
        }
        lo = p;
        step <<= 1;
    }
    while (hi - lo > 1) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (tt[mid] >= bound) hi = mid;
        else lo = mid;
    }
    return hi;
}

// ------------------------------------------------------------ segments
//
// The four kernels of the fast path (k_window_lo, k_star_pair_list,
// k_tri_jobs, k_tri_join) count a table of segments in one pass each: a
// segment is an entry range of one graph (whole edges: both entries of each
// of its edges lie inside), its window delta and its 56 cells. One graph is
// one segment; the components of a tm_build_many graph, the graphs of a batch
// and the windows of a multi-delta call are one segment each. Scratch arrays
// are indexed by x = the segment's xbase + (entry - its begin), so every
// segment owns the scratch ranges [xbase, xbase + len) (window starts, the
// list of back-active entries) and [xbase / 2, (xbase + len) / 2) (the Tri
// joins, at most one per edge).
//
// Work is cut into units that never straddle two segments, taken by
// persistent warps (or blocks) in index order: echunk consecutive entries for
// the streaming passes, SP_CHUNK listed entries for the Star/Pair sweep, 32
// joins for the Tri join.
constexpr int SP_CHUNK = THREADS;  // listed entries per block unit of the Star/Pair sweep

struct SegArgs {
    Segment seg0;          // the segment when segs is null
    const Segment *segs;   // device table of the segments, or null: one segment, seg0
    const int32_t *eunit;  // device, with segs: k, then the prefix over the segments of
                           // ceil(len / echunk) (k + 1 values)
    int32_t echunk;        // entries per warp unit of the streaming passes (a multiple of 128)
    const int32_t *own;    // per node, the shard that owns it as a centre, or null: all
    int32_t own_rank;      // the shard counted (centres u with own[u] == own_rank)
};

__device__ __forceinline__ bool owns(const SegArgs &A, uint32_t u) {
    return A.own == nullptr || A.own[u] == A.own_rank;
}

// ONE: the kernel counts the single segment A.seg0 (read in place from the
// kernel's parameter space); otherwise the device table A.segs.
template <bool ONE>
__device__ __forceinline__ int32_t seg_count(const SegArgs &A) {
    return ONE ? 1 : A.eunit[0];
}

template <bool ONE>
__device__ __forceinline__ const Segment &seg_ref(const SegArgs &A, int32_t c) {
    if constexpr (ONE) return A.seg0;
    else return A.segs[c];
}

// Largest c in [0, k) with pre[c] <= u (pre ascending, pre[0] = 0).
__device__ __forceinline__ int32_t prefix_find(const int32_t *pre, int32_t k, int64_t u) {
    int32_t lo = 0, hi = k;
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (pre[mid] <= u) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Number of streaming units over all segments, and the segment and first
// entry of unit u.
template <bool ONE>
__device__ __forceinline__ int64_t seg_units(const SegArgs &A) {
    if constexpr (ONE) return ((int64_t)A.seg0.end - A.seg0.begin + A.echunk - 1) / A.echunk;
    else return A.eunit[1 + A.eunit[0]];
}

template <bool ONE>
__device__ __forceinline__ int32_t unit_seg(const SegArgs &A, int64_t u, int64_t *first) {
    if constexpr (ONE) {
        *first = u;
        return 0;
    } else {
        const int32_t c = prefix_find(A.eunit + 1, A.eunit[0], u);
        *first = u - A.eunit[1 + c];
        return c;
    }
}

// A warp's buffered list entries (cnt of them, < 64) are appended to the
// segment's list at list + xbase, 32 at a time or all at once (flush_all).
__device__ __forceinline__ void warp_append(int32_t *buf, int &cnt, bool flush_all,
                                            int32_t *__restrict__ list,
                                            int32_t *__restrict__ count) {
    const int lane = threadIdx.x & 31;
    while (cnt >= 32 || (flush_all && cnt > 0)) {
        const int take = cnt >= 32 ? 32 : cnt;
        int32_t first = 0;
        if (lane == 0) first = atomicAdd(count, take);
        first = __shfl_sync(0xffffffffu, first, 0);
        if (lane < take) list[first + lane] = buf[cnt - take + lane];
        cnt -= take;
        __syncwarp();
    }
}

// lo(r) for every entry r of every segment: the first entry of W(r), r
// itself when the window is empty, written to wl[x(r)]. A warp takes a unit
// of echunk consecutive entries of one segment as groups of 32; a lane's
// entry in group g is 32 entries after its entry in group g-1, and lo never
// decreases along one centre, so when both are of the same centre the lane
// searches forwards from its previous lo (the window has slid by about 32
// entries) instead of backwards from r.
// With `act`, the back-active entries (lk.x >= lo(r): a few percent, and the
// only ones with Star/Pair contributions) are listed there as well, in the
// segment's own range act[xbase ...) with its count nact[c]; each warp
// gathers them in shared memory and reserves space 32 at a time. The order
// of a list is immaterial: every entry adds its counts.
template <bool ONE>
__global__ void __launch_bounds__(THREADS)
    k_window_lo(const __grid_constant__ SegArgs A, int32_t *__restrict__ wl,
                int32_t *__restrict__ act, int32_t *__restrict__ nact) {
    __shared__ int32_t buf[THREADS / 32][64];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t *wb = buf[warp];
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nu = seg_units<ONE>(A);
    for (int64_t u = wid; u < nu; u += nwarps) {
        int64_t ui;
        const int32_t c = unit_seg<ONE>(A, u, &ui);
        const Segment &sg = seg_ref<ONE>(A, c);
        const DevGraph &g = sg.g;
        const int64_t delta = sg.delta;
        const int64_t c0 = sg.begin + ui * A.echunk;
        const int64_t end = c0 + A.echunk < sg.end ? c0 + A.echunk : sg.end;
        int cnt = 0;  // entries held in wb (warp-uniform, < 32 between groups)
        int32_t prev_u = -1, prev_lo = 0;
        for (int gi = 0; gi < A.echunk / 32; gi++) {
            const int64_t i = c0 + gi * 32 + lane;
            bool active = false;
            if (i < end) {
                const int32_t r = (int32_t)i;
                const int64_t tr = g.tt[r];
                const int32_t cu = g.tc[r];
                int32_t lo = r;
                if (cu == prev_u) {
                    lo = gallop_fwd(g.tt, prev_lo, r, tr - delta, 32);
                } else {
                    const int32_t sb = g.off[cu];
                    if (r > sb && tr - g.tt[r - 1] <= delta) lo = gallop_lo(g.tt, sb, r, tr - delta);
                }
                prev_u = cu;
                prev_lo = lo;
                wl[sg.xbase + (i - sg.begin)] = lo;
                active = act != nullptr && lo < r && g.lk[r].x >= lo && owns(A, (uint32_t)cu);
            }
            if (act == nullptr) continue;
            const unsigned bal = __ballot_sync(0xffffffffu, active);
            if (active) wb[cnt + __popc(bal & ((1u << lane) - 1u))] = (int32_t)i;
            cnt += __popc(bal);
            __syncwarp();
            warp_append(wb, cnt, false, act + sg.xbase, nact + c);
        }
        if (act != nullptr) warp_append(wb, cnt, true, act + sg.xbase, nact + c);
    }
}

// Prefix over the k segments of ceil(count[c] / chunk): out[0..k], one block.
__global__ void k_unit_prefix(const int32_t *__restrict__ meta, const int32_t *__restrict__ count,
                              int32_t chunk, int32_t *__restrict__ out) {
    __shared__ int32_t carry;
    const int32_t k = meta[0];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int32_t b = 0; b < k; b += blockDim.x) {
        const int32_t c = b + threadIdx.x;
        const int32_t v = c < k ? (count[c] + chunk - 1) / chunk : 0;
        int32_t inc = warp_incl_scan_i32(v);
        __shared__ int32_t wsum[32];
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 31) wsum[w] = inc;
        __syncthreads();
        if (w == 0) {
            const int32_t x = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
            const int32_t xi = warp_incl_scan_i32(x);
            wsum[lane] = xi - x;
        }
        __syncthreads();
        inc += wsum[w];
        if (c < k) out[c + 1] = carry + inc;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += inc;
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = 0;
}

// Units of `chunk` listed items over the segments: with a table, from the
// prefix pre (k_unit_prefix); for one segment, from its count.
template <bool ONE>
__device__ __forceinline__ int64_t list_units(const SegArgs &A, const int32_t *pre,
                                              const int32_t *count, int32_t chunk) {
    if constexpr (ONE) return (count[0] + chunk - 1) / chunk;
    else return pre[A.eunit[0]];
}

template <bool ONE>
__device__ __forceinline__ int32_t list_unit_seg(const SegArgs &A, const int32_t *pre, int64_t u,
                                                 int64_t *first) {
    if constexpr (ONE) {
        *first = u;
        return 0;
    } else {
        const int32_t c = prefix_find(pre, A.eunit[0], u);
        *first = u - pre[c];
        return c;
    }
}

// The 32 Star/Pair cells of the block's copies (cell i of lane copy l at
// sacc[i * SP_COPIES + l]) added into cells (Star 0..23, Pair 24..31).
__device__ __forceinline__ void flush_lane_copies(const unsigned long long *sacc,
                                                  unsigned long long *__restrict__ cells) {
    if (threadIdx.x < 32) {
        const int c = threadIdx.x;
        unsigned long long v = 0;
        for (int k = 0; k < 32; k++) v += sacc[c * SP_COPIES + k];
        if (v) atomicAdd(&cells[c < 8 ? 24 + c : c - 8], v);
    }
}

// The Star/Pair sweep of the back-active entries that k_window_lo listed, 32
// to a warp with every lane busy. A block takes units of SP_CHUNK listed
// entries of one segment from a shared head (one atomic per unit, in index
// order) and adds into its shared copies of the cells, which it flushes into
// the segment's cells when the next unit belongs to another segment, and at
// the end.
template <bool ONE>
__global__ void __launch_bounds__(THREADS, 5)
    k_star_pair_list(const __grid_constant__ SegArgs A, const int32_t *__restrict__ wl,
                     const int32_t *__restrict__ act, const int32_t *__restrict__ nact,
                     const int32_t *__restrict__ sp_pre, int32_t *__restrict__ head) {
    // one copy of the 32 cells per lane index (shared by the block's warps),
    // so the lanes of a warp never add to the same word
    __shared__ unsigned long long sacc[32 * SP_COPIES];
    for (int i = threadIdx.x; i < 32 * SP_COPIES; i += blockDim.x) sacc[i] = 0;
    __syncthreads();
    unsigned long long *mine = sacc + (threadIdx.x & 31);
    const int64_t nu = list_units<ONE>(A, sp_pre, nact, SP_CHUNK);
    int32_t cur = -1;
    unsigned long long *cur_cells = nullptr;
    __shared__ int32_t next;
    while (true) {
        // the next unit from the shared head: blocks that drew short units take more
        __syncthreads();
        if (threadIdx.x == 0) next = atomicAdd(head, 1);
        __syncthreads();
        const int64_t u = next;
        if (u >= nu) break;
        int64_t ui;
        const int32_t c = list_unit_seg<ONE>(A, sp_pre, u, &ui);  // block-uniform
        const Segment &sg = seg_ref<ONE>(A, c);
        if constexpr (!ONE) {
            if (c != cur) {
                if (cur >= 0) {
                    __syncthreads();
                    flush_lane_copies(sacc, cur_cells);
                    __syncthreads();
                    for (int i = threadIdx.x; i < 32 * SP_COPIES; i += blockDim.x) sacc[i] = 0;
                    __syncthreads();
                }
                cur = c;
                cur_cells = sg.cells;
            }
        }
        const int32_t n = nact[c];
        for (int j = 0; j < SP_CHUNK / THREADS; j++) {
            const int64_t idx = ui * SP_CHUNK + j * THREADS + threadIdx.x;
            if (idx >= n) break;
            const int32_t r = act[sg.xbase + idx];
            star_pair_back_active(sg.g, sg.delta, r, sg.g.lk[r], wl[sg.xbase + (r - sg.begin)],
                                  mine);
        }
    }
    __syncthreads();
    if constexpr (ONE) flush_lane_copies(sacc, A.seg0.cells);
    else if (cur >= 0) flush_lane_copies(sacc, cur_cells);
}

// The Star/Pair sweep without scratch (window bounds searched per entry).
__global__ void __launch_bounds__(THREADS, 5)
    k_star_pair(const DevGraph g, int64_t delta, int32_t begin, int32_t end,
                unsigned long long *__restrict__ cells) {
    __shared__ unsigned long long sacc[32];
    if (threadIdx.x < 32) sacc[threadIdx.x] = 0;
    __syncthreads();
    star_pair_range(g, delta, begin, end, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                    (int64_t)gridDim.x * blockDim.x, sacc);
    __syncthreads();
    flush_star_pair(sacc, cells);
}

// Raw hash slot of a node pair: (begin, end) of its run, the single edge
// encoded in the slot (begin < 0), or (0, 0) if the pair has no edge.
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

// Edges of E_(big, x) inside [rank_lo, rank_hi), split at rank `at`:
// nb / na = how many lie before / after `at`, fb / fa = how many of those have
// the smaller node id as source.
struct PairCounts {
    int32_t nb, na, fb, fa;
};

// L2 eviction policy "keep": the Bloom filter is read by every probe. The
// policy is created once per call of a probe loop and passed to its loads.
__device__ __forceinline__ uint64_t keep_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ uint64_t load_keep_pol(const uint64_t *p, uint64_t pol) {
    uint64_t v;
    asm volatile("ld.global.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ uint64_t load_keep(const uint64_t *p) {
    return load_keep_pol(p, keep_policy());
}

// As pair_counts, for a pair that passed the Bloom filter.
__device__ __forceinline__ bool pair_counts_hashed(const DevGraph &g, uint64_t key, int32_t rank_lo,
                                                   int32_t rank_hi, int32_t at, PairCounts &c) {
    const int2 run = find_pair(g.hash, g.hash_mask, key);
    if (run.x < 0) {  // single edge kept in the slot
        const int32_t r1 = -run.x - 1;
        if (r1 < rank_lo || r1 >= rank_hi) return false;
        const bool before = r1 < at;
        c.nb = before;
        c.na = !before;
        c.fb = before ? run.y : 0;
        c.fa = before ? 0 : run.y;
        return true;
    }
    if (run.x == run.y) return false;
    // the three lower bounds (rank_lo, rank_hi, at) searched over the whole
    // run side by side, so that their loads are in flight together; the
    // item's bound is then clamped into [k0, k1]
    int32_t b0 = run.x, e0 = run.y, b1 = run.x, e1 = run.y, b2 = run.x, e2 = run.y;
    while (b0 < e0 || b1 < e1 || b2 < e2) {
        const int32_t m0 = b0 + ((e0 - b0) >> 1), m1 = b1 + ((e1 - b1) >> 1),
                      m2 = b2 + ((e2 - b2) >> 1);
        const int32_t r0 = b0 < e0 ? g.pl[m0].x : 0;
        const int32_t r1 = b1 < e1 ? g.pl[m1].x : 0;
        const int32_t r2 = b2 < e2 ? g.pl[m2].x : 0;
        if (b0 < e0) {
            if (r0 < rank_lo) b0 = m0 + 1;
            else e0 = m0;
        }
        if (b1 < e1) {
            if (r1 < rank_hi) b1 = m1 + 1;
            else e1 = m1;
        }
        if (b2 < e2) {
            if (r2 < at) b2 = m2 + 1;
            else e2 = m2;
        }
    }
    const int32_t k0 = b0, k1 = b1 > k0 ? b1 : k0;
    if (k0 == k1) return false;
    const int32_t ks = b2 < k0 ? k0 : (b2 > k1 ? k1 : b2);
    const int32_t c0 = g.pl[k0].y, cs = g.pl[ks].y, c1 = g.pl[k1].y;
    c.nb = ks - k0;
    c.na = k1 - ks;
    c.fb = cs - c0;
    c.fa = c1 - cs;
    return true;
}

__device__ __forceinline__ bool pair_counts(const DevGraph &g, uint64_t key, int32_t rank_lo,
                                            int32_t rank_hi, int32_t at, PairCounts &c) {
    uint32_t word;
    const uint64_t bits = bloom_bits(key, g.bloom_mask, &word);
    if ((load_keep(g.bloom + word) & bits) != bits) return false;  // the pair never met
    return pair_counts_hashed(g, key, rank_lo, rank_hi, at, c);
}

// The join of one edge e_j = u -> w (u its source): the smaller of the two
// endpoint windows is enumerated, the matches are looked up in the other.
struct TriEdge {
    int32_t small_lo;     // smaller window: entries [small_lo, small_lo + work)
    int32_t work;
    int32_t rank_lo_big;  // rank of the first entry of the bigger window; bit 30 / 31: do
                          // not count the triangles centred at u / at w (a shard's join)
    uint32_t rj_s;        // rank of e_j; bit 31: the smaller window is W_u
    uint32_t big;         // the bigger window's centre
    __device__ __forceinline__ int32_t rank_j() const { return (int32_t)(rj_s & 0x7fffffffu); }
    __device__ __forceinline__ bool small_is_u() const { return (rj_s >> 31) != 0; }
};

// The join of edge e_j (rank rank_j, source entry r at centre u, other endpoint
// w, entry twin at w) given both window starts, when both windows are
// non-empty.
__device__ __forceinline__ TriEdge make_tri_edge(const DevGraph &g, int32_t r, uint32_t u,
                                                 uint32_t w, int32_t rank_j, int32_t lo_u,
                                                 int32_t twin, int32_t lo_w) {
    const int32_t wu = r - lo_u, ww = twin - lo_w;
    const bool su = wu <= ww;
    TriEdge E;
    E.small_lo = su ? lo_u : lo_w;
    E.work = su ? wu : ww;
    E.rank_lo_big = (int32_t)g.tn[su ? lo_w : lo_u].y;
    E.rj_s = (uint32_t)rank_j | (su ? 0x80000000u : 0u);
    E.big = su ? w : u;
    return E;
}

// Tri type-II cells: acc[IX(di, dj, dk)]. At the source u, e_j is outward
// (dj = 0); at the destination w it is inward (dj = 1). A match ranked after
// the item is centred at the item's centre, one ranked before it at the big
// window's centre.
template <bool SHARD = false>
__device__ __forceinline__ void tri_probe_hashed(const DevGraph &g, uint32_t big,
                                                 int32_t rank_lo_big, uint32_t rj_s,
                                                 const uint2 it, uint64_t key,
                                                 unsigned long long (&acc)[8]) {
    const uint32_t x = node_of(it.x);
    PairCounts c;
    if (!pair_counts_hashed(g, key, rank_lo_big & 0x3fffffff, (int32_t)(rj_s & 0x7fffffffu),
                            (int32_t)it.y, c))
        return;
    // a big-side edge big -> x is outward at big and inward at x
    const bool big_is_min = big < x;
    int32_t b_out_big = big_is_min ? c.fb : c.nb - c.fb;  // before the item, source == big
    int32_t a_out_big = big_is_min ? c.fa : c.na - c.fa;  // after the item, source == big
    const int di = dir_of(it.x);                          // item w.r.t. its centre
    if (SHARD && (rank_lo_big & 0xc0000000)) {
        // a shard's join: the matches after the item are centred at the item's
        // centre, those before it at the big window's centre
        const bool skip_u = (rank_lo_big >> 30) & 1, skip_w = (uint32_t)rank_lo_big >> 31;
        const bool skip_after = (rj_s >> 31) ? skip_u : skip_w;
        const bool skip_before = (rj_s >> 31) ? skip_w : skip_u;
        if (skip_after) {
            c.na = 0;
            a_out_big = 0;
        }
        if (skip_before) {
            c.nb = 0;
            b_out_big = 0;
        }
    }
    if (rj_s >> 31) {  // the smaller window is W_u
        // item a in W_u (node x), matches k in W_w.
        // after a: centre u, (e_i = a, e_k = k): Tri[II][d_a][0][dir of k w.r.t. x]
        // before a: centre w, (e_i = k, e_k = a): Tri[II][dir of k w.r.t. w][1][dir of a w.r.t. x]
        if (di) {
            acc[IX(1, 0, 0)] += (unsigned long long)(c.na - a_out_big);  // k: x -> w, o at x
            acc[IX(1, 0, 1)] += (unsigned long long)a_out_big;
            acc[IX(0, 1, 0)] += (unsigned long long)b_out_big;          // a: x -> u, o at x
            acc[IX(1, 1, 0)] += (unsigned long long)(c.nb - b_out_big);
        } else {
            acc[IX(0, 0, 0)] += (unsigned long long)(c.na - a_out_big);
            acc[IX(0, 0, 1)] += (unsigned long long)a_out_big;
            acc[IX(0, 1, 1)] += (unsigned long long)b_out_big;          // a: u -> x, in at x
            acc[IX(1, 1, 1)] += (unsigned long long)(c.nb - b_out_big);
        }
    } else {
        // item k in W_w (node x), matches a in W_u.
        // before k: centre u, (e_i = a, e_k = k): Tri[II][dir of a w.r.t. u][0][dir of k w.r.t. x]
        // after k: centre w, (e_i = k, e_k = a): Tri[II][d_k][1][dir of a w.r.t. x]
        if (di) {
            acc[IX(0, 0, 0)] += (unsigned long long)b_out_big;          // k: x -> w, o at x
            acc[IX(1, 0, 0)] += (unsigned long long)(c.nb - b_out_big);
            acc[IX(1, 1, 0)] += (unsigned long long)(c.na - a_out_big);  // a: x -> u, o at x
            acc[IX(1, 1, 1)] += (unsigned long long)a_out_big;
        } else {
            acc[IX(0, 0, 1)] += (unsigned long long)b_out_big;
            acc[IX(1, 0, 1)] += (unsigned long long)(c.nb - b_out_big);
            acc[IX(0, 1, 0)] += (unsigned long long)(c.na - a_out_big);
            acc[IX(0, 1, 1)] += (unsigned long long)a_out_big;
        }
    }
}

constexpr int TRI_WARPS = THREADS / 32;

// The probes of the (up to) 32 joins staged in edges[] by one warp, `incl`
// the inclusive prefix of their sizes and `total` its last value: lane j
// takes probes j, j + 32, ... of the flattened list, so a lane never waits
// for another lane's long window.
__device__ __forceinline__ void tri_probes(const DevGraph &g, const TriEdge *edges,
                                           const int32_t *incl, int32_t total,
                                           unsigned long long (&acc)[8]) {
    const int lane = threadIdx.x & 31;
    for (int32_t jb = 0; jb < total; jb += 32) {
        const int32_t j = jb + lane;
        if (j >= total) continue;
        // owner: the first lane whose inclusive prefix exceeds j
        int lo = 0, hi = 31;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (incl[mid] > j) hi = mid;
            else lo = mid + 1;
        }
        const TriEdge &B = edges[lo];
        const uint2 it = g.tn[B.small_lo + (j - (incl[lo] - B.work))];
        const uint32_t x = node_of(it.x);
        if (x == B.big) continue;  // an edge of the pair (u, w) itself
        const uint64_t key = pair_key(B.big, x);
        uint32_t word;
        const uint64_t bits = bloom_bits(key, g.bloom_mask, &word);
        if ((load_keep(g.bloom + word) & bits) != bits) continue;  // the pair never met
        tri_probe_hashed(g, B.big, B.rank_lo_big, B.rj_s, it, key, acc);
    }
}

// A probe that passed the Bloom filter, waiting for the hash lookup.
struct TriProbe {
    uint2 it;
    uint64_t key;
    uint32_t big;
    int32_t rank_lo_big;
    uint32_t rj_s;
    uint32_t pad;
};

// As tri_probes, in two stages: the Bloom test of every probe, then the hash
// and pair-list lookups of the fifth that pass it, gathered in the warp's
// queue q (TRI_QUEUE slots, qn of them in use) and run 32 at a time with
// every lane busy. Each lane tests two probes per step, so that their
// dependent reads (item, then Bloom word) are in flight together. Probes still
// queued when the caller's list ends stay for the next call; the caller runs
// the rest at its end.
constexpr int TRI_QUEUE = 96;

template <bool SHARD = false>
__device__ __forceinline__ void tri_run_queue(const DevGraph &g, const TriProbe *q, int n,
                                              unsigned long long (&acc)[8]) {
    const int lane = threadIdx.x & 31;
    if (lane < n) {
        const TriProbe p = q[lane];
        tri_probe_hashed<SHARD>(g, p.big, p.rank_lo_big, p.rj_s, p.it, p.key, acc);
    }
}

template <bool SHARD = false>
__device__ __forceinline__ void tri_probes_queued(const DevGraph &g, const TriEdge *edges,
                                                  const int32_t *incl, int32_t total,
                                                  TriProbe *q, int &qn,
                                                  unsigned long long (&acc)[8]) {
    const int lane = threadIdx.x & 31;
    const uint64_t pol = keep_policy();
    int last[2] = {0, 0};
    for (int32_t jb = 0; jb < total; jb += 64) {
        int32_t j[2], own[2];
        bool ok[2];
#pragma unroll
        for (int k = 0; k < 2; k++) {
            j[k] = jb + 32 * k + lane;
            ok[k] = j[k] < total;
            // owner: the first lane whose inclusive prefix exceeds j, galloping
            // forwards from this lane's previous owner (j only grows)
            int o = last[k];
            if (ok[k] && incl[o] <= j[k]) {
                int lo = o, hi = 31, step = 1;
                while (lo + step < 31) {
                    if (incl[lo + step] > j[k]) {
                        hi = lo + step;
                        break;
                    }
                    lo += step;
                    step <<= 1;
                }
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (incl[mid] > j[k]) hi = mid;
                    else lo = mid;
                }
                o = hi;
            }
            last[k] = o;
            own[k] = o;
        }
        uint2 it[2];
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const TriEdge &B = edges[own[k]];
            it[k] = ok[k] ? g.tn[B.small_lo + (j[k] - (incl[own[k]] - B.work))] : make_uint2(0, 0);
        }
        uint64_t key[2], bits[2], bw[2];
        bool cand[2];
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const uint32_t big = edges[own[k]].big;
            const uint32_t x = node_of(it[k].x);
            cand[k] = ok[k] && x != big;  // not an edge of the pair (u, w) itself
            key[k] = pair_key(big, x);
            uint32_t word;
            bits[k] = bloom_bits(key[k], g.bloom_mask, &word);
            bw[k] = cand[k] ? load_keep_pol(g.bloom + word, pol) : 0;
        }
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const bool pass = cand[k] && (bw[k] & bits[k]) == bits[k];
            const unsigned bal = __ballot_sync(0xffffffffu, pass);
            if (pass) {
                const TriEdge &B = edges[own[k]];
                TriProbe p;
                p.it = it[k];
                p.key = key[k];
                p.big = B.big;
                p.rank_lo_big = B.rank_lo_big;
                p.rj_s = B.rj_s;
                q[qn + __popc(bal & ((1u << lane) - 1u))] = p;
            }
            qn += __popc(bal);
        }
        __syncwarp();
        while (qn >= 32) {
            tri_run_queue<SHARD>(g, q + qn - 32, 32, acc);  // the newest 32: nothing to move
            qn -= 32;
            __syncwarp();
        }
    }
}

// Tri joins of the edges whose source entries lie in [begin, end), visited
// 32 entries at a time by warps wid, wid + nwarps, ...; each edge is taken
// once, at its source entry (direction o). Each edge e_j = (u -> w) is the
// later centre edge of the type-II triangles at u and at w, whose other
// centre edges lie in the windows W_u(e_j) and W_w(e_j), so one join of the
// two windows on the neighbour node counts both. `edges` and `incl` are the
// calling warp's shared-memory staging (32 slots each).
__device__ __forceinline__ void tri_range(const DevGraph &g, int64_t delta, int64_t begin,
                                          int64_t end, int64_t wid, int64_t nwarps,
                                          TriEdge *edges, int32_t *incl,
                                          unsigned long long (&acc)[8]) {
    const int lane = threadIdx.x & 31;
    for (int64_t base = begin + wid * 32; base < end; base += nwarps * 32) {
        const int64_t r = base + lane;
        TriEdge E;
        E.work = 0;
        if (r < end) {
            const uint2 en = g.tn[r];
            if (dir_of(en.x) == 0) {
                const int64_t et = g.tt[r];
                const uint32_t u = (uint32_t)g.tc[r];
                const int32_t sb = g.off[u];
                if (r > sb && et - g.tt[r - 1] <= delta) {
                    const uint32_t w = node_of(en.x);
                    const int32_t twin = g.pos_dst[en.y];
                    const int32_t wb = g.off[w];
                    if (twin > wb && et - g.tt[twin - 1] <= delta) {
                        const int32_t lo_u = gallop_lo(g.tt, sb, (int32_t)r, et - delta);
                        const int32_t lo_w = gallop_lo(g.tt, wb, twin, et - delta);
                        E = make_tri_edge(g, (int32_t)r, u, w, (int32_t)en.y, lo_u, twin, lo_w);
                    }
                }
            }
        }
        const int32_t inc = warp_incl_scan_i32(E.work);
        const int32_t total = __shfl_sync(0xffffffffu, inc, 31);
        if (total == 0) continue;
        edges[lane] = E;
        incl[lane] = inc;
        __syncwarp();
        tri_probes(g, edges, incl, total, acc);
        __syncwarp();
    }
}

// Whole-graph Tri (type II) over the entries [begin, end) without scratch:
// the window starts are searched for here.
__global__ void __launch_bounds__(THREADS)
    k_tri(const DevGraph g, int64_t delta, int32_t begin, int32_t end,
          unsigned long long *__restrict__ cells) {
    __shared__ TriEdge edges[TRI_WARPS][32];
    __shared__ int32_t incl[TRI_WARPS][32];
    unsigned long long acc[8];
#pragma unroll
    for (int c = 0; c < 8; c++) acc[c] = 0;
    const int warp = threadIdx.x >> 5;
    tri_range(g, delta, begin, end, blockIdx.x * (int64_t)TRI_WARPS + warp,
              (int64_t)gridDim.x * TRI_WARPS, edges[warp], incl[warp], acc);
    // type II lives at Tri cells 8..15 (T = 1)
    block_flush<8, 0>(acc, 32 + 8, cells);
}

constexpr int JOB_U = 4;  // groups of 32 entries per warp and step: chains of reads in flight

// One step of k_tri_jobs: the joins of the source entries among the 32 * JOB_U
// entries from base (below end) are added to the warp's buffer wb (cnt of
// them, warp-uniform); full groups of 32 are appended to jobs (count *njobs).
template <bool SHARD>
__device__ __forceinline__ void tri_jobs_step(const SegArgs &A, const DevGraph &g,
                                              const int32_t *__restrict__ swl, int64_t base,
                                              int64_t end, TriEdge *wb, int &cnt,
                                              TriEdge *__restrict__ jobs,
                                              int32_t *__restrict__ njobs) {
    const int lane = threadIdx.x & 31;
    uint2 en[JOB_U];
    int32_t lo_u[JOB_U], lo_w[JOB_U], twin[JOB_U];
#pragma unroll
    for (int k = 0; k < JOB_U; k++) {
        const int64_t r = base + k * 32 + lane;
        en[k] = make_uint2(0x80000000u, 0);  // inward: no join
        lo_u[k] = 0;
        if (r < end) {
            en[k] = g.tn[r];
            lo_u[k] = swl[r];
        }
    }
#pragma unroll
    for (int k = 0; k < JOB_U; k++) {
        const int64_t r = base + k * 32 + lane;
        twin[k] = -1;
        if (dir_of(en[k].x) == 0 && lo_u[k] < r) twin[k] = g.pos_dst[en[k].y];
    }
#pragma unroll
    for (int k = 0; k < JOB_U; k++) lo_w[k] = twin[k] >= 0 ? swl[twin[k]] : 0;
#pragma unroll
    for (int k = 0; k < JOB_U; k++) {
        const int64_t r = base + k * 32 + lane;
        bool has = twin[k] >= 0 && lo_w[k] < twin[k];
        TriEdge E;
        if (has) {
            const uint32_t u = (uint32_t)g.tc[r], w = node_of(en[k].x);
            E = make_tri_edge(g, (int32_t)r, u, w, (int32_t)en[k].y, lo_u[k], twin[k], lo_w[k]);
            if (SHARD) {
                const bool cu = owns(A, u), cw = owns(A, w);
                has = cu || cw;
                E.rank_lo_big |= (cu ? 0 : 0x40000000) | (cw ? 0 : (int32_t)0x80000000);
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, has);
        if (has) wb[cnt + __popc(bal & ((1u << lane) - 1u))] = E;
        cnt += __popc(bal);
    }
    __syncwarp();
    while (cnt >= 32) {
        int32_t first = 0;
        if (lane == 0) first = atomicAdd(njobs, 32);
        first = __shfl_sync(0xffffffffu, first, 0);
        jobs[first + lane] = wb[cnt - 32 + lane];
        cnt -= 32;
        __syncwarp();
    }
}

// As tri_jobs_step, over the 32 * JOB_U edges of ranks from base (below m)
// of a whole graph: an edge's two entries come from the position arrays and
// its endpoints from the rank-ordered (src, dst) words, all read coalesced;
// the window starts of its two entries are then random reads, but within the
// thin band of every centre's entries around the edge's time, which the
// warps of the grid sweep together (rank order is time order).
template <bool SHARD>
__device__ __forceinline__ void tri_jobs_step_ranks(const SegArgs &A, const DevGraph &g,
                                                    const int32_t *__restrict__ swl, int64_t base,
                                                    int64_t m, TriEdge *wb, int &cnt,
                                                    TriEdge *__restrict__ jobs,
                                                    int32_t *__restrict__ njobs) {
    const int lane = threadIdx.x & 31;
    int32_t r[JOB_U], tw[JOB_U], lo_u[JOB_U], lo_w[JOB_U];
    uint64_t uw[JOB_U];
#pragma unroll
    for (int k = 0; k < JOB_U; k++) {
        const int64_t j = base + k * 32 + lane;
        r[k] = tw[k] = 0;
        uw[k] = 0;
        if (j < m) {
            r[k] = g.pos_src[j];
            tw[k] = g.pos_dst[j];
            uw[k] = g.sd[j];
        }
    }
#pragma unroll
    for (int k = 0; k < JOB_U; k++) {
        const int64_t j = base + k * 32 + lane;
        lo_u[k] = r[k];
        lo_w[k] = tw[k];
        if (j < m) {
            lo_u[k] = swl[r[k]];
            lo_w[k] = swl[tw[k]];
        }
    }
#pragma unroll
    for (int k = 0; k < JOB_U; k++) {
        const int64_t j = base + k * 32 + lane;
        bool has = j < m && lo_u[k] < r[k] && lo_w[k] < tw[k];
        TriEdge E;
        if (has) {
            const uint32_t u = (uint32_t)(uw[k] >> 32), w = (uint32_t)uw[k];
            E = make_tri_edge(g, r[k], u, w, (int32_t)j, lo_u[k], tw[k], lo_w[k]);
            if (SHARD) {
                const bool cu = owns(A, u), cw = owns(A, w);
                has = cu || cw;
                E.rank_lo_big |= (cu ? 0 : 0x40000000) | (cw ? 0 : (int32_t)0x80000000);
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, has);
        if (has) wb[cnt + __popc(bal & ((1u << lane) - 1u))] = E;
        cnt += __popc(bal);
    }
    __syncwarp();
    while (cnt >= 32) {
        int32_t first = 0;
        if (lane == 0) first = atomicAdd(njobs, 32);
        first = __shfl_sync(0xffffffffu, first, 0);
        jobs[first + lane] = wb[cnt - 32 + lane];
        cnt -= 32;
        __syncwarp();
    }
}

// The warp's last cnt (< 32) buffered joins appended to jobs.
__device__ __forceinline__ void tri_jobs_flush(const TriEdge *wb, int cnt,
                                               TriEdge *__restrict__ jobs,
                                               int32_t *__restrict__ njobs) {
    const int lane = threadIdx.x & 31;
    if (cnt > 0) {
        int32_t first = 0;
        if (lane == 0) first = atomicAdd(njobs, cnt);
        first = __shfl_sync(0xffffffffu, first, 0);
        if (lane < cnt) jobs[first + lane] = wb[lane];
    }
    __syncwarp();
}

// Whole-graph Tri in two steps, with the window starts wl of k_window_lo.
// k_tri_jobs: every edge (at its source entry) whose two windows are both
// non-empty becomes one join, appended to its segment's range of `jobs`
// (from xbase / 2, count njobs[c]). The order of the jobs is immaterial: each
// adds its counts. Only a quarter of the edges have such a join on the large
// workloads, so the joining warps below get full lists instead of sparse
// ones, and the chain of dependent reads that finds a join is paid here, in
// a kernel that does nothing else. A warp gathers its jobs in shared memory
// and reserves space 32 at a time, so the shared counter takes one atomic per
// 32 jobs. On one graph the warps sweep steps of 32 * JOB_U entries strided
// over the grid (all warps together stream one region of the arrays, and an
// empty source window is seen in a coalesced read) and flush once at the
// end; on a table a warp takes units of echunk entries of one segment and
// flushes at the end of each unit. k_tri_jobs_ranks is the sweep in rank
// order for a whole graph whose entries are concentrated on few nodes.
template <bool ONE, bool SHARD>
__global__ void __launch_bounds__(THREADS)
    k_tri_jobs(const __grid_constant__ SegArgs A, const int32_t *__restrict__ wl,
               TriEdge *__restrict__ jobs, int32_t *__restrict__ njobs) {
    __shared__ TriEdge buf[TRI_WARPS][32 * (JOB_U + 1)];
    const int warp = threadIdx.x >> 5;
    TriEdge *wb = buf[warp];
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * TRI_WARPS;
    int cnt = 0;  // jobs held in wb (warp-uniform, < 32 between steps)
    if constexpr (ONE) {
        const Segment &sg = A.seg0;
        const int32_t *__restrict__ swl = wl + (sg.xbase - sg.begin);  // swl[r] = wl[x(r)]
        TriEdge *sjobs = jobs + sg.xbase / 2;
        for (int64_t base = sg.begin + wid * (32 * JOB_U); base < sg.end;
             base += nwarps * (32 * JOB_U))
            tri_jobs_step<SHARD>(A, sg.g, swl, base, sg.end, wb, cnt, sjobs, njobs);
        tri_jobs_flush(wb, cnt, sjobs, njobs);
    } else {
        const int64_t nu = seg_units<ONE>(A);
        for (int64_t u = wid; u < nu; u += nwarps) {
            int64_t ui;
            const int32_t c = unit_seg<ONE>(A, u, &ui);
            const Segment &sg = seg_ref<ONE>(A, c);
            const int64_t c0 = sg.begin + ui * A.echunk;
            const int64_t end = c0 + A.echunk < sg.end ? c0 + A.echunk : sg.end;
            const int32_t *__restrict__ swl = wl + (sg.xbase - sg.begin);
            TriEdge *sjobs = jobs + sg.xbase / 2;
            for (int64_t base = c0; base < end; base += 32 * JOB_U)
                tri_jobs_step<SHARD>(A, sg.g, swl, base, end, wb, cnt, sjobs, njobs + c);
            tri_jobs_flush(wb, cnt, sjobs, njobs + c);
            cnt = 0;
        }
    }
}

// k_tri_jobs for a whole graph (segment [0, 2m)) that kept its rank-ordered
// endpoints (g.sd: the build keeps them when 15 % or more of the entries sit
// at centres holding 1/64 of them each): the edges are swept in rank order,
// which is time order, so at any moment the grid's random reads (the window
// starts, the big window's first rank) fall in one thin time band of every
// centre, which L2 holds; an entry-order sweep over a hub's long segment
// scatters them over all of its times. A kernel of its own, so that the
// entry-order sweep keeps its registers and occupancy.
template <bool SHARD>
__global__ void __launch_bounds__(THREADS)
    k_tri_jobs_ranks(const __grid_constant__ SegArgs A, const int32_t *__restrict__ wl,
                     TriEdge *__restrict__ jobs, int32_t *__restrict__ njobs) {
    __shared__ TriEdge buf[TRI_WARPS][32 * (JOB_U + 1)];
    const int warp = threadIdx.x >> 5;
    TriEdge *wb = buf[warp];
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * TRI_WARPS;
    int cnt = 0;
    const Segment &sg = A.seg0;
    const int32_t *__restrict__ swl = wl + sg.xbase;  // the segment starts at entry 0
    TriEdge *sjobs = jobs + sg.xbase / 2;
    for (int64_t base = wid * (32 * JOB_U); base < sg.g.m; base += nwarps * (32 * JOB_U))
        tri_jobs_step_ranks<SHARD>(A, sg.g, swl, base, sg.g.m, wb, cnt, sjobs, njobs);
    tri_jobs_flush(wb, cnt, sjobs, njobs);
}

// Adds each lane's 8 type-II counters of the warp into cells[40..47] (Tri
// cells, T = II) and clears them.
__device__ __forceinline__ void warp_flush_tri(unsigned long long (&acc)[8],
                                               unsigned long long *__restrict__ cells) {
#pragma unroll
    for (int c = 0; c < 8; c++) {
        unsigned long long v = acc[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&cells[32 + 8 + c], v);
        acc[c] = 0;
    }
}

// k_tri_join: each warp takes units of 32 consecutive jobs of one segment
// from a shared head (one atomic per unit, in index order) and runs their
// probes as one flattened list, the hash lookups through the warp's queue. When its next unit belongs to another segment the warp
// drains its queue and adds its counters into the segment's cells.
template <bool ONE, bool SHARD>
__global__ void __launch_bounds__(THREADS, 5)
    k_tri_join(const __grid_constant__ SegArgs A, const TriEdge *__restrict__ jobs,
               const int32_t *__restrict__ njobs, const int32_t *__restrict__ tj_pre,
               int32_t *__restrict__ head) {
    __shared__ TriEdge edges[TRI_WARPS][32];
    __shared__ int32_t incl[TRI_WARPS][32];
    __shared__ TriProbe queue[TRI_WARPS][TRI_QUEUE];
    unsigned long long acc[8];
#pragma unroll
    for (int c = 0; c < 8; c++) acc[c] = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nu = list_units<ONE>(A, tj_pre, njobs, 32);
    int qn = 0;
    int32_t cur = -1;
    while (true) {
        // the next unit from the shared head: the joins of hub pairs are long,
        // so warps draw units as they finish instead of a fixed share
        int32_t un = 0;
        if (lane == 0) un = atomicAdd(head, 1);
        const int64_t u = __shfl_sync(0xffffffffu, un, 0);
        if (u >= nu) break;
        int64_t ui;
        const int32_t c = list_unit_seg<ONE>(A, tj_pre, u, &ui);  // warp-uniform
        if constexpr (!ONE) {
            if (c != cur && cur >= 0) {
                const Segment &prev = seg_ref<ONE>(A, cur);
                tri_run_queue<SHARD>(prev.g, queue[warp], qn, acc);
                qn = 0;
                __syncwarp();
                warp_flush_tri(acc, prev.cells);
            }
            cur = c;
        }
        const Segment &sg = seg_ref<ONE>(A, c);
        const int64_t j = ui * 32 + lane;
        TriEdge E;
        E.work = 0;
        if (j < njobs[c]) E = jobs[sg.xbase / 2 + j];
        const int32_t inc = warp_incl_scan_i32(E.work);
        const int32_t total = __shfl_sync(0xffffffffu, inc, 31);
        edges[warp][lane] = E;
        incl[warp][lane] = inc;
        __syncwarp();
        tri_probes_queued<SHARD>(sg.g, edges[warp], incl[warp], total, queue[warp], qn, acc);
        __syncwarp();
    }
    if constexpr (ONE) {
        tri_run_queue<SHARD>(A.seg0.g, queue[warp], qn, acc);
        block_flush<8, 0>(acc, 32 + 8, A.seg0.cells);
    } else if (cur >= 0) {
        const Segment &last = seg_ref<ONE>(A, cur);
        tri_run_queue<SHARD>(last.g, queue[warp], qn, acc);
        warp_flush_tri(acc, last.cells);
    }
}

// Type II at the listed centres only: the entries of one centre, each as the
// later centre edge e_j, joined with the window of its other endpoint; only
// the matches whose type-II centre is this centre are counted.
__global__ void __launch_bounds__(THREADS)
    k_tri_centre(const DevGraph g, int64_t delta, int32_t begin, int32_t end,
                 unsigned long long *__restrict__ cells) {
    unsigned long long acc[8];
#pragma unroll
    for (int c = 0; c < 8; c++) acc[c] = 0;
    for (int64_t i = begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < end;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = (int32_t)i;
        const uint2 en = g.tn[r];
        const int64_t et = g.tt[r];
        const int dj = dir_of(en.x);
        const uint32_t u = (uint32_t)g.tc[r], w = node_of(en.x);
        const int32_t rank_j = (int32_t)en.y;
        const int32_t lo_u = gallop_lo(g.tt, g.off[u], r, et - delta);
        if (lo_u == r) continue;
        const int32_t twin = dj ? g.pos_src[rank_j] : g.pos_dst[rank_j];
        const int32_t lo_w = gallop_lo(g.tt, g.off[w], twin, et - delta);
        if (lo_w == twin) continue;
        const int32_t rank_lo_w = (int32_t)g.tn[lo_w].y;
        // items a of W_u, matches k of W_w ranked after a: centred at u
        for (int32_t a = lo_u; a < r; a++) {
            const uint2 ea = g.tn[a];
            const uint32_t x = node_of(ea.x);
            if (x == w) continue;
            PairCounts c;
            if (!pair_counts(g, pair_key(w, x), rank_lo_w, rank_j, (int32_t)ea.y, c)) continue;
            const int32_t from_x = x < w ? c.fa : c.na - c.fa;  // e_k = x -> w: o w.r.t. x
            const int32_t cnt = c.na;
            const int di = dir_of(ea.x);
            if (di) {
                if (dj) { acc[IX(1, 1, 0)] += from_x; acc[IX(1, 1, 1)] += cnt - from_x; }
                else { acc[IX(1, 0, 0)] += from_x; acc[IX(1, 0, 1)] += cnt - from_x; }
            } else {
                if (dj) { acc[IX(0, 1, 0)] += from_x; acc[IX(0, 1, 1)] += cnt - from_x; }
                else { acc[IX(0, 0, 0)] += from_x; acc[IX(0, 0, 1)] += cnt - from_x; }
            }
        }
    }
    block_flush<8, 0>(acc, 32 + 8, cells);
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

// ------------------------------------------------------- several windows
//
// A sorted list of windows delta_0 <= ... <= delta_{K-1} in one sweep
// (K <= MAX_DELTAS). The windows of one entry nest, W_0(r) within ... within
// W_{K-1}(r), so one pass finds every entry's K window starts (the largest by
// the usual search, each smaller one by galloping forwards from the next
// larger), and one walk of a back-active entry's same-neighbour links serves
// every window: the entries a >= lo_k(r) of the walk (a prefix of it, as the
// walk goes backwards) make window k's W terms, and the links up to hi_k(p)
// (a prefix of the forward walk) its F term. The Tri joins then run one
// segment per window on these window starts.
constexpr int MAX_DELTAS = 8;

struct DeltaList {
    int64_t d[MAX_DELTAS];  // ascending
    int32_t k;
};

// wl[k * 2m + r] = lo_k(r) for every entry r and window k; the back-active
// entries of the largest window are listed in act (count *nact).
template <int K>
__global__ void __launch_bounds__(THREADS)
    k_window_lo_multi(const __grid_constant__ DevGraph g, const __grid_constant__ DeltaList D,
                      int32_t *__restrict__ wl, int32_t *__restrict__ act,
                      int32_t *__restrict__ nact) {
    __shared__ int32_t buf[THREADS / 32][64];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t *wb = buf[warp];
    const int64_t n2 = 2 * g.m;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t dmax = D.d[K - 1];
    for (int64_t c0 = wid * COUNT_ECHUNK; c0 < n2; c0 += nwarps * COUNT_ECHUNK) {
        const int64_t end = c0 + COUNT_ECHUNK < n2 ? c0 + COUNT_ECHUNK : n2;
        int cnt = 0;
        int32_t prev_u = -1;
        int32_t prev_lo[MAX_DELTAS];  // this lane's window starts 32 entries before
        for (int gi = 0; gi < COUNT_ECHUNK / 32; gi++) {
            const int64_t i = c0 + gi * 32 + lane;
            bool active = false;
            if (i < end) {
                const int32_t r = (int32_t)i;
                const int64_t tr = g.tt[r];
                const int32_t cu = g.tc[r];
                int32_t lo = r;
                if (cu == prev_u) {
                    // every window slid by about 32 entries: search forwards from the
                    // lane's previous start of the same window
#pragma unroll
                    for (int k = K - 1; k >= 0; k--) {
                        const int32_t l = gallop_fwd(g.tt, prev_lo[k], r, tr - D.d[k], 32);
                        prev_lo[k] = l;
                        wl[(int64_t)k * n2 + r] = l;
                    }
                    lo = prev_lo[K - 1];
                } else {
                    // a new centre: the largest window by the backward search, each
                    // smaller one by galloping forwards from the next larger
                    const int32_t sb = g.off[cu];
                    if (r > sb && tr - g.tt[r - 1] <= dmax) lo = gallop_lo(g.tt, sb, r, tr - dmax);
                    int32_t l = lo;
#pragma unroll
                    for (int k = K - 1; k >= 0; k--) {
                        if (k < K - 1 && l < r) l = gallop_fwd(g.tt, l, r, tr - D.d[k], 1);
                        prev_lo[k] = l;
                        wl[(int64_t)k * n2 + r] = l;
                    }
                }
                prev_u = cu;
                active = lo < r && g.lk[r].x >= lo;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, active);
            if (active) wb[cnt + __popc(bal & ((1u << lane) - 1u))] = (int32_t)i;
            cnt += __popc(bal);
            __syncwarp();
            warp_append(wb, cnt, false, act, nact);
        }
        warp_append(wb, cnt, true, act, nact);
    }
}

// Window k's W(r) terms from the running sums over the entries a >= lo of
// the walk (as in star_pair_back_active), into the lane copies `sacc`.
__device__ __forceinline__ void emit_w_terms(const DevGraph &g, int D3, int32_t r, int32_t seg_end,
                                             int64_t cin_r, int64_t cin_end, int32_t lo,
                                             const uint64_t (&n)[2], const uint64_t (&c2s)[2][2],
                                             const uint64_t (&X)[2][2], const uint64_t (&Yp)[2][2],
                                             unsigned long long *sacc) {
    const int64_t cin_lo = g.cin[lo];
    const int64_t co_lo = (int64_t)lo - cin_lo;
#pragma unroll
    for (int d1 = 0; d1 < 2; d1++)
#pragma unroll
        for (int d2 = 0; d2 < 2; d2++) {
            const uint64_t sp = c2s[d1][d2];
            lane_add(sacc, IX(d1, d2, D3), sp);                                  // Pair
            lane_add(sacc, 16 + IX(d1, d2, D3), X[d1][d2] - sp);                 // Star-II
            const uint64_t base = d1 ? (uint64_t)cin_lo : (uint64_t)co_lo;      // C_d1(lo)
            lane_add(sacc, 8 + IX(d1, d2, D3), Yp[d2][d1] - n[d2] * base - sp);  // Star-I
            lane_add(sacc, 24 + IX(d1, d2, D3), 0 - sp);                         // Star-III
        }
    const int64_t after_in = cin_end - (cin_r + D3);
    const int64_t after_o = (int64_t)(seg_end - r - 1) - after_in;
#pragma unroll
    for (int d1 = 0; d1 < 2; d1++) {
        lane_add(sacc, 24 + IX(d1, D3, 0), n[d1] * (uint64_t)after_o);
        lane_add(sacc, 24 + IX(d1, D3, 1), n[d1] * (uint64_t)after_in);
    }
}

// The Star/Pair terms of the listed entry r (back-active in the largest
// window) for every window it is back-active in, from one backward and one
// forward walk of its same-neighbour links. Window k's copies of the 32 cells
// start at sacc + k * 32 * SP_COPIES.
// The element k of a (register-resident) array, k known only at run time.
template <int K>
__device__ __forceinline__ int32_t pick(const int32_t (&a)[K], int k) {
    int32_t v = a[0];
#pragma unroll
    for (int i = 1; i < K; i++)
        if (k == i) v = a[i];
    return v;
}

template <int K>
__device__ __forceinline__ void star_pair_back_active_multi(const DevGraph &g, const DeltaList &D,
                                                            const int32_t *__restrict__ wl,
                                                            int32_t r,
                                                            unsigned long long *sacc) {
    const int64_t *__restrict__ tt = g.tt;
    const int64_t n2 = 2 * g.m;
    const int32_t u = g.tc[r];
    const int32_t seg_end = g.off[u + 1];
    const int D3 = dir_of(g.tn[r].x);
    const int64_t cin_end = g.cin[seg_end];
    const int64_t cin_r = g.cin[r];
    const int2 lr = g.lk[r];
    int32_t lo[K];
#pragma unroll
    for (int k = 0; k < K; k++) lo[k] = wl[(int64_t)k * n2 + r];
    {
        // backward walk: window k takes the prefix of entries a >= lo[k]
        // running sums in scalars (as in star_pair_back_active), so that they stay
        // in registers
        uint64_t n0 = 0, n1 = 0, c00 = 0, c01 = 0, c10 = 0, c11 = 0;
        uint64_t X00 = 0, X01 = 0, X10 = 0, X11 = 0, Y00 = 0, Y01 = 0, Y10 = 0, Y11 = 0;
        int32_t a = lr.x, cur = r;
        int k = 0;  // windows finished so far (smallest first: their starts are highest)
        while (true) {
            const bool more = a >= lo[K - 1] && a < cur;  // links strictly decrease: ends
            while (k < K && (!more || a < pick(lo, k))) {
                const int32_t lok = pick(lo, k);
                if (lr.x >= lok) {
                    const uint64_t n[2] = {n0, n1};
                    const uint64_t c2s[2][2] = {{c00, c01}, {c10, c11}};
                    const uint64_t X[2][2] = {{X00, X01}, {X10, X11}};
                    const uint64_t Yp[2][2] = {{Y00, Y01}, {Y10, Y11}};
                    emit_w_terms(g, D3, r, seg_end, cin_r, cin_end, lok, n, c2s, X, Yp,
                                 sacc + k * 32 * SP_COPIES);
                }
                k++;
            }
            if (!more) break;
            const int da = dir_of(g.tn[a].x);
            const int64_t cin_a = g.cin[a];
            const uint64_t between_in = (uint64_t)(cin_r - (cin_a + da));
            const uint64_t between_o = (uint64_t)(r - a - 1) - between_in;
            const uint64_t co_a = (uint64_t)(a - cin_a), ci_a = (uint64_t)cin_a;
            if (da) {
                c10 += n0;
                c11 += n1;
                n1 += 1;
                X10 += between_o;
                X11 += between_in;
                Y10 += co_a;
                Y11 += ci_a;
            } else {
                c00 += n0;
                c01 += n1;
                n0 += 1;
                X00 += between_o;
                X01 += between_in;
                Y00 += co_a;
                Y01 += ci_a;
            }
            cur = a;
            a = g.lk[a].x;
        }
    }
    {
        // forward walk from r for the predecessor p: window k takes the links
        // up to hi_k(p), for the windows in which r is back-active
        const int32_t p = lr.x;
        const int64_t tp = tt[p];
        const int Dp = dir_of(g.tn[p].x);
        int k = 0;
        while (k < K && lr.x < pick(lo, k)) k++;  // r is back-active in windows k..K-1
        // hi_j(p) of those windows, each searched from the previous one's
        int32_t his[K];
        int32_t h = r;
#pragma unroll
        for (int j = 0; j < K; j++) {
            if (j >= k) h = gallop_hi(tt, h, seg_end, tp, D.d[j]);
            his[j] = h;
        }
        const int32_t hmax = his[K - 1];
        int32_t hi = pick(his, k < K ? k : K - 1);
        uint64_t f0 = 0, f1 = 0;
        int32_t b = r, cur = p;
        while (k < K) {
            const bool more = b > cur && b <= hmax;  // links strictly increase: ends
            while (k < K && (!more || b > hi)) {
                const int64_t cin_h1 = (int64_t)g.cin[hi] + dir_of(g.tn[hi].x);  // C_in(hi+1)
                const int64_t after_in = cin_end - cin_h1;
                const int64_t after_o = (int64_t)(seg_end - hi - 1) - after_in;
                unsigned long long *sk = sacc + k * 32 * SP_COPIES;
                lane_add(sk, 24 + IX(Dp, 0, 0), 0 - f0 * (uint64_t)after_o);
                lane_add(sk, 24 + IX(Dp, 0, 1), 0 - f0 * (uint64_t)after_in);
                lane_add(sk, 24 + IX(Dp, 1, 0), 0 - f1 * (uint64_t)after_o);
                lane_add(sk, 24 + IX(Dp, 1, 1), 0 - f1 * (uint64_t)after_in);
                k++;
                if (k < K) hi = pick(his, k);
            }
            if (!more) break;
            if (dir_of(g.tn[b].x)) f1 += 1;
            else f0 += 1;
            cur = b;
            b = g.lk[b].y;
        }
    }
}

// The Star/Pair sweep of several windows: the entries listed by
// k_window_lo_multi, with K sets of lane copies of the 32 cells in dynamic
// shared memory; window k's cells go to cells + 56 k.
template <int K>
__global__ void __launch_bounds__(THREADS, 4)
    k_star_pair_list_multi(const __grid_constant__ DevGraph g, const __grid_constant__ DeltaList D,
                           const int32_t *__restrict__ wl, const int32_t *__restrict__ act,
                           const int32_t *__restrict__ nact_ptr, int32_t *__restrict__ head,
                           unsigned long long *__restrict__ cells) {
    extern __shared__ unsigned long long msacc[];  // [K][32 * SP_COPIES]
    for (int i = threadIdx.x; i < K * 32 * SP_COPIES; i += blockDim.x) msacc[i] = 0;
    const int32_t nact = *nact_ptr;
    unsigned long long *mine = msacc + (threadIdx.x & 31);
    __shared__ int32_t next;
    while (true) {
        // units of SP_CHUNK listed entries from a shared head, as k_star_pair_list
        __syncthreads();
        if (threadIdx.x == 0) next = atomicAdd(head, 1);
        __syncthreads();
        const int64_t u = next;
        if (u * SP_CHUNK >= nact) break;
        for (int j = 0; j < SP_CHUNK / THREADS; j++) {
            const int64_t i = u * SP_CHUNK + j * THREADS + threadIdx.x;
            if (i >= nact) break;
            star_pair_back_active_multi<K>(g, D, wl, act[i], mine);
        }
    }
    __syncthreads();
    for (int k = 0; k < K; k++)
        flush_lane_copies(msacc + k * 32 * SP_COPIES, cells + (size_t)NCELLS * k);
}

// Type-I/III Tri cells of every segment from its type-II cells.
template <bool ONE>
__global__ void k_fill_tri_types_seg(const __grid_constant__ SegArgs A) {
    const int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= seg_count<ONE>(A)) return;
    unsigned long long *tri = seg_ref<ONE>(A, c).cells + 32;
    for (int di = 0; di < 2; di++)
        for (int dj = 0; dj < 2; dj++)
            for (int dk = 0; dk < 2; dk++) {
                const unsigned long long v = tri[8 + IX(di, dj, dk)];
                tri[IX(1 - dk, 1 - dj, 1 - di)] = v;  // type I
                tri[16 + IX(1 - di, dk, dj)] = v;     // type III
            }
}

}  // namespace

int kernel_binary_version() {
    cudaFuncAttributes a;
    TM_CUDA(cudaFuncGetAttributes(&a, k_fill_tri_types));
    return a.binaryVersion;
}

namespace {

template <typename K>
int occupancy(K kernel) {
    int nb = 0;
    TM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, THREADS, 0));
    return nb > 0 ? nb : 1;
}

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

size_t count_scratch_bytes(int64_t entries, int32_t k) {
    const int64_t e = entries > 0 ? entries : 1;
    return align_up(sizeof(int32_t) * e) + align_up(sizeof(int32_t) * e) +
           align_up(sizeof(TriEdge) * (e / 2 + 1)) + align_up(sizeof(int32_t) * (4 * (size_t)k + 4));
}

void count_scratch_carve(void *base, int64_t entries, int32_t k, CountScratch &sc) {
    const int64_t e = entries > 0 ? entries : 1;
    char *p = static_cast<char *>(base);
    sc.wl = reinterpret_cast<int32_t *>(p);
    p += align_up(sizeof(int32_t) * e);
    sc.act = reinterpret_cast<int32_t *>(p);
    p += align_up(sizeof(int32_t) * e);
    sc.jobs = p;
    p += align_up(sizeof(TriEdge) * (e / 2 + 1));
    // heads[2] | nact[k] | njobs[k] | sp_pre[k+1] | tj_pre[k+1]
    sc.counts = reinterpret_cast<int32_t *>(p);
    sc.k_cap = k;
}

int count_join_blocks_per_sm() { return occupancy(k_tri_join<false, false>); }

void launch_count_segments(const Segment *one, const Segment *d_segs, const int32_t *d_meta,
                           int32_t k_cap, bool star_pair, bool tri, bool fill,
                           const CountScratch &sc, cudaStream_t s, int join_blocks_per_sm,
                           int32_t echunk, const int32_t *own, int32_t own_rank,
                           bool windows_ready) {
    if (echunk < 128 || echunk % 128) fail(TM_EINVAL, "entries per unit must be a multiple of 128");
    SegArgs A;
    std::memset(&A, 0, sizeof(A));
    A.echunk = echunk;
    A.own = own;
    A.own_rank = own_rank;
    const int sms = num_sms();
    // the streaming passes: one block per 8 units, at most 8 blocks per SM (a
    // table's unit count is only known on the device: the cap)
    int64_t stream_blocks = (int64_t)sms * 8;
    if (one) {
        A.seg0 = *one;
        const int64_t units = ((int64_t)one->end - one->begin + echunk - 1) / echunk;
        if (units == 0) return;
        stream_blocks = std::min(stream_blocks, (units + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK);
    } else {
        A.segs = d_segs;
        A.eunit = d_meta;
    }
    const int k = one ? 1 : k_cap;
    int32_t *heads = sc.counts, *nact = sc.counts + 2, *njobs = sc.counts + 2 + k,
            *sp_pre = sc.counts + 2 + 2 * k, *tj_pre = sc.counts + 3 + 3 * k;
    TM_CUDA(cudaMemsetAsync(sc.counts, 0, sizeof(int32_t) * (2 + 2 * k), s));
    {
        PhaseTimer pt(TM_PH_STAR_PAIR, s);
        int32_t *act = star_pair ? sc.act : nullptr;
        if (windows_ready && star_pair) fail(TM_EINVAL, "window starts given without a list");
        if (windows_ready) {
            // the caller wrote sc.wl
        } else if (one) {
            TM_LAUNCH(k_window_lo<true>, (unsigned)stream_blocks, THREADS, 0, s, A, sc.wl, act, nact);
        } else {
            TM_LAUNCH(k_window_lo<false>, (unsigned)stream_blocks, THREADS, 0, s, A, sc.wl, act, nact);
        }
        if (star_pair) {
            const unsigned grid = (unsigned)(sms * occupancy(k_star_pair_list<true>));
            if (one) {
                TM_LAUNCH(k_star_pair_list<true>, grid, THREADS, 0, s, A, sc.wl, sc.act, nact, sp_pre,
                          heads);
            } else {
                TM_LAUNCH(k_unit_prefix, 1, 1024, 0, s, d_meta, nact, SP_CHUNK, sp_pre);
                TM_LAUNCH(k_star_pair_list<false>, grid, THREADS, 0, s, A, sc.wl, sc.act, nact, sp_pre,
                          heads);
            }
        }
    }
    if (tri) {
        PhaseTimer pt(TM_PH_TRI, s);
        TriEdge *jobs = static_cast<TriEdge *>(sc.jobs);
        const int occ = occupancy(k_tri_join<true, false>);
        const int bps = join_blocks_per_sm > 0 ? std::min(join_blocks_per_sm, occ) : occ;
        // a whole graph that kept its rank-ordered endpoints: jobs in rank order
        const bool ranks = one && one->g.sd != nullptr && one->begin == 0 &&
                           (int64_t)one->end == 2 * one->g.m;
        if (one && own) {
            if (ranks)
                TM_LAUNCH((k_tri_jobs_ranks<true>), (unsigned)stream_blocks, THREADS, 0, s, A,
                          sc.wl, jobs, njobs);
            else
                TM_LAUNCH((k_tri_jobs<true, true>), (unsigned)stream_blocks, THREADS, 0, s, A,
                          sc.wl, jobs, njobs);
            TM_LAUNCH((k_tri_join<true, true>), (unsigned)(sms * bps), THREADS, 0, s, A, jobs, njobs,
                      tj_pre, heads + 1);
            if (fill) TM_LAUNCH(k_fill_tri_types_seg<true>, 1, 128, 0, s, A);
        } else if (one) {
            if (ranks)
                TM_LAUNCH((k_tri_jobs_ranks<false>), (unsigned)stream_blocks, THREADS, 0, s, A,
                          sc.wl, jobs, njobs);
            else
                TM_LAUNCH((k_tri_jobs<true, false>), (unsigned)stream_blocks, THREADS, 0, s, A,
                          sc.wl, jobs, njobs);
            TM_LAUNCH((k_tri_join<true, false>), (unsigned)(sms * bps), THREADS, 0, s, A, jobs,
                      njobs, tj_pre, heads + 1);
            if (fill) TM_LAUNCH(k_fill_tri_types_seg<true>, 1, 128, 0, s, A);
        } else {
            if (own) fail(TM_EINVAL, "a shard of centres needs one segment");
            TM_LAUNCH((k_tri_jobs<false, false>), (unsigned)stream_blocks, THREADS, 0, s, A, sc.wl,
                      jobs, njobs);
            TM_LAUNCH(k_unit_prefix, 1, 1024, 0, s, d_meta, njobs, 32, tj_pre);
            TM_LAUNCH((k_tri_join<false, false>), (unsigned)(sms * bps), THREADS, 0, s, A, jobs,
                      njobs, tj_pre, heads + 1);
            if (fill)
                TM_LAUNCH(k_fill_tri_types_seg<false>, (unsigned)((k + 127) / 128), 128, 0, s, A);
        }
    }
}

void launch_count(const DevGraph &g, int64_t delta, int32_t begin, int32_t end,
                  unsigned long long *dev_cells, cudaStream_t s) {
    if (end <= begin) return;
    const int64_t n = end - begin;
    int64_t blocks = (n + THREADS - 1) / THREADS;
    const int64_t cap = (int64_t)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    if (begin == 0 && end == 2 * g.m) {
        launch_count_parts(g, delta, true, true, dev_cells, s, false);
        return;
    }
    {
        PhaseTimer pt(TM_PH_STAR_PAIR, s);
        TM_LAUNCH(k_star_pair, (unsigned)blocks, THREADS, 0, s, g, delta, begin, end, dev_cells);
    }
    {
        PhaseTimer pt(TM_PH_TRI, s);
        TM_LAUNCH(k_tri_centre, (unsigned)blocks, THREADS, 0, s, g, delta, begin, end, dev_cells);
    }
}

// The window pass and the Star/Pair sweep of K windows.
template <int K>
void multi_sweep(const DevGraph &g, const DeltaList &D, const CountScratch &sc, int32_t *nact,
                 int32_t *head, unsigned long long *dev_cells, unsigned blocks, cudaStream_t s) {
    TM_LAUNCH(k_window_lo_multi<K>, blocks, THREADS, 0, s, g, D, sc.wl, sc.act, nact);
    const size_t smem = sizeof(unsigned long long) * 32 * SP_COPIES * K;
    static std::atomic<unsigned long long> attr_devices{0};
    const int dev = current_device_id();
    if (dev >= 64 || !((attr_devices.load() >> dev) & 1ull)) {
        TM_CUDA(cudaFuncSetAttribute(k_star_pair_list_multi<K>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (dev < 64) attr_devices.fetch_or(1ull << dev);
    }
    int per_sm = 0;
    TM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_star_pair_list_multi<K>,
                                                          THREADS, smem));
    TM_LAUNCH(k_star_pair_list_multi<K>, (unsigned)(num_sms() * std::max(1, per_sm)), THREADS,
              smem, s, g, D, sc.wl, sc.act, nact, head, dev_cells);
}

void launch_count_multi_delta(const DevGraph &g, const int64_t *deltas, int32_t k,
                              unsigned long long *dev_cells, cudaStream_t s) {
    const int64_t n2 = 2 * g.m;
    if (n2 == 0 || k <= 0) return;
    if (k > MAX_DELTAS) fail(TM_EINVAL, "at most 8 windows per sweep");
    DeltaList D;
    std::memset(&D, 0, sizeof D);
    D.k = k;
    for (int32_t i = 0; i < k; i++) {
        if (deltas[i] < 0 || (i > 0 && deltas[i] < deltas[i - 1]))
            fail(TM_EINVAL, "windows must be >= 0 and ascending");
        D.d[i] = deltas[i];
    }
    const int64_t total = n2 * k;
    if (total >= (int64_t(1) << 31)) fail(TM_EINVAL, "2m * windows must be < 2^31");
    // one segment per window, all on the whole graph, their scratch one after another
    std::vector<Segment> segs(k);
    for (int32_t i = 0; i < k; i++) {
        segs[i].g = g;
        segs[i].delta = deltas[i];
        segs[i].cells = dev_cells + (size_t)NCELLS * i;
        segs[i].begin = 0;
        segs[i].end = (int32_t)n2;
        segs[i].xbase = n2 * i;
    }
    void *mem = dev_alloc(count_scratch_bytes(total, k), s);
    CountScratch sc;
    count_scratch_carve(mem, total, k, sc);
    try {
        // list count and unit head (free until the Tri launches clear the counters)
        int32_t *nact = sc.counts, *head = sc.counts + 1;
        TM_CUDA(cudaMemsetAsync(nact, 0, sizeof(int32_t) * 2, s));
        const int sms = num_sms();
        {
            PhaseTimer pt(TM_PH_STAR_PAIR, s);
            int64_t blocks = (n2 / COUNT_ECHUNK + WARPS_PER_BLOCK) / WARPS_PER_BLOCK;
            blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sms * 8));
            switch (k) {
                case 1: multi_sweep<1>(g, D, sc, nact, head, dev_cells, (unsigned)blocks, s); break;
                case 2: multi_sweep<2>(g, D, sc, nact, head, dev_cells, (unsigned)blocks, s); break;
                case 3: multi_sweep<3>(g, D, sc, nact, head, dev_cells, (unsigned)blocks, s); break;
                case 4: multi_sweep<4>(g, D, sc, nact, head, dev_cells, (unsigned)blocks, s); break;
                case 5: multi_sweep<5>(g, D, sc, nact, head, dev_cells, (unsigned)blocks, s); break;
                case 6: multi_sweep<6>(g, D, sc, nact, head, dev_cells, (unsigned)blocks, s); break;
                case 7: multi_sweep<7>(g, D, sc, nact, head, dev_cells, (unsigned)blocks, s); break;
                default: multi_sweep<8>(g, D, sc, nact, head, dev_cells, (unsigned)blocks, s); break;
            }
        }
        // the Tri joins of each window on its window starts, one segment at a time
        // (the graph read in place from the kernels' parameters)
        for (int32_t i = 0; i < k; i++)
            launch_count_segments(&segs[i], nullptr, nullptr, 1, false, true, true, sc, s, 0,
                                  COUNT_ECHUNK, nullptr, 0, true);
    } catch (...) {
        dev_free(mem, s);
        throw;
    }
    dev_free(mem, s);
}

void launch_count_parts(const DevGraph &g, int64_t delta, bool star_pair, bool tri,
                        unsigned long long *dev_cells, cudaStream_t s, bool fill,
                        const int32_t *own, int32_t own_rank) {
    const int64_t n = 2 * g.m;
    if (n == 0) return;
    Segment one;
    one.g = g;
    one.delta = delta;
    one.cells = dev_cells;
    one.begin = 0;
    one.end = (int32_t)n;
    one.xbase = 0;
    void *mem = dev_alloc(count_scratch_bytes(n, 1), s);
    CountScratch sc;
    count_scratch_carve(mem, n, 1, sc);
    launch_count_segments(&one, nullptr, nullptr, 1, star_pair, tri, fill, sc, s, 0,
                          COUNT_ECHUNK, own, own_rank);
    dev_free(mem, s);
}

void launch_count_untimed(const DevGraph &g, int64_t delta, unsigned long long *dev_cells,
                          cudaStream_t s) {
    const int64_t n = 2 * g.m;
    if (n == 0) return;
    int64_t blocks = (n + THREADS - 1) / THREADS;
    const int64_t cap = (int64_t)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    TM_LAUNCH(k_star_pair, (unsigned)blocks, THREADS, 0, s, g, delta, 0, (int32_t)n, dev_cells);
    TM_LAUNCH(k_tri, (unsigned)blocks, THREADS, 0, s, g, delta, 0, (int32_t)n, dev_cells);
    TM_LAUNCH(k_fill_tri_types, 1, 32, 0, s, dev_cells);
}

void launch_fill_tri_types(unsigned long long *dev_cells, cudaStream_t s) {
    TM_LAUNCH(k_fill_tri_types, 1, 32, 0, s, dev_cells);
}

}  // namespace tmi
