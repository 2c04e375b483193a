// count_common.cuh -- device helpers shared by the counting kernels (the
// ordered DFS in count.cu and the pivoting counter in sct.cu): launch
// context, the colour hash of cFFF_k, 128-bit total accumulation, and the
// G+(u) bitmap builders.
#pragma once

#include <climits>

#include "kc_internal.cuh"

namespace kc {
namespace cc {

// One oriented graph as the kernels see it (device pointers).
struct GraphDesc {
    const int64_t* offp;
    const int32_t* adjp;
    const int32_t* queue;
    const int32_t* perm;
};

// Launch context of one owner class.  Single-graph mode (ng == 0): item i is
// the owner at queue position q0 + qoff + i * qstride (qoff/qstride select a
// part of the owners).  Batch mode (ng > 0): item i belongs to graph g with
// gpre[g] <= i < gpre[g+1] and is the owner at position gq0[g] + i - gpre[g]
// of that graph's queue; totals are per graph.
struct Ctx {
    const int64_t* __restrict__ offp;
    const int32_t* __restrict__ adjp;
    const int32_t* __restrict__ queue;
    const int32_t* __restrict__ perm;
    int64_t q0, q1;
    int64_t nitems;
    int64_t qoff, qstride;
    const GraphDesc* gd;
    const int64_t* gq0;
    const int64_t* gpre;
    int ng;
    int k;
    uint32_t colours;
    uint64_t seed;
    int pair;        // plain pair sampling instead of colours (Sec. 6)
    uint64_t pthr;   // pair kept iff its hash < pthr
    unsigned long long* total;
    unsigned long long* pv;
    unsigned long long* po;
    unsigned long long* cursor;
    unsigned long long* work;  // nullable: bitmap word-operations executed
};

// The owner (rank r) of class item `item`, with a context whose graph
// pointers and total are that owner's graph's.  False past the last item.
__device__ __forceinline__ bool resolve(const Ctx& b, int64_t item, Ctx& c, int32_t& r)
{
    if (item >= b.nitems) return false;
    c = b;
    if (b.ng == 0) {
        r = b.queue[b.q0 + b.qoff + item * b.qstride];
        return true;
    }
    int lo = 0, hi = b.ng;  // largest g with gpre[g] <= item
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (b.gpre[mid] <= item) lo = mid; else hi = mid;
    }
    const GraphDesc gd = b.gd[lo];
    c.offp = gd.offp;
    c.adjp = gd.adjp;
    c.queue = gd.queue;
    c.perm = gd.perm;
    c.total = b.total + 2 * lo;
    r = gd.queue[b.gq0[lo] + (item - b.gpre[lo])];
    return true;
}

// colour(u, x): splitmix64 output function over seed ^ (G * (u<<32 | x)),
// reduced to [0, c) by a 64x64 multiply-high (Sec. 6; spec in kc.h).
__device__ __forceinline__ uint32_t colour_of(uint64_t seed, int32_t u, int32_t x, uint32_t c)
{
    uint64_t key = ((uint64_t)(uint32_t)u << 32) | (uint64_t)(uint32_t)x;
    uint64_t z = seed ^ (0x9E3779B97F4A7C15ull * key);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (uint32_t)__umul64hi(z, (uint64_t)c);
}

// Pair sampling (Sec. 6, plain pair sampling): the pair {x, y} of Gamma+(u)
// is kept iff h < thr, h = F(F(seed ^ G (u<<32 | a)) ^ G b) with a < b the
// two original ids and F the splitmix64 output function (spec in kc.h).
__device__ __forceinline__ bool pair_kept(uint64_t seed, int32_t u, uint32_t x, uint32_t y, uint64_t thr)
{
    const uint32_t a = x < y ? x : y, b = x < y ? y : x;
    uint64_t z = seed ^ (0x9E3779B97F4A7C15ull * (((uint64_t)(uint32_t)u << 32) | (uint64_t)a));
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    z ^= 0x9E3779B97F4A7C15ull * (uint64_t)b;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z < thr;
}

// The per-node label a sampling filter keeps for x_j of Gamma+(u) (ur, xid:
// original ids): its colour under cFFF_k, its id under pair sampling.
__device__ __forceinline__ uint32_t sample_label(const Ctx& c, int32_t ur, int32_t xid)
{
    return c.pair ? (uint32_t)xid : colour_of(c.seed, ur, xid, c.colours);
}

// Whether the pair with labels li, lj survives the sampling filter.
__device__ __forceinline__ bool sample_keep(const Ctx& c, int32_t ur, uint32_t li, uint32_t lj)
{
    return c.pair ? pair_kept(c.seed, ur, li, lj, c.pthr) : li == lj;
}

// cFFF_k: a sampled (k-1)-clique of G+(u) lies inside one colour class
// (Map 2 emits monochromatic pairs only), so a vertex whose class in Gamma+(u)
// has fewer than k-1 members lies in none, and its Gamma+ list need not be
// read at all (Round 2 shrinks with the sampling).  Such a vertex's label
// gets kSkipLabel; the flag is the same for its whole class, so labels still
// compare equal exactly within a class, and the builders skip its row.
// Colours are below c <= 2^31 (the flag bit is no colour); plain pair
// sampling (labels are ids) is not filtered.
constexpr uint32_t kSkipLabel = 0x80000000u;

__device__ __forceinline__ bool class_filter_on(const Ctx& c) { return !c.pair && c.colours <= kSkipLabel; }

// Lane j holds the label of x_j (j < d): flags small classes (match_any).
__device__ __forceinline__ uint32_t class_flag_w1(const Ctx& c, uint32_t col, int d, int need, int lane)
{
    if (!class_filter_on(c)) return col;
    const uint32_t key = lane < d ? col : kSkipLabel + (uint32_t)lane;
    const uint32_t peers = __match_any_sync(kFull, key);
    return (lane < d && __popc(peers) < need) ? (col | kSkipLabel) : col;
}

// Labels sCol[0..d) in shared memory, threads t0, t0+nt, ... of the caller
// (d <= 32 nt): flags small classes.  CTA: every thread of the block calls
// it (two __syncthreads), else the lanes of one warp (two __syncwarp).
template <bool CTA>
__device__ __forceinline__ void class_flags_smem(const Ctx& c, uint32_t* sCol, int d, int need, int t0, int nt)
{
    if (!class_filter_on(c)) return;
    uint32_t small = 0;  // bit q: element t0 + q nt is in a class smaller than need
    for (int q = 0; q < 32; ++q) {
        const int j = t0 + q * nt;
        if (j >= d) break;
        const uint32_t cj = sCol[j];
        int cnt = 0;
        for (int i = 0; i < d && cnt < need; ++i) cnt += sCol[i] == cj;
        if (cnt < need) small |= 1u << q;
    }
    if (CTA) __syncthreads(); else __syncwarp();
    for (int q = 0; q < 32; ++q) {
        const int j = t0 + q * nt;
        if (j >= d) break;
        if ((small >> q) & 1u) sCol[j] |= kSkipLabel;
    }
    if (CTA) __syncthreads(); else __syncwarp();
}

// 128-bit total as (lo, hi) words.
__device__ __forceinline__ void add_total(unsigned long long* t, unsigned long long v)
{
    if (v == 0) return;
    unsigned long long old = atomicAdd(&t[0], v);
    if (old + v < old) atomicAdd(&t[1], 1ull);
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ uint32_t mask_above(int b) { return b >= 31 ? 0u : (kFull << (b + 1)); }
__device__ __forceinline__ uint32_t mask_below(int b) { return (1u << b) - 1u; }


// Rows of G+(u) for an owner with d <= 32 (Map 2 pairs kept by Reduce 2):
// lane j holds x_j (rank, INT_MAX past d); returns, in lane i, the word whose
// bit j (j > i) is set iff x_j is in Gamma+(x_i) -- each Gamma+(x_i) chunk of
// 32 entries is searched for x_j by a shuffle binary search, and the scan
// stops at max Gamma+(u).  Under sampling (COL) lane j holds x_j's label and
// only pairs passing sample_keep are kept (ur: u's original id).
template <bool COL>
__device__ __forceinline__ uint32_t build_rows_w1(const Ctx& c, int32_t x, int d, uint32_t col, int32_t ur,
                                                  int lane)
{
    const int32_t maxL = __shfl_sync(kFull, x, d - 1);
    uint32_t up = 0;
    for (int i = 0; i < d - 1; ++i) {
        if (COL && (__shfl_sync(kFull, col, i) & kSkipLabel)) continue;  // too small a colour class
        const int32_t xi = __shfl_sync(kFull, x, i);
        const int64_t s0 = c.offp[xi], s1 = c.offp[xi + 1];
        uint32_t row = 0;
        for (int64_t p0 = s0; p0 < s1; p0 += 32) {
            const int64_t p = p0 + lane;
            const int32_t y = p < s1 ? c.adjp[p] : INT_MAX;
            int lo = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int32_t yy = __shfl_sync(kFull, y, lo + step - 1);
                if (yy < x) lo += step;
            }
            const int32_t yl = __shfl_sync(kFull, y, lo);
            row |= __ballot_sync(kFull, lane > i && lane < d && yl == x);
            if (__shfl_sync(kFull, y, 31) >= maxL) break;
        }
        if (COL) row &= __ballot_sync(kFull, sample_keep(c, ur, __shfl_sync(kFull, col, i), col));
        if (lane == i) up = row;
    }
    return up;
}

// Lower half of the symmetric G+(u) bitmap from the upper rows (bit i of
// row j for every i < j with bit j in row i).
__device__ __forceinline__ uint32_t lower_rows_w1(uint32_t up, int d, int lane)
{
    uint32_t low = 0;
    for (int j = 1; j < d; ++j) {
        const uint32_t colj = __ballot_sync(kFull, (up >> j) & 1u);
        if (lane == j) low = colj;
    }
    return low;
}

// Direct-address table over the rank span [lo, lo + 32 words) of Gamma+(u):
// bit (y - lo) set iff y is in Gamma+(u), pre[w] = number of elements below
// lo + 32 w, so y's local index is pre[w] + popc(bits[w] below y's bit).
// words == 0: no table (the span is too wide); searches fall back to binary
// search in sL.
struct SpanTable {
    uint32_t* bits;
    uint16_t* pre;
    int32_t lo;
    int words;
};

// Fill T for sL[0..d) (ascending) by the threads of the CTA when the span
// fits maxw words; ends with __syncthreads().  Every thread must call it.
__device__ __forceinline__ void span_table_build(SpanTable& T, const int32_t* sL, int d, int maxw)
{
    const int64_t span = (int64_t)sL[d - 1] - sL[0] + 1;
    T.lo = sL[0];
    T.words = span <= 32LL * maxw ? (int)((span + 31) >> 5) : 0;
    if (T.words == 0) return;
    for (int w = threadIdx.x; w < T.words; w += blockDim.x) T.bits[w] = 0u;
    __syncthreads();
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const int off = sL[j] - T.lo;
        atomicOr(&T.bits[off >> 5], 1u << (off & 31));
    }
    for (int w = threadIdx.x; w < T.words; w += blockDim.x) {
        const int32_t key = T.lo + 32 * w;
        int a = 0, z = d;
        while (a < z) {
            const int mid = (a + z) >> 1;
            if (sL[mid] < key) a = mid + 1; else z = mid;
        }
        T.pre[w] = (uint16_t)a;
    }
    __syncthreads();
}

// Rows of G+(u) into a bitmap A (row stride RS words, zeroed beforehand) by
// warps w0, w0+nw, ... of the caller; sL holds Gamma+(u) (ranks, ascending),
// sCol their sampling labels (COL; ur: u's original id).  With SYM the
// bitmap is made symmetric.
template <bool SYM, bool COL>
__device__ __forceinline__ void build_rows(const Ctx& c, const int32_t* sL, const uint32_t* sCol, int d,
                                           uint32_t* A, int RS, int w0, int nw, int lane, int32_t ur = 0,
                                           const SpanTable* T = nullptr)
{
    const int32_t maxL = sL[d - 1];
    const bool direct = T && T->words > 0;
    for (int i = w0; i < d - 1; i += nw) {
        const uint32_t ci = COL ? sCol[i] : 0u;
        if (COL && (ci & kSkipLabel)) continue;  // too small a colour class: no sampled clique
        const int32_t xi = sL[i];
        const int64_t s0 = c.offp[xi], s1 = c.offp[xi + 1];
        for (int64_t p0 = s0; p0 < s1; p0 += 32) {
            const int64_t pp = p0 + lane;
            const int32_t y = pp < s1 ? c.adjp[pp] : INT_MAX;
            if (y <= maxL) {
                int lo = i + 1;
                bool hit;
                if (direct) {  // y > x_i >= lo: inside the span
                    const int off = y - T->lo;
                    const uint32_t wv = T->bits[off >> 5];
                    hit = (wv >> (off & 31)) & 1u;
                    lo = (int)T->pre[off >> 5] + __popc(wv & mask_below(off & 31));
                } else {
                    int hi = d;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (sL[mid] < y) lo = mid + 1; else hi = mid;
                    }
                    hit = lo < d && sL[lo] == y;
                }
                if (hit && (!COL || sample_keep(c, ur, ci, sCol[lo]))) {
                    atomicOr(&A[(int64_t)i * RS + (lo >> 5)], 1u << (lo & 31));
                    if (SYM) atomicOr(&A[(int64_t)lo * RS + (i >> 5)], 1u << (i & 31));
                }
            }
            if (__shfl_sync(kFull, y, 31) >= maxL) break;
        }
    }
}

// Opt a kernel in to `smem` bytes of dynamic shared memory.  The default
// limit (48 KB) covers static and dynamic shared memory together, so the
// attribute is set whenever the dynamic part alone comes near it.
template <typename K>
inline cudaError_t allow_smem(K kernel, size_t smem)
{
    if (smem <= 32 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename K>
inline int blocks_per_sm(K kernel, int threads, size_t smem)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess || nb < 1)
        nb = 1;
    return nb;
}

}  // namespace cc
}  // namespace kc
