// list.cu -- k-clique listing: every k-clique of G once, as k caller ids in
// the order < (owner first), streamed through a caller buffer in chunks.
//
// The exact algorithm lists as well as counts (Sec. 1; Reduce 3 of Sec. 3
// enumerates the (k-1)-cliques of each G+(u)); the output can be far larger
// than device memory (Table 1's counts), so it is produced in chunks:
//   1. per-owner counts q_{u,k-1} by the counting kernels;
//   2. on the host, the owner queue is cut into consecutive runs whose counts
//      fit the caller's buffer, and each owner gets its offset in the run;
//   3. per run, one CTA per owner rebuilds G+(u) (upper bitmap rows), counts
//      the cliques under each first-level vertex x_i1, scans those counts and
//      writes every clique at its owner's offset plus its sub-tree's offset
//      -- a deterministic layout, so the warps of a CTA write without any
//      global atomics;
//   4. the run is handed to the caller's callback, then the buffer is reused.
// Inside a sub-tree one warp walks the ordered chains x_i1 < x_i2 < ... with
// its candidate sets in a per-warp stack (lanes over words) and writes the
// last level's elements by rank selection, 32 cliques at a time.
#include <algorithm>
#include <climits>
#include <vector>

#include "count_common.cuh"

namespace kc {

int num_sms();

namespace {

using cc::Ctx;

constexpr int kListWarps = 8;

// Lowest element of the W-word set S at or above word `low`, removed from S;
// -1 when none is left.  `low` advances to the word of the element.
__device__ int set_pop(uint32_t* S, int& low, int W, int lane)
{
    while (low < W) {
        const int w = low + lane;
        const uint32_t v = w < W ? S[w] : 0u;
        const uint32_t nz = __ballot_sync(kFull, v != 0u);
        if (nz) {
            const int f = __ffs(nz) - 1;
            const uint32_t vf = __shfl_sync(kFull, v, f);
            __syncwarp();
            if (lane == f) S[w] = vf & (vf - 1u);
            __syncwarp();
            low += f;
            return low * 32 + __ffs(vf) - 1;
        }
        low += 32;
    }
    return -1;
}

// Elements of S (words low..W-1) as the last clique member: counts them and,
// with WRITE, stores clique number pos + j for the j-th element.  Lanes
// 0..t-1 hold the ids of the chain's levels in `chid`.
template <bool WRITE>
__device__ uint64_t leaves(const uint32_t* S, int low, int W, const int32_t* sL, const int32_t* perm,
                           int32_t uid, int32_t e1id, int t, int32_t chid, int32_t* out, int kk, int64_t pos,
                           int64_t lim, int lane)
{
    uint64_t run = 0;
    for (int g0 = low; g0 < W; g0 += 32) {
        const int w = g0 + lane;
        const uint32_t v = w < W ? S[w] : 0u;
        const uint32_t pc = (uint32_t)__popc(v);
        uint32_t pre = pc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(kFull, pre, o);
            if (lane >= o) pre += x;
        }
        const uint32_t gt = __shfl_sync(kFull, pre, 31);
        if (WRITE) {
            const uint32_t excl = pre - pc;
            for (uint32_t b = 0; b < gt; b += 32) {
                const uint32_t j = b + (uint32_t)lane;
                int ww = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const uint32_t p = __shfl_sync(kFull, pre, ww + step - 1);
                    if (p <= j) ww += step;
                }
                const uint32_t vw = __shfl_sync(kFull, v, ww);
                const uint32_t ex = __shfl_sync(kFull, excl, ww);
                const int64_t row = pos + (int64_t)run + (int64_t)j;
                const bool ok = j < gt && row < lim;  // rows past the run's buffer are never written
                int32_t* o = out + row * kk;
                for (int c = 0; c < t; ++c) {
                    const int32_t id = __shfl_sync(kFull, chid, c);
                    if (ok) o[2 + c] = id;
                }
                if (ok) {
                    const int leaf = (g0 + ww) * 32 + (int)__fns(vw, 0, (int)(j - ex) + 1);
                    o[0] = uid;
                    o[1] = e1id;
                    o[kk - 1] = perm[sL[leaf]];
                }
            }
        }
        run += gt;
    }
    return run;
}

// Cliques of `need` more vertices inside the set in stk[0..W) (words from
// low0 on), each completed by the chain; stk holds `need` levels of W words.
template <bool WRITE>
__device__ uint64_t warp_enum(uint32_t* stk, int W, int need, int low0, const uint32_t* A, int RS,
                              const int32_t* sL, const int32_t* perm, int32_t uid, int32_t e1id, int32_t* out,
                              int kk, int64_t pos, int64_t lim, int lane)
{
    uint64_t total = 0;
    int t = 0, low = low0;
    int lowr = low0;
    int32_t chid = 0;
    for (;;) {
        uint32_t* S = stk + (int64_t)t * W;
        if (need - t == 1) {
            total += leaves<WRITE>(S, low, W, sL, perm, uid, e1id, t, chid, out, kk, pos + (int64_t)total, lim,
                                   lane);
            if (t == 0) break;
            --t;
            low = __shfl_sync(kFull, lowr, t);
            continue;
        }
        const int e = set_pop(S, low, W, lane);
        if (e < 0) {
            if (t == 0) break;
            --t;
            low = __shfl_sync(kFull, lowr, t);
            continue;
        }
        uint32_t* D = S + W;
        const int lc = e >> 5;  // upper rows: the child set lies above e
        const uint32_t* Ae = A + (int64_t)e * RS;
        int cnt = 0;
        for (int w = lc + lane; w < W; w += 32) {
            const uint32_t v = S[w] & Ae[w];
            D[w] = v;
            cnt += __popc(v);
        }
        cnt = (int)__reduce_add_sync(kFull, (unsigned)cnt);
        __syncwarp();
        if (cnt < need - t - 1) continue;
        if (lane == t) {
            lowr = low;
            chid = perm[sL[e]];
        }
        ++t;
        low = lc;
    }
    return total;
}

struct LLayout {
    int64_t L, cnt, A, stk, total;
};

__host__ __device__ inline LLayout make_llayout(int W, int RS, int NW, int levels)
{
    const int64_t D = 32LL * W;
    LLayout l;
    l.L = 0;
    l.cnt = D;                 // uint64 per first-level vertex
    l.A = l.cnt + 2 * D;
    l.stk = l.A + D * RS;
    l.total = l.stk + (int64_t)NW * levels * W;
    return l;
}

// One CTA per owner of the run: G+(u), per-x_i1 counts, their scan, writes.
template <bool HEAVY>
__global__ void __launch_bounds__(256) k_list(Ctx cb, int W, int levels, const unsigned long long* ooff,
                                              int32_t* out, int64_t lim, uint32_t* gscratch, int64_t tile_words)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, NW = blockDim.x >> 5;
    const int RS = HEAVY ? W : W + 1;
    const LLayout lay = make_llayout(W, RS, NW, levels);
    uint32_t* base = HEAVY ? gscratch + (int64_t)blockIdx.x * tile_words : smem;
    int32_t* sL = (int32_t*)(base + lay.L);
    unsigned long long* cnt1 = (unsigned long long*)(base + lay.cnt);
    uint32_t* A = base + lay.A;
    uint32_t* stk = base + lay.stk + (int64_t)wid * levels * W;
    __shared__ long long s_item;
    const int kk = cb.k, need = kk - 2;

    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(cb.cursor, 1ull);
        __syncthreads();
        const long long item = s_item;
        Ctx c;
        int32_t r;
        if (!cc::resolve(cb, (int64_t)item, c, r)) break;
        const int64_t b = c.offp[r];
        const int d = (int)(c.offp[r + 1] - b);
        const int32_t uid = c.perm[r];
        const int64_t o = (int64_t)ooff[item];
        for (int j = threadIdx.x; j < d; j += blockDim.x) sL[j] = c.adjp[b + j];
        for (int64_t j = threadIdx.x; j < (int64_t)d * RS; j += blockDim.x) A[j] = 0u;
        __syncthreads();
        cc::build_rows<false, false>(c, sL, nullptr, d, A, RS, wid, NW, lane);
        __syncthreads();

        // pass 1: cliques under each first-level vertex
        for (int e1 = wid; e1 < d; e1 += NW) {
            const int lo = e1 >> 5;
            int pc = 0;
            for (int w = lo + lane; w < W; w += 32) {
                const uint32_t v = A[(int64_t)e1 * RS + w];
                stk[w] = v;
                pc += __popc(v);
            }
            pc = (int)__reduce_add_sync(kFull, (unsigned)pc);
            __syncwarp();
            const unsigned long long n1 =
                pc < need ? 0ull
                          : warp_enum<false>(stk, W, need, lo, A, RS, sL, c.perm, uid, 0, out, kk, 0, 0, lane);
            if (lane == 0) cnt1[e1] = n1;
        }
        __syncthreads();
        if (wid == 0) {  // exclusive scan of cnt1 by warp 0
            unsigned long long carry = 0;
            for (int b0 = 0; b0 < d; b0 += 32) {
                const int j = b0 + lane;
                const unsigned long long v = j < d ? cnt1[j] : 0ull;
                unsigned long long incl = v;
#pragma unroll
                for (int s = 1; s < 32; s <<= 1) {
                    const unsigned long long x = __shfl_up_sync(kFull, incl, s);
                    if (lane >= s) incl += x;
                }
                if (j < d) cnt1[j] = carry + incl - v;
                carry += __shfl_sync(kFull, incl, 31);
            }
        }
        __syncthreads();

        // pass 2: write each sub-tree at its offset
        for (int e1 = wid; e1 < d; e1 += NW) {
            const int lo = e1 >> 5;
            int pc = 0;
            for (int w = lo + lane; w < W; w += 32) {
                const uint32_t v = A[(int64_t)e1 * RS + w];
                stk[w] = v;
                pc += __popc(v);
            }
            pc = (int)__reduce_add_sync(kFull, (unsigned)pc);
            __syncwarp();
            if (pc < need) continue;
            warp_enum<true>(stk, W, need, lo, A, RS, sL, c.perm, uid, c.perm[sL[e1]], out, kk,
                            o + (int64_t)cnt1[e1], lim, lane);
        }
        __syncthreads();
    }
}

// k = 1 (every vertex) and k = 2 (every edge u < x, x in Gamma+(u)).
__global__ void k_list_small(Ctx cb, const unsigned long long* ooff, int32_t* out, int64_t lim)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t item = warp; item < cb.nitems; item += nwarps) {
        Ctx c;
        int32_t r;
        if (!cc::resolve(cb, item, c, r)) break;
        const int64_t o = (int64_t)ooff[item];
        const int32_t uid = c.perm[r];
        if (cb.k == 1) {
            if (lane == 0 && o < lim) out[o] = uid;
            continue;
        }
        const int64_t b = c.offp[r];
        const int d = (int)(c.offp[r + 1] - b);
        for (int j = lane; j < d && o + j < lim; j += 32) {
            out[(o + j) * 2] = uid;
            out[(o + j) * 2 + 1] = c.perm[c.adjp[b + j]];
        }
    }
}

}  // namespace

kc_status list_run(const kc_graph* g, int k, unsigned flags, int32_t* buf, int64_t cap, kc_list_fn fn, void* user,
                   uint64_t* listed, cudaStream_t s)
{
    const bool dev = (flags & KC_DEVICE_PTRS) != 0;
    const int32_t n = g->n;
    *listed = 0;
    if (n == 0) return KC_OK;
    Scratch sc(s);
    unsigned long long* small = nullptr;  // [0..1] total, [2..15] cursors
    KC_TRY(sc.get(&small, 24));
    KC_CK(cudaMemsetAsync(small, 0, 24 * sizeof(unsigned long long), s));

    // queue (owners by d+ descending) and per-owner counts, on the host
    std::vector<int32_t> hq(n);
    KC_CK(cudaMemcpyAsync(hq.data(), g->queue, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    std::vector<unsigned long long> cnt(n, 0ull);  // rank space
    int64_t qend = n;
    if (k == 1) {
        std::fill(cnt.begin(), cnt.end(), 1ull);
    } else if (k == 2) {
        std::vector<int32_t> dp(n);
        KC_CK(cudaMemcpyAsync(dp.data(), g->dplus, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        KC_CK(cudaStreamSynchronize(s));
        for (int32_t r = 0; r < n; ++r) cnt[r] = (unsigned long long)dp[r];
        qend = ge_at(g, 1);
    } else {
        qend = ge_at(g, k - 1);
        unsigned long long* po = nullptr;
        KC_TRY(sc.get(&po, n));
        KC_CK(cudaMemsetAsync(po, 0, (size_t)n * sizeof(unsigned long long), s));
        Plan plan;
        const bool planned = find_plan(g, k, false, &plan);
        int64_t slot_words = 0;
        const int64_t hw = heavy_scratch_words(g, k, &slot_words, planned ? &plan : nullptr);
        uint32_t* heavy = nullptr;
        if (hw > 0) KC_TRY(sc.get(&heavy, hw));
        CountArgs a;
        a.plan = planned ? &plan : nullptr;
        a.k = k;
        a.colours = 0;
        a.seed = 0;
        a.per_vertex = false;
        a.total = small;
        a.pv = nullptr;
        a.po = po;
        a.work = nullptr;
        a.sc = &sc;
        KC_TRY(count_launch(g, a, small + 2, heavy, hw, s));
        KC_CK(cudaMemcpyAsync(cnt.data(), po, (size_t)n * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    }
    KC_CK(cudaStreamSynchronize(s));
    if (qend <= 0) return KC_OK;

    // device buffers for one run
    unsigned long long* doff = nullptr;
    KC_TRY(sc.get(&doff, qend));
    int32_t* dbuf = buf;
    if (!dev) KC_TRY(sc.get(&dbuf, cap * (int64_t)k));
    unsigned long long* cursors = small + 2;

    // widest-owner tiles for the listing kernel
    const int Wh = std::max(1, (g->max_dplus + 31) / 32);
    const int levels = std::max(1, k - 2);
    const LLayout hl = make_llayout(Wh, Wh, kListWarps, levels);
    const int64_t tile_words = (hl.total + 3) & ~3LL;  // keeps every tile 16-byte aligned
    int64_t h0 = 0, h1 = 0;
    class_range(g, k, 0, &h0, &h1);
    const int sms = num_sms();
    const int64_t htiles = k >= 3 ? std::min<int64_t>(std::max<int64_t>(h1 - h0, 0), sms) : 0;
    uint32_t* htile = nullptr;
    if (htiles > 0) KC_TRY(sc.get(&htile, tile_words * htiles));

    std::vector<unsigned long long> hoff;
    uint64_t delivered = 0;
    int64_t a0 = 0;
    while (a0 < qend) {
        unsigned long long T = 0;
        int64_t b0 = a0;
        while (b0 < qend) {
            const unsigned long long cu = cnt[hq[b0]];
            if (cu > (unsigned long long)cap) return KC_ENOMEM;  // one owner's cliques exceed the buffer
            if (T + cu > (unsigned long long)cap) break;
            T += cu;
            ++b0;
        }
        if (T == 0) {  // only owners without cliques remain in this run
            a0 = b0;
            continue;
        }
        hoff.assign((size_t)(b0 - a0), 0ull);
        unsigned long long acc = 0;
        for (int64_t i = a0; i < b0; ++i) {
            hoff[(size_t)(i - a0)] = acc;
            acc += cnt[hq[i]];
        }
        KC_CK(cudaMemcpyAsync(doff, hoff.data(), hoff.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice,
                              s));
        KC_CK(cudaMemsetAsync(cursors, 0, kCursorWords * sizeof(unsigned long long), s));
        Ctx base;
        base.offp = g->offp;
        base.adjp = g->adjp;
        base.queue = g->queue;
        base.perm = g->perm;
        base.qoff = 0;
        base.qstride = 1;
        base.gd = nullptr;
        base.gq0 = nullptr;
        base.gpre = nullptr;
        base.ng = 0;
        base.k = k;
        base.colours = 0;
        base.seed = 0;
        base.pair = 0;
        base.pthr = 0;
        base.total = small;
        base.pv = nullptr;
        base.po = nullptr;
        base.work = nullptr;
        if (k <= 2) {
            Ctx c = base;
            c.q0 = a0;
            c.q1 = b0;
            c.nitems = b0 - a0;
            c.cursor = cursors;
            const int grid = (int)std::min<int64_t>((c.nitems + 7) / 8, (int64_t)sms * 16);
            k_list_small<<<grid, 256, 0, s>>>(c, doff, dbuf, (int64_t)T);
            KC_LAUNCHED();
        } else {
            for (int slot = 0; slot < kOwnerSlots; ++slot) {
                int64_t q0 = 0, q1 = 0;
                class_range(g, k, slot, &q0, &q1);
                const int64_t lo = std::max(q0, a0), hi = std::min(q1, b0);
                if (hi <= lo) continue;
                Ctx c = base;
                c.q0 = lo;
                c.q1 = hi;
                c.nitems = hi - lo;
                c.cursor = cursors + slot;
                const unsigned long long* off = doff + (lo - a0);
                if (slot == 0) {
                    const int grid = (int)std::min<int64_t>(c.nitems, htiles);
                    k_list<true><<<grid, kListWarps * 32, 0, s>>>(c, Wh, levels, off, dbuf, (int64_t)T, htile,
                                                                   tile_words);
                    KC_LAUNCHED();
                    continue;
                }
                const int W = slot_words(slot);
                const int NW = W == 1 ? 1 : kListWarps;
                const LLayout l = make_llayout(W, W + 1, NW, levels);
                const size_t smem = (size_t)l.total * 4;
                auto kern = k_list<false>;
                KC_CK(cc::allow_smem(kern, smem));
                const int grid =
                    (int)std::min<int64_t>(c.nitems, (int64_t)sms * cc::blocks_per_sm(kern, NW * 32, smem));
                kern<<<grid, NW * 32, smem, s>>>(c, W, levels, off, dbuf, (int64_t)T, nullptr, 0);
                KC_LAUNCHED();
            }
        }
        if (!dev)
            KC_CK(cudaMemcpyAsync(buf, dbuf, (size_t)T * k * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        KC_CK(cudaStreamSynchronize(s));
        delivered += T;
        *listed = delivered;
        if (fn(user, buf, (int64_t)T) != 0) return KC_ECANCELED;
        a0 = b0;
    }
    return KC_OK;
}

}  // namespace kc
