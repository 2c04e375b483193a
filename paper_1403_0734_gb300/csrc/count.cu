// count.cu -- Rounds 2-3 of Algorithm 1 (Sec. 3) and the colour filter of
// cFFF_k (Sec. 6) on the device.
//
// For every owner u (rank r) with d = |Gamma+(u)| >= k-1:
//   (b) build G+(u) as a bitmap: local ids 0..d-1 are the positions of
//       Gamma+(u) in the order; bit j of row i is set iff x_j is in
//       Gamma+(x_i) -- exactly the pairs x_i < x_j that Map 2 emits and
//       Reduce 2 keeps because they are edges.  Each Gamma+(x_i) list is
//       streamed and its entries are searched in the sorted Gamma+(u); the
//       scan stops at max Gamma+(u).  With per-vertex counts the bitmap is
//       kept symmetric (bit i of row j too).
//   (d) cFFF_k: a pair is kept only if colour(u, x_i) == colour(u, x_j).
//   (c) count the (k-1)-cliques of G+(u) (Reduce 3) by a depth-first
//       search that ANDs rows: a chain i1 < i2 < ... with candidate set
//       C_t = C_{t-1} & row(i_t) restricted to ids above i_t.  The last two
//       levels are closed in one step: with C the candidates after k-3
//       choices, the cliques completed are the edges inside C,
//       sum_{e in C} popc(C & row_up(e)), and (per-vertex mode) vertex e of C
//       lies in popc(C & row(e)) of them -- no per-clique work.
//       Chain members and u are credited with the sub-tree totals.
// Owners come from the queue (|Gamma+| descending) in classes by bitmap
// width W = ceil(d/32): W = 1 runs one warp per owner with the rows in
// registers; W in {2..32} one CTA per owner with the rows in shared memory;
// wider owners use the same CTA code on a global-memory tile.
#include <algorithm>
#include <climits>
#include <cstring>
#include <functional>
#include <mutex>
#include <queue>

#include "count_common.cuh"

namespace kc {

int num_sms();

// Process-wide knob: widest bitmap row (in 32-bit words) kept in shared memory.
static int g_smem_max_words = kNumSmemClasses > 0 ? kClassWords[kNumSmemClasses - 1] : 1;

int smem_max_words() { return g_smem_max_words; }

// Process-wide choice of the Reduce 3 counter: the ordered depth-first search
// (default) or the pivoting clique tree.
static int g_algo = KC_ALGO_DFS;
int count_algo() { return g_algo; }
kc_status set_count_algo(int64_t v)
{
    if (v != KC_ALGO_PIVOT && v != KC_ALGO_DFS) return KC_EINVAL;
    g_algo = (int)v;
    return KC_OK;
}

int64_t sct_heavy_words_w(int W, int k, int64_t nheavy);
int parts_per_owner(int W, int k);
kc_status sct_launch_slot(int slot, int Wh, const cc::Ctx& c, bool pv, bool col, uint32_t* heavy,
                          int64_t heavy_words, cudaStream_t s);
bool dfs_reg_supported(int k);
kc_status tri_launch_slot(int slot, int Wh, const cc::Ctx& c, bool pv, cudaStream_t s);
kc_status dfs_reg_launch(const cc::Ctx& c, int W, bool pv, bool col, Scratch* sc, int parts, cudaStream_t s);
int64_t dfs_tile_words(int W, int k, int64_t items, int parts);
kc_status w2_launch(const cc::Ctx& c, bool pv, bool col, cudaStream_t s);

kc_status set_smem_max_words(int64_t v)
{
    // a class width: the queue is grouped by these classes, so every
    // shared-memory / global-tile split falls on a class boundary
    if (v < 1 || v > kClassWords[kNumSmemClasses - 1] || (v & (v - 1)) != 0) return KC_EINVAL;
    g_smem_max_words = (int)v;
    return KC_OK;
}

namespace {

using cc::Ctx;
using cc::add_total;
using cc::mask_above;
using cc::mask_below;
using cc::warp_sum64;

// ------------------------------------------------------------ W = 1 class

// Edges inside C (one word; lane l owns local vertex l).  pvl += degree of
// the lane's vertex inside C (per-vertex mode).
template <bool PV>
__device__ __forceinline__ unsigned long long leaf2_w1(uint32_t C, uint32_t up, uint32_t A, int lane,
                                                       unsigned long long& pvl)
{
    const bool in = (C >> lane) & 1u;
    const uint32_t e = in ? (uint32_t)__popc(C & up) : 0u;
    if (PV && in) pvl += (unsigned long long)__popc(C & A);
    return (unsigned long long)__reduce_add_sync(kFull, e);
}

template <bool PV, bool COL>
__global__ void __launch_bounds__(256) k_count_w1(Ctx cb)
{
    const int lane = threadIdx.x & 31;
    const int r0 = cb.k - 1;  // vertices to choose inside G+(u)
    for (;;) {
        unsigned long long pos = 0;
        if (lane == 0) pos = atomicAdd(cb.cursor, 1ull);
        pos = __shfl_sync(kFull, pos, 0);
        Ctx c;
        int32_t r;
        if (!cc::resolve(cb, (int64_t)pos, c, r)) break;
        const int64_t b = c.offp[r];
        const int d = (int)(c.offp[r + 1] - b);
        const int32_t x = lane < d ? c.adjp[b + lane] : INT_MAX;
        uint32_t col = 0;
        const int32_t ur = COL ? c.perm[r] : 0;
        if (COL && lane < d) col = cc::sample_label(c, ur, c.perm[x]);
        if (COL) col = cc::class_flag_w1(c, col, d, r0, lane);

        // (b) rows: lane j searches x_j in each 32-entry chunk of Gamma+(x_i)
        const uint32_t up = cc::build_rows_w1<COL>(c, x, d, col, ur, lane);
        const uint32_t A = PV ? (up | cc::lower_rows_w1(up, d, lane)) : up;

        // (c) depth-first search; level t's state of the chain is kept in lane t
        unsigned long long tot = 0, pvl = 0, wk = 0;
        const bool cw = c.work != nullptr;
        const uint32_t C1 = d >= 32 ? kFull : ((1u << d) - 1u);
        if (r0 == 2) {
            tot = leaf2_w1<PV>(C1, up, A, lane, pvl);
            if (cw) wk += (unsigned long long)__popc(C1) * (PV ? 2 : 1);
        } else {
            uint32_t st_rem = 0;
            int st_e = 0;
            unsigned long long st_sub = 0;
            int t = 0;
            uint32_t cur = C1;
            unsigned long long cur_sub = 0;
            for (;;) {
                if (cur == 0) {
                    if (t == 0) break;
                    const unsigned long long sdone = cur_sub;
                    --t;
                    cur = __shfl_sync(kFull, st_rem, t);
                    const int pe = __shfl_sync(kFull, st_e, t);
                    cur_sub = __shfl_sync(kFull, st_sub, t) + sdone;
                    if (PV && lane == pe) pvl += sdone;
                    continue;
                }
                const int e = __ffs(cur) - 1;
                cur &= cur - 1u;
                const uint32_t Cn = cur & __shfl_sync(kFull, up, e);
                const int need = r0 - t - 1;
                if (cw) wk += 1;
                if (__popc(Cn) < need) continue;
                if (need == 2) {
                    if (cw) wk += (unsigned long long)__popc(Cn) * (PV ? 2 : 1);
                    const unsigned long long E = leaf2_w1<PV>(Cn, up, A, lane, pvl);
                    tot += E;
                    cur_sub += E;
                    if (PV && lane == e) pvl += E;
                } else {
                    if (lane == t) {
                        st_rem = cur;
                        st_e = e;
                        st_sub = cur_sub;
                    }
                    ++t;
                    cur = Cn;
                    cur_sub = 0;
                }
            }
        }
        if (lane == 0) {
            add_total(c.total, tot);
            if (c.po) c.po[r] = tot;
            if (PV && tot) atomicAdd(&c.pv[r], tot);
            if (cw && wk) atomicAdd(c.work, wk);
        }
        if (PV && lane < d && pvl) atomicAdd(&c.pv[x], pvl);
    }
}

// ----------------------------------------------------- wide classes (CTA)

// Next element (ascending) of the word set `set` from word `low`; removes it.
__device__ __forceinline__ int warp_next(uint32_t* set, int& low, int W, int lane)
{
    while (low < W) {
        const int w = low + lane;
        const uint32_t v = w < W ? set[w] : 0u;
        const uint32_t nz = __ballot_sync(kFull, v != 0u);
        if (nz) {
            const int f = __ffs(nz) - 1;
            const uint32_t vf = __shfl_sync(kFull, v, f);
            const int e = (low + f) * 32 + __ffs(vf) - 1;
            __syncwarp();
            if (lane == 0) set[low + f] = vf & (vf - 1u);
            __syncwarp();
            low += f;
            return e;
        }
        low += 32;
    }
    return -1;
}

// out = a & b over words [low, W); returns the population count.
__device__ __forceinline__ int warp_and(const uint32_t* a, const uint32_t* b, uint32_t* out, int low, int W,
                                        int lane)
{
    int cnt = 0;
    for (int w = low + lane; w < W; w += 32) {
        const uint32_t v = a[w] & b[w];
        out[w] = v;
        cnt += __popc(v);
    }
    __syncwarp();
    return (int)__reduce_add_sync(kFull, (unsigned)cnt);
}

// Edges inside the word set C (words [low, W)); per-vertex mode adds each
// element's degree inside C to pv.
template <bool PV>
__device__ unsigned long long warp_leaf2(const uint32_t* C, int low, int W, const uint32_t* A, int RS,
                                         int32_t* el, unsigned long long* pv, int lane,
                                         unsigned long long* wk)
{
    int nel = 0, hiw = low;
    const uint32_t lt = mask_below(lane);
    for (int w0 = low; w0 < W; w0 += 32) {
        const int w = w0 + lane;
        const uint32_t v = w < W ? C[w] : 0u;
        uint32_t nz = __ballot_sync(kFull, v != 0u);
        while (nz) {
            const int f = __ffs(nz) - 1;
            nz &= nz - 1u;
            const uint32_t bits = __shfl_sync(kFull, v, f);
            if ((bits >> lane) & 1u) el[nel + __popc(bits & lt)] = (w0 + f) * 32 + lane;
            nel += __popc(bits);
            hiw = w0 + f + 1;
        }
    }
    __syncwarp();
    unsigned long long E = 0, wl = 0;
    for (int p = lane; p < nel; p += 32) {
        const int e = el[p];
        const int we = e >> 5, be = e & 31;
        const uint32_t* Ae = A + (int64_t)e * RS;
        uint32_t cnt = (uint32_t)__popc(C[we] & Ae[we] & mask_above(be));
        for (int w = we + 1; w < hiw; ++w) cnt += (uint32_t)__popc(C[w] & Ae[w]);
        E += cnt;
        if (wk) wl += (unsigned long long)(hiw - we) + (PV ? (unsigned long long)(we - low + 1) : 0ull);
        if (PV) {
            uint32_t lowc = (uint32_t)__popc(C[we] & Ae[we] & mask_below(be));
            for (int w = low; w < we; ++w) lowc += (uint32_t)__popc(C[w] & Ae[w]);
            if (cnt + lowc) atomicAdd(&pv[e], (unsigned long long)(cnt + lowc));
        }
    }
    __syncwarp();
    if (wk) *wk += warp_sum64(wl);
    return warp_sum64(E);
}

// Depth-first search below a chosen prefix.  stk level 0 holds the candidate
// set (elements above the prefix's last vertex, starting at word low0);
// need0 >= 3 vertices are still to be chosen.  Chain state of level t lives
// in lane t.  Returns the number of cliques completed in the sub-tree and
// credits chain members inside it.
template <bool PV>
__device__ unsigned long long warp_dfs(uint32_t* stk, int SW, int W, int low0, int need0, const uint32_t* A,
                                       int RS, int32_t* el, unsigned long long* pv, int lane,
                                       unsigned long long* wk)
{
    unsigned long long total = 0, cur_sub = 0, st_sub = 0;
    int t = 0, low = low0, st_low = 0, st_e = 0;
    for (;;) {
        const int e = warp_next(stk + (int64_t)t * SW, low, W, lane);
        if (e < 0) {
            if (t == 0) break;
            const unsigned long long sdone = cur_sub;
            --t;
            low = __shfl_sync(kFull, st_low, t);
            const int pe = __shfl_sync(kFull, st_e, t);
            cur_sub = __shfl_sync(kFull, st_sub, t) + sdone;
            if (PV && lane == 0 && sdone) atomicAdd(&pv[pe], sdone);
            continue;
        }
        const int need = need0 - t - 1;
        const int we = e >> 5;
        const int cnt = warp_and(stk + (int64_t)t * SW, A + (int64_t)e * RS, stk + (int64_t)(t + 1) * SW, we, W, lane);
        if (wk) *wk += (unsigned long long)(W - we);
        if (cnt < need) continue;
        if (need == 2) {
            const unsigned long long E = warp_leaf2<PV>(stk + (int64_t)(t + 1) * SW, we, W, A, RS, el, pv, lane, wk);
            total += E;
            cur_sub += E;
            if (PV && lane == 0 && E) atomicAdd(&pv[e], E);
        } else {
            if (lane == t) {
                st_low = low;
                st_e = e;
                st_sub = cur_sub;
            }
            ++t;
            low = we;
            cur_sub = 0;
        }
    }
    return total;
}

// Layout of the per-CTA working set (shared memory, or a global slot for the
// heavy class).  All sizes in 32-bit words.
struct Layout {
    int64_t L, col, pv, A, stk, el, total;
};

__host__ __device__ inline Layout make_layout(int W, int RS, int NW, int levels, bool pv, bool col)
{
    const int64_t D = 32LL * W;
    Layout l;
    l.L = 0;
    l.col = l.L + D;
    l.pv = l.col + (col ? D : 0);
    l.A = l.pv + (pv ? 2 * D : 0);
    l.stk = l.A + D * RS;
    l.el = l.stk + (int64_t)NW * levels * W;
    l.total = l.el + (int64_t)NW * D;
    return l;
}

template <bool PV, bool COL, bool HEAVY>
__global__ void __launch_bounds__(256) k_count_cta(Ctx cb, int W, int levels, uint32_t* gscratch,
                                                   int64_t slot_words)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, NW = blockDim.x >> 5;
    const int RS = HEAVY ? W : W + 1;
    const Layout lay = make_layout(W, RS, NW, levels, PV, COL);
    uint32_t* base = HEAVY ? gscratch + (int64_t)blockIdx.x * slot_words : smem;
    int32_t* sL = (int32_t*)(base + lay.L);
    uint32_t* sCol = base + lay.col;
    unsigned long long* sPV = (unsigned long long*)(base + lay.pv);
    uint32_t* sA = base + lay.A;
    uint32_t* stk = base + lay.stk + (int64_t)wid * levels * W;
    int32_t* el = (int32_t*)(base + lay.el) + (int64_t)wid * 32 * W;
    __shared__ int s_next;
    __shared__ unsigned long long s_tot;
    __shared__ long long s_item;

    const int r0 = cb.k - 1;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(cb.cursor, 1ull);
        __syncthreads();
        Ctx c;
        int32_t r;
        if (!cc::resolve(cb, (int64_t)s_item, c, r)) break;
        const int64_t b = c.offp[r];
        const int d = (int)(c.offp[r + 1] - b);
        const int32_t ur = COL ? c.perm[r] : 0;
        for (int j = threadIdx.x; j < d; j += blockDim.x) {
            const int32_t x = c.adjp[b + j];
            sL[j] = x;
            if (COL) sCol[j] = cc::sample_label(c, ur, c.perm[x]);
            if (PV) sPV[j] = 0ull;
        }
        for (int64_t j = threadIdx.x; j < (int64_t)d * RS; j += blockDim.x) sA[j] = 0u;
        if (threadIdx.x == 0) {
            s_next = 0;
            s_tot = 0ull;
        }
        __syncthreads();
        const int Wd = (d + 31) >> 5;  // words in use by this owner
        if (COL) cc::class_flags_smem<true>(c, sCol, d, r0, threadIdx.x, blockDim.x);

        // (b) + (d): rows, split over warps
        cc::build_rows<PV, COL>(c, sL, sCol, d, sA, RS, wid, NW, lane, ur);
        __syncthreads();

        // (c) count
        unsigned long long wtot = 0, wk = 0;
        unsigned long long* wkp = c.work ? &wk : nullptr;
        if (r0 == 2) {
            for (int e = wid; e < d; e += NW) {
                const uint32_t* Ae = sA + (int64_t)e * RS;
                const int we = e >> 5, be = e & 31;
                unsigned up = 0, all = 0;
                for (int w = we + lane; w < Wd; w += 32) {
                    const uint32_t v = Ae[w];
                    up += (unsigned)__popc(w == we ? (v & mask_above(be)) : v);
                }
                if (PV)
                    for (int w = lane; w < Wd; w += 32) all += (unsigned)__popc(Ae[w]);
                up = __reduce_add_sync(kFull, up);
                wtot += up;
                if (wkp) wk += (unsigned long long)(Wd - we) + (PV ? (unsigned long long)Wd : 0ull);
                if (PV) {
                    all = __reduce_add_sync(kFull, all);
                    if (lane == 0 && all) sPV[e] += all;
                }
            }
        } else {
            const int need0 = r0 - 1;
            for (;;) {
                int e1 = 0;
                if (lane == 0) e1 = atomicAdd(&s_next, 1);
                e1 = __shfl_sync(kFull, e1, 0);
                if (e1 >= d) break;
                const int we = e1 >> 5, be = e1 & 31;
                const uint32_t* Ae = sA + (int64_t)e1 * RS;
                int cnt = 0;
                for (int w = we + lane; w < Wd; w += 32) {
                    uint32_t v = Ae[w];
                    if (w == we) v &= mask_above(be);
                    stk[w] = v;
                    cnt += __popc(v);
                }
                __syncwarp();
                cnt = (int)__reduce_add_sync(kFull, (unsigned)cnt);
                if (wkp) wk += (unsigned long long)(Wd - we);
                if (cnt < need0) continue;
                const unsigned long long sub =
                    need0 == 2 ? warp_leaf2<PV>(stk, we, Wd, sA, RS, el, sPV, lane, wkp)
                               : warp_dfs<PV>(stk, W, Wd, we, need0, sA, RS, el, sPV, lane, wkp);
                wtot += sub;
                if (PV && lane == 0 && sub) atomicAdd(&sPV[e1], sub);
            }
        }
        if (lane == 0 && wtot) atomicAdd(&s_tot, wtot);
        if (lane == 0 && wk) atomicAdd(c.work, wk);
        __syncthreads();
        const unsigned long long tot = s_tot;
        if (threadIdx.x == 0) {
            add_total(c.total, tot);
            if (c.po) c.po[r] = tot;
            if (PV && tot) atomicAdd(&c.pv[r], tot);
        }
        if (PV)
            for (int j = threadIdx.x; j < d; j += blockDim.x) {
                const unsigned long long v = sPV[j];
                if (v) atomicAdd(&c.pv[sL[j]], v);
            }
        __syncthreads();
    }
}

int warps_for_width(int W)
{
    if (W <= 2) return 2;
    if (W <= 4) return 4;
    return 8;
}

// One owner class of the ordered DFS: slot 0 = global tiles (rows wider than
// the shared-memory limit), slots 1..5 = shared-memory rows of 32, 16, 8, 4, 2
// words, slot 6 = one word (registers).  Wh is the global-tile row width.
template <bool PV, bool COL>
kc_status launch_slot_dfs(int slot, int Wh, const Ctx& c, uint32_t* heavy, int64_t heavy_words, Scratch* sc,
                          int parts, cudaStream_t s)
{
    if (c.nitems <= 0) return KC_OK;
    const int sms = num_sms();
    const int k = c.k;
    const int levels = k > 3 ? k - 3 : 1;
    if (slot == 0) {
        const int NW = 8;
        const Layout lay = make_layout(Wh, Wh, NW, levels, PV, COL);
        const int64_t nslots = heavy_words / lay.total;
        if (nslots < 1) return KC_ENOMEM;
        const int grid = (int)std::min<int64_t>(std::min<int64_t>(nslots, c.nitems), sms);
        k_count_cta<PV, COL, true><<<grid, NW * 32, 0, s>>>(c, Wh, levels, heavy, lay.total);
        KC_LAUNCHED();
        return KC_OK;
    }
    if (slot == kOwnerSlots - 1) {
        auto kern = k_count_w1<PV, COL>;
        const int grid = (int)std::min<int64_t>((c.nitems + 7) / 8, (int64_t)sms * cc::blocks_per_sm(kern, 256, 0));
        kern<<<grid, 256, 0, s>>>(c);
        KC_LAUNCHED();
        return KC_OK;
    }
    const int W = slot_words(slot);
    if (W == 2 && parts <= 1 && !(PV && COL) && dfs_reg_supported(k))
        return w2_launch(c, PV, COL, s);  // a warp per owner, rows in registers
    if (dfs_reg_supported(k)) return dfs_reg_launch(c, W, PV, COL, sc, parts, s);  // register-resident search
    const int NW = warps_for_width(W);
    const Layout lay = make_layout(W, W + 1, NW, levels, PV, COL);
    const size_t smem = (size_t)lay.total * 4;
    auto kern = k_count_cta<PV, COL, false>;
    KC_CK(cc::allow_smem(kern, smem));
    const int grid = (int)std::min<int64_t>(c.nitems, (int64_t)sms * cc::blocks_per_sm(kern, NW * 32, smem));
    kern<<<grid, NW * 32, smem, s>>>(c, W, levels, nullptr, 0);
    KC_LAUNCHED();
    return KC_OK;
}

kc_status launch_slot(int slot, int Wh, const Ctx& c, bool pv, bool col, uint32_t* heavy, int64_t heavy_words,
                      Scratch* sc, const Plan* plan, cudaStream_t s)
{
    if (c.k == 3 && !col && tri_enabled()) return tri_launch_slot(slot, Wh, c, pv, s);  // no bitmaps for k = 3
    const int algo = plan ? plan->algo[slot] : count_algo();
    const int parts = plan ? plan->parts[slot] : 0;
    if (algo == KC_ALGO_PIVOT) return sct_launch_slot(slot, Wh, c, pv, col, heavy, heavy_words, s);
    if (pv) {
        if (col) return KC_ENOTSUP;
        return launch_slot_dfs<true, false>(slot, Wh, c, heavy, heavy_words, sc, parts, s);
    }
    if (col) return launch_slot_dfs<false, true>(slot, Wh, c, heavy, heavy_words, sc, parts, s);
    return launch_slot_dfs<false, false>(slot, Wh, c, heavy, heavy_words, sc, parts, s);
}

Ctx base_ctx(const CountArgs& a)
{
    Ctx c;
    c.offp = nullptr;
    c.adjp = nullptr;
    c.queue = nullptr;
    c.perm = nullptr;
    c.q0 = c.q1 = 0;
    c.nitems = 0;
    c.qoff = 0;
    c.qstride = 1;
    c.gd = nullptr;
    c.gq0 = nullptr;
    c.gpre = nullptr;
    c.ng = 0;
    c.k = a.k;
    c.colours = a.colours;
    c.seed = a.seed;
    c.pair = a.pair ? 1 : 0;
    c.pthr = a.pthr;
    c.total = a.total;
    c.pv = a.pv;
    c.po = a.po;
    c.cursor = nullptr;
    c.work = a.work;
    return c;
}

}  // namespace

int slot_words(int slot)
{
    if (slot <= 0 || slot >= kOwnerSlots) return slot == kOwnerSlots - 1 ? 1 : 0;
    return kClassWords[kNumSmemClasses - slot];
}

void class_range(const kc_graph* g, int k, int slot, int64_t* q0, int64_t* q1)
{
    auto ge_at = [&](int64_t t) -> int64_t { return kc::ge_at(g, t); };
    const int64_t dmin = k - 1;  // Reduce 1 filter
    const int maxw = smem_max_words();
    *q0 = *q1 = 0;
    if (slot == 0) {
        *q1 = ge_at(std::max<int64_t>(32LL * maxw + 1, dmin));
    } else if (slot == kOwnerSlots - 1) {
        *q0 = ge_at(33);
        *q1 = ge_at(std::max<int64_t>(1, dmin));
    } else {
        const int cl = kNumSmemClasses - slot;  // index into kClassWords
        const int W = kClassWords[cl];
        if (W > maxw) return;
        const int64_t dlo = 32LL * kClassWords[cl - 1] + 1, dhi = 32LL * W;
        *q0 = ge_at(dhi + 1);
        *q1 = ge_at(std::max(dlo, dmin));
    }
    if (*q1 < *q0) *q1 = *q0;
}

int64_t heavy_scratch_words_w(int W, int k, int64_t nheavy, int64_t* slot_words, int algo)
{
    *slot_words = 0;
    if (nheavy <= 0) return 0;
    if ((algo < 0 ? count_algo() : algo) == KC_ALGO_PIVOT) {
        *slot_words = sct_heavy_words_w(W, k, 1);
        return sct_heavy_words_w(W, k, nheavy);
    }
    const int levels = k > 3 ? k - 3 : 1;
    const Layout lay = make_layout(W, W, 8, levels, true, true);
    const int64_t slots = std::min<int64_t>(nheavy, num_sms());
    *slot_words = lay.total;
    return lay.total * slots;
}

int64_t split_scratch_words(const kc_graph* g, int k, const Plan* plan)
{
    if (!dfs_reg_supported(k)) return 0;
    int64_t words = 0;
    for (int slot = 1; slot < kOwnerSlots - 1; ++slot) {
        if ((plan ? plan->algo[slot] : count_algo()) != KC_ALGO_DFS) continue;
        int64_t q0 = 0, q1 = 0;
        class_range(g, k, slot, &q0, &q1);
        words += dfs_tile_words(slot_words(slot), k, q1 - q0, plan ? plan->parts[slot] : 0);
    }
    return words;
}

int64_t heavy_scratch_words(const kc_graph* g, int k, int64_t* slot_words, const Plan* plan)
{
    int64_t q0 = 0, q1 = 0;
    class_range(g, k, 0, &q0, &q1);
    return heavy_scratch_words_w((g->max_dplus + 31) / 32, k, q1 - q0, slot_words, plan ? plan->algo[0] : -1);
}

bool find_plan(const kc_graph* g, int k, bool pv, Plan* out)
{
    for (const kc_tuning& t : g->tunings)
        if (t.k == k && (t.per_vertex != 0) == pv) {
            for (int i = 0; i < kOwnerSlots; ++i) {
                out->algo[i] = t.algo[i];
                out->parts[i] = t.parts[i];
            }
            return true;
        }
    return false;
}

kc_status count_launch(const kc_graph* g, const CountArgs& a, unsigned long long* cursors,
                       uint32_t* heavy_scratch, int64_t heavy_words, cudaStream_t s)
{
    Ctx base = base_ctx(a);
    base.offp = g->offp;
    base.adjp = g->adjp;
    base.queue = g->queue;
    base.perm = g->perm;
    const kc_graph::Parts* parts = nullptr;
    if (a.nparts > 1) KC_TRY(graph_parts(g, a.nparts, s, &parts));
    const bool col = a.colours >= 2 || a.pair;  // one colour keeps every pair
    const int Wh = (g->max_dplus + 31) / 32;
    for (int slot = 0; slot < kOwnerSlots; ++slot) {
        Ctx c = base;
        class_range(g, a.k, slot, &c.q0, &c.q1);
        if (parts) {  // this part's owners of the class: a contiguous run of its own queue
            const std::vector<int64_t>& pos = parts->pos[(size_t)a.part];
            const int64_t p0 = std::lower_bound(pos.begin(), pos.end(), c.q0) - pos.begin();
            const int64_t p1 = std::lower_bound(pos.begin(), pos.end(), c.q1) - pos.begin();
            c.queue = parts->queue + parts->off[(size_t)a.part];
            c.q0 = p0;
            c.q1 = p1;
        }
        c.nitems = c.q1 - c.q0;
        c.cursor = cursors + slot;
        KC_TRY(launch_slot(slot, Wh, c, a.per_vertex, col, heavy_scratch, heavy_words, a.sc, a.plan, s));
    }
    return KC_OK;
}

namespace {

// w[r] = sum over x in Gamma+(r) of |Gamma+(x)| for every owner r.
__global__ void k_work_estimate(const int64_t* __restrict__ offp, const int32_t* __restrict__ adjp,
                                const int32_t* __restrict__ dplus, int32_t n, unsigned long long* __restrict__ w)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < n; r += nwarps) {
        unsigned long long acc = 0;
        for (int64_t p = offp[r] + lane; p < offp[r + 1]; p += 32) acc += (unsigned long long)dplus[adjp[p]];
        acc = cc::warp_sum64(acc);
        if (lane == 0) w[r] = acc;
    }
}

// sum over owners with d+ >= dmin of 4 w(u) + 20 d+(u) (Round 2 input bytes)
__global__ void k_round2_bytes(const int64_t* __restrict__ offp, const int32_t* __restrict__ adjp,
                               const int32_t* __restrict__ dplus, int32_t n, int dmin,
                               unsigned long long* __restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long acc = 0;
    for (int64_t r = warp; r < n; r += nwarps) {
        const int64_t b = offp[r], e = offp[r + 1];
        if (e - b < dmin) continue;
        for (int64_t p = b + lane; p < e; p += 32) acc += 4ull * (unsigned long long)dplus[adjp[p]] + 20ull;
    }
    acc = cc::warp_sum64(acc);
    if (lane == 0 && acc) atomicAdd(out, acc);
}

}  // namespace

kc_status round2_bytes(const kc_graph* g, int k, uint64_t* bytes, cudaStream_t s)
{
    *bytes = 0;
    if (g->n <= 0 || k < 3) return KC_OK;
    Scratch sc(s);
    unsigned long long* d = nullptr;
    KC_TRY(sc.get(&d, 1));
    KC_CK(cudaMemsetAsync(d, 0, sizeof(unsigned long long), s));
    k_round2_bytes<<<std::min<int64_t>(((int64_t)g->n + 7) / 8, (int64_t)num_sms() * 16), 256, 0, s>>>(
        g->offp, g->adjp, g->dplus, g->n, k - 1, d);
    KC_LAUNCHED();
    unsigned long long h = 0;
    KC_CK(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
    KC_CK(cudaStreamSynchronize(s));
    *bytes = h;
    return KC_OK;
}

// Greedy LPT: owners taken by work estimate w(u) descending (ties by queue
// position), each given to the part with the least work so far (ties: the
// lowest part), so the parts' sums of w(u) differ by at most one owner's.
kc_status graph_parts(const kc_graph* g, int nparts, cudaStream_t s, const kc_graph::Parts** out)
{
    std::lock_guard<std::mutex> lock(g->mu);
    for (const kc_graph::Parts& p : g->parts)
        if (p.nparts == nparts) {
            *out = &p;
            return KC_OK;
        }
    const int32_t n = g->n;
    std::vector<unsigned long long> w((size_t)std::max(n, 1));
    std::vector<int32_t> q((size_t)std::max(n, 1));
    if (n > 0) {
        Scratch sc(s);
        unsigned long long* dw = nullptr;
        KC_TRY(sc.get(&dw, n));
        k_work_estimate<<<std::min<int64_t>(((int64_t)n + 7) / 8, (int64_t)num_sms() * 16), 256, 0, s>>>(
            g->offp, g->adjp, g->dplus, n, dw);
        KC_LAUNCHED();
        KC_CK(cudaMemcpyAsync(w.data(), dw, (size_t)n * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        KC_CK(cudaMemcpyAsync(q.data(), g->queue, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        KC_CK(cudaStreamSynchronize(s));
    }
    // positions in queue order; their estimates
    std::vector<int64_t> order((size_t)n);
    for (int64_t i = 0; i < n; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
        return w[(size_t)q[(size_t)x]] > w[(size_t)q[(size_t)y]];
    });
    kc_graph::Parts P;
    P.nparts = nparts;
    P.pos.assign((size_t)nparts, {});
    // min-heap of (load, part): the least loaded part, the lowest on ties
    std::priority_queue<std::pair<unsigned long long, int>, std::vector<std::pair<unsigned long long, int>>,
                        std::greater<std::pair<unsigned long long, int>>>
        heap;
    for (int p = 0; p < nparts; ++p) heap.push({0ull, p});
    for (int64_t i : order) {
        auto [load, best] = heap.top();
        heap.pop();
        P.pos[(size_t)best].push_back(i);
        heap.push({load + w[(size_t)q[(size_t)i]] + 1, best});
    }
    std::vector<int32_t> hq;
    hq.reserve((size_t)n);
    P.off.assign((size_t)nparts, 0);
    for (int p = 0; p < nparts; ++p) {
        std::sort(P.pos[(size_t)p].begin(), P.pos[(size_t)p].end());
        P.off[(size_t)p] = (int64_t)hq.size();
        for (int64_t i : P.pos[(size_t)p]) hq.push_back(q[(size_t)i]);
    }
    void* dq = nullptr;
    KC_TRY(pool_alloc(&dq, std::max<size_t>(hq.size(), 1) * sizeof(int32_t), s));
    if (!hq.empty()) KC_CK(cudaMemcpyAsync(dq, hq.data(), hq.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    KC_CK(cudaStreamSynchronize(s));
    P.queue = (int32_t*)dq;
    g->parts.push_back(std::move(P));
    *out = &g->parts.back();
    return KC_OK;
}

void batch_tables(const kc_graph* const* gs, int ng, int k, std::vector<int64_t>& host_tables)
{
    // per slot: gq0[ng] then gpre[ng + 1]
    const int64_t per = 2LL * ng + 1;
    host_tables.assign((size_t)(per * kOwnerSlots), 0);
    for (int slot = 0; slot < kOwnerSlots; ++slot) {
        int64_t* hq0 = host_tables.data() + slot * per;
        int64_t* hpre = hq0 + ng;
        hpre[0] = 0;
        for (int g = 0; g < ng; ++g) {
            int64_t q0 = 0, q1 = 0;
            class_range(gs[g], k, slot, &q0, &q1);
            hq0[g] = q0;
            hpre[g + 1] = hpre[g] + (q1 - q0);
        }
    }
}

kc_status count_batch_run(const kc_graph* const* gs, int ng, const CountArgs& a, const void* descs,
                          const int64_t* tables, const std::vector<int64_t>& host_tables, unsigned long long* cursors,
                          uint32_t* heavy_scratch, int64_t heavy_words, cudaStream_t s)
{
    Ctx base = base_ctx(a);
    base.gd = (const cc::GraphDesc*)descs;
    base.ng = ng;
    const bool col = a.colours >= 2 || a.pair;
    int Wh = 1;
    for (int g = 0; g < ng; ++g) Wh = std::max(Wh, (gs[g]->max_dplus + 31) / 32);
    const int64_t per = 2LL * ng + 1;
    for (int slot = 0; slot < kOwnerSlots; ++slot) {
        Ctx c = base;
        c.gq0 = tables + slot * per;
        c.gpre = c.gq0 + ng;
        c.nitems = host_tables[(size_t)(slot * per + ng + ng)];
        c.cursor = cursors + slot;
        KC_TRY(launch_slot(slot, Wh, c, false, col, heavy_scratch, heavy_words, a.sc, a.plan, s));
    }
    return KC_OK;
}

kc_status count_batch_launch(const kc_graph* const* gs, int ng, const CountArgs& a, const void* descs,
                             int64_t* tables, unsigned long long* cursors, uint32_t* heavy_scratch,
                             int64_t heavy_words, std::vector<int64_t>& host_tables, cudaStream_t s)
{
    batch_tables(gs, ng, a.k, host_tables);
    KC_CK(cudaMemcpyAsync(tables, host_tables.data(), host_tables.size() * sizeof(int64_t),
                          cudaMemcpyHostToDevice, s));
    return count_batch_run(gs, ng, a, descs, tables, host_tables, cursors, heavy_scratch, heavy_words, s);
}

// ---------------------------------------------------------------- autotuner

// For every owner class of the graphs gs: run each candidate plan on the
// class's first owners (queue order: the heaviest of one graph, or the first
// graphs' owners of a batch), at most kTuneSample of them, once to warm up
// and once timed with events on s, and keep the fastest.  The outputs of the
// sample runs go to scratch and are discarded.
kc_status tune(const kc_graph* const* gs, int ng, int k, bool pv, cudaStream_t s, kc_tuning* out)
{
    constexpr int64_t kTuneSample = 256;
    std::memset(out, 0, sizeof(*out));
    out->k = k;
    out->per_vertex = pv ? 1 : 0;
    for (int i = 0; i < kOwnerSlots; ++i) {
        out->algo[i] = KC_ALGO_DFS;
        out->parts[i] = (i >= 1 && i < kOwnerSlots - 1) ? parts_per_owner(slot_words(i), k) : 1;
    }
    if (k <= 3 || ng < 1) return KC_OK;
    if (pv && ng > 1) return KC_EINVAL;  // per-vertex output exists for single graphs only
    Scratch sc(s);
    int32_t nmax = 1;
    int Wh = 1;
    int64_t nheavy = 0;
    for (int i = 0; i < ng; ++i) {
        nmax = std::max(nmax, gs[i]->n);
        Wh = std::max(Wh, (gs[i]->max_dplus + 31) / 32);
        int64_t q0 = 0, q1 = 0;
        class_range(gs[i], k, 0, &q0, &q1);
        nheavy += q1 - q0;
    }
    unsigned long long* small = nullptr;  // [0..1] total, [2..15] cursors, then 2 words per graph
    KC_TRY(sc.get(&small, 24 + 2 * (int64_t)ng));
    unsigned long long *pvr = nullptr, *por = nullptr;
    if (pv) {
        KC_TRY(sc.get(&pvr, nmax));
        KC_TRY(sc.get(&por, nmax));
    }
    int64_t sw = 0;
    const int64_t hs = std::min<int64_t>(nheavy, kTuneSample);
    const int64_t hw = std::max(heavy_scratch_words_w(Wh, k, hs, &sw, KC_ALGO_DFS),
                                heavy_scratch_words_w(Wh, k, hs, &sw, KC_ALGO_PIVOT));
    uint32_t* heavy = nullptr;
    if (hw > 0) KC_TRY(sc.get(&heavy, hw));

    CountArgs a;
    a.k = k;
    a.colours = 0;
    a.seed = 0;
    a.per_vertex = pv;
    a.total = small;
    a.pv = pvr;
    a.po = por;
    a.work = nullptr;
    Ctx base = base_ctx(a);
    std::vector<int64_t> host_tables;
    int64_t* tables = nullptr;
    cc::GraphDesc* dd = nullptr;
    const int64_t per = 2LL * ng + 1;
    if (ng == 1) {
        base.offp = gs[0]->offp;
        base.adjp = gs[0]->adjp;
        base.queue = gs[0]->queue;
        base.perm = gs[0]->perm;
    } else {
        std::vector<cc::GraphDesc> hd((size_t)ng);
        for (int i = 0; i < ng; ++i) hd[(size_t)i] = {gs[i]->offp, gs[i]->adjp, gs[i]->queue, gs[i]->perm};
        host_tables.assign((size_t)(per * kOwnerSlots), 0);
        for (int slot = 0; slot < kOwnerSlots; ++slot) {
            int64_t* hq0 = host_tables.data() + slot * per;
            int64_t* hpre = hq0 + ng;
            for (int i = 0; i < ng; ++i) {
                int64_t q0 = 0, q1 = 0;
                class_range(gs[i], k, slot, &q0, &q1);
                hq0[i] = q0;
                hpre[i + 1] = hpre[i] + (q1 - q0);
            }
        }
        KC_TRY(sc.get(&dd, ng));
        KC_TRY(sc.get(&tables, (int64_t)host_tables.size()));
        KC_CK(cudaMemcpyAsync(dd, hd.data(), hd.size() * sizeof(cc::GraphDesc), cudaMemcpyHostToDevice, s));
        KC_CK(cudaMemcpyAsync(tables, host_tables.data(), host_tables.size() * sizeof(int64_t),
                              cudaMemcpyHostToDevice, s));
        KC_CK(cudaStreamSynchronize(s));
        base.gd = dd;
        base.ng = ng;
        base.total = small + 16;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    KC_CK(cudaEventCreate(&e0));
    KC_CK(cudaEventCreate(&e1));
    struct Ev {
        cudaEvent_t a, b;
        ~Ev()
        {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } ev{e0, e1};

    for (int slot = 0; slot < kOwnerSlots; ++slot) {
        Ctx c = base;
        int64_t nitems = 0;
        if (ng == 1) {
            class_range(gs[0], k, slot, &c.q0, &c.q1);
            nitems = c.q1 - c.q0;
        } else {
            c.gq0 = tables + slot * per;
            c.gpre = c.gq0 + ng;
            nitems = host_tables[(size_t)(slot * per + ng + ng)];
        }
        if (nitems <= 0) continue;
        c.nitems = std::min(nitems, kTuneSample);
        c.cursor = small + 2 + slot;  // slot's cursor and (+ kOwnerSlots) its search cursor
        const int W = slot_words(slot);
        std::vector<std::pair<int, int>> cand;  // (algo, parts)
        cand.push_back({KC_ALGO_DFS, 1});
        if (slot >= 1 && slot < kOwnerSlots - 1 && W >= 4 && k >= 5 && dfs_reg_supported(k)) {
            cand.push_back({KC_ALGO_DFS, 4});
            cand.push_back({KC_ALGO_DFS, 16});
        }
        cand.push_back({KC_ALGO_PIVOT, 1});
        float best = -1.0f;
        for (const auto& cd : cand) {
            Plan pl;
            for (int i = 0; i < kOwnerSlots; ++i) {
                pl.algo[i] = cd.first;
                pl.parts[i] = cd.second;
            }
            float ms = 0.0f;
            for (int rep = 0; rep < 2; ++rep) {
                KC_CK(cudaMemsetAsync(small, 0, (24 + 2 * (size_t)ng) * sizeof(unsigned long long), s));
                KC_CK(cudaEventRecord(e0, s));
                KC_TRY(launch_slot(slot, Wh, c, pv, false, heavy, hw, &sc, &pl, s));
                KC_CK(cudaEventRecord(e1, s));
                KC_CK(cudaEventSynchronize(e1));
                KC_CK(cudaEventElapsedTime(&ms, e0, e1));
            }
            if (best < 0.0f || ms < best) {
                best = ms;
                out->algo[slot] = cd.first;
                out->parts[slot] = cd.second;
                out->ms[slot] = ms;
            }
        }
    }
    return KC_OK;
}

}  // namespace kc
