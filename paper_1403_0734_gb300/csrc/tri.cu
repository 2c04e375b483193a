// tri.cu -- triangle path for exact k = 3 (no bitmaps).
//
// For k = 3 Reduce 3 has nothing to search: q_{u,2} is the number of edges
// of G+(u), i.e. the number of pairs x_i < y with y in Gamma+(x_i) and y in
// Gamma+(u) -- the node-iterator count of the paper's triangle baselines
// (Sec. 4, the one- and two-round triangle algorithms it compares with).
// These kernels count those matches directly, without building G+(u):
//   * owners with |Gamma+(u)| <= 32: one warp per owner, Gamma+(u) in
//     registers (lane j holds x_j), every entry y of a 32-entry chunk of
//     Gamma+(x_i) located by a shuffle binary search;
//   * wider owners: one CTA per owner, Gamma+(u) in shared memory, and when
//     its rank span max - min + 1 is at most 32 kSpanWords a direct-address
//     table over the span -- a bitmap with a per-word prefix count -- so
//     that membership and local index of y cost two independent shared loads
//     instead of a dependent binary search.
// Memberships (per-vertex output): u gains q_{u,2}; x_i gains its matches;
// every matched x_j gains one per match.  Counts match the bitmap path
// exactly (same owners, same pairs).
#include <algorithm>
#include <climits>

#include "count_common.cuh"

namespace kc {

int num_sms();

namespace {

using cc::add_total;
using cc::Ctx;
using cc::mask_below;

constexpr int kSpanWords = 1024;                // direct table: spans up to 32768 ranks
constexpr int kWarpItems = 4;                    // owners a warp takes per cursor step

// --------------------------------------------------------- d+ <= 32

template <bool PV>
__global__ void __launch_bounds__(256) k_tri_warp(Ctx cb)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long pos0 = 0;
        if (lane == 0) pos0 = atomicAdd(cb.cursor, (unsigned long long)kWarpItems);
        pos0 = __shfl_sync(kFull, pos0, 0);
        if ((int64_t)pos0 >= cb.nitems) break;
        for (int it = 0; it < kWarpItems; ++it) {
            Ctx c;
            int32_t r;
            if (!cc::resolve(cb, (int64_t)pos0 + it, c, r)) break;
            const int64_t b = c.offp[r];
            const int d = (int)(c.offp[r + 1] - b);
            const int32_t x = lane < d ? c.adjp[b + lane] : INT_MAX;
            // offsets of every Gamma+(x_j) at once
            const int64_t o0 = lane < d ? c.offp[x] : 0, o1 = lane < d ? c.offp[x + 1] : 0;
            const int32_t maxL = __shfl_sync(kFull, x, d - 1);
            uint32_t tot = 0, pvl = 0;
            for (int i = 0; i < d - 1; ++i) {
                const int64_t s0 = __shfl_sync(kFull, o0, i), s1 = __shfl_sync(kFull, o1, i);
                uint32_t cnt = 0;
                for (int64_t p0 = s0; p0 < s1; p0 += 32) {
                    const int64_t p = p0 + lane;
                    const int32_t y = p < s1 ? c.adjp[p] : INT_MAX;
                    int lo = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const int32_t xx = __shfl_sync(kFull, x, lo + step - 1);
                        if (xx < y) lo += step;
                    }
                    const int32_t xl = __shfl_sync(kFull, x, lo);
                    const bool hit = y <= maxL && xl == y;
                    cnt += (uint32_t)__popc(__ballot_sync(kFull, hit));
                    if (PV) pvl += (__reduce_or_sync(kFull, hit ? (1u << lo) : 0u) >> lane) & 1u;
                    if (__shfl_sync(kFull, y, 31) >= maxL) break;
                }
                tot += cnt;
                if (PV && lane == i) pvl += cnt;
            }
            if (lane == 0) {
                add_total(c.total, tot);
                if (c.po) c.po[r] = tot;
                if (PV && tot) atomicAdd(&c.pv[r], (unsigned long long)tot);
            }
            if (PV && lane < d && pvl) atomicAdd(&c.pv[x], (unsigned long long)pvl);
        }
    }
}

// ---------------------------------------------------------- d+ > 32

// Shared layout (32-bit words): sL[D] ranks, sCnt[D] memberships (PV), the
// span table's bitmap (kSpanWords) and 16-bit prefix counts (kSpanWords / 2).
template <bool PV>
__global__ void __launch_bounds__(256) k_tri_cta(Ctx cb, int D)
{
    extern __shared__ __align__(16) uint32_t smem[];
    int32_t* sL = (int32_t*)smem;
    uint32_t* sCnt = smem + D;
    uint32_t* sBits = sCnt + (PV ? D : 0);
    uint16_t* sPre = (uint16_t*)(sBits + kSpanWords);
    __shared__ unsigned long long s_tot;
    __shared__ long long s_item;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, NW = blockDim.x >> 5;

    for (;;) {
        if (threadIdx.x == 0) {
            s_item = (long long)atomicAdd(cb.cursor, 1ull);
            s_tot = 0ull;
        }
        __syncthreads();
        Ctx c;
        int32_t r;
        if (!cc::resolve(cb, (int64_t)s_item, c, r)) break;
        const int64_t b = c.offp[r];
        const int d = (int)(c.offp[r + 1] - b);
        for (int j = threadIdx.x; j < d; j += blockDim.x) {
            sL[j] = c.adjp[b + j];
            if (PV) sCnt[j] = 0u;
        }
        __syncthreads();
        const int32_t lo = sL[0], maxL = sL[d - 1];
        cc::SpanTable T{sBits, sPre, 0, 0};
        cc::span_table_build(T, sL, d, kSpanWords);
        const bool direct = T.words > 0;

        unsigned long long wtot = 0;
        for (int i = wid; i < d - 1; i += NW) {
            const int32_t xi = sL[i];
            const int64_t s0 = c.offp[xi], s1 = c.offp[xi + 1];
            uint32_t cnt = 0;
            for (int64_t p0 = s0; p0 < s1; p0 += 32) {
                const int64_t p = p0 + lane;
                const int32_t y = p < s1 ? c.adjp[p] : INT_MAX;
                bool hit = false;
                int j = 0;
                if (y <= maxL) {
                    if (direct) {
                        const int off = y - lo;
                        const uint32_t wv = sBits[off >> 5];
                        if ((wv >> (off & 31)) & 1u) {
                            hit = true;
                            j = (int)sPre[off >> 5] + __popc(wv & mask_below(off & 31));
                        }
                    } else {
                        int a = i + 1, z = d;
                        while (a < z) {
                            const int mid = (a + z) >> 1;
                            if (sL[mid] < y) a = mid + 1; else z = mid;
                        }
                        hit = a < d && sL[a] == y;
                        j = a;
                    }
                }
                cnt += (uint32_t)__popc(__ballot_sync(kFull, hit));
                if (PV && hit) atomicAdd(&sCnt[j], 1u);
                if (__shfl_sync(kFull, y, 31) >= maxL) break;
            }
            wtot += cnt;
            if (PV && lane == 0 && cnt) atomicAdd(&sCnt[i], cnt);
        }
        if (lane == 0 && wtot) atomicAdd(&s_tot, wtot);
        __syncthreads();
        const unsigned long long tot = s_tot;
        if (threadIdx.x == 0) {
            add_total(c.total, tot);
            if (c.po) c.po[r] = tot;
            if (PV && tot) atomicAdd(&c.pv[r], tot);
        }
        if (PV)
            for (int j = threadIdx.x; j < d; j += blockDim.x)
                if (sCnt[j]) atomicAdd(&c.pv[sL[j]], (unsigned long long)sCnt[j]);
        __syncthreads();
    }
}

}  // namespace

static int g_tri = 1;
int tri_enabled() { return g_tri; }
kc_status set_tri(int64_t v)
{
    if (v != 0 && v != 1) return KC_EINVAL;
    g_tri = (int)v;
    return KC_OK;
}

// Owner slot `slot` (0: d+ above the shared-memory classes, 1..5 classes of
// W words, 6: d+ <= 32) of an exact k = 3 count.
kc_status tri_launch_slot(int slot, int Wh, const cc::Ctx& c, bool pv, cudaStream_t s)
{
    if (c.nitems <= 0) return KC_OK;
    const int sms = num_sms();
    if (slot == kOwnerSlots - 1) {
        auto kern = pv ? k_tri_warp<true> : k_tri_warp<false>;
        const int64_t warps = (c.nitems + kWarpItems - 1) / kWarpItems;
        const int grid = (int)std::min<int64_t>((warps + 7) / 8, (int64_t)sms * cc::blocks_per_sm(kern, 256, 0));
        kern<<<grid, 256, 0, s>>>(c);
        KC_LAUNCHED();
        return KC_OK;
    }
    const int W = slot == 0 ? Wh : slot_words(slot);
    const int D = 32 * W;
    const size_t smem = (size_t)(D * (pv ? 2 : 1) + kSpanWords + kSpanWords / 2) * 4;
    auto kern = pv ? k_tri_cta<true> : k_tri_cta<false>;
    KC_CK(cc::allow_smem(kern, smem));
    const int grid = (int)std::min<int64_t>(c.nitems, (int64_t)sms * cc::blocks_per_sm(kern, 256, smem));
    kern<<<grid, 256, smem, s>>>(c, D);
    KC_LAUNCHED();
    return KC_OK;
}

}  // namespace kc
