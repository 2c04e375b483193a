// dfs.cu -- ordered depth-first counter (Reduce 3, Alg. 1; Sec. 3) for owners
// whose G+(u) bitmap fits in shared memory (|Gamma+(u)| <= 1024), k <= 8.
//
// Same search as the generic kernel in count.cu -- chains x_i1 < x_i2 < ...
// of G+(u) with candidate sets C_t = C_{t-1} & row(i_t), the last two levels
// closed by population counts -- laid out for instruction efficiency:
//   * a candidate set lives in registers, lane w holding its word w, so an
//     intersection is one shared load and one AND per lane, and the stack of
//     the search (at most k-3 levels) is a register array;
//   * the last level picks its elements by rank (a warp prefix scan of word
//     population counts, a shuffle binary search and __fns), so no list of
//     elements is written to shared memory;
//   * the per-element word loop is uniform across the warp: every lane reads
//     the same candidate word by a broadcast shuffle and its own row word;
//   * memberships accumulate in 32-bit shared counters with a carry word;
//   * once a candidate set has at most 64 elements and at least three more
//     vertices are to be chosen, its induced subgraph is compressed into
//     64-bit rows (one ballot per row; lane j holds the rows of elements j
//     and j+32) and the rest of that sub-tree runs on registers only.
// Work items are (owner u, part c) with c < R: the item's CTA builds G+(u)
// in shared memory (its warps together), then its warps take the first-level
// vertices i1 = c, c+R, c+2R, ... from a shared counter.  R > 1 splits a heavy
// owner's count across CTAs by first-level vertex -- the postponed,
// neighbour-keyed counting of heavy G+(u) proposed in Sec. 7 -- so that the
// largest owners do not leave the rest of the GPU idle at the end.
#include <algorithm>
#include <type_traits>

#include "count_common.cuh"

namespace kc {

int num_sms();

namespace {

using cc::add_total;
using cc::Ctx;
using cc::mask_above;
using cc::mask_below;
using cc::warp_sum64;

constexpr int kMaxLev = 5;  // register stack levels: k - 3 <= 5, i.e. k <= 8

}  // namespace

// Size window [lo, hi] (hi <= 64) of candidate sets that switch to the compact
// sub-tree; hi = 0 turns the compact mode off.
static int g_compact_lo = 1, g_compact_hi = 64;
int compact_lo() { return g_compact_lo; }
int compact_hi() { return g_compact_hi; }
kc_status set_compact_window(int64_t lo, int64_t hi)
{
    if (lo < 1 || hi < 0 || hi > 64) return KC_EINVAL;
    g_compact_lo = (int)lo;
    g_compact_hi = (int)hi;
    return KC_OK;
}

static int g_complement = 1;

int complement_enabled() { return g_complement; }
kc_status set_complement(int64_t v)
{
    if (v != 0 && v != 1) return KC_EINVAL;
    g_complement = (int)v;
    return KC_OK;
}

namespace {

struct RLayout {
    int64_t L, col, pvlo, pvhi, A, sbits, spre, total;
};

constexpr int kSpanWords = 1024;  // direct table of the build: spans up to 32768 ranks
constexpr int kPairChunk = 4;     // (e1, e2) tasks taken per counter update

__host__ __device__ inline RLayout make_rlayout(int W, int RS, bool pv, bool col, int NW = 0)
{
    const int64_t D = 32LL * W;
    RLayout l;
    l.L = 0;
    l.col = l.L + D;
    l.pvlo = l.col + (col ? D : 0);
    l.pvhi = l.pvlo + (pv ? D : 0);
    l.A = l.pvhi + (pv ? D : 0);
    l.sbits = l.A + D * RS;
    l.spre = l.sbits + kSpanWords;
    l.total = l.spre + kSpanWords / 2;
    (void)NW;
    return l;
}

// Row stride: W + 1 words (odd, conflict-free) for the generic path; a
// multiple of 4 words (W + 4) for the 128-bit loads of the width-templated
// path, which also staggers rows across banks.
__host__ __device__ inline int row_stride(int W, int WM) { return WM >= 4 ? W + 4 : (WM > 0 ? 4 : W + 1); }

// 64-bit membership increment as 32-bit shared atomics with a carry word.
__device__ __forceinline__ void pv_add(uint32_t* lo, uint32_t* hi, int e, unsigned long long v)
{
    const uint32_t v0 = (uint32_t)v, v1 = (uint32_t)(v >> 32);
    if (v0) {
        const uint32_t old = atomicAdd(&lo[e], v0);
        if (old + v0 < old) atomicAdd(&hi[e], 1u);
    }
    if (v1) atomicAdd(&hi[e], v1);
}

__device__ __forceinline__ uint32_t st_get(const uint32_t (&st)[kMaxLev], int t)
{
    uint32_t v = st[0];
#pragma unroll
    for (int i = 1; i < kMaxLev; ++i)
        if (t == i) v = st[i];
    return v;
}

__device__ __forceinline__ void st_set(uint32_t (&st)[kMaxLev], int t, uint32_t v)
{
#pragma unroll
    for (int i = 0; i < kMaxLev; ++i)
        if (t == i) st[i] = v;
}

// Edges inside C (lane w holds word w; words below w0 and from Wd on are 0).
// Every element e of C takes one lane and sums popc(C & row(e)) over the
// words: with upper-triangular rows that is the number of higher neighbours
// of e in C, and the sum over e is the edge count; with symmetric rows
// (per-vertex mode) it is e's degree inside C -- its membership increment --
// and the edge count is half the sum.
template <bool PV>
__device__ __forceinline__ uint32_t leaf2_reg(uint32_t C, int w0, int Wd, const uint32_t* A, int RS,
                                              uint32_t* pvlo, uint32_t* pvhi, int lane,
                                              unsigned long long* wk)
{
    const uint32_t pc = (uint32_t)__popc(C);
    uint32_t pre = pc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, pre, o);
        if (lane >= o) pre += t;
    }
    const uint32_t total = __shfl_sync(kFull, pre, 31);
    const uint32_t excl = pre - pc;
    uint32_t S = 0;
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t j = base + (uint32_t)lane;
        // word of the j-th element: first lane whose inclusive count exceeds j
        int w = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t pv_ = __shfl_sync(kFull, pre, w + step - 1);
            if (pv_ <= j) w += step;
        }
        const uint32_t cw = __shfl_sync(kFull, C, w);
        const uint32_t ex = __shfl_sync(kFull, excl, w);
        const bool valid = j < total;
        const int e = w * 32 + (valid ? (int)__fns(cw, 0, (int)(j - ex) + 1) : 0);
        const uint32_t* Ae = A + (int64_t)(valid ? e : 0) * RS;
        // upper rows hold nothing below the first element's word of the pass
        const int xs = PV ? w0 : __shfl_sync(kFull, w, 0);
        uint32_t f = 0;
#pragma unroll 4
        for (int x = xs; x < Wd; ++x) f += (uint32_t)__popc(__shfl_sync(kFull, C, x) & (valid ? Ae[x] : 0u));
        if (valid) {
            S += f;
            if (PV && f) pv_add(pvlo, pvhi, e, f);
        }
        if (wk) *wk += (unsigned long long)__reduce_add_sync(kFull, valid ? (unsigned)(Wd - xs) : 0u);
    }
    const uint32_t E = __reduce_add_sync(kFull, S);
    return PV ? E / 2u : E;
}

// Same count as leaf2_reg, for rows of at most WM words: the candidate set
// is first copied into every lane's registers (WM broadcast shuffles), so
// each lane runs through its element's whole row alone with 128-bit shared
// loads and no shuffle in the loop.  Row stride RS is a multiple of 4 words.
template <bool PV, int WM>
__device__ __forceinline__ uint32_t leaf2_rep(uint32_t C, int Wd, const uint32_t* A, int RS, uint32_t* pvlo,
                                              uint32_t* pvhi, int lane, unsigned long long* wk)
{
    uint32_t Cr[WM];
#pragma unroll
    for (int w = 0; w < WM; ++w) Cr[w] = __shfl_sync(kFull, C, w);
    // 128-bit groups where C is non-zero (warp-uniform)
    const uint32_t nz = __ballot_sync(kFull, lane < WM && C != 0u);
    const int glo = nz ? (__ffs(nz) - 1) >> 2 : 0, ghi = nz ? (31 - __clz(nz)) >> 2 : -1;
    const uint32_t pc = (uint32_t)__popc(C);
    uint32_t pre = pc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, pre, o);
        if (lane >= o) pre += t;
    }
    const uint32_t total = __shfl_sync(kFull, pre, 31);
    const uint32_t excl = pre - pc;
    uint32_t S = 0;
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t j = base + (uint32_t)lane;
        int w = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t pv_ = __shfl_sync(kFull, pre, w + step - 1);
            if (pv_ <= j) w += step;
        }
        const uint32_t cw = __shfl_sync(kFull, C, w);
        const uint32_t ex = __shfl_sync(kFull, excl, w);
        unsigned words = 0;
        if (j < total) {
            const int e = w * 32 + (int)__fns(cw, 0, (int)(j - ex) + 1);
            uint32_t f = 0;
            if (WM >= 4) {
                // upper rows (no memberships) hold nothing below e's group
                const int elo = PV ? glo : max(glo, e >> 7);
                const uint4* A4 = (const uint4*)(A + (int64_t)e * RS);
#pragma unroll
                for (int q = 0; q < WM / 4; ++q) {
                    if (q < elo || q > ghi) continue;
                    const uint4 a = A4[q];
                    f += (uint32_t)(__popc(Cr[4 * q] & a.x) + __popc(Cr[4 * q + 1] & a.y) +
                                    __popc(Cr[4 * q + 2] & a.z) + __popc(Cr[4 * q + 3] & a.w));
                }
                words = (unsigned)(4 * (ghi - elo + 1));
            } else {
                const uint32_t* Ae = A + (int64_t)e * RS;
#pragma unroll
                for (int q = 0; q < WM; ++q) f += (uint32_t)__popc(Cr[q] & Ae[q]);
                words = (unsigned)WM;
            }
            S += f;
            if (PV && f) pv_add(pvlo, pvhi, e, f);
        }
        if (wk) *wk += (unsigned long long)__reduce_add_sync(kFull, words);
    }
    const uint32_t E = __reduce_add_sync(kFull, S);
    return PV ? E / 2u : E;
}

// Last level for a class of row width WM (0: generic loop).
template <bool PV, int WM>
__device__ __forceinline__ uint32_t leaf2_any(uint32_t C, int w0, int Wd, const uint32_t* A, int RS, uint32_t* pvlo,
                                              uint32_t* pvhi, int lane, unsigned long long* wk)
{
    if (WM > 0) return leaf2_rep<PV, (WM > 0 ? WM : 1)>(C, Wd, A, RS, pvlo, pvhi, lane, wk);
    return leaf2_reg<PV>(C, w0, Wd, A, RS, pvlo, pvhi, lane, wk);
}

// Triangles of a dense G[C] through its complement (per-vertex mode,
// symmetric rows).  With c = |C|, d_v the degree of v in G[C], nb_v = c-1-d_v,
// X_v the non-neighbours of v in C (v excluded) and M the non-edges of G[C]:
// the triangles through v are the edges inside N(v), i.e. C(d_v, 2) less the
// non-edges inside N(v), and splitting the M non-edges by how they meet v
// gives  M = nb_v + nonedges(N(v)) + sum_{a in X_v} (nb_a - 1) - nonedges(X_v),
// so a lane reads its element's row once and then only the rows of the
// element's few non-neighbours a: nb_a comes from a per-warp byte table (255 =
// too large for a byte, recounted from the row) and the non-edges inside X_v
// from popc(X_v & ~row(a)) over the words.
// A first pass fills the table and sums the degrees (so M); the second runs
// only if G[C] is dense enough for this to pay (non-edges below a quarter of
// the edges), else the call returns false and nothing is credited.  C words
// are read from sC; groups outside [glo, ghi] of C are empty.
template <int WM>
__device__ __forceinline__ uint32_t nonadj_words(const uint4* C4, const uint4* F4, int glo, int ghi)
{
    uint32_t na = 0;
#pragma unroll
    for (int r = 0; r < WM / 4; ++r) {
        if (r < glo || r > ghi) continue;
        const uint4 f = F4[r], c4 = C4[r];
        na += (uint32_t)(__popc(c4.x & ~f.x) + __popc(c4.y & ~f.y) + __popc(c4.z & ~f.z) + __popc(c4.w & ~f.w));
    }
    return na;
}

template <int WM>
__device__ bool penult3_co(const uint32_t* sC, uint8_t* nb, int glo, int ghi, uint32_t total, uint32_t pre,
                           uint32_t excl, uint32_t C, const uint32_t* A, int RS, uint32_t* pvlo, uint32_t* pvhi,
                           int lane, unsigned long long* wk, unsigned long long* out)
{
    const uint4* C4 = (const uint4*)sC;
    const unsigned ng4 = 4u * (unsigned)(ghi - glo + 1);
    uint32_t nbl = 0;
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t j = base + (uint32_t)lane;
        int w = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t pv_ = __shfl_sync(kFull, pre, w + step - 1);
            if (pv_ <= j) w += step;
        }
        const uint32_t cw = __shfl_sync(kFull, C, w);
        const uint32_t ex = __shfl_sync(kFull, excl, w);
        if (j < total) {
            const int e = w * 32 + (int)__fns(cw, 0, (int)(j - ex) + 1);
            const uint4* Ae4 = (const uint4*)(A + (int64_t)e * RS);
            uint32_t dg = 0;
#pragma unroll
            for (int q = 0; q < WM / 4; ++q) {
                if (q < glo || q > ghi) continue;
                const uint4 a = Ae4[q], c4 = C4[q];
                dg += (uint32_t)(__popc(c4.x & a.x) + __popc(c4.y & a.y) + __popc(c4.z & a.z) + __popc(c4.w & a.w));
            }
            const uint32_t nbe = total - 1u - dg;
            nb[e] = (uint8_t)min(nbe, 255u);
            nbl += nbe;
        }
    }
    const uint32_t nbsum = __reduce_add_sync(kFull, nbl);  // 2M
    if (wk) *wk += (unsigned long long)total * ng4;
    const uint32_t dsum = total * (total - 1u) - nbsum;   // 2 |E(G[C])|
    if (4ull * nbsum >= (unsigned long long)dsum) return false;
    __syncwarp();
    const long long M = (long long)(nbsum >> 1);
    unsigned long long tot = 0, wl = 0;
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t j = base + (uint32_t)lane;
        int w = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t pv_ = __shfl_sync(kFull, pre, w + step - 1);
            if (pv_ <= j) w += step;
        }
        const uint32_t cw = __shfl_sync(kFull, C, w);
        const uint32_t ex = __shfl_sync(kFull, excl, w);
        const bool valid = j < total;
        const int e = valid ? w * 32 + (int)__fns(cw, 0, (int)(j - ex) + 1) : 0;
        const uint4* Ae4 = (const uint4*)(A + (int64_t)e * RS);
        uint32_t X[WM];
#pragma unroll
        for (int q = 0; q < WM / 4; ++q) {
            if (!valid || q < glo || q > ghi) {
                X[4 * q] = X[4 * q + 1] = X[4 * q + 2] = X[4 * q + 3] = 0u;
                continue;
            }
            const uint4 a = Ae4[q], c4 = C4[q];
            X[4 * q] = c4.x & ~a.x;
            X[4 * q + 1] = c4.y & ~a.y;
            X[4 * q + 2] = c4.z & ~a.z;
            X[4 * q + 3] = c4.w & ~a.w;
        }
        // X holds e itself (rows have no loops): nb_e = |X| - 1
        uint32_t px = 0;
#pragma unroll
        for (int q = 0; q < WM; ++q) px += (uint32_t)__popc(X[q]);
        const uint32_t nbe = valid ? px - 1u : 0u;
        // S1 = sum over a in X_e of (nb_a - 1); E2 = twice the non-edges inside
        // X_e.  The groups of X are visited by a runtime loop (the per-element
        // body is unrolled over the four words of a group only).
        uint32_t S1 = 0, E2 = 0;
#pragma unroll 1
        for (int g = glo; g <= ghi; ++g) {
            uint32_t xg[4] = {X[0], X[1], X[2], X[3]};
#pragma unroll
            for (int h = 1; h < WM / 4; ++h)
                if (g == h) {
                    xg[0] = X[4 * h];
                    xg[1] = X[4 * h + 1];
                    xg[2] = X[4 * h + 2];
                    xg[3] = X[4 * h + 3];
                }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint32_t bits = xg[i];
                while (bits) {
                    const int a = (4 * g + i) * 32 + __ffs(bits) - 1;
                    bits &= bits - 1u;
                    if (a == e) continue;
                    const uint4* F4 = (const uint4*)(A + (int64_t)a * RS);
                    uint32_t na = nb[a];
                    if (na == 255u) na = nonadj_words<WM>(C4, F4, glo, ghi) - 1u;
                    S1 += na - 1u;
                    uint32_t xa = 0;
#pragma unroll
                    for (int r = 0; r < WM / 4; ++r) {
                        if (r < glo || r > ghi) continue;
                        const uint4 f = F4[r];
                        xa += (uint32_t)(__popc(X[4 * r] & ~f.x) + __popc(X[4 * r + 1] & ~f.y) +
                                         __popc(X[4 * r + 2] & ~f.z) + __popc(X[4 * r + 3] & ~f.w));
                    }
                    E2 += xa - 2u;  // X minus N(a) holds a and e
                    wl += ng4;
                }
            }
        }
        const uint32_t XE = E2 >> 1;
        if (valid) {
            const long long de = (long long)(total - 1u - nbe);
            const long long te = de * (de - 1) / 2 - (M - (long long)nbe - (long long)S1 + (long long)XE);
            tot += (unsigned long long)te;
            if (te) pv_add(pvlo, pvhi, e, (unsigned long long)te);
        }
    }
    if (wk) *wk += warp_sum64(wl) + (unsigned long long)total * ng4;
    *out = warp_sum64(tot) / 3ull;
    return true;
}

// All children of a node whose candidate set C (lane w holds word w) still
// needs three vertices: the cliques below are the triangles of G[C].  Each
// lane takes one element e of C and forms Ce = C & N(e) in its own
// registers: without memberships N(e) is e's upper row (the elements above
// e), and the lane counts the edges inside Ce -- the triangles whose smallest
// vertex is e; with memberships (symmetric rows) N(e) is e's whole row and
// the lane counts the edges inside it -- the triangles of G[C] through e,
// e's membership increment (so no lane writes another lane's counter); the
// number of triangles is a third of their sum.  The edges inside Ce are
// counted as the sum over f in Ce of popc(Ce & up(f)), where up(f) is f's
// row above f: only the words from f's own word on are read (with symmetric
// rows the lower part is masked off).  sC: per-warp buffer of WM words
// (16-byte aligned).  The work counter gets the words actually ANDed.
template <bool PV, int WM>
__device__ unsigned long long penult3(uint32_t C, int Wd, const uint32_t* A, int RS, uint32_t* pvlo,
                                      uint32_t* pvhi, uint32_t* sC, uint8_t* nb, int lane, unsigned long long* wk)
{
    if (lane < WM) sC[lane] = C;
    __syncwarp();
    // 128-bit groups of words where C (hence every Ce) can be non-zero: the
    // same for the whole warp, so the row loops skip the rest uniformly
    const uint32_t nz = __ballot_sync(kFull, lane < WM && C != 0u);
    if (nz == 0u) return 0ull;
    const int glo = (__ffs(nz) - 1) >> 2, ghi = (31 - __clz(nz)) >> 2;
    const int xhi = 4 * ghi + 3;  // last word that can be non-zero
    const uint32_t pc = (uint32_t)__popc(C);
    uint32_t pre = pc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, pre, o);
        if (lane >= o) pre += t;
    }
    const uint32_t total = __shfl_sync(kFull, pre, 31);
    const uint32_t excl = pre - pc;
    if (PV && nb) {
        unsigned long long co = 0;
        const bool done = penult3_co<WM>(sC, nb, glo, ghi, total, pre, excl, C, A, RS, pvlo, pvhi, lane, wk, &co);
        if (done) {
            __syncwarp();
            return co;
        }
    }
    unsigned long long tot = 0, wl = 0;
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t j = base + (uint32_t)lane;
        int w = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t pv_ = __shfl_sync(kFull, pre, w + step - 1);
            if (pv_ <= j) w += step;
        }
        const uint32_t cw = __shfl_sync(kFull, C, w);
        const uint32_t ex = __shfl_sync(kFull, excl, w);
        if (j < total) {
            const int e = w * 32 + (int)__fns(cw, 0, (int)(j - ex) + 1);
            // Ce = C & N(e): upper rows hold nothing below e's group
            const int elo = PV ? glo : max(glo, e >> 7);
            uint32_t Ce[WM];
            const uint4* Ae4 = (const uint4*)(A + (int64_t)e * RS);
            const uint4* C4 = (const uint4*)sC;
#pragma unroll
            for (int q = 0; q < WM / 4; ++q) {
                if (q < elo || q > ghi) {
                    Ce[4 * q] = Ce[4 * q + 1] = Ce[4 * q + 2] = Ce[4 * q + 3] = 0u;
                    continue;
                }
                const uint4 a = Ae4[q], cc4 = C4[q];
                Ce[4 * q] = cc4.x & a.x;
                Ce[4 * q + 1] = cc4.y & a.y;
                Ce[4 * q + 2] = cc4.z & a.z;
                Ce[4 * q + 3] = cc4.w & a.w;
            }
            if (wk) wl += (unsigned long long)(4 * (ghi - elo + 1));
            uint32_t S = 0;
#pragma unroll
            for (int q = 0; q < WM; ++q) {  // f in word q of Ce: words q.. of up(f)
                if (q > xhi) continue;
                uint32_t bits = Ce[q];
                while (bits) {
                    const int fb = __ffs(bits) - 1;
                    bits &= bits - 1u;
                    const uint32_t* F = A + (int64_t)(q * 32 + fb) * RS;
                    const uint4* F4 = (const uint4*)F;
                    uint32_t dgr = 0;
#pragma unroll
                    for (int r = q / 4; r < WM / 4; ++r) {
                        if (r > ghi) continue;
                        const uint4 a = F4[r];
                        const uint32_t ax = 4 * r + 0 < q ? 0u : (4 * r + 0 == q ? (PV ? a.x & cc::mask_above(fb) : a.x) : a.x);
                        const uint32_t ay = 4 * r + 1 < q ? 0u : (4 * r + 1 == q ? (PV ? a.y & cc::mask_above(fb) : a.y) : a.y);
                        const uint32_t az = 4 * r + 2 < q ? 0u : (4 * r + 2 == q ? (PV ? a.z & cc::mask_above(fb) : a.z) : a.z);
                        const uint32_t aw = 4 * r + 3 < q ? 0u : (4 * r + 3 == q ? (PV ? a.w & cc::mask_above(fb) : a.w) : a.w);
                        dgr += (uint32_t)(__popc(Ce[4 * r] & ax) + __popc(Ce[4 * r + 1] & ay) +
                                          __popc(Ce[4 * r + 2] & az) + __popc(Ce[4 * r + 3] & aw));
                    }
                    S += dgr;
                    if (wk) wl += (unsigned long long)(xhi + 1 - q);
                }
            }
            tot += S;
            if (PV && S) pv_add(pvlo, pvhi, e, S);
        }
    }
    if (wk) *wk += warp_sum64(wl);
    __syncwarp();
    const unsigned long long all = warp_sum64(tot);
    return PV ? all / 3ull : all;
}

// ------------------------------------------------ compact sub-tree (<= 64)

__device__ __forceinline__ unsigned long long mask64_above(int b) { return b >= 63 ? 0ull : (~0ull << (b + 1)); }

// Row of compact vertex v (held by lane v & 31, word v >> 5).
__device__ __forceinline__ unsigned long long crow(unsigned long long r0, unsigned long long r1, int v)
{
    const unsigned long long a = __shfl_sync(kFull, r0, v & 31);
    const unsigned long long b = __shfl_sync(kFull, r1, v & 31);
    return v < 32 ? a : b;
}

// Edges inside the compact set C.  Per-vertex mode: each member's degree
// inside C (full rows f) is its membership increment and the edge count is
// half their sum; otherwise the upper rows u count higher neighbours.
template <bool PV>
__device__ __forceinline__ unsigned long long cleaf2(unsigned long long C, unsigned long long u0,
                                                     unsigned long long u1, unsigned long long f0,
                                                     unsigned long long f1, int lane, unsigned long long& a0,
                                                     unsigned long long& a1)
{
    const bool in0 = (C >> lane) & 1ull, in1 = (C >> (lane + 32)) & 1ull;
    if (PV) {
        const unsigned d0 = in0 ? (unsigned)__popcll(C & f0) : 0u;
        const unsigned d1 = in1 ? (unsigned)__popcll(C & f1) : 0u;
        a0 += d0;
        a1 += d1;
        return (unsigned long long)(__reduce_add_sync(kFull, d0 + d1) / 2u);
    }
    unsigned e = 0;
    if (in0) e += (unsigned)__popcll(C & u0);
    if (in1) e += (unsigned)__popcll(C & u1);
    return (unsigned long long)__reduce_add_sync(kFull, e);
}

// Cliques of `need` (>= 2) vertices chosen from the n-vertex compact graph
// (upper rows u, full rows f in per-vertex mode), with memberships in a0/a1.
template <bool PV>
__device__ unsigned long long cdfs(unsigned long long u0, unsigned long long u1, unsigned long long f0,
                                   unsigned long long f1, int n, int need, int lane, unsigned long long& a0,
                                   unsigned long long& a1, unsigned long long* wk)
{
    const unsigned long long all = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
    if (need == 2) {
        if (wk) *wk += (unsigned long long)n * (PV ? 4 : 2);
        return cleaf2<PV>(all, u0, u1, f0, f1, lane, a0, a1);
    }
    unsigned long long tot = 0, cur = all, cur_sub = 0;
    unsigned long long st_rem = 0, st_sub = 0;
    int st_e = 0, t = 0;
    for (;;) {
        if (cur == 0ull) {
            if (t == 0) break;
            const unsigned long long sdone = cur_sub;
            --t;
            cur = __shfl_sync(kFull, st_rem, t);
            const int pe = __shfl_sync(kFull, st_e, t);
            cur_sub = __shfl_sync(kFull, st_sub, t) + sdone;
            if (PV && lane == (pe & 31)) {
                if (pe < 32) a0 += sdone; else a1 += sdone;
            }
            continue;
        }
        const int e = __ffsll((long long)cur) - 1;
        cur &= cur - 1ull;
        const unsigned long long Cn = cur & crow(u0, u1, e);
        const int nd = need - t - 1;
        if (wk) *wk += 2;
        if (__popcll(Cn) < nd) continue;
        if (nd == 2) {
            if (wk) *wk += (unsigned long long)__popcll(Cn) * (PV ? 4 : 2);
            const unsigned long long E = cleaf2<PV>(Cn, u0, u1, f0, f1, lane, a0, a1);
            tot += E;
            cur_sub += E;
            if (PV && lane == (e & 31)) {
                if (e < 32) a0 += E; else a1 += E;
            }
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
    return tot;
}

// The sub-tree below a candidate set C (lane w holds word w, n = |C| <= 64
// elements, `need` >= 3 vertices still to choose), on a compact copy of G[C].
template <bool PV>
__device__ unsigned long long compact_count(uint32_t C, int n, int need, const uint32_t* A, int RS,
                                            uint32_t* pvlo, uint32_t* pvhi, int lane, unsigned long long* wk)
{
    // elements p_j (lane j: p_j and p_{j+32}) by rank
    const uint32_t pc = (uint32_t)__popc(C);
    uint32_t pre = pc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, pre, o);
        if (lane >= o) pre += t;
    }
    const uint32_t excl = pre - pc;
    int p[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint32_t j = (uint32_t)(lane + 32 * h);
        int w = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t pv_ = __shfl_sync(kFull, pre, w + step - 1);
            if (pv_ <= j) w += step;
        }
        const uint32_t cw = __shfl_sync(kFull, C, w);
        const uint32_t ex = __shfl_sync(kFull, excl, w);
        p[h] = j < (uint32_t)n ? w * 32 + (int)__fns(cw, 0, (int)(j - ex) + 1) : 0;
    }
    // compact rows: bit j of row i = adjacency of p_i and p_j
    unsigned long long r0 = 0, r1 = 0;
    for (int i = 0; i < n; ++i) {
        const int pi = __shfl_sync(kFull, i < 32 ? p[0] : p[1], i & 31);
        const uint32_t* Ai = A + (int64_t)pi * RS;
        const bool b0 = lane < n && ((Ai[p[0] >> 5] >> (p[0] & 31)) & 1u);
        const bool b1 = lane + 32 < n && ((Ai[p[1] >> 5] >> (p[1] & 31)) & 1u);
        const unsigned long long row =
            (unsigned long long)__ballot_sync(kFull, b0) | ((unsigned long long)__ballot_sync(kFull, b1) << 32);
        if (lane == (i & 31)) {
            if (i < 32) r0 = row; else r1 = row;
        }
    }
    if (wk) *wk += (unsigned long long)n * 2;
    const unsigned long long u0 = r0 & mask64_above(lane), u1 = r1 & mask64_above(lane + 32);
    unsigned long long a0 = 0, a1 = 0;
    const unsigned long long tot = cdfs<PV>(u0, u1, r0, r1, n, need, lane, a0, a1, wk);
    if (PV) {
        if (a0 && lane < n) pv_add(pvlo, pvhi, p[0], a0);
        if (a1 && lane + 32 < n) pv_add(pvlo, pvhi, p[1], a1);
    }
    return tot;
}

// Owners with 33..64 elements (two-word rows), one warp each, without shared
// memory: lane j holds x_j and x_{j+32} and, as 64-bit words, their rows of
// G+(u) -- built like the one-word class (each 32-entry chunk of Gamma+(x_i)
// searched for both elements of every lane by shuffle binary search, four
// rows' first chunks loaded together) -- then the compact search (cdfs)
// counts the (k-1)-cliques on those registers.  No block barrier, no
// per-owner set-up beyond the loads: these owners are too many and too small
// for a CTA each.
template <bool PV, bool COL>
__global__ void __launch_bounds__(256) k_count_w2(Ctx cb)
{
    const int lane = threadIdx.x & 31;
    const int need = cb.k - 1;  // vertices to choose inside G+(u)
    for (;;) {
        unsigned long long pos = 0;
        if (lane == 0) pos = atomicAdd(cb.cursor, 1ull);
        pos = __shfl_sync(kFull, pos, 0);
        Ctx c;
        int32_t r;
        if (!cc::resolve(cb, (int64_t)pos, c, r)) break;
        const int64_t b = c.offp[r];
        const int d = (int)(c.offp[r + 1] - b);  // 33..64
        const int32_t xa = lane < d ? c.adjp[b + lane] : INT_MAX;
        const int32_t xb = lane + 32 < d ? c.adjp[b + 32 + lane] : INT_MAX;
        const int32_t ur = COL ? c.perm[r] : 0;
        uint32_t cola = 0, colb = 0;
        if (COL) {
            if (lane < d) cola = cc::sample_label(c, ur, c.perm[xa]);
            if (lane + 32 < d) colb = cc::sample_label(c, ur, c.perm[xb]);
        }
        const int32_t maxL = __shfl_sync(kFull, xb, (d - 33) & 31);
        const bool ha = lane < d - 1, hb = lane + 32 < d - 1;
        const int64_t la0 = ha ? c.offp[xa] : 0, la1 = ha ? c.offp[xa + 1] : 0;
        const int64_t lb0 = hb ? c.offp[xb] : 0, lb1 = hb ? c.offp[xb + 1] : 0;
        unsigned long long u0 = 0, u1 = 0;  // upper rows of elements lane, lane + 32
        for (int i0 = 0; i0 < d - 1; i0 += 4) {
            int32_t y[4];
            int64_t s0[4], s1[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int i = i0 + t;
                const int64_t a0 = __shfl_sync(kFull, la0, i & 31), a1 = __shfl_sync(kFull, la1, i & 31);
                const int64_t b0 = __shfl_sync(kFull, lb0, i & 31), b1 = __shfl_sync(kFull, lb1, i & 31);
                s0[t] = i < 32 ? a0 : b0;
                s1[t] = i < 32 ? a1 : b1;
                if (i >= d - 1) s1[t] = s0[t];
                const int64_t p = s0[t] + lane;
                y[t] = p < s1[t] ? c.adjp[p] : INT_MAX;
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int i = i0 + t;
                if (i >= d - 1) break;
                unsigned long long row = 0;
                for (int64_t p0 = s0[t];;) {
                    int la = 0, lb = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const int32_t ya = __shfl_sync(kFull, y[t], la + step - 1);
                        if (ya < xa) la += step;
                        const int32_t yb = __shfl_sync(kFull, y[t], lb + step - 1);
                        if (yb < xb) lb += step;
                    }
                    const bool hit_a = __shfl_sync(kFull, y[t], la) == xa && lane > i && lane < d;
                    const bool hit_b = __shfl_sync(kFull, y[t], lb) == xb && lane + 32 > i && lane + 32 < d;
                    row |= (unsigned long long)__ballot_sync(kFull, hit_a) |
                           ((unsigned long long)__ballot_sync(kFull, hit_b) << 32);
                    p0 += 32;
                    if (p0 >= s1[t] || __shfl_sync(kFull, y[t], 31) >= maxL) break;
                    const int64_t p = p0 + lane;
                    y[t] = p < s1[t] ? c.adjp[p] : INT_MAX;
                }
                if (COL) {
                    const uint32_t ci = i < 32 ? __shfl_sync(kFull, cola, i & 31) : __shfl_sync(kFull, colb, i & 31);
                    row &= (unsigned long long)__ballot_sync(kFull, cc::sample_keep(c, ur, ci, cola)) |
                           ((unsigned long long)__ballot_sync(kFull, cc::sample_keep(c, ur, ci, colb)) << 32);
                }
                if (lane == (i & 31)) {
                    if (i < 32) u0 = row; else u1 = row;
                }
            }
        }
        unsigned long long f0 = u0, f1 = u1;  // full rows (memberships): add the transpose
        if (PV) {
            for (int j = 1; j < d; ++j) {
                const unsigned long long colj = (unsigned long long)__ballot_sync(kFull, (u0 >> j) & 1ull) |
                                                ((unsigned long long)__ballot_sync(kFull, (u1 >> j) & 1ull) << 32);
                if (lane == (j & 31)) {
                    if (j < 32) f0 |= colj; else f1 |= colj;
                }
            }
        }
        unsigned long long a0 = 0, a1 = 0, wk = 0;
        const unsigned long long tot = cdfs<PV>(u0, u1, f0, f1, d, need, lane, a0, a1, c.work ? &wk : nullptr);
        if (lane == 0) {
            add_total(c.total, tot);
            if (c.po) c.po[r] = tot;
            if (PV && tot) atomicAdd(&c.pv[r], tot);
            if (c.work && wk) atomicAdd(c.work, wk);
        }
        if (PV) {
            if (a0 && lane < d) atomicAdd(&c.pv[xa], a0);
            if (a1 && lane + 32 < d) atomicAdd(&c.pv[xb], a1);
        }
    }
}

// Chains below a first-level choice: level 0 holds C (elements above i1),
// need0 >= 3 vertices still to choose.  Returns the cliques completed and
// credits chain members with their sub-tree totals (per-vertex mode).
template <bool PV, int WM>
__device__ unsigned long long dfs_reg(uint32_t c0, int need0, int Wd, const uint32_t* A, int RS, uint32_t* pvlo,
                                      uint32_t* pvhi, uint32_t* sC, uint8_t* nb, int lane, unsigned long long* wk,
                                      int clo, int chi)
{
    uint32_t st[kMaxLev];
#pragma unroll
    for (int i = 0; i < kMaxLev; ++i) st[i] = 0u;
    st[0] = c0;
    int t = 0;
    unsigned long long total = 0, cur_sub = 0, f_sub = 0;
    int f_e = 0;  // lane t: chain element chosen at level t
    for (;;) {
        uint32_t rem = st_get(st, t);
        const uint32_t nz = __ballot_sync(kFull, rem != 0u);
        if (nz == 0u) {
            if (t == 0) break;
            const unsigned long long sdone = cur_sub;
            --t;
            const int pe = __shfl_sync(kFull, f_e, t);
            cur_sub = __shfl_sync(kFull, f_sub, t) + sdone;
            if (PV && lane == 0 && sdone) pv_add(pvlo, pvhi, pe, sdone);
            continue;
        }
        const int fw = __ffs(nz) - 1;
        const uint32_t vw = __shfl_sync(kFull, rem, fw);
        const int e = fw * 32 + __ffs(vw) - 1;
        if (lane == fw) rem &= rem - 1u;
        st_set(st, t, rem);
        const uint32_t* Ae = A + (int64_t)e * RS;
        const uint32_t cn = (lane >= fw && lane < Wd) ? (rem & Ae[lane]) : 0u;
        const int cnt = (int)__reduce_add_sync(kFull, (unsigned)__popc(cn));
        if (wk) *wk += (unsigned long long)(Wd - fw);
        const int need = need0 - t - 1;
        if (cnt < need) continue;
        const bool tri = WM >= 4 && need == 3;
        const bool compact = !tri && cnt >= clo && cnt <= chi;
        if (need == 2 || compact || tri) {
            const unsigned long long E =
                need == 2 ? (unsigned long long)leaf2_any<PV, WM>(cn, fw, Wd, A, RS, pvlo, pvhi, lane, wk)
                : compact ? compact_count<PV>(cn, cnt, need, A, RS, pvlo, pvhi, lane, wk)
                          : penult3<PV, (WM >= 4 ? WM : 4)>(cn, Wd, A, RS, pvlo, pvhi, sC, nb, lane, wk);
            total += E;
            cur_sub += E;
            if (PV && lane == 0 && E) pv_add(pvlo, pvhi, e, E);
        } else {
            if (lane == t) {
                f_e = e;
                f_sub = cur_sub;
            }
            ++t;
            st_set(st, t, cn);
            cur_sub = 0;
        }
    }
    return total;
}

// The sub-tree below a candidate set C (lane w holds word w; cnt elements,
// the lowest in word fw) when `need` >= 2 vertices are still to be chosen:
// edges of G[C] (need 2), triangles (need 3; in the 4..16-word classes
// always on the bitmap rows, whose dense sets the complement count closes in
// about one pass), a compact copy (small C, need >= 4 there), or the
// register search below.  Credits the members met inside.
template <bool PV, int WM>
__device__ __forceinline__ unsigned long long subtree(uint32_t C, int cnt, int need, int fw, int Wd, const uint32_t* A,
                                                      int RS, uint32_t* pvlo, uint32_t* pvhi, uint32_t* sC, uint8_t* nb,
                                                      int lane, unsigned long long* wk, int clo, int chi)
{
    if (need == 2) return (unsigned long long)leaf2_any<PV, WM>(C, fw, Wd, A, RS, pvlo, pvhi, lane, wk);
    if (WM >= 4 && need == 3) return penult3<PV, (WM >= 4 ? WM : 4)>(C, Wd, A, RS, pvlo, pvhi, sC, nb, lane, wk);
    if (cnt >= clo && cnt <= chi) return compact_count<PV>(C, cnt, need, A, RS, pvlo, pvhi, lane, wk);
    return dfs_reg<PV, WM>(C, need, Wd, A, RS, pvlo, pvhi, sC, nb, lane, wk, clo, chi);
}

// Row e of G+(u) above e, one word per lane (lane w: word w).
__device__ __forceinline__ uint32_t upper_word(const uint32_t* A, int RS, int e, int Wd, int lane)
{
    const int we = e >> 5;
    uint32_t v = (lane >= we && lane < Wd) ? A[(int64_t)e * RS + lane] : 0u;
    if (lane == we) v &= mask_above(e & 31);
    return v;
}

// Work items of one owner u of the class: its search is cut into tasks --
// first-level vertices e1 for k <= 5; pairs (e1, e2), e2 a neighbour of e1
// above it, for k >= 6 (the second level of the heavy-owner split, Sec. 7:
// (k-2)-cliques of G+(u) counted under the key (u, e1), each of those cut
// again by e2).  Item i of the class launch is (owner i / R, part i % R);
// the R parts of an owner share its task counter, so they stay balanced
// however uneven the tasks are.
//   TILE = false: R == 1; the item's CTA builds G+(u) in shared memory (its
//       warps together) and hands out the tasks from a shared counter.
//   TILE = true: G+(u) was built once, by k_tile_build, into the owner's
//       global tile; every part copies it into shared memory and takes tasks
//       from the owner's global counter.
template <bool PV, bool COL, int WM, bool TILE>
__global__ void __launch_bounds__(256, 4) k_dfs_reg(Ctx cb, int W, int R, int clo, int chi, int co, const uint32_t* tiles,
                                                  int64_t tile_words, unsigned int* task_ctr)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, NW = blockDim.x >> 5;
    const int RS = row_stride(W, WM);
    const RLayout lay = make_rlayout(W, RS, PV, COL, NW);
    int32_t* sL = (int32_t*)(smem + lay.L);
    uint32_t* sCol = smem + lay.col;
    uint32_t* pvlo = smem + lay.pvlo;
    uint32_t* pvhi = smem + lay.pvhi;
    uint32_t* sA = smem + lay.A;
    // task prefix over first-level vertices (k >= 6): aliases the span table,
    // which is only used while the rows are built
    unsigned int* sP = smem + lay.sbits;
    // per-warp byte table of the complement count (classes of 4..16 words:
    // 8 warps x 32 W bytes fit in the span table after the 512 words of sP)
    uint8_t* nbw = co ? (uint8_t*)(smem + lay.sbits + 512) + wid * 32 * W : nullptr;
    __shared__ __align__(16) uint32_t s_c[8][32];  // per-warp candidate-set buffer
    __shared__ unsigned int s_ntask;
    __shared__ unsigned int s_next;
    __shared__ unsigned long long s_tot, s_wk;
    __shared__ long long s_item;
    const int r0 = cb.k - 1;
    const bool pairs = r0 >= 5;  // k >= 6: tasks are (e1, e2)

    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(cb.cursor, 1ull);
        __syncthreads();
        const int64_t oi = s_item / R;
        Ctx c;
        int32_t r;
        if (!cc::resolve(cb, oi, c, r)) break;
        const int64_t b = c.offp[r];
        const int d = (int)(c.offp[r + 1] - b);
        const int Wd = (d + 31) >> 5;
        for (int j = threadIdx.x; j < d; j += blockDim.x) {
            const int32_t x = c.adjp[b + j];
            sL[j] = x;
            if (!TILE && COL) sCol[j] = cc::sample_label(c, c.perm[r], c.perm[x]);
        }
        if (TILE) {
            const uint4* src = (const uint4*)(tiles + oi * tile_words);
            uint4* dst = (uint4*)sA;
            for (int64_t j = threadIdx.x; j < ((int64_t)d * RS + 3) / 4; j += blockDim.x) dst[j] = src[j];
        } else {
            for (int64_t j = threadIdx.x; j < (int64_t)d * RS; j += blockDim.x) sA[j] = 0u;
        }
        if (threadIdx.x == 0) {
            s_next = 0u;
            s_tot = 0ull;
            s_wk = 0ull;
        }
        __syncthreads();
        if (!TILE) {
            const int32_t ur = COL ? c.perm[r] : 0;
            if (COL) cc::class_flags_smem<true>(c, sCol, d, r0, threadIdx.x, blockDim.x);
            cc::SpanTable T{smem + lay.sbits, (uint16_t*)(smem + lay.spre), 0, 0};
            cc::span_table_build(T, sL, d, kSpanWords);
            cc::build_rows<PV, COL>(c, sL, sCol, d, sA, RS, wid, NW, lane, ur, &T);
            __syncthreads();
        }
        if (PV)
            for (int j = threadIdx.x; j < d; j += blockDim.x) {
                pvlo[j] = 0u;
                pvhi[j] = 0u;
            }
        unsigned int ntasks = (unsigned int)d;
        if (pairs) {  // sP[e] = number of pairs (e', e2) with e' < e
            for (int e = threadIdx.x; e < d; e += blockDim.x) {
                const uint32_t* Ae = sA + (int64_t)e * RS;
                unsigned int cnt = (unsigned int)__popc(Ae[e >> 5] & mask_above(e & 31));
                for (int w = (e >> 5) + 1; w < Wd; ++w) cnt += (unsigned int)__popc(Ae[w]);
                sP[e] = cnt;
            }
            __syncthreads();
            // exclusive scan of sP[0..d) by warp 0 (d <= 1024: 32 per lane)
            if (wid == 0) {
                const int per = (d + 31) / 32;
                unsigned int loc = 0;
                for (int q = 0; q < per; ++q) {
                    const int e = lane * per + q;
                    if (e < d) loc += sP[e];
                }
                unsigned int inc = loc;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned int t = __shfl_up_sync(kFull, inc, o);
                    if (lane >= o) inc += t;
                }
                unsigned int run = inc - loc;
                for (int q = 0; q < per; ++q) {
                    const int e = lane * per + q;
                    if (e < d) {
                        const unsigned int v = sP[e];
                        sP[e] = run;
                        run += v;
                    }
                }
                if (lane == 31) s_ntask = inc;
            }
            __syncthreads();
            ntasks = s_ntask;
        }
        unsigned int* ctr = TILE ? task_ctr + oi : &s_next;

        unsigned long long wtot = 0, wk = 0;
        unsigned long long* wkp = c.work ? &wk : nullptr;
        // pair tasks are taken kPairChunk at a time: one counter update per
        // chunk, and the chunk's later pairs follow row e1 without a search
        const unsigned int chunk = pairs ? (unsigned int)kPairChunk : 1u;
        for (;;) {
            unsigned int t0 = 0;
            if (lane == 0) t0 = atomicAdd(ctr, chunk);
            t0 = __shfl_sync(kFull, t0, 0);
            if (t0 >= ntasks) break;
            const unsigned int tend = min(t0 + chunk, ntasks);
            int e1 = 0, e2 = -1;
            uint32_t u1 = 0;
            for (unsigned int t = t0; t < tend; ++t) {
                if (r0 == 2) {  // k = 3: edges of G+(u) from e1 = t
                    const int e = (int)t;
                    const uint32_t* Ae = sA + (int64_t)e * RS;
                    const int we = e >> 5, be = e & 31;
                    uint32_t up = 0, all = 0;
                    if (lane < Wd) {
                        const uint32_t v = Ae[lane];
                        up = lane > we ? (uint32_t)__popc(v)
                                       : (lane == we ? (uint32_t)__popc(v & mask_above(be)) : 0u);
                        all = (uint32_t)__popc(v);
                    }
                    up = __reduce_add_sync(kFull, up);
                    wtot += up;
                    if (PV) {
                        all = __reduce_add_sync(kFull, all);
                        if (lane == 0 && all) pv_add(pvlo, pvhi, e, all);
                    }
                    if (wkp) wk += (unsigned long long)(PV ? Wd : Wd - we);
                    continue;
                }
                uint32_t cset;
                int need;
                if (!pairs) {
                    e1 = (int)t;
                    cset = upper_word(sA, RS, e1, Wd, lane);
                    need = r0 - 1;
                    if (wkp) wk += (unsigned long long)(Wd - (e1 >> 5));
                } else {
                    if (t == t0) {
                        // e1: the last vertex whose prefix is <= t (binary search in sP)
                        int lo = 0, hi = d;
                        while (hi - lo > 1) {
                            const int mid = (lo + hi) >> 1;
                            if (sP[mid] <= t) lo = mid; else hi = mid;
                        }
                        e1 = lo;
                        const unsigned int j = t - sP[e1];
                        // e2: the j-th element of row e1 above e1
                        u1 = upper_word(sA, RS, e1, Wd, lane);
                        const unsigned int pc = (unsigned int)__popc(u1);
                        unsigned int inc = pc;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const unsigned int x = __shfl_up_sync(kFull, inc, o);
                            if (lane >= o) inc += x;
                        }
                        const uint32_t hit = __ballot_sync(kFull, inc > j && inc - pc <= j);
                        const int hw = __ffs(hit) - 1;
                        const uint32_t hv = __shfl_sync(kFull, u1, hw);
                        const unsigned int hx = __shfl_sync(kFull, inc - pc, hw);
                        e2 = hw * 32 + (int)__fns(hv, 0, (int)(j - hx) + 1);
                    } else {
                        // the next pair: the next element of row e1 above e2, else
                        // the first element of the next row with any (pairs are
                        // numbered row by row, so t < ntasks guarantees one)
                        const int w2 = e2 >> 5;
                        uint32_t rest = lane > w2 ? u1 : (lane == w2 ? (u1 & mask_above(e2 & 31)) : 0u);
                        uint32_t nzm = __ballot_sync(kFull, rest != 0u);
                        while (nzm == 0u && e1 + 1 < d) {
                            ++e1;
                            u1 = upper_word(sA, RS, e1, Wd, lane);
                            rest = u1;
                            nzm = __ballot_sync(kFull, rest != 0u);
                        }
                        if (nzm == 0u) break;
                        const int hw = __ffs(nzm) - 1;
                        e2 = hw * 32 + __ffs(__shfl_sync(kFull, rest, hw)) - 1;
                    }
                    cset = u1 & upper_word(sA, RS, e2, Wd, lane);
                    need = r0 - 2;
                    if (wkp) wk += (unsigned long long)(2 * (Wd - (e1 >> 5)));
                }
                const int cnt = (int)__reduce_add_sync(kFull, (unsigned)__popc(cset));
                if (cnt < need) continue;
                const int fw = __ffs(__ballot_sync(kFull, cset != 0u)) - 1;
                const unsigned long long sub =
                    subtree<PV, WM>(cset, cnt, need, fw, Wd, sA, RS, pvlo, pvhi, s_c[wid], nbw, lane, wkp, clo, chi);
                wtot += sub;
                if (PV && lane == 0 && sub) {
                    pv_add(pvlo, pvhi, e1, sub);
                    if (pairs) pv_add(pvlo, pvhi, e2, sub);
                }
            }
        }
        if (lane == 0 && wtot) atomicAdd(&s_tot, wtot);
        if (lane == 0 && wk) atomicAdd(&s_wk, wk);
        __syncthreads();
        const unsigned long long tot = s_tot;
        if (threadIdx.x == 0) {
            add_total(c.total, tot);
            if (c.po && tot) atomicAdd(&c.po[r], tot);  // the R parts add up
            if (PV && c.pv && tot) atomicAdd(&c.pv[r], tot);
            if (c.work && s_wk) atomicAdd(c.work, s_wk);
        }
        if (PV && c.pv)  // (no output array: symmetric rows chosen for speed only)
            for (int j = threadIdx.x; j < d; j += blockDim.x) {
                const unsigned long long v = ((unsigned long long)pvhi[j] << 32) | pvlo[j];
                if (v) atomicAdd(&c.pv[sL[j]], v);
            }
        __syncthreads();
    }
}

// G+(u) of every owner of the class, built once into its global tile (the
// shared-memory row layout, d rows of RS words), for the split search.
template <bool PV, bool COL, int WM>
__global__ void __launch_bounds__(256) k_tile_build(Ctx cb, int W, uint32_t* tiles, int64_t tile_words)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, NW = blockDim.x >> 5;
    const int RS = row_stride(W, WM);
    const RLayout lay = make_rlayout(W, RS, false, COL, NW);
    int32_t* sL = (int32_t*)(smem + lay.L);
    uint32_t* sCol = smem + lay.col;
    uint32_t* sA = smem + lay.A;
    __shared__ long long s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(cb.cursor, 1ull);
        __syncthreads();
        const int64_t oi = s_item;
        Ctx c;
        int32_t r;
        if (!cc::resolve(cb, oi, c, r)) break;
        const int64_t b = c.offp[r];
        const int d = (int)(c.offp[r + 1] - b);
        const int32_t ur = COL ? c.perm[r] : 0;
        for (int j = threadIdx.x; j < d; j += blockDim.x) {
            const int32_t x = c.adjp[b + j];
            sL[j] = x;
            if (COL) sCol[j] = cc::sample_label(c, ur, c.perm[x]);
        }
        for (int64_t j = threadIdx.x; j < (int64_t)d * RS; j += blockDim.x) sA[j] = 0u;
        __syncthreads();
        if (COL) cc::class_flags_smem<true>(c, sCol, d, cb.k - 1, threadIdx.x, blockDim.x);
        cc::SpanTable T{smem + lay.sbits, (uint16_t*)(smem + lay.spre), 0, 0};
        cc::span_table_build(T, sL, d, kSpanWords);
        cc::build_rows<PV, COL>(c, sL, sCol, d, sA, RS, wid, NW, lane, ur, &T);
        __syncthreads();
        uint4* dst = (uint4*)(tiles + oi * tile_words);
        const uint4* src = (const uint4*)sA;
        for (int64_t j = threadIdx.x; j < ((int64_t)d * RS + 3) / 4; j += blockDim.x) dst[j] = src[j];
        __syncthreads();
    }
}

}  // namespace

bool dfs_reg_supported(int k) { return k >= 3 && k - 3 <= kMaxLev; }

// The two-word class (|Gamma+| 33..64), one warp per owner on registers.
kc_status w2_launch(const cc::Ctx& c, bool pv, bool col, cudaStream_t s)
{
    if (c.nitems <= 0) return KC_OK;
    auto go = [&](auto kern) -> kc_status {
        const int grid =
            (int)std::min<int64_t>((c.nitems + 7) / 8, (int64_t)num_sms() * cc::blocks_per_sm(kern, 256, 0));
        kern<<<grid, 256, 0, s>>>(c);
        KC_LAUNCHED();
        return KC_OK;
    };
    if (pv) return col ? KC_ENOTSUP : go(k_count_w2<true, false>);
    return col ? go(k_count_w2<false, true>) : go(k_count_w2<false, false>);
}

// Parts per owner: heavy owners (rows of 8+ words) are split for k >= 5,
// where one owner's search can outlast the rest of the class.
int parts_per_owner(int W, int k)
{
    if (k < 5) return 1;
    if (W >= 16) return 16;
    if (W >= 8) return 4;
    return 1;
}

// Tile memory (32-bit words) a class of width W with `items` owners needs for
// the split search at k (0: no split).
int64_t dfs_tile_words(int W, int k, int64_t items, int parts)
{
    if ((parts > 0 ? parts : parts_per_owner(W, k)) <= 1 || items <= 0) return 0;
    const int WM = W <= 16 ? W : 0;
    const int64_t per = 32LL * W * row_stride(W, WM);
    return per * items + (items + 3);  // tiles, then the task counters
}

// Launch the shared-memory class of width W (words) over its queue range.
// With an allocator and R > 1 the owners' rows are built once into global
// tiles (k_tile_build) and the R parts copy them; without one (the
// allocation-free entry point) every owner is searched by one CTA.
kc_status dfs_reg_launch(const cc::Ctx& c, int W, bool pv, bool col, Scratch* sc, int parts, cudaStream_t s)
{
    const int sms = num_sms();
    int R = parts > 0 ? parts : parts_per_owner(W, c.k);
    if (!sc) R = 1;
    const int NW = W <= 4 ? 4 : 8;
    const int WM = W <= 16 ? W : 0;  // widest class keeps the generic last level
    // Totals at k >= 6 in the 4..16-word classes run on symmetric rows too:
    // their dense need-3 sets then take the complement count, which beats
    // closing them on upper rows; the memberships stay in shared memory
    // (c.pv is null) and are dropped.  The layout follows the kernel chosen.
    const bool sym = pv || (!col && g_complement && c.k >= 6 && WM >= 4);
    const int RS = row_stride(W, WM);
    const RLayout lay = make_rlayout(W, RS, sym, col, NW);
    const size_t smem = (size_t)lay.total * 4;
    uint32_t* tiles = nullptr;
    unsigned int* ctr = nullptr;
    const int64_t tile_words = 32LL * W * RS;
    if (R > 1) {
        KC_TRY(sc->get(&tiles, dfs_tile_words(W, c.k, c.nitems, R)));
        ctr = tiles + tile_words * c.nitems;
        KC_CK(cudaMemsetAsync(ctr, 0, (size_t)c.nitems * sizeof(unsigned int), s));
    }
    auto pick = [&](auto kern, auto build) -> kc_status {
        if (R > 1) {
            // the build pass takes owners from the class cursor; the search
            // pass then counts items from a second cursor (the slot's next word)
            const RLayout bl = make_rlayout(W, RS, false, col, 8);
            const size_t bsm = (size_t)bl.total * 4;
            KC_CK(cc::allow_smem(build, bsm));
            const int bgrid = (int)std::min<int64_t>(c.nitems, (int64_t)sms * cc::blocks_per_sm(build, 256, bsm));
            build<<<bgrid, 256, bsm, s>>>(c, W, tiles, tile_words);
            KC_LAUNCHED();
        }
        cc::Ctx cs = c;
        if (R > 1) cs.cursor = c.cursor + kc::kOwnerSlots;  // a fresh zeroed cursor for the search
        KC_CK(cc::allow_smem(kern, smem));
        const int grid =
            (int)std::min<int64_t>(c.nitems * R, (int64_t)sms * cc::blocks_per_sm(kern, NW * 32, smem));
        kern<<<grid, NW * 32, smem, s>>>(cs, W, R, g_compact_lo, g_compact_hi, g_complement, tiles, tile_words, ctr);
        KC_LAUNCHED();
        return KC_OK;
    };
    auto by_width = [&](auto pv_t, auto col_t) -> kc_status {
        constexpr bool P = decltype(pv_t)::value, Q = decltype(col_t)::value;
        const bool split = R > 1;
#define KC_DFS_PICK(WMV)                                                                              \
    return split ? pick(k_dfs_reg<P, Q, WMV, true>, k_tile_build<P, Q, WMV>)                          \
                 : pick(k_dfs_reg<P, Q, WMV, false>, k_tile_build<P, Q, WMV>)
        switch (WM) {
        case 2: KC_DFS_PICK(2);
        case 4: KC_DFS_PICK(4);
        case 8: KC_DFS_PICK(8);
        case 16: KC_DFS_PICK(16);
        default: KC_DFS_PICK(0);
        }
#undef KC_DFS_PICK
    };
    if (sym) return col ? KC_ENOTSUP : by_width(std::true_type{}, std::false_type{});
    return col ? by_width(std::false_type{}, std::true_type{}) : by_width(std::false_type{}, std::false_type{});
}

}  // namespace kc
