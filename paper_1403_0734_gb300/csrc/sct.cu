// sct.cu -- Reduce 3 (Alg. 1; Sec. 3) by a pivoting clique tree.
//
// The paper leaves the local (k-1)-clique counter open (Sec. 4: a counter
// "based on neighborhood intersection"); any exact counter gives the same
// q_{u,k-1}.  This one walks G+(u) with Bron-Kerbosch pivoting, as in the
// succinct clique trees of Jain & Seshadhri (WSDM 2020), so that dense
// pieces of G+(u) -- the near-complete hub cores of power-law graphs -- cost a
// handful of nodes instead of one node per clique prefix.
//
// A node holds a candidate set S together with the "hold" vertices H and the
// "pivot" vertices P on its path from the root S = Gamma+(u).  With pivot
// p = argmax_{v in S} |S & N(v)| and S \ (N(p) + p) = {v_1, .., v_t}, the
// children are (S & N(v_i) minus v_1..v_{i-1}, hold v_i) for every i, and
// (S & N(p), pivot p).  Every clique of G+(u) is represented exactly once as
// H plus a subset of P of a leaf (S empty), so a leaf stands for
// C(|P|, k-1-|H|) k-cliques owned by u; per-vertex memberships follow: u and
// every hold get that number, every pivot C(|P|-1, k-2-|H|).
// Hold children are walked first and the pivot child last as a tail step, so
// the stack only grows with holds (at most k-1 frames).  The sub-tree of a
// node represents exactly the cliques H + Q + K' with Q a subset of P and K'
// a clique of G[S]; with t = k-1-|H| vertices still to choose this closes
// small cases without branching: t = 0 gives 1, t = 1 gives |P| + |S|,
// t = 2 gives C(|P|,2) + |P||S| + |E(G[S])| (the degrees inside S are computed
// for the pivot anyway), and a set S that is a clique gives C(|P|+|S|, t).
// Nodes with |H|+|P|+|S| < k-1 are pruned.
// The bitmap rows are symmetric here (N(v) within G+(u)).
#include <algorithm>

#include "count_common.cuh"

namespace kc {

int num_sms();
int smem_max_words();
int slot_words(int slot);

namespace {

using cc::add_total;
using cc::Ctx;

// C(n, r) for 0 <= r, exact; sets *ovf when the value does not fit 64 bits.
__device__ __forceinline__ unsigned long long binom(int n, int r, bool* ovf)
{
    if (r < 0 || n < 0 || r > n) return 0ull;
    if (r > n - r) r = n - r;
    unsigned __int128 c = 1;
    for (int i = 1; i <= r; ++i) {
        c = c * (unsigned __int128)(n - r + i) / (unsigned __int128)i;
        if (c >> 64) {
            *ovf = true;
            return 0ull;
        }
    }
    return (unsigned long long)c;
}

// ------------------------------------------------------------ W = 1 class

template <bool PV, bool COL>
__global__ void __launch_bounds__(256) k_sct_w1(Ctx cb)
{
    const int lane = threadIdx.x & 31;
    const int need = cb.k - 1;  // clique vertices inside G+(u)
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
        if (COL) col = cc::class_flag_w1(c, col, d, c.k - 1, lane);
        const uint32_t up = cc::build_rows_w1<COL>(c, x, d, col, ur, lane);
        const uint32_t A = up | cc::lower_rows_w1(up, d, lane);  // N(lane) inside G+(u)

        const bool cw = c.work != nullptr;
        unsigned long long tot = 0, pvl = 0, wk = 0;
        bool ovf = false;
        // frame f lives in lane f: candidate set, pivot, hold and pivot masks
        uint32_t fr_S = 0, fr_Hm = 0, fr_Pm = 0;
        int fr_p = 0;
        uint32_t S = d >= 32 ? kFull : ((1u << d) - 1u);
        uint32_t Hm = 0, Pm = 0;
        int nf = 0;
        for (;;) {
            const int h = __popc(Hm), pc = __popc(Pm), sz = __popc(S);
            const int t = need - h;  // clique vertices still to choose
            const bool in = (S >> lane) & 1u;
            if (t == 0) {
                if (tot + 1 < tot) ovf = true;
                tot += 1;
                if (PV && ((Hm >> lane) & 1u)) pvl += 1;
            } else if (pc + sz < t) {
                // pruned: no k-clique below
            } else if (t == 1) {  // one more vertex: a pivot or any vertex of S
                const unsigned long long T = (unsigned long long)(pc + sz);
                if (tot + T < tot) ovf = true;
                tot += T;
                if (PV) {
                    if ((Hm >> lane) & 1u) pvl += T;
                    if (((Pm >> lane) & 1u) || in) pvl += 1;
                }
            } else if (sz == 0) {
                const unsigned long long T = binom(pc, t, &ovf);
                if (tot + T < tot) ovf = true;
                tot += T;
                if (PV) {
                    if ((Hm >> lane) & 1u) pvl += T;
                    if ((Pm >> lane) & 1u) pvl += binom(pc - 1, t - 1, &ovf);
                }
            } else {
                const int deg = in ? __popc(S & A) : 0;
                if (cw) wk += (unsigned long long)sz;
                const unsigned dmin = __reduce_min_sync(kFull, in ? (unsigned)deg : 64u);
                if (t == 2) {  // two more: pivot pairs, pivot + S, edges of G[S]
                    const unsigned e2 = __reduce_add_sync(kFull, (unsigned)deg) / 2u;
                    const unsigned long long T = binom(pc, 2, &ovf) + (unsigned long long)pc * sz + e2;
                    if (tot + T < tot) ovf = true;
                    tot += T;
                    if (PV) {
                        if ((Hm >> lane) & 1u) pvl += T;
                        if ((Pm >> lane) & 1u) pvl += (unsigned long long)(pc - 1 + sz);
                        if (in) pvl += (unsigned long long)(pc + deg);
                    }
                } else if ((int)dmin == sz - 1) {  // S is a clique: all of it joins P
                    const unsigned long long T = binom(pc + sz, t, &ovf);
                    if (tot + T < tot) ovf = true;
                    tot += T;
                    if (PV) {
                        if ((Hm >> lane) & 1u) pvl += T;
                        if (((Pm >> lane) & 1u) || in) pvl += binom(pc + sz - 1, t - 1, &ovf);
                    }
                } else {
                    const unsigned key = in ? (((unsigned)deg << 5) | (31u - (unsigned)lane)) : 0u;
                    const int p = 31 - (int)(__reduce_max_sync(kFull, key) & 31u);
                    const uint32_t Ap = __shfl_sync(kFull, A, p);
                    const uint32_t R = S & ~Ap & ~(1u << p);
                    if (cw) wk += 1;
                    if (R) {  // push a frame, enter the first hold child
                        const int v = __ffs(R) - 1;
                        if (lane == nf) {
                            fr_S = S & ~(1u << v);
                            fr_p = p;
                            fr_Hm = Hm;
                            fr_Pm = Pm;
                        }
                        ++nf;
                        S &= __shfl_sync(kFull, A, v);
                        Hm |= 1u << v;
                    } else {  // tail step into the pivot child
                        S &= Ap;
                        Pm |= 1u << p;
                    }
                    continue;
                }
            }
            // next node: the next hold child of the top frame, or its pivot child
            if (nf == 0) break;
            const int f = nf - 1;
            const uint32_t fS = __shfl_sync(kFull, fr_S, f);
            const int fp = __shfl_sync(kFull, fr_p, f);
            const uint32_t fHm = __shfl_sync(kFull, fr_Hm, f);
            const uint32_t fPm = __shfl_sync(kFull, fr_Pm, f);
            const uint32_t Afp = __shfl_sync(kFull, A, fp);
            const uint32_t R = fS & ~Afp & ~(1u << fp);
            if (cw) wk += 1;
            if (R) {
                const int v = __ffs(R) - 1;
                if (lane == f) fr_S = fS & ~(1u << v);
                S = fS & __shfl_sync(kFull, A, v);
                Hm = fHm | (1u << v);
                Pm = fPm;
            } else {
                --nf;
                S = fS & Afp;
                Hm = fHm;
                Pm = fPm | (1u << fp);
            }
        }
        if (lane == 0) {
            add_total(c.total, tot);
            if (ovf) atomicAdd(&c.total[1], 1ull);
            if (c.po) c.po[r] = tot;
            if (PV && tot) atomicAdd(&c.pv[r], tot);
            if (cw && wk) atomicAdd(c.work, wk);
        }
        if (PV && lane < d && pvl) atomicAdd(&c.pv[x], pvl);
    }
}

// ------------------------------------------------- wider owners (warp each)

// Per-warp working set, in 32-bit words (D = 32 W local ids).
struct WLayout {
    int64_t L, col, pv, A, el, piv, fr, cur, total;
};

__host__ __device__ inline WLayout make_wlayout(int W, int RS, int need, bool pv, bool col)
{
    const int64_t D = 32LL * W;
    WLayout l;
    l.L = 0;
    l.col = l.L + D;
    l.pv = l.col + (col ? D : 0);
    l.pv += l.pv & 1;  // 8-byte alignment of the 64-bit counters
    l.A = l.pv + (pv ? 2 * D : 0);
    l.el = l.A + D * RS;
    l.piv = l.el + D;
    l.fr = l.piv + D;
    l.cur = l.fr + (int64_t)(need > 0 ? need : 1) * W;
    l.total = l.cur + W;
    l.total += l.total & 1;
    return l;
}

template <bool PV, bool COL, bool HEAVY>
__global__ void __launch_bounds__(256) k_sct_warp(Ctx cb, int W, uint32_t* gscratch, int64_t slot_words)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int need = cb.k - 1;
    const int RS = HEAVY ? W : W + 1;
    const WLayout lay = make_wlayout(W, RS, need, PV, COL);
    uint32_t* base = HEAVY ? gscratch + ((int64_t)blockIdx.x * (blockDim.x >> 5) + wid) * slot_words
                           : smem + (int64_t)wid * lay.total;
    int32_t* sL = (int32_t*)(base + lay.L);
    uint32_t* sCol = base + lay.col;
    unsigned long long* sPV = (unsigned long long*)(base + lay.pv);
    uint32_t* sA = base + lay.A;
    int32_t* el = (int32_t*)(base + lay.el);
    int32_t* piv = (int32_t*)(base + lay.piv);
    uint32_t* fr = base + lay.fr;
    uint32_t* cur = base + lay.cur;
    const uint32_t lt = (1u << lane) - 1u;

    for (;;) {
        unsigned long long pos = 0;
        if (lane == 0) pos = atomicAdd(cb.cursor, 1ull);
        pos = __shfl_sync(kFull, pos, 0);
        Ctx c;
        int32_t r;
        if (!cc::resolve(cb, (int64_t)pos, c, r)) break;
        const int64_t b = c.offp[r];
        const int d = (int)(c.offp[r + 1] - b);
        const int Wd = (d + 31) >> 5;
        const int32_t ur = COL ? c.perm[r] : 0;
        for (int j = lane; j < d; j += 32) {
            const int32_t xj = c.adjp[b + j];
            sL[j] = xj;
            if (COL) sCol[j] = cc::sample_label(c, ur, c.perm[xj]);
            if (PV) sPV[j] = 0ull;
        }
        for (int64_t j = lane; j < (int64_t)d * RS; j += 32) sA[j] = 0u;
        for (int w = lane; w < Wd; w += 32) cur[w] = w < (d >> 5) ? kFull : ((1u << (d & 31)) - 1u);
        __syncwarp();
        if (COL) cc::class_flags_smem<false>(c, sCol, d, c.k - 1, lane, 32);
        cc::build_rows<true, COL>(c, sL, sCol, d, sA, RS, 0, 1, lane, ur);
        __syncwarp();

        const bool cw = c.work != nullptr;
        unsigned long long tot = 0, wk = 0;
        bool ovf = false;
        int fr_p = 0, fr_pc = 0, fr_lo = 0, fr_hi = 0;  // frame f in lane f
        int hold_v = 0;                                  // hold j in lane j
        int h = 0, pc = 0, lo = 0, hi = Wd;
        for (;;) {
            // ---- node: S = cur[lo..hi)
            int sz = 0;
            for (int w = lo + lane; w < hi; w += 32) sz += __popc(cur[w]);
            sz = (int)__reduce_add_sync(kFull, (unsigned)sz);
            const int t = need - h;  // clique vertices still to choose
            // Closed sub-tree: holds (and u) get T, path pivots cp, vertices of
            // S (listed in el when el_ok) cs plus, when ds, their degree in S.
            bool closed = true, el_ok = false;
            unsigned long long T = 0, cp = 0, cs = 0, ds = 0;
            if (t == 0) {
                T = 1;
            } else if (pc + sz < t) {
                T = 0;  // pruned
            } else if (sz == 0) {
                T = binom(pc, t, &ovf);
                cp = binom(pc - 1, t - 1, &ovf);
            } else {
                // list S in el[0..sz) and tighten the word bounds
                int nel = 0, nlo = hi, nhi = lo;
                for (int w0 = lo; w0 < hi; w0 += 32) {
                    const int w = w0 + lane;
                    const uint32_t v = w < hi ? cur[w] : 0u;
                    uint32_t nz = __ballot_sync(kFull, v != 0u);
                    if (nz) {
                        nlo = min(nlo, w0 + __ffs(nz) - 1);
                        nhi = w0 + 32 - __clz(nz);
                    }
                    while (nz) {
                        const int f = __ffs(nz) - 1;
                        nz &= nz - 1u;
                        const uint32_t bits = __shfl_sync(kFull, v, f);
                        if ((bits >> lane) & 1u) el[nel + __popc(bits & lt)] = (w0 + f) * 32 + lane;
                        nel += __popc(bits);
                    }
                }
                lo = nlo;
                hi = nhi;
                el_ok = true;
                __syncwarp();
                if (t == 1) {
                    T = (unsigned long long)(pc + sz);
                    cp = 1;
                    cs = 1;
                } else {
                    // degrees inside S: pivot = argmax, edges of G[S], clique test
                    unsigned long long best = 0, esum = 0;
                    int dmin = INT_MAX;
                    for (int j = lane; j < nel; j += 32) {
                        const int e = el[j];
                        const uint32_t* Ae = sA + (int64_t)e * RS;
                        int deg = 0;
                        for (int w = lo; w < hi; ++w) deg += __popc(cur[w] & Ae[w]);
                        dmin = min(dmin, deg);
                        esum += (unsigned long long)deg;
                        const unsigned long long key = ((unsigned long long)(unsigned)deg << 32) | (unsigned)(~e);
                        best = key > best ? key : best;
                    }
                    if (cw) wk += (unsigned long long)nel * (unsigned long long)(hi - lo);
                    dmin = (int)__reduce_min_sync(kFull, (unsigned)dmin);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const unsigned long long ob = __shfl_xor_sync(kFull, best, o);
                        best = ob > best ? ob : best;
                        esum += __shfl_xor_sync(kFull, esum, o);
                    }
                    if (t == 2) {  // two more: pivot pairs, pivot + S, edges of G[S]
                        T = binom(pc, 2, &ovf) + (unsigned long long)pc * sz + esum / 2;
                        cp = (unsigned long long)(pc - 1 + sz);
                        cs = (unsigned long long)pc;
                        ds = 1;
                    } else if (dmin == sz - 1) {  // S is a clique: all of it joins P
                        T = binom(pc + sz, t, &ovf);
                        cp = cs = binom(pc + sz - 1, t - 1, &ovf);
                    } else {
                        closed = false;
                        const int p = (int)~(unsigned)(best & 0xffffffffull);
                        const uint32_t* Ap = sA + (int64_t)p * RS;
                        // first element of R = S \ (N(p) + p)
                        int v = -1;
                        for (int w0 = lo; w0 < hi && v < 0; w0 += 32) {
                            const int w = w0 + lane;
                            uint32_t rv = 0;
                            if (w < hi) {
                                rv = cur[w] & ~Ap[w];
                                if (w == (p >> 5)) rv &= ~(1u << (p & 31));
                            }
                            const uint32_t nz = __ballot_sync(kFull, rv != 0u);
                            if (nz) {
                                const int f = __ffs(nz) - 1;
                                v = (w0 + f) * 32 + __ffs(__shfl_sync(kFull, rv, f)) - 1;
                            }
                        }
                        if (cw) wk += (unsigned long long)(hi - lo);
                        if (v >= 0) {  // push frame h, enter hold child v
                            uint32_t* F = fr + (int64_t)h * W;
                            const uint32_t* Av = sA + (int64_t)v * RS;
                            for (int w = lo + lane; w < hi; w += 32) {
                                const uint32_t sw = cur[w];
                                F[w] = (w == (v >> 5)) ? (sw & ~(1u << (v & 31))) : sw;
                                cur[w] = sw & Av[w];
                            }
                            if (lane == h) {
                                fr_p = p;
                                fr_pc = pc;
                                fr_lo = lo;
                                fr_hi = hi;
                                hold_v = v;
                            }
                            ++h;
                        } else {  // tail step into the pivot child
                            for (int w = lo + lane; w < hi; w += 32) cur[w] &= Ap[w];
                            if (lane == 0) piv[pc] = p;
                            ++pc;
                        }
                        __syncwarp();
                    }
                }
            }
            if (!closed) continue;
            if (T) {
                if (tot + T < tot) ovf = true;
                tot += T;
                if (PV) {
                    if (lane < h) sPV[hold_v] += T;
                    if (cp)
                        for (int j = lane; j < pc; j += 32) sPV[piv[j]] += cp;
                    if (el_ok && (cs || ds)) {
                        for (int j = lane; j < sz; j += 32) {
                            const int e = el[j];
                            unsigned long long add = cs;
                            if (ds) {
                                const uint32_t* Ae = sA + (int64_t)e * RS;
                                int deg = 0;
                                for (int w = lo; w < hi; ++w) deg += __popc(cur[w] & Ae[w]);
                                add += (unsigned long long)deg;
                            }
                            if (add) sPV[e] += add;
                        }
                    }
                    __syncwarp();
                }
            }
            // ---- next: the top frame's next hold child, or its pivot child
            if (h == 0) break;
            const int f = h - 1;
            const int fp = __shfl_sync(kFull, fr_p, f);
            const int fpc = __shfl_sync(kFull, fr_pc, f);
            lo = __shfl_sync(kFull, fr_lo, f);
            hi = __shfl_sync(kFull, fr_hi, f);
            uint32_t* F = fr + (int64_t)f * W;
            const uint32_t* Afp = sA + (int64_t)fp * RS;
            int v = -1;
            for (int w0 = lo; w0 < hi && v < 0; w0 += 32) {
                const int w = w0 + lane;
                uint32_t rv = 0;
                if (w < hi) {
                    rv = F[w] & ~Afp[w];
                    if (w == (fp >> 5)) rv &= ~(1u << (fp & 31));
                }
                const uint32_t nz = __ballot_sync(kFull, rv != 0u);
                if (nz) {
                    const int g = __ffs(nz) - 1;
                    v = (w0 + g) * 32 + __ffs(__shfl_sync(kFull, rv, g)) - 1;
                }
            }
            if (cw) wk += (unsigned long long)(hi - lo);
            pc = fpc;
            if (v >= 0) {
                const uint32_t* Av = sA + (int64_t)v * RS;
                for (int w = lo + lane; w < hi; w += 32) {
                    const uint32_t sw = F[w];
                    cur[w] = sw & Av[w];
                    if (w == (v >> 5)) F[w] = sw & ~(1u << (v & 31));
                }
                if (lane == f) hold_v = v;
                h = f + 1;
            } else {
                for (int w = lo + lane; w < hi; w += 32) cur[w] = F[w] & Afp[w];
                if (lane == 0) piv[pc] = fp;
                ++pc;
                h = f;
            }
            __syncwarp();
        }
        if (lane == 0) {
            add_total(c.total, tot);
            if (ovf) atomicAdd(&c.total[1], 1ull);
            if (c.po) c.po[r] = tot;
            if (PV && tot) atomicAdd(&c.pv[r], tot);
            if (cw && wk) atomicAdd(c.work, wk);
        }
        if (PV)
            for (int j = lane; j < d; j += 32) {
                const unsigned long long v = sPV[j];
                if (v) atomicAdd(&c.pv[sL[j]], v);
            }
        __syncwarp();
    }
}

template <bool PV, bool COL>
kc_status launch_slot_sct(int slot, int Wh, const Ctx& c, uint32_t* heavy, int64_t heavy_words, cudaStream_t s)
{
    if (c.nitems <= 0) return KC_OK;
    const int sms = num_sms();
    const int need = c.k - 1;
    if (slot == 0) {  // rows wider than the shared-memory limit: global tiles, one warp each
        const WLayout lay = make_wlayout(Wh, Wh, need, PV, COL);
        const int64_t slots = heavy_words / lay.total;
        if (slots < 1) return KC_ENOMEM;
        const int NW = (int)std::min<int64_t>(4, slots);
        const int64_t warps = std::min<int64_t>(slots, c.nitems);
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(warps / NW, (int64_t)sms * 8));
        k_sct_warp<PV, COL, true><<<grid, NW * 32, 0, s>>>(c, Wh, heavy, lay.total);
        KC_LAUNCHED();
        return KC_OK;
    }
    if (slot == kOwnerSlots - 1) {
        auto kern = k_sct_w1<PV, COL>;
        const int grid = (int)std::min<int64_t>((c.nitems + 7) / 8, (int64_t)sms * cc::blocks_per_sm(kern, 256, 0));
        kern<<<grid, 256, 0, s>>>(c);
        KC_LAUNCHED();
        return KC_OK;
    }
    const int W = slot_words(slot);
    const WLayout lay = make_wlayout(W, W + 1, need, PV, COL);
    const size_t per_warp = (size_t)lay.total * 4;
    const int NW = (int)std::max<size_t>(1, std::min<size_t>(8, (size_t)(100 * 1024) / per_warp));
    const size_t smem = per_warp * NW;
    auto kern = k_sct_warp<PV, COL, false>;
    KC_CK(cc::allow_smem(kern, smem));
    const int64_t ctas = (c.nitems + NW - 1) / NW;
    const int grid = (int)std::min<int64_t>(ctas, (int64_t)sms * cc::blocks_per_sm(kern, NW * 32, smem));
    kern<<<grid, NW * 32, smem, s>>>(c, W, nullptr, 0);
    KC_LAUNCHED();
    return KC_OK;
}

}  // namespace

int64_t sct_heavy_words_w(int W, int k, int64_t nheavy)
{
    const WLayout lay = make_wlayout(W, W, k - 1, true, true);
    const int64_t slots = std::min<int64_t>(nheavy, (int64_t)num_sms() * 4);
    return lay.total * slots;
}

kc_status sct_launch_slot(int slot, int Wh, const cc::Ctx& c, bool pv, bool col, uint32_t* heavy,
                          int64_t heavy_words, cudaStream_t s)
{
    if (pv) {
        if (col) return KC_ENOTSUP;
        return launch_slot_sct<true, false>(slot, Wh, c, heavy, heavy_words, s);
    }
    if (col) return launch_slot_sct<false, true>(slot, Wh, c, heavy, heavy_words, s);
    return launch_slot_sct<false, false>(slot, Wh, c, heavy, heavy_words, s);
}

}  // namespace kc
