// orient.cu -- Round 1 of Algorithm 1 (Sec. 3) on the device, asynchronous on
// the caller's stream (no host round trip, scratch from the library pool).
//
//   a1  d(v) = off[v+1] - off[v]                                   (Sec. 2)
//   a2  rank: stable LSD radix sort of the vertices by degree (ties keep id
//       order), so rank follows x < y iff d(x) < d(y) or d(x) = d(y), x < y
//   a3+a4  one gather pass over the adjacency: each row Gamma(v) is mapped
//       to ranks, filtered to Gamma+(v) = {x : rank x > rank v} and sorted
//       ascending, and written at the row's own input offset (a scratch copy
//       with the input's layout); |Gamma+(v)| goes to dplus[rank v]
//       -- offsets of the oriented CSR: scan of dplus in rank order
//       -- rows copied into rank order (no gathers)
//   a5  owner queue: by bitmap class (|Gamma+| in 1..32, 33..64, ...,
//       513..1024, > 1024: widest class first); inside the one-word class by
//       |Gamma+| descending, so the Reduce 1 filter |Gamma+(u)| >= k-1 is a
//       prefix of the queue for every k; inside the wider classes by the work
//       estimate w(u) = sum over x in Gamma+(u) of |Gamma+(x)| (the Gamma+(x)
//       entries Round 2 reads for u), descending; ties by rank.
//
// The gather pass reads every adjacency entry once and looks up its rank, a
// random 4-byte load from a 4n-byte table that stays in L2; that pass bounds
// the orientation (2m L2 gathers).  The sorts and the scan are single-pass
// (decoupled look-back: each tile publishes its aggregate and adds its
// predecessors'); their waits are bounded and report KC_ETIMEOUT.
#include <algorithm>
#include <climits>
#include <cstring>
#include <new>

#include "kc_internal.cuh"

namespace kc {

int num_sms();

namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------- control

// Device-side control block of one orientation (zeroed at the start).
struct Ctl {
    OrientStats st;                  // copied to the host at the end
    unsigned int dhist[4][256];      // degree digit histograms
    unsigned int qhist[1][256];      // queue-key histogram
    unsigned int tickets[16];        // tile / row tickets of the kernels
    unsigned int nlong_gather;       // rows deferred to k_gamma_long
    unsigned int nlong_rows;         // rows deferred to k_rows_long
    unsigned int nwide_rows;         // rows deferred to k_rows_wide
};

constexpr unsigned long long kFlagAgg = 1ull << 62;  // tile aggregate published
constexpr unsigned long long kFlagInc = 2ull << 62;  // inclusive prefix published
constexpr unsigned long long kValMask = (1ull << 62) - 1;
constexpr int kSpinLimit = 1 << 22;                  // bounded look-back wait

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p)
{
    return *(const volatile unsigned long long*)p;
}

// Exclusive prefix of tile `tile` from its predecessors' published words
// (value = low 62 bits): predecessors are read kLookBatch at a time (all in
// flight together), summed back to the nearest inclusive prefix.  A wait
// that runs out sets *err.
constexpr int kLookBatch = 8;

__device__ __forceinline__ unsigned long long look_back(const unsigned long long* status, int64_t tile, int64_t stride,
                                                     int* err)
{
    unsigned long long excl = 0;
    int64_t j = tile - 1;
    while (j >= 0) {
        unsigned long long w[kLookBatch];
#pragma unroll
        for (int i = 0; i < kLookBatch; ++i) w[i] = j - i >= 0 ? ld_volatile(status + (j - i) * stride) : 0ull;
        bool done = false;
#pragma unroll
        for (int i = 0; i < kLookBatch; ++i) {
            if (done || j - i < 0) continue;
            int spins = 0;
            while ((w[i] >> 62) == 0 && ++spins < kSpinLimit) w[i] = ld_volatile(status + (j - i) * stride);
            if ((w[i] >> 62) == 0) {
                atomicOr(err, 1);
                return excl;
            }
            excl += w[i] & kValMask;
            if (w[i] & kFlagInc) done = true;
        }
        if (done) break;
        j -= kLookBatch;
    }
    return excl;
}

// Histogram add, aggregated over the lanes of a warp that hit the same bin.
__device__ __forceinline__ void hist_add(unsigned int* h, uint32_t bin, bool valid)
{
    const uint32_t key = valid ? bin : 0xffffffffu;
    const uint32_t peers = __match_any_sync(kFull, key);
    if (valid && (peers & ((1u << (threadIdx.x & 31)) - 1u)) == 0) atomicAdd(&h[bin], (unsigned)__popc(peers));
}

// Sort passes the degree keys need: 8 bits each.
__device__ __forceinline__ int degree_passes(unsigned int max_deg)
{
    int bits = 0;
    while (bits < 32 && (max_deg >> bits)) ++bits;
    return (bits + 7) / 8;
}

// ---------------------------------------------------------------- a1

// Degrees, their digit histograms and their maximum.
__global__ void __launch_bounds__(kThreads) k_degree(const int64_t* __restrict__ off, int32_t n,
                                                    uint32_t* __restrict__ key, Ctl* ctl)
{
    __shared__ unsigned int h[4][256];
    for (int i = threadIdx.x; i < 4 * 256; i += kThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    unsigned int mx = 0;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t b = (int64_t)blockIdx.x * kThreads; b < n; b += stride) {  // warp-uniform bounds
        const int64_t v = b + threadIdx.x;
        const bool valid = v < n;
        const uint32_t d = valid ? (uint32_t)(off[v + 1] - off[v]) : 0u;
        if (valid) key[v] = d;
        mx = max(mx, d);
#pragma unroll
        for (int p = 0; p < 4; ++p) hist_add(h[p], (d >> (8 * p)) & 255u, valid);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * 256; i += kThreads) {
        const unsigned int c = (&h[0][0])[i];
        if (c) atomicAdd(&(&ctl->dhist[0][0])[i], c);
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(&ctl->st.max_deg, mx);
}

// ---------------------------------------------------------------- a2, a5

constexpr int kSwWarps = kThreads / 32;
constexpr int kSwPerLane = 16;
constexpr int kSwPerWarp = 32 * kSwPerLane;       // 512
constexpr int kSwTile = kSwWarps * kSwPerWarp;     // 4096

struct SweepArgs {
    const uint32_t* kin;
    const int32_t* vin;            // null: value = index
    uint32_t* kout;                // null: keys not kept
    int32_t* vout;
    int64_t n;
    int shift;
    const unsigned int* hist;      // [256] global histogram of this pass's digit
    unsigned long long* status;    // [tiles * 256], zeroed
    unsigned int* ticket;          // zeroed
    const unsigned int* max_deg;   // non-null: run iff pass < degree_passes(*max_deg)
    int pass;
    int* err;
};

// One stable counting-sort pass on an 8-bit digit (single pass: per-tile
// digit counts, decoupled look-back across tiles, scatter).  Tiles are taken
// in ticket order, so a tile waits only on tiles already running.
__global__ void __launch_bounds__(kThreads) k_sweep(SweepArgs a)
{
    if (a.max_deg && a.pass >= degree_passes(*a.max_deg)) return;
    __shared__ unsigned int cnt[kSwWarps][256];
    __shared__ unsigned int gbase[256];
    __shared__ unsigned int s_wsum[kSwWarps];
    __shared__ unsigned int s_tile;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(a.ticket, 1u);
    for (int i = tid; i < kSwWarps * 256; i += kThreads) (&cnt[0][0])[i] = 0;
    // exclusive offset of digit tid over the whole array
    const unsigned int hv = a.hist[tid];
    unsigned int hinc = hv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int t = __shfl_up_sync(kFull, hinc, o);
        if (lane >= o) hinc += t;
    }
    if (lane == 31) s_wsum[wid] = hinc;
    __syncthreads();
    unsigned int dig_off = hinc - hv;
    for (int w = 0; w < wid; ++w) dig_off += s_wsum[w];
    const int64_t tile = s_tile;
    const int64_t base = tile * kSwTile + (int64_t)wid * kSwPerWarp;
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t key[kSwPerLane], rnk[kSwPerLane];
    int32_t val[kSwPerLane];
#pragma unroll
    for (int j = 0; j < kSwPerLane; ++j) {
        const int64_t i = base + j * 32 + lane;
        const bool valid = i < a.n;
        key[j] = valid ? a.kin[i] : 0u;
        val[j] = valid ? (a.vin ? a.vin[i] : (int32_t)i) : 0;
    }
#pragma unroll
    for (int j = 0; j < kSwPerLane; ++j) {
        const int64_t i = base + j * 32 + lane;
        const bool valid = i < a.n;
        const uint32_t dig = valid ? (key[j] >> a.shift) & 255u : 256u + (uint32_t)lane;
        const uint32_t peers = __match_any_sync(kFull, dig);
        const uint32_t lower = (uint32_t)__popc(peers & lt);
        const uint32_t before = valid ? cnt[wid][dig] : 0u;
        __syncwarp();
        if (valid && lower == 0) cnt[wid][dig] = before + (uint32_t)__popc(peers);
        __syncwarp();
        rnk[j] = before + lower;
    }
    __syncthreads();
    {
        unsigned int run = 0;
#pragma unroll
        for (int w = 0; w < kSwWarps; ++w) {
            const unsigned int c = cnt[w][tid];
            cnt[w][tid] = run;
            run += c;
        }
        unsigned long long* st = a.status + tile * 256 + tid;
        unsigned long long excl = 0;
        if (tile == 0) {
            atomicExch(st, kFlagInc | run);
        } else {
            atomicExch(st, kFlagAgg | run);
            excl = look_back(a.status + tid, tile, 256, a.err);
            atomicExch(st, kFlagInc | (excl + run));
        }
        gbase[tid] = dig_off + (unsigned int)excl;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kSwPerLane; ++j) {
        const int64_t i = base + j * 32 + lane;
        if (i < a.n) {
            const uint32_t dig = (key[j] >> a.shift) & 255u;
            const unsigned int pos = gbase[dig] + cnt[wid][dig] + rnk[j];
            if (a.kout) a.kout[pos] = key[j];
            a.vout[pos] = val[j];
        }
    }
}

// perm / rank / degree in rank space from the finished degree sort: after p
// passes the pairs are in buffer A (p even) or B (p odd); with p = 0 every
// degree is 0 and the order is the id order.
__global__ void k_rank(Ctl* __restrict__ ctl, int launched, const uint32_t* __restrict__ kA,
                       const int32_t* __restrict__ vA, const uint32_t* __restrict__ kB, const int32_t* __restrict__ vB,
                       int32_t n, int32_t* __restrict__ perm, int32_t* __restrict__ rank, int32_t* __restrict__ deg_r)
{
    int np = degree_passes(ctl->st.max_deg);
    if (np > launched) {  // a degree above the host bound: the CSR is not what it claims
        np = launched;
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ctl->st.err_input, 1);
    }
    const uint32_t* k = (np & 1) ? kB : kA;
    const int32_t* v = np == 0 ? nullptr : ((np & 1) ? vB : vA);
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const int32_t x = v ? v[r] : r;
        perm[r] = x;
        rank[x] = r;
        deg_r[r] = (int32_t)k[r];
    }
}

// ---------------------------------------------------------------- a3, a4

// Ascending bitonic sort of N values in registers (N a power of two).
template <int N>
__device__ __forceinline__ void reg_sort(int32_t (&x)[N])
{
#pragma unroll
    for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const int32_t a = x[i], b = x[j];
                    if ((a > b) == up) {
                        x[i] = b;
                        x[j] = a;
                    }
                }
            }
        }
    }
}

// One compare-exchange step of a bitonic network over N (a power of two)
// values, by `nt` threads starting at `t0`: the merge step (mirrored pairs)
// when `mirror`, else the half-cleaner of width 2 * stride.  Pairs whose
// upper index is at or past `len` compare against a virtual +inf and stay
// (pass len >= N when the array is padded).
__device__ __forceinline__ void bitonic_step(int32_t* s, int N, int len, int lg, bool mirror, int t0, int nt)
{
    const int half = 1 << lg;
    for (int i = t0; i < N / 2; i += nt) {
        int lo, hi;
        if (mirror) {  // size = 2 * half
            lo = ((i >> lg) << (lg + 1)) + (i & (half - 1));
            hi = ((i >> lg) << (lg + 1)) + 2 * half - 1 - (i & (half - 1));
        } else {
            lo = ((i >> lg) << (lg + 1)) + (i & (half - 1));
            hi = lo + half;
        }
        if (hi < len) {
            const int32_t a = s[lo], c = s[hi];
            if (c < a) { s[lo] = c; s[hi] = a; }
        }
    }
}

// Ascending sort of s[0..len) in shared memory by one warp (bitonic over the
// next power of two, at least 64; the tail is padded with +inf).
__device__ void warp_smem_sort(int32_t* s, int len, int lane)
{
    int N = 64, lgN = 6;
    while (N < len) { N <<= 1; ++lgN; }
    for (int j = len + lane; j < N; j += 32) s[j] = INT_MAX;
    __syncwarp();
    for (int lsz = 1; lsz <= lgN; ++lsz) {
        bitonic_step(s, N, N, lsz - 1, true, lane, 32);
        __syncwarp();
        for (int ls = lsz - 2; ls >= 0; --ls) {
            bitonic_step(s, N, N, ls, false, lane, 32);
            __syncwarp();
        }
    }
}

constexpr int kGatherLong = 512;   // rows with more entries are gathered by one CTA each
constexpr int kGatherGroups = 4;   // 32-entry groups in flight per lane

// The gather pass.  For every vertex v, the ranks of Gamma(v) above rank v
// (= Gamma+(v) in rank space), in no particular order, are written to
// tmp[off[v] ..] (the input's layout), and their number to dplus[rank v].  A
// warp takes 32 consecutive vertices and walks their rows as one flat range
// of entries (rows of consecutive vertices are adjacent in the CSR), four
// 32-entry groups at a time; the lanes of a group that fall in the same row
// form a segment, compacted by ballot.  Units are taken from a ticket, so the
// warps stay balanced however the long rows fall.  Rows longer than
// kGatherLong are listed for k_gamma_long.
__global__ void __launch_bounds__(kThreads) k_gamma(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                                                   const int32_t* __restrict__ rank, int32_t n,
                                                   int32_t* __restrict__ tmp, int32_t* __restrict__ dplus,
                                                   int32_t* __restrict__ longrows, int64_t long_cap, Ctl* ctl)
{
    __shared__ unsigned int cnt_s[kThreads / 32][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t le = lane == 31 ? kFull : ((2u << lane) - 1u);
    unsigned int* cnt = cnt_s[wid];
    for (;;) {
        unsigned int unit = 0;
        if (lane == 0) unit = atomicAdd(&ctl->tickets[12], 1u);
        const int64_t v0 = (int64_t)__shfl_sync(kFull, unit, 0) * 32;
        if (v0 >= n) break;
        const int64_t v = v0 + lane;
        const bool valid = v < n;
        const int64_t b = valid ? off[v] : 0;
        const int d = valid ? (int)(off[v + 1] - b) : 0;
        const int32_t rv = valid ? rank[v] : 0;
        const bool lng = d > kGatherLong;
        if (lng) {
            const unsigned int i = atomicAdd(&ctl->nlong_gather, 1u);
            if (i < long_cap) longrows[i] = (int32_t)v;
            else atomicOr(&ctl->st.err_input, 1);  // more long rows than 2m allows
        }
        const int dd = lng ? 0 : d;
        int inc = dd;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += t;
        }
        const int pre = inc - dd;
        const int T = __shfl_sync(kFull, inc, 31);
        cnt[lane] = 0u;
        __syncwarp();
        for (int f0 = 0; f0 < T; f0 += 32 * kGatherGroups) {
            int row[kGatherGroups];
            int32_t y[kGatherGroups];
            int64_t rb[kGatherGroups];
#pragma unroll
            for (int u = 0; u < kGatherGroups; ++u) {
                const int f = f0 + u * 32 + lane;
                int lo = 0;  // the row of entry f: last lane whose prefix is <= f
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int pp = __shfl_sync(kFull, pre, lo + step);
                    if (pp <= f) lo += step;
                }
                row[u] = lo;
                rb[u] = __shfl_sync(kFull, b, lo);
                const int fr = f - __shfl_sync(kFull, pre, lo);
                y[u] = f < T ? adj[rb[u] + fr] : -1;
            }
#pragma unroll
            for (int u = 0; u < kGatherGroups; ++u) y[u] = y[u] >= 0 ? rank[y[u]] : INT_MIN;
#pragma unroll
            for (int u = 0; u < kGatherGroups; ++u) {
                const int rw = row[u];
                const bool keep = y[u] > __shfl_sync(kFull, rv, rw);
                const int prev = __shfl_up_sync(kFull, rw, 1);
                const uint32_t starts = __ballot_sync(kFull, lane == 0 || rw != prev);
                const int seg = 31 - __clz(starts & le);
                const uint32_t mine = ~((1u << seg) - 1u);  // lanes from my segment's start on
                const uint32_t km = __ballot_sync(kFull, keep);
                const unsigned int before = cnt[rw];
                __syncwarp();
                if (keep) tmp[rb[u] + before + __popc(km & lt & mine)] = y[u];
                const bool last = lane == 31 || ((starts >> (lane + 1)) & 1u);
                if (last) cnt[rw] = before + (unsigned int)__popc(km & le & mine);
                __syncwarp();
            }
        }
        if (valid && !lng) dplus[rv] = (int32_t)cnt[lane];
        __syncwarp();
    }
}

// Rows longer than kGatherLong: one CTA per row, warps taking 32-entry
// groups; kept entries are appended to tmp[off[v] ..] (one shared-memory
// atomic per group) in no particular order.
__global__ void __launch_bounds__(kThreads) k_gamma_long(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                                                        const int32_t* __restrict__ rank, const int32_t* __restrict__ longrows,
                                                        int64_t long_cap, int32_t* __restrict__ tmp,
                                                        int32_t* __restrict__ dplus, Ctl* ctl)
{
    __shared__ int s_cnt;
    __shared__ unsigned int s_row;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const unsigned int nlong = min(ctl->nlong_gather, (unsigned int)long_cap);
    for (;;) {
        if (threadIdx.x == 0) {
            s_row = atomicAdd(&ctl->tickets[14], 1u);
            s_cnt = 0;
        }
        __syncthreads();
        const unsigned int row = s_row;
        if (row >= nlong) break;
        const int32_t v = longrows[row];
        const int64_t b = off[v], e = off[v + 1];
        const int32_t rv = rank[v];
        for (int64_t p0 = b + (int64_t)wid * 32 * kGatherGroups; p0 < e; p0 += (int64_t)kThreads * kGatherGroups) {
            int32_t y[kGatherGroups];
#pragma unroll
            for (int u = 0; u < kGatherGroups; ++u) {
                const int64_t p = p0 + u * 32 + lane;
                y[u] = p < e ? adj[p] : -1;
            }
#pragma unroll
            for (int u = 0; u < kGatherGroups; ++u) y[u] = y[u] >= 0 ? rank[y[u]] : INT_MIN;
#pragma unroll
            for (int u = 0; u < kGatherGroups; ++u) {
                const bool keep = y[u] > rv;
                const uint32_t km = __ballot_sync(kFull, keep);
                int base = 0;
                if (lane == 0 && km) base = atomicAdd(&s_cnt, __popc(km));
                base = __shfl_sync(kFull, base, 0);
                if (keep) tmp[b + base + __popc(km & lt)] = y[u];
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) dplus[rv] = s_cnt;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- offsets

constexpr int kScPerThread = 16;
constexpr int kScTile = kThreads * kScPerThread;  // 4096

// offp = exclusive scan of dplus (rank order), single pass with decoupled
// look-back, plus the statistics of d+ (maximum, wedges, class counts).
__global__ void __launch_bounds__(kThreads) k_offsets(const int32_t* __restrict__ dplus, int32_t n, int64_t m,
                                                     int64_t* __restrict__ offp, unsigned long long* __restrict__ status,
                                                     Ctl* ctl)
{
    __shared__ unsigned int s_tile;
    __shared__ unsigned long long s_warp[kThreads / 32];
    __shared__ unsigned long long s_base;
    __shared__ unsigned int h[40];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(&ctl->tickets[0], 1u);
    if (tid < 40) h[tid] = 0;
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t r0 = tile * kScTile + (int64_t)tid * kScPerThread;
    int32_t x[kScPerThread];
    unsigned long long sum = 0, wedges = 0;
    unsigned int mx = 0;
#pragma unroll
    for (int j = 0; j < kScPerThread; ++j) {
        const int64_t r = r0 + j;
        x[j] = r < n ? dplus[r] : 0;
        sum += (unsigned long long)x[j];
        const unsigned long long d = (unsigned long long)x[j];
        wedges += d * (d - (d > 0)) / 2;
        mx = max(mx, (unsigned int)x[j]);
    }
    // block exclusive scan of the per-thread sums
    unsigned long long inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) s_warp[wid] = inc;
    __syncthreads();
    if (tid == 0) {
        unsigned long long run = 0;
        for (int w = 0; w < kThreads / 32; ++w) {
            const unsigned long long c = s_warp[w];
            s_warp[w] = run;
            run += c;
        }
        unsigned long long excl = 0;
        if (tile == 0) {
            atomicExch(status, kFlagInc | run);
        } else {
            atomicExch(status + tile, kFlagAgg | run);
            excl = look_back(status, tile, 1, &ctl->st.err_timeout);
            atomicExch(status + tile, kFlagInc | (excl + run));
        }
        s_base = excl;
        if ((tile + 1) * kScTile >= n) {  // last tile: the total
            offp[n] = (int64_t)(excl + run);
            if ((int64_t)(excl + run) != m) atomicOr(&ctl->st.err_input, 1);
        }
    }
    __syncthreads();
    unsigned long long pre = s_base + s_warp[wid] + inc - sum;
#pragma unroll
    for (int j = 0; j < kScPerThread; ++j) {
        const int64_t r = r0 + j;
        if (r < n) offp[r] = (int64_t)pre;
        pre += (unsigned long long)x[j];
    }
    // class histogram: d+ = 0..32 one bin each, then 33..64, ..., > 1024
#pragma unroll
    for (int j = 0; j < kScPerThread; ++j) {
        const unsigned int d = (unsigned int)x[j];
        unsigned int bin = d;
        if (d > 32) {
            bin = 33;
            while (bin < 38 && d > (32u << (bin - 32))) ++bin;
        }
        hist_add(h, bin, r0 + j < n);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(kFull, mx, o));
        wedges += __shfl_xor_sync(kFull, wedges, o);
    }
    if (lane == 0) {
        if (mx) atomicMax(&ctl->st.max_dplus, mx);
        if (wedges) atomicAdd(&ctl->st.wedges, wedges);
    }
    __syncthreads();
    if (tid < 33 && h[tid]) atomicAdd(&ctl->st.eq[tid], (unsigned long long)h[tid]);
    if (tid >= 33 && tid < 39 && h[tid]) atomicAdd(&ctl->st.cls[tid - 33], (unsigned long long)h[tid]);
}

// ---------------------------------------------------------------- rows, queue key

// Work-estimate quantisation: two steps per doubling above 2^10, 0..31.
__device__ __forceinline__ uint32_t quantise_work(unsigned long long w)
{
    const unsigned long long x = w + 1;
    const int b = 63 - __clzll((long long)x);
    const int f = b >= 1 ? (int)((x >> (b - 1)) & 1ull) : 0;
    const int q = 2 * b + f - 20;
    return q < 0 ? 0u : (q > 31 ? 31u : (uint32_t)q);
}

// Queue key (8 bits, ascending key = queue order) of an owner with
// |Gamma+| = d and work estimate w: class 0 (d > 1024) .. 5 (33..64),
// 6 (1..32), 7 (d = 0) in the top three bits; below them 32 - d in class 6
// and 31 - quantised w in classes 0..5.
__device__ __forceinline__ uint32_t queue_key(int d, unsigned long long w)
{
    if (d == 0) return 7u << 5;
    if (d <= 32) return (6u << 5) | (uint32_t)(32 - d);
    uint32_t cls = 0;
    if (d <= 64) cls = 5;
    else if (d <= 128) cls = 4;
    else if (d <= 256) cls = 3;
    else if (d <= 512) cls = 2;
    else if (d <= 1024) cls = 1;
    return (cls << 5) | (31u - quantise_work(w));
}

// Sort of one row of at most N entries held in shared memory, by one lane.
template <int N>
__device__ __forceinline__ void lane_sort(int32_t* s, int d)
{
    int32_t x[N];
#pragma unroll
    for (int j = 0; j < N; ++j) x[j] = j < d ? s[j] : INT_MAX;
    reg_sort<N>(x);
#pragma unroll
    for (int j = 0; j < N; ++j)
        if (j < d) s[j] = x[j];
}

constexpr int kRowsLane = 32;     // rows with at most this many entries: sorted by their lane
constexpr int kRowsWarp = 512;     // rows up to this many: one warp each; longer: one CTA each
constexpr int kRowsThreads = 128;  // four warps per CTA
constexpr int kRowsBuf = 32 * kRowsLane;  // entries a warp stages: 32 rows of at most kRowsLane

// Rows into rank order, sorted: adjp[offp[r] ..] = sort(tmp[off[perm r] ..])
// (length dplus[r]), for rows of at most kRowsLane entries, and the queue key
// of those owners.  A warp takes 32 consecutive ranks (a ticket): their rows
// are staged in shared memory in batches of whole rows (coalesced loads along
// each row), sorted there by their own lane in registers, and stored back
// coalesced (the rows of consecutive ranks are adjacent in the output).
// Longer rows are listed for k_rows_wide / k_rows_long.  A row that would end
// past m (a CSR that is not symmetric) is not copied and flags the input.
__global__ void __launch_bounds__(kRowsThreads) k_rows(const int64_t* __restrict__ off, const int32_t* __restrict__ perm,
                                                      const int32_t* __restrict__ dplus, const int64_t* __restrict__ offp,
                                                      const int32_t* __restrict__ tmp, int32_t n, int64_t m,
                                                      int32_t* __restrict__ adjp, uint32_t* __restrict__ qkey,
                                                      int32_t* __restrict__ widerows, int32_t* __restrict__ longrows,
                                                      int64_t long_cap, Ctl* ctl)
{
    __shared__ unsigned int h[256];
    __shared__ int32_t buf[kRowsThreads / 32][kRowsBuf];
    for (int i = threadIdx.x; i < 256; i += kRowsThreads) h[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t* sb = buf[wid];
    for (;;) {
        unsigned int unit = 0;
        if (lane == 0) unit = atomicAdd(&ctl->tickets[13], 1u);
        const int64_t r0 = (int64_t)__shfl_sync(kFull, unit, 0) * 32;
        if (r0 >= n) break;
        const int64_t r = r0 + lane;
        const bool valid = r < n;
        const int32_t v = valid ? perm[r] : 0;
        const int d = valid ? dplus[r] : 0;
        const int64_t src = valid ? off[v] : 0;
        const int64_t dst = valid ? offp[r] : 0;
        const bool fits = dst + d <= m;
        if (valid && !fits) atomicOr(&ctl->st.err_input, 1);
        if (valid && d > kRowsWarp) {
            const unsigned int i = atomicAdd(&ctl->nlong_rows, 1u);
            if (i < long_cap) longrows[i] = (int32_t)r;
            else atomicOr(&ctl->st.err_input, 1);
        } else if (valid && d > kRowsLane) {
            widerows[atomicAdd(&ctl->nwide_rows, 1u)] = (int32_t)r;
        }
        const int dd = d <= kRowsLane ? d : 0;
        int inc = dd;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += t;
        }
        const int pre = inc - dd;
        const int T = __shfl_sync(kFull, inc, 31);  // at most 32 * kRowsLane <= kRowsBuf
        for (int f0 = 0; f0 < T; f0 += 32) {
            const int f = f0 + lane;
            int lo = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int pp = __shfl_sync(kFull, pre, lo + step);
                if (pp <= f) lo += step;
            }
            const int64_t rs = __shfl_sync(kFull, src, lo);
            const int fr = f - __shfl_sync(kFull, pre, lo);
            if (f < T) sb[f] = tmp[rs + fr];
        }
        __syncwarp();
        if (dd > 1) {
            int32_t* row = sb + pre;
            if (dd <= 8) lane_sort<8>(row, dd);
            else if (dd <= 16) lane_sort<16>(row, dd);
            else lane_sort<32>(row, dd);
        }
        __syncwarp();
        for (int f0 = 0; f0 < T; f0 += 32) {
            const int f = f0 + lane;
            int lo = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int pp = __shfl_sync(kFull, pre, lo + step);
                if (pp <= f) lo += step;
            }
            const int64_t rd0 = __shfl_sync(kFull, dst, lo);
            const bool rf = __shfl_sync(kFull, (int)fits, lo) != 0;
            const int fr = f - __shfl_sync(kFull, pre, lo);
            if (f < T && rf) adjp[rd0 + fr] = sb[f];
        }
        __syncwarp();
        const bool here = valid && d <= kRowsLane;
        const uint32_t key = queue_key(d, 0);
        if (here) qkey[r] = key;
        hist_add(h, key, here);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += kRowsThreads) {
        const unsigned int c = h[i];
        if (c) atomicAdd(&ctl->qhist[0][i], c);
    }
}

// Ascending bitonic sort of 32 K values held by a warp, element k * 32 + lane
// in register x[k] of `lane`: exchanges across lanes by shuffles, within a
// lane by register swaps.
template <int K>
__device__ __forceinline__ void warp_reg_sort(int32_t (&x)[K], int lane)
{
#pragma unroll
    for (int size = 2; size <= 32 * K; size <<= 1) {
#pragma unroll
        for (int j = size >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int kj = j >> 5;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const int kk = k ^ kj;
                    if (kk > k) {
                        const bool up = ((k * 32) & size) == 0;  // same for both (j < size)
                        const int32_t a = x[k], b = x[kk];
                        if ((a > b) == up) {
                            x[k] = b;
                            x[kk] = a;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const int i = k * 32 + lane;
                    const int32_t o = __shfl_xor_sync(kFull, x[k], j);
                    const bool up = (i & size) == 0;
                    const bool lower = (lane & j) == 0;
                    x[k] = (lower == up) ? min(x[k], o) : max(x[k], o);
                }
            }
        }
    }
}

// One row of kRowsLane+1 .. 32 K entries by one warp, in registers: load,
// work estimate w = sum over the entries x of |Gamma+(x)|, sort, store.
template <int K>
__device__ __forceinline__ unsigned long long wide_row(const int32_t* __restrict__ src, int d,
                                                      const int32_t* __restrict__ dplus, int32_t* __restrict__ dst,
                                                      bool fits, int lane)
{
    int32_t x[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int j = k * 32 + lane;
        x[k] = j < d ? src[j] : INT_MAX;
    }
    unsigned long long w = 0;
#pragma unroll
    for (int k = 0; k < K; ++k)
        if (x[k] != INT_MAX) w += (unsigned long long)dplus[x[k]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(kFull, w, o);
    warp_reg_sort<K>(x, lane);
    if (fits) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int j = k * 32 + lane;
            if (j < d) dst[j] = x[k];
        }
    }
    return w;
}

constexpr int kWideBatch = 4;  // rows per ticket (their metadata loads overlap)

// Rows of kRowsLane+1 .. kRowsWarp entries: one warp per row (tickets of
// kWideBatch rows) loads it into registers, sums the work estimate w = sum |Gamma+(x)| over
// its entries, sorts it, stores it, and sets the owner's queue key.
__global__ void __launch_bounds__(kRowsThreads) k_rows_wide(const int64_t* __restrict__ off, const int32_t* __restrict__ perm,
                                                           const int32_t* __restrict__ dplus,
                                                           const int64_t* __restrict__ offp,
                                                           const int32_t* __restrict__ tmp, int64_t m,
                                                           int32_t* __restrict__ adjp, uint32_t* __restrict__ qkey,
                                                           const int32_t* __restrict__ widerows, Ctl* ctl)
{
    __shared__ unsigned int h[256];
    for (int i = threadIdx.x; i < 256; i += kRowsThreads) h[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const unsigned int nwide = ctl->nwide_rows;
    for (;;) {
        unsigned int b0 = 0;
        if (lane == 0) b0 = atomicAdd(&ctl->tickets[11], (unsigned int)kWideBatch);
        b0 = __shfl_sync(kFull, b0, 0);
        if (b0 >= nwide) break;
        // the metadata of kWideBatch rows, one lane each, loaded together
        const unsigned int mi = b0 + (unsigned int)lane;
        const bool mv = lane < kWideBatch && mi < nwide;
        const int32_t mr = mv ? widerows[mi] : 0;
        const int md = mv ? dplus[mr] : 0;
        const int64_t msrc = mv ? off[perm[mr]] : 0;
        const int64_t mdst = mv ? offp[mr] : 0;
        const int cnt = (int)min((unsigned int)kWideBatch, nwide - b0);
        for (int q = 0; q < cnt; ++q) {
            const int32_t r = __shfl_sync(kFull, mr, q);
            const int d = __shfl_sync(kFull, md, q);
            const int32_t* src = tmp + __shfl_sync(kFull, msrc, q);
            const int64_t dst = __shfl_sync(kFull, mdst, q);
            const bool fits = dst + d <= m;
            unsigned long long w;
            if (d <= 64) w = wide_row<2>(src, d, dplus, adjp + dst, fits, lane);
            else if (d <= 128) w = wide_row<4>(src, d, dplus, adjp + dst, fits, lane);
            else if (d <= 256) w = wide_row<8>(src, d, dplus, adjp + dst, fits, lane);
            else w = wide_row<16>(src, d, dplus, adjp + dst, fits, lane);
            if (lane == 0) {
                if (!fits) atomicOr(&ctl->st.err_input, 1);
                const uint32_t key = queue_key(d, w);
                qkey[r] = key;
                atomicAdd(&h[key], 1u);
            }
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 256; t += kRowsThreads) {
        const unsigned int c = h[t];
        if (c) atomicAdd(&ctl->qhist[0][t], c);
    }
}

constexpr int kLongCap = 8192;  // kept entries a CTA sorts in shared memory

// Rows of more than kRowsWarp entries: one CTA per row sorts it (in shared
// memory up to kLongCap entries, else in place in tmp), copies it, and sets
// its queue key.
__global__ void __launch_bounds__(kThreads) k_rows_long(const int64_t* __restrict__ off, const int32_t* __restrict__ perm,
                                                       const int32_t* __restrict__ dplus,
                                                       const int64_t* __restrict__ offp, int32_t* __restrict__ tmp,
                                                       int64_t m, int32_t* __restrict__ adjp,
                                                       uint32_t* __restrict__ qkey, const int32_t* __restrict__ longrows,
                                                       int64_t long_cap, Ctl* ctl)
{
    __shared__ int32_t sb[kLongCap];
    __shared__ unsigned int s_row;
    __shared__ unsigned long long s_w;
    const unsigned int nlong = min(ctl->nlong_rows, (unsigned int)long_cap);
    for (;;) {
        if (threadIdx.x == 0) {
            s_row = atomicAdd(&ctl->tickets[15], 1u);
            s_w = 0ull;
        }
        __syncthreads();
        const unsigned int row = s_row;
        if (row >= nlong) break;
        const int32_t r = longrows[row];
        const int len = dplus[r];
        int32_t* seg = tmp + off[perm[r]];
        const int64_t dst = offp[r];
        const bool fits = dst + len <= m;
        int N = 1, lgN = 0;
        while (N < len) { N <<= 1; ++lgN; }
        const bool in_smem = N <= kLongCap;
        unsigned long long w = 0;
        for (int j = threadIdx.x; j < len; j += kThreads) w += (unsigned long long)dplus[seg[j]];
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(kFull, w, o);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(&s_w, w);
        int32_t* s = in_smem ? sb : seg;
        if (in_smem)
            for (int j = threadIdx.x; j < N; j += kThreads) sb[j] = j < len ? seg[j] : INT_MAX;
        __syncthreads();
        const int lim = in_smem ? N : len;  // padded in shared memory; virtual +inf in place
        for (int lsz = 1; lsz <= lgN; ++lsz) {
            bitonic_step(s, N, lim, lsz - 1, true, threadIdx.x, kThreads);
            __syncthreads();
            for (int ls = lsz - 2; ls >= 0; --ls) {
                bitonic_step(s, N, lim, ls, false, threadIdx.x, kThreads);
                __syncthreads();
            }
        }
        if (fits)
            for (int j = threadIdx.x; j < len; j += kThreads) adjp[dst + j] = s[j];
        if (threadIdx.x == 0) {
            if (!fits) atomicOr(&ctl->st.err_input, 1);
            const uint32_t key = queue_key(len, s_w);
            qkey[r] = key;
            atomicAdd(&ctl->qhist[0][key], 1u);
        }
        __syncthreads();
    }
}

// KC_VALIDATE: rows strictly increasing, in range, no self-loop, and every
// (u, v) has its mirror (v, u) (binary search in row v).  Sets *bad on failure.
__global__ void k_validate(const int64_t* __restrict__ off, const int32_t* __restrict__ adj, int32_t n,
                           int64_t m2, int* __restrict__ bad)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < n; u += nwarps) {
        const int64_t b = off[u], e = off[u + 1];
        bool ok = b >= 0 && e >= b && e <= m2;
        if (ok) {
            for (int64_t p = b + lane; p < e; p += 32) {
                int32_t v = adj[p];
                if (v < 0 || v >= n || v == (int32_t)u || (p > b && adj[p - 1] >= v)) { ok = false; break; }
                int64_t lo = off[v], hi = off[v + 1];
                if (lo < 0 || hi < lo || hi > m2) { ok = false; break; }
                while (lo < hi) {
                    int64_t mid = lo + (hi - lo) / 2;
                    if (adj[mid] < (int32_t)u) lo = mid + 1; else hi = mid;
                }
                if (lo >= off[v + 1] || adj[lo] != (int32_t)u) { ok = false; break; }
            }
        }
        if (!__all_sync(kFull, ok) && lane == 0) atomicExch(bad, 1);
    }
}

__global__ void k_zero_offset(int64_t* offp) { offp[0] = 0; }

int grid_for(int64_t work, int per_block, int max_blocks)
{
    int64_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return (int)g;
}

template <typename T>
T* carve(char*& p, int64_t count)
{
    T* r = (T*)p;
    p += ((size_t)std::max<int64_t>(count, 1) * sizeof(T) + 255) & ~(size_t)255;
    return r;
}

template <typename T>
size_t carve_bytes(int64_t count)
{
    return ((size_t)std::max<int64_t>(count, 1) * sizeof(T) + 255) & ~(size_t)255;
}

}  // namespace

int num_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

kc_status orient(const int64_t* off_in, const int32_t* adj_in, int32_t n, int64_t m, unsigned flags,
                 cudaStream_t s, kc_graph** out)
{
    *out = nullptr;
    if (n < 0 || m < 0 || (n == 0 && m != 0)) return KC_EINVAL;
    if (!off_in || (m > 0 && !adj_in)) return KC_EINVAL;
    kc_graph* g = new (std::nothrow) kc_graph();
    if (!g) return KC_ENOMEM;
    KC_CK(cudaGetDevice(&g->device));
    g->n = n;
    g->m = m;
    struct Guard {
        kc_graph* g;
        bool keep = false;
        ~Guard() { if (!keep) kc_free(g); }
    } guard{g};

    const int sms = num_sms();
    const int64_t n1 = (int64_t)n + 1;
    const int64_t m2 = 2 * m;
    const int64_t nn = n > 0 ? n : 1;

    // resident arrays: one pool block
    {
        const size_t bytes = 5 * carve_bytes<int32_t>(nn) + carve_bytes<int64_t>(n1) + carve_bytes<int32_t>(m);
        KC_TRY(pool_alloc(&g->block, bytes, s));
        char* p = (char*)g->block;
        g->rank = carve<int32_t>(p, nn);
        g->perm = carve<int32_t>(p, nn);
        g->deg = carve<int32_t>(p, nn);
        g->dplus = carve<int32_t>(p, nn);
        g->queue = carve<int32_t>(p, nn);
        g->offp = carve<int64_t>(p, n1);
        g->adjp = carve<int32_t>(p, m);
        g->bytes = (int64_t)bytes;
    }
    g->hstats = stats_slot_get();
    if (!g->hstats) return KC_ENOMEM;
    std::memset(g->hstats, 0, sizeof(OrientStats));
    KC_CK(cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming));

    // scratch: input copies (host inputs), sort ping-pong, gathered rows,
    // deferred-row lists, look-back status words, control block
    const int64_t tiles = (nn + kSwTile - 1) / kSwTile;
    const int64_t gather_cap = m2 / (kGatherLong + 1) + 1;  // rows with d > kGatherLong
    const int64_t rows_cap = m / (kRowsWarp + 1) + 1;        // rows with d+ > kRowsWarp
    int deg_bits = 0;  // host bound on the degree bits: d <= min(n - 1, 2m)
    {
        const uint64_t bound = (uint64_t)std::min<int64_t>(n > 0 ? n - 1 : 0, m2);
        while (deg_bits < 32 && (bound >> deg_bits)) ++deg_bits;
    }
    const int deg_launches = (deg_bits + 7) / 8;  // passes actually run: decided on the device
    const int sweeps = deg_launches + 1;
    const bool host_in = !(flags & KC_DEVICE_PTRS);
    const size_t scratch_bytes = (host_in ? carve_bytes<int64_t>(n1) + carve_bytes<int32_t>(m2) : 0) +
                                 2 * carve_bytes<uint32_t>(nn) + 2 * carve_bytes<int32_t>(nn) +
                                 carve_bytes<int32_t>(m2) + carve_bytes<int32_t>(gather_cap) +
                                 carve_bytes<int32_t>(rows_cap) + carve_bytes<int32_t>(nn) +
                                 carve_bytes<unsigned long long>(tiles * 256 * sweeps) +
                                 carve_bytes<unsigned long long>(tiles) + carve_bytes<Ctl>(1) +
                                 carve_bytes<int>(1);
    Scratch sc(s);
    char* sp = nullptr;
    KC_TRY(sc.get(&sp, (int64_t)scratch_bytes));
    const int64_t* off = off_in;
    const int32_t* adj = adj_in;
    if (host_in) {
        int64_t* d_off = carve<int64_t>(sp, n1);
        int32_t* d_adj = carve<int32_t>(sp, m2);
        KC_CK(cudaMemcpyAsync(d_off, off_in, n1 * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        if (m2 > 0) KC_CK(cudaMemcpyAsync(d_adj, adj_in, m2 * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        off = d_off;
        adj = d_adj;
    }
    uint32_t* kA = carve<uint32_t>(sp, nn);
    uint32_t* kB = carve<uint32_t>(sp, nn);
    int32_t* vA = carve<int32_t>(sp, nn);
    int32_t* vB = carve<int32_t>(sp, nn);
    int32_t* tmp = carve<int32_t>(sp, m2);
    int32_t* gather_rows = carve<int32_t>(sp, gather_cap);
    int32_t* sort_rows = carve<int32_t>(sp, rows_cap);
    int32_t* wide_rows = carve<int32_t>(sp, nn);
    unsigned long long* sw_status = carve<unsigned long long>(sp, tiles * 256 * sweeps);
    unsigned long long* sc_status = carve<unsigned long long>(sp, tiles);
    Ctl* ctl = carve<Ctl>(sp, 1);
    int* bad = carve<int>(sp, 1);
    KC_CK(cudaMemsetAsync(sw_status, 0, (size_t)tiles * 256 * sweeps * sizeof(unsigned long long), s));
    KC_CK(cudaMemsetAsync(sc_status, 0, (size_t)tiles * sizeof(unsigned long long), s));
    KC_CK(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));

    if (flags & KC_VALIDATE) {
        int64_t first = 0, last = 0;
        KC_CK(cudaMemcpyAsync(&first, off, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        KC_CK(cudaMemcpyAsync(&last, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        KC_CK(cudaStreamSynchronize(s));
        if (first != 0 || last != m2) return KC_EINVAL;
        int hbad = 0;
        if (n > 0) {
            KC_CK(cudaMemsetAsync(bad, 0, sizeof(int), s));
            k_validate<<<grid_for((int64_t)n * 32, kThreads, sms * 16), kThreads, 0, s>>>(off, adj, n, m2, bad);
            KC_LAUNCHED();
            KC_CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
            KC_CK(cudaStreamSynchronize(s));
        }
        if (hbad) return KC_EINVAL;
    }

    if (n == 0) {
        k_zero_offset<<<1, 1, 0, s>>>(g->offp);
        KC_LAUNCHED();
    } else {
        const int unit_grid = grid_for(((int64_t)n + 31) / 32 * 32, kThreads, sms * 8);
        // a1, a2: degrees, sort by degree (stable: ties in id order)
        k_degree<<<grid_for(n, kThreads, sms * 2), kThreads, 0, s>>>(off, n, kA, ctl);
        KC_LAUNCHED();
        for (int p = 0; p < deg_launches; ++p) {
            SweepArgs a;
            a.kin = (p & 1) ? kB : kA;
            a.vin = p == 0 ? nullptr : ((p & 1) ? vB : vA);
            a.kout = (p & 1) ? kA : kB;
            a.vout = (p & 1) ? vA : vB;
            a.n = n;
            a.shift = 8 * p;
            a.hist = ctl->dhist[p];
            a.status = sw_status + (int64_t)p * tiles * 256;
            a.ticket = &ctl->tickets[1 + p];
            a.max_deg = &ctl->st.max_deg;
            a.pass = p;
            a.err = &ctl->st.err_timeout;
            k_sweep<<<(unsigned)tiles, kThreads, 0, s>>>(a);
            KC_LAUNCHED();
        }
        k_rank<<<grid_for(n, kThreads, sms * 8), kThreads, 0, s>>>(ctl, deg_launches, kA, vA, kB, vB, n, g->perm,
                                                                    g->rank, g->deg);
        KC_LAUNCHED();

        // a3, a4: Gamma+ rows (the one gather pass), offsets, rows in rank order
        k_gamma<<<unit_grid, kThreads, 0, s>>>(off, adj, g->rank, n, tmp, g->dplus, gather_rows, gather_cap, ctl);
        KC_LAUNCHED();
        k_gamma_long<<<sms * 8, kThreads, 0, s>>>(off, adj, g->rank, gather_rows, gather_cap, tmp, g->dplus, ctl);
        KC_LAUNCHED();
        k_offsets<<<(unsigned)((n + kScTile - 1) / kScTile), kThreads, 0, s>>>(g->dplus, n, m, g->offp, sc_status,
                                                                             ctl);
        KC_LAUNCHED();
        k_rows<<<grid_for(((int64_t)n + 31) / 32 * 32, kRowsThreads, sms * 8), kRowsThreads, 0, s>>>(
            off, g->perm, g->dplus, g->offp, tmp, n, m, g->adjp, kA, wide_rows, sort_rows, rows_cap, ctl);
        KC_LAUNCHED();
        k_rows_wide<<<sms * 16, kRowsThreads, 0, s>>>(off, g->perm, g->dplus, g->offp, tmp, m, g->adjp, kA, wide_rows,
                                                     ctl);
        KC_LAUNCHED();
        k_rows_long<<<sms * 2, kThreads, 0, s>>>(off, g->perm, g->dplus, g->offp, tmp, m, g->adjp, kA, sort_rows,
                                                 rows_cap, ctl);
        KC_LAUNCHED();

        // a5: owner queue (one pass on the 8-bit key; stable, so ties by rank)
        {
            SweepArgs a;
            a.kin = kA;
            a.vin = nullptr;
            a.kout = nullptr;
            a.vout = g->queue;
            a.n = n;
            a.shift = 0;
            a.hist = ctl->qhist[0];
            a.status = sw_status + (int64_t)deg_launches * tiles * 256;
            a.ticket = &ctl->tickets[8];
            a.max_deg = nullptr;
            a.pass = 0;
            a.err = &ctl->st.err_timeout;
            k_sweep<<<(unsigned)tiles, kThreads, 0, s>>>(a);
            KC_LAUNCHED();
        }
    }
    KC_CK(cudaMemcpyAsync(g->hstats, &ctl->st, sizeof(OrientStats), cudaMemcpyDeviceToHost, s));
    KC_CK(cudaEventRecord(g->done, s));
    guard.keep = true;
    *out = g;
    return KC_OK;
}

}  // namespace kc
