// orient.cu -- Round 1 of Algorithm 1 (Sec. 3) on the device.
//
//   a1  d(v) = off[v+1] - off[v]                                   (Sec. 2)
//   a2  rank: stable radix sort of the vertices by degree; ties keep id
//       order, so rank follows x < y iff d(x) < d(y) or d(x) = d(y), x < y
//   a3  |Gamma+(u)| = #{v in Gamma(u) : rank v > rank u}, scan -> offsets
//   a4  Gamma+(u) gathered into rank space and sorted ascending (= in the
//       order), one warp per short row, one CTA per long row (bitonic)
//   a5  owner queue: ranks by |Gamma+| descending (the Reduce 1 filter
//       |Gamma+(u)| >= k-1 becomes a prefix of this queue for every k)
//
// All steps stream the CSR once or twice; the rank array (4n bytes) is the
// only random-access structure and stays in L2.
#include <algorithm>
#include <climits>
#include <vector>

#include "kc_internal.cuh"

namespace kc {
namespace {

constexpr int kThreads = 256;

__global__ void k_degree(const int64_t* __restrict__ off, int32_t n, uint32_t* __restrict__ deg,
                         int32_t* __restrict__ ids, unsigned int* __restrict__ maxdeg)
{
    unsigned int mx = 0;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint32_t d = (uint32_t)(off[v + 1] - off[v]);
        deg[v] = d;
        ids[v] = v;
        mx = max(mx, d);
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(maxdeg, mx);
}

__global__ void k_rank_from_perm(const int32_t* __restrict__ perm, const uint32_t* __restrict__ sdeg,
                                 int32_t n, int32_t* __restrict__ rank, int32_t* __restrict__ deg_r)
{
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        rank[perm[r]] = r;
        deg_r[r] = (int32_t)sdeg[r];
    }
}

// a3: one warp per vertex (original id), lanes stride its row.
__global__ void k_orient_count(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                               const int32_t* __restrict__ rank, int32_t n,
                               int32_t* __restrict__ dplus)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        const int32_t rv = rank[v];
        const int64_t b = off[v], e = off[v + 1];
        int cnt = 0;
        for (int64_t p = b + lane; p < e; p += 32) cnt += rank[adj[p]] > rv;
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
        if (lane == 0) dplus[rv] = cnt;
    }
}

// Statistics: max d+ and sum C(d+, 2); histogram of d+ for the queue classes.
__global__ void k_dplus_stats(const int32_t* __restrict__ dplus, int32_t n,
                              unsigned int* __restrict__ maxd, unsigned long long* __restrict__ wedges,
                              uint32_t* __restrict__ qkey, int32_t* __restrict__ qval)
{
    unsigned int mx = 0;
    unsigned long long w = 0;
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        uint32_t d = (uint32_t)dplus[r];
        mx = max(mx, d);
        w += (unsigned long long)d * (d - (d > 0)) / 2;
        qval[r] = r;
        qkey[r] = d;
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(kFull, mx, o));
        w += __shfl_xor_sync(kFull, w, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (mx) atomicMax(maxd, mx);
        if (w) atomicAdd(wedges, w);
    }
}

// queue sort key: descending d+ -> ascending (maxd - d+)
__global__ void k_queue_keys(uint32_t* __restrict__ qkey, int32_t n, uint32_t maxd,
                             int32_t* __restrict__ hist)
{
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        uint32_t d = qkey[r];
        atomicAdd(&hist[d], 1);
        qkey[r] = maxd - d;
    }
}

// Mirrored bitonic sort of 32 values held one per lane (ascending).
__device__ __forceinline__ int32_t warp_sort32(int32_t v, int lane)
{
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
        int p = lane ^ (size - 1);
        int32_t o = __shfl_sync(kFull, v, p);
        v = (lane < p) ? min(v, o) : max(v, o);
#pragma unroll
        for (int stride = size >> 2; stride > 0; stride >>= 1) {
            p = lane ^ stride;
            o = __shfl_sync(kFull, v, p);
            v = (lane < p) ? min(v, o) : max(v, o);
        }
    }
    return v;
}

// a4, short rows (1 <= d+ <= 32): one warp per owner from the queue range.
__global__ void k_fill_warp(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                            const int32_t* __restrict__ rank, const int32_t* __restrict__ perm,
                            const int32_t* __restrict__ queue, int64_t q0, int64_t q1,
                            const int64_t* __restrict__ offp, int32_t* __restrict__ adjp)
{
    __shared__ int32_t buf[kThreads / 32][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    for (int64_t q = q0 + warp; q < q1; q += nwarps) {
        const int32_t r = queue[q];
        const int32_t v = perm[r];
        const int64_t b = off[v], e = off[v + 1];
        int cnt = 0;
        for (int64_t p0 = b; p0 < e; p0 += 32) {
            int64_t p = p0 + lane;
            int32_t rb = p < e ? rank[adj[p]] : INT_MIN;
            bool keep = rb > r;
            uint32_t bal = __ballot_sync(kFull, keep);
            if (keep) buf[wid][cnt + __popc(bal & lt)] = rb;
            cnt += __popc(bal);
        }
        __syncwarp();
        int32_t x = lane < cnt ? buf[wid][lane] : INT_MAX;
        __syncwarp();
        x = warp_sort32(x, lane);
        if (lane < cnt) adjp[offp[r] + lane] = x;
    }
}

// a4, long rows (32 < d+ <= cap): one CTA per owner, bitonic sort in shared
// memory over the next power of two (padding +inf).
__global__ void __launch_bounds__(kThreads) k_fill_block(
    const int64_t* __restrict__ off, const int32_t* __restrict__ adj, const int32_t* __restrict__ rank,
    const int32_t* __restrict__ perm, const int32_t* __restrict__ queue, int64_t q0, int64_t q1,
    const int64_t* __restrict__ offp, int32_t* __restrict__ adjp, int cap)
{
    extern __shared__ int32_t sbuf[];
    __shared__ int s_cnt;
    for (int64_t q = q0 + blockIdx.x; q < q1; q += gridDim.x) {
        const int32_t r = queue[q];
        const int32_t v = perm[r];
        const int64_t b = off[v], e = off[v + 1];
        const int len = (int)(offp[r + 1] - offp[r]);
        int N = 64;
        while (N < len) N <<= 1;
        if (threadIdx.x == 0) s_cnt = 0;
        for (int j = threadIdx.x; j < N; j += blockDim.x) sbuf[j] = INT_MAX;
        __syncthreads();
        for (int64_t p = b + threadIdx.x; p < e; p += blockDim.x) {
            int32_t rb = rank[adj[p]];
            if (rb > r) sbuf[atomicAdd(&s_cnt, 1)] = rb;
        }
        __syncthreads();
        for (int size = 2; size <= N; size <<= 1) {
            const int half = size >> 1;
            for (int i = threadIdx.x; i < N / 2; i += blockDim.x) {
                int lo = (i / half) * size + (i % half);
                int hi = (i / half) * size + size - 1 - (i % half);
                int32_t a = sbuf[lo], c = sbuf[hi];
                if (c < a) { sbuf[lo] = c; sbuf[hi] = a; }
            }
            __syncthreads();
            for (int stride = size >> 2; stride > 0; stride >>= 1) {
                for (int i = threadIdx.x; i < N / 2; i += blockDim.x) {
                    int lo = (i / stride) * stride * 2 + (i % stride);
                    int hi = lo + stride;
                    int32_t a = sbuf[lo], c = sbuf[hi];
                    if (c < a) { sbuf[lo] = c; sbuf[hi] = a; }
                }
                __syncthreads();
            }
        }
        for (int j = threadIdx.x; j < len; j += blockDim.x) adjp[offp[r] + j] = sbuf[j];
        __syncthreads();
        (void)cap;
    }
}

// a4, very long rows (d+ > shared-memory cap): gather unsorted into the
// output segment, then the same mirrored bitonic network in place in global
// memory (pairs whose upper index is past the row end compare against a
// virtual +inf and are skipped).
__global__ void __launch_bounds__(kThreads) k_fill_global(
    const int64_t* __restrict__ off, const int32_t* __restrict__ adj, const int32_t* __restrict__ rank,
    const int32_t* __restrict__ perm, const int32_t* __restrict__ queue, int64_t q0, int64_t q1,
    const int64_t* __restrict__ offp, int32_t* __restrict__ adjp)
{
    __shared__ int s_cnt;
    for (int64_t q = q0 + blockIdx.x; q < q1; q += gridDim.x) {
        const int32_t r = queue[q];
        const int32_t v = perm[r];
        const int64_t b = off[v], e = off[v + 1];
        int32_t* seg = adjp + offp[r];
        const int len = (int)(offp[r + 1] - offp[r]);
        int N = 1;
        while (N < len) N <<= 1;
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        for (int64_t p = b + threadIdx.x; p < e; p += blockDim.x) {
            int32_t rb = rank[adj[p]];
            if (rb > r) seg[atomicAdd(&s_cnt, 1)] = rb;
        }
        __syncthreads();
        for (int size = 2; size <= N; size <<= 1) {
            const int half = size >> 1;
            for (int i = threadIdx.x; i < N / 2; i += blockDim.x) {
                int lo = (i / half) * size + (i % half);
                int hi = (i / half) * size + size - 1 - (i % half);
                if (hi < len) {
                    int32_t a = seg[lo], c = seg[hi];
                    if (c < a) { seg[lo] = c; seg[hi] = a; }
                }
            }
            __syncthreads();
            for (int stride = size >> 2; stride > 0; stride >>= 1) {
                for (int i = threadIdx.x; i < N / 2; i += blockDim.x) {
                    int lo = (i / stride) * stride * 2 + (i % stride);
                    int hi = lo + stride;
                    if (hi < len) {
                        int32_t a = seg[lo], c = seg[hi];
                        if (c < a) { seg[lo] = c; seg[hi] = a; }
                    }
                }
                __syncthreads();
            }
        }
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

int grid_for(int64_t work, int per_block, int max_blocks)
{
    int64_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return (int)g;
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};

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

    // device copies of the input CSR (when given host pointers)
    DevBuf d_off_buf, d_adj_buf;
    const int64_t* off = off_in;
    const int32_t* adj = adj_in;
    if (!(flags & KC_DEVICE_PTRS)) {
        KC_CK(cudaMalloc(&d_off_buf.p, n1 * sizeof(int64_t)));
        KC_CK(cudaMemcpyAsync(d_off_buf.p, off_in, n1 * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        if (m2 > 0) {
            KC_CK(cudaMalloc(&d_adj_buf.p, m2 * sizeof(int32_t)));
            KC_CK(cudaMemcpyAsync(d_adj_buf.p, adj_in, m2 * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        }
        off = (const int64_t*)d_off_buf.p;
        adj = (const int32_t*)d_adj_buf.p;
    }

    // scratch: keys/vals ping-pong (2 x n each), histograms, scan temp
    const int64_t nn = n > 0 ? n : 1;
    const int64_t hist_elems = radix_hist_elems(nn);
    const size_t scan_elems = std::max(scan_tmp_elems(hist_elems), scan_tmp_elems(nn + 1)) + 16;
    DevBuf scratch;
    const size_t scratch_bytes = 4 * nn * sizeof(uint32_t) + hist_elems * sizeof(int32_t) +
                                 (hist_elems + 1) * sizeof(int64_t) + scan_elems * sizeof(int64_t) +
                                 64 * sizeof(unsigned long long);
    KC_CK(cudaMalloc(&scratch.p, scratch_bytes));
    char* sp = (char*)scratch.p;
    uint32_t* keyA = (uint32_t*)sp; sp += nn * sizeof(uint32_t);
    int32_t* valA = (int32_t*)sp;   sp += nn * sizeof(int32_t);
    uint32_t* keyB = (uint32_t*)sp; sp += nn * sizeof(uint32_t);
    int32_t* valB = (int32_t*)sp;   sp += nn * sizeof(int32_t);
    int32_t* hist = (int32_t*)sp;   sp += hist_elems * sizeof(int32_t);
    int64_t* hscan = (int64_t*)sp;  sp += (hist_elems + 1) * sizeof(int64_t);
    int64_t* stmp = (int64_t*)sp;   sp += scan_elems * sizeof(int64_t);
    unsigned long long* stats = (unsigned long long*)sp;  // [0] maxdeg, [1] maxd+, [2] wedges, [3] bad
    KC_CK(cudaMemsetAsync(stats, 0, 64 * sizeof(unsigned long long), s));

    // resident graph arrays
    KC_CK(cudaMalloc(&g->rank, nn * sizeof(int32_t)));
    KC_CK(cudaMalloc(&g->perm, nn * sizeof(int32_t)));
    KC_CK(cudaMalloc(&g->deg, nn * sizeof(int32_t)));
    KC_CK(cudaMalloc(&g->dplus, nn * sizeof(int32_t)));
    KC_CK(cudaMalloc(&g->queue, nn * sizeof(int32_t)));
    KC_CK(cudaMalloc(&g->offp, n1 * sizeof(int64_t)));
    KC_CK(cudaMalloc(&g->adjp, (m > 0 ? m : 1) * sizeof(int32_t)));
    g->bytes = (int64_t)(5 * nn * sizeof(int32_t) + n1 * sizeof(int64_t) + (m > 0 ? m : 1) * sizeof(int32_t));

    if (flags & KC_VALIDATE) {
        int64_t first = 0, last = 0;
        KC_CK(cudaMemcpyAsync(&first, off, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        KC_CK(cudaMemcpyAsync(&last, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        KC_CK(cudaStreamSynchronize(s));
        if (first != 0 || last != m2) return KC_EINVAL;
        if (n > 0) {
            k_validate<<<grid_for((int64_t)n * 32, kThreads, sms * 16), kThreads, 0, s>>>(off, adj, n, m2,
                                                                                      (int*)(stats + 3));
            KC_LAUNCHED();
        }
        unsigned long long bad = 0;
        KC_CK(cudaMemcpyAsync(&bad, stats + 3, sizeof(bad), cudaMemcpyDeviceToHost, s));
        KC_CK(cudaStreamSynchronize(s));
        if (bad) return KC_EINVAL;
    }

    if (n == 0) {
        KC_CK(cudaMemsetAsync(g->offp, 0, sizeof(int64_t), s));
        KC_CK(cudaStreamSynchronize(s));
        g->ge.assign(2, 0);
        guard.keep = true;
        *out = g;
        return KC_OK;
    }

    // a1: degrees
    k_degree<<<grid_for(n, kThreads, sms * 8), kThreads, 0, s>>>(off, n, keyA, valA, (unsigned int*)stats);
    KC_LAUNCHED();
    unsigned int maxdeg = 0;
    KC_CK(cudaMemcpyAsync(&maxdeg, stats, sizeof(maxdeg), cudaMemcpyDeviceToHost, s));
    KC_CK(cudaStreamSynchronize(s));
    int bits = 0;
    while (bits < 32 && (maxdeg >> bits)) ++bits;

    // a2: stable sort by degree -> perm; rank = inverse
    uint32_t* kk = keyA;
    int32_t* vv = valA;
    KC_TRY(radix_sort_pairs(&kk, &vv, keyB, valB, n, bits, hist, hscan, stmp, s));
    KC_CK(cudaMemcpyAsync(g->perm, vv, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    k_rank_from_perm<<<grid_for(n, kThreads, sms * 8), kThreads, 0, s>>>(g->perm, kk, n, g->rank, g->deg);
    KC_LAUNCHED();

    // a3: |Gamma+| per rank, offsets
    k_orient_count<<<grid_for((int64_t)n * 32, kThreads, sms * 16), kThreads, 0, s>>>(off, adj, g->rank, n,
                                                                                   g->dplus);
    KC_LAUNCHED();
    KC_TRY(scan_i32_to_i64(g->dplus, g->offp, n, stmp, s));

    // statistics + queue keys
    k_dplus_stats<<<grid_for(n, kThreads, sms * 8), kThreads, 0, s>>>(g->dplus, n, (unsigned int*)(stats + 1),
                                                                     stats + 2, keyA, valA);
    KC_LAUNCHED();
    unsigned long long st[3] = {0, 0, 0};
    KC_CK(cudaMemcpyAsync(st, stats, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    KC_CK(cudaStreamSynchronize(s));
    g->max_dplus = (int32_t)(uint32_t)st[1];
    g->wedges = (int64_t)st[2];
    const uint32_t maxd = (uint32_t)g->max_dplus;

    // a5: queue by d+ descending (stable: ties by rank)
    int32_t* dhist = hist;  // reuse: max_dplus+1 counters (hist has >= 256 entries; grow if needed)
    DevBuf dhist_buf;
    if ((int64_t)maxd + 1 > hist_elems) {
        KC_CK(cudaMalloc(&dhist_buf.p, ((int64_t)maxd + 1) * sizeof(int32_t)));
        dhist = (int32_t*)dhist_buf.p;
    }
    KC_CK(cudaMemsetAsync(dhist, 0, ((int64_t)maxd + 1) * sizeof(int32_t), s));
    k_queue_keys<<<grid_for(n, kThreads, sms * 8), kThreads, 0, s>>>(keyA, n, maxd, dhist);
    KC_LAUNCHED();
    std::vector<int32_t> h_hist((size_t)maxd + 1);
    KC_CK(cudaMemcpyAsync(h_hist.data(), dhist, ((int64_t)maxd + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    KC_CK(cudaStreamSynchronize(s));
    int qbits = 0;
    while (qbits < 32 && (maxd >> qbits)) ++qbits;
    kk = keyA;
    vv = valA;
    KC_TRY(radix_sort_pairs(&kk, &vv, keyB, valB, n, qbits, hist, hscan, stmp, s));
    KC_CK(cudaMemcpyAsync(g->queue, vv, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    g->ge.assign((size_t)maxd + 2, 0);
    {
        int64_t acc = 0;
        for (int64_t t = maxd; t >= 0; --t) {
            acc += h_hist[(size_t)t];
            g->ge[(size_t)t] = acc;
        }
    }
    auto ge_at = [&](int64_t t) -> int64_t { return t <= (int64_t)maxd ? g->ge[(size_t)(t < 0 ? 0 : t)] : 0; };

    // a4: fill + sort Gamma+ rows, by class (queue is sorted by d+ descending)
    const int kBlockCap = 8192;  // 32 KB of shared memory per row
    {
        int64_t q0 = ge_at(33), q1 = ge_at(1);
        if (q1 > q0) {
            k_fill_warp<<<grid_for((q1 - q0) * 32, kThreads, sms * 16), kThreads, 0, s>>>(
                off, adj, g->rank, g->perm, g->queue, q0, q1, g->offp, g->adjp);
            KC_LAUNCHED();
        }
        q0 = ge_at(kBlockCap + 1);
        q1 = ge_at(33);
        if (q1 > q0) {
            k_fill_block<<<grid_for(q1 - q0, 1, sms * 8), kThreads, kBlockCap * sizeof(int32_t), s>>>(
                off, adj, g->rank, g->perm, g->queue, q0, q1, g->offp, g->adjp, kBlockCap);
            KC_LAUNCHED();
        }
        q0 = 0;
        q1 = ge_at(kBlockCap + 1);
        if (q1 > q0) {
            k_fill_global<<<grid_for(q1 - q0, 1, sms * 4), kThreads, 0, s>>>(off, adj, g->rank, g->perm,
                                                                          g->queue, q0, q1, g->offp, g->adjp);
            KC_LAUNCHED();
        }
    }
    KC_CK(cudaStreamSynchronize(s));
    guard.keep = true;
    *out = g;
    return KC_OK;
}

}  // namespace kc
