// prims.cu -- device-wide exclusive scan and stable LSD radix sort (pairs).
//
// Both are small, HBM-streaming helpers for the orientation step: the scan
// turns |Gamma+| counts into CSR offsets, the radix sort ranks vertices by
// degree (stable, so ties keep id order -- exactly the (degree, id) order of
// Sec. 2) and orders the owner queue by |Gamma+|.
#include "kc_internal.cuh"

namespace kc {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread (256 threads); returns the
// exclusive prefix and writes the block total to *total.
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* total)
{
    __shared__ int64_t s_warp[kScanThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t inc = warp_incl_scan(v, lane);
    if (lane == 31) s_warp[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int64_t w = lane < kScanThreads / 32 ? s_warp[lane] : 0;
        int64_t wi = warp_incl_scan(w, lane);
        if (lane < kScanThreads / 32) s_warp[lane] = wi - w;  // exclusive
        if (lane == kScanThreads / 32 - 1) *total = wi;
    }
    __syncthreads();
    int64_t r = s_warp[wid] + inc - v;
    __syncthreads();
    return r;
}

template <typename Tin>
__global__ void __launch_bounds__(kScanThreads) k_scan_tile_sums(const Tin* __restrict__ in, int64_t n,
                                                                int64_t* __restrict__ sums)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
    for (int j = threadIdx.x; j < kScanTile; j += kScanThreads) {
        int64_t i = base + j;
        if (i < n) s += (int64_t)in[i];
    }
    __shared__ int64_t tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <typename Tin>
__global__ void __launch_bounds__(kScanThreads) k_scan_tile_apply(const Tin* __restrict__ in, int64_t n,
                                                                 const int64_t* __restrict__ offs,
                                                                 int64_t* __restrict__ out)
{
    __shared__ int64_t tile[kScanTile + kScanTile / 32];  // padded: index j + j/32
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    for (int j = threadIdx.x; j < kScanTile; j += kScanThreads) {
        int64_t i = base + j;
        tile[j + (j >> 5)] = i < n ? (int64_t)in[i] : 0;
    }
    __syncthreads();
    int64_t loc[kScanItems];
    int64_t sum = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        int j = threadIdx.x * kScanItems + q;
        loc[q] = tile[j + (j >> 5)];
        sum += loc[q];
    }
    __shared__ int64_t tot;
    int64_t pre = block_excl_scan(sum, &tot);
    const int64_t off = offs ? offs[blockIdx.x] : 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        int j = threadIdx.x * kScanItems + q;
        tile[j + (j >> 5)] = pre;
        pre += loc[q];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < kScanTile; j += kScanThreads) {
        int64_t i = base + j;
        if (i < n) out[i] = tile[j + (j >> 5)] + off;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = off + tot;
}

template <typename Tin>
kc_status scan_impl(const Tin* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s)
{
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb <= 1) {
        k_scan_tile_apply<Tin><<<1, kScanThreads, 0, s>>>(in, n, nullptr, out);
        KC_LAUNCHED();
        return KC_OK;
    }
    int64_t* sums = tmp;
    int64_t* sums_scan = tmp + nb;
    k_scan_tile_sums<Tin><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums);
    KC_LAUNCHED();
    KC_TRY(scan_impl<int64_t>(sums, sums_scan, nb, tmp + 2 * nb + 1, s));
    k_scan_tile_apply<Tin><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums_scan, out);
    KC_LAUNCHED();
    return KC_OK;
}

// ------------------------------------------------------------ radix sort

constexpr int kRsThreads = 256;
constexpr int kRsChunks = 8;
constexpr int kRsTile = kRsThreads * kRsChunks;  // 2048 items per block
constexpr int kRsWarps = kRsThreads / 32;

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint32_t* __restrict__ keys, int64_t n,
                                                       int shift, int64_t ntiles,
                                                       int32_t* __restrict__ hist)
{
    __shared__ int32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int j = threadIdx.x; j < kRsTile; j += kRsThreads) {
        int64_t i = base + j;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint32_t* __restrict__ keys,
                                                          const int32_t* __restrict__ vals, int64_t n,
                                                          int shift, int64_t ntiles,
                                                          const int64_t* __restrict__ hscan,
                                                          uint32_t* __restrict__ keys_out,
                                                          int32_t* __restrict__ vals_out)
{
    __shared__ int64_t base[256];
    __shared__ int64_t wc[kRsWarps][256];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    base[tid] = hscan[(int64_t)tid * ntiles + blockIdx.x];
    for (int j = tid; j < kRsWarps * 256; j += kRsThreads) (&wc[0][0])[j] = 0;
    __syncthreads();
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int64_t tbase = (int64_t)blockIdx.x * kRsTile;
    for (int c = 0; c < kRsChunks; ++c) {
        const int64_t i = tbase + (int64_t)c * kRsThreads + tid;
        const bool valid = i < n;
        uint32_t key = valid ? keys[i] : 0u;
        int32_t val = valid ? vals[i] : 0;
        uint32_t dig = valid ? ((key >> shift) & 255u) : (256u + (uint32_t)lane);
        uint32_t peers = __match_any_sync(kFull, dig);
        int lower = __popc(peers & lt_mask);
        if (valid && lower == 0) wc[wid][dig] = __popc(peers);
        __syncthreads();
        {
            int64_t run = base[tid];
#pragma unroll
            for (int w = 0; w < kRsWarps; ++w) {
                int64_t t = wc[w][tid];
                wc[w][tid] = run;
                run += t;
            }
            base[tid] = run;
        }
        __syncthreads();
        if (valid) {
            int64_t pos = wc[wid][dig] + lower;
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
        for (int j = tid; j < kRsWarps * 256; j += kRsThreads) (&wc[0][0])[j] = 0;
        __syncthreads();
    }
}

}  // namespace

size_t scan_tmp_elems(int64_t n)
{
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb <= 1) return 1;
    return (size_t)(2 * nb + 1) + scan_tmp_elems(nb);
}

kc_status scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s)
{
    return scan_impl<int32_t>(in, out, n, tmp, s);
}

int64_t radix_hist_elems(int64_t n)
{
    int64_t ntiles = (n + kRsTile - 1) / kRsTile;
    if (ntiles < 1) ntiles = 1;
    return 256 * ntiles;
}

kc_status radix_sort_pairs(uint32_t** keys, int32_t** vals, uint32_t* keys_alt, int32_t* vals_alt,
                           int64_t n, int bits, int32_t* hist, int64_t* hist_scan, int64_t* tmp,
                           cudaStream_t s)
{
    if (n <= 1 || bits <= 0) return KC_OK;
    const int64_t ntiles = (n + kRsTile - 1) / kRsTile;
    uint32_t* k_in = *keys;
    int32_t* v_in = *vals;
    uint32_t* k_out = keys_alt;
    int32_t* v_out = vals_alt;
    for (int shift = 0; shift < bits; shift += 8) {
        k_rs_hist<<<(unsigned)ntiles, kRsThreads, 0, s>>>(k_in, n, shift, ntiles, hist);
        KC_LAUNCHED();
        KC_TRY(scan_impl<int32_t>(hist, hist_scan, 256 * ntiles, tmp, s));
        k_rs_scatter<<<(unsigned)ntiles, kRsThreads, 0, s>>>(k_in, v_in, n, shift, ntiles, hist_scan,
                                                            k_out, v_out);
        KC_LAUNCHED();
        uint32_t* tk = k_in; k_in = k_out; k_out = tk;
        int32_t* tv = v_in; v_in = v_out; v_out = tv;
    }
    *keys = k_in;
    *vals = v_in;
    return KC_OK;
}

}  // namespace kc
