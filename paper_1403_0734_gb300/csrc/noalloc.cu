// noalloc.cu -- kc_count_static: the exact count of kc_count without any
// device memory allocation.
//
// Who needs it.  kc_count takes its scratch (the 128-bit total, the owner-class
// cursors and, for owners wider than the shared-memory limit, global bitmap
// tiles) from cudaMallocAsync.  Some callers cannot allocate at the moment they
// want a count: a serving process whose memory manager has already reserved
// the device for its own pool and accounts for every byte in advance (a
// surprise cudaMalloc would fail or break that accounting), and
// latency-critical code that must not pay for, or be serialised behind, an
// allocation call.  This entry point takes the same scratch from one
// file-scope __device__ array instead.
//
// Cost and limits.  The array is kStaticScratchBytes (16 MiB); every GPU on
// which the library is loaded holds it until the process exits.  The global
// tiles of wide owners are carved from it (as many concurrent tiles as fit);
// a graph whose single widest owner needs a tile larger than the array is
// rejected with KC_ENOTSUP before anything runs.  Per-vertex and per-owner
// outputs are not offered (they would need n-sized scratch).
//
// Sharing.  All calls in the process share the one array per device, and it
// keeps whatever the last call left in it; each call clears the words that
// must start at zero (total and cursors) on its stream before its kernels run.
// Calls whose work overlaps on the GPU (different streams, or different host
// threads) race on the array and give wrong counts: serialise them.
//
// Set-up.  The device address of the array is looked up with
// cudaGetSymbolAddress on the first call on each device (with that device
// current) and cached; the array's name in host code is only a host-side
// stand-in and is never passed to a kernel.  Under lazy module loading (the
// CUDA default) that first call is also when the module holding the array is
// loaded and its 16 MiB are committed on the device: a caller that must not
// allocate later makes one warm-up call (any graph, k = 3) at start-up,
// before its memory manager reserves the device and before any stream
// capture is started.
#include <mutex>

#include "kc_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB per device
constexpr size_t kSmallBytes = 256;                      // total + cursors
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_dev_ptr[kMaxDevices] = {};

// q_1 or q_2 into the first two words of the static array (low, high).
__global__ void k_set_total(unsigned long long* t, unsigned long long q)
{
    t[0] = q;
    t[1] = 0ull;
}

// Device address of g_static_scratch on `dev` (which must be current).
kc_status scratch_address(int dev, void** out)
{
    if (dev < 0 || dev >= kMaxDevices) return KC_ENOTSUP;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            kc::set_cuda_error(e, "cudaGetSymbolAddress(g_static_scratch)");
            return KC_ECUDA;
        }
        g_dev_ptr[dev] = p;
    }
    *out = g_dev_ptr[dev];
    return KC_OK;
}

}  // namespace

extern "C" kc_status kc_count_static(const kc_graph* g, int k, unsigned flags, uint64_t* total, void* stream)
{
    if (!g || !total || k < 1 || k > KC_MAX_K) return KC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const bool dev_out = (flags & KC_DEVICE_PTRS) != 0;
    int prev = -1;
    KC_CK(cudaGetDevice(&prev));
    if (prev != g->device) KC_CK(cudaSetDevice(g->device));
    struct Restore {
        int prev, dev;
        ~Restore() { if (prev >= 0 && prev != dev) cudaSetDevice(prev); }
    } restore{prev, g->device};
    KC_TRY(kc::ready(g));

    const unsigned long long q12 = k == 1 ? (unsigned long long)g->n : (unsigned long long)g->m;
    if (k <= 2 && !dev_out) {  // q_1 = n, q_2 = m: nothing runs on the device
        *total = q12;
        return KC_OK;
    }

    void* base = nullptr;
    KC_TRY(scratch_address(g->device, &base));
    if (k <= 2) {  // device output: written on the stream, asynchronously like every device output
        k_set_total<<<1, 1, 0, s>>>((unsigned long long*)base, q12);
        KC_LAUNCHED();
        KC_CK(cudaMemcpyAsync(total, base, 2 * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        return KC_OK;
    }
    unsigned long long* small = (unsigned long long*)base;  // [0..1] total, [2..15] cursors
    uint32_t* tiles = (uint32_t*)((char*)base + kSmallBytes);
    const int64_t tile_words = (int64_t)((kStaticScratchBytes - kSmallBytes) / sizeof(uint32_t));

    int64_t per_slot = 0;
    // exact k = 3 takes the triangle path (no bitmaps, no tiles) when it is on
    const int64_t need = (k == 3 && kc::tri_enabled()) ? 0 : kc::heavy_scratch_words(g, k, &per_slot);
    int64_t use_words = 0;
    if (need > 0) {
        if (per_slot > tile_words) return KC_ENOTSUP;  // widest owner does not fit the static array
        use_words = need < tile_words ? need : (tile_words / per_slot) * per_slot;
    }

    KC_CK(cudaMemsetAsync(small, 0, kSmallBytes, s));
    if (g->n > 0) {
        kc::CountArgs a;
        a.k = k;
        a.colours = 0;
        a.seed = 0;
        a.per_vertex = false;
        a.total = small;
        a.pv = nullptr;
        a.po = nullptr;
        a.work = nullptr;
        a.sc = nullptr;  // no allocator: every owner is searched by one CTA (no split tiles)
        KC_TRY(kc::count_launch(g, a, small + 2, need > 0 ? tiles : nullptr, use_words, s));
    }
    if (dev_out) {
        KC_CK(cudaMemcpyAsync(total, small, 2 * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        return KC_OK;
    }
    unsigned long long th[2] = {0, 0};
    KC_CK(cudaMemcpyAsync(th, small, sizeof(th), cudaMemcpyDeviceToHost, s));
    KC_CK(cudaStreamSynchronize(s));
    *total = th[0];
    return th[1] ? KC_EOVERFLOW : KC_OK;
}
