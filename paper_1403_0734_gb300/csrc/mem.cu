// mem.cu -- device memory pool, pinned statistics slots, and the wait for an
// orientation's host statistics.
#include <cstring>
#include <mutex>
#include <vector>

#include "kc_internal.cuh"

namespace kc {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};

// The library's pool on `dev`: device memory, never trimmed at
// synchronisation points (release threshold = max), so the orientation's and
// the counts' scratch is reused from call to call without cudaMalloc.
kc_status pool_of(int dev, cudaMemPool_t* out)
{
    if (dev < 0 || dev >= kMaxDevices) return KC_ENOTSUP;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        KC_CK(cudaMemPoolCreate(&p, &props));
        uint64_t thr = ~0ull;
        KC_CK(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr));
        g_pool[dev] = p;
    }
    *out = g_pool[dev];
    return KC_OK;
}

// Pinned statistics slots, allocated in chunks and recycled.
std::mutex g_slot_mu;
std::vector<OrientStats*> g_free_slots;
constexpr int kSlotsPerChunk = 1024;

}  // namespace

kc_status pool_alloc(void** p, size_t bytes, cudaStream_t s)
{
    int dev = 0;
    KC_CK(cudaGetDevice(&dev));
    cudaMemPool_t pool = nullptr;
    KC_TRY(pool_of(dev, &pool));
    KC_CK(cudaMallocFromPoolAsync(p, bytes > 0 ? bytes : 1, pool, s));
    return KC_OK;
}

void pool_free(void* p, cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
}

OrientStats* stats_slot_get()
{
    std::lock_guard<std::mutex> lock(g_slot_mu);
    if (g_free_slots.empty()) {
        void* chunk = nullptr;
        if (cudaMallocHost(&chunk, sizeof(OrientStats) * kSlotsPerChunk) != cudaSuccess) return nullptr;
        OrientStats* c = (OrientStats*)chunk;
        for (int i = kSlotsPerChunk - 1; i >= 0; --i) g_free_slots.push_back(c + i);
    }
    OrientStats* p = g_free_slots.back();
    g_free_slots.pop_back();
    return p;
}

void stats_slot_put(OrientStats* p)
{
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_slot_mu);
    g_free_slots.push_back(p);
}

kc_status ready(const kc_graph* g)
{
    std::lock_guard<std::mutex> lock(g->mu);
    if (g->is_ready) return g->ready_status;
    kc_graph* w = const_cast<kc_graph*>(g);
    kc_status st = KC_OK;
    if (g->done) {
        cudaError_t e = cudaEventSynchronize(g->done);
        if (e != cudaSuccess) {
            set_cuda_error(e, "cudaEventSynchronize(orientation)");
            st = KC_ECUDA;
        }
    }
    if (st == KC_OK && g->hstats) {
        const OrientStats& hs = *g->hstats;
        if (hs.err_timeout) st = KC_ETIMEOUT;
        else if (hs.err_input) st = KC_EINVAL;
        w->max_dplus = (int32_t)hs.max_dplus;
        w->wedges = (int64_t)hs.wedges;
        int64_t above = 0;  // d+ >= 33
        for (int i = 0; i < 6; ++i) above += (int64_t)hs.cls[i];
        w->ge_small[33] = above;
        for (int t = 32; t >= 0; --t) w->ge_small[t] = w->ge_small[t + 1] + (int64_t)hs.eq[t];
        w->ge_cls[6] = 0;
        for (int i = 5; i >= 0; --i) w->ge_cls[i] = w->ge_cls[i + 1] + (int64_t)hs.cls[i];
    }
    w->ready_status = st;
    w->is_ready = true;
    return st;
}

int64_t ge_at(const kc_graph* g, int64_t t)
{
    if (t <= 0) return g->n;
    if (t <= 33) return g->ge_small[t];
    for (int i = 1; i <= 5; ++i)
        if (t == (32LL << i) + 1) return g->ge_cls[i];
    // not a class boundary: the nearest boundary at or above t (callers
    // only ask for boundaries)
    for (int i = 1; i <= 5; ++i)
        if (t <= (32LL << i) + 1) return g->ge_cls[i];
    return 0;
}

}  // namespace kc
