// api.cu -- the extern "C" entry points of libkc (declared in include/kc.h).
#include <cmath>
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "count_common.cuh"

namespace kc {

kc_status orient(const int64_t* off, const int32_t* adj, int32_t n, int64_t m, unsigned flags,
                 cudaStream_t s, kc_graph** out);
int num_sms();

namespace {

thread_local char g_cuda_err[256] = "no error";
std::atomic<int64_t> g_launches{0};
}  // namespace

bool g_work_enabled = false;
unsigned long long g_last_work = 0;

namespace {

// out[perm[r]] = in[r]  (rank space -> caller ids)
__global__ void k_permute_u64(const unsigned long long* __restrict__ in, const int32_t* __restrict__ perm,
                              int32_t n, unsigned long long* __restrict__ out)
{
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
        out[perm[r]] = in[r];
}

__global__ void k_permute_i32_to_u64(const int32_t* __restrict__ in, const int32_t* __restrict__ perm,
                                     int32_t n, unsigned long long* __restrict__ out)
{
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
        out[perm[r]] = (unsigned long long)in[r];
}

__global__ void k_fill_u64(unsigned long long* __restrict__ out, int32_t n, unsigned long long v)
{
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) out[r] = v;
}

int grid1d(int64_t n)
{
    int64_t g = (n + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 8;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}



// Host-ordered output of an n-array: device array `src` -> `dst` (host or
// device per `dev`).
kc_status copy_out_u64(uint64_t* dst, const unsigned long long* src, int32_t n, bool dev, cudaStream_t s)
{
    if (!dst || n <= 0) return KC_OK;
    KC_CK(cudaMemcpyAsync(dst, src, (size_t)n * sizeof(uint64_t),
                          dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    return KC_OK;
}

// Shared body of kc_count and kc_estimate.
kc_status run_count(const kc_graph* g, int k, uint32_t colours, uint64_t seed, unsigned flags,
                    uint64_t* total, uint64_t* per_vertex, uint64_t* per_owner, cudaStream_t s, int part = 0,
                    int nparts = 1, bool pair = false, uint64_t pthr = 0)
{
    const bool dev = (flags & KC_DEVICE_PTRS) != 0;
    const int32_t n = g->n;
    Scratch sc(s);
    unsigned long long* small = nullptr;  // [0..1] total lo/hi, [2..15] cursors, [16] work
    KC_TRY(sc.get(&small, 24));
    KC_CK(cudaMemsetAsync(small, 0, 24 * sizeof(unsigned long long), s));

    // outputs: write permuted results straight into device outputs, else into temps
    unsigned long long* out_pv = nullptr;
    unsigned long long* out_po = nullptr;
    if (per_vertex) {
        if (dev) out_pv = (unsigned long long*)per_vertex;
        else KC_TRY(sc.get(&out_pv, n));
    }
    if (per_owner) {
        if (dev) out_po = (unsigned long long*)per_owner;
        else KC_TRY(sc.get(&out_po, n));
    }

    if (k <= 2 && nparts > 1) return KC_ENOTSUP;  // q_1, q_2 have no owner split
    if (k <= 2) {
        const unsigned long long q = k == 1 ? (unsigned long long)n : (unsigned long long)g->m;
        k_fill_u64<<<1, 32, 0, s>>>(small, 1, q);
        KC_LAUNCHED();
        if (n > 0) {
            if (out_pv) {
                if (k == 1) k_fill_u64<<<grid1d(n), 256, 0, s>>>(out_pv, n, 1ull);
                else k_permute_i32_to_u64<<<grid1d(n), 256, 0, s>>>(g->deg, g->perm, n, out_pv);
                KC_LAUNCHED();
            }
            if (out_po) {
                if (k == 1) k_fill_u64<<<grid1d(n), 256, 0, s>>>(out_po, n, 1ull);
                else k_permute_i32_to_u64<<<grid1d(n), 256, 0, s>>>(g->dplus, g->perm, n, out_po);
                KC_LAUNCHED();
            }
        }
    } else if (n > 0) {
        unsigned long long* pv_rank = nullptr;
        unsigned long long* po_rank = nullptr;
        if (per_vertex) {
            KC_TRY(sc.get(&pv_rank, n));
            KC_CK(cudaMemsetAsync(pv_rank, 0, (size_t)n * sizeof(unsigned long long), s));
        }
        if (per_owner) {
            KC_TRY(sc.get(&po_rank, n));
            KC_CK(cudaMemsetAsync(po_rank, 0, (size_t)n * sizeof(unsigned long long), s));
        }
        // the attached plan for k (exact counts; colour-sampled estimates use its
        // choice of counter per class too -- plain pair sampling keeps the knobs)
        Plan plan;
        const bool planned = !pair && find_plan(g, k, per_vertex != nullptr, &plan);
        int64_t slot_words = 0;
        const int64_t hw = heavy_scratch_words(g, k, &slot_words, planned ? &plan : nullptr);
        uint32_t* heavy = nullptr;
        if (hw > 0) KC_TRY(sc.get(&heavy, hw));
        CountArgs a;
        a.plan = planned ? &plan : nullptr;
        a.k = k;
        a.colours = colours;
        a.seed = seed;
        a.pair = pair;
        a.pthr = pthr;
        a.per_vertex = per_vertex != nullptr;
        a.total = small;
        a.pv = pv_rank;
        a.po = po_rank;
        a.work = g_work_enabled ? small + 16 : nullptr;
        a.part = part;
        a.nparts = nparts;
        a.sc = &sc;
        KC_TRY(count_launch(g, a, small + 2, heavy, hw, s));
        if (pv_rank) {
            k_permute_u64<<<grid1d(n), 256, 0, s>>>(pv_rank, g->perm, n, out_pv);
            KC_LAUNCHED();
        }
        if (po_rank) {
            k_permute_u64<<<grid1d(n), 256, 0, s>>>(po_rank, g->perm, n, out_po);
            KC_LAUNCHED();
        }
    }

    if (dev) {
        KC_CK(cudaMemcpyAsync(total, small, 2 * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        return KC_OK;
    }
    unsigned long long th[17] = {0};
    KC_CK(cudaMemcpyAsync(th, small, sizeof(th), cudaMemcpyDeviceToHost, s));
    KC_TRY(copy_out_u64(per_vertex, out_pv, n, false, s));
    KC_TRY(copy_out_u64(per_owner, out_po, n, false, s));
    KC_CK(cudaStreamSynchronize(s));
    *total = th[0];
    if (g_work_enabled) g_last_work = th[16];
    return th[1] ? KC_EOVERFLOW : KC_OK;
}

}  // namespace

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
void reset_launch_count() { g_launches.store(0, std::memory_order_relaxed); }

void set_cuda_error(cudaError_t e, const char* what)
{
    std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s (%d)", what, cudaGetErrorString(e), (int)e);
}

}  // namespace kc

extern "C" {

const char* kc_strerror(kc_status s)
{
    switch (s) {
    case KC_OK: return "ok";
    case KC_EINVAL: return "invalid argument";
    case KC_ENOMEM: return "out of memory";
    case KC_EOVERFLOW: return "count overflow";
    case KC_ETIMEOUT: return "device wait timed out";
    case KC_ECUDA: return "CUDA error";
    case KC_ENOTSUP: return "not supported";
    case KC_ECANCELED: return "stopped by the callback";
    }
    return "unknown status";
}

const char* kc_last_cuda_error(void) { return kc::g_cuda_err; }

const char* kc_version(void) { return "kc 0.1 sm_103a"; }

kc_status kc_build_csr(int32_t n, const int32_t* src, const int32_t* dst, int64_t ne, int64_t* off,
                       int32_t* adj, int64_t* m_out)
{
    if (n < 0 || ne < 0 || !off || !m_out || (ne > 0 && (!src || !dst || !adj))) return KC_EINVAL;
    std::vector<uint64_t> keys;
    try {
        keys.reserve((size_t)ne * 2);
    } catch (...) {
        return KC_ENOMEM;
    }
    for (int64_t i = 0; i < ne; ++i) {
        const int32_t a = src[i], b = dst[i];
        if (a < 0 || a >= n || b < 0 || b >= n) return KC_EINVAL;
        if (a == b) continue;
        keys.push_back(((uint64_t)(uint32_t)a << 32) | (uint32_t)b);
        keys.push_back(((uint64_t)(uint32_t)b << 32) | (uint32_t)a);
    }
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    std::fill(off, off + (size_t)n + 1, 0);
    for (size_t i = 0; i < keys.size(); ++i) {
        off[(keys[i] >> 32) + 1]++;
        adj[i] = (int32_t)(keys[i] & 0xffffffffu);
    }
    for (int32_t v = 0; v < n; ++v) off[v + 1] += off[v];
    *m_out = (int64_t)keys.size() / 2;
    return KC_OK;
}

kc_status kc_orient(const int64_t* off, const int32_t* adj, int32_t n, int64_t m, unsigned flags, void* stream,
                    kc_graph** out)
{
    if (!out) return KC_EINVAL;
    *out = nullptr;
    return kc::orient(off, adj, n, m, flags, (cudaStream_t)stream, out);
}

void kc_free(kc_graph* g)
{
    if (!g) return;
    kc::DeviceGuard dg(g->device);
    if (g->done) {
        cudaEventSynchronize(g->done);  // the orientation may still be running
        cudaEventDestroy(g->done);
    }
    kc::pool_free(g->block, 0);
    for (const kc_graph::Parts& p : g->parts) kc::pool_free(p.queue, 0);
    kc::stats_slot_put(g->hstats);
    delete g;
}

kc_status kc_info(const kc_graph* g, kc_graph_info* info)
{
    if (!g || !info) return KC_EINVAL;
    KC_TRY(kc::ready(g));
    info->n = g->n;
    info->m = g->m;
    info->max_dplus = g->max_dplus;
    info->wedges = g->wedges;
    info->device_bytes = g->bytes;
    return KC_OK;
}

kc_status kc_export(const kc_graph* g, unsigned flags, int32_t* rank, int32_t* perm, int64_t* off_plus,
                    int32_t* adj_plus, int32_t* queue, void* stream)
{
    if (!g) return KC_EINVAL;
    kc::DeviceGuard dg(g->device);
    KC_TRY(kc::ready(g));
    cudaStream_t s = (cudaStream_t)stream;
    const cudaMemcpyKind kind = (flags & KC_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const size_t n = (size_t)g->n;
    if (rank && n) KC_CK(cudaMemcpyAsync(rank, g->rank, n * sizeof(int32_t), kind, s));
    if (perm && n) KC_CK(cudaMemcpyAsync(perm, g->perm, n * sizeof(int32_t), kind, s));
    if (off_plus) KC_CK(cudaMemcpyAsync(off_plus, g->offp, (n + 1) * sizeof(int64_t), kind, s));
    if (adj_plus && g->m) KC_CK(cudaMemcpyAsync(adj_plus, g->adjp, (size_t)g->m * sizeof(int32_t), kind, s));
    if (queue && n) KC_CK(cudaMemcpyAsync(queue, g->queue, n * sizeof(int32_t), kind, s));
    KC_CK(cudaStreamSynchronize(s));
    return KC_OK;
}

kc_status kc_count(const kc_graph* g, int k, unsigned flags, uint64_t* total, uint64_t* per_vertex,
                   uint64_t* per_owner, void* stream)
{
    if (!g || !total || k < 1 || k > KC_MAX_K) return KC_EINVAL;
    kc::DeviceGuard dg(g->device);
    KC_TRY(kc::ready(g));
    return kc::run_count(g, k, 0, 0, flags, total, per_vertex, per_owner, (cudaStream_t)stream);
}

kc_status kc_estimate(const kc_graph* g, int k, uint32_t colours, uint64_t seed, unsigned flags,
                      uint64_t* sampled, double* estimate, uint64_t* per_owner, void* stream)
{
    if (!g || !sampled || k < 1 || k > KC_MAX_K || colours < 1) return KC_EINVAL;
    kc::DeviceGuard dg(g->device);
    KC_TRY(kc::ready(g));
    kc_status st = kc::run_count(g, k, colours, seed, flags, sampled, nullptr, per_owner, (cudaStream_t)stream);
    if (st != KC_OK) return st;
    if (estimate && !(flags & KC_DEVICE_PTRS)) {
        double f = 1.0;
        for (int i = 0; i < k - 2; ++i) f *= (double)colours;
        *estimate = (double)*sampled * f;
    }
    return KC_OK;
}

kc_status kc_estimate_pairs(const kc_graph* g, int k, double p, uint64_t seed, unsigned flags, uint64_t* sampled,
                            double* estimate, uint64_t* per_owner, void* stream)
{
    if (!g || !sampled || k < 1 || k > KC_MAX_K || !(p > 0.0 && p <= 1.0)) return KC_EINVAL;
    kc::DeviceGuard dg(g->device);
    KC_TRY(kc::ready(g));
    // p = 1 keeps every pair: the exact count
    const bool pair = p < 1.0;
    const uint64_t thr = pair ? (uint64_t)std::ldexp(p, 64) : 0;
    kc_status st = kc::run_count(g, k, 0, seed, flags, sampled, nullptr, per_owner, (cudaStream_t)stream, 0, 1,
                                 pair, thr);
    if (st != KC_OK) return st;
    if (estimate && !(flags & KC_DEVICE_PTRS)) {
        double f = 1.0;
        for (int i = 0; i < (k - 1) * (k - 2) / 2; ++i) f *= p;
        *estimate = (double)*sampled / f;
    }
    return KC_OK;
}

kc_status kc_list(const kc_graph* g, int k, unsigned flags, int32_t* buf, int64_t cap, kc_list_fn fn, void* user,
                  uint64_t* listed, void* stream)
{
    if (!g || !buf || !fn || !listed || k < 1 || k > KC_MAX_K || cap < 1) return KC_EINVAL;
    kc::DeviceGuard dg(g->device);
    KC_TRY(kc::ready(g));
    return kc::list_run(g, k, flags, buf, cap, fn, user, listed, (cudaStream_t)stream);
}

kc_status kc_footprint(const kc_graph* g, int k, int per_vertex, int per_owner, int host_outputs,
                       uint64_t* bytes)
{
    if (!g || !bytes || k < 1 || k > KC_MAX_K) return KC_EINVAL;
    KC_TRY(kc::ready(g));
    const uint64_t n = (uint64_t)(g->n > 0 ? g->n : 1);
    uint64_t b = 256;  // total, cursors, work counter
    const uint64_t arrays = (per_vertex ? 1 : 0) + (per_owner ? 1 : 0);
    if (k >= 3) b += arrays * n * 8;           // rank-space accumulators
    if (host_outputs) b += arrays * n * 8;     // staging for the copy back
    if (k >= 3) {
        kc::Plan plan;
        const bool planned = kc::find_plan(g, k, per_vertex != 0, &plan);
        int64_t slot_words = 0;
        b += (uint64_t)kc::heavy_scratch_words(g, k, &slot_words, planned ? &plan : nullptr) * 4;
        b += (uint64_t)kc::split_scratch_words(g, k, planned ? &plan : nullptr) * 4;
        b += 256 * 8;  // alignment of the scratch blocks
    }
    *bytes = b;
    return KC_OK;
}

kc_status kc_round2_bytes(const kc_graph* g, int k, uint64_t* bytes, void* stream)
{
    if (!g || !bytes || k < 1 || k > KC_MAX_K) return KC_EINVAL;
    kc::DeviceGuard dg(g->device);
    KC_TRY(kc::ready(g));
    return kc::round2_bytes(g, k, bytes, (cudaStream_t)stream);
}

kc_status kc_count_part(const kc_graph* g, int k, int part, int nparts, unsigned flags, uint64_t* total,
                        uint64_t* per_vertex, uint64_t* per_owner, void* stream)
{
    if (!g || !total || k < 3 || k > KC_MAX_K || nparts < 1 || part < 0 || part >= nparts) return KC_EINVAL;
    kc::DeviceGuard dg(g->device);
    KC_TRY(kc::ready(g));
    return kc::run_count(g, k, 0, 0, flags, total, per_vertex, per_owner, (cudaStream_t)stream, part, nparts);
}

kc_status kc_count_batch(const kc_graph* const* gs, int ng, int k, unsigned flags, uint64_t* totals, void* stream)
{
    if (!gs || ng < 0 || !totals || k < 1 || k > KC_MAX_K) return KC_EINVAL;
    if (ng == 0) return KC_OK;
    for (int i = 0; i < ng; ++i)
        if (!gs[i] || gs[i]->device != gs[0]->device) return KC_EINVAL;
    kc::DeviceGuard dg(gs[0]->device);
    for (int i = 0; i < ng; ++i) KC_TRY(kc::ready(gs[i]));
    cudaStream_t s = (cudaStream_t)stream;
    const bool dev = (flags & KC_DEVICE_PTRS) != 0;
    if (k <= 2) {
        std::vector<unsigned long long> h((size_t)(dev ? 2 * ng : ng), 0ull);
        for (int i = 0; i < ng; ++i) {
            const unsigned long long q = k == 1 ? (unsigned long long)gs[i]->n : (unsigned long long)gs[i]->m;
            h[(size_t)(dev ? 2 * i : i)] = q;
        }
        if (dev) {
            KC_CK(cudaMemcpyAsync(totals, h.data(), h.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
            KC_CK(cudaStreamSynchronize(s));
        } else {
            std::copy(h.begin(), h.end(), totals);
        }
        return KC_OK;
    }
    kc::Scratch sc(s);
    std::vector<kc::cc::GraphDesc> hd((size_t)ng);
    int Wh = 1;
    int64_t nheavy = 0;
    for (int i = 0; i < ng; ++i) {
        hd[(size_t)i] = {gs[i]->offp, gs[i]->adjp, gs[i]->queue, gs[i]->perm};
        Wh = std::max(Wh, (gs[i]->max_dplus + 31) / 32);
        int64_t q0 = 0, q1 = 0;
        kc::class_range(gs[i], k, 0, &q0, &q1);
        nheavy += q1 - q0;
    }
    kc::cc::GraphDesc* dd = nullptr;
    int64_t* tables = nullptr;
    unsigned long long* small = nullptr;  // cursors [0..15], then 2 words per graph
    KC_TRY(sc.get(&dd, ng));
    KC_TRY(sc.get(&tables, (int64_t)kc::kOwnerSlots * (2 * ng + 1)));
    KC_TRY(sc.get(&small, 16 + 2 * (int64_t)ng));
    KC_CK(cudaMemcpyAsync(dd, hd.data(), hd.size() * sizeof(kc::cc::GraphDesc), cudaMemcpyHostToDevice, s));
    KC_CK(cudaMemsetAsync(small, 0, (16 + 2 * (size_t)ng) * sizeof(unsigned long long), s));
    kc::Plan plan;
    const bool planned = kc::find_plan(gs[0], k, false, &plan);
    int64_t slot_words = 0;
    const int64_t hw = kc::heavy_scratch_words_w(Wh, k, nheavy, &slot_words, planned ? plan.algo[0] : -1);
    uint32_t* heavy = nullptr;
    if (hw > 0) KC_TRY(sc.get(&heavy, hw));
    kc::CountArgs a;
    a.plan = planned ? &plan : nullptr;
    a.k = k;
    a.colours = 0;
    a.seed = 0;
    a.per_vertex = false;
    a.total = small + 16;
    a.pv = nullptr;
    a.po = nullptr;
    a.work = nullptr;
    a.sc = &sc;
    std::vector<int64_t> host_tables;
    KC_TRY(kc::count_batch_launch(gs, ng, a, dd, tables, small, heavy, hw, host_tables, s));
    std::vector<unsigned long long> th((size_t)(2 * ng));
    if (dev) {
        KC_CK(cudaMemcpyAsync(totals, small + 16, 2 * (size_t)ng * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        KC_CK(cudaStreamSynchronize(s));  // host tables are read by the copy above
        return KC_OK;
    }
    KC_CK(cudaMemcpyAsync(th.data(), small + 16, th.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    KC_CK(cudaStreamSynchronize(s));
    kc_status st = KC_OK;
    for (int i = 0; i < ng; ++i) {
        totals[i] = th[(size_t)(2 * i)];
        if (th[(size_t)(2 * i + 1)]) st = KC_EOVERFLOW;
    }
    return st;
}

}  // extern "C"

struct kc_batch {
    int device = 0;
    int ng = 0;
    int k = 0;
    std::vector<const kc_graph*> gs;
    std::vector<int64_t> host_tables;
    kc::Plan plan;
    bool planned = false;
    void* dev = nullptr;  // descriptors, then tables
    kc::cc::GraphDesc* descs = nullptr;
    int64_t* tables = nullptr;
    int64_t heavy_words = 0;
};

extern "C" {

kc_status kc_batch_create(const kc_graph* const* gs, int ng, int k, unsigned flags, void* stream, kc_batch** out)
{
    if (!out) return KC_EINVAL;
    *out = nullptr;
    if (!gs || ng < 1 || k < 3 || k > KC_MAX_K || flags != 0) return KC_EINVAL;
    for (int i = 0; i < ng; ++i)
        if (!gs[i] || gs[i]->device != gs[0]->device) return KC_EINVAL;
    kc::DeviceGuard dg(gs[0]->device);
    for (int i = 0; i < ng; ++i) KC_TRY(kc::ready(gs[i]));
    cudaStream_t s = (cudaStream_t)stream;
    kc_batch* b = new (std::nothrow) kc_batch();
    if (!b) return KC_ENOMEM;
    b->device = gs[0]->device;
    b->ng = ng;
    b->k = k;
    b->gs.assign(gs, gs + ng);
    b->planned = kc::find_plan(gs[0], k, false, &b->plan);
    kc::batch_tables(gs, ng, k, b->host_tables);
    std::vector<kc::cc::GraphDesc> hd((size_t)ng);
    int Wh = 1;
    int64_t nheavy = 0;
    for (int i = 0; i < ng; ++i) {
        hd[(size_t)i] = {gs[i]->offp, gs[i]->adjp, gs[i]->queue, gs[i]->perm};
        Wh = std::max(Wh, (gs[i]->max_dplus + 31) / 32);
        int64_t q0 = 0, q1 = 0;
        kc::class_range(gs[i], k, 0, &q0, &q1);
        nheavy += q1 - q0;
    }
    int64_t slot_words = 0;
    b->heavy_words = kc::heavy_scratch_words_w(Wh, k, nheavy, &slot_words, b->planned ? b->plan.algo[0] : -1);
    const size_t dbytes = ((hd.size() * sizeof(kc::cc::GraphDesc) + 255) & ~(size_t)255) +
                          b->host_tables.size() * sizeof(int64_t);
    kc_status st = kc::pool_alloc(&b->dev, dbytes, s);
    if (st != KC_OK) {
        delete b;
        return st;
    }
    b->descs = (kc::cc::GraphDesc*)b->dev;
    b->tables = (int64_t*)((char*)b->dev + ((hd.size() * sizeof(kc::cc::GraphDesc) + 255) & ~(size_t)255));
    cudaError_t e = cudaMemcpyAsync(b->descs, hd.data(), hd.size() * sizeof(kc::cc::GraphDesc),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->tables, b->host_tables.data(), b->host_tables.size() * sizeof(int64_t),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        kc::set_cuda_error(e, "kc_batch_create");
        kc_batch_free(b);
        return KC_ECUDA;
    }
    *out = b;
    return KC_OK;
}

kc_status kc_batch_count(kc_batch* b, uint64_t* totals, void* stream)
{
    if (!b || !totals) return KC_EINVAL;
    kc::DeviceGuard dg(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    kc::Scratch sc(s);
    unsigned long long* cursors = nullptr;
    KC_TRY(sc.get(&cursors, 16));
    KC_CK(cudaMemsetAsync(cursors, 0, 16 * sizeof(unsigned long long), s));
    KC_CK(cudaMemsetAsync(totals, 0, 2 * (size_t)b->ng * sizeof(uint64_t), s));
    uint32_t* heavy = nullptr;
    if (b->heavy_words > 0) KC_TRY(sc.get(&heavy, b->heavy_words));
    kc::CountArgs a;
    a.k = b->k;
    a.colours = 0;
    a.seed = 0;
    a.per_vertex = false;
    a.total = (unsigned long long*)totals;
    a.pv = nullptr;
    a.po = nullptr;
    a.work = nullptr;
    a.sc = &sc;
    a.plan = b->planned ? &b->plan : nullptr;
    return kc::count_batch_run(b->gs.data(), b->ng, a, b->descs, b->tables, b->host_tables, cursors, heavy,
                               b->heavy_words, s);
}

void kc_batch_free(kc_batch* b)
{
    if (!b) return;
    kc::DeviceGuard dg(b->device);
    kc::pool_free(b->dev, 0);
    delete b;
}

kc_status kc_tune(const kc_graph* const* gs, int ng, int k, unsigned flags, void* stream, kc_tuning* out)
{
    if (!gs || ng < 1 || !out || k < 1 || k > KC_MAX_K) return KC_EINVAL;
    for (int i = 0; i < ng; ++i)
        if (!gs[i] || gs[i]->device != gs[0]->device) return KC_EINVAL;
    kc::DeviceGuard dg(gs[0]->device);
    for (int i = 0; i < ng; ++i) KC_TRY(kc::ready(gs[i]));
    return kc::tune(gs, ng, k, (flags & KC_TUNE_PER_VERTEX) != 0, (cudaStream_t)stream, out);
}

kc_status kc_set_tuning(kc_graph* g, const kc_tuning* t)
{
    if (!g) return KC_EINVAL;
    if (!t) {
        g->tunings.clear();
        return KC_OK;
    }
    if (t->k < 1 || t->k > KC_MAX_K) return KC_EINVAL;
    for (int i = 0; i < kc::kOwnerSlots; ++i) {
        if (t->algo[i] != KC_ALGO_DFS && t->algo[i] != KC_ALGO_PIVOT) return KC_EINVAL;
        if (t->parts[i] < 1 || t->parts[i] > 64) return KC_EINVAL;
    }
    for (kc_tuning& x : g->tunings)
        if (x.k == t->k && (x.per_vertex != 0) == (t->per_vertex != 0)) {
            x = *t;
            return KC_OK;
        }
    g->tunings.push_back(*t);
    return KC_OK;
}

kc_status kc_set_param(int param, int64_t value)
{
    if (param == KC_PARAM_SMEM_MAX_WORDS) return kc::set_smem_max_words(value);
    if (param == KC_PARAM_LAUNCH_COUNT) {
        if (value != 0) return KC_EINVAL;
        kc::reset_launch_count();
        return KC_OK;
    }
    if (param == KC_PARAM_ALGO) return kc::set_count_algo(value);
    if (param == KC_PARAM_TRI) return kc::set_tri(value);
    if (param == KC_PARAM_COMPLEMENT) return kc::set_complement(value);
    if (param == KC_PARAM_COMPACT_LO) return kc::set_compact_window(value, kc::compact_hi());
    if (param == KC_PARAM_COMPACT_HI) return kc::set_compact_window(kc::compact_lo(), value);
    if (param == KC_PARAM_WORK_COUNT) {
        if (value != 0 && value != 1) return KC_EINVAL;
        kc::g_work_enabled = value != 0;
        return KC_OK;
    }
    return KC_EINVAL;
}

kc_status kc_get_param(int param, int64_t* value)
{
    if (!value) return KC_EINVAL;
    if (param == KC_PARAM_SMEM_MAX_WORDS) {
        *value = kc::smem_max_words();
        return KC_OK;
    }
    if (param == KC_PARAM_LAUNCH_COUNT) {
        *value = kc::launch_count();
        return KC_OK;
    }
    if (param == KC_PARAM_ALGO) {
        *value = kc::count_algo();
        return KC_OK;
    }
    if (param == KC_PARAM_TRI) {
        *value = kc::tri_enabled();
        return KC_OK;
    }
    if (param == KC_PARAM_COMPLEMENT) {
        *value = kc::complement_enabled();
        return KC_OK;
    }
    if (param == KC_PARAM_COMPACT_LO) {
        *value = kc::compact_lo();
        return KC_OK;
    }
    if (param == KC_PARAM_COMPACT_HI) {
        *value = kc::compact_hi();
        return KC_OK;
    }
    if (param == KC_PARAM_WORK_COUNT) {
        *value = (int64_t)kc::g_last_work;
        return KC_OK;
    }
    return KC_EINVAL;
}

kc_status kc_count_csr(const int64_t* off, const int32_t* adj, int32_t n, int64_t m, int k, unsigned flags,
                       uint64_t* total, uint64_t* per_vertex, uint64_t* per_owner, void* stream)
{
    kc_graph* g = nullptr;
    kc_status st = kc_orient(off, adj, n, m, flags, stream, &g);
    if (st != KC_OK) return st;
    st = kc_count(g, k, flags, total, per_vertex, per_owner, stream);
    if (st == KC_OK && (flags & KC_DEVICE_PTRS)) {
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) {
            kc::set_cuda_error(e, "cudaStreamSynchronize");
            st = KC_ECUDA;
        }
    }
    kc_free(g);
    return st;
}

kc_status kc_estimate_csr(const int64_t* off, const int32_t* adj, int32_t n, int64_t m, int k, uint32_t colours,
                          uint64_t seed, unsigned flags, uint64_t* sampled, double* estimate, void* stream)
{
    kc_graph* g = nullptr;
    kc_status st = kc_orient(off, adj, n, m, flags, stream, &g);
    if (st != KC_OK) return st;
    st = kc_estimate(g, k, colours, seed, flags, sampled, estimate, nullptr, stream);
    if (st == KC_OK && (flags & KC_DEVICE_PTRS)) {
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) {
            kc::set_cuda_error(e, "cudaStreamSynchronize");
            st = KC_ECUDA;
        }
    }
    kc_free(g);
    return st;
}

}  // extern "C"
