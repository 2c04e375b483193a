// kc_internal.cuh -- internal declarations of libkc (not part of the ABI).
#pragma once

#include <algorithm>
#include <cstdint>
#include <cstddef>
#include <deque>
#include <mutex>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/kc.h"

namespace kc {

// ---------------------------------------------------------------- errors

void set_cuda_error(cudaError_t e, const char* what);

#define KC_CK(call)                                                   \
    do {                                                              \
        cudaError_t kc_e_ = (call);                                   \
        if (kc_e_ != cudaSuccess) {                                   \
            ::kc::set_cuda_error(kc_e_, #call);                       \
            return kc_e_ == cudaErrorMemoryAllocation ? KC_ENOMEM     \
                                                      : KC_ECUDA;     \
        }                                                             \
    } while (0)

// Every kernel launch is followed by KC_LAUNCHED(): it counts the launch
// (process-wide, readable through kc_get_param) and checks the launch error.
void note_launch();
#define KC_LAUNCHED()                                                 \
    do {                                                              \
        ::kc::note_launch();                                          \
        KC_CK(cudaGetLastError());                                    \
    } while (0)

#define KC_TRY(expr)                                                  \
    do {                                                              \
        kc_status kc_s_ = (expr);                                     \
        if (kc_s_ != KC_OK) return kc_s_;                             \
    } while (0)

// ------------------------------------------------------------ constants

constexpr int kWarp = 32;
constexpr uint32_t kFull = 0xffffffffu;

// Owner classes by |Gamma+(u)|: rows of W 32-bit words hold a bitmap row of
// G+(u).  Class c covers d+ in (32*W(c-1), 32*W(c)].
constexpr int kNumSmemClasses = 6;               // W = 1, 2, 4, 8, 16, 32
constexpr int kClassWords[kNumSmemClasses] = {1, 2, 4, 8, 16, 32};
// Owner slots in launch order: 0 = rows wider than the shared-memory limit
// (global tiles), 1..5 = shared-memory rows of 32, 16, 8, 4, 2 words,
// 6 = one word (registers).
constexpr int kOwnerSlots = 7;
// Zeroed cursor words a count needs: one per owner slot, and a second one
// per slot for the search pass of a split class.
constexpr int kCursorWords = 2 * kOwnerSlots;

// ---------------------------------------------------------- graph handle

// Statistics of an orientation, written by the orientation kernels and
// copied to (pinned) host memory at the end of kc_orient.
struct OrientStats {
    unsigned long long wedges;       // sum over u of C(d+(u), 2)
    unsigned long long eq[33];       // #{u : d+(u) == t}, t = 0..32
    unsigned long long cls[6];       // #{u : d+(u) in (32*2^i, 64*2^i]}, i = 0..4; cls[5]: d+ > 1024
    unsigned int max_dplus;
    unsigned int max_deg;
    int err_timeout;                 // a bounded device-side wait gave up
    int err_input;                   // sum of d+ != m: the CSR was not symmetric and simple
};

}  // namespace kc

struct kc_graph {
    int device = 0;
    int32_t n = 0;
    int64_t m = 0;
    int32_t max_dplus = 0;
    int64_t wedges = 0;
    int32_t* rank = nullptr;   // [n]  vertex id -> rank in the order
    int32_t* perm = nullptr;   // [n]  rank -> vertex id
    int32_t* deg = nullptr;    // [n]  degree, rank space
    int32_t* dplus = nullptr;  // [n]  |Gamma+|, rank space
    int64_t* offp = nullptr;   // [n+1] oriented CSR offsets, rank space
    int32_t* adjp = nullptr;   // [m]  oriented CSR columns (ranks), rows ascending
    int32_t* queue = nullptr;  // [n]  owners (ranks): bitmap class, then work estimate (see kc.h)
    void* block = nullptr;     // one pool allocation holding the arrays above
    int64_t bytes = 0;
    // host statistics: valid once ready() has returned KC_OK
    kc::OrientStats* hstats = nullptr;  // pinned slot the orientation copies its statistics into
    cudaEvent_t done = nullptr;         // recorded after the last orientation kernel
    mutable std::mutex mu;
    mutable bool is_ready = false;
    mutable kc_status ready_status = KC_OK;
    int64_t ge_small[34] = {};          // #{u : d+(u) >= t}, t = 0..33
    int64_t ge_cls[7] = {};             // #{u : d+(u) >= 32*2^i + 1}, i = 0..5; [6] = 0
    std::vector<kc_tuning> tunings;     // attached plans (kc_set_tuning), one per (k, per_vertex)
    // owner partitions for kc_count_part, built on first use per number of parts
    struct Parts {
        int nparts = 0;
        std::vector<std::vector<int64_t>> pos;  // per part: its queue positions, ascending
        std::vector<int64_t> off;               // per part: start of its owners in `queue`
        int32_t* queue = nullptr;               // device: every part's owners (ranks), queue order
    };
    mutable std::deque<Parts> parts;          // deque: references stay valid as parts are added
};

namespace kc {

// ------------------------------------------------------------ counting

// Per-class launch plan of one count (from a kc_tuning); null: the knobs.
struct Plan {
    int algo[kOwnerSlots];
    int parts[kOwnerSlots];
};

struct CountArgs {
    int k;
    uint32_t colours;       // 0: exact FFF_k; >= 1: cFFF_k
    uint64_t seed;
    bool pair = false;      // plain pair sampling (Sec. 6): keep a pair iff its hash < pthr
    uint64_t pthr = 0;
    bool per_vertex;        // accumulate memberships into pv (rank space)
    unsigned long long* total;  // [2] 128-bit total (lo, hi)
    unsigned long long* pv;     // [n] rank space, nullable
    unsigned long long* po;     // [n] rank space, nullable
    unsigned long long* work;   // [1] bitmap word-operations executed, nullable
    int part = 0, nparts = 1;   // count only owners at queue positions = part (mod nparts)
    struct Scratch* sc = nullptr;  // allocator for the split search's tiles (null: no split)
    const Plan* plan = nullptr;    // per-class counter and parts (null: process-wide knobs)
};

// cursors: kCursorWords zeroed counters.
kc_status count_launch(const kc_graph* g, const CountArgs& a, unsigned long long* cursors,
                       uint32_t* heavy_scratch, int64_t heavy_words, cudaStream_t s);

// One launch sequence over the owners of ng graphs.  descs: device array of
// ng graph descriptors; tables: device scratch of kOwnerSlots * (2 ng + 1)
// int64; a.total: 2 words per graph; host_tables must stay alive until the
// stream has consumed it.
kc_status count_batch_launch(const kc_graph* const* gs, int ng, const CountArgs& a, const void* descs,
                             int64_t* tables, unsigned long long* cursors, uint32_t* heavy_scratch,
                             int64_t heavy_words, std::vector<int64_t>& host_tables, cudaStream_t s);

// Per-class tables of a batch (host) and the launches over device copies of
// them (no host transfer: capturable in a CUDA graph).
void batch_tables(const kc_graph* const* gs, int ng, int k, std::vector<int64_t>& host_tables);
kc_status count_batch_run(const kc_graph* const* gs, int ng, const CountArgs& a, const void* descs,
                          const int64_t* tables, const std::vector<int64_t>& host_tables, unsigned long long* cursors,
                          uint32_t* heavy_scratch, int64_t heavy_words, cudaStream_t s);

// Queue range of owner slot `slot` for k under the current knobs.
void class_range(const kc_graph* g, int k, int slot, int64_t* q0, int64_t* q1);
int slot_words(int slot);
int64_t heavy_scratch_words_w(int W, int k, int64_t nheavy, int64_t* slot_words, int algo = -1);

extern bool g_work_enabled;
extern unsigned long long g_last_work;
int64_t launch_count();
void reset_launch_count();
int smem_max_words();
kc_status set_smem_max_words(int64_t v);

int compact_lo();
int compact_hi();
kc_status set_compact_window(int64_t lo, int64_t hi);
int count_algo();
kc_status set_count_algo(int64_t v);
kc_status list_run(const kc_graph* g, int k, unsigned flags, int32_t* buf, int64_t cap, kc_list_fn fn, void* user,
                   uint64_t* listed, cudaStream_t s);
int tri_enabled();
kc_status set_tri(int64_t v);
int complement_enabled();
kc_status set_complement(int64_t v);

// Stream-ordered allocation from the library's memory pool of the current
// device (a cudaMemPool that keeps freed memory for reuse instead of
// returning it at every synchronisation, so repeated calls do not pay for
// cudaMalloc).  Free with pool_free on a stream ordered after the last use.
kc_status pool_alloc(void** p, size_t bytes, cudaStream_t s);
void pool_free(void* p, cudaStream_t s);

// Pinned host slot for one graph's OrientStats (process-wide free list).
OrientStats* stats_slot_get();
void stats_slot_put(OrientStats* p);

// Waits (once per graph) for the orientation to finish and fills the host
// statistics; returns the orientation's status (KC_ETIMEOUT, KC_EINVAL for a
// CSR that was not symmetric and simple, KC_ECUDA).  Every entry point that
// reads g's host statistics or runs on another stream calls it first.
kc_status ready(const kc_graph* g);

// #{u : d+(u) >= t}; t must be <= 33 or one of 65, 129, 257, 513, 1025
// (the boundaries of the bitmap classes).
int64_t ge_at(const kc_graph* g, int64_t t);

// Stream-ordered scratch, released on scope exit (after the stream's work).
struct Scratch {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit Scratch(cudaStream_t st) : s(st) {}
    ~Scratch()
    {
        for (void* p : ptrs) pool_free(p, s);
    }
    template <typename T>
    kc_status get(T** p, int64_t count)
    {
        void* q = nullptr;
        KC_TRY(pool_alloc(&q, (size_t)std::max<int64_t>(count, 1) * sizeof(T), s));
        ptrs.push_back(q);
        *p = (T*)q;
        return KC_OK;
    }
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Words of global scratch the heavy (global-bitmap) class needs for k under
// the current settings; *slot_words receives the size of one tile slot.
int64_t heavy_scratch_words(const kc_graph* g, int k, int64_t* slot_words, const Plan* plan = nullptr);

// Words of global tiles the split search of the shared-memory classes needs
// for k (allocated by the count from its Scratch).
int64_t split_scratch_words(const kc_graph* g, int k, const Plan* plan = nullptr);

// The plan attached to g for (k, per-vertex output), if any.
bool find_plan(const kc_graph* g, int k, bool pv, Plan* out);

// The LPT partition of g's owners into nparts parts (built once, cached in g).
kc_status graph_parts(const kc_graph* g, int nparts, cudaStream_t s, const kc_graph::Parts** out);

// Round 2 input bytes for k (kc_round2_bytes).
kc_status round2_bytes(const kc_graph* g, int k, uint64_t* bytes, cudaStream_t s);

// Autotuner (count.cu).
kc_status tune(const kc_graph* const* gs, int ng, int k, bool pv, cudaStream_t s, kc_tuning* out);

}  // namespace kc
