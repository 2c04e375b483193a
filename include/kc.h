/*
 * kc.h -- C ABI of libkc, a GB300 (sm_103a) implementation of the hot path of
 * the exact k-clique counting algorithm FFF_k and its colour-sampling
 * estimator cFFF_k (Finocchi, Finocchi & Fusco, "Clique counting in
 * MapReduce: theory and experiments", arXiv:1403.0734).
 *
 * The method: order the vertices by (degree, id) (Sec. 2); every k-clique is
 * counted once, by its smallest vertex u (Sec. 3); u counts the (k-1)-cliques
 * of G+(u), the subgraph induced by its high-neighbourhood Gamma+(u)
 * (Algorithm 1, rounds 1-3).  cFFF_k colours every Gamma+(u) independently
 * with c colours, keeps only monochromatic pairs, and scales the sampled
 * count by c^(k-2) (Sec. 6, "Color-based sampling").
 *
 * Conventions shared by every entry point
 *   - Graphs are undirected and simple, given as a CSR: off[n+1] (int64,
 *     off[0] = 0, off[n] = 2m) and adj[2m] (int32); every edge {u,v} appears
 *     as v in row u and u in row v; rows sorted ascending; no self-loops or
 *     repeats (the paper's preprocessed input, Sec. 4).  Vertex ids are the
 *     caller's ids 0..n-1 and break degree ties (Sec. 2).
 *   - Inputs are owned by the caller and only read.  A kc_graph is owned by
 *     the library from kc_orient until kc_free.  Outputs are caller-allocated.
 *   - Pointers are host pointers unless KC_DEVICE_PTRS is set in `flags`, in
 *     which case the pointer arguments documented as "array" are device
 *     pointers of the current CUDA device.
 *   - `stream` is a cudaStream_t (NULL: the legacy default stream).  Calls
 *     with host outputs return after the result is on the host; calls with
 *     KC_DEVICE_PTRS outputs are asynchronous on `stream`.
 *   - Every failure is reported as a kc_status; nothing aborts or traps.
 *     Kernel-side waits are bounded and report KC_ETIMEOUT.
 *   - Counts are exact unsigned 64-bit integers; a total that does not fit
 *     returns KC_EOVERFLOW.
 */
#ifndef KC_H
#define KC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kc_graph kc_graph;

typedef enum {
    KC_OK = 0,
    KC_EINVAL = 1,     /* bad argument, or (with KC_VALIDATE) a malformed CSR */
    KC_ENOMEM = 2,     /* device or host allocation failed */
    KC_EOVERFLOW = 3,  /* a count exceeded 2^64 - 1 */
    KC_ETIMEOUT = 4,   /* a bounded device-side wait gave up */
    KC_ECUDA = 5,      /* a CUDA runtime call failed (see kc_last_cuda_error) */
    KC_ENOTSUP = 6,    /* request outside the supported range */
    KC_ECANCELED = 7   /* a caller's callback asked to stop */
} kc_status;

/* flags */
#define KC_DEVICE_PTRS 0x1u  /* array arguments are device pointers */
#define KC_VALIDATE    0x2u  /* kc_orient / kc_count_csr: check the CSR first */

/* Largest k accepted by kc_count / kc_estimate. */
#define KC_MAX_K 32

/* Human-readable name of a status (static storage). */
const char* kc_strerror(kc_status s);

/* Text of the last CUDA error seen by this thread (static storage). */
const char* kc_last_cuda_error(void);

/* Library version, e.g. "kc 0.1 sm_103a". */
const char* kc_version(void);

/*
 * kc_build_csr -- preprocessing (Sec. 4: the graphs are made undirected):
 * turn an arbitrary edge list into the canonical CSR above.  Host-side.
 *   n        number of vertices; every endpoint must be in [0, n)
 *   src,dst  ne endpoints (host arrays); either direction, self-loops and
 *            repeated edges allowed (they are dropped)
 *   off      out, host array of n+1
 *   adj      out, host array with room for 2*ne entries
 *   m_out    out, number of undirected edges kept
 * Errors: KC_EINVAL (endpoint out of range, n < 0, ne < 0), KC_ENOMEM.
 */
kc_status kc_build_csr(int32_t n, const int32_t* src, const int32_t* dst, int64_t ne,
                       int64_t* off, int32_t* adj, int64_t* m_out);

/*
 * kc_orient -- Round 1 of Algorithm 1 (Sec. 3, "high-neighborhood
 * computation") on the device: degrees d(v) (Sec. 2), the total order
 * x < y iff d(x) < d(y) or (d(x) = d(y) and x < y) (Sec. 2), and every
 * Gamma+(u) = {x in Gamma(u) : u < x}.  The result is kept resident as an
 * oriented CSR in rank space (vertex r is the r-th smallest in the order;
 * row r lists the ranks of Gamma+(r) ascending, i.e. in the order), plus the
 * work queue used by the counting kernels (see kc_export).
 *   off, adj  the canonical CSR (arrays; host or, with KC_DEVICE_PTRS, device)
 *   n, m      vertices and undirected edges (adj has 2m entries); n >= 0
 *   flags     KC_DEVICE_PTRS, KC_VALIDATE (symmetry, sorted rows, no loops,
 *             no repeats; failures return KC_EINVAL)
 *   out       receives the new graph handle (NULL on failure)
 * Asynchronous on `stream` (without KC_VALIDATE): host inputs are copied
 * before the call returns; device inputs must stay unchanged until the
 * orientation has run on `stream`.  The handle can be passed on at once: the
 * first later call that needs the orientation's results on the host (any
 * count, estimate, listing, kc_info, kc_export, kc_footprint) waits for it,
 * and reports a failure of the orientation itself there (KC_ETIMEOUT, or
 * KC_EINVAL for a CSR that is not symmetric and simple).  Device memory comes
 * from a pool owned by the library, which keeps freed blocks for reuse.
 * Errors: KC_EINVAL, KC_ENOMEM, KC_ECUDA.
 */
kc_status kc_orient(const int64_t* off, const int32_t* adj, int32_t n, int64_t m,
                    unsigned flags, void* stream, kc_graph** out);

/* Release a graph and its device memory (back to the library's pool).  NULL
 * is ignored.  Waits for the graph's orientation if it is still running; the
 * caller must ensure no other call using `g` is still running on any stream. */
void kc_free(kc_graph* g);

typedef struct {
    int32_t n;              /* vertices */
    int64_t m;              /* undirected edges = sum over u of |Gamma+(u)| */
    int32_t max_dplus;      /* max |Gamma+(u)|, at most 2 sqrt(m) (App. B, Thm I) */
    int64_t wedges;         /* sum over u of C(|Gamma+(u)|, 2): Map 2 pairs (App. B, Thm 1) */
    int64_t device_bytes;   /* device memory held by the handle */
} kc_graph_info;

/* Statistics of an oriented graph (host struct).  Errors: KC_EINVAL. */
kc_status kc_info(const kc_graph* g, kc_graph_info* info);

/*
 * kc_export -- copy the oriented graph out, for checking Round 1.
 *   rank     array of n: rank[v] = position of vertex v in the order
 *   perm     array of n: perm[r] = vertex with rank r
 *   off_plus array of n+1: row offsets of the oriented CSR (rank space)
 *   adj_plus array of m: ranks of Gamma+ of each row, ascending
 *   queue    array of n: the owners (ranks) in the order the counting
 *            kernels take them.  Owners are grouped by the width of their
 *            bitmap row: |Gamma+| > 1024 first, then 513..1024, 257..512,
 *            129..256, 65..128, 33..64, 1..32, and 0 last.  In the 1..32
 *            group they go by |Gamma+| descending (so the Reduce 1 filter
 *            |Gamma+| >= k-1 keeps a prefix of the queue); in the wider groups
 *            by the work estimate w(u) = sum over x in Gamma+(u) of
 *            |Gamma+(x)|, descending, compared after quantisation to
 *            q(w) = min(31, max(0, 2 b + f - 20)), b = floor(log2(w + 1))
 *            and f the bit of w + 1 below its leading one; ties by rank.
 * Any array may be NULL.  Errors: KC_EINVAL, KC_ECUDA.
 */
kc_status kc_export(const kc_graph* g, unsigned flags, int32_t* rank, int32_t* perm,
                    int64_t* off_plus, int32_t* adj_plus, int32_t* queue, void* stream);

/*
 * kc_count -- FFF_k Rounds 2-3 (Algorithm 1; Sec. 3): for every owner u with
 * |Gamma+(u)| >= k-1 (the Reduce 1 filter), build G+(u) (the pairs x_i < x_j
 * of Gamma+(u) that are edges: Map 2 / Reduce 2) and count its (k-1)-cliques
 * q_{u,k-1} (Reduce 3).  q_k is the sum over u (each clique is counted by its
 * smallest vertex, Sec. 3).
 *   k          1..KC_MAX_K; k = 1 gives n and k = 2 gives m (the paper's
 *              tables list n as q_1 and m as q_2)
 *   total      out: q_k.  Host pointer; with KC_DEVICE_PTRS a device array of
 *              two uint64 words (low, high) of the 128-bit sum, high != 0
 *              meaning the count overflowed
 *   per_vertex out array of n, nullable: number of k-cliques containing v
 *              (the per-node counts of Sec. 3, summed over all G+(u));
 *              their sum is k * q_k
 *   per_owner  out array of n, nullable: q_{u,k-1}, the Reduce 3 output of
 *              owner u; their sum is q_k
 * Both arrays are indexed by the caller's vertex ids.
 * Errors: KC_EINVAL (k out of range, g NULL), KC_ENOMEM, KC_EOVERFLOW,
 * KC_ETIMEOUT, KC_ECUDA.
 */
kc_status kc_count(const kc_graph* g, int k, unsigned flags, uint64_t* total,
                   uint64_t* per_vertex, uint64_t* per_owner, void* stream);

/*
 * kc_estimate -- cFFF_k (Sec. 6, "Color-based sampling"): every owner u colours
 * each x in Gamma+(u) with colour(u, x) in [0, colours), independently per
 * owner; Map 2 emits only monochromatic pairs; Reduce 3 counts the
 * (k-1)-cliques of the sampled G+(u).
 *   colour(u, x) = floor(h * colours / 2^64) with
 *   h = mix(seed XOR (0x9E3779B97F4A7C15 * ((uint64)u << 32 | x))), where
 *   mix is the splitmix64 output function (z ^= z>>30; z *= 0xBF58476D1CE4E5B9;
 *   z ^= z>>27; z *= 0x94D049BB133111EB; z ^= z>>31), and u, x are the
 *   caller's vertex ids.
 *   sampled    out: S = sum of the sampled per-owner counts (exact); with
 *              KC_DEVICE_PTRS a device array of two uint64 words (low, high)
 *   estimate   out, host pointer, nullable: S * colours^(k-2) rounded as
 *              fl(fl(S) * fl(colours^(k-2))) (the Reduce 3 scaling of Sec. 6);
 *              ignored with KC_DEVICE_PTRS
 *   per_owner  out array of n, nullable: sampled q_u of every owner
 *   colours    >= 1; colours = 1 gives exactly kc_count's q_k
 * Errors: as kc_count.
 */
kc_status kc_estimate(const kc_graph* g, int k, uint32_t colours, uint64_t seed,
                      unsigned flags, uint64_t* sampled, double* estimate,
                      uint64_t* per_owner, void* stream);

/*
 * kc_estimate_pairs -- plain pair sampling (Sec. 6, "Plain pair sampling",
 * analysed in App. B): Map 2 of owner u emits each pair x_i < x_j of
 * Gamma+(u) with probability p, independently of every other pair and of
 * every other owner; Reduce 3 counts the (k-1)-cliques of the sampled G+(u).
 * A clique is sampled when all C(k-1, 2) pairs among its non-owner members
 * were emitted, so S / p^((k-1)(k-2)/2) is an unbiased estimate of q_k.
 *   p          in (0, 1]; pair {x, y} of Gamma+(u) is kept iff h < thr with
 *              thr = floor(p * 2^64) (exact for p >= 2^-11) and
 *              h = mix(mix(seed XOR (G * ((uint64)u << 32 | a))) XOR (G * b)),
 *              G = 0x9E3779B97F4A7C15, mix the splitmix64 output function
 *              (as for kc_estimate), a < b the caller's ids of x and y, u the
 *              caller's id of the owner.  p = 1 keeps every pair (S = q_k).
 *   sampled    out: S = sum of the sampled per-owner counts (exact); with
 *              KC_DEVICE_PTRS a device array of two uint64 words (low, high)
 *   estimate   out, host pointer, nullable: fl(S) / P where P is
 *              p^((k-1)(k-2)/2) formed by repeated multiplication in double,
 *              starting from 1.0; ignored with KC_DEVICE_PTRS
 *   per_owner  out array of n, nullable: sampled q_u of every owner
 * Errors: KC_EINVAL also for p outside (0, 1] or NaN; otherwise as kc_count.
 */
kc_status kc_estimate_pairs(const kc_graph* g, int k, double p, uint64_t seed,
                            unsigned flags, uint64_t* sampled, double* estimate,
                            uint64_t* per_owner, void* stream);

/*
 * kc_list -- k-clique listing (the exact algorithm lists as well as counts,
 * Sec. 1; Reduce 3 of Sec. 3 enumerates the (k-1)-cliques of every G+(u)).
 * Every k-clique of G is delivered exactly once, as k caller ids ordered by
 * the total order of Sec. 2 (its smallest vertex, the owner u, first), in
 * runs of at most `cap` cliques: the library fills `buf` (cap * k int32,
 * row-major, one clique per row) with a run, then calls
 * fn(user, buf, count) on the calling thread with the run complete; after fn
 * returns the buffer is reused.  A run holds the cliques of consecutive
 * owners of the work queue, so the order of runs and of rows inside a run is
 * deterministic but unspecified.
 *   k        1..KC_MAX_K (k = 1: every vertex; k = 2: every edge)
 *   buf      host buffer, or with KC_DEVICE_PTRS a device buffer (fn then
 *            receives the device pointer; the run is complete on `stream`)
 *   cap      >= the largest per-owner count q_{u,k-1} (kc_count's per_owner
 *            output); a smaller cap returns KC_ENOMEM before anything is
 *            delivered from that owner
 *   fn       non-NULL; a non-zero return stops the listing (KC_ECANCELED)
 *   listed   out, host: number of cliques delivered to fn so far
 * Errors: KC_EINVAL (bad k, cap < 1, NULL argument), KC_ENOMEM, KC_ECANCELED,
 * KC_ECUDA.
 */
typedef int (*kc_list_fn)(void* user, const int32_t* cliques, int64_t count);
kc_status kc_list(const kc_graph* g, int k, unsigned flags, int32_t* buf, int64_t cap,
                  kc_list_fn fn, void* user, uint64_t* listed, void* stream);

/*
 * kc_round2_bytes -- the input volume of Round 2 for k (Sec. 3; App. B bounds
 * it): the bytes of the lists a count reads to build every G+(u) of an owner
 * u with |Gamma+(u)| >= k-1, namely 4 |Gamma+(x)| + 16 (the list and its
 * offsets) for each x in Gamma+(u), plus 4 |Gamma+(u)| for Gamma+(u) itself:
 * the sum over those owners of 4 w(u) + 20 |Gamma+(u)|, with
 * w(u) = sum over x in Gamma+(u) of |Gamma+(x)|.  Computed by one pass over
 * the oriented graph on `stream` (synchronous).
 *   bytes  out, host
 * Errors: KC_EINVAL, KC_ENOMEM, KC_ECUDA.
 */
kc_status kc_round2_bytes(const kc_graph* g, int k, uint64_t* bytes, void* stream);

/*
 * kc_footprint -- device memory a kc_count / kc_estimate call on g for k
 * allocates (stream-ordered) while it runs, for admission control.
 *   per_vertex, per_owner  nonzero if those outputs are requested
 *   host_outputs           nonzero if outputs are host arrays
 *   bytes                  out
 * Errors: KC_EINVAL.
 */
kc_status kc_footprint(const kc_graph* g, int k, int per_vertex, int per_owner, int host_outputs,
                       uint64_t* bytes);

/*
 * kc_count_part -- the share of kc_count contributed by one part of the
 * owners.  The owners are split into nparts parts by greedy LPT over the work
 * estimate w(u) = sum over x in Gamma+(u) of |Gamma+(x)|: taken by w(u)
 * descending (ties in queue order), each owner joins the part with the least
 * estimated work so far (ties: the lowest part), so the parts are balanced.
 * The partition is built on the first call for a given nparts (one pass over
 * the oriented graph and a host sort, synchronous on `stream`) and kept with
 * the graph.  Every clique is counted by exactly one owner (Sec. 3), so the
 * totals, per-vertex and per-owner arrays of parts 0..nparts-1 add up to
 * kc_count's.  This is how the count is sharded over GPUs (each GPU holds a
 * replica of the oriented graph and counts one part; the partial totals and
 * arrays are summed).
 *   k          3..KC_MAX_K
 *   part       0..nparts-1; other arguments as kc_count
 * Errors: as kc_count.
 */
kc_status kc_count_part(const kc_graph* g, int k, int part, int nparts, unsigned flags, uint64_t* total,
                        uint64_t* per_vertex, uint64_t* per_owner, void* stream);

/*
 * kc_count_batch -- kc_count's total for each of ng graphs (all on one
 * device) in a single launch sequence: the owners of all graphs form one
 * queue per owner class, so many small, uneven graphs fill the GPU together
 * instead of one launch each.  Uses the plan (kc_set_tuning) attached to
 * gs[0] for k without per-vertex output, if any.
 *   gs      host array of ng graph handles
 *   totals  out: host array of ng counts, or with KC_DEVICE_PTRS a device
 *           array of 2*ng words (low, high per graph)
 * Synchronous.  Errors: KC_EINVAL (a NULL handle, graphs on different
 * devices), KC_ENOMEM, KC_EOVERFLOW (some count), KC_ECUDA.
 */
kc_status kc_count_batch(const kc_graph* const* gs, int ng, int k, unsigned flags, uint64_t* totals,
                         void* stream);

/*
 * Tuning knobs (process-wide; they change speed, never results).
 *   KC_PARAM_SMEM_MAX_WORDS  owners whose bitmap rows need at most this many
 *       32-bit words (|Gamma+(u)| <= 32 * value) keep G+(u) in shared memory;
 *       wider owners use global-memory tiles.  1, 2, 4, 8, 16 or 32 (the
 *       queue's group widths), default 32.
 *   KC_PARAM_LAUNCH_COUNT  read: kernels launched by this process so far;
 *       write 0 to reset.
 *   KC_PARAM_WORK_COUNT  write 1 (0) to turn on (off) work counting in the
 *       counting kernels; read: bitmap word-operations (a 32-bit AND plus
 *       population count) executed by the last synchronous kc_count /
 *       kc_estimate on this process while counting was on.
 *   KC_PARAM_ALGO  the Reduce 3 counter used by kc_count / kc_estimate:
 *       KC_ALGO_DFS (default) enumerates ordered chains x_i1 < x_i2 < ... and
 *       closes the last two levels by population counts; KC_ALGO_PIVOT walks
 *       G+(u) with Bron-Kerbosch pivoting and counts each leaf by binomial
 *       coefficients (fewer nodes on near-complete G+(u)).  Both give
 *       identical results.
 *   KC_PARAM_COMPACT_LO, KC_PARAM_COMPACT_HI  candidate sets of the ordered
 *       search with LO..HI elements (HI <= 64, default 1..64; HI = 0 off) are
 *       finished on a compact register copy of their induced subgraph.
 *   KC_PARAM_TRI  1 (default): exact k = 3 counts take the triangle path --
 *       each y of Gamma+(x_i) found in Gamma+(u) is counted directly (node
 *       iterator, no G+(u) bitmap); 0: the bitmap path used for larger k.
 *   KC_PARAM_COMPLEMENT  1 (default): the ordered search of the 4-, 8- and
 *       16-word classes closes a candidate set C that still needs three
 *       vertices through the complement of G[C] when C is dense (non-edges
 *       below a quarter of the edges): the triangles through each v of C
 *       follow from the degrees in G[C] and the rows of v's non-neighbours,
 *       so only the rows of non-neighbours are read.  It needs symmetric
 *       rows: per-vertex counts have them, and totals at k >= 6 in those
 *       classes take them for this (their memberships are dropped).  0: every
 *       such set is closed on its edges (one row read per neighbour) and
 *       totals keep upper-triangular rows.
 * kc_set_param returns KC_EINVAL for an unknown knob or a value out of range.
 */
#define KC_PARAM_SMEM_MAX_WORDS 1
#define KC_PARAM_LAUNCH_COUNT   2
#define KC_PARAM_WORK_COUNT     3
#define KC_PARAM_ALGO           4
#define KC_PARAM_COMPACT_LO     5
#define KC_PARAM_COMPACT_HI     6
#define KC_PARAM_TRI            7
#define KC_PARAM_COMPLEMENT     8
#define KC_ALGO_PIVOT 0
#define KC_ALGO_DFS   1
kc_status kc_set_param(int param, int64_t value);
kc_status kc_get_param(int param, int64_t* value);

/*
 * kc_batch -- a batch of graphs prepared once for repeated counts at one k:
 * the per-class owner tables of kc_count_batch are built and uploaded at
 * creation, so kc_batch_count only launches kernels on its stream (no host
 * transfer, no synchronisation) and can be captured into a CUDA graph and
 * replayed.  The graphs must stay alive (and unchanged) while the batch is.
 *   kc_batch_create  gs, ng, k as kc_count_batch (k = 3..KC_MAX_K); flags 0;
 *                    uses the plan attached to gs[0] (kc_set_tuning) at
 *                    creation; synchronous on `stream`
 *   kc_batch_count   totals: device array of 2 * ng uint64 words (low, high
 *                    per graph; high != 0: overflow), overwritten; asynchronous
 *                    on `stream` (not the legacy default stream when captured)
 *   kc_batch_free    releases the batch (NULL ignored); no kc_batch_count of
 *                    it may still be running
 * Errors: KC_EINVAL, KC_ENOMEM, KC_ECUDA.
 */
typedef struct kc_batch kc_batch;
kc_status kc_batch_create(const kc_graph* const* gs, int ng, int k, unsigned flags, void* stream, kc_batch** out);
kc_status kc_batch_count(kc_batch* b, uint64_t* totals, void* stream);
void kc_batch_free(kc_batch* b);

/*
 * Autotuning (batching, owner classes).  The counting kernels take owners in
 * classes by the width of their bitmap row (the queue groups of kc_export):
 *   class 0: |Gamma+| above the shared-memory limit (global-memory tiles),
 *   classes 1..5: rows of 32, 16, 8, 4, 2 words (shared memory),
 *   class 6: rows of one word (registers).
 * For each class a plan names the Reduce 3 counter (KC_ALGO_DFS or
 * KC_ALGO_PIVOT, see KC_PARAM_ALGO) and, for the ordered search of classes
 * 1..5, the number of CTAs that share one owner (parts: 1 = no split; the
 * split owners' G+(u) is built once into a global tile).  A plan changes
 * speed only, never results.
 */
typedef struct {
    int32_t k;           /* the k the plan is for */
    int32_t per_vertex;  /* 1: for counts with per-vertex output, 0: without */
    int32_t algo[7];     /* per class: KC_ALGO_DFS or KC_ALGO_PIVOT */
    int32_t parts[7];    /* per class: CTAs per owner (ordered search), >= 1 */
    float ms[7];         /* per class: measured sample time of the choice (ms) */
} kc_tuning;

#define KC_TUNE_PER_VERTEX 0x10u  /* kc_tune: tune for counts with per-vertex output */

/*
 * kc_tune -- measure, for every owner class of the ng graphs (one graph:
 * ng = 1), the candidate plans -- the ordered search with 1, 4 or 16 parts
 * per owner (4 and 16 only for classes of 8+ words at k >= 5) and the
 * pivoting counter -- on a sample of the class's heaviest owners (its first
 * owners in queue order, at most 256), and return the fastest in `out`.  The
 * graphs are not changed (attach the plan with kc_set_tuning).  Runs
 * synchronously on `stream`.
 *   k      3..KC_MAX_K (k <= 2 needs no plan: out gets the defaults)
 *   flags  KC_TUNE_PER_VERTEX
 * Errors: KC_EINVAL, KC_ENOMEM, KC_ECUDA.
 */
kc_status kc_tune(const kc_graph* const* gs, int ng, int k, unsigned flags, void* stream, kc_tuning* out);

/*
 * kc_set_tuning -- attach a plan to g: later exact counts of g (kc_count,
 * kc_count_part, kc_list, kc_count_batch with g as its first graph) and
 * colour-sampled estimates (kc_estimate) for the plan's k and output mode
 * use it.  t = NULL removes every plan of g.
 * Errors: KC_EINVAL (bad k, algorithm or parts).
 */
kc_status kc_set_tuning(kc_graph* g, const kc_tuning* t);

/*
 * kc_count_csr / kc_estimate_csr -- one-shot forms: kc_orient, then kc_count
 * (or kc_estimate), then kc_free.  Arguments as above; KC_DEVICE_PTRS
 * applies to the inputs and the outputs alike.
 */
kc_status kc_count_csr(const int64_t* off, const int32_t* adj, int32_t n, int64_t m, int k,
                       unsigned flags, uint64_t* total, uint64_t* per_vertex,
                       uint64_t* per_owner, void* stream);
kc_status kc_estimate_csr(const int64_t* off, const int32_t* adj, int32_t n, int64_t m,
                          int k, uint32_t colours, uint64_t seed, unsigned flags,
                          uint64_t* sampled, double* estimate, void* stream);

/*
 * kc_count_static -- the total q_k of kc_count, computed without allocating
 * any device memory.  The paper has no counterpart: this is for callers that
 * cannot call cudaMalloc when they need a count -- a process whose memory
 * manager has already reserved the device and accounts for every byte, or
 * latency-critical code that must not wait on an allocation.
 *   g, k, flags, stream  as kc_count (k = 1..KC_MAX_K); no per-vertex or
 *              per-owner outputs
 *   total      out: q_k; host pointer, or with KC_DEVICE_PTRS a device array
 *              of two uint64 words (low, high)
 * Scratch comes from one 16 MiB __device__ array in the library, held by every
 * GPU that loads it until exit.  The first call on each device looks up the
 * array's device address, and under lazy module loading (the CUDA default)
 * that is also when the array's 16 MiB are committed on the device: make one
 * warm-up call (any graph, k = 3) at start-up, before the caller's memory
 * manager reserves the device and before any stream capture.  All calls
 * share the array: calls that overlap on the GPU race and must be serialised
 * by the caller.  A graph whose widest owner needs a global tile larger than
 * the array returns KC_ENOTSUP without running (never for exact k = 3 with
 * the triangle path on, which uses no tiles).  Owners are not split across
 * CTAs here (the split needs per-call tiles).
 * Errors: as kc_count, plus KC_ENOTSUP.
 */
kc_status kc_count_static(const kc_graph* g, int k, unsigned flags, uint64_t* total, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* KC_H */
