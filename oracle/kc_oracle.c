/*
 * kc_oracle.c -- plain CPU oracle for k-clique counting by the exact algorithm
 * FFF_k and the colour-sampling estimator cFFF_k of Finocchi, Finocchi &
 * Fusco, "Clique counting in MapReduce: theory and experiments".
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this library.  It shares no code, header, table or
 * helper with the CUDA library, and it is deliberately plain and slow: every
 * step follows the paper's definitions in the paper's order, with no blocking,
 * bitmaps, relabelling or reordering.
 *
 * Input convention (the paper's preprocessed input, Sec. 4): an undirected
 * simple graph as a CSR, off[n+1] int64 and adj[off[n]] int32, every edge
 * stored in both directions, rows sorted ascending by vertex id, no
 * self-loops, no repeats.  Vertex ids are the "comparable labels" of Sec. 2.
 *
 * Pins (tests/test_oracle.py): brute force over all k-subsets, closed forms
 * for complete and complete multipartite graphs, invariants (sum of
 * memberships = k * q_k, sum of owner counts = q_k), relabelling invariance,
 * and exhaustive colourings for the estimator's expectation.
 *
 * Status codes: 0 ok, 1 count overflowed uint64, 2 invalid argument,
 * 3 out of memory.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

enum { OR_OK = 0, OR_OVERFLOW = 1, OR_EINVAL = 2, OR_ENOMEM = 3 };

/* ----------------------------------------------------------- Sec. 2 */

/* d(u) = |Gamma(u)| */
static int64_t degree(const int64_t* off, int32_t u) { return off[u + 1] - off[u]; }

/* x precedes y iff d(x) < d(y), or d(x) = d(y) and x < y  (Sec. 2) */
static int precedes(const int64_t* off, int32_t x, int32_t y)
{
    int64_t dx = degree(off, x), dy = degree(off, y);
    return dx < dy || (dx == dy && x < y);
}

int oracle_precedes(const int64_t* off, int32_t x, int32_t y) { return precedes(off, x, y); }

/* (x, y) is an edge: y appears in the sorted row of x (binary search). */
static int adjacent(const int64_t* off, const int32_t* adj, int32_t x, int32_t y)
{
    int64_t lo = off[x], hi = off[x + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (adj[mid] < y) lo = mid + 1;
        else hi = mid;
    }
    return lo < off[x + 1] && adj[lo] == y;
}

/* Stable merge sort of vertex ids by the total order (needs scratch of len). */
static void sort_by_order(const int64_t* off, int32_t* a, int32_t* tmp, int64_t len)
{
    if (len < 2) return;
    int64_t h = len / 2;
    sort_by_order(off, a, tmp, h);
    sort_by_order(off, a + h, tmp, len - h);
    int64_t i = 0, j = h, t = 0;
    while (i < h && j < len) tmp[t++] = precedes(off, a[j], a[i]) ? a[j++] : a[i++];
    while (i < h) tmp[t++] = a[i++];
    while (j < len) tmp[t++] = a[j++];
    memcpy(a, tmp, (size_t)len * sizeof(int32_t));
}

/* All vertices listed in increasing order of precedence. */
int oracle_order(const int64_t* off, int32_t n, int32_t* order)
{
    int32_t* tmp = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!tmp) return OR_ENOMEM;
    for (int32_t v = 0; v < n; ++v) order[v] = v;
    sort_by_order(off, order, tmp, n);
    free(tmp);
    return OR_OK;
}

/* High-neighbourhood Gamma+(u) = {x in Gamma(u) : u precedes x} (Sec. 2),
 * listed in increasing order of precedence.  `out` needs room for d(u);
 * `tmp` likewise.  Returns |Gamma+(u)|. */
static int32_t gamma_plus(const int64_t* off, const int32_t* adj, int32_t u,
                          int32_t* out, int32_t* tmp)
{
    int32_t len = 0;
    for (int64_t e = off[u]; e < off[u + 1]; ++e)
        if (precedes(off, u, adj[e])) out[len++] = adj[e];
    sort_by_order(off, out, tmp, len);
    return len;
}

int32_t oracle_gamma_plus(const int64_t* off, const int32_t* adj, int32_t u, int32_t* out)
{
    int64_t d = degree(off, u);
    int32_t* tmp = (int32_t*)malloc((size_t)(d > 0 ? d : 1) * sizeof(int32_t));
    if (!tmp) return -1;
    int32_t len = gamma_plus(off, adj, u, out, tmp);
    free(tmp);
    return len;
}

/* ------------------------------------------------ cFFF colour (Sec. 6) */

/* Colour of x in the colouring of Gamma+(u): every (owner, node) pair gets an
 * independent colour (the paper colours the nodes of each Gamma+(u)
 * separately, App. B).  Counter-based: z = seed XOR (G * key) with
 * key = u<<32 | x and G = 0x9E3779B97F4A7C15, mixed by the splitmix64 output
 * function (Steele, Lea & Flood 2014), then mapped to [0, c) by the
 * multiply-high reduction floor(z * c / 2^64) (Lemire 2019). */
static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t oracle_colour_hash(uint64_t seed, int32_t u, int32_t x)
{
    uint64_t key = ((uint64_t)(uint32_t)u << 32) | (uint64_t)(uint32_t)x;
    return mix64(seed ^ (0x9E3779B97F4A7C15ULL * key));
}

uint32_t oracle_colour(uint64_t seed, int32_t u, int32_t x, uint32_t c)
{
    return (uint32_t)(((u128)oracle_colour_hash(seed, u, x) * (u128)c) >> 64);
}

/* ---------------------------------- plain pair sampling (Sec. 6) */

/* Map 2 of owner u emits the pair {x, y} of Gamma+(u) with probability p,
 * independently per pair and per owner (Sec. 6, App. B).  Counter-based: with
 * a < b the two ids, h = mix(mix(seed XOR G * (u<<32 | a)) XOR G * b), and the
 * pair is emitted iff h < thr, thr = floor(p * 2^64) (p < 1). */
uint64_t oracle_pair_hash(uint64_t seed, int32_t u, int32_t x, int32_t y)
{
    uint32_t a = (uint32_t)x < (uint32_t)y ? (uint32_t)x : (uint32_t)y;
    uint32_t b = (uint32_t)x < (uint32_t)y ? (uint32_t)y : (uint32_t)x;
    uint64_t z = mix64(seed ^ (0x9E3779B97F4A7C15ULL * (((uint64_t)(uint32_t)u << 32) | a)));
    return mix64(z ^ (0x9E3779B97F4A7C15ULL * (uint64_t)b));
}

/* floor(p * 2^64) for 0 < p < 1 (the product by a power of two is exact). */
uint64_t oracle_pair_threshold(double p)
{
    return (uint64_t)(p * 18446744073709551616.0);
}

/* Estimate of plain pair sampling: fl(S) / p^((k-1)(k-2)/2), the power formed
 * by repeated multiplication in double starting from 1.0 (Sec. 6). */
double oracle_scale_pairs(uint64_t sampled, double p, int k)
{
    double f = 1.0;
    for (int i = 0; i < (k - 1) * (k - 2) / 2; ++i) f *= p;
    return (double)sampled / f;
}

/* -------------------------------------- Reduce 3: cliques in G+(u) */

typedef struct {
    int k;                 /* clique size being counted in G */
    const int32_t* L;      /* Gamma+(u) in precedence order (original ids) */
    int32_t** out;         /* out[i]: local j > i with (x_i, x_j) kept, ascending */
    int32_t* outlen;
    int32_t* chain;        /* local ids chosen so far below the current level */
    int32_t u;
    uint64_t* per_vertex;  /* nullable: membership counts, atomically updated */
    int overflow;
    int listing;           /* enumerate the cliques (count them in list_n) */
    int32_t* list;         /* nullable: listing output, k ids per clique */
    int64_t list_cap, list_n;
} rec_ctx;

static void add_u64(uint64_t* p, uint64_t v, int* overflow)
{
    uint64_t old;
#ifdef _OPENMP
#pragma omp atomic capture
#endif
    { old = *p; *p += v; }
    if (old + v < old) *overflow = 1;
}

/* Number of cliques of size (k - s) to be completed inside `cand`, a set of
 * local ids all adjacent (in G+(u)) to the s vertices already chosen (u and
 * chain[0..s-2]).  When s == k-1 each candidate completes one k-clique: the
 * leaves are enumerated one by one and credited to their members. */
static u128 count_rec(rec_ctx* c, const int32_t* cand, int32_t ncand, int s)
{
    if (s == c->k - 1) {
        if (c->listing) {  /* listing: u, the chain, then each candidate */
            for (int32_t i = 0; i < ncand; ++i, ++c->list_n) {
                if (!c->list || c->list_n >= c->list_cap) continue;
                int32_t* row = c->list + c->list_n * c->k;
                row[0] = c->u;
                for (int t = 0; t < s - 1; ++t) row[1 + t] = c->L[c->chain[t]];
                row[c->k - 1] = c->L[cand[i]];
            }
        }
        if (c->per_vertex && ncand > 0) {
            add_u64(&c->per_vertex[c->u], (uint64_t)ncand, &c->overflow);
            for (int t = 0; t < s - 1; ++t)
                add_u64(&c->per_vertex[c->L[c->chain[t]]], (uint64_t)ncand, &c->overflow);
            for (int32_t i = 0; i < ncand; ++i)
                add_u64(&c->per_vertex[c->L[cand[i]]], 1, &c->overflow);
        }
        return (u128)ncand;
    }
    u128 total = 0;
    int32_t* next = (int32_t*)malloc((size_t)(ncand > 0 ? ncand : 1) * sizeof(int32_t));
    if (!next) { c->overflow = -1; return 0; }
    for (int32_t a = 0; a < ncand; ++a) {
        int32_t x = cand[a];
        /* cand intersected with out[x]: both ascending, sorted merge */
        int32_t nn = 0, i = 0, j = 0;
        const int32_t* ox = c->out[x];
        while (i < ncand && j < c->outlen[x]) {
            if (cand[i] < ox[j]) ++i;
            else if (cand[i] > ox[j]) ++j;
            else { next[nn++] = cand[i]; ++i; ++j; }
        }
        c->chain[s - 1] = x;
        total += count_rec(c, next, nn, s + 1);
    }
    free(next);
    return total;
}

/* FFF_k, cFFF_k or plain pair sampling work for one owner u: Round 1 gives
 * Gamma+(u); Reduce 1 drops u when |Gamma+(u)| < k-1; Map 2 emits the pairs
 * x_i precedes x_j of Gamma+(u) (only monochromatic pairs under cFFF_k, only
 * the pairs whose coin came up under pair sampling, Sec. 6); Reduce 2 keeps a
 * pair when it is an edge of G (the "$" marker); Reduce 3 counts the
 * (k-1)-cliques of the resulting G+(u).  An explicit colour array or kept-pair
 * matrix (indexed like Gamma+(u)) overrides the hash when given. */
typedef struct {
    uint32_t colours;             /* cFFF_k: >= 1 colours (0: no colouring) */
    uint64_t seed;
    const uint32_t* given_colour; /* explicit colouring of Gamma+(u), or NULL */
    int pair;                     /* plain pair sampling with threshold pthr */
    uint64_t pthr;
    const uint8_t* given_kept;    /* explicit emitted pairs (d+ x d+, row i, column j > i), or NULL */
} sampler;

static int owner_work_list(const int64_t* off, const int32_t* adj, int32_t u, int k,
                           const sampler* sm, uint64_t* per_vertex, u128* q_u,
                           int32_t* list, int64_t list_cap, int64_t* list_n);

static int owner_work(const int64_t* off, const int32_t* adj, int32_t u, int k,
                      const sampler* sm, uint64_t* per_vertex, u128* q_u)
{
    return owner_work_list(off, adj, u, k, sm, per_vertex, q_u, NULL, 0, NULL);
}

static int owner_work_list(const int64_t* off, const int32_t* adj, int32_t u, int k,
                           const sampler* sm, uint64_t* per_vertex, u128* q_u,
                           int32_t* list, int64_t list_cap, int64_t* list_n)
{
    uint32_t colours = sm->colours;
    uint64_t seed = sm->seed;
    const uint32_t* given_colour = sm->given_colour;
    *q_u = 0;
    int64_t d = degree(off, u);
    int32_t* L = (int32_t*)malloc((size_t)(d > 0 ? d : 1) * sizeof(int32_t));
    int32_t* tmp = (int32_t*)malloc((size_t)(d > 0 ? d : 1) * sizeof(int32_t));
    if (!L || !tmp) { free(L); free(tmp); return OR_ENOMEM; }
    int32_t dp = gamma_plus(off, adj, u, L, tmp);
    free(tmp);
    if (dp < k - 1) { free(L); return OR_OK; } /* Reduce 1 filter */

    uint32_t* col = NULL;
    if (given_colour || colours >= 1) {
        col = (uint32_t*)malloc((size_t)(dp > 0 ? dp : 1) * sizeof(uint32_t));
        if (!col) { free(L); return OR_ENOMEM; }
        for (int32_t i = 0; i < dp; ++i)
            col[i] = given_colour ? given_colour[i] : oracle_colour(seed, u, L[i], colours);
    }
    int32_t** out = (int32_t**)calloc((size_t)(dp > 0 ? dp : 1), sizeof(int32_t*));
    int32_t* outlen = (int32_t*)calloc((size_t)(dp > 0 ? dp : 1), sizeof(int32_t));
    int32_t* chain = (int32_t*)malloc((size_t)(k > 0 ? k : 1) * sizeof(int32_t));
    int32_t* all = (int32_t*)calloc((size_t)(dp > 0 ? dp : 1), sizeof(int32_t));
    int st = OR_OK;
    if (!out || !outlen || !chain || !all) { st = OR_ENOMEM; goto done; }
    if (k >= 3) {
        for (int32_t i = 0; i < dp; ++i) {
            out[i] = (int32_t*)malloc((size_t)(dp - i > 0 ? dp - i : 1) * sizeof(int32_t));
            if (!out[i]) { st = OR_ENOMEM; goto done; }
            for (int32_t j = i + 1; j < dp; ++j) {
                if (col && col[i] != col[j]) continue;          /* Map 2 sampling */
                if (sm->given_kept && !sm->given_kept[(int64_t)i * dp + j]) continue;
                if (!sm->given_kept && sm->pair &&
                    oracle_pair_hash(sm->seed, u, L[i], L[j]) >= sm->pthr) continue;
                if (adjacent(off, adj, L[i], L[j]))            /* Reduce 2 "$" */
                    out[i][outlen[i]++] = j;
            }
        }
    }
    for (int32_t i = 0; i < dp; ++i) all[i] = i;
    rec_ctx c = { k, L, out, outlen, chain, u, per_vertex, 0, list_n != NULL, list, list_cap, list_n ? *list_n : 0 };
    *q_u = count_rec(&c, all, dp, 1);                            /* Reduce 3 */
    if (list_n) *list_n = c.list_n;
    if (c.overflow < 0) st = OR_ENOMEM;
    else if (c.overflow) st = OR_OVERFLOW;
done:
    if (out) for (int32_t i = 0; i < dp; ++i) free(out[i]);
    free(out); free(outlen); free(chain); free(all); free(col); free(L);
    return st;
}

/* Count (or estimate) over owners u in [u_lo, u_hi).
 *   k >= 1; colours == 0 means exact FFF_k, colours >= 1 cFFF_k with that many
 *   colours (colours == 1 reproduces FFF_k).
 *   total_lo/total_hi: the 128-bit sum of the per-owner counts (for cFFF_k the
 *   sampled count S, before scaling by c^(k-2)).
 *   per_owner[n], per_vertex[n]: nullable; accumulated (+=), so zero them.
 *   nthreads: OpenMP threads over owners (<= 0: library default).
 * k = 1 counts vertices (q_1 = n) and k = 2 edges (q_2 = m), as in the
 * paper's tables. */
static int fff_run(const int64_t* off, const int32_t* adj, int32_t n, int k,
                   const sampler* sm, int32_t u_lo, int32_t u_hi,
                   int nthreads, uint64_t* total_lo, uint64_t* total_hi,
                   uint64_t* per_owner, uint64_t* per_vertex)
{
    if (n < 0 || k < 1 || u_lo < 0 || u_hi > n || u_lo > u_hi) return OR_EINVAL;
    u128 total = 0;
    int st = OR_OK;
    if (k == 1) {
        for (int32_t u = u_lo; u < u_hi; ++u) {
            total += 1;
            if (per_owner) per_owner[u] += 1;
            if (per_vertex) per_vertex[u] += 1;
        }
    } else {
#ifdef _OPENMP
        if (nthreads > 0) omp_set_num_threads(nthreads);
#else
        (void)nthreads;
#endif
        int nt = 1;
#ifdef _OPENMP
        nt = omp_get_max_threads();
#endif
        u128* part = (u128*)calloc((size_t)nt, sizeof(u128));
        if (!part) return OR_ENOMEM;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
        for (int32_t u = u_lo; u < u_hi; ++u) {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            u128 q = 0;
            int s = owner_work(off, adj, u, k, sm, per_vertex, &q);
            if (s != OR_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
                { if (st == OR_OK) st = s; }
            }
            part[tid] += q;
            if (per_owner) {
                if (q >> 64) {
#ifdef _OPENMP
#pragma omp critical
#endif
                    { if (st == OR_OK) st = OR_OVERFLOW; }
                }
                per_owner[u] += (uint64_t)q;
            }
        }
        for (int t = 0; t < nt; ++t) total += part[t];
        free(part);
    }
    *total_lo = (uint64_t)total;
    *total_hi = (uint64_t)(total >> 64);
    if (st == OR_OK && *total_hi) st = OR_OVERFLOW;
    return st;
}

int oracle_fff(const int64_t* off, const int32_t* adj, int32_t n, int k,
               uint32_t colours, uint64_t seed, int32_t u_lo, int32_t u_hi,
               int nthreads, uint64_t* total_lo, uint64_t* total_hi,
               uint64_t* per_owner, uint64_t* per_vertex)
{
    sampler sm = { colours, seed, NULL, 0, 0, NULL };
    return fff_run(off, adj, n, k, &sm, u_lo, u_hi, nthreads, total_lo, total_hi, per_owner, per_vertex);
}

/* Exact FFF_k Reduce 3 counts q_{u,k-1} of an explicit list of owners (Sec. 3:
 * each clique is counted by its smallest vertex), one owner per OpenMP task:
 * out[i] = q_{owners[i],k-1}.  The same per-owner routine as oracle_fff; this
 * only lets a test check scattered owners of a large graph without running
 * every owner in between. */
int oracle_fff_owners(const int64_t* off, const int32_t* adj, int32_t n, int k,
                      const int32_t* owners, int32_t nowners, int nthreads, uint64_t* out)
{
    if (n < 0 || k < 1 || nowners < 0 || (nowners > 0 && (!owners || !out))) return OR_EINVAL;
    for (int32_t i = 0; i < nowners; ++i)
        if (owners[i] < 0 || owners[i] >= n) return OR_EINVAL;
    int st = OR_OK;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#else
    (void)nthreads;
#endif
    for (int32_t i = 0; i < nowners; ++i) {
        u128 q = 0;
        int s = OR_OK;
        if (k == 1) q = 1;
        else s = owner_work(off, adj, owners[i], k, &(sampler){ 0, 0, NULL, 0, 0, NULL }, NULL, &q);
        if (s == OR_OK && (q >> 64)) s = OR_OVERFLOW;
        if (s != OR_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
            { if (st == OR_OK) st = s; }
        }
        out[i] = (uint64_t)q;
    }
    return st;
}

/* Plain pair sampling (Sec. 6) over owners u in [u_lo, u_hi): the sampled
 * count S (before scaling) and per-owner sampled counts; p in (0, 1], p = 1
 * emits every pair. */
int oracle_fff_pairs(const int64_t* off, const int32_t* adj, int32_t n, int k,
                     double p, uint64_t seed, int32_t u_lo, int32_t u_hi,
                     int nthreads, uint64_t* total_lo, uint64_t* total_hi,
                     uint64_t* per_owner)
{
    if (!(p > 0.0 && p <= 1.0)) return OR_EINVAL;
    sampler sm = { 0, seed, NULL, p < 1.0, p < 1.0 ? oracle_pair_threshold(p) : 0, NULL };
    return fff_run(off, adj, n, k, &sm, u_lo, u_hi, nthreads, total_lo, total_hi, per_owner, NULL);
}

/* Reduce 3 output for one owner u under an explicit colouring of Gamma+(u)
 * (colour[i] is the colour of the i-th element in precedence order). */
int oracle_owner_coloured(const int64_t* off, const int32_t* adj, int32_t u, int k,
                          const uint32_t* colour, uint64_t* q_lo, uint64_t* q_hi)
{
    u128 q = 0;
    sampler sm = { 0, 0, colour, 0, 0, NULL };
    int st = owner_work(off, adj, u, k, &sm, NULL, &q);
    *q_lo = (uint64_t)q;
    *q_hi = (uint64_t)(q >> 64);
    return st;
}

/* Reduce 3 output for one owner u when Map 2 emitted exactly the pairs with
 * kept[i * d + j] != 0 (i < j indices of Gamma+(u) in precedence order,
 * d = |Gamma+(u)|). */
int oracle_owner_pairs(const int64_t* off, const int32_t* adj, int32_t u, int k,
                       const uint8_t* kept, uint64_t* q_lo, uint64_t* q_hi)
{
    u128 q = 0;
    sampler sm = { 0, 0, NULL, 1, 0, kept };
    int st = owner_work(off, adj, u, k, &sm, NULL, &q);
    *q_lo = (uint64_t)q;
    *q_hi = (uint64_t)(q >> 64);
    return st;
}

/* cFFF_k estimate: S * c^(k-2) rounded to double as fl(fl(S) * fl(c^(k-2))),
 * with c^(k-2) formed by repeated multiplication in double (Sec. 6). */
double oracle_scale_estimate(uint64_t sampled, uint32_t colours, int k)
{
    double f = 1.0;
    for (int i = 0; i < k - 2; ++i) f *= (double)colours;
    return (double)sampled * f;
}

/* ------------------------------------------------------- listing */

/* Every k-clique once (Reduce 3 enumerates the (k-1)-cliques of each G+(u),
 * Sec. 3), as k ids in precedence order, owner first: k = 1 lists every
 * vertex, k = 2 every edge (u, x) with u preceding x.  Owners in id order,
 * single-threaded.  Writes at most cap rows; *count receives the number of
 * cliques (which may exceed cap). */
int oracle_list(const int64_t* off, const int32_t* adj, int32_t n, int k,
                int32_t* out, int64_t cap, int64_t* count)
{
    if (n < 0 || k < 1 || cap < 0) return OR_EINVAL;
    int64_t nl = 0;
    for (int32_t u = 0; u < n; ++u) {
        if (k == 1) {
            if (nl < cap) out[nl] = u;
            ++nl;
            continue;
        }
        if (k == 2) {
            for (int64_t p = off[u]; p < off[u + 1]; ++p) {
                int32_t x = adj[p];
                if (!precedes(off, u, x)) continue;
                if (nl < cap) { out[2 * nl] = u; out[2 * nl + 1] = x; }
                ++nl;
            }
            continue;
        }
        sampler sm = { 0, 0, NULL, 0, 0, NULL };
        u128 q = 0;
        int st = owner_work_list(off, adj, u, k, &sm, NULL, &q, out, cap, &nl);
        if (st != OR_OK) return st;
    }
    *count = nl;
    return OR_OK;
}

/* ------------------------------------------------------- brute force */

/* Definition of q_k: the number of k-subsets of V that are cliques.  Every
 * k-subset v_1 < ... < v_k is visited in lexicographic order and all of its
 * C(k,2) pairs are tested in a dense adjacency matrix (n <= 4096).  No degree
 * order and no orientation are involved.  per_vertex (nullable) receives
 * |{S : v in S}|. */
int oracle_brute_force(const int64_t* off, const int32_t* adj, int32_t n, int k,
                       uint64_t* total_lo, uint64_t* total_hi, uint64_t* per_vertex)
{
    if (n < 0 || n > 4096 || k < 1 || k > 16) return OR_EINVAL;
    *total_lo = *total_hi = 0;
    if (k > n) return OR_OK;
    uint8_t* A = (uint8_t*)calloc((size_t)n * (size_t)n + 1, 1);
    if (!A) return OR_ENOMEM;
    for (int32_t v = 0; v < n; ++v)
        for (int64_t e = off[v]; e < off[v + 1]; ++e) A[(size_t)v * n + adj[e]] = 1;
    int32_t s[16];
    for (int i = 0; i < k; ++i) s[i] = i;
    u128 total = 0;
    for (;;) {
        int ok = 1;
        for (int i = 0; i < k && ok; ++i)
            for (int j = i + 1; j < k; ++j)
                if (!A[(size_t)s[i] * n + s[j]]) { ok = 0; break; }
        if (ok) {
            total += 1;
            if (per_vertex) for (int i = 0; i < k; ++i) per_vertex[s[i]] += 1;
        }
        /* next k-combination of {0..n-1} in lexicographic order */
        int i = k - 1;
        while (i >= 0 && s[i] == n - k + i) --i;
        if (i < 0) break;
        s[i]++;
        for (int j = i + 1; j < k; ++j) s[j] = s[j - 1] + 1;
    }
    free(A);
    *total_lo = (uint64_t)total;
    *total_hi = (uint64_t)(total >> 64);
    return OR_OK;
}

/* Number of worker threads OpenMP would use (1 without OpenMP). */
int oracle_max_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}
