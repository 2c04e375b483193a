/*
 * kcgen.c -- seeded synthetic graph generators.
 *
 * These generators are shared input plumbing: they produce the graphs that
 * both the CUDA library and the CPU oracle are run on.  They hold none of the
 * clique-counting arithmetic (no degree order, no orientation, no counting).
 *
 * Every generator returns a canonical undirected simple graph as a CSR:
 *   off[n+1] (int64), adj[off[n]] (int32), every edge stored in both
 *   directions, rows sorted ascending, no self-loops, no duplicates.
 * That is the input convention the paper assumes after its preprocessing
 * (Sec. 4: graphs made undirected; isolated nodes allowed).
 *
 * Determinism: all randomness comes from xoshiro256** (Blackman & Vigna,
 * 2018) seeded through splitmix64 (Steele, Lea & Flood, 2014).  Floating
 * point is restricted to +,-,*,/ (correctly rounded in IEEE-754) plus the
 * series-based log/exp below, and the file is compiled with
 * -ffp-contract=off, so x86-64 and aarch64 produce bit-identical graphs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------ RNG */

static uint64_t sm64_next(uint64_t* state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } kg_rng;

static uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static void rng_seed(kg_rng* r, uint64_t seed)
{
    uint64_t st = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = sm64_next(&st);
}

static uint64_t rng_next(kg_rng* r)
{
    uint64_t* s = r->s;
    const uint64_t result = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

/* Uniform integer in [0, bound), bound >= 1, by rejection (no modulo bias). */
static uint64_t rng_below(kg_rng* r, uint64_t bound)
{
    uint64_t lim = (uint64_t)(-bound) % bound; /* 2^64 mod bound */
    for (;;) {
        uint64_t x = rng_next(r);
        if (x >= lim) return x % bound;
    }
}

/* Bernoulli(p) with p given as a 53-bit fixed-point threshold. */
static int rng_bernoulli(kg_rng* r, uint64_t thresh53)
{
    return (rng_next(r) >> 11) < thresh53;
}

static uint64_t prob_to_thresh53(double p)
{
    if (p <= 0.0) return 0;
    if (p >= 1.0) return (uint64_t)1 << 53;
    return (uint64_t)(p * 9007199254740992.0); /* p * 2^53, exact scaling */
}

/* Exported for the generator's own tests (pinned against published values). */
uint64_t kg_splitmix64_output(uint64_t state) { return sm64_next(&state); }
uint64_t kg_xoshiro_first(uint64_t seed)
{
    kg_rng r;
    rng_seed(&r, seed);
    return rng_next(&r);
}

/* --------------------------------------- deterministic log / exp / pow */

static const double KG_LN2 = 0.6931471805599453094172321214581765680755;

/* ln(x) for finite x > 0: x = m * 2^e with m in [1/sqrt2, sqrt2), then
 * ln m = 2 atanh(s), s = (m-1)/(m+1), summed as an odd power series. */
static double kg_log(double x)
{
    int e;
    double m = frexp(x, &e); /* exact: m in [0.5, 1) */
    if (m < 0.70710678118654752440) { m *= 2.0; e -= 1; }
    double s = (m - 1.0) / (m + 1.0);
    double s2 = s * s, term = s, sum = 0.0;
    for (int k = 1; k < 60; k += 2) {
        double t = term / (double)k;
        sum += t;
        if (t < 1e-20 && t > -1e-20) break;
        term *= s2;
    }
    return 2.0 * sum + (double)e * KG_LN2;
}

/* exp(y): y = j ln2 + r with |r| <= ln2/2, exp(r) by its Taylor series. */
static double kg_exp(double y)
{
    double jf = y / KG_LN2;
    long j = (long)(jf >= 0 ? jf + 0.5 : jf - 0.5);
    double r = y - (double)j * KG_LN2;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 40; ++k) {
        term = term * r / (double)k;
        sum += term;
        if (term < 1e-20 && term > -1e-20) break;
    }
    return ldexp(sum, (int)j);
}

static double kg_pow(double x, double y) { return kg_exp(y * kg_log(x)); }

double kg_pow_export(double x, double y) { return kg_pow(x, y); }

/* ------------------------------------------------- radix sort (uint64) */

/* LSD radix sort, 16-bit digits; passes whose digit is constant are skipped. */
static int radix_sort_u64(uint64_t* a, int64_t n)
{
    if (n <= 1) return 0;
    uint64_t* tmp = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
    int64_t* cnt = (int64_t*)malloc(65536 * sizeof(int64_t));
    if (!tmp || !cnt) { free(tmp); free(cnt); return -1; }
    uint64_t* src = a;
    uint64_t* dst = tmp;
    for (int pass = 0; pass < 4; ++pass) {
        int sh = 16 * pass;
        memset(cnt, 0, 65536 * sizeof(int64_t));
        for (int64_t i = 0; i < n; ++i) cnt[(src[i] >> sh) & 0xFFFF]++;
        int trivial = 0;
        for (int d = 0; d < 65536; ++d)
            if (cnt[d] == n) { trivial = 1; break; }
        if (trivial) continue;
        int64_t acc = 0;
        for (int d = 0; d < 65536; ++d) { int64_t c = cnt[d]; cnt[d] = acc; acc += c; }
        for (int64_t i = 0; i < n; ++i) dst[cnt[(src[i] >> sh) & 0xFFFF]++] = src[i];
        uint64_t* t = src; src = dst; dst = t;
    }
    if (src != a) memcpy(a, src, (size_t)n * sizeof(uint64_t));
    free(tmp);
    free(cnt);
    return 0;
}

/* ----------------------------------------------------- CSR construction */

typedef struct {
    int32_t n;
    int64_t m;        /* undirected edges after canonicalisation */
    int64_t* off;     /* n+1 */
    int32_t* adj;     /* 2m  */
} kg_graph;

void kg_free(kg_graph* g)
{
    if (!g) return;
    free(g->off);
    free(g->adj);
    free(g);
}

/* Canonicalise an undirected edge-key list (keys lo<<32|hi, lo<hi, repeats
 * allowed) into a kg_graph.  Consumes `keys` (freed). */
static kg_graph* graph_from_keys(int32_t n, uint64_t* keys, int64_t nk)
{
    kg_graph* g = (kg_graph*)calloc(1, sizeof(kg_graph));
    if (!g) { free(keys); return NULL; }
    g->n = n;
    if (radix_sort_u64(keys, nk) != 0) { free(keys); free(g); return NULL; }
    int64_t m = 0;
    for (int64_t i = 0; i < nk; ++i)
        if (i == 0 || keys[i] != keys[m - 1]) keys[m++] = keys[i];
    g->m = m;
    /* both directions as keys row<<32|col; sorting them gives sorted rows */
    uint64_t* dir = (uint64_t*)malloc((size_t)(2 * m > 0 ? 2 * m : 1) * sizeof(uint64_t));
    g->off = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    g->adj = (int32_t*)malloc((size_t)(2 * m > 0 ? 2 * m : 1) * sizeof(int32_t));
    if (!dir || !g->off || !g->adj) { free(dir); free(keys); kg_free(g); return NULL; }
    for (int64_t i = 0; i < m; ++i) {
        uint64_t a = keys[i] >> 32, b = keys[i] & 0xFFFFFFFFu;
        dir[2 * i] = (a << 32) | b;
        dir[2 * i + 1] = (b << 32) | a;
    }
    free(keys);
    if (radix_sort_u64(dir, 2 * m) != 0) { free(dir); kg_free(g); return NULL; }
    for (int64_t i = 0; i < 2 * m; ++i) {
        g->off[(dir[i] >> 32) + 1]++;
        g->adj[i] = (int32_t)(dir[i] & 0xFFFFFFFFu);
    }
    free(dir);
    for (int32_t v = 0; v < n; ++v) g->off[v + 1] += g->off[v];
    return g;
}

static uint64_t edge_key(int32_t a, int32_t b)
{
    uint32_t lo = (uint32_t)(a < b ? a : b), hi = (uint32_t)(a < b ? b : a);
    return ((uint64_t)lo << 32) | hi;
}

/* Build a canonical CSR from an arbitrary edge list (either direction,
 * self-loops and duplicates allowed; they are removed).  Returns NULL on
 * allocation failure or an out-of-range endpoint. */
kg_graph* kg_from_edges(int32_t n, const int32_t* src, const int32_t* dst, int64_t ne)
{
    uint64_t* keys = (uint64_t*)malloc((size_t)(ne > 0 ? ne : 1) * sizeof(uint64_t));
    if (!keys) return NULL;
    int64_t nk = 0;
    for (int64_t i = 0; i < ne; ++i) {
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) { free(keys); return NULL; }
        if (src[i] == dst[i]) continue;
        keys[nk++] = edge_key(src[i], dst[i]);
    }
    return graph_from_keys(n, keys, nk);
}

/* Relabel vertex ids by a seeded uniform permutation (Fisher-Yates). */
static int32_t* random_permutation(int32_t n, kg_rng* r)
{
    int32_t* p = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!p) return NULL;
    for (int32_t i = 0; i < n; ++i) p[i] = i;
    for (int32_t i = n - 1; i > 0; --i) {
        int32_t j = (int32_t)rng_below(r, (uint64_t)i + 1);
        int32_t t = p[i]; p[i] = p[j]; p[j] = t;
    }
    return p;
}

static void relabel_keys(uint64_t* keys, int64_t nk, const int32_t* perm)
{
    for (int64_t i = 0; i < nk; ++i) {
        int32_t a = perm[keys[i] >> 32], b = perm[keys[i] & 0xFFFFFFFFu];
        keys[i] = edge_key(a, b);
    }
}

/* ------------------------------------------------------------ generators */

/* Erdos-Renyi G(n, m): exactly m distinct uniform pairs, drawn by rejection
 * of self-loops and repeats (repeats are removed and redrawn in rounds). */
kg_graph* kg_erdos_renyi(int32_t n, int64_t m, uint64_t seed)
{
    if (n < 2 || m < 0 || (double)m > (double)n * (double)(n - 1) / 2.0) return NULL;
    kg_rng r;
    rng_seed(&r, seed);
    uint64_t* keys = (uint64_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(uint64_t));
    if (!keys) return NULL;
    int64_t have = 0;
    while (have < m) {
        for (int64_t i = have; i < m; ++i) {
            int32_t a, b;
            do {
                a = (int32_t)rng_below(&r, (uint64_t)n);
                b = (int32_t)rng_below(&r, (uint64_t)n);
            } while (a == b);
            keys[i] = edge_key(a, b);
        }
        radix_sort_u64(keys, m);
        int64_t u = 0;
        for (int64_t i = 0; i < m; ++i)
            if (i == 0 || keys[i] != keys[u - 1]) keys[u++] = keys[i];
        have = u;
    }
    return graph_from_keys(n, keys, m);
}

/* Chung-Lu: weights w_i = a (i + i0)^(-1/(gamma-1)), i = 0..n-1, with a and
 * i0 chosen so that w_0 = wmax and sum(w) ~= 2m.  m edges are drawn with
 * both endpoints independent and proportional to w; self-loops and repeats
 * are dropped (so the realised edge count is a little below m); finally the
 * ids are shuffled by a seeded permutation. */
static double cl_weight_sum(int32_t n, double i0, double beta)
{
    /* exact for the first K terms, midpoint integral for the tail */
    int32_t K = n < 4096 ? n : 4096;
    double s = 0.0;
    for (int32_t i = 0; i < K; ++i) s += kg_pow(((double)i + i0) / i0, -beta);
    if (K < n) {
        double lo = (double)K - 0.5 + i0, hi = (double)n - 0.5 + i0;
        double e = 1.0 - beta;
        s += (kg_pow(hi / i0, e) - kg_pow(lo / i0, e)) * i0 / e;
    }
    return s;
}

kg_graph* kg_chung_lu(int32_t n, int64_t m, double gamma, double wmax, uint64_t seed)
{
    if (n < 2 || m < 1 || gamma <= 2.0 || wmax < 1.0) return NULL;
    double beta = 1.0 / (gamma - 1.0);
    double target = 2.0 * (double)m / wmax; /* sum of (w_i / wmax) */
    if (target >= (double)n) target = (double)n * 0.999;
    /* bisection on log i0: the normalised sum grows with i0 */
    double lo = -20.0, hi = 40.0;
    for (int it = 0; it < 100; ++it) {
        double mid = 0.5 * (lo + hi);
        if (cl_weight_sum(n, kg_exp(mid), beta) < target) lo = mid; else hi = mid;
    }
    double i0 = kg_exp(0.5 * (lo + hi));
    /* integer weights (fixed point 2^16), cumulative */
    uint64_t* cum = (uint64_t*)malloc(((size_t)n + 1) * sizeof(uint64_t));
    if (!cum) return NULL;
    cum[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        double w = wmax * kg_pow(((double)i + i0) / i0, -beta);
        uint64_t wi = (uint64_t)(w * 65536.0);
        if (wi == 0) wi = 1;
        cum[i + 1] = cum[i] + wi;
    }
    kg_rng r;
    rng_seed(&r, seed);
    uint64_t* keys = (uint64_t*)malloc((size_t)m * sizeof(uint64_t));
    if (!keys) { free(cum); return NULL; }
    int64_t nk = 0;
    for (int64_t e = 0; e < m; ++e) {
        int32_t ends[2];
        for (int s = 0; s < 2; ++s) {
            uint64_t x = rng_below(&r, cum[n]);
            /* largest i with cum[i] <= x */
            int32_t a = 0, b = n; /* cum[a] <= x < cum[b] */
            while (b - a > 1) {
                int32_t c = a + (b - a) / 2;
                if (cum[c] <= x) a = c; else b = c;
            }
            ends[s] = a;
        }
        if (ends[0] != ends[1]) keys[nk++] = edge_key(ends[0], ends[1]);
    }
    free(cum);
    int32_t* perm = random_permutation(n, &r);
    if (!perm) { free(keys); return NULL; }
    relabel_keys(keys, nk, perm);
    free(perm);
    return graph_from_keys(n, keys, nk);
}

/* Stochastic block model: n/b blocks of b contiguous ids; every intra-block
 * pair is an edge with probability p_in; then uniform distinct inter-block
 * pairs are added until the total reaches m_total; ids are shuffled last. */
kg_graph* kg_sbm(int32_t n, int32_t b, double p_in, int64_t m_total, uint64_t seed)
{
    if (n < 2 || b < 1 || n % b != 0) return NULL;
    int32_t nb = n / b;
    kg_rng r;
    rng_seed(&r, seed);
    uint64_t th = prob_to_thresh53(p_in);
    /* intra edges, counted first with a clone of the stream, then drawn */
    int64_t intra = 0;
    {
        kg_rng c = r;
        for (int32_t blk = 0; blk < nb; ++blk)
            for (int32_t i = 0; i < b; ++i)
                for (int32_t j = i + 1; j < b; ++j) intra += rng_bernoulli(&c, th);
    }
    int64_t inter = m_total > intra ? m_total - intra : 0;
    if (nb < 2) inter = 0;
    uint64_t* keys = (uint64_t*)malloc((size_t)(intra + inter > 0 ? intra + inter : 1) * sizeof(uint64_t));
    if (!keys) return NULL;
    int64_t nk = 0;
    for (int32_t blk = 0; blk < nb; ++blk) {
        int32_t base = blk * b;
        for (int32_t i = 0; i < b; ++i)
            for (int32_t j = i + 1; j < b; ++j)
                if (rng_bernoulli(&r, th)) keys[nk++] = edge_key(base + i, base + j);
    }
    /* inter edges: distinct uniform cross-block pairs, redrawn in rounds */
    int64_t have = 0;
    uint64_t* ik = keys + intra;
    while (have < inter) {
        for (int64_t i = have; i < inter; ++i) {
            int32_t a, c;
            do {
                a = (int32_t)rng_below(&r, (uint64_t)n);
                c = (int32_t)rng_below(&r, (uint64_t)n);
            } while (a / b == c / b);
            ik[i] = edge_key(a, c);
        }
        radix_sort_u64(ik, inter);
        int64_t u = 0;
        for (int64_t i = 0; i < inter; ++i)
            if (i == 0 || ik[i] != ik[u - 1]) ik[u++] = ik[i];
        have = u;
    }
    nk = intra + inter;
    int32_t* perm = random_permutation(n, &r);
    if (!perm) { free(keys); return NULL; }
    relabel_keys(keys, nk, perm);
    free(perm);
    return graph_from_keys(n, keys, nk);
}

/* R-MAT (Chakrabarti, Zhan & Faloutsos 2004): edge_factor * 2^scale edges,
 * each placed by `scale` recursive quadrant choices with probabilities
 * (a, b, c, 1-a-b-c); self-loops and repeats dropped; ids scrambled. */
kg_graph* kg_rmat(int scale, int edge_factor, double a, double b, double c, uint64_t seed)
{
    if (scale < 1 || scale > 30 || edge_factor < 1) return NULL;
    int32_t n = (int32_t)1 << scale;
    int64_t ne = (int64_t)edge_factor << scale;
    uint64_t ta = prob_to_thresh53(a), tab = prob_to_thresh53(a + b),
             tabc = prob_to_thresh53(a + b + c);
    kg_rng r;
    rng_seed(&r, seed);
    uint64_t* keys = (uint64_t*)malloc((size_t)ne * sizeof(uint64_t));
    if (!keys) return NULL;
    int64_t nk = 0;
    for (int64_t e = 0; e < ne; ++e) {
        uint32_t u = 0, v = 0;
        for (int l = 0; l < scale; ++l) {
            uint64_t x = rng_next(&r) >> 11;
            uint32_t bu = 0, bv = 0;
            if (x < ta) { }
            else if (x < tab) { bv = 1; }
            else if (x < tabc) { bu = 1; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        if (u != v) keys[nk++] = edge_key((int32_t)u, (int32_t)v);
    }
    int32_t* perm = random_permutation(n, &r);
    if (!perm) { free(keys); return NULL; }
    relabel_keys(keys, nk, perm);
    free(perm);
    return graph_from_keys(n, keys, nk);
}

/* Accessors for the Python wrapper. */
int32_t kg_n(const kg_graph* g) { return g->n; }
int64_t kg_m(const kg_graph* g) { return g->m; }
const int64_t* kg_off(const kg_graph* g) { return g->off; }
const int32_t* kg_adj(const kg_graph* g) { return g->adj; }

/* xoshiro256** from an explicit state, for pinning against published outputs. */
void kg_xoshiro_from_state(uint64_t s0, uint64_t s1, uint64_t s2, uint64_t s3,
                           int32_t nout, uint64_t* out)
{
    kg_rng r = { { s0, s1, s2, s3 } };
    for (int32_t i = 0; i < nout; ++i) out[i] = rng_next(&r);
}
