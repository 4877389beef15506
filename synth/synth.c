/*
 * synth.c -- seeded synthetic workloads for regular-expression matching.
 *
 * This module only PRODUCES inputs: random expression trees in the node-array
 * format below, strings drawn from an expression's language by a random walk
 * over its syntax tree, uniformly random strings and small random edits.  It
 * contains no matching arithmetic (no closures, no continuation wiring, no
 * membership decision); both the CPU oracle and the GPU library consume what
 * it writes.
 *
 * Randomness: splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014).  Item i of a stream with base seed s gets
 * its own generator seeded with the i-th splitmix64 output of s, so every item
 * is reproducible independently of threading.
 *
 * Node array format (shared input interface, 12 bytes per node):
 *   kind u8 (0 CHAR, 1 EPS, 2 STAR, 3 CAT, 4 ALT), byte u8, pad u16,
 *   l i32, r i32 (-1 when absent).  Nodes are emitted in preorder; the root
 *   is node 0.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define K_CHAR 0
#define K_EPS 1
#define K_STAR 2
#define K_CAT 3
#define K_ALT 4

typedef struct {
    uint8_t kind, byte;
    uint16_t pad;
    int32_t l, r;
} sy_node;

/* ---------------------------------------------------------------- rng */
#define GOLDEN 0x9e3779b97f4a7c15ULL
static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
typedef struct { uint64_t s; } rng_t;
static inline uint64_t rnext(rng_t* g) { g->s += GOLDEN; return mix64(g->s); }
static inline double runif(rng_t* g) { return (double)(rnext(g) >> 11) * (1.0 / 9007199254740992.0); }
/* uniform integer in [lo, hi] */
static inline int64_t rint_in(rng_t* g, int64_t lo, int64_t hi) {
    if (hi <= lo) return lo;
    uint64_t span = (uint64_t)(hi - lo) + 1;
    return lo + (int64_t)(rnext(g) % span);
}
/* the seed of item i in the stream with base seed s */
uint64_t sy_item_seed(uint64_t s, uint64_t i) { return mix64(s + GOLDEN * (i + 1)); }

/* ------------------------------------------------------ expression trees */
typedef struct {
    rng_t g;
    sy_node* out;
    int n, cap;
    int max_depth;
    double w[5]; /* weights: char, eps, cat, alt, star */
    const uint8_t* alpha;
    int alpha_n;
    double eps_loop_p;
} gen_t;

/* most nodes a subtree of height <= h can hold (binary nodes) */
static int64_t max_nodes(int h) {
    if (h < 0) return 0;
    if (h >= 40) return (int64_t)1 << 40;
    return ((int64_t)1 << (h + 1)) - 1;
}

static int new_node(gen_t* G, int kind) {
    if (G->n >= G->cap) return -1;
    int id = G->n++;
    G->out[id].kind = (uint8_t)kind;
    G->out[id].byte = 0;
    G->out[id].pad = 0;
    G->out[id].l = -1;
    G->out[id].r = -1;
    return id;
}

static int gen_rec(gen_t* G, int64_t b, int depth);

static int gen_leaf(gen_t* G) {
    double wc = G->w[0], we = G->w[1];
    int is_char = (wc + we <= 0.0) ? 1 : (runif(&G->g) * (wc + we) < wc);
    int id = new_node(G, is_char ? K_CHAR : K_EPS);
    if (id >= 0 && is_char) G->out[id].byte = G->alpha[rint_in(&G->g, 0, G->alpha_n - 1)];
    return id;
}

static int gen_rec(gen_t* G, int64_t b, int depth) {
    int h = G->max_depth - depth; /* remaining height */
    if (b <= 1 || h <= 0) return gen_leaf(G);
    int64_t child_cap = max_nodes(h - 1);
    /* deliberate epsilon loop (eps* | e)*: four wrapper nodes, e two levels down */
    if (G->eps_loop_p > 0.0 && b >= 5 && h >= 3 && b - 4 <= max_nodes(h - 2) &&
        runif(&G->g) < G->eps_loop_p) {
        int s1 = new_node(G, K_STAR);
        int a = new_node(G, K_ALT);
        int s2 = new_node(G, K_STAR);
        int e = new_node(G, K_EPS);
        if (s1 < 0 || a < 0 || s2 < 0 || e < 0) return -1;
        G->out[s1].l = a;
        G->out[a].l = s2;
        G->out[s2].l = e;
        int c = gen_rec(G, b - 4, depth + 2);
        if (c < 0) return -1;
        G->out[a].r = c;
        return s1;
    }
    double ws = (b - 1 <= child_cap) ? G->w[4] : 0.0;
    int bin_ok = (b >= 3) && (b - 1 <= 2 * child_cap);
    double wcat = bin_ok ? G->w[2] : 0.0, walt = bin_ok ? G->w[3] : 0.0;
    double tot = ws + wcat + walt;
    int kind;
    if (tot <= 0.0) {
        kind = (b - 1 <= child_cap) ? K_STAR : K_CAT;
    } else {
        double u = runif(&G->g) * tot;
        kind = (u < ws) ? K_STAR : (u < ws + wcat ? K_CAT : K_ALT);
    }
    int id = new_node(G, kind);
    if (id < 0) return -1;
    if (kind == K_STAR) {
        int c = gen_rec(G, b - 1, depth + 1);
        if (c < 0) return -1;
        G->out[id].l = c;
    } else {
        int64_t lo = b - 1 - child_cap;
        if (lo < 1) lo = 1;
        int64_t hi = b - 2;
        if (hi > child_cap) hi = child_cap;
        int64_t bl = rint_in(&G->g, lo, hi);
        int l = gen_rec(G, bl, depth + 1);
        if (l < 0) return -1;
        int r = gen_rec(G, b - 1 - bl, depth + 1);
        if (r < 0) return -1;
        G->out[id].l = l;
        G->out[id].r = r;
    }
    return id;
}

/*
 * Random expression tree with `nodes` nodes (when the depth bound allows it),
 * kinds drawn from mix = {char, eps, cat, alt, star} restricted to the kinds
 * that fit the remaining budget and height, split budgets uniform.  Returns the
 * node count written (root = node 0) or -1 when `cap` is too small.
 */
int sy_gen_regex(int nodes, int max_depth, const double* mix, const uint8_t* alpha, int alpha_n,
                 double eps_loop_p, uint64_t seed, sy_node* out, int cap) {
    gen_t G;
    G.g.s = seed;
    G.out = out;
    G.n = 0;
    G.cap = cap;
    G.max_depth = max_depth;
    for (int i = 0; i < 5; i++) G.w[i] = mix[i];
    G.alpha = alpha;
    G.alpha_n = alpha_n;
    G.eps_loop_p = eps_loop_p;
    int64_t b = nodes;
    if (b > max_nodes(max_depth)) b = max_nodes(max_depth);
    if (b < 1) b = 1;
    int root = gen_rec(&G, b, 0);
    if (root != 0) return -1;
    return G.n;
}

/* ------------------------------------------------ language sampling walk */
typedef struct {
    const sy_node* nd;
    rng_t g;
    uint8_t* buf;
    int64_t len, cap, target;
    double pc; /* probability that a star takes another iteration below target */
    int overflow;
} walk_t;

static void walk(walk_t* W, int p) {
    if (W->overflow) return;
    const sy_node* x = &W->nd[p];
    switch (x->kind) {
    case K_CHAR:
        if (W->len >= W->cap) { W->overflow = 1; return; }
        W->buf[W->len++] = x->byte;
        return;
    case K_EPS:
        return;
    case K_CAT:
        walk(W, x->l);
        walk(W, x->r);
        return;
    case K_ALT:
        walk(W, (rnext(&W->g) & 1) ? x->r : x->l);
        return;
    case K_STAR:
        for (;;) {
            if (W->len >= W->target) return;
            if (runif(&W->g) >= W->pc) return;
            int64_t before = W->len;
            walk(W, x->l);
            if (W->overflow || W->len == before) return;
        }
    }
}

/* one language sample aimed at `target` bytes: best of a few walks */
static int64_t sample_one(const sy_node* nd, int nnodes, int64_t target, int64_t minlen, int64_t maxlen,
                          rng_t* g, uint8_t* buf, uint8_t* tmp, int64_t cap) {
    static const double pcs[6] = {0.7, 0.9, 0.97, 0.995, 0.9995, 1.0};
    int64_t best = -1, bestd = INT64_MAX;
    (void)nnodes;
    for (int a = 0; a < 6; a++) {
        walk_t W;
        W.nd = nd;
        W.g.s = rnext(g);
        W.buf = tmp;
        W.len = 0;
        W.cap = cap;
        W.target = target;
        W.pc = pcs[a];
        W.overflow = 0;
        walk(&W, 0);
        if (W.overflow || W.len < minlen || W.len > maxlen) continue;
        int64_t d = W.len > target ? W.len - target : target - W.len;
        if (d < bestd) {
            bestd = d;
            best = W.len;
            memcpy(buf, tmp, (size_t)W.len);
        }
        if (d <= target / 16) break;
    }
    return best;
}

/* ---------------------------------------------------------- string sets */
/*
 * Strings for one expression.  Item i: target length uniform in [lmin, lmax]
 * (log-uniform when log_len != 0); with probability p_lang a language sample,
 * otherwise (mode 0) uniform random over the alphabet or (mode 1) a language
 * sample with 1-3 random edits.  Language samples that cannot reach the
 * length range fall back to a uniform string (counted in *n_fallback).
 * Output: malloc'd bytes and offsets (n+1) -- free with sy_free.
 */
typedef struct {
    uint8_t* bytes;
    int64_t* offsets;
    int64_t total;
    int64_t n_fallback;
    uint8_t* kind; /* per item: 0 uniform, 1 language, 2 edited language, 3 fallback */
} sy_strings;

static void uniform_fill(rng_t* g, uint8_t* dst, int64_t len, const uint8_t* alpha, int alpha_n) {
    for (int64_t i = 0; i < len; i++) dst[i] = alpha[rnext(g) % (uint64_t)alpha_n];
}

static int64_t draw_len(rng_t* g, int64_t lmin, int64_t lmax, int log_len) {
    if (!log_len) return rint_in(g, lmin, lmax);
    if (lmin < 1) {
        /* log-uniform on [1, lmax + 1], shifted down by one: [0, lmax] */
        const double b = log((double)lmax + 2.0);
        int64_t L = (int64_t)floor(exp(b * runif(g))) - 1;
        if (L < 0) L = 0;
        if (L > lmax) L = lmax;
        return L;
    }
    double a = log((double)lmin), b = log((double)lmax + 1.0);
    int64_t L = (int64_t)floor(exp(a + (b - a) * runif(g)));
    if (L < lmin) L = lmin;
    if (L > lmax) L = lmax;
    return L;
}

/* 1-3 edits (substitute / insert / delete) with lengths kept in [lmin, lmax] */
static int64_t edit_string(rng_t* g, uint8_t* s, int64_t len, int64_t lmin, int64_t lmax, const uint8_t* alpha,
                           int alpha_n) {
    int k = (int)rint_in(g, 1, 3);
    for (int e = 0; e < k; e++) {
        int op = (int)rint_in(g, 0, 2);
        if (op == 1 && len + 1 > lmax) op = 0;
        if (op == 2 && len - 1 < lmin) op = 0;
        if (op == 0 && len == 0) op = 1;
        if (op == 0) {
            int64_t p = rint_in(g, 0, len - 1);
            uint8_t c = alpha[rnext(g) % (uint64_t)alpha_n];
            if (alpha_n > 1)
                while (c == s[p]) c = alpha[rnext(g) % (uint64_t)alpha_n];
            s[p] = c;
        } else if (op == 1) {
            int64_t p = rint_in(g, 0, len);
            memmove(s + p + 1, s + p, (size_t)(len - p));
            s[p] = alpha[rnext(g) % (uint64_t)alpha_n];
            len++;
        } else {
            int64_t p = rint_in(g, 0, len - 1);
            memmove(s + p, s + p + 1, (size_t)(len - p - 1));
            len--;
        }
    }
    return len;
}

int sy_gen_strings(const sy_node* nd, int nnodes, int64_t n, int64_t lmin, int64_t lmax, int log_len, double p_lang,
                   int mode, const uint8_t* alpha, int alpha_n, uint64_t seed, sy_strings* res) {
    memset(res, 0, sizeof(*res));
    int64_t* lens = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    uint8_t** parts = (uint8_t**)calloc((size_t)(n > 0 ? n : 1), sizeof(uint8_t*));
    uint8_t* kinds = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
    if (!lens || !parts || !kinds) return -1;
    int64_t nfb = 0;
    int failed = 0;
#pragma omp parallel reduction(+ : nfb)
    {
        int64_t tcap = 0;
        uint8_t* tmp = NULL;
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; i++) {
            rng_t g;
            g.s = sy_item_seed(seed, (uint64_t)i);
            int64_t target = draw_len(&g, lmin, lmax, log_len);
            int lang = runif(&g) < p_lang;
            int64_t cap = lmax + 4 * (int64_t)nnodes + 64;
            if (cap > tcap) {
                free(tmp);
                tmp = (uint8_t*)malloc((size_t)cap);
                tcap = cap;
            }
            uint8_t* s = (uint8_t*)malloc((size_t)cap + 4);
            if (!s || !tmp) { failed = 1; continue; }
            int64_t len;
            uint8_t kind = 0;
            if (lang || mode == 1) {
                len = sample_one(nd, nnodes, target, lmin, lmax, &g, s, tmp, cap);
                kind = 1;
                if (len < 0) {
                    len = target;
                    uniform_fill(&g, s, len, alpha, alpha_n);
                    kind = 3;
                    nfb++;
                } else if (!lang) {
                    len = edit_string(&g, s, len, lmin, lmax, alpha, alpha_n);
                    kind = 2;
                }
            } else {
                len = target;
                uniform_fill(&g, s, len, alpha, alpha_n);
            }
            lens[i] = len;
            parts[i] = s;
            kinds[i] = kind;
        }
        free(tmp);
    }
    if (failed) return -1;
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!off) return -1;
    off[0] = 0;
    for (int64_t i = 0; i < n; i++) off[i + 1] = off[i] + lens[i];
    uint8_t* bytes = (uint8_t*)malloc((size_t)(off[n] > 0 ? off[n] : 1));
    if (!bytes) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        memcpy(bytes + off[i], parts[i], (size_t)lens[i]);
        free(parts[i]);
    }
    free(parts);
    free(lens);
    res->bytes = bytes;
    res->offsets = off;
    res->total = off[n];
    res->n_fallback = nfb;
    res->kind = kinds;
    return 0;
}

/*
 * One long text in the language of e* (e = the given tree), cut to `total`
 * bytes: independent segments of about 1 MiB, each a concatenation of WHOLE
 * language samples of e (target lengths uniform in [1, piece]), joined end
 * to end, so every prefix of the text is a prefix of a member of e*.  Only
 * the last sample may be cut.  Segment k uses item seed k, so the text is
 * reproducible whatever the thread count.  *last_end (optional) receives the
 * end offset of the last whole segment (a member of e* ends there).
 */
int sy_gen_star_text(const sy_node* nd, int nnodes, int64_t total, int64_t piece, uint64_t seed, uint8_t* out,
                     int64_t* last_end) {
    const int64_t SEG = 1 << 20;
    int64_t nseg = (total + SEG - 1) / SEG;
    if (nseg < 1) nseg = 1;
    uint8_t** bufs = (uint8_t**)calloc((size_t)nseg, sizeof(uint8_t*));
    int64_t* lens = (int64_t*)calloc((size_t)nseg, sizeof(int64_t));
    if (!bufs || !lens) return -1;
    int failed = 0;
#pragma omp parallel
    {
        int64_t cap = piece + 4 * (int64_t)nnodes + 64;
        uint8_t* tmp = (uint8_t*)malloc((size_t)cap);
        uint8_t* one = (uint8_t*)malloc((size_t)cap);
#pragma omp for schedule(dynamic, 1)
        for (int64_t k = 0; k < nseg; k++) {
            if (!tmp || !one) { failed = 1; continue; }
            rng_t g;
            g.s = sy_item_seed(seed, (uint64_t)k);
            uint8_t* buf = (uint8_t*)malloc((size_t)(SEG + cap));
            if (!buf) { failed = 1; continue; }
            int64_t pos = 0;
            int stuck = 0;
            while (pos < SEG) {
                int64_t target = rint_in(&g, 1, piece);
                int64_t len = sample_one(nd, nnodes, target, 1, cap, &g, one, tmp, cap);
                if (len <= 0) {
                    if (++stuck > 64) { failed = 2; break; }
                    continue;
                }
                memcpy(buf + pos, one, (size_t)len);
                pos += len;
            }
            bufs[k] = buf;
            lens[k] = pos;
        }
        free(tmp);
        free(one);
    }
    int64_t pos = 0, lastb = 0;
    for (int64_t k = 0; k < nseg && !failed; k++) {
        int64_t take = lens[k] < total - pos ? lens[k] : total - pos;
        if (take > 0) memcpy(out + pos, bufs[k], (size_t)take);
        if (take == lens[k]) lastb = pos + take;
        pos += take;
    }
    /* more segments than needed never happens (each holds >= 1 MiB); if the
       segments fall short, repeat them (still whole samples) */
    while (!failed && pos < total) {
        for (int64_t k = 0; k < nseg && pos < total; k++) {
            int64_t take = lens[k] < total - pos ? lens[k] : total - pos;
            memcpy(out + pos, bufs[k], (size_t)take);
            if (take == lens[k]) lastb = pos + take;
            pos += take;
        }
    }
    for (int64_t k = 0; k < nseg; k++) free(bufs[k]);
    free(bufs);
    free(lens);
    if (last_end) *last_end = lastb;
    return failed ? -1 : 0;
}

/* uniform random bytes from the alphabet */
void sy_uniform(uint8_t* out, int64_t len, const uint8_t* alpha, int alpha_n, uint64_t seed) {
    int64_t nseg = (len + (1 << 20) - 1) >> 20;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nseg; k++) {
        rng_t g;
        g.s = sy_item_seed(seed, (uint64_t)k);
        int64_t pos = k << 20, end = pos + (1 << 20);
        if (end > len) end = len;
        uniform_fill(&g, out + pos, end - pos, alpha, alpha_n);
    }
}

/* a batch of uniform doubles / integers from an item stream (for Python drivers) */
void sy_uniform_f64(double* out, int64_t n, uint64_t seed) {
    for (int64_t i = 0; i < n; i++) {
        rng_t g;
        g.s = sy_item_seed(seed, (uint64_t)i);
        out[i] = runif(&g);
    }
}

void sy_free(sy_strings* r) {
    free(r->bytes);
    free(r->offsets);
    free(r->kind);
    memset(r, 0, sizeof(*r));
}
