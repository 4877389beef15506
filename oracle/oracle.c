/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.  A plain, slow CPU statement of what
 * the matcher computes, used to check the GPU library.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load this code; the
 * library itself never does.  It shares no code, header or table with the GPU
 * path: it reads the same node-array input format and nothing else.
 *
 * Rathnayake & Thielecke, "Regular Expression Matching and Operational
 * Semantics" (SOS 2011):
 *
 *   O1  -- the big-step matching relation e |v w of Fig 2.1 (rules Seq, Match,
 *          Epsilon, Kleene1, Kleene2, Alt1, Alt2), read as the least relation
 *          closed under the rules, memoised over (node, start index).
 *   O1 search -- unanchored search from the same tables: the earliest end j
 *          of a substring w[i..j) with e |v w[i..j) (not in the paper).
 *   O2 search -- the same answer from the machine of Fig 6.1 with the root
 *          pushed back at every macro step (streaming; long texts).
 *   O2  -- the sequential lockstep machine <c; t; n; w> of Def 6.2 / Fig 6.1
 *          with the add-unique function psi of Def 6.1, over the pointer tree
 *          of Section 4 with the cont function of Def 4.4.
 *   cont -- Def 4.4, computed by a walk from the root.
 *
 * Node array format (input interface, 12 bytes per node): kind u8 (0 CHAR,
 * 1 EPS, 2 STAR, 3 CAT, 4 ALT), byte u8, pad u16, l i32, r i32.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

enum { CHAR = 0, EPS = 1, STAR = 2, CAT = 3, ALT = 4 };

typedef struct {
    uint8_t kind, byte;
    uint16_t pad;
    int32_t l, r;
} or_node;

#define NUL (-1) /* the distinguished address null */

/* ------------------------------------------------------------- cont (Def 4.4)
 * cont(root) = null; for p1|p2 both children inherit cont(p); for p1.p2,
 * cont(p1) = p2 and cont(p2) = cont(p); for p1*, cont(p1) = p.
 * Returns 0, or -1 if a child index is out of range. */
int or_cont(const or_node* nd, int nn, int root, int32_t* cont) {
    int32_t* stack = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nn + 1));
    if (!stack) return -1;
    for (int i = 0; i < nn; i++) cont[i] = NUL;
    int sp = 0;
    stack[sp++] = root;
    cont[root] = NUL;
    int rc = 0, visits = 0;
    while (sp > 0) {
        int p = stack[--sp];
        if (++visits > nn) { rc = -1; break; }
        const or_node* x = &nd[p];
        if (x->kind == ALT) {
            if (x->l < 0 || x->l >= nn || x->r < 0 || x->r >= nn) { rc = -1; break; }
            cont[x->l] = cont[p];
            cont[x->r] = cont[p];
            stack[sp++] = x->l;
            stack[sp++] = x->r;
        } else if (x->kind == CAT) {
            if (x->l < 0 || x->l >= nn || x->r < 0 || x->r >= nn) { rc = -1; break; }
            cont[x->l] = x->r;
            cont[x->r] = cont[p];
            stack[sp++] = x->l;
            stack[sp++] = x->r;
        } else if (x->kind == STAR) {
            if (x->l < 0 || x->l >= nn) { rc = -1; break; }
            cont[x->l] = p;
            stack[sp++] = x->l;
        }
    }
    free(stack);
    return rc;
}

/* ------------------------------------------------------------------ O1
 * ends(e, i) = { j : e |v w[i..j) } as an (L+1)-bit set, for every node e and
 * every start i, computed for i = L down to 0 with children before parents:
 *   Match   a      : { i+1 } if i < L and w[i] = a, else {}
 *   Epsilon        : { i }
 *   Alt1/2  e1|e2  : ends(e1,i) U ends(e2,i)
 *   Seq     e1 e2  : U_{k in ends(e1,i)} ends(e2,k)          (k >= i)
 *   Kleene2 e*     : { i }
 *   Kleene1 e*     : U_{k in ends(e,i)} ends(e*,k)
 * In Kleene1 the term k = i is ends(e*,i) itself; under the least-relation
 * reading it adds nothing, so only k > i (already computed) contributes.
 * e |v w  iff  L in ends(root, 0).
 * Returns 1 / 0, or -1 when the tables would exceed max_bytes. */
static int postorder(const or_node* nd, int nn, int root, int32_t* order) {
    int32_t* stack = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * nn + 2));
    if (!stack) return -1;
    int sp = 0, k = 0;
    stack[sp++] = root;
    /* reverse of a (node, right, left) preorder is a valid children-first order */
    while (sp > 0) {
        int p = stack[--sp];
        if (k >= nn) { free(stack); return -1; }
        order[k++] = p;
        const or_node* x = &nd[p];
        if (x->kind == CAT || x->kind == ALT) {
            stack[sp++] = x->l;
            stack[sp++] = x->r;
        } else if (x->kind == STAR) {
            stack[sp++] = x->l;
        }
    }
    free(stack);
    for (int a = 0, b = k - 1; a < b; a++, b--) {
        int32_t t = order[a];
        order[a] = order[b];
        order[b] = t;
    }
    return k;
}

/* The ends tables for every node and start: nn * (L+1) sets of *words
 * 64-bit words; NULL when they would exceed max_bytes (or on a malformed
 * tree).  The caller frees. */
static uint64_t* o1_tables(const or_node* nd, int nn, int root, const uint8_t* w, int64_t L, int64_t max_bytes,
                           int64_t* words_out) {
    int64_t words = (L + 1 + 63) / 64;
    int64_t need = (int64_t)nn * (L + 1) * words * 8;
    if (need > max_bytes) return NULL;
    uint64_t* E = (uint64_t*)calloc((size_t)need / 8, 8);
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)nn);
    if (!E || !order) { free(E); free(order); return NULL; }
    int k = postorder(nd, nn, root, order);
    if (k < 0) { free(E); free(order); return NULL; }
#define ENDS(e, i) (E + (((int64_t)(e) * (L + 1) + (i)) * words))
#define SETB(s, j) ((s)[(j) >> 6] |= 1ULL << ((j) & 63))
#define GETB(s, j) (((s)[(j) >> 6] >> ((j) & 63)) & 1ULL)
    for (int64_t i = L; i >= 0; i--) {
        for (int q = 0; q < k; q++) {
            int e = order[q];
            const or_node* x = &nd[e];
            uint64_t* dst = ENDS(e, i);
            switch (x->kind) {
            case CHAR:
                if (i < L && w[i] == x->byte) SETB(dst, i + 1);
                break;
            case EPS:
                SETB(dst, i);
                break;
            case ALT: {
                uint64_t *a = ENDS(x->l, i), *b = ENDS(x->r, i);
                for (int64_t z = 0; z < words; z++) dst[z] = a[z] | b[z];
                break;
            }
            case CAT: {
                uint64_t* a = ENDS(x->l, i);
                for (int64_t kk = i; kk <= L; kk++)
                    if (GETB(a, kk)) {
                        uint64_t* b = ENDS(x->r, kk);
                        for (int64_t z = 0; z < words; z++) dst[z] |= b[z];
                    }
                break;
            }
            case STAR: {
                SETB(dst, i);
                uint64_t* a = ENDS(x->l, i);
                for (int64_t kk = i + 1; kk <= L; kk++)
                    if (GETB(a, kk)) {
                        uint64_t* b = ENDS(e, kk);
                        for (int64_t z = 0; z < words; z++) dst[z] |= b[z];
                    }
                break;
            }
            }
        }
    }
    free(order);
    *words_out = words;
    return E;
}

int or_o1(const or_node* nd, int nn, int root, const uint8_t* w, int64_t L, int64_t max_bytes) {
    int64_t words = 0;
    uint64_t* E = o1_tables(nd, nn, root, w, L, max_bytes, &words);
    if (!E) return -1;
    int res = (int)GETB(ENDS(root, 0), L);
    free(E);
    return res;
}

/* ------------------------------------------------------------ O1 search
 * Unanchored search (not in the paper; the hot path's search mode): the
 * smallest j such that e |v w[i..j) for some i <= j, from the same ends
 * tables -- min over i of the lowest j in ends(root, i).  -1 if there is no
 * such j; -2 when the tables would exceed max_bytes. */
int64_t or_o1_search(const or_node* nd, int nn, int root, const uint8_t* w, int64_t L, int64_t max_bytes) {
    int64_t words = 0;
    uint64_t* E = o1_tables(nd, nn, root, w, L, max_bytes, &words);
    if (!E) return -2;
    int64_t best = -1;
    for (int64_t i = 0; i <= L; i++) {
        const uint64_t* s = ENDS(root, i);
        for (int64_t j = i; j <= L && (best < 0 || j < best); j++)
            if (GETB(s, j)) {
                best = j;
                break;
            }
    }
#undef ENDS
#undef SETB
#undef GETB
    free(E);
    return best;
}

/* ------------------------------------------------------------------ O2
 * Lists are stacks whose head is the last array element.  NUL is stored as
 * the id nn.  psi(p, l1, l2) = p::l1 if p not in l1@l2, else l1 (Def 6.1).
 * The membership test "p in c@t" is kept as a mark per id: within one macro
 * step an id only moves from c to t, so it stays in c@t once pushed; the one
 * exception is null, which the rules drop from c without pushing it to t,
 * so its mark is cleared when it is popped.  "p in n" is a second mark.
 * Marks carry the macro-step number, so starting a step invalidates them.
 * (The lists, their order and every rule are as in the figure; only the
 * test of Def 6.1 is answered from the marks instead of a scan.)
 *
 * Fig 6.1, rule by rule (c = p::c'):
 *   p = p1|p2 : c := psi(p2, psi(p1, c', t), t);          t := p::t
 *   p = p1.p2 : c := psi(p1, c', t);                      t := p::t
 *   p = p1*   : c := psi(cont p, psi(p1, c', t), t);      t := p::t
 *               (the figure prints psi(p, ...) in the inner call; the child
 *                p1 is meant -- Fig 4.2 moves a star to its child and to its
 *                continuation, and the process translation of Section 7 sends
 *                to both -- with p itself the star would never reach p1)
 *   p = eps   : c := psi(cont p, c', t);                  t := p::t
 *   p = null, input a w        : c := c'                 (dropped)
 *   p = a,    input a w        : n := psi(cont p, n, []); t := p::t
 *   p = b,    input a w, b!=a  : t := p::t                (dropped)
 *   p = a,    input empty      : t := p::t                (dropped)
 *   c = [], input a w, n != [] : c := n; t := []; n := []; input := w
 * Accepting: null at the head of c with the input empty.  Anything else
 * with no applicable rule is stuck, i.e. rejects.
 *
 * trace (optional, L+1 rows of nn+1 bytes each): row k marks the CHAR
 * nodes popped during macro step k (the evolved set of Def 5.1) and, in
 * column nn, whether null was popped.  In trace mode the last macro step
 * keeps evolving after null is found, so its row is complete.
 * ntrace (optional, L rows of nn+1 bytes): the list n handed to macro step
 * k+1, i.e. the set S' of Def 5.2 after reading w[k]. */
typedef struct {
    int32_t* a;
    int len;
} olist;

/* the lists of the machine and the membership marks of Def 6.1's test */
typedef struct {
    olist c, t, n;
    int64_t* in_ct; /* in_ct[p] == step  iff  p in c@t */
    int64_t* in_n;  /* in_n[p] == step   iff  p in n   */
    int64_t step;
} o2m;

/* c := psi(p, c, t) */
static void psi_ct(o2m* m, int32_t p) {
    if (m->in_ct[p] == m->step) return;
    m->in_ct[p] = m->step;
    m->c.a[m->c.len++] = p;
}
/* n := psi(p, n, []) */
static void psi_n(o2m* m, int32_t p) {
    if (m->in_n[p] == m->step) return;
    m->in_n[p] = m->step;
    m->n.a[m->n.len++] = p;
}
/* c = [], input a w: c := n; t := []; n := [] (the next macro step) */
static void next_step(o2m* m) {
    m->step++;
    memcpy(m->c.a, m->n.a, sizeof(int32_t) * (size_t)m->n.len);
    m->c.len = m->n.len;
    for (int i = 0; i < m->c.len; i++) m->in_ct[m->c.a[i]] = m->step;
    m->t.len = 0;
    m->n.len = 0;
}
/* machine over buf: 6 (nn+1) int32 for the lists, then 2 (nn+1) int64 marks */
static void o2m_init(o2m* m, int nn, int32_t* buf) {
    int cap = 2 * (nn + 1);
    m->c = (olist){buf, 0};
    m->t = (olist){buf + cap, 0};
    m->n = (olist){buf + 2 * cap, 0};
    m->in_ct = (int64_t*)(buf + 3 * cap);
    m->in_n = m->in_ct + (nn + 1);
    for (int i = 0; i <= nn; i++) m->in_ct[i] = m->in_n[i] = -1;
    m->step = 0;
}
#define O2_BUF_BYTES(nn) (sizeof(int32_t) * (size_t)(6 * ((nn) + 1)) + sizeof(int64_t) * (size_t)(2 * ((nn) + 1)))

static int o2_run(const or_node* nd, int nn, int root, const int32_t* cont, const uint8_t* w, int64_t L,
                  uint8_t* trace, uint8_t* ntrace, int32_t* buf) {
    /* every list holds distinct ids from [0, nn]; give each nn+1 slots (plus
     * slack for null, which can be re-pushed after being dropped) */
    o2m m;
    o2m_init(&m, nn, buf);
    int32_t nul = nn;
    int accept = 0;
    int64_t pos = 0;
    psi_ct(&m, root);
    for (;;) {
        if (m.c.len > 0) {
            int32_t p = m.c.a[--m.c.len];
            if (p == nul) {
                m.in_ct[nul] = -1; /* dropped: no longer in c@t */
                if (trace) trace[pos * (nn + 1) + nn] = 1;
                if (pos == L) {
                    accept = 1;
                    if (!trace) return 1;
                }
                continue;
            }
            const or_node* x = &nd[p];
            int32_t k = cont[p] < 0 ? nul : cont[p];
            switch (x->kind) {
            case ALT:
                psi_ct(&m, x->l);
                psi_ct(&m, x->r);
                break;
            case CAT:
                psi_ct(&m, x->l);
                break;
            case STAR:
                psi_ct(&m, x->l);
                psi_ct(&m, k);
                break;
            case EPS:
                psi_ct(&m, k);
                break;
            case CHAR:
                if (trace) trace[pos * (nn + 1) + p] = 1;
                if (pos < L && w[pos] == x->byte) psi_n(&m, k);
                break;
            }
            m.t.a[m.t.len++] = p;
            continue;
        }
        /* c = [] */
        if (pos < L && m.n.len > 0) {
            if (ntrace)
                for (int i = 0; i < m.n.len; i++) ntrace[pos * (nn + 1) + m.n.a[i]] = 1;
            next_step(&m);
            pos++;
            continue;
        }
        return accept; /* stuck */
    }
}

int or_o2(const or_node* nd, int nn, int root, const uint8_t* w, int64_t L, uint8_t* trace, uint8_t* ntrace) {
    int32_t* cont = (int32_t*)malloc(sizeof(int32_t) * (size_t)nn);
    int32_t* buf = (int32_t*)malloc(O2_BUF_BYTES(nn));
    if (!cont || !buf || or_cont(nd, nn, root, cont) != 0) { free(cont); free(buf); return -1; }
    int r = o2_run(nd, nn, root, cont, w, L, trace, ntrace, buf);
    free(cont);
    free(buf);
    return r;
}

/* ------------------------------------------------------------ O2 search
 * Unanchored search with the machine of Fig 6.1 (not in the paper): the
 * root is pushed into c at the start of every macro step, so a match may
 * begin at any position; the first time null is popped, at input position
 * pos, pos is the earliest end of a matching substring.  -1 when the input
 * is exhausted without null. */
int64_t or_o2_search(const or_node* nd, int nn, int root, const uint8_t* w, int64_t L) {
    int32_t* cont = (int32_t*)malloc(sizeof(int32_t) * (size_t)nn);
    int32_t* buf = (int32_t*)malloc(O2_BUF_BYTES(nn));
    if (!cont || !buf || or_cont(nd, nn, root, cont) != 0) { free(cont); free(buf); return -2; }
    o2m m;
    o2m_init(&m, nn, buf);
    int32_t nul = nn;
    int64_t pos = 0, res = -1;
    psi_ct(&m, root);
    for (;;) {
        if (m.c.len > 0) {
            int32_t p = m.c.a[--m.c.len];
            if (p == nul) {
                res = pos;
                break;
            }
            const or_node* x = &nd[p];
            int32_t k = cont[p] < 0 ? nul : cont[p];
            switch (x->kind) {
            case ALT:
                psi_ct(&m, x->l);
                psi_ct(&m, x->r);
                break;
            case CAT:
                psi_ct(&m, x->l);
                break;
            case STAR:
                psi_ct(&m, x->l);
                psi_ct(&m, k);
                break;
            case EPS:
                psi_ct(&m, k);
                break;
            case CHAR:
                if (pos < L && w[pos] == x->byte) psi_n(&m, k);
                break;
            }
            m.t.a[m.t.len++] = p;
            continue;
        }
        /* c = []: the next macro step, with the root added back */
        if (pos >= L) break;
        next_step(&m);
        pos++;
        psi_ct(&m, root);
    }
    free(cont);
    free(buf);
    return res;
}

int or_o2_search_batch(const or_node* nd, int nn, int root, const uint8_t* bytes, const int64_t* off, int64_t n,
                       int64_t* out, int nthreads) {
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
    for (int64_t i = 0; i < n; i++) out[i] = or_o2_search(nd, nn, root, bytes + off[i], off[i + 1] - off[i]);
    return 0;
}

/* ------------------------------------------------------------ batches
 * One expression against n strings (bytes + offsets[n+1]); out[i] = 0/1, or
 * 255 when O1 declined (tables too large).  Plain loop over strings, spread
 * over nthreads OpenMP threads (0 = runtime default). */
int or_o2_batch(const or_node* nd, int nn, int root, const uint8_t* bytes, const int64_t* off, int64_t n,
                uint8_t* out, int nthreads) {
    int32_t* cont = (int32_t*)malloc(sizeof(int32_t) * (size_t)nn);
    if (!cont || or_cont(nd, nn, root, cont) != 0) { free(cont); return -1; }
    int failed = 0;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
    {
        int32_t* buf = (int32_t*)malloc(O2_BUF_BYTES(nn));
        if (!buf) failed = 1;
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < n; i++) {
            if (!buf) continue;
            out[i] = (uint8_t)o2_run(nd, nn, root, cont, bytes + off[i], off[i + 1] - off[i], NULL, NULL, buf);
        }
        free(buf);
    }
    free(cont);
    return failed ? -1 : 0;
}

int or_o1_search_batch(const or_node* nd, int nn, int root, const uint8_t* bytes, const int64_t* off, int64_t n,
                       int64_t* out, int64_t max_bytes, int nthreads) {
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
    for (int64_t i = 0; i < n; i++) out[i] = or_o1_search(nd, nn, root, bytes + off[i], off[i + 1] - off[i], max_bytes);
    return 0;
}

int or_o1_batch(const or_node* nd, int nn, int root, const uint8_t* bytes, const int64_t* off, int64_t n,
                uint8_t* out, int64_t max_bytes, int nthreads) {
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
    for (int64_t i = 0; i < n; i++) {
        int r = or_o1(nd, nn, root, bytes + off[i], off[i + 1] - off[i], max_bytes);
        out[i] = (uint8_t)(r < 0 ? 255 : r);
    }
    return 0;
}

/* Pairs: n (expression, string) pairs, pair i decided by O2 for expression
 * pr[i] on string i.  The expressions are concatenated node arrays:
 * expression r is nd[ns[r] .. ns[r+1]) with its root at index root[r] of
 * that slice.  A plain loop over the pairs, spread over nthreads OpenMP
 * threads; out[i] = 0/1.  Returns -1 on a malformed tree. */
int or_o2_pairs(const or_node* nd, const int64_t* ns, const int32_t* root, int64_t nreg, const int32_t* pr,
                const uint8_t* bytes, const int64_t* off, int64_t n, uint8_t* out, int nthreads) {
    int64_t total = ns[nreg];
    int32_t* cont = (int32_t*)malloc(sizeof(int32_t) * (size_t)(total > 0 ? total : 1));
    if (!cont) return -1;
    int failed = 0, maxnn = 0;
    for (int64_t r = 0; r < nreg; r++) {
        int nn = (int)(ns[r + 1] - ns[r]);
        if (nn > maxnn) maxnn = nn;
        if (or_cont(nd + ns[r], nn, root[r], cont + ns[r]) != 0) failed = 1;
    }
    if (failed) { free(cont); return -1; }
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
    {
        int32_t* buf = (int32_t*)malloc(O2_BUF_BYTES(maxnn));
        if (!buf) failed = 1;
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < n; i++) {
            if (!buf) continue;
            int64_t r = pr[i];
            int nn = (int)(ns[r + 1] - ns[r]);
            out[i] = (uint8_t)o2_run(nd + ns[r], nn, root[r], cont + ns[r], bytes + off[i], off[i + 1] - off[i],
                                     NULL, NULL, buf);
        }
        free(buf);
    }
    free(cont);
    return failed ? -1 : 0;
}
