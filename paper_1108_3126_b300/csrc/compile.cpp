// compile.cpp -- host compiler: pattern text -> pointer tree with cont ->
// evolutions (Def 5.1) -> per-byte successor tables (Def 5.2) -> optional
// cache of macro steps.  Everything here runs once per expression; nothing
// here runs per input byte.
//
// Rathnayake & Thielecke, "Regular Expression Matching and Operational
// Semantics" (SOS 2011): the tree is the heap pi of Section 4 (Defs 4.1-4.3),
// cont is Def 4.4, the epsilon edges walked by the closure are the unlabelled
// transitions of Fig 4.2, and the closure's visited set keyed by node id is
// the pointer-equality redundancy elimination of Sections 3 and 6 (psi of
// Def 6.1), which is what terminates epsilon loops such as (eps*)*.
#include <algorithm>
#include <cstring>
#include <unordered_map>

#include "rx_internal.h"

namespace rx {

namespace {

// ------------------------------------------------------------------ parser
struct Parser {
    const uint8_t* s;
    size_t n, pos = 0;
    std::vector<rx_node>& out;
    int depth = 0;
    bool failed = false;
    bool too_large = false;

    Parser(const uint8_t* s_, size_t n_, std::vector<rx_node>& o) : s(s_), n(n_), out(o) {}

    int mk(uint8_t kind, uint8_t byte, int l, int r) {
        if (out.size() >= (size_t)RX_MAX_NODES) {
            too_large = failed = true;
            return -1;
        }
        rx_node x;
        x.kind = kind;
        x.byte = byte;
        x.pad = 0;
        x.l = l;
        x.r = r;
        out.push_back(x);
        return (int)out.size() - 1;
    }
    bool at(uint8_t c) const { return pos < n && s[pos] == c; }

    int alt() {
        if (++depth > 20000) {
            too_large = failed = true;
            return -1;
        }
        int t = cat();
        while (!failed && at('|')) {
            pos++;
            int r = cat();
            if (failed) break;
            t = mk(RX_ALT, 0, t, r);
        }
        depth--;
        return t;
    }
    int cat() {
        int t = -1;
        while (!failed && pos < n && s[pos] != '|' && s[pos] != ')') {
            int x = post();
            if (failed) return -1;
            t = (t < 0) ? x : mk(RX_CAT, 0, t, x);
        }
        if (!failed && t < 0) t = mk(RX_EPS, 0, -1, -1);
        return t;
    }
    int post() {
        int t = atom();
        while (!failed && at('*')) {
            pos++;
            t = mk(RX_STAR, 0, t, -1);
        }
        return t;
    }
    static int hexv(uint8_t c) {
        if (c >= '0' && c <= '9') return c - '0';
        if (c >= 'a' && c <= 'f') return c - 'a' + 10;
        if (c >= 'A' && c <= 'F') return c - 'A' + 10;
        return -1;
    }
    int atom() {
        uint8_t c = s[pos];
        if (c == '(') {
            pos++;
            int t = alt();
            if (failed) return -1;
            if (!at(')')) {
                failed = true;
                return -1;
            }
            pos++;
            return t;
        }
        if (c == '*') {
            failed = true;
            return -1;
        }
        if (c == '\\') {
            if (pos + 1 >= n) {
                failed = true;
                return -1;
            }
            uint8_t d = s[pos + 1];
            if (d == 'e') {
                pos += 2;
                return mk(RX_EPS, 0, -1, -1);
            }
            if (d == 'x') {
                int h1 = pos + 2 < n ? hexv(s[pos + 2]) : -1;
                int h2 = pos + 3 < n ? hexv(s[pos + 3]) : -1;
                if (h1 < 0 || h2 < 0) {
                    failed = true;
                    return -1;
                }
                pos += 4;
                return mk(RX_CHAR, (uint8_t)(h1 * 16 + h2), -1, -1);
            }
            pos += 2;
            return mk(RX_CHAR, d, -1, -1);
        }
        pos++;
        return mk(RX_CHAR, c, -1, -1);
    }
};

inline void setbit(uint32_t* v, int b) { v[b >> 5] |= 1u << (b & 31); }

}  // namespace

rx_status parse_pattern(const char* pat, size_t len, std::vector<rx_node>& nodes, size_t& err_pos,
                        std::string& msg) {
    nodes.clear();
    Parser P((const uint8_t*)pat, len, nodes);
    int root = P.alt();
    if (!P.failed && P.pos != len) P.failed = true;  // stray ')'
    if (P.failed) {
        err_pos = P.pos;
        if (P.too_large) {
            msg = "pattern too large or too deeply nested";
            return RX_ERR_TOO_LARGE;
        }
        msg = "syntax error at byte " + std::to_string(P.pos);
        return RX_ERR_PARSE;
    }
    // renumber in preorder (root = 0)
    std::vector<rx_node> pre;
    pre.reserve(nodes.size());
    std::vector<std::pair<int, int>> st;  // (old id, new parent slot encoded)
    std::vector<int> newid(nodes.size(), -1);
    std::vector<int> stack{root};
    while (!stack.empty()) {
        int p = stack.back();
        stack.pop_back();
        newid[p] = (int)pre.size();
        pre.push_back(nodes[p]);
        const rx_node& x = nodes[p];
        if (x.kind == RX_CAT || x.kind == RX_ALT) {
            stack.push_back(x.r);
            stack.push_back(x.l);
        } else if (x.kind == RX_STAR) {
            stack.push_back(x.l);
        }
    }
    for (auto& x : pre) {
        if (x.l >= 0) x.l = newid[x.l];
        if (x.r >= 0) x.r = newid[x.r];
    }
    nodes.swap(pre);
    return RX_OK;
}

rx_status compile_tree(const rx_node* in, size_t n, int32_t root, uint32_t flags, Compiled& C,
                       std::string& msg) {
    if (!in || n == 0 || root < 0 || (size_t)root >= n) {
        msg = "empty tree or root out of range";
        return RX_ERR_INVALID_ARG;
    }
    if (n > (size_t)(1 << 26)) {
        msg = "node array too large";
        return RX_ERR_TOO_LARGE;
    }
    // ---- 1. walk the tree from the root in preorder; reject sharing/cycles
    std::vector<int32_t> newid(n, -1);
    std::vector<int32_t> stack{root};
    C.nodes.clear();
    C.orig_id.clear();
    while (!stack.empty()) {
        int p = stack.back();
        stack.pop_back();
        if (p < 0 || (size_t)p >= n) {
            msg = "child index out of range";
            return RX_ERR_INVALID_ARG;
        }
        if (newid[p] >= 0) {
            msg = "node " + std::to_string(p) + " reachable twice (shared subtree or cycle)";
            return RX_ERR_INVALID_ARG;
        }
        if (C.nodes.size() >= (size_t)RX_MAX_NODES) {
            msg = "more than RX_MAX_NODES nodes";
            return RX_ERR_TOO_LARGE;
        }
        newid[p] = (int32_t)C.nodes.size();
        rx_node x = in[p];
        x.pad = 0;
        switch (x.kind) {
        case RX_CHAR:
        case RX_EPS:
            x.l = x.r = -1;
            break;
        case RX_STAR:
            x.r = -1;
            stack.push_back(x.l);
            break;
        case RX_CAT:
        case RX_ALT:
            stack.push_back(x.r);
            stack.push_back(x.l);
            break;
        default:
            msg = "unknown node kind " + std::to_string((int)x.kind);
            return RX_ERR_INVALID_ARG;
        }
        C.nodes.push_back(x);
        C.orig_id.push_back(p);
    }
    const int nn = (int)C.nodes.size();
    for (auto& x : C.nodes) {
        if (x.l >= 0) x.l = newid[x.l];
        if (x.r >= 0) x.r = newid[x.r];
    }
    // ---- 2. cont (Def 4.4); preorder puts parents before children
    C.cont.assign(nn, -1);
    for (int p = 0; p < nn; p++) {
        const rx_node& x = C.nodes[p];
        if (x.kind == RX_ALT) {
            C.cont[x.l] = C.cont[p];
            C.cont[x.r] = C.cont[p];
        } else if (x.kind == RX_CAT) {
            C.cont[x.l] = x.r;
            C.cont[x.r] = C.cont[p];
        } else if (x.kind == RX_STAR) {
            C.cont[x.l] = p;
        }
    }
    // ---- 3. positions: CHAR nodes in preorder = left to right
    C.pos_node.clear();
    std::vector<int32_t> pos_of(nn, -1);
    for (int p = 0; p < nn; p++)
        if (C.nodes[p].kind == RX_CHAR) {
            pos_of[p] = (int32_t)C.pos_node.size();
            C.pos_node.push_back(p);
        }
    C.m = (int)C.pos_node.size();
    const int m = C.m;
    if (m > RX_MAX_POSITIONS) {
        msg = "more than RX_MAX_POSITIONS positions";
        return RX_ERR_TOO_LARGE;
    }
    // ---- 4. bit layout: positions grouped by byte so that the positions a
    // byte can advance are contiguous bits.  When every group has at most
    // kGroupMaxBits bits and the groups pack into two words without
    // straddling a word boundary, the thread variant can index its tables
    // with one shift-and-mask per byte.
    std::vector<std::vector<int>> groups(256);
    for (int q = 0; q < m; q++) groups[C.nodes[C.pos_node[q]].byte].push_back(q);
    C.pos_bit.assign(m, -1);
    bool packed = false;
    {
        int maxg = 0;
        for (auto& g : groups) maxg = std::max(maxg, (int)g.size());
        if (maxg <= kGroupMaxBits && m + 1 <= 64) {
            std::vector<int> order;
            for (int c = 0; c < 256; c++)
                if (!groups[c].empty()) order.push_back(c);
            std::stable_sort(order.begin(), order.end(),
                             [&](int a, int b) { return groups[a].size() > groups[b].size(); });
            int fill[2] = {0, 0};
            std::vector<int> word_of(256, -1);
            bool ok = true;
            for (int c : order) {
                int g = (int)groups[c].size();
                int w = (fill[0] + g <= 32) ? 0 : ((fill[1] + g <= 32) ? 1 : -1);
                if (w < 0) {
                    ok = false;
                    break;
                }
                word_of[c] = w;
                fill[w] += g;
            }
            // null takes one more bit
            int null_w = (fill[0] < 32) ? 0 : ((fill[1] < 32) ? 1 : -1);
            if (ok && null_w >= 0) {
                int nxt[2] = {0, 32};
                for (int c : order)
                    for (int q : groups[c]) C.pos_bit[q] = nxt[word_of[c]]++;
                C.null_bit = nxt[null_w]++;
                C.nbits = (fill[1] > 0 || null_w == 1) ? nxt[1] : nxt[0];
                packed = true;
            }
        }
    }
    if (!packed) {
        int b = 0;
        for (int c = 0; c < 256; c++)
            for (int q : groups[c]) C.pos_bit[q] = b++;
        C.null_bit = b++;
        C.nbits = b;
    }
    C.W = (C.nbits + 31) / 32;
    const int W = C.W;
    // ---- 5. evolutions (Def 5.1) of {root} and of {cont p}, by a depth-first
    // walk over the unlabelled transitions of Fig 4.2:
    //   p1|p2 -> p1, p2     p1.p2 -> p1     p1* -> p1, cont p     eps -> cont p
    // stopping at CHAR nodes (which wait for a byte) and at null.  The walk
    // visits each node at most once (visited set keyed by node id).
    std::vector<int32_t> stamp(nn, -1);
    int cur_stamp = 0;
    std::unordered_map<int32_t, std::vector<uint32_t>> memo;
    auto closure = [&](int32_t q) -> const std::vector<uint32_t>& {
        auto it = memo.find(q);
        if (it != memo.end()) return it->second;
        std::vector<uint32_t> v(W, 0u);
        int s = cur_stamp++;
        std::vector<int32_t> st;
        auto push = [&](int32_t x) {
            if (x < 0) {
                setbit(v.data(), C.null_bit);
                return;
            }
            if (stamp[x] == s) return;
            stamp[x] = s;
            st.push_back(x);
        };
        push(q);
        while (!st.empty()) {
            int32_t p = st.back();
            st.pop_back();
            const rx_node& x = C.nodes[p];
            switch (x.kind) {
            case RX_CHAR:
                setbit(v.data(), C.pos_bit[pos_of[p]]);
                break;
            case RX_EPS:
                push(C.cont[p]);
                break;
            case RX_STAR:
                push(x.l);
                push(C.cont[p]);
                break;
            case RX_CAT:
                push(x.l);
                break;
            case RX_ALT:
                push(x.l);
                push(x.r);
                break;
            }
        }
        return memo.emplace(q, std::move(v)).first->second;
    };
    C.start = closure(0);
    C.follow_pos.assign((size_t)m * W, 0u);
    C.follow_bit.assign((size_t)C.nbits * W, 0u);
    for (int q = 0; q < m; q++) {
        const std::vector<uint32_t>& f = closure(C.cont[C.pos_node[q]]);
        std::copy(f.begin(), f.end(), C.follow_pos.begin() + (size_t)q * W);
        std::copy(f.begin(), f.end(), C.follow_bit.begin() + (size_t)C.pos_bit[q] * W);
    }
    C.nullable = (C.start[C.null_bit >> 5] >> (C.null_bit & 31)) & 1u;
    // ---- 6. B[c]: the positions a byte c can advance (Def 5.2: pi(p) = a)
    C.B.assign((size_t)256 * W, 0u);
    for (int q = 0; q < m; q++) setbit(&C.B[(size_t)C.nodes[C.pos_node[q]].byte * W], C.pos_bit[q]);
    // ---- 7. thread-variant tables: for byte c with group bits [lo, lo+g) in
    // one word, entry x (0 <= x < 2^g) holds the union of follow over the
    // positions whose group bits are set in x.  Entry 0 of the table area is
    // the empty set (bytes labelling no position).
    C.gl_ok = packed && W <= 2;
    C.gl_desc.assign(256, make_uint2(0u, 0u));
    C.gl_tt.clear();
    if (C.gl_ok) {
        C.gl_tt.assign(W, 0u);  // shared empty entry
        for (int c = 0; c < 256; c++) {
            const auto& g = groups[c];
            if (g.empty()) continue;
            int lo = C.pos_bit[g[0]];
            int cnt = (int)g.size();
            for (int i = 1; i < cnt; i++)
                if (C.pos_bit[g[i]] != lo + i) C.gl_ok = false;
            uint32_t base = (uint32_t)C.gl_tt.size();
            for (int x = 0; x < (1 << cnt); x++) {
                std::vector<uint32_t> e(W, 0u);
                for (int i = 0; i < cnt; i++)
                    if ((x >> i) & 1)
                        for (int k = 0; k < W; k++) e[k] |= C.follow_bit[(size_t)(lo + i) * W + k];
                C.gl_tt.insert(C.gl_tt.end(), e.begin(), e.end());
            }
            uint32_t mask = (1u << cnt) - 1u;
            C.gl_desc[c] = make_uint2((uint32_t)(lo & 31) | ((uint32_t)(lo >> 5) << 5) | (mask << 8), base);
        }
    }
    // ---- 8. cache of macro steps: every active set reachable from the
    // start, each byte's successor computed by Def 5.2 from the tables
    // above.  Kept only when it stays small.
    C.memo_K = 0;
    C.memo_T.clear();
    C.memo_acc.clear();
    C.wide_K = 0;
    C.wide_T.clear();
    if (!(flags & RX_COMPILE_NO_MEMO)) {
        struct VHash {
            size_t operator()(const std::vector<uint32_t>& v) const {
                uint64_t h = 1469598103934665603ull;
                for (uint32_t x : v) h = (h ^ x) * 1099511628211ull;
                return (size_t)h;
            }
        };
        std::unordered_map<std::vector<uint32_t>, int, VHash> id;
        std::vector<std::vector<uint32_t>> states;
        std::vector<uint32_t> zero(W, 0u);
        id[zero] = 0;
        states.push_back(zero);
        auto get = [&](const std::vector<uint32_t>& v) -> int {
            auto it = id.find(v);
            if (it != id.end()) return it->second;
            int k = (int)states.size();
            id.emplace(v, k);
            states.push_back(v);
            return k;
        };
        int s0 = get(C.start);
        std::vector<int> labels;
        for (int c = 0; c < 256; c++)
            if (!groups[c].empty()) labels.push_back(c);
        std::vector<uint32_t> T;
        bool ok = true;
        // explores states [from, ...) until every successor is known or the
        // count passes `limit` (then false); T gets their rows (ids * 256).
        // Both passes share one budget of kWideMaxWork word operations.
        long long work = 0;
        auto explore = [&](size_t from, int limit) {
            for (size_t k = from; k < states.size(); k++) {
                if ((int)states.size() > limit || work > kWideMaxWork) return false;
                T.resize((k + 1) * 256, 0u);
                for (int c : labels) {
                    std::vector<uint32_t> nx(W, 0u);
                    for (int w = 0; w < W; w++) {
                        uint32_t s = states[k][w] & C.B[(size_t)c * W + w];
                        while (s) {
                            int b = __builtin_ctz(s);
                            s &= s - 1;
                            const uint32_t* row = &C.follow_bit[(size_t)(w * 32 + b) * W];
                            for (int z = 0; z < W; z++) nx[z] |= row[z];
                            work += W;
                        }
                    }
                    int t = get(nx);
                    T[k * 256 + c] = (uint32_t)t * 256u;
                }
            }
            return (int)states.size() <= limit;
        };
        ok = explore(0, kMemoMaxStates);
        if (!ok && W > kSparseMaxWords && !(flags & RX_COMPILE_NO_WIDE)) {
            // 8b. the wide tier, for sets too wide for a thread: go on from
            // the first state without a row (the first pass stops between rows)
            if (explore(T.size() / 256, kWideMaxStates)) {
                const int K = (int)states.size();
                std::vector<uint32_t> img_off(257, 0);
                std::vector<uint16_t> img, imgpos((size_t)K * 256, 0);
                std::vector<int> at(K);
                int maximg = 0;
                for (int c = 0; c < 256 && maximg <= kWideMaxImg; c++) {
                    std::fill(at.begin(), at.end(), -1);
                    for (int k = 0; k < K; k++) at[T[(size_t)k * 256 + c] / 256u] = 0;
                    int n = 0;
                    for (int k = 0; k < K; k++)
                        if (at[k] >= 0) {
                            at[k] = n++;
                            img.push_back((uint16_t)k);
                        }
                    for (int k = 0; k < K; k++)
                        imgpos[(size_t)c * K + k] = (uint16_t)at[T[(size_t)k * 256 + c] / 256u];
                    img_off[c + 1] = (uint32_t)img.size();
                    maximg = std::max(maximg, n);
                }
                if (maximg <= kWideMaxImg) {
                    C.wide_K = K;
                    C.wide_maximg = maximg;
                    C.wide_T.resize((size_t)K * 256);
                    for (size_t i = 0; i < C.wide_T.size(); i++) C.wide_T[i] = (uint16_t)(T[i] / 256u);
                    C.wide_acc.resize(K);
                    for (int k = 0; k < K; k++)
                        C.wide_acc[k] = (states[k][C.null_bit >> 5] >> (C.null_bit & 31)) & 1u;
                    C.wide_start = (uint32_t)s0;
                    C.wide_img_off.swap(img_off);
                    C.wide_img.swap(img);
                    C.wide_imgpos.swap(imgpos);
                }
            }
        }
        if (ok && (int)states.size() <= kMemoMaxStates) {
            C.memo_K = (int)states.size();
            C.memo_T.swap(T);
            C.memo_T.resize((size_t)C.memo_K * 256, 0u);
            C.memo_acc.resize(C.memo_K);
            for (int k = 0; k < C.memo_K; k++)
                C.memo_acc[k] = (states[k][C.null_bit >> 5] >> (C.null_bit & 31)) & 1u;
            C.memo_start = (uint32_t)s0 * 256u;
            // 8a. the image of every byte's column: after one byte c every
            // incoming state is one of these few states, so the effect of a
            // chunk starting with c is fixed by its effect on them
            C.memo_img_off.assign(257, 0);
            C.memo_img.clear();
            C.memo_imgpos.assign((size_t)C.memo_K * 256, 0);
            std::vector<int> at(C.memo_K);
            for (int c = 0; c < 256; c++) {
                std::fill(at.begin(), at.end(), -1);
                for (int k = 0; k < C.memo_K; k++) at[C.memo_T[(size_t)k * 256 + c] / 256u] = 0;
                int n = 0;
                for (int k = 0; k < C.memo_K; k++)
                    if (at[k] >= 0) {
                        at[k] = n++;
                        C.memo_img.push_back((uint8_t)k);
                    }
                for (int k = 0; k < C.memo_K; k++)
                    C.memo_imgpos[(size_t)c * C.memo_K + k] = (uint8_t)at[C.memo_T[(size_t)k * 256 + c] / 256u];
                C.memo_img_off[c + 1] = (uint16_t)C.memo_img.size();
            }
        }
    }
    // ---- 8c. cache for unanchored search (a match may start at any
    // position): the sets reachable when the start set is added back after
    // every byte, S' = (macro step of S on c) U Start, from S0 = Start.  A
    // set holding null marks the end of a match.  States are renumbered so
    // that these accepting sets come last (ids >= srch_acc0).
    C.srch_K = 0;
    C.srch_T.clear();
    if ((flags & RX_COMPILE_SEARCH) && !(flags & RX_COMPILE_NO_MEMO)) {
        struct VHash2 {
            size_t operator()(const std::vector<uint32_t>& v) const {
                uint64_t h = 1469598103934665603ull;
                for (uint32_t x : v) h = (h ^ x) * 1099511628211ull;
                return (size_t)h;
            }
        };
        std::unordered_map<std::vector<uint32_t>, int, VHash2> id;
        std::vector<std::vector<uint32_t>> states;
        auto get = [&](const std::vector<uint32_t>& v) -> int {
            auto it = id.find(v);
            if (it != id.end()) return it->second;
            int k = (int)states.size();
            id.emplace(v, k);
            states.push_back(v);
            return k;
        };
        get(C.start);
        std::vector<int> T;
        bool ok = true;
        for (size_t k = 0; k < states.size() && ok; k++) {
            T.resize((k + 1) * 256, 0);
            for (int c = 0; c < 256; c++) {
                std::vector<uint32_t> nx(C.start.begin(), C.start.end());
                if (!groups[c].empty())
                    for (int w = 0; w < W; w++) {
                        uint32_t sb = states[k][w] & C.B[(size_t)c * W + w];
                        while (sb) {
                            int b = __builtin_ctz(sb);
                            sb &= sb - 1;
                            const uint32_t* row = &C.follow_bit[(size_t)(w * 32 + b) * W];
                            for (int z = 0; z < W; z++) nx[z] |= row[z];
                        }
                    }
                T[k * 256 + c] = get(nx);
                if ((int)states.size() > kMemoMaxStates) {
                    ok = false;
                    break;
                }
            }
        }
        if (ok) {
            const int K = (int)states.size();
            auto accepts = [&](int k) { return (states[k][C.null_bit >> 5] >> (C.null_bit & 31)) & 1u; };
            std::vector<int> newid(K);
            int nacc = 0;
            for (int k = 0; k < K; k++) nacc += accepts(k) ? 1 : 0;
            int lo = 0, hi = K - nacc;
            for (int k = 0; k < K; k++) newid[k] = accepts(k) ? hi++ : lo++;
            C.srch_K = K;
            C.srch_acc0 = K - nacc;
            C.srch_start = (uint32_t)newid[0] * 256u;
            C.srch_T.assign((size_t)K * 256, 0u);
            for (int k = 0; k < K; k++)
                for (int c = 0; c < 256; c++) C.srch_T[(size_t)newid[k] * 256 + c] = (uint32_t)newid[T[k * 256 + c]] * 256u;
        }
    }
    // ---- 8b. two macro steps per lookup: when every label lies in one
    // aligned window of 32 byte values, entry 32*j + i of a state's pair row
    // is the state after reading byte lo+i then byte lo+j (two steps of the
    // cache above); bytes outside the window use the single-byte row.  The
    // device gets these rows rearranged into planes of 8 states (see
    // DevTables::bgp_T), where a lookup is one add to the state's address.
    C.bg_T.clear();
    C.bgp_T.clear();
    C.bg_lo = -1;
    if (C.memo_K > 0 && C.memo_K <= kPairMaxStates && m > 0) {
        int lo = 256, hi = -1;
        for (int c = 0; c < 256; c++)
            if (!groups[c].empty()) {
                lo = std::min(lo, c);
                hi = std::max(hi, c);
            }
        int w0 = lo & ~31;
        if (hi < w0 + 32) {
            const int K = C.memo_K;
            C.bg_lo = w0;
            C.bg_T.assign((size_t)K * 1280, 0);
            for (int k = 0; k < K; k++) {
                uint16_t* row = &C.bg_T[(size_t)k * 1280];
                for (int i = 0; i < 32; i++) {
                    uint32_t mid = C.memo_T[(size_t)k * 256 + w0 + i] / 256u;
                    for (int j = 0; j < 32; j++) row[j * 32 + i] = (uint16_t)(C.memo_T[(size_t)mid * 256 + w0 + j] / 256u);
                }
                for (int c = 0; c < 256; c++) row[1024 + c] = (uint16_t)(C.memo_T[(size_t)k * 256 + c] / 256u);
            }
            // planes of 8 states: 32 pair rows of 258 entries (256 + a 4-byte
            // pad, so that the second byte moves a lookup across the banks),
            // then 8 single-byte rows of 256; 10,304 entries a plane
            auto code = [](uint32_t s) { return (uint16_t)((s >> 3) * 322u + (s & 7u)); };
            const int planes = (K + 7) / 8;
            C.bgp_T.assign((size_t)planes * 10304, 0);
            for (int k = 0; k < K; k++) {
                uint16_t* P = &C.bgp_T[(size_t)(k >> 3) * 10304 + (size_t)(k & 7) * 32];
                const uint16_t* row = &C.bg_T[(size_t)k * 1280];
                for (int j = 0; j < 32; j++)
                    for (int i = 0; i < 32; i++) P[j * 258 + i] = code(row[j * 32 + i]);
                for (int c = 0; c < 256; c++) P[8256 + (c >> 5) * 256 + (c & 31)] = code(row[1024 + c]);
            }
        }
    }
    // ---- 9. which kernel variants can run this expression
    C.variants = 0;
    if (C.memo_K > 0) C.variants |= 1u << RX_VARIANT_MEMO;
    if (C.gl_ok) C.variants |= 1u << RX_VARIANT_THREAD;
    if (W <= kSparseMaxWords) C.variants |= 1u << RX_VARIANT_SPARSE;
    if (W <= kWarpMaxWords) C.variants |= 1u << RX_VARIANT_WARP;
    C.variants |= 1u << RX_VARIANT_PAPER;
    return RX_OK;
}

}  // namespace rx
