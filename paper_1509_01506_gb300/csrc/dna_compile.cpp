// dna_compile.cpp -- the library's host-side pattern compilers and automaton analysis.
//
// Regex route: syntax tree -> Glushkov position automaton (nullable / first / last /
// follow sets) -> direct subset construction of Sigma*.L (the first positions are
// enabled at every step, which is the Sigma* prefix) -> Hopcroft minimisation ->
// canonical breadth-first numbering.
// k-mer route: Aho-Corasick trie with breadth-first failure links, completed into the
// failure-free DFA of Sec. III-B.1 (every state has a transition for every base, so
// every symbol costs the same work), then the same minimisation.
// Analysis: the definite depth of an automaton (pair-graph longest path), which bounds
// how many symbols before a chunk determine its start state exactly.

#include <algorithm>
#include <array>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include "../../include/dna_dfa.h"
#include "dna_internal.h"

namespace dnalib {
namespace {

int base_index(char c) {
    switch (c) {
        case 'A': case 'a': return 0;
        case 'C': case 'c': return 1;
        case 'G': case 'g': return 2;
        case 'T': case 't': return 3;
        default: return -1;
    }
}

// ----------------------------------------------------------------- syntax tree

enum Kind { LEAF, CAT, ALT, STAR, OPT };

struct Node {
    Kind kind;
    uint8_t set = 0;      // LEAF: accepted bases (bit s)
    int a = -1, b = -1;   // children
};

struct Parser {
    const char *s;
    size_t i = 0;
    std::vector<Node> nodes;
    int err = DNA_OK;

    int add(Node n) { nodes.push_back(n); return (int)nodes.size() - 1; }

    // Deep copy of a subtree (bounded repeats are expanded into copies, each copy with
    // its own Glushkov positions).
    int clone(int x) {
        Node n = nodes[x];
        if (n.a >= 0) n.a = clone(n.a);
        if (n.b >= 0) n.b = clone(n.b);
        return add(n);
    }

    bool number(int &v) {
        size_t st = i;
        v = 0;
        while (s[i] >= '0' && s[i] <= '9') {
            v = v * 10 + (s[i] - '0');
            if (v > 100000) return false;
            ++i;
        }
        return i > st;
    }

    int atom() {
        char c = s[i];
        if (c == '(') {
            ++i;
            int r = alt();
            if (err) return -1;
            if (s[i] != ')') { err = DNA_ERR_SYNTAX; return -1; }
            ++i;
            return r;
        }
        Node n; n.kind = LEAF;
        if (c == '[') {
            ++i;
            while (s[i] && s[i] != ']') {
                int b = base_index(s[i]);
                if (b < 0) { err = DNA_ERR_SYNTAX; return -1; }
                n.set |= (uint8_t)(1u << b);
                ++i;
            }
            if (s[i] != ']' || !n.set) { err = DNA_ERR_SYNTAX; return -1; }
            ++i;
            return add(n);
        }
        if (c == '.') { ++i; n.set = 15; return add(n); }
        int b = base_index(c);
        if (b < 0) { err = DNA_ERR_SYNTAX; return -1; }
        ++i;
        n.set = (uint8_t)(1u << b);
        return add(n);
    }

    int cat2(int x, int y) { if (x < 0) return y; Node n; n.kind = CAT; n.a = x; n.b = y; return add(n); }
    int star(int x) { Node n; n.kind = STAR; n.a = x; return add(n); }
    int opt(int x) { Node n; n.kind = OPT; n.a = x; return add(n); }

    // x{lo,hi}: lo copies, then hi-lo optional copies (or a starred copy).
    int repeat(int x, int lo, int hi) {
        int r = -1;
        for (int k = 0; k < lo; ++k) r = cat2(r, k == 0 ? x : clone(x));
        if (hi < 0) {
            int c = lo == 0 ? x : clone(x);
            r = cat2(r, star(c));
        } else {
            for (int k = lo; k < hi; ++k) {
                int c = (k == 0) ? x : clone(x);
                r = cat2(r, opt(c));
            }
        }
        return r;
    }

    int rep() {
        int x = atom();
        if (err) return -1;
        for (;;) {
            char c = s[i];
            if (c == '*') { ++i; x = star(x); }
            else if (c == '+') { ++i; x = cat2(x, star(clone(x))); }
            else if (c == '?') { ++i; x = opt(x); }
            else if (c == '{') {
                ++i;
                int lo, hi;
                if (!number(lo)) { err = DNA_ERR_SYNTAX; return -1; }
                if (s[i] == '}') { hi = lo; ++i; }
                else if (s[i] == ',') {
                    ++i;
                    if (s[i] == '}') { hi = -1; ++i; }
                    else {
                        if (!number(hi) || s[i] != '}' || hi < lo) { err = DNA_ERR_SYNTAX; return -1; }
                        ++i;
                    }
                } else { err = DNA_ERR_SYNTAX; return -1; }
                if (lo == 0 && hi == 0) { err = DNA_ERR_SYNTAX; return -1; }
                x = repeat(x, lo, hi);
            } else break;
        }
        return x;
    }

    int concat() {
        int r = -1;
        while (s[i] && s[i] != '|' && s[i] != ')') {
            int x = rep();
            if (err) return -1;
            r = cat2(r, x);
        }
        if (r < 0) err = DNA_ERR_SYNTAX;
        return r;
    }

    int alt() {
        int r = concat();
        if (err) return -1;
        while (s[i] == '|') {
            ++i;
            int y = concat();
            if (err) return -1;
            Node n; n.kind = ALT; n.a = r; n.b = y;
            r = add(n);
        }
        return r;
    }
};

// --------------------------------------------------------- Glushkov positions

using Bits = std::vector<uint64_t>;

struct Glushkov {
    int n_pos = 0;
    std::vector<uint8_t> pos_set;     // bases accepted at each position
    std::vector<Bits> follow;
    Bits first, last;
    bool nullable = false;
};

struct Info { bool nullable; Bits first, last; };

void bits_or(Bits &a, const Bits &b) { for (size_t k = 0; k < a.size(); ++k) a[k] |= b[k]; }

// 'roots_last' (optional): receives the last-position set of each listed subtree.
void build_glushkov(const std::vector<Node> &nodes, int root, Glushkov &g,
                    const std::vector<int> *roots = nullptr, std::vector<Bits> *roots_last = nullptr,
                    std::vector<bool> *roots_nullable = nullptr) {
    // assign positions to leaves reachable from root (iterative post-order)
    std::vector<int> order, stack{root};
    while (!stack.empty()) {
        int x = stack.back(); stack.pop_back();
        order.push_back(x);
        if (nodes[x].a >= 0) stack.push_back(nodes[x].a);
        if (nodes[x].b >= 0) stack.push_back(nodes[x].b);
    }
    std::vector<int> pos_of(nodes.size(), -1);
    for (int x : order)
        if (nodes[x].kind == LEAF) { pos_of[x] = g.n_pos++; g.pos_set.push_back(nodes[x].set); }
    size_t words = (size_t)(g.n_pos + 63) / 64;
    g.follow.assign(g.n_pos, Bits(words, 0));
    std::vector<Info> info(nodes.size());
    // children appear after parents in 'order', so reverse order is a post-order
    for (auto it = order.rbegin(); it != order.rend(); ++it) {
        int x = *it;
        const Node &n = nodes[x];
        Info &r = info[x];
        r.first.assign(words, 0);
        r.last.assign(words, 0);
        if (n.kind == LEAF) {
            int p = pos_of[x];
            r.nullable = false;
            r.first[p >> 6] |= 1ull << (p & 63);
            r.last[p >> 6] |= 1ull << (p & 63);
        } else if (n.kind == CAT) {
            const Info &A = info[n.a], &B = info[n.b];
            r.nullable = A.nullable && B.nullable;
            r.first = A.first; if (A.nullable) bits_or(r.first, B.first);
            r.last = B.last; if (B.nullable) bits_or(r.last, A.last);
            for (int p = 0; p < g.n_pos; ++p)
                if (A.last[p >> 6] >> (p & 63) & 1) bits_or(g.follow[p], B.first);
        } else if (n.kind == ALT) {
            const Info &A = info[n.a], &B = info[n.b];
            r.nullable = A.nullable || B.nullable;
            r.first = A.first; bits_or(r.first, B.first);
            r.last = A.last; bits_or(r.last, B.last);
        } else if (n.kind == STAR) {
            const Info &A = info[n.a];
            r.nullable = true; r.first = A.first; r.last = A.last;
            for (int p = 0; p < g.n_pos; ++p)
                if (A.last[p >> 6] >> (p & 63) & 1) bits_or(g.follow[p], A.first);
        } else {  // OPT
            const Info &A = info[n.a];
            r.nullable = true; r.first = A.first; r.last = A.last;
        }
    }
    g.first = info[root].first;
    g.last = info[root].last;
    g.nullable = info[root].nullable;
    if (roots && roots_last) {
        roots_last->clear();
        if (roots_nullable) roots_nullable->clear();
        for (int r : *roots) {
            roots_last->push_back(info[r].last);
            if (roots_nullable) roots_nullable->push_back(info[r].nullable);
        }
    }
}

// Direct subset construction of Sigma*.L over Glushkov positions: a DFA state is the
// set of positions that the last symbol can have matched. On base c the next set is
// every position p labelled with c that is either a first position (the Sigma* prefix
// lets a match start anywhere) or follows a position in the current set.
// 'lasts' (optional) holds one last-position set per pattern of a union: a DFA state's
// accept mask then has bit i set when its set meets pattern i's last positions.
int glushkov_dfa(const Glushkov &g, HostDfa &out, const std::vector<Bits> *lasts = nullptr) {
    size_t words = (size_t)(g.n_pos + 63) / 64;
    std::map<Bits, uint32_t> ids;
    std::vector<Bits> sets;
    Bits empty(words, 0);
    ids[empty] = 0;
    sets.push_back(empty);
    out.table.clear();
    out.accept.clear();
    out.accept.push_back(0);
    for (size_t d = 0; d < sets.size(); ++d) {
        Bits reach = g.first;
        for (int p = 0; p < g.n_pos; ++p)
            if (sets[d][p >> 6] >> (p & 63) & 1) bits_or(reach, g.follow[p]);
        for (int c = 0; c < 4; ++c) {
            Bits nx(words, 0);
            for (int p = 0; p < g.n_pos; ++p)
                if ((reach[p >> 6] >> (p & 63) & 1) && (g.pos_set[p] >> c & 1))
                    nx[p >> 6] |= 1ull << (p & 63);
            auto it = ids.find(nx);
            uint32_t id;
            if (it == ids.end()) {
                id = (uint32_t)sets.size();
                if (id >= (1u << 22)) return DNA_ERR_CAPACITY;
                ids.emplace(nx, id);
                uint32_t mask = 0;
                if (lasts) {
                    for (size_t i = 0; i < lasts->size(); ++i) {
                        bool hit = false;
                        for (size_t k = 0; k < words; ++k) hit |= (nx[k] & (*lasts)[i][k]) != 0;
                        if (hit) mask |= 1u << i;
                    }
                } else {
                    bool acc = false;
                    for (size_t k = 0; k < words; ++k) acc |= (nx[k] & g.last[k]) != 0;
                    mask = acc ? 1u : 0u;
                }
                sets.push_back(nx);
                out.accept.push_back(mask);
            } else {
                id = it->second;
            }
            out.table.push_back(id);
        }
    }
    out.n_states = (uint32_t)sets.size();
    return DNA_OK;
}

// ------------------------------------------------------- Hopcroft minimisation

int hopcroft(const HostDfa &in, HostDfa &out) {
    const uint32_t n = in.n_states;
    // inverse transitions per symbol (CSR)
    std::vector<uint32_t> inv_start[4], inv[4];
    for (int c = 0; c < 4; ++c) {
        inv_start[c].assign(n + 1, 0);
        for (uint32_t s = 0; s < n; ++s) inv_start[c][in.table[4 * s + c] + 1]++;
        for (uint32_t t = 0; t < n; ++t) inv_start[c][t + 1] += inv_start[c][t];
        inv[c].resize(n);
        std::vector<uint32_t> fill(inv_start[c].begin(), inv_start[c].end() - 1);
        for (uint32_t s = 0; s < n; ++s) inv[c][fill[in.table[4 * s + c]]++] = s;
    }
    // blocks as contiguous ranges of 'elems'
    std::vector<uint32_t> elems(n), where(n), block(n);
    std::vector<uint32_t> bstart, bend, marked;
    {
        // one initial block per distinct accept mask (for a single pattern: F and Q \ F)
        std::vector<uint32_t> masks(in.accept.begin(), in.accept.begin() + n);
        std::sort(masks.begin(), masks.end());
        masks.erase(std::unique(masks.begin(), masks.end()), masks.end());
        uint32_t k = 0;
        for (uint32_t m : masks) {
            uint32_t st = k;
            for (uint32_t s = 0; s < n; ++s)
                if (in.accept[s] == m) { elems[k] = s; where[s] = k; ++k; }
            uint32_t b = (uint32_t)bstart.size();
            bstart.push_back(st); bend.push_back(k); marked.push_back(0);
            for (uint32_t i = st; i < k; ++i) block[elems[i]] = b;
        }
    }
    std::vector<std::vector<uint8_t>> in_work;
    std::deque<std::pair<uint32_t, int>> work;
    for (uint32_t b = 0; b < bstart.size(); ++b) {
        in_work.push_back(std::vector<uint8_t>(4, 1));
        for (int c = 0; c < 4; ++c) work.emplace_back(b, c);
    }
    std::vector<uint32_t> touched, xs;
    while (!work.empty()) {
        auto [B, c] = work.front();
        work.pop_front();
        in_work[B][c] = 0;
        xs.clear();
        for (uint32_t i = bstart[B]; i < bend[B]; ++i) {
            uint32_t t = elems[i];
            for (uint32_t k = inv_start[c][t]; k < inv_start[c][t + 1]; ++k) xs.push_back(inv[c][k]);
        }
        touched.clear();
        for (uint32_t s : xs) {
            uint32_t Y = block[s];
            uint32_t front = bstart[Y] + marked[Y];
            if (where[s] < front) continue;  // already marked
            // swap s to the front region of its block
            uint32_t other = elems[front];
            std::swap(elems[where[s]], elems[front]);
            where[other] = where[s];
            where[s] = front;
            if (marked[Y]++ == 0) touched.push_back(Y);
        }
        for (uint32_t Y : touched) {
            uint32_t m = marked[Y], size = bend[Y] - bstart[Y];
            marked[Y] = 0;
            if (m == size) continue;
            uint32_t Z = (uint32_t)bstart.size();  // new block = the marked front part
            bstart.push_back(bstart[Y]); bend.push_back(bstart[Y] + m); marked.push_back(0);
            bstart[Y] += m;
            for (uint32_t i = bstart[Z]; i < bend[Z]; ++i) block[elems[i]] = Z;
            in_work.push_back(std::vector<uint8_t>(4, 0));
            for (int d = 0; d < 4; ++d) {
                if (in_work[Y][d]) { in_work[Z][d] = 1; work.emplace_back(Z, d); }
                else {
                    uint32_t small = (bend[Z] - bstart[Z] <= bend[Y] - bstart[Y]) ? Z : Y;
                    in_work[small][d] = 1;
                    work.emplace_back(small, d);
                }
            }
        }
    }
    // canonical breadth-first numbering of the blocks from the block of state 0
    uint32_t nb = (uint32_t)bstart.size();
    std::vector<int64_t> newid(nb, -1);
    std::vector<uint32_t> queue;
    newid[block[0]] = 0;
    queue.push_back(block[0]);
    for (size_t h = 0; h < queue.size(); ++h) {
        uint32_t rep = elems[bstart[queue[h]]];
        for (int c = 0; c < 4; ++c) {
            uint32_t d = block[in.table[4 * rep + c]];
            if (newid[d] < 0) { newid[d] = (int64_t)queue.size(); queue.push_back(d); }
        }
    }
    out.n_states = (uint32_t)queue.size();
    out.table.assign(4 * (size_t)out.n_states, 0);
    out.accept.assign(out.n_states, 0);
    for (uint32_t i = 0; i < out.n_states; ++i) {
        uint32_t rep = elems[bstart[queue[i]]];
        out.accept[i] = in.accept[rep];
        for (int c = 0; c < 4; ++c) out.table[4 * i + c] = (uint32_t)newid[block[in.table[4 * rep + c]]];
    }
    return DNA_OK;
}

}  // namespace

int minimise(const HostDfa &in, HostDfa &out) {
    if (in.n_states == 0) return DNA_ERR_INVALID_ARG;
    return hopcroft(in, out);
}

int compile_regex(const char *pattern, HostDfa &out) {
    if (!pattern) return DNA_ERR_INVALID_ARG;
    Parser ps;
    ps.s = pattern;
    int root = ps.alt();
    if (!ps.err && pattern[ps.i] != '\0') ps.err = DNA_ERR_SYNTAX;
    if (ps.err) return ps.err;
    Glushkov g;
    build_glushkov(ps.nodes, root, g);
    if (g.nullable) return DNA_ERR_EMPTY_WORD;
    HostDfa raw;
    int rc = glushkov_dfa(g, raw);
    if (rc) return rc;
    return hopcroft(raw, out);
}

int compile_regex_set(const std::vector<std::string> &patterns, HostDfa &out) {
    if (patterns.empty() || patterns.size() > 32) return DNA_ERR_INVALID_ARG;
    Parser ps;
    std::vector<int> roots;
    for (const std::string &pat : patterns) {
        ps.s = pat.c_str();
        ps.i = 0;
        int r = ps.alt();
        if (!ps.err && pat[ps.i] != '\0') ps.err = DNA_ERR_SYNTAX;
        if (ps.err) return ps.err;
        roots.push_back(r);
    }
    // the union of the patterns: every pattern keeps its own positions
    int root = roots[0];
    for (size_t i = 1; i < roots.size(); ++i) {
        Node n; n.kind = ALT; n.a = root; n.b = roots[i];
        root = ps.add(n);
    }
    Glushkov g;
    std::vector<Bits> lasts;
    std::vector<bool> nullable;
    build_glushkov(ps.nodes, root, g, &roots, &lasts, &nullable);
    for (bool nb : nullable)
        if (nb) return DNA_ERR_EMPTY_WORD;
    HostDfa raw;
    int rc = glushkov_dfa(g, raw, &lasts);
    if (rc) return rc;
    return hopcroft(raw, out);
}

int compile_kmers(const std::vector<std::string> &kmers, HostDfa &out) {
    if (kmers.empty()) return DNA_ERR_INVALID_ARG;
    std::vector<std::array<int32_t, 4>> go(1);
    go[0].fill(-1);
    std::vector<uint8_t> term(1, 0);
    for (const std::string &w : kmers) {
        if (w.empty()) return DNA_ERR_EMPTY_WORD;
        int32_t q = 0;
        for (char ch : w) {
            int c = base_index(ch);
            if (c < 0) return DNA_ERR_SYNTAX;
            if (go[q][c] < 0) {
                go[q][c] = (int32_t)go.size();
                go.emplace_back();
                go.back().fill(-1);
                term.push_back(0);
            }
            q = go[q][c];
        }
        term[q] = 1;
    }
    const uint32_t n = (uint32_t)go.size();
    if (n >= (1u << 24)) return DNA_ERR_CAPACITY;
    HostDfa raw;
    raw.n_states = n;
    raw.table.assign(4 * (size_t)n, 0);
    raw.accept.assign(n, 0);
    std::vector<uint32_t> fail(n, 0), order;
    order.reserve(n);
    // root: missing gotos loop back to the root
    for (int c = 0; c < 4; ++c) {
        if (go[0][c] >= 0) { raw.table[c] = (uint32_t)go[0][c]; order.push_back((uint32_t)go[0][c]); }
        else raw.table[c] = 0;
    }
    for (size_t h = 0; h < order.size(); ++h) {
        uint32_t q = order[h];
        raw.accept[q] = (uint32_t)(term[q] | raw.accept[fail[q]]);
        for (int c = 0; c < 4; ++c) {
            uint32_t via_fail = raw.table[4 * (size_t)fail[q] + c];
            if (go[q][c] >= 0) {
                uint32_t ch = (uint32_t)go[q][c];
                fail[ch] = via_fail;
                raw.table[4 * (size_t)q + c] = ch;
                order.push_back(ch);
            } else {
                raw.table[4 * (size_t)q + c] = via_fail;
            }
        }
    }
    return hopcroft(raw, out);
}

// Pair-graph analysis. For two distinct states p, q let f(p,q) be the number of
// symbols after which every word has brought them together; f = 1 + max over bases c
// of f(delta(p,c), delta(q,c)), with f(r,r) = 0. The definite depth is the maximum of
// f over all pairs (0 for a single state); a cycle among unmerged pairs means no
// finite depth. Computed bottom-up (Kahn's order on the reversed pair graph).
int definite_depth(const uint32_t *table, uint32_t n, int cap, uint32_t max_states) {
    if (n <= 1) return 0;
    if (n > max_states) return -1;
    auto tri = [n](uint32_t p, uint32_t q) -> uint64_t {  // p < q
        return (uint64_t)p * (2ull * n - p - 1) / 2 + (q - p - 1);
    };
    const uint64_t npairs = (uint64_t)n * (n - 1) / 2;
    std::vector<uint8_t> remaining(npairs, 4), level(npairs, 0);
    std::vector<uint32_t> inv_start[4], inv[4];
    for (int c = 0; c < 4; ++c) {
        inv_start[c].assign(n + 1, 0);
        for (uint32_t s = 0; s < n; ++s) inv_start[c][table[4 * (size_t)s + c] + 1]++;
        for (uint32_t t = 0; t < n; ++t) inv_start[c][t + 1] += inv_start[c][t];
        inv[c].resize(n);
        std::vector<uint32_t> fill(inv_start[c].begin(), inv_start[c].end() - 1);
        for (uint32_t s = 0; s < n; ++s) inv[c][fill[table[4 * (size_t)s + c]]++] = s;
    }
    std::vector<uint64_t> queue;  // finished pairs, packed p * n + q (p < q)
    int depth = 0;
    auto finish_pred = [&](uint32_t p, uint32_t q, int lvl) {
        if (p > q) std::swap(p, q);
        uint64_t k = tri(p, q);
        if (level[k] < lvl) level[k] = (uint8_t)std::min(lvl, 255);
        if (--remaining[k] == 0) queue.push_back((uint64_t)p * n + q);
    };
    // diagonal pairs (r, r) are merged at level 0
    for (uint32_t r = 0; r < n; ++r)
        for (int c = 0; c < 4; ++c)
            for (uint32_t i = inv_start[c][r]; i < inv_start[c][r + 1]; ++i)
                for (uint32_t j = i + 1; j < inv_start[c][r + 1]; ++j)
                    finish_pred(inv[c][i], inv[c][j], 1);
    size_t done = 0;
    for (size_t h = 0; h < queue.size(); ++h) {
        uint32_t r = (uint32_t)(queue[h] / n), s = (uint32_t)(queue[h] % n);
        int lvl = level[tri(r, s)];
        depth = std::max(depth, lvl);
        ++done;
        if (lvl > cap) continue;  // deeper than anything we use; predecessors only deeper
        for (int c = 0; c < 4; ++c)
            for (uint32_t i = inv_start[c][r]; i < inv_start[c][r + 1]; ++i)
                for (uint32_t j = inv_start[c][s]; j < inv_start[c][s + 1]; ++j)
                    finish_pred(inv[c][i], inv[c][j], lvl + 1);
    }
    if (done != npairs || depth > cap) return -1;
    return depth;
}

}  // namespace dnalib

// ------------------------------------------------------------------- C ABI

namespace {
int export_dfa(const dnalib::HostDfa &d, uint32_t **table_out, uint8_t **accept_out,
               uint32_t *n_out) {
    uint32_t *t = (uint32_t *)malloc(sizeof(uint32_t) * 4 * (size_t)d.n_states);
    uint8_t *a = (uint8_t *)calloc((d.n_states + 7) / 8, 1);
    if (!t || !a) { free(t); free(a); return DNA_ERR_NOMEM; }
    memcpy(t, d.table.data(), sizeof(uint32_t) * 4 * (size_t)d.n_states);
    for (uint32_t q = 0; q < d.n_states; ++q)
        if (d.accept[q]) a[q >> 3] |= (uint8_t)(1u << (q & 7));
    *table_out = t;
    *accept_out = a;
    *n_out = d.n_states;
    return DNA_OK;
}
}  // namespace

extern "C" int dna_compile_regex(const char *pattern, uint32_t **table_out,
                                 uint8_t **accept_out, uint32_t *n_states_out) {
    if (!pattern || !table_out || !accept_out || !n_states_out) return DNA_ERR_INVALID_ARG;
    try {
        dnalib::HostDfa d;
        int rc = dnalib::compile_regex(pattern, d);
        if (rc) return rc;
        return export_dfa(d, table_out, accept_out, n_states_out);
    } catch (const std::bad_alloc &) {
        return DNA_ERR_NOMEM;
    }
}

extern "C" int dna_compile_kmers(const char *const *kmers, uint32_t n_kmers,
                                 uint32_t **table_out, uint8_t **accept_out,
                                 uint32_t *n_states_out) {
    if (!kmers || n_kmers == 0 || !table_out || !accept_out || !n_states_out)
        return DNA_ERR_INVALID_ARG;
    try {
        std::vector<std::string> v;
        v.reserve(n_kmers);
        for (uint32_t i = 0; i < n_kmers; ++i) {
            if (!kmers[i]) return DNA_ERR_INVALID_ARG;
            v.emplace_back(kmers[i]);
        }
        dnalib::HostDfa d;
        int rc = dnalib::compile_kmers(v, d);
        if (rc) return rc;
        return export_dfa(d, table_out, accept_out, n_states_out);
    } catch (const std::bad_alloc &) {
        return DNA_ERR_NOMEM;
    }
}

extern "C" int dna_compile_regex_set(const char *const *patterns, uint32_t n_patterns,
                                     uint32_t **table_out, uint32_t **labels_out,
                                     uint32_t *n_states_out) {
    if (!patterns || n_patterns == 0 || n_patterns > 32 || !table_out || !labels_out || !n_states_out)
        return DNA_ERR_INVALID_ARG;
    try {
        std::vector<std::string> v;
        for (uint32_t i = 0; i < n_patterns; ++i) {
            if (!patterns[i]) return DNA_ERR_INVALID_ARG;
            v.emplace_back(patterns[i]);
        }
        dnalib::HostDfa d;
        int rc = dnalib::compile_regex_set(v, d);
        if (rc) return rc;
        uint32_t *t = (uint32_t *)malloc(sizeof(uint32_t) * 4 * (size_t)d.n_states);
        uint32_t *l = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)d.n_states);
        if (!t || !l) { free(t); free(l); return DNA_ERR_NOMEM; }
        memcpy(t, d.table.data(), sizeof(uint32_t) * 4 * (size_t)d.n_states);
        memcpy(l, d.accept.data(), sizeof(uint32_t) * (size_t)d.n_states);
        *table_out = t;
        *labels_out = l;
        *n_states_out = d.n_states;
        return DNA_OK;
    } catch (const std::bad_alloc &) {
        return DNA_ERR_NOMEM;
    }
}

extern "C" void dna_free_host(void *p) { free(p); }

extern "C" int dfa_analyze(const uint32_t *table, uint32_t n_states, int32_t *definite_depth) {
    if (!table || !definite_depth || n_states == 0 || n_states > (1u << 24)) return DNA_ERR_INVALID_ARG;
    for (uint64_t i = 0; i < 4ull * n_states; ++i)
        if (table[i] >= n_states) return DNA_ERR_INVALID_ARG;
    try {
        *definite_depth = dnalib::definite_depth(table, n_states, 64, 4096);
    } catch (const std::bad_alloc &) {
        return DNA_ERR_NOMEM;
    }
    return DNA_OK;
}
