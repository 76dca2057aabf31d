/*
 * oracle.c -- the plain, slow, obviously correct CPU oracle for the DNA DFA scan.
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline / reference leg may load this library. It shares no code, header, table
 * or constant with the CUDA library in paper_1509_01506_gb300/, and the library
 * never loads it.
 *
 * What it computes (Memeti & Pllana, Sec. II and Alg. 1):
 *   A DFA is the quintuple (Q, Sigma, delta, q0, F) of Sec. II with Sigma = {A,C,G,T}.
 *   Each input byte is a symbol: A/a, C/c, G/g, T/t are the four bases; every other
 *   byte (N, IUPAC codes, newline, ...) is the reset symbol, which sends any state to
 *   q0 (state 0). The scan starts in q0, takes one transition per byte and tests the
 *   post-transition state for membership in F (Alg. 1: the state is updated and then
 *   tested against F, for every character). count = number of such steps; the
 *   positions are the 0-based indices of those bytes, ascending.
 *   For a pattern language L (a literal, a k-mer set, a regular expression), the DFA
 *   is the complete DFA of Sigma* . L, so a position j is reported iff some non-empty
 *   substring seq[i..j] with no reset byte in it is a word of L. Overlapping
 *   occurrences are all reported (Sec. II: Aho-Corasick finds overlapping
 *   occurrences; Sec. IV-A: the DFA finds the overlapping ones too).
 *
 * Pattern compilers (all written out step by step, no shared code with the library):
 *   regex  -> syntax tree -> Thompson NFA (with a Sigma* self-loop in front)
 *          -> subset construction over the 4 bases -> Moore minimisation
 *          -> canonical breadth-first state numbering.
 *   k-mers -> Aho-Corasick trie -> breadth-first failure links -> the failure-free
 *             ("modified") AC DFA of Sec. III-B.1 / Fig. 2, where each missing goto is
 *             replaced by the transition the failure chain would take
 *          -> optional Moore minimisation + canonical numbering.
 *
 * Regex syntax (case-insensitive): A C G T literals, '.' (any base), classes [ACGT...],
 * grouping ( ), alternation |, quantifiers * + ? {n} {n,} {n,m}. A pattern whose
 * language contains the empty word is rejected (a match needs at least one byte).
 *
 * Table layout used here: int32 table[q*4 + s] with s = 0..3 for A, C, G, T; accept[q]
 * is 0 or 1 (one byte per state).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_ERR_SYNTAX   -1
#define OR_ERR_CAPACITY -2
#define OR_ERR_EMPTYWORD -3
#define OR_ERR_NOMEM    -4
#define OR_ERR_ARG      -5

/* ---------------------------------------------------------------- symbols */

/* Byte -> symbol: case-insensitive bases; every other byte is the reset symbol (the
 * paper never mentions non-base bytes; N and IUPAC codes are read as breaking a match). */
int or_symbol_of_byte(int byte)
{
    switch (byte) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    default: return 4; /* reset symbol */
    }
}

/* ------------------------------------------------------------- the run itself */

/*
 * The definition (Sec. II; Alg. 1 transition-then-test): one transition per byte from
 * q0, reset bytes go to state 0, a step counts when its post-transition state is in F.
 * Writes at most pos_cap positions; returns the full count (or a negative error).
 */
int64_t or_run(const int32_t *table, const uint8_t *accept, int32_t n_states,
               const uint8_t *seq, int64_t n, int64_t *pos_out, int64_t pos_cap)
{
    if (n_states <= 0 || !table || !accept || (n > 0 && !seq)) return OR_ERR_ARG;
    int32_t q = 0;
    int64_t count = 0;
    for (int64_t j = 0; j < n; j++) {
        int s = or_symbol_of_byte(seq[j]);
        if (s == 4) q = 0;
        else q = table[(int64_t)q * 4 + s];
        if (q < 0 || q >= n_states) return OR_ERR_ARG;
        if (accept[q]) {
            if (pos_out && count < pos_cap) pos_out[count] = j;
            count++;
        }
    }
    return count;
}

/* Same run, also returning the final state (used by tests of the join invariant). */
int64_t or_run_from(const int32_t *table, const uint8_t *accept, int32_t n_states,
                    int32_t q_start, const uint8_t *seq, int64_t n, int32_t *q_end)
{
    if (n_states <= 0 || q_start < 0 || q_start >= n_states) return OR_ERR_ARG;
    int32_t q = q_start;
    int64_t count = 0;
    for (int64_t j = 0; j < n; j++) {
        int s = or_symbol_of_byte(seq[j]);
        q = (s == 4) ? 0 : table[(int64_t)q * 4 + s];
        if (accept[q]) count++;
    }
    if (q_end) *q_end = q;
    return count;
}

/*
 * The run of one piece of a longer sequence (Sec. III-B: a chunk scanned from a given
 * start state): as or_run_from, also writing the first pos_cap positions, counted from
 * the piece's first byte.
 */
int64_t or_run_piece(const int32_t *table, const uint8_t *accept, int32_t n_states,
                     int32_t q_start, const uint8_t *seq, int64_t n, int32_t *q_end,
                     int64_t *pos_out, int64_t pos_cap)
{
    if (n_states <= 0 || !table || !accept || (n > 0 && !seq)) return OR_ERR_ARG;
    if (q_start < 0 || q_start >= n_states) return OR_ERR_ARG;
    int32_t q = q_start;
    int64_t count = 0;
    for (int64_t j = 0; j < n; j++) {
        int s = or_symbol_of_byte(seq[j]);
        q = (s == 4) ? 0 : table[(int64_t)q * 4 + s];
        if (q < 0 || q >= n_states) return OR_ERR_ARG;
        if (accept[q]) {
            if (pos_out && count < pos_cap) pos_out[count] = j;
            count++;
        }
    }
    if (q_end) *q_end = q;
    return count;
}

/* ------------------------------------------------------------ regex parser */

enum { RX_SET = 1, RX_CAT, RX_ALT, RX_REP };

typedef struct {
    int kind;
    int set;      /* RX_SET: bit s set = base s accepted */
    int left, right; /* children (RX_CAT, RX_ALT); left = child of RX_REP */
    int lo, hi;   /* RX_REP bounds; hi < 0 means unbounded */
} rx_node;

typedef struct {
    const char *p;
    rx_node *nodes;
    int n, cap;
    int err;
} rx_parser;

static int rx_new(rx_parser *ps, int kind)
{
    if (ps->n == ps->cap) {
        int nc = ps->cap ? ps->cap * 2 : 64;
        rx_node *nn = (rx_node *)realloc(ps->nodes, sizeof(rx_node) * nc);
        if (!nn) { ps->err = OR_ERR_NOMEM; return -1; }
        ps->nodes = nn; ps->cap = nc;
    }
    rx_node *x = &ps->nodes[ps->n];
    memset(x, 0, sizeof(*x));
    x->kind = kind; x->left = x->right = -1;
    return ps->n++;
}

static int base_bit(char c)
{
    int s = or_symbol_of_byte((unsigned char)c);
    return s < 4 ? (1 << s) : 0;
}

static int rx_alt(rx_parser *ps);

static int rx_number(rx_parser *ps, int *out)
{
    int v = 0, any = 0;
    while (*ps->p >= '0' && *ps->p <= '9') {
        v = v * 10 + (*ps->p - '0');
        if (v > 100000) { ps->err = OR_ERR_SYNTAX; return 0; }
        ps->p++; any = 1;
    }
    *out = v;
    return any;
}

static int rx_atom(rx_parser *ps)
{
    char c = *ps->p;
    if (c == '(') {
        ps->p++;
        int r = rx_alt(ps);
        if (ps->err) return -1;
        if (*ps->p != ')') { ps->err = OR_ERR_SYNTAX; return -1; }
        ps->p++;
        return r;
    }
    if (c == '[') {
        ps->p++;
        int set = 0;
        while (*ps->p && *ps->p != ']') {
            int b = base_bit(*ps->p);
            if (!b) { ps->err = OR_ERR_SYNTAX; return -1; }
            set |= b; ps->p++;
        }
        if (*ps->p != ']' || set == 0) { ps->err = OR_ERR_SYNTAX; return -1; }
        ps->p++;
        int x = rx_new(ps, RX_SET);
        if (x >= 0) ps->nodes[x].set = set;
        return x;
    }
    if (c == '.') {
        ps->p++;
        int x = rx_new(ps, RX_SET);
        if (x >= 0) ps->nodes[x].set = 15;
        return x;
    }
    int b = base_bit(c);
    if (!b) { ps->err = OR_ERR_SYNTAX; return -1; }
    ps->p++;
    int x = rx_new(ps, RX_SET);
    if (x >= 0) ps->nodes[x].set = b;
    return x;
}

static int rx_rep(rx_parser *ps)
{
    int a = rx_atom(ps);
    if (ps->err) return -1;
    for (;;) {
        char c = *ps->p;
        int lo, hi;
        if (c == '*') { lo = 0; hi = -1; ps->p++; }
        else if (c == '+') { lo = 1; hi = -1; ps->p++; }
        else if (c == '?') { lo = 0; hi = 1; ps->p++; }
        else if (c == '{') {
            ps->p++;
            if (!rx_number(ps, &lo)) { ps->err = OR_ERR_SYNTAX; return -1; }
            if (*ps->p == '}') { hi = lo; ps->p++; }
            else if (*ps->p == ',') {
                ps->p++;
                if (*ps->p == '}') { hi = -1; ps->p++; }
                else {
                    if (!rx_number(ps, &hi) || *ps->p != '}' || hi < lo) { ps->err = OR_ERR_SYNTAX; return -1; }
                    ps->p++;
                }
            } else { ps->err = OR_ERR_SYNTAX; return -1; }
            if (ps->err) return -1;
            if (hi == 0) { ps->err = OR_ERR_SYNTAX; return -1; } /* zero-width repeat */
        } else break;
        int r = rx_new(ps, RX_REP);
        if (r < 0) return -1;
        ps->nodes[r].left = a; ps->nodes[r].lo = lo; ps->nodes[r].hi = hi;
        a = r;
    }
    return a;
}

static int rx_cat(rx_parser *ps)
{
    int a = -1;
    while (*ps->p && *ps->p != '|' && *ps->p != ')') {
        int b = rx_rep(ps);
        if (ps->err) return -1;
        if (a < 0) a = b;
        else {
            int c = rx_new(ps, RX_CAT);
            if (c < 0) return -1;
            ps->nodes[c].left = a; ps->nodes[c].right = b;
            a = c;
        }
    }
    if (a < 0) ps->err = OR_ERR_SYNTAX; /* empty branch */
    return a;
}

static int rx_alt(rx_parser *ps)
{
    int a = rx_cat(ps);
    if (ps->err) return -1;
    while (*ps->p == '|') {
        ps->p++;
        int b = rx_cat(ps);
        if (ps->err) return -1;
        int c = rx_new(ps, RX_ALT);
        if (c < 0) return -1;
        ps->nodes[c].left = a; ps->nodes[c].right = b;
        a = c;
    }
    return a;
}

/* ------------------------------------------------------------ Thompson NFA */

typedef struct {
    int set;      /* symbol edge: bases in 'set' lead to 'to' */
    int to;
    int eps1, eps2;
} nfa_state;

typedef struct {
    nfa_state *st;
    int n, cap;
    int err;
} nfa;

static int nfa_new(nfa *a)
{
    if (a->n == a->cap) {
        int nc = a->cap ? a->cap * 2 : 256;
        nfa_state *ns = (nfa_state *)realloc(a->st, sizeof(nfa_state) * nc);
        if (!ns) { a->err = OR_ERR_NOMEM; return -1; }
        a->st = ns; a->cap = nc;
    }
    a->st[a->n].set = 0; a->st[a->n].to = -1;
    a->st[a->n].eps1 = a->st[a->n].eps2 = -1;
    return a->n++;
}

static void nfa_eps(nfa *a, int from, int to)
{
    if (a->st[from].eps1 < 0) a->st[from].eps1 = to;
    else a->st[from].eps2 = to;
}

/* Builds a Thompson fragment for node x; returns start, writes the single exit state. */
static int nfa_build(nfa *a, const rx_node *nodes, int x, int *out)
{
    const rx_node *nd = &nodes[x];
    if (a->err) return -1;
    if (nd->kind == RX_SET) {
        int s = nfa_new(a), f = nfa_new(a);
        if (a->err) return -1;
        a->st[s].set = nd->set; a->st[s].to = f;
        *out = f; return s;
    }
    if (nd->kind == RX_CAT) {
        int o1, o2;
        int s1 = nfa_build(a, nodes, nd->left, &o1);
        int s2 = nfa_build(a, nodes, nd->right, &o2);
        if (a->err) return -1;
        nfa_eps(a, o1, s2);
        *out = o2; return s1;
    }
    if (nd->kind == RX_ALT) {
        int s = nfa_new(a), f = nfa_new(a), o1, o2;
        int s1 = nfa_build(a, nodes, nd->left, &o1);
        int s2 = nfa_build(a, nodes, nd->right, &o2);
        if (a->err) return -1;
        nfa_eps(a, s, s1); nfa_eps(a, s, s2);
        nfa_eps(a, o1, f); nfa_eps(a, o2, f);
        *out = f; return s;
    }
    /* RX_REP: lo mandatory copies, then either a star or (hi-lo) optional copies. */
    int s = nfa_new(a);
    if (a->err) return -1;
    int cur = s;
    for (int i = 0; i < nd->lo; i++) {
        int o, c = nfa_build(a, nodes, nd->left, &o);
        if (a->err) return -1;
        nfa_eps(a, cur, c); cur = o;
    }
    if (nd->hi < 0) {
        int hub = nfa_new(a), f = nfa_new(a), o;
        if (a->err) return -1;
        int c = nfa_build(a, nodes, nd->left, &o);
        if (a->err) return -1;
        nfa_eps(a, cur, hub);
        nfa_eps(a, hub, c); nfa_eps(a, hub, f);
        nfa_eps(a, o, hub);
        cur = f;
    } else {
        for (int i = nd->lo; i < nd->hi; i++) {
            int j = nfa_new(a), o;
            if (a->err) return -1;
            int c = nfa_build(a, nodes, nd->left, &o);
            if (a->err) return -1;
            nfa_eps(a, cur, c); nfa_eps(a, cur, j);
            nfa_eps(a, o, j);
            cur = j;
        }
    }
    *out = cur; return s;
}

/* ------------------------------------------------------- subset construction */

typedef struct {
    int words;
    uint64_t *bits;   /* dfa states' NFA sets, words per state */
    int n, cap;
    int32_t *trans;   /* 4 per state */
    uint8_t *acc;
    int *hash_head, hash_size;
    int *hash_next;
} subset_ctx;

static uint64_t set_hash(const uint64_t *b, int words)
{
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < words; i++) { h ^= b[i]; h *= 1099511628211ull; h ^= h >> 29; }
    return h;
}

static void eps_closure(const nfa *a, uint64_t *set, int *stack)
{
    int sp = 0;
    for (int i = 0; i < a->n; i++)
        if (set[i >> 6] >> (i & 63) & 1) stack[sp++] = i;
    while (sp) {
        int u = stack[--sp];
        int e[2] = {a->st[u].eps1, a->st[u].eps2};
        for (int k = 0; k < 2; k++) {
            int v = e[k];
            if (v >= 0 && !(set[v >> 6] >> (v & 63) & 1)) {
                set[v >> 6] |= 1ull << (v & 63);
                stack[sp++] = v;
            }
        }
    }
}

/* Returns the index of the DFA state with this NFA set, adding it if new. */
static int subset_find_or_add(subset_ctx *c, const uint64_t *set, int final_state, int *added)
{
    uint64_t h = set_hash(set, c->words);
    int bucket = (int)(h % (uint64_t)c->hash_size);
    for (int i = c->hash_head[bucket]; i >= 0; i = c->hash_next[i])
        if (memcmp(c->bits + (size_t)i * c->words, set, sizeof(uint64_t) * c->words) == 0) {
            *added = 0; return i;
        }
    if (c->n == c->cap) {
        int nc = c->cap * 2;
        uint64_t *nb = (uint64_t *)realloc(c->bits, sizeof(uint64_t) * (size_t)nc * c->words);
        int32_t *nt = (int32_t *)realloc(c->trans, sizeof(int32_t) * 4 * (size_t)nc);
        uint8_t *na = (uint8_t *)realloc(c->acc, (size_t)nc);
        int *nn = (int *)realloc(c->hash_next, sizeof(int) * (size_t)nc);
        if (!nb || !nt || !na || !nn) return OR_ERR_NOMEM;
        c->bits = nb; c->trans = nt; c->acc = na; c->hash_next = nn; c->cap = nc;
    }
    int id = c->n++;
    memcpy(c->bits + (size_t)id * c->words, set, sizeof(uint64_t) * c->words);
    c->acc[id] = (uint8_t)((set[final_state >> 6] >> (final_state & 63)) & 1);
    c->hash_next[id] = c->hash_head[bucket];
    c->hash_head[bucket] = id;
    *added = 1;
    return id;
}

/* ------------------------------------------------------ Moore minimisation */

/*
 * Moore's partition refinement: start from {F, Q\F}; repeatedly split classes by the
 * classes of the four successors until the number of classes stops growing. Then
 * number the classes breadth-first from the class of q0, visiting A, C, G, T in order
 * (a canonical numbering: two minimal DFAs of the same language get equal tables).
 */
static int cmp_u32(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* The same refinement for states that carry a key (a pattern label mask): the starting
 * partition puts states with equal keys together, so states that report different
 * patterns are never merged. */
static int moore_minimise_keys(int n, const int32_t *trans, const uint32_t *key,
                               int32_t *out_table, uint32_t *out_key, int cap)
{
    int64_t *cls = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *ncls = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *sig = (int64_t *)malloc(sizeof(int64_t) * 5 * (size_t)n);
    int *order = (int *)malloc(sizeof(int) * (size_t)n);
    uint32_t *keys = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    if (!cls || !ncls || !sig || !order || !keys) {
        free(cls); free(ncls); free(sig); free(order); free(keys); return OR_ERR_NOMEM;
    }
    /* the starting classes are the key values themselves; k = how many distinct ones */
    for (int q = 0; q < n; q++) { cls[q] = key[q]; keys[q] = key[q]; }
    qsort(keys, (size_t)n, sizeof(uint32_t), cmp_u32);
    int k = n > 0 ? 1 : 0;
    for (int i = 1; i < n; i++) if (keys[i] != keys[i - 1]) k++;
    free(keys);
    for (;;) {
        /* signature of q = (class q, class of each successor); classes are then the
         * distinct signatures, numbered by first appearance in a sorted order. */
        for (int q = 0; q < n; q++) {
            sig[5 * q] = cls[q];
            for (int s = 0; s < 4; s++) sig[5 * q + 1 + s] = cls[trans[4 * q + s]];
            order[q] = q;
        }
        /* insertion sort by signature would be O(n^2); use a simple merge sort */
        {
            int *tmp = (int *)malloc(sizeof(int) * (size_t)n);
            if (!tmp) { free(cls); free(ncls); free(sig); free(order); return OR_ERR_NOMEM; }
            for (int width = 1; width < n; width *= 2) {
                for (int lo = 0; lo < n; lo += 2 * width) {
                    int mid = lo + width < n ? lo + width : n;
                    int hi = lo + 2 * width < n ? lo + 2 * width : n;
                    int i = lo, j = mid, t = lo;
                    while (i < mid && j < hi) {
                        int a = order[i], b = order[j], cmp = 0;
                        for (int f = 0; f < 5 && !cmp; f++)
                            cmp = sig[5 * a + f] < sig[5 * b + f] ? -1 : (sig[5 * a + f] > sig[5 * b + f] ? 1 : 0);
                        tmp[t++] = (cmp <= 0) ? order[i++] : order[j++];
                    }
                    while (i < mid) tmp[t++] = order[i++];
                    while (j < hi) tmp[t++] = order[j++];
                }
                memcpy(order, tmp, sizeof(int) * (size_t)n);
            }
            free(tmp);
        }
        int nk = 0;
        for (int i = 0; i < n; i++) {
            int q = order[i];
            if (i > 0) {
                int p = order[i - 1], same = 1;
                for (int f = 0; f < 5; f++) if (sig[5 * p + f] != sig[5 * q + f]) { same = 0; break; }
                if (!same) nk++;
            }
            ncls[q] = nk;
        }
        nk++;
        memcpy(cls, ncls, sizeof(int64_t) * (size_t)n);
        if (nk == k) break;
        k = nk;
    }
    if (k > cap) { free(cls); free(ncls); free(sig); free(order); return OR_ERR_CAPACITY; }
    /* canonical breadth-first numbering from the class of q0 */
    /* after the loop the classes are numbered 0..k-1 */
    int *rep = (int *)malloc(sizeof(int) * (size_t)k);   /* a member state of each class */
    int *newid = (int *)malloc(sizeof(int) * (size_t)k);
    int *queue = (int *)malloc(sizeof(int) * (size_t)k);
    for (int c = 0; c < k; c++) { rep[c] = -1; newid[c] = -1; }
    for (int q = 0; q < n; q++) if (rep[cls[q]] < 0) rep[cls[q]] = q;
    int head = 0, tail = 0;
    newid[cls[0]] = 0; queue[tail++] = cls[0];
    while (head < tail) {
        int c = queue[head++];
        for (int s = 0; s < 4; s++) {
            int d = cls[trans[4 * rep[c] + s]];
            if (newid[d] < 0) { newid[d] = tail; queue[tail++] = d; }
        }
    }
    int reach = tail;
    for (int i = 0; i < reach; i++) {
        int c = queue[i];
        out_key[i] = key[rep[c]];
        for (int s = 0; s < 4; s++) out_table[4 * i + s] = newid[cls[trans[4 * rep[c] + s]]];
    }
    free(rep); free(newid); free(queue);
    free(cls); free(ncls); free(sig); free(order);
    return reach;
}

/* Moore minimisation with accept flags (0/1): the keyed refinement on {F, Q \ F}. */
static int moore_minimise(int n, const int32_t *trans, const uint8_t *acc,
                          int32_t *out_table, uint8_t *out_acc, int cap)
{
    uint32_t *key = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    uint32_t *okey = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    if (!key || !okey) { free(key); free(okey); return OR_ERR_NOMEM; }
    for (int q = 0; q < n; q++) key[q] = acc[q] ? 1u : 0u;
    int r = moore_minimise_keys(n, trans, key, out_table, okey, cap);
    for (int i = 0; i < r; i++) out_acc[i] = (uint8_t)okey[i];
    free(key); free(okey);
    return r;
}

/* ------------------------------------------------------ regex -> DFA (public) */

/*
 * Compiles a regex to the DFA of Sigma*.L. minimise = 0 returns the raw subset
 * construction (states numbered in discovery order, q0 = 0); minimise = 1 returns the
 * Moore-minimal DFA with canonical numbering. Returns the number of states or < 0.
 */
int32_t or_compile_regex(const char *pattern, int minimise, int32_t *table_out,
                         uint8_t *accept_out, int32_t cap_states)
{
    if (!pattern || !table_out || !accept_out || cap_states <= 0) return OR_ERR_ARG;
    rx_parser ps; memset(&ps, 0, sizeof(ps));
    ps.p = pattern;
    int root = rx_alt(&ps);
    if (!ps.err && *ps.p != '\0') ps.err = OR_ERR_SYNTAX;
    if (ps.err) { free(ps.nodes); return ps.err; }

    nfa a; memset(&a, 0, sizeof(a));
    int loop = nfa_new(&a);          /* Sigma* self-loop in front of the pattern */
    int pout, pstart = nfa_build(&a, ps.nodes, root, &pout);
    free(ps.nodes);
    if (a.err) { free(a.st); return a.err; }
    a.st[loop].set = 15; a.st[loop].to = loop;
    nfa_eps(&a, loop, pstart);
    int final_state = pout;

    int words = (a.n + 63) / 64;
    int *stack = (int *)malloc(sizeof(int) * (size_t)a.n * 2);
    uint64_t *tmp = (uint64_t *)calloc((size_t)words, sizeof(uint64_t));
    subset_ctx c; memset(&c, 0, sizeof(c));
    c.words = words; c.cap = 256; c.hash_size = 1 << 16;
    c.bits = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)c.cap * words);
    c.trans = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)c.cap);
    c.acc = (uint8_t *)malloc((size_t)c.cap);
    c.hash_next = (int *)malloc(sizeof(int) * (size_t)c.cap);
    c.hash_head = (int *)malloc(sizeof(int) * (size_t)c.hash_size);
    int rc = 0;
    if (!stack || !tmp || !c.bits || !c.trans || !c.acc || !c.hash_next || !c.hash_head) rc = OR_ERR_NOMEM;
    if (!rc) {
        for (int i = 0; i < c.hash_size; i++) c.hash_head[i] = -1;
        tmp[loop >> 6] |= 1ull << (loop & 63);
        eps_closure(&a, tmp, stack);
        if ((tmp[final_state >> 6] >> (final_state & 63)) & 1) rc = OR_ERR_EMPTYWORD;
    }
    if (!rc) {
        int added;
        subset_find_or_add(&c, tmp, final_state, &added);
        for (int d = 0; d < c.n && !rc; d++) {
            for (int s = 0; s < 4 && !rc; s++) {
                memset(tmp, 0, sizeof(uint64_t) * words);
                const uint64_t *cur = c.bits + (size_t)d * words;
                for (int u = 0; u < a.n; u++)
                    if ((cur[u >> 6] >> (u & 63) & 1) && (a.st[u].set >> s & 1)) {
                        int v = a.st[u].to;
                        tmp[v >> 6] |= 1ull << (v & 63);
                    }
                eps_closure(&a, tmp, stack);
                int id = subset_find_or_add(&c, tmp, final_state, &added);
                if (id < 0) { rc = id; break; }
                c.trans[4 * d + s] = id;
                if (c.n > (1 << 22)) rc = OR_ERR_CAPACITY;
            }
        }
    }
    int32_t result = rc;
    if (!rc) {
        if (minimise) {
            result = moore_minimise(c.n, c.trans, c.acc, table_out, accept_out, cap_states);
        } else if (c.n > cap_states) {
            result = OR_ERR_CAPACITY;
        } else {
            memcpy(table_out, c.trans, sizeof(int32_t) * 4 * (size_t)c.n);
            memcpy(accept_out, c.acc, (size_t)c.n);
            result = c.n;
        }
    }
    free(stack); free(tmp); free(a.st);
    free(c.bits); free(c.trans); free(c.acc); free(c.hash_next); free(c.hash_head);
    return result;
}

/* -------------------------------------- several patterns with labels (public) */

/*
 * One automaton for several regexes, as the paper scans the nine regex-dna expressions
 * of Table V with one DFA and keeps a counter per accepting state (Alg. 1, the switch
 * into final_states[]): the NFA has one Sigma* loop in front of every pattern, each
 * pattern keeps its own exit state, and a DFA state's label mask has bit i set when
 * pattern i's exit state is in its NFA set. 'patterns' holds up to 32 regexes separated
 * by newlines. minimise = 1 applies the keyed Moore refinement from the partition by
 * label mask. Returns the number of states or < 0.
 */
int32_t or_compile_regex_set(const char *patterns, int minimise, int32_t *table_out,
                             uint32_t *labels_out, int32_t cap_states)
{
    if (!patterns || !table_out || !labels_out || cap_states <= 0) return OR_ERR_ARG;
    nfa a; memset(&a, 0, sizeof(a));
    int loop = nfa_new(&a);
    int hook = loop;   /* every pattern start hangs off a chain of fork states (two eps each) */
    int exits[32], n_pat = 0, rc = 0;
    const char *p = patterns;
    char *buf = (char *)malloc(strlen(patterns) + 1);
    if (!buf) { free(a.st); return OR_ERR_NOMEM; }
    while (!rc) {
        const char *e = strchr(p, '\n');
        size_t len = e ? (size_t)(e - p) : strlen(p);
        if (n_pat == 32) { rc = OR_ERR_ARG; break; }
        memcpy(buf, p, len); buf[len] = '\0';
        rx_parser ps; memset(&ps, 0, sizeof(ps));
        ps.p = buf;
        int root = rx_alt(&ps);
        if (!ps.err && *ps.p != '\0') ps.err = OR_ERR_SYNTAX;
        if (ps.err) { rc = ps.err; free(ps.nodes); break; }
        int pout, pstart = nfa_build(&a, ps.nodes, root, &pout);
        free(ps.nodes);
        int fork = nfa_new(&a);
        if (a.err) { rc = a.err; break; }
        nfa_eps(&a, hook, fork);
        nfa_eps(&a, fork, pstart);
        hook = fork;
        exits[n_pat++] = pout;
        if (!e) break;
        p = e + 1;
    }
    free(buf);
    if (rc) { free(a.st); return rc; }
    a.st[loop].set = 15; a.st[loop].to = loop;   /* the Sigma* self-loop */

    int words = (a.n + 63) / 64;
    int *stack = (int *)malloc(sizeof(int) * (size_t)a.n * 2);
    uint64_t *tmp = (uint64_t *)calloc((size_t)words, sizeof(uint64_t));
    subset_ctx c; memset(&c, 0, sizeof(c));
    c.words = words; c.cap = 256; c.hash_size = 1 << 16;
    c.bits = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)c.cap * words);
    c.trans = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)c.cap);
    c.acc = (uint8_t *)malloc((size_t)c.cap);
    c.hash_next = (int *)malloc(sizeof(int) * (size_t)c.cap);
    c.hash_head = (int *)malloc(sizeof(int) * (size_t)c.hash_size);
    if (!stack || !tmp || !c.bits || !c.trans || !c.acc || !c.hash_next || !c.hash_head) rc = OR_ERR_NOMEM;
    if (!rc) {
        for (int i = 0; i < c.hash_size; i++) c.hash_head[i] = -1;
        tmp[loop >> 6] |= 1ull << (loop & 63);
        eps_closure(&a, tmp, stack);
        for (int i = 0; i < n_pat; i++)
            if ((tmp[exits[i] >> 6] >> (exits[i] & 63)) & 1) rc = OR_ERR_EMPTYWORD;
    }
    if (!rc) {
        int added;
        subset_find_or_add(&c, tmp, exits[0], &added);
        for (int d = 0; d < c.n && !rc; d++) {
            for (int s = 0; s < 4 && !rc; s++) {
                memset(tmp, 0, sizeof(uint64_t) * words);
                const uint64_t *cur = c.bits + (size_t)d * words;
                for (int u = 0; u < a.n; u++)
                    if ((cur[u >> 6] >> (u & 63) & 1) && (a.st[u].set >> s & 1)) {
                        int v = a.st[u].to;
                        tmp[v >> 6] |= 1ull << (v & 63);
                    }
                eps_closure(&a, tmp, stack);
                int id = subset_find_or_add(&c, tmp, exits[0], &added);
                if (id < 0) { rc = id; break; }
                c.trans[4 * d + s] = id;
                if (c.n > (1 << 22)) rc = OR_ERR_CAPACITY;
            }
        }
    }
    int32_t result = rc;
    uint32_t *lab = NULL;
    if (!rc) {
        /* label mask of every DFA state: which patterns' exit states its set holds */
        lab = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)c.n);
        if (!lab) result = OR_ERR_NOMEM;
        else {
            for (int d = 0; d < c.n; d++) {
                const uint64_t *set = c.bits + (size_t)d * words;
                uint32_t m = 0;
                for (int i = 0; i < n_pat; i++)
                    if ((set[exits[i] >> 6] >> (exits[i] & 63)) & 1) m |= 1u << i;
                lab[d] = m;
            }
            if (minimise) {
                result = moore_minimise_keys(c.n, c.trans, lab, table_out, labels_out, cap_states);
            } else if (c.n > cap_states) {
                result = OR_ERR_CAPACITY;
            } else {
                memcpy(table_out, c.trans, sizeof(int32_t) * 4 * (size_t)c.n);
                memcpy(labels_out, lab, sizeof(uint32_t) * (size_t)c.n);
                result = c.n;
            }
        }
    }
    free(lab);
    free(stack); free(tmp); free(a.st);
    free(c.bits); free(c.trans); free(c.acc); free(c.hash_next); free(c.hash_head);
    return result;
}

/*
 * The plain run with labels (Alg. 1's count per accepting state, reported per pattern):
 * one transition per byte from q0, reset bytes to state 0; a step whose post-transition
 * state has a non-zero mask counts once in the total and once for every pattern in the
 * mask. Writes at most pos_cap positions and masks; returns the total count.
 */
int64_t or_run_labels(const int32_t *table, const uint32_t *labels, int32_t n_states,
                      const uint8_t *seq, int64_t n, int64_t *label_counts, int32_t n_labels,
                      int64_t *pos_out, uint32_t *pos_lab_out, int64_t pos_cap)
{
    if (n_states <= 0 || !table || !labels || !label_counts || n_labels <= 0 || n_labels > 32 ||
        (n > 0 && !seq)) return OR_ERR_ARG;
    for (int i = 0; i < n_labels; i++) label_counts[i] = 0;
    int32_t q = 0;
    int64_t count = 0;
    for (int64_t j = 0; j < n; j++) {
        int s = or_symbol_of_byte(seq[j]);
        if (s == 4) q = 0;
        else q = table[(int64_t)q * 4 + s];
        if (q < 0 || q >= n_states) return OR_ERR_ARG;
        uint32_t m = labels[q];
        if (m) {
            if (pos_out && count < pos_cap) {
                pos_out[count] = j;
                if (pos_lab_out) pos_lab_out[count] = m;
            }
            count++;
            for (int i = 0; i < n_labels; i++)
                if ((m >> i) & 1u) label_counts[i]++;
        }
    }
    return count;
}

/* ------------------------------------------------- Aho-Corasick (public) */

/*
 * Builds the failure-free Aho-Corasick DFA (Sec. II; Sec. III-B.1, Fig. 2) for a set of
 * base strings given as one string separated by ',' or whitespace. Trie states are
 * numbered in insertion order (root = 0); goto(q, s) for a missing child is
 * goto(fail(q), s), and the root's missing children loop to the root. A state
 * accepts iff some pattern is a suffix of its string. minimise = 1 applies Moore
 * minimisation and canonical numbering. Returns the number of states or < 0.
 */
int32_t or_compile_kmers(const char *patterns, int minimise, int32_t *table_out,
                         uint8_t *accept_out, int32_t cap_states)
{
    if (!patterns || !table_out || !accept_out || cap_states <= 0) return OR_ERR_ARG;
    size_t len = strlen(patterns);
    int cap = (int)len + 2;
    int32_t *child = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)cap);
    int32_t *fail = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    uint8_t *out = (uint8_t *)calloc((size_t)cap, 1);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    int32_t *delta = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)cap);
    if (!child || !fail || !out || !queue || !delta) {
        free(child); free(fail); free(out); free(queue); free(delta); return OR_ERR_NOMEM;
    }
    for (int i = 0; i < 4 * cap; i++) child[i] = -1;
    int n = 1, cur = 0, npat = 0, plen = 0, rc = 0;
    for (size_t i = 0; i <= len; i++) {
        char ch = patterns[i];
        if (ch == '\0' || ch == ',' || ch == ' ' || ch == '\n' || ch == '\t' || ch == '\r') {
            if (plen > 0) { out[cur] = 1; npat++; }
            cur = 0; plen = 0;
            continue;
        }
        int s = or_symbol_of_byte((unsigned char)ch);
        if (s == 4) { rc = OR_ERR_SYNTAX; break; }
        if (child[4 * cur + s] < 0) child[4 * cur + s] = n++;
        cur = child[4 * cur + s];
        plen++;
    }
    if (!rc && npat == 0) rc = OR_ERR_SYNTAX;
    int32_t result = rc;
    if (!rc) {
        /* breadth-first failure links; goto completed along the way */
        int head = 0, tail = 0;
        fail[0] = 0;
        for (int s = 0; s < 4; s++) {
            int c = child[s];
            if (c >= 0) { fail[c] = 0; delta[s] = c; queue[tail++] = c; }
            else delta[s] = 0;
        }
        while (head < tail) {
            int q = queue[head++];
            if (out[fail[q]]) out[q] = 1;   /* a pattern ends at a suffix of q's string */
            for (int s = 0; s < 4; s++) {
                int c = child[4 * q + s];
                if (c >= 0) {
                    fail[c] = delta[4 * fail[q] + s];
                    delta[4 * q + s] = c;
                    queue[tail++] = c;
                } else {
                    delta[4 * q + s] = delta[4 * fail[q] + s];
                }
            }
        }
        if (minimise) {
            result = moore_minimise(n, delta, out, table_out, accept_out, cap_states);
        } else if (n > cap_states) {
            result = OR_ERR_CAPACITY;
        } else {
            memcpy(table_out, delta, sizeof(int32_t) * 4 * (size_t)n);
            memcpy(accept_out, out, (size_t)n);
            result = n;
        }
    }
    free(child); free(fail); free(out); free(queue); free(delta);
    return result;
}

/* Moore minimisation of an arbitrary complete table (canonical numbering). */
int32_t or_minimise_table(const int32_t *table, const uint8_t *accept, int32_t n_states,
                          int32_t *table_out, uint8_t *accept_out, int32_t cap_states)
{
    if (!table || !accept || n_states <= 0) return OR_ERR_ARG;
    for (int64_t i = 0; i < 4 * (int64_t)n_states; i++)
        if (table[i] < 0 || table[i] >= n_states) return OR_ERR_ARG;
    return moore_minimise(n_states, table, accept, table_out, accept_out, cap_states);
}
