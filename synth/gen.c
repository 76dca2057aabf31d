/*
 * gen.c -- seeded synthetic DNA inputs shared by the tests, the bench and the oracle
 * leg. It holds no DFA or scan arithmetic: it only produces bytes.
 *
 * Generators: splitmix64 seeding -> xoshiro256** (Blackman & Vigna, public domain
 * definitions restated here). Sequences:
 *   syn_uniform : i.i.d. uniform over A/C/G/T (uppercase).
 *   syn_markov2 : order-2 Markov chain over A/C/G/T. Each of the 16 contexts (x1,x2)
 *                 draws its weights as base * U[0.5,1.5] with base A=T=0.295,
 *                 C=G=0.205, damps the CpG step (x2 = C, next = G) by 0.25, then a
 *                 common C/G multiplier is bisected so that the stationary GC
 *                 fraction equals gc_target.
 *   syn_overlay_runs : paints runs over an existing sequence: case-folds runs to
 *                 lowercase (soft masking) and/or replaces runs with 'N'. Run and gap
 *                 lengths are geometric with the requested means and coverage.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef struct { uint64_t s[4]; } xo_state;

static uint64_t splitmix64(uint64_t *x)
{
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void xo_seed(xo_state *st, uint64_t seed)
{
    uint64_t x = seed;
    for (int i = 0; i < 4; i++) st->s[i] = splitmix64(&x);
}

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t xo_next(xo_state *st)
{
    uint64_t *s = st->s;
    uint64_t r = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl(s[3], 45);
    return r;
}

static inline double xo_unit(xo_state *st) /* (0, 1] */
{
    return ((xo_next(st) >> 11) + 1) * (1.0 / 9007199254740992.0);
}

static const char BASES[4] = {'A', 'C', 'G', 'T'};

void syn_uniform(uint64_t seed, uint8_t *out, uint64_t n)
{
    xo_state st; xo_seed(&st, seed);
    uint64_t i = 0;
    while (i < n) {
        uint64_t r = xo_next(&st);
        for (int k = 0; k < 32 && i < n; k++, i++) { out[i] = (uint8_t)BASES[r & 3]; r >>= 2; }
    }
}

/* Weights for the 16 contexts before GC calibration. */
static void markov_weights(uint64_t seed, double w[16][4])
{
    static const double base[4] = {0.295, 0.205, 0.205, 0.295};
    xo_state st; xo_seed(&st, seed ^ 0x6D61726B6F76ull);
    for (int c = 0; c < 16; c++)
        for (int b = 0; b < 4; b++) {
            double u = 0.5 + (double)(xo_next(&st) >> 11) * (1.0 / 9007199254740992.0);
            w[c][b] = base[b] * u;
            if ((c & 3) == 1 && b == 2) w[c][b] *= 0.25; /* x2 = C, next = G */
        }
}

static void markov_probs(const double w[16][4], double g, double p[16][4])
{
    for (int c = 0; c < 16; c++) {
        double t = 0;
        for (int b = 0; b < 4; b++) { p[c][b] = w[c][b] * ((b == 1 || b == 2) ? g : 1.0); t += p[c][b]; }
        for (int b = 0; b < 4; b++) p[c][b] /= t;
    }
}

static double stationary_gc(const double p[16][4])
{
    double pi[16], nx[16];
    for (int c = 0; c < 16; c++) pi[c] = 1.0 / 16;
    for (int it = 0; it < 2000; it++) {
        memset(nx, 0, sizeof(nx));
        for (int c = 0; c < 16; c++)
            for (int b = 0; b < 4; b++) nx[((c & 3) << 2) | b] += pi[c] * p[c][b];
        memcpy(pi, nx, sizeof(pi));
    }
    double gc = 0;
    for (int c = 0; c < 16; c++) gc += pi[c] * (p[c][1] + p[c][2]);
    return gc;
}

/* Writes the calibrated 16x4 transition probabilities (context = 4*x1 + x2). */
void syn_markov2_params(uint64_t seed, double gc_target, double *probs_out)
{
    double w[16][4], p[16][4];
    markov_weights(seed, w);
    double lo = 0.05, hi = 20.0;
    for (int it = 0; it < 100; it++) {
        double mid = sqrt(lo * hi);
        markov_probs(w, mid, p);
        if (stationary_gc(p) < gc_target) lo = mid; else hi = mid;
    }
    markov_probs(w, sqrt(lo * hi), p);
    memcpy(probs_out, p, sizeof(p));
}

void syn_markov2(uint64_t seed, double gc_target, uint8_t *out, uint64_t n)
{
    double p[16][4];
    syn_markov2_params(seed, gc_target, &p[0][0]);
    uint64_t thr[16][3];
    for (int c = 0; c < 16; c++) {
        double acc = 0;
        for (int b = 0; b < 3; b++) {
            acc += p[c][b];
            double t = acc * 18446744073709551616.0;
            thr[c][b] = t >= 18446744073709551615.0 ? UINT64_MAX : (uint64_t)t;
        }
    }
    xo_state st; xo_seed(&st, seed);
    int ctx = (int)(xo_next(&st) & 15);
    for (uint64_t i = 0; i < n; i++) {
        uint64_t r = xo_next(&st);
        int b = (r < thr[ctx][0]) ? 0 : (r < thr[ctx][1]) ? 1 : (r < thr[ctx][2]) ? 2 : 3;
        out[i] = (uint8_t)BASES[b];
        ctx = ((ctx & 3) << 2) | b;
    }
}

static uint64_t geometric(xo_state *st, double mean)
{
    if (mean <= 1.0) return 1;
    double p = 1.0 / mean;
    return 1 + (uint64_t)floor(log(xo_unit(st)) / log1p(-p));
}

/*
 * Paints runs over seq[0, n): mode 0 = lowercase (soft-mask) the run, mode 1 =
 * overwrite the run with 'N'. Runs have geometric length with mean run_mean; gaps are
 * geometric with the mean that gives the requested coverage fraction.
 * Returns the number of bytes painted.
 */
uint64_t syn_overlay_runs(uint64_t seed, uint8_t *seq, uint64_t n, double coverage,
                          double run_mean, int mode)
{
    if (coverage <= 0.0) return 0;
    xo_state st; xo_seed(&st, seed ^ (mode ? 0x4E52554Eull : 0x4C4F5745ull));
    double gap_mean = run_mean * (1.0 - coverage) / coverage;
    uint64_t i = geometric(&st, gap_mean), painted = 0;
    while (i < n) {
        uint64_t len = geometric(&st, run_mean);
        uint64_t end = i + len < n ? i + len : n;
        for (uint64_t j = i; j < end; j++) {
            if (mode) seq[j] = 'N';
            else if (seq[j] >= 'A' && seq[j] <= 'Z') seq[j] = (uint8_t)(seq[j] + 32);
        }
        painted += end - i;
        i = end + geometric(&st, gap_mean);
    }
    return painted;
}
