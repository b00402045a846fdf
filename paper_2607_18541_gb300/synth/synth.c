/*
 * Seeded synthetic input generators.
 *
 * This module produces the raw inputs that both the CPU oracle and the GPU
 * library consume: byte streams to be compressed (order-2 Markov bytes,
 * FASTQ-like text, order-3 Markov word text), token streams generated
 * directly (the synthetic copy sweep of the paper's Table II experiment),
 * stream-size draws for the batched workload and request traces for the
 * serving loop.  It holds none of the codec's arithmetic: no parsing, no
 * prefix sums of token lengths, no wave scheduling, no hashing of output.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through
 * splitmix64 (Steele, Lea & Flood, 2014), both written from their published
 * definitions.  Floating point is used only through +, -, *, /, sqrt and the
 * series-based s_ln / s_exp below, and the file is compiled with
 * -ffp-contract=off, so every generator returns the same bytes on x86-64 and
 * on AArch64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define SYNTH_OK 0
#define SYNTH_E_INVAL (-1)
#define SYNTH_E_CAPACITY (-2)
#define SYNTH_E_NOMEM (-3)

/* ------------------------------------------------------------------ rng */

typedef struct { uint64_t s[4]; } synth_rng;

static uint64_t splitmix64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static inline uint64_t rotl64(uint64_t v, int k) { return (v << k) | (v >> (64 - k)); }

static void rng_seed(synth_rng *r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64_next(&x);
    if ((r->s[0] | r->s[1] | r->s[2] | r->s[3]) == 0) r->s[0] = 1;
}

static inline uint64_t rng_next(synth_rng *r) {
    uint64_t *s = r->s;
    uint64_t result = rotl64(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

/* uniform integer in [0, n) by the high half of a 64x64 product */
static inline uint64_t rng_below(synth_rng *r, uint64_t n) {
    unsigned __int128 m = (unsigned __int128)rng_next(r) * (unsigned __int128)n;
    return (uint64_t)(m >> 64);
}

/* uniform double in [0, 1) with 53 random bits */
static inline double rng_unit(synth_rng *r) {
    return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0);
}

/* uniform double in (0, 1) */
static inline double rng_unit_open(synth_rng *r) {
    return ((double)(rng_next(r) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------- platform-independent ln/exp */

static const double S_LN2 = 0.6931471805599453;
static const double s_inv[64] = {0.0, 1.0 / 1.0, 1.0 / 2.0, 1.0 / 3.0, 1.0 / 4.0, 1.0 / 5.0, 1.0 / 6.0, 1.0 / 7.0, 1.0 / 8.0, 1.0 / 9.0, 1.0 / 10.0, 1.0 / 11.0, 1.0 / 12.0, 1.0 / 13.0, 1.0 / 14.0, 1.0 / 15.0, 1.0 / 16.0, 1.0 / 17.0, 1.0 / 18.0, 1.0 / 19.0, 1.0 / 20.0, 1.0 / 21.0, 1.0 / 22.0, 1.0 / 23.0, 1.0 / 24.0, 1.0 / 25.0, 1.0 / 26.0, 1.0 / 27.0, 1.0 / 28.0, 1.0 / 29.0, 1.0 / 30.0, 1.0 / 31.0, 1.0 / 32.0, 1.0 / 33.0, 1.0 / 34.0, 1.0 / 35.0, 1.0 / 36.0, 1.0 / 37.0, 1.0 / 38.0, 1.0 / 39.0, 1.0 / 40.0, 1.0 / 41.0, 1.0 / 42.0, 1.0 / 43.0, 1.0 / 44.0, 1.0 / 45.0, 1.0 / 46.0, 1.0 / 47.0, 1.0 / 48.0, 1.0 / 49.0, 1.0 / 50.0, 1.0 / 51.0, 1.0 / 52.0, 1.0 / 53.0, 1.0 / 54.0, 1.0 / 55.0, 1.0 / 56.0, 1.0 / 57.0, 1.0 / 58.0, 1.0 / 59.0, 1.0 / 60.0, 1.0 / 61.0, 1.0 / 62.0, 1.0 / 63.0};

/* natural log of a positive normal double: x = m 2^e, m in [1/sqrt2, sqrt2),
 * ln m = 2 atanh((m-1)/(m+1)) summed as an odd power series. */
static double s_ln(double x) {
    uint64_t b;
    memcpy(&b, &x, 8);
    int e = (int)((b >> 52) & 0x7ff) - 1023;
    b = (b & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL;
    double m;
    memcpy(&m, &b, 8);
    if (m > 1.4142135623730951) { m *= 0.5; e += 1; }
    double t = (m - 1.0) / (m + 1.0), t2 = t * t, p = t, s = 0.0;
    for (int k = 1; k < 44; k += 2) { s += p * s_inv[k]; p *= t2; }
    return 2.0 * s + (double)e * S_LN2;
}

/* e^x: x = k ln2 + r, Taylor series for e^r, scaled exactly by 2^k. */
static double s_exp(double x) {
    if (x < -700.0) return 0.0;
    double kf = floor(x / S_LN2 + 0.5);
    double r = x - kf * S_LN2;
    double s = 1.0, term = 1.0;
    for (int i = 1; i < 28; i++) { term *= r * s_inv[i]; s += term; }
    return ldexp(s, (int)kf);
}

static double s_pow(double a, double b) { return s_exp(b * s_ln(a)); }

/* ----------------------------------------------------- distributions */

/* geometric on {1,2,...} with success probability 1/mean (mean `mean`) */
static uint64_t geom1(synth_rng *r, uint64_t mean) {
    uint64_t k = 1;
    while (rng_below(r, mean) != 0) k++;
    return k;
}

/* geometric on {0,1,...} with mean `mean` (success probability 1/(mean+1)) */
static uint64_t geom0(synth_rng *r, uint64_t mean) {
    uint64_t k = 0;
    while (rng_below(r, mean + 1) != 0) k++;
    return k;
}

/* standard normal by the Marsaglia polar method */
static double normal01(synth_rng *r) {
    for (;;) {
        double u = 2.0 * rng_unit(r) - 1.0, v = 2.0 * rng_unit(r) - 1.0;
        double s = u * u + v * v;
        if (s >= 1.0 || s == 0.0) continue;
        return u * sqrt(-2.0 * s_ln(s) / s);
    }
}

/* Gamma(alpha, 1) by Marsaglia & Tsang (2000), with the U^(1/alpha) boost
 * for alpha < 1. */
static double gamma_draw(synth_rng *r, double alpha) {
    double a = alpha < 1.0 ? alpha + 1.0 : alpha;
    double d = a - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d), g;
    for (;;) {
        double x = normal01(r), v = 1.0 + c * x;
        if (v <= 0.0) continue;
        v = v * v * v;
        double u = rng_unit_open(r);
        if (s_ln(u) < 0.5 * x * x + d - d * v + d * s_ln(v)) { g = d * v; break; }
    }
    if (alpha < 1.0) g *= s_pow(rng_unit_open(r), 1.0 / alpha);
    return g;
}

/* cumulative 32-bit thresholds from non-negative weights: symbol i is drawn
 * when cum[i-1] <= u < cum[i] for u uniform in [0, 2^32). */
static void weights_to_cum32(const double *w, int n, uint64_t *cum) {
    double tot = 0.0;
    for (int i = 0; i < n; i++) tot += w[i];
    double acc = 0.0;
    uint64_t prev = 0;
    for (int i = 0; i < n; i++) {
        acc += w[i];
        uint64_t c = (i == n - 1) ? (1ULL << 32) : (uint64_t)(acc / tot * 4294967296.0);
        if (c < prev) c = prev;
        if (c > (1ULL << 32)) c = 1ULL << 32;
        cum[i] = c;
        prev = c;
    }
}

static int draw_cum32(synth_rng *r, const uint64_t *cum, int n) {
    uint64_t u = rng_next(r) >> 32;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (cum[mid] > u) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* ============================================= order-2 Markov byte stream */

/* Model: 64 symbols 0x30..0x6F; each of the 64*64 contexts draws its
 * next-symbol distribution from Dirichlet(alpha), stored as an alias table
 * (Vose's method): draw column i uniformly, keep it with probability
 * prob[i] / 2^32, else take alias[i]. */
typedef struct {
    uint32_t prob[4096][64];
    uint8_t alias[4096][64];
} markov_model;

static void alias_build(const double *w, int n, uint32_t *prob, uint8_t *alias) {
    double tot = 0.0, q[64];
    int small[64], large[64], ns = 0, nl = 0;
    for (int i = 0; i < n; i++) tot += w[i];
    for (int i = 0; i < n; i++) {
        q[i] = w[i] / tot * (double)n;
        if (q[i] < 1.0) small[ns++] = i; else large[nl++] = i;
    }
    while (ns && nl) {
        int s1 = small[--ns], l1 = large[nl - 1];
        prob[s1] = (uint32_t)(q[s1] * 4294967296.0 > 4294967295.0 ? 4294967295.0 : q[s1] * 4294967296.0);
        alias[s1] = (uint8_t)l1;
        q[l1] = (q[l1] + q[s1]) - 1.0;
        if (q[l1] < 1.0) { nl--; small[ns++] = l1; }
    }
    while (nl) { int l1 = large[--nl]; prob[l1] = 0xffffffffu; alias[l1] = (uint8_t)l1; }
    while (ns) { int s1 = small[--ns]; prob[s1] = 0xffffffffu; alias[s1] = (uint8_t)s1; }
}

void *synth_markov_model_new(uint64_t model_seed, double alpha) {
    if (!(alpha > 0.0)) return NULL;
    markov_model *m = (markov_model *)malloc(sizeof(markov_model));
    if (!m) return NULL;
    synth_rng r;
    rng_seed(&r, model_seed);
    double w[64];
    for (int c = 0; c < 4096; c++) {
        for (int i = 0; i < 64; i++) w[i] = gamma_draw(&r, alpha);
        alias_build(w, 64, m->prob[c], m->alias[c]);
    }
    return m;
}

void synth_markov_model_free(void *m) { free(m); }

/* A sequence from the model: at each position a verbatim repeat starts with
 * probability 1/repeat_every, of geometric length (mean repeat_mean, on
 * 1,2,...) copied from a source uniform in [0, pos - len] (skipped when
 * pos < len); the Markov context resumes from the last two bytes. */
int synth_markov2_gen(const void *model, uint8_t *out, uint64_t n, uint64_t seed,
                      uint32_t repeat_every, uint32_t repeat_mean) {
    if (!model || (!out && n) || repeat_every == 0 || repeat_mean == 0) return SYNTH_E_INVAL;
    const markov_model *m = (const markov_model *)model;
    synth_rng r;
    rng_seed(&r, seed ^ 0x3a4b5c6d7e8f9012ULL);
    int s1 = (int)rng_below(&r, 64), s2 = (int)rng_below(&r, 64);
    uint64_t pos = 0;
    while (pos < n) {
        if (rng_below(&r, repeat_every) == 0) {
            uint64_t len = geom1(&r, repeat_mean);
            if (pos >= len) {
                uint64_t src = rng_below(&r, pos - len + 1);
                uint64_t take = len;
                if (take > n - pos) take = n - pos;
                memmove(out + pos, out + src, take);
                pos += take;
                if (pos >= 2) { s1 = out[pos - 2] - 0x30; s2 = out[pos - 1] - 0x30; }
                continue;
            }
        }
        const int c = s1 * 64 + s2;
        const uint64_t x = rng_next(&r);
        const int col = (int)(x >> 58);
        const int s = ((uint32_t)x < m->prob[c][col]) ? col : m->alias[c][col];
        out[pos++] = (uint8_t)(0x30 + s);
        s1 = s2;
        s2 = s;
    }
    return SYNTH_OK;
}

int synth_markov2(uint8_t *out, uint64_t n, uint64_t seed, uint32_t repeat_every,
                  uint32_t repeat_mean, double alpha) {
    void *m = synth_markov_model_new(seed, alpha);
    if (!m) return SYNTH_E_NOMEM;
    int rc = synth_markov2_gen(m, out, n, seed, repeat_every, repeat_mean);
    synth_markov_model_free(m);
    return rc;
}

/* ============================================================ FASTQ-like */

#define FQ_READ 150
#define FQ_GENOME 4600000ULL
#ifndef FQ_QTOP
#define FQ_QTOP 37      /* quality level the chain starts near */
#define FQ_QDRIFT 8     /* downward drift of the level over one read */
#define FQ_QSPREAD 2    /* half-width of the reversion window */
#define FQ_T_STAY 700   /* per-mille thresholds of the transition kinds */
#define FQ_T_DN1 790
#define FQ_T_UP1 850
#define FQ_T_REV 992
#endif

static int fq_next_q(synth_rng *r, int prev, int i) {
    int mu = FQ_QTOP - (i * FQ_QDRIFT) / FQ_READ;
    uint64_t u = rng_below(r, 1000);
    int q;
    if (u < FQ_T_STAY) q = prev;
    else if (u < FQ_T_DN1) q = prev - 1;
    else if (u < FQ_T_UP1) q = prev + 1;
    else if (u < FQ_T_REV) q = mu + (int)rng_below(r, 2 * FQ_QSPREAD + 1) - FQ_QSPREAD;
    else q = 2 + (int)rng_below(r, 38);
    if (q < 2) q = 2;
    if (q > 39) q = 39;
    return q;
}

/* Records "@SIM.<id>\n<150 bases>\n+\n<150 Phred+33 qualities>\n" with ids
 * from 1; reads start uniformly on a seeded 4.6 Mbase uniform ACGT
 * reference (forward strand); each base is substituted with probability 1%
 * and then replaced by 'N' (quality '#') with probability 0.1%; qualities
 * follow a per-position order-1 Markov chain on Q in [2, 39] that drifts
 * downwards along the read.  Exactly n bytes (the last record truncated). */
int synth_fastq(uint8_t *out, uint64_t n, uint64_t seed) {
    if (!out && n) return SYNTH_E_INVAL;
    static const char ACGT[4] = {'A', 'C', 'G', 'T'};
    uint8_t *genome = (uint8_t *)malloc(FQ_GENOME);
    if (!genome) return SYNTH_E_NOMEM;
    synth_rng r;
    rng_seed(&r, seed ^ 0x5eedfa57a0000001ULL);
    for (uint64_t i = 0; i < FQ_GENOME; i++) genome[i] = (uint8_t)ACGT[rng_below(&r, 4)];
    rng_seed(&r, seed);
    char rec[512];
    uint64_t pos = 0, id = 1;
    while (pos < n) {
        int k = 0;
        rec[k++] = '@'; rec[k++] = 'S'; rec[k++] = 'I'; rec[k++] = 'M'; rec[k++] = '.';
        char dig[24];
        int nd = 0;
        uint64_t v = id;
        do { dig[nd++] = (char)('0' + v % 10); v /= 10; } while (v);
        while (nd) rec[k++] = dig[--nd];
        rec[k++] = '\n';
        uint64_t start = rng_below(&r, FQ_GENOME - FQ_READ + 1);
        int isn[FQ_READ];
        for (int j = 0; j < FQ_READ; j++) {
            int b = genome[start + j];
            if (rng_below(&r, 100) == 0) {
                int idx = (b == 'A') ? 0 : (b == 'C') ? 1 : (b == 'G') ? 2 : 3;
                int o = (int)rng_below(&r, 3);
                b = ACGT[(idx + 1 + o) & 3];
            }
            isn[j] = 0;
            if (rng_below(&r, 1000) == 0) { b = 'N'; isn[j] = 1; }
            rec[k++] = (char)b;
        }
        rec[k++] = '\n'; rec[k++] = '+'; rec[k++] = '\n';
        int q = FQ_QTOP - 4 + (int)rng_below(&r, 6);
        for (int j = 0; j < FQ_READ; j++) {
            q = (j == 0) ? q : fq_next_q(&r, q, j);
            rec[k++] = (char)(33 + (isn[j] ? 2 : q));
        }
        rec[k++] = '\n';
        uint64_t take = (uint64_t)k;
        if (take > n - pos) take = n - pos;
        memcpy(out + pos, rec, take);
        pos += take;
        id++;
    }
    free(genome);
    return SYNTH_OK;
}

/* ================================================= order-3 Markov words */

typedef struct {
    uint32_t n_words;
    char *chars;        /* concatenated words */
    uint32_t *off;      /* n_words + 1 offsets */
    uint64_t *zcum;     /* Zipf CDF over ranks, 2^32 scale */
    uint64_t zcum16[16];
} synth_vocab;

static uint64_t mix64(uint64_t a, uint64_t b) {
    uint64_t x = a ^ (b + 0x9e3779b97f4a7c15ULL + (a << 6) + (a >> 2));
    return splitmix64_next(&x);
}

static int draw_zipf(synth_rng *r, const uint64_t *cum, uint32_t n) {
    return draw_cum32(r, cum, (int)n);
}

static void vocab_free(synth_vocab *v) {
    free(v->chars); free(v->off); free(v->zcum);
    memset(v, 0, sizeof(*v));
}

/* 50k distinct lowercase words, length 1 + Poisson(4); Zipf(s) over ranks. */
static int vocab_build(synth_vocab *v, uint64_t seed, uint32_t n_words, double s) {
    memset(v, 0, sizeof(*v));
    v->n_words = n_words;
    v->chars = (char *)malloc((size_t)n_words * 40);
    v->off = (uint32_t *)malloc(sizeof(uint32_t) * (n_words + 1));
    v->zcum = (uint64_t *)malloc(sizeof(uint64_t) * n_words);
    uint32_t hcap = 1;
    while (hcap < 4 * n_words) hcap <<= 1;
    uint32_t *htab = (uint32_t *)malloc(sizeof(uint32_t) * hcap);
    if (!v->chars || !v->off || !v->zcum || !htab) { free(htab); vocab_free(v); return SYNTH_E_NOMEM; }
    for (uint32_t i = 0; i < hcap; i++) htab[i] = 0xffffffffu;
    synth_rng r;
    rng_seed(&r, seed ^ 0x70cab0000000000dULL);
    double L = s_exp(-4.0);
    uint32_t used = 0;
    v->off[0] = 0;
    for (uint32_t w = 0; w < n_words;) {
        int k = 0;
        double p = 1.0;
        do { k++; p *= rng_unit(&r); } while (p > L);
        int len = 1 + (k - 1);
        if (len > 38) len = 38;
        char buf[40];
        uint64_t h = 1469598103934665603ULL;
        for (int i = 0; i < len; i++) {
            buf[i] = (char)('a' + rng_below(&r, 26));
            h = (h ^ (uint8_t)buf[i]) * 1099511628211ULL;
        }
        h = mix64(h, (uint64_t)len);
        uint32_t slot = (uint32_t)(h & (hcap - 1));
        int dup = 0;
        while (htab[slot] != 0xffffffffu) {
            uint32_t o = htab[slot];
            uint32_t ol = v->off[o + 1] - v->off[o];
            if (ol == (uint32_t)len && memcmp(v->chars + v->off[o], buf, len) == 0) { dup = 1; break; }
            slot = (slot + 1) & (hcap - 1);
        }
        if (dup) continue;
        htab[slot] = w;
        memcpy(v->chars + used, buf, len);
        used += len;
        v->off[w + 1] = used;
        w++;
    }
    free(htab);
    double *wt = (double *)malloc(sizeof(double) * n_words);
    if (!wt) { vocab_free(v); return SYNTH_E_NOMEM; }
    for (uint32_t i = 0; i < n_words; i++) wt[i] = s_exp(-s * s_ln((double)(i + 1)));
    weights_to_cum32(wt, (int)n_words, v->zcum);
    double w16[16];
    for (int i = 0; i < 16; i++) w16[i] = s_exp(-s * s_ln((double)(i + 1)));
    weights_to_cum32(w16, 16, v->zcum16);
    free(wt);
    return SYNTH_OK;
}

/* One independent chunk of order-3 Markov word text: with probability 3/4
 * the next word is entry j (j ~ Zipf(s) over 16) of the successor list of
 * the three-word context, whose entries are Zipf-drawn from a generator
 * seeded by hashing (seed, context, j); otherwise a global Zipf draw.
 * Words are separated by single spaces; the context restarts per chunk. */
static void wordtext_fill(const synth_vocab *v, uint8_t *out, uint64_t n, uint64_t seed,
                          uint64_t chunk) {
    synth_rng r;
    rng_seed(&r, mix64(seed, chunk + 1));
    uint32_t c1 = (uint32_t)draw_zipf(&r, v->zcum, v->n_words);
    uint32_t c2 = (uint32_t)draw_zipf(&r, v->zcum, v->n_words);
    uint32_t c3 = (uint32_t)draw_zipf(&r, v->zcum, v->n_words);
    uint64_t pos = 0;
    while (pos < n) {
        uint32_t w;
        if (rng_below(&r, 4) != 0) {
            int j = draw_cum32(&r, v->zcum16, 16);
            uint64_t h = mix64(mix64(mix64(mix64(seed, c1), c2), c3), (uint64_t)j);
            synth_rng lr;
            lr.s[0] = splitmix64_next(&h); lr.s[1] = splitmix64_next(&h);
            lr.s[2] = splitmix64_next(&h); lr.s[3] = splitmix64_next(&h) | 1;
            w = (uint32_t)draw_zipf(&lr, v->zcum, v->n_words);
        } else {
            w = (uint32_t)draw_zipf(&r, v->zcum, v->n_words);
        }
        uint32_t wl = v->off[w + 1] - v->off[w];
        const char *ws = v->chars + v->off[w];
        for (uint32_t i = 0; i < wl && pos < n; i++) out[pos++] = (uint8_t)ws[i];
        if (pos < n) out[pos++] = ' ';
        c1 = c2; c2 = c3; c3 = w;
    }
}

/* Opaque vocabulary handle so callers can generate chunks in parallel. */
void *synth_vocab_new(uint64_t seed, uint32_t n_words, double zipf_s) {
    synth_vocab *v = (synth_vocab *)malloc(sizeof(synth_vocab));
    if (!v) return NULL;
    if (vocab_build(v, seed, n_words, zipf_s) != SYNTH_OK) { free(v); return NULL; }
    return v;
}

void synth_vocab_free(void *vp) {
    if (!vp) return;
    vocab_free((synth_vocab *)vp);
    free(vp);
}

int synth_wordtext_chunk(const void *vp, uint8_t *out, uint64_t n, uint64_t seed, uint64_t chunk) {
    if (!vp || (!out && n)) return SYNTH_E_INVAL;
    wordtext_fill((const synth_vocab *)vp, out, n, seed, chunk);
    return SYNTH_OK;
}

/* word text of exactly n bytes made of chunks of chunk_bytes */
int synth_wordtext(uint8_t *out, uint64_t n, uint64_t seed, uint64_t chunk_bytes) {
    if ((!out && n) || chunk_bytes == 0) return SYNTH_E_INVAL;
    void *v = synth_vocab_new(seed, 50000, 1.1);
    if (!v) return SYNTH_E_NOMEM;
    for (uint64_t c = 0; c * chunk_bytes < n; c++) {
        uint64_t lo = c * chunk_bytes, len = n - lo < chunk_bytes ? n - lo : chunk_bytes;
        wordtext_fill((const synth_vocab *)v, out + lo, len, seed, c);
    }
    synth_vocab_free(v);
    return SYNTH_OK;
}

/* ======================================================= copy sweep tokens */

/* Tokens generated directly, block by block, until `total` output bytes:
 * a literal run of geometric length (mean lit_mean) of uniform random bytes,
 * then, if the match position mpos satisfies mpos > L and mpos + L fits in
 * the block, a match of length L from a source uniform in [0, mpos - L)
 * (or, with sorted_src, the same draw taken from a per-block sorted batch).
 * Otherwise the block is finished by one literal-only token holding all its
 * remaining bytes.  Arrays are caller-allocated; returns the token count or
 * a negative error. */
static int64_t copy_sweep_table(uint64_t total, uint32_t block_size, const uint32_t *table, uint64_t n_table,
                                uint32_t lit_mean, uint64_t seed, uint32_t *blk_ntok, uint32_t *lit_len,
                                uint32_t *match_len, uint64_t *src, uint64_t tok_cap, uint8_t *literals,
                                uint64_t lit_cap, uint64_t *out_nlit) {
    if (block_size == 0 || !table || n_table == 0 || !blk_ntok || !lit_len || !match_len || !src || !out_nlit)
        return SYNTH_E_INVAL;
    for (uint64_t k = 0; k < n_table; k++)
        if (table[k] == 0) return SYNTH_E_INVAL;
    synth_rng r;
    rng_seed(&r, seed);
    uint64_t nb = (total + block_size - 1) / block_size;
    uint64_t nt = 0, nl = 0;
    for (uint64_t b = 0; b < nb; b++) {
        uint64_t bstart = b * block_size;
        uint64_t bend = bstart + block_size < total ? bstart + block_size : total;
        uint64_t pos = bstart;
        uint32_t cnt = 0;
        while (pos < bend) {
            uint64_t lit = geom0(&r, lit_mean);
            /* a one-entry table draws nothing: the fixed-length sweep */
            const uint64_t L = n_table == 1 ? table[0] : table[rng_below(&r, n_table)];
            uint64_t mpos = pos + lit;
            if (mpos > L && mpos + L <= bend) {
                if (nt >= tok_cap || nl + lit > lit_cap) return SYNTH_E_CAPACITY;
                for (uint64_t i = 0; i < lit; i++) literals[nl + i] = (uint8_t)(rng_next(&r) >> 56);
                nl += lit;
                lit_len[nt] = (uint32_t)lit;
                match_len[nt] = (uint32_t)L;
                src[nt] = rng_below(&r, mpos - L);
                nt++;
                cnt++;
                pos = mpos + L;
            } else {
                uint64_t rest = bend - pos;
                if (nt >= tok_cap || nl + rest > lit_cap) return SYNTH_E_CAPACITY;
                for (uint64_t i = 0; i < rest; i++) literals[nl + i] = (uint8_t)(rng_next(&r) >> 56);
                nl += rest;
                lit_len[nt] = (uint32_t)rest;
                match_len[nt] = 0;
                src[nt] = 0;
                nt++;
                cnt++;
                pos = bend;
            }
        }
        blk_ntok[b] = cnt;
    }
    *out_nlit = nl;
    return (int64_t)nt;
}

int64_t synth_copy_sweep(uint64_t total, uint32_t block_size, uint32_t L, uint32_t lit_mean,
                         uint64_t seed, uint32_t *blk_ntok, uint32_t *lit_len, uint32_t *match_len,
                         uint64_t *src, uint64_t tok_cap, uint8_t *literals, uint64_t lit_cap,
                         uint64_t *out_nlit) {
    const uint32_t table[1] = {L};
    if (L == 0) return SYNTH_E_INVAL;
    return copy_sweep_table(total, block_size, table, 1, lit_mean, seed, blk_ntok, lit_len, match_len, src,
                            tok_cap, literals, lit_cap, out_nlit);
}

/* The copy sweep with each match length drawn uniformly from table[0, n)
 * (an empirical match-length distribution) instead of a fixed L; a length
 * that does not fit ends the block with literals, as a fixed L does. */
int64_t synth_copy_sweep_lengths(uint64_t total, uint32_t block_size, const uint32_t *table, uint64_t n_table,
                                 uint32_t lit_mean, uint64_t seed, uint32_t *blk_ntok, uint32_t *lit_len,
                                 uint32_t *match_len, uint64_t *src, uint64_t tok_cap, uint8_t *literals,
                                 uint64_t lit_cap, uint64_t *out_nlit) {
    return copy_sweep_table(total, block_size, table, n_table, lit_mean, seed, blk_ntok, lit_len, match_len, src,
                            tok_cap, literals, lit_cap, out_nlit);
}

/* ====================================================== batched workload */

/* Output sizes log-uniform in [lo, hi] for n streams, and per-stream seeds. */
int synth_stream_sizes(uint32_t n, uint64_t lo, uint64_t hi, uint64_t seed, uint64_t *sizes,
                       uint64_t *seeds) {
    if (!sizes || !seeds || lo == 0 || hi < lo) return SYNTH_E_INVAL;
    synth_rng r;
    rng_seed(&r, seed);
    double a = s_ln((double)lo), b = s_ln((double)hi);
    for (uint32_t i = 0; i < n; i++) {
        double u = rng_unit(&r);
        uint64_t s = (uint64_t)(s_exp(a + u * (b - a)) + 0.5);
        if (s < lo) s = lo;
        if (s > hi) s = hi;
        sizes[i] = s;
        uint64_t x = seed + 0x1000 + i;
        seeds[i] = splitmix64_next(&x);
    }
    return SYNTH_OK;
}

/* ======================================================= request traces */

/* Poisson arrivals at rate `rate_per_s`; sizes log-uniform in [lo, hi];
 * starts uniform in [0, corpus - size]. */
int synth_requests(uint32_t n, double rate_per_s, uint64_t lo, uint64_t hi, uint64_t corpus,
                   uint64_t seed, double *arrival_s, uint64_t *start, uint64_t *size) {
    if (!arrival_s || !start || !size || lo == 0 || hi < lo || corpus < hi || !(rate_per_s > 0))
        return SYNTH_E_INVAL;
    synth_rng r;
    rng_seed(&r, seed);
    double a = s_ln((double)lo), b = s_ln((double)hi), t = 0.0;
    for (uint32_t i = 0; i < n; i++) {
        t += -s_ln(rng_unit_open(&r)) / rate_per_s;
        arrival_s[i] = t;
        uint64_t s = (uint64_t)(s_exp(a + rng_unit(&r) * (b - a)) + 0.5);
        if (s < lo) s = lo;
        if (s > hi) s = hi;
        size[i] = s;
        start[i] = rng_below(&r, corpus - s + 1);
    }
    return SYNTH_OK;
}

/* raw access for tests of the generator itself */
uint64_t synth_rng_sequence(uint64_t seed, uint64_t *out, uint64_t n) {
    synth_rng r;
    rng_seed(&r, seed);
    for (uint64_t i = 0; i < n; i++) out[i] = rng_next(&r);
    return n;
}

double synth_ln(double x) { return s_ln(x); }
double synth_exp(double x) { return s_exp(x); }
