/*
 * CPU oracle for absolute-offset LZ77 (test infrastructure only).
 *
 * This file is the plain, slow, obviously-correct statement of what the GPU
 * library computes.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load it; the product library never does, and
 * the two share no code.
 *
 * What it follows:
 *  - back-references name absolute output positions (abstract; Sec. I);
 *  - lossless, bit-perfect decode checked by byte compare and FNV
 *    (abstract; Sec. II);
 *  - LZ blocks set at encode time are the unit of decode parallelism
 *    (Sec. II, Sec. V);
 *  - a floor on match length per distance class, bands d < 128, < 16384,
 *    < 2097152, >= 2097152, presets 6/8/10/12 and 12/16/24/32 (Sec. IV-B),
 *    and 16/24/32/48 (Sec. IV-C);
 *  - wavefront decode of matches whose sources are not yet written (Sec. I,
 *    the GPU wavefront decode of the format's first paper).
 * The paper gives no byte layout, no parser and no wave rule; the readings
 * used here (container layout, greedy exact-prefix chain parse, minimal wave
 * tags, chunked FNV, order-0 tile entropy estimate) are listed in the
 * design notes and restated beside each function.
 *
 * Parity pins: round trip, invariants, brute-force greedy and optimal parses
 * on tiny inputs, closed forms and published FNV test vectors (tests/).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------ format v1 */
#define OR_MAGIC0 'A'
#define OR_MAGIC1 'C'
#define OR_MAGIC2 'L'
#define OR_MAGIC3 'Z'
#define OR_VERSION 1
#define OR_F_WAVES 1u
#define OR_HDR 64
#define OR_DIRENT 32
#define OR_TOK 16
#define OR_SRC_MASK ((1ULL << 40) - 1)
#define OR_MAX_WAVE ((1u << 24) - 1)

#define OR_OK 0
#define OR_E_INVAL (-1)
#define OR_E_CORRUPT (-2)
#define OR_E_NOMEM (-3)
#define OR_E_CAPACITY (-4)

static const uint64_t OR_DIST_BOUND[3] = {128, 16384, 2097152};

static uint16_t rd16(const uint8_t *p) { return (uint16_t)(p[0] | (p[1] << 8)); }
static uint32_t rd32(const uint8_t *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static uint64_t rd64(const uint8_t *p) { return (uint64_t)rd32(p) | ((uint64_t)rd32(p + 4) << 32); }
static void wr16(uint8_t *p, uint16_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
static void wr32(uint8_t *p, uint32_t v) {
    for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i));
}
static void wr64(uint8_t *p, uint64_t v) {
    for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i));
}

/* distance class of d = dst - src (Sec. IV-B bands) */
static int dist_class(uint64_t d) {
    if (d < OR_DIST_BOUND[0]) return 0;
    if (d < OR_DIST_BOUND[1]) return 1;
    if (d < OR_DIST_BOUND[2]) return 2;
    return 3;
}

/* Parsed view of a container.  Field meanings follow the v1 layout:
 * header 64 B, directory of 32-B entries, 16-B tokens, literal bytes. */
typedef struct {
    uint64_t total_len, n_tokens, n_literals;
    uint32_t block_size, n_blocks, n_waves;
    uint16_t flags;
    uint8_t mm[4];
    const uint8_t *dir, *tok, *lit;
} or_view;

static int or_parse(const uint8_t *c, uint64_t clen, or_view *v) {
    if (!c || clen < OR_HDR) return OR_E_CORRUPT;
    if (c[0] != OR_MAGIC0 || c[1] != OR_MAGIC1 || c[2] != OR_MAGIC2 || c[3] != OR_MAGIC3)
        return OR_E_CORRUPT;
    if (rd16(c + 4) != OR_VERSION) return OR_E_CORRUPT;
    v->flags = rd16(c + 6);
    v->total_len = rd64(c + 8);
    v->block_size = rd32(c + 16);
    v->n_blocks = rd32(c + 20);
    v->n_tokens = rd64(c + 24);
    v->n_literals = rd64(c + 32);
    v->n_waves = rd32(c + 40);
    memcpy(v->mm, c + 44, 4);
    if (v->block_size == 0 || v->block_size % 16) return OR_E_CORRUPT;
    if (v->total_len > OR_SRC_MASK) return OR_E_CORRUPT;
    uint64_t nb = (v->total_len + v->block_size - 1) / v->block_size;
    if (nb != v->n_blocks) return OR_E_CORRUPT;
    uint64_t need = OR_HDR + (uint64_t)OR_DIRENT * v->n_blocks;
    if (v->n_tokens > (clen - (need < clen ? need : clen)) / OR_TOK) return OR_E_CORRUPT;
    need += (uint64_t)OR_TOK * v->n_tokens;
    if (need > clen || v->n_literals != clen - need) return OR_E_CORRUPT;
    v->dir = c + OR_HDR;
    v->tok = v->dir + (uint64_t)OR_DIRENT * v->n_blocks;
    v->lit = v->tok + (uint64_t)OR_TOK * v->n_tokens;
    return OR_OK;
}

typedef struct { uint32_t lit_len, match_len; uint64_t src; uint32_t wave; } or_tok;

static or_tok tok_at(const or_view *v, uint64_t i) {
    const uint8_t *p = v->tok + (uint64_t)OR_TOK * i;
    or_tok t;
    t.lit_len = rd32(p);
    t.match_len = rd32(p + 4);
    uint64_t sw = rd64(p + 8);
    t.src = sw & OR_SRC_MASK;
    t.wave = (uint32_t)(sw >> 40);
    return t;
}

/* ---------------------------------------------------------- validation */

/* Structural validity of a container: directory contiguity, per-block
 * token lengths summing to the block length, matches strictly before
 * their targets (src + len <= dst), match_len == 0 only on a block's last
 * token, literal counts.  If the wave flag is set, the tags must also be
 * legal (tag >= the minimal requirement of the wave rule). */
int oracle_validate(const uint8_t *c, uint64_t clen);

static int or_structure(const or_view *v) {
    uint64_t tok_next = 0, lit_next = 0;
    for (uint32_t b = 0; b < v->n_blocks; b++) {
        const uint8_t *d = v->dir + (uint64_t)OR_DIRENT * b;
        uint64_t tok_off = rd64(d), lit_off = rd64(d + 8);
        uint32_t ntok = rd32(d + 16);
        if (tok_off != tok_next || lit_off != lit_next) return OR_E_CORRUPT;
        if (ntok == 0 || tok_off + ntok > v->n_tokens) return OR_E_CORRUPT;
        uint64_t bstart = (uint64_t)b * v->block_size;
        uint64_t bend = bstart + v->block_size < v->total_len ? bstart + v->block_size : v->total_len;
        uint64_t pos = bstart;
        for (uint32_t k = 0; k < ntok; k++) {
            or_tok t = tok_at(v, tok_off + k);
            if (t.match_len == 0 && (k + 1 != ntok || t.src != 0 || t.wave != 0)) return OR_E_CORRUPT;
            if ((uint64_t)t.lit_len > bend - pos) return OR_E_CORRUPT;
            pos += t.lit_len;
            lit_next += t.lit_len;
            if (t.match_len) {
                if ((uint64_t)t.match_len > bend - pos) return OR_E_CORRUPT;
                if (t.src + t.match_len > pos) return OR_E_CORRUPT;
                pos += t.match_len;
            }
        }
        if (pos != bend) return OR_E_CORRUPT;
        tok_next = tok_off + ntok;
    }
    if (tok_next != v->n_tokens || lit_next != v->n_literals) return OR_E_CORRUPT;
    return OR_OK;
}

/* ------------------------------------------------------- sequential decode */

/* The plain definition of decode: for each block in order, for each token
 * in order, append lit_len literal bytes, then append match_len bytes read
 * one at a time from absolute position src.  Wave tags do not enter. */
int oracle_decode(const uint8_t *c, uint64_t clen, uint8_t *out, uint64_t cap) {
    or_view v;
    int rc = or_parse(c, clen, &v);
    if (rc) return rc;
    if ((rc = or_structure(&v))) return rc;
    if (cap < v.total_len) return OR_E_CAPACITY;
    uint64_t pos = 0, li = 0;
    for (uint64_t i = 0; i < v.n_tokens; i++) {
        or_tok t = tok_at(&v, i);
        for (uint32_t k = 0; k < t.lit_len; k++) out[pos++] = v.lit[li++];
        for (uint32_t k = 0; k < t.match_len; k++) { out[pos] = out[t.src + k]; pos++; }
    }
    return pos == v.total_len ? OR_OK : OR_E_CORRUPT;
}

/* ------------------------------------------------------------ wave tags */

/* Minimal wave tags (one per token; 0 for literal-only tokens).  fin(p) is
 * the wave in which output byte p becomes final: 0 for literal bytes and
 * the tag of the covering match otherwise.  For a match m in block b,
 *   tag(m) = max(0, max_{p in src, p in b} fin(p), max_{p in src, p not in b} fin(p) + 1)
 * computed in token order, which sees every source byte final because
 * sources lie strictly before their targets.  With `given` non-NULL the
 * function instead checks given[i] >= requirement(i) under fin = given
 * tags and returns OR_E_CORRUPT on the first violation; with `extra`
 * non-NULL it assigns tag(m) = requirement(m) + extra[m] (a legal,
 * non-minimal tagging). */
static int or_tags(const or_view *v, const uint32_t *given, const uint32_t *extra, uint32_t *tags,
                   uint32_t *max_tag) {
    uint32_t *fin = (uint32_t *)malloc(sizeof(uint32_t) * (v->total_len ? v->total_len : 1));
    if (!fin) return OR_E_NOMEM;
    uint64_t pos = 0;
    uint32_t mx = 0;
    for (uint32_t b = 0; b < v->n_blocks; b++) {
        const uint8_t *d = v->dir + (uint64_t)OR_DIRENT * b;
        uint64_t tok_off = rd64(d);
        uint32_t ntok = rd32(d + 16);
        uint64_t bstart = (uint64_t)b * v->block_size;
        uint64_t bend = bstart + v->block_size;
        for (uint32_t k = 0; k < ntok; k++) {
            uint64_t i = tok_off + k;
            or_tok t = tok_at(v, i);
            for (uint32_t j = 0; j < t.lit_len; j++) fin[pos++] = 0;
            uint32_t tag = 0;
            if (t.match_len) {
                uint32_t req = 0;
                for (uint32_t j = 0; j < t.match_len; j++) {
                    uint64_t p = t.src + j;
                    uint32_t f = fin[p] + ((p >= bstart && p < bend) ? 0u : 1u);
                    if (f > req) req = f;
                }
                if (given) {
                    if (given[i] < req) { free(fin); return OR_E_CORRUPT; }
                    tag = given[i];
                } else {
                    tag = req + (extra ? extra[i] : 0);
                }
                if (tag > OR_MAX_WAVE) { free(fin); return OR_E_CAPACITY; }
                for (uint32_t j = 0; j < t.match_len; j++) fin[pos++] = tag;
            } else if (given && given[i] != 0) {
                free(fin);
                return OR_E_CORRUPT;
            }
            if (tags) tags[i] = tag;
            if (tag > mx) mx = tag;
        }
    }
    free(fin);
    if (max_tag) *max_tag = mx;
    return OR_OK;
}

int oracle_validate(const uint8_t *c, uint64_t clen) {
    or_view v;
    int rc = or_parse(c, clen, &v);
    if (rc) return rc;
    if ((rc = or_structure(&v))) return rc;
    if (v.flags & OR_F_WAVES) {
        uint32_t *given = (uint32_t *)malloc(sizeof(uint32_t) * (v.n_tokens ? v.n_tokens : 1));
        if (!given) return OR_E_NOMEM;
        uint32_t mx = 0;
        for (uint64_t i = 0; i < v.n_tokens; i++) {
            given[i] = tok_at(&v, i).wave;
            if (given[i] > mx) mx = given[i];
        }
        rc = or_tags(&v, given, NULL, NULL, NULL);
        free(given);
        if (rc) return rc;
        if (v.n_tokens && v.n_waves != mx + 1) return OR_E_CORRUPT;
    }
    return OR_OK;
}

/* minimal tags of a container's tokens (ignores any tags it carries) */
int oracle_min_tags(const uint8_t *c, uint64_t clen, uint32_t *tags, uint32_t *n_waves) {
    or_view v;
    int rc = or_parse(c, clen, &v);
    if (rc) return rc;
    if ((rc = or_structure(&v))) return rc;
    uint32_t mx = 0;
    rc = or_tags(&v, NULL, NULL, tags, &mx);
    if (n_waves) *n_waves = v.n_tokens ? mx + 1 : 0;
    return rc;
}

/* rewrite a container's tags in place: minimal tags plus extra[i] at each
 * match (extra NULL = minimal), setting the wave flag and count. */
int oracle_retag(uint8_t *c, uint64_t clen, const uint32_t *extra) {
    or_view v;
    int rc = or_parse(c, clen, &v);
    if (rc) return rc;
    if ((rc = or_structure(&v))) return rc;
    uint32_t *tags = (uint32_t *)malloc(sizeof(uint32_t) * (v.n_tokens ? v.n_tokens : 1));
    if (!tags) return OR_E_NOMEM;
    uint32_t mx = 0;
    rc = or_tags(&v, NULL, extra, tags, &mx);
    if (rc) { free(tags); return rc; }
    uint8_t *tok = c + (v.tok - c);
    for (uint64_t i = 0; i < v.n_tokens; i++) {
        uint8_t *p = tok + (uint64_t)OR_TOK * i;
        uint64_t sw = rd64(p + 8);
        sw = (sw & OR_SRC_MASK) | ((uint64_t)tags[i] << 40);
        wr64(p + 8, sw);
    }
    free(tags);
    wr16(c + 6, (uint16_t)(v.flags | OR_F_WAVES));
    wr32(c + 40, v.n_tokens ? mx + 1 : 0);
    return OR_OK;
}

/* clear the tags of a container (flag off, all tags 0, wave count 0,
 * per-block max wave 0) */
int oracle_strip_tags(uint8_t *c, uint64_t clen) {
    or_view v;
    int rc = or_parse(c, clen, &v);
    if (rc) return rc;
    for (uint32_t b = 0; b < v.n_blocks; b++) wr16(c + OR_HDR + (uint64_t)OR_DIRENT * b + 20, 0);
    uint8_t *tok = c + (v.tok - c);
    for (uint64_t i = 0; i < v.n_tokens; i++) {
        uint8_t *p = tok + (uint64_t)OR_TOK * i;
        wr64(p + 8, rd64(p + 8) & OR_SRC_MASK);
    }
    wr16(c + 6, (uint16_t)(v.flags & ~OR_F_WAVES));
    wr32(c + 40, 0);
    return OR_OK;
}

/* ------------------------------------------------------------- packing */

uint64_t oracle_container_bytes(uint64_t total_len, uint32_t block_size, uint64_t n_tokens,
                                uint64_t n_literals) {
    uint64_t nb = block_size ? (total_len + block_size - 1) / block_size : 0;
    return OR_HDR + (uint64_t)OR_DIRENT * nb + (uint64_t)OR_TOK * n_tokens + n_literals;
}

static void or_write_header(uint8_t *c, uint64_t total_len, uint32_t bs, uint32_t nb,
                            uint64_t nt, uint64_t nl, const uint8_t mm[4]) {
    memset(c, 0, OR_HDR);
    c[0] = OR_MAGIC0; c[1] = OR_MAGIC1; c[2] = OR_MAGIC2; c[3] = OR_MAGIC3;
    wr16(c + 4, OR_VERSION);
    wr16(c + 6, 0);
    wr64(c + 8, total_len);
    wr32(c + 16, bs);
    wr32(c + 20, nb);
    wr64(c + 24, nt);
    wr64(c + 32, nl);
    wr32(c + 40, 0);
    memcpy(c + 44, mm, 4);
    for (int i = 0; i < 3; i++) wr32(c + 48 + 4 * i, (uint32_t)OR_DIST_BOUND[i]);
}

/* Assemble a container from token arrays (blk_ntok per block; lit_len,
 * match_len, src per token; the literal bytes) and, when with_tags, give it
 * minimal tags (without tags the wave flag stays clear; the per-byte tag
 * pass needs 4 bytes per output byte).  Returns the container size or a
 * negative error. */
int64_t oracle_pack(uint64_t total_len, uint32_t block_size, const uint8_t mm[4],
                    const uint32_t *blk_ntok, const uint32_t *lit_len, const uint32_t *match_len,
                    const uint64_t *src, uint64_t n_tokens, const uint8_t *literals,
                    uint64_t n_literals, uint8_t *out, uint64_t cap, int with_tags) {
    if (block_size == 0 || block_size % 16) return OR_E_INVAL;
    uint64_t nb = (total_len + block_size - 1) / block_size;
    if (nb > 0xffffffffULL) return OR_E_INVAL;
    uint64_t need = oracle_container_bytes(total_len, block_size, n_tokens, n_literals);
    if (cap < need) return OR_E_CAPACITY;
    or_write_header(out, total_len, block_size, (uint32_t)nb, n_tokens, n_literals, mm);
    uint8_t *dir = out + OR_HDR, *tok = dir + OR_DIRENT * nb, *lit = tok + OR_TOK * n_tokens;
    uint64_t t = 0, l = 0;
    for (uint64_t b = 0; b < nb; b++) {
        uint8_t *d = dir + OR_DIRENT * b;
        memset(d, 0, OR_DIRENT);
        wr64(d, t);
        wr64(d + 8, l);
        wr32(d + 16, blk_ntok[b]);
        memcpy(d + 24, mm, 4);
        for (uint32_t k = 0; k < blk_ntok[b]; k++, t++) {
            if (t >= n_tokens) return OR_E_INVAL;
            uint8_t *p = tok + OR_TOK * t;
            wr32(p, lit_len[t]);
            wr32(p + 4, match_len[t]);
            wr64(p + 8, match_len[t] ? (src[t] & OR_SRC_MASK) : 0);
            l += lit_len[t];
        }
    }
    if (t != n_tokens || l != n_literals) return OR_E_INVAL;
    memcpy(lit, literals, n_literals);
    if (!with_tags) return (int64_t)need;
    int rc = oracle_retag(out, need, NULL);
    if (rc) return rc;
    /* per-block max wave, informational */
    or_view v;
    or_parse(out, need, &v);
    for (uint64_t b = 0; b < nb; b++) {
        uint8_t *d = dir + OR_DIRENT * b;
        uint64_t off = rd64(d);
        uint32_t n = rd32(d + 16), mw = 0;
        for (uint32_t k = 0; k < n; k++) {
            uint32_t w = tok_at(&v, off + k).wave;
            if (w > mw) mw = w;
        }
        wr16(d + 20, (uint16_t)(mw > 0xffff ? 0xffff : mw));
    }
    return (int64_t)need;
}

/* ------------------------------------------------------------- encoder */

/* Exact previous-occurrence links: prev[p] is the largest q < p with
 * x[q..q+3] == x[p..p+3] (or -1), for p <= n - 4.  Built with an
 * open-addressing map from the 4-byte value to its last position. */
static int64_t *or_prev_links(const uint8_t *x, uint64_t n) {
    uint64_t np = n >= 4 ? n - 3 : 0;
    int64_t *prev = (int64_t *)malloc(sizeof(int64_t) * (np ? np : 1));
    if (!prev) return NULL;
    uint64_t cap = 1024;
    while (cap < 2 * np && cap < (1ULL << 30)) cap <<= 1;
    uint32_t *keys = NULL;
    int64_t *last = NULL;
    uint64_t used = 0;
    for (;;) {
        keys = (uint32_t *)malloc(sizeof(uint32_t) * cap);
        last = (int64_t *)malloc(sizeof(int64_t) * cap);
        if (!keys || !last) { free(keys); free(last); free(prev); return NULL; }
        for (uint64_t i = 0; i < cap; i++) last[i] = -1;
        used = 0;
        int grow = 0;
        for (uint64_t p = 0; p < np; p++) {
            uint32_t k = rd32(x + p);
            uint64_t h = ((uint64_t)k * 0x9E3779B97F4A7C15ULL) >> 20;
            uint64_t s = h & (cap - 1);
            while (last[s] >= 0 && keys[s] != k) s = (s + 1) & (cap - 1);
            if (last[s] < 0) {
                keys[s] = k;
                prev[p] = -1;
                if (++used * 2 > cap) { grow = 1; break; }
            } else {
                prev[p] = last[s];
            }
            last[s] = (int64_t)p;
        }
        free(keys);
        free(last);
        if (!grow) break;
        cap <<= 1;
    }
    return prev;
}

/* Greedy parse (one block at a time, in order).  At position p (with at
 * least 4 bytes left in the stream) the candidates are the earlier
 * positions with the same 4-byte prefix, most recent first, at most
 * chain_depth of them and at distance <= window.  Candidate s gives
 * len = common prefix of x[s..] and x[p..] capped at min(p - s, block_end - p);
 * it is valid when len >= T[class(p - s)] with T the block's thresholds.
 * The longest valid candidate wins, ties to the nearest (first found).  A
 * match is emitted and p advances by len; otherwise p advances by one
 * literal byte.  The block's trailing literals form a last token with
 * match_len = 0.  Tags are then the minimal wave tags. */
int64_t oracle_encode(const uint8_t *x, uint64_t n, uint32_t block_size, const uint8_t mm[4],
                      const uint8_t *block_mm, uint32_t chain_depth, uint64_t window,
                      uint8_t *out, uint64_t cap) {
    if (block_size == 0 || block_size % 16 || n > OR_SRC_MASK) return OR_E_INVAL;
    for (int i = 0; i < 4; i++) if (mm[i] < 4) return OR_E_INVAL;
    uint64_t nb = (n + block_size - 1) / block_size;
    if (block_mm)
        for (uint64_t i = 0; i < 4 * nb; i++) if (block_mm[i] < 4) return OR_E_INVAL;
    uint64_t maxtok = n / 4 + nb + 1;
    uint32_t *ll = (uint32_t *)malloc(sizeof(uint32_t) * maxtok);
    uint32_t *ml = (uint32_t *)malloc(sizeof(uint32_t) * maxtok);
    uint64_t *sr = (uint64_t *)malloc(sizeof(uint64_t) * maxtok);
    uint32_t *bn = (uint32_t *)malloc(sizeof(uint32_t) * (nb ? nb : 1));
    uint8_t *lits = (uint8_t *)malloc(n ? n : 1);
    int64_t *prev = or_prev_links(x, n);
    if (!ll || !ml || !sr || !bn || !lits || !prev) {
        free(ll); free(ml); free(sr); free(bn); free(lits); free(prev);
        return OR_E_NOMEM;
    }
    uint64_t nt = 0, nl = 0;
    for (uint64_t b = 0; b < nb; b++) {
        const uint8_t *T = block_mm ? block_mm + 4 * b : mm;
        uint64_t bstart = b * block_size, bend = bstart + block_size < n ? bstart + block_size : n;
        uint64_t p = bstart, lit_start = bstart;
        uint32_t cnt = 0;
        while (p < bend) {
            uint64_t best_len = 0, best_src = 0;
            if (p + 4 <= n) {
                int64_t q = prev[p];
                uint32_t seen = 0;
                while (q >= 0 && p - (uint64_t)q <= window && seen < chain_depth) {
                    seen++;
                    uint64_t d = p - (uint64_t)q;
                    uint64_t lim = d < bend - p ? d : bend - p;
                    uint64_t len = 0;
                    while (len < lim && x[q + len] == x[p + len]) len++;
                    if (len >= T[dist_class(d)] && len > best_len) { best_len = len; best_src = (uint64_t)q; }
                    q = prev[q];
                }
            }
            if (best_len) {
                uint64_t lit = p - lit_start;
                memcpy(lits + nl, x + lit_start, lit);
                nl += lit;
                ll[nt] = (uint32_t)lit;
                ml[nt] = (uint32_t)best_len;
                sr[nt] = best_src;
                nt++;
                cnt++;
                p += best_len;
                lit_start = p;
            } else {
                p++;
            }
        }
        if (lit_start < bend || cnt == 0) {
            uint64_t lit = bend - lit_start;
            memcpy(lits + nl, x + lit_start, lit);
            nl += lit;
            ll[nt] = (uint32_t)lit;
            ml[nt] = 0;
            sr[nt] = 0;
            nt++;
            cnt++;
        }
        bn[b] = cnt;
    }
    int64_t rc = oracle_pack(n, block_size, mm, bn, ll, ml, sr, nt, lits, nl, out, cap, 1);
    if (rc > 0 && block_mm) {
        for (uint64_t b = 0; b < nb; b++) memcpy(out + OR_HDR + OR_DIRENT * b + 24, block_mm + 4 * b, 4);
    }
    free(ll); free(ml); free(sr); free(bn); free(lits); free(prev);
    return rc;
}

uint64_t oracle_encode_bound(uint64_t n, uint32_t block_size) {
    uint64_t nb = block_size ? (n + block_size - 1) / block_size : 0;
    return oracle_container_bytes(n, block_size, n / 4 + nb + 1, n);
}

/* Every match satisfies its block's distance-class minimum length. */
int oracle_check_thresholds(const uint8_t *c, uint64_t clen) {
    or_view v;
    int rc = or_parse(c, clen, &v);
    if (rc) return rc;
    if ((rc = or_structure(&v))) return rc;
    uint64_t pos = 0;
    for (uint32_t b = 0; b < v.n_blocks; b++) {
        const uint8_t *d = v.dir + (uint64_t)OR_DIRENT * b;
        uint64_t off = rd64(d);
        uint32_t n = rd32(d + 16);
        const uint8_t *T = d + 24;
        for (uint32_t k = 0; k < n; k++) {
            or_tok t = tok_at(&v, off + k);
            pos += t.lit_len;
            if (t.match_len) {
                if (t.match_len < T[dist_class(pos - t.src)]) return OR_E_CORRUPT;
                pos += t.match_len;
            }
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ FNV */

/* FNV-1a 64: offset basis 14695981039346656037, prime 1099511628211. */
uint64_t oracle_fnv1a64(const uint8_t *p, uint64_t n, uint64_t h) {
    for (uint64_t i = 0; i < n; i++) { h ^= p[i]; h *= 1099511628211ULL; }
    return h;
}

/* Chunked stream hash: FNV-1a 64 of each 64 KiB chunk, then FNV-1a 64 of
 * the chunk hashes (8 little-endian bytes each) followed by the total
 * length (8 little-endian bytes). */
uint64_t oracle_fnv_chunked(const uint8_t *p, uint64_t n) {
    const uint64_t B = 14695981039346656037ULL, CH = 65536;
    uint64_t h = B;
    uint8_t le[8];
    for (uint64_t off = 0; off < n; off += CH) {
        uint64_t len = n - off < CH ? n - off : CH;
        wr64(le, oracle_fnv1a64(p + off, len, B));
        h = oracle_fnv1a64(le, 8, h);
    }
    wr64(le, n);
    return oracle_fnv1a64(le, 8, h);
}

/* ---------------------------------------------------- entropy estimate */

static double or_h0_bytes(const uint8_t *s, uint64_t n) {
    /* order-0 cost in bytes of one tile plus a 512-byte table */
    uint64_t cnt[256] = {0};
    for (uint64_t i = 0; i < n; i++) cnt[s[i]]++;
    double bits = 0.0;
    for (int i = 0; i < 256; i++)
        if (cnt[i]) bits -= (double)cnt[i] * log2((double)cnt[i] / (double)n);
    return bits / 8.0 + 512.0;
}

static double or_stream_cost(const uint8_t *s, uint64_t n) {
    double c = 0.0;
    for (uint64_t off = 0; off < n; off += 65536) c += or_h0_bytes(s + off, n - off < 65536 ? n - off : 65536);
    return c;
}

static uint64_t or_leb128(uint8_t *dst, uint64_t v) {
    uint64_t k = 0;
    do {
        uint8_t b = v & 0x7f;
        v >>= 7;
        dst[k++] = (uint8_t)(b | (v ? 0x80 : 0));
    } while (v);
    return k;
}

/* Estimated entropy-coded size: header + directory + the order-0 cost of
 * 64 KiB tiles of four separated streams: literal bytes, LEB128 lit_len of
 * every token, LEB128 match_len of every token, and the source position of
 * every match as w little-endian bytes, w the fewest bytes that hold
 * total_len - 1.  An ideal tile coder standing in for tile-ANS (Sec. II). */
int oracle_est_bytes(const uint8_t *c, uint64_t clen, double *out) {
    or_view v;
    int rc = or_parse(c, clen, &v);
    if (rc) return rc;
    int w = 1;
    while (w < 8 && v.total_len > 1 && ((v.total_len - 1) >> (8 * w)) != 0) w++;
    uint8_t *ls = (uint8_t *)malloc(10 * (v.n_tokens + 1));
    uint8_t *ms = (uint8_t *)malloc(10 * (v.n_tokens + 1));
    uint8_t *os = (uint8_t *)malloc((uint64_t)w * (v.n_tokens + 1));
    if (!ls || !ms || !os) { free(ls); free(ms); free(os); return OR_E_NOMEM; }
    uint64_t nl = 0, nm = 0, no = 0;
    for (uint64_t i = 0; i < v.n_tokens; i++) {
        or_tok t = tok_at(&v, i);
        nl += or_leb128(ls + nl, t.lit_len);
        nm += or_leb128(ms + nm, t.match_len);
        if (t.match_len)
            for (int k = 0; k < w; k++) os[no++] = (uint8_t)(t.src >> (8 * k));
    }
    double tot = (double)OR_HDR + (double)OR_DIRENT * v.n_blocks;
    tot += or_stream_cost(v.lit, v.n_literals) + or_stream_cost(ls, nl) + or_stream_cost(ms, nm) +
           or_stream_cost(os, no);
    free(ls); free(ms); free(os);
    *out = tot;
    return OR_OK;
}

/* ----------------------------------------------------------- statistics */

/* out[0] matches, [1] match bytes, [2] literal bytes, [3] matches < 16 B,
 * [4] matches < 32 B, [5..8] matches per distance class, [9] tokens,
 * [10] blocks, [11] total_len */
int oracle_stats(const uint8_t *c, uint64_t clen, uint64_t *out) {
    or_view v;
    int rc = or_parse(c, clen, &v);
    if (rc) return rc;
    memset(out, 0, sizeof(uint64_t) * 12);
    uint64_t pos = 0;
    for (uint64_t i = 0; i < v.n_tokens; i++) {
        or_tok t = tok_at(&v, i);
        pos += t.lit_len;
        out[2] += t.lit_len;
        if (t.match_len) {
            out[0]++;
            out[1] += t.match_len;
            if (t.match_len < 16) out[3]++;
            if (t.match_len < 32) out[4]++;
            out[5 + dist_class(pos - t.src)]++;
            pos += t.match_len;
        }
    }
    out[9] = v.n_tokens;
    out[10] = v.n_blocks;
    out[11] = v.total_len;
    return OR_OK;
}
