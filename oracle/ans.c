/* Tile entropy layer of the CPU oracle (test infrastructure only).
 *
 * In the paper's pipeline an ANS entropy stage works on 64 KB tiles, many
 * at once, ahead of the match kernel (Sec. II), with no coder parameters
 * given.  Our reading:
 *
 *  - every byte stream is cut into tiles of 65536 bytes (the last shorter);
 *  - each tile is coded on its own with an order-0 range-variant asymmetric
 *    numeral system (rANS, Duda): symbol probabilities are the tile's byte
 *    counts quantised to frequencies f_s summing to M = 2^12;
 *  - 32 coder states run interleaved: symbol i of the tile belongs to state
 *    (i mod 32), so a 32-lane warp decodes 32 consecutive bytes per step;
 *  - states live in [L, 2^32) with L = 2^16 and renormalise by 16-bit words
 *    kept in one stream per tile; within a decode step the states that need
 *    a word take the next ones in increasing lane order.
 *
 * The plain definitions, one symbol at a time:
 *   encode s from state x:  while x >= 2^20 * f_s: emit x mod 2^16, x >>= 16
 *                           x <- floor(x / f_s) * M + (x mod f_s) + c_s
 *   decode from state x:    r = x mod M, s = the symbol with c_s <= r < c_s + f_s
 *                           x <- f_s * floor(x / M) + r - c_s
 *                           if x < L: x <- x * 2^16 + next word
 * with c_s the cumulative frequency of the symbols below s.  The encoder
 * runs from the last symbol to the first, so the words it emits are
 * consumed in reverse order by the decoder.
 *
 * Tile payload (little-endian): u16 freq[256], u32 state[32] (the states
 * after encoding, which the decoder starts from), u32 n_words, then the
 * 16-bit words in decode order.
 *
 * Container "ACLE" (entropy-coded form of a v1 container): the v1 header and
 * block directory stored raw, then 17 streams coded by tiles: the 16 byte
 * planes of the token array (plane k holds byte k of every 16-byte token)
 * and the literal bytes.  Layout:
 *   0   "ACLE", u32 version = 1, u64 v1 container size, u64 raw prefix bytes,
 *       u32 n_streams = 17, u32 tile size = 65536, u64 n_tokens,
 *       u64 n_literals, u64 n_tiles, u64 payload offset  (64 bytes)
 *   64  raw prefix (v1 header and directory), padded to 16 bytes
 *   ..  stream table: per stream u64 length, u64 first tile    (16 B each)
 *   ..  tile table: per tile u64 payload offset (from the payload base),
 *       u32 payload bytes, u32 symbols                        (16 B each)
 *   ..  payloads, each starting on a 16-byte boundary
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ANS_OK 0
#define ANS_E_INVAL (-1)
#define ANS_E_CORRUPT (-2)
#define ANS_E_NOMEM (-3)
#define ANS_E_CAPACITY (-4)

#define ANS_M_LOG 12u
#define ANS_M (1u << ANS_M_LOG)
#define ANS_L (1u << 16)
#define ANS_LANES 32u
#define ANS_TILE 65536u
#define ANS_HDR (512u + 4u * ANS_LANES + 4u)

#define ACLE_HDR 64u
#define ACLE_STREAMS 17u

static void put16(uint8_t *p, uint16_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
static void put32(uint8_t *p, uint32_t v) { for (int k = 0; k < 4; k++) p[k] = (uint8_t)(v >> (8 * k)); }
static void put64(uint8_t *p, uint64_t v) { for (int k = 0; k < 8; k++) p[k] = (uint8_t)(v >> (8 * k)); }
static uint16_t get16(const uint8_t *p) { return (uint16_t)(p[0] | (p[1] << 8)); }
static uint32_t get32(const uint8_t *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static uint64_t get64(const uint8_t *p) { return (uint64_t)get32(p) | ((uint64_t)get32(p + 4) << 32); }

/* Frequencies from byte counts: a single distinct symbol takes all of M;
 * otherwise each present symbol gets max(1, floor(count * M / n)), and the
 * difference to M is settled on the largest frequencies (ties to the
 * smaller byte value): added to the largest, or taken one at a time from
 * the current largest while it stays >= 1. */
int oracle_ans_quantize(const uint64_t *counts, uint64_t n, uint16_t *freq) {
    if (!counts || !freq) return ANS_E_INVAL;
    uint64_t total = 0;
    int distinct = 0, only = -1;
    for (int s = 0; s < 256; s++) {
        total += counts[s];
        if (counts[s]) { distinct++; only = s; }
    }
    if (total != n) return ANS_E_INVAL;
    memset(freq, 0, 256 * sizeof(uint16_t));
    if (n == 0) return ANS_OK;
    if (distinct == 1) {
        freq[only] = (uint16_t)ANS_M;
        return ANS_OK;
    }
    int64_t sum = 0;
    for (int s = 0; s < 256; s++) {
        if (!counts[s]) continue;
        uint64_t f = (uint64_t)(((unsigned __int128)counts[s] * ANS_M) / n);
        freq[s] = (uint16_t)(f ? f : 1);
        sum += freq[s];
    }
    if (sum < (int64_t)ANS_M) {
        int best = 0;
        for (int s = 1; s < 256; s++)
            if (freq[s] > freq[best]) best = s;
        freq[best] = (uint16_t)(freq[best] + (ANS_M - sum));
    }
    while (sum > (int64_t)ANS_M) {
        int best = 0;
        for (int s = 1; s < 256; s++)
            if (freq[s] > freq[best]) best = s;
        if (freq[best] <= 1) return ANS_E_INVAL;  /* cannot happen for <= 256 symbols */
        freq[best]--;
        sum--;
    }
    return ANS_OK;
}

/* Largest payload a tile of n bytes can take. */
uint64_t oracle_ans_tile_bound(uint64_t n) { return ANS_HDR + 2 * (n + ANS_LANES); }

int oracle_ans_encode_tile(const uint8_t *src, uint32_t n, uint8_t *out, uint64_t cap, uint64_t *size) {
    if ((n && !src) || !out || !size || n > ANS_TILE) return ANS_E_INVAL;
    if (cap < oracle_ans_tile_bound(n)) return ANS_E_CAPACITY;
    uint64_t counts[256] = {0};
    for (uint32_t i = 0; i < n; i++) counts[src[i]]++;
    uint16_t freq[256];
    int rc = oracle_ans_quantize(counts, n, freq);
    if (rc) return rc;
    uint32_t cum[257];
    cum[0] = 0;
    for (int s = 0; s < 256; s++) cum[s + 1] = cum[s] + freq[s];
    uint32_t x[ANS_LANES];
    for (uint32_t k = 0; k < ANS_LANES; k++) x[k] = ANS_L;
    /* words in emission order; reversed at the end into decode order */
    uint16_t *w = (uint16_t *)malloc(sizeof(uint16_t) * (n + ANS_LANES));
    if (!w) return ANS_E_NOMEM;
    uint64_t nw = 0;
    for (uint32_t i = n; i-- > 0;) {
        const uint32_t lane = i % ANS_LANES, s = src[i], f = freq[s];
        uint32_t v = x[lane];
        while ((uint64_t)v >= ((uint64_t)1 << 20) * f) {
            w[nw++] = (uint16_t)(v & 0xffffu);
            v >>= 16;
        }
        x[lane] = (v / f) * ANS_M + (v % f) + cum[s];
    }
    for (int s = 0; s < 256; s++) put16(out + 2 * s, freq[s]);
    for (uint32_t k = 0; k < ANS_LANES; k++) put32(out + 512 + 4 * k, x[k]);
    put32(out + 512 + 4 * ANS_LANES, (uint32_t)nw);
    uint8_t *p = out + ANS_HDR;
    for (uint64_t j = 0; j < nw; j++) put16(p + 2 * j, w[nw - 1 - j]);
    free(w);
    *size = ANS_HDR + 2 * nw;
    return ANS_OK;
}

int oracle_ans_decode_tile(const uint8_t *in, uint64_t size, uint8_t *out, uint32_t n) {
    if (!in || (n && !out) || n > ANS_TILE) return ANS_E_INVAL;
    if (size < ANS_HDR) return ANS_E_CORRUPT;
    uint16_t freq[256];
    uint32_t cum[257];
    cum[0] = 0;
    for (int s = 0; s < 256; s++) {
        freq[s] = get16(in + 2 * s);
        cum[s + 1] = cum[s] + freq[s];
    }
    if (n && cum[256] != ANS_M) return ANS_E_CORRUPT;
    uint32_t x[ANS_LANES];
    for (uint32_t k = 0; k < ANS_LANES; k++) x[k] = get32(in + 512 + 4 * k);
    const uint64_t nw = get32(in + 512 + 4 * ANS_LANES);
    if (size != ANS_HDR + 2 * nw) return ANS_E_CORRUPT;
    const uint8_t *words = in + ANS_HDR;
    uint64_t next = 0;
    for (uint32_t i = 0; i < n; i++) {
        const uint32_t lane = i % ANS_LANES;
        uint32_t v = x[lane];
        if (v < ANS_L) return ANS_E_CORRUPT;
        const uint32_t r = v & (ANS_M - 1);
        int s = 0;
        while (cum[s + 1] <= r) s++;  /* the symbol whose interval holds r */
        out[i] = (uint8_t)s;
        v = freq[s] * (v >> ANS_M_LOG) + r - cum[s];
        if (v < ANS_L) {
            if (next >= nw) return ANS_E_CORRUPT;
            v = (v << 16) | get16(words + 2 * next);
            next++;
        }
        x[lane] = v;
    }
    if (next != nw) return ANS_E_CORRUPT;
    for (uint32_t k = 0; k < ANS_LANES; k++)
        if (x[k] != ANS_L) return ANS_E_CORRUPT;  /* every state back at its start */
    return ANS_OK;
}

/* ------------------------------------------------------------ ACLE */

static uint64_t pad16(uint64_t v) { return (v + 15) & ~(uint64_t)15; }

/* The v1 container's sections: header + directory (raw), token array,
 * literal bytes.  Checks only what the split needs. */
static int v1_sections(const uint8_t *c, uint64_t n, uint64_t *prefix, uint64_t *n_tok, uint64_t *n_lit) {
    if (!c || n < 64 || memcmp(c, "ACLZ", 4) != 0) return ANS_E_CORRUPT;
    /* v1 header: ver u16 @4, flags u16 @6, total u64 @8, block size u32 @16,
     * n_blocks u32 @20, n_tokens u64 @24, n_literals u64 @32 */
    const uint64_t nb = get32(c + 20);
    *n_tok = get64(c + 24);
    *n_lit = get64(c + 32);
    *prefix = 64 + 32 * nb;
    if (*n_tok > n / 16 || *n_lit > n || *prefix + 16 * *n_tok + *n_lit != n) return ANS_E_CORRUPT;
    return ANS_OK;
}

/* Byte k of every token, or the literal bytes (stream 16). */
static void stream_bytes(const uint8_t *c, uint64_t prefix, uint64_t n_tok, int k, uint64_t off, uint32_t len,
                         uint8_t *dst) {
    if (k < 16) {
        const uint8_t *tok = c + prefix;
        for (uint32_t i = 0; i < len; i++) dst[i] = tok[16 * (off + i) + (uint64_t)k];
    } else {
        memcpy(dst, c + prefix + 16 * n_tok + off, len);
    }
}

static uint64_t n_tiles_of(uint64_t len) { return (len + ANS_TILE - 1) / ANS_TILE; }

/* Bytes an ACLE of the given v1 container can take at most. */
int oracle_acle_bound(const uint8_t *c, uint64_t n, uint64_t *out) {
    uint64_t prefix, n_tok, n_lit;
    int rc = v1_sections(c, n, &prefix, &n_tok, &n_lit);
    if (rc) return rc;
    const uint64_t tiles = 16 * n_tiles_of(n_tok) + n_tiles_of(n_lit);
    *out = ACLE_HDR + pad16(prefix) + 16 * ACLE_STREAMS + 16 * tiles +
           tiles * (pad16(ANS_HDR + 2 * (ANS_TILE + ANS_LANES)));
    return ANS_OK;
}

int oracle_acle_encode(const uint8_t *c, uint64_t n, uint8_t *out, uint64_t cap, uint64_t *size) {
    if (!out || !size) return ANS_E_INVAL;
    uint64_t prefix, n_tok, n_lit, bound;
    int rc = v1_sections(c, n, &prefix, &n_tok, &n_lit);
    if (rc) return rc;
    oracle_acle_bound(c, n, &bound);
    if (cap < bound) return ANS_E_CAPACITY;
    uint64_t len[ACLE_STREAMS], first[ACLE_STREAMS], tiles = 0;
    for (uint32_t k = 0; k < ACLE_STREAMS; k++) {
        len[k] = k < 16 ? n_tok : n_lit;
        first[k] = tiles;
        tiles += n_tiles_of(len[k]);
    }
    const uint64_t st_off = ACLE_HDR + pad16(prefix);
    const uint64_t tt_off = st_off + 16 * ACLE_STREAMS;
    const uint64_t pay_off = tt_off + 16 * tiles;
    memset(out, 0, pay_off);
    memcpy(out, "ACLE", 4);
    put32(out + 4, 1);
    put64(out + 8, n);
    put64(out + 16, prefix);
    put32(out + 24, ACLE_STREAMS);
    put32(out + 28, ANS_TILE);
    put64(out + 32, n_tok);
    put64(out + 40, n_lit);
    put64(out + 48, tiles);
    put64(out + 56, pay_off);
    memcpy(out + ACLE_HDR, c, prefix);
    uint8_t *buf = (uint8_t *)malloc(ANS_TILE);
    if (!buf) return ANS_E_NOMEM;
    uint64_t pos = 0, t = 0;
    for (uint32_t k = 0; k < ACLE_STREAMS; k++) {
        put64(out + st_off + 16 * k, len[k]);
        put64(out + st_off + 16 * k + 8, first[k]);
        for (uint64_t off = 0; off < len[k]; off += ANS_TILE, t++) {
            const uint32_t m = (uint32_t)(len[k] - off < ANS_TILE ? len[k] - off : ANS_TILE);
            stream_bytes(c, prefix, n_tok, (int)k, off, m, buf);
            uint64_t sz = 0;
            rc = oracle_ans_encode_tile(buf, m, out + pay_off + pos, cap - pay_off - pos, &sz);
            if (rc) { free(buf); return rc; }
            put64(out + tt_off + 16 * t, pos);
            put32(out + tt_off + 16 * t + 8, (uint32_t)sz);
            put32(out + tt_off + 16 * t + 12, m);
            const uint64_t next = pad16(pos + sz);
            memset(out + pay_off + pos + sz, 0, next - pos - sz);
            pos = next;
        }
    }
    free(buf);
    *size = pay_off + pos;
    return ANS_OK;
}

/* Size of the v1 container an ACLE decodes to (0 on a bad header). */
uint64_t oracle_acle_decoded_size(const uint8_t *e, uint64_t n) {
    if (!e || n < ACLE_HDR || memcmp(e, "ACLE", 4) != 0) return 0;
    return get64(e + 8);
}

int oracle_acle_decode(const uint8_t *e, uint64_t n, uint8_t *out, uint64_t cap) {
    if (!e || !out) return ANS_E_INVAL;
    if (n < ACLE_HDR || memcmp(e, "ACLE", 4) != 0 || get32(e + 4) != 1) return ANS_E_CORRUPT;
    const uint64_t size = get64(e + 8), prefix = get64(e + 16);
    const uint64_t n_tok = get64(e + 32), n_lit = get64(e + 40), tiles = get64(e + 48);
    const uint64_t pay_off = get64(e + 56);
    if (get32(e + 24) != ACLE_STREAMS || get32(e + 28) != ANS_TILE) return ANS_E_CORRUPT;
    if (cap < size) return ANS_E_CAPACITY;
    if (prefix + 16 * n_tok + n_lit != size || ACLE_HDR + prefix > n) return ANS_E_CORRUPT;
    const uint64_t st_off = ACLE_HDR + pad16(prefix), tt_off = st_off + 16 * ACLE_STREAMS;
    if (tt_off + 16 * tiles != pay_off || pay_off > n) return ANS_E_CORRUPT;
    memcpy(out, e + ACLE_HDR, prefix);
    uint8_t *buf = (uint8_t *)malloc(ANS_TILE);
    if (!buf) return ANS_E_NOMEM;
    int rc = ANS_OK;
    for (uint32_t k = 0; k < ACLE_STREAMS && rc == ANS_OK; k++) {
        const uint64_t len = get64(e + st_off + 16 * k), first = get64(e + st_off + 16 * k + 8);
        if (len != (k < 16 ? n_tok : n_lit) || first + n_tiles_of(len) > tiles) { rc = ANS_E_CORRUPT; break; }
        for (uint64_t off = 0, t = first; off < len; off += ANS_TILE, t++) {
            const uint64_t po = get64(e + tt_off + 16 * t);
            const uint32_t sz = get32(e + tt_off + 16 * t + 8), m = get32(e + tt_off + 16 * t + 12);
            if (m != (len - off < ANS_TILE ? len - off : ANS_TILE) || pay_off + po + sz > n) {
                rc = ANS_E_CORRUPT;
                break;
            }
            rc = oracle_ans_decode_tile(e + pay_off + po, sz, buf, m);
            if (rc) break;
            if (k < 16) {
                uint8_t *tok = out + prefix;
                for (uint32_t i = 0; i < m; i++) tok[16 * (off + i) + k] = buf[i];
            } else {
                memcpy(out + prefix + 16 * n_tok + off, buf, m);
            }
        }
    }
    free(buf);
    return rc;
}
