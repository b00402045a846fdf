// Host encoder of the tile entropy stage: the ACLE form of a v1 container
// (the layout and coder are those aclz_upload_acle decodes; see aclz.h).
//
// In the paper's pipeline an ANS stage works on 64 KB tiles on the GPU
// ahead of the match phase (Sec. II); no coder parameters are given.  Here
// each tile is coded on its own with order-0 rANS: the tile's byte counts
// are scaled to frequencies that sum to 2^12, 32 coder states share the
// tile (byte i on state i mod 32), and a state that would leave
// [2^16, 2^32) while coding gives up its low 16 bits as a word.  Tiles are
// independent, so they are coded in parallel on the host threads.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <thread>
#include <vector>

#include "aclz_internal.h"

using namespace aclz;

namespace {

constexpr uint32_t kTileBytes = 65536;
constexpr uint32_t kLanes = 32;
constexpr uint32_t kScaleBits = 12, kScale = 1u << kScaleBits;
constexpr uint32_t kStateLow = 1u << 16;
constexpr uint32_t kPayloadHeader = 2 * 256 + 4 * kLanes + 4;
constexpr uint32_t kStreamCount = 17;  // 16 token byte planes, then the literals

void put_le(uint8_t *p, uint64_t v, int bytes) {
    for (int k = 0; k < bytes; k++) p[k] = (uint8_t)(v >> (8 * k));
}
uint64_t round16(uint64_t v) { return (v + 15) & ~(uint64_t)15; }

// Frequencies of one tile: the only byte value takes all of 2^12; otherwise
// each present value gets max(1, floor(count * 2^12 / n)) and the difference
// to 2^12 goes to (or, one unit at a time, comes from) the largest frequency,
// the lowest byte value among equals.
void scale_counts(const uint32_t *count, uint32_t n, uint16_t *f) {
    std::fill(f, f + 256, (uint16_t)0);
    if (n == 0) return;
    int present = 0, last = 0;
    for (int s = 0; s < 256; s++)
        if (count[s]) { present++; last = s; }
    if (present == 1) {
        f[last] = (uint16_t)kScale;
        return;
    }
    uint32_t sum = 0;
    for (int s = 0; s < 256; s++) {
        if (!count[s]) continue;
        const uint32_t q = (uint32_t)(((uint64_t)count[s] << kScaleBits) / n);
        f[s] = (uint16_t)std::max<uint32_t>(q, 1);
        sum += f[s];
    }
    auto largest = [&]() { return (int)(std::max_element(f, f + 256) - f); };  // first of the maxima
    if (sum < kScale) f[largest()] = (uint16_t)(f[largest()] + (kScale - sum));
    for (; sum > kScale; sum--) f[largest()]--;
}

// One tile's payload: freq[256], the 32 final states, the word count and
// the words in the order the decoder takes them.
std::vector<uint8_t> code_tile(const uint8_t *src, uint32_t n) {
    uint32_t count[256] = {};
    for (uint32_t i = 0; i < n; i++) count[src[i]]++;
    uint16_t f[256];
    scale_counts(count, n, f);
    uint32_t start[256], acc = 0;
    for (int s = 0; s < 256; s++) { start[s] = acc; acc += f[s]; }
    uint32_t state[kLanes];
    std::fill(state, state + kLanes, kStateLow);
    std::vector<uint16_t> emitted;
    emitted.reserve(n / 2 + kLanes);
    // last byte first: the decoder runs forward and takes the words in reverse
    for (uint32_t i = n; i-- > 0;) {
        uint32_t &x = state[i % kLanes];
        const uint32_t s = src[i], fs = f[s];
        if ((uint64_t)x >= ((uint64_t)fs << 20)) {  // one word always brings x below the limit
            emitted.push_back((uint16_t)x);
            x >>= 16;
        }
        x = (x / fs) * kScale + (x % fs) + start[s];
    }
    std::vector<uint8_t> out(kPayloadHeader + 2 * emitted.size());
    for (int s = 0; s < 256; s++) put_le(out.data() + 2 * s, f[s], 2);
    for (uint32_t k = 0; k < kLanes; k++) put_le(out.data() + 512 + 4 * k, state[k], 4);
    put_le(out.data() + 512 + 4 * kLanes, emitted.size(), 4);
    uint8_t *w = out.data() + kPayloadHeader;
    for (size_t j = 0; j < emitted.size(); j++) put_le(w + 2 * j, emitted[emitted.size() - 1 - j], 2);
    return out;
}

struct Plan {
    View v;
    uint64_t prefix = 0;
    uint64_t len[kStreamCount] = {};
    uint64_t first[kStreamCount] = {};
    uint64_t tiles = 0;
};

int make_plan(const void *host_container, uint64_t n, Plan *pl) {
    if (!host_container) return ACLZ_E_INVAL;
    int rc = parse_container((const uint8_t *)host_container, n, &pl->v, true);
    if (rc) return rc;
    pl->prefix = 64 + 32 * (uint64_t)pl->v.n_blocks;
    for (uint32_t k = 0; k < kStreamCount; k++) {
        pl->len[k] = k < 16 ? pl->v.n_tokens : pl->v.n_literals;
        pl->first[k] = pl->tiles;
        pl->tiles += (pl->len[k] + kTileBytes - 1) / kTileBytes;
    }
    return ACLZ_OK;
}

uint64_t tables_end(const Plan &pl) { return 64 + round16(pl.prefix) + 16 * kStreamCount + 16 * pl.tiles; }

}  // namespace

extern "C" int aclz_acle_bound(const void *host_container, uint64_t n, uint64_t *out) {
    if (!out) return ACLZ_E_INVAL;
    Plan pl;
    int rc = make_plan(host_container, n, &pl);
    if (rc) return rc;
    uint64_t b = tables_end(pl);
    for (uint32_t k = 0; k < kStreamCount; k++)
        for (uint64_t off = 0; off < pl.len[k]; off += kTileBytes)
            b += round16(kPayloadHeader + 2 * std::min<uint64_t>(kTileBytes, pl.len[k] - off));
    *out = b;
    return ACLZ_OK;
}

extern "C" int aclz_acle_encode(const void *host_container, uint64_t n, int threads, void *host_out, uint64_t cap,
                                uint64_t *out_size) {
    if (!host_out || !out_size || threads < 0) return ACLZ_E_INVAL;
    Plan pl;
    int rc = make_plan(host_container, n, &pl);
    if (rc) return rc;
    const uint8_t *c = (const uint8_t *)host_container;
    const uint8_t *tok = c + pl.prefix, *lit = tok + 16 * pl.v.n_tokens;
    // tile t of stream k: (k, offset)
    std::vector<std::pair<uint32_t, uint64_t>> where;
    where.reserve(pl.tiles);
    for (uint32_t k = 0; k < kStreamCount; k++)
        for (uint64_t off = 0; off < pl.len[k]; off += kTileBytes) where.emplace_back(k, off);
    std::vector<std::vector<uint8_t>> pay(pl.tiles);
    std::atomic<uint64_t> next{0};
    auto work = [&]() {
        std::vector<uint8_t> buf(kTileBytes);
        for (uint64_t t; (t = next.fetch_add(1)) < pl.tiles;) {
            const uint32_t k = where[t].first;
            const uint64_t off = where[t].second;
            const uint32_t m = (uint32_t)std::min<uint64_t>(kTileBytes, pl.len[k] - off);
            if (k < 16) {
                for (uint32_t i = 0; i < m; i++) buf[i] = tok[16 * (off + i) + k];
            } else {
                std::memcpy(buf.data(), lit + off, m);
            }
            pay[t] = code_tile(buf.data(), m);
        }
    };
    unsigned nt = threads ? (unsigned)threads : std::max(1u, std::thread::hardware_concurrency());
    nt = (unsigned)std::min<uint64_t>(nt, std::max<uint64_t>(1, pl.tiles));
    std::vector<std::thread> pool;
    for (unsigned i = 1; i < nt; i++) pool.emplace_back(work);
    work();
    for (auto &th : pool) th.join();
    const uint64_t pay_off = tables_end(pl);
    uint64_t total = pay_off;
    for (const auto &p : pay) total += round16(p.size());
    if (cap < total) return ACLZ_E_CAPACITY;
    uint8_t *o = (uint8_t *)host_out;
    std::memset(o, 0, total);
    std::memcpy(o, "ACLE", 4);
    put_le(o + 4, 1, 4);
    put_le(o + 8, n, 8);
    put_le(o + 16, pl.prefix, 8);
    put_le(o + 24, kStreamCount, 4);
    put_le(o + 28, kTileBytes, 4);
    put_le(o + 32, pl.v.n_tokens, 8);
    put_le(o + 40, pl.v.n_literals, 8);
    put_le(o + 48, pl.tiles, 8);
    put_le(o + 56, pay_off, 8);
    std::memcpy(o + 64, c, pl.prefix);
    const uint64_t st = 64 + round16(pl.prefix), tt = st + 16 * kStreamCount;
    for (uint32_t k = 0; k < kStreamCount; k++) {
        put_le(o + st + 16 * k, pl.len[k], 8);
        put_le(o + st + 16 * k + 8, pl.first[k], 8);
    }
    uint64_t pos = 0;
    for (uint64_t t = 0; t < pl.tiles; t++) {
        const uint32_t k = where[t].first;
        const uint64_t m = std::min<uint64_t>(kTileBytes, pl.len[k] - where[t].second);
        put_le(o + tt + 16 * t, pos, 8);
        put_le(o + tt + 16 * t + 8, pay[t].size(), 4);
        put_le(o + tt + 16 * t + 12, m, 4);
        std::memcpy(o + pay_off + pos, pay[t].data(), pay[t].size());
        pos += round16(pay[t].size());
    }
    *out_size = total;
    return ACLZ_OK;
}
