// Host side of libaclz: encoder parameters, the container writer (pack),
// the multi-threaded greedy encoder and host-side container parsing.
//
// The encoder is the paper's CPU-side producer of the format (Sec. II:
// block size fixed at encode time; Sec. IV-B: minimum match length by
// distance class; Sec. VI: encode is a CPU program with no speed claim).
// It never decodes; every decode step runs on the GPU.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

#include "aclz_internal.h"

using namespace aclz;

namespace {

const uint8_t kPresets[3][4] = {{6, 8, 10, 12}, {12, 16, 24, 32}, {16, 24, 32, 48}};
const uint32_t kBounds[3] = {128, 16384, 2097152};

inline int dclass(uint64_t d) {
    return d < kBounds[0] ? 0 : d < kBounds[1] ? 1 : d < kBounds[2] ? 2 : 3;
}

void write_header(uint8_t *c, uint64_t total, uint32_t bs, uint32_t nb, uint64_t nt, uint64_t nl,
                  const uint8_t mm[4]) {
    std::memset(c, 0, kHdr);
    c[0] = 'A'; c[1] = 'C'; c[2] = 'L'; c[3] = 'Z';
    wr16(c + 4, 1);
    wr16(c + 6, 0);
    wr64(c + 8, total);
    wr32(c + 16, bs);
    wr32(c + 20, nb);
    wr64(c + 24, nt);
    wr64(c + 32, nl);
    wr32(c + 40, 0);
    std::memcpy(c + 44, mm, 4);
    for (int i = 0; i < 3; i++) wr32(c + 48 + 4 * i, kBounds[i]);
}

int n_threads(int req) {
    if (req > 0) return req;
    unsigned h = std::thread::hardware_concurrency();
    return h ? (int)h : 1;
}

// Exact previous-occurrence links stored as u32 distances (0 = none):
// prev[p] = p - q for the largest q < p with the same 4-byte value, when
// p - q < 2^32.  Keys are split by hash across threads; each thread scans
// every position but only inserts its own keys, so no locking is needed.
bool build_prev(const uint8_t *x, uint64_t n, uint32_t *prev, int threads) {
    if (n < 4) return true;
    const uint64_t np = n - 3;
    std::atomic<bool> ok{true};
    auto work = [&](int t) {
        uint64_t cap = 1 << 16;
        std::vector<uint32_t> keys(cap);
        std::vector<uint64_t> last(cap, ~0ULL);
        uint64_t used = 0;
        for (uint64_t p = 0; p < np; p++) {
            uint32_t k;
            std::memcpy(&k, x + p, 4);
            uint64_t h = (uint64_t)k * 0x9E3779B97F4A7C15ULL;
            if ((int)((h >> 58) % (uint64_t)threads) != t) continue;
            uint64_t s = (h >> 20) & (cap - 1);
            while (last[s] != ~0ULL && keys[s] != k) s = (s + 1) & (cap - 1);
            if (last[s] == ~0ULL) {
                // a new key: stored with its position before any growth, so
                // the rehash carries it over
                keys[s] = k;
                last[s] = p;
                prev[p] = 0;
                if (++used * 2 > cap) {
                    // grow and rehash
                    uint64_t ncap = cap * 2;
                    std::vector<uint32_t> nk(ncap);
                    std::vector<uint64_t> nl(ncap, ~0ULL);
                    for (uint64_t i = 0; i < cap; i++) {
                        if (last[i] == ~0ULL) continue;
                        uint64_t hh = ((uint64_t)keys[i] * 0x9E3779B97F4A7C15ULL >> 20) & (ncap - 1);
                        while (nl[hh] != ~0ULL) hh = (hh + 1) & (ncap - 1);
                        nk[hh] = keys[i];
                        nl[hh] = last[i];
                    }
                    keys.swap(nk);
                    last.swap(nl);
                    cap = ncap;
                }
                continue;
            }
            const uint64_t d = p - last[s];
            prev[p] = d < (1ULL << 32) ? (uint32_t)d : 0;
            last[s] = p;
        }
    };
    std::vector<std::thread> ts;
    for (int t = 1; t < threads; t++) ts.emplace_back(work, t);
    work(0);
    for (auto &th : ts) th.join();
    return ok.load();
}

struct BlockOut {
    std::vector<uint32_t> ll, ml;
    std::vector<uint64_t> src;
    std::vector<uint8_t> lits;
};

void parse_block(const uint8_t *x, uint64_t n, uint64_t bstart, uint64_t bend, const uint8_t T[4],
                 const uint32_t *prev, uint32_t depth, uint64_t window, BlockOut &o) {
    o.ll.clear(); o.ml.clear(); o.src.clear(); o.lits.clear();
    uint64_t p = bstart, ls = bstart;
    while (p < bend) {
        uint64_t best = 0, bsrc = 0;
        if (p + 4 <= n) {
            uint64_t q = p;
            uint32_t seen = 0;
            while (seen < depth) {
                uint32_t dd = prev[q];
                if (!dd) break;
                if (p - (q - dd) > window) break;
                q -= dd;
                seen++;
                uint64_t d = p - q;
                uint64_t lim = std::min<uint64_t>(d, bend - p);
                uint64_t need = T[dclass(d)];
                if (lim < need || lim <= best) continue;
                // only a longer match replaces the best, so the byte at
                // offset best must agree (best < lim keeps it in range)
                if (best && x[q + best] != x[p + best]) continue;
                // compare 8 bytes at a time
                uint64_t len = 0;
                while (len + 8 <= lim) {
                    uint64_t a, b;
                    std::memcpy(&a, x + q + len, 8);
                    std::memcpy(&b, x + p + len, 8);
                    if (a != b) {
                        uint64_t diff = a ^ b;
                        len += (uint64_t)(__builtin_ctzll(diff) >> 3);
                        goto done;
                    }
                    len += 8;
                }
                while (len < lim && x[q + len] == x[p + len]) len++;
            done:
                if (len > lim) len = lim;
                if (len >= need && len > best) {
                    best = len;
                    bsrc = q;
                    if (best == bend - p) break;  // nothing can be longer
                }
            }
        }
        if (best) {
            o.ll.push_back((uint32_t)(p - ls));
            o.ml.push_back((uint32_t)best);
            o.src.push_back(bsrc);
            o.lits.insert(o.lits.end(), x + ls, x + p);
            p += best;
            ls = p;
        } else {
            p++;
        }
    }
    if (ls < bend || o.ll.empty()) {
        o.ll.push_back((uint32_t)(bend - ls));
        o.ml.push_back(0);
        o.src.push_back(0);
        o.lits.insert(o.lits.end(), x + ls, x + bend);
    }
}

}  // namespace

namespace aclz {

namespace {
std::atomic<int> g_last_cuda_error{0};
}

void note_cuda_error(int cuda_error_code) { g_last_cuda_error.store(cuda_error_code); }

int parse_container(const uint8_t *c, uint64_t n, View *v, bool check_directory) {
    if (!c || n < kHdr) return ACLZ_E_CORRUPT;
    if (c[0] != 'A' || c[1] != 'C' || c[2] != 'L' || c[3] != 'Z') return ACLZ_E_CORRUPT;
    if (rd16(c + 4) != 1) return ACLZ_E_CORRUPT;
    v->flags = rd16(c + 6);
    v->total_len = rd64(c + 8);
    v->block_size = rd32(c + 16);
    v->n_blocks = rd32(c + 20);
    v->n_tokens = rd64(c + 24);
    v->n_literals = rd64(c + 32);
    v->n_waves = rd32(c + 40);
    std::memcpy(v->mm, c + 44, 4);
    if (v->block_size == 0 || v->block_size % 16) return ACLZ_E_CORRUPT;
    if (v->total_len > kSrcMask) return ACLZ_E_CORRUPT;
    uint64_t nb = (v->total_len + v->block_size - 1) / v->block_size;
    if (nb != v->n_blocks) return ACLZ_E_CORRUPT;
    uint64_t need = kHdr + (uint64_t)kDirent * v->n_blocks;
    if (need > n) return ACLZ_E_CORRUPT;
    if (v->n_tokens > (n - need) / kTok) return ACLZ_E_CORRUPT;
    need += (uint64_t)kTok * v->n_tokens;
    if (v->n_literals != n - need) return ACLZ_E_CORRUPT;
    v->dir = c + kHdr;
    v->tok = v->dir + (uint64_t)kDirent * v->n_blocks;
    v->lit = v->tok + (uint64_t)kTok * v->n_tokens;
    if (check_directory) {
        uint64_t t = 0, l = 0;
        for (uint32_t b = 0; b < v->n_blocks; b++) {
            const uint8_t *d = v->dir + (uint64_t)kDirent * b;
            uint64_t to = rd64(d), lo = rd64(d + 8);
            uint32_t nt = rd32(d + 16);
            if (to != t || lo < l || lo > v->n_literals) return ACLZ_E_CORRUPT;
            if (nt == 0 || nt > v->block_size || to + nt > v->n_tokens) return ACLZ_E_CORRUPT;
            t = to + nt;
            l = lo;
        }
        if (t != v->n_tokens) return ACLZ_E_CORRUPT;
    }
    return ACLZ_OK;
}

}  // namespace aclz

extern "C" {

int aclz_encode_params_default(aclz_encode_params *p, int preset) {
    if (!p || preset < 0 || preset > 2) return ACLZ_E_INVAL;
    std::memset(p, 0, sizeof(*p));
    p->block_size = 65536;
    std::memcpy(p->min_match, kPresets[preset], 4);
    p->chain_depth = 64;
    p->window = ~0ULL;
    return ACLZ_OK;
}

uint64_t aclz_pack_bytes(uint64_t total_len, uint32_t block_size, uint64_t n_tokens,
                         uint64_t n_literals) {
    uint64_t nb = block_size ? (total_len + block_size - 1) / block_size : 0;
    return kHdr + (uint64_t)kDirent * nb + (uint64_t)kTok * n_tokens + n_literals;
}

uint64_t aclz_encode_bound(uint64_t n, uint32_t block_size) {
    uint64_t nb = block_size ? (n + block_size - 1) / block_size : 0;
    return aclz_pack_bytes(n, block_size, n / 4 + nb + 1, n);
}

int aclz_pack(uint64_t total_len, uint32_t block_size, const uint8_t min_match[4],
              const uint32_t *blk_ntok, const uint32_t *lit_len, const uint32_t *match_len,
              const uint64_t *src, uint64_t n_tokens, const uint8_t *literals,
              uint64_t n_literals, void *host_out, uint64_t cap, uint64_t *out_size) {
    if (!min_match || !host_out || !out_size || block_size == 0 || block_size % 16)
        return ACLZ_E_INVAL;
    if (total_len > kSrcMask) return ACLZ_E_INVAL;
    uint64_t nb = (total_len + block_size - 1) / block_size;
    if (nb > 0xffffffffULL) return ACLZ_E_INVAL;
    if (nb && (!blk_ntok || !lit_len || !match_len || !src)) return ACLZ_E_INVAL;
    if (n_literals && !literals) return ACLZ_E_INVAL;
    uint64_t need = aclz_pack_bytes(total_len, block_size, n_tokens, n_literals);
    if (cap < need) return ACLZ_E_CAPACITY;
    uint8_t *c = (uint8_t *)host_out;
    write_header(c, total_len, block_size, (uint32_t)nb, n_tokens, n_literals, min_match);
    uint8_t *dir = c + kHdr, *tok = dir + kDirent * nb, *lit = tok + kTok * n_tokens;
    uint64_t t = 0, l = 0;
    for (uint64_t b = 0; b < nb; b++) {
        uint8_t *d = dir + kDirent * b;
        std::memset(d, 0, kDirent);
        wr64(d, t);
        wr64(d + 8, l);
        wr32(d + 16, blk_ntok[b]);
        std::memcpy(d + 24, min_match, 4);
        for (uint32_t k = 0; k < blk_ntok[b]; k++, t++) {
            if (t >= n_tokens) return ACLZ_E_INVAL;
            uint8_t *p = tok + kTok * t;
            wr32(p, lit_len[t]);
            wr32(p + 4, match_len[t]);
            wr64(p + 8, match_len[t] ? (src[t] & kSrcMask) : 0);
            l += lit_len[t];
        }
    }
    if (t != n_tokens || l != n_literals) return ACLZ_E_INVAL;
    if (n_literals) std::memcpy(lit, literals, n_literals);
    *out_size = need;
    return ACLZ_OK;
}

int aclz_encode(const void *host_src, uint64_t n, const aclz_encode_params *p,
                const uint8_t *block_min_match, int threads, void *host_out, uint64_t cap,
                uint64_t *out_size) {
    if (!p || !host_out || !out_size || (n && !host_src)) return ACLZ_E_INVAL;
    if (!is_pow2(p->block_size) || p->block_size < kMinBlock || p->block_size > kMaxBlock)
        return ACLZ_E_INVAL;
    if (n > kSrcMask) return ACLZ_E_INVAL;
    for (int i = 0; i < 4; i++)
        if (p->min_match[i] < 4) return ACLZ_E_INVAL;
    const uint64_t bs = p->block_size;
    const uint64_t nb = (n + bs - 1) / bs;
    if (block_min_match)
        for (uint64_t i = 0; i < 4 * nb; i++)
            if (block_min_match[i] < 4) return ACLZ_E_INVAL;
    if (cap < aclz_encode_bound(n, p->block_size)) return ACLZ_E_CAPACITY;
    const uint8_t *x = (const uint8_t *)host_src;
    const int T = n_threads(threads);
    uint32_t *prev = nullptr;
    if (n >= 4) {
        prev = (uint32_t *)std::malloc(sizeof(uint32_t) * (n - 3));
        if (!prev) return ACLZ_E_NOMEM;
        build_prev(x, n, prev, std::min<int>(T, 64));
    }
    // parse blocks in parallel into per-thread batches of consecutive blocks
    const uint64_t batch = std::max<uint64_t>(1, std::min<uint64_t>(64, nb / (uint64_t)(4 * T) + 1));
    const uint64_t nbatch = (nb + batch - 1) / batch;
    std::vector<std::vector<BlockOut>> outs(nbatch);
    std::atomic<uint64_t> next{0};
    auto work = [&]() {
        BlockOut tmp;
        for (;;) {
            uint64_t k = next.fetch_add(1);
            if (k >= nbatch) break;
            auto &v = outs[k];
            uint64_t b0 = k * batch, b1 = std::min(nb, b0 + batch);
            v.resize(b1 - b0);
            for (uint64_t b = b0; b < b1; b++) {
                const uint8_t *Tm = block_min_match ? block_min_match + 4 * b : p->min_match;
                uint64_t s = b * bs, e = std::min(n, s + bs);
                parse_block(x, n, s, e, Tm, prev, p->chain_depth, p->window, v[b - b0]);
            }
        }
    };
    {
        std::vector<std::thread> ts;
        for (int t = 1; t < T; t++) ts.emplace_back(work);
        work();
        for (auto &th : ts) th.join();
    }
    std::free(prev);
    uint64_t nt = 0, nl = 0;
    for (auto &v : outs)
        for (auto &o : v) { nt += o.ll.size(); nl += o.lits.size(); }
    uint64_t need = aclz_pack_bytes(n, p->block_size, nt, nl);
    if (need > cap) return ACLZ_E_CAPACITY;
    uint8_t *c = (uint8_t *)host_out;
    write_header(c, n, p->block_size, (uint32_t)nb, nt, nl, p->min_match);
    uint8_t *dir = c + kHdr, *tok = dir + kDirent * nb, *lit = tok + kTok * nt;
    uint64_t t = 0, l = 0, b = 0;
    for (auto &v : outs) {
        for (auto &o : v) {
            uint8_t *d = dir + kDirent * b;
            std::memset(d, 0, kDirent);
            wr64(d, t);
            wr64(d + 8, l);
            wr32(d + 16, (uint32_t)o.ll.size());
            std::memcpy(d + 24, block_min_match ? block_min_match + 4 * b : p->min_match, 4);
            for (size_t k = 0; k < o.ll.size(); k++, t++) {
                uint8_t *q = tok + kTok * t;
                wr32(q, o.ll[k]);
                wr32(q + 4, o.ml[k]);
                wr64(q + 8, o.src[k]);
            }
            if (!o.lits.empty()) std::memcpy(lit + l, o.lits.data(), o.lits.size());
            l += o.lits.size();
            b++;
        }
    }
    *out_size = need;
    return ACLZ_OK;
}

int aclz_batch_merge(uint32_t n, const void *const *host_bufs, const uint64_t *sizes, void *host_out,
                     uint64_t cap, uint64_t *out_size, uint64_t *out_offsets) {
    if (n == 0 || !host_bufs || !sizes || !out_size || !out_offsets) return ACLZ_E_INVAL;
    std::vector<View> vs(n);
    uint32_t bs = 0;
    bool all_tags = true;
    uint32_t max_waves = 0;
    for (uint32_t i = 0; i < n; i++) {
        int rc = parse_container((const uint8_t *)host_bufs[i], sizes[i], &vs[i], true);
        if (rc) return rc;
        if (i == 0) bs = vs[i].block_size;
        if (vs[i].block_size != bs) return ACLZ_E_INVAL;
        if (!(vs[i].flags & kFlagWaves)) all_tags = false;
        max_waves = std::max(max_waves, vs[i].n_waves);
    }
    // sizes of the merged container
    uint64_t total = 0, nt = 0, nl = 0, nb = 0;
    std::vector<uint64_t> pad(n, 0);
    for (uint32_t i = 0; i < n; i++) {
        const View &v = vs[i];
        out_offsets[i] = total;
        if (v.total_len == 0) continue;
        pad[i] = (i + 1 < n && v.total_len % bs) ? bs - v.total_len % bs : 0;
        total += v.total_len + pad[i];
        nb += v.n_blocks;
        nt += v.n_tokens;
        nl += v.n_literals + pad[i];
        if (pad[i]) {
            // a padded block ending in a match gets one more token
            const uint8_t *last = v.tok + (uint64_t)kTok * (v.n_tokens - 1);
            if (rd32(last + 4) != 0) nt++;
        }
    }
    if (total > kSrcMask || nb > 0xffffffffULL) return ACLZ_E_UNSUPPORTED;
    const uint64_t need = aclz_pack_bytes(total, bs, nt, nl);
    if (!host_out) { *out_size = need; return ACLZ_OK; }
    if (cap < need) return ACLZ_E_CAPACITY;
    uint8_t *c = (uint8_t *)host_out;
    write_header(c, total, bs, (uint32_t)nb, nt, nl, vs[0].mm);
    uint8_t *dir = c + kHdr, *tok = dir + (uint64_t)kDirent * nb, *lit = tok + (uint64_t)kTok * nt;
    uint64_t b = 0, t = 0, l = 0;
    for (uint32_t i = 0; i < n; i++) {
        const View &v = vs[i];
        if (v.total_len == 0) continue;
        const uint64_t base = out_offsets[i];
        for (uint32_t k = 0; k < v.n_blocks; k++, b++) {
            const uint8_t *d = v.dir + (uint64_t)kDirent * k;
            uint8_t *o = dir + (uint64_t)kDirent * b;
            std::memcpy(o, d, kDirent);
            wr64(o, t);
            wr64(o + 8, l);
            const uint64_t t0 = rd64(d);
            uint32_t ntok = rd32(d + 16);
            const bool last_block = k + 1 == v.n_blocks;
            for (uint32_t j = 0; j < ntok; j++) {
                const uint8_t *src = v.tok + (uint64_t)kTok * (t0 + j);
                uint8_t *dt = tok + (uint64_t)kTok * t;
                std::memcpy(dt, src, kTok);
                const uint64_t sw = rd64(src + 8);
                if (rd32(src + 4)) wr64(dt + 8, ((sw & kSrcMask) + base) | (all_tags ? (sw & ~kSrcMask) : 0));
                else if (!all_tags) wr64(dt + 8, 0);
                t++;
            }
            // literal bytes of the block, in token order
            const uint64_t l0 = rd64(d + 8);
            const uint64_t l1 = k + 1 < v.n_blocks ? rd64(d + kDirent + 8) : v.n_literals;
            std::memcpy(lit + l, v.lit + l0, l1 - l0);
            l += l1 - l0;
            if (last_block && pad[i]) {
                uint8_t *lt = tok + (uint64_t)kTok * (t - 1);
                if (rd32(lt + 4) == 0) {
                    wr32(lt, rd32(lt) + (uint32_t)pad[i]);
                } else {
                    uint8_t *dt = tok + (uint64_t)kTok * t;
                    wr32(dt, (uint32_t)pad[i]);
                    wr32(dt + 4, 0);
                    wr64(dt + 8, 0);
                    t++;
                    ntok++;
                }
                std::memset(lit + l, 0, pad[i]);
                l += pad[i];
            }
            wr32(o + 16, ntok);
            if (!all_tags) wr16(o + 20, 0);
        }
    }
    if (all_tags) {
        wr16(c + 6, kFlagWaves);
        wr32(c + 40, nt ? std::max<uint32_t>(max_waves, 1) : 0);
    }
    *out_size = need;
    return (b == nb && t == nt && l == nl) ? ACLZ_OK : ACLZ_E_CORRUPT;
}

int aclz_container_info(const void *host_buf, uint64_t n, aclz_info *out) {
    if (!host_buf || !out) return ACLZ_E_INVAL;
    View v;
    int rc = parse_container((const uint8_t *)host_buf, n, &v, false);
    if (rc) return rc;
    std::memset(out, 0, sizeof(*out));
    out->total_len = v.total_len;
    out->n_tokens = v.n_tokens;
    out->n_literals = v.n_literals;
    out->block_size = v.block_size;
    out->n_blocks = v.n_blocks;
    out->n_waves = v.n_waves;
    out->flags = v.flags;
    std::memcpy(out->min_match, v.mm, 4);
    return ACLZ_OK;
}

int aclz_last_cuda_error(void) { return g_last_cuda_error.load(); }

const char *aclz_strerror(int code) {
    switch (code) {
        case ACLZ_OK: return "ok";
        case ACLZ_E_INVAL: return "invalid argument";
        case ACLZ_E_CORRUPT: return "corrupt container";
        case ACLZ_E_NOMEM: return "out of memory";
        case ACLZ_E_CAPACITY: return "buffer too small";
        case ACLZ_E_CUDA: return "CUDA runtime error";
        case ACLZ_E_TIMEOUT: return "bounded device wait ran out";
        case ACLZ_E_DEVICE: return "device-side error";
        case ACLZ_E_UNSUPPORTED: return "unsupported container";
        default: return "unknown error";
    }
}

}  // extern "C"
