// Tile entropy stage in front of the match phase (Sec. II places an ANS
// stage on 64 KB tiles, many in parallel, ahead of the match kernel).
//
// An ACLE container holds a v1 container's header and block directory raw
// and its 16 token byte planes and literal bytes as order-0 rANS tiles of
// 64 KiB: per tile a frequency table summing to 2^12, 32 interleaved coder
// states (byte i of the tile on state i mod 32) in [2^16, 2^32), and one
// stream of 16-bit renormalisation words, taken in increasing lane order
// within each step of 32 bytes.  One warp decodes one tile: lane k owns
// state k, a slot-to-symbol table of 4096 entries sits in shared memory, and
// every step writes 32 consecutive bytes.  The planes are then transposed
// into 16-byte tokens and the upload continues as for a v1 container.
#include <algorithm>
#include <cstring>
#include <vector>

#include "aclz_device.cuh"
#include "aclz_internal.h"

using namespace aclz;

namespace {

constexpr uint32_t kTile = 65536;
constexpr uint32_t kStreams = 17;
constexpr uint32_t kProbBits = 12, kProb = 1u << kProbBits;
constexpr uint32_t kStateLow = 1u << 16;
constexpr uint32_t kTileHeader = 512 + 4 * 32 + 4;  // freq[256], state[32], n_words
constexpr int kWarps = 8;                             // tiles per CTA
constexpr uint32_t kWarpSmem = 4096 + 512 + 512;      // slot table, freq[256], cum[256]

struct TileDesc {
    uint64_t payload;  // offset in the payload area
    uint64_t dst;      // offset in [planes | literals]
    uint32_t m;        // bytes in the tile
    uint32_t n_words;
    uint32_t pad[2];
};

uint32_t rd32le(const uint8_t *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
uint64_t rd64le(const uint8_t *p) { return (uint64_t)rd32le(p) | ((uint64_t)rd32le(p + 4) << 32); }

__global__ void __launch_bounds__(kWarps * 32) k_ans_tiles(const uint8_t *__restrict__ pay,
                                                          const TileDesc *__restrict__ td, uint64_t n_tiles,
                                                          uint8_t *planes, uint64_t plane_bytes, uint8_t *lits,
                                                          uint32_t *err) {
    extern __shared__ __align__(16) uint8_t sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t t = (uint64_t)blockIdx.x * kWarps + warp;
    if (t >= n_tiles) return;
    uint8_t *lut = sm + warp * kWarpSmem;
    uint16_t *freq = reinterpret_cast<uint16_t *>(lut + 4096);
    uint16_t *cum = freq + 256;
    const TileDesc d = td[t];
    const uint8_t *p = pay + d.payload;
    // frequencies: 8 per lane, cumulative by a warp scan
    const uint4 fv = __ldg(reinterpret_cast<const uint4 *>(p) + lane);
    const uint32_t fw[4] = {fv.x, fv.y, fv.z, fv.w};
    uint32_t f8[8], local = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        f8[k] = (fw[k >> 1] >> (16 * (k & 1))) & 0xffffu;
        local += f8[k];
    }
    uint32_t incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (d.m && total != kProb) {  // checked on the host; never index the table with a bad one
        if (lane == 0) atomicOr(err, kErrCorrupt);
        return;
    }
    uint32_t c = incl - local;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        freq[8 * lane + k] = (uint16_t)f8[k];
        cum[8 * lane + k] = (uint16_t)c;
        c += f8[k];
    }
    __syncwarp();
    // slot r -> the last symbol s with cum[s] <= r (its frequency is then > 0)
    if (d.m) {
        for (uint32_t r = lane; r < kProb; r += 32) {
            uint32_t lo = 0, hi = 255;
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (cum[mid] <= r) lo = mid; else hi = mid - 1;
            }
            lut[r] = (uint8_t)lo;
        }
    }
    __syncwarp();
    uint32_t x = __ldg(reinterpret_cast<const uint32_t *>(p + 512) + lane);  // little-endian
    const uint16_t *words = reinterpret_cast<const uint16_t *>(p + kTileHeader);
    uint8_t *out = d.dst < plane_bytes ? planes + d.dst : lits + (d.dst - plane_bytes);
    uint32_t next = 0;
    bool bad = x < kStateLow;
    for (uint32_t base = 0; base < d.m; base += 32) {
        const uint32_t i = base + (uint32_t)lane;
        const bool act = i < d.m && !bad;
        uint32_t y = x;
        if (act) {
            const uint32_t r = x & (kProb - 1);
            const uint32_t s = lut[r];
            out[i] = (uint8_t)s;
            y = (uint32_t)freq[s] * (x >> kProbBits) + r - cum[s];
        }
        const bool need = act && y < kStateLow;
        const unsigned bm = __ballot_sync(0xffffffffu, need);
        const uint32_t idx = next + (uint32_t)__popc(bm & ((1u << lane) - 1u));
        if (need) {
            if (idx < d.n_words) y = (y << 16) | (uint32_t)__ldg(words + idx);
            else bad = true;
        }
        next += (uint32_t)__popc(bm);
        x = y;
    }
    if (next != d.n_words || x != kStateLow) bad = true;  // every state back where encoding began
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(err, kErrCorrupt);
}

// 16 byte planes -> 16-byte tokens (byte k of token t is plane k, entry t).
__global__ void k_planes_to_tokens(const uint8_t *__restrict__ planes, uint64_t nt, uint4 *tok) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < nt; t += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
        for (int k = 0; k < 16; k++) w[k >> 2] |= (uint32_t)__ldg(planes + (uint64_t)k * nt + t) << (8 * (k & 3));
        tok[t] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

struct AcleCtx {
    const uint8_t *pay = nullptr;  // host payload area
    uint64_t pay_bytes = 0;
    std::vector<TileDesc> tiles;
    uint64_t plane_bytes = 0;
    cudaEvent_t ev_begin = nullptr, ev_end = nullptr;  // optional: around the tile decode
};

int fill_from_acle(aclz_handle *h, const View &v, const void *ctx, void *stream) {
    const AcleCtx &a = *static_cast<const AcleCtx *>(ctx);
    cudaStream_t st = (cudaStream_t)stream;
    uint8_t *d_pay = nullptr, *d_planes = nullptr;
    TileDesc *d_td = nullptr;
    uint32_t *d_err = nullptr;
    int rc = ACLZ_OK;
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == ACLZ_OK) {
            note_cuda_error(e);
            rc = e == cudaErrorMemoryAllocation ? ACLZ_E_NOMEM : ACLZ_E_CUDA;
        }
        return rc == ACLZ_OK;
    };
    const uint64_t nt = a.tiles.size();
    if (ck(cudaMalloc(&d_pay, a.pay_bytes ? a.pay_bytes : 16)) &&
        ck(cudaMalloc(&d_td, sizeof(TileDesc) * (nt ? nt : 1))) &&
        ck(cudaMalloc(&d_planes, a.plane_bytes ? a.plane_bytes : 16)) && ck(cudaMalloc(&d_err, 4)) &&
        ck(cudaMemsetAsync(d_err, 0, 4, st)) &&
        (!a.pay_bytes || ck(cudaMemcpyAsync(d_pay, a.pay, a.pay_bytes, cudaMemcpyHostToDevice, st))) &&
        (!nt || ck(cudaMemcpyAsync(d_td, a.tiles.data(), sizeof(TileDesc) * nt, cudaMemcpyHostToDevice, st)))) {
        if (a.ev_begin) ck(cudaEventRecord(a.ev_begin, st));
        if (nt) {
            const unsigned grid = (unsigned)((nt + kWarps - 1) / kWarps);
            k_ans_tiles<<<grid, kWarps * 32, kWarps * kWarpSmem, st>>>(d_pay, d_td, nt, d_planes, a.plane_bytes,
                                                                         h->d_lit, d_err);
            ck(cudaGetLastError());
        }
        if (rc == ACLZ_OK && v.n_tokens) {
            const unsigned grid = (unsigned)std::min<uint64_t>((v.n_tokens + 255) / 256, 65535u);
            k_planes_to_tokens<<<grid, 256, 0, st>>>(d_planes, v.n_tokens, (uint4 *)h->d_tok);
            ck(cudaGetLastError());
        }
        if (a.ev_end) ck(cudaEventRecord(a.ev_end, st));
        uint32_t err = 0;
        if (rc == ACLZ_OK && ck(cudaMemcpyAsync(&err, d_err, 4, cudaMemcpyDeviceToHost, st)) &&
            ck(cudaStreamSynchronize(st)) && err)
            rc = ACLZ_E_CORRUPT;
    }
    cudaStreamSynchronize(st);
    for (void *q : {(void *)d_pay, (void *)d_td, (void *)d_planes, (void *)d_err})
        if (q) cudaFree(q);
    return rc;
}

}  // namespace

extern "C" int aclz_upload_acle_ev(const void *host_buf, uint64_t n, uint32_t flags, void *stream, aclz_handle **out,
                                   void *ev_begin, void *ev_end) {
    if (!host_buf || !out) return ACLZ_E_INVAL;
    *out = nullptr;
    if (flags & ~(uint32_t)ACLZ_UPLOAD_FLATTEN) return ACLZ_E_INVAL;
    const uint8_t *e = static_cast<const uint8_t *>(host_buf);
    if (n < 64 || std::memcmp(e, "ACLE", 4) != 0 || rd32le(e + 4) != 1) return ACLZ_E_CORRUPT;
    const uint64_t size = rd64le(e + 8), prefix = rd64le(e + 16);
    const uint64_t n_tok = rd64le(e + 32), n_lit = rd64le(e + 40), n_tiles = rd64le(e + 48);
    const uint64_t pay_off = rd64le(e + 56);
    if (rd32le(e + 24) != kStreams || rd32le(e + 28) != kTile) return ACLZ_E_CORRUPT;
    if (prefix < 64 || prefix > n - 64 || n_tok > size / 16 || n_lit > size || prefix + 16 * n_tok + n_lit != size)
        return ACLZ_E_CORRUPT;
    // the raw v1 header and directory (tokens and literals come from the
    // tiles): the directory must lie inside the stored prefix before it is
    // walked, since the v1 size above only says what the fields claim
    if (64 + 32 * (uint64_t)rd32le(e + 64 + 20) != prefix) return ACLZ_E_CORRUPT;
    View v;
    int rc = parse_container(e + 64, size, &v, true);
    if (rc) return rc;
    if (64 + 32 * (uint64_t)v.n_blocks != prefix || v.n_tokens != n_tok || v.n_literals != n_lit)
        return ACLZ_E_CORRUPT;
    const uint64_t st_off = 64 + ((prefix + 15) & ~(uint64_t)15);
    const uint64_t tt_off = st_off + 16 * kStreams;
    if (tt_off > n || n_tiles > (n - tt_off) / 16 || tt_off + 16 * n_tiles != pay_off || pay_off > n)
        return ACLZ_E_CORRUPT;
    AcleCtx a;
    a.pay = e + pay_off;
    a.pay_bytes = n - pay_off;
    a.plane_bytes = 16 * n_tok;
    a.tiles.reserve(n_tiles);
    for (uint32_t k = 0; k < kStreams; k++) {
        const uint64_t len = rd64le(e + st_off + 16 * k), first = rd64le(e + st_off + 16 * k + 8);
        const uint64_t cnt = (len + kTile - 1) / kTile;
        if (len != (k < 16 ? n_tok : n_lit) || first != a.tiles.size() || first + cnt > n_tiles)
            return ACLZ_E_CORRUPT;
        for (uint64_t j = 0; j < cnt; j++) {
            const uint8_t *te = e + tt_off + 16 * (first + j);
            const uint64_t po = rd64le(te);
            const uint32_t sz = rd32le(te + 8), m = rd32le(te + 12);
            const uint64_t want = std::min<uint64_t>(kTile, len - j * kTile);
            if (m != want || po % 16 || sz < kTileHeader || po > a.pay_bytes || sz > a.pay_bytes - po)
                return ACLZ_E_CORRUPT;
            const uint8_t *tp = a.pay + po;
            uint32_t fsum = 0;
            for (int s = 0; s < 256; s++) fsum += (uint32_t)tp[2 * s] | ((uint32_t)tp[2 * s + 1] << 8);
            const uint32_t nw = rd32le(tp + 512 + 128);
            if (fsum != kProb || (uint64_t)kTileHeader + 2ull * nw != sz) return ACLZ_E_CORRUPT;
            TileDesc d{};
            d.payload = po;
            d.dst = (k < 16 ? (uint64_t)k * n_tok : 16 * n_tok) + j * kTile;
            d.m = m;
            d.n_words = nw;
            a.tiles.push_back(d);
        }
    }
    if (a.tiles.size() != n_tiles) return ACLZ_E_CORRUPT;
    a.ev_begin = (cudaEvent_t)ev_begin;
    a.ev_end = (cudaEvent_t)ev_end;
    return upload_view(v, flags, stream, fill_from_acle, &a, out);
}

extern "C" int aclz_upload_acle(const void *host_buf, uint64_t n, uint32_t flags, void *stream, aclz_handle **out) {
    return aclz_upload_acle_ev(host_buf, n, flags, stream, out, nullptr, nullptr);
}
