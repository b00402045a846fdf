// Match-phase decode: the device-resident hot path.
//
// Wave 0 (k_wave0): one G-lane group per LZ block (Sec. II) walks the
// block's tokens G at a time, prefix-sums literal and match lengths into
// absolute output offsets, copies every literal run and every match whose
// source is already final in block order (tag 0), and writes each deferred
// match as a (dst, src, len) triplet into its wave's worklist.
//
// Waves w >= 1 (k_wave_copy): the worklist of wave w holds the matches
// whose sources became final in earlier waves (the wavefront of Sec. I),
// in block order.  Groups take contiguous ranges cut at block boundaries,
// and only matches of one block whose source overlaps an earlier match of
// the same block in the same pass are serialised.
//
// All copies go through group_copy: every lane owns one aligned 16-byte
// output chunk, so short matches from several tokens share one pass
// instead of leaving most of the group idle (the work-granularity
// mechanism of Sec. III-C).
#include <cstring>

#include "aclz_device.cuh"
#include "aclz_internal.h"

using namespace aclz;

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 4;

__device__ __forceinline__ uint64_t tri_dst(const uint4 t) { return (uint64_t)t.x | ((uint64_t)(t.y & 0xffu) << 32); }
__device__ __forceinline__ uint64_t tri_src(const uint4 t) { return (uint64_t)t.z | ((uint64_t)(t.w & 0xffu) << 32); }
__device__ __forceinline__ uint32_t tri_len(const uint4 t) { return t.w >> 8; }

template <int G>
__global__ void __launch_bounds__(kThreads) k_wave0(const uint4 *__restrict__ tok,
                                                    const uint8_t *__restrict__ lit,
                                                    const uint64_t *__restrict__ blk_tok,
                                                    const uint64_t *__restrict__ blk_lit,
                                                    const uint32_t *__restrict__ slot,
                                                    uint4 *__restrict__ tri, uint8_t *out, uint32_t nb,
                                                    uint32_t log2bs) {
    Group<G> g;
    const uint32_t b = (uint32_t)((blockIdx.x * (uint64_t)kThreads + threadIdx.x) / G);
    if (b >= nb) return;
    const uint64_t t0 = blk_tok[b], t1 = blk_tok[b + 1];
    uint64_t lbase = blk_lit[b];
    uint64_t pos = (uint64_t)b << log2bs;
    for (uint64_t w = t0; w < t1; w += G) {
        const uint64_t i = w + g.lane;
        const bool v = i < t1;
        const uint4 t = v ? __ldg(tok + i) : make_uint4(0, 0, 0, 0);
        const uint32_t ll = t.x, ml = t.y;
        const uint32_t tag = t.w >> 8;
        const uint64_t src = (uint64_t)t.z | ((uint64_t)(t.w & 0xffu) << 32);
        const uint32_t incl = g.scan_incl(ll + ml);
        const uint32_t lincl = g.scan_incl(ll);
        const uint64_t dl = pos + incl - (ll + ml);
        const uint64_t dm = dl + ll;
        const uint8_t *ls = lit + (lbase + lincl - ll);
        // literal runs: sources in the literal array, always independent
        group_copy<G, kUnroll>(g, out, dl, ls, ll);
        // deferred matches go to their wave's worklist
        if (v && ml && tag) {
            const uint32_t sl = __ldg(slot + i);
            tri[sl] = make_uint4((uint32_t)dm, (uint32_t)(dm >> 32), (uint32_t)src,
                                 (uint32_t)(src >> 32) | (ml << 8));
        }
        g.sync();
        // in-order matches, batched so no batch reads what it writes
        const bool m0 = v && ml && tag == 0;
        unsigned rem = g.ballot(m0);
        while (rem) {
            const int f = __ffs(rem) - 1;
            const uint64_t fd = g.shfl(dm, f);
            const bool dep = m0 && ((rem >> g.lane) & 1u) && g.lane > f && (src + ml > fd);
            const unsigned dmask = g.ballot(dep);
            const unsigned lim = dmask & (0u - dmask);
            const unsigned batch = lim ? (rem & (lim - 1u)) : rem;
            const bool mine = (batch >> g.lane) & 1u;
            group_copy<G, kUnroll>(g, out, dm, out + src, mine ? ml : 0u);
            g.sync();
            rem &= ~batch;
        }
        pos += g.shfl(incl, G - 1);
        lbase += g.shfl(lincl, G - 1);
    }
}

// Copy one wave's worklist.  Group k owns the segments (runs of one block)
// that start in [k*T, (k+1)*T); a segment crossing the range end is
// finished by the group that started it.
template <int G, int ITEMS>
__global__ void __launch_bounds__(kThreads) k_wave_copy(const uint4 *__restrict__ tri, uint64_t n,
                                                        uint8_t *out, uint32_t log2bs) {
    Group<G> g;
    constexpr uint64_t T = (uint64_t)G * ITEMS;
    const uint64_t gid = (blockIdx.x * (uint64_t)kThreads + threadIdx.x) / G;
    const uint64_t a = gid * T;
    if (a >= n) return;
    const uint64_t e = a + T < n ? a + T : n;
    // first segment start in [a, e)
    uint64_t s = ~0ULL;
    for (uint64_t w = a; w < e; w += G) {
        const uint64_t i = w + g.lane;
        bool st = false;
        if (i < e) {
            const uint64_t bi = tri_dst(__ldg(tri + i)) >> log2bs;
            st = (i == 0) || (bi != (tri_dst(__ldg(tri + i - 1)) >> log2bs));
        }
        const unsigned m = g.ballot(st);
        if (m) { s = w + (uint64_t)(__ffs(m) - 1); break; }
    }
    if (s == ~0ULL) return;
    for (uint64_t cur = s; cur < n; cur += G) {
        const uint64_t i = cur + g.lane;
        const bool v = i < n;
        const uint4 t = v ? __ldg(tri + i) : make_uint4(0, 0, 0, 0);
        const uint64_t d = tri_dst(t), sr = tri_src(t);
        const uint32_t len = v ? tri_len(t) : 0u;
        const uint64_t blk = d >> log2bs;
        uint64_t pblk = g.shfl_up(blk, 1);
        if (g.lane == 0) pblk = (i == s || i == 0) ? ~0ULL : (tri_dst(__ldg(tri + i - 1)) >> log2bs);
        const bool st = v && (i == s || blk != pblk);
        const unsigned stop = g.ballot(st && i >= e && i != s);
        unsigned act = g.ballot(v);
        if (stop) act &= (stop & (0u - stop)) - 1u;
        const unsigned S = g.ballot(st);
        unsigned rem = act;
        while (rem) {
            const int f = __ffs(rem) - 1;
            const unsigned upto = (g.lane == 31) ? 0xffffffffu : ((2u << g.lane) - 1u);
            const unsigned sm = (S | (1u << f)) & ~((1u << f) - 1u) & upto;
            const int fs = sm ? 31 - __clz(sm) : f;
            const uint64_t fsd = g.shfl(d, fs);
            const bool dep = ((rem >> g.lane) & 1u) && g.lane > fs && (sr + len > fsd);
            const unsigned dmask = g.ballot(dep);
            const unsigned lim = dmask & (0u - dmask);
            const unsigned batch = lim ? (rem & (lim - 1u)) : rem;
            const bool mine = (batch >> g.lane) & 1u;
            group_copy<G, kUnroll>(g, out, d, out + sr, mine ? len : 0u);
            g.sync();
            rem &= ~batch;
        }
        if (stop) break;
    }
}

template <int G>
int launch_waves(aclz_handle *h, uint8_t *out, cudaStream_t st) {
    constexpr int gpc = kThreads / G;  // groups per CTA
    const unsigned grid0 = (h->n_blocks + gpc - 1) / gpc;
    k_wave0<G><<<grid0, kThreads, 0, st>>>((const uint4 *)h->d_tok, h->d_lit, h->d_blk_tok,
                                            h->d_blk_lit, h->d_slot, (uint4 *)h->d_tri, out,
                                            h->n_blocks, h->log2_bs);
    constexpr int ITEMS = 2;
    for (uint32_t w = 1; w < h->n_waves; w++) {
        const uint64_t a = h->wave_start[w], n = h->wave_start[w + 1] - a;
        if (!n) continue;
        const uint64_t groups = (n + (uint64_t)G * ITEMS - 1) / ((uint64_t)G * ITEMS);
        const unsigned grid = (unsigned)((groups + gpc - 1) / gpc);
        k_wave_copy<G, ITEMS><<<grid, kThreads, 0, st>>>((const uint4 *)h->d_tri + a, n, out, h->log2_bs);
    }
    return cudaGetLastError() == cudaSuccess ? ACLZ_OK : ACLZ_E_CUDA;
}

}  // namespace

extern "C" int aclz_decode_all(aclz_handle *h, void *d_out, uint64_t cap, const aclz_decode_cfg *cfg,
                               void *stream) {
    if (!h || (!d_out && h->total_len)) return ACLZ_E_INVAL;
    if (cap < h->total_len) return ACLZ_E_CAPACITY;
    if (reinterpret_cast<uintptr_t>(d_out) & 15) return ACLZ_E_INVAL;
    aclz_decode_cfg c = {32, ACLZ_MODE_WAVES, 0, 0};
    if (cfg) c = *cfg;
    if (c.G != 8 && c.G != 16 && c.G != 32) return ACLZ_E_INVAL;
    if (c.mode != ACLZ_MODE_WAVES && c.mode != ACLZ_MODE_PERSISTENT) return ACLZ_E_INVAL;
    if (h->n_blocks == 0) return ACLZ_OK;
    cudaStream_t st = (cudaStream_t)stream;
    uint8_t *out = (uint8_t *)d_out;
    if (c.mode == ACLZ_MODE_PERSISTENT) return ACLZ_E_UNSUPPORTED;
    switch (c.G) {
        case 8: return launch_waves<8>(h, out, st);
        case 16: return launch_waves<16>(h, out, st);
        default: return launch_waves<32>(h, out, st);
    }
}

extern "C" int aclz_device_status(aclz_handle *h, void *stream) {
    if (!h) return ACLZ_E_INVAL;
    uint32_t e = 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&e, h->d_err, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return ACLZ_E_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return ACLZ_E_CUDA;
    if (e) {
        cudaMemsetAsync(h->d_err, 0, 4, st);
        cudaStreamSynchronize(st);
    }
    if (e & kErrTimeout) return ACLZ_E_TIMEOUT;
    if (e) return ACLZ_E_DEVICE;
    return ACLZ_OK;
}
