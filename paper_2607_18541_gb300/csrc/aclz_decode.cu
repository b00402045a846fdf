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
#include <algorithm>
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

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

constexpr uint32_t kSpinLimit = 1u << 22;  // bounded waits: ~0.3-1 s at most

// Spin (bounded) until *p >= v; returns false when the limit ran out or
// when another group already gave up (err has kErrTimeout), so one stuck
// wait ends the whole launch within about a second.
__device__ __forceinline__ bool wait_at_least(const uint32_t *p, uint32_t v, uint32_t *err) {
    uint32_t spins = 0;
    while (ld_acquire(p) < v) {
        if (++spins > kSpinLimit) {
            atomicOr(err, kErrTimeout);
            return false;
        }
        if ((spins & 255) == 0 && (*(volatile uint32_t *)err & kErrTimeout)) return false;
        __nanosleep(spins < 64 ? 32 : 256);
    }
    return true;
}

// Wave 0 of one block: scan, literal runs, in-order (tag 0) matches, and
// the deferred matches' triplets.
template <int G>
__device__ __forceinline__ void block_wave0(const Group<G> &g, uint32_t b, const uint4 *__restrict__ tok,
                                            const uint8_t *__restrict__ lit,
                                            const uint64_t *__restrict__ blk_tok,
                                            const uint64_t *__restrict__ blk_lit,
                                            const uint32_t *__restrict__ slot, uint4 *tri, uint8_t *out,
                                            uint32_t log2bs) {
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
            __stcg(tri + sl, make_uint4((uint32_t)dm, (uint32_t)(dm >> 32), (uint32_t)src,
                                        (uint32_t)(src >> 32) | (ml << 8)));
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
    block_wave0<G>(g, b, tok, lit, blk_tok, blk_lit, slot, tri, out, log2bs);
}

// One block's segment of wave w >= 1 inside the persistent decode: wait
// until every source block has finished the waves below w, then copy with
// same-block dependencies serialised.
template <int G>
__device__ __forceinline__ bool block_segment(const Group<G> &g, uint32_t b, uint32_t w,
                                              const uint4 *tri, uint64_t n, const uint32_t *prog,
                                              uint8_t *out, uint32_t log2bs, uint32_t *err) {
    bool ok = true;
    for (uint64_t cur = 0; cur < n; cur += G) {
        const uint64_t i = cur + g.lane;
        const bool v = i < n;
        const uint4 t = v ? __ldcg(tri + i) : make_uint4(0, 0, 0, 0);
        const uint64_t d = tri_dst(t), sr = tri_src(t);
        const uint32_t len = v ? tri_len(t) : 0u;
        if (v) {
            const uint64_t b0 = sr >> log2bs, b1 = (sr + len - 1) >> log2bs;
            for (uint64_t bb = b0; bb <= b1; bb++)
                if (bb != b && !wait_at_least(prog + bb, w, err)) ok = false;
        }
        g.sync();
        unsigned rem = g.ballot(v);
        while (rem) {
            const int f = __ffs(rem) - 1;
            const uint64_t fd = g.shfl(d, f);
            const bool dep = ((rem >> g.lane) & 1u) && g.lane > f && (sr + len > fd);
            const unsigned dmask = g.ballot(dep);
            const unsigned lim = dmask & (0u - dmask);
            const unsigned batch = lim ? (rem & (lim - 1u)) : rem;
            const bool mine = (batch >> g.lane) & 1u;
            group_copy<G, kUnroll>(g, out, d, out + sr, mine ? len : 0u);
            g.sync();
            rem &= ~batch;
        }
    }
    return ok;
}

// Persistent decode: one cooperative launch; group k takes items k,
// k + K, k + 2K, ... of the wave-major item list.  An item waits only for
// items earlier in that list (its own block's earlier waves, and earlier
// waves of the blocks its sources lie in), all groups are co-resident, and
// each group takes its items in increasing order, so every wait ends.
template <int G>
__global__ void __launch_bounds__(kThreads) k_persistent(const uint4 *__restrict__ items,
                                                         const uint32_t *__restrict__ next,
                                                         uint64_t n_items, uint32_t *prog,
                                                         const uint4 *__restrict__ tok,
                                                         const uint8_t *__restrict__ lit,
                                                         const uint64_t *__restrict__ blk_tok,
                                                         const uint64_t *__restrict__ blk_lit,
                                                         const uint32_t *__restrict__ slot, uint4 *tri,
                                                         uint8_t *out, uint32_t log2bs, uint32_t *err) {
    Group<G> g;
    const uint64_t gid = (blockIdx.x * (uint64_t)kThreads + threadIdx.x) / G;
    const uint64_t ng = (uint64_t)gridDim.x * (kThreads / G);
    bool ok = true;
    for (uint64_t it = gid; it < n_items; it += ng) {
        const uint4 item = __ldg(items + it);
        const uint32_t b = item.x, w = item.y;
        if (w == 0) {
            block_wave0<G>(g, b, tok, lit, blk_tok, blk_lit, slot, tri, out, log2bs);
        } else {
            if (g.lane == 0 && !wait_at_least(prog + b, w, err)) ok = false;
            g.sync();
            if (!block_segment<G>(g, b, w, tri + item.z, item.w, prog, out, log2bs, err)) ok = false;
        }
        __threadfence();
        g.sync();
        if (g.lane == 0) st_release(prog + b, __ldg(next + it));
    }
    if (g.ballot(!ok) && g.lane == 0) atomicOr(err, kErrTimeout);
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

template <int G>
int launch_persistent(aclz_handle *h, uint8_t *out, uint32_t ctas_per_sm, cudaStream_t st) {
    static int max_per_sm = -1, sms = 0;
    auto fn = k_persistent<G>;
    if (max_per_sm < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        int m = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, fn, kThreads, 0) != cudaSuccess) return ACLZ_E_CUDA;
        max_per_sm = m;
    }
    int per_sm = max_per_sm;
    if (ctas_per_sm && (int)ctas_per_sm < per_sm) per_sm = (int)ctas_per_sm;
    if (per_sm < 1) return ACLZ_E_UNSUPPORTED;
    uint64_t need = (h->n_items + (kThreads / G) - 1) / (kThreads / G);
    unsigned grid = (unsigned)std::min<uint64_t>((uint64_t)per_sm * sms, need ? need : 1);
    if (cudaMemsetAsync(h->d_prog, 0, 4 * (size_t)h->n_blocks, st) != cudaSuccess) return ACLZ_E_CUDA;
    const uint4 *items = (const uint4 *)h->d_items;
    const uint32_t *next = h->d_next;
    uint64_t n_items = h->n_items;
    uint32_t *prog = h->d_prog;
    const uint4 *tok = (const uint4 *)h->d_tok;
    const uint8_t *lit = h->d_lit;
    const uint64_t *bt = h->d_blk_tok, *bl = h->d_blk_lit;
    const uint32_t *slot = h->d_slot;
    uint4 *tri = (uint4 *)h->d_tri;
    uint32_t log2bs = h->log2_bs;
    uint32_t *err = h->d_err;
    void *args[] = {&items, &next, &n_items, &prog, &tok, &lit, &bt, &bl, &slot, &tri, &out, &log2bs, &err};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)fn, dim3(grid), dim3(kThreads), args, 0, st);
    return e == cudaSuccess ? ACLZ_OK : ACLZ_E_CUDA;
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
    if (c.mode == ACLZ_MODE_PERSISTENT) {
        switch (c.G) {
            case 8: return launch_persistent<8>(h, out, c.ctas_per_sm, st);
            case 16: return launch_persistent<16>(h, out, c.ctas_per_sm, st);
            default: return launch_persistent<32>(h, out, c.ctas_per_sm, st);
        }
    }
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
