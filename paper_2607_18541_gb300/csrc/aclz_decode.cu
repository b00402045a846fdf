// Match-phase decode: the device-resident hot path.
//
// Wave 0 (k_wave0): one G-lane group per LZ block (Sec. II) walks the
// block's tokens G at a time, prefix-sums literal and match lengths into
// absolute output offsets, copies every literal run and every match whose
// source is already final in block order (tag 0), and writes each deferred
// match as a (dst, src, len) triplet into its wave's worklist.
//
// Waves w >= 1 hold the matches whose sources become final only in earlier
// waves (the wavefront of Sec. I), block-ordered within each wave.  Two
// schedules run them:
//  - ACLZ_MODE_WAVES: one kernel per wave (k_wave_copy), kernel boundaries
//    as the wave barrier;
//  - ACLZ_MODE_PERSISTENT: one cooperative launch (k_ranges) over ranges of
//    consecutive (block, wave) segments in wave-major order, with bounded
//    waits on per-block completed-wave bits instead of wave barriers, so a
//    match is copied as soon as the blocks it reads have finished the waves
//    below its own.
//
// All copies are 16-byte vectorised with every lane owning aligned output
// chunks, so short matches from several tokens share one pass instead of
// leaving most of the group idle (the work-granularity mechanism of
// Sec. III-C); long matches in the persistent schedule are staged through
// shared memory by TMA bulk copies (cp.async.bulk + mbarrier).
#include <algorithm>
#include <cstring>
#include <mutex>

#include "aclz_device.cuh"
#include "aclz_internal.h"

using namespace aclz;

namespace {

constexpr int kThreads = 256;
// per-wave copy CTAs, and the CTAs of that size per SM the register cap
// is set for (the same 85 registers a thread as 3 x 256)
constexpr int kWaveThreads = 64, kWaveMinCtas = 768 / kWaveThreads;
// chunks per lane per round in the wave-0 pass: before per-wave copies
// (short matches; more resident warps without spills) and before the
// persistent schedule (long in-order matches)
constexpr int kUnrollWaveShort = 1, kUnrollWaveLong = 2;
constexpr int kUnrollCopy = 3;   // chunks per lane per round in per-wave match copies
constexpr int kUnrollRanges = 4; // the same in the persistent schedule's register copies
// staged (TMA) copies: jobs of at least kTmaMin bytes, pieces of <= kPiece
constexpr uint32_t kTmaMin = 192;
constexpr uint32_t kPiece = 2048;
constexpr uint32_t kSmemPerSm = 220u * 1024u;  // stage memory shared by the CTAs of one SM
// per-wave copies put full chunks first when deferred matches average
// at least this many bytes
constexpr double kFullFirstMin = 48.0;
// per-wave kernels are launched with programmatic stream serialization
constexpr int kWavePdl = 1;
// wave 0 reads literals through the non-coherent L1 path; before
// per-wave copies (short tokens) it also prefetches the next window's
// literal lines into L1 and the tokens two windows ahead into L2
constexpr bool kWave0Ro = true;

__device__ __forceinline__ uint64_t tri_dst(const uint4 t) { return (uint64_t)t.x | ((uint64_t)(t.y & 0xffu) << 32); }
__device__ __forceinline__ uint64_t tri_src(const uint4 t) { return (uint64_t)t.z | ((uint64_t)(t.w & 0xffu) << 32); }
__device__ __forceinline__ uint32_t tri_len(const uint4 t) { return t.w >> 8; }
// set at upload on the triplets of segments without an internal chain: a
// per-wave group may start or stop at any of them
__device__ __forceinline__ bool tri_cut(const uint4 t) { return (t.y >> 8) & 1u; }

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Programmatic dependent launch (per-wave kernels): a kernel lets the next
// kernel of its stream start once all of its CTAs have begun, and that
// kernel reads nothing the previous one writes before griddep_wait, which
// returns when the previous grid has completed and its writes are visible.
__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Bounded waits: spin_limit polls (sleeping up to 256 ns each) before a wait
// gives up.  The host scales it with the wave count, from 2^22 (about a
// second) to 2^26: a range deep in a long chain legitimately waits for most
// of the launch.  A wait also gives up when another group already gave up
// (err has kErrTimeout), so one stuck wait ends the whole launch.
constexpr uint32_t kSpinLimitMin = 1u << 22, kSpinLimitMax = 1u << 26;

// Spin (bounded) until every wave below w of one block is done: its done
// bits (ww 64-bit words, empty waves preset) are all set below bit w.
__device__ __forceinline__ bool wait_waves_below(const unsigned long long *done, uint32_t w, uint32_t *err,
                                                 uint32_t spin_limit) {
    for (uint32_t k = 0; k * 64 < w; k++) {
        const uint32_t nbits = w - k * 64;
        const unsigned long long want = nbits >= 64 ? ~0ULL : ((1ULL << nbits) - 1ULL);
        uint32_t spins = 0;
        while ((ld_acquire64(done + k) & want) != want) {
            if (++spins > spin_limit) {
                atomicOr(err, kErrTimeout);
                return false;
            }
            if ((spins & 255) == 0 && (*(volatile uint32_t *)err & kErrTimeout)) return false;
            __nanosleep(spins < 64 ? 32 : 256);
        }
    }
    return true;
}

// Exact same-wave dependencies inside one window of triplets (one per
// lane): bit j of the result is set when this lane's source overlaps the
// output of lane j < this lane.  Only matches of one block can depend on
// each other within a wave (a source in another block was final a wave
// earlier), so lanes whose source does not end in their own block skip the
// test.
template <int G>
__device__ __forceinline__ unsigned same_wave_deps(const Group<G> &g, bool v, uint64_t d, uint64_t sr,
                                                   uint32_t len, uint32_t log2bs) {
    const uint64_t blk = d >> log2bs;
    const bool local = v && ((sr + len - 1) >> log2bs) == blk;
    unsigned m = 0;
    if (!g.ballot(local)) return 0u;
    for (int j = 0; j < G; j++) {
        const uint64_t dj = g.shfl(d, j);
        const uint32_t nj = g.shfl(len, j);
        if (local && j < g.lane && nj && (dj >> log2bs) == blk && sr < dj + nj && dj < sr + len) m |= 1u << j;
    }
    return m;
}

// ------------------------------------------------------------- wave 0

// Wave 0 of one block: scan, literal runs, in-order (tag 0) matches, and
// the deferred matches' triplets.  The next window's tokens are loaded
// while the current window is copied.
template <int G, int UW, bool PF>
__device__ __forceinline__ void block_wave0(const Group<G> &g, uint32_t b, const uint4 *__restrict__ tok,
                                            const uint8_t *__restrict__ lit,
                                            const uint64_t *__restrict__ blk_tok,
                                            const uint64_t *__restrict__ blk_lit,
                                            const uint32_t *__restrict__ slot, uint4 *tri, uint8_t *out,
                                            uint32_t log2bs) {
    const uint64_t t0 = blk_tok[b], t1 = blk_tok[b + 1];
    uint64_t lbase = blk_lit[b];
    const uint64_t lend = blk_lit[b + 1];
    uint64_t pos = (uint64_t)b << log2bs;
    // the next window's tokens and worklist slots are loaded while the
    // current window is copied
    uint4 nt = t0 + g.lane < t1 ? __ldg(tok + t0 + g.lane) : make_uint4(0, 0, 0, 0);
    uint32_t ns = (tri && t0 + g.lane < t1) ? __ldg(slot + t0 + g.lane) : 0u;
    for (uint64_t w = t0; w < t1; w += G) {
        const uint64_t i = w + g.lane;
        const bool v = i < t1;
        const uint4 t = v ? nt : make_uint4(0, 0, 0, 0);
        const uint32_t sl = ns;
        if (w + G + g.lane < t1) {
            nt = __ldg(tok + w + G + g.lane);
            if (tri) ns = __ldg(slot + w + G + g.lane);
        }
        const uint32_t ll = t.x, ml = t.y;
        const uint32_t tag = t.w >> 8;
        const uint64_t src = (uint64_t)t.z | ((uint64_t)(t.w & 0xffu) << 32);
        const uint32_t incl = g.scan_incl(ll + ml);
        const uint32_t lincl = g.scan_incl(ll);
        const uint64_t dl = pos + incl - (ll + ml);
        const uint64_t dm = dl + ll;
        // deferred matches go to their wave's worklist
        if (tri && v && ml && tag) {
            __stcg(tri + sl, make_uint4((uint32_t)dm, (uint32_t)(dm >> 32), (uint32_t)src,
                                        (uint32_t)(src >> 32) | (ml << 8)));
        }
        // literal runs: sources in the literal array, always independent
        if (PF) {  // addresses inside this block's literals and tokens only
            const uint64_t nl = lbase + g.shfl(lincl, G - 1) + 128 * g.lane;
            if (g.lane < 2 && nl < lend) asm volatile("prefetch.global.L1 [%0];" ::"l"(lit + nl));
            const uint64_t nt2 = w + 2 * G + 8 * (g.lane - 4);
            if (g.lane >= 4 && g.lane < 8 && nt2 < t1) asm volatile("prefetch.global.L2 [%0];" ::"l"(tok + nt2));
        }
        group_copy<G, UW, false, kWave0Ro>(g, out, dl, lit + (lbase + lincl - ll), ll);
        g.sync();
        // in-order matches, batched so no batch reads what it writes: each
        // batch takes the lanes whose sources overlap no output of a lane
        // still to be copied (exact pairwise overlaps; the sources of
        // in-order matches lie in their own block)
        const bool m0 = v && ml && tag == 0;
        unsigned rem = g.ballot(m0);
        const unsigned deps0 = rem ? same_wave_deps<G>(g, m0, dm, src, ml, log2bs) & rem : 0u;
        while (rem) {
            const unsigned batch = g.ballot(((rem >> g.lane) & 1u) && (deps0 & rem) == 0u);
            const bool mine = (batch >> g.lane) & 1u;
            group_copy<G, UW>(g, out, dm, out + src, mine ? ml : 0u);
            g.sync();
            rem &= ~batch;
        }
        pos += g.shfl(incl, G - 1);
        lbase += g.shfl(lincl, G - 1);
    }
}

// Wave 0 of every block, one group per block.  With done non-null (the
// persistent schedule follows), each block's done bits start as its empty
// waves plus wave 0.
template <int G, int UW, bool PF>
__global__ void __launch_bounds__(kThreads, 3) k_wave0(const uint4 *__restrict__ tok,
                                                       const uint8_t *__restrict__ lit,
                                                       const uint64_t *__restrict__ blk_tok,
                                                       const uint64_t *__restrict__ blk_lit,
                                                       const uint32_t *__restrict__ slot,
                                                       uint4 *__restrict__ tri, uint8_t *out, uint32_t nb,
                                                       uint32_t log2bs, const uint64_t *__restrict__ pending,
                                                       uint64_t *done, uint32_t ww) {
    Group<G> g;
    griddep_launch_dependents();
    const uint32_t b = (uint32_t)((blockIdx.x * (uint64_t)kThreads + threadIdx.x) / G);
    if (b >= nb) return;
    block_wave0<G, UW, PF>(g, b, tok, lit, blk_tok, blk_lit, slot, tri, out, log2bs);
    if (done)
        for (uint32_t k = g.lane; k < ww; k += G)
            done[(uint64_t)b * ww + k] = ~__ldg(pending + (uint64_t)b * ww + k) | (k == 0 ? 1ULL : 0ULL);
}

// ------------------------------------------------ persistent schedule

// One look, without waiting, at whether every block of [sr, sr + len) has
// finished its waves below w (w <= 64, at most 4 blocks); acquire loads.
__device__ __forceinline__ bool waves_below_now(const unsigned long long *done, uint32_t ww, uint64_t sr,
                                                uint32_t len, uint32_t w, uint32_t log2bs) {
    if (w > 64) return false;
    const uint64_t b0 = sr >> log2bs, b1 = (sr + len - 1) >> log2bs;
    if (b1 - b0 > 3) return false;
    const unsigned long long want = w >= 64 ? ~0ULL : ((1ULL << w) - 1ULL);
    for (uint64_t bb = b0; bb <= b1; bb++)
        if ((ld_acquire64(done + bb * ww) & want) != want) return false;
    return true;
}

// Waves >= 1 in one cooperative launch, by ranges: range r holds the
// consecutive triplets [first, next range's first) of one wave.  Each match
// waits (bounded) until every block its source touches has finished its
// waves below w (per-block done bits; empty waves are preset); the range
// copies its matches window by window, in dependency levels within a
// window (a match that reads another's output of the same wave goes after
// it); then it marks bit w of each block it finished.  A segment (one
// block's matches of one wave) cut into several ranges is finished by the
// last of its ranges to end, found with a per-segment counter.  Ranges
// wait only for ranges of lower waves, earlier in the list; all groups are
// co-resident and take their ranges in increasing order (r, r + K, r + 2K,
// ...), so every wait ends.
// STAGED: matches of at least kTmaMin bytes go through the group's
// shared-memory stage by TMA bulk copies, and a group looks at its next
// range before releasing the current one: when that range's sources are
// already final, its first fill is issued at once, so the bulk copy runs
// while the current range's stores drain and its blocks are released.
// Otherwise all copies go through registers and the kernel runs at higher
// occupancy.
template <int G, bool STAGED>
__global__ void __launch_bounds__(kThreads, STAGED ? 2 : 3)
    k_ranges(const uint4 *__restrict__ ranges, uint64_t n_ranges, const uint4 *__restrict__ seg,
             const uint32_t *__restrict__ pieces, uint32_t *seg_cnt, unsigned long long *done, uint32_t ww,
             const uint4 *__restrict__ tri, uint8_t *out, uint32_t log2bs, uint32_t stage_bytes, uint32_t *err,
             uint32_t spin_limit) {
    extern __shared__ __align__(128) uint8_t smem[];
    Group<G> g;
    constexpr int kGroups = kThreads / G;
    Stage st;
    uint32_t piece = 0;
    if (STAGED) {
        const int gi = threadIdx.x / G;
        st.bar = reinterpret_cast<uint64_t *>(smem) + gi;
        st.buf = smem + 128 * ((8 * kGroups + 127) / 128) + (size_t)gi * stage_bytes;
        st.bytes = stage_bytes;
        st.phase = 0;
        if (g.lane == 0) mbar_init(st.bar, 1);
        fence_mbar_init();
        __syncthreads();
        piece = min(kPiece, stage_bytes - 32u);
    }
    const uint64_t gid = (blockIdx.x * (uint64_t)kThreads + threadIdx.x) / G;
    const uint64_t ng = (uint64_t)gridDim.x * kGroups;
    const uint4 z4 = make_uint4(0, 0, 0, 0);
    bool ok = true;
    // ranges[n_ranges] is a sentinel: the end of range r is ranges[r + 1].w.
    // Loaded ahead: the descriptor and first window of this group's next
    // range (rn, tn, nt2) and the descriptor of the one after (rn3, tn3).
    auto desc = [&](uint64_t k, uint4 &rd, uint32_t &te) {
        rd = k < n_ranges ? __ldg(ranges + k) : z4;
        te = k < n_ranges ? __ldg(ranges + k + 1).w : 0u;
    };
    uint4 rc, rn, rn3;
    uint32_t tc, tn, tn3;
    desc(gid, rc, tc);
    desc(gid + ng, rn, tn);
    uint4 nt = rc.w + g.lane < tc ? __ldg(tri + rc.w + g.lane) : z4;
    uint4 nt2 = rn.w + g.lane < tn ? __ldg(tri + rn.w + g.lane) : z4;
    Fill pre = {0, 0, 0, 0};
    bool pre_on = false;  // the first batch of range `it` has its first fill in flight
    for (uint64_t it = gid; it < n_ranges; it += ng) {
        const uint4 r = rc;
        const uint64_t t_begin = r.w, t_end = tc;
        desc(it + 2 * ng, rn3, tn3);
        const uint32_t w = r.x, s0 = r.y, s1 = r.z;
        const bool has_next = it + ng < n_ranges;
        for (uint64_t cur = t_begin; cur < t_end; cur += G) {
            const bool v = cur + g.lane < t_end;
            const uint4 t = v ? nt : z4;
            if (cur + G < t_end) nt = cur + G + g.lane < t_end ? __ldg(tri + cur + G + g.lane) : z4;
            const uint64_t d = tri_dst(t), sr = tri_src(t);
            const uint32_t len = v ? tri_len(t) : 0u;
            const bool ahead = pre_on && cur == t_begin;
            if (!ahead) {
                // every block the source touches (its own included) has
                // finished its waves below w
                if (v) {
                    const uint64_t b0 = sr >> log2bs, b1 = (sr + len - 1) >> log2bs;
                    for (uint64_t bb = b0; bb <= b1; bb++)
                        if (!wait_waves_below(done + bb * ww, w, err, spin_limit)) ok = false;
                }
                g.sync();
            }
            const unsigned deps = same_wave_deps<G>(g, v, d, sr, len, log2bs);
            unsigned rem = g.ballot(v);
            bool issued = ahead;
            while (rem) {
                const unsigned batch = g.ballot(((rem >> g.lane) & 1u) && (deps & rem) == 0u);
                const bool mine = (batch >> g.lane) & 1u;
                if (STAGED) {
                    if (!issued) fence_proxy_async_global();
                    const bool longj = mine && len >= kTmaMin;
                    group_copy<G, 2>(g, out, d, out + sr, (mine && !longj) ? len : 0u);
                    if (issued || g.ballot(longj)) {
                        if (!staged_copy_fills<G>(g, st, out, d, out + sr, longj ? len : 0u, piece, pre, issued,
                                                  err))
                            return;  // a bulk copy did not complete: no further copies into the stage
                    }
                } else {
                    group_copy<G, kUnrollRanges>(g, out, d, out + sr, mine ? len : 0u);
                }
                g.sync();
                rem &= ~batch;
                issued = false;
            }
        }
        pre_on = false;
        // a look at the next range of this group: when the sources of its
        // first window are final already, its first fill is issued now, so
        // the bulk copy runs while this range's stores drain and its blocks
        // are released
        if (STAGED && has_next && g.ballot(!ok) == 0u) {
            const bool v2 = rn.w + g.lane < tn;
            const uint64_t d2 = tri_dst(nt2), s2 = tri_src(nt2);
            const uint32_t n2 = v2 ? tri_len(nt2) : 0u;
            const bool ready = !v2 || waves_below_now(done, ww, s2, n2, rn.x, log2bs);
            if (g.ballot(!ready) == 0u) {
                const unsigned deps2 = same_wave_deps<G>(g, v2, d2, s2, n2, log2bs);
                const unsigned all2 = g.ballot(v2);
                const bool long2 = v2 && n2 >= kTmaMin && (deps2 & all2) == 0u;
                if (g.ballot(long2)) {
                    fence_proxy_async_global();
                    pre.done = 0;
                    fill_issue<G>(g, st, out + s2, long2 ? n2 : 0u, piece, pre);
                    pre_on = true;
                }
            }
        }
        // release: this range's writes, then bit w of every block it
        // finished (of a shared segment, only the last range to end)
        __threadfence();
        g.sync();
        const unsigned long long bit = 1ULL << (w % 64);
        for (uint32_t k = s0 + g.lane; k < s1; k += G) {
            const uint64_t word = (uint64_t)__ldg(seg + k).x * ww + w / 64;
            const uint32_t pc = __ldg(pieces + k);
            if (pc > 1) {
                if (atomicAdd(seg_cnt + k, 1u) != pc - 1) continue;
                seg_cnt[k] = 0;  // the last range of the segment resets the count for the next decode
                __threadfence();
            }
            atomicOr(done + word, bit);
        }
        // shift the loaded-ahead state by one range
        nt = nt2;
        rc = rn;
        tc = tn;
        rn = rn3;
        tn = tn3;
        nt2 = rn.w + g.lane < tn ? __ldg(tri + rn.w + g.lane) : z4;
    }
    if (!ok) atomicOr(err, kErrTimeout);
}

// ------------------------------------------------------ wave schedule

// Copy one wave's worklist.  Group k owns the segments (runs of one block)
// that start in [k*T, (k+1)*T); a segment crossing the range end is
// finished by the group that started it.  FULL_FIRST: the matches' full
// 16-byte chunks are copied before their partial ones (for matches of
// several chunks); otherwise chunks go in match order.
template <int G, int ITEMS, bool FULL_FIRST>
__global__ void __launch_bounds__(kWaveThreads, kWaveMinCtas) k_wave_copy(const uint4 *__restrict__ tri, uint64_t n,
                                                        uint8_t *out, uint32_t log2bs) {
    Group<G> g;
    constexpr uint64_t T = (uint64_t)G * ITEMS;
    griddep_launch_dependents();
    const uint64_t gid = (blockIdx.x * (uint64_t)kWaveThreads + threadIdx.x) / G;
    const uint64_t a = gid * T;
    if (a >= n) return;
    const uint64_t e = a + T < n ? a + T : n;
    // first cut point in [a, e): a segment start, or any triplet of a
    // segment without an internal chain
    uint64_t s = ~0ULL;
    for (uint64_t w = a; w < e; w += G) {
        const uint64_t i = w + g.lane;
        bool st = false;
        if (i < e) {
            const uint4 ti = __ldg(tri + i);
            const uint64_t bi = tri_dst(ti) >> log2bs;
            st = (i == 0) || tri_cut(ti) || (bi != (tri_dst(__ldg(tri + i - 1)) >> log2bs));
        }
        const unsigned m = g.ballot(st);
        if (m) { s = w + (uint64_t)(__ffs(m) - 1); break; }
    }
    if (s == ~0ULL) return;
    // the next window's triplets are loaded while the current one is copied;
    // lane 0 takes the block of the triplet before its window from the last
    // lane of the previous window (every lane of which was valid)
    uint4 nt = s + g.lane < n ? __ldg(tri + s + g.lane) : make_uint4(0, 0, 0, 0);
    uint64_t prev_blk = ~0ULL;
    // the worklist was written at upload; the sources, by earlier waves
    griddep_wait();
    for (uint64_t cur = s; cur < n; cur += G) {
        const uint64_t i = cur + g.lane;
        const bool v = i < n;
        const uint4 t = v ? nt : make_uint4(0, 0, 0, 0);
        if (cur + G + g.lane < n) nt = __ldg(tri + cur + G + g.lane);
        const uint64_t d = tri_dst(t), sr = tri_src(t);
        const uint32_t len = v ? tri_len(t) : 0u;
        const uint64_t blk = d >> log2bs;
        uint64_t pblk = g.shfl_up(blk, 1);
        if (g.lane == 0) pblk = (i == s) ? ~0ULL : prev_blk;
        prev_blk = g.shfl(blk, G - 1);
        const bool st = v && (i == s || blk != pblk || tri_cut(t));
        const unsigned stop = g.ballot(st && i >= e && i != s);
        unsigned act = g.ballot(v);
        if (stop) act &= (stop & (0u - stop)) - 1u;
        // exact same-wave dependencies inside the window (only sources that
        // end in their own block can have any); each batch takes the lanes
        // whose dependencies are all copied
        const unsigned deps = same_wave_deps<G>(g, (act >> g.lane) & 1u, d, sr, len, log2bs) & act;
        unsigned rem = act;
        while (rem) {
            const unsigned batch = g.ballot(((rem >> g.lane) & 1u) && (deps & rem) == 0u);
            const bool mine = (batch >> g.lane) & 1u;
            if (FULL_FIRST)
                group_copy_full_first<G, kUnrollCopy>(g, out, d, out + sr, mine ? len : 0u);
            else
                group_copy<G, kUnrollCopy>(g, out, d, out + sr, mine ? len : 0u);
            g.sync();
            rem &= ~batch;
        }
        if (stop) break;
    }
}

template <int G>
int launch_waves(aclz_handle *h, uint8_t *out, cudaStream_t st, cudaEvent_t phase) {
    constexpr int gpc = kThreads / G;  // groups per CTA
    const unsigned grid0 = (h->n_blocks + gpc - 1) / gpc;
    k_wave0<G, kUnrollWaveShort, true><<<grid0, kThreads, 0, st>>>((const uint4 *)h->d_tok, h->d_lit, h->d_blk_tok,
                                                              h->d_blk_lit, h->d_slot, nullptr, out,
                                                              h->n_blocks, h->log2_bs, nullptr, nullptr, 0);
    if (phase) cudaEventRecord(phase, st);
    // one window of G triplets per group: the most resident groups per wave
    constexpr int ITEMS = 1;
    // deferred matches of three or more 16-byte chunks on average: full
    // chunks first
    const bool ff = h->mean_deferred_len >= (double)kFullFirstMin;
    for (uint32_t w = 1; w < h->n_waves; w++) {
        const uint64_t a = h->wave_start[w], n = h->wave_start[w + 1] - a;
        if (!n) continue;
        const uint64_t per = (uint64_t)G * ITEMS;
        const uint64_t groups = (n + per - 1) / per;
        constexpr int gpcw = kWaveThreads / G;
        const unsigned grid = (unsigned)((groups + gpcw - 1) / gpcw);
        const uint4 *t = (const uint4 *)h->d_tri + a;
        auto k = ff ? k_wave_copy<G, ITEMS, true> : k_wave_copy<G, ITEMS, false>;
        // programmatic stream serialization: this wave's CTAs may start (and
        // load their worklist) while the previous kernel's last CTAs finish
        cudaLaunchConfig_t lc = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = kWavePdl;
        lc.gridDim = dim3(grid);
        lc.blockDim = dim3(kWaveThreads);
        lc.dynamicSmemBytes = 0;
        lc.stream = st;
        lc.attrs = at;
        lc.numAttrs = 1;
        uint32_t lb = h->log2_bs;
        if (cudaError_t e = cudaLaunchKernelEx(&lc, k, t, n, out, lb); e != cudaSuccess) {
            note_cuda_error(e);
            return ACLZ_E_CUDA;
        }
    }
    if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) {
        note_cuda_error(e);
        return ACLZ_E_CUDA;
    }
    return ACLZ_OK;
}

struct Occ {
    int per_sm = 0;
    uint32_t stage_bytes = 0;
    size_t smem = 0;
};

// Dynamic shared memory limit last set on each staged kernel instance.
template <int G, bool STAGED>
size_t &smem_attr() {
    static size_t v = 0;
    return v;
}

// Persistent mode: the wave-0 kernel (no dependencies) initialises the
// per-block done bits, then one cooperative launch runs every range of
// waves >= 1.
template <int G, bool STAGED>
int launch_persistent(aclz_handle *h, uint8_t *out, uint32_t ctas_per_sm, cudaStream_t st, cudaEvent_t phase) {
    constexpr int gpc = kThreads / G;
    const unsigned grid0 = (h->n_blocks + gpc - 1) / gpc;
    k_wave0<G, kUnrollWaveLong, false><<<grid0, kThreads, 0, st>>>((const uint4 *)h->d_tok, h->d_lit, h->d_blk_tok,
                                                             h->d_blk_lit, h->d_slot, nullptr, out,
                                                             h->n_blocks, h->log2_bs, h->d_pending, h->d_done,
                                                             h->n_wave_words);
    if (phase) cudaEventRecord(phase, st);
    if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) {
        note_cuda_error(e);
        return ACLZ_E_CUDA;
    }
    if (!h->n_ranges) return ACLZ_OK;
    auto fn = k_ranges<G, STAGED>;
    static int sms = 0;
    static Occ occ[5][33];  // [ctas_per_sm request 0..4][G]
    // the occupancy cache and the kernel's shared-memory attribute are
    // process-wide: host threads take turns from the lookup to the launch
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    const uint32_t req = std::min<uint32_t>(ctas_per_sm, 4);
    Occ &o = occ[req][G];
    if (!o.per_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (STAGED) {
            cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
            const uint32_t cps = req ? req : 1;
            const size_t bar = 128 * ((8 * gpc + 127) / 128);
            o.stage_bytes = (uint32_t)(((kSmemPerSm / cps - bar) / gpc) & ~127u);
            o.smem = bar + (size_t)gpc * o.stage_bytes;
            if (cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)o.smem);
                e != cudaSuccess) {
                note_cuda_error(e);
                return ACLZ_E_CUDA;
            }
            smem_attr<G, STAGED>() = o.smem;
        }
        int m = 0;
        if (cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, fn, kThreads, o.smem);
            e != cudaSuccess) {
            note_cuda_error(e);
            return ACLZ_E_CUDA;
        }
        if (!STAGED && req && (int)req < m) m = (int)req;
        o.per_sm = m > 0 ? m : -1;
    }
    if (o.per_sm < 1) return ACLZ_E_UNSUPPORTED;
    if (STAGED && smem_attr<G, STAGED>() != o.smem) {
        if (cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)o.smem);
            e != cudaSuccess) {
            note_cuda_error(e);
            return ACLZ_E_CUDA;
        }
        smem_attr<G, STAGED>() = o.smem;
    }
    const uint64_t need = (h->n_ranges + gpc - 1) / gpc;
    unsigned grid = (unsigned)std::min<uint64_t>((uint64_t)o.per_sm * sms, need ? need : 1);
    const uint4 *ranges = (const uint4 *)h->d_ranges;
    uint64_t n_ranges = h->n_ranges;
    const uint4 *seg = (const uint4 *)h->d_seg;
    const uint32_t *pieces = h->d_seg_pieces;
    uint32_t *seg_cnt = h->d_seg_cnt;
    unsigned long long *done = (unsigned long long *)h->d_done;
    uint32_t ww = h->n_wave_words;
    const uint4 *tri = (const uint4 *)h->d_tri;
    uint32_t log2bs = h->log2_bs;
    uint32_t sb = o.stage_bytes;
    uint32_t *err = h->d_err;
    uint32_t spin_limit =
        (uint32_t)std::min<uint64_t>(kSpinLimitMax, (uint64_t)kSpinLimitMin * std::max<uint32_t>(1u, h->n_waves / 256));
    void *args[] = {&ranges, &n_ranges, &seg, &pieces, &seg_cnt, &done, &ww, &tri, &out, &log2bs, &sb, &err, &spin_limit};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)fn, dim3(grid), dim3(kThreads), args, o.smem, st);
    if (e == cudaErrorCooperativeLaunchTooLarge && o.per_sm > 1) {
        // fewer co-resident CTAs than the occupancy estimate: one per SM
        cudaGetLastError();
        o.per_sm = 1;
        grid = (unsigned)std::min<uint64_t>((uint64_t)sms, need ? need : 1);
        e = cudaLaunchCooperativeKernel((const void *)fn, dim3(grid), dim3(kThreads), args, o.smem, st);
    }
    if (e != cudaSuccess) {
        note_cuda_error(e);
        return ACLZ_E_CUDA;
    }
    return ACLZ_OK;
}

template <int G>
int launch_persistent_auto(aclz_handle *h, uint8_t *out, const aclz_decode_cfg &c, cudaStream_t st,
                           cudaEvent_t phase) {
    bool staged = h->mean_deferred_len >= (double)kTmaMin;
    if (c.flags & ACLZ_FLAG_STAGED) staged = true;
    if (c.flags & ACLZ_FLAG_REGISTERS) staged = false;
    return staged ? launch_persistent<G, true>(h, out, c.ctas_per_sm, st, phase)
                  : launch_persistent<G, false>(h, out, c.ctas_per_sm, st, phase);
}

}  // namespace

namespace {

// Checks cfg and resolves ACLZ_MODE_AUTO for this handle.
int resolve_cfg(const aclz_handle *h, const aclz_decode_cfg *cfg, aclz_decode_cfg &c) {
    c = {32, ACLZ_MODE_AUTO, 0, 0};
    if (cfg) c = *cfg;
    if (c.G != 8 && c.G != 16 && c.G != 32) return ACLZ_E_INVAL;
    if (c.mode != ACLZ_MODE_WAVES && c.mode != ACLZ_MODE_PERSISTENT && c.mode != ACLZ_MODE_AUTO)
        return ACLZ_E_INVAL;
    if (c.mode == ACLZ_MODE_AUTO) {
        // long deferred matches: one persistent launch with TMA staging;
        // short ones: the per-wave kernels
        c.mode = h->mean_deferred_len >= (double)kTmaMin ? ACLZ_MODE_PERSISTENT : ACLZ_MODE_WAVES;
        if (c.mode == ACLZ_MODE_PERSISTENT && !(c.flags & ACLZ_FLAG_REGISTERS)) c.flags |= ACLZ_FLAG_STAGED;
    }
    if ((c.flags & ACLZ_FLAG_STAGED) && (c.flags & ACLZ_FLAG_REGISTERS)) return ACLZ_E_INVAL;
    if (c.mode == ACLZ_MODE_PERSISTENT && !(c.flags & (ACLZ_FLAG_STAGED | ACLZ_FLAG_REGISTERS)))
        c.flags |= h->mean_deferred_len >= (double)kTmaMin ? ACLZ_FLAG_STAGED : ACLZ_FLAG_REGISTERS;
    return ACLZ_OK;
}

}  // namespace

extern "C" int aclz_decode_plan(const aclz_handle *h, const aclz_decode_cfg *cfg, aclz_decode_cfg *resolved,
                                uint32_t *launches) {
    if (!h) return ACLZ_E_INVAL;
    aclz_decode_cfg c;
    if (int rc = resolve_cfg(h, cfg, c)) return rc;
    uint32_t n = 0;
    if (h->n_blocks) {
        n = 1;
        if (c.mode == ACLZ_MODE_PERSISTENT) {
            n += h->n_ranges ? 1 : 0;
        } else {
            for (uint32_t w = 1; w < h->n_waves; w++) n += h->wave_start[w + 1] > h->wave_start[w];
        }
    }
    if (resolved) *resolved = c;
    if (launches) *launches = n;
    return ACLZ_OK;
}

extern "C" int aclz_decode_all_ev(aclz_handle *h, void *d_out, uint64_t cap, const aclz_decode_cfg *cfg,
                                  void *stream, void *phase_event) {
    if (!h || (!d_out && h->total_len)) return ACLZ_E_INVAL;
    if (cap < h->total_len) return ACLZ_E_CAPACITY;
    if (reinterpret_cast<uintptr_t>(d_out) & 15) return ACLZ_E_INVAL;
    aclz_decode_cfg c;
    if (int rc = resolve_cfg(h, cfg, c)) return rc;
    if (h->n_blocks == 0) return ACLZ_OK;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t ev = (cudaEvent_t)phase_event;
    uint8_t *out = (uint8_t *)d_out;
    if (c.mode == ACLZ_MODE_PERSISTENT) {
        switch (c.G) {
            case 8: return launch_persistent_auto<8>(h, out, c, st, ev);
            case 16: return launch_persistent_auto<16>(h, out, c, st, ev);
            default: return launch_persistent_auto<32>(h, out, c, st, ev);
        }
    }
    switch (c.G) {
        case 8: return launch_waves<8>(h, out, st, ev);
        case 16: return launch_waves<16>(h, out, st, ev);
        default: return launch_waves<32>(h, out, st, ev);
    }
}

extern "C" int aclz_decode_all(aclz_handle *h, void *d_out, uint64_t cap, const aclz_decode_cfg *cfg,
                               void *stream) {
    return aclz_decode_all_ev(h, d_out, cap, cfg, stream, nullptr);
}

namespace {

// One group waits, bounded, for wave bit 0 of a block whose bits nothing
// sets: the wait the persistent decode does on a stuck source.
__global__ void k_wait_selftest(const unsigned long long *done, uint32_t spin_limit, uint32_t *err) {
    wait_waves_below(done, 1u, err, spin_limit);
}

}  // namespace

extern "C" int aclz_selftest_wait(uint32_t spin_limit, void *stream) {
    if (spin_limit == 0 || spin_limit > kSpinLimitMin) return ACLZ_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    void *buf = nullptr;
    if (cudaError_t e = cudaMalloc(&buf, 64); e != cudaSuccess) {
        note_cuda_error(e);
        return ACLZ_E_NOMEM;
    }
    uint32_t err = 0;
    cudaError_t e = cudaMemsetAsync(buf, 0, 64, st);
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 32, 0, st>>>((const unsigned long long *)buf, spin_limit, (uint32_t *)buf + 8);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, (uint32_t *)buf + 8, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(buf);
    if (e != cudaSuccess) {
        note_cuda_error(e);
        return ACLZ_E_CUDA;
    }
    return (err & kErrTimeout) ? ACLZ_E_TIMEOUT : ACLZ_OK;
}

extern "C" int aclz_device_status(aclz_handle *h, void *stream) {
    if (!h) return ACLZ_E_INVAL;
    uint32_t e = 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&e, h->d_err, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return ACLZ_E_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return ACLZ_E_CUDA;
    if (e) {
        // a failed persistent decode may leave segment counts mid-way
        cudaMemsetAsync(h->d_err, 0, 4, st);
        if (h->d_seg_cnt) cudaMemsetAsync(h->d_seg_cnt, 0, 4 * h->n_seg, st);
        cudaStreamSynchronize(st);
    }
    if (e & kErrTimeout) return ACLZ_E_TIMEOUT;
    if (e) return ACLZ_E_DEVICE;
    return ACLZ_OK;
}

// ------------------------------------------------------------- graphs

struct aclz_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" int aclz_graph_create(aclz_handle *h, void *d_out, uint64_t cap, const aclz_decode_cfg *cfg,
                                 void *stream, aclz_graph **out) {
    if (!h || !out) return ACLZ_E_INVAL;
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    // one plain decode first: sets kernel attributes and occupancy caches
    int rc = aclz_decode_all(h, d_out, cap, cfg, stream);
    if (rc) return rc;
    if (cudaStreamSynchronize(st) != cudaSuccess) return ACLZ_E_CUDA;
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return ACLZ_E_CUDA;
    aclz_graph *g = new aclz_graph();
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = aclz_decode_all(h, d_out, cap, cfg, cs);
        e = cudaStreamEndCapture(cs, &g->graph);
        if (e == cudaSuccess && rc == ACLZ_OK) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess || rc != ACLZ_OK) {
        if (e != cudaSuccess) note_cuda_error(e);
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return rc ? rc : ACLZ_E_CUDA;
    }
    *out = g;
    return ACLZ_OK;
}

extern "C" int aclz_graph_launch(aclz_graph *g, void *stream) {
    if (!g) return ACLZ_E_INVAL;
    cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        note_cuda_error(e);
        return ACLZ_E_CUDA;
    }
    return ACLZ_OK;
}

extern "C" int aclz_graph_free(aclz_graph *g) {
    if (!g) return ACLZ_E_INVAL;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return ACLZ_OK;
}
