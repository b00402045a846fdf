// Upload of a container and construction of its decode index on the GPU.
//
//  1. k_index_scan   per block: prefix-sum of token lengths, per-token
//                    validation (lengths fill the block, every source lies
//                    strictly before its target, Sec. I), block-relative
//                    token offsets for the seek path.
//  2. k_tags_min     minimal wave tags (a match waits one wave for every
//                    cross-block hop of its source chain; same-block sources
//                    are ordered within the block), computed in one launch:
//                    blocks are taken in increasing order and a block waits
//                    (bounded) for the earlier blocks its sources lie in.
//     k_tags_check   legality of tags supplied by the container.
//  3. k_wave_hist, an exclusive scan and k_slots: the wave-major, block-
//     ordered worklist slot of every deferred match.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "aclz_device.cuh"
#include "aclz_internal.h"

using namespace aclz;

namespace {

constexpr uint32_t kSpinLimit = 1u << 24;  // bounded waits (x ~64-256 ns)

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---------------------------------------------------------------- scan
__global__ void __launch_bounds__(256) k_index_scan(const uint4 *__restrict__ tok,
                                                    const uint64_t *__restrict__ blk_tok,
                                                    const uint64_t *__restrict__ blk_lit,
                                                    uint32_t *__restrict__ tokdst,
                                                    uint32_t *__restrict__ toklit, uint32_t nb,
                                                    uint32_t log2bs, uint64_t total, int has_tags,
                                                    uint32_t *err, unsigned long long *first_bad) {
    Group<32> g;
    const uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= nb) return;
    const uint64_t t0 = blk_tok[b], t1 = blk_tok[b + 1];
    const uint64_t bstart = (uint64_t)b << log2bs;
    const uint64_t blen = min((uint64_t)1 << log2bs, total - bstart);
    uint64_t carry = 0, lcarry = 0;
    bool bad = false;
    for (uint64_t w = t0; w < t1; w += 32) {
        const uint64_t i = w + g.lane;
        const bool v = i < t1;
        uint4 t = v ? __ldg(tok + i) : make_uint4(0, 0, 0, 0);
        const uint64_t lit = t.x, ml = t.y;
        const uint64_t sw = (uint64_t)t.z | ((uint64_t)t.w << 32);
        const uint64_t tot = lit + ml;
        const uint64_t incl = g.scan_incl(tot);
        const uint64_t rel = carry + incl - tot;
        const uint64_t lsum = g.scan_incl(lit);
        if (v) {
            bool ok = rel + tot <= blen;
            if (ml == 0) {
                ok = ok && (i == t1 - 1) && sw == 0;
            } else {
                const uint64_t src = sw & kSrcMask;
                const uint64_t dm = bstart + rel + lit;
                ok = ok && ml < (1u << 24) && src + ml <= dm;
                if (!has_tags) ok = ok && (sw >> 40) == 0;
            }
            if (!ok) {
                bad = true;
                atomicMin(first_bad, (unsigned long long)i);
            }
            tokdst[i] = (uint32_t)rel;
            toklit[i] = (uint32_t)(lcarry + lsum - lit);
        }
        carry += g.shfl(incl, 31);
        lcarry += g.shfl(lsum, 31);
    }
    if (g.lane == 0 && (carry != blen || blk_lit[b] + lcarry != blk_lit[b + 1])) bad = true;
    if (g.ballot(bad) && g.lane == 0) atomicOr(err, kErrCorrupt);
}

// Requirement of match i under the current tags: max over the tokens its
// source range overlaps of (0 for literal bytes, tag for match bytes) plus
// one when that token lies in another block.  Sets *inwin when a covering
// token has index >= win0 (same window, still being resolved).
__device__ uint32_t match_requirement(const uint4 *__restrict__ tok, const uint64_t *__restrict__ blk_tok,
                                      const uint32_t *__restrict__ tokdst, const uint32_t *tags,
                                      uint64_t src, uint64_t ml, uint32_t b, uint32_t log2bs,
                                      uint64_t n_tok, uint64_t win0, bool *inwin) {
    uint64_t bp = src >> log2bs;
    uint64_t lo = blk_tok[bp], hi = blk_tok[bp + 1] - 1;
    const uint32_t rel = (uint32_t)(src - (bp << log2bs));
    // last token of block bp with tokdst <= rel
    while (lo < hi) {
        const uint64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(tokdst + mid) <= rel) lo = mid; else hi = mid - 1;
    }
    uint64_t t = lo;
    uint64_t bend_tok = blk_tok[bp + 1];
    const uint64_t e = src + ml;
    uint32_t req = 0;
    for (;;) {
        const uint64_t ts = (bp << log2bs) + __ldg(tokdst + t);
        if (ts >= e) break;
        const uint4 tk = __ldg(tok + t);
        const uint32_t cross = (bp != b) ? 1u : 0u;
        const uint64_t le = ts + tk.x;  // end of literal part
        if (tk.x && le > src) req = max(req, cross);
        if (tk.y && le < e && le + tk.y > src) {
            const uint32_t tg = __ldcg(tags + t);
            req = max(req, tg + cross);
            if (t >= win0) *inwin = true;
        }
        t++;
        if (t >= n_tok) break;
        if (t >= bend_tok) {
            bp++;
            bend_tok = blk_tok[bp + 1];
        }
    }
    return req;
}

// Requirement of match i when only wave 0 versus later matters (the
// flattened schedule): 0 when every source byte lies in block b and is a
// literal byte or a byte of an in-order (tag 0) match of the block, else 1.
// Sets *inwin when a covering token has index >= win0.
__device__ uint32_t local_requirement(const uint4 *__restrict__ tok, const uint64_t *__restrict__ blk_tok,
                                      const uint32_t *__restrict__ tokdst, const uint32_t *tags, uint64_t src,
                                      uint64_t ml, uint32_t b, uint32_t log2bs, uint64_t win0, bool *inwin) {
    const uint64_t bstart = (uint64_t)b << log2bs;
    if ((src >> log2bs) != b || ((src + ml - 1) >> log2bs) != b) return 1;
    uint64_t lo = blk_tok[b], hi = blk_tok[b + 1] - 1;
    const uint32_t rel = (uint32_t)(src - bstart);
    while (lo < hi) {
        const uint64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(tokdst + mid) <= rel) lo = mid; else hi = mid - 1;
    }
    const uint64_t e = src + ml;
    uint32_t req = 0;
    for (uint64_t t = lo; t < blk_tok[b + 1]; t++) {
        const uint64_t ts = bstart + __ldg(tokdst + t);
        if (ts >= e) break;
        const uint4 tk = __ldg(tok + t);
        const uint64_t le = ts + tk.x;
        if (tk.y && le < e && le + tk.y > src) {
            req = max(req, min(__ldcg(tags + t), 1u));
            if (t >= win0) *inwin = true;
        }
    }
    return req;
}

// Wave-0-or-later tags for the flattened schedule: one warp per block, no
// cross-block waits (a source in another block is always "later"); in-window
// dependencies resolved by iterating the window to its fixed point.
__global__ void __launch_bounds__(256) k_tags_local(const uint4 *__restrict__ tok,
                                                    const uint64_t *__restrict__ blk_tok,
                                                    const uint32_t *__restrict__ tokdst, uint32_t *tags,
                                                    uint32_t nb, uint32_t log2bs, uint32_t *maxtag) {
    Group<32> g;
    const uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= nb) return;
    const uint64_t t0 = blk_tok[b], t1 = blk_tok[b + 1];
    uint32_t mx = 0;
    for (uint64_t w = t0; w < t1; w += 32) {
        const uint64_t i = w + g.lane;
        const bool v = i < t1;
        const uint4 t = v ? __ldg(tok + i) : make_uint4(0, 0, 0, 0);
        const uint64_t ml = t.y;
        const uint64_t src = ((uint64_t)t.z | ((uint64_t)t.w << 32)) & kSrcMask;
        const bool m = v && ml;
        if (v) __stcg(tags + i, 0u);
        __threadfence_block();
        g.sync();
        bool pending = m;
        uint32_t cur = 0;
        for (int it = 0; it < 40; it++) {
            bool inwin = false, changed = false;
            if (pending) {
                const uint32_t req = local_requirement(tok, blk_tok, tokdst, tags, src, ml, b, log2bs, w, &inwin);
                changed = req != cur;
                cur = req;
            }
            if (changed) __stcg(tags + i, cur);
            __threadfence_block();
            g.sync();
            pending = pending && inwin;
            if (!g.ballot(changed) || !g.ballot(pending)) break;
        }
        if (m) mx = max(mx, cur);
    }
    for (int o = 16; o; o >>= 1) mx = max(mx, g.shfl(mx, (g.lane + o) & 31));
    if (g.lane == 0) atomicMax(maxtag, mx);
}

// Minimal tags.  Warps take blocks in increasing order from a counter; a
// block's matches whose sources lie in earlier blocks wait (bounded) for
// those blocks' done flags; in-window dependencies are resolved by
// iterating the window to its fixed point.
__global__ void __launch_bounds__(256) k_tags_min(const uint4 *__restrict__ tok,
                                                  const uint64_t *__restrict__ blk_tok,
                                                  const uint32_t *__restrict__ tokdst,
                                                  uint32_t *tags, uint32_t *done, uint32_t *ctr,
                                                  uint32_t nb, uint32_t log2bs, uint64_t n_tok,
                                                  uint32_t *maxtag, uint32_t *err) {
    Group<32> g;
    for (;;) {
        uint32_t b = 0;
        if (g.lane == 0) b = atomicAdd(ctr, 1u);
        b = g.shfl(b, 0);
        if (b >= nb) return;
        const uint64_t t0 = blk_tok[b], t1 = blk_tok[b + 1];
        uint32_t mx = 0;
        bool timed_out = false;
        for (uint64_t w = t0; w < t1; w += 32) {
            const uint64_t i = w + g.lane;
            const bool v = i < t1;
            uint4 t = v ? __ldg(tok + i) : make_uint4(0, 0, 0, 0);
            const uint64_t ml = t.y;
            const uint64_t src = ((uint64_t)t.z | ((uint64_t)t.w << 32)) & kSrcMask;
            const bool m = v && ml;
            if (v) __stcg(tags + i, 0u);
            // wait for the earlier blocks this match reads
            if (m) {
                const uint64_t b0 = src >> log2bs, b1 = (src + ml - 1) >> log2bs;
                for (uint64_t bb = b0; bb <= b1 && bb < b; bb++) {
                    uint32_t spins = 0;
                    while (ld_acquire(done + bb) == 0) {
                        if (++spins > kSpinLimit) { timed_out = true; break; }
                        __nanosleep(64);
                    }
                }
            }
            __threadfence_block();
            g.sync();
            // fixed point of the window: requirements only grow, and an
            // in-window chain of length k settles after k + 1 passes
            bool pending = m;
            uint32_t cur = 0;
            for (int it = 0; it < 40; it++) {
                bool inwin = false, changed = false;
                if (pending) {
                    const uint32_t req = match_requirement(tok, blk_tok, tokdst, tags, src, ml, b,
                                                           log2bs, n_tok, w, &inwin);
                    changed = req != cur;
                    cur = req;
                }
                if (changed) __stcg(tags + i, cur);
                __threadfence_block();
                g.sync();
                pending = pending && inwin;
                if (!g.ballot(changed) || !g.ballot(pending)) break;
            }
            if (m) mx = max(mx, cur);
        }
        if (g.ballot(timed_out) && g.lane == 0) atomicOr(err, kErrTimeout);
        for (int o = 16; o; o >>= 1) mx = max(mx, g.shfl(mx, (g.lane + o) & 31));
        __threadfence();
        g.sync();
        if (g.lane == 0) {
            atomicMax(maxtag, mx);
            st_release(done + b, 1u);
        }
    }
}

// Legality of given tags: tag >= requirement for every match, 0 for
// literal-only tokens.
__global__ void __launch_bounds__(256) k_tags_check(const uint4 *__restrict__ tok,
                                                    const uint64_t *__restrict__ blk_tok,
                                                    const uint32_t *__restrict__ tokdst,
                                                    uint32_t *tags, uint32_t nb, uint32_t log2bs,
                                                    uint64_t n_tok, uint32_t *maxtag, uint32_t *err) {
    Group<32> g;
    const uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= nb) return;
    const uint64_t t0 = blk_tok[b], t1 = blk_tok[b + 1];
    uint32_t mx = 0;
    bool bad = false;
    for (uint64_t w = t0; w < t1; w += 32) {
        const uint64_t i = w + g.lane;
        if (i < t1) {
            const uint4 t = __ldg(tok + i);
            const uint64_t sw = (uint64_t)t.z | ((uint64_t)t.w << 32);
            const uint32_t tg = (uint32_t)(sw >> 40);
            if (t.y) {
                bool inwin = false;
                const uint32_t req = match_requirement(tok, blk_tok, tokdst, tags, sw & kSrcMask, t.y, b,
                                                       log2bs, n_tok, n_tok, &inwin);
                if (req > tg) bad = true;
            } else if (tg) {
                bad = true;
            }
            mx = max(mx, tg);
        }
    }
    for (int o = 16; o; o >>= 1) mx = max(mx, g.shfl(mx, (g.lane + o) & 31));
    if (g.lane == 0) atomicMax(maxtag, mx);
    if (g.ballot(bad) && g.lane == 0) atomicOr(err, kErrCorrupt);
}

// One pass of the parallel minimal-tag computation: every match's tag is
// raised to its requirement under the current tags (read as other warps
// leave them).  Requirements only grow with the tags, so from all-zero
// tags the passes climb to the least fixed point, which is the minimal
// tagging; a pass that raises nothing (changed stays 0) proves it reached.
// Also folds the largest tag into *maxtag.
__global__ void __launch_bounds__(256) k_tags_relax(const uint4 *__restrict__ tok,
                                                    const uint64_t *__restrict__ blk_tok,
                                                    const uint32_t *__restrict__ tokdst, uint32_t *tags,
                                                    uint32_t nb, uint32_t log2bs, uint64_t n_tok,
                                                    uint32_t *changed, uint32_t *maxtag) {
    Group<32> g;
    const uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= nb) return;
    const uint64_t t0 = blk_tok[b], t1 = blk_tok[b + 1];
    uint32_t mx = 0;
    bool raised = false;
    for (uint64_t w = t0; w < t1; w += 32) {
        const uint64_t i = w + g.lane;
        if (i < t1) {
            const uint4 t = __ldg(tok + i);
            if (t.y) {
                const uint64_t src = ((uint64_t)t.z | ((uint64_t)t.w << 32)) & kSrcMask;
                bool inwin = false;
                const uint32_t req = match_requirement(tok, blk_tok, tokdst, tags, src, t.y, b, log2bs, n_tok,
                                                       n_tok, &inwin);
                const uint32_t cur = __ldcg(tags + i);
                if (req > cur) {
                    __stcg(tags + i, req);
                    raised = true;
                }
                mx = max(mx, max(req, cur));
            }
        }
        g.sync();
    }
    for (int o = 16; o; o >>= 1) mx = max(mx, g.shfl(mx, (g.lane + o) & 31));
    if (g.ballot(raised) && g.lane == 0) *changed = 1u;
    if (g.lane == 0 && mx) atomicMax(maxtag, mx);
}

__global__ void k_extract_tags(const uint4 *__restrict__ tok, uint32_t *tags, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        tags[i] = __ldg(tok + i).w >> 8;
}

__global__ void k_store_tags(uint4 *tok, const uint32_t *tags, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint4 t = tok[i];
        t.w = (t.w & 0xffu) | (tags[i] << 8);
        tok[i] = t;
    }
}

// counts per (wave >= 1, block), wave-major, and the deferred bytes
__global__ void __launch_bounds__(256) k_wave_hist(const uint4 *__restrict__ tok,
                                                   const uint64_t *__restrict__ blk_tok,
                                                   uint32_t *cnt, uint32_t nb,
                                                   unsigned long long *def_bytes) {
    const uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= nb) return;
    unsigned long long bytes = 0;
    for (uint64_t i = blk_tok[b] + lane; i < blk_tok[b + 1]; i += 32) {
        const uint4 t = __ldg(tok + i);
        const uint32_t tg = t.w >> 8;
        if (t.y && tg) {
            atomicAdd(cnt + (uint64_t)(tg - 1) * nb + b, 1u);
            bytes += t.y;
        }
    }
    for (int o = 16; o; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
    if (lane == 0 && bytes) atomicAdd(def_bytes, bytes);
}

// slot of every deferred match: its (wave, block) segment base plus its
// rank among that segment's matches in token order
__global__ void __launch_bounds__(256) k_slots(const uint4 *__restrict__ tok,
                                               const uint64_t *__restrict__ blk_tok, uint32_t *cursor,
                                               uint32_t *slot, uint32_t nb) {
    Group<32> g;
    const uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= nb) return;
    const uint64_t t0 = blk_tok[b], t1 = blk_tok[b + 1];
    for (uint64_t w = t0; w < t1; w += 32) {
        const uint64_t i = w + g.lane;
        const bool v = i < t1;
        uint4 t = v ? __ldg(tok + i) : make_uint4(0, 0, 0, 0);
        const uint32_t tg = t.w >> 8;
        const bool def = v && t.y && tg;
        const unsigned long long key = def ? (unsigned long long)(tg - 1) * nb + b : ~0ULL;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(peers) - 1;
        uint32_t basev = 0;
        if (def && g.lane == leader) {
            basev = cursor[key];
            cursor[key] = basev + __popc(peers);
        }
        basev = __shfl_sync(0xffffffffu, basev, leader);
        if (v) slot[i] = def ? basev + __popc(peers & g.lanemask_lt()) : 0xffffffffu;
        __syncwarp();
    }
}

// Triplets of the deferred matches, written once at upload: tri[slot[i]]
// = (dst, src, len) of deferred match token i, so the worklists are in
// wave-major, block order and in token order within a block.
__global__ void __launch_bounds__(256) k_tri_build(const uint4 *__restrict__ tok,
                                                   const uint64_t *__restrict__ blk_tok,
                                                   const uint32_t *__restrict__ tokdst,
                                                   const uint32_t *__restrict__ slot, uint32_t nb,
                                                   uint32_t log2bs, uint4 *__restrict__ tri) {
    const uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= nb) return;
    const uint64_t bstart = (uint64_t)b << log2bs;
    for (uint64_t i = blk_tok[b] + lane; i < blk_tok[b + 1]; i += 32) {
        const uint32_t sl = __ldg(slot + i);
        if (sl == 0xffffffffu) continue;
        const uint4 t = __ldg(tok + i);
        const uint64_t dm = bstart + __ldg(tokdst + i) + t.x;
        tri[sl] = make_uint4((uint32_t)dm, (uint32_t)(dm >> 32), t.z, (t.w & 0xffu) | (t.y << 8));
    }
}

// flag[k] = 1 when (wave, block) segment k is non-empty; base is the
// exclusive scan of the segment counts, *total its sum
__global__ void k_seg_flags(const uint32_t *base, uint64_t M, const uint32_t *total, uint32_t *flag) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < M;
         k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t nxt = k + 1 < M ? base[k + 1] : *total;
        flag[k] = nxt > base[k] ? 1u : 0u;
    }
}

// Segments of the persistent decode, wave-major: seg[pos[k]] for every
// non-empty (wave, block) cell k, and the block's pending-wave bits.
__global__ void k_segs_build(const uint32_t *base, const uint32_t *pos, const uint32_t *total,
                             uint32_t nb, uint32_t nw1, uint32_t ww, uint4 *seg,
                             unsigned long long *pending) {
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const uint64_t M = (uint64_t)nw1 * nb;
    unsigned long long word = 1ULL;  // wave 0
    uint32_t wk = 0;
    for (uint32_t w = 1; w <= nw1; w++) {
        if (w / 64 != wk) {
            pending[(uint64_t)b * ww + wk] = word;
            wk = w / 64;
            word = 0;
        }
        const uint64_t k = (uint64_t)(w - 1) * nb + b;
        const uint32_t nxt = k + 1 < M ? base[k + 1] : *total;
        const uint32_t c = nxt - base[k];
        if (!c) continue;
        seg[pos[k]] = make_uint4(b, w, base[k], c);
        word |= 1ULL << (w % 64);
    }
    pending[(uint64_t)b * ww + wk] = word;
    for (uint32_t k2 = wk + 1; k2 < ww; k2++) pending[(uint64_t)b * ww + k2] = 0;
}

// seg_of[t] = the segment holding triplet t (segments are consecutive
// runs of the triplet array).
__global__ void k_seg_of(const uint4 *__restrict__ seg, uint64_t nseg, uint32_t *__restrict__ seg_of) {
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < nseg;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 a = seg[s];
        for (uint32_t k = 0; k < a.w; k++) seg_of[a.z + k] = (uint32_t)s;
    }
}

// segdep[s] = 1 when a match of segment s reads bytes that an earlier
// match of the same segment writes (a chain inside one block and wave):
// such a segment is never cut between two ranges.  The outputs of one
// segment are disjoint and in increasing order, so the last earlier output
// starting below the source's end decides.
__global__ void k_seg_dep(const uint4 *__restrict__ tri, const uint4 *__restrict__ seg,
                          const uint32_t *__restrict__ seg_of, uint64_t n, uint32_t *segdep) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t s = seg_of[t];
        const uint64_t a = seg[s].z;
        if (t == a) continue;
        const uint4 x = tri[t];
        const uint64_t src = (uint64_t)x.z | ((uint64_t)(x.w & 0xffu) << 32);
        const uint64_t se = src + (x.w >> 8);
        uint64_t lo = a, hi = t;  // first j in [a, t) with dst_j >= se
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            const uint4 y = tri[mid];
            const uint64_t dj = (uint64_t)y.x | ((uint64_t)(y.y & 0xffu) << 32);
            if (dj < se) lo = mid + 1; else hi = mid;
        }
        if (lo > a) {
            const uint4 y = tri[lo - 1];
            const uint64_t dj = (uint64_t)y.x | ((uint64_t)(y.y & 0xffu) << 32);
            if (dj + (y.w >> 8) > src) segdep[s] = 1u;
        }
    }
}

// Bit 8 of a triplet's .y (above its destination's high byte) marks the
// triplets of segments without an internal chain: the per-wave kernel may
// cut such a segment between groups at any triplet.
__global__ void k_tri_cuttable(uint4 *tri, const uint32_t *__restrict__ seg_of, const uint32_t *__restrict__ segdep,
                               uint64_t n) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n;
         t += (uint64_t)gridDim.x * blockDim.x)
        tri[t].y = (tri[t].y & 0xffu) | (segdep[seg_of[t]] ? 0u : 0x100u);
}

// Range starts.  In wave w (triplets from wstart[w]) a range starts every
// wT[w] triplets, except inside a segment with an internal chain, whose
// candidate starts move to the end of that segment.
__global__ void k_range_flags(const uint4 *__restrict__ seg, const uint32_t *__restrict__ seg_of,
                              const uint32_t *__restrict__ segdep, const uint64_t *__restrict__ wstart,
                              const uint32_t *__restrict__ wT, uint64_t n, uint32_t *flag) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t s = seg_of[t];
        const uint4 a = seg[s];
        const uint64_t ws = wstart[a.y];
        const uint64_t T = wT[a.y];
        bool f;
        if (t == ws) {
            f = true;
        } else if (segdep[s] && t > a.z) {
            f = false;
        } else if ((t - ws) % T == 0) {
            f = true;
        } else if (t == a.z && s > 0) {
            const uint4 p = seg[s - 1];
            f = p.y == a.y && segdep[s - 1] && (t - 1 - ws) / T > (p.z - ws) / T;
        } else {
            f = false;
        }
        flag[t] = f ? 1u : 0u;
    }
}

// ranges[r] = {wave, first segment, end segment, first triplet} from the
// exclusive scan ex of the range-start flags (nr ranges); ranges[nr] is a
// sentinel whose first triplet is n.
__global__ void k_range_build(const uint4 *__restrict__ seg, const uint32_t *__restrict__ seg_of,
                              const uint32_t *__restrict__ flag, const uint32_t *__restrict__ ex, uint64_t n,
                              uint32_t nr, uint4 *ranges) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n;
         t += (uint64_t)gridDim.x * blockDim.x) {
        if (flag[t]) {
            const uint32_t r = ex[t];
            const uint32_t s = seg_of[t];
            ranges[r].x = seg[s].y;
            ranges[r].y = s;
            ranges[r].w = (uint32_t)t;
            if (r > 0) ranges[r - 1].z = seg_of[t - 1] + 1;
        }
        if (t + 1 == n) {
            ranges[nr - 1].z = seg_of[t] + 1;
            ranges[nr] = make_uint4(0u, seg_of[t] + 1, seg_of[t] + 1, (uint32_t)n);
        }
    }
}

// pieces[s] = number of ranges that hold triplets of segment s.
__global__ void k_seg_pieces(const uint4 *__restrict__ seg, const uint32_t *__restrict__ flag,
                             const uint32_t *__restrict__ ex, uint64_t nseg, uint32_t *pieces) {
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < nseg;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 a = seg[s];
        const uint64_t f = a.z, l = a.z + a.w - 1;
        pieces[s] = (ex[l] + flag[l]) - (ex[f] + flag[f]) + 1;
    }
}

// ------------------------------------------------- exclusive scan (u32)
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ uint32_t block_excl_scan(uint32_t v, uint32_t *sh, uint32_t *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t y = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += t;
        }
        sh[lane] = y;
    }
    __syncthreads();
    const uint32_t off = wid ? sh[wid - 1] : 0;
    *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return off + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *in, uint64_t n,
                                                              uint32_t *part) {
    __shared__ uint32_t sh[32];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
    for (int k = 0; k < kScanItems; k++)
        if (base + k < n) s += in[base + k];
    uint32_t tot;
    block_excl_scan(s, sh, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_parts(uint32_t *part, uint64_t np) {
    __shared__ uint32_t sh[32];
    uint32_t carry = 0;
    for (uint64_t b = 0; b < np; b += kScanThreads) {
        const uint64_t i = b + threadIdx.x;
        const uint32_t v = i < np ? part[i] : 0;
        uint32_t tot;
        const uint32_t ex = block_excl_scan(v, sh, &tot);
        if (i < np) part[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) part[np] = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(uint32_t *io, uint64_t n,
                                                             const uint32_t *part) {
    __shared__ uint32_t sh[32];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems], s = 0;
    for (int k = 0; k < kScanItems; k++) {
        v[k] = base + k < n ? io[base + k] : 0;
        s += v[k];
    }
    uint32_t tot;
    uint32_t ex = block_excl_scan(s, sh, &tot) + part[blockIdx.x];
    for (int k = 0; k < kScanItems; k++) {
        if (base + k < n) io[base + k] = ex;
        ex += v[k];
    }
}

__global__ void k_gather_starts(const uint32_t *base, uint64_t nb, uint32_t nw1, const uint32_t *total,
                                uint64_t *starts) {
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w <= nw1; w += gridDim.x * blockDim.x)
        starts[w] = w < nw1 ? base[(uint64_t)w * nb] : *total;
}

// ---------------------------------------------------------- host helpers
struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

int cuda_rc(cudaError_t e) {
    if (e == cudaSuccess) return ACLZ_OK;
    return e == cudaErrorMemoryAllocation ? ACLZ_E_NOMEM : ACLZ_E_CUDA;
}

#define CK(x)                                \
    do {                                     \
        int _rc = cuda_rc(x);                \
        if (_rc) { cleanup(); return _rc; }  \
    } while (0)

}  // namespace

// Exclusive scan of n u32 in place (device), total to *d_total (device).
// Temporary partials are allocated stream-ordered.
int aclz::device_excl_scan(uint32_t *d, uint64_t n, uint32_t *d_total, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t ntile = (n + kScanTile - 1) / kScanTile;
    uint32_t *part = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&part, sizeof(uint32_t) * (ntile + 1), st);
    if (e != cudaSuccess) return cuda_rc(e);
    if (ntile) k_scan_reduce<<<(unsigned)ntile, kScanThreads, 0, st>>>(d, n, part);
    k_scan_parts<<<1, kScanThreads, 0, st>>>(part, ntile);
    if (ntile) k_scan_apply<<<(unsigned)ntile, kScanThreads, 0, st>>>(d, n, part);
    cudaMemcpyAsync(d_total, part + ntile, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
    cudaFreeAsync(part, st);
    return cuda_rc(cudaGetLastError());
}

// Minimal wave tags of h's tokens into d_tags (and the largest into
// *d_maxtag) by parallel relaxation passes from all-zero tags, checked every
// kRelaxBatch passes; true when a pass raised nothing within kRelaxMax
// passes.  A stream whose copy chains are deeper than that is left to the
// ordered pass (false; d_tags then holds partial tags).
namespace {
constexpr uint32_t kRelaxBatch = 8, kRelaxMax = 512;
bool relax_tags(aclz_handle *h, uint32_t *d_tags, uint32_t *d_maxtag, cudaStream_t st) {
    const uint32_t nb = h->n_blocks;
    const uint64_t nt = h->n_tokens;
    if (!nb) return true;
    DevBuf flags;
    if (cudaMalloc(&flags.p, 4 * kRelaxBatch) != cudaSuccess) return false;
    uint32_t *changed = (uint32_t *)flags.p;
    if (cudaMemsetAsync(d_tags, 0, 4 * (nt ? nt : 1), st) != cudaSuccess) return false;
    const unsigned wblocks = (nb + 7) / 8;
    for (uint32_t done_passes = 0; done_passes < kRelaxMax; done_passes += kRelaxBatch) {
        if (cudaMemsetAsync(changed, 0, 4 * kRelaxBatch, st) != cudaSuccess) return false;
        for (uint32_t k = 0; k < kRelaxBatch; k++)
            k_tags_relax<<<wblocks, 256, 0, st>>>((const uint4 *)h->d_tok, h->d_blk_tok, h->d_tokdst, d_tags, nb,
                                                   h->log2_bs, nt, changed + k, d_maxtag);
        uint32_t last = 1;
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&last, changed + kRelaxBatch - 1, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return false;
        if (!last) return true;
    }
    return false;
}
}  // namespace

// Decode index of h from its device tokens (d_tok with n_tokens entries,
// d_blk_tok, d_blk_lit, d_lit): per-token validation and offsets, wave
// tags (given ones checked, else minimal ones; local 0/1 ones for the
// flattened schedule), worklist slots and the persistent schedule.
// Allocates d_tokdst, d_toklit, d_slot and the schedule arrays (freed first
// when present).  Synchronizes the stream.
int aclz::build_index(aclz_handle *h, bool has_tags, uint32_t given_waves, bool flat_local, void *stream_) {
    auto cleanup = []() {};
    void *stream = stream_;
    cudaStream_t st = (cudaStream_t)stream_;
    const bool flat_up = flat_local;
    const uint32_t nb = h->n_blocks;
    const uint64_t nt = h->n_tokens;
    int rc = ACLZ_OK;
    for (void **pp : {(void **)&h->d_tokdst, (void **)&h->d_toklit, (void **)&h->d_slot, &h->d_tri, &h->d_seg,
                      &h->d_ranges, (void **)&h->d_pending, (void **)&h->d_done}) {
        if (*pp) cudaFree(*pp);
        *pp = nullptr;
    }
    h->n_seg = h->n_ranges = 0;
    h->n_deferred = 0;
    CK(cudaMalloc((void **)&h->d_tokdst, 4 * (nt ? nt : 1)));
    CK(cudaMalloc((void **)&h->d_toklit, 4 * (nt ? nt : 1)));
    CK(cudaMalloc((void **)&h->d_slot, 4 * (nt ? nt : 1)));
    CK(cudaMemsetAsync(h->d_err, 0, 64, st));
    // scratch words: [0] err (handle), work: maxtag, counter, total, first_bad
    DevBuf work;
    CK(cudaMalloc(&work.p, 64));
    uint32_t *d_maxtag = (uint32_t *)work.p, *d_ctr = d_maxtag + 1, *d_total = d_maxtag + 2;
    // words: [0] max tag, [1] counter, [2] deferred total, [3] segment count,
    // [4] range count; bytes 32..39: first bad token
    unsigned long long *d_first_bad = (unsigned long long *)((char *)work.p + 32);
    CK(cudaMemsetAsync(work.p, 0, 32, st));
    CK(cudaMemsetAsync(d_first_bad, 0xff, 8, st));
    const unsigned wblocks = (nb + 7) / 8;  // 8 warps per CTA
    k_index_scan<<<wblocks, 256, 0, st>>>((const uint4 *)h->d_tok, h->d_blk_tok, h->d_blk_lit, h->d_tokdst,
                                           h->d_toklit, nb, h->log2_bs, h->total_len, has_tags, h->d_err,
                                           d_first_bad);
    CK(cudaGetLastError());
    uint32_t herr = 0;
    CK(cudaMemcpyAsync(&herr, h->d_err, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (herr) { cleanup(); return ACLZ_E_CORRUPT; }
    // tags
    DevBuf tags, done;
    CK(cudaMalloc(&tags.p, 4 * (nt ? nt : 1)));
    uint32_t *d_tags = (uint32_t *)tags.p;
    h->local_tags = false;
    if (has_tags) {
        k_extract_tags<<<1024, 256, 0, st>>>((const uint4 *)h->d_tok, d_tags, nt);
        k_tags_check<<<wblocks, 256, 0, st>>>((const uint4 *)h->d_tok, h->d_blk_tok, h->d_tokdst,
                                               d_tags, nb, h->log2_bs, nt, d_maxtag, h->d_err);
    } else if (flat_up) {
        h->local_tags = true;
        k_tags_local<<<wblocks, 256, 0, st>>>((const uint4 *)h->d_tok, h->d_blk_tok, h->d_tokdst, d_tags, nb,
                                               h->log2_bs, d_maxtag);
        k_store_tags<<<1024, 256, 0, st>>>((uint4 *)h->d_tok, d_tags, nt);
    } else if (relax_tags(h, d_tags, d_maxtag, st)) {
        // minimal tags by parallel passes (the chains were shallow enough)
        k_store_tags<<<1024, 256, 0, st>>>((uint4 *)h->d_tok, d_tags, nt);
    } else {
        CK(cudaMemsetAsync(d_maxtag, 0, 4, st));
        CK(cudaMalloc(&done.p, 4 * nb));
        CK(cudaMemsetAsync(done.p, 0, 4 * nb, st));
        int dev_sms = 0;
        cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, h->device);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tags_min, 256, 0);
        unsigned grid = (unsigned)std::max(1, dev_sms * std::max(1, per_sm));
        grid = std::min<unsigned>(grid, wblocks);
        k_tags_min<<<grid, 256, 0, st>>>((const uint4 *)h->d_tok, h->d_blk_tok, h->d_tokdst, d_tags,
                                          (uint32_t *)done.p, d_ctr, nb, h->log2_bs, nt, d_maxtag,
                                          h->d_err);
        k_store_tags<<<1024, 256, 0, st>>>((uint4 *)h->d_tok, d_tags, nt);
    }
    CK(cudaGetLastError());
    uint32_t hw[2] = {0, 0};
    CK(cudaMemcpyAsync(&hw[0], d_maxtag, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&hw[1], h->d_err, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hw[1] & kErrTimeout) { cleanup(); return ACLZ_E_TIMEOUT; }
    if (hw[1]) { cleanup(); return ACLZ_E_CORRUPT; }
    const uint32_t maxtag = hw[0];
    if (maxtag > kMaxWave) { cleanup(); return ACLZ_E_UNSUPPORTED; }
    if (has_tags && given_waves != maxtag + 1) { cleanup(); return ACLZ_E_CORRUPT; }
    h->n_waves = maxtag + 1;
    h->wave_start.assign(h->n_waves + 1, 0);
    CK(cudaMemsetAsync(h->d_slot, 0xff, 4 * nt, st));
    unsigned long long defb_total = 0;
    // The plain schedule keeps a dense (wave, block) count table and
    // per-block wave bitmasks, quadratic in the chain depth; beyond 2^28
    // cells the upload builds the flattened two-wave schedule instead.
    h->needs_flatten = maxtag > 0 && (uint64_t)maxtag * nb > (1ULL << 28);
    if (maxtag > 0 && !h->needs_flatten) {
        const uint64_t M = (uint64_t)maxtag * nb;
        DevBuf cnt, starts;
        CK(cudaMalloc(&cnt.p, 4 * M));
        CK(cudaMalloc(&starts.p, 8 * (maxtag + 1)));
        CK(cudaMemsetAsync(cnt.p, 0, 4 * M, st));
        unsigned long long *d_def_bytes = (unsigned long long *)((char *)work.p + 40);
        CK(cudaMemsetAsync(d_def_bytes, 0, 8, st));
        k_wave_hist<<<wblocks, 256, 0, st>>>((const uint4 *)h->d_tok, h->d_blk_tok, (uint32_t *)cnt.p, nb,
                                              d_def_bytes);
        CK(cudaGetLastError());
        rc = device_excl_scan((uint32_t *)cnt.p, M, d_total, st);
        if (rc) { cleanup(); return rc; }
        k_gather_starts<<<(maxtag + 256) / 256, 256, 0, st>>>((const uint32_t *)cnt.p, nb, maxtag, d_total,
                                                            (uint64_t *)starts.p);
        // persistent-mode segments and ranges, from the segment bases
        // (before k_slots turns the bases into cursors)
        {
            DevBuf flag;
            CK(cudaMalloc(&flag.p, 4 * M));
            k_seg_flags<<<1024, 256, 0, st>>>((const uint32_t *)cnt.p, M, d_total, (uint32_t *)flag.p);
            uint32_t *d_nseg = d_total + 1;
            rc = device_excl_scan((uint32_t *)flag.p, M, d_nseg, st);
            if (rc) { cleanup(); return rc; }
            uint32_t nseg = 0;
            CK(cudaMemcpyAsync(&nseg, d_nseg, 4, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            h->n_seg = nseg;
            h->n_wave_words = (maxtag + 1 + 63) / 64;
            CK(cudaMalloc(&h->d_seg, 16 * (size_t)(nseg ? nseg : 1)));
            CK(cudaMalloc((void **)&h->d_pending, 8 * (size_t)nb * h->n_wave_words));
            k_segs_build<<<(nb + 255) / 256, 256, 0, st>>>((const uint32_t *)cnt.p, (const uint32_t *)flag.p,
                                                          d_total, nb, maxtag, h->n_wave_words,
                                                          (uint4 *)h->d_seg,
                                                          (unsigned long long *)h->d_pending);
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(&defb_total, d_def_bytes, 8, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            CK(cudaStreamSynchronize(st));
        }
        k_slots<<<wblocks, 256, 0, st>>>((const uint4 *)h->d_tok, h->d_blk_tok, (uint32_t *)cnt.p,
                                          h->d_slot, nb);
        CK(cudaGetLastError());
        // wave_start[0] = wave_start[1] = 0: wave 0 has no triplets
        CK(cudaMemcpyAsync(h->wave_start.data() + 1, starts.p, 8 * (maxtag + 1), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        h->n_deferred = h->wave_start[h->n_waves];
        if (h->n_deferred) {
            CK(cudaMalloc(&h->d_tri, 16 * h->n_deferred));
            k_tri_build<<<wblocks, 256, 0, st>>>((const uint4 *)h->d_tok, h->d_blk_tok, h->d_tokdst, h->d_slot,
                                                  nb, h->log2_bs, (uint4 *)h->d_tri);
            CK(cudaGetLastError());
        }
        h->mean_deferred_len = h->n_deferred ? (double)defb_total / (double)h->n_deferred : 0.0;
        rc = aclz_set_range_bytes(h, h->range_bytes, stream);
        if (rc) { cleanup(); return rc; }
    }
    if (!h->d_pending) {  // no deferred matches: wave 0 finishes every block
        h->n_wave_words = 1;
        std::vector<uint64_t> ones(nb, 1ULL);
        CK(cudaMalloc((void **)&h->d_pending, 8 * (size_t)nb));
        CK(cudaMemcpyAsync(h->d_pending, ones.data(), 8 * (size_t)nb, cudaMemcpyHostToDevice, st));
    }
    CK(cudaMalloc((void **)&h->d_done, 8 * (size_t)nb * h->n_wave_words));
    CK(cudaStreamSynchronize(st));
    return ACLZ_OK;
}

extern "C" int aclz_upload(const void *host_buf, uint64_t n, void *stream, aclz_handle **out) {
    return aclz_upload_ex(host_buf, n, 0, stream, out);
}

namespace aclz {

// Token array and literal bytes of a host container: copied as they are.
static int fill_from_host(aclz_handle *h, const View &v, const void *, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (v.n_tokens && cudaMemcpyAsync(h->d_tok, v.tok, kTok * v.n_tokens, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return ACLZ_E_CUDA;
    if (v.n_literals && cudaMemcpyAsync(h->d_lit, v.lit, v.n_literals, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return ACLZ_E_CUDA;
    return ACLZ_OK;
}

int upload_view(const View &v, uint32_t flags, void *stream, FillFn fill, const void *ctx, aclz_handle **out) {
    if (flags & ~(uint32_t)ACLZ_UPLOAD_FLATTEN) return ACLZ_E_INVAL;
    const bool flat_up = (flags & ACLZ_UPLOAD_FLATTEN) != 0;
    if (!out) return ACLZ_E_INVAL;
    *out = nullptr;
    if (!is_pow2(v.block_size) || v.block_size < kMinBlock || v.block_size > kMaxBlock)
        return ACLZ_E_UNSUPPORTED;
    if (v.n_tokens >= 0xffffffffULL) return ACLZ_E_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    aclz_handle *h = new aclz_handle();
    auto cleanup = [&]() { aclz_free(h); };
    cudaGetDevice(&h->device);
    h->total_len = v.total_len;
    h->n_tokens = v.n_tokens;
    h->n_literals = v.n_literals;
    h->block_size = v.block_size;
    h->log2_bs = log2u(v.block_size);
    h->n_blocks = v.n_blocks;
    h->flags = v.flags;
    std::memcpy(h->mm, v.mm, 4);
    const uint32_t nb = v.n_blocks;
    const uint64_t nt = v.n_tokens;
    // directory -> (nb + 1) offset arrays
    std::vector<uint64_t> bt(nb + 1), bl(nb + 1);
    for (uint32_t b = 0; b < nb; b++) {
        bt[b] = rd64(v.dir + (uint64_t)kDirent * b);
        bl[b] = rd64(v.dir + (uint64_t)kDirent * b + 8);
    }
    bt[nb] = nt;
    bl[nb] = v.n_literals;
    CK(cudaMalloc(&h->d_tok, kTok * (nt ? nt : 1)));
    CK(cudaMalloc((void **)&h->d_lit, v.n_literals + 32));
    CK(cudaMalloc((void **)&h->d_blk_tok, 8 * (nb + 1)));
    CK(cudaMalloc((void **)&h->d_blk_lit, 8 * (nb + 1)));
    CK(cudaMalloc((void **)&h->d_err, 64));
    CK(cudaMemsetAsync(h->d_err, 0, 64, st));
    CK(cudaMemsetAsync(h->d_lit + v.n_literals, 0, 32, st));
    if (int rc = fill(h, v, ctx, stream); rc != ACLZ_OK) {
        cleanup();
        return rc;
    }
    CK(cudaMemcpyAsync(h->d_blk_tok, bt.data(), 8 * (nb + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(h->d_blk_lit, bl.data(), 8 * (nb + 1), cudaMemcpyHostToDevice, st));
    if (nb == 0) {
        h->n_waves = 0;
        h->wave_start.assign(1, 0);
        CK(cudaStreamSynchronize(st));
        *out = h;
        return ACLZ_OK;
    }
    int rc = build_index(h, (v.flags & kFlagWaves) != 0, v.n_waves, flat_up, stream);
    if (rc) { cleanup(); return rc; }
    if (flat_up || h->needs_flatten) {
        rc = aclz_flatten(h, stream);
        if (rc) { cleanup(); return rc; }
    }
    *out = h;
    return ACLZ_OK;
}

}  // namespace aclz

extern "C" int aclz_upload_ex(const void *host_buf, uint64_t n, uint32_t flags, void *stream, aclz_handle **out) {
    if (flags & ~(uint32_t)ACLZ_UPLOAD_FLATTEN) return ACLZ_E_INVAL;
    if (!host_buf || !out) return ACLZ_E_INVAL;
    *out = nullptr;
    View v;
    int rc = parse_container((const uint8_t *)host_buf, n, &v, true);
    if (rc) return rc;
    return upload_view(v, flags, stream, fill_from_host, nullptr, out);
}

extern "C" int aclz_free(aclz_handle *h) {
    if (!h) return ACLZ_E_INVAL;
    void *ps[] = {h->d_tok, h->d_lit,    h->d_blk_tok, h->d_blk_lit,      h->d_slot,      h->d_tokdst,
                  h->d_toklit, h->d_tri, h->d_err,     h->d_seg,          h->d_ranges,    h->d_seg_pieces,
                  h->d_seg_cnt, h->d_pending, h->d_done};
    for (void *p : ps)
        if (p) cudaFree(p);
    delete h;
    return ACLZ_OK;
}

extern "C" int aclz_handle_info(const aclz_handle *h, aclz_info *out) {
    if (!h || !out) return ACLZ_E_INVAL;
    std::memset(out, 0, sizeof(*out));
    out->total_len = h->total_len;
    out->n_tokens = h->n_tokens;
    out->n_literals = h->n_literals;
    out->n_deferred = h->n_deferred;
    out->block_size = h->block_size;
    out->n_blocks = h->n_blocks;
    out->n_waves = h->n_waves;
    out->flags = h->flags;
    std::memcpy(out->min_match, h->mm, 4);
    return ACLZ_OK;
}

extern "C" int aclz_wave_counts(const aclz_handle *h, uint64_t *counts, uint32_t cap) {
    if (!h || (!counts && cap)) return ACLZ_E_INVAL;
    for (uint32_t w = 0; w < cap && w < h->n_waves; w++)
        counts[w] = h->wave_start[w + 1] - h->wave_start[w];
    return ACLZ_OK;
}

extern "C" int aclz_tags(const aclz_handle *h, uint32_t *host_tags, uint64_t cap) {
    if (!h || (!host_tags && cap)) return ACLZ_E_INVAL;
    if (cap < h->n_tokens) return ACLZ_E_CAPACITY;
    if (!h->n_tokens) return ACLZ_OK;
    std::vector<uint32_t> raw(4 * h->n_tokens);
    if (cudaMemcpy(raw.data(), h->d_tok, 16 * h->n_tokens, cudaMemcpyDeviceToHost) != cudaSuccess)
        return ACLZ_E_CUDA;
    for (uint64_t i = 0; i < h->n_tokens; i++) host_tags[i] = raw[4 * i + 3] >> 8;
    return ACLZ_OK;
}

extern "C" int aclz_set_range_bytes(aclz_handle *h, uint32_t range_bytes, void *stream) {
    if (!h || range_bytes == 0) return ACLZ_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    h->range_bytes = range_bytes;
    h->range_T = range_matches(range_bytes, h->mean_deferred_len);
    for (void **pp : {&h->d_ranges, (void **)&h->d_seg_pieces, (void **)&h->d_seg_cnt}) {
        if (*pp) cudaFree(*pp);
        *pp = nullptr;
    }
    h->n_ranges = 0;
    const uint64_t nseg = h->n_seg, n = h->n_deferred;
    if (!nseg || !n) return ACLZ_OK;
    // matches per range by wave: range_T in large waves; a small wave is cut
    // into about kRangesPerSm ranges per SM (down to one match each), so its
    // matches spread over the resident groups and every dependency hop of
    // the wavefront costs the latency of a short range, not of a long one
    int dev_sms = 0;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, h->device);
    const uint64_t P = (uint64_t)std::max(1, dev_sms) * kRangesPerSm;
    const uint32_t nw = h->n_waves;
    std::vector<uint32_t> wT(nw, 1u);
    for (uint32_t w = 1; w < nw; w++) {
        const uint64_t nwv = h->wave_start[w + 1] - h->wave_start[w];
        wT[w] = (uint32_t)std::min<uint64_t>(h->range_T, std::max<uint64_t>(1, (nwv + P - 1) / P));
    }
    DevBuf b_of, b_dep, b_flag, b_ex, b_ws, b_wT;
    int rc = ACLZ_OK;
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == ACLZ_OK) {
            note_cuda_error(e);
            rc = e == cudaErrorMemoryAllocation ? ACLZ_E_NOMEM : ACLZ_E_CUDA;
        }
        return rc == ACLZ_OK;
    };
    if (!ck(cudaMalloc(&b_of.p, 4 * n)) || !ck(cudaMalloc(&b_dep.p, 4 * nseg)) ||
        !ck(cudaMalloc(&b_flag.p, 4 * n)) || !ck(cudaMalloc(&b_ex.p, 4 * n + 16)) ||
        !ck(cudaMalloc(&b_ws.p, 8 * ((size_t)nw + 1))) || !ck(cudaMalloc(&b_wT.p, 4 * (size_t)nw)))
        return rc;
    uint32_t *seg_of = (uint32_t *)b_of.p, *segdep = (uint32_t *)b_dep.p, *flag = (uint32_t *)b_flag.p,
             *ex = (uint32_t *)b_ex.p, *d_nr = ex + n;
    const uint4 *seg = (const uint4 *)h->d_seg;
    const unsigned grid = (unsigned)std::min<uint64_t>(4096, (n + 255) / 256);
    const unsigned gseg = (unsigned)std::min<uint64_t>(4096, (nseg + 255) / 256);
    ck(cudaMemcpyAsync(b_ws.p, h->wave_start.data(), 8 * ((size_t)nw + 1), cudaMemcpyHostToDevice, st));
    ck(cudaMemcpyAsync(b_wT.p, wT.data(), 4 * (size_t)nw, cudaMemcpyHostToDevice, st));
    ck(cudaMemsetAsync(segdep, 0, 4 * nseg, st));
    if (rc) return rc;
    k_seg_of<<<gseg, 256, 0, st>>>(seg, nseg, seg_of);
    k_seg_dep<<<grid, 256, 0, st>>>((const uint4 *)h->d_tri, seg, seg_of, n, segdep);
    k_tri_cuttable<<<grid, 256, 0, st>>>((uint4 *)h->d_tri, seg_of, segdep, n);
    k_range_flags<<<grid, 256, 0, st>>>(seg, seg_of, segdep, (const uint64_t *)b_ws.p, (const uint32_t *)b_wT.p, n,
                                         flag);
    ck(cudaGetLastError());
    ck(cudaMemcpyAsync(ex, flag, 4 * n, cudaMemcpyDeviceToDevice, st));
    if (rc) return rc;
    rc = device_excl_scan(ex, n, d_nr, st);
    uint32_t nr = 0;
    if (rc == ACLZ_OK) ck(cudaMemcpyAsync(&nr, d_nr, 4, cudaMemcpyDeviceToHost, st));
    if (rc == ACLZ_OK) ck(cudaStreamSynchronize(st));
    if (rc == ACLZ_OK && nr) {
        if (ck(cudaMalloc(&h->d_ranges, 16 * ((size_t)nr + 1))) && ck(cudaMalloc((void **)&h->d_seg_pieces, 4 * nseg)) &&
            ck(cudaMalloc((void **)&h->d_seg_cnt, 4 * nseg))) {
            k_range_build<<<grid, 256, 0, st>>>(seg, seg_of, flag, ex, n, nr, (uint4 *)h->d_ranges);
            k_seg_pieces<<<gseg, 256, 0, st>>>(seg, flag, ex, nseg, h->d_seg_pieces);
            ck(cudaGetLastError());
            ck(cudaMemsetAsync(h->d_seg_cnt, 0, 4 * nseg, st));
            ck(cudaStreamSynchronize(st));
            if (rc == ACLZ_OK) h->n_ranges = nr;
        }
    }
    return rc;
}

extern "C" int aclz_export(const aclz_handle *h, void *host_out, uint64_t cap, uint64_t *out_size) {
    if (!h || !out_size || h->local_tags) return ACLZ_E_INVAL;
    const uint64_t nt = h->n_tokens, nl = h->n_literals;
    const uint32_t nb = h->n_blocks;
    const uint64_t need = kHdr + (uint64_t)kDirent * nb + (uint64_t)kTok * nt + nl;
    *out_size = need;
    if (!host_out) return ACLZ_OK;
    if (cap < need) return ACLZ_E_CAPACITY;
    uint8_t *c = (uint8_t *)host_out;
    uint8_t *dir = c + kHdr, *tok = dir + (uint64_t)kDirent * nb, *lit = tok + (uint64_t)kTok * nt;
    std::vector<uint64_t> bt(nb + 1), bl(nb + 1);
    cudaError_t e = cudaSuccess;
    if (nb) {
        e = cudaMemcpy(bt.data(), h->d_blk_tok, 8 * ((size_t)nb + 1), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(bl.data(), h->d_blk_lit, 8 * ((size_t)nb + 1), cudaMemcpyDeviceToHost);
    }
    if (e == cudaSuccess && nt) e = cudaMemcpy(tok, h->d_tok, kTok * nt, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && nl) e = cudaMemcpy(lit, h->d_lit, nl, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        note_cuda_error(e);
        return ACLZ_E_CUDA;
    }
    uint32_t waves = 0;  // the tags' wave count (the schedule may be flattened)
    for (uint64_t t = 0; t < nt; t++) waves = std::max(waves, (rd32(tok + kTok * t + 12) >> 8) + 1);
    const bool tagged = nt > 0;
    std::memset(c, 0, kHdr);
    c[0] = 'A'; c[1] = 'C'; c[2] = 'L'; c[3] = 'Z';
    wr16(c + 4, 1);
    wr16(c + 6, tagged ? kFlagWaves : 0);
    wr64(c + 8, h->total_len);
    wr32(c + 16, h->block_size);
    wr32(c + 20, nb);
    wr64(c + 24, nt);
    wr64(c + 32, nl);
    wr32(c + 40, tagged ? waves : 0);
    std::memcpy(c + 44, h->mm, 4);
    const uint32_t bounds[3] = {128, 16384, 2097152};
    for (int i = 0; i < 3; i++) wr32(c + 48 + 4 * i, bounds[i]);
    for (uint32_t b = 0; b < nb; b++) {
        uint8_t *d = dir + (uint64_t)kDirent * b;
        std::memset(d, 0, kDirent);
        wr64(d, bt[b]);
        wr64(d + 8, bl[b]);
        wr32(d + 16, (uint32_t)(bt[b + 1] - bt[b]));
        uint32_t mw = 0;
        for (uint64_t t = bt[b]; t < bt[b + 1]; t++) mw = std::max(mw, rd32(tok + kTok * t + 12) >> 8);
        wr16(d + 20, (uint16_t)std::min<uint32_t>(mw, 0xffffu));
        std::memcpy(d + 24, h->mm, 4);
    }
    return ACLZ_OK;
}
