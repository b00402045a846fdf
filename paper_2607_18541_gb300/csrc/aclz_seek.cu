// Range decode (seek): out = decode(x)[lo, hi) without decoding the rest.
//
// Absolute back-references make any output byte resolvable on its own
// (abstract; Sec. I: a region of the stream can be read without decoding
// the whole of it).  A byte inside a match at position p comes from
// src + (p - dst); following that chain always moves strictly backwards and
// ends in a literal.  The range is cut into segments of at most kSeg0
// bytes; each warp resolves its segments depth first with a stack in
// shared memory: it finds the tokens covering a segment, copies the
// literal pieces straight from the literal array, and pushes each match
// piece remapped to its absolute source.  Only literals are ever read, so
// requests never wait on one another or on a full decode.
//
// Stack bound: a popped segment is replaced by pieces whose lengths sum to
// at most its own, so the total length on a stack never exceeds the first
// segment's (kSeg0) and, every piece holding at least one byte, neither
// does the number of entries.
#include <algorithm>
#include <cstring>
#include <vector>

#include "aclz_device.cuh"
#include "aclz_internal.h"

using namespace aclz;

namespace {

constexpr int kSeekThreads = 256;
constexpr int kSeekWarps = kSeekThreads / 32;
constexpr uint32_t kSeg0 = 256;
constexpr uint32_t kStack = kSeg0 + 8;

// One request: output [lo, hi) into out; seg_base = initial segments of
// the requests before it.
struct SeekReq {
    uint64_t lo, hi;
    uint8_t *out;
    uint64_t seg_base;
};

struct SeekIndex {
    const uint4 *tok;
    const uint8_t *lit;
    const uint64_t *blk_tok, *blk_lit;
    const uint32_t *tokdst, *toklit;
    uint64_t n_tok;
    uint32_t log2bs;
};

// Last token of block bp whose first byte is at or before block offset rel
// (warp-parallel 32-ary search).
__device__ __forceinline__ uint64_t find_token(const SeekIndex &ix, uint64_t bp, uint32_t rel, int lane) {
    uint64_t lo = ix.blk_tok[bp], hi = ix.blk_tok[bp + 1];  // answer in [lo, hi)
    while (hi - lo > 32) {
        const uint64_t step = (hi - lo + 31) / 32;
        const uint64_t p = lo + (uint64_t)lane * step;
        const bool ok = p < hi && __ldg(ix.tokdst + p) <= rel;
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        const int j = 31 - __clz(m);  // lane 0 always qualifies (tokdst[lo] == 0 <= rel)
        lo = lo + (uint64_t)j * step;
        hi = min(hi, lo + step);
    }
    const uint64_t p = lo + (uint64_t)lane;
    const bool ok = p < hi && __ldg(ix.tokdst + p) <= rel;
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    return lo + (uint64_t)(31 - __clz(m));
}

__global__ void __launch_bounds__(kSeekThreads) k_seek(const SeekReq *__restrict__ reqs, SeekReq one,
                                                       uint32_t nreq, uint64_t nseg, SeekIndex ix,
                                                       uint32_t *err) {
    __shared__ uint4 stack[kSeekWarps][kStack];
    Group<32> g;
    const int wl = threadIdx.x >> 5;
    uint4 *stk = stack[wl];
    const uint64_t nw = (uint64_t)gridDim.x * kSeekWarps;
    bool overflow = false;
    for (uint64_t gs = blockIdx.x * (uint64_t)kSeekWarps + wl; gs < nseg; gs += nw) {
        // the request holding initial segment gs
        SeekReq rq = one;
        if (nreq > 1) {
            uint32_t lo = 0, hi = nreq - 1;
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (__ldg(&reqs[mid].seg_base) <= gs) lo = mid; else hi = mid - 1;
            }
            rq = reqs[lo];
        }
        const uint64_t a0 = rq.lo + (gs - rq.seg_base) * kSeg0;
        const uint64_t b0 = min(a0 + kSeg0, rq.hi);
        // stack entries: {a lo, a hi, len, out offset}
        uint32_t sp = 0;
        if (g.lane == 0)
            stk[0] = make_uint4((uint32_t)a0, (uint32_t)(a0 >> 32), (uint32_t)(b0 - a0), (uint32_t)(a0 - rq.lo));
        sp = 1;
        __syncwarp();
        while (sp) {
            sp--;
            const uint4 e = stk[sp];
            __syncwarp();
            const uint64_t a = (uint64_t)e.x | ((uint64_t)e.y << 32);
            const uint64_t b = a + e.z;
            const uint32_t oo = e.w;
            uint64_t bp = a >> ix.log2bs;
            uint64_t t = find_token(ix, bp, (uint32_t)(a - (bp << ix.log2bs)), g.lane);
            for (;;) {
                const uint64_t ti = t + (uint64_t)g.lane;
                bool v = ti < ix.n_tok;
                uint64_t bb = bp, ts = ~0ULL, te = 0;
                uint4 tk = make_uint4(0, 0, 0, 0);
                if (v) {
                    while (ti >= __ldg(ix.blk_tok + bb + 1)) bb++;
                    ts = (bb << ix.log2bs) + __ldg(ix.tokdst + ti);
                    tk = __ldg(ix.tok + ti);
                    te = ts + tk.x + tk.y;
                    v = ts < b;
                }
                // literal piece
                uint32_t ln = 0;
                uint64_t ld = 0;
                const uint8_t *ls = ix.lit;
                if (v && tk.x) {
                    const uint64_t x = max(ts, a), y = min(ts + tk.x, b);
                    if (y > x) {
                        ln = (uint32_t)(y - x);
                        ld = oo + (x - a);
                        ls = ix.lit + __ldg(ix.blk_lit + bb) + __ldg(ix.toklit + ti) + (x - ts);
                    }
                }
                group_copy<32, 2>(g, rq.out, ld, ls, ln);
                // match piece: push its source
                bool push = false;
                uint4 ne = make_uint4(0, 0, 0, 0);
                if (v && tk.y) {
                    const uint64_t m0 = ts + tk.x;
                    const uint64_t x = max(m0, a), y = min(m0 + tk.y, b);
                    if (y > x) {
                        const uint64_t src = ((uint64_t)tk.z | ((uint64_t)(tk.w & 0xffu) << 32)) + (x - m0);
                        ne = make_uint4((uint32_t)src, (uint32_t)(src >> 32), (uint32_t)(y - x),
                                        oo + (uint32_t)(x - a));
                        push = true;
                    }
                }
                const unsigned pm = g.ballot(push);
                const uint32_t cnt = __popc(pm);
                if (sp + cnt > kStack) {
                    overflow = true;
                } else if (push) {
                    stk[sp + __popc(pm & g.lanemask_lt())] = ne;
                }
                sp = min(sp + cnt, kStack);
                __syncwarp();
                // more tokens needed when every lane's token ended before b
                const bool more = g.ballot(v && te < b) == 0xffffffffu;
                if (!more) break;
                t += 32;
            }
        }
    }
    if (g.ballot(overflow) && g.lane == 0) atomicOr(err, kErrBounds);
}

int seek_launch(aclz_handle *h, const SeekReq *d_reqs, const SeekReq &one, uint32_t nreq, uint64_t nseg,
                cudaStream_t st) {
    if (!nseg) return ACLZ_OK;
    // SM count and resident CTAs, found once (thread-safe static init)
    static const uint64_t slots = [] {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_seek, kSeekThreads, 0);
        return (uint64_t)std::max(sms, 1) * (uint64_t)std::max(per_sm, 1);
    }();
    const uint64_t need = (nseg + kSeekWarps - 1) / kSeekWarps;
    const unsigned grid = (unsigned)std::min<uint64_t>(slots, need);
    SeekIndex ix;
    ix.tok = (const uint4 *)h->d_tok;
    ix.lit = h->d_lit;
    ix.blk_tok = h->d_blk_tok;
    ix.blk_lit = h->d_blk_lit;
    ix.tokdst = h->d_tokdst;
    ix.toklit = h->d_toklit;
    ix.n_tok = h->n_tokens;
    ix.log2bs = h->log2_bs;
    k_seek<<<grid, kSeekThreads, 0, st>>>(d_reqs, one, nreq, nseg, ix, h->d_err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        note_cuda_error(e);
        return ACLZ_E_CUDA;
    }
    return ACLZ_OK;
}

}  // namespace

extern "C" int aclz_decode_range(aclz_handle *h, uint64_t lo, uint64_t hi, void *d_out, void *stream) {
    if (!h) return ACLZ_E_INVAL;
    if (lo > hi || hi > h->total_len) return ACLZ_E_INVAL;
    if (hi == lo) return ACLZ_OK;
    if (!d_out || (reinterpret_cast<uintptr_t>(d_out) & 15)) return ACLZ_E_INVAL;
    if (hi - lo >= (1ULL << 32)) return ACLZ_E_UNSUPPORTED;
    SeekReq one;
    one.lo = lo;
    one.hi = hi;
    one.out = (uint8_t *)d_out;
    one.seg_base = 0;
    const uint64_t nseg = (hi - lo + kSeg0 - 1) / kSeg0;
    return seek_launch(h, nullptr, one, 1, nseg, (cudaStream_t)stream);
}

extern "C" int aclz_ranges_scratch_bytes(uint32_t n_requests, uint64_t *out) {
    if (!out) return ACLZ_E_INVAL;
    *out = (uint64_t)n_requests * sizeof(SeekReq);
    return ACLZ_OK;
}

extern "C" int aclz_decode_ranges(aclz_handle *h, uint32_t n, const uint64_t *host_lo, const uint64_t *host_hi,
                                  void *const *host_out, void *d_scratch, uint64_t scratch_cap, void *stream) {
    if (!h || (n && (!host_lo || !host_hi || !host_out))) return ACLZ_E_INVAL;
    if (n == 0) return ACLZ_OK;
    if ((uint64_t)n * sizeof(SeekReq) > scratch_cap) return ACLZ_E_CAPACITY;
    if (!d_scratch || (reinterpret_cast<uintptr_t>(d_scratch) & 15)) return ACLZ_E_INVAL;
    std::vector<SeekReq> rq;
    rq.reserve(n);
    uint64_t nseg = 0;
    for (uint32_t i = 0; i < n; i++) {
        const uint64_t lo = host_lo[i], hi = host_hi[i];
        if (lo > hi || hi > h->total_len) return ACLZ_E_INVAL;
        if (hi - lo >= (1ULL << 32)) return ACLZ_E_UNSUPPORTED;
        if (hi > lo && (!host_out[i] || (reinterpret_cast<uintptr_t>(host_out[i]) & 15))) return ACLZ_E_INVAL;
        SeekReq r;
        r.lo = lo;
        r.hi = hi;
        r.out = (uint8_t *)host_out[i];
        r.seg_base = nseg;
        nseg += (hi - lo + kSeg0 - 1) / kSeg0;
        rq.push_back(r);
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(d_scratch, rq.data(), sizeof(SeekReq) * n, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return ACLZ_E_CUDA;
    // the host table must outlive the copy
    if (cudaStreamSynchronize(st) != cudaSuccess) return ACLZ_E_CUDA;
    return seek_launch(h, (const SeekReq *)d_scratch, rq[0], n, nseg, st);
}

extern "C" int aclz_decode_ranges_async(aclz_handle *h, uint32_t n, aclz_range_req *reqs, void *stream) {
    static_assert(sizeof(aclz_range_req) == sizeof(SeekReq), "request layout");
    if (!h || (n && !reqs)) return ACLZ_E_INVAL;
    if (n == 0) return ACLZ_OK;
    uint64_t nseg = 0;
    for (uint32_t i = 0; i < n; i++) {
        aclz_range_req &r = reqs[i];
        if (r.lo > r.hi || r.hi > h->total_len) return ACLZ_E_INVAL;
        if (r.hi - r.lo >= (1ULL << 32)) return ACLZ_E_UNSUPPORTED;
        if (r.hi > r.lo && (!r.d_out || (reinterpret_cast<uintptr_t>(r.d_out) & 15))) return ACLZ_E_INVAL;
        r.seg_base = nseg;
        nseg += (r.hi - r.lo + kSeg0 - 1) / kSeg0;
    }
    const SeekReq *dev = reinterpret_cast<const SeekReq *>(reqs);
    SeekReq first;
    std::memcpy(&first, reqs, sizeof(first));
    return seek_launch(h, dev, first, n, nseg, (cudaStream_t)stream);
}
