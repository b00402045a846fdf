// Flattening: re-point every deferred match at the bytes its source copies
// from that are final after wave 0, so the whole decode is two waves.
//
// Back-references name absolute output positions (abstract; Sec. I), so a
// match whose source bytes were themselves written by another match can
// equally copy them from where that match read them: the bytes are equal.
// Chains of such copies are what forces the wavefront (Sec. I) to run many
// waves; on FASTQ-like data at 6/8/10/12 the chain crosses every LZ block
// (each record's header copies the previous one), so the wave count grows
// with the stream.  Flattening removes the chains at upload time: every
// deferred match becomes a list of pieces (offset in the match, length,
// source), each piece's source lying in literal bytes or in in-order
// (tag 0) match bytes.  Decode stays the same kernels: wave 0 writes
// literals and in-order matches, then one wave copies all pieces, which are
// independent.  The output bytes are unchanged.
//
// Pieces are found by pointer doubling.  Round r replaces each piece whose
// source overlaps deferred match bytes by the round r-1 pieces of those
// matches over the overlapped sub-range, so after r rounds a piece has
// skipped 2^r links of its chain; rounds stop when no piece overlaps
// deferred bytes (at most about log2(waves) + 1 rounds).  Each round counts
// the children of every piece, scans the counts and emits the children in
// order, so the pieces of a match stay contiguous and sorted by offset.
#include <algorithm>
#include <vector>

#include "aclz_device.cuh"
#include "aclz_internal.h"

using namespace aclz;

namespace {

struct FlatIdx {
    const uint4 *tok;
    const uint64_t *blk_tok;
    const uint32_t *tokdst;
    const uint32_t *defscan;  // per token: deferred matches before it
    const uint4 *P;           // pieces {offset in match, length, src lo, src hi}
    const uint64_t *off;      // per deferred match: first piece (D + 1 entries)
    uint32_t log2bs;
};

// Last token of block bp whose first byte is at or before block offset rel.
__device__ __forceinline__ uint64_t token_at(const FlatIdx &ix, uint64_t bp, uint32_t rel) {
    uint64_t lo = ix.blk_tok[bp], hi = ix.blk_tok[bp + 1] - 1;  // tokdst[lo] == 0 <= rel
    while (lo < hi) {
        const uint64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(ix.tokdst + mid) <= rel) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Visit the parts of source range [s, s + L) of a piece at offset o of its
// match: f(child offset, length, source, through_deferred).  Literal bytes
// and in-order match bytes are final; deferred match bytes are replaced by
// the current pieces of that match over the overlapped sub-range.
template <class F>
__device__ __forceinline__ bool walk(const FlatIdx &ix, uint32_t o, uint32_t L, uint64_t s, F &&f) {
    const uint64_t e = s + L;
    uint64_t bp = s >> ix.log2bs;
    uint64_t t = token_at(ix, bp, (uint32_t)(s - (bp << ix.log2bs)));
    uint64_t pos = s;
    bool deferred = false;
    while (pos < e) {
        while (t >= ix.blk_tok[bp + 1]) bp++;
        const uint4 tk = __ldg(ix.tok + t);
        const uint64_t ts = (bp << ix.log2bs) + __ldg(ix.tokdst + t);
        const uint64_t tl = ts + tk.x, te = tl + tk.y;
        if (pos < tl) {  // literal part
            const uint64_t n = (e < tl ? e : tl) - pos;
            f(o + (uint32_t)(pos - s), (uint32_t)n, pos, false);
            pos += n;
            continue;
        }
        if (pos < te) {
            const uint64_t n = (e < te ? e : te) - pos;
            const uint32_t tag = tk.w >> 8;
            if (tag == 0) {
                f(o + (uint32_t)(pos - s), (uint32_t)n, pos, false);
            } else {
                deferred = true;
                const uint32_t q = __ldg(ix.defscan + t);
                const uint64_t a = pos - tl, b = a + n;
                uint64_t lo = ix.off[q], hi = ix.off[q + 1];
                // first piece of q ending after a
                while (lo < hi) {
                    const uint64_t mid = (lo + hi) >> 1;
                    const uint4 pm = ix.P[mid];
                    if ((uint64_t)pm.x + pm.y <= a) lo = mid + 1; else hi = mid;
                }
                for (uint64_t j = lo; j < ix.off[q + 1]; j++) {
                    const uint4 pj = ix.P[j];
                    if (pj.x >= b) break;
                    const uint64_t x0 = a > pj.x ? a : pj.x;
                    const uint64_t x1 = b < (uint64_t)pj.x + pj.y ? b : (uint64_t)pj.x + pj.y;
                    const uint64_t ps = ((uint64_t)pj.z | ((uint64_t)pj.w << 32)) + (x0 - pj.x);
                    f(o + (uint32_t)(pos - s + (x0 - a)), (uint32_t)(x1 - x0), ps, true);
                }
            }
            pos += n;
        }
        t++;
    }
    return deferred;
}

// Round 0: one piece per deferred match, its end position, and the bytes.
__global__ void __launch_bounds__(256) k_fl_init(const uint4 *__restrict__ tok, const uint64_t *__restrict__ blk_tok,
                                                 const uint32_t *__restrict__ tokdst,
                                                 const uint32_t *__restrict__ defscan, uint32_t nb, uint32_t log2bs,
                                                 uint4 *P, uint32_t *owner, uint64_t *off, uint64_t *dmk,
                                                 unsigned long long *bytes) {
    const uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= nb) return;
    unsigned long long acc = 0;
    for (uint64_t t = blk_tok[b] + lane; t < blk_tok[b + 1]; t += 32) {
        const uint4 tk = __ldg(tok + t);
        if (!tk.y || !(tk.w >> 8)) continue;
        const uint32_t k = defscan[t];
        P[k] = make_uint4(0u, tk.y, tk.z, tk.w & 0xffu);
        owner[k] = k;
        off[k] = k;
        dmk[k] = ((uint64_t)b << log2bs) + tokdst[t] + tk.x;
        acc += tk.y;
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0 && acc) atomicAdd(bytes, acc);
}

__global__ void k_is_deferred(const uint4 *__restrict__ tok, uint64_t nt, uint32_t *flag) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < nt; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 tk = __ldg(tok + t);
        flag[t] = (tk.y && (tk.w >> 8)) ? 1u : 0u;
    }
}

__global__ void k_fl_count(FlatIdx ix, uint64_t np, uint32_t *cnt, uint32_t *any_def) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < np; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 p = ix.P[i];
        uint32_t c = 0;
        const bool d = walk(ix, p.x, p.y, (uint64_t)p.z | ((uint64_t)p.w << 32),
                            [&](uint32_t, uint32_t, uint64_t, bool) { c++; });
        cnt[i] = c;
        if (d) *any_def = 1u;
    }
}

__global__ void k_fl_emit(FlatIdx ix, uint64_t np, const uint32_t *__restrict__ pos, const uint32_t *__restrict__ owner,
                          uint4 *P2, uint32_t *owner2) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < np; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 p = ix.P[i];
        uint64_t w = pos[i];
        const uint32_t ow = owner[i];
        walk(ix, p.x, p.y, (uint64_t)p.z | ((uint64_t)p.w << 32), [&](uint32_t o, uint32_t n, uint64_t s, bool) {
            P2[w] = make_uint4(o, n, (uint32_t)s, (uint32_t)(s >> 32));
            owner2[w] = ow;
            w++;
        });
    }
}

// new first piece of every match: the scanned position of its old first
// piece (off[D] = np maps to the new total)
__global__ void k_fl_off(const uint64_t *__restrict__ off, uint64_t D, uint64_t np, const uint32_t *__restrict__ pos,
                         const uint32_t *__restrict__ total, uint64_t *off2) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k <= D; k += (uint64_t)gridDim.x * blockDim.x)
        off2[k] = off[k] < np ? pos[off[k]] : *total;
}

// pieces -> decode triplets {dst:40, src:40, len:24}
__global__ void k_fl_tri(const uint4 *__restrict__ P, const uint32_t *__restrict__ owner,
                         const uint64_t *__restrict__ dmk, uint64_t np, uint4 *tri) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < np; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 p = P[i];
        const uint64_t d = dmk[owner[i]] + p.x;
        tri[i] = make_uint4((uint32_t)d, (uint32_t)(d >> 32) & 0xffu, p.z, (p.w & 0xffu) | (p.y << 8));
    }
}

// per block: its pieces [off[first deferred match], off[last + 1]) and the
// segment flag; pending bits = wave 0, plus wave 1 when it has pieces
__global__ void k_fl_blocks(const uint64_t *__restrict__ blk_tok, const uint32_t *__restrict__ defscan,
                            const uint64_t *__restrict__ off, uint32_t nb, uint32_t *flag, uint64_t *pending) {
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const uint64_t c = off[defscan[blk_tok[b + 1]]] - off[defscan[blk_tok[b]]];
        flag[b] = c ? 1u : 0u;
        pending[b] = 1ULL | (c ? 2ULL : 0ULL);
    }
}

__global__ void k_fl_segs(const uint64_t *__restrict__ blk_tok, const uint32_t *__restrict__ defscan,
                          const uint64_t *__restrict__ off, const uint32_t *__restrict__ pos, uint32_t nb,
                          uint4 *seg) {
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const uint64_t a = off[defscan[blk_tok[b]]], e = off[defscan[blk_tok[b + 1]]];
        if (e > a) seg[pos[b]] = make_uint4(b, 1u, (uint32_t)a, (uint32_t)(e - a));
    }
}

struct Dev {
    void *p = nullptr;
    ~Dev() {
        if (p) cudaFree(p);
    }
    template <class T>
    T *as() const {
        return (T *)p;
    }
};

int rc_of(cudaError_t e) {
    if (e == cudaSuccess) return ACLZ_OK;
    note_cuda_error((int)e);
    return e == cudaErrorMemoryAllocation ? ACLZ_E_NOMEM : ACLZ_E_CUDA;
}

#define FCK(x)                       \
    do {                             \
        int _rc = rc_of(x);          \
        if (_rc) return _rc;         \
    } while (0)

unsigned grid_for(uint64_t n) { return (unsigned)std::min<uint64_t>((n + 255) / 256, 152ull * 32); }

// Pieces of every deferred match after up to max_rounds doubling rounds
// (fewer when no piece overlaps deferred bytes any more: final).
struct Pieces {
    Dev defscan, P, owner, off, dmk;
    uint64_t np = 0, D = 0;
    unsigned long long def_bytes = 0;
    bool final = false;
};

int make_pieces(aclz_handle *h, cudaStream_t st, int max_rounds, Pieces &pc) {
    const uint64_t nt = h->n_tokens;
    const uint32_t nb = h->n_blocks;
    // deferred matches in token order: defscan[t] = rank, defscan[nt] = D
    Dev work;
    FCK(cudaMalloc(&pc.defscan.p, 4 * (nt + 1)));
    FCK(cudaMalloc(&work.p, 64));
    uint32_t *d_any = work.as<uint32_t>(), *d_total = work.as<uint32_t>() + 1;
    unsigned long long *d_bytes = (unsigned long long *)(work.as<char>() + 8);
    FCK(cudaMemsetAsync(work.p, 0, 64, st));
    k_is_deferred<<<grid_for(nt), 256, 0, st>>>((const uint4 *)h->d_tok, nt, pc.defscan.as<uint32_t>());
    FCK(cudaGetLastError());
    if (int rc = device_excl_scan(pc.defscan.as<uint32_t>(), nt, pc.defscan.as<uint32_t>() + nt, st)) return rc;
    uint32_t d32 = 0;
    FCK(cudaMemcpyAsync(&d32, pc.defscan.as<uint32_t>() + nt, 4, cudaMemcpyDeviceToHost, st));
    FCK(cudaStreamSynchronize(st));
    const uint64_t D = d32;
    pc.D = D;
    if (D == 0) return ACLZ_OK;
    // round 0: one piece per match
    uint64_t np = D;
    FCK(cudaMalloc(&pc.P.p, 16 * np));
    FCK(cudaMalloc(&pc.owner.p, 4 * np));
    FCK(cudaMalloc(&pc.off.p, 8 * (D + 1)));
    FCK(cudaMalloc(&pc.dmk.p, 8 * D));
    FCK(cudaMemcpyAsync(pc.off.as<uint64_t>() + D, &np, 8, cudaMemcpyHostToDevice, st));
    k_fl_init<<<(nb + 7) / 8, 256, 0, st>>>((const uint4 *)h->d_tok, h->d_blk_tok, h->d_tokdst,
                                             pc.defscan.as<uint32_t>(), nb, h->log2_bs, pc.P.as<uint4>(),
                                             pc.owner.as<uint32_t>(), pc.off.as<uint64_t>(), pc.dmk.as<uint64_t>(),
                                             d_bytes);
    FCK(cudaGetLastError());
    FCK(cudaMemcpyAsync(&pc.def_bytes, d_bytes, 8, cudaMemcpyDeviceToHost, st));
    pc.final = false;
    for (int round = 0;; round++) {
        if (round > 64) return ACLZ_E_UNSUPPORTED;
        FlatIdx ix{(const uint4 *)h->d_tok, h->d_blk_tok, h->d_tokdst, pc.defscan.as<uint32_t>(), pc.P.as<uint4>(),
                   pc.off.as<uint64_t>(), h->log2_bs};
        Dev cnt;
        FCK(cudaMalloc(&cnt.p, 4 * np + 4));
        FCK(cudaMemsetAsync(d_any, 0, 4, st));
        k_fl_count<<<grid_for(np), 256, 0, st>>>(ix, np, cnt.as<uint32_t>(), d_any);
        FCK(cudaGetLastError());
        uint32_t any = 0;
        FCK(cudaMemcpyAsync(&any, d_any, 4, cudaMemcpyDeviceToHost, st));
        FCK(cudaStreamSynchronize(st));
        if (!any) {
            pc.final = true;
            break;
        }
        if (round >= max_rounds) break;
        if (int rc = device_excl_scan(cnt.as<uint32_t>(), np, d_total, st)) return rc;
        uint32_t total = 0;
        FCK(cudaMemcpyAsync(&total, d_total, 4, cudaMemcpyDeviceToHost, st));
        FCK(cudaStreamSynchronize(st));
        if (total >= 0xfffffff0u) return ACLZ_E_UNSUPPORTED;
        Dev P2, owner2, off2;
        FCK(cudaMalloc(&P2.p, 16 * (uint64_t)total));
        FCK(cudaMalloc(&owner2.p, 4 * (uint64_t)total));
        FCK(cudaMalloc(&off2.p, 8 * (D + 1)));
        k_fl_emit<<<grid_for(np), 256, 0, st>>>(ix, np, cnt.as<uint32_t>(), pc.owner.as<uint32_t>(),
                                                 P2.as<uint4>(), owner2.as<uint32_t>());
        k_fl_off<<<grid_for(D + 1), 256, 0, st>>>(pc.off.as<uint64_t>(), D, np, cnt.as<uint32_t>(), d_total,
                                                   off2.as<uint64_t>());
        FCK(cudaGetLastError());
        FCK(cudaStreamSynchronize(st));
        std::swap(pc.P.p, P2.p);
        std::swap(pc.owner.p, owner2.p);
        std::swap(pc.off.p, off2.p);
        np = total;
    }
    pc.np = np;
    return ACLZ_OK;
}

}  // namespace

extern "C" int aclz_flatten(aclz_handle *h, void *stream) {
    if (!h) return ACLZ_E_INVAL;
    if (h->flat) return ACLZ_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t nb = h->n_blocks;
    if (nb == 0) {
        h->flat = true;
        return ACLZ_OK;
    }
    Pieces pc;
    if (int rc = make_pieces(h, st, 1 << 30, pc)) return rc;
    const uint64_t D = pc.D;
    if (D == 0) {  // nothing deferred: the schedule is wave 0 alone
        h->flat = true;
        return ACLZ_OK;
    }
    Dev &defscan = pc.defscan, &P = pc.P, &owner = pc.owner, &off = pc.off, &dmk = pc.dmk;
    const uint64_t np = pc.np;
    const unsigned long long def_bytes = pc.def_bytes;
    // the two-wave schedule: triplets, per-block segments, pending bits
    Dev tri, bflag, seg, pending, done;
    FCK(cudaMalloc(&tri.p, 16 * np));
    k_fl_tri<<<grid_for(np), 256, 0, st>>>(P.as<uint4>(), owner.as<uint32_t>(), dmk.as<uint64_t>(), np,
                                            tri.as<uint4>());
    FCK(cudaMalloc(&bflag.p, 4 * ((uint64_t)nb + 1)));
    FCK(cudaMalloc(&pending.p, 8 * (uint64_t)nb));
    FCK(cudaMalloc(&done.p, 8 * (uint64_t)nb));
    k_fl_blocks<<<grid_for(nb), 256, 0, st>>>(h->d_blk_tok, defscan.as<uint32_t>(), off.as<uint64_t>(), nb,
                                               bflag.as<uint32_t>(), pending.as<uint64_t>());
    FCK(cudaGetLastError());
    if (int rc = device_excl_scan(bflag.as<uint32_t>(), nb, bflag.as<uint32_t>() + nb, st)) return rc;
    uint32_t nseg = 0;
    FCK(cudaMemcpyAsync(&nseg, bflag.as<uint32_t>() + nb, 4, cudaMemcpyDeviceToHost, st));
    FCK(cudaStreamSynchronize(st));
    FCK(cudaMalloc(&seg.p, 16 * (uint64_t)(nseg ? nseg : 1)));
    k_fl_segs<<<grid_for(nb), 256, 0, st>>>(h->d_blk_tok, defscan.as<uint32_t>(), off.as<uint64_t>(),
                                             bflag.as<uint32_t>(), nb, seg.as<uint4>());
    FCK(cudaGetLastError());
    FCK(cudaStreamSynchronize(st));
    // install
    cudaFree(h->d_tri);
    cudaFree(h->d_seg);
    cudaFree(h->d_pending);
    cudaFree(h->d_done);
    h->d_tri = tri.p;
    tri.p = nullptr;
    h->d_seg = seg.p;
    seg.p = nullptr;
    h->d_pending = pending.as<uint64_t>();
    pending.p = nullptr;
    h->d_done = done.as<uint64_t>();
    done.p = nullptr;
    h->n_seg = nseg;
    h->n_wave_words = 1;
    h->n_matches_deferred = D;
    h->n_deferred = np;
    h->n_waves = 2;
    h->wave_start.assign(3, 0);
    h->wave_start[2] = np;
    h->mean_deferred_len = (double)def_bytes / (double)np;
    h->flat = true;
    return aclz_set_range_bytes(h, h->range_bytes, stream);
}

// ------------------------------------------------------------- reshape
//
// Shorter chains for the wavefront schedule itself: a few doubling rounds,
// then every deferred match is written back as consecutive tokens, one per
// piece (the first keeps the match's literal run, the others have none), and
// the decode index (minimal tags, worklists, persistent schedule) is rebuilt
// for the new token array.  Each piece copies the same bytes from an earlier
// copy of them, so its source still lies strictly before it and within the
// stream; the thresholds by distance class no longer hold for the new
// tokens, and the decode does not need them.

namespace {

__global__ void k_rs_count(const uint4 *__restrict__ tok, const uint32_t *__restrict__ defscan,
                           const uint64_t *__restrict__ off, uint64_t nt, uint32_t *cnt) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < nt; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 tk = __ldg(tok + t);
        if (tk.y && (tk.w >> 8)) {
            const uint32_t q = defscan[t];
            cnt[t] = (uint32_t)(off[q + 1] - off[q]);
        } else {
            cnt[t] = 1u;
        }
    }
}

__global__ void k_rs_emit(const uint4 *__restrict__ tok, const uint32_t *__restrict__ defscan,
                          const uint64_t *__restrict__ off, const uint4 *__restrict__ P,
                          const uint32_t *__restrict__ pos, uint64_t nt, uint4 *tok2) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < nt; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 tk = __ldg(tok + t);
        uint64_t w = pos[t];
        if (tk.y && (tk.w >> 8)) {
            const uint32_t q = defscan[t];
            for (uint64_t j = off[q]; j < off[q + 1]; j++, w++) {
                const uint4 p = P[j];
                tok2[w] = make_uint4(j == off[q] ? tk.x : 0u, p.y, p.z, p.w & 0xffu);
            }
        } else {
            tok2[w] = make_uint4(tk.x, tk.y, tk.z, tk.w & 0xffu);
        }
    }
}

__global__ void k_rs_blk(const uint64_t *__restrict__ blk_tok, const uint32_t *__restrict__ pos, uint32_t nb,
                         uint64_t nt2, uint64_t *blk_tok2) {
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b <= nb; b += gridDim.x * blockDim.x)
        blk_tok2[b] = b < nb ? pos[blk_tok[b]] : nt2;
}

}  // namespace

extern "C" int aclz_reshape(aclz_handle *h, uint32_t rounds, void *stream) {
    if (!h || h->flat) return ACLZ_E_INVAL;
    if (rounds == 0 || h->n_deferred == 0) return ACLZ_OK;
    if (rounds > 32) return ACLZ_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t nt = h->n_tokens;
    const uint32_t nb = h->n_blocks;
    Pieces pc;
    if (int rc = make_pieces(h, st, (int)rounds, pc)) return rc;
    if (pc.D == 0) return ACLZ_OK;
    Dev cnt, tok2, blk2;
    FCK(cudaMalloc(&cnt.p, 4 * (nt + 1)));
    k_rs_count<<<grid_for(nt), 256, 0, st>>>((const uint4 *)h->d_tok, pc.defscan.as<uint32_t>(), pc.off.as<uint64_t>(),
                                              nt, cnt.as<uint32_t>());
    FCK(cudaGetLastError());
    if (int rc = device_excl_scan(cnt.as<uint32_t>(), nt, cnt.as<uint32_t>() + nt, st)) return rc;
    uint32_t nt2 = 0;
    FCK(cudaMemcpyAsync(&nt2, cnt.as<uint32_t>() + nt, 4, cudaMemcpyDeviceToHost, st));
    FCK(cudaStreamSynchronize(st));
    if (nt2 >= 0xfffffff0u) return ACLZ_E_UNSUPPORTED;
    FCK(cudaMalloc(&tok2.p, 16 * (uint64_t)nt2));
    FCK(cudaMalloc(&blk2.p, 8 * ((uint64_t)nb + 1)));
    k_rs_emit<<<grid_for(nt), 256, 0, st>>>((const uint4 *)h->d_tok, pc.defscan.as<uint32_t>(), pc.off.as<uint64_t>(),
                                             pc.P.as<uint4>(), cnt.as<uint32_t>(), nt, tok2.as<uint4>());
    k_rs_blk<<<grid_for(nb + 1), 256, 0, st>>>(h->d_blk_tok, cnt.as<uint32_t>(), nb, nt2, blk2.as<uint64_t>());
    FCK(cudaGetLastError());
    FCK(cudaStreamSynchronize(st));
    cudaFree(h->d_tok);
    cudaFree(h->d_blk_tok);
    h->d_tok = tok2.p;
    tok2.p = nullptr;
    h->d_blk_tok = blk2.as<uint64_t>();
    blk2.p = nullptr;
    h->n_tokens = nt2;
    h->flags &= (uint16_t)~kFlagWaves;
    return build_index(h, false, 0, false, stream);
}
