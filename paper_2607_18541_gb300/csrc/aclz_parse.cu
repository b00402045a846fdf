// Greedy parse on the GPU: the container the host encoder writes (greedy
// longest match over exact 4-byte-prefix chains, nearest on ties, minimum
// length by distance class), built from the input bytes by kernels.
//
// The chains do not depend on the parse: every earlier position with the
// same 4-byte prefix is a candidate, nearest first.  Sorting the positions
// by (prefix, position) therefore lays every chain out contiguously, so the
// candidates of position p are the entries just before p in that order.
// The parse itself is sequential only within an LZ block (a match never
// crosses its block's end), so one warp parses each block, its lanes
// scoring up to 32 candidates at a time.
//
//  1. k_keys          prefix of every position with 4 bytes left
//  2. radix sort      stable, 8-bit digits: k_rs_hist, exclusive scan,
//                     k_rs_scatter (4 passes)
//  3. k_rank          rank of each position in the sorted order
//  4. k_parse_blocks  one warp per block: greedy walk, tokens to a per-block
//                     slot array
//  5. scans of the per-block token and literal counts, then k_emit writes
//     the directory, the tokens and the literal bytes of the container
#include <algorithm>
#include <cstring>
#include <vector>

#include "aclz_device.cuh"
#include "aclz_internal.h"

using namespace aclz;

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr uint32_t kSortPerWarp = 512;                        // 16 chunks of 32
constexpr uint32_t kSortTile = kSortWarps * kSortPerWarp;    // 4096 elements per CTA

__global__ void k_keys(const uint8_t *__restrict__ x, uint64_t m, uint32_t *__restrict__ key,
                       uint32_t *__restrict__ val) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < m;
         p += (uint64_t)gridDim.x * blockDim.x) {
        key[p] = (uint32_t)x[p] | ((uint32_t)x[p + 1] << 8) | ((uint32_t)x[p + 2] << 16) |
                 ((uint32_t)x[p + 3] << 24);
        val[p] = (uint32_t)p;
    }
}

// Digit counts of one tile, digit-major: hist[d * ntiles + tile].
__global__ void __launch_bounds__(kSortThreads) k_rs_hist(const uint32_t *__restrict__ key, uint64_t m, int shift,
                                                          uint32_t ntiles, uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t a = (uint64_t)blockIdx.x * kSortTile;
    for (uint32_t k = threadIdx.x; k < kSortTile; k += kSortThreads)
        if (a + k < m) atomicAdd(&h[(key[a + k] >> shift) & 255u], 1u);
    __syncthreads();
    hist[(uint64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile: element i of the tile goes to
// base[digit][tile] + (number of earlier elements of the tile with the same
// digit).  Each warp owns 512 consecutive elements, walked 32 at a time in
// order; equal digits within 32 are ranked by lane.
__global__ void __launch_bounds__(kSortThreads) k_rs_scatter(const uint32_t *__restrict__ key,
                                                             const uint32_t *__restrict__ val, uint64_t m, int shift,
                                                             uint32_t ntiles, const uint32_t *__restrict__ base,
                                                             uint32_t *__restrict__ key_out,
                                                             uint32_t *__restrict__ val_out) {
    __shared__ uint32_t cnt[kSortWarps][256];
    const int w = threadIdx.x / 32, lane = threadIdx.x & 31;
    for (int d = lane; d < 256; d += 32) cnt[w][d] = 0;
    __syncwarp();
    const uint64_t a = (uint64_t)blockIdx.x * kSortTile + (uint64_t)w * kSortPerWarp;
    // digit counts of this warp's elements
    for (uint32_t c = 0; c < kSortPerWarp; c += 32) {
        const uint64_t i = a + c + lane;
        const bool v = i < m;
        const uint32_t d = v ? (key[i] >> shift) & 255u : 256u + lane;  // invalid lanes get private keys
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (v && lane == __ffs(peers) - 1) cnt[w][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps, per digit, plus the tile's global base
    {
        const uint32_t d = threadIdx.x;
        uint32_t run = base[(uint64_t)d * ntiles + blockIdx.x];
        for (int k = 0; k < kSortWarps; k++) {
            const uint32_t c = cnt[k][d];
            cnt[k][d] = run;
            run += c;
        }
    }
    __syncthreads();
    for (uint32_t c = 0; c < kSortPerWarp; c += 32) {
        const uint64_t i = a + c + lane;
        const bool v = i < m;
        const uint32_t kk = v ? key[i] : 0u;
        const uint32_t d = v ? (kk >> shift) & 255u : 256u + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (v) {
            const uint32_t dst = cnt[w][d] + __popc(peers & ((1u << lane) - 1u));
            key_out[dst] = kk;
            val_out[dst] = val[i];
        }
        __syncwarp();
        if (v && lane == __ffs(peers) - 1) cnt[w][d] += __popc(peers);
        __syncwarp();
    }
}

__global__ void k_rank(const uint32_t *__restrict__ val_s, uint64_t m, uint32_t *__restrict__ rank) {
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < m;
         r += (uint64_t)gridDim.x * blockDim.x)
        rank[val_s[r]] = (uint32_t)r;
}

// 8 bytes at a (little endian) from two aligned words; needs a + 16 <= the
// padded end of the buffer.
__device__ __forceinline__ uint64_t ld8u(const uint8_t *a) {
    const uintptr_t u = reinterpret_cast<uintptr_t>(a);
    const uint64_t *w = reinterpret_cast<const uint64_t *>(u & ~(uintptr_t)7);
    const uint32_t sh = (uint32_t)(u & 7) * 8;
    const uint64_t lo = w[0];
    if (!sh) return lo;
    return (lo >> sh) | (w[1] << (64 - sh));
}

// Common prefix of x[q..] and x[p..], at most lim bytes (q < p).
__device__ __forceinline__ uint32_t common_len(const uint8_t *x, uint64_t q, uint64_t p, uint32_t lim) {
    uint32_t len = 0;
    while (len + 8 <= lim) {
        const uint64_t a = ld8u(x + q + len), b = ld8u(x + p + len);
        if (a != b) return len + (uint32_t)(__ffsll((long long)(a ^ b)) - 1) / 8;
        len += 8;
    }
    while (len < lim && x[q + len] == x[p + len]) len++;
    return len;
}

__device__ __forceinline__ int dclass(uint64_t d) { return d < 128 ? 0 : d < 16384 ? 1 : d < 2097152 ? 2 : 3; }

struct TokOut {
    uint32_t lit, len;
    uint64_t src;
};

// One warp per block: the greedy walk.  Candidates of p: the entries
// rank[p] - 1, rank[p] - 2, ... of the sorted order while their prefix is
// p's, at most depth of them and no farther than window; the longest whose
// length (capped at the distance and the block end) meets its distance
// class minimum wins, the nearest on ties.  Tokens go to
// slots[b * cap_tok ...]; ntok[b] and nlit[b] receive the counts.
__global__ void __launch_bounds__(256) k_parse_blocks(const uint8_t *__restrict__ x, uint64_t n, uint32_t bs,
                                                      uint32_t nb, const uint32_t *__restrict__ key_s,
                                                      const uint32_t *__restrict__ val_s,
                                                      const uint32_t *__restrict__ rank, const uint8_t *mm,
                                                      const uint8_t *__restrict__ block_mm, uint32_t depth,
                                                      uint64_t window, uint32_t cap_tok, TokOut *__restrict__ slots,
                                                      uint32_t *__restrict__ ntok, uint32_t *__restrict__ nlit) {
    const uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= nb) return;
    const uint8_t *Tp = block_mm ? block_mm + 4 * (uint64_t)b : mm;
    const uint32_t T0 = Tp[0], T1 = Tp[1], T2 = Tp[2], T3 = Tp[3];
    const uint64_t bstart = (uint64_t)b * bs;
    const uint64_t bend = bstart + bs < n ? bstart + bs : n;
    TokOut *out = slots + (uint64_t)b * cap_tok;
    uint64_t p = bstart, lit_start = bstart;
    uint32_t cnt = 0, lits = 0;
    while (p < bend) {
        uint32_t best_len = 0;
        uint64_t best_src = 0;
        if (p + 4 <= n) {
            const uint32_t r = rank[p];
            const uint32_t kp = key_s[r];
            bool more = true;
            for (uint32_t k0 = 0; k0 < depth && more; k0 += 32) {
                const uint32_t k = k0 + lane;
                // candidate k exists when it is in the chain, in the window
                // and among the first depth
                bool ok = k < depth && r >= k + 1;
                uint64_t q = 0;
                if (ok) {
                    const uint32_t rr = r - 1 - k;
                    ok = key_s[rr] == kp;
                    q = val_s[rr];
                    ok = ok && p - q <= window;
                }
                uint32_t len = 0;
                if (ok) {
                    const uint64_t d = p - q;
                    const uint64_t lim = d < bend - p ? d : bend - p;
                    len = common_len(x, q, p, (uint32_t)lim);
                    const int c = dclass(d);
                    const uint32_t t = c == 0 ? T0 : c == 1 ? T1 : c == 2 ? T2 : T3;
                    if (len < t) len = 0;
                }
                // longest, then nearest (smallest k): one 64-bit key per lane
                unsigned long long key = len ? ((unsigned long long)len << 32) | (0xffffffffu - k) : 0ULL;
#pragma unroll
                for (int o = 16; o; o >>= 1) {
                    const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
                    key = other > key ? other : key;
                }
                if (key) {
                    const uint32_t l = (uint32_t)(key >> 32);
                    const uint32_t kk = 0xffffffffu - (uint32_t)key;
                    if (l > best_len) {  // an earlier round keeps its ties (nearer)
                        best_len = l;
                        best_src = (uint64_t)val_s[r - 1 - kk];
                    }
                }
                more = __all_sync(0xffffffffu, !(k < depth) || ok);  // the chain went on past this round
            }
        }
        if (best_len) {
            if (lane == 0) out[cnt] = TokOut{(uint32_t)(p - lit_start), best_len, best_src};
            lits += (uint32_t)(p - lit_start);
            cnt++;
            p += best_len;
            lit_start = p;
        } else {
            p++;
        }
    }
    if (lit_start < bend || cnt == 0) {
        if (lane == 0) out[cnt] = TokOut{(uint32_t)(bend - lit_start), 0u, 0ULL};
        lits += (uint32_t)(bend - lit_start);
        cnt++;
    }
    if (lane == 0) {
        ntok[b] = cnt;
        nlit[b] = lits;
    }
}

// One warp per block: directory entry, tokens and literal bytes of the
// container (tok_off / lit_off: exclusive scans of the counts).
__global__ void __launch_bounds__(256) k_emit(const uint8_t *__restrict__ x, uint64_t n, uint32_t bs, uint32_t nb,
                                              const TokOut *__restrict__ slots, uint32_t cap_tok,
                                              const uint32_t *__restrict__ ntok, const uint32_t *__restrict__ tok_off,
                                              const uint32_t *__restrict__ lit_off, const uint8_t *mm,
                                              const uint8_t *__restrict__ block_mm, uint8_t *__restrict__ dir,
                                              uint8_t *__restrict__ tok, uint8_t *__restrict__ lit) {
    const uint32_t b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= nb) return;
    const uint32_t nt = ntok[b];
    const uint64_t t0 = tok_off[b], l0 = lit_off[b];
    if (lane < 8) {
        // tok_off u64, lit_off u64, n_tok u32, max_wave u16 0, flags u16 0,
        // min_match[4], pad u32 0: 32 bytes as eight words
        const uint8_t *T = block_mm ? block_mm + 4 * (uint64_t)b : mm;
        uint32_t v = 0;
        switch (lane) {
            case 0: v = (uint32_t)t0; break;
            case 1: v = (uint32_t)(t0 >> 32); break;
            case 2: v = (uint32_t)l0; break;
            case 3: v = (uint32_t)(l0 >> 32); break;
            case 4: v = nt; break;
            case 6: v = (uint32_t)T[0] | ((uint32_t)T[1] << 8) | ((uint32_t)T[2] << 16) | ((uint32_t)T[3] << 24); break;
            default: v = 0; break;
        }
        reinterpret_cast<uint32_t *>(dir + 32 * (uint64_t)b)[lane] = v;
    }
    const TokOut *in = slots + (uint64_t)b * cap_tok;
    uint64_t pos = (uint64_t)b * bs, lbase = l0;
    for (uint32_t w = 0; w < nt; w += 32) {
        const uint32_t i = w + lane;
        const bool v = i < nt;
        const TokOut t = v ? in[i] : TokOut{0u, 0u, 0ULL};
        // output position of this token's literals: block start + the
        // lengths of the tokens before it
        uint64_t tot = (uint64_t)t.lit + t.len, incl = tot;
        uint64_t lincl = t.lit;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t a = __shfl_up_sync(0xffffffffu, incl, o);
            const uint64_t c = __shfl_up_sync(0xffffffffu, lincl, o);
            if (lane >= o) {
                incl += a;
                lincl += c;
            }
        }
        if (v) {
            uint32_t *tw = reinterpret_cast<uint32_t *>(tok + 16 * (t0 + i));
            tw[0] = t.lit;
            tw[1] = t.len;
            tw[2] = t.len ? (uint32_t)t.src : 0u;
            tw[3] = t.len ? (uint32_t)(t.src >> 32) & 0xffu : 0u;
        }
        // literal runs, one after another, each copied by the whole warp
        const uint64_t ps = pos + incl - tot;        // first literal byte in the input
        const uint64_t ls = lbase + lincl - t.lit;   // its place in the literal array
        for (int j = 0; j < 32; j++) {
            const uint32_t lj = __shfl_sync(0xffffffffu, v ? t.lit : 0u, j);
            const uint64_t pj = __shfl_sync(0xffffffffu, ps, j), qj = __shfl_sync(0xffffffffu, ls, j);
            for (uint32_t k = lane; k < lj; k += 32) lit[qj + k] = x[pj + k];
        }
        pos += __shfl_sync(0xffffffffu, incl, 31);
        lbase += __shfl_sync(0xffffffffu, lincl, 31);
    }
}

struct Dev {
    void *p = nullptr;
    ~Dev() {
        if (p) cudaFree(p);
    }
};

}  // namespace

extern "C" int aclz_encode_gpu(const void *host_src, uint64_t n, const aclz_encode_params *p,
                               const uint8_t *block_min_match, void *stream, void *host_out, uint64_t cap,
                               uint64_t *out_size) {
    if (!p || !out_size || (n && !host_src)) return ACLZ_E_INVAL;
    const uint32_t bs = p->block_size;
    if (!is_pow2(bs) || bs < kMinBlock || bs > kMaxBlock) return ACLZ_E_INVAL;
    for (int i = 0; i < 4; i++)
        if (p->min_match[i] < 4) return ACLZ_E_INVAL;
    // positions, ranks and counts are 32-bit here
    if (n >= (1ULL << 32) - 64) return ACLZ_E_UNSUPPORTED;
    const uint32_t nb = (uint32_t)((n + bs - 1) / bs);
    if (block_min_match)
        for (uint64_t i = 0; i < 4ULL * nb; i++)
            if (block_min_match[i] < 4) return ACLZ_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t m = n >= 4 ? n - 3 : 0;
    const uint32_t cap_tok = bs / 4 + 1;
    int rc = ACLZ_OK;
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == ACLZ_OK) {
            note_cuda_error(e);
            rc = e == cudaErrorMemoryAllocation ? ACLZ_E_NOMEM : ACLZ_E_CUDA;
        }
        return rc == ACLZ_OK;
    };
    Dev dx, dk0, dv0, dk1, dv1, drank, dhist, dslots, dntok, dnlit, dtoff, dloff, dmm, dbmm, dcont;
    const uint32_t ntiles = (uint32_t)((m + kSortTile - 1) / kSortTile);
    // the input with 16 zero bytes after it (the 8-byte compares read
    // whole aligned words)
    if (!ck(cudaMalloc(&dx.p, n + 64)) || !ck(cudaMemsetAsync((uint8_t *)dx.p + (n & ~(uint64_t)15), 0, 48, st)) ||
        (n && !ck(cudaMemcpyAsync(dx.p, host_src, n, cudaMemcpyHostToDevice, st))))
        return rc;
    const uint64_t mm1 = m ? m : 1;
    if (!ck(cudaMalloc(&dk0.p, 4 * mm1)) || !ck(cudaMalloc(&dv0.p, 4 * mm1)) || !ck(cudaMalloc(&dk1.p, 4 * mm1)) ||
        !ck(cudaMalloc(&dv1.p, 4 * mm1)) || !ck(cudaMalloc(&drank.p, 4 * mm1)) ||
        !ck(cudaMalloc(&dhist.p, 4 * (256ULL * (ntiles ? ntiles : 1) + 4))))
        return rc;
    uint32_t *k0 = (uint32_t *)dk0.p, *v0 = (uint32_t *)dv0.p, *k1 = (uint32_t *)dk1.p, *v1 = (uint32_t *)dv1.p;
    if (m) {
        const unsigned g = (unsigned)std::min<uint64_t>(8192, (m + 255) / 256);
        k_keys<<<g, 256, 0, st>>>((const uint8_t *)dx.p, m, k0, v0);
        uint32_t *hist = (uint32_t *)dhist.p;
        const uint64_t hn = 256ULL * ntiles;
        for (int pass = 0; pass < 4 && rc == ACLZ_OK; pass++) {
            const int shift = 8 * pass;
            k_rs_hist<<<ntiles, kSortThreads, 0, st>>>(k0, m, shift, ntiles, hist);
            ck(cudaGetLastError());
            if (rc) break;
            rc = device_excl_scan(hist, hn, hist + hn, st);
            if (rc) break;
            k_rs_scatter<<<ntiles, kSortThreads, 0, st>>>(k0, v0, m, shift, ntiles, hist, k1, v1);
            ck(cudaGetLastError());
            std::swap(k0, k1);
            std::swap(v0, v1);
        }
        if (rc) return rc;
        k_rank<<<g, 256, 0, st>>>(v0, m, (uint32_t *)drank.p);
        ck(cudaGetLastError());
    }
    // thresholds
    if (!ck(cudaMalloc(&dmm.p, 16)) || !ck(cudaMemcpyAsync(dmm.p, p->min_match, 4, cudaMemcpyHostToDevice, st)))
        return rc;
    if (block_min_match && (!ck(cudaMalloc(&dbmm.p, 4ULL * nb)) ||
                            !ck(cudaMemcpyAsync(dbmm.p, block_min_match, 4ULL * nb, cudaMemcpyHostToDevice, st))))
        return rc;
    if (!ck(cudaMalloc(&dslots.p, sizeof(TokOut) * (uint64_t)cap_tok * (nb ? nb : 1))) ||
        !ck(cudaMalloc(&dntok.p, 4ULL * nb + 16)) || !ck(cudaMalloc(&dnlit.p, 4ULL * nb + 16)) ||
        !ck(cudaMalloc(&dtoff.p, 4ULL * nb + 16)) || !ck(cudaMalloc(&dloff.p, 4ULL * nb + 16)))
        return rc;
    const uint64_t window = p->window;
    if (nb) {
        k_parse_blocks<<<(nb + 7) / 8, 256, 0, st>>>((const uint8_t *)dx.p, n, bs, nb, k0, v0,
                                                     (const uint32_t *)drank.p, (const uint8_t *)dmm.p,
                                                     (const uint8_t *)dbmm.p, p->chain_depth, window, cap_tok,
                                                     (TokOut *)dslots.p, (uint32_t *)dntok.p, (uint32_t *)dnlit.p);
        if (!ck(cudaGetLastError())) return rc;
        ck(cudaMemcpyAsync(dtoff.p, dntok.p, 4ULL * nb, cudaMemcpyDeviceToDevice, st));
        ck(cudaMemcpyAsync(dloff.p, dnlit.p, 4ULL * nb, cudaMemcpyDeviceToDevice, st));
        if (rc) return rc;
        if ((rc = device_excl_scan((uint32_t *)dtoff.p, nb, (uint32_t *)dtoff.p + nb, st))) return rc;
        if ((rc = device_excl_scan((uint32_t *)dloff.p, nb, (uint32_t *)dloff.p + nb, st))) return rc;
    }
    uint32_t tot[2] = {0, 0};
    if (nb) {
        ck(cudaMemcpyAsync(&tot[0], (uint32_t *)dtoff.p + nb, 4, cudaMemcpyDeviceToHost, st));
        ck(cudaMemcpyAsync(&tot[1], (uint32_t *)dloff.p + nb, 4, cudaMemcpyDeviceToHost, st));
        ck(cudaStreamSynchronize(st));
        if (rc) return rc;
    }
    const uint64_t nt = tot[0], nl = tot[1];
    const uint64_t need = kHdr + (uint64_t)kDirent * nb + (uint64_t)kTok * nt + nl;
    *out_size = need;
    if (!host_out) return ACLZ_OK;
    if (cap < need) return ACLZ_E_CAPACITY;
    if (!ck(cudaMalloc(&dcont.p, need ? need : 16))) return rc;
    uint8_t *c = (uint8_t *)dcont.p;
    if (nb) {
        k_emit<<<(nb + 7) / 8, 256, 0, st>>>((const uint8_t *)dx.p, n, bs, nb, (const TokOut *)dslots.p, cap_tok,
                                             (const uint32_t *)dntok.p, (const uint32_t *)dtoff.p,
                                             (const uint32_t *)dloff.p, (const uint8_t *)dmm.p,
                                             (const uint8_t *)dbmm.p, c + kHdr, c + kHdr + (uint64_t)kDirent * nb,
                                             c + kHdr + (uint64_t)kDirent * nb + (uint64_t)kTok * nt);
        if (!ck(cudaGetLastError())) return rc;
    }
    // header: "ACLZ", v1, no tags, sizes, thresholds, distance bounds
    uint8_t h[kHdr];
    std::memset(h, 0, kHdr);
    h[0] = 'A'; h[1] = 'C'; h[2] = 'L'; h[3] = 'Z';
    wr16(h + 4, 1);
    wr16(h + 6, 0);
    wr64(h + 8, n);
    wr32(h + 16, bs);
    wr32(h + 20, nb);
    wr64(h + 24, nt);
    wr64(h + 32, nl);
    wr32(h + 40, 0);
    std::memcpy(h + 44, p->min_match, 4);
    const uint32_t bounds[3] = {128, 16384, 2097152};
    for (int i = 0; i < 3; i++) wr32(h + 48 + 4 * i, bounds[i]);
    std::memcpy(host_out, h, kHdr);
    if (need > kHdr) ck(cudaMemcpyAsync((uint8_t *)host_out + kHdr, c + kHdr, need - kHdr, cudaMemcpyDeviceToHost, st));
    ck(cudaStreamSynchronize(st));
    return rc;
}
