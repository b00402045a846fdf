// Device-side building blocks of the decode kernels: G-lane groups
// (G in {8, 16, 32} lanes of one warp cooperate on one LZ block, Sec. II),
// group scans and ballots, and the packed 16-byte-vectorised copy that maps
// every lane to one aligned 16-byte chunk of output (Sec. III-C: short
// matches leave lanes idle unless several are packed into one pass).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace aclz {

// device status bits latched in a handle's error word
constexpr uint32_t kErrTimeout = 1u;
constexpr uint32_t kErrCorrupt = 2u;
constexpr uint32_t kErrBounds = 4u;

template <int G>
struct Group {
    static_assert(G == 8 || G == 16 || G == 32, "G must be 8, 16 or 32");
    unsigned mask;  // this group's lanes within the warp
    int lane;       // 0..G-1
    int shift;      // first warp lane of the group

    __device__ __forceinline__ Group() {
        const int wl = threadIdx.x & 31;
        lane = wl & (G - 1);
        shift = wl - lane;
        mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << shift);
    }
    __device__ __forceinline__ void sync() const { __syncwarp(mask); }
    __device__ __forceinline__ unsigned ballot(bool p) const {
        return (__ballot_sync(mask, p) & mask) >> shift;
    }
    template <typename T>
    __device__ __forceinline__ T shfl(T v, int src) const { return __shfl_sync(mask, v, src, G); }
    template <typename T>
    __device__ __forceinline__ T shfl_up(T v, int d) const { return __shfl_up_sync(mask, v, d, G); }
    // inclusive prefix sum over the group's lanes
    template <typename T>
    __device__ __forceinline__ T scan_incl(T v) const {
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
            T t = shfl_up(v, o);
            if (lane >= o) v += t;
        }
        return v;
    }
    __device__ __forceinline__ unsigned lanemask_lt() const { return (1u << lane) - 1u; }
};

__device__ __forceinline__ uint4 ldcg16(const uint8_t *p) {
    return __ldcg(reinterpret_cast<const uint4 *>(p));
}

// Bytes [r, r + 16) of the 32-byte little-endian concatenation a || b.
__device__ __forceinline__ uint4 window16(uint4 a, uint4 b, uint32_t r) {
    uint32_t v0 = a.x, v1 = a.y, v2 = a.z, v3 = a.w, v4 = b.x, v5 = b.y, v6 = b.z, v7 = b.w;
    const uint32_t q = r >> 2, sh = (r & 3) * 8;
    uint32_t w0, w1, w2, w3, w4;
    if (q == 0) { w0 = v0; w1 = v1; w2 = v2; w3 = v3; w4 = v4; }
    else if (q == 1) { w0 = v1; w1 = v2; w2 = v3; w3 = v4; w4 = v5; }
    else if (q == 2) { w0 = v2; w1 = v3; w2 = v4; w3 = v5; w4 = v6; }
    else { w0 = v3; w1 = v4; w2 = v5; w3 = v6; w4 = v7; }
    uint4 o;
    o.x = __funnelshift_r(w0, w1, sh);
    o.y = __funnelshift_r(w1, w2, sh);
    o.z = __funnelshift_r(w2, w3, sh);
    o.w = __funnelshift_r(w3, w4, sh);
    return o;
}

// Store bytes [lo, hi) of the 16-byte word v at the aligned address p.
__device__ __forceinline__ void store_partial16(uint8_t *p, uint4 v, uint32_t lo, uint32_t hi) {
    uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (uint32_t t = 0; t < 16; t++) {
        if (t >= lo && t < hi) p[t] = (uint8_t)(w[t >> 2] >> (8 * (t & 3)));
    }
}

// One aligned 16-byte output chunk of a copy job: output bytes
// [A + lo, A + hi) receive source bytes starting at s (s is the source of
// output byte A + lo).  Loads only the aligned source words that hold
// needed bytes, so reads never leave the 16-byte words of the source range.
struct Chunk {
    uint8_t *dst;       // A, 16-byte aligned
    const uint8_t *s;   // source of byte A + lo
    uint32_t lo, hi;    // 0 <= lo < hi <= 16
};

__device__ __forceinline__ void chunk_load(const Chunk &c, uint4 &w0, uint4 &w1, uint32_t &r) {
    // virtual source of output byte A is s - lo
    const uintptr_t vs = reinterpret_cast<uintptr_t>(c.s) - c.lo;
    const uintptr_t base = vs & ~(uintptr_t)15;
    r = (uint32_t)(vs & 15);
    const uintptr_t s0 = reinterpret_cast<uintptr_t>(c.s);
    const uintptr_t s1 = s0 + (c.hi - c.lo);  // one past the last needed source byte
    w0 = make_uint4(0, 0, 0, 0);
    w1 = make_uint4(0, 0, 0, 0);
    if (base + 16 > s0) w0 = ldcg16(reinterpret_cast<const uint8_t *>(base));
    if (s1 > base + 16) w1 = ldcg16(reinterpret_cast<const uint8_t *>(base + 16));
}

__device__ __forceinline__ void chunk_store(const Chunk &c, uint4 w0, uint4 w1, uint32_t r) {
    uint4 v = window16(w0, w1, r);
    if (c.lo == 0 && c.hi == 16)
        *reinterpret_cast<uint4 *>(c.dst) = v;
    else
        store_partial16(c.dst, v, c.lo, c.hi);
}

// Packed group copy.  Each lane holds one job (d: output offset, s: source
// pointer, n: length; n == 0 for none).  The jobs' output chunks are
// numbered in lane order and dealt to the group's lanes, U per lane per
// round, loads issued before stores.  Jobs must be independent: no job's
// source may overlap another job's output in the same call.
template <int G, int U>
__device__ __forceinline__ void group_copy(const Group<G> &g, uint8_t *out, uint64_t d,
                                           const uint8_t *s, uint32_t n) {
    const uint32_t c = n ? (uint32_t)(((d + n - 1) >> 4) - (d >> 4) + 1) : 0u;
    const uint32_t incl = g.scan_incl(c);
    const uint32_t total = g.shfl(incl, G - 1);
    for (uint32_t base = 0; base < total; base += (uint32_t)G * U) {
        Chunk ch[U];
        uint4 a[U], b[U];
        uint32_t r[U];
        bool act[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint32_t k = base + (uint32_t)u * G + (uint32_t)g.lane;
            act[u] = k < total;
            // owner: first lane j with incl_j > k
            int lo = 0, hi = G - 1;
#pragma unroll
            for (int st = G; st > 1; st >>= 1) {
                const int mid = (lo + hi) >> 1;
                const uint32_t v = g.shfl(incl, mid);
                if (v > k) hi = mid; else lo = mid + 1;
            }
            const int j = lo;
            const uint32_t cj = g.shfl(c, j);
            const uint32_t ej = g.shfl(incl, j) - cj;
            const uint64_t dj = g.shfl(d, j);
            const uint8_t *sj = reinterpret_cast<const uint8_t *>(
                g.shfl(reinterpret_cast<unsigned long long>(s), j));
            const uint32_t nj = g.shfl(n, j);
            const uint32_t q = k - ej;
            const uint64_t A = ((dj >> 4) + q) << 4;
            const uint64_t blo = dj > A ? dj : A;
            const uint64_t bhi = (dj + nj) < (A + 16) ? (dj + nj) : (A + 16);
            ch[u].dst = out + A;
            ch[u].s = sj + (blo - dj);
            ch[u].lo = (uint32_t)(blo - A);
            ch[u].hi = (uint32_t)(bhi - A);
            if (act[u]) chunk_load(ch[u], a[u], b[u], r[u]);
        }
#pragma unroll
        for (int u = 0; u < U; u++)
            if (act[u]) chunk_store(ch[u], a[u], b[u], r[u]);
    }
}

}  // namespace aclz
