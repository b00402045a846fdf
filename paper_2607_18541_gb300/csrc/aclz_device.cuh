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

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint4 lds16(const uint8_t *p) {
    uint4 v;
    asm("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(smem_u32(p)));
    return v;
}

__device__ __forceinline__ uint4 lds16_u32(uint32_t a) {
    uint4 v;
    asm("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
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

// Store bytes [lo, hi) of the 16-byte word v at the aligned address p,
// as at most seven naturally aligned 1/2/4/8-byte stores.
__device__ __forceinline__ void store_partial16(uint8_t *p, uint4 v, uint32_t lo, uint32_t hi) {
    const unsigned long long q0 = (unsigned long long)v.x | ((unsigned long long)v.y << 32);
    const unsigned long long q1 = (unsigned long long)v.z | ((unsigned long long)v.w << 32);
    // byte t of the word, t in [0, 16), and the little-endian field at t
    auto field = [&](uint32_t t) -> unsigned long long { return t < 8 ? (q0 >> (8 * t)) | (t ? q1 << (64 - 8 * t) : 0ULL) : q1 >> (8 * (t - 8)); };
    uint32_t t = lo;
    if ((t & 1) && t + 1 <= hi) { p[t] = (uint8_t)field(t); t += 1; }
    if ((t & 2) && t + 2 <= hi) { *reinterpret_cast<uint16_t *>(p + t) = (uint16_t)field(t); t += 2; }
    if ((t & 4) && t + 4 <= hi) { *reinterpret_cast<uint32_t *>(p + t) = (uint32_t)field(t); t += 4; }
    if ((t & 8) && t + 8 <= hi) { *reinterpret_cast<unsigned long long *>(p + t) = field(t); t += 8; }
    while (t + 8 <= hi) { *reinterpret_cast<unsigned long long *>(p + t) = field(t); t += 8; }
    if (t + 4 <= hi) { *reinterpret_cast<uint32_t *>(p + t) = (uint32_t)field(t); t += 4; }
    if (t + 2 <= hi) { *reinterpret_cast<uint16_t *>(p + t) = (uint16_t)field(t); t += 2; }
    if (t + 1 <= hi) { p[t] = (uint8_t)field(t); }
}

// One aligned 16-byte output chunk of a copy job: output bytes
// [A + lo, A + hi) receive source bytes starting at s (the source of
// output byte A + lo).  Only the aligned source words holding needed bytes
// are read, so reads never leave the 16-byte words of the source range.
// SMEM: the source is a shared-memory staging copy whose addresses are
// congruent mod 16 to the global source.  RO: the source is global memory
// that no thread writes during the kernel (the literal array), read through
// the non-coherent L1 path.
template <bool SMEM, bool RO = false>
__device__ __forceinline__ void chunk_load(const uint8_t *s, uint32_t lo, uint32_t hi, uint4 &w0, uint4 &w1,
                                           uint32_t &r) {
    const uintptr_t vs = reinterpret_cast<uintptr_t>(s) - lo;
    const uintptr_t base = vs & ~(uintptr_t)15;
    r = (uint32_t)(vs & 15);
    const uintptr_t s0 = reinterpret_cast<uintptr_t>(s);
    const uintptr_t s1 = s0 + (hi - lo);  // one past the last needed source byte
    w0 = make_uint4(0, 0, 0, 0);
    w1 = make_uint4(0, 0, 0, 0);
    if (SMEM) {
        if (base + 16 > s0) w0 = lds16(reinterpret_cast<const uint8_t *>(base));
        if (s1 > base + 16) w1 = lds16(reinterpret_cast<const uint8_t *>(base + 16));
    } else if (RO) {
        if (base + 16 > s0) w0 = __ldg(reinterpret_cast<const uint4 *>(base));
        if (s1 > base + 16) w1 = __ldg(reinterpret_cast<const uint4 *>(base + 16));
    } else {
        if (base + 16 > s0) w0 = ldcg16(reinterpret_cast<const uint8_t *>(base));
        if (s1 > base + 16) w1 = ldcg16(reinterpret_cast<const uint8_t *>(base + 16));
    }
}

__device__ __forceinline__ void chunk_store(uint8_t *dst, uint32_t lo, uint32_t hi, uint4 w0, uint4 w1,
                                            uint32_t r) {
    uint4 v = window16(w0, w1, r);
    if (lo == 0 && hi == 16)
        *reinterpret_cast<uint4 *>(dst) = v;
    else
        store_partial16(dst, v, lo, hi);
}

// Lane of the group's first job whose inclusive prefix count exceeds k.
template <int G>
__device__ __forceinline__ int owner_lane(const Group<G> &g, uint32_t incl, uint32_t k) {
    int lo = 0, hi = G - 1;
#pragma unroll
    for (int st = G; st > 1; st >>= 1) {
        const int mid = (lo + hi) >> 1;
        const uint32_t v = g.shfl(incl, mid);
        if (v > k) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// Packed group copy, chunks in job order: the jobs' aligned 16-byte output
// chunks (c per lane, inclusive prefix incl, total in all) are numbered in
// lane order and dealt to the group's lanes, U per lane per round, loads
// issued before stores.
template <int G, int U, bool SMEM, bool RO = false>
__device__ __forceinline__ void copy_chunks_in_order(const Group<G> &g, uint8_t *out, uint64_t d,
                                                     const uint8_t *s, uint32_t n, uint32_t c,
                                                     uint32_t incl, uint32_t total) {
    for (uint32_t base = 0; base < total; base += (uint32_t)G * U) {
        uint8_t *dst[U];
        uint32_t lohi[U];
        uint4 a[U], b[U];
        uint32_t r[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            lohi[u] = 0u;
            const uint32_t k0 = base + (uint32_t)u * G;  // the same on every lane
            if (k0 >= total) continue;
            const uint32_t k = k0 + (uint32_t)g.lane;
            const int j = owner_lane<G>(g, incl, k);
            const uint32_t ej = g.shfl(incl - c, j);
            const uint64_t dj = g.shfl(d, j);
            const uint8_t *sj = reinterpret_cast<const uint8_t *>(
                g.shfl(reinterpret_cast<unsigned long long>(s), j));
            const uint32_t nj = g.shfl(n, j);
            const uint64_t A = ((dj >> 4) + (k - ej)) << 4;
            const uint64_t blo = dj > A ? dj : A;
            const uint64_t bhi = (dj + nj) < (A + 16) ? (dj + nj) : (A + 16);
            const uint32_t clo = (uint32_t)(blo - A), chi = (uint32_t)(bhi - A);
            dst[u] = out + A;
            if (k < total) {
                lohi[u] = clo | (chi << 8);
                chunk_load<SMEM, RO>(sj + (blo - dj), clo, chi, a[u], b[u], r[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++)
            if (lohi[u]) chunk_store(dst[u], lohi[u] & 0xff, lohi[u] >> 8, a[u], b[u], r[u]);
    }
}

// Packed group copy, full chunks first: every job's full 16-byte chunks
// (in lane order), then the partial head and tail chunks, dealt as above.
// A slot of G chunks is then all full 16-byte stores or all narrow partial
// stores, except the one slot at the boundary, so the narrow-store path
// runs once per G partial chunks instead of in every slot.
template <int G, int U, bool SMEM>
__device__ __forceinline__ void copy_chunks_full_first(const Group<G> &g, uint8_t *out, uint64_t d,
                                                       const uint8_t *s, uint32_t n, uint32_t c) {
    const uint64_t e = d + n;
    // chunk 0 is partial unless it starts at d and is filled; the last
    // chunk (if another) is partial unless the job ends on a boundary
    const uint32_t p0 = (n && ((d & 15) || (c == 1 && (e & 15)))) ? 1u : 0u;
    const uint32_t np = p0 + ((c >= 2 && (e & 15)) ? 1u : 0u);
    const uint32_t nf = c - np;
    const uint32_t inclF = g.scan_incl(nf);
    const uint32_t inclP = g.scan_incl(np);
    const uint32_t exF = inclF - nf, exP = inclP - np;
    const uint32_t cf = c | (p0 << 31);  // c < 2^21 (jobs are shorter than 2^25 bytes)
    const uint32_t F = g.shfl(inclF, G - 1);
    const uint32_t total = F + g.shfl(inclP, G - 1);
    for (uint32_t base = 0; base < total; base += (uint32_t)G * U) {
        uint8_t *dst[U];
        uint32_t lohi[U];
        uint4 a[U], b[U];
        uint32_t r[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            lohi[u] = 0u;
            const uint32_t k0 = base + (uint32_t)u * G;  // the same on every lane
            if (k0 >= total) continue;
            const uint32_t k = k0 + (uint32_t)g.lane;
            const bool full = k < F;
            // owner among the full chunks, the partial ones, or both (only
            // in the slot that straddles the boundary); branches are uniform
            int j;
            uint32_t exj;
            if (k0 + G <= F) {
                j = owner_lane<G>(g, inclF, k);
                exj = g.shfl(exF, j);
            } else if (k0 >= F) {
                j = owner_lane<G>(g, inclP, k - F);
                exj = g.shfl(exP, j);
            } else {
                const int jf = owner_lane<G>(g, inclF, k);
                const int jp = owner_lane<G>(g, inclP, k - F);
                j = full ? jf : jp;
                const uint32_t xf = g.shfl(exF, j), xp = g.shfl(exP, j);
                exj = full ? xf : xp;
            }
            const uint64_t dj = g.shfl(d, j);
            const uint8_t *sj = reinterpret_cast<const uint8_t *>(
                g.shfl(reinterpret_cast<unsigned long long>(s), j));
            const uint32_t nj = g.shfl(n, j);
            const uint32_t cfj = g.shfl(cf, j);
            const uint32_t cj = cfj & 0x7fffffffu, p0j = cfj >> 31;
            // chunk index within the job: full chunks are [p0j, p0j + nf);
            // the partial ones are chunk 0 (if p0j) then chunk cj - 1
            const uint32_t idx = full ? p0j + (k - exj) : ((k - F == exj && p0j) ? 0u : cj - 1u);
            const uint64_t A = ((dj >> 4) + idx) << 4;
            const uint64_t blo = dj > A ? dj : A;
            const uint64_t bhi = (dj + nj) < (A + 16) ? (dj + nj) : (A + 16);
            const uint32_t clo = (uint32_t)(blo - A), chi = (uint32_t)(bhi - A);
            dst[u] = out + A;
            if (k < total) {
                lohi[u] = clo | (chi << 8);
                chunk_load<SMEM>(sj + (blo - dj), clo, chi, a[u], b[u], r[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++)
            if (lohi[u]) chunk_store(dst[u], lohi[u] & 0xff, lohi[u] >> 8, a[u], b[u], r[u]);
    }
}

// Packed group copies.  Each lane holds one job (d: output offset, s:
// source pointer, n: length; n == 0 for none), cut into aligned 16-byte
// output chunks.  group_copy deals the chunks in job order and suits short
// jobs (literal runs, in-block matches of wave 0); group_copy_full_first
// deals every job's full chunks first, for match copies of a few chunks or
// more.  Jobs must be independent: no job's source may overlap another
// job's output in the same call.
template <int G, int U, bool SMEM = false, bool RO = false>
__device__ __forceinline__ void group_copy(const Group<G> &g, uint8_t *out, uint64_t d,
                                           const uint8_t *s, uint32_t n) {
    const uint32_t c = n ? (uint32_t)(((d + n - 1) >> 4) - (d >> 4) + 1) : 0u;
    const uint32_t incl = g.scan_incl(c);
    const uint32_t total = g.shfl(incl, G - 1);
    copy_chunks_in_order<G, U, SMEM, RO>(g, out, d, s, n, c, incl, total);
}

template <int G, int U, bool SMEM = false>
__device__ __forceinline__ void group_copy_full_first(const Group<G> &g, uint8_t *out, uint64_t d,
                                                      const uint8_t *s, uint32_t n) {
    const uint32_t c = n ? (uint32_t)(((d + n - 1) >> 4) - (d >> 4) + 1) : 0u;
    if (!g.ballot(n > 0)) return;
    copy_chunks_full_first<G, U, SMEM>(g, out, d, s, n, c);
}

// Bytes [r, r + 16) of a || b for a shift r that is the same on every lane
// (a uniform branch picks the word offset).
__device__ __forceinline__ uint4 window16_uniform(const uint4 &a, const uint4 &b, uint32_t q, uint32_t sh) {
    uint32_t w0, w1, w2, w3, w4;
    switch (q) {
        case 0: w0 = a.x; w1 = a.y; w2 = a.z; w3 = a.w; w4 = b.x; break;
        case 1: w0 = a.y; w1 = a.z; w2 = a.w; w3 = b.x; w4 = b.y; break;
        case 2: w0 = a.z; w1 = a.w; w2 = b.x; w3 = b.y; w4 = b.z; break;
        default: w0 = a.w; w1 = b.x; w2 = b.y; w3 = b.z; w4 = b.w; break;
    }
    uint4 o;
    o.x = __funnelshift_r(w0, w1, sh);
    o.y = __funnelshift_r(w1, w2, sh);
    o.z = __funnelshift_r(w2, w3, sh);
    o.w = __funnelshift_r(w3, w4, sh);
    return o;
}

// ------------------------------------------------------- TMA staging

// Per-group staging area for 1-D bulk copies (cp.async.bulk) from global
// memory into shared memory, tracked by one mbarrier (transaction bytes).
struct Stage {
    uint8_t *buf;
    uint64_t *bar;
    uint32_t bytes;
    uint32_t phase;
};

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// orders this thread's view of global memory (including data acquired from
// other threads) before its later bulk-copy reads
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_load_1d(void *dst_smem, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

constexpr uint32_t kMbarSpinLimit = 1u << 26;

// Wait for the stage's current phase (bounded; sets kErrTimeout on err).
// A false return means the bulk copy may still be writing the stage: the
// caller must issue no further copies into it and end the launch.
__device__ __forceinline__ bool stage_wait(Stage &st, uint32_t *err) {
    uint32_t spins = 0;
    while (!mbar_try_wait(st.bar, st.phase)) {
        if (++spins > kMbarSpinLimit) {
            atomicOr(err, kErrTimeout);
            return false;
        }
    }
    st.phase ^= 1u;
    return true;
}

// Realign-and-store of one staged job: output [d, d + n) from the shared
// copy at s (congruent to the global source mod 16).  The partial head and
// tail words go out as single bytes, one per lane, in one pass (a chain of
// narrow stores from one lane is far slower); the aligned 16-byte body
// words go to consecutive lanes, two per lane per round, each built from
// two aligned shared words and one shift common to the whole job.
template <int G>
__device__ __forceinline__ void store_staged_job(const Group<G> &g, uint8_t *out, uint64_t d,
                                                 const uint8_t *s, uint32_t n) {
    const uint64_t e = d + n;
    uint64_t a0 = (d + 15) & ~(uint64_t)15;  // first aligned body word
    uint64_t a1 = e & ~(uint64_t)15;         // end of the aligned body
    if (a0 > e) a0 = e;
    if (a1 < a0) a1 = a0;
    const uint32_t nh = (uint32_t)(a0 - d), nt = (uint32_t)(e - a1);
    for (uint32_t t = g.lane; t < nh + nt; t += G) {
        const uint32_t o = t < nh ? t : (uint32_t)(a1 - d) + (t - nh);
        out[d + o] = s[o];
    }
    if (a1 <= a0) return;
    // body: source of output word a0 + 16k is shared byte sa + (a0 - d) + 16k
    const uint32_t sb = smem_u32(s) + (uint32_t)(a0 - d);
    const uint32_t r = sb & 15u, base = sb & ~15u, q = r >> 2, sh = (r & 3u) * 8u;
    const uint32_t nw = (uint32_t)((a1 - a0) >> 4);
    uint8_t *ob = out + a0;
    for (uint32_t k = g.lane; k < nw; k += 2 * G) {
        const uint32_t k2 = k + G;
        uint4 x0 = lds16_u32(base + 16 * k), y0 = make_uint4(0, 0, 0, 0);
        uint4 x1 = make_uint4(0, 0, 0, 0), y1 = make_uint4(0, 0, 0, 0);
        if (r) y0 = lds16_u32(base + 16 * k + 16);
        if (k2 < nw) {
            x1 = lds16_u32(base + 16 * k2);
            if (r) y1 = lds16_u32(base + 16 * k2 + 16);
        }
        *reinterpret_cast<uint4 *>(ob + 16 * (uint64_t)k) = r ? window16_uniform(x0, y0, q, sh) : x0;
        if (k2 < nw) *reinterpret_cast<uint4 *>(ob + 16 * (uint64_t)k2) = r ? window16_uniform(x1, y1, q, sh) : x1;
    }
}

// One fill of a group's stage, split in two steps so that a fill can be
// issued ahead (while the group finishes other work) and consumed later.
// Per lane: done = bytes of its job written by earlier fills, off = stage
// offset of its aligned source span in the fill in flight, len = bytes of
// its piece in that fill (0: none), head = offset of the piece's first byte
// within the span.
struct Fill {
    uint32_t done, off, len, head;
};

// Issue one fill for every lane's job (s, n) from f.done on: pieces of at
// most `piece` bytes packed in lane order while they fit, one bulk copy per
// piece.  Returns false, issuing nothing, when no lane has bytes left.  The
// caller has made the sources final and visible to bulk copies.
template <int G>
__device__ __forceinline__ bool fill_issue(const Group<G> &g, Stage &st, const uint8_t *s, uint32_t n,
                                           uint32_t piece, Fill &f) {
    const uint32_t rem = n - f.done;
    f.len = 0;
    if (!g.ballot(rem > 0)) return false;
    const uint32_t len = rem < piece ? rem : piece;
    const uintptr_t ps = reinterpret_cast<uintptr_t>(s) + f.done;
    const uintptr_t sa = ps & ~(uintptr_t)15;
    const uint32_t span = rem ? (uint32_t)(((ps + len + 15) & ~(uintptr_t)15) - sa) : 0u;
    const uint32_t incl = g.scan_incl(span);
    const bool take = rem > 0 && incl <= st.bytes;
    const unsigned tm = g.ballot(take);
    const uint32_t tx = g.shfl(incl, 31 - __clz(tm));
    if (g.lane == 0) mbar_expect_tx(st.bar, tx);
    g.sync();
    f.off = incl - span;
    f.head = (uint32_t)(ps - sa);
    if (take) {
        tma_load_1d(st.buf + f.off, reinterpret_cast<const void *>(sa), span, st.bar);
        f.len = len;
    }
    return true;
}

// Wait for the fill in flight and write its pieces to out[d + done, ...),
// one job after another (store_staged_job).  False, on every lane of the
// group, when a lane's wait timed out (see stage_wait).
template <int G>
__device__ __forceinline__ bool fill_consume(const Group<G> &g, Stage &st, uint8_t *out, uint64_t d, Fill &f,
                                             uint32_t *err) {
    const bool waited = stage_wait(st, err);
    if (g.ballot(!waited)) return false;
    const uint8_t *src = st.buf + f.off + f.head;
    for (unsigned m = g.ballot(f.len > 0); m; m &= m - 1) {
        const int j = __ffs(m) - 1;
        const uint64_t dj = g.shfl(d + f.done, j);
        const uint8_t *sj = reinterpret_cast<const uint8_t *>(g.shfl(reinterpret_cast<unsigned long long>(src), j));
        const uint32_t nj = g.shfl(f.len, j);
        store_staged_job<G>(g, out, dj, sj, nj);
    }
    g.sync();
    fence_proxy_async_shared();
    f.done += f.len;
    f.len = 0;
    return true;
}

// Staged copy of every lane's job (d, s, n) through fills; `issued` says
// that the first fill of these jobs (f.done = 0) is already in flight.
template <int G>
__device__ __forceinline__ bool staged_copy_fills(const Group<G> &g, Stage &st, uint8_t *out, uint64_t d,
                                                  const uint8_t *s, uint32_t n, uint32_t piece, Fill &f,
                                                  bool issued, uint32_t *err) {
    if (!issued) {
        f.done = 0;
        if (!fill_issue<G>(g, st, s, n, piece, f)) return true;
    }
    for (;;) {
        if (!fill_consume<G>(g, st, out, d, f, err)) return false;
        if (!fill_issue<G>(g, st, s, n, piece, f)) return true;
    }
}

}  // namespace aclz
