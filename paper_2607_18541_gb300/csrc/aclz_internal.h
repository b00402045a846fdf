// Internal declarations shared by the translation units of libaclz.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/aclz.h"

namespace aclz {

constexpr uint32_t kHdr = 64;
constexpr uint32_t kDirent = 32;
constexpr uint32_t kTok = 16;
constexpr uint64_t kSrcMask = (1ULL << 40) - 1;
constexpr uint32_t kMaxWave = (1u << 24) - 1;
constexpr uint16_t kFlagWaves = 1;
constexpr uint32_t kMinBlock = 64;
constexpr uint32_t kMaxBlock = 1u << 24;

// little-endian field access in host buffers
inline uint16_t rd16(const uint8_t *p) { return (uint16_t)(p[0] | (p[1] << 8)); }
inline uint32_t rd32(const uint8_t *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
inline uint64_t rd64(const uint8_t *p) { return (uint64_t)rd32(p) | ((uint64_t)rd32(p + 4) << 32); }
inline void wr16(uint8_t *p, uint16_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
inline void wr32(uint8_t *p, uint32_t v) {
    for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i));
}
inline void wr64(uint8_t *p, uint64_t v) {
    for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i));
}

inline bool is_pow2(uint64_t v) { return v && !(v & (v - 1)); }
inline uint32_t log2u(uint64_t v) {
    uint32_t k = 0;
    while ((1ULL << k) < v) k++;
    return k;
}

// Parsed header plus pointers into a host container.
struct View {
    uint64_t total_len = 0, n_tokens = 0, n_literals = 0;
    uint32_t block_size = 0, n_blocks = 0, n_waves = 0;
    uint16_t flags = 0;
    uint8_t mm[4] = {0, 0, 0, 0};
    const uint8_t *dir = nullptr, *tok = nullptr, *lit = nullptr;
};

// Header and directory checks on the host (O(n_blocks)); per-token checks
// run on the device during upload.
int parse_container(const uint8_t *c, uint64_t n, View *v, bool check_directory);

// Remember the last CUDA runtime error for aclz_last_cuda_error().
void note_cuda_error(int cuda_error_code);

// Exclusive scan of n u32 in place on the device, the total to *d_total
// (device); stream-ordered, temporary storage allocated on the stream.
int device_excl_scan(uint32_t *d, uint64_t n, uint32_t *d_total, void *stream);

}  // namespace aclz

struct aclz_handle;

namespace aclz {

// Decode index of h from its device tokens (validation, offsets, wave tags,
// worklists, schedule); see aclz_index.cu.
int build_index(aclz_handle *h, bool has_tags, uint32_t given_waves, bool flat_local, void *stream);

// Upload from a parsed container view: allocates the handle's arrays, has
// fill(h, v, ctx, stream) place the token array in h->d_tok and the literal
// bytes in h->d_lit (stream-ordered), then builds the decode index as
// aclz_upload_ex does.
using FillFn = int (*)(aclz_handle *h, const View &v, const void *ctx, void *stream);
int upload_view(const View &v, uint32_t flags, void *stream, FillFn fill, const void *ctx, aclz_handle **out);

// Ranges per SM a small wave is cut into (about one per resident group).
constexpr uint32_t kRangesPerSm = 16;

// Matches per work range for a target byte size of deferred matches.
inline uint32_t range_matches(uint32_t range_bytes, double mean_len) {
    double t = mean_len > 0 ? (double)range_bytes / mean_len : 16.0;
    if (t < 8) t = 8;
    if (t > 4096) t = 4096;
    return (uint32_t)t;
}

}  // namespace aclz

// Library handle: device copies of a container plus its decode index.
struct aclz_handle {
    int device = 0;
    uint64_t total_len = 0, n_tokens = 0, n_literals = 0, n_deferred = 0;
    uint32_t block_size = 0, log2_bs = 0, n_blocks = 0, n_waves = 0;
    uint16_t flags = 0;
    uint8_t mm[4] = {0, 0, 0, 0};
    // device arrays (owned)
    void *d_tok = nullptr;        // n_tokens x 16 B, tags filled in
    uint8_t *d_lit = nullptr;     // n_literals + 32 zero bytes of padding
    uint64_t *d_blk_tok = nullptr;  // n_blocks + 1 token offsets
    uint64_t *d_blk_lit = nullptr;  // n_blocks + 1 literal offsets
    uint32_t *d_slot = nullptr;   // per token: triplet slot of a deferred match, else ~0u
    uint32_t *d_tokdst = nullptr; // per token: block-relative offset of its first byte
    uint32_t *d_toklit = nullptr; // per token: block-relative offset of its first literal
    void *d_tri = nullptr;        // n_deferred x 16 B triplets (dst, src, len), built at upload
    uint32_t *d_err = nullptr;    // latched device status bits
    std::vector<uint64_t> wave_start;  // n_waves + 1 entries into the triplet array
    // persistent-mode schedule.  A segment is the run of one block's
    // matches in one wave's worklist: seg[s] = {block, wave, triplet offset,
    // count}, wave-major then block order.  A range is a run of consecutive
    // triplets of one wave: range[r] = {wave, first segment, end segment,
    // first triplet}, with a sentinel after the last.  Ranges hold up to
    // range_T triplets in large waves and fewer in small ones; they may cut
    // a segment in pieces unless one of its matches reads another's output.
    // seg_pieces[s] counts the ranges that share segment s, and seg_cnt[s]
    // counts the finished ones during a decode (reset by the last).
    void *d_seg = nullptr;
    void *d_ranges = nullptr;
    uint32_t *d_seg_pieces = nullptr;
    uint32_t *d_seg_cnt = nullptr;
    uint64_t n_seg = 0, n_ranges = 0;
    uint32_t range_T = 16;         // matches per range in large waves (from range_bytes / mean length)
    uint32_t range_bytes = 20480;
    double mean_deferred_len = 0;  // mean length of the deferred matches
    // per block, n_wave_words 64-bit words: bit w of pending = block has work
    // in wave w (bit 0 always); done = waves finished (empty waves preset)
    uint32_t n_wave_words = 0;
    uint64_t *d_pending = nullptr;
    uint64_t *d_done = nullptr;
    // set by aclz_flatten: the deferred work items are origin pieces in one
    // wave, built at flatten time
    bool flat = false;
    // set when the (wave, block) tables of the plain schedule would be too
    // large (deep copy chains): the upload then flattens
    bool needs_flatten = false;
    // the stored tags are the 0/1 "in order or not" tags of the flattening
    // upload, not a legal wave tagging of the container
    bool local_tags = false;
    uint64_t n_matches_deferred = 0;  // deferred matches before flattening
};
