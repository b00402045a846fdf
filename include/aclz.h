/*
 * aclz — device-resident match phase of absolute-offset LZ77 decode on
 * GB300 (sm_103a).  C ABI of libaclz.so.
 *
 * The codec follows the paper "What Governs Decode Throughput in
 * Absolute-Offset GPU LZ77?": every back-reference names an absolute
 * position of the output (abstract; Sec. I), LZ blocks fixed at encode time are the unit of decode
 * parallelism (Sec. II), minimum match lengths are set per distance class
 * (Sec. IV-B), matches whose sources are not yet written are decoded in
 * later waves (Sec. I), and results are verified by byte compare and FNV
 * (abstract; Sec. II).
 *
 * Conventions for every entry point:
 *  - Return value: ACLZ_OK (0) or a negative ACLZ_E_* code; aclz_strerror()
 *    names it.  Nothing is allocated or launched when an argument is
 *    rejected.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Decode calls only enqueue work; errors found on the device
 *    (a bounded wait that ran out) are latched in the handle and returned
 *    by aclz_device_status().
 *  - Pointers named host_* are host memory, d_* are device memory of the
 *    current CUDA device.  The caller owns every buffer it passes; the
 *    library owns the device copies it makes in aclz_upload() until
 *    aclz_free().
 *  - Device output buffers must be 16-byte aligned.  Kernels write only
 *    [d_out, d_out + length); they may read (never write) bytes up to the
 *    end of the 16-byte word holding the last output byte.
 *
 * Container format v1 (little endian; the paper gives no byte layout, this
 * is the reading the library and its oracle agree on):
 *   header 64 B : "ACLZ", u16 version=1, u16 flags (bit0: wave tags
 *                 present), u64 total_len, u32 block_size, u32 n_blocks,
 *                 u64 n_tokens, u64 n_literals, u32 n_waves, u8 min_match[4],
 *                 u32 distance bounds[3] = {128, 16384, 2097152}, u32 0
 *   directory   : n_blocks x 32 B: u64 tok_off, u64 lit_off, u32 n_tok,
 *                 u16 max_wave, u16 flags, u8 min_match[4], u32 0
 *   tokens      : n_tokens x 16 B: u32 lit_len, u32 match_len,
 *                 u64 (src : 40 bits | wave : 24 bits)
 *   literals    : n_literals bytes
 * Block b covers output [b*block_size, min((b+1)*block_size, total_len)).
 * A token appends lit_len literals, then match_len bytes copied from
 * absolute position src, with src + match_len <= the match's own position;
 * match_len == 0 only on a block's last token.
 */
#ifndef ACLZ_H
#define ACLZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ACLZ_OK 0
#define ACLZ_E_INVAL (-1)       /* bad argument */
#define ACLZ_E_CORRUPT (-2)     /* container fails validation */
#define ACLZ_E_NOMEM (-3)       /* host or device allocation failed */
#define ACLZ_E_CAPACITY (-4)    /* output or scratch buffer too small */
#define ACLZ_E_CUDA (-5)        /* a CUDA runtime call failed */
#define ACLZ_E_TIMEOUT (-6)     /* a bounded device-side wait ran out */
#define ACLZ_E_DEVICE (-7)      /* another device-side error was latched */
#define ACLZ_E_UNSUPPORTED (-8) /* valid container this build cannot decode */

/* Encoder parameters (Sec. II: block size set at encode time; Sec. IV-B:
 * minimum match length per distance class d < 128, < 16384, < 2097152,
 * >= 2097152).  block_size: power of two, 64 B .. 16 MiB.  min_match >= 4.
 * chain_depth: candidates examined per position.  window: largest match
 * distance considered. */
typedef struct aclz_encode_params {
    uint32_t block_size;
    uint8_t min_match[4];
    uint32_t chain_depth;
    uint32_t flags; /* reserved, 0 */
    uint64_t window;
} aclz_encode_params;

#define ACLZ_PRESET_BASE 0  /* 6/8/10/12 (Sec. IV-B) */
#define ACLZ_PRESET_TUNED 1 /* 12/16/24/32 (Sec. IV-B) */
#define ACLZ_PRESET_PUSH 2  /* 16/24/32/48 (Sec. IV-C) */

/* Fill *p with a preset: block_size 65536, chain_depth 64, unbounded
 * window.  Returns ACLZ_E_INVAL for an unknown preset or NULL p. */
int aclz_encode_params_default(aclz_encode_params *p, int preset);

/* Upper bound of the container size for n input bytes. */
uint64_t aclz_encode_bound(uint64_t n, uint32_t block_size);

/* Greedy encoder on the host (the paper's encoder is a CPU program,
 * Sec. VI).  At each position with >= 4 bytes left, the candidates are the
 * earlier positions with the same 4-byte prefix, nearest first, up to
 * chain_depth of them within the window; the longest candidate whose
 * length (capped at the distance and at the block end) meets its distance
 * class minimum wins, ties to the nearest.  block_min_match (4 bytes per
 * block, or NULL) overrides the thresholds block by block.  threads <= 0
 * uses all host cores.  The container carries no wave tags (aclz_upload
 * computes them).  *out_size receives the container size. */
int aclz_encode(const void *host_src, uint64_t n, const aclz_encode_params *p,
                const uint8_t *block_min_match, int threads, void *host_out, uint64_t cap,
                uint64_t *out_size);

/* aclz_encode with the parse on the GPU (the paper's encoder is a CPU
 * program and makes no speed claim, Sec. VI): the same container, byte for
 * byte, from the same arguments.  Every candidate chain of the greedy parse
 * is an ordered run of positions with one 4-byte prefix, so the device sorts
 * the positions by (prefix, position), then parses every LZ block with one
 * warp whose lanes score up to 32 candidates at a time, and lays the
 * container out by scans.  host_src: n input bytes (host); n < 2^32 - 64
 * (else ACLZ_E_UNSUPPORTED).  With host_out NULL only *out_size is set (the
 * parse still runs); otherwise cap must hold *out_size bytes
 * (ACLZ_E_CAPACITY).  Allocates device memory of about 25 bytes per input
 * byte for the call (sorted prefixes, ranks, per-block token slots) and
 * frees it before returning; synchronizes the stream. */
int aclz_encode_gpu(const void *host_src, uint64_t n, const aclz_encode_params *p,
                    const uint8_t *block_min_match, void *stream, void *host_out, uint64_t cap,
                    uint64_t *out_size);

/* Container from token arrays (host): blk_ntok[n_blocks] tokens per
 * block, lit_len/match_len/src per token, the literal bytes.  min_match is
 * recorded, not enforced.  No wave tags. */
int aclz_pack(uint64_t total_len, uint32_t block_size, const uint8_t min_match[4],
              const uint32_t *blk_ntok, const uint32_t *lit_len, const uint32_t *match_len,
              const uint64_t *src, uint64_t n_tokens, const uint8_t *literals,
              uint64_t n_literals, void *host_out, uint64_t cap, uint64_t *out_size);

/* Size of the container aclz_pack writes. */
uint64_t aclz_pack_bytes(uint64_t total_len, uint32_t block_size, uint64_t n_tokens,
                         uint64_t n_literals);

typedef struct aclz_info {
    uint64_t total_len, n_tokens, n_literals, n_deferred;
    uint32_t block_size, n_blocks, n_waves, flags;
    uint8_t min_match[4];
    uint32_t reserved;
} aclz_info;

/* Header fields of a host container (checks magic, version and sizes). */
int aclz_container_info(const void *host_buf, uint64_t n, aclz_info *out);

typedef struct aclz_handle aclz_handle;

/* Copy a host container to the current device and build its decode index
 * on the GPU: validation of every token (lengths sum to the block length,
 * src + match_len <= dst), wave tags (the minimal legal tags when the
 * container has none; a legality check when it has them), and the
 * wave-ordered worklist slots of deferred matches.  Synchronizes the
 * stream.  ACLZ_E_CORRUPT for an invalid container. */
int aclz_upload(const void *host_buf, uint64_t n, void *stream, aclz_handle **out);

/* aclz_upload with options.  ACLZ_UPLOAD_FLATTEN: build the two-wave
 * flattened schedule of aclz_flatten directly.  For a container without
 * tags, the upload then needs only whether each match is in order within
 * its block (wave 0) or not, which every block settles on its own: no
 * ordered pass over the blocks, so deep chains of copies do not slow the
 * upload, and aclz_tags returns these 0/1 tags.  A container with tags has
 * them checked as by aclz_upload first.  flags other than
 * ACLZ_UPLOAD_FLATTEN: ACLZ_E_INVAL.  Without the flag, an upload whose
 * plain schedule would need more than 2^28 (wave, block) cells (copy chains
 * thousands of waves deep) also flattens. */
#define ACLZ_UPLOAD_FLATTEN 1u

int aclz_upload_ex(const void *host_buf, uint64_t n, uint32_t flags, void *stream, aclz_handle **out);

/* Upload an entropy-coded (ACLE) container and decode its entropy stage on
 * the GPU, then build the decode index as aclz_upload_ex(flags) does.  The
 * entropy stage is the one Sec. II puts in front of the match kernel
 * (an ANS stage on 64 KB tiles, many at once); its coder is
 * order-0 rANS per 64 KiB tile with frequencies summing to 2^12, 32
 * interleaved states in [2^16, 2^32) (byte i of a tile on state i mod 32)
 * and one stream of 16-bit renormalisation words per tile, taken in
 * increasing lane order within each step of 32 bytes.
 * Layout (little-endian): a 64-byte header ("ACLE", u32 version 1, u64 size
 * of the v1 container, u64 raw prefix bytes, u32 streams = 17, u32 tile
 * size = 65536, u64 n_tokens, u64 n_literals, u64 n_tiles, u64 payload
 * offset); the v1 header and block directory raw, padded to 16 bytes; per
 * stream (the 16 byte planes of the token array, plane k = byte k of every
 * token, then the literal bytes) u64 length and u64 first tile; per tile
 * u64 payload offset (16-byte aligned, from the payload offset), u32
 * payload bytes, u32 tile bytes; the payloads: u16 freq[256], u32
 * state[32], u32 n_words, u16 words[n_words].
 * host_buf is read during the call only; the handle owns the decoded
 * tokens and literals (the v1 layout) like any handle.  Synchronizes the
 * stream.  ACLZ_E_CORRUPT for a malformed ACLE, a tile whose table does
 * not sum to 2^12, or a tile whose decode does not consume exactly its
 * words and end every state at 2^16; then as aclz_upload_ex. */
int aclz_upload_acle(const void *host_buf, uint64_t n, uint32_t flags, void *stream, aclz_handle **out);

/* aclz_upload_acle that also records two caller events (cudaEvent_t, each
 * created by the caller, or NULL) on the stream: ev_begin just before the
 * device tile decode (after the copies to the device) and ev_end after the
 * byte planes are turned into tokens, so the entropy stage can be timed
 * alone.  A measurement aid; the paper times its entropy stage apart from
 * the match phase as well (ANS 9% / match 91%, Sec. V). */
int aclz_upload_acle_ev(const void *host_buf, uint64_t n, uint32_t flags, void *stream, aclz_handle **out,
                        void *ev_begin, void *ev_end);

/* Host side of the entropy stage: the ACLE form (layout above) of the v1
 * container host_container[0, n).  Each 64 KiB tile of each stream is coded
 * on its own (frequencies: the only byte value present takes all of 2^12;
 * otherwise each present value max(1, floor(count * 2^12 / n)), the
 * difference to 2^12 settled on the largest frequency, lowest byte value
 * first), so the tiles are coded in parallel on `threads` host threads
 * (0: all hardware threads); the output does not depend on the thread
 * count.  aclz_acle_bound gives the largest size the call can write.
 * ACLZ_E_CORRUPT for an invalid v1 container, ACLZ_E_CAPACITY when cap is
 * too small (nothing written past cap). */
int aclz_acle_bound(const void *host_container, uint64_t n, uint64_t *out);
int aclz_acle_encode(const void *host_container, uint64_t n, int threads, void *host_out, uint64_t cap,
                     uint64_t *out_size);

/* Write the handle's stream back as a host container, with the wave tags
 * the upload computed (flag and n_waves set, per-block max wave in the
 * directory), so a later upload of it only checks the tags, in parallel,
 * instead of computing them in block order.  The container format and the
 * tags are those the encoder could have written (Sec. I: the wavefront's
 * waves); a reshaped handle exports its rewritten tokens.  host_out NULL:
 * only *out_size.  ACLZ_E_CAPACITY when cap is too small, ACLZ_E_INVAL for
 * a handle uploaded with ACLZ_UPLOAD_FLATTEN from an untagged container
 * (its 0/1 tags are not a legal wave tagging). */
int aclz_export(const aclz_handle *h, void *host_out, uint64_t cap, uint64_t *out_size);

/* Free a handle and its device memory (after its work has completed). */
int aclz_free(aclz_handle *h);

/* Sizes of the uploaded stream and of its decode schedule: total_len,
 * n_tokens, n_literals, block_size, n_blocks, min_match as in the
 * container; n_waves and n_deferred (work items of waves >= 1) as the
 * schedule stands (after aclz_flatten: 2 and the number of pieces). */
int aclz_handle_info(const aclz_handle *h, aclz_info *out);

/* Per-wave deferred-match counts (wave 0 holds literals and in-order
 * matches and reports 0); writes min(cap, n_waves) values. */
int aclz_wave_counts(const aclz_handle *h, uint64_t *counts, uint32_t cap);

/* Wave tags as computed or validated at upload (one per token), copied
 * to host memory. */
int aclz_tags(const aclz_handle *h, uint32_t *host_tags, uint64_t cap);

/* Re-point every deferred match at the bytes it copies that are final
 * after wave 0 (literal bytes or in-order match bytes), splitting it into
 * pieces, and rebuild the decode schedule as two waves: wave 0, then all
 * pieces, which are independent.  Absolute back-references (abstract;
 * Sec. I) make this exact: a match may copy equal bytes from wherever the
 * match that wrote them read them.  Removes the chains that force many
 * waves in the wavefront decode (Sec. I) on data whose copies copy copies
 * (for example FASTQ-like records at 6/8/10/12).  Decode output is
 * unchanged; afterwards aclz_handle_info reports n_waves = 2 and
 * n_deferred = the number of pieces (16 B of device memory each), and
 * aclz_tags still returns the container's wave tags.  Pointer doubling on
 * the GPU, about log2(waves) + 1 rounds.  Synchronizes the stream; no
 * decode of h may be in flight.  Idempotent.  ACLZ_E_NOMEM when the pieces
 * do not fit, ACLZ_E_UNSUPPORTED beyond 2^32 - 16 pieces. */
int aclz_flatten(aclz_handle *h, void *stream);

/* Shorten the copy chains of the wavefront schedule: `rounds` rounds of the
 * pointer doubling of aclz_flatten (each halving the chains a match's
 * source bytes go through), after which every deferred match is rewritten
 * as consecutive tokens, one per piece (the first keeps its literal run),
 * and the decode index (minimal wave tags, worklists, schedule) is rebuilt
 * for them.  Fewer waves (about halved per round) for more, shorter
 * matches.  Decode and seek output are unchanged; aclz_handle_info then
 * reports the new token and wave counts and aclz_tags the new tags.
 * rounds 0 (or no deferred match) is a no-op; rounds > 32 or a flattened
 * handle: ACLZ_E_INVAL.  Synchronizes; no decode of h may be in flight.
 * After any other error the handle is left part-way and must be freed. */
int aclz_reshape(aclz_handle *h, uint32_t rounds, void *stream);

/* Regroup the persistent schedule into work ranges: runs of consecutive
 * deferred matches of one wave (wave-major, block order), of about
 * range_bytes of matches (at least 8 matches, at most 4096) in large waves;
 * a wave with fewer matches than about 16 ranges per SM of that size is cut
 * into that many ranges (down to one match each), so the short dependency
 * hops at the start and end of the wavefront (Sec. I) run one match per
 * group.  A range may cut one block's matches of a wave in two, unless one
 * of them reads another's output.  Upload picks 20 KiB.  Synchronizes the
 * stream.  Used by the autotuner. */
int aclz_set_range_bytes(aclz_handle *h, uint32_t range_bytes, void *stream);

typedef struct aclz_decode_cfg {
    uint32_t G;           /* cooperating lanes per group: 8, 16 or 32 */
    uint32_t mode;        /* ACLZ_MODE_WAVES or ACLZ_MODE_PERSISTENT */
    uint32_t ctas_per_sm; /* persistent mode: resident CTAs per SM (0 = most) */
    uint32_t flags;       /* ACLZ_FLAG_* */
} aclz_decode_cfg;

#define ACLZ_MODE_WAVES 0      /* wave 0, then one kernel per wave */
#define ACLZ_MODE_PERSISTENT 1 /* wave 0, then one launch with bounded per-block waits */
#define ACLZ_MODE_AUTO 2       /* persistent + staged when deferred matches average >= 192 B, else waves */
#define ACLZ_FLAG_STAGED 1u    /* persistent: stage long matches through shared memory (TMA) */
#define ACLZ_FLAG_REGISTERS 2u /* persistent: copy through registers only */

/* Decode the whole stream into d_out (cap >= total_len bytes, 16-byte
 * aligned).  Enqueues on stream; capturable in a CUDA graph (no allocation,
 * no synchronization).  cfg NULL = {32, ACLZ_MODE_AUTO, 0, 0}.  The
 * persistent mode stages long matches through shared memory when the
 * deferred matches average at least 192 bytes, unless a flag forces one
 * copy path. */
int aclz_decode_all(aclz_handle *h, void *d_out, uint64_t cap, const aclz_decode_cfg *cfg,
                    void *stream);

/* aclz_decode_all that also records phase_event (a cudaEvent_t owned by the
 * caller) on stream between its two phases: after the wave-0 kernel
 * (literals and in-order matches; the wavefront decode of Sec. I) and before the deferred
 * matches of waves >= 1.  With its own events before and after the call a
 * caller times each phase on the launching stream.  phase_event NULL is
 * aclz_decode_all; a failed record is reported by the next CUDA call. */
int aclz_decode_all_ev(aclz_handle *h, void *d_out, uint64_t cap, const aclz_decode_cfg *cfg,
                       void *stream, void *phase_event);

/* What aclz_decode_all would launch for this handle and cfg (no GPU work):
 * *resolved = cfg with ACLZ_MODE_AUTO resolved and the copy-path flag set;
 * *launches = kernel launches of one call (wave 0, then one persistent
 * launch or one per non-empty wave >= 1; 0 for an empty stream).  Either
 * output may be NULL.  ACLZ_E_INVAL for a bad cfg, as aclz_decode_all. */
int aclz_decode_plan(const aclz_handle *h, const aclz_decode_cfg *cfg, aclz_decode_cfg *resolved,
                     uint32_t *launches);

/* Range decode (seek): write decode(stream)[lo, hi) to d_out (16-byte
 * aligned, hi - lo bytes) without decoding the rest.  Absolute
 * back-references let every output byte be traced back to the literal it
 * copies (abstract; Sec. I: random access without whole-file
 * decompression); only literals are read, never the output of other
 * calls.  0 <= lo <= hi <= total_len, hi - lo < 4 GiB.  Enqueues on stream;
 * no allocation. */
int aclz_decode_range(aclz_handle *h, uint64_t lo, uint64_t hi, void *d_out, void *stream);

/* Device scratch bytes that aclz_decode_ranges needs for n requests. */
int aclz_ranges_scratch_bytes(uint32_t n_requests, uint64_t *out);

/* Several range decodes in one launch: request i writes
 * decode(stream)[host_lo[i], host_hi[i]) to host_out[i] (device pointers,
 * 16-byte aligned).  The request table is copied to d_scratch
 * (aclz_ranges_scratch_bytes) and the stream is synchronized once for that
 * copy before the launch is enqueued. */
int aclz_decode_ranges(aclz_handle *h, uint32_t n, const uint64_t *host_lo, const uint64_t *host_hi,
                       void *const *host_out, void *d_scratch, uint64_t scratch_cap, void *stream);

/* One range request for aclz_decode_ranges_async: decode(stream)[lo, hi)
 * into d_out (device, 16-byte aligned); seg_base is filled in by the call. */
typedef struct aclz_range_req {
    uint64_t lo, hi;
    void *d_out;
    uint64_t seg_base;
} aclz_range_req;

/* Like aclz_decode_ranges without any copy or synchronization: reqs must
 * be host memory the device can read (pinned, e.g. cudaHostAlloc) and must
 * stay allocated and unchanged until the launch has completed on stream;
 * the kernel reads the table from there.  For serving loops that overlap
 * many batches. */
int aclz_decode_ranges_async(aclz_handle *h, uint32_t n, aclz_range_req *reqs, void *stream);

/* Batched decode (many independent streams in one launch): merge n host
 * containers of one block size into one container whose stream i starts
 * on a block boundary at *out_offsets[i]; its sources are rebased by that
 * offset (streams never reference one another) and its last block is
 * padded with zero literals up to the block size.  Decoding the merged
 * container writes stream i to [out_offsets[i], out_offsets[i] +
 * total_len_i).  host_out NULL: only *out_size (the size needed) and the
 * offsets are computed.  Wave tags are kept when every input has them. */
int aclz_batch_merge(uint32_t n, const void *const *host_bufs, const uint64_t *sizes, void *host_out,
                     uint64_t cap, uint64_t *out_size, uint64_t *out_offsets);

/* CUDA graph of one aclz_decode_all(h, d_out, cap, cfg) call, captured on
 * a private stream after one plain decode on `stream` (which it
 * synchronizes).  Launching the graph repeats the whole decode.  Errors as
 * aclz_decode_all; *out is owned by the caller (aclz_graph_free). */
typedef struct aclz_graph aclz_graph;
int aclz_graph_create(aclz_handle *h, void *d_out, uint64_t cap, const aclz_decode_cfg *cfg, void *stream,
                      aclz_graph **out);

/* Enqueue the captured decode on `stream` (asynchronous; the handle, the
 * output buffer and the graph must stay alive until it completes). */
int aclz_graph_launch(aclz_graph *g, void *stream);

/* Destroy a graph (after its launches have completed). */
int aclz_graph_free(aclz_graph *g);

/* ---- learned per-block thresholds (no counterpart in the paper's
 * decoder; the paper's lever, Sec. IV-B/IV-C, is a fixed vector of minimum
 * match lengths by distance class, and the network chooses one of K such
 * vectors per block).  FP32 MLP 24 -> 64 -> 64 -> K (2 <= K <= 16), ReLU,
 * parameters one flat device array in the order W1[24][64], b1[64],
 * W2[64][64], b2[64], W3[64][K], b3[K] (row-major). */
uint32_t aclz_mlp_param_count(uint32_t K);

/* Bytes of scratch aclz_mlp_grad needs for a batch. */
uint64_t aclz_mlp_scratch_bytes(uint32_t K, uint32_t batch);

/* logits[batch][K] = MLP(x[batch][24]). */
int aclz_mlp_forward(const float *d_params, uint32_t K, const float *d_x, uint32_t batch, float *d_logits,
                     void *stream);

/* Mean softmax cross-entropy of labels y (0 <= y < K) and its gradient
 * with respect to every parameter (d_grad, param_count floats; *d_loss one
 * float, may be NULL).  Per-tile partials are summed in a fixed order. */
int aclz_mlp_grad(const float *d_params, uint32_t K, const float *d_x, const int32_t *d_y, uint32_t batch,
                  float *d_grad, float *d_loss, void *d_scratch, uint64_t scratch_bytes, void *stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected; step
 * counts from 1) on d_params with moments d_m, d_v. */
int aclz_mlp_adam(float *d_params, float *d_m, float *d_v, const float *d_grad, uint32_t K, uint32_t step,
                  float lr, void *stream);

/* Ten byte statistics per block of block_size bytes of d_x (n bytes):
 * order-0 entropy / 8, distinct byte values / 256, fraction of bytes equal
 * to the previous one, 4-gram and 8-gram repeat rates (linear counting over
 * a 65536-bit hash map), fractions of digits, lowercase, uppercase,
 * space/punctuation and other bytes.  d_feat: [n_blocks][10] floats. */
int aclz_block_features(const void *d_x, uint64_t n, uint32_t block_size, float *d_feat, void *stream);

/* Synchronize stream and return the device status latched by decode
 * calls on h since the last call (ACLZ_OK, ACLZ_E_TIMEOUT, ACLZ_E_DEVICE). */
int aclz_device_status(aclz_handle *h, void *stream);

/* Failure-detection self-test (no counterpart in the paper): one group waits
 * on a completion word that nothing sets, with the bounded wait the
 * persistent decode uses on its source blocks, for at most spin_limit polls
 * (1 .. 2^22).  Returns ACLZ_E_TIMEOUT, the expected outcome: the wait gave
 * up, set the error word and the kernel returned, leaving the context
 * usable.  ACLZ_OK would mean the wait did not time out.  Synchronizes. */
int aclz_selftest_wait(uint32_t spin_limit, void *stream);

/* FNV-1a 64 of each 64 KiB chunk of d_buf, then FNV-1a 64 of the chunk
 * hashes (8 LE bytes each) followed by n (8 LE bytes).  Synchronous:
 * *out_hash holds the result on return.  Allocates stream-ordered scratch
 * of 8 bytes per chunk. */
int aclz_fnv(const void *d_buf, uint64_t n, uint64_t *out_hash, void *stream);

/* Same hash as aclz_fnv, for callers that must not allocate device memory
 * during the call (a nearly full device, memory owned by an arena or pool
 * manager, a latency-critical path that must stay out of the allocator).
 * The paper has no counterpart; this is a library convenience.  The chunk
 * hashes go to one fixed 512 KiB array inside the library, so n is limited
 * to 4 GiB (65536 chunks of 64 KiB): larger n returns ACLZ_E_CAPACITY.
 * The first call on each device looks up that array's device address (make
 * that first call before any stream capture).  All calls share the array:
 * calls that overlap on the GPU race and may return wrong hashes.
 * Synchronous: *out_hash holds the result on return.  No cudaMalloc or
 * cudaFree is made. */
int aclz_fnv_noalloc(const void *d_buf, uint64_t n, uint64_t *out_hash, void *stream);

const char *aclz_strerror(int code);

/* The cudaError_t value behind the most recent ACLZ_E_CUDA (0 if none),
 * process-wide. */
int aclz_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ACLZ_H */
