/*
 * aceapex.h — C ABI of the GB300 (sm_103a) decoder for the blockwise
 * absolute-offset LZ77 format studied in "What Actually Serializes GPU LZ77
 * Decode" (format v1).
 *
 * What the paper defines (section names of the paper):
 *  - Setup: every back-reference is an absolute position in the decompressed
 *    output; the encoder searches matches globally and cuts the output into
 *    fixed 16 KiB blocks; a block can be decoded once the blocks holding its
 *    sources exist; each block stores four streams — literals, lengths,
 *    absolute offsets, commands — behind an ANS entropy stage (Table 1).
 *  - "The Last Sequential Element": repeat matches take their distance from
 *    a four-entry history; lengths are varints; everything else in the parse
 *    is a prefix sum; an encoder flag drops the history (history-free
 *    encoding, same format, same decoder).
 *  - "What Does: Periods, Not Chains": a self-overlapping match is the
 *    periodic fill out[dst+k] = out[src + (k mod dist)].
 * The byte layout the paper leaves open is fixed by format v1 (see the
 * design notes): 64-byte header, four 256-entry frequency tables summing to
 * 4096, a 40-byte index entry per block, and per-block payloads of four
 * stream bodies (stored, or interleaved rANS with K <= 128 lanes, 32-bit
 * states, 16-bit words, 12-bit probabilities).
 *
 * Conventions for every function:
 *  - Return value: ACEAPEX_OK (0) or a negative ACEAPEX_E_* status.  The
 *    library never prints; aceapex_last_error() gives a message.
 *  - "device pointer": memory of the context's CUDA device (cudaMalloc or a
 *    framework allocator); "host pointer": ordinary host memory.
 *  - "stream": a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Decode calls enqueue work on it; the synchronous variants then
 *    synchronise that stream and read the device error word.
 *  - A context is not thread-safe and its scratch is reused by every call:
 *    use one context per concurrently running stream.
 *  - Corrupt input never traps or hangs: it returns ACEAPEX_E_CORRUPT (or
 *    ACEAPEX_E_TIMEOUT if a dependency wait ran out); the output content is
 *    then undefined.
 */
#ifndef ACEAPEX_H
#define ACEAPEX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ACEAPEX_OK 0
#define ACEAPEX_E_ARG (-1)      /* bad argument (null pointer, too-small buffer, ...) */
#define ACEAPEX_E_CORRUPT (-2)  /* archive violates format v1 */
#define ACEAPEX_E_NOMEM (-3)    /* host or device allocation failed */
#define ACEAPEX_E_CUDA (-4)     /* a CUDA runtime call failed */
#define ACEAPEX_E_TIMEOUT (-5)  /* a device-side dependency wait exceeded its limit */
#define ACEAPEX_E_RANGE (-6)    /* requested range outside the archive */
#define ACEAPEX_E_BUSY (-7)     /* admission refused (serving) */

#define ACEAPEX_BLOCK_SIZE 16384u

typedef struct aceapex_ctx aceapex_ctx;
typedef struct aceapex_archive aceapex_archive;

/* Encoder parameters (0 fields select defaults). */
typedef struct {
    int no_rep;          /* 1: history-free encoding (no repeat codes; paper's encoder flag) */
    uint32_t min_match;  /* minimum match length, >= 4 (default 4) */
    uint32_t max_lanes;  /* rANS lane cap K, power of two <= 128 (default 32) */
    int threads;         /* encoder threads (default: hardware concurrency) */
    int latest_source;   /* 1: long-range matches point at the latest earlier copy of their
                            content (classic hash-chain choice); 0 (default): at the first
                            occurrence, which costs the same with absolute offsets and keeps
                            cross-block dependency chains short */
    uint32_t max_depth;  /* cap on the chain depth of any byte (a match only reads bytes whose
                            own chains are shorter); 0 = default 16, 0xFFFFFFFF = no cap.
                            Paper, "Depth Does Not Govern Latency": a depth bound is an
                            encode-time choice of matches */
    int short_latest;    /* 1: short-range matches point at the latest copy (default 0: the
                            oldest copy inside the short-range window) */
    int deps;            /* 1: write each block's dependency list (the earlier blocks its matches
                            read), so range decodes touch only a block's dependency closure
                            (paper, Random Access at Scale); 0 (default): no lists, a range
                            decode then covers every block up to the range */
    uint64_t segment;    /* 0 (default): one parse over the whole input.  Else a multiple of
                            16 KiB: the input is parsed as independent segments of this size
                            (sources stay inside their segment, like a genome's chromosomes),
                            in parallel on `threads` threads, into one archive */
    int levels;          /* 1: write each block's level body (flags bit1): one byte per token, its
                            cross-block level (see aceapex_enc_stats), a scheduling hint for a
                            cross-block pass that takes the levels in order (paper, "Depth Does
                            Not Govern Latency": waves).  Decoders may ignore it; it never changes
                            the decoded bytes.  0 (default): no level bodies */
} aceapex_enc_params;

/* Decoder variants. */
#define ACEAPEX_VARIANT_FAST 0   /* scan parse + periodic fill + dependency dataflow */
#define ACEAPEX_VARIANT_PLAIN 1  /* serial parse with history, byte-serial copies (comparison) */
#define ACEAPEX_VARIANT_FUSED 2  /* FAST, with a whole-archive decode's entropy stage and local pass in one
                                    kernel, entropy warps and local groups side by side on every SM
                                    (comparison: slower on GB300, see the design notes) */

typedef struct {
    uint32_t variant;     /* ACEAPEX_VARIANT_* */
    uint32_t timeout_us;  /* limit of every device-side dependency wait (default 2,000,000) */
    uint32_t ctas_per_sm; /* persistent CTAs per SM for the local pass (0 = occupancy maximum) */
    uint32_t rans_ctas_per_sm; /* persistent CTAs per SM for the entropy stage (0 = occupancy maximum) */
    uint32_t queue_chunk; /* blocks a warp (entropy stage) or CTA (local pass) takes per queue ticket (0 = 1) */
    uint32_t wait_ns;     /* cross-block pass, first round: how long a match piece may wait for its sources
                             before it is left to the later, barrier-separated rounds; 0xFFFFFFFF = no limit
                             short of timeout_us (pieces are handed out in output order, so the lowest
                             unfinished one always has final sources and the first round finishes them all);
                             0 = automatic: no limit while the pending pieces are at most 16 per thread of the
                             pass's grid and 256 per block, else 4000 (many pieces with long chains would clog
                             the hand-out), or, for an archive with level bodies, level order with 20000 */
    uint32_t ignore_levels; /* 0: a whole-archive decode of an archive with level bodies (flags bit1) takes
                               the cross-block matches level by level (paper, "Depth Does Not Govern
                               Latency": one round per wave, every piece attempted once, a piece whose
                               hint proves too low left to the later rounds); 1: ignore the level bodies */
} aceapex_dec_params;

/* Timing of the last call, measured with CUDA events on the call's stream
 * (filled only when stats is non-NULL; timing adds event records). */
typedef struct {
    double ms_total;  /* whole call, device time */
    double ms_ans;    /* entropy stage (rANS decode of the four streams); with the fused kernel only the
                         reset launches before it */
    double ms_parse;  /* local pass: parse, literals and in-block matches; with the fused kernel the
                         entropy stage and the local pass together */
    double ms_copy;   /* cross-block pass: matches whose source chain leaves their block */
    uint64_t blocks;  /* blocks decoded */
    uint64_t bytes;   /* bytes written to the output */
    uint64_t pending_spans;  /* matches left to the cross-block pass */
    uint64_t wait_polls;     /* cross-block rounds after the first (the dependency depth met) */
    uint64_t pending_bytes;  /* bytes of the matches left to the cross-block pass */
} aceapex_stats;

typedef struct {
    uint64_t total_size;    /* decompressed bytes */
    uint32_t n_blocks;
    uint32_t flags;         /* bit0: encoded history-free */
    uint32_t min_match;
    uint32_t max_tokens;    /* largest token count of a block */
    uint64_t archive_bytes;
    uint64_t tokens;        /* total tokens */
} aceapex_archive_info;

/* Status code -> static message. */
const char* aceapex_status_string(int status);
/* Last error message of a context (static storage inside the context). */
const char* aceapex_last_error(const aceapex_ctx* ctx);

/* Create a context on CUDA device `device`.  params may be NULL (defaults).
 * The context owns the decode scratch (device memory, grown on demand by
 * the decode calls, freed by aceapex_ctx_destroy). */
int aceapex_ctx_create(int device, const aceapex_dec_params* params, aceapex_ctx** out);
int aceapex_ctx_destroy(aceapex_ctx* ctx);
int aceapex_ctx_set_params(aceapex_ctx* ctx, const aceapex_dec_params* params);

/*
 * Encode n bytes (host pointer src) into a format v1 archive.  *out is
 * allocated by the library (host memory) and must be released with
 * aceapex_free.  Paper, Setup: global match search, absolute offsets, 16 KiB
 * blocks; "The Last Sequential Element": no_rep drops the repeat codes.
 */
int aceapex_encode(const uint8_t* src, uint64_t n, const aceapex_enc_params* params, uint8_t** out,
                   uint64_t* out_len);
void aceapex_free(void* p);

/*
 * Chain-depth statistics of an encode (paper, "Depth Does Not Govern
 * Latency": the depth of the copy chains, and how a cap on it is an
 * encode-time choice).  A literal byte has depth 0; the bytes of a match have
 * depth 1 + the deepest byte of the source window the match reads ([src,
 * src + min(distance, length)): one period of a self-overlapping match).
 * Depths saturate at 255.  block_max_depth[d] counts the blocks whose deepest
 * byte has depth d; match_depth[d] counts the matches of depth d.
 */
typedef struct {
    uint64_t blocks, matches;
    uint64_t block_max_depth[256];
    uint64_t match_depth[256];
    /* Cross-block levels: a match whose source window lies in its own block and
     * holds only level-0 bytes is finished by the decoder's local pass (level
     * 0); any other match has level 1 + the highest level in its window.
     * match_level[l] / level_bytes[l]: matches of level l and their bytes.  A
     * cross-block pass that took the levels in order would finish every match
     * of level l in its l-th round, so the highest level is the number of such
     * rounds (paper, "Depth Does Not Govern Latency": waves). */
    uint64_t match_level[256];
    uint64_t level_bytes[256];
} aceapex_enc_stats;
/* aceapex_encode that also fills *stats (host pointer, may be NULL). */
int aceapex_encode_ex(const uint8_t* src, uint64_t n, const aceapex_enc_params* params, uint8_t** out,
                      uint64_t* out_len, aceapex_enc_stats* stats);

/*
 * Open an archive for decoding.  d_arc: device pointer to the archive bytes
 * (caller-owned, must stay valid until aceapex_archive_close).  h_arc: host
 * pointer to the same bytes (read during this call only; the header, index
 * and block descriptors are validated here and a device-resident decode plan
 * is built).  The archive object owns the plan (device memory).
 */
int aceapex_archive_open(aceapex_ctx* ctx, const void* d_arc, const void* h_arc, uint64_t arc_len,
                         aceapex_archive** out);
int aceapex_archive_close(aceapex_archive* arc);
/* Host-only structural validation of an archive (header, tables, index,
 * payload descriptors); no device work.  info may be NULL.  Returns
 * ACEAPEX_OK or ACEAPEX_E_CORRUPT. */
int aceapex_archive_check(const void* h_arc, uint64_t arc_len, aceapex_archive_info* info);
int aceapex_archive_get_info(const aceapex_archive* arc, aceapex_archive_info* info);

/*
 * Decode the whole archive into d_out (device pointer, out_cap >= total
 * size) — the paper's full device-resident decode (Table 2: ANS + parse +
 * copy).  Enqueued on `stream`; the _async variant returns after enqueueing
 * (errors accumulate in the context until aceapex_sync), the plain variant
 * synchronises the stream and returns the decode status.  The cross-block
 * pass is a cooperative launch; the library orders all of its cooperative
 * launches on a device (each waits, on its stream, for the previous one to
 * complete), so decodes on different streams or contexts overlap in their
 * other stages only.  (Launches recorded into a CUDA graph are not ordered.)
 */
int aceapex_decode_all(aceapex_ctx* ctx, aceapex_archive* arc, void* d_out, uint64_t out_cap, void* stream,
                       aceapex_stats* stats);
int aceapex_decode_all_async(aceapex_ctx* ctx, aceapex_archive* arc, void* d_out, uint64_t out_cap,
                             void* stream);
/* Synchronise `stream` and return (and clear) the context's device error status. */
int aceapex_sync(aceapex_ctx* ctx, void* stream);

/*
 * Build the archive's match index: a parse-only pass on the device (entropy
 * stage without literals, then the token scans) lists every match's
 * destination, length and absolute source; the index is kept in host memory
 * with the archive (about 12 bytes per match) until aceapex_archive_close.
 * With it, range decodes and servers follow the byte-level closure of a
 * region (paper, Random Access at Scale and "The byte-level refutation": a
 * byte needs only the bytes it was copied from) instead of whole blocks.
 * Synchronous; uses the context's stream-independent scratch.
 */
int aceapex_archive_index(aceapex_ctx* ctx, aceapex_archive* arc);

/*
 * Parse statistics of an archive, counted from the device's parse-only pass
 * (the same pass that builds the match index; it is run if the archive has
 * no index yet).  Paper, "The Last Sequential Element": the commands that
 * read the four-entry history (repeat codes) are the parse's only sequential
 * element; the runs between them are what a scan parse can take at once.
 *  - runs: each block's tokens are cut at every repeat-coded token; a run is
 *    the count of non-repeat tokens before a repeat-coded token, back to the
 *    previous one or the block start, plus one trailing run per block (the
 *    history resets per block, so a block boundary ends a run).  Runs of
 *    length 0 count.  median_run is the element of rank floor(runs / 2) of
 *    the sorted run lengths.
 *  - multibyte_values: length values of 128 or more (two or more LEB128
 *    bytes in a canonical encoding).
 *  - overlap_matches: matches with distance < length (periodic fills);
 *    external_matches: matches whose source starts before their block.
 * Blocks the parse finds corrupt are left out and counted in bad_blocks.
 * Synchronous; stats must not be NULL.
 */
typedef struct {
    uint64_t blocks, tokens, new_matches, rep_matches[4], lit_only;
    uint64_t values, multibyte_values;
    uint64_t literal_bytes, match_bytes, overlap_matches, external_matches;
    uint64_t max_tokens_block;
    uint64_t runs, run_len_sum, median_run, max_run;
    uint64_t bad_blocks;
} aceapex_parse_stats;
int aceapex_archive_parse_stats(aceapex_ctx* ctx, aceapex_archive* arc, aceapex_parse_stats* stats);

/*
 * Decode the original bytes [start, start + len) into d_out (device pointer,
 * len bytes).  Paper, Random Access at Scale: only what the region depends on
 * is decoded, into context scratch, and the region is gathered out.  With a
 * match index (aceapex_archive_index) that is the byte-level closure: the
 * matches writing the region's bytes, their source windows, and so on, the
 * other matches of those blocks being left undone.  Otherwise it is the
 * block-level closure: through the archive's dependency lists when it has
 * them (aceapex_enc_params.deps), else every block up to the region's last.
 * A source outside its block's dependency list is ACEAPEX_E_CORRUPT.
 * Returns ACEAPEX_E_RANGE when the region leaves the archive.  Synchronises
 * `stream`; stats (may be NULL): blocks = closure size, bytes = len, ms_copy
 * includes the gather.
 */
int aceapex_decode_range(aceapex_ctx* ctx, aceapex_archive* arc, uint64_t start, uint64_t len, void* d_out,
                         void* stream, aceapex_stats* stats);

/*
 * Sharded decode over several GPUs (one process per GPU): the output blocks
 * are split into n_ranks contiguous ranges of nearly equal block counts, and
 * rank `rank` gets [*start, *start + *len).  Each rank decodes its range with
 * aceapex_decode_range — its byte-level closure, so the sources it needs from
 * other ranks' ranges are decoded redundantly and no collective is on the
 * path; an all-gather of the ranges (if the caller wants the whole output on
 * every GPU) comes after.  Pure arithmetic, no device work.
 */
int aceapex_shard_range(uint64_t total, int n_ranks, int rank, uint64_t* start, uint64_t* len);

/*
 * Serving: a request loop over one archive held compressed in device memory
 * with a bounded cache of decoded blocks (paper, Random Access at Scale; the
 * paper's persistent seek queue).  A worker thread admits the requests that
 * have arrived, in arrival order, while the cache can hold their byte-level
 * dependency closure (the match index is built at creation if the archive
 * has none), and decodes each tick's union of closures, minus the bytes the
 * cache keeps, with one launch sequence into cache slots followed by one
 * gather into the requests' buffers.  Ticks go to `streams` lanes (each a
 * stream with its own context and scratch, up to two ticks deep), so that a
 * tick formed while others run starts on the device beside them; a tick
 * that reads a block another unfinished tick decodes, or decodes a block
 * another unfinished tick reads, waits for that tick's completion.
 * Requests that arrive while ticks run join the next tick.  Admission is by memory: a request waits while its closure needs more free
 * or evictable slots than there are, and completes with ACEAPEX_E_BUSY if it
 * could never fit.  Blocks read by unfinished ticks are pinned; the others
 * are evicted least recently used first.  The archive must stay open while
 * the server exists; the server uses its own context and stream.
 */
typedef struct aceapex_server aceapex_server;
typedef struct {
    uint64_t cache_bytes;        /* decoded-block cache (device memory; default 4 GiB) */
    uint32_t max_tick_blocks;    /* blocks one tick decodes at most (default 16384) */
    uint32_t max_tick_requests;  /* requests one tick gathers at most (default 4096) */
    uint32_t streams;            /* tick lanes, 1..16 (default 2) */
} aceapex_server_params;
typedef struct {
    uint64_t id;
    int status;               /* ACEAPEX_OK, ACEAPEX_E_BUSY (can never fit), or a decode error */
    uint32_t closure_blocks;  /* blocks the request read (decoded or kept) */
    uint32_t decoded_blocks;  /* blocks it added to its tick's decode */
    double latency_us;        /* arrival -> completion seen by the server */
    double queue_us;          /* arrival -> admission */
} aceapex_completion;
typedef struct {
    uint64_t completed, failed, refused, bytes, ticks, blocks_decoded, blocks_hit;
    double p50_us, p99_us, mean_us, max_us;   /* latency of the completed requests */
    double closure_mean, closure_p50, closure_p99;
    double seconds;           /* first arrival -> last completion */
    double gbs;               /* bytes delivered / seconds */
    uint64_t tick_overlaps;   /* pairs of ticks whose device work overlapped in time */
    uint64_t tick_waits;      /* ticks that waited for a tick on another lane */
    double tick_host_ms;      /* host time forming the launched ticks (walks, admission, launches) */
    double walk_ms;           /* ... of which closure walks */
    double launch_ms;         /* ... of which staging, ordering, copies and launches on the lane's stream */
} aceapex_server_stats;

/* ctx: its device and decoder parameters are used (the server creates its own
 * context).  arc: opened on that device.  params may be NULL. */
int aceapex_server_create(aceapex_ctx* ctx, aceapex_archive* arc, const aceapex_server_params* params,
                          aceapex_server** out);
/* Nanoseconds since the server was created (its clock for arrivals). */
int64_t aceapex_server_now_ns(const aceapex_server* server);
/* Queue n requests: region [start[i], start[i] + len[i]) into d_out[i]
 * (device pointers, len[i] bytes, valid until the request completes),
 * arriving at at_ns[i] on the server clock (a later time schedules an
 * open-loop arrival; negative or at_ns NULL: now).  ids (may be NULL) gets
 * the request ids.  ACEAPEX_E_RANGE if a region leaves the archive (nothing
 * is queued then). */
int aceapex_server_submit_many(aceapex_server* server, int n, const uint64_t* start, const uint64_t* len,
                               void* const* d_out, const int64_t* at_ns, uint64_t* ids);
int aceapex_server_submit(aceapex_server* server, uint64_t start, uint64_t len, void* d_out, int64_t at_ns,
                          uint64_t* id);
/* Move up to max completions into out, waiting up to wait_ms for the first;
 * returns how many (or a negative status). */
int aceapex_server_poll(aceapex_server* server, aceapex_completion* out, int max, int wait_ms);
/* Wait until every submitted request has completed (ACEAPEX_E_TIMEOUT after timeout_ms). */
int aceapex_server_drain(aceapex_server* server, int timeout_ms);
/* Latency percentiles, throughput and cache figures since the last reset. */
int aceapex_server_get_stats(aceapex_server* server, int reset, aceapex_server_stats* out);
const char* aceapex_server_last_error(const aceapex_server* server);
int aceapex_server_destroy(aceapex_server* server);

/*
 * End-to-end decode from host memory: copies the archive (host pointer
 * h_arc, arc_len bytes, ideally pinned) to the device, decodes it, and copies
 * the output to h_out (host pointer, out_cap >= total size).  Device buffers
 * are context scratch.  `arc` must be an archive opened from the same bytes
 * (its plan is reused); pass NULL to open a temporary one.  The call is a
 * pipeline over chunks of blocks (512, then 1536, then 4096 each): a chunk's
 * payload bytes go up on a context stream, the chunk decodes on `stream` once
 * they have landed (its sources lie in its own or earlier blocks), and its
 * output comes down on a second context stream while the next chunk decodes.
 * The call returns when the last bytes are in h_out; work queued on `stream`
 * before it runs first.
 */
int aceapex_decode_host(aceapex_ctx* ctx, aceapex_archive* arc, const void* h_arc, uint64_t arc_len,
                        void* h_out, uint64_t out_cap, void* stream, aceapex_stats* stats);

/*
 * Batched decode: many archives decoded by one set of launches.  Paper,
 * Setup (Table 1): a persistent queue over blocks, whose time follows the
 * token count rather than the number of archives.  Here the kernels take
 * (archive, block) items from shared device tickets, so archives of any
 * size and encoding (history-bound or history-free) share the GPU.
 *
 * One item per archive: `arc` an archive opened on the batch's context (its
 * device bytes must stay valid while the batch exists), `d_out` a device
 * pointer with out_cap >= the archive's total size; `status` is written by
 * aceapex_batch_wait / aceapex_batch_run / aceapex_batch_decode with that
 * archive's own status (a corrupt archive fails alone: the others decode).
 * At most 3000 archives per batch.
 */
typedef struct {
    aceapex_archive* arc;
    void* d_out;
    uint64_t out_cap;
    int status;
} aceapex_batch_item;

typedef struct aceapex_batch aceapex_batch;

#define ACEAPEX_BATCH_GRAPH 1u  /* capture the decode launches into a CUDA graph once; runs replay it */

/* Build a reusable batch: validates the items, allocates the batch's own
 * device scratch (one partition per archive) and the device job table, and
 * with ACEAPEX_BATCH_GRAPH captures the launches into a CUDA graph.  The
 * context's decoder parameters at this call apply to every run.  The items
 * array is read during this call only; the batch decodes into the d_out
 * pointers given here. */
int aceapex_batch_create(aceapex_ctx* ctx, const aceapex_batch_item* items, int n, uint32_t flags,
                         aceapex_batch** out);
/* Enqueue one decode of every archive of the batch on `stream` (a graph
 * replay with ACEAPEX_BATCH_GRAPH).  Runs of one batch must not overlap. */
int aceapex_batch_run_async(aceapex_batch* batch, void* stream);
/* Synchronise `stream`, write each item's status into items[0..n) (may be
 * NULL), fill stats (may be NULL; the stage split only without a graph) and
 * return the first error of the run (ACEAPEX_OK when every archive decoded). */
int aceapex_batch_wait(aceapex_batch* batch, void* stream, aceapex_batch_item* items, aceapex_stats* stats);
/* aceapex_batch_run_async then aceapex_batch_wait. */
int aceapex_batch_run(aceapex_batch* batch, void* stream, aceapex_batch_item* items, aceapex_stats* stats);
int aceapex_batch_destroy(aceapex_batch* batch);
/* One-shot batch: create (no graph), run, destroy. */
int aceapex_batch_decode(aceapex_ctx* ctx, aceapex_batch_item* items, int n, void* stream, aceapex_stats* stats);

/*
 * Autotuner (the paper has none; its decoders fix their launch shapes).
 * Decodes the items as one batch under every point of the launch space —
 * persistent CTAs per SM of the local pass (1..its occupancy) and of the
 * entropy stage (1..its occupancy), blocks per queue ticket (1, 4, 16) — with
 * the L2 flushed before each timed run (median of `reps` after one warm-up),
 * writes up to max_points measured points, sets the context's parameters to
 * the fastest (variant and timeout unchanged) and copies them to *best.
 * The items' outputs are overwritten.  The encode-side lever of the same
 * tuning, the rANS lane count, is a property of the archive (encoder
 * max_lanes).
 */
typedef struct {
    uint32_t ctas_per_sm, rans_ctas_per_sm, queue_chunk;
    double ms;
} aceapex_tune_point;
int aceapex_autotune(aceapex_ctx* ctx, const aceapex_batch_item* items, int n, int reps, aceapex_tune_point* points,
                     int max_points, int* n_points, aceapex_dec_params* best);

/*
 * Decode without allocating anything (the paper has no counterpart: this is a
 * service of this library).  For callers that may not allocate device memory
 * at decode time: processes whose device memory belongs to a framework's pool,
 * and latency-bound paths where an allocation may stall or fail.  It needs no
 * context and no opened archive: d_arc (device pointer, arc_len bytes) is
 * validated and planned on the device, and all scratch lives in one static
 * device array of about 5.3 MiB that every device loading this library holds
 * until the process exits.  Limits: at most 64 blocks (1 MiB of output), at
 * most 2 MiB of decoded streams and 96K pending pieces; valid archives beyond
 * them return ACEAPEX_E_ARG, and an archive that aceapex_decode_all would
 * find corrupt returns ACEAPEX_E_CORRUPT.  Dependency lists, when the archive
 * has them, are checked as in aceapex_decode_all.  The output goes to d_out
 * (device pointer, out_cap >= the decompressed size).  The call enqueues on
 * `stream`, reads the device plan's summary back to the host and synchronises
 * the stream (twice), and returns the decode status; so it cannot be recorded
 * into a CUDA graph.  The first call on a device looks up the array's device
 * address.  Every call on a device shares the array and finds the previous
 * call's contents there (the call clears what must start at zero): calls that
 * overlap on the GPU (from other streams or threads) race and must be
 * serialised by the caller.
 */
int aceapex_decode_noalloc(const void* d_arc, uint64_t arc_len, void* d_out, uint64_t out_cap, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ACEAPEX_H */
