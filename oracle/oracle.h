/*
 * CPU oracle for the blockwise absolute-offset LZ77 format ("ACEAPEX",
 * format v1).  TEST INFRASTRUCTURE ONLY: plain, slow, single-threaded C that
 * states what the GPU decoder must compute.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it; the product
 * library never links or calls it, and it shares no code with the product.
 *
 * Paper facts it follows (section names of the paper):
 *  - Setup: back-references are absolute positions in the decompressed
 *    output; the output is cut into fixed 16 KiB blocks; each block stores
 *    four streams (literals, lengths, absolute offsets, commands).
 *  - Table 1 / Setup: an ANS entropy stage sits in front of the streams.
 *  - "The Last Sequential Element": a four-entry distance history serves
 *    repeat matches; lengths are varints; an encoder flag (history-free,
 *    NO_REP) suppresses repeat codes without changing the format.
 *  - "What Does: Periods, Not Chains": a self-overlapping match equals the
 *    periodic fill out[dst+k] = out[src + k mod dist].
 * Everything the paper leaves open (byte layout, ANS variant and parameters,
 * command codes, initial history) is fixed by the format v1 readings listed
 * in the design notes, and this header restates them where used.
 */
#ifndef ACEAPEX_ORACLE_H
#define ACEAPEX_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_OK 0
#define ORC_E_ARG -1
#define ORC_E_CORRUPT -2
#define ORC_E_NOMEM -3

#define ORC_BLOCK 16384u
#define ORC_PROB_BITS 12u
#define ORC_M 4096u
#define ORC_L 65536u

enum { ORC_CMD = 0, ORC_LEN = 1, ORC_OFF = 2, ORC_LIT = 3 };

/* FNV-1a, 64-bit (offset basis 0xcbf29ce484222325, prime 0x100000001b3). */
uint64_t orc_fnv1a64(const uint8_t* p, uint64_t n);

/* Normalise symbol counts to frequencies summing to 4096 (every present
 * symbol gets f >= 1).  All-zero counts give an all-zero table. */
int orc_normalize(const uint64_t counts[256], uint16_t freq[256]);

/* Interleaved rANS, K lanes, 32-bit states, 16-bit renormalisation words,
 * 12-bit probabilities.  Body = K u32 states (zero padded to 16 bytes), then
 * u16 words in decode order.  Returns the body length in bytes, or < 0. */
int64_t orc_rans_encode(const uint8_t* sym, uint32_t n, uint32_t K, const uint16_t freq[256], uint8_t* out,
                        uint64_t cap);
int orc_rans_decode(const uint8_t* body, uint64_t enc_len, uint32_t n, uint32_t K, const uint16_t freq[256],
                    uint8_t* out);

typedef struct {
    int no_rep;          /* 1: never emit repeat codes (history-free) */
    uint32_t min_match;  /* minimum match length (>= 4), also stored in the header */
    uint32_t new_min;    /* minimum length for an explicit-offset (NEW) match */
    uint32_t max_lanes;  /* rANS lane cap K (power of two, 1..128) */
    uint32_t chain;      /* hash-chain candidates examined per position */
} orc_enc_params;

void orc_enc_defaults(orc_enc_params* p);
/* Encode n bytes into a format v1 archive; *out is malloc'ed (free with orc_free). */
int orc_encode(const uint8_t* src, uint64_t n, const orc_enc_params* p, uint8_t** out, uint64_t* out_len);
void orc_free(void* p);

/* Decode a whole archive (byte-serial reference decode).  verify_fnv = 1
 * also checks each block's stored FNV-1a 64. */
int orc_decode(const uint8_t* arc, uint64_t arc_len, uint8_t* out, uint64_t out_cap, int verify_fnv);
/* Total decompressed size and block count from the header (validated). */
int orc_info(const uint8_t* arc, uint64_t arc_len, uint64_t* total, uint32_t* n_blocks, uint32_t* flags,
             uint32_t* min_match);

/* Per-token parse of one block from the oracle's sequential parse.  Arrays
 * must hold cap entries; returns the token count or < 0.  dst = output
 * position of the match start (after the literal run), src = absolute match
 * source, lit = index of the token's first literal in the block's literal
 * stream.  Needs the previous blocks only for validation of nothing: the
 * parse of a block is independent of all other blocks. */
int64_t orc_parse_block(const uint8_t* arc, uint64_t arc_len, uint32_t b, uint64_t cap, uint8_t* cmd,
                        uint32_t* ll, uint32_t* ml, uint64_t* dst, uint64_t* src, uint32_t* lit);

/* Decoded (pre-parse) stream of one block: which = ORC_CMD..ORC_LIT. */
int64_t orc_block_stream(const uint8_t* arc, uint64_t arc_len, uint32_t b, int which, uint8_t* out, uint64_t cap);

/* The level body of one block (archives with flags bit1): one byte per token,
 * returned as stored (hints, not checked).  ORC_E_ARG when the archive has
 * none. */
int64_t orc_block_levels(const uint8_t* arc, uint64_t arc_len, uint32_t b, uint8_t* out, uint64_t cap);

typedef struct {
    uint64_t n_blocks, n_tokens, n_new, n_rep[4], n_litonly;
    uint64_t n_values, n_multibyte_values;  /* varint values, and those longer than one byte */
    uint64_t n_match_bytes, n_literal_bytes, n_overlap_tokens;
    uint64_t n_external_tokens;             /* match source starts in an earlier block */
    uint64_t max_tokens_block;
    uint64_t hist_dependent;                /* tokens whose source comes from the history (REP) */
    uint64_t runs, run_len_sum, median_run;  /* dependency-free runs between REP tokens */
    uint64_t stream_raw[4], stream_enc[4];
} orc_stats;

int orc_archive_stats(const uint8_t* arc, uint64_t arc_len, orc_stats* st);

#ifdef __cplusplus
}
#endif
#endif
