// Internal definitions shared by the host library and the CUDA kernels.
// Format v1 constants and the device-resident decode plan.
#pragma once
#include <stdint.h>

namespace acx {

constexpr uint32_t kBlock = 16384;     // fixed block size (paper, Setup / Reproducibility: 16,384 B)
constexpr uint32_t kProbBits = 12;     // rANS probability precision
constexpr uint32_t kM = 1u << kProbBits;
constexpr uint32_t kL = 1u << 16;      // rANS lower bound of the state interval [L, 2^32)
constexpr int kCmd = 0, kLen = 1, kOff = 2, kLit = 3;
constexpr uint32_t kMaxLanes = 128;
constexpr uint32_t kMaxStreamRaw = 4 * kBlock + 16;

// Command codes of the cmd stream.
constexpr uint8_t kNew = 0;       // explicit absolute offset
constexpr uint8_t kRep0 = 1;      // 1..4: distance from history entry 0..3
constexpr uint8_t kLitOnly = 5;   // final literal run without a match

// Per-block decode plan (device-resident, built by the host at archive open).
struct BlockDev {
    uint64_t payload;      // archive offset of the block payload
    uint64_t scratch;      // offset of the block's decoded streams in the stream scratch
    uint32_t raw_len;      // decompressed bytes of the block
    uint32_t n_tok;        // tokens (= cmd stream length)
    uint32_t n_new;        // NEW tokens (= off stream length / 5)
    uint32_t rans_mask;    // bit s: stream s is rANS coded
    uint32_t s_raw[4];     // decoded lengths of cmd, len, off, lit
    uint32_t s_body[4];    // body offset relative to the payload
    uint32_t s_enc[4];     // body length in bytes (without padding)
    uint32_t s_off[4];     // offset of each decoded stream inside the block's scratch region
    uint8_t s_K[4];        // rANS lanes
    uint32_t span_base;    // first pending-span slot of the block (n_tok + kSpanSlack slots per block)
    uint32_t dep_off;      // the block's dependency list: deps[dep_off, dep_off + n_deps) (archives with lists)
    uint32_t n_deps;
    uint32_t lvl_body;     // payload offset of the block's level body (archives with levels), else 0
    uint32_t pad[3];
};
static_assert(sizeof(BlockDev) % 16 == 0, "BlockDev alignment");

// A pending piece: at most kPiece bytes of a match whose source chain leaves
// its block, left for the cross-block pass.  Long matches are cut into pieces
// so every piece is one lane's small copy.
//   x = source bits 0..31, y = source bits 32..39 | phase << 8 | level << 24,
//   z = destination offset in the block | length << 16, w = period.
// (phase < period < 16384; level: the token's level byte in level-ordered
// jobs, a scheduling hint, else 0.)
// period 0: byte j comes from source + j; otherwise from
// source + ((phase + j) mod period), source being the start of the match's
// period window (the periodic fill of a self-overlapping match).
constexpr uint32_t kPiece = 32;
constexpr uint32_t kSpanSlack = kBlock / kPiece;  // pieces a block may add beyond one per token
struct alignas(16) SpanRec {
    uint32_t x, y, z, w;
};

// One work item of a job that decodes chosen blocks of an archive (range
// decodes, serving ticks): the block, and where its pending pieces and
// decoded streams go in the job's scratch.
struct ItemDev {
    uint32_t block;
    uint32_t slot;            // output slot of the block
    uint32_t span_base;       // first pending-piece slot (n_tok + kSpanSlack slots)
    uint32_t need_n;          // 0: every byte of the block is wanted; else the wanted bytes are the
    uint64_t scratch;         // offset of the block's decoded streams
    uint32_t need_off;        //   need_n intervals ArcJob::need[need_off ..] (start | end << 16)
    uint32_t pad;
};
constexpr uint32_t kNoSlot = 0xffffffffu;  // slot-table entry of a block not in the output

// One region to copy out of the block slots after a subset decode.
struct GatherReq {
    uint8_t* dst;             // device destination (len bytes)
    uint64_t start, len;      // original byte range
};

// One archive inside a decode job.
struct ArcJob {
    const uint8_t* arc;       // archive bytes (device)
    const BlockDev* blk;      // plan
    const uint32_t* dtab;     // 4 x 4096 rANS decode entries: sym | (f-1)<<8 | (slot-c)<<20
    uint8_t* scratch;         // decoded streams
    uint8_t* out;             // output: block b at out + b*kBlock
    uint32_t* npend;          // per block: number of pending spans after the local pass
    uint32_t* pmap;           // per block pending-byte bitmap, 512 words (valid when npend > 0)
    SpanRec* spans;           // pending pieces, slots [span_base, span_base + n_tok + kSpanSlack) per block
    uint64_t total;           // decompressed size
    uint32_t n_blocks;
    uint32_t lo, hi;          // blocks [lo, hi) are decoded by this job
    uint32_t min_match;
    uint32_t item_base;       // first item index of this archive in the job's item space
    uint32_t pad;
    const uint32_t* deps;     // dependency lists (BlockDev::dep_off / n_deps), or nullptr: when present,
                              // every source outside a block must lie in a listed block
    // Subset decodes (both nullptr for whole-archive jobs, where item i is
    // block lo + i with the plan's offsets and block b lives at out + b*kBlock):
    const ItemDev* items;     // item i (counted from item_base) of this archive; hi - lo = item count
    const uint32_t* need;     // wanted-byte intervals of the items (see ItemDev::need_n), or nullptr
    uint32_t* slot;           // block -> output slot: block b's bytes at out + slot[b]*kBlock, its
                              // pending count at npend[slot[b]] and bitmap at pmap + slot[b]*512;
                              // the entropy stage writes the entries of the job's items
    const uint32_t* order;    // whole-archive jobs (items == nullptr, lo = 0): the entropy stage's
                              // ticket t decodes item order[t] (blocks with the most symbols first,
                              // so the stage's last wave is short); nullptr: ticket t is item t
};

constexpr uint32_t kMaxArcsPerJob = 3000;  // rANS tickets [3, 3 + n_arcs) stay below kTrace
constexpr uint32_t kTrace = 3800;        // [kTrace + 3r]: cross-block round r list size, start time lo, hi
constexpr uint32_t kTraceRounds = 64;
constexpr uint32_t kLvStripes = 8;       // level-order hand-out: striped ticket counters
constexpr uint32_t kLvTickets = 4000;    // [kLvTickets, + kLvStripes): their counts
constexpr uint32_t kListCnt = 4086;      // [kListCnt + 0/1]: entries of the two cross-block work lists
constexpr uint32_t kBarCount = 4088;     // grid barrier arrivals
constexpr uint32_t kBarGen = 4089;       // grid barrier generation
constexpr uint32_t kStatPendBytes = 4090; // [4090, 4091]: u64 bytes of the pending pieces
constexpr uint32_t kStatPending = 4093;
constexpr uint32_t kStatPolls = 4094;    // cross-block rounds
constexpr uint32_t kCounterWords = 4096;

// Job flags.  kJobIndex: parse only — the entropy stage skips the literal
// stream and the local pass writes one token record per token (SpanRec: x/y
// source, z = destination offset | match length << 16, w = command) at the
// item's span_base instead of decoding the block; a corrupt block sets
// npend[item's slot] to 1 (the caller zeroes it first).
constexpr uint32_t kJobIndex = 1;
// kJobNeed: some items want only some of their bytes (ItemDev::need_n): the
// local pass leaves the matches outside them undone (their bytes are then
// undefined) and cuts pieces only for wanted matches, so a block's sources
// outside its wanted bytes' chains are never read.
constexpr uint32_t kJobNeed = 2;
// kJobLevels: the job's archive has level bodies and the local pass sorts
// each block's pending pieces by level (JobDev::lvl_tab).
constexpr uint32_t kJobLevels = 4;

struct JobDev {
    ArcJob one;               // the archive when arcs == nullptr
    const ArcJob* arcs;       // device array of archives (batched jobs), or nullptr
    uint32_t n_arcs;
    uint32_t n_items;         // total blocks over all archives
    uint32_t* counters;       // [1] local ticket, [2] external ticket, [3 + a] rANS ticket of archive a,
                              // [kStatPending] pending spans, [kStatPolls] empty cross-block polls
    int* err;                 // first error status (0 = ok)
    int* arc_err;             // per archive: first error status of that archive (batched jobs), or nullptr
    uint64_t timeout_ns;
    uint32_t max_tok;         // shared-memory sizing of the assembly kernel
    uint32_t max_lenb;
    uint32_t flags;           // kJob* bits
    uint32_t chunk;           // work items per ticket of the entropy stage and the local pass (0 = 1)
    uint32_t wait_ns;         // cross-block round 0: how long a piece may wait for its sources before it
                              // is left to the later rounds (0xffffffff: until the deadline)
    struct alignas(8) ListEnt {
        uint32_t x, y;        // span slot, item
    };
    ListEnt* lists[2];        // cross-block work lists
    uint32_t* ready;          // fused decodes: per item, nonzero once its streams are decoded (else nullptr)
    // Level-ordered cross-block rounds (whole single-archive jobs over an
    // archive with level bodies, else nullptr / 0): the local pass writes
    // each block's pending pieces sorted by level (a piece's level is its
    // token's, at least 1) and lvl_tab[b * (n_levels + 1) + l] = the number
    // of the block's pieces of level <= l; cross-block round l takes level l.
    uint32_t* lvl_tab;
    uint32_t n_levels;        // highest level of the archive (<= kMaxLevel)
    // The level list (k_level_scan, k_level_fill): level l's pieces at
    // lvl_list[base(l) ..], base(l) = lvl_off[Lg * n_items + Lg + l - 1]
    // (Lg = n_levels); lvl_off also holds per level and item the item's offset
    // in its level ((l-1) * n_items + item) and the level totals
    // (Lg * n_items + l - 1): Lg * n_items + 2 * Lg + 1 words.
    uint32_t* lvl_off;
    ListEnt* lvl_list;
    uint32_t lvl_cap;         // entries lvl_list holds
    uint32_t lvl_min_pieces;  // automatic policy (wait_ns 0): level order only above this many pending pieces
};
constexpr uint32_t kMaxLevel = 255;

}  // namespace acx
