// Host-side decode plan of one archive (format v1).
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "internal.h"

namespace acx {

struct Plan {
    uint64_t total = 0, archive_bytes = 0, tokens = 0, scratch_bytes = 0, span_slots = 0;
    uint32_t n_blocks = 0, flags = 0, min_match = 0, max_tok = 0, max_lenb = 0;
    uint16_t freq[4][256];
    bool table_ok[4];
    std::vector<uint32_t> dtab;   // 4 x 4096 decode entries
    std::vector<BlockDev> blk;
    bool has_deps = false;        // the archive carries dependency lists
    std::vector<uint32_t> deps;   // all lists, block b's at [blk[b].dep_off, + blk[b].n_deps)
    // Level bodies (flags bit1: one cross-block level per token, a scheduling
    // hint): block b's at payload offset lvl_off[b]; empty without them.
    std::vector<uint32_t> lvl_off;
    uint32_t max_level = 0;       // highest level byte of the level bodies (0 without them)
};
constexpr uint32_t kFlagLevels = 2;

// Validate the archive structure and build its plan.  Returns 0 or -2
// (corrupt) with a reason in *why.
int build_plan(const uint8_t* a, uint64_t len, Plan* P, std::string* why);

// Library encoder (format v1); out is malloc'ed.
// Optional statistics: per-block maximum and per-match chain-depth histograms
// (see aceapex_enc_stats).
struct EncDepthStats {
    uint64_t blocks = 0, matches = 0;
    uint64_t block_max_depth[256] = {};
    uint64_t match_depth[256] = {};
    uint64_t match_level[256] = {};
    uint64_t level_bytes[256] = {};
};
int encode_archive(const uint8_t* src, uint64_t n, int no_rep, uint32_t min_match, uint32_t max_lanes, int threads,
                   int latest, uint32_t max_depth, int short_latest, int deps, uint64_t segment, int levels,
                   uint8_t** out, uint64_t* out_len, EncDepthStats* stats = nullptr);

// FNV-1a 64.
uint64_t fnv1a64(const uint8_t* p, uint64_t n);

}  // namespace acx
