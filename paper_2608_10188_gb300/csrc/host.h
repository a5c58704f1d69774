// Host-side state of the C ABI: device buffers, contexts, opened archives.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <utility>
#include <vector>

#include "../../include/aceapex.h"
#include "internal.h"
#include "launch.h"
#include "plan.h"

namespace acx {

// A device allocation that only grows (by at least a quarter each time, so a
// sequence of slightly larger requests does not reallocate every call).
struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t n) {
        if (n <= cap) return cudaSuccess;
        const size_t want = std::max(n, cap + cap / 4);
        release();
        cudaError_t e = cudaMalloc(&p, want);
        if (e == cudaSuccess) {
            cap = want;
            return e;
        }
        e = cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        cap = n;
        return cudaSuccess;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

// Sorted, disjoint byte intervals [first, second) of one block.
typedef std::vector<std::pair<uint32_t, uint32_t>> Ivs;

// Every match of an archive, block by block (from a parse-only pass over the
// archive): match k of block b, for k in [first[b], first[b+1]), writes
// [o[k], o[k] + ml[k]) of its block from the absolute source src[k].
struct MatchIndex {
    std::vector<uint64_t> first;
    std::vector<uint16_t> o, ml;
    std::vector<uint64_t> src;
    std::vector<uint8_t> bad;  // per block: 1 if the parse found it corrupt (it then lists no matches)
    aceapex_parse_stats stats{};  // counted from the same pass's token records
};

}  // namespace acx

struct aceapex_ctx {
    int device = 0;
    aceapex_dec_params params{};
    std::string err;
    int n_sms = 0;
    acx::DevBuf streams, npend, pmap, spans, lists, arcs, in_arc, out_buf;
    acx::DevBuf slot_out, items, need;   // range decodes: decoded closure blocks, work items, wanted bytes
    acx::DevBuf ready;                   // fused decodes: per block, its streams are decoded
    acx::DevBuf lvl_tab, lvl_off, lvl_list;  // level-ordered decodes: per block level counts, the level list
    uint32_t* counters = nullptr;  // device
    int* d_err = nullptr;          // device
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaStream_t s_up = nullptr, s_down = nullptr;  // decode_host: upload and download streams
    std::vector<cudaEvent_t> pipe_ev;              // decode_host: per chunk, uploaded and decoded
    int occ_rans = 0, occ_ext = 0, occ_plain = 0;
    size_t occ_local_smem = 0;  // the local pass's CTAs per SM for its last workspace size
    int occ_local = 0;
};

struct aceapex_archive {
    aceapex_ctx* ctx = nullptr;
    const void* d_arc = nullptr;
    acx::Plan plan;
    acx::BlockDev* d_blk = nullptr;
    uint32_t* d_dtab = nullptr;
    uint32_t* d_deps = nullptr;    // dependency lists (archives that carry them)
    uint32_t* d_order = nullptr;   // blocks by decreasing symbol count (entropy-stage hand-out order)
    uint32_t* d_slot = nullptr;    // block -> output slot of subset decodes (allocated on first use)
    acx::MatchIndex* midx = nullptr;  // match index (aceapex_archive_index), or nullptr
    std::vector<uint32_t> seen;    // closure walk marks (epoch per block)
    uint32_t epoch = 0;
};

namespace acx {

inline int fail(aceapex_ctx* c, int code, const std::string& m) {
    if (c) c->err = m;
    return code;
}
inline int cuda_fail(aceapex_ctx* c, cudaError_t e, const char* where) {
    return fail(c, ACEAPEX_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Text of a device-reported error (err[0..2] as the kernels write it).
std::string device_error_text(const int h[3]);

// Grid sizes and variant of one decode job.
struct LaunchPlan {
    uint32_t variant = 0, chunk = 1, wait_ns = 0;
    int grid_rans = 0, grid_local = 0, grid_plain = 0, grid_ext = 0;
    int fused_groups = 0, grid_fused = 0;  // fused entropy + local pass (whole single-archive jobs), 0: staged
};
// Grids for a job whose largest block has max_tok tokens and max_lenb length
// bytes, under decoder parameters p (fails when a block cannot fit the local
// pass's shared memory).  whole_single: the job decodes one whole archive,
// which the default variant may do with the fused entropy + local kernel.
int launch_plan(aceapex_ctx* c, const aceapex_dec_params& p, uint32_t max_tok, uint32_t max_lenb, LaunchPlan* lp,
                uint32_t job_flags = 0, bool whole_single = false);
inline uint32_t lvl_auto_min_pieces(const aceapex_ctx* c) { return lvl_auto_min_pieces_for(c->occ_ext * c->n_sms); }
// Synchronise st and return (and clear) the context's device error status.
int ctx_read_status(aceapex_ctx* c, cudaStream_t st);

// Block-dependency closure of blocks [b0, b1] of an opened archive, sorted:
// with dependency lists the blocks reachable through them, without lists
// every block up to b1 (sources always precede their destinations).
void block_closure(aceapex_archive* A, uint32_t b0, uint32_t b1, std::vector<uint32_t>* out);

// Work items of a job that decodes `blocks` (ascending) of plan P into the
// output slots `slots`: per item its piece base and stream offset, and the
// job's scratch sizes.
struct SubsetPlan {
    std::vector<ItemDev> items;
    uint64_t scratch_bytes = 0, span_slots = 0;
    uint32_t max_tok = 1, max_lenb = 1;
};
void subset_plan(const Plan& P, const uint32_t* blocks, const uint32_t* slots, size_t n, SubsetPlan* S);

// Build the archive's match index with a parse-only pass on the device.
int build_match_index(aceapex_ctx* c, aceapex_archive* A);

// The span-refined dependency closure of byte ranges (paper, Random Access at
// Scale; its byte-level view of dependencies): a wanted byte range of a block
// needs the matches that write it, each match needs its whole source window,
// and so on back to literals.  `valid(b)` gives the bytes of block b already
// decoded and kept (nullptr: none); a range inside them needs nothing.  The
// walk adds to a tick's state (blocks to decode with their wanted intervals,
// matches taken, blocks read) and journals its changes so that they can be
// undone when the request is not admitted.
struct TickState {
    // Per block and per match, marks stamped with the tick's epoch (no
    // clearing between ticks), and the tick's lists.
    uint32_t epoch = 0, req = 0;
    std::vector<uint32_t> sched_mark, used_mark, touch_req;  // per block
    std::vector<Ivs> need;                                    // per block: wanted intervals (when scheduled)
    std::vector<uint32_t> sched;                              // blocks to decode, in scheduling order
    std::vector<uint32_t> used;                               // every block read (decoded or kept)
    struct R {
        uint32_t b, s, e;
    };
    std::vector<R> stack;
    Ivs parts;
    // Start a tick over an archive of n_blocks blocks.
    void begin(uint32_t n_blocks);
    bool scheduled(uint32_t b) const { return sched_mark[b] == epoch; }
};
struct WalkJournal {
    std::vector<std::pair<uint32_t, Ivs>> saved;  // need of a block scheduled by an earlier request, before this one
    size_t sched0 = 0, used0 = 0;                 // list lengths before the request
    bool bad = false;                             // the region depends on a block the parse found corrupt
};
typedef const Ivs* (*ValidFn)(void* self, uint32_t block);
// Walk one request's region; returns nothing, the tick state grows.  The
// blocks the request scheduled are T->sched[J->sched0 ..], the blocks it read
// first are T->used[J->used0 ..].
void span_walk(const Plan& P, const MatchIndex& M, uint64_t start, uint64_t len, ValidFn valid, void* self,
               TickState* T, WalkJournal* J);
void span_undo(TickState* T, const WalkJournal& J);
// v |= [s, e) for a sorted disjoint interval list.
void iv_union(Ivs& v, uint32_t s, uint32_t e);
// The interval list of a block to decode, or empty when it covers the block.
void need_intervals(const Ivs& need, uint32_t raw_len, std::vector<uint32_t>* out);

// Make sure the archive's device slot table exists (all kNoSlot at first).
int ensure_slot_table(aceapex_ctx* c, aceapex_archive* A);

// Enqueue the decode launches of `job` on st (see api.cpp).
int enqueue_job(aceapex_ctx* c, const JobDev& job, const LaunchPlan& lp, uint32_t n_counters, int* errs,
                uint32_t n_errs, cudaStream_t st, cudaEvent_t* ev);

}  // namespace acx
