// Decodes of chosen blocks (aceapex_decode_range): the block-dependency
// closure of a region, the work items that decode it into output slots, and
// the gather of the region out of the slots.
//
// Paper, Random Access at Scale: a region is served by decoding the blocks it
// covers and, transitively, the earlier blocks their matches read; the rest
// of the archive is never touched.  With dependency lists in the archive the
// closure is exact (and the local pass rejects a source outside its block's
// list); without them it is every block up to the region's last.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "host.h"

using namespace acx;

void acx::block_closure(aceapex_archive* A, uint32_t b0, uint32_t b1, std::vector<uint32_t>* out) {
    out->clear();
    const Plan& P = A->plan;
    if (!P.has_deps) {
        for (uint32_t b = 0; b <= b1; b++) out->push_back(b);
        return;
    }
    if (A->seen.size() != P.n_blocks) A->seen.assign(P.n_blocks, 0);
    if (++A->epoch == 0) {  // marks wrapped: start over
        std::fill(A->seen.begin(), A->seen.end(), 0);
        A->epoch = 1;
    }
    const uint32_t ep = A->epoch;
    std::vector<uint32_t> stack;
    for (uint32_t b = b0; b <= b1; b++) {
        A->seen[b] = ep;
        stack.push_back(b);
    }
    while (!stack.empty()) {
        const uint32_t b = stack.back();
        stack.pop_back();
        out->push_back(b);
        const BlockDev& bd = P.blk[b];
        for (uint32_t k = 0; k < bd.n_deps; k++) {
            const uint32_t d = P.deps[bd.dep_off + k];
            if (A->seen[d] != ep) {
                A->seen[d] = ep;
                stack.push_back(d);
            }
        }
    }
    std::sort(out->begin(), out->end());
}

void acx::subset_plan(const Plan& P, const uint32_t* blocks, const uint32_t* slots, size_t n, SubsetPlan* S) {
    S->items.resize(n);
    S->scratch_bytes = 0;
    S->span_slots = 0;
    S->max_tok = 1;
    S->max_lenb = 1;
    for (size_t i = 0; i < n; i++) {
        const BlockDev& bd = P.blk[blocks[i]];
        ItemDev& it = S->items[i];
        it.block = blocks[i];
        it.slot = slots[i];
        it.span_base = (uint32_t)S->span_slots;
        it.pad = 0;
        it.scratch = S->scratch_bytes;
        S->scratch_bytes += (bd.s_off[3] + bd.s_raw[3] + 15) & ~15ull;
        S->span_slots += bd.n_tok + kSpanSlack;
        S->max_tok = std::max(S->max_tok, bd.n_tok);
        S->max_lenb = std::max(S->max_lenb, bd.s_raw[kLen]);
    }
    S->scratch_bytes += 64;
}

int acx::ensure_slot_table(aceapex_ctx* c, aceapex_archive* A) {
    if (A->d_slot) return ACEAPEX_OK;
    const size_t nb = std::max<size_t>(A->plan.n_blocks, 1);
    cudaError_t e = cudaMalloc(&A->d_slot, nb * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(A->d_slot, 0xff, nb * sizeof(uint32_t));
    if (e != cudaSuccess) {
        if (A->d_slot) cudaFree(A->d_slot);
        A->d_slot = nullptr;
        return cuda_fail(c, e, "slot table");
    }
    return ACEAPEX_OK;
}

extern "C" int aceapex_decode_range(aceapex_ctx* c, aceapex_archive* A, uint64_t start, uint64_t len, void* d_out,
                                    void* stream, aceapex_stats* stats) {
    if (!c || !A || (!d_out && len)) return fail(c, ACEAPEX_E_ARG, "decode_range: null argument");
    const Plan& P = A->plan;
    if (start > P.total || len > P.total - start) return fail(c, ACEAPEX_E_RANGE, "decode_range: range outside the archive");
    if (stats) memset(stats, 0, sizeof *stats);
    if (len == 0) return ACEAPEX_OK;
    cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t b0 = (uint32_t)(start / kBlock), b1 = (uint32_t)((start + len - 1) / kBlock);
    std::vector<uint32_t> blocks, slots, need;
    std::vector<uint32_t> need_off, need_n;
    uint32_t flags = 0;
    if (A->midx) {
        // byte-level closure through the match index: only the wanted bytes' chains
        TickState T;
        WalkJournal Jn;
        T.begin(P.n_blocks);
        span_walk(P, *A->midx, start, len, [](void*, uint32_t) -> const Ivs* { return nullptr; }, nullptr, &T, &Jn);
        if (Jn.bad) return fail(c, ACEAPEX_E_CORRUPT, "decode_range: the region depends on a corrupt block");
        blocks.assign(T.sched.begin(), T.sched.end());
        std::sort(blocks.begin(), blocks.end());
        std::vector<uint32_t> iv;
        for (uint32_t b : blocks) {
            need_intervals(T.need[b], P.blk[b].raw_len, &iv);
            need_off.push_back((uint32_t)need.size());
            need_n.push_back((uint32_t)iv.size());
            need.insert(need.end(), iv.begin(), iv.end());
        }
        if (!need.empty()) flags = kJobNeed;
    } else {
        block_closure(A, b0, b1, &blocks);
    }
    const size_t k = blocks.size();
    slots.resize(k);
    for (size_t i = 0; i < k; i++) slots[i] = (uint32_t)i;
    SubsetPlan S;
    subset_plan(P, blocks.data(), slots.data(), k, &S);
    for (size_t i = 0; i < need_off.size(); i++) {
        S.items[i].need_off = need_off[i];
        S.items[i].need_n = need_n[i];
    }
    int rc = ensure_slot_table(c, A);
    if (rc) return rc;
    cudaError_t e;
    if ((e = c->streams.ensure(S.scratch_bytes)) != cudaSuccess || (e = c->npend.ensure(k * 4)) != cudaSuccess ||
        (e = c->pmap.ensure(k * (kBlock / 8))) != cudaSuccess ||
        (e = c->spans.ensure(S.span_slots * sizeof(SpanRec))) != cudaSuccess ||
        (e = c->lists.ensure(2 * S.span_slots * sizeof(JobDev::ListEnt))) != cudaSuccess ||
        (e = c->slot_out.ensure(k * kBlock)) != cudaSuccess || (e = c->items.ensure(k * sizeof(ItemDev))) != cudaSuccess ||
        (e = c->need.ensure(std::max<size_t>(need.size(), 1) * sizeof(uint32_t))) != cudaSuccess)
        return cuda_fail(c, e, "decode_range: scratch");
    if ((e = cudaMemcpyAsync(c->items.p, S.items.data(), k * sizeof(ItemDev), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (!need.empty() && (e = cudaMemcpyAsync(c->need.p, need.data(), need.size() * sizeof(uint32_t),
                                               cudaMemcpyHostToDevice, st)) != cudaSuccess))
        return cuda_fail(c, e, "decode_range: work items");
    JobDev job{};
    ArcJob& J = job.one;
    J.arc = (const uint8_t*)A->d_arc;
    J.blk = A->d_blk;
    J.dtab = A->d_dtab;
    J.scratch = (uint8_t*)c->streams.p;
    J.out = (uint8_t*)c->slot_out.p;
    J.npend = (uint32_t*)c->npend.p;
    J.pmap = (uint32_t*)c->pmap.p;
    J.spans = (SpanRec*)c->spans.p;
    J.total = P.total;
    J.n_blocks = P.n_blocks;
    J.lo = 0;
    J.hi = (uint32_t)k;
    J.min_match = P.min_match;
    J.item_base = 0;
    J.deps = A->d_deps;
    J.items = (const ItemDev*)c->items.p;
    J.need = (const uint32_t*)c->need.p;
    J.slot = A->d_slot;
    job.n_arcs = 1;
    job.n_items = (uint32_t)k;
    job.counters = c->counters;
    job.err = c->d_err;
    job.timeout_ns = (uint64_t)c->params.timeout_us * 1000ull;
    job.max_tok = S.max_tok;
    job.max_lenb = S.max_lenb;
    job.lists[0] = (JobDev::ListEnt*)c->lists.p;
    job.lists[1] = job.lists[0] + S.span_slots;
    job.flags = flags;
    LaunchPlan lp;
    if ((rc = launch_plan(c, c->params, S.max_tok, S.max_lenb, &lp, flags))) return rc;
    if ((rc = enqueue_job(c, job, lp, 4, nullptr, 0, st, stats ? c->ev : nullptr))) return rc;
    const GatherReq req{(uint8_t*)d_out, start, len};
    if ((e = launch_gather(&req, nullptr, 1, len, J.out, A->d_slot, st)) != cudaSuccess)
        return cuda_fail(c, e, "gather launch");
    if (stats && (e = cudaEventRecord(c->ev[3], st)) != cudaSuccess) return cuda_fail(c, e, "event");
    rc = ctx_read_status(c, st);
    if (rc == ACEAPEX_OK && stats) {
        float a = 0, b = 0, x = 0, t = 0;
        cudaEventElapsedTime(&a, c->ev[0], c->ev[1]);
        cudaEventElapsedTime(&b, c->ev[1], c->ev[2]);
        cudaEventElapsedTime(&x, c->ev[2], c->ev[3]);
        cudaEventElapsedTime(&t, c->ev[0], c->ev[3]);
        stats->ms_ans = a;
        stats->ms_parse = b;
        stats->ms_copy = x;
        stats->ms_total = t;
        stats->blocks = k;
        stats->bytes = len;
    }
    return rc;
}
