// C ABI of the GB300 decoder (see include/aceapex.h): contexts, archive
// plans, and the orchestration of the decode kernels on a caller's stream.
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "host.h"

using namespace acx;

static constexpr uint32_t kMaxCounters = kCounterWords;

extern "C" {

const char* aceapex_status_string(int s) {
    switch (s) {
        case ACEAPEX_OK: return "ok";
        case ACEAPEX_E_ARG: return "invalid argument";
        case ACEAPEX_E_CORRUPT: return "corrupt archive";
        case ACEAPEX_E_NOMEM: return "out of memory";
        case ACEAPEX_E_CUDA: return "CUDA error";
        case ACEAPEX_E_TIMEOUT: return "device dependency wait timed out";
        case ACEAPEX_E_RANGE: return "range outside the archive";
        case ACEAPEX_E_BUSY: return "admission refused";
        default: return "unknown status";
    }
}

const char* aceapex_last_error(const aceapex_ctx* c) { return c ? c->err.c_str() : "null context"; }

int aceapex_ctx_create(int device, const aceapex_dec_params* params, aceapex_ctx** out) {
    if (!out) return ACEAPEX_E_ARG;
    *out = nullptr;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return ACEAPEX_E_CUDA;
    aceapex_ctx* c = new (std::nothrow) aceapex_ctx();
    if (!c) return ACEAPEX_E_NOMEM;
    c->device = device;
    if (params) c->params = *params;
    if (!c->params.timeout_us) c->params.timeout_us = 2000000;
    if (cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc(&c->counters, kMaxCounters * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&c->d_err, 4 * sizeof(int)) != cudaSuccess ||
        cudaMemset(c->counters, 0, kMaxCounters * sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(c->d_err, 0, 4 * sizeof(int)) != cudaSuccess) {
        aceapex_ctx_destroy(c);
        return ACEAPEX_E_CUDA;
    }
    note_sm_count(c->n_sms);
    for (auto& ev : c->ev) {
        if (cudaEventCreate(&ev) != cudaSuccess) {
            aceapex_ctx_destroy(c);
            return ACEAPEX_E_CUDA;
        }
    }
    c->occ_rans = std::max(1, rans_occupancy());
    c->occ_ext = std::max(1, external_occupancy());
    c->occ_plain = std::max(1, plain_occupancy());
    *out = c;
    return ACEAPEX_OK;
}

int aceapex_ctx_destroy(aceapex_ctx* c) {
    if (!c) return ACEAPEX_E_ARG;
    cudaSetDevice(c->device);
    c->streams.release();
    c->npend.release();
    c->pmap.release();
    c->spans.release();
    c->lists.release();
    c->arcs.release();
    c->in_arc.release();
    c->out_buf.release();
    c->slot_out.release();
    c->items.release();
    c->need.release();
    c->ready.release();
    c->lvl_tab.release();
    c->lvl_off.release();
    c->lvl_list.release();
    if (c->counters) cudaFree(c->counters);
    if (c->d_err) cudaFree(c->d_err);
    for (auto& ev : c->pipe_ev) cudaEventDestroy(ev);
    if (c->s_up) cudaStreamDestroy(c->s_up);
    if (c->s_down) cudaStreamDestroy(c->s_down);
    for (auto& ev : c->ev)
        if (ev) cudaEventDestroy(ev);
    delete c;
    return ACEAPEX_OK;
}

int aceapex_ctx_set_params(aceapex_ctx* c, const aceapex_dec_params* p) {
    if (!c || !p) return ACEAPEX_E_ARG;
    c->params = *p;
    if (!c->params.timeout_us) c->params.timeout_us = 2000000;
    return ACEAPEX_OK;
}

int aceapex_encode(const uint8_t* src, uint64_t n, const aceapex_enc_params* p, uint8_t** out, uint64_t* out_len) {
    return aceapex_encode_ex(src, n, p, out, out_len, nullptr);
}

int aceapex_encode_ex(const uint8_t* src, uint64_t n, const aceapex_enc_params* p, uint8_t** out, uint64_t* out_len,
                      aceapex_enc_stats* stats) {
    aceapex_enc_params d{};
    if (p) d = *p;
    EncDepthStats S;
    const int rc = encode_archive(src, n, d.no_rep, d.min_match, d.max_lanes, d.threads, d.latest_source, d.max_depth,
                                  d.short_latest, d.deps, d.segment, d.levels, out, out_len, stats ? &S : nullptr);
    if (rc == 0 && stats) {
        stats->blocks = S.blocks;
        stats->matches = S.matches;
        memcpy(stats->block_max_depth, S.block_max_depth, sizeof S.block_max_depth);
        memcpy(stats->match_depth, S.match_depth, sizeof S.match_depth);
        memcpy(stats->match_level, S.match_level, sizeof S.match_level);
        memcpy(stats->level_bytes, S.level_bytes, sizeof S.level_bytes);
    }
    return rc;
}

void aceapex_free(void* p) { free(p); }

int aceapex_archive_open(aceapex_ctx* c, const void* d_arc, const void* h_arc, uint64_t len, aceapex_archive** out) {
    if (!c || !out || !h_arc || !d_arc) return fail(c, ACEAPEX_E_ARG, "archive_open: null argument");
    *out = nullptr;
    cudaSetDevice(c->device);
    aceapex_archive* A = new (std::nothrow) aceapex_archive();
    if (!A) return fail(c, ACEAPEX_E_NOMEM, "archive_open: host allocation");
    std::string why;
    if (build_plan((const uint8_t*)h_arc, len, &A->plan, &why) != 0) {
        delete A;
        return fail(c, ACEAPEX_E_CORRUPT, "archive_open: " + why);
    }
    A->ctx = c;
    A->d_arc = d_arc;
    const size_t nb = A->plan.blk.size();
    cudaError_t e = cudaMalloc(&A->d_blk, std::max<size_t>(nb, 1) * sizeof(BlockDev));
    if (e == cudaSuccess) e = cudaMalloc(&A->d_dtab, 4 * kM * sizeof(uint32_t));
    if (e == cudaSuccess && nb) e = cudaMemcpy(A->d_blk, A->plan.blk.data(), nb * sizeof(BlockDev), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(A->d_dtab, A->plan.dtab.data(), 4 * kM * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && A->plan.has_deps) {
        const size_t nd = std::max<size_t>(A->plan.deps.size(), 1);
        e = cudaMalloc(&A->d_deps, nd * sizeof(uint32_t));
        if (e == cudaSuccess && !A->plan.deps.empty())
            e = cudaMemcpy(A->d_deps, A->plan.deps.data(), A->plan.deps.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && nb) {
        // entropy-stage hand-out order: most symbols first (longest-first
        // scheduling keeps the last wave of the persistent warps short)
        std::vector<uint32_t> ord(nb);
        std::vector<uint64_t> key(nb);
        for (size_t b = 0; b < nb; b++) {
            const BlockDev& bd = A->plan.blk[b];
            ord[b] = (uint32_t)b;
            key[b] = (uint64_t)bd.s_raw[0] + bd.s_raw[1] + bd.s_raw[2] + bd.s_raw[3];
        }
        std::stable_sort(ord.begin(), ord.end(), [&](uint32_t x, uint32_t y) { return key[x] > key[y]; });
        e = cudaMalloc(&A->d_order, nb * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMemcpy(A->d_order, ord.data(), nb * sizeof(uint32_t), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        aceapex_archive_close(A);
        return cuda_fail(c, e, "archive_open");
    }
    *out = A;
    return ACEAPEX_OK;
}

int aceapex_archive_close(aceapex_archive* A) {
    if (!A) return ACEAPEX_E_ARG;
    if (A->ctx) cudaSetDevice(A->ctx->device);
    if (A->d_blk) cudaFree(A->d_blk);
    if (A->d_dtab) cudaFree(A->d_dtab);
    if (A->d_deps) cudaFree(A->d_deps);
    if (A->d_order) cudaFree(A->d_order);
    if (A->d_slot) cudaFree(A->d_slot);
    delete A->midx;
    delete A;
    return ACEAPEX_OK;
}

int aceapex_archive_check(const void* h_arc, uint64_t len, aceapex_archive_info* info) {
    if (!h_arc) return ACEAPEX_E_ARG;
    Plan P;
    std::string why;
    if (build_plan((const uint8_t*)h_arc, len, &P, &why) != 0) return ACEAPEX_E_CORRUPT;
    if (info) {
        info->total_size = P.total;
        info->n_blocks = P.n_blocks;
        info->flags = P.flags;
        info->min_match = P.min_match;
        info->max_tokens = P.max_tok;
        info->archive_bytes = P.archive_bytes;
        info->tokens = P.tokens;
    }
    return ACEAPEX_OK;
}

int aceapex_shard_range(uint64_t total, int n_ranks, int rank, uint64_t* start, uint64_t* len) {
    if (n_ranks <= 0 || rank < 0 || rank >= n_ranks || !start || !len) return ACEAPEX_E_ARG;
    const uint64_t nb = (total + kBlock - 1) / kBlock;
    const uint64_t b0 = nb * (uint64_t)rank / (uint64_t)n_ranks, b1 = nb * (uint64_t)(rank + 1) / (uint64_t)n_ranks;
    const uint64_t s = std::min(total, b0 * kBlock), e = std::min(total, b1 * kBlock);
    *start = s;
    *len = e - s;
    return ACEAPEX_OK;
}

// Diagnostics (not part of the documented ABI): copy the context's device
// counter block (tickets, statistics, cross-block round trace) to host memory.
int acx_debug_counters(aceapex_ctx* c, uint32_t* out, uint32_t n) {
    if (!c || !out || n > kCounterWords) return ACEAPEX_E_ARG;
    cudaSetDevice(c->device);
    return cudaMemcpy(out, c->counters, n * sizeof(uint32_t), cudaMemcpyDeviceToHost) == cudaSuccess ? 0
                                                                                                   : ACEAPEX_E_CUDA;
}

int aceapex_archive_get_info(const aceapex_archive* A, aceapex_archive_info* info) {
    if (!A || !info) return ACEAPEX_E_ARG;
    info->total_size = A->plan.total;
    info->n_blocks = A->plan.n_blocks;
    info->flags = A->plan.flags;
    info->min_match = A->plan.min_match;
    info->max_tokens = A->plan.max_tok;
    info->archive_bytes = A->plan.archive_bytes;
    info->tokens = A->plan.tokens;
    return ACEAPEX_OK;
}

}  // extern "C"

// Enqueue the whole decode of one archive: ticket reset, entropy stage,
// local parse + match pass, cross-block pass.  With `timed`, events bracket
// the three stages.
static int enqueue_decode(aceapex_ctx* c, aceapex_archive* A, const void* d_arc, void* d_out, cudaStream_t st,
                          bool timed, uint32_t lo = 0, uint32_t hi = 0xffffffffu) {
    const Plan& P = A->plan;
    if (hi > P.n_blocks) hi = P.n_blocks;
    cudaError_t e;
    const size_t nb = std::max<size_t>(P.n_blocks, 1);
    if ((e = c->streams.ensure(P.scratch_bytes)) != cudaSuccess) return cuda_fail(c, e, "scratch allocation");
    if ((e = c->npend.ensure(nb * 4)) != cudaSuccess) return cuda_fail(c, e, "pending-count allocation");
    if ((e = c->pmap.ensure(nb * (kBlock / 8))) != cudaSuccess) return cuda_fail(c, e, "bitmap allocation");
    if ((e = c->spans.ensure(std::max<uint64_t>(P.span_slots, 1) * sizeof(SpanRec))) != cudaSuccess)
        return cuda_fail(c, e, "span allocation");
    if ((e = c->lists.ensure(2 * std::max<uint64_t>(P.span_slots, 1) * sizeof(JobDev::ListEnt))) != cudaSuccess)
        return cuda_fail(c, e, "work-list allocation");
    JobDev job{};
    ArcJob& J = job.one;
    J.arc = (const uint8_t*)d_arc;
    J.blk = A->d_blk;
    J.dtab = A->d_dtab;
    J.scratch = (uint8_t*)c->streams.p;
    J.out = (uint8_t*)d_out;
    J.npend = (uint32_t*)c->npend.p;
    J.pmap = (uint32_t*)c->pmap.p;
    J.spans = (SpanRec*)c->spans.p;
    J.total = P.total;
    J.n_blocks = P.n_blocks;
    J.lo = lo;  // blocks [lo, hi): item i is block lo + i (the whole archive, or one chunk of a pipelined decode)
    J.hi = hi;
    J.min_match = P.min_match;
    J.item_base = 0;
    J.deps = A->d_deps;
    J.order = lo == 0 && hi == P.n_blocks ? A->d_order : nullptr;
    job.arcs = nullptr;
    job.n_arcs = 1;
    job.n_items = hi - lo;
    job.counters = c->counters;
    job.err = c->d_err;
    job.timeout_ns = (uint64_t)c->params.timeout_us * 1000ull;
    job.max_tok = P.max_tok;
    job.max_lenb = P.max_lenb;
    job.lists[0] = (JobDev::ListEnt*)c->lists.p;
    job.lists[1] = (JobDev::ListEnt*)c->lists.p + std::max<uint64_t>(P.span_slots, 1);
    if (hi <= lo) return ACEAPEX_OK;
    if ((P.flags & kFlagLevels) && !c->params.ignore_levels && c->params.variant != ACEAPEX_VARIANT_PLAIN) {
        // level-ordered cross-block rounds: one row of the level table per block
        const uint32_t Lg = std::max<uint32_t>(1, std::min<uint32_t>(P.max_level, kMaxLevel));
        if ((e = c->lvl_tab.ensure(nb * (Lg + 1) * 4)) != cudaSuccess) return cuda_fail(c, e, "level-table allocation");
        if ((e = c->lvl_off.ensure((nb * Lg + 2 * Lg + 1) * 4)) != cudaSuccess)
            return cuda_fail(c, e, "level-offset allocation");
        if ((e = c->lvl_list.ensure(std::max<uint64_t>(P.span_slots, 1) * sizeof(JobDev::ListEnt))) != cudaSuccess)
            return cuda_fail(c, e, "level-list allocation");
        job.lvl_tab = (uint32_t*)c->lvl_tab.p;
        job.lvl_off = (uint32_t*)c->lvl_off.p;
        job.lvl_list = (JobDev::ListEnt*)c->lvl_list.p;
        job.lvl_cap = (uint32_t)std::max<uint64_t>(P.span_slots, 1);
        job.lvl_min_pieces = lvl_auto_min_pieces(c);
        job.n_levels = Lg;
        job.flags |= kJobLevels;
    }
    LaunchPlan lp;
    int rc = launch_plan(c, c->params, P.max_tok, P.max_lenb, &lp, job.flags, true);
    if (rc) return rc;
    if (lp.fused_groups) {
        if ((e = c->ready.ensure(nb * 4)) != cudaSuccess) return cuda_fail(c, e, "ready-flag allocation");
        job.ready = (uint32_t*)c->ready.p;
    }
    return enqueue_job(c, job, lp, 3 + 1, nullptr, 0, st, timed ? c->ev : nullptr);
}

int acx::launch_plan(aceapex_ctx* c, const aceapex_dec_params& p, uint32_t max_tok, uint32_t max_lenb,
                     LaunchPlan* lp, uint32_t job_flags, bool whole_single) {
    // parse-only and wanted-byte jobs run the scan decoder (the serial one has neither mode)
    lp->variant = (job_flags & (kJobIndex | kJobNeed)) ? (uint32_t)ACEAPEX_VARIANT_FAST : p.variant;
    if (lp->variant > ACEAPEX_VARIANT_FUSED) return fail(c, ACEAPEX_E_ARG, "unknown decoder variant");
    lp->chunk = p.queue_chunk ? p.queue_chunk : 1;
    lp->wait_ns = p.wait_ns;
    lp->grid_rans = (p.rans_ctas_per_sm ? std::min<int>(c->occ_rans, (int)p.rans_ctas_per_sm) : c->occ_rans) * c->n_sms;
    lp->grid_ext = c->occ_ext * c->n_sms;
    lp->grid_plain = c->occ_plain * c->n_sms;
    lp->grid_local = 0;
    if (lp->variant != ACEAPEX_VARIANT_PLAIN) {
        const size_t lsm =
            local_smem_bytes(max_tok, max_lenb, (job_flags & kJobNeed) != 0, (job_flags & kJobLevels) != 0);
        if (lsm > 227 * 1024) return fail(c, ACEAPEX_E_CORRUPT, "block too large for the local pass");
        if (c->occ_local_smem != lsm) {  // (an occupancy query per launch costs the serving ticks host time)
            c->occ_local = local_occupancy(lsm);
            c->occ_local_smem = lsm;
        }
        int occ = std::max(1, c->occ_local);
        if (p.ctas_per_sm) occ = std::min<int>(occ, (int)p.ctas_per_sm);
        lp->grid_local = occ * c->n_sms;
    }
    // the fused variant: entropy stage and local pass in one kernel when the
    // job is one whole archive and a CTA holds the tables and a workspace
    if (whole_single && lp->variant == ACEAPEX_VARIANT_FUSED && !(job_flags & (kJobIndex | kJobNeed))) {
        const bool lvl = (job_flags & kJobLevels) != 0;
        const int G = fused_groups(max_tok, max_lenb, lvl);
        if (G > 0 && fused_occupancy(G, max_tok, max_lenb, lvl) >= 1) {
            lp->fused_groups = G;
            lp->grid_fused = c->n_sms;
        }
    }
    return ACEAPEX_OK;
}

// The four launches of a decode job on `st`: ticket/status reset, entropy
// stage, local pass (or the plain serial pass), cross-block pass.  With
// `ev` (4 events), events bracket the three stages.
int acx::enqueue_job(aceapex_ctx* c, const JobDev& job_in, const LaunchPlan& lp, uint32_t n_counters, int* errs,
                     uint32_t n_errs, cudaStream_t st, cudaEvent_t* ev) {
    JobDev job = job_in;
    job.chunk = lp.chunk;
    job.wait_ns = lp.wait_ns;
    cudaError_t e;
    if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return cuda_fail(c, e, "event");
    if ((e = launch_prologue(job.counters, n_counters, st, errs, n_errs)) != cudaSuccess)
        return cuda_fail(c, e, "prologue launch");
    if (lp.fused_groups && job.ready) {
        // fused: one launch for the entropy stage and the local pass (the
        // stage split reports it as the local pass)
        if ((e = cudaMemsetAsync(job.ready, 0, (size_t)job.n_items * 4, st)) != cudaSuccess)
            return cuda_fail(c, e, "ready-flag reset");
        if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return cuda_fail(c, e, "event");
        if ((e = launch_fused(job, lp.fused_groups, lp.grid_fused, st)) != cudaSuccess)
            return cuda_fail(c, e, "fused launch");
    } else {
        job.ready = nullptr;
        if ((e = launch_rans(job, lp.grid_rans, st)) != cudaSuccess) return cuda_fail(c, e, "rANS launch");
        if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return cuda_fail(c, e, "event");
    }
    if (lp.fused_groups && job.ready) {
    } else if (lp.variant == ACEAPEX_VARIANT_PLAIN) {
        if ((e = launch_plain(job, lp.grid_plain, st)) != cudaSuccess) return cuda_fail(c, e, "plain launch");
    } else {
        if ((e = launch_local(job, lp.grid_local, st)) != cudaSuccess) return cuda_fail(c, e, "local launch");
    }
    if (ev && (e = cudaEventRecord(ev[2], st)) != cudaSuccess) return cuda_fail(c, e, "event");
    if ((job.flags & kJobLevels) && (e = launch_level_list(job, st)) != cudaSuccess)
        return cuda_fail(c, e, "level-list launch");
    if (!(job.flags & kJobIndex) && (e = launch_external(job, lp.grid_ext, st)) != cudaSuccess)
        return cuda_fail(c, e, "external launch");
    if (ev && (e = cudaEventRecord(ev[3], st)) != cudaSuccess) return cuda_fail(c, e, "event");
    return ACEAPEX_OK;
}

std::string acx::device_error_text(const int h[3]) {
    static const char* stages[] = {"?", "rANS stream", "varint lengths", "token sums/commands",
                                   "offsets/history", "dependency wait", "plain parse", "block limits"};
    const int st = (h[1] >> 24) & 7;
    std::string m = std::string("device reported: ") + aceapex_status_string(h[0]) + " (" + stages[st];
    if (st == 1) m += " " + std::to_string(h[1] & 0xff);
    m += ", block " + std::to_string((unsigned)h[2]) + ")";
    return m;
}

int acx::ctx_read_status(aceapex_ctx* c, cudaStream_t st) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
    int h[4] = {0, 0, 0, 0};
    if ((e = cudaMemcpy(h, c->d_err, sizeof(h), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(c, e, "error word");
    if (h[0]) {
        cudaMemset(c->d_err, 0, sizeof(h));
        return fail(c, h[0], device_error_text(h));
    }
    return ACEAPEX_OK;
}

static void fill_stats(aceapex_ctx* c, const Plan& P, aceapex_stats* s) {
    float a = 0, b = 0, x = 0, t = 0;
    cudaEventElapsedTime(&a, c->ev[0], c->ev[1]);
    cudaEventElapsedTime(&b, c->ev[1], c->ev[2]);
    cudaEventElapsedTime(&x, c->ev[2], c->ev[3]);
    cudaEventElapsedTime(&t, c->ev[0], c->ev[3]);
    s->ms_ans = a;
    s->ms_parse = b;
    s->ms_copy = x;
    s->ms_total = t;
    s->blocks = P.n_blocks;
    s->bytes = P.total;
    uint32_t st[6] = {0, 0, 0, 0, 0, 0};
    cudaMemcpy(st, c->counters + kStatPendBytes, sizeof st, cudaMemcpyDeviceToHost);
    s->pending_bytes = (uint64_t)st[0] | ((uint64_t)st[1] << 32);
    s->pending_spans = st[kStatPending - kStatPendBytes];
    s->wait_polls = st[kStatPolls - kStatPendBytes];
}

extern "C" {

int aceapex_decode_all_async(aceapex_ctx* c, aceapex_archive* A, void* d_out, uint64_t out_cap, void* stream) {
    if (!c || !A || (!d_out && A->plan.total)) return fail(c, ACEAPEX_E_ARG, "decode_all: null argument");
    if (out_cap < A->plan.total) return fail(c, ACEAPEX_E_ARG, "decode_all: output buffer too small");
    cudaSetDevice(c->device);
    return enqueue_decode(c, A, A->d_arc, d_out, (cudaStream_t)stream, false);
}

int aceapex_sync(aceapex_ctx* c, void* stream) {
    if (!c) return ACEAPEX_E_ARG;
    cudaSetDevice(c->device);
    return ctx_read_status(c, (cudaStream_t)stream);
}

int aceapex_decode_all(aceapex_ctx* c, aceapex_archive* A, void* d_out, uint64_t out_cap, void* stream,
                       aceapex_stats* stats) {
    if (!c || !A || (!d_out && A->plan.total)) return fail(c, ACEAPEX_E_ARG, "decode_all: null argument");
    if (out_cap < A->plan.total) return fail(c, ACEAPEX_E_ARG, "decode_all: output buffer too small");
    cudaSetDevice(c->device);
    int rc = enqueue_decode(c, A, A->d_arc, d_out, (cudaStream_t)stream, stats != nullptr);
    if (rc) return rc;
    rc = ctx_read_status(c, (cudaStream_t)stream);
    if (rc == ACEAPEX_OK && stats) fill_stats(c, A->plan, stats);
    return rc;
}

}  // extern "C"

// The end-to-end decode of an archive held in host memory, as a pipeline over
// chunks of blocks: the payload bytes of chunk k are uploaded on one stream,
// its decode runs on the caller's stream as soon as they have landed, and its
// output is downloaded on a third stream while chunk k + 1 decodes.  A
// chunk's cross-block sources lie in its own or earlier blocks (every source
// precedes its destination), all final when its decode runs.  The download
// is the slowest leg (the host link carries about 190 GB/s, the decode about
// 280), so the first chunk is small, to start it early, and the later ones
// large, to keep the per-launch costs of the decode low.
static uint32_t host_chunk_end(uint32_t lo, uint32_t n_blocks) {
    const uint32_t hi = lo == 0 ? 512 : lo < 2048 ? 2048 : lo + 4096;
    return std::min(hi, n_blocks);
}

static int host_pipeline(aceapex_ctx* c, aceapex_archive* A, const uint8_t* h_arc, uint64_t arc_len, uint8_t* h_out,
                         cudaStream_t st) {
    const Plan& P = A->plan;
    cudaError_t e;
    if (!c->s_up) {
        if ((e = cudaStreamCreateWithFlags(&c->s_up, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&c->s_down, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(c, e, "decode_host: streams");
    }
    uint32_t n_chunks = 0;
    for (uint32_t lo = 0; lo < P.n_blocks; lo = host_chunk_end(lo, P.n_blocks)) n_chunks++;
    while (c->pipe_ev.size() < 2 * (size_t)n_chunks + 1) {
        cudaEvent_t ev;
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(c, e, "decode_host: events");
        c->pipe_ev.push_back(ev);
    }
    cudaEvent_t* ev_up = c->pipe_ev.data();
    cudaEvent_t* ev_dec = ev_up + n_chunks;
    cudaEvent_t ev_start = ev_dec[n_chunks];
    // the upload and download streams start after what the caller queued before
    if ((e = cudaEventRecord(ev_start, st)) != cudaSuccess || (e = cudaStreamWaitEvent(c->s_up, ev_start, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(c->s_down, ev_start, 0)) != cudaSuccess)
        return cuda_fail(c, e, "decode_host: stream order");
    for (uint32_t k = 0, lo = 0; k < n_chunks; k++, lo = host_chunk_end(lo, P.n_blocks)) {
        const uint32_t hi = host_chunk_end(lo, P.n_blocks);
        // the chunk's payload bytes (whatever their order in the archive)
        uint64_t a0 = ~0ull, a1 = 0;
        for (uint32_t b = lo; b < hi; b++) {
            const BlockDev& bd = P.blk[b];
            uint64_t end = 48;
            for (int q = 0; q < 4; q++) end = std::max<uint64_t>(end, (uint64_t)bd.s_body[q] + bd.s_enc[q]);
            if (bd.lvl_body) end = std::max<uint64_t>(end, (uint64_t)bd.lvl_body + bd.n_tok);
            a0 = std::min<uint64_t>(a0, bd.payload);
            a1 = std::max<uint64_t>(a1, std::min<uint64_t>(arc_len, (bd.payload + end + 15) & ~15ull));
        }
        if (a1 > a0 && (e = cudaMemcpyAsync((uint8_t*)c->in_arc.p + a0, h_arc + a0, a1 - a0, cudaMemcpyHostToDevice,
                                            c->s_up)) != cudaSuccess)
            return cuda_fail(c, e, "decode_host: archive upload");
        if ((e = cudaEventRecord(ev_up[k], c->s_up)) != cudaSuccess || (e = cudaStreamWaitEvent(st, ev_up[k], 0)) != cudaSuccess)
            return cuda_fail(c, e, "decode_host: upload order");
        const int rc = enqueue_decode(c, A, c->in_arc.p, c->out_buf.p, st, false, lo, hi);
        if (rc) return rc;
        if ((e = cudaEventRecord(ev_dec[k], st)) != cudaSuccess || (e = cudaStreamWaitEvent(c->s_down, ev_dec[k], 0)) != cudaSuccess)
            return cuda_fail(c, e, "decode_host: decode order");
        const uint64_t o0 = (uint64_t)lo * kBlock, o1 = std::min<uint64_t>(P.total, (uint64_t)hi * kBlock);
        if ((e = cudaMemcpyAsync(h_out + o0, (uint8_t*)c->out_buf.p + o0, o1 - o0, cudaMemcpyDeviceToHost, c->s_down)) !=
            cudaSuccess)
            return cuda_fail(c, e, "decode_host: output download");
    }
    // the caller's stream ends after the last download
    if ((e = cudaEventRecord(ev_up[0], c->s_down)) != cudaSuccess || (e = cudaStreamWaitEvent(st, ev_up[0], 0)) != cudaSuccess)
        return cuda_fail(c, e, "decode_host: completion order");
    return ACEAPEX_OK;
}

extern "C" {

int aceapex_decode_host(aceapex_ctx* c, aceapex_archive* A, const void* h_arc, uint64_t arc_len, void* h_out,
                        uint64_t out_cap, void* stream, aceapex_stats* stats) {
    if (!c || !h_arc || !h_out) return fail(c, ACEAPEX_E_ARG, "decode_host: null argument");
    cudaSetDevice(c->device);
    aceapex_archive* tmp = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = c->in_arc.ensure(arc_len + 16)) != cudaSuccess) return cuda_fail(c, e, "archive buffer");
    if (!A) {
        int rc = aceapex_archive_open(c, c->in_arc.p, h_arc, arc_len, &tmp);
        if (rc) return rc;
        A = tmp;
    }
    int rc = ACEAPEX_OK;
    if (out_cap < A->plan.total) rc = fail(c, ACEAPEX_E_ARG, "decode_host: output buffer too small");
    else if ((e = c->out_buf.ensure(A->plan.total + 16)) != cudaSuccess) rc = cuda_fail(c, e, "output buffer");
    if (rc == ACEAPEX_OK && stats && (e = cudaEventRecord(c->ev[0], st)) != cudaSuccess) rc = cuda_fail(c, e, "event");
    if (rc == ACEAPEX_OK)
        rc = host_pipeline(c, A, (const uint8_t*)h_arc, arc_len, (uint8_t*)h_out, st);
    if (rc == ACEAPEX_OK && stats && (e = cudaEventRecord(c->ev[3], st)) != cudaSuccess) rc = cuda_fail(c, e, "event");
    if (rc == ACEAPEX_OK) rc = ctx_read_status(c, st);
    if (rc == ACEAPEX_OK && stats) {
        float ms = 0;
        cudaEventElapsedTime(&ms, c->ev[0], c->ev[3]);
        memset(stats, 0, sizeof *stats);
        stats->ms_total = ms;
        stats->blocks = A->plan.n_blocks;
        stats->bytes = A->plan.total;
    }
    if (tmp) aceapex_archive_close(tmp);
    return rc;
}

}  // extern "C"
